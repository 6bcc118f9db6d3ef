// Ahead-of-time kernels (compiled for sm_103a with the library).
//
// The unfused evaluator: Bandicoot's own evaluation strategy, kept as the
// comparison baseline for the fused kernels.  In the paper each node of an
// expression is evaluated by its apply() function, which launches at least
// one GPU kernel and writes its result to a temporary (Section 7); scalar
// forms such as "k * A" are one node (eop_scalar_times), and the last node
// writes straight into the destination with the type conversion fused into
// that kernel ("two-way" kernels, Section 7).  coot_unfused_eval does
// exactly that: one launch per operator node, temporaries in HBM in the
// compute type.  Each kernel is a grid-stride loop with 128-bit accesses
// when every operand allows them, so the baseline is a fair one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "coot_internal.h"

namespace {

enum UOp { U_NEG = COOT_OP_NEG, U_ABS, U_EXP, U_LOG, U_SQRT, U_SQUARE, U_COPY = 100 };

struct Operand {
  const void* ptr;  // nullptr: the scalar `k`
  int64_t ld;
  int dtype;
  double k;
};

template <typename R>
__device__ __forceinline__ R load_as(const Operand& o, int64_t i, int64_t j) {
  if (o.ptr == nullptr) return (R)o.k;
  const int64_t idx = i + j * o.ld;
  switch (o.dtype) {
    case COOT_F32: return (R)((const float*)o.ptr)[idx];
    case COOT_F64: return (R)((const double*)o.ptr)[idx];
    case COOT_BF16: {
      const unsigned short h = ((const unsigned short*)o.ptr)[idx];
      return (R)__uint_as_float(((unsigned)h) << 16);
    }
    case COOT_I32: return (R)((const int*)o.ptr)[idx];
    case COOT_U32: return (R)((const unsigned*)o.ptr)[idx];
    default: {
      const unsigned short h = ((const unsigned short*)o.ptr)[idx];
      float f;
      asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
      return (R)f;
    }
  }
}

// integer storage: rounded toward zero, saturated, NaN -> 0
__device__ __forceinline__ int to_s32(float v) {
  int r;
  asm("cvt.rzi.s32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ int to_s32(double v) {
  int r;
  asm("cvt.rzi.s32.f64 %0, %1;" : "=r"(r) : "d"(v));
  return r;
}
__device__ __forceinline__ unsigned to_u32(float v) {
  unsigned r;
  asm("cvt.rzi.u32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ unsigned to_u32(double v) {
  unsigned r;
  asm("cvt.rzi.u32.f64 %0, %1;" : "=r"(r) : "d"(v));
  return r;
}

template <typename R>
__device__ __forceinline__ void store_as(void* ptr, int dtype, int64_t idx, R v) {
  switch (dtype) {
    case COOT_F32: ((float*)ptr)[idx] = (float)v; break;
    case COOT_F64: ((double*)ptr)[idx] = (double)v; break;
    case COOT_BF16: {
      unsigned short h;
      const float f = (float)v;
      asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
      ((unsigned short*)ptr)[idx] = h;
      break;
    }
    case COOT_I32:
      ((int*)ptr)[idx] = v != v ? 0 : to_s32(v);
      break;
    case COOT_U32:
      ((unsigned*)ptr)[idx] = v != v ? 0u : to_u32(v);
      break;
    default: {
      unsigned short h;
      const float f = (float)v;
      asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
      ((unsigned short*)ptr)[idx] = h;
    }
  }
}

template <typename R>
__device__ __forceinline__ R apply_unary(int op, R a) {
  switch (op) {
    case U_NEG: return -a;
    case U_ABS: return fabs(a);
    case U_EXP: return exp(a);
    case U_LOG: return log(a);
    case U_SQRT: return sqrt(a);
    case U_SQUARE: return a * a;
    case COOT_OP_LOG10: return log10(a);
    case COOT_OP_SIN: return sin(a);
    case COOT_OP_COS: return cos(a);
    case COOT_OP_TAN: return tan(a);
    case COOT_OP_ASIN: return asin(a);
    case COOT_OP_ACOS: return acos(a);
    case COOT_OP_ATAN: return atan(a);
    default: return a;
  }
}

template <typename R>
__device__ __forceinline__ R apply_binary(int op, R a, R b) {
  switch (op) {
    case COOT_OP_ADD: return a + b;
    case COOT_OP_SUB: return a - b;
    case COOT_OP_MUL: return a * b;
    case COOT_OP_DIV: return a / b;
    case COOT_OP_LT: return a < b ? (R)1 : (R)0;
    case COOT_OP_LE: return a <= b ? (R)1 : (R)0;
    case COOT_OP_GT: return a > b ? (R)1 : (R)0;
    case COOT_OP_GE: return a >= b ? (R)1 : (R)0;
    case COOT_OP_EQ: return a == b ? (R)1 : (R)0;
    case COOT_OP_NE: return a != b ? (R)1 : (R)0;
    default: return pow(a, b);
  }
}

template <>
__device__ __forceinline__ float apply_binary<float>(int op, float a, float b) {
  switch (op) {
    case COOT_OP_ADD: return a + b;
    case COOT_OP_SUB: return a - b;
    case COOT_OP_MUL: return a * b;
    case COOT_OP_DIV: return a / b;
    case COOT_OP_LT: return a < b ? 1.0f : 0.0f;
    case COOT_OP_LE: return a <= b ? 1.0f : 0.0f;
    case COOT_OP_GT: return a > b ? 1.0f : 0.0f;
    case COOT_OP_GE: return a >= b ? 1.0f : 0.0f;
    case COOT_OP_EQ: return a == b ? 1.0f : 0.0f;
    case COOT_OP_NE: return a != b ? 1.0f : 0.0f;
    default: return powf(a, b);
  }
}

// float specialisations use the single-precision functions
template <>
__device__ __forceinline__ float apply_unary<float>(int op, float a) {
  switch (op) {
    case U_NEG: return -a;
    case U_ABS: return fabsf(a);
    case U_EXP: return expf(a);
    case U_LOG: return logf(a);
    case U_SQRT: return sqrtf(a);
    case U_SQUARE: return a * a;
    case COOT_OP_LOG10: return log10f(a);
    case COOT_OP_SIN: return sinf(a);
    case COOT_OP_COS: return cosf(a);
    case COOT_OP_TAN: return tanf(a);
    case COOT_OP_ASIN: return asinf(a);
    case COOT_OP_ACOS: return acosf(a);
    case COOT_OP_ATAN: return atanf(a);
    default: return a;
  }
}

// One node: dst = op(a) or op(a, b) over an n_rows x n_cols operand set.
// nb = 1 for unary nodes.  `dense4` selects the 128-bit path (every operand
// FP32, dense and 16-byte aligned, or a scalar).
template <typename R>
__global__ void __launch_bounds__(256) node_kernel(int op, int nb, Operand a, Operand b, void* dst, int dst_dtype,
                                                   int64_t dst_ld, int64_t n_rows, int64_t n_cols, int dense4) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (dense4) {
    const int64_t n = n_rows * n_cols;
    const int64_t n4 = n / 4;
    for (int64_t q = tid; q < n4; q += stride) {
      float4 x = a.ptr ? ((const float4*)a.ptr)[q] : make_float4((float)a.k, (float)a.k, (float)a.k, (float)a.k);
      float4 r;
      if (nb == 1) {
        r.x = apply_unary<R>(op, (R)x.x);
        r.y = apply_unary<R>(op, (R)x.y);
        r.z = apply_unary<R>(op, (R)x.z);
        r.w = apply_unary<R>(op, (R)x.w);
      } else {
        float4 y = b.ptr ? ((const float4*)b.ptr)[q] : make_float4((float)b.k, (float)b.k, (float)b.k, (float)b.k);
        r.x = apply_binary<R>(op, (R)x.x, (R)y.x);
        r.y = apply_binary<R>(op, (R)x.y, (R)y.y);
        r.z = apply_binary<R>(op, (R)x.z, (R)y.z);
        r.w = apply_binary<R>(op, (R)x.w, (R)y.w);
      }
      ((float4*)dst)[q] = r;
    }
    for (int64_t e = n4 * 4 + tid; e < n; e += stride) {
      const R x = load_as<R>(a, e, 0);
      const R r = nb == 1 ? apply_unary<R>(op, x) : apply_binary<R>(op, x, load_as<R>(b, e, 0));
      store_as<R>(dst, dst_dtype, e, r);
    }
    return;
  }
  const int64_t n = n_rows * n_cols;
  for (int64_t e = tid; e < n; e += stride) {
    const int64_t j = e / n_rows, i = e - j * n_rows;
    const R x = load_as<R>(a, i, j);
    const R r = nb == 1 ? apply_unary<R>(op, x) : apply_binary<R>(op, x, load_as<R>(b, i, j));
    store_as<R>(dst, dst_dtype, i + j * dst_ld, r);
  }
}

int dsize(int dt) { return dt == COOT_F64 ? 8 : (dt == COOT_F32 || dt == COOT_I32 || dt == COOT_U32 ? 4 : 2); }

// 1.0 in device memory: the source of device-to-device copies that write a
// constant result (all() of an empty object) in stream order, also under
// graph capture.
__device__ const double g_one = 1.0;

// Status word of the kernels' bounded waits (0, or the coot_status of a
// wait that gave up).
__device__ unsigned g_status = 0;

}  // namespace

namespace coot {

// Device address of a 1.0 (looked up once per device).
coot_status device_one(const double** out) {
  static std::mutex mu;
  static const double* addr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return fail(COOT_ERR_CUDA, "no current device");
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_one);
    if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    addr[dev] = static_cast<const double*>(p);
  }
  *out = addr[dev];
  return COOT_OK;
}

coot_status device_status_word(unsigned** out) {
  static std::mutex mu;
  static unsigned* addr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return fail(COOT_ERR_CUDA, "no current device");
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_status);
    if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    addr[dev] = static_cast<unsigned*>(p);
  }
  *out = addr[dev];
  return COOT_OK;
}

}  // namespace coot

extern "C" coot_status coot_device_status(int* status) {
  coot::clear_error();
  if (status == nullptr) return coot::fail(COOT_ERR_INVALID_ARG, "status is NULL");
  unsigned* word = nullptr;
  coot_status s = coot::device_status_word(&word);
  if (s != COOT_OK) return s;
  unsigned v = 0;
  cudaError_t e = cudaMemcpy(&v, word, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    const unsigned zero = 0;
    e = cudaMemcpy(word, &zero, sizeof zero, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return coot::fail(COOT_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  *status = (int)v;
  return COOT_OK;
}

extern "C" coot_status coot_host_device_pointer(const void* host, void** device) {
  coot::clear_error();
  if (host == nullptr || device == nullptr) return coot::fail(COOT_ERR_INVALID_ARG, "pointer is NULL");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, host);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return coot::fail(COOT_ERR_INVALID_ARG, std::string("not CUDA host memory: ") + cudaGetErrorString(e));
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr)
    return coot::fail(COOT_ERR_INVALID_ARG, "not pinned host memory mapped for the device");
  *device = a.devicePointer;
  return COOT_OK;
}

extern "C" {

/* Number of temporaries coot_unfused_eval needs for a tree (one per operator
 * node except the root); each holds n_rows * n_cols values of the compute
 * type. */
coot_status coot_unfused_tmp_count(const uint8_t* tree, size_t len, int* n_tmp) {
  coot::clear_error();
  coot::Tree t;
  coot_status s = coot::parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  if (!n_tmp) return coot::fail(COOT_ERR_INVALID_ARG, "n_tmp is NULL");
  int k = 0;
  for (size_t i = 0; i + 1 < t.nodes.size(); ++i)
    if (t.nodes[i].op != COOT_OP_INPUT && t.nodes[i].op != COOT_OP_CONST) ++k;
  *n_tmp = k;
  return COOT_OK;
}

coot_status coot_unfused_eval(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, const coot_mat* out,
                              void* tmp, size_t tmp_bytes, void* stream) {
  coot::clear_error();
  coot::Tree t;
  coot_status s = coot::parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  if (coot::canonical_enabled()) {
    coot::Tree c;
    coot::canonicalize(t, nullptr, &c, nullptr, true);
    t = std::move(c);
  }
  if (!in || !out || n_in != t.n_inputs) return coot::fail(COOT_ERR_INVALID_ARG, "bad operands");
  const int64_t R = in[0].n_rows, C = in[0].n_cols;
  for (int i = 0; i < n_in; ++i)
    if (in[i].n_rows != R || in[i].n_cols != C) return coot::fail(COOT_ERR_SHAPE, "operands need equal sizes");
  if (out->n_rows != R || out->n_cols != C) return coot::fail(COOT_ERR_SHAPE, "output shape differs");
  if (R * C == 0) return COOT_OK;
  const int rdt = t.compute;  // temporaries in the compute type
  const size_t tmp_elems = (size_t)R * (size_t)C;
  int n_tmp = 0;
  coot_unfused_tmp_count(tree, len, &n_tmp);
  if ((size_t)n_tmp * tmp_elems * dsize(rdt) > tmp_bytes || (n_tmp > 0 && tmp == nullptr))
    return coot::fail(COOT_ERR_WORKSPACE, "temporaries too small");
  // where each node's value lives
  std::vector<Operand> val(t.nodes.size());
  int next_tmp = 0;
  bool all_dense = true;
  for (int i = 0; i < n_in; ++i) all_dense = all_dense && (in[i].ld == R || C == 1);
  all_dense = all_dense && (out->ld == R || C == 1);
  const coot::Device& d = coot::device();
  const int grid = std::max(1, d.sm_count) * 8;
  for (size_t k = 0; k < t.nodes.size(); ++k) {
    const coot::Node& nd = t.nodes[k];
    if (nd.op == COOT_OP_INPUT) {
      val[k] = Operand{in[nd.a].ptr, in[nd.a].ld, in[nd.a].dtype, 0.0};
      continue;
    }
    if (nd.op == COOT_OP_CONST) {
      val[k] = Operand{nullptr, 1, rdt, rdt == COOT_F32 ? (double)(float)nd.imm : nd.imm};
      continue;
    }
    const bool root = k + 1 == t.nodes.size();
    void* dst;
    int dst_dtype;
    int64_t dst_ld;
    if (root) {
      dst = out->ptr;
      dst_dtype = out->dtype;
      dst_ld = out->ld;
    } else {
      dst = (char*)tmp + (size_t)next_tmp++ * tmp_elems * dsize(rdt);
      dst_dtype = rdt;
      dst_ld = R;
    }
    const bool unary = (nd.op >= COOT_OP_NEG && nd.op <= COOT_OP_SQUARE) ||
                       (nd.op >= COOT_OP_LOG10 && nd.op <= COOT_OP_ATAN);
    Operand a = val[nd.a];
    Operand b = unary ? Operand{nullptr, 1, rdt, 0.0} : val[nd.b];
    auto ok4 = [&](const Operand& o) {
      return o.ptr == nullptr || (o.dtype == COOT_F32 && ((uintptr_t)o.ptr % 16) == 0);
    };
    const int dense4 = all_dense && rdt == COOT_F32 && ok4(a) && ok4(b) && dst_dtype == COOT_F32 &&
                       ((uintptr_t)dst % 16) == 0;
    if (rdt == COOT_F32) {
      node_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>(nd.op, unary ? 1 : 2, a, b, dst, dst_dtype, dst_ld,
                                                                  R, C, dense4);
    } else {
      node_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(nd.op, unary ? 1 : 2, a, b, dst, dst_dtype, dst_ld,
                                                                   R, C, 0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return coot::fail(COOT_ERR_CUDA, std::string("unfused launch: ") + cudaGetErrorString(e));
    val[k] = Operand{dst, dst_ld, dst_dtype, 0.0};
  }
  const coot::Node& last = t.nodes.back();
  if (last.op == COOT_OP_INPUT || last.op == COOT_OP_CONST) {
    // the tree is a leaf: one copy (or fill) kernel into the destination
    Operand a = val.back();
    node_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(U_COPY, 1, a, a, out->ptr, out->dtype, out->ld, R, C,
                                                                 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return coot::fail(COOT_ERR_CUDA, std::string("unfused launch: ") + cudaGetErrorString(e));
  }
  return COOT_OK;
}

}  // extern "C"
