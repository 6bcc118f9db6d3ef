// Row sums with library-owned scratch: an entry point that allocates
// nothing.
//
// Some callers cannot allocate device memory at the point where they need a
// reduction.  Examples: code that runs while memory is reserved up front by
// an allocator the caller does not control, code on a path that must not
// synchronise the device (cudaMalloc and cudaFree can), and plain C callers
// with no CUDA allocator of their own.  coot_sum_dim asks such callers for a
// workspace they would have to allocate.  coot_sum_rows_f32_static instead
// keeps its scratch in one fixed array that lives inside this library's
// device image.  Every GPU that loads the library holds the array until the
// process exits.  The caller passes only the input and the output.
//
// The scratch holds one arrival counter per panel of rows and the FP64
// partial row sums of every column chunk.  Its size fixes the largest row
// count the entry point accepts (COOT_STATIC_MAX_ROWS in coot.h).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "coot_internal.h"

namespace {

constexpr int kBlock = 64;                 // threads per block
constexpr int kVec = 4;                    // rows per thread
constexpr int kPanel = kBlock * kVec;      // rows per panel
constexpr int kChunks = 16;                // column chunks (partials per row)
constexpr size_t kCounterBytes = 16384;    // one 32-bit counter per panel
constexpr size_t kPartialBytes = (size_t)kChunks * COOT_STATIC_MAX_ROWS * sizeof(double);
constexpr size_t kScratchBytes = kCounterBytes + kPartialBytes;
static_assert(COOT_STATIC_MAX_ROWS / kPanel * 4 <= (int)kCounterBytes, "counter area too small");

// The scratch array.  Host code must not use its name as an address: the
// host-side symbol is only a handle.  The device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

__device__ __forceinline__ void two_sum(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

__device__ __forceinline__ double pair(float s, float c) {
  const double sd = (double)s;
  return isfinite(sd) ? sd + (double)c : sd;
}

// Unit u = (chunk, panel): the rows of one panel over one chunk of columns.
// Each thread sums kVec rows in FP32 with TwoSum; with more than one chunk
// the partials go to the scratch and the last block of a panel to arrive
// adds them in chunk order, so the result does not depend on timing.
template <bool kVector>
__global__ void __launch_bounds__(kBlock) rowsum_static_kernel(const float* __restrict__ a, int64_t ld,
                                                               int64_t n_rows, int64_t n_cols, int64_t chunks,
                                                               float* __restrict__ out, unsigned char* scratch) {
  __shared__ int is_last;
  unsigned* counters = reinterpret_cast<unsigned*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + kCounterBytes);
  const int64_t n_panels = (n_rows + kPanel - 1) / kPanel;
  const int64_t per_chunk = (n_cols + chunks - 1) / chunks;
  for (int64_t u = blockIdx.x; u < n_panels * chunks; u += gridDim.x) {
    const int64_t chunk = u / n_panels;
    const int64_t panel = u - chunk * n_panels;
    const int64_t i0 = panel * kPanel + (int64_t)threadIdx.x * kVec;
    const int64_t jb = chunk * per_chunk;
    const int64_t je = jb + per_chunk < n_cols ? jb + per_chunk : n_cols;
    float s[kVec], c[kVec];
#pragma unroll
    for (int v = 0; v < kVec; ++v) s[v] = c[v] = 0.f;
    if (kVector && i0 + kVec <= n_rows) {
#pragma unroll 4
      for (int64_t j = jb; j < je; ++j) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(a + j * ld + i0));
        two_sum(s[0], c[0], x.x);
        two_sum(s[1], c[1], x.y);
        two_sum(s[2], c[2], x.z);
        two_sum(s[3], c[3], x.w);
      }
    } else {
      for (int64_t j = jb; j < je; ++j)
#pragma unroll
        for (int v = 0; v < kVec; ++v)
          if (i0 + v < n_rows) two_sum(s[v], c[v], __ldg(a + j * ld + i0 + v));
    }
    if (chunks == 1) {
#pragma unroll
      for (int v = 0; v < kVec; ++v)
        if (i0 + v < n_rows) out[i0 + v] = (float)pair(s[v], c[v]);
      continue;
    }
#pragma unroll
    for (int v = 0; v < kVec; ++v)
      if (i0 + v < n_rows) partials[chunk * n_rows + i0 + v] = pair(s[v], c[v]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(counters + panel, 1u) == (unsigned)(chunks - 1);
    __syncthreads();
    if (is_last) {
      __threadfence();
#pragma unroll
      for (int v = 0; v < kVec; ++v) {
        if (i0 + v < n_rows) {
          double t = 0.0;
          for (int64_t q = 0; q < chunks; ++q) t += __ldcg(partials + q * n_rows + i0 + v);
          out[i0 + v] = (float)t;
        }
      }
      if (threadIdx.x == 0) counters[panel] = 0u;  // ready for the next call
    }
    __syncthreads();
  }
}

// Device address of the scratch, looked up once per device.
std::mutex g_mu;
void* g_addr[64] = {};
int g_sms[64] = {};

}  // namespace

extern "C" coot_status coot_sum_rows_f32_static(const coot_mat* a, const coot_mat* out, void* stream) {
  coot::clear_error();
  if (a == nullptr || out == nullptr) return coot::fail(COOT_ERR_INVALID_ARG, "a and out must not be NULL");
  if (a->dtype != COOT_F32 || out->dtype != COOT_F32)
    return coot::fail(COOT_ERR_DTYPE, "coot_sum_rows_f32_static reads and writes FP32 only");
  if (a->n_rows < 0 || a->n_cols < 0 || a->ld < (a->n_rows > 1 ? a->n_rows : 1) || a->reserved || out->reserved)
    return coot::fail(COOT_ERR_INVALID_ARG, "bad input matrix");
  if (out->n_rows != a->n_rows || out->n_cols != 1) return coot::fail(COOT_ERR_SHAPE, "out must be n_rows x 1");
  if (a->n_rows > COOT_STATIC_MAX_ROWS)
    return coot::fail(COOT_ERR_UNSUPPORTED, "n_rows " + std::to_string(a->n_rows) +
                                                " exceeds the static scratch limit of " +
                                                std::to_string(COOT_STATIC_MAX_ROWS) + " rows");
  if (a->n_rows == 0) return COOT_OK;
  if ((a->ptr == nullptr && a->n_cols > 0) || out->ptr == nullptr)
    return coot::fail(COOT_ERR_INVALID_ARG, "NULL data pointer");
  if (out->ld < 1) return coot::fail(COOT_ERR_INVALID_ARG, "bad output matrix");
  // blocks write their rows of out while others may still read a's columns
  if (coot::mats_overlap(*out, *a)) return coot::fail(COOT_ERR_ALIAS, "out overlaps a");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return coot::fail(COOT_ERR_CUDA, "no current CUDA device");
  void* scratch = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev] == nullptr) {
      // first call on this device: find the array's device address
      e = cudaGetSymbolAddress(&g_addr[dev], g_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return coot::fail(COOT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      if (cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g_sms[dev] = 132;
    }
    scratch = g_addr[dev];
    sms = g_sms[dev];
  }
  const int64_t chunks = a->n_cols < kChunks ? (a->n_cols > 0 ? a->n_cols : 1) : kChunks;
  const int64_t n_panels = (a->n_rows + kPanel - 1) / kPanel;
  if (chunks > 1) {
    // the counters must start at zero; the array keeps whatever the last
    // call left, so clear them on the caller's stream first
    e = cudaMemsetAsync(scratch, 0, (size_t)n_panels * sizeof(unsigned), (cudaStream_t)stream);
    if (e != cudaSuccess) return coot::fail(COOT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  int64_t grid = n_panels * chunks;
  if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
  const bool vec = ((uintptr_t)a->ptr % 16 == 0) && (a->ld % 4 == 0 || a->n_cols <= 1);
  const float* ap = static_cast<const float*>(a->ptr);
  float* op = static_cast<float*>(out->ptr);
  unsigned char* sp = static_cast<unsigned char*>(scratch);
  if (vec) {
    rowsum_static_kernel<true><<<(unsigned)grid, kBlock, 0, (cudaStream_t)stream>>>(ap, a->ld, a->n_rows, a->n_cols,
                                                                                     chunks, op, sp);
  } else {
    rowsum_static_kernel<false><<<(unsigned)grid, kBlock, 0, (cudaStream_t)stream>>>(ap, a->ld, a->n_rows, a->n_cols,
                                                                                      chunks, op, sp);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return coot::fail(COOT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return COOT_OK;
}
