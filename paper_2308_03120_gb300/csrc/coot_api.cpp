// The C ABI (coot.h): argument checks, launch-shape selection and kernel
// launches.  Everything that runs per element runs in the generated
// kernels; this file only decides which kernel and which grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "coot_internal.h"

namespace coot {

static thread_local std::string g_err;

coot_status fail(coot_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
void clear_error() { g_err.clear(); }

coot_status init_device(int dev, unsigned flags);               // coot_jit.cpp
coot_status compile_only(const std::string& source, const std::string& arch, size_t* bytes);

static int dtype_size(int dt) {
  switch (dt) {
    case COOT_F32: return 4;
    case COOT_BF16: return 2;
    case COOT_F16: return 2;
    case COOT_F64: return 8;
    case COOT_I32: return 4;
    case COOT_U32: return 4;
  }
  return 0;
}

static bool is_float(int dt) { return dt == COOT_F32 || dt == COOT_BF16 || dt == COOT_F16 || dt == COOT_F64; }

static coot_status check_mat(const coot_mat* m, const char* what) {
  if (m == nullptr) return fail(COOT_ERR_INVALID_ARG, std::string(what) + " is NULL");
  if (dtype_size(m->dtype) == 0) return fail(COOT_ERR_DTYPE, std::string(what) + ": unknown dtype");
  if (m->reserved != 0) return fail(COOT_ERR_INVALID_ARG, std::string(what) + ": reserved field is not 0");
  if (m->n_rows < 0 || m->n_cols < 0) return fail(COOT_ERR_INVALID_ARG, std::string(what) + ": negative size");
  if (m->ld < std::max<int64_t>(m->n_rows, 1)) return fail(COOT_ERR_INVALID_ARG, std::string(what) + ": ld < n_rows");
  if (m->n_rows > 0 && m->n_cols > 0 && m->ptr == nullptr)
    return fail(COOT_ERR_INVALID_ARG, std::string(what) + ": NULL data pointer");
  if (m->n_rows > (int64_t(1) << 40) || m->n_cols > (int64_t(1) << 40) || m->ld > (int64_t(1) << 40))
    return fail(COOT_ERR_INVALID_ARG, std::string(what) + ": size too large");
  return COOT_OK;
}

static int64_t n_elem(const coot_mat& m) { return m.n_rows * m.n_cols; }

// [first, last) byte range a matrix touches
static void byte_range(const coot_mat& m, uintptr_t* b, uintptr_t* e) {
  const uintptr_t base = (uintptr_t)m.ptr;
  *b = base;
  *e = base + (uintptr_t)((m.n_cols - 1) * m.ld + m.n_rows) * dtype_size(m.dtype);
}

static bool same_mat(const coot_mat& a, const coot_mat& b) {
  return a.ptr == b.ptr && a.dtype == b.dtype && a.n_rows == b.n_rows && a.n_cols == b.n_cols && a.ld == b.ld;
}

// Tree, operand count, operand checks and equal shapes, then the call's
// canonical form: the tree rewritten exactly and the operands it reads,
// each distinct matrix once.
struct Operands {
  Tree t;
  coot_mat in[COOT_TREE_MAX_INPUTS];
  int n = 0;
};

static coot_status check_operands(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, Operands* ops) {
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  if (in == nullptr) return fail(COOT_ERR_INVALID_ARG, "inputs are NULL");
  if (n_in != t.n_inputs)
    return fail(COOT_ERR_INVALID_ARG, "tree has " + std::to_string(t.n_inputs) + " inputs, " +
                                          std::to_string(n_in) + " given");
  for (int i = 0; i < n_in; ++i) {
    s = check_mat(&in[i], "input");
    if (s != COOT_OK) return s;
    if (in[i].n_rows != in[0].n_rows || in[i].n_cols != in[0].n_cols)
      return fail(COOT_ERR_SHAPE, "element-wise operands need equal sizes: input " + std::to_string(i) + " is " +
                                      std::to_string(in[i].n_rows) + "x" + std::to_string(in[i].n_cols) +
                                      ", input 0 is " + std::to_string(in[0].n_rows) + "x" +
                                      std::to_string(in[0].n_cols));
  }
  if (!canonical_enabled()) {
    ops->t = std::move(t);
    for (int i = 0; i < n_in; ++i) ops->in[i] = in[i];
    ops->n = n_in;
    return COOT_OK;
  }
  int alias[COOT_TREE_MAX_INPUTS];
  for (int i = 0; i < n_in; ++i) {
    alias[i] = i;
    for (int j = 0; j < i; ++j)
      if (alias[j] == j && in[i].ptr == in[j].ptr && in[i].dtype == in[j].dtype && in[i].ld == in[j].ld) {
        alias[i] = j;
        break;
      }
  }
  std::vector<int> kept;
  canonicalize(t, alias, &ops->t, &kept, false);
  ops->n = (int)kept.size();
  for (int k = 0; k < ops->n; ++k) ops->in[k] = in[kept[k]];
  return COOT_OK;
}

// Whether two matrices share an element.  With the same dtype and ld they
// are compared as views of one column-major parent (row and column ranges,
// so disjoint submatrices of one matrix do not overlap); otherwise by their
// byte ranges, which may report an overlap that is not there.
static bool overlaps(const coot_mat& a, const coot_mat& b) {
  if (n_elem(a) == 0 || n_elem(b) == 0) return false;
  uintptr_t ab, ae, bb, be;
  byte_range(a, &ab, &ae);
  byte_range(b, &bb, &be);
  if (!(ab < be && bb < ae)) return false;
  if (a.dtype != b.dtype || a.ld != b.ld) return true;
  const int64_t es = dtype_size(a.dtype);
  const int64_t diff = (int64_t)((intptr_t)b.ptr - (intptr_t)a.ptr);
  if (diff % es != 0) return true;
  const int64_t d = diff / es;  // b's first element from a's, in elements
  const int64_t col = d >= 0 ? d / a.ld : -((-d + a.ld - 1) / a.ld);  // floor(d / ld)
  const int64_t row = d - col * a.ld;                                 // 0 <= row < ld
  if (row + b.n_rows > a.ld) return true;  // b's columns wrap: not a view of a's parent
  return row < a.n_rows && col < a.n_cols && col + b.n_cols > 0;
}

bool mats_overlap(const coot_mat& a, const coot_mat& b) { return overlaps(a, b); }

// Output aliasing: identical to an input is allowed (and disables the
// non-coherent load path), any other overlap is an error.
static coot_status check_alias(const coot_mat& out, const coot_mat* in, int n_in, bool allow_identical, bool* aliased) {
  *aliased = false;
  if (n_elem(out) == 0) return COOT_OK;
  for (int i = 0; i < n_in; ++i) {
    if (overlaps(out, in[i])) {
      if (allow_identical && same_mat(out, in[i])) {
        *aliased = true;
      } else {
        return fail(COOT_ERR_ALIAS, "output overlaps input " + std::to_string(i) + " without being identical to it");
      }
    }
  }
  return COOT_OK;
}

// Operands as the kernels see them: a 2-D column-major view (n_rows x
// n_cols, per-operand ld).  When every operand is dense (ld == n_rows or a
// single column) the whole object is one long column.
struct View {
  const void* ptr[8];
  int64_t ld[8];
  int dtype[8];
  int n = 0;  // operands (inputs, then the stored outputs if any)
  int64_t n_rows = 0, n_cols = 0;
};

static View make_view(const coot_mat* in, int n_in, const coot_mat* out, const coot_mat* const* more_outs = nullptr,
                      int n_more = 0) {
  View v;
  v.n_rows = in[0].n_rows;
  v.n_cols = in[0].n_cols;
  for (int i = 0; i < n_in; ++i) {
    v.ptr[v.n] = in[i].ptr;
    v.ld[v.n] = in[i].ld;
    v.dtype[v.n] = in[i].dtype;
    ++v.n;
  }
  if (out) {
    v.ptr[v.n] = out->ptr;
    v.ld[v.n] = out->ld;
    v.dtype[v.n] = out->dtype;
    ++v.n;
  }
  for (int i = 0; i < n_more; ++i) {
    v.ptr[v.n] = more_outs[i]->ptr;
    v.ld[v.n] = more_outs[i]->ld;
    v.dtype[v.n] = more_outs[i]->dtype;
    ++v.n;
  }
  bool dense = true;
  for (int i = 0; i < v.n; ++i) dense = dense && (v.ld[i] == v.n_rows || v.n_cols <= 1);
  if (dense && v.n_cols > 1) {
    v.n_rows = v.n_rows * v.n_cols;
    v.n_cols = 1;
    for (int i = 0; i < v.n; ++i) v.ld[i] = v.n_rows;
  }
  return v;
}

// Largest vector width (elements) with every access aligned: at most 16
// bytes per access for the widest operand, every base pointer aligned to
// the access, and every ld a multiple of it when there are several columns.
static int pick_vec(const View& v, int max_vec = 8) {
  int widest = 1;
  for (int i = 0; i < v.n; ++i) widest = std::max(widest, dtype_size(v.dtype[i]));
  for (int vec = max_vec; vec > 1; vec >>= 1) {
    if (vec * widest > 16) continue;
    bool ok = true;
    for (int i = 0; i < v.n && ok; ++i) {
      ok = ((uintptr_t)v.ptr[i] % (uintptr_t)(vec * dtype_size(v.dtype[i]))) == 0;
      if (v.n_cols > 1) ok = ok && (v.ld[i] % vec == 0);
    }
    if (ok) return vec;
  }
  return 1;
}

// ------------------------------------------------------------ launch policy

struct Launch {
  int vec = 1, unroll = 1, block = 256;
  int blocks_per_sm = 0;  // 0: as many as fit
  int64_t split = 0;      // 0: chosen from the shape
};

// A launch shape set by the caller for the calls that follow on this
// thread (tuning, learned selection); block == 0 means "not set".
static thread_local Launch g_override[KIND_COUNT] = {{1, 1, 0}, {1, 1, 0}, {1, 1, 0}, {1, 1, 0}, {1, 1, 0},
                                                     {1, 1, 0}, {1, 1, 0}, {1, 1, 0}, {1, 1, 0}};
// The shape of the last launch on this thread.
static thread_local Launch g_last;
static thread_local int64_t g_last_grid = 0;

static CallInfo call_info(int kind, const Tree& t, const coot_mat* in, int n_in, int out_dtype, unsigned heads,
                          const View& v) {
  CallInfo c;
  c.kind = kind;
  c.tree = &t;
  c.in_bytes = 1;
  for (int i = 0; i < n_in; ++i) c.in_bytes = std::max(c.in_bytes, dtype_size(in[i].dtype));
  c.out_bytes = out_dtype >= 0 ? dtype_size(out_dtype) : 0;
  c.heads = heads;
  c.n_rows = in[0].n_rows;
  c.n_cols = in[0].n_cols;
  c.dense = true;
  for (int i = 0; i < n_in; ++i) c.dense = c.dense && (in[i].ld == in[i].n_rows || in[i].n_cols <= 1);
  (void)v;
  return c;
}

// The learned policy's choice for a call: the candidate shape with the
// lowest predicted time, cached per distinct call.
static std::mutex g_choice_mu;
static std::unordered_map<uint64_t, Launch> g_choice;

static bool learned_choice(int kind, const View& v, const CallInfo& ci, Launch* out) {
  if (kind > KIND_ROWSUM || policy() != COOT_POLICY_LEARNED || !model_ready()) return false;
  const int64_t key_fields[] = {kind, ci.in_bytes, ci.out_bytes, (int64_t)ci.heads, ci.n_rows, ci.n_cols,
                                ci.dense, pick_vec(v), device().id};
  const uint64_t key = fnv1a(key_fields, sizeof key_fields, ci.tree->hash);
  {
    std::lock_guard<std::mutex> lock(g_choice_mu);
    auto it = g_choice.find(key);
    if (it != g_choice.end()) {
      *out = it->second;
      return true;
    }
  }
  const int (*cand)[4] = nullptr;
  const int n = candidates(kind, &cand);
  double best = 0.0;
  int best_i = -1;
  float f[COOT_MODEL_FEATURES];
  for (int i = 0; i < n; ++i) {
    const int vec = cand[i][1] ? pick_vec(v, cand[i][1]) : pick_vec(v);
    call_features(ci, cand[i][0], vec, cand[i][2], cand[i][3], f);
    const double y = model_predict(f);
    if (best_i < 0 || y < best) {
      best = y;
      best_i = i;
    }
  }
  if (best_i < 0) return false;
  Launch l;
  l.block = cand[best_i][0];
  l.vec = cand[best_i][1] ? pick_vec(v, cand[best_i][1]) : pick_vec(v);
  l.unroll = cand[best_i][2];
  l.split = cand[best_i][3];
  std::lock_guard<std::mutex> lock(g_choice_mu);
  g_choice[key] = l;
  *out = l;
  return true;
}

static int popcount(unsigned m) {
  int k = 0;
  for (; m; m &= m - 1) ++k;
  return k;
}

static Launch heuristic(int kind, int n_in, const View& v, const CallInfo* ci = nullptr) {
  Launch l;
  const Launch& o = g_override[kind];
  if (!o.block && ci && learned_choice(kind, v, *ci, &l)) return l;
  // built-in choices, from exhaustive sweeps on GB300 (see the tuning
  // module): many bytes in flight per thread beat occupancy for these
  // streaming kernels
  l.vec = pick_vec(v);
  l.block = 256;
  if (kind == KIND_ROWSUM) {
    l.block = 512;
    l.unroll = n_in >= 3 ? 4 : 8;
  } else if (kind == KIND_COLSUM) {
    l.unroll = 4;
  } else if (kind == KIND_COLSTATS) {
    // the statistics' accumulators leave room for 8 accesses in flight;
    // 128-thread blocks (one input at 8192²: 0.0622 ms at block 256,
    // 0.0572 ms at 128, vec 4, unroll 8)
    l.unroll = 8;
    l.block = 128;
    if (n_in >= 3) l.vec = std::min(l.vec, pick_vec(v, 2));
  } else if (kind == KIND_ROWSTATS) {
    l.block = 128;
    l.unroll = 8;
    l.vec = std::min(l.vec, pick_vec(v, 2));
  } else {
    l.unroll = n_in >= 3 ? 4 : 8;
    if (kind == KIND_REDUCE && n_in == 1 && ci != nullptr &&
        popcount(ci->heads & (COOT_HEAD_SUM | COOT_HEAD_SUMSQ | COOT_HEAD_NORM2 | COOT_HEAD_SUMABS)) >= 2) {
      // two compensated sums of one stream: issue-bound, so many loads in
      // flight per thread and, for 2-byte storage, one 1024-thread block
      // per SM (a sweep over block 256 / 512 / 1024 and unroll 4 / 8 / 16
      // on 2^28 BF16 / FP16 / FP32 values: accu + norm2 from 69% / 66% /
      // 92% of measured HBM bandwidth to 80% / 77% / 100%)
      l.unroll = 16;
      if (ci->in_bytes <= 2) l.block = 1024;
    }
    // Small inputs: fewer elements per thread until the grid covers the
    // GPU, about 4 blocks per SM for element-wise evaluation and 1.5 for
    // calls with reduction heads, whose last block combines one partial
    // per block (sweeps over block, vector width and unroll on a 10^6
    // vector, each call replayed in a CUDA graph: 3.5 -> 2.6 us for
    // 2x + 3z, 6.8 -> 5.9 us for accu(x % z)).
    const bool heads = kind == KIND_REDUCE || (ci != nullptr && ci->heads != 0);
    const int64_t want = heads ? (int64_t)device().sm_count * 3 / 2 : (int64_t)device().sm_count * 4;
    auto units = [&](int unroll) {
      const int64_t tile = (int64_t)l.block * l.vec * unroll;
      return ((v.n_rows + tile - 1) / tile) * v.n_cols;
    };
    while (l.unroll > 1 && units(l.unroll) < want) l.unroll /= 2;
  }
  if (o.block) {
    l.block = o.block;
    if (o.vec) l.vec = pick_vec(v, o.vec);
    if (o.unroll) l.unroll = o.unroll;
    l.blocks_per_sm = o.blocks_per_sm;
    l.split = o.split;
  }
  return l;
}

static void fill_io(coot_params_host* p, const View& v, int n_in) {
  std::memset(p, 0, sizeof *p);
  for (int i = 0; i < n_in; ++i) {
    p->in[i] = v.ptr[i];
    p->ld_in[i] = v.ld[i];
  }
  for (int i = n_in; i < 4; ++i) p->ld_in[i] = 1;
  p->n_rows = v.n_rows;
  p->n_cols = v.n_cols;
}

static coot_status launch(const Compiled* c, int64_t units, int64_t max_grid, const Launch& l, coot_params_host* p,
                          void* stream, void* kernel_params = nullptr, size_t dyn_smem = 0) {
  int bps = std::max(1, c->max_blocks_per_sm);
  if (l.blocks_per_sm > 0) bps = std::min(bps, l.blocks_per_sm);
  int64_t grid = (int64_t)device().sm_count * bps;
  grid = std::min(grid, std::max<int64_t>(units, 1));
  grid = std::min(grid, max_grid);
  grid = std::max<int64_t>(grid, 1);
  void* args[] = {kernel_params ? kernel_params : (void*)p};
  cudaError_t e = cudaLaunchKernel((const void*)c->kernel, dim3((unsigned)grid), dim3(l.block), args, dyn_smem,
                                   (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  g_last = l;
  g_last.split = p->split;
  g_last_grid = grid;
  return COOT_OK;
}


static int tile_rows(const Launch& l) { return l.block * l.vec * l.unroll; }

// Element-wise evaluation and/or full reductions of one tree.
// The heads of reductions over an empty object, for `n` groups of heads
// (masks[k], results one group after another in increasing bit order):
// sums, norms and any() are 0, all() is 1; min / max are an error.
static coot_status empty_heads(double* res, const unsigned* masks, int n, void* stream) {
  unsigned any_mask = 0;
  int total = 0;
  for (int k = 0; k < n; ++k) {
    any_mask |= masks[k];
    total += popcount(masks[k]);
  }
  if (any_mask & (COOT_HEAD_MIN | COOT_HEAD_MAX)) return fail(COOT_ERR_EMPTY, "min/max of an empty object");
  cudaError_t e = cudaMemsetAsync(res, 0, sizeof(double) * total, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  int base = 0;
  for (int k = 0; k < n; ++k) {
    if (masks[k] & COOT_HEAD_ALL) {
      const double* one = nullptr;
      coot_status s = device_one(&one);
      if (s != COOT_OK) return s;
      e = cudaMemcpyAsync(res + base + popcount(masks[k] & (COOT_HEAD_ALL - 1)), one, sizeof(double),
                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
      if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    }
    base += popcount(masks[k]);
  }
  return COOT_OK;
}

static coot_status run_map_reduce(const Tree& t, const coot_mat* in, int n_in, unsigned heads, const coot_mat* out,
                                  double* res, void* ws, size_t ws_bytes, void* stream) {
  const bool store = out != nullptr;
  const int64_t n = n_elem(in[0]);
  if (heads) {
    if (res == nullptr) return fail(COOT_ERR_INVALID_ARG, "result pointer is NULL");
    if (n == 0) return empty_heads(res, &heads, 1, stream);
    if (ws == nullptr || ws_bytes < COOT_WS_PARTIALS_OFF + sizeof(double) * popcount(heads))
      return fail(COOT_ERR_WORKSPACE, "reductions need a workspace (coot_workspace_size)");
  } else if (n == 0) {
    return COOT_OK;
  }
  bool aliased = false;
  if (store) {
    coot_status s = check_mat(out, "output");
    if (s != COOT_OK) return s;
    if (out->n_rows != in[0].n_rows || out->n_cols != in[0].n_cols)
      return fail(COOT_ERR_SHAPE, "output shape differs from the operands'");
    s = check_alias(*out, in, n_in, true, &aliased);
    if (s != COOT_OK) return s;
  }
  const View v = make_view(in, n_in, store ? out : nullptr);
  const int kind = heads ? (store ? KIND_MAP : KIND_REDUCE) : KIND_MAP;
  const CallInfo ci = call_info(kind, t, in, n_in, store ? out->dtype : -1, heads, v);
  const Launch l = heuristic(kind, n_in, v, &ci);
  KernelSpec spec;
  spec.kind = kind;
  for (int i = 0; i < n_in; ++i) spec.in_dtype[i] = in[i].dtype;
  spec.out_dtype = store ? out->dtype : 0;
  spec.store = store;
  spec.heads = heads;
  spec.vec = l.vec;
  spec.unroll = l.unroll;
  spec.block = l.block;
  spec.nc = !aliased;
  const Compiled* c = nullptr;
  coot_status s = kernel_for(t, spec, &c);
  if (s != COOT_OK) return s;
  coot_params_host p;
  fill_io(&p, v, n_in);
  if (store) {
    p.out = v.ptr[n_in] ? const_cast<void*>(v.ptr[n_in]) : nullptr;
    p.ld_out = v.ld[n_in];
  }
  p.ws = (unsigned char*)ws;
  p.res = res;
  const int64_t tile = tile_rows(l);
  const int64_t units = ((v.n_rows + tile - 1) / tile) * v.n_cols;
  int64_t max_grid = INT32_MAX;
  if (heads) {
    const int64_t fit = (int64_t)((ws_bytes - COOT_WS_PARTIALS_OFF) / (sizeof(double) * popcount(heads)));
    max_grid = std::min<int64_t>(COOT_MAX_GRID, fit);
  }
  return launch(c, units, max_grid, l, &p, stream);
}

static coot_status run_sum_dim(const Tree& t, const coot_mat* in, int n_in, int dim, const coot_mat* out, void* ws,
                               size_t ws_bytes, void* stream) {
  coot_status s = check_mat(out, "output");
  if (s != COOT_OK) return s;
  const int64_t R = in[0].n_rows, Cn = in[0].n_cols;
  if (dim == 0) {
    if (out->n_rows != 1 || out->n_cols != Cn)
      return fail(COOT_ERR_SHAPE, "sum(dim=0) output must be 1 x n_cols");
  } else if (dim == 1) {
    if (out->n_rows != R || out->n_cols != 1)
      return fail(COOT_ERR_SHAPE, "sum(dim=1) output must be n_rows x 1");
  } else {
    return fail(COOT_ERR_INVALID_ARG, "dim must be 0 or 1");
  }
  if (!is_float(out->dtype)) return fail(COOT_ERR_DTYPE, "sums are stored in a floating-point type");
  bool aliased = false;
  s = check_alias(*out, in, n_in, false, &aliased);
  if (s != COOT_OK) return s;
  if (n_elem(*out) == 0) return COOT_OK;
  // the element layout of the operands; the output is addressed separately
  View v;
  v.n_rows = R;
  v.n_cols = Cn;
  for (int i = 0; i < n_in; ++i) {
    v.ptr[i] = in[i].ptr;
    v.ld[i] = in[i].ld;
    v.dtype[i] = in[i].dtype;
  }
  v.n = n_in;
  const int kind = dim == 0 ? KIND_COLSUM : KIND_ROWSUM;
  const CallInfo ci = call_info(kind, t, in, n_in, -1, 0, v);
  Launch l = heuristic(kind, n_in, v, &ci);
  const Device& d = device();
  KernelSpec spec;
  spec.kind = kind;
  for (int i = 0; i < n_in; ++i) spec.in_dtype[i] = in[i].dtype;
  spec.out_dtype = out->dtype;
  spec.vec = l.vec;
  spec.unroll = l.unroll;
  spec.block = l.block;
  spec.nc = true;
  const Compiled* c = nullptr;
  s = kernel_for(t, spec, &c);
  if (s != COOT_OK) return s;
  coot_params_host p;
  fill_io(&p, v, n_in);
  p.out = out->ptr;
  p.ld_out = out->ld;
  p.ws = (unsigned char*)ws;
  const int64_t resident = (int64_t)d.sm_count * std::max(1, c->max_blocks_per_sm);
  const size_t part_bytes = ws ? (ws_bytes > COOT_WS_PARTIALS_OFF ? ws_bytes - COOT_WS_PARTIALS_OFF : 0) : 0;
  int64_t units;  // blocks' worth of work
  if (dim == 0) {
    // a warp per (column, segment); with fewer columns than about 1.5 per
    // resident warp, split the columns into segments up to that count
    const int64_t warps = l.block / 32;
    const int64_t wt = 32LL * l.vec * l.unroll;  // rows per warp tile
    const int64_t target = 3 * resident * warps / 2;
    int64_t S = 1;
    if (Cn < target && R > wt && Cn <= COOT_WS_MAX_COUNTERS) {
      S = std::min<int64_t>((target + Cn - 1) / Cn, (R + wt - 1) / wt);
      // a segment partial is a double-word pair of the compute type
      const int64_t entry = 2 * (t.compute == COOT_F64 ? 8 : 4);
      S = std::min<int64_t>(S, (int64_t)(part_bytes / (entry * std::max<int64_t>(Cn, 1))));
      S = std::max<int64_t>(S, 1);
    }
    if (l.split > 0 && Cn <= COOT_WS_MAX_COUNTERS) {
      const int64_t entry = 2 * (t.compute == COOT_F64 ? 8 : 4);
      S = std::min<int64_t>(l.split, (R + wt - 1) / wt);
      S = std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)(part_bytes / (entry * std::max<int64_t>(Cn, 1)))));
    }
    int64_t rps = (R + S - 1) / S;
    rps = std::max<int64_t>(((rps + wt - 1) / wt) * wt, wt);
    if (S > 1) S = std::max<int64_t>((R + rps - 1) / rps, 1);
    p.split = S;
    p.rows_per_split = rps;
    units = (Cn * S + warps - 1) / warps;
  } else {
    // panels of 64 * vec rows; chunks of columns until there are about 1.5
    // units per SM (large units: few partials, little per-unit overhead)
    const int64_t groups = std::max(1, l.block / 64);
    const int64_t panel = 64LL * l.vec;
    const int64_t n_panels = (R + panel - 1) / panel;
    const int64_t target = 3 * (int64_t)d.sm_count / 2;
    int64_t C = std::max<int64_t>(1, (target + n_panels - 1) / n_panels);
    if (l.split > 0) C = l.split;
    C = std::min<int64_t>(C, std::max<int64_t>((Cn + groups - 1) / groups, 1));
    C = std::min<int64_t>(C, COOT_MAX_ROW_CHUNKS);
    // a chunk partial is a double-word pair of the compute type per row
    const int64_t entry = 2 * (t.compute == COOT_F64 ? 8 : 4);
    C = std::min<int64_t>(C, (int64_t)(part_bytes / (entry * std::max<int64_t>(R, 1))));
    if (n_panels > COOT_WS_MAX_COUNTERS) C = 1;
    C = std::max<int64_t>(C, 1);
    p.split = C;
    units = n_panels * C;
  }
  if (p.split > 1 && ws == nullptr) return fail(COOT_ERR_WORKSPACE, "split sums need a workspace");
  return launch(c, units, INT32_MAX, l, &p, stream);
}

// Statistics of each column (dim 0) or row (dim 1): the column / row sum
// kernels' work division, with a partial of NC components per line.
static coot_status run_stats_dim(const Tree& t, const coot_mat* in, int n_in, int dim, unsigned stats, int norm_type,
                                 const coot_mat* out, void* ws, size_t ws_bytes, void* stream) {
  if (dim != 0 && dim != 1) return fail(COOT_ERR_INVALID_ARG, "dim must be 0 or 1");
  if (stats == 0 || (stats & ~COOT_STAT_MASK)) return fail(COOT_ERR_INVALID_ARG, "stats must be a nonzero COOT_STAT_* mask");
  if (norm_type != 0 && norm_type != 1) return fail(COOT_ERR_INVALID_ARG, "norm_type must be 0 or 1");
  if (out == nullptr) return fail(COOT_ERR_INVALID_ARG, "outputs are NULL");
  const int64_t R = in[0].n_rows, Cn = in[0].n_cols;
  const int64_t lines = dim == 0 ? Cn : R, N = dim == 0 ? R : Cn;
  int n_out = 0;
  for (unsigned m = stats; m; m &= m - 1) ++n_out;
  for (int k = 0; k < n_out; ++k) {
    coot_status s = check_mat(&out[k], "output");
    if (s != COOT_OK) return s;
    if (dim == 0 ? (out[k].n_rows != 1 || out[k].n_cols != Cn) : (out[k].n_rows != R || out[k].n_cols != 1))
      return fail(COOT_ERR_SHAPE, dim == 0 ? "statistics along dim 0 are 1 x n_cols" : "statistics along dim 1 are n_rows x 1");
    if (out[k].dtype != COOT_F32 && out[k].dtype != COOT_F64)
      return fail(COOT_ERR_DTYPE, "statistics are stored as FP32 or FP64");
    if (out[k].dtype != out[0].dtype) return fail(COOT_ERR_DTYPE, "every statistics output needs the same dtype");
    bool aliased = false;
    s = check_alias(out[k], in, n_in, false, &aliased);
    if (s != COOT_OK) return s;
    s = check_alias(out[k], out, k, false, &aliased);
    if (s != COOT_OK) return fail(COOT_ERR_ALIAS, "statistics outputs overlap each other");
  }
  if (lines == 0) return COOT_OK;
  if (N == 0 && (stats & (COOT_STAT_MIN | COOT_STAT_MAX)))
    return fail(COOT_ERR_EMPTY, "min/max along a dimension of length 0");
  View v;
  v.n_rows = R;
  v.n_cols = Cn;
  for (int i = 0; i < n_in; ++i) {
    v.ptr[i] = in[i].ptr;
    v.ld[i] = in[i].ld;
    v.dtype[i] = in[i].dtype;
  }
  v.n = n_in;
  const int kind = dim == 0 ? KIND_COLSTATS : KIND_ROWSTATS;
  Launch l = heuristic(kind, n_in, v);
  const int real = t.compute == COOT_F64 ? 8 : 4;
  if (kind == KIND_ROWSTATS) {
    // the block's shared partials: at most 256 threads and 16-byte rows
    l.block = std::min(l.block, 256);
    l.vec = std::min(l.vec, pick_vec(v, 16 / real));
  }
  const Device& d = device();
  KernelSpec spec;
  spec.kind = kind;
  for (int i = 0; i < n_in; ++i) spec.in_dtype[i] = in[i].dtype;
  spec.out_dtype = out[0].dtype;
  spec.heads = stats;
  spec.vec = l.vec;
  spec.unroll = l.unroll;
  spec.block = l.block;
  spec.nc = true;
  const Compiled* c = nullptr;
  coot_status s = kernel_for(t, spec, &c);
  if (s != COOT_OK) return s;
  coot_stats_params_host sp;
  std::memset(&sp, 0, sizeof sp);
  fill_io(&sp.b, v, n_in);
  sp.b.ws = (unsigned char*)ws;
  int k = 0;
  for (int b = 0; b < 6; ++b) {
    if (!(stats & (1u << b))) continue;
    sp.out[k] = out[k].ptr;
    sp.inc[k] = dim == 0 ? out[k].ld : 1;
    ++k;
  }
  sp.norm_type = norm_type;
  // components of a partial: the sum, the shifted sum (rows only) and the
  // shifted sum of squares as pairs, min, max
  const bool s1 = stats & (COOT_STAT_SUM | COOT_STAT_MEAN);
  const bool dv = stats & (COOT_STAT_VAR | COOT_STAT_STDDEV);
  // (the column statistics keep the sum whenever they need the variance,
  // and no shifted sum)
  const int64_t entry = dim == 0
      ? (2 * (s1 || dv) + 2 * dv + !!(stats & COOT_STAT_MIN) + !!(stats & COOT_STAT_MAX)) * real
      : (2 * s1 + 4 * dv + !!(stats & COOT_STAT_MIN) + !!(stats & COOT_STAT_MAX)) * real;
  const int64_t resident = (int64_t)d.sm_count * std::max(1, c->max_blocks_per_sm);
  const size_t part_bytes = ws ? (ws_bytes > COOT_WS_PARTIALS_OFF ? ws_bytes - COOT_WS_PARTIALS_OFF : 0) : 0;
  int64_t units;
  if (dim == 0) {
    // about one (column, segment) unit per resident warp
    const int64_t warps = l.block / 32;
    const int64_t wt = 32LL * l.vec * l.unroll;
    const int64_t target = resident * warps;
    int64_t S = 1;
    if (Cn < target && R > wt && Cn <= COOT_WS_MAX_COUNTERS) S = std::min<int64_t>((target + Cn - 1) / Cn, (R + wt - 1) / wt);
    if (l.split > 0) S = std::min<int64_t>(l.split, std::max<int64_t>((R + wt - 1) / wt, 1));
    if (Cn > COOT_WS_MAX_COUNTERS) S = 1;
    S = std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)(part_bytes / (entry * std::max<int64_t>(Cn, 1)))));
    int64_t rps = (R + S - 1) / S;
    rps = std::max<int64_t>(((rps + wt - 1) / wt) * wt, wt);
    if (S > 1) S = std::max<int64_t>((R + rps - 1) / rps, 1);
    sp.b.split = S;
    sp.b.rows_per_split = rps;
    units = (Cn * S + warps - 1) / warps;
  } else {
    // about 7 units per SM: small units keep enough row panels in flight
    // for the statistics' longer per-element work (at 8192², 16 column
    // chunks against 15: one input 0.0614 -> 0.0589 ms, four inputs
    // 0.1754 -> 0.1714 ms)
    const int64_t groups = std::max(1, l.block / 64);
    const int64_t panel = 64LL * l.vec;
    const int64_t n_panels = (R + panel - 1) / panel;
    const int64_t target = 7 * (int64_t)d.sm_count;
    int64_t C = std::max<int64_t>(1, (target + n_panels - 1) / n_panels);
    if (l.split > 0) C = l.split;
    C = std::min<int64_t>(C, std::max<int64_t>((Cn + groups - 1) / groups, 1));
    C = std::min<int64_t>(C, COOT_MAX_ROW_CHUNKS);
    C = std::min<int64_t>(C, (int64_t)(part_bytes / (entry * std::max<int64_t>(R, 1))));
    if (n_panels > COOT_WS_MAX_COUNTERS) C = 1;
    C = std::max<int64_t>(C, 1);
    sp.b.split = C;
    units = n_panels * C;
  }
  if (sp.b.split > 1 && ws == nullptr) return fail(COOT_ERR_WORKSPACE, "split statistics need a workspace");
  return launch(c, units, INT32_MAX, l, &sp.b, stream, &sp);
}

}  // namespace coot

using namespace coot;

extern "C" {

coot_status coot_init(int dev, unsigned flags) {
  clear_error();
  return init_device(dev, flags);
}

coot_status coot_finalize(void) {
  clear_error();
  drop_kernels();
  return COOT_OK;
}

const char* coot_last_error(void) { return g_err.c_str(); }

const char* coot_status_string(coot_status s) {
  switch (s) {
    case COOT_OK: return "COOT_OK";
    case COOT_ERR_INVALID_ARG: return "COOT_ERR_INVALID_ARG";
    case COOT_ERR_BAD_TREE: return "COOT_ERR_BAD_TREE";
    case COOT_ERR_SHAPE: return "COOT_ERR_SHAPE";
    case COOT_ERR_DTYPE: return "COOT_ERR_DTYPE";
    case COOT_ERR_ALIAS: return "COOT_ERR_ALIAS";
    case COOT_ERR_EMPTY: return "COOT_ERR_EMPTY";
    case COOT_ERR_UNSUPPORTED: return "COOT_ERR_UNSUPPORTED";
    case COOT_ERR_COMPILE: return "COOT_ERR_COMPILE";
    case COOT_ERR_CUDA: return "COOT_ERR_CUDA";
    case COOT_ERR_TIMEOUT: return "COOT_ERR_TIMEOUT";
    case COOT_ERR_NOT_INIT: return "COOT_ERR_NOT_INIT";
    case COOT_ERR_WORKSPACE: return "COOT_ERR_WORKSPACE";
  }
  return "COOT_ERR_UNKNOWN";
}

int coot_version(void) { return 100; }

coot_status coot_set_launch_config(int kind, int block, int vec, int unroll, int blocks_per_sm, int64_t split) {
  clear_error();
  if (kind < 0 || kind >= KIND_COUNT) return fail(COOT_ERR_INVALID_ARG, "kind must be 0..8");
  if (block == 0) {
    g_override[kind] = Launch{1, 1, 0};
    return COOT_OK;
  }
  if (block < 64 || block > 1024 || block % 64 != 0) return fail(COOT_ERR_INVALID_ARG, "block must be 64..1024, a multiple of 64");
  if (!(vec == 0 || vec == 1 || vec == 2 || vec == 4 || vec == 8)) return fail(COOT_ERR_INVALID_ARG, "vec must be 0, 1, 2, 4 or 8");
  if (unroll < 0 || unroll > 16) return fail(COOT_ERR_INVALID_ARG, "unroll must be 0..16");
  if (blocks_per_sm < 0 || blocks_per_sm > 32) return fail(COOT_ERR_INVALID_ARG, "blocks_per_sm must be 0..32");
  if (split < 0 || split > 4096) return fail(COOT_ERR_INVALID_ARG, "split must be 0..4096");
  Launch o;
  o.block = block;
  o.vec = vec;
  o.unroll = unroll;
  o.blocks_per_sm = blocks_per_sm;
  o.split = split;
  g_override[kind] = o;
  return COOT_OK;
}

// The canonical form of a tree whose input slots are given positionally
// (no call-time merging), when canonical forms are on.
static void canonical_in_place(Tree* t) {
  if (!canonical_enabled()) return;
  Tree c;
  canonicalize(*t, nullptr, &c, nullptr, true);
  *t = std::move(c);
}

coot_status coot_prepare(const uint8_t* tree, size_t len, int kind, const int32_t* dtypes, int out_dtype,
                         unsigned heads, int block, int vec, int unroll) {
  clear_error();
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  canonical_in_place(&t);
  if (kind < 0 || kind >= KIND_COUNT || !dtypes) return fail(COOT_ERR_INVALID_ARG, "bad arguments");
  if (kind == KIND_MULTI || kind == KIND_DIMS)
    return fail(COOT_ERR_UNSUPPORTED, "the several-tree kernels are compiled by their first call");
  if (block < 64 || block > 1024 || block % 64) return fail(COOT_ERR_INVALID_ARG, "block must be 64..1024, a multiple of 64");
  if (!(vec == 1 || vec == 2 || vec == 4 || vec == 8) || unroll < 1 || unroll > 16)
    return fail(COOT_ERR_INVALID_ARG, "vec must be 1, 2, 4 or 8 and unroll 1..16");
  KernelSpec spec;
  spec.kind = kind;
  for (int i = 0; i < t.n_inputs; ++i) {
    if (dtype_size(dtypes[i]) == 0) return fail(COOT_ERR_DTYPE, "unknown dtype");
    spec.in_dtype[i] = dtypes[i];
  }
  spec.out_dtype = out_dtype >= 0 ? out_dtype : 0;
  spec.store = kind == KIND_MAP || kind == KIND_BATCHED;
  spec.heads = (kind == KIND_MAP || kind == KIND_REDUCE || kind == KIND_COLSTATS || kind == KIND_ROWSTATS) ? heads : 0;
  spec.vec = vec;
  spec.unroll = unroll;
  spec.block = block;
  spec.nc = true;
  const Compiled* c = nullptr;
  return kernel_for(t, spec, &c);
}

coot_status coot_call_features(const uint8_t* tree, size_t len, int kind, const int32_t* dtypes, int out_dtype,
                               unsigned heads, int64_t n_rows, int64_t n_cols, int dense, int block, int vec,
                               int unroll, int64_t split, float* features) {
  clear_error();
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  canonical_in_place(&t);
  if (kind < 0 || kind > 3 || !dtypes || !features || block < 1) return fail(COOT_ERR_INVALID_ARG, "bad arguments");
  CallInfo c;
  c.kind = kind;
  c.tree = &t;
  c.in_bytes = 1;
  for (int i = 0; i < t.n_inputs; ++i) {
    if (dtype_size(dtypes[i]) == 0) return fail(COOT_ERR_DTYPE, "unknown dtype");
    c.in_bytes = std::max(c.in_bytes, dtype_size(dtypes[i]));
  }
  c.out_bytes = out_dtype >= 0 ? dtype_size(out_dtype) : 0;
  c.heads = heads;
  c.n_rows = n_rows;
  c.n_cols = n_cols;
  c.dense = dense != 0;
  call_features(c, block, vec, unroll, split, features);
  return COOT_OK;
}

coot_status coot_last_launch(int* block, int* vec, int* unroll, int64_t* grid, int64_t* split) {
  clear_error();
  if (block) *block = g_last.block;
  if (vec) *vec = g_last.vec;
  if (unroll) *unroll = g_last.unroll;
  if (grid) *grid = g_last_grid;
  if (split) *split = g_last.split;
  return COOT_OK;
}

coot_status coot_workspace_size(int64_t max_rows, size_t* bytes) {
  clear_error();
  if (bytes == nullptr || max_rows < 0) return fail(COOT_ERR_INVALID_ARG, "bad workspace query");
  size_t part = (size_t)COOT_MAX_GRID * 8 * sizeof(double);
  part = std::max(part, (size_t)COOT_MAX_ROW_CHUNKS * (size_t)max_rows * sizeof(double));
  part = std::max(part, (size_t)COOT_WS_MAX_COUNTERS * 8 * sizeof(double));
  *bytes = COOT_WS_PARTIALS_OFF + part;
  return COOT_OK;
}

coot_status coot_tree_check(const uint8_t* tree, size_t len, int* n_inputs, int* compute, uint64_t* hash) {
  clear_error();
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  if (n_inputs) *n_inputs = t.n_inputs;
  if (compute) *compute = t.compute;
  if (hash) *hash = t.hash;
  return COOT_OK;
}

static coot_status spec_for(const Tree& t, int kind, int in_dtype, int out_dtype, unsigned heads, KernelSpec* spec) {
  if (kind < 0 || kind >= KIND_COUNT) return fail(COOT_ERR_INVALID_ARG, "kind must be 0..8");
  if (dtype_size(in_dtype) == 0 || dtype_size(out_dtype) == 0) return fail(COOT_ERR_DTYPE, "unknown dtype");
  spec->kind = kind;
  for (int i = 0; i < 4; ++i) spec->in_dtype[i] = i < t.n_inputs ? in_dtype : 0;
  spec->out_dtype = out_dtype;
  spec->store = kind == KIND_MAP || kind == KIND_BATCHED;
  spec->heads = (kind == KIND_MAP || kind == KIND_REDUCE || kind == KIND_COLSTATS || kind == KIND_ROWSTATS) ? heads : 0;
  if (kind == KIND_MULTI || kind == KIND_DIMS) {
    // one tree, stored and reduced by `heads` (and, for kind 8, its column
    // and row sums, in FP64 for FP64 storage, else FP32)
    spec->store = false;
    spec->n_trees = 1;
    spec->trees = &t;
    spec->tree_heads[0] = heads;
    spec->tree_out[0] = out_dtype;
    if (kind == KIND_DIMS) {
      // the dimension bits of `heads` (both when neither is given)
      unsigned dims = heads & (COOT_HEAD_COLSUM | COOT_HEAD_ROWSUM);
      if (dims == 0) dims = COOT_HEAD_COLSUM | COOT_HEAD_ROWSUM;
      spec->tree_heads[0] = heads | dims;
      const int sum_dt = out_dtype == COOT_F64 ? COOT_F64 : COOT_F32;
      if (dims & COOT_HEAD_COLSUM) spec->tree_cs[0] = sum_dt;
      if (dims & COOT_HEAD_ROWSUM) spec->tree_rs[0] = sum_dt;
      spec->min_blocks = 2;
    }
  }
  spec->vec = std::max(1, 16 / std::max(dtype_size(in_dtype), dtype_size(out_dtype)));
  spec->unroll = 2;
  spec->block = 256;
  return COOT_OK;
}

coot_status coot_tree_source(const uint8_t* tree, size_t len, int kind, char* buf, size_t buf_len, size_t* out_len) {
  clear_error();
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  KernelSpec spec;
  const unsigned heads = kind == KIND_REDUCE ? COOT_HEAD_SUM : (kind >= KIND_COLSTATS ? COOT_STAT_MASK : 0);
  s = spec_for(t, kind, COOT_F32, COOT_F32, heads, &spec);
  if (s != COOT_OK) return s;
  const std::string src = generate_source(t, spec);
  if (out_len) *out_len = src.size();
  if (buf && buf_len) {
    const size_t n = std::min(buf_len - 1, src.size());
    std::memcpy(buf, src.data(), n);
    buf[n] = '\0';
  }
  return COOT_OK;
}

coot_status coot_tree_compile(const uint8_t* tree, size_t len, int kind, int in_dtype, int out_dtype, unsigned heads,
                              const char* arch, size_t* cubin_bytes) {
  clear_error();
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  if (arch == nullptr) return fail(COOT_ERR_INVALID_ARG, "arch is NULL");
  KernelSpec spec;
  s = spec_for(t, kind, in_dtype, out_dtype, heads, &spec);
  if (s != COOT_OK) return s;
  return compile_only(generate_source(t, spec), arch, cubin_bytes);
}

coot_status coot_expr_eval(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, const coot_mat* out,
                           void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  if (out == nullptr) return fail(COOT_ERR_INVALID_ARG, "output is NULL");
  return run_map_reduce(o.t, o.in, o.n, 0, out, nullptr, ws, ws_bytes, stream);
}

coot_status coot_expr_reduce(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, unsigned heads,
                             const coot_mat* out, double* out_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  if (heads & ~COOT_HEAD_MASK) return fail(COOT_ERR_INVALID_ARG, "unknown head bits");
  if (heads == 0 && out == nullptr) return fail(COOT_ERR_INVALID_ARG, "nothing to compute");
  return run_map_reduce(o.t, o.in, o.n, heads, out, out_dev, ws, ws_bytes, stream);
}

// Trees, operands, stored outputs and heads of a several-tree call, checked
// (shared by coot_expr_multi and coot_expr_multi_dims).
struct MultiCall {
  Tree ts[4];
  KernelSpec spec;           // kind, trees, heads (with the dimension bits), stored types
  const coot_mat* stored[4];
  int n_stored = 0;
  bool aliased = false;      // a stored tree is identical to an input
  int total_heads = 0;       // full heads of every tree (one result each)
  unsigned all_heads = 0;
};

static coot_status multi_check(const uint8_t* const* trees, const size_t* tree_lens, int n_trees, const coot_mat* in,
                               int n_in, const coot_mat* outs, const unsigned* heads, unsigned allowed,
                               MultiCall* mc) {
  if (trees == nullptr || tree_lens == nullptr || n_trees < 1 || n_trees > 4)
    return fail(COOT_ERR_INVALID_ARG, "1 to 4 trees");
  if (in == nullptr || n_in < 1 || n_in > COOT_TREE_MAX_INPUTS) return fail(COOT_ERR_INVALID_ARG, "1 to 4 inputs");
  for (int i = 0; i < n_in; ++i) {
    coot_status s = check_mat(&in[i], "input");
    if (s != COOT_OK) return s;
    if (in[i].n_rows != in[0].n_rows || in[i].n_cols != in[0].n_cols)
      return fail(COOT_ERR_SHAPE, "element-wise operands need equal sizes: input " + std::to_string(i));
  }
  KernelSpec& spec = mc->spec;
  spec.kind = KIND_MULTI;
  spec.n_trees = n_trees;
  spec.trees = mc->ts;
  for (int k = 0; k < n_trees; ++k) {
    const std::string at = "tree " + std::to_string(k) + ": ";
    coot_status s = parse_tree(trees[k], tree_lens[k], &mc->ts[k]);
    if (s != COOT_OK) return fail(s, at + coot_last_error());
    canonical_in_place(&mc->ts[k]);
    if (mc->ts[k].n_inputs > n_in) return fail(COOT_ERR_INVALID_ARG, at + "uses more inputs than given");
    if (mc->ts[k].compute != mc->ts[0].compute) return fail(COOT_ERR_DTYPE, at + "compute type differs from tree 0's");
    const unsigned h = heads ? heads[k] : 0u;
    if (h & ~allowed) return fail(COOT_ERR_INVALID_ARG, at + "unknown head bits");
    spec.tree_heads[k] = h;
    mc->all_heads |= h;
    mc->total_heads += popcount(h & COOT_HEAD_MASK);
    if (outs != nullptr && outs[k].ptr != nullptr) {
      s = check_mat(&outs[k], "output");
      if (s != COOT_OK) return fail(s, at + coot_last_error());
      if (outs[k].n_rows != in[0].n_rows || outs[k].n_cols != in[0].n_cols)
        return fail(COOT_ERR_SHAPE, at + "output shape differs from the operands'");
      spec.tree_out[k] = outs[k].dtype;
      mc->stored[mc->n_stored++] = &outs[k];
    } else if (h == 0) {
      return fail(COOT_ERR_INVALID_ARG, at + "nothing to compute (no output, no heads)");
    }
  }
  // outputs: each may be identical to an input (every element's inputs are
  // read before any tree's value is stored), none may overlap another
  for (int a = 0; a < mc->n_stored; ++a) {
    bool al = false;
    coot_status s = check_alias(*mc->stored[a], in, n_in, true, &al);
    if (s != COOT_OK) return s;
    mc->aliased = mc->aliased || al;
    for (int b = 0; b < a; ++b)
      if (overlaps(*mc->stored[a], *mc->stored[b])) return fail(COOT_ERR_ALIAS, "two stored trees overlap");
  }
  for (int i = 0; i < n_in; ++i) mc->spec.in_dtype[i] = in[i].dtype;
  return COOT_OK;
}

// The several-tree kernel (kind 7) over a checked call.
static coot_status run_multi(MultiCall& mc, const coot_mat* in, int n_in, double* out_dev, void* ws, size_t ws_bytes,
                             void* stream) {
  KernelSpec& spec = mc.spec;
  const int64_t n = n_elem(in[0]);
  if (mc.total_heads > 0) {
    if (out_dev == nullptr) return fail(COOT_ERR_INVALID_ARG, "result pointer is NULL");
    if (n == 0) return empty_heads(out_dev, spec.tree_heads, spec.n_trees, stream);
    if (ws == nullptr || ws_bytes < COOT_WS_PARTIALS_OFF + sizeof(double) * mc.total_heads)
      return fail(COOT_ERR_WORKSPACE, "reductions need a workspace (coot_workspace_size)");
  } else if (n == 0) {
    return COOT_OK;
  }
  // one launch: the synthetic tree carries the inputs and the compute type
  Tree t;
  t.n_inputs = n_in;
  t.compute = mc.ts[0].compute;
  t.hash = 0;
  const View v = make_view(in, n_in, nullptr, mc.stored, mc.n_stored);
  CallInfo ci = call_info(KIND_MULTI, mc.ts[0], in, n_in, mc.n_stored ? mc.stored[0]->dtype : -1, mc.all_heads, v);
  const Launch l = heuristic(KIND_MULTI, n_in, v, &ci);
  spec.kind = KIND_MULTI;
  spec.vec = l.vec;
  spec.unroll = l.unroll;
  spec.block = l.block;
  spec.nc = !mc.aliased;
  const Compiled* c = nullptr;
  coot_status s = kernel_for(t, spec, &c);
  if (s != COOT_OK) return s;
  coot_multi_params_host mp;
  std::memset(&mp, 0, sizeof mp);
  fill_io(&mp.b, v, n_in);
  for (int k = 0, j = 0; k < spec.n_trees; ++k) {
    if (spec.tree_out[k] < 0) continue;
    mp.out[k] = const_cast<void*>(v.ptr[n_in + j]);
    mp.ld_out[k] = v.ld[n_in + j];
    ++j;
  }
  mp.b.ws = (unsigned char*)ws;
  mp.b.res = out_dev;
  const int64_t tile = tile_rows(l);
  const int64_t units = ((v.n_rows + tile - 1) / tile) * v.n_cols;
  int64_t max_grid = INT32_MAX;
  if (mc.total_heads > 0) {
    const int64_t fit = (int64_t)((ws_bytes - COOT_WS_PARTIALS_OFF) / (sizeof(double) * mc.total_heads));
    max_grid = std::min<int64_t>(COOT_MAX_GRID, fit);
  }
  return launch(c, units, max_grid, l, &mp.b, stream, &mp);
}

coot_status coot_expr_multi(const uint8_t* const* trees, const size_t* tree_lens, int n_trees, const coot_mat* in,
                            int n_in, const coot_mat* outs, const unsigned* heads, double* out_dev, void* ws,
                            size_t ws_bytes, void* stream) {
  clear_error();
  MultiCall mc;
  coot_status s = multi_check(trees, tree_lens, n_trees, in, n_in, outs, heads, COOT_HEAD_MASK, &mc);
  if (s != COOT_OK) return s;
  return run_multi(mc, in, n_in, out_dev, ws, ws_bytes, stream);
}

// Zeros into a 1 x n or n x 1 sum of an empty object (element k at
// ptr + k * stride elements; every float type's zero is all-zero bits).
static coot_status zero_sums(const coot_mat& m, void* stream) {
  const int64_t n = n_elem(m);
  if (n == 0) return COOT_OK;
  const size_t es = dtype_size(m.dtype);
  const int64_t stride = m.n_rows == 1 ? m.ld : 1;
  cudaError_t e = stride == 1 ? cudaMemsetAsync(m.ptr, 0, es * n, (cudaStream_t)stream)
                              : cudaMemset2DAsync(m.ptr, es * stride, 0, es, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
  return COOT_OK;
}

// The column / row sums of a several-tree call by the single-purpose
// kernels (kinds 2 and 3, each reading the inputs again), then the stores
// and full heads by the several-tree kernel: the route for shapes whose
// partials do not fit the workspace.  The sums come first, so they read the
// inputs before any stored tree can overwrite one.
static coot_status run_dims_split(MultiCall& mc, const coot_mat* in, int n_in, const coot_mat* colsums,
                                  const coot_mat* rowsums, double* out_dev, void* ws, size_t ws_bytes, void* stream) {
  for (int k = 0; k < mc.spec.n_trees; ++k) {
    const unsigned h = mc.spec.tree_heads[k];
    const int nk = std::max(mc.ts[k].n_inputs, 1);
    if (h & COOT_HEAD_COLSUM) {
      coot_status s = run_sum_dim(mc.ts[k], in, nk, 0, &colsums[k], ws, ws_bytes, stream);
      if (s != COOT_OK) return s;
    }
    if (h & COOT_HEAD_ROWSUM) {
      coot_status s = run_sum_dim(mc.ts[k], in, nk, 1, &rowsums[k], ws, ws_bytes, stream);
      if (s != COOT_OK) return s;
    }
  }
  // the trees with something left to do, in order (their heads keep their
  // places in out_dev: a tree without full heads adds none)
  MultiCall rest;
  int m = 0;
  for (int k = 0; k < mc.spec.n_trees; ++k) {
    const unsigned h = mc.spec.tree_heads[k] & COOT_HEAD_MASK;
    if (h == 0 && mc.spec.tree_out[k] < 0) continue;
    rest.ts[m] = mc.ts[k];
    rest.spec.tree_heads[m] = h;
    rest.spec.tree_out[m] = mc.spec.tree_out[k];
    rest.all_heads |= h;
    rest.total_heads += popcount(h);
    ++m;
  }
  if (m == 0) return COOT_OK;
  rest.spec.n_trees = m;
  rest.spec.trees = rest.ts;
  for (int i = 0; i < n_in; ++i) rest.spec.in_dtype[i] = in[i].dtype;
  for (int a = 0; a < mc.n_stored; ++a) rest.stored[a] = mc.stored[a];
  rest.n_stored = mc.n_stored;
  rest.aliased = mc.aliased;
  return run_multi(rest, in, n_in, out_dev, ws, ws_bytes, stream);
}

coot_status coot_expr_multi_dims(const uint8_t* const* trees, const size_t* tree_lens, int n_trees,
                                 const coot_mat* in, int n_in, const coot_mat* outs, const unsigned* heads,
                                 double* out_dev, const coot_mat* colsums, const coot_mat* rowsums, void* ws,
                                 size_t ws_bytes, void* stream) {
  clear_error();
  MultiCall mc;
  coot_status s = multi_check(trees, tree_lens, n_trees, in, n_in, outs, heads,
                              COOT_HEAD_MASK | COOT_HEAD_COLSUM | COOT_HEAD_ROWSUM, &mc);
  if (s != COOT_OK) return s;
  const int64_t R = in[0].n_rows, Cn = in[0].n_cols;
  // the sums' outputs: shapes, float types, no overlap with any operand,
  // stored tree or other sum
  const coot_mat* sums[8];
  int n_sums = 0, ncs = 0, nrs = 0;
  for (int k = 0; k < n_trees; ++k) {
    const std::string at = "tree " + std::to_string(k) + ": ";
    const unsigned h = mc.spec.tree_heads[k];
    for (int d = 0; d < 2; ++d) {
      if (!(h & (d == 0 ? COOT_HEAD_COLSUM : COOT_HEAD_ROWSUM))) continue;
      const coot_mat* arr = d == 0 ? colsums : rowsums;
      if (arr == nullptr || arr[k].ptr == nullptr)
        return fail(COOT_ERR_INVALID_ARG, at + (d == 0 ? "column" : "row") + " sums requested without an output");
      const coot_mat& o = arr[k];
      s = check_mat(&o, d == 0 ? "column sums" : "row sums");
      if (s != COOT_OK) return fail(s, at + coot_last_error());
      if (d == 0 ? (o.n_rows != 1 || o.n_cols != Cn) : (o.n_rows != R || o.n_cols != 1))
        return fail(COOT_ERR_SHAPE, at + (d == 0 ? "column sums must be 1 x n_cols" : "row sums must be n_rows x 1"));
      if (!is_float(o.dtype)) return fail(COOT_ERR_DTYPE, at + "sums are stored in a floating-point type");
      bool al = false;
      s = check_alias(o, in, n_in, false, &al);
      if (s != COOT_OK) return fail(s, at + coot_last_error());
      for (int a = 0; a < mc.n_stored; ++a)
        if (overlaps(o, *mc.stored[a])) return fail(COOT_ERR_ALIAS, at + "a sum overlaps a stored tree");
      for (int b = 0; b < n_sums; ++b)
        if (overlaps(o, *sums[b])) return fail(COOT_ERR_ALIAS, at + "two sums overlap");
      sums[n_sums++] = &o;
      if (d == 0) {
        mc.spec.tree_cs[k] = o.dtype;
        ++ncs;
      } else {
        mc.spec.tree_rs[k] = o.dtype;
        ++nrs;
      }
    }
  }
  if (ncs + nrs == 0) return run_multi(mc, in, n_in, out_dev, ws, ws_bytes, stream);
  if (mc.total_heads > 0 && out_dev == nullptr) return fail(COOT_ERR_INVALID_ARG, "result pointer is NULL");
  if (R == 0 || Cn == 0) {
    for (int b = 0; b < n_sums; ++b) {
      s = zero_sums(*sums[b], stream);
      if (s != COOT_OK) return s;
    }
    return mc.total_heads > 0 ? empty_heads(out_dev, mc.spec.tree_heads, n_trees, stream) : COOT_OK;
  }
  if (ws == nullptr) return fail(COOT_ERR_WORKSPACE, "sums along a dimension need a workspace (coot_workspace_size)");

  // ---- launch shape: warps on one row segment of 32 x vec x unroll rows,
  // each warp a column at a time; the 2-D view (never flattened)
  View v;
  v.n_rows = R;
  v.n_cols = Cn;
  for (int i = 0; i < n_in; ++i) {
    v.ptr[v.n] = in[i].ptr;
    v.ld[v.n] = in[i].ld;
    v.dtype[v.n] = in[i].dtype;
    ++v.n;
  }
  for (int a = 0; a < mc.n_stored; ++a) {
    v.ptr[v.n] = mc.stored[a]->ptr;
    v.ld[v.n] = mc.stored[a]->ld;
    v.dtype[v.n] = mc.stored[a]->dtype;
    ++v.n;
  }
  const int real = mc.ts[0].compute == COOT_F64 ? 8 : 4;
  Launch l;
  l.block = 256;
  l.vec = pick_vec(v);
  l.unroll = 4;
  const Launch& o = g_override[KIND_DIMS];
  if (o.block) {
    l.block = o.block;
    if (o.vec) l.vec = pick_vec(v, o.vec);
    if (o.unroll) l.unroll = o.unroll;
    l.blocks_per_sm = o.blocks_per_sm;
    l.split = o.split;
  }
  // no wider than the column needs
  while (l.vec > 1 && 32 * l.vec > std::max<int64_t>(R, 32)) l.vec /= 2;
  while (l.unroll > 1 && 32 * (int64_t)l.vec * (l.unroll - 1) >= R) --l.unroll;
  // at most 16 values per lane and input in flight; the next column's
  // loads are issued before the current one is computed when both columns'
  // values fit 32 registers each
  const bool own_unroll = o.block != 0 && o.unroll != 0;
  while (!own_unroll && l.unroll > 1 && l.vec * l.unroll > 16) --l.unroll;
  const bool prefetch = n_in * l.vec * l.unroll <= 32;
  // Each warp's shared memory (the kernel's COOT_WREG): its column tables
  // (summed trees x CB columns x 33 lane entries of 2 values, CB the largest
  // power of two up to 16 / trees for FP32, 8 / trees for FP64) or the row
  // pairs of its segment (2 x 32 x vec x unroll values); the block's share
  // stays within 44 KB of static shared memory.
  int cb = (real == 4 ? 16 : 8) / std::max(ncs, 1);
  for (int b = 16; b >= 1; b >>= 1)
    if (cb >= b) {
      cb = b;
      break;
    }
  cb = std::max(cb, 1);
  const size_t col_bytes = ncs > 0 ? (size_t)ncs * cb * 33 * 2 * real : 0;
  auto warp_bytes = [&](const Launch& x) {
    const size_t row_bytes = nrs > 0 ? (size_t)2 * 32 * x.vec * x.unroll * real : 0;
    return std::max(col_bytes, row_bytes);
  };
  const size_t smem_cap = 44 * 1024;
  while (l.unroll > 1 && (size_t)(l.block / 32) * warp_bytes(l) > smem_cap) --l.unroll;
  while (l.block > 64 && (size_t)(l.block / 32) * warp_bytes(l) > smem_cap) l.block -= 64;
  if ((size_t)(l.block / 32) * warp_bytes(l) > smem_cap)
    return run_dims_split(mc, in, n_in, colsums, rowsums, out_dev, ws, ws_bytes, stream);
  const int64_t seg_rows = 32 * (int64_t)l.vec * l.unroll;
  const int64_t n_seg = (R + seg_rows - 1) / seg_rows;
  mc.spec.kind = KIND_DIMS;
  mc.spec.vec = l.vec;
  mc.spec.unroll = l.unroll;
  mc.spec.block = l.block;
  mc.spec.nc = !mc.aliased;
  mc.spec.min_blocks = l.block <= 256 ? 2 : 1;
  mc.spec.prefetch = prefetch ? 1 : 0;
  Tree t;
  t.n_inputs = n_in;
  t.compute = mc.ts[0].compute;
  t.hash = 0;
  const Compiled* c = nullptr;
  s = kernel_for(t, mc.spec, &c);
  if (s != COOT_OK) return s;
  int bps = std::max(1, c->max_blocks_per_sm);
  if (l.blocks_per_sm > 0) bps = std::min(bps, l.blocks_per_sm);
  const int64_t resident = (int64_t)device().sm_count * bps;
  // column chunks: enough units for every resident block, at most 64 (the
  // row partials the workspace is sized for); among up to twice that many,
  // the count whose units fill the last wave of blocks best
  const int64_t max_chunks = std::min<int64_t>(Cn, nrs > 0 ? COOT_MAX_ROW_CHUNKS : Cn);
  int64_t n_chunk = std::max<int64_t>(1, (resident + n_seg - 1) / n_seg);
  if (l.split > 0) {
    n_chunk = l.split;
  } else {
    double best = 2.0;
    const int64_t c0 = std::min(n_chunk, max_chunks);
    for (int64_t c = c0; c <= std::min<int64_t>(2 * c0, max_chunks); ++c) {
      const int64_t u = n_seg * c;
      const double waste = (double)(((u + resident - 1) / resident) * resident - u) / (double)u;
      if (waste < best - 1e-9) {
        best = waste;
        n_chunk = c;
      }
    }
  }
  n_chunk = std::min<int64_t>(n_chunk, max_chunks);
  int64_t chunk_cols = (Cn + n_chunk - 1) / n_chunk;
  n_chunk = (Cn + chunk_cols - 1) / chunk_cols;
  // counters, partials and the workspace they need
  const int64_t units = n_seg * n_chunk;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>({resident, units, (int64_t)COOT_MAX_GRID}));
  auto round256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t head_bytes = round256(sizeof(double) * (size_t)grid * (size_t)mc.total_heads);
  const size_t cpart = COOT_WS_PARTIALS_OFF + head_bytes;
  const size_t cbytes = n_seg > 1 ? (size_t)ncs * 2 * (size_t)Cn * (size_t)n_seg * real : 0;
  const size_t rpart = cpart + round256(cbytes);
  auto rbytes = [&](int64_t nc) { return nc > 1 ? (size_t)nrs * 2 * (size_t)nc * (size_t)R * real : (size_t)0; };
  while (n_chunk > 1 && rpart + rbytes(n_chunk) > ws_bytes) {
    // fewer chunks: fewer row partials
    n_chunk = std::max<int64_t>(1, n_chunk / 2);
    chunk_cols = (Cn + n_chunk - 1) / n_chunk;
    n_chunk = (Cn + chunk_cols - 1) / chunk_cols;
  }
  const int64_t counters = (ncs > 0 && n_seg > 1 ? Cn : 0) + (nrs > 0 && n_chunk > 1 ? n_seg : 0);
  if (rpart + rbytes(n_chunk) > ws_bytes || counters > COOT_WS_MAX_COUNTERS)
    return run_dims_split(mc, in, n_in, colsums, rowsums, out_dev, ws, ws_bytes, stream);
  coot_dims_params_host dp;
  std::memset(&dp, 0, sizeof dp);
  fill_io(&dp.b, v, n_in);
  for (int k = 0, j = 0; k < n_trees; ++k) {
    if (mc.spec.tree_out[k] >= 0) {
      dp.out[k] = const_cast<void*>(v.ptr[n_in + j]);
      dp.ld_out[k] = v.ld[n_in + j];
      ++j;
    }
    if (mc.spec.tree_cs[k] >= 0) {
      dp.cs[k] = colsums[k].ptr;
      dp.ld_cs[k] = colsums[k].ld;  // 1 x n_cols: element j at j * ld
    }
    if (mc.spec.tree_rs[k] >= 0) dp.rs[k] = rowsums[k].ptr;
  }
  dp.b.ws = (unsigned char*)ws;
  dp.b.res = out_dev;
  dp.b.split = n_chunk;
  dp.n_seg = n_seg;
  dp.n_chunk = n_chunk;
  dp.chunk_cols = chunk_cols;
  dp.cpart = (int64_t)cpart;
  dp.rpart = (int64_t)rpart;
  return launch(c, units, grid, l, &dp.b, stream, &dp);
}

coot_status coot_accu(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, double* out_dev, void* ws,
                      size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  return run_map_reduce(o.t, o.in, o.n, COOT_HEAD_SUM, nullptr, out_dev, ws, ws_bytes, stream);
}

coot_status coot_minmax(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, double* out_dev, void* ws,
                        size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  return run_map_reduce(o.t, o.in, o.n, COOT_HEAD_MIN | COOT_HEAD_MAX, nullptr, out_dev, ws, ws_bytes, stream);
}

coot_status coot_norm(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, int p, double* out_dev,
                      void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  const bool is_vec = in[0].n_rows == 1 || in[0].n_cols == 1 || n_elem(in[0]) == 0;
  unsigned head;
  if (p == COOT_NORM_FRO || (p == 2 && is_vec)) {
    head = COOT_HEAD_NORM2;
  } else if (p == 2) {
    return fail(COOT_ERR_UNSUPPORTED, "norm(A, 2) of a matrix is the spectral norm (needs an SVD)");
  } else if (p == 1 || p == COOT_NORM_INF || p == COOT_NORM_NEG_INF) {
    if (!is_vec) return fail(COOT_ERR_UNSUPPORTED, "norm p = 1 / inf / -inf is implemented for vectors");
    head = p == 1 ? COOT_HEAD_SUMABS : (p == COOT_NORM_INF ? COOT_HEAD_MAXABS : COOT_HEAD_MINABS);
  } else {
    return fail(COOT_ERR_INVALID_ARG, "p must be 1, 2, COOT_NORM_INF, COOT_NORM_NEG_INF or COOT_NORM_FRO");
  }
  return run_map_reduce(o.t, o.in, o.n, head, nullptr, out_dev, ws, ws_bytes, stream);
}

coot_status coot_sum_dim(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, int dim, const coot_mat* out,
                         void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  return run_sum_dim(o.t, o.in, o.n, dim, out, ws, ws_bytes, stream);
}

coot_status coot_submat(const coot_mat* m, int64_t r0, int64_t c0, int64_t r1, int64_t c1, coot_mat* view) {
  clear_error();
  coot_status s = check_mat(m, "matrix");
  if (s != COOT_OK) return s;
  if (view == nullptr) return fail(COOT_ERR_INVALID_ARG, "view is NULL");
  if (r0 < 0 || c0 < 0 || r1 < r0 || c1 < c0 || r1 >= m->n_rows || c1 >= m->n_cols)
    return fail(COOT_ERR_SHAPE, "submatrix bounds outside the matrix");
  coot_mat v = *m;
  v.ptr = (char*)m->ptr + (r0 + c0 * m->ld) * dtype_size(m->dtype);
  v.n_rows = r1 - r0 + 1;
  v.n_cols = c1 - c0 + 1;
  *view = v;
  return COOT_OK;
}

coot_status coot_diag(const coot_mat* m, int64_t k, coot_mat* view) {
  clear_error();
  coot_status s = check_mat(m, "matrix");
  if (s != COOT_OK) return s;
  if (view == nullptr) return fail(COOT_ERR_INVALID_ARG, "view is NULL");
  const int64_t r0 = k < 0 ? -k : 0, c0 = k > 0 ? k : 0;
  if (r0 >= m->n_rows || c0 >= m->n_cols) return fail(COOT_ERR_SHAPE, "diagonal outside the matrix");
  coot_mat v = *m;
  v.ptr = (char*)m->ptr + (r0 + c0 * m->ld) * dtype_size(m->dtype);
  v.n_rows = 1;
  v.n_cols = std::min(m->n_rows - r0, m->n_cols - c0);
  v.ld = m->ld + 1;  // element j of the diagonal is (r0 + j, c0 + j)
  *view = v;
  return COOT_OK;
}

coot_status coot_stats_dim(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, int dim, unsigned stats,
                           int norm_type, const coot_mat* out, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  return run_stats_dim(o.t, o.in, o.n, dim, stats, norm_type, out, ws, ws_bytes, stream);
}

coot_status coot_all_any(const uint8_t* tree, size_t len, const coot_mat* in, int n_in, double* out_dev, void* ws,
                         size_t ws_bytes, void* stream) {
  clear_error();
  Operands o;
  coot_status s = check_operands(tree, len, in, n_in, &o);
  if (s != COOT_OK) return s;
  return run_map_reduce(o.t, o.in, o.n, COOT_HEAD_ALL | COOT_HEAD_ANY, nullptr, out_dev, ws, ws_bytes, stream);
}

// ------------------------------------------------------------ batched evaluation

struct WorkUnit {
  int32_t item, col0, n_cols, pad;
};
static_assert(sizeof(coot_batch_item) == 14 * 8, "coot_batch_item layout");
static_assert(sizeof(WorkUnit) == 16, "work unit layout");

// Columns of one matrix in one work unit (one block): about
// COOT_BATCH_UNIT elements, whole columns.
static int64_t cols_per_unit(int64_t n_rows) {
  const int64_t target = COOT_BATCH_UNIT;
  if (n_rows <= 0) return target;
  int64_t k = std::max<int64_t>(1, target / n_rows);
  // keep col0 * n_rows a multiple of 4 elements, so that a unit of a
  // 16-byte aligned matrix starts 16-byte aligned (vector accesses)
  const int64_t m = n_rows % 4 == 0 ? 1 : (n_rows % 2 == 0 ? 2 : 4);
  if (k >= m) k -= k % m;
  return k;
}

coot_status coot_batch_plan_size(const coot_batch_item* items, int n_items, size_t* bytes, int64_t* n_work) {
  clear_error();
  if ((items == nullptr && n_items > 0) || n_items < 0 || bytes == nullptr)
    return fail(COOT_ERR_INVALID_ARG, "bad batch");
  int64_t w = 0;
  for (int i = 0; i < n_items; ++i) {
    if (items[i].n_rows < 0 || items[i].n_cols < 0) return fail(COOT_ERR_INVALID_ARG, "negative size in batch");
    const int64_t k = cols_per_unit(items[i].n_rows);
    w += (items[i].n_cols + k - 1) / k;
  }
  *bytes = sizeof(coot_batch_item) * (size_t)n_items + sizeof(WorkUnit) * (size_t)w;
  if (n_work) *n_work = w;
  return COOT_OK;
}

coot_status coot_batch_plan_build(const coot_batch_item* items, int n_items, int n_inputs, void* plan_host,
                                  size_t plan_bytes) {
  clear_error();
  if (n_inputs < 1 || n_inputs > 4) return fail(COOT_ERR_INVALID_ARG, "n_inputs must be 1..4");
  size_t need = 0;
  int64_t n_work = 0;
  coot_status s = coot_batch_plan_size(items, n_items, &need, &n_work);
  if (s != COOT_OK) return s;
  if (plan_host == nullptr || plan_bytes < need) return fail(COOT_ERR_INVALID_ARG, "plan buffer too small");
  for (int i = 0; i < n_items; ++i) {
    const coot_batch_item& it = items[i];
    const std::string at = "batch item " + std::to_string(i) + ": ";
    if (it.n_rows > INT32_MAX || it.n_cols > INT32_MAX) return fail(COOT_ERR_INVALID_ARG, at + "too large");
    const bool empty = it.n_rows == 0 || it.n_cols == 0;
    for (int k = 0; k < n_inputs; ++k) {
      if (it.in[k] == nullptr && !empty) return fail(COOT_ERR_INVALID_ARG, at + "input " + std::to_string(k) + " is NULL");
      if (it.ld_in[k] < std::max<int64_t>(it.n_rows, 1)) return fail(COOT_ERR_INVALID_ARG, at + "ld < n_rows");
    }
    if (it.out && it.ld_out < std::max<int64_t>(it.n_rows, 1)) return fail(COOT_ERR_INVALID_ARG, at + "ld_out < n_rows");
    if (it.colsum && it.ld_colsum < 1) return fail(COOT_ERR_INVALID_ARG, at + "ld_colsum < 1");
  }
  std::memcpy(plan_host, items, sizeof(coot_batch_item) * (size_t)n_items);
  WorkUnit* w = reinterpret_cast<WorkUnit*>(static_cast<char*>(plan_host) + sizeof(coot_batch_item) * (size_t)n_items);
  for (int i = 0; i < n_items; ++i) {
    const int64_t k = cols_per_unit(items[i].n_rows);
    for (int64_t c = 0; c < items[i].n_cols; c += k) {
      *w++ = WorkUnit{i, (int32_t)c, (int32_t)std::min<int64_t>(k, items[i].n_cols - c), 0};
    }
  }
  return COOT_OK;
}

coot_status coot_expr_eval_batched(const uint8_t* tree, size_t len, const int32_t* in_dtypes, int32_t out_dtype,
                                   int32_t colsum_dtype, const void* plan_dev, int n_items, int64_t n_work,
                                   void* stream) {
  clear_error();
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  canonical_in_place(&t);
  if (in_dtypes == nullptr) return fail(COOT_ERR_INVALID_ARG, "in_dtypes is NULL");
  for (int i = 0; i < t.n_inputs; ++i)
    if (dtype_size(in_dtypes[i]) == 0) return fail(COOT_ERR_DTYPE, "unknown input dtype");
  if (dtype_size(out_dtype) == 0) return fail(COOT_ERR_DTYPE, "unknown output dtype");
  if (colsum_dtype != COOT_F32 && colsum_dtype != COOT_F64)
    return fail(COOT_ERR_DTYPE, "column sums are stored as FP32 or FP64");
  if (n_items < 0 || n_work < 0) return fail(COOT_ERR_INVALID_ARG, "negative batch size");
  if (n_work == 0) return COOT_OK;
  if (plan_dev == nullptr) return fail(COOT_ERR_INVALID_ARG, "plan is NULL");
  KernelSpec spec;
  spec.kind = KIND_BATCHED;
  for (int i = 0; i < t.n_inputs; ++i) spec.in_dtype[i] = in_dtypes[i];
  spec.out_dtype = out_dtype;
  spec.store = true;
  spec.vec = 4;
  spec.unroll = 2;
  spec.block = 224;  // consumer threads; the launch adds the producer warp
  // Shared memory: two stages of COOT_BATCH_UNIT elements per input, each
  // with the unit's values when they cannot overwrite input 0 in place, a
  // 128-byte unit header and two mbarriers, plus the consumers' mbarrier
  // (at most 2 x (4 x 2048 x 8 B + 16 KB) + 16 B, always within the 227 KB
  // of a block)
  const int real = t.compute == COOT_F64 ? 8 : 4;
  size_t buf = 0;
  for (int i = 0; i < t.n_inputs; ++i) buf += (size_t)COOT_BATCH_UNIT * (size_t)dtype_size(in_dtypes[i]);
  const size_t vals = dtype_size(in_dtypes[0]) == real ? 0 : (size_t)COOT_BATCH_UNIT * (size_t)real;
  const size_t smem = 2 * (buf + vals + sizeof(coot_batch_item) + 16 + 2 * 8) + 16;
  if (smem > 227u * 1024u) return fail(COOT_ERR_UNSUPPORTED, "batched: two units of the inputs exceed shared memory");
  // blocks per SM: as many as their shared memory allows (228 KB per SM, 1 KB
  // of it reserved per block), at most 4 (a sweep over units of 1024, 2048,
  // 4096 and 8192 elements and 1 to 8 blocks per SM chose 2048 x 4)
  const int max_blocks = (int)std::max<size_t>(1, std::min<size_t>(4, (228u * 1024u) / (smem + 1024)));
  Launch l;
  l.blocks_per_sm = max_blocks;
  const Launch& o = g_override[KIND_BATCHED];
  if (o.block) {
    spec.block = std::min(o.block, 992);
    if (o.unroll) spec.unroll = o.unroll;
    if (o.blocks_per_sm > 0 && o.blocks_per_sm <= max_blocks) l.blocks_per_sm = o.blocks_per_sm;
  }
  l.block = spec.block + 32;
  l.unroll = spec.unroll;
  l.vec = spec.vec;
  const Compiled* c = nullptr;
  s = kernel_for(t, spec, &c);
  if (s != COOT_OK) return s;
  coot_params_host p;
  std::memset(&p, 0, sizeof p);
  p.plan = plan_dev;
  p.split = n_items;
  p.n_work = n_work;
  p.rows_per_split = colsum_dtype;
  {
    // the shared memory limit of each batched kernel, set once
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> set;
    std::lock_guard<std::mutex> lock(mu);
    auto it = set.find(c->kernel);
    if (it == set.end() || it->second < smem) {
      cudaError_t e = cudaFuncSetAttribute((const void*)c->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("shared memory size: ") + cudaGetErrorString(e));
      set[c->kernel] = smem;
    }
  }
  unsigned* status = nullptr;
  s = device_status_word(&status);
  if (s != COOT_OK) return s;
  p.res = (double*)status;
  const char* f = std::getenv("COOT_FAULT");
  if (f && std::string(f) == "batched_wait") p.n_cols = 1;  // a staged unit with no copy: its wait runs out
  return launch(c, n_work, INT32_MAX, l, &p, stream, nullptr, smem);
}

coot_status coot_dot(const coot_mat* a, const coot_mat* b, double* out_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  coot_status s = check_mat(a, "a");
  if (s != COOT_OK) return s;
  s = check_mat(b, "b");
  if (s != COOT_OK) return s;
  if (n_elem(*a) != n_elem(*b)) return fail(COOT_ERR_SHAPE, "dot needs equal element counts");
  coot_mat m[2] = {*a, *b};
  if (a->n_rows != b->n_rows || a->n_cols != b->n_cols) {
    // different shapes with equal counts: both must be dense to share one
    // column-major element order
    const bool da = a->ld == a->n_rows || a->n_cols <= 1;
    const bool db = b->ld == b->n_rows || b->n_cols <= 1;
    const bool ra = a->n_rows == 1 && a->ld != 1 && a->n_cols > 1;
    const bool rb = b->n_rows == 1 && b->ld != 1 && b->n_cols > 1;
    if (!da || !db || ra || rb)
      return fail(COOT_ERR_UNSUPPORTED, "dot of differently shaped strided operands");
    for (auto& x : m) {
      x.n_rows = n_elem(x);
      x.n_cols = 1;
      x.ld = std::max<int64_t>(x.n_rows, 1);
    }
  }
  // the tree x0 % x1 in FP32 (FP64 if either operand is FP64)
  const bool f64 = a->dtype == COOT_F64 || b->dtype == COOT_F64;
  uint8_t buf[16 + 3 * 16];
  std::memset(buf, 0, sizeof buf);
  std::memcpy(buf, "COOT", 4);
  buf[4] = 1;
  buf[6] = 3;
  buf[8] = 2;
  buf[9] = f64 ? COOT_F64 : COOT_F32;
  buf[16 + 16] = COOT_OP_INPUT;
  buf[16 + 16 + 2] = 1;
  buf[16 + 32] = COOT_OP_MUL;
  buf[16 + 32 + 4] = 1;
  Tree t;
  s = parse_tree(buf, sizeof buf, &t);
  if (s != COOT_OK) return s;
  if (!canonical_enabled()) return run_map_reduce(t, m, 2, COOT_HEAD_SUM, nullptr, out_dev, ws, ws_bytes, stream);
  // dot(x, x): one operand, read once
  const int alias[2] = {0, (m[1].ptr == m[0].ptr && m[1].dtype == m[0].dtype && m[1].ld == m[0].ld &&
                           m[1].n_rows == m[0].n_rows) ? 0 : 1};
  Tree c;
  std::vector<int> kept;
  canonicalize(t, alias, &c, &kept, false);
  coot_mat mk[2];
  for (size_t k = 0; k < kept.size(); ++k) mk[k] = m[kept[k]];
  return run_map_reduce(c, mk, (int)kept.size(), COOT_HEAD_SUM, nullptr, out_dev, ws, ws_bytes, stream);
}

}  // extern "C"
