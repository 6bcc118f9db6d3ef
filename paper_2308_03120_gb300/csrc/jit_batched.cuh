// Batched evaluation (kind 4); part of the device runtime embedded after
// jit_rt.cuh.

// ================================================================ kind 4: batched evaluation

// One matrix of a batch (the layout of coot_batch_item in coot.h; every
// field is 8 bytes).
struct coot_batch_item_d {
  const void* in[4];
  coot_i64 ld_in[4];
  void* out;
  coot_i64 ld_out;
  void* colsum;
  coot_i64 ld_colsum;
  coot_i64 n_rows;
  coot_i64 n_cols;
};

// One unit of the work list: columns [col0, col0 + n_cols) of one matrix,
// handled by one block; units hold up to about 8K elements, so the cost of
// reading the unit and its matrix descriptor is spread over many loads.
struct coot_work_d {
  int item;
  int col0;
  int n_cols;
  int pad;
};

#if COOT_KIND == 4
// staged element values of one unit (32 KB)
#define COOT_STAGE (32768 / (int)sizeof(COOT_REAL))

__device__ __forceinline__ void coot_load_item(const coot_batch_item_d& it, coot_i64 j, coot_i64 row,
                                               COOT_REAL (&x)[4]) {
#define COOT_LOAD_B(I)                                                                    \
  if constexpr (I < COOT_NIN) {                                                           \
    constexpr int S = coot_in_code<I>::S;                                                 \
    typedef typename coot_st<S>::T T;                                                     \
    x[I] = coot_sload<S>((const T*)it.in[I] + (j * it.ld_in[I] + row));                  \
  } else {                                                                                \
    x[I] = (COOT_REAL)0;                                                                  \
  }
  COOT_LOAD_B(0)
  COOT_LOAD_B(1)
  COOT_LOAD_B(2)
  COOT_LOAD_B(3)
#undef COOT_LOAD_B
}

// element e of the flat (dense) range starting at element b
__device__ __forceinline__ void coot_load_flat(const coot_batch_item_d& it, coot_i64 e, COOT_REAL (&x)[4]) {
#define COOT_LOAD_F(I)                                                                    \
  if constexpr (I < COOT_NIN) {                                                           \
    constexpr int S = coot_in_code<I>::S;                                                 \
    typedef typename coot_st<S>::T T;                                                     \
    x[I] = coot_sload<S>((const T*)it.in[I] + e);                                         \
  } else {                                                                                \
    x[I] = (COOT_REAL)0;                                                                  \
  }
  COOT_LOAD_F(0)
  COOT_LOAD_F(1)
  COOT_LOAD_F(2)
  COOT_LOAD_F(3)
#undef COOT_LOAD_F
}

// COOT_VEC consecutive elements of every input from element e of the
// (shifted, dense) run; e is a multiple of COOT_VEC and the run is aligned
__device__ __forceinline__ void coot_load_flat_vec(const coot_batch_item_d& it, int e,
                                                   COOT_REAL (&x)[4][COOT_VEC]) {
#define COOT_LOAD_V(I)                                                                    \
  if constexpr (I < COOT_NIN) {                                                           \
    constexpr int S = coot_in_code<I>::S;                                                 \
    typedef typename coot_st<S>::T T;                                                     \
    coot_vload<S, COOT_VEC>((const T*)it.in[I] + e, x[I]);                                \
  } else {                                                                                \
    _Pragma("unroll") for (int v = 0; v < COOT_VEC; ++v) x[I][v] = (COOT_REAL)0;          \
  }
  COOT_LOAD_V(0)
  COOT_LOAD_V(1)
  COOT_LOAD_V(2)
  COOT_LOAD_V(3)
#undef COOT_LOAD_V
}

template <int S>
__device__ __forceinline__ bool coot_aligned16(const void* p) {
  return ((unsigned long long)p & 15ull) == 0;
}

// a column sum held as a double-word pair (h, l), stored in FP64 or FP32
__device__ __forceinline__ void coot_store_colsum(const coot_batch_item_d& it, coot_i64 j, COOT_REAL h, COOT_REAL l,
                                                  bool sum64) {
  if (sum64) {
    ((double*)it.colsum)[j * it.ld_colsum] = coot_dw_store<3>(h, l);
  } else {
    ((float*)it.colsum)[j * it.ld_colsum] = coot_dw_store<0>(h, l);
  }
}

// p.plan: items (p.split of them) followed by the work list (p.n_work units).
// COOT_TO is the storage code of the element-wise outputs; the column sums
// are stored in the storage code given by p.rows_per_split (0 FP32, 3 FP64).
//
// Dense units (every operand's ld equals n_rows, so the unit's columns are
// one contiguous run) that fit the stage: every thread streams the run
// flat, COOT_UNROLL elements per input in flight, writes the values and
// keeps them in shared memory; the column sums are then taken from shared
// memory (a warp per column with a double-word shuffle sum for columns of
// at least 32 rows, a thread per column below that), each in a fixed order.
// Other units: warp w of the block takes columns w, w + warps, ...; lanes
// stride down the rows.
// at least 1024 threads resident per SM: the per-unit barriers leave
// latency that only other blocks can hide
extern "C" __global__ void __launch_bounds__(COOT_BLOCK, (COOT_BLOCK < 1024 ? 1024 / COOT_BLOCK : 1))
    COOT_ENTRY(const __grid_constant__ coot_params p) {
  __shared__ COOT_REAL stage[COOT_STAGE];
  __shared__ coot_batch_item_d sit;
  __shared__ coot_work_d swk;
  typedef typename coot_st<COOT_TO>::T TO;
  const coot_batch_item_d* items = (const coot_batch_item_d*)p.plan;
  const coot_work_d* work = (const coot_work_d*)(items + p.split);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool sum64 = p.rows_per_split == 3;
  for (coot_i64 w = blockIdx.x; w < p.n_work; w += gridDim.x) {
    __syncthreads();  // the previous unit is done with sit, swk and stage
    if (threadIdx.x == 0) {
      swk = work[w];
      sit = items[swk.item];
    }
    __syncthreads();
    // a register copy: read from shared memory, the pointers would be
    // reloaded after every store and serialise the loads
    coot_batch_item_d it = sit;
    const coot_i64 R = it.n_rows;
    const coot_i64 c0 = swk.col0, nc = swk.n_cols;
    bool dense = (it.out == nullptr || it.ld_out == R);
#pragma unroll
    for (int k = 0; k < COOT_NIN; ++k) dense = dense && it.ld_in[k] == R;
    const coot_i64 n = nc * R;
    if (dense && n <= COOT_STAGE) {
      // the unit's run starts at element b of every operand
      const coot_i64 b = c0 * R;
#define COOT_SHIFT(I)                                                                                   \
  if constexpr (I < COOT_NIN) it.in[I] = (const typename coot_st<coot_in_code<I>::S>::T*)it.in[I] + b;
      COOT_SHIFT(0)
      COOT_SHIFT(1)
      COOT_SHIFT(2)
      COOT_SHIFT(3)
#undef COOT_SHIFT
      TO* out = it.out ? (TO*)it.out + b : (TO*)nullptr;
      const int ni = (int)n;
      // vectors of COOT_VEC elements when every operand's run is 16-byte
      // aligned (the plan cuts units so that it usually is)
      bool va = out == nullptr || coot_aligned16<0>(out);
#pragma unroll
      for (int k = 0; k < COOT_NIN; ++k) va = va && coot_aligned16<0>(it.in[k]);
      const int nv = va ? ni / COOT_VEC : 0;
      for (int v0 = 0; v0 < nv; v0 += COOT_BLOCK * COOT_UNROLL) {
        COOT_REAL xv[COOT_UNROLL][4][COOT_VEC];
#pragma unroll
        for (int q = 0; q < COOT_UNROLL; ++q) {
          const int v = v0 + q * COOT_BLOCK + (int)threadIdx.x;
          if (v < nv) coot_load_flat_vec(it, v * COOT_VEC, xv[q]);
        }
#pragma unroll
        for (int q = 0; q < COOT_UNROLL; ++q) {
          const int v = v0 + q * COOT_BLOCK + (int)threadIdx.x;
          if (v < nv) {
            COOT_REAL y[COOT_VEC];
#pragma unroll
            for (int k = 0; k < COOT_VEC; ++k) {
              const COOT_REAL x[4] = {xv[q][0][k], xv[q][1][k], xv[q][2][k], xv[q][3][k]};
              y[k] = coot_f(x);
              stage[v * COOT_VEC + k] = y[k];
            }
            if (out) coot_vstore<COOT_TO, COOT_VEC>(out + v * COOT_VEC, y);
          }
        }
      }
      for (int e = nv * COOT_VEC + (int)threadIdx.x; e < ni; e += COOT_BLOCK) {
        COOT_REAL x[4];
        coot_load_flat(it, e, x);
        const COOT_REAL y = coot_f(x);
        if (out) out[e] = coot_from_real<COOT_TO>(y);
        stage[e] = y;
      }
      if (it.colsum) {
        __syncthreads();
        const int Ri = (int)R, nci = (int)nc;
        if (Ri >= 32) {
          for (int cj = warp; cj < nci; cj += COOT_WARPS) {
            COOT_REAL s = 0, c = 0;
            for (int r = lane; r < Ri; r += 32) coot_two_sum(s, c, stage[cj * Ri + r]);
            COOT_REAL vh, vl;
            coot_dw_norm(s, c, vh, vl);
            coot_dw_warp_sum(vh, vl);
            if (lane == 0) coot_store_colsum(it, c0 + cj, vh, vl, sum64);
          }
        } else {
          for (int cj = threadIdx.x; cj < nci; cj += COOT_BLOCK) {
            COOT_REAL s = 0, c = 0;
            for (int r = 0; r < Ri; ++r) coot_two_sum(s, c, stage[cj * Ri + r]);
            COOT_REAL vh, vl;
            coot_dw_norm(s, c, vh, vl);
            coot_store_colsum(it, c0 + cj, vh, vl, sum64);
          }
        }
      }
      continue;
    }
    // strided operands or a unit larger than the stage: a warp per column
    for (coot_i64 cj = warp; cj < nc; cj += COOT_WARPS) {
      const coot_i64 j = c0 + cj;
      COOT_REAL s = 0, c = 0;
      for (coot_i64 r0 = 0; r0 < R; r0 += 32 * COOT_UNROLL) {
        COOT_REAL xv[COOT_UNROLL][4];
#pragma unroll
        for (int q = 0; q < COOT_UNROLL; ++q) {
          const coot_i64 r = r0 + 32 * q + lane;
          if (r < R) coot_load_item(it, j, r, xv[q]);
        }
#pragma unroll
        for (int q = 0; q < COOT_UNROLL; ++q) {
          const coot_i64 r = r0 + 32 * q + lane;
          if (r < R) {
            const COOT_REAL y = coot_f(xv[q]);
            if (it.out) ((TO*)it.out)[j * it.ld_out + r] = coot_from_real<COOT_TO>(y);
            coot_two_sum(s, c, y);
          }
        }
      }
      if (it.colsum) {
        COOT_REAL vh, vl;
        coot_dw_norm(s, c, vh, vl);
        coot_dw_warp_sum(vh, vl);
        if (lane == 0) coot_store_colsum(it, j, vh, vl, sum64);
      }
    }
  }
}
#endif
