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
// handled by one block; units hold a few thousand elements, so the cost of
// reading the unit and its matrix descriptor is spread over many loads.
struct coot_work_d {
  int item;
  int col0;
  int n_cols;
  int pad;
};

#if COOT_KIND == 4
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
// Columns of at least 32 rows: warp w of the block takes columns w, w +
// warps, ... of the unit, lanes stride down the rows, COOT_UNROLL rows per
// lane in flight, then a warp-shuffle sum.  Shorter columns: floor(32 /
// n_rows) columns side by side in one warp, summed through shared memory
// in row order.
extern "C" __global__ void __launch_bounds__(COOT_BLOCK) COOT_ENTRY(const __grid_constant__ coot_params p) {
  __shared__ COOT_REAL wbuf[COOT_WARPS][32];
  __shared__ coot_batch_item_d sit;
  __shared__ coot_work_d swk;
  typedef typename coot_st<COOT_TO>::T TO;
  const coot_batch_item_d* items = (const coot_batch_item_d*)p.plan;
  const coot_work_d* work = (const coot_work_d*)(items + p.split);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool sum64 = p.rows_per_split == 3;
  for (coot_i64 w = blockIdx.x; w < p.n_work; w += gridDim.x) {
    __syncthreads();  // the previous unit is done with sit / swk
    if (threadIdx.x == 0) {
      swk = work[w];
      sit = items[swk.item];
    }
    __syncthreads();
    // a register copy: read from shared memory, the pointers would be
    // reloaded after every store and serialise the loads
    const coot_batch_item_d it = sit;
    const coot_i64 R = it.n_rows;
    const coot_i64 c0 = swk.col0, nc = swk.n_cols;
    if (R >= 32) {
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
    } else {
      // k short columns side by side per warp: lane -> (column, row)
      const int Ri = (int)R;
      const int k = Ri > 0 ? 32 / Ri : 32;
      for (coot_i64 g0 = (coot_i64)warp * k; g0 < nc; g0 += (coot_i64)COOT_WARPS * k) {
        const int kk = (int)min((coot_i64)k, nc - g0);
        COOT_REAL y = 0;
        if (lane < kk * Ri) {
          const int cl = lane / Ri, r = lane - cl * Ri;
          const coot_i64 j = c0 + g0 + cl;
          COOT_REAL x[4];
          coot_load_item(it, j, r, x);
          y = coot_f(x);
          if (it.out) ((TO*)it.out)[j * it.ld_out + r] = coot_from_real<COOT_TO>(y);
        }
        if (it.colsum) {
          wbuf[warp][lane] = y;
          __syncwarp();
          if (lane < kk) {
            COOT_REAL t = 0, tc = 0;
            for (int r = 0; r < Ri; ++r) coot_two_sum(t, tc, wbuf[warp][lane * Ri + r]);
            COOT_REAL th, tl;
            coot_dw_norm(t, tc, th, tl);
            coot_store_colsum(it, c0 + g0 + lane, th, tl, sum64);
          }
          __syncwarp();
        }
      }
    }
  }
}
#endif
