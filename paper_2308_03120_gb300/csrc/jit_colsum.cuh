// Column sums (kind 2); part of the device runtime embedded after jit_rt.cuh.

// ================================================================ kind 2: column sums (dim = 0)

// One warp per unit u = (column j, segment s): rows [s R, min((s + 1) R,
// n_rows)) of column j with R = p.rows_per_split (a multiple of the warp
// tile), p.split segments per column.  No block-level barrier is needed;
// with several segments per column the segment sums go to the workspace and
// the last warp of a column to arrive adds them in segment order.
#if COOT_KIND == 2
extern "C" __global__ void __launch_bounds__(COOT_BLOCK) COOT_ENTRY(const __grid_constant__ coot_params p) {
  constexpr coot_i64 WT = (coot_i64)32 * COOT_VEC * COOT_UNROLL;  // rows per warp tile
  typedef typename coot_st<COOT_TO>::T TO;
  const int lane = threadIdx.x & 31;
  const coot_i64 S = p.split;
  const coot_i64 units = p.n_cols * S;
  const coot_i64 n_warps = (coot_i64)gridDim.x * COOT_WARPS;
  for (coot_i64 u = (coot_i64)blockIdx.x * COOT_WARPS + (threadIdx.x >> 5); u < units; u += n_warps) {
    const coot_i64 j = u / S;
    const coot_i64 s = u - j * S;
    const coot_i64 rb = s * p.rows_per_split;
    const coot_i64 re = min(p.n_rows, rb + p.rows_per_split);
    COOT_REAL acc = 0, accc = 0;
    coot_i64 r0 = rb;
    for (; r0 + WT <= re; r0 += WT) {
      COOT_REAL xv[COOT_UNROLL][4][COOT_VEC];
#pragma unroll
      for (int k = 0; k < COOT_UNROLL; ++k) coot_load_vec(p, j, r0 + ((coot_i64)k * 32 + lane) * COOT_VEC, xv[k]);
#pragma unroll
      for (int k = 0; k < COOT_UNROLL; ++k) {
        COOT_REAL y[COOT_VEC];
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          const COOT_REAL x[4] = {xv[k][0][v], xv[k][1][v], xv[k][2][v], xv[k][3][v]};
          y[v] = coot_f(x);
        }
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) coot_two_sum(acc, accc, y[v]);
      }
    }
#pragma unroll 1
    for (coot_i64 row = r0 + lane; row < re; row += 32) {
      COOT_REAL x[4];
      coot_load_one(p, j, row, x);
      coot_two_sum(acc, accc, coot_f(x));
    }
    COOT_REAL vh, vl;
    coot_dw_norm(acc, accc, vh, vl);
    coot_dw_warp_sum(vh, vl);
    if (lane == 0) {
      if (S == 1) {
        ((TO*)p.out)[j * p.ld_out] = coot_dw_store<COOT_TO>(vh, vl);
      } else {
        // segment partials as double-word pairs: n_cols * S high parts,
        // then n_cols * S low parts
        COOT_REAL* part_h = (COOT_REAL*)(p.ws + COOT_WS_PARTIALS_OFF);
        COOT_REAL* part_l = part_h + p.n_cols * S;
        coot_u32* cnt = (coot_u32*)(p.ws + COOT_WS_COUNTERS_OFF);
        part_h[j * S + s] = vh;
        part_l[j * S + s] = vl;
        __threadfence();
        if (atomicAdd(cnt + j, 1u) == (coot_u32)(S - 1)) {
          __threadfence();
          COOT_REAL th = 0, tl = 0;
          for (coot_i64 q = 0; q < S; ++q) coot_dw_add(th, tl, __ldcg(part_h + j * S + q), __ldcg(part_l + j * S + q));
          ((TO*)p.out)[j * p.ld_out] = coot_dw_store<COOT_TO>(th, tl);
          cnt[j] = 0u;
        }
      }
    }
  }
}
#endif
