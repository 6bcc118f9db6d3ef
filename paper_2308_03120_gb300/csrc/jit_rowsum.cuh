// Row sums (kind 3); part of the device runtime embedded after jit_rt.cuh.

// ================================================================ kind 3: row sums (dim = 1)

// A block is COOT_RT row threads x (COOT_BLOCK / COOT_RT) column groups and
// owns a panel of COOT_RT * COOT_VEC rows over one chunk of columns; column
// group g takes the chunk's columns g, g + CG, ... with COOT_UNROLL of them
// in flight, each thread keeping a TwoSum pair per row.  The groups are
// added in shared memory in group order as double-word numbers; with
// several chunks the chunk sums go to the workspace as double-word pairs
// and the last block of a panel to arrive adds them (group g a strided
// subset of the chunks in chunk order, then the groups in order), so the
// order is fixed and no FP64 arithmetic is needed before the final
// conversion.
#if COOT_KIND == 3
#define COOT_RT 64
#define COOT_CG (COOT_BLOCK / COOT_RT)
#define COOT_PANEL (COOT_RT * COOT_VEC)
extern "C" __global__ void __launch_bounds__(COOT_BLOCK) COOT_ENTRY(const __grid_constant__ coot_params p) {
  __shared__ COOT_REAL red_h[COOT_CG][COOT_PANEL];
  __shared__ COOT_REAL red_l[COOT_CG][COOT_PANEL];
  __shared__ int is_last;
  typedef typename coot_st<COOT_TO>::T TO;
  const int tx = threadIdx.x % COOT_RT, ty = threadIdx.x / COOT_RT;
  const coot_i64 n_panels = (p.n_rows + COOT_PANEL - 1) / COOT_PANEL;
  const coot_i64 C = p.split;                               // column chunks
  const coot_i64 Q = (p.n_cols + C - 1) / C;                // columns per chunk
  const coot_i64 units = n_panels * C;
  // chunk partials: C x n_rows high parts, then C x n_rows low parts
  COOT_REAL* part_h = (COOT_REAL*)(p.ws + COOT_WS_PARTIALS_OFF);
  COOT_REAL* part_l = part_h + C * p.n_rows;
  coot_u32* cnt = (coot_u32*)(p.ws + COOT_WS_COUNTERS_OFF);
  for (coot_i64 u = blockIdx.x; u < units; u += gridDim.x) {
    const coot_i64 chunk = u / n_panels;
    const coot_i64 panel = u - chunk * n_panels;
    const coot_i64 i0 = panel * COOT_PANEL + (coot_i64)tx * COOT_VEC;
    const coot_i64 jb = chunk * Q;
    const coot_i64 je = min(p.n_cols, jb + Q);
    COOT_REAL s[COOT_VEC], c[COOT_VEC];
#pragma unroll
    for (int v = 0; v < COOT_VEC; ++v) s[v] = c[v] = 0;
    if (panel * COOT_PANEL + COOT_PANEL <= p.n_rows) {
      coot_i64 j = jb + ty;
      for (; j + (coot_i64)(COOT_UNROLL - 1) * COOT_CG < je; j += (coot_i64)COOT_UNROLL * COOT_CG) {
        COOT_REAL xv[COOT_UNROLL][4][COOT_VEC];
#pragma unroll
        for (int k = 0; k < COOT_UNROLL; ++k) coot_load_vec(p, j + (coot_i64)k * COOT_CG, i0, xv[k]);
#pragma unroll
        for (int k = 0; k < COOT_UNROLL; ++k)
#pragma unroll
          for (int v = 0; v < COOT_VEC; ++v) {
            const COOT_REAL x[4] = {xv[k][0][v], xv[k][1][v], xv[k][2][v], xv[k][3][v]};
            coot_two_sum(s[v], c[v], coot_f(x));
          }
      }
      for (; j < je; j += COOT_CG) {
        COOT_REAL xv[4][COOT_VEC];
        coot_load_vec(p, j, i0, xv);
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          const COOT_REAL x[4] = {xv[0][v], xv[1][v], xv[2][v], xv[3][v]};
          coot_two_sum(s[v], c[v], coot_f(x));
        }
      }
    } else {
#pragma unroll 1
      for (coot_i64 j = jb + ty; j < je; j += COOT_CG) {
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          if (i0 + v < p.n_rows) {
            COOT_REAL x[4];
            coot_load_one(p, j, i0 + v, x);
            coot_two_sum(s[v], c[v], coot_f(x));
          }
        }
      }
    }
    // column groups in order -> the block's sum of each row over the chunk
#pragma unroll
    for (int v = 0; v < COOT_VEC; ++v) coot_dw_norm(s[v], c[v], red_h[ty][tx * COOT_VEC + v], red_l[ty][tx * COOT_VEC + v]);
    __syncthreads();
    COOT_REAL th[COOT_VEC], tl[COOT_VEC];
    if (ty == 0) {
#pragma unroll
      for (int v = 0; v < COOT_VEC; ++v) {
        th[v] = red_h[0][tx * COOT_VEC + v];
        tl[v] = red_l[0][tx * COOT_VEC + v];
#pragma unroll
        for (int g = 1; g < COOT_CG; ++g) coot_dw_add(th[v], tl[v], red_h[g][tx * COOT_VEC + v], red_l[g][tx * COOT_VEC + v]);
      }
    }
    if (C == 1) {
      if (ty == 0) {
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v)
          if (i0 + v < p.n_rows) ((TO*)p.out)[i0 + v] = coot_dw_store<COOT_TO>(th[v], tl[v]);
      }
      __syncthreads();  // red is rewritten by the next unit
      continue;
    }
    if (ty == 0) {
#pragma unroll
      for (int v = 0; v < COOT_VEC; ++v) {
        if (i0 + v < p.n_rows) {
          part_h[chunk * p.n_rows + i0 + v] = th[v];
          part_l[chunk * p.n_rows + i0 + v] = tl[v];
        }
      }
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(cnt + panel, 1u) == (coot_u32)(C - 1));
    __syncthreads();
    if (is_last) {
      __threadfence();
      // group g adds chunks g, g + CG, ... for its rows; then group order
      COOT_REAL gh[COOT_VEC], gl[COOT_VEC];
#pragma unroll
      for (int v = 0; v < COOT_VEC; ++v) gh[v] = gl[v] = 0;
#pragma unroll 4
      for (coot_i64 q = ty; q < C; q += COOT_CG) {
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v)
          if (i0 + v < p.n_rows)
            coot_dw_add(gh[v], gl[v], __ldcg(part_h + q * p.n_rows + i0 + v), __ldcg(part_l + q * p.n_rows + i0 + v));
      }
#pragma unroll
      for (int v = 0; v < COOT_VEC; ++v) {
        red_h[ty][tx * COOT_VEC + v] = gh[v];
        red_l[ty][tx * COOT_VEC + v] = gl[v];
      }
      __syncthreads();
      if (ty == 0) {
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          COOT_REAL wh = red_h[0][tx * COOT_VEC + v], wl = red_l[0][tx * COOT_VEC + v];
#pragma unroll
          for (int g = 1; g < COOT_CG; ++g) coot_dw_add(wh, wl, red_h[g][tx * COOT_VEC + v], red_l[g][tx * COOT_VEC + v]);
          if (i0 + v < p.n_rows) ((TO*)p.out)[i0 + v] = coot_dw_store<COOT_TO>(wh, wl);
        }
      }
      if (threadIdx.x == 0) cnt[panel] = 0u;
    }
    __syncthreads();  // red and is_last are rewritten by the next unit
  }
}
#endif
