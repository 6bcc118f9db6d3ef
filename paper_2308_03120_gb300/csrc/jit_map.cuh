// Element-wise evaluation and full reductions (kinds 0 and 1); part of the
// device runtime embedded after jit_rt.cuh.

// ================================================================ kind 0/1: evaluation and full reductions

#if COOT_KIND == 0 || COOT_KIND == 1
extern "C" __global__ void __launch_bounds__(COOT_BLOCK) COOT_ENTRY(const __grid_constant__ coot_params p) {
  constexpr coot_i64 TILE = (coot_i64)COOT_BLOCK * COOT_VEC * COOT_UNROLL;
  const coot_i64 upc = (p.n_rows + TILE - 1) / TILE;  // tiles per column
  const coot_i64 units = upc * p.n_cols;
  typedef typename coot_st<COOT_TO>::T TO;
  coot_acc acc;
  acc.init();
  for (coot_i64 u = blockIdx.x; u < units; u += gridDim.x) {
    // (one column, the dense case: no 64-bit division per unit)
    const coot_i64 j = p.n_cols == 1 ? 0 : u / upc;
    const coot_i64 r0 = (u - j * upc) * TILE;
    if (r0 + TILE <= p.n_rows) {
      COOT_REAL xv[COOT_UNROLL][4][COOT_VEC];
#pragma unroll
      for (int k = 0; k < COOT_UNROLL; ++k)
        coot_load_vec(p, j, r0 + ((coot_i64)k * COOT_BLOCK + threadIdx.x) * COOT_VEC, xv[k]);
#pragma unroll
      for (int k = 0; k < COOT_UNROLL; ++k) {
        COOT_REAL y[COOT_VEC];
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          const COOT_REAL x[4] = {xv[k][0][v], xv[k][1][v], xv[k][2][v], xv[k][3][v]};
          y[v] = coot_f(x);
        }
        acc.add_vec<COOT_VEC>(y);
#if COOT_STORE
        coot_vstore<COOT_TO, COOT_VEC>(
            (TO*)p.out + (j * p.ld_out + r0 + ((coot_i64)k * COOT_BLOCK + threadIdx.x) * COOT_VEC), y);
#endif
      }
    } else {
      // the ragged end of a column: whole vectors where they fit (a
      // column of a strided view ends in one of these every time), then
      // single elements
#pragma unroll 1
      for (int k = 0; k < COOT_UNROLL; ++k) {
        const coot_i64 row0 = r0 + ((coot_i64)k * COOT_BLOCK + threadIdx.x) * COOT_VEC;
        if (row0 + COOT_VEC <= p.n_rows) {
          COOT_REAL xv[4][COOT_VEC];
          coot_load_vec(p, j, row0, xv);
          COOT_REAL y[COOT_VEC];
#pragma unroll
          for (int v = 0; v < COOT_VEC; ++v) {
            const COOT_REAL x[4] = {xv[0][v], xv[1][v], xv[2][v], xv[3][v]};
            y[v] = coot_f(x);
          }
          acc.add_vec<COOT_VEC>(y);
#if COOT_STORE
          coot_vstore<COOT_TO, COOT_VEC>((TO*)p.out + (j * p.ld_out + row0), y);
#endif
        } else {
#pragma unroll 1
          for (int v = 0; v < COOT_VEC; ++v) {
            const coot_i64 row = row0 + v;
            if (row < p.n_rows) {
              COOT_REAL x[4];
              coot_load_one(p, j, row, x);
              const COOT_REAL y = coot_f(x);
              acc.add(y);
#if COOT_STORE
              coot_sstore<COOT_TO>((TO*)p.out + (j * p.ld_out + row), y);
#endif
            }
          }
        }
      }
    }
  }
#if COOT_NHEADS > 0
  coot_finish_full(acc, p);
#endif
}
#endif
