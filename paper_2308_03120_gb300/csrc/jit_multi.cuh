// Several trees over the same operands in one pass (kind 7); part of the
// device runtime embedded after jit_rt.cuh.
//
// COOT_NT trees (1 to 4) are compiled as coot_ft0 .. coot_ft3, all over the
// same COOT_NIN inputs.  Tree t is stored when COOT_STORE_t (storage code
// COOT_TO_t, matrix mp.out[t] with leading dimension mp.ld_out[t]) and
// reduced by the heads in the mask COOT_HEADS_t.  Every input element is
// loaded once for all trees; the work division, vector accesses and ragged
// column tiles are those of the element-wise kernel (kind 0), and the heads
// of all trees are combined as one list: tree 0's heads in bit order, then
// tree 1's, and so on, into p.res.

#if COOT_KIND == 7 || COOT_KIND == 8

#define COOT_MULTI_NH(H)                                                                         \
  ((((H) >> 0) & 1) + (((H) >> 1) & 1) + (((H) >> 2) & 1) + (((H) >> 3) & 1) + (((H) >> 4) & 1) + \
   (((H) >> 5) & 1) + (((H) >> 6) & 1) + (((H) >> 7) & 1) + (((H) >> 8) & 1) + (((H) >> 9) & 1))
#define COOT_MULTI_NH_ALL \
  (COOT_MULTI_NH(COOT_HEADS_0) + COOT_MULTI_NH(COOT_HEADS_1) + COOT_MULTI_NH(COOT_HEADS_2) + COOT_MULTI_NH(COOT_HEADS_3))

// the combine rule of head k of the concatenated list
__device__ __forceinline__ unsigned coot_multi_bit(int k) {
  if (k < COOT_MULTI_NH(COOT_HEADS_0)) return coot_head_bit_of<COOT_HEADS_0>(k);
  k -= COOT_MULTI_NH(COOT_HEADS_0);
  if (k < COOT_MULTI_NH(COOT_HEADS_1)) return coot_head_bit_of<COOT_HEADS_1>(k);
  k -= COOT_MULTI_NH(COOT_HEADS_1);
  if (k < COOT_MULTI_NH(COOT_HEADS_2)) return coot_head_bit_of<COOT_HEADS_2>(k);
  k -= COOT_MULTI_NH(COOT_HEADS_2);
  return coot_head_bit_of<COOT_HEADS_3>(k);
}

// the trees' values of VEC consecutive elements: y[t][v]
__device__ __forceinline__ void coot_multi_f(const COOT_REAL (&xv)[4][COOT_VEC], COOT_REAL (&y)[4][COOT_VEC]) {
#pragma unroll
  for (int v = 0; v < COOT_VEC; ++v) {
    const COOT_REAL x[4] = {xv[0][v], xv[1][v], xv[2][v], xv[3][v]};
    y[0][v] = coot_ft0(x);
    if constexpr (COOT_NT > 1) y[1][v] = coot_ft1(x);
    if constexpr (COOT_NT > 2) y[2][v] = coot_ft2(x);
    if constexpr (COOT_NT > 3) y[3][v] = coot_ft3(x);
  }
}

#endif

#if COOT_KIND == 7
// Launch parameters (every field 8 bytes; mirrored on the host).
struct coot_multi_params {
  coot_params b;          // inputs, shape, workspace, results
  void* out[4];           // stored trees (NULL when not stored)
  coot_i64 ld_out[4];
};

extern "C" __global__ void __launch_bounds__(COOT_BLOCK) COOT_ENTRY(const __grid_constant__ coot_multi_params mp) {
  const coot_params& p = mp.b;
  constexpr coot_i64 TILE = (coot_i64)COOT_BLOCK * COOT_VEC * COOT_UNROLL;
  const coot_i64 upc = (p.n_rows + TILE - 1) / TILE;  // tiles per column
  const coot_i64 units = upc * p.n_cols;
  coot_acc_h<COOT_HEADS_0> acc0;
  coot_acc_h<COOT_HEADS_1> acc1;
  coot_acc_h<COOT_HEADS_2> acc2;
  coot_acc_h<COOT_HEADS_3> acc3;
  acc0.init();
  acc1.init();
  acc2.init();
  acc3.init();
  typedef typename coot_st<COOT_TO_0>::T TO0;
  typedef typename coot_st<COOT_TO_1>::T TO1;
  typedef typename coot_st<COOT_TO_2>::T TO2;
  typedef typename coot_st<COOT_TO_3>::T TO3;
  // tree t's values y[t] at element (row, j): stored and accumulated
#define COOT_MULTI_USE_VEC(j, row, y)                                                                     \
  {                                                                                                       \
    acc0.add_vec<COOT_VEC>(y[0]);                                                                         \
    if constexpr (COOT_STORE_0) coot_vstore<COOT_TO_0, COOT_VEC>((TO0*)mp.out[0] + ((j) * mp.ld_out[0] + (row)), y[0]); \
    if constexpr (COOT_NT > 1) {                                                                          \
      acc1.add_vec<COOT_VEC>(y[1]);                                                                       \
      if constexpr (COOT_STORE_1) coot_vstore<COOT_TO_1, COOT_VEC>((TO1*)mp.out[1] + ((j) * mp.ld_out[1] + (row)), y[1]); \
    }                                                                                                     \
    if constexpr (COOT_NT > 2) {                                                                          \
      acc2.add_vec<COOT_VEC>(y[2]);                                                                       \
      if constexpr (COOT_STORE_2) coot_vstore<COOT_TO_2, COOT_VEC>((TO2*)mp.out[2] + ((j) * mp.ld_out[2] + (row)), y[2]); \
    }                                                                                                     \
    if constexpr (COOT_NT > 3) {                                                                          \
      acc3.add_vec<COOT_VEC>(y[3]);                                                                       \
      if constexpr (COOT_STORE_3) coot_vstore<COOT_TO_3, COOT_VEC>((TO3*)mp.out[3] + ((j) * mp.ld_out[3] + (row)), y[3]); \
    }                                                                                                     \
  }
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
        COOT_REAL y[4][COOT_VEC];
        coot_multi_f(xv[k], y);
        COOT_MULTI_USE_VEC(j, r0 + ((coot_i64)k * COOT_BLOCK + threadIdx.x) * COOT_VEC, y)
      }
    } else {
      // the ragged end of a column: whole vectors where they fit, then
      // single elements
#pragma unroll 1
      for (int k = 0; k < COOT_UNROLL; ++k) {
        const coot_i64 row0 = r0 + ((coot_i64)k * COOT_BLOCK + threadIdx.x) * COOT_VEC;
        if (row0 + COOT_VEC <= p.n_rows) {
          COOT_REAL xv[4][COOT_VEC];
          coot_load_vec(p, j, row0, xv);
          COOT_REAL y[4][COOT_VEC];
          coot_multi_f(xv, y);
          COOT_MULTI_USE_VEC(j, row0, y)
        } else {
#pragma unroll 1
          for (int v = 0; v < COOT_VEC; ++v) {
            const coot_i64 row = row0 + v;
            if (row < p.n_rows) {
              COOT_REAL x[4];
              coot_load_one(p, j, row, x);
              const COOT_REAL y0 = coot_ft0(x);
              acc0.add(y0);
              if constexpr (COOT_STORE_0) coot_sstore<COOT_TO_0>((TO0*)mp.out[0] + (j * mp.ld_out[0] + row), y0);
              if constexpr (COOT_NT > 1) {
                const COOT_REAL y1 = coot_ft1(x);
                acc1.add(y1);
                if constexpr (COOT_STORE_1) coot_sstore<COOT_TO_1>((TO1*)mp.out[1] + (j * mp.ld_out[1] + row), y1);
              }
              if constexpr (COOT_NT > 2) {
                const COOT_REAL y2 = coot_ft2(x);
                acc2.add(y2);
                if constexpr (COOT_STORE_2) coot_sstore<COOT_TO_2>((TO2*)mp.out[2] + (j * mp.ld_out[2] + row), y2);
              }
              if constexpr (COOT_NT > 3) {
                const COOT_REAL y3 = coot_ft3(x);
                acc3.add(y3);
                if constexpr (COOT_STORE_3) coot_sstore<COOT_TO_3>((TO3*)mp.out[3] + (j * mp.ld_out[3] + row), y3);
              }
            }
          }
        }
      }
    }
  }
#undef COOT_MULTI_USE_VEC
#if COOT_MULTI_NH_ALL > 0
  {
    // the heads of every tree, in tree order
    COOT_REAL h[COOT_MULTI_NH_ALL], l[COOT_MULTI_NH_ALL];
    int k = 0;
    if constexpr (COOT_MULTI_NH(COOT_HEADS_0) > 0) { acc0.values(h + k, l + k); k += COOT_MULTI_NH(COOT_HEADS_0); }
    if constexpr (COOT_MULTI_NH(COOT_HEADS_1) > 0) { acc1.values(h + k, l + k); k += COOT_MULTI_NH(COOT_HEADS_1); }
    if constexpr (COOT_MULTI_NH(COOT_HEADS_2) > 0) { acc2.values(h + k, l + k); k += COOT_MULTI_NH(COOT_HEADS_2); }
    if constexpr (COOT_MULTI_NH(COOT_HEADS_3) > 0) { acc3.values(h + k, l + k); k += COOT_MULTI_NH(COOT_HEADS_3); }
    (void)k;
    coot_finish_heads<COOT_MULTI_NH_ALL>(h, l, [](int i) { return coot_multi_bit(i); }, p);
  }
#endif
}
#endif
