// Several trees with column and row sums in the same pass (kind 8); part of
// the device runtime embedded after jit_rt.cuh and jit_multi.cuh.
//
// The trees, stored outputs and full heads are those of the several-tree
// kernel (COOT_NT, COOT_STORE_t, COOT_TO_t, COOT_HEADS_t); in addition tree t
// may have its column sums (COOT_CS_t, stored in code COOT_TCS_t into a
// 1 x n_cols matrix) and its row sums (COOT_RS_t, code COOT_TRS_t, into an
// n_rows x 1 vector) formed from the values as they are computed, so a sum
// along a dimension (Table 6) costs no second pass over a stored result.
//
// Work division.  The matrix is cut into row segments of COOT_SEG =
// 32 * COOT_VEC * COOT_UNROLL rows and column chunks of dp.chunk_cols
// columns; unit u = (chunk u / n_seg, segment u % n_seg) is one block's.
// Warp w of the block takes the chunk's columns w, w + warps, ...: for each
// column every lane loads COOT_UNROLL vectors of COOT_VEC rows of every input
// (32 lanes cover 32 * COOT_VEC consecutive rows per vector, so each warp
// load is one contiguous run of the column), evaluates the trees, stores
// them, feeds the full heads, and adds each value
//   * to the lane's running pair for that row (TwoSum), and
//   * to the lane's pair for the column (TwoSum), which a warp shuffle tree
//     of double-word additions turns into the column's sum over the segment.
// With one segment per column that is the column sum; otherwise the
// segment's partial goes to the workspace and the last warp to finish a
// column (arrival counter per column) adds the column's partials in segment
// order.  At the end of a unit the warps' row pairs are added in warp order
// in shared memory; with one chunk that is the row sum, otherwise the
// chunk's partial goes to the workspace and the last block to finish a
// segment (counter per segment) adds the chunk partials in chunk order.
// Every order is fixed, so the results do not depend on timing.
//
// Workspace: the full heads' block partials at COOT_WS_PARTIALS_OFF (as in
// every kernel with heads), the column partials at byte dp.cpart (high
// parts, then low parts, per summed tree: n_cols x n_seg each) and the row
// partials at byte dp.rpart (per summed tree: n_chunk x n_rows high parts,
// then low parts); column counters at COOT_WS_COUNTERS_OFF, then one
// counter per segment.  The last arrival resets every counter it used.

#if COOT_KIND == 8
struct coot_dims_params {
  coot_params b;          // inputs, shape, workspace, results
  void* out[4];           // stored trees (NULL when not stored)
  coot_i64 ld_out[4];
  void* cs[4];            // column sums of tree t: element j at cs[t] + j * ld_cs[t]
  coot_i64 ld_cs[4];
  void* rs[4];            // row sums of tree t (contiguous)
  coot_i64 n_seg;         // row segments of COOT_SEG rows
  coot_i64 n_chunk;       // column chunks
  coot_i64 chunk_cols;    // columns per chunk
  coot_i64 cpart;         // byte offset of the column partials in the workspace
  coot_i64 rpart;         // byte offset of the row partials in the workspace
};

#define COOT_SEG (32 * COOT_VEC * COOT_UNROLL)
#ifndef COOT_MINB
#define COOT_MINB 1
#endif
#define COOT_NCS (COOT_CS_0 + COOT_CS_1 + COOT_CS_2 + COOT_CS_3)
#define COOT_NRS (COOT_RS_0 + COOT_RS_1 + COOT_RS_2 + COOT_RS_3)

// index of tree t among the trees with column (row) sums
template <int T> struct coot_cs_slot {
  static constexpr int K = (T > 0 ? COOT_CS_0 : 0) + (T > 1 ? COOT_CS_1 : 0) + (T > 2 ? COOT_CS_2 : 0);
};
template <int T> struct coot_rs_slot {
  static constexpr int K = (T > 0 ? COOT_RS_0 : 0) + (T > 1 ? COOT_RS_1 : 0) + (T > 2 ? COOT_RS_2 : 0);
};
template <int T> struct coot_tree_flags;
template <> struct coot_tree_flags<0> {
  static constexpr bool CS = COOT_CS_0, RS = COOT_RS_0, ST = COOT_STORE_0;
  static constexpr int TCS = COOT_TCS_0, TRS = COOT_TRS_0, TO = COOT_TO_0;
};
template <> struct coot_tree_flags<1> {
  static constexpr bool CS = COOT_CS_1, RS = COOT_RS_1, ST = COOT_STORE_1;
  static constexpr int TCS = COOT_TCS_1, TRS = COOT_TRS_1, TO = COOT_TO_1;
};
template <> struct coot_tree_flags<2> {
  static constexpr bool CS = COOT_CS_2, RS = COOT_RS_2, ST = COOT_STORE_2;
  static constexpr int TCS = COOT_TCS_2, TRS = COOT_TRS_2, TO = COOT_TO_2;
};
template <> struct coot_tree_flags<3> {
  static constexpr bool CS = COOT_CS_3, RS = COOT_RS_3, ST = COOT_STORE_3;
  static constexpr int TCS = COOT_TCS_3, TRS = COOT_TRS_3, TO = COOT_TO_3;
};

// The warp's sum of double-word numbers, valid in every lane (xor-shuffle
// tree of fixed shape; the double-word addition is commutative -- TwoSum's
// pair does not depend on the order of its operands -- so both lanes of an
// exchange form the same sum).
__device__ __forceinline__ void coot_dw_warp_allsum(COOT_REAL& h, COOT_REAL& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const COOT_REAL yh = __shfl_xor_sync(0xffffffffu, h, o);
    const COOT_REAL yl = __shfl_xor_sync(0xffffffffu, l, o);
    coot_dw_add(h, l, yh, yl);
  }
}

extern "C" __global__ void __launch_bounds__(COOT_BLOCK, COOT_MINB) COOT_ENTRY(const __grid_constant__ coot_dims_params dp) {
  const coot_params& p = dp.b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const coot_i64 n_seg = dp.n_seg, n_chunk = dp.n_chunk;
  const coot_i64 units = n_seg * n_chunk;
  coot_acc_h<COOT_HEADS_0> acc0;
  coot_acc_h<COOT_HEADS_1> acc1;
  coot_acc_h<COOT_HEADS_2> acc2;
  coot_acc_h<COOT_HEADS_3> acc3;
  acc0.init();
  acc1.init();
  acc2.init();
  acc3.init();
#if COOT_NRS > 0
  // the warps' row pairs of one summed tree, added in warp order
  __shared__ __align__(16) COOT_REAL red_h[COOT_WARPS][COOT_SEG];
  __shared__ __align__(16) COOT_REAL red_l[COOT_WARPS][COOT_SEG];
  __shared__ int is_last;
#endif
  // this lane's row pairs: rows (k * 32 + lane) * VEC + v of the segment
  // (declared without row sums too: the code that does not use them still
  // names them)
  COOT_REAL rsum[COOT_NRS > 0 ? COOT_NRS : 1][COOT_UNROLL][COOT_VEC];
  COOT_REAL rcmp[COOT_NRS > 0 ? COOT_NRS : 1][COOT_UNROLL][COOT_VEC];
  coot_u32* cnt_col = (coot_u32*)(p.ws + COOT_WS_COUNTERS_OFF);
  coot_u32* cnt_seg = cnt_col + ((COOT_NCS > 0 && n_seg > 1) ? p.n_cols : 0);

  for (coot_i64 u = blockIdx.x; u < units; u += gridDim.x) {
    const coot_i64 chunk = u / n_seg;
    const coot_i64 seg = u - chunk * n_seg;
    const coot_i64 rb = seg * COOT_SEG;
    const coot_i64 jb = chunk * dp.chunk_cols;
    const coot_i64 je = min(p.n_cols, jb + dp.chunk_cols);
    const bool whole = rb + COOT_SEG <= p.n_rows;
#if COOT_NRS > 0
#pragma unroll
    for (int t = 0; t < COOT_NRS; ++t)
#pragma unroll
      for (int k = 0; k < COOT_UNROLL; ++k)
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) rsum[t][k][v] = rcmp[t][k][v] = (COOT_REAL)0;
#endif
    for (coot_i64 j = jb + warp; j < je; j += COOT_WARPS) {
      COOT_REAL csum[COOT_NCS > 0 ? COOT_NCS : 1], ccmp[COOT_NCS > 0 ? COOT_NCS : 1];
#pragma unroll
      for (int t = 0; t < (COOT_NCS > 0 ? COOT_NCS : 1); ++t) csum[t] = ccmp[t] = (COOT_REAL)0;
      // tree T's values y at rows (k, v) of this lane: stored, reduced,
      // summed into the row and column pairs
#define COOT_DIMS_USE(TT, k, row, yv, NV)                                                                      \
  if constexpr (TT < COOT_NT) {                                                                                \
    typedef coot_tree_flags<TT> F;                                                                             \
    if constexpr (TT == 0) acc0.add_vec<NV>(yv); else if constexpr (TT == 1) acc1.add_vec<NV>(yv);              \
    else if constexpr (TT == 2) acc2.add_vec<NV>(yv); else acc3.add_vec<NV>(yv);                               \
    if constexpr (F::ST) {                                                                                    \
      typedef typename coot_st<F::TO>::T TOT;                                                                 \
      if constexpr (NV == COOT_VEC) coot_vstore<F::TO, COOT_VEC>((TOT*)dp.out[TT] + (j * dp.ld_out[TT] + (row)), yv); \
      else coot_sstore<F::TO>((TOT*)dp.out[TT] + (j * dp.ld_out[TT] + (row)), yv[0]);                          \
    }                                                                                                         \
    if constexpr (F::RS) {                                                                                    \
      _Pragma("unroll") for (int v = 0; v < NV; ++v)                                                         \
        coot_two_sum(rsum[coot_rs_slot<TT>::K][k][v + vo], rcmp[coot_rs_slot<TT>::K][k][v + vo], yv[v]);      \
    }                                                                                                         \
    if constexpr (F::CS) {                                                                                    \
      _Pragma("unroll") for (int v = 0; v < NV; ++v)                                                         \
        coot_two_sum(csum[coot_cs_slot<TT>::K], ccmp[coot_cs_slot<TT>::K], yv[v]);                            \
    }                                                                                                         \
  }
      if (whole) {
        COOT_REAL xv[COOT_UNROLL][4][COOT_VEC];
#pragma unroll
        for (int k = 0; k < COOT_UNROLL; ++k) coot_load_vec(p, j, rb + ((coot_i64)k * 32 + lane) * COOT_VEC, xv[k]);
#pragma unroll
        for (int k = 0; k < COOT_UNROLL; ++k) {
          COOT_REAL y[4][COOT_VEC];
          coot_multi_f(xv[k], y);
          const coot_i64 row = rb + ((coot_i64)k * 32 + lane) * COOT_VEC;
          constexpr int vo = 0;
          COOT_DIMS_USE(0, k, row, y[0], COOT_VEC)
          COOT_DIMS_USE(1, k, row, y[1], COOT_VEC)
          COOT_DIMS_USE(2, k, row, y[2], COOT_VEC)
          COOT_DIMS_USE(3, k, row, y[3], COOT_VEC)
        }
      } else {
        // the last, partial segment: whole vectors where they fit, then
        // single elements
#pragma unroll
        for (int k = 0; k < COOT_UNROLL; ++k) {
          const coot_i64 row0 = rb + ((coot_i64)k * 32 + lane) * COOT_VEC;
          if (row0 + COOT_VEC <= p.n_rows) {
            COOT_REAL xv[4][COOT_VEC];
            coot_load_vec(p, j, row0, xv);
            COOT_REAL y[4][COOT_VEC];
            coot_multi_f(xv, y);
            constexpr int vo = 0;
            COOT_DIMS_USE(0, k, row0, y[0], COOT_VEC)
            COOT_DIMS_USE(1, k, row0, y[1], COOT_VEC)
            COOT_DIMS_USE(2, k, row0, y[2], COOT_VEC)
            COOT_DIMS_USE(3, k, row0, y[3], COOT_VEC)
          } else {
#pragma unroll
            for (int vo = 0; vo < COOT_VEC; ++vo) {
              const coot_i64 row = row0 + vo;
              if (row < p.n_rows) {
                COOT_REAL x[4];
                coot_load_one(p, j, row, x);
                COOT_REAL y[4][1];
                y[0][0] = coot_ft0(x);
                if constexpr (COOT_NT > 1) y[1][0] = coot_ft1(x);
                if constexpr (COOT_NT > 2) y[2][0] = coot_ft2(x);
                if constexpr (COOT_NT > 3) y[3][0] = coot_ft3(x);
                COOT_DIMS_USE(0, k, row, y[0], 1)
                COOT_DIMS_USE(1, k, row, y[1], 1)
                COOT_DIMS_USE(2, k, row, y[2], 1)
                COOT_DIMS_USE(3, k, row, y[3], 1)
              }
            }
          }
        }
      }
#undef COOT_DIMS_USE
#if COOT_NCS > 0
      // the column's sum over the segment, in every lane
      COOT_REAL ch[COOT_NCS], cl[COOT_NCS];
#pragma unroll
      for (int t = 0; t < COOT_NCS; ++t) {
        coot_dw_norm(csum[t], ccmp[t], ch[t], cl[t]);
        coot_dw_warp_allsum(ch[t], cl[t]);
      }
      // column sum of tree T (summed-tree slot K) from the pair (h, l)
#define COOT_CS_STORE(TT, h, l)                                                                                \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::CS) {                                                     \
    typedef typename coot_st<coot_tree_flags<TT>::TCS>::T TCT;                                                 \
    ((TCT*)dp.cs[TT])[j * dp.ld_cs[TT]] = coot_dw_store<coot_tree_flags<TT>::TCS>(h[coot_cs_slot<TT>::K], l[coot_cs_slot<TT>::K]); \
  }
      if (n_seg == 1) {
        if (lane == 0) {
          COOT_CS_STORE(0, ch, cl)
          COOT_CS_STORE(1, ch, cl)
          COOT_CS_STORE(2, ch, cl)
          COOT_CS_STORE(3, ch, cl)
        }
      } else {
        // partials: tree slot t's high parts at [t][j][seg], then its low parts
        COOT_REAL* ph = (COOT_REAL*)(p.ws + dp.cpart);
        const coot_i64 per = p.n_cols * n_seg;
        if (lane == 0) {
#pragma unroll
          for (int t = 0; t < COOT_NCS; ++t) {
            ph[2 * t * per + j * n_seg + seg] = ch[t];
            ph[(2 * t + 1) * per + j * n_seg + seg] = cl[t];
          }
          __threadfence();
        }
        unsigned last = 0;
        if (lane == 0) last = atomicAdd(cnt_col + j, 1u) == (coot_u32)(n_seg - 1);
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
          __threadfence();
          // lane q adds segments q, q + 32, ... in order; then the fixed tree
          COOT_REAL sh[COOT_NCS], sl[COOT_NCS];
#pragma unroll
          for (int t = 0; t < COOT_NCS; ++t) {
            sh[t] = sl[t] = (COOT_REAL)0;
            for (coot_i64 q = lane; q < n_seg; q += 32)
              coot_dw_add(sh[t], sl[t], __ldcg(ph + 2 * t * per + j * n_seg + q),
                          __ldcg(ph + (2 * t + 1) * per + j * n_seg + q));
            coot_dw_warp_allsum(sh[t], sl[t]);
          }
          if (lane == 0) {
            COOT_CS_STORE(0, sh, sl)
            COOT_CS_STORE(1, sh, sl)
            COOT_CS_STORE(2, sh, sl)
            COOT_CS_STORE(3, sh, sl)
            cnt_col[j] = 0u;  // ready for the next call
          }
        }
      }
#undef COOT_CS_STORE
#endif
    }
#if COOT_NRS > 0
    // rows of the segment over the chunk: the warps' pairs added in warp
    // order, one summed tree at a time
    COOT_REAL* rph = (COOT_REAL*)(p.ws + dp.rpart);
    const coot_i64 rper = n_chunk * p.n_rows;
#define COOT_RS_TREE(TT)                                                                                       \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::RS) {                                                     \
    constexpr int K = coot_rs_slot<TT>::K;                                                                     \
    typedef typename coot_st<coot_tree_flags<TT>::TRS>::T TRT;                                                 \
    _Pragma("unroll") for (int k = 0; k < COOT_UNROLL; ++k)                                                  \
      _Pragma("unroll") for (int v = 0; v < COOT_VEC; ++v) {                                                 \
        const int r = (k * 32 + lane) * COOT_VEC + v;                                                         \
        coot_dw_norm(rsum[K][k][v], rcmp[K][k][v], red_h[warp][r], red_l[warp][r]);                          \
      }                                                                                                       \
    __syncthreads();                                                                                          \
    for (int r = threadIdx.x; r < COOT_SEG; r += COOT_BLOCK) {                                               \
      COOT_REAL h = red_h[0][r], l = red_l[0][r];                                                             \
      _Pragma("unroll") for (int w = 1; w < COOT_WARPS; ++w) coot_dw_add(h, l, red_h[w][r], red_l[w][r]);   \
      const coot_i64 row = rb + r;                                                                            \
      if (row < p.n_rows) {                                                                                   \
        if (n_chunk == 1) {                                                                                   \
          ((TRT*)dp.rs[TT])[row] = coot_dw_store<coot_tree_flags<TT>::TRS>(h, l);                               \
        } else {                                                                                              \
          rph[2 * K * rper + chunk * p.n_rows + row] = h;                                                     \
          rph[(2 * K + 1) * rper + chunk * p.n_rows + row] = l;                                               \
        }                                                                                                     \
      }                                                                                                       \
    }                                                                                                         \
    __syncthreads();                                                                                          \
  }
    COOT_RS_TREE(0)
    COOT_RS_TREE(1)
    COOT_RS_TREE(2)
    COOT_RS_TREE(3)
#undef COOT_RS_TREE
    if (n_chunk > 1) {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) is_last = atomicAdd(cnt_seg + seg, 1u) == (coot_u32)(n_chunk - 1);
      __syncthreads();
      if (is_last) {
        __threadfence();
        // the segment's rows: the chunk partials in chunk order
#define COOT_RS_LAST(TT)                                                                                       \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::RS) {                                                     \
    constexpr int K = coot_rs_slot<TT>::K;                                                                     \
    typedef typename coot_st<coot_tree_flags<TT>::TRS>::T TRT;                                                 \
    for (int r = threadIdx.x; r < COOT_SEG; r += COOT_BLOCK) {                                               \
      const coot_i64 row = rb + r;                                                                            \
      if (row < p.n_rows) {                                                                                   \
        COOT_REAL h = 0, l = 0;                                                                               \
        _Pragma("unroll 4") for (coot_i64 c = 0; c < n_chunk; ++c)                                            \
          coot_dw_add(h, l, __ldcg(rph + 2 * K * rper + c * p.n_rows + row),                                 \
                      __ldcg(rph + (2 * K + 1) * rper + c * p.n_rows + row));                                 \
        ((TRT*)dp.rs[TT])[row] = coot_dw_store<coot_tree_flags<TT>::TRS>(h, l);                                 \
      }                                                                                                       \
    }                                                                                                         \
  }
        COOT_RS_LAST(0)
        COOT_RS_LAST(1)
        COOT_RS_LAST(2)
        COOT_RS_LAST(3)
#undef COOT_RS_LAST
        if (threadIdx.x == 0) cnt_seg[seg] = 0u;  // ready for the next call
      }
      __syncthreads();  // is_last is rewritten by the next unit
    }
#endif
  }
#if COOT_MULTI_NH_ALL > 0
  {
    // the full heads of every tree, in tree order
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
