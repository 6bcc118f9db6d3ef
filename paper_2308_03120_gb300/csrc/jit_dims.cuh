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
// them, feeds the full heads, and adds each value with TwoSum (two rows per
// packed FP32-pair instruction)
//   * to the lane's running pair for that row, and
//   * to the lane's pair for the column.
// Column sums.  A lane's column pair goes to the warp's shared-memory table
// (a row of 32 lane pairs per column, COOT_CB columns per batch); once the
// batch is full, lanes add the table's rows in lane order (COOT_CB entries
// each, then a fixed xor-shuffle tree over the 32 / COOT_CB lanes of a
// column), which gives each column's sum over the segment with a few
// additions per value instead of a shuffle tree per column.  With one
// segment per column that is the column sum; otherwise the segment's
// partial goes to the workspace, and at the end of the unit (one fence per
// warp) every column of the warp counts an arrival; the last lane to arrive
// at a column adds the column's partials in segment order.
// Row sums.  At the end of a unit the warps' row pairs are added in warp
// order in shared memory; with one chunk that is the row sum, otherwise the
// chunk's partial goes to the workspace and the last block to finish a
// segment (counter per segment) adds the chunk partials in chunk order.
// A tree whose plain sum (accu) is a head and whose row (else column) sums
// are formed takes that head from the summed pairs instead of adding every
// value a third time.  Every order is fixed, so the results do not depend
// on timing.
//
// Workspace: the full heads' block partials at COOT_WS_PARTIALS_OFF (as in
// every kernel with heads), the column partials at byte dp.cpart (per summed
// tree: n_cols x n_seg high parts, then as many low parts) and the row
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
#ifndef COOT_PREFETCH
#define COOT_PREFETCH 0
#endif
#define COOT_NCS (COOT_CS_0 + COOT_CS_1 + COOT_CS_2 + COOT_CS_3)
#define COOT_NRS (COOT_RS_0 + COOT_RS_1 + COOT_RS_2 + COOT_RS_3)
#define COOT_NCS1 (COOT_NCS > 0 ? COOT_NCS : 1)
#define COOT_NRS1 (COOT_NRS > 0 ? COOT_NRS : 1)
// columns per batch of column reductions: the largest power of two up to
// 16 (FP32) or 8 (FP64) per summed tree, so every table has the same bytes
#define COOT_CB0 ((sizeof(COOT_REAL) == 4 ? 16 : 8) / COOT_NCS1)
#define COOT_CB (COOT_CB0 >= 16 ? 16 : COOT_CB0 >= 8 ? 8 : COOT_CB0 >= 4 ? 4 : COOT_CB0 >= 2 ? 2 : 1)
// values per lane and row added as packed FP32 pairs
#define COOT_PACK (!COOT_REAL_F64 && (COOT_VEC % 2 == 0))
#define COOT_RV (COOT_PACK ? COOT_VEC / 2 : COOT_VEC)
#define COOT_RSTEP (COOT_PACK ? 2 : 1)
// a table entry: a lane's column sum as {sum, compensation}
#define COOT_ENT 2
// each warp's shared memory: its column tables (COOT_CB columns x 33 lane
// entries each), or (after its columns) its row pairs of one summed tree
#define COOT_CTAB (COOT_CB * 33 * COOT_ENT)
#define COOT_WREG_C (COOT_NCS > 0 ? COOT_NCS * COOT_CTAB : 0)
#define COOT_WREG_R (COOT_NRS > 0 ? 2 * COOT_SEG : 0)
#define COOT_WREG (COOT_WREG_C > COOT_WREG_R ? COOT_WREG_C : COOT_WREG_R)

// index of tree t among the trees with column (row) sums
template <int T> struct coot_cs_slot {
  static constexpr int K = (T > 0 ? COOT_CS_0 : 0) + (T > 1 ? COOT_CS_1 : 0) + (T > 2 ? COOT_CS_2 : 0);
};
template <int T> struct coot_rs_slot {
  static constexpr int K = (T > 0 ? COOT_RS_0 : 0) + (T > 1 ? COOT_RS_1 : 0) + (T > 2 ? COOT_RS_2 : 0);
};
template <int T> struct coot_tree_flags;
#define COOT_TREE_FLAGS(I)                                                                                   \
  template <> struct coot_tree_flags<I> {                                                                    \
    static constexpr bool CS = COOT_CS_##I, RS = COOT_RS_##I, ST = COOT_STORE_##I;                         \
    static constexpr int TCS = COOT_TCS_##I, TRS = COOT_TRS_##I, TO = COOT_TO_##I;                         \
    static constexpr unsigned H = COOT_HEADS_##I;                                                            \
    /* the plain sum taken from the row (else column) pairs */                                               \
    static constexpr bool SUM_ROWS = RS && (H & COOT_HEAD_SUM) != 0;                                         \
    static constexpr bool SUM_COLS = !RS && CS && (H & COOT_HEAD_SUM) != 0;                                  \
    static constexpr unsigned SKIP = (SUM_ROWS || SUM_COLS) ? COOT_HEAD_SUM : 0u;                            \
  };
COOT_TREE_FLAGS(0)
COOT_TREE_FLAGS(1)
COOT_TREE_FLAGS(2)
COOT_TREE_FLAGS(3)
#undef COOT_TREE_FLAGS

// A running (sum, compensation) pair of values per lane: packed FP32 pairs
// (two TwoSum lanes per instruction) or plain TwoSum.
#if COOT_PACK
typedef coot_f2 coot_racc;
__device__ __forceinline__ void coot_racc_zero(coot_racc& a) { a = 0ull; }
// x[0] enters lane 0, x[1] lane 1
__device__ __forceinline__ void coot_racc_add(coot_racc& s, coot_racc& c, const COOT_REAL* x) {
  coot_two_sum2(s, c, coot_pack(x[0], x[1]));
}
// the lanes as normalised double-word numbers: h[w], l[w] for w < COOT_RSTEP
__device__ __forceinline__ void coot_racc_pairs(coot_racc s, coot_racc c, COOT_REAL* h, COOT_REAL* l) {
  float sa, sb, ca, cb;
  coot_unpack(s, sa, sb);
  coot_unpack(c, ca, cb);
  coot_dw_norm(sa, ca, h[0], l[0]);
  coot_dw_norm(sb, cb, h[1], l[1]);
}
// the two lanes as one {sum, compensation}: the sums with TwoSum, the error
// and both compensations added
__device__ __forceinline__ void coot_racc_entry(coot_racc s2, coot_racc c2, COOT_REAL* out) {
  float sa, sb, ca, cb;
  coot_unpack(s2, sa, sb);
  coot_unpack(c2, ca, cb);
  float s = sa, c = ca;
  coot_two_sum(s, c, sb);
  out[0] = s;
  out[1] = c + cb;
}
#else
typedef COOT_REAL coot_racc;
__device__ __forceinline__ void coot_racc_zero(coot_racc& a) { a = (COOT_REAL)0; }
__device__ __forceinline__ void coot_racc_add(coot_racc& s, coot_racc& c, const COOT_REAL* x) {
  coot_two_sum(s, c, x[0]);
}
__device__ __forceinline__ void coot_racc_pairs(coot_racc s, coot_racc c, COOT_REAL* h, COOT_REAL* l) {
  coot_dw_norm(s, c, h[0], l[0]);
}
__device__ __forceinline__ void coot_racc_entry(coot_racc s, coot_racc c, COOT_REAL* out) {
  out[0] = s;
  out[1] = c;
}
#endif

// The warp's sum over lanes that share a column: xor-shuffle tree over the
// lane bits from `from` up (the double-word addition is commutative, so
// both lanes of an exchange form the same sum).
__device__ __forceinline__ void coot_dw_xor_sum(COOT_REAL& h, COOT_REAL& l, int from) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (o < from) break;
    const COOT_REAL yh = __shfl_xor_sync(0xffffffffu, h, o);
    const COOT_REAL yl = __shfl_xor_sync(0xffffffffu, l, o);
    coot_dw_add(h, l, yh, yl);
  }
}

// the plain sum of tree TT from a summed pair
#define COOT_ADD_PAIR(TT, h, l)                                                                               \
  {                                                                                                           \
    if constexpr (TT == 0) acc0.add_pair(h, l);                                                               \
    else if constexpr (TT == 1) acc1.add_pair(h, l);                                                          \
    else if constexpr (TT == 2) acc2.add_pair(h, l);                                                          \
    else acc3.add_pair(h, l);                                                                                 \
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
  __shared__ __align__(16) COOT_REAL wsm[COOT_WARPS][COOT_WREG];
#if COOT_NRS > 0
  __shared__ int is_last;
#endif
  COOT_REAL* const mine = wsm[warp];
  // this lane's row pairs: rows (k * 32 + lane) * VEC + q * RSTEP + w of the
  // segment (declared without row sums too: the code that does not use them
  // still names them)
  coot_racc rsum[COOT_NRS1][COOT_UNROLL][COOT_RV];
  coot_racc rcmp[COOT_NRS1][COOT_UNROLL][COOT_RV];
  coot_u32* cnt_col = (coot_u32*)(p.ws + COOT_WS_COUNTERS_OFF);
  coot_u32* cnt_seg = cnt_col + ((COOT_NCS > 0 && n_seg > 1) ? p.n_cols : 0);
  COOT_REAL* const cph = (COOT_REAL*)(p.ws + dp.cpart);
  const coot_i64 cper = p.n_cols * n_seg;
  (void)cnt_seg;
  (void)cph;
  (void)cper;

  for (coot_i64 u = blockIdx.x; u < units; u += gridDim.x) {
    const coot_i64 chunk = u / n_seg;
    const coot_i64 seg = u - chunk * n_seg;
    const coot_i64 rb = seg * COOT_SEG;
    const coot_i64 jb = chunk * dp.chunk_cols;
    const coot_i64 je = min(p.n_cols, jb + dp.chunk_cols);
    const bool whole = rb + COOT_SEG <= p.n_rows;
#pragma unroll
    for (int t = 0; t < COOT_NRS1; ++t)
#pragma unroll
      for (int k = 0; k < COOT_UNROLL; ++k)
#pragma unroll
        for (int q = 0; q < COOT_RV; ++q) {
          coot_racc_zero(rsum[t][k][q]);
          coot_racc_zero(rcmp[t][k][q]);
        }
    int nb = 0;            // columns in the current batch
    coot_i64 jfirst = 0;   // the batch's first column (then every COOT_WARPS-th)
    (void)jfirst;
    // Column batch: each lane adds COOT_CB of a column's lane pairs, then
    // the lanes of a column combine; the (column, segment) sums are stored
    // or become partials.
    auto flush = [&]() {
#if COOT_NCS > 0
      __syncwarp();
      constexpr int G = 32 / COOT_CB;  // lanes per column
      const int c = lane % COOT_CB, part = lane / COOT_CB;
      const coot_i64 j = jfirst + (coot_i64)c * COOT_WARPS;
      const bool mine_col = part == 0 && c < nb;
      COOT_REAL ch[COOT_NCS1], cl[COOT_NCS1];
#pragma unroll
      for (int t = 0; t < COOT_NCS; ++t) {
        // lane entries part * CB .. part * CB + CB of column c, in order,
        // into a running TwoSum pair (each entry's sums enter exactly, its
        // compensations are added to the pair's)
        COOT_REAL s = (COOT_REAL)0, e = (COOT_REAL)0;
        if (c < nb) {
          const COOT_REAL* tab = mine + t * COOT_CTAB + (c * 33 + part * COOT_CB) * COOT_ENT;
#pragma unroll
          for (int i = 0; i < COOT_CB; ++i) {
            COOT_REAL en[COOT_ENT];
#pragma unroll
            for (int w = 0; w < COOT_ENT; ++w) en[w] = tab[i * COOT_ENT + w];
            coot_two_sum(s, e, en[0]);
            e += en[1];
          }
        }
        coot_dw_norm(s, e, ch[t], cl[t]);
        if constexpr (G > 1) coot_dw_xor_sum(ch[t], cl[t], COOT_CB);
      }
      __syncwarp();  // the tables are rewritten by the next batch
      // the plain sum of a tree without row sums, from its column sums
#define COOT_SUM_FROM_COLS(TT)                                                                                \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::SUM_COLS) {                                              \
    if (mine_col) COOT_ADD_PAIR(TT, ch[coot_cs_slot<TT>::K], cl[coot_cs_slot<TT>::K])                         \
  }
      COOT_SUM_FROM_COLS(0)
      COOT_SUM_FROM_COLS(1)
      COOT_SUM_FROM_COLS(2)
      COOT_SUM_FROM_COLS(3)
#undef COOT_SUM_FROM_COLS
      // column sum of tree TT (summed-tree slot K) from the pair (h, l)
#define COOT_CS_STORE(TT, h, l)                                                                               \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::CS) {                                                   \
    typedef typename coot_st<coot_tree_flags<TT>::TCS>::T TCT;                                                \
    ((TCT*)dp.cs[TT])[j * dp.ld_cs[TT]] =                                                                     \
        coot_dw_store<coot_tree_flags<TT>::TCS>(h[coot_cs_slot<TT>::K], l[coot_cs_slot<TT>::K]);             \
  }
      if (n_seg == 1) {
        if (mine_col) {
          COOT_CS_STORE(0, ch, cl)
          COOT_CS_STORE(1, ch, cl)
          COOT_CS_STORE(2, ch, cl)
          COOT_CS_STORE(3, ch, cl)
        }
      } else {
        // partials: summed-tree slot t's high parts at [t][j][seg], then its
        // low parts (made visible, and counted, at the end of the unit)
        if (mine_col) {
#pragma unroll
          for (int t = 0; t < COOT_NCS; ++t) {
            cph[2 * t * cper + j * n_seg + seg] = ch[t];
            cph[(2 * t + 1) * cper + j * n_seg + seg] = cl[t];
          }
        }
      }
#undef COOT_CS_STORE
      nb = 0;
#endif
    };

    // The warp's columns (with COOT_PREFETCH, each one's inputs loaded
    // while the previous one is computed, in two register buffers).  In the
    // last, partial segment the vector that crosses the end is loaded
    // element by element with 0 past the end, and the values of rows past
    // the end are neither stored nor reduced.
    COOT_REAL xa[COOT_UNROLL][4][COOT_VEC], xb[COOT_UNROLL][4][COOT_VEC];
    auto load_col = [&](coot_i64 j, COOT_REAL (&x)[COOT_UNROLL][4][COOT_VEC]) {
#pragma unroll
      for (int k = 0; k < COOT_UNROLL; ++k) {
        const coot_i64 row0 = rb + ((coot_i64)k * 32 + lane) * COOT_VEC;
        if (whole || row0 + COOT_VEC <= p.n_rows) {
          coot_load_vec(p, j, row0, x[k]);
        } else {
#pragma unroll
          for (int v = 0; v < COOT_VEC; ++v) {
            COOT_REAL e[4] = {(COOT_REAL)0, (COOT_REAL)0, (COOT_REAL)0, (COOT_REAL)0};
            if (row0 + v < p.n_rows) coot_load_one(p, j, row0 + v, e);
#pragma unroll
            for (int i = 0; i < 4; ++i) x[k][i][v] = e[i];
          }
        }
      }
    };
    // one column's values: stored, reduced, summed
    auto process = [&](coot_i64 j, const COOT_REAL (&xc)[COOT_UNROLL][4][COOT_VEC]) {
        if (nb == 0) jfirst = j;
        coot_racc csum[COOT_NCS1], ccmp[COOT_NCS1];
#pragma unroll
        for (int t = 0; t < COOT_NCS1; ++t) {
          coot_racc_zero(csum[t]);
          coot_racc_zero(ccmp[t]);
        }
        // tree TT's COOT_VEC values yv at rows row .. row + VEC of this lane
        // (vector k): stored, reduced, added to the row and column pairs; in
        // the partial segment only the first n_ok of them are rows
  #define COOT_DIMS_USE(TT, k, row, yv, n_ok)                                                                   \
    if constexpr (TT < COOT_NT) {                                                                               \
      typedef coot_tree_flags<TT> F;                                                                            \
      if (n_ok >= COOT_VEC) {                                                                                   \
        if constexpr (TT == 0) acc0.add_vec<COOT_VEC, F::SKIP>(yv);                                              \
        else if constexpr (TT == 1) acc1.add_vec<COOT_VEC, F::SKIP>(yv);                                         \
        else if constexpr (TT == 2) acc2.add_vec<COOT_VEC, F::SKIP>(yv);                                         \
        else acc3.add_vec<COOT_VEC, F::SKIP>(yv);                                                                \
        if constexpr (F::ST) {                                                                                  \
          typedef typename coot_st<F::TO>::T TOT;                                                               \
          coot_vstore<F::TO, COOT_VEC>((TOT*)dp.out[TT] + (j * dp.ld_out[TT] + (row)), yv);                     \
        }                                                                                                       \
      } else {                                                                                                  \
        _Pragma("unroll") for (int v = 0; v < COOT_VEC; ++v) {                                                 \
          if (v < n_ok) {                                                                                       \
            if constexpr (TT == 0) acc0.add_vec<1, F::SKIP>(yv + v);                                             \
            else if constexpr (TT == 1) acc1.add_vec<1, F::SKIP>(yv + v);                                        \
            else if constexpr (TT == 2) acc2.add_vec<1, F::SKIP>(yv + v);                                        \
            else acc3.add_vec<1, F::SKIP>(yv + v);                                                               \
            if constexpr (F::ST) {                                                                              \
              typedef typename coot_st<F::TO>::T TOT;                                                           \
              coot_sstore<F::TO>((TOT*)dp.out[TT] + (j * dp.ld_out[TT] + (row) + v), yv[v]);                    \
            }                                                                                                   \
          } else {                                                                                              \
            yv[v] = (COOT_REAL)0; /* adds nothing to the row and column pairs */                                \
          }                                                                                                     \
        }                                                                                                       \
      }                                                                                                         \
      if constexpr (F::RS) {                                                                                    \
        _Pragma("unroll") for (int q = 0; q < COOT_RV; ++q)                                                    \
          coot_racc_add(rsum[coot_rs_slot<TT>::K][k][q], rcmp[coot_rs_slot<TT>::K][k][q], yv + q * COOT_RSTEP);  \
      }                                                                                                         \
      if constexpr (F::CS) {                                                                                    \
        _Pragma("unroll") for (int q = 0; q < COOT_RV; ++q)                                                    \
          coot_racc_add(csum[coot_cs_slot<TT>::K], ccmp[coot_cs_slot<TT>::K], yv + q * COOT_RSTEP);             \
      }                                                                                                         \
    }
  #pragma unroll
        for (int k = 0; k < COOT_UNROLL; ++k) {
          COOT_REAL y[4][COOT_VEC];
          coot_multi_f(xc[k], y);
          const coot_i64 row = rb + ((coot_i64)k * 32 + lane) * COOT_VEC;
          const coot_i64 left = p.n_rows - row;
          const int n_ok = whole ? COOT_VEC : (int)(left < 0 ? 0 : (left > COOT_VEC ? COOT_VEC : left));
          COOT_DIMS_USE(0, k, row, y[0], n_ok)
          COOT_DIMS_USE(1, k, row, y[1], n_ok)
          COOT_DIMS_USE(2, k, row, y[2], n_ok)
          COOT_DIMS_USE(3, k, row, y[3], n_ok)
        }
  #undef COOT_DIMS_USE
  #if COOT_NCS > 0
        // the lane's column pair into the batch table
  #pragma unroll
        for (int t = 0; t < COOT_NCS; ++t) {
          // the accumulator's lanes merged (TwoSum of the sums, the error
          // and the compensations added) into one table entry
          COOT_REAL en[COOT_ENT];
          coot_racc_entry(csum[t], ccmp[t], en);
          COOT_REAL* dst = mine + t * COOT_CTAB + (nb * 33 + lane) * COOT_ENT;
#pragma unroll
          for (int w = 0; w < COOT_ENT; ++w) dst[w] = en[w];
        }
        if (++nb == COOT_CB) flush();
  #endif
    };
#if COOT_PREFETCH
    // two register buffers: column j + warps loads while column j computes
    coot_i64 j = jb + warp;
    if (j < je) load_col(j, xa);
    while (j < je) {
      if (j + COOT_WARPS < je) load_col(j + COOT_WARPS, xb);
      process(j, xa);
      j += COOT_WARPS;
      if (j >= je) break;
      if (j + COOT_WARPS < je) load_col(j + COOT_WARPS, xa);
      process(j, xb);
      j += COOT_WARPS;
    }
#else
    for (coot_i64 j = jb + warp; j < je; j += COOT_WARPS) {
      load_col(j, xa);
      process(j, xa);
    }
#endif
#if COOT_NCS > 0
    if (nb > 0) flush();
    if (n_seg > 1) {
      // one fence for the warp's partials of this unit, then an arrival per
      // column; the last lane to arrive at a column adds its partials in
      // segment order (lane L takes the warp's columns L, L + 32, ...)
      __threadfence();
      __syncwarp();
      const coot_i64 n_mine = je > jb + warp ? (je - jb - warp + COOT_WARPS - 1) / COOT_WARPS : 0;
      for (coot_i64 i = lane; i < n_mine; i += 32) {
        const coot_i64 j = jb + warp + i * COOT_WARPS;
        if (atomicAdd(cnt_col + j, 1u) == (coot_u32)(n_seg - 1)) {
          __threadfence();
          COOT_REAL sh[COOT_NCS1], sl[COOT_NCS1];
#pragma unroll
          for (int t = 0; t < COOT_NCS; ++t) {
            sh[t] = sl[t] = (COOT_REAL)0;
            for (coot_i64 q = 0; q < n_seg; ++q)
              coot_dw_add(sh[t], sl[t], __ldcg(cph + 2 * t * cper + j * n_seg + q),
                          __ldcg(cph + (2 * t + 1) * cper + j * n_seg + q));
          }
#define COOT_CS_STORE(TT, h, l)                                                                               \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::CS) {                                                   \
    typedef typename coot_st<coot_tree_flags<TT>::TCS>::T TCT;                                                \
    ((TCT*)dp.cs[TT])[j * dp.ld_cs[TT]] =                                                                     \
        coot_dw_store<coot_tree_flags<TT>::TCS>(h[coot_cs_slot<TT>::K], l[coot_cs_slot<TT>::K]);             \
  }
          COOT_CS_STORE(0, sh, sl)
          COOT_CS_STORE(1, sh, sl)
          COOT_CS_STORE(2, sh, sl)
          COOT_CS_STORE(3, sh, sl)
#undef COOT_CS_STORE
          cnt_col[j] = 0u;  // ready for the next call
        }
      }
    }
#endif
#if COOT_NRS > 0
    // rows of the segment over the chunk: the warps' pairs added in warp
    // order, one summed tree at a time
    COOT_REAL* rph = (COOT_REAL*)(p.ws + dp.rpart);
    const coot_i64 rper = n_chunk * p.n_rows;
    __syncwarp();  // this warp's column tables are no longer read
#define COOT_RS_TREE(TT)                                                                                      \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::RS) {                                                   \
    constexpr int K = coot_rs_slot<TT>::K;                                                                    \
    typedef typename coot_st<coot_tree_flags<TT>::TRS>::T TRT;                                                \
    _Pragma("unroll") for (int k = 0; k < COOT_UNROLL; ++k)                                                  \
      _Pragma("unroll") for (int q = 0; q < COOT_RV; ++q) {                                                  \
        COOT_REAL h[COOT_RSTEP], l[COOT_RSTEP];                                                               \
        coot_racc_pairs(rsum[K][k][q], rcmp[K][k][q], h, l);                                                  \
        _Pragma("unroll") for (int w = 0; w < COOT_RSTEP; ++w) {                                             \
          const int r = (k * 32 + lane) * COOT_VEC + q * COOT_RSTEP + w;                                      \
          mine[r] = h[w];                                                                                     \
          mine[COOT_SEG + r] = l[w];                                                                          \
          if constexpr (coot_tree_flags<TT>::SUM_ROWS) COOT_ADD_PAIR(TT, h[w], l[w])                          \
        }                                                                                                     \
      }                                                                                                       \
    __syncthreads();                                                                                          \
    for (int r = threadIdx.x; r < COOT_SEG; r += COOT_BLOCK) {                                               \
      COOT_REAL h = wsm[0][r], l = wsm[0][COOT_SEG + r];                                                      \
      _Pragma("unroll") for (int w = 1; w < COOT_WARPS; ++w) coot_dw_add(h, l, wsm[w][r], wsm[w][COOT_SEG + r]); \
      const coot_i64 row = rb + r;                                                                            \
      if (row < p.n_rows) {                                                                                   \
        if (n_chunk == 1) {                                                                                   \
          ((TRT*)dp.rs[TT])[row] = coot_dw_store<coot_tree_flags<TT>::TRS>(h, l);                             \
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
#define COOT_RS_LAST(TT)                                                                                      \
  if constexpr (TT < COOT_NT && coot_tree_flags<TT>::RS) {                                                   \
    constexpr int K = coot_rs_slot<TT>::K;                                                                    \
    typedef typename coot_st<coot_tree_flags<TT>::TRS>::T TRT;                                                \
    for (int r = threadIdx.x; r < COOT_SEG; r += COOT_BLOCK) {                                               \
      const coot_i64 row = rb + r;                                                                            \
      if (row < p.n_rows) {                                                                                   \
        COOT_REAL h = 0, l = 0;                                                                               \
        _Pragma("unroll 4") for (coot_i64 c = 0; c < n_chunk; ++c)                                            \
          coot_dw_add(h, l, __ldcg(rph + 2 * K * rper + c * p.n_rows + row),                                 \
                      __ldcg(rph + (2 * K + 1) * rper + c * p.n_rows + row));                                 \
        ((TRT*)dp.rs[TT])[row] = coot_dw_store<coot_tree_flags<TT>::TRS>(h, l);                               \
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
#else
    __syncwarp();  // this warp's column tables are rewritten by the next unit
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
#undef COOT_ADD_PAIR
#endif
