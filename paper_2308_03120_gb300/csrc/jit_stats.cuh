// Statistics along a dimension (kinds 5 and 6); part of the device runtime
// embedded after jit_rt.cuh.  COOT_HEADS holds the mask of statistics
// (COOT_STAT_* in coot.h): sum, mean, var, stddev, min, max of each column
// (kind 5) or each row (kind 6), all from ONE pass over the inputs.
//
// Sum and mean come from the exact per-thread sum of the values (TwoSum on
// every element).  The variance is taken about a shift K, the value of the
// line's first element: d = y - K (exact by Sterbenz' lemma whenever y is
// within a factor of two of K, which is the case that matters -- a mean
// large against the spread), D1 = sum d and D2 = sum d^2, each group of
// values added pairwise and the group total with TwoSum.  The column
// statistics form D1 at the end as S - N K in FP64 from the exact sum S
// (about 48 bits; its error costs about 2 |mean| |mean - K| 2^-48 / var of
// the variance, far below the bound below) instead of accumulating it,
// which saves a pairwise sum and a TwoSum per group.  Then
//   var = (D2 - D1 * D1 / N) / (N - 1 + norm_type)
// in FP64, where the cancellation costs a factor 1 + (mean - K)^2 / var
// (about 2 for a typical K) instead of 1 + mean^2 / var.  The error is at
// most about 11 u sum (y - K)^2 / (N - 1 + norm_type), u the compute type's
// unit roundoff.  Threads combine as double-word numbers in a fixed order.

#if COOT_KIND == 5 || COOT_KIND == 6
#define COOT_ST_SUM (1u << 0)
#define COOT_ST_MEAN (1u << 1)
#define COOT_ST_VAR (1u << 2)
#define COOT_ST_STDDEV (1u << 3)
#define COOT_ST_MIN (1u << 4)
#define COOT_ST_MAX (1u << 5)
#define COOT_ST_D ((COOT_HEADS & (COOT_ST_VAR | COOT_ST_STDDEV)) != 0)
// column statistics (kind 5) form the shifted sum at the end as S - N K from
// the exact sum instead of accumulating it
#define COOT_ST_D1S (COOT_KIND == 5)
#define COOT_ST_S1 ((COOT_HEADS & (COOT_ST_SUM | COOT_ST_MEAN)) != 0 || (COOT_ST_D1S && COOT_ST_D))
#define COOT_ST_MN ((COOT_HEADS & COOT_ST_MIN) != 0)
#define COOT_ST_MX ((COOT_HEADS & COOT_ST_MAX) != 0)
// components of a line's partial: sum (hi, lo), shifted sum (hi, lo; not
// for columns), shifted sum of squares (hi, lo), minimum, maximum -- those
// the statistics need, in that order
#define COOT_ST_NC (2 * COOT_ST_S1 + (COOT_ST_D1S ? 2 : 4) * COOT_ST_D + COOT_ST_MN + COOT_ST_MX)

// Launch parameters (every field 8 bytes; mirrored on the host).
struct coot_stats_params {
  coot_params b;       // inputs, shape, split, workspace
  void* out[6];        // one output per set statistic, in bit order
  coot_i64 inc[6];     // element stride of each output
  coot_i64 norm_type;  // variance divisor N - 1 + norm_type
};

struct coot_sacc {
  COOT_REAL s, sc;    // sum and its TwoSum compensation
  COOT_REAL d1, d1c;  // shifted sum
  COOT_REAL d2, d2c;  // shifted sum of squares
  COOT_REAL mn, mx;

  __device__ __forceinline__ void init() {
    s = sc = d1 = d1c = d2 = d2c = (COOT_REAL)0;
    mn = (COOT_REAL)COOT_INF_F;
    mx = -(COOT_REAL)COOT_INF_F;
  }
  // one value of the line
  __device__ __forceinline__ void add(COOT_REAL y, COOT_REAL K) {
    if constexpr (COOT_ST_S1) coot_two_sum(s, sc, y);
    if constexpr (COOT_ST_D) {
      const COOT_REAL d = y - K;
      if constexpr (!COOT_ST_D1S) coot_two_sum(d1, d1c, d);
      coot_two_sum(d2, d2c, coot_sq(d));
    }
    if constexpr (COOT_ST_MN) mn = coot_min(mn, y);
    if constexpr (COOT_ST_MX) mx = coot_max(mx, y);
  }
  // G values of the line: the shifted sums add the group pairwise
  template <int G>
  __device__ __forceinline__ void add_group(const COOT_REAL* y, COOT_REAL K) {
    if constexpr (COOT_ST_D) {
      COOT_REAL d[G];
#pragma unroll
      for (int g = 0; g < G; ++g) d[g] = y[g] - K;
      if constexpr (!COOT_ST_D1S) coot_two_sum(d1, d1c, coot_pairwise<G>(d, 0));
      coot_two_sum(d2, d2c, coot_pairwise<G>(d, 1));
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if constexpr (COOT_ST_S1) coot_two_sum(s, sc, y[g]);
      if constexpr (COOT_ST_MN) mn = coot_min(mn, y[g]);
      if constexpr (COOT_ST_MX) mx = coot_max(mx, y[g]);
    }
  }
  // the components of this accumulator (sums as normalised pairs)
  __device__ __forceinline__ void comps(COOT_REAL (&c)[COOT_ST_NC]) const {
    int k = 0;
    if constexpr (COOT_ST_S1) {
      coot_dw_norm(s, sc, c[k], c[k + 1]);
      k += 2;
    }
    if constexpr (COOT_ST_D && !COOT_ST_D1S) {
      coot_dw_norm(d1, d1c, c[k], c[k + 1]);
      coot_dw_norm(d2, d2c, c[k + 2], c[k + 3]);
      k += 4;
    }
    if constexpr (COOT_ST_D && COOT_ST_D1S) {
      coot_dw_norm(d2, d2c, c[k], c[k + 1]);
      k += 2;
    }
    if constexpr (COOT_ST_MN) c[k++] = mn;
    if constexpr (COOT_ST_MX) c[k++] = mx;
    (void)k;
  }
};

__device__ __forceinline__ void coot_st_identity(COOT_REAL (&c)[COOT_ST_NC]) {
  int k = 0;
  if constexpr (COOT_ST_S1) { c[k] = c[k + 1] = (COOT_REAL)0; k += 2; }
  if constexpr (COOT_ST_D) {
#pragma unroll
    for (int q = 0; q < (COOT_ST_D1S ? 2 : 4); ++q) c[k + q] = (COOT_REAL)0;
    k += COOT_ST_D1S ? 2 : 4;
  }
  if constexpr (COOT_ST_MN) c[k++] = (COOT_REAL)COOT_INF_F;
  if constexpr (COOT_ST_MX) c[k++] = -(COOT_REAL)COOT_INF_F;
  (void)k;
}

// x <- x combined with y, component by component
__device__ __forceinline__ void coot_st_combine(COOT_REAL (&x)[COOT_ST_NC], const COOT_REAL (&y)[COOT_ST_NC]) {
  int k = 0;
  if constexpr (COOT_ST_S1) { coot_dw_add(x[k], x[k + 1], y[k], y[k + 1]); k += 2; }
  if constexpr (COOT_ST_D) {
    coot_dw_add(x[k], x[k + 1], y[k], y[k + 1]);
    if constexpr (!COOT_ST_D1S) coot_dw_add(x[k + 2], x[k + 3], y[k + 2], y[k + 3]);
    k += COOT_ST_D1S ? 2 : 4;
  }
  if constexpr (COOT_ST_MN) { x[k] = coot_min(x[k], y[k]); ++k; }
  if constexpr (COOT_ST_MX) { x[k] = coot_max(x[k], y[k]); ++k; }
  (void)k;
}

// The shift of a line: the tree's value at its first element (row 0 of
// column `line` for kind 5, column 0 of row `line` for kind 6); 0 for an
// empty line.
__device__ __forceinline__ COOT_REAL coot_st_shift(const coot_params& p, coot_i64 line) {
  if constexpr (!COOT_ST_D) {
    return (COOT_REAL)0;
  } else {
    if (p.n_rows == 0 || p.n_cols == 0) return (COOT_REAL)0;
    COOT_REAL x[4];
    if constexpr (COOT_KIND == 5) {
      coot_load_one(p, line, 0, x);
    } else {
      coot_load_one(p, 0, line, x);
    }
    return coot_f(x);
  }
}

// The statistics of line `i` (N elements, shift K) from its combined
// components, written to the outputs in bit order.  Outputs are FP32 or
// FP64.
__device__ void coot_st_store(const coot_stats_params& sp, coot_i64 i, coot_i64 N, COOT_REAL K,
                              const COOT_REAL (&c)[COOT_ST_NC]) {
  typedef typename coot_st<COOT_TO>::T TO;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  int k = 0;
  COOT_REAL s1h = 0, s1l = 0, mn = 0, mx = 0;
  double s1 = 0.0, d1 = 0.0, d2 = 0.0;
  if constexpr (COOT_ST_S1) {
    s1h = c[k];
    s1l = c[k + 1];
    s1 = coot_dw_to_double(s1h, s1l);
    k += 2;
  }
  if constexpr (COOT_ST_D && !COOT_ST_D1S) {
    d1 = coot_dw_to_double(c[k], c[k + 1]);
    d2 = coot_dw_to_double(c[k + 2], c[k + 3]);
    k += 4;
  }
  if constexpr (COOT_ST_D && COOT_ST_D1S) {
    // the shifted sum from the exact sum: S - N K in FP64 (S carries about
    // 48 bits, N K is exact up to 2^29 elements)
    d1 = s1 - (double)N * (double)K;
    d2 = coot_dw_to_double(c[k], c[k + 1]);
    k += 2;
  }
  if constexpr (COOT_ST_MN) mn = c[k++];
  if constexpr (COOT_ST_MX) mx = c[k++];
  (void)k;
  double var = nan;
  if constexpr (COOT_ST_D) {
    if (N == 1 && sp.norm_type == 0) {
      var = isfinite((double)K) ? 0.0 : nan;
    } else if (N > 0 && isfinite(d1) && isfinite(d2)) {
      var = (d2 - d1 * (d1 / (double)N)) / (double)(N - 1 + sp.norm_type);
      if (var < 0.0) var = 0.0;  // rounding of a (near) constant line
    }
  }
  (void)K;
  int o = 0;
  if constexpr ((COOT_HEADS & COOT_ST_SUM) != 0) {
    ((TO*)sp.out[o])[i * sp.inc[o]] = coot_dw_store<COOT_TO>(s1h, s1l);
    ++o;
  }
  if constexpr ((COOT_HEADS & COOT_ST_MEAN) != 0) {
    ((TO*)sp.out[o])[i * sp.inc[o]] = (TO)(N > 0 ? s1 / (double)N : nan);
    ++o;
  }
  if constexpr ((COOT_HEADS & COOT_ST_VAR) != 0) {
    ((TO*)sp.out[o])[i * sp.inc[o]] = (TO)var;
    ++o;
  }
  if constexpr ((COOT_HEADS & COOT_ST_STDDEV) != 0) {
    ((TO*)sp.out[o])[i * sp.inc[o]] = (TO)sqrt(var);
    ++o;
  }
  if constexpr ((COOT_HEADS & COOT_ST_MIN) != 0) {
    ((TO*)sp.out[o])[i * sp.inc[o]] = (TO)mn;
    ++o;
  }
  if constexpr ((COOT_HEADS & COOT_ST_MAX) != 0) {
    ((TO*)sp.out[o])[i * sp.inc[o]] = (TO)mx;
    ++o;
  }
  (void)o;
}
#endif

// ================================================================ kind 5: statistics of each column

// A warp per unit (column j, segment s) as for the column sums: rows
// [s R, min((s + 1) R, n_rows)), R = p.rows_per_split.  With several
// segments per column the segment partials go to the workspace
// (component-major: NC x n_cols x S) and the last warp of a column to
// arrive combines them in segment order.
#if COOT_KIND == 5
extern "C" __global__ void __launch_bounds__(COOT_BLOCK) COOT_ENTRY(const __grid_constant__ coot_stats_params sp) {
  const coot_params& p = sp.b;
  constexpr coot_i64 WT = (coot_i64)32 * COOT_VEC * COOT_UNROLL;  // rows per warp tile
  const int lane = threadIdx.x & 31;
  const coot_i64 S = p.split;
  const coot_i64 units = p.n_cols * S;
  const coot_i64 n_warps = (coot_i64)gridDim.x * COOT_WARPS;
  for (coot_i64 u = (coot_i64)blockIdx.x * COOT_WARPS + (threadIdx.x >> 5); u < units; u += n_warps) {
    const coot_i64 j = u / S;
    const coot_i64 s = u - j * S;
    const coot_i64 rb = s * p.rows_per_split;
    const coot_i64 re = min(p.n_rows, rb + p.rows_per_split);
    const COOT_REAL K = coot_st_shift(p, j);
    coot_sacc acc;
    acc.init();
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
        acc.add_group<COOT_VEC>(y, K);
      }
    }
#pragma unroll 1
    for (coot_i64 row = r0 + lane; row < re; row += 32) {
      COOT_REAL x[4];
      coot_load_one(p, j, row, x);
      acc.add(coot_f(x), K);
    }
    COOT_REAL c[COOT_ST_NC];
    acc.comps(c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      COOT_REAL y[COOT_ST_NC];
#pragma unroll
      for (int k = 0; k < COOT_ST_NC; ++k) y[k] = __shfl_down_sync(0xffffffffu, c[k], o);
      coot_st_combine(c, y);
    }
    if (lane == 0) {
      if (S == 1) {
        coot_st_store(sp, j, p.n_rows, K, c);
      } else {
        COOT_REAL* part = (COOT_REAL*)(p.ws + COOT_WS_PARTIALS_OFF);
        const coot_i64 stride = p.n_cols * S;
        coot_u32* cnt = (coot_u32*)(p.ws + COOT_WS_COUNTERS_OFF);
#pragma unroll
        for (int k = 0; k < COOT_ST_NC; ++k) part[k * stride + j * S + s] = c[k];
        __threadfence();
        if (atomicAdd(cnt + j, 1u) == (coot_u32)(S - 1)) {
          __threadfence();
          COOT_REAL t[COOT_ST_NC];
          coot_st_identity(t);
          for (coot_i64 q = 0; q < S; ++q) {
            COOT_REAL y[COOT_ST_NC];
#pragma unroll
            for (int k = 0; k < COOT_ST_NC; ++k) y[k] = __ldcg(part + k * stride + j * S + q);
            coot_st_combine(t, y);
          }
          coot_st_store(sp, j, p.n_rows, K, t);
          cnt[j] = 0u;
        }
      }
    }
  }
}
#endif

// ================================================================ kind 6: statistics of each row

// As the row sums: a block is COOT_RT row threads x (COOT_BLOCK / COOT_RT)
// column groups over a panel of COOT_RT * COOT_VEC rows and a chunk of
// columns; groups combine in shared memory in group order; with several
// chunks the chunk partials go to the workspace (component-major:
// NC x chunks x n_rows) and the last block of a panel combines them.
#if COOT_KIND == 6
#define COOT_RT 64
#define COOT_CG (COOT_BLOCK / COOT_RT)
#define COOT_PANEL (COOT_RT * COOT_VEC)
extern "C" __global__ void __launch_bounds__(COOT_BLOCK) COOT_ENTRY(const __grid_constant__ coot_stats_params sp) {
  const coot_params& p = sp.b;
  __shared__ COOT_REAL red[COOT_CG][COOT_ST_NC][COOT_PANEL];
  __shared__ int is_last;
  const int tx = threadIdx.x % COOT_RT, ty = threadIdx.x / COOT_RT;
  const coot_i64 n_panels = (p.n_rows + COOT_PANEL - 1) / COOT_PANEL;
  const coot_i64 C = p.split;                 // column chunks
  const coot_i64 Q = (p.n_cols + C - 1) / C;  // columns per chunk
  const coot_i64 units = n_panels * C;
  COOT_REAL* part = (COOT_REAL*)(p.ws + COOT_WS_PARTIALS_OFF);
  const coot_i64 stride = C * p.n_rows;       // one component of every chunk
  coot_u32* cnt = (coot_u32*)(p.ws + COOT_WS_COUNTERS_OFF);
  for (coot_i64 u = blockIdx.x; u < units; u += gridDim.x) {
    const coot_i64 chunk = u / n_panels;
    const coot_i64 panel = u - chunk * n_panels;
    const coot_i64 i0 = panel * COOT_PANEL + (coot_i64)tx * COOT_VEC;
    const coot_i64 jb = chunk * Q;
    const coot_i64 je = min(p.n_cols, jb + Q);
    COOT_REAL K[COOT_VEC];
#pragma unroll
    for (int v = 0; v < COOT_VEC; ++v) K[v] = i0 + v < p.n_rows ? coot_st_shift(p, i0 + v) : (COOT_REAL)0;
    coot_sacc acc[COOT_VEC];
#pragma unroll
    for (int v = 0; v < COOT_VEC; ++v) acc[v].init();
    if (panel * COOT_PANEL + COOT_PANEL <= p.n_rows) {
      coot_i64 j = jb + ty;
      for (; j + (coot_i64)(COOT_UNROLL - 1) * COOT_CG < je; j += (coot_i64)COOT_UNROLL * COOT_CG) {
        COOT_REAL xv[COOT_UNROLL][4][COOT_VEC];
#pragma unroll
        for (int k = 0; k < COOT_UNROLL; ++k) coot_load_vec(p, j + (coot_i64)k * COOT_CG, i0, xv[k]);
        // the UNROLL columns in flight are a group of the same rows
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          COOT_REAL y[COOT_UNROLL];
#pragma unroll
          for (int k = 0; k < COOT_UNROLL; ++k) {
            const COOT_REAL x[4] = {xv[k][0][v], xv[k][1][v], xv[k][2][v], xv[k][3][v]};
            y[k] = coot_f(x);
          }
          acc[v].add_group<COOT_UNROLL>(y, K[v]);
        }
      }
      for (; j < je; j += COOT_CG) {
        COOT_REAL xv[4][COOT_VEC];
        coot_load_vec(p, j, i0, xv);
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          const COOT_REAL x[4] = {xv[0][v], xv[1][v], xv[2][v], xv[3][v]};
          acc[v].add(coot_f(x), K[v]);
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
            acc[v].add(coot_f(x), K[v]);
          }
        }
      }
    }
    // column groups in order -> the block's partial of each row over the chunk
#pragma unroll
    for (int v = 0; v < COOT_VEC; ++v) {
      COOT_REAL c[COOT_ST_NC];
      acc[v].comps(c);
#pragma unroll
      for (int k = 0; k < COOT_ST_NC; ++k) red[ty][k][tx * COOT_VEC + v] = c[k];
    }
    __syncthreads();
    COOT_REAL t[COOT_VEC][COOT_ST_NC];
    if (ty == 0) {
#pragma unroll
      for (int v = 0; v < COOT_VEC; ++v) {
#pragma unroll
        for (int k = 0; k < COOT_ST_NC; ++k) t[v][k] = red[0][k][tx * COOT_VEC + v];
#pragma unroll
        for (int g = 1; g < COOT_CG; ++g) {
          COOT_REAL y[COOT_ST_NC];
#pragma unroll
          for (int k = 0; k < COOT_ST_NC; ++k) y[k] = red[g][k][tx * COOT_VEC + v];
          coot_st_combine(t[v], y);
        }
      }
    }
    if (C == 1) {
      if (ty == 0) {
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v)
          if (i0 + v < p.n_rows) coot_st_store(sp, i0 + v, p.n_cols, K[v], t[v]);
      }
      __syncthreads();  // red is rewritten by the next unit
      continue;
    }
    if (ty == 0) {
#pragma unroll
      for (int v = 0; v < COOT_VEC; ++v)
        if (i0 + v < p.n_rows) {
#pragma unroll
          for (int k = 0; k < COOT_ST_NC; ++k) part[k * stride + chunk * p.n_rows + i0 + v] = t[v][k];
        }
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(cnt + panel, 1u) == (coot_u32)(C - 1));
    __syncthreads();
    if (is_last) {
      __threadfence();
      // group g combines chunks g, g + CG, ... for its rows; then group order
#pragma unroll
      for (int v = 0; v < COOT_VEC; ++v) {
        COOT_REAL g[COOT_ST_NC];
        coot_st_identity(g);
        if (i0 + v < p.n_rows) {
          for (coot_i64 q = ty; q < C; q += COOT_CG) {
            COOT_REAL y[COOT_ST_NC];
#pragma unroll
            for (int k = 0; k < COOT_ST_NC; ++k) y[k] = __ldcg(part + k * stride + q * p.n_rows + i0 + v);
            coot_st_combine(g, y);
          }
        }
#pragma unroll
        for (int k = 0; k < COOT_ST_NC; ++k) red[ty][k][tx * COOT_VEC + v] = g[k];
      }
      __syncthreads();
      if (ty == 0) {
#pragma unroll
        for (int v = 0; v < COOT_VEC; ++v) {
          COOT_REAL w[COOT_ST_NC];
#pragma unroll
          for (int k = 0; k < COOT_ST_NC; ++k) w[k] = red[0][k][tx * COOT_VEC + v];
#pragma unroll
          for (int g = 1; g < COOT_CG; ++g) {
            COOT_REAL y[COOT_ST_NC];
#pragma unroll
            for (int k = 0; k < COOT_ST_NC; ++k) y[k] = red[g][k][tx * COOT_VEC + v];
            coot_st_combine(w, y);
          }
          if (i0 + v < p.n_rows) coot_st_store(sp, i0 + v, p.n_cols, K[v], w);
        }
      }
      if (threadIdx.x == 0) cnt[panel] = 0u;
    }
    __syncthreads();  // red and is_last are rewritten by the next unit
  }
}
#endif
