// Device runtime of the fused expression kernels.
//
// This file is not compiled on its own: the library embeds it as a string
// and, for every (tree, kind, storage types, launch shape), compiles it at
// run time with NVRTC for the device's architecture (sm_103a on GB300),
// after a prelude that defines
//   COOT_KIND     0 element-wise evaluation (optionally with reductions),
//                 1 full reductions only, 2 column sums, 3 row sums,
//                 4 batched evaluation over a work list, 5 column
//                 statistics, 6 row statistics, 7 several trees in one
//                 pass, 8 several trees with column / row sums
//   COOT_NIN      number of input slots (1..4)
//   COOT_TI0..3   storage code of each input (0 FP32, 1 BF16, 2 FP16, 3 FP64)
//   COOT_TO       storage code of the stored output
//   COOT_STORE    1 if element values are stored
//   COOT_HEADS    mask of reduction heads (COOT_HEAD_* in coot.h); for the
//                 statistics kinds the mask of statistics (COOT_STAT_*)
//   COOT_REAL     float or double (the tree's compute type)
//   COOT_VEC      elements per vector access, COOT_UNROLL vectors in flight
//                 per thread and input, COOT_BLOCK threads per block
//   COOT_NC       1 if inputs may be read through the non-coherent path
// and the tree itself as `COOT_REAL coot_f(const COOT_REAL* x)`, one
// straight-line function of the input values (the paper's expression type,
// Section 7, instantiated for a single element).
//
// Every kernel is a persistent grid-stride loop over "units" (a tile of rows
// of one column for evaluation and column sums, a panel of rows times a
// range of columns for row sums), so any grid size covers any shape.
// Reductions add in FP32 (or FP64) with TwoSum compensation per thread,
// then combine per-thread results as double-word numbers through warp
// shuffles and shared memory into one FP64 partial per block; the last
// block to finish combines the partials in FP64 in a fixed order, so a
// result does not depend on timing.

typedef unsigned short coot_u16;
typedef unsigned int coot_u32;
typedef long long coot_i64;
typedef unsigned long long coot_u64;

// Launch parameters; every field is 8 bytes so the host-side copy of this
// struct has the same layout.
struct coot_params {
  const void* in[4];
  coot_i64 ld_in[4];
  void* out;
  coot_i64 ld_out;
  coot_i64 n_rows;
  coot_i64 n_cols;
  coot_i64 split;           // column sums: blocks per column; row sums: column chunks
  coot_i64 rows_per_split;  // column sums: rows per block when split > 1
  unsigned char* ws;        // workspace (counters + partials)
  double* res;              // reduction results
  const void* plan;         // batched: work list
  coot_i64 n_work;          // batched: number of work items
};

#define COOT_WS_COUNTER_OFF 128
#define COOT_WS_COUNTERS_OFF 256
#define COOT_WS_PARTIALS_OFF 65536

#define COOT_HEAD_SUM (1u << 0)
#define COOT_HEAD_SUMSQ (1u << 1)
#define COOT_HEAD_NORM2 (1u << 2)
#define COOT_HEAD_SUMABS (1u << 3)
#define COOT_HEAD_MIN (1u << 4)
#define COOT_HEAD_MAX (1u << 5)
#define COOT_HEAD_MINABS (1u << 6)
#define COOT_HEAD_MAXABS (1u << 7)
#define COOT_HEAD_ALL (1u << 8)
#define COOT_HEAD_ANY (1u << 9)

#define COOT_WARPS (COOT_BLOCK / 32)
#define COOT_INF_F __int_as_float(0x7f800000)
#define COOT_INF_D __longlong_as_double(0x7ff0000000000000ll)

// ---------------------------------------------------------------- storage

template <int S> struct coot_st;
template <> struct coot_st<0> { typedef float T; };
template <> struct coot_st<1> { typedef coot_u16 T; };
template <> struct coot_st<2> { typedef coot_u16 T; };
template <> struct coot_st<3> { typedef double T; };
template <> struct coot_st<4> { typedef int T; };
template <> struct coot_st<5> { typedef coot_u32 T; };

template <int S>
__device__ __forceinline__ COOT_REAL coot_to_real(typename coot_st<S>::T v) {
  if constexpr (S == 0) {
    return (COOT_REAL)v;
  } else if constexpr (S == 1) {
    // a BF16 number is the top half of the FP32 number with the same bits
    return (COOT_REAL)__uint_as_float(((coot_u32)v) << 16);
  } else if constexpr (S == 2) {
    float f;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(v));
    return (COOT_REAL)f;
  } else {
    // FP64 (rounded to nearest for an FP32 tree) and the integers (nearest
    // FP32, exact up to 2^24; exact in FP64)
    return (COOT_REAL)v;
  }
}

// integer storage of a compute-type value: rounded toward zero, saturated
// to the type's range, NaN -> 0 (the float-to-integer conversion of PTX)
__device__ __forceinline__ int coot_f2s32(float v) {
  int r;
  asm("cvt.rzi.s32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ int coot_f2s32(double v) {
  int r;
  asm("cvt.rzi.s32.f64 %0, %1;" : "=r"(r) : "d"(v));
  return r;
}
__device__ __forceinline__ coot_u32 coot_f2u32(float v) {
  coot_u32 r;
  asm("cvt.rzi.u32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ coot_u32 coot_f2u32(double v) {
  coot_u32 r;
  asm("cvt.rzi.u32.f64 %0, %1;" : "=r"(r) : "d"(v));
  return r;
}
// (the FP64 conversions do not map NaN to 0 by themselves: NaN is tested)
template <int S>
__device__ __forceinline__ typename coot_st<S>::T coot_to_int(COOT_REAL v) {
  if constexpr (S == 4) {
    return v != v ? 0 : coot_f2s32(v);
  } else {
    return v != v ? 0u : coot_f2u32(v);
  }
}

template <int S>
__device__ __forceinline__ typename coot_st<S>::T coot_from_real(COOT_REAL v) {
  if constexpr (S == 0) {
    return (float)v;
  } else if constexpr (S == 1) {
    float f = (float)v;
    coot_u16 h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return h;
  } else if constexpr (S == 2) {
    float f = (float)v;
    coot_u16 h;
    asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return h;
  } else if constexpr (S == 3) {
    return (double)v;
  } else {
    return coot_to_int<S>(v);
  }
}

template <int S>
__device__ __forceinline__ typename coot_st<S>::T coot_from_double(double v) {
  if constexpr (S == 3) {
    return v;
  } else if constexpr (S >= 4) {
    return coot_from_real<S>((COOT_REAL)v);
  } else {
    float f = (float)v;  // nearest FP32, then nearest storage value
    if constexpr (S == 0) {
      return f;
    } else if constexpr (S == 1) {
      coot_u16 h;
      asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
      return h;
    } else {
      coot_u16 h;
      asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
      return h;
    }
  }
}

// ---------------------------------------------------------------- memory

#if COOT_NC
#define COOT_LD "ld.global.nc.L1::no_allocate"
#else
#define COOT_LD "ld.global"
#endif

__device__ __forceinline__ uint4 coot_ld16(const void* p) {
  uint4 r;
  asm(COOT_LD ".v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}
__device__ __forceinline__ uint2 coot_ld8(const void* p) {
  uint2 r;
  asm(COOT_LD ".v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ coot_u32 coot_ld4(const void* p) {
  coot_u32 r;
  asm(COOT_LD ".u32 %0, [%1];" : "=r"(r) : "l"(p));
  return r;
}
__device__ __forceinline__ coot_u16 coot_ld2(const void* p) {
  coot_u16 r;
  asm(COOT_LD ".u16 %0, [%1];" : "=h"(r) : "l"(p));
  return r;
}
__device__ __forceinline__ void coot_st16(void* p, uint4 v) {
  asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};"
               :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}
__device__ __forceinline__ void coot_st8(void* p, uint2 v) {
  asm volatile("st.global.v2.u32 [%0], {%1, %2};" :: "l"(p), "r"(v.x), "r"(v.y) : "memory");
}
__device__ __forceinline__ void coot_st4(void* p, coot_u32 v) {
  asm volatile("st.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void coot_st2(void* p, coot_u16 v) {
  asm volatile("st.global.u16 [%0], %1;" :: "l"(p), "h"(v) : "memory");
}

// V consecutive elements of storage S at p (p aligned to V * sizeof(T))
template <int S, int V>
__device__ __forceinline__ void coot_vload(const typename coot_st<S>::T* p, COOT_REAL* x) {
  typedef typename coot_st<S>::T T;
  constexpr int B = V * (int)sizeof(T);
  union {
    uint4 q[B >= 16 ? B / 16 : 1];
    uint2 d;
    coot_u32 w;
    coot_u16 h;
    T e[V];
  } u;
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i) u.q[i] = coot_ld16((const char*)p + 16 * i);
  } else if constexpr (B == 8) {
    u.d = coot_ld8(p);
  } else if constexpr (B == 4) {
    u.w = coot_ld4(p);
  } else {
    u.h = coot_ld2(p);
  }
  if constexpr (S == 1 && B % 4 == 0 && sizeof(COOT_REAL) == 4) {
    // BF16 pairs widened with a byte permute (low half) and a mask (high
    // half), both integer-pipe instructions, which leaves the FMA pipes to
    // the arithmetic of the 2-byte reductions
    const coot_u32* w = (const coot_u32*)u.e;
#pragma unroll
    for (int i = 0; i < V / 2; ++i) {
      coot_u32 lo;
      asm("prmt.b32 %0, %1, %2, 0x1044;" : "=r"(lo) : "r"(w[i]), "r"(0u));
      x[2 * i] = __uint_as_float(lo);
      x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = coot_to_real<S>(u.e[v]);
  }
}

template <int S>
__device__ __forceinline__ COOT_REAL coot_sload(const typename coot_st<S>::T* p) {
  typedef typename coot_st<S>::T T;
  if constexpr (sizeof(T) == 8) {
    uint2 r = coot_ld8(p);
    return coot_to_real<S>(__longlong_as_double(((coot_i64)r.y << 32) | r.x));
  } else if constexpr (sizeof(T) == 4) {
    union {
      coot_u32 w;
      T e;
    } u;
    u.w = coot_ld4(p);
    return coot_to_real<S>(u.e);
  } else {
    return coot_to_real<S>(coot_ld2(p));
  }
}

template <int S, int V>
__device__ __forceinline__ void coot_vstore(typename coot_st<S>::T* p, const COOT_REAL* y) {
  typedef typename coot_st<S>::T T;
  constexpr int B = V * (int)sizeof(T);
  union {
    uint4 q[B >= 16 ? B / 16 : 1];
    uint2 d;
    coot_u32 w;
    coot_u16 h;
    T e[V];
  } u;
#pragma unroll
  for (int v = 0; v < V; ++v) u.e[v] = coot_from_real<S>(y[v]);
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i) coot_st16((char*)p + 16 * i, u.q[i]);
  } else if constexpr (B == 8) {
    coot_st8(p, u.d);
  } else if constexpr (B == 4) {
    coot_st4(p, u.w);
  } else {
    coot_st2(p, u.h);
  }
}

template <int S>
__device__ __forceinline__ void coot_sstore(typename coot_st<S>::T* p, COOT_REAL y) {
  *p = coot_from_real<S>(y);
}

template <int I> struct coot_in_code;
template <> struct coot_in_code<0> { static constexpr int S = COOT_TI0; };
template <> struct coot_in_code<1> { static constexpr int S = COOT_TI1; };
template <> struct coot_in_code<2> { static constexpr int S = COOT_TI2; };
template <> struct coot_in_code<3> { static constexpr int S = COOT_TI3; };

// VEC elements of every input at (row, j)
__device__ __forceinline__ void coot_load_vec(const coot_params& p, coot_i64 j, coot_i64 row,
                                              COOT_REAL (&x)[4][COOT_VEC]) {
#define COOT_LOAD_ONE(I)                                                                  \
  if constexpr (I < COOT_NIN) {                                                           \
    constexpr int S = coot_in_code<I>::S;                                                 \
    typedef typename coot_st<S>::T T;                                                     \
    coot_vload<S, COOT_VEC>((const T*)p.in[I] + (j * p.ld_in[I] + row), x[I]);           \
  } else {                                                                                \
    _Pragma("unroll") for (int v = 0; v < COOT_VEC; ++v) x[I][v] = (COOT_REAL)0;          \
  }
  COOT_LOAD_ONE(0)
  COOT_LOAD_ONE(1)
  COOT_LOAD_ONE(2)
  COOT_LOAD_ONE(3)
#undef COOT_LOAD_ONE
}

// one element of every input at (row, j)
__device__ __forceinline__ void coot_load_one(const coot_params& p, coot_i64 j, coot_i64 row,
                                              COOT_REAL (&x)[4]) {
#define COOT_LOAD_S(I)                                                                    \
  if constexpr (I < COOT_NIN) {                                                           \
    constexpr int S = coot_in_code<I>::S;                                                 \
    typedef typename coot_st<S>::T T;                                                     \
    x[I] = coot_sload<S>((const T*)p.in[I] + (j * p.ld_in[I] + row));                    \
  } else {                                                                                \
    x[I] = (COOT_REAL)0;                                                                  \
  }
  COOT_LOAD_S(0)
  COOT_LOAD_S(1)
  COOT_LOAD_S(2)
  COOT_LOAD_S(3)
#undef COOT_LOAD_S
}

// ---------------------------------------------------------------- arithmetic helpers

// NaN-propagating minimum / maximum
__device__ __forceinline__ float coot_min(float a, float b) {
  float r;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float coot_max(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ double coot_min(double a, double b) {
  return (a != a) ? a : ((b != b) ? b : fmin(a, b));
}
__device__ __forceinline__ double coot_max(double a, double b) {
  return (a != a) ? a : ((b != b) ? b : fmax(a, b));
}

// s + c += x with TwoSum (Knuth): the rounding error of every addition is
// carried in c, so the pair holds the running sum to about twice the
// working precision.
__device__ __forceinline__ void coot_two_sum(COOT_REAL& s, COOT_REAL& c, COOT_REAL x) {
  const COOT_REAL t = s + x;
  const COOT_REAL bp = t - s;
  const COOT_REAL e = (s - (t - bp)) + (x - bp);
  s = t;
  c += e;
}

// ---------------------------------------------------------------- double-word sums
//
// Values that are combined across threads travel as unevaluated pairs
// (hi, lo) of the compute type ("double-word" numbers): on this GPU FP64
// arithmetic runs at 1/64 of the FP32 rate, so FP64 is kept for the one
// conversion per block and the final combine of the block partials.  The
// pair addition is the accurate double-word sum of Joldes, Muller and
// Popescu ("Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 2017), relative error about 3u^2.

// s + e = a + b exactly, if |a| >= |b| or a == 0 (Dekker's Fast2Sum)
__device__ __forceinline__ void coot_fast_two(COOT_REAL a, COOT_REAL b, COOT_REAL& s, COOT_REAL& e) {
  s = a + b;
  e = b - (s - a);
}

// s + e = a + b exactly, any a, b (Knuth's TwoSum)
__device__ __forceinline__ void coot_two(COOT_REAL a, COOT_REAL b, COOT_REAL& s, COOT_REAL& e) {
  s = a + b;
  const COOT_REAL bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// (xh, xl) += (yh, yl); both pairs normalised (|lo| <= ulp(hi) / 2).  A
// non-finite high part is passed on with a zero low part.
__device__ __forceinline__ void coot_dw_add(COOT_REAL& xh, COOT_REAL& xl, COOT_REAL yh, COOT_REAL yl) {
  COOT_REAL sh, sl, th, tl, vh, vl, zh, zl;
  coot_two(xh, yh, sh, sl);
  coot_two(xl, yl, th, tl);
  sl = sl + th;
  coot_fast_two(sh, sl, vh, vl);
  vl = vl + tl;
  coot_fast_two(vh, vl, zh, zl);
  const bool fin = isfinite(sh);
  xh = fin ? zh : sh;
  xl = fin ? zl : (COOT_REAL)0;
}

// a running (sum, compensation) pair as a normalised double-word number
__device__ __forceinline__ void coot_dw_norm(COOT_REAL s, COOT_REAL c, COOT_REAL& h, COOT_REAL& l) {
  coot_two(s, c, h, l);
  if (!isfinite(s)) {
    h = s;
    l = (COOT_REAL)0;
  }
}

// warp sum of double-word numbers (fixed shuffle tree; the result is valid
// in lane 0)
__device__ __forceinline__ void coot_dw_warp_sum(COOT_REAL& h, COOT_REAL& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const COOT_REAL yh = __shfl_down_sync(0xffffffffu, h, o);
    const COOT_REAL yl = __shfl_down_sync(0xffffffffu, l, o);
    coot_dw_add(h, l, yh, yl);
  }
}

__device__ __forceinline__ double coot_dw_to_double(COOT_REAL h, COOT_REAL l) {
  const double hd = (double)h;
  return isfinite(hd) ? hd + (double)l : hd;
}

// A double-word sum stored in storage type S: FP64 storage gets h + l in
// FP64; any other type gets h + l rounded in the compute type (one rounding
// of the normalised pair, no FP64 instruction), then converted.
template <int S>
__device__ __forceinline__ typename coot_st<S>::T coot_dw_store(COOT_REAL h, COOT_REAL l) {
  if constexpr (S == 3) {
    return coot_dw_to_double(h, l);
  } else {
    return coot_from_real<S>(isfinite(h) ? h + l : h);
  }
}

// the pair as one FP64 value; once the sum is infinite or NaN the
// compensation carries inf - inf and is dropped
__device__ __forceinline__ double coot_pair(COOT_REAL s, COOT_REAL c) {
  const double sd = (double)s;
  return isfinite(sd) ? sd + (double)c : sd;
}

__device__ __forceinline__ COOT_REAL coot_sq(COOT_REAL y) {
  // a separate rounding of the square: the TwoSum that follows relies on it
  if constexpr (sizeof(COOT_REAL) == 4) {
    return __fmul_rn(y, y);
  } else {
    return __dmul_rn(y, y);
  }
}

__device__ __forceinline__ COOT_REAL coot_abs(COOT_REAL y) {
  if constexpr (sizeof(COOT_REAL) == 4) {
    return fabsf(y);
  } else {
    return fabs(y);
  }
}

// Pairwise sum of V values (what = 0: the values, 1: their squares, each
// rounded separately, 2: their magnitudes): ((y0 + y1) + (y2 + y3)) + ...
template <int V>
__device__ __forceinline__ COOT_REAL coot_pairwise(const COOT_REAL* y, int what) {
  COOT_REAL t[V];
#pragma unroll
  for (int v = 0; v < V; ++v) t[v] = what == 0 ? y[v] : (what == 1 ? coot_sq(y[v]) : coot_abs(y[v]));
#pragma unroll
  for (int w = 1; w < V; w *= 2)
#pragma unroll
    for (int v = 0; v + w < V; v += 2 * w) t[v] = t[v] + t[v + w];
  return t[0];
}

// ---------------------------------------------------------------- packed FP32 pairs
//
// sm_100-family FP32 pair instructions (add / sub / mul .rn.f32x2) carry two
// independent lanes in one 64-bit register and one instruction; with the
// explicit rounding mode they are never contracted into FMAs, so TwoSum keeps
// its exactness lane by lane.  They halve the instruction count of the
// per-element sums that otherwise make 2-byte inputs issue-bound.
#if !COOT_REAL_F64
typedef coot_u64 coot_f2;
__device__ __forceinline__ coot_f2 coot_pack(float a, float b) {
  coot_f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void coot_unpack(coot_f2 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ coot_f2 coot_add2(coot_f2 a, coot_f2 b) {
  coot_f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ coot_f2 coot_sub2(coot_f2 a, coot_f2 b) {
  coot_f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ coot_f2 coot_mul2(coot_f2 a, coot_f2 b) {
  coot_f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// two TwoSums, one per lane
__device__ __forceinline__ void coot_two_sum2(coot_f2& s, coot_f2& c, coot_f2 x) {
  const coot_f2 t = coot_add2(s, x);
  const coot_f2 bp = coot_sub2(t, s);
  const coot_f2 e = coot_add2(coot_sub2(s, coot_sub2(t, bp)), coot_sub2(x, bp));
  s = t;
  c = coot_add2(c, e);
}
// Pairwise sum of V (even) values, what = 1: their squares (each rounded),
// 2: their magnitudes, as one packed pair: lanes hold the even and odd
// elements, each added in a tree of depth log2(V / 2).
template <int V>
__device__ __forceinline__ coot_f2 coot_pairwise2(const float* y, int what) {
  coot_f2 t[V / 2];
#pragma unroll
  for (int v = 0; v < V / 2; ++v) {
    const coot_f2 p = coot_pack(y[2 * v], y[2 * v + 1]);
    t[v] = what == 1 ? coot_mul2(p, p) : (p & 0x7fffffff7fffffffull);
  }
#pragma unroll
  for (int w = 1; w < V / 2; w *= 2)
#pragma unroll
    for (int v = 0; v + w < V / 2; v += 2 * w) t[v] = coot_add2(t[v], t[v + w]);
  return t[0];
}
#endif

#if !COOT_REAL_F64
// (h, l) += both lanes of a packed (sum, compensation) pair, each lane an
// exact pair normalised first
__device__ __forceinline__ void coot_add_lanes(coot_f2 s2, coot_f2 c2, float& h, float& l) {
  float sa, sb, ca, cb;
  coot_unpack(s2, sa, sb);
  coot_unpack(c2, ca, cb);
  float ha, la, hb, lb;
  coot_dw_norm(sa, ca, ha, la);
  coot_dw_norm(sb, cb, hb, lb);
  coot_dw_add(h, l, ha, la);
  coot_dw_add(h, l, hb, lb);
}
#endif

// ---------------------------------------------------------------- accumulators

#ifndef COOT_HEADS
#define COOT_HEADS 0
#endif
#if COOT_KIND == 0 || COOT_KIND == 1
#define COOT_NHEADS (((COOT_HEADS >> 0) & 1) + ((COOT_HEADS >> 1) & 1) + ((COOT_HEADS >> 2) & 1) + \
                     ((COOT_HEADS >> 3) & 1) + ((COOT_HEADS >> 4) & 1) + ((COOT_HEADS >> 5) & 1) + \
                     ((COOT_HEADS >> 6) & 1) + ((COOT_HEADS >> 7) & 1) + ((COOT_HEADS >> 8) & 1) + \
                     ((COOT_HEADS >> 9) & 1))
#else
#define COOT_NHEADS 0
#endif

// all / any: 1 for a nonzero value (NaN included), else 0
__device__ __forceinline__ COOT_REAL coot_nonzero(COOT_REAL y) { return y != (COOT_REAL)0 ? (COOT_REAL)1 : (COOT_REAL)0; }

// The extremum of V values (W = 0: min, 1: max, 2: min of magnitudes,
// 3: max of magnitudes, 4: min of nonzero indicators, 5: max of them), as
// a tree of depth log2 V.
template <int V, int W>
__device__ __forceinline__ COOT_REAL coot_tree_ext(const COOT_REAL* y) {
  COOT_REAL t[V];
#pragma unroll
  for (int v = 0; v < V; ++v) t[v] = (W == 2 || W == 3) ? coot_abs(y[v]) : (W >= 4 ? coot_nonzero(y[v]) : y[v]);
#pragma unroll
  for (int w = 1; w < V; w *= 2)
#pragma unroll
    for (int v = 0; v + w < V; v += 2 * w) t[v] = (W % 2 == 0) ? coot_min(t[v], t[v + w]) : coot_max(t[v], t[v + w]);
  return t[0];
}

// Per-thread accumulators of the reduction heads in the mask H
// (COOT_HEAD_* bits).
template <unsigned H>
struct coot_acc_h {
  COOT_REAL s, sc;   // sum
  COOT_REAL q, qc;   // sum of squares
  COOT_REAL a, ac;   // sum of magnitudes
  COOT_REAL mn, mx;  // min, max
  COOT_REAL mna, mxa;  // min, max magnitude
  COOT_REAL alz, anz;  // all: smallest nonzero indicator; any: largest
#if !COOT_REAL_F64
  // packed accumulators, two lanes each (even and odd elements): the sum in
  // two chains (alternate pairs of a vector), squares and magnitudes in one
  coot_f2 s2[2], sc2[2], q2, qc2, a2, ac2;
#endif

  __device__ __forceinline__ void init() {
#if !COOT_REAL_F64
    s2[0] = s2[1] = sc2[0] = sc2[1] = q2 = qc2 = a2 = ac2 = 0ull;
#endif
    s = sc = q = qc = a = ac = (COOT_REAL)0;
    mn = mna = alz = (COOT_REAL)COOT_INF_F;
    mx = anz = -(COOT_REAL)COOT_INF_F;
    mxa = (COOT_REAL)0;
  }
  __device__ __forceinline__ void add(COOT_REAL y) {
    if constexpr ((H & COOT_HEAD_SUM) != 0) coot_two_sum(s, sc, y);
    if constexpr ((H & (COOT_HEAD_SUMSQ | COOT_HEAD_NORM2)) != 0) coot_two_sum(q, qc, coot_sq(y));
    if constexpr ((H & COOT_HEAD_SUMABS) != 0) coot_two_sum(a, ac, coot_abs(y));
    if constexpr ((H & COOT_HEAD_MIN) != 0) mn = coot_min(mn, y);
    if constexpr ((H & COOT_HEAD_MAX) != 0) mx = coot_max(mx, y);
    if constexpr ((H & COOT_HEAD_MINABS) != 0) mna = coot_min(mna, coot_abs(y));
    if constexpr ((H & COOT_HEAD_MAXABS) != 0) mxa = coot_max(mxa, coot_abs(y));
    if constexpr ((H & COOT_HEAD_ALL) != 0) alz = coot_min(alz, coot_nonzero(y));
    if constexpr ((H & COOT_HEAD_ANY) != 0) anz = coot_max(anz, coot_nonzero(y));
  }
  // V consecutive values.  The plain sum adds every value with TwoSum (no
  // rounding is lost however the terms cancel).  Sums of squares and of
  // magnitudes have no cancellation: their vector is added pairwise (a tree
  // of depth log2 V) and the result enters the running pair with one
  // TwoSum, which keeps 2-byte inputs memory-bound.  Extrema are taken
  // element by element.
  // (SKIP: heads whose values this call leaves out, e.g. a plain sum that
  // the caller feeds from already-summed pairs with add_pair)
  template <int V, unsigned SKIP = 0u>
  __device__ __forceinline__ void add_vec(const COOT_REAL* y) {
    constexpr unsigned HH = H & ~SKIP;
#if !COOT_REAL_F64
    constexpr bool packed = V % 2 == 0;
#else
    constexpr bool packed = false;
#endif
    if constexpr (packed) {
#if !COOT_REAL_F64
      if constexpr ((HH & COOT_HEAD_SUM) != 0) {
#pragma unroll
        for (int v = 0; v < V / 2; ++v) coot_two_sum2(s2[v & 1], sc2[v & 1], coot_pack(y[2 * v], y[2 * v + 1]));
      }
      if constexpr ((HH & (COOT_HEAD_SUMSQ | COOT_HEAD_NORM2)) != 0) coot_two_sum2(q2, qc2, coot_pairwise2<V>(y, 1));
      if constexpr ((HH & COOT_HEAD_SUMABS) != 0) coot_two_sum2(a2, ac2, coot_pairwise2<V>(y, 2));
#endif
    } else {
      if constexpr ((HH & (COOT_HEAD_SUMSQ | COOT_HEAD_NORM2)) != 0) coot_two_sum(q, qc, coot_pairwise<V>(y, 1));
      if constexpr ((HH & COOT_HEAD_SUMABS) != 0) coot_two_sum(a, ac, coot_pairwise<V>(y, 2));
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if constexpr ((HH & COOT_HEAD_SUM) != 0 && !packed) coot_two_sum(s, sc, y[v]);
    }
    // extrema: the V values in a tree of depth log2 V first, then one step
    // of the running value (exact in any order; NaN propagates either way),
    // so the running chain grows by one instruction per vector
    if constexpr ((HH & COOT_HEAD_MIN) != 0) mn = coot_min(mn, coot_tree_ext<V, 0>(y));
    if constexpr ((HH & COOT_HEAD_MAX) != 0) mx = coot_max(mx, coot_tree_ext<V, 1>(y));
    if constexpr ((HH & COOT_HEAD_MINABS) != 0) mna = coot_min(mna, coot_tree_ext<V, 2>(y));
    if constexpr ((HH & COOT_HEAD_MAXABS) != 0) mxa = coot_max(mxa, coot_tree_ext<V, 3>(y));
    if constexpr ((HH & COOT_HEAD_ALL) != 0) alz = coot_min(alz, coot_tree_ext<V, 4>(y));
    if constexpr ((HH & COOT_HEAD_ANY) != 0) anz = coot_max(anz, coot_tree_ext<V, 5>(y));
  }
  // the plain sum's share of a normalised double-word partial sum (h, l):
  // h enters the running pair with TwoSum, l its compensation
  __device__ __forceinline__ void add_pair(COOT_REAL h, COOT_REAL l) {
    if constexpr ((H & COOT_HEAD_SUM) != 0) {
      coot_two_sum(s, sc, h);
      sc += l;
    }
  }
  // per-head values as FP64, in head-bit order
  // per-head values as double-word pairs in head-bit order (sums
  // normalised; extrema as (value, 0))
  __device__ __forceinline__ void values(COOT_REAL* h, COOT_REAL* l) const {
    int k = 0;
    if constexpr ((H & COOT_HEAD_SUM) != 0) {
      coot_dw_norm(s, sc, h[k], l[k]);
#if !COOT_REAL_F64
      coot_add_lanes(s2[0], sc2[0], h[k], l[k]);
      coot_add_lanes(s2[1], sc2[1], h[k], l[k]);
#endif
      ++k;
    }
    // sums of squares and magnitudes: the scalar pair plus the packed lanes
    COOT_REAL qh, ql, ah, al;
    coot_dw_norm(q, qc, qh, ql);
    coot_dw_norm(a, ac, ah, al);
#if !COOT_REAL_F64
    coot_add_lanes(q2, qc2, qh, ql);
    coot_add_lanes(a2, ac2, ah, al);
#endif
    if constexpr ((H & COOT_HEAD_SUMSQ) != 0) { h[k] = qh; l[k] = ql; ++k; }
    if constexpr ((H & COOT_HEAD_NORM2) != 0) { h[k] = qh; l[k] = ql; ++k; }
    if constexpr ((H & COOT_HEAD_SUMABS) != 0) { h[k] = ah; l[k] = al; ++k; }
    if constexpr ((H & COOT_HEAD_MIN) != 0) { h[k] = mn; l[k] = 0; ++k; }
    if constexpr ((H & COOT_HEAD_MAX) != 0) { h[k] = mx; l[k] = 0; ++k; }
    if constexpr ((H & COOT_HEAD_MINABS) != 0) { h[k] = mna; l[k] = 0; ++k; }
    if constexpr ((H & COOT_HEAD_MAXABS) != 0) { h[k] = mxa; l[k] = 0; ++k; }
    if constexpr ((H & COOT_HEAD_ALL) != 0) { h[k] = alz; l[k] = 0; ++k; }
    if constexpr ((H & COOT_HEAD_ANY) != 0) { h[k] = anz; l[k] = 0; ++k; }
    (void)k;
  }
};
typedef coot_acc_h<COOT_HEADS> coot_acc;

// combine rule of head number k of the mask H (in bit order among the set
// bits)
template <unsigned H>
__device__ __forceinline__ unsigned coot_head_bit_of(int k) {
  unsigned m = H;
  for (int i = 0; i < k; ++i) m &= m - 1;
  return m & (~m + 1);
}
__device__ __forceinline__ unsigned coot_head_bit(int k) { return coot_head_bit_of<COOT_HEADS>(k); }

// heads combined by a minimum / a maximum (the rest are sums)
__device__ __forceinline__ bool coot_min_head(unsigned bit) {
  return bit == COOT_HEAD_MIN || bit == COOT_HEAD_MINABS || bit == COOT_HEAD_ALL;
}
__device__ __forceinline__ bool coot_max_head(unsigned bit) {
  return bit == COOT_HEAD_MAX || bit == COOT_HEAD_MAXABS || bit == COOT_HEAD_ANY;
}

__device__ __forceinline__ double coot_combine(unsigned bit, double a, double b) {
  if (coot_min_head(bit)) return coot_min(a, b);
  if (coot_max_head(bit)) return coot_max(a, b);
  return a + b;
}

__device__ __forceinline__ double coot_identity(unsigned bit) {
  if (coot_min_head(bit)) return COOT_INF_D;
  if (bit == COOT_HEAD_MAX || bit == COOT_HEAD_ANY) return -COOT_INF_D;
  return 0.0;
}

#if COOT_NHEADS > 0 || COOT_KIND == 7 || COOT_KIND == 8
__device__ __forceinline__ COOT_REAL coot_identity_r(unsigned bit) {
  if (coot_min_head(bit)) return (COOT_REAL)COOT_INF_F;
  if (bit == COOT_HEAD_MAX || bit == COOT_HEAD_ANY) return -(COOT_REAL)COOT_INF_F;
  return (COOT_REAL)0;
}

// head `bit`'s combine of two double-word values
__device__ __forceinline__ void coot_combine_dw(unsigned bit, COOT_REAL& h, COOT_REAL& l, COOT_REAL yh, COOT_REAL yl) {
  if (coot_min_head(bit)) {
    h = coot_min(h, yh);
  } else if (coot_max_head(bit)) {
    h = coot_max(h, yh);
  } else {
    coot_dw_add(h, l, yh, yl);
  }
}

// Block-level combine of NH heads in double-word arithmetic (head k,
// this thread's value (h[k], l[k]), combined by the rule bit(k)), one FP64
// partial per block and head, and the last-arriving block's ordered FP64
// combine of the partials into p.res[0 .. NH).
template <int NH, typename Bit>
__device__ void coot_finish_heads(COOT_REAL (&h)[NH], COOT_REAL (&l)[NH], Bit bit_of, const coot_params& p) {
  __shared__ COOT_REAL red_h[NH][COOT_WARPS];
  __shared__ COOT_REAL red_l[NH][COOT_WARPS];
  __shared__ double red64[COOT_WARPS];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    const unsigned bit = bit_of(k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const COOT_REAL yh = __shfl_down_sync(0xffffffffu, h[k], o);
      const COOT_REAL yl = __shfl_down_sync(0xffffffffu, l[k], o);
      coot_combine_dw(bit, h[k], l[k], yh, yl);
    }
    if (lane == 0) {
      red_h[k][warp] = h[k];
      red_l[k][warp] = l[k];
    }
  }
  __syncthreads();
  double* part = (double*)(p.ws + COOT_WS_PARTIALS_OFF);
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      const unsigned bit = bit_of(k);
      COOT_REAL wh = lane < COOT_WARPS ? red_h[k][lane] : coot_identity_r(bit);
      COOT_REAL wl = lane < COOT_WARPS ? red_l[k][lane] : (COOT_REAL)0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const COOT_REAL yh = __shfl_down_sync(0xffffffffu, wh, o);
        const COOT_REAL yl = __shfl_down_sync(0xffffffffu, wl, o);
        coot_combine_dw(bit, wh, wl, yh, yl);
      }
      if (lane == 0) part[(coot_i64)k * gridDim.x + blockIdx.x] = coot_dw_to_double(wh, wl);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    coot_u32* counter = (coot_u32*)(p.ws + COOT_WS_COUNTER_OFF);
    is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // the last block: every thread folds a strided subset of the partials in
  // index order (FP64), then the block combines the thread results
  for (int k = 0; k < NH; ++k) {
    const unsigned bit = bit_of(k);
    double w = coot_identity(bit);
    for (coot_u32 b = threadIdx.x; b < gridDim.x; b += COOT_BLOCK)
      w = coot_combine(bit, w, __ldcg(part + (coot_i64)k * gridDim.x + b));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = coot_combine(bit, w, __shfl_down_sync(0xffffffffu, w, o));
    __syncthreads();
    if (lane == 0) red64[warp] = w;
    __syncthreads();
    if (warp == 0) {
      w = lane < COOT_WARPS ? red64[lane] : coot_identity(bit);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w = coot_combine(bit, w, __shfl_down_sync(0xffffffffu, w, o));
      // norm2 is the root of its sum; all / any become 1 or 0 (an empty
      // object leaves the identities +inf / -inf)
      if (lane == 0)
        p.res[k] = (bit == COOT_HEAD_NORM2) ? sqrt(w)
                   : (bit == COOT_HEAD_ALL || bit == COOT_HEAD_ANY) ? (w > 0.0 ? 1.0 : 0.0) : w;
    }
  }
  if (threadIdx.x == 0) *(coot_u32*)(p.ws + COOT_WS_COUNTER_OFF) = 0u;
}

#if COOT_NHEADS > 0
// every head of the kernel's mask COOT_HEADS
__device__ void coot_finish_full(const coot_acc& acc, const coot_params& p) {
  COOT_REAL h[COOT_NHEADS], l[COOT_NHEADS];
  acc.values(h, l);
  coot_finish_heads<COOT_NHEADS>(h, l, [](int k) { return coot_head_bit(k); }, p);
}
#endif

#endif
