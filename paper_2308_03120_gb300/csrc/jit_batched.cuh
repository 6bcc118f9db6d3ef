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
// handled by one block; units hold up to about 2K elements (whole columns),
// so the cost of reading the unit and its matrix descriptor is spread over
// many loads.
struct coot_work_d {
  int item;
  int col0;
  int n_cols;
  int pad;
};

#if COOT_KIND == 4
// element (row, j) of every input of a batch item (strided)
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

// element e of every input's flat (dense) run
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
// Up to four blocks per SM, each warp-specialised: a producer warp copies
// the next dense units' inputs into a ring of shared-memory stages with bulk
// asynchronous copies (cp.async.bulk, completion counted in bytes on the
// stage's `full` mbarrier) while the consumer warps compute the current
// unit from another stage.  A unit qualifies when every operand is dense
// (its columns are one contiguous run), it holds at most COOT_UNIT
// elements, and every input run starts on a 16-byte boundary; the run's
// last bytes beyond a multiple of 16 are read directly.
//
// A staged unit: every consumer thread takes COOT_VEC elements at a time
// from the stage (16-byte shared-memory accesses), writes the values and
// keeps them in shared memory (over input 0 when the types allow); the
// column sums are then taken from shared memory, a warp per column from 256
// rows up and g lanes per column below that (each lane adding 8 or more
// values, then a double-word shuffle sum over the g lanes), each in a fixed
// order.  Other units (strided, unaligned or too large): consumer warp w
// takes columns w, w + warps, ... from global memory; lanes stride down the
// rows.
//
// Every wait in the kernel is bounded, and no thread waits at a barrier that
// a thread which gave up could leave unfilled.  After the one block-wide
// barrier at the start, threads meet only on mbarriers, each waited on with
// a bounded try_wait: the consumers' `full` stages, the producer's `empty`
// stages and the consumers' per-unit barrier `cons` (one arrival per
// consumer warp).  Each warp votes on every wait's outcome (__all_sync), so
// its lanes leave together and the warp-wide shuffles keep every lane.  A
// warp that gives up records COOT_ERR_TIMEOUT in the status word (p.res)
// and returns; the warps that depended on it then run out their own
// bounded waits and return too.  Before the producer returns, by any path,
// it waits (bounded) for the bulk copies it started, so no copy lands in
// shared memory after the block has left.
#define COOT_UNIT 2048
template <int I>
struct coot_in_bytes {
  static constexpr int B = I < COOT_NIN ? (int)sizeof(typename coot_st<coot_in_code<I>::S>::T) * COOT_UNIT : 0;
};
#define COOT_BUF_BYTES (coot_in_bytes<0>::B + coot_in_bytes<1>::B + coot_in_bytes<2>::B + coot_in_bytes<3>::B)
#define COOT_VALS_IN_PLACE (sizeof(typename coot_st<COOT_TI0>::T) == sizeof(COOT_REAL))

__device__ __forceinline__ unsigned coot_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// bounded wait for phase `parity` of the mbarrier at bar
__device__ __forceinline__ bool coot_mbar_wait(unsigned bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 22); ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it >= 64) __nanosleep(128);
  }
  return false;
}

// input k's slot in a buffer
template <int I>
__device__ __forceinline__ int coot_slot_off() {
  int o = 0;
  if constexpr (I > 0) o += coot_in_bytes<0>::B;
  if constexpr (I > 1) o += coot_in_bytes<1>::B;
  if constexpr (I > 2) o += coot_in_bytes<2>::B;
  return o;
}

// a stage's unit: its matrix descriptor and work-list entry (pad = 1 when
// the unit's inputs are staged)
struct coot_stage_hdr {
  coot_batch_item_d it;
  coot_work_d wk;
};
static_assert(sizeof(coot_batch_item_d) == 112 && sizeof(coot_stage_hdr) == 128, "stage header layout");

// The producer warp: write unit (work entry wk, this lane's word iw of the
// unit's matrix descriptor) into the header h; when the unit qualifies,
// lane 0 starts the bulk copies of its inputs into buf, counted on the
// full mbarrier bar, else it arrives on bar at once.  The consumers
// released buf through its empty mbarrier; the proxy fence orders their
// accesses before the copies.
__device__ __forceinline__ void coot_stage_unit(const coot_params& p, int4 wk, unsigned long long iw, int lane,
                                                coot_stage_hdr* h, unsigned char* buf, unsigned bar) {
  if (lane < 14) ((unsigned long long*)&h->it)[lane] = iw;
  __syncwarp();
  if (lane == 0) {
    const coot_batch_item_d& it = h->it;
    const coot_i64 R = it.n_rows, n = (coot_i64)wk.z * R, b0 = (coot_i64)wk.y * R;
    bool ok = n > 0 && n <= COOT_UNIT && (it.out == nullptr || it.ld_out == R);
    unsigned tx = 0;
#define COOT_CHECK_IN(I)                                                                    \
  if constexpr (I < COOT_NIN) {                                                             \
    typedef typename coot_st<coot_in_code<I>::S>::T T;                                      \
    const T* src = (const T*)it.in[I] + b0;                                                 \
    const unsigned bytes16 = (unsigned)(n * (coot_i64)sizeof(T)) & ~15u;                    \
    ok = ok && it.ld_in[I] == R && ((unsigned long long)src & 15ull) == 0 && bytes16 > 0;   \
    tx += bytes16;                                                                          \
  }
    COOT_CHECK_IN(0)
    COOT_CHECK_IN(1)
    COOT_CHECK_IN(2)
    COOT_CHECK_IN(3)
#undef COOT_CHECK_IN
    h->wk = coot_work_d{wk.x, wk.y, wk.z, ok ? 1 : 0};
    // p.n_cols == 1 is the status test: the unit is marked staged but no
    // copy is started, so its wait runs out (nothing is in flight)
    if (ok && p.n_cols != 1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
#define COOT_COPY_IN(I)                                                                     \
  if constexpr (I < COOT_NIN) {                                                             \
    typedef typename coot_st<coot_in_code<I>::S>::T T;                                      \
    const T* src = (const T*)it.in[I] + b0;                                                 \
    const unsigned bytes16 = (unsigned)(n * (coot_i64)sizeof(T)) & ~15u;                    \
    asm volatile(                                                                           \
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" \
        ::"r"(coot_smem_addr(buf + coot_slot_off<I>())), "l"(src), "r"(bytes16), "r"(bar)   \
        : "memory");                                                                        \
  }
      COOT_COPY_IN(0)
      COOT_COPY_IN(1)
      COOT_COPY_IN(2)
      COOT_COPY_IN(3)
#undef COOT_COPY_IN
    } else if (!ok) {
      // read from global memory by the consumers: the header is all they wait for
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    }
  }
  __syncwarp();
}

// V consecutive elements of storage S at shared-memory address a (aligned
// to V * sizeof(T)), one vector access
template <int S, int V>
__device__ __forceinline__ void coot_lds_vec(unsigned a, COOT_REAL* x) {
  typedef typename coot_st<S>::T T;
  constexpr int B = V * (int)sizeof(T);
  union {
    uint4 q[B >= 16 ? B / 16 : 1];
    uint2 d;
    coot_u32 w;
    T e[V];
  } u;
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i)
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(u.q[i].x), "=r"(u.q[i].y), "=r"(u.q[i].z), "=r"(u.q[i].w) : "r"(a + 16 * i));
  } else if constexpr (B == 8) {
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(u.d.x), "=r"(u.d.y) : "r"(a));
  } else if constexpr (B == 4) {
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(u.w) : "r"(a));
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) u.e[v] = ((const T*)__cvta_shared_to_generic(a))[v];
  }
#pragma unroll
  for (int v = 0; v < V; ++v) x[v] = coot_to_real<S>(u.e[v]);
}

// V values of the compute type to shared-memory address a (aligned to
// V * sizeof(COOT_REAL)), 16-byte accesses
template <int V>
__device__ __forceinline__ void coot_sts_real(unsigned a, const COOT_REAL* y) {
  constexpr int B = V * (int)sizeof(COOT_REAL);
  union {
    uint4 q[B >= 16 ? B / 16 : 1];
    COOT_REAL e[V];
  } u;
#pragma unroll
  for (int v = 0; v < V; ++v) u.e[v] = y[v];
  if constexpr (B >= 16 && B % 16 == 0) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i)
      asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};"
                   :: "r"(a + 16 * i), "r"(u.q[i].x), "r"(u.q[i].y), "r"(u.q[i].z), "r"(u.q[i].w) : "memory");
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) ((COOT_REAL*)__cvta_shared_to_generic(a))[v] = y[v];
  }
}

// VEC consecutive staged elements of every input at element e
__device__ __forceinline__ void coot_load_staged(const unsigned char* buf, int e, COOT_REAL (&x)[4][COOT_VEC]) {
  const unsigned base = coot_smem_addr(buf);
#define COOT_LDS(I)                                                                          \
  if constexpr (I < COOT_NIN) {                                                              \
    constexpr int S = coot_in_code<I>::S;                                                    \
    typedef typename coot_st<S>::T T;                                                        \
    coot_lds_vec<S, COOT_VEC>(base + coot_slot_off<I>() + e * (unsigned)sizeof(T), x[I]);   \
  } else {                                                                                   \
    _Pragma("unroll") for (int v = 0; v < COOT_VEC; ++v) x[I][v] = (COOT_REAL)0;             \
  }
  COOT_LDS(0)
  COOT_LDS(1)
  COOT_LDS(2)
  COOT_LDS(3)
#undef COOT_LDS
}

// COOT_BLOCK consumer threads (COOT_WARPS warps) plus one producer warp per
// block (launched with COOT_BLOCK + 32 threads); COOT_STAGES stages of
// inputs in shared memory, each with a `full` mbarrier (the producer's
// arrival and the copied bytes) and an `empty` one (one arrival per
// consumer warp).  The consumers synchronise among themselves once per
// staged unit with column sums (the `cons` mbarrier, one arrival per
// consumer warp, before the column sums) and release a stage with a
// non-blocking arrival, so a warp done with a unit's column sums goes on
// to the next unit while others finish theirs.
#define COOT_STAGES 2
extern "C" __global__ void __launch_bounds__(COOT_BLOCK + 32, (COOT_BLOCK + 32 <= 256 ? 4 : 2))
    COOT_ENTRY(const __grid_constant__ coot_params p) {
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned char* bufs = dsm;                                                   // COOT_STAGES x COOT_BUF_BYTES
  COOT_REAL* vals_sep = (COOT_REAL*)(dsm + COOT_STAGES * COOT_BUF_BYTES);      // per stage, unless in place
  coot_stage_hdr* hdr = (coot_stage_hdr*)(dsm + COOT_STAGES * COOT_BUF_BYTES +
                                          (COOT_VALS_IN_PLACE ? 0 : COOT_STAGES * COOT_UNIT * sizeof(COOT_REAL)));
  unsigned long long* full = (unsigned long long*)(hdr + COOT_STAGES);
  unsigned long long* empty = full + COOT_STAGES;
  unsigned long long* cons = empty + COOT_STAGES;
  typedef typename coot_st<COOT_TO>::T TO;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool sum64 = p.rows_per_split == 3;
  const coot_i64 G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < COOT_STAGES; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(coot_smem_addr(full + k)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(coot_smem_addr(empty + k)), "r"(COOT_WARPS)
                   : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(coot_smem_addr(cons)), "r"(COOT_WARPS) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the only block-wide barrier
  if (warp == 0) {
    // ---- producer: stage the block's units in order, COOT_STAGES ahead of
    // the consumers; the work entry and descriptor of each unit are loaded
    // one unit before it is staged
    const coot_batch_item_d* items = (const coot_batch_item_d*)p.plan;
    const int4* work = (const int4*)(items + p.split);
    const int4 zero4 = make_int4(0, 0, 0, 0);
#define COOT_ITEM_WORD(w, u) \
  ((u) < p.n_work && lane < 14 ? __ldg((const unsigned long long*)(items + (w).x) + lane) : 0ull)
    const coot_i64 u0 = blockIdx.x;
    int4 wk = u0 < p.n_work ? __ldg(work + u0) : zero4;
    unsigned long long iw = COOT_ITEM_WORD(wk, u0);
    int4 wn = u0 + G < p.n_work ? __ldg(work + u0 + G) : zero4;
    unsigned eph = 0u;  // bit s: the parity of empty[s]'s next phase
    unsigned fph = 0u;  // bit s: the parity of full[s]'s phase last armed
    unsigned inflight = 0u;  // bit s: copies into stage s were started
    bool ok = true;
    int st = 0;
    coot_i64 k = 0;
    for (coot_i64 u = u0; u < p.n_work; u += G, ++k) {
      if (k >= COOT_STAGES) {
        ok = __all_sync(0xffffffffu, coot_mbar_wait(coot_smem_addr(empty + st), (eph >> st) & 1u));
        if (!ok) break;
        eph ^= 1u << st;
        fph ^= 1u << st;  // full[st]'s previous phase completed before the consumers released it
      }
      coot_stage_unit(p, wk, iw, lane, &hdr[st], bufs + st * COOT_BUF_BYTES, coot_smem_addr(full + st));
      // whether lane 0 started copies (the header's staged flag, on the
      // normal path; the status test starts none)
      if (hdr[st].wk.pad && p.n_cols != 1) inflight |= 1u << st; else inflight &= ~(1u << st);
      iw = COOT_ITEM_WORD(wn, u + G);
      wk = wn;
      wn = u + 2 * G < p.n_work ? __ldg(work + u + 2 * G) : zero4;
      st = st + 1 == COOT_STAGES ? 0 : st + 1;
    }
#undef COOT_ITEM_WORD
    // wait (bounded) for the copies still in flight: phase fph of full[s]
    // completes once the stage's bytes have landed
    for (int s = 0; s < COOT_STAGES; ++s)
      if ((inflight >> s) & 1u) ok = __all_sync(0xffffffffu, coot_mbar_wait(coot_smem_addr(full + s), (fph >> s) & 1u)) && ok;
    if (!ok && lane == 0 && p.res) atomicExch((unsigned*)p.res, 10u);  // COOT_ERR_TIMEOUT
    return;
  }
  // ---- consumers: thread ct of COOT_BLOCK, warp cw of COOT_WARPS
  const int ct = (int)threadIdx.x - 32, cw = warp - 1;
  unsigned fph = 0u;  // bit s: the parity of full[s]'s next phase
  unsigned cph = 0u;  // the parity of cons's next phase
  int st = 0;
  for (coot_i64 w = blockIdx.x; w < p.n_work; w += G) {
    if (!__all_sync(0xffffffffu, coot_mbar_wait(coot_smem_addr(full + st), (fph >> st) & 1u))) {
      if (lane == 0 && p.res) atomicExch((unsigned*)p.res, 10u);  // COOT_ERR_TIMEOUT
      return;
    }
    fph ^= 1u << st;
    const coot_batch_item_d it = hdr[st].it;
    const coot_work_d wk = hdr[st].wk;
    const coot_i64 R = it.n_rows;
    const coot_i64 c0 = wk.col0, nc = wk.n_cols;
    if (wk.pad) {
      const unsigned char* buf = bufs + st * COOT_BUF_BYTES;
      const int ni = (int)(nc * R);
      const coot_i64 b0 = c0 * R;
      COOT_REAL* vals = COOT_VALS_IN_PLACE ? (COOT_REAL*)buf : vals_sep + st * COOT_UNIT;
      TO* out = it.out ? (TO*)it.out + b0 : (TO*)nullptr;
      // elements staged for every input
      int ns = ni;
#define COOT_NS(I)                                                                           \
  if constexpr (I < COOT_NIN) {                                                              \
    constexpr int E = (int)sizeof(typename coot_st<coot_in_code<I>::S>::T);                  \
    ns = min(ns, (int)(((unsigned)(ni * E) & ~15u) / E));                                    \
  }
      COOT_NS(0)
      COOT_NS(1)
      COOT_NS(2)
      COOT_NS(3)
#undef COOT_NS
      ns -= ns % COOT_VEC;
      const bool va = out == nullptr || coot_aligned16(out);
      for (int e = ct * COOT_VEC; e < ns; e += COOT_BLOCK * COOT_VEC) {
        COOT_REAL xv[4][COOT_VEC];
        coot_load_staged(buf, e, xv);
        COOT_REAL y[COOT_VEC];
#pragma unroll
        for (int k = 0; k < COOT_VEC; ++k) {
          const COOT_REAL x[4] = {xv[0][k], xv[1][k], xv[2][k], xv[3][k]};
          y[k] = coot_f(x);
        }
        if (out) {
          if (va) {
            coot_vstore<COOT_TO, COOT_VEC>(out + e, y);
          } else {
#pragma unroll
            for (int k = 0; k < COOT_VEC; ++k) out[e + k] = coot_from_real<COOT_TO>(y[k]);
          }
        }
        if (it.colsum) coot_sts_real<COOT_VEC>(coot_smem_addr(vals + e), y);
      }
      if (ns < ni) {
        // the last elements of the run, past the copied multiple of 16 bytes
        coot_batch_item_d sh = it;
#define COOT_SHIFT_T(I)                                                                                  \
  if constexpr (I < COOT_NIN) sh.in[I] = (const typename coot_st<coot_in_code<I>::S>::T*)it.in[I] + b0;
        COOT_SHIFT_T(0)
        COOT_SHIFT_T(1)
        COOT_SHIFT_T(2)
        COOT_SHIFT_T(3)
#undef COOT_SHIFT_T
        for (int e = ns + ct; e < ni; e += COOT_BLOCK) {
          COOT_REAL x[4];
          coot_load_flat(sh, e, x);
          const COOT_REAL y = coot_f(x);
          if (out) out[e] = coot_from_real<COOT_TO>(y);
          if (it.colsum) vals[e] = y;
        }
      }
      if (it.colsum) {
        // the consumer warps only (the producer never waits here): each
        // warp's values are in shared memory before its lane 0 arrives
        // (release), and every lane's wait acquires the other warps' values
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(coot_smem_addr(cons)) : "memory");
        if (!__all_sync(0xffffffffu, coot_mbar_wait(coot_smem_addr(cons), cph))) {
          if (lane == 0 && p.res) atomicExch((unsigned*)p.res, 10u);  // COOT_ERR_TIMEOUT
          return;
        }
        cph ^= 1u;
        // g lanes per column, g the largest power of two up to 32 that
        // leaves each lane 8 or more of the column's values (one lane per
        // column below 16 rows), 32 / g columns per warp pass.  Lane `sub`
        // of a column adds rows sub, sub + g, ... in chunks of g rows,
        // starting at a column-dependent chunk so that the columns of one
        // pass read different banks (one lane per column: only for even
        // lengths, odd ones already spread); then the g lanes combine.
        const int Ri = (int)R, nci = (int)nc;
        int g = 32;
        while (g > 1 && g * 8 > Ri) g >>= 1;
        const int cpw = 32 / g, sub = lane & (g - 1);
        const int nch = (Ri + g - 1) / g;
        for (int cb = cw * cpw; cb < nci; cb += COOT_WARPS * cpw) {
          const int jj = cb + lane / g;
          COOT_REAL s = 0, c = 0;
          if (jj < nci) {
            const COOT_REAL* col = vals + jj * Ri;
            if (g == 32) {
              for (int r = lane; r < Ri; r += 32) coot_two_sum(s, c, col[r]);
            } else {
              int ch = (g > 1 || (Ri & 1) == 0) ? jj % nch : 0;
              for (int i = 0; i < nch; ++i) {
                const int r = ch * g + sub;
                if (r < Ri) coot_two_sum(s, c, col[r]);
                if (++ch == nch) ch = 0;
              }
            }
          }
          COOT_REAL vh, vl;
          coot_dw_norm(s, c, vh, vl);
          for (int o = g >> 1; o > 0; o >>= 1) {
            const COOT_REAL yh = __shfl_down_sync(0xffffffffu, vh, o);
            const COOT_REAL yl = __shfl_down_sync(0xffffffffu, vl, o);
            coot_dw_add(vh, vl, yh, yl);
          }
          if (jj < nci && sub == 0) coot_store_colsum(it, c0 + jj, vh, vl, sum64);
        }
      }
    } else {
      // strided, large or unaligned units: a warp per column from global memory
      for (coot_i64 cj = cw; cj < nc; cj += COOT_WARPS) {
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
    // stage st is free for the producer once every consumer warp is done
    // with it (the proxy fence orders this thread's accesses before the
    // next bulk copies into it)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(coot_smem_addr(empty + st)) : "memory");
    st = st + 1 == COOT_STAGES ? 0 : st + 1;
  }
}
#endif
