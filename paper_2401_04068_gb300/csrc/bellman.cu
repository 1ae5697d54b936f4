// Robust Bellman step (Eq. 2 / Eq. 3) with O-maximization (Sec. 4) for sm_103a.
//
// One launch performs one value-iteration step V_{k-1} -> V_k for every problem
// of a batch that is still running.
//
// Data movement. The launch is persistent (one CTA per SM). The model is cut into
// state-aligned tiles (consecutive states of one problem, <= kTileEntries
// entries); states that do not fit a stage or that have columns of kWideCol
// entries or more are "wide" and run in bellman_wide_kernel (a 4-warp CTA per
// state, beside this kernel on a second stream, or before it). A producer warp
// streams each tile's destination indices and bound pairs into a three-stage
// shared-memory ring with bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier), while the consumer warps
// work on the tiles already landed: 15 of them (16 warps, four per SM
// sub-partition, 96 registers per thread), or 23 (24 warps, 80 registers) when
// the tiles hold 16 or more columns on average, where the extra warps hide more
// of the V gathers' latency. Every entry crosses HBM once per iteration.
//
// O-maximization without a sort. For a pessimistic adversary the procedure of
// Sec. 4 orders the destinations by ascending V, starts from p = lower and hands
// out rem = 1 - sum(lower) gap by gap along that order. Its result depends only
// on the threshold: the first destination (in that order) at which the inclusive
// prefix of gaps reaches rem. Everything before it receives its full gap, the
// threshold receives what is left, everything after it keeps its lower bound.
// Destinations with equal V are interchangeable (the sum is the same whichever of
// them gets the mass), so
//     q = sum_i V_i P_lo,i + sum_{V_i < v*} V_i gap_i + v* (rem - sum_{V_i < v*} gap_i),
//     v* = the smallest V_i with sum_{V_j <= V_i} gap_j >= rem.
// Keys are the Q1.63 values (complemented for an optimistic adversary so that the
// order is always ascending). A consumer warp handles one column at a time:
//   0. warm start: the entry that held the threshold in the previous iteration is
//      tried first; one pass over the column checks F(<v) < rem <= F(<=v) exactly
//      and, when it holds (the usual case once V settles), yields q directly;
//      when it fails, one more pass tries the adjacent distinct key in the
//      direction the sums point to (where most thresholds move);
//   1. otherwise it gathers the keys and takes their min/max (redux.sync on
//      32-bit halves);
//   2. histograms the gaps (and counts) into 64 bins of [min, max] and scans the
//      bins: the bin where the prefix crosses rem holds the threshold, entries in
//      lower bins are fully "below";
//   3. compacts the entries of that bin (usually one to a few) into a list of at
//      most 32 and resolves them exactly: each takes its gap, clipped to what the
//      entries before it in (key, position) order leave of rem.
// A crossing bin with more than 32 entries is narrowed by further rounds over its
// key range; a bin whose entries share one key is resolved as a group. Sums are
// exact 64-bit integer sums (gap sums saturate instead of wrapping), so results
// do not depend on the order in which lanes or bins are combined. The warp that
// finishes a tile's last column takes the optimum over each state's actions,
// applies the reach/avoid mask and writes V, the policy and the residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <mutex>

#include "imdp_internal.h"

namespace imdp {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBins = 64;
// Consumer warps per CTA of the tiled kernel (plus one producer warp): 15 (96
// registers per thread) in general, 23 (80 registers) for tiles of many short
// columns, where more warps in flight hide more of the gathers' latency.
constexpr int kConsumersLong = 15;
constexpr int kConsumersShort = 23;
constexpr int kShortColsPerTile = 16;  // mean columns per tile that selects 23
constexpr int kStages = 3;
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz: bound of every wait

// Per-warp scratch. The histogram is dead by the time the candidate list is
// written (the list is filled in the final pass), so the two share storage.
struct WarpScratch {
  union {
    struct {
      unsigned int hl[kBins];    // gap sum per bin, low 32 bits (wraps)
      unsigned int hh[kBins];    // gap sum per bin, high 32 bits plus the low part's carries
      unsigned int hc[kBins];    // entry count per bin
      unsigned int hsat[2];      // bins whose sum passed 2^64 (saturated)
    };
    struct {
      unsigned long long ck[32]; // compacted candidates: key
      unsigned long long cg[32]; //                       gap
      int ci[32];                //                       entry index
    };
  };
};

// One ring stage: a tile's data and metadata, each array a 16-byte-aligned
// bulk-copy window (so its first element may sit a few slots in).
struct Stage {
  int32_t rows[kTileEntries + 8];        // destinations
  ulonglong2 lg[kTileEntries];           // {lower, gap}
  unsigned long long q[kTileCols];       // per-column O-maximization values
  unsigned long long rem[kTileCols + 4]; // 1 - sum(lower) per column
  int32_t sptr[kTileStates + 8];         // stateptr window
  int32_t cptr[kTileCols + 8];           // colptr window
  int32_t hint[kTileCols + 8];           // threshold-hint window
  int32_t shift[kTileCols + 8];          // per-column shift window (32-bit storage)
  uint8_t fixed[kTileStates + 32];       // reach/avoid mask window
  Problem prob;                          // descriptor of the tile's problem
  Tile tile;                             // set by the producer: the tile in this stage
  int32_t active;                        //                      the problem still runs
  int32_t k_iter;                        //                      iteration being computed
  int32_t fixed_off;                     //                      offset of state s0 in `fixed`
  unsigned int done;                     // slots of this tile finished so far
};

template <int W>
struct Smem {
  Stage st[kStages];
  WarpScratch ws[W];
  unsigned long long full[kStages];
  unsigned long long empty[kStages];
  int is_last;
};
static_assert(sizeof(int32_t) * (kTileEntries + 8) % 16 == 0, "lg must stay 16-byte aligned");
static_assert(offsetof(Stage, rem) % 16 == 0 && offsetof(Stage, sptr) % 16 == 0 && offsetof(Stage, cptr) % 16 == 0 &&
                  offsetof(Stage, fixed) % 16 == 0 && offsetof(Stage, prob) % 16 == 0 && offsetof(Stage, hint) % 16 == 0 && offsetof(Stage, shift) % 16 == 0 && sizeof(Problem) % 16 == 0,
              "bulk-copy destinations must be 16-byte aligned");
static_assert(sizeof(Stage) % 16 == 0, "stage alignment");
static_assert(sizeof(Smem<kConsumersLong>) <= 232448 && sizeof(Smem<kConsumersShort>) <= 232448,
              "shared memory budget of one CTA");

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about `ns` nanoseconds pass, instead of spinning.
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of an mbarrier, giving up after kWaitCycles or when
// another thread has flagged an error (unless `drain`). Returns false on give-up.
__device__ bool wait_phase(unsigned long long* bar, uint32_t parity, unsigned* err, bool drain) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    // each try sleeps up to ~20 us unless the phase completes first; the error
    // word (another CTA gave up) and the clock are checked between tries
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    if (!drain && (i & 7) == 7 && *(volatile unsigned*)err) return false;
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, 1u);
      return false;
    }
  }
}

// ---------------------------------------------------------------- warp reductions

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
  const unsigned hi = __reduce_min_sync(kFull, (unsigned)(x >> 32));
  const unsigned lo = __reduce_min_sync(kFull, ((unsigned)(x >> 32) == hi) ? (unsigned)x : 0xffffffffu);
  return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t x) {
  const unsigned hi = __reduce_max_sync(kFull, (unsigned)(x >> 32));
  const unsigned lo = __reduce_max_sync(kFull, ((unsigned)(x >> 32) == hi) ? (unsigned)x : 0u);
  return ((uint64_t)hi << 32) | lo;
}
// Exact 64-bit warp sum from three 22/22/20-bit partial sums (no carries lost).
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
  const unsigned a = __reduce_add_sync(kFull, (unsigned)(x & 0x3fffffu));
  const unsigned b = __reduce_add_sync(kFull, (unsigned)((x >> 22) & 0x3fffffu));
  const unsigned c = __reduce_add_sync(kFull, (unsigned)(x >> 44));
  return (uint64_t)a + ((uint64_t)b << 22) + ((uint64_t)c << 44);
}

// ---------------------------------------------------------------- saturating sums
//
// Gap sums decide only whether a prefix reaches rem (<= 2^63), and any sum that
// is below rem is needed exactly. So every gap enters the sums clipped to rem
// (which changes no decision: a gap >= rem reaches rem on its own), and sums
// saturate at 2^64 - 1 instead of wrapping (a column's upper bounds may add up
// to far more than 1).

__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
  const uint64_t c = a + b;
  return c < a ? ~0ull : c;
}
// Warp sum of per-lane values <= 2^63, saturating at 2^64 - 1.
__device__ __forceinline__ uint64_t warp_sum_sat(uint64_t x) {
  x = x > kOne ? kOne : x;
  const unsigned a = __reduce_add_sync(kFull, (unsigned)(x & 0x3fffffu));
  const unsigned b = __reduce_add_sync(kFull, (unsigned)((x >> 22) & 0x1fffffu));
  const unsigned c = __reduce_add_sync(kFull, (unsigned)(x >> 43));
  const unsigned __int128 t = (unsigned __int128)a + ((unsigned __int128)b << 22) + ((unsigned __int128)c << 43);
  return (t >> 64) ? ~0ull : (uint64_t)t;
}
__device__ __forceinline__ uint64_t warp_excl_scan_sat(uint64_t x, int lane) {
  uint64_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl = sat_add(incl, y);
  }
  // exclusive = inclusive of the previous lane
  const uint64_t ex = __shfl_up_sync(kFull, incl, 1);
  return lane == 0 ? 0ull : ex;
}

// ---------------------------------------------------------------- one column

// Entries [0, k) of one column: destinations `rows`, bound pairs `lg` (shared
// or global memory). Keys are recomputed from V on every pass (V is read
// through L1). `hint` is the entry that held the threshold in the previous
// iteration (-1: none); the entry that holds it now is returned in *hint_out.
// Returns q in Q2.62.
//
// Loads from global memory: a column's destinations and bounds (default L1
// policy: a column whose warm start misses is read again by the search, from
// L1), and the values V_{k-1}, gathered by many columns and kept (L1
// evict-last). All of them are read-only during a launch (V_k goes to the
// other buffer), so the non-coherent path is used. A destination or bound load
// guarded by a bounds test in C++ is volatile asm, so that the compiler never
// executes it speculatively ahead of the test (entries past a column's end may
// lie past the end of the array). The gathers of V always read a valid state,
// and the predicated loads below carry their guard inside the asm: those are
// plain asm, which the compiler may schedule freely. (Volatile asm keeps its
// program order, so a volatile gather would hold every later load behind the
// load its address waits for.)
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p) {
  int32_t v;
  asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ ulonglong2 ld_stream_u64x2(const ulonglong2* p) {
  ulonglong2 v;
  asm volatile("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream_u32x2(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint64_t ld_value(const uint64_t* p) {
  uint64_t v;
  asm("ld.global.nc.L1::evict_last.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
// High 32 bits of a value word (the whole value of a problem on 32-bit
// storage, whose values keep their low 32 bits zero).
__device__ __forceinline__ uint32_t ld_value_hi(const uint64_t* p) {
  uint32_t v;
  asm("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(reinterpret_cast<const uint32_t*>(p) + 1));
  return v;
}

// The same loads under a predicate: a lane with `ok` false issues no memory
// request and gets zeros (the slice kernel's lanes past their column's end).
// Results come back in 32-bit registers and are assembled after the asm.
__device__ __forceinline__ int32_t ld_stream_i32_if(const int32_t* p, bool ok) {
  int32_t v;
  asm(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\tmov.b32 %0, 0;\n\t@q ld.global.nc.s32 %0, [%1];\n\t}"
      : "=r"(v)
      : "l"(p), "r"((int)ok));
  return v;
}
__device__ __forceinline__ ulonglong2 ld_stream_u64x2_if(const ulonglong2* p, bool ok) {
  uint32_t a, b, c, d;
  asm(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\tmov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\tmov.b32 %2, 0;\n\t"
      "mov.b32 %3, 0;\n\t@q ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
      : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
      : "l"(p), "r"((int)ok));
  return make_ulonglong2(((uint64_t)b << 32) | a, ((uint64_t)d << 32) | c);
}
__device__ __forceinline__ uint2 ld_stream_u32x2_if(const uint2* p, bool ok) {
  uint32_t a, b;
  asm(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\tmov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\t"
      "@q ld.global.nc.v2.u32 {%0, %1}, [%2];\n\t}"
      : "=r"(a), "=r"(b)
      : "l"(p), "r"((int)ok));
  return make_uint2(a, b);
}
__device__ __forceinline__ uint64_t ld_value_if(const uint64_t* p, bool ok) {
  uint32_t a, b;
  asm(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\tmov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\t"
      "@q ld.global.nc.L1::evict_last.v2.u32 {%0, %1}, [%2];\n\t}"
      : "=r"(a), "=r"(b)
      : "l"(p), "r"((int)ok));
  return ((uint64_t)b << 32) | a;
}
__device__ __forceinline__ uint32_t ld_value_hi_if(const uint64_t* p, bool ok) {
  uint32_t v;
  asm(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\tmov.b32 %0, 0;\n\t"
      "@q ld.global.nc.L1::evict_last.u32 %0, [%1];\n\t}"
      : "=r"(v)
      : "l"(reinterpret_cast<const uint32_t*>(p) + 1), "r"((int)ok));
  return v;
}

// Where the column routines read a column's destinations and bounds (`gmem`):
// 0 shared memory (a plain pointer), 1 contiguous in global memory (streamed
// loads), 2 one column of a slice of the slice layout, whose entry idx sits
// 32 idx slots after its first (streamed loads).
constexpr int kSliceStride = 32;
struct GRows {
  const int32_t* p;
  __device__ __forceinline__ int32_t operator[](int idx) const { return ld_stream_i32(p + idx); }
};
struct SRows {
  const int32_t* p;
  __device__ __forceinline__ int32_t operator[](int idx) const {
    return ld_stream_i32(p + (size_t)idx * kSliceStride);
  }
};
template <int gmem>
struct RowsOf {
  typedef const int32_t* type;
};
template <>
struct RowsOf<1> {
  typedef GRows type;
};
template <>
struct RowsOf<2> {
  typedef SRows type;
};

// Entry idx's destination when `ok`, else 0 (a valid state); from global
// memory a predicated load, which the compiler may schedule freely.
__device__ __forceinline__ int32_t row_if(const int32_t* rows, int idx, bool ok) { return ok ? rows[idx] : 0; }
__device__ __forceinline__ int32_t row_if(GRows rows, int idx, bool ok) { return ld_stream_i32_if(rows.p + idx, ok); }
__device__ __forceinline__ int32_t row_if(SRows rows, int idx, bool ok) {
  return ld_stream_i32_if(rows.p + (size_t)idx * kSliceStride, ok);
}

// Bounds of one column as {lower, gap} in Q1.63, from 64-bit storage or from
// 32-bit mantissas shifted up by `down` = 32 - shift_j; read as `gmem` says.
// `at_if`: entry idx's pair when `ok`, else {0, 0} (predicated in global memory).
template <bool f32, int gmem = 0>
struct Bounds {
  const void* p;
  int down;
  __device__ __forceinline__ ulonglong2 operator[](int idx) const {
    const size_t at = gmem == 2 ? (size_t)idx * kSliceStride : (size_t)idx;
    if (f32) {
      const uint2 m = gmem ? ld_stream_u32x2(static_cast<const uint2*>(p) + at) : static_cast<const uint2*>(p)[at];
      return make_ulonglong2((uint64_t)m.x << down, (uint64_t)m.y << down);
    }
    return gmem ? ld_stream_u64x2(static_cast<const ulonglong2*>(p) + at) : static_cast<const ulonglong2*>(p)[at];
  }
  __device__ __forceinline__ ulonglong2 at_if(int idx, bool ok) const {
    if (gmem == 0) return ok ? (*this)[idx] : make_ulonglong2(0, 0);
    const size_t at = gmem == 2 ? (size_t)idx * kSliceStride : (size_t)idx;
    if (f32) {
      const uint2 m = ld_stream_u32x2_if(static_cast<const uint2*>(p) + at, ok);
      return make_ulonglong2((uint64_t)m.x << down, (uint64_t)m.y << down);
    }
    return ld_stream_u64x2_if(static_cast<const ulonglong2*>(p) + at, ok);
  }
};

// Where the column routines read V_{k-1}: gathers from global memory (the
// tiled kernels; read-only during a launch, L1 evict-last), or from shared
// memory (the single-CTA kernel, which keeps a small problem's values there
// across its iterations). `hi` is the high word, the whole value of a problem
// on 32-bit storage.
struct GlobalV {
  const uint64_t* p;
  __device__ __forceinline__ uint64_t at(int32_t r) const { return ld_value(p + r); }
  __device__ __forceinline__ uint32_t hi(int32_t r) const { return ld_value_hi(p + r); }
};
struct SharedV {
  const uint64_t* p;
  __device__ __forceinline__ uint64_t at(int32_t r) const { return p[r]; }
  __device__ __forceinline__ uint32_t hi(int32_t r) const { return (uint32_t)(p[r] >> 32); }
};

// One pass of the warm start over a column: acc = sum of V times (upper below
// v_k, lower elsewhere), flt = gap sum of the entries below v_k, geq = gap sum of
// the entries at v_k. The trip count is warp-uniform; padding entries read row 0
// and contribute zero. With `carry` the per-lane gap sums count their wraps and
// saturate; without it the column is narrow (all its gaps add up to < 2^64), so
// no sum can wrap.
// Trips of a warm pass from global memory whose loads are in flight ahead of
// the gather being consumed (three measured no faster on 64-bit storage and
// slower on 32-bit, whose deeper unroll then runs short of registers).
constexpr int kPipe = 2;

template <bool carry, bool f32, int gmem, class VP>
__device__ __forceinline__ void warm_pass(const typename RowsOf<gmem>::type rows, const Bounds<f32, gmem> lg, int32_t k,
                                          const VP V, uint64_t vk, bool pess, int lane,
                                          uint64_t& acc, uint64_t& flt, uint64_t& geq) {
  uint32_t fc = 0, gc = 0;
  const int nb = (k + 31) >> 5;
  // from global memory the loop is software-pipelined kPipe trips deep: the
  // destinations and bounds of the next trips are requested before this
  // trip's gather (from shared memory, where the loads are short, the plain
  // loop is faster)
  constexpr bool pipe = gmem != 0;
  int idx = lane;
  int32_t rq[kPipe];
  ulonglong2 bq[kPipe];
#pragma unroll
  for (int d = 0; d < kPipe; ++d) {
    rq[d] = pipe ? row_if(rows, idx + 32 * d, idx + 32 * d < k) : 0;
    bq[d] = pipe ? lg.at_if(idx + 32 * d, idx + 32 * d < k) : make_ulonglong2(0, 0);
  }
  // the gather of the next trip is issued before this trip's arithmetic
  uint64_t vnext = pipe ? V.at(rq[0]) : 0ull;
#pragma unroll 2
  for (int it = 0; it < nb; ++it) {
    if (!pipe) {
      rq[0] = row_if(rows, idx, idx < k);
      bq[0] = lg.at_if(idx, idx < k);
    }
    const ulonglong2 b = bq[0];
    const uint64_t v = pipe ? vnext : V.at(rq[0]);
    idx += 32;
    if (pipe) {
#pragma unroll
      for (int d = 0; d + 1 < kPipe; ++d) {
        rq[d] = rq[d + 1];
        bq[d] = bq[d + 1];
      }
      const int nx = idx + 32 * (kPipe - 1);
      rq[kPipe - 1] = row_if(rows, nx, nx < k);
      bq[kPipe - 1] = lg.at_if(nx, nx < k);
      vnext = V.at(rq[0]);
    }
    const bool below = pess ? (v < vk) : (v > vk);
    acc += __umul64hi(v, b.x + (below ? b.y : 0ull));
    const uint64_t gb = below ? b.y : 0ull, ge = v == vk ? b.y : 0ull;
    flt += gb;
    geq += ge;
    if (carry) {
      fc += flt < gb ? 1u : 0u;
      gc += geq < ge ? 1u : 0u;
    }
  }
  if (carry) {
    flt = fc ? ~0ull : flt;
    geq = gc ? ~0ull : geq;
  }
}

// The warm pass on 32-bit storage, in 32-bit arithmetic (unrolled four trips
// deep: a trip's loads in flight take half the registers of the 64-bit pass's,
// and the deeper unroll keeps twice as many in flight). Values are the high
// words vh (Q1.31) of value words whose low words are zero; bounds are the
// column's mantissas m (value m 2^-(31+s), s = shift_j). Each product vh * m is
// exact in 64 bits, and (vh * m) >> s equals the 64-bit routines' product
// hi64((vh << 32) * (m << (32 - s))) exactly, so this pass gives the same acc,
// and the same decisions from its gap sums (kept in mantissa units, where no
// sum can wrap), as warm_pass on the widened bounds: one 32x32 multiply, a
// shift and a 64-bit add per entry instead of a 64x64 multiply-high.
template <int gmem, class VP>
__device__ __forceinline__ void warm_pass32(const typename RowsOf<gmem>::type rows, const uint2* __restrict__ m,
                                            int32_t k, const VP V, uint32_t vk, int s, bool pess,
                                            int lane, uint64_t& acc, uint64_t& flt, uint64_t& geq) {
  const int nb = (k + 31) >> 5;
  if (gmem == 0) {
#pragma unroll 4
    for (int it = 0; it < nb; ++it) {
      const int idx = it * 32 + lane;
      const bool ok = idx < k;
      const uint32_t v = V.hi(ok ? rows[idx] : 0);
      uint2 b = make_uint2(0, 0);
      if (ok) b = m[idx];
      const bool below = pess ? (v < vk) : (v > vk);
      const uint32_t g = below ? b.y : 0u;
      acc += ((uint64_t)v * (uint64_t)(b.x + g)) >> s;
      flt += g;
      geq += v == vk ? b.y : 0u;
    }
    return;
  }
  // global memory: software-pipelined as in warm_pass
  int idx = lane;
  int32_t rq[kPipe];
  uint2 bq[kPipe];
#pragma unroll
  for (int d = 0; d < kPipe; ++d) {
    rq[d] = row_if(rows, idx + 32 * d, idx + 32 * d < k);
    bq[d] = ld_stream_u32x2_if(m + idx + 32 * d, idx + 32 * d < k);
  }
  uint32_t vnext = V.hi(rq[0]);
#pragma unroll 4
  for (int it = 0; it < nb; ++it) {
    const uint2 b = bq[0];
    const uint32_t v = vnext;
    idx += 32;
#pragma unroll
    for (int d = 0; d + 1 < kPipe; ++d) {
      rq[d] = rq[d + 1];
      bq[d] = bq[d + 1];
    }
    const int nx = idx + 32 * (kPipe - 1);
    rq[kPipe - 1] = row_if(rows, nx, nx < k);
    bq[kPipe - 1] = ld_stream_u32x2_if(m + nx, nx < k);
    vnext = V.hi(rq[0]);
    const bool below = pess ? (v < vk) : (v > vk);
    const uint32_t g = below ? b.y : 0u;
    acc += ((uint64_t)v * (uint64_t)(b.x + g)) >> s;
    flt += g;
    geq += v == vk ? b.y : 0u;
  }
}

// floor(a * b / 2^s) for a < 2^32, b < 2^64, 0 <= s < 64.
__device__ __forceinline__ uint64_t mul_shr(uint64_t a, uint64_t b, int s) {
  const uint64_t lo = a * b, hi = __umul64hi(a, b);
  return s ? (hi << (64 - s)) | (lo >> s) : lo;
}
// x << d, saturating at 2^64 - 1.
__device__ __forceinline__ uint64_t shl_sat(uint64_t x, int d) { return (x >> (64 - d)) ? ~0ull : x << d; }

// `rem_word` is rem = 1 - sum(lower) in Q1.63 (<= 2^63); when 0 < rem < 2^63 and
// the column's gaps add up to < 2^64 ("narrow"), model creation sets bit 63 as a
// flag on top of rem.
__device__ __forceinline__ uint64_t rem_of(uint64_t rem_word) {
  return ((rem_word >> 63) && (rem_word << 1)) ? (rem_word & (kOne - 1)) : rem_word;
}
__device__ __forceinline__ bool narrow_of(uint64_t rem_word) { return (rem_word >> 63) && (rem_word << 1); }

// Warm start. Decides the column without a search when rem = 0 (every entry keeps
// its lower bound) or when last iteration's threshold entry `hint` still holds
// the threshold: with kappa its key it does exactly when F(< kappa) < rem <=
// F(<= kappa), F being the gap sum; then one pass gives q. Comparisons run on V
// itself: key < kappa is V < V_kappa for a pessimistic adversary, V > V_kappa for
// an optimistic one. Returns true with *q set (Q2.62) when decided.
// What a failed warm start leaves for the neighbour check: the tried key's V,
// the pass's dot product and its gap sums below and at that key.
struct WarmMiss {
  uint64_t vk, acc, flt, geq;
  bool valid;
};

template <bool f32, int gmem, class VP>
__device__ __forceinline__ bool column_warm(const typename RowsOf<gmem>::type rows, const Bounds<f32, gmem> lg, int32_t k, uint64_t rem_word,
                                            const VP V, bool pess, int lane, int32_t hint,
                                            uint64_t* q, WarmMiss* miss) {
  miss->valid = false;
  const uint64_t rem = rem_of(rem_word);
  if (rem == 0) {
    uint64_t acc = 0;
#pragma unroll 4
    for (int idx = lane; idx < k; idx += 32) acc += __umul64hi(V.at(rows[idx]), lg[idx].x);
    *q = warp_sum_u64(acc);
    return true;
  }
  if (hint < 0 || hint >= k) return false;
  if (f32) {
    // 32-bit storage: the pass in 32-bit arithmetic (same words as below)
    const int down = lg.down, sh = 32 - down;
    const uint32_t vk32 = V.hi(rows[hint]);
    uint64_t acc = 0, flt = 0, geq = 0;
    warm_pass32<gmem>(rows, static_cast<const uint2*>(lg.p), k, V, vk32, sh, pess, lane, acc, flt, geq);
    acc = warp_sum_u64(acc);
    flt = warp_sum_u64(flt);
    geq = warp_sum_u64(geq);
    const uint64_t rem_m = rem >> down;  // exact: rem is a multiple of 2^down
    if (flt < rem_m && rem_m - flt <= geq) {
      *q = acc + mul_shr(vk32, rem_m - flt, sh);
      return true;
    }
    *miss = WarmMiss{(uint64_t)vk32 << 32, acc, shl_sat(flt, down), shl_sat(geq, down), true};
    return false;
  }
  const uint64_t vk = V.at(rows[hint]);
  uint64_t acc = 0, flt = 0, geq = 0;
  if (narrow_of(rem_word)) {
    // every gap sum of a narrow column is below 2^64: plain exact sums
    warm_pass<false, f32, gmem>(rows, lg, k, V, vk, pess, lane, acc, flt, geq);
    flt = warp_sum_u64(flt);
    geq = warp_sum_u64(geq);
  } else {
    warm_pass<true, f32, gmem>(rows, lg, k, V, vk, pess, lane, acc, flt, geq);
    flt = warp_sum_sat(flt);
    geq = warp_sum_sat(geq);
  }
  acc = warp_sum_u64(acc);
  if (flt < rem && rem - flt <= geq) {
    *q = acc + __umul64hi(vk, rem - flt);
    return true;
  }
  *miss = WarmMiss{vk, acc, flt, geq, true};
  return false;
}

// Neighbour check after a failed warm start at key kappa. If F(< kappa) >= rem the
// threshold lies below kappa, else above it; in most misses it is the adjacent
// distinct key. One pass finds that key (kappa- = the largest key below kappa, or
// kappa+ = the smallest above), the gap sum G of its entries, and the change of
// the warm pass's dot product when the entries between the two keys switch from
// upper to lower bound (or back): D = sum (hi(V (L + G)) - hi(V L)). Then
//   below: F(< kappa-) = F(< kappa) - G, holds when < rem;
//   above: F(< kappa+) = F(<= kappa), holds when F(<= kappa) + G >= rem;
// and q is the warm formula at the new key, to the bit. Returns false when the
// threshold moved further (or a sum is not exact), leaving the full search.
template <bool f32, int gmem, class VP>
__device__ __forceinline__ bool column_neighbor(const typename RowsOf<gmem>::type rows, const Bounds<f32, gmem> lg, int32_t k, uint64_t rem,
                                                const VP V, bool pess, int lane,
                                                const WarmMiss& w, uint64_t* q, int32_t* hint_out) {
  const bool down = w.flt >= rem;
  if (down && w.flt >= kOne) return false;  // F(< kappa) clipped: not exact
  const uint64_t kap = pess ? w.vk : kOne - w.vk;
  uint64_t best = 0, gs = 0, ds = 0, dk = 0;
  bool have = false;
  int32_t bi = -1;
  const int nb = (k + 31) >> 5;
  for (int it = 0; it < nb; ++it) {
    const int idx = it * 32 + lane;
    if (idx >= k) break;
    const uint64_t v = V.at(rows[idx]);
    const uint64_t key = pess ? v : kOne - v;
    const ulonglong2 b = lg[idx];
    const uint64_t d = __umul64hi(v, b.x + b.y) - __umul64hi(v, b.x);
    const bool side = down ? key < kap : key > kap;
    if (side) {
      const bool better = !have || (down ? key > best : key < best);
      if (better) {
        best = key;
        gs = b.y;
        ds = d;
        bi = idx;
        have = true;
      } else if (key == best) {
        gs = sat_add(gs, b.y);
        ds += d;
      }
    } else if (!down && key == kap) {
      dk += d;
    }
  }
  if (!__any_sync(kFull, have)) return false;
  const uint64_t tgt = down ? warp_max_u64(have ? best : 0ull) : warp_min_u64(have ? best : ~0ull);
  const bool mine = have && best == tgt;
  const uint64_t G = warp_sum_sat(mine ? gs : 0ull);
  const uint64_t D = warp_sum_u64(mine ? ds : 0ull);
  const unsigned mm = __ballot_sync(kFull, mine);
  const int32_t h = __shfl_sync(kFull, bi, __ffs(mm) - 1);
  const uint64_t vt = pess ? tgt : kOne - tgt;
  if (down) {
    const uint64_t fl = w.flt - G;  // G <= F(< kappa) < 2^63
    if (fl >= rem) return false;
    *q = w.acc - D + __umul64hi(vt, rem - fl);
  } else {
    const uint64_t DK = warp_sum_u64(dk);
    const uint64_t fl = w.flt + w.geq;  // < rem, exact
    if (sat_add(fl, G) < rem) return false;
    *q = w.acc + DK + __umul64hi(vt, rem - fl);
  }
  *hint_out = h;
  return true;
}

// Threshold search over a column with rem > 0 (the warm start failed or had no
// hint). Returns q in Q2.62 and the threshold entry in *hint_out.
template <bool f32, int gmem, class VP>
__device__ uint64_t column_search(const typename RowsOf<gmem>::type rows, const Bounds<f32, gmem> lg, int32_t k, uint64_t rem_word,
                                  const VP V, bool pess, WarpScratch* ws, int lane,
                                  int32_t* hint_out) {
  const uint64_t rem = rem_of(rem_word);
  auto key_of = [&](int idx) -> uint64_t {
    const uint64_t v = V.at(rows[idx]);
    return pess ? v : (kOne - v);
  };

  // 2. key range
  uint64_t lmin = ~0ull, lmax = 0;
  const int nb = (k + 31) >> 5;
#pragma unroll 4
  for (int it = 0; it < nb; ++it) {
    const int idx = it * 32 + lane;
    if (idx < k) {
      const uint64_t key = key_of(idx);
      lmin = key < lmin ? key : lmin;
      lmax = key > lmax ? key : lmax;
    }
  }
  // 3. threshold search: after it, keys < lo are below (full gap), keys > hi are
  // above (lower bound), keys in [lo, hi] are candidates sharing rem - fb.
  uint64_t lo = 0, hi = kOne, fb = 0;
  bool all_below = false, uniform = false;
  uint64_t cmin = warp_min_u64(lmin), cmax = warp_max_u64(lmax);
  for (int round = 0; round < 12; ++round) {
    if (cmin > cmax) {  // no entry: nothing absorbs rem
      all_below = true;
      break;
    }
    if (cmin == cmax) {  // the candidates share one key
      lo = hi = cmin;
      uniform = true;
      break;
    }
    const int bits = 64 - __clzll((long long)(cmax - cmin));
    const int shift = bits > 6 ? bits - 6 : 0;
    ws->hl[lane] = 0;
    ws->hl[lane + 32] = 0;
    ws->hh[lane] = 0;
    ws->hh[lane + 32] = 0;
    ws->hc[lane] = 0;
    ws->hc[lane + 32] = 0;
    if (lane == 0) ws->hsat[0] = ws->hsat[1] = 0;
    __syncwarp();
    for (int idx = lane; idx < k; idx += 32) {
      const uint64_t key = key_of(idx);
      if (key >= lo && key <= hi) {
        const int b = (int)((key - cmin) >> shift);
        const uint64_t g = lg[idx].y < rem ? lg[idx].y : rem;
        // exact 64-bit bin sums from native 32-bit atomics: the adder whose
        // low-word addition wraps carries one into the high word; a wrap of the
        // high word marks the bin saturated
        const unsigned gl = (unsigned)g;
        const unsigned old = atomicAdd(&ws->hl[b], gl);
        const unsigned up = (unsigned)(g >> 32) + ((old + gl) < old ? 1u : 0u);
        if (up) {
          const unsigned oh = atomicAdd(&ws->hh[b], up);
          if (oh + up < oh) atomicOr(&ws->hsat[b >> 5], 1u << (b & 31));
        }
        atomicAdd(&ws->hc[b], 1u);
      }
    }
    __syncwarp();
    const unsigned sat = ws->hsat[lane >> 4];
    const uint64_t h0 = ((sat >> ((2 * lane) & 31)) & 1u) ? ~0ull
                                                          : (((uint64_t)ws->hh[2 * lane] << 32) | ws->hl[2 * lane]);
    const uint64_t h1 = ((sat >> ((2 * lane + 1) & 31)) & 1u)
                            ? ~0ull
                            : (((uint64_t)ws->hh[2 * lane + 1] << 32) | ws->hl[2 * lane + 1]);
    const uint64_t ex = warp_excl_scan_sat(sat_add(h0, h1), lane);
    const uint64_t i0 = sat_add(sat_add(fb, ex), h0), i1 = sat_add(i0, h1);
    const unsigned cross = __ballot_sync(kFull, i1 >= rem);
    if (cross == 0) {  // first round only: the gaps cannot absorb rem
      all_below = true;
      break;
    }
    const int L = __ffs(cross) - 1;
    const bool first = i0 >= rem;
    const int b = __shfl_sync(kFull, first ? 2 * lane : 2 * lane + 1, L);
    fb = __shfl_sync(kFull, first ? sat_add(fb, ex) : i0, L);  // < rem by the choice of b
    const unsigned cnt = ws->hc[b];
    __syncwarp();
    lo = cmin + ((uint64_t)b << shift);
    const uint64_t top = lo + ((1ull << shift) - 1ull);
    hi = top < cmax ? top : cmax;
    if (cnt <= 32) break;
    // narrow to the min/max of the crossing bin's entries
    uint64_t a = ~0ull, z = 0;
    for (int idx = lane; idx < k; idx += 32) {
      const uint64_t key = key_of(idx);
      if (key >= lo && key <= hi) {
        a = key < a ? key : a;
        z = key > z ? key : z;
      }
    }
    cmin = warp_min_u64(a);
    cmax = warp_max_u64(z);
  }

  // 4. final pass: lower bounds everywhere, full gaps below the candidates,
  // candidates compacted (or summed when they share one key).
  uint64_t acc = 0, gsum = 0;
  unsigned pos = 0;
  int first_cand = -1;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = 0; base < k; base += 32) {
    const int idx = base + lane;
    const bool valid = idx < k;
    uint64_t key = 0;
    ulonglong2 b = make_ulonglong2(0, 0);
    if (valid) {
      key = key_of(idx);
      b = lg[idx];
    }
    const bool below = all_below || key < lo;
    const bool cand = valid && !all_below && key >= lo && key <= hi;
    if (valid) acc += __umul64hi(pess ? key : (kOne - key), below ? b.x + b.y : b.x);
    const unsigned m = __ballot_sync(kFull, cand);
    if (m && first_cand < 0) first_cand = base + __ffs(m) - 1;
    if (!uniform) {
      if (cand) {
        // < 32: a crossing bin of more than 32 entries was narrowed above
        const unsigned at = min(pos + __popc(m & lt), 31u);
        ws->ck[at] = key;
        ws->cg[at] = b.y < rem ? b.y : rem;
        ws->ci[at] = idx;
      }
      pos += __popc(m);
    } else if (cand) {
      gsum = sat_add(gsum, b.y < rem ? b.y : rem);
    }
  }
  acc = warp_sum_u64(acc);
  if (all_below) {
    *hint_out = -1;
    return acc;
  }
  pos = min(pos, 32u);
  const uint64_t r2 = rem - fb;  // > 0 by construction of the crossing bin
  if (uniform) {
    // one key for all candidates: they take min(r2, their total gap) together
    const uint64_t g = warp_sum_sat(gsum);
    *hint_out = first_cand;
    return acc + __umul64hi(pess ? lo : (kOne - lo), g < r2 ? g : r2);
  }
  __syncwarp();
  // Resolve the <= 32 candidates exactly: candidate i takes its gap clipped to
  // what the candidates ordered before it (by key, then list position) leave;
  // the one that takes the last of r2 is the threshold.
  uint64_t extra = 0;
  int thr = -1;
  if (lane < (int)pos) {
    const uint64_t ki = ws->ck[lane], gi = ws->cg[lane];
    uint64_t before = 0;
    for (unsigned j = 0; j < pos; ++j) {
      const uint64_t kj = ws->ck[j];
      if (kj < ki || (kj == ki && j < (unsigned)lane)) before = sat_add(before, ws->cg[j]);
    }
    const uint64_t left = r2 > before ? r2 - before : 0;
    extra = __umul64hi(pess ? ki : (kOne - ki), gi < left ? gi : left);
    if (left > 0 && left <= gi) thr = ws->ci[lane];
  }
  const unsigned tm = __ballot_sync(kFull, thr >= 0);
  *hint_out = tm ? __shfl_sync(kFull, thr, __ffs(tm) - 1) : -1;
  __syncwarp();
  return acc + warp_sum_u64(extra);
}

// One column, warm start first: q in Q2.62, the threshold entry in *hint_out.
template <bool f32, int gmem, class VP>
__device__ uint64_t column_q(const typename RowsOf<gmem>::type rows, const Bounds<f32, gmem> lg, int32_t k, uint64_t rem_word,
                             const VP V, bool pess, WarpScratch* ws, int lane, int32_t hint,
                             int32_t* hint_out) {
  // A hint of -2 - i names entry i as well and records that the column's last
  // value came from the full search: its threshold is moving fast, so a miss
  // goes to the search without trying the neighbour.
  const bool moving = hint <= -2;
  const int32_t entry = moving ? -2 - hint : hint;
  uint64_t q;
  WarmMiss miss;
  if (column_warm<f32, gmem>(rows, lg, k, rem_word, V, pess, lane, entry, &q, &miss)) {
    *hint_out = entry;
    return q;
  }
  if (miss.valid && !moving &&
      column_neighbor<f32, gmem>(rows, lg, k, rem_of(rem_word), V, pess, lane, miss, &q, hint_out))
    return q;
  int32_t found;
  q = column_search<f32, gmem>(rows, lg, k, rem_word, V, pess, ws, lane, &found);
  *hint_out = found >= 0 ? -2 - found : -1;
  return q;
}

// ---------------------------------------------------------------- the step kernel

__device__ __forceinline__ bool problem_active(const StepLaunch& L, int p, int32_t* k_iter) {
  const IterState& it = L.its[p];
  const Problem& P = L.probs[p];
  *k_iter = it.iter + 1;
  return !it.done && (P.infinite || *k_iter <= P.horizon);
}

// V, policy and residual of state s once its actions' values are known.
__device__ __forceinline__ void finish_state(const Problem& P, int32_t s, int32_t k_iter, uint64_t vnew, int32_t best,
                                             const uint64_t* __restrict__ Vin, uint64_t* __restrict__ Vout,
                                             unsigned long long& dmax) {
  Vout[s] = vnew;
  if (P.policy_mode == 1)
    P.policy[(size_t)(P.horizon - k_iter) * P.n_states + s] = best;
  else if (P.policy_mode == 2)
    P.policy[s] = best;
  if (P.infinite) {
    const uint64_t vold = Vin[s];
    const uint64_t d = vnew > vold ? vnew - vold : vold - vnew;
    dmax = d > dmax ? d : dmax;
  }
}

// Best action of a state over columns [jb, je): first index attaining the optimum.
template <class QAt>
__device__ __forceinline__ void best_action(const Problem& P, int32_t jb, int32_t je, QAt q_at, uint64_t* bestq,
                                            int32_t* best) {
  uint64_t bq = 0;
  int32_t bb = -1;
  for (int32_t jj = jb; jj < je; ++jj) {
    const uint64_t q = q_at(jj);
    if (bb < 0 || (P.maximize ? q > bq : q < bq)) {
      bq = q;
      bb = jj - jb;
    }
  }
  *bestq = bq;
  *best = bb;
}

// V_k(s) of a free state from the optimum over its actions (Q2.62): the
// reachability value clamped at 1, or the reward update W_k = c_s + gamma T(W_{k-1})
// in signed Q2.62, clamped to [0, 1].
// A problem on 32-bit storage keeps its values at 32 bits (rounded to nearest,
// low word zero), which its warm passes read as Q1.31.
__device__ __forceinline__ uint64_t free_state_value(const Problem& P, int32_t s, uint64_t bestq) {
  uint64_t v;
  if (P.property == kPropReward) {
    const int64_t tt = (int64_t)(__umul64hi(P.gamma_fix, bestq) << 1);
    int64_t w = P.rbias[s] + tt;
    w = w < 0 ? 0 : (w > (int64_t)(kOne >> 1) ? (int64_t)(kOne >> 1) : w);
    v = (uint64_t)w << 1;
  } else {
    v = bestq >= (kOne >> 1) ? kOne : (bestq << 1);  // Q2.62 -> Q1.63, clamp at 1
  }
  if (P.lg32) v = round_value32(v);
  return v;
}

// State epilogue of a tile (one warp): opt over actions, reach/avoid mask,
// reward update, V / policy / residual. `fixed_at(s)` gives the mask of state s,
// `best_of(s, &q, &a)` the optimal action value and index.
template <class FixedAt, class BestOf>
__device__ void tile_epilogue(const StepLaunch& L, const Problem& P, const Tile& T, int32_t k_iter, int lane,
                              FixedAt fixed_at, BestOf best_of) {
  const uint64_t* __restrict__ Vin = P.V[(k_iter - 1) & 1];
  uint64_t* __restrict__ Vout = P.V[k_iter & 1];
  unsigned long long dmax = 0;
  for (int32_t s = T.s0 + lane; s < T.s1; s += 32) {
    const uint8_t fx = fixed_at(s);
    uint64_t vnew;
    int32_t best = -1;
    if (fx == 1) {
      vnew = kOne;
    } else if (fx == 2) {
      vnew = 0;
    } else {
      uint64_t bestq;
      best_of(s, &bestq, &best);
      vnew = free_state_value(P, s, bestq);
    }
    finish_state(P, s, k_iter, vnew, best, Vin, Vout, dmax);
  }
  if (P.infinite) {
    const uint64_t m = warp_max_u64(dmax);
    if (lane == 0 && m) atomicMax(&L.its[T.p].resmax, (unsigned long long)m);
  }
}

// One column of a staged tile: leaves q in st.q[li] and updates the hint.
template <bool f32>
__device__ __forceinline__ void stage_column(Stage& st, const Tile& T, int32_t li, int32_t k_iter, WarpScratch* ws,
                                             int lane) {
  const Problem& P = st.prob;
  const int32_t c = T.c0 + li;
  const int32_t eb = T.e0 & ~3, cb = T.c0 & ~3, mb = T.c0 & ~1;
  const int32_t ca = st.cptr[c - cb], ce = st.cptr[c + 1 - cb];
  const int32_t h = P.hint ? st.hint[c - cb] : -1;
  if (f32 && P.xoff) {
    // a correction column of 32-bit storage: its exact pairs are staged after
    // the tile's mantissa pairs (at its offset within the tile's range of lgx)
    const int32_t xo = __ldg(P.xoff + c);
    if (xo >= 0) {
      const int32_t qb = T.e0 & ~1, qe = (T.e1 + 1) & ~1;
      const ulonglong2* xs = reinterpret_cast<const ulonglong2*>(reinterpret_cast<const unsigned char*>(st.lg) +
                                                                  (size_t)(qe - qb) * 8u);
      int32_t hout;
      const uint64_t q = column_q<false, false>(st.rows + (ca - eb), Bounds<false>{xs + (xo - T.x0), 0}, ce - ca,
                                                st.rem[c - mb], GlobalV{P.V[(k_iter - 1) & 1]}, P.pessimistic != 0, ws, lane,
                                                h, &hout);
      if (lane == 0) {
        st.q[li] = q;
        if (P.hint && hout != h) P.hint[c] = hout;
      }
      return;
    }
  }
  Bounds<f32> bd;
  if (f32)
    bd = Bounds<f32>{reinterpret_cast<const uint2*>(st.lg) + (ca - (T.e0 & ~1)), 32 - st.shift[c - cb]};
  else
    bd = Bounds<f32>{st.lg + (ca - T.e0), 0};
  int32_t hout;
  const uint64_t q = column_q<f32, false>(st.rows + (ca - eb), bd, ce - ca, st.rem[c - mb], GlobalV{P.V[(k_iter - 1) & 1]},
                                   P.pessimistic != 0, ws, lane, h, &hout);
  if (lane == 0) {
    st.q[li] = q;
    if (P.hint && hout != h) P.hint[c] = hout;
  }
}

__device__ void end_of_launch(const StepLaunch& L, int* is_last);

// Tiles this launch visits: the running prefix recorded by the previous launch.
__device__ __forceinline__ int32_t tiles_to_visit(const StepLaunch& L) {
  const int32_t lim = L.ctl->tile_limit;
  return lim > 0 && lim - 1 < L.n_tiles ? lim - 1 : L.n_tiles;
}


template <int W>
__global__ void __launch_bounds__(32 * (W + 1), 1) bellman_step_kernel(StepLaunch L) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<W>& S = *reinterpret_cast<Smem<W>*>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned* err = &L.ctl->error;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      S.st[s].done = 0;  // shared memory starts undefined in every launch
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], W);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == W) {
    // ------------------------------------------------------------ producer
    if (lane == 0 && !L.stall) {
      int i = 0;
      bool ok = true;
      int pending_round[kStages];
      for (int s = 0; s < kStages; ++s) pending_round[s] = -1;
      const int32_t nt = tiles_to_visit(L);
      for (int32_t t = blockIdx.x; t < nt; t += gridDim.x, ++i) {
        const int stage = i % kStages, round = i / kStages;
        if (round > 0 && !wait_phase(&S.empty[stage], (round - 1) & 1, err, false)) {
          ok = false;
          break;
        }
        pending_round[stage] = -1;
        const Tile T = L.tiles[t];
        Stage& st = S.st[stage];
        int32_t k_iter;
        const bool act = problem_active(L, T.p, &k_iter);
        st.tile = T;
        st.active = act ? 1 : 0;
        st.k_iter = k_iter;
        if (act) {
          const Problem& P = L.probs[T.p];
          // 16-byte-aligned windows of every array the tile needs
          const int32_t eb = T.e0 & ~3, ee = (T.e1 + 3) & ~3;
          const int32_t sb = T.s0 & ~3, se = (T.s1 + 4) & ~3;
          const int32_t cb = T.c0 & ~3, ce = (T.c1 + 4) & ~3;
          const int32_t mb = T.c0 & ~1, me = (T.c1 + 1) & ~1;
          const uintptr_t f0 = (uintptr_t)(P.fixed + T.s0), fa = f0 & ~(uintptr_t)15;
          const uintptr_t fe = ((uintptr_t)(P.fixed + T.s1) + 15) & ~(uintptr_t)15;
          st.fixed_off = (int32_t)(f0 - fa);
          const uint32_t rb = (uint32_t)(ee - eb) * 4u;
          // bounds: 16-byte pairs, or (32-bit storage) 8-byte pairs from an aligned
          // window plus the per-column shift window
          const int32_t qb = T.e0 & ~1, qe = (T.e1 + 1) & ~1;
          const uint32_t xbytes = P.lg32 ? (uint32_t)(T.x1 - T.x0) * 16u : 0u;
          const uint32_t gb = P.lg32 ? (uint32_t)(qe - qb) * 8u + (uint32_t)(((T.c1 + 4) & ~3) - (T.c0 & ~3)) * 4u +
                                           xbytes
                                     : (uint32_t)(T.e1 - T.e0) * 16u;
          const uint32_t sbytes = (uint32_t)(se - sb) * 4u, cbytes = (uint32_t)(ce - cb) * 4u;
          const uint32_t mbytes = (uint32_t)(me - mb) * 8u, fbytes = (uint32_t)(fe - fa);
          const uint32_t hbytes = P.hint ? cbytes : 0u;  // same window as colptr
          mbar_arrive_expect_tx(&S.full[stage],
                                rb + gb + sbytes + cbytes + mbytes + fbytes + hbytes + (uint32_t)sizeof(Problem));
          if (hbytes) bulk_g2s(st.hint, P.hint + cb, hbytes, &S.full[stage]);
          bulk_g2s(&st.prob, &P, (uint32_t)sizeof(Problem), &S.full[stage]);
          if (sbytes) bulk_g2s(st.sptr, P.stateptr + sb, sbytes, &S.full[stage]);
          if (cbytes) bulk_g2s(st.cptr, P.colptr + cb, cbytes, &S.full[stage]);
          if (mbytes) bulk_g2s(st.rem, P.rem + mb, mbytes, &S.full[stage]);
          if (fbytes) bulk_g2s(st.fixed, (const void*)fa, fbytes, &S.full[stage]);
          if (rb) bulk_g2s(st.rows, P.rowval + eb, rb, &S.full[stage]);
          if (P.lg32) {
            const uint32_t qbytes = (uint32_t)(qe - qb) * 8u;
            if (qbytes) bulk_g2s(st.lg, P.lg32 + qb, qbytes, &S.full[stage]);
            bulk_g2s(st.shift, P.shift + cb, cbytes, &S.full[stage]);
            // the correction columns' exact pairs, after the mantissas (the
            // planner keeps both within the bound area)
            if (xbytes) bulk_g2s(reinterpret_cast<unsigned char*>(st.lg) + qbytes, P.lgx + T.x0, xbytes, &S.full[stage]);
          } else if (gb) {
            bulk_g2s(st.lg, P.lg + T.e0, gb, &S.full[stage]);
          }
          pending_round[stage] = round;
        } else {
          mbar_arrive(&S.full[stage]);  // releases the plain stores above as well
        }
      }
      if (!ok) {
        // give-up path: let the copies already issued land before the CTA exits
        for (int s = 0; s < kStages; ++s)
          if (pending_round[s] >= 0) wait_phase(&S.full[s], pending_round[s] & 1, err, true);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    // The CTA's tiles t_j = blockIdx.x + j*gridDim.x are visited in order by
    // every consumer warp: wait until tile j has landed, work on its own slots,
    // arrive on the stage's "empty" barrier. A slot is a column. Slots are dealt
    // round-robin across tiles, so a warp that has nothing left in tile j moves
    // on to tile j+1 while the others finish. Because every warp visits every
    // tile, no warp can fall two rounds behind a stage, which keeps the parity
    // waits unambiguous. The warp that completes a tile's last slot runs the
    // tile's state epilogue before it arrives, so the producer refills a stage
    // only after the epilogue.
    WarpScratch* ws = &S.ws[warp];
    int32_t slot_base = 0;  // global slot index of tile j's first slot
    int j = 0;
    const int32_t nt = tiles_to_visit(L);  // the producer visits the same tiles
    for (int32_t t = blockIdx.x; t < nt; t += gridDim.x, ++j) {
      const int stage = j % kStages, round = j / kStages;
      int got = 1;
      if (lane == 0) got = wait_phase(&S.full[stage], round & 1, err, false) ? 1 : 0;
      got = __shfl_sync(kFull, got, 0);
      if (!got) break;
      (void)mbar_try_wait(&S.full[stage], round & 1);  // completed phase: acquire for every lane
      Stage& st = S.st[stage];
      const Tile T = st.tile;
      const int32_t nslots = T.c1 - T.c0;
      const int32_t k_iter = st.k_iter;
      const bool active = st.active != 0;
      // first local slot of this warp: global slot g with g % W == warp
      int32_t first = warp - (slot_base % W);
      if (first < 0) first += W;
      for (int32_t ls = first; ls < nslots; ls += W) {
        if (active) {
          if (st.prob.lg32)
            stage_column<true>(st, T, ls, k_iter, ws, lane);
          else
            stage_column<false>(st, T, ls, k_iter, ws, lane);
        }
        // count the slot; the warp that completes the tile finishes its states
        unsigned prev = 0;
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();
          prev = atomicAdd(&st.done, 1u);
        }
        prev = __shfl_sync(kFull, prev, 0);
        if (prev + 1 == (unsigned)nslots) {
          __threadfence_block();
          if (active) {
            const Problem& P = st.prob;
            const int32_t sb = T.s0 & ~3;
            tile_epilogue(L, P, T, k_iter, lane,
                          [&](int32_t s) { return st.fixed[st.fixed_off + (s - T.s0)]; },
                          [&](int32_t s, uint64_t* bq, int32_t* bb) {
                            const int32_t jb = st.sptr[s - sb], je = st.sptr[s + 1 - sb];
                            best_action(P, jb, je, [&](int32_t jj) { return st.q[jj - T.c0]; }, bq, bb);
                          });
          }
          __syncwarp();
          if (lane == 0) st.done = 0;
        }
      }
      slot_base += nslots;
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.empty[stage]);  // this warp is done with tile j
    }

  }

  end_of_launch(L, &S.is_last);
}

// The last CTA of the launch (of either step kernel) advances every running
// problem's iteration state and resets the launch counters.
__device__ void end_of_launch(const StepLaunch& L, int* is_last) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(&L.ctl->finished, 1u);
    *is_last = (prev == (unsigned)L.grid_total - 1u);
  }
  __syncthreads();
  if (!*is_last) return;
  __threadfence();
  for (int q = threadIdx.x; q < L.count; q += blockDim.x) {
    IterState* it = &L.its[q];
    const Problem& PQ = L.probs[q];
    if (it->done) continue;
    const int32_t kq = it->iter + 1;
    if (!PQ.infinite && kq > PQ.horizon) {  // horizon 0: nothing ran
      it->done = 1;
      it->k_final = it->iter;
      continue;
    }
    it->iter = kq;
    if (PQ.infinite) {
      const unsigned long long r = it->resmax;
      it->resmax = 0;
      if (r < PQ.eps_fix && !PQ.external_stop) {
        it->done = 1;
        it->k_final = kq;
      } else if (kq >= PQ.horizon) {
        it->done = 1;
        it->k_final = kq;
        it->noconv = 1;
      }
    } else if (kq >= PQ.horizon) {
      it->done = 1;
      it->k_final = kq;
    }
  }
  if (threadIdx.x == 0) {
    L.ctl->finished = 0;
    L.ctl->wide_next = 0;
    L.ctl->tile_next = 0;
    *is_last = -1;  // reused below: the largest rank still running
  }
  if (!L.rank_of) return;
  // Tiles are laid out by rank, so the next launch needs only the prefix that
  // belongs to problems still running (a finished problem's tiles are never
  // visited again).
  __syncthreads();
  int rmax = -1;
  for (int q = threadIdx.x; q < L.count; q += blockDim.x)
    if (!L.its[q].done) rmax = max(rmax, L.rank_of[q]);
  if (rmax >= 0) atomicMax(is_last, rmax);
  __syncthreads();
  if (threadIdx.x == 0) L.ctl->tile_limit = (*is_last >= 0 ? L.rank_tile_end[*is_last] : 0) + 1;
}



// ---------------------------------------------------------------- direct kernel
//
// The same Bellman step over the same tile list without the shared-memory ring:
// every warp takes the next tile (atomic counter), streams its columns straight
// from global memory (destinations and bounds with L1 evict-first loads, the
// values V_{k-1} with evict-last gathers) and finishes each state itself. There
// is no producer warp, no barrier and no staging buffer, so the whole L1 holds
// V_{k-1} and the columns being searched, and as many columns are in flight as
// there are warps (the ring holds three tiles per SM). Columns of states held
// fixed by the property (reach / avoid) are not read: Eq. 2 sets those values
// directly. Each column runs the same exact routines as in the ring kernel,
// so both kernels give the same words.

// Bulk prefetch of [p, p + bytes) into L2, widened to 16-byte boundaries (the
// model's arrays are padded so that such windows stay inside them).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a = (uintptr_t)p & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes + 15) & ~(uintptr_t)15;
  if (e > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// Column metadata of 32 consecutive columns, one per lane.
struct ColChunk {
  int32_t base = -1;
  int32_t ca = 0, ce = 0, hint = -1, shift = 0, xoff = -1;
  uint64_t rem = 0;
};

template <bool f32>
__device__ void direct_tile(const StepLaunch& L, const Tile& T, int32_t k_iter, WarpScratch* ws, int lane) {
  const Problem& P = L.probs[T.p];
  const uint64_t* __restrict__ Vin = P.V[(k_iter - 1) & 1];
  uint64_t* __restrict__ Vout = P.V[k_iter & 1];
  const bool pess = P.pessimistic != 0;
  const bool maxi = P.maximize != 0;
  const int32_t* __restrict__ colptr = P.colptr;
  int32_t* hint = P.hint;
  unsigned long long dmax = 0;
  ColChunk cc;
  for (int32_t sb = T.s0; sb < T.s1; sb += 32) {
    // per-state metadata, one state per lane
    const int32_t ms = sb + lane;
    int32_t m_jb = 0, m_je = 0, m_fx = 0;
    if (ms < T.s1) {
      m_jb = __ldg(P.stateptr + ms);
      m_je = __ldg(P.stateptr + ms + 1);
      m_fx = __ldg(P.fixed + ms);
    }
    const int ns = T.s1 - sb < 32 ? T.s1 - sb : 32;
    for (int i = 0; i < ns; ++i) {
      const int32_t s = sb + i;
      const int32_t fx = __shfl_sync(kFull, m_fx, i);
      uint64_t vnew;
      int32_t best = -1;
      if (fx == 1) {
        vnew = kOne;
      } else if (fx == 2) {
        vnew = 0;
      } else {
        const int32_t jb = __shfl_sync(kFull, m_jb, i), je = __shfl_sync(kFull, m_je, i);
        uint64_t bq = 0;
        for (int32_t c = jb; c < je; ++c) {
          if (cc.base < 0 || c - cc.base >= 32) {  // next 32 columns' metadata, one per lane
            cc.base = c;
            const int32_t mc = c + lane;
            if (mc < T.c1) {
              cc.ca = __ldg(colptr + mc);
              cc.ce = __ldg(colptr + mc + 1);
              cc.rem = __ldg(P.rem + mc);
              cc.hint = hint ? hint[mc] : -1;
              if (f32) {
                cc.shift = __ldg(P.shift + mc);
                cc.xoff = P.xoff ? __ldg(P.xoff + mc) : -1;
              }
            }
          }
          const int src = c - cc.base;
          const int32_t ca = __shfl_sync(kFull, cc.ca, src), ce = __shfl_sync(kFull, cc.ce, src);
          // start pulling the next column of the chunk into L2 while this one runs
          // (its bounds and destinations are contiguous after this column's)
          const int32_t cn = src + 1 < 32 ? __shfl_sync(kFull, cc.ce, src + 1) : ce;
          if (lane == 0 && cn > ce && c + 1 < T.c1) {
            prefetch_l2(P.rowval + ce, (size_t)(cn - ce) * sizeof(int32_t));
            if (f32)
              prefetch_l2(P.lg32 + ce, (size_t)(cn - ce) * sizeof(uint2));
            else
              prefetch_l2(P.lg + ce, (size_t)(cn - ce) * sizeof(ulonglong2));
          }
          const int32_t h = __shfl_sync(kFull, cc.hint, src);
          const uint64_t rw = __shfl_sync(kFull, cc.rem, src);
          int32_t hout;
          uint64_t q;
          const int32_t xo = f32 ? __shfl_sync(kFull, cc.xoff, src) : -1;
          if (f32 && xo < 0)
            q = column_q<true, true>(GRows{P.rowval + ca},
                                     Bounds<true, true>{P.lg32 + ca, 32 - __shfl_sync(kFull, cc.shift, src)}, ce - ca,
                                     rw, GlobalV{Vin}, pess, ws, lane, h, &hout);
          else if (f32)  // correction column: its exact bounds
            q = column_q<false, true>(GRows{P.rowval + ca}, Bounds<false, true>{P.lgx + xo, 0}, ce - ca, rw, GlobalV{Vin},
                                      pess, ws, lane, h, &hout);
          else
            q = column_q<false, true>(GRows{P.rowval + ca}, Bounds<false, true>{P.lg + ca, 0}, ce - ca, rw, GlobalV{Vin}, pess,
                                      ws, lane, h, &hout);
          if (lane == 0 && hint && hout != h) hint[c] = hout;
          if (best < 0 || (maxi ? q > bq : q < bq)) {
            bq = q;
            best = c - jb;
          }
        }
        vnew = free_state_value(P, s, bq);
      }
      if (lane == 0) finish_state(P, s, k_iter, vnew, best, Vin, Vout, dmax);
    }
  }
  if (P.infinite && lane == 0 && dmax) atomicMax(&L.its[T.p].resmax, dmax);
}

template <int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) bellman_direct_kernel(StepLaunch L) {
  __shared__ WarpScratch ws_all[NW];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31;
  WarpScratch* ws = &ws_all[threadIdx.x >> 5];
  const int32_t nt = tiles_to_visit(L);
  for (;;) {
    int32_t t = 0;
    if (lane == 0) t = (int32_t)atomicAdd(&L.ctl->tile_next, 1u);
    t = __shfl_sync(kFull, t, 0);
    if (t >= nt) break;
    const Tile T = L.tiles[t];
    int32_t k_iter;
    if (!problem_active(L, T.p, &k_iter)) continue;
    if (L.probs[T.p].lg32)
      direct_tile<true>(L, T, k_iter, ws, lane);
    else
      direct_tile<false>(L, T, k_iter, ws, lane);
  }
  end_of_launch(L, &is_last);
}

// ---------------------------------------------------------------- slice kernel
//
// The same Bellman step over the slice layout (one lane per column): every warp
// takes the next slice (atomic counter) and each lane runs the warm start of
// the O-maximization (Sec. 4) for its own column, sequentially over the
// column's entries. The warp's loads of entry t of its 32 columns are one
// contiguous run, and the sums a column needs stay in its lane, so a column
// costs no warp reduction and no per-column bookkeeping; in the tiled kernels
// these cost more issue slots than the entries themselves when columns are
// short. Columns whose warm start fails (or that have no hint yet), and the
// exact columns of 32-bit storage, then go through the exact neighbour check
// and threshold search one at a time with the whole warp, reading the column
// through the slice layout's stride (from L2: the warp has just streamed it).
// Each column's q goes to a per-column buffer; the warp that completes the last
// slice of a window (whole states) finishes the window's states. Every step of
// a column is the routine the other kernels run, so the words are theirs.

// One lane's warm pass over its column on 64-bit storage: entry t at rows[32 t],
// lg[32 t]; `len` trips (the slice's longest column), loads off past k. The sums
// of warm_pass; with `carry`, gap sums that pass 2^64 saturate.
// Trips are taken kLaneGroup at a time and software-pipelined: the next
// group's destination and bound loads are issued before this group's gathers
// and arithmetic, so each lane keeps two groups of streamed loads in flight.
// (Groups of eight trips on 32-bit storage measured no faster and spill more.
// The 32-bit pass, whose trips take half the registers, also issues the next
// group's gathers before this group's arithmetic; the same third stage on
// 64-bit storage spills.)
constexpr int kLaneGroup = 4;
template <bool carry>
__device__ __forceinline__ void lane_pass64(const int32_t* rows, const ulonglong2* lg, int32_t len, int32_t k,
                                            const uint64_t* __restrict__ V, uint64_t vk, bool pess, uint64_t& acc,
                                            uint64_t& flt, uint64_t& geq) {
  uint32_t fc = 0, gc = 0;
  int32_t r[kLaneGroup];
  ulonglong2 b[kLaneGroup];
#pragma unroll
  for (int u = 0; u < kLaneGroup; ++u) {
    r[u] = ld_stream_i32_if(rows + (size_t)u * kSliceStride, u < k);
    b[u] = ld_stream_u64x2_if(lg + (size_t)u * kSliceStride, u < k);
  }
  for (int32_t t0 = 0; t0 < len; t0 += kLaneGroup) {
    uint64_t v[kLaneGroup];
#pragma unroll
    for (int u = 0; u < kLaneGroup; ++u) v[u] = ld_value_if(V + r[u], t0 + u < k);
    int32_t rn[kLaneGroup];
    ulonglong2 bn[kLaneGroup];
#pragma unroll
    for (int u = 0; u < kLaneGroup; ++u) {
      const int32_t t = t0 + kLaneGroup + u;
      rn[u] = ld_stream_i32_if(rows + (size_t)t * kSliceStride, t < k);
      bn[u] = ld_stream_u64x2_if(lg + (size_t)t * kSliceStride, t < k);
    }
#pragma unroll
    for (int u = 0; u < kLaneGroup; ++u) {
      const bool below = pess ? (v[u] < vk) : (v[u] > vk);
      const uint64_t gb = below ? b[u].y : 0ull, ge = v[u] == vk ? b[u].y : 0ull;
      acc += __umul64hi(v[u], b[u].x + gb);
      flt += gb;
      geq += ge;
      if (carry) {
        fc += flt < gb ? 1u : 0u;
        gc += geq < ge ? 1u : 0u;
      }
    }
#pragma unroll
    for (int u = 0; u < kLaneGroup; ++u) {
      r[u] = rn[u];
      b[u] = bn[u];
    }
  }
  if (carry) {
    flt = fc ? ~0ull : flt;
    geq = gc ? ~0ull : geq;
  }
}

// The same on 32-bit storage, in 32-bit arithmetic: the sums of warm_pass32.
__device__ __forceinline__ void lane_pass32(const int32_t* rows, const uint2* m, int32_t len, int32_t k,
                                            const uint64_t* __restrict__ V, uint32_t vk, int s, bool pess,
                                            uint64_t& acc, uint64_t& flt, uint64_t& geq) {
  // three stages in flight: destinations and bounds of group t0 + 2G, the
  // gathers of group t0 + G, the arithmetic of group t0 (G = kLaneGroup)
  constexpr int G = kLaneGroup;
  int32_t r1[G];
  uint2 b0[G], b1[G];
  uint32_t v0[G];
  {
    int32_t r0[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      r0[u] = ld_stream_i32_if(rows + (size_t)u * kSliceStride, u < k);
      b0[u] = ld_stream_u32x2_if(m + (size_t)u * kSliceStride, u < k);
    }
#pragma unroll
    for (int u = 0; u < G; ++u) v0[u] = ld_value_hi_if(V + r0[u], u < k);
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int32_t t = G + u;
      r1[u] = ld_stream_i32_if(rows + (size_t)t * kSliceStride, t < k);
      b1[u] = ld_stream_u32x2_if(m + (size_t)t * kSliceStride, t < k);
    }
  }
  for (int32_t t0 = 0; t0 < len; t0 += G) {
    uint32_t vn[G];
#pragma unroll
    for (int u = 0; u < G; ++u) vn[u] = ld_value_hi_if(V + r1[u], t0 + G + u < k);
    int32_t r2[G];
    uint2 b2[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int32_t t = t0 + 2 * G + u;
      r2[u] = ld_stream_i32_if(rows + (size_t)t * kSliceStride, t < k);
      b2[u] = ld_stream_u32x2_if(m + (size_t)t * kSliceStride, t < k);
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const bool below = pess ? (v0[u] < vk) : (v0[u] > vk);
      const uint32_t g = below ? b0[u].y : 0u;
      acc += ((uint64_t)v0[u] * (uint64_t)(b0[u].x + g)) >> s;
      flt += g;
      geq += v0[u] == vk ? b0[u].y : 0u;
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      v0[u] = vn[u];
      b0[u] = b1[u];
      r1[u] = r2[u];
      b1[u] = b2[u];
    }
  }
}

// One slice g of window (tile) t: q of its columns into P.qcol, hints updated;
// the warp that completes the window finishes its states.
template <bool f32>
__device__ void slice_run(const StepLaunch& L, const Problem& P, const Tile& T, int32_t t, int32_t g, int32_t k_iter,
                          WarpScratch* ws, int lane) {
  const uint64_t* __restrict__ Vin = P.V[(k_iter - 1) & 1];
  const bool pess = P.pessimistic != 0;
  const SliceMeta sm = P.sl_meta[g];
  const int2 sl = P.sl_slot[(size_t)g * 32 + lane];
  const int32_t c = sl.x, k = sl.y;
  uint64_t rem_word = 0;
  int32_t h = -1, sh = 0, xo = -1;
  if (c >= 0) {
    rem_word = __ldg(P.rem + c);
    h = P.hint ? P.hint[c] : -1;
    if (f32) {
      sh = __ldg(P.shift + c);
      xo = P.xoff ? __ldg(P.xoff + c) : -1;
    }
  }
  // hint -2 - i: entry i, and the column's threshold is moving (no neighbour check)
  const int32_t entry = h <= -2 ? -2 - h : h;
  const uint64_t rem = rem_of(rem_word);
  const int32_t* rows = P.sl_rows + sm.off + lane;
  // lanes that run the warm start: rem = 0 (every entry at its lower bound), or a hint
  const bool warm = c >= 0 && xo < 0 && (rem == 0 || (entry >= 0 && entry < k));
  const int32_t kk = warm ? k : 0;
  const int32_t len = (int32_t)__reduce_max_sync(kFull, (unsigned)kk);  // trips any lane needs
  uint64_t acc = 0, flt = 0, geq = 0, q = 0;
  int32_t hout = h;
  bool done = false;
  WarmMiss miss;
  miss.valid = false;
  if (f32) {
    const uint2* lg = static_cast<const uint2*>(P.sl_lg) + sm.off + lane;
    // rem = 0: a key no value passes, so every entry keeps its lower bound
    uint32_t vk = pess ? 0u : 0xffffffffu;
    if (warm && rem != 0) vk = ld_value_hi(Vin + ld_stream_i32(rows + (size_t)entry * kSliceStride));
    lane_pass32(rows, lg, len, kk, Vin, vk, sh, pess, acc, flt, geq);
    if (warm) {
      const int down = 32 - sh;
      const uint64_t rem_m = rem >> down;  // exact: rem is a multiple of 2^down
      if (rem == 0) {
        q = acc;
        done = true;
      } else if (flt < rem_m && rem_m - flt <= geq) {
        q = acc + mul_shr(vk, rem_m - flt, sh);
        done = true;
      } else {
        miss = WarmMiss{(uint64_t)vk << 32, acc, shl_sat(flt, down), shl_sat(geq, down), true};
      }
    }
  } else {
    const ulonglong2* lg = static_cast<const ulonglong2*>(P.sl_lg) + sm.off + lane;
    uint64_t vk = pess ? 0ull : ~0ull;
    if (warm && rem != 0) vk = ld_value(Vin + ld_stream_i32(rows + (size_t)entry * kSliceStride));
    // narrow columns (every gap sum < 2^64) need no saturation
    if (__all_sync(kFull, !warm || rem == 0 || narrow_of(rem_word)))
      lane_pass64<false>(rows, lg, len, kk, Vin, vk, pess, acc, flt, geq);
    else
      lane_pass64<true>(rows, lg, len, kk, Vin, vk, pess, acc, flt, geq);
    if (warm) {
      if (rem == 0) {
        q = acc;
        done = true;
      } else if (flt < rem && rem - flt <= geq) {
        q = acc + __umul64hi(vk, rem - flt);
        done = true;
      } else {
        miss = WarmMiss{vk, acc, flt, geq, true};
      }
    }
  }
  if (done) hout = entry;
  // the rest, one column at a time with the whole warp
  unsigned need = __ballot_sync(kFull, c >= 0 && !done);
  while (need) {
    const int src = __ffs(need) - 1;
    need &= need - 1;
    const int32_t cs = __shfl_sync(kFull, c, src), ks = __shfl_sync(kFull, k, src);
    const int32_t hs = __shfl_sync(kFull, h, src);
    const uint64_t rws = __shfl_sync(kFull, rem_word, src);
    const int32_t xs = f32 ? __shfl_sync(kFull, xo, src) : -1;
    uint64_t qq;
    int32_t ho;
    const int32_t ca = __ldg(P.colptr + cs);
    if (f32 && xs >= 0) {
      // a correction column (no entries in the slice arrays): its exact bounds
      const int32_t ce = __ldg(P.colptr + cs + 1);
      qq = column_q<false, 1>(GRows{P.rowval + ca}, Bounds<false, 1>{P.lgx + xs, 0}, ce - ca, rws, GlobalV{Vin}, pess,
                              ws, lane, hs, &ho);
    } else {
      WarmMiss w;
      w.valid = __shfl_sync(kFull, miss.valid ? 1 : 0, src) != 0;
      w.vk = __shfl_sync(kFull, miss.vk, src);
      w.acc = __shfl_sync(kFull, miss.acc, src);
      w.flt = __shfl_sync(kFull, miss.flt, src);
      w.geq = __shfl_sync(kFull, miss.geq, src);
      // the column's CSC copy: contiguous, so the passes below are coalesced
      const GRows rs{P.rowval + ca};
      const void* bp = f32 ? static_cast<const void*>(P.lg32 + ca) : static_cast<const void*>(P.lg + ca);
      const Bounds<f32, 1> bs{bp, f32 ? 32 - __shfl_sync(kFull, sh, src) : 0};
      const bool nb = w.valid && hs > -2 &&
                      column_neighbor<f32, 1>(rs, bs, ks, rem_of(rws), GlobalV{Vin}, pess, lane, w, &qq, &ho);
      if (!nb) {
        int32_t found;
        qq = column_search<f32, 1>(rs, bs, ks, rws, GlobalV{Vin}, pess, ws, lane, &found);
        ho = found >= 0 ? -2 - found : -1;
      }
    }
    if (lane == src) {
      q = qq;
      hout = ho;
    }
  }
  if (c >= 0) {
    P.qcol[c] = q;
    if (P.hint && hout != h) P.hint[c] = hout;
  }
  // count the slice; the warp that completes the window finishes its states
  __threadfence();
  __syncwarp();
  unsigned prev = 0;
  if (lane == 0) prev = atomicAdd(&L.win_cnt[t], 1u);
  prev = __shfl_sync(kFull, prev, 0);
  if (prev + 1 == (unsigned)(T.x1 - T.x0)) {
    __threadfence();
    const unsigned long long* qc = reinterpret_cast<const unsigned long long*>(P.qcol);
    tile_epilogue(L, P, T, k_iter, lane, [&](int32_t s) { return (uint8_t)__ldg(P.fixed + s); },
                  [&](int32_t s, uint64_t* bq, int32_t* bb) {
                    const int32_t jb = __ldg(P.stateptr + s), je = __ldg(P.stateptr + s + 1);
                    best_action(P, jb, je, [&](int32_t jj) { return (uint64_t)__ldcg(qc + jj); }, bq, bb);
                  });
    if (lane == 0) L.win_cnt[t] = 0;  // for the next launch
  }
}

template <int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) bellman_slice_kernel(StepLaunch L) {
  __shared__ WarpScratch ws_all[NW];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31;
  WarpScratch* ws = &ws_all[threadIdx.x >> 5];
  const int32_t nt = tiles_to_visit(L);
  const int32_t ni = nt <= 0 ? 0 : (nt >= L.n_tiles ? L.n_items : L.tile_item_end[nt - 1]);
  for (;;) {
    int32_t i = 0;
    if (lane == 0) i = (int32_t)atomicAdd(&L.ctl->tile_next, 1u);
    i = __shfl_sync(kFull, i, 0);
    if (i >= ni) break;
    const int2 it = L.items[i];
    const Tile T = L.tiles[it.x];
    int32_t k_iter;
    if (!problem_active(L, T.p, &k_iter)) continue;
    const Problem& P = L.probs[T.p];
    if (P.lg32)
      slice_run<true>(L, P, T, it.x, it.y, k_iter, ws, lane);
    else
      slice_run<false>(L, P, T, it.x, it.y, k_iter, ws, lane);
  }
  end_of_launch(L, &is_last);
}

// ---------------------------------------------------------------- small problems
//
// One CTA runs all n iterations of a session holding one small problem in a
// single launch: the model (destinations, bound pairs, column words, hints) and
// both value buffers are copied into shared memory once, each iteration
// computes the problem's states from there (warps take states), and the
// iteration state advances exactly as end_of_launch advances it after every
// launch of the tiled kernels. The columns run the same exact routines (V read
// from shared memory), so the words are those of the tiled kernels. This
// removes the per-iteration launch (a few microseconds each, more than the
// work of such a problem).
constexpr int kTinyWarps = 4;

struct TinyLayout {
  size_t lg, v, rem, sptr, cptr, rows, hint, shift, xoff, fixed, ws, bytes;
};

__host__ __device__ inline TinyLayout tiny_layout(int32_t n, int32_t m, int32_t nnz, bool f32) {
  auto up = [](size_t x) { return (x + 15) & ~size_t(15); };
  TinyLayout t;
  size_t o = 0;
  t.lg = o;    o = up(o + (size_t)nnz * (f32 ? sizeof(uint2) : sizeof(ulonglong2)));
  t.v = o;     o = up(o + 2 * (size_t)n * sizeof(uint64_t));
  t.rem = o;   o = up(o + (size_t)m * sizeof(uint64_t));
  t.sptr = o;  o = up(o + (size_t)(n + 1) * sizeof(int32_t));
  t.cptr = o;  o = up(o + (size_t)(m + 1) * sizeof(int32_t));
  t.rows = o;  o = up(o + (size_t)nnz * sizeof(int32_t));
  t.hint = o;  o = up(o + (size_t)m * sizeof(int32_t));
  t.shift = o; o = up(o + (size_t)m * sizeof(int32_t));
  t.xoff = o;  o = up(o + (size_t)m * sizeof(int32_t));
  t.fixed = o; o = up(o + (size_t)n);
  t.ws = o;    o = up(o + kTinyWarps * sizeof(WarpScratch));
  t.bytes = o;
  return t;
}

template <bool f32>
__global__ void __launch_bounds__(32 * kTinyWarps, 1) bellman_tiny_kernel(StepLaunch L, int32_t n_iters) {
  extern __shared__ __align__(16) unsigned char sm[];
  const Problem& P = L.probs[0];
  const int32_t n = P.n_states;
  const int32_t m = P.stateptr[n];
  const int32_t nnz = P.colptr[m];
  const TinyLayout lay = tiny_layout(n, m, nnz, f32);
  uint64_t* V0 = reinterpret_cast<uint64_t*>(sm + lay.v);
  uint64_t* rem = reinterpret_cast<uint64_t*>(sm + lay.rem);
  int32_t* sptr = reinterpret_cast<int32_t*>(sm + lay.sptr);
  int32_t* cptr = reinterpret_cast<int32_t*>(sm + lay.cptr);
  int32_t* rows = reinterpret_cast<int32_t*>(sm + lay.rows);
  int32_t* hint = reinterpret_cast<int32_t*>(sm + lay.hint);
  int32_t* shift = reinterpret_cast<int32_t*>(sm + lay.shift);
  int32_t* xoff = reinterpret_cast<int32_t*>(sm + lay.xoff);
  uint8_t* fixed = sm + lay.fixed;
  WarpScratch* ws = reinterpret_cast<WarpScratch*>(sm + lay.ws) + (threadIdx.x >> 5);
  __shared__ IterState it;
  __shared__ unsigned long long dmax_b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int32_t i = tid; i < nnz; i += nt) {
    rows[i] = P.rowval[i];
    if (f32)
      reinterpret_cast<uint2*>(sm + lay.lg)[i] = P.lg32[i];
    else
      reinterpret_cast<ulonglong2*>(sm + lay.lg)[i] = P.lg[i];
  }
  for (int32_t i = tid; i < n; i += nt) {
    V0[i] = P.V[0][i];
    V0[n + i] = P.V[1][i];
    fixed[i] = P.fixed[i];
  }
  for (int32_t i = tid; i <= n; i += nt) sptr[i] = P.stateptr[i];
  for (int32_t i = tid; i <= m; i += nt) cptr[i] = P.colptr[i];
  for (int32_t c = tid; c < m; c += nt) {
    rem[c] = P.rem[c];
    hint[c] = P.hint ? P.hint[c] : -1;
    if (f32) {
      shift[c] = P.shift[c];
      xoff[c] = P.xoff ? P.xoff[c] : -1;
    }
  }
  if (tid == 0) it = L.its[0];
  __syncthreads();

  const bool pess = P.pessimistic != 0, maxi = P.maximize != 0;
  for (int32_t step = 0; step < n_iters; ++step) {
    if (it.done) break;  // later launches would change nothing
    const int32_t k_iter = it.iter + 1;
    const bool active = P.infinite || k_iter <= P.horizon;
    if (tid == 0) dmax_b = 0;
    __syncthreads();
    if (active) {
      const SharedV Vin{V0 + (size_t)((k_iter - 1) & 1) * n};
      uint64_t* Vout = V0 + (size_t)(k_iter & 1) * n;
      unsigned long long dmax = 0;
      for (int32_t s = warp; s < n; s += kTinyWarps) {
        if (fixed[s]) continue;  // Eq. 2 fixes reach and avoid states (both buffers hold their values)
        const int32_t jb = sptr[s], je = sptr[s + 1];
        uint64_t bq = 0;
        int32_t best = -1;
        for (int32_t c = jb; c < je; ++c) {
          const int32_t ca = cptr[c], ce = cptr[c + 1];
          const int32_t h = hint[c];
          int32_t hout;
          uint64_t q;
          if (f32 && xoff[c] >= 0)  // correction column: its exact pairs from global memory
            q = column_q<false, true>(GRows{P.rowval + ca}, Bounds<false, true>{P.lgx + xoff[c], 0}, ce - ca, rem[c],
                                      Vin, pess, ws, lane, h, &hout);
          else if (f32)
            q = column_q<true, false>(rows + ca, Bounds<true>{reinterpret_cast<const uint2*>(sm + lay.lg) + ca,
                                                              32 - shift[c]},
                                      ce - ca, rem[c], Vin, pess, ws, lane, h, &hout);
          else
            q = column_q<false, false>(rows + ca, Bounds<false>{reinterpret_cast<const ulonglong2*>(sm + lay.lg) + ca, 0},
                                       ce - ca, rem[c], Vin, pess, ws, lane, h, &hout);
          if (lane == 0) hint[c] = hout;
          if (best < 0 || (maxi ? q > bq : q < bq)) {
            bq = q;
            best = c - jb;
          }
        }
        const uint64_t vnew = free_state_value(P, s, bq);
        if (lane == 0) {
          Vout[s] = vnew;
          if (P.policy_mode == 1)
            P.policy[(size_t)(P.horizon - k_iter) * P.n_states + s] = best;
          else if (P.policy_mode == 2)
            P.policy[s] = best;
          if (P.infinite) {
            const uint64_t vold = Vin.p[s];
            const uint64_t d = vnew > vold ? vnew - vold : vold - vnew;
            dmax = d > dmax ? d : dmax;
          }
        }
      }
      if (lane == 0 && dmax) atomicMax(&dmax_b, dmax);
    }
    __syncthreads();
    if (tid == 0) {  // the iteration state, as end_of_launch advances it
      const int32_t kq = it.iter + 1;
      if (!P.infinite && kq > P.horizon) {
        it.done = 1;
        it.k_final = it.iter;
      } else {
        it.iter = kq;
        if (P.infinite) {
          if (dmax_b < P.eps_fix && !P.external_stop) {
            it.done = 1;
            it.k_final = kq;
          } else if (kq >= P.horizon) {
            it.done = 1;
            it.k_final = kq;
            it.noconv = 1;
          }
        } else if (kq >= P.horizon) {
          it.done = 1;
          it.k_final = kq;
        }
      }
    }
    __syncthreads();
  }

  for (int32_t i = tid; i < n; i += nt) {
    P.V[0][i] = V0[i];
    P.V[1][i] = V0[n + i];
  }
  if (P.hint)
    for (int32_t c = tid; c < m; c += nt) P.hint[c] = hint[c];
  if (tid == 0) {
    IterState out = it;
    out.resmax = 0;
    L.its[0] = out;
  }
}

// ---------------------------------------------------------------- wide states
//
// A state whose entries do not fit one stage, or that has a column of kWideCol
// entries or more, is handled by the 4 warps of a CTA together: thread t takes
// entries t, t + 128, ... of each column, and the warps' partial sums are
// combined through shared memory between __syncthreads (no spin waits). Every
// sum is the same multiset of exact integer terms as in the one-warp routines
// (and candidate ties are ordered by entry index, as there), so a wide state
// gets the same result, to the bit, as it would in a tile.

constexpr int kWideWarps = 4;
constexpr int kWideThreads = 32 * kWideWarps;

struct WideShared {
  unsigned long long r[4][kWideWarps];  // per-warp partials
  int32_t ri[kWideWarps];
  int32_t rh[kWideWarps];
  unsigned int hl[kBins];               // histogram as in WarpScratch
  unsigned int hh[kBins];
  unsigned int hc[kBins];
  unsigned int hsat[2];
  unsigned long long ck[32];            // candidates: key, gap, entry
  unsigned long long cg[32];
  int32_t ci[32];
  unsigned int ncand;
  int32_t first_cand;
  unsigned long long bc[4];             // values broadcast by warp 0
  int32_t bci[2];
};

// Block sums of per-thread values: a mod 2^64, f and g saturating (inputs as for
// warp_sum_sat). Two barriers: the partials are published, then free again.
__device__ __forceinline__ void block_sum3(WideShared& W, int warp, int lane, uint64_t& a, uint64_t& f,
                                           uint64_t& g) {
  a = warp_sum_u64(a);
  f = warp_sum_sat(f);
  g = warp_sum_sat(g);
  if (lane == 0) {
    W.r[0][warp] = a;
    W.r[1][warp] = f;
    W.r[2][warp] = g;
  }
  __syncthreads();
  a = f = g = 0;
  for (int w = 0; w < kWideWarps; ++w) {
    a += W.r[0][w];
    f = sat_add(f, W.r[1][w]);
    g = sat_add(g, W.r[2][w]);
  }
  __syncthreads();
}

__device__ __forceinline__ void block_minmax(WideShared& W, int warp, int lane, uint64_t& mn, uint64_t& mx) {
  mn = warp_min_u64(mn);
  mx = warp_max_u64(mx);
  if (lane == 0) {
    W.r[0][warp] = mn;
    W.r[1][warp] = mx;
  }
  __syncthreads();
  mn = ~0ull;
  mx = 0;
  for (int w = 0; w < kWideWarps; ++w) {
    mn = W.r[0][w] < mn ? W.r[0][w] : mn;
    mx = W.r[1][w] > mx ? W.r[1][w] : mx;
  }
  __syncthreads();
}

// Neighbour check of column_neighbor, block-wide.
template <bool f32>
__device__ bool wide_neighbor(const int32_t* __restrict__ rows, const Bounds<f32> lg, int32_t k, uint64_t rem,
                              const uint64_t* __restrict__ V, bool pess, uint64_t vk, uint64_t acc, uint64_t flt,
                              uint64_t geq, uint64_t* q, int32_t* hint_out, WideShared& W) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool down = flt >= rem;
  if (down && flt >= kOne) return false;
  const uint64_t kap = pess ? vk : kOne - vk;
  uint64_t best = 0, gs = 0, ds = 0, dk = 0;
  bool have = false;
  int32_t bi = -1;
#pragma unroll 4
  for (int idx = tid; idx < k; idx += kWideThreads) {
    const uint64_t v = ld_value(V + rows[idx]);
    const uint64_t key = pess ? v : kOne - v;
    const ulonglong2 b = lg[idx];
    const uint64_t d = __umul64hi(v, b.x + b.y) - __umul64hi(v, b.x);
    const bool side = down ? key < kap : key > kap;
    if (side) {
      if (!have || (down ? key > best : key < best)) {
        best = key;
        gs = b.y;
        ds = d;
        bi = idx;
        have = true;
      } else if (key == best) {
        gs = sat_add(gs, b.y);
        ds += d;
        bi = idx < bi ? idx : bi;
      }
    } else if (!down && key == kap) {
      dk += d;
    }
  }
  const bool any = __any_sync(kFull, have);
  const uint64_t tw = down ? warp_max_u64(have ? best : 0ull) : warp_min_u64(have ? best : ~0ull);
  const bool mine = have && best == tw;
  const uint64_t Gw = warp_sum_sat(mine ? gs : 0ull);
  const uint64_t Dw = warp_sum_u64(mine ? ds : 0ull);
  const uint64_t DKw = warp_sum_u64(dk);
  const int32_t hw = __reduce_min_sync(kFull, mine ? (unsigned)bi : 0x7fffffffu);
  if (lane == 0) {
    W.rh[warp] = any ? 1 : 0;
    W.r[0][warp] = tw;
    W.r[1][warp] = Gw;
    W.r[2][warp] = Dw;
    W.r[3][warp] = DKw;
    W.ri[warp] = hw;
  }
  __syncthreads();
  bool anyb = false;
  uint64_t t = down ? 0ull : ~0ull;
  for (int w = 0; w < kWideWarps; ++w)
    if (W.rh[w]) {
      anyb = true;
      t = down ? (W.r[0][w] > t ? W.r[0][w] : t) : (W.r[0][w] < t ? W.r[0][w] : t);
    }
  uint64_t G = 0, D = 0, DK = 0;
  int32_t h = 0x7fffffff;
  for (int w = 0; w < kWideWarps; ++w) {
    DK += W.r[3][w];
    if (W.rh[w] && W.r[0][w] == t) {
      G = sat_add(G, W.r[1][w]);
      D += W.r[2][w];
      h = W.ri[w] < h ? W.ri[w] : h;
    }
  }
  __syncthreads();
  if (!anyb) return false;
  const uint64_t vt = pess ? t : kOne - t;
  if (down) {
    const uint64_t fl = flt - G;
    if (fl >= rem) return false;
    *q = acc - D + __umul64hi(vt, rem - fl);
  } else {
    const uint64_t fl = flt + geq;
    if (sat_add(fl, G) < rem) return false;
    *q = acc + DK + __umul64hi(vt, rem - fl);
  }
  *hint_out = h;
  return true;
}

// Threshold search of column_search, block-wide.
template <bool f32>
__device__ uint64_t wide_search(const int32_t* __restrict__ rows, const Bounds<f32> lg, int32_t k, uint64_t rem,
                                const uint64_t* __restrict__ V, bool pess, int32_t* found, WideShared& W) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto key_of = [&](int idx) -> uint64_t {
    const uint64_t v = ld_value(V + rows[idx]);
    return pess ? v : (kOne - v);
  };
  uint64_t cmin = ~0ull, cmax = 0;
#pragma unroll 4
  for (int idx = tid; idx < k; idx += kWideThreads) {
    const uint64_t key = key_of(idx);
    cmin = key < cmin ? key : cmin;
    cmax = key > cmax ? key : cmax;
  }
  block_minmax(W, warp, lane, cmin, cmax);
  uint64_t lo = 0, hi = kOne, fb = 0;
  bool all_below = false, uniform = false;
  for (int round = 0; round < 12; ++round) {
    if (cmin > cmax) {
      all_below = true;
      break;
    }
    if (cmin == cmax) {
      lo = hi = cmin;
      uniform = true;
      break;
    }
    const int bits = 64 - __clzll((long long)(cmax - cmin));
    const int shift = bits > 6 ? bits - 6 : 0;
    if (tid < kBins) {
      W.hl[tid] = 0;
      W.hh[tid] = 0;
      W.hc[tid] = 0;
    }
    if (tid == 0) W.hsat[0] = W.hsat[1] = 0;
    __syncthreads();
#pragma unroll 4
    for (int idx = tid; idx < k; idx += kWideThreads) {
      const uint64_t key = key_of(idx);
      if (key >= lo && key <= hi) {
        const int b = (int)((key - cmin) >> shift);
        const uint64_t g = lg[idx].y < rem ? lg[idx].y : rem;
        const unsigned gl = (unsigned)g;
        const unsigned old = atomicAdd(&W.hl[b], gl);
        const unsigned up = (unsigned)(g >> 32) + ((old + gl) < old ? 1u : 0u);
        if (up) {
          const unsigned oh = atomicAdd(&W.hh[b], up);
          if (oh + up < oh) atomicOr(&W.hsat[b >> 5], 1u << (b & 31));
        }
        atomicAdd(&W.hc[b], 1u);
      }
    }
    __syncthreads();
    if (warp == 0) {
      const unsigned sat = W.hsat[lane >> 4];
      const uint64_t h0 = ((sat >> ((2 * lane) & 31)) & 1u) ? ~0ull
                                                            : (((uint64_t)W.hh[2 * lane] << 32) | W.hl[2 * lane]);
      const uint64_t h1 = ((sat >> ((2 * lane + 1) & 31)) & 1u)
                              ? ~0ull
                              : (((uint64_t)W.hh[2 * lane + 1] << 32) | W.hl[2 * lane + 1]);
      const uint64_t ex = warp_excl_scan_sat(sat_add(h0, h1), lane);
      const uint64_t i0 = sat_add(sat_add(fb, ex), h0), i1 = sat_add(i0, h1);
      const unsigned cross = __ballot_sync(kFull, i1 >= rem);
      if (cross == 0) {
        if (lane == 0) W.bci[0] = -1;
      } else {
        const int L = __ffs(cross) - 1;
        const bool first = i0 >= rem;
        const int b = __shfl_sync(kFull, first ? 2 * lane : 2 * lane + 1, L);
        const uint64_t f2 = __shfl_sync(kFull, first ? sat_add(fb, ex) : i0, L);
        if (lane == 0) {
          W.bci[0] = b;
          W.bci[1] = (int32_t)W.hc[b];
          W.bc[0] = f2;
        }
      }
    }
    __syncthreads();
    const int b = W.bci[0];
    const unsigned cnt = (unsigned)W.bci[1];
    const uint64_t f2 = W.bc[0];
    __syncthreads();
    if (b < 0) {  // first round only: the gaps cannot absorb rem
      all_below = true;
      break;
    }
    fb = f2;
    lo = cmin + ((uint64_t)b << shift);
    const uint64_t top = lo + ((1ull << shift) - 1ull);
    hi = top < cmax ? top : cmax;
    if (cnt <= 32) break;
    uint64_t a = ~0ull, z = 0;
#pragma unroll 4
    for (int idx = tid; idx < k; idx += kWideThreads) {
      const uint64_t key = key_of(idx);
      if (key >= lo && key <= hi) {
        a = key < a ? key : a;
        z = key > z ? key : z;
      }
    }
    block_minmax(W, warp, lane, a, z);
    cmin = a;
    cmax = z;
  }
  // final pass
  if (tid == 0) {
    W.ncand = 0;
    W.first_cand = 0x7fffffff;
  }
  __syncthreads();
  uint64_t acc = 0, gsum = 0, unused = 0;
#pragma unroll 4
  for (int idx = tid; idx < k; idx += kWideThreads) {
    const uint64_t key = key_of(idx);
    const ulonglong2 b = lg[idx];
    const bool below = all_below || key < lo;
    const bool cand = !all_below && key >= lo && key <= hi;
    acc += __umul64hi(pess ? key : (kOne - key), below ? b.x + b.y : b.x);
    if (cand) {
      atomicMin(&W.first_cand, idx);
      const uint64_t g = b.y < rem ? b.y : rem;
      if (uniform) {
        gsum = sat_add(gsum, g);
      } else {
        const unsigned at = atomicAdd(&W.ncand, 1u);
        if (at < 32) {
          W.ck[at] = key;
          W.cg[at] = g;
          W.ci[at] = idx;
        }
      }
    }
  }
  block_sum3(W, warp, lane, acc, gsum, unused);
  if (all_below) {
    *found = -1;
    return acc;
  }
  const uint64_t r2 = rem - fb;
  if (uniform) {
    *found = W.first_cand;
    return acc + __umul64hi(pess ? lo : (kOne - lo), gsum < r2 ? gsum : r2);
  }
  // resolve the <= 32 candidates in (key, entry) order, as the one-warp search does
  if (warp == 0) {
    const unsigned pos = W.ncand < 32u ? W.ncand : 32u;
    uint64_t extra = 0;
    int thr = -1;
    if (lane < (int)pos) {
      const uint64_t ki = W.ck[lane], gi = W.cg[lane];
      const int32_t ii = W.ci[lane];
      uint64_t before = 0;
      for (unsigned j = 0; j < pos; ++j) {
        const uint64_t kj = W.ck[j];
        if (kj < ki || (kj == ki && W.ci[j] < ii)) before = sat_add(before, W.cg[j]);
      }
      const uint64_t left = r2 > before ? r2 - before : 0;
      extra = __umul64hi(pess ? ki : (kOne - ki), gi < left ? gi : left);
      if (left > 0 && left <= gi) thr = ii;
    }
    extra = warp_sum_u64(extra);
    const int32_t t = __reduce_min_sync(kFull, thr >= 0 ? (unsigned)thr : 0x7fffffffu);
    if (lane == 0) {
      W.bc[1] = extra;
      W.bci[0] = t == 0x7fffffff ? -1 : t;
    }
  }
  __syncthreads();
  const uint64_t q = acc + W.bc[1];
  *found = W.bci[0];
  __syncthreads();
  return q;
}

// One column of a wide state: warm start, neighbour check, search (the same
// sequence and hint encoding as column_q).
template <bool f32>
__device__ uint64_t wide_column_q(const int32_t* __restrict__ rows, const Bounds<f32> lg, int32_t k,
                                  uint64_t rem_word, const uint64_t* __restrict__ V, bool pess, int32_t hint,
                                  int32_t* hint_out, WideShared& W) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t rem = rem_of(rem_word);
  const bool moving = hint <= -2;
  const int32_t entry = moving ? -2 - hint : hint;
  if (rem == 0) {
    uint64_t a = 0, f = 0, g = 0;
#pragma unroll 4
  for (int idx = tid; idx < k; idx += kWideThreads) a += __umul64hi(ld_value(V + rows[idx]), lg[idx].x);
    block_sum3(W, warp, lane, a, f, g);
    *hint_out = entry;
    return a;
  }
  if (entry >= 0 && entry < k) {
    const uint64_t vk = ld_value(V + rows[entry]);
    uint64_t acc = 0, flt = 0, geq = 0;
    uint32_t fc = 0, gc = 0;
#pragma unroll 4
    for (int idx = tid; idx < k; idx += kWideThreads) {
      const uint64_t v = ld_value(V + rows[idx]);
      const ulonglong2 b = lg[idx];
      const bool below = pess ? (v < vk) : (v > vk);
      acc += __umul64hi(v, b.x + (below ? b.y : 0ull));
      const uint64_t gb = below ? b.y : 0ull, ge = v == vk ? b.y : 0ull;
      flt += gb;
      fc += flt < gb ? 1u : 0u;
      geq += ge;
      gc += geq < ge ? 1u : 0u;
    }
    flt = fc ? ~0ull : flt;
    geq = gc ? ~0ull : geq;
    block_sum3(W, warp, lane, acc, flt, geq);
    if (flt < rem && rem - flt <= geq) {
      *hint_out = entry;
      return acc + __umul64hi(vk, rem - flt);
    }
    uint64_t q;
    int32_t h;
    if (!moving && wide_neighbor<f32>(rows, lg, k, rem, V, pess, vk, acc, flt, geq, &q, &h, W)) {
      *hint_out = h;
      return q;
    }
  }
  int32_t found;
  const uint64_t q = wide_search<f32>(rows, lg, k, rem, V, pess, &found, W);
  *hint_out = found >= 0 ? -2 - found : -1;
  return q;
}

// One Bellman step of the wide states: each CTA takes the next wide state until
// none is left. It runs beside bellman_step_kernel (on a second stream, in the
// room one persistent tiled CTA leaves on each SM) or before it: both read
// V_{k-1} and write disjoint states of V_k, and whichever CTA of the two
// kernels finishes last advances the iteration state.
__global__ void __launch_bounds__(kWideThreads, 6) bellman_wide_kernel(StepLaunch L) {
  __shared__ WideShared W;
  __shared__ int take;
  __shared__ int is_last;
  for (;;) {
    if (threadIdx.x == 0) take = (int)atomicAdd(&L.ctl->wide_next, 1u);
    __syncthreads();
    const int32_t w = take;
    __syncthreads();
    if (w >= L.n_wide) break;
    const int2 ps = L.wide[w];
    const Problem& P = L.probs[ps.x];
    int32_t k_iter;
    if (!problem_active(L, ps.x, &k_iter)) continue;
    const int32_t s = ps.y;
    const uint8_t fx = P.fixed[s];
    const uint64_t* __restrict__ Vin = P.V[(k_iter - 1) & 1];
    uint64_t* __restrict__ Vout = P.V[k_iter & 1];
    uint64_t vnew;
    int32_t best = -1;
    if (fx == 1) {
      vnew = kOne;
    } else if (fx == 2) {
      vnew = 0;
    } else {
      const bool pess = P.pessimistic != 0;
      const int32_t c0 = __ldg(P.stateptr + s), c1 = __ldg(P.stateptr + s + 1);
      uint64_t bestq = 0;
      for (int32_t c = c0; c < c1; ++c) {
        const int32_t ca = __ldg(P.colptr + c), ce = __ldg(P.colptr + c + 1);
        const int32_t h = P.hint ? P.hint[c] : -1;
        int32_t hout;
        uint64_t q;
        const int32_t xo = P.xoff ? __ldg(P.xoff + c) : -1;
        if (P.lg32 && xo < 0)
          q = wide_column_q<true>(P.rowval + ca, Bounds<true>{P.lg32 + ca, 32 - __ldg(P.shift + c)}, ce - ca,
                                  __ldg(P.rem + c), Vin, pess, h, &hout, W);
        else if (P.lg32)  // correction column: its exact bounds
          q = wide_column_q<false>(P.rowval + ca, Bounds<false>{P.lgx + xo, 0}, ce - ca, __ldg(P.rem + c), Vin, pess,
                                   h, &hout, W);
        else
          q = wide_column_q<false>(P.rowval + ca, Bounds<false>{P.lg + ca, 0}, ce - ca, __ldg(P.rem + c), Vin, pess,
                                   h, &hout, W);
        if (threadIdx.x == 0 && P.hint && hout != h) P.hint[c] = hout;
        if (best < 0 || (P.maximize ? q > bestq : q < bestq)) {
          bestq = q;
          best = c - c0;
        }
      }
      vnew = free_state_value(P, s, bestq);
    }
    if (threadIdx.x == 0) {
      unsigned long long dmax = 0;
      finish_state(P, s, k_iter, vnew, best, Vin, Vout, dmax);
      if (P.infinite && dmax) atomicMax(&L.its[ps.x].resmax, dmax);
    }
  }
  end_of_launch(L, &is_last);
}

}  // namespace

void plan_tiles(const DevModel* m, int32_t problem, std::vector<Tile>& out, std::vector<int32_t>& wide,
                int32_t tile_entries, int32_t wide_col, const uint8_t* fixed) {
  const std::vector<int32_t>& sp = m->h_stateptr;
  const std::vector<int32_t>& cp = m->h_colptr;
  const int32_t n = m->own1;  // owned states only
  const int32_t te = tile_entries > 0 && tile_entries < kTileEntries ? tile_entries : kTileEntries;
  const int32_t wc = wide_col > 0 ? wide_col : kWideCol;
  // states whose values the property fixes (Eq. 2) are in no tile and no wide list
  auto is_fixed = [&](int32_t s) { return fixed && fixed[s]; };
  // 32-bit storage with correction columns: a stage's bound area holds the
  // tile's 8-byte mantissa pairs followed by its correction columns' 16-byte
  // exact pairs
  const std::vector<int32_t>& xo = m->h_xoff;
  auto stage_fits = [&](int32_t c0, int32_t c1, int32_t e0, int32_t e1) {
    if (xo.empty()) return true;
    int64_t x = 0;
    for (int32_t c = c0; c < c1; ++c)
      if (xo[c] >= 0) x += cp[c + 1] - cp[c];
    const int64_t pairs32 = (((int64_t)e1 + 1) & ~1) - (e0 & ~1);
    return 8 * pairs32 + 16 * x <= (int64_t)sizeof(ulonglong2) * kTileEntries;
  };
  auto is_wide = [&](int32_t s) {
    if (cp[sp[s + 1]] - cp[sp[s]] > kTileEntries || sp[s + 1] - sp[s] > kTileCols) return true;
    if (!stage_fits(sp[s], sp[s + 1], cp[sp[s]], cp[sp[s + 1]])) return true;
    for (int32_t c = sp[s]; c < sp[s + 1]; ++c)
      if (cp[c + 1] - cp[c] >= wc) return true;
    return false;
  };
  int32_t s = m->own0;
  while (s < n) {
    if (is_fixed(s)) {
      ++s;
      continue;
    }
    if (is_wide(s)) {
      wide.push_back(s);
      ++s;
      continue;
    }
    Tile T;
    T.p = problem;
    T.s0 = s;
    T.c0 = sp[s];
    T.e0 = cp[sp[s]];
    int32_t t = s + 1;
    while (t < n && !is_fixed(t) && !is_wide(t) && cp[sp[t + 1]] - T.e0 <= te && sp[t + 1] - T.c0 <= kTileCols &&
           t + 1 - s <= kTileStates && stage_fits(T.c0, sp[t + 1], T.e0, cp[sp[t + 1]]))
      ++t;
    T.s1 = t;
    T.c1 = sp[T.s1];
    T.e1 = cp[T.c1];
    T.x0 = T.x1 = 0;
    if (!xo.empty()) {  // the correction columns' entries are consecutive in lgx
      int32_t a = -1, b = -1;
      for (int32_t c = T.c0; c < T.c1; ++c)
        if (xo[c] >= 0) {
          if (a < 0) a = xo[c];
          b = xo[c] + (cp[c + 1] - cp[c]);
        }
      if (a >= 0) {
        T.x0 = a;
        T.x1 = b;
      }
    }
    out.push_back(T);
    s = T.s1;
  }
}

int bellman_grid() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;  // persistent: one CTA per SM
}

std::atomic<int> g_stall_producer{0};

cudaError_t launch_bellman_tiny(const StepLaunch& L, int32_t n_iters, bool f32, cudaStream_t st) {
  static std::atomic<int> configured[64];
  static std::mutex setup;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev].load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lk(setup);
    if (!configured[dev].load(std::memory_order_relaxed)) {
      const int most = (int)tiny_layout(kTinyMaxStates, kTinyMaxCols, kTinyMaxEntries, false).bytes;
      cudaError_t e = cudaFuncSetAttribute(bellman_tiny_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bellman_tiny_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
      if (e != cudaSuccess) return e;
      configured[dev].store(1, std::memory_order_release);
    }
  }
  if (n_iters <= 0) return cudaSuccess;
  const size_t bytes = tiny_layout(L.tiny_states, L.tiny_cols, L.tiny_entries, f32).bytes;
  if (f32)
    bellman_tiny_kernel<true><<<1, 32 * kTinyWarps, bytes, st>>>(L, n_iters);
  else
    bellman_tiny_kernel<false><<<1, 32 * kTinyWarps, bytes, st>>>(L, n_iters);
  return cudaGetLastError();
}

LaunchConfig resolve_launch(const StepLaunch& L, const LaunchConfig* cfg) {
  LaunchConfig r;
  if (cfg) r = *cfg;
  if (r.kernel == kKernelTiny || (r.kernel == kKernelRule && L.tiny_ok)) {
    if (L.tiny_ok) {
      r.kernel = kKernelTiny;
      r.cta_warps = kTinyWarps;
      r.ctas_per_sm = 1;
      if (r.tile_entries <= 0 || r.tile_entries > kTileEntries) r.tile_entries = kTileEntries;
      if (r.wide_col <= 0) r.wide_col = kWideCol;
      return r;
    }
    r.kernel = kKernelRule;
  }
  if (r.kernel == kKernelRule && L.shape_rule) {
    r.kernel = L.shape_rule;
    if (r.ctas_per_sm <= 0) r.ctas_per_sm = (r.kernel == kKernelSlice && L.shape_f32) ? 4 : 3;
    if (r.kernel == kKernelDirect && r.tile_entries <= 0) r.tile_entries = kRuleDirectTile;
  }
  if (r.kernel == kKernelSlice) {
    r.cta_warps = kSliceWarps;
    r.ctas_per_sm = r.ctas_per_sm == 3 ? 3 : 4;
    r.tile_entries = kTileEntries;  // no tile plan: windows of the slice layout
    r.wide_col = kWideCol;
    return r;
  }
  if (r.kernel != kKernelDirect) r.kernel = kKernelRing;
  if (r.kernel == kKernelDirect) {
    r.cta_warps = kDirectWarps;
    r.ctas_per_sm = r.ctas_per_sm == 3 ? 3 : 4;
  } else {
    // 24 warps (23 consumers) for tiles of many short columns; never beside wide
    // CTAs (a 24-warp CTA leaves no registers for one)
    const bool can24 = L.n_wide == 0;
    const bool rule24 = can24 && L.tile_cols >= (int64_t)kShortColsPerTile * L.n_tiles;
    r.cta_warps = (r.cta_warps == 24 && can24) || (r.cta_warps != 16 && r.cta_warps != 24 && rule24)
                      ? kConsumersShort + 1
                      : kConsumersLong + 1;
    r.ctas_per_sm = 1;
  }
  if (r.tile_entries <= 0 || r.tile_entries > kTileEntries) r.tile_entries = kTileEntries;
  if (r.wide_col <= 0) r.wide_col = kWideCol;
  return r;
}

cudaError_t launch_bellman_step(const StepLaunch& L0, int grid, cudaStream_t st, const SideStream* side,
                                const LaunchConfig* cfg) {
  // per-device setup, once (sessions, servers and the allocation-free entry
  // point may launch from several threads)
  static std::atomic<int> configured[64];
  static int wide_blocks[64] = {0};
  static std::mutex setup;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev].load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lk(setup);
    if (!configured[dev].load(std::memory_order_relaxed)) {
      cudaError_t e = cudaFuncSetAttribute(bellman_step_kernel<kConsumersLong>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(Smem<kConsumersLong>));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bellman_step_kernel<kConsumersShort>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(Smem<kConsumersShort>));
      if (e != cudaSuccess) return e;
      int per_sm = 1, sms = 152;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bellman_wide_kernel, kWideThreads, 0);
      if (e != cudaSuccess) return e;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      wide_blocks[dev] = std::max(1, per_sm) * sms;
      configured[dev].store(1, std::memory_order_release);
    }
  }
  StepLaunch L = L0;
  L.stall = g_stall_producer.load(std::memory_order_relaxed);
  const LaunchConfig rc = resolve_launch(L, cfg);
  const int kind = rc.kernel;
  const int direct_per_sm = rc.ctas_per_sm;
  const bool short_cols = kind == kKernelRing && rc.cta_warps == kConsumersShort + 1;
  const int wg = L.n_wide > 0 ? std::min(L.n_wide, wide_blocks[dev]) : 0;
  // one CTA still takes part in the end-of-launch ticket when there are no tiles
  const int mg = L.n_tiles <= 0 ? 1 : ((kind == kKernelDirect || kind == kKernelSlice) ? grid * direct_per_sm : grid);
  L.grid_total = mg + wg;
  const auto tiled = [&](cudaStream_t s) {
    if (kind == kKernelSlice) {
      if (direct_per_sm == 3)
        bellman_slice_kernel<kSliceWarps, 3><<<mg, 32 * kSliceWarps, 0, s>>>(L);
      else
        bellman_slice_kernel<kSliceWarps, 4><<<mg, 32 * kSliceWarps, 0, s>>>(L);
    } else if (kind == kKernelDirect) {
      if (direct_per_sm == 3)
        bellman_direct_kernel<kDirectWarps, 3><<<mg, 32 * kDirectWarps, 0, s>>>(L);
      else
        bellman_direct_kernel<kDirectWarps, 4><<<mg, 32 * kDirectWarps, 0, s>>>(L);
    } else if (short_cols) {
      bellman_step_kernel<kConsumersShort>
          <<<mg, 32 * (kConsumersShort + 1), sizeof(Smem<kConsumersShort>), s>>>(L);
    } else {
      bellman_step_kernel<kConsumersLong><<<mg, 32 * (kConsumersLong + 1), sizeof(Smem<kConsumersLong>), s>>>(L);
    }
    return cudaGetLastError();
  };
  cudaError_t e = cudaSuccess;
  if (wg > 0 && side && side->stream && L.n_tiles > 0) {
    // fork / join: the tiled kernel is issued first so that its CTAs hold the
    // SMs; wide CTAs run in the room left beside them
    e = cudaEventRecord(side->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side->stream, side->fork, 0);
    if (e != cudaSuccess) return e;
    if ((e = tiled(st)) != cudaSuccess) return e;
    bellman_wide_kernel<<<wg, kWideThreads, 0, side->stream>>>(L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaEventRecord(side->join, side->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, side->join, 0);
    return e;
  }
  if (wg > 0) {
    bellman_wide_kernel<<<wg, kWideThreads, 0, st>>>(L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return tiled(st);
}

}  // namespace imdp
