// Internal declarations shared by the library's translation units.
//
// Number format. Every probability bound and every value-function entry of a
// reachability problem lies in [0, 1] (Sec. 2). The kernels keep them as
// unsigned 64-bit fixed point with 63 fractional bits ("Q1.63": x -> round(x * 2^63),
// 1.0 = 2^63). Bellman arithmetic is then integer: products use the high half of a
// 64x64-bit multiply, sums are exact and associative, so results do not depend on
// the reduction order or on the thread mapping. On GB300 the FP64 pipe issues ~60x
// fewer operations per cycle than the 32-bit integer/FP32 pipes, which is why the
// hot loop avoids binary64 altogether.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <atomic>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/imdp.h"

namespace imdp {

constexpr uint64_t kOne = 1ull << 63;  // 1.0 in Q1.63

// A value in [0, 1] (Q1.63) rounded to nearest at 32 bits (low word zero):
// the values of a problem on 32-bit storage.
__host__ __device__ __forceinline__ uint64_t round_value32(uint64_t v) {
  return v >= kOne - (1ull << 31) ? kOne : (v + (1ull << 31)) & ~0xffffffffull;
}

// Property kinds inside the kernels.
enum : int32_t { kPropReach = 0, kPropReachAvoid = 1, kPropReward = 2 };

// A tile is a run of consecutive states of one problem whose entries are
// streamed into shared memory by one bulk copy per array (state-aligned, so a
// CTA finishes the opt over actions on its own). A state whose entries do not
// fit one stage, or that has a column of kWideCol entries or more, is "wide": a
// whole CTA works on it (bellman_wide_kernel) and it belongs to no tile.
constexpr int kTileEntries = 3072;  // entries per tile (rowval 12 KB + bounds 48 KB + keys 24 KB)
constexpr int kTileCols = 256;      // columns per tile
constexpr int kTileStates = 256;    // states per tile
constexpr int kWideCol = 1280;      // columns this long make their state wide
struct Tile {
  int32_t p;      // problem
  int32_t s0, s1; // states [s0, s1) of that problem
  int32_t c0, c1; // columns [c0, c1)
  int32_t e0, e1; // entries [e0, e1)
  int32_t x0, x1; // 32-bit storage: the tile's correction entries, [x0, x1) of the model's lgx
};

// Slice layout of a model (the slice kernel; a second copy of the CSC arrays of
// Sec. 3.1 arranged for one lane per column). The owned states are cut into
// windows of whole states of at most kSliceWindowCols columns; inside a window
// the columns are ordered by length (longest first) and dealt to slices of 32
// slots. Entry t of the column in slot l of a slice sits at off + 32 t + l, so a
// warp reading entry t of its 32 columns reads one contiguous run; entries keep
// their order within the column (a threshold hint names the same entry in both
// layouts). A slice runs to its longest column (the lanes of shorter ones idle
// without loads); ordering by length keeps that padding to a few percent.
constexpr int kSliceWindowCols = 256;
struct SliceMeta {
  long long off;  // first entry of the slice in rows / lg
  int32_t len;    // entries of its longest column (trips of the slice's loop)
  int32_t pad;
};
struct SliceLayout {
  int32_t n_windows = 0;
  int32_t n_slices = 0;
  int64_t entries = 0;              // entries including padding (32 per trip of every slice)
  std::vector<int32_t> h_win_s0;    // n_windows + 1: state boundaries of the windows
  std::vector<int32_t> h_win_sl0;   // n_windows + 1: slice boundaries of the windows
  int2* slot = nullptr;             // 32 per slice: {column, entries in the slice arrays}; column -1: empty
                                    // slot; 32-bit correction columns hold 0 entries here (their exact
                                    // bounds are read from lgx)
  SliceMeta* meta = nullptr;        // per slice
  int32_t* rows = nullptr;          // destinations, padding 0
  void* lg = nullptr;               // ulonglong2 (64-bit) or uint2 (32-bit) bound pairs, padding {0, 0}
  void* block = nullptr;            // the one allocation holding the arrays above
  size_t bytes = 0;
};

// Device-resident model (the "IntervalMDP.cu(problem)" transfer of Sec. 3.2,
// CSC layout of Sec. 3.1 / Appendix A).
struct DevModel {
  int32_t n_states = 0;
  int32_t n_cols = 0;
  int64_t nnz = 0;
  int32_t max_col = 0;     // largest column (entries)
  int32_t own0 = 0;        // states [own0, own1) have columns and are updated; the rest
  int32_t own1 = 0;        // (a slice of a state-sharded model) only hold exchanged values
  int32_t dtype = IMDP_F64;
  int32_t* stateptr = nullptr;  // n_states + 1
  int32_t* colptr = nullptr;    // n_cols + 1
  int32_t* rowval = nullptr;    // nnz
  ulonglong2* lg = nullptr;     // IMDP_F64: nnz x {lower, gap = upper - lower} in Q1.63
  uint2* lg32 = nullptr;        // IMDP_F32: nnz x {lower, gap} as 32-bit mantissas, value = m * 2^-(31 + shift_j)
  int32_t* shift = nullptr;     // IMDP_F32: per-column shift_j (padded like colptr)
  int32_t* xoff = nullptr;      // IMDP_F32: per column, offset of its exact bounds in lgx (-1: 32-bit column);
                                // nullptr when every column is 32-bit
  ulonglong2* lgx = nullptr;    // IMDP_F32: exact {lower, gap} of the correction columns (compact)
  int32_t n_exact = 0;          // IMDP_F32: correction columns
  int64_t exact_entries = 0;    //           and their transitions
  double f32_budget = 0.0;      // IMDP_F32: the per-iteration budget the columns were sorted by
  double err_bound = 0.0;       // IMDP_F32: guaranteed per-iteration error bound (see imdp_model_error_bound)
  uint64_t* rem = nullptr;      // n_cols: 1 - sum(lower) in Q1.63 (clamped at 0)
  size_t bytes = 0;
  std::vector<int32_t> h_stateptr;  // host copies of the structure (tile planning)
  std::vector<int32_t> h_colptr;
  std::vector<int32_t> h_xoff;      // IMDP_F32 with correction columns: host copy of xoff
  std::vector<Tile> h_tiles;        // tile plan of this model (problem index 0)
  Tile* tiles = nullptr;            // device copy of h_tiles
  int32_t n_tiles = 0;
  int64_t tile_cols = 0;            // columns in all of h_tiles
  std::vector<int32_t> h_wide;      // wide states (in no tile)
  int2* wide = nullptr;             // device copy as (problem 0, state)
  int32_t n_wide = 0;
  SliceLayout* slices = nullptr;    // built on first use by a session that runs the slice kernel
  std::mutex slices_mu;
};



// One problem of a batch as the step kernel sees it (read-only during a launch).
struct alignas(16) Problem {
  const int32_t* stateptr;
  const int32_t* colptr;
  const int32_t* rowval;
  const ulonglong2* lg;
  const uint64_t* rem;
  const uint2* lg32;      // 32-bit storage (nullptr for 64-bit models)
  const int32_t* shift;   // per-column shift of the 32-bit storage
  const int32_t* xoff;    // 32-bit storage: per column, offset of its exact bounds in lgx (-1: 32-bit); nullable
  const ulonglong2* lgx;  // 32-bit storage: exact bounds of the correction columns
  const uint8_t* fixed;   // n_states: 0 free, 1 held at 1 (reach target), 2 held at 0 (avoid)
  uint64_t* V[2];         // ping-pong value buffers; iteration k writes V[k & 1]
  int32_t* policy;        // nullable; see policy_mode
  const int64_t* rbias;   // reward: per-state term c_s of W_k = c_s + gamma T(W_{k-1}), signed Q2.62
  int32_t* hint;          // per column: entry that held the O-maximization threshold last iteration (-1: none)
  // slice kernel only (nullptr otherwise): the model's slice layout and the
  // per-column q of the running iteration
  const int2* sl_slot;
  const SliceMeta* sl_meta;
  const int32_t* sl_rows;
  const void* sl_lg;
  uint64_t* qcol;
  int32_t n_states;
  int32_t pessimistic;
  int32_t maximize;
  int32_t property;
  int32_t horizon;        // K (finite) or iteration cap (infinite)
  int32_t infinite;
  int32_t policy_mode;    // 0 none, 1 time-dependent K x n, 2 stationary n
  int32_t external_stop;  // infinite horizon on a slice: the caller tests the residual of all slices
  uint64_t eps_fix;       // infinite horizon: stop when max |dV| < eps_fix
  uint64_t gamma_fix;     // reward: discount in Q1.63
};

// Mutable per-problem iteration state (device memory).
struct IterState {
  int32_t iter;     // completed iterations
  int32_t done;     // 1 once the problem has finished
  int32_t k_final;  // iterations performed when done
  int32_t noconv;   // infinite horizon stopped at the cap
  unsigned long long resmax;  // max |V_k - V_{k-1}| of the running iteration
};

struct StepControl {
  unsigned int finished;   // CTAs (of both step kernels) finished in the running launch
  unsigned int error;      // nonzero: a bounded wait inside the kernel gave up
  unsigned int wide_next;  // next wide state to take in the running launch
  unsigned int tile_next;  // next tile to take in the running launch (direct kernel)
  int32_t tile_limit;      // 0: every tile; t + 1: only tiles [0, t) belong to running problems
};

// Launch configuration of the Bellman step (per session; chosen by rule or by
// the autotuner). Zero fields mean "by rule".
enum : int32_t { kKernelRule = 0, kKernelRing = 1, kKernelDirect = 2, kKernelTiny = 3, kKernelSlice = 4 };
// A session of one problem this small runs all its iterations in one launch of
// one CTA, with the model and values in shared memory (bellman_tiny_kernel).
constexpr int32_t kTinyMaxStates = 1024, kTinyMaxCols = 1024, kTinyMaxEntries = 4096;
// The rule for a session's shape (the choices the autotuner makes on GB300 for
// the benchmark shapes): problems whose columns hold kRuleLongColumn entries or
// more on average run the direct kernel (3 CTAs per SM, kRuleDirectTile-entry
// tiles); shorter columns run the slice kernel (3 CTAs per SM on 64-bit
// storage, 4 on 32-bit) when the device has room for its second copy of the
// models, else the ring kernel.
constexpr int64_t kRuleLongColumn = 256;
constexpr int32_t kRuleDirectTile = 1024;
constexpr int kDirectWarps = 8;  // warps per CTA of the direct kernel
constexpr int kSliceWarps = 8;   // warps per CTA of the slice kernel
struct LaunchConfig {
  int32_t kernel = kKernelRule;  // ring: TMA-fed shared-memory tiles; direct: warps stream tiles from global
                                 // memory; slice: one lane per column over the slice layout
  int32_t cta_warps = 0;         // ring: 16 or 24 warps per CTA; direct and slice: 8
  int32_t ctas_per_sm = 0;       // direct and slice: 3 or 4 CTAs per SM
  int32_t tile_entries = 0;      // tile plan: entries per tile (<= kTileEntries)
  int32_t wide_col = 0;          // columns this long make their state wide
};

// Second stream on which the wide-state kernel runs beside the tiled one.
struct SideStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    return e;
  }
  void destroy() {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (stream) cudaStreamDestroy(stream);
    stream = nullptr;
    fork = join = nullptr;
  }
};

struct StepLaunch {
  const Problem* probs;
  IterState* its;
  const int32_t* state_base;  // count + 1 prefix of n_states
  StepControl* ctl;
  int32_t count;
  int32_t total_states;
  int32_t any_infinite;
  const Tile* tiles;
  int32_t n_tiles;
  int32_t n_wide;
  const int2* wide;  // (problem, state) of every wide state
  int64_t tile_cols;   // columns in all tiles (the launcher picks the CTA shape from it)
  // Tiles laid out by problem rank (longest horizon first; nullable): after a
  // launch, the tiles of running problems are a prefix, [0, rank_tile_end[r])
  // with r the largest rank still running.
  const int32_t* rank_of;        // count: rank of each problem
  const int32_t* rank_tile_end;  // count: tiles of ranks 0..r
  // the kernel "by rule" stands for when the single-CTA kernel does not apply
  // (0: the ring kernel; a session sets it from its problems' shape, see
  // kRuleLongColumn) and whether every problem has 32-bit storage
  int32_t shape_rule;
  int32_t shape_f32;
  int32_t tiny_ok;     // one small problem (sizes below): the single-CTA kernel may run it
  int32_t tiny_states, tiny_cols, tiny_entries;
  // slice kernel: the work items (tile = window, slice of the model's layout) in
  // tile order, the items of tiles [0, t] (per tile), and per tile the count of
  // its slices finished in the running launch (zero between launches)
  const int2* items;
  const int32_t* tile_item_end;
  unsigned int* win_cnt;
  int32_t n_items;
  int32_t grid_total;  // CTAs of both step kernels in this launch (set by the launcher)
  int32_t stall;       // test hook: the producer issues nothing, so every wait runs out
};

// NVTX range for the host-side phases (model upload, session steps, server
// chunks); shows up in Nsight timelines, free when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
};

// bellman.cu
// Test hook (imdp_debug_stall_producer): launches made while set leave the
// consumers' waits unsatisfied, to exercise the bounded-wait error path.
extern std::atomic<int> g_stall_producer;
// One Bellman iteration: the wide-state kernel (on `side`, beside the tiled one,
// when given) and the tiled kernel; the last CTA of the two advances the
// iteration state.
// `cfg` (nullable) picks the tiled kernel and its shape; the tile list in `L`
// must follow the same configuration's tile plan.
cudaError_t launch_bellman_step(const StepLaunch& L, int grid, cudaStream_t st, const SideStream* side = nullptr,
                                const LaunchConfig* cfg = nullptr);
// n_iters Bellman iterations of a session's single small problem (L.tiny_ok) in
// one launch of one CTA.
cudaError_t launch_bellman_tiny(const StepLaunch& L, int32_t n_iters, bool f32, cudaStream_t st);
// CTAs of the persistent tiled kernel: one per SM.
int bellman_grid();
// The configuration a launch of `L` with `cfg` (nullable) actually uses: kernel,
// warps per CTA and CTAs per SM resolved by the rule where `cfg` leaves them open.
LaunchConfig resolve_launch(const StepLaunch& L, const LaunchConfig* cfg);
// Tile plan for one problem's model (host): tiles appended to `out`, wide
// states (no tile) appended to `wide`. Tiles hold at most `tile_entries`
// entries (<= kTileEntries; 0: kTileEntries); a state with a column of
// `wide_col` entries or more (0: kWideCol) is wide. States with a nonzero
// `fixed` entry (nullable; n_states of the problem) belong to neither.
void plan_tiles(const DevModel* m, int32_t problem, std::vector<Tile>& out, std::vector<int32_t>& wide,
                int32_t tile_entries = 0, int32_t wide_col = 0, const uint8_t* fixed = nullptr);

// slices.cu
// The model's slice layout, built on `st` on first use (thread-safe; kept until
// the model is destroyed).
imdp_status model_slice_layout(DevModel* m, cudaStream_t st, const SliceLayout** out);
void slice_layout_free(SliceLayout* l);

// model.cu
// Per-iteration error budget of 32-bit storage when the caller names none:
// 1e-6 over the paper's benchmark horizon of K = 200 iterations.
constexpr double kDefaultF32Budget = 5e-9;
imdp_status model_create_csc(int32_t n_states, int32_t n_cols, int64_t nnz, const int32_t* stateptr,
                             const int32_t* colptr, const int32_t* rowval, const double* lower,
                             const double* upper, imdp_dtype dtype, cudaStream_t st, DevModel** out,
                             int32_t own0 = 0, int32_t own1 = -1, double budget = kDefaultF32Budget);
void model_destroy(DevModel* m);
inline bool is_slice(const DevModel* m) { return m->own0 != 0 || m->own1 != m->n_states; }

// session.cu: resident device state of value iteration for a batch of problems.
// Padding of the per-state / per-column arrays so that 16-byte-aligned bulk-copy
// windows around any index range stay inside their allocations.
inline size_t padded_i32(size_t n) { return ((n + 3) & ~size_t(3)) + 4; }
inline size_t padded_u64(size_t n) { return ((n + 1) & ~size_t(1)) + 2; }
inline size_t padded_u8(size_t n) { return ((n + 15) & ~size_t(15)) + 16; }

struct Session {
  int device = 0;
  int count = 0;
  int64_t total = 0;
  std::vector<DevModel*> models;
  std::vector<Problem> probs_h;
  std::vector<int32_t> base_h;
  std::vector<int64_t> policy_cells;
  std::vector<int32_t> order;             // problems by rank: longest horizon (infinite) first
  std::vector<uint8_t> fixed_h;           // total states: 1 reach, 2 avoid (planned out of the tiles)
  int32_t* rank_of = nullptr;             // device copies for the running-prefix bound
  int32_t* rank_tile_end = nullptr;
  std::vector<double> v_offset, v_scale;  // V = offset + scale * W (reward: affine map; reach: 0, 1)
  std::vector<uint64_t*> w0;              // reward: device copy of W_0 for resets (nullptr otherwise)
  int32_t* hints = nullptr;               // sum of n_cols: threshold hints of every problem
  int64_t total_cols = 0;
  int32_t max_horizon = 0;
  bool any_infinite = false;
  uint8_t* fixed = nullptr;
  uint64_t* V = nullptr;
  int32_t* base = nullptr;
  Problem* probs = nullptr;
  IterState* its = nullptr;
  StepControl* ctl = nullptr;
  Tile* tiles = nullptr;
  int32_t n_tiles = 0;
  int2* wide = nullptr;
  int32_t n_wide = 0;
  int64_t wide_entries = 0;  // transitions of the wide states (host count)
  // slice kernel: per-column q of every problem (offsets as `hints`), the work
  // items and window counters of the installed plan
  uint64_t* qbuf = nullptr;
  int2* items = nullptr;
  int32_t* tile_item_end = nullptr;
  unsigned int* win_cnt = nullptr;
  // Point every problem at its model's slice layout (built if needed) and
  // allocate the per-column q; idempotent.
  imdp_status prepare_slices(cudaStream_t st);
  SideStream side;  // created when the session has both tiles and wide states
  LaunchConfig cfg;  // launch configuration (rule, set_launch or the autotuner)
  StepLaunch L{};
  int grid = 1;
  cudaGraphExec_t graph = nullptr;
  bool graph_stalled = false;  // captured while the failure-detection test hook was on
  int64_t launches = 0;
  int64_t launched_since_reset = 0;
  std::vector<void*> allocs;

  ~Session();
  template <class T> T* alloc(size_t n);
  static imdp_status create(const std::vector<DevModel*>& ms, const std::vector<const imdp_spec*>& specs,
                            const int32_t* want_policy, cudaStream_t st, Session** out);
  imdp_status reset(cudaStream_t st);
  // Upload a tile plan (tiles and wide states of every problem) and point the
  // launch at it.
  // `slice`: the plan is the slice kernel's (windows), which also takes work items.
  imdp_status install_plan(const std::vector<Tile>& tiles, const std::vector<int2>& wide, cudaStream_t st,
                           bool slice = false);
  // Tile plan of every problem (rank order) under the plan limits of `c`,
  // leaving out the states the properties fix.
  void build_plan(const LaunchConfig& c, std::vector<Tile>& tiles, std::vector<int2>& wide) const;
  // Use launch configuration `c` from the next step on (re-plans the tiles
  // when its plan limits differ; drops the captured graph).
  imdp_status set_launch(const LaunchConfig& c, cudaStream_t st);
  imdp_status step(int32_t n, cudaStream_t st);
  imdp_status run(int32_t check_every, cudaStream_t st);
  imdp_status read_states(std::vector<IterState>& out, cudaStream_t st);
  imdp_status read(int32_t p, double* V_out, int32_t* k_out, double* res_out, int32_t* pol_out, cudaStream_t st);
};
imdp_status check_spec(const DevModel* m, const imdp_spec* sp);
// Affine map V = lo + D W of a reward problem (rewards r, discount g, horizon K).
void reward_map(const double* r, int32_t n, double g, int32_t K, bool infinite, double* lo, double* D);

// api.cu
void set_error(const std::string& msg);
bool have_device();
bool is_device_pointer(const void* p);
imdp_status cuda_status(cudaError_t e, const char* where);

}  // namespace imdp

struct imdp_model {
  imdp::DevModel* dev;
  int device;
};

struct imdp_session {
  imdp::Session* s;
};
