// Value iteration without any device allocation on the query path.
//
// Who needs this: callers that load their models once at start-up and afterwards
// may not allocate device memory, e.g. a controller that re-plans every cycle
// under a fixed memory budget, or code running inside a process whose device
// memory is handed out by another framework's allocator. imdp_value_iteration
// allocates its value buffers and iteration state per call; this entry point
// keeps them in one file-scope device array instead.
//
// The array below is the only scratch. Every GPU that loads this library holds
// it (kNoAllocBytes, about 3.7 MB) until the process exits. Its host-side name is
// only a stand-in: host code obtains the device address with
// cudaGetSymbolAddress, once per device, on the first call made with that
// device current (so that first call should happen before any stream capture).
// All calls share the array and it keeps the previous call's contents, so each
// call re-initialises what it reads; two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "imdp_internal.h"

namespace imdp {

namespace {

constexpr int32_t kNoAllocMaxStates = 131072;
// Layout of the scratch array (offsets in bytes, each 256-aligned).
constexpr size_t kOffProblem = 0;
constexpr size_t kOffIter = 256;
constexpr size_t kOffCtl = 512;
constexpr size_t kOffBase = 768;
constexpr size_t kOffFlag = 1024;
constexpr size_t kOffMask = 1280;
constexpr size_t kOffIdx = kOffMask + kNoAllocMaxStates;                 // reach + avoid indices
constexpr size_t kOffV = kOffIdx + sizeof(int32_t) * kNoAllocMaxStates;  // 2 x n values
// Per-column threshold hints (the warm start of the next iteration) for models
// of up to kNoAllocMaxHintCols columns, padded as a session pads them.
constexpr int32_t kNoAllocMaxHintCols = 262144;
constexpr size_t kOffHint = kOffV + 2 * sizeof(uint64_t) * kNoAllocMaxStates;
constexpr size_t kNoAllocBytes = kOffHint + sizeof(int32_t) * (((size_t)kNoAllocMaxHintCols + 3) / 4 * 4 + 4);
static_assert(sizeof(Problem) <= 256 && sizeof(IterState) <= 256 && sizeof(StepControl) <= 256, "layout");
static_assert(kOffIdx % 256 == 0 && kOffV % 256 == 0 && kOffHint % 256 == 0, "alignment");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (set up on first use).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return cudaSuccess;
}

// Mark reach states 1 and avoid states 2; flag a state that is in both sets.
__global__ void noalloc_mask_kernel(int32_t n_reach, int32_t n_avoid, const int32_t* __restrict__ idx,
                                    uint8_t* __restrict__ mask, int32_t* __restrict__ flag) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_reach; i += gridDim.x * blockDim.x)
    mask[idx[i]] = 1;
  __syncthreads();  // single block: reach marks are visible before avoid marks
  for (int32_t i = threadIdx.x; i < n_avoid; i += blockDim.x) {
    const int32_t s = idx[n_reach + i];
    if (mask[s] == 1) atomicExch(flag, 1);
    else mask[s] = 2;
  }
}

__global__ void noalloc_init_kernel(int32_t n, const uint8_t* __restrict__ mask, uint64_t* __restrict__ V0) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    V0[i] = mask[i] == 1 ? kOne : 0ull;
}

// V_k -> binary64, where k is read from the iteration state on the device.
__global__ void noalloc_export_kernel(int32_t n, const IterState* __restrict__ it, const uint64_t* __restrict__ V,
                                      double* __restrict__ out) {
  const int32_t k = it->done ? it->k_final : it->iter;
  const uint64_t* Vk = V + (size_t)(k & 1) * n;
  const double scale = 1.0 / 9223372036854775808.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (double)Vk[i] * scale;
}

}  // namespace

}  // namespace imdp

using namespace imdp;

extern "C" IMDP_API imdp_status imdp_value_iteration_noalloc(imdp_model* m, const imdp_spec* spec, double* V_out,
                                                             int32_t* k_out, void* stream) {
  set_error("");
  if (!m || !spec || !V_out) { set_error("NULL model, spec or V_out"); return IMDP_EINVAL; }
  const DevModel* dm = m->dev;
  if (dm->n_states > kNoAllocMaxStates) {
    set_error("imdp_value_iteration_noalloc: model has more than 131072 states (the fixed scratch limit)");
    return IMDP_EINVAL;
  }
  if (is_slice(dm)) { set_error("slices of a state-sharded model run in sessions only"); return IMDP_EINVAL; }
  imdp_status s = check_spec(dm, spec);
  if (s != IMDP_OK) return s;
  if (spec->property == IMDP_REWARD) {
    set_error("imdp_value_iteration_noalloc: reward properties are not offered here");
    return IMDP_EINVAL;
  }
  const int32_t n_avoid = spec->property == IMDP_REACH_AVOID ? spec->n_avoid : 0;
  if ((int64_t)spec->n_reach + n_avoid > kNoAllocMaxStates) {
    set_error("imdp_value_iteration_noalloc: more than 131072 reach + avoid indices");
    return IMDP_EINVAL;
  }
  if (!is_device_pointer(V_out)) { set_error("imdp_value_iteration_noalloc: V_out must be device memory"); return IMDP_EINVAL; }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != m->device) { set_error("imdp_value_iteration_noalloc: make the model's device current"); return IMDP_EINVAL; }

  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress");
  Problem* d_prob = (Problem*)(base + kOffProblem);
  IterState* d_it = (IterState*)(base + kOffIter);
  StepControl* d_ctl = (StepControl*)(base + kOffCtl);
  int32_t* d_base = (int32_t*)(base + kOffBase);
  int32_t* d_flag = (int32_t*)(base + kOffFlag);
  uint8_t* d_mask = base + kOffMask;
  int32_t* d_idx = (int32_t*)(base + kOffIdx);
  uint64_t* d_V = (uint64_t*)(base + kOffV);
  int32_t* d_hint = (int32_t*)(base + kOffHint);
  const int32_t n = dm->n_states;

  Problem P;
  std::memset(&P, 0, sizeof(P));
  P.stateptr = dm->stateptr;
  P.colptr = dm->colptr;
  P.rowval = dm->rowval;
  P.lg = dm->lg;
  P.rem = dm->rem;
  P.lg32 = dm->lg32;
  P.shift = dm->shift;
  P.xoff = dm->xoff;
  P.lgx = dm->lgx;
  P.fixed = d_mask;
  // hints when the model's columns fit the fixed region (else every column
  // takes the full threshold search, with the same result)
  const bool hints = dm->n_cols <= kNoAllocMaxHintCols;
  P.hint = hints ? d_hint : nullptr;
  P.V[0] = d_V;
  P.V[1] = d_V + n;
  P.n_states = n;
  P.pessimistic = spec->pessimistic ? 1 : 0;
  P.maximize = spec->maximize ? 1 : 0;
  P.property = spec->property;
  P.infinite = spec->infinite_time ? 1 : 0;
  P.horizon = spec->infinite_time ? (spec->horizon > 0 ? spec->horizon : 1000000) : spec->horizon;
  if (P.infinite) {
    const double x = spec->eps * 9223372036854775808.0;
    uint64_t f = spec->eps >= 1.0 ? kOne + 1 : (uint64_t)x;
    if (spec->eps < 1.0 && (double)f < x) f += 1;
    P.eps_fix = f;
  }
  const int32_t base_h[2] = {0, n};

  // Re-initialise everything this call reads from the shared array.
  e = cudaMemsetAsync(base, 0, kOffMask, st);  // problem, iteration state, ticket, flag
  if (e == cudaSuccess) e = cudaMemsetAsync(d_mask, 0, n, st);
  if (e == cudaSuccess && hints)  // -1: no hint yet (the previous call's hints belong to another query)
    e = cudaMemsetAsync(d_hint, 0xff, sizeof(int32_t) * padded_i32((size_t)dm->n_cols), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_prob, &P, sizeof(P), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_base, base_h, sizeof(base_h), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && spec->n_reach > 0)
    e = cudaMemcpyAsync(d_idx, spec->reach, sizeof(int32_t) * spec->n_reach, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_avoid > 0)
    e = cudaMemcpyAsync(d_idx + spec->n_reach, spec->avoid, sizeof(int32_t) * n_avoid, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "noalloc setup");
  noalloc_mask_kernel<<<1, 256, 0, st>>>(spec->n_reach, n_avoid, d_idx, d_mask, d_flag);
  int32_t flag = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(flag), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "noalloc mask");
  if (flag) { set_error("a state is in both the reach and the avoid set"); return IMDP_EINVAL; }
  const int g = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  noalloc_init_kernel<<<g, 256, 0, st>>>(n, d_mask, d_V);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "noalloc init");

  StepLaunch L{};
  L.probs = d_prob;
  L.its = d_it;
  L.state_base = d_base;
  L.ctl = d_ctl;
  L.count = 1;
  L.total_states = n;
  L.any_infinite = P.infinite;
  L.tiles = dm->tiles;  // the model's own tile plan (problem index 0)
  L.n_tiles = dm->n_tiles;
  L.tile_cols = dm->tile_cols;
  L.wide = dm->wide;
  L.n_wide = dm->n_wide;
  const int grid = bellman_grid();
  IterState hs;
  std::memset(&hs, 0, sizeof(hs));
  if (!P.infinite) {
    for (int32_t k = 0; k < P.horizon; ++k)
      if ((e = launch_bellman_step(L, grid, st)) != cudaSuccess) return cuda_status(e, "bellman step");
  } else {
    int32_t launched = 0;
    while (launched < P.horizon) {
      const int32_t chunk = P.horizon - launched < 32 ? P.horizon - launched : 32;
      for (int32_t k = 0; k < chunk; ++k)
        if ((e = launch_bellman_step(L, grid, st)) != cudaSuccess) return cuda_status(e, "bellman step");
      launched += chunk;
      e = cudaMemcpyAsync(&hs, d_it, sizeof(hs), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_status(e, "convergence check");
      if (hs.done) break;
    }
  }
  noalloc_export_kernel<<<g, 256, 0, st>>>(n, d_it, d_V, V_out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, d_it, sizeof(hs), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "noalloc export");
  StepControl hc;
  std::memset(&hc, 0, sizeof(hc));
  e = cudaMemcpyAsync(&hc, d_ctl, sizeof(hc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "noalloc status");
  if (hc.error) {
    set_error("a bounded wait inside the Bellman kernel gave up");
    return IMDP_ETIMEOUT;
  }
  if (k_out) *k_out = hs.done ? hs.k_final : hs.iter;
  if (hs.noconv) {
    set_error("infinite horizon did not converge within the iteration cap");
    return IMDP_ENOCONV;
  }
  return IMDP_OK;
}
