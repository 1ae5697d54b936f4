// State-sharded value iteration: one model's states split into contiguous ranges
// (one per GPU), each range iterated by its own session on a slice of the model,
// and the iterates exchanged between the slices after every Bellman step.
//
// Eq. 2 updates every state from V_{k-1} of all states, and the states are
// independent of one another within an iteration (Sec. 4), so a slice that owns
// states [s0, s1) computes V_k[s0, s1) exactly as the whole model would, as long
// as its copy of V_{k-1} is complete. The caller moves the slices' values
// between steps (an all-gather across GPUs); these entry points give the owned
// ranges, build the slices and read / write the raw iterates.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "imdp_internal.h"

using namespace imdp;

namespace {

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

imdp_status values_window(imdp_session* s, int32_t index, int32_t k, int32_t s0, int32_t s1, uint64_t** base) {
  if (!s || !s->s) { set_error("NULL session"); return IMDP_EINVAL; }
  Session* S = s->s;
  if (index < 0 || index >= S->count) { set_error("problem index out of range"); return IMDP_EINVAL; }
  const int32_t n = S->base_h[index + 1] - S->base_h[index];
  if (k < 0 || s0 < 0 || s1 > n || s0 > s1) { set_error("iteration or state range out of range"); return IMDP_EINVAL; }
  *base = S->V + (size_t)(k & 1) * (size_t)S->total + S->base_h[index] + s0;
  return IMDP_OK;
}

// max |V_k - V_{k-1}| over a range of raw iterates (one atomic per warp).
__global__ void range_residual_kernel(int32_t n, const uint64_t* __restrict__ a, const uint64_t* __restrict__ b,
                                      unsigned long long* __restrict__ out) {
  unsigned long long m = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t x = a[i], y = b[i];
    const unsigned long long d = x > y ? x - y : y - x;
    m = d > m ? d : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

}  // namespace

extern "C" {

IMDP_API imdp_status imdp_session_residual(imdp_session* s, int32_t index, int32_t k, int32_t s0, int32_t s1,
                                           uint64_t* dst, void* stream) {
  set_error("");
  uint64_t* cur = nullptr;
  imdp_status st = values_window(s, index, k, s0, s1, &cur);
  if (st != IMDP_OK) return st;
  if (k < 1) { set_error("the residual needs k >= 1"); return IMDP_EINVAL; }
  if (!dst || !is_device_pointer(dst)) { set_error("dst must be device memory"); return IMDP_EINVAL; }
  uint64_t* prev = nullptr;
  values_window(s, index, k - 1, s0, s1, &prev);
  DeviceScope g(s->s->device);
  const cudaStream_t st_ = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(dst, 0, sizeof(uint64_t), st_);
  const int32_t n = s1 - s0;
  if (e == cudaSuccess && n > 0) {
    range_residual_kernel<<<std::min((n + 255) / 256, 1024), 256, 0, st_>>>(n, cur, prev, (unsigned long long*)dst);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? IMDP_OK : cuda_status(e, "residual");
}

IMDP_API imdp_status imdp_session_stop_threshold(const imdp_session* s, int32_t index, uint64_t* eps_raw) {
  set_error("");
  if (!s || !s->s || !eps_raw) { set_error("NULL argument"); return IMDP_EINVAL; }
  if (index < 0 || index >= s->s->count) { set_error("problem index out of range"); return IMDP_EINVAL; }
  const Problem& P = s->s->probs_h[index];
  if (!P.infinite) { set_error("the problem has a finite horizon"); return IMDP_EINVAL; }
  *eps_raw = P.eps_fix;
  return IMDP_OK;
}


IMDP_API imdp_status imdp_partition_states(int32_t n_states, const int32_t* stateptr, const int32_t* colptr,
                                           int32_t n_parts, int32_t* bounds) {
  set_error("");
  if (!stateptr || !colptr || !bounds) { set_error("NULL argument"); return IMDP_EINVAL; }
  if (n_states < 1 || n_parts < 1 || n_parts > n_states) {
    set_error("need 1 <= n_parts <= n_states");
    return IMDP_EINVAL;
  }
  // work of state s in one iteration: the algorithmic bytes the step streams for
  // it (20 per transition, 12 per column, 20 per state)
  std::vector<double> pre((size_t)n_states + 1, 0.0);
  for (int32_t s = 0; s < n_states; ++s) {
    const int32_t c0 = stateptr[s], c1 = stateptr[s + 1];
    if (c1 < c0 || colptr[c1] < colptr[c0]) { set_error("stateptr / colptr must be nondecreasing"); return IMDP_EINVAL; }
    pre[s + 1] = pre[s] + 20.0 * (double)(colptr[c1] - colptr[c0]) + 12.0 * (double)(c1 - c0) + 20.0;
  }
  const double total = pre[n_states];
  bounds[0] = 0;
  for (int32_t i = 1; i < n_parts; ++i) {
    const double target = total * (double)i / (double)n_parts;
    int32_t b = (int32_t)(std::lower_bound(pre.begin(), pre.end(), target) - pre.begin());
    if (b > 0 && target - pre[b - 1] < pre[b] - target) --b;  // the nearer boundary
    // every part keeps at least one state
    b = std::max(b, bounds[i - 1] + 1);
    b = std::min(b, n_states - (n_parts - i));
    bounds[i] = b;
  }
  bounds[n_parts] = n_states;
  return IMDP_OK;
}

IMDP_API imdp_status imdp_create_csc_slice(int32_t n_states, int32_t s0, int32_t s1, int32_t n_cols, int64_t nnz,
                                           const int32_t* stateptr, const int32_t* colptr, const int32_t* rowval,
                                           const double* lower, const double* upper, imdp_dtype dtype, void* stream,
                                           imdp_model** out) {
  set_error("");
  if (!out) { set_error("out is NULL"); return IMDP_EINVAL; }
  *out = nullptr;
  if (!have_device()) { set_error("no CUDA device"); return IMDP_EDEVICE; }
  if (n_states < 1 || s0 < 0 || s1 > n_states || s0 >= s1 || !stateptr) {
    set_error("need 0 <= s0 < s1 <= n_states");
    return IMDP_EINVAL;
  }
  if (stateptr[0] != 0 || stateptr[s1 - s0] != n_cols) {
    set_error("slice stateptr must start at 0 and end at n_cols");
    return IMDP_EINVAL;
  }
  // whole-model stateptr: no columns before s0 or after s1
  std::vector<int32_t> sp((size_t)n_states + 1, 0);
  for (int32_t s = s0; s <= s1; ++s) sp[s] = stateptr[s - s0];
  for (int32_t s = s1 + 1; s <= n_states; ++s) sp[s] = n_cols;
  DevModel* m = nullptr;
  imdp_status st = model_create_csc(n_states, n_cols, nnz, sp.data(), colptr, rowval, lower, upper, dtype,
                                    (cudaStream_t)stream, &m, s0, s1);
  if (st != IMDP_OK) return st;
  imdp_model* h = new imdp_model();
  h->dev = m;
  cudaGetDevice(&h->device);
  *out = h;
  return IMDP_OK;
}

IMDP_API imdp_status imdp_session_values_get(imdp_session* s, int32_t index, int32_t k, int32_t s0, int32_t s1,
                                             uint64_t* dst, void* stream) {
  set_error("");
  uint64_t* base = nullptr;
  imdp_status st = values_window(s, index, k, s0, s1, &base);
  if (st != IMDP_OK) return st;
  if (s1 == s0) return IMDP_OK;
  if (!dst || !is_device_pointer(dst)) { set_error("dst must be device memory"); return IMDP_EINVAL; }
  DeviceScope g(s->s->device);
  const cudaError_t e = cudaMemcpyAsync(dst, base, sizeof(uint64_t) * (size_t)(s1 - s0), cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? IMDP_OK : cuda_status(e, "values get");
}

IMDP_API imdp_status imdp_session_values_put(imdp_session* s, int32_t index, int32_t k, int32_t s0, int32_t s1,
                                             const uint64_t* src, void* stream) {
  set_error("");
  uint64_t* base = nullptr;
  imdp_status st = values_window(s, index, k, s0, s1, &base);
  if (st != IMDP_OK) return st;
  if (s1 == s0) return IMDP_OK;
  if (!src || !is_device_pointer(src)) { set_error("src must be device memory"); return IMDP_EINVAL; }
  DeviceScope g(s->s->device);
  const cudaError_t e = cudaMemcpyAsync(base, src, sizeof(uint64_t) * (size_t)(s1 - s0), cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? IMDP_OK : cuda_status(e, "values put");
}

}  // extern "C"
