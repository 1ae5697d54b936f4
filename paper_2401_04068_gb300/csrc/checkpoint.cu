// Checkpoint and resume of one problem of a session. Value iteration (Eq. 2)
// carries nothing from one iteration to the next but the iterate V_k and the
// count k, so those two are the whole state: a checkpoint copies them out, a
// restore writes them into a session of the same model and specification and
// resets the problem's iteration state so that the next launch computes
// iteration k + 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

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

imdp_status check_index(imdp_session* s, int32_t index) {
  if (!s || !s->s) {
    set_error("NULL session");
    return IMDP_EINVAL;
  }
  if (index < 0 || index >= s->s->count) {
    set_error("problem index out of range");
    return IMDP_EINVAL;
  }
  return IMDP_OK;
}

}  // namespace

extern "C" {

IMDP_API imdp_status imdp_session_checkpoint(imdp_session* s, int32_t index, uint64_t* raw_V, int32_t* k,
                                             void* stream) {
  set_error("");
  imdp_status r = check_index(s, index);
  if (r != IMDP_OK) return r;
  if (!raw_V || !k) {
    set_error("NULL raw_V or k");
    return IMDP_EINVAL;
  }
  Session* S = s->s;
  DeviceScope g(S->device);
  const cudaStream_t st = (cudaStream_t)stream;
  std::vector<IterState> its;
  r = S->read_states(its, st);  // synchronizes the stream, reports a failed bounded wait
  if (r != IMDP_OK) return r;
  const IterState& it = its[index];
  const int32_t kk = it.done ? it.k_final : it.iter;
  const Problem& P = S->probs_h[index];
  cudaError_t e = cudaMemcpyAsync(raw_V, P.V[kk & 1], sizeof(uint64_t) * (size_t)P.n_states, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "checkpoint");
  *k = kk;
  return IMDP_OK;
}

IMDP_API imdp_status imdp_session_restore(imdp_session* s, int32_t index, const uint64_t* raw_V, int32_t k,
                                          void* stream) {
  set_error("");
  imdp_status r = check_index(s, index);
  if (r != IMDP_OK) return r;
  Session* S = s->s;
  const Problem& P = S->probs_h[index];
  if (!raw_V) {
    set_error("NULL raw_V");
    return IMDP_EINVAL;
  }
  if (k < 0 || k > P.horizon) {
    set_error("k must lie in [0, horizon] (the iteration cap for an infinite horizon)");
    return IMDP_EINVAL;
  }
  DeviceScope g(S->device);
  const cudaStream_t st = (cudaStream_t)stream;
  IterState it;
  std::memset(&it, 0, sizeof(it));
  it.iter = k;
  if (k == P.horizon) {  // nothing left to compute
    it.done = 1;
    it.k_final = k;
    it.noconv = P.infinite ? 1 : 0;
  }
  cudaError_t e = cudaMemcpyAsync(P.V[k & 1], raw_V, sizeof(uint64_t) * (size_t)P.n_states, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->its + index, &it, sizeof(it), cudaMemcpyHostToDevice, st);
  // the saved hints belong to the interrupted run: start this problem without any
  if (e == cudaSuccess)
    e = cudaMemsetAsync(P.hint, 0xff, sizeof(int32_t) * padded_i32((size_t)S->models[index]->n_cols), st);
  // the problem may run again: the next launch visits every tile (the running
  // prefix is recomputed when it ends)
  if (e == cudaSuccess) e = cudaMemsetAsync(&S->ctl->tile_limit, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `it` lives on this stack frame
  if (e != cudaSuccess) return cuda_status(e, "restore");
  // The session's launch count since its reset bounds how many more launches
  // imdp_session_run issues; a problem restored to iteration k needs up to
  // horizon - k more, whatever the session ran before (extra launches skip
  // finished problems on the device).
  S->launched_since_reset = std::min<int64_t>(S->launched_since_reset, k);
  return IMDP_OK;
}

}  // extern "C"
