// C ABI (include/imdp.h): model creation, value_iteration / control_synthesis
// (Sec. 3.2) for one problem or a batch, status strings.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "imdp_internal.h"

namespace imdp {

namespace {
thread_local std::string g_last_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else if (prev == dev) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

bool have_device() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

void set_error(const std::string& msg) { g_last_error = msg; }

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

imdp_status cuda_status(cudaError_t e, const char* where) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  set_error(buf);
  if (e == cudaErrorMemoryAllocation) return IMDP_ENOMEM;
  return IMDP_EDEVICE;
}

}  // namespace imdp

using namespace imdp;

extern "C" {

const char* imdp_status_string(imdp_status s) {
  switch (s) {
    case IMDP_OK: return "ok";
    case IMDP_EINVAL: return "invalid argument";
    case IMDP_EINFEASIBLE: return "infeasible interval model";
    case IMDP_ENOMEM: return "out of memory";
    case IMDP_EDEVICE: return "CUDA device error";
    case IMDP_ETIMEOUT: return "timed out";
    case IMDP_EBUSY: return "busy";
    case IMDP_ENOCONV: return "not converged";
    case IMDP_ENOTFOUND: return "not found";
    case IMDP_EPENDING: return "pending";
    case IMDP_EIO: return "file input/output error";
  }
  return "unknown status";
}

const char* imdp_last_error(void) { return g_last_error.c_str(); }

const char* imdp_version(void) { return "0.1.0"; }

imdp_status imdp_create_csc(int32_t n_states, int32_t n_cols, int64_t nnz, const int32_t* stateptr,
                            const int32_t* colptr, const int32_t* rowval, const double* lower,
                            const double* upper, imdp_dtype dtype, void* stream, imdp_model** out) {
  set_error("");
  if (!have_device()) { set_error("no CUDA device"); return IMDP_EDEVICE; }
  DevModel* m = nullptr;
  imdp_status s = model_create_csc(n_states, n_cols, nnz, stateptr, colptr, rowval, lower, upper, dtype,
                                   (cudaStream_t)stream, &m);
  if (s != IMDP_OK) return s;
  imdp_model* h = new imdp_model();
  h->dev = m;
  cudaGetDevice(&h->device);
  *out = h;
  return IMDP_OK;
}

imdp_status imdp_create_dense(int32_t n_states, const int32_t* n_actions, const double* lower, const double* upper,
                              imdp_dtype dtype, void* stream, imdp_model** out) {
  set_error("");
  if (!out) { set_error("out is NULL"); return IMDP_EINVAL; }
  *out = nullptr;
  if (n_states < 1 || !n_actions || !lower || !upper) { set_error("bad dense arguments"); return IMDP_EINVAL; }
  std::vector<int32_t> stateptr(n_states + 1, 0);
  for (int32_t s = 0; s < n_states; ++s) {
    if (n_actions[s] < 1) { set_error("every state needs at least one action"); return IMDP_EINVAL; }
    stateptr[s + 1] = stateptr[s] + n_actions[s];
  }
  const int32_t n_cols = stateptr[n_states];
  std::vector<int32_t> colptr(n_cols + 1, 0), rowval;
  std::vector<double> lo, up;
  for (int32_t j = 0; j < n_cols; ++j) {
    for (int32_t d = 0; d < n_states; ++d) {
      const size_t i = (size_t)j * n_states + d;
      if (upper[i] == 0.0 && lower[i] == 0.0) continue;  // structural zero
      rowval.push_back(d);
      lo.push_back(lower[i]);
      up.push_back(upper[i]);
    }
    colptr[j + 1] = (int32_t)rowval.size();
  }
  return imdp_create_csc(n_states, n_cols, (int64_t)rowval.size(), stateptr.data(), colptr.data(), rowval.data(),
                         lo.data(), up.data(), dtype, stream, out);
}

void imdp_model_destroy(imdp_model* m) {
  if (!m) return;
  {
    DeviceGuard g(m->device);
    model_destroy(m->dev);
  }
  delete m;
}

imdp_status imdp_create_csc_f32(int32_t n_states, int32_t n_cols, int64_t nnz, const int32_t* stateptr,
                                const int32_t* colptr, const int32_t* rowval, const double* lower,
                                const double* upper, double budget_per_iteration, void* stream, imdp_model** out) {
  set_error("");
  if (!have_device()) { set_error("no CUDA device"); return IMDP_EDEVICE; }
  DevModel* m = nullptr;
  imdp_status s = model_create_csc(n_states, n_cols, nnz, stateptr, colptr, rowval, lower, upper, IMDP_F32,
                                   (cudaStream_t)stream, &m, 0, -1, budget_per_iteration);
  if (s != IMDP_OK) return s;
  imdp_model* h = new imdp_model();
  h->dev = m;
  cudaGetDevice(&h->device);
  *out = h;
  return IMDP_OK;
}

imdp_status imdp_model_exact_columns(const imdp_model* m, int32_t* n_exact, int64_t* exact_entries,
                                     double* budget_per_iteration) {
  set_error("");
  if (!m || !m->dev) { set_error("model is NULL"); return IMDP_EINVAL; }
  if (n_exact) *n_exact = m->dev->n_exact;
  if (exact_entries) *exact_entries = m->dev->exact_entries;
  if (budget_per_iteration) *budget_per_iteration = m->dev->f32_budget;
  return IMDP_OK;
}

imdp_status imdp_model_info(const imdp_model* m, int32_t* n_states, int32_t* n_cols, int64_t* nnz,
                            size_t* device_bytes, int32_t* max_col_nnz) {
  if (!m) { set_error("model is NULL"); return IMDP_EINVAL; }
  if (n_states) *n_states = m->dev->n_states;
  if (n_cols) *n_cols = m->dev->n_cols;
  if (nnz) *nnz = m->dev->nnz;
  if (device_bytes) *device_bytes = m->dev->bytes;
  if (max_col_nnz) *max_col_nnz = m->dev->max_col;
  return IMDP_OK;
}

void imdp_debug_stall_producer(int32_t on) { g_stall_producer.store(on ? 1 : 0); }

imdp_status imdp_model_plan(const imdp_model* m, int32_t* n_tiles, int32_t* n_wide, int64_t* wide_entries) {
  set_error("");
  if (!m || !m->dev) { set_error("NULL model"); return IMDP_EINVAL; }
  const DevModel* d = m->dev;
  if (n_tiles) *n_tiles = d->n_tiles;
  if (n_wide) *n_wide = d->n_wide;
  if (wide_entries) {
    int64_t e = 0;
    for (int32_t s : d->h_wide) e += d->h_colptr[d->h_stateptr[s + 1]] - d->h_colptr[d->h_stateptr[s]];
    *wide_entries = e;
  }
  return IMDP_OK;
}

imdp_status imdp_model_error_bound(const imdp_model* m, double* per_iteration) {
  if (!m || !per_iteration) { set_error("NULL argument"); return IMDP_EINVAL; }
  *per_iteration = m->dev->err_bound;
  return IMDP_OK;
}

imdp_status imdp_value_iteration(imdp_model* m, const imdp_spec* spec, double* V_out, int32_t* k_out,
                                 double* residual_out, int32_t* policy_out, void* stream) {
  set_error("");
  if (!m || !spec || !V_out) { set_error("NULL model, spec or V_out"); return IMDP_EINVAL; }
  if (!have_device()) { set_error("no CUDA device"); return IMDP_EDEVICE; }
  DeviceGuard g(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  Session* S = nullptr;
  const int32_t want = policy_out ? 1 : 0;
  imdp_status s = Session::create({m->dev}, {spec}, &want, st, &S);
  if (s != IMDP_OK) return s;
  s = S->run(32, st);
  if (s == IMDP_OK) s = S->read(0, V_out, k_out, residual_out, policy_out, st);
  delete S;
  return s;
}

imdp_status imdp_value_iteration_polished(imdp_model* m32, imdp_model* m64, const imdp_spec* spec,
                                          const imdp_launch_config* cfg32, const imdp_launch_config* cfg64,
                                          double* V_out, int32_t* k32_out, int32_t* k_out, double* residual_out,
                                          int32_t* policy_out, void* stream) {
  set_error("");
  if (!m32 || !m64 || !spec || !V_out) { set_error("NULL model, spec or V_out"); return IMDP_EINVAL; }
  if (m32->dev->dtype != IMDP_F32 || m64->dev->dtype != IMDP_F64) {
    set_error("polishing takes the 32-bit model first and the 64-bit model of the same IMDP second");
    return IMDP_EINVAL;
  }
  const DevModel* a = m32->dev;
  const DevModel* b = m64->dev;
  if (m32->device != m64->device || a->n_states != b->n_states || a->n_cols != b->n_cols || a->nnz != b->nnz ||
      a->h_stateptr != b->h_stateptr || a->h_colptr != b->h_colptr) {
    set_error("the two models must have the same structure and live on one device");
    return IMDP_EINVAL;
  }
  if (is_slice(a) || is_slice(b)) { set_error("state slices stop on the residual of every slice"); return IMDP_EINVAL; }
  if (!spec->infinite_time) { set_error("polishing needs an infinite horizon"); return IMDP_EINVAL; }
  if (!have_device()) { set_error("no CUDA device"); return IMDP_EDEVICE; }
  DeviceGuard g(m32->device);
  cudaStream_t st = (cudaStream_t)stream;
  // 1. 32-bit storage to its own fixed point
  Session* S32 = nullptr;
  imdp_status r = Session::create({m32->dev}, {spec}, nullptr, st, &S32);
  if (r != IMDP_OK) return r;
  if (cfg32) {
    imdp_session h{S32};
    r = imdp_session_set_launch(&h, cfg32, stream);
    if (r != IMDP_OK) { delete S32; return r; }
  }
  std::vector<IterState> its;
  r = S32->run(32, st);
  if (r == IMDP_OK) r = S32->read_states(its, st);
  if (r != IMDP_OK) { delete S32; return r; }
  const int32_t k32 = its[0].done ? its[0].k_final : its[0].iter;
  // 2. the 64-bit operator from that iterate: V_k32 and the threshold hints
  // (entry indices, the same in both storages) move over, and the problem
  // resumes at iteration k32 until its own residual test passes
  const int32_t want = policy_out ? 1 : 0;
  Session* S64 = nullptr;
  r = Session::create({m64->dev}, {spec}, &want, st, &S64);
  if (r != IMDP_OK) { delete S32; return r; }
  if (cfg64) {
    imdp_session h{S64};
    r = imdp_session_set_launch(&h, cfg64, stream);
    if (r != IMDP_OK) { delete S32; delete S64; return r; }
  }
  const Problem& P32 = S32->probs_h[0];
  const Problem& P64 = S64->probs_h[0];
  IterState it;
  std::memset(&it, 0, sizeof(it));
  it.iter = k32;
  if (k32 >= P64.horizon) {  // the 32-bit phase used every iteration the cap allows
    it.done = 1;
    it.k_final = k32;
    it.noconv = 1;
  }
  cudaError_t e = cudaMemcpyAsync(P64.V[k32 & 1], P32.V[k32 & 1], sizeof(uint64_t) * (size_t)P64.n_states,
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P64.hint, P32.hint, sizeof(int32_t) * padded_i32((size_t)b->n_cols), cudaMemcpyDeviceToDevice,
                        st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S64->its, &it, sizeof(it), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `it` lives on this stack frame
  delete S32;
  if (e != cudaSuccess) { delete S64; return cuda_status(e, "polishing"); }
  r = S64->run(32, st);
  if (r == IMDP_OK) r = S64->read(0, V_out, k_out, residual_out, policy_out, st);
  delete S64;
  if (r == IMDP_OK && k32_out) *k32_out = k32;
  return r;
}

imdp_status imdp_value_iteration_batch(imdp_model* const* models, const imdp_spec* specs, int32_t count,
                                       double* const* V_out, int32_t* k_out, void* stream) {
  set_error("");
  if (count < 0 || (count > 0 && (!models || !specs || !V_out))) { set_error("bad batch arguments"); return IMDP_EINVAL; }
  if (count == 0) return IMDP_OK;
  if (!have_device()) { set_error("no CUDA device"); return IMDP_EDEVICE; }
  std::vector<DevModel*> ms(count);
  std::vector<const imdp_spec*> sp(count);
  for (int32_t i = 0; i < count; ++i) {
    if (!models[i] || !V_out[i]) { set_error("NULL model or output in batch"); return IMDP_EINVAL; }
    if (models[i]->device != models[0]->device) { set_error("batch models must live on one device"); return IMDP_EINVAL; }
    ms[i] = models[i]->dev;
    sp[i] = &specs[i];
  }
  DeviceGuard g(models[0]->device);
  cudaStream_t st = (cudaStream_t)stream;
  Session* S = nullptr;
  imdp_status s = Session::create(ms, sp, nullptr, st, &S);
  if (s != IMDP_OK) return s;
  s = S->run(32, st);
  imdp_status worst = s;
  for (int32_t i = 0; i < count && s == IMDP_OK; ++i) {
    int32_t k = 0;
    imdp_status r = S->read(i, V_out[i], &k, nullptr, nullptr, st);
    if (r != IMDP_OK && r != IMDP_ENOCONV) { worst = r; break; }
    if (r == IMDP_ENOCONV) worst = r;
    if (k_out) k_out[i] = k;
  }
  delete S;
  return worst;
}

imdp_status imdp_session_create(imdp_model* const* models, const imdp_spec* specs, int32_t count,
                                const int32_t* want_policy, void* stream, imdp_session** out) {
  set_error("");
  if (!out || count < 1 || !models || !specs) { set_error("bad session arguments"); return IMDP_EINVAL; }
  *out = nullptr;
  if (!have_device()) { set_error("no CUDA device"); return IMDP_EDEVICE; }
  std::vector<DevModel*> ms(count);
  std::vector<const imdp_spec*> sp(count);
  for (int32_t i = 0; i < count; ++i) {
    if (!models[i]) { set_error("NULL model in session"); return IMDP_EINVAL; }
    if (models[i]->device != models[0]->device) { set_error("session models must live on one device"); return IMDP_EINVAL; }
    ms[i] = models[i]->dev;
    sp[i] = &specs[i];
  }
  DeviceGuard g(models[0]->device);
  Session* S = nullptr;
  imdp_status s = Session::create(ms, sp, want_policy, (cudaStream_t)stream, &S);
  if (s != IMDP_OK) return s;
  *out = new imdp_session{S};
  return IMDP_OK;
}

imdp_status imdp_session_reset(imdp_session* s, void* stream) {
  if (!s) { set_error("session is NULL"); return IMDP_EINVAL; }
  DeviceGuard g(s->s->device);
  return s->s->reset((cudaStream_t)stream);
}

imdp_status imdp_session_step(imdp_session* s, int32_t n_iters, void* stream) {
  if (!s || n_iters < 0) { set_error("bad session step arguments"); return IMDP_EINVAL; }
  DeviceGuard g(s->s->device);
  return s->s->step(n_iters, (cudaStream_t)stream);
}

imdp_status imdp_session_run(imdp_session* s, int32_t check_every, void* stream) {
  if (!s) { set_error("session is NULL"); return IMDP_EINVAL; }
  DeviceGuard g(s->s->device);
  return s->s->run(check_every, (cudaStream_t)stream);
}

imdp_status imdp_session_read(imdp_session* s, int32_t index, double* V_out, int32_t* k_out, double* residual_out,
                              int32_t* policy_out, void* stream) {
  if (!s) { set_error("session is NULL"); return IMDP_EINVAL; }
  DeviceGuard g(s->s->device);
  return s->s->read(index, V_out, k_out, residual_out, policy_out, (cudaStream_t)stream);
}

int64_t imdp_session_launches(const imdp_session* s) { return s ? s->s->launches : 0; }

void imdp_session_destroy(imdp_session* s) {
  if (!s) return;
  {
    DeviceGuard g(s->s->device);
    delete s->s;
  }
  delete s;
}

}  // extern "C"
