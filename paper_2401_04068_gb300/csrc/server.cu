// Continuous-batching server: many value-iteration requests (each a resident
// model plus a specification) share the Bellman launches of one slotted batch.
// A worker thread owns the device state; requests are admitted whenever a slot
// and enough of the server's HBM budget are free, join the running batch between
// chunks of iterations, and retire independently when their own horizon or
// convergence test says so. Because every problem's arithmetic is independent
// and exact-integer, a result is the same whether the request ran alone or in
// the mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "imdp_internal.h"

namespace imdp {

namespace {

using Clock = std::chrono::steady_clock;

// V_0 = 1_G in both value buffers (states the property fixes are in no tile,
// so no launch writes them).
__global__ void srv_init_kernel(int32_t n, const uint8_t* __restrict__ fixed, uint64_t* __restrict__ V0) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    V0[i] = V0[n + i] = fixed[i] == 1 ? kOne : 0ull;
}

__global__ void srv_export_kernel(int32_t n, const uint64_t* __restrict__ W, double offset, double scale_v,
                                  double* __restrict__ out) {
  const double scale = scale_v / 9223372036854775808.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = offset + (double)W[i] * scale;
}

// First-fit allocator over one device arena (offsets, 256-byte granules).
class Arena {
 public:
  explicit Arena(size_t bytes) : size_(bytes & ~size_t(255)) { free_[0] = size_; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }

 private:
  size_t size_;
  std::map<size_t, size_t> free_;
};

struct Request {
  uint64_t ticket = 0;
  DevModel* model = nullptr;
  imdp_spec spec{};
  std::vector<int32_t> reach, avoid;
  std::vector<double> reward;
  Clock::time_point submitted, finished;
  int slot = -1;
  size_t off = 0, bytes = 0;   // arena block
  double v_offset = 0.0, v_scale = 1.0;
  std::vector<double> result;
  int32_t k = 0;
  imdp_status status = IMDP_EPENDING;
  bool done = false;
  std::vector<Tile> tiles;     // tile plan under the server's launch configuration (fixed states left out)
  std::vector<int32_t> wide;   // wide states
};

size_t working_bytes(const DevModel* m, const imdp_spec* sp) {
  const size_t n = (size_t)m->n_states;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
  add(2 * n * sizeof(uint64_t));               // V ping-pong
  add(padded_u8(n));                           // reach/avoid mask
  add(padded_i32(m->n_cols) * sizeof(int32_t));  // threshold hints (padded for bulk copies)
  add(n * sizeof(double));                     // exported values
  if (sp->property == IMDP_REWARD) {
    add(n * sizeof(int64_t));                  // c_s
    add(n * sizeof(uint64_t));                 // W_0
  }
  return b;
}

}  // namespace

struct Server {
  int device = 0;
  int32_t max_active = 1024;
  int32_t chunk = 8;
  Arena arena;
  unsigned char* base = nullptr;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  std::vector<Request*> slots;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // device tables
  Problem* d_probs = nullptr;
  IterState* d_its = nullptr;
  StepControl* d_ctl = nullptr;
  int32_t* d_base = nullptr;
  Tile* d_tiles = nullptr;
  size_t tile_cap = 0;
  std::vector<Problem> probs_h;
  imdp_status fatal = IMDP_OK;
  LaunchConfig cfg;  // kernel shape and tile plan limits of the launches (worker reads it under mu)
  // statistics (worker thread; read under mu): device time of the chunks (CUDA
  // events around each chunk's launches), wall time of the loop while requests
  // were running, chunks, and requests in the launches summed over chunks
  double st_device_ms = 0.0, st_wall_ms = 0.0, st_slots = 0.0;
  int64_t st_chunks = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  explicit Server(size_t budget) : arena(budget) {}
  ~Server() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    if (worker.joinable()) worker.join();
    cudaSetDevice(device);
    if (stream) cudaStreamDestroy(stream);
    cudaFree(base);
    cudaFree(d_probs);
    cudaFree(d_its);
    cudaFree(d_ctl);
    cudaFree(d_base);
    cudaFree(d_tiles);
    cudaFree(d_wide);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    side.destroy();
    for (auto& kv : all) delete kv.second;
  }

  // Worker side ------------------------------------------------------------

  bool admit(Request* r, int slot) {
    // called with mu held; sets up device state on the worker stream
    size_t off;
    if (!arena.alloc(r->bytes, &off)) return false;
    r->off = off;
    r->slot = slot;
    const DevModel* m = r->model;
    const int32_t n = m->n_states;
    unsigned char* p = base + off;
    auto take = [&](size_t x) {
      unsigned char* q = p;
      p += (x + 255) & ~size_t(255);
      return q;
    };
    uint64_t* V = (uint64_t*)take(2 * (size_t)n * sizeof(uint64_t));
    uint8_t* mask = take(padded_u8(n));
    int32_t* hints = (int32_t*)take(padded_i32(m->n_cols) * sizeof(int32_t));
    take((size_t)n * sizeof(double));  // export buffer (address recomputed on retire)
    Problem P;
    std::memset(&P, 0, sizeof(P));
    P.stateptr = m->stateptr;
    P.colptr = m->colptr;
    P.rowval = m->rowval;
    P.lg = m->lg;
    P.rem = m->rem;
    P.lg32 = m->lg32;
    P.shift = m->shift;
    P.xoff = m->xoff;
    P.lgx = m->lgx;
    P.fixed = mask;
    P.V[0] = V;
    P.V[1] = V + n;
    P.hint = hints;
    P.n_states = n;
    const imdp_spec* sp = &r->spec;
    P.pessimistic = sp->pessimistic ? 1 : 0;
    P.maximize = sp->maximize ? 1 : 0;
    P.property = sp->property;
    P.infinite = sp->infinite_time ? 1 : 0;
    P.horizon = sp->infinite_time ? (sp->horizon > 0 ? sp->horizon : 1000000) : sp->horizon;
    std::vector<uint8_t> f((size_t)n, 0);
    if (sp->property != IMDP_REWARD) {
      for (int32_t v : r->reach) f[v] = 1;
      for (int32_t v : r->avoid) f[v] = 2;
    }
    {
      const LaunchConfig rc = resolve_launch(StepLaunch{}, &cfg);
      r->tiles.clear();
      r->wide.clear();
      plan_tiles(m, 0, r->tiles, r->wide, rc.tile_entries, rc.wide_col, f.data());
    }
    cudaError_t e = cudaMemsetAsync(mask, 0, padded_u8(n), stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mask, f.data(), n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hints, 0xff, padded_i32(m->n_cols) * sizeof(int32_t), stream);
    if (sp->property == IMDP_REWARD) {
      int64_t* c = (int64_t*)take((size_t)n * sizeof(int64_t));
      uint64_t* w0 = (uint64_t*)take((size_t)n * sizeof(uint64_t));
      double lo, D;
      reward_map(r->reward.data(), n, sp->discount, P.horizon, P.infinite != 0, &lo, &D);
      r->v_offset = lo;
      r->v_scale = D;
      std::vector<int64_t> ch(n);
      std::vector<uint64_t> wh(n);
      for (int32_t s = 0; s < n; ++s) {
        ch[s] = (int64_t)std::llround((r->reward[s] - lo * (1.0 - sp->discount)) / D * 4611686018427387904.0);
        const double ws = std::min(1.0, std::max(0.0, (r->reward[s] - lo) / D));
        wh[s] = (uint64_t)std::llround(ws * 4611686018427387904.0) << 1;
        if (m->lg32) wh[s] = round_value32(wh[s]);  // values of 32-bit storage keep 32 bits
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(c, ch.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(V, wh.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // host vectors go out of scope
      P.rbias = c;
      P.gamma_fix = sp->discount >= 1.0 ? kOne : (uint64_t)std::llround(sp->discount * 9223372036854775808.0);
      P.eps_fix = P.infinite ? eps_fixed(sp->eps / D) : 0;
      (void)w0;
    } else {
      P.eps_fix = P.infinite ? eps_fixed(sp->eps) : 0;
      if (e == cudaSuccess) {
        srv_init_kernel<<<std::min((n + 255) / 256, 1024), 256, 0, stream>>>(n, mask, V);
        e = cudaGetLastError();
      }
    }
    IterState it;
    std::memset(&it, 0, sizeof(it));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_its + slot, &it, sizeof(it), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // `f` and `it` are stack/heap temporaries
    if (e != cudaSuccess) {
      arena.release(r->off, r->bytes);
      r->slot = -1;
      r->status = cuda_status(e, "server admit");
      r->done = true;
      r->finished = Clock::now();
      return true;  // consumed (failed)
    }
    probs_h[slot] = P;
    slots[slot] = r;
    return true;
  }

  imdp_status upload_tables(int32_t count) {
    std::vector<Tile> tiles;
    std::vector<int2> wide;
    int64_t cols = 0;
    for (int32_t s = 0; s < count; ++s) {
      Request* r = slots[s];
      if (!r) continue;
      const size_t at = tiles.size();
      tiles.insert(tiles.end(), r->tiles.begin(), r->tiles.end());
      for (size_t t = at; t < tiles.size(); ++t) {
        tiles[t].p = s;
        cols += tiles[t].c1 - tiles[t].c0;
      }
      for (int32_t st : r->wide) wide.push_back(make_int2(s, st));
    }
    if (wide.size() > wide_cap) {
      cudaFree(d_wide);
      wide_cap = std::max(wide.size(), wide_cap * 2);
      if (cudaMalloc(&d_wide, sizeof(int2) * wide_cap) != cudaSuccess) {
        cudaGetLastError();
        d_wide = nullptr;
        wide_cap = 0;
        set_error("server: wide-state table allocation failed");
        return IMDP_ENOMEM;
      }
    }
    if (tiles.size() > tile_cap) {
      cudaFree(d_tiles);
      tile_cap = std::max(tiles.size(), tile_cap * 2);
      if (cudaMalloc(&d_tiles, sizeof(Tile) * tile_cap) != cudaSuccess) {
        cudaGetLastError();
        d_tiles = nullptr;
        tile_cap = 0;
        set_error("server: tile table allocation failed");
        return IMDP_ENOMEM;
      }
    }
    cudaError_t e = cudaSuccess;
    if (!tiles.empty())
      e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && !wide.empty())
      e = cudaMemcpyAsync(d_wide, wide.data(), sizeof(int2) * wide.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_probs, probs_h.data(), sizeof(Problem) * count, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e, "server tables");
    n_tiles = (int32_t)tiles.size();
    n_wide = (int32_t)wide.size();
    tile_cols = cols;
    return IMDP_OK;
  }

  int32_t n_tiles = 0;
  int64_t tile_cols = 0;
  int32_t n_wide = 0;
  SideStream side;
  int2* d_wide = nullptr;
  size_t wide_cap = 0;

  void retire(Request* r, const IterState& it) {
    const DevModel* m = r->model;
    const int32_t n = m->n_states;
    const int32_t k = it.done ? it.k_final : it.iter;
    unsigned char* p = base + r->off;
    auto step = [&](size_t x) { return (x + 255) & ~size_t(255); };
    uint64_t* V = (uint64_t*)p;
    double* out = (double*)(p + step(2 * (size_t)n * 8) + step(padded_u8(n)) + step(padded_i32(m->n_cols) * 4));
    r->result.resize(n);
    srv_export_kernel<<<std::min((n + 255) / 256, 1024), 256, 0, stream>>>(n, V + (size_t)(k & 1) * n, r->v_offset,
                                                                        r->v_scale, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->result.data(), out, sizeof(double) * n, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    r->k = k;
    r->status = e != cudaSuccess ? cuda_status(e, "server retire") : (it.noconv ? IMDP_ENOCONV : IMDP_OK);
    r->finished = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    arena.release(r->off, r->bytes);
    slots[r->slot] = nullptr;
    std::memset(&probs_h[r->slot], 0, sizeof(Problem));
    r->slot = -1;
    r->done = true;
    cv.notify_all();
  }

  void run() {
    cudaSetDevice(device);
    std::vector<IterState> its;
    int32_t count = 0;  // slots [0, count) are in the launch
    while (true) {
      bool changed = false;
      const Clock::time_point h0 = Clock::now();
      {
        std::unique_lock<std::mutex> lk(mu);
        bool any_active = false;
        for (Request* r : slots) any_active = any_active || r;
        if (!any_active && queue.empty()) {
          cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop || !queue.empty(); });
        }
        if (stop) return;
        // admit in arrival order while a slot and budget are free
        while (!queue.empty()) {
          int slot = -1;
          for (int s = 0; s < max_active; ++s)
            if (!slots[s]) {
              slot = s;
              break;
            }
          if (slot < 0) break;
          Request* r = queue.front();
          if (!admit(r, slot)) break;  // wait for budget
          queue.pop_front();
          changed = true;
        }
      }
      int32_t hi = 0;
      for (int s = 0; s < max_active; ++s)
        if (slots[s]) hi = s + 1;
      if (hi == 0) continue;
      if (changed || hi != count) {
        // slots without a request keep done = 1 (set at creation, kept on retire)
        count = hi;
        const imdp_status st = upload_tables(count);
        if (st != IMDP_OK) {
          std::lock_guard<std::mutex> lk(mu);
          fatal = st;
          for (Request* r : slots)
            if (r) {
              r->status = st;
              r->done = true;
            }
          cv.notify_all();
          return;
        }
      }
      pending_host_ms = std::chrono::duration<double, std::milli>(Clock::now() - h0).count();
      StepLaunch L{};
      L.probs = d_probs;
      L.its = d_its;
      L.state_base = d_base;
      L.ctl = d_ctl;
      L.count = count;
      L.total_states = 0;
      L.any_infinite = 1;
      L.tiles = d_tiles;
      L.n_tiles = n_tiles;
      L.tile_cols = tile_cols;
      L.wide = d_wide;
      L.n_wide = n_wide;
      const int grid = bellman_grid();
      TraceRange trace("imdp server chunk");
      LaunchConfig lc;
      {
        std::lock_guard<std::mutex> lk(mu);
        lc = cfg;
      }
      const Clock::time_point w0 = Clock::now();
      cudaError_t e = cudaSuccess;
      if (!ev0) {
        e = cudaEventCreate(&ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&ev1);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev0, stream);
      for (int i = 0; i < chunk && e == cudaSuccess; ++i) e = launch_bellman_step(L, grid, stream, &side, &lc);
      if (e == cudaSuccess) e = cudaEventRecord(ev1, stream);
      its.resize(count);
      StepControl c{};
      if (e == cudaSuccess) e = cudaMemcpyAsync(its.data(), d_its, sizeof(IterState) * count, cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&c, d_ctl, sizeof(c), cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess || c.error) {
        std::lock_guard<std::mutex> lk(mu);
        fatal = e != cudaSuccess ? cuda_status(e, "server step") : IMDP_ETIMEOUT;
        for (Request* r : slots)
          if (r) {
            r->status = fatal;
            r->done = true;
          }
        cv.notify_all();
        return;
      }
      float dev_ms = 0.f;
      cudaEventElapsedTime(&dev_ms, ev0, ev1);
      int active = 0;
      for (int s = 0; s < count; ++s) {
        Request* r = slots[s];
        active += r ? 1 : 0;
        if (r && its[s].done) retire(r, its[s]);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        st_device_ms += dev_ms;
        st_chunks += 1;
        st_slots += active;
        // wall time from this chunk's launches to the end of its retirements;
        // admission and table uploads before the next chunk are added there
        st_wall_ms += std::chrono::duration<double, std::milli>(Clock::now() - w0).count() + pending_host_ms;
      }
      pending_host_ms = 0.0;
    }
  }
  double pending_host_ms = 0.0;  // admission and table work before the next chunk (worker only)

  static uint64_t eps_fixed(double eps) {
    if (eps >= 1.0) return kOne + 1;
    const double x = eps * 9223372036854775808.0;
    uint64_t f = (uint64_t)x;
    if ((double)f < x) f += 1;
    return f;
  }
};

}  // namespace imdp

using namespace imdp;

struct imdp_server {
  Server* s;
};

extern "C" {

imdp_status imdp_server_stats(imdp_server* srv, double* device_ms, double* wall_ms, int64_t* chunks,
                              double* mean_requests) {
  set_error("");
  if (!srv || !srv->s) { set_error("NULL server"); return IMDP_EINVAL; }
  Server* S = srv->s;
  std::lock_guard<std::mutex> lk(S->mu);
  if (device_ms) *device_ms = S->st_device_ms;
  if (wall_ms) *wall_ms = S->st_wall_ms;
  if (chunks) *chunks = S->st_chunks;
  if (mean_requests) *mean_requests = S->st_chunks ? S->st_slots / (double)S->st_chunks : 0.0;
  return IMDP_OK;
}

imdp_status imdp_server_set_launch(imdp_server* srv, const imdp_launch_config* cfg) {
  set_error("");
  if (!srv || !srv->s || !cfg) { set_error("NULL server or configuration"); return IMDP_EINVAL; }
  if (cfg->kernel < 0 || cfg->kernel > 2 || cfg->tile_entries < 0 || cfg->wide_col < 0) {
    set_error("bad launch configuration");
    return IMDP_EINVAL;
  }
  LaunchConfig c;
  c.kernel = cfg->kernel;
  c.cta_warps = cfg->cta_warps;
  c.ctas_per_sm = cfg->ctas_per_sm;
  c.tile_entries = cfg->tile_entries;
  c.wide_col = cfg->wide_col;
  std::lock_guard<std::mutex> lk(srv->s->mu);
  srv->s->cfg = c;  // requests admitted from now on are planned with its limits
  return IMDP_OK;
}

imdp_status imdp_server_create(size_t hbm_budget, imdp_server** out) {
  set_error("");
  if (!out || hbm_budget < (size_t(1) << 20)) { set_error("server needs out and a budget of at least 1 MiB"); return IMDP_EINVAL; }
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    set_error("no CUDA device");
    return IMDP_EDEVICE;
  }
  Server* S = new Server(hbm_budget);
  cudaGetDevice(&S->device);
  S->slots.assign(S->max_active, nullptr);
  S->probs_h.assign(S->max_active, Problem{});
  cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = S->side.create();
  if (e == cudaSuccess) e = cudaMalloc(&S->base, S->arena.size());
  if (e == cudaSuccess) e = cudaMalloc(&S->d_probs, sizeof(Problem) * S->max_active);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_its, sizeof(IterState) * S->max_active);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_ctl, sizeof(StepControl));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_base, sizeof(int32_t) * 2);
  if (e == cudaSuccess) e = cudaMemset(S->d_ctl, 0, sizeof(StepControl));
  if (e == cudaSuccess) e = cudaMemset(S->d_base, 0, sizeof(int32_t) * 2);
  if (e == cudaSuccess) e = cudaMemset(S->d_probs, 0, sizeof(Problem) * S->max_active);
  if (e != cudaSuccess) {
    const imdp_status st = cuda_status(e, "server create");
    delete S;
    return st;
  }
  // every slot starts "done" (empty)
  std::vector<IterState> init(S->max_active);
  for (auto& it : init) {
    std::memset(&it, 0, sizeof(it));
    it.done = 1;
  }
  e = cudaMemcpy(S->d_its, init.data(), sizeof(IterState) * S->max_active, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    const imdp_status st = cuda_status(e, "server create");
    delete S;
    return st;
  }
  S->worker = std::thread([S] { S->run(); });
  *out = new imdp_server{S};
  return IMDP_OK;
}

imdp_status imdp_server_submit(imdp_server* srv, imdp_model* m, const imdp_spec* spec, uint64_t* ticket) {
  set_error("");
  if (!srv || !m || !spec || !ticket) { set_error("NULL argument"); return IMDP_EINVAL; }
  Server* S = srv->s;
  if (m->device != S->device) { set_error("model and server must be on one device"); return IMDP_EINVAL; }
  if (is_slice(m->dev)) { set_error("slices of a state-sharded model run in sessions only"); return IMDP_EINVAL; }
  imdp_status st = check_spec(m->dev, spec);
  if (st != IMDP_OK) return st;
  Request* r = new Request();
  r->model = m->dev;
  r->spec = *spec;
  if (spec->n_reach > 0) r->reach.assign(spec->reach, spec->reach + spec->n_reach);
  if (spec->property == IMDP_REACH_AVOID && spec->n_avoid > 0) r->avoid.assign(spec->avoid, spec->avoid + spec->n_avoid);
  if (spec->property == IMDP_REWARD) r->reward.assign(spec->reward, spec->reward + m->dev->n_states);
  for (int32_t v : r->avoid)
    if (std::find(r->reach.begin(), r->reach.end(), v) != r->reach.end()) {
      delete r;
      set_error("a state is in both the reach and the avoid set");
      return IMDP_EINVAL;
    }
  r->spec.reach = nullptr;
  r->spec.avoid = nullptr;
  r->spec.reward = nullptr;
  r->bytes = working_bytes(m->dev, spec);
  if (r->bytes > S->arena.size()) {
    delete r;
    set_error("request needs more device memory than the server's budget");
    return IMDP_ENOMEM;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->fatal != IMDP_OK) {
    delete r;
    set_error("server stopped after a device error");
    return S->fatal;
  }
  if (S->queue.size() >= 1000000) {
    delete r;
    set_error("server queue full");
    return IMDP_EBUSY;
  }
  r->ticket = S->next_ticket++;
  r->submitted = Clock::now();
  S->queue.push_back(r);
  S->all[r->ticket] = r;
  *ticket = r->ticket;
  S->cv.notify_all();
  return IMDP_OK;
}

imdp_status imdp_server_poll(imdp_server* srv, uint64_t ticket, double* V_out, int32_t* k_out, double* latency_ms) {
  if (!srv) { set_error("NULL server"); return IMDP_EINVAL; }
  Server* S = srv->s;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) { set_error("unknown ticket"); return IMDP_ENOTFOUND; }
  Request* r = it->second;
  if (!r->done) return IMDP_EPENDING;
  const imdp_status st = r->status;
  if (st == IMDP_OK || st == IMDP_ENOCONV) {
    if (V_out) {
      if (is_device_pointer(V_out)) {
        cudaMemcpy(V_out, r->result.data(), sizeof(double) * r->result.size(), cudaMemcpyHostToDevice);
      } else {
        std::memcpy(V_out, r->result.data(), sizeof(double) * r->result.size());
      }
    }
    if (k_out) *k_out = r->k;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->finished - r->submitted).count();
  }
  S->all.erase(it);
  delete r;
  return st;
}

imdp_status imdp_server_wait(imdp_server* srv, uint64_t ticket, double timeout_ms, double* V_out, int32_t* k_out,
                             double* latency_ms) {
  if (!srv) { set_error("NULL server"); return IMDP_EINVAL; }
  Server* S = srv->s;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("unknown ticket"); return IMDP_ENOTFOUND; }
    Request* r = it->second;
    const bool ok = S->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] { return r->done; });
    if (!ok) { set_error("timed out waiting for the request"); return IMDP_ETIMEOUT; }
  }
  return imdp_server_poll(srv, ticket, V_out, k_out, latency_ms);
}

void imdp_server_destroy(imdp_server* srv) {
  if (!srv) return;
  delete srv->s;
  delete srv;
}

}  // extern "C"
