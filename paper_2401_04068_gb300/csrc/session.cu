// Resident solver sessions: device state of value iteration (Eq. 2) for a batch
// of problems, the iteration driver (graph-captured chunks of Bellman steps)
// and the export of (V, k, residual, policy) as value_iteration returns them
// (Sec. 3.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "imdp_internal.h"

namespace imdp {

namespace {

__global__ void init_values_kernel(int64_t n, const uint8_t* __restrict__ fixed, uint64_t* __restrict__ V0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    V0[i] = fixed[i] == 1 ? kOne : 0ull;
}

// W (Q1.63) -> V = offset + scale * W in binary64; with `prev`, writes
// scale * (W - prev), the Bellman residual V_k - V_{k-1}.
__global__ void export_values_kernel(int32_t n, const uint64_t* __restrict__ V, const uint64_t* __restrict__ prev,
                                     double offset, double scale_v, double* __restrict__ out) {
  const double scale = scale_v / 9223372036854775808.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (prev) {
      const uint64_t a = V[i], b = prev[i];
      out[i] = a >= b ? (double)(a - b) * scale : -(double)(b - a) * scale;
    } else {
      out[i] = offset + (double)V[i] * scale;
    }
  }
}


__global__ void fill_i32_kernel(int64_t n, int32_t* p, int32_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// eps in Q1.63 rounded up, so an integer residual r satisfies r < eps_fix
// exactly when r * 2^-63 < eps.
uint64_t eps_to_fixed(double eps) {
  if (eps >= 1.0) return kOne + 1;
  const double x = eps * 9223372036854775808.0;
  uint64_t f = (uint64_t)x;
  if ((double)f < x) f += 1;
  return f;
}

constexpr int kGraphChunk = 16;

}  // namespace

// Affine map of a reward problem into [0, 1] (V = lo + D W). Rewards r, discount
// g, horizon K: if V_{k-1} lies in [a, b], the averaging operator keeps
// T(V_{k-1}) in [a, b], so V_k = r + g T(V_{k-1}) lies in [rmin + g a, rmax + g b];
// from V_0 = r this gives V_k in [rmin A_k, rmax A_k] with A_k = sum_{i<=k} g^i,
// and every V_k, k <= K, lies in [min(rmin, rmin A), max(rmax, rmax A)].
void reward_map(const double* r, int32_t n, double g, int32_t K, bool infinite, double* lo, double* D) {
  double rmin = r[0], rmax = r[0];
  for (int32_t s = 1; s < n; ++s) {
    rmin = r[s] < rmin ? r[s] : rmin;
    rmax = r[s] > rmax ? r[s] : rmax;
  }
  double A;
  if (infinite) A = 1.0 / (1.0 - g);
  else if (g == 1.0) A = (double)K + 1.0;
  else A = (1.0 - std::pow(g, (double)K + 1.0)) / (1.0 - g);
  const double a = std::min(rmin, rmin * A), b = std::max(rmax, rmax * A);
  // widen by a relative margin so rounding never pushes W outside [0, 1]
  const double span = b - a, pad = 1e-9 * (span > 0 ? span : 1.0) + 1e-300;
  *lo = a - pad;
  *D = (span > 0 ? span : 1.0) + 2 * pad;
}

imdp_status check_spec(const DevModel* m, const imdp_spec* sp) {
  if (!sp) { set_error("spec is NULL"); return IMDP_EINVAL; }
  if (sp->property != IMDP_REACH && sp->property != IMDP_REACH_AVOID && sp->property != IMDP_REWARD) {
    set_error("unknown property"); return IMDP_EINVAL;
  }
  if (sp->property == IMDP_REWARD) {
    // Sec. 3.2: rewards per state, discount in (0, 1] (strictly below 1 for an infinite horizon)
    if (!sp->reward) { set_error("reward property needs a reward vector"); return IMDP_EINVAL; }
    if (!(sp->discount > 0.0) || !(sp->discount <= 1.0) || (sp->infinite_time && !(sp->discount < 1.0))) {
      set_error("discount must be in (0, 1] (finite horizon) or (0, 1) (infinite horizon)"); return IMDP_EINVAL;
    }
    for (int32_t s = 0; s < m->n_states; ++s)
      if (!(sp->reward[s] == sp->reward[s]) || sp->reward[s] > 1e300 || sp->reward[s] < -1e300) {
        set_error("rewards must be finite"); return IMDP_EINVAL;
      }
  }
  if (sp->horizon < 0) { set_error("horizon must be >= 0"); return IMDP_EINVAL; }
  if (sp->infinite_time && !(sp->eps > 0.0)) { set_error("eps must be > 0 for an infinite horizon"); return IMDP_EINVAL; }
  if (sp->n_reach < 0 || (sp->n_reach > 0 && !sp->reach)) { set_error("bad reach set"); return IMDP_EINVAL; }
  if (sp->property == IMDP_REACH_AVOID && (sp->n_avoid < 0 || (sp->n_avoid > 0 && !sp->avoid))) {
    set_error("bad avoid set"); return IMDP_EINVAL;
  }
  for (int32_t i = 0; i < sp->n_reach; ++i)
    if (sp->reach[i] < 0 || sp->reach[i] >= m->n_states) { set_error("reach state out of range"); return IMDP_EINVAL; }
  if (sp->property == IMDP_REACH_AVOID)
    for (int32_t i = 0; i < sp->n_avoid; ++i)
      if (sp->avoid[i] < 0 || sp->avoid[i] >= m->n_states) { set_error("avoid state out of range"); return IMDP_EINVAL; }
  return IMDP_OK;
}

Session::~Session() {
  if (graph) cudaGraphExecDestroy(graph);
  side.destroy();
  for (void* p : allocs) cudaFree(p);
}

template <class T>
T* Session::alloc(size_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  allocs.push_back(p);
  return (T*)p;
}

imdp_status Session::create(const std::vector<DevModel*>& ms, const std::vector<const imdp_spec*>& specs,
                            const int32_t* want_policy, cudaStream_t st, Session** out) {
  *out = nullptr;
  const int count = (int)ms.size();
  for (int p = 0; p < count; ++p) {
    imdp_status s = check_spec(ms[p], specs[p]);
    if (s != IMDP_OK) return s;
  }
  Session* S = new Session();
  S->count = count;
  S->models = ms;
  cudaGetDevice(&S->device);
  S->base_h.assign(count + 1, 0);
  for (int p = 0; p < count; ++p) S->base_h[p + 1] = S->base_h[p] + ms[p]->n_states;
  const int64_t total = S->base_h[count];
  if (total >= (int64_t(1) << 31)) { delete S; set_error("batch too large"); return IMDP_EINVAL; }
  S->total = total;
  std::vector<uint8_t> fixed((size_t)total, 0);
  for (int p = 0; p < count; ++p) {
    const imdp_spec* sp = specs[p];
    uint8_t* f = fixed.data() + S->base_h[p];
    if (sp->property != IMDP_REWARD)
      for (int32_t i = 0; i < sp->n_reach; ++i) f[sp->reach[i]] = 1;
    if (sp->property == IMDP_REACH_AVOID)
      for (int32_t i = 0; i < sp->n_avoid; ++i) {
        if (f[sp->avoid[i]] == 1) { delete S; set_error("a state is in both the reach and the avoid set"); return IMDP_EINVAL; }
        f[sp->avoid[i]] = 2;
      }
  }
  S->v_offset.assign(count, 0.0);
  S->v_scale.assign(count, 1.0);
  S->w0.assign(count, nullptr);
  // rank problems by horizon, longest first (infinite horizons first of all):
  // tiles laid out in this order leave the finished problems' tiles at the end
  S->order.resize(count);
  for (int p = 0; p < count; ++p) S->order[p] = p;
  std::stable_sort(S->order.begin(), S->order.end(), [&](int a, int b) {
    const int64_t ka = specs[a]->infinite_time ? INT64_MAX : specs[a]->horizon;
    const int64_t kb = specs[b]->infinite_time ? INT64_MAX : specs[b]->horizon;
    return ka > kb;
  });
  S->fixed_h = fixed;
  S->rank_of = S->alloc<int32_t>(count);
  S->rank_tile_end = S->alloc<int32_t>(count);
  // each problem's hint block starts on a 16-byte boundary and is padded, so
  // the kernel's bulk copies of hint windows stay aligned and in bounds
  for (int p = 0; p < count; ++p) S->total_cols += (int64_t)padded_i32(ms[p]->n_cols);
  S->hints = S->alloc<int32_t>((size_t)S->total_cols);
  S->fixed = S->alloc<uint8_t>(padded_u8(total));
  S->V = S->alloc<uint64_t>(2 * total);
  S->base = S->alloc<int32_t>(count + 1);
  S->probs = S->alloc<Problem>(count);
  S->its = S->alloc<IterState>(count);
  S->ctl = S->alloc<StepControl>(1);
  if (!S->hints || !S->fixed || !S->V || !S->base || !S->probs || !S->its || !S->ctl || !S->rank_of ||
      !S->rank_tile_end) {
    delete S; set_error("device allocation failed (session)"); return IMDP_ENOMEM;
  }
  S->probs_h.resize(count);
  S->policy_cells.assign(count, 0);
  int64_t col_off = 0;
  for (int p = 0; p < count; ++p) {
    DevModel* m = ms[p];
    const imdp_spec* sp = specs[p];
    Problem& P = S->probs_h[p];
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
    P.fixed = S->fixed + S->base_h[p];
    P.hint = S->hints + col_off;
    col_off += (int64_t)padded_i32(m->n_cols);
    P.V[0] = S->V + S->base_h[p];
    P.V[1] = S->V + total + S->base_h[p];
    P.n_states = m->n_states;
    P.pessimistic = sp->pessimistic ? 1 : 0;
    P.maximize = sp->maximize ? 1 : 0;
    P.property = sp->property;
    P.infinite = sp->infinite_time ? 1 : 0;
    // a slice holds part of the states: its own residual decides nothing, the
    // caller stops it on the residual of all slices (imdp_session_residual)
    P.external_stop = (P.infinite && is_slice(m)) ? 1 : 0;
    P.horizon = sp->infinite_time ? (sp->horizon > 0 ? sp->horizon : 1000000) : sp->horizon;
    P.eps_fix = sp->infinite_time ? eps_to_fixed(sp->eps) : 0;
    if (sp->property == IMDP_REWARD) {
      const int32_t n = m->n_states;
      double lo, D;
      reward_map(sp->reward, n, sp->discount, P.horizon, P.infinite != 0, &lo, &D);
      S->v_offset[p] = lo;
      S->v_scale[p] = D;
      std::vector<int64_t> c(n);
      std::vector<uint64_t> w(n);
      const double g = sp->discount;
      for (int32_t s = 0; s < n; ++s) {
        // W_k = c_s + g T(W_{k-1}),  c_s = (r_s - lo (1 - g)) / D  (signed Q2.62)
        const double cs = (sp->reward[s] - lo * (1.0 - g)) / D;
        c[s] = (int64_t)std::llround(cs * 4611686018427387904.0);
        const double ws = std::min(1.0, std::max(0.0, (sp->reward[s] - lo) / D));
        w[s] = (uint64_t)std::llround(ws * 4611686018427387904.0) << 1;
        if (m->lg32) w[s] = round_value32(w[s]);  // values of 32-bit storage keep 32 bits
      }
      int64_t* d_c = S->alloc<int64_t>(n);
      uint64_t* d_w = S->alloc<uint64_t>(n);
      if (!d_c || !d_w) { delete S; set_error("device allocation failed (reward)"); return IMDP_ENOMEM; }
      cudaError_t er = cudaMemcpyAsync(d_c, c.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st);
      if (er == cudaSuccess) er = cudaMemcpyAsync(d_w, w.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st);
      if (er == cudaSuccess) er = cudaStreamSynchronize(st);
      if (er != cudaSuccess) { delete S; return cuda_status(er, "reward setup"); }
      P.rbias = d_c;
      S->w0[p] = d_w;
      P.gamma_fix = g >= 1.0 ? kOne : (uint64_t)std::llround(g * 9223372036854775808.0);
      if (P.infinite) P.eps_fix = eps_to_fixed(sp->eps / D);
    }
    S->max_horizon = std::max(S->max_horizon, P.horizon);
    S->any_infinite = S->any_infinite || P.infinite;
    if (want_policy && want_policy[p]) {
      const size_t cells = (size_t)(P.infinite ? 1 : P.horizon) * m->n_states;
      P.policy = S->alloc<int32_t>(cells);
      if (!P.policy) { delete S; set_error("device allocation failed (policy)"); return IMDP_ENOMEM; }
      P.policy_mode = P.infinite ? 2 : 1;
      S->policy_cells[p] = (int64_t)cells;
    }
  }
  cudaError_t e = cudaMemsetAsync(S->fixed, 0, padded_u8(total), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->fixed, fixed.data(), total, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->base, S->base_h.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->probs, S->probs_h.data(), sizeof(Problem) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host staging vectors go out of scope
  if (e != cudaSuccess) { delete S; return cuda_status(e, "session setup"); }
  S->L.probs = S->probs;
  S->L.its = S->its;
  S->L.state_base = S->base;
  S->L.ctl = S->ctl;
  S->L.count = count;
  S->L.total_states = (int32_t)total;
  S->L.any_infinite = S->any_infinite ? 1 : 0;
  if (count == 1 && !is_slice(ms[0]) && ms[0]->n_states <= kTinyMaxStates && ms[0]->n_cols <= kTinyMaxCols &&
      ms[0]->nnz <= kTinyMaxEntries) {
    S->L.tiny_ok = 1;
    S->L.tiny_states = ms[0]->n_states;
    S->L.tiny_cols = ms[0]->n_cols;
    S->L.tiny_entries = (int32_t)ms[0]->nnz;
  }
  // the kernel by rule for this batch's shape: long columns (the mean over
  // all problems) the direct kernel; short ones the slice kernel when every
  // model already carries its slice layout (building one costs about as much as
  // 450 iterations of the slice kernel save on the pendulum shape), else ring
  {
    int64_t nnz = 0, cols = 0;
    bool all32 = true, laid_out = true;
    for (DevModel* m : ms) {
      nnz += m->nnz;
      cols += m->n_cols;
      all32 = all32 && m->lg32 != nullptr;
      std::lock_guard<std::mutex> lk(m->slices_mu);
      laid_out = laid_out && m->slices != nullptr;
    }
    if (nnz >= kRuleLongColumn * std::max<int64_t>(cols, 1))
      S->L.shape_rule = kKernelDirect;
    else if (laid_out)
      S->L.shape_rule = kKernelSlice;
    S->L.shape_f32 = all32 ? 1 : 0;
  }
  S->grid = bellman_grid();
  const bool slice = resolve_launch(S->L, &S->cfg).kernel == kKernelSlice;
  imdp_status r = slice ? S->prepare_slices(st) : IMDP_OK;
  if (r != IMDP_OK) { delete S; return r; }
  std::vector<Tile> tiles;
  std::vector<int2> wide;
  S->build_plan(S->cfg, tiles, wide);
  r = S->install_plan(tiles, wide, st, slice);
  if (r != IMDP_OK) { delete S; return r; }
  r = S->reset(st);
  if (r != IMDP_OK) { delete S; return r; }
  *out = S;
  return IMDP_OK;
}

imdp_status Session::install_plan(const std::vector<Tile>& tl, const std::vector<int2>& wl, cudaStream_t st,
                                  bool slice) {
  auto release = [&](void* p) {
    if (!p) return;
    allocs.erase(std::remove(allocs.begin(), allocs.end(), p), allocs.end());
    cudaFree(p);
  };
  cudaError_t e = cudaStreamSynchronize(st);  // launches in flight may still read the old plan
  if (e != cudaSuccess) return cuda_status(e, "session plan");
  release(tiles);
  release(wide);
  release(items);
  release(tile_item_end);
  release(win_cnt);
  items = nullptr;
  tile_item_end = nullptr;
  win_cnt = nullptr;
  tiles = alloc<Tile>(tl.size());
  wide = alloc<int2>(wl.size());
  if (!tiles || !wide) { set_error("device allocation failed (tile plan)"); return IMDP_ENOMEM; }
  // slice kernel: one work item per slice of every window (tile), in tile order
  std::vector<int2> it;
  std::vector<int32_t> tend;
  if (slice) {
    tend.resize(tl.size());
    for (size_t t = 0; t < tl.size(); ++t) {
      for (int32_t g = tl[t].x0; g < tl[t].x1; ++g) it.push_back(make_int2((int32_t)t, g));
      tend[t] = (int32_t)it.size();
    }
    items = alloc<int2>(it.size());
    tile_item_end = alloc<int32_t>(tend.size());
    win_cnt = alloc<unsigned int>(tl.size());
    if (!items || !tile_item_end || !win_cnt) { set_error("device allocation failed (slice plan)"); return IMDP_ENOMEM; }
    if (!it.empty()) e = cudaMemcpyAsync(items, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !tend.empty())
      e = cudaMemcpyAsync(tile_item_end, tend.data(), sizeof(int32_t) * tend.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(win_cnt, 0, sizeof(unsigned int) * std::max<size_t>(tl.size(), 1), st);
    if (e != cudaSuccess) return cuda_status(e, "session plan");
  }
  L.items = items;
  L.tile_item_end = tile_item_end;
  L.win_cnt = win_cnt;
  L.n_items = (int32_t)it.size();
  if (!tl.empty()) e = cudaMemcpyAsync(tiles, tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !wl.empty())
    e = cudaMemcpyAsync(wide, wl.data(), sizeof(int2) * wl.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors belong to the caller
  if (e != cudaSuccess) return cuda_status(e, "session plan");
  // tiles of ranks 0..r (the plan lists problems in rank order)
  std::vector<int32_t> rank(count), end(count, 0);
  for (int r = 0; r < count; ++r) rank[order[r]] = r;
  for (const Tile& T : tl) ++end[rank[T.p]];
  for (int r = 1; r < count; ++r) end[r] += end[r - 1];
  e = cudaMemcpyAsync(rank_of, rank.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rank_tile_end, end.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->tile_limit, 0, sizeof(int32_t), st);  // every tile, until a launch ends
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "session plan");
  L.rank_of = rank_of;
  L.rank_tile_end = rank_tile_end;
  n_tiles = (int32_t)tl.size();
  n_wide = (int32_t)wl.size();
  wide_entries = 0;
  for (const int2& w : wl) {
    const DevModel* m = models[w.x];
    wide_entries += m->h_colptr[m->h_stateptr[w.y + 1]] - m->h_colptr[m->h_stateptr[w.y]];
  }
  L.tiles = tiles;
  L.n_tiles = n_tiles;
  L.wide = wide;
  L.n_wide = n_wide;
  L.tile_cols = 0;
  for (const Tile& T : tl) L.tile_cols += T.c1 - T.c0;
  if (n_wide > 0 && n_tiles > 0 && !side.stream && (e = side.create()) != cudaSuccess)
    return cuda_status(e, "session side stream");
  if (graph) {
    cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  return IMDP_OK;
}

imdp_status Session::prepare_slices(cudaStream_t st) {
  if (qbuf) return IMDP_OK;
  for (int p = 0; p < count; ++p) {
    const SliceLayout* l = nullptr;
    imdp_status r = model_slice_layout(models[p], st, &l);
    if (r != IMDP_OK) return r;
  }
  uint64_t* q = alloc<uint64_t>((size_t)total_cols);
  if (!q) { set_error("device allocation failed (slice kernel)"); return IMDP_ENOMEM; }
  cudaError_t e = cudaStreamSynchronize(st);  // launches in flight read the problem descriptors
  if (e != cudaSuccess) return cuda_status(e, "slice kernel setup");
  int64_t col_off = 0;
  for (int p = 0; p < count; ++p) {
    const SliceLayout* l = models[p]->slices;
    Problem& P = probs_h[p];
    P.sl_slot = l->slot;
    P.sl_meta = l->meta;
    P.sl_rows = l->rows;
    P.sl_lg = l->lg;
    P.qcol = q + col_off;  // same offsets as the hints
    col_off += (int64_t)padded_i32(models[p]->n_cols);
  }
  e = cudaMemcpyAsync(probs, probs_h.data(), sizeof(Problem) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "slice kernel setup");
  qbuf = q;
  return IMDP_OK;
}

void Session::build_plan(const LaunchConfig& c, std::vector<Tile>& tl, std::vector<int2>& wl) const {
  const LaunchConfig r = resolve_launch(L, &c);
  if (r.kernel == kKernelSlice) {
    // the windows of every problem's slice layout (prepare_slices built them);
    // x0 / x1 are the window's slices
    for (int p : order) {
      const DevModel* m = models[p];
      const SliceLayout* l = m->slices;
      for (int32_t w = 0; w < l->n_windows; ++w) {
        Tile T;
        T.p = p;
        T.s0 = l->h_win_s0[w];
        T.s1 = l->h_win_s0[w + 1];
        T.c0 = m->h_stateptr[T.s0];
        T.c1 = m->h_stateptr[T.s1];
        T.e0 = m->h_colptr[T.c0];
        T.e1 = m->h_colptr[T.c1];
        T.x0 = l->h_win_sl0[w];
        T.x1 = l->h_win_sl0[w + 1];
        tl.push_back(T);
      }
    }
    return;
  }
  for (int p : order) {
    std::vector<int32_t> ws;
    const size_t at = tl.size();
    plan_tiles(models[p], p, tl, ws, r.tile_entries, r.wide_col, fixed_h.data() + base_h[p]);
    for (size_t t = at; t < tl.size(); ++t) tl[t].p = p;
    for (int32_t s : ws) wl.push_back(make_int2(p, s));
  }
}

imdp_status Session::set_launch(const LaunchConfig& c, cudaStream_t st) {
  const LaunchConfig old = resolve_launch(L, &cfg), now = resolve_launch(L, &c);
  const bool slice = now.kernel == kKernelSlice;
  if (now.tile_entries != old.tile_entries || now.wide_col != old.wide_col || slice != (old.kernel == kKernelSlice)) {
    if (slice) {
      imdp_status r = prepare_slices(st);
      if (r != IMDP_OK) return r;
    }
    std::vector<Tile> tl;
    std::vector<int2> wl;
    build_plan(c, tl, wl);
    imdp_status r = install_plan(tl, wl, st, slice);
    if (r != IMDP_OK) return r;
  }
  cfg = c;
  if (graph) {
    cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  return IMDP_OK;
}

imdp_status Session::reset(cudaStream_t st) {
  TraceRange trace("imdp session reset");
  // the failure-detection test hook ends with a reset; a graph captured while it
  // was on replays launches that issue no copies, so it is captured again
  g_stall_producer.store(0);
  if (graph && graph_stalled) {
    cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  // both buffers: states the property fixes are in no tile, so no launch writes them
  init_values_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 8192), 256, 0, st>>>(total, fixed, V);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    init_values_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 8192), 256, 0, st>>>(total, fixed, V + total);
    e = cudaGetLastError();
  }
  for (int p = 0; p < count && e == cudaSuccess; ++p)
    if (w0[p]) e = cudaMemcpyAsync(probs_h[p].V[0], w0[p], sizeof(uint64_t) * probs_h[p].n_states,
                                   cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(hints, 0xff, sizeof(int32_t) * (size_t)total_cols, st);  // -1: no hint
  if (e == cudaSuccess) e = cudaMemsetAsync(its, 0, sizeof(IterState) * count, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(StepControl), st);
  for (int p = 0; p < count && e == cudaSuccess; ++p)
    if (policy_cells[p] > 0) {
      fill_i32_kernel<<<(int)std::min<int64_t>((policy_cells[p] + 255) / 256, 4096), 256, 0, st>>>(
          policy_cells[p], probs_h[p].policy, -1);
      e = cudaGetLastError();
    }
  if (e != cudaSuccess) return cuda_status(e, "session reset");
  launched_since_reset = 0;
  return IMDP_OK;
}

imdp_status Session::step(int32_t n, cudaStream_t st) {
  if (n <= 0) return IMDP_OK;
  TraceRange trace("imdp session step");
  cudaError_t e = cudaSuccess;
  if (resolve_launch(L, &cfg).kernel == kKernelTiny) {
    // one small problem: all n iterations in one launch of one CTA
    e = launch_bellman_tiny(L, n, models[0]->lg32 != nullptr, st);
    if (e != cudaSuccess) return cuda_status(e, "bellman step");
    launches += n;
    launched_since_reset += n;
    return IMDP_OK;
  }
  int32_t done = 0;
  if (st != nullptr && n >= kGraphChunk) {
    if (!graph) {
      cudaGraph_t g = nullptr;
      graph_stalled = g_stall_producer.load() != 0;
      e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      for (int i = 0; i < kGraphChunk && e == cudaSuccess; ++i) e = launch_bellman_step(L, grid, st, &side, &cfg);
      cudaError_t e2 = cudaStreamEndCapture(st, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        graph = nullptr;
        return cuda_status(e, "graph capture");
      }
    }
    for (; done + kGraphChunk <= n && e == cudaSuccess; done += kGraphChunk) e = cudaGraphLaunch(graph, st);
  }
  for (; done < n && e == cudaSuccess; ++done) e = launch_bellman_step(L, grid, st, &side, &cfg);
  if (e != cudaSuccess) return cuda_status(e, "bellman step");
  launches += n;
  launched_since_reset += n;
  return IMDP_OK;
}

imdp_status Session::read_states(std::vector<IterState>& out, cudaStream_t st) {
  out.resize(count);
  StepControl c{};
  cudaError_t e = cudaMemcpyAsync(out.data(), its, sizeof(IterState) * count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctl, sizeof(StepControl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "read iteration state");
  if (c.error) {
    set_error("a bounded wait inside the Bellman kernel gave up (results of this session are invalid)");
    return IMDP_ETIMEOUT;
  }
  return IMDP_OK;
}

imdp_status Session::run(int32_t check_every, cudaStream_t st) {
  for (const Problem& P : probs_h)
    if (P.external_stop) {
      set_error("an infinite horizon on a state-sharded slice stops on the residual of every slice: step it and "
                "test imdp_session_residual across the slices");
      return IMDP_EINVAL;
    }
  if (!any_infinite) {
    // Every problem finishes within max_horizon launches of the reset.
    return step(std::max<int32_t>(0, max_horizon - (int32_t)std::min<int64_t>(launched_since_reset, max_horizon)), st);
  }
  if (check_every <= 0) check_every = 32;
  std::vector<IterState> s;
  while (launched_since_reset < max_horizon) {
    const int32_t n = (int32_t)std::min<int64_t>(check_every, max_horizon - launched_since_reset);
    imdp_status r = step(n, st);
    if (r != IMDP_OK) return r;
    r = read_states(s, st);
    if (r != IMDP_OK) return r;
    bool all = true;
    for (int p = 0; p < count; ++p) all = all && s[p].done;
    if (all) break;
  }
  return IMDP_OK;
}

imdp_status Session::read(int32_t p, double* V_out, int32_t* k_out, double* res_out, int32_t* pol_out,
                          cudaStream_t st) {
  if (p < 0 || p >= count) { set_error("problem index out of range"); return IMDP_EINVAL; }
  std::vector<IterState> s;
  imdp_status r = read_states(s, st);
  if (r != IMDP_OK) return r;
  const Problem& P = probs_h[p];
  const int32_t k = s[p].done ? s[p].k_final : s[p].iter;
  if (k_out) *k_out = k;
  const int32_t n = P.n_states;
  const uint64_t* Vk = P.V[k & 1];
  const uint64_t* Vk1 = P.V[(k + 1) & 1];
  const int g = std::min((n + 255) / 256, 4096);
  std::vector<void*> tmp;
  auto cleanup = [&]() { for (void* t : tmp) cudaFree(t); };
  auto emit = [&](double* out, const uint64_t* prev) -> cudaError_t {
    if (!out) return cudaSuccess;
    double* dst = out;
    const bool host = !is_device_pointer(out);
    if (host) {
      void* t = nullptr;
      cudaError_t ea = cudaMalloc(&t, sizeof(double) * std::max(n, 1));
      if (ea != cudaSuccess) return ea;
      tmp.push_back(t);
      dst = (double*)t;
    }
    if (prev == nullptr || k >= 1) {
      export_values_kernel<<<g, 256, 0, st>>>(n, Vk, prev, v_offset[p], v_scale[p], dst);
    } else {
      cudaMemsetAsync(dst, 0, sizeof(double) * n, st);
    }
    cudaError_t e2 = cudaGetLastError();
    if (e2 == cudaSuccess && host) e2 = cudaMemcpyAsync(out, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    return e2;
  };
  cudaError_t e = emit(V_out, nullptr);
  if (e == cudaSuccess) e = emit(res_out, Vk1);
  if (e == cudaSuccess && pol_out) {
    if (!P.policy) {
      cleanup();
      set_error("policy was not requested when the session was created");
      return IMDP_EINVAL;
    }
    e = cudaMemcpyAsync(pol_out, P.policy, sizeof(int32_t) * policy_cells[p], cudaMemcpyDefault, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_status(e, "session read");
  if (s[p].noconv) {
    set_error("infinite horizon did not converge within the iteration cap");
    return IMDP_ENOCONV;
  }
  return IMDP_OK;
}

}  // namespace imdp
