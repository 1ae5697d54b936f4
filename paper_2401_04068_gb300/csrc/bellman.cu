// Robust Bellman step (Eq. 2 / Eq. 3) with O-maximization (Sec. 4) for sm_103a.
//
// One launch performs one value-iteration step V_{k-1} -> V_k for every problem
// of a batch that is still running. A warp owns one state at a time and walks
// its actions (the CSC columns of that state); the optimum over actions, the
// target/avoid mask, the policy record and the residual are fused in.
//
// O-maximization without a sort. For a pessimistic adversary the procedure of
// Sec. 4 orders the destinations by ascending V, starts from p = lower and hands
// out rem = 1 - sum(lower) gap by gap along that order. Its result depends only
// on the *threshold*: the first destination (in that order) at which the
// inclusive prefix of gaps reaches rem. Everything before it receives its full
// gap, the threshold receives what is left, everything after it keeps its lower
// bound. Destinations with equal V are interchangeable (the value of the sum is
// the same whichever of them gets the mass), so the threshold can be taken on
// the value itself:
//     q = sum_i V_i P_lo,i + sum_{V_i < v*} V_i gap_i + v* (rem - sum_{V_i < v*} gap_i),
//     v* = the smallest V_i with sum_{V_j <= V_i} gap_j >= rem.
// The kernel finds v* by a weighted selection on integer keys (the Q1.63 value,
// complemented for an optimistic adversary so that the order is always
// ascending): each round takes the min/max key of the remaining candidates,
// histograms their gaps into 32 bins of the key range, and keeps the bin in
// which the prefix crosses rem. Each round shrinks the key range by >= 16x and
// usually isolates a single key after two or three rounds; no element moves.
// A final pass applies the threshold and forms the dot product.
#include <cuda_runtime.h>

#include "imdp_internal.h"

namespace imdp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t y = __shfl_xor_sync(kFull, x, o);
    x = y < x ? y : x;
  }
  return x;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t y = __shfl_xor_sync(kFull, x, o);
    x = y > x ? y : x;
  }
  return x;
}
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Result of the threshold search over one column.
struct Threshold {
  uint64_t key;   // threshold key; ~0 when the gaps cannot absorb rem (all below)
  uint64_t fb;    // sum of gaps of entries with key < threshold
  bool all_below;
};

// One selection round's bookkeeping shared by the register and streaming paths.
// Given the warp-wide min/max of the candidate keys and the per-lane histogram
// value h (bin = lane), decide the next window. Returns true when done.
__device__ __forceinline__ bool select_round_finish(uint64_t h, int lane, uint64_t rem, uint64_t cmin, int shift,
                                                    uint64_t cmax, uint64_t& fb, uint64_t& lo, uint64_t& hi,
                                                    bool& all_below) {
  uint64_t incl = warp_incl_scan_u64(h, lane);
  unsigned cross = __ballot_sync(kFull, fb + incl >= rem);
  if (cross == 0) {  // only possible in the first round: sum of all gaps < rem
    all_below = true;
    return true;
  }
  int b = __ffs(cross) - 1;
  uint64_t excl_b = __shfl_sync(kFull, incl - h, b);
  fb += excl_b;
  lo = cmin + ((uint64_t)b << shift);
  uint64_t top = lo + ((1ull << shift) - 1ull);
  hi = top < cmax ? top : cmax;
  return false;
}

// Column held in registers: up to 32*E entries, entry idx = lane + 32*e.
template <int E>
__device__ __forceinline__ uint64_t column_q_regs(const int32_t* __restrict__ rowval,
                                                  const ulonglong2* __restrict__ lg, int32_t c0, int32_t k,
                                                  uint64_t rem, const uint64_t* __restrict__ V, bool pess,
                                                  unsigned long long* hist, int lane) {
  uint64_t key[E], lo_[E], gap[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    int idx = lane + 32 * e;
    if (idx < k) {
      int32_t r = __ldg(rowval + c0 + idx);
      ulonglong2 p = __ldg(lg + c0 + idx);
      uint64_t v = __ldg(V + r);
      key[e] = pess ? v : (kOne - v);
      lo_[e] = p.x;
      gap[e] = p.y;
    } else {
      key[e] = ~0ull;  // never a candidate, never below a finite threshold
      lo_[e] = 0;
      gap[e] = 0;
    }
  }

  uint64_t thr = ~0ull, fb = 0;
  bool all_below = false;
  if (rem != 0) {
    uint64_t lo = 0, hi = kOne;
    for (int round = 0; round < 20; ++round) {
      uint64_t cmin = ~0ull, cmax = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        bool c = key[e] >= lo && key[e] <= hi;
        if (c) {
          cmin = key[e] < cmin ? key[e] : cmin;
          cmax = key[e] > cmax ? key[e] : cmax;
        }
      }
      cmin = warp_min_u64(cmin);
      cmax = warp_max_u64(cmax);
      if (cmin > cmax) {  // no candidate at all (cannot happen for a feasible column)
        all_below = true;
        break;
      }
      if (cmin == cmax) {
        thr = cmin;
        break;
      }
      int bits = 64 - __clzll((long long)(cmax - cmin));
      int shift = bits > 5 ? bits - 5 : 0;
      hist[lane] = 0;
      __syncwarp();
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (key[e] >= cmin && key[e] <= cmax && key[e] >= lo && key[e] <= hi && gap[e] != 0)
          atomicAdd(&hist[(key[e] - cmin) >> shift], (unsigned long long)gap[e]);
      }
      __syncwarp();
      uint64_t h = hist[lane];
      __syncwarp();
      if (select_round_finish(h, lane, rem, cmin, shift, cmax, fb, lo, hi, all_below)) break;
    }
    if (all_below) thr = ~0ull;
  }
  // rem == 0: every entry keeps its lower bound; thr stays ~0 but nothing is
  // "below" in the sense of receiving a gap, handled by the rem test.

  uint64_t acc = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (key[e] != ~0ull) {
      uint64_t v = pess ? key[e] : (kOne - key[e]);
      uint64_t w = (rem != 0 && key[e] < thr) ? lo_[e] + gap[e] : lo_[e];
      acc += __umul64hi(v, w);
    }
  }
  acc = warp_sum_u64(acc);
  if (rem != 0 && !all_below) {
    uint64_t vthr = pess ? thr : (kOne - thr);
    acc += __umul64hi(vthr, rem - fb);
  }
  return acc;  // Q2.62
}

// Column too long for registers: the same rounds, re-reading the column from
// global memory (L1/L2) on every pass, one entry per lane per step.
__device__ uint64_t column_q_stream(const int32_t* __restrict__ rowval, const ulonglong2* __restrict__ lg,
                                    int32_t c0, int32_t k, uint64_t rem, const uint64_t* __restrict__ V, bool pess,
                                    unsigned long long* hist, int lane) {
  auto load_key = [&](int idx) -> uint64_t {
    uint64_t v = __ldg(V + __ldg(rowval + c0 + idx));
    return pess ? v : (kOne - v);
  };
  uint64_t thr = ~0ull, fb = 0;
  bool all_below = false;
  if (rem != 0) {
    uint64_t lo = 0, hi = kOne;
    for (int round = 0; round < 20; ++round) {
      uint64_t cmin = ~0ull, cmax = 0;
      for (int idx = lane; idx < k; idx += 32) {
        uint64_t key = load_key(idx);
        if (key >= lo && key <= hi) {
          cmin = key < cmin ? key : cmin;
          cmax = key > cmax ? key : cmax;
        }
      }
      cmin = warp_min_u64(cmin);
      cmax = warp_max_u64(cmax);
      if (cmin > cmax) {  // no candidate at all (cannot happen for a feasible column)
        all_below = true;
        break;
      }
      if (cmin == cmax) {
        thr = cmin;
        break;
      }
      int bits = 64 - __clzll((long long)(cmax - cmin));
      int shift = bits > 5 ? bits - 5 : 0;
      hist[lane] = 0;
      __syncwarp();
      for (int idx = lane; idx < k; idx += 32) {
        uint64_t key = load_key(idx);
        if (key >= lo && key <= hi) {
          uint64_t g = __ldg(lg + c0 + idx).y;
          if (g) atomicAdd(&hist[(key - cmin) >> shift], (unsigned long long)g);
        }
      }
      __syncwarp();
      uint64_t h = hist[lane];
      __syncwarp();
      if (select_round_finish(h, lane, rem, cmin, shift, cmax, fb, lo, hi, all_below)) break;
    }
    if (all_below) thr = ~0ull;
  }
  uint64_t acc = 0;
  for (int idx = lane; idx < k; idx += 32) {
    uint64_t key = load_key(idx);
    ulonglong2 p = __ldg(lg + c0 + idx);
    uint64_t v = pess ? key : (kOne - key);
    uint64_t w = (rem != 0 && key < thr) ? p.x + p.y : p.x;
    acc += __umul64hi(v, w);
  }
  acc = warp_sum_u64(acc);
  if (rem != 0 && !all_below) {
    uint64_t vthr = pess ? thr : (kOne - thr);
    acc += __umul64hi(vthr, rem - fb);
  }
  return acc;
}

__device__ __forceinline__ int find_problem(const int32_t* __restrict__ base, int count, int32_t g) {
  int lo = 0, hi = count;  // base[lo] <= g < base[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= g) lo = mid; else hi = mid;
  }
  return lo;
}

template <int E>
__global__ void __launch_bounds__(kThreads) bellman_step_kernel(StepLaunch L) {
  __shared__ unsigned long long hist_all[kWarpsPerBlock][32];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  unsigned long long* hist = hist_all[warp];
  const int32_t n_warps = gridDim.x * kWarpsPerBlock;

  int cur_p = -1;
  unsigned long long run_max = 0;  // residual max of cur_p seen by this warp

  for (int32_t g = blockIdx.x * kWarpsPerBlock + warp; g < L.total_states; g += n_warps) {
    const int p = L.count == 1 ? 0 : find_problem(L.state_base, L.count, g);
    const Problem& P = L.probs[p];
    const IterState& it = L.its[p];
    if (it.done) continue;
    const int32_t k_iter = it.iter + 1;
    if (!P.infinite && k_iter > P.horizon) continue;
    if (p != cur_p) {
      if (cur_p >= 0 && run_max && lane == 0 && L.probs[cur_p].infinite)
        atomicMax(&L.its[cur_p].resmax, run_max);
      cur_p = p;
      run_max = 0;
    }
    const int32_t s = g - (L.count == 1 ? 0 : __ldg(L.state_base + p));
    const uint64_t* __restrict__ Vin = P.V[(k_iter - 1) & 1];
    uint64_t* __restrict__ Vout = P.V[k_iter & 1];
    const uint8_t fx = P.fixed ? P.fixed[s] : 0;
    uint64_t vnew;
    int32_t best = -1;
    if (fx == 1) {
      vnew = kOne;
    } else if (fx == 2) {
      vnew = 0;
    } else {
      const bool pess = P.pessimistic != 0;
      const int32_t jb = __ldg(P.stateptr + s), je = __ldg(P.stateptr + s + 1);
      uint64_t bestq = 0;
      for (int32_t j = jb; j < je; ++j) {
        const int32_t c0 = __ldg(P.colptr + j);
        const int32_t kk = __ldg(P.colptr + j + 1) - c0;
        const uint64_t rem = __ldg(P.rem + j);
        uint64_t q;
        if (kk <= 32 * E)
          q = column_q_regs<E>(P.rowval, P.lg, c0, kk, rem, Vin, pess, hist, lane);
        else
          q = column_q_stream(P.rowval, P.lg, c0, kk, rem, Vin, pess, hist, lane);
        const bool better = best < 0 || (P.maximize ? q > bestq : q < bestq);
        if (better) {
          bestq = q;
          best = j - jb;
        }
      }
      vnew = bestq >= (kOne >> 1) ? kOne : (bestq << 1);  // Q2.62 -> Q1.63, clamp at 1
    }
    if (lane == 0) {
      Vout[s] = vnew;
      if (P.policy_mode == 1)
        P.policy[(size_t)(P.horizon - k_iter) * P.n_states + s] = best;
      else if (P.policy_mode == 2)
        P.policy[s] = best;
    }
    if (P.infinite) {
      const uint64_t vold = Vin[s];
      const uint64_t d = vnew > vold ? vnew - vold : vold - vnew;
      run_max = d > run_max ? d : run_max;
    }
  }
  if (cur_p >= 0 && run_max && lane == 0 && L.probs[cur_p].infinite) atomicMax(&L.its[cur_p].resmax, run_max);

  // The last block to finish advances every running problem's iteration state.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(&L.ctl->finished, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int p = threadIdx.x; p < L.count; p += blockDim.x) {
    IterState* it = &L.its[p];
    const Problem& P = L.probs[p];
    if (it->done) continue;
    const int32_t k_iter = it->iter + 1;
    if (!P.infinite && k_iter > P.horizon) {  // horizon 0: nothing ran
      it->done = 1;
      it->k_final = it->iter;
      continue;
    }
    it->iter = k_iter;
    if (P.infinite) {
      const unsigned long long r = it->resmax;
      it->resmax = 0;
      if (r < P.eps_fix) {
        it->done = 1;
        it->k_final = k_iter;
      } else if (k_iter >= P.horizon) {
        it->done = 1;
        it->k_final = k_iter;
        it->noconv = 1;
      }
    } else if (k_iter >= P.horizon) {
      it->done = 1;
      it->k_final = k_iter;
    }
  }
  if (threadIdx.x == 0) L.ctl->finished = 0;
}

}  // namespace

int choose_col_class(int32_t max_col) {
  if (max_col <= 32) return 1;
  if (max_col <= 64) return 2;
  if (max_col <= 128) return 4;
  if (max_col <= 256) return 8;
  return 16;
}

int bellman_grid(int total_states, int col_class) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = col_class >= 16 ? 2 : (col_class >= 8 ? 3 : 4);
  const int want = (total_states + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int cap = sms * per_sm * 8;  // a few waves of resident blocks
  return want < cap ? (want > 0 ? want : 1) : cap;
}

cudaError_t launch_bellman_step(const StepLaunch& L, int grid, cudaStream_t st) {
  switch (L.col_class) {
    case 1: bellman_step_kernel<1><<<grid, kThreads, 0, st>>>(L); break;
    case 2: bellman_step_kernel<2><<<grid, kThreads, 0, st>>>(L); break;
    case 4: bellman_step_kernel<4><<<grid, kThreads, 0, st>>>(L); break;
    case 8: bellman_step_kernel<8><<<grid, kThreads, 0, st>>>(L); break;
    default: bellman_step_kernel<16><<<grid, kThreads, 0, st>>>(L); break;
  }
  return cudaGetLastError();
}

}  // namespace imdp
