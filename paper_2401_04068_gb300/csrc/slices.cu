// Slice layout of a model: the CSC arrays of Sec. 3.1 / Appendix A rearranged so
// that one lane of a warp owns one column (the slice kernel). The plan (windows,
// column order, slice offsets) is made on the host from the model's host copy
// of its structure; one gather kernel then copies destinations and bound pairs
// into the interleaved arrays.
#include <algorithm>
#include <memory>

#include "imdp_internal.h"

namespace imdp {
namespace {

// One warp per slice: entry t of the column in slot l goes to off + 32 t + l;
// slots past a column's end (and empty slots) get destination 0 and bounds
// {0, 0}, which add nothing to any sum of the Bellman step.
template <class Pair>
__global__ void gather_slices_kernel(int32_t n_slices, const int2* __restrict__ slot,
                                     const SliceMeta* __restrict__ meta, const int32_t* __restrict__ colptr,
                                     const int32_t* __restrict__ rowval, const Pair* __restrict__ lg,
                                     int32_t* __restrict__ rows_out, Pair* __restrict__ lg_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n_slices; g += warps) {
    const SliceMeta sm = meta[g];
    const int2 sl = slot[g * 32 + lane];
    const int32_t ca = sl.x >= 0 ? colptr[sl.x] : 0;
    for (int32_t t = 0; t < sm.len; ++t) {
      const int64_t at = sm.off + (int64_t)t * 32 + lane;
      int32_t r = 0;
      Pair b{};
      if (t < sl.y) {
        r = rowval[ca + t];
        b = lg[ca + t];
      }
      rows_out[at] = r;
      lg_out[at] = b;
    }
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

void slice_layout_free(SliceLayout* l) {
  if (!l) return;
  if (l->block) cudaFree(l->block);
  delete l;
}

imdp_status model_slice_layout(DevModel* m, cudaStream_t st, const SliceLayout** out) {
  std::lock_guard<std::mutex> lk(m->slices_mu);
  if (m->slices) {
    *out = m->slices;
    return IMDP_OK;
  }
  TraceRange trace("imdp slice layout");
  const std::vector<int32_t>& sp = m->h_stateptr;
  const std::vector<int32_t>& cp = m->h_colptr;
  const std::vector<int32_t>& xo = m->h_xoff;
  const bool f32 = m->dtype == IMDP_F32;
  std::unique_ptr<SliceLayout> L(new SliceLayout());
  std::vector<int2> slot;
  std::vector<SliceMeta> meta;
  struct Col {
    int32_t k, c;  // entries in the slice arrays, column
  };
  std::vector<Col> cols;
  L->h_win_s0.push_back(m->own0);
  L->h_win_sl0.push_back(0);
  int64_t off = 0;
  int32_t s = m->own0;
  while (s < m->own1) {
    // a window: whole states, at most kSliceWindowCols columns (one state at least)
    const int32_t s0 = s;
    int32_t ncol = 0;
    while (s < m->own1 && (ncol == 0 || ncol + (sp[s + 1] - sp[s]) <= kSliceWindowCols)) {
      ncol += sp[s + 1] - sp[s];
      ++s;
    }
    cols.clear();
    for (int32_t c = sp[s0]; c < sp[s]; ++c) {
      const bool exact = !xo.empty() && xo[c] >= 0;  // read from lgx, not from the slice arrays
      cols.push_back(Col{exact ? 0 : cp[c + 1] - cp[c], c});
    }
    std::stable_sort(cols.begin(), cols.end(), [](const Col& a, const Col& b) { return a.k > b.k; });
    // a window without columns still gets one (empty) slice: its states are
    // finished by the warp that completes the window's last slice
    const size_t n = std::max<size_t>(cols.size(), 1);
    for (size_t i = 0; i < n; i += 32) {
      SliceMeta sm;
      sm.off = off;
      sm.len = 0;
      sm.pad = 0;
      for (size_t l = 0; l < 32; ++l) {
        if (i + l < cols.size()) {
          slot.push_back(make_int2(cols[i + l].c, cols[i + l].k));
          sm.len = std::max(sm.len, cols[i + l].k);
        } else {
          slot.push_back(make_int2(-1, 0));
        }
      }
      meta.push_back(sm);
      off += 32 * (int64_t)sm.len;
    }
    L->h_win_s0.push_back(s);
    L->h_win_sl0.push_back((int32_t)meta.size());
  }
  if (meta.size() >= (size_t)INT32_MAX / 32) {
    set_error("model too large for the slice layout");
    return IMDP_EINVAL;
  }
  L->n_windows = (int32_t)L->h_win_s0.size() - 1;
  L->n_slices = (int32_t)meta.size();
  L->entries = off;
  const size_t pair = f32 ? sizeof(uint2) : sizeof(ulonglong2);
  const size_t b_slot = align256(sizeof(int2) * slot.size()), b_meta = align256(sizeof(SliceMeta) * meta.size());
  const size_t b_rows = align256(sizeof(int32_t) * (size_t)off), b_lg = align256(pair * (size_t)off);
  L->bytes = b_slot + b_meta + b_rows + b_lg;
  cudaError_t e = cudaMalloc(&L->block, std::max<size_t>(L->bytes, 256));
  if (e != cudaSuccess) {
    L->block = nullptr;
    set_error("device allocation failed (slice layout)");
    return IMDP_ENOMEM;
  }
  unsigned char* b = static_cast<unsigned char*>(L->block);
  L->slot = reinterpret_cast<int2*>(b);
  L->meta = reinterpret_cast<SliceMeta*>(b + b_slot);
  L->rows = reinterpret_cast<int32_t*>(b + b_slot + b_meta);
  L->lg = b + b_slot + b_meta + b_rows;
  e = cudaMemcpyAsync(L->slot, slot.data(), sizeof(int2) * slot.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L->meta, meta.data(), sizeof(SliceMeta) * meta.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && L->n_slices > 0) {
    const int grid = (int)std::min<int64_t>(((int64_t)L->n_slices + 7) / 8, 4096);
    if (f32)
      gather_slices_kernel<uint2><<<grid, 256, 0, st>>>(L->n_slices, L->slot, L->meta, m->colptr, m->rowval, m->lg32,
                                                        L->rows, static_cast<uint2*>(L->lg));
    else
      gather_slices_kernel<ulonglong2><<<grid, 256, 0, st>>>(L->n_slices, L->slot, L->meta, m->colptr, m->rowval,
                                                             m->lg, L->rows, static_cast<ulonglong2*>(L->lg));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
  if (e != cudaSuccess) {
    cudaFree(L->block);
    L->block = nullptr;
    return cuda_status(e, "slice layout");
  }
  m->slices = L.release();
  *out = m->slices;
  return IMDP_OK;
}

}  // namespace imdp
