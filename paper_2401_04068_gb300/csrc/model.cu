// Model creation: copy CSC arrays to the device, check feasibility of every
// column (Sec. 2: 0 <= P_lo <= P_up <= 1 and sum P_lo <= 1 <= sum P_up) and
// convert the bounds to the kernels' Q1.63 fixed point as (lower, gap) pairs
// plus rem = 1 - sum(lower) per column (the quantities of the O-maximization
// procedure, Sec. 4; the paper also stores lower and gap, Sec. 5).
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include <atomic>

#include "imdp_internal.h"

namespace imdp {

namespace {

constexpr double kFeasTol = 1e-12;
enum : unsigned { kErrStruct = 1u, kErrInfeasible = 2u };

// Per-column word of the Bellman kernel: rem = 1 - sum(lower) in Q1.63 (0 when
// the lower bounds reach 1), with bit 63 set on top of it when 0 < rem < 2^63
// and the column's gaps add up to less than 2^64 (saturated sum `gsum`): the
// kernel then sums gaps without wrap checks.
__device__ __forceinline__ unsigned long long rem_word(unsigned long long lsum, unsigned long long gsum) {
  const unsigned long long r = lsum >= kOne ? 0ull : kOne - lsum;
  return (r > 0 && r < kOne && gsum != ~0ull) ? (r | kOne) : r;
}

// One warp per column: range/order checks of the destinations, bound checks,
// binary64 sums for the feasibility test, and the fixed-point conversion.
__global__ void convert_columns_kernel(int32_t n_states, int32_t n_cols, const int32_t* __restrict__ colptr,
                                       const int32_t* __restrict__ rowval, const double* __restrict__ lower,
                                       const double* __restrict__ upper, ulonglong2* __restrict__ lg,
                                       uint64_t* __restrict__ rem, unsigned* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int32_t warps = gridDim.x * (blockDim.x >> 5);
  for (int32_t j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_cols; j += warps) {
    const int32_t a = colptr[j], b = colptr[j + 1];
    double slo = 0.0, sup = 0.0;
    unsigned long long lsum = 0, gsum = 0;
    unsigned bad = 0;
    for (int32_t i = a + lane; i < b; i += 32) {
      const int32_t r = rowval[i];
      if (r < 0 || r >= n_states) bad |= kErrStruct;
      if (i > a && rowval[i - 1] >= r) bad |= kErrStruct;
      const double lo = lower[i], up = upper[i];
      if (!(lo >= 0.0) || !(up <= 1.0) || !(lo <= up)) {
        bad |= kErrInfeasible;
        lg[i] = make_ulonglong2(0, 0);
        continue;
      }
      slo += lo;
      sup += up;
      const unsigned long long L = __double2ull_rn(lo * 9223372036854775808.0);
      const unsigned long long U = __double2ull_rn(up * 9223372036854775808.0);
      lg[i] = make_ulonglong2(L, U - L);
      gsum = gsum + (U - L) < gsum ? ~0ull : gsum + (U - L);
      const unsigned long long t = lsum + L;
      if (t < lsum) bad |= kErrInfeasible;  // sum of lower bounds far above 1
      lsum = t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      slo += __shfl_xor_sync(0xffffffffu, slo, o);
      sup += __shfl_xor_sync(0xffffffffu, sup, o);
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, lsum, o);
      if (lsum + t < lsum) bad |= kErrInfeasible;
      lsum += t;
      const unsigned long long g = __shfl_xor_sync(0xffffffffu, gsum, o);
      gsum = gsum + g < gsum ? ~0ull : gsum + g;
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
      if (slo > 1.0 + kFeasTol || sup < 1.0 - kFeasTol) bad |= kErrInfeasible;
      rem[j] = rem_word(lsum, gsum);
      if (bad) atomicOr(err, bad);
    }
  }
}

// 32-bit storage: per column, shift s = the largest value with max(upper) <
// 2^(64 - s) in Q1.63, so every bound is m * 2^(32 - s) in Q1.63 with m < 2^32
// (resolution 2^-(31 + s) in probability, i.e. ~2^-31 of the column's largest
// bound). Lower and upper are rounded to nearest, the gap is their difference,
// rem is recomputed exactly from the rounded lower bounds, and the column's
// total rounding error sum |dlower| + |dupper| is reported.
__global__ void quantize_columns_kernel(int32_t n_cols, const int32_t* __restrict__ colptr,
                                        const ulonglong2* __restrict__ lg, uint2* __restrict__ lg32,
                                        int32_t* __restrict__ shift, uint64_t* __restrict__ rem32,
                                        double* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int32_t warps = gridDim.x * (blockDim.x >> 5);
  for (int32_t j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_cols; j += warps) {
    const int32_t a = colptr[j], b = colptr[j + 1];
    unsigned long long umax = 0;
    for (int32_t i = a + lane; i < b; i += 32) {
      const unsigned long long u = lg[i].x + lg[i].y;
      umax = u > umax ? u : umax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, umax, o);
      umax = t > umax ? t : umax;
    }
    const int bl = umax ? 64 - __clzll((long long)umax) : 1;  // bit length of the largest bound
    int sh = 64 - bl;                                          // umax < 2^(64 - sh)
    sh = sh > 31 ? 31 : sh;
    const int down = 32 - sh;                                  // Q1.63 = m << down
    const unsigned long long half = 1ull << (down - 1);
    unsigned long long lsum = 0, gsum = 0;
    double e = 0.0;
    for (int32_t i = a + lane; i < b; i += 32) {
      const unsigned long long L = lg[i].x, U = lg[i].x + lg[i].y;
      unsigned long long mL = (L >> down) + (((L & ((1ull << down) - 1)) >= half) ? 1ull : 0ull);
      unsigned long long mU = (U >> down) + (((U & ((1ull << down) - 1)) >= half) ? 1ull : 0ull);
      mL = mL > 0xffffffffull ? 0xffffffffull : mL;
      mU = mU > 0xffffffffull ? 0xffffffffull : mU;
      lg32[i] = make_uint2((unsigned)mL, (unsigned)(mU - mL));
      const unsigned long long Lq = mL << down, Uq = mU << down;
      lsum += Lq;
      gsum = gsum + (Uq - Lq) < gsum ? ~0ull : gsum + (Uq - Lq);
      e += (double)(Lq > L ? Lq - L : L - Lq) + (double)(Uq > U ? Uq - U : U - Uq);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      const unsigned long long g = __shfl_xor_sync(0xffffffffu, gsum, o);
      gsum = gsum + g < gsum ? ~0ull : gsum + g;
      e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    if (lane == 0) {
      shift[j] = sh;
      rem32[j] = rem_word(lsum, gsum);
      err[j] = e / 9223372036854775808.0;
    }
  }
}

// Correction columns of 32-bit storage: a column whose rounding error is above
// the budget keeps its 64-bit bounds, copied to lgx[xoff[j] ...], and its exact
// rem word; every other column takes the 32-bit rem word (one warp per column).
__global__ void select_columns_kernel(int32_t n_cols, const int32_t* __restrict__ colptr,
                                      const ulonglong2* __restrict__ lg, const int32_t* __restrict__ xoff,
                                      ulonglong2* __restrict__ lgx, const uint64_t* __restrict__ rem32,
                                      uint64_t* __restrict__ rem) {
  const int lane = threadIdx.x & 31;
  const int32_t warps = gridDim.x * (blockDim.x >> 5);
  for (int32_t j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_cols; j += warps) {
    const int32_t x = xoff[j];
    if (x < 0) {
      if (lane == 0) rem[j] = rem32[j];
      continue;
    }
    const int32_t a = colptr[j], b = colptr[j + 1];
    for (int32_t i = a + lane; i < b; i += 32) lgx[x + (i - a)] = lg[i];
  }
}

// Address at which kernels can read the array `p` in place, or nullptr if it
// has to be copied to the device first.
const double* device_view(const double* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost) return (const double*)a.devicePointer;  // pinned, mapped
  int dev = 0, pageable = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev);
  return pageable ? p : nullptr;
}

// Staging buffer in stream order (cudaMallocAsync / cudaFreeAsync): creating a
// model never waits for work that other streams have in flight (a plain
// cudaFree would synchronize the whole device).
struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  bool alloc(size_t bytes, cudaStream_t st) {
    s = st;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    return true;
  }
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

}  // namespace

void model_destroy(DevModel* m) {
  if (!m) return;
  // the model's buffers come from the stream-ordered pool; wait for all work
  // that may still read them (what cudaFree would do) before handing them back
  cudaDeviceSynchronize();
  for (void* p : {(void*)m->stateptr, (void*)m->colptr, (void*)m->rowval, (void*)m->lg, (void*)m->rem,
                  (void*)m->tiles, (void*)m->wide, (void*)m->lg32, (void*)m->shift, (void*)m->xoff, (void*)m->lgx})
    if (p) cudaFreeAsync(p, nullptr);
  cudaStreamSynchronize(nullptr);
  slice_layout_free(m->slices);
  delete m;
}

// Device buffers of a model come from the device's default stream-ordered pool
// (cudaMallocAsync on the creating stream): unlike cudaMalloc, this never waits
// for kernels in flight (a server keeps creating models while it iterates), and
// with the pool's release threshold raised, memory of destroyed models is
// reused without being mapped again.
template <class T>
bool pool_alloc(T** p, size_t bytes, cudaStream_t st) {
  static std::atomic<bool> configured[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev].exchange(true)) {  // once per device (idempotent)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  void* q = nullptr;
  if (cudaMallocAsync(&q, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  *p = (T*)q;
  return true;
}

imdp_status model_create_csc(int32_t n_states, int32_t n_cols, int64_t nnz, const int32_t* stateptr,
                             const int32_t* colptr, const int32_t* rowval, const double* lower,
                             const double* upper, imdp_dtype dtype, cudaStream_t st, DevModel** out,
                             int32_t own0, int32_t own1, double budget) {
  TraceRange trace("imdp model create");
  if (!(budget >= 0.0)) {
    set_error("the per-iteration error budget of 32-bit storage must be >= 0");
    return IMDP_EINVAL;
  }
  if (!out) { set_error("out is NULL"); return IMDP_EINVAL; }
  *out = nullptr;
  if (own1 < 0) own1 = n_states;
  if (n_states < 1 || own0 < 0 || own1 > n_states || own0 >= own1 || n_cols < own1 - own0 || nnz < 0 ||
      nnz >= (int64_t(1) << 31)) {
    set_error("dimensions out of range (need n_states >= 1, n_cols >= owned states, 0 <= nnz < 2^31)");
    return IMDP_EINVAL;
  }
  if (!stateptr || !colptr || (nnz > 0 && (!rowval || !lower || !upper))) {
    set_error("NULL array");
    return IMDP_EINVAL;
  }
  if (dtype != IMDP_F64 && dtype != IMDP_F32) {
    set_error("dtype must be IMDP_F64 or IMDP_F32");
    return IMDP_EINVAL;
  }
  // Structure arrays are small (states + columns): check them on the host.
  std::vector<int32_t> hs(n_states + 1), hc(n_cols + 1);
  cudaError_t e;
  e = cudaMemcpyAsync(hs.data(), stateptr, sizeof(int32_t) * hs.size(), cudaMemcpyDefault, st);
  if (e != cudaSuccess) return cuda_status(e, "copy stateptr");
  e = cudaMemcpyAsync(hc.data(), colptr, sizeof(int32_t) * hc.size(), cudaMemcpyDefault, st);
  if (e != cudaSuccess) return cuda_status(e, "copy colptr");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "sync");
  if (hs[0] != 0 || hs[n_states] != n_cols) { set_error("stateptr must start at 0 and end at n_cols"); return IMDP_EINVAL; }
  for (int32_t s = 0; s < n_states; ++s) {
    const bool own = s >= own0 && s < own1;
    if (own && hs[s + 1] <= hs[s]) { set_error("every state needs at least one action (stateptr strictly increasing)"); return IMDP_EINVAL; }
    if (!own && hs[s + 1] != hs[s]) { set_error("states outside the slice carry no columns"); return IMDP_EINVAL; }
  }
  if (hc[0] != 0 || hc[n_cols] != nnz) { set_error("colptr must start at 0 and end at nnz"); return IMDP_EINVAL; }
  int32_t max_col = 0;
  for (int32_t j = 0; j < n_cols; ++j) {
    const int32_t k = hc[j + 1] - hc[j];
    if (k < 0) { set_error("colptr must be nondecreasing"); return IMDP_EINVAL; }
    max_col = std::max(max_col, k);
  }

  DevModel* m = new DevModel();
  m->n_states = n_states;
  m->own0 = own0;
  m->own1 = own1;
  m->n_cols = n_cols;
  m->nnz = nnz;
  m->max_col = max_col;
  m->dtype = dtype;
  const size_t nz = (size_t)std::max<int64_t>(nnz, 1);
  // rowval is padded to a multiple of 4 entries plus 4, so that bulk copies of
  // 16-byte-aligned windows around any entry range stay inside the allocation.
  const size_t nz_rows = ((nz + 3) & ~size_t(3)) + 4;
  const size_t ns_pad = padded_i32(n_states + 1), nc_pad = padded_i32(n_cols + 1), nr_pad = padded_u64(n_cols);
  const bool ok = pool_alloc(&m->stateptr, sizeof(int32_t) * ns_pad, st) &&
                  pool_alloc(&m->colptr, sizeof(int32_t) * nc_pad, st) &&
                  pool_alloc(&m->rowval, sizeof(int32_t) * nz_rows, st) &&
                  pool_alloc(&m->lg, sizeof(ulonglong2) * nz, st) && pool_alloc(&m->rem, sizeof(uint64_t) * nr_pad, st);
  if (!ok) {
    cudaGetLastError();
    model_destroy(m);
    set_error("device allocation failed for the model");
    return IMDP_ENOMEM;
  }
  m->bytes = sizeof(int32_t) * (ns_pad + nc_pad + nz_rows) + sizeof(ulonglong2) * nz + sizeof(uint64_t) * nr_pad;

  // Bounds: the conversion kernel reads them in place when the device can
  // (device memory, pinned host memory, and on systems where the GPU reads
  // pageable host memory, such as Grace through NVLink-C2C, any host array);
  // otherwise they are staged.
  DevBuf dlo, dup, derr;
  const double* lo_d = nnz > 0 ? device_view(lower) : lower;
  const double* up_d = nnz > 0 ? device_view(upper) : upper;
  if (!lo_d) {
    if (!dlo.alloc(sizeof(double) * nz, st)) { model_destroy(m); set_error("staging allocation failed"); return IMDP_ENOMEM; }
    lo_d = (const double*)dlo.p;
  }
  if (!up_d) {
    if (!dup.alloc(sizeof(double) * nz, st)) { model_destroy(m); set_error("staging allocation failed"); return IMDP_ENOMEM; }
    up_d = (const double*)dup.p;
  }
  if (!derr.alloc(sizeof(unsigned), st)) { model_destroy(m); set_error("allocation failed"); return IMDP_ENOMEM; }

  e = cudaMemsetAsync(m->stateptr, 0, sizeof(int32_t) * ns_pad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->colptr, 0, sizeof(int32_t) * nc_pad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->rem, 0, sizeof(uint64_t) * nr_pad, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->stateptr, hs.data(), sizeof(int32_t) * hs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->colptr, hc.data(), sizeof(int32_t) * hc.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->rowval + nnz, 0, sizeof(int32_t) * (nz_rows - nnz), st);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(m->rowval, rowval, sizeof(int32_t) * nnz, cudaMemcpyDefault, st);
  if (e == cudaSuccess && dlo.p) e = cudaMemcpyAsync(dlo.p, lower, sizeof(double) * nnz, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && dup.p) e = cudaMemcpyAsync(dup.p, upper, sizeof(double) * nnz, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr.p, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) { model_destroy(m); return cuda_status(e, "upload model"); }

  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int warps_needed = n_cols;
  int grid = std::min((warps_needed + 7) / 8, sms * 16);
  if (grid < 1) grid = 1;
  convert_columns_kernel<<<grid, 256, 0, st>>>(n_states, n_cols, m->colptr, m->rowval, lo_d, up_d, m->lg, m->rem,
                                               (unsigned*)derr.p);
  e = cudaGetLastError();
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { model_destroy(m); return cuda_status(e, "convert model"); }
  if (herr & kErrStruct) {
    model_destroy(m);
    set_error("rowval out of range or not strictly increasing within a column");
    return IMDP_EINVAL;
  }
  if (herr & kErrInfeasible) {
    model_destroy(m);
    set_error("infeasible column: need 0 <= lower <= upper <= 1 and sum lower <= 1 <= sum upper (tol 1e-12)");
    return IMDP_EINFEASIBLE;
  }
  if (dtype == IMDP_F32) {
    // Re-encode the bounds in 32 bits and drop the 64-bit copy, except for the
    // correction columns: those whose rounding error (plus the rounding of the
    // values to 32 bits) would exceed the per-iteration budget keep their exact
    // bounds in a compact 64-bit array and run the 64-bit routines.
    const size_t nz32 = ((nz + 1) & ~size_t(1)) + 2;  // padded for 16-byte bulk-copy windows
    DevBuf derr2, drem32;
    if (!pool_alloc(&m->lg32, sizeof(uint2) * nz32, st) || !pool_alloc(&m->shift, sizeof(int32_t) * nc_pad, st) ||
        !pool_alloc(&m->xoff, sizeof(int32_t) * nc_pad, st) || !derr2.alloc(sizeof(double) * n_cols, st) ||
        !drem32.alloc(sizeof(uint64_t) * std::max<size_t>(n_cols, 1), st)) {
      cudaGetLastError();
      model_destroy(m);
      set_error("device allocation failed for 32-bit storage");
      return IMDP_ENOMEM;
    }
    e = cudaMemsetAsync(m->lg32, 0, sizeof(uint2) * nz32, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->shift, 0, sizeof(int32_t) * nc_pad, st);
    if (e == cudaSuccess) {
      quantize_columns_kernel<<<grid, 256, 0, st>>>(n_cols, m->colptr, m->lg, m->lg32, m->shift,
                                                    (uint64_t*)drem32.p, (double*)derr2.p);
      e = cudaGetLastError();
    }
    std::vector<double> herrs(n_cols);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(herrs.data(), derr2.p, sizeof(double) * n_cols, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { model_destroy(m); return cuda_status(e, "32-bit storage"); }
    // per-iteration error of a 32-bit column: its rounding plus the rounding of
    // the values to 32 bits (products are exact to 2^-62, counted below)
    const double vround = std::ldexp(1.0, -32);
    std::vector<int32_t> xo(nc_pad, -1);
    int64_t xn = 0;
    double worst32 = 0.0;
    for (int32_t j = 0; j < n_cols; ++j) {
      if (herrs[j] + vround > budget) {
        xo[j] = (int32_t)xn;
        xn += hc[j + 1] - hc[j];
        ++m->n_exact;
      } else {
        worst32 = std::max(worst32, herrs[j]);
      }
    }
    if (xn >= (int64_t(1) << 31)) { model_destroy(m); set_error("too many correction entries"); return IMDP_EINVAL; }
    m->exact_entries = xn;
    m->err_bound = worst32 + vround + std::ldexp((double)m->max_col + 1.0, -62);
    m->f32_budget = budget;
    if (xn > 0 && !pool_alloc(&m->lgx, sizeof(ulonglong2) * (size_t)xn, st)) {
      cudaGetLastError();
      model_destroy(m);
      set_error("device allocation failed for the correction columns");
      return IMDP_ENOMEM;
    }
    e = cudaMemcpyAsync(m->xoff, xo.data(), sizeof(int32_t) * nc_pad, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      select_columns_kernel<<<grid, 256, 0, st>>>(n_cols, m->colptr, m->lg, m->xoff, m->lgx,
                                                  (const uint64_t*)drem32.p, m->rem);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `xo` is a host staging vector
    if (e != cudaSuccess) { model_destroy(m); return cuda_status(e, "32-bit storage"); }
    cudaFreeAsync(m->lg, st);
    m->lg = nullptr;
    if (m->n_exact == 0) {  // no correction column: nothing reads the offsets
      cudaFreeAsync(m->xoff, st);
      m->xoff = nullptr;
    } else {
      xo.resize(n_cols);
      m->h_xoff = std::move(xo);  // the tile planner stages each tile's correction entries
    }
    m->bytes = m->bytes - sizeof(ulonglong2) * nz + sizeof(uint2) * nz32 + sizeof(int32_t) * nc_pad +
               (m->xoff ? sizeof(int32_t) * nc_pad : 0) + sizeof(ulonglong2) * (size_t)xn;
  }
  m->h_stateptr = std::move(hs);
  m->h_colptr = std::move(hc);
  plan_tiles(m, 0, m->h_tiles, m->h_wide);
  m->n_tiles = (int32_t)m->h_tiles.size();
  for (const Tile& t : m->h_tiles) m->tile_cols += t.c1 - t.c0;
  m->n_wide = (int32_t)m->h_wide.size();
  std::vector<int2> wide2(m->h_wide.size());
  for (size_t i = 0; i < wide2.size(); ++i) wide2[i] = make_int2(0, m->h_wide[i]);
  if (!pool_alloc(&m->tiles, sizeof(Tile) * std::max<size_t>(m->h_tiles.size(), 1), st) ||
      !pool_alloc(&m->wide, sizeof(int2) * std::max<size_t>(wide2.size(), 1), st)) {
    cudaGetLastError();
    model_destroy(m);
    set_error("device allocation failed for the tile plan");
    return IMDP_ENOMEM;
  }
  m->bytes += sizeof(Tile) * m->h_tiles.size();
  m->bytes += sizeof(int2) * wide2.size();
  e = cudaSuccess;
  if (!m->h_tiles.empty())
    e = cudaMemcpyAsync(m->tiles, m->h_tiles.data(), sizeof(Tile) * m->h_tiles.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !wide2.empty())
    e = cudaMemcpyAsync(m->wide, wide2.data(), sizeof(int2) * wide2.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { model_destroy(m); return cuda_status(e, "upload tile plan"); }
  *out = m;
  return IMDP_OK;
}

}  // namespace imdp
