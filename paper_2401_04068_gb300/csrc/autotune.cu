// Launch configuration of a session and its autotuner (no counterpart in the
// paper: the Bellman step of Eq. 2 computes the same words in every
// configuration; the configurations differ in speed only).
//
// The tuner times candidate configurations on the session itself with CUDA
// events and keeps the fastest, caching the choice in a small JSON file keyed
// by the session's shape, so that a later session of the same shape starts
// with the tuned configuration without timing anything.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
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

imdp_launch_config to_public(const LaunchConfig& c) {
  imdp_launch_config o;
  o.kernel = c.kernel;
  o.cta_warps = c.cta_warps;
  o.ctas_per_sm = c.ctas_per_sm;
  o.tile_entries = c.tile_entries;
  o.wide_col = c.wide_col;
  return o;
}

LaunchConfig from_public(const imdp_launch_config& o) {
  LaunchConfig c;
  c.kernel = o.kernel;
  c.cta_warps = o.cta_warps;
  c.ctas_per_sm = o.ctas_per_sm;
  c.tile_entries = o.tile_entries;
  c.wide_col = o.wide_col;
  return c;
}

int log2_bucket(double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); }

// Shape key of a session: storage, mean transitions per column, columns per
// state, states per problem and problems (log2 buckets), wide states present.
std::string shape_key(const Session* S) {
  int64_t nnz = 0, cols = 0, states = 0, wide = 0;
  int32_t max_col = 0;
  bool f32 = false, f64 = false;
  for (const DevModel* m : S->models) {
    nnz += m->nnz;
    cols += m->n_cols;
    states += m->n_states;
    wide += m->n_wide;
    max_col = std::max(max_col, m->max_col);
    (m->lg32 ? f32 : f64) = true;
  }
  const double k = cols ? (double)nnz / (double)cols : 0.0;
  const double a = states ? (double)cols / (double)states : 0.0;
  char buf[160];
  std::snprintf(buf, sizeof(buf), "%s|k%d|a%d|n%d|p%d|c%d|w%d", f32 && f64 ? "mixed" : (f32 ? "f32" : "f64"),
                log2_bucket(k), (int)std::lround(a * 2.0), log2_bucket((double)states / std::max(1, S->count)),
                log2_bucket((double)S->count), log2_bucket((double)max_col), wide > 0 ? 1 : 0);
  return buf;
}

// The cache file: {"key": {"kernel": 2, "cta_warps": 8, ...}, ...} as written below.
std::map<std::string, std::string> read_cache(const char* path) {
  std::map<std::string, std::string> out;
  if (!path) return out;
  FILE* f = std::fopen(path, "rb");
  if (!f) return out;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
  std::fclose(f);
  size_t i = 0;
  while (true) {
    const size_t q0 = text.find('"', i);
    if (q0 == std::string::npos) break;
    const size_t q1 = text.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    const size_t b0 = text.find('{', q1);
    const size_t b1 = b0 == std::string::npos ? b0 : text.find('}', b0);
    if (b1 == std::string::npos) break;
    out[text.substr(q0 + 1, q1 - q0 - 1)] = text.substr(b0, b1 - b0 + 1);
    i = b1 + 1;
  }
  return out;
}

bool field(const std::string& body, const char* name, double* v) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t at = body.find(pat);
  if (at == std::string::npos) return false;
  return std::sscanf(body.c_str() + at + pat.size(), "%lf", v) == 1;
}

bool parse_entry(const std::string& body, LaunchConfig* c) {
  double k, w, p, t, wc;
  if (!field(body, "kernel", &k) || !field(body, "cta_warps", &w) || !field(body, "ctas_per_sm", &p) ||
      !field(body, "tile_entries", &t) || !field(body, "wide_col", &wc))
    return false;
  c->kernel = (int32_t)k;
  c->cta_warps = (int32_t)w;
  c->ctas_per_sm = (int32_t)p;
  c->tile_entries = (int32_t)t;
  c->wide_col = (int32_t)wc;
  return true;
}

bool write_cache(const char* path, const std::map<std::string, std::string>& entries) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  std::fputs("{\n", f);
  size_t i = 0;
  for (const auto& kv : entries) {
    std::fprintf(f, "  \"%s\": %s%s\n", kv.first.c_str(), kv.second.c_str(), ++i < entries.size() ? "," : "");
  }
  std::fputs("}\n", f);
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path) == 0;
}

std::string entry_body(const LaunchConfig& c, double ms) {
  char buf[256];
  std::snprintf(buf, sizeof(buf),
                "{\"kernel\": %d, \"cta_warps\": %d, \"ctas_per_sm\": %d, \"tile_entries\": %d, \"wide_col\": %d, "
                "\"ms_per_iter\": %.6f}",
                c.kernel, c.cta_warps, c.ctas_per_sm, c.tile_entries, c.wide_col, ms);
  return buf;
}

// Time one configuration: reset + `iters` steps, once untimed, then timed.
imdp_status time_config(Session* S, const LaunchConfig& c, int32_t iters, cudaStream_t st, cudaEvent_t e0,
                        cudaEvent_t e1, double* ms) {
  imdp_status r = S->set_launch(c, st);
  if (r != IMDP_OK) return r;
  float best = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    if ((r = S->reset(st)) != IMDP_OK) return r;
    cudaError_t e = cudaEventRecord(e0, st);
    if (e != cudaSuccess) return cuda_status(e, "autotune");
    if ((r = S->step(iters, st)) != IMDP_OK) return r;
    if ((e = cudaEventRecord(e1, st)) == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) return cuda_status(e, "autotune");
    best = t;  // the second (timed) run is kept
  }
  std::vector<IterState> its;
  if ((r = S->read_states(its, st)) != IMDP_OK) return r;  // a bounded wait that gave up fails the tuning
  *ms = (double)best / std::max(1, iters);
  return IMDP_OK;
}

}  // namespace

extern "C" {

IMDP_API imdp_status imdp_session_set_launch(imdp_session* s, const imdp_launch_config* cfg, void* stream) {
  set_error("");
  if (!s || !s->s || !cfg) { set_error("NULL session or configuration"); return IMDP_EINVAL; }
  if (cfg->kernel < 0 || cfg->kernel > 4 || cfg->tile_entries < 0 || cfg->wide_col < 0) {
    set_error("bad launch configuration");
    return IMDP_EINVAL;
  }
  if (cfg->kernel == kKernelTiny && !s->s->L.tiny_ok) {
    set_error("the single-CTA kernel runs one problem of at most 1024 states, 1024 columns and 4096 transitions");
    return IMDP_EINVAL;
  }
  DeviceScope g(s->s->device);
  return s->s->set_launch(from_public(*cfg), (cudaStream_t)stream);
}

IMDP_API imdp_status imdp_session_get_launch(const imdp_session* s, imdp_launch_config* cfg) {
  set_error("");
  if (!s || !s->s || !cfg) { set_error("NULL session or configuration"); return IMDP_EINVAL; }
  *cfg = to_public(resolve_launch(s->s->L, &s->s->cfg));
  return IMDP_OK;
}

IMDP_API imdp_status imdp_session_plan(const imdp_session* s, int32_t* n_tiles, int32_t* n_wide,
                                      int64_t* wide_entries) {
  set_error("");
  if (!s || !s->s) { set_error("NULL session"); return IMDP_EINVAL; }
  if (n_tiles) *n_tiles = s->s->n_tiles;
  if (n_wide) *n_wide = s->s->n_wide;
  if (wide_entries) *wide_entries = s->s->wide_entries;
  return IMDP_OK;
}

IMDP_API imdp_status imdp_session_autotune(imdp_session* s, int32_t iters, const char* cache_path, void* stream,
                                           imdp_launch_config* chosen, double* ms_per_iter) {
  set_error("");
  if (!s || !s->s) { set_error("NULL session"); return IMDP_EINVAL; }
  if (iters < 1) { set_error("iters must be >= 1"); return IMDP_EINVAL; }
  Session* S = s->s;
  DeviceScope g(S->device);
  const cudaStream_t st = (cudaStream_t)stream;
  const std::string key = shape_key(S);
  std::map<std::string, std::string> cache = read_cache(cache_path);
  LaunchConfig best;
  double best_ms = 0.0;
  imdp_status r = IMDP_OK;
  auto it = cache.find(key);
  if (it != cache.end() && parse_entry(it->second, &best)) {
    r = S->set_launch(best, st);
  } else {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      return cuda_status(e, "autotune events");
    }
    int32_t max_col = 0;
    bool wide_default = false;
    for (const DevModel* m : S->models) {
      max_col = std::max(max_col, m->max_col);
      wide_default = wide_default || m->n_wide > 0;
    }
    // stage 1: kernel and CTA shape on the default tile plan
    std::vector<LaunchConfig> cands;
    auto add = [&](int32_t kernel, int32_t warps, int32_t per_sm, int32_t te, int32_t wc) {
      LaunchConfig c;
      c.kernel = kernel;
      c.cta_warps = warps;
      c.ctas_per_sm = per_sm;
      c.tile_entries = te;
      c.wide_col = wc;
      cands.push_back(c);
    };
    if (S->L.tiny_ok) add(kKernelTiny, 0, 0, kTileEntries, kWideCol);
    add(kKernelRing, 16, 1, kTileEntries, kWideCol);
    if (!wide_default) add(kKernelRing, 24, 1, kTileEntries, kWideCol);
    add(kKernelDirect, kDirectWarps, 4, kTileEntries, kWideCol);
    add(kKernelDirect, kDirectWarps, 3, kTileEntries, kWideCol);
    add(kKernelDirect, kDirectWarps, 4, 1024, kWideCol);
    add(kKernelDirect, kDirectWarps, 3, 1024, kWideCol);
    add(kKernelSlice, kSliceWarps, 4, kTileEntries, kWideCol);
    add(kKernelSlice, kSliceWarps, 3, kTileEntries, kWideCol);
    bool have = false;
    for (const LaunchConfig& c : cands) {
      double ms = 0.0;
      if ((r = time_config(S, c, iters, st, e0, e1, &ms)) != IMDP_OK) break;
      if (!have || ms < best_ms) {
        best = c;
        best_ms = ms;
        have = true;
      }
    }
    // stage 2: the wide-state threshold, for models with long columns
    if (r == IMDP_OK && max_col >= 640 && best.kernel != kKernelTiny && best.kernel != kKernelSlice) {
      for (int32_t wc : {640, 2560, 1 << 30}) {
        LaunchConfig c = best;
        c.wide_col = wc;
        if (c.kernel == kKernelRing && c.cta_warps == 24) c.cta_warps = 16;  // wide states may appear
        double ms = 0.0;
        if ((r = time_config(S, c, iters, st, e0, e1, &ms)) != IMDP_OK) break;
        if (ms < best_ms) {
          best = c;
          best_ms = ms;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r == IMDP_OK) r = S->set_launch(best, st);
    if (r == IMDP_OK && cache_path) {
      cache[key] = entry_body(best, best_ms);
      if (!write_cache(cache_path, cache)) {
        set_error(std::string("autotune: cannot write the cache file ") + cache_path);
        r = IMDP_EIO;
      }
    }
  }
  if (r == IMDP_OK) r = S->reset(st);
  if (r == IMDP_OK || r == IMDP_EIO) {
    if (chosen) *chosen = to_public(resolve_launch(S->L, &S->cfg));
    if (ms_per_iter) *ms_per_iter = best_ms;
  }
  return r;
}

}  // extern "C"
