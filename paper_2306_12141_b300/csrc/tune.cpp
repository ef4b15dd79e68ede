// Autotuner for batched decoding: picks coder lanes a thread (one split a
// warp, or two in lockstep), warps per CTA, the split size a batch is
// combined to and, for adaptive models over up to 256 symbols, which table
// layout is staged (paired or one-byte guide), by timing each candidate on
// the caller's own streams.
//
// Candidates differ only in how streams are split, so they share the bulk of
// the device image (words and tables): it is uploaded once and each candidate
// uploads only its descriptors. Each candidate gets one warm-up decode and
// `steps` timed decodes (CUDA events on the caller's stream); the median
// decides. Results can be cached in a text file keyed by the GPU and the batch
// shape, so a serving process tunes once.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <vector>

#include "recoil_internal.h"

namespace recoil {
namespace {

const uint32_t kWarps[] = {4, 8, 16, 24, 32};
const uint32_t kSplit[] = {32768, 65536, 131072, 262144};

// Candidate options: lanes a thread (1 or 2) x warps x split sizes, or lanes
// x warps alone on the streams' own splits, every shape a kernel is built for
// with each kind in the batch, and both table layouts where an adaptive
// model has the paired one. 32-warp CTAs only where a large table leaves
// room for one CTA an SM (adaptive models, 16-bit static models); 8-bit
// static kinds keep 4 to 16.
std::vector<recoil_batch_opts> candidates(bool keep_splits, bool has_static, bool has_adaptive, bool pairable,
                                          bool wide_static) {
  std::vector<recoil_batch_opts> c;
  for (uint32_t layout : {0u, RECOIL_BATCH_NO_PAIRS}) {
    if (layout && !pairable) continue;
    for (uint32_t lanes : {1u, 2u}) {
      for (uint32_t w : kWarps) {
        if (has_static && !shape_supported(false, w, lanes)) continue;
        if (has_adaptive && !shape_supported(true, w, lanes)) continue;
        if (lanes == 1 && w == 32 && !has_adaptive && !wide_static) continue;
        const uint32_t flags = (lanes == 2 ? RECOIL_BATCH_TWO_LANES : 0) | layout;
        if (keep_splits) {
          c.push_back(recoil_batch_opts{w, 0, 0, flags});
          continue;
        }
        for (uint32_t sp : kSplit) c.push_back(recoil_batch_opts{w, 0, sp, flags});
      }
    }
  }
  return c;
}

std::string tune_key(const recoil_stream* const* s, uint32_t count) {
  int dev = 0, sms = 0;
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof prop);
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaGetDeviceProperties(&prop, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  uint64_t total = 0;
  uint32_t nmask = 0, bmask = 0;
  for (uint32_t i = 0; i < count; i++) {
    total += s[i]->n_syms * s[i]->sym_bytes;
    nmask |= 1u << (s[i]->n_bits & 31);
    bmask |= s[i]->sym_bytes;
  }
  std::ostringstream k;
  for (const char* c = prop.name; *c; c++) k << (*c == ' ' ? '_' : *c);
  k << "|sm" << sms << "|c" << (count ? (int)std::log2((double)count) : 0) << "|b"
    << (total ? (int)std::log2((double)total) : 0) << "|n" << nmask << "|s" << bmask;
  return k.str();
}

// Cache lines: key, warps, split symbols, lanes a thread, table layout (0:
// paired where a model has it, 1: one-byte guide), time (ms). Lines without
// the layout field read as layout 0.
bool cache_lookup(const char* path, const std::string& key, recoil_batch_opts* best, float* ms) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  bool hit = false;
  while (std::getline(f, line)) {
    std::istringstream in(line);
    std::string k;
    std::vector<double> v;
    double x = 0;
    if (!(in >> k) || k != key) continue;
    while (in >> x) v.push_back(x);
    if (v.size() != 4 && v.size() != 5) continue;
    const uint32_t w = (uint32_t)v[0], sp = (uint32_t)v[1], lanes = (uint32_t)v[2];
    const uint32_t layout = v.size() == 5 ? (uint32_t)v[3] : 0u;
    if ((lanes == 1 || lanes == 2) && layout <= 1 &&
        (lanes == 2 ? (w == 4 || w == 8 || w == 16 || w == 24) : warps_supported(w))) {
      *best = recoil_batch_opts{w, 0, sp, (lanes == 2 ? RECOIL_BATCH_TWO_LANES : 0u) |
                                              (layout ? RECOIL_BATCH_NO_PAIRS : 0u)};
      *ms = (float)v.back();
      hit = true;                          // the last line for a key wins
    }
  }
  return hit;
}

void cache_store(const char* path, const std::string& key, const recoil_batch_opts& b, float ms) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << ' ' << b.warps_per_cta << ' ' << b.split_symbols << ' '
    << ((b.flags & RECOIL_BATCH_TWO_LANES) ? 2 : 1) << ' ' << ((b.flags & RECOIL_BATCH_NO_PAIRS) ? 1 : 0) << ' '
    << ms << '\n';
}

struct Candidate {
  recoil_batch_opts opts;
  recoil_plan* plan = nullptr;
};

bool any_adaptive(const recoil_stream* const* s, uint32_t count) {
  for (uint32_t i = 0; i < count; i++)
    if (s && s[i] && s[i]->adaptive()) return true;
  return false;
}

bool any_static(const recoil_stream* const* s, uint32_t count) {
  for (uint32_t i = 0; i < count; i++)
    if (s && s[i] && !s[i]->adaptive()) return true;
  return false;
}

// A static model over 16-bit symbols (its tables may fill most of an SM's shared memory).
bool any_static16(const recoil_stream* const* s, uint32_t count) {
  for (uint32_t i = 0; i < count; i++)
    if (s && s[i] && !s[i]->adaptive() && s[i]->sym_bytes == 2) return true;
  return false;
}

// An adaptive model with the paired layout (one-byte guide entries: up to 256 symbols).
bool any_pairable(const recoil_stream* const* s, uint32_t count) {
  for (uint32_t i = 0; i < count; i++)
    if (s && s[i] && s[i]->adaptive() && s[i]->alphabet() <= 256) return true;
  return false;
}

}  // namespace
}  // namespace recoil

using namespace recoil;

extern "C" {

int recoil_autotune_workspace_size(const recoil_stream* const* streams, uint32_t count, size_t* bytes) {
  clear_error();
  if (!bytes) return fail(RECOIL_EINVAL, "null argument");
  size_t mx = 0;
  for (bool keep : {false, true})
    for (recoil_batch_opts o :
         candidates(keep, any_static(streams, count), any_adaptive(streams, count), any_pairable(streams, count),
                    any_static16(streams, count))) {
      size_t b = 0;
      int rc = recoil_workspace_size(streams, count, &o, &b);
      if (rc) return rc;
      mx = std::max(mx, b);
    }
  *bytes = mx;
  return RECOIL_OK;
}

int recoil_autotune(const recoil_stream* const* streams, uint32_t count, void* const* d_outs, void* d_ws,
                    size_t ws_bytes, void* cuda_stream, const recoil_tune_opts* topts, recoil_batch_opts* best,
                    float* best_ms) {
  clear_error();
  if (!best || (count && (!streams || !d_outs))) return fail(RECOIL_EINVAL, "null argument");
  const uint32_t steps = topts && topts->steps ? topts->steps : 3;
  const char* cache = topts ? topts->cache_path : nullptr;
  const bool refresh = topts && (topts->flags & RECOIL_TUNE_REFRESH);
  const bool keep = topts && (topts->flags & RECOIL_TUNE_KEEP_SPLITS);
  const std::string key = tune_key(streams, count) + (keep ? "|keep" : "");
  float ms = 0;
  recoil_batch_opts hit{};
  if (!refresh && cache_lookup(cache, key, &hit, &ms)) {
    *best = hit;
    if (best_ms) *best_ms = ms;
    return RECOIL_OK;
  }
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  std::vector<Candidate> cands;
  auto cleanup = [&]() {
    for (Candidate& c : cands) recoil_plan_free(c.plan);
  };
  size_t bulk = 0;
  for (const recoil_batch_opts& o :
       candidates(keep, any_static(streams, count), any_adaptive(streams, count), any_pairable(streams, count),
                    any_static16(streams, count))) {
    Candidate c;
    c.opts = o;
    int rc = recoil_plan_create(streams, count, &c.opts, &c.plan);
    if (rc) {
      cleanup();
      return rc;
    }
    size_t need = 0;
    recoil_plan_workspace_size(c.plan, &need);
    if (need > ws_bytes) {
      recoil_plan_free(c.plan);
      cleanup();
      return fail(RECOIL_ENOMEM, "workspace too small for tuning (see recoil_autotune_workspace_size)");
    }
    if (cands.empty()) bulk = plan_bulk_bytes(c.plan);
    if (plan_bulk_bytes(c.plan) != bulk) {
      recoil_plan_free(c.plan);
      cleanup();
      return fail(RECOIL_EINVAL, "internal: candidates disagree on the bulk layout");
    }
    cands.push_back(c);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cleanup();
    return fail(RECOIL_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
  }
  int rc = RECOIL_OK;
  float best_t = 0;
  int best_i = -1;
  for (size_t i = 0; i < cands.size() && !rc; i++) {
    rc = plan_upload_parts(cands[i].plan, d_ws, ws_bytes, cs, i == 0, true);
    if (!rc) rc = recoil_plan_decode(cands[i].plan, d_outs, cs);          // warm-up
    std::vector<float> t;
    for (uint32_t k = 0; k < steps && !rc; k++) {
      cudaEventRecord(e0, cs);
      rc = recoil_plan_decode(cands[i].plan, d_outs, cs);
      cudaEventRecord(e1, cs);
      if (!rc && (ce = cudaEventSynchronize(e1)) != cudaSuccess)
        rc = fail(RECOIL_ECUDA, std::string("tuning: ") + cudaGetErrorString(ce));
      float v = 0;
      if (!rc) cudaEventElapsedTime(&v, e0, e1);
      t.push_back(v);
    }
    if (rc) break;
    uint32_t flags = 0;
    rc = recoil_plan_errors(cands[i].plan, cuda_stream, &flags);
    std::sort(t.begin(), t.end());
    const float med = t[t.size() / 2];
    if (!rc && (best_i < 0 || med < best_t)) {
      best_t = med;
      best_i = (int)i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc && best_i >= 0) {
    *best = cands[best_i].opts;
    if (best_ms) *best_ms = best_t;
    cache_store(cache, key, *best, best_t);
  }
  cleanup();
  return rc;
}

}  // extern "C"
