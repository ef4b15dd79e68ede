// Host-to-host decoding with copy/compute overlap: recoil_pipeline_*.
//
// The streams are cut into groups of about equal output bytes; each group has
// its own plan and its own region of the workspace and of the device staging
// buffer. At creation each group's words, table numbers and tables are laid
// out in one page-locked image of its workspace region, so a run copies a
// group in with two copies (that image and the descriptors), and copies its
// symbols out with one copy per run of members whose host buffers follow
// each other (the staging packs the outputs back to back). One run queues,
// per group g,
//   copy-in stream:  descriptors, tables and words of g (page-locked sources)
//   compute stream:  the persistent decode of g, after g's copy-in
//   copy-out stream: the decoded symbols of g to the caller's host buffers
// so group g+1 is copied in while g decodes and g-1 is copied out; the
// host<->device links in both directions and the SMs work at the same time.
// A run waits for the caller's stream before it starts and makes the
// caller's stream wait for its last copy-out. A group's regions are reused by
// the next run only after this run's decode / copy-out of that group.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "recoil_internal.h"

using namespace recoil;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Group {
  recoil_plan* plan = nullptr;
  std::vector<uint32_t> members;     // caller stream indices
  size_t ws_off = 0, ws_bytes = 0;
  size_t stage_off = 0, stage_bytes = 0;
  std::vector<size_t> out_off;       // per member, inside the group's staging
  std::vector<size_t> out_len;       // per member: bytes decoded (a run: its symbol range)
  std::vector<size_t> host_off;      // per member: where they go in the caller's buffer
  uint8_t* meta = nullptr;           // page-locked copies of the plan's descriptors and tables
  size_t meta_bytes = 0, off_meta = 0, off_outs = 0;
  uint8_t* bulk = nullptr;           // page-locked image of the bulk region (words, table numbers, tables)
  size_t bulk_bytes = 0;
  cudaEvent_t in = nullptr, dec = nullptr, out = nullptr;
  bool used = false;
  uint8_t* bound_ws = nullptr;       // workspace region the plan was last bound to
  uint8_t* bound_stage = nullptr;
};

}  // namespace

struct recoil_pipeline {
  std::vector<Group> groups;
  std::vector<std::unique_ptr<recoil_stream>> owned;   // streams combined before being cut into runs
  std::vector<size_t> out_bytes;
  size_t ws_bytes = 0, stage_bytes = 0;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t start = nullptr, end = nullptr;

  ~recoil_pipeline() {
    for (cudaStream_t s : {s_in, s_comp, s_out})
      if (s) cudaStreamSynchronize(s);
    for (Group& g : groups) {
      if (g.plan) recoil_plan_free(g.plan);
      if (g.meta) cudaFreeHost(g.meta);
      if (g.bulk) cudaFreeHost(g.bulk);
      for (cudaEvent_t e : {g.in, g.dec, g.out})
        if (e) cudaEventDestroy(e);
    }
    for (cudaStream_t s : {s_in, s_comp, s_out})
      if (s) cudaStreamDestroy(s);
    if (start) cudaEventDestroy(start);
    if (end) cudaEventDestroy(end);
  }
};

extern "C" {

int recoil_pipeline_create(const recoil_stream* const* streams, uint32_t count, const recoil_batch_opts* opts,
                           uint32_t groups, recoil_pipeline** out) {
  clear_error();
  if (!out || (count && !streams)) return fail(RECOIL_EINVAL, "null argument");
  *out = nullptr;
  if (groups < 1) groups = 8;
  try {
    std::unique_ptr<recoil_pipeline> P(new recoil_pipeline());
    P->out_bytes.resize(count);
    uint64_t total = 0;
    for (uint32_t i = 0; i < count; i++) {
      if (!streams[i]) return fail(RECOIL_EINVAL, "null stream");
      P->out_bytes[i] = streams[i]->n_syms * streams[i]->sym_bytes;
      total += P->out_bytes[i];
    }
    // Streams of more than total / groups output bytes are cut into runs of
    // splits (shard plans: each run decodes a contiguous symbol range and
    // stages only the words it reads), one group per run; the other streams
    // form contiguous groups of about total / groups output bytes.
    const uint64_t share = std::max<uint64_t>(1, (total + groups - 1) / groups);
    recoil_batch_opts run_opts{};
    if (opts) run_opts = *opts;
    run_opts.split_symbols = 0;
    uint64_t acc = 0;
    bool group_open = false;
    cudaError_t e = cudaSuccess;
    for (uint32_t i = 0; i < count; i++) {
      const recoil_stream* s = streams[i];
      const uint64_t runs = P->out_bytes[i] / share;
      if (runs < 2) {
        if (!group_open) {
          P->groups.emplace_back();
          group_open = true;
          acc = 0;
        }
        Group& G = P->groups.back();
        G.members.push_back(i);
        G.out_len.push_back(P->out_bytes[i]);
        G.host_off.push_back(0);
        acc += P->out_bytes[i];
        if (acc >= share) group_open = false;
        continue;
      }
      group_open = false;
      const recoil_stream* src = s;
      if (opts && opts->split_symbols) {
        // the split size the caller asked for, rounded to whole CTAs, before cutting into runs
        const uint32_t w = opts->warps_per_cta ? opts->warps_per_cta : 8;
        uint64_t want = std::max<uint64_t>(1, (s->n_syms + opts->split_symbols - 1) / opts->split_symbols);
        want = (want + w - 1) / w * w;
        recoil_stream* c = nullptr;
        int rc = recoil_combine_splits(s, (uint32_t)std::min<uint64_t>(want, 0xffffffffu), &c);
        if (rc) return rc;
        P->owned.emplace_back(c);
        src = c;
      }
      for (uint64_t r = 0; r < runs; r++) {
        Group G;
        uint64_t lo = 0, hi = 0;
        int rc = recoil_plan_create_shard(src, (uint32_t)runs, (uint32_t)r, &run_opts, &G.plan, &lo, &hi);
        if (rc) return rc;
        G.members.push_back(i);
        G.out_len.push_back((hi - lo) * s->sym_bytes);
        G.host_off.push_back(lo * s->sym_bytes);
        P->groups.push_back(std::move(G));
      }
    }
    for (Group& G : P->groups) {
      if (!G.plan) {
        std::vector<const recoil_stream*> sub;
        for (uint32_t i : G.members) sub.push_back(streams[i]);
        int rc = recoil_plan_create(sub.data(), (uint32_t)sub.size(), opts, &G.plan);
        if (rc) return rc;
      }
      recoil_plan_workspace_size(G.plan, &G.ws_bytes);
      G.ws_off = P->ws_bytes;
      P->ws_bytes += align_up(G.ws_bytes, kAlign);
      G.stage_off = P->stage_bytes;
      for (size_t k = 0; k < G.members.size(); k++) {   // back to back, each on its element size
        G.stage_bytes = align_up(G.stage_bytes, streams[G.members[k]]->sym_bytes);
        G.out_off.push_back(G.stage_bytes);
        G.stage_bytes += G.out_len[k];
      }
      G.stage_bytes = align_up(std::max<size_t>(1, G.stage_bytes), kAlign);
      P->stage_bytes += G.stage_bytes;
      PlanImage img;
      plan_image(G.plan, &img);
      G.meta_bytes = img.meta_bytes;
      G.off_meta = plan_bulk_bytes(G.plan);
      G.off_outs = img.off_outs;
      G.bulk_bytes = plan_bulk_bytes(G.plan);
      if (e == cudaSuccess) e = cudaHostAlloc((void**)&G.meta, std::max<size_t>(1, G.meta_bytes), cudaHostAllocDefault);
      if (e == cudaSuccess) e = cudaHostAlloc((void**)&G.bulk, std::max<size_t>(1, G.bulk_bytes), cudaHostAllocDefault);
      if (e != cudaSuccess) break;
      std::memcpy(G.meta, img.meta, G.meta_bytes);
      plan_bulk_image(G.plan, G.bulk);
      for (cudaEvent_t* ev : {&G.in, &G.dec, &G.out})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    for (cudaStream_t* s : {&P->s_in, &P->s_comp, &P->s_out})
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->end, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(RECOIL_ECUDA, std::string("pipeline setup: ") + cudaGetErrorString(e));
    *out = P.release();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

int recoil_pipeline_sizes(const recoil_pipeline* P, size_t* ws_bytes, size_t* staging_bytes) {
  clear_error();
  if (!P) return fail(RECOIL_EINVAL, "null argument");
  if (ws_bytes) *ws_bytes = P->ws_bytes;
  if (staging_bytes) *staging_bytes = P->stage_bytes;
  return RECOIL_OK;
}

int recoil_pipeline_run(recoil_pipeline* P, void* const* h_outs, void* d_ws, size_t ws_bytes, void* d_staging,
                        size_t staging_bytes, void* cuda_stream) {
  clear_error();
  if (!P || !d_ws || (!h_outs && !P->out_bytes.empty())) return fail(RECOIL_EINVAL, "null argument");
  if (ws_bytes < P->ws_bytes || staging_bytes < P->stage_bytes || (!d_staging && P->stage_bytes))
    return fail(RECOIL_ENOMEM, "workspace or staging buffer too small (see recoil_pipeline_sizes)");
  if (((uintptr_t)d_ws) % kAlign || ((uintptr_t)d_staging) % kAlign)
    return fail(RECOIL_EINVAL, "workspace and staging must be 256-byte aligned");
  cudaStream_t user = (cudaStream_t)cuda_stream;
  uint8_t* ws = (uint8_t*)d_ws;
  uint8_t* stage = (uint8_t*)d_staging;
  cudaError_t e = cudaEventRecord(P->start, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_in, P->start, 0);
  for (size_t gi = 0; gi < P->groups.size() && e == cudaSuccess; gi++) {
    Group& G = P->groups[gi];
    uint8_t* gws = ws + G.ws_off;
    std::vector<void*> outs(G.members.size());
    for (size_t k = 0; k < G.members.size(); k++) outs[k] = stage + G.stage_off + G.out_off[k];
    if (G.bound_stage != stage) {
      // the descriptor copy carries the output pointers, as the kernels index
      // them (a run's are shifted back to its first symbol): write them once
      // the previous copy-in from this page-locked buffer has finished
      if (G.used && (e = cudaEventSynchronize(G.in)) != cudaSuccess) break;
      std::vector<void*> dev(outs.size());
      plan_kernel_outs(G.plan, outs.data(), dev.data());
      std::memcpy(G.meta + G.off_outs, dev.data(), dev.size() * sizeof(void*));
    }
    // copy-in, once the previous run's decode of this group is done with the region
    if (G.used) e = cudaStreamWaitEvent(P->s_in, G.dec, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gws + G.off_meta, G.meta, G.meta_bytes, cudaMemcpyHostToDevice, P->s_in);
    if (e == cudaSuccess && G.bulk_bytes)
      e = cudaMemcpyAsync(gws, G.bulk, G.bulk_bytes, cudaMemcpyHostToDevice, P->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(G.in, P->s_in);
    if (e != cudaSuccess) break;
    // decode, once the copy-in is there and the previous copy-out left the staging
    // bind the plan to its region once: rebinding re-sends its output pointers,
    // a pageable copy that would stall the host behind the compute stream
    if (G.bound_ws != gws || G.bound_stage != stage) {
      int rc = plan_upload_parts(G.plan, gws, G.ws_bytes, P->s_comp, false, false);
      if (rc) return rc;
      G.bound_ws = gws;
      G.bound_stage = stage;
    }
    int rc = RECOIL_OK;
    e = cudaStreamWaitEvent(P->s_comp, G.in, 0);
    if (e == cudaSuccess && G.used) e = cudaStreamWaitEvent(P->s_comp, G.out, 0);
    if (e != cudaSuccess) break;
    rc = recoil_plan_decode(G.plan, outs.data(), P->s_comp);
    if (rc) return rc;
    e = cudaEventRecord(G.dec, P->s_comp);
    // copy-out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_out, G.dec, 0);
    for (size_t k = 0; k < G.members.size() && e == cudaSuccess;) {
      // one copy for each run of members that follow each other on both sides
      uint8_t* dst = (uint8_t*)h_outs[G.members[k]] + G.host_off[k];
      size_t bytes = G.out_len[k], j = k + 1;
      while (j < G.members.size()) {
        if ((uint8_t*)h_outs[G.members[j]] + G.host_off[j] != dst + bytes || G.out_off[j] != G.out_off[k] + bytes) break;
        bytes += G.out_len[j];
        j++;
      }
      if (bytes) e = cudaMemcpyAsync(dst, outs[k], bytes, cudaMemcpyDeviceToHost, P->s_out);
      k = j;
    }
    if (e == cudaSuccess) e = cudaEventRecord(G.out, P->s_out);
    G.used = true;
  }
  if (e == cudaSuccess) e = cudaEventRecord(P->end, P->s_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, P->end, 0);
  if (e != cudaSuccess) return fail(RECOIL_ECUDA, std::string("pipeline run: ") + cudaGetErrorString(e));
  return RECOIL_OK;
}

int recoil_pipeline_errors(recoil_pipeline* P, uint32_t* flags) {
  clear_error();
  if (!P || !flags) return fail(RECOIL_EINVAL, "null argument");
  *flags = 0;
  for (Group& G : P->groups) {
    uint32_t f = 0;
    int rc = recoil_plan_errors(G.plan, P->s_comp, &f);
    *flags |= f;
    if (rc && rc != RECOIL_ECORRUPT) return rc;
  }
  if (*flags) return fail(RECOIL_ECORRUPT, "decoder found an inconsistent stream");
  return RECOIL_OK;
}

void recoil_pipeline_free(recoil_pipeline* P) { delete P; }

}  // extern "C"
