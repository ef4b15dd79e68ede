// Serving runtime: continuous batching of decode requests on one GPU.
//
// A pool of encoded streams (the content a server holds) is made resident once:
// its words and decoder tables are uploaded into the caller's arena. Requests
// (a pool stream and an arrival time) are replayed in real time. The loop
//   - retires finished launches (device events) and frees their memory,
//   - admits arrived requests in FIFO order while the device-memory budget and
//     a launch slot allow, up to max_batch per launch (8 x max_batch when
//     more than max_batch have arrived and wait),
//   - combines each admitted stream to its share of the warp slots that are
//     free at that moment (Sec. 3.3: the decoder's parallelism decides the
//     split count) by picking entries of the pool stream, whose descriptors
//     are built and made resident once for the whole pool before the run,
//     sends one 16-byte reference per kept split to the slot's descriptor
//     area, expands them there into descriptors on the device and launches
//     one persistent decode for the whole admission on the slot's own CUDA
//     stream,
// so requests that arrive while others run are admitted as memory and slots
// free up, and their decodes overlap on the device. Latency is arrival to the
// device completion of the launch that carried the request.
//
// With RECOIL_SERVE_PER_REQUEST the same loop is the per-stream baseline: one
// launch per request with every encoded split, one slot, FIFO.
//
// All waits are bounded by opts->timeout_s (host wall clock); kernels have no
// waits of their own.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "recoil_internal.h"

namespace recoil {
namespace {

constexpr size_t kAlign = 256;
// A launch slot's descriptor area, and how many max_batch a backlog admission
// may take. Measured at a saturating load (20 000 requests at once, the batch
// pool): 4 MiB / 4x 429-459 GB/s, 16 MiB / 8x 564-582, 16 MiB / 16x 592-629
// but with p99 outliers above 1 ms at 10k-20k req/s; 16 MiB / 8x kept.
constexpr size_t kDefaultMeta = (size_t)16 << 20;
constexpr size_t kBacklogBatches = 8;   // admission size under a backlog, in max_batch
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

double now_s() {
  using C = std::chrono::steady_clock;
  return std::chrono::duration<double>(C::now().time_since_epoch()).count();
}

// Bytes of the resident descriptor set: every entry of every pool stream and
// its final-state entry.
size_t pool_desc_bytes(const recoil_stream* const* pool, uint32_t pool_count) {
  uint64_t n = 0;
  for (uint32_t i = 0; i < pool_count; i++) n += pool[i]->entries.size() + 1;
  return align_up(n * sizeof(DevEntry), kAlign);
}

// First-fit allocator over [0, size) of the output heap (offsets only).
class Heap {
 public:
  explicit Heap(size_t size) { free_[0] = size; }
  bool alloc(size_t n, size_t* off) {
    n = align_up(std::max<size_t>(n, 1), 512);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = align_up(std::max<size_t>(n, 1), 512);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
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
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint8_t* host = nullptr;          // pinned staging of the descriptors
  uint8_t* dev = nullptr;           // descriptor area in the arena
  bool busy = false;
  std::vector<uint32_t> reqs;       // requests carried by the current launch
  std::vector<size_t> out_off;      // their heap offsets (when the heap is used)
  uint32_t warps_used = 0;
  uint32_t launch_id = 0;
};

}  // namespace
}  // namespace recoil

using namespace recoil;

extern "C" {

int recoil_serve_arena_size(const recoil_stream* const* pool, uint32_t pool_count, const recoil_serve_opts* opts,
                            size_t* bytes) {
  clear_error();
  if (!pool || !opts || !bytes) return fail(RECOIL_EINVAL, "null argument");
  recoil_plan* P = nullptr;
  recoil_batch_opts bo{opts->warps_per_cta ? opts->warps_per_cta : 8, 0, 0xffffffffu, 0};
  int rc = recoil_plan_create(pool, pool_count, &bo, &P);
  if (rc) return rc;
  const size_t bulk = plan_bulk_bytes(P);
  recoil_plan_free(P);
  const uint32_t slots = opts->max_inflight ? opts->max_inflight : 8;
  const size_t meta = opts->meta_bytes ? opts->meta_bytes : kDefaultMeta;
  *bytes = align_up(bulk, kAlign) + pool_desc_bytes(pool, pool_count) + slots * align_up(meta, kAlign) +
           align_up(opts->budget_bytes, kAlign);
  return RECOIL_OK;
}

int recoil_serve(const recoil_stream* const* pool, uint32_t pool_count, const uint32_t* req_stream,
                 const double* req_arrival_s, uint32_t n_req, void* d_arena, size_t arena_bytes,
                 void* const* d_req_outs, const recoil_serve_opts* opts, recoil_request_result* results,
                 recoil_serve_stats* stats) {
  clear_error();
  if (!pool || !opts || !d_arena || (n_req && (!req_stream || !req_arrival_s || !results)))
    return fail(RECOIL_EINVAL, "null argument");
  for (uint32_t r = 0; r < n_req; r++)
    if (req_stream[r] >= pool_count) return fail(RECOIL_EINVAL, "request names a stream outside the pool");
  const bool per_request = opts->flags & RECOIL_SERVE_PER_REQUEST;
  const uint32_t warps = opts->warps_per_cta ? opts->warps_per_cta : (per_request ? 4 : 8);
  const uint32_t nslots = per_request ? 1 : (opts->max_inflight ? opts->max_inflight : 8);
  const uint32_t max_batch = per_request ? 1 : (opts->max_batch ? opts->max_batch : 64);
  const size_t meta_cap = align_up(opts->meta_bytes ? opts->meta_bytes : kDefaultMeta, kAlign);
  const double timeout = opts->timeout_s > 0 ? opts->timeout_s : 60.0;
  const uint64_t max_split = opts->max_split_symbols ? opts->max_split_symbols : 131072;
  if (!warps_supported(warps)) return fail(RECOIL_EINVAL, "warps_per_cta must be 1, 2, 4, 8, 16 or 32");

  // resident pool: words and tables of every pool stream, uploaded once
  recoil_plan* poolplan = nullptr;
  recoil_batch_opts bo{warps, 0, 0xffffffffu, 0};   // only its words/tables layout is used: keep entries few
  int rc = recoil_plan_create(pool, pool_count, &bo, &poolplan);
  if (rc) return rc;
  std::unique_ptr<recoil_plan, void (*)(recoil_plan*)> pool_guard(poolplan, recoil_plan_free);
  PlanImage img;
  plan_image(poolplan, &img);
  const size_t bulk = align_up(plan_bulk_bytes(poolplan), kAlign);
  const size_t descs = pool_desc_bytes(pool, pool_count);
  const size_t need = bulk + descs + nslots * meta_cap + (d_req_outs ? 0 : align_up(opts->budget_bytes, kAlign));
  if (arena_bytes < need) return fail(RECOIL_ENOMEM, "arena smaller than recoil_serve_arena_size");
  if (((uintptr_t)d_arena) % kAlign) return fail(RECOIL_EINVAL, "arena must be 256-byte aligned");
  uint8_t* arena = (uint8_t*)d_arena;
  std::vector<DevStream> pool_ds(pool_count);
  std::memcpy(pool_ds.data(), img.meta + img.off_streams, pool_count * sizeof(DevStream));
  uint32_t kind_smem[kKinds];
  for (uint32_t k = 0; k < kKinds; k++) kind_smem[k] = (img.kind_smem[k] + 15) / 16 * 16;

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(RECOIL_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  int per_sm[kKinds] = {};
  for (uint32_t k = 0; k < kKinds; k++)
    if (occupancy_ctas_per_sm(k, warps, 1, img.kind_staged[k] != 0, kind_smem[k], &per_sm[k]) != 0 || per_sm[k] <= 0)
      per_sm[k] = 1;
  const uint32_t total_warps = (uint32_t)(per_sm[kPacked8] * sms) * warps;

  std::vector<Slot> slots(nslots);
  cudaEvent_t t0ev = nullptr;
  auto cleanup = [&]() {
    for (Slot& s : slots) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      if (s.done) cudaEventDestroy(s.done);
      if (s.stream) cudaStreamDestroy(s.stream);
      if (s.host) cudaFreeHost(s.host);
    }
    if (t0ev) cudaEventDestroy(t0ev);
  };
  for (uint32_t i = 0; i < nslots && e == cudaSuccess; i++) {
    e = cudaStreamCreateWithFlags(&slots[i].stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&slots[i].done);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&slots[i].host, meta_cap + sizeof(DevControl), cudaHostAllocDefault);
    slots[i].dev = arena + bulk + descs + i * meta_cap;
  }
  if (e == cudaSuccess) e = cudaEventCreate(&t0ev);
  if (e == cudaSuccess) rc = plan_upload_parts(poolplan, arena, arena_bytes, slots[0].stream, true, false);
  if (e == cudaSuccess && !rc) e = cudaStreamSynchronize(slots[0].stream);
  if (e != cudaSuccess || rc) {
    cleanup();
    return rc ? rc : fail(RECOIL_ECUDA, std::string("serve setup: ") + cudaGetErrorString(e));
  }
  uint8_t* heap_base = arena + bulk + descs + nslots * meta_cap;
  Heap heap(d_req_outs ? 0 : opts->budget_bytes);
  size_t budget_used = 0;                         // with caller outputs: bytes of admitted outputs
  std::vector<size_t> out_bytes(n_req);
  for (uint32_t r = 0; r < n_req; r++) {
    const Stream& s = *pool[req_stream[r]];
    out_bytes[r] = s.n_syms * s.sym_bytes;
    if (align_up(out_bytes[r], 512) > opts->budget_bytes) {
      cleanup();
      return fail(RECOIL_EINVAL, "a request's output alone exceeds the device-memory budget");
    }
  }

  // every entry descriptor of every pool stream, built once and made resident
  // like the words (a server prepares its content before it takes requests);
  // pool stream i's descriptors start at pool_first[i], its final-state entry last
  std::vector<uint64_t> pool_first(pool_count + 1, 0);
  std::vector<uint32_t> pool_hi1;                        // each resident descriptor's owned end
  {
    std::vector<DevEntry> flat, one;
    try {
      for (uint32_t i = 0; i < pool_count; i++) {
        one.clear();                                       // build_entries appends
        build_entries(*pool[i], 0, one);
        pool_first[i] = flat.size();
        flat.insert(flat.end(), one.begin(), one.end());
      }
    } catch (const std::bad_alloc&) {
      cleanup();
      return fail(RECOIL_ENOMEM, "host allocation failed");
    }
    pool_first[pool_count] = flat.size();
    if (flat.size() > 0xffffffffull) {
      cleanup();
      return fail(RECOIL_EINVAL, "the pool holds more than 2^32 split descriptors");
    }
    try {
      pool_hi1.resize(flat.size());
    } catch (const std::bad_alloc&) {
      cleanup();
      return fail(RECOIL_ENOMEM, "host allocation failed");
    }
    for (size_t x = 0; x < flat.size(); x++) pool_hi1[x] = flat[x].hi1;
    e = cudaMemcpy(arena + bulk, flat.data(), flat.size() * sizeof(DevEntry), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cleanup();
      return fail(RECOIL_ECUDA, std::string("serve setup: ") + cudaGetErrorString(e));
    }
  }
  const DevEntry* pool_dev = reinterpret_cast<const DevEntry*>(arena + bulk);

  // the run clock: host t0 and a device event recorded at the same moment
  e = cudaEventRecord(t0ev, slots[0].stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(t0ev);
  const double t0 = now_s();
  uint32_t next = 0, done = 0, launches = 0, inflight = 0, max_inflight_seen = 0;
  uint32_t warps_busy = 0;
  double first_arrival = n_req ? req_arrival_s[0] : 0.0, last_done = 0.0;
  uint64_t sym_bytes_total = 0;
  std::vector<DevItem> items;
  std::vector<uint32_t> item_kind;
  std::vector<std::vector<uint32_t>> keeps;     // per admitted request: its kept regular entries
  std::vector<size_t> ent_first;                // per admitted request: its first descriptor
  std::vector<uint32_t> memo_target(pool_count, 0);                 // per pool stream: its last combine
  std::vector<std::vector<uint32_t>> memo_keep(pool_count);
  int status = RECOIL_OK;

  while (done < n_req && e == cudaSuccess && status == RECOIL_OK) {
    bool progressed = false;
    // retire finished launches
    for (Slot& sl : slots) {
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        e = q;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, t0ev, sl.done);
      const double t_done = ms * 1e-3;
      DevControl ctl;                              // copied back behind the kernel on the slot stream
      std::memcpy(&ctl, sl.host + meta_cap, sizeof ctl);
      if (ctl.errors) status = fail(RECOIL_ECORRUPT, "decoder found an inconsistent stream while serving");
      for (size_t k = 0; k < sl.reqs.size(); k++) {
        const uint32_t r = sl.reqs[k];
        results[r].done_s = t_done;
        if (!d_req_outs) heap.release(sl.out_off[k], out_bytes[r]);
        else budget_used -= align_up(out_bytes[r], 512);
        last_done = std::max(last_done, t_done);
        done++;
      }
      warps_busy -= sl.warps_used;
      sl.busy = false;
      inflight--;
      progressed = true;
    }
    if (e != cudaSuccess) break;
    const double t = now_s() - t0;
    if (t > timeout) {
      status = fail(RECOIL_ETIMEOUT, "serving run exceeded its time limit");
      break;
    }
    // admit arrived requests into a free slot
    Slot* free_slot = nullptr;
    for (Slot& sl : slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (free_slot && next < n_req && req_arrival_s[next] <= t) {
      Slot& sl = *free_slot;
      sl.reqs.clear();
      sl.out_off.clear();
      uint64_t syms_batch = 0;
      // a backlog (more arrived requests than one launch takes) is admitted
      // up to 8 x max_batch at once: the free warps are shared by more
      // requests, so each gets fewer splits and the host builds fewer
      // descriptors per decoded byte; the admission stops before its
      // descriptors could outgrow the slot's area. Two bounds on its split
      // count hold: every request's encoded entries, and every free warp plus
      // each request's long-split minimum, rounding and final entry.
      const uint32_t free_w0 = total_warps > warps_busy ? total_warps - warps_busy : warps;
      uint32_t waiting = 0;
      while (next + waiting < n_req && req_arrival_s[next + waiting] <= t && waiting <= max_batch) waiting++;
      const size_t cap_n = per_request ? 1 : (waiting > max_batch ? kBacklogBatches * (size_t)max_batch : max_batch);
      uint64_t sum_entries = 0, sum_share = free_w0;
      auto meta_bound = [&](size_t n, uint64_t ents_max) {
        return sizeof(DevControl) + align_up(n * 8, kAlign) + align_up(n * sizeof(DevStream), kAlign) +
               align_up(ents_max * sizeof(DevItem), kAlign) + align_up(ents_max * sizeof(EntryRef), kAlign) +
               ents_max * sizeof(DevEntry);
      };
      while (next < n_req && req_arrival_s[next] <= t && sl.reqs.size() < cap_n) {
        const uint32_t r = next;
        const Stream& src_r = *pool[req_stream[r]];
        const uint64_t k_r = src_r.entries.size() + 1;
        const uint64_t s_r = (src_r.n_syms + max_split - 1) / max_split + warps + 1;
        const uint64_t bound = per_request ? sum_entries + k_r : std::min(sum_entries + k_r, sum_share + s_r);
        if (!sl.reqs.empty() && meta_bound(sl.reqs.size() + 1, bound) > meta_cap) break;
        size_t off = 0;
        if (!d_req_outs) {
          if (!heap.alloc(out_bytes[r], &off)) break;        // FIFO: wait for memory
        } else {
          if (budget_used + align_up(out_bytes[r], 512) > opts->budget_bytes) break;
          budget_used += align_up(out_bytes[r], 512);
        }
        sl.reqs.push_back(r);
        sl.out_off.push_back(off);
        sum_entries += k_r;
        sum_share += s_r;
        syms_batch += pool[req_stream[r]]->n_syms;
        results[r].arrival_s = req_arrival_s[r];
        results[r].admit_s = t;
        next++;
      }
      if (!sl.reqs.empty()) {
        // split counts: this admission's share of the free warp slots
        const uint32_t free_w = total_warps > warps_busy ? total_warps - warps_busy : warps;
        const size_t n = sl.reqs.size();
        const size_t off_outs = sizeof(DevControl);
        const size_t off_streams = off_outs + align_up(n * 8, kAlign);
        const size_t off_items = off_streams + align_up(n * sizeof(DevStream), kAlign);
        if (keeps.size() < n) keeps.resize(n);
        ent_first.resize(n + 1);
        // each request's kept entries (combine, Sec. 3.3, without building a
        // combined stream: the picks index the pool stream's descriptors)
        for (size_t k = 0; k < n; k++) {
          const recoil_stream* src = pool[req_stream[sl.reqs[k]]];
          uint32_t target = (uint32_t)src->entries.size() + 1;
          if (!per_request) {
            // the request's share of the free warps, but splits no longer than
            // max_split: a split is one warp's sequential work
            const double share = syms_batch ? (double)src->n_syms / (double)syms_batch : 1.0;
            uint64_t want = (uint64_t)std::max(1.0, std::floor(free_w * share));
            want = std::max<uint64_t>(want, (src->n_syms + max_split - 1) / max_split);
            want = (want + warps - 1) / warps * warps;
            target = (uint32_t)std::min<uint64_t>(target, want);
          }
          // the same pool stream combined to the same count again (common
          // under a backlog, where most requests get one CTA's splits): reuse
          const uint32_t sid = req_stream[sl.reqs[k]];
          if (memo_target[sid] != target) {
            combine_picks(*src, target, memo_keep[sid]);
            memo_target[sid] = target;
          }
          keeps[k] = memo_keep[sid];
        }
        items.clear();
        item_kind.clear();
        uint32_t warps_launch = 0;
        std::vector<DevStream> ds(n);
        std::vector<void*> outp(n);
        size_t n_ents = 0;
        for (size_t k = 0; k < n; k++) {
          const uint32_t r = sl.reqs[k];
          const recoil_stream* src = pool[req_stream[r]];
          const size_t first = n_ents, count = keeps[k].size() + 1;     // kept entries and the final one
          ent_first[k] = first;
          n_ents += count;
          results[r].splits = (uint32_t)count;
          results[r].launch = launches;
          ds[k] = pool_ds[req_stream[r]];
          outp[k] = d_req_outs ? d_req_outs[r] : (void*)(heap_base + sl.out_off[k]);
          for (size_t x = first; x < n_ents; x += warps) {
            DevItem it;
            it.stream = (uint32_t)k;
            it.entry = (uint32_t)x;
            it.count = (uint32_t)std::min<size_t>(warps, n_ents - x);
            it.work = (uint32_t)std::min<uint64_t>(src->n_syms / count, 0x7fffffff);
            items.push_back(it);
            item_kind.push_back(ds[k].kind);
          }
        }
        ent_first[n] = n_ents;
        // the area: control, output pointers, streams, items, the split
        // references (all copied from the host), then the descriptors the
        // device expands from the references
        const size_t off_refs = off_items + align_up(items.size() * sizeof(DevItem), kAlign);
        const size_t off_entries = off_refs + align_up(n_ents * sizeof(EntryRef), kAlign);
        const size_t meta_bytes = off_refs + n_ents * sizeof(EntryRef);
        if (off_entries + n_ents * sizeof(DevEntry) > meta_cap) {
          status = fail(RECOIL_ENOMEM, "descriptors of one admission exceed meta_bytes; raise it or lower max_batch");
          break;
        }
        // items by kind, longest first within a kind
        std::vector<uint32_t> order(items.size());
        for (uint32_t x = 0; x < order.size(); x++) order[x] = x;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
          if (item_kind[a] != item_kind[b]) return item_kind[a] < item_kind[b];
          return items[a].work > items[b].work;
        });
        uint8_t* h = sl.host;
        std::memset(h, 0, off_refs);                        // control (queue heads, flags) starts at zero
        std::memcpy(h + off_outs, outp.data(), n * 8);
        std::memcpy(h + off_streams, ds.data(), n * sizeof(DevStream));
        DevItem* hi = reinterpret_cast<DevItem*>(h + off_items);
        uint32_t kind_first[kKinds] = {}, kind_count[kKinds] = {};
        for (uint32_t x = 0; x < order.size(); x++) {
          hi[x] = items[order[x]];
          const uint32_t k = item_kind[order[x]];
          if (!kind_count[k]) kind_first[k] = x;
          kind_count[k]++;
        }
        // a reference per kept split into the staging area, each owning from
        // the previous kept split's end
        EntryRef* hr = reinterpret_cast<EntryRef*>(h + off_refs);
        for (size_t k = 0; k < n; k++) {
          const uint64_t base = pool_first[req_stream[sl.reqs[k]]];
          const uint64_t last = pool_first[req_stream[sl.reqs[k]] + 1] - 1;   // the final-state entry
          EntryRef* d = hr + ent_first[k];
          uint32_t prev_end = 0;
          for (uint32_t pk : keeps[k]) {
            *d++ = EntryRef{(uint32_t)(base + pk), prev_end, (uint32_t)k, 0};
            prev_end = pool_hi1[base + pk];
          }
          *d = EntryRef{(uint32_t)last, prev_end, (uint32_t)k, 0};
        }
        e = cudaMemcpyAsync(sl.dev, h, meta_bytes, cudaMemcpyHostToDevice, sl.stream);
        if (e == cudaSuccess)
          e = launch_expand_entries(pool_dev, reinterpret_cast<const EntryRef*>(sl.dev + off_refs),
                                    reinterpret_cast<DevEntry*>(sl.dev + off_entries), (uint32_t)n_ents, sl.stream);
        LaunchArgs a{};
        a.streams = reinterpret_cast<const DevStream*>(sl.dev + off_streams);
        a.entries = reinterpret_cast<const DevEntry*>(sl.dev + off_entries);
        a.word_pool = reinterpret_cast<const uint16_t*>(arena);
        a.table_pool = arena + img.ws_off_tables;
        a.outs = reinterpret_cast<void* const*>(sl.dev + off_outs);
        a.control = reinterpret_cast<DevControl*>(sl.dev);
        a.warps = warps;
        const DevItem* ditems = reinterpret_cast<const DevItem*>(sl.dev + off_items);
        for (uint32_t k = 0; k < kKinds && e == cudaSuccess; k++) {
          if (!kind_count[k]) continue;
          a.items = ditems + kind_first[k];
          a.n_items = kind_count[k];
          a.kind = k;
          a.persistent = 1;
          a.table_smem = kind_smem[k];
          a.tid_staged = img.kind_staged[k];
          const unsigned grid = (unsigned)std::min<uint64_t>(a.n_items, (uint64_t)per_sm[k] * sms);
          e = launch_decode(k, a, grid, sl.stream);
          warps_launch += grid * warps;
        }
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(sl.host + meta_cap, sl.dev, sizeof(DevControl), cudaMemcpyDeviceToHost, sl.stream);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        if (e != cudaSuccess) break;
        for (uint32_t r : sl.reqs) sym_bytes_total += out_bytes[r];
        sl.warps_used = std::min(warps_launch, total_warps);
        warps_busy += sl.warps_used;
        sl.busy = true;
        sl.launch_id = launches++;
        inflight++;
        max_inflight_seen = std::max(max_inflight_seen, inflight);
        progressed = true;
      }
    }
    if (!progressed) {
      // nothing to do this instant: wait a little for an arrival or a completion
      const double until = next < n_req ? req_arrival_s[next] : t + 1e-5;
      if (until - (now_s() - t0) > 2e-5) std::this_thread::yield();
    }
  }
  cudaError_t se = cudaSuccess;
  for (Slot& sl : slots) {
    cudaError_t q = cudaStreamSynchronize(sl.stream);
    if (q != cudaSuccess) se = q;
  }
  if (e == cudaSuccess) e = se;
  cleanup();
  if (e != cudaSuccess) return fail(RECOIL_ECUDA, std::string("serve: ") + cudaGetErrorString(e));
  if (status != RECOIL_OK) return status;

  if (stats) {
    std::memset(stats, 0, sizeof *stats);
    std::vector<double> lat(n_req);
    double sum = 0;
    for (uint32_t r = 0; r < n_req; r++) {
      lat[r] = (results[r].done_s - results[r].arrival_s) * 1e3;
      sum += lat[r];
    }
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) { return n_req ? lat[std::min<size_t>(n_req - 1, (size_t)std::ceil(p * n_req) - 1)] : 0.0; };
    stats->requests = n_req;
    stats->launches = launches;
    stats->symbol_bytes = sym_bytes_total;
    stats->makespan_s = last_done - first_arrival;
    stats->decoded_gbs = stats->makespan_s > 0 ? sym_bytes_total / stats->makespan_s / 1e9 : 0;
    stats->p50_ms = pct(0.50);
    stats->p99_ms = pct(0.99);
    stats->mean_ms = n_req ? sum / n_req : 0;
    stats->max_inflight = max_inflight_seen;
  }
  return RECOIL_OK;
}

}  // extern "C"
