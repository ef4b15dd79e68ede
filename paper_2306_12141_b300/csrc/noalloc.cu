// Decoding without any device allocation by the library or the caller's
// allocator: recoil_decode_noalloc.
//
// Some callers cannot call cudaMalloc (or an allocator built on it) at the
// point where they decode: code that runs inside a host framework which owns
// every device allocation and hands out only fixed buffers, or code on a path
// where an allocation could block or fail at an unacceptable moment. They can
// still hand over device buffers they already hold for the inputs and the
// output. This entry point needs nothing else: the per-call device data the
// decoder derives from the stream (split descriptors, decoder tables, the work
// queue counters and error flags) lives in one file-scope device array.
//
// That array is a fixed RECOIL_NOALLOC_SCRATCH_BYTES per GPU that loads the
// library and stays allocated until the process exits. Every call shares it
// and it keeps the previous call's contents: each call rewrites the parts it
// uses and clears the queue counters and error flags first. Calls whose GPU
// work overlaps (from several host threads or on several CUDA streams) race
// on the array and must not be issued.
#include <cstring>
#include <vector>

#include "recoil_internal.h"

namespace recoil {
namespace {

constexpr size_t kScratchBytes = RECOIL_NOALLOC_SCRATCH_BYTES;

// The decoder's per-call device data. In host code this name is only a host
// stand-in for the symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device. Looked up on
// every call (a host-side lookup): after a device reset the module is loaded
// again and the array may sit elsewhere, so no address is kept between calls.
int scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return fail(RECOIL_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return RECOIL_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace recoil

using namespace recoil;

extern "C" int recoil_decode_noalloc(const recoil_stream* s, const void* d_words, size_t words_bytes, void* d_out,
                                     void* cuda_stream) {
  clear_error();
  if (!s || (!d_out && s->n_syms)) return fail(RECOIL_EINVAL, "null argument");
  if (s->adaptive())
    return fail(RECOIL_EINVAL, "adaptive streams keep their table numbers in a workspace: use the plan API");
  const size_t need_words = (s->n_words() + kChunkWords - 1) / kChunkWords * kChunkWords * 2;
  if (need_words && (!d_words || words_bytes < need_words))
    return fail(RECOIL_EINVAL, "d_words must hold the stream's words padded to a multiple of 256 words (" +
                                   std::to_string(need_words) + " bytes)");
  if (((uintptr_t)d_words) % 16) return fail(RECOIL_EINVAL, "d_words must be 16-byte aligned");

  const recoil_stream* one[1] = {s};
  recoil_plan* plan = nullptr;
  int rc = recoil_plan_create(one, 1, nullptr, &plan);
  if (rc) return rc;
  PlanImage img;
  plan_image(plan, &img);
  const size_t off_tables = align256(img.meta_bytes);
  const size_t need = off_tables + img.table_bytes;
  if (need > kScratchBytes) {
    recoil_plan_free(plan);
    return fail(RECOIL_EINVAL, "stream needs " + std::to_string(need) + " bytes of decoder scratch, more than the " +
                                   std::to_string(kScratchBytes) +
                                   " bytes recoil_decode_noalloc holds; combine it to fewer splits");
  }
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) {
    recoil_plan_free(plan);
    return rc;
  }
  uint8_t* scratch = static_cast<uint8_t*>(base);
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  int sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    recoil_plan_free(plan);
    return fail(RECOIL_ECUDA, std::string("recoil_decode_noalloc: ") + cudaGetErrorString(e));
  }
  // every occupancy query before anything is enqueued, so that no error
  // return leaves work queued on cuda_stream
  int per_sm[kKinds] = {};
  for (uint32_t k = 0; k < kKinds; k++) {
    if (!img.kind_count[k]) continue;
    const uint32_t smem = (uint32_t)((img.kind_smem[k] + 15) / 16 * 16);
    if (occupancy_ctas_per_sm(k, img.warps, img.lanes, img.kind_staged[k] != 0, smem, &per_sm[k]) != 0 || per_sm[k] <= 0) {
      recoil_plan_free(plan);
      return fail(RECOIL_ECUDA, "occupancy query failed");
    }
  }

  // Host copy of the descriptors with the output pointer filled in; the
  // control block at its start is zero, which clears the previous call's
  // queue counters and error flags.
  std::vector<uint8_t> meta(img.meta, img.meta + img.meta_bytes);
  void* outp = d_out;
  std::memcpy(meta.data() + img.off_outs, &outp, sizeof outp);
  e = cudaMemcpyAsync(scratch, meta.data(), meta.size(), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && img.table_bytes)
    e = cudaMemcpyAsync(scratch + off_tables, img.tables, img.table_bytes, cudaMemcpyHostToDevice, cs);

  LaunchArgs a{};
  a.streams = reinterpret_cast<const DevStream*>(scratch + img.off_streams);
  a.entries = reinterpret_cast<const DevEntry*>(scratch + img.off_entries);
  a.word_pool = static_cast<const uint16_t*>(d_words);
  a.table_pool = scratch + off_tables;
  a.outs = reinterpret_cast<void* const*>(scratch + img.off_outs);
  a.control = reinterpret_cast<DevControl*>(scratch);
  a.warps = img.warps;
  a.lanes = img.lanes;
  const DevItem* items = reinterpret_cast<const DevItem*>(scratch + img.off_items);
  for (uint32_t k = 0; e == cudaSuccess && k < kKinds; k++) {
    if (!img.kind_count[k]) continue;
    a.items = items + img.kind_first[k];
    a.n_items = img.kind_count[k];
    a.kind = k;
    a.persistent = 1;
    a.table_smem = (uint32_t)((img.kind_smem[k] + 15) / 16 * 16);
    a.warp_queue = img.kind_warp_queue[k];
    a.tid_staged = img.kind_staged[k];
    e = launch_decode(k, a, launch_grid(a, per_sm[k], sms), cs);
  }
  // read the error flags back (this also makes the call return after the decode)
  DevControl ctl;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, scratch, sizeof ctl, cudaMemcpyDeviceToHost, cs);
  // whatever failed above, nothing the call queued may still run once it returns
  const cudaError_t es = cudaStreamSynchronize(cs);
  if (e == cudaSuccess) e = es;
  recoil_plan_free(plan);
  if (e != cudaSuccess) return fail(RECOIL_ECUDA, std::string("recoil_decode_noalloc: ") + cudaGetErrorString(e));
  if (ctl.errors)
    return fail(RECOIL_ECORRUPT, "decoder found an inconsistent stream (flags " + std::to_string(ctl.errors) + ")");
  return RECOIL_OK;
}
