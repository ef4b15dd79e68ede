// Internal types of the Recoil library: the host stream object, plan
// images and the host-side entry points shared between translation units.
// Not part of the C-ABI; the device-side descriptors are in device_types.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "device_types.h"

namespace recoil {

// One split entry as kept on the host (Sec. 4.1 metadata, unpacked).
struct Entry {
  uint64_t word;             // split word q: the decoder's first read
  uint32_t idx[kW];          // recorded symbol index per coder (last symbol coded before the renorm)
  uint16_t y[kW];            // state right after that renormalisation (< L by Lemma 3.1)
  uint64_t wlo = 0;          // lowest word read by the thread that stops at this entry's smallest
                             // index (the first word written for a symbol at or above it); 0 if unknown
};

// Host stream: everything the encoder produced. Words are shared between a
// stream and the streams combined from it, so combining copies no bitstream.
struct Stream {
  uint32_t n_bits = 0;
  uint32_t sym_bytes = 1;
  uint64_t n_syms = 0;
  std::vector<uint32_t> freq;                      // quantised PDF f over the alphabet (adaptive: n_tables rows)
  uint32_t n_tables = 0;                           // adaptive model: PDF rows (0: one static PDF)
  std::shared_ptr<const std::vector<uint8_t>> tid; // adaptive model: PDF row of every symbol index (Sec. 3.1)
  std::shared_ptr<const std::vector<uint16_t>> words;
  std::shared_ptr<const uint16_t> pinned_words;    // optional page-locked copy, shared with combined streams
  uint32_t final_x[kW] = {};
  std::vector<Entry> entries;                      // regular entries, increasing word; final is implicit

  // caches of the device-side images (built on first use)
  mutable std::mutex cache_mu;
  mutable std::vector<uint8_t> table_img;          // decoder tables, padded to 16 B
  mutable uint32_t table_kind = 0;
  mutable std::vector<uint32_t> owned_end;         // per regular entry: its smallest recorded index
  mutable bool owned_end_ready = false;

  uint64_t n_words() const { return words ? words->size() : 0; }
  const uint16_t* word_data() const { return pinned_words ? pinned_words.get() : (words ? words->data() : nullptr); }
  uint32_t alphabet() const { return (uint32_t)(n_tables ? freq.size() / n_tables : freq.size()); }
  bool adaptive() const { return n_tables != 0; }
  bool constant() const;                           // a single symbol owns all 2^n slots (static model)
  const std::vector<uint32_t>& owned_ends() const; // owned_end, built on first use (entries never change)
};

// Regular entries of `in` kept when combining it to `target` splits
// (recoil_combine_splits' rule; the final entry is always kept besides them).
void combine_picks(const Stream& in, uint32_t target, std::vector<uint32_t>& keep);

// Host images of a plan (plan.cpp), for entry points that place them in
// device memory of their own. meta = control, output pointers, stream
// descriptors, items, entries (offsets relative to meta); tables separate.
struct PlanImage {
  const uint8_t* meta;
  size_t meta_bytes;
  size_t off_outs, off_streams, off_items, off_entries;
  const uint8_t* tables;
  size_t table_bytes;
  size_t ws_off_tables;      // workspace offset of the tables (words start at 0)
  uint32_t warps;
  uint32_t lanes;            // coder lanes a thread
  uint32_t kind_first[kKinds], kind_count[kKinds], kind_smem[kKinds], kind_warp_queue[kKinds];
  uint32_t kind_staged[kKinds];   // adaptive launch kinds that stage table numbers in shared memory
};
}  // namespace recoil
struct recoil_plan;
namespace recoil {
void plan_image(const recoil_plan* plan, PlanImage* out);
// Device entries of a stream's kept splits, the final-state entry last (plan.cpp).
// word_base: the first word staged in the workspace (entries' q count from it).
void build_entries(const Stream& s, uint32_t stream_index, std::vector<DevEntry>& out, uint64_t word_base = 0);
// Upload the bulk region (words, tables) and/or the descriptors of a plan.
int plan_upload_parts(recoil_plan* plan, void* d_ws, size_t ws_bytes, cudaStream_t s, bool bulk, bool meta);
// Bytes of the bulk region at the start of a plan's workspace.
size_t plan_bulk_bytes(const recoil_plan* plan);
// The streams a plan decodes (after combining).
const std::vector<const Stream*>& plan_streams(const recoil_plan* plan);
// Copy stream k's bulk data (words; table numbers of an adaptive stream) to its place in ws.
cudaError_t plan_upload_stream(const recoil_plan* plan, size_t k, uint8_t* ws, cudaStream_t s);
// Output pointers as the kernels index them (symbol i of stream k at dev[k] +
// i * sym_bytes): the caller's pointers, shifted back by the first owned
// symbol for a shard plan, whose buffer starts there.
void plan_kernel_outs(const recoil_plan* plan, void* const* outs, void** dev);
// Host image of the bulk region (words, table numbers, tables) exactly as it
// sits at the start of the workspace: plan_bulk_bytes bytes written to dst.
void plan_bulk_image(const recoil_plan* plan, uint8_t* dst);

// Serving (serve_kernels.cu): a kept split of an admission as a reference to
// a resident pool descriptor, with the owned low end and the stream index the
// admission gives it; the device expands the references into descriptors.
struct EntryRef {
  uint32_t src;              // index of the descriptor in the resident pool set
  uint32_t lo;               // first owned symbol (the previous kept split's end)
  uint32_t stream;           // the request's place among the launch's streams
  uint32_t pad;
};
static_assert(sizeof(EntryRef) == 16, "EntryRef layout");
cudaError_t launch_expand_entries(const DevEntry* pool, const EntryRef* refs, DevEntry* out, uint32_t n,
                                  cudaStream_t s);

// Error reporting (thread-local message).
int fail(int code, const std::string& msg);
void clear_error();

}  // namespace recoil

struct recoil_stream : recoil::Stream {};
