// Types and constants the decode kernels are compiled against: coder
// parameters, table kinds, and the device-side descriptors a plan lays out in
// the workspace (entries, streams, work items, the control block, launch
// arguments). Host-only structures live in recoil_internal.h.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "recoil.h"

namespace recoil {

constexpr int kW = RECOIL_W;                 // interleaved coders = warp width
constexpr int kLgL = RECOIL_LOG2_L;          // L = 2^16
constexpr uint32_t kL = 1u << kLgL;
constexpr int kB = RECOIL_B;                 // 16-bit renormalisation words
constexpr int kChunkWords = 256;             // words per refill of a warp's ring (512 B)
constexpr int kRingWords = 512;              // words a warp keeps staged (two chunks)
constexpr int kRingSlots = 2 * kRingWords;   // each staged word is stored twice (wrap-free reads)

// Decoder table kinds.
enum TableKind : uint32_t {
  kPacked8 = 0,    // 8-bit symbols, n <= 12, f < 4096: one u32 per slot = bias | sym << 12 | f << 20
  kGeneric8 = 1,   // 8-bit symbols otherwise: u16 slot -> symbol, u32 symbol -> (f-1) << 16 | F
  kGeneric16 = 2,  // 16-bit symbols: same tables as kGeneric8, 16-bit stores
  // adaptive model (a PDF row per symbol index): one u16 CDF row per PDF and
  // a bucket guide per row that narrows the search
  kAdaptive8 = 3,       // 8-bit symbols; one-byte guide entries
  kAdaptive16 = 4,      // 16-bit symbols, alphabet <= 256; one-byte guide entries
  kAdaptive16Wide = 5,  // 16-bit symbols, alphabet <= 4096; two-byte guide entries
  // the same models as kAdaptive8 / kAdaptive16 in the paired layout: a block
  // per PDF of one u32 F(s) | H(s+1) << 16 per symbol and a byte guide over
  // 2^10 buckets (a plan stages it where it keeps as many splits resident)
  kAdaptive8Pair = 6,
  kAdaptive16Pair = 7,
  // 16-bit symbols, alphabet <= 4096, n <= 15, every f <= 1023: one u32 per
  // slot = bias | f << 10 | sym << 20 (one shared read a symbol)
  kPacked16 = 8,
  kKinds = 9,
};

static_assert(RECOIL_KERNEL_PACKED8 == 1u << kPacked8 && RECOIL_KERNEL_GENERIC8 == 1u << kGeneric8 &&
                  RECOIL_KERNEL_GENERIC16 == 1u << kGeneric16 && RECOIL_KERNEL_ADAPTIVE8 == 1u << kAdaptive8 &&
                  RECOIL_KERNEL_ADAPTIVE16 == 1u << kAdaptive16 &&
                  RECOIL_KERNEL_ADAPTIVE16_WIDE == 1u << kAdaptive16Wide &&
                  RECOIL_KERNEL_ADAPTIVE8_PAIR == 1u << kAdaptive8Pair &&
                  RECOIL_KERNEL_ADAPTIVE16_PAIR == 1u << kAdaptive16Pair && RECOIL_KERNEL_PACKED16 == 1u << kPacked16,
              "kernel bits follow the table kinds");

__host__ __device__ constexpr bool is_adaptive_kind(uint32_t k) { return k >= kAdaptive8 && k <= kAdaptive16Pair; }
__host__ __device__ constexpr bool is_pair_kind(uint32_t k) { return k == kAdaptive8Pair || k == kAdaptive16Pair; }
// The paired kind of an adaptive kind with one-byte guide entries (itself otherwise).
__host__ __device__ constexpr uint32_t pair_kind_of(uint32_t k) {
  return k == kAdaptive8 ? kAdaptive8Pair : k == kAdaptive16 ? kAdaptive16Pair : k;
}
// Bytes of a guide entry (a symbol number) of an adaptive kind.
__host__ __device__ constexpr uint32_t adaptive_guide_entry_bytes(uint32_t k) { return k == kAdaptive16Wide ? 2 : 1; }
// The guide of a row: 2^g buckets over the 2^n slots (at most 2^n). A plan
// stages g = 9, or 10 where it can afford twice the guide's shared memory,
// or 0 (one bucket: the whole row is searched) where even 9 does not fit, or
// the paired layout with 2^10 buckets (kGuidePairs, for one-byte entries).
constexpr uint32_t kGuideBits = 9;
constexpr uint32_t kGuideBitsFine = 10;
constexpr uint32_t kGuideBitsNone = 0;
constexpr uint32_t kGuidePairs = 0x100 | kGuideBitsFine;   // variant code, not a width: 2^10 buckets, paired

// Longest alphabet of an adaptive model (the decoder's CDF search covers 2^12 symbols).
constexpr uint32_t kMaxAdaptiveAlphabet = 4096;
// Most PDF rows of an adaptive model (a table number is one byte per symbol).
constexpr uint32_t kMaxTables = 256;

// ------------------------------------------------------------ device images

// One decoder thread (one warp): a kept entry with its owned range.
struct alignas(16) DevEntry {
  int32_t q;                 // first word read (-1: the stream has no words)
  int32_t g_top;             // first group visited
  uint32_t lo;               // first owned symbol
  uint32_t hi1;              // one past the last owned symbol (lo == hi1: nothing owned)
  uint32_t x0[kW];           // state a coder takes when it joins
  int32_t act[kW];           // group at which a coder joins (takes x0, renormalises)
  uint32_t stream;           // stream (index into the launch's streams) the entry belongs to
  uint32_t pad[3];
};
static_assert(sizeof(DevEntry) == 32 + 8 * kW, "DevEntry layout");

struct alignas(16) DevStream {
  uint64_t words;            // element offset of the stream's words in the word pool (multiple of 256)
  uint64_t table;            // byte offset of the stream's tables in the table pool (multiple of 16)
  int64_t tid;               // adaptive: element offset (16-bit units) in the word pool of the table number of
                             // symbol 0 (a shard plan stages a window of them, so this may point before it)
  uint32_t n_words;
  uint32_t n_bits;
  uint32_t kind;             // TableKind
  uint32_t alphabet;
  uint32_t sym_bytes;
  uint32_t table_bytes;      // bytes of the table image (multiple of 16)
  union {
    uint32_t slot_bytes;     // generic kinds: bytes of the slot -> symbol part (multiple of 16)
    uint32_t guide_bits;     // adaptive kinds: log2 of the guide buckets per row
  };
  uint32_t row_stride;       // adaptive: entries between CDF rows, an odd number of 32-bit words
                             // (16-bit entries; paired kinds: 32-bit words between a PDF's blocks)
  uint32_t n_tables;         // adaptive: CDF rows
  uint32_t guide_stride;     // adaptive kinds: bytes between guide rows (after all CDF rows; one entry per bucket
                             // boundary); paired kinds: byte offset of the guide within a PDF's block
};
static_assert(sizeof(DevStream) == 64, "DevStream layout");

// A unit of work for one CTA: consecutive entries of one stream or of
// consecutive streams whose decoder tables are identical; the CTA's warps pop
// them one at a time.
struct alignas(16) DevItem {
  uint32_t stream;
  uint32_t entry;            // first DevEntry
  uint32_t count;            // number of entries
  uint32_t work;             // estimated symbols decoded (for ordering)
};

struct alignas(16) DevControl {
  uint32_t head[16];         // persistent queue position, one per table kind
  uint32_t errors;           // kErr* bits
  uint32_t bad_entry;        // an entry that raised an error (+1), 0 if none
  uint32_t pad[46];
};
static_assert(sizeof(DevControl) == 256, "DevControl layout");
static_assert(kKinds <= 16, "one queue head per table kind");

// Error flags raised by kernels.
constexpr uint32_t kErrCorrupt = 1u;         // a state differs from the previous entry's record, or the
                                             // first thread did not end at p = -1 with every state = L
constexpr uint32_t kErrUnderrun = 2u;        // a read went below word 0

// Arguments of one kernel launch.
struct LaunchArgs {
  const DevItem* items;      // items of this launch (one table kind)
  uint32_t n_items;
  uint32_t kind;
  uint32_t persistent;       // 1: CTAs pop items from control->head; 0: one item per CTA
  const DevStream* streams;
  const DevEntry* entries;
  const uint16_t* word_pool;
  const uint8_t* table_pool;
  void* const* outs;         // device array: output pointer per stream
  DevControl* control;
  uint32_t table_smem;       // bytes reserved for tables in shared memory
  uint32_t warps;            // warps per CTA
  uint32_t warp_queue;       // 1: every item is one entry and all share one table; warps pop items alone
  uint32_t lanes;            // coder lanes a thread (splits a warp decodes at once): 1 (0 reads as 1) or 2
  uint32_t tid_staged;       // adaptive kinds, one lane a thread: stage table numbers in shared memory
};

// Grid of a persistent launch: enough CTAs for the items, at most the resident ones.
inline unsigned launch_grid(const LaunchArgs& a, int ctas_per_sm, int sms) {
  const uint64_t per_cta = (uint64_t)a.warps * (a.lanes > 1 ? a.lanes : 1);
  const uint64_t need = a.warp_queue ? (a.n_items + per_cta - 1) / per_cta : a.n_items;
  const uint64_t cap = (uint64_t)ctas_per_sm * (uint64_t)sms;
  return (unsigned)(need < cap ? need : cap);
}

// Kernel launchers (decode_kernels.cu).
cudaError_t launch_decode(uint32_t kind, const LaunchArgs& a, unsigned grid, cudaStream_t s);
int occupancy_ctas_per_sm(uint32_t kind, uint32_t warps, uint32_t lanes, bool staged, uint32_t table_smem, int* out);
// Shared memory a warp of a `kind` kernel holds besides the tables: a word ring
// per lane a thread, and for adaptive kinds at one lane a thread whose launch
// stages them the table numbers of three steady blocks.
size_t warp_smem(uint32_t kind, uint32_t lanes, bool staged);
bool warps_supported(uint32_t warps);   // CTA sizes the kernels are built for: 1, 2, 4, 8, 16, 32 warps
bool adaptive_warps_supported(uint32_t warps);   // adaptive kinds: 4, 8, 16, 32 warps
// CTA shapes built: one lane a thread as above; two lanes a thread: static
// kinds 4, 8, 16 warps, adaptive kinds 8, 16, 24 warps
bool shape_supported(bool adaptive, uint32_t warps, uint32_t lanes);

}  // namespace recoil
