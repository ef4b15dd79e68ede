// Decode plans: the device image of a batch of streams (words, decoder
// tables, one descriptor per kept split entry) and the CTA work queue, plus
// upload and launch. A single stream is a batch of one.
//
// Workspace layout (caller-owned device memory, every segment 256-B aligned):
//   words (each stream's words start on a 512-B chunk) | decoder tables |
//   control | output pointers | stream descriptors | work items | entries
// The words and tables depend only on the list of streams, so plans that
// differ only in how they split the streams share that bulk region.
#include <algorithm>
#include <cstring>
#include <new>

#include "recoil_internal.h"

namespace recoil {
namespace {

constexpr size_t kAlign = 256;
constexpr uint32_t kMaxSmem = 227 * 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// A static 16-bit model whose every slot packs into a u32 (kPacked16):
// symbols below 2^12, n <= 15 (a LUT of at most 128 KB) and every f <= 1023.
bool packed16_fits(const Stream& s) {
  if (s.n_bits > 15 || s.alphabet() > 4096) return false;
  for (uint32_t f : s.freq)
    if (f > 1023) return false;
  return true;
}

uint32_t table_kind_of(const Stream& s) {
  if (s.adaptive()) {
    if (s.sym_bytes == 1) return kAdaptive8;
    return s.alphabet() <= 256 ? kAdaptive16 : kAdaptive16Wide;
  }
  if (s.sym_bytes == 2) return packed16_fits(s) ? kPacked16 : kGeneric16;
  if (s.n_bits <= 12 && !s.constant()) return kPacked8;
  return kGeneric8;
}

// 16-bit entries between the CDF rows of an adaptive model: at least A + 1,
// an odd number of 32-bit words so that the same position in different rows
// falls in different shared-memory banks.
uint32_t adaptive_row_stride(uint32_t A) {
  uint32_t words = (A + 2) / 2;
  if (!(words & 1)) words++;
  return 2 * words;
}

uint32_t guide_bits(uint32_t n, uint32_t g) { return std::min<uint32_t>(g, n); }

// Bytes between guide rows: 2^g + 1 entries of `eb` bytes, an odd number of
// 32-bit words (rows start in different banks).
uint32_t guide_stride(uint32_t n, uint32_t g, uint32_t eb) {
  uint32_t words = (((1u << guide_bits(n, g)) + 1) * eb + 3) / 4;
  if (!(words & 1)) words++;
  return 4 * words;
}

// Paired layout (one-byte guide entries only): a block per PDF, an odd
// number of 32-bit words apart so that blocks start in different banks: the
// u32 F(s) | H(s+1) << 16 of each symbol (F(s) modulo 2^16: exact for every
// symbol of nonzero frequency), then the guide row, one byte for each of the
// 2^g + 1 bucket boundaries (g = 10, or n if smaller).
uint32_t pair_guide_bits(uint32_t n) { return guide_bits(n, kGuideBitsFine); }
uint32_t pair_block_words(uint32_t A, uint32_t n) {
  uint32_t words = A + ((1u << pair_guide_bits(n)) + 1 + 3) / 4;
  if (!(words & 1)) words++;
  return words;
}

// An adaptive stream's table image holds four variants: the CDF rows followed
// by a guide row per PDF with 2^9 buckets, with 2^10 buckets, with one bucket,
// and (one-byte guide entries only) the paired layout with 2^10 buckets; a
// plan stages one of them. The variants in image order:
constexpr uint32_t kGuideVariants[4] = {kGuideBits, kGuideBitsFine, kGuideBitsNone, kGuidePairs};

// Bytes of the variant `v` of a stream's image (0: not built for this model).
size_t variant_bytes(const Stream& s, uint32_t v) {
  const uint32_t eb = adaptive_guide_entry_bytes(table_kind_of(s));
  if (v == kGuidePairs) {
    if (eb != 1) return 0;
    return align_up((size_t)s.n_tables * pair_block_words(s.alphabet(), s.n_bits) * 4, 16);
  }
  const size_t rows = (size_t)s.n_tables * adaptive_row_stride(s.alphabet()) * 2;
  return align_up(rows + (size_t)s.n_tables * guide_stride(s.n_bits, v, eb), 16);
}

// Offset and size of the variant `g` within the image.
void guide_variant(const Stream& s, uint32_t g, size_t* off, size_t* bytes) {
  size_t o = 0;
  for (uint32_t v : kGuideVariants) {
    const size_t b = variant_bytes(s, v);
    if (v == g) {
      *off = o;
      *bytes = b;
      return;
    }
    o += b;
  }
  *off = 0;
  *bytes = 0;
}

// Decoder tables of a stream (built once and cached on the stream).
const std::vector<uint8_t>& table_image(const Stream& s, uint32_t* kind, uint32_t* slot_bytes) {
  std::lock_guard<std::mutex> g(s.cache_mu);
  const uint32_t n = s.n_bits, slots = 1u << n, A = s.alphabet();
  const uint32_t k = table_kind_of(s);
  const uint32_t sb = (uint32_t)align_up((size_t)slots * 2, 16);
  if (s.table_img.empty()) {
    if (is_adaptive_kind(k)) {
      // one row per PDF: H(s) = F(s) - 1 modulo 2^16 for s = 0..A (H(0) = 0xffff,
      // H(A) = 2^n - 1), then a guide row per PDF: for each of the 2^g buckets
      // of slots the symbol owning its first slot, and after them the owner of
      // the last slot, so that entries b and b + 1 bracket the symbol of any
      // slot in bucket b. The image holds the rows once per guide width.
      const uint32_t stride = adaptive_row_stride(A);
      const size_t rows_bytes = (size_t)s.n_tables * stride * 2;
      const uint32_t eb = adaptive_guide_entry_bytes(k);
      size_t total = 0, off = 0, bytes = 0;
      for (uint32_t v : kGuideVariants) {
        guide_variant(s, v, &off, &bytes);
        total = off + bytes;
      }
      s.table_img.assign(total, 0);
      std::vector<uint32_t> F(A + 1);
      for (uint32_t v : kGuideVariants) {
        if (v == kGuidePairs) continue;
        guide_variant(s, v, &off, &bytes);
        uint16_t* cdf = reinterpret_cast<uint16_t*>(s.table_img.data() + off);
        uint8_t* guide = s.table_img.data() + off + rows_bytes;
        const uint32_t gb = guide_bits(n, v), gstride = guide_stride(n, v, eb);
        for (uint32_t t = 0; t < s.n_tables; t++) {
          F[0] = 0;
          for (uint32_t sym = 0; sym < A; sym++) F[sym + 1] = F[sym] + s.freq[(size_t)t * A + sym];
          for (uint32_t sym = 0; sym <= A; sym++) cdf[(size_t)t * stride + sym] = (uint16_t)(F[sym] - 1);
          uint32_t sym = 0;
          for (uint32_t b = 0; b <= (1u << gb); b++) {
            const uint32_t slot = std::min<uint32_t>(b << (n - gb), (1u << n) - 1);
            while (F[sym + 1] <= slot) sym++;              // the symbol whose slots hold `slot`
            uint8_t* e = guide + (size_t)t * gstride + (size_t)b * eb;
            e[0] = (uint8_t)sym;
            if (eb == 2) e[1] = (uint8_t)(sym >> 8);       // little-endian 16-bit entry
          }
        }
      }
      if (eb == 1) {
        // paired layout: per PDF, u32 F(s) | H(s+1) << 16 per symbol, then per
        // bucket boundary b the symbol owning slot b << (n - g) (the last slot
        // for b = 2^g)
        guide_variant(s, kGuidePairs, &off, &bytes);
        const uint32_t bw = pair_block_words(A, n), gb = pair_guide_bits(n);
        for (uint32_t t = 0; t < s.n_tables; t++) {
          uint8_t* blk = s.table_img.data() + off + (size_t)t * bw * 4;
          F[0] = 0;
          for (uint32_t sym = 0; sym < A; sym++) F[sym + 1] = F[sym] + s.freq[(size_t)t * A + sym];
          for (uint32_t sym = 0; sym < A; sym++) {
            const uint32_t v = (F[sym] & 0xffffu) | (((F[sym + 1] - 1) & 0xffffu) << 16);
            std::memcpy(blk + (size_t)sym * 4, &v, 4);
          }
          uint32_t sym = 0;
          for (uint32_t b = 0; b <= (1u << gb); b++) {
            const uint32_t slot = std::min<uint32_t>(b << (n - gb), (1u << n) - 1);
            while (F[sym + 1] <= slot) sym++;
            blk[(size_t)A * 4 + b] = (uint8_t)sym;
          }
        }
      }
    } else if (k == kPacked8) {
      s.table_img.assign(align_up((size_t)slots * 4, 16), 0);
      uint32_t* lut = reinterpret_cast<uint32_t*>(s.table_img.data());
      uint32_t F = 0;
      for (uint32_t sym = 0; sym < A; sym++) {
        const uint32_t f = s.freq[sym];
        for (uint32_t b = 0; b < f; b++) lut[F + b] = b | (sym << 12) | (f << 20);
        F += f;
      }
    } else if (k == kPacked16) {
      s.table_img.assign(align_up((size_t)slots * 4, 16), 0);
      uint32_t* lut = reinterpret_cast<uint32_t*>(s.table_img.data());
      uint32_t F = 0;
      for (uint32_t sym = 0; sym < A; sym++) {
        const uint32_t f = s.freq[sym];
        for (uint32_t b = 0; b < f; b++) lut[F + b] = b | (f << 10) | (sym << 20);
        F += f;
      }
    } else {
      s.table_img.assign(sb + align_up((size_t)A * 4, 16), 0);
      uint16_t* slot_sym = reinterpret_cast<uint16_t*>(s.table_img.data());
      uint32_t* symtab = reinterpret_cast<uint32_t*>(s.table_img.data() + sb);
      uint32_t F = 0;
      for (uint32_t sym = 0; sym < A; sym++) {
        const uint32_t f = s.freq[sym];
        for (uint32_t b = 0; b < f; b++) slot_sym[F + b] = (uint16_t)sym;
        symtab[sym] = f ? (((f - 1) << 16) | F) : 0;
        F += f;
      }
    }
    s.table_kind = k;
  }
  *kind = s.table_kind;
  *slot_bytes = (k == kGeneric8 || k == kGeneric16) ? sb : 0;
  return s.table_img;
}

}  // namespace

// Device entries of a stream: kept regular entries in order, then the final one.
void build_entries(const Stream& s, uint32_t stream_index, std::vector<DevEntry>& out, uint64_t word_base) {
  const uint32_t N = (uint32_t)s.n_syms;
  uint32_t prev_m = 0;
  for (const Entry& e : s.entries) {
    DevEntry d;
    std::memset(&d, 0, sizeof d);
    d.stream = stream_index;
    uint32_t mn = e.idx[0], mx = e.idx[0];
    for (int j = 0; j < kW; j++) {
      d.x0[j] = e.y[j];
      d.act[j] = (int32_t)(e.idx[j] / kW) + 1;      // joins one group above its recorded symbol
      mn = std::min(mn, e.idx[j]);
      mx = std::max(mx, e.idx[j]);
    }
    d.q = (int32_t)((int64_t)e.word - (int64_t)word_base);
    d.g_top = (int32_t)(mx / kW) + 1;
    d.lo = prev_m;
    d.hi1 = mn;                                      // owns [previous m, m - 1] (Sec. 4.1.3)
    prev_m = mn;
    out.push_back(d);
  }
  DevEntry d;
  std::memset(&d, 0, sizeof d);
  d.stream = stream_index;
  int32_t top = 0;
  for (int j = 0; j < kW; j++) {
    d.x0[j] = s.final_x[j];
    if ((uint32_t)j < N) {
      const uint32_t last = (uint32_t)j + kW * ((N - 1 - (uint32_t)j) / kW);
      d.act[j] = (int32_t)(last / kW) + 1;
    } else {
      d.act[j] = 0;                                  // coder never coded a symbol
    }
    top = std::max(top, d.act[j]);
  }
  d.q = (int32_t)((int64_t)s.n_words() - 1 - (int64_t)word_base);
  d.g_top = top;
  d.lo = prev_m;
  d.hi1 = N;
  out.push_back(d);
}

}  // namespace recoil

using namespace recoil;

struct recoil_plan {
  std::vector<std::unique_ptr<recoil_stream>> owned;   // combined copies
  std::vector<const Stream*> streams;
  recoil_batch_opts opts{};
  uint32_t warps = 16;
  uint32_t lanes = 1;                                  // coder lanes a thread (splits a warp decodes at once)

  std::vector<uint8_t> meta;                           // control .. entries
  std::vector<uint8_t> tables;
  size_t off_outs = 0, off_streams = 0, off_items = 0, off_entries = 0;
  size_t off_tables = 0, off_meta = 0, ws_bytes = 0;   // words start at 0
  std::vector<uint64_t> word_off;                      // per stream: its staged words' place in the pool, in words
  std::vector<uint64_t> word_lo, word_cnt;             // per stream: first staged word and how many are staged
  std::vector<uint64_t> tid_off;                       // per adaptive stream: its staged table numbers, in words
  std::vector<uint64_t> tid_lo, tid_cnt;               // per adaptive stream: first staged symbol and how many
  uint32_t n_items = 0;
  uint32_t kind_first[kKinds] = {}, kind_count[kKinds] = {}, kind_smem[kKinds] = {}, kind_warp_queue[kKinds] = {};
  uint32_t kind_staged[kKinds] = {};                   // adaptive launch kinds staging table numbers in shared memory
  std::vector<uint32_t> stream_kind, stream_item_first, stream_item_count;
  // shard plans (one stream): only entries [entry_first, entry_last) get work
  // items; the others stay in the entry array as the previous-entry guards
  // the decoders read. out_shift = first owned symbol (outputs start there).
  bool shard = false;
  uint32_t entry_first = 0, entry_last = 0;
  uint64_t out_shift = 0;

  uint8_t* d_ws = nullptr;
  bool uploaded = false;
  std::vector<void*> outs;                             // caller's output pointers
  std::vector<void*> outs_dev;                         // as the kernels index them
  bool outs_on_device = false;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  uint32_t launches = 0;
  int sms = 0;

  ~recoil_plan() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};

// Symbols one entry's walk visits (for longest-first ordering of work items).
static uint32_t entry_work(const DevEntry& de) {
  const int64_t span = (int64_t)de.g_top * kW - (int64_t)de.lo;
  return (uint32_t)std::max<int64_t>(0, std::min<int64_t>(span, 0x7fffffff));
}

static int device_sms();

// CTAs of `warps` warps that one SM holds when each needs `smem` bytes of
// shared memory; adaptive kernels are built for 32 resident warps an SM
// (64 registers a thread).
static uint64_t adaptive_ctas_per_sm(uint32_t warps, uint32_t lanes, size_t smem) {
  int dev = 0, per_sm = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();
    per_sm = 228 * 1024;                           // sm_100 / sm_103
    reserved = 1024;
  }
  // registers: 32 warps an SM with one lane a thread, 24 with two
  return std::min<uint64_t>((uint64_t)per_sm / (smem + (size_t)reserved), (lanes == 2 ? 24 : 32) / warps);
}

// Guide width of each adaptive kind in a plan: 2^10 buckets (about a third
// fewer search steps on wide PDFs than 2^9) unless those larger tables lower
// the number of the kind's splits that the GPU decodes at once; else 2^9;
// one bucket where not even the 2^9 guide fits beside the decoder rings.
static void choose_guides(const recoil_plan* P, uint32_t* guide) {
  uint64_t entries[kKinds] = {};
  size_t coarse[kKinds] = {}, fine[kKinds] = {}, paired[kKinds] = {};
  bool pairable[kKinds];
  for (uint32_t k = 0; k < kKinds; k++) {
    guide[k] = kGuideBits;
    pairable[k] = true;
  }
  for (const Stream* s : P->streams) {
    const uint32_t k = table_kind_of(*s);
    if (!is_adaptive_kind(k)) continue;
    entries[k] += P->shard ? P->entry_last - P->entry_first : s->entries.size() + 1;
    size_t off = 0, bytes = 0;
    guide_variant(*s, kGuideBits, &off, &bytes);
    coarse[k] = std::max(coarse[k], bytes);
    guide_variant(*s, kGuideBitsFine, &off, &bytes);
    fine[k] = std::max(fine[k], bytes);
    guide_variant(*s, kGuidePairs, &off, &bytes);
    paired[k] = std::max(paired[k], bytes);
    pairable[k] = pairable[k] && bytes > 0;
  }
  // every adaptive kind alike; table-number staging is decided afterwards,
  // only where it costs neither guide width nor residency
  const size_t rings = (size_t)P->warps * warp_smem(kAdaptive8, P->lanes, false) + 16;
  const uint64_t per_cta = (uint64_t)P->warps * P->lanes;   // splits a CTA decodes at once
  const uint64_t sms = (uint64_t)device_sms();
  for (uint32_t k = 0; k < kKinds; k++) {
    if (!entries[k]) continue;
    if (coarse[k] + rings > kMaxSmem) {
      guide[k] = kGuideBitsNone;
      continue;
    }
    // the variant that keeps the most splits resident; on a tie the finer
    // guide, and the paired layout before either
    uint64_t best = std::min(entries[k], adaptive_ctas_per_sm(P->warps, P->lanes, coarse[k] + rings) * sms * per_cta);
    if (fine[k] + rings <= kMaxSmem) {
      const uint64_t cap10 =
          std::min(entries[k], adaptive_ctas_per_sm(P->warps, P->lanes, fine[k] + rings) * sms * per_cta);
      if (cap10 >= best) {
        guide[k] = kGuideBitsFine;
        best = cap10;
      }
    }
    if (pairable[k] && !(P->opts.flags & RECOIL_BATCH_NO_PAIRS) && paired[k] + rings <= kMaxSmem) {
      const uint64_t capp =
          std::min(entries[k], adaptive_ctas_per_sm(P->warps, P->lanes, paired[k] + rings) * sms * per_cta);
      if (capp >= best) guide[k] = kGuidePairs;
    }
  }
}

static int plan_build(recoil_plan* P) {
  const uint32_t count = (uint32_t)P->streams.size();
  const bool per_stream = P->opts.flags & RECOIL_BATCH_PER_STREAM;
  const uint32_t warps = P->warps;
  for (const Stream* s : P->streams)
    if (!shape_supported(s->adaptive(), warps, P->lanes))
      return fail(RECOIL_EINVAL, P->lanes == 2 ? (s->adaptive() ? "two lanes a thread: adaptive streams decode with 8, 16 or 24 warps per CTA"
                                                                : "two lanes a thread: static streams decode with 4, 8 or 16 warps per CTA")
                                               : "adaptive streams decode with 4, 8, 16 or 32 warps per CTA");
  uint32_t guide[kKinds];
  choose_guides(P, guide);
  std::vector<DevStream> ds(count);
  std::vector<DevEntry> entries;
  struct ItemK { DevItem it; uint32_t kind; };
  std::vector<ItemK> items;
  size_t table_off = 0;
  uint64_t word_off = 0;
  P->word_off.resize(count);
  P->word_lo.assign(count, 0);
  P->word_cnt.assign(count, 0);
  P->tid_off.assign(count, 0);
  P->tid_lo.assign(count, 0);
  P->tid_cnt.assign(count, 0);
  P->stream_kind.resize(count);
  std::vector<std::pair<size_t, const std::vector<uint8_t>*>> tabs;
  for (uint32_t i = 0; i < count; i++) {
    const Stream& s = *P->streams[i];
    uint32_t kind = 0, slot_bytes = 0;
    const std::vector<uint8_t>& img = table_image(s, &kind, &slot_bytes);
    const uint32_t base_kind = kind;                  // the model's kind; the staged layout may pair it
    if (is_adaptive_kind(kind) && guide[kind] == kGuidePairs) kind = pair_kind_of(kind);
    DevStream& d = ds[i];
    std::memset(&d, 0, sizeof d);
    d.words = word_off;
    d.table = table_off;
    d.n_words = (uint32_t)s.n_words();
    d.n_bits = s.n_bits;
    d.kind = kind;
    d.alphabet = s.alphabet();
    d.sym_bytes = s.sym_bytes;
    d.table_bytes = (uint32_t)img.size();
    d.slot_bytes = slot_bytes;
    // staged words: all of them, or for a shard plan the window its run reads,
    // from the lowest word of the thread that stops at the run's low end
    // (recorded at encoding) to the highest split word of the run, in chunks
    uint64_t wlo = 0, whi = s.n_words();
    if (P->shard) {
      const uint32_t K = (uint32_t)s.entries.size() + 1;
      if (P->entry_first >= P->entry_last) {
        whi = 0;
      } else {
        if (P->entry_first > 0) wlo = s.entries[P->entry_first - 1].wlo / kChunkWords * kChunkWords;
        if (P->entry_last < K)
          whi = std::min<uint64_t>(s.n_words(), (s.entries[P->entry_last - 1].word / kChunkWords + 1) * kChunkWords);
        if (whi < wlo) whi = wlo;
      }
    }
    P->word_off[i] = word_off;
    P->word_lo[i] = wlo;
    P->word_cnt[i] = whi - wlo;
    P->stream_kind[i] = kind;
    tabs.push_back({table_off, &img});
    table_off += img.size();
    word_off += align_up(whi - wlo, kChunkWords);
    if (s.adaptive()) {
      // the table numbers follow the words, one byte per symbol, on a chunk
      // boundary; a shard plan stages those of the symbols its run decodes,
      // from its low end to the highest recorded index of its last split
      uint64_t tlo = 0, thi = s.n_syms;
      if (P->shard) {
        const uint32_t K = (uint32_t)s.entries.size() + 1;
        if (P->entry_first >= P->entry_last) {
          thi = 0;
        } else {
          if (P->entry_first > 0) {
            const Entry& e = s.entries[P->entry_first - 1];
            tlo = *std::min_element(e.idx, e.idx + kW) / (2 * kChunkWords) * (2 * kChunkWords);
          }
          if (P->entry_last < K) {
            const Entry& e = s.entries[P->entry_last - 1];
            thi = std::min<uint64_t>(s.n_syms, (uint64_t)*std::max_element(e.idx, e.idx + kW) + 1);
          }
          if (thi < tlo) thi = tlo;
        }
      }
      d.tid = (int64_t)word_off - (int64_t)(tlo / 2);
      d.n_tables = s.n_tables;
      {
        // stage the variant of the plan's guide width (or the paired layout)
        const uint32_t g = guide[base_kind];
        size_t voff = 0, vbytes = 0;
        guide_variant(s, g, &voff, &vbytes);
        d.table += voff;
        d.table_bytes = (uint32_t)vbytes;
        if (g == kGuidePairs) {
          d.row_stride = pair_block_words(s.alphabet(), s.n_bits);
          d.guide_bits = pair_guide_bits(s.n_bits);
          d.guide_stride = s.alphabet() * 4;
        } else {
          d.row_stride = adaptive_row_stride(s.alphabet());
          d.guide_bits = guide_bits(s.n_bits, g);
          d.guide_stride = guide_stride(s.n_bits, g, adaptive_guide_entry_bytes(base_kind));
        }
      }
      P->tid_off[i] = word_off;
      P->tid_lo[i] = tlo;
      P->tid_cnt[i] = thi - tlo;
      word_off += align_up((thi - tlo + 1) / 2, kChunkWords);
    }
    P->kind_smem[kind] = std::max<uint32_t>(P->kind_smem[kind], d.table_bytes);

    const size_t first = entries.size();
    build_entries(s, i, entries, wlo);
    size_t end_e = entries.size();
    if (P->shard) {
      end_e = first + P->entry_last;
    }
    // a stream whose tables equal the previous stream's may fill up the
    // previous stream's last work item (one staged table serves both)
    const bool same_table = i > 0 && !per_stream && !items.empty() && items.back().kind == kind &&
                            P->streams[i - 1]->n_bits == s.n_bits && P->streams[i - 1]->sym_bytes == s.sym_bytes &&
                            P->streams[i - 1]->n_tables == s.n_tables && P->streams[i - 1]->freq == s.freq &&
                            items.back().it.entry + items.back().it.count == first;
    size_t e = first + (P->shard ? P->entry_first : 0);
    // items of one CTA round: longer items (several rounds) leave longer tails
    // at the end of the queue and measured much slower on uneven batches
    const uint32_t cap = warps * P->lanes;
    if (same_table && !P->shard && items.back().it.count < cap) {
      const uint32_t take = (uint32_t)std::min<size_t>(cap - items.back().it.count, end_e - e);
      items.back().it.count += take;
      for (uint32_t k = 0; k < take; k++) items.back().it.work = std::max(items.back().it.work, entry_work(entries[e + k]));
      e += take;
    }
    for (; e < end_e; e += cap) {
      ItemK ik;
      ik.it.stream = i;
      ik.it.entry = (uint32_t)e;
      ik.it.count = (uint32_t)std::min<size_t>(cap, end_e - e);
      ik.it.work = 0;
      for (uint32_t k = 0; k < ik.it.count; k++) ik.it.work = std::max(ik.it.work, entry_work(entries[e + k]));
      ik.kind = kind;
      items.push_back(ik);
    }
  }
  for (uint32_t k = 0; k < kKinds; k++) {
    if (P->kind_smem[k] + warps * warp_smem(k, P->lanes, false) > kMaxSmem)
      return fail(RECOIL_EINVAL, "decoder tables too large for shared memory (alphabet or n too large)");
    // adaptive kinds at one lane a thread stage each steady block's table
    // numbers in shared memory where that still fits and keeps as many CTAs
    // resident; the L1 holds little next to their tables. Measured: paired
    // latents +4%, wide alphabets +9%; the one-byte-guide kinds over up to
    // 256 symbols -1 to -2%, so those keep the L1 path
    P->kind_staged[k] = 0;
    if (is_adaptive_kind(k) && k != kAdaptive8 && k != kAdaptive16 && P->lanes == 1 && P->kind_smem[k]) {
      const size_t plain = P->kind_smem[k] + warps * warp_smem(k, 1, false) + 16;
      const size_t staged = P->kind_smem[k] + warps * warp_smem(k, 1, true) + 16;
      if (staged <= kMaxSmem && adaptive_ctas_per_sm(warps, 1, staged) >= adaptive_ctas_per_sm(warps, 1, plain))
        P->kind_staged[k] = 1;
    }
  }
  // Kinds whose items all decode with one table (one stream, or streams with
  // identical models) are staged once per CTA; their entries become items of
  // one entry each that warps pop on their own, so no warp waits at a CTA
  // barrier for the slowest split of its item.
  const Stream* table_of[kKinds] = {};
  bool one_table[kKinds];
  for (uint32_t k = 0; k < kKinds; k++) one_table[k] = !per_stream;
  for (const ItemK& ik : items) {
    const Stream* st = P->streams[ik.it.stream];
    const Stream*& t = table_of[ik.kind];
    if (!t) t = st;
    else if (st != t && !(st->n_bits == t->n_bits && st->sym_bytes == t->sym_bytes && st->n_tables == t->n_tables &&
                          st->freq == t->freq))
      one_table[ik.kind] = false;
  }
  for (uint32_t k = 0; k < kKinds; k++) P->kind_warp_queue[k] = table_of[k] && one_table[k];
  {
    std::vector<ItemK> split;
    split.reserve(items.size());
    for (const ItemK& ik : items) {
      if (!P->kind_warp_queue[ik.kind]) {
        split.push_back(ik);
        continue;
      }
      for (uint32_t j = 0; j < ik.it.count; j++) {
        ItemK one = ik;
        one.it.entry = ik.it.entry + j;
        one.it.count = 1;
        one.it.work = entry_work(entries[ik.it.entry + j]);
        one.it.stream = entries[ik.it.entry + j].stream;
        split.push_back(one);
      }
    }
    items.swap(split);
  }
  // item order: by kind; persistent mode longest first, per-stream mode by stream
  const bool sort = !per_stream && !(P->opts.flags & RECOIL_BATCH_NO_SORT);
  std::stable_sort(items.begin(), items.end(), [&](const ItemK& a, const ItemK& b) {
    if (per_stream) return a.it.stream < b.it.stream;
    if (a.kind != b.kind) return a.kind < b.kind;
    return sort ? a.it.work > b.it.work : false;
  });
  P->n_items = (uint32_t)items.size();
  P->stream_item_first.assign(count, 0);
  P->stream_item_count.assign(count, 0);
  for (uint32_t k = 0; k < kKinds; k++) P->kind_count[k] = 0;
  for (uint32_t x = 0; x < P->n_items; x++) {
    const uint32_t k = items[x].kind, s = items[x].it.stream;
    if (P->kind_count[k] == 0) P->kind_first[k] = x;
    P->kind_count[k]++;
    if (P->stream_item_count[s] == 0) P->stream_item_first[s] = x;
    P->stream_item_count[s]++;
  }

  P->off_outs = sizeof(DevControl);
  P->off_streams = P->off_outs + align_up((size_t)count * 8, kAlign);
  P->off_items = P->off_streams + align_up((size_t)count * sizeof(DevStream), kAlign);
  P->off_entries = P->off_items + align_up(items.size() * sizeof(DevItem), kAlign);
  const size_t meta_bytes = P->off_entries + align_up(entries.size() * sizeof(DevEntry), kAlign);
  P->off_tables = align_up((size_t)(word_off + kChunkWords) * 2, kAlign);
  P->off_meta = P->off_tables + align_up(table_off, kAlign);
  P->ws_bytes = P->off_meta + meta_bytes;

  P->meta.assign(meta_bytes, 0);
  std::memcpy(P->meta.data() + P->off_streams, ds.data(), ds.size() * sizeof(DevStream));
  DevItem* it = reinterpret_cast<DevItem*>(P->meta.data() + P->off_items);
  for (size_t x = 0; x < items.size(); x++) it[x] = items[x].it;
  std::memcpy(P->meta.data() + P->off_entries, entries.data(), entries.size() * sizeof(DevEntry));
  P->tables.assign(align_up(table_off, 16), 0);
  for (auto& t : tabs) std::memcpy(P->tables.data() + t.first, t.second->data(), t.second->size());
  return RECOIL_OK;
}

namespace recoil {
void plan_image(const recoil_plan* P, PlanImage* o) {
  o->meta = P->meta.data();
  o->meta_bytes = P->meta.size();
  o->off_outs = P->off_outs;
  o->off_streams = P->off_streams;
  o->off_items = P->off_items;
  o->off_entries = P->off_entries;
  o->tables = P->tables.data();
  o->table_bytes = P->tables.size();
  o->ws_off_tables = P->off_tables;
  o->warps = P->warps;
  o->lanes = P->lanes;
  for (uint32_t k = 0; k < kKinds; k++) {
    o->kind_first[k] = P->kind_first[k];
    o->kind_count[k] = P->kind_count[k];
    o->kind_smem[k] = P->kind_smem[k];
    o->kind_warp_queue[k] = P->kind_warp_queue[k];
    o->kind_staged[k] = P->kind_staged[k];
  }
}
}  // namespace recoil

// SMs of the current device (148 on a B300 when no device can be asked).
static int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    return 148;
  }
  return sms;
}

// warps_per_cta 0: about one CTA round of splits per SM, i.e. the power of
// two nearest below splits / SMs, within [4, 16]. Few splits run faster in
// small CTAs spread over every SM (a split is one warp's dependent chain);
// measured on 1 GiB Zipf: 148-1184 splits +14-19% against 16-warp CTAs,
// 2368 and more within 1% of the best size. Adaptive streams with 64 or more
// splits an SM take 32-warp CTAs, one per SM, which leaves room for the finer
// guide (adaptive latents at 9472 splits: 1000 against 945 GB/s).
static uint32_t auto_warps(uint64_t splits, bool adaptive, bool big_lut, uint32_t lanes) {
  const uint64_t per_sm = splits / lanes / (uint64_t)device_sms();   // warps' worth of splits an SM
  if (adaptive && per_sm >= 64 / lanes) return lanes == 2 ? 24 : 32;
  // a 128 KB packed 16-bit LUT leaves room for one CTA an SM: make it 32 warps
  if (big_lut && lanes == 1 && per_sm >= 32) return 32;
  uint32_t w = adaptive && lanes == 2 ? 8 : 4;
  while (w < 16 && (uint64_t)w * 2 <= per_sm) w *= 2;
  return w;
}

// CTA sizes some kernel exists for (per kind checked by shape_supported).
static bool shape_warps_ok(uint32_t warps, uint32_t lanes) {
  return lanes == 2 ? (warps == 4 || warps == 8 || warps == 16 || warps == 24) : warps_supported(warps);
}

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(RECOIL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace recoil {
cudaError_t plan_upload_stream(const recoil_plan* P, size_t i, uint8_t* ws, cudaStream_t cs) {
  const Stream& s = *P->streams[i];
  cudaError_t e = cudaSuccess;
  if (P->word_cnt[i])
    e = cudaMemcpyAsync(ws + P->word_off[i] * 2, s.word_data() + P->word_lo[i], P->word_cnt[i] * 2,
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && s.adaptive() && P->tid_cnt[i])
    e = cudaMemcpyAsync(ws + P->tid_off[i] * 2, s.tid->data() + P->tid_lo[i], P->tid_cnt[i], cudaMemcpyHostToDevice, cs);
  return e;
}

size_t plan_bulk_bytes(const recoil_plan* P) { return P->off_meta; }

void plan_kernel_outs(const recoil_plan* P, void* const* outs, void** dev) {
  const size_t count = P->streams.size();
  for (size_t i = 0; i < count; i++) dev[i] = outs[i];
  if (P->shard && count == 1 && dev[0])            // the buffer starts at the first owned symbol
    dev[0] = (void*)((uintptr_t)dev[0] - P->out_shift * P->streams[0]->sym_bytes);
}

void plan_bulk_image(const recoil_plan* P, uint8_t* dst) {
  std::memset(dst, 0, P->off_meta);
  for (size_t i = 0; i < P->streams.size(); i++) {
    const Stream& s = *P->streams[i];
    if (P->word_cnt[i]) std::memcpy(dst + P->word_off[i] * 2, s.word_data() + P->word_lo[i], P->word_cnt[i] * 2);
    if (s.adaptive() && P->tid_cnt[i]) std::memcpy(dst + P->tid_off[i] * 2, s.tid->data() + P->tid_lo[i], P->tid_cnt[i]);
  }
  if (!P->tables.empty()) std::memcpy(dst + P->off_tables, P->tables.data(), P->tables.size());
}
const std::vector<const Stream*>& plan_streams(const recoil_plan* P) { return P->streams; }

int plan_upload_parts(recoil_plan* P, void* d_ws, size_t ws_bytes, cudaStream_t cs, bool bulk, bool meta) {
  if (!P || !d_ws) return fail(RECOIL_EINVAL, "null argument");
  if (ws_bytes < (meta ? P->ws_bytes : P->off_meta)) return fail(RECOIL_ENOMEM, "workspace too small");
  if (((uintptr_t)d_ws) % kAlign) return fail(RECOIL_EINVAL, "workspace must be 256-byte aligned");
  uint8_t* ws = (uint8_t*)d_ws;
  if (P->sms == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
  }
  cudaError_t e = cudaSuccess;
  if (meta) e = cudaMemcpyAsync(ws + P->off_meta, P->meta.data(), P->meta.size(), cudaMemcpyHostToDevice, cs);
  if (bulk) {
    if (e == cudaSuccess && !P->tables.empty())
      e = cudaMemcpyAsync(ws + P->off_tables, P->tables.data(), P->tables.size(), cudaMemcpyHostToDevice, cs);
    for (size_t i = 0; e == cudaSuccess && i < P->streams.size(); i++) e = plan_upload_stream(P, i, ws, cs);
  }
  if (e != cudaSuccess) return cuda_fail(e, "upload");
  if (P->d_ws != ws && P->graph) {
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  P->d_ws = ws;
  P->uploaded = true;
  P->outs_on_device = false;
  return RECOIL_OK;
}
}  // namespace recoil

static int plan_launch(recoil_plan* P, cudaStream_t cs) {
  P->launches = 0;
  uint8_t* meta = P->d_ws + P->off_meta;
  DevControl* ctl = reinterpret_cast<DevControl*>(meta);
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(DevControl), cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  LaunchArgs a{};
  a.streams = reinterpret_cast<const DevStream*>(meta + P->off_streams);
  a.entries = reinterpret_cast<const DevEntry*>(meta + P->off_entries);
  a.word_pool = reinterpret_cast<const uint16_t*>(P->d_ws);
  a.table_pool = P->d_ws + P->off_tables;
  a.outs = reinterpret_cast<void* const*>(meta + P->off_outs);
  a.control = ctl;
  a.warps = P->warps;
  a.lanes = P->lanes;
  const DevItem* items = reinterpret_cast<const DevItem*>(meta + P->off_items);
  if (P->opts.flags & RECOIL_BATCH_PER_STREAM) {
    for (size_t s = 0; s < P->streams.size(); s++) {
      if (!P->stream_item_count[s]) continue;
      const uint32_t k = P->stream_kind[s];
      a.items = items + P->stream_item_first[s];
      a.n_items = P->stream_item_count[s];
      a.kind = k;
      a.persistent = 0;
      a.table_smem = (uint32_t)align_up(P->kind_smem[k], 16);
      e = launch_decode(k, a, a.n_items, cs);
      if (e != cudaSuccess) return cuda_fail(e, "decode launch");
      P->launches++;
    }
    return RECOIL_OK;
  }
  for (uint32_t k = 0; k < kKinds; k++) {
    if (!P->kind_count[k]) continue;
    a.items = items + P->kind_first[k];
    a.n_items = P->kind_count[k];
    a.kind = k;
    a.persistent = 1;
    a.table_smem = (uint32_t)align_up(P->kind_smem[k], 16);
    a.warp_queue = P->kind_warp_queue[k];
    a.tid_staged = P->kind_staged[k];
    int per_sm = (int)P->opts.ctas_per_sm;
    if (per_sm <= 0 && occupancy_ctas_per_sm(k, P->warps, P->lanes, a.tid_staged != 0, a.table_smem, &per_sm) != 0)
      return fail(RECOIL_ECUDA, "occupancy query failed");
    if (per_sm <= 0) return fail(RECOIL_EINVAL, "kernel does not fit on an SM with these options");
    const unsigned grid = launch_grid(a, per_sm, P->sms);
    e = launch_decode(k, a, grid, cs);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    P->launches++;
  }
  return RECOIL_OK;
}

extern "C" {

int recoil_plan_create(const recoil_stream* const* streams, uint32_t count, const recoil_batch_opts* opts,
                       recoil_plan** out) {
  clear_error();
  if (!out || (count && !streams)) return fail(RECOIL_EINVAL, "null argument");
  *out = nullptr;
  try {
    std::unique_ptr<recoil_plan> P(new recoil_plan());
    if (opts) P->opts = *opts;
    P->warps = P->opts.warps_per_cta;
    P->lanes = (P->opts.flags & RECOIL_BATCH_TWO_LANES) ? 2 : 1;
    if (!P->warps) {
      uint64_t splits = 0;
      bool adaptive = count > 0, big_lut = false;
      for (uint32_t i = 0; i < count; i++) {
        if (!streams[i]) return fail(RECOIL_EINVAL, "null stream");
        splits += P->opts.split_symbols
                      ? std::max<uint64_t>(1, (streams[i]->n_syms + P->opts.split_symbols - 1) / P->opts.split_symbols)
                      : streams[i]->entries.size() + 1;
        adaptive = adaptive && streams[i]->adaptive();
        big_lut = big_lut || (table_kind_of(*streams[i]) == kPacked16 && streams[i]->n_bits >= 15);
      }
      P->warps = auto_warps(splits, adaptive, big_lut, P->lanes);
    }
    if (!shape_warps_ok(P->warps, P->lanes))
      return fail(RECOIL_EINVAL, P->lanes == 2 ? "two lanes a thread: warps_per_cta must be 4, 8, 16 or 24"
                                               : "warps_per_cta must be 1, 2, 4, 8, 16 or 32");
    for (uint32_t i = 0; i < count; i++) {
      if (!streams[i]) return fail(RECOIL_EINVAL, "null stream");
      const recoil_stream* s = streams[i];
      if (P->opts.split_symbols) {
        // about split_symbols per split, rounded up to whole CTAs so that every
        // work item keeps all its warps busy on splits of equal size
        uint64_t want = std::max<uint64_t>(1, (s->n_syms + P->opts.split_symbols - 1) / P->opts.split_symbols);
        const uint64_t per_cta = (uint64_t)P->warps * P->lanes;
        want = (want + per_cta - 1) / per_cta * per_cta;
        recoil_stream* c = nullptr;
        int rc = recoil_combine_splits(s, (uint32_t)std::min<uint64_t>(want, 0xffffffffu), &c);
        if (rc) return rc;
        P->owned.emplace_back(c);
        P->streams.push_back(c);
      } else {
        P->streams.push_back(s);
      }
    }
    int rc = plan_build(P.get());
    if (rc) return rc;
    *out = P.release();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

int recoil_plan_workspace_size(const recoil_plan* P, size_t* bytes) {
  clear_error();
  if (!P || !bytes) return fail(RECOIL_EINVAL, "null argument");
  *bytes = P->ws_bytes;
  return RECOIL_OK;
}

int recoil_plan_upload(recoil_plan* P, void* d_ws, size_t ws_bytes, void* stream) {
  clear_error();
  return plan_upload_parts(P, d_ws, ws_bytes, (cudaStream_t)stream, true, true);
}

int recoil_plan_decode(recoil_plan* P, void* const* d_outs, void* stream) {
  clear_error();
  if (!P || (!d_outs && !P->streams.empty())) return fail(RECOIL_EINVAL, "null argument");
  if (!P->uploaded) return fail(RECOIL_EINVAL, "plan not uploaded");
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t count = P->streams.size();
  bool same = P->outs_on_device && P->outs.size() == count;
  for (size_t i = 0; same && i < count; i++) same = P->outs[i] == d_outs[i];
  if (!same) {
    for (size_t i = 0; i < count; i++)
      if (!d_outs[i] && P->streams[i]->n_syms && !(P->shard && P->n_items == 0))
        return fail(RECOIL_EINVAL, "null output buffer");
    P->outs.assign(d_outs, d_outs + count);
    P->outs_dev.resize(count);
    plan_kernel_outs(P, d_outs, P->outs_dev.data());
    cudaError_t e = cudaMemcpyAsync(P->d_ws + P->off_meta + P->off_outs, P->outs_dev.data(), count * 8,
                                    cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "output pointer upload");
    P->outs_on_device = true;
  }
  const bool use_graph = (P->opts.flags & RECOIL_BATCH_GRAPH) && cs != nullptr &&
                         !(P->opts.flags & RECOIL_BATCH_PER_STREAM);
  if (!use_graph) return plan_launch(P, cs);
  if (!P->graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    int rc = plan_launch(P, cs);
    e = cudaStreamEndCapture(cs, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&P->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  }
  cudaError_t e = cudaGraphLaunch(P->graph, cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return RECOIL_OK;
}

int recoil_plan_errors(recoil_plan* P, void* stream, uint32_t* flags) {
  clear_error();
  if (!P || !flags) return fail(RECOIL_EINVAL, "null argument");
  if (!P->uploaded) return fail(RECOIL_EINVAL, "plan not uploaded");
  DevControl c;
  cudaError_t e = cudaMemcpyAsync(&c, P->d_ws + P->off_meta, sizeof c, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "error readback");
  *flags = c.errors;
  if (c.errors)
    return fail(RECOIL_ECORRUPT, "decoder found an inconsistent stream (flags " + std::to_string(c.errors) +
                                     ", entry " + std::to_string((long long)c.bad_entry - 1) + ")");
  return RECOIL_OK;
}

uint32_t recoil_plan_launches(const recoil_plan* P) { return P ? P->launches : 0; }

uint32_t recoil_plan_warps_per_cta(const recoil_plan* P) { return P ? P->warps : 0; }

uint32_t recoil_plan_kernels(const recoil_plan* P) {
  if (!P) return 0;
  uint32_t m = 0;
  for (uint32_t k = 0; k < kKinds; k++)
    if (P->kind_count[k]) m |= 1u << k;
  return m;
}

void recoil_plan_free(recoil_plan* P) { delete P; }

int recoil_workspace_size(const recoil_stream* const* streams, uint32_t count, const recoil_batch_opts* opts,
                          size_t* bytes) {
  recoil_plan* P = nullptr;
  int rc = recoil_plan_create(streams, count, opts, &P);
  if (rc) return rc;
  rc = recoil_plan_workspace_size(P, bytes);
  recoil_plan_free(P);
  return rc;
}

int recoil_decode_batch(const recoil_stream* const* streams, uint32_t count, void* const* d_outs, void* d_ws,
                        size_t ws_bytes, void* stream, const recoil_batch_opts* opts) {
  recoil_plan* P = nullptr;
  int rc = recoil_plan_create(streams, count, opts, &P);
  if (rc) return rc;
  recoil_batch_opts o = P->opts;
  o.flags &= ~RECOIL_BATCH_GRAPH;                 // a one-shot plan has nothing to replay
  P->opts = o;
  rc = recoil_plan_upload(P, d_ws, ws_bytes, stream);
  if (!rc) rc = recoil_plan_decode(P, d_outs, stream);
  recoil_plan_free(P);
  return rc;
}

int recoil_shard(const recoil_stream* const* streams, uint32_t count, uint32_t world, uint32_t* rank_of) {
  clear_error();
  if (!rank_of || world < 1 || (count && !streams)) return fail(RECOIL_EINVAL, "null argument or world < 1");
  std::vector<uint32_t> order(count);
  for (uint32_t i = 0; i < count; i++) {
    if (!streams[i]) return fail(RECOIL_EINVAL, "null stream");
    order[i] = i;
  }
  auto bytes = [&](uint32_t i) { return streams[i]->n_syms * streams[i]->sym_bytes; };
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return bytes(a) > bytes(b); });
  std::vector<uint64_t> load(world, 0);
  for (uint32_t i : order) {
    uint32_t r = 0;
    for (uint32_t k = 1; k < world; k++)
      if (load[k] < load[r]) r = k;
    rank_of[i] = r;
    load[r] += bytes(i);
  }
  return RECOIL_OK;
}

int recoil_plan_create_shard(const recoil_stream* s, uint32_t world, uint32_t rank, const recoil_batch_opts* opts,
                             recoil_plan** out, uint64_t* sym_lo, uint64_t* sym_hi) {
  clear_error();
  if (!s || !out || !sym_lo || !sym_hi || world < 1 || rank >= world)
    return fail(RECOIL_EINVAL, "null argument, world < 1 or rank >= world");
  if (opts && opts->split_symbols) return fail(RECOIL_EINVAL, "combine the stream before sharding (split_symbols must be 0)");
  *out = nullptr;
  try {
    // owned ranges of the kept entries: entry k owns [m_{k-1}, m_k), the final one up to N
    std::vector<DevEntry> ents;
    build_entries(*s, 0, ents);
    const uint32_t K = (uint32_t)ents.size();
    // run boundaries: rank r starts at the first entry whose owned range ends
    // past r * N / world (contiguous, monotone, every entry in exactly one run)
    auto start_of = [&](uint32_t r) -> uint32_t {
      if (r == 0) return 0;
      if (r >= world) return K;
      const uint64_t target = (uint64_t)s->n_syms * r / world;
      uint32_t k = 0;
      while (k < K && (uint64_t)ents[k].hi1 <= target) k++;
      return k;
    };
    const uint32_t first = start_of(rank), last = start_of(rank + 1);
    *sym_lo = first < K ? ents[first].lo : s->n_syms;
    *sym_hi = last < K ? ents[last].lo : s->n_syms;
    if (first >= last) *sym_hi = *sym_lo;
    std::unique_ptr<recoil_plan> P(new recoil_plan());
    if (opts) P->opts = *opts;
    P->lanes = (P->opts.flags & RECOIL_BATCH_TWO_LANES) ? 2 : 1;
    P->warps = P->opts.warps_per_cta ? P->opts.warps_per_cta
                                     : auto_warps(std::max(first, last) - first, s->adaptive(),
                                                  table_kind_of(*s) == kPacked16 && s->n_bits >= 15, P->lanes);
    if (!shape_warps_ok(P->warps, P->lanes))
      return fail(RECOIL_EINVAL, P->lanes == 2 ? "two lanes a thread: warps_per_cta must be 4, 8, 16 or 24"
                                               : "warps_per_cta must be 1, 2, 4, 8, 16 or 32");
    P->streams.push_back(s);
    P->shard = true;
    P->entry_first = first;
    P->entry_last = std::max(first, last);
    P->out_shift = *sym_lo;
    int rc = plan_build(P.get());
    if (rc) return rc;
    *out = P.release();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

int recoil_decode(const recoil_stream* s, void* d_out, void* d_ws, size_t ws_bytes, void* stream) {
  const recoil_stream* ss[1] = {s};
  void* outs[1] = {d_out};
  return recoil_decode_batch(ss, 1, outs, d_ws, ws_bytes, stream, nullptr);
}

}  // extern "C"
