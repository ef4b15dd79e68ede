// Recoil split decoders for sm_103a.
//
// One warp decodes one split entry; lane j is interleaved coder j (Sec. 2.2,
// W = 32 matches the warp, Sec. 4.4). Per group step (32 symbols, decreasing
// index) every lane:
//   decode   slot = x mod 2^n, table lookup, x = f (x >> n) + slot - F   (Eq. 2)
//   renorm   coders with x < L read one 16-bit word each (Eq. 4, one step
//            since b >= n): the warp ballots the need mask, lane j takes the
//            word p - popc(mask above j) because decoders read in decreasing
//            coder order (Sec. 2.2), and p drops by popc(mask).
// A coder joins when the walk reaches one past its recorded symbol (takes the
// recorded state and renormalises at once, Sec. 4.1.1); groups before every
// coder has joined are walked with per-lane predicates, the steady middle
// without. The walk continues into the previous split's synchronisation
// section and stops at the owned low end (Sec. 4.1.2, 4.1.3).
//
// Memory: decoder tables are staged in shared memory once per work item
// (Sec. 4.4 packs symbol, f and F into one 32-bit entry for 8-bit symbols and
// n <= 12; adaptive models stage one CDF row and one bucket guide per PDF,
// Sec. 3.1); the
// compressed words a warp is about to consume sit in a per-warp shared ring
// refilled 512 bytes at a time with one 16-byte load per lane, issued a chunk
// ahead so that the dependent renormalisation reads never wait on HBM.
// Symbol stores are one coalesced 32-byte (or 64-byte) warp store per group
// step.
//
// Scheduling: persistent CTAs pop work items (up to `warps` entries of one
// stream) from a device counter and their warps take the item's entries from
// a shared counter; a CTA restages tables only when the stream changes. When
// one table serves the whole launch, every entry is an item of its own and
// each warp pops items alone (no CTA barrier between splits). Every loop is
// bounded by the entry's group range, every word read comes from the shared
// ring (in bounds by construction) and every global load of a chunk is
// guarded by the chunk index, so a corrupt stream yields an error flag, never
// a fault or a hang.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "device_types.h"

namespace recoil {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTidBlock = 8 * kW;       // table numbers of one steady block (8 group steps)
constexpr int kTidSlots = 3;            // staged blocks a warp keeps: current, next, the one after

__device__ __forceinline__ uint32_t lanemask_gt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_gt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------- tables

template <uint32_t KIND>
struct Tables;

// bias | sym << 12 | f << 20  (bias = slot - F < f < 4096)
template <>
struct Tables<kPacked8> {
  const uint32_t* lut;
  __device__ __forceinline__ void bind(const unsigned char* smem, const DevStream&) {
    lut = reinterpret_cast<const uint32_t*>(smem);
  }
  __device__ __forceinline__ uint32_t step(uint32_t& x, uint32_t n, uint32_t mask) const {
    const uint32_t e = lut[x & mask];
    x = (e >> 20) * (x >> n) + (e & 0xfffu);
    return e >> 12;                        // low byte is the symbol
  }
};

// bias | f << 10 | sym << 20  (16-bit symbols below 2^12, bias = slot - F < f < 2^10)
template <>
struct Tables<kPacked16> {
  const uint32_t* lut;
  __device__ __forceinline__ void bind(const unsigned char* smem, const DevStream&) {
    lut = reinterpret_cast<const uint32_t*>(smem);
  }
  __device__ __forceinline__ uint32_t step(uint32_t& x, uint32_t n, uint32_t mask) const {
    const uint32_t e = lut[x & mask];
    x = ((e >> 10) & 0x3ffu) * (x >> n) + (e & 0x3ffu);
    return e >> 20;
  }
};

// u16 slot -> symbol, then u32 symbol -> (f - 1) << 16 | F
template <uint32_t KIND>
struct Tables {
  const uint16_t* slot_sym;
  const uint32_t* symtab;
  __device__ __forceinline__ void bind(const unsigned char* smem, const DevStream& st) {
    slot_sym = reinterpret_cast<const uint16_t*>(smem);
    symtab = reinterpret_cast<const uint32_t*>(smem + st.slot_bytes);
  }
  __device__ __forceinline__ uint32_t step(uint32_t& x, uint32_t n, uint32_t mask) const {
    const uint32_t slot = x & mask;
    const uint32_t s = slot_sym[slot];
    const uint32_t e = symtab[s];
    x = ((e >> 16) + 1u) * (x >> n) + slot - (e & 0xffffu);
    return s;
  }
};

// Adaptive model (Sec. 3.1): symbol i is coded with PDF row tid[i]. Row t
// holds H(s) = F(s) - 1 modulo 2^16 of PDF t for s = 0..A (H(0) = 0xffff,
// H(A) = 2^n - 1): the symbol is the last s with F(s) <= slot, i.e. with
// H(s) < slot for s >= 1; then F(s) = H(s) + 1 and f = H(s+1) - H(s), both
// modulo 2^16 and exact since every f of an adaptive model is below 2^16.
//
// The row's guide holds, for each of 2^g equal buckets of slots, the symbol
// owning the bucket's first slot (G: one byte for alphabets up to 256, else
// two), then the owner of the last slot; the symbol of `slot` lies between
// the entries of its bucket and the next, and a binary search narrows that
// range (usually empty: one lookup; with g = 0 it is the whole row).
template <typename G>
struct AdaptiveTables {
  const uint16_t* cdf;
  const G* guide;
  uint32_t stride, gstride, gshift;
  __device__ __forceinline__ void bind(const unsigned char* smem, const DevStream& st) {
    cdf = reinterpret_cast<const uint16_t*>(smem);
    guide = reinterpret_cast<const G*>(smem + (size_t)st.n_tables * st.row_stride * 2);
    stride = st.row_stride;
    gstride = st.guide_stride / sizeof(G);
    gshift = st.n_bits > st.guide_bits ? st.n_bits - st.guide_bits : 0;
  }
  __device__ __forceinline__ uint32_t step(uint32_t& x, uint32_t n, uint32_t mask, uint32_t t) const {
    const uint32_t slot = x & mask;
    const uint16_t* row = cdf + t * stride;
    const G* gb = guide + t * gstride + (slot >> gshift);
    uint32_t s = gb[0];
    uint32_t hi = gb[1];
    while (s < hi) {                                    // bounded: hi - s halves
      const uint32_t mid = (s + hi + 1) >> 1;
      if (row[mid] < slot) s = mid; else hi = mid - 1;
    }
    const uint32_t h0 = row[s];
    const uint32_t f = (row[s + 1] - h0) & 0xffffu;
    x = f * (x >> n) + slot - ((h0 + 1u) & 0xffffu);
    return s;
  }
};

// Adaptive model, paired layout (alphabets up to 256): one block per PDF row
// t, holding for every symbol s the u32 F(s) | H(s+1) << 16, with H as above
// (F(s) < 2^16 for every symbol that can be decoded: its f is at least one),
// then the guide: a byte per bucket boundary, the symbol owning the first
// slot of each of 2^10 buckets and the owner of the last slot. One guide read
// gives the bracket's low end s; row[s] and row[s+1], read together, give
// F(s) and f(s) of s and of s + 1, and H(s+1) (the high half of row[s])
// decides between the two without a branch. Only a bracket of three or more
// symbols whose symbol lies past s + 1 (under 2% of warp steps on Gaussian
// rows) reads the bracket's high end and bisects.
struct PairTables {
  const unsigned char* blocks;
  uint32_t bstride, goff, gshift;
  __device__ __forceinline__ void bind(const unsigned char* smem, const DevStream& st) {
    blocks = smem;
    bstride = st.row_stride * 4;
    goff = st.guide_stride;
    gshift = st.n_bits > st.guide_bits ? st.n_bits - st.guide_bits : 0;
  }
  __device__ __forceinline__ uint32_t step(uint32_t& x, uint32_t n, uint32_t mask, uint32_t t) const {
    const uint32_t slot = x & mask;
    const unsigned char* blk = blocks + t * bstride;
    const uint32_t* row = reinterpret_cast<const uint32_t*>(blk);
    const uint8_t* gb = blk + goff + (slot >> gshift);
    uint32_t s = gb[0];
    uint32_t p = row[s];
    const uint32_t p1 = row[s + 1];                     // s = A - 1: p's H(A) = 2^n - 1 keeps s
    const bool up = (p >> 16) < slot;
    s += up ? 1u : 0u;
    p = up ? p1 : p;
    if ((p >> 16) < slot) {                             // past s + 1: bisect up to the bracket's end
      const uint16_t* low = reinterpret_cast<const uint16_t*>(row);   // F(s) at low[2 s] (little-endian)
      uint32_t a = s + 1, b = gb[1];
      while (a < b) {                                   // bounded: b - a halves
        const uint32_t mid = (a + b + 1) >> 1;
        if (low[2 * mid] <= slot) a = mid; else b = mid - 1;
      }
      s = a;
      p = row[s];
    }
    const uint32_t F = p & 0xffffu;
    const uint32_t f = (p >> 16) + 1u - F;
    x = f * (x >> n) + (slot - F);
    return s;
  }
};

template <uint32_t KIND>
__host__ __device__ constexpr bool is_adaptive() {
  return is_adaptive_kind(KIND);
}

// Decoder tables of a kind.
template <uint32_t KIND, bool ADAPTIVE = is_adaptive_kind(KIND)>
struct TablesOf {
  using T = Tables<KIND>;
};
template <uint32_t KIND>
struct TablesOf<KIND, true> {
  using T = typename std::conditional<
      is_pair_kind(KIND), PairTables,
      AdaptiveTables<typename std::conditional<adaptive_guide_entry_bytes(KIND) == 2, uint16_t, uint8_t>::type>>::type;
};

template <uint32_t KIND>
struct SymOut {
  using T = uint8_t;
};
template <>
struct SymOut<kGeneric16> {
  using T = uint16_t;
};
template <>
struct SymOut<kAdaptive16> {
  using T = uint16_t;
};
template <>
struct SymOut<kAdaptive16Wide> {
  using T = uint16_t;
};
template <>
struct SymOut<kAdaptive16Pair> {
  using T = uint16_t;
};
template <>
struct SymOut<kPacked16> {
  using T = uint16_t;
};

__device__ __forceinline__ uint32_t smem_addr32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bring the cache line of p into L1 (no register, no wait).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" : : "l"(p));
}

// Asynchronous 8-byte global-to-shared copies (completion tracked per thread
// in commit groups).
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" : : "r"(smem_addr32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" : : : "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" : : "n"(N) : "memory"); }

// A read-only load kept where it is written (volatile asm is neither merged
// with an earlier load of the same address nor hoisted).
__device__ __forceinline__ int ld_keep(const int* p) {
  int v;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// ------------------------------------------------------------- word ring
// Word w of the stream sits at ring[(w mod 512)] and ring[(w mod 512) + 512];
// with rp = (p mod 512) + 512, word p - k (0 <= k < 32) is ring[rp - k] for
// any p, and rp drifts down by at most 256 between normalisations (8 steps
// of at most 32 words), so reads stay inside the ring.

__device__ __forceinline__ uint4 load_chunk(const uint16_t* __restrict__ words, int chunk, int lane) {
  if (chunk < 0) return make_uint4(0, 0, 0, 0);
  const uint4* src = reinterpret_cast<const uint4*>(words + (size_t)chunk * kChunkWords) + lane;
  return __ldg(src);
}

__device__ __forceinline__ void put_chunk(uint16_t* ring, int chunk, int lane, uint4 v) {
  const int off = (chunk & 1) * kChunkWords + lane * 8;
  *reinterpret_cast<uint4*>(ring + off) = v;
  *reinterpret_cast<uint4*>(ring + off + kRingWords) = v;
}

struct Walker {
  uint32_t x;          // coder state
  int p;               // next word to read (stream index), uniform
  int rp;              // ring position of word p, uniform
  int cbase;           // first word of the chunk holding p (ring holds cbase-256 .. cbase+255)
  uint4 pre;           // prefetched chunk (cbase/256 - 2)
};

template <uint32_t KIND>
struct EntryDecoder {
  typename TablesOf<KIND>::T T;
  const uint16_t* __restrict__ words;
  const uint8_t* __restrict__ tid;     // adaptive kinds: PDF row of every symbol index
  uint8_t* tbuf;                       // adaptive kinds, one lane a thread: kTidSlots staged blocks of table numbers
  bool staged;                         // the launch stages table numbers in tbuf (else they come through L1)
  uint16_t* ring;
  typename SymOut<KIND>::T* __restrict__ out;
  uint32_t n, mask, gt;
  int lane;

  // Eq. 2 for symbol i (the table row is the symbol's own under an adaptive model)
  __device__ __forceinline__ uint32_t dec(uint32_t& x, int i) const {
    if constexpr (is_adaptive<KIND>())
      return T.step(x, n, mask, __ldg(tid + i));
    else
      return T.step(x, n, mask);
  }

  // Eq. 2 for symbol i with its table number from the staged buffer at byte
  // toff (toff >= 0), else read like dec does
  __device__ __forceinline__ uint32_t dec_at(uint32_t& x, int i, int toff) const {
    if constexpr (is_adaptive<KIND>())
      return T.step(x, n, mask, toff >= 0 ? (uint32_t)tbuf[toff] : (uint32_t)__ldg(tid + i));
    else
      return T.step(x, n, mask);
  }

  // Where this lane's table number of group gg sits in the staged buffer when
  // it holds the kTidSlots blocks of 8 groups from group go down, the first in
  // slot b0 and the next ones in the slots after it (wrapping); -1 if outside.
  __device__ __forceinline__ int toff_of(int go, int b0, int gg) const {
    const int off = go - gg;
    if (off < 0 || off >= kTidSlots * 8) return -1;
    int slot = b0 + (off >> 3);
    if (slot >= kTidSlots) slot -= kTidSlots;
    return slot * kTidBlock + (7 - (off & 7)) * kW + lane;
  }

  __device__ __forceinline__ void refill(Walker& w) {
    __syncwarp();
    const int cnew = (w.cbase >> 8) - 2;
    if (cnew >= 0) put_chunk(ring, cnew, lane, w.pre);
    w.cbase -= kChunkWords;
    w.pre = load_chunk(words, cnew - 1, lane);
    __syncwarp();
  }

  // Eq. 4 for the whole warp: coders with `need` read their word in decreasing
  // coder order. Only the ring position moves; callers catch p up from it.
  __device__ __forceinline__ void renorm(Walker& w, bool need) {
    const uint32_t m = __ballot_sync(kFull, need);
    if (need) {
      const int k = __popc(m & gt);
      w.x = (w.x << 16) | ring[w.rp - k];
    }
    w.rp -= __popc(m);
  }

  // Bring p up to date with the ring position (rp0 = ring position when p was
  // last exact), renormalise the ring position and refill if p left the chunk.
  __device__ __forceinline__ void settle(Walker& w, int rp0) {
    w.p -= rp0 - w.rp;
    w.rp = (w.p & (kRingWords - 1)) + kRingWords;
    if (w.p < w.cbase) refill(w);
  }

  // A group step with per-lane predicates (synchronisation phase and range edges).
  // At the group where coder j of the previous entry joined (act_p), the
  // state right after decoding must be that entry's recorded state x_p: the
  // previous split's metadata is exactly the state this thread carries across
  // the boundary (Sec. 3.1, 4.1.3), so any corrupt word or state shows here.
  __device__ __forceinline__ void pstep(Walker& w, int g, int act, uint32_t x0, int lo, int hi1,
                                        int act_p, uint32_t x_p, bool& bad, int toff = -1) {
    const int i = g * kW + lane;
    const bool dec = (g < act) && (i >= lo);
    const bool join = (g == act);
    if (dec) {
      const uint32_t s = this->dec_at(w.x, i, toff);
      if (i < hi1) out[i] = (typename SymOut<KIND>::T)s;
    }
    if (join) w.x = x0;
    if (g == act_p && w.x != x_p) bad = true;
    const int rp0 = w.rp;
    renorm(w, (dec || join) && w.x < kL);
    settle(w, rp0);
  }

  // Adaptive kinds stage table numbers in shared memory with asynchronous
  // copies, in blocks of 8 groups (256 bytes, 8 per lane): the per-symbol
  // read is then a shared read, not an L1 miss (the L1 holds little next to
  // the tables). The steady loop stages two blocks ahead; the synchronisation
  // phase at the top and the groups below the steady loop read blocks staged
  // beforehand. Chunks of groups below glo (the walk's lowest group) are not
  // copied; every call commits one group so the waits can count blocks.
  __device__ __forceinline__ void stage_tids(int gtop, int glo, int slot) {
    if (gtop - 7 + (lane >> 2) >= glo)
      cp_async8(tbuf + slot * kTidBlock + lane * 8, tid + (size_t)(gtop - 7) * kW + lane * 8);
    cp_async_commit();
  }

  // A group step where every coder decodes and every symbol is owned (i: its index).
  __device__ __forceinline__ void sstep(Walker& w, typename SymOut<KIND>::T* o, int i) {
    const uint32_t s = dec(w.x, i);
    *o = (typename SymOut<KIND>::T)s;
    renorm(w, w.x < kL);
  }

  // Where one split's walk stands between its phases.
  struct Span {
    int g;             // next group to visit (decreasing)
    int steady_lo;     // lowest group of the steady loop
    bool bad;          // a state differed from the previous entry's record
  };

  // Prologue and synchronisation phase of entry `ent`: stages its first word
  // chunks and walks the groups before every coder has joined, leaving g at
  // the first group of the steady loop. False for an empty owned range.
  __device__ __forceinline__ bool begin(const DevEntry* __restrict__ ent, Walker& w, Span& sp) {
    const int lo = (int)ent->lo, hi1 = (int)ent->hi1;
    if (lo >= hi1) return false;
    const int act = ent->act[lane];
    const uint32_t x0 = ent->x0[lane];
    int g = ent->g_top;

    w.x = 0;
    w.p = ent->q;
    w.cbase = (w.p >> 8) << 8;                       // p = -1 gives -256: nothing staged
    {
      const int c = w.cbase >> 8;
      const uint4 a = load_chunk(words, c, lane);
      const uint4 b = load_chunk(words, c - 1, lane);
      if (c >= 0) put_chunk(ring, c, lane, a);
      if (c >= 1) put_chunk(ring, c - 1, lane, b);
      w.pre = load_chunk(words, c - 2, lane);
    }
    __syncwarp();
    w.rp = (w.p & (kRingWords - 1)) + kRingWords;

    const int g_full = __reduce_min_sync(kFull, act);            // below it every coder has joined
    const int steady_hi = min(g_full - 1, (hi1 >> 5) - 1);       // whole groups owned ...
    // the previous entry of the same stream (there is one whenever lo > 0)
    int act_p = -1, gtop_p = -1;
    uint32_t x_p = 0;
    if (lo > 0) {
      act_p = ent[-1].act[lane];
      x_p = ent[-1].x0[lane];
      gtop_p = ent[-1].g_top;
    }
    sp.steady_lo = max((lo + kW - 1) >> 5, gtop_p + 1);          // ... fully decodable, above the check
    sp.bad = false;
    for (; g > steady_hi && g >= (lo >> 5); --g) pstep(w, g, act, x0, lo, hi1, act_p, x_p, sp.bad);
    sp.g = g;
    return true;
  }

  // One block of 8 steady group steps (the caller checks g - 7 >= steady_lo).
  // 8 steps consume at most 256 words: with p >= cbase at the start of a
  // block, every read stays inside the two staged chunks.
  __device__ __forceinline__ void block(Walker& w, Span& sp) {
    const int rp0 = w.rp;
    const int i0 = sp.g * kW + lane;
    typename SymOut<KIND>::T* o = out + (size_t)sp.g * kW + lane;
    // adaptive: table numbers of the block after next into L1 (256 bytes, 8 per lane),
    // only of groups this walk decodes (a shard plan stages no others)
    if constexpr (is_adaptive<KIND>())
      if (sp.g - 23 >= sp.steady_lo) prefetch_l1(tid + (sp.g - 23) * kW + lane * 8);
#pragma unroll
    for (int u = 0; u < 8; ++u) sstep(w, o - u * kW, i0 - u * kW);
    sp.g -= 8;
    settle(w, rp0);
  }

  // Two splits' blocks in lockstep, step by step: two independent chains of
  // dependent table and word reads for the scheduler to overlap.
  __device__ __forceinline__ void block2(Walker& w, Span& sp, EntryDecoder& B, Walker& wb, Span& sb) {
    const int rp0 = w.rp, rpb0 = wb.rp;
    const int i0 = sp.g * kW + lane, ib0 = sb.g * kW + lane;
    typename SymOut<KIND>::T* o = out + (size_t)sp.g * kW + lane;
    typename SymOut<KIND>::T* ob = B.out + (size_t)sb.g * kW + lane;
    if constexpr (is_adaptive<KIND>()) {
      if (sp.g - 23 >= sp.steady_lo) prefetch_l1(tid + (sp.g - 23) * kW + lane * 8);
      if (sb.g - 23 >= sb.steady_lo) prefetch_l1(B.tid + (sb.g - 23) * kW + lane * 8);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      sstep(w, o - u * kW, i0 - u * kW);
      B.sstep(wb, ob - u * kW, ib0 - u * kW);
    }
    sp.g -= 8;
    sb.g -= 8;
    settle(w, rp0);
    B.settle(wb, rpb0);
  }

  // The rest of a walk: steady blocks, single steady steps, the predicated
  // tail down to the owned low end, and the end checks.
  __device__ __forceinline__ void finish(const DevEntry* __restrict__ ent, Walker& w, Span& sp, DevControl* ctl,
                                         uint32_t entry_id) {
    while (sp.g - 7 >= sp.steady_lo) block(w, sp);
    int g = sp.g;
    if (g >= sp.steady_lo) {
      typename SymOut<KIND>::T* o = out + (size_t)g * kW + lane;
      for (; g >= sp.steady_lo; --g) {
        const int rp0 = w.rp;
        sstep(w, o, g * kW + lane);
        o -= kW;
        settle(w, rp0);
      }
    }

    // Reload what the tail needs instead of keeping it live across the steady
    // loop (non-coherent loads the compiler cannot merge with the first ones).
    const int lo = ld_keep(reinterpret_cast<const int*>(&ent->lo));
    const int hi1 = ld_keep(reinterpret_cast<const int*>(&ent->hi1));
    const int act = ld_keep(&ent->act[lane]);
    const uint32_t x0 = (uint32_t)ld_keep(reinterpret_cast<const int*>(&ent->x0[lane]));
    int act_p = -1;
    uint32_t x_p = 0;
    if (lo > 0) {
      act_p = ld_keep(&ent[-1].act[lane]);
      x_p = (uint32_t)ld_keep(reinterpret_cast<const int*>(&ent[-1].x0[lane]));
    }
    for (; g >= (lo >> 5); --g) pstep(w, g, act, x0, lo, hi1, act_p, x_p, sp.bad);

    // The first thread of a stream must end where the encoder started (Eqs. 1-4 invert).
    uint32_t err = 0;
    if (w.p < -1) err |= kErrUnderrun;
    if (lo == 0 && (w.p != -1 || __any_sync(kFull, w.x != kL))) err |= kErrCorrupt;
    if (__any_sync(kFull, sp.bad)) err |= kErrCorrupt;
    if (err && lane == 0) {
      atomicOr(&ctl->errors, err);
      atomicExch(&ctl->bad_entry, entry_id + 1);
    }
  }

  // One split per warp (one coder lane per thread): the walk of begin and
  // finish written as one function, which keeps fewer values live across
  // the steady loop.
  __device__ void run(const DevEntry* __restrict__ ent, DevControl* ctl, uint32_t entry_id) {
    int lo = (int)ent->lo, hi1 = (int)ent->hi1;
    if (lo >= hi1) return;
    int act = ent->act[lane];
    uint32_t x0 = ent->x0[lane];
    int g = ent->g_top;

    Walker w;
    w.x = 0;
    w.p = ent->q;
    w.cbase = (w.p >> 8) << 8;                       // p = -1 gives -256: nothing staged
    {
      const int c = w.cbase >> 8;
      const uint4 a = load_chunk(words, c, lane);
      const uint4 b = load_chunk(words, c - 1, lane);
      if (c >= 0) put_chunk(ring, c, lane, a);
      if (c >= 1) put_chunk(ring, c - 1, lane, b);
      w.pre = load_chunk(words, c - 2, lane);
    }
    // table numbers of the synchronisation phase: the three blocks from the
    // top group, copied while the ring's chunks load
    const bool st = is_adaptive<KIND>() ? staged : false;
    if (st)
      for (int k = 0; k < kTidSlots; ++k) stage_tids(g - 8 * k, lo >> 5, k);
    __syncwarp();
    w.rp = (w.p & (kRingWords - 1)) + kRingWords;

    const int g_full = __reduce_min_sync(kFull, act);            // below it every coder has joined
    const int steady_hi = min(g_full - 1, (hi1 >> 5) - 1);       // whole groups owned ...
    // the previous entry of the same stream (there is one whenever lo > 0)
    int act_p = -1, gtop_p = -1;
    uint32_t x_p = 0;
    if (lo > 0) {
      act_p = ent[-1].act[lane];
      x_p = ent[-1].x0[lane];
      gtop_p = ent[-1].g_top;
    }
    const int steady_lo = max((lo + kW - 1) >> 5, gtop_p + 1);   // ... fully decodable, above the check
    bool bad = false;

    int go = g, b0 = 0;                     // staged blocks: from group go down, the first in slot b0
    if (st) {
      cp_async_wait<0>();
      __syncwarp();
    }
    for (; g > steady_hi && g >= (lo >> 5); --g)
      pstep(w, g, act, x0, lo, hi1, act_p, x_p, bad, st ? toff_of(go, b0, g) : -1);

    if (g >= steady_lo) {
      typename SymOut<KIND>::T* o = out + (size_t)g * kW + lane;
      // 8 steps consume at most 256 words: with p >= cbase at the start of a
      // block, every read stays inside the two staged chunks
      if constexpr (is_adaptive<KIND>()) {
        if (staged) {
          // the first two blocks' table numbers (only groups this walk
          // decodes: a shard plan stages no others), once every lane has
          // read the synchronisation phase's
          __syncwarp();
          stage_tids(g, lo >> 5, 0);
          stage_tids(g - 8, lo >> 5, 1);
          int blk = 0;
          while (g - 7 >= steady_lo) {
            const int rp0 = w.rp;
            // this block's table numbers have landed (the next block's may
            // not have); then the block after next goes into the slot the
            // previous block read
            cp_async_wait<1>();
            __syncwarp();
            const uint8_t* tb = tbuf + blk * kTidBlock + lane;
            stage_tids(g - 16, lo >> 5, blk == 0 ? kTidSlots - 1 : blk - 1);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const uint32_t s = T.step(w.x, n, mask, tb[(7 - u) * kW]);
              o[-u * kW] = (typename SymOut<KIND>::T)s;
              renorm(w, w.x < kL);
            }
            blk = blk == kTidSlots - 1 ? 0 : blk + 1;
            o -= 8 * kW;
            g -= 8;
            settle(w, rp0);
          }
          // the block after next as well: the groups below the steady loop
          // read the three blocks from here; nothing stays in flight
          stage_tids(g - 16, lo >> 5, blk == 0 ? kTidSlots - 1 : blk - 1);
          cp_async_wait<0>();
          __syncwarp();
          go = g;
          b0 = blk;
        } else {
          while (g - 7 >= steady_lo) {
            const int rp0 = w.rp;
            const int i0 = g * kW + lane;
            // table numbers of the block after next into L1 (256 bytes, 8 per lane),
            // only of groups this walk decodes (a shard plan stages no others)
            if (g - 23 >= steady_lo) prefetch_l1(tid + (g - 23) * kW + lane * 8);
#pragma unroll
            for (int u = 0; u < 8; ++u) sstep(w, o - u * kW, i0 - u * kW);
            o -= 8 * kW;
            g -= 8;
            settle(w, rp0);
          }
        }
      } else {
        while (g - 7 >= steady_lo) {
          const int rp0 = w.rp;
          const int i0 = g * kW + lane;
#pragma unroll
          for (int u = 0; u < 8; ++u) sstep(w, o - u * kW, i0 - u * kW);
          o -= 8 * kW;
          g -= 8;
          settle(w, rp0);
        }
      }
      for (; g >= steady_lo; --g) {
        const int rp0 = w.rp;
        *o = (typename SymOut<KIND>::T)dec_at(w.x, g * kW + lane, st ? toff_of(go, b0, g) : -1);
        renorm(w, w.x < kL);
        o -= kW;
        settle(w, rp0);
      }
    }

    // Reload what the tail needs instead of keeping it live across the steady
    // loop (non-coherent loads the compiler cannot merge with the first ones).
    lo = ld_keep(reinterpret_cast<const int*>(&ent->lo));
    hi1 = ld_keep(reinterpret_cast<const int*>(&ent->hi1));
    act = ld_keep(&ent->act[lane]);
    x0 = (uint32_t)ld_keep(reinterpret_cast<const int*>(&ent->x0[lane]));
    if (lo > 0) {
      act_p = ld_keep(&ent[-1].act[lane]);
      x_p = (uint32_t)ld_keep(reinterpret_cast<const int*>(&ent[-1].x0[lane]));
    }
    for (; g >= (lo >> 5); --g) pstep(w, g, act, x0, lo, hi1, act_p, x_p, bad, st ? toff_of(go, b0, g) : -1);

    // The first thread of a stream must end where the encoder started (Eqs. 1-4 invert).
    uint32_t err = 0;
    if (w.p < -1) err |= kErrUnderrun;
    if (lo == 0 && (w.p != -1 || __any_sync(kFull, w.x != kL))) err |= kErrCorrupt;
    if (__any_sync(kFull, bad)) err |= kErrCorrupt;
    if (err && lane == 0) {
      atomicOr(&ctl->errors, err);
      atomicExch(&ctl->bad_entry, entry_id + 1);
    }
  }

  // Two splits per warp (two coder lanes per thread, one of each split, each
  // split with its own word ring): both synchronisation phases, then their
  // steady blocks in lockstep while both have one, then each alone.
  __device__ void run2(const DevEntry* __restrict__ ent, uint32_t entry_id, EntryDecoder& B,
                       const DevEntry* __restrict__ entb, uint32_t entb_id, DevControl* ctl) {
    Walker w, wb;
    Span sp, sb;
    const bool a = begin(ent, w, sp);
    const bool b = B.begin(entb, wb, sb);
    if (a && b)
      while (sp.g - 7 >= sp.steady_lo && sb.g - 7 >= sb.steady_lo) block2(w, sp, B, wb, sb);
    if (a) finish(ent, w, sp, ctl, entry_id);
    if (b) B.finish(entb, wb, sb, ctl, entb_id);
  }
};

// Blocks of WARPS warps; the second launch bound asks for enough resident
// blocks to keep RECOIL_RESIDENT_WARPS warps per SM, which caps registers at
// 65536 / (32 * RECOIL_RESIDENT_WARPS) a thread.
#ifndef RECOIL_RESIDENT_WARPS
#define RECOIL_RESIDENT_WARPS 56
#endif
// The adaptive step needs more registers (the CDF search): 32 warps per SM.
#ifndef RECOIL_RESIDENT_WARPS_ADAPTIVE
#define RECOIL_RESIDENT_WARPS_ADAPTIVE 32
#endif
// Two lanes a thread hold two walks' state: 32 warps (64 splits) per SM for
// the static kinds, 24 warps (48 splits) for the adaptive ones.
#ifndef RECOIL_RESIDENT_WARPS_TWO_LANES
#define RECOIL_RESIDENT_WARPS_TWO_LANES 32
#endif
#ifndef RECOIL_RESIDENT_WARPS_TWO_LANES_ADAPTIVE
#define RECOIL_RESIDENT_WARPS_TWO_LANES_ADAPTIVE 24
#endif
template <uint32_t KIND, int WARPS, int LANES>
struct Residency {
  static constexpr int kWarps =
      LANES == 2 ? (is_adaptive<KIND>() ? RECOIL_RESIDENT_WARPS_TWO_LANES_ADAPTIVE : RECOIL_RESIDENT_WARPS_TWO_LANES)
                 : (is_adaptive<KIND>() ? RECOIL_RESIDENT_WARPS_ADAPTIVE : RECOIL_RESIDENT_WARPS);
  static constexpr int kWant = kWarps / WARPS;
  static constexpr int kMinBlocks = kWant < 1 ? 1 : (kWant > 32 ? 32 : kWant);
};

// LANES coder lanes per thread: each warp decodes LANES splits at once, lane
// j of each split on thread j, every split with its own word ring.
template <uint32_t KIND, int WARPS, int LANES>
__global__ void __launch_bounds__(WARPS * 32, (Residency<KIND, WARPS, LANES>::kMinBlocks))
    decode_kernel(const LaunchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_item;
  const int warp = threadIdx.x >> 5;
  uint16_t* ring = reinterpret_cast<uint16_t*>(smem + a.table_smem) + warp * LANES * kRingSlots;
  // adaptive kinds, one lane a thread: each warp's staged table numbers follow all rings
  uint8_t* tbuf = smem + a.table_smem + (size_t)WARPS * LANES * kRingSlots * 2 + (size_t)warp * kTidSlots * kTidBlock;

  auto stage = [&](const DevStream& st) {
    const uint4* src = reinterpret_cast<const uint4*>(a.table_pool + st.table);
    uint4* dst = reinterpret_cast<uint4*>(smem);
    const uint32_t n16 = st.table_bytes >> 4;
    for (uint32_t k = threadIdx.x; k < n16; k += WARPS * 32) dst[k] = __ldg(src + k);
  };
  auto decoder = [&](EntryDecoder<KIND>& d, const DevStream& st, const DevEntry* ent, uint16_t* r) {
    // the entry's own stream: an item may span streams that share one table
    const uint32_t sid = ent->stream;
    d.T.bind(smem, st);
    d.words = a.word_pool + a.streams[sid].words;
    d.tid = reinterpret_cast<const uint8_t*>(a.word_pool + a.streams[sid].tid);
    d.ring = r;
    d.tbuf = tbuf;
    d.staged = LANES == 1 && a.tid_staged;
    d.out = reinterpret_cast<typename SymOut<KIND>::T*>(a.outs[sid]);
    d.n = st.n_bits;
    d.mask = (1u << st.n_bits) - 1u;
    d.gt = lanemask_gt();
    d.lane = threadIdx.x & 31;
  };
  auto decode_entry = [&](const DevStream& st, uint32_t entry) {
    EntryDecoder<KIND> d;
    decoder(d, st, a.entries + entry, ring);
    d.run(a.entries + entry, a.control, entry);
  };
  // two entries, one lane of each per thread
  auto decode_pair = [&](const DevStream& st, uint32_t e0, uint32_t e1) {
    EntryDecoder<KIND> d, db;
    decoder(d, st, a.entries + e0, ring);
    decoder(db, st, a.entries + e1, ring + kRingSlots);
    d.run2(a.entries + e0, e0, db, a.entries + e1, e1, a.control);
  };

  if (a.warp_queue) {
    // one table for the whole launch, one entry per item: stage once, then
    // every warp pops LANES items at a time on its own (no barrier between entries)
    const DevStream& st = a.streams[a.items[0].stream];
    stage(st);
    __syncthreads();
    for (;;) {
      uint32_t it = 0;
      if ((threadIdx.x & 31) == 0) it = atomicAdd(&a.control->head[a.kind], (uint32_t)LANES);
      it = __shfl_sync(kFull, it, 0);
      if (it >= a.n_items) break;
      if constexpr (LANES == 2) {
        if (it + 1 < a.n_items) {
          decode_pair(st, a.items[it].entry, a.items[it + 1].entry);
          continue;
        }
      }
      decode_entry(st, a.items[it].entry);
    }
    return;
  }

  // CTA items: up to WARPS * LANES entries of one stream (or of streams
  // sharing one table); the table is restaged when the stream changes and the
  // warps pop the item's entries, LANES at a time, from a shared counter
  __shared__ uint32_t s_next;
  uint32_t staged = 0xffffffffu;
  uint32_t it = blockIdx.x;
  for (;;) {
    if (a.persistent) {
      if (threadIdx.x == 0) s_item = atomicAdd(&a.control->head[a.kind], 1u);
    }
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    if (a.persistent) it = s_item;
    if (it >= a.n_items) break;
    const DevItem item = a.items[it];
    const DevStream& st = a.streams[item.stream];
    if (item.stream != staged) {
      stage(st);
      staged = item.stream;
      __syncthreads();
    }
    for (;;) {
      uint32_t k = 0;
      if ((threadIdx.x & 31) == 0) k = atomicAdd(&s_next, (uint32_t)LANES);
      k = __shfl_sync(kFull, k, 0);
      if (k >= item.count) break;
      if constexpr (LANES == 2) {
        if (k + 1 < item.count) {
          decode_pair(st, item.entry + k, item.entry + k + 1);
          continue;
        }
      }
      decode_entry(st, item.entry + k);
    }
    if (!a.persistent) break;
    __syncthreads();
  }
}

size_t smem_bytes(uint32_t kind, uint32_t warps, uint32_t lanes, bool staged, uint32_t table_smem) {
  return (size_t)table_smem + (size_t)warps * warp_smem(kind, lanes, staged);
}

// The dynamic shared memory a kernel may use is raised only when a launch
// needs more than was allowed before on that device: setting the attribute is
// a host call of several microseconds, too slow to repeat for every launch
// when one stream is decoded per launch. The value kept per device is only a
// hint: a launch that fails raises the attribute again and retries once (a
// device reset drops the attribute, not this record).
constexpr int kMaxDevices = 64;

template <uint32_t KIND, int WARPS, int LANES>
cudaError_t allow_smem(size_t sm, bool force) {
  static std::atomic<int> allowed[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = -1;
  if (!force && dev >= 0 && allowed[dev].load(std::memory_order_relaxed) >= (int)sm) return cudaSuccess;
  const int want = dev >= 0 && !force ? std::max<int>((int)sm, allowed[dev].load(std::memory_order_relaxed)) : (int)sm;
  const cudaError_t e =
      cudaFuncSetAttribute(decode_kernel<KIND, WARPS, LANES>, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (e == cudaSuccess && dev >= 0) allowed[dev].store(want, std::memory_order_relaxed);
  return e;
}

template <uint32_t KIND, int WARPS, int LANES>
cudaError_t launch_kw(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  const size_t sm = smem_bytes(KIND, WARPS, LANES, a.tid_staged != 0, a.table_smem);
  for (int attempt = 0; attempt < 2; attempt++) {
    cudaError_t e = allow_smem<KIND, WARPS, LANES>(sm, attempt > 0);
    if (e != cudaSuccess) return e;
    decode_kernel<KIND, WARPS, LANES><<<grid, WARPS * 32, sm, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaErrorInvalidValue || attempt > 0) return e;
  }
  return cudaErrorInvalidValue;
}

template <uint32_t KIND, int WARPS, int LANES>
int occupancy_kw(uint32_t table_smem, bool staged, int* out) {
  const size_t sm = smem_bytes(KIND, WARPS, LANES, staged, table_smem);
  if (allow_smem<KIND, WARPS, LANES>(sm, false) != cudaSuccess) return -1;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, decode_kernel<KIND, WARPS, LANES>, WARPS * 32, sm) ==
                 cudaSuccess
             ? 0
             : -1;
}

// One lane a thread: static kinds in every CTA size, adaptive kinds in 4, 8,
// 16 and 32 warps. Two lanes a thread: static kinds in 4, 8 and 16 warps,
// adaptive kinds in 8, 16 and 24 warps.
template <uint32_t KIND, typename F>
auto by_shape(uint32_t warps, uint32_t lanes, F&& f) {
  if (lanes == 2) {
    if constexpr (is_adaptive<KIND>()) {
      switch (warps) {
        case 8: return f(std::integral_constant<int, 8>(), std::integral_constant<int, 2>());
        case 16: return f(std::integral_constant<int, 16>(), std::integral_constant<int, 2>());
        case 24: return f(std::integral_constant<int, 24>(), std::integral_constant<int, 2>());
      }
    } else {
      switch (warps) {
        case 4: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 2>());
        case 8: return f(std::integral_constant<int, 8>(), std::integral_constant<int, 2>());
        case 16: return f(std::integral_constant<int, 16>(), std::integral_constant<int, 2>());
      }
    }
  } else if (lanes <= 1) {
    if constexpr (is_adaptive<KIND>()) {
      switch (warps) {
        case 4: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 1>());
        case 8: return f(std::integral_constant<int, 8>(), std::integral_constant<int, 1>());
        case 16: return f(std::integral_constant<int, 16>(), std::integral_constant<int, 1>());
        case 32: return f(std::integral_constant<int, 32>(), std::integral_constant<int, 1>());
      }
    } else {
      switch (warps) {
        case 1: return f(std::integral_constant<int, 1>(), std::integral_constant<int, 1>());
        case 2: return f(std::integral_constant<int, 2>(), std::integral_constant<int, 1>());
        case 4: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 1>());
        case 8: return f(std::integral_constant<int, 8>(), std::integral_constant<int, 1>());
        case 16: return f(std::integral_constant<int, 16>(), std::integral_constant<int, 1>());
        case 32: return f(std::integral_constant<int, 32>(), std::integral_constant<int, 1>());
      }
    }
  }
  return f(std::integral_constant<int, 0>(), std::integral_constant<int, 0>());
}

template <uint32_t KIND>
cudaError_t launch_k(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  return by_shape<KIND>(a.warps, a.lanes, [&](auto w, auto l) -> cudaError_t {
    if constexpr (decltype(w)::value == 0) return cudaErrorInvalidValue;
    else return launch_kw<KIND, decltype(w)::value, decltype(l)::value>(a, grid, s);
  });
}

template <uint32_t KIND>
int occupancy_k(uint32_t warps, uint32_t lanes, bool staged, uint32_t table_smem, int* out) {
  return by_shape<KIND>(warps, lanes, [&](auto w, auto l) -> int {
    if constexpr (decltype(w)::value == 0) return -1;
    else return occupancy_kw<KIND, decltype(w)::value, decltype(l)::value>(table_smem, staged, out);
  });
}

}  // namespace

bool warps_supported(uint32_t w) { return w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32; }

bool adaptive_warps_supported(uint32_t w) { return w == 4 || w == 8 || w == 16 || w == 32; }

bool shape_supported(bool adaptive, uint32_t warps, uint32_t lanes) {
  if (lanes == 2) return adaptive ? (warps == 8 || warps == 16 || warps == 24) : (warps == 4 || warps == 8 || warps == 16);
  if (lanes > 1) return false;
  return adaptive ? adaptive_warps_supported(warps) : warps_supported(warps);
}

cudaError_t launch_decode(uint32_t kind, const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  switch (kind) {
    case kPacked8: return launch_k<kPacked8>(a, grid, s);
    case kGeneric8: return launch_k<kGeneric8>(a, grid, s);
    case kGeneric16: return launch_k<kGeneric16>(a, grid, s);
    case kAdaptive8: return launch_k<kAdaptive8>(a, grid, s);
    case kAdaptive16: return launch_k<kAdaptive16>(a, grid, s);
    case kAdaptive16Wide: return launch_k<kAdaptive16Wide>(a, grid, s);
    case kAdaptive8Pair: return launch_k<kAdaptive8Pair>(a, grid, s);
    case kAdaptive16Pair: return launch_k<kAdaptive16Pair>(a, grid, s);
    case kPacked16: return launch_k<kPacked16>(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

int occupancy_ctas_per_sm(uint32_t kind, uint32_t warps, uint32_t lanes, bool staged, uint32_t table_smem, int* out) {
  switch (kind) {
    case kPacked8: return occupancy_k<kPacked8>(warps, lanes, staged, table_smem, out);
    case kGeneric8: return occupancy_k<kGeneric8>(warps, lanes, staged, table_smem, out);
    case kGeneric16: return occupancy_k<kGeneric16>(warps, lanes, staged, table_smem, out);
    case kAdaptive8: return occupancy_k<kAdaptive8>(warps, lanes, staged, table_smem, out);
    case kAdaptive16: return occupancy_k<kAdaptive16>(warps, lanes, staged, table_smem, out);
    case kAdaptive16Wide: return occupancy_k<kAdaptive16Wide>(warps, lanes, staged, table_smem, out);
    case kAdaptive8Pair: return occupancy_k<kAdaptive8Pair>(warps, lanes, staged, table_smem, out);
    case kAdaptive16Pair: return occupancy_k<kAdaptive16Pair>(warps, lanes, staged, table_smem, out);
    case kPacked16: return occupancy_k<kPacked16>(warps, lanes, staged, table_smem, out);
  }
  return -1;
}

size_t warp_smem(uint32_t kind, uint32_t lanes, bool staged) {
  const size_t l = lanes > 1 ? lanes : 1;
  return l * kRingSlots * sizeof(uint16_t) + (is_adaptive_kind(kind) && l == 1 && staged ? (size_t)kTidSlots * kTidBlock : 0);
}

}  // namespace recoil
