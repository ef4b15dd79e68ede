// Serialised streams: what a content server stores and sends (Sec. 3.3, 4.3).
//
// Layout (little-endian): "RCL1", n_bits (u8), sym_bytes (u8), 2 zero bytes,
// alphabet (u32), the quantised PDF (u32 each), the W final states (u32 each),
// the word count (u64), the words (u16 each), the metadata length (u64), then
// the packed split metadata of Sec. 4.3:
//   header   M (32 bits: splits including the final-state one), B (64: words), N (64: symbols)
//   series   word offset of split point i minus i*ceil(B/M), i = 1..M-1 (signed)
//   series   anchor (largest group ID) of split point i minus i*ceil(ceil(N/W)/M) (signed)
//   per split point: W states as-is (16 bits each), then the series of anchor
//            minus each coder's group ID (unsigned); group ID = index / W + 1
// A series is (w-1) in a 4-bit (unsigned, values up to 16 bits) or 5-bit
// (signed, up to 32 bits) field, then each value in w bits, signed values
// preceded by a sign bit; w is the bit length of the largest magnitude (1 for
// all zeros). Bits are written most significant first; the section is padded
// to whole bytes. Dropping entries (recoil_combine_splits) before serialising
// is how a server matches the split count to a decoder (Sec. 3.3).
#include <algorithm>
#include <cstring>
#include <new>

#include "recoil_internal.h"

namespace recoil {
namespace {

class BitWriter {
 public:
  explicit BitWriter(std::vector<uint8_t>& out) : out_(out) {}
  void put(uint64_t v, int width) {
    for (int k = width - 1; k >= 0; k--) {
      acc_ = (acc_ << 1) | ((v >> k) & 1);
      if (++nacc_ == 8) {
        out_.push_back((uint8_t)acc_);
        acc_ = 0;
        nacc_ = 0;
      }
    }
  }
  void flush() {
    if (nacc_) out_.push_back((uint8_t)(acc_ << (8 - nacc_)));
    acc_ = 0;
    nacc_ = 0;
  }

 private:
  std::vector<uint8_t>& out_;
  uint32_t acc_ = 0;
  int nacc_ = 0;
};

class BitReader {
 public:
  BitReader(const uint8_t* p, uint64_t n) : p_(p), nbits_(n * 8) {}
  bool get(int width, uint64_t* v) {
    if (pos_ + (uint64_t)width > nbits_) return false;
    uint64_t r = 0;
    for (int k = 0; k < width; k++, pos_++) r = (r << 1) | ((p_[pos_ >> 3] >> (7 - (pos_ & 7))) & 1);
    *v = r;
    return true;
  }

 private:
  const uint8_t* p_;
  uint64_t nbits_, pos_ = 0;
};

int bitlen(uint64_t v) {
  int w = 0;
  while (v) {
    w++;
    v >>= 1;
  }
  return std::max(w, 1);
}

bool put_unsigned(BitWriter& bw, const std::vector<uint64_t>& v) {
  int w = 1;
  for (uint64_t x : v) w = std::max(w, bitlen(x));
  if (w > 16) return false;
  bw.put((uint64_t)(w - 1), 4);
  for (uint64_t x : v) bw.put(x, w);
  return true;
}

bool put_signed(BitWriter& bw, const std::vector<int64_t>& v) {
  int w = 1;
  for (int64_t x : v) w = std::max(w, bitlen((uint64_t)(x < 0 ? -x : x)));
  if (w > 32) return false;
  bw.put((uint64_t)(w - 1), 5);
  for (int64_t x : v) {
    bw.put(x < 0 ? 1 : 0, 1);
    bw.put((uint64_t)(x < 0 ? -x : x), w);
  }
  return true;
}

bool get_unsigned(BitReader& br, size_t count, std::vector<uint64_t>& v) {
  uint64_t w = 0;
  if (!br.get(4, &w)) return false;
  v.resize(count);
  for (size_t i = 0; i < count; i++)
    if (!br.get((int)w + 1, &v[i])) return false;
  return true;
}

bool get_signed(BitReader& br, size_t count, std::vector<int64_t>& v) {
  uint64_t w = 0;
  if (!br.get(5, &w)) return false;
  v.resize(count);
  for (size_t i = 0; i < count; i++) {
    uint64_t neg = 0, mag = 0;
    if (!br.get(1, &neg) || !br.get((int)w + 1, &mag)) return false;
    v[i] = neg ? -(int64_t)mag : (int64_t)mag;
  }
  return true;
}

uint64_t ceil_div(uint64_t a, uint64_t b) { return b ? (a + b - 1) / b : 0; }

int pack_metadata(const Stream& s, std::vector<uint8_t>& out) {
  if (s.adaptive()) return fail(RECOIL_EINVAL, "adaptive streams are not serialised (their model travels with the codec)");
  const uint64_t M = s.entries.size() + 1, B = s.n_words(), N = s.n_syms;
  const uint64_t Eb = ceil_div(B, M), Eg = ceil_div(ceil_div(N, kW), M);
  BitWriter bw(out);
  bw.put(M, 32);
  bw.put(B, 64);
  bw.put(N, 64);
  std::vector<int64_t> dq, da;
  std::vector<uint64_t> anchor(s.entries.size());
  for (size_t i = 0; i < s.entries.size(); i++) {
    const Entry& e = s.entries[i];
    uint64_t a = 0;
    for (int j = 0; j < kW; j++) a = std::max<uint64_t>(a, e.idx[j] / kW + 1);
    anchor[i] = a;
    dq.push_back((int64_t)e.word - (int64_t)((i + 1) * Eb));
    da.push_back((int64_t)a - (int64_t)((i + 1) * Eg));
  }
  if (!put_signed(bw, dq) || !put_signed(bw, da)) return fail(RECOIL_EINVAL, "split offsets too far from expectation");
  std::vector<uint64_t> diffs(kW);
  for (size_t i = 0; i < s.entries.size(); i++) {
    const Entry& e = s.entries[i];
    for (int j = 0; j < kW; j++) bw.put(e.y[j], 16);
    for (int j = 0; j < kW; j++) diffs[j] = anchor[i] - (e.idx[j] / kW + 1);
    if (!put_unsigned(bw, diffs)) return fail(RECOIL_EINVAL, "synchronisation section too long to pack (group difference above 16 bits)");
  }
  bw.flush();
  return RECOIL_OK;
}

template <typename T>
void put_le(std::vector<uint8_t>& out, T v) {
  for (size_t k = 0; k < sizeof(T); k++) out.push_back((uint8_t)(v >> (8 * k)));
}

template <typename T>
bool get_le(const uint8_t*& p, const uint8_t* end, T* v) {
  if ((size_t)(end - p) < sizeof(T)) return false;
  T r = 0;
  for (size_t k = 0; k < sizeof(T); k++) r |= (T)p[k] << (8 * k);
  p += sizeof(T);
  *v = r;
  return true;
}

int serialize(const Stream& s, std::vector<uint8_t>& out, uint64_t* meta_bytes) {
  out.clear();
  out.insert(out.end(), {'R', 'C', 'L', '1'});
  out.push_back((uint8_t)s.n_bits);
  out.push_back((uint8_t)s.sym_bytes);
  out.push_back(0);
  out.push_back(0);
  put_le<uint32_t>(out, s.alphabet());
  for (uint32_t f : s.freq) put_le<uint32_t>(out, f);
  for (int j = 0; j < kW; j++) put_le<uint32_t>(out, s.final_x[j]);
  put_le<uint64_t>(out, s.n_words());
  const uint16_t* w = s.word_data();
  for (uint64_t k = 0; k < s.n_words(); k++) put_le<uint16_t>(out, w[k]);
  std::vector<uint8_t> meta;
  int rc = pack_metadata(s, meta);
  if (rc) return rc;
  put_le<uint64_t>(out, meta.size());
  out.insert(out.end(), meta.begin(), meta.end());
  if (meta_bytes) *meta_bytes = meta.size();
  return RECOIL_OK;
}

}  // namespace
}  // namespace recoil

using namespace recoil;

extern "C" {

int recoil_serialized_size(const recoil_stream* s, uint64_t* bytes, uint64_t* metadata_bytes) {
  clear_error();
  if (!s || !bytes) return fail(RECOIL_EINVAL, "null argument");
  try {
    std::vector<uint8_t> meta;
    int rc = pack_metadata(*s, meta);
    if (rc) return rc;
    *bytes = 4 + 4 + 4 + 4ull * s->alphabet() + 4ull * kW + 8 + 2 * s->n_words() + 8 + meta.size();
    if (metadata_bytes) *metadata_bytes = meta.size();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

int recoil_serialize(const recoil_stream* s, void* buf, uint64_t cap, uint64_t* written) {
  clear_error();
  if (!s || !buf || !written) return fail(RECOIL_EINVAL, "null argument");
  try {
    std::vector<uint8_t> out;
    int rc = serialize(*s, out, nullptr);
    if (rc) return rc;
    if (out.size() > cap) return fail(RECOIL_ENOMEM, "buffer too small (see recoil_serialized_size)");
    std::memcpy(buf, out.data(), out.size());
    *written = out.size();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

int recoil_deserialize(const void* buf, uint64_t size, recoil_stream** out) {
  clear_error();
  if (!buf || !out) return fail(RECOIL_EINVAL, "null argument");
  *out = nullptr;
  const uint8_t* p = (const uint8_t*)buf;
  const uint8_t* end = p + size;
  if (size < 12 || std::memcmp(p, "RCL1", 4) != 0) return fail(RECOIL_ECORRUPT, "not a serialised recoil stream");
  p += 4;
  recoil_params params{p[0], p[1], RECOIL_SPLIT_REMAINING, 0};
  p += 4;
  uint32_t alphabet = 0;
  if (!get_le(p, end, &alphabet) || alphabet == 0 || alphabet > 65536 ||
      (uint64_t)(end - p) < 4ull * alphabet + 4ull * kW + 8)
    return fail(RECOIL_ECORRUPT, "truncated stream header");
  try {
    std::vector<uint32_t> freq(alphabet);
    for (uint32_t k = 0; k < alphabet; k++) get_le(p, end, &freq[k]);
    uint32_t final_x[kW];
    for (int j = 0; j < kW; j++) get_le(p, end, &final_x[j]);
    uint64_t nw = 0, mbytes = 0;
    get_le(p, end, &nw);
    if ((uint64_t)(end - p) < 2 * nw + 8) return fail(RECOIL_ECORRUPT, "truncated words");
    std::vector<uint16_t> words(nw);
    for (uint64_t k = 0; k < nw; k++) get_le(p, end, &words[k]);
    get_le(p, end, &mbytes);
    if ((uint64_t)(end - p) < mbytes) return fail(RECOIL_ECORRUPT, "truncated metadata");
    BitReader br(p, mbytes);
    uint64_t M = 0, B = 0, N = 0;
    if (!br.get(32, &M) || !br.get(64, &B) || !br.get(64, &N) || M < 1 || B != nw)
      return fail(RECOIL_ECORRUPT, "bad metadata header");
    const uint64_t R = M - 1, Eb = ceil_div(B, M), Eg = ceil_div(ceil_div(N, kW), M);
    if (R > mbytes * 8 / (kW * 16 + 4)) return fail(RECOIL_ECORRUPT, "metadata shorter than its split count");
    std::vector<int64_t> dq, da;
    if (!get_signed(br, R, dq) || !get_signed(br, R, da)) return fail(RECOIL_ECORRUPT, "truncated metadata series");
    std::vector<uint64_t> ew(R), ei(R * kW);
    std::vector<uint16_t> es(R * kW);
    std::vector<uint64_t> diffs;
    for (uint64_t i = 0; i < R; i++) {
      ew[i] = (uint64_t)((int64_t)((i + 1) * Eb) + dq[i]);
      const int64_t anchor = (int64_t)((i + 1) * Eg) + da[i];
      for (int j = 0; j < kW; j++) {
        uint64_t v = 0;
        if (!br.get(16, &v)) return fail(RECOIL_ECORRUPT, "truncated states");
        es[i * kW + j] = (uint16_t)v;
      }
      if (!get_unsigned(br, kW, diffs)) return fail(RECOIL_ECORRUPT, "truncated group differences");
      for (int j = 0; j < kW; j++) {
        const int64_t g = anchor - (int64_t)diffs[j];
        if (g < 1) return fail(RECOIL_ECORRUPT, "group ID below 1");
        ei[i * kW + j] = (uint64_t)(g - 1) * kW + (uint64_t)j;
      }
    }
    // everything else (ranges, ordering, congruences, table sum) is checked by the importer
    return recoil_stream_import(&params, N, alphabet, freq.data(), words.data(), nw, final_x, (uint32_t)R,
                                ew.data(), ei.data(), es.data(), out);
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

}  // extern "C"
