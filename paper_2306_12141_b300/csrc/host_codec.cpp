// Host codec of the Recoil library: quantiser, serial interleaved encoder with
// split recording, split heuristic, combining, import/export and validation.
//
// The encoder is serial by design (Sec. 6: Recoil trades encoder throughput
// for decoder-adaptive parallelism). It is written for speed, not for
// reading: divisions by f use exact multiply-high reciprocals and the
// heuristic keeps its per-coder state incrementally.
#include <algorithm>
#include <cstring>
#include <limits>
#include <new>

#include "recoil_internal.h"

namespace recoil {

namespace {
thread_local std::string g_last_error;

// floor(x / f) for x < 2^32, 1 <= f <= 2^16, via m = ceil(2^(32+l) / f),
// l = ceil(log2 f): the error term x (m f - 2^(32+l)) / (f 2^(32+l)) is below
// 1/f, so the floor is exact (Granlund & Montgomery, PLDI 1994, Thm. 4.2).
struct Divider {
  uint64_t m;
  uint32_t shift;
  void set(uint32_t f) {
    uint32_t l = 0;
    while ((1u << l) < f) l++;
    shift = 32 + l;
    const unsigned __int128 num = ((unsigned __int128)1) << shift;
    m = (uint64_t)((num + f - 1) / f);
  }
  uint32_t div(uint32_t x) const { return (uint32_t)(((unsigned __int128)x * m) >> shift); }
};

struct EncSym {
  uint32_t f;
  uint32_t F;
  uint32_t xmax;        // renormalise while x > xmax (x >= 2^(32-n) f), saturated
  Divider d;
};

}  // namespace

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

void clear_error() { g_last_error.clear(); }

bool Stream::constant() const {
  if (adaptive()) return false;
  for (uint32_t f : freq)
    if (f == (1u << n_bits)) return true;
  return false;
}

const std::vector<uint32_t>& Stream::owned_ends() const {
  std::lock_guard<std::mutex> g(cache_mu);
  if (!owned_end_ready) {
    owned_end.resize(entries.size());
    for (size_t e = 0; e < entries.size(); e++)
      owned_end[e] = *std::min_element(entries[e].idx, entries[e].idx + kW);
    owned_end_ready = true;
  }
  return owned_end;
}

// Sec. 3.3: the combined splits should own close symbol counts. For split k
// the kept entry is the one whose owned end (smallest recorded index) lies
// nearest to (k+1) N / Mp, searched after the previous kept entry and leaving
// one entry for each later split (ties: the smaller end, then the earlier
// entry); the final entry is always kept. Owned ends never decrease, so each
// choice is a gallop from the previous pick and a binary search.
void combine_picks(const Stream& in, uint32_t target, std::vector<uint32_t>& keep) {
  keep.clear();
  if (target < 1) target = 1;
  const uint64_t R = in.entries.size();                     // regular entries
  const uint64_t Mp = std::min<uint64_t>(target, R + 1);
  const std::vector<uint32_t>& m = in.owned_ends();        // cached: serving combines per request
  keep.reserve(Mp - 1);
  uint64_t first = 0;
  for (uint64_t k = 0; k + 1 < Mp; k++) {
    const uint64_t last = R - (Mp - 1 - k);
    const uint64_t t = (uint64_t)((unsigned __int128)(k + 1) * in.n_syms / Mp);
    // the first end >= t in [first, last]: gallop from the previous pick
    // (targets are about R / Mp entries apart), then bisect the last stride
    uint64_t below = first, step = 1;
    while (below + step <= last && m[below + step - 1] < t) {
      below += step;
      step *= 2;
    }
    const auto lo = m.begin() + first;
    const uint64_t b = std::lower_bound(m.begin() + below, m.begin() + std::min(below + step, last + 1), t) - m.begin();
    uint64_t pick;
    if (b == first) {
      pick = b;
    } else {
      const uint64_t a = m[b - 1];                                // the largest end below t
      if (b <= last && m[b] - t < t - a) pick = b;
      else pick = std::lower_bound(lo, m.begin() + b, (uint32_t)a) - m.begin();
    }
    keep.push_back((uint32_t)pick);
    first = pick + 1;
  }
}

// --------------------------------------------------------------- quantiser
// Present symbols get max(1, round_half_even(c 2^n / N)); then the sum is
// corrected to 2^n one unit at a time, cycling over present symbols in order
// of decreasing first-pass f (ties: smaller symbol), adding while the sum is
// short and removing (never below 1) while it is over.
static int quantize(const std::vector<uint64_t>& c, uint32_t n, std::vector<uint32_t>& f) {
  const uint64_t total = 1ull << n;
  uint64_t N = 0;
  std::vector<uint32_t> present;
  for (size_t s = 0; s < c.size(); s++) {
    N += c[s];
    if (c[s]) present.push_back((uint32_t)s);
  }
  if (N == 0) return fail(RECOIL_EINVAL, "no symbols to quantise");
  if (present.size() > total) return fail(RECOIL_EINVAL, "more distinct symbols than 2^n slots");
  f.assign(c.size(), 0);
  uint64_t sum = 0;
  for (uint32_t s : present) {
    const unsigned __int128 num = (unsigned __int128)c[s] << n;
    uint64_t q = (uint64_t)(num / N);
    const uint64_t r = (uint64_t)(num - (unsigned __int128)q * N);
    if (2 * (unsigned __int128)r > N || (2 * (unsigned __int128)r == N && (q & 1))) q++;
    f[s] = (uint32_t)std::max<uint64_t>(q, 1);
    sum += f[s];
  }
  std::stable_sort(present.begin(), present.end(), [&](uint32_t a, uint32_t b) { return f[a] > f[b]; });
  size_t pos = 0;
  while (sum != total) {
    const uint32_t s = present[pos];
    if (sum < total) {
      f[s]++;
      sum++;
    } else if (f[s] > 1) {
      f[s]--;
      sum--;
    }
    pos = (pos + 1 == present.size()) ? 0 : pos + 1;
  }
  return RECOIL_OK;
}

// ------------------------------------------------------------------ encoder
namespace {

// Renormalisation record of word p: the symbol whose coding triggered it
// (coder = sym % W, recorded index = sym - W) and the state right after.
struct Records {
  std::vector<uint32_t> sym;
  std::vector<uint16_t> y;
};

// tab holds one EncSym per symbol of each PDF row; with a table-number array
// (adaptive model, Sec. 3.1) symbol i uses row tid[i], else row 0.
template <typename T, bool ADAPTIVE>
void encode_loop(const T* syms, uint64_t N, const std::vector<EncSym>& tab, uint32_t A, const uint8_t* tid,
                 uint32_t n, std::vector<uint16_t>& words, Records& rec, uint32_t* final_x) {
  uint32_t x[kW];
  for (int j = 0; j < kW; j++) x[j] = kL;
  uint16_t* wp = words.data();
  uint32_t* rs = rec.sym.data();
  uint16_t* ry = rec.y.data();
  uint64_t p = 0;
  for (uint64_t i = 0; i < N; i++) {
    const int j = (int)(i & (kW - 1));
    const EncSym& e = ADAPTIVE ? tab[(size_t)tid[i] * A + syms[i]] : tab[syms[i]];
    uint32_t v = x[j];
    if (v > e.xmax) {                        // Eq. 3: one step suffices since b >= n
      wp[p] = (uint16_t)v;
      v >>= kB;
      rs[p] = (uint32_t)i;
      ry[p] = (uint16_t)v;
      p++;
    }
    const uint32_t q = e.f == 1 ? v : e.d.div(v);
    x[j] = (q << n) + e.F + (v - q * e.f);   // Eq. 1
  }
  words.resize(p);
  rec.sym.resize(p);
  rec.y.resize(p);
  for (int j = 0; j < kW; j++) final_x[j] = x[j];
}

// Split placement by the heuristic of Def. 4.1 / Eq. 7, scanning words
// forward. For a word q the backward scan of Sec. 4.1 gives, per coder, its
// latest record at or before q; this keeps those incrementally. top is the
// index recorded at q itself, m the smallest over coders.
void place_splits(const Records& rec, uint64_t N, uint32_t M, uint32_t rule, std::vector<uint64_t>& out) {
  out.clear();
  const int64_t nw = (int64_t)rec.sym.size();
  if (M < 2 || nw == 0) return;
  int64_t last[kW];
  int seen = 0;
  for (int j = 0; j < kW; j++) last[j] = std::numeric_limits<int64_t>::min();
  int64_t minv = std::numeric_limits<int64_t>::min();
  int minlane = 0;
  auto recompute_min = [&]() {
    minv = last[0];
    minlane = 0;
    for (int j = 1; j < kW; j++)
      if (last[j] < minv) { minv = last[j]; minlane = j; }
  };
  auto apply = [&](int64_t q) {
    const int j = (int)(rec.sym[q] & (kW - 1));
    if (last[j] == std::numeric_limits<int64_t>::min()) seen++;
    last[j] = (int64_t)rec.sym[q] - kW;
    if (j == minlane) recompute_min();       // any other coder's new index is above the minimum
  };

  int64_t lo = 0, q = 0;
  while (out.size() + 1 < M) {
    // expected symbols per split: over what is left (ceil(N / M) for the first
    // split), or ceil(N / M) throughout as Def. 4.1 prints it
    const int64_t left = (int64_t)M - (int64_t)out.size();
    const int64_t T = rule == RECOIL_SPLIT_EQ7 ? ((int64_t)N + M - 1) / M : ((int64_t)N - lo + left - 1) / left;
    int64_t best = -1, bestH = 0;
    for (; q < nw; q++) {
      apply(q);
      if (seen < kW || minv < 0) continue;
      const int64_t top = (int64_t)rec.sym[q] - kW, m = minv;
      if (best >= 0 && m - lo - T > bestH) break;
      const int64_t t = top + 1 - lo, ts = top + 1 - m;
      const int64_t H = std::llabs(t - T) + std::llabs(t - ts - T);
      if (best < 0 || H < bestH) { best = q; bestH = H; }
    }
    if (best < 0) break;
    out.push_back((uint64_t)best);
    // rewind the per-coder state to the chosen word: backward scan from it
    for (int j = 0; j < kW; j++) last[j] = std::numeric_limits<int64_t>::min();
    seen = 0;
    for (int64_t k = best; k >= 0 && seen < kW; k--) {
      const int j = (int)(rec.sym[k] & (kW - 1));
      if (last[j] != std::numeric_limits<int64_t>::min()) continue;
      last[j] = (int64_t)rec.sym[k] - kW;
      seen++;
    }
    recompute_min();
    lo = minv;
    q = best + 1;
  }
}

// Entry at word q: each coder's latest record at or before q (Sec. 4.1).
bool entry_at(const Records& rec, uint64_t q, Entry& e) {
  uint32_t found = 0;
  e.word = q;
  for (int64_t k = (int64_t)q; k >= 0 && found != 0xffffffffu; k--) {
    const int j = (int)(rec.sym[k] & (kW - 1));
    if (found & (1u << j)) continue;
    found |= 1u << j;
    if (rec.sym[k] < (uint32_t)kW) return false;
    e.idx[j] = rec.sym[k] - kW;
    e.y[j] = rec.y[k];
  }
  return found == 0xffffffffu;
}

}  // namespace

static int make_table_syms(const void* syms, uint64_t N, uint32_t sb, uint32_t n,
                           std::vector<uint32_t>& freq) {
  size_t A = sb == 1 ? 256 : 65536;
  std::vector<uint64_t> c(A, 0);
  if (sb == 1) {
    const uint8_t* s = (const uint8_t*)syms;
    uint64_t h[4][256] = {};
    uint64_t i = 0;
    for (; i + 4 <= N; i += 4) { h[0][s[i]]++; h[1][s[i + 1]]++; h[2][s[i + 2]]++; h[3][s[i + 3]]++; }
    for (; i < N; i++) h[0][s[i]]++;
    for (int k = 0; k < 256; k++) c[k] = h[0][k] + h[1][k] + h[2][k] + h[3][k];
  } else {
    const uint16_t* s = (const uint16_t*)syms;
    for (uint64_t i = 0; i < N; i++) c[s[i]]++;
  }
  size_t top = A;
  while (top > 1 && c[top - 1] == 0) top--;
  c.resize(top);
  if (N == 0) c.assign(1, 1);                  // empty input: a one-symbol table
  return quantize(c, n, freq);
}

}  // namespace recoil

using namespace recoil;

extern "C" {

const char* recoil_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// Encode with given quantised PDFs (validated by the callers), place splits.
// n_tables == 0: one static PDF; else freq holds n_tables rows and tid the
// row of every symbol.
static int encode_common(const void* syms, uint64_t n_syms, const recoil_params* params, std::vector<uint32_t> freq,
                         uint32_t n_tables, const uint8_t* tid, uint32_t max_splits, recoil_stream** out) {
  try {
    std::unique_ptr<recoil_stream> s(new recoil_stream());
    s->n_bits = params->n_bits;
    s->sym_bytes = params->sym_bytes;
    s->n_syms = n_syms;
    s->freq = std::move(freq);
    s->n_tables = n_tables;
    if (n_tables) s->tid = std::make_shared<const std::vector<uint8_t>>(tid, tid + n_syms);
    const uint32_t n = params->n_bits, A = s->alphabet();
    std::vector<EncSym> tab(s->freq.size());
    uint32_t F = 0;
    for (size_t k = 0; k < tab.size(); k++) {
      if (k % A == 0) F = 0;                               // each row is its own CDF
      const uint32_t f = s->freq[k];
      tab[k].f = f;
      tab[k].F = F;
      F += f;
      const uint64_t bound = (uint64_t)f << (32 - n);     // 2^(b-n) L f
      tab[k].xmax = bound == 0 ? 0xffffffffu : (uint32_t)std::min<uint64_t>(bound - 1, 0xffffffffull);
      if (f) tab[k].d.set(f);
    }
    auto words = std::make_shared<std::vector<uint16_t>>();
    words->resize(n_syms + 1);
    Records rec;
    rec.sym.resize(n_syms + 1);
    rec.y.resize(n_syms + 1);
    const uint8_t* t = n_tables ? s->tid->data() : nullptr;
    if (params->sym_bytes == 1) {
      if (n_tables) encode_loop<uint8_t, true>((const uint8_t*)syms, n_syms, tab, A, t, n, *words, rec, s->final_x);
      else encode_loop<uint8_t, false>((const uint8_t*)syms, n_syms, tab, A, t, n, *words, rec, s->final_x);
    } else {
      if (n_tables) encode_loop<uint16_t, true>((const uint16_t*)syms, n_syms, tab, A, t, n, *words, rec, s->final_x);
      else encode_loop<uint16_t, false>((const uint16_t*)syms, n_syms, tab, A, t, n, *words, rec, s->final_x);
    }
    words->shrink_to_fit();
    std::vector<uint64_t> qs;
    place_splits(rec, n_syms, max_splits, params->split_rule, qs);
    s->entries.resize(qs.size());
    for (size_t k = 0; k < qs.size(); k++) {
      Entry& e = s->entries[k];
      if (!entry_at(rec, qs[k], e)) return fail(RECOIL_ECORRUPT, "internal: split word not usable");
      // the decoder reads word p right after decoding symbol rec.sym[p] (Eq. 4
      // mirrors Eq. 3), so the thread that stops at symbol m reads no word
      // below the first one recorded for a symbol >= m
      const uint32_t m = *std::min_element(e.idx, e.idx + kW);
      e.wlo = (uint64_t)(std::lower_bound(rec.sym.begin(), rec.sym.end(), m) - rec.sym.begin());
      s->owned_end.push_back(m);
    }
    s->owned_end_ready = true;
    s->words = words;
    *out = s.release();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

static int check_params(const void* syms, uint64_t n_syms, const recoil_params* params, recoil_stream** out) {
  if (!params || !out || (!syms && n_syms)) return fail(RECOIL_EINVAL, "null argument");
  if (params->n_bits < 1 || params->n_bits > 16) return fail(RECOIL_EINVAL, "n_bits must be in [1, 16]");
  if (params->sym_bytes != 1 && params->sym_bytes != 2) return fail(RECOIL_EINVAL, "sym_bytes must be 1 or 2");
  if (params->split_rule != RECOIL_SPLIT_REMAINING && params->split_rule != RECOIL_SPLIT_EQ7)
    return fail(RECOIL_EINVAL, "split_rule must be RECOIL_SPLIT_REMAINING or RECOIL_SPLIT_EQ7");
  if (n_syms >= (1ull << 31)) return fail(RECOIL_EINVAL, "streams are limited to 2^31 - 1 symbols");
  *out = nullptr;
  return RECOIL_OK;
}

extern "C" {

int recoil_encode_with_splits(const void* syms, uint64_t n_syms, const recoil_params* params,
                              uint32_t max_splits, recoil_stream** out) {
  clear_error();
  int rc = check_params(syms, n_syms, params, out);
  if (rc) return rc;
  std::vector<uint32_t> freq;
  try {
    rc = make_table_syms(syms, n_syms, params->sym_bytes, params->n_bits, freq);
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
  if (rc) return rc;
  return encode_common(syms, n_syms, params, std::move(freq), 0, nullptr, std::max<uint32_t>(max_splits, 1), out);
}

int recoil_encode_with_table(const void* syms, uint64_t n_syms, const recoil_params* params, const uint32_t* freq,
                             uint32_t alphabet, uint32_t max_splits, recoil_stream** out) {
  clear_error();
  int rc = check_params(syms, n_syms, params, out);
  if (rc) return rc;
  if (!freq || alphabet < 1 || alphabet > (params->sym_bytes == 1 ? 256u : 65536u))
    return fail(RECOIL_EINVAL, "frequency table missing or alphabet out of range");
  uint64_t sum = 0;
  for (uint32_t k = 0; k < alphabet; k++) sum += freq[k];
  if (sum != (1ull << params->n_bits)) return fail(RECOIL_EINVAL, "frequencies must sum to 2^n");
  for (uint64_t i = 0; i < n_syms; i++) {
    const uint32_t v = params->sym_bytes == 1 ? ((const uint8_t*)syms)[i] : ((const uint16_t*)syms)[i];
    if (v >= alphabet || !freq[v]) return fail(RECOIL_EINVAL, "a symbol has no probability in the table");
  }
  return encode_common(syms, n_syms, params, std::vector<uint32_t>(freq, freq + alphabet), 0, nullptr,
                       std::max<uint32_t>(max_splits, 1), out);
}

int recoil_encode_adaptive(const void* syms, uint64_t n_syms, const recoil_params* params, const uint32_t* freq,
                           uint32_t n_tables, uint32_t alphabet, const uint8_t* table_index, uint32_t max_splits,
                           recoil_stream** out) {
  clear_error();
  int rc = check_params(syms, n_syms, params, out);
  if (rc) return rc;
  if (!freq || (!table_index && n_syms)) return fail(RECOIL_EINVAL, "null argument");
  if (n_tables < 1 || n_tables > kMaxTables) return fail(RECOIL_EINVAL, "n_tables must be in [1, 256]");
  const uint32_t amax = std::min<uint32_t>(params->sym_bytes == 1 ? 256u : kMaxAdaptiveAlphabet, 1u << params->n_bits);
  if (alphabet < 2 || alphabet > amax)
    return fail(RECOIL_EINVAL, "alphabet must be in [2, min(2^n, 4096)] (256 for 8-bit symbols)");
  for (uint32_t t = 0; t < n_tables; t++) {
    uint64_t sum = 0;
    for (uint32_t k = 0; k < alphabet; k++) {
      const uint32_t f = freq[(size_t)t * alphabet + k];
      if (f == 0) return fail(RECOIL_EINVAL, "an adaptive PDF row gives a symbol no probability");
      sum += f;
    }
    if (sum != (1ull << params->n_bits)) return fail(RECOIL_EINVAL, "every PDF row must sum to 2^n");
  }
  for (uint64_t i = 0; i < n_syms; i++) {
    const uint32_t v = params->sym_bytes == 1 ? ((const uint8_t*)syms)[i] : ((const uint16_t*)syms)[i];
    if (v >= alphabet) return fail(RECOIL_EINVAL, "a symbol lies outside the alphabet");
    if (table_index[i] >= n_tables) return fail(RECOIL_EINVAL, "a table number is not below n_tables");
  }
  return encode_common(syms, n_syms, params, std::vector<uint32_t>(freq, freq + (size_t)n_tables * alphabet),
                       n_tables, table_index, std::max<uint32_t>(max_splits, 1), out);
}

int recoil_combine_splits(const recoil_stream* in, uint32_t target, recoil_stream** out) {
  clear_error();
  if (!in || !out) return fail(RECOIL_EINVAL, "null argument");
  *out = nullptr;
  try {
    std::unique_ptr<recoil_stream> s(new recoil_stream());
    s->n_bits = in->n_bits;
    s->sym_bytes = in->sym_bytes;
    s->n_syms = in->n_syms;
    s->freq = in->freq;
    s->n_tables = in->n_tables;
    s->tid = in->tid;
    s->words = in->words;
    s->pinned_words = in->pinned_words;
    std::memcpy(s->final_x, in->final_x, sizeof s->final_x);
    std::vector<uint32_t> keep;
    combine_picks(*in, target, keep);
    const std::vector<uint32_t>& m = in->owned_ends();
    s->entries.reserve(keep.size());
    s->owned_end.reserve(keep.size());
    for (uint32_t pick : keep) {
      s->entries.push_back(in->entries[pick]);
      s->owned_end.push_back(m[pick]);
    }
    s->owned_end_ready = true;
    *out = s.release();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

int recoil_stream_info(const recoil_stream* s, recoil_info* o) {
  clear_error();
  if (!s || !o) return fail(RECOIL_EINVAL, "null argument");
  std::memset(o, 0, sizeof *o);
  o->n_syms = s->n_syms;
  o->n_words = s->n_words();
  o->n_entries = (uint32_t)s->entries.size() + 1;
  o->n_bits = s->n_bits;
  o->sym_bytes = s->sym_bytes;
  o->alphabet = s->alphabet();
  o->n_tables = s->n_tables;
  o->bitstream_bytes = 2 * o->n_words + 4ull * kW;
  o->metadata_bytes = (uint64_t)s->entries.size() * (8 + 2 * kW + 4 * kW);
  for (const Entry& e : s->entries) {
    uint32_t mn = e.idx[0], mx = e.idx[0];
    for (int j = 1; j < kW; j++) { mn = std::min(mn, e.idx[j]); mx = std::max(mx, e.idx[j]); }
    o->max_sync = std::max<uint64_t>(o->max_sync, (uint64_t)(mx - mn) + 1);
  }
  return RECOIL_OK;
}

int recoil_stream_export(const recoil_stream* s, uint32_t* freq, uint16_t* words, uint32_t* final_states,
                         uint64_t* entry_word, uint64_t* entry_index, uint16_t* entry_state) {
  clear_error();
  if (!s) return fail(RECOIL_EINVAL, "null argument");
  if (freq) std::memcpy(freq, s->freq.data(), s->freq.size() * 4);
  if (words && s->n_words()) std::memcpy(words, s->word_data(), s->n_words() * 2);
  if (final_states) std::memcpy(final_states, s->final_x, sizeof s->final_x);
  for (size_t k = 0; k < s->entries.size(); k++) {
    const Entry& e = s->entries[k];
    if (entry_word) entry_word[k] = e.word;
    for (int j = 0; j < kW; j++) {
      if (entry_index) entry_index[k * kW + j] = e.idx[j];
      if (entry_state) entry_state[k * kW + j] = e.y[j];
    }
  }
  return RECOIL_OK;
}

int recoil_stream_import(const recoil_params* params, uint64_t n_syms, uint32_t alphabet,
                         const uint32_t* freq, const uint16_t* words, uint64_t n_words,
                         const uint32_t* final_states, uint32_t n_regular, const uint64_t* entry_word,
                         const uint64_t* entry_index, const uint16_t* entry_state, recoil_stream** out) {
  clear_error();
  if (!params || !out || !freq || !final_states || (!words && n_words) ||
      (n_regular && (!entry_word || !entry_index || !entry_state)))
    return fail(RECOIL_EINVAL, "null argument");
  *out = nullptr;
  const uint32_t n = params->n_bits;
  if (n < 1 || n > 16) return fail(RECOIL_EINVAL, "n_bits must be in [1, 16]");
  if (params->sym_bytes != 1 && params->sym_bytes != 2) return fail(RECOIL_EINVAL, "sym_bytes must be 1 or 2");
  if (params->split_rule != RECOIL_SPLIT_REMAINING && params->split_rule != RECOIL_SPLIT_EQ7)
    return fail(RECOIL_EINVAL, "split_rule must be RECOIL_SPLIT_REMAINING or RECOIL_SPLIT_EQ7");
  if (alphabet < 1 || alphabet > (params->sym_bytes == 1 ? 256u : 65536u))
    return fail(RECOIL_EINVAL, "alphabet out of range");
  if (n_syms >= (1ull << 31) || n_words >= (1ull << 31)) return fail(RECOIL_EINVAL, "stream too long");
  uint64_t sum = 0;
  for (uint32_t k = 0; k < alphabet; k++) sum += freq[k];
  if (sum != (1ull << n)) return fail(RECOIL_ECORRUPT, "frequencies do not sum to 2^n");
  for (int j = 0; j < kW; j++)
    if (final_states[j] < kL) return fail(RECOIL_ECORRUPT, "final state below L");
  try {
    std::unique_ptr<recoil_stream> s(new recoil_stream());
    s->n_bits = n;
    s->sym_bytes = params->sym_bytes;
    s->n_syms = n_syms;
    s->freq.assign(freq, freq + alphabet);
    s->words = std::make_shared<std::vector<uint16_t>>(words, words + n_words);
    std::memcpy(s->final_x, final_states, sizeof s->final_x);
    s->entries.resize(n_regular);
    uint64_t prev_word = 0, prev_min = 0;
    for (uint32_t k = 0; k < n_regular; k++) {
      Entry& e = s->entries[k];
      e.word = entry_word[k];
      if (e.word >= n_words || (k && e.word <= prev_word))
        return fail(RECOIL_ECORRUPT, "split words must increase and lie inside the bitstream");
      uint64_t mn = ~0ull, mx = 0;
      for (int j = 0; j < kW; j++) {
        const uint64_t i = entry_index[(uint64_t)k * kW + j];
        if (i >= n_syms || (i & (kW - 1)) != (uint64_t)j)
          return fail(RECOIL_ECORRUPT, "recorded index not congruent to its coder or out of range");
        if (i + kW >= n_syms) return fail(RECOIL_ECORRUPT, "recorded index has no following symbol");
        e.idx[j] = (uint32_t)i;
        e.y[j] = entry_state[(uint64_t)k * kW + j];   // 16-bit: < L by construction (Lemma 3.1)
        mn = std::min(mn, i);
        mx = std::max(mx, i);
      }
      if (k && mn < prev_min) return fail(RECOIL_ECORRUPT, "entries' smallest indices must not decrease");
      (void)mx;
      prev_word = e.word;
      prev_min = mn;
      s->owned_end.push_back(mn);
    }
    s->owned_end_ready = true;
    *out = s.release();
    return RECOIL_OK;
  } catch (const std::bad_alloc&) {
    return fail(RECOIL_ENOMEM, "host allocation failed");
  }
}

int recoil_stream_pin(recoil_stream* s) {
  clear_error();
  if (!s) return fail(RECOIL_EINVAL, "null argument");
  if (s->pinned_words || !s->n_words()) return RECOIL_OK;
  void* p = nullptr;
  cudaError_t e = cudaHostAlloc(&p, s->n_words() * 2, cudaHostAllocPortable);
  if (e != cudaSuccess) return fail(RECOIL_ECUDA, std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
  std::memcpy(p, s->words->data(), s->n_words() * 2);
  s->pinned_words = std::shared_ptr<const uint16_t>((const uint16_t*)p, [](const uint16_t* q) {
    cudaFreeHost(const_cast<uint16_t*>(q));
  });
  return RECOIL_OK;
}

void recoil_free(recoil_stream* s) { delete s; }

}  // extern "C"
