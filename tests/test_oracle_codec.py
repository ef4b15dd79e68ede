"""Pins of the oracle's quantiser, encoder and serial decoder (no GPU).

What fixes each expectation:
* the codec is lossless, so the input symbols are ground truth (Sec. 2.1:
  encoding and decoding are inverse transforms, "rANS works like a stack");
* the serial decoder must end where the encoder started: every coder back at
  L and every word consumed (Eqs. 2 and 4 undo Eqs. 1 and 3);
* Lemma 3.1: a state taken right after an encoder renormalisation is < L;
* with f = 1 for all 256 byte values and n = 8, Eq. 1 is x -> 256 x + s, so a
  coder's state is a base-256 number and its words are pairs of its symbols
  (a closed form derived by hand, independent of the code);
* the code length of a static-model rANS coder is within a fraction of a
  percent of the quantised cross-entropy;
* the paper's Table 4 sizes for rand_lambda at n = 16 (Sec. 5.1).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ quantiser
@pytest.mark.parametrize("counts,n,want", [
    ([2, 1, 1], 2, [2, 1, 1]),            # exact proportions
    ([1, 1, 1, 1], 2, [1, 1, 1, 1]),
    ([3, 1], 3, [6, 2]),
    ([5, 3], 2, [2, 2]),                  # 2.5 -> 2 and 1.5 -> 2 (half to even)
    ([1, 1000], 4, [1, 15]),              # floor at 1, correction taken from the largest
    ([0, 7, 0, 1], 3, [0, 7, 0, 1]),      # absent symbols stay at 0
    ([10, 10, 10], 2, [2, 1, 1]),         # sum 3 -> one +1, given to the first of the ties
])
def test_quantize_hand_cases(counts, n, want):
    assert oracle.quantize(counts, n).tolist() == want


def test_quantize_rejects_too_many_symbols():
    with pytest.raises(ValueError):
        oracle.quantize([1, 1, 1, 1, 1], 2)


@pytest.mark.parametrize("seed", range(20))
def test_quantize_invariants(seed):
    g = np.random.default_rng(seed)
    A = int(g.integers(1, 300))
    n = int(g.integers(max(1, math.ceil(math.log2(A))), 17))
    c = g.integers(0, 1000, size=A) * (g.random(A) < 0.7)
    if c.sum() == 0:
        c[0] = 1
    if (c > 0).sum() > (1 << n):
        return
    f = oracle.quantize(c, n)
    assert int(f.sum()) == 1 << n
    assert np.all((f > 0) == (c > 0))


# ----------------------------------------------------------------- round trip
CASES = [
    ("laplace", dict(mean=128.0, scale=8.0), 11, 1),
    ("zipf", dict(s=1.2), 12, 1),
    ("skewed", dict(p0=0.95), 12, 1),
    ("uniform", {}, 12, 1),
    ("gauss16", dict(mean=2048.0, sigma=200.0, k=4096), 15, 2),
    ("expbytes", dict(lam=500.0), 16, 1),
]


def _stream(dist, params, n, sb, N, seed):
    return workloads.Stream("t", N, sb, n, dist, params, seed=seed).symbols()


@pytest.mark.parametrize("dist,params,n,sb", CASES)
@pytest.mark.parametrize("N", [0, 1, 31, 33, 1000, 65537])
def test_round_trip_and_end_state(dist, params, n, sb, N):
    s = _stream(dist, params, n, sb, max(N, 1), 11)[:N]
    A = 256 if sb == 1 else 4096
    counts = np.bincount(s, minlength=A) if N else np.eye(1, A, 0, dtype=np.int64)[0]
    f = oracle.quantize(counts, n)
    words, final, ev_sym, ev_y = oracle.encode(s, f, n)
    out, end_x, end_p = oracle.decode_serial(words, final, N, f, n)
    assert np.array_equal(out, s)
    assert end_p == -1
    assert np.all(end_x == 1 << 16)


@pytest.mark.parametrize("dist,params,n,sb", CASES)
def test_lemma_and_decoder_meets_every_record(dist, params, n, sb):
    """Each record (word p, state y) is exactly what the decoder holds after the symbol."""
    N = 20000
    s = _stream(dist, params, n, sb, N, 12)
    A = 256 if sb == 1 else 4096
    f = oracle.quantize(np.bincount(s, minlength=A), n)
    words, final, ev_sym, ev_y = oracle.encode(s, f, n)
    assert np.all(ev_y < (1 << 16))                      # Lemma 3.1
    out, _, _, tr_x, tr_p = oracle.decode_serial(words, final, N, f, n, trace=True)
    assert np.array_equal(out, s)
    p = np.arange(len(words))
    assert np.all(np.diff(ev_sym) > 0)                   # one word per symbol at most (b >= n)
    assert np.array_equal(tr_x[ev_sym], ev_y)
    assert np.array_equal(tr_p[ev_sym], p)


def _base256_words(sym, W):
    """Words of the f = 1, n = 8 code, built from digit pairs (no rANS arithmetic)."""
    lanes = [list(sym[j::W]) for j in range(W)]
    words = []
    for i in range(len(sym)):
        j, m = i % W, i // W
        t = lanes[j]
        if m == 1:
            words.append(int(t[0]))
        elif m >= 3 and m % 2 == 1:
            words.append((int(t[m - 2]) << 8) | int(t[m - 1]))
    final = []
    for j in range(W):
        t, k = lanes[j], len(lanes[j])
        if k == 0:
            final.append(1 << 16)
        elif k == 1:
            final.append((1 << 24) + int(t[0]))
        elif k % 2 == 1:
            final.append((1 << 24) + (int(t[k - 2]) << 8) + int(t[k - 1]))
        else:
            final.append((1 << 16) + int(t[k - 1]))
    return words, final


@pytest.mark.parametrize("N", [0, 1, 5, 32, 63, 64, 65, 500, 4099])
@pytest.mark.parametrize("W", [1, 4, 32])
def test_uniform_bytes_closed_form(N, W):
    s = np.random.default_rng(N * 7 + W).integers(0, 256, size=N).astype(np.uint32)
    f = np.ones(256, dtype=np.uint32)
    words, final, _, _ = oracle.encode(s, f, 8, W=W)
    want_words, want_final = _base256_words(s, W)
    assert words.tolist() == want_words
    assert final.tolist() == want_final


@pytest.mark.parametrize("dist,params,n,sb", CASES)
def test_size_near_quantised_cross_entropy(dist, params, n, sb):
    N = 1 << 20
    s = _stream(dist, params, n, sb, N, 13)
    A = 256 if sb == 1 else 4096
    c = np.bincount(s, minlength=A)
    f = oracle.quantize(c, n)
    words, final, _, _ = oracle.encode(s, f, n)
    nz = c > 0
    xent = float(-(c[nz] * np.log2(f[nz] / float(1 << n))).sum())
    bits = 16 * len(words) + 32 * 32
    assert bits >= xent * 0.999
    assert bits <= xent * 1.003 + 2 * 32 * 32 + 16


def test_table4_rand_sizes_n16():
    """Sec. 5.1, Table 4: compressed sizes of the rand_lambda files at n = 16."""
    gold = json.load(open(os.path.join(GOLDEN, "table4_rand_sizes.json")))
    for lam, kb in gold["compressed_kb_n16"].items():
        st = workloads.expbytes_10mb(float(lam))
        s = st.symbols()
        f = oracle.quantize(np.bincount(s, minlength=256), 16)
        words, final, _, _ = oracle.encode(s, f, 16)
        ours = (2 * len(words) + 4 * 32) / 1000.0
        assert abs(ours - kb) / kb < 0.03, (lam, ours, kb)
