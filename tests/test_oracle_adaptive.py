"""Pins of the oracle's adaptive coding (Sec. 3.1: the PDF of every coding step
is chosen by the symbol index, as in hyperprior image codecs) -- no GPU.

* One table, or identical tables, reduce to the static coder already pinned
  (same words, final states and records).
* A closed form (n = 8, derived by hand): a uniform table with f = 1 makes
  every symbol a base-256 digit; a table that gives one symbol all 2^n slots
  leaves the state unchanged (x -> floor(x / 2^n) 2^n + x mod 2^n) and never
  renormalises. Mixing the two per index, the words must be exactly the
  digit pairs of the uniform-coded symbols, in coding order.
* Brute force: every symbol sequence and every table assignment over two
  tables of a 2-symbol alphabet, lengths up to 6, W = 1..3, decoded serially
  and from every subset of usable split words.
* Code length within a fraction of a percent of the ideal cost
  sum_i -log2(f_{t_i}(s_i) / 2^n) (a coder using the wrong row for a symbol
  pays for it here, even though it would still decode).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import workloads

SMALL = dict(n=2, lgL=4, b=4)


def _static_stream(N, seed):
    return workloads.Stream("t", N, 1, 11, "laplace", {"mean": 128.0, "scale": 6.0}, seed=seed).symbols()


@pytest.mark.parametrize("N", [0, 1, 31, 33, 5000, 70001])
def test_one_table_is_the_static_coder(N):
    s = _static_stream(max(N, 1), N)[:N].astype(np.uint32)
    counts = np.bincount(s, minlength=256) if N else np.ones(256)
    f = oracle.quantize(counts, 11)
    a = oracle.encode_adaptive(s, np.zeros(N, dtype=np.uint32), f[None, :], 11)
    b = oracle.encode(s, f, 11)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_identical_rows_are_the_static_coder():
    s = _static_stream(40000, 3).astype(np.uint32)
    f = oracle.quantize(np.bincount(s, minlength=256), 11)
    tid = np.random.default_rng(4).integers(0, 5, size=len(s))
    a = oracle.encode_adaptive(s, tid, np.stack([f] * 5), 11)
    b = oracle.encode(s, f, 11)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    out, end_x, end_p = oracle.decode_serial_adaptive(a[0], a[1], tid, np.stack([f] * 5), 11)
    assert np.array_equal(out, s) and end_p == -1 and np.all(end_x == 1 << 16)


def _digit_words(sym, tid, W):
    """Words and final states of the uniform/certain mix, from digit pairs (no rANS arithmetic)."""
    lanes = [[] for _ in range(W)]
    words = []
    for i in range(len(sym)):
        j = i % W
        if tid[i] == 1:
            continue                          # coded with certainty: no state change, no word
        t = lanes[j]
        m = len(t)
        t.append(int(sym[i]))
        if m == 1:
            words.append(t[0])
        elif m >= 3 and m % 2 == 1:
            words.append((t[m - 2] << 8) | t[m - 1])
    final = []
    for t in lanes:
        k = len(t)
        if k == 0:
            final.append(1 << 16)
        elif k == 1:
            final.append((1 << 24) + t[0])
        elif k % 2 == 1:
            final.append((1 << 24) + (t[k - 2] << 8) + t[k - 1])
        else:
            final.append((1 << 16) + t[k - 1])
    return words, final


@pytest.mark.parametrize("N", [0, 1, 7, 64, 65, 999, 4097])
@pytest.mark.parametrize("W", [1, 4, 32])
def test_uniform_and_certain_rows_closed_form(N, W):
    rng = np.random.default_rng(N * 31 + W)
    tid = rng.integers(0, 2, size=N).astype(np.uint32)
    sym = np.where(tid == 0, rng.integers(0, 256, size=N), 0).astype(np.uint32)
    tables = np.zeros((2, 256), dtype=np.uint32)
    tables[0, :] = 1                          # uniform: f = 1 for every byte, n = 8
    tables[1, 0] = 256                        # certain: symbol 0 owns all 2^8 slots
    words, final, _, _ = oracle.encode_adaptive(sym, tid, tables, 8, W=W)
    want_words, want_final = _digit_words(sym, tid, W)
    assert words.tolist() == want_words
    assert final.tolist() == want_final
    out, end_x, end_p = oracle.decode_serial_adaptive(words, final, tid, tables, 8, W=W)
    assert np.array_equal(out, sym) and end_p == -1 and np.all(end_x == 1 << 16)


def _usable_words(ev_sym, ev_y, W):
    return [q for q in range(len(ev_sym)) if oracle.scan(ev_sym, ev_y, q, W)[0]]


def test_brute_force_tables_and_splits():
    tables = np.array([[1, 3], [3, 1]], dtype=np.uint32)     # n = 2
    decodes = 0
    for N in range(0, 7):
        for seq in itertools.product(range(2), repeat=N):
            s = np.asarray(seq, dtype=np.uint32)
            for tseq in itertools.product(range(2), repeat=N):
                tid = np.asarray(tseq, dtype=np.uint32)
                for W in (1, 2, 3):
                    words, final, ev_sym, ev_y = oracle.encode_adaptive(s, tid, tables, W=W, **SMALL)
                    out, end_x, end_p = oracle.decode_serial_adaptive(words, final, tid, tables, W=W, **SMALL)
                    assert np.array_equal(out, s) and end_p == -1 and np.all(end_x == 16)
                    assert np.all(ev_y < 16)                 # Lemma 3.1 with per-index PDFs
                    usable = _usable_words(ev_sym, ev_y, W)
                    for r in range(len(usable) + 1):
                        for qs in itertools.combinations(usable, r):
                            idx, y = oracle.entries_for(ev_sym, ev_y, list(qs), W)
                            y[-1] = final
                            st = oracle.OracleStream(N, SMALL["n"], W, SMALL["lgL"], SMALL["b"], tables, words,
                                                     final, ev_sym, ev_y, np.asarray(qs, dtype=np.int64), idx,
                                                     y, tid)
                            assert np.array_equal(oracle.decode_splits(st), s), (seq, tseq, W, qs)
                            decodes += 1
    assert decodes > 20000


def test_code_length_near_ideal_cost():
    a = workloads.AdaptiveStream("t", 1 << 20, seed=11)
    tables = a.tables()
    s, tid = a.draw()
    words, final, _, _ = oracle.encode_adaptive(s, tid, tables, a.n_bits)
    ideal = float(-np.log2(tables[tid, s].astype(np.float64) / (1 << a.n_bits)).sum())
    bits = 16.0 * len(words)
    state_bits = 32 * 32                     # the final states carry the rest of the message
    assert ideal - state_bits <= bits <= ideal * 1.003 + state_bits, (bits, ideal)
    # the same symbols coded with every index's neighbouring row cost clearly more
    shifted = np.minimum(tid.astype(np.int64) + 8, a.n_tables - 1)
    wrong = float(-np.log2(tables[shifted, s].astype(np.float64) / (1 << a.n_bits)).sum())
    assert wrong > 1.05 * ideal


@pytest.mark.parametrize("M", [1, 16, 64])
def test_split_decode_of_adaptive_stream(M):
    a = workloads.AdaptiveStream("t", 300_001, seed=12)
    tables = a.tables()
    s, tid = a.draw()
    o = oracle.encode_adaptive_with_splits(s, tid, tables, a.n_bits, 64)
    st = oracle.combined(o, M)
    assert np.array_equal(oracle.decode_splits(st), s)
    # every thread alone reproduces its own range
    for k in range(st.K):
        lo, hi = oracle.owned_range(st, k)
        out = oracle.decode_thread(st, k)
        assert np.array_equal(out[lo:hi + 1], s[lo:hi + 1])
