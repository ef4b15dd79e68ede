"""Pins of the oracle's split metadata, split decoder, heuristic and combining (no GPU).

* Brute force: every sequence over 2- and 3-symbol alphabets up to length 8,
  W = 1..4, tiny parameters (n = 2, L = 2^4, b = 4); decoding from every
  subset of usable split words must give the input back (lossless codec,
  Sec. 3.1: decoding may start from any recorded intermediate state).
* The Sec. 4.1 walkthrough: which coders join in which order, which symbols
  of the synchronisation section are decoded and which are skipped, and the
  order of the renormalisation records the decoder consumes, all as the
  paper's prose states them.
* Def. 4.1 / Eq. 7: the chosen split word attains the minimum of H over all
  usable words after the previous split (exhaustive check of the early stop).
* Sec. 3.3 / 4.2: combining keeps every ceil(K/M')-th entry when M' divides
  K, always keeps the final entry, and never changes the decoded output.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SMALL = dict(n=2, lgL=4, b=4)


def _usable_words(ev_sym, ev_y, W):
    return [q for q in range(len(ev_sym)) if oracle.scan(ev_sym, ev_y, q, W)[0]]


def _stream_from_words(sym, f, W, qs, words, final, ev_sym, ev_y):
    idx, y = oracle.entries_for(ev_sym, ev_y, qs, W)
    y[-1] = final
    return oracle.OracleStream(len(sym), SMALL["n"], W, SMALL["lgL"], SMALL["b"], f, words, final,
                               ev_sym, ev_y, np.asarray(qs, dtype=np.int64), idx, y)


def test_brute_force_every_split_subset():
    decodes = 0
    for A in (2, 3):
        for N in range(0, 9):
            for seq in itertools.product(range(A), repeat=N):
                s = np.asarray(seq, dtype=np.uint32)
                counts = np.bincount(s, minlength=A) if N else np.ones(A, dtype=np.int64)
                f = oracle.quantize(counts, SMALL["n"])
                for W in (1, 2, 3, 4):
                    words, final, ev_sym, ev_y = oracle.encode(s, f, W=W, **SMALL)
                    out, end_x, end_p = oracle.decode_serial(words, final, N, f, W=W, **SMALL)
                    assert np.array_equal(out, s) and end_p == -1 and np.all(end_x == 16)
                    assert np.all(ev_y < 16)
                    usable = _usable_words(ev_sym, ev_y, W)
                    for r in range(len(usable) + 1):
                        for qs in itertools.combinations(usable, r):
                            st = _stream_from_words(s, f, W, list(qs), words, final, ev_sym, ev_y)
                            assert np.array_equal(oracle.decode_splits(st), s), (seq, W, qs)
                            decodes += 1
    assert decodes > 50000


def test_walkthrough_of_section_4_1():
    g = json.load(open(os.path.join(GOLDEN, "walkthrough_w4.json")))
    W = g["W"]
    P = dict(n=g["n"], lgL=g["lgL"], b=g["b"])
    s = np.asarray(g["symbols"], dtype=np.uint32)
    f = np.asarray(g["f"], dtype=np.uint32)
    words, final, ev_sym, ev_y = oracle.encode(s, f, W=W, **P)
    q = g["split_word"]
    ok, idx, y, wp = oracle.scan(ev_sym, ev_y, q, W)
    assert ok
    # paper (1-based): x_{9,1}, x_{14,2}, x_{11,3}, x_{16,4}
    assert [int(v) + 1 for v in idx] == [9, 14, 11, 16]
    # group IDs ceil(i / W) of Table 2 and their anchor
    assert [-(-(int(v) + 1) // W) for v in idx] == [3, 4, 3, 4]

    st = oracle.OracleStream(len(s), P["n"], W, P["lgL"], P["b"], f, words, final, ev_sym, ev_y,
                             np.asarray([q]), np.vstack([idx, np.zeros(W, np.int64)]),
                             np.vstack([y, final]))
    out, tr, tw = oracle.decode_thread(st, 1, trace=True)      # the thread that crosses into it
    lo, hi = oracle.owned_range(st, 1)
    assert lo == 8                                             # stops at s_9 (1-based), Sec. 4.1.3
    out0, tr0, tw0 = oracle.decode_thread(st, 0, trace=True)   # the thread starting at the split

    sync = range(8, 16)                                        # s_9 .. s_16 (1-based)
    decoded = [i + 1 for i in sync if tr0[i] in (oracle.TR_DECODE, oracle.TR_STORE)]
    skipped = [i + 1 for i in sync if tr0[i] in (oracle.TR_SKIP, oracle.TR_INIT)]
    assert sorted(decoded) == [9, 10, 11, 12, 14, 16]          # Sec. 4.1.1
    assert sorted(skipped) == [13, 15]
    joins = [int(i) % W + 1 for i in range(len(tr0) - 1, -1, -1) if tr0[i] == oracle.TR_INIT]
    assert joins == [4, 2, 3, 1]                               # D4, D2, D3, D1
    # records consumed in the synchronisation phase: a5 (E4), ea (E2), 26 (E4), then E3, E1
    last_join = min(i for i in range(len(tr0)) if tr0[i] == oracle.TR_INIT)
    reads = [(int(i), int(tw0[i])) for i in range(len(tr0) - 1, last_join - 1, -1) if tw0[i] >= 0]
    assert [w for _, w in reads] == [q, q - 1, q - 2, q - 3, q - 4]
    assert [int(ev_sym[w]) % W + 1 for _, w in reads] == [4, 2, 4, 3, 1]
    # nothing of the synchronisation section is stored by the thread that starts there
    assert all(tr0[i] != oracle.TR_STORE for i in sync)
    # the crossing thread decodes and stores the whole section, ending at s_9
    assert all(tr[i] == oracle.TR_STORE for i in range(8, len(s)))
    full = out.copy()
    full[:8] = out0[:8]
    assert np.array_equal(full, s)


def _H(top, m, lo, T):
    t, ts = top + 1 - lo, top + 1 - m
    return abs(t - T) + abs(t - ts - T)


@pytest.mark.parametrize("dist,params,n,M", [
    ("laplace", dict(mean=128.0, scale=8.0), 11, 16),
    ("zipf", dict(s=1.2), 12, 9),
    ("skewed", dict(p0=0.95), 12, 5),
])
def test_heuristic_attains_minimum_of_eq7(dist, params, n, M):
    s = workloads.Stream("t", 12000, 1, n, dist, params, seed=3).symbols()
    st = oracle.encode_with_splits(s, n, M)
    lo, qprev = 0, -1
    cand = []
    for q in range(len(st.words)):
        ok, idx, _, _ = oracle.scan(st.ev_sym, st.ev_y, q, 32)
        if ok:
            cand.append((q, int(idx.max()), int(idx.min())))
    for k, q in enumerate(st.q):
        T = -(-(st.N - lo) // (M - k))                 # expected symbols per remaining split
        rest = [(c, _H(top, m, lo, T)) for c, top, m in cand if c > qprev]
        best = min(h for _, h in rest)
        first = min(c for c, h in rest if h == best)
        assert q == first
        lo = int(st.idx[k].min())
        qprev = q
    assert st.K <= M


@pytest.mark.parametrize("K,Mp", [(64, 16), (64, 1), (64, 64), (65536, 148), (10, 3), (7, 20), (9, 9)])
def test_combine_keep_rule(K, Mp):
    """Sec. 3.3: on evenly spaced splits, keeping the entries nearest to equal
    symbol counts is the paper's simple rule, every (K/M')-th entry."""
    N = 1000 * K
    m = np.arange(1, K) * 1000                      # regular entry e owns [1000 e, 1000 (e + 1))
    keep = oracle.combine_keep(m, N, Mp)
    assert len(keep) == min(K, Mp)
    assert keep[-1] == K - 1
    assert np.all(np.diff(keep) > 0)
    if Mp <= K and K % Mp == 0:
        assert keep.tolist() == list(range(K // Mp - 1, K, K // Mp))


def test_combine_keep_hand_cases():
    # nearest owned end wins
    assert oracle.combine_keep([10, 19, 33], 40, 2).tolist() == [1, 3]
    # equidistant ends: the smaller one, and the first of equal ends
    assert oracle.combine_keep([10, 10, 30], 40, 2).tolist() == [0, 3]
    # each later target keeps an entry of its own
    assert oracle.combine_keep([5, 6, 7, 100], 200, 4).tolist() == [1, 2, 3, 4]
    # a target past every end takes the last entry that still leaves room
    assert oracle.combine_keep([1, 2, 3, 4, 5], 1000, 3).tolist() == [3, 4, 5]
    # nothing to combine
    assert oracle.combine_keep([], 7, 5).tolist() == [0]


def test_combine_balances_uneven_splits():
    """Sec. 3.3 asks for combined splits of close symbol counts. Splits encoded
    on a skewed source own fewer symbols than T early on (long synchronisation
    sections) and more towards the end; every ceil(K/M')-th entry would pass
    that drift on, the nearest-end rule does not."""
    s = workloads.Stream("sk", 1 << 20, 1, 12, "skewed", {"p0": 0.95}, seed=3).symbols()
    o = oracle.encode_with_splits(s, 12, 256)
    mins = o.idx[:-1].min(axis=1)
    enc_owned = np.diff(np.concatenate([[0], mins, [len(s)]]))
    every = np.diff(np.concatenate([[0], mins[np.arange(1, 16) * o.K // 16 - 1], [len(s)]]))
    assert enc_owned[-16:].mean() > 1.5 * enc_owned[:16].mean()        # the drift exists
    assert every.max() > 1.3 * len(s) / 16
    c = oracle.combined(o, 16)
    owned = np.diff(np.concatenate([[0], c.idx[:-1].min(axis=1), [len(s)]]))
    assert np.abs(owned - len(s) / 16).max() <= enc_owned.max()
    assert np.array_equal(oracle.decode_splits(c), s)


def test_config1_split_decodes_and_combines():
    st = workloads.laplace_1mib()
    s = st.symbols()
    o = oracle.encode_with_splits(s, st.n_bits, 64)
    assert o.K == 64
    assert np.all(o.y[:-1] < (1 << 16))
    assert np.all(np.diff(o.q) > 0)
    mins = o.idx[:-1].min(axis=1)
    assert np.all(np.diff(mins) >= 0)
    for Mp in (64, 16, 1):
        c = oracle.combined(o, Mp)
        assert np.array_equal(oracle.decode_splits(c), s)
    # every split, the final one included, owns T give or take two synchronisation sections
    T = -(-len(s) // 64)
    sync = int((o.idx[:-1].max(axis=1) - mins).max()) + 32
    owned = np.diff(np.concatenate([[0], mins, [len(s)]]))
    assert np.all(np.abs(owned - T) <= 2 * sync)


@pytest.mark.parametrize("M", [4, 32])
def test_lowest_word_read_by_a_thread(M):
    """A thread that stops at symbol lo reads no word below the first word whose renormalisation
    event is at a symbol >= lo (decoding mirrors encoding word for word), and does read that one:
    shard plans stage words from there on."""
    st = workloads.Stream("z", 200_003, 1, 12, "zipf", {"s": 1.2}, seed=90).symbols()
    o = oracle.encode_with_splits(st, 12, M)
    for k in range(1, o.K):
        lo, hi = oracle.owned_range(o, k)
        out, tr, tw = oracle.decode_thread(o, k, trace=True)
        read = tw[tw >= 0]
        want = int(np.searchsorted(o.ev_sym, lo, side="left"))
        assert read.min() == want, (k, read.min(), want)
