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


@pytest.mark.parametrize("rule", ["eq7", "remaining"])
@pytest.mark.parametrize("dist,params,n,M", [
    ("laplace", dict(mean=128.0, scale=8.0), 11, 16),
    ("zipf", dict(s=1.2), 12, 9),
    ("skewed", dict(p0=0.95), 12, 5),
])
def test_heuristic_attains_minimum_of_eq7(dist, params, n, M, rule):
    """Every split word is the first usable word after the previous one that minimises
    Eq. 7, over all usable words (no early stop); T = ceil(N/M) as printed ("eq7") or
    over the symbols left ("remaining")."""
    s = workloads.Stream("t", 12000, 1, n, dist, params, seed=3).symbols()
    st = oracle.encode_with_splits(s, n, M, rule=rule)
    lo, qprev = 0, -1
    cand = []
    for q in range(len(st.words)):
        ok, idx, _, _ = oracle.scan(st.ev_sym, st.ev_y, q, 32)
        if ok:
            cand.append((q, int(idx.max()), int(idx.min())))
    for k, q in enumerate(st.q):
        T = -(-st.N // M) if rule == "eq7" else -(-(st.N - lo) // (M - k))
        rest = [(c, _H(top, m, lo, T)) for c, top, m in cand if c > qprev]
        best = min(h for _, h in rest)
        first = min(c for c, h in rest if h == best)
        assert q == first
        lo = int(st.idx[k].min())
        qprev = q
    assert st.K <= M


def _digit_stream(N):
    """One coder (W = 1), n = 8, every f = 1, L = 2^16, b = 16: each symbol is a base-256
    digit of the state, so a word leaves every second symbol. Worked by hand from
    Eqs. 1 and 3: from x = 2^16, coding a symbol gives 2^24 + s, the next one first
    writes the low 16 bits and leaves 2^8, so word q is written while coding symbol
    2q + 1 and its record (Sec. 4.1) is the state 2^8 at index 2q."""
    s = np.random.default_rng(N).integers(0, 256, N).astype(np.uint32)
    words, final, ev_sym, ev_y = oracle.encode(s, np.ones(256, dtype=np.uint32), 8, 1, 16, 16)
    assert len(words) == N // 2
    assert np.array_equal(ev_sym, 2 * np.arange(N // 2) + 1) and np.all(ev_y == 256)
    return ev_sym, ev_y


@pytest.mark.parametrize("N,M,eq7,remaining", [
    # T = ceil(100 / 3) = 34 (even): word q gives t = 2q + 1 - lo, t_s = 1, so
    # H = |2q + 1 - lo - T| + |2q - lo - T| is 1 exactly at 2q = lo + T: q = 17, then
    # lo = 34 and q = 34. With T over what is left the second split has
    # T = ceil(66 / 2) = 33 (odd), where H = 1 at 2q = lo + T - 1: q = 33.
    (100, 3, [17, 34], [17, 33]),
    # T = 25 (odd): 2q = lo + 24 each time, q = 12, 24, 36. Left-over T: 25, then
    # ceil(76 / 3) = 26 (2q = 24 + 26, q = 25), then ceil(50 / 2) = 25 (2q = 50 + 24, q = 37).
    (100, 4, [12, 24, 36], [12, 25, 37]),
    # T = ceil(99 / 3) = 33: q = 16 (m = 32), then q = 32. Left over: ceil(67 / 2) = 34, q = 33.
    (99, 3, [16, 32], [16, 33]),
    # T = 51: q = 25 for both (one split word only).
    (101, 2, [25], [25]),
])
def test_heuristic_hand_cases(N, M, eq7, remaining):
    """Def. 4.1 / Eq. 7 on a stream whose records are known in closed form: the split
    words derived by hand for the printed T = ceil(N/M) and for T over the symbols left."""
    ev_sym, ev_y = _digit_stream(N)
    assert oracle.heuristic(ev_sym, ev_y, N, M, 1, "eq7").tolist() == eq7
    assert oracle.heuristic(ev_sym, ev_y, N, M, 1, "remaining").tolist() == remaining


@pytest.mark.parametrize("N", [200, 1001, 4096])
@pytest.mark.parametrize("M", [2, 5, 16, 33])
def test_heuristic_eq7_closed_form(N, M):
    """On the digit stream the printed rule has a closed form: with t_s = 1, Eq. 7 is 1
    exactly at the even owned end lo + 2 floor(T / 2), so split k ends at
    (k + 1) 2 floor(T / 2) with T = ceil(N / M): equal splits, and the final one takes
    what is left over."""
    ev_sym, ev_y = _digit_stream(N)
    T = -(-N // M)
    want = [(k + 1) * (T // 2) for k in range(M - 1) if (k + 1) * (T // 2) < N // 2]
    assert oracle.heuristic(ev_sym, ev_y, N, M, 1, "eq7").tolist() == want


def test_printed_rule_piles_the_shortfall_into_the_final_split():
    """With T = ceil(N/M) every split is short of T by about half its synchronisation
    section and the final split collects the rest; with T over the symbols left the
    final split stays near T (the reason the library takes that reading by default)."""
    s = workloads.Stream("z", 1 << 18, 1, 12, "zipf", {"s": 1.2}, seed=4).symbols()
    M = 256
    T = -(-len(s) // M)
    last = {}
    for rule in ("eq7", "remaining"):
        st = oracle.encode_with_splits(s, 12, M, rule=rule)
        assert st.K == M
        owned = np.diff(np.r_[0, st.idx[:-1].min(axis=1), len(s)])
        assert owned.sum() == len(s)
        if rule == "eq7":
            assert owned[:-1].mean() < T                     # regular splits fall short of T on average
        last[rule] = int(owned[-1])
    assert last["eq7"] > 4 * T
    assert last["remaining"] < 2 * T


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
