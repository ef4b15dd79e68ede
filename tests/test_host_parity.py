"""Host side of the library against the oracle (no GPU).

The library's encoder, split placement and combiner are separate code from
the oracle's, written to the same rules (quantiser reading, Eqs. 1 and 3,
Sec. 4.1 backward scan, Def. 4.1 / Eq. 7, Sec. 3.3 combining). Everything is
integer, so parity is bit-exact: frequency table, words, final states, split
words, recorded indices and states.
"""
import numpy as np
import pytest

import oracle
import workloads


def _cases():
    yield workloads.laplace_1mib()
    yield workloads.Stream("zipf", 300_001, 1, 12, "zipf", {"s": 1.2}, seed=21)
    yield workloads.Stream("skewed", 200_003, 1, 12, "skewed", {"p0": 0.95}, seed=22)
    yield workloads.Stream("uniform", 100_000, 1, 12, "uniform", {}, seed=23)
    yield workloads.Stream("gauss16", 150_017, 2, 15, "gauss16", {"mean": 2048.0, "sigma": 200.0, "k": 4096}, seed=24)
    yield workloads.Stream("exp_n16", 120_000, 1, 16, "expbytes", {"lam": 200.0}, seed=25)
    yield workloads.Stream("lap_n8", 70_001, 1, 8, "laplace", {"mean": 128.0, "scale": 3.0}, seed=26)


def _same(R, s, n, M, rule="remaining"):
    p = R.encode_with_splits(s, n, M, rule=rule)
    o = oracle.encode_with_splits(s, n, M, alphabet=None, rule=rule)
    e = p.export()
    assert np.array_equal(e["freq"], o.f)
    assert np.array_equal(e["words"], o.words)
    assert np.array_equal(e["final"], o.final)
    assert np.array_equal(e["entry_word"].astype(np.int64), o.q)
    assert np.array_equal(e["entry_index"].astype(np.int64), o.idx[:-1])
    assert np.array_equal(e["entry_state"].astype(np.uint32), o.y[:-1])
    return p, o


@pytest.mark.parametrize("st", list(_cases()), ids=lambda s: s.name)
@pytest.mark.parametrize("M", [1, 2, 64, 1000])
def test_encoder_matches_oracle(recoil_lib, st, M):
    _same(recoil_lib, st.symbols(), st.n_bits, M)


@pytest.mark.parametrize("st", list(_cases())[1:4], ids=lambda s: s.name)
@pytest.mark.parametrize("M", [2, 64, 1000])
def test_encoder_matches_oracle_printed_rule(recoil_lib, st, M):
    """The printed T = ceil(N/M) of Def. 4.1 (RECOIL_SPLIT_EQ7): same split words as the oracle."""
    _same(recoil_lib, st.symbols(), st.n_bits, M, rule="eq7")


def test_split_rules_differ_and_default(recoil_lib):
    """The two rules place different words on a skewed source; the default is the remaining rule."""
    s = workloads.Stream("sk", 200_003, 1, 12, "skewed", {"p0": 0.95}, seed=22).symbols()
    a = recoil_lib.encode_with_splits(s, 12, 64).export()["entry_word"]
    r = recoil_lib.encode_with_splits(s, 12, 64, rule="remaining").export()["entry_word"]
    e = recoil_lib.encode_with_splits(s, 12, 64, rule="eq7").export()["entry_word"]
    assert np.array_equal(a, r) and not np.array_equal(r, e)
    with pytest.raises(ValueError):
        recoil_lib.encode_with_splits(s, 12, 64, rule="other")


@pytest.mark.parametrize("N", [0, 1, 2, 31, 32, 33, 63, 64, 65, 100, 1023])
@pytest.mark.parametrize("M", [1, 3, 16])
def test_edge_lengths_match_oracle(recoil_lib, N, M):
    s = workloads.Stream("t", max(N, 1), 1, 10, "laplace", {"mean": 128.0, "scale": 2.0}, seed=N).symbols()[:N]
    if N == 0:
        p = recoil_lib.encode_with_splits(s, 10, M)
        assert p.info["n_words"] == 0 and p.info["n_entries"] == 1
        return
    _same(recoil_lib, s, 10, M)


@pytest.mark.parametrize("sym", [0, 7, 255])
@pytest.mark.parametrize("n", [1, 12, 16])
def test_single_symbol_stream(recoil_lib, sym, n):
    s = np.full(5000, sym, dtype=np.uint8)
    p, o = _same(recoil_lib, s, n, 8)
    assert p.info["n_words"] == 0 and p.info["n_entries"] == 1      # f = 2^n never renormalises
    assert np.all(o.final == 1 << 16)


@pytest.mark.parametrize("K,Mp", [(64, 16), (64, 1), (64, 64), (64, 100), (37, 5), (9472, 148)])
def test_combine_matches_oracle_rule(recoil_lib, K, Mp):
    s = workloads.Stream("t", K * 600, 1, 11, "laplace", {"mean": 128.0, "scale": 8.0}, seed=K).symbols()
    p = recoil_lib.encode_with_splits(s, 11, K)
    assert p.info["n_entries"] == K
    c = recoil_lib.combine_splits(p, Mp)
    ep, ec = p.export(), c.export()
    keep = oracle.combine_keep(ep["entry_index"].astype(np.int64).min(axis=1), len(s), Mp)
    regular = [k for k in keep if k < K - 1]
    assert c.info["n_entries"] == len(keep)
    assert np.array_equal(ec["entry_word"], ep["entry_word"][regular])
    assert np.array_equal(ec["entry_index"], ep["entry_index"][regular])
    assert np.array_equal(ec["words"], ep["words"])


def test_combine_matches_oracle_rule_on_uneven_splits(recoil_lib):
    """A skewed source: encoded split sizes drift along the stream and many entries share an
    owned end, so the nearest-end choice, its ties and the window that leaves room for later
    targets all matter; every target count from 1 to K agrees with the oracle."""
    s = workloads.Stream("sk", 1 << 18, 1, 12, "skewed", {"p0": 0.95}, seed=8).symbols()
    p = recoil_lib.encode_with_splits(s, 12, 96)
    ep = p.export()
    K = p.info["n_entries"]
    ends = ep["entry_index"].astype(np.int64).min(axis=1)
    for Mp in range(1, K + 2):
        c = recoil_lib.combine_splits(p, Mp)
        keep = oracle.combine_keep(ends, len(s), Mp)
        regular = [k for k in keep if k < K - 1]
        assert np.array_equal(c.export()["entry_word"], ep["entry_word"][regular]), Mp


def test_import_round_trip_and_validation(recoil_lib):
    R = recoil_lib
    st = workloads.laplace_1mib(1 << 16)
    o = oracle.encode_with_splits(st.symbols(), 11, 8)
    args = dict(n_bits=11, sym_bytes=1, n_syms=o.N, freq=o.f, words=o.words, final=o.final,
                entry_word=o.q, entry_index=o.idx[:-1], entry_state=o.y[:-1])
    s = R.stream_import(**args)
    e = s.export()
    assert np.array_equal(e["words"], o.words) and np.array_equal(e["entry_word"].astype(np.int64), o.q)

    def bad(**kw):
        a = dict(args)
        a.update(kw)
        with pytest.raises(R.RecoilError) as err:
            R.stream_import(**a)
        return err.value.code

    f = o.f.copy()
    f[0] += 1
    assert bad(freq=f) == R.ECORRUPT                               # does not sum to 2^n
    idx = o.idx[:-1].copy()
    idx[0, 3] += 1
    assert bad(entry_index=idx) == R.ECORRUPT                      # not congruent to its coder
    assert bad(entry_word=o.q[::-1].copy()) == R.ECORRUPT          # words not increasing
    fin = o.final.copy()
    fin[5] = 10
    assert bad(final=fin) == R.ECORRUPT                            # final state below L
    assert bad(n_bits=17) == R.EINVAL


def test_encode_with_given_table_matches_oracle(recoil_lib):
    R = recoil_lib
    s = workloads.Stream("z", 200_000, 1, 12, "zipf", {"s": 1.2}, seed=71).symbols()
    f = oracle.quantize(np.bincount(s, minlength=256), 12)
    parts = [s[i:i + 20_000] for i in range(0, len(s), 20_000)]      # partitions share one model
    for part in parts:
        p = R.encode_with_table(part, 12, f, 4)
        words, final, ev_sym, ev_y = oracle.encode(part, f, 12)
        e = p.export()
        assert np.array_equal(e["freq"], f) and np.array_equal(e["words"], words)
        assert np.array_equal(e["final"], final)
    bad = f.copy()
    bad[s[0]] = 0
    bad[255] += f[s[0]]
    with pytest.raises(R.RecoilError):
        R.encode_with_table(s, 12, bad, 4)                        # an occurring symbol without probability
    with pytest.raises(R.RecoilError):
        R.encode_with_table(s, 12, f[:-1], 4) if f[-1] else R.encode_with_table(s, 12, f * 2, 4)


def test_shard_plans_stage_only_their_word_window(recoil_lib):
    """A shard plan's workspace holds the words its run reads, not the whole stream: with four
    ranks each stages about a quarter of the words (plus descriptors); an imported stream, whose
    lowest-word records are unknown, stages every word from the start of the stream."""
    R = recoil_lib
    st = workloads.Stream("z", 3_000_017, 1, 12, "zipf", {"s": 1.2}, seed=91)
    s = st.symbols()
    p = R.combine_splits(R.encode_with_splits(s, 12, 512), 64)
    words = 2 * p.info["n_words"]
    full = R.Plan([p], {"warps_per_cta": 8}).workspace_size
    sizes = [R.Plan.shard(p, 4, r, {"warps_per_cta": 8})[0].workspace_size for r in range(4)]
    assert all(sz < full - words // 2 for sz in sizes), (sizes, full, words)
    assert sum(sizes) < full + words // 4 + 4 * (full - words)
    e = p.export()
    imp = R.stream_import(12, 1, len(s), e["freq"], e["words"], e["final"], e["entry_word"], e["entry_index"],
                          e["entry_state"])
    imp_sizes = [R.Plan.shard(imp, 4, r, {"warps_per_cta": 8})[0].workspace_size for r in range(4)]
    assert imp_sizes[0] == sizes[0] and all(a > b for a, b in zip(imp_sizes[1:], sizes[1:]))
    assert imp_sizes[3] >= words


def test_adaptive_shard_plans_stage_a_window_of_table_numbers(recoil_lib):
    R = recoil_lib
    a = workloads.AdaptiveStream("t", 2_000_003, seed=92)
    tables = a.tables()
    s, tid = a.draw()
    p = R.combine_splits(R.encode_adaptive(s, 16, tables, tid, 512), 64)
    full = R.Plan([p], {"warps_per_cta": 8}).workspace_size
    sizes = [R.Plan.shard(p, 4, r, {"warps_per_cta": 8})[0].workspace_size for r in range(4)]
    staged = 2 * p.info["n_words"] + len(s)               # words + one table number per symbol
    assert all(sz < full - staged // 2 for sz in sizes), (sizes, full, staged)
