"""Adaptive coding (Sec. 3.1: the PDF of every coding step is chosen by the
symbol index) in the library, against the oracle.

CPU: the library's adaptive encoder gives the oracle's words, final states and
split entries bit for bit, and rejects malformed models. GPU: the adaptive
decode kernels reproduce the input and the oracle's split decode, alone, in
batches mixed with static streams, at every combine count and CTA size.
"""
import numpy as np
import pytest

import oracle
import workloads


def _case(N, seed, n_bits=16, sym_bytes=2, n_tables=64, alphabet=256):
    a = workloads.AdaptiveStream("t", N, n_bits=n_bits, sym_bytes=sym_bytes, n_tables=n_tables,
                                 alphabet=alphabet, seed=seed)
    tables = a.tables()
    s, tid = a.draw()
    return a, tables, s, tid


def _same(R, s, tid, tables, n, M):
    p = R.encode_adaptive(s, n, tables, tid, M)
    o = oracle.encode_adaptive_with_splits(s, tid, tables, n, M)
    e = p.export()
    assert np.array_equal(e["freq"].reshape(tables.shape), tables)
    assert np.array_equal(e["words"], o.words)
    assert np.array_equal(e["final"], o.final)
    assert np.array_equal(e["entry_word"].astype(np.int64), o.q)
    assert np.array_equal(e["entry_index"].astype(np.int64), o.idx[:-1])
    assert np.array_equal(e["entry_state"].astype(np.uint32), o.y[:-1])
    return p, o


CASES = [
    dict(n_bits=16, sym_bytes=2, n_tables=64, alphabet=256),
    dict(n_bits=12, sym_bytes=1, n_tables=16, alphabet=256),
    dict(n_bits=11, sym_bytes=2, n_tables=3, alphabet=1000),
    dict(n_bits=14, sym_bytes=2, n_tables=8, alphabet=4096),
    dict(n_bits=8, sym_bytes=1, n_tables=256, alphabet=12),
]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: f"n{c['n_bits']}_A{c['alphabet']}_T{c['n_tables']}")
@pytest.mark.parametrize("M", [1, 7, 200])
def test_adaptive_encoder_matches_oracle(recoil_lib, cfg, M):
    a, tables, s, tid = _case(100_003, 5, **cfg)
    p, _ = _same(recoil_lib, s, tid, tables, cfg["n_bits"], M)
    info = p.info
    assert info["n_tables"] == cfg["n_tables"] and info["alphabet"] == cfg["alphabet"]


@pytest.mark.parametrize("N", [0, 1, 31, 32, 33, 65, 1023])
def test_adaptive_edge_lengths(recoil_lib, N):
    a, tables, s, tid = _case(max(N, 1), N + 100)
    s, tid = s[:N], tid[:N]
    if N == 0:
        p = recoil_lib.encode_adaptive(s, 16, tables, tid, 4)
        assert p.info["n_words"] == 0 and p.info["n_entries"] == 1
        return
    _same(recoil_lib, s, tid, tables, 16, 4)


def test_combine_keeps_the_model(recoil_lib):
    R = recoil_lib
    a, tables, s, tid = _case(50_000, 9)
    p = R.encode_adaptive(s, 16, tables, tid, 40)
    c = R.combine_splits(p, 5)
    assert c.info["n_tables"] == 64 and c.info["n_entries"] == 5
    assert np.array_equal(R.stream_freq(c), tables)
    with pytest.raises(R.RecoilError):
        R.serialize(c)                            # the model travels with the codec


def test_adaptive_rejects_bad_models(recoil_lib):
    R = recoil_lib
    a, tables, s, tid = _case(2000, 10)
    bad = tables.copy()
    bad[3, 7] += 1                                # row 3 sums to 2^n + 1
    zero = tables.copy()
    zero[5, 0] += zero[5, 1] - 0
    zero[5, 1] = 0                                # a zero frequency (sum unchanged)
    big_tid = tid.copy()
    big_tid[17] = 64                              # table number out of range
    big_sym = s.copy()
    big_sym[3] = 256                              # symbol outside the alphabet
    for args in ((s, 16, bad, tid), (s, 16, zero, tid), (s, 16, tables, big_tid), (big_sym, 16, tables, tid),
                 (s, 7, tables, tid)):            # alphabet 256 > 2^7
        with pytest.raises(R.RecoilError) as e:
            R.encode_adaptive(*args, 8)
        assert e.value.code == R.EINVAL
    with pytest.raises(R.RecoilError):
        R.encode_adaptive(s, 16, tables[:1].repeat(257, axis=0), np.zeros_like(tid), 8)   # 257 tables


def test_adaptive_rejected_by_noalloc_and_small_ctas(recoil_lib):
    R = recoil_lib
    a, tables, s, tid = _case(4000, 11)
    p = R.encode_adaptive(s, 16, tables, tid, 4)
    for w in (1, 2):
        with pytest.raises(R.RecoilError):
            R.Plan([p], {"warps_per_cta": w})
    for w in (4, 32):                             # two lanes a thread: 8, 16 or 24 warps
        with pytest.raises(R.RecoilError):
            R.Plan([p], {"warps_per_cta": w, "flags": R.BATCH_TWO_LANES})
    assert R.Plan([p], {"warps_per_cta": 24, "flags": R.BATCH_TWO_LANES}).warps_per_cta == 24


def test_adaptive_plan_rejects_rows_beyond_shared_memory(recoil_lib):
    """256 PDFs over 1000 symbols need 513 KB of CDF rows: the plan refuses them with an
    error (no guide width makes them fit), while 64 such PDFs (128 KB) plan."""
    R = recoil_lib
    for T, ok in ((256, False), (64, True)):
        a, tables, s, tid = _case(20_000, 25, n_bits=16, sym_bytes=2, n_tables=T, alphabet=1000)
        p = R.encode_adaptive(s, 16, tables, tid, 8)
        if ok:
            assert R.Plan([p], {"warps_per_cta": 8}).workspace_size > 0
        else:
            with pytest.raises(R.RecoilError):
                R.Plan([p], {"warps_per_cta": 8})


# ------------------------------------------------------------------- GPU
def _gpu_decode(R, streams, opts=None):
    import torch
    plan = R.Plan(streams, opts)
    ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device="cuda")
    infos = [s.info for s in streams]
    outs = [torch.full((max(1, i["n_syms"] * i["sym_bytes"]),), 0xAB, dtype=torch.uint8, device="cuda")
            for i in infos]
    plan.upload(ws)
    plan.decode([o.data_ptr() for o in outs])
    assert plan.errors() == 0, R.recoil_last_error()
    res = []
    for o, i in zip(outs, infos):
        x = o.cpu().numpy()[: i["n_syms"] * i["sym_bytes"]]
        res.append(x.view(np.uint16) if i["sym_bytes"] == 2 else x)
    return res


@pytest.mark.gpu
@pytest.mark.parametrize("cfg", CASES, ids=lambda c: f"n{c['n_bits']}_A{c['alphabet']}_T{c['n_tables']}")
def test_gpu_adaptive_matches_oracle(recoil_lib, cfg):
    R = recoil_lib
    a, tables, s, tid = _case(400_009, 21, **cfg)
    p = R.encode_adaptive(s, cfg["n_bits"], tables, tid, 256)
    o = oracle.encode_adaptive_with_splits(s, tid, tables, cfg["n_bits"], 256)
    for Mp in (256, 37, 1):
        (out,) = _gpu_decode(R, [R.combine_splits(p, Mp)])
        assert np.array_equal(out, s), Mp
        assert np.array_equal(out, oracle.decode_splits(oracle.combined(o, Mp)).astype(out.dtype)), Mp


@pytest.mark.gpu
@pytest.mark.parametrize("cfg", [c for c in CASES if c["alphabet"] <= 256],
                         ids=lambda c: f"n{c['n_bits']}_A{c['alphabet']}_T{c['n_tables']}")
@pytest.mark.parametrize("warps", [8, 32])
def test_gpu_adaptive_paired_and_byte_layouts(recoil_lib, cfg, warps):
    """Alphabets up to 256 have two staged layouts: the paired one (a block per PDF: u32
    F(s) | H(s+1) << 16 per symbol, then a byte per boundary of 2^10 guide buckets) where it
    keeps as many splits resident, and the one-byte guide layout (RECOIL_BATCH_NO_PAIRS forces it). Both decode to the input
    and to the oracle's split decode; the paired image is the larger one when it is staged."""
    R = recoil_lib
    a, tables, s, tid = _case(300_007, 26, **cfg)
    p = R.encode_adaptive(s, cfg["n_bits"], tables, tid, 512)
    o = oracle.encode_adaptive_with_splits(s, tid, tables, cfg["n_bits"], 512)
    pair = R.KERNEL_ADAPTIVE8_PAIR if cfg["sym_bytes"] == 1 else R.KERNEL_ADAPTIVE16_PAIR
    byte = R.KERNEL_ADAPTIVE8 if cfg["sym_bytes"] == 1 else R.KERNEL_ADAPTIVE16
    seen = set()
    for flags in (0, R.BATCH_NO_PAIRS, R.BATCH_NO_PAIRS | R.BATCH_GRAPH, R.BATCH_GRAPH):
        for Mp in (512, 41):
            c = R.combine_splits(p, Mp)
            kernels = R.Plan([c], {"warps_per_cta": warps, "flags": flags}).kernels
            assert kernels in (pair, byte)
            assert kernels == byte or not flags & R.BATCH_NO_PAIRS
            seen.add(kernels)
            (out,) = _gpu_decode(R, [c], {"warps_per_cta": warps, "flags": flags})
            assert np.array_equal(out, s), (flags, Mp)
            assert np.array_equal(out, oracle.decode_splits(oracle.combined(o, Mp)).astype(out.dtype)), (flags, Mp)
    assert seen == {pair, byte}


def test_adaptive_paired_layout_staged_where_it_fits(recoil_lib):
    """Host side of the layout choice: 64 PDFs over 256 symbols at n = 16 take 131 KB paired,
    which fits beside the rings of one 32-warp CTA (as the 2^10-bucket byte layout does), so
    the paired image is staged; RECOIL_BATCH_NO_PAIRS stages the byte layout instead."""
    R = recoil_lib
    a, tables, s, tid = _case(20_000, 27)
    p = R.encode_adaptive(s, 16, tables, tid, 64)
    assert R.Plan([p], {"warps_per_cta": 32}).kernels == R.KERNEL_ADAPTIVE16_PAIR
    assert R.Plan([p], {"warps_per_cta": 32, "flags": R.BATCH_NO_PAIRS}).kernels == R.KERNEL_ADAPTIVE16
    # 256 PDFs: 264 KB paired, more than the shared memory; the byte layout (one-bucket guide) stays
    a, tables, s, tid = _case(20_000, 28, n_tables=256)
    p = R.encode_adaptive(s, 16, tables, tid, 64)
    assert R.Plan([p], {"warps_per_cta": 8}).kernels == R.KERNEL_ADAPTIVE16
    # wide alphabets have no paired layout
    a, tables, s, tid = _case(20_000, 29, n_tables=4, alphabet=1000)
    p = R.encode_adaptive(s, 16, tables, tid, 64)
    assert R.Plan([p], {"warps_per_cta": 32}).kernels == R.KERNEL_ADAPTIVE16_WIDE


@pytest.mark.gpu
@pytest.mark.parametrize("warps", [8, 32])
def test_gpu_adaptive_long_and_short_synchronisation_phases(recoil_lib, warps):
    """The groups a split decodes outside its steady loop read table numbers from blocks staged
    beforehand (three blocks of 8 groups from the split's top group, and from where the steady
    loop stops), else from global memory. A near-deterministic PDF (one symbol holds all but 255
    slots: a coder reads a word every few hundred symbols) in long runs gives synchronisation
    phases far longer than 24 groups; 3000 splits over 200 K symbols give splits of a few groups.
    Both decode to the input and to the oracle's split decode, paired and byte layouts."""
    R = recoil_lib
    g = np.random.default_rng(61)
    A, n, N = 256, 16, 200_003
    tables = np.ones((3, A), dtype=np.uint32)
    tables[0, 128] = (1 << n) - (A - 1)
    tables[1, :] = (1 << n) // A
    tables[2] = workloads.AdaptiveStream("t", 1, n_tables=3).tables()[1]
    runs = g.integers(1, 4000, size=400)
    tid = np.repeat(g.integers(0, 3, size=len(runs)), runs)[:N].astype(np.uint8)
    tid = np.concatenate([tid, np.zeros(N - len(tid), np.uint8)])
    cdf = np.cumsum(tables, axis=1) / float(1 << n)
    s = np.array([np.searchsorted(cdf[t], u, side="right") for t, u in zip(tid, g.random(N))], dtype=np.uint16)
    p = R.encode_adaptive(s, n, tables, tid, 3000)
    o = oracle.encode_adaptive_with_splits(s, tid, tables, n, 3000)
    idx = p.export()["entry_index"].astype(np.int64) // 32
    assert (idx.max(1) - idx.min(1)).max() > 24            # phases beyond the three staged blocks
    assert np.diff(np.sort(idx.max(1))).min() < 24          # splits shorter than the staged blocks
    for flags in (R.BATCH_GRAPH, R.BATCH_NO_PAIRS):
        for Mp in (3000, 300, 37):
            c = R.combine_splits(p, Mp)
            (out,) = _gpu_decode(R, [c], {"warps_per_cta": warps, "flags": flags})
            assert np.array_equal(out, s), (flags, Mp)
            assert np.array_equal(out, oracle.decode_splits(oracle.combined(o, Mp)).astype(out.dtype)), (flags, Mp)


@pytest.mark.gpu
@pytest.mark.parametrize("warps", [4, 8, 16, 32])
def test_gpu_adaptive_cta_sizes_and_graph(recoil_lib, warps):
    R = recoil_lib
    a, tables, s, tid = _case(1_000_003, 22)
    p = R.encode_adaptive(s, 16, tables, tid, 1024)
    for opts in ({"warps_per_cta": warps}, {"warps_per_cta": warps, "flags": R.BATCH_GRAPH},
                 {"warps_per_cta": warps, "flags": R.BATCH_PER_STREAM}, {"warps_per_cta": warps,
                                                                         "split_symbols": 20000}):
        (out,) = _gpu_decode(R, [p], opts)
        assert np.array_equal(out, s), opts


@pytest.mark.gpu
@pytest.mark.parametrize("cfg", CASES, ids=lambda c: f"n{c['n_bits']}_A{c['alphabet']}_T{c['n_tables']}")
@pytest.mark.parametrize("warps", [8, 24])
def test_gpu_adaptive_two_lanes_per_thread(recoil_lib, cfg, warps):
    """Two coder lanes a thread for adaptive streams (8, 16 or 24 warps per CTA): every
    layout the plan stages, at even and odd split counts, against the oracle."""
    R = recoil_lib
    a, tables, s, tid = _case(300_007, 31, **cfg)
    p = R.encode_adaptive(s, cfg["n_bits"], tables, tid, 300)
    o = oracle.encode_adaptive_with_splits(s, tid, tables, cfg["n_bits"], 300)
    for flags in (R.BATCH_TWO_LANES, R.BATCH_TWO_LANES | R.BATCH_NO_PAIRS | R.BATCH_GRAPH):
        for Mp in (300, 51):
            (out,) = _gpu_decode(R, [R.combine_splits(p, Mp)], {"warps_per_cta": warps, "flags": flags})
            assert np.array_equal(out, s), (flags, Mp)
            assert np.array_equal(out, oracle.decode_splits(oracle.combined(o, Mp)).astype(out.dtype)), (flags, Mp)


@pytest.mark.gpu
@pytest.mark.parametrize("warps", [8, 32])
def test_gpu_adaptive_tables_too_large_for_a_guide(recoil_lib, warps):
    """256 PDFs over 256 symbols at n = 16: the CDF rows take 132 KB, so no 2^9-bucket guide
    fits beside them (another 132 KB); the plan stages the one-bucket guide and the decoder
    searches whole rows."""
    R = recoil_lib
    a, tables, s, tid = _case(300_007, 23, n_bits=16, sym_bytes=2, n_tables=256, alphabet=256)
    p = R.encode_adaptive(s, 16, tables, tid, 512)
    (out,) = _gpu_decode(R, [p], {"warps_per_cta": warps})
    assert np.array_equal(out, s)


@pytest.mark.gpu
def test_gpu_adaptive_wide_alphabet_guides(recoil_lib):
    """4096-symbol alphabets take two-byte guide entries. 20 PDFs: 164 KB of CDF rows, with
    a 2^9-bucket guide 184 KB, with 2^10 buckets 204 KB; 4-warp CTAs stage the finer guide,
    16-warp CTAs (32 KB of rings) the coarser one. Each against the oracle's split decode."""
    R = recoil_lib
    a, tables, s, tid = _case(2_000_003, 24, n_bits=16, sym_bytes=2, n_tables=20, alphabet=4096)
    p = R.encode_adaptive(s, 16, tables, tid, 4096)
    o = oracle.encode_adaptive_with_splits(s, tid, tables, 16, 4096)
    for Mp, w in ((64, 4), (4096, 16), (4096, 8)):
        (out,) = _gpu_decode(R, [R.combine_splits(p, Mp)], {"warps_per_cta": w})
        assert np.array_equal(out, s), (Mp, w)
        assert np.array_equal(out, oracle.decode_splits(oracle.combined(o, Mp)).astype(np.uint16)), (Mp, w)


@pytest.mark.gpu
def test_gpu_adaptive_mixed_batch(recoil_lib):
    """Adaptive streams of both symbol sizes next to static streams of every kind, one plan."""
    R = recoil_lib
    streams, want = [], []
    for k, cfg in enumerate(CASES):
        a, tables, s, tid = _case(50_000 + 7919 * k, 30 + k, **cfg)
        streams.append(R.encode_adaptive(s, cfg["n_bits"], tables, tid, 20))
        want.append(s)
    for k, st in enumerate([workloads.Stream("z", 70_001, 1, 12, "zipf", {"s": 1.2}, seed=40),
                            workloads.Stream("g", 30_011, 2, 15, "gauss16",
                                             {"mean": 2048.0, "sigma": 200.0, "k": 4096}, seed=41),
                            workloads.Stream("e", 20_000, 1, 16, "expbytes", {"lam": 100.0}, seed=42)]):
        s = st.symbols()
        streams.append(R.encode_with_splits(s, st.n_bits, 9))
        want.append(s)
    order = np.random.default_rng(3).permutation(len(streams))
    outs = _gpu_decode(R, [streams[i] for i in order], {"warps_per_cta": 8})
    for out, i in zip(outs, order):
        assert np.array_equal(out, want[i]), i


@pytest.mark.gpu
@pytest.mark.parametrize("warps", [8, 32])
def test_gpu_adaptive_full_size_sampled(recoil_lib, warps):
    """The 256 MiB adaptive workload at 9472 splits: the whole output against the input,
    and a sample of split threads against the oracle's. 8-warp CTAs stage the 2^9-bucket
    guide (the finer one would halve the resident CTAs), 32-warp CTAs (the launch shape
    the benchmark picks) the 2^10-bucket one."""
    R = recoil_lib
    a = workloads.adaptive_256mib()
    tables = a.tables()
    s, tid = a.draw()
    p = R.encode_adaptive(s, a.n_bits, tables, tid, 65536)
    c = R.combine_splits(p, 9472)
    (out,) = _gpu_decode(R, [c], {"warps_per_cta": warps})
    assert np.array_equal(out, s)
    # sampled threads of the oracle on the same entries
    e = c.export()
    K = c.info["n_entries"]
    idx = np.vstack([e["entry_index"].astype(np.int64), np.zeros((1, 32), dtype=np.int64)])
    y = np.vstack([e["entry_state"].astype(np.uint32), e["final"][None, :]])
    st = oracle.OracleStream(len(s), a.n_bits, 32, 16, 16, tables, e["words"], e["final"], None, None,
                             e["entry_word"].astype(np.int64), idx, y, tid)
    for k in np.random.default_rng(5).choice(K, size=6, replace=False):
        lo, hi = oracle.owned_range(st, int(k))
        ref = oracle.decode_thread(st, int(k))
        assert np.array_equal(out[lo:hi + 1], ref[lo:hi + 1].astype(np.uint16)), k


def _adaptive_pool(R, count, seed):
    g = np.random.default_rng(seed)
    syms, streams = [], []
    for k in range(count):
        N = int(g.integers(1, 300_000))
        if k % 3 == 2:
            st = workloads.Stream("l", N, 1, 12, "laplace", {"mean": 128.0, "scale": float(g.uniform(2, 64))},
                                  seed=seed + k)
            s = st.symbols()
            streams.append(R.encode_with_splits(s, st.n_bits, max(1, N // 4096)))
        else:
            cfg = CASES[k % len(CASES)]
            a, tables, s, tid = _case(N, seed + k, **cfg)
            streams.append(R.encode_adaptive(s, cfg["n_bits"], tables, tid, max(1, N // 4096)))
        syms.append(s)
    return syms, streams


@pytest.mark.gpu
def test_gpu_adaptive_in_serving_pipeline_and_autotune(recoil_lib, tmp_path):
    """Adaptive streams next to static ones through the serving runtime, the host-to-host
    pipeline and the autotuner: every output is the input."""
    import torch
    R = recoil_lib
    syms, pool = _adaptive_pool(R, 18, 60)
    cs = torch.cuda.current_stream()
    # serving: Poisson arrivals over the mixed pool
    n_req = 200
    picks = workloads.request_picks(len(pool), n_req, seed=61)
    arrive = workloads.poisson_arrivals(20_000.0, n_req, seed=61)
    outs = [torch.full((max(1, len(syms[p]) * syms[p].itemsize),), 0xAB, dtype=torch.uint8, device="cuda")
            for p in picks]
    budget = 64 << 20
    need = R.serve_arena_size(pool, budget, warps_per_cta=8)
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    res, stats = R.serve(pool, picks, arrive, arena, need, budget, outs=[o.data_ptr() for o in outs],
                         warps_per_cta=8, max_inflight=4, max_batch=16, timeout_s=60.0)
    assert stats["requests"] == n_req
    for r, p in enumerate(picks):
        s = syms[p]
        assert np.array_equal(outs[r].cpu().numpy()[: len(s) * s.itemsize].view(s.dtype), s), r
    # host to host
    for st in pool:
        R.stream_pin(st)
    pipe = R.Pipeline(pool, {"warps_per_cta": 8, "split_symbols": 32768}, groups=3)
    wsb, stb = pipe.sizes
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    stage = torch.empty(stb, dtype=torch.uint8, device="cuda")
    host = [torch.full((max(1, len(s) * s.itemsize),), 0xAB, dtype=torch.uint8, pin_memory=True) for s in syms]
    s2 = torch.cuda.Stream()
    pipe.run([h.data_ptr() for h in host], ws, wsb, stage, stb, s2)
    s2.synchronize()
    assert pipe.errors() == 0
    for s, h in zip(syms, host):
        assert np.array_equal(h.numpy()[: len(s) * s.itemsize].view(s.dtype), s)
    # autotuner
    need = R.autotune_workspace_size(pool)
    tws = torch.empty(need, dtype=torch.uint8, device="cuda")
    touts = [torch.zeros(max(1, len(s) * s.itemsize), dtype=torch.uint8, device="cuda") for s in syms]
    best, ms = R.autotune(pool, [o.data_ptr() for o in touts], tws, need, cs, steps=2,
                          cache_path=str(tmp_path / "tune.txt"))
    assert best["warps_per_cta"] in (4, 8, 16, 32) and ms > 0
    for s, o in zip(syms, touts):
        assert np.array_equal(o.cpu().numpy()[: len(s) * s.itemsize].view(s.dtype), s)


@pytest.mark.gpu
def test_gpu_autotune_chooses_the_table_layout(recoil_lib, tmp_path):
    """Adaptive models over up to 256 symbols give the autotuner both table layouts (paired and
    one-byte guide): its cache line records the layout it chose, a cached byte-guide line comes
    back with RECOIL_BATCH_NO_PAIRS (the plan then stages the byte layout) and a paired one
    without, and every choice decodes to the input."""
    import torch
    R = recoil_lib
    a, tables, s, tid = _case(300_007, 31)
    p = R.combine_splits(R.encode_adaptive(s, 16, tables, tid, 512), 296)
    need = R.autotune_workspace_size([p])
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.zeros(len(s) * 2, dtype=torch.uint8, device="cuda")
    cs = torch.cuda.current_stream()
    cache = str(tmp_path / "tune.txt")
    best, ms = R.autotune([p], [out.data_ptr()], ws, need, cs, steps=2, cache_path=cache, keep_splits=True)
    assert ms > 0 and np.array_equal(out.cpu().numpy().view(np.uint16), s)
    key, w, sp, lanes, layout, t = open(cache).read().split("\n")[0].split()
    assert layout in ("0", "1") and (layout == "1") == bool(best["flags"] & R.BATCH_NO_PAIRS)
    chosen = {}
    for lay, kernel in (("1", R.KERNEL_ADAPTIVE16), ("0", R.KERNEL_ADAPTIVE16_PAIR)):
        with open(cache, "a") as f:
            f.write(f"{key} 32 0 1 {lay} {t}\n")
        got, _ = R.autotune([p], [out.data_ptr()], ws, need, cs, cache_path=cache, keep_splits=True)
        assert got["warps_per_cta"] == 32 and bool(got["flags"] & R.BATCH_NO_PAIRS) == (lay == "1")
        assert R.Plan([p], got).kernels == kernel
        chosen[lay] = got
    for opts in (best, *chosen.values()):
        (o,) = _gpu_decode(R, [p], opts)
        assert np.array_equal(o, s), opts


@pytest.mark.gpu
def test_gpu_adaptive_corrupt_words_flagged(recoil_lib):
    """Words flipped in the uploaded device image of an adaptive stream are reported by
    the decoders' state cross-check (no fault, no hang), and the context stays usable."""
    import torch
    R = recoil_lib
    a, tables, s, tid = _case(200_000, 70)
    p = R.encode_adaptive(s, 16, tables, tid, 8)
    nw = p.info["n_words"]
    out = torch.zeros(2 * len(s), dtype=torch.uint8, device="cuda")
    plan = R.Plan([p], {"warps_per_cta": 8})
    ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    torch.cuda.synchronize()
    words = ws[: 2 * nw].view(torch.int16)                # the first stream's words start the workspace
    words[nw // 3: nw // 3 + 40] ^= 0x5A5A
    plan.decode([out.data_ptr()])
    assert plan.errors() != 0
    plan.upload(ws)                                       # a clean image: exact again
    plan.decode([out.data_ptr()])
    assert plan.errors() == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint16), s)


@pytest.mark.gpu
@pytest.mark.parametrize("N", [1, 31, 32, 33, 1023, 4097])
def test_gpu_adaptive_edge_lengths(recoil_lib, N):
    """Short adaptive streams (idle coders in the top group, a single group), alone and as a
    batch of one-table streams (warp-queue launch)."""
    R = recoil_lib
    a, tables, s, tid = _case(N, 300 + N)
    p = R.encode_adaptive(s, 16, tables, tid, 4)
    (out,) = _gpu_decode(R, [p], {"warps_per_cta": 4})
    assert np.array_equal(out, s)
    o = oracle.encode_adaptive_with_splits(s, tid, tables, 16, 4)
    assert np.array_equal(out, oracle.decode_splits(o).astype(np.uint16))
    many = [R.encode_adaptive(s[: max(1, N - k)], 16, tables, tid[: max(1, N - k)], 4) for k in range(6)]
    outs = _gpu_decode(R, many, {"warps_per_cta": 8})
    for k, o2 in enumerate(outs):
        assert np.array_equal(o2, s[: max(1, N - k)]), k
