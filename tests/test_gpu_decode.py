"""GPU parity: the CUDA split decoders against the oracle, bit for bit.

All decoding goes through the C-ABI (plan, upload, decode). Expected values
are the input symbols (the codec is lossless) and the oracle's own split
decode of the same stream; streams made by the oracle's encoder are imported
so that the kernels are also checked on metadata the library did not produce.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_decode(R, streams, opts=None, cuda_stream=None, check=True, repeat=1):
    plan = R.Plan(streams, opts)
    ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device="cuda")
    infos = [s.info for s in streams]
    outs = [torch.full((max(1, i["n_syms"] * i["sym_bytes"]),), 0xAB, dtype=torch.uint8, device="cuda")
            for i in infos]
    cs = cuda_stream or torch.cuda.current_stream()
    plan.upload(ws, stream=cs)
    for _ in range(repeat):
        plan.decode([o.data_ptr() for o in outs], cs)
    flags = plan.errors(cs)
    if check:
        assert flags == 0, R.recoil_last_error()
    res = []
    for o, i in zip(outs, infos):
        a = o.cpu().numpy()[: i["n_syms"] * i["sym_bytes"]]
        res.append(a.view(np.uint16) if i["sym_bytes"] == 2 else a)
    return (res, flags, plan) if not check else res


def _import(R, o: oracle.OracleStream, sym_bytes=1):
    return R.stream_import(o.n, sym_bytes, o.N, o.f, o.words, o.final, o.q, o.idx[:-1], o.y[:-1])


def test_config1_decodes_at_64_16_1_splits(recoil_lib):
    R = recoil_lib
    st = workloads.laplace_1mib()
    s = st.symbols()
    p = R.encode_with_splits(s, st.n_bits, 64)
    o = oracle.encode_with_splits(s, st.n_bits, 64)
    assert p.info["n_entries"] == 64
    for Mp in (64, 16, 1):
        c = R.combine_splits(p, Mp)
        (out,) = gpu_decode(R, [c])
        assert np.array_equal(out, s)
        assert np.array_equal(out, oracle.decode_splits(oracle.combined(o, Mp)).astype(np.uint8))


@pytest.mark.parametrize("dist,params,n,sb", [
    ("zipf", {"s": 1.2}, 12, 1),
    ("skewed", {"p0": 0.95}, 12, 1),
    ("gauss16", {"mean": 2048.0, "sigma": 200.0, "k": 4096}, 15, 2),
])
def test_printed_rule_streams_decode_on_gpu(recoil_lib, dist, params, n, sb):
    """Splits placed with the printed T = ceil(N/M) of Def. 4.1 (RECOIL_SPLIT_EQ7), the long
    final split included: the library's stream and the oracle's (imported) decode to the
    input and to the oracle's split decode at several combined counts."""
    R = recoil_lib
    s = workloads.Stream("t", 300_007, sb, n, dist, params, seed=37).symbols()
    p = R.encode_with_splits(s, n, 256, rule="eq7")
    o = oracle.encode_with_splits(s, n, 256, rule="eq7")
    assert np.array_equal(p.export()["entry_word"].astype(np.int64), o.q)
    imp = _import(R, o, sb)
    for Mp in (256, 37, 4):
        want = oracle.decode_splits(oracle.combined(o, Mp))
        for st in (R.combine_splits(p, Mp), R.combine_splits(imp, Mp)):
            (out,) = gpu_decode(R, [st])
            assert np.array_equal(out, s)
            assert np.array_equal(out, want.astype(out.dtype))


DISTS = [
    ("laplace", {"mean": 128.0, "scale": 8.0}, 11, 1),
    ("zipf", {"s": 1.2}, 12, 1),
    ("skewed", {"p0": 0.95}, 12, 1),
    ("uniform", {}, 12, 1),
    ("gauss16", {"mean": 2048.0, "sigma": 200.0, "k": 4096}, 15, 2),
    ("expbytes", {"lam": 200.0}, 16, 1),
    ("laplace", {"mean": 128.0, "scale": 30.0}, 13, 1),
]


@pytest.mark.parametrize("dist,params,n,sb", DISTS)
def test_oracle_made_streams_decode_on_gpu(recoil_lib, dist, params, n, sb):
    R = recoil_lib
    s = workloads.Stream("t", 200_003, sb, n, dist, params, seed=31).symbols()
    o = oracle.encode_with_splits(s, n, 97)
    want = oracle.decode_splits(o)
    assert np.array_equal(want, s)
    (out,) = gpu_decode(R, [_import(R, o, sb)])
    assert np.array_equal(out.astype(np.uint32), want)


def test_random_subsets_of_split_entries(recoil_lib):
    R = recoil_lib
    s = workloads.Stream("t", 120_000, 1, 11, "laplace", {"mean": 128.0, "scale": 8.0}, seed=32).symbols()
    o = oracle.encode_with_splits(s, 11, 300)
    g = np.random.default_rng(5)
    streams = []
    for t in range(24):
        keep = np.sort(g.choice(o.K - 1, size=int(g.integers(0, o.K - 1)), replace=False))
        sub = oracle.OracleStream(o.N, o.n, o.W, o.lgL, o.b, o.f, o.words, o.final, o.ev_sym, o.ev_y,
                                  o.q[keep], np.vstack([o.idx[keep], o.idx[-1:]]), np.vstack([o.y[keep], o.y[-1:]]))
        assert np.array_equal(oracle.decode_splits(sub), s)
        streams.append(_import(R, sub))
    outs = gpu_decode(R, streams)
    for out in outs:
        assert np.array_equal(out, s)


@pytest.mark.parametrize("N", [0, 1, 5, 31, 32, 33, 64, 95, 1000, 4097, 65_539])
@pytest.mark.parametrize("M", [1, 2, 7, 64])
def test_edge_lengths(recoil_lib, N, M):
    R = recoil_lib
    s = workloads.Stream("t", max(N, 1), 1, 9, "laplace", {"mean": 128.0, "scale": 4.0}, seed=N + 3).symbols()[:N]
    p = R.encode_with_splits(s, 9, M)
    (out,) = gpu_decode(R, [p])
    assert np.array_equal(out, s)


@pytest.mark.parametrize("n,sb", [(1, 1), (12, 1), (16, 1), (15, 2), (16, 2)])
def test_single_symbol_streams(recoil_lib, n, sb):
    R = recoil_lib
    s = np.full(10_001, 3, dtype=np.uint8 if sb == 1 else np.uint16)
    (out,) = gpu_decode(R, [R.encode_with_splits(s, n, 8)])
    assert np.array_equal(out, s)


def _batch_streams(R, count=60, seed=40):
    g = np.random.default_rng(seed)
    syms, streams = [], []
    for k in range(count):
        N = int(g.integers(0, 300_000)) if k % 7 else int(g.integers(0, 100))
        kind = k % 5
        if kind == 4:
            st = workloads.Stream("g", max(N, 1), 2, 15, "gauss16", {"mean": 2048.0, "sigma": 150.0, "k": 4096}, seed=k)
        elif kind == 3:
            st = workloads.Stream("e", max(N, 1), 1, 16, "expbytes", {"lam": 100.0}, seed=k)
        else:
            st = workloads.Stream("l", max(N, 1), 1, 12, "laplace", {"mean": 128.0, "scale": float(g.uniform(2, 64))}, seed=k)
        s = st.symbols()[:N]
        syms.append(s)
        streams.append(R.encode_with_splits(s, st.n_bits, max(1, N // 4096)))
    return syms, streams


@pytest.mark.parametrize("opts", [
    None,
    {"warps_per_cta": 4},
    {"warps_per_cta": 8, "ctas_per_sm": 2},
    {"warps_per_cta": 32},
    {"warps_per_cta": 1},
    {"split_symbols": 16384},
    {"warps_per_cta": 4, "flags": 1},            # one launch per stream
    {"flags": 2},                                # stream-major order
])
def test_batch_of_uneven_streams(recoil_lib, opts):
    R = recoil_lib
    syms, streams = _batch_streams(R)
    outs = gpu_decode(R, streams, opts)
    for s, out in zip(syms, outs):
        assert np.array_equal(out, s)


@pytest.mark.parametrize("opts", [
    {"warps_per_cta": 4, "flags": 16},
    {"warps_per_cta": 8, "flags": 16 | 4},       # two lanes a thread, graph replay
    {"warps_per_cta": 16, "flags": 16, "split_symbols": 16384},
    {"warps_per_cta": 8, "flags": 16 | 1},       # two lanes, one launch per stream
    {"flags": 16},                               # two lanes, automatic CTA size
])
def test_batch_two_lanes_per_thread(recoil_lib, opts):
    """Two coder lanes a thread (RECOIL_BATCH_TWO_LANES): each warp decodes two splits in
    lockstep, one coder of each per thread; uneven batches of every static kind, with odd
    item counts (a warp left with one split) and empty streams, decode exactly."""
    R = recoil_lib
    syms, streams = _batch_streams(R)
    outs = gpu_decode(R, streams, opts)
    for s, out in zip(syms, outs):
        assert np.array_equal(out, s)


@pytest.mark.parametrize("dist,params,n,sb", DISTS[:5])
@pytest.mark.parametrize("warps", [4, 16])
def test_two_lanes_single_stream_against_oracle(recoil_lib, dist, params, n, sb, warps):
    """One stream (the warp-queue launch: warps pop two splits at a time) at several combined
    counts, odd ones included, against the input and the oracle's split decode."""
    R = recoil_lib
    s = workloads.Stream("t", 200_003, sb, n, dist, params, seed=33).symbols()
    p = R.encode_with_splits(s, n, 300)
    o = oracle.encode_with_splits(s, n, 300)
    for Mp in (300, 77, 2, 1):
        c = R.combine_splits(p, Mp)
        plan = R.Plan([c], {"warps_per_cta": warps, "flags": R.BATCH_TWO_LANES})
        assert plan.warps_per_cta == warps
        (out,) = gpu_decode(R, [c], {"warps_per_cta": warps, "flags": R.BATCH_TWO_LANES})
        assert np.array_equal(out, s), Mp
        assert np.array_equal(out, oracle.decode_splits(oracle.combined(o, Mp)).astype(out.dtype)), Mp


def test_two_lanes_rejects_unbuilt_shapes(recoil_lib):
    R = recoil_lib
    s = workloads.Stream("t", 10_000, 1, 12, "zipf", {"s": 1.2}, seed=3).symbols()
    p = R.encode_with_splits(s, 12, 8)
    for w in (1, 2, 32, 24):
        with pytest.raises(R.RecoilError):
            R.Plan([p], {"warps_per_cta": w, "flags": R.BATCH_TWO_LANES})


def test_batch_graph_replay_and_new_outputs(recoil_lib):
    R = recoil_lib
    syms, streams = _batch_streams(R, count=30, seed=41)
    plan = R.Plan(streams, {"flags": R.BATCH_GRAPH})
    ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device="cuda")
    cs = torch.cuda.Stream()
    with torch.cuda.stream(cs):
        plan.upload(ws, stream=cs)
        for rep in range(3):
            outs = [torch.zeros(max(1, len(s) * s.itemsize), dtype=torch.uint8, device="cuda") for s in syms]
            for _ in range(2):
                plan.decode([o.data_ptr() for o in outs], cs)
            assert plan.errors(cs) == 0
            for s, o in zip(syms, outs):
                a = o.cpu().numpy()[: len(s) * s.itemsize]
                assert np.array_equal(a.view(s.dtype), s)
    assert plan.launches >= 1


def test_one_shot_decode_and_batch_entry_points(recoil_lib):
    R = recoil_lib
    syms, streams = _batch_streams(R, count=12, seed=42)
    need = R.workspace_size(streams)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    outs = [torch.zeros(max(1, len(s) * s.itemsize), dtype=torch.uint8, device="cuda") for s in syms]
    cs = torch.cuda.current_stream()
    R.decode_batch(streams, [o.data_ptr() for o in outs], ws, need, cs)
    torch.cuda.synchronize()
    for s, o in zip(syms, outs):
        assert np.array_equal(o.cpu().numpy()[: len(s) * s.itemsize].view(s.dtype), s)
    one = R.workspace_size([streams[1]])
    out1 = torch.zeros(max(1, len(syms[1]) * syms[1].itemsize), dtype=torch.uint8, device="cuda")
    R.decode(streams[1], out1, ws, one, cs)
    torch.cuda.synchronize()
    assert np.array_equal(out1.cpu().numpy()[: len(syms[1]) * syms[1].itemsize].view(syms[1].dtype), syms[1])
    with pytest.raises(R.RecoilError):
        R.decode(streams[1], out1, ws, 16, cs)                # workspace too small


def test_corrupt_words_raise_an_error_flag_not_a_fault(recoil_lib):
    """Corruption made on the host; the kernel's loops are bounded, so it reports, never hangs."""
    R = recoil_lib
    s = workloads.Stream("t", 50_000, 1, 11, "laplace", {"mean": 128.0, "scale": 8.0}, seed=43).symbols()
    o = oracle.encode_with_splits(s, 11, 4)
    bad = o.words.copy()
    bad[len(bad) // 3: len(bad) // 3 + 50] ^= 0x5A5A
    st = R.stream_import(11, 1, o.N, o.f, bad, o.final, o.q, o.idx[:-1], o.y[:-1])
    outs, flags, plan = gpu_decode(R, [st], check=False)
    assert flags != 0
    short = R.stream_import(11, 1, o.N, o.f, o.words[: len(o.words) // 2], o.final, [], np.zeros((0, 32)),
                            np.zeros((0, 32)))
    outs, flags, plan = gpu_decode(R, [short], check=False)
    assert flags != 0
    # the context is still usable
    (out,) = gpu_decode(R, [_import(R, o)])
    assert np.array_equal(out, s)


@pytest.mark.parametrize("target", [148, 592, 2368, 9472])
def test_zipf_1gib_full_size(recoil_lib, zipf_1gib, target):
    """1 GiB Zipf(1.2), n = 12, encoded at 65536 splits, combined as the benchmark sweeps."""
    R = recoil_lib
    s_dev, stream, s = zipf_1gib
    c = R.combine_splits(stream, target)
    plan = R.Plan([c])
    ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device="cuda")
    out = torch.empty(len(s), dtype=torch.uint8, device="cuda")
    cs = torch.cuda.current_stream()
    plan.upload(ws, stream=cs)
    plan.decode([out.data_ptr()], cs)
    assert plan.errors(cs) == 0
    assert torch.equal(out, s_dev)
    # sampled threads against the oracle, one by one
    e = c.export()
    info = c.info
    K = info["n_entries"]
    for k in (0, K // 2, K - 1):
        lo = 0 if k == 0 else int(e["entry_index"][k - 1].min())
        hi = len(s) - 1 if k == K - 1 else int(e["entry_index"][k].min()) - 1
        if hi - lo > 10_000_000:
            continue
        ost = oracle.OracleStream(len(s), 12, 32, 16, 16, e["freq"], e["words"], e["final"], None, None,
                                  e["entry_word"].astype(np.int64),
                                  np.vstack([e["entry_index"].astype(np.int64), np.zeros((1, 32), np.int64)]),
                                  np.vstack([e["entry_state"].astype(np.uint32), e["final"][None, :]]))
        want = oracle.decode_thread(ost, k)[lo:hi + 1]
        assert np.array_equal(out[lo:hi + 1].cpu().numpy(), want.astype(np.uint8))


@pytest.fixture(scope="module")
def zipf_1gib(recoil_lib):
    st = workloads.zipf_1gib()
    s = st.symbols()
    stream = recoil_lib.encode_with_splits(s, st.n_bits, 65536)
    assert stream.info["n_entries"] == 65536
    return torch.from_numpy(s).cuda(), stream, s


def test_autotune_chooses_a_working_configuration(recoil_lib, tmp_path):
    R = recoil_lib
    syms, streams = _batch_streams(R, count=40, seed=44)
    need = R.autotune_workspace_size(streams)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    outs = [torch.zeros(max(1, len(s) * s.itemsize), dtype=torch.uint8, device="cuda") for s in syms]
    ptrs = [o.data_ptr() for o in outs]
    cs = torch.cuda.current_stream()
    cache = str(tmp_path / "tune.txt")
    best, ms = R.autotune(streams, ptrs, ws, need, cs, steps=2, cache_path=cache)
    # 32-warp CTAs are candidates here: the batch holds 16-bit static models
    assert best["warps_per_cta"] in (4, 8, 16, 32) and best["split_symbols"] in (32768, 65536, 131072, 262144)
    assert ms > 0
    for s, o in zip(syms, outs):                               # the tuning decodes are exact too
        assert np.array_equal(o.cpu().numpy()[: len(s) * s.itemsize].view(s.dtype), s)
    again, ms2 = R.autotune(streams, ptrs, ws, need, cs, cache_path=cache)
    assert again == best and abs(ms2 - ms) < 1e-3               # served from the cache
    res = gpu_decode(R, streams, best)
    for s, out in zip(syms, res):
        assert np.array_equal(out, s)
    # CTA size only, on the streams' own split counts (cached under its own key)
    keep, ms3 = R.autotune(streams, ptrs, ws, need, cs, steps=2, cache_path=cache, keep_splits=True)
    assert keep["warps_per_cta"] in (4, 8, 16, 32) and keep["split_symbols"] == 0 and ms3 > 0
    for s, out in zip(syms, gpu_decode(R, streams, keep)):
        assert np.array_equal(out, s)
    # cache lines carry the lanes a thread and the table layout: key, warps, split symbols, lanes,
    # layout, ms (a line without the layout reads as layout 0); the last line of a key wins, so an
    # appended two-lane line is what the next lookup returns
    lines = open(cache).read().split("\n")
    key, w, sp, lanes, layout, t = lines[0].split()
    assert lanes in ("1", "2") and int(w) == best["warps_per_cta"] and int(sp) == best["split_symbols"]
    assert layout == "0"                                          # static streams have one layout
    with open(cache, "a") as f:
        f.write(f"{key} 8 65536 2 0 {t}\n")
    two, _ = R.autotune(streams, ptrs, ws, need, cs, cache_path=cache)
    assert two["warps_per_cta"] == 8 and two["split_symbols"] == 65536 and two["flags"] & R.BATCH_TWO_LANES
    for s, out in zip(syms, gpu_decode(R, streams, two)):
        assert np.array_equal(out, s)
    with open(cache, "a") as f:
        f.write(f"{key} 16 32768 1 {t}\n")
    old, _ = R.autotune(streams, ptrs, ws, need, cs, cache_path=cache)
    assert old["warps_per_cta"] == 16 and old["split_symbols"] == 32768 and old["flags"] == 0


def test_pipeline_decodes_host_to_host(recoil_lib):
    R = recoil_lib
    syms, streams = _batch_streams(R, count=50, seed=45)
    for st in streams:
        R.stream_pin(st)
    pipe = R.Pipeline(streams, {"warps_per_cta": 8, "split_symbols": 32768}, groups=5)
    wsb, stb = pipe.sizes
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    cs = torch.cuda.Stream()
    for rep in range(2):
        stage = torch.empty(stb + 256 * rep, dtype=torch.uint8, device="cuda")[256 * rep:]
        host = [torch.full((max(1, len(s) * s.itemsize),), 0xAB, dtype=torch.uint8, pin_memory=True) for s in syms]
        pipe.run([h.data_ptr() for h in host], ws, wsb, stage, stb, cs)
        pipe.run([h.data_ptr() for h in host], ws, wsb, stage, stb, cs)      # back to back
        cs.synchronize()
        assert pipe.errors() == 0
        for s, h in zip(syms, host):
            assert np.array_equal(h.numpy()[: len(s) * s.itemsize].view(s.dtype), s)


@pytest.mark.parametrize("make", [workloads.skewed_256mib, workloads.uniform_256mib, workloads.gauss16_256mib],
                         ids=["skewed", "uniform", "gauss16"])
def test_distribution_extremes_full_size(recoil_lib, make):
    """256 MiB each: P(0) = 0.95 (long synchronisation sections), uniform bytes, uint16 Gaussian at n = 15."""
    R = recoil_lib
    st = make()
    s = st.symbols()
    enc = R.encode_with_splits(s, st.n_bits, max(1, len(s) // 4096 // 4))
    info = enc.info
    if st.dist == "uniform":
        assert abs(info["n_words"] - len(s) // 2) <= 2 * 32       # 8 bits per symbol exactly
    ref = torch.from_numpy(s.view(np.uint8)).cuda()
    for target in (9472, 148 * 48):
        c = R.combine_splits(enc, target)
        plan = R.Plan([c], {"warps_per_cta": 16})
        ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device="cuda")
        out = torch.empty(len(s) * s.itemsize, dtype=torch.uint8, device="cuda")
        cs = torch.cuda.current_stream()
        plan.upload(ws, stream=cs)
        plan.decode([out.data_ptr()], cs)
        assert plan.errors(cs) == 0
        assert torch.equal(out, ref)


@pytest.mark.parametrize("warps", [1, 4, 16])
def test_partitions_sharing_one_model(recoil_lib, warps):
    """Conventional partitioning (Sec. 2.3): independent streams with one shared table.

    Work items then span several streams, one staged table serving all of them."""
    R = recoil_lib
    s = workloads.Stream("z", 3_000_000, 1, 12, "zipf", {"s": 1.2}, seed=72).symbols()
    f = oracle.quantize(np.bincount(s, minlength=256), 12)
    cuts = np.sort(np.random.default_rng(3).choice(len(s), size=150, replace=False))
    parts = np.split(s, cuts)
    streams = [R.encode_with_table(p, 12, f, 1 + len(p) // 40_000) for p in parts]
    outs = gpu_decode(R, streams, {"warps_per_cta": warps})
    assert np.array_equal(np.concatenate(outs), s)


@pytest.mark.parametrize("world", [1, 2, 3, 8, 100])
def test_shard_plans_tile_one_stream(recoil_lib, world):
    """recoil_plan_create_shard: each rank's run decodes into a buffer of its own range only;
    the ranks run one after another on this GPU and their ranges concatenate to the stream."""
    R = recoil_lib
    st = workloads.Stream("zipf", 2_000_003, 1, 12, "zipf", {"s": 1.2}, seed=81)
    s = st.symbols()
    p = R.combine_splits(R.encode_with_splits(s, st.n_bits, 512), 64)
    pieces, prev_hi = [], 0
    for r in range(world):
        plan, lo, hi = R.Plan.shard(p, world, r, {"warps_per_cta": 8})
        assert lo == prev_hi
        prev_hi = hi
        ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device="cuda")
        buf = torch.full((max(1, hi - lo) + 64,), 0xAB, dtype=torch.uint8, device="cuda")
        plan.upload(ws)
        plan.decode([buf.data_ptr()])
        assert plan.errors() == 0
        b = buf.cpu().numpy()
        assert np.all(b[hi - lo:] == 0xAB)                   # nothing written past the range
        pieces.append(b[:hi - lo])
    assert prev_hi == len(s)
    assert np.array_equal(np.concatenate(pieces), s)


def test_shard_plans_adaptive_stream(recoil_lib):
    R = recoil_lib
    a = workloads.AdaptiveStream("t", 1_000_003, seed=82)
    tables = a.tables()
    s, tid = a.draw()
    p = R.encode_adaptive(s, a.n_bits, tables, tid, 300)
    pieces = []
    for r in range(4):
        plan, lo, hi = R.Plan.shard(p, 4, r, {"warps_per_cta": 16})
        ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device="cuda")
        buf = torch.zeros(max(1, 2 * (hi - lo)), dtype=torch.uint8, device="cuda")
        plan.upload(ws)
        plan.decode([buf.data_ptr()])
        assert plan.errors() == 0
        pieces.append(buf.cpu().numpy()[: 2 * (hi - lo)].view(np.uint16))
    assert np.array_equal(np.concatenate(pieces), s)


@pytest.mark.parametrize("groups", [1, 3, 8])
def test_pipeline_cuts_a_large_stream_into_runs(recoil_lib, groups):
    """One large stream (and a small one beside it) host to host: the large one is cut into
    runs of splits that stage only their word windows, decode and copy out in turn."""
    R = recoil_lib
    big = workloads.Stream("z", 3_000_017, 1, 12, "zipf", {"s": 1.2}, seed=95).symbols()
    small = workloads.Stream("l", 20_011, 1, 11, "laplace", {"mean": 128.0, "scale": 5.0}, seed=96).symbols()
    a = workloads.AdaptiveStream("t", 1_000_003, seed=97)
    tables = a.tables()
    sa, tid = a.draw()
    streams = [R.encode_with_splits(big, 12, 512), R.encode_with_splits(small, 11, 4),
               R.encode_adaptive(sa, 16, tables, tid, 256)]
    want = [big, small, sa]
    pipe = R.Pipeline(streams, {"warps_per_cta": 8}, groups=groups)
    wsb, stb = pipe.sizes
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    cs = torch.cuda.Stream()
    for rep in range(2):                          # a second staging buffer rebinds the plans
        stage = torch.empty(stb + 256 * rep, dtype=torch.uint8, device="cuda")[256 * rep:]
        host = [torch.full((len(s) * s.itemsize,), 0xAB, dtype=torch.uint8, pin_memory=True) for s in want]
        for _ in range(3):                        # runs after the first reuse the bound descriptors
            pipe.run([h.data_ptr() for h in host], ws, wsb, stage, stb, cs)
        cs.synchronize()
        assert pipe.errors() == 0
        for s, h in zip(want, host):
            assert np.array_equal(h.numpy().view(s.dtype), s)


def test_batch_full_size_in_the_benchmark_launch_shape(recoil_lib):
    """The 4096-stream uneven batch at full size (3.47 GB of symbols), decoded as the benchmark
    times it: 8-warp CTAs, streams combined to 128 Ki-symbol splits, one persistent launch
    replayed from a CUDA graph. Every stream against its input on the device, and a sample of
    split threads against the oracle's split decoder on the same combined entries."""
    from concurrent.futures import ThreadPoolExecutor
    R = recoil_lib
    specs = workloads.batch_specs()
    syms = workloads.batch_symbols(specs)
    with ThreadPoolExecutor(32) as ex:
        streams = list(ex.map(lambda k: R.encode_with_splits(syms[k], 12, workloads.batch_split_count(len(syms[k]))),
                              range(len(specs))))
    opts = {"warps_per_cta": 8, "split_symbols": 131072, "flags": R.BATCH_GRAPH}
    plan = R.Plan(streams, opts)
    ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device="cuda")
    outs = [torch.empty(max(1, len(s)), dtype=torch.uint8, device="cuda") for s in syms]
    cs = torch.cuda.current_stream()
    plan.upload(ws, stream=cs)
    for _ in range(2):                                   # a replay writes the same bytes again
        plan.decode([o.data_ptr() for o in outs], cs)
    assert plan.errors(cs) == 0
    for s, o in zip(syms, outs):
        assert torch.equal(o[: len(s)], torch.from_numpy(s).cuda())
    # sampled threads: the plan combines each stream to ceil(N / 128 Ki) splits rounded up to
    # whole 8-warp CTAs; the oracle decodes the same entries thread by thread
    rng = np.random.default_rng(11)
    big = sorted(range(len(syms)), key=lambda k: -len(syms[k]))[:3]
    for k in big + [int(v) for v in rng.choice(len(syms), size=3, replace=False)]:
        s = syms[k]
        want = -(-len(s) // 131072)
        c = R.combine_splits(streams[k], -(-want // 8) * 8)
        e = c.export()
        K = c.info["n_entries"]
        ost = oracle.OracleStream(len(s), 12, 32, 16, 16, e["freq"], e["words"], e["final"], None, None,
                                  e["entry_word"].astype(np.int64),
                                  np.vstack([e["entry_index"].astype(np.int64), np.zeros((1, 32), np.int64)]),
                                  np.vstack([e["entry_state"].astype(np.uint32), e["final"][None, :]]))
        got = outs[k][: len(s)].cpu().numpy()
        for t in {0, K // 2, K - 1}:
            lo, hi = oracle.owned_range(ost, t)
            if hi < lo:
                continue
            ref = oracle.decode_thread(ost, t)
            assert np.array_equal(got[lo:hi + 1], ref[lo:hi + 1].astype(np.uint8)), (k, t)
