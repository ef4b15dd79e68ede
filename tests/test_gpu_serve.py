"""Serving runtime: continuous batching with admission by device memory.

Each request's output must be the same bytes whether its stream is decoded
alone (recoil_decode) or inside the serving mix, where it is combined to a
different split count and shares launches with other requests (the codec is
lossless and combining never changes output, Sec. 3.3).
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pool(R, count=24, seed=50):
    g = np.random.default_rng(seed)
    syms, streams = [], []
    for k in range(count):
        N = int(g.integers(1, 400_000))
        if k % 6 == 5:
            st = workloads.Stream("g", N, 2, 15, "gauss16", {"mean": 2048.0, "sigma": 150.0, "k": 4096}, seed=k)
        elif k % 6 == 4:
            st = workloads.Stream("e", N, 1, 16, "expbytes", {"lam": 50.0}, seed=k)
        else:
            st = workloads.Stream("l", N, 1, 12, "laplace", {"mean": 128.0, "scale": float(g.uniform(2, 64))}, seed=k)
        s = st.symbols()
        syms.append(s)
        streams.append(R.encode_with_splits(s, st.n_bits, max(1, N // 4096)))
    return syms, streams


def _alone(R, stream, nbytes):
    need = R.workspace_size([stream])
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.zeros(max(1, nbytes), dtype=torch.uint8, device="cuda")
    R.decode(stream, out, ws, need, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()[:nbytes]


def test_each_result_is_the_same_alone_and_in_the_mix(recoil_lib):
    R = recoil_lib
    syms, pool = _pool(R)
    alone = [_alone(R, st, len(s) * s.itemsize) for s, st in zip(syms, pool)]
    for a, s in zip(alone, syms):
        assert np.array_equal(a.view(s.dtype), s)
    n_req = 400
    picks = workloads.request_picks(len(pool), n_req, seed=51)
    arrive = workloads.poisson_arrivals(20_000.0, n_req, seed=51)
    outs = [torch.full((max(1, len(syms[p]) * syms[p].itemsize),), 0xAB, dtype=torch.uint8, device="cuda")
            for p in picks]
    budget = 64 << 20
    need = R.serve_arena_size(pool, budget)
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    res, stats = R.serve(pool, picks, arrive, arena, need, budget, outs=[o.data_ptr() for o in outs],
                         max_inflight=4, max_batch=16, timeout_s=60.0)
    assert stats["requests"] == n_req and stats["launches"] <= n_req
    for r, p in enumerate(picks):
        got = outs[r].cpu().numpy()[: len(alone[p])]
        assert np.array_equal(got, alone[p]), r
    assert np.all(res["done_s"] >= res["arrival_s"]) and np.all(res["admit_s"] >= res["arrival_s"] - 1e-9)
    assert stats["p50_ms"] <= stats["p99_ms"]
    # split counts adapt to the free warps: some request was combined below its encoded count
    enc = np.array([pool[p].info["n_entries"] for p in picks])
    assert np.any(res["splits"] <= enc)


def test_arena_outputs_budget_and_per_request_baseline(recoil_lib):
    R = recoil_lib
    syms, pool = _pool(R, count=10, seed=52)
    n_req = 200
    picks = workloads.request_picks(len(pool), n_req, seed=53)
    arrive = workloads.poisson_arrivals(50_000.0, n_req, seed=53)
    budget = max(len(s) * s.itemsize for s in syms) * 3         # forces admission to wait for memory
    for per_request in (False, True):
        need = R.serve_arena_size(pool, budget)
        arena = torch.empty(need, dtype=torch.uint8, device="cuda")
        res, stats = R.serve(pool, picks, arrive, arena, need, budget, per_request=per_request, timeout_s=60.0)
        assert stats["requests"] == n_req
        if per_request:
            assert stats["launches"] == n_req and stats["max_inflight"] == 1
            assert np.all(res["splits"] == np.array([pool[p].info["n_entries"] for p in picks]))


def test_timeout_is_reported_not_hung(recoil_lib):
    R = recoil_lib
    syms, pool = _pool(R, count=4, seed=54)
    picks = np.zeros(50, dtype=np.int64)
    arrive = np.linspace(0.0, 20.0, 50)                           # arrivals far beyond the limit
    need = R.serve_arena_size(pool, 16 << 20)
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RecoilError) as e:
        R.serve(pool, picks, arrive, arena, need, 16 << 20, timeout_s=0.3)
    assert e.value.code == R.ETIMEOUT


def test_admission_bounds_split_length(recoil_lib):
    """Every request is combined to at least n_syms / max_split_symbols splits (rounded to
    whole CTAs, capped by its encoded entries), however busy the device is."""
    R = recoil_lib
    syms, pool = _pool(R, count=12, seed=55)
    n_req = 300
    picks = workloads.request_picks(len(pool), n_req, seed=56)
    arrive = workloads.poisson_arrivals(50_000.0, n_req, seed=56)
    budget = 256 << 20
    need = R.serve_arena_size(pool, budget)
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    max_split, warps = 8192, 8
    res, stats = R.serve(pool, picks, arrive, arena, need, budget, warps_per_cta=warps, max_inflight=4,
                         max_split_symbols=max_split, timeout_s=60.0)
    assert stats["requests"] == n_req
    for r, p in enumerate(picks):
        n, enc = pool[p].info["n_syms"], pool[p].info["n_entries"]
        floor = -(-n // max_split)
        floor = -(-floor // warps) * warps
        assert res["splits"][r] >= min(enc, floor), (r, res["splits"][r], enc, floor)


def test_backlog_admits_larger_batches_within_the_descriptor_area(recoil_lib):
    """Every request arrives at once (a saturating load): admissions take up to 8 x max_batch
    requests while their descriptors fit the slot's area, with a small area forcing early
    cuts; every output is the request's input."""
    R = recoil_lib
    syms, pool = _pool(R, count=16, seed=57)
    n_req = 600
    picks = workloads.request_picks(len(pool), n_req, seed=58)
    arrive = np.zeros(n_req)
    outs = [torch.full((max(1, len(syms[p]) * syms[p].itemsize),), 0xAB, dtype=torch.uint8, device="cuda")
            for p in picks]
    budget = 1 << 30
    for meta in (0, 256 << 10):                                   # default 16 MiB, and 256 KiB
        need = R.serve_arena_size(pool, budget, meta_bytes=meta)
        arena = torch.empty(need, dtype=torch.uint8, device="cuda")
        res, stats = R.serve(pool, picks, arrive, arena, need, budget, outs=[o.data_ptr() for o in outs],
                             max_inflight=4, max_batch=16, meta_bytes=meta, timeout_s=60.0)
        assert stats["requests"] == n_req
        per_launch = np.bincount(res["launch"])
        assert per_launch.max() <= 128
        if meta == 0:
            assert per_launch.max() > 16                              # the backlog took larger batches
        for r, p in enumerate(picks):
            s = syms[p]
            assert np.array_equal(outs[r].cpu().numpy()[: len(s) * s.itemsize].view(s.dtype), s), (meta, r)
            outs[r].fill_(0xAB)
