"""Randomised GPU parity: streams drawn at random (alphabet, n, length, skew, symbol width; static
models, and adaptive ones with a random PDF row per symbol index), encoded by the library, combined
to a random split count and decoded on the GPU with a random CTA shape, alone and all together in
one batch; every output is the input and the oracle's split decode."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _draw(k):
    g = np.random.default_rng(1000 + k)
    n = int(g.integers(1, 17))
    sym_bytes = int(g.integers(1, 3))
    A = int(g.integers(1, min(1 << n, 256 if sym_bytes == 1 else 4096) + 1))
    N = int(g.choice([int(g.integers(1, 100)), int(g.integers(100, 200_000))]))
    p = g.random(A) ** (1.0 + 12.0 * g.random())
    p /= p.sum()
    s = g.choice(A, size=N, p=p).astype(np.uint8 if sym_bytes == 1 else np.uint16)
    return s, n, int(g.integers(1, 400)), int(g.integers(1, 500)), int(g.choice([1, 2, 4, 8, 16, 32]))


def _decode(R, streams, warps):
    plan = R.Plan(streams, {"warps_per_cta": warps})
    ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device="cuda")
    outs = [torch.full((max(1, st.info["n_syms"] * st.info["sym_bytes"]),), 0xAB, dtype=torch.uint8, device="cuda")
            for st in streams]
    plan.upload(ws)
    plan.decode([o.data_ptr() for o in outs])
    assert plan.errors() == 0, R.recoil_last_error()
    res = []
    for o, st in zip(outs, streams):
        a = o.cpu().numpy()[: st.info["n_syms"] * st.info["sym_bytes"]]
        res.append(a.view(np.uint16) if st.info["sym_bytes"] == 2 else a)
    return res


CASES = [_draw(k) for k in range(40)]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_random_stream_decodes_exactly(recoil_lib, k):
    R = recoil_lib
    s, n, M, target, warps = CASES[k]
    c = R.combine_splits(R.encode_with_splits(s, n, M), target)
    (got,) = _decode(R, [c], warps)
    assert np.array_equal(got, s)
    o = oracle.combined(oracle.encode_with_splits(s, n, M, alphabet=None), target)
    assert np.array_equal(got, oracle.decode_splits(o).astype(s.dtype))


def test_random_streams_in_one_batch(recoil_lib):
    """Every kind of table the draws produce, decoded together (one launch per kind)."""
    R = recoil_lib
    streams = [R.combine_splits(R.encode_with_splits(s, n, M), t) for s, n, M, t, _ in CASES]
    for warps in (4, 16):
        for got, (s, *_rest) in zip(_decode(R, streams, warps), CASES):
            assert np.array_equal(got, s)


def _quantised_rows(g, T, A, n):
    """T random PDFs over A symbols, each quantised to frequencies >= 1 summing to 2^n."""
    rows = np.empty((T, A), dtype=np.uint32)
    for t in range(T):
        p = g.random(A) ** (1.0 + 12.0 * g.random())
        p /= p.sum()
        f = np.floor(p * ((1 << n) - A)).astype(np.int64) + 1
        f[np.argmax(f)] += (1 << n) - f.sum()
        rows[t] = f
    return rows


def _draw_adaptive(k):
    g = np.random.default_rng(5000 + k)
    n = int(g.integers(2, 17))
    sym_bytes = int(g.integers(1, 3))
    A = int(g.integers(2, min(1 << n, 256 if sym_bytes == 1 else 4096) + 1))
    T = int(g.integers(1, 9))
    tables = _quantised_rows(g, T, A, n)
    N = int(g.choice([int(g.integers(1, 100)), int(g.integers(100, 120_000))]))
    tid = g.integers(0, T, size=N).astype(np.uint8)
    cdf = np.cumsum(tables, axis=1) / float(1 << n)
    u = g.random(N)
    s = np.array([np.searchsorted(cdf[t], x, side="right") for t, x in zip(tid, u)])
    s = np.minimum(s, A - 1).astype(np.uint8 if sym_bytes == 1 else np.uint16)
    return s, n, tables, tid, int(g.integers(1, 300)), int(g.integers(1, 400)), int(g.choice([4, 8, 16, 32]))


ADAPTIVE = [_draw_adaptive(k) for k in range(16)]


@pytest.mark.parametrize("k", range(len(ADAPTIVE)))
def test_random_adaptive_stream_decodes_exactly(recoil_lib, k):
    R = recoil_lib
    s, n, tables, tid, M, target, warps = ADAPTIVE[k]
    c = R.combine_splits(R.encode_adaptive(s, n, tables, tid, M), target)
    for flags in (0, R.BATCH_NO_PAIRS):
        plan = R.Plan([c], {"warps_per_cta": warps, "flags": flags})
        ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device="cuda")
        out = torch.full((max(1, len(s) * s.itemsize),), 0xAB, dtype=torch.uint8, device="cuda")
        plan.upload(ws)
        plan.decode([out.data_ptr()])
        assert plan.errors() == 0, R.recoil_last_error()
        got = out.cpu().numpy()[: len(s) * s.itemsize].view(s.dtype)
        assert np.array_equal(got, s), flags
    o = oracle.combined(oracle.encode_adaptive_with_splits(s, tid, tables, n, M), target)
    assert np.array_equal(oracle.decode_splits(o).astype(s.dtype), s)


@pytest.mark.parametrize("k", range(6))
def test_random_serving_runs(recoil_lib, k):
    """Serving with a random pool (static models of every table kind, and adaptive ones), random
    request picks, bursty arrivals, a random CTA size, backlog factor and descriptor area: every
    request's output is its stream's input, whatever admission carried it."""
    R = recoil_lib
    g = np.random.default_rng(9000 + k)
    members = [CASES[int(i)] for i in g.choice(len(CASES), size=6, replace=False)]
    pool = [R.encode_with_splits(s, n, max(1, min(M, len(s) // 64 + 1))) for s, n, M, _t, _w in members]
    syms = [m[0] for m in members]
    if k % 2:
        s, n, tables, tid, M, _t, _w = ADAPTIVE[int(g.integers(len(ADAPTIVE)))]
        pool.append(R.encode_adaptive(s, n, tables, tid, max(1, min(M, len(s) // 64 + 1))))
        syms.append(s)
    n_req = int(g.integers(50, 400))
    picks = g.integers(0, len(pool), size=n_req)
    gaps = np.where(g.random(n_req) < 0.3, 0.0, g.exponential(1.0 / float(g.choice([2e3, 2e4, 2e5])), size=n_req))
    arrive = np.cumsum(gaps)
    outs = [torch.full((max(1, len(syms[p]) * syms[p].itemsize),), 0xAB, dtype=torch.uint8, device="cuda")
            for p in picks]
    budget = 1 << 30
    meta = int(g.choice([0, 1 << 20, 4 << 20]))
    warps = int(g.choice([4, 8, 16]))
    need = R.serve_arena_size(pool, budget, meta_bytes=meta, warps_per_cta=warps)
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    res, stats = R.serve(pool, picks, arrive, arena, need, budget, outs=[o.data_ptr() for o in outs],
                         warps_per_cta=warps, max_inflight=int(g.integers(1, 6)), max_batch=int(g.integers(1, 40)),
                         meta_bytes=meta, timeout_s=60.0)
    assert stats["requests"] == n_req
    for r, p in enumerate(picks):
        s = syms[p]
        got = outs[r].cpu().numpy()[: len(s) * s.itemsize].view(s.dtype)
        assert np.array_equal(got, s), (k, r, int(p))
