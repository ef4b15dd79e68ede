"""Which decoder tables a plan stages for a static model, and (GPU) that the packed 16-bit
tables decode exactly at the edges of their packing.

A static model is decoded with one packed u32 per slot where its numbers fit: 8-bit symbols
with n <= 12 (bias | sym << 12 | f << 20), or 16-bit symbols below 2^12 with n <= 15 and every
f <= 1023 (bias | f << 10 | sym << 20); otherwise with a slot -> symbol array and a symbol ->
(f, F) array (two shared reads a symbol). Plans are built on the host, so the choice is checked
without a GPU; the GPU cases compare with the input and with the oracle's split decode.
"""
import numpy as np
import pytest

import oracle
import workloads


def _kinds(R, s, n, M=64, warps=8):
    return R.Plan([R.encode_with_splits(s, n, M)], {"warps_per_cta": warps}).kernels


def _two_symbols(N, f_big, n, seed):
    """uint16 symbols 0 and 1 with P(0) = f_big / 2^n (the quantised f(0) lands at or near f_big)."""
    g = np.random.default_rng(seed)
    s = (g.random(N) >= f_big / float(1 << n)).astype(np.uint16)
    return s


def test_static_models_pick_their_tables(recoil_lib):
    R = recoil_lib
    g16 = workloads.Stream("g", 100_003, 2, 15, "gauss16", {"mean": 2048.0, "sigma": 200.0, "k": 4096}, seed=3).symbols()
    assert _kinds(R, g16, 15) == R.KERNEL_PACKED16                  # max f ~ 65 at n = 15
    assert _kinds(R, g16, 16) == R.KERNEL_GENERIC16                 # n = 16: the LUT would be 256 KB
    narrow = workloads.Stream("g", 100_003, 2, 15, "gauss16", {"mean": 2048.0, "sigma": 3.0, "k": 4096}, seed=4).symbols()
    assert _kinds(R, narrow, 15) == R.KERNEL_GENERIC16              # f of the mode above 1023
    wide = np.random.default_rng(5).integers(0, 8192, size=50_000).astype(np.uint16)
    assert _kinds(R, wide, 15) == R.KERNEL_GENERIC16                # symbols beyond 2^12
    lap = workloads.Stream("l", 100_003, 1, 12, "laplace", {"mean": 128.0, "scale": 8.0}, seed=6).symbols()
    assert _kinds(R, lap, 12) == R.KERNEL_PACKED8
    assert _kinds(R, lap, 13) == R.KERNEL_GENERIC8


def test_packed16_limits_on_the_host(recoil_lib):
    """f = 1023 still packs, an f above it does not; every value of a 4096-symbol alphabet packs."""
    R = recoil_lib
    n = 10
    s = _two_symbols(200_000, 1023, n, seed=7)
    p = R.encode_with_splits(s, n, 16)
    assert R.stream_freq(p).max() == 1023
    assert R.Plan([p], {"warps_per_cta": 8}).kernels == R.KERNEL_PACKED16
    s = _two_symbols(200_000, 1024, 11, seed=8)
    q = R.encode_with_splits(s, 11, 16)
    assert R.stream_freq(q).max() > 1023                             # 1022 and 1026 of 2048 slots
    assert R.Plan([q], {"warps_per_cta": 8}).kernels == R.KERNEL_GENERIC16
    every = np.repeat(np.arange(4096, dtype=np.uint16), 8)
    np.random.default_rng(9).shuffle(every)
    assert _kinds(R, every, 12) == R.KERNEL_PACKED16                 # f = 1 for all 4096 symbols


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["f1023_n10", "alphabet4096_n12", "gauss_n15", "gauss_n14"])
@pytest.mark.parametrize("warps", [4, 32])
def test_packed16_decodes_exactly(recoil_lib, case, warps):
    import torch
    R = recoil_lib
    if case == "f1023_n10":
        s, n = _two_symbols(300_007, 1023, 10, seed=11), 10
    elif case == "alphabet4096_n12":
        s = np.repeat(np.arange(4096, dtype=np.uint16), 40)
        np.random.default_rng(12).shuffle(s)
        n = 12
    else:
        n = 15 if case == "gauss_n15" else 14
        s = workloads.Stream("g", 300_007, 2, n, "gauss16", {"mean": 2048.0, "sigma": 200.0, "k": 4096},
                             seed=13).symbols()
    p = R.encode_with_splits(s, n, 300)
    o = oracle.encode_with_splits(s, n, 300, alphabet=None)
    for M in (300, 37, 1):
        c = R.combine_splits(p, M)
        plan = R.Plan([c], {"warps_per_cta": warps})
        assert plan.kernels == R.KERNEL_PACKED16
        ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device="cuda")
        out = torch.full((len(s) * 2,), 0xAB, dtype=torch.uint8, device="cuda")
        plan.upload(ws)
        plan.decode([out.data_ptr()])
        assert plan.errors() == 0, R.recoil_last_error()
        got = out.cpu().numpy().view(np.uint16)
        assert np.array_equal(got, s), (case, M)
        assert np.array_equal(got, oracle.decode_splits(oracle.combined(o, M)).astype(np.uint16)), (case, M)
