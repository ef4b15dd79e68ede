"""recoil_decode_noalloc: decoding for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc where they decode (code inside a host
framework that owns every device allocation and lends only fixed buffers, or a
path where an allocation could block or fail). They pass device buffers they
already hold for the compressed words and the output, and the library keeps
its per-call data in a fixed device array. These tests call that entry point
through the C-ABI twice in a row and require exactly the bytes the regular
workspace entry point (recoil_decode) produces: decoding is integer work, so
the tolerance is zero. This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _device_words(R, stream):
    """The stream's words in a device buffer padded to whole 256-word chunks."""
    words = stream.export()["words"]
    nbytes = R.noalloc_words_bytes(stream)
    buf = torch.zeros(max(16, nbytes), dtype=torch.uint8, device="cuda")
    if len(words):
        buf[: 2 * len(words)] = torch.from_numpy(words.view(np.uint8)).cuda()
    return buf, nbytes


def _regular(R, stream, cs):
    info = stream.info
    need = R.workspace_size([stream])
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.zeros(max(1, info["n_syms"] * info["sym_bytes"]), dtype=torch.uint8, device="cuda")
    R.decode(stream, out, ws, need, cs)
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_workspace_decode_on_consecutive_calls(recoil_lib):
    R = recoil_lib
    cs = torch.cuda.current_stream()
    lap = workloads.laplace_1mib()
    gauss = workloads.Stream("g", 300_001, 2, 15, "gauss16", {"mean": 2048.0, "sigma": 200.0, "k": 4096}, seed=9)
    streams = [R.encode_with_splits(lap.symbols(), lap.n_bits, 64),
               R.encode_with_splits(gauss.symbols(), gauss.n_bits, 37)]
    # two calls in a row on each stream, alternating, so each call finds the
    # other stream's descriptors in the shared array
    for rnd in range(2):
        for st in streams:
            info = st.info
            want = _regular(R, st, cs)
            words, nbytes = _device_words(R, st)
            out = torch.full_like(want, 0xAB)
            R.decode_noalloc(st, words, nbytes, out, cs)
            assert torch.equal(out, want), (rnd, info)


def test_noalloc_rejects_what_does_not_fit(recoil_lib):
    R = recoil_lib
    s = workloads.Stream("t", 20_000 * 600, 1, 11, "laplace", {"mean": 128.0, "scale": 8.0}, seed=10).symbols()
    big = R.encode_with_splits(s, 11, 20_000)
    words, nbytes = _device_words(R, big)
    out = torch.empty(len(s), dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RecoilError) as e:
        R.decode_noalloc(big, words, nbytes, out)
    assert e.value.code == R.EINVAL and "fewer splits" in str(e.value)
    small = R.combine_splits(big, 64)
    with pytest.raises(R.RecoilError) as e:
        R.decode_noalloc(small, words, 16, out)
    assert e.value.code == R.EINVAL
    R.decode_noalloc(small, words, nbytes, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), s)
