"""Randomised host parity (no GPU): the library's encoder, split placement and combiner against
the oracle on streams drawn at random, so that cases nobody wrote down are also checked.

Each example draws an alphabet size, a quantisation precision n (with no more distinct symbols
than 2^n slots), a length (including lengths below and around one group of 32), a skew of the
symbol distribution, a split count, a split rule (the remaining-symbols reading or the printed
T = ceil(N/M) of Def. 4.1) and a combine target. Everything is integer, so the comparison is
bit for bit: frequencies, words, final states, split words, recorded indices and states, and the
entries kept by a combine (Sec. 3.3)."""
import numpy as np
import pytest

import oracle

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


@st.composite
def streams(draw):
    n = draw(st.integers(1, 16))
    sym_bytes = draw(st.sampled_from([1, 2]))
    max_a = min(1 << n, 256 if sym_bytes == 1 else 4096)
    A = draw(st.integers(1, max_a))
    N = draw(st.one_of(st.integers(1, 70), st.integers(71, 6000)))   # empty streams: test_host_parity
    skew = draw(st.floats(0.0, 3.0))
    seed = draw(st.integers(0, 2**31 - 1))
    g = np.random.default_rng(seed)
    p = g.random(A) ** (1.0 + 4.0 * skew)
    p /= p.sum()
    s = g.choice(A, size=N, p=p).astype(np.uint8 if sym_bytes == 1 else np.uint16)
    M = draw(st.integers(1, 60))
    rule = draw(st.sampled_from(["remaining", "eq7"]))
    target = draw(st.integers(1, 70))
    return s, n, M, rule, target


@settings(max_examples=300, deadline=None, derandomize=True)
@given(streams())
def test_library_matches_oracle_on_random_streams(recoil_lib, case):
    R = recoil_lib
    s, n, M, rule, target = case
    p = R.encode_with_splits(s, n, M, rule=rule)
    o = oracle.encode_with_splits(s, n, M, alphabet=None, rule=rule)
    e = p.export()
    assert np.array_equal(e["freq"][: len(o.f)], o.f)
    assert np.array_equal(e["words"], o.words)
    assert np.array_equal(e["final"], o.final)
    assert np.array_equal(e["entry_word"].astype(np.int64), o.q)
    assert np.array_equal(e["entry_index"].astype(np.int64), o.idx[:-1])
    assert np.array_equal(e["entry_state"].astype(np.uint32), o.y[:-1])
    # combining keeps the same entries as the oracle's rule, and the same final entry
    c = R.combine_splits(p, target).export()
    oc = oracle.combined(o, target)
    assert np.array_equal(c["entry_word"].astype(np.int64), oc.q)
    assert np.array_equal(c["entry_index"].astype(np.int64), oc.idx[:-1])
    assert np.array_equal(c["words"], o.words) and np.array_equal(c["final"], o.final)
    # and the oracle's own split decode of the combined stream gives the input back
    assert np.array_equal(oracle.decode_splits(oc).astype(s.dtype), s)
