"""Host side of serving (no GPU): the arena recoil_serve asks for holds, besides the pool's
words and tables, one descriptor per split of every pool stream (288 bytes each, made resident
before the run so that an admission sends 16-byte references to them), one descriptor area per
launch slot and the output budget."""
import workloads


def _laplace(R, max_splits, seed=1, N=200_003):
    s = workloads.Stream("l", N, 1, 12, "laplace", {"mean": 128.0, "scale": 8.0}, seed=seed).symbols()
    return R.encode_with_splits(s, 12, max_splits)


def _desc_bytes(count):
    return -(-count * 288 // 256) * 256


def test_arena_holds_every_pool_descriptor(recoil_lib):
    R = recoil_lib
    few, many = _laplace(R, 24), _laplace(R, 48)
    assert few.info["n_words"] == many.info["n_words"]           # same bitstream, more split entries
    n_few, n_many = few.info["n_entries"], many.info["n_entries"]
    assert n_many > n_few
    budget = 1 << 20
    grow = R.serve_arena_size([many], budget) - R.serve_arena_size([few], budget)
    assert grow == _desc_bytes(n_many) - _desc_bytes(n_few)
    # a pool of several streams: the descriptors of all of them, counted once
    pool = [_laplace(R, k, seed=2 + k) for k in (8, 16, 40)]
    one = [R.serve_arena_size([p], budget) for p in pool]
    both = R.serve_arena_size(pool[:2], budget)
    assert both > max(one[:2])


def test_arena_grows_with_slots_and_budget(recoil_lib):
    R = recoil_lib
    p = _laplace(R, 16)
    base = R.serve_arena_size([p], 1 << 20)
    assert R.serve_arena_size([p], 2 << 20) - base == 1 << 20
    assert R.serve_arena_size([p], 1 << 20, meta_bytes=1 << 20, max_inflight=2) < base
