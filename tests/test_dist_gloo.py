"""Multi-rank host logic on CPU (gloo, world size 2).

A batch decodes stream by stream, so ranks need no exchange while decoding:
recoil_shard assigns streams to ranks, each rank decodes its shard (here with
the oracle, on CPU), and the union of the shards is the whole batch. The
bench's job-level numbers take the slowest rank's time and all ranks' bytes.

One stream over several ranks: recoil_plan_create_shard gives each rank a
contiguous run of splits owning a contiguous symbol range; the ranks decode
their runs (the oracle's split threads here) and the concatenation of the
ranges is the stream.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import workloads


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import paper_2306_12141_b300 as R
    specs = workloads.batch_specs(count=24, seed=61, scale_sizes=0.02)
    syms = workloads.batch_symbols(specs)
    streams = [R.encode_with_splits(s, sp.n_bits, workloads.batch_split_count(len(s))) for s, sp in zip(syms, specs)]
    owner = R.shard(streams, world)
    mine = [i for i in range(len(streams)) if owner[i] == rank]
    decoded = {}
    for i in mine:
        o = oracle.encode_with_splits(syms[i], specs[i].n_bits, workloads.batch_split_count(len(syms[i])))
        decoded[i] = oracle.decode_splits(o).astype(np.uint8).tobytes()
    got = [None] * world
    td.all_gather_object(got, decoded)
    ms, total = bench.aggregate(1.0 + rank, sum(len(syms[i]) for i in mine), torch.device("cpu"))
    if rank == 0:
        merged = {}
        for d in got:
            assert not (set(d) & set(merged))            # shards are disjoint
            merged.update(d)
        ok = sorted(merged) == list(range(len(syms))) and all(merged[i] == syms[i].tobytes() for i in merged)
        loads = [sum(len(syms[i]) for i in range(len(syms)) if owner[i] == r) for r in range(world)]
        q.put((ok, ms, total, sum(len(s) for s in syms), loads, max(len(s) for s in syms)))
    td.destroy_process_group()


def test_two_ranks_shard_decode_and_aggregate(recoil_lib):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    ok, ms, total, expect, loads, biggest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ok
    assert ms == 2.0 and total == expect                  # slowest rank's time, every rank's bytes
    assert max(loads) - min(loads) <= biggest             # longest-first keeps ranks within one stream


def _stream_rank_main(rank, world, port, q):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2306_12141_b300 as R
    st = workloads.Stream("z", 300_007, 1, 12, "zipf", {"s": 1.1}, seed=71)
    s = st.symbols()
    p = R.encode_with_splits(s, st.n_bits, 40)
    plan, lo, hi = R.Plan.shard(p, world, rank, {"warps_per_cta": 8})
    # the oracle decodes this rank's run: the split threads whose owned ranges lie in [lo, hi)
    o = oracle.encode_with_splits(s, st.n_bits, 40)
    out = np.zeros(len(s), dtype=np.uint32)
    threads = 0
    for k in range(o.K):
        a, b = oracle.owned_range(o, k)
        if lo <= a and b < hi:
            oracle.decode_thread(o, k, out=out)
            threads += 1
    got = [None] * world
    td.all_gather_object(got, (lo, hi, out[lo:hi].astype(np.uint8).tobytes(), threads))
    if rank == 0:
        got.sort()
        tiles = all(got[r][1] == got[r + 1][0] for r in range(world - 1)) and got[0][0] == 0 and got[-1][1] == len(s)
        whole = b"".join(g[2] for g in got) == s.tobytes()
        q.put((tiles, whole, [g[3] for g in got], o.K, [g[1] - g[0] for g in got]))
    td.destroy_process_group()


def test_two_ranks_shard_one_stream(recoil_lib):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_stream_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    tiles, whole, threads, K, sizes = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tiles and whole
    assert sum(threads) == K                              # every split thread runs on exactly one rank
    assert max(sizes) - min(sizes) <= 2 * max(sizes) // 40 + 1   # balanced within about one split
