"""Benchmark: decoded GB/s of the uneven-stream batch on B300, batched persistent vs per-stream.

Workload (default): 4096 independent streams, lognormal sizes (median 256 KiB,
sigma 1.5, clipped to 4 KiB .. 64 MiB, about 3.3 GB of symbols), each of
Laplace(128, b) bytes with its own b ~ U(2, 64) and its own 12-bit table,
encoded at one split entry per 4096 symbols; all streams decoded in one
persistent launch from a device work queue (CUDA graph replay). A step is one
decode of the whole batch. Inputs (3.3 GB out, ~2 GB in) exceed the 126 MB L2.

JSON line keys follow the harness contract; `value` is kernel-side decoded
GB/s (output symbol bytes / device time), `e2e` the same through the public
API with the compressed inputs copied from pinned host memory and the decoded
symbols copied back every step, `per_stream` the one-launch-per-stream
baseline on the same streams, `roofline` the dominant kernel against the
measured HBM copy bandwidth, `cpu_baseline` the oracle on host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "decoded GB/s per B300 (batched persistent vs per-stream Recoil); p50/p99 decode latency"
BATCH_WORKLOAD = ("uneven batch: 4096 Laplace(128, b ~ U(2,64)) byte streams, lognormal sizes median 256 KiB "
                  "sigma 1.5 clipped 4 KiB-64 MiB, n=12, W=32, own table each, 1 split entry per 4096 symbols")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--streams", type=int, default=workloads.BATCH_STREAMS)
    ap.add_argument("--scale", type=float, default=1.0, help="shrink stream sizes (testing only)")
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2],
                    help="coder lanes a thread (0: the autotuner's choice where it runs, else 1)")
    ap.add_argument("--split-symbols", type=int, default=-1)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--per-stream-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "single", "zipf", "serve", "conventional", "adaptive"])
    ap.add_argument("--dist", default="zipf", choices=["zipf", "skewed", "uniform", "gauss16", "laplace"],
                    help="single: which stream (zipf 1 GiB, the 256 MiB extremes, laplace 1 MiB)")
    ap.add_argument("--splits", type=int, default=9472, help="zipf: decoder split count")
    ap.add_argument("--alphabet", type=int, default=256, help="adaptive: symbols per PDF (up to 4096)")
    ap.add_argument("--tables", type=int, default=64, help="adaptive: PDFs (table numbers drawn N(20, 12))")
    ap.add_argument("--sweep", type=lambda v: [int(x) for x in v.split(",") if x], default=[148, 592, 2368, 9472],
                    help="zipf: split counts to sweep (empty to skip)")
    ap.add_argument("--soak", type=float, default=1.0, help="seconds of untimed steps while sampling clocks")
    ap.add_argument("--serve-rates", type=lambda v: [float(x) for x in v.split(",") if x],
                    default=SERVE_RATES + [SATURATING_HZ],
                    help="batch: serving request rates (Poisson, per second; the last one saturates the device)")
    ap.add_argument("--e2e-groups", type=int, default=16, help="stream groups of the end-to-end pipeline")
    ap.add_argument("--serve-requests", type=int, default=20000, help="requests per serving rate (0: skip)")
    ap.add_argument("--no-configs", action="store_true", help="batch: skip the block of the other workloads")
    ap.add_argument("--configs-scale", type=float, default=1.0, help="shrink the other workloads (testing only)")
    ap.add_argument("--rr-streams", type=int, default=8,
                    help="CUDA streams of the round-robin per-stream baseline (0: skip)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def aggregate(ms_local: float, bytes_local: int, device=None):
    """Job time = slowest rank; job bytes = all ranks' symbols (one rank: unchanged)."""
    import torch
    import torch.distributed as td
    if device is None or not td.is_initialized() or td.get_world_size() == 1:
        return ms_local, bytes_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    b = torch.tensor([float(bytes_local)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    td.all_reduce(b, op=td.ReduceOp.SUM)
    return float(t.item()), int(b.item())


def code_only(source: str) -> str:
    """C++/CUDA source without comments and blank runs, so that the recorded counts stay tied to
    what compiles, not to how it is annotated."""
    import re
    source = re.sub(r"/\*.*?\*/", " ", source, flags=re.S)
    source = re.sub(r"//[^\n]*", "", source)
    return "\n".join(line.rstrip() for line in source.splitlines() if line.strip())


def recorded_traffic(key: str, what: str = "traffic_bytes"):
    """A per-launch count recorded by an ncu capture (DRAM bytes, or warp instructions with
    what="instructions"), if the kernel sources still match the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "decode_kernel_traffic.md")
    src = os.path.join(ROOT, "paper_2306_12141_b300", "csrc")
    try:
        text = open(path).read()
        h = hashlib.sha256()
        for f in ("decode_kernels.cu", "device_types.h"):
            h.update(code_only(open(os.path.join(src, f)).read()).encode())
    except OSError:
        return None
    want = f"kernel_sources_sha256_16: {h.hexdigest()[:16]}"
    if want not in text:
        return None
    for line in text.splitlines():
        line = line.strip()
        if line.startswith(f"{what} {key}:"):
            return int(line.split(":")[1])
    return None


def issue_rate(key: str, mean_ms: float, dev, clocks: dict):
    """The decode launch against the SMs' instruction-issue rate: warp instructions per launch
    (ncu, recorded with the traffic) over the launch time measured here, against one warp
    instruction per clock on each of 4 schedulers of every SM at the sampled SM clock. The
    kernel is bound by integer issue long before HBM, so this is the fraction that says how
    close it runs to its own limit; None without a matching record."""
    import torch
    inst = recorded_traffic(key, "instructions")
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if inst is None or not mhz:
        return None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    achieved = inst / (mean_ms * 1e-3)
    peak = sms * 4 * mhz * 1e6
    return {"achieved": achieved, "peak": peak, "unit": "warp instructions/s", "frac": achieved / peak,
            "instructions_per_launch": inst, "peak_from": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz (sampled)"}


KERNEL_NAMES = ("kPacked8", "kGeneric8", "kGeneric16", "kAdaptive8", "kAdaptive16", "kAdaptive16Wide",
                "kAdaptive8Pair", "kAdaptive16Pair", "kPacked16")


def kernel_of(plan) -> tuple[str, str]:
    """(symbol dtype, decode kernels) of a plan, from the table kinds it launches."""
    dtype = "u16" if plan.streams[0].info["sym_bytes"] == 2 else "u8"
    names = [n for k, n in enumerate(KERNEL_NAMES) if plan.kernels >> k & 1]
    return dtype, " + ".join(f"decode_kernel<{n}>" for n in names)


NOMINAL_HBM_GBS = 8000.0      # HBM3e nominal (~8 TB/s), a second denominator beside the measured copy


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6400.0, "source": "fallback"}


def build_batch(R, count: int, scale: float, rank: int = 0):
    specs = workloads.batch_specs(count=count, seed=6 + 1000 * rank, scale_sizes=scale)
    syms = workloads.batch_symbols(specs)
    threads = max(1, min(64, os.cpu_count() or 1))

    def enc(k):
        return R.encode_with_splits(syms[k], specs[k].n_bits, workloads.batch_split_count(len(syms[k])))

    with ThreadPoolExecutor(threads) as ex:
        streams = list(ex.map(enc, range(count)))
    return specs, syms, streams


# -------------------------------------------------------------- CPU oracle
def _oracle_job(spec, sym):
    import oracle
    f = oracle.quantize(np.bincount(sym, minlength=256), spec.n_bits)
    words, final, _, _ = oracle.encode(sym, f, spec.n_bits)
    return f, words, final


def oracle_rate(specs, syms, seconds: float, threads: int, seed: int = 0):
    """Decoded GB/s of the oracle's decoder (plain C, one instance per thread) on random batch streams.

    Streams are encoded by the oracle, then decoded in parallel, one stream per
    thread at a time, until `seconds` of wall time have been spent decoding.
    """
    import oracle
    order = np.random.default_rng(seed).permutation(len(specs))
    done, wall, picked, pos = 0, 0.0, 0, 0
    with ThreadPoolExecutor(threads) as ex:
        while wall < seconds and pos < len(order):
            ks = order[pos:pos + 4 * threads]
            pos += len(ks)
            enc = list(ex.map(lambda k: _oracle_job(specs[k], syms[k]), ks))

            def dec(a):
                k, (f, words, final) = a
                out, _, end_p = oracle.decode_serial(words, final, len(syms[k]), f, specs[k].n_bits)
                return end_p == -1 and np.array_equal(out, syms[k])

            t = time.perf_counter()
            ok = list(ex.map(dec, zip(ks, enc)))
            wall += time.perf_counter() - t
            assert all(ok)
            done += sum(len(syms[k]) for k in ks)
            picked += len(ks)
    return done / wall / 1e9, picked, done


def cpu_baseline(specs, syms, seconds: float) -> dict:
    threads = os.cpu_count() or 1
    v, picked, done = oracle_rate(specs, syms, seconds, threads)
    v1, picked1, done1 = oracle_rate(specs, syms, max(1.0, seconds / 4), 1, seed=1)
    return {"value": v, "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"{picked} of {len(specs)} batch streams ({done / 1e6:.1f} MB of symbols); oracle "
                      f"interleaved decoder (plain C -O2), one instance per host thread, decode wall time",
            "single_core": {"value": v1, "unit": "GB/s", "cores": 1,
                            "sample": f"{picked1} streams ({done1 / 1e6:.1f} MB), one thread"}}


def run_reference(a):
    """--impl reference: the oracle timed on the host cores, each step a bounded sample of the batch."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    specs = workloads.batch_specs(count=a.streams, scale_sizes=a.scale)
    threads = os.cpu_count() or 1
    budget = max(1.0, 60.0 / max(1, a.steps + a.warmup))
    rates, sizes = [], []
    for step in range(a.warmup + a.steps):
        g = np.random.default_rng(100 + step)
        ks = g.choice(len(specs), size=min(len(specs), 16 * threads), replace=False)
        sub = [specs[k] for k in ks]
        syms = workloads.batch_symbols(sub)
        v, picked, done = oracle_rate(sub, syms, budget, threads, seed=step)
        if step >= a.warmup:
            rates.append(v)
            sizes.append(done)
    v = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * statistics.mean(sizes) / (v * 1e9),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step: up to {16 * threads} random batch streams, "
                                       f"about {budget:.1f} s of decode"},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
SINGLE = {
    "zipf": (workloads.zipf_1gib, 1 << 30, "1 GiB of Zipf(s=1.2) bytes over 256 symbols, n=12"),
    "skewed": (workloads.skewed_256mib, 1 << 28, "256 MiB of bytes with P(0)=0.95, the rest uniform, n=12"),
    "uniform": (workloads.uniform_256mib, 1 << 28, "256 MiB of uniform bytes, n=12"),
    "gauss16": (workloads.gauss16_256mib, 1 << 27, "2^27 uint16 symbols, Normal(2048, 200) clipped to 0..4095, n=15"),
    "laplace": (workloads.laplace_1mib, 1 << 20, "1 MiB of Laplace(128, 8) bytes, n=11"),
}


SERVE_RATES = [2000, 5000, 10000, 20000, 50000]
# offered load far above what the device decodes: every request arrives within a few ms, so the
# decoded GB/s is set by the device and the admission loop, not by the arrivals
SATURATING_HZ = 10_000_000.0


def serving(R, torch, dev, pool, rate, n_req, budget, arena, per_request):
    """One serving run over the pool at a Poisson rate; latency and throughput summary."""
    picks = workloads.request_picks(len(pool), n_req, seed=7)
    arrive = workloads.poisson_arrivals(float(rate), n_req, seed=7)
    res, st = R.serve(pool, picks, arrive, arena, arena.numel(), budget, per_request=per_request,
                      timeout_s=300.0)
    return {"p50_ms": round(st["p50_ms"], 4), "p99_ms": round(st["p99_ms"], 4), "mean_ms": round(st["mean_ms"], 4),
            "decoded_gbs": round(st["decoded_gbs"], 2), "launches": st["launches"],
            "max_inflight": st["max_inflight"], "mean_splits": round(float(np.mean(res["splits"])), 1),
            "makespan_s": round(st["makespan_s"], 4)}


def serving_block(R, torch, dev, pool, rates, n_req, budget=20 << 30):
    """Both arms (continuous batching, and one launch per request with every encoded split) at every
    rate; the key of the saturating load is "saturating"."""
    arena = torch.empty(R.serve_arena_size(pool, budget), dtype=torch.uint8, device=dev)
    out = {}
    for rate in rates:
        key = "saturating" if rate >= SATURATING_HZ else str(int(rate))
        out[key] = {"recoil": serving(R, torch, dev, pool, rate, n_req, budget, arena, False),
                    "per_request": serving(R, torch, dev, pool, rate, n_req, budget, arena, True)}
        out[key]["offered_hz"] = rate
    del arena
    return out


def make_workload(a, R, rank):
    """(description, specs, symbols, encoded streams, streams to decode) of the chosen workload."""
    if a.workload == "batch":
        specs, syms, streams = build_batch(R, a.streams, a.scale, rank)
        return BATCH_WORKLOAD, specs, syms, streams, streams
    make, n_full, what = SINGLE[a.dist]
    st = make(int(n_full * a.scale))
    s = st.symbols()
    enc_splits = 64 if a.dist == "laplace" else max(1, min(65536, len(s) // 4096))
    enc = R.encode_with_splits(s, st.n_bits, enc_splits)
    desc = (f"single stream: {what}, W=32, encoded at {enc_splits} splits and combined to the decoder's "
            f"split count")
    return desc, [st], [s], [enc], [R.combine_splits(enc, a.splits)]


def run_conventional(a):
    """--workload conventional: Recoil splits vs the conventional scheme (Sec. 2.3) on the same input.

    The 1 GiB Zipf input is decoded (1) as one Recoil stream combined to P splits and (2) cut into P
    equal partitions, each an independent interleaved stream with its own final states under the same
    quantised model (the paper's baseline B). Same kernel, same launch shape; reports both decode
    rates and both compressed sizes (Recoil: bitstream + split metadata packed as in Sec. 4.3;
    conventional: every partition's words and final states + an offset table). `overhead_bytes` is
    the growth over the same input coded as one interleaved stream (the paper's variation (a))."""
    import torch
    import paper_2306_12141_b300 as R
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    st = workloads.zipf_1gib(int((1 << 30) * a.scale))
    s = st.symbols()
    enc = R.encode_with_splits(s, st.n_bits, max(1, min(65536, len(s) // 4096)))
    P = a.splits
    rec = R.combine_splits(enc, P)
    freq = R.stream_freq(enc)
    parts = np.array_split(s, P)
    with ThreadPoolExecutor(max(1, min(64, os.cpu_count() or 1))) as ex:
        conv = list(ex.map(lambda p: R.encode_with_table(p, st.n_bits, freq, 1), parts))
    warps = a.warps or 16
    lane_flag = R.BATCH_TWO_LANES if a.lanes == 2 else 0
    cs = torch.cuda.Stream(device=dev)
    ref = torch.from_numpy(s).to(dev)
    res = {}
    for name, streams in (("recoil", [rec]), ("conventional", conv)):
        plan = R.Plan(streams, {"warps_per_cta": warps, "flags": R.BATCH_GRAPH | lane_flag})
        ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device=dev)
        out = torch.empty(len(s), dtype=torch.uint8, device=dev)
        if name == "recoil":
            ptrs = [out.data_ptr()]
        else:
            offs = np.concatenate([[0], np.cumsum([len(p) for p in parts])])
            ptrs = [out.data_ptr() + int(o) for o in offs[:-1]]
        with torch.cuda.stream(cs):
            plan.upload(ws, stream=cs)
            for _ in range(a.warmup):
                plan.decode(ptrs, cs)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
            for e0, e1 in ev:
                e0.record(cs)
                plan.decode(ptrs, cs)
                e1.record(cs)
            torch.cuda.synchronize()
            assert plan.errors(cs) == 0
        assert torch.equal(out, ref), name
        ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
        infos = [x.info for x in streams]
        nbytes = sum(i["bitstream_bytes"] for i in infos)  # words + final states
        if name == "conventional":
            extra = 8 * len(streams)                       # offset table of the partitions
        else:
            extra = R.serialized_size(rec)[1]              # split metadata packed as in Sec. 4.3
        res[name] = {"gbs": len(s) / (ms * 1e-3) / 1e9, "ms": ms, "compressed_bytes": int(nbytes + extra),
                     "overhead_bytes": int(nbytes + extra - enc.info["bitstream_bytes"]),
                     "streams": len(streams), "splits": sum(i["n_entries"] for i in infos)}
        del ws, out
    line = {"metric": METRIC, "value": res["recoil"]["gbs"], "unit": "GB/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": res["recoil"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"Recoil vs conventional partitioning at {P} splits/partitions on 1 GiB of "
                                   f"Zipf(1.2) bytes, n=12, same quantised model, {warps} warps per CTA",
                       "scale": a.scale},
            "recoil": res["recoil"], "conventional": res["conventional"],
            "recoil_vs_conventional_speed": res["recoil"]["gbs"] / res["conventional"]["gbs"]}
    print(json.dumps(line), flush=True)


def _oracle_adaptive_rate(tables, n_bits, sym, tid, seconds: float, threads: int):
    """Decoded GB/s of the oracle's adaptive serial decoder, one 16 Mi-symbol piece per host thread."""
    import oracle
    piece = 1 << 24
    ks = list(range(0, len(sym), piece))

    def enc(k):
        return oracle.encode_adaptive(sym[k:k + piece], tid[k:k + piece], tables, n_bits)

    done, wall, pos = 0, 0.0, 0
    with ThreadPoolExecutor(threads) as ex:
        while wall < seconds and pos < len(ks):
            batch = ks[pos:pos + threads]
            pos += len(batch)
            codes = list(ex.map(enc, batch))

            def dec(a):
                k, (words, final, _, _) = a
                out, _, end_p = oracle.decode_serial_adaptive(words, final, tid[k:k + piece], tables, n_bits)
                return end_p == -1 and np.array_equal(out, sym[k:k + piece])

            t = time.perf_counter()
            ok = list(ex.map(dec, zip(batch, codes)))
            wall += time.perf_counter() - t
            assert all(ok)
            done += sum(min(piece, len(sym) - k) for k in batch) * sym.itemsize
    return done / wall / 1e9, done


def run_adaptive(a):
    """--workload adaptive: latents of a hyperprior image codec, each symbol with its own PDF (Sec. 3.1).

    2^27 uint16 symbols (256 MiB decoded), 64 Gaussian scale tables over 256 values, n = 16 -- the
    paper's image setting (16-bit symbols, a Gaussian per symbol, Sec. 5.1). Encoded at 65536 splits and
    combined to --splits; the decoder reads one table-number byte per symbol, so the algorithmic bytes
    are the words and the table numbers in plus the symbols out."""
    import torch
    import paper_2306_12141_b300 as R
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    st = workloads.adaptive_256mib(int((1 << 27) * a.scale), alphabet=a.alphabet, n_tables=a.tables)
    default_model = a.alphabet == 256 and a.tables == 64
    tables = st.tables()
    s, tid = st.draw()
    enc = R.encode_adaptive(s, st.n_bits, tables, tid, max(1, min(65536, len(s) // 4096)))
    warps = a.warps                                    # 0: the library picks the CTA size
    lane_flag = R.BATCH_TWO_LANES if a.lanes == 2 else 0
    layout_flag = 0                                    # the paired layout where the model has one

    def layout_name(flag):
        return "two-byte guide" if a.alphabet > 256 else ("one-byte guide" if flag else "paired")
    cs = torch.cuda.Stream(device=dev)
    out = torch.empty(len(s) * 2, dtype=torch.uint8, device=dev)
    ref = torch.from_numpy(s.view(np.uint8)).to(dev)
    out_bytes = len(s) * 2

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            e0.record(cs)
            fn()
            e1.record(cs)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    sweep = {}
    with torch.cuda.stream(cs):
        for k in a.sweep:
            sp = R.Plan([R.combine_splits(enc, k)], {"warps_per_cta": warps, "flags": R.BATCH_GRAPH | lane_flag})
            sws = torch.empty(sp.workspace_size, dtype=torch.uint8, device=dev)
            sp.upload(sws, stream=cs)
            t = timed(lambda: sp.decode([out.data_ptr()], cs), 5, 2)
            assert sp.errors(cs) == 0 and torch.equal(out, ref)
            sweep[str(k)] = round(out_bytes / (statistics.mean(t) * 1e-3) / 1e9, 1)
            del sws
        c = R.combine_splits(enc, a.splits)
        tuned = None
        if not warps:
            # the autotuner picks the CTA size for the workload's split count (untimed)
            tws = torch.empty(R.autotune_workspace_size([c]), dtype=torch.uint8, device=dev)
            best, tms = R.autotune([c], [out.data_ptr()], tws, tws.numel(), cs, steps=3, keep_splits=True)
            warps = best["warps_per_cta"]
            lane_flag = best["flags"] & R.BATCH_TWO_LANES
            layout_flag = best["flags"] & R.BATCH_NO_PAIRS
            tuned = {"warps_per_cta": warps, "lanes_per_thread": 2 if lane_flag else 1,
                     "table_layout": layout_name(layout_flag), "ms": round(tms, 4)}
            del tws
        plan = R.Plan([c], {"warps_per_cta": warps, "flags": R.BATCH_GRAPH | lane_flag | layout_flag})
        warps = plan.warps_per_cta
        ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device=dev)
        plan.upload(ws, stream=cs)
        decode = lambda: plan.decode([out.data_ptr()], cs)  # noqa: E731
        with Clocks(local) as clk:
            t_end = time.time() + a.soak
            while time.time() < t_end:
                decode()
                torch.cuda.synchronize()
            ms = timed(decode, a.steps, a.warmup)
        clocks = clk.summary()
        clocks["note"] = f"sampled every 100 ms over a {a.soak:.1f} s soak of the same step and the timed steps"
        assert plan.errors(cs) == 0, R.recoil_last_error()
        assert torch.equal(out, ref)
        launches = plan.launches
        e2e = None
        if not a.no_e2e:
            R.stream_pin(c)
            pipe = R.Pipeline([c], {"warps_per_cta": warps, "split_symbols": 0, "flags": lane_flag | layout_flag},
                              groups=a.e2e_groups)
            wsb, stb = pipe.sizes
            pws = torch.empty(wsb, dtype=torch.uint8, device=dev)
            stage = torch.empty(stb, dtype=torch.uint8, device=dev)
            host = torch.empty(out_bytes, dtype=torch.uint8, pin_memory=True)
            e_ms = timed(lambda: pipe.run([host.data_ptr()], pws, wsb, stage, stb, cs), max(3, a.steps // 2), 1)
            assert pipe.errors() == 0 and np.array_equal(host.numpy(), s.view(np.uint8))
            e2e = {"value": out_bytes / (statistics.mean(e_ms) * 1e-3) / 1e9, "unit": "GB/s",
                   "h2d_bytes_per_step": int(2 * c.info["n_words"] + len(s)), "d2h_bytes_per_step": out_bytes,
                   "ms_per_step": statistics.mean(e_ms),
                   "groups": a.e2e_groups,
                   "note": "recoil_pipeline_run: the stream cut into runs of splits; H2D of each run's words "
                           "and the table numbers, decode, D2H of its symbols, overlapped across runs"}
            del pws, stage
    mean_ms = statistics.mean(ms)
    in_bytes = 2 * c.info["n_words"] + 4 * 32 + len(s)
    peaks = measured_peaks()
    achieved = (out_bytes + in_bytes) / (mean_ms * 1e-3) / 1e9
    line = {"metric": "decoded GB/s of an adaptive (per-symbol PDF) Recoil stream", "value": out_bytes / (mean_ms * 1e-3) / 1e9,
            "unit": "GB/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": mean_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": f"adaptive: 2^27 uint16 latents, symbol i = clip(rint({a.alphabet // 2} + sigma_t Z)) "
                                   f"with t_i ~ clip(rint(N(20, 12)), 0, {a.tables - 1}), {a.tables} log-spaced "
                                   f"Gaussian scale tables (0.11..256) over {a.alphabet} values, n=16, W=32",
                       "splits": c.info["n_entries"], "warps_per_cta": warps,
                       "lanes_per_thread": 2 if lane_flag else 1, "autotuned": tuned,
                       "table_layout": layout_name(layout_flag),
                       "symbols_bytes": out_bytes,
                       "compressed_bytes": 2 * c.info["n_words"] + 4 * 32, "table_number_bytes": len(s),
                       "l2": "inputs larger than L2 (no flush)", "scale": a.scale},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                         "traffic": (recorded_traffic(f"adaptive w{warps} k{a.splits} l{2 if lane_flag else 1}")
                                     if a.scale == 1.0 and default_model and not layout_flag else None),
                         "issue": (issue_rate(f"adaptive w{warps} k{a.splits} l{2 if lane_flag else 1}", mean_ms, dev, clocks)
                                   if a.scale == 1.0 and default_model and not layout_flag else None),
                         "peak_source": peaks["source"],
                         "kernel": "decode_kernel<kAdaptive16>" if a.alphabet <= 256 else "decode_kernel<kAdaptive16Wide>",
                         "bytes": "compressed words + table numbers in, symbols out"},
            "clocks": clocks, "gpu_launches": launches * a.steps, "e2e": e2e, "split_sweep_gbs": sweep}
    if not a.no_cpu:
        threads = os.cpu_count() or 1
        v, done = _oracle_adaptive_rate(tables, st.n_bits, s, tid, a.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": v, "unit": "GB/s", "cores": threads, "kind": "oracle",
                                "sample": f"{done / 1e6:.0f} MB of symbols in 16 Mi-symbol pieces, oracle adaptive "
                                          f"serial decoder (plain C -O2), one piece per host thread"}
    print(json.dumps(line), flush=True)


def time_events(fn, cs, steps: int, warmup: int, gate_ms: float = 2.0) -> list[float]:
    """Milliseconds of each of `steps` calls of fn, CUDA events on cs, after `warmup` calls. The
    timed calls are queued behind a short device-side sleep (gate_ms, untimed), so the device runs
    them back to back and a host scheduling delay while they are queued cannot enter an event pair
    (it would dominate decodes of tens of microseconds)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(cs):
        sleep = getattr(torch.cuda, "_sleep", None)          # torch's bounded spin kernel (clock cycles)
        if gate_ms > 0 and sleep is not None:
            sleep(int(gate_ms * 1e-3 * 2.0e9))                # ~gate_ms at the B300's 2 GHz SM clock
        for e0, e1 in ev:
            e0.record(cs)
            fn()
            e1.record(cs)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def per_stream_round_robin(R, torch, dev, streams, out_ptrs, warps: int, split_symbols: int, n_cuda: int,
                           steps: int, lane_flag: int = 0) -> dict:
    """Per-stream baseline with the batch's own launch shape: one launch per stream (each combined to
    the autotuned split size, the autotuned CTA size), stream i on CUDA stream i mod n_cuda so that
    launches of different streams overlap on the device; one step decodes every stream."""
    main = torch.cuda.current_stream(dev)
    groups = [list(range(g, len(streams), n_cuda)) for g in range(n_cuda)]
    plans = [R.Plan([streams[i] for i in grp], {"warps_per_cta": warps, "split_symbols": split_symbols,
                                                 "flags": R.BATCH_PER_STREAM | lane_flag}) for grp in groups]
    wss = [torch.empty(max(256, p.workspace_size), dtype=torch.uint8, device=dev) for p in plans]
    side = [torch.cuda.Stream(device=dev) for _ in range(n_cuda)]
    ptrs = [[out_ptrs[i] for i in grp] for grp in groups]
    for p, ws, c in zip(plans, wss, side):
        p.upload(ws, stream=c)
    torch.cuda.synchronize()

    def step():
        start = torch.cuda.Event()
        start.record(main)
        for p, c, pp in zip(plans, side, ptrs):
            c.wait_event(start)
            p.decode(pp, c)
            done = torch.cuda.Event()
            done.record(c)
            main.wait_event(done)

    ms = time_events(step, main, steps, 1, gate_ms=0)   # the launches' host cost is part of this baseline
    errors = sum(p.errors(c) for p, c in zip(plans, side))
    assert errors == 0, R.recoil_last_error()
    return {"ms_per_step": statistics.mean(ms), "launches_per_step": sum(p.launches for p in plans),
            "cuda_streams": n_cuda, "warps_per_cta": warps, "split_symbols": split_symbols,
            "lanes_per_thread": 2 if lane_flag else 1}


def _single_input(R, dist: str, scale: float):
    """(symbols, encoded stream, description) of a single-stream workload (one serial encode)."""
    make, n_full, what = SINGLE[dist]
    st = make(int(n_full * scale))
    s = st.symbols()
    enc_splits = 64 if dist == "laplace" else max(1, min(65536, len(s) // 4096))
    return s, R.encode_with_splits(s, st.n_bits, enc_splits), st.n_bits, what


def _adaptive_input(R, scale: float):
    st = workloads.adaptive_256mib(int((1 << 27) * scale))
    tables = st.tables()
    s, tid = st.draw()
    return s, tid, R.encode_adaptive(s, st.n_bits, tables, tid, max(1, min(65536, len(s) // 4096)))


def configs_block(R, torch, dev, cs, scale: float, steps: int, warmup: int) -> dict:
    """Every other workload beside the batch, each decoded on the device, timed with CUDA events
    and compared with its input on the device: the 1 MiB Laplace stream at 64 / 16 / 1 splits, the
    1 GiB Zipf stream at 148 / 592 / 2368 / 9472 splits, the 256 MiB distribution extremes at 9472
    splits, Recoil against conventional partitioning at 9472, and the adaptive latents at 9472.
    `frac` is (compressed bytes in + symbol bytes out) / time against the measured HBM copy."""
    peak = measured_peaks()["hbm_gbs"]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(6) as ex:                    # the serial encodes run side by side
        futs = {d: ex.submit(_single_input, R, d, scale) for d in ("laplace", "zipf", "skewed", "uniform", "gauss16")}
        fut_ad = ex.submit(_adaptive_input, R, scale)
        single = {d: f.result() for d, f in futs.items()}
        ad = fut_ad.result()
    host_s = time.perf_counter() - t0
    res = {"host_encode_s": round(host_s, 1), "scale": scale, "steps": steps, "warmup": warmup}

    def run(streams, out, ref, warps, extra_in=0, tuned=False, lane_flag=0):
        """Decode `streams` into `out` (one tensor; streams concatenated); GB/s, frac, exactness."""
        if tuned and not warps:
            tws = torch.empty(R.autotune_workspace_size(streams), dtype=torch.uint8, device=dev)
            best, _ = R.autotune(streams, [out.data_ptr()], tws, tws.numel(), cs, steps=3, keep_splits=True)
            warps = best["warps_per_cta"]
            lane_flag = best["flags"] & (R.BATCH_TWO_LANES | R.BATCH_NO_PAIRS)   # lanes and table layout
            del tws
        plan = R.Plan(streams, {"warps_per_cta": warps, "flags": R.BATCH_GRAPH | lane_flag})
        ws = torch.empty(max(256, plan.workspace_size), dtype=torch.uint8, device=dev)
        plan.upload(ws, stream=cs)
        offs, o = [], 0
        for st in streams:
            offs.append(out.data_ptr() + o)
            o += st.info["n_syms"] * st.info["sym_bytes"]
        out.fill_(0xAB)
        ms = time_events(lambda: plan.decode(offs, cs), cs, steps, warmup)
        errors = plan.errors(cs)
        exact = bool(errors == 0 and torch.equal(out, ref))
        nbytes = out.numel()
        words = sum(2 * st.info["n_words"] + 4 * 32 for st in streams)
        t = statistics.mean(ms) * 1e-3
        r = {"gbs": round(nbytes / t / 1e9, 1), "us": round(t * 1e6, 1), "warps_per_cta": plan.warps_per_cta,
             "lanes_per_thread": 2 if lane_flag & R.BATCH_TWO_LANES else 1,
             "splits": sum(st.info["n_entries"] for st in streams),
             "frac": round((nbytes + words + extra_in) / t / 1e9 / peak, 4), "exact": exact}
        del ws
        return r

    with torch.cuda.stream(cs):
        # configuration 1: 1 MiB Laplace, encoded at 64 splits, decoded as 64, 16 and 1
        s, enc, n, what = single["laplace"]
        out = torch.empty(len(s), dtype=torch.uint8, device=dev)
        ref = torch.from_numpy(s).to(dev)
        res["laplace_1mib"] = {"workload": what, **{str(k): run([R.combine_splits(enc, k)], out, ref, 0)
                                                   for k in (64, 16, 1)}}
        # configuration 2: 1 GiB Zipf, 65536 encoded splits combined to the decoder's count
        s, enc, n, what = single["zipf"]
        out = torch.empty(len(s), dtype=torch.uint8, device=dev)
        ref = torch.from_numpy(s).to(dev)
        z = {"workload": what}
        for k in (148, 592, 2368, 9472):
            z[str(k)] = run([R.combine_splits(enc, k)], out, ref, 0)
        z["9472_tuned"] = run([R.combine_splits(enc, 9472)], out, ref, 0, tuned=True)
        res["zipf_1gib"] = z
        # Recoil against the conventional scheme (Sec. 2.3): the same input cut into 9472 partitions
        # under the same quantised model, each with its own final states; same kernel and CTA size
        warps = z["9472_tuned"]["warps_per_cta"]
        lf = R.BATCH_TWO_LANES if z["9472_tuned"]["lanes_per_thread"] == 2 else 0
        freq = R.stream_freq(enc)
        parts = np.array_split(s, 9472)
        with ThreadPoolExecutor(max(1, min(64, os.cpu_count() or 1))) as ex:
            conv = list(ex.map(lambda q: R.encode_with_table(q, n, freq, 1), parts))
        rec = R.combine_splits(enc, 9472)
        res["recoil_vs_conventional"] = {
            "workload": "1 GiB Zipf(1.2) bytes as one stream at 9472 splits vs 9472 independent partitions",
            "recoil": run([rec], out, ref, warps, lane_flag=lf), "conventional": run(conv, out, ref, warps, lane_flag=lf),
            "recoil_size_bytes": int(rec.info["bitstream_bytes"] + R.serialized_size(rec)[1]),
            "conventional_size_bytes": int(sum(c.info["bitstream_bytes"] for c in conv) + 8 * len(conv))}
        del conv, parts
        # configuration 3: the distribution extremes at 9472 splits, CTA size autotuned
        for d in ("skewed", "uniform", "gauss16"):
            s, enc, n, what = single[d]
            out = torch.empty(len(s) * s.itemsize, dtype=torch.uint8, device=dev)
            ref = torch.from_numpy(s.view(np.uint8)).to(dev)
            res[f"{d}_256mib"] = {"workload": what, "9472": run([R.combine_splits(enc, 9472)], out, ref, 0, tuned=True)}
        # adaptive latents (Sec. 3.1) at 9472 splits: table numbers are read too
        s, tid, enc = ad
        out = torch.empty(len(s) * 2, dtype=torch.uint8, device=dev)
        ref = torch.from_numpy(s.view(np.uint8)).to(dev)
        res["adaptive_latents"] = {"workload": "2^27 uint16 latents, 64 Gaussian PDFs over 256 values, n=16",
                                   "9472": run([R.combine_splits(enc, 9472)], out, ref, 0, extra_in=len(s), tuned=True)}
        del out, ref
    res["all_exact"] = all(v.get("exact", True) for blk in res.values() if isinstance(blk, dict)
                           for v in blk.values() if isinstance(v, dict))
    return res


def cpu_split_parallel(R, seconds: float) -> dict:
    """The paper's CPU recipe (Sec. 4.4, one split per core) on the oracle: the first 2^26 symbols of
    the 1 GiB Zipf stream, encoded by the oracle at one split per host thread, decoded by the oracle's
    split decoder with one thread per split, repeated until `seconds` of decode wall time."""
    import oracle
    threads = os.cpu_count() or 1
    st = workloads.zipf_1gib(1 << 26)
    s = st.symbols()
    o = oracle.encode_with_splits(s, st.n_bits, threads)
    out = np.zeros(len(s), dtype=np.uint32)
    wall, reps = 0.0, 0
    with ThreadPoolExecutor(threads) as ex:
        while wall < seconds or reps < 2:
            t = time.perf_counter()
            list(ex.map(lambda k: oracle.decode_thread(o, k, out=out), range(o.K)))
            wall += time.perf_counter() - t
            reps += 1
    assert np.array_equal(out, s)
    return {"value": reps * len(s) / wall / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"first 2^26 symbols of the 1 GiB Zipf stream, {o.K} splits (one per thread), oracle split "
                      f"decoder (plain C -O2), {reps} decodes"}


def run_ours(a):
    import torch
    import paper_2306_12141_b300 as R

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    desc, specs, syms, encoded, streams = make_workload(a, R, rank)
    out_bytes = sum(len(s) * s.itemsize for s in syms)
    in_bytes = sum(2 * st.info["n_words"] + 4 * 32 for st in streams)
    batch = a.workload == "batch"

    outs = [torch.empty(max(1, len(s) * s.itemsize), dtype=torch.uint8, device=dev) for s in syms]
    out_ptrs = [o.data_ptr() for o in outs]
    cs = torch.cuda.Stream(device=dev)
    tuned = None
    if batch and a.warps == 0 and a.split_symbols < 0:
        # the library's autotuner picks warps per CTA and the split size on this batch (untimed)
        tws = torch.empty(R.autotune_workspace_size(streams), dtype=torch.uint8, device=dev)
        with torch.cuda.stream(cs):
            best, tms = R.autotune(streams, out_ptrs, tws, tws.numel(), cs, steps=3)
        lanes = 2 if best["flags"] & R.BATCH_TWO_LANES else 1
        tuned = {"warps_per_cta": best["warps_per_cta"], "split_symbols": best["split_symbols"],
                 "lanes_per_thread": lanes, "ms": round(tms, 4)}
        split_symbols, warps = best["split_symbols"], best["warps_per_cta"]
        del tws
    elif not batch and a.warps == 0:
        # the split count is the workload's; the autotuner picks the CTA size for it (untimed)
        tws = torch.empty(R.autotune_workspace_size(streams), dtype=torch.uint8, device=dev)
        with torch.cuda.stream(cs):
            best, tms = R.autotune(streams, out_ptrs, tws, tws.numel(), cs, steps=3, keep_splits=True)
        lanes = 2 if best["flags"] & R.BATCH_TWO_LANES else 1
        tuned = {"warps_per_cta": best["warps_per_cta"], "split_symbols": 0, "lanes_per_thread": lanes,
                 "ms": round(tms, 4),
                 "candidates": "one or two lanes a thread x the CTA sizes built for each, at the workload's split count"}
        split_symbols, warps = 0, best["warps_per_cta"]
        del tws
    else:
        split_symbols = (65536 if a.split_symbols < 0 else a.split_symbols) if batch else 0
        warps = a.warps or (8 if batch else 0)         # 0: the library picks the CTA size from the split count
        lanes = a.lanes or 1
    lane_flag = R.BATCH_TWO_LANES if lanes == 2 else 0
    opts = {"warps_per_cta": warps, "ctas_per_sm": a.ctas_per_sm, "split_symbols": split_symbols,
            "flags": R.BATCH_GRAPH | lane_flag}
    t_host = time.perf_counter()
    plan = R.Plan(streams, opts)
    plan_ms = (time.perf_counter() - t_host) * 1e3       # host: combining (Sec. 3.3) + descriptors
    opts["warps_per_cta"] = warps = plan.warps_per_cta
    combine_us = None
    if not batch:
        reps = 20
        t_host = time.perf_counter()
        for _ in range(reps):
            R.combine_splits(encoded[0], a.splits)
        combine_us = (time.perf_counter() - t_host) / reps * 1e6
    ws = torch.empty(plan.workspace_size, dtype=torch.uint8, device=dev)

    def barrier():
        if dist:
            torch.distributed.barrier()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            e0.record(cs)
            fn()
            e1.record(cs)
        torch.cuda.synchronize()
        barrier()
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    def exact():
        bad = 0
        for s, o in zip(syms, outs):
            if len(s) and not torch.equal(o[: len(s) * s.itemsize], torch.from_numpy(s.view(np.uint8)).to(dev)):
                bad += 1
        assert bad == 0, f"{bad} streams decoded wrong"

    extra = {}
    with torch.cuda.stream(cs):
        plan.upload(ws, stream=cs)
        decode = lambda: plan.decode(out_ptrs, cs)  # noqa: E731
        with Clocks(local) as clk:
            t_end = time.time() + a.soak                 # keep the step running so the sampler sees load
            while time.time() < t_end:
                decode()
                torch.cuda.synchronize()
            ms = timed(decode, a.steps, a.warmup)
        clocks = clk.summary()
        clocks["note"] = f"sampled every 100 ms over a {a.soak:.1f} s soak of the same step and the timed steps"
        launches = plan.launches
        assert plan.errors(cs) == 0, R.recoil_last_error()
        exact()                                           # the last timed decode reproduces every stream

        if batch and a.per_stream_steps > 0:
            # per-stream baseline: one launch per stream, 128-thread blocks, every encoded split
            base = R.Plan(streams, {"warps_per_cta": 4, "flags": R.BATCH_PER_STREAM})
            bws = torch.empty(base.workspace_size, dtype=torch.uint8, device=dev)
            base.upload(bws, stream=cs)
            base_ms = timed(lambda: base.decode(out_ptrs, cs), a.per_stream_steps, 1)
            assert base.errors(cs) == 0
            exact()
            extra["per_stream"] = {"value": out_bytes / (statistics.mean(base_ms) * 1e-3) / 1e9, "unit": "GB/s",
                                   "ms_per_step": statistics.mean(base_ms), "launches_per_step": base.launches,
                                   "speedup": statistics.mean(base_ms) / statistics.mean(ms),
                                   "shape": "one launch per stream on one CUDA stream, 4-warp CTAs, every "
                                            "encoded split (the paper's launch)"}
            del bws
            if a.rr_streams > 0:
                rr = per_stream_round_robin(R, torch, dev, streams, out_ptrs, warps, split_symbols or 65536,
                                            a.rr_streams, a.per_stream_steps, lane_flag)
                exact()
                rr["value"] = out_bytes / (rr["ms_per_step"] * 1e-3) / 1e9
                rr["unit"] = "GB/s"
                rr["speedup"] = rr["ms_per_step"] / statistics.mean(ms)
                rr["shape"] = (f"one launch per stream at the batch's split size and CTA size, stream i on "
                               f"CUDA stream i mod {a.rr_streams}")
                extra["per_stream"]["round_robin"] = rr

        if not batch and a.sweep:
            sweep = {}
            for k in a.sweep:
                c = R.combine_splits(encoded[0], k)
                sp = R.Plan([c], {"warps_per_cta": a.warps, "flags": R.BATCH_GRAPH | lane_flag})
                sws = torch.empty(sp.workspace_size, dtype=torch.uint8, device=dev)
                sp.upload(sws, stream=cs)
                t = timed(lambda: sp.decode(out_ptrs, cs), 5, 2)
                assert sp.errors(cs) == 0
                sweep[str(c.info["n_entries"])] = round(out_bytes / (statistics.mean(t) * 1e-3) / 1e9, 1)
                del sws
            exact()
            extra["split_sweep_gbs"] = sweep

        if batch and a.serve_requests > 0 and a.serve_rates:
            # continuous-batching serving over the same pool (Poisson arrivals, 20 GiB budget), both
            # arms at every rate, the last rate saturating the device
            extra["serving"] = {"requests_per_rate": a.serve_requests, "budget_gib": 20,
                                "rates_hz": serving_block(R, torch, dev, streams, a.serve_rates, a.serve_requests)}

        if batch and not a.no_configs and world == 1:
            extra["configs"] = configs_block(R, torch, dev, cs, a.configs_scale, 10, 3)

        e2e = None
        if not a.no_e2e:
            # end to end through the public API: the pipeline copies the words in from
            # page-locked host memory, decodes and copies the symbols back, every step
            for st in streams:
                R.stream_pin(st)
            pipe = R.Pipeline(streams, dict(opts, flags=lane_flag), groups=a.e2e_groups)
            wsb, stb = pipe.sizes
            pws = torch.empty(wsb, dtype=torch.uint8, device=dev)
            stage = torch.empty(stb, dtype=torch.uint8, device=dev)
            host = torch.empty(out_bytes + 256 * len(syms), dtype=torch.uint8, pin_memory=True)
            offs = np.concatenate([[0], np.cumsum([max(1, len(s) * s.itemsize) for s in syms])])
            host_ptrs = [host.data_ptr() + int(o) for o in offs[:-1]]
            e_ms = timed(lambda: pipe.run(host_ptrs, pws, wsb, stage, stb, cs), max(3, a.steps // 2), 1)
            assert pipe.errors() == 0
            hv = host.numpy()
            bad = sum(1 for s, o in zip(syms, offs[:-1]) if not np.array_equal(hv[int(o): int(o) + len(s) * s.itemsize],
                                                                                s.view(np.uint8)))
            assert bad == 0, f"{bad} streams wrong end to end"
            h2d = sum(2 * st.info["n_words"] for st in streams)
            # whole job: the slowest rank's time, every rank's bytes (collectives on all ranks)
            e_job_ms, e_job_bytes = aggregate(statistics.mean(e_ms), out_bytes, dev if dist else None)
            _, h2d_job = aggregate(statistics.mean(e_ms), h2d, dev if dist else None)
            e2e = {"value": e_job_bytes / (e_job_ms * 1e-3) / 1e9, "unit": "GB/s",
                   "h2d_bytes_per_step": int(h2d_job), "d2h_bytes_per_step": int(e_job_bytes),
                   "ms_per_step": e_job_ms, "groups": a.e2e_groups,
                   "note": "recoil_pipeline_run: H2D of words (+ descriptors, tables), decode, D2H of the symbols, "
                           "overlapped across stream groups (a stream larger than its share is cut into runs "
                           "of splits)"}
            del pws, stage

    mean_ms, total_bytes = aggregate(statistics.mean(ms), out_bytes, dev if dist else None)
    value = total_bytes / (mean_ms * 1e-3) / 1e9
    peaks = measured_peaks()
    achieved = (out_bytes + in_bytes) / (mean_ms * 1e-3) / 1e9
    tkey = (f"batch w{opts['warps_per_cta']} s{split_symbols} l{lanes}" if batch
            else f"{a.dist} w{opts['warps_per_cta']} k{a.splits} l{lanes}")
    traffic = recorded_traffic(tkey) if a.scale == 1.0 and a.streams == workloads.BATCH_STREAMS else None
    dtype, kernel = kernel_of(plan)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": desc, "symbols_bytes": out_bytes, "compressed_bytes": in_bytes,
                   "splits": sum(st.info["n_entries"] for st in plan.streams) if not batch else None,
                   "split_symbols": split_symbols, "warps_per_cta": opts["warps_per_cta"],
                   "lanes_per_thread": lanes,
                   "autotuned": tuned,
                   "host_plan_ms": round(plan_ms, 3),
                   "host_combine_us": round(combine_us, 1) if combine_us is not None else None,
                   "parallelism": f"weak x{world}", "l2": "inputs larger than L2 (no flush)",
                   "scale": a.scale},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peaks["source"],
                     "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                     "issue": (issue_rate(tkey, mean_ms, dev, clocks)
                               if a.scale == 1.0 and a.streams == workloads.BATCH_STREAMS else None),
                     "kernel": kernel, "bytes": "compressed words in + symbols out"},
        "clocks": clocks,
        "gpu_launches": launches * a.steps * world,          # every rank's launches in the timed steps
        "e2e": e2e,
    }
    line.update(extra)
    if rank == 0 and not a.no_cpu:
        if batch:
            line["cpu_baseline"] = cpu_baseline(specs, syms, a.cpu_seconds)
            line["cpu_baseline"]["split_parallel"] = cpu_split_parallel(R, max(2.0, a.cpu_seconds / 2))
        else:                                             # the oracle sees the stream in 16 Mi-symbol pieces
            piece = 1 << 24
            parts = [syms[0][i:i + piece] for i in range(0, min(len(syms[0]), 64 * piece), piece)]
            line["cpu_baseline"] = cpu_baseline([specs[0]] * len(parts), parts, a.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


def run_serve(a):
    """--workload serve: the serving sweep (rates 2k-50k/s, 20000 requests each) over the batch pool."""
    import torch
    import paper_2306_12141_b300 as R
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    specs, syms, streams = build_batch(R, a.streams, a.scale)
    n_req = a.serve_requests if a.serve_requests > 0 else 20000
    with Clocks(dev.index) as clk:
        sweep = serving_block(R, torch, dev, streams, a.serve_rates, n_req)
    rated = [k for k in sweep if k != "saturating"]
    top = sweep[rated[-1] if rated else "saturating"]     # the highest Poisson rate run (else the saturating load)
    line = {"metric": METRIC, "value": top["recoil"]["decoded_gbs"], "unit": "GB/s", "n_gpus": 1,
            "steps": len(a.serve_rates), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals over the " + BATCH_WORKLOAD + ", 20 GiB budget",
                       "requests_per_rate": n_req},
            "latency": {r: {"p50_ms": v["recoil"]["p50_ms"], "p99_ms": v["recoil"]["p99_ms"]} for r, v in sweep.items()},
            "serving": sweep, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.workload == "zipf":
        args.workload, args.dist = "single", "zipf"
    if args.workload == "single" and args.dist == "laplace" and args.splits == 9472:
        args.splits = 64
    if args.workload == "single" and args.dist == "laplace":
        args.sweep = [k for k in args.sweep if k <= 64] or [64, 16, 1]
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "conventional":
        run_conventional(args)
    elif args.workload == "adaptive":
        run_adaptive(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)
