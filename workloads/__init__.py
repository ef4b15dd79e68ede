"""Seeded synthetic inputs for the Recoil decoder and its oracle.

This module only draws symbols. It holds none of the coding arithmetic: no
quantiser, no encoder, no decoder. Both the oracle (tests, CPU baseline) and
the CUDA library path take their inputs from here, so the two sides see the
same bytes for the same seed.

Every draw is a numpy ``Generator(PCG64)`` seeded through ``SeedSequence``.
Large arrays are drawn in 16 Mi-symbol chunks, each chunk from its own
spawned child seed, so the result does not depend on the thread count.

A discrete distribution is sampled through an inverse-CDF table of 2^20
cells: each symbol receives round(P * 2^20) cells (largest remainders break
ties), and a uniform 20-bit integer picks a cell. The sampled law is the
target law rounded to multiples of 2^-20, which is far below anything the
coder can see at these sizes.

Workloads (the paper's datasets are not available; these stand in for them):

* ``laplace``: clip(rint(Laplace(mean, scale)), 0, 255), 8-bit symbols.
* ``zipf``: P(k) proportional to (k+1)^-s over k = 0..255.
* ``skewed``: P(0) = 0.95, every other byte 0.05/255.
* ``uniform``: uniform bytes.
* ``gauss16``: clip(rint(Normal(mean, sigma)), 0, 4095) as uint16.
* ``expbytes``: min(255, floor(Exp(scale = 256/lambda))), the reading used
  here for the paper's ``rand_lambda`` files (Sec. 5.1, Table 4).
* ``adaptive``: latents of a hyperprior image codec (Sec. 3.1, 5.1): symbol i
  has its own Gaussian scale, chosen by a per-index table number t_i, and is
  clip(rint(A/2 + sigma_{t_i} Z), 0, A-1). The model (one quantised PDF per
  scale) is an input too: it is built here from the Gaussian by the
  largest-remainder rule, every symbol keeping at least one slot.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

CHUNK = 1 << 24          # symbols per independently seeded chunk
TABLE_BITS = 20          # inverse-CDF table resolution


# --------------------------------------------------------------------------- pmfs
def laplace_pmf(mean: float, scale: float, k: int = 256) -> np.ndarray:
    """P(clip(rint(X), 0, k-1) = v) for X ~ Laplace(mean, scale)."""
    def cdf(x):
        x = np.asarray(x, dtype=np.float64)
        z = (x - mean) / scale
        return np.where(z < 0, 0.5 * np.exp(np.minimum(z, 0)), 1 - 0.5 * np.exp(-np.maximum(z, 0)))
    edges = np.arange(k + 1, dtype=np.float64) - 0.5
    c = cdf(edges)
    c[0], c[-1] = 0.0, 1.0
    return np.diff(c)


def gauss_pmf(mean: float, sigma: float, k: int) -> np.ndarray:
    """P(clip(rint(X), 0, k-1) = v) for X ~ Normal(mean, sigma)."""
    from scipy.special import ndtr
    edges = (np.arange(k + 1, dtype=np.float64) - 0.5 - mean) / sigma
    c = ndtr(edges)
    c[0], c[-1] = 0.0, 1.0
    return np.diff(c)


def zipf_pmf(s: float, k: int = 256) -> np.ndarray:
    w = (np.arange(k, dtype=np.float64) + 1.0) ** (-s)
    return w / w.sum()


def skewed_pmf(p0: float = 0.95, k: int = 256) -> np.ndarray:
    p = np.full(k, (1.0 - p0) / (k - 1), dtype=np.float64)
    p[0] = p0
    return p


def expbytes_pmf(lam: float) -> np.ndarray:
    """min(255, floor(E)) for E ~ Exp(scale = 256/lam)."""
    scale = 256.0 / lam
    k = np.arange(256, dtype=np.float64)
    p = np.exp(-k / scale) * (1.0 - math.exp(-1.0 / scale))
    p[255] = math.exp(-255.0 / scale)
    return p


def uniform_pmf(k: int = 256) -> np.ndarray:
    return np.full(k, 1.0 / k)


# ------------------------------------------------------------------------- sampler
def cell_table(pmf: np.ndarray, bits: int = TABLE_BITS) -> np.ndarray:
    """Inverse-CDF table: symbol v owns round(P(v) * 2^bits) consecutive cells."""
    pmf = np.asarray(pmf, dtype=np.float64)
    pmf = pmf / pmf.sum()
    cells = 1 << bits
    raw = pmf * cells
    cnt = np.floor(raw).astype(np.int64)
    short = cells - int(cnt.sum())
    if short > 0:
        order = np.argsort(-(raw - cnt), kind="stable")
        cnt[order[:short]] += 1
    dtype = np.uint8 if len(pmf) <= 256 else np.uint16
    return np.repeat(np.arange(len(pmf), dtype=dtype), cnt)


def _chunks(n: int):
    return [(s, min(CHUNK, n - s)) for s in range(0, n, CHUNK)]


def _seedseq(seed) -> np.random.SeedSequence:
    """A fresh SeedSequence for seed (copied, since spawning advances a sequence's counter)."""
    if isinstance(seed, np.random.SeedSequence):
        return np.random.SeedSequence(seed.entropy, spawn_key=seed.spawn_key, pool_size=seed.pool_size)
    return np.random.SeedSequence(seed)


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def sample_pmf(pmf: np.ndarray, n: int, seed, threads: int | None = None) -> np.ndarray:
    """n i.i.d. draws from pmf, deterministic in (pmf, n, seed)."""
    table = cell_table(pmf)
    out = np.empty(n, dtype=table.dtype)
    parts = _chunks(n)
    kids = _seedseq(seed).spawn(max(1, len(parts)))

    def fill(k):
        s, m = parts[k]
        g = np.random.Generator(np.random.PCG64(kids[k]))
        idx = g.integers(0, 1 << TABLE_BITS, size=m, dtype=np.uint32)
        np.take(table, idx, out=out[s:s + m])

    if len(parts) <= 1:
        for k in range(len(parts)):
            fill(k)
    else:
        with ThreadPoolExecutor(threads or _threads()) as ex:
            list(ex.map(fill, range(len(parts))))
    return out


def sample_uniform(n: int, seed, k: int = 256, threads: int | None = None) -> np.ndarray:
    dtype = np.uint8 if k <= 256 else np.uint16
    out = np.empty(n, dtype=dtype)
    parts = _chunks(n)
    kids = _seedseq(seed).spawn(max(1, len(parts)))

    def fill(c):
        s, m = parts[c]
        g = np.random.Generator(np.random.PCG64(kids[c]))
        out[s:s + m] = g.integers(0, k, size=m, dtype=dtype)

    with ThreadPoolExecutor(threads or _threads()) as ex:
        list(ex.map(fill, range(len(parts))))
    return out


# ------------------------------------------------------------------------ workloads
@dataclass
class Stream:
    """One synthetic symbol stream and the coding parameters it is used with."""
    name: str
    n_syms: int
    sym_bytes: int
    n_bits: int
    dist: str
    params: dict = field(default_factory=dict)
    seed: object = 0

    def pmf(self) -> np.ndarray:
        d, p = self.dist, self.params
        if d == "laplace":
            return laplace_pmf(p["mean"], p["scale"])
        if d == "zipf":
            return zipf_pmf(p["s"])
        if d == "skewed":
            return skewed_pmf(p.get("p0", 0.95))
        if d == "uniform":
            return uniform_pmf(256 if self.sym_bytes == 1 else p.get("k", 65536))
        if d == "gauss16":
            return gauss_pmf(p["mean"], p["sigma"], p.get("k", 4096))
        if d == "expbytes":
            return expbytes_pmf(p["lam"])
        raise ValueError(d)

    def symbols(self, threads: int | None = None) -> np.ndarray:
        if self.dist == "uniform":
            k = 256 if self.sym_bytes == 1 else self.params.get("k", 65536)
            return sample_uniform(self.n_syms, self.seed, k, threads)
        return sample_pmf(self.pmf(), self.n_syms, self.seed, threads)


def laplace_1mib(n_syms: int = 1 << 20) -> Stream:
    """1 MiB of Laplace(128, 8) bytes, n = 11; encoded with 64 splits."""
    return Stream("laplace_1MiB_n11", n_syms, 1, 11, "laplace", {"mean": 128.0, "scale": 8.0}, seed=1)


def zipf_1gib(n_syms: int = 1 << 30) -> Stream:
    """1 GiB of Zipf(1.2) bytes over 256 symbols, n = 12; encoded with 65536 splits."""
    return Stream("zipf_1GiB_n12", n_syms, 1, 12, "zipf", {"s": 1.2}, seed=2)


def skewed_256mib(n_syms: int = 1 << 28) -> Stream:
    return Stream("skewed_256MiB_n12", n_syms, 1, 12, "skewed", {"p0": 0.95}, seed=3)


def uniform_256mib(n_syms: int = 1 << 28) -> Stream:
    return Stream("uniform_256MiB_n12", n_syms, 1, 12, "uniform", {}, seed=4)


def gauss16_256mib(n_syms: int = 1 << 27) -> Stream:
    """2^27 uint16 symbols (256 MiB), Normal(2048, 200) clipped to 0..4095, n = 15."""
    return Stream("gauss16_256MiB_n15", n_syms, 2, 15, "gauss16",
                  {"mean": 2048.0, "sigma": 200.0, "k": 4096}, seed=5)


def expbytes_10mb(lam: float, n_syms: int = 10_000_000, n_bits: int = 16) -> Stream:
    return Stream(f"rand_{int(lam)}", n_syms, 1, n_bits, "expbytes", {"lam": float(lam)},
                  seed=int(1000 + lam))


# Batch of uneven streams: lognormal sizes (median 256 KiB, sigma 1.5, clipped to
# 4 KiB .. 64 MiB), Laplace(128, b) bytes with b ~ U(2, 64) per stream, n = 12.
BATCH_STREAMS = 4096
BATCH_MEDIAN = 1 << 18
BATCH_SIGMA = 1.5
BATCH_MIN, BATCH_MAX = 1 << 12, 1 << 26
SPLIT_GRAIN = 4096       # one encoded split entry per 4096 symbols, at most 9472


def batch_specs(count: int = BATCH_STREAMS, seed: int = 6, scale_sizes: float = 1.0) -> list[Stream]:
    """Stream specs of the uneven batch; ``scale_sizes`` < 1 shrinks every size (tests)."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    sizes = np.exp(g.normal(math.log(BATCH_MEDIAN), BATCH_SIGMA, size=count))
    sizes = np.clip(np.rint(sizes), BATCH_MIN, BATCH_MAX).astype(np.int64)
    scales = g.uniform(2.0, 64.0, size=count)
    kids = np.random.SeedSequence(seed).spawn(count)
    out = []
    for k in range(count):
        n = max(1, int(sizes[k] * scale_sizes))
        out.append(Stream(f"batch{k:04d}", n, 1, 12, "laplace",
                          {"mean": 128.0, "scale": float(scales[k])}, seed=kids[k]))
    return out


def batch_split_count(n_syms: int) -> int:
    """Split entries a batch stream is encoded with: clamp(floor(N / 4096), 1, 9472)."""
    return int(min(max(n_syms // SPLIT_GRAIN, 1), 9472))


def batch_symbols(specs: list[Stream], threads: int | None = None) -> list[np.ndarray]:
    """Draw every stream of a batch; small streams are drawn in parallel."""
    with ThreadPoolExecutor(threads or _threads()) as ex:
        return list(ex.map(lambda s: s.symbols(threads=1), specs))


# ------------------------------------------------------------------ adaptive model
SCALE_MIN, SCALE_MAX = 0.11, 256.0      # Gaussian scales of the table set, log-spaced


def scale_table(n_tables: int) -> np.ndarray:
    return np.exp(np.linspace(math.log(SCALE_MIN), math.log(SCALE_MAX), n_tables))


def gauss_freq_row(sigma: float, alphabet: int, n_bits: int) -> np.ndarray:
    """Quantised PDF of clip(rint(A/2 + sigma Z), 0, A-1): 1 + floor(P * (2^n - A)) per symbol,
    the slots left over going to the largest remainders (ties: smaller symbol)."""
    pmf = gauss_pmf(alphabet // 2, sigma, alphabet)
    spare = (1 << n_bits) - alphabet
    if spare < 0:
        raise ValueError("alphabet larger than 2^n")
    raw = pmf * spare
    f = 1 + np.floor(raw).astype(np.int64)
    short = (1 << n_bits) - int(f.sum())
    order = np.argsort(-(raw - np.floor(raw)), kind="stable")
    f[order[:short]] += 1
    return f.astype(np.uint32)


@dataclass
class AdaptiveStream:
    """Symbols with a per-index distribution (adaptive coding keyed by the symbol index)."""
    name: str
    n_syms: int
    n_bits: int = 16
    sym_bytes: int = 2
    n_tables: int = 64
    alphabet: int = 256
    seed: int = 8
    index_mean: float = 20.0       # table numbers t_i ~ clip(rint(Normal(mean, sd)), 0, T-1)
    index_sd: float = 12.0

    def tables(self) -> np.ndarray:
        """n_tables x alphabet quantised frequencies, each row summing to 2^n."""
        return np.stack([gauss_freq_row(float(sg), self.alphabet, self.n_bits)
                         for sg in scale_table(self.n_tables)])

    def draw(self, threads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
        """(symbols, table numbers): deterministic in the seed, chunked like every other draw."""
        n = self.n_syms
        sym = np.empty(n, dtype=np.uint8 if self.sym_bytes == 1 else np.uint16)
        tid = np.empty(n, dtype=np.uint8)
        scales = scale_table(self.n_tables)
        parts = _chunks(n)
        kids = _seedseq(self.seed).spawn(max(1, len(parts)))

        def fill(k):
            s, m = parts[k]
            g = np.random.Generator(np.random.PCG64(kids[k]))
            t = np.clip(np.rint(g.normal(self.index_mean, self.index_sd, size=m)), 0, self.n_tables - 1)
            tid[s:s + m] = t.astype(np.uint8)
            v = np.rint(self.alphabet // 2 + scales[tid[s:s + m]] * g.standard_normal(size=m))
            sym[s:s + m] = np.clip(v, 0, self.alphabet - 1).astype(sym.dtype)

        if len(parts) <= 1:
            for k in range(len(parts)):
                fill(k)
        else:
            with ThreadPoolExecutor(threads or _threads()) as ex:
                list(ex.map(fill, range(len(parts))))
        return sym, tid


def adaptive_256mib(n_syms: int = 1 << 27, alphabet: int = 256, n_tables: int = 64) -> AdaptiveStream:
    """2^27 uint16 latents (256 MiB decoded), 64 Gaussian scale tables over 256 values, n = 16
    (other alphabets and table counts for the wide-alphabet variant)."""
    return AdaptiveStream("adaptive", n_syms, alphabet=alphabet, n_tables=n_tables)


def poisson_arrivals(rate_hz: float, count: int, seed: int = 7) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, int(rate_hz)])))
    return np.cumsum(g.exponential(1.0 / rate_hz, size=count))


def request_picks(pool: int, count: int, seed: int = 7) -> np.ndarray:
    """Which pool stream each serving request decodes (uniform over the pool)."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 1])))
    return g.integers(0, pool, size=count, dtype=np.int64)
