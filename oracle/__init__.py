"""Recoil oracle -- TEST INFRASTRUCTURE ONLY.

Python face of ``recoil_oracle.c``: a plain, slow, single-threaded CPU
restatement of the Recoil method (rANS Eqs. 1-4, interleaving Sec. 2.2,
Lemma 3.1, split metadata and the three decoding phases of Sec. 4.1, the
heuristic of Def. 4.1 / Eq. 7, combining of Sec. 3.3, adaptive coding keyed
by the symbol index of Sec. 3.1). Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it. It shares no code with the CUDA library and imports nothing from it.

Every function here is pinned by ``tests/test_oracle_*.py`` against facts the
paper or the mathematics fixes (lossless round trip, brute force over tiny
alphabets, the Sec. 4.1 walkthrough, closed forms, entropy bounds, the
paper's Table 4 sizes). The quantiser is a reading of the paper, which gives
no procedure: its exact output is "parity unpinned" against the paper and
pinned only by hand cases and invariants. The heuristic comes in the printed
form (T = ceil(N/M)) and in the remaining-symbols reading of T; both are pinned
by hand-derived split words and the exhaustive argmin of Eq. 7.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "recoil_oracle.c")
LIB = os.path.join(HERE, "_recoil_oracle.so")

# Recommended parameters of the paper (Sec. 4.4, Table 3).
W_DEFAULT, LGL_DEFAULT, B_DEFAULT = 32, 16, 16

TR_SKIP, TR_INIT, TR_DECODE, TR_STORE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vectorisation tricks needed)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                               SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        p = C.c_void_p
        i64, i32 = C.c_int64, C.c_int
        L.oracle_params_check.argtypes = [i32, i32, i32, i32]
        L.oracle_quantize.argtypes = [p, i32, i32, p]
        L.oracle_encode.argtypes = [p, i64, p, i32, i32, i32, i32, i32, p, i64, p, p, p]
        L.oracle_encode.restype = i64
        L.oracle_decode_serial.argtypes = [p, i64, p, i64, p, i32, i32, i32, i32, i32, p, p, p, p, p]
        L.oracle_scan.argtypes = [p, p, i64, i32, p, p, p]
        for name in ("oracle_heuristic_eq7", "oracle_heuristic_remaining"):
            getattr(L, name).argtypes = [p, p, i64, i64, i32, i64, p]
            getattr(L, name).restype = i64
        L.oracle_combine.argtypes = [i64, i64, p, i64, p]
        L.oracle_combine.restype = i64
        L.oracle_decode_thread.argtypes = [p, i64, p, i64, p, i32, i32, i32, i32, i32,
                                           i32, p, p, i64, i64, i64, p, p, p]
        L.oracle_decode_splits.argtypes = [p, i64, p, i64, p, i32, i32, i32, i32, i32,
                                           i64, p, p, p, p]
        L.oracle_encode_adaptive.argtypes = [p, i64, p, i32, i32, p, i32, i32, i32, i32, p, i64, p, p, p]
        L.oracle_encode_adaptive.restype = i64
        L.oracle_decode_serial_adaptive.argtypes = [p, i64, p, i64, p, i32, i32, p, i32, i32, i32, i32,
                                                    p, p, p]
        L.oracle_decode_splits_adaptive.argtypes = [p, i64, p, i64, p, i32, i32, p, i32, i32, i32, i32,
                                                    i64, p, p, p, p]
        L.oracle_decode_thread_adaptive.argtypes = [p, i64, p, i64, p, i32, i32, p, i32, i32, i32, i32,
                                                    i32, p, p, i64, i64, i64, p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    """Pointer argument for a C call; it holds a reference to the array, so a
    temporary (e.g. a dtype conversion) lives until the call returns."""
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# ------------------------------------------------------------------- primitives
def quantize(counts, n: int) -> np.ndarray:
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    f = np.zeros(len(c), dtype=np.uint32)
    rc = lib().oracle_quantize(_ptr(c), len(c), n, _ptr(f))
    if rc:
        raise ValueError(f"oracle_quantize failed ({rc})")
    return f


def encode(sym, f, n: int, W: int = W_DEFAULT, lgL: int = LGL_DEFAULT, b: int = B_DEFAULT):
    """Interleaved encode (Eqs. 1, 3). Returns (words u16, final u32[W], ev_sym i64, ev_y u32)."""
    s = _u32(sym)
    f = _u32(f)
    N = len(s)
    cap = N + W + 16          # b >= n: at most one word per coded symbol (Sec. 4.4)
    B = np.zeros(cap, dtype=np.uint16)
    xf = np.zeros(W, dtype=np.uint32)
    ev_sym = np.zeros(cap, dtype=np.int64)
    ev_y = np.zeros(cap, dtype=np.uint32)
    nw = lib().oracle_encode(_ptr(s), N, _ptr(f), len(f), W, n, lgL, b,
                             _ptr(B), cap, _ptr(xf), _ptr(ev_sym), _ptr(ev_y))
    if nw < 0:
        raise ValueError(f"oracle_encode failed ({nw})")
    return B[:nw].copy(), xf, ev_sym[:nw].copy(), ev_y[:nw].copy()


def decode_serial(B, xf, N: int, f, n: int, W: int = W_DEFAULT, lgL: int = LGL_DEFAULT,
                  b: int = B_DEFAULT, trace: bool = False):
    """Serial interleaved decode (Eqs. 2, 4). Returns (out, end_x, end_p[, tr_x, tr_p])."""
    B = np.ascontiguousarray(B, dtype=np.uint16)
    xf = _u32(xf)
    f = _u32(f)
    out = np.zeros(N, dtype=np.uint32)
    end_x = np.zeros(W, dtype=np.uint32)
    end_p = np.zeros(1, dtype=np.int64)
    tr_x = np.zeros(N, dtype=np.uint32) if trace else None
    tr_p = np.zeros(N, dtype=np.int64) if trace else None
    rc = lib().oracle_decode_serial(_ptr(B), len(B), _ptr(xf), N, _ptr(f), len(f), W, n, lgL, b,
                                    _ptr(out), _ptr(end_x), _ptr(end_p), _ptr(tr_x), _ptr(tr_p))
    if rc:
        raise ValueError(f"oracle_decode_serial failed ({rc})")
    if trace:
        return out, end_x, int(end_p[0]), tr_x, tr_p
    return out, end_x, int(end_p[0])


def encode_adaptive(sym, tid, tables, n: int, W: int = W_DEFAULT, lgL: int = LGL_DEFAULT,
                    b: int = B_DEFAULT):
    """Encode with PDF row tid[i] of tables (T x A) for symbol i (Sec. 3.1). Same returns as encode."""
    s = _u32(sym)
    t = _u32(tid)
    tab = np.ascontiguousarray(np.atleast_2d(tables), dtype=np.uint32)
    N = len(s)
    if len(t) != N:
        raise ValueError("one table index per symbol")
    cap = N + W + 16
    B = np.zeros(cap, dtype=np.uint16)
    xf = np.zeros(W, dtype=np.uint32)
    ev_sym = np.zeros(cap, dtype=np.int64)
    ev_y = np.zeros(cap, dtype=np.uint32)
    nw = lib().oracle_encode_adaptive(_ptr(s), N, _ptr(tab), tab.shape[0], tab.shape[1], _ptr(t), W, n, lgL, b,
                                      _ptr(B), cap, _ptr(xf), _ptr(ev_sym), _ptr(ev_y))
    if nw < 0:
        raise ValueError(f"oracle_encode_adaptive failed ({nw})")
    return B[:nw].copy(), xf, ev_sym[:nw].copy(), ev_y[:nw].copy()


def decode_serial_adaptive(B, xf, tid, tables, n: int, W: int = W_DEFAULT, lgL: int = LGL_DEFAULT,
                           b: int = B_DEFAULT):
    """Serial decode with the adaptive model. Returns (out, end_x, end_p)."""
    B = np.ascontiguousarray(B, dtype=np.uint16)
    t = _u32(tid)
    tab = np.ascontiguousarray(np.atleast_2d(tables), dtype=np.uint32)
    N = len(t)
    out = np.zeros(N, dtype=np.uint32)
    end_x = np.zeros(W, dtype=np.uint32)
    end_p = np.zeros(1, dtype=np.int64)
    rc = lib().oracle_decode_serial_adaptive(_ptr(B), len(B), _ptr(_u32(xf)), N, _ptr(tab), tab.shape[0],
                                             tab.shape[1], _ptr(t), W, n, lgL, b, _ptr(out), _ptr(end_x),
                                             _ptr(end_p))
    if rc:
        raise ValueError(f"oracle_decode_serial_adaptive failed ({rc})")
    return out, end_x, int(end_p[0])


def scan(ev_sym, ev_y, q: int, W: int = W_DEFAULT):
    """Backward scan from word q (Sec. 4.1). Returns (usable, idx[W], y[W], word[W])."""
    idx = np.zeros(W, dtype=np.int64)
    y = np.zeros(W, dtype=np.uint32)
    wp = np.zeros(W, dtype=np.int64)
    ok = lib().oracle_scan(_ptr(_i64(ev_sym)), _ptr(_u32(ev_y)), q, W, _ptr(idx), _ptr(y), _ptr(wp))
    return bool(ok), idx, y, wp


RULES = ("remaining", "eq7")


def heuristic(ev_sym, ev_y, N: int, M: int, W: int = W_DEFAULT, rule: str = "remaining") -> np.ndarray:
    """Split words chosen by Def. 4.1 / Eq. 7 for M splits (at most M-1 words).

    rule "eq7": T = ceil(N / M) for every split, as printed; rule "remaining":
    T = ceil((N - lo) / (M - k)) over the symbols left (the library's default)."""
    if rule not in RULES:
        raise ValueError(f"rule must be one of {RULES}")
    fn = lib().oracle_heuristic_eq7 if rule == "eq7" else lib().oracle_heuristic_remaining
    q = np.zeros(max(1, M), dtype=np.int64)
    k = fn(_ptr(_i64(ev_sym)), _ptr(_u32(ev_y)), len(ev_sym), N, W, M, _ptr(q))
    if k < 0:
        raise ValueError("oracle heuristic failed")
    return q[:k].copy()


def combine_keep(m, N: int, Mp: int) -> np.ndarray:
    """Kept entry numbers when combining to Mp (m: owned ends of the K-1 regular entries)."""
    mm = _i64(np.asarray(m, dtype=np.int64))
    K = len(mm) + 1
    keep = np.zeros(max(1, min(K, Mp)), dtype=np.int64)
    k = lib().oracle_combine(K, Mp, _ptr(mm) if len(mm) else None, N, _ptr(keep))
    if k < 0:
        raise ValueError("oracle_combine failed")
    return keep[:k].copy()


# -------------------------------------------------------------- stream objects
@dataclass
class OracleStream:
    """Everything the oracle's encoder produced for one input."""
    N: int
    n: int
    W: int
    lgL: int
    b: int
    f: np.ndarray          # quantised PDF (adaptive: T x A, one row per table)
    words: np.ndarray      # u16 bitstream
    final: np.ndarray      # u32[W] final states
    ev_sym: np.ndarray     # per word: symbol index whose coding triggered it
    ev_y: np.ndarray       # per word: state right after the renormalisation
    q: np.ndarray          # split words of the regular entries (increasing)
    idx: np.ndarray        # K x W recorded symbol indices (last row: final entry, unused)
    y: np.ndarray          # K x W states (last row: final states)
    tid: np.ndarray | None = None   # adaptive model: PDF row of every symbol index (Sec. 3.1)

    @property
    def K(self) -> int:
        return len(self.q) + 1


def entries_for(ev_sym, ev_y, qs, W: int):
    """Rows (idx, y) of the entries at words qs, plus a last row for the final entry."""
    K = len(qs) + 1
    idx = np.zeros((K, W), dtype=np.int64)
    y = np.zeros((K, W), dtype=np.uint32)
    for k, q in enumerate(qs):
        ok, idx[k], y[k], _ = scan(ev_sym, ev_y, int(q), W)
        if not ok:
            raise ValueError(f"word {q} is not a usable split point")
    return idx, y


def encode_with_splits(sym, n: int, M: int, W: int = W_DEFAULT, lgL: int = LGL_DEFAULT,
                       b: int = B_DEFAULT, alphabet: int | None = None, rule: str = "remaining") -> OracleStream:
    """Quantise from the symbol counts, encode, and place M splits by the heuristic (`rule`: T of Eq. 7)."""
    s = _u32(sym)
    A = alphabet if alphabet is not None else (int(s.max()) + 1 if len(s) else 1)
    counts = np.bincount(s, minlength=A).astype(np.uint64)
    f = quantize(counts, n)
    words, final, ev_sym, ev_y = encode(s, f, n, W, lgL, b)
    qs = heuristic(ev_sym, ev_y, len(s), M, W, rule)
    idx, y = entries_for(ev_sym, ev_y, qs, W)
    y[-1] = final
    return OracleStream(len(s), n, W, lgL, b, f, words, final, ev_sym, ev_y, qs, idx, y)


def encode_adaptive_with_splits(sym, tid, tables, n: int, M: int, W: int = W_DEFAULT,
                                lgL: int = LGL_DEFAULT, b: int = B_DEFAULT, rule: str = "remaining") -> OracleStream:
    """Adaptive encode (PDF row tid[i] for symbol i) and M splits placed by the heuristic."""
    s = _u32(sym)
    tab = np.ascontiguousarray(np.atleast_2d(tables), dtype=np.uint32)
    words, final, ev_sym, ev_y = encode_adaptive(s, tid, tab, n, W, lgL, b)
    qs = heuristic(ev_sym, ev_y, len(s), M, W, rule)
    idx, y = entries_for(ev_sym, ev_y, qs, W)
    y[-1] = final
    return OracleStream(len(s), n, W, lgL, b, tab, words, final, ev_sym, ev_y, qs, idx, y, _u32(tid))


def combined(st: OracleStream, Mp: int) -> OracleStream:
    """The same stream with only Mp entries kept (the final entry always stays)."""
    keep = combine_keep(st.idx[:-1].min(axis=1) if st.K > 1 else [], st.N, Mp)
    regular = [k for k in keep if k < st.K - 1]
    return OracleStream(st.N, st.n, st.W, st.lgL, st.b, st.f, st.words, st.final, st.ev_sym,
                        st.ev_y, st.q[regular], np.vstack([st.idx[regular], st.idx[-1:]]),
                        np.vstack([st.y[regular], st.y[-1:]]), st.tid)


def decode_splits(st: OracleStream) -> np.ndarray:
    """Split decode of every entry of st, threads run one after another."""
    out = np.zeros(st.N, dtype=np.uint32)
    idx = _i64(st.idx)
    y = _u32(st.y)
    q = _i64(np.concatenate([st.q, [0]]))
    if st.tid is not None:
        tab = np.ascontiguousarray(st.f, dtype=np.uint32)
        rc = lib().oracle_decode_splits_adaptive(_ptr(st.words), len(st.words), _ptr(st.final), st.N,
                                                 _ptr(tab), tab.shape[0], tab.shape[1], _ptr(_u32(st.tid)),
                                                 st.W, st.n, st.lgL, st.b, st.K, _ptr(idx), _ptr(y), _ptr(q),
                                                 _ptr(out))
    else:
        rc = lib().oracle_decode_splits(_ptr(st.words), len(st.words), _ptr(st.final), st.N,
                                        _ptr(_u32(st.f)), len(st.f), st.W, st.n, st.lgL, st.b,
                                        st.K, _ptr(idx), _ptr(y), _ptr(q), _ptr(out))
    if rc:
        raise ValueError(f"oracle_decode_splits failed ({rc})")
    return out


def owned_range(st: OracleStream, k: int) -> tuple[int, int]:
    """[lo, hi] owned by thread k (hi = lo - 1 when empty)."""
    lo = 0 if k == 0 else int(st.idx[k - 1].min())
    hi = st.N - 1 if k == st.K - 1 else int(st.idx[k].min()) - 1
    return lo, hi


def decode_thread(st: OracleStream, k: int, trace: bool = False, out: np.ndarray | None = None):
    """Run split-decoder thread k alone. Returns out (and the trace arrays if asked)."""
    lo, hi = owned_range(st, k)
    is_final = int(k == st.K - 1)
    if out is None:
        out = np.zeros(st.N, dtype=np.uint32)
    start = st.N - 1 if is_final else int(st.idx[k].max()) + st.W
    tr = np.full(max(1, start + 1), -1, dtype=np.int8) if trace else None
    tw = np.full(max(1, start + 1), -1, dtype=np.int64) if trace else None
    idx = _i64(st.idx[k])
    y = _u32(st.y[k])
    q = 0 if is_final else int(st.q[k])
    if st.tid is not None:
        if trace:
            raise ValueError("traces are kept for the static model only")
        tab = np.ascontiguousarray(st.f, dtype=np.uint32)
        rc = lib().oracle_decode_thread_adaptive(_ptr(st.words), len(st.words), _ptr(st.final), st.N,
                                                 _ptr(tab), tab.shape[0], tab.shape[1], _ptr(_u32(st.tid)),
                                                 st.W, st.n, st.lgL, st.b, is_final, _ptr(idx), _ptr(y), q,
                                                 lo, hi, _ptr(out))
        if rc:
            raise ValueError(f"oracle_decode_thread_adaptive failed ({rc})")
        return out
    rc = lib().oracle_decode_thread(_ptr(st.words), len(st.words), _ptr(st.final), st.N,
                                    _ptr(_u32(st.f)), len(st.f), st.W, st.n, st.lgL, st.b,
                                    is_final, _ptr(idx), _ptr(y), q, lo, hi, _ptr(out),
                                    _ptr(tr), _ptr(tw))
    if rc:
        raise ValueError(f"oracle_decode_thread failed ({rc})")
    return (out, tr, tw) if trace else out
