"""Python binding of the B300 Recoil decoder (``librecoil.so``, C-ABI in include/recoil.h).

Argument marshalling only: every step runs in the native library (host
encoder, combiner, planner) or in its CUDA kernels (decoding). Device memory
and CUDA streams come from the caller (e.g. torch tensors and
``torch.cuda.Stream``); pass device pointers as ints or as objects with a
``data_ptr()`` method and streams as ints or objects with a ``cuda_stream``
attribute. There is no fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librecoil.so")

W = 32
OK, EINVAL, ECORRUPT, ENOMEM, ECUDA, ETIMEOUT = 0, -1, -2, -3, -4, -5
BATCH_PER_STREAM, BATCH_NO_SORT, BATCH_GRAPH, BATCH_NO_PAIRS, BATCH_TWO_LANES = 1, 2, 4, 8, 16
(KERNEL_PACKED8, KERNEL_GENERIC8, KERNEL_GENERIC16, KERNEL_ADAPTIVE8, KERNEL_ADAPTIVE16, KERNEL_ADAPTIVE16_WIDE,
 KERNEL_ADAPTIVE8_PAIR, KERNEL_ADAPTIVE16_PAIR, KERNEL_PACKED16) = (1 << k for k in range(9))


class RecoilError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"recoil error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("n_bits", C.c_uint32), ("sym_bytes", C.c_uint32), ("split_rule", C.c_uint32),
                ("reserved", C.c_uint32)]


SPLIT_REMAINING, SPLIT_EQ7 = 0, 1
_SPLIT_RULES = {"remaining": SPLIT_REMAINING, "eq7": SPLIT_EQ7}


def _params(n_bits: int, sym_bytes: int, rule: str = "remaining") -> Params:
    if rule not in _SPLIT_RULES:
        raise ValueError(f"rule must be one of {tuple(_SPLIT_RULES)}")
    return Params(n_bits, sym_bytes, _SPLIT_RULES[rule], 0)


class Info(C.Structure):
    _fields_ = [("n_syms", C.c_uint64), ("n_words", C.c_uint64), ("n_entries", C.c_uint32),
                ("n_bits", C.c_uint32), ("sym_bytes", C.c_uint32), ("alphabet", C.c_uint32),
                ("bitstream_bytes", C.c_uint64), ("metadata_bytes", C.c_uint64), ("max_sync", C.c_uint64),
                ("n_tables", C.c_uint32), ("reserved", C.c_uint32)]


class BatchOpts(C.Structure):
    _fields_ = [("warps_per_cta", C.c_uint32), ("ctas_per_sm", C.c_uint32),
                ("split_symbols", C.c_uint32), ("flags", C.c_uint32)]


class ServeOpts(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_inflight", C.c_uint32), ("max_batch", C.c_uint32),
                ("warps_per_cta", C.c_uint32), ("flags", C.c_uint32), ("meta_bytes", C.c_size_t),
                ("timeout_s", C.c_double), ("max_split_symbols", C.c_uint32), ("reserved", C.c_uint32)]


class RequestResult(C.Structure):
    _fields_ = [("arrival_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("splits", C.c_uint32), ("launch", C.c_uint32)]


class ServeStats(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("launches", C.c_uint64), ("symbol_bytes", C.c_uint64),
                ("makespan_s", C.c_double), ("decoded_gbs", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_inflight", C.c_uint32)]


SERVE_PER_REQUEST = 1


class TuneOpts(C.Structure):
    _fields_ = [("steps", C.c_uint32), ("flags", C.c_uint32), ("cache_path", C.c_char_p)]


TUNE_REFRESH = 1
TUNE_KEEP_SPLITS = 2

EXPORTS = [
    "recoil_encode_with_splits", "recoil_combine_splits", "recoil_stream_info", "recoil_stream_export",
    "recoil_stream_import", "recoil_stream_pin", "recoil_free", "recoil_last_error",
    "recoil_plan_create", "recoil_plan_workspace_size", "recoil_plan_upload", "recoil_plan_decode",
    "recoil_plan_errors", "recoil_plan_launches", "recoil_plan_free", "recoil_workspace_size",
    "recoil_decode", "recoil_decode_batch", "recoil_decode_noalloc", "recoil_autotune",
    "recoil_autotune_workspace_size", "recoil_serve", "recoil_serve_arena_size",
    "recoil_pipeline_create", "recoil_pipeline_sizes", "recoil_pipeline_run", "recoil_pipeline_errors",
    "recoil_pipeline_free", "recoil_shard", "recoil_encode_with_table",
    "recoil_serialized_size", "recoil_serialize", "recoil_deserialize", "recoil_encode_adaptive",
    "recoil_plan_create_shard", "recoil_plan_warps_per_cta", "recoil_plan_kernels",
]

_lib = None


def lib():
    """The loaded native library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2306_12141_b300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        pp = C.POINTER(C.c_void_p)
        L.recoil_encode_with_splits.argtypes = [vp, u64, C.POINTER(Params), u32, pp]
        L.recoil_combine_splits.argtypes = [vp, u32, pp]
        L.recoil_encode_with_table.argtypes = [vp, u64, C.POINTER(Params), vp, u32, u32, pp]
        L.recoil_encode_adaptive.argtypes = [vp, u64, C.POINTER(Params), vp, u32, u32, vp, u32, pp]
        L.recoil_stream_info.argtypes = [vp, C.POINTER(Info)]
        L.recoil_stream_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.recoil_stream_import.argtypes = [C.POINTER(Params), u64, u32, vp, vp, u64, vp, u32, vp, vp, vp, pp]
        L.recoil_stream_pin.argtypes = [vp]
        L.recoil_serialized_size.argtypes = [vp, C.POINTER(u64), C.POINTER(u64)]
        L.recoil_serialize.argtypes = [vp, vp, u64, C.POINTER(u64)]
        L.recoil_deserialize.argtypes = [vp, u64, pp]
        L.recoil_free.argtypes = [vp]
        L.recoil_free.restype = None
        L.recoil_last_error.restype = C.c_char_p
        L.recoil_plan_create.argtypes = [vp, u32, C.POINTER(BatchOpts), pp]
        L.recoil_plan_workspace_size.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.recoil_plan_upload.argtypes = [vp, vp, C.c_size_t, vp]
        L.recoil_plan_decode.argtypes = [vp, vp, vp]
        L.recoil_plan_errors.argtypes = [vp, vp, C.POINTER(u32)]
        L.recoil_plan_launches.argtypes = [vp]
        L.recoil_plan_warps_per_cta.argtypes = [vp]
        L.recoil_plan_warps_per_cta.restype = u32
        L.recoil_plan_launches.restype = u32
        L.recoil_plan_kernels.argtypes = [vp]
        L.recoil_plan_kernels.restype = u32
        L.recoil_plan_free.argtypes = [vp]
        L.recoil_plan_free.restype = None
        L.recoil_workspace_size.argtypes = [vp, u32, C.POINTER(BatchOpts), C.POINTER(C.c_size_t)]
        L.recoil_decode.argtypes = [vp, vp, vp, C.c_size_t, vp]
        L.recoil_decode_batch.argtypes = [vp, u32, vp, vp, C.c_size_t, vp, C.POINTER(BatchOpts)]
        L.recoil_decode_noalloc.argtypes = [vp, vp, C.c_size_t, vp, vp]
        L.recoil_shard.argtypes = [vp, u32, u32, vp]
        L.recoil_plan_create_shard.argtypes = [vp, u32, u32, C.POINTER(BatchOpts), pp, C.POINTER(u64), C.POINTER(u64)]
        L.recoil_pipeline_create.argtypes = [vp, u32, C.POINTER(BatchOpts), u32, pp]
        L.recoil_pipeline_sizes.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        L.recoil_pipeline_run.argtypes = [vp, vp, vp, C.c_size_t, vp, C.c_size_t, vp]
        L.recoil_pipeline_errors.argtypes = [vp, C.POINTER(u32)]
        L.recoil_pipeline_free.argtypes = [vp]
        L.recoil_pipeline_free.restype = None
        L.recoil_serve_arena_size.argtypes = [vp, u32, C.POINTER(ServeOpts), C.POINTER(C.c_size_t)]
        L.recoil_serve.argtypes = [vp, u32, vp, vp, u32, vp, C.c_size_t, vp, C.POINTER(ServeOpts),
                                   C.POINTER(RequestResult), C.POINTER(ServeStats)]
        L.recoil_autotune_workspace_size.argtypes = [vp, u32, C.POINTER(C.c_size_t)]
        L.recoil_autotune.argtypes = [vp, u32, vp, vp, C.c_size_t, vp, C.POINTER(TuneOpts),
                                      C.POINTER(BatchOpts), C.POINTER(C.c_float)]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise RecoilError(rc, lib().recoil_last_error().decode(errors="replace"))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream_handle(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _opts(opts) -> BatchOpts | None:
    if opts is None:
        return None
    if isinstance(opts, BatchOpts):
        return opts
    return BatchOpts(**opts)


# ------------------------------------------------------------------ streams
class Stream:
    """A host recoil_stream (owned; freed when garbage collected)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.recoil_free(self.handle)
            self.handle = None

    @property
    def info(self) -> dict:
        return stream_info(self)

    def export(self) -> dict:
        return stream_export(self)


def recoil_encode_with_splits(symbols: np.ndarray, n_bits: int, max_splits: int, rule: str = "remaining") -> Stream:
    """rule: T of Eq. 7, "remaining" (over the symbols left, default) or "eq7" (ceil(N / M) as printed)."""
    s = np.ascontiguousarray(symbols)
    if s.dtype not in (np.uint8, np.uint16):
        raise TypeError("symbols must be uint8 or uint16")
    p = _params(n_bits, s.dtype.itemsize, rule)
    h = C.c_void_p()
    _check(lib().recoil_encode_with_splits(s.ctypes.data if s.size else None, s.size, C.byref(p),
                                           max_splits, C.byref(h)))
    return Stream(h.value)


def recoil_encode_with_table(symbols: np.ndarray, n_bits: int, freq, max_splits: int,
                             rule: str = "remaining") -> Stream:
    s = np.ascontiguousarray(symbols)
    if s.dtype not in (np.uint8, np.uint16):
        raise TypeError("symbols must be uint8 or uint16")
    f = np.ascontiguousarray(freq, dtype=np.uint32)
    p = _params(n_bits, s.dtype.itemsize, rule)
    h = C.c_void_p()
    _check(lib().recoil_encode_with_table(s.ctypes.data if s.size else None, s.size, C.byref(p), _ptr(f), len(f),
                                          max_splits, C.byref(h)))
    return Stream(h.value)


def recoil_encode_adaptive(symbols: np.ndarray, n_bits: int, tables, table_index, max_splits: int,
                           rule: str = "remaining") -> Stream:
    """Adaptive coding (Sec. 3.1): symbol i coded with PDF row table_index[i] of tables (T x A)."""
    s = np.ascontiguousarray(symbols)
    if s.dtype not in (np.uint8, np.uint16):
        raise TypeError("symbols must be uint8 or uint16")
    f = np.ascontiguousarray(np.atleast_2d(tables), dtype=np.uint32)
    t = np.ascontiguousarray(table_index, dtype=np.uint8)
    if t.shape != s.shape:
        raise ValueError("one table number per symbol")
    p = _params(n_bits, s.dtype.itemsize, rule)
    h = C.c_void_p()
    _check(lib().recoil_encode_adaptive(s.ctypes.data if s.size else None, s.size, C.byref(p), _ptr(f), f.shape[0],
                                        f.shape[1], t.ctypes.data if t.size else None, max_splits, C.byref(h)))
    return Stream(h.value)


def recoil_combine_splits(stream: Stream, target_splits: int) -> Stream:
    h = C.c_void_p()
    _check(lib().recoil_combine_splits(stream.handle, target_splits, C.byref(h)))
    return Stream(h.value)


def recoil_stream_info(stream: Stream) -> dict:
    i = Info()
    _check(lib().recoil_stream_info(stream.handle, C.byref(i)))
    return {k: getattr(i, k) for k, _ in Info._fields_}


def recoil_stream_export(stream: Stream) -> dict:
    info = recoil_stream_info(stream)
    R = info["n_entries"] - 1
    out = {
        "freq": np.zeros(max(1, info["n_tables"]) * info["alphabet"], dtype=np.uint32),
        "words": np.zeros(info["n_words"], dtype=np.uint16),
        "final": np.zeros(W, dtype=np.uint32),
        "entry_word": np.zeros(R, dtype=np.uint64),
        "entry_index": np.zeros((R, W), dtype=np.uint64),
        "entry_state": np.zeros((R, W), dtype=np.uint16),
    }
    _check(lib().recoil_stream_export(stream.handle, *[_ptr(out[k]) if out[k].size else None for k in
                                                       ("freq", "words", "final", "entry_word",
                                                        "entry_index", "entry_state")]))
    return out


def stream_freq(stream: Stream) -> np.ndarray:
    """The stream's quantised PDF only (adaptive: n_tables x alphabet), via recoil_stream_export."""
    info = stream_info(stream)
    f = np.zeros(max(1, info["n_tables"]) * info["alphabet"], dtype=np.uint32)
    _check(lib().recoil_stream_export(stream.handle, _ptr(f), None, None, None, None, None))
    return f.reshape(info["n_tables"], info["alphabet"]) if info["n_tables"] else f


def recoil_stream_import(n_bits: int, sym_bytes: int, n_syms: int, freq, words, final,
                         entry_word, entry_index, entry_state) -> Stream:
    freq = np.ascontiguousarray(freq, dtype=np.uint32)
    words = np.ascontiguousarray(words, dtype=np.uint16)
    final = np.ascontiguousarray(final, dtype=np.uint32)
    ew = np.ascontiguousarray(entry_word, dtype=np.uint64)
    ei = np.ascontiguousarray(entry_index, dtype=np.uint64)
    es = np.ascontiguousarray(entry_state, dtype=np.uint16)
    p = Params(n_bits, sym_bytes)
    h = C.c_void_p()
    _check(lib().recoil_stream_import(C.byref(p), n_syms, len(freq), _ptr(freq), _ptr(words) if words.size else None,
                                      words.size, _ptr(final), len(ew), _ptr(ew) if ew.size else None,
                                      _ptr(ei) if ei.size else None, _ptr(es) if es.size else None, C.byref(h)))
    return Stream(h.value)


def recoil_stream_pin(stream: Stream) -> None:
    _check(lib().recoil_stream_pin(stream.handle))


def recoil_serialized_size(stream: Stream) -> tuple[int, int]:
    """(container bytes, packed split-metadata bytes) of the stream's serialised form (Sec. 4.3)."""
    total, meta = C.c_uint64(), C.c_uint64()
    _check(lib().recoil_serialized_size(stream.handle, C.byref(total), C.byref(meta)))
    return total.value, meta.value


def recoil_serialize(stream: Stream) -> bytes:
    """The stream's serialised form: model, final states, words and packed split metadata."""
    total, _ = recoil_serialized_size(stream)
    buf = C.create_string_buffer(max(1, total))
    written = C.c_uint64()
    _check(lib().recoil_serialize(stream.handle, buf, total, C.byref(written)))
    return buf.raw[:written.value]


def recoil_deserialize(data: bytes) -> Stream:
    """Parse a serialised stream (validated like recoil_stream_import)."""
    data = bytes(data)
    h = C.c_void_p()
    _check(lib().recoil_deserialize(data, len(data), C.byref(h)))
    return Stream(h.value)


# -------------------------------------------------------------------- plans
def _handles(streams) -> C.Array:
    arr = (C.c_void_p * max(1, len(streams)))()
    for k, s in enumerate(streams):
        arr[k] = s.handle
    return arr


def _ptr_array(ptrs) -> C.Array:
    arr = (C.c_void_p * max(1, len(ptrs)))()
    for k, p in enumerate(ptrs):
        arr[k] = _ptr(p)
    return arr


class Plan:
    """A recoil_plan: device image layout and work queue of a batch of streams."""

    def __init__(self, streams, opts=None, _handle=None):
        self.streams = list(streams)          # keep the host streams alive
        if _handle is not None:
            self.handle = _handle
            return
        h = C.c_void_p()
        o = _opts(opts)
        _check(lib().recoil_plan_create(_handles(self.streams), len(self.streams),
                                        C.byref(o) if o is not None else None, C.byref(h)))
        self.handle = h.value

    @classmethod
    def shard(cls, stream, world: int, rank: int, opts=None):
        """recoil_plan_create_shard: (plan, sym_lo, sym_hi) of rank's contiguous run of splits."""
        h = C.c_void_p()
        o = _opts(opts)
        lo, hi = C.c_uint64(), C.c_uint64()
        _check(lib().recoil_plan_create_shard(stream.handle, world, rank, C.byref(o) if o is not None else None,
                                              C.byref(h), C.byref(lo), C.byref(hi)))
        return cls([stream], _handle=h.value), lo.value, hi.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.recoil_plan_free(self.handle)
            self.handle = None

    @property
    def workspace_size(self) -> int:
        n = C.c_size_t()
        _check(lib().recoil_plan_workspace_size(self.handle, C.byref(n)))
        return n.value

    def upload(self, workspace, nbytes: int | None = None, stream=None) -> None:
        nb = self.workspace_size if nbytes is None else nbytes
        _check(lib().recoil_plan_upload(self.handle, _ptr(workspace), nb, _stream_handle(stream)))

    def decode(self, outs, stream=None) -> None:
        self._outs = _ptr_array(outs)
        _check(lib().recoil_plan_decode(self.handle, self._outs, _stream_handle(stream)))

    def errors(self, stream=None) -> int:
        f = C.c_uint32()
        rc = lib().recoil_plan_errors(self.handle, _stream_handle(stream), C.byref(f))
        if rc not in (OK, ECORRUPT):
            _check(rc)
        return f.value

    @property
    def launches(self) -> int:
        return int(lib().recoil_plan_launches(self.handle))

    @property
    def kernels(self) -> int:
        """Bit mask of the decoder kernels the plan launches (KERNEL_*)."""
        return int(lib().recoil_plan_kernels(self.handle))

    @property
    def warps_per_cta(self) -> int:
        return int(lib().recoil_plan_warps_per_cta(self.handle))


def recoil_plan_create(streams, opts=None) -> Plan:
    return Plan(streams, opts)


def recoil_plan_warps_per_cta(plan: Plan) -> int:
    return plan.warps_per_cta


def recoil_plan_create_shard(stream, world: int, rank: int, opts=None):
    """(plan, sym_lo, sym_hi): rank's contiguous run of the stream's splits (see recoil.h)."""
    return Plan.shard(stream, world, rank, opts)


def recoil_workspace_size(streams, opts=None) -> int:
    n = C.c_size_t()
    o = _opts(opts)
    _check(lib().recoil_workspace_size(_handles(streams), len(streams), C.byref(o) if o is not None else None,
                                       C.byref(n)))
    return n.value


def recoil_shard(streams, world: int) -> np.ndarray:
    """Rank of each stream when a batch is split over `world` GPUs (longest first)."""
    out = np.zeros(max(1, len(streams)), dtype=np.uint32)
    _check(lib().recoil_shard(_handles(streams), len(streams), world, _ptr(out)))
    return out[: len(streams)]


def recoil_decode(stream: Stream, out, workspace, nbytes: int, cuda_stream=None) -> None:
    _check(lib().recoil_decode(stream.handle, _ptr(out), _ptr(workspace), nbytes, _stream_handle(cuda_stream)))


def recoil_decode_batch(streams, outs, workspace, nbytes: int, cuda_stream=None, opts=None) -> None:
    o = _opts(opts)
    _check(lib().recoil_decode_batch(_handles(streams), len(streams), _ptr_array(outs), _ptr(workspace), nbytes,
                                     _stream_handle(cuda_stream), C.byref(o) if o is not None else None))


def recoil_free(stream: Stream) -> None:
    """Release a stream now instead of at garbage collection."""
    if stream.handle:
        lib().recoil_free(stream.handle)
        stream.handle = None


def recoil_last_error() -> str:
    return lib().recoil_last_error().decode(errors="replace")


def recoil_plan_workspace_size(plan: Plan) -> int:
    return plan.workspace_size


def recoil_plan_upload(plan: Plan, workspace, nbytes: int | None = None, cuda_stream=None) -> None:
    plan.upload(workspace, nbytes, cuda_stream)


def recoil_plan_decode(plan: Plan, outs, cuda_stream=None) -> None:
    plan.decode(outs, cuda_stream)


def recoil_plan_errors(plan: Plan, cuda_stream=None) -> int:
    return plan.errors(cuda_stream)


def recoil_plan_launches(plan: Plan) -> int:
    return plan.launches


def recoil_plan_kernels(plan: Plan) -> int:
    return plan.kernels


def recoil_plan_free(plan: Plan) -> None:
    if plan.handle:
        lib().recoil_plan_free(plan.handle)
        plan.handle = None


def recoil_autotune_workspace_size(streams) -> int:
    n = C.c_size_t()
    _check(lib().recoil_autotune_workspace_size(_handles(streams), len(streams), C.byref(n)))
    return n.value


def recoil_autotune(streams, outs, workspace, nbytes: int, cuda_stream=None, steps: int = 3,
                    cache_path: str | None = None, refresh: bool = False,
                    keep_splits: bool = False) -> tuple[dict, float]:
    """Measured best batch options for these streams: ({warps_per_cta, split_symbols, ...}, ms).
    keep_splits: tune warps_per_cta only, on the streams' own split counts."""
    flags = (TUNE_REFRESH if refresh else 0) | (TUNE_KEEP_SPLITS if keep_splits else 0)
    t = TuneOpts(steps, flags, cache_path.encode() if cache_path else None)
    best = BatchOpts()
    ms = C.c_float()
    _check(lib().recoil_autotune(_handles(streams), len(streams), _ptr_array(outs), _ptr(workspace), nbytes,
                                 _stream_handle(cuda_stream), C.byref(t), C.byref(best), C.byref(ms)))
    return {k: getattr(best, k) for k, _ in BatchOpts._fields_}, float(ms.value)


class Pipeline:
    """Host-to-host decoding of a batch with copy/compute overlap (recoil_pipeline_*)."""

    def __init__(self, streams, opts=None, groups: int = 8):
        self.streams = list(streams)
        h = C.c_void_p()
        o = _opts(opts)
        _check(lib().recoil_pipeline_create(_handles(self.streams), len(self.streams),
                                            C.byref(o) if o is not None else None, groups, C.byref(h)))
        self.handle = h.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.recoil_pipeline_free(self.handle)
            self.handle = None

    @property
    def sizes(self) -> tuple[int, int]:
        a, b = C.c_size_t(), C.c_size_t()
        _check(lib().recoil_pipeline_sizes(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def run(self, host_outs, workspace, ws_bytes: int, staging, staging_bytes: int, stream=None) -> None:
        self._outs = _ptr_array(host_outs)
        _check(lib().recoil_pipeline_run(self.handle, self._outs, _ptr(workspace), ws_bytes, _ptr(staging),
                                         staging_bytes, _stream_handle(stream)))

    def errors(self) -> int:
        f = C.c_uint32()
        rc = lib().recoil_pipeline_errors(self.handle, C.byref(f))
        if rc not in (OK, ECORRUPT):
            _check(rc)
        return f.value


def recoil_pipeline_create(streams, opts=None, groups: int = 8) -> Pipeline:
    return Pipeline(streams, opts, groups)


def recoil_pipeline_sizes(p: Pipeline) -> tuple[int, int]:
    return p.sizes


def recoil_pipeline_run(p: Pipeline, host_outs, workspace, ws_bytes, staging, staging_bytes, stream=None):
    p.run(host_outs, workspace, ws_bytes, staging, staging_bytes, stream)


def recoil_pipeline_errors(p: Pipeline) -> int:
    return p.errors()


def recoil_pipeline_free(p: Pipeline) -> None:
    if p.handle:
        lib().recoil_pipeline_free(p.handle)
        p.handle = None


def _serve_opts(budget_bytes, max_inflight=0, max_batch=0, warps_per_cta=0, per_request=False, meta_bytes=0,
                timeout_s=0.0, max_split_symbols=0):
    return ServeOpts(int(budget_bytes), max_inflight, max_batch, warps_per_cta,
                     SERVE_PER_REQUEST if per_request else 0, meta_bytes, timeout_s, max_split_symbols, 0)


def recoil_serve_arena_size(pool, budget_bytes, **kw) -> int:
    o = _serve_opts(budget_bytes, **kw)
    n = C.c_size_t()
    _check(lib().recoil_serve_arena_size(_handles(pool), len(pool), C.byref(o), C.byref(n)))
    return n.value


def recoil_serve(pool, req_stream, req_arrival_s, arena, arena_bytes: int, budget_bytes: int, outs=None, **kw):
    """Continuous-batching serving run. Returns (per-request results as a dict of arrays, stats dict)."""
    o = _serve_opts(budget_bytes, **kw)
    rs = np.ascontiguousarray(req_stream, dtype=np.uint32)
    ra = np.ascontiguousarray(req_arrival_s, dtype=np.float64)
    n = len(rs)
    res = (RequestResult * max(1, n))()
    st = ServeStats()
    optr = _ptr_array(outs) if outs is not None else None
    _check(lib().recoil_serve(_handles(pool), len(pool), _ptr(rs), _ptr(ra), n, _ptr(arena), arena_bytes, optr,
                              C.byref(o), res, C.byref(st)))
    out = {k: np.array([getattr(res[i], k) for i in range(n)]) for k, _ in RequestResult._fields_}
    return out, {k: getattr(st, k) for k, _ in ServeStats._fields_}


NOALLOC_SCRATCH_BYTES = 4 << 20


def noalloc_words_bytes(stream: Stream) -> int:
    """Bytes of the device word buffer recoil_decode_noalloc reads (words padded to 256-word chunks)."""
    return -(-stream.info["n_words"] // 256) * 512


def recoil_decode_noalloc(stream: Stream, d_words, words_bytes: int, d_out, cuda_stream=None) -> None:
    """Decode without device allocation: words and output are caller device buffers (see recoil.h)."""
    _check(lib().recoil_decode_noalloc(stream.handle, _ptr(d_words), words_bytes, _ptr(d_out),
                                       _stream_handle(cuda_stream)))


# short aliases
encode_with_splits = recoil_encode_with_splits
combine_splits = recoil_combine_splits
encode_with_table = recoil_encode_with_table
encode_adaptive = recoil_encode_adaptive
stream_info = recoil_stream_info
stream_export = recoil_stream_export
stream_import = recoil_stream_import
stream_pin = recoil_stream_pin
serialized_size = recoil_serialized_size
serialize = recoil_serialize
deserialize = recoil_deserialize
workspace_size = recoil_workspace_size
decode = recoil_decode
decode_batch = recoil_decode_batch
shard = recoil_shard
decode_noalloc = recoil_decode_noalloc
autotune = recoil_autotune
serve = recoil_serve
serve_arena_size = recoil_serve_arena_size
autotune_workspace_size = recoil_autotune_workspace_size
