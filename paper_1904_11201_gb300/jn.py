"""Python binding of libjn (include/jn.h): argument marshalling only.

Every join step runs in the CUDA library; this module converts torch
tensors into ``jn_table`` structures, calls the C entry points of the same
names, and wraps library-allocated results as torch tensors.  It never
computes a join itself and fails loudly when the library is missing.

Columns may be CUDA tensors or CPU tensors (the library stages host
columns to the device).  Pairs come back as an (n, 2) int32 tensor of
(r, s) = (R.payload, S.payload).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libjn.so")

JN_OK, JN_ERR_INVALID, JN_ERR_OOM, JN_ERR_CAPACITY, JN_ERR_CUDA, JN_ERR_TIMEOUT, \
    JN_ERR_UNSUPPORTED = range(7)
JN_KEY_I32, JN_KEY_I64 = 4, 8
JN_EQ, JN_NE, JN_LT, JN_LE, JN_GT, JN_GE, JN_ANY = range(7)
JN_ALGO_NLJ, JN_ALGO_HASH, JN_ALGO_THETA, JN_ALGO_SORT = range(4)
OPS = {"=": JN_EQ, "!=": JN_NE, "<": JN_LT, "<=": JN_LE, ">": JN_GT, ">=": JN_GE, "any": JN_ANY}


class JoinError(RuntimeError):
    def __init__(self, status, msg, required=None):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status
        self.required = required


class Table(ctypes.Structure):
    _fields_ = [("key", ctypes.c_void_p), ("key2", ctypes.c_void_p), ("payload", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("key_type", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Pred(ctypes.Structure):
    _fields_ = [("op_a", ctypes.c_int32), ("op_k", ctypes.c_int32), ("band", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("prefilter", ctypes.c_int32), ("radix_bits", ctypes.c_int32),
                ("radix_bits1", ctypes.c_int32), ("filter_bits", ctypes.c_int32),
                ("heavy", ctypes.c_int32), ("theta_groups", ctypes.c_int32),
                ("nlj_tile_r", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("part_rows", ctypes.c_int32), ("host_io", ctypes.c_int32),
                ("hash_path", ctypes.c_int32), ("table_rows", ctypes.c_int32),
                ("sms", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Join(ctypes.Structure):
    _fields_ = [("R", Table), ("S", Table), ("op", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("band", ctypes.c_int64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("coalesce_rows", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("memory_budget", ctypes.c_uint64), ("small_slots", ctypes.c_int32),
                ("hold_wait_ms", ctypes.c_int32), ("small_sms", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("r_handle", ctypes.c_int32), ("s_handle", ctypes.c_int32), ("R", Table), ("S", Table),
                ("op", ctypes.c_int32), ("reserved", ctypes.c_int32), ("band", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("pairs", ctypes.c_uint64),
                ("out", ctypes.c_void_p), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "batches", "queued",
                                               "held_bytes", "peak_bytes", "resident_bytes",
                                               "kernel_launches")]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double)]


class RunInfo(ctypes.Structure):
    _fields_ = [("result", ctypes.c_uint64), ("r_survivors", ctypes.c_uint64),
                ("s_survivors", ctypes.c_uint64), ("partitions", ctypes.c_uint64),
                ("work_items", ctypes.c_uint64), ("heavy_keys", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("prefilter", ctypes.c_int32),
                ("radix_bits", ctypes.c_int32), ("radix_bits1", ctypes.c_int32),
                ("filter_bits", ctypes.c_int32), ("scratch_peak", ctypes.c_uint64),
                ("heavy_pairs", ctypes.c_uint64), ("cartesian_bound", ctypes.c_uint64),
                ("hash_path", ctypes.c_uint64), ("table_rows", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64 * 1)]


ADMIT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64)


class Pair(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("s", ctypes.c_int32)]


_lib = None

# name -> (restype, argtypes); kept in step with include/jn.h
_P = ctypes.c_void_p
_SIGS = {
    "jn_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "jn_destroy": (None, [_P]),
    "jn_set_stream": (ctypes.c_int, [_P, _P]),
    "jn_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    "jn_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    "jn_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "jn_last_error": (ctypes.c_char_p, [_P]),
    "jn_version": (ctypes.c_char_p, []),
    "jn_count": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Table), ctypes.POINTER(Table),
                                ctypes.POINTER(Pred), ctypes.POINTER(ctypes.c_uint64)]),
    "jn_aggregate": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Table), ctypes.POINTER(Table),
                                    ctypes.POINTER(Pred), ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.POINTER(ctypes.c_uint64)]),
    "jn_nested_loop": (ctypes.c_int, [_P, ctypes.POINTER(Table), ctypes.POINTER(Table),
                                      ctypes.POINTER(Pred), ctypes.POINTER(_P), ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "jn_hash": (ctypes.c_int, [_P, ctypes.POINTER(Table), ctypes.POINTER(Table), ctypes.POINTER(_P),
                               ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "jn_sort_merge": (ctypes.c_int, [_P, ctypes.POINTER(Table), ctypes.POINTER(Table), ctypes.POINTER(_P),
                                     ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "jn_theta": (ctypes.c_int, [_P, ctypes.POINTER(Table), ctypes.POINTER(Table), ctypes.c_int32,
                                ctypes.c_int64, ctypes.POINTER(_P), ctypes.c_uint64,
                                ctypes.POINTER(ctypes.c_uint64)]),
    "jn_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Join), ctypes.POINTER(_P), ctypes.c_uint64,
                                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64)]),
    "jn_free": (None, [_P, _P]),
    "jn_star": (ctypes.c_int, [_P, ctypes.POINTER(Table), ctypes.POINTER(Table), ctypes.POINTER(Table),
                               ctypes.POINTER(_P), ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "jn_star_count": (ctypes.c_int, [_P, ctypes.POINTER(Table), ctypes.POINTER(Table), ctypes.POINTER(Table),
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "jn_free_triples": (None, [_P, _P]),
    "jn_batch_count": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Join), _P, _P]),
    "jn_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Table), ctypes.POINTER(Table),
                                   ctypes.POINTER(Pred), ctypes.POINTER(Tuning)]),
    "jn_autotune_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Join), ctypes.POINTER(Tuning)]),
    "jn_nested_loop_noalloc": (ctypes.c_int, [ctypes.POINTER(Table), ctypes.POINTER(Table), ctypes.POINTER(Pred),
                                              _P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _P]),
    "jn_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ServerConfig)]),
    "jn_server_destroy": (None, [_P]),
    "jn_server_register": (ctypes.c_int, [_P, ctypes.POINTER(Table), ctypes.POINTER(ctypes.c_int32)]),
    "jn_server_unregister": (ctypes.c_int, [_P, ctypes.c_int32]),
    "jn_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "jn_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "jn_server_wait_any": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Result),
                                          ctypes.c_int64]),
    "jn_server_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "jn_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "jn_set_profiling": (ctypes.c_int, [_P, ctypes.c_int32]),
    "jn_set_memory_limit": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "jn_set_admission": (ctypes.c_int, [_P, _P, _P]),
    "jn_kernel_stats": (ctypes.c_int, [_P, ctypes.POINTER(KernelStat), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)]),
    "jn_reset_stats": (ctypes.c_int, [_P]),
    "jn_last_run_info": (ctypes.c_int, [_P, ctypes.POINTER(RunInfo)]),
    "jn_launch_count": (ctypes.c_uint64, [_P]),
    "jn_pointer_is_device": (ctypes.c_int32, [_P]),
    "jn_selftest_wait": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]),
}


def exported_symbols():
    """Names the binding expects libjn.so to export (the jn.h entry points)."""
    return sorted(_SIGS)


def load(path: str = LIB_PATH):
    """Loads libjn.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libjn.so not found at %s: build it with "
                               "`python -m paper_1904_11201_gb300.build`" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(ctx, st, required=None):
    if st != JN_OK:
        lib = load()
        msg = lib.jn_last_error(ctx.handle if ctx else None)
        msg = (msg or b"").decode() or lib.jn_status_str(st).decode()
        raise JoinError(st, msg, required)


class Context:
    """Owns a jn_ctx on one device and stream."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = _P()
        st = lib.jn_create(ctypes.byref(h), device, _P(stream.cuda_stream))
        if st != JN_OK:
            raise JoinError(st, "jn_create failed: %s" % lib.jn_status_str(st).decode())
        self.handle = h
        self.device = device
        self.closed = False

    def close(self):
        if not self.closed:
            load().jn_destroy(self.handle)
            self.closed = True

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, **kw):
        t = Tuning()
        load().jn_get_tuning(self.handle, ctypes.byref(t))
        for k, v in kw.items():
            setattr(t, k, v)
        _check(self, load().jn_set_tuning(self.handle, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = Tuning()
        load().jn_get_tuning(self.handle, ctypes.byref(t))
        return {f: getattr(t, f) for f, _ in Tuning._fields_ if f != "reserved"}

    def set_memory_limit(self, nbytes: int):
        """Refuse (JN_ERR_OOM, after the exact count) runs whose output + scratch exceed nbytes."""
        _check(self, load().jn_set_memory_limit(self.handle, nbytes))

    def set_admission(self, fn):
        """fn(out_bytes, scratch_bytes) -> status, called between the count and
        the output allocation; None removes the hook."""
        if fn is None:
            self._admit = None
            _check(self, load().jn_set_admission(self.handle, None, None))
            return
        cb = ADMIT_FN(lambda user, ob, sb: int(fn(int(ob), int(sb))))
        self._admit = cb  # keeps the callback alive while the context holds it
        _check(self, load().jn_set_admission(self.handle, ctypes.cast(cb, _P), None))

    def set_profiling(self, on: bool):
        _check(self, load().jn_set_profiling(self.handle, 1 if on else 0))

    def kernel_stats(self) -> dict:
        arr = (KernelStat * 64)()
        n = ctypes.c_int32()
        _check(self, load().jn_kernel_stats(self.handle, arr, 64, ctypes.byref(n)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms)) for i in range(n.value)}

    def reset_stats(self):
        _check(self, load().jn_reset_stats(self.handle))

    def run_info(self) -> dict:
        ri = RunInfo()
        load().jn_last_run_info(self.handle, ctypes.byref(ri))
        return {f: getattr(ri, f) for f, _ in RunInfo._fields_ if f != "reserved"}

    def launch_count(self) -> int:
        return int(load().jn_launch_count(self.handle))


class TableRef:
    """A jn_table plus references keeping its tensors alive."""

    def __init__(self, key, key2=None, payload=None):
        if key.dtype not in (torch.int32, torch.int64):
            raise TypeError("key columns must be int32 or int64")
        cols = [key] + [c for c in (key2,) if c is not None]
        for c in cols:
            if c.dtype != key.dtype or c.dim() != 1 or not c.is_contiguous():
                raise TypeError("key columns must be contiguous 1-D tensors of one dtype")
        if payload is not None and (payload.dtype != torch.int32 or payload.shape != key.shape
                                    or not payload.is_contiguous()):
            raise TypeError("payload must be a contiguous int32 tensor like the key")
        self.refs = (key, key2, payload)
        n = key.shape[0]
        self.t = Table(key.data_ptr() if n else None,
                       key2.data_ptr() if (key2 is not None and n) else None,
                       payload.data_ptr() if (payload is not None and n) else None,
                       n, JN_KEY_I32 if key.dtype == torch.int32 else JN_KEY_I64, 0)


def table(key, key2=None, payload=None) -> TableRef:
    return TableRef(key, key2, payload)


def pred(op_a=JN_EQ, op_k=JN_ANY, band=-1) -> Pred:
    return Pred(op_a, op_k, band)


class _DeviceResult:
    """Library-allocated pairs (width 2) or star-join triples (width 3)
    exposed through __cuda_array_interface__."""

    def __init__(self, ctx, ptr, n, width=2):
        self._ctx = ctx
        self._ptr = ptr
        self._width = width
        self.__cuda_array_interface__ = {"shape": (n, width), "typestr": "<i4", "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}

    def __del__(self):
        lib = load()
        ctx = self._ctx
        h = None if ctx.closed else ctx.handle
        if self._width == 3:
            lib.jn_free_triples(h, _P(self._ptr))
        else:
            lib.jn_free(h, _P(self._ptr))


def _result(ctx, out_ptr, n, user_out):
    if user_out is not None:
        return user_out[:n]
    if n == 0 or not out_ptr.value:
        return torch.empty((0, 2), dtype=torch.int32, device="cuda:%d" % ctx.device)
    return torch.as_tensor(_DeviceResult(ctx, out_ptr.value, n), device="cuda:%d" % ctx.device)


def _emit(ctx, fn, args, out):
    n = ctypes.c_uint64()
    if out is None:
        p = _P(None)
        cap = 0
    else:
        if out.dtype != torch.int32 or out.dim() != 2 or out.shape[1] != 2 or not out.is_contiguous():
            raise TypeError("out must be a contiguous (cap, 2) int32 tensor")
        p = _P(out.data_ptr())
        cap = out.shape[0]
    st = fn(ctx.handle, *args, ctypes.byref(p), cap, ctypes.byref(n))
    _check(ctx, st, required=int(n.value) if st in (JN_ERR_CAPACITY, JN_ERR_OOM) else None)
    return _result(ctx, p, int(n.value), out)


# ------------------------------------------------------------ entry points --

def jn_count(ctx: Context, algo: int, R: TableRef, S: TableRef, pr: Pred = None) -> int:
    c = ctypes.c_uint64()
    st = load().jn_count(ctx.handle, algo, ctypes.byref(R.t), ctypes.byref(S.t),
                         ctypes.byref(pr) if pr is not None else None, ctypes.byref(c))
    _check(ctx, st)
    return int(c.value)


def jn_aggregate(ctx: Context, algo: int, R: TableRef, S: TableRef, pr: Pred = None):
    c = ctypes.c_uint64()
    h = ctypes.c_uint64()
    st = load().jn_aggregate(ctx.handle, algo, ctypes.byref(R.t), ctypes.byref(S.t),
                             ctypes.byref(pr) if pr is not None else None, ctypes.byref(c),
                             ctypes.byref(h))
    _check(ctx, st)
    return int(c.value), int(h.value)


def jn_nested_loop(ctx: Context, R: TableRef, S: TableRef, pr: Pred = None, out=None):
    return _emit(ctx, load().jn_nested_loop,
                 (ctypes.byref(R.t), ctypes.byref(S.t), ctypes.byref(pr) if pr is not None else None),
                 out)


def jn_star(ctx: Context, R: TableRef, S1: TableRef, S2: TableRef, out=None):
    """Star join: R (key = fk1, key2 = fk2) with S1 on fk1 and S2 on fk2;
    an (n, 3) int32 tensor of (R, S1, S2) payloads."""
    n = ctypes.c_uint64()
    if out is None:
        p, cap = _P(None), 0
    else:
        if out.dtype != torch.int32 or out.dim() != 2 or out.shape[1] != 3 or not out.is_contiguous():
            raise TypeError("out must be a contiguous (cap, 3) int32 tensor")
        p, cap = _P(out.data_ptr()), out.shape[0]
    st = load().jn_star(ctx.handle, ctypes.byref(R.t), ctypes.byref(S1.t), ctypes.byref(S2.t), ctypes.byref(p),
                        cap, ctypes.byref(n))
    _check(ctx, st, required=int(n.value) if st in (JN_ERR_CAPACITY, JN_ERR_OOM) else None)
    m = int(n.value)
    if out is not None:
        return out[:m]
    if m == 0 or not p.value:
        return torch.empty((0, 3), dtype=torch.int32, device="cuda:%d" % ctx.device)
    return torch.as_tensor(_DeviceResult(ctx, p.value, m, 3), device="cuda:%d" % ctx.device)


def jn_star_count(ctx: Context, R: TableRef, S1: TableRef, S2: TableRef) -> int:
    c = ctypes.c_uint64()
    st = load().jn_star_count(ctx.handle, ctypes.byref(R.t), ctypes.byref(S1.t), ctypes.byref(S2.t),
                              ctypes.byref(c))
    _check(ctx, st)
    return int(c.value)


def jn_hash(ctx: Context, R: TableRef, S: TableRef, out=None):
    return _emit(ctx, load().jn_hash, (ctypes.byref(R.t), ctypes.byref(S.t)), out)


def jn_sort_merge(ctx: Context, R: TableRef, S: TableRef, out=None):
    return _emit(ctx, load().jn_sort_merge, (ctypes.byref(R.t), ctypes.byref(S.t)), out)


def jn_theta(ctx: Context, R: TableRef, S: TableRef, op: int, band: int = -1, out=None):
    return _emit(ctx, load().jn_theta, (ctypes.byref(R.t), ctypes.byref(S.t), op, band), out)


def jn_batch(ctx: Context, joins, out=None):
    """Runs a batch of joins [(R, S, op, band), ...] (band < 0: equi-join).

    Returns (pairs, first, count): the pairs of join i are
    pairs[first[i] : first[i] + count[i]].
    """
    n = len(joins)
    arr = (Join * max(n, 1))()
    for i, (R, S, op, band) in enumerate(joins):
        arr[i] = Join(R.t, S.t, op, 0, band)
    first = (ctypes.c_uint64 * max(n, 1))()
    cnt = (ctypes.c_uint64 * max(n, 1))()
    total = ctypes.c_uint64()
    if out is None:
        p = _P(None)
        cap = 0
    else:
        p = _P(out.data_ptr())
        cap = out.shape[0]
    st = load().jn_batch(ctx.handle, n, arr, ctypes.byref(p), cap, ctypes.byref(total), first, cnt)
    _check(ctx, st, required=int(total.value) if st == JN_ERR_CAPACITY else None)
    res = _result(ctx, p, int(total.value), out)
    return res, [int(first[i]) for i in range(n)], [int(cnt[i]) for i in range(n)]


class _View:
    """A non-owning view of device pairs (valid until the owner releases them)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n, 2), "typestr": "<i4", "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}


class Server:
    """jn_server: a request loop over the library (see jn.h, serving)."""

    def __init__(self, device=0, slots=4, coalesce_rows=1 << 18, max_batch=64, memory_budget=64 << 30,
                 graphs=False, small_slots=0, hold_wait_ms=2000, small_sms=0):
        lib = load()
        cfg = ServerConfig(slots, coalesce_rows, max_batch, 1 if graphs else 0, memory_budget, small_slots,
                           hold_wait_ms, small_sms, 0)
        h = _P()
        st = lib.jn_server_create(ctypes.byref(h), device, ctypes.byref(cfg))
        if st != JN_OK:
            raise JoinError(st, "jn_server_create failed")
        self.handle = h
        self.device = device
        self._keep = {}

    def close(self):
        if self.handle:
            load().jn_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, t: TableRef) -> int:
        hnd = ctypes.c_int32()
        st = load().jn_server_register(self.handle, ctypes.byref(t.t), ctypes.byref(hnd))
        if st != JN_OK:
            raise JoinError(st, "jn_server_register failed")
        return int(hnd.value)

    def unregister(self, handle: int):
        st = load().jn_server_unregister(self.handle, handle)
        if st != JN_OK:
            raise JoinError(st, "jn_server_unregister failed")

    def submit(self, R=None, S=None, op=JN_EQ, band=-1, r_handle=0, s_handle=0) -> int:
        """R, S: TableRef (device columns) or None with a registered handle."""
        empty = Table(None, None, None, 0, JN_KEY_I32, 0)
        req = Request(r_handle, s_handle, R.t if R is not None else empty, S.t if S is not None else empty,
                      op, 0, band)
        if r_handle and R is None and S is not None:
            req.R.key_type = S.t.key_type
        if s_handle and S is None and R is not None:
            req.S.key_type = R.t.key_type
        tk = ctypes.c_uint64()
        st = load().jn_server_submit(self.handle, ctypes.byref(req), ctypes.byref(tk))
        if st != JN_OK:
            raise JoinError(st, "jn_server_submit failed")
        self._keep[int(tk.value)] = (R, S)  # columns stay alive until the request is released
        return int(tk.value)

    @staticmethod
    def _res(r) -> dict:
        return {"status": r.status, "pairs": int(r.pairs), "out": r.out, "queue_ms": r.queue_ms,
                "run_ms": r.run_ms, "total_ms": r.total_ms}

    def wait(self, ticket: int) -> dict:
        r = Result()
        st = load().jn_server_wait(self.handle, ticket, ctypes.byref(r))
        if st != JN_OK:
            raise JoinError(st, "jn_server_wait failed")
        return self._res(r)

    def wait_any(self, timeout_ms: int = -1):
        """(ticket, result) of the oldest completion not yet returned by a wait;
        None on timeout."""
        r = Result()
        t = ctypes.c_uint64()
        st = load().jn_server_wait_any(self.handle, ctypes.byref(t), ctypes.byref(r), timeout_ms)
        if st == JN_ERR_TIMEOUT:
            return None
        if st != JN_OK:
            raise JoinError(st, "jn_server_wait_any failed")
        return int(t.value), self._res(r)

    def pairs(self, res: dict):
        """Copies a finished request's pairs into a new CUDA tensor."""
        if res["status"] != JN_OK:
            raise JoinError(res["status"], "request failed")
        if res["pairs"] == 0:
            return torch.empty((0, 2), dtype=torch.int32, device="cuda:%d" % self.device)
        if not res["out"] or not load().jn_pointer_is_device(_P(res["out"])):
            raise JoinError(JN_ERR_CUDA, "request output is not device memory: %r" % (res["out"],))
        v = torch.as_tensor(_View(res["out"], res["pairs"]), device="cuda:%d" % self.device)
        return v.clone()

    def release(self, ticket: int):
        load().jn_server_release(self.handle, ticket)
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        x = ServerStats()
        load().jn_server_stats_get(self.handle, ctypes.byref(x))
        return {f: int(getattr(x, f)) for f, _ in ServerStats._fields_}


def jn_nested_loop_noalloc(R: TableRef, S: TableRef, pr: Pred = None, out=None, stream=None):
    """The allocation-free nested-loop join: pairs go to the caller's `out`
    (a (cap, 2) int32 CUDA tensor); returns the filled view."""
    if out is None:
        raise ValueError("jn_nested_loop_noalloc writes to a caller buffer: pass out=")
    if (out.dtype != torch.int32 or out.dim() != 2 or out.shape[1] != 2 or not out.is_contiguous()
            or not out.is_cuda):
        raise ValueError("out must be a contiguous (capacity, 2) int32 CUDA tensor")
    for c in R.refs + S.refs:
        if c is not None and c.device != out.device:
            raise ValueError("columns and out must be on the same CUDA device")
    n = ctypes.c_uint64()
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load().jn_nested_loop_noalloc(ctypes.byref(R.t), ctypes.byref(S.t),
                                       ctypes.byref(pr) if pr is not None else None, _P(out.data_ptr()),
                                       out.shape[0], ctypes.byref(n), _P(st.cuda_stream))
    if rc != JN_OK:
        raise JoinError(rc, load().jn_status_str(rc).decode(), int(n.value) if rc == JN_ERR_CAPACITY else None)
    return out[:int(n.value)]


def jn_autotune(ctx: Context, algo: int, R: TableRef, S: TableRef, pr: Pred = None) -> dict:
    """Times candidate tunings through the count pass; applies and returns the fastest."""
    t = Tuning()
    st = load().jn_autotune(ctx.handle, algo, ctypes.byref(R.t), ctypes.byref(S.t),
                            ctypes.byref(pr) if pr is not None else None, ctypes.byref(t))
    _check(ctx, st)
    return {f: getattr(t, f) for f, _ in Tuning._fields_ if f != "reserved"}


def jn_autotune_batch(ctx: Context, joins) -> dict:
    n = len(joins)
    arr = (Join * max(n, 1))()
    for i, (R, S, op, band) in enumerate(joins):
        arr[i] = Join(R.t, S.t, op, 0, band)
    t = Tuning()
    _check(ctx, load().jn_autotune_batch(ctx.handle, n, arr, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in Tuning._fields_ if f != "reserved"}


def jn_batch_count(ctx: Context, joins) -> list:
    """Per-join result sizes of a batch [(R, S, op, band), ...] without emitting pairs."""
    n = len(joins)
    arr = (Join * max(n, 1))()
    for i, (R, S, op, band) in enumerate(joins):
        arr[i] = Join(R.t, S.t, op, 0, band)
    cnt = (ctypes.c_uint64 * max(n, 1))()
    _check(ctx, load().jn_batch_count(ctx.handle, n, arr, cnt, None))
    return [int(cnt[i]) for i in range(n)]


def jn_selftest_wait(ctx: Context, polls: int, arrive: bool):
    """Runs the bounded-wait diagnostic; returns (status, elapsed_ns) without raising."""
    ns = ctypes.c_uint64(0)
    st = load().jn_selftest_wait(ctx.handle, polls, 1 if arrive else 0, ctypes.byref(ns))
    return int(st), int(ns.value)
