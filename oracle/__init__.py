"""CPU oracle for the join path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product library never does: it
shares no code with the oracle, and the oracle never imports the product.

``jn_oracle.c`` holds the plain definitions (see its header); this module
compiles it with gcc into ``oracle/_build/libjn_oracle.so`` and wraps each
function for numpy arrays.  Inputs are numpy arrays (int32 or int64 keys,
int32 payloads or None for "payload = row index").  Pairs come back as an
(n, 2) int32 array of (r, s).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jn_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libjn_oracle.so")

EQ, NE, LT, LE, GT, GE, ANY = range(7)
OPS = {"=": EQ, "!=": NE, "<": LT, "<=": LE, ">": GT, ">=": GE, "any": ANY}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no target-specific flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I64, U64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
        lib.or_nested_loop.restype = U64
        lib.or_nested_loop.argtypes = [P, P, P, I64, P, P, P, I64, I, I, I, I64, P, U64]
        lib.or_hash_join.restype = U64
        lib.or_hash_join.argtypes = [P, P, I64, P, P, I64, I, P, U64]
        lib.or_sort_merge_join.restype = U64
        lib.or_sort_merge_join.argtypes = [P, P, I64, P, P, I64, I, P, U64]
        lib.or_checksum_pairs.restype = U64
        lib.or_checksum_pairs.argtypes = [P, U64]
        lib.or_mix64.restype = U64
        lib.or_mix64.argtypes = [U64]
        lib.or_f.restype = U64
        lib.or_f.argtypes = [ctypes.c_int32]
        lib.or_g.restype = U64
        lib.or_g.argtypes = [ctypes.c_int32]
        lib.or_equi_count_checksum.restype = None
        lib.or_equi_count_checksum.argtypes = [P, P, I64, P, P, I64, I, P, P]
        lib.or_band_join_sorted.restype = U64
        lib.or_band_join_sorted.argtypes = [P, P, P, I64, P, P, P, I64, I, I, I64, P, U64]
        lib.or_band_count_sweep.restype = U64
        lib.or_band_count_sweep.argtypes = [P, P, I64, P, P, I64, I, I, I64]
        lib.or_prefilter_grouped_join.restype = U64
        lib.or_prefilter_grouped_join.argtypes = [P, P, I64, P, P, I64, I, I64, P, U64, P, P]
        lib.or_theta_regions.restype = U64
        lib.or_theta_regions.argtypes = [P, P, I64, P, P, I64, I, I, I64, P, U64, P, P]
        lib.or_thread_ranges.restype = None
        lib.or_thread_ranges.argtypes = [I64, I64, P, P]
        lib.or_star_nested_loop.restype = U64
        lib.or_star_nested_loop.argtypes = [P, P, P, I64, P, P, I64, P, P, I64, I, P, U64]
        _lib = lib
    return _lib


def _keys(a):
    a = np.ascontiguousarray(a)
    if a.dtype not in (np.int32, np.int64):
        raise TypeError("keys must be int32 or int64")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _pay(p, n):
    if p is None:
        return None
    p = np.ascontiguousarray(p, dtype=np.int32)
    assert p.shape[0] == n
    return p


def _ksize(*cols):
    ks = {c.dtype.itemsize for c in cols if c is not None}
    if len(ks) != 1:
        raise TypeError("all key columns must share one type")
    return ks.pop()


def _two_call(fn, *args):
    """Run an emitting oracle function: count first, then fill exactly."""
    total = fn(*args, None, 0)
    if total == 2 ** 64 - 1:
        raise ValueError("oracle rejected the arguments")
    out = np.empty((max(total, 1), 2), dtype=np.int32)
    again = fn(*args, out.ctypes.data, total)
    assert again == total
    return out[:total]


def nested_loop(rkey, skey, rkey2=None, skey2=None, rpay=None, spay=None,
                op_a=EQ, op_k=ANY, band=-1, count_only=False):
    """O1/O3: nested-loop join with a one- or two-column predicate."""
    lib = _load()
    rkey, skey = _keys(rkey), _keys(skey)
    rkey2 = None if rkey2 is None else _keys(rkey2)
    skey2 = None if skey2 is None else _keys(skey2)
    ks = _ksize(rkey, skey, rkey2, skey2)
    rp, sp = _pay(rpay, len(rkey)), _pay(spay, len(skey))
    args = (_ptr(rkey), _ptr(rkey2), _ptr(rp), len(rkey),
            _ptr(skey), _ptr(skey2), _ptr(sp), len(skey), ks, op_a, op_k, band)
    if count_only:
        return int(lib.or_nested_loop(*args, None, 0))
    return _two_call(lib.or_nested_loop, *args)


def star_join(rfk1, rfk2, s1key, s2key, rpay=None, s1pay=None, s2pay=None, count_only=False):
    """O6: star join of R (two join columns) with S1 on fk1 and S2 on fk2, as
    three nested loops; (n, 3) int32 triples (r, s1, s2)."""
    lib = _load()
    rfk1, rfk2, s1key, s2key = _keys(rfk1), _keys(rfk2), _keys(s1key), _keys(s2key)
    ks = _ksize(rfk1, rfk2, s1key, s2key)
    assert len(rfk1) == len(rfk2)
    rp, p1, p2 = _pay(rpay, len(rfk1)), _pay(s1pay, len(s1key)), _pay(s2pay, len(s2key))
    args = (_ptr(rfk1), _ptr(rfk2), _ptr(rp), len(rfk1), _ptr(s1key), _ptr(p1), len(s1key),
            _ptr(s2key), _ptr(p2), len(s2key), ks)
    total = int(lib.or_star_nested_loop(*args, None, 0))
    if count_only:
        return total
    out = np.empty((max(total, 1), 3), dtype=np.int32)
    assert lib.or_star_nested_loop(*args, out.ctypes.data, total) == total
    return out[:total]


def hash_join(rkey, skey, rpay=None, spay=None, count_only=False):
    """O2: chained hash join, build on R, probe with S."""
    lib = _load()
    rkey, skey = _keys(rkey), _keys(skey)
    ks = _ksize(rkey, skey)
    rp, sp = _pay(rpay, len(rkey)), _pay(spay, len(skey))
    args = (_ptr(rkey), _ptr(rp), len(rkey), _ptr(skey), _ptr(sp), len(skey), ks)
    if count_only:
        return int(lib.or_hash_join(*args, None, 0))
    return _two_call(lib.or_hash_join, *args)


def sort_merge_join(rkey, skey, rpay=None, spay=None, count_only=False):
    """O5: sort-merge equi join (sort both tables, walk them in key order)."""
    lib = _load()
    rkey, skey = _keys(rkey), _keys(skey)
    ks = _ksize(rkey, skey)
    rp, sp = _pay(rpay, len(rkey)), _pay(spay, len(skey))
    args = (_ptr(rkey), _ptr(rp), len(rkey), _ptr(skey), _ptr(sp), len(skey), ks)
    if count_only:
        return int(lib.or_sort_merge_join(*args, None, 0))
    return _two_call(lib.or_sort_merge_join, *args)


def band_join_sorted(rkey, rkey2, skey, skey2, op_a, band, rpay=None, spay=None,
                     count_only=False):
    """O4: band join by sorting S on key2 and binary search per R row."""
    lib = _load()
    cols = [_keys(c) for c in (rkey, rkey2, skey, skey2)]
    ks = _ksize(*cols)
    rp, sp = _pay(rpay, len(cols[0])), _pay(spay, len(cols[2]))
    args = (_ptr(cols[0]), _ptr(cols[1]), _ptr(rp), len(cols[0]),
            _ptr(cols[2]), _ptr(cols[3]), _ptr(sp), len(cols[2]), ks, op_a, band)
    if count_only:
        return int(lib.or_band_join_sorted(*args, None, 0))
    return _two_call(lib.or_band_join_sorted, *args)


def band_count_sweep(rkey, rkey2, skey, skey2, op_a, band):
    """Exact band-join size by the Fenwick dominance sweep."""
    lib = _load()
    cols = [_keys(c) for c in (rkey, rkey2, skey, skey2)]
    ks = _ksize(*cols)
    v = lib.or_band_count_sweep(_ptr(cols[0]), _ptr(cols[1]), len(cols[0]),
                                _ptr(cols[2]), _ptr(cols[3]), len(cols[2]), ks, op_a, band)
    if v == 2 ** 64 - 1:
        raise ValueError("unsupported op for the sweep")
    return int(v)


def equi_count_checksum(rkey, skey, rpay=None, spay=None):
    """Closed-form equi-join size and separable checksum from key groups."""
    lib = _load()
    rkey, skey = _keys(rkey), _keys(skey)
    ks = _ksize(rkey, skey)
    rp, sp = _pay(rpay, len(rkey)), _pay(spay, len(skey))
    c = ctypes.c_uint64()
    h = ctypes.c_uint64()
    lib.or_equi_count_checksum(_ptr(rkey), _ptr(rp), len(rkey), _ptr(skey), _ptr(sp),
                               len(skey), ks, ctypes.byref(c), ctypes.byref(h))
    return int(c.value), int(h.value)


def checksum_pairs(pairs) -> int:
    """Separable checksum of a result multiset, by its definition."""
    lib = _load()
    p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    return int(lib.or_checksum_pairs(_ptr(p), p.shape[0]))


def f_mix(r: int) -> int:
    return int(_load().or_f(r))


def g_mix(s: int) -> int:
    return int(_load().or_g(s))


def prefilter_grouped_join(rkey, skey, alpha, rpay=None, spay=None):
    """Algorithm 1 (two Map-Reduce rounds) then per-group NLJ.

    Returns (pairs, rsize, survivors): rsize is Eq. (rsize)'s storage bound
    (sum over groups of |T'_i| * |S'_i|), survivors the tuples kept by the
    pre-filter.
    """
    lib = _load()
    rkey, skey = _keys(rkey), _keys(skey)
    ks = _ksize(rkey, skey)
    rp, sp = _pay(rpay, len(rkey)), _pay(spay, len(skey))
    rs = ctypes.c_uint64()
    sv = ctypes.c_uint64()
    args = (_ptr(rkey), _ptr(rp), len(rkey), _ptr(skey), _ptr(sp), len(skey), ks, alpha)
    total = lib.or_prefilter_grouped_join(*args, None, 0, ctypes.byref(rs), ctypes.byref(sv))
    out = np.empty((max(total, 1), 2), dtype=np.int32)
    again = lib.or_prefilter_grouped_join(*args, out.ctypes.data, total,
                                          ctypes.byref(rs), ctypes.byref(sv))
    assert again == total
    return out[:total], int(rs.value), int(sv.value)


def theta_regions(rkey, skey, op, kq, rpay=None, spay=None):
    """Algorithm 3 with kq ranges: returns (pairs, region_kind, stats)."""
    lib = _load()
    rkey, skey = _keys(rkey), _keys(skey)
    ks = _ksize(rkey, skey)
    rp, sp = _pay(rpay, len(rkey)), _pay(spay, len(skey))
    st = np.zeros(3, dtype=np.uint64)
    args = (_ptr(rkey), _ptr(rp), len(rkey), _ptr(skey), _ptr(sp), len(skey), ks, op, kq)
    total = lib.or_theta_regions(*args, None, 0, None, st.ctypes.data)
    out = np.empty((max(total, 1), 2), dtype=np.int32)
    kind = np.empty(max(total, 1), dtype=np.uint8)
    again = lib.or_theta_regions(*args, out.ctypes.data, total, kind.ctypes.data, st.ctypes.data)
    assert again == total
    return out[:total], kind[:total], [int(x) for x in st]


def thread_ranges(n, threads):
    """Per-thread [begin, end) rows of Eqs. (NBS)/(IDS) with the clamp at n."""
    lib = _load()
    b = np.empty(threads, dtype=np.int64)
    e = np.empty(threads, dtype=np.int64)
    lib.or_thread_ranges(n, threads, b.ctypes.data, e.ctypes.data)
    return b, e


def sort_pairs(p) -> np.ndarray:
    """Canonical order of a pair multiset: by r, then s."""
    p = np.asarray(p, dtype=np.int32).reshape(-1, 2)
    if p.shape[0] == 0:
        return p
    key = (p[:, 0].astype(np.int64) << 32) | (p[:, 1].astype(np.int64) & 0xFFFFFFFF)
    return p[np.argsort(key, kind="stable")]
