"""GPU parity: the CUDA join path (through the C ABI) against the CPU oracle.

Every comparison is exact: result multisets of (r, s) pairs are compared
after sorting (output order is unspecified), counts and separable checksums
must be equal.  Inputs come from the seeded generators only.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_11201_gb300 import build as B
from paper_1904_11201_gb300 import datagen
from paper_1904_11201_gb300 import jn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
I32_MIN, I32_MAX = -(2 ** 31), 2 ** 31 - 1
I64_MIN, I64_MAX = -(2 ** 63), 2 ** 63 - 1


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = jn.Context(0)
    yield c
    c.close()


def canon(p):
    if isinstance(p, torch.Tensor):
        p = p.cpu().numpy()
    return O.sort_pairs(p)


def keys(n, lo, hi, seed, stream, dtype=torch.int32):
    return datagen.uniform_keys(n, lo, hi, seed, stream, dtype=dtype)


def with_edges(t, edges, seed):
    t = t.clone()
    if t.numel():
        idx = datagen.uniform_int(len(edges), 0, t.numel(), seed, 77, dtype=torch.int64)
        for i, v in zip(idx.tolist(), edges):
            t[i] = v
    return t


# ------------------------------------------------------ config 1 (16K x 64K) --

def test_uniform_16k_64k_hash_and_nested_loop(ctx):
    r = keys(16384, 0, 65536, 0, 0)
    s = keys(65536, 0, 65536, 0, 1)
    rp, sp = datagen.row_ids(16384), datagen.row_ids(65536)
    exp = canon(O.hash_join(r.numpy(), s.numpy(), rp.numpy(), sp.numpy()))
    R = jn.table(r.to(DEV), payload=rp.to(DEV))
    S = jn.table(s.to(DEV), payload=sp.to(DEV))
    assert np.array_equal(canon(jn.jn_hash(ctx, R, S)), exp)
    assert np.array_equal(canon(jn.jn_nested_loop(ctx, R, S)), exp)
    assert jn.jn_count(ctx, jn.JN_ALGO_HASH, R, S) == exp.shape[0]
    assert jn.jn_count(ctx, jn.JN_ALGO_NLJ, R, S) == exp.shape[0]
    cnt, chk = O.equi_count_checksum(r.numpy(), s.numpy(), rp.numpy(), sp.numpy())
    assert jn.jn_aggregate(ctx, jn.JN_ALGO_HASH, R, S) == (cnt, chk)
    assert jn.jn_aggregate(ctx, jn.JN_ALGO_NLJ, R, S) == (cnt, chk)


# --------------------------------------------------------- hash join cases --

HASH_CASES = [
    # (nr, ns, lo, hi, dtype)
    (0, 100, 0, 10, torch.int32),
    (100, 0, 0, 10, torch.int32),
    (1, 1, 5, 6, torch.int32),
    (64, 64, 7, 8, torch.int32),              # all keys equal: full Cartesian product
    (1000, 3001, 0, 1 << 20, torch.int32),    # mostly misses
    (4097, 12289, 0, 300, torch.int32),       # many duplicates, ragged sizes
    (20000, 50001, I32_MIN, I32_MAX, torch.int32),
    (5003, 7001, 0, 1000, torch.int64),
    (30000, 20000, I64_MIN // 4, I64_MAX // 4, torch.int64),
]


def reported_prefilter(path, pre, nr, ns):
    """Tables the pre-filter thins, as jn_run_info reports it: the two-pass path
    filters what it is asked to; the region path filters one table (the larger
    one, S on a tie, when both are asked for)."""
    if path == 1 or pre in (0, 2, 3):
        return pre
    return 2 if ns >= nr else 3


@pytest.mark.parametrize("case", HASH_CASES)
@pytest.mark.parametrize("pre", [0, 1, 2, 3])  # off, both tables, only S, only R
@pytest.mark.parametrize("path", [1, 2])        # two radix passes, regions
def test_hash_cases(ctx, case, pre, path):
    nr, ns, lo, hi, dt = case
    r = keys(nr, lo, hi, 3, 0, dt)
    s = keys(ns, lo, hi, 3, 1, dt)
    if dt == torch.int32:
        r, s = with_edges(r, [I32_MIN, I32_MAX], 5), with_edges(s, [I32_MAX, I32_MIN], 6)
    else:
        r, s = with_edges(r, [I64_MIN, I64_MAX], 5), with_edges(s, [I64_MAX, I64_MIN], 6)
    exp = canon(O.hash_join(r.numpy(), s.numpy()))
    ctx.set_tuning(prefilter=pre, hash_path=path)
    try:
        got = jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
        if nr and ns:
            info = ctx.run_info()
            assert info["prefilter"] == reported_prefilter(path, pre, nr, ns)
            assert info["hash_path"] == path
        c, h = jn.jn_aggregate(ctx, jn.JN_ALGO_HASH, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
    finally:
        ctx.set_tuning(prefilter=-1, hash_path=0)
    assert np.array_equal(canon(got), exp)
    assert c == exp.shape[0] and h == O.checksum_pairs(exp)


@pytest.mark.parametrize("sizes", [(1 << 20, (1 << 22) + 3, 2), ((1 << 22) + 5, 1 << 20, 3),
                                   ((1 << 21) + 7, (1 << 21) + 1, 1)])
@pytest.mark.parametrize("path", [1, 2])
def test_hash_auto_prefilter_sides(ctx, sizes, path):
    # the automatic choice filters only the larger table when one is 2x the
    # other; the region path always filters one table (the larger one)
    nr, ns, side = sizes
    r = keys(nr, 0, 1 << 23, 41, 0)
    s = keys(ns, 0, 1 << 23, 41, 1)
    exp = canon(O.hash_join(r.numpy(), s.numpy()))
    ctx.set_tuning(prefilter=-1, hash_path=path)
    try:
        got = jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
        assert ctx.run_info()["prefilter"] == reported_prefilter(path, side, nr, ns)
    finally:
        ctx.set_tuning(hash_path=0)
    assert np.array_equal(canon(got), exp)


@pytest.mark.parametrize("bits", [(1, 1), (3, 2), (5, 0), (12, 6), (16, 8), (18, 10), (19, 10)])
@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("table_rows", [0, 2048])
def test_hash_result_independent_of_partitioning(ctx, bits, path, table_rows):
    # partition bits, partition path and R rows per shared-memory table shape
    # the work, never the result (1 and 3 bits leave 9000-row partitions:
    # several table-sized items each)
    b, b1 = bits
    r = keys(30000, 0, 9000, 8, 0)
    s = keys(45000, 0, 9000, 8, 1)
    exp = canon(O.hash_join(r.numpy(), s.numpy()))
    ctx.set_tuning(radix_bits=b, radix_bits1=b1, prefilter=1, hash_path=path, table_rows=table_rows)
    try:
        got = jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
        info = ctx.run_info()
        # the region path holds up to 10 + 8 bits; beyond, two radix passes run
        taken = 1 if path == 1 or b - (b1 or min(b, 10)) > 8 else 2
        assert info["hash_path"] == taken
        assert info["table_rows"] == (table_rows or 4096)
    finally:
        ctx.set_tuning(radix_bits=0, radix_bits1=0, prefilter=-1, hash_path=0, table_rows=0)
    assert np.array_equal(canon(got), exp)


@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
@pytest.mark.parametrize("half", [False, True])
def test_table_rows_skewed_int64_and_sort_merge(ctx, dt, half):
    # the smaller table with frequent keys (the skewed build), int64 keys and
    # the sort-merge join, against the oracle's count and checksum and pairs
    nr, ns = 40000, 70000
    r = skewed(nr, 1 << 13, 1.0, 31, 0, dt)
    s = skewed(ns, 1 << 13, 1.0, 31, 1, dt)
    rp = datagen.uniform_int(nr, I32_MIN, I32_MAX, 31, 5)
    sp = datagen.uniform_int(ns, I32_MIN, I32_MAX, 31, 6)
    cnt, chk = O.equi_count_checksum(r.numpy(), s.numpy(), rp.numpy(), sp.numpy())
    R = jn.table(r.to(DEV), payload=rp.to(DEV))
    S = jn.table(s.to(DEV), payload=sp.to(DEV))
    full = 4096 if dt == torch.int32 else 2048
    rows = full // 2 if half else full
    for algo in (jn.JN_ALGO_HASH, jn.JN_ALGO_SORT):
        for heavy in (64, 0):
            ctx.set_tuning(table_rows=rows, heavy=heavy, radix_bits=4)
            try:
                assert jn.jn_aggregate(ctx, algo, R, S) == (cnt, chk)
                assert ctx.run_info()["table_rows"] == rows
                got = jn.jn_hash(ctx, R, S) if algo == jn.JN_ALGO_HASH else jn.jn_sort_merge(ctx, R, S)
            finally:
                ctx.set_tuning(table_rows=0, heavy=-1, radix_bits=0)
            assert got.shape[0] == cnt and O.checksum_pairs(got.cpu().numpy()) == chk


@pytest.mark.parametrize("sms", [1, 37, 100000])
def test_sm_budget_never_changes_results(ctx, sms):
    # grids sized for fewer SMs (or more than the device has) do the same work
    r = skewed(60000, 1 << 14, 0.8, 81, 0)
    s = skewed(90000, 1 << 14, 0.8, 81, 1)
    ra, rk = datagen.band_columns(5000, 14, seed=81, stream=2)
    sa, sk = datagen.band_columns(9000, 14, seed=81, stream=3)
    ctx.set_tuning(sms=sms)
    try:
        assert ctx.tuning()["sms"] == sms
        got = jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
        gotb = jn.jn_theta(ctx, jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV)), jn.JN_LT, 9)
    finally:
        ctx.set_tuning(sms=0)
    assert np.array_equal(canon(got), canon(O.hash_join(r.numpy(), s.numpy())))
    assert np.array_equal(canon(gotb), canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(),
                                                                O.LT, 9)))


def test_table_rows_rejected_or_taken_as_the_nearer_size(ctx):
    # jn_set_tuning takes 0, 1024, 2048 and 4096; a join takes a size outside
    # its key type's two (full, half) as the nearer one, so one context tuned
    # for int32 keys still joins int64 keys
    for bad in (-1, 1000, 3072, 8192):
        with pytest.raises(jn.JoinError):
            ctx.set_tuning(table_rows=bad)
    for dt, rows, used in ((torch.int32, 1024, 2048), (torch.int64, 4096, 2048), (torch.int64, 1024, 1024)):
        r = keys(5000, 0, 900, 9, 0, dt)
        s = keys(7000, 0, 900, 9, 1, dt)
        ctx.set_tuning(table_rows=rows)
        try:
            got = jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
            assert ctx.run_info()["table_rows"] == used
        finally:
            ctx.set_tuning(table_rows=0)
        assert np.array_equal(canon(got), canon(O.hash_join(r.numpy(), s.numpy())))


@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
@pytest.mark.parametrize("pre", [0, 2, 3])
def test_region_path_many_chunks_ragged(ctx, dt, pre):
    # level-1 chunks of several tiles, a ragged last tile in every chunk and
    # region, both filter directions, payloads off a 16-byte boundary
    nr, ns = 3 * 8192 * 152 + 4099, 2 * 8192 * 152 + 777
    r = keys(nr, 0, 1 << 22, 13, 0, dt)
    s = keys(ns, 0, 1 << 22, 13, 1, dt)
    rp = datagen.uniform_int(nr + 1, I32_MIN, I32_MAX, 13, 2)
    sp = datagen.uniform_int(ns + 3, I32_MIN, I32_MAX, 13, 3)
    rpd, spd = rp.to(DEV), sp.to(DEV)
    R = jn.table(r.to(DEV), payload=rpd[1:])
    S = jn.table(s.to(DEV), payload=spd[3:])
    cnt, chk = O.equi_count_checksum(r.numpy(), s.numpy(), rp[1:].numpy(), sp[3:].numpy())
    ctx.set_tuning(prefilter=pre, hash_path=2)
    try:
        got = jn.jn_hash(ctx, R, S)
        info = ctx.run_info()
        assert info["hash_path"] == 2 and info["prefilter"] == pre
        agg = jn.jn_aggregate(ctx, jn.JN_ALGO_HASH, R, S)
    finally:
        ctx.set_tuning(prefilter=-1, hash_path=0)
    assert agg == (cnt, chk)
    assert got.shape[0] == cnt and O.checksum_pairs(got.cpu().numpy()) == chk
    exp = canon(O.hash_join(r.numpy(), s.numpy(), rp[1:].numpy(), sp[3:].numpy()))
    assert np.array_equal(canon(got), exp)
    # rows kept: every non-heavy row of the unfiltered table, a superset of the
    # rows with a common key in the filtered one
    kept = (info["r_survivors"], info["s_survivors"])
    common_r = int(np.isin(r.numpy(), s.numpy()).sum())
    common_s = int(np.isin(s.numpy(), r.numpy()).sum())
    assert kept[0] >= common_r and kept[1] >= common_s
    if pre == 0:
        assert kept == (nr, ns)


def test_hash_unaligned_and_host_columns(ctx):
    r = keys(10001, 0, 2000, 9, 0)
    s = keys(20003, 0, 2000, 9, 1)
    rp = datagen.uniform_int(10001, I32_MIN, I32_MAX, 9, 2)
    sp = datagen.uniform_int(20003, I32_MIN, I32_MAX, 9, 3)
    exp = canon(O.hash_join(r[1:].numpy(), s[3:].numpy(), rp[1:].numpy(), sp[3:].numpy()))
    # device columns starting off a 16-byte boundary
    rd, sd, rpd, spd = r.to(DEV), s.to(DEV), rp.to(DEV), sp.to(DEV)
    got = jn.jn_hash(ctx, jn.table(rd[1:], payload=rpd[1:]), jn.table(sd[3:], payload=spd[3:]))
    assert np.array_equal(canon(got), exp)
    # host (pageable and pinned) columns, host output buffer
    out = torch.empty((exp.shape[0] + 5, 2), dtype=torch.int32)
    got = jn.jn_hash(ctx, jn.table(r[1:].clone(), payload=rp[1:].clone()),
                     jn.table(s[3:].clone().pin_memory(), payload=sp[3:].clone()), out=out)
    assert np.array_equal(canon(got), exp)
    # page-locked host columns read in place (off a 16-byte boundary too) and a
    # page-locked host output written in place
    rh, sh = r.clone().pin_memory(), s.clone().pin_memory()
    rph, sph = rp.clone().pin_memory(), sp.clone().pin_memory()
    outp = torch.empty((exp.shape[0] + 5, 2), dtype=torch.int32).pin_memory()
    r2 = keys(300000, 0, 5000, 19, 0).pin_memory()
    s2 = keys(200000, 0, 5000, 19, 1).pin_memory()
    exp2 = canon(O.hash_join(r2.numpy(), s2.numpy()))
    for io in (1, 2, 3):
        ctx.set_tuning(host_io=io)
        try:
            got = jn.jn_hash(ctx, jn.table(rh[1:], payload=rph[1:]), jn.table(sh[3:], payload=sph[3:]), out=outp)
            assert np.array_equal(canon(got), exp)
            # the heavy-key path, more rows than one tile of a pass
            ctx.set_tuning(heavy=64)
            out2 = torch.empty((exp2.shape[0], 2), dtype=torch.int32).pin_memory()
            got = jn.jn_hash(ctx, jn.table(r2), jn.table(s2), out=out2)
            assert np.array_equal(canon(got), exp2)
        finally:
            ctx.set_tuning(heavy=-1, host_io=0)


def test_host_mapped_outputs_band_and_nested_loop(ctx):
    ra, rk = datagen.band_columns(3000, 12, seed=44, stream=0)
    sa, sk = datagen.band_columns(7000, 12, seed=44, stream=1)
    exp = canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.GT, 3))
    R = jn.table(ra.to(DEV), rk.to(DEV))
    S = jn.table(sa.to(DEV), sk.to(DEV))
    out = torch.empty((exp.shape[0], 2), dtype=torch.int32).pin_memory()
    ctx.set_tuning(host_io=2)
    try:
        assert np.array_equal(canon(jn.jn_theta(ctx, R, S, jn.JN_GT, 3, out=out)), exp)
        out.zero_()
        assert np.array_equal(canon(jn.jn_nested_loop(ctx, R, S, jn.pred(jn.JN_GT, jn.JN_ANY, 3), out=out)), exp)
    finally:
        ctx.set_tuning(host_io=0)
    # pinned host columns on the paths that copy them
    Rh = jn.table(ra.pin_memory(), rk.pin_memory())
    Sh = jn.table(sa.pin_memory(), sk.pin_memory())
    assert np.array_equal(canon(jn.jn_theta(ctx, Rh, Sh, jn.JN_GT, 3)), exp)


def test_capacity_error_writes_nothing(ctx):
    r = keys(3000, 0, 100, 10, 0)
    s = keys(3000, 0, 100, 10, 1)
    m = O.hash_join(r.numpy(), s.numpy(), count_only=True)
    out = torch.full((m - 1, 2), -7, dtype=torch.int32, device=DEV)
    with pytest.raises(jn.JoinError) as e:
        jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)), out=out)
    assert e.value.status == jn.JN_ERR_CAPACITY and e.value.required == m
    assert bool((out == -7).all())
    out = torch.empty((m, 2), dtype=torch.int32, device=DEV)
    got = jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)), out=out)
    assert np.array_equal(canon(got), canon(O.hash_join(r.numpy(), s.numpy())))


def test_invalid_arguments(ctx):
    r = keys(10, 0, 5, 1, 0)
    s = keys(10, 0, 5, 1, 1, torch.int64)
    with pytest.raises(jn.JoinError) as e:
        jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
    assert e.value.status == jn.JN_ERR_INVALID
    with pytest.raises(jn.JoinError) as e:
        jn.jn_count(ctx, jn.JN_ALGO_HASH, jn.table(r.to(DEV)), jn.table(r.to(DEV)), jn.pred(jn.JN_LT))
    assert e.value.status == jn.JN_ERR_UNSUPPORTED
    with pytest.raises(jn.JoinError) as e:  # band needs key2
        jn.jn_theta(ctx, jn.table(r.to(DEV)), jn.table(r.to(DEV)), jn.JN_LT, 3)
    assert e.value.status == jn.JN_ERR_INVALID


# --------------------------------------------------- nested loop predicates --

@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
def test_nested_loop_all_predicates(ctx, dt):
    nr, ns = 700, 2100
    ra, rk = keys(nr, -20, 20, 11, 0, dt), keys(nr, -50, 50, 11, 1, dt)
    sa, sk = keys(ns, -20, 20, 11, 2, dt), keys(ns, -50, 50, 11, 3, dt)
    lo, hi = (I32_MIN, I32_MAX) if dt == torch.int32 else (I64_MIN, I64_MAX)
    ra, sa = with_edges(ra, [lo, hi], 1), with_edges(sa, [hi, lo], 2)
    rk, sk = with_edges(rk, [hi, lo], 3), with_edges(sk, [lo, hi], 4)
    R = jn.table(ra.to(DEV), rk.to(DEV))
    S = jn.table(sa.to(DEV), sk.to(DEV))
    for op_a in range(7):
        for op_k in range(7):
            exp = O.nested_loop(ra.numpy(), sa.numpy(), rk.numpy(), sk.numpy(), op_a=op_a, op_k=op_k,
                                count_only=True)
            got = jn.jn_count(ctx, jn.JN_ALGO_NLJ, R, S, jn.pred(op_a, op_k))
            assert got == exp, (op_a, op_k)
    for op_a, op_k, band in [(jn.JN_LT, 0, 5), (jn.JN_NE, 0, 0), (jn.JN_GE, 0, 2 ** 40), (jn.JN_EQ, 5, -1),
                             (jn.JN_ANY, jn.JN_GT, -1), (jn.JN_LE, jn.JN_NE, -1)]:
        exp = canon(O.nested_loop(ra.numpy(), sa.numpy(), rk.numpy(), sk.numpy(), op_a=op_a,
                                  op_k=op_k, band=band))
        got = jn.jn_nested_loop(ctx, R, S, jn.pred(op_a, op_k, band))
        assert np.array_equal(canon(got), exp), (op_a, op_k, band)
        c, h = jn.jn_aggregate(ctx, jn.JN_ALGO_NLJ, R, S, jn.pred(op_a, op_k, band))
        assert c == exp.shape[0] and h == O.checksum_pairs(exp)


@pytest.mark.parametrize("tile_r", [0, 512, 4096])
def test_nested_loop_conjunctive_band_64k_scaled(ctx, tile_r):
    # the two-column band predicate of the 64K x 1M tiled workload, at 8K x 64K
    # (plus ragged tails), for the default and the smallest and largest R tiles
    nr, ns, w = 8192 + 77, 65536 + 1001, 24414 // 16
    ra, rk = datagen.band_columns(nr, 24, seed=4, stream=0)
    sa, sk = datagen.band_columns(ns, 24, seed=4, stream=1)
    exp = canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.LT, w))
    ctx.set_tuning(nlj_tile_r=tile_r)
    try:
        R, S = jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV))
        got = jn.jn_nested_loop(ctx, R, S, jn.pred(jn.JN_LT, jn.JN_ANY, w))
        assert jn.jn_count(ctx, jn.JN_ALGO_NLJ, R, S, jn.pred(jn.JN_LT, jn.JN_ANY, w)) == exp.shape[0]
    finally:
        ctx.set_tuning(nlj_tile_r=0)
    assert np.array_equal(canon(got), exp)


# -------------------------------------------------------------- theta / band --

@pytest.mark.parametrize("op", [jn.JN_LT, jn.JN_LE, jn.JN_GT, jn.JN_GE, jn.JN_EQ, jn.JN_NE, jn.JN_ANY])
def test_band_join_all_ops(ctx, op):
    nr, ns, w = 1 << 13, 1 << 16, 40
    ra, rk = datagen.band_columns(nr, 16, seed=5, stream=0)
    sa, sk = datagen.band_columns(ns, 16, seed=5, stream=1)
    exp = canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), op, w))
    R = jn.table(ra.to(DEV), rk.to(DEV))
    S = jn.table(sa.to(DEV), sk.to(DEV))
    got = jn.jn_theta(ctx, R, S, op, w)
    assert np.array_equal(canon(got), exp)
    c, h = jn.jn_aggregate(ctx, jn.JN_ALGO_THETA, R, S, jn.pred(op, jn.JN_ANY, w))
    assert c == exp.shape[0] and h == O.checksum_pairs(exp)


@pytest.mark.parametrize("band", [0, 1, 1000, 70000, 2 ** 33])
@pytest.mark.parametrize("groups", [0, 2, 10])
def test_band_join_widths_and_groups(ctx, band, groups):
    nr, ns = 3000, 9000
    ra, rk = keys(nr, 0, 100, 6, 0), keys(nr, -40000, 40000, 6, 1)
    sa, sk = keys(ns, 0, 100, 6, 2), keys(ns, -40000, 40000, 6, 3)
    rk, sk = with_edges(rk, [I32_MIN, I32_MAX], 8), with_edges(sk, [I32_MAX, I32_MIN], 9)
    exp = canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.GE, band))
    ctx.set_tuning(theta_groups=groups)
    try:
        got = jn.jn_theta(ctx, jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV)),
                          jn.JN_GE, band)
    finally:
        ctx.set_tuning(theta_groups=0)
    assert np.array_equal(canon(got), exp)


@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
@pytest.mark.parametrize("n", [1, 7, 1000, 300001])
def test_band_groups_follow_the_key_range(ctx, dt, n):
    # the groups cut [min k, max k] over both tables: with correct extremes a
    # narrow band compares each S group with about three R groups, far fewer
    # than |R| * |S| pairs; column lengths leave most threads of the min/max
    # reduction without elements, and the columns start off a 16-byte boundary
    nr, ns = n, 2 * n + 5
    ra, rk = keys(nr + 1, 0, 100, 29, 0, dt), keys(nr + 1, -(1 << 30), 1 << 30, 29, 1, dt)
    sa, sk = keys(ns, 0, 100, 29, 2, dt), keys(ns, -(1 << 30), 1 << 30, 29, 3, dt)
    R = jn.table(ra[1:].to(DEV), rk[1:].to(DEV))
    S = jn.table(sa.to(DEV), sk.to(DEV))
    exp = canon(O.band_join_sorted(ra[1:].numpy(), rk[1:].numpy(), sa.numpy(), sk.numpy(), O.LT, 7))
    assert np.array_equal(canon(jn.jn_theta(ctx, R, S, jn.JN_LT, 7)), exp)
    info = ctx.run_info()
    assert info["partitions"] >= 4
    if n >= 1000:
        assert info["cartesian_bound"] <= nr * ns * 8 // info["partitions"]


@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
@pytest.mark.parametrize("op", [jn.JN_LT, jn.JN_NE])
def test_band_join_narrow_and_wide_items(ctx, dt, op):
    # sparse R keys leave every S row a handful of candidates (its matches
    # are recorded by the count pass and gathered), except near a dense
    # cluster of R keys, where S rows have hundreds (those items are emitted
    # by testing again); several S chunks per group and a ragged last one
    nr, ns = 60000, 300000
    ra = keys(nr, 0, 1000, 23, 0, dt)
    rk = keys(nr, 0, 1 << 22, 23, 1, dt)
    rk[:3000] = keys(3000, 2000000, 2000040, 23, 2, dt)
    sa = keys(ns, 0, 1000, 23, 3, dt)
    sk = keys(ns, 0, 1 << 22, 23, 4, dt)
    sk[:5000] = keys(5000, 1999990, 2000050, 23, 5, dt)
    band = 20
    exp = canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), op, band))
    R = jn.table(ra.to(DEV), rk.to(DEV))
    S = jn.table(sa.to(DEV), sk.to(DEV))
    for groups in (0, 6, 10):
        ctx.set_tuning(theta_groups=groups)
        try:
            got = jn.jn_theta(ctx, R, S, op, band)
            cnt = jn.jn_count(ctx, jn.JN_ALGO_THETA, R, S, jn.pred(op, jn.JN_ANY, band))
        finally:
            ctx.set_tuning(theta_groups=0)
        assert cnt == exp.shape[0]
        assert np.array_equal(canon(got), exp)


@pytest.mark.parametrize("op", [jn.JN_LT, jn.JN_LE, jn.JN_GT, jn.JN_GE, jn.JN_EQ, jn.JN_NE, jn.JN_ANY])
@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
def test_one_column_theta_regions(ctx, op, dt):
    nr, ns = 900, 1300
    r = keys(nr, -3000, 3000, 12, 0, dt)
    s = keys(ns, -2000, 5000, 12, 1, dt)
    exp = canon(O.nested_loop(r.numpy(), s.numpy(), op_a=op))
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    got = jn.jn_theta(ctx, R, S, op, -1)
    assert np.array_equal(canon(got), exp)
    c, h = jn.jn_aggregate(ctx, jn.JN_ALGO_THETA, R, S, jn.pred(op, jn.JN_ANY, -1))
    assert c == exp.shape[0] and h == O.checksum_pairs(exp)


# ------------------------------------------------------------- skewed keys --

def skewed(n, d, theta, seed, stream, dtype=torch.int32):
    ranks = datagen.zipf_ranks(n, theta, d, seed, stream)
    if dtype == torch.int32:
        return datagen.rank_to_key32(ranks, 20, seed)
    return datagen.rank_to_key64(ranks, seed)


@pytest.mark.parametrize("theta", [0.5, 1.0])
@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
def test_hash_heavy_keys(ctx, theta, dt):
    nr, ns, d = 60000, 90000, 1 << 14
    r = skewed(nr, d, theta, 21, 0, dt)
    s = skewed(ns, d, theta, 21, 1, dt)
    rp = datagen.uniform_int(nr, I32_MIN, I32_MAX, 21, 5)
    sp = datagen.uniform_int(ns, I32_MIN, I32_MAX, 21, 6)
    cnt, chk = O.equi_count_checksum(r.numpy(), s.numpy(), rp.numpy(), sp.numpy())
    R = jn.table(r.to(DEV), payload=rp.to(DEV))
    S = jn.table(s.to(DEV), payload=sp.to(DEV))
    for heavy, pre, path in ((64, 1, 1), (0, 1, 1), (64, 2, 1), (64, 3, 1), (64, 1, 2), (0, 1, 2), (64, 3, 2),
                             (64, 0, 2)):
        ctx.set_tuning(heavy=heavy, prefilter=pre, hash_path=path)
        try:
            assert jn.jn_aggregate(ctx, jn.JN_ALGO_HASH, R, S) == (cnt, chk)
            info = ctx.run_info()
            if heavy:
                assert info["heavy_keys"] > 0
            if cnt <= 30_000_000:
                got = jn.jn_hash(ctx, R, S)
                assert got.shape[0] == cnt
                assert O.checksum_pairs(got.cpu().numpy()) == chk
        finally:
            ctx.set_tuning(heavy=-1, prefilter=-1, hash_path=0)
    if cnt <= 3_000_000:
        ctx.set_tuning(heavy=64)
        try:
            got = jn.jn_hash(ctx, R, S)
        finally:
            ctx.set_tuning(heavy=-1)
        exp = canon(O.hash_join(r.numpy(), s.numpy(), rp.numpy(), sp.numpy()))
        assert np.array_equal(canon(got), exp)


def test_hash_one_key_everywhere(ctx):
    # every row carries the same key: a single heavy key, output = |R| * |S|
    r = torch.full((3000,), 42, dtype=torch.int32)
    s = torch.full((5000,), 42, dtype=torch.int32)
    for heavy in (2, 0):
        ctx.set_tuning(heavy=heavy)
        try:
            got = jn.jn_hash(ctx, jn.table(r.to(DEV)), jn.table(s.to(DEV)))
        finally:
            ctx.set_tuning(heavy=-1)
        assert got.shape[0] == 3000 * 5000
        g = got.cpu().numpy()
        assert np.array_equal(np.bincount(g[:, 0], minlength=3000), np.full(3000, 5000))
        assert np.array_equal(np.bincount(g[:, 1], minlength=5000), np.full(5000, 3000))


# ------------------------------------------------------------------ batch --

@pytest.mark.parametrize("graphs", [0, 1])
def test_batch_matches_oracle_per_join(ctx, graphs):
    sizes = datagen.log_uniform_int(40, 1, 30000, seed=31, stream=0).tolist()
    sizes2 = datagen.log_uniform_int(40, 1, 50000, seed=31, stream=1).tolist()
    joins, exp, keep = [], [], []
    for i, (nr, ns) in enumerate(zip(sizes, sizes2)):
        if i % 3 == 2:  # band join
            ra, rk = datagen.band_columns(nr, 14, seed=40 + i, stream=0)
            sa, sk = datagen.band_columns(ns, 14, seed=40 + i, stream=1)
            w = i % 7
            keep.append((ra, rk, sa, sk))
            joins.append((jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV)), jn.JN_LT, w))
            exp.append(canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.LT, w)))
        else:
            d = max(16, (nr + ns) // (1 + i % 4))
            r = keys(nr, 0, d, 50 + i, 0)
            s = keys(ns, 0, d, 50 + i, 1)
            rp = datagen.uniform_int(nr, I32_MIN, I32_MAX, 60 + i, 2)
            keep.append((r, s, rp))
            joins.append((jn.table(r.to(DEV), payload=rp.to(DEV)), jn.table(s.to(DEV)), jn.JN_EQ, -1))
            exp.append(canon(O.hash_join(r.numpy(), s.numpy(), rp.numpy(), None)))
    ctx.set_tuning(graphs=graphs)
    try:
        pairs, first, cnt = jn.jn_batch(ctx, joins)
    finally:
        ctx.set_tuning(graphs=0)
    got = pairs.cpu().numpy()
    assert got.shape[0] == sum(cnt)
    for i in range(len(joins)):
        assert cnt[i] == exp[i].shape[0], i
        assert np.array_equal(canon(got[first[i]:first[i] + cnt[i]]), exp[i]), i
    # alone and in the batch: the same pairs
    for i in (0, 1, 2):
        R, S, op, band = joins[i]
        alone = jn.jn_hash(ctx, R, S) if band < 0 else jn.jn_theta(ctx, R, S, op, band)
        assert np.array_equal(canon(alone), exp[i])


def test_batch_capacity_and_empty(ctx):
    r = keys(1000, 0, 50, 70, 0)
    s = keys(1000, 0, 50, 70, 1)
    joins = [(jn.table(r.to(DEV)), jn.table(s.to(DEV)), jn.JN_EQ, -1),
             (jn.table(r[:0].to(DEV)), jn.table(s.to(DEV)), jn.JN_EQ, -1)]
    m = O.hash_join(r.numpy(), s.numpy(), count_only=True)
    small = torch.empty((m - 1, 2), dtype=torch.int32, device=DEV)
    with pytest.raises(jn.JoinError) as e:
        jn.jn_batch(ctx, joins, out=small)
    assert e.value.status == jn.JN_ERR_CAPACITY and e.value.required == m
    pairs, first, cnt = jn.jn_batch(ctx, joins)
    assert cnt == [m, 0]


def test_heavy_keys_are_the_most_frequent(ctx):
    # 3000 keys of 100 rows and one of 5000 rows on each side: more candidates
    # than the heavy set holds, so the threshold rises and the largest key is
    # taken (its 25M pairs go through the cross-product path)
    base = torch.arange(3000, dtype=torch.int32).repeat_interleave(100)
    big = torch.full((5000,), 7_777_777, dtype=torch.int32)
    r = torch.cat([base, big])[datagen.uniform_int(305000, 0, 1 << 30, 41, 0, dtype=torch.int64).argsort()]
    s = torch.cat([base, big])[datagen.uniform_int(305000, 0, 1 << 30, 41, 1, dtype=torch.int64).argsort()]
    cnt, chk = O.equi_count_checksum(r.numpy(), s.numpy())
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    ctx.set_tuning(heavy=64)
    try:
        assert jn.jn_aggregate(ctx, jn.JN_ALGO_HASH, R, S) == (cnt, chk)
        info = ctx.run_info()
        assert info["heavy_keys"] <= 1024
        assert info["heavy_pairs"] >= 5000 * 5000
    finally:
        ctx.set_tuning(heavy=-1)


def test_host_output_copied_back_in_slices(ctx):
    # more than 2^24 pairs into a host buffer: the emit pass runs in slices and
    # each slice's pairs are copied back while the next one emits
    r = keys(4_500_000, 0, 1 << 20, 51, 0)
    s = keys(4_500_000, 0, 1 << 20, 51, 1)
    cnt, chk = O.equi_count_checksum(r.numpy(), s.numpy())
    assert cnt >= 1 << 24
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    for pin in (False, True):
        out = torch.full((cnt + 3, 2), -1, dtype=torch.int32)
        if pin:
            out = out.pin_memory()
        got = jn.jn_hash(ctx, R, S, out=out)
        assert got.shape[0] == cnt
        assert O.checksum_pairs(got.numpy()) == chk
        assert bool((out[cnt:] == -1).all())
        # every pair joins equal keys
        g = got.long()
        assert torch.equal(r[g[:, 0]], s[g[:, 1]])


# ------------------------------------------------ Eq. (rsize) bound report --

def test_cartesian_bound_reports(ctx):
    # the bound the paper would allocate, against the exact count the joins use
    r = keys(30000, 0, 5000, 61, 0)
    s = keys(50000, 0, 5000, 61, 1)
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    n = O.hash_join(r.numpy(), s.numpy(), count_only=True)
    for pre, bits in ((0, 4), (1, 4), (0, 1)):
        ctx.set_tuning(prefilter=pre, radix_bits=bits)
        try:
            assert jn.jn_count(ctx, jn.JN_ALGO_HASH, R, S) == n
            info = ctx.run_info()
        finally:
            ctx.set_tuning(prefilter=-1, radix_bits=0)
        assert n <= info["cartesian_bound"] <= 30000 * 50000
    # one key on both sides: one partition (or the cross-product path) holds it all
    one_r, one_s = torch.full((3000,), 7, dtype=torch.int32), torch.full((2000,), 7, dtype=torch.int32)
    for heavy in (0, 64):
        ctx.set_tuning(heavy=heavy)
        try:
            assert jn.jn_count(ctx, jn.JN_ALGO_HASH, jn.table(one_r.to(DEV)), jn.table(one_s.to(DEV))) == 6_000_000
            assert ctx.run_info()["cartesian_bound"] == 6_000_000
        finally:
            ctx.set_tuning(heavy=-1)
    # disjoint keys, both tables filtered: nothing survives, nothing is allocated
    ctx.set_tuning(prefilter=1)
    try:
        assert jn.jn_count(ctx, jn.JN_ALGO_HASH, jn.table(keys(9000, 0, 100, 62, 0).to(DEV)),
                           jn.table(keys(9000, 200, 300, 62, 1).to(DEV))) == 0
        assert ctx.run_info()["cartesian_bound"] == 0
    finally:
        ctx.set_tuning(prefilter=-1)
    # the nested loop compares every pair; the theta join its regions
    ra, rk = datagen.band_columns(4000, 16, seed=63, stream=0)
    sa, sk = datagen.band_columns(9000, 16, seed=63, stream=1)
    RB, SB = jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV))
    pr = jn.pred(jn.JN_LT, jn.JN_ANY, 30)
    exp = O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.LT, 30, count_only=True)
    assert jn.jn_count(ctx, jn.JN_ALGO_NLJ, RB, SB, pr) == exp
    assert ctx.run_info()["cartesian_bound"] == 4000 * 9000
    assert jn.jn_count(ctx, jn.JN_ALGO_THETA, RB, SB, pr) == exp
    assert exp <= ctx.run_info()["cartesian_bound"] < 4000 * 9000
    one = jn.pred(jn.JN_LT)
    exp1 = O.nested_loop(ra.numpy(), sa.numpy(), op_a=O.LT, count_only=True)
    assert jn.jn_count(ctx, jn.JN_ALGO_THETA, RB, SB, one) == exp1
    assert exp1 <= ctx.run_info()["cartesian_bound"] <= 4000 * 9000


# ------------------------------------------------------ sort-merge join --

@pytest.mark.parametrize("case", HASH_CASES)
@pytest.mark.parametrize("pre", [0, 1])
def test_sort_merge_cases(ctx, case, pre):
    nr, ns, lo, hi, dt = case
    r = keys(nr, lo, hi, 13, 0, dt)
    s = keys(ns, lo, hi, 13, 1, dt)
    if dt == torch.int32:
        r, s = with_edges(r, [I32_MIN, I32_MAX], 15), with_edges(s, [I32_MAX, I32_MIN], 16)
    else:
        r, s = with_edges(r, [I64_MIN, I64_MAX], 15), with_edges(s, [I64_MAX, I64_MIN], 16)
    exp = canon(O.sort_merge_join(r.numpy(), s.numpy()))
    ctx.set_tuning(prefilter=pre)
    try:
        R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
        got = jn.jn_sort_merge(ctx, R, S)
        assert jn.jn_count(ctx, jn.JN_ALGO_SORT, R, S) == exp.shape[0]
    finally:
        ctx.set_tuning(prefilter=-1)
    assert np.array_equal(canon(got), exp)


@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
def test_sort_merge_full_chunks_and_extreme_keys(ctx, dt):
    # one radix bit: partitions hold many full R chunks (4096 / 2048 rows), so
    # the in-chunk sort runs at its full length; the largest key equals the
    # padding's sort key and must still sort before the padding
    top = I32_MAX if dt == torch.int32 else I64_MAX
    bot = I32_MIN if dt == torch.int32 else I64_MIN
    r = torch.cat([torch.full((5000,), top, dtype=dt), keys(20000, -40, 40, 17, 0, dt),
                   torch.full((300,), bot, dtype=dt)])
    s = torch.cat([keys(7000, -40, 40, 17, 1, dt), torch.full((3,), top, dtype=dt),
                   torch.full((2,), bot, dtype=dt)])
    r = r[datagen.uniform_int(r.numel(), 0, 1 << 30, 18, 0, dtype=torch.int64).argsort()]
    rp = datagen.uniform_int(r.numel(), I32_MIN, I32_MAX, 18, 1)
    sp = datagen.uniform_int(s.numel(), I32_MIN, I32_MAX, 18, 2)
    exp = canon(O.sort_merge_join(r.numpy(), s.numpy(), rp.numpy(), sp.numpy()))
    cnt, chk = O.equi_count_checksum(r.numpy(), s.numpy(), rp.numpy(), sp.numpy())
    R = jn.table(r.to(DEV), payload=rp.to(DEV))
    S = jn.table(s.to(DEV), payload=sp.to(DEV))
    for heavy in (0, 64):
        ctx.set_tuning(radix_bits=1, radix_bits1=1, prefilter=0, heavy=heavy)
        try:
            got = jn.jn_sort_merge(ctx, R, S)
            assert jn.jn_aggregate(ctx, jn.JN_ALGO_SORT, R, S) == (cnt, chk)
        finally:
            ctx.set_tuning(radix_bits=0, radix_bits1=0, prefilter=-1, heavy=-1)
        assert np.array_equal(canon(got), exp)


def test_sort_merge_equals_hash_join_zipf(ctx):
    r = skewed(200000, 1 << 16, 0.8, 19, 0, torch.int32)
    s = skewed(300000, 1 << 16, 0.8, 19, 1, torch.int32)
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    a = canon(jn.jn_hash(ctx, R, S))
    b = canon(jn.jn_sort_merge(ctx, R, S))
    assert np.array_equal(a, b)
    assert a.shape[0] == O.hash_join(r.numpy(), s.numpy(), count_only=True)
    with pytest.raises(jn.JoinError):
        jn.jn_count(ctx, jn.JN_ALGO_SORT, R, S, jn.pred(jn.JN_LT))


# ------------------------------------------------------------------ star join

def star_tables(nr, n1, n2, d1, d2, seed, dt, zipf=None):
    if zipf is None:
        f1, f2 = keys(nr, 0, d1, seed, 0, dt), keys(nr, 0, d2, seed, 1, dt)
        k1, k2 = keys(n1, 0, d1, seed, 2, dt), keys(n2, 0, d2, seed, 3, dt)
    else:
        f1, f2 = skewed(nr, d1, zipf, seed, 0, dt), skewed(nr, d2, zipf, seed, 1, dt)
        k1, k2 = skewed(n1, d1, zipf, seed, 2, dt), skewed(n2, d2, zipf, seed, 3, dt)
    rp = datagen.uniform_int(nr, I32_MIN, I32_MAX, seed, 4)
    p1 = datagen.uniform_int(n1, I32_MIN, I32_MAX, seed, 5)
    p2 = datagen.uniform_int(n2, I32_MIN, I32_MAX, seed, 6)
    return f1, f2, k1, k2, rp, p1, p2


def canon3(t):
    t = t.cpu().numpy() if isinstance(t, torch.Tensor) else t
    if t.shape[0] == 0:
        return t.reshape(0, 3)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]


@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
@pytest.mark.parametrize("zipf", [None, 1.0])
def test_star_join_matches_oracle(ctx, dt, zipf):
    # duplicate keys on every side (several S1 and S2 rows per key), several
    # partitions and tiles; Zipf keys send the frequent ones down the heavy path
    # (smaller tables there: a frequent key multiplies through both joins)
    sizes = (20000, 3000, 4000) if zipf is None else (5000, 800, 1000)
    f1, f2, k1, k2, rp, p1, p2 = star_tables(*sizes, 1000, 1500, 71, dt, zipf)
    exp = canon3(O.star_join(f1.numpy(), f2.numpy(), k1.numpy(), k2.numpy(), rp.numpy(), p1.numpy(), p2.numpy()))
    R = jn.table(f1.to(DEV), f2.to(DEV), rp.to(DEV))
    S1 = jn.table(k1.to(DEV), payload=p1.to(DEV))
    S2 = jn.table(k2.to(DEV), payload=p2.to(DEV))
    got = jn.jn_star(ctx, R, S1, S2)
    assert got.shape == (exp.shape[0], 3)
    assert np.array_equal(canon3(got), exp)
    assert jn.jn_star_count(ctx, R, S1, S2) == exp.shape[0]


def test_star_join_edges_and_buffers(ctx):
    f1, f2, k1, k2, rp, p1, p2 = star_tables(3000, 500, 700, 300, 200, 72, torch.int32)
    R = jn.table(f1.to(DEV), f2.to(DEV))  # payload = row index
    S1, S2 = jn.table(k1.to(DEV)), jn.table(k2.to(DEV), payload=p2.to(DEV))
    exp = canon3(O.star_join(f1.numpy(), f2.numpy(), k1.numpy(), k2.numpy(), s2pay=p2.numpy()))
    m = exp.shape[0]
    assert m > 0
    assert np.array_equal(canon3(jn.jn_star(ctx, R, S1, S2)), exp)
    # caller buffers: device exact, host, too small (nothing written, count returned)
    dev = torch.full((m, 3), -5, dtype=torch.int32, device=DEV)
    assert np.array_equal(canon3(jn.jn_star(ctx, R, S1, S2, out=dev)), exp)
    host = torch.full((m + 3, 3), -5, dtype=torch.int32)
    got = jn.jn_star(ctx, R, S1, S2, out=host)
    assert np.array_equal(canon3(got), exp) and (host[m:] == -5).all()
    small = torch.full((m - 1, 3), -5, dtype=torch.int32, device=DEV)
    with pytest.raises(jn.JoinError) as e:
        jn.jn_star(ctx, R, S1, S2, out=small)
    assert e.value.status == jn.JN_ERR_CAPACITY and e.value.required == m
    assert (small == -5).all()
    # empty tables and no matches give nothing
    empty = torch.empty(0, dtype=torch.int32, device=DEV)
    assert jn.jn_star(ctx, jn.table(empty, empty), S1, S2).shape == (0, 3)
    assert jn.jn_star(ctx, R, jn.table(empty), S2).shape == (0, 3)
    assert jn.jn_star(ctx, R, S1, jn.table(empty)).shape == (0, 3)
    far = (k2 + 10 ** 6).to(DEV)
    assert jn.jn_star_count(ctx, R, S1, jn.table(far)) == 0
    # R's second column and payloads must be on the device
    with pytest.raises(jn.JoinError) as e:
        jn.jn_star(ctx, jn.table(f1.to(DEV), f2.pin_memory()), S1, S2)
    assert e.value.status == jn.JN_ERR_INVALID


@pytest.mark.parametrize("dt", [torch.int32, torch.int64])
def test_star_join_unique_dimensions_closed_form(ctx, dt):
    # a fact table of 4M rows against two dimension tables with unique keys
    # (the usual star schema): each fact row gives at most one triple, the
    # one whose dimension rows hold its keys, so the whole result is known in
    # closed form without the oracle
    nr, n1, n2 = 4 << 20, 1 << 18, 3 << 16
    gen = torch.Generator().manual_seed(73)
    d1 = torch.randperm(1 << 20, generator=gen)[:n1].to(dt) * 3 + 7    # unique S1 keys
    d2 = torch.randperm(1 << 19, generator=gen)[:n2].to(dt) * 5 - 11   # unique S2 keys
    f1 = torch.cat([d1, d1 + 1])[torch.randint(0, 2 * n1, (nr,), generator=gen)]  # half miss S1
    f2 = torch.cat([d2, d2 + 2])[torch.randint(0, 2 * n2, (nr,), generator=gen)]  # half miss S2
    R = jn.table(f1.to(DEV), f2.to(DEV))
    S1 = jn.table(d1.to(DEV))
    S2 = jn.table(d2.to(DEV))
    got = canon3(jn.jn_star(ctx, R, S1, S2))

    def lookup(dim, fk):  # row of dim holding each fk, and whether one does
        order = np.argsort(dim)
        srt = dim[order]
        i = np.minimum(np.searchsorted(srt, fk), len(srt) - 1)
        return order[i], srt[i] == fk

    r1, ok1 = lookup(d1.numpy(), f1.numpy())
    r2, ok2 = lookup(d2.numpy(), f2.numpy())
    keep = ok1 & ok2
    exp = np.stack([np.nonzero(keep)[0], r1[keep], r2[keep]], axis=1).astype(np.int32)
    assert 0 < exp.shape[0] < nr
    assert got.shape == exp.shape
    assert np.array_equal(got, canon3(exp))
