"""Parity at the benchmark's full sizes, in the configuration bench.py times.

The full outputs are too large for a pair-by-pair oracle comparison, so each
test checks properties that hold at any size (every pair satisfies the
predicate, no pair repeats, the count equals the closed form from key
histograms, each S row has as many pairs as its key has R rows) and compares a
seeded sample of S rows pair by pair with the oracle, or the whole result's
count and separable checksum with the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_11201_gb300 import build as B
from paper_1904_11201_gb300 import datagen as D
from paper_1904_11201_gb300 import jn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = jn.Context(0)
    yield c
    c.close()


def key_counts(keys, others):
    """Rows of `keys` with each value of `others` (int32 or int64 columns):
    the multiplicity c(k) of every row's key in the other table."""
    u, c = torch.unique(keys, return_counts=True)
    pos = torch.searchsorted(u, others).clamp(max=u.numel() - 1)
    return torch.where(u[pos] == others, c[pos], torch.zeros_like(c[pos]))


def check_materialised(r, s, out, sample_seed=3):
    """Properties of a materialised equi-join of row-id payloads that hold at
    any size, plus a seeded sample of S rows pair by pair against oracle O2."""
    n_r, n_s = r.numel(), s.numel()
    m = out.shape[0]
    c_r_of_s = key_counts(r, s)  # for every S row: R rows with its key
    c_s_of_r = key_counts(s, r)
    assert m == int(c_r_of_s.sum())  # closed form: sum over keys of c_R * c_S
    pr, ps = out[:, 0].long(), out[:, 1].long()
    assert bool((pr >= 0).all() and (pr < n_r).all() and (ps >= 0).all() and (ps < n_s).all())
    for lo in range(0, m, 1 << 28):  # every pair joins equal keys
        hi = min(m, lo + (1 << 28))
        assert torch.equal(r[pr[lo:hi]], s[ps[lo:hi]])
    assert torch.equal(torch.bincount(ps, minlength=n_s), c_r_of_s)  # each S row: all its matches
    assert torch.equal(torch.bincount(pr, minlength=n_r), c_s_of_r)  # each R row: all its matches
    del c_r_of_s, c_s_of_r
    code, _ = torch.sort(pr * n_s + ps)
    assert not bool((code[1:] == code[:-1]).any())  # no pair twice
    del code
    # a seeded sample of S rows, pair by pair against the oracle (the sample
    # is the build side, all of R probes it)
    idx = D.uniform_int(512, 0, n_s, seed=sample_seed, stream=0, dtype=torch.int64)
    sk = s.cpu()[idx].numpy()
    exp = O.hash_join(sk, r.cpu().numpy(), idx.numpy().astype(np.int32), None)
    exp = O.sort_pairs(exp[:, ::-1].copy())  # (r row, s row)
    sel = torch.isin(ps, idx.to(DEV))
    got = O.sort_pairs(torch.stack([pr[sel], ps[sel]], 1).int().cpu().numpy())
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_equi_256m_x_256m(ctx, theta):
    # theta = 0: 2.7e8 pairs; theta = 0.5: 1.34e9 pairs (10.7 GB), frequent keys
    n, bits = 1 << 28, 28
    cdf = D.zipf_cdf(theta, 1 << bits, DEV) if theta else None
    r = D.zipf_keys(n, theta, bits, seed=0, stream=0, device=DEV, cdf=cdf)
    s = D.zipf_keys(n, theta, bits, seed=0, stream=1, device=DEV, cdf=cdf)
    del cdf
    ids = D.row_ids(n, DEV)
    R, S = jn.table(r, payload=ids), jn.table(s, payload=ids)
    jn.jn_autotune(ctx, jn.JN_ALGO_HASH, R, S)  # the bench's launch configuration
    out = torch.as_tensor(jn.jn_hash(ctx, R, S), device=DEV)
    if theta:
        assert ctx.run_info()["heavy_keys"] > 0  # the frequent-key path took part
    check_materialised(r, s, out)


def test_equi_256m_x_256m_theta1_count_and_checksum(ctx):
    # about 3e14 pairs: counted, not stored (Sec. 5.3's "results not stored"
    # mode); the count is the exact closed form, the checksum the oracle's
    n, bits = 1 << 28, 28
    cdf = D.zipf_cdf(1.0, 1 << bits, DEV)
    r = D.zipf_keys(n, 1.0, bits, seed=0, stream=0, device=DEV, cdf=cdf)
    s = D.zipf_keys(n, 1.0, bits, seed=0, stream=1, device=DEV, cdf=cdf)
    del cdf
    ids = D.row_ids(n, DEV)
    R, S = jn.table(r, payload=ids), jn.table(s, payload=ids)
    cnt, chk = jn.jn_aggregate(ctx, jn.JN_ALGO_HASH, R, S)
    assert ctx.run_info()["heavy_keys"] > 0
    c_r = torch.bincount(r, minlength=1 << bits)
    c_s = torch.bincount(s, minlength=1 << bits)
    assert cnt == int((c_r * c_s).sum())
    del c_r, c_s
    ecnt, echk = O.equi_count_checksum(r.cpu().numpy(), s.cpu().numpy(), ids.cpu().numpy(), ids.cpu().numpy())
    assert (cnt, chk) == (ecnt, echk)


def test_equi_int64_128m_x_128m(ctx):
    n = 1 << 27
    r = D.zipf_keys(n, 0.0, 28, seed=0, stream=0, device=DEV, dtype=torch.int64)
    s = D.zipf_keys(n, 0.0, 28, seed=0, stream=1, device=DEV, dtype=torch.int64)
    ids = D.row_ids(n, DEV)
    R, S = jn.table(r, payload=ids), jn.table(s, payload=ids)
    jn.jn_autotune(ctx, jn.JN_ALGO_HASH, R, S)
    out = torch.as_tensor(jn.jn_hash(ctx, R, S), device=DEV)
    check_materialised(r, s, out, sample_seed=4)


def test_band_1m_x_16m_w95(ctx):
    nr, ns = 1 << 20, 1 << 24
    ra, rk = D.band_columns(nr, 24, seed=0, stream=0, device=DEV)
    sa, sk = D.band_columns(ns, 24, seed=0, stream=1, device=DEV)
    R = jn.table(ra, rk, D.row_ids(nr, DEV))
    S = jn.table(sa, sk, D.row_ids(ns, DEV))
    pr_ = jn.pred(jn.JN_LT, jn.JN_ANY, 95)
    jn.jn_autotune(ctx, jn.JN_ALGO_THETA, R, S, pr_)
    got_cnt, got_chk = jn.jn_aggregate(ctx, jn.JN_ALGO_THETA, R, S, pr_)
    exp = O.band_join_sorted(ra.cpu().numpy(), rk.cpu().numpy(), sa.cpu().numpy(), sk.cpu().numpy(), O.LT, 95)
    assert got_cnt == exp.shape[0]
    assert got_chk == O.checksum_pairs(exp)
    out = torch.as_tensor(jn.jn_theta(ctx, R, S, jn.JN_LT, 95), device=DEV)
    assert out.shape[0] == exp.shape[0]
    assert O.checksum_pairs(out.cpu().numpy()) == O.checksum_pairs(exp)


def test_nested_loop_64k_x_1m_band(ctx):
    nr, ns, w = 1 << 16, 1 << 20, 24414
    ra, rk = D.band_columns(nr, 24, seed=0, stream=0, device=DEV)
    sa, sk = D.band_columns(ns, 24, seed=0, stream=1, device=DEV)
    R = jn.table(ra, rk, D.row_ids(nr, DEV))
    S = jn.table(sa, sk, D.row_ids(ns, DEV))
    pr_ = jn.pred(jn.JN_LT, jn.JN_ANY, w)
    got_cnt, got_chk = jn.jn_aggregate(ctx, jn.JN_ALGO_NLJ, R, S, pr_)
    exp = O.band_join_sorted(ra.cpu().numpy(), rk.cpu().numpy(), sa.cpu().numpy(), sk.cpu().numpy(), O.LT, w)
    assert got_cnt == exp.shape[0]
    assert got_chk == O.checksum_pairs(exp)


@pytest.mark.parametrize("op", [jn.JN_NE, jn.JN_GE])
def test_one_column_theta_cross_regions_dominate(ctx, op):
    # R.key != S.key and R.key >= S.key over 16K x 48K rows: 4e8 - 8e8 pairs,
    # almost all from the regions Algorithm 3 emits without comparing.  The
    # expected count and checksum come from closed forms: the complement of the
    # equi-join for !=, suffix sums over R sorted by key for >=.
    nr, ns = 16384, 49152
    r = D.uniform_keys(nr, -10 ** 6, 10 ** 6, seed=41, stream=0, device=DEV)
    s = D.uniform_keys(ns, -10 ** 6, 10 ** 6, seed=41, stream=1, device=DEV)
    R = jn.table(r, payload=D.row_ids(nr, DEV))
    S = jn.table(s, payload=D.row_ids(ns, DEV))
    lib = O._load()
    f = np.array([lib.or_f(i) for i in range(nr)], dtype=np.uint64)  # payload = row id
    g = np.array([lib.or_g(i) for i in range(ns)], dtype=np.uint64)
    rk, sk = r.cpu().numpy(), s.cpu().numpy()
    with np.errstate(over="ignore"):
        if op == jn.JN_NE:
            ecnt, echk = O.equi_count_checksum(rk, sk)
            exp_cnt = nr * ns - ecnt
            exp_chk = int((f.sum(dtype=np.uint64) * g.sum(dtype=np.uint64)) - np.uint64(echk))
        else:
            order = np.argsort(rk, kind="stable")
            rs, fs = rk[order], f[order]
            suffix = np.concatenate([np.cumsum(fs[::-1], dtype=np.uint64)[::-1], np.zeros(1, np.uint64)])
            pos = np.searchsorted(rs, sk, side="left")  # first R key >= the S key
            exp_cnt = int((nr - pos).sum())
            exp_chk = int((g * suffix[pos]).sum(dtype=np.uint64))
    assert exp_cnt == O.nested_loop(rk, sk, op_a=op, count_only=True)
    assert jn.jn_aggregate(ctx, jn.JN_ALGO_THETA, R, S, jn.pred(op, jn.JN_ANY, -1)) == (exp_cnt, exp_chk % 2 ** 64)
    out = torch.as_tensor(jn.jn_theta(ctx, R, S, op, -1), device=DEV)
    assert out.shape[0] == exp_cnt
    pr, ps = out[:, 0].long(), out[:, 1].long()
    for lo in range(0, exp_cnt, 1 << 28):  # every pair satisfies the predicate
        hi = min(exp_cnt, lo + (1 << 28))
        a, b = r[pr[lo:hi]], s[ps[lo:hi]]
        assert bool((a != b).all()) if op == jn.JN_NE else bool((a >= b).all())
    code, _ = torch.sort(pr * ns + ps)
    assert not bool((code[1:] == code[:-1]).any())  # no pair twice
    del code
    assert O.checksum_pairs(out.cpu().numpy()) == exp_chk % 2 ** 64
