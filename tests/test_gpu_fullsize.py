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


def test_equi_256m_x_256m_theta0(ctx):
    n, bits = 1 << 28, 28
    r = D.zipf_keys(n, 0.0, bits, seed=0, stream=0, device=DEV)
    s = D.zipf_keys(n, 0.0, bits, seed=0, stream=1, device=DEV)
    ids = D.row_ids(n, DEV)
    R, S = jn.table(r, payload=ids), jn.table(s, payload=ids)
    jn.jn_autotune(ctx, jn.JN_ALGO_HASH, R, S)  # the bench's launch configuration
    out = torch.as_tensor(jn.jn_hash(ctx, R, S), device=DEV)
    m = out.shape[0]
    c_r = torch.bincount(r, minlength=1 << bits)
    c_s = torch.bincount(s, minlength=1 << bits)
    assert m == int((c_r * c_s).sum())  # closed form: sum over keys of c_R * c_S
    pr, ps = out[:, 0].long(), out[:, 1].long()
    del out
    assert torch.equal(r[pr], s[ps])  # every pair joins equal keys
    assert torch.equal(torch.bincount(ps, minlength=n), c_r[s.long()])  # each S row: all its matches
    del c_s
    code, _ = torch.sort(pr * n + ps)
    assert not bool((code[1:] == code[:-1]).any())  # no pair twice
    del code
    # a seeded sample of S rows, pair by pair against the oracle (the sample
    # is the build side, all of R probes it)
    idx = D.uniform_int(512, 0, n, seed=3, stream=0, dtype=torch.int64)
    sk = s.cpu()[idx].numpy()
    exp = O.hash_join(sk, r.cpu().numpy(), idx.numpy().astype(np.int32), None)
    exp = O.sort_pairs(exp[:, ::-1].copy())  # (r row, s row)
    sel = torch.isin(ps, idx.to(DEV))
    got = O.sort_pairs(torch.stack([pr[sel], ps[sel]], 1).int().cpu().numpy())
    assert np.array_equal(got, exp)


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
