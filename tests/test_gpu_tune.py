"""Autotuner and batch counting on the GPU: a tuned context gives the same
result as the oracle, the tuner's choice lies in its candidate set and is
cached per size class, and jn_batch_count equals jn_batch's per-join counts."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_11201_gb300 import build as B
from paper_1904_11201_gb300 import datagen
from paper_1904_11201_gb300 import jn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture()
def ctx():
    B.build()
    c = jn.Context(0)
    yield c
    c.close()


def canon(p):
    if isinstance(p, torch.Tensor):
        p = p.cpu().numpy()
    return O.sort_pairs(p)


def test_autotune_hash_then_join_equals_oracle(ctx):
    r = datagen.uniform_keys(300000, 0, 1 << 20, 201, 0)
    s = datagen.uniform_keys(500000, 0, 1 << 20, 201, 1)
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    t = jn.jn_autotune(ctx, jn.JN_ALGO_HASH, R, S)
    assert t["prefilter"] in (0, 1, 2, 3) and 1 <= t["radix_bits"] <= 20
    assert t["table_rows"] in (2048, 4096)  # the tuner picks the table size too
    assert t["hash_path"] in (1, 2)  # and the partition path
    assert ctx.tuning()["radix_bits"] == t["radix_bits"]
    jn.jn_hash(ctx, R, S)
    assert ctx.run_info()["table_rows"] == t["table_rows"]
    assert np.array_equal(canon(jn.jn_hash(ctx, R, S)), canon(O.hash_join(r.numpy(), s.numpy())))
    # the same size class reuses the cached choice
    r2 = datagen.uniform_keys(300001, 0, 1 << 20, 202, 0)
    assert jn.jn_autotune(ctx, jn.JN_ALGO_HASH, jn.table(r2.to(DEV)), S) == t


def test_autotune_theta_and_nested_loop(ctx):
    ra, rk = datagen.band_columns(20000, 16, seed=210, stream=0)
    sa, sk = datagen.band_columns(60000, 16, seed=210, stream=1)
    R, S = jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV))
    pr = jn.pred(jn.JN_LE, jn.JN_ANY, 3)
    t = jn.jn_autotune(ctx, jn.JN_ALGO_THETA, R, S, pr)
    assert 2 <= t["theta_groups"] <= 10
    exp = canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.LE, 3))
    assert np.array_equal(canon(jn.jn_theta(ctx, R, S, jn.JN_LE, 3)), exp)
    t2 = jn.jn_autotune(ctx, jn.JN_ALGO_NLJ, R, S, pr)
    assert t2["nlj_tile_r"] in (512, 1024, 2048, 4096)
    assert np.array_equal(canon(jn.jn_nested_loop(ctx, R, S, pr)), exp)


def test_batch_count_and_autotune_batch(ctx):
    joins, keep, exp = [], [], []
    for i in range(24):
        nr = 500 + 997 * i
        ns = 300 + 1511 * i
        if i % 3 == 2:
            ra, rk = datagen.band_columns(nr, 13, seed=220 + i, stream=0)
            sa, sk = datagen.band_columns(ns, 13, seed=220 + i, stream=1)
            keep.append((ra, rk, sa, sk))
            joins.append((jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV)), jn.JN_GT, i % 4))
            exp.append(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.GT, i % 4).shape[0])
        else:
            r = datagen.uniform_keys(nr, 0, 4 * nr, 240 + i, 0)
            s = datagen.uniform_keys(ns, 0, 4 * nr, 240 + i, 1)
            keep.append((r, s))
            joins.append((jn.table(r.to(DEV)), jn.table(s.to(DEV)), jn.JN_EQ, -1))
            exp.append(O.hash_join(r.numpy(), s.numpy(), count_only=True))
    assert jn.jn_batch_count(ctx, joins) == exp
    t = jn.jn_autotune_batch(ctx, joins)
    assert t["part_rows"] in (1024, 2048, 4096) and t["graphs"] in (0, 1)
    pairs, first, cnt = jn.jn_batch(ctx, joins)
    assert cnt == exp
    assert jn.jn_batch_count(ctx, []) == []
