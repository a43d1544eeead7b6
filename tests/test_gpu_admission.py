"""Admission by exact bytes on the GPU: a context's memory limit and its
admission hook see the exact output size after the count pass and before any
output allocation; the server admits, defers and refuses requests with it."""
import threading
import time

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


def test_memory_limit_refuses_after_exact_count(ctx):
    r = datagen.uniform_keys(20000, 0, 64, 301, 0)
    s = datagen.uniform_keys(30000, 0, 64, 301, 1)
    m = O.hash_join(r.numpy(), s.numpy(), count_only=True)
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    ctx.set_memory_limit(8 * m // 2)
    with pytest.raises(jn.JoinError) as e:
        jn.jn_hash(ctx, R, S)
    assert e.value.status == jn.JN_ERR_OOM and e.value.required == m
    ctx.set_memory_limit(0)
    assert np.array_equal(canon(jn.jn_hash(ctx, R, S)), canon(O.hash_join(r.numpy(), s.numpy())))


def test_admission_hook_sees_exact_bytes(ctx):
    ra, rk = datagen.band_columns(5000, 12, seed=302, stream=0)
    sa, sk = datagen.band_columns(9000, 12, seed=302, stream=1)
    exp = canon(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.GE, 2))
    R, S = jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV))
    calls = []
    ctx.set_admission(lambda ob, sb: (calls.append((ob, sb)), jn.JN_ERR_OOM)[1])
    with pytest.raises(jn.JoinError) as e:
        jn.jn_theta(ctx, R, S, jn.JN_GE, 2)
    assert e.value.status == jn.JN_ERR_OOM and e.value.required == exp.shape[0]
    assert calls[-1][0] == 8 * exp.shape[0] and calls[-1][1] > 0
    ctx.set_admission(lambda ob, sb: (calls.append((ob, sb)), jn.JN_OK)[1])
    assert np.array_equal(canon(jn.jn_theta(ctx, R, S, jn.JN_GE, 2)), exp)
    # a caller-supplied device buffer needs no output allocation
    out = torch.empty((exp.shape[0], 2), dtype=torch.int32, device=DEV)
    jn.jn_theta(ctx, R, S, jn.JN_GE, 2, out=out)
    assert calls[-1][0] == 0
    # a batch is admitted once, by its total
    joins = [(R, S, jn.JN_GE, 2), (R, S, jn.JN_GE, 2)]
    pairs, first, cnt = jn.jn_batch(ctx, joins)
    assert calls[-1][0] == 8 * 2 * exp.shape[0]
    ctx.set_admission(None)


@pytest.mark.timeout(300)
def test_server_defers_until_memory_is_released():
    B.build()
    r = datagen.uniform_keys(3000, 0, 2, 303, 0)   # about 4.5M pairs: 36 MB of output
    s = datagen.uniform_keys(3000, 0, 2, 303, 1)
    m = O.hash_join(r.numpy(), s.numpy(), count_only=True)
    srv = jn.Server(0, slots=2, coalesce_rows=0, max_batch=1, memory_budget=64 << 20, hold_wait_ms=20000)
    try:
        R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
        torch.cuda.synchronize()
        ta = srv.submit(R, S)
        a = srv.wait(ta)
        assert a["status"] == jn.JN_OK and a["pairs"] == m
        tb = srv.submit(R, S)
        time.sleep(1.0)  # B cannot fit next to A's held output
        assert srv.stats()["completed"] == 1
        exp = canon(O.hash_join(r.numpy(), s.numpy()))
        assert np.array_equal(canon(srv.pairs(a)), exp)
        srv.release(ta)
        b = srv.wait(tb)
        assert b["status"] == jn.JN_OK
        assert np.array_equal(canon(srv.pairs(b)), exp)
        srv.release(tb)
        st = srv.stats()
        assert st["held_bytes"] == 0 and st["peak_bytes"] <= 64 << 20
    finally:
        srv.close()
