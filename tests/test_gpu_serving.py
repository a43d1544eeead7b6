"""Serving engine (jn_server) on the GPU: every request's result equals the
oracle and the result of the same join run alone, whatever mix it ran in."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_11201_gb300 import build as B
from paper_1904_11201_gb300 import datagen
from paper_1904_11201_gb300 import jn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def canon(p):
    if isinstance(p, torch.Tensor):
        p = p.cpu().numpy()
    return O.sort_pairs(p)


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = jn.Context(0)
    yield c
    c.close()


def make_requests():
    reqs = []
    sizes = datagen.log_uniform_int(48, 100, 200000, seed=91, stream=0).tolist()
    for i, n in enumerate(sizes):
        ns = max(1, int(n * 1.7))
        if i % 4 == 3:
            ra, rk = datagen.band_columns(n, 16, seed=100 + i, stream=0)
            sa, sk = datagen.band_columns(ns, 16, seed=100 + i, stream=1)
            reqs.append(("band", (ra, rk), (sa, sk), jn.JN_GE, i % 5))
        else:
            d = max(8, n // (1 + i % 3))
            r = datagen.uniform_keys(n, 0, d, 120 + i, 0)
            s = datagen.uniform_keys(ns, 0, d, 120 + i, 1)
            reqs.append(("equi", (r,), (s,), jn.JN_EQ, -1))
    return reqs


def oracle_of(kind, R, S, op, band):
    if kind == "band":
        return canon(O.band_join_sorted(R[0].numpy(), R[1].numpy(), S[0].numpy(), S[1].numpy(), op, band))
    return canon(O.hash_join(R[0].numpy(), S[0].numpy()))


@pytest.mark.parametrize("slots,coalesce,graphs", [(1, 0, False), (1, 20000, False), (3, 20000, False),
                                                  (3, 20000, True)])
def test_served_results_equal_alone_and_oracle(ctx, slots, coalesce, graphs):
    reqs = make_requests()
    srv = jn.Server(0, slots=slots, coalesce_rows=coalesce, max_batch=16, memory_budget=8 << 30, graphs=graphs)
    try:
        # a resident table reused by several requests
        hot = datagen.uniform_keys(50000, 0, 20000, 7, 3)
        hid = srv.register(jn.table(hot))
        dev_in = [(jn.table(*[c.to(DEV) for c in R]), jn.table(*[c.to(DEV) for c in S])) for _, R, S, _, _ in reqs]
        hot_probe = datagen.uniform_keys(30000, 0, 20000, 8, 4)
        hp = jn.table(hot_probe.to(DEV))
        torch.cuda.synchronize()  # server workers read the columns on their own streams
        tickets = [srv.submit(Rt, St, op, band) for (Rt, St), (_, _, _, op, band) in zip(dev_in, reqs)]
        t_hot = [srv.submit(None, hp, jn.JN_EQ, -1, r_handle=hid) for _ in range(3)]
        for (kind, R, S, op, band), tk in zip(reqs, tickets):
            res = srv.wait(tk)
            assert res["status"] == jn.JN_OK, res
            got = canon(srv.pairs(res))
            exp = oracle_of(kind, R, S, op, band)
            assert np.array_equal(got, exp)
            alone = (jn.jn_theta(ctx, jn.table(R[0].to(DEV), R[1].to(DEV)), jn.table(S[0].to(DEV), S[1].to(DEV)),
                                 op, band) if kind == "band"
                     else jn.jn_hash(ctx, jn.table(R[0].to(DEV)), jn.table(S[0].to(DEV))))
            assert np.array_equal(canon(alone), got)
            srv.release(tk)
        exp_hot = canon(O.hash_join(hot.numpy(), hot_probe.numpy()))
        for tk in t_hot:
            res = srv.wait(tk)
            assert res["status"] == jn.JN_OK
            assert np.array_equal(canon(srv.pairs(res)), exp_hot)
            srv.release(tk)
        st = srv.stats()
        assert st["completed"] == len(reqs) + 3 and st["failed"] == 0
        if coalesce:
            assert st["batches"] >= 1
        assert st["held_bytes"] == 0
    finally:
        srv.close()


def test_admission_refuses_what_never_fits():
    srv = jn.Server(0, slots=2, coalesce_rows=0, max_batch=1, memory_budget=64 << 20)
    try:
        r = datagen.uniform_keys(4000, 0, 2, 1, 0)   # ~8M pairs: 64 MB of output
        s = datagen.uniform_keys(4000, 0, 2, 1, 1)
        small_r = datagen.uniform_keys(100, 0, 50, 2, 0)
        small_s = datagen.uniform_keys(100, 0, 50, 2, 1)
        big_r, big_s = jn.table(r.to(DEV)), jn.table(s.to(DEV))
        sm_r, sm_s = jn.table(small_r.to(DEV)), jn.table(small_s.to(DEV))
        torch.cuda.synchronize()
        t_big = srv.submit(big_r, big_s)
        t_small = srv.submit(sm_r, sm_s)
        big = srv.wait(t_big)
        small = srv.wait(t_small)
        assert big["status"] == jn.JN_ERR_OOM
        assert small["status"] == jn.JN_OK
        assert np.array_equal(canon(srv.pairs(small)), canon(O.hash_join(small_r.numpy(), small_s.numpy())))
        srv.release(t_big)
        srv.release(t_small)
    finally:
        srv.close()
