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


@pytest.mark.parametrize("hold_ms", [0, 300])
def test_held_results_refuse_after_a_bounded_wait(hold_ms):
    # the client keeps the first result while it waits for the second, which
    # fits the budget only once that result is released: with nothing else
    # running the server waits hold_wait_ms for a release, then refuses it
    # (JN_ERR_OOM) instead of waiting for a release that waits on it;
    # released results let the same request through
    import time
    srv = jn.Server(0, slots=1, coalesce_rows=0, max_batch=1, memory_budget=40 << 20, hold_wait_ms=hold_ms)
    try:
        r = datagen.uniform_keys(2000, 0, 2, 3, 0)  # ~2M pairs: 16 MB of output each
        s = datagen.uniform_keys(2000, 0, 2, 3, 1)
        R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
        exp = O.hash_join(r.numpy(), s.numpy(), count_only=True)
        torch.cuda.synchronize()
        t1 = srv.submit(R, S)
        first = srv.wait(t1)
        assert first["status"] == jn.JN_OK and first["pairs"] == exp
        t0 = time.perf_counter()
        t2 = srv.submit(R, S)
        second = srv.wait(t2)  # returns: refused, not a hang
        assert second["status"] == jn.JN_ERR_OOM
        assert time.perf_counter() - t0 >= hold_ms * 1e-3
        srv.release(t2)
        srv.release(t1)
        t3 = srv.submit(R, S)
        third = srv.wait(t3)
        assert third["status"] == jn.JN_OK and third["pairs"] == exp
        srv.release(t3)
    finally:
        srv.close()


@pytest.mark.parametrize("small_slots,small_sms", [(0, 0), (1, 0), (2, 0), (1, 24)])
def test_wait_any_returns_completions_once(small_slots, small_sms):
    # with a small-request lane of 1 or 2 of the 3 slots (and the other
    # slots' grids leaving it SMs), small and large requests both complete,
    # each exactly once
    srv = jn.Server(0, slots=3, coalesce_rows=1 << 12, max_batch=8, memory_budget=1 << 30,
                    small_slots=small_slots, small_sms=small_sms)
    try:
        tabs = []
        for i in range(12):
            r = datagen.uniform_keys(500 + 3000 * i, 0, 4000, 40 + i, 0)
            s = datagen.uniform_keys(800 + 2000 * i, 0, 4000, 40 + i, 1)
            tabs.append((r, s, jn.table(r.to(DEV)), jn.table(s.to(DEV))))
        torch.cuda.synchronize()
        tickets = {srv.submit(R, S): i for i, (_, _, R, S) in enumerate(tabs)}
        seen = set()
        for _ in range(len(tickets)):
            t, res = srv.wait_any(-1)
            assert t in tickets and t not in seen and res["status"] == jn.JN_OK
            seen.add(t)
            r, s, _, _ = tabs[tickets[t]]
            assert np.array_equal(canon(srv.pairs(res)), canon(O.hash_join(r.numpy(), s.numpy())))
            srv.release(t)
        with pytest.raises(jn.JoinError):  # nothing outstanding
            srv.wait_any(10)
    finally:
        srv.close()
