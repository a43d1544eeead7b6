"""The bounded device-side wait of the TMA staging pipelines, run out on purpose.

Every TMA pipeline waits on an mbarrier for at most a fixed number of polls.
Here a block waits on an mbarrier that nothing arrives on (a flag that
nothing sets), so the wait runs out: the kernel must record JN_ERR_TIMEOUT,
return, and leave the context usable.  No copy is in flight and no address
is invalid.
"""
import pytest
import torch

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


def test_wait_completes_when_the_phase_completes(ctx):
    st, ns = jn.jn_selftest_wait(ctx, 1024, True)
    assert st == jn.JN_OK


def test_wait_runs_out_and_reports_timeout(ctx):
    polls = 4096
    st, ns = jn.jn_selftest_wait(ctx, polls, False)
    assert st == jn.JN_ERR_TIMEOUT
    assert "wait" in jn.load().jn_last_error(ctx.handle).decode()
    assert 0 < ns < 5_000_000_000
    # the pipelines' limit is 2^19 polls: it must stay a bounded, short wait
    limit_s = ns / polls * (1 << 19) / 1e9
    print("poll %.1f ns; 2^19 polls = %.2f s" % (ns / polls, limit_s))
    assert limit_s < 20
    # the error word was cleared by the read-back: the next wait succeeds
    assert jn.jn_selftest_wait(ctx, 1024, True)[0] == jn.JN_OK


def test_context_usable_after_timeout(ctx):
    assert jn.jn_selftest_wait(ctx, 256, False)[0] == jn.JN_ERR_TIMEOUT
    n, bits = 300_001, 12
    r = D.zipf_keys(n, 0.0, bits, seed=5, stream=0, device=DEV)
    s = D.zipf_keys(n, 0.0, bits, seed=5, stream=1, device=DEV)
    ids = D.row_ids(n, DEV)
    R, S = jn.table(r, payload=ids), jn.table(s, payload=ids)
    exp = int((torch.bincount(r, minlength=1 << bits) * torch.bincount(s, minlength=1 << bits)).sum())
    assert jn.jn_count(ctx, jn.JN_ALGO_HASH, R, S) == exp
    out = torch.as_tensor(jn.jn_hash(ctx, R, S), device=DEV)
    assert out.shape[0] == exp
    assert torch.equal(r[out[:, 0].long()], s[out[:, 1].long()])


def test_poll_count_checked_on_host(ctx):
    launches = jn.load().jn_launch_count(ctx.handle)
    for polls in (0, (1 << 20) + 1):
        assert jn.jn_selftest_wait(ctx, polls, False)[0] == jn.JN_ERR_INVALID
    assert jn.load().jn_launch_count(ctx.handle) == launches
