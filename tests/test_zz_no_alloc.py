"""The allocation-free nested-loop join (jn_nested_loop_noalloc).

It exists for callers that may not allocate device memory (an application
that owns every byte of the device, or a latency-critical loop that must not
call any allocator).  Its scratch is a fixed array inside the library, so
this test checks that two calls in a row, which reuse that array, give
exactly the oracle's pairs (and those of the allocating jn_nested_loop), and
that sizes beyond the fixed array and misplaced outputs are refused.  Exact comparison: all
arithmetic is integer.  It runs last (file name) so a failure here leaves the
rest of the suite already run, and it passes on its own in a fresh process.
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


def canon(p):
    return O.sort_pairs(p.cpu().numpy())


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = jn.Context(0)
    yield c
    c.close()


def test_noalloc_matches_oracle_twice(ctx):
    # an equi-join against oracle O1 (nested loop) and a band join against
    # oracle O4 (sorted band join), each called twice in a row
    cases = []
    r = datagen.uniform_keys(5000, 0, 3000, 301, 0)
    s = datagen.uniform_keys(70001, 0, 3000, 301, 1)
    cases.append((jn.table(r.to(DEV)), jn.table(s.to(DEV)), None, O.sort_pairs(O.nested_loop(r.numpy(), s.numpy()))))
    ra, rk = datagen.band_columns(3000, 16, seed=302, stream=0)
    sa, sk = datagen.band_columns(40000, 16, seed=302, stream=1)
    cases.append((jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV)),
                  jn.pred(jn.JN_LT, jn.JN_ANY, 30),
                  O.sort_pairs(O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.LT, 30))))
    for R, S, pr, exp in cases:
        for _ in range(2):  # the second call reuses the fixed scratch of the first
            out = torch.full((exp.shape[0] + 3, 2), -1, dtype=torch.int32, device=DEV)
            got = jn.jn_nested_loop_noalloc(R, S, pr, out=out)
            torch.cuda.synchronize()
            assert np.array_equal(canon(got), exp)
            assert bool((out[exp.shape[0]:] == -1).all())  # nothing past the result
        # the allocating entry point gives the same pairs
        assert np.array_equal(canon(jn.jn_nested_loop(ctx, R, S, pr)), exp)


def test_noalloc_refuses_what_does_not_fit():
    r = datagen.uniform_keys(1000, 0, 10, 303, 0)
    s = datagen.uniform_keys(1000, 0, 10, 303, 1)
    R, S = jn.table(r.to(DEV)), jn.table(s.to(DEV))
    m = O.hash_join(r.numpy(), s.numpy(), count_only=True)
    small = torch.zeros((m - 1, 2), dtype=torch.int32, device=DEV)
    with pytest.raises(jn.JoinError) as e:
        jn.jn_nested_loop_noalloc(R, S, out=small)
    assert e.value.status == jn.JN_ERR_CAPACITY and e.value.required == m
    assert bool((small == 0).all())
    big = torch.zeros(300 * 1024, dtype=torch.int32, device=DEV)  # 300 x 300 tiles > 65536
    with pytest.raises(jn.JoinError) as e:
        jn.jn_nested_loop_noalloc(jn.table(big), jn.table(big), out=small)
    assert e.value.status == jn.JN_ERR_INVALID
    with pytest.raises(ValueError):  # the output must be a (capacity, 2) int32 tensor
        jn.jn_nested_loop_noalloc(R, S, out=torch.zeros((8,), dtype=torch.int64, device=DEV))
