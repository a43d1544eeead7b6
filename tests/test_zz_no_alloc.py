"""The allocation-free nested-loop join (jn_nested_loop_noalloc).

It exists for callers that may not allocate device memory (an application
that owns every byte of the device, or a latency-critical loop that must not
call any allocator).  Its scratch is a fixed array inside the library, so
this test checks that two calls in a row, which reuse that array, give
exactly the pairs of the allocating jn_nested_loop on the same inputs, and
that sizes beyond the fixed array are refused.  Exact comparison: all
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


def test_noalloc_matches_allocating_entry_point_twice(ctx):
    cases = []
    r = datagen.uniform_keys(5000, 0, 3000, 301, 0)
    s = datagen.uniform_keys(70001, 0, 3000, 301, 1)
    cases.append((jn.table(r.to(DEV)), jn.table(s.to(DEV)), None))
    ra, rk = datagen.band_columns(3000, 16, seed=302, stream=0)
    sa, sk = datagen.band_columns(40000, 16, seed=302, stream=1)
    cases.append((jn.table(ra.to(DEV), rk.to(DEV)), jn.table(sa.to(DEV), sk.to(DEV)),
                  jn.pred(jn.JN_LT, jn.JN_ANY, 30)))
    for R, S, pr in cases:
        ref = canon(jn.jn_nested_loop(ctx, R, S, pr))
        for _ in range(2):  # the second call reuses the fixed scratch of the first
            out = torch.full((ref.shape[0] + 3, 2), -1, dtype=torch.int32, device=DEV)
            got = jn.jn_nested_loop_noalloc(R, S, pr, out=out)
            torch.cuda.synchronize()
            assert np.array_equal(canon(got), ref)


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
