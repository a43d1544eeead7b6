"""Pins for the CPU oracle (runs without a GPU).

Each check ties an oracle function to something other than itself: values
worked by hand from the paper's definitions (tests/golden), brute force in
pure Python on tiny inputs, closed forms, special cases with a known answer,
and invariants the paper states (pre-filtering never changes the result,
Eq. (rsize) bounds the count, Algorithm 3's regions classify correctly).
"""
import collections
import itertools
import os
import random

import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_11201_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
I32_MIN, I32_MAX = -(2 ** 31), 2 ** 31 - 1
I64_MIN, I64_MAX = -(2 ** 63), 2 ** 63 - 1


def py_pred(op, x, y):
    return {O.EQ: x == y, O.NE: x != y, O.LT: x < y, O.LE: x <= y,
            O.GT: x > y, O.GE: x >= y, O.ANY: True}[op]


def brute(ra, sa, op_a=O.EQ, rk=None, sk=None, op_k=O.ANY, band=-1):
    """Pure-Python nested loop over Python ints (no overflow possible)."""
    out = []
    for m, x in enumerate(ra):
        for n, y in enumerate(sa):
            if not py_pred(op_a, int(x), int(y)):
                continue
            if rk is not None:
                if band >= 0:
                    if abs(int(rk[m]) - int(sk[n])) > band:
                        continue
                elif not py_pred(op_k, int(rk[m]), int(sk[n])):
                    continue
            out.append((m, n))
    return sorted(out)


def as_list(p):
    return sorted(map(tuple, np.asarray(p).reshape(-1, 2).tolist()))


def read_golden(name):
    blocks, rows = {}, {"R": [], "S": []}
    cur = None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] in ("R", "S"):
                rows[tok[0]].append([int(t) for t in tok[1:]])
            elif tok[0] == "end":
                break
            elif len(tok) >= 2 and not tok[0].lstrip("-").isdigit():
                cur = tuple(tok[:-1])
                blocks[cur] = (int(tok[-1]), [])
            else:
                blocks[cur][1].append((int(tok[0]), int(tok[1])))
    return rows, blocks


# --------------------------------------------------------------- golden --

def test_golden_equi_and_theta():
    rows, blocks = read_golden("equi_theta_small.txt")
    r = np.array(rows["R"][0], dtype=np.int32)
    s = np.array(rows["S"][0], dtype=np.int32)
    cnt, pairs = blocks[("=",)]
    assert len(pairs) == cnt
    assert as_list(O.nested_loop(r, s, op_a=O.EQ)) == sorted(pairs)
    assert as_list(O.hash_join(r, s)) == sorted(pairs)
    assert as_list(O.sort_merge_join(r, s)) == sorted(pairs)
    c, _ = O.equi_count_checksum(r, s)
    assert c == cnt
    cnt, pairs = blocks[("<",)]
    assert len(pairs) == cnt
    assert as_list(O.nested_loop(r, s, op_a=O.LT)) == sorted(pairs)
    got, _, _ = O.theta_regions(r, s, O.LT, 3)
    assert as_list(got) == sorted(pairs)


def test_golden_band():
    rows, blocks = read_golden("band_small.txt")
    R = np.array(rows["R"], dtype=np.int32)
    S = np.array(rows["S"], dtype=np.int32)
    for (tag, w), (cnt, pairs) in blocks.items():
        w = int(w)
        assert len(pairs) == cnt
        got = O.nested_loop(R[:, 0], S[:, 0], R[:, 1], S[:, 1], op_a=O.LT, band=w)
        assert as_list(got) == sorted(pairs)
        got4 = O.band_join_sorted(R[:, 0], R[:, 1], S[:, 0], S[:, 1], O.LT, w)
        assert as_list(got4) == sorted(pairs)
        assert O.band_count_sweep(R[:, 0], R[:, 1], S[:, 0], S[:, 1], O.LT, w) == cnt


# ---------------------------------------------------------- brute force --

def _rand_keys(rng, n, dtype, lo, hi, edges):
    v = [rng.randint(lo, hi) for _ in range(n)]
    for i in range(min(len(edges), n)):
        v[rng.randrange(n)] = edges[i]
    return np.array(v, dtype=dtype)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_nested_loop_vs_brute_force_all_ops(dtype):
    rng = random.Random(11)
    edges = [I32_MIN, I32_MAX, 0, -1] if dtype == np.int32 else [I64_MIN, I64_MAX, 0, -1]
    for trial in range(40):
        nr, ns = rng.randint(0, 23), rng.randint(0, 29)
        lo, hi = (-4, 4) if trial % 2 else (-50, 50)
        ra = _rand_keys(rng, nr, dtype, lo, hi, edges)
        sa = _rand_keys(rng, ns, dtype, lo, hi, edges[::-1])
        rk = _rand_keys(rng, nr, dtype, lo, hi, edges)
        sk = _rand_keys(rng, ns, dtype, lo, hi, edges)
        for op_a in range(7):
            exp = brute(ra, sa, op_a)
            assert as_list(O.nested_loop(ra, sa, op_a=op_a)) == exp
        for op_a, op_k in itertools.product(range(7), repeat=2):
            if (op_a * 7 + op_k + trial) % 5:
                continue
            exp = brute(ra, sa, op_a, rk, sk, op_k)
            assert as_list(O.nested_loop(ra, sa, rk, sk, op_a=op_a, op_k=op_k)) == exp
        for band in (0, 1, 3, 2 ** 31):
            exp = brute(ra, sa, O.LT, rk, sk, band=band)
            assert as_list(O.nested_loop(ra, sa, rk, sk, op_a=O.LT, band=band)) == exp


def test_band_extreme_values_no_overflow():
    # |INT64_MIN - INT64_MAX| does not fit in int64; the definition must hold.
    rk = np.array([I64_MIN, I64_MAX, 0], dtype=np.int64)
    sk = np.array([I64_MAX, I64_MIN, 5], dtype=np.int64)
    ra = np.zeros(3, dtype=np.int64)
    sa = np.zeros(3, dtype=np.int64)
    for band in (0, 5, I64_MAX):
        exp = brute(ra, sa, O.ANY, rk, sk, band=band)
        assert as_list(O.nested_loop(ra, sa, rk, sk, op_a=O.ANY, band=band)) == exp
        assert as_list(O.band_join_sorted(ra, rk, sa, sk, O.ANY, band)) == exp


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_sort_merge_join_equals_brute_force(dtype):
    # O5 against the pure-Python definition, with both extremes of the type
    # (where a careless order key or sentinel would merge the wrong runs)
    lo, hi = (I32_MIN, I32_MAX) if dtype == np.int32 else (I64_MIN, I64_MAX)
    rng = np.random.default_rng(9)
    for trial in range(25):
        nr, ns = int(rng.integers(0, 60)), int(rng.integers(0, 80))
        ra = rng.integers(-3, 4, nr).astype(dtype)
        sa = rng.integers(-3, 4, ns).astype(dtype)
        if nr > 2:
            ra[0], ra[1] = lo, hi
        if ns > 2:
            sa[-1], sa[-2] = hi, lo
        assert as_list(O.sort_merge_join(ra, sa)) == brute(ra, sa, O.EQ)
        assert O.sort_merge_join(ra, sa, count_only=True) == len(brute(ra, sa, O.EQ))
    assert as_list(O.sort_merge_join(np.array([], dtype=dtype), np.array([1], dtype=dtype))) == []


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_hash_join_equals_nested_loop(dtype):
    rng = np.random.default_rng(5)
    for trial in range(30):
        nr, ns = int(rng.integers(0, 300)), int(rng.integers(0, 400))
        dom = int(rng.choice([1, 3, 17, 1000]))
        ra = rng.integers(-dom, dom + 1, nr).astype(dtype)
        sa = rng.integers(-dom, dom + 1, ns).astype(dtype)
        rp = rng.integers(-2 ** 31, 2 ** 31, nr).astype(np.int32)
        sp = rng.integers(-2 ** 31, 2 ** 31, ns).astype(np.int32)
        a = O.sort_pairs(O.nested_loop(ra, sa, rpay=rp, spay=sp))
        b = O.sort_pairs(O.hash_join(ra, sa, rp, sp))
        assert np.array_equal(a, b)
        assert np.array_equal(a, O.sort_pairs(O.sort_merge_join(ra, sa, rp, sp)))


# ---------------------------------------------------------- closed form --

@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_equi_count_closed_form(dtype):
    rng = np.random.default_rng(9)
    for dom in (1, 7, 100, 5000):
        ra = rng.integers(0, dom, 2000).astype(dtype)
        sa = rng.integers(0, dom, 3000).astype(dtype)
        cr, cs = collections.Counter(ra.tolist()), collections.Counter(sa.tolist())
        m = sum(c * cs.get(k, 0) for k, c in cr.items())
        cnt, chk = O.equi_count_checksum(ra, sa)
        assert cnt == m
        assert O.hash_join(ra, sa, count_only=True) == m
        pairs = O.hash_join(ra, sa)
        assert pairs.shape[0] == m
        assert O.checksum_pairs(pairs) == chk


def test_checksum_is_separable_and_order_free():
    rng = np.random.default_rng(3)
    p = rng.integers(-2 ** 31, 2 ** 31, (500, 2)).astype(np.int32)
    direct = sum(O.f_mix(int(r)) * O.g_mix(int(s)) for r, s in p) % 2 ** 64
    assert O.checksum_pairs(p) == direct
    assert O.checksum_pairs(p[::-1].copy()) == direct
    # f and g differ (a transposed pair changes the sum)
    assert O.checksum_pairs(p[:, ::-1].copy()) != direct


def test_special_cases():
    e = np.zeros(0, dtype=np.int32)
    k = np.array([7, 7, 7], dtype=np.int32)
    assert O.nested_loop(e, k).shape[0] == 0
    assert O.hash_join(k, e).shape[0] == 0
    assert O.equi_count_checksum(e, e) == (0, 0)
    # all keys equal: the full Cartesian product
    r = np.full(37, 5, dtype=np.int32)
    s = np.full(41, 5, dtype=np.int32)
    full = sorted(itertools.product(range(37), range(41)))
    assert as_list(O.hash_join(r, s)) == full
    # disjoint keys: nothing
    assert O.hash_join(r, s + 1).shape[0] == 0
    # unique keys and a permutation: exactly one partner each
    perm = np.random.default_rng(1).permutation(1000).astype(np.int32)
    rr = np.arange(1000, dtype=np.int32)
    got = as_list(O.hash_join(rr, perm))
    assert got == sorted((int(perm[n]), n) for n in range(1000))


def test_uniform_expected_count():
    # E[M] = N_R * N_S / D for independent uniform keys over D values.
    nr, ns, d = 16384, 65536, 65536
    r = datagen.uniform_keys(nr, 0, d, seed=0, stream=0).numpy()
    s = datagen.uniform_keys(ns, 0, d, seed=0, stream=1).numpy()
    cnt, _ = O.equi_count_checksum(r, s)
    mean = nr * ns / d
    # Var[M] ~ mean * (1 + (nr + ns) / d) for this draw; allow 6 sigma
    sd = (mean * (1 + (nr + ns) / d)) ** 0.5
    assert abs(cnt - mean) < 6 * sd


# ---------------------------------------------------------------- band --

def test_band_sorted_and_sweep_vs_nested_loop():
    rng = np.random.default_rng(21)
    for trial in range(12):
        nr, ns = int(rng.integers(1, 200)), int(rng.integers(1, 300))
        dom = int(rng.choice([4, 50, 1000]))
        ra, rk = rng.integers(0, dom, nr).astype(np.int32), rng.integers(0, dom, nr).astype(np.int32)
        sa, sk = rng.integers(0, dom, ns).astype(np.int32), rng.integers(0, dom, ns).astype(np.int32)
        for op in (O.LT, O.LE, O.GT, O.GE, O.ANY, O.EQ, O.NE):
            band = int(rng.integers(0, dom))
            ref = O.sort_pairs(O.nested_loop(ra, sa, rk, sk, op_a=op, band=band))
            got = O.sort_pairs(O.band_join_sorted(ra, rk, sa, sk, op, band))
            assert np.array_equal(ref, got)
            if op not in (O.EQ, O.NE):
                assert O.band_count_sweep(ra, rk, sa, sk, op, band) == ref.shape[0]


def test_band_complement_identities():
    rng = np.random.default_rng(4)
    ra, rk = rng.integers(0, 30, 400).astype(np.int32), rng.integers(0, 500, 400).astype(np.int32)
    sa, sk = rng.integers(0, 30, 600).astype(np.int32), rng.integers(0, 500, 600).astype(np.int32)
    w = 17
    c = {op: O.band_count_sweep(ra, rk, sa, sk, op, w) for op in (O.LT, O.LE, O.GT, O.GE, O.ANY)}
    eq = O.band_join_sorted(ra, rk, sa, sk, O.EQ, w, count_only=True)
    assert c[O.LT] + c[O.GE] == c[O.ANY]
    assert c[O.GT] + c[O.LE] == c[O.ANY]
    assert c[O.LT] + eq + c[O.GT] == c[O.ANY]
    # a < b and b > a are the same pairs seen from the other table
    swapped = O.band_count_sweep(sa, sk, ra, rk, O.GT, w)
    assert swapped == c[O.LT]


def test_band_expected_count_closed_form():
    # Independent uniform a, k over D values: P(a_r < a_s) = (D-1)/(2D) and
    # P(|k_r - k_s| <= w) = ((2w+1)D - w(w+1)) / D^2.
    d, w, nr, ns = 1 << 16, 40, 20000, 200000
    ra, rk = datagen.band_columns(nr, 16, seed=3, stream=0)
    sa, sk = datagen.band_columns(ns, 16, seed=3, stream=1)
    got = O.band_count_sweep(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.LT, w)
    mean = nr * ns * ((d - 1) / (2 * d)) * (((2 * w + 1) * d - w * (w + 1)) / d ** 2)
    assert abs(got - mean) < 6 * (mean * 3) ** 0.5


# ---------------------------------------------------- Algorithm 1 (rsize) --

@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_prefilter_never_changes_result(dtype):
    rng = np.random.default_rng(8)
    for trial in range(10):
        nr, ns = int(rng.integers(0, 300)), int(rng.integers(0, 300))
        ra = rng.integers(-60, 60, nr).astype(dtype)
        sa = rng.integers(-30, 90, ns).astype(dtype)
        ref = O.sort_pairs(O.nested_loop(ra, sa))
        common = set(ra.tolist()) & set(sa.tolist())
        surv = sum(1 for v in ra.tolist() if v in common) + sum(1 for v in sa.tolist() if v in common)
        for alpha in (1, 2, 7, 1000):
            pairs, rsize, sv = O.prefilter_grouped_join(ra, sa, alpha)
            assert np.array_equal(O.sort_pairs(pairs), ref)
            assert sv == surv
            assert rsize >= ref.shape[0]           # Eq. (rsize) is an upper bound
            if alpha == 1:
                assert rsize == ref.shape[0]       # one key per reducer: exact
        # one group holding every survivor: rsize = |T'| * |S'|
        _, rsize, _ = O.prefilter_grouped_join(ra, sa, 10 ** 6)
        cr = sum(1 for v in ra.tolist() if v in common)
        cs = sum(1 for v in sa.tolist() if v in common)
        if all(-10 ** 6 <= v < 10 ** 6 for v in common) and common and \
                len({v // 10 ** 6 for v in common}) == 1:
            assert rsize == cr * cs


# ---------------------------------------------------- Algorithm 3 regions --

@pytest.mark.parametrize("op", [O.EQ, O.NE, O.LT, O.LE, O.GT, O.GE, O.ANY])
def test_theta_regions_equal_nested_loop(op):
    rng = np.random.default_rng(100 + op)
    for kq in (1, 2, 4, 7):
        ra = rng.integers(-40, 40, 90).astype(np.int32)
        sa = rng.integers(-35, 50, 110).astype(np.int32)
        pairs, kind, stats = O.theta_regions(ra, sa, op, kq)
        assert as_list(pairs) == brute(ra, sa, op)
        # every pair taken from a cross-join region satisfies the predicate
        for (m, n), k in zip(pairs.tolist(), kind.tolist()):
            if k == 1:
                assert py_pred(op, int(ra[m]), int(sa[n]))
        nd, nt, nf = stats
        assert nd == kq and nd + nt + nf == kq * kq
        expect_true = {O.EQ: 0, O.NE: kq * (kq - 1), O.ANY: kq * (kq - 1)}.get(op, kq * (kq - 1) // 2)
        assert nt == expect_true


# ------------------------------------------------- Eqs. (NBS)/(IDS) ranges --

def test_thread_ranges_cover_each_row_once():
    for n in (0, 1, 5, 31, 32, 33, 1000, 65536, 65537):
        for t in (1, 2, 7, 32, 256, 1000):
            b, e = O.thread_ranges(n, t)
            cover = np.zeros(n, dtype=np.int64)
            for lo, hi in zip(b.tolist(), e.tolist()):
                assert 0 <= lo <= hi <= n
                cover[lo:hi] += 1
            assert (cover == 1).all()
            nb = n // t + 1
            assert b[0] == 0 and (e - b).max(initial=0) <= nb


# ------------------------------------------------------------ generators --

def test_splitmix64_reference_vector():
    # First outputs of SplitMix64 with state 0 (published test vector).
    base = datagen._fmix(torch.tensor([datagen._s64(0x9E3779B97F4A7C15)], dtype=torch.int64))
    assert int(base[0]) & (2 ** 64 - 1) == 0xE220A8397B1DCDAF


def test_checksum_mixers_splitmix64():
    # The oracle's checksum mixers f and g are the SplitMix64 output mixer
    # applied to a constant xor the payload.  The mixer is pinned to the first
    # outputs of SplitMix64 with state 0 (the published sequence: state
    # advances by 0x9E3779B97F4A7C15, output = mix(state)); f, g and the pair
    # checksum are then checked against their definitions.
    lib = O._load()
    golden = 0x9E3779B97F4A7C15
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for i, want in enumerate(published):
        assert lib.or_mix64((golden * (i + 1)) & (2 ** 64 - 1)) == want
    for x in (0, 1, -1, 12345, -(2 ** 31), 2 ** 31 - 1):
        ux = x & 0xFFFFFFFF
        assert lib.or_f(x) == lib.or_mix64(0x243F6A8885A308D3 ^ ux)
        assert lib.or_g(x) == lib.or_mix64(0x13198A2E03707344 ^ ux)
    assert lib.or_f(7) != lib.or_g(7)  # two different mixers
    pairs = np.array([[3, 9], [3, 9], [-5, 2 ** 31 - 1]], dtype=np.int32)
    want = sum(lib.or_f(int(r)) * lib.or_g(int(s)) for r, s in pairs) % 2 ** 64
    assert O.checksum_pairs(pairs) == want


def test_generators_reproducible_and_in_range():
    a = datagen.uniform_keys(1000, 0, 65536, seed=0, stream=1)
    b = datagen.uniform_keys(1000, 0, 65536, seed=0, stream=1)
    c = datagen.uniform_keys(1000, 0, 65536, seed=0, stream=0)
    assert torch.equal(a, b) and not torch.equal(a, c)
    assert int(a.min()) >= 0 and int(a.max()) < 65536
    # the same draws, asked for piecewise at an offset
    w = datagen.raw_u64(100, 5, 2)
    assert torch.equal(w[40:], datagen.raw_u64(60, 5, 2, offset=40))


def test_zipf_ranks_follow_the_law():
    d, n, theta = 64, 400000, 1.0
    r = datagen.zipf_ranks(n, theta, d, seed=2).numpy()
    freq = np.bincount(r, minlength=d) / n
    p = 1.0 / np.arange(1, d + 1) ** theta
    p /= p.sum()
    assert np.abs(freq - p).max() < 6 * np.sqrt(p.max() / n)
    keys = datagen.rank_to_key32(torch.arange(1 << 12), 12, seed=0)
    assert len(set(keys.tolist())) == 1 << 12        # the rank -> key map is a bijection


# ------------------------------------------------------------- star join (O6)

def _star_brute(f1, f2, k1, k2, rp, p1, p2):
    """Three tables, every combination tested: the definition, in Python."""
    out = []
    for (m, a, b) in itertools.product(range(len(f1)), range(len(k1)), range(len(k2))):
        if f1[m] == k1[a] and f2[m] == k2[b]:
            out.append((rp[m], p1[a], p2[b]))
    return sorted(out)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_star_join_equals_brute_force(dtype):
    rng = random.Random(61)
    for trial in range(30):
        nr, n1, n2 = rng.randint(0, 12), rng.randint(0, 9), rng.randint(0, 9)
        lo, hi = (-3, 3) if trial % 2 else (-(2 ** 31), -(2 ** 31) + 4)
        if dtype == np.int64 and trial % 3 == 0:
            lo, hi = 2 ** 62, 2 ** 62 + 3
        f1 = np.array([rng.randint(lo, hi) for _ in range(nr)], dtype=dtype)
        f2 = np.array([rng.randint(lo, hi) for _ in range(nr)], dtype=dtype)
        k1 = np.array([rng.randint(lo, hi) for _ in range(n1)], dtype=dtype)
        k2 = np.array([rng.randint(lo, hi) for _ in range(n2)], dtype=dtype)
        rp = np.array([rng.randint(-1000, 1000) for _ in range(nr)], dtype=np.int32)
        p1 = np.array([rng.randint(-1000, 1000) for _ in range(n1)], dtype=np.int32)
        p2 = np.array([rng.randint(-1000, 1000) for _ in range(n2)], dtype=np.int32)
        got = sorted(map(tuple, O.star_join(f1, f2, k1, k2, rp, p1, p2).tolist()))
        assert got == _star_brute(f1, f2, k1, k2, rp, p1, p2)
        # payloads left out are the row indices
        got_idx = sorted(map(tuple, O.star_join(f1, f2, k1, k2).tolist()))
        assert got_idx == _star_brute(f1, f2, k1, k2, range(nr), range(n1), range(n2))


def test_star_join_count_closed_form():
    # |R join S1 join S2| = sum over rows m of R of c1(fk1[m]) * c2(fk2[m]),
    # c1 and c2 the key histograms of S1 and S2
    rng = np.random.default_rng(62)
    f1 = rng.integers(0, 50, 3000).astype(np.int32)
    f2 = rng.integers(0, 70, 3000).astype(np.int32)
    k1 = rng.integers(0, 60, 400).astype(np.int32)
    k2 = rng.integers(0, 40, 500).astype(np.int32)
    c1 = np.bincount(k1, minlength=100)
    c2 = np.bincount(k2, minlength=100)
    expect = int((c1[f1].astype(np.int64) * c2[f2]).sum())
    assert O.star_join(f1, f2, k1, k2, count_only=True) == expect
    assert O.star_join(f1, f2, k1, k2).shape == (expect, 3)


def test_star_join_reduces_to_two_table_join():
    # S2 holding every fk2 value exactly once: each (r, s1) pair of R join S1
    # gains exactly the one S2 row of its fk2, so the triples are the pinned
    # two-table join's pairs with that row appended
    rng = np.random.default_rng(63)
    f1 = rng.integers(0, 30, 500).astype(np.int64)
    f2 = rng.integers(0, 25, 500).astype(np.int64)
    k1 = rng.integers(0, 30, 200).astype(np.int64)
    k2 = rng.permutation(25).astype(np.int64)
    p2 = (np.arange(25, dtype=np.int32) * 7 + 3)
    tri = O.star_join(f1, f2, k1, k2, s2pay=p2)
    pairs = O.hash_join(f1, k1)
    where = {int(k): i for i, k in enumerate(k2)}
    exp = sorted((int(r), int(s), int(p2[where[int(f2[r])]])) for r, s in pairs)
    assert sorted(map(tuple, tri.tolist())) == exp


def test_star_join_sides_are_not_interchangeable():
    # fk1 meets only S1 and fk2 only S2: swapping the dimension tables swaps
    # the roles, which changes the result unless the columns are swapped too
    f1 = np.array([1, 1, 2], dtype=np.int32)
    f2 = np.array([5, 6, 5], dtype=np.int32)
    k1 = np.array([1, 2, 2], dtype=np.int32)
    k2 = np.array([5, 5, 6], dtype=np.int32)
    a = sorted(map(tuple, O.star_join(f1, f2, k1, k2).tolist()))
    assert a == [(0, 0, 0), (0, 0, 1), (1, 0, 2), (2, 1, 0), (2, 1, 1), (2, 2, 0), (2, 2, 1)]
    assert O.star_join(f1, f2, k2, k1, count_only=True) == 0
    b = sorted((r, s1, s2) for r, s2, s1 in O.star_join(f2, f1, k2, k1).tolist())
    assert b == a
