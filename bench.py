"""Benchmark of the GPU join path.

Default workload: the large equi-join, R = S = 2^28 rows of (int32 key,
int32 payload = row id), keys Zipf(theta) over 2^28 values (theta = 0 by
default), run as the pre-filtered, radix-partitioned hash join with the exact
count pass and one exact output allocation.  A step is one full jn_hash call
(partition with the pre-filter, count pass, scan, allocation, emit); the
partition path is the one the library takes (regions by default: one radix
pass, then one block per region splits it and keeps the pre-filter's bitmap
slice of the region in shared memory).

Prints one JSON line.  `value` = (|R| + |S| + M) / time per step, in
tuples/s ("join tuples/s in+out"), with the inputs already in device memory.
`e2e` repeats the step through the C ABI with host buffers: the library
copies the host columns in and the pairs out inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload hash|hash_int64|sortmerge|band|nlj|nlj_band|batch|serve|star]
                       [--theta T] [--sweep]
Under torchrun (N > 1) every rank runs its own replica of the workload
(the join does not shard without a collective); value sums all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# Thread instructions the nested-loop kernels issue per pair evaluated with the
# two-column band predicate (ncu smsp__thread_inst_executed.sum over 4096 x
# 65536 pairs: 1.736e9 count pass, 1.682e9 emit pass)
NLJ_THREAD_INSTR_PER_PAIR = {"nlj_count": 6.47, "nlj_emit": 6.27}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------- workloads --

def make_workload(name, theta, device, small=False, rows_log2=0, r_rows_log2=0):
    from paper_1904_11201_gb300 import datagen as D
    if name in ("hash", "hash_int64", "sortmerge"):
        i64 = name == "hash_int64"
        n = (1 << 27) if i64 else (1 << 28)
        dbits = 28
        if small:
            n, dbits = 1 << 20, 20
        if rows_log2:
            n, dbits = 1 << rows_log2, rows_log2
        dt = torch.int64 if i64 else torch.int32
        nr = (1 << r_rows_log2) if r_rows_log2 else n
        cdf = None
        if theta != 0:
            cdf = D.zipf_cdf(theta, 1 << dbits, device)
        r = D.zipf_keys(nr, theta, dbits, seed=0, stream=0, device=device, dtype=dt, cdf=cdf)
        s = D.zipf_keys(n, theta, dbits, seed=0, stream=1, device=device, dtype=dt, cdf=cdf)
        del cdf
        sm = name == "sortmerge"
        return {"kind": "hash", "sort": sm, "R": (r, None, D.row_ids(nr, device)), "S": (s, None, D.row_ids(n, device)),
                "config": {"workload": "equi %s join %dM x %dM %s keys, Zipf theta=%g over 2^%d"
                           % ("sort-merge" if sm else "hash", nr >> 20, n >> 20, "int64" if i64 else "int32", theta,
                              dbits),
                           "R_rows": nr, "S_rows": n, "key": "int64" if i64 else "int32",
                           "zipf_theta": theta, "key_domain": 1 << dbits, "payload": "int32 row id",
                           "algo": "jn_sort_merge" if sm else "jn_hash"}}
    if name == "band":
        nr, ns = (1 << 20, 1 << 24) if not small else (1 << 16, 1 << 20)
        ra, rk = D.band_columns(nr, 24, seed=0, stream=0, device=device)
        sa, sk = D.band_columns(ns, 24, seed=0, stream=1, device=device)
        return {"kind": "band", "band": 95, "op": 2,
                "R": (ra, rk, D.row_ids(nr, device)), "S": (sa, sk, D.row_ids(ns, device)),
                "config": {"workload": "band join R.a < S.a and |R.k - S.k| <= 95, 1M x 16M int32",
                           "R_rows": nr, "S_rows": ns, "key": "int32", "band": 95,
                           "algo": "jn_theta(op <, band 95)"}}
    if name == "nlj_band":
        nr, ns = (1 << 16, 1 << 20) if not small else (1 << 12, 1 << 16)
        ra, rk = D.band_columns(nr, 24, seed=0, stream=0, device=device)
        sa, sk = D.band_columns(ns, 24, seed=0, stream=1, device=device)
        return {"kind": "nlj", "pred": (2, 6, 24414),
                "R": (ra, rk, D.row_ids(nr, device)), "S": (sa, sk, D.row_ids(ns, device)),
                "config": {"workload": "tiled nested loop R.a < S.a and |R.k - S.k| <= 24414, 64K x 1M int32",
                           "R_rows": nr, "S_rows": ns, "key": "int32", "band": 24414,
                           "algo": "jn_nested_loop (two-column predicate)"}}
    if name == "nlj":
        nr, ns = 1 << 14, 1 << 16
        r = D.uniform_keys(nr, 0, 65536, seed=0, stream=0, device=device)
        s = D.uniform_keys(ns, 0, 65536, seed=0, stream=1, device=device)
        return {"kind": "nlj", "R": (r, None, D.row_ids(nr, device)), "S": (s, None, D.row_ids(ns, device)),
                "config": {"workload": "equi nested-loop join 16K x 64K int32 uniform [0, 65536)",
                           "R_rows": nr, "S_rows": ns, "key": "int32", "algo": "jn_nested_loop"}}
    raise ValueError(name)


class Counted:
    """Result of a count-and-checksum step (pairs counted, not stored)."""

    def __init__(self, n, checksum):
        self.shape = (n, 2)
        self.checksum = checksum


def run_step(jn, ctx, w, R, S, out=None):
    if w.get("aggregate"):
        algo = {"hash": jn.JN_ALGO_SORT if w.get("sort") else jn.JN_ALGO_HASH, "band": jn.JN_ALGO_THETA,
                "nlj": jn.JN_ALGO_NLJ}[w["kind"]]
        pr = jn.pred(w["op"], jn.JN_ANY, w["band"]) if w["kind"] == "band" else None
        if "pred" in w:
            pr = jn.pred(*w["pred"])
        return Counted(*jn.jn_aggregate(ctx, algo, R, S, pr))
    if w["kind"] == "hash":
        return (jn.jn_sort_merge if w.get("sort") else jn.jn_hash)(ctx, R, S, out=out)
    if w["kind"] == "band":
        return jn.jn_theta(ctx, R, S, w["op"], w["band"], out=out)
    pr = jn.pred(*w["pred"]) if "pred" in w else None
    return jn.jn_nested_loop(ctx, R, S, pr, out=out)


# ------------------------------------------------------------ roofline --

def algorithmic_bytes(kind, info, nr, ns, m, ksize):
    """Algorithmic bytes per kernel for one step, as the partitioned join's
    floor counts them: the partition step reads every input tuple once and writes
    every surviving tuple once; the join reads the partitioned copy once and
    writes 8 bytes per pair.  Intermediate copies (a second partition pass,
    the region path's level-1 rows) are not algorithmic, so where a step is
    split over kernels each byte of the floor is credited to exactly one:
      two radix passes: the four scatter launches together make one pass;
      region path: level 1 reads the input, level 2 writes the partitioned copy.
    Kernels outside the floor (histograms, the pre-filter's key read, the count
    pass, which the floor counts as overhead) get the bytes they must move at least."""
    sr, ss = info["r_survivors"], info["s_survivors"]
    surv = sr + ss
    row = ksize + 4
    if kind == "hash":
        heavy = info.get("heavy_pairs", 0)
        return {
            "presence": ksize * (nr + ns),
            "chunk_hist": ksize * (nr + ns),
            "scatter": row * (nr + ns) + row * surv,
            "region1": row * (nr + ns),
            "region2": row * surv,
            "histogram": ksize * surv,
            "hash_count": row * surv,
            "hash_emit": row * surv + 8 * (m - heavy),
            "sort_chunks": 2 * row * sr,
            "sort_count": row * surv,
            "sort_emit": row * surv + 8 * (m - heavy),
            "cross_emit": 8 * heavy,
        }
    if kind == "band":
        return {
            "minmax": 4 * (nr + ns),
            "histogram": 4 * (nr + ns),
            "scatter": 2 * 12 * (nr + ns),
            "theta_count": 12 * (nr + ns),
            "theta_emit": 12 * (nr + ns) + 8 * m,
            "theta_gather": 12 * (nr + ns) + 8 * m,
        }
    return {}


class ClockSampler:
    FIELDS = "timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        """Keep only samples that arrived inside [t0, t1] (plus one interval)."""
        self.window = (t0, t1 + 0.25)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        mhz, mx, reasons = [], None, set()
        for ts, ln in self.lines:
            if self.window and not (self.window[0] <= ts <= self.window[1]):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                mhz.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                               f[6:10]):
                if v.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return None
        mhz.sort()
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


class PinnedHost:
    """Page-locked host buffers for the end-to-end leg.  "thp": anonymous
    memory advised for transparent huge pages, touched, then registered with
    CUDA (few large pages keep the device's DMA fast even when host memory is
    fragmented); "pin": torch's pin_memory."""

    def __init__(self, kind):
        self.kind = kind
        self.maps = []
        self.regs = []

    def empty(self, shape, dtype):
        if self.kind == "pin":
            return torch.empty(shape, dtype=dtype).pin_memory()
        import mmap
        import numpy as np
        n = 1
        for d in shape:
            n *= d
        nbytes = max(n * torch.empty((), dtype=dtype).element_size(), 1)
        size = (nbytes + (2 << 20) - 1) & ~((2 << 20) - 1)
        mm = mmap.mmap(-1, size, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        if hasattr(mm, "madvise") and hasattr(mmap, "MADV_HUGEPAGE"):
            mm.madvise(mmap.MADV_HUGEPAGE)
        arr = np.frombuffer(mm, dtype=np.uint8, count=size)
        arr[::4096] = 0  # touch every page before it is locked
        t = torch.from_numpy(arr[:nbytes]).view(dtype).view(shape)
        rc = torch.cuda.cudart().cudaHostRegister(t.data_ptr(), size, 0)
        if int(rc) != 0:
            raise RuntimeError("cudaHostRegister failed: %s" % rc)
        self.maps.append((mm, arr))
        self.regs.append(t.data_ptr())
        return t

    def copy_of(self, t):
        h = self.empty(tuple(t.shape), t.dtype)
        h.copy_(t)
        return h

    def close(self):
        for p in self.regs:
            torch.cuda.cudart().cudaHostUnregister(p)
        self.regs = []


# ------------------------------------------------------------ cpu baseline --

def cpu_baseline(kind, budget_s=12.0):
    """The CPU oracle timed on a bounded sample of the same workload shape."""
    import numpy as np
    import oracle as O
    from paper_1904_11201_gb300 import datagen as D
    if kind == "hash":
        n = 1 << 22
        r = D.uniform_keys(n, 0, n, seed=0, stream=0).numpy()
        s = D.uniform_keys(n, 0, n, seed=0, stream=1).numpy()
        rp = np.arange(n, dtype=np.int32)
        t0 = time.perf_counter()
        reps, units = 0, 0
        while True:
            m = O.hash_join(r, s, rp, rp, count_only=False).shape[0]
            reps += 1
            units += 2 * n + m
            if time.perf_counter() - t0 > budget_s or reps >= 8:
                break
        dt = time.perf_counter() - t0
        return {"value": units / dt, "unit": "tuples/s", "cores": 1, "kind": "oracle",
                "sample": "chained hash join (oracle O2), R = S = 2^22 rows, uniform keys over 2^22 "
                          "(same rows-per-key density as the 2^28 workload), %d run(s), %.1f s" % (reps, dt)}
    if kind == "band":
        nr, ns = 1 << 16, 1 << 20
        ra, rk = D.band_columns(nr, 20, seed=0, stream=0)
        sa, sk = D.band_columns(ns, 20, seed=0, stream=1)
        t0 = time.perf_counter()
        m = O.band_join_sorted(ra.numpy(), rk.numpy(), sa.numpy(), sk.numpy(), O.LT, 95).shape[0]
        dt = time.perf_counter() - t0
        return {"value": (nr + ns + m) / dt, "unit": "tuples/s", "cores": 1, "kind": "oracle",
                "sample": "sorted band join (oracle O4), 64K x 1M over 2^20 with w = 95, %.1f s" % dt}
    r = D.uniform_keys(4096, 0, 65536, seed=0, stream=0).numpy()
    s = D.uniform_keys(65536, 0, 65536, seed=0, stream=1).numpy()
    t0 = time.perf_counter()
    m = O.nested_loop(r, s, count_only=False).shape[0]
    dt = time.perf_counter() - t0
    return {"value": (r.shape[0] + s.shape[0] + m) / dt, "unit": "tuples/s", "cores": 1, "kind": "oracle",
            "sample": "nested loop (oracle O1), 4K x 64K, %.1f s" % dt}


# ------------------------------------------------------- batched joins --

def make_batch(dev, count, lo, hi, seed=4):
    """Independent join instances: |R|, |S| log-uniform in [lo, hi], selectivity
    log-uniform in [1e-6, 1e-3]; even instances are equi-joins over a key
    domain of 1/sel values, odd ones band joins R.a < S.a and |R.k - S.k| <= w
    with k over (2w + 1) / (2 sel) values.  Where that domain would give more
    pairs than input rows it is widened to keep |result| <= max(|R|, |S|)."""
    import math
    from paper_1904_11201_gb300 import datagen as D
    nr = D.log_uniform_int(count, lo, hi, seed, 0).tolist()
    ns = D.log_uniform_int(count, lo, hi, seed, 1).tolist()
    u = D.uniform_float(count, seed, 2).tolist()
    ws = D.uniform_int(count, 0, 17, seed, 3).tolist()
    inst = []
    for i in range(count):
        sel = math.exp(math.log(1e-6) + u[i] * (math.log(1e-3) - math.log(1e-6)))
        big = max(nr[i], ns[i])
        if i % 2 == 0:
            dom = min(max(int(math.ceil(1.0 / sel)), big), 1 << 31)
            r = D.uniform_keys(nr[i], 0, dom, seed + 10 + i, 0, device=dev)
            s = D.uniform_keys(ns[i], 0, dom, seed + 10 + i, 1, device=dev)
            inst.append({"band": -1, "op": 0, "R": (r, None), "S": (s, None), "domain": dom})
        else:
            w = ws[i]
            dom = min(max(int(math.ceil((2 * w + 1) / (2 * sel))), (2 * w + 1) * big // 2 + 1), 1 << 31)
            ra = D.uniform_keys(nr[i], 0, 1 << 24, seed + 10 + i, 2, device=dev)
            rk = D.uniform_keys(nr[i], 0, dom, seed + 10 + i, 3, device=dev)
            sa = D.uniform_keys(ns[i], 0, 1 << 24, seed + 10 + i, 4, device=dev)
            sk = D.uniform_keys(ns[i], 0, dom, seed + 10 + i, 5, device=dev)
            inst.append({"band": w, "op": 2, "R": (ra, rk), "S": (sa, sk), "domain": dom})
    return inst


def batch_main(args, world, rank, local, dev, stream, jn, ctx):
    """A step is one jn_batch call over all instances (one exact allocation)."""
    count, lo, hi = (256, 1000, 1 << 16) if args.small else (args.batch_count, 1000, 4 << 20)
    inst = make_batch(dev, count, lo, hi)
    joins = [(jn.table(*x["R"]), jn.table(*x["S"]), x["op"], x["band"]) for x in inst]
    rows = sum(x["R"][0].shape[0] + x["S"][0].shape[0] for x in inst)
    eq_rows = sum(x["R"][0].shape[0] + x["S"][0].shape[0] for x in inst if x["band"] < 0)
    torch.cuda.synchronize()
    tune = ctx.tuning() if args.no_autotune else jn.jn_autotune_batch(ctx, joins)
    counts = jn.jn_batch_count(ctx, joins)
    m = sum(counts)
    m_eq = sum(c for c, x in zip(counts, inst) if x["band"] < 0)
    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        out, first, cnt = jn.jn_batch(ctx, joins)
        del out
    assert cnt == counts
    l0 = ctx.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    tw0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out, first, cnt = jn.jn_batch(ctx, joins)
        del out
    e1.record(stream)
    torch.cuda.synchronize()
    clk.mark(tw0, time.time())
    barrier(world)
    clocks = clk.stop()
    launches = ctx.launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)

    # one at a time: the same joins, each its own library call
    reps = 0 if args.no_compare else max(1, min(args.steps, 3))
    one_counts = []
    torch.cuda.synchronize()
    o0 = torch.cuda.Event(enable_timing=True)
    o1 = torch.cuda.Event(enable_timing=True)
    o0.record(stream)
    for rep in range(reps):
        for R, S, op, band in joins:
            res = jn.jn_hash(ctx, R, S) if band < 0 else jn.jn_theta(ctx, R, S, op, band)
            if rep == 0:
                one_counts.append(res.shape[0])
            del res
    o1.record(stream)
    torch.cuda.synchronize()
    ms_one = o0.elapsed_time(o1) / reps if reps else float("nan")

    # kernel breakdown from profiled steps (per-launch events; graphs off)
    ctx.reset_stats()
    ctx.set_profiling(True)
    psteps = 2
    for _ in range(psteps):
        out, first, cnt = jn.jn_batch(ctx, joins)
        del out
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.set_profiling(False)
    bn = rows - eq_rows
    abytes = {"histogram": 4 * eq_rows + 4 * bn, "scatter": 12 * eq_rows + 20 * bn, "hash_count": 8 * eq_rows,
              "hash_emit": 8 * eq_rows + 8 * m_eq, "minmax": 4 * bn, "theta_count": 12 * bn,
              "theta_emit": 12 * bn + 8 * (m - m_eq)}
    kern, roof = kernel_table(stats, psteps, abytes)
    units = rows + m
    value = world * units / (ms * 1e-3)
    if rank == 0:
        line = {"metric": "join tuples/s in+out", "value": value, "unit": "tuples/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": "batched joins: %d instances (half equi, half band R.a < S.a and "
                                       "|R.k - S.k| <= w), |R|, |S| log-uniform in [%d, %d], selectivity "
                                       "log-uniform in [1e-6, 1e-3], int32 keys, no payload" % (count, lo, hi),
                           "instances": count, "input_rows": rows, "result_pairs": m, "tuning": tune,
                           "l2": "inputs larger than L2 (no flush needed)" if 4 * rows > (129 << 20)
                           else "inputs fit in L2",
                           "parallelism": "replicas" if world > 1 else "1 GPU",
                           "algo": "jn_batch: one partition pass, one count and one emit launch per phase"},
                "one_at_a_time": None if not reps else
                {"ms_per_step": ms_one, "value": world * units / (ms_one * 1e-3),
                 "counts_match": one_counts == counts, "speedup_of_batch": ms_one / ms},
                "roofline": roof, "cpu_baseline": None,
                "e2e": None, "e2e_note": "batched inputs and outputs stay in device memory",
                "clocks": clocks, "gpu_launches": launches, "kernels": kern}
        print(json.dumps(line), flush=True)


def kernel_table(stats, steps, abytes):
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    kern = {}
    for name, (cnt, tms) in stats.items():
        kern[name] = {"launches_per_step": cnt / steps, "ms_per_step": tms / steps, "share": 0.0,
                      "avg_launch_ms": tms / max(cnt, 1)}
        if name in abytes and tms > 0:
            kern[name]["algorithmic_gb_per_step"] = abytes[name] / 1e9
            kern[name]["achieved_gbs"] = abytes[name] / (tms / steps * 1e-3) / 1e9
    tot = sum(v["ms_per_step"] for v in kern.values()) or 1.0
    for v in kern.values():
        v["share"] = v["ms_per_step"] / tot
    dom = max((k for k in kern if "achieved_gbs" in kern[k]), key=lambda k: kern[k]["ms_per_step"], default=None)
    roof = None
    if dom:
        a = kern[dom]["achieved_gbs"]
        roof = {"bound": "hbm", "kernel": dom, "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                "peak_kind": pk_kind + " (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)", "traffic": None,
                "algorithmic_bytes_per_launch": abytes[dom] / max(kern[dom]["launches_per_step"], 1)}
    return kern, roof


def star_main(args, world, rank, local, dev, stream, jn, ctx):
    """A step is one jn_star call: a 64M-row fact table with two foreign keys
    against two 1M-row dimension tables of unique keys (every fact key found),
    so the result is one triple per fact row."""
    from paper_1904_11201_gb300 import datagen as D
    nf, nd = ((1 << 22), (1 << 16)) if args.small else ((1 << 26), (1 << 20))
    gen = torch.Generator(device="cpu").manual_seed(0)
    d1 = (torch.randperm(1 << 24, generator=gen)[:nd].to(torch.int32) * 7 + 1).to(dev)
    d2 = (torch.randperm(1 << 24, generator=gen)[:nd].to(torch.int32) * 5 + 3).to(dev)
    f1 = d1[D.uniform_int(nf, 0, nd, 0, 0, dev, torch.int64)]
    f2 = d2[D.uniform_int(nf, 0, nd, 0, 1, dev, torch.int64)]
    R = jn.table(f1, f2, D.row_ids(nf, dev))
    S1 = jn.table(d1, payload=D.row_ids(nd, dev))
    S2 = jn.table(d2, payload=D.row_ids(nd, dev))
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        out = jn.jn_star(ctx, R, S1, S2)
        m = out.shape[0]
        del out
    l0 = ctx.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    tw0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = jn.jn_star(ctx, R, S1, S2)
        del out
    e1.record(stream)
    torch.cuda.synchronize()
    clk.mark(tw0, time.time())
    barrier(world)
    clocks = clk.stop()
    launches = ctx.launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    ctx.reset_stats()
    ctx.set_profiling(True)
    out = jn.jn_star(ctx, R, S1, S2)
    del out
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.set_profiling(False)
    kern, _ = kernel_table(stats, 1, {})
    pk, pk_kind = peaks()
    # read the three tables once (fact: two keys and a payload; dimensions: key
    # and payload) and write 12 bytes per triple
    floor = 12 * nf + 8 * 2 * nd + 12 * m
    units = nf + 2 * nd + m
    if rank == 0:
        line = {"metric": "join tuples/s in+out", "value": world * units / (ms * 1e-3), "unit": "tuples/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": "star join: %dM-row fact table (fk1, fk2, payload) x two %dK-row "
                                       "dimension tables of unique keys, every fact key found"
                                       % (nf >> 20, nd >> 10),
                           "fact_rows": nf, "dimension_rows": nd, "result_triples": m,
                           "algo": "jn_star: two hash joins (left-deep), fk2 gathered between them",
                           "l2": "inputs larger than L2 (no flush needed)",
                           "parallelism": "replicas" if world > 1 else "1 GPU"},
                "join_floor": {"bytes": floor, "definition": "12*|R| + 8*(|S1|+|S2|) + 12*M",
                               "frac_of_hbm_peak": floor / (ms * 1e-3) / (pk.get("hbm_gbs", 6800.0) * 1e9)},
                "roofline": None, "cpu_baseline": None, "e2e": None,
                "e2e_note": "tables stay in device memory", "clocks": clocks, "gpu_launches": launches,
                "kernels": kern}
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------- serving --

def make_pool(dev, n_i32, n_i64, lo, hi, seed=5):
    """Device tables with Zipf(theta ~ U[0, 1]) keys over 2^28 ranks; every
    table maps ranks to keys with its own rotation of one shared bijection, so
    the popular keys of two tables are different keys.  int64 keys sit above
    2^40.  A second column a, uniform in [0, 2^24), serves band requests."""
    from paper_1904_11201_gb300 import datagen as D
    bits = 28
    sizes = D.log_uniform_int(n_i32 + n_i64, lo, hi, seed, 0).tolist()
    th = D.uniform_float(n_i32 + n_i64, seed, 1).tolist()
    rot = D.uniform_int(n_i32 + n_i64, 0, 1 << bits, seed, 2, dtype=torch.int64).tolist()
    pool = []
    for i, n in enumerate(sizes):
        i64 = i >= n_i32
        ranks = D.zipf_ranks(n, th[i], 1 << bits, seed + 20 + i, 0, dev)
        ranks = (ranks + rot[i]) & ((1 << bits) - 1)
        k = D.rank_to_key32(ranks, bits, seed).to(torch.int64 if i64 else torch.int32)
        if i64:
            k = k + (0x5A5A << 32)
        a = D.uniform_int(n, 0, 1 << 24, seed + 20 + i, 1, dev, torch.int64 if i64 else torch.int32)
        pool.append({"key": k, "a": a, "i64": i64, "theta": th[i], "rows": n})
        del ranks
    return pool


def serve_main(args, world, rank, local, dev, stream, jn, ctx):
    """Open-loop Poisson request streams against jn_server at fractions of the
    one-at-a-time capacity; a step is one request."""
    import random
    small = args.small
    pool = make_pool(dev, 5 if small else 9, 5 if small else 9, 10000, pool_hi(small))
    n_req = 200 if small else args.serve_requests
    budget = 32 << 30
    rng = random.Random(0)
    i32 = [i for i, t in enumerate(pool) if not t["i64"]]
    i64 = [i for i, t in enumerate(pool) if t["i64"]]
    resident = set(i32[: len(i32) // 2] + i64[: len(i64) // 2])
    eq_t = {i: jn.table(t["key"]) for i, t in enumerate(pool)}
    bd_t = {i: jn.table(t["a"], t["key"]) for i, t in enumerate(pool)}
    torch.cuda.synchronize()
    reqs = []
    for _ in range(n_req):
        ids = i32 if rng.random() < 0.5 else i64
        s = rng.choice(ids)
        if rng.random() < 0.7:
            # 5/7 of the equi requests (half of all) name a resident R by handle
            use_h = rng.random() < 5.0 / 7
            r = rng.choice([i for i in ids if i != s and (i in resident or not use_h)])
            reqs.append({"kind": "equi", "r": r, "s": s, "op": 0, "band": -1, "resident": use_h})
        else:
            r = rng.choice([i for i in ids if i != s])  # two different tables: their popular keys differ
            reqs.append({"kind": "band", "r": r, "s": s, "op": 2, "band": rng.randint(0, 4), "resident": False})

    # one at a time, through the library on one context, admitted by the same budget
    ctx.set_memory_limit(budget)

    def note(msg):
        if args.verbose:
            print("[serve %.1fs] %s" % (time.perf_counter() - t_start, msg), file=sys.stderr, flush=True)

    t_start = time.perf_counter()
    note("pool of %d tables ready" % len(pool))

    def one(q):
        t = time.perf_counter()
        try:
            if q["kind"] == "equi":
                m = jn.jn_hash(ctx, eq_t[q["r"]], eq_t[q["s"]]).shape[0]
            else:
                m = jn.jn_theta(ctx, bd_t[q["r"]], bd_t[q["s"]], q["op"], q["band"]).shape[0]
        except jn.JoinError as e:
            if e.status != jn.JN_ERR_OOM:
                raise
            m = -1
        dt = time.perf_counter() - t
        if dt > 1.0:
            note("slow request %s: %d x %d rows, theta %.2f / %.2f, %.1f s, %d pairs"
                 % (q["kind"], pool[q["r"]]["rows"], pool[q["s"]]["rows"], pool[q["r"]]["theta"],
                    pool[q["s"]]["theta"], dt, m))
        return m

    for q in reqs[:16]:
        one(q)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m_of = [one(q) for q in reqs]
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    note("one at a time: %d requests in %.1f s" % (n_req, t_one))
    ctx.set_memory_limit(0)
    rows = [pool[q["r"]]["rows"] + pool[q["s"]]["rows"] for q in reqs]
    units = sum(rows[i] + m_of[i] for i in range(n_req) if m_of[i] >= 0)
    cap_rps = n_req / t_one

    srv = jn.Server(local, slots=args.serve_slots, coalesce_rows=1 << 18, max_batch=64,
                    small_slots=args.serve_small_slots, small_sms=args.serve_small_sms,
                    memory_budget=budget, graphs=False)
    handles = {i: srv.register(eq_t[i]) for i in resident}

    def submit(q):
        if q["resident"]:
            return srv.submit(None, eq_t[q["s"]], 0, -1, r_handle=handles[q["r"]])
        if q["kind"] == "equi":
            return srv.submit(eq_t[q["r"]], eq_t[q["s"]], 0, -1)
        return srv.submit(bd_t[q["r"]], bd_t[q["s"]], q["op"], q["band"])

    def run_stream(rate, count):
        """rate None: everything submitted at once (saturation)."""
        arr = [0.0] * count
        if rate:
            g = random.Random(11)
            t = 0.0
            for i in range(count):
                t += g.expovariate(rate)
                arr[i] = t
        tickets = [None] * count
        lat = [0.0] * count
        status = [0] * count
        got_m = [0] * count
        run = [0.0] * count

        def waiter():
            # results are collected and released in completion order, so
            # held outputs never wait on an earlier, slower request
            while tickets[0] is None:
                time.sleep(0.0002)
            t0 = tickets[0]  # this stream's tickets are consecutive
            for _ in range(count):
                got = None
                while got is None:
                    try:
                        got = srv.wait_any(1000)
                        if got is None:
                            st = srv.stats()
                            note("waiting 1 s for a completion: %d of %d collected, %d queued, %d MB held"
                                 % (_, count, st["queued"], st["held_bytes"] >> 20))
                    except jn.JoinError as e:  # every result so far collected: more to come
                        if e.status != jn.JN_ERR_INVALID:
                            raise
                        time.sleep(0.0002)
                t, res = got
                i = t - t0
                status[i] = res["status"]
                lat[i] = res["total_ms"]
                run[i] = res["run_ms"]
                got_m[i] = res["pairs"]
                srv.release(t)

        th = threading.Thread(target=waiter)
        th.start()
        start = time.perf_counter()
        for i in range(count):
            d = start + arr[i] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets[i] = submit(reqs[i])
        th.join()
        wall = time.perf_counter() - start
        ok = [i for i in range(count) if status[i] == 0]
        ls = sorted(lat[i] for i in ok)
        pct = (lambda p: ls[min(len(ls) - 1, int(p * len(ls)))] if ls else None)
        refused = [i for i in range(count) if status[i] == jn.JN_ERR_OOM]
        if args.verbose:
            small_ok = sorted((i for i in ok if rows[i] < (1 << 18)), key=lambda i: -lat[i])[:5]
            for i in small_ok:
                q = reqs[i]
                note("slowest small: %s %d x %d rows, band %d, latency %.2f ms, run %.2f ms, %d pairs"
                     % (q["kind"], pool[q["r"]]["rows"], pool[q["s"]]["rows"], q["band"], lat[i], run[i], got_m[i]))
        rs = sorted(run[i] for i in ok)
        run_pct = (lambda p: rs[min(len(rs) - 1, int(p * len(rs)))] if rs else None)
        # slowdown: latency over the request's own run time (queueing it saw)
        sds = sorted(lat[i] / max(run[i], 1e-3) for i in ok)
        sd_pct = (lambda p: sds[min(len(sds) - 1, int(p * len(sds)))] if sds else None)
        by_class = {}
        for name, sel in (("small", lambda i: rows[i] < (1 << 18)), ("large", lambda i: rows[i] >= (1 << 18))):
            lc = sorted(lat[i] for i in ok if sel(i))
            rc = sorted(run[i] for i in ok if sel(i))
            if lc:
                q = min(len(lc) - 1, int(0.99 * len(lc)))
                by_class[name] = {"n": len(lc), "p50_ms": lc[len(lc) // 2], "p99_ms": lc[q],
                                  "run_p50_ms": rc[len(rc) // 2], "run_p99_ms": rc[q]}
        return {"offered_req_s": rate, "achieved_req_s": len(ok) / wall, "wall_s": wall, "ok": len(ok),
                "refused_oom": len(refused), "failed": count - len(ok) - len(refused),
                "p50_ms": pct(0.5), "p99_ms": pct(0.99), "by_size": by_class,
                "run_p50_ms": run_pct(0.5), "run_p99_ms": run_pct(0.99),
                "slowdown_p50": sd_pct(0.5), "slowdown_p99": sd_pct(0.99),
                "tuples_per_s": sum(rows[i] + got_m[i] for i in ok) / wall,
                "results_match": all(got_m[i] == m_of[i] for i in ok)
                and all(m_of[i] < 0 for i in refused)}

    clk = ClockSampler(local)
    clk.start()
    run_stream(None, min(n_req, 500))  # warm-up: worker contexts, pools
    note("server warm-up done")
    tw0 = time.time()
    sat = run_stream(None, n_req)
    note("saturation: %.1f req/s" % sat["achieved_req_s"])
    rates = []
    for f in (0.5, 0.8, 0.95):
        rates.append(dict(run_stream(f * cap_rps, n_req), fraction=f))
        note("Poisson at %.2f of one-at-a-time: p50 %.2f ms, p99 %.2f ms" % (f, rates[-1]["p50_ms"], rates[-1]["p99_ms"]))
    clk.mark(tw0, time.time())
    clocks = clk.stop()
    st = srv.stats()
    srv.close()
    if rank == 0:
        line = {"metric": "join tuples/s in+out", "value": world * sat["tuples_per_s"], "unit": "tuples/s",
                "n_gpus": world, "steps": n_req, "warmup": min(n_req, 500),
                "ms_per_step": 1e3 * sat["wall_s"] / n_req,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+int64",
                "data": "synthetic",
                "config": {"workload": "serving: %d requests (70%% equi, 30%% band R.a < S.a and |R.k - S.k| <= w),"
                                       " tables of %d-%d rows, int32/int64 50/50, Zipf(theta ~ U[0,1]) keys over "
                                       "2^28 ranks, half the requests on resident tables by handle"
                                       % (n_req, 10000, pool_hi(small)),
                           "pool_tables": len(pool), "slots": args.serve_slots, "small_slots": args.serve_small_slots,
                           "small_sms": args.serve_small_sms,
                           "coalesce_rows": 1 << 18,
                           "memory_budget": budget, "resident_requests": sum(q["resident"] for q in reqs),
                           "l2": "tables up to 64M rows; no flush between requests",
                           "parallelism": "replicas" if world > 1 else "1 GPU"},
                "one_at_a_time": {"req_s": cap_rps, "tuples_per_s": units / t_one,
                                  "refused_oom": sum(1 for x in m_of if x < 0)},
                "saturation": sat, "poisson": rates, "server_stats": st,
                "roofline": None, "cpu_baseline": None, "e2e": None,
                "e2e_note": "requests name device-resident columns; latency is submit to pairs ready",
                "clocks": clocks, "gpu_launches": st["kernel_launches"]}
        print(json.dumps(line), flush=True)


def sweep_main(args, world, rank, stream, jn, ctx, w, R, S):
    """The partition fan-out sweep (the paper's alpha, Sec. 5.1.4 and 5.2.4): the
    same join timed at every partition-bit count (hash) or group count (band),
    the rest of the tuning as chosen before; one JSON line with every point."""
    if w["kind"] == "hash":
        knob, values = "radix_bits", list(range(10, 20))  # pass 1 takes <= 9 bits beside the frequent-key digit
    elif w["kind"] == "band":
        knob, values = "theta_groups", list(range(2, 11))
    else:
        raise SystemExit("--sweep: hash and band workloads only")
    base = ctx.tuning()
    points = []
    for v in values:
        ctx.set_tuning(**{knob: v})
        for _ in range(2):
            del_out = run_step(jn, ctx, w, R, S)
            del del_out
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            out = run_step(jn, ctx, w, R, S)
            m = out.shape[0]
            del out
        e1.record(stream)
        torch.cuda.synchronize()
        info = ctx.run_info()
        points.append({knob: v, "ms_per_step": e0.elapsed_time(e1) / args.steps, "pairs": m,
                       "partitions": int(info["partitions"]), "work_items": int(info["work_items"]),
                       "eq_rsize_bound_pairs": int(info["cartesian_bound"])})
    ctx.set_tuning(**{knob: base[knob]})
    if rank == 0:
        print(json.dumps({"metric": "fan-out sweep", "knob": knob, "steps": args.steps,
                          "config": w["config"], "points": points}), flush=True)


def pool_hi(small):
    return (1 << 20) if small else (64 << 20)


_POOL_DATA = {}


def _pool_init(r, s):
    _POOL_DATA["r"], _POOL_DATA["s"] = r, s


def _pool_slice(bounds):
    import numpy as np
    import oracle as O
    lo, hi = bounds
    r, s = _POOL_DATA["r"], _POOL_DATA["s"]
    rp = np.arange(lo, hi, dtype=np.int32)
    sp = np.arange(s.shape[0], dtype=np.int32)
    return O.hash_join(r[lo:hi], s, rp, sp).shape[0]


def cpu_baseline_all_cores(budget_s=12.0):
    """The oracle O2 on every host core: worker i joins its slice of R with all
    of S (the parallelism is the caller's, the oracle is unchanged)."""
    import multiprocessing as mp
    import numpy as np
    import oracle as O
    from paper_1904_11201_gb300 import datagen as D
    O.build()  # built once here, loaded by the workers
    n = 1 << 22
    r = D.uniform_keys(n, 0, n, seed=0, stream=0).numpy()
    s = D.uniform_keys(n, 0, n, seed=0, stream=1).numpy()
    cores = os.cpu_count() or 1
    bounds = [(i * n // cores, (i + 1) * n // cores) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores, initializer=_pool_init, initargs=(r, s)) as pool:
        pool.map(_pool_slice, [(0, 1)] * cores)  # workers up and the oracle loaded
        t0 = time.perf_counter()
        reps, units = 0, 0
        while True:
            m = sum(pool.map(_pool_slice, bounds))
            reps += 1
            units += 2 * n + m
            if time.perf_counter() - t0 > budget_s or reps >= 8:
                break
        dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": "tuples/s", "cores": cores, "kind": "oracle",
            "sample": "chained hash join (oracle O2), R = S = 2^22 rows uniform over 2^22, R split over %d "
                      "spawned processes, each probing all of S, %d run(s), %.1f s" % (cores, reps, dt)}


# ------------------------------------------------------------------ main --

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, dev):
    if world <= 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reference_arm(args, world, rank):
    """The oracle, as it stands, on the host cores: each step a bounded sample."""
    if rank != 0:
        return
    kind = {"hash": "hash", "hash_int64": "hash", "band": "band", "nlj": "nlj", "nlj_band": "nlj",
            "batch": "hash", "serve": "hash"}[args.workload]
    import oracle as O  # noqa: F401
    for _ in range(args.warmup):
        cpu_baseline(kind, budget_s=0.0)
    t0 = time.perf_counter()
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(kind, budget_s=0.0))
    dt = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    cb = dict(vals[0])
    cb["value"] = v
    w = {"hash": "equi hash join 256M x 256M int32 keys, Zipf theta=%g over 2^28" % args.theta,
         "band": "band join R.a < S.a and |R.k - S.k| <= 95, 1M x 16M int32",
         "nlj": "equi nested-loop join 16K x 64K int32 uniform [0, 65536)"}[kind]
    print(json.dumps({"impl": "reference", "metric": "join tuples/s in+out", "value": v, "unit": "tuples/s",
                      "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1000.0 * dt / max(args.steps, 1), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                      "config": {"workload": w, "sample": cb["sample"]},
                      "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": "tuples/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jn")
    ap.add_argument("--workload", default="hash")
    ap.add_argument("--theta", type=float, default=0.0)
    ap.add_argument("--small", action="store_true", help="small inputs (profiling runs)")
    ap.add_argument("--rows-log2", type=int, default=0,
                    help="hash workloads: 2^N rows per table over a 2^N key domain (profiling runs)")
    ap.add_argument("--r-rows-log2", type=int, default=0,
                    help="hash workloads: 2^N rows in R only, S and the key domain unchanged")
    ap.add_argument("--prefilter", type=int, default=-1,
                    help="-1 auto, 0 off, 1 both tables, 2 only S, 3 only R")
    ap.add_argument("--radix-bits", type=int, default=0)
    ap.add_argument("--table-rows", type=int, default=0,
                    help="hash: R rows per shared-memory table (0 = the key type's full table)")
    ap.add_argument("--theta-groups", type=int, default=0, help="band: log2 of the key groups (0 = autotune)")
    ap.add_argument("--aggregate", action="store_true",
                    help="count + checksum without storing pairs (results too large to store)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default tuning")
    ap.add_argument("--no-compare", action="store_true", help="batch: skip the one-at-a-time comparison")
    ap.add_argument("--host-alloc", default="pin", choices=("thp", "pin"),
                    help="e2e host buffers: huge-page-advised memory registered with CUDA, or torch pin_memory")
    ap.add_argument("--host-io", type=int, default=0,
                    help="e2e: 0 copy host buffers, 1 read inputs in place, 2 write pairs in place, 3 both")
    ap.add_argument("--batch-count", type=int, default=4096, help="batch workload: number of joins")
    ap.add_argument("--sweep", action="store_true",
                    help="time the join at every partition-bit (hash) or group (band) count; one JSON line")
    ap.add_argument("--serve-requests", type=int, default=10000, help="serve workload: requests per stream")
    ap.add_argument("--serve-slots", type=int, default=4, help="serve workload: server worker slots")
    ap.add_argument("--serve-small-slots", type=int, default=1,
                    help="serve workload: slots that take only small requests (a lane for them)")
    ap.add_argument("--serve-small-sms", type=int, default=16,
                    help="serve workload: SMs the other slots' grids leave free for the small lane")
    ap.add_argument("--verbose", action="store_true", help="progress lines on stderr")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    profiling_run = args.small or args.rows_log2 > 0 or args.r_rows_log2 > 0
    if not profiling_run:
        args.warmup = max(args.warmup, 3)

    from paper_1904_11201_gb300 import build as B
    from paper_1904_11201_gb300 import jn
    if rank == 0 or world == 1:
        B.build()
    barrier(world)
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    stream = torch.cuda.current_stream(local)
    ctx = jn.Context(local, stream)
    if args.prefilter != -1 or args.radix_bits or args.theta_groups or args.table_rows:
        ctx.set_tuning(prefilter=args.prefilter, radix_bits=args.radix_bits, theta_groups=args.theta_groups,
                       table_rows=args.table_rows)
    if args.workload in ("batch", "serve", "star"):
        {"batch": batch_main, "serve": serve_main, "star": star_main}[args.workload](
            args, world, rank, local, dev, stream, jn, ctx)
        ctx.close()
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    w = make_workload(args.workload, args.theta, dev, args.small, args.rows_log2, args.r_rows_log2)
    if args.aggregate:
        w["aggregate"] = True
        w["config"]["mode"] = "count + separable checksum (pairs not stored)"
        args.no_e2e = True
    (rk, rk2, rp), (sk, sk2, sp) = w["R"], w["S"]
    R = jn.table(rk, rk2, rp)
    S = jn.table(sk, sk2, sp)
    nr, ns = rk.shape[0], sk.shape[0]
    ksize = rk.element_size()
    torch.cuda.synchronize()
    if (args.prefilter == -1 and not args.radix_bits and not args.theta_groups and not args.table_rows
            and not args.no_autotune):
        # the library's autotuner times its candidate tunings before the warm-up
        algo = {"hash": jn.JN_ALGO_SORT if w.get("sort") else jn.JN_ALGO_HASH, "band": jn.JN_ALGO_THETA,
                "nlj": jn.JN_ALGO_NLJ}[w["kind"]]
        pr = None
        if w["kind"] == "band":
            pr = jn.pred(w["op"], jn.JN_ANY, w["band"])
        elif "pred" in w:
            pr = jn.pred(*w["pred"])
        w["config"]["tuning"] = jn.jn_autotune(ctx, algo, R, S, pr)
        w["config"]["autotuned"] = True
    if args.sweep:
        sweep_main(args, world, rank, stream, jn, ctx, w, R, S)
        ctx.close()
        return

    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        out = run_step(jn, ctx, w, R, S)
        m = out.shape[0]
        del out
    info = ctx.run_info()
    if w["kind"] == "hash":
        w["config"]["algo"] += (" (region partition: one radix pass, a block per region splits it with the "
                                "pre-filter's bitmap slice in shared memory; count, emit)"
                                if info.get("hash_path") == 2 else
                                " (pre-filter bitmaps, two radix passes, count, emit)")
        w["config"]["table_rows"] = int(info["table_rows"])  # R rows per shared-memory table

    ctx.reset_stats()
    ctx.set_profiling(True)
    l0 = ctx.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    tw0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = run_step(jn, ctx, w, R, S)
        del out
    e1.record(stream)
    torch.cuda.synchronize()
    clk.mark(tw0, time.time())
    barrier(world)
    clocks = clk.stop()
    launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    stats = ctx.kernel_stats()
    ctx.set_profiling(False)

    units = nr + ns + m
    value = world * units / (ms * 1e-3)
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    abytes = algorithmic_bytes(w["kind"], info, nr, ns, m, ksize)
    kern = {}
    for name, (cnt, tms) in stats.items():
        per_launch = tms / max(cnt, 1)
        kern[name] = {"launches_per_step": cnt / args.steps, "ms_per_step": tms / args.steps,
                      "share": 0.0}
        if name in abytes:
            gbs = abytes[name] / (tms / args.steps * 1e-3) / 1e9 if tms > 0 else 0.0
            kern[name]["algorithmic_gb_per_step"] = abytes[name] / 1e9
            kern[name]["achieved_gbs"] = gbs
        kern[name]["avg_launch_ms"] = per_launch
    tot = sum(v["ms_per_step"] for v in kern.values()) or 1.0
    for v in kern.values():
        v["share"] = v["ms_per_step"] / tot
    dom = max((k for k in kern if k in abytes), key=lambda k: kern[k]["ms_per_step"], default=None)
    roof = None
    if dom:
        a = kern[dom]["achieved_gbs"]
        roof = {"bound": "hbm", "kernel": dom, "achieved": a, "peak": hbm, "unit": "GB/s",
                "frac": a / hbm, "peak_kind": pk_kind + " (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)",
                "traffic": None,
                "algorithmic_bytes_per_launch": abytes[dom] / max(kern[dom]["launches_per_step"], 1)}
    if w["kind"] == "nlj":
        # compare-bound: every launch evaluates all n_R x n_S pairs.  The peak is
        # the SMs' issue rate (4 schedulers x 32 lanes per SM per clock) over the
        # thread instructions the kernel issues per pair, as ncu counted them
        # (smsp__thread_inst_executed.sum / pairs, 4K x 64K two-column band
        # predicate, profiles/nested_loop_64Kx1M.md)
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        cand = [k for k in ("nlj_count", "nlj_emit") if k in kern]
        two = "pred" in w and (w["pred"][1] != 6 or w["pred"][2] >= 0)
        if cand and two:
            dk = max(cand, key=lambda k: kern[k]["ms_per_step"])
            ipp = NLJ_THREAD_INSTR_PER_PAIR[dk]
            peak = nsm * 4 * 32 * sm_mhz * 1e6 / ipp
            a = nr * ns / (kern[dk]["avg_launch_ms"] * 1e-3)
            roof = {"bound": "alu", "kernel": dk, "achieved": a, "peak": peak, "unit": "pair evaluations/s",
                    "frac": a / peak, "traffic": None, "thread_instructions_per_pair": ipp,
                    "peak_kind": "issue rate: %d SMs x 128 lanes x %.0f MHz / %.2f thread instructions per pair "
                                 "(ncu)" % (nsm, sm_mhz, ipp)}
    # DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) is not taken
    # here: it comes from ncu captures of the current kernels (profiles/)
    if roof:
        roof["traffic"] = None
    floor = None
    if w["kind"] in ("hash", "band"):
        fb = 24 * (nr + ns) + 8 * m
        floor = {"bytes": fb, "frac_of_hbm_peak": fb / (ms * 1e-3) / (hbm * 1e9)}

    # ---- end to end: host columns in, host pairs out, through the C ABI ----
    e2e = None
    if not args.no_e2e:
        host = PinnedHost(args.host_alloc)
        hr = tuple(None if t is None else host.copy_of(t) for t in w["R"])
        hs = tuple(None if t is None else host.copy_of(t) for t in w["S"])
        HR, HS = jn.table(*hr), jn.table(*hs)
        hout = host.empty((m, 2), torch.int32)
        if args.host_io:
            ctx.set_tuning(host_io=args.host_io)
        run_step(jn, ctx, w, HR, HS, out=hout)  # warm-up of the staging path
        torch.cuda.synchronize()
        barrier(world)
        # each step timed on its own (the call returns once the pairs are in
        # host memory); the median damps the host link's sharing with other
        # jobs on the machine, every sample is reported
        samples = []
        for _ in range(max(1, min(args.steps, 5))):
            t0 = time.perf_counter()
            got = run_step(jn, ctx, w, HR, HS, out=hout)
            torch.cuda.synchronize()
            samples.append(time.perf_counter() - t0)
        te = sorted(samples)[len(samples) // 2]
        te = max_over_ranks(te, world, dev)
        hb = sum(t.numel() * t.element_size() for t in hr + hs if t is not None)
        e2e = {"value": world * units / te, "unit": "tuples/s", "h2d_bytes_per_step": hb,
               "d2h_bytes_per_step": 8 * m, "ms_per_step": te * 1e3, "stat": "median of %d steps" % len(samples),
               "samples_ms": [round(x * 1e3, 2) for x in samples], "host_io": args.host_io,
               "host_alloc": args.host_alloc}
        del got, hout, hr, hs, HR, HS
        host.close()

    cb = cb_all = None
    if rank == 0 and world == 1 and not args.no_cpu and not profiling_run:
        cb = cpu_baseline(w["kind"])
        if w["kind"] == "hash":
            try:
                cb_all = cpu_baseline_all_cores()
            except Exception as e:  # the one-core figure stands alone
                cb_all = {"unavailable": str(e)[:200]}
    if rank == 0:
        line = {"metric": "join tuples/s in+out", "value": value, "unit": "tuples/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": dict(w["config"], l2="inputs larger than L2 (no flush needed)"
                               if (nr + ns) * (ksize + 4) > (129 << 20) else "inputs fit in L2",
                               parallelism="replicas" if world > 1 else "1 GPU"),
                "input_tuples_per_s": world * (nr + ns) / (ms * 1e-3),
                "output_tuples_per_s": world * m / (ms * 1e-3),
                "result_pairs": m, "join_floor": floor, "roofline": roof, "cpu_baseline": cb,
                "cpu_baseline_all_cores": cb_all,
                # what sizing the output by Eq. (rsize) would have allocated for the
                # same decomposition, against the exact count the library allocates
                "eq_rsize_bound": {"pairs": int(info.get("cartesian_bound", 0)),
                                   "bytes": 8 * int(info.get("cartesian_bound", 0)),
                                   "over_exact": int(info.get("cartesian_bound", 0)) / m if m else None},
                "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
                "run_info": {k: int(v) for k, v in info.items()}, "kernels": kern}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
