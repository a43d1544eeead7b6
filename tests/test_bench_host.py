"""The benchmark's roofline arithmetic, on the host.

The per-kernel algorithmic bytes are restated here from their definitions
(what each kernel must read and write at least) and checked against the
benchmark's table; the dominant kernel, shares and fractions follow from
synthetic per-kernel timings.
"""
import bench


def test_hash_algorithmic_bytes():
    # the floor: the partition step reads every input tuple once (8 B, int32)
    # and writes every surviving tuple once (8 B); the join reads the
    # partitioned copy once and writes 8 B per pair
    nr, ns, m = 1000, 3000, 777
    info = {"r_survivors": 600, "s_survivors": 2100, "heavy_pairs": 7}
    ab = bench.algorithmic_bytes("hash", info, nr, ns, m, 4)
    surv = 600 + 2100
    assert ab["presence"] == 4 * (nr + ns)  # every key read once
    # two radix passes: the scatter launches together make one partition step
    assert ab["scatter"] == 8 * (nr + ns) + 8 * surv
    # region path: level 1 reads the input, level 2 writes the partitioned copy
    assert ab["region1"] == 8 * (nr + ns)
    assert ab["region2"] == 8 * surv
    assert ab["region1"] + ab["region2"] == ab["scatter"]
    assert ab["hash_count"] == 8 * surv
    assert ab["hash_emit"] == 8 * surv + 8 * (m - 7)
    assert ab["cross_emit"] == 8 * 7
    assert ab["sort_chunks"] == 16 * 600  # R survivors read and written sorted
    # the whole-join floor is the partition step plus the emit pass
    assert ab["scatter"] + ab["hash_emit"] + ab["cross_emit"] == 8 * (nr + ns) + 16 * surv + 8 * m
    ab8 = bench.algorithmic_bytes("hash", info, nr, ns, m, 8)
    assert ab8["presence"] == 8 * (nr + ns) and ab8["hash_count"] == 12 * surv


def test_band_algorithmic_bytes():
    ab = bench.algorithmic_bytes("band", {"r_survivors": 0, "s_survivors": 0}, 100, 300, 50, 4)
    assert ab["theta_count"] == 12 * 400
    assert ab["theta_emit"] == 12 * 400 + 8 * 50


def test_kernel_table_dominant_kernel_and_fraction():
    steps = 4
    # name -> (launches over the steps, summed ms)
    stats = {"scatter": (16, 20.0), "presence": (8, 8.0), "scan_top": (40, 0.4)}
    abytes = {"scatter": 12e9, "presence": 2e9}
    kern, roof = bench.kernel_table(stats, steps, abytes)
    assert abs(sum(v["share"] for v in kern.values()) - 1.0) < 1e-12
    assert kern["scatter"]["launches_per_step"] == 4 and kern["scatter"]["ms_per_step"] == 5.0
    assert roof["kernel"] == "scatter"
    # 12 GB per step in 5 ms per step = 2400 GB/s
    assert abs(roof["achieved"] - 2400.0) < 1e-6
    assert abs(roof["frac"] - 2400.0 / roof["peak"]) < 1e-12
    assert roof["algorithmic_bytes_per_launch"] == 12e9 / 4
    assert "achieved_gbs" not in kern["scan_top"]
