"""The bench's roofline entries on the CPU: the dominant-kernel entry picks the largest
kind and divides its algorithmic bytes (FP32) or flops (FP64) per launch by its mean
launch time; the aggregate FP32 inner-solve entry sums bytes and times over every FP32
pass kind but the network's."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _bench():
    import bench
    return bench


def _kind(ms, launches, gb=0.0, gflop=0.0):
    return {"ms": ms, "timed": launches, "launches": launches, "bytes": gb * 1e9, "flops": gflop * 1e9}


def test_aggregate_fp32_roofline_sums_bytes_and_times_and_skips_the_network():
    b = _bench()
    prof = {("fp32", "xmid"): _kind(3.0, 10, gb=8.0), ("fp32", "col_fwd"): _kind(1.0, 30, gb=16.0),
            ("fp32", "net_conv"): _kind(50.0, 4, gb=1.0), ("fp64", "xmid"): _kind(20.0, 3, gflop=15.0)}
    r = b.pcg_roofline(prof, 1000, 6000.0, "measured")
    # 24 GB in 4 ms = 6000 GB/s; 10 operator applications (x middle passes)
    assert abs(r["achieved"] - 6000.0) < 1e-9 and abs(r["frac"] - 1.0) < 1e-12
    assert abs(r["ms_per_application"] - 0.4) < 1e-12
    assert abs(r["alg_bytes_per_voxel_application"] - 24e9 / 10 / 1000) < 1e-6
    assert b.pcg_roofline({("fp32", "net_conv"): _kind(1.0, 1, gb=1.0)}, 1, 1.0, "measured") is None


def test_dominant_kernel_roofline_uses_the_bound_of_its_precision():
    b = _bench()
    prof = {("fp32", "col_fwd"): _kind(2.0, 4, gb=8.0), ("fp64", "xmid"): _kind(6.0, 3, gflop=15.0)}
    r = b.roofline(prof, 256 ** 3, 6000.0, "measured")
    # FP64 x middle pass: 5 GFLOP per launch in 2 ms = 2500 GFLOP/s against the FP64 FMA rate
    assert r["bound"] == "alu" and abs(r["achieved"] - 2500.0) < 1e-9
    assert abs(r["frac"] - 2500.0 / b.FP64_PEAK_GFLOPS) < 1e-12
    prof[("fp32", "col_fwd")] = _kind(9.0, 4, gb=8.0)
    r = b.roofline(prof, 256 ** 3, 6000.0, "measured")
    # FP32 plain y pass: 2 GB per launch in 2.25 ms
    assert r["bound"] == "hbm" and abs(r["achieved"] - 2.0e9 / 2.25e-3 / 1e9) < 1e-9
