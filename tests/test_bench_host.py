"""Host logic of the benchmark (no GPU): the recorded DRAM traffic is used
only for the exact kernel source and settings it was captured with, and the
derived FP32 peak follows the unit counts and the clock."""
import json

import bench


def _recs():
    return json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))["k_force32"]


def test_recorded_traffic_matches_only_its_configuration():
    recs = _recs()
    assert isinstance(recs, list) and recs
    captured = [r["tuning"] for r in recs]
    for rec in recs:
        tuning = dict(rec["tuning"])
        got = bench.recorded_traffic("k_force32", rec["workload"], rec["N"], rec["key_frame"], tuning)
        assert got == rec["bytes_per_launch"]
        for key, alts in (("n_g", (128, 256, 192)), ("chunk", (64, 96)), ("order_window", (8192, 0)),
                          ("sched", (0, 2)), ("warps", (2, 8))):
            for alt in alts:
                t = dict(tuning, **{key: alt})
                if t == tuning or any(all(t.get(k) == c.get(k) for k in c) for c in captured):
                    continue
                assert bench.recorded_traffic("k_force32", rec["workload"], rec["N"], rec["key_frame"], t) is None
        assert bench.recorded_traffic("k_force32", rec["workload"], rec["N"] // 2, rec["key_frame"], tuning) is None
        assert bench.recorded_traffic("k_force32", rec["workload"], rec["N"], 1 - rec["key_frame"], tuning) is None
        assert bench.recorded_traffic("k_force32", "patches64", rec["N"], rec["key_frame"], tuning) is None


def test_traffic_record_follows_the_kernel_source():
    """The committed record carries the hash of the force kernel's source
    and of the list expansion as they are now (a change to either must
    retake or drop the number)."""
    import hashlib
    assert {"force32.cu", "force_common.cuh", "walk.cu"} <= set(bench.TRAFFIC_SOURCES)
    h = hashlib.sha256()
    for f in bench.TRAFFIC_SOURCES:
        with open(bench.os.path.join(bench.ROOT, "paper_1907_02289_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    for rec in _recs():
        assert rec["source_sha256"] == h.hexdigest()


def test_fp32_peak_from_unit_counts():
    assert abs(bench.fp32_peak_tflops(2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert bench.fp32_peak_tflops(1035.0) * 2 == bench.fp32_peak_tflops(2070.0)
