"""Host logic of the benchmark (no GPU): the recorded DRAM traffic is used
only for the exact kernel source and settings it was captured with, and the
derived FP32 peak follows the unit counts and the clock."""
import json

import bench


def _recs():
    return json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))["k_force32"]


def _source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in bench.TRAFFIC_SOURCES:
        with open(bench.os.path.join(bench.ROOT, "paper_1907_02289_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def test_recorded_traffic_matches_only_its_configuration(tmp_path):
    """A record is used for its own workload, size, frame and launch
    settings only, and only with the kernel source it was taken with."""
    tuning = {"n_g": 192, "chunk": 96, "warps": 8, "sched": 2, "order_by_cost": 1, "order_window": 0}
    rec = {"workload": "ring64m_fp32", "N": 1 << 26, "key_frame": 1, "tuning": tuning,
           "bytes_per_launch": 123, "source_sha256": _source_hash()}
    path = str(tmp_path / "traffic.json")
    json.dump({"k_force32": [rec]}, open(path, "w"))
    got = bench.recorded_traffic("k_force32", rec["workload"], rec["N"], rec["key_frame"], tuning, path)
    assert got == 123
    for key, alts in (("n_g", (128, 256)), ("chunk", (64,)), ("order_window", (8192,)), ("sched", (0,)),
                      ("warps", (2,))):
        for alt in alts:
            t = dict(tuning, **{key: alt})
            assert bench.recorded_traffic("k_force32", rec["workload"], rec["N"], rec["key_frame"], t, path) is None
    assert bench.recorded_traffic("k_force32", rec["workload"], rec["N"] // 2, rec["key_frame"], tuning, path) is None
    assert bench.recorded_traffic("k_force32", rec["workload"], rec["N"], 0, tuning, path) is None
    assert bench.recorded_traffic("k_force32", "patches64", rec["N"], rec["key_frame"], tuning, path) is None
    json.dump({"k_force32": [dict(rec, source_sha256="0" * 64)]}, open(path, "w"))
    assert bench.recorded_traffic("k_force32", rec["workload"], rec["N"], rec["key_frame"], tuning, path) is None


def test_traffic_record_follows_the_kernel_source():
    """The committed record carries the hash of the force kernel's source
    and of the list expansion as they are now (a change to either must
    retake or drop the number)."""
    assert {"force32.cu", "force_common.cuh", "walk.cu"} <= set(bench.TRAFFIC_SOURCES)
    for rec in _recs():
        assert rec["source_sha256"] == _source_hash()


def test_fp32_peak_from_unit_counts():
    assert abs(bench.fp32_peak_tflops(2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert bench.fp32_peak_tflops(1035.0) * 2 == bench.fp32_peak_tflops(2070.0)
