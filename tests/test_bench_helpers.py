"""Host-side helpers of the measurement: the resolution of equal error
(log-log interpolation of the plain solver's errors), the DRAM-traffic
record that is valid only for the kernel sources it was captured on, and the
compact summary at the end of the bench line.  No GPU."""
import hashlib
import json
import math
import os

import pytest

import bench
from paper_2602_08670_gb300 import train as TR


def test_resolution_of_equal_error_recovers_a_power_law():
    # err = C N^-p is a straight line in log-log: interpolation is exact
    C, p = 40.0, 1.7
    errs = {n: C * n ** -p for n in (256, 384, 512, 768)}
    for n in (256, 300, 384, 450.5, 700, 768):
        got = TR._interp_resolution(errs, C * n ** -p)
        assert got == pytest.approx(n, rel=1e-12), (n, got)
    # outside the sampled range there is no bracket
    assert TR._interp_resolution(errs, C * 1000 ** -p) is None
    assert TR._interp_resolution(errs, C * 200 ** -p) is None


def test_resolution_of_equal_error_between_kinks():
    # piecewise: the bracketing pair decides, each segment log-log linear
    errs = {256: 0.5, 384: 0.3, 512: 0.25, 768: 0.1}
    e = math.sqrt(0.3 * 0.25)                       # log-midpoint of 384..512
    assert TR._interp_resolution(errs, e) == pytest.approx(math.sqrt(384 * 512), rel=1e-12)


def _write_record(root, key, src_rel, content, nbytes):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    os.makedirs(os.path.dirname(os.path.join(root, src_rel)), exist_ok=True)
    with open(os.path.join(root, src_rel), "wb") as f:
        f.write(content)
    rec = {key: {"bytes": nbytes, "sources": [src_rel],
                 "source_sha256": hashlib.sha256(content).hexdigest()}}
    with open(os.path.join(root, "profiles", "traffic.json"), "w") as f:
        json.dump(rec, f)


def test_traffic_record_holds_only_for_its_sources(tmp_path, monkeypatch):
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    _write_record(root, "pair", "src/k.cu", b"kernel v1\n", 123456)
    assert bench.captured_traffic("pair") == 123456
    assert bench.captured_traffic("other") is None
    with open(os.path.join(root, "src/k.cu"), "wb") as f:   # the kernel changed after the capture
        f.write(b"kernel v2\n")
    assert bench.captured_traffic("pair") is None


def test_committed_traffic_record_names_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for entry in rec.values():
        assert entry["bytes"] > 0
        for src in entry["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, src)), src


def test_summary_is_compact_and_marks_lower_bounds():
    def horizon(err, n_eq, lower, wins):
        return {"learned_error": err, "plain_error_same_n": 0.5123, "n_eq": n_eq, "n_eq_is_lower_bound": lower,
                "learned_rate": 5.2971e9, "learned_rate_times_r3": 1.4e11, "plain_rate_at_n_eq": 6.4e10,
                "learned_wins": wins, "members_on_fallback": 1}
    am = {name: {"accuracy_matched_by_horizon": {"64": horizon(0.02891, 677.36, False, True),
                                                 "2000": horizon(0.0431, 768.0, True, True)}}
          for name in ("stencil", "face_state")}
    line = {"value": 6.3499e10, "learned": {"accuracy_matched": am},
            "serving": {"capacity": {"throughput_cell_updates_per_s": 3.6812e9},
                        "kernel_bound_cell_updates_per_s": 8.3475e9,
                        "load": [{"rate_fraction_of_capacity": 0.9, "p50_latency_s": 0.20213,
                                  "p99_latency_s": 0.95198, "requests": 128}]}}
    out = bench.summary(line)
    assert out["plain_cell_updates_per_s"] == 6.35e10
    assert out["stencil"]["64"][:3] == [0.029, 0.51, "677.0"]
    assert out["face_state"]["2000"][2] == ">768.0"
    assert out["stencil"]["2000"][6] is True and out["stencil"]["2000"][7] == 1
    assert out["serving"]["p50_p99_s"]["0.9"] == [0.202, 0.952, 128]
    assert list(out)[-1] == "serving" and "legend" in out
    json.dumps(out)                                            # serialisable as it stands
