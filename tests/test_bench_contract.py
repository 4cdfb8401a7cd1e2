"""bench.py's roofline bookkeeping (CPU): the algorithmic bytes per launch of each kernel kind,
and the ncu DRAM-traffic lookup, which reports a committed figure only for the kernel sources it
was measured on."""
import json
import os

import bench
from paper_2111_07886_gb300 import synth


def test_algorithmic_bytes_of_the_stacked_workload():
    w = synth.config_stacked_256x89(seed=0)
    b = bench.algorithmic_bytes(w)
    q = 256 * 256 * 89                      # image elements
    sub = (288 // 24) * 357 * 89            # bins of one subset, all planes
    every = 288 * 357 * 89                  # bins of all views
    # f read, counts + gamma read, ratio written
    assert b["forward_ratio"] == 4 * q + 12 * sub
    # w read, f read and written, 1/p read (one plane)
    assert b["update"] == 4 * sub + 8 * q + 4 * 256 * 256
    assert b["mu_sum"] == 4 * q
    assert b["obj_forward"] == 4 * q + 8 * every
    assert abs(b["update"] / 1e6 - 48.45) < 0.01 and abs(b["forward_ratio"] / 1e6 - 27.91) < 0.01


def _write_traffic(root, source_hash, update_bytes):
    os.makedirs(os.path.join(root, "profiles"))
    with open(os.path.join(root, "profiles", "traffic.json"), "w") as fh:
        json.dump({"source_hash": source_hash, "update": update_bytes}, fh)


def test_traffic_reported_only_for_the_sources_it_was_measured_on(tmp_path, monkeypatch):
    current = bench.kernel_source_hash()
    root_ok, root_old = str(tmp_path / "ok"), str(tmp_path / "old")
    _write_traffic(root_ok, current, 123)
    _write_traffic(root_old, "0" * 16, 456)
    monkeypatch.setattr(bench, "ROOT", root_ok)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: current)
    assert bench.ncu_traffic("update") == 123
    assert bench.ncu_traffic("forward_ratio") is None          # no figure for this kind
    monkeypatch.setattr(bench, "ROOT", root_old)
    assert bench.ncu_traffic("update") is None                 # sources changed since


def test_source_hash_covers_the_kernel_sources():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
