"""Host logic of bench.py (no GPU): the command-line defaults the measurement
contract relies on, the roofline arithmetic, and the traffic figure taken from
the committed chain profile only while the chain sources match it."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.warmup, a.batch, a.impl, a.workload) == (1, 3, 48, "native", "square24")
    assert a.warmup >= 3 and a.steps >= 1


def _prof(**ms):
    kinds = ["leaves", "transpose", "gate", "gemm", "trace", "other", "chain"]
    p = {k: {"launches": 0, "ms": 0.0, "bytes": 0.0, "macs": 0.0} for k in kinds}
    for k, (launches, t, b, m) in ms.items():
        p[k] = {"launches": launches, "ms": t, "bytes": b, "macs": m}
    return p


def test_roofline_of_hbm_kernel():
    # 10 chain launches, 1 GB each, 2 ms total: 0.2 ms per launch -> 5000 GB/s
    r = bench.roofline_of(_prof(chain=(10, 2.0, 10e9, 0.0), gate=(5, 0.5, 1e9, 0.0)), None)
    pk, how = bench.peaks()
    assert r["kernel"] == "chain" and r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(5000.0)
    assert r["frac"] == pytest.approx(5000.0 / pk["hbm_gbs"])
    assert r["avg_launch_ms"] == pytest.approx(0.2)


def test_roofline_of_alu_kernel():
    # 4 GEMM launches, 1e12 multiply-adds each (2 tropical ops), 400 ms: 20 T ops/s
    r = bench.roofline_of(_prof(gemm=(4, 400.0, 1e9, 4e12)), None)
    assert r["bound"] == "alu" and r["kernel"] == "gemm"
    assert r["achieved"] == pytest.approx(20.0)
    assert r["peak"] == pytest.approx(152 * 128 * 2070e6 * 1e-12)


def test_traffic_only_for_matching_sources(monkeypatch):
    recorded = None
    for line in open(os.path.join(ROOT, "profiles", "chain_kernel_square24.md")):
        if line.startswith("- chain sources sha256[:16]: "):
            recorded = line.rsplit(": ", 1)[1].strip()
    assert recorded is not None
    t = bench.traffic_from_profiles("chain")
    if bench.sources_hash() == recorded:
        assert t is not None and t > 1e9
    else:
        assert t is None
    monkeypatch.setattr(bench, "sources_hash", lambda: "0000000000000000")
    assert bench.traffic_from_profiles("chain") is None
    assert bench.traffic_from_profiles("gate") is None       # no profile for it


def test_elimination_work_counts_table_entries():
    # 2x2 lattice eliminated 0, 1, 2, 3: bucket scopes {0,1,2}, {1,2,3}, {2,3}, {3}
    import instances as I
    inst = I.square_lattice(2, coupling="pm1", seed=0)
    assert bench.elimination_work(inst, [0, 1, 2, 3]) == [8.0, 16.0, 20.0, 22.0]
    w = bench.elimination_work(I.square_lattice(24, coupling="gauss", seed=0),
                               I.square_sweep_order(24))
    assert len(w) == 576 and all(b > a for a, b in zip(w, w[1:]))
    # the row sweep's frontier holds 25 spins at its widest
    assert max(b - a for a, b in zip(w, w[1:])) == 2.0 ** 25


def test_reference_arm_reports_the_native_config():
    cfg = bench.workload_config(48, 1)
    assert cfg["workload"] == bench.WORKLOAD and cfg["global_batch"] == 48
    assert set(cfg) == {"workload", "global_batch", "instances_per_step_per_gpu", "l2"}
