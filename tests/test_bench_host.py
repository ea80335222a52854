"""Host-side logic of bench.py, on CPU: the algorithmic-bytes formula, the
lookup of recorded DRAM traffic, the parsing of clock samples taken during the
timed region, and the bounded sample the CPU oracle is timed on."""
import json
import os
import shutil

import numpy as np
import pytest

import bench
import oracle
from bfc_inputs import generators as G


def test_algorithmic_bytes_formula():
    # 4 B per wedge, 12 B per oriented edge and per start; all outputs read
    # the same again in the second walk, write and read 2m slot sums of 8 B,
    # read 2m edge ids of 4 B and write 8 B per edge and per vertex
    W, m, n = 3_286_555_729, 20_000_000, 1_500_000
    assert bench.algorithmic_bytes(W, m, n) == 13_404_222_916
    assert bench.algorithmic_bytes(W, m, n, "all") == 2 * 13_404_222_916 + 48 * m + 8 * n
    assert bench.algorithmic_bytes(0, 0, 0) == 0


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    """A copy of the count sources and an empty profiles folder under a
    temporary root, so the traffic table can be written freely."""
    src = os.path.join(bench.ROOT, "paper_1812_00283_gb300", "csrc")
    dst = tmp_path / "paper_1812_00283_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("count.cu", "bfc_internal.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _write_entries(root, entries):
    with open(root / "profiles" / "count_traffic.json", "w") as f:
        json.dump(dict(entries=entries), f)


def test_recorded_traffic_matches_source_workload_outputs_orientation(fake_root):
    h = bench.count_kernel_hash()
    _write_entries(fake_root, [
        dict(workload="powerlaw_20m", outputs="total", orientation=0, source_sha256=h,
             dram_bytes_per_launch=111),
        dict(workload="shopping_300m", outputs="all", source_sha256=h, dram_bytes_per_launch=222),
        dict(workload="powerlaw_20m", outputs="total", orientation=1, source_sha256="0" * 64,
             dram_bytes_per_launch=333),
    ])
    assert bench.recorded_traffic("powerlaw_20m", "total", 0) == 111
    assert bench.recorded_traffic("shopping_300m", "all", 0) == 222   # orientation defaults to 0
    # an Algorithm 3 launch is not Algorithm 2's, and a stale capture is not used
    assert bench.recorded_traffic("powerlaw_20m", "total", 1) is None
    assert bench.recorded_traffic("powerlaw_20m", "all", 0) is None
    assert bench.recorded_traffic("shopping_300m", "total", 0) is None
    # any change to the kernel source invalidates every entry
    with open(fake_root / "paper_1812_00283_gb300" / "csrc" / "count.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench.recorded_traffic("powerlaw_20m", "total", 0) is None


def test_recorded_traffic_without_table(fake_root):
    assert bench.recorded_traffic("powerlaw_20m") is None


def test_committed_traffic_table_is_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "count_traffic.json")) as f:
        d = json.load(f)
    assert d["entries"]
    for e in d["entries"]:
        assert len(e["source_sha256"]) == 64 and e["dram_bytes_per_launch"] > 0
        assert e["outputs"] in ("total", "all") and e.get("orientation", 0) in (0, 1)
        assert "--clock-control none" in e["command"]


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler("0")
    s.proc = _Done()
    s.lines = lines
    return s


def test_clock_samples_parsed():
    got = _sampler([
        "2070, 2070, 800.1, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1350.0, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 900.0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 10, Not Active, Not Active, Not Active, Not Active",
    ]).stop()
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"] and got["samples"] == 3


def test_clock_slowdown_reasons_reported():
    got = _sampler(["1500, 2070, 1400, Active, Active, Active, Not Active"]).stop()
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert got["sm_mhz"] == 1500.0


def test_clock_sampler_without_nvidia_smi():
    got = bench.ClockSampler("0").stop()
    assert got["sm_mhz"] is None and got["reasons"] == ["nvidia-smi unavailable"]


def test_oracle_sample_is_a_subgraph_of_u():
    g = G.chung_lu_bipartite(3000, 1500, 40_000, 2.1, 2.1, 5)
    s, frac, r, dt = bench.oracle_sample(g, "total", 1, 0.05)
    assert 0 < frac <= 1.0 and dt >= 0
    assert r["total"] == oracle.vp(s)["total"]
    # same id spaces; every U row is kept whole or emptied
    assert (s.num_u, s.num_l) == (g.num_u, g.num_l) and s.num_edges <= g.num_edges
    kept = 0
    for u in range(g.num_u):
        row = s.adj_u[s.off_u[u]:s.off_u[u + 1]]
        if len(row):
            assert np.array_equal(row, g.adj_u[g.off_u[u]:g.off_u[u + 1]])
            kept += 1
    assert kept > 0
    desc = bench.sample_desc("powerlaw_20m", frac, s, r, "total")
    assert str(s.num_edges) in desc and f"W={r['wedges']}" in desc
    if frac < 1.0:
        assert "seeded" in desc


def test_default_outputs_and_peaks():
    assert bench.default_outputs("shopping_300m") == "all"
    assert bench.default_outputs("powerlaw_20m") == "total"
    pk = bench.measured_peaks()
    assert pk["hbm_gbs"] > 1000 and pk["source"] in ("measured", "fallback")


def test_reference_arm_json_contract():
    # the reference arm (the oracle on the host cores) on the small workload:
    # one JSON line with the contract's keys, its e2e equal to its value
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--workload", "uniform_small", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=root,
                       env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "impl", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
