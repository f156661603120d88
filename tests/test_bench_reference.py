"""`bench.py --impl reference` (the CPU oracle timed as the reference arm)
prints one JSON line with the contract's keys, on a small workload (2D 24^2)
so that it runs in seconds on the CPU.  The oracle times a bounded sample of
the workload (here sample 1 and four of the eight right-hand sides), and the
line's config says so: its solves_per_step and ms_per_step are those of the
timed sample, not of the whole pass."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line_has_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "t2d_24", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    cfg = line["config"]
    assert cfg["workload"] == "t2d_24" and cfg["solves_per_pass"] == 2 * 8
    assert cfg["solves_per_step"] == 4 < cfg["solves_per_pass"]            # the timed sample, not the pass
    assert "RHS [0, 1, 2, 3]" in cfg["timed_sample"]
    # ms_per_step is the time of one step of the timed sample
    assert abs(line["value"] - cfg["solves_per_step"] / (line["ms_per_step"] / 1e3)) <= 1e-3 * line["value"]   # ms_per_step is rounded
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_contender_line_has_the_contract_keys():
    """The GPU arm's JSON line, built from a synthetic result record (no GPU needed)."""
    import argparse
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(workload="c2_3d64", steps=5, warmup=3)
    res = dict(value=4000.0, ms=80.0, learn={}, solves_per_step=320, rank_V=117, mean_iters=39.0,
               phases={"check": 6.0, "cg": 52.0}, seed_s=2.0,
               roofline={"bound": "hbm", "achieved": 5900.0, "peak": 6800.0, "unit": "GB/s", "frac": 0.87,
                         "traffic": None},
               e2e={"value": 3990.0, "unit": "solves/s", "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1},
               clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, launches=2490, base=None,
               nolearn=None)
    cpu = {"value": 5.0, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": "s"}
    line = bench.contender_line(args, 1, res, cpu)
    json.dumps(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in line, k
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    assert line["config"]["workload"] == "c2_3d64" and line["config"]["solves_per_step"] == 320
    assert line["n_gpus"] == 1 and line["config"]["parallelism"] == "single GPU"


def test_reference_line_at_192_cubed_is_unavailable_with_its_reason():
    """The oracle cannot seed the 192^3 configuration within a bench run (its
    ARPACK eigensolver alone takes longer), so the reference arm says so
    instead of timing another workload under this one's name."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "c5_3d192", "--steps", "20", "--warmup", "5"], capture_output=True, text=True, timeout=120,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "ARPACK" in line["unavailable"]
