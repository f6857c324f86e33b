"""bench.py --impl reference on the CPU: the oracle timed on a bounded sample,
printed as one JSON line with the keys of the benchmark contract; and the
command-line form of the host checkpoint merge."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-points", "32"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    for k in ("metric", "value", "unit", "ms_per_step", "higher_is_better", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_duct_json_line():
    """The reference arm of the one-homogeneous-direction workload."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "duct_16x9x7_s4", "--steps", "1", "--warmup", "0", "--ref-points", "64"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "duct_16x9x7_s4"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_merge_command_line(tmp_path):
    from paper_1910_06409_gb300 import merge as M
    ny = 5
    rng = np.random.default_rng(7)
    paths = []
    parts = []
    for r in range(2):
        ck = {"header": {"nx": 8, "nz": 8, "ny": ny, "precision": 0, "pair_domain": 0, "nzt": 0, "nxt": 0,
                         "term_set": 127, "mean_count": 1.0, "snap_count": 1.0, "Lx": 1.0, "Lz": 1.0, "nu": 0.1},
              "mean_sum": rng.standard_normal(4 * ny), "stats": rng.standard_normal(M.NSTAT * ny),
              "mean": np.linspace(0.0, 1.0, 4 * ny), "acc": rng.standard_normal(6) + 1j * rng.standard_normal(6)}
        p = str(tmp_path / f"j{r}.ckpt")
        M.write(p, ck)
        paths.append(p)
        parts.append(ck)
    out = str(tmp_path / "out.ckpt")
    r = subprocess.run([sys.executable, "-m", "paper_1910_06409_gb300.merge", out, *paths], capture_output=True,
                       text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    got = M.read(out)
    assert np.array_equal(got["acc"], parts[0]["acc"] + parts[1]["acc"])
    assert got["header"]["snap_count"] == 2.0
