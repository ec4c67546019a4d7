"""bench.py's reference arm (`--impl reference`: the oracle's OpenMP build timed on
the host cores on bounded samples of the 65536-cell workload) needs no GPU: it
prints one JSON line with the contract's keys, and a rank other than 0 of a
multi-rank launch prints nothing and exits 0; and the per-field error figures of
the bench line on a case computed by hand."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, args=("--steps", "1", "--warmup", "0")):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           *args], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    p = _run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "cell-updates/s (x RK stages) of the hybrid HWENO step"
    assert d["unit"] == "cell-stages/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "sample" in cb
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("1D Euler two-state, 65536 cells")


def test_reference_arm_other_ranks_are_silent():
    p = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_field_errors_by_hand():
    """The per-field figures of the bench line on a hand-made case: one cell of
    one field off by 0.5 out of sums of 4 (averages) and 2 (first moments)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    ref = np.zeros((3, 2, 4))
    ref[:, 0] = 1.0   # averages: sum 4 per component
    ref[:, 1] = 0.5   # first moments: sum 2
    a = ref.copy()
    a[1, 1, 2] += 0.5  # m first moment, one cell
    a[2, 0, 0] -= 0.25  # E average, one cell
    e = bench.field_errors(a, ref)
    assert e["rho_average"] == {"L1": 0.0, "Linf": 0.0, "rel_L1": 0.0}
    assert e["m_first_moment"]["L1"] == 0.125 and e["m_first_moment"]["Linf"] == 0.5
    assert e["m_first_moment"]["rel_L1"] == 0.25
    assert e["m_first_moment"]["L1_over_avg_scale"] == 0.5  # 0.5 / (4 / 4)
    assert e["E_average"]["rel_L1"] == 0.0625 and e["E_average"]["Linf"] == 0.25
    assert set(e) == {"%s_%s" % (n, m) for n in ("rho", "m", "E")
                      for m in ("average", "first_moment")}
