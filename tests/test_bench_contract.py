"""The benchmark's output contract on the CPU: the reference arm (the oracle on the host cores)
prints one JSON line with the keys the harness reads, and the solver's flop accounting is additive
over spaces and grows with the iteration count."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "n10",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "active spaces/s" and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("n10: 10 orbitals (3 occ, 7 virt)")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_solver_flops_additive_and_increasing():
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(0)
    a = rng.integers(0, 6, 500)
    b = rng.integers(0, 6, 300)
    fa, fb, fab = bench.solver_flops(a), bench.solver_flops(b), bench.solver_flops(np.concatenate([a, b]))
    assert abs(fab - (fa + fb)) <= 1e-9 * fab
    per = [bench.solver_flops(np.array([m])) for m in range(8)]
    assert all(x < y for x, y in zip(per, per[1:]))
    # a space that stays at Phi costs its Phi column only; one that iterates applies sigma each time
    assert per[0] == 2 * 153 + 2 * 117
    assert per[2] - per[1] > 400 * (2 * 12 * 12)
