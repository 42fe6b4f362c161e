"""Host-side parts of bench.py's studies (CPU only)."""
import numpy as np

import bench
from inputs import radial, states


def test_radial_comparison_of_the_reference_with_itself():
    """The radial reference sampled at scattered points compares with itself with L1 errors at
    the interpolation level and the same shock radius (to a shell width)."""
    rref, wref = radial.explosion_reference(t_end=0.1, n=1500, R=1.75)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1.0, 1.0, size=(20000, 3))
    r = np.linalg.norm(x, axis=1)
    w = np.stack([np.interp(r, rref, wref[:, j]) for j in range(3)], axis=1)
    vel = w[:, 1:2] * x / np.maximum(r, 1e-12)[:, None]
    q = states.primitive_to_conserved(w[:, 0], vel, w[:, 2])
    ptr = np.arange(0, 20001, 10)
    vol = np.full(2000, 8.0 / 2000)
    out = bench.compare_with_radial(x, q, ptr, vol, rref, wref)
    assert max(out["l1_vs_radial_reference"].values()) < 1e-12
    assert abs(out["shock_radius"] - out["shock_radius_reference"]) <= 0.95 / 95 + 1e-12
    assert 0.55 < out["shock_radius_reference"] < 0.9


def test_reference_arm_prints_one_valid_line():
    """`bench.py --impl reference` (the oracle timed on the host) prints one JSON line with
    the contract's keys, its own cpu_baseline and an e2e object with no transfers."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--order", "1",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
