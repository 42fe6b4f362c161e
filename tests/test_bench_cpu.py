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


def test_predictor_roofline_by_hand():
    """The roofline fields of the bench line recomputed by hand for the 32^3 N = 3 workload's
    figures: HBM-bound when the bytes take longer than the 3xTF32 contractions plus the FMA
    work, the fraction being achieved GB/s over the measured copy bandwidth; tensor-bound
    (3xTF32 rate = half the BF16 burst over three) otherwise."""
    peaks = {"hbm_gbs": 6800.3, "bf16_tflops": 1896.7, "sm_max_mhz": 2070.0}
    f_con, f_pw, abytes, ms = 425031110760.0, 56814155560.0, 14161675240.0, 14.1808256149292
    r = bench.predictor_roofline(f_con, f_pw, abytes, ms, peaks)
    t_hbm = abytes / 6800.3e9
    t_ten = f_con / (1896.7 / 2 / 3 * 1e12)
    t_fma = f_pw / (152 * 128 * 2 * 2070e6)
    assert t_hbm > t_ten + t_fma and r["bound"] == "hbm"
    assert abs(r["frac"] - (abytes / (ms / 1e3) / 1e9) / 6800.3) < 1e-12
    assert abs(r["frac"] - 0.14685) < 1e-4
    assert abs(r["roofline_ms"] - 1e3 * t_hbm) < 1e-9 and abs(r["frac_roofline_time"] - r["frac"]) < 1e-12
    # ten times the contraction work: the tensor pipe sets the roofline
    r2 = bench.predictor_roofline(10 * f_con, f_pw, abytes, ms, peaks)
    assert r2["bound"] == "tensor"
    assert abs(r2["roofline_ms"] - 1e3 * (10 * t_ten + t_fma)) < 1e-9
    assert abs(r2["frac"] - (10 * f_con / (ms / 1e3) / 1e12) / (1896.7 / 6)) < 1e-12
