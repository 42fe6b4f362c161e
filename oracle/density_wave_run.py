"""Full-length oracle run of the density-wave convergence case.

TEST INFRASTRUCTURE ONLY (see the package docstring): a command-line check that integrates
the density wave rho = 1 + 0.2 sin(2 pi (x+y+z)), u = (1,1,1), p = 1 on a periodic
jittered-Voronoi mesh to t = 0.1 with equal steps (the CFL step of the initial state,
shortened to land on t = 0.1) and prints the error in rho against the exact solution: the
volume-weighted nodal L2 norm sqrt(sum_i |P_i| mean_{n in P_i} e_n^2) and the max norm, the
numbers the GPU accuracy study reports for the same mesh, order and CFL.

    python -m oracle.density_wave_run --n 8 --N 2 --cfl 0.2 [--thin 0.04] [--flat 0]

The stored result tests/golden/density_wave_8c_N2.json was written by this command with
the defaults (``> tests/golden/density_wave_8c_N2.json``).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from inputs import states
from inputs.voronoi import FLAT, THIN, periodic_voronoi

from . import scheme
from .mesh import from_polymesh


def run(n, N, cfl, t_end=0.1, thin=THIN, flat=FLAT):
    m = from_polymesh(periodic_voronoi(n, thin=thin, flat=flat), N)
    x = m.node_coords()
    uc = m.split(states.density_wave(x))
    prm = scheme.Params(cfl=cfl)
    nsteps = int(math.ceil(t_end / scheme.cfl_dt(m, uc, [0.0] * m.n_cells, prm) - 1e-9))
    dt = t_end / nsteps
    t0 = time.perf_counter()
    for _ in range(nsteps):
        uc, _ = scheme.step(m, uc, prm, dt=dt)
    e2 = (np.concatenate(uc)[:, 0] - states.density_wave(x, t=t_end)[:, 0]) ** 2
    l2 = math.sqrt(sum(c.vol * float(np.mean(e2[m.node_ptr[i]:m.node_ptr[i + 1]])) for i, c in enumerate(m.cells)))
    return {"n": n, "N": N, "cfl": cfl, "thin": thin, "flat": flat, "steps": nsteps, "dt": dt, "l2_rho": l2,
            "linf_rho": float(np.sqrt(e2.max())), "seconds": time.perf_counter() - t0}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--N", type=int, default=2)
    ap.add_argument("--cfl", type=float, default=0.2)
    ap.add_argument("--thin", type=float, default=THIN)
    ap.add_argument("--flat", type=float, default=FLAT)
    a = ap.parse_args()
    print(json.dumps(run(a.n, a.N, a.cfl, thin=a.thin, flat=a.flat)))
