"""Local amplification of one cell under the ADER-AFE step, from oracle steps.

TEST INFRASTRUCTURE ONLY (see the package docstring): a command-line analysis.  Around the
uniform state rho = 1, u = (1, 1, 1), p = 1 the density wave reduces to linear advection of
rho, so one step maps a density perturbation linearly.  G_ii is that map restricted to the
nodes of cell i with its face neighbours held at the background: column j is the response
of the cell's densities to a perturbation of its node j (finite differences of oracle
steps on a sub-mesh made of the cell and its face neighbours).  A spectral radius above 1
means the cell amplifies a perturbation of its own by itself, whatever its neighbours do.
The time step is the CFL step of the whole mesh, dt = CFL h_min / ((2N+1) lambda) with
lambda = |u| + c of the background.

    python -m oracle.local_amplification --n 32 --N 3 --cfl 0.15 --cells 6044 [--flat 0]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from inputs.voronoi import FLAT, periodic_voronoi

from . import scheme
from .mesh import OracleMesh


def cell_lengths(pm):
    """6|P|/|dP| per cell and the smallest height of a cell centre over its fan triangles."""
    X = pm.subtet_coords()
    det = np.abs(np.linalg.det(X[:, 1:] - X[:, :1]))
    cell = np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr))
    vol = np.bincount(cell, weights=det / 6.0, minlength=pm.n_cells)
    tri = 0.5 * np.linalg.norm(np.cross(X[:, 2] - X[:, 1], X[:, 3] - X[:, 1]), axis=1)  # the fan triangle
    area = np.bincount(cell, weights=tri, minlength=pm.n_cells)
    height = np.full(pm.n_cells, np.inf)
    np.minimum.at(height, cell, det / (2.0 * tri))
    return 6.0 * vol / area, height


def face_neighbours(pm):
    """Cells sharing at least three vertex ids (a face) with each cell."""
    ptr, vtx = pm.cell_subtet_ptr, pm.subtet_vtx
    vsets = [set(vtx[ptr[c]:ptr[c + 1]].ravel().tolist()) for c in range(pm.n_cells)]
    owners: dict = {}
    for c, vs in enumerate(vsets):
        for v in vs:
            owners.setdefault(v, []).append(c)

    def nbrs(c):
        count: dict = {}
        for v in vsets[c]:
            for d in owners[v]:
                if d != c:
                    count[d] = count.get(d, 0) + 1
        return sorted(d for d, k in count.items() if k >= 3)
    return nbrs


def local_map(pm, c, nbrs, N, dt, eps=1e-6):
    """G_ii of cell c (density response on its own nodes), [N_i, N_i]."""
    cells = [c] + nbrs(c)
    ptr, vtx, sh = [0], [], []
    for d in cells:
        k0, k1 = pm.cell_subtet_ptr[d], pm.cell_subtet_ptr[d + 1]
        vtx.append(pm.subtet_vtx[k0:k1])
        sh.append(pm.subtet_shift[k0:k1])
        ptr.append(ptr[-1] + k1 - k0)
    m = OracleMesh(pm.xyz, np.array(ptr), np.concatenate(vtx), np.concatenate(sh).astype(np.int64), pm.period, N,
                   periodic=False)
    gamma = scheme.Params().gamma
    bg = np.array([1.0, 1.0, 1.0, 1.0, 1.0 / (gamma - 1.0) + 1.5])
    drho = np.array([1.0, 1.0, 1.0, 1.0, 1.5])                 # d(q)/d(rho) at fixed u, p
    u0 = [np.tile(bg, (len(cd.nodes), 1)) for cd in m.cells]
    prm = scheme.Params(picard_tol=1e-13, picard_max=200)
    base, _ = scheme.step(m, u0, prm, dt=dt, cells=[0])
    n_i = len(m.cells[0].nodes)
    G = np.zeros((n_i, n_i))
    for j in range(n_i):
        u = [x.copy() for x in u0]
        u[0][j] += eps * drho
        new, _ = scheme.step(m, u, prm, dt=dt, cells=[0])
        G[:, j] = (new[0][:, 0] - base[0][:, 0]) / eps
    return G


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--N", type=int, default=3)
    ap.add_argument("--cfl", type=float, nargs="+", default=[0.15])
    ap.add_argument("--cells", type=int, nargs="*", default=None, help="default: the 3 smallest centre heights")
    ap.add_argument("--flat", type=float, default=FLAT)
    a = ap.parse_args()
    pm = periodic_voronoi(a.n, flat=a.flat)
    h, height = cell_lengths(pm)
    cells = a.cells if a.cells else [int(c) for c in np.argsort(height)[:3]]
    nbrs = face_neighbours(pm)
    lam = math.sqrt(3.0) + math.sqrt(scheme.Params().gamma)
    for c in cells:
        rho = []
        for cfl in a.cfl:
            G = local_map(pm, c, nbrs, a.N, cfl * h.min() / ((2 * a.N + 1) * lam))
            rho.append([cfl, float(max(abs(np.linalg.eigvals(G))))])
        print(json.dumps({"cell": c, "N": a.N, "centre_height_over_spacing": float(height[c] * a.n),
                          "spectral_radius": rho}), flush=True)


if __name__ == "__main__":
    main()
