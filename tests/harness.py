"""Shared test plumbing: run the oracle and the C-ABI library on the same seeded inputs.

The two sides share no arithmetic: each builds its own AFE nodes.  Nodes are paired per
cell by position only to compare results, and both sides start from the same nodal
values, computed at the oracle's node positions.
"""
from __future__ import annotations

import numpy as np

from oracle import scheme
from oracle.mesh import from_polymesh


def oracle_params(p) -> scheme.Params:
    """Oracle parameters equal to an afe_params (Euler ignores mu; kappa < 0 only for NS)."""
    ns = p.equations == 1
    return scheme.Params(gamma=p.gamma, R=p.R, mu=p.mu if ns else 0.0, Pr=p.Pr,
                         kappa=p.kappa if ns else max(p.kappa, 0.0), cfl=p.cfl, limiter=bool(p.limiter),
                         m1=p.m1, picard_tol=p.picard_tol, picard_max=p.picard_max,
                         visc_dt_subtet=bool(p.visc_dt_subtet), h_diameter=bool(p.h_diameter))


def node_permutation(om, lib_xyz, lib_ptr):
    """perm[lib_node] = oracle global node with the same position in the same cell."""
    perm = np.empty(len(lib_xyz), np.int64)
    for c, cd in enumerate(om.cells):
        a, b = lib_ptr[c], lib_ptr[c + 1]
        if b - a != len(cd.nodes):
            raise AssertionError(f"cell {c}: library has {b - a} nodes, oracle {len(cd.nodes)}")
        X = lib_xyz[a:b]
        d2 = ((X[:, None, :] - cd.nodes[None, :, :]) ** 2).sum(-1)
        j = np.argmin(d2, axis=1)
        if len(set(j.tolist())) != len(j) or d2[np.arange(len(j)), j].max() > 1e-20:
            raise AssertionError(f"cell {c}: node positions do not pair up")
        perm[a:b] = om.node_ptr[c] + j
    return perm


def rel_linf(a, b):
    """max over variables of max|a - b| / max|b| (per conserved variable)."""
    return max(np.abs(a[:, v] - b[:, v]).max() / max(np.abs(b[:, v]).max(), 1e-300) for v in range(a.shape[1]))


def rel_l2(a, b):
    return max(np.linalg.norm(a[:, v] - b[:, v]) / max(np.linalg.norm(b[:, v]), 1e-300) for v in range(a.shape[1]))


def rel_l2_fields(a, b):
    """max of the relative L2 errors of the density, the momentum vector field and the total
    energy.  The momentum is normalised as one vector field: in flows where one component
    vanishes identically at t = 0 (w in the Taylor-Green vortex) that component's own norm
    is many orders below the others, and its error, set by FP32 rounding of terms that scale
    with the pressure, measured against it says nothing about the accuracy of the flow."""
    def rel(x, y):
        return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)
    return max(rel(a[:, 0], b[:, 0]), rel(a[:, 1:4], b[:, 1:4]), rel(a[:, 4], b[:, 4]))


class Pair:
    """An oracle mesh and a library handle built from the same PolyMesh."""

    def __init__(self, pm, params, om=None):
        from paper_2605_00619_gb300 import afe
        self.afe = afe
        self.pm = pm
        self.p = params
        self.om = om if om is not None else from_polymesh(pm, params.order)
        self.prm = oracle_params(params)
        self.h = afe.create_from_polymesh(pm, params)
        self.lib_ptr = afe.afe_node_ptr(self.h, pm.n_cells)
        self.lib_xyz = afe.afe_get_node_coords(self.h)
        self.perm = node_permutation(self.om, self.lib_xyz, self.lib_ptr)

    def set_state(self, u_oracle):
        self.u = u_oracle.copy()
        self.afe.afe_set_state(self.h, u_oracle[self.perm])

    def lib_state(self):
        out = np.empty_like(self.u)
        out[self.perm] = self.afe.afe_get_state(self.h)
        return out

    def oracle_step(self, dt=None):
        new, info = scheme.step(self.om, self.om.split(self.u), self.prm, dt=dt)
        self.u = np.concatenate(new)
        return info

    def lib_step(self, dt=0.0, check=True):
        return self.afe.afe_step(self.h, dt, check=check)

    def close(self):
        self.afe.afe_mesh_destroy(self.h)
        self.h = None
