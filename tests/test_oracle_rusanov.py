"""Pins of the oracle's Rusanov face flux (Sec. 4.4, Eq. 3.33) by hand computations on a
lattice of cubes, independent of the oracle's face routines.

Eq. 3.33 at a face node: G = 1/2 (F+ + F-) . n - 1/2 (s + 2 eps |lambda^v|) (q+ - q-), with
s the largest |v . n| + c over the nodes of the polygonal face on both sides,
|lambda^v| = max(4 mu / (3 rho), gamma mu / (Pr rho)) over both sides, and
eps = (2N + 1) / ((h+ + h-) sqrt(pi / 2)).  Every quantity in these tests is formed here
from the textbook Euler flux and the cube geometry; only the predictor (pinned elsewhere
against a dense space-time solve) is taken from the oracle.

The cell totals make the face flux visible on its own: the volume term sums to zero over a
cell (the basis sums to one, so its gradients sum to zero), hence the change of
sum_m (M_i u_i)_m in one step is minus the face integral of G, and on a sub-triangle the
face mass 2 * area * Z^ has column sums area / 3 at N = 1 (area times 1/2 in total).
"""
import math

import numpy as np
import pytest

from inputs import states
from inputs.lattice import split_cube_lattice
from oracle import scheme
from oracle.mesh import from_polymesh

GAMMA = 1.4


def _euler_flux(q):
    """[..., 5] conserved -> [..., 3 (direction), 5] textbook Euler flux."""
    rho = q[..., 0]
    v = q[..., 1:4] / rho[..., None]
    p = (GAMMA - 1.0) * (q[..., 4] - 0.5 * rho * np.sum(v * v, -1))
    F = np.empty(q.shape[:-1] + (3, 5))
    for e in range(3):
        F[..., e, 0] = q[..., 1 + e]
        for a in range(3):
            F[..., e, 1 + a] = q[..., 1 + a] * v[..., e] + (p if a == e else 0.0)
        F[..., e, 4] = (q[..., 4] + p) * v[..., e]
    return F


def _speed(q, n):
    rho = q[..., 0]
    v = q[..., 1:4] / rho[..., None]
    p = (GAMMA - 1.0) * (q[..., 4] - 0.5 * rho * np.sum(v * v, -1))
    return np.abs(v @ n) + np.sqrt(GAMMA * p / rho)


def _cell_totals(m, u):
    return np.array([c.wvec @ x for c, x in zip(m.cells, m.split(u))])


def _face_of(cube_centre, pts):
    """(axis, outward sign) of the cube face holding the points pts [k, 3]."""
    ax = int(np.argmin(np.ptp(pts, axis=0)))
    return ax, float(np.sign(pts[0, ax] - cube_centre[ax]))


@pytest.mark.parametrize("N", [1, 2])
@pytest.mark.parametrize("viscous", [False, True])
def test_rusanov_on_cellwise_constant_states(N, viscous):
    """Constant state in each cube (different from cube to cube): the predictor keeps it
    (q_bar = dt u, F_bar = dt F(u)), viscous stresses and heat flux vanish, and the total
    change of an interior cube over one step is
      -dt d^2 sum_faces [1/2 (F(u_j) + F(u_i)) . n - 1/2 (s + 2 eps |lambda^v|) (u_j - u_i)]
    with s = max(|v_i . n| + c_i, |v_j . n| + c_j).  Velocities have tangential parts, so
    |v| + c in place of |v . n| + c, a missing 1/2, another eps or a one-sided |lambda^v|
    would each change the result by far more than the tolerance."""
    n, d = 3, 0.4
    pm = split_cube_lattice((n, n, n), (1, 1, 1), d)
    m = from_polymesh(pm, N)
    rng = np.random.default_rng(7)
    C = m.n_cells
    rho = rng.uniform(0.7, 1.3, C)
    vel = rng.uniform(-0.6, 0.6, (C, 3))
    p = rng.uniform(0.6, 1.4, C)
    u = np.concatenate([np.tile(states.primitive_to_conserved(rho[i], vel[i], p[i]), (len(c.nodes), 1))
                        for i, c in enumerate(m.cells)])
    mu, Pr = (0.02, 0.71) if viscous else (0.0, 0.71)
    prm = scheme.Params(mu=mu, Pr=Pr, kappa=-1.0 if viscous else 0.0)
    dt = 2e-3
    new, _ = scheme.step(m, m.split(u), prm, dt=dt)
    dU = _cell_totals(m, np.concatenate(new)) - _cell_totals(m, u)
    centres = np.array([c.nodes.mean(axis=0) for c in m.cells])
    eps = (2 * N + 1) / ((d + d) * math.sqrt(math.pi / 2.0))
    i = int(np.argmin(np.linalg.norm(centres - 1.5 * d, axis=1)))      # the interior cube
    assert np.allclose(centres[i], 1.5 * d)
    qi = states.primitive_to_conserved(rho[i], vel[i], p[i])
    expect = np.zeros(5)
    for ax in range(3):
        for sgn in (-1.0, 1.0):
            nrm = np.zeros(3)
            nrm[ax] = sgn
            j = int(np.argmin(np.linalg.norm(centres - (centres[i] + d * nrm), axis=1)))
            assert np.isclose(np.linalg.norm(centres[j] - centres[i]), d)
            qj = states.primitive_to_conserved(rho[j], vel[j], p[j])
            s = max(_speed(qi, nrm), _speed(qj, nrm))
            lam_v = max(max(4.0 * mu / (3.0 * r), GAMMA * mu / (Pr * r)) for r in (rho[i], rho[j]))
            G = 0.5 * (_euler_flux(qi) + _euler_flux(qj)).transpose(1, 0) @ nrm - 0.5 * (s + 2 * eps * lam_v) * (qj - qi)
            expect -= dt * d * d * G
    np.testing.assert_allclose(dU[i], expect, rtol=0, atol=1e-11 * np.abs(expect).max())
    # the same with |v| + c in place of |v . n| + c differs by far more than the tolerance
    wrong = np.zeros(5)
    for ax in range(3):
        for sgn in (-1.0, 1.0):
            nrm = np.zeros(3)
            nrm[ax] = sgn
            j = int(np.argmin(np.linalg.norm(centres - (centres[i] + d * nrm), axis=1)))
            qj = states.primitive_to_conserved(rho[j], vel[j], p[j])
            s = max(np.linalg.norm(vel[i]) + math.sqrt(GAMMA * p[i] / rho[i]),
                    np.linalg.norm(vel[j]) + math.sqrt(GAMMA * p[j] / rho[j]))
            lam_v = max(max(4.0 * mu / (3.0 * r), GAMMA * mu / (Pr * r)) for r in (rho[i], rho[j]))
            G = 0.5 * (_euler_flux(qi) + _euler_flux(qj)).transpose(1, 0) @ nrm - 0.5 * (s + 2 * eps * lam_v) * (qj - qi)
            wrong -= dt * d * d * G
    assert np.abs(wrong - expect).max() > 1e3 * 1e-11 * np.abs(expect).max()


def _hand_face_total(m, i, qbar, Fbar, dt, N, d, scope):
    """-sum over the boundary sub-triangles of cell i of (area/3) sum_b G_b at N = 1, with the
    wave speed s taken over ``scope``: "face" (all nodes of the square face, both sides; the
    reading of Eq. 3.33), "tri" (the sub-triangle's nodes) or "node" (the node itself)."""
    cd = m.cells[i]
    ci = cd.nodes.mean(axis=0)
    eps = (2 * N + 1) / ((d + d) * math.sqrt(math.pi / 2.0))
    tris = []
    for bt in cd.bfaces:
        X = cd.nodes[bt.nodes]
        ax, sgn = _face_of(ci, X)
        nrm = np.zeros(3)
        nrm[ax] = sgn
        j = bt.nbr
        Xj = m.cells[j].nodes
        # pair the neighbour's nodes by position (not through the oracle's matching)
        pj = [int(np.argmin(np.linalg.norm(Xj - x, axis=1))) for x in X]
        assert max(np.linalg.norm(Xj[pj] - X, axis=1)) < 1e-12
        qm, qp = qbar[i][bt.nodes], qbar[j][pj]
        Fm, Fp = Fbar[i][bt.nodes], Fbar[j][pj]
        area = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
        tris.append((ax, sgn, nrm, qm, qp, Fm, Fp, area))
    smax_face = {}
    for ax, sgn, nrm, qm, qp, *_ in tris:
        s = max(_speed(qm / dt, nrm).max(), _speed(qp / dt, nrm).max())
        smax_face[(ax, sgn)] = max(smax_face.get((ax, sgn), 0.0), s)
    tot = np.zeros(5)
    for ax, sgn, nrm, qm, qp, Fm, Fp, area in tris:
        if scope == "face":
            s = np.full(3, smax_face[(ax, sgn)])
        elif scope == "tri":
            s = np.full(3, max(_speed(qm / dt, nrm).max(), _speed(qp / dt, nrm).max()))
        else:
            s = np.maximum(_speed(qm / dt, nrm), _speed(qp / dt, nrm))
        G = 0.5 * np.einsum("bev,e->bv", Fp + Fm, nrm) - 0.5 * s[:, None] * (qp - qm)
        tot -= area / 3.0 * G.sum(axis=0)
    return tot


def test_rusanov_wave_speed_is_the_maximum_over_the_polygonal_face():
    """Per-cube linear densities (different gradients in every cube) with uniform velocity
    and pressure, P1: the face-node states differ along each face, so the largest
    |v . n| + c over the whole square face (both sides), over one sub-triangle, or at one
    node are different numbers.  The oracle's one-step change of an interior cube's totals
    equals the hand-assembled face integral with the face-wide maximum (q_bar from the
    oracle's predictor, F_bar formed here from the nodal q with the Euler flux), and the
    two other scopes miss it by far more than the tolerance."""
    n, d, N = 3, 0.4, 1
    pm = split_cube_lattice((n, n, n), (1, 1, 1), d)
    m = from_polymesh(pm, N)
    rng = np.random.default_rng(11)
    vel = np.array([0.35, -0.2, 0.15])
    parts = []
    for c in m.cells:
        cc = c.nodes.mean(axis=0)
        rho = rng.uniform(0.8, 1.2) + (c.nodes - cc) @ rng.uniform(-0.6, 0.6, 3)
        parts.append(states.primitive_to_conserved(rho, np.tile(vel, (len(rho), 1)), np.ones(len(rho))))
    u = np.concatenate(parts)
    prm = scheme.Params()
    dt = 4e-3
    uc = m.split(u)
    new, _ = scheme.step(m, uc, prm, dt=dt)
    dU = _cell_totals(m, np.concatenate(new)) - _cell_totals(m, u)
    R = m.R
    qbar, Fbar = [], []
    for k in range(m.n_cells):
        q, _ = scheme.predictor(m, k, uc[k], dt, 0.0, 0.0, prm)
        qbar.append(dt * np.einsum("t,ntv->nv", R.w, q))
        Fbar.append(dt * np.einsum("t,ntev->nev", R.w, _euler_flux(q)))
    centres = np.array([c.nodes.mean(axis=0) for c in m.cells])
    i = int(np.argmin(np.linalg.norm(centres - 1.5 * d, axis=1)))
    face = _hand_face_total(m, i, qbar, Fbar, dt, N, d, "face")
    tol = 1e-12 * np.abs(face).max()
    np.testing.assert_allclose(dU[i], face, rtol=0, atol=tol)
    for scope in ("tri", "node"):
        other = _hand_face_total(m, i, qbar, Fbar, dt, N, d, scope)
        assert np.abs(other - face).max() > 1e3 * tol, scope
