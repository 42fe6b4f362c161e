"""One explicit ADER-AFE-DG step, written as plain loops over cells in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Order of one step (readings of Sec. 4 listed beside each function):
  1. artificial-viscosity detector at t^n (Sec. 4.5): beta_i, mu_i;
  2. time step from the CFL condition (Sec. 4.2, Eq. timestep);
  3. space-time predictor per cell, the fixed-point iteration of Eq. ader4;
  4. time-integrated predictor and fluxes (Eq. TAvectors);
  5. Rusanov fluxes on every cell-boundary sub-triangle (Eq. 3.33);
  6. corrector M_i (u^{n+1} - u^n) = volume term - face term (Sec. 4.4).
Conserved variables are ordered (rho, rho u, rho v, rho w, rho E).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .mesh import OracleMesh


@dataclass
class Params:
    gamma: float = 1.4
    R: float = 1.0            # gas constant (Sec. 5: R = 1)
    mu: float = 0.0           # dynamic viscosity
    Pr: float = 0.71
    kappa: float = 0.0        # heat conduction; < 0 means mu_i * gamma * c_v / Pr
    cfl: float = 0.3
    limiter: bool = False
    m1: float = 0.1           # Sec. 4.5
    picard_tol: float = 1e-12
    picard_max: int = 64
    visc_dt_subtet: bool = False  # viscous term of the time step with the smallest sub-tet length
    h_diameter: bool = False      # h_i = the cell's diameter instead of 6|P_i| / |dP_i|

    @property
    def cv(self):
        return self.R / (self.gamma - 1.0)


# ---------------------------------------------------------------------------
# pointwise physics (Sec. 2)


def primitives(Q, gamma):
    rho = Q[..., 0]
    v = Q[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (Q[..., 4] - 0.5 * rho * np.sum(v * v, axis=-1))
    return rho, v, p


def flux(Q, gradQ, mu, kappa, prm: Params):
    """Physical flux tensor F(Q, grad Q) at points: returns [..., 3 (direction e), 5].

    F_e = (rho v_e, rho v v_e + sigma[:, e], v . (rho E I + sigma)[:, e] - kappa dT/dx_e),
    sigma = (p + 2/3 mu div v) I - mu (grad v + grad v^T)  (Eq. stress_tensor);
    gradQ[..., e, var] = dQ_var / dx_e (ignored when mu = kappa = 0).
    """
    g = prm.gamma
    rho, v, p = primitives(Q, g)
    E = Q[..., 4]
    sigma = p[..., None, None] * np.eye(3)
    heat = np.zeros(Q.shape[:-1] + (3,))
    if mu != 0.0 or kappa != 0.0:
        drho = gradQ[..., :, 0]                                     # [..., e]
        dm = gradQ[..., :, 1:4]                                     # [..., e, a]
        dv = (dm - v[..., None, :] * drho[..., :, None]) / rho[..., None, None]   # dv_a/dx_e at [..., e, a]
        gv = np.swapaxes(dv, -1, -2)                                # [..., a, e] = dv_a/dx_e
        div = np.trace(gv, axis1=-2, axis2=-1)
        dE = gradQ[..., :, 4]
        vv = np.sum(v * v, axis=-1)
        dp = (g - 1.0) * (dE - 0.5 * vv[..., None] * drho - rho[..., None] * np.einsum("...a,...ea->...e", v, dv))
        dT = (dp / rho[..., None] - p[..., None] * drho / rho[..., None] ** 2) / prm.R
        sigma = sigma + (2.0 / 3.0) * mu * div[..., None, None] * np.eye(3) - mu * (gv + np.swapaxes(gv, -1, -2))
        heat = kappa * dT
    F = np.empty(Q.shape[:-1] + (3, 5))
    F[..., :, 0] = rho[..., None] * v
    F[..., :, 1:4] = rho[..., None, None] * v[..., None, :] * v[..., :, None] + np.swapaxes(sigma, -1, -2)
    F[..., :, 4] = E[..., None] * v + np.einsum("...a,...ae->...e", v, sigma) - heat
    return F


def sound_speed(rho, p, gamma):
    return np.sqrt(gamma * p / rho)


def viscous_eigen(rho, mu, kappa, prm: Params):
    """|lambda^v| = max(4 mu/(3 rho), gamma mu/(Pr rho)) with Pr = mu gamma c_v / kappa (Sec. 2)."""
    return np.maximum(4.0 * mu / (3.0 * rho), kappa / (prm.cv * rho))


def cell_kappa(mu_i, prm: Params):
    return prm.kappa if prm.kappa >= 0.0 else mu_i * prm.gamma * prm.cv / prm.Pr


# ---------------------------------------------------------------------------
# Sec. 4.5 detector and artificial viscosity


def cell_means(mesh: OracleMesh, u_cells):
    """u_bar_i = (1^T M_i u_i) / |P_i| : the mean of the AFE polynomial over P_i."""
    return np.array([c.wvec @ u for c, u in zip(mesh.cells, u_cells)]) / \
        np.array([c.vol for c in mesh.cells])[:, None]


def limiter(mesh: OracleMesh, u_cells, prm: Params):
    """Flattener beta_i (Eq. beta3D) and mu_i = mu + beta_i rho_i |lambda|_i h_s with h_s = h_i/(2N+1).

    div v_i = (1/|P_i|) sum over cell-boundary sub-triangles of area (v_nbr - v_i) . n with
    cell-mean velocities; c_min over the cell and its face neighbours; domain-boundary
    faces contribute nothing.
    """
    ub = cell_means(mesh, u_cells)
    C = mesh.n_cells
    beta = np.zeros(C)
    mu_c = np.full(C, prm.mu)
    for i in range(C):
        beta[i], mu_c[i] = limiter_cell(mesh, i, ub, prm)
    return beta, mu_c


def limiter_cell(mesh: OracleMesh, i, ub, prm: Params):
    """beta_i and mu_i of cell i from the cell means ``ub`` (indexable by cell: the cell's own
    and its face neighbours' means are read)."""
    rho, v, p = primitives(ub[i], prm.gamma)
    c_i = sound_speed(rho, p, prm.gamma)
    cd = mesh.cells[i]
    div = 0.0
    cmin = c_i
    for bt in cd.bfaces:
        if bt.nbr < 0:
            continue
        rn, vn, pn = primitives(ub[bt.nbr], prm.gamma)
        div += bt.area * float((vn - v) @ bt.normal)
        cmin = min(cmin, sound_speed(rn, pn, prm.gamma))
    div /= cd.vol
    beta = min(1.0, max(0.0, -(div + prm.m1 * cmin) / (prm.m1 * cmin)))
    lam = np.linalg.norm(v) + c_i
    return beta, prm.mu + beta * rho * lam * cell_length(cd, prm) / (2 * mesh.N + 1)


# ---------------------------------------------------------------------------
# Sec. 4.2 time step


def cell_length(cd, prm: Params) -> float:
    """The characteristic length h_i of Sec. 4.2: 6|P_i| / |dP_i|, or the cell's diameter
    (the paper's example) when ``prm.h_diameter``."""
    return cd.diam if prm.h_diameter else cd.h


def cfl_dt(mesh: OracleMesh, u_cells, mu_c, prm: Params):
    """dt = CFL min h / ((2N+1) max(|lambda| + 2 |lambda^v| (2N+1)/h)) over all nodes at t^n."""
    worst, h_min = cfl_pieces(mesh, u_cells, mu_c, prm, range(mesh.n_cells))
    return cfl_from_pieces(mesh, worst, h_min, prm)


def cfl_pieces(mesh: OracleMesh, u_cells, mu_c, prm: Params, cells):
    """The two reductions of the CFL time step over ``cells``: the largest bracket
    |lambda| + 2 |lambda^v| (2N+1)/h at their nodes, and the smallest characteristic length."""
    N = mesh.N
    worst = 0.0
    for i in cells:
        cd, u = mesh.cells[i], u_cells[i]
        rho, v, p = primitives(u, prm.gamma)
        lam = np.linalg.norm(v, axis=1) + sound_speed(rho, p, prm.gamma)
        lv = viscous_eigen(rho, mu_c[i], cell_kappa(mu_c[i], prm), prm)
        hv = cd.hsub if prm.visc_dt_subtet else cell_length(cd, prm)
        worst = max(worst, float(np.max(lam + 2.0 * lv * (2 * N + 1) / hv)))
    h_min = min(cell_length(mesh.cells[i], prm) for i in cells)
    return worst, h_min


def cfl_from_pieces(mesh: OracleMesh, worst, h_min, prm: Params):
    return prm.cfl * h_min / ((2 * mesh.N + 1) * worst)


# ---------------------------------------------------------------------------
# Sec. 4.3 space-time predictor


def subtet_fluxes(mesh: OracleMesh, i, qt, mu, kappa, prm):
    """Physical flux at the P_N nodes of every sub-tet of cell i for one time slice.

    qt: [N_i, 5] nodal state.  Returns [S, Np, 3, 5].  The viscous part uses the
    gradient of the sub-tet's own polynomial (grad_x = J^{-T} grad_xi).
    """
    cd = mesh.cells[i]
    R = mesh.R
    Q = qt[cd.A]                                              # [S, Np, 5]
    if mu == 0.0 and kappa == 0.0:
        return flux(Q, None, 0.0, 0.0, prm)
    gxi = np.einsum("djl,slv->sdjv", R.D, Q, optimize=True)                  # d/dxi_d at node j
    gx = np.einsum("sde,sdjv->sjev", cd.Jinv, gxi, optimize=True)            # d/dx_e at node j
    return flux(Q, gx, mu, kappa, prm)


def predictor(mesh: OracleMesh, i, u_i, dt, mu, kappa, prm: Params):
    """Fixed-point iteration of Eq. ader4 for cell i.

    K_1,i q^{r+1} = F_0 u^ - sum_k |J_ik| (K_xi f*_ik + K_eta g*_ik + K_zeta h*_ik),
    with the space-time matrices factorised through theta = phi (x) psi:
      K_1,i = M_i (x) K1t,   F_0 u^ = (M_i u^) (x) psi(0),
      K_d   = diag(w) (x) S^_d,   |J_ik| f*_d = dt * adj(J_ik)[d, :] . F.
    Initial guess q^0 = u^ at every time node.  Stops when
    max |q^{r+1} - q^r| <= tol * max(1, max |q^r|), or after picard_max iterations.
    Returns q [N_i, Nt, 5] and the iteration count.
    """
    R = mesh.R
    cd = mesh.cells[i]
    Nt = R.Nt
    q = np.repeat(u_i[:, None, :], Nt, axis=1)
    G = dt * cd.adj                                           # [S, 3(d), 3(e)]
    F0u = (cd.M @ u_i)[:, None, :] * R.psi0[None, :, None]
    it = 0
    for it in range(1, prm.picard_max + 1):
        rhs = np.zeros_like(q)
        for t in range(Nt):
            F = subtet_fluxes(mesh, i, q[:, t], mu, kappa, prm)  # [S, Np, 3, 5]
            Fstar = np.einsum("sde,sjev->sdjv", G, F, optimize=True)             # |J| f*, |J| g*, |J| h*
            contrib = R.w[t] * np.einsum("dmj,sdjv->smv", R.S, Fstar, optimize=True)
            np.add.at(rhs[:, t], cd.A, contrib)             # sum_k A_k^T (.)
        Y = (cd.Minv @ (F0u - rhs).reshape(len(cd.nodes), -1)).reshape(q.shape)   # (M_i^-1 (x) 1)
        qn = np.einsum("st,ntv->nsv", R.K1t_inv, Y)                               # (1 (x) K1t^-1)
        res = np.max(np.abs(qn - q))
        scale = max(1.0, float(np.max(np.abs(q))))
        q = qn
        if res <= prm.picard_tol * scale:
            break
    return q, it


def time_integrate(mesh: OracleMesh, i, q, dt, mu, kappa, prm):
    """Eq. TAvectors: q_bar = dt sum_t w_t q_t (nodal) and F_bar = dt sum_t w_t F(q_t) per sub-tet node."""
    R = mesh.R
    qbar = dt * np.einsum("t,ntv->nv", R.w, q)
    Fbar = sum(dt * R.w[t] * subtet_fluxes(mesh, i, q[:, t], mu, kappa, prm) for t in range(R.Nt))
    return qbar, Fbar


def volume_term(mesh: OracleMesh, i, Fbar):
    """sum_k |J_ik| (V_xi f_bar + V_eta g_bar + V_zeta h_bar) = int_{P_i} grad phi_m . F_bar.

    V_d = S^_d^T (V_d[m, j] = int d_d phi_m phi_j); the transformed flux of sub-tet k is
    adj(J_ik) F_bar (Sec. 4.4).
    """
    cd = mesh.cells[i]
    R = mesh.R
    vol = np.zeros((len(cd.nodes), 5))
    Fs = np.einsum("sde,sjev->sdjv", cd.adj, Fbar, optimize=True)
    contrib = np.einsum("djm,sdjv->smv", R.S, Fs, optimize=True)            # S^_d[j, m] = V_d[m, j]
    np.add.at(vol, cd.A, contrib)
    return vol


def rusanov(qm, Fm, qp, Fp, normal, s, lam_v, h_m, h_p, N):
    """Eq. 3.33 at the face nodes: 1/2 (F+ + F-) . n - 1/2 (|lambda| + 2 eps |lambda^v|) (q+ - q-),
    eps = (2N+1) / ((h+ + h-) sqrt(pi/2)); '-' is the cell's own side, n its outward normal."""
    eps = (2 * N + 1) / ((h_m + h_p) * math.sqrt(math.pi / 2.0))
    Fn = 0.5 * np.einsum("jev,e->jv", Fp + Fm, normal)
    return Fn - 0.5 * (s + 2.0 * eps * lam_v) * (qp - qm)


def face_term(mesh: OracleMesh, i, Gs):
    """sum over cell-boundary sub-triangles of |dP_ik| Z G_k: the boundary integral of
    phi_m times the nodal interpolant of G, with the physical face mass 2 * area * Z^."""
    cd = mesh.cells[i]
    face = np.zeros((len(cd.nodes), 5))
    for bt, G in zip(cd.bfaces, Gs):
        face[bt.nodes] += 2.0 * bt.area * (mesh.R.Z @ G)
    return face


# ---------------------------------------------------------------------------


@dataclass
class StepInfo:
    dt: float
    iterations: np.ndarray
    beta: np.ndarray
    mu: np.ndarray


def step(mesh: OracleMesh, u_cells, prm: Params, dt=None, cells=None):
    """One ADER-AFE-DG step.  ``cells`` restricts the corrector to a subset (the
    predictor then runs on the subset and its face neighbours only)."""
    C = mesh.n_cells
    N = mesh.N
    R = mesh.R
    if prm.limiter:
        beta, mu_c = limiter(mesh, u_cells, prm)
    else:
        beta, mu_c = np.zeros(C), np.full(C, prm.mu)
    kap = np.array([cell_kappa(m, prm) for m in mu_c])
    if dt is None:
        dt = cfl_dt(mesh, u_cells, mu_c, prm)
    out_cells = list(range(C)) if cells is None else list(cells)
    need = set(out_cells)
    for i in out_cells:
        for bt in mesh.cells[i].bfaces:
            if bt.nbr >= 0:
                need.add(bt.nbr)
    iters = np.zeros(C, np.int64)
    pred = {}
    for i in sorted(need):
        q, it = predictor(mesh, i, u_cells[i], dt, mu_c[i], kap[i], prm)
        iters[i] = it
        pred[i] = time_integrate(mesh, i, q, dt, mu_c[i], kap[i], prm)

    new = [u.copy() for u in u_cells]
    for i in out_cells:
        qbar_i, Fbar_i = pred[i]

        def outer(bt, i=i):
            nb = mesh.cells[bt.nbr].bfaces[bt.nbr_tri]
            qbar_j, Fbar_j = pred[bt.nbr]
            return (qbar_j[nb.nodes], Fbar_j[nb.k][nb.local], cell_length(mesh.cells[bt.nbr], prm), mu_c[bt.nbr],
                    kap[bt.nbr])

        new[i] = corrector_cell(mesh, i, u_cells[i], qbar_i, Fbar_i, outer, dt, mu_c[i], kap[i], prm)
    return new, StepInfo(dt=dt, iterations=iters, beta=beta, mu=mu_c)


def corrector_cell(mesh: OracleMesh, i, u_i, qbar_i, Fbar_i, outer, dt, mu_i, kap_i, prm: Params):
    """u_i^{n+1} of cell i (Sec. 4.4): the volume term, Rusanov fluxes on every boundary
    sub-triangle with the wave speeds maximised over each polygonal face and both sides, the
    face term and the M_i^-1 update.  ``outer(bt)`` gives, for a sub-triangle with a
    neighbour, the neighbour side's (q_bar at the face nodes, F_bar at them, h, mu, kappa) in
    the sub-triangle's face-node order."""
    cd = mesh.cells[i]
    N = mesh.N
    vol = volume_term(mesh, i, Fbar_i)
    # per-node states on both sides of every boundary sub-triangle
    sides = []
    for bt in cd.bfaces:
        qm = qbar_i[bt.nodes]
        Fm = Fbar_i[bt.k][bt.local]
        if bt.nbr >= 0:
            qp, Fp, hp, mup, kp = outer(bt)
        else:  # transmissive boundary: outer state = inner state
            qp, Fp, hp, mup, kp = qm, Fm, cell_length(cd, prm), mu_i, kap_i
        sides.append((qm, Fm, qp, Fp, hp, mup, kp))
    # wave speeds: max over all nodes of the polyhedral face, both sides (Eq. 3.33)
    smax: dict = {}
    vmax: dict = {}
    for bt, (qm, Fm, qp, Fp, hp, mup, kp) in zip(cd.bfaces, sides):
        sm = 0.0
        sv = 0.0
        for qq, mm, kk in ((qm / dt, mu_i, kap_i), (qp / dt, mup, kp)):
            rho, v, p = primitives(qq, prm.gamma)
            sm = max(sm, float(np.max(np.abs(v @ bt.normal) + sound_speed(rho, p, prm.gamma))))
            sv = max(sv, float(np.max(viscous_eigen(rho, mm, kk, prm))))
        smax[bt.group] = max(smax.get(bt.group, 0.0), sm)
        vmax[bt.group] = max(vmax.get(bt.group, 0.0), sv)
    Gs = []
    for bt, (qm, Fm, qp, Fp, hp, mup, kp) in zip(cd.bfaces, sides):
        Gs.append(rusanov(qm, Fm, qp, Fp, bt.normal, smax[bt.group], vmax[bt.group], cell_length(cd, prm), hp, N))
    face = face_term(mesh, i, Gs)
    return u_i + cd.Minv @ (vol - face)


def conserved_totals(mesh: OracleMesh, u_cells):
    """sum_i 1^T M_i u_i: the integral of each conserved variable over the domain."""
    return sum(c.wvec @ u for c, u in zip(mesh.cells, u_cells))


# ---------------------------------------------------------------------------
# error norm (Sec. 5.1): L_p norms of rho_h - rho_e integrated over the cells


def tet_rule(n):
    """Collapsed-coordinate Gauss rule with n^3 points on the reference tet (weights sum to 1/6)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    a, b, c = np.meshgrid(x, x, x, indexing="ij")
    wa, wb, wc = np.meshgrid(w, w, w, indexing="ij")
    xi = np.stack([a, b * (1 - a), c * (1 - a) * (1 - b)], -1).reshape(-1, 3)
    return xi, (wa * wb * wc * (1 - a) ** 2 * (1 - b)).ravel()


def error_norms(mesh: OracleMesh, u_cells, exact, var=0):
    """(L1, L2) of u_h[var] - exact(x)[var] by an (N+3)^3-point rule on every sub-tet."""
    R = mesh.R
    xi, wq = tet_rule(mesh.N + 3)
    phi = R.eval_phi(xi)                                     # [q, Np]
    e1 = 0.0
    e2 = 0.0
    for cd, u in zip(mesh.cells, u_cells):
        for k in range(len(cd.A)):
            X = cd.X[k]
            J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
            x = X[0] + xi @ J.T
            uh = phi @ u[cd.A[k], var]
            err = uh - exact(x)[:, var]
            e1 += cd.det[k] * np.sum(wq * np.abs(err))
            e2 += cd.det[k] * np.sum(wq * err * err)
    return e1, math.sqrt(e2)
