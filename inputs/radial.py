"""One-dimensional reference solutions for the spherical explosion (Sec. 5.4).

The explosion is radially symmetric, so its solution is that of the Euler equations in the
radial coordinate alone; the paper compares its three-dimensional result with such a
solution computed by a second-order MUSCL scheme with the Rusanov flux on 15,000 points of
r in [0, 1].  This module provides that reference and the exact planar Riemann solution
that pins it.  It is problem data (like the closed forms of ``inputs.states``): none of
the ADER-AFE scheme's arithmetic is here.

* ``exact_riemann``: the exact self-similar solution of the planar Riemann problem for an
  ideal gas: the star pressure is the root of the sum of the two wave curves (shock branch
  from the Rankine-Hugoniot conditions, rarefaction branch from the isentropic relations),
  found by Newton's method; the solution at x/t is sampled from the resulting wave pattern
  (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, Ch. 4).
* ``radial_muscl``: finite volumes in the radial coordinate with geometry exponent
  alpha (2 spherical, 1 cylindrical, 0 planar): cell volumes and face areas of the
  radial shells, minmod-limited linear reconstruction of the primitive variables, the
  Rusanov flux, the pressure-area term of the momentum equation evaluated with the cell
  pressure (so a gas at rest stays at rest exactly), a mirror cell at r = 0 and a
  transmissive outer boundary, and Heun's second-order Runge-Kutta method in time.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


# ---------------------------------------------------------------------------
# exact planar Riemann solution


def _wave_curve(p, rho_k, p_k, gamma):
    """Velocity change across the wave of one side to reach pressure p, and its derivative."""
    c_k = math.sqrt(gamma * p_k / rho_k)
    if p > p_k:  # shock: Rankine-Hugoniot
        a = 2.0 / ((gamma + 1.0) * rho_k)
        b = (gamma - 1.0) / (gamma + 1.0) * p_k
        q = math.sqrt(a / (p + b))
        return (p - p_k) * q, q * (1.0 - 0.5 * (p - p_k) / (p + b))
    # rarefaction: isentropic expansion
    e = (gamma - 1.0) / (2.0 * gamma)
    f = 2.0 * c_k / (gamma - 1.0) * ((p / p_k) ** e - 1.0)
    return f, (p / p_k) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho_k * c_k)


def star_state(left, right, gamma=GAMMA, tol=1e-14, maxit=100):
    """(p*, u*) of the planar Riemann problem with primitive states (rho, u, p) left/right."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    if 2.0 * (cl + cr) / (gamma - 1.0) <= ur - ul:
        raise ValueError("the data generate vacuum")
    p = max(1e-12, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))  # linearised guess
    for _ in range(maxit):
        fl, dl = _wave_curve(p, rl, pl, gamma)
        fr, dr = _wave_curve(p, rr, pr, gamma)
        step = (fl + fr + ur - ul) / (dl + dr)
        p_new = max(1e-12, p - step)
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _wave_curve(p, rl, pl, gamma)
    fr, _ = _wave_curve(p, rr, pr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def exact_riemann(xi, left, right, gamma=GAMMA):
    """Primitive variables (rho, u, p) [len(xi), 3] of the exact solution at x/t = xi."""
    ps, us = star_state(left, right, gamma)
    out = np.empty((len(xi), 3))
    g1, g2 = (gamma - 1.0) / (gamma + 1.0), 2.0 / (gamma + 1.0)
    for n, s in enumerate(np.asarray(xi, np.float64)):
        # work on the left side; the right side is its mirror image
        if s <= us:
            rho_k, u_k, p_k, sgn, x = left[0], left[1], left[2], 1.0, s
        else:
            rho_k, u_k, p_k, sgn, x = right[0], -right[1], right[2], -1.0, -s
        u_star = sgn * us
        c_k = math.sqrt(gamma * p_k / rho_k)
        if ps > p_k:  # shock moving into the k state
            shock = u_k - c_k * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / p_k + (gamma - 1.0) / (2.0 * gamma))
            if x <= shock:
                w = (rho_k, u_k, p_k)
            else:
                w = (rho_k * (ps / p_k + g1) / (g1 * ps / p_k + 1.0), u_star, ps)
        else:  # rarefaction fan between head and tail
            c_star = c_k * (ps / p_k) ** ((gamma - 1.0) / (2.0 * gamma))
            head, tail = u_k - c_k, u_star - c_star
            if x <= head:
                w = (rho_k, u_k, p_k)
            elif x >= tail:
                w = (rho_k * (ps / p_k) ** (1.0 / gamma), u_star, ps)
            else:
                c = g2 * (c_k + 0.5 * (gamma - 1.0) * (u_k - x))
                u = g2 * (c_k + 0.5 * (gamma - 1.0) * u_k + x)
                rho = rho_k * (c / c_k) ** (2.0 / (gamma - 1.0))
                w = (rho, u, p_k * (c / c_k) ** (2.0 * gamma / (gamma - 1.0)))
        out[n] = (w[0], sgn * w[1], w[2])
    return out


# ---------------------------------------------------------------------------
# radial MUSCL finite volumes


def _minmod(a, b):
    return np.where(a * b > 0.0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def _cons(w, gamma):
    rho, u, p = w[..., 0], w[..., 1], w[..., 2]
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u], axis=-1)


def _prim(U, gamma):
    rho = U[..., 0]
    u = U[..., 1] / rho
    return np.stack([rho, u, (gamma - 1.0) * (U[..., 2] - 0.5 * rho * u * u)], axis=-1)


def _flux(w, gamma):
    rho, u, p = w[..., 0], w[..., 1], w[..., 2]
    E = p / (gamma - 1.0) + 0.5 * rho * u * u
    return np.stack([rho * u, rho * u * u + p, u * (E + p)], axis=-1)


class RadialGrid:
    """n cells of [0, R]: centres r, faces rf, shell volumes V and face areas A (per unit
    solid angle), with geometry exponent alpha."""

    def __init__(self, n, R=1.0, alpha=2):
        self.n, self.R, self.alpha = n, R, alpha
        self.rf = np.linspace(0.0, R, n + 1)
        self.r = 0.5 * (self.rf[1:] + self.rf[:-1])
        self.V = (self.rf[1:] ** (alpha + 1) - self.rf[:-1] ** (alpha + 1)) / (alpha + 1)
        self.A = self.rf ** alpha


def _rhs(U, g: RadialGrid, gamma):
    w = _prim(U, gamma)
    # two ghost cells per side: mirror at r = 0, copies at r = R
    wl = w[1::-1].copy()
    wl[:, 1] *= -1.0
    wg = np.concatenate([wl, w, w[-1:], w[-1:]])
    d = _minmod(wg[1:-1] - wg[:-2], wg[2:] - wg[1:-1])        # slopes of cells -1 .. n
    left = wg[1:-2] + 0.5 * d[:-1]                             # face i - 1/2: from cell i - 1
    right = wg[2:-1] - 0.5 * d[1:]                             # face i - 1/2: from cell i
    cl = np.sqrt(gamma * left[:, 2] / left[:, 0])
    cr = np.sqrt(gamma * right[:, 2] / right[:, 0])
    s = np.maximum(np.abs(left[:, 1]) + cl, np.abs(right[:, 1]) + cr)
    F = 0.5 * (_flux(left, gamma) + _flux(right, gamma)) - 0.5 * s[:, None] * (_cons(right, gamma) - _cons(left, gamma))
    AF = g.A[:, None] * F                                      # faces 0 .. n
    out = -(AF[1:] - AF[:-1]) / g.V[:, None]
    out[:, 1] += w[:, 2] * (g.A[1:] - g.A[:-1]) / g.V          # pressure on the shell's side walls
    return out, float(np.max(np.abs(w[:, 1]) + np.sqrt(gamma * w[:, 2] / w[:, 0])))


def radial_muscl(w0, t_end, R=1.0, alpha=2, cfl=0.4, gamma=GAMMA):
    """Advance primitive cell values w0 [n, 3] (rho, u, p) at the centres of n equal cells of
    [0, R] to t_end; returns (grid, w [n, 3], steps)."""
    w0 = np.asarray(w0, np.float64)
    g = RadialGrid(len(w0), R, alpha)
    U = _cons(w0, gamma)
    dx = R / len(w0)
    t, steps = 0.0, 0
    while t < t_end:
        k1, smax = _rhs(U, g, gamma)
        dt = min(cfl * dx / smax, t_end - t)
        U1 = U + dt * k1
        k2, _ = _rhs(U1, g, gamma)
        U = 0.5 * (U + U1 + dt * k2)
        t += dt
        steps += 1
        if not np.all(np.isfinite(U)):
            raise FloatingPointError("non-finite state in the radial reference")
    return g, _prim(U, gamma), steps


def explosion_reference(t_end=0.25, n=15000, R=1.0, radius=0.5, rho_in=1.0, rho_out=0.125, p_in=1.0,
                        p_out=0.1, alpha0=None, gamma=GAMMA):
    """Radial reference of the spherical explosion at t_end: (r [n], (rho, u, p) [n, 3]).
    ``alpha0`` smooths the initial jump as ``inputs.states.spherical_riemann`` does."""
    g = RadialGrid(n, R, 2)
    if alpha0 is None:
        inside = g.r < radius
        rho = np.where(inside, rho_in, rho_out)
        p = np.where(inside, p_in, p_out)
    else:
        from scipy.special import erf
        s = erf((g.r - radius) / alpha0)
        rho = 0.5 * (rho_out + rho_in) + 0.5 * (rho_out - rho_in) * s
        p = 0.5 * (p_out + p_in) + 0.5 * (p_out - p_in) * s
    w0 = np.stack([rho, np.zeros(n), p], axis=1)
    g, w, _ = radial_muscl(w0, t_end, R, 2, gamma=gamma)
    return g.r, w
