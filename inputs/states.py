"""Seeded synthetic initial data, evaluated pointwise at given positions.

Each function maps positions ``x`` [n, 3] to conserved variables
``(rho, rho*u, rho*v, rho*w, rho*E)`` [n, 5] through the ideal-gas relation
``rho*E = p/(gamma-1) + rho*|v|^2/2`` (Sec. 2).  These are the problem
definitions of the workloads; they hold none of the scheme's arithmetic.
Both the oracle and the CUDA path are initialised from the same values:
nodal interpolation at the cell nodes.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


def primitive_to_conserved(rho, vel, p, gamma=GAMMA):
    rho = np.asarray(rho, np.float64)
    vel = np.asarray(vel, np.float64)
    p = np.asarray(p, np.float64)
    out = np.empty(rho.shape + (5,), np.float64)
    out[..., 0] = rho
    out[..., 1:4] = rho[..., None] * vel
    out[..., 4] = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return out


def conserved_to_primitive(q, gamma=GAMMA):
    rho = q[..., 0]
    vel = q[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (q[..., 4] - 0.5 * rho * np.sum(vel * vel, axis=-1))
    return rho, vel, p


def constant(x, rho=1.0, vel=(0.3, -0.2, 0.1), p=1.0, gamma=GAMMA):
    n = len(x)
    return primitive_to_conserved(np.full(n, rho), np.tile(np.asarray(vel, np.float64), (n, 1)),
                                  np.full(n, p), gamma)


def density_wave(x, t=0.0, amp=0.2, vel=(1.0, 1.0, 1.0), p=1.0, gamma=GAMMA):
    """rho = 1 + amp*sin(2*pi*(x+y+z - (u+v+w) t)), uniform velocity and pressure."""
    vel = np.asarray(vel, np.float64)
    xs = np.asarray(x, np.float64) - vel * t
    rho = 1.0 + amp * np.sin(2.0 * math.pi * xs.sum(axis=1))
    n = len(rho)
    return primitive_to_conserved(rho, np.tile(vel, (n, 1)), np.full(n, p), gamma)


def spherical_riemann(x, centre=(0.0, 0.0, 0.0), radius=0.5, rho_in=1.0, rho_out=0.125,
                      p_in=1.0, p_out=0.1, alpha0=None, gamma=GAMMA):
    """Spherical explosion data (Sec. 5.4); with ``alpha0`` the erf-smoothed form.

    The smoothed form is P = (P_out+P_in)/2 + (P_out-P_in)/2 * erf((r-R)/alpha0),
    which tends to P_in inside and P_out outside.
    """
    from scipy.special import erf

    r = np.linalg.norm(np.asarray(x, np.float64) - np.asarray(centre, np.float64), axis=1)
    if alpha0 is None:
        inside = r < radius
        rho = np.where(inside, rho_in, rho_out)
        p = np.where(inside, p_in, p_out)
    else:
        s = erf((r - radius) / alpha0)
        rho = 0.5 * (rho_out + rho_in) + 0.5 * (rho_out - rho_in) * s
        p = 0.5 * (p_out + p_in) + 0.5 * (p_out - p_in) * s
    return primitive_to_conserved(rho, np.zeros((len(r), 3)), p, gamma)


def taylor_green_3d(x, p0=100.0, gamma=GAMMA):
    """u = sin x cos y cos z, v = -cos x sin y cos z, w = 0, rho = 1,
    p = p0 + (cos 2x + cos 2y)(cos 2z + 2)/16."""
    X, Y, Z = np.asarray(x, np.float64).T
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    return primitive_to_conserved(np.ones_like(u), np.stack([u, v, w], 1), p, gamma)


def shear_layers(x, nu, t=0.0, v_in=0.1, v_out=-0.1, t0=0.05, gamma=GAMMA):
    """Periodic form of the first problem of Stokes (Sec. 5, viscous tests): rho = 1,
    p = 1/gamma, u = w = 0 and the shear velocity v(x) = v_in on 1/4 < x < 3/4, v_out outside,
    each jump diffused as an error function of width 2 sqrt(nu (t + t0)).  Exact for the
    linearised (incompressible) shear flow while the two layers do not overlap, i.e. for
    sqrt(nu (t + t0)) well below 1/4; ``t`` gives the closed form at a later time."""
    X = np.asarray(x, np.float64)[:, 0] % 1.0
    s = 2.0 * math.sqrt(nu * (t + t0))
    from scipy.special import erf
    # rises from v_out to v_in at x = 1/4, falls back at x = 3/4
    v = v_out + 0.5 * (v_in - v_out) * (erf((X - 0.25) / s) - erf((X - 0.75) / s))
    n = len(v)
    vel = np.zeros((n, 3))
    vel[:, 1] = v
    return primitive_to_conserved(np.ones(n), vel, np.full(n, 1.0 / gamma), gamma)


def isentropic_vortex(x, t=0.0, eps=5.0, centre=(5.0, 5.0), vel=(0.0, 0.0, 0.0), period=10.0, gamma=GAMMA):
    """Two-dimensional isentropic vortex (Sec. 5.1, steady and travelling forms) on the
    periodic box [0, period)^3: background rho = p = 1 and velocity ``vel``; around the axis
    through ``centre`` + vel t (parallel to z; the periodic image nearest to each point)
    the temperature drops by dT = -(gamma-1) eps^2 / (8 gamma pi^2) exp(1 - r^2), with
    rho = (1 + dT)^(1/(gamma-1)), p = (1 + dT)^(gamma/(gamma-1)), and the swirl
    (du, dv) = eps / (2 pi) exp((1 - r^2) / 2) (-(y - y_c), x - x_c).  The swirl exponent is
    read as (1 - r^2)/2 (the printed (1 - gamma^2)/2 does not depend on r).  The state is an
    exact steady solution of the Euler equations in the vortex's frame; the periodic
    images it ignores differ from it by O(exp(-(period/2)^2 / 2)) at the box faces."""
    X = np.asarray(x, np.float64)
    c = np.asarray(centre, np.float64) + t * np.asarray(vel[:2], np.float64)
    d = X[:, :2] - c
    d -= period * np.round(d / period)
    r2 = np.sum(d * d, axis=1)
    dT = -(gamma - 1.0) * eps ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    p = (1.0 + dT) ** (gamma / (gamma - 1.0))
    s = eps / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    v = np.tile(np.asarray(vel, np.float64), (len(X), 1))
    v[:, 0] -= s * d[:, 1]
    v[:, 1] += s * d[:, 0]
    return primitive_to_conserved(rho, v, p, gamma)
