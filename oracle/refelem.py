"""Reference-element algebra of the AFE scheme, in exact rational arithmetic.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

* Reference tetrahedron T^ = {(r,s,t): r,s,t >= 0, r+s+t <= 1}, barycentric
  coordinates lambda_1 = 1-r-s-t, lambda_2 = r, lambda_3 = s, lambda_4 = t (App. A).
* P_N nodes: the equispaced lattice (r,s,t) = (i,j,k)/N with i+j+k <= N
  (App. A lists them for N = 1..4); the build's own ordering, since the node
  numbering and the basis numbering printed for P3 in App. A disagree.
* Lagrange basis phi_j by the nodal property phi_j(x_m) = delta_jm (Sec. 4.1),
  built as Silvester's product of the barycentric coordinates,
  phi_alpha = prod_m prod_{p < alpha_m} (N*lambda_m - p)/(p+1).
* Universal matrices as exact integrals of polynomials over T^ (Sec. 4.3, 4.4):
  mass M^[m,l] = int phi_m phi_l, stiffness S^_d[m,l] = int phi_m d_d phi_l
  (the spatial factor of K_xi, K_eta, K_zeta), face mass Z^ on the unit right
  triangle, with int_T^ r^a s^b t^c = a! b! c! / (a+b+c+3)!.
* Time basis (Sec. 4.3): Lagrange polynomials psi_t of degree N through the
  N+1 Gauss-Legendre points of [0,1], weights w_t; time-upwind matrix
  K1t[s,t] = psi_s(1) psi_t(1) - int_0^1 psi_s' psi_t dtau (Eq. ADER-localCauchy)
  and the time-integration weights T_tau = int_0^1 psi_t = w_t (Eq. TAvectors).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

# ---------------------------------------------------------------------------
# polynomials in (r, s, t) with rational coefficients: {(a, b, c): Fraction}


def p_add(p, q):
    out = dict(p)
    for k, v in q.items():
        out[k] = out.get(k, Fraction(0)) + v
    return {k: v for k, v in out.items() if v != 0}


def p_mul(p, q):
    out: dict = {}
    for (a1, b1, c1), v1 in p.items():
        for (a2, b2, c2), v2 in q.items():
            k = (a1 + a2, b1 + b2, c1 + c2)
            out[k] = out.get(k, Fraction(0)) + v1 * v2
    return {k: v for k, v in out.items() if v != 0}


def p_scale(p, c):
    return {k: v * c for k, v in p.items() if v * c != 0}


def p_deriv(p, d):
    out: dict = {}
    for k, v in p.items():
        if k[d] == 0:
            continue
        kk = list(k)
        kk[d] -= 1
        out[tuple(kk)] = out.get(tuple(kk), Fraction(0)) + v * k[d]
    return out


def p_eval(p, x):
    """Evaluate at a point; exact if x holds Fractions, float otherwise."""
    acc = 0
    for (a, b, c), v in p.items():
        acc = acc + v * x[0] ** a * x[1] ** b * x[2] ** c
    return acc


def int_tet_monomial(a, b, c):
    """int over T^ of r^a s^b t^c = a! b! c! / (a+b+c+3)!."""
    return Fraction(math.factorial(a) * math.factorial(b) * math.factorial(c),
                    math.factorial(a + b + c + 3))


def int_tri_monomial(a, b):
    """int over the unit right triangle {u,v >= 0, u+v <= 1} of u^a v^b = a! b! / (a+b+2)!."""
    return Fraction(math.factorial(a) * math.factorial(b), math.factorial(a + b + 2))


def p_int_tet(p):
    return sum((v * int_tet_monomial(*k) for k, v in p.items()), Fraction(0))


def p_int_tri(p):
    """p given in (u, v, 0) monomials."""
    return sum((v * int_tri_monomial(k[0], k[1]) for k, v in p.items() if k[2] == 0), Fraction(0))


ONE = {(0, 0, 0): Fraction(1)}
LAMBDA = [
    {(0, 0, 0): Fraction(1), (1, 0, 0): Fraction(-1), (0, 1, 0): Fraction(-1), (0, 0, 1): Fraction(-1)},
    {(1, 0, 0): Fraction(1)},
    {(0, 1, 0): Fraction(1)},
    {(0, 0, 1): Fraction(1)},
]
# barycentric coordinates of the unit right triangle in (u, v): mu_1 = 1-u-v, mu_2 = u, mu_3 = v
MU = [
    {(0, 0, 0): Fraction(1), (1, 0, 0): Fraction(-1), (0, 1, 0): Fraction(-1)},
    {(1, 0, 0): Fraction(1)},
    {(0, 1, 0): Fraction(1)},
]


def tet_lattice(N):
    """Barycentric multi-indices (alpha_1..alpha_4), sum N, of the P_N nodes; order: t, s, r loops."""
    out = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - k - j):
                out.append((N - i - j - k, i, j, k))
    return out


def tri_lattice(N):
    out = []
    for j in range(N + 1):
        for i in range(N + 1 - j):
            out.append((N - i - j, i, j))
    return out


def silvester(alpha, N, bary):
    """Lagrange basis function of the equispaced node with multi-index alpha."""
    p = ONE
    for m, am in enumerate(alpha):
        for q in range(am):
            fac = p_add(p_scale(bary[m], Fraction(N)), {(0, 0, 0): Fraction(-q)})
            p = p_mul(p, p_scale(fac, Fraction(1, q + 1)))
    return p


# ---------------------------------------------------------------------------


class RefElement:
    """All universal (mesh-independent) quantities for polynomial degree N."""

    def __init__(self, N: int):
        if N < 1:
            raise ValueError("N >= 1")
        self.N = N
        self.bary = tet_lattice(N)
        self.Np = len(self.bary)
        assert self.Np == (N + 1) * (N + 2) * (N + 3) // 6  # Sec. 4.1
        self.nodes_exact = [tuple(Fraction(a, N) for a in al[1:]) for al in self.bary]
        self.nodes = np.array([[float(v) for v in x] for x in self.nodes_exact])
        self.phi = [silvester(al, N, LAMBDA) for al in self.bary]
        self.dphi = [[p_deriv(p, d) for p in self.phi] for d in range(3)]

        Np = self.Np
        self.M_exact = [[p_int_tet(p_mul(self.phi[m], self.phi[l])) for l in range(Np)] for m in range(Np)]
        self.S_exact = [[[p_int_tet(p_mul(self.phi[m], self.dphi[d][l])) for l in range(Np)]
                         for m in range(Np)] for d in range(3)]
        self.D_exact = [[[p_eval(self.dphi[d][l], self.nodes_exact[j]) for l in range(Np)]
                         for j in range(Np)] for d in range(3)]
        self.M = np.array(self.M_exact, dtype=np.float64)
        self.S = np.array(self.S_exact, dtype=np.float64)          # [3, Np, Np]
        self.D = np.array(self.D_exact, dtype=np.float64)          # [3, Np, Np]

        # faces of T^: face o is opposite local vertex o; its nodes have alpha_o = 0
        self.face_nodes = []
        for o in range(4):
            self.face_nodes.append([j for j, al in enumerate(self.bary) if al[o] == 0])
        # triangle lattice and face mass on the unit right triangle (area 1/2)
        self.tri_bary = tri_lattice(N)
        self.Nf = len(self.tri_bary)
        tri_phi = [silvester(b, N, MU) for b in self.tri_bary]
        self.Z_exact = [[p_int_tri(p_mul(tri_phi[a], tri_phi[b])) for b in range(self.Nf)]
                        for a in range(self.Nf)]
        self.Z = np.array(self.Z_exact, dtype=np.float64)
        self._tri_index = {b: i for i, b in enumerate(self.tri_bary)}

        # time basis through Gauss-Legendre points on [0, 1]
        x, w = np.polynomial.legendre.leggauss(N + 1)
        self.tau = 0.5 * (x + 1.0)
        self.w = 0.5 * w
        Nt = N + 1
        self.Nt = Nt
        self.psi0 = np.array([self.psi(s, 0.0) for s in range(Nt)])
        self.psi1 = np.array([self.psi(s, 1.0) for s in range(Nt)])
        self.dpsi = np.array([[self.dpsi_at(s, self.tau[r]) for r in range(Nt)] for s in range(Nt)])
        # K1t[s, t] = psi_s(1) psi_t(1) - int psi_s' psi_t; GL with N+1 points is exact for degree 2N-1
        self.K1t = np.outer(self.psi1, self.psi1) - self.dpsi * self.w[None, :]
        self.K1t_inv = np.linalg.inv(self.K1t)

    # -- time basis -------------------------------------------------------
    def psi(self, s, tau):
        v = 1.0
        for r in range(self.N + 1):
            if r != s:
                v *= (tau - self.tau[r]) / (self.tau[s] - self.tau[r])
        return v

    def dpsi_at(self, s, tau):
        tot = 0.0
        for q in range(self.N + 1):
            if q == s:
                continue
            v = 1.0 / (self.tau[s] - self.tau[q])
            for r in range(self.N + 1):
                if r != s and r != q:
                    v *= (tau - self.tau[r]) / (self.tau[s] - self.tau[r])
            tot += v
        return tot

    # -- spatial basis evaluation ------------------------------------------
    def eval_phi(self, xi):
        """phi_j at points xi [n, 3] -> [n, Np] (float)."""
        xi = np.atleast_2d(np.asarray(xi, np.float64))
        out = np.zeros((len(xi), self.Np))
        for j, p in enumerate(self.phi):
            for (a, b, c), v in p.items():
                out[:, j] += float(v) * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c
        return out

    def eval_dphi(self, xi):
        """grad_xi phi_j at points xi [n, 3] -> [n, 3, Np]."""
        xi = np.atleast_2d(np.asarray(xi, np.float64))
        out = np.zeros((len(xi), 3, self.Np))
        for d in range(3):
            for j, p in enumerate(self.dphi[d]):
                for (a, b, c), v in p.items():
                    out[:, d, j] += float(v) * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c
        return out

    def tri_index(self, beta):
        return self._tri_index[tuple(beta)]


@lru_cache(maxsize=None)
def ref_element(N: int) -> RefElement:
    return RefElement(N)
