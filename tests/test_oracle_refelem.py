"""Pins of the oracle's reference-element algebra against what App. A and the mathematics fix.

Each check is independent of the oracle's own construction: the printed App. A
node sets and basis formulas (tests/golden), closed-form integrals, brute-force
collapsed-coordinate Gauss quadrature, integration by parts, and Gauss-Legendre
exactness.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.refelem import p_eval, ref_element

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_nodes():
    out = {}
    for line in open(os.path.join(GOLDEN, "appendix_a_nodes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        deg, idx, *xyz = line.split()
        out.setdefault(int(deg), {})[int(idx)] = tuple(Fraction(v) for v in xyz)
    return out


def _read_basis():
    out = {}
    for line in open(os.path.join(GOLDEN, "appendix_a_basis.txt")):
        if line.startswith("#") or not line.strip():
            continue
        deg, idx, expr = line.split(None, 2)
        out.setdefault(int(deg), {})[int(idx)] = expr.strip()
    return out


def _eval_printed(expr, x):
    r, s, t = x
    env = {"l1": 1 - r - s - t, "l2": r, "l3": s, "l4": t, "F": Fraction, "__builtins__": {}}
    return eval(expr, env)  # noqa: S307 - committed fixture, restricted namespace


def _tet_quadrature(n):
    """Collapsed-coordinate (Duffy) Gauss rule on the reference tet: points [m,3], weights [m]."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1)
    w = 0.5 * w
    a, b, c = np.meshgrid(x, x, x, indexing="ij")
    wa, wb, wc = np.meshgrid(w, w, w, indexing="ij")
    r = a
    s = b * (1 - a)
    t = c * (1 - a) * (1 - b)
    jac = (1 - a) ** 2 * (1 - b)
    return np.stack([r, s, t], -1).reshape(-1, 3), (wa * wb * wc * jac).ravel()


def _tri_quadrature(n):
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1)
    w = 0.5 * w
    a, b = np.meshgrid(x, x, indexing="ij")
    wa, wb = np.meshgrid(w, w, indexing="ij")
    return np.stack([a, b * (1 - a)], -1).reshape(-1, 2), (wa * wb * (1 - a)).ravel()


@pytest.mark.parametrize("N", [1, 2, 3])
def test_node_set_matches_appendix(N):
    printed = set(_read_nodes()[N].values())
    R = ref_element(N)
    assert len(R.nodes_exact) == (N + 1) * (N + 2) * (N + 3) // 6
    assert set(R.nodes_exact) == printed


def test_p4_lattice_counts():
    """App. A.4: 35 equispaced nodes; 4 vertices, 18 edge nodes, 12 face nodes, 1 interior
    (the printed text swaps the edge and face counts)."""
    R = ref_element(4)
    assert R.Np == 35
    kinds = {0: 0, 1: 0, 2: 0, 3: 0}
    for al in R.bary:
        kinds[sum(1 for a in al if a == 0)] += 1
    # zeros in the multi-index: 3 -> vertex, 2 -> edge, 1 -> face, 0 -> interior
    assert (kinds[3], kinds[2], kinds[1], kinds[0]) == (4, 18, 12, 1)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_nodal_property_and_partition_of_unity(N):
    R = ref_element(N)
    for j, p in enumerate(R.phi):
        for m, x in enumerate(R.nodes_exact):
            assert p_eval(p, x) == (1 if j == m else 0)
    tot = {}
    for p in R.phi:
        for k, v in p.items():
            tot[k] = tot.get(k, 0) + v
    assert {k: v for k, v in tot.items() if v != 0} == {(0, 0, 0): 1}


@pytest.mark.parametrize("N", [1, 2, 3])
def test_printed_basis_functions(N):
    """Every App. A formula is one of the oracle's basis functions (equal at the nodes and at
    random rational points).  For P1 and P2 the printed numbering of functions and nodes
    agrees; for P3 it does not (e.g. the printed phi_7 peaks at (0, 1/3, 0), not at x_7), so
    each printed function is matched to the node where it equals one."""
    nodes = _read_nodes()[N]
    basis = _read_basis()[N]
    R = ref_element(N)
    rng = np.random.default_rng(7)
    pts = [tuple(Fraction(int(v), 97) for v in rng.integers(0, 30, 3)) for _ in range(12)]
    mismatched = []
    for idx, expr in basis.items():
        vals = [_eval_printed(expr, x) for x in R.nodes_exact]
        ones = [j for j, v in enumerate(vals) if v == 1]
        assert len(ones) == 1 and all(v == 0 for j, v in enumerate(vals) if j != ones[0])
        j = ones[0]
        for x in pts:
            assert _eval_printed(expr, x) == p_eval(R.phi[j], x)
        if R.nodes_exact[j] != nodes[idx]:
            mismatched.append(idx)
    if N < 3:
        assert mismatched == []
    else:
        assert 7 in mismatched and len(mismatched) > 0


@pytest.mark.parametrize("N", [1, 2, 3])
def test_universal_matrices_closed_forms(N):
    R = ref_element(N)
    assert sum(sum(row) for row in R.M_exact) == Fraction(1, 6)  # int phi_m phi_l summed = |T^|
    for d in range(3):
        for m in range(R.Np):
            assert sum(R.S_exact[d][m]) == 0  # d_d of sum_l phi_l = d_d 1 = 0
    if N == 1:
        for m in range(4):
            for l in range(4):
                assert R.M_exact[m][l] == Fraction(1 + (m == l), 120)
        for a in range(3):
            for b in range(3):
                assert R.Z_exact[a][b] == Fraction(1 + (a == b), 24)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_universal_matrices_against_quadrature(N):
    R = ref_element(N)
    xq, wq = _tet_quadrature(N + 4)
    phi = R.eval_phi(xq)                       # [q, Np]
    dphi = R.eval_dphi(xq)                     # [q, 3, Np]
    M = np.einsum("q,qm,ql->ml", wq, phi, phi)
    S = np.einsum("q,qm,qdl->dml", wq, phi, dphi)
    np.testing.assert_allclose(R.M, M, atol=1e-15)
    np.testing.assert_allclose(R.S, S, atol=1e-15)
    # D^_d[j, l] = d_d phi_l at node j
    np.testing.assert_allclose(R.D, np.transpose(R.eval_dphi(R.nodes), (1, 0, 2)), atol=1e-13)
    # face mass on the unit right triangle by quadrature of the restricted tet basis (face t = 0)
    uq, wt = _tri_quadrature(N + 3)
    ph = R.eval_phi(np.c_[uq, np.zeros(len(uq))])
    o = 3
    fn = R.face_nodes[o]
    Zq = np.einsum("q,qa,qb->ab", wt, ph[:, fn], ph[:, fn])
    idx = [R.tri_index(tuple(al[m] for m in range(4) if m != o)) for al in (R.bary[j] for j in fn)]
    np.testing.assert_allclose(R.Z[np.ix_(idx, idx)], Zq, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_integration_by_parts_pins_stiffness_to_face_mass(N):
    """S^_d + S^_d^T = sum over the four faces of n_d * (2 area) * Z^ on that face."""
    R = ref_element(N)
    normals = {0: np.ones(3) / math.sqrt(3), 1: -np.eye(3)[0], 2: -np.eye(3)[1], 3: -np.eye(3)[2]}
    areas = {0: math.sqrt(3) / 2, 1: 0.5, 2: 0.5, 3: 0.5}
    rhs = np.zeros((3, R.Np, R.Np))
    for o in range(4):
        fn = R.face_nodes[o]
        idx = [R.tri_index(tuple(R.bary[j][m] for m in range(4) if m != o)) for j in fn]
        Zf = 2 * areas[o] * R.Z[np.ix_(idx, idx)]
        for d in range(3):
            rhs[d][np.ix_(fn, fn)] += normals[o][d] * Zf
    np.testing.assert_allclose(R.S + np.transpose(R.S, (0, 2, 1)), rhs, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_time_basis(N):
    R = ref_element(N)
    assert abs(R.w.sum() - 1) < 1e-15
    for k in range(2 * N + 2):   # N+1 Gauss points are exact to degree 2N+1
        assert abs(np.sum(R.w * R.tau ** k) - 1.0 / (k + 1)) < 1e-15
    for s in range(R.Nt):
        for r in range(R.Nt):
            assert abs(R.psi(s, R.tau[r]) - (s == r)) < 1e-14
    np.testing.assert_allclose(R.K1t @ np.ones(R.Nt), R.psi0, atol=1e-13)
    np.testing.assert_allclose(R.K1t_inv @ R.psi0, np.ones(R.Nt), atol=1e-12)
    # K1t from its definition, with a 12-point rule for int psi_s' psi_t
    x, w = np.polynomial.legendre.leggauss(12)
    x = 0.5 * (x + 1)
    w = 0.5 * w
    K = np.empty((R.Nt, R.Nt))
    for s in range(R.Nt):
        for t in range(R.Nt):
            ds = np.array([R.dpsi_at(s, xx) for xx in x])
            pt = np.array([R.psi(t, xx) for xx in x])
            K[s, t] = R.psi(s, 1.0) * R.psi(t, 1.0) - np.sum(w * ds * pt)
    np.testing.assert_allclose(R.K1t, K, atol=1e-13)
    # derivative of psi_s against a central difference
    for s in range(R.Nt):
        fd = (R.psi(s, 0.3 + 1e-6) - R.psi(s, 0.3 - 1e-6)) / 2e-6
        assert abs(R.dpsi_at(s, 0.3) - fd) < 1e-6
