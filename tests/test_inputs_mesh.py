"""Checks of the seeded synthetic meshes: volumes, conformity, orientation, topology."""
import numpy as np
import pytest

from inputs import voronoi as V


def _subtet_stats(pm):
    X = pm.subtet_coords()
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], -1)
    return np.linalg.det(J)


def _tri_key(pm, t, o):
    vid = pm.subtet_vtx[t]
    sh = np.zeros((4, 3), np.int64) if pm.subtet_shift is None else pm.subtet_shift[t].astype(np.int64)
    ms = [m for m in range(4) if m != o]
    ref = min((int(vid[m]), tuple(sh[m])) for m in ms)
    return tuple(sorted((int(vid[m]), tuple(int(x) for x in sh[m] - np.array(ref[1]))) for m in ms)), ref


@pytest.mark.parametrize("gen,n", [(V.periodic_voronoi, 2), (V.periodic_voronoi, 4), (V.box_voronoi, 3)])
def test_mesh_volumes_and_orientation(gen, n):
    pm = gen(n)
    det = _subtet_stats(pm)
    assert np.all(det > 0)
    vol = det.sum() / 6
    dom = np.prod(pm.hi - pm.lo)
    if pm.periodic:
        assert abs(vol - dom) < 1e-12 * dom
    else:
        # edge collapse may move vertices on the box planes inward slightly
        assert abs(vol - dom) < 5e-3 * dom
    assert pm.n_cells == n ** 3


@pytest.mark.parametrize("gen,n", [(V.periodic_voronoi, 2), (V.periodic_voronoi, 3), (V.box_voronoi, 3)])
def test_mesh_conformity_and_ball_topology(gen, n):
    """Inside a cell every subgrid triangle is shared by <= 2 sub-tets; a cell-boundary
    triangle is matched by exactly one triangle of another cell (or lies on the box); the
    subgrid of each cell has Euler characteristic 1 (a ball)."""
    pm = gen(n)
    glob: dict = {}
    for c in range(pm.n_cells):
        local: dict = {}
        V_, E_, F_ = set(), set(), set()
        for t in range(pm.cell_subtet_ptr[c], pm.cell_subtet_ptr[c + 1]):
            vk = [(int(pm.subtet_vtx[t, m]),
                   (0, 0, 0) if pm.subtet_shift is None else tuple(int(x) for x in pm.subtet_shift[t, m]))
                  for m in range(4)]
            V_.update(vk)
            for a in range(4):
                for b in range(a + 1, 4):
                    E_.add(tuple(sorted((vk[a], vk[b]))))
            for o in range(4):
                tk = tuple(sorted(vk[m] for m in range(4) if m != o))
                F_.add(tk)
                local.setdefault(tk, []).append((t, o))
        ntet = pm.cell_subtet_ptr[c + 1] - pm.cell_subtet_ptr[c]
        assert len(V_) - len(E_) + len(F_) - ntet == 1
        for tk, lst in local.items():
            assert len(lst) <= 2
            if len(lst) == 1:
                key, _ = _tri_key(pm, *lst[0])
                glob.setdefault(key, []).append(c)
    for key, cells in glob.items():
        if pm.periodic:
            assert len(cells) == 2
        else:
            assert len(cells) in (1, 2)


def test_mesh_is_seeded_and_reproducible():
    a = V.periodic_voronoi(3, seed=5)
    b = V.periodic_voronoi(3, seed=5)
    c = V.periodic_voronoi(3, seed=6)
    np.testing.assert_array_equal(a.subtet_vtx, b.subtet_vtx)
    np.testing.assert_array_equal(a.xyz, b.xyz)
    assert a.xyz.shape != c.xyz.shape or not np.array_equal(a.xyz, c.xyz)


def test_collapse_removes_short_edges():
    pm = V.periodic_voronoi(4)
    X = pm.subtet_coords()
    edge = np.linalg.norm(X[:, 3] - X[:, 2], axis=1)
    assert edge.min() >= V.COLLAPSE * 0.25 * 0.999
    raw = V.periodic_voronoi(4, collapse=0.0)
    Xr = raw.subtet_coords()
    assert np.linalg.norm(Xr[:, 3] - Xr[:, 2], axis=1).min() < edge.min()


@pytest.mark.parametrize("n", [8, 12])
def test_quality_step_leaves_no_degenerate_sub_tets(n):
    """After the Lloyd steps and the collapse (with its fold retry) no sub-tet is a needle:
    every edge of the fan is longer than 0.15 lattice spacings and every sub-tet holds at
    least 2 % of its cell's mean sub-tet volume."""
    pm = V.periodic_voronoi(n)
    P = pm.subtet_coords()
    h = 1.0 / n
    edge = np.linalg.norm(P[:, 3] - P[:, 2], axis=1) / h
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6.0
    cell = np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr))
    mean = np.bincount(cell, weights=vol) / np.bincount(cell)
    assert edge.min() > 0.15
    assert (vol / mean[cell]).min() > 0.02


def test_flatness_option_lifts_the_smallest_centre_height():
    """With ``flat`` the generator collapses faces whose fan triangles pass within flat
    spacings of the cell centre: on the 12^3 periodic mesh (smallest height 0.11 spacings
    without it) no fan sub-tet keeps its centre closer than 0.15 spacings to its triangle."""
    def min_height(pm, a):
        X = pm.subtet_coords()
        det = np.abs(np.linalg.det(X[:, 1:] - X[:, :1]))
        tri = 0.5 * np.linalg.norm(np.cross(X[:, 2] - X[:, 1], X[:, 3] - X[:, 1]), axis=1)
        return float((det / (2.0 * tri)).min() / a)

    n = 12
    assert min_height(V.periodic_voronoi(n), 1.0 / n) < 0.15
    pm = V.periodic_voronoi(n, flat=0.15)
    assert min_height(pm, 1.0 / n) >= 0.15
    assert pm.info["flat"] == 0.15
