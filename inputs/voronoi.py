"""Seeded synthetic polyhedral meshes: jittered-lattice Voronoi cells with a fan subgrid.

This module is input generation only.  It builds the polyhedra {P_i} and their
tetrahedral subgrids {T_ik} (Sec. 4.1: each polyhedron is split into conforming
sub-tetrahedra) and returns them in the array form that the C-ABI entry point
``afe_mesh_create`` and the CPU oracle both take.  It contains none of the
scheme's arithmetic (no basis functions, no matrices, no fluxes).

Recipe
------
* Seeds: ``(i + 1/2 + U(-0.3, 0.3)) * L / n`` per coordinate on an ``n^3`` lattice,
  the jitter drawn from ``numpy.random.default_rng(seed)`` as one
  ``uniform(-0.3, 0.3, size=(n, n, n, 3))`` array in C order.
* Periodic cube ``[0, L)^3``: the Voronoi tessellation of the seeds and their
  periodic images; vertices are welded topologically by the set of generating
  seeds (translated to a canonical image), never by a coordinate tolerance.
* Box ``[lo, hi]^3`` (transmissive boundaries): the Voronoi tessellation of the
  seeds and their mirror images across the six box planes, so that every cell
  is the Voronoi cell clipped to the box.
* Fan subgrid: each cell is split by joining its centre (the mean of its
  Voronoi vertices) to a fan triangulation of each face about the face centre
  (the mean of the face's vertices): one sub-tet per face edge.

Array form (matches ``afe_mesh_create``)
----------------------------------------
``xyz`` [n_vertices, 3] float64; ``cell_subtet_ptr`` [n_cells + 1] int64 (CSR);
``subtet_vtx`` [n_subtets, 4] int64 global vertex ids; ``subtet_shift``
[n_subtets, 4, 3] int8 periodic image of each sub-tet vertex (``None`` for the
box); the physical position of a sub-tet vertex is ``xyz[id] + shift * L``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import Voronoi

JITTER = 0.3
# Voronoi edges shorter than COLLAPSE * (lattice spacing) are collapsed
COLLAPSE = 0.2


@dataclass
class PolyMesh:
    xyz: np.ndarray               # [nv, 3] f64
    cell_subtet_ptr: np.ndarray   # [C+1] i64
    subtet_vtx: np.ndarray        # [T, 4] i64
    subtet_shift: np.ndarray | None  # [T, 4, 3] i8
    periodic: bool
    period: tuple                 # (Lx, Ly, Lz); zeros for the box
    lo: np.ndarray                # domain lower corner
    hi: np.ndarray                # domain upper corner
    seeds: np.ndarray             # [C, 3]
    faces_per_cell: np.ndarray    # [C] number of polyhedral faces
    info: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return len(self.cell_subtet_ptr) - 1

    @property
    def n_subtets(self) -> int:
        return len(self.subtet_vtx)

    def subtet_coords(self) -> np.ndarray:
        """[T, 4, 3] physical vertex positions of every sub-tet."""
        X = self.xyz[self.subtet_vtx]
        if self.subtet_shift is not None:
            X = X + self.subtet_shift.astype(np.float64) * np.asarray(self.period)
        return X


def jittered_seeds(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-JITTER, JITTER, size=(n, n, n, 3))
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    return (lo + (idx + 0.5 + jit) * (hi - lo) / n).reshape(-1, 3)


def _order_polygon(pts: np.ndarray, normal: np.ndarray) -> np.ndarray:
    """Indices ordering the vertices of a convex planar polygon counter-clockwise about ``normal``."""
    c = pts.mean(axis=0)
    nrm = normal / np.linalg.norm(normal)
    a = pts[0] - c
    a = a - nrm * (a @ nrm)
    a /= np.linalg.norm(a)
    b = np.cross(nrm, a)
    d = pts - c
    ang = np.arctan2(d @ b, d @ a)
    return np.argsort(ang, kind="stable")


def _fan_subtets(cell_polys, cc_id, fc_ids, out_vtx, out_shift, fc_shifts, positions):
    """Append the fan sub-tets of one cell.

    cell_polys: list of (vertex ids, vertex shifts) per face, ordered CCW seen from outside.
    positions: callable (ids, shifts) -> coords in the cell frame.
    """
    cc_pos = positions(np.array([cc_id]), np.zeros((1, 3), np.int64))[0]
    for f, (vids, vsh) in enumerate(cell_polys):
        m = len(vids)
        fc = fc_ids[f]
        fsh = fc_shifts[f]
        fpos = positions(np.array([fc]), fsh[None])[0]
        vpos = positions(vids, vsh)
        for e in range(m):
            a, b = e, (e + 1) % m
            J = np.stack([fpos - cc_pos, vpos[a] - cc_pos, vpos[b] - cc_pos], axis=1)
            if not np.linalg.det(J) > 0:
                raise RuntimeError("folded fan sub-tet (face polygon not star-shaped about its centre)")
            out_vtx.append((cc_id, fc, vids[a], vids[b]))
            out_shift.append((np.zeros(3, np.int64), fsh, vsh[a], vsh[b]))


def _collapse_short_edges(vpos, cell_polys_all, L, tol):
    """Merge the end points of every Voronoi edge shorter than ``tol``.

    Short Voronoi edges give needle-shaped fan sub-tets, whose tiny support makes
    the cell operators stiff; this plays the role of the quality step of the
    paper's own mesh generator (Sec. 3: admissible control volumes).  Vertices
    are merged topologically (union-find over canonical vertex ids, with the
    periodic image offset of each merge), so every cell sees the same merge.
    Faces left with fewer than three distinct vertices disappear on both sides.
    Returns the new vertex positions and polygons, and the number of merges.
    """
    nv = len(vpos)
    parent = list(range(nv))
    off = [np.zeros(3, np.int64) for _ in range(nv)]
    Lf = 0.0 if L is None else L

    def find(x):
        o = np.zeros(3, np.int64)
        path = []
        while parent[x] != x:
            path.append(x)
            o = o + off[x]
            x = parent[x]
        # path compression
        acc = o.copy()
        for y in path:
            nxt = acc - off[y]
            off[y] = acc
            parent[y] = x
            acc = nxt
        return x, o

    merges = 0
    for polys in cell_polys_all:
        for ids, shs, _ in polys:
            m = len(ids)
            for e in range(m):
                a, b = int(ids[e]), int(ids[(e + 1) % m])
                pa = vpos[a] + shs[e] * Lf
                pb = vpos[b] + shs[(e + 1) % m] * Lf
                if np.linalg.norm(pa - pb) >= tol:
                    continue
                ra, oa = find(a)
                rb, ob = find(b)
                rel = oa + shs[e] - ob - shs[(e + 1) % m]
                if ra == rb:
                    if np.any(rel != 0):
                        raise RuntimeError("short-edge cluster wraps around the period")
                    continue
                parent[rb] = ra
                off[rb] = rel
                merges += 1
    members: dict = {}
    for x in range(nv):
        r, o = find(x)
        members.setdefault(r, []).append(vpos[x] - o * Lf)
    new_id = {r: i for i, r in enumerate(members)}
    new_pos = [np.mean(members[r], axis=0) for r in members]
    out = []
    for polys in cell_polys_all:
        npolys = []
        for ids, shs, b in polys:
            vs = []
            for i, sh in zip(ids, shs):
                r, o = find(int(i))
                vs.append((new_id[r], tuple(int(x) for x in sh + o)))
            ded = [v for k, v in enumerate(vs) if v != vs[k - 1]] if len(set(vs)) > 1 else vs[:1]
            if len(set(ded)) != len(ded):
                raise RuntimeError("pinched face after edge collapse")
            if len(ded) < 3:
                continue
            npolys.append((np.array([v[0] for v in ded], np.int64),
                           np.array([v[1] for v in ded], np.int64), b))
        out.append(npolys)
    return new_pos, out, merges


def periodic_voronoi(n: int, L: float = 1.0, seed: int = 0, collapse: float = COLLAPSE) -> PolyMesh:
    """Periodic jittered-lattice Voronoi mesh of ``[0, L)^3`` with fan subgrids."""
    seeds = jittered_seeds(n, 0.0, L, seed)
    C = n ** 3
    margin = min(2.5 * L / n, L)
    pts, pid, psh = [seeds], [np.arange(C)], [np.zeros((C, 3), np.int64)]
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                if sx == sy == sz == 0:
                    continue
                s = np.array([sx, sy, sz])
                p = seeds + s * L
                keep = np.all((p > -margin) & (p < L + margin), axis=1)
                pts.append(p[keep])
                pid.append(np.nonzero(keep)[0])
                psh.append(np.tile(s, (int(keep.sum()), 1)))
    P = np.concatenate(pts)
    pid = np.concatenate(pid)
    psh = np.concatenate(psh)
    vor = Voronoi(P)

    # generators of every Voronoi vertex (points whose region holds it)
    gens: dict[int, list[int]] = {}
    for p in range(len(P)):
        for v in vor.regions[vor.point_region[p]]:
            if v >= 0:
                gens.setdefault(v, []).append(p)

    def canon(members):
        """Canonical translate of a generator set: (key, shift of the frame)."""
        lab = [(int(pid[p]), tuple(int(x) for x in psh[p])) for p in members]
        ref = min(lab)
        rs = np.array(ref[1])
        key = tuple(sorted((s, tuple(int(x) for x in np.array(sh) - rs)) for s, sh in lab))
        return key, rs

    vkey_id: dict = {}
    vpos: list = []
    vcache: dict[int, tuple[int, np.ndarray]] = {}

    def vertex(v):
        if v in vcache:
            return vcache[v]
        key, rs = canon(gens[v])
        if key not in vkey_id:
            vkey_id[key] = len(vpos)
            vpos.append(vor.vertices[v] - rs * L)
        out = (vkey_id[key], rs)
        vcache[v] = out
        return out

    # ridges of original cells
    ridges_of = [[] for _ in range(C)]
    for r, (a, b) in enumerate(vor.ridge_points):
        if a < C:
            ridges_of[a].append((r, b))
        if b < C:
            ridges_of[b].append((r, a))

    cell_polys_all = []
    for a in range(C):
        polys = []
        for r, b in ridges_of[a]:
            rv = vor.ridge_vertices[r]
            if -1 in rv:
                raise RuntimeError("unbounded ridge next to an original cell; margin too small")
            rv = np.array(rv)
            nrm = P[b] - P[a]
            order = _order_polygon(vor.vertices[rv], nrm)
            rv = rv[order]
            ids, shs = zip(*(vertex(int(v)) for v in rv))
            polys.append((np.array(ids, np.int64), np.array(shs, np.int64), b))
        cell_polys_all.append(polys)
    merges = 0
    if collapse > 0:
        vpos, cell_polys_all, merges = _collapse_short_edges(vpos, cell_polys_all, L, collapse * L / n)
    n_voro = len(vpos)
    xyz_list = list(vpos)

    def positions(ids, shifts):
        return np.array([xyz_list[i] for i in ids]) + np.asarray(shifts, np.float64) * L

    # face centres (canonical per generator pair), then cell centres
    fkey_id: dict = {}
    sub_vtx, sub_sh, ptr, nfaces = [], [], [0], []
    for a in range(C):
        polys = cell_polys_all[a]
        fc_ids, fc_sh = [], []
        for ids, shs, b in polys:
            key, rs = canon([a, b])
            if key not in fkey_id:
                fkey_id[key] = len(xyz_list)
                xyz_list.append(positions(ids, shs).mean(axis=0) - rs * L)
            fc_ids.append(fkey_id[key])
            fc_sh.append(rs)
        allv = {}
        for ids, shs, _ in polys:
            for i, s in zip(ids, shs):
                allv[(int(i), tuple(int(x) for x in s))] = None
        vv = list(allv)
        cc = positions([i for i, _ in vv], [s for _, s in vv]).mean(axis=0)
        cc_id = len(xyz_list)
        xyz_list.append(cc)
        _fan_subtets([(ids, shs) for ids, shs, _ in polys], cc_id, fc_ids, sub_vtx, sub_sh, fc_sh, positions)
        ptr.append(len(sub_vtx))
        nfaces.append(len(polys))

    xyz = np.array(xyz_list, np.float64)
    shift = np.array([[np.asarray(s) for s in row] for row in sub_sh], np.int64)
    if np.abs(shift).max() > 127:
        raise RuntimeError("image shift out of int8 range")
    return PolyMesh(
        xyz=xyz,
        cell_subtet_ptr=np.array(ptr, np.int64),
        subtet_vtx=np.array(sub_vtx, np.int64),
        subtet_shift=shift.astype(np.int8),
        periodic=True,
        period=(L, L, L),
        lo=np.zeros(3),
        hi=np.full(3, L),
        seeds=seeds,
        faces_per_cell=np.array(nfaces, np.int64),
        info={"n_voronoi_vertices": n_voro, "n": n, "L": L, "seed": seed, "collapsed_edges": merges,
              "collapse": collapse},
    )


def box_voronoi(n: int, lo: float = -1.0, hi: float = 1.0, seed: int = 0,
                collapse: float = COLLAPSE) -> PolyMesh:
    """Jittered-lattice Voronoi mesh of the box ``[lo, hi]^3`` with fan subgrids."""
    seeds = jittered_seeds(n, lo, hi, seed)
    C = n ** 3
    h = (hi - lo) / n
    margin = 2.5 * h
    pts = [seeds]
    for d in range(3):
        for plane in (lo, hi):
            near = np.abs(seeds[:, d] - plane) < margin
            q = seeds[near].copy()
            q[:, d] = 2.0 * plane - q[:, d]
            pts.append(q)
    P = np.concatenate(pts)
    vor = Voronoi(P)

    ridges_of = [[] for _ in range(C)]
    for r, (a, b) in enumerate(vor.ridge_points):
        if a < C:
            ridges_of[a].append((r, b))
        if b < C:
            ridges_of[b].append((r, a))

    vmap: dict[int, int] = {}
    xyz_list: list = []

    def vid(v):
        if v not in vmap:
            vmap[v] = len(xyz_list)
            xyz_list.append(vor.vertices[v])
        return vmap[v]

    cell_polys_all = []
    for a in range(C):
        polys = []
        for r, b in ridges_of[a]:
            rv = vor.ridge_vertices[r]
            if -1 in rv:
                raise RuntimeError("unbounded ridge next to an original cell")
            rv = np.array(rv)
            order = _order_polygon(vor.vertices[rv], P[b] - P[a])
            rv = rv[order]
            ids = np.array([vid(int(v)) for v in rv], np.int64)
            polys.append((ids, np.zeros((len(ids), 3), np.int64), b))
        cell_polys_all.append(polys)
    merges = 0
    if collapse > 0:
        xyz_list, cell_polys_all, merges = _collapse_short_edges(xyz_list, cell_polys_all, None, collapse * h)
        xyz_list = list(xyz_list)
    n_voro = len(xyz_list)

    def positions(ids, shifts):
        return np.array([xyz_list[i] for i in ids])

    fkey_id: dict = {}
    sub_vtx, sub_sh, ptr, nfaces = [], [], [0], []
    zero = np.zeros(3, np.int64)
    for a in range(C):
        polys = cell_polys_all[a]
        fc_ids = []
        for ids, _, b in polys:
            key = (min(a, b), max(a, b)) if b < C else (a, -1 - int(b))
            if key not in fkey_id:
                fkey_id[key] = len(xyz_list)
                xyz_list.append(positions(ids, None).mean(axis=0))
            fc_ids.append(fkey_id[key])
        allv = sorted({int(i) for ids, _, _ in polys for i in ids})
        cc_id = len(xyz_list)
        xyz_list.append(positions(allv, None).mean(axis=0))
        _fan_subtets([(ids, z) for ids, z, _ in polys], cc_id, fc_ids, sub_vtx, sub_sh,
                     [zero] * len(polys), positions)
        ptr.append(len(sub_vtx))
        nfaces.append(len(polys))

    return PolyMesh(
        xyz=np.array(xyz_list, np.float64),
        cell_subtet_ptr=np.array(ptr, np.int64),
        subtet_vtx=np.array(sub_vtx, np.int64),
        subtet_shift=None,
        periodic=False,
        period=(0.0, 0.0, 0.0),
        lo=np.full(3, lo),
        hi=np.full(3, hi),
        seeds=seeds,
        faces_per_cell=np.array(nfaces, np.int64),
        info={"n_voronoi_vertices": n_voro, "n": n, "lo": lo, "hi": hi, "seed": seed,
              "collapsed_edges": merges, "collapse": collapse},
    )
