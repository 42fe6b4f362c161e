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
* Quality step: Voronoi edges shorter than ``COLLAPSE`` times the lattice spacing
  are collapsed (their end points merged topologically).  Short edges give
  needle-shaped fan sub-tets whose tiny support makes the element-local
  operators stiff enough to stall the predictor's fixed-point iteration; this
  step stands in for the admissible-cell guarantee of the paper's own mesh
  generator (Sec. 3).  A merge that would fold a sub-tet is skipped.
* Lloyd steps: before the tessellation used, each jittered seed is moved ``LLOYD``
  times to the volume centroid of its own Voronoi cell.  Together with the collapse
  this removes the thin faces and needle sub-tets that otherwise leave cells whose
  predictor iteration diverges at CFL 0.3 (with one step and a collapse threshold
  of 0.2, the smallest critical CFL of the fixed-point iteration over a 16^3 mesh
  at N = 2 is 0.27; with four steps and 0.25 it is 0.44).
* Thin faces: a face whose centre lies closer than ``THIN`` times the lattice
  spacing to the line of one of its edges has its shortest edge collapsed too.
* Flat sub-tets: likewise a face one of whose fan triangles lies in a plane passing closer
  than ``FLAT`` times the lattice spacing to the cell centre (a face warped by the
  collapse); such a sub-tet makes the ADER step locally unstable at the CFL numbers used.
* Fan subgrid: each cell is split by joining its centre (the mean of its
  vertices) to a fan triangulation of each face about the face centre (the mean
  of the face's vertices): one sub-tet per face edge.

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
COLLAPSE = 0.25
# fan triangles whose face centre is closer than THIN * (lattice spacing) to their edge
# mark a thin face; its shortest edge is collapsed too
THIN = 0.08
# Lloyd steps applied to the jittered seeds (each moves a seed to its cell's centroid)
LLOYD = 4
# fan triangles whose plane passes closer than FLAT * (lattice spacing) to the cell centre
# (flat sub-tets of warped faces) mark the face like a thin one; 0 turns the test off
FLAT = 0.1


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


class _Fold(Exception):
    """A non-positive fan sub-tet: ``near`` holds the vertices of the offending edges,
    ``face`` all vertices of the faces involved."""

    def __init__(self, near, face=None):
        super().__init__("folded fan sub-tet")
        self.near = list(near)
        self.face = list(face if face is not None else near)


def _original_faces(vor, P, C):
    """Faces of the original cells (< C) as flat arrays: cell, neighbour point, CSR offsets
    and scipy vertex ids ordered counter-clockwise about the outward normal."""
    rp = vor.ridge_points
    sel = np.nonzero((rp[:, 0] < C) | (rp[:, 1] < C))[0]
    cells, nbrs, rid = [], [], []
    for a_is in (0, 1):
        side = sel[rp[sel, a_is] < C]
        cells.append(rp[side, a_is])
        nbrs.append(rp[side, 1 - a_is])
        rid.append(side)
    cells = np.concatenate(cells)
    nbrs = np.concatenate(nbrs)
    rid = np.concatenate(rid)
    order = np.lexsort((rid, cells))
    cells, nbrs, rid = cells[order], nbrs[order], rid[order]
    verts = [vor.ridge_vertices[r] for r in rid]
    cnt = np.array([len(v) for v in verts])
    ptr = np.concatenate([[0], np.cumsum(cnt)])
    flat = np.concatenate([np.asarray(v) for v in verts])
    if np.any(flat < 0):
        raise RuntimeError("unbounded ridge next to an original cell; margin too small")
    # qhull lists the vertices of a 3-d ridge in cyclic order; orient about the outward normal
    X = vor.vertices[flat]
    nxt = np.arange(len(flat)) + 1
    nxt[ptr[1:] - 1] = ptr[:-1]
    area = np.add.reduceat(np.cross(X, X[nxt]), ptr[:-1], axis=0)
    flip = np.einsum("fd,fd->f", area, P[nbrs] - P[cells]) < 0
    fidx = np.repeat(np.arange(len(cnt)), cnt)
    local = np.arange(len(flat)) - ptr[fidx]
    src = np.where(flip[fidx], ptr[fidx] + cnt[fidx] - 1 - local, np.arange(len(flat)))
    return cells, nbrs, ptr, flat[src]


def _next_index(ptr):
    nxt = np.arange(ptr[-1]) + 1
    nxt[ptr[1:] - 1] = ptr[:-1]
    return nxt


def _collapse(pos, ptr, fv, fs, L, tol, exclude, force=(), anchor=()):
    """Union-find merge of the end points of Voronoi edges shorter than tol.

    pos: canonical vertex positions [nv, 3]; (ptr, fv, fs): per face the vertex ids and their
    image shifts in the cell frame.  A vertex in ``exclude`` is never merged.  A merged
    vertex sits at the mean of its members, or at the position of its member listed in
    ``anchor``.  Returns merged positions, the new faces (ptr, fv, fs), kept face indices,
    merge count and the members of each merged vertex.
    """
    nv = len(pos)
    Lf = 0.0 if L is None else L
    nxt = _next_index(ptr)
    P = pos[fv] + fs * Lf
    d = np.linalg.norm(P - P[nxt], axis=1)

    par = list(range(nv))
    ofs = [(0, 0, 0)] * nv

    def find(x):
        o0 = o1 = o2 = 0
        while par[x] != x:
            a = ofs[x]
            o0 += a[0]
            o1 += a[1]
            o2 += a[2]
            x = par[x]
        return x, (o0, o1, o2)

    merges = 0
    cand = d < tol
    if len(force):
        cand[np.asarray(sorted(force), np.int64)] = True
    fvl = fv.tolist()
    fsl = [tuple(r) for r in fs.tolist()]
    nxl = nxt.tolist()
    for e in np.nonzero(cand)[0].tolist():
        a, b = fvl[e], fvl[nxl[e]]
        if a in exclude or b in exclude:
            continue
        ra, oa = find(a)
        rb, ob = find(b)
        sa, sb = fsl[e], fsl[nxl[e]]
        rel = (oa[0] + sa[0] - ob[0] - sb[0], oa[1] + sa[1] - ob[1] - sb[1], oa[2] + sa[2] - ob[2] - sb[2])
        if ra == rb:
            if rel != (0, 0, 0):
                raise RuntimeError("short-edge cluster wraps around the period")
            continue
        par[rb] = ra
        ofs[rb] = rel
        merges += 1
    parent = np.asarray(par, np.int64)
    off = np.asarray(ofs, np.int64).reshape(nv, 3)
    # pointer jumping: root of every vertex and its image offset relative to the root
    p = parent.copy()
    roff = off.copy()
    while True:
        pp = p[p]
        if np.array_equal(pp, p):
            break
        roff = roff + roff[p]
        p = pp
    uniq, new_id = np.unique(p, return_inverse=True)
    size = np.bincount(new_id)
    order = np.argsort(new_id, kind="stable")
    bounds = np.concatenate([[0], np.cumsum(size)])
    members = [order[bounds[i]:bounds[i + 1]].tolist() for i in range(len(uniq))]
    acc = np.zeros((len(uniq), 3))
    np.add.at(acc, new_id, pos - roff * Lf)
    new_pos = acc / size[:, None]
    for v in anchor:
        if size[new_id[v]] > 1:
            new_pos[new_id[v]] = pos[v] - roff[v] * Lf
    ids = new_id[fv]
    sh = fs + roff[fv]
    # drop cyclically repeated vertices (collapsed edges), then faces left with < 3 vertices
    same = (ids == ids[nxt]) & np.all(sh == sh[nxt], axis=1)
    keep_e = ~same
    cnt2 = np.add.reduceat(keep_e.astype(np.int64), ptr[:-1])
    fidx = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    # a face whose vertices all merged keeps none; a pinched face repeats a vertex
    rows = np.concatenate([fidx[keep_e][:, None], ids[keep_e][:, None], sh[keep_e]], 1)
    nuniq = np.bincount(np.unique(rows, axis=0)[:, 0], minlength=len(ptr) - 1)
    pinched = np.nonzero(nuniq != cnt2)[0]
    if len(pinched):
        f = int(pinched[0])
        raise _Fold([int(x) for x in ids[ptr[f]:ptr[f + 1]]])
    keep_f = cnt2 >= 3
    keep_e &= keep_f[fidx]
    cnt3 = cnt2[keep_f]
    ptr2 = np.concatenate([[0], np.cumsum(cnt3)])
    return new_pos, ptr2, ids[keep_e], sh[keep_e], np.nonzero(keep_f)[0], merges, members, new_id


def _fan(pos, cells, ptr, fv, fs, L, C, face_key, allow_fold=False):
    """Face centres, cell centres and fan sub-tets; raises _Fold on a non-positive sub-tet
    unless ``allow_fold`` (sub-tets used only for cell centroids)."""
    Lf = 0.0 if L is None else L
    cnt = np.diff(ptr)
    X = pos[fv] + fs * Lf
    fpos = np.add.reduceat(X, ptr[:-1], axis=0) / cnt[:, None]
    # face centres: one vertex per face pair, in a canonical frame
    nf = len(cnt)
    krows, fc_sh = face_key(np.arange(nf))
    _, first, inv = np.unique(krows, axis=0, return_index=True, return_inverse=True)
    inv = inv.ravel()
    extra = fpos[first] - fc_sh[first] * Lf
    fc_id = len(pos) + inv
    fidx = np.repeat(np.arange(nf), cnt)
    fcell = cells[fidx]
    # cell centres: mean of the distinct vertices of each cell
    rows = np.concatenate([fcell[:, None], fv[:, None], fs], 1)
    u = np.unique(rows, axis=0)
    upos = pos[u[:, 1]] + u[:, 2:] * Lf
    csum = np.zeros((C, 3))
    np.add.at(csum, u[:, 0], upos)
    ccen = csum / np.bincount(u[:, 0], minlength=C)[:, None]
    cc_id = len(pos) + len(extra) + np.arange(C)
    xyz = np.concatenate([pos, extra, ccen])
    # fan sub-tets (cell centre, face centre, v_i, v_i+1)
    nxt = _next_index(ptr)
    vtx = np.stack([cc_id[fcell], fc_id[fidx], fv, fv[nxt]], 1)
    sh = np.stack([np.zeros_like(fs), fc_sh[fidx], fs, fs[nxt]], 1)
    P = xyz[vtx] + sh * Lf
    det = np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], -1))
    bad = np.nonzero(~(det > 0))[0]
    if len(bad) and not allow_fold:
        near = sorted({int(v) for j in bad for v in (fv[j], fv[nxt[j]])})
        face = sorted({int(v) for f in set(fidx[bad].tolist()) for v in fv[ptr[f]:ptr[f + 1]]})
        raise _Fold(near, face)
    sub_ptr = np.concatenate([[0], np.cumsum(np.bincount(fcell, minlength=C))])
    return xyz, sub_ptr, vtx, sh


def _thin_faces(xyz, vtx, sh, L, h, thin, flatness=0.0):
    """Fan sub-tets whose face centre lies within thin*h of the line of their face edge, or
    (flatness > 0) whose fan triangle's plane passes within flatness*h of the cell centre."""
    Lf = 0.0 if L is None else L
    P = xyz[vtx] + sh * Lf
    e = P[:, 3] - P[:, 2]
    u = e / np.linalg.norm(e, axis=1)[:, None]
    w = P[:, 1] - P[:, 2]
    dist = np.linalg.norm(w - u * np.einsum("ij,ij->i", w, u)[:, None], axis=1)
    bad = dist < thin * h
    if flatness > 0:
        nrm = np.cross(P[:, 2] - P[:, 1], P[:, 3] - P[:, 1])
        height = np.abs(np.einsum("ij,ij->i", P[:, 0] - P[:, 1], nrm)) / np.linalg.norm(nrm, axis=1)
        bad |= height < flatness * h
    return np.nonzero(bad)[0]


def _assemble(pos, cells, ptr, fv, fs, nbrs, L, C, tol, face_key_of, thin=THIN, h=0.0, flatness=FLAT,
              allow_fold=False):
    exclude: set = set()
    force: set = set()
    anchor: set = set()
    tried: dict = {}  # merge group -> members already tried as its position
    nxt0 = _next_index(ptr)
    for _ in range(400):
        if tol > 0:
            new_pos, ptr2, fv2, fs2, keep, merges, members, new_id = _collapse(pos, ptr, fv, fs, L, tol, exclude,
                                                                               force, anchor)
        else:
            new_pos, ptr2, fv2, fs2, keep, merges = pos, ptr, fv, fs, np.arange(len(ptr) - 1), 0
            members = [[i] for i in range(len(pos))]
            new_id = np.arange(len(pos))
        try:
            kc = cells[keep]
            kn = nbrs[keep]
            xyz, sub_ptr, vtx, sh = _fan(new_pos, kc, ptr2, fv2, fs2, L, C, lambda f: face_key_of(kc[f], kn[f]),
                                         allow_fold)
        except _Fold as e:
            # first place a merged vertex at the folded edges at one of its members instead of
            # the members' mean (a short edge collapses onto an end point); when every choice
            # folds, undo the fewest merges: those at the folded edges, then the whole face
            moved = False
            seen = set()
            for v in e.near:  # every folded place at once
                grp = members[v] if v < len(members) else []
                key = frozenset(grp)
                if len(grp) < 2 or key in seen or any(g in exclude for g in grp):
                    continue
                seen.add(key)
                k = tried.get(key, 0)
                if k < len(grp):
                    tried[key] = k + 1
                    anchor.difference_update(grp)
                    anchor.add(sorted(grp)[k])
                    moved = True
            if moved:
                continue
            for group in (e.near, e.face):
                grow = set()
                for v in group:
                    if len(members[v]) > 1:
                        grow |= set(members[v])
                if not grow <= exclude:
                    break
            else:
                raise RuntimeError("cannot build a fold-free fan subgrid")
            exclude |= grow
            anchor.difference_update(grow)
            continue
        if tol > 0 and thin > 0:
            # thin faces: collapse the shortest edge of every face with a thin fan triangle
            bad = _thin_faces(xyz, vtx, sh, L, h, thin, flatness)
            added = False
            if len(bad):
                cnt2 = np.diff(ptr2)
                fidx2 = np.repeat(np.arange(len(cnt2)), cnt2)
                nxt2 = _next_index(ptr2)
                P = new_pos[fv2] + fs2 * (0.0 if L is None else L)
                elen = np.linalg.norm(P - P[nxt2], axis=1)
                for f in sorted(set(fidx2[bad].tolist())):
                    j = ptr2[f] + int(np.argmin(elen[ptr2[f]:ptr2[f + 1]]))
                    A, B = fv2[j], fv2[nxt2[j]]
                    of = keep[f]
                    for e in range(ptr[of], ptr[of + 1]):
                        if (new_id[fv[e]], new_id[fv[nxt0[e]]]) in ((A, B), (B, A)) and e not in force \
                                and fv[e] not in exclude and fv[nxt0[e]] not in exclude:
                            force.add(e)
                            added = True
                            break
            if added:
                continue
        return xyz, sub_ptr, vtx, sh, merges, len(new_pos), np.bincount(kc, minlength=C)
    raise RuntimeError("edge collapse did not settle")


def _periodic_voronoi(n: int, L: float = 1.0, seed: int = 0, collapse: float = COLLAPSE,
                      seeds: np.ndarray | None = None, thin: float = THIN, flatness: float = FLAT,
                      allow_fold: bool = False) -> PolyMesh:
    """Periodic jittered-lattice Voronoi mesh of ``[0, L)^3`` with fan subgrids."""
    if seeds is None:
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
    cells, nbrs, ptr, flat = _original_faces(vor, P, C)

    # generators of every Voronoi vertex (points whose region holds it)
    # generators of every used Voronoi vertex (the points whose region holds it), as codes
    # pid*125 + (shift+2) in base 5: ordering the codes orders by (seed, image shift)
    used = np.unique(flat)
    regs = [vor.regions[vor.point_region[p]] for p in range(len(P))]
    rv = np.concatenate([np.asarray(r, np.int64) for r in regs])
    rp = np.repeat(np.arange(len(P)), [len(r) for r in regs])
    keep = (rv >= 0) & np.isin(rv, used)
    rv, rp = rv[keep], rp[keep]
    order = np.lexsort((rp, rv))
    rv, rp = rv[order], rp[order]
    w5 = np.array([25, 5, 1])
    code = pid[rp] * 125 + (psh[rp] + 2) @ w5
    ngen = np.bincount(np.searchsorted(used, rv), minlength=len(used))
    gptr = np.concatenate([[0], np.cumsum(ngen)])
    # reference generator (smallest code) and codes relative to its image
    ref_code = np.minimum.reduceat(code, gptr[:-1])
    ref_sh = ((ref_code[:, None] // w5) % 5) - 2
    rel_sh = psh[rp] - np.repeat(ref_sh, ngen, axis=0)
    rel = pid[rp] * 125 + (rel_sh + 2) @ w5
    maxg = int(ngen.max())
    keys = np.full((len(used), maxg), -1, np.int64)
    col = np.arange(len(rv)) - np.repeat(gptr[:-1], ngen)
    keys[np.repeat(np.arange(len(used)), ngen), col] = rel
    keys = -np.sort(-keys, axis=1)                      # sorted, padding last
    _, first, vid = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    vid = vid.ravel()
    vsh = ref_sh
    pos = vor.vertices[used[first]] - ref_sh[first] * L
    # faces keep the order of first appearance of their vertices irrelevant: positions by id
    loc = np.searchsorted(used, flat)
    fv = vid[loc]
    fs = vsh[loc]

    def face_key_of(a, b):
        """Canonical key rows and frame shifts of the faces between points a and b (arrays)."""
        ca = pid[a] * 125 + (psh[a] + 2) @ w5
        cb = pid[b] * 125 + (psh[b] + 2) @ w5
        r = np.minimum(ca, cb)
        rs = ((r[:, None] // w5) % 5) - 2
        ka = pid[a] * 125 + (psh[a] - rs + 2) @ w5
        kb = pid[b] * 125 + (psh[b] - rs + 2) @ w5
        return np.stack([np.minimum(ka, kb), np.maximum(ka, kb)], 1), rs

    xyz, sub_ptr, vtx, sh, merges, nvor, nfaces = _assemble(pos, cells, ptr, fv, fs, nbrs, L, C,
                                                            collapse * L / n, face_key_of, thin=thin, h=L / n,
                                                            flatness=flatness, allow_fold=allow_fold)
    if np.abs(sh).max() > 127:
        raise RuntimeError("image shift out of int8 range")
    return PolyMesh(xyz=xyz, cell_subtet_ptr=sub_ptr.astype(np.int64), subtet_vtx=vtx.astype(np.int64),
                    subtet_shift=sh.astype(np.int8), periodic=True, period=(L, L, L), lo=np.zeros(3),
                    hi=np.full(3, L), seeds=seeds, faces_per_cell=nfaces,
                    info={"n_voronoi_vertices": nvor, "n": n, "L": L, "seed": seed, "collapsed_edges": merges,
                          "collapse": collapse})


def _box_voronoi(n: int, lo: float = -1.0, hi: float = 1.0, seed: int = 0,
                 collapse: float = COLLAPSE, seeds: np.ndarray | None = None, thin: float = THIN,
                 flatness: float = FLAT, allow_fold: bool = False) -> PolyMesh:
    """Jittered-lattice Voronoi mesh of the box ``[lo, hi]^3`` with fan subgrids."""
    if seeds is None:
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
    cells, nbrs, ptr, flat = _original_faces(vor, P, C)
    used = np.unique(flat)
    pos = vor.vertices[used]
    fv = np.searchsorted(used, flat)
    fs = np.zeros((len(fv), 3), np.int64)

    def face_key_of(a, b):
        a = np.asarray(a)
        b = np.asarray(b)
        inner = b < C
        k0 = np.where(inner, np.minimum(a, b), a)
        k1 = np.where(inner, np.maximum(a, b), -1 - b)
        return np.stack([k0, k1], 1), np.zeros((len(a), 3), np.int64)

    xyz, sub_ptr, vtx, sh, merges, nvor, nfaces = _assemble(pos, cells, ptr, fv, fs, nbrs, None, C,
                                                            collapse * h, face_key_of, thin=thin, h=h,
                                                            flatness=flatness, allow_fold=allow_fold)
    return PolyMesh(xyz=xyz, cell_subtet_ptr=sub_ptr.astype(np.int64), subtet_vtx=vtx.astype(np.int64),
                    subtet_shift=None, periodic=False, period=(0.0, 0.0, 0.0), lo=np.full(3, lo),
                    hi=np.full(3, hi), seeds=seeds, faces_per_cell=nfaces,
                    info={"n_voronoi_vertices": nvor, "n": n, "lo": lo, "hi": hi, "seed": seed,
                          "collapsed_edges": merges, "collapse": collapse})


def cell_centroids(pm: PolyMesh) -> np.ndarray:
    """Volume centroids of the cells (from the sub-tets), in the frame of each cell."""
    X = pm.subtet_coords()
    vol = np.abs(np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], -1))) / 6
    cell = np.repeat(np.arange(pm.n_cells), np.diff(pm.cell_subtet_ptr))
    num = np.zeros((pm.n_cells, 3))
    np.add.at(num, cell, vol[:, None] * X.mean(axis=1))
    return num / np.bincount(cell, weights=vol, minlength=pm.n_cells)[:, None]


def periodic_voronoi(n: int, L: float = 1.0, seed: int = 0, collapse: float = COLLAPSE,
                     lloyd: int = LLOYD, thin: float = THIN, flat: float = FLAT) -> PolyMesh:
    """Periodic jittered-lattice Voronoi mesh of ``[0, L)^3`` with fan subgrids, after
    ``lloyd`` Lloyd steps of the jittered seeds, the short-edge collapse and the thin-face
    collapse (``thin``: the threshold in lattice spacings)."""
    seeds = jittered_seeds(n, 0.0, L, seed)
    for _ in range(lloyd):
        # (raw cells: a degenerate face may give a flat or folded fan sub-tet, harmless here)
        seeds = np.mod(cell_centroids(_periodic_voronoi(n, L, collapse=0.0, seeds=seeds, allow_fold=True)), L)
    pm = _periodic_voronoi(n, L, seed, collapse, seeds=seeds, thin=thin, flatness=flat)
    pm.info["lloyd"] = lloyd
    pm.info["thin"] = thin
    pm.info["flat"] = flat
    return pm


def box_voronoi(n: int, lo: float = -1.0, hi: float = 1.0, seed: int = 0, collapse: float = COLLAPSE,
                lloyd: int = LLOYD, thin: float = THIN, flat: float = FLAT) -> PolyMesh:
    """Jittered-lattice Voronoi mesh of the box ``[lo, hi]^3`` with fan subgrids, after
    ``lloyd`` Lloyd steps of the jittered seeds, the short-edge collapse and the thin-face
    collapse (``thin``: the threshold in lattice spacings)."""
    seeds = jittered_seeds(n, lo, hi, seed)
    for _ in range(lloyd):
        seeds = cell_centroids(_box_voronoi(n, lo, hi, collapse=0.0, seeds=seeds, allow_fold=True))
    pm = _box_voronoi(n, lo, hi, seed, collapse, seeds=seeds, thin=thin, flatness=flat)
    pm.info["lloyd"] = lloyd
    pm.info["thin"] = thin
    pm.info["flat"] = flat
    return pm
