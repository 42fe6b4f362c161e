"""Hand-built box meshes of cubes whose edges carry extra vertices (input generation only).

Each cube of an ``nx x ny x nz`` lattice (side ``d``, lower corner at the origin) is a
polyhedron whose six square faces are polygons: every cube edge along axis a is split into
``splits[a]`` equal segments, so a face normal to axis a has ``2 (splits[b] + splits[c])``
polygon edges.  The fan subgrid is built exactly as for the Voronoi meshes: the cube centre
joined to a fan of each face polygon about the face centre, one sub-tet per polygon edge.
The split points are shared by all cubes around an edge, so the subgrid is conforming.

More polygon edges mean more sub-tets and more AFE nodes per cell than a jittered Voronoi
cell has (a cube with splits (4, 3, 3) has 80 sub-tets and, at N = 3, 567 nodes), which is
what tests of the library's large-cell code paths need.  Boundary: transmissive box.
Nothing here computes any part of the scheme.
"""
from __future__ import annotations

import numpy as np

from .voronoi import PolyMesh


def split_cube_lattice(shape=(1, 1, 1), splits=(1, 1, 1), d: float = 0.5) -> PolyMesh:
    """Box mesh of ``shape`` cubes of side ``d`` with ``splits[a]`` segments per edge along a."""
    shape = tuple(int(s) for s in shape)
    splits = tuple(int(s) for s in splits)
    if min(shape) < 1 or min(splits) < 1:
        raise ValueError("shape and splits must be positive")
    ids: dict = {}
    xyz: list = []

    def vid(key, pos):
        if key not in ids:
            ids[key] = len(xyz)
            xyz.append(np.asarray(pos, np.float64))
        return ids[key]

    def grid_vertex(g):
        # g: refined integer coordinates (cube index * splits + offset along each axis)
        return vid(("v",) + tuple(g), [g[a] * d / splits[a] for a in range(3)])

    vtx, ptr, nfaces = [], [0], []
    for ci in range(shape[0]):
        for cj in range(shape[1]):
            for ck in range(shape[2]):
                base = (ci, cj, ck)
                corner0 = [base[a] * splits[a] for a in range(3)]
                centre = vid(("c",) + base, [(base[a] + 0.5) * d for a in range(3)])
                for ax in range(3):
                    e1, e2 = (ax + 1) % 3, (ax + 2) % 3
                    for side in (0, 1):
                        # polygon ring around the face: along e1, e2, back along e1, back along e2
                        ring = []
                        walk = [(e1, splits[e1], +1), (e2, splits[e2], +1), (e1, splits[e1], -1),
                                (e2, splits[e2], -1)]
                        g = list(corner0)
                        g[ax] += side * splits[ax]
                        for axis, m, sgn in walk:
                            for _ in range(m):
                                ring.append(grid_vertex(g))
                                g[axis] += sgn
                        fpos = [(base[a] + 0.5) * d for a in range(3)]
                        fpos[ax] = (base[ax] + side) * d
                        f = vid(("f", ax) + tuple(2 * base[a] + (2 * side if a == ax else 1) for a in range(3)), fpos)
                        for r in range(len(ring)):
                            vtx.append((centre, f, ring[r], ring[(r + 1) % len(ring)]))
                ptr.append(len(vtx))
                nfaces.append(6)
    xyz_a = np.array(xyz)
    hi = np.array([shape[a] * d for a in range(3)])
    return PolyMesh(xyz=xyz_a, cell_subtet_ptr=np.array(ptr, np.int64), subtet_vtx=np.array(vtx, np.int64),
                    subtet_shift=None, periodic=False, period=(0.0, 0.0, 0.0), lo=np.zeros(3), hi=hi,
                    seeds=np.array([[(i + 0.5) * d, (j + 0.5) * d, (k + 0.5) * d] for i in range(shape[0])
                                    for j in range(shape[1]) for k in range(shape[2])]),
                    faces_per_cell=np.array(nfaces, np.int64),
                    info={"shape": shape, "splits": splits, "d": d})
