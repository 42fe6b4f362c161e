"""Per-mesh precompute of the AFE scheme: cell nodes, Jacobians, mass matrices, faces.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 4.1 and the matrix definitions of Sec. 4.3-4.4:

* Each polyhedron P_i is covered by conforming sub-tets T_ik with the affine
  map x = X_0 + J_ik xi, J_ik = dx/dxi (Sec. 4.3); a sub-tet with det J < 0 is
  reoriented by swapping two of its vertices.
* The AFE degrees of freedom of P_i are the union, without repetition, of the
  P_N nodes of its sub-tets (Sec. 4.1, Eq. interp_u).  A node is identified
  topologically by the vertices it lies between and its integer barycentric
  weights, never by its coordinates.
* Cell mass matrix M_i = sum_k |J_ik| A_k^T M^ A_k, with A_k the gather from
  cell nodes to the P_N nodes of T_ik (the reading of the |P_i| prefactor of
  Sec. 4.3-4.4 as assembly by sub-tet Jacobians), and its inverse, stored per
  cell as Sec. 4.3 prescribes for K_1,i.
* Cell faces: every sub-tet triangle not shared inside P_i lies on the cell
  boundary; it is matched to the sub-triangle of the neighbour cell with the
  same vertices (and periodic image) or marked as a domain-boundary face.
* h_i = 6|P_i| / |dP_i| (the characteristic length of Sec. 4.2, read as the
  insphere-equivalent diameter); the cell's diameter (largest vertex distance, the paper's
  example) is kept beside it for the option that uses it instead.
"""
from __future__ import annotations

import numpy as np

from .refelem import ref_element


class CellData:
    __slots__ = ("nodes", "X", "A", "det", "adj", "Jinv", "M", "Minv", "wvec", "vol",
                 "bfaces", "area", "h", "hsub", "diam", "node_key")


class BoundaryTri:
    """One cell-boundary sub-triangle of a cell (the side seen from that cell)."""
    __slots__ = ("k", "o", "nodes", "local", "normal", "area", "nbr", "nbr_tri", "group",
                 "vkeys_sorted", "ref_shift", "canon")


class OracleMesh:
    def __init__(self, xyz, cell_subtet_ptr, subtet_vtx, subtet_shift, period, N, periodic=True):
        self.N = N
        self.R = R = ref_element(N)
        self.period = np.asarray(period, np.float64)
        self.periodic = periodic
        xyz = np.asarray(xyz, np.float64)
        ptr = np.asarray(cell_subtet_ptr, np.int64)
        vtx = np.asarray(subtet_vtx, np.int64)
        shift = None if subtet_shift is None else np.asarray(subtet_shift, np.int64)
        self.n_cells = C = len(ptr) - 1
        self.cells: list[CellData] = []
        for i in range(C):
            self.cells.append(self._build_cell(xyz, vtx, shift, ptr[i], ptr[i + 1]))
        self._match_faces()
        self.node_ptr = np.concatenate([[0], np.cumsum([len(c.nodes) for c in self.cells])])
        self.h_min = min(c.h for c in self.cells)

    # ------------------------------------------------------------------
    def _build_cell(self, xyz, vtx, shift, k0, k1):
        R, N = self.R, self.N
        cd = CellData()
        node_key: dict = {}
        coords = []
        A, X_all, dets, adjs, jinvs, vkeys_all = [], [], [], [], [], []
        for kk in range(k0, k1):
            vk = []
            X = np.empty((4, 3))
            for m in range(4):
                s = (0, 0, 0) if shift is None else tuple(int(v) for v in shift[kk, m])
                vk.append((int(vtx[kk, m]), s))
                X[m] = xyz[vtx[kk, m]] + np.asarray(s, np.float64) * self.period
            J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
            det = np.linalg.det(J)
            if det < 0:  # reorient
                vk[1], vk[2] = vk[2], vk[1]
                X[[1, 2]] = X[[2, 1]]
                J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
                det = np.linalg.det(J)
            if not det > 0:
                raise ValueError("degenerate sub-tet")
            loc = []
            for al in R.bary:
                key = tuple(sorted((vk[m], al[m]) for m in range(4) if al[m] > 0))
                if key not in node_key:
                    node_key[key] = len(coords)
                    coords.append(sum(al[m] / N * X[m] for m in range(4)))
                loc.append(node_key[key])
            Jinv = np.linalg.inv(J)
            A.append(loc)
            X_all.append(X)
            dets.append(det)
            jinvs.append(Jinv)
            adjs.append(det * Jinv)
            vkeys_all.append(vk)
        cd.nodes = np.array(coords)
        cd.node_key = node_key
        cd.A = np.array(A, np.int64)
        cd.X = np.array(X_all)
        cd.det = np.array(dets)
        cd.adj = np.array(adjs)
        cd.Jinv = np.array(jinvs)
        Ni = len(coords)
        M = np.zeros((Ni, Ni))
        for k in range(len(A)):
            idx = cd.A[k]
            M[np.ix_(idx, idx)] += cd.det[k] * R.M
        cd.M = M
        cd.Minv = np.linalg.inv(M)
        cd.wvec = M @ np.ones(Ni)
        cd.vol = cd.det.sum() / 6.0

        # cell-boundary sub-triangles: triangles of the subgrid seen once inside the cell
        count: dict = {}
        for k, vk in enumerate(vkeys_all):
            for o in range(4):
                tk = tuple(sorted(vk[m] for m in range(4) if m != o))
                count.setdefault(tk, []).append((k, o))
        bf = []
        for tk, lst in count.items():
            if len(lst) > 2:
                raise ValueError("non-conforming subgrid")
            if len(lst) == 1:
                k, o = lst[0]
                bt = BoundaryTri()
                bt.k, bt.o = k, o
                others = [m for m in range(4) if m != o]
                X = cd.X[k]
                nrm = np.cross(X[others[1]] - X[others[0]], X[others[2]] - X[others[0]])
                if nrm @ (X[o] - X[others[0]]) > 0:
                    nrm = -nrm
                bt.area = 0.5 * np.linalg.norm(nrm)
                bt.normal = nrm / np.linalg.norm(nrm)
                vk = vkeys_all[k]
                ref = min(vk[m] for m in others)
                rs = np.array(ref[1])
                bt.ref_shift = rs
                bt.canon = tuple(sorted((vk[m][0], tuple(int(x) for x in np.array(vk[m][1]) - rs))
                                        for m in others))
                # face-node order: triangle lattice over the vertices sorted canonically
                order = sorted(others, key=lambda m: (vk[m][0], tuple(np.array(vk[m][1]) - rs)))
                loc_nodes, loc_local = [], []
                for beta in R.tri_bary:
                    al = [0, 0, 0, 0]
                    for b, m in zip(beta, order):
                        al[m] = b
                    j = R.bary.index(tuple(al))
                    loc_local.append(j)
                    loc_nodes.append(cd.A[k][j])
                bt.local = np.array(loc_local)
                bt.nodes = np.array(loc_nodes)
                bf.append(bt)
        cd.bfaces = bf
        area = sum(b.area for b in bf)
        cd.area = area
        cd.h = 6.0 * cd.vol / area
        # smallest sub-tet length 6 |T_k| / |dT_k| (option of the time step's viscous term)
        faces = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
        cd.hsub = min(cd.det[k] / sum(0.5 * np.linalg.norm(np.cross(X[b] - X[a], X[c] - X[a]))
                                      for a, b, c in faces)
                      for k, X in enumerate(cd.X))
        # diameter: the largest distance between two vertices of the cell
        V = cd.X.reshape(-1, 3)
        cd.diam = float(np.sqrt(((V[:, None, :] - V[None, :, :]) ** 2).sum(-1).max()))
        return cd

    def _match_faces(self):
        table: dict = {}
        for i, cd in enumerate(self.cells):
            for f, bt in enumerate(cd.bfaces):
                table.setdefault(bt.canon, []).append((i, f))
        self.n_boundary_tris = 0
        for key, lst in table.items():
            if len(lst) == 2:
                (i, f), (j, g) = lst
                a = self.cells[i].bfaces[f]
                b = self.cells[j].bfaces[g]
                a.nbr, a.nbr_tri = j, g
                b.nbr, b.nbr_tri = i, f
                off = tuple(int(x) for x in (a.ref_shift - b.ref_shift))
                a.group = ("int", j, off)
                b.group = ("int", i, tuple(-x for x in off))
            elif len(lst) == 1:
                if self.periodic:
                    raise ValueError("unmatched face on a periodic mesh")
                i, f = lst[0]
                a = self.cells[i].bfaces[f]
                a.nbr, a.nbr_tri = -1, -1
                a.group = ("bnd", f)
                self.n_boundary_tris += 1
            else:
                raise ValueError("face shared by more than two cells")

    # ------------------------------------------------------------------
    @property
    def n_nodes(self) -> int:
        return int(self.node_ptr[-1])

    def node_coords(self) -> np.ndarray:
        return np.concatenate([c.nodes for c in self.cells])

    def split(self, u):
        """Global node-major [n_nodes, 5] -> list of per-cell views."""
        return [u[self.node_ptr[i]:self.node_ptr[i + 1]] for i in range(self.n_cells)]


def from_polymesh(pm, N) -> OracleMesh:
    return OracleMesh(pm.xyz, pm.cell_subtet_ptr, pm.subtet_vtx, pm.subtet_shift, pm.period, N,
                      periodic=pm.periodic)
