"""Cell partition of one mesh over several ranks and the bookkeeping of its one exchange per step.

The predictor of Sec. 4.3 is local to each cell, so a mesh splits across ranks (one GPU
each) by cells.  One step then needs, besides each rank's own cells:

* the time step: the CFL bracket's maximum over all nodes and the smallest characteristic
  length (Sec. 4.2) -- one max / min all-reduce of two numbers;
* with the limiter (Sec. 4.5), the cell means of the face neighbours on other ranks before
  the detector;
* before the Rusanov fluxes (Sec. 4.4, Eq. 3.33) on the sub-triangles between two ranks:
  the other side's time-integrated predictor and flux at the sub-triangle's face nodes, and
  the other cell's viscosity and characteristic length.

This module computes, from the mesh arrays alone (the same arrays ``afe_mesh_create`` takes),
a recursive-coordinate-bisection partition and, per pair of ranks, the matched lists of
cross-partition sub-triangles and cells in one order both ranks derive independently, so
that item i of what rank r sends to rank s is item i of what s receives from r.  A
sub-triangle is identified by its owning cell and its vertices (global ids with their
periodic images relative to the smallest id), which is independent of any node numbering.
``exchange`` moves numpy buffers between ranks with ``torch.distributed`` point-to-point
calls (gloo on CPU, NCCL between GPUs); nothing here touches GPU memory of another device.

``RankMesh`` is the library side: a rank's own cells plus ghost-cell layers as one handle,
stepped with the global time step after the ghosts' states arrive from their owners
(``step_rank_distributed`` with one process per rank, ``step_ranks_in_process`` when the
ranks share a process).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np


def cell_centroids(pm) -> np.ndarray:
    """Volume centroids of the cells from their sub-tets (each in its own cell's frame)."""
    X = np.asarray(pm.xyz, np.float64)[np.asarray(pm.subtet_vtx)]
    if pm.subtet_shift is not None:
        X = X + np.asarray(pm.subtet_shift, np.float64) * np.asarray(pm.period, np.float64)
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], -1)
    vol = np.abs(np.linalg.det(J)) / 6.0
    cell = np.repeat(np.arange(len(pm.cell_subtet_ptr) - 1), np.diff(pm.cell_subtet_ptr))
    C = len(pm.cell_subtet_ptr) - 1
    num = np.zeros((C, 3))
    np.add.at(num, cell, vol[:, None] * X.mean(axis=1))
    return num / np.bincount(cell, weights=vol, minlength=C)[:, None]


def bisect(points: np.ndarray, nparts: int) -> np.ndarray:
    """Recursive coordinate bisection: split the cells at the median of the coordinate with the
    largest extent, in proportion to the parts each side gets, until there are ``nparts``
    parts.  Ties are broken by cell index, so the result is deterministic."""
    points = np.asarray(points, np.float64)
    labels = np.zeros(len(points), np.int64)

    def split(idx: np.ndarray, first: int, parts: int):
        if parts == 1:
            labels[idx] = first
            return
        p = points[idx]
        axis = int(np.argmax(p.max(axis=0) - p.min(axis=0))) if len(idx) else 0
        order = idx[np.lexsort((idx, p[:, axis]))]
        left_parts = parts // 2
        cut = int(round(len(order) * left_parts / parts))
        split(order[:cut], first, left_parts)
        split(order[cut:], first + left_parts, parts - left_parts)

    split(np.arange(len(points)), 0, int(nparts))
    return labels


def _tri_key(vid, sh, others):
    ref = min((int(vid[m]), tuple(int(x) for x in sh[m])) for m in others)
    rs = np.array(ref[1])
    return tuple(sorted((int(vid[m]), tuple(int(x) for x in np.array(sh[m]) - rs)) for m in others))


def boundary_triangles(pm) -> Dict[tuple, List[int]]:
    """canonical triangle key -> the cells having it as a cell-boundary sub-triangle (one or two)."""
    vtx = np.asarray(pm.subtet_vtx)
    shift = None if pm.subtet_shift is None else np.asarray(pm.subtet_shift)
    ptr = np.asarray(pm.cell_subtet_ptr)
    table: Dict[tuple, List[int]] = {}
    zero = np.zeros((4, 3), np.int64)
    for c in range(len(ptr) - 1):
        count: Dict[tuple, int] = {}
        for k in range(ptr[c], ptr[c + 1]):
            sh = zero if shift is None else shift[k]
            for o in range(4):
                key = _tri_key(vtx[k], sh, [m for m in range(4) if m != o])
                count[key] = count.get(key, 0) + 1
        for key, n in count.items():
            if n == 1:  # not shared inside the cell: on its boundary
                table.setdefault(key, []).append(c)
    return table


@dataclass
class Peer:
    """What one rank exchanges with one other rank, in the order both derive."""
    rank: int
    tris: List[Tuple[int, tuple]] = field(default_factory=list)        # (own cell, triangle key)
    partner_cells: List[int] = field(default_factory=list)             # the other side's cell, same order
    send_cells: List[int] = field(default_factory=list)                # own cells next to the peer
    recv_cells: List[int] = field(default_factory=list)                # the peer's cells next to us


@dataclass
class HaloPlan:
    rank: int
    nparts: int
    labels: np.ndarray
    owned: np.ndarray
    peers: Dict[int, Peer]

    def n_halo_tris(self) -> int:
        return sum(len(p.tris) for p in self.peers.values())


def halo_plan(pm, labels: np.ndarray, rank: int) -> HaloPlan:
    """The exchange plan of ``rank`` for the partition ``labels`` (cell -> rank)."""
    labels = np.asarray(labels, np.int64)
    nparts = int(labels.max()) + 1
    pairs: Dict[int, List[Tuple[tuple, int, int]]] = {}
    for key, cells in boundary_triangles(pm).items():
        if len(cells) != 2:
            continue
        a, b = cells
        la, lb = labels[a], labels[b]
        if la == lb or rank not in (la, lb):
            continue
        mine, other = (a, b) if la == rank else (b, a)
        pairs.setdefault(int(labels[other]), []).append((key, mine, other))
    peers = {}
    for s, lst in sorted(pairs.items()):
        lst.sort(key=lambda e: (e[0], min(e[1], e[2]), max(e[1], e[2])))  # same order on both ranks
        p = Peer(rank=s)
        for key, mine, other in lst:
            p.tris.append((mine, key))
            p.partner_cells.append(other)
        p.send_cells = sorted({mine for _, mine, _ in lst})
        p.recv_cells = sorted({other for _, _, other in lst})
        peers[s] = p
    return HaloPlan(rank=rank, nparts=nparts, labels=labels, owned=np.flatnonzero(labels == rank), peers=peers)


def exchange(dist, plan: HaloPlan, send: Dict[int, np.ndarray], recv_shapes: Dict[int, tuple],
             dtype=np.float64) -> Dict[int, np.ndarray]:
    """Send ``send[s]`` to every peer s and receive an array of ``recv_shapes[s]`` from it
    (non-blocking sends, then blocking receives: no ordering deadlock between two ranks)."""
    import torch
    reqs = []
    for s in sorted(plan.peers):
        t = torch.from_numpy(np.ascontiguousarray(send[s], dtype=dtype))
        reqs.append((dist.isend(t, dst=s), t))
    out = {}
    for s in sorted(plan.peers):
        t = torch.empty(recv_shapes[s], dtype=torch.float64 if dtype == np.float64 else torch.float32)
        dist.recv(t, src=s)
        out[s] = t.numpy()
    for r, _ in reqs:
        r.wait()
    return out


def allreduce_max_min(dist, x_max: float, x_min: float, device=None) -> Tuple[float, float]:
    """(max over ranks of x_max, min over ranks of x_min): the two reductions of the time step."""
    import torch
    t = torch.tensor([x_max, -x_min], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0]), float(-t[1])


def cell_neighbours(pm) -> List[set]:
    """Face neighbours of every cell (cells sharing a cell-boundary sub-triangle)."""
    C = len(pm.cell_subtet_ptr) - 1
    nb = [set() for _ in range(C)]
    for cells in boundary_triangles(pm).values():
        if len(cells) == 2 and cells[0] != cells[1]:
            nb[cells[0]].add(cells[1])
            nb[cells[1]].add(cells[0])
    return nb


def ghost_cells(nb: List[set], labels: np.ndarray, rank: int, layers: int) -> List[int]:
    """The ghost cells of `rank`: `layers` layers of face neighbours around its own cells, layer
    by layer, each in index order."""
    own = set(int(c) for c in np.flatnonzero(np.asarray(labels) == rank))
    inside, ghosts, front = set(own), [], set(own)
    for _ in range(layers):
        nxt = sorted({j for c in front for j in nb[c]} - inside)
        ghosts += nxt
        inside |= set(nxt)
        front = set(nxt)
    return ghosts


class RankMesh:
    """One rank's part of a partitioned mesh as a library handle: its own cells followed by
    `layers` layers of ghost cells (the face neighbours on other ranks; two layers when the
    limiter is on, so that the ghosts' artificial viscosity, which reads their neighbours'
    cell means, is the owner's).  A step of the whole mesh is then, on every rank: receive the
    ghost cells' states from their owners (`pack` / `unpack`), reduce the CFL pieces of the own
    cells over the ranks (`cfl_pieces`, then max / min), and step the handle with that dt.  The
    own cells end with the one-mesh result: their predictors, their neighbours' predictors and
    every flux across their faces see the same data; the ghosts' results are discarded (their
    outer faces are transmissive) and replaced at the next exchange.  The library kernels only
    ever read this rank's device memory; the exchange moves host (gloo) or device (NCCL)
    buffers through ``torch.distributed`` or any equivalent transport.
    """

    def __init__(self, pm, labels, rank: int, params, layers: int = None, stream: int = 0):
        from . import afe as _afe
        self.afe = _afe
        labels = np.asarray(labels, np.int64)
        self.rank, self.labels = rank, labels
        if layers is None:
            layers = 2 if int(params.limiter) else 1
        nb = cell_neighbours(pm)
        own = [int(c) for c in np.flatnonzero(labels == rank)]
        ghosts = ghost_cells(nb, labels, rank, layers)
        self.layers = layers
        self.own, self.ghosts = own, ghosts
        self.cells = own + ghosts
        self.local = {c: i for i, c in enumerate(self.cells)}
        ptr = np.asarray(pm.cell_subtet_ptr)
        sel = [np.arange(ptr[c], ptr[c + 1]) for c in self.cells]
        sub_ptr = np.concatenate([[0], np.cumsum([len(x) for x in sel])]).astype(np.int64)
        idx = np.concatenate(sel)
        vtx = np.asarray(pm.subtet_vtx)[idx]
        shift = None if pm.subtet_shift is None else np.asarray(pm.subtet_shift)[idx]
        if shift is not None:
            for d in range(3):
                params.period[d] = pm.period[d]
        # the ghosts' outer faces are unmatched: a transmissive handle (faces between its cells,
        # periodic images included, are matched by their vertices all the same)
        self.h = _afe.afe_mesh_create(params, pm.xyz, sub_ptr, vtx, shift, _afe.AFE_BC_TRANSMISSIVE, stream)
        self.node_ptr = _afe.afe_node_ptr(self.h, len(self.cells))
        self.n_nodes = int(self.node_ptr[-1])
        self.cfl = float(params.cfl)
        self.N = int(params.order)
        # which of its cells I need from each peer, and which of mine each peer holds as ghosts
        # (the same layer rule applied to the peer), both in index order
        self.recv = {}
        for g in ghosts:
            self.recv.setdefault(int(labels[g]), []).append(g)
        self.send = {}
        mine = set(own)
        for s in range(int(labels.max()) + 1):
            if s != rank:
                theirs = [g for g in ghost_cells(nb, labels, s, layers) if g in mine]
                if theirs:
                    self.send[s] = theirs

    def node_coords(self):
        return self.afe.afe_get_node_coords(self.h)

    def rows(self, cells):
        """Node rows of the given cells (global ids) in this handle's state."""
        return np.concatenate([np.arange(self.node_ptr[self.local[c]], self.node_ptr[self.local[c] + 1])
                               for c in cells]) if cells else np.zeros(0, np.int64)

    def pack(self, state, peer: int) -> np.ndarray:
        """The rows of my cells that `peer` holds as ghosts, from my current state [n_nodes, 5]."""
        return state[self.rows(self.send.get(peer, []))]

    def unpack(self, state, peer: int, buf: np.ndarray):
        """Write `peer`'s rows of my ghost cells into my state (in place)."""
        state[self.rows(self.recv.get(peer, []))] = buf

    def cfl_pieces(self):
        return self.afe.afe_cfl_pieces(self.h, len(self.own))

    def dt_from(self, bracket_max: float, h_min: float) -> float:
        """The global time step from the reduced pieces (the library's own expression)."""
        return self.cfl * h_min / ((2 * self.N + 1) * bracket_max)

    def close(self):
        self.afe.afe_mesh_destroy(self.h)
        self.h = None


def step_ranks_in_process(ranks: List[RankMesh], states: List[np.ndarray], exchange: bool = True):
    """One step of a partitioned mesh whose ranks live in one process (one GPU or several):
    the ghost exchange through host buffers, the reductions of the time step, a step of every
    rank.  `states` holds each rank's host copy of its state (updated).  Returns the dt."""
    afe = ranks[0].afe
    if exchange:
        for r in ranks:
            for s in ranks:
                if s.rank != r.rank and r.rank in s.send:
                    r.unpack(states[r.rank], s.rank, s.pack(states[s.rank], r.rank))
            afe.afe_set_state(r.h, states[r.rank])
    pieces = [r.cfl_pieces() for r in ranks]
    dt = ranks[0].dt_from(max(b for b, _ in pieces), min(h for _, h in pieces))
    status = [afe.afe_step(r.h, dt, check=False) for r in ranks]
    for r in ranks:
        states[r.rank] = afe.afe_get_state(r.h)
    return dt, status


def step_rank_distributed(dist, r: RankMesh, state: np.ndarray, device=None):
    """One step of rank `r` of a partitioned mesh, one process per rank: the ghost exchange
    (isend / recv of host buffers for gloo; with `device` set, of tensors on that device, as
    NCCL needs), the max / min all-reduce of the time step's pieces, the step.  Returns
    (dt, status, state)."""
    afe = r.afe
    peers = sorted(set(r.send) | set(r.recv))
    import torch
    reqs = []
    for s in peers:
        t = torch.from_numpy(np.ascontiguousarray(r.pack(state, s)))
        if device is not None:
            t = t.to(device)
        reqs.append((dist.isend(t, dst=s), t))
    for s in peers:
        n = len(r.rows(r.recv.get(s, [])))
        t = torch.empty((n, 5), dtype=torch.float64, device=device)
        dist.recv(t, src=s)
        r.unpack(state, s, t.cpu().numpy())
    for q, _ in reqs:
        q.wait()
    afe.afe_set_state(r.h, state)
    b, h = r.cfl_pieces()
    b, h = allreduce_max_min(dist, b, h, device)
    dt = r.dt_from(b, h)
    st = afe.afe_step(r.h, dt, check=False)
    return dt, st, afe.afe_get_state(r.h)
