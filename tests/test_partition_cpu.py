"""The cell partition of one mesh over two ranks and its one exchange per step, over gloo (CPU).

Each rank steps only its own cells with the oracle's per-cell pieces (limiter, CFL
reductions, predictor, corrector) and receives everything else through the halo plan of
paper_2605_00619_gb300.partition: the neighbours' cell means before the detector, a max/min
all-reduce for the time step, and the other side's time-integrated predictor and flux (with
its viscosity and length) at the face nodes of every cross-partition sub-triangle before the
Rusanov fluxes.  The result equals the one-rank oracle step bit for bit.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from inputs.voronoi import box_voronoi, periodic_voronoi
from paper_2605_00619_gb300 import partition as P


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("gen,n,parts", [(periodic_voronoi, 3, 2), (box_voronoi, 3, 3), (periodic_voronoi, 4, 4)])
def test_bisection_and_plans_are_consistent(gen, n, parts):
    """Parts differ in size by at most one cell; for every pair of ranks the two plans list the
    same sub-triangles in the same order, each side's cell being the other's partner; the
    cells sent are exactly the neighbours the other side receives."""
    pm = gen(n)
    labels = P.bisect(P.cell_centroids(pm), parts)
    sizes = np.bincount(labels, minlength=parts)
    assert sizes.max() - sizes.min() <= 1 and sizes.sum() == pm.n_cells
    assert np.array_equal(labels, P.bisect(P.cell_centroids(pm), parts))
    plans = [P.halo_plan(pm, labels, r) for r in range(parts)]
    for r, pr in enumerate(plans):
        assert np.array_equal(pr.owned, np.flatnonzero(labels == r))
        for s, peer in pr.peers.items():
            back = plans[s].peers[r]
            assert [k for _, k in peer.tris] == [k for _, k in back.tris]
            assert [c for c, _ in peer.tris] == back.partner_cells
            assert peer.partner_cells == [c for c, _ in back.tris]
            assert peer.send_cells == back.recv_cells and peer.recv_cells == back.send_cells
            assert all(labels[c] == r for c, _ in peer.tris) and all(labels[c] == s for c in peer.partner_cells)
    # every cross-partition sub-triangle appears once per side
    bt = P.boundary_triangles(pm)
    cross = sum(1 for cells in bt.values() if len(cells) == 2 and labels[cells[0]] != labels[cells[1]])
    assert sum(p.n_halo_tris() for p in plans) == 2 * cross


def _partitioned_steps(rank, world, port, case, nsteps, q):
    import torch.distributed as dist

    from inputs import states
    from oracle import scheme
    from oracle.mesh import from_polymesh

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if case == "box-limiter":
            pm = box_voronoi(3)
            prm = scheme.Params(limiter=True, visc_dt_subtet=True)
        else:
            pm = periodic_voronoi(3)
            prm = scheme.Params(mu=0.01, kappa=-1.0)
        N = 2
        om = from_polymesh(pm, N)
        x = om.node_coords()
        u = states.primitive_to_conserved(1.0 + 0.1 * np.sin(3.0 * x.sum(axis=1)), -0.5 * (x - x.mean(axis=0)), 1.0)
        labels = P.bisect(P.cell_centroids(pm), world)
        plan = P.halo_plan(pm, labels, rank)
        own = [int(c) for c in plan.owned]
        # the oracle's boundary sub-triangles of each own cell, by the partition's triangle key
        tri_of = {c: {bt.canon: bt for bt in om.cells[c].bfaces} for c in own}
        Nf = len(om.R.tri_bary)
        ref = om.split(u.copy())
        mine = {c: ref[c].copy() for c in own}
        for _ in range(nsteps):
            ref, info = scheme.step(om, ref, prm)            # the one-rank step, for comparison
            # limiter: own means, the neighbours' from their ranks
            ub = {c: om.cells[c].wvec @ mine[c] / om.cells[c].vol for c in own}
            mu_c, kap = {}, {}
            if prm.limiter:
                send = {s: np.array([ub[c] for c in p.send_cells]) for s, p in plan.peers.items()}
                got = P.exchange(dist, plan, send, {s: (len(p.recv_cells), 5) for s, p in plan.peers.items()})
                for s, p in plan.peers.items():
                    ub.update({c: got[s][i] for i, c in enumerate(p.recv_cells)})
                for c in own:
                    _, mu_c[c] = scheme.limiter_cell(om, c, ub, prm)
            else:
                mu_c = {c: prm.mu for c in own}
            kap = {c: scheme.cell_kappa(mu_c[c], prm) for c in own}
            # time step: two reductions over all ranks
            mu_full = np.zeros(om.n_cells)
            for c in own:
                mu_full[c] = mu_c[c]
            worst, h_min = scheme.cfl_pieces(om, mine, mu_full, prm, own)
            worst, h_min = P.allreduce_max_min(dist, worst, h_min)
            dt = scheme.cfl_from_pieces(om, worst, h_min, prm)
            assert dt == info.dt
            # predictors of the own cells only
            pred = {}
            for c in own:
                qn, _ = scheme.predictor(om, c, mine[c], dt, mu_c[c], kap[c], prm)
                pred[c] = scheme.time_integrate(om, c, qn, dt, mu_c[c], kap[c], prm)
            # the exchange before the Rusanov fluxes: per cross-partition sub-triangle the face-node
            # q_bar [Nf, 5] and F_bar [Nf, 3, 5] of its side, and the cell's h, mu, kappa
            send = {}
            for s, p in plan.peers.items():
                rows = []
                for c, key in p.tris:
                    bt = tri_of[c][key]
                    qb, Fb = pred[c]
                    rows.append(np.concatenate([qb[bt.nodes].ravel(), Fb[bt.k][bt.local].ravel(),
                                                [scheme.cell_length(om.cells[c], prm), mu_c[c], kap[c]]]))
                send[s] = np.array(rows)
            width = Nf * 5 + Nf * 15 + 3
            got = P.exchange(dist, plan, send, {s: (len(p.tris), width) for s, p in plan.peers.items()})
            remote = {}
            for s, p in plan.peers.items():
                for i, (c, key) in enumerate(p.tris):
                    row = got[s][i]
                    remote[(c, key)] = (row[:Nf * 5].reshape(Nf, 5), row[Nf * 5:Nf * 20].reshape(Nf, 3, 5),
                                        row[-3], row[-2], row[-1])
            new = {}
            for c in own:
                def outer(bt, c=c):
                    if labels[bt.nbr] != rank:
                        return remote[(c, bt.canon)]
                    nb = om.cells[bt.nbr].bfaces[bt.nbr_tri]
                    qj, Fj = pred[bt.nbr]
                    return (qj[nb.nodes], Fj[nb.k][nb.local], scheme.cell_length(om.cells[bt.nbr], prm),
                            mu_c[bt.nbr], kap[bt.nbr])
                new[c] = scheme.corrector_cell(om, c, mine[c], pred[c][0], pred[c][1], outer, dt, mu_c[c], kap[c], prm)
            mine = new
        same = all(np.array_equal(mine[c], ref[c]) for c in own)
        q.put((rank, same, len(own), plan.n_halo_tris()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("box-limiter", 2), ("periodic-ns", 2)])
def test_two_rank_partitioned_step_equals_one_rank_oracle(case, world):
    pytest.importorskip("torch.distributed")
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_partitioned_steps, args=(r, world, port, case, 2, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert all(same for _, same, _, _ in res), res
    assert sum(n for _, _, n, _ in res) == 27 and all(h > 0 for _, _, _, h in res)


@pytest.mark.parametrize("layers", [1, 2])
def test_ghost_layers_and_send_lists(layers):
    """The ghost layers of every rank and the send lists its peers derive from the same rule
    agree: what rank s holds as ghosts from rank r is what r sends to s."""
    pm = periodic_voronoi(4)
    labels = P.bisect(P.cell_centroids(pm), 3)
    nb = P.cell_neighbours(pm)
    ghosts = {r: P.ghost_cells(nb, labels, r, layers) for r in range(3)}
    for r in range(3):
        own = set(np.flatnonzero(labels == r).tolist())
        g = ghosts[r]
        assert not (own & set(g)) and len(g) == len(set(g))
        # layer 1 is exactly the off-rank face neighbours of the own cells
        layer1 = {j for c in own for j in nb[c]} - own
        assert layer1 <= set(g)
        if layers == 1:
            assert set(g) == layer1
    assert all(len(v) > 0 for v in nb)
