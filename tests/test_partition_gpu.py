"""The library side of a partitioned mesh on one GPU: each rank's handle holds its own cells
and ghost-cell layers, the ghosts' states come from their owners, the time step is reduced
over the ranks (afe_cfl_pieces), and the own cells then equal the one-handle step of the
whole mesh.  Both ranks live in this process and step one after the other (no kernel of one
waits on the other); the exchange goes through host buffers, the same packing the
one-process-per-rank path sends with torch.distributed.
"""
import numpy as np
import pytest

from inputs import states
from inputs.voronoi import box_voronoi, periodic_voronoi
from paper_2605_00619_gb300 import partition as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_00619_gb300 import afe as mod
    mod.lib()
    return mod


def _params(afe, case):
    if case == "box-limiter-fp64":
        return afe.afe_default_params(2, limiter=1, visc_dt_subtet=1)
    if case == "periodic-fp32":
        return afe.afe_default_params(2, precision=afe.AFE_FP32, picard_tol=1e-6, picard_max=128)
    return afe.afe_default_params(2)


def _ic(x, case):
    if case == "box-limiter-fp64":  # converging flow: the detector flags cells
        return states.primitive_to_conserved(1.0 + 0.1 * np.sin(x.sum(axis=1)), -(x - x.mean(axis=0)), 1.0)
    return states.density_wave(x)


@pytest.mark.parametrize("case,parts", [("periodic-fp64", 2), ("box-limiter-fp64", 2), ("periodic-fp32", 2),
                                        ("periodic-fp64", 3)])
def test_partitioned_handles_equal_the_one_mesh_step(afe, case, parts):
    pm = box_voronoi(3) if case.startswith("box") else periodic_voronoi(3)
    labels = P.bisect(P.cell_centroids(pm), parts)
    ranks = [P.RankMesh(pm, labels, r, _params(afe, case)) for r in range(parts)]
    ref = afe.create_from_polymesh(pm, _params(afe, case))
    xr = afe.afe_get_node_coords(ref)
    ref_ptr = afe.afe_node_ptr(ref, pm.n_cells)
    afe.afe_set_state(ref, _ic(xr, case))
    st = []
    for r in ranks:
        x = r.node_coords()
        afe.afe_set_state(r.h, _ic(x, case))
        # the own cells' nodes come in the one-mesh handle's order
        for c in r.own:
            np.testing.assert_allclose(x[r.rows([c])], xr[ref_ptr[c]:ref_ptr[c + 1]], rtol=0, atol=1e-14)
        st.append(afe.afe_get_state(r.h))
        assert sum(len(v) for v in r.send.values()) > 0 and len(r.ghosts) > 0
    # every ghost of one rank is sent by its owner
    for r in ranks:
        for s, cells in r.recv.items():
            assert ranks[s].send[r.rank] == cells
    fp64 = not case.endswith("fp32")
    for _ in range(4):
        dt, status = P.step_ranks_in_process(ranks, st)
        assert all(x in (0, afe.AFE_ENOCONV) for x in status)
        assert afe.afe_step(ref, 0.0, check=False) in (0, afe.AFE_ENOCONV)
        assert abs(dt - afe.afe_get_stats(ref).dt) <= 1e-13 * dt
    q = afe.afe_get_state(ref)
    scale = np.abs(q).max(axis=0)
    worst = 0.0
    for r in ranks:
        for c in r.own:
            d = np.abs(st[r.rank][r.rows([c])] - q[ref_ptr[c]:ref_ptr[c + 1]]) / scale
            worst = max(worst, float(d.max()))
    assert worst <= (1e-12 if fp64 else 1e-6), worst
    for r in ranks:
        r.close()
    afe.afe_mesh_destroy(ref)


def test_cfl_pieces_rejects_bad_counts(afe):
    pm = periodic_voronoi(2)
    h = afe.create_from_polymesh(pm, afe.afe_default_params(1))
    afe.afe_set_state(h, states.density_wave(afe.afe_get_node_coords(h)))
    b, hm = afe.afe_cfl_pieces(h, pm.n_cells)
    dt = afe.afe_compute_dt(h)
    assert dt == 0.3 * hm / (3 * b)
    for n in (0, pm.n_cells + 1):
        with pytest.raises(afe.AfeError):
            afe.afe_cfl_pieces(h, n)
    afe.afe_mesh_destroy(h)
