"""GPU parity of the reduced-precision (FP32) form against the FP64 oracle on the paths the
density-wave test does not reach: viscous fluxes, the artificial-viscosity limiter, cells
large enough for the predictor's narrow chunks and one-stage M_i^-1 ring, cells too large
for the shared-memory plan (the global-scratch kernel), and the bounded-wait failure path.

Bar: relative L2 <= 1e-5 per conserved variable after the stated steps (the reduced-
precision tolerance), with the momentum compared as one vector field where a component
vanishes initially; the path each case takes is asserted from afe_plan_info.
"""
import math

import numpy as np
import pytest

from inputs import states
from inputs.lattice import split_cube_lattice
from inputs.voronoi import box_voronoi, periodic_voronoi
from tests.harness import Pair, rel_l2, rel_l2_fields

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def afe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_00619_gb300 import afe as mod
    mod.lib()
    return mod


def _fp32(afe, N, **kw):
    return afe.afe_default_params(N, precision=afe.AFE_FP32, picard_tol=1e-6, picard_max=128, **kw)


def _steps(pr, n, allowed=(0,)):
    infos = []
    for _ in range(n):
        info = pr.oracle_step()
        st = pr.lib_step(info.dt, check=False)
        assert st in allowed, pr.afe.afe_last_error()
        infos.append(info)
    return infos


@pytest.mark.parametrize("variant", [0, 1])
def test_fp32_navier_stokes_against_the_oracle(afe, variant):
    """Navier-Stokes Taylor-Green data (mu 0.005, kappa from Pr): the FP32 viscous flux with
    per-sub-tet gradients in the predictor and the face-node fluxes (both forms of the
    M_i^-1 apply)."""
    pm = periodic_voronoi(2)
    p = _fp32(afe, 2, equations=afe.AFE_NAVIER_STOKES, mu=0.005, kappa=-1.0, Pr=0.71)
    pr = Pair(pm, p)
    afe.afe_set_predictor_variant(pr.h, variant)
    assert afe.afe_plan_info(pr.h).fp32_shared == 1 and afe.afe_plan_info(pr.h).tcgen05 == variant
    pr.set_state(states.taylor_green_3d(2 * math.pi * pr.om.node_coords(), p0=10.0))
    _steps(pr, 3)
    # w vanishes at t = 0: the momentum is compared as one vector field
    assert rel_l2_fields(pr.lib_state(), pr.u) <= FP32_TOL
    pr.close()


def test_fp32_limiter_against_the_oracle(afe):
    """Converging flow v = -(x - x0) on a box mesh with the limiter: the detector flags the
    compressed cells (beta_i > 0), whose artificial viscosity mu_i > 0 runs the FP32 viscous
    flux inside an Euler problem."""
    pm = box_voronoi(3)
    p = _fp32(afe, 2, limiter=1, visc_dt_subtet=1)
    pr = Pair(pm, p)
    x = pr.om.node_coords()
    pr.set_state(states.primitive_to_conserved(1.0 + 0.1 * np.sin(x.sum(axis=1)), -(x - x.mean(axis=0)), 1.0))
    infos = _steps(pr, 3, allowed=(0, 5))
    assert max(info.beta.max() for info in infos) > 0.0
    _, _, beta, mu = afe.afe_get_diagnostics(pr.h, pm.n_cells, qbar=False)
    assert (beta > 0).sum() > 0
    np.testing.assert_allclose(beta, infos[-1].beta, rtol=0, atol=1e-4)
    assert rel_l2(pr.lib_state(), pr.u) <= FP32_TOL
    pr.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_fp32_large_cells_take_narrow_chunks_and_a_one_stage_ring(afe, variant):
    """Two cubes whose edges are split (4, 4, 3): 88 sub-tets and 623 nodes per cell at N = 3.
    The mma.sync form (variant 0) takes 8-sub-tet chunks and a single 32-row stage of M_i^-1;
    the tensor-memory form (variant 1, five 128-row tiles, single-buffered tensor memory)
    takes a single 8-row stage.  623 is not a multiple of either, so the last stage is
    partial."""
    pm = split_cube_lattice((2, 1, 1), (4, 4, 3), d=0.5)
    p = _fp32(afe, 3)
    pr = Pair(pm, p)
    afe.afe_set_predictor_variant(pr.h, variant)
    plan = afe.afe_plan_info(pr.h)
    print(f"plan variant {variant}: tcgen05 {plan.tcgen05} smem {plan.smem_bytes} ring {plan.ring_min}-"
          f"{plan.ring_max} rows {plan.stage_rows_min} narrow {plan.narrow_cells} masked {plan.masked_cells}")
    assert plan.fp32_shared == 1 and plan.max_nodes == 623 and plan.max_subtets == 88
    assert plan.tcgen05 == variant
    assert plan.ring_min == 1 and plan.masked_cells == 2
    if variant == 0:  # q and RHS rows leave too little room for 16-sub-tet chunks
        assert plan.narrow_cells == 2 and plan.stage_rows_min == 32
    else:  # no RHS rows, but the two-part right-hand-side operand leaves room for 8-row stages only
        assert plan.narrow_cells == 0 and plan.stage_rows_min == 8
    x = pr.om.node_coords()
    pr.set_state(states.density_wave(x, amp=0.1, vel=(0.5, -0.3, 0.2)))
    _steps(pr, 3)
    assert rel_l2(pr.lib_state(), pr.u) <= FP32_TOL
    pr.close()


def test_fp32_cells_beyond_the_shared_memory_plan(afe):
    """A cube with every edge split in four: 96 sub-tets and 679 nodes at N = 3, beyond the
    640 nodes of the shared-memory predictor; the FP32 form runs its global-scratch kernel
    on the CUDA cores and still meets the reduced-precision bar."""
    pm = split_cube_lattice((2, 1, 1), (4, 4, 4), d=0.5)
    p = _fp32(afe, 3)
    pr = Pair(pm, p)
    plan = afe.afe_plan_info(pr.h)
    assert plan.max_nodes == 679 and plan.fp32_shared == 0 and plan.corrector_block == 1
    pr.set_state(states.density_wave(pr.om.node_coords(), amp=0.1, vel=(0.5, -0.3, 0.2)))
    _steps(pr, 2)
    assert rel_l2(pr.lib_state(), pr.u) <= FP32_TOL
    pr.close()


def test_plan_report_of_a_voronoi_mesh(afe):
    pm = periodic_voronoi(3)
    h = afe.create_from_polymesh(pm, _fp32(afe, 3))
    plan = afe.afe_plan_info(h)
    ptr = afe.afe_node_ptr(h, pm.n_cells)
    Ni = np.diff(ptr)
    assert plan.fp32_shared == 1 and plan.max_nodes == Ni.max() and plan.tcgen05 == 0
    assert 1 <= plan.ring_min <= plan.ring_max <= 8
    assert plan.stage_rows_min == 32 and plan.narrow_cells == 0
    assert plan.masked_cells == int(np.sum(Ni % 32 != 0))
    afe.afe_set_predictor_variant(h, 1)
    plan = afe.afe_plan_info(h)
    assert plan.tcgen05 == 1 and 1 <= plan.ring_min <= plan.ring_max <= 8
    assert plan.masked_cells == int(np.sum(Ni % plan.stage_rows_min != 0)) and plan.narrow_cells == 0
    with pytest.raises(afe.AfeError):
        afe.afe_set_predictor_variant(h, 2)
    afe.afe_mesh_destroy(h)
    h = afe.create_from_polymesh(pm, afe.afe_default_params(3))
    assert afe.afe_plan_info(h).fp32_shared == 0 and afe.afe_plan_info(h).smem_bytes == 0
    afe.afe_mesh_destroy(h)


def test_bounded_wait_gives_up_and_reports_timeout(afe):
    """The predictor's first wait per cell limited to zero polls gives up at once: every
    block waits (with the normal limit) for the copy it issued and leaves, the step reports
    AFE_ETIMEOUT, and the device stays usable -- a fresh handle then steps and matches the
    oracle."""
    pm = periodic_voronoi(2)
    p = _fp32(afe, 2)
    h = afe.create_from_polymesh(pm, p)
    afe.afe_set_state(h, states.density_wave(afe.afe_get_node_coords(h)))
    afe.afe_set_wait_limit(h, 0)
    assert afe.afe_step(h, 0.0, check=False) == afe.AFE_ETIMEOUT
    assert "bounded wait" in afe.afe_last_error()
    with pytest.raises(afe.AfeError):
        afe.afe_set_wait_limit(h, -1)
    afe.afe_mesh_destroy(h)
    pr = Pair(pm, p)
    pr.set_state(states.density_wave(pr.om.node_coords()))
    _steps(pr, 2)
    assert rel_l2(pr.lib_state(), pr.u) <= FP32_TOL
    pr.close()


@pytest.mark.parametrize("N", [1, 2, 3])
def test_tensor_memory_and_mma_sync_forms_agree(afe, N):
    """The two forms of the M_i^-1 apply (tcgen05 with tensor memory, and mma.sync) compute the
    same 3xTF32 product: after 3 steps of the density wave they agree to FP32 rounding, and
    each meets the oracle bar."""
    pm = periodic_voronoi(3 if N < 3 else 2)
    p = _fp32(afe, N)
    pr = Pair(pm, p)
    h1 = afe.create_from_polymesh(pm, p)
    afe.afe_set_predictor_variant(pr.h, 1)
    assert afe.afe_plan_info(pr.h).tcgen05 == 1 and afe.afe_plan_info(h1).tcgen05 == 0
    u0 = states.density_wave(pr.om.node_coords())
    pr.set_state(u0)
    afe.afe_set_state(h1, u0[pr.perm])
    for _ in range(3):
        info = pr.oracle_step()
        assert pr.lib_step(info.dt) == 0
        assert afe.afe_step(h1, info.dt) == 0
    a = pr.lib_state()
    b = np.empty_like(a)
    b[pr.perm] = afe.afe_get_state(h1)
    assert rel_l2(a, b) <= 1e-6
    assert rel_l2(a, pr.u) <= FP32_TOL and rel_l2(b, pr.u) <= FP32_TOL
    afe.afe_mesh_destroy(h1)
    pr.close()
