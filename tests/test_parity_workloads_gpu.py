"""GPU parity on the paper's own smooth test problems (Sec. 5): the travelling isentropic
vortex (Sec. 5.1) in both forms and the first problem of Stokes (two shear layers, the
viscous tests of Sec. 5) in the FP64 form, against the oracle on the same seeded inputs.

The vortex is two-dimensional (w = 0, and it stays zero up to round-off), so the momentum is
compared as one vector field, normalised by the largest momentum magnitude, rather than per
component (a component that is zero up to round-off has no scale of its own).  Bars: FP64
relative L-infinity <= 1e-11, FP32 relative L2 <= 1e-5, as in the other parity tests."""
import numpy as np
import pytest

from inputs import states
from inputs.voronoi import periodic_voronoi
from tests.harness import Pair, rel_l2_fields

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def afe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_00619_gb300 import afe as mod
    mod.lib()
    return mod


def rel_linf_fields(a, b):
    """max of the relative L-infinity errors of the density, the momentum vector field and the
    total energy, each normalised by the largest magnitude of that field in b"""
    def rel(x, y):
        return np.abs(x - y).max() / max(np.abs(y).max(), 1e-300)
    mom = np.linalg.norm(a[:, 1:4] - b[:, 1:4], axis=1).max() / max(np.linalg.norm(b[:, 1:4], axis=1).max(), 1e-300)
    return max(rel(a[:, 0], b[:, 0]), mom, rel(a[:, 4], b[:, 4]))


def _steps(pr, n):
    for _ in range(n):
        pr.oracle_step()
        assert pr.lib_step() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_travelling_vortex(afe, prec):
    """Sec. 5.1's vortex moving with u = (1, 1, 0) on the periodic box [0, 10)^3, N = 2."""
    pm = periodic_voronoi(3, L=10.0)
    kw = {"precision": afe.AFE_FP32, "picard_tol": 1e-6, "picard_max": 128} if prec == "fp32" else {}
    p = afe.afe_default_params(2, cfl=0.3, **kw)
    pr = Pair(pm, p)
    pr.set_state(states.isentropic_vortex(pr.om.node_coords(), vel=(1.0, 1.0, 0.0)))
    _steps(pr, 3)
    if prec == "fp64":
        assert rel_linf_fields(pr.lib_state(), pr.u) <= FP64_TOL
    else:
        assert rel_l2_fields(pr.lib_state(), pr.u) <= FP32_TOL
    pr.close()


def test_stokes_shear_layers_navier_stokes(afe):
    """Two shear layers (rho = 1, p = 1/gamma, v(x) with diffused jumps) with mu = 0.01, N = 2."""
    pm = periodic_voronoi(3)
    p = afe.afe_default_params(2, equations=afe.AFE_NAVIER_STOKES, mu=0.01, kappa=-1.0, Pr=0.71, cfl=0.3)
    pr = Pair(pm, p)
    pr.set_state(states.shear_layers(pr.om.node_coords(), nu=0.01))
    _steps(pr, 2)
    assert rel_linf_fields(pr.lib_state(), pr.u) <= FP64_TOL
    pr.close()
