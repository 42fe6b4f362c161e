"""The workloads' initial data satisfy what defines them (CPU only)."""
import math

import numpy as np

from inputs import states


def test_isentropic_vortex_is_an_exact_steady_euler_state():
    """Isentropic (p = rho^gamma), divergence-free, and in radial balance
    dp/dr = rho v_theta^2 / r (by central differences along a ray); the travelling form is
    the steady form shifted by vel t; far from the axis it is the background state."""
    g = states.GAMMA
    r = np.linspace(0.05, 4.0, 400)
    h = 1e-5
    ray = lambda rr: np.stack([5.0 + rr, np.full_like(rr, 5.0), np.full_like(rr, 2.0)], axis=1)  # noqa: E731
    q = states.isentropic_vortex(ray(r))
    rho, v, p = q[:, 0], q[:, 1:4] / q[:, :1], (g - 1.0) * (q[:, 4] - 0.5 * np.sum(q[:, 1:4] ** 2, 1) / q[:, 0])
    np.testing.assert_allclose(p, rho ** g, rtol=1e-13)
    assert np.abs(v[:, 0]).max() < 1e-15 and np.abs(v[:, 2]).max() == 0.0  # swirl is tangential on the ray
    qp, qm = states.isentropic_vortex(ray(r + h)), states.isentropic_vortex(ray(r - h))
    pres = lambda qq: (g - 1.0) * (qq[:, 4] - 0.5 * np.sum(qq[:, 1:4] ** 2, 1) / qq[:, 0])  # noqa: E731
    dpdr = (pres(qp) - pres(qm)) / (2 * h)
    np.testing.assert_allclose(dpdr, rho * v[:, 1] ** 2 / r, rtol=1e-6, atol=1e-9)
    # divergence of the swirl by central differences at scattered points
    rng = np.random.default_rng(3)
    x = rng.uniform(2.0, 8.0, size=(50, 3))
    div = 0.0
    for d in range(2):
        e = np.zeros(3)
        e[d] = h
        up, um = states.isentropic_vortex(x + e), states.isentropic_vortex(x - e)
        div = div + (up[:, 1 + d] / up[:, 0] - um[:, 1 + d] / um[:, 0]) / (2 * h)
    assert np.abs(div).max() < 1e-8
    # travelling form = steady form shifted; background far away
    vel = (1.0, 1.0, 0.0)
    xs = rng.uniform(0.0, 10.0, size=(30, 3))
    a = states.isentropic_vortex(xs, t=0.7, vel=vel)
    b = states.isentropic_vortex(xs - 0.7 * np.array(vel), vel=vel)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    far = states.isentropic_vortex(np.array([[0.0, 0.0, 0.0]]))
    np.testing.assert_allclose(far[0], [1, 0, 0, 0, 1.0 / (g - 1.0)], atol=1e-9)
    # peak temperature drop at the axis
    ax = states.isentropic_vortex(np.array([[5.0, 5.0, 1.0]]))
    T = (g - 1.0) * (ax[0, 4] - 0.0) / ax[0, 0]
    assert math.isclose(T, 1.0 - (g - 1.0) * 25.0 / (8.0 * g * math.pi ** 2) * math.e, rel_tol=1e-13)


def test_shear_layers_closed_form():
    """At t the shear profile equals the initial one with the jump width grown as
    2 sqrt(nu (t + t0)); the mean velocity over a period is zero."""
    nu = 1e-3
    x = np.zeros((2000, 3))
    x[:, 0] = (np.arange(2000) + 0.5) / 2000
    q0 = states.shear_layers(x, nu, t=0.0, t0=0.25)
    q1 = states.shear_layers(x, nu, t=0.2, t0=0.05)
    np.testing.assert_allclose(q0, q1, atol=1e-15)
    assert abs(q0[:, 2].mean()) < 1e-12
    assert q0[:, 2].max() <= 0.1 and q0[:, 2].min() >= -0.1
