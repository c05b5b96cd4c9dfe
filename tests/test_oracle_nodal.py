"""Pins of the oracle's nodal velocity (reading R15: a velocity given at the Gauss nodes, the
containing element's interpolant, linear in time, averaged on faces), against analytic fields
and the other velocity kinds."""
import numpy as np

from oracle import sl_oracle as O


def field_1d(setup, f0, f1=None, t0=0.0, t1=1.0):
    X = O.node_coords_1d(setup)
    return O.NodalField(setup, t0, t1, f0(X), (f1 or f0)(X))


def field_2d(setup, fu, fv, t0=0.0, t1=1.0):
    X = np.zeros((setup.ky, setup.kx, setup.n, setup.n))
    Y = np.zeros_like(X)
    for ey in range(setup.ky):
        for ex in range(setup.kx):
            X[ey, ex], Y[ey, ex] = O.node_coords_2d(setup, ex, ey)
    return O.NodalField(setup, t0, t1, fu(X, Y), fu(X, Y), fv(X, Y), fv(X, Y))


def test_polynomial_field_is_reproduced_1d():
    """Degree n-1 data: the interpolant is the polynomial itself, inside, on faces and (extrapolated)
    outside a non-periodic domain; the divergence is its derivative."""
    s = O.Setup(1, 5, 1, (-0.5, 1.5, 0, 0), 5, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 4, 0.0)
    p = lambda x: 0.3 + 0.5 * x - 0.2 * x ** 2 + 0.05 * x ** 4
    dp = lambda x: 0.5 - 0.4 * x + 0.2 * x ** 3
    f = field_1d(s, p)
    xq = np.concatenate([np.linspace(-0.7, 1.7, 41), -0.5 + 0.4 * np.arange(6)])   # faces too
    u, v, dv = O.nodal_velocity(f, xq, None, 0.4)
    assert np.max(np.abs(u - p(xq))) < 1e-13
    assert np.max(np.abs(dv - dp(xq))) < 1e-12
    assert np.all(v == 0.0)


def test_rotation_samples_are_reproduced_2d():
    """A linear field (solid-body rotation) sampled at the nodes is the rotation everywhere,
    divergence zero."""
    s = O.Setup(2, 3, 4, (0.0, 1.0, 0.0, 1.0), 4, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 4, 0.0)
    om, cx, cy = 2 * np.pi, 0.5, 0.45
    f = field_2d(s, lambda x, y: -om * (y - cy), lambda x, y: om * (x - cx))
    rng = np.random.default_rng(3)
    xq = np.concatenate([rng.uniform(-0.1, 1.1, 40), np.array([1 / 3, 2 / 3, 0.0, 0.5])])
    yq = np.concatenate([rng.uniform(-0.1, 1.1, 40), np.array([0.5, 0.25, 0.75, 0.5])])
    u, v, dv = O.nodal_velocity(f, xq, yq, 0.2)
    assert np.max(np.abs(u + om * (yq - cy))) < 1e-12
    assert np.max(np.abs(v - om * (xq - cx))) < 1e-12
    assert np.max(np.abs(dv)) < 1e-11


def test_linear_in_time():
    s = O.Setup(1, 3, 1, (0.0, 1.0, 0, 0), 4, O.GAUSS_LEGENDRE, (O.BC_PERIODIC,) * 4, 0.0)
    f = field_1d(s, lambda x: 0.0 * x + 0.8, lambda x: 0.0 * x - 0.4, t0=2.0, t1=2.5)
    for th in (0.0, 0.25, 0.5, 1.0):
        u, _, dv = O.nodal_velocity(f, np.array([0.1, 0.5, 1 / 3]), None, 2.0 + 0.5 * th)
        assert np.allclose(u, (1 - th) * 0.8 + th * (-0.4), rtol=0, atol=1e-15)
        assert np.allclose(dv, 0.0, atol=1e-13)


def test_faces_average_the_elements_sharing_them():
    """Element-wise constant data c_k: c_k inside element k, (c_{k-1} + c_k) / 2 on an interior
    face, the wrap partner's value averaged in on a periodic domain face, and the boundary
    element alone on a non-periodic one (and beyond it)."""
    K = 4
    c = np.array([1.0, 3.0, -2.0, 0.5])
    for bc in (O.BC_PERIODIC, O.BC_INFLOW):
        s = O.Setup(1, K, 1, (0.0, 2.0, 0, 0), 3, O.GAUSS_LEGENDRE, (bc,) * 4, 0.0)
        f = O.NodalField(s, 0.0, 1.0, np.repeat(c[:, None], 3, 1), np.repeat(c[:, None], 3, 1))
        u, _, _ = O.nodal_velocity(f, np.array([0.25, 0.75, 1.25, 1.75, 0.5, 1.0, 1.5]), None, 0.0)
        assert np.allclose(u, [1.0, 3.0, -2.0, 0.5, 2.0, 0.5, -0.75], atol=1e-15)
        u, _, _ = O.nodal_velocity(f, np.array([0.0, 2.0, -0.25, 2.25]), None, 0.0)
        if bc == O.BC_PERIODIC:
            assert np.allclose(u, [0.75, 0.75, 0.5, 1.0], atol=1e-15)
        else:
            assert np.allclose(u, [1.0, 0.5, 1.0, 0.5], atol=1e-15)


def test_constant_nodal_field_steps_like_const():
    """A constant nodal field gives the constant-velocity step (1D and 2D, mass and energy rows)."""
    s = O.Setup(1, 6, 1, (0.0, 1.0, 0, 0), 6, O.GAUSS_LEGENDRE, (O.BC_PERIODIC,) * 4, 0.0)
    X = O.node_coords_1d(s)
    phi = 1.0 + 0.4 * np.sin(2 * np.pi * X) + 0.1 * np.cos(6 * np.pi * X)
    vc = O.Vel(O.VEL_CONST, (0.7, 0, 0, 0, 0, 0))
    dt = O.max_dt(s, vc, rule="paper")
    vn = O.Vel(O.VEL_NODAL, (), field_1d(s, lambda x: 0.0 * x + 0.7, t0=0.1, t1=0.1 + dt))
    for cons in (1, 3, 7):
        a, _ = O.step_1d(s, phi, O.StepOpts(vc, 0.1, dt, cons, 4))
        b, _ = O.step_1d(s, phi, O.StepOpts(vn, 0.1, dt, cons, 4))
        assert np.max(np.abs(a - b)) < 1e-13
    s2 = O.Setup(2, 3, 3, (0.0, 1.0, 0.0, 1.0), 5, O.GAUSS_LEGENDRE, (O.BC_PERIODIC,) * 4, 0.0)
    ph2 = np.zeros((3, 3, 5, 5))
    for ey in range(3):
        for ex in range(3):
            x, y = O.node_coords_2d(s2, ex, ey)
            ph2[ey, ex] = 1.0 + 0.3 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    vc2 = O.Vel(O.VEL_CONST, (0.6, -0.3, 0, 0, 0, 0))
    dt2 = O.max_dt(s2, vc2, rule="paper")
    f2 = field_2d(s2, lambda x, y: 0.0 * x + 0.6, lambda x, y: 0.0 * x - 0.3, t0=0.0, t1=dt2)
    vn2 = O.Vel(O.VEL_NODAL, (), f2)
    a, _ = O.step_2d(s2, ph2, O.StepOpts(vc2, 0.0, dt2, 3, 4))
    b, _ = O.step_2d(s2, ph2, O.StepOpts(vn2, 0.0, dt2, 3, 4))
    assert np.max(np.abs(a - b)) < 1e-12


def test_rotation_nodal_field_steps_like_rotation():
    """Nodal samples of the solid-body rotation give the rotation step: a linear field is exact."""
    s = O.Setup(2, 3, 3, (0.0, 1.0, 0.0, 1.0), 5, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 4, 0.1)
    ph = np.zeros((3, 3, 5, 5))
    for ey in range(3):
        for ex in range(3):
            x, y = O.node_coords_2d(s, ex, ey)
            ph[ey, ex] = np.exp(-((x - 0.4) ** 2 + (y - 0.5) ** 2) / 0.05)
    om = 2 * np.pi
    vr = O.Vel(O.VEL_ROTATION, (om, 0.5, 0.5, 0, 0, 0))
    dt = O.max_dt(s, vr, rule="paper")
    vn = O.Vel(O.VEL_NODAL, (), field_2d(s, lambda x, y: -om * (y - 0.5), lambda x, y: om * (x - 0.5), 0.2,
                                         0.2 + dt))
    a, _ = O.step_2d(s, ph, O.StepOpts(vr, 0.2, dt, 3, 4))
    b, _ = O.step_2d(s, ph, O.StepOpts(vn, 0.2, dt, 3, 4))
    assert np.max(np.abs(a - b)) < 1e-12


def test_sinx_nodal_field_steps_like_sinx():
    """u = -sin x sampled at 12 nodes per element: the step follows the analytic u = -sin x step
    (Sec. 5.2) to the interpolation error, divergence term included (dropping it, or its sign,
    changes the step by about dt |cos x| ~ 1e-2)."""
    s = O.Setup(1, 4, 1, (0.0, 2 * np.pi, 0, 0), 12, O.CHEB_GAUSS, (O.BC_PERIODIC,) * 4, 0.0)
    X = O.node_coords_1d(s)
    phi = 1.0 + 0.2 * np.cos(X)
    vs = O.Vel(O.VEL_SINX, (0, 0, 0, 0, 0, 0))
    dt = O.max_dt(s, vs, rule="paper")
    vn = O.Vel(O.VEL_NODAL, (), field_1d(s, lambda x: -np.sin(x), t0=0.0, t1=dt))
    for cons in (1, 3):
        a, _ = O.step_1d(s, phi, O.StepOpts(vs, 0.0, dt, cons, 4, O.FIT_SOFT))
        b, _ = O.step_1d(s, phi, O.StepOpts(vn, 0.0, dt, cons, 4, O.FIT_SOFT))
        assert np.max(np.abs(a - b)) < 1e-9, np.max(np.abs(a - b))
