"""Pins of the 3D tensor-product oracle (oracle/sl_oracle3d.py; Sec. 3 eq. 3.4 with the step of
Sec. 4), each against mathematics the paper fixes, not against the oracle's own formulas:
exact translation of polynomial data under constant velocity (boundary rows, hard and soft fit,
and with the mass row where the RK4 flux quadrature is exact), the constant-velocity remap as
the element's own polynomial shifted back, the rank of the face rows (the boundary nodes of an
n^3 grid), uniqueness of the interface values (eq. 4.12a) and upwind locality (which catches a
reversed upwind rule that exact translation cannot see), global mass telescoping on a periodic
box, and the RK step against the exact rotation."""
import numpy as np
import pytest

import sl_inputs
from oracle import sl_oracle as O
from oracle import sl_oracle3d as O3

A, B, C = 0.6, -0.4, 0.3


def poly(x, y, z):
    """Degree <= 3 in each direction (and a cubic in total where the mass flux needs it)."""
    return 1.0 + 0.5 * x - 0.3 * y ** 2 + 0.2 * x * y * z + 0.4 * z ** 3 - 0.1 * x ** 2 * y


def translated(t0):
    return lambda x, y, z, t: poly(np.asarray(x) - A * (t - t0), np.asarray(y) - B * (t - t0),
                                   np.asarray(z) - C * (t - t0))


@pytest.mark.parametrize("cons,fit", [(O.C_BOUNDARY, O.FIT_HARD), (O.C_BOUNDARY, O.FIT_SOFT),
                                      (O.C_BOUNDARY | O.C_MASS, O.FIT_HARD)])
def test_exact_translation_of_polynomial_data(cons, fit):
    t0 = 0.2
    s = O3.Setup3(2, 2, 2, (0.0, 1.0, -0.5, 0.5, 0.0, 1.0), 4, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 6,
                  translated(t0))
    vel = O3.Vel3(O.VEL_CONST, (A, B, C))
    dt = O3.max_dt3(s, vel)
    phi = O3.project_3d(s, poly)
    out, infos = O3.step_3d(s, phi, O3.StepOpts3(vel, t0, dt, cons, 4, fit))
    exact = O3.project_3d(s, lambda x, y, z: translated(t0)(x, y, z, t0 + dt))
    assert np.max(np.abs(out - exact)) < 1e-12, np.max(np.abs(out - exact))
    assert all(i["converged"] for i in infos.values())


def test_constant_velocity_remap_is_the_shifted_polynomial():
    """With constant velocity the particles carry phi^n to x + u dt, so the collocation polynomial
    is phi^n's own polynomial shifted: at the nodes, phi^n evaluated at x - u dt."""
    s = O3.Setup3(1, 1, 1, (0.0, 1.0, 0.0, 1.0, 0.0, 1.0), 5, O.GAUSS_LEGENDRE)
    rng = np.random.default_rng(4)
    phi = rng.uniform(-1, 1, (1, 1, 1, 5, 5, 5))
    vel = O3.Vel3(O.VEL_CONST, (A, B, C))
    dt = O3.max_dt3(s, vel)
    ph = O3.remap_3d(s, phi, 0, 0, 0, O3.StepOpts3(vel, 0.0, dt))
    X, Y, Z = O3.node_coords_3d(s, 0, 0, 0)
    direct = O3.poly_3d(s, phi[0, 0, 0], 0, 0, 0, X.ravel() - A * dt, Y.ravel() - B * dt, Z.ravel() - C * dt)
    assert np.max(np.abs(ph.ravel() - direct)) < 1e-11


@pytest.mark.parametrize("n", [3, 4, 5])
def test_face_rows_span_the_boundary_nodes(n):
    """The traces at the 6 n^2 face points constrain exactly the boundary nodes of an n^3 grid:
    rank n^3 - (n - 2)^3 = 6 n^2 - 12 n + 8 (n dependencies per edge, one per corner back)."""
    s = O3.Setup3(1, 1, 1, (0.0, 1.0, 0.0, 1.0, 0.0, 1.0), n)
    Cm = np.vstack([O3.face_rows_3d(s, f) for f in range(6)])
    assert np.linalg.matrix_rank(Cm) == n ** 3 - (n - 2) ** 3


def test_interface_values_are_unique_and_mass_telescopes():
    """Periodic box, rough data, an oblique constant velocity, boundary + mass rows: at every
    shared face point both elements' boundary-row right-hand sides are equal (eq. 4.12a), and the
    global mass is conserved to round-off over two steps."""
    s = O3.Setup3(3, 2, 2, (0.0, 1.5, 0.0, 1.0, 0.0, 1.0), 3, O.GAUSS_LEGENDRE)
    phi = 1.0 + 0.3 * sl_inputs.random_state((2, 2, 3, 3, 3, 3), 11)
    vel = O3.Vel3(O.VEL_CONST, (A, B, C))
    dt = O3.max_dt3(s, vel)
    o = O3.StepOpts3(vel, 0.0, dt, O.C_BOUNDARY | O.C_MASS)
    m0 = O3.mass_3d(s, phi)
    out, infos = O3.step_3d(s, phi, o)
    nq = 9
    for (ex, ey, ez), info in infos.items():
        for face in (1, 3, 5):                                 # E, N, T against the neighbour's W, S, B
            nb = O3.nb_3d(s, ex, ey, ez, face)
            mine = info["d"][face * nq:(face + 1) * nq]
            theirs = infos[nb]["d"][(face - 1) * nq:face * nq]
            assert np.allclose(mine, theirs, rtol=0, atol=1e-14)
    o2 = O3.StepOpts3(vel, dt, dt, O.C_BOUNDARY | O.C_MASS)
    out2, _ = O3.step_3d(s, out, o2)
    assert abs(O3.mass_3d(s, out2) - m0) <= 1e-13 * abs(m0)


def test_rk_step_against_exact_rotation():
    """Solid-body rotation about the z-parallel line through (cx, cy): one RK4 step matches the
    exact rotation to O(dt^5), z is untouched, and the error falls by about 32 when dt halves."""
    om, cx, cy = 2 * np.pi, 0.5, 0.4
    vel = O3.Vel3(O.VEL_ROTATION, (om, cx, cy))
    rng = np.random.default_rng(2)
    x, y, z = rng.uniform(0, 1, 20), rng.uniform(0, 1, 20), rng.uniform(0, 1, 20)
    errs = []
    for dt in (0.02, 0.01):
        xs, ys, zs, ps = O3.rk_particles3(vel, x, y, z, np.ones(20), 0.0, dt, 4)
        c, sn = np.cos(om * dt), np.sin(om * dt)
        xe = cx + c * (x - cx) - sn * (y - cy)
        ye = cy + sn * (x - cx) + c * (y - cy)
        errs.append(np.max(np.hypot(xs - xe, ys - ye)))
        assert np.array_equal(zs, z) and np.all(ps == 1.0)
    assert 20 < errs[0] / errs[1] < 45, errs


def test_upwind_locality():
    """Boundary rows only: a change of phi^n in one element reaches, besides itself, exactly the
    three neighbours its faces flow into (velocity (+, -, +): east, south, top), never the
    upstream ones (eq. 4.12a: an interface value is the trace of the element the flow leaves)."""
    s = O3.Setup3(3, 3, 3, (0.0, 1.0, 0.0, 1.0, 0.0, 1.0), 3, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 6, 0.0)
    phi = 1.0 + 0.3 * sl_inputs.random_state((3, 3, 3, 3, 3, 3), 5)
    vel = O3.Vel3(O.VEL_CONST, (A, B, C))
    o = O3.StepOpts3(vel, 0.0, O3.max_dt3(s, vel), O.C_BOUNDARY)
    a, _ = O3.step_3d(s, phi, o)
    pert = phi.copy()
    pert[1, 1, 1] += 0.1 * sl_inputs.random_state((3, 3, 3), 6)
    b, _ = O3.step_3d(s, pert, o)
    changed = {(ex, ey, ez) for ez in range(3) for ey in range(3) for ex in range(3)
               if np.max(np.abs(a[ez, ey, ex] - b[ez, ey, ex])) > 1e-14}
    assert changed == {(1, 1, 1), (2, 1, 1), (1, 0, 1), (1, 1, 2)}, changed


def test_energy_row_on_linear_data():
    """Boundary + mass + energy rows, linear data under constant velocity with the exact inflow:
    the face fluxes of phi and phi^2 are polynomials of degree <= 2 in time, which the RK4 flux
    quadrature integrates exactly, so the energy target is the translate's energy and the step
    stays the exact translate."""
    lin = lambda x, y, z: 1.0 + 0.3 * x - 0.2 * y + 0.25 * z
    t0 = 0.1
    ghost = lambda x, y, z, t: lin(np.asarray(x) - A * (t - t0), np.asarray(y) - B * (t - t0), np.asarray(z) - C * (t - t0))
    s = O3.Setup3(2, 2, 2, (0.0, 1.0, 0.0, 1.0, 0.0, 1.0), 4, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 6, ghost)
    vel = O3.Vel3(O.VEL_CONST, (A, B, C))
    dt = O3.max_dt3(s, vel)
    out, infos = O3.step_3d(s, O3.project_3d(s, lin), O3.StepOpts3(vel, t0, dt, O.C_BOUNDARY | O.C_MASS | O.C_ENERGY))
    exact = O3.project_3d(s, lambda x, y, z: ghost(x, y, z, t0 + dt))
    assert np.max(np.abs(out - exact)) < 1e-12
    assert all(i["converged"] for i in infos.values())
