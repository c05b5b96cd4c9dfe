"""Pins of the oracle's p-adaptive 2D step (per-element node counts; the reading for
p-nonconforming faces, which the paper does not treat: the upwind value at a face point is the
neighbour's remapped polynomial evaluated there, and the face flux is integrated once with the
Gauss rule of the side with more nodes, shared by both elements).

- polynomial data that every element represents exactly is translated exactly (a wrong face
  point, neighbour or evaluation would break it);
- equal node counts everywhere reproduce the uniform-mesh step;
- on a periodic mesh with mixed node counts, mass and energy telescope (each face flux is the
  same number for both elements only if both use the same rule)."""
import numpy as np
import pytest

from oracle import sl_oracle as O

CONST = O.Vel(O.VEL_CONST, (0.8, 0.45, 0, 0, 0, 0))


def poly2(x, y):
    return 0.2 + x - 0.7 * y + 1.3 * x * y - 0.5 * x * x * y + 0.8 * y ** 3


def flat(nested):
    return np.concatenate([e.ravel() for row in nested for e in row])


@pytest.mark.parametrize("cons", [O.C_BOUNDARY, O.C_BOUNDARY | O.C_MASS])
@pytest.mark.parametrize("fit", [O.FIT_HARD, O.FIT_SOFT])
def test_padaptive_exact_translation(cons, fit):
    """Constant velocity, inflow ghost = the exact translate, cubic data, node counts 4..8 per
    element: phi^{n+1} is the exact translate on every element (with the mass row, the RK4
    flux quadrature is exact for this cubic data)."""
    a, b = 0.8, 0.45
    orders = np.array([[4, 7, 5], [8, 4, 6], [5, 6, 4]])
    s = O.Setup(2, 3, 3, (0, 1, 0, 1), 8, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 4,
                lambda x, y, t: poly2(np.asarray(x) - a * t, np.asarray(y) - b * t), orders)
    phi = O.project_2d(s, poly2)
    dt = O.max_dt(s, CONST)
    out, _ = O.step_2d(s, phi, O.StepOpts(CONST, 0.0, dt, cons, 4, fit))
    exact = O.project_2d(s, lambda x, y: poly2(x - a * dt, y - b * dt))
    np.testing.assert_allclose(flat(out), flat(exact), atol=1e-12)


def test_padaptive_equal_orders_is_uniform():
    n = 6
    orders = np.full((3, 4), n)
    vel = O.Vel(O.VEL_ROTATION, (2 * np.pi, 0.5, 0.5, 0, 0, 0))
    su = O.Setup(2, 4, 3, (0, 1, 0, 1), n, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 4, 0.1)
    sp = O.Setup(2, 4, 3, (0, 1, 0, 1), n, O.GAUSS_LEGENDRE, (O.BC_INFLOW,) * 4, 0.1, orders)
    f = lambda x, y: np.exp(-((x - 0.4) ** 2 + (y - 0.5) ** 2) / 0.05)
    pu, pp = O.project_2d(su, f), O.project_2d(sp, f)
    dt = O.max_dt(su, vel)
    o = O.StepOpts(vel, 0.0, dt, O.C_BOUNDARY | O.C_MASS, 4)
    ou, _ = O.step_2d(su, pu, o)
    op, _ = O.step_2d(sp, pp, o)
    np.testing.assert_array_equal(ou.ravel(), flat(op))


def test_padaptive_periodic_mass_energy_telescope():
    orders = np.array([[4, 7, 5, 6], [8, 5, 6, 4], [5, 6, 4, 7], [6, 4, 7, 5]])
    s = O.Setup(2, 4, 4, (0, 1, 0, 1), 8, O.GAUSS_LEGENDRE, (O.BC_PERIODIC,) * 4, 0.0, orders)
    vel = O.Vel(O.VEL_SWIRL, (5.0, 0, 0, 0, 0, 0))
    phi = O.project_2d(s, lambda x, y: 1.0 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
    dt = O.max_dt(s, vel)
    o = O.StepOpts(vel, 0.3, dt, O.C_BOUNDARY | O.C_MASS | O.C_ENERGY, 4)
    m0, e0 = O.mass(s, phi), O.energy(s, phi)
    out, inf = O.step_2d(s, phi, o)
    assert all(i["converged"] for i in inf.values())
    assert abs(O.mass(s, out) - m0) < 1e-13 * abs(m0)
    assert abs(O.energy(s, out) - e0) < 1e-13 * abs(e0)


def test_padaptive_own_rule_would_not_telescope(monkeypatch):
    """The same mesh with each element integrating its faces on its own rule (a plausible
    misreading) loses mass: the shared-rule reading is what the telescoping test pins."""
    orders = np.array([[4, 7, 5, 6], [8, 5, 6, 4], [5, 6, 4, 7], [6, 4, 7, 5]])
    s = O.Setup(2, 4, 4, (0, 1, 0, 1), 8, O.GAUSS_LEGENDRE, (O.BC_PERIODIC,) * 4, 0.0, orders)
    vel = O.Vel(O.VEL_SWIRL, (5.0, 0, 0, 0, 0, 0))
    phi = O.project_2d(s, lambda x, y: 1.0 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))
    dt = O.max_dt(s, vel)
    o = O.StepOpts(vel, 0.3, dt, O.C_BOUNDARY | O.C_MASS, 4)
    m0 = O.mass(s, phi)
    monkeypatch.setattr(O, "face_rule_points", lambda n, n_nb: n)   # each side on its own rule
    out, _ = O.step_2d(s, phi, o)
    assert abs(O.mass(s, out) - m0) > 1e-10 * abs(m0)
