"""Pins of the oracle's interface values (eq. 4.12a, reading R8), no GPU.

Eq. 4.12a gives each face point ONE value at t^{n+1}: the trace of the element upwind of it.  So
at every face point shared by two elements, the right-hand side of the boundary-constraint row
of one element equals that of the other.  This holds whatever the sign of u.n, including ties
(u.n = 0: axis-aligned velocities make every face of one direction a tie, and u = -sin x is zero
on the faces at 0 and pi), across periodic wraps, and next to inflow domain faces.  Planting the
plausible mistake "a tie keeps the element's own trace" breaks it."""
import numpy as np
import pytest

import sl_inputs
from oracle import sl_oracle as O


def _face_values_1d(s, phi, o):
    _, infos = O.step_1d(s, phi, o)
    return {k: infos[k]["d"][:2] for k in infos}


def _check_1d(s, phi, o):
    d = _face_values_1d(s, phi, o)
    K = s.kx
    shared = [(k, k + 1) for k in range(K - 1)]
    if s.bc[0] == O.BC_PERIODIC:
        shared.append((K - 1, 0))
    worst = 0.0
    for left, right in shared:
        worst = max(worst, abs(d[left][1] - d[right][0]))
    return worst


@pytest.mark.parametrize("vel,box,bc", [
    (O.Vel(O.VEL_CONST, (1.0, 0.0)), (0.0, 1.0), O.BC_PERIODIC),
    (O.Vel(O.VEL_CONST, (-0.8, 0.0)), (0.0, 1.0), O.BC_INFLOW),
    (O.Vel(O.VEL_SINX, ()), (0.0, 2 * np.pi), O.BC_PERIODIC),     # ties at x = 0 and x = pi
])
def test_1d_interface_value_unique(vel, box, bc):
    s = O.Setup(1, 4, 1, box, 6, O.CHEB_GAUSS, (bc,) * 4, ghost=0.3)
    phi = 1.0 + 0.5 * sl_inputs.random_state((4, 6), 11)
    dt = O.max_dt(s, vel, rule="paper")
    o = O.StepOpts(vel, 0.1, dt, O.C_BOUNDARY, 4)
    assert _check_1d(s, phi, o) == 0.0


def _check_2d(s, phi, o):
    _, infos = O.step_2d(s, phi, o)
    n = s.n
    worst = 0.0
    ties = 0
    for (ex, ey), inf in infos.items():
        d = inf["d"]
        for f in range(4):
            nb = O._nb_2d(s, ex, ey, f)
            if nb is None:
                continue
            dn = infos[nb]["d"]
            mine = d[f * n:(f + 1) * n]
            theirs = dn[(f ^ 1) * n:((f ^ 1) + 1) * n]
            worst = max(worst, float(np.max(np.abs(mine - theirs))))
            xf, yf, nrm, _ = O._face_points(s, ex, ey, f, n)
            u, v, _ = O.velocity(o.vel, xf, yf, o.t + o.dt)
            ties += int(np.sum(np.abs(u * nrm[0] + v * nrm[1]) <= O.TIE))
    return worst, ties


CASES_2D = [
    (O.Vel(O.VEL_CONST, (1.0, 0.0)), (O.BC_PERIODIC,) * 4),                 # S/N faces all ties
    (O.Vel(O.VEL_CONST, (0.0, -0.7)), (O.BC_INFLOW,) * 4),                  # W/E faces all ties
    (O.Vel(O.VEL_CONST, (1.0, 0.5)), (O.BC_PERIODIC, O.BC_PERIODIC, O.BC_INFLOW, O.BC_INFLOW)),
    (O.Vel(O.VEL_ROTATION, (2 * np.pi, 0.5, 0.5)), (O.BC_INFLOW,) * 4),    # u.n = 0 on the axes
    (O.Vel(O.VEL_SWIRL, (5.0,)), (O.BC_PERIODIC,) * 4),
]


@pytest.mark.parametrize("vel,bc", CASES_2D)
def test_2d_interface_value_unique(vel, bc):
    s = O.Setup(2, 4, 4, (0.0, 1.0, 0.0, 1.0), 4, O.GAUSS_LEGENDRE, bc, ghost=0.25)
    phi = 1.0 + 0.5 * sl_inputs.random_state((4, 4, 4, 4), 5)
    dt = O.max_dt(s, vel, rule="paper")
    o = O.StepOpts(vel, 0.05, dt, O.C_BOUNDARY, 4)
    worst, _ = _check_2d(s, phi, o)
    assert worst == 0.0


def test_planted_tie_mistake_breaks_uniqueness(monkeypatch):
    """'A tie keeps the element's own trace' gives the two elements of a tie face different
    values: the pin above must catch it (in 1D at the zeros of -sin x, in 2D on axis-aligned
    flow)."""
    def own_on_tie(un, own, other, interior):
        if un < -O.TIE:
            return other
        return own
    monkeypatch.setattr(O, "upwind_value", own_on_tie)
    s1 = O.Setup(1, 4, 1, (0.0, 2 * np.pi), 6, O.CHEB_GAUSS, (O.BC_PERIODIC,) * 4)
    phi1 = 1.0 + 0.5 * sl_inputs.random_state((4, 6), 11)
    vel1 = O.Vel(O.VEL_SINX, ())
    o1 = O.StepOpts(vel1, 0.1, O.max_dt(s1, vel1, rule="paper"), O.C_BOUNDARY, 4)
    assert _check_1d(s1, phi1, o1) > 1e-6
    s = O.Setup(2, 4, 4, (0.0, 1.0, 0.0, 1.0), 4, O.GAUSS_LEGENDRE, (O.BC_PERIODIC,) * 4)
    phi = 1.0 + 0.5 * sl_inputs.random_state((4, 4, 4, 4), 5)
    vel = O.Vel(O.VEL_CONST, (1.0, 0.0))
    o = O.StepOpts(vel, 0.05, O.max_dt(s, vel, rule="paper"), O.C_BOUNDARY, 4)
    worst, ties = _check_2d(s, phi, o)
    assert ties > 0 and worst > 1e-6


def test_axis_aligned_cases_have_ties():
    """The axis-aligned cases above really exercise the tie branch (every face of one direction)."""
    s = O.Setup(2, 4, 4, (0.0, 1.0, 0.0, 1.0), 4, O.GAUSS_LEGENDRE, (O.BC_PERIODIC,) * 4)
    phi = 1.0 + 0.5 * sl_inputs.random_state((4, 4, 4, 4), 5)
    vel = O.Vel(O.VEL_CONST, (1.0, 0.0))
    o = O.StepOpts(vel, 0.05, O.max_dt(s, vel, rule="paper"), O.C_BOUNDARY, 4)
    _, ties = _check_2d(s, phi, o)
    assert ties == 16 * 2 * 4      # every element: both y-faces, 4 points each
