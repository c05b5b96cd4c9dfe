"""Pins of the oracle's tables, basis and time integrator against things other than itself:
library routines (numpy's Gauss-Legendre), closed forms (Fejer weights, solid-body rotation),
exactness properties and the time step printed in the paper (Sec. 5.2)."""
import math
import os

import numpy as np
import pytest

from oracle import sl_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden(key):
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            if k == key:
                return float(v)
    raise KeyError(key)


@pytest.mark.parametrize("n", list(range(1, 21)))
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre_01(n)
    rx, rw = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (rx + 1.0), atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * rw, atol=2e-15)


@pytest.mark.parametrize("n", [2, 5, 9, 13, 17])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = O.gauss_legendre_01(n)
    for p in range(2 * n):
        assert abs(np.dot(w, x ** p) - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 7, 8, 12])
def test_chebyshev_gauss_nodes_closed_form(n):
    xi = O.chebyshev_gauss_01(n)
    # roots of T_n mapped to [0, 1]: T_n(1 - 2 xi) = 0 and symmetric about 1/2
    t = np.cos(n * np.arccos(1.0 - 2.0 * xi))
    assert np.max(np.abs(t)) < 1e-13
    np.testing.assert_allclose(xi + xi[::-1], 1.0, atol=1e-15)
    assert np.all(np.diff(xi) > 0)


@pytest.mark.parametrize("n", [2, 3, 6, 7, 10])
def test_fejer_weights_closed_form(n):
    """Interpolatory weights on Chebyshev-Gauss nodes equal Fejer's first-rule closed form."""
    _, w = O.nodes_weights(n, O.CHEB_GAUSS)
    th = (2 * np.arange(n) + 1) * np.pi / (2 * n)
    ref = np.ones(n)
    for j in range(1, n // 2 + 1):
        ref -= 2.0 * np.cos(2 * j * th) / (4 * j * j - 1)
    ref *= 2.0 / n
    np.testing.assert_allclose(w, 0.5 * ref, atol=1e-14)
    xi, _ = O.nodes_weights(n, O.CHEB_GAUSS)
    for p in range(n):
        assert abs(np.dot(w, xi ** p) - 1.0 / (p + 1)) < 1e-13


@pytest.mark.parametrize("basis", [O.GAUSS_LEGENDRE, O.CHEB_GAUSS])
@pytest.mark.parametrize("n", [1, 2, 5, 9, 16])
def test_lagrange_cardinal_partition_and_reproduction(basis, n):
    xi, _ = O.nodes_weights(n, basis)
    L = O.lagrange(xi, xi)
    np.testing.assert_allclose(L, np.eye(n), atol=1e-13)
    xs = np.linspace(-0.1, 1.1, 37)
    Ls = O.lagrange(xi, xs)
    np.testing.assert_allclose(Ls.sum(axis=1), 1.0, atol=1e-11)
    for p in range(n):
        np.testing.assert_allclose(Ls @ xi ** p, xs ** p, atol=1e-10)


def test_paper_time_step_sinx():
    """Sec. 5.2 prints dt = 1.97e-2 for H=4, P=6 on [0, 2 pi] with |u|max = 1: reproduced by
    n = P + 1 = 7 Chebyshev-Gauss nodes and the edge-gap rule (readings R1, R9)."""
    s = O.Setup(1, 4, 1, (0.0, 2 * np.pi, 0, 0), 7, O.CHEB_GAUSS)
    dt = O.max_dt(s, O.Vel(O.VEL_SINX, (0,) * 6), rule="paper")
    assert round(dt, 4) == golden("dt_sinx_H4_P6")
    # neighbouring node counts do not reproduce the printed value
    for n in (6, 8):
        s2 = O.Setup(1, 4, 1, (0.0, 2 * np.pi, 0, 0), n, O.CHEB_GAUSS)
        assert round(O.max_dt(s2, O.Vel(O.VEL_SINX, (0,) * 6), rule="paper"), 4) != golden("dt_sinx_H4_P6")


def test_half_spacing_rule_values():
    """Half the minimum node spacing (GL, n=9): 0.5 * 0.066065 / K for unit speed."""
    s = O.Setup(1, 16, 1, (0.0, 1.0, 0, 0), 9)
    dt = O.max_dt(s, O.Vel(O.VEL_CONST, (1.0, 0, 0, 0, 0, 0)))
    xi = 0.5 * (np.polynomial.legendre.leggauss(9)[0] + 1)
    assert abs(dt - 0.5 * np.min(np.diff(xi)) / 16) < 1e-15
    s2 = O.Setup(2, 256, 256, (0, 1, 0, 1), 16)
    dt2 = O.max_dt(s2, O.Vel(O.VEL_ROTATION, (2 * np.pi, 0.5, 0.5, 0, 0, 0)))
    xi16 = 0.5 * (np.polynomial.legendre.leggauss(16)[0] + 1)
    assert abs(dt2 - 0.5 * np.min(np.diff(xi16)) / 256 / np.pi) < 1e-15


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_rk_constant_velocity_exact(order):
    x = np.linspace(0, 1, 7)
    y = np.linspace(0, 2, 7)
    xs, ys, ps = O.rk_particles(O.Vel(O.VEL_CONST, (0.7, -0.3, 0, 0, 0, 0)), x, y, np.ones(7), 0.3, 0.01, order)
    np.testing.assert_allclose(xs, x + 0.007, atol=1e-15)
    np.testing.assert_allclose(ys, y - 0.003, atol=1e-15)
    np.testing.assert_allclose(ps, 1.0, atol=0)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_rk_rotation_order(order):
    """Solid-body rotation has the closed-form flow map; one-step error must scale as dt^(p+1)."""
    vel = O.Vel(O.VEL_ROTATION, (2 * np.pi, 0.5, 0.5, 0, 0, 0))
    x, y = np.array([0.25, 0.8]), np.array([0.5, 0.1])

    def err(dt):
        xs, ys, _ = O.rk_particles(vel, x, y, np.ones(2), 0.0, dt, order)
        a = 2 * np.pi * dt
        ex = 0.5 + (x - 0.5) * np.cos(a) - (y - 0.5) * np.sin(a)
        ey = 0.5 + (x - 0.5) * np.sin(a) + (y - 0.5) * np.cos(a)
        return np.max(np.hypot(xs - ex, ys - ey))

    e1, e2 = err(1e-2), err(5e-3)
    rate = math.log2(e1 / e2)
    assert abs(rate - (order + 1)) < 0.2, rate


def test_rk4_swirl_full_period_returns():
    """The swirl flow reverses at t = T/2; over [0, T] the flow map is the identity."""
    vel = O.Vel(O.VEL_SWIRL, (5.0, 0, 0, 0, 0, 0))
    x0, y0 = np.array([0.3, 0.5, 0.7]), np.array([0.6, 0.75, 0.2])
    errs = []
    for nsteps in (200, 400):
        x, y, p = x0.copy(), y0.copy(), np.ones(3)
        dt = 5.0 / nsteps
        for i in range(nsteps):
            x, y, p = O.rk_particles(vel, x, y, p, i * dt, dt, 4)
        errs.append(np.max(np.hypot(x - x0, y - y0)))
    assert errs[1] < 1e-6 and errs[0] / errs[1] > 10.0


def test_rk_sinx_value_equation():
    """dx/dt = -sin x, dphi/dt = phi cos x (Sec. 5.2 with eq. 2.4): phi * sin(x) is invariant
    along the path, since d(sin x)/dt = -cos x sin x."""
    vel = O.Vel(O.VEL_SINX, (0,) * 6)
    x = np.array([0.5, 1.5, 2.5, 4.0])
    p = np.array([1.0, 2.0, -1.0, 0.5])
    inv0 = p * np.sin(x)
    for i in range(50):
        x, _, p = O.rk_particles(vel, x, np.zeros(4), p, i * 0.01, 0.01, 4)
    np.testing.assert_allclose(p * np.sin(x), inv0, rtol=1e-9)
