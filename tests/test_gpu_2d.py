"""GPU parity of the 2D DSEM-SL step (FP64 path, C ABI) against the FP64 oracle.

Bound: relative L2 <= 1e-12 per step on elements whose energy iteration converged in the
oracle.  Velocity fields: constant (Sec. 5.3), solid-body rotation, swirling deformation."""
import numpy as np
import pytest

import sl_inputs
from oracle import sl_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06476_gb300 import build as B
    B.build()
    import paper_1910_06476_gb300 as pkg
    return pkg


def vel_pair(sl, kind, p):
    return sl.velocity(kind, *p), O.Vel(kind, tuple(p) + (0,) * (6 - len(p)))


def run_case(sl, kx, ky, n, kind, p, bc, cons, rk=4, fit=0, basis=0, ghost=0.0, data=None, t=0.3, seed=0,
             bvalue=0):
    box = (0.0, 1.0, 0.0, 1.0)
    ctx = sl.Context(2, kx, ky, box, n, basis, sl.FP64, (bc,) * 4, ghost)
    setup = O.Setup(2, kx, ky, box, n, basis, (bc,) * 4, ghost)
    gv, ov = vel_pair(sl, kind, p)
    x, y = ctx.node_coords()
    if data is None:
        phi = 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.05 * sl_inputs.random_state(x.shape, seed)
    else:
        phi = data(x, y)
    dt = ctx.max_dt(gv)
    a = torch.tensor(phi.ravel(), device="cuda")
    b = torch.empty_like(a)
    ctx.step(a, b, gv, t, dt, sl.options(cons, rk, fit, bvalue))
    bits = ctx.sync()
    got = b.cpu().numpy().reshape(ky, kx, n, n)
    ref, infos = O.step_2d(setup, phi, O.StepOpts(ov, t, dt, cons, rk, fit, bvalue))
    conv = np.array([[infos[(ex, ey)]["converged"] for ex in range(kx)] for ey in range(ky)])
    return setup, got, ref, conv, bits


def check(setup, got, ref, conv, bits, sl):
    assert conv.mean() > 0.5
    if conv.all():
        assert bits & ~sl.ST_PICARD_NOCONV == 0 and bits == 0, bits
    keep = conv[:, :, None, None]
    num = np.sum(np.where(keep, (got - ref) ** 2, 0.0))
    den = np.sum(np.where(keep, ref ** 2, 0.0))
    rel = np.sqrt(num / den)
    assert rel <= TOL, rel
    return rel


CASES = [
    # kx, ky, n, kind, params, bc, cons, rk, fit, basis
    (6, 5, 9, 0, (1.0, 0.5), 0, 3, 4, 0, 0),          # config 3 shape
    (6, 5, 9, 0, (1.0, 0.5), 0, 1, 4, 0, 0),
    (4, 4, 5, 0, (-0.8, 0.6), 0, 7, 4, 0, 0),
    (4, 3, 4, 0, (0.7, -0.4), 0, 3, 2, 1, 0),         # soft fit
    (5, 4, 6, 0, (1.0, 0.5), 0, 3, 1, 0, 1),          # Chebyshev-Gauss, first order
    (5, 4, 6, 0, (1.0, 0.5), 0, 3, 3, 0, 0),
    (1, 1, 7, 0, (1.0, 0.5), 0, 3, 4, 0, 0),          # single element wrapping onto itself
    (1, 3, 5, 0, (0.3, 1.0), 0, 3, 4, 0, 0),
    (6, 6, 6, 1, (2 * np.pi, 0.5, 0.5), 1, 3, 4, 0, 0),   # rotation, inflow ghost (config 4 shape)
    (5, 5, 8, 2, (5.0,), 1, 7, 4, 0, 0),              # swirl, mass + energy (config 5 shape)
    (5, 5, 8, 2, (5.0,), 1, 3, 4, 0, 0),
    (4, 4, 3, 1, (2 * np.pi, 0.5, 0.5), 1, 2, 4, 0, 0),
    (3, 3, 12, 0, (1.0, 0.5), 0, 3, 4, 0, 0),
    (2, 2, 16, 1, (2 * np.pi, 0.5, 0.5), 1, 3, 4, 0, 0),
    (2, 2, 17, 0, (0.6, 0.9), 0, 3, 4, 0, 0),
    (3, 2, 2, 0, (0.6, 0.9), 0, 3, 4, 0, 0),
    # axis-aligned constant velocity: every face of one direction is an upwind tie (eq. 4.12a,
    # reading R8: interior ties average both traces, inflow domain faces keep their own)
    (5, 4, 6, 0, (1.0, 0.0), 0, 3, 4, 0, 0),
    (4, 5, 7, 0, (0.0, -0.7), 1, 3, 4, 0, 0),
    (4, 4, 5, 0, (0.0, -0.7), 0, 7, 4, 0, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}n{c[2]}v{c[3]}bc{c[5]}c{c[6]}rk{c[7]}f{c[8]}b{c[9]}"
                                             for c in CASES])
def test_2d_step_parity(sl, case):
    kx, ky, n, kind, p, bc, cons, rk, fit, basis = case
    r = run_case(sl, kx, ky, n, kind, p, bc, cons, rk, fit, basis, ghost=0.2 if bc else 0.0, seed=kx * 7 + n)
    check(*r, sl)


BT_CASES = [
    # kx, ky, n, kind, params, bc, cons, rk, fit, basis: backtracked interface values (eq. 4.11)
    (6, 5, 9, 0, (1.0, 0.5), 0, 3, 4, 0, 0),
    (4, 4, 5, 0, (-0.8, 0.6), 0, 7, 4, 0, 0),
    (4, 3, 4, 0, (0.7, -0.4), 0, 1, 2, 1, 0),         # soft fit, second order
    (5, 4, 6, 0, (1.0, 0.0), 0, 3, 4, 0, 1),          # axis-aligned, Chebyshev-Gauss
    (1, 1, 7, 0, (1.0, 0.5), 0, 3, 4, 0, 0),          # single element wrapping onto itself
    (6, 6, 6, 1, (2 * np.pi, 0.5, 0.5), 1, 3, 4, 0, 0),   # rotation, inflow ghost
    (5, 5, 8, 2, (5.0,), 1, 7, 4, 0, 0),              # swirl, mass + energy
    (5, 5, 8, 2, (5.0,), 0, 3, 3, 0, 0),              # swirl, periodic, third order
    (2, 2, 16, 1, (2 * np.pi, 0.5, 0.5), 1, 3, 4, 0, 0),
]


@pytest.mark.parametrize("case", BT_CASES, ids=[f"{c[0]}x{c[1]}n{c[2]}v{c[3]}bc{c[5]}c{c[6]}rk{c[7]}"
                                                for c in BT_CASES])
def test_2d_backtracked_interface_parity(sl, case):
    kx, ky, n, kind, p, bc, cons, rk, fit, basis = case
    r = run_case(sl, kx, ky, n, kind, p, bc, cons, rk, fit, basis, ghost=0.2 if bc else 0.0, seed=kx * 5 + n,
                 bvalue=sl.BV_BACKTRACK)
    check(*r, sl)


def test_2d_backtracked_differs_from_interpolated(sl):
    """The two interface rules give different steps on under-resolved data (the GPU takes the
    rule it is given), and the same step on data the element polynomials hold exactly."""
    a = run_case(sl, 4, 4, 5, 2, (5.0,), 0, 3, bvalue=sl.BV_INTERP, seed=3)
    b = run_case(sl, 4, 4, 5, 2, (5.0,), 0, 3, bvalue=sl.BV_BACKTRACK, seed=3)
    assert np.abs(a[1] - b[1]).max() > 1e-6
    lin = lambda x, y: 1.0 + 0.3 * x - 0.2 * y
    a = run_case(sl, 4, 4, 5, 0, (0.6, 0.3), 0, 3, data=lin, bvalue=sl.BV_INTERP)
    b = run_case(sl, 4, 4, 5, 0, (0.6, 0.3), 0, 3, data=lin, bvalue=sl.BV_BACKTRACK)
    assert np.abs(a[1] - b[1]).max() < 1e-12


def test_2d_cosine_bell_and_hill_data(sl):
    """Exactly-zero regions (cosine bell) and the Gaussian hill, as in the large configurations."""
    r = run_case(sl, 6, 6, 8, 2, (5.0,), 1, 7, data=sl_inputs.cosine_bell_2d, t=0.7)
    check(*r, sl)
    r = run_case(sl, 6, 6, 7, 1, (2 * np.pi, 0.5, 0.5), 1, 3, data=sl_inputs.hill_2d)
    check(*r, sl)


def test_2d_multistep_parity_and_mass(sl):
    """Ten steps of config 3's problem at 4 x 4 elements: stays within 1e-12 of the oracle and
    conserves mass (periodic, mass constraint) to round-off."""
    prob = sl_inputs.config3_2d_const(n=7, k=4)
    ctx = sl.Context(2, 4, 4, prob.box, 7, 0, sl.FP64, prob.bc, 0.0)
    setup = O.setup_from_problem(prob)
    gv = sl.velocity(sl.VEL_CONST, 1.0, 0.5)
    dt = ctx.max_dt(gv, sl_inputs.rule_code(prob))
    x, y = ctx.node_coords()
    a = torch.tensor(prob.phi0(x, y).ravel(), device="cuda")
    b = torch.empty_like(a)
    ref = O.project_2d(setup, prob.phi0)
    m0 = ctx.mass(a)
    o = O.StepOpts(O.Vel(O.VEL_CONST, (1.0, 0.5, 0, 0, 0, 0)), 0.0, dt, prob.constraints, 4)
    for s in range(10):
        ctx.step(a, b, gv, s * dt, dt, sl.options(prob.constraints, 4))
        a, b = b, a
        ref, _ = O.step_2d(setup, ref, o)
        o.t += dt
    assert ctx.sync() == 0
    got = a.cpu().numpy().reshape(4, 4, 7, 7)
    assert O.rel_l2(setup, got, ref) < TOL
    assert abs(ctx.mass(a) - m0) < 1e-13 * max(1.0, abs(m0))


def test_config3_full_size_sampled(sl):
    """Config 3 at full size (512 x 512, n = 9, boundary + mass): sampled elements recomputed by
    the oracle from the GPU's own pre-step state."""
    prob = sl_inputs.config3_2d_const()
    K = prob.kx
    ctx = sl.Context(2, K, K, prob.box, prob.n, 0, sl.FP64, prob.bc, 0.0)
    setup = O.setup_from_problem(prob)
    gv = sl.velocity(sl.VEL_CONST, 1.0, 0.5)
    dt = ctx.max_dt(gv)
    x, y = ctx.node_coords()
    a = torch.tensor(prob.phi0(x, y).ravel(), device="cuda")
    b = torch.empty_like(a)
    opts = sl.options(prob.constraints, 4)
    ctx.step(a, b, gv, 0.0, dt, opts)
    a, b = b, a
    pre = a.cpu().numpy().reshape(K, K, 9, 9)
    ctx.step(a, b, gv, dt, dt, opts)
    assert ctx.sync() == 0
    got = b.cpu().numpy().reshape(K, K, 9, 9)
    idx = sl_inputs.sample_elements(60, K * K, 11)
    elems = [(int(e % K), int(e // K)) for e in idx] + [(0, 0), (K - 1, K - 1), (0, K - 1)]
    ref, _ = O.step_2d(setup, pre, O.StepOpts(O.Vel(O.VEL_CONST, (1.0, 0.5, 0, 0, 0, 0)), dt, dt,
                                              prob.constraints, 4), elements=elems)
    for ex, ey in elems:
        d = np.max(np.abs(got[ey, ex] - ref[ey, ex]))
        assert d <= 1e-12 * max(1.0, np.max(np.abs(ref[ey, ex]))), (ex, ey, d)
