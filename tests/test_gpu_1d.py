"""GPU parity of the 1D DSEM-SL step (C ABI) against the FP64 oracle, element by element.

FP64 path: relative L2 (quadrature weighted) <= 1e-12 per step, and max abs difference
<= 1e-12 * max|phi| + 1e-14.  Meshes span several CTAs (126 elements each) with a ragged
tail; the full 2^20-element workload is checked on sampled elements recomputed by the
oracle from the GPU's own pre-step state."""
import numpy as np
import pytest

import sl_inputs
from oracle import sl_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_REL = 1e-12


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06476_gb300 import build as B
    B.build()
    import paper_1910_06476_gb300 as pkg
    return pkg


def make(sl, K, n, basis=0, bc=0, ghost=0.0, box=(0.0, 1.0, 0, 0), precision=0):
    ctx = sl.Context(1, K, 1, box, n, basis, precision, (bc,) * 4, ghost)
    setup = O.Setup(1, K, 1, box, n, basis, (bc,) * 4, ghost)
    return ctx, setup


def gpu_step(sl, ctx, phi, vel, t, dt, opts):
    a = torch.tensor(phi, device="cuda", dtype=ctx.dtype)
    b = torch.empty_like(a)
    ctx.step(a, b, vel, t, dt, opts)
    bits = ctx.sync()
    return b.double().cpu().numpy(), bits


def compare(setup, got, ref, tol=TOL_REL):
    rel = O.rel_l2(setup, got, ref)
    mad = np.max(np.abs(got - ref))
    assert rel <= tol, (rel, mad)
    assert mad <= tol * max(1.0, np.max(np.abs(ref))) * 10 + 1e-14, (rel, mad)
    return rel


CASES = [
    # K, n, basis, bc, vel, cons, rk, fit, bvalue
    (16, 9, 0, 0, ("const", 1.0), 1, 4, 0, 0),
    (16, 9, 0, 0, ("const", 1.0), 3, 4, 0, 0),
    (16, 9, 0, 0, ("const", 1.0), 7, 4, 0, 0),
    (300, 5, 0, 0, ("const", 0.7), 7, 4, 0, 0),
    (300, 5, 0, 0, ("const", -0.7), 7, 2, 0, 0),
    (257, 13, 0, 0, ("const", 1.0), 3, 3, 0, 0),
    (130, 17, 0, 0, ("const", 1.0), 7, 4, 0, 0),
    (130, 2, 0, 0, ("const", 1.0), 3, 4, 0, 0),
    (40, 7, 1, 0, ("const", 1.0), 3, 1, 1, 0),
    (40, 7, 1, 0, ("const", 1.0), 7, 2, 1, 0),
    (40, 6, 0, 1, ("const", 0.9), 3, 4, 0, 0),
    (40, 6, 0, 1, ("const", -0.9), 7, 4, 0, 1),
    (24, 7, 1, 0, ("sinx",), 3, 4, 0, 0),
    (24, 7, 1, 0, ("sinx",), 1, 2, 1, 1),
    (24, 8, 0, 0, ("sinx",), 3, 3, 0, 0),
    (1, 6, 0, 0, ("const", 1.0), 3, 4, 0, 0),
    (2, 6, 0, 1, ("const", 1.0), 7, 4, 0, 0),
    (127, 4, 0, 0, ("const", 1.0), 2, 4, 0, 0),
    (127, 4, 0, 0, ("const", 1.0), 4, 4, 1, 0),
]


def velocity_pair(sl, v):
    if v[0] == "const":
        return sl.velocity(sl.VEL_CONST, v[1]), O.Vel(O.VEL_CONST, (v[1], 0, 0, 0, 0, 0))
    return sl.velocity(sl.VEL_SINX), O.Vel(O.VEL_SINX, (0,) * 6)


@pytest.mark.parametrize("case", CASES, ids=[f"K{c[0]}n{c[1]}b{c[2]}bc{c[3]}{c[4][0]}c{c[5]}rk{c[6]}f{c[7]}bv{c[8]}"
                                             for c in CASES])
def test_step_parity_random(sl, case):
    K, n, basis, bc, v, cons, rk, fit, bvalue = case
    box = (0.0, 2 * np.pi, 0, 0) if v[0] == "sinx" else (0.0, 1.0, 0, 0)
    ctx, setup = make(sl, K, n, basis, bc, 0.25, box)
    gv, ov = velocity_pair(sl, v)
    rng = np.random.default_rng(K * 100 + n)
    # smooth field plus noise: keeps energy targets reachable while exercising every term
    x, _ = ctx.node_coords()
    phi = 1.0 + 0.5 * np.sin(2 * np.pi * x / (box[1] - box[0])) + 0.05 * sl_inputs.random_state(x.shape, K + n)
    dt = ctx.max_dt(gv)
    t = 0.37
    got, bits = gpu_step(sl, ctx, phi, gv, t, dt, sl.options(cons, rk, fit, bvalue))
    ref, infos = O.step_1d(setup, phi, O.StepOpts(ov, t, dt, cons, rk, fit, bvalue))
    conv = np.array([infos[k]["converged"] for k in range(K)])
    if conv.all():
        assert bits == 0
    else:
        assert bits & sl.ST_PICARD_NOCONV
    # first-order energy targets are often unreachable (the paper's MEF instability)
    assert conv.mean() > 0.5
    # elements whose energy iteration did not converge carry no unique answer: compare the rest
    keep = np.where(conv)[0]
    compare(O.Setup(1, len(keep), 1, (0, len(keep) * setup.hx, 0, 0), n, basis), got[keep], ref[keep])


def test_config1_one_period_exact_and_oracle(sl):
    """Config 1 (K=16, 9 GL nodes, u=1, sin 2 pi x, boundary only, RK4) to T=1."""
    prob = sl_inputs.config1_1d_sine()
    ctx, setup = make(sl, prob.kx, prob.n)
    gv = sl.velocity(sl.VEL_CONST, 1.0)
    nsteps, dt = sl_inputs.steps_to(1.0, ctx.max_dt(gv))
    assert nsteps == 485
    x, _ = ctx.node_coords()
    a = torch.tensor(prob.phi0(x), device="cuda")
    b = torch.empty_like(a)
    opts = sl.options(sl.C_BOUNDARY, 4)
    ref = O.project_1d(setup, prob.phi0)
    o = O.StepOpts(O.Vel(O.VEL_CONST, (1.0, 0, 0, 0, 0, 0)), 0.0, dt, O.C_BOUNDARY, 4)
    for s in range(nsteps):
        ctx.step(a, b, gv, s * dt, dt, opts)
        a, b = b, a
        if s < 20:
            ref, _ = O.step_1d(setup, ref, o)
            o.t += dt
            compare(setup, a.cpu().numpy(), ref)
    assert ctx.sync() == 0
    exact = prob.phi0(x - 1.0)
    assert O.rel_l2(setup, a.cpu().numpy(), exact) < 1e-11


def test_full_size_sampled_parity(sl):
    """Config 2 shape at full size (K = 2^20, n = 9, boundary+mass+energy): sampled elements
    plus both ends, recomputed by the oracle from the GPU's own pre-step state."""
    prob = sl_inputs.config2_1d_gauss(9)
    ctx, setup = make(sl, prob.kx, prob.n)
    gv = sl.velocity(sl.VEL_CONST, 1.0)
    dt = ctx.max_dt(gv, sl_inputs.rule_code(prob))
    x, _ = ctx.node_coords()
    a = torch.tensor(prob.phi0(x), device="cuda")
    b = torch.empty_like(a)
    opts = sl.options(prob.constraints, 4)
    for s in range(3):
        ctx.step(a, b, gv, s * dt, dt, opts)
        a, b = b, a
    pre = a.cpu().numpy()
    ctx.step(a, b, gv, 3 * dt, dt, opts)
    assert ctx.sync() == 0
    got = b.cpu().numpy()
    K = prob.kx
    sample = np.concatenate([[0, 1, K - 1], sl_inputs.sample_elements(200, K, 7),
                             np.arange(K // 2 - 20, K // 2 + 20)])
    sample = np.unique(sample)
    o = O.StepOpts(O.Vel(O.VEL_CONST, (1.0, 0, 0, 0, 0, 0)), 3 * dt, dt, prob.constraints, 4)
    ref, _ = O.step_1d(setup, pre, o, elements=sample)
    g, r = got[sample], ref[sample]
    scale = np.max(np.abs(r)) + 1e-300
    assert np.max(np.abs(g - r)) <= 1e-12 * max(scale, 1e-3) + 1e-15


def test_mass_energy_diagnostics(sl):
    ctx, setup = make(sl, 300, 7)
    phi = sl_inputs.random_state((300, 7), 3)
    a = torch.tensor(phi, device="cuda")
    assert abs(ctx.mass(a) - O.mass(setup, phi)) < 1e-13
    assert abs(ctx.energy(a) - O.energy(setup, phi)) < 1e-13


def test_periodic_mass_conserved_many_steps(sl):
    ctx, setup = make(sl, 64, 8)
    gv = sl.velocity(sl.VEL_CONST, 1.0)
    dt = ctx.max_dt(gv)
    x, _ = ctx.node_coords()
    a = torch.tensor(1.0 + np.sin(2 * np.pi * x) ** 3, device="cuda")
    b = torch.empty_like(a)
    m0, e0 = ctx.mass(a), ctx.energy(a)
    opts = sl.options(sl.C_BOUNDARY | sl.C_MASS | sl.C_ENERGY, 4)
    for s in range(200):
        ctx.step(a, b, gv, s * dt, dt, opts)
        a, b = b, a
    assert ctx.sync() == 0
    assert abs(ctx.mass(a) - m0) < 1e-13 * abs(m0)
    # the energy row is skipped when the linear fit already meets it to 1e-12 (per element)
    assert abs(ctx.energy(a) - e0) < 200 * 1e-12 * abs(e0)


def test_status_bits_and_errors(sl):
    ctx, setup = make(sl, 8, 5)
    gv = sl.velocity(sl.VEL_CONST, 1.0)
    dt = ctx.max_dt(gv)
    phi = np.ones((8, 5))
    phi[3, 2] = np.nan
    _, bits = gpu_step(sl, ctx, phi, gv, 0.0, dt, sl.options(sl.C_BOUNDARY, 4))
    assert bits & sl.ST_NONFINITE
    phi = 1.0 + 0.3 * sl_inputs.random_state((8, 5), 1)
    _, bits = gpu_step(sl, ctx, phi, gv, 0.0, dt, sl.options(7, 4, picard_rtol=1e-300, picard_cap=1))
    assert bits & sl.ST_PICARD_NOCONV
    a = torch.zeros(40, device="cuda", dtype=torch.float64)
    with pytest.raises(sl.SlError) as e:
        ctx.step(a, torch.empty_like(a), gv, 0.0, 0.2, sl.options())
    assert e.value.status == sl.SL_ECFL
    with pytest.raises(ValueError):
        ctx.step(a.float(), torch.empty_like(a), gv, 0.0, dt, sl.options())
    with pytest.raises(sl.SlError):
        ctx.step(a, a, gv, 0.0, dt, sl.options())


def test_run_host_matches_device_steps(sl):
    ctx, setup = make(sl, 200, 9)
    gv = sl.velocity(sl.VEL_CONST, 1.0)
    dt = ctx.max_dt(gv)
    phi = sl_inputs.random_state((200, 9), 2)
    opts = sl.options(3, 4)
    host_in = torch.tensor(phi.ravel()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ctx.run_host(host_in, host_out, gv, 0.0, dt, 3, opts)
    a = torch.tensor(phi, device="cuda")
    b = torch.empty_like(a)
    for s in range(3):
        ctx.step(a, b, gv, s * dt, dt, opts)
        a, b = b, a
    assert torch.equal(a.cpu().ravel(), host_out)


def test_energy_row_in_skip_band_fp64(sl):
    """Gaussian pulse, K = 256, n = 9, boundary + mass + energy: about 150 elements miss the energy
    target by a relative 1e-12 .. 1e-9 after the linear fit.  The oracle applies the energy row
    there (reading R7, threshold 1e-12), and so must the FP64 kernel: parity at 1e-12 holds on
    every element, including those of the band."""
    K, n = 256, 9
    ctx, setup = make(sl, K, n)
    gv = sl.velocity(sl.VEL_CONST, 1.0)
    dt = ctx.max_dt(gv, sl.RULE_PAPER)
    x, _ = ctx.node_coords()
    phi = np.exp(-((x - 0.5) / 0.05) ** 2)
    got, bits = gpu_step(sl, ctx, phi, gv, 0.0, dt, sl.options(7, 4))
    ref, infos = O.step_1d(setup, phi, O.StepOpts(O.Vel(O.VEL_CONST, (1.0, 0.0)), 0.0, dt, 7, 4))
    miss = np.array([infos[k]["energy_miss"] for k in range(K)])
    band = np.where((miss > 1e-12) & (miss <= 1e-9))[0]
    assert band.size > 100, band.size
    assert all(infos[k]["converged"] for k in range(K)) and bits == 0
    compare(setup, got, ref)
    relb = np.sqrt(np.sum((got[band] - ref[band]) ** 2) / np.sum(ref[band] ** 2))
    assert relb <= TOL_REL, relb
