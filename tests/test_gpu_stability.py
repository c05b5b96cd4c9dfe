"""The time-step restriction of the paper (eq. 1d_delt_condition, 2d_delt_condition: the gap from
the element edge to its first node over |u|max, so that no particle leaves its element) is what
keeps the scheme stable for non-uniform velocity on coarse meshes.  With twice that displacement
(half the minimum node spacing) particles leave their elements and the rotation and swirl runs grow
without bound, for every constraint set and fit; with the paper's step they stay bounded at 24 x 24
elements.  On fine meshes the paper's step is itself the limit (half of it is what the deforming
configurations run at; test_gpu_long_horizon).  FP64 path, n = 8."""
import numpy as np
import pytest

import sl_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06476_gb300 import build as B
    B.build()
    import paper_1910_06476_gb300 as pkg
    return pkg


def run_max(sl, kind, p, data, rule, steps, cons=3):
    c = sl.Context(2, 24, 24, (0, 1, 0, 1), 8, 0, sl.FP64, (1,) * 4, 0.0)
    gv = sl.velocity(kind, *p)
    dt = c.max_dt(gv, rule)
    x, y = c.node_coords()
    a = torch.tensor(data(x, y).ravel(), device="cuda")
    b = torch.empty_like(a)
    for s in range(steps):
        c.step(a, b, gv, s * dt, dt, sl.options(cons, 4))
        a, b = b, a
    c.sync()
    return a.abs().max().item()


@pytest.mark.parametrize("kind,p,data", [(2, (5.0,), sl_inputs.cosine_bell_2d),
                                         (1, (2 * np.pi, 0.5, 0.5), sl_inputs.hill_2d)])
def test_paper_time_step_is_stable_half_spacing_is_not(sl, kind, p, data):
    assert run_max(sl, kind, p, data, sl.RULE_PAPER, 600) <= 1.01
    assert not run_max(sl, kind, p, data, sl.RULE_HALF_MIN_SPACING, 600) <= 10.0


def test_swirl_amplification_fp64(sl):
    """The amplification that makes the paper's step the stability limit on the swirl is a
    property of the scheme, not of the float arithmetic: in FP64 (config 5's problem, 256 x 256,
    n = 8, boundary + mass, the paper's step) a 1e-12 perturbation grows by more than 1e3 within
    300 steps (at 512 x 512 it runs away: test_gpu_long_horizon), while the solution stays bounded."""
    prob = sl_inputs.config5_swirl(n=8, k=256)
    c = sl.Context(2, 256, 256, prob.box, 8, 0, sl.FP64, prob.bc, prob.ghost)
    gv = sl.velocity(sl.VEL_SWIRL, 5.0)
    dt = c.max_dt(gv, sl.RULE_PAPER)
    x, y = c.node_coords()
    phi = torch.tensor(prob.phi0(x, y).ravel(), device="cuda")
    pert = torch.tensor(sl_inputs.random_state(phi.shape, 5), device="cuda") * 1e-12 * (phi != 0)
    a1 = c.run(phi.clone(), torch.empty_like(phi), gv, 0.0, dt, 300, sl.options(3, 4))
    a2 = c.run(phi + pert, torch.empty_like(phi), gv, 0.0, dt, 300, sl.options(3, 4))
    c.sync()
    growth = (a2 - a1).abs().max().item() / 1e-12
    assert growth > 1e3, growth
    assert a1.abs().max().item() <= 1.01
