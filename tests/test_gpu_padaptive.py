"""GPU parity of p-adaptive 2D meshes (per-element node counts, CSR state) and of batches of
independent problems, through the C ABI, against the FP64 oracle (which reads each
p-nonconforming face the same way: the neighbour's remapped polynomial at this element's face
points; the face flux with the Gauss rule of the finer side).

Bounds: FP64 relative L2 <= 1e-12 per step; mixed <= 1e-6 after 1 and 1000 steps.  A batch
step equals the problems' own steps exactly (same kernels, same arithmetic)."""
import numpy as np
import pytest

import sl_inputs
from oracle import sl_oracle as O

# The mixed paths decide the energy row's skip at a 1e-9 relative miss (the float resolution of
# the mismatch they form from increments); the oracle takes the same threshold for them.  FP64
# comparisons use the oracle's default of 1e-12.
MIXED_SKIP = 1e-9

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL64 = 1e-12
TOLM = 1e-6


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06476_gb300 import build as B
    B.build()
    import paper_1910_06476_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def to_nested(flat, orders):
    ky, kx = orders.shape
    out, o = [], 0
    for ey in range(ky):
        row = []
        for ex in range(kx):
            n = int(orders[ey, ex])
            row.append(np.asarray(flat[o:o + n * n]).reshape(n, n))
            o += n * n
        out.append(row)
    return out


def to_flat(nested):
    return np.concatenate([e.ravel() for row in nested for e in row])


VELS = {"rot": (1, (2 * np.pi, 0.5, 0.5)), "const": (0, (0.7, -0.4)), "swirl": (2, (5.0,))}
DATA = {"hill": sl_inputs.hill_2d, "bell": sl_inputs.cosine_bell_2d,
        "sincos": lambda x, y: 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)}

CASES = [
    # kx, ky, order range, velocity, bc, cons, rk, data, seed
    (5, 4, (3, 9), "rot", 1, 3, 4, "hill", 1),
    (4, 4, (4, 8), "const", 0, 7, 4, "sincos", 2),
    (4, 4, (3, 7), "swirl", 1, 7, 4, "bell", 3),
    (3, 5, (2, 6), "rot", 1, 1, 3, "sincos", 4),
    (4, 3, (5, 12), "const", 0, 2, 2, "sincos", 5),
    (2, 2, (12, 17), "rot", 1, 3, 4, "sincos", 6),
]


def _setup(sl, case, precision):
    kx, ky, (lo, hi), vk, bc, cons, rk, data, seed = case
    orders = np.random.default_rng(seed).integers(lo, hi + 1, (ky, kx)).astype(np.int32)
    box = (0.0, 1.0, 0.0, 1.0)
    ghost = 0.1 if bc else 0.0
    ctx = sl.Context(2, kx, ky, box, int(orders.max()), 0, precision, (bc,) * 4, ghost, orders=orders)
    setup = O.Setup(2, kx, ky, box, int(orders.max()), 0, (bc,) * 4, ghost, orders)
    kind, p = VELS[vk]
    gv = sl.velocity(kind, *p)
    ov = O.Vel(kind, tuple(p) + (0,) * (6 - len(p)))
    x, y = ctx.node_coords()
    phi = DATA[data](x, y) + 0.02 * sl_inputs.random_state(x.shape, seed)
    dt = ctx.max_dt(gv, sl.RULE_PAPER)
    return ctx, setup, orders, gv, ov, phi, dt, cons, rk


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}n{c[2][0]}-{c[2][1]}{c[3]}c{c[5]}" for c in CASES])
def test_padaptive_step_parity(sl, case, precision):
    prec = sl.FP64 if precision == "fp64" else sl.MIXED
    ctx, setup, orders, gv, ov, phi, dt, cons, rk = _setup(sl, case, prec)
    a = ctx.pack(torch.tensor(phi.ravel(), device="cuda"))
    b = ctx.new_state()
    ctx.step(a, b, gv, 0.2, dt, sl.options(cons, rk))
    bits = ctx.sync()
    got = ctx.unpack(b).cpu().numpy()
    ref, infos = O.step_2d(setup, to_nested(phi.ravel(), orders), O.StepOpts(ov, 0.2, dt, cons, rk,
                                                                          energy_skip_rtol=None if prec == sl.FP64 else MIXED_SKIP))
    conv = np.array([i["converged"] for i in infos.values()])
    assert bits & ~sl.ST_PICARD_NOCONV == 0, bits
    if conv.all():
        assert bits == 0, bits
    err = rel(got, to_flat(ref))
    assert err <= (TOL64 if prec == sl.FP64 else TOLM), err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uniform_orders_match_uniform_mesh(sl, precision):
    """A p-adaptive mesh whose elements all have the same node count advances exactly like the
    uniform mesh (same kernels through the element map)."""
    prec = sl.FP64 if precision == "fp64" else sl.MIXED
    kx, ky, n = 6, 5, 6
    box = (0.0, 1.0, 0.0, 1.0)
    u = sl.Context(2, kx, ky, box, n, 0, prec, (1,) * 4, 0.0)
    m = sl.Context(2, kx, ky, box, n, 0, prec, (1,) * 4, 0.0, orders=np.full((ky, kx), n))
    gv = sl.velocity(1, 2 * np.pi, 0.5, 0.5)
    x, y = u.node_coords()
    phi = torch.tensor(sl_inputs.hill_2d(x, y).ravel() + 0.01 * sl_inputs.random_state(x.size, 9), device="cuda")
    dt = u.max_dt(gv, sl.RULE_PAPER)
    au, bu, am, bm = u.pack(phi), u.new_state(), m.pack(phi), m.new_state()
    for s in range(3):
        u.step(au, bu, gv, s * dt, dt, sl.options(3, 4))
        m.step(am, bm, gv, s * dt, dt, sl.options(3, 4))
        au, bu, am, bm = bu, au, bm, am
    assert u.sync() == 0 and m.sync() == 0
    assert torch.equal(u.unpack(au), m.unpack(am))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_problems(sl, precision):
    """A batch of three problems (uniform, p-adaptive, uniform; different sizes and steps) advances
    each problem exactly as its own context does."""
    prec = sl.FP64 if precision == "fp64" else sl.MIXED
    box = (0.0, 1.0, 0.0, 1.0)
    gv = sl.velocity(1, 2 * np.pi, 0.5, 0.5)
    probs = [sl.Context(2, 6, 5, box, 5, 0, prec, (1,) * 4, 0.0),
             sl.Context(2, 4, 4, box, 9, 0, prec, (1,) * 4, 0.0,
                        orders=np.random.default_rng(3).integers(3, 10, (4, 4))),
             sl.Context(2, 3, 7, box, 7, 0, prec, (1,) * 4, 0.0)]
    batch = sl.Batch(probs)
    assert batch.offset(len(probs)) == batch.size == sum(p.size for p in probs)
    states, phis = [], []
    for i, p in enumerate(probs):
        x, y = p.node_coords()
        phi = torch.tensor((sl_inputs.hill_2d(x, y) + 0.01 * sl_inputs.random_state(x.shape, i)).ravel(),
                           device="cuda")
        phis.append(phi)
        states.append(p.pack(phi))
    dts = [p.max_dt(gv, sl.RULE_PAPER) for p in probs]
    ba = batch.pack(torch.cat(phis))
    bb = batch.new_state()
    opts = sl.options(3, 4)
    for s in range(2):
        outs = []
        for p, a, dt in zip(probs, states, dts):
            o = p.new_state()
            p.step(a, o, gv, s * dt, dt, opts)
            outs.append(o)
        states = outs
        batch.batch_step(ba, bb, gv, [s * d for d in dts], dts, opts)
        ba, bb = bb, ba
    assert batch.sync() == 0 and all(p.sync() == 0 for p in probs)
    got = batch.unpack(ba)
    for i, (p, st) in enumerate(zip(probs, states)):
        assert torch.equal(got[batch.offset(i):batch.offset(i + 1)], p.unpack(st)), i


def test_padaptive_mass_telescopes(sl):
    """Periodic p-adaptive mesh with the mass row: the face fluxes of neighbours of different
    node counts use the same points, so global mass is constant to rounding."""
    kx = ky = 6
    orders = np.random.default_rng(11).integers(3, 10, (ky, kx))
    box = (0.0, 1.0, 0.0, 1.0)
    ctx = sl.Context(2, kx, ky, box, 9, 0, sl.FP64, (0,) * 4, 0.0, orders=orders)
    gv = sl.velocity(0, 0.8, 0.45)
    x, y = ctx.node_coords()
    a = torch.tensor(DATA["sincos"](x, y).ravel(), device="cuda")
    b = torch.empty_like(a)
    m0 = ctx.mass(a)
    dt = ctx.max_dt(gv, sl.RULE_PAPER)
    for s in range(20):
        ctx.step(a, b, gv, s * dt, dt, sl.options(3, 4))
        a, b = b, a
    assert ctx.sync() == 0
    assert abs(ctx.mass(a) - m0) <= 1e-13 * abs(m0)


def test_config4_mixed_against_fp64(sl):
    """Config 4 at full size: 256 x 256 elements, node counts n in 4..16 drawn with seed 0
    (7.46M nodes), rotation, inflow ghost 0, boundary + mass.  Mixed vs the FP64 GPU path after
    1 and 1000 steps, and 48 sampled elements recomputed by the oracle from the mixed state."""
    prob = sl_inputs.config4_rotation()
    K = prob.kx
    orders = prob.orders
    c64 = sl.Context(2, K, K, prob.box, 16, 0, sl.FP64, prob.bc, prob.ghost, orders=orders)
    cm = sl.Context(2, K, K, prob.box, 16, 0, sl.MIXED, prob.bc, prob.ghost, orders=orders)
    assert c64.size == int(np.sum(orders.astype(np.int64) ** 2))
    gv = sl.velocity(1, 2 * np.pi, 0.5, 0.5)
    dt = c64.max_dt(gv, sl_inputs.rule_code(prob))
    x, y = c64.node_coords()
    phi = torch.tensor(prob.phi0(x, y), device="cuda")
    del x, y
    a64, b64 = phi.clone(), torch.empty_like(phi)
    am, bm = cm.pack(phi), cm.new_state()
    opts = sl.options(prob.constraints, 4)
    errs = {}
    pre = None
    for s in range(1000):
        if s == 999:
            pre = cm.unpack(am).cpu().numpy()
        c64.step(a64, b64, gv, s * dt, dt, opts)
        cm.step(am, bm, gv, s * dt, dt, opts)
        a64, b64 = b64, a64
        am, bm = bm, am
        if s + 1 in (1, 1000):
            d = cm.unpack(am) - a64
            errs[s + 1] = (d.norm() / a64.norm()).item()
    assert c64.sync() == 0 and cm.sync() == 0
    assert errs[1] <= TOLM and errs[1000] <= TOLM, errs
    # sampled oracle check of the last step, from the mixed pre-step state
    setup = O.setup_from_problem(prob)
    got = to_nested(cm.unpack(am).cpu().numpy(), orders)
    pre_n = to_nested(pre, orders)
    idx = sl_inputs.sample_elements(40, K * K, 7)
    elems = [(int(e % K), int(e // K)) for e in idx] + [(0, 0), (K - 1, 0), (0, K - 1), (K - 1, K - 1),
                                                         (64, 128), (65, 128), (128, 64), (128, 65)]
    ref, _ = O.step_2d(setup, pre_n, O.StepOpts(O.Vel(O.VEL_ROTATION, (2 * np.pi, 0.5, 0.5, 0, 0, 0)), 999 * dt,
                                                dt, prob.constraints, 4), elements=elems)
    g = np.concatenate([got[ey][ex].ravel() for ex, ey in elems])
    r = np.concatenate([ref[ey][ex].ravel() for ex, ey in elems])
    assert rel(g, r) <= TOLM
