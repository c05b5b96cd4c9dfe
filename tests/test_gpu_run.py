"""sl_run (steps captured into a CUDA graph and replayed) against the same steps taken one
sl_step call at a time: the graph launches the same kernels with the same arguments, so the
states agree exactly, on every path (1D FP64 and mixed, 2D FP64, the 2D mixed general and
shared-operator kernels, p-adaptive meshes and batches)."""
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


BOX = (0.0, 1.0, 0.0, 1.0)


def _case(sl, name):
    if name == "1d_fp64":
        ctx = sl.Context(1, 16, 1, (0.0, 1.0, 0.0, 1.0), 9, 0, sl.FP64, (0, 0, 0, 0))
        vel, cons = sl.velocity(0, 1.0), 3
    elif name == "1d_mixed":
        ctx = sl.Context(1, 4096, 1, (0.0, 1.0, 0.0, 1.0), 9, 0, sl.MIXED, (0, 0, 0, 0))
        vel, cons = sl.velocity(0, 1.0), 7
    elif name == "2d_fp64":
        ctx = sl.Context(2, 6, 5, BOX, 6, 0, sl.FP64, (1,) * 4, 0.0)
        vel, cons = sl.velocity(1, 2 * np.pi, 0.5, 0.5), 3
    elif name == "2d_mixed_general":
        ctx = sl.Context(2, 6, 5, BOX, 6, 0, sl.MIXED, (1,) * 4, 0.0)
        vel, cons = sl.velocity(1, 2 * np.pi, 0.5, 0.5), 3
    elif name == "2d_mixed_shared":
        ctx = sl.Context(2, 20, 12, BOX, 9, 0, sl.MIXED, (0,) * 4, 0.0)
        vel, cons = sl.velocity(0, 1.0, 0.5), 3
    elif name == "2d_padaptive":
        ctx = sl.Context(2, 5, 4, BOX, 9, 0, sl.MIXED, (1,) * 4, 0.0,
                         orders=np.random.default_rng(2).integers(3, 10, (4, 5)))
        vel, cons = sl.velocity(1, 2 * np.pi, 0.5, 0.5), 3
    else:
        raise KeyError(name)
    x, y = ctx.node_coords()
    f = np.sin(2 * np.pi * x) if ctx.dim == 1 else sl_inputs.hill_2d(x, y) + 0.3 * np.cos(2 * np.pi * x)
    phi = torch.tensor(np.ascontiguousarray(f).ravel(), device="cuda")
    return ctx, vel, sl.options(cons, 4), phi


def _steps(ctx, a, vel, t0, dt, n, opts):
    b = ctx.new_state()
    for s in range(n):
        ctx.step(a, b, vel, t0 + s * dt, dt, opts)
        a, b = b, a
    return a


@pytest.mark.parametrize("name", ["1d_fp64", "1d_mixed", "2d_fp64", "2d_mixed_general", "2d_mixed_shared",
                                  "2d_padaptive"])
def test_run_equals_steps(sl, name):
    ctx, vel, opts, phi = _case(sl, name)
    dt = ctx.max_dt(vel, sl.RULE_PAPER)
    ref = ctx.unpack(_steps(ctx, ctx.pack(phi), vel, 0.1, dt, 7, opts))
    for _ in range(2):                         # capture, then replay of the cached graph
        a, b = ctx.pack(phi), ctx.new_state()
        out = ctx.run(a, b, vel, 0.1, dt, 7, opts)
        assert out is b
        assert torch.equal(ctx.unpack(out), ref)
    a, b = ctx.pack(phi), ctx.new_state()      # another step count: a new capture
    out = ctx.run(a, b, vel, 0.1, dt, 4, opts)
    assert out is a
    assert torch.equal(ctx.unpack(out), ctx.unpack(_steps(ctx, ctx.pack(phi), vel, 0.1, dt, 4, opts)))
    assert ctx.sync() == 0


def test_run_replay_after_operator_change(sl):
    """A cached graph reads the shared operator; a step with another dt rebuilds that operator, so
    the replay must restore the operator of its own dt first."""
    ctx, vel, opts, phi = _case(sl, "2d_mixed_shared")
    dt = ctx.max_dt(vel, sl.RULE_PAPER)
    ref = ctx.unpack(_steps(ctx, ctx.pack(phi), vel, 0.0, dt, 3, opts))
    a, b = ctx.pack(phi), ctx.new_state()
    ctx.run(a, b, vel, 0.0, dt, 3, opts)
    _steps(ctx, ctx.pack(phi), vel, 0.0, 0.5 * dt, 1, opts)
    a, b = ctx.pack(phi), ctx.new_state()
    out = ctx.run(a, b, vel, 0.0, dt, 3, opts)
    assert torch.equal(ctx.unpack(out), ref)


def test_run_batch(sl):
    probs = [sl.Context(2, 6, 5, BOX, 5, 0, sl.MIXED, (1,) * 4, 0.0),
             sl.Context(2, 4, 4, BOX, 9, 0, sl.MIXED, (1,) * 4, 0.0,
                        orders=np.random.default_rng(5).integers(3, 10, (4, 4)))]
    batch = sl.Batch(probs)
    vel = sl.velocity(1, 2 * np.pi, 0.5, 0.5)
    opts = sl.options(3, 4)
    dt = batch.max_dt(vel, sl.RULE_PAPER)
    phis = []
    for p in probs:
        x, y = p.node_coords()
        phis.append(torch.tensor(sl_inputs.hill_2d(x, y).ravel(), device="cuda"))
    phi = torch.cat(phis)
    ref = batch.unpack(_steps(batch, batch.pack(phi), vel, 0.0, dt, 5, opts))
    a, b = batch.pack(phi), batch.new_state()
    out = batch.run(a, b, vel, 0.0, dt, 5, opts)
    assert torch.equal(batch.unpack(out), ref)
    assert batch.sync() == 0
