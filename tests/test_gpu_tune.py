"""The launch-shape autotuner (sl_tune): it picks among compiled tile shapes (elements per CTA) of
the 2D shared-operator kernel and among resident-CTA counts of the general mixed kernels'
persistent grids, records the choice in a JSON cache, and applies a cached choice without timing.
The grid size leaves every element's arithmetic as it is (bitwise equal results); the tile shapes
are separate compilations of the same per-element arithmetic, whose floating-point contractions
the compiler may schedule differently, so they agree to the float rounding of the increments."""
import json

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


def _setup(sl, kx, ky, n, vel, cons, ghost=0.0, bc=0):
    ctx = sl.Context(2, kx, ky, (0.0, 1.0, 0.0, 1.0), n, 0, sl.MIXED, (bc,) * 4, ghost)
    x, y = ctx.node_coords()
    phi = 1.0 + 0.4 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.02 * sl_inputs.random_state(x.shape, n)
    a = ctx.pack(torch.tensor(phi.ravel(), device="cuda"))
    return ctx, a, ctx.max_dt(vel, sl.RULE_PAPER), sl.options(cons, 4)


def _force(path, key_prefix, value):
    """Rewrite every entry of the cache whose key starts with key_prefix."""
    data = json.loads(path.read_text())
    for k in data:
        if k.startswith(key_prefix):
            data[k] = value
    path.write_text(json.dumps(data))


@pytest.mark.parametrize("n", [5, 9, 11, 14])
def test_tune_shared_operator_tiles(sl, tmp_path, n):
    vel = sl.velocity(sl.VEL_CONST, 0.7, -0.4)
    ctx, a, dt, opts = _setup(sl, 13, 11, n, vel, sl.C_BOUNDARY | sl.C_MASS, bc=1, ghost=0.2)
    cache = tmp_path / "tune.json"
    b = ctx.new_state()
    r = ctx.tune(a, b, vel, 0.1, dt, opts, cache)
    assert not r["cached"] and 0 <= r["tile"] <= 2
    data = json.loads(cache.read_text())
    assert len(data) == 1 and next(iter(data)).startswith("k2c_tile|")
    # the same key again: applied from the cache, no timing
    ctx2, a2, _, _ = _setup(sl, 13, 11, n, vel, sl.C_BOUNDARY | sl.C_MASS, bc=1, ghost=0.2)
    assert ctx2.tune(a2, ctx2.new_state(), vel, 0.1, dt, opts, cache)["cached"]
    # every candidate tile gives the same result to float rounding
    outs = []
    for tile in range(3 if n <= 12 else 2):
        _force(cache, "k2c_tile|", f"tile={tile}")
        c = sl.Context(2, 13, 11, (0.0, 1.0, 0.0, 1.0), n, 0, sl.MIXED, (1,) * 4, 0.2)
        assert c.tune(a, c.new_state(), vel, 0.1, dt, opts, cache) == {
            "tile": tile, "per_sm_phase1": 0, "per_sm_phase2": 0, "cached": True}
        out = c.new_state()
        c.step(a, out, vel, 0.1, dt, opts)
        assert c.sync() == 0
        outs.append(c.unpack(out))
    for o in outs[1:]:
        rel = ((o - outs[0]).norm() / outs[0].norm()).item()
        assert rel <= 1e-7, rel                  # a wrong shape would differ at O(1)


def test_tune_general_kernel_per_sm(sl, tmp_path):
    vel = sl.velocity(sl.VEL_SWIRL, 5.0)
    ctx, a, dt, opts = _setup(sl, 40, 40, 8, vel, sl.C_BOUNDARY | sl.C_MASS | sl.C_ENERGY, bc=1)
    cache = tmp_path / "tune.json"
    r = ctx.tune(a, ctx.new_state(), vel, 0.0, dt, opts, cache)
    assert not r["cached"] and r["per_sm_phase1"] in (0, 1, 2) and r["per_sm_phase2"] in (0, 1, 2)
    outs = []
    for p1, p2 in ((0, 0), (1, 2), (2, 1)):
        _force(cache, "k2m_per_sm|", f"p1={p1},p2={p2}")
        c = sl.Context(2, 40, 40, (0.0, 1.0, 0.0, 1.0), 8, 0, sl.MIXED, (1,) * 4, 0.0)
        r = c.tune(a, c.new_state(), vel, 0.0, dt, opts, cache)
        assert r["cached"] and (r["per_sm_phase1"], r["per_sm_phase2"]) == (p1, p2)
        out = c.new_state()
        c.step(a, out, vel, 0.0, dt, opts)
        c.sync()
        outs.append(out)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_tune_nothing_to_tune_and_bad_cache(sl, tmp_path):
    c = sl.Context(1, 50, 1, (0.0, 1.0, 0.0, 0.0), 6, 0, sl.FP64, (0,) * 4, 0.0)
    a = torch.zeros(c.size, dtype=torch.float64, device="cuda")
    vel = sl.velocity(sl.VEL_CONST, 1.0)
    r = c.tune(a, torch.empty_like(a), vel, 0.0, 1e-3, sl.options(1, 4), tmp_path / "none.json")
    assert r == {"tile": 0, "per_sm_phase1": 0, "per_sm_phase2": 0, "cached": False}
    assert not (tmp_path / "none.json").exists()
    bad = tmp_path / "bad.json"
    bad.write_text("[1, 2]")
    vel2 = sl.velocity(sl.VEL_CONST, 0.7, -0.4)
    ctx, a2, dt, opts = _setup(sl, 8, 8, 5, vel2, sl.C_BOUNDARY)
    with pytest.raises(sl.SlError):
        ctx.tune(a2, ctx.new_state(), vel2, 0.0, dt, opts, bad)
