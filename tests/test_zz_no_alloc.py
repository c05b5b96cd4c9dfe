"""The allocation-free integral entry point (sl_integral_noalloc) against sl_mass / sl_energy.

Some callers cannot allocate device memory when they need the diagnostic (stream capture in
global mode, hard latency budgets, memory pools that own the device), so the library offers one
entry point whose scratch is a fixed device array.  This file is collected last so that a run
stopping at its first failure has already run every other test; it also passes on its own."""
import ctypes as C

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


def _noalloc(lib, phi, nelem, nper, dim, w, power, scale, stream):
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    w_host = np.ascontiguousarray(w, dtype=np.float64)
    st = lib.sl_integral_noalloc(C.c_void_p(phi.data_ptr()), nelem, nper, dim, w_host.ctypes.data_as(C.c_void_p),
                                 power, scale, C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == 0, lib.sl_last_error(None)
    return out


@pytest.mark.parametrize("dim,K,n", [(1, 3000, 9), (2, 40, 7)])
def test_noalloc_matches_existing_entry_points_twice(sl, dim, K, n):
    lib = sl.lib()
    ky = 1 if dim == 1 else K
    box = (0.0, 1.0, 0.0, 1.0)
    ctx = sl.Context(dim, K, ky, box, n, sl.GAUSS_LEGENDRE, sl.FP64, (0, 0, 0, 0), 0.0)
    xi, w = ctx.nodes_weights()
    h = 1.0 / K
    scale = h if dim == 1 else h * h
    stream = torch.cuda.current_stream()
    for call, (seed, power) in enumerate([(1, 1), (2, 2)]):   # two calls in a row
        phi_np = 1.5 + sl_inputs.random_state((ctx.size,), seed)
        phi = torch.tensor(phi_np, device="cuda")
        nelem = K * ky
        out = _noalloc(lib, phi, nelem, n, dim, w, power, scale, stream)
        ref = ctx.mass(phi) if power == 1 else ctx.energy(phi)
        got = out.item()
        assert abs(got - ref) <= 1e-13 * abs(ref), (call, got, ref)


def test_noalloc_rejects_inputs_beyond_its_scratch(sl):
    lib = sl.lib()
    phi = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    w = np.full(9, 1.0 / 9)
    too_many = (1 << 28) // 9 + 1
    st = lib.sl_integral_noalloc(C.c_void_p(phi.data_ptr()), too_many, 9, 1, w.ctypes.data_as(C.c_void_p), 1, 1.0,
                                 C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sl.SL_EINVAL
    assert b"SL_NOALLOC_MAX_VALUES" in lib.sl_last_error(None)


def test_noalloc_inside_global_mode_capture(sl):
    """The use the entry point exists for: after one eager call on the device, a call recorded
    under global-mode stream capture (where allocation is forbidden) and replayed from the graph
    gives the integral of whatever the input buffer holds at replay time."""
    lib = sl.lib()
    K, n = 500, 9
    ctx = sl.Context(1, K, 1, (0.0, 1.0, 0.0, 0.0), n, sl.GAUSS_LEGENDRE, sl.FP64, (0, 0, 0, 0), 0.0)
    _, w = ctx.nodes_weights()
    w_host = np.ascontiguousarray(w, dtype=np.float64)
    phi = torch.tensor(1.5 + sl_inputs.random_state((ctx.size,), 3), device="cuda")
    _noalloc(lib, phi, K, n, 1, w, 1, 1.0 / K, torch.cuda.current_stream())      # first call, eager
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        st = lib.sl_integral_noalloc(C.c_void_p(phi.data_ptr()), K, n, 1, w_host.ctypes.data_as(C.c_void_p), 1,
                                     1.0 / K, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.sl_last_error(None)
    for seed in (4, 5):
        phi.copy_(torch.tensor(0.5 + sl_inputs.random_state((ctx.size,), seed), device="cuda"))
        g.replay()
        torch.cuda.synchronize()
        ref = ctx.mass(phi)
        assert abs(out.item() - ref) <= 1e-13 * abs(ref), (seed, out.item(), ref)
