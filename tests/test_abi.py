"""The C-ABI library loads and exports every function include/sl.h declares; host-side
argument checks reject bad input before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sl_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_06476_gb300 import build as B
    B.build()
    from paper_1910_06476_gb300 import binding
    return binding.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sl_init", "sl_step", "sl_mass", "sl_energy", "sl_free", "sl_sync"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1910_06476_gb300 import binding
    names = declared_functions()
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTS) == names


def _mesh(binding, **kw):
    m = binding.SlMesh()
    m.dim, m.kx, m.ky = kw.get("dim", 1), kw.get("kx", 4), kw.get("ky", 1)
    m.x0, m.x1, m.y0, m.y1 = 0.0, 1.0, 0.0, 1.0
    for i in range(4):
        m.bc[i] = kw.get("bc", 0)
    m.ghost = 0.0
    m.order = C.POINTER(C.c_int32)()
    return m


@pytest.mark.parametrize("kw,n", [({"dim": 3}, 5), ({"kx": 0}, 5), ({"dim": 1, "ky": 2}, 5), ({}, 1), ({}, 18),
                                  ({"bc": 7}, 5)])
def test_init_rejects_bad_arguments(lib, kw, n):
    from paper_1910_06476_gb300 import binding
    m = _mesh(binding, **kw)
    h = C.c_void_p()
    st = lib.sl_init(C.byref(m), n, 0, 0, None, C.byref(h))
    assert st == binding.SL_EINVAL
    assert h.value is None
    assert lib.sl_last_error(None)


def test_init_rejects_null_and_bad_enums(lib):
    from paper_1910_06476_gb300 import binding
    h = C.c_void_p()
    assert lib.sl_init(None, 5, 0, 0, None, C.byref(h)) == binding.SL_EINVAL
    m = _mesh(binding)
    assert lib.sl_init(C.byref(m), 5, 9, 0, None, C.byref(h)) == binding.SL_EINVAL
    assert lib.sl_init(C.byref(m), 5, 0, 9, None, C.byref(h)) == binding.SL_EINVAL


def test_null_context_calls_are_rejected(lib):
    from paper_1910_06476_gb300 import binding
    assert lib.sl_step(None, None, None, None, 0.0, 0.1, None) == binding.SL_EINVAL
    assert lib.sl_mass(None, None, None) == binding.SL_EINVAL
    assert lib.sl_state_size(None) == -1
    lib.sl_free(None)
