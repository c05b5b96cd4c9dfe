"""Thin ctypes binding of the DSEM-SL C ABI (include/sl.h).

Argument marshalling only: every step of the method runs in the CUDA library.  PyTorch is
used for device memory and streams.  The library must have been built
(``paper_1910_06476_gb300.build.build()``); importing this module raises if it is missing."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsl.so")

SL_OK, SL_EINVAL, SL_ENOMEM, SL_ECUDA, SL_ECFL, SL_EDEVICE, SL_EUNSUPPORTED = range(7)
GAUSS_LEGENDRE, CHEB_GAUSS = 0, 1
FP64, MIXED = 0, 1
BC_PERIODIC, BC_INFLOW = 0, 1
INFLOW_RECORD = 10                       # doubles per step of sl_set_inflow
VEL_CONST, VEL_ROTATION, VEL_SWIRL, VEL_SINX, VEL_NODAL = 0, 1, 2, 3, 4
C_BOUNDARY, C_MASS, C_ENERGY = 1, 2, 4
FIT_HARD, FIT_SOFT = 0, 1
BV_INTERP, BV_BACKTRACK = 0, 1
RULE_HALF_MIN_SPACING, RULE_PAPER, RULE_HALF_PAPER = 0, 1, 2
ST_NONFINITE, ST_PICARD_NOCONV, ST_SOLVE_NOCONV, ST_TIMEOUT, ST_SOLVE_FLOOR = 1, 2, 4, 8, 16
COUNTERS = ("elems", "solve_iters", "solve_floor", "solve_noconv", "energy_applied", "picard_iters",
            "picard_noconv", "feet")

EXPORTS = ["sl_init", "sl_free", "sl_step", "sl_run", "sl_run_host", "sl_pack", "sl_unpack", "sl_mass", "sl_energy",
           "sl_sync", "sl_max_dt", "sl_state_size", "sl_state_bytes", "sl_node_coords", "sl_nodes_weights",
           "sl_integral_noalloc", "sl_batch_create", "sl_batch_step", "sl_batch_offset", "sl_counters",
           "sl_timing", "sl_timing_read", "sl_set_inflow", "sl_tune", "sl_last_error"]


class SlMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("kx", C.c_int), ("ky", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("bc", C.c_int * 4), ("ghost", C.c_double), ("order", C.POINTER(C.c_int32))]


class SlVelocity(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 6), ("nodal", C.c_void_p), ("nodal_step", C.c_int64)]


class SlOptions(C.Structure):
    _fields_ = [("constraints", C.c_uint), ("rk_order", C.c_int), ("fit", C.c_int), ("bvalue", C.c_int),
                ("picard_rtol", C.c_double), ("picard_cap", C.c_int)]


class SlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sl status {status}: {msg}")
        self.status = status


def load_library(path=LIB_PATH):
    """Load libsl.so and declare every exported signature.  Raises if it was not built."""
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1910_06476_gb300.build.build() "
                          "(the library has no CPU fallback)")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.sl_init.argtypes = [C.POINTER(SlMesh), C.c_int, C.c_int, C.c_int, P, C.POINTER(P)]
    lib.sl_free.argtypes = [P]
    lib.sl_free.restype = None
    lib.sl_step.argtypes = [P, P, P, C.POINTER(SlVelocity), C.c_double, C.c_double, C.POINTER(SlOptions)]
    lib.sl_run_host.argtypes = [P, P, P, C.POINTER(SlVelocity), C.c_double, C.c_double, C.c_int,
                                C.POINTER(SlOptions)]
    lib.sl_run.argtypes = [P, P, P, C.POINTER(SlVelocity), C.c_double, C.c_double, C.c_int, C.POINTER(SlOptions)]
    lib.sl_pack.argtypes = [P, P, P]
    lib.sl_unpack.argtypes = [P, P, P]
    lib.sl_state_bytes.argtypes = [P]
    lib.sl_state_bytes.restype = C.c_int64
    lib.sl_mass.argtypes = [P, P, C.POINTER(C.c_double)]
    lib.sl_energy.argtypes = [P, P, C.POINTER(C.c_double)]
    lib.sl_sync.argtypes = [P, C.POINTER(C.c_uint32)]
    lib.sl_counters.argtypes = [P, C.POINTER(C.c_uint64)]
    lib.sl_timing.argtypes = [P, C.c_int]
    lib.sl_set_inflow.argtypes = [P, P, C.c_int64]
    lib.sl_tune.argtypes = [P, P, P, C.POINTER(SlVelocity), C.c_double, C.c_double, C.POINTER(SlOptions), C.c_char_p,
                            C.POINTER(C.c_int)]
    lib.sl_timing_read.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.sl_max_dt.argtypes = [P, C.POINTER(SlVelocity), C.c_int, C.POINTER(C.c_double)]
    lib.sl_state_size.argtypes = [P]
    lib.sl_state_size.restype = C.c_int64
    lib.sl_node_coords.argtypes = [P, P, P]
    lib.sl_nodes_weights.argtypes = [P, C.c_int, P, P]
    lib.sl_integral_noalloc.argtypes = [P, C.c_int64, C.c_int, C.c_int, P, C.c_int, C.c_double, P, P]
    lib.sl_batch_create.argtypes = [C.c_int, C.POINTER(P), C.POINTER(P)]
    lib.sl_batch_step.argtypes = [P, P, P, C.POINTER(SlVelocity), P, P, C.POINTER(SlOptions)]
    lib.sl_batch_offset.argtypes = [P, C.c_int]
    lib.sl_batch_offset.restype = C.c_int64
    lib.sl_last_error.argtypes = [P]
    lib.sl_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("sl_free", "sl_state_size", "sl_state_bytes", "sl_batch_offset", "sl_last_error"):
            getattr(lib, name).restype = C.c_int
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def velocity(kind, *p):
    v = SlVelocity()
    v.kind = int(kind)
    for i, x in enumerate(p[:6]):
        v.p[i] = float(x)
    return v


def nodal_velocity(values, umax, vmax=0.0, step=0):
    """SL_VEL_NODAL from a contiguous CUDA float64 tensor of node velocities laid out
    [2][dim][state values] (u, v at t and at t + dt); umax, vmax bound |u|, |v|.  The returned
    structure keeps the tensor referenced."""
    import torch
    if not (values.is_cuda and values.dtype == torch.float64 and values.is_contiguous()):
        raise ValueError("nodal velocity: a contiguous CUDA float64 tensor")
    v = velocity(VEL_NODAL, umax, vmax)
    v.nodal = values.data_ptr()
    v.nodal_step = int(step)
    v._keep = values
    return v


def options(constraints=C_BOUNDARY, rk_order=4, fit=FIT_HARD, bvalue=BV_INTERP, picard_rtol=0.0, picard_cap=0):
    o = SlOptions()
    o.constraints, o.rk_order, o.fit, o.bvalue = int(constraints), int(rk_order), int(fit), int(bvalue)
    o.picard_rtol, o.picard_cap = float(picard_rtol), int(picard_cap)
    return o


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Context:
    """One mesh on one GPU stream (sl_init ... sl_free)."""

    def __init__(self, dim, kx, ky, box, n, basis=GAUSS_LEGENDRE, precision=FP64, bc=(0, 0, 0, 0),
                 ghost=0.0, stream=None, orders=None):
        """orders: optional (ky, kx) integer array of per-element node counts (p-adaptive 2D
        mesh); the state is then flat, element by element (row-major), n_e^2 values each."""
        import torch
        self._lib = lib()
        m = SlMesh()
        m.dim, m.kx, m.ky = int(dim), int(kx), int(ky)
        m.x0, m.x1, m.y0, m.y1 = [float(v) for v in box]
        for i in range(4):
            m.bc[i] = int(bc[i])
        m.ghost = float(ghost)
        self.orders = None
        if orders is not None:
            self.orders = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(ky, kx))
            m.order = self.orders.ctypes.data_as(C.POINTER(C.c_int32))
        else:
            m.order = C.POINTER(C.c_int32)()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = self._lib.sl_init(C.byref(m), int(n), int(basis), int(precision),
                               C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SL_OK:
            raise SlError(st, self._lib.sl_last_error(None).decode())
        self._h = h
        self.dim, self.kx, self.ky, self.n, self.precision = dim, kx, ky, n, precision
        self._setup(h, precision)
        self.shape = (self.size,) if orders is not None else (kx, n) if dim == 1 else (ky, kx, n, n)

    def _setup(self, h, precision):
        import torch
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self.size = int(self._lib.sl_state_size(h))
        # number of state elements of self.dtype in one state buffer (two float planes when mixed)
        self.numel = int(self._lib.sl_state_bytes(h)) // (8 if precision == FP64 else 4)

    def _check(self, st):
        if st != SL_OK:
            raise SlError(st, self._lib.sl_last_error(self._h).decode())

    def _state(self, t, name):
        if not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != self.numel:
            raise ValueError(f"{name} must be a contiguous CUDA {self.dtype} tensor of {self.numel} values")

    def new_state(self):
        import torch
        return torch.empty(self.numel, dtype=self.dtype, device="cuda")

    def pack(self, phi64):
        """Device doubles (state layout) -> a new state buffer in this context's format."""
        import torch
        if not phi64.is_cuda or phi64.dtype != torch.float64 or not phi64.is_contiguous() or phi64.numel() != self.size:
            raise ValueError("pack expects a contiguous CUDA float64 tensor of the state size")
        out = self.new_state()
        self._check(self._lib.sl_pack(self._h, _ptr(phi64), _ptr(out)))
        return out

    def unpack(self, state):
        """A state buffer -> a new CUDA float64 tensor of node values (state layout)."""
        import torch
        self._state(state, "state")
        out = torch.empty(self.size, dtype=torch.float64, device="cuda")
        self._check(self._lib.sl_unpack(self._h, _ptr(state), _ptr(out)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sl_free(self._h)
            self._h = None

    __del__ = close

    def step(self, phi_in, phi_out, vel, t, dt, opts):
        self._state(phi_in, "phi_in")
        self._state(phi_out, "phi_out")
        self._check(self._lib.sl_step(self._h, _ptr(phi_in), _ptr(phi_out), C.byref(vel), float(t), float(dt),
                                      C.byref(opts)))

    def run(self, phi_a, phi_b, vel, t0, dt, nsteps, opts):
        """nsteps graph-replayed steps alternating between phi_a (initial state) and phi_b;
        returns the buffer that holds the result."""
        self._state(phi_a, "phi_a")
        self._state(phi_b, "phi_b")
        self._check(self._lib.sl_run(self._h, _ptr(phi_a), _ptr(phi_b), C.byref(vel), float(t0), float(dt),
                                     int(nsteps), C.byref(opts)))
        return phi_a if nsteps % 2 == 0 else phi_b

    def run_host(self, host_in, host_out, vel, t0, dt, nsteps, opts):
        """host_in/host_out: CPU float64 tensors (pinned for speed) of node values."""
        import torch
        for t in (host_in, host_out):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != self.size:
                raise ValueError("host buffers must be contiguous CPU float64 tensors of the state size")
        self._check(self._lib.sl_run_host(self._h, C.c_void_p(host_in.data_ptr()), C.c_void_p(host_out.data_ptr()),
                                          C.byref(vel), float(t0), float(dt), int(nsteps), C.byref(opts)))

    def mass(self, phi):
        self._state(phi, "phi")
        out = C.c_double()
        self._check(self._lib.sl_mass(self._h, _ptr(phi), C.byref(out)))
        return out.value

    def energy(self, phi):
        self._state(phi, "phi")
        out = C.c_double()
        self._check(self._lib.sl_energy(self._h, _ptr(phi), C.byref(out)))
        return out.value

    def sync(self):
        bits = C.c_uint32()
        st = self._lib.sl_sync(self._h, C.byref(bits))
        if st not in (SL_OK, SL_EDEVICE):
            self._check(st)
        return bits.value

    def counters(self):
        """Work counters of the 2D mixed general kernels since the last call (sl_counters), by name."""
        arr = (C.c_uint64 * len(COUNTERS))()
        self._check(self._lib.sl_counters(self._h, arr))
        return dict(zip(COUNTERS, (int(v) for v in arr)))

    def set_inflow(self, values, step_stride=INFLOW_RECORD):
        """Time-dependent inflow records (sl_set_inflow): a CUDA float64 tensor of records of
        INFLOW_RECORD values per step (kept referenced here while set), or None."""
        if values is None:
            self._inflow = None
            self._check(self._lib.sl_set_inflow(self._h, None, 0))
            return
        import torch
        if not (values.is_cuda and values.dtype == torch.float64 and values.is_contiguous()):
            raise ValueError("inflow records: a contiguous CUDA float64 tensor")
        self._check(self._lib.sl_set_inflow(self._h, _ptr(values), int(step_stride)))
        self._inflow = values

    def tune(self, phi_in, phi_out, vel, t, dt, opts, cache_path=None):
        """Autotune the launch shapes of this step (sl_tune); returns {"tile", "per_sm_phase1",
        "per_sm_phase2", "cached"}."""
        self._state(phi_in, "phi_in")
        self._state(phi_out, "phi_out")
        out = (C.c_int * 4)()
        path = None if cache_path is None else str(cache_path).encode()
        self._check(self._lib.sl_tune(self._h, _ptr(phi_in), _ptr(phi_out), C.byref(vel), float(t), float(dt),
                                      C.byref(opts), path, out))
        return {"tile": out[0], "per_sm_phase1": out[1], "per_sm_phase2": out[2], "cached": bool(out[3])}

    def timing(self, enable):
        """Start (True) or end (False) a kernel-timing session (sl_timing)."""
        self._check(self._lib.sl_timing(self._h, 1 if enable else 0))

    def timing_read(self):
        """(phase-1 ms, phase-2 ms, total ms, timed steps) of the session so far (sl_timing_read)."""
        ms = (C.c_double * 3)()
        k = C.c_int()
        self._check(self._lib.sl_timing_read(self._h, ms, C.byref(k)))
        return ms[0], ms[1], ms[2], k.value

    def max_dt(self, vel, rule=RULE_HALF_MIN_SPACING):
        out = C.c_double()
        self._check(self._lib.sl_max_dt(self._h, C.byref(vel), int(rule), C.byref(out)))
        return out.value

    def node_coords(self):
        x = np.empty(self.size)
        y = np.empty(self.size) if self.dim == 2 else None
        self._check(self._lib.sl_node_coords(self._h, x.ctypes.data_as(C.c_void_p),
                                             y.ctypes.data_as(C.c_void_p) if y is not None else None))
        return (x.reshape(self.shape), y.reshape(self.shape) if y is not None else None)

    def nodes_weights(self, n=None):
        n = self.n if n is None else n
        xi, w = np.empty(n), np.empty(n)
        self._check(self._lib.sl_nodes_weights(self._h, int(n), xi.ctypes.data_as(C.c_void_p),
                                               w.ctypes.data_as(C.c_void_p)))
        return xi, w


class Batch(Context):
    """Independent 2D problems advanced together (sl_batch_create): the batch state is the
    problems' states concatenated; problem p's values start at offset(p)."""

    def __init__(self, problems):
        self._lib = lib()
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        h = C.c_void_p()
        st = self._lib.sl_batch_create(len(self.problems), arr, C.byref(h))
        if st != SL_OK:
            raise SlError(st, self._lib.sl_last_error(None).decode())
        self._h = h
        p0 = self.problems[0]
        self.dim, self.n, self.precision, self.stream = 2, None, p0.precision, p0.stream
        self._setup(h, p0.precision)
        self.shape = (self.size,)

    def offset(self, p):
        return int(self._lib.sl_batch_offset(self._h, int(p)))

    def batch_step(self, phi_in, phi_out, vel, t, dt, opts):
        """t, dt: one time and step per problem."""
        self._state(phi_in, "phi_in")
        self._state(phi_out, "phi_out")
        ta = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
        da = np.ascontiguousarray(np.asarray(dt, dtype=np.float64))
        if ta.size != len(self.problems) or da.size != len(self.problems):
            raise ValueError("one t and one dt per problem")
        self._check(self._lib.sl_batch_step(self._h, _ptr(phi_in), _ptr(phi_out), C.byref(vel),
                                            ta.ctypes.data_as(C.c_void_p), da.ctypes.data_as(C.c_void_p),
                                            C.byref(opts)))
