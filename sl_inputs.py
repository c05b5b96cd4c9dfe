"""Seeded synthetic workloads for the semi-Lagrangian spectral transport step.

This module is shared by the oracle, the tests, ``bench.py`` and ``smoke()``.  It holds
NO arithmetic of the method: no nodes, no basis, no advection, no remap or fit.  It only
states the problems (domains, element counts, velocity parameters, analytic initial data
as plain functions of physical position) and draws seeded random numbers.  Each side
(oracle and CUDA library) computes its own node positions and evaluates the initial data
there itself.

Workloads follow the shapes of the paper's tests (1D constant velocity, Sec. 5.1; 1D
variable velocity, Sec. 5.2; 2D constant velocity, Sec. 5.3) and the five large
synthetic configurations the library is measured on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# velocity kinds (values match the C ABI enumeration)
VEL_CONST, VEL_ROTATION, VEL_SWIRL, VEL_SINX = 0, 1, 2, 3
# boundary kinds
BC_PERIODIC, BC_INFLOW = 0, 1
# constraint bits
C_BOUNDARY, C_MASS, C_ENERGY = 1, 2, 4
# bases
GAUSS_LEGENDRE, CHEB_GAUSS = 0, 1
# fit modes
FIT_HARD, FIT_SOFT = 0, 1


@dataclass
class Velocity:
    kind: int
    p: tuple = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)


@dataclass
class Problem:
    """One transport problem: mesh, polynomial order, velocity, data and step options."""
    name: str
    dim: int
    kx: int
    ky: int
    box: tuple              # (x0, x1, y0, y1); 1D ignores y
    n: int                  # nodes per direction (polynomial degree N = n - 1)
    basis: int
    velocity: Velocity
    bc: tuple               # (W, E, S, N) kinds
    ghost: float
    constraints: int
    rk_order: int
    fit: int = FIT_HARD
    t0: float = 0.0
    phi0: object = None     # callable phi0(x[, y]) -> array (plain numpy)
    orders: object = None   # optional per-element node counts (p-adaptive), shape (ky, kx)
    dt_rule: str = "paper"  # "paper": edge-node gap, factor 1; "half_min_spacing": half the min spacing;
                            # "half_paper": half the paper's step (the 2D deforming flows)
    extra: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------- data


def sine_1d(x):
    return np.sin(2.0 * np.pi * x)


def gaussian_1d(x):
    return np.exp(-(((x - 0.5) / 0.05) ** 2))


def sincos_2d(x, y):
    return np.sin(2.0 * np.pi * x) * np.cos(2.0 * np.pi * y)


def sinsin_2d(x, y):
    return np.sin(2.0 * np.pi * x) * np.sin(2.0 * np.pi * y)


def hill_2d(x, y):
    return np.exp(-((x - 0.25) ** 2 + (y - 0.5) ** 2) / 0.01)


def cosine_bell_2d(x, y):
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.75) ** 2)
    return np.where(r < 0.15, 0.5 * (1.0 + np.cos(np.pi * np.minimum(r, 0.15) / 0.15)), 0.0)


def sinx_initial(x):
    """Initial data of the variable-velocity test (Sec. 5.2): sin(2 atan(e^-1 tan(x/2))) / sin x."""
    s = np.sin(x)
    num = np.sin(2.0 * np.arctan(np.exp(-1.0) * np.tan(x / 2.0)))
    safe = np.where(np.abs(s) < 1e-12, 1.0, s)
    # limit at x -> 0 and x -> 2 pi is e^-1, at x -> pi it is e
    lim = np.where(np.abs(x - np.pi) < 1e-6, np.e, np.exp(-1.0))
    return np.where(np.abs(s) < 1e-12, lim, num / safe)


# ----------------------------------------------------------------------------- configs


def config1_1d_sine(n=9, k=16):
    """1D periodic [0,1], u = 1, sin(2 pi x), K=16, 9 Gauss-Legendre nodes, boundary only, RK4, FP64."""
    return Problem("1d_sine_K16_n9", 1, k, 1, (0.0, 1.0, 0.0, 0.0), n, GAUSS_LEGENDRE,
                   Velocity(VEL_CONST, (1.0, 0, 0, 0, 0, 0)), (BC_PERIODIC,) * 4, 0.0,
                   C_BOUNDARY, 4, phi0=sine_1d, dt_rule="half_min_spacing")


def config2_1d_gauss(n=9, k=1 << 20):
    """1D periodic [0,1], a = 1, Gaussian pulse, K = 2^20, boundary + mass + energy, RK4."""
    return Problem(f"1d_gauss_K{k}_n{n}", 1, k, 1, (0.0, 1.0, 0.0, 0.0), n, GAUSS_LEGENDRE,
                   Velocity(VEL_CONST, (1.0, 0, 0, 0, 0, 0)), (BC_PERIODIC,) * 4, 0.0,
                   C_BOUNDARY | C_MASS | C_ENERGY, 4, phi0=gaussian_1d)


def config3_2d_const(n=9, k=512):
    """2D periodic unit square, velocity (1, 0.5), sin 2 pi x cos 2 pi y, boundary (4 faces) + mass."""
    return Problem(f"2d_const_K{k}x{k}_n{n}", 2, k, k, (0.0, 1.0, 0.0, 1.0), n, GAUSS_LEGENDRE,
                   Velocity(VEL_CONST, (1.0, 0.5, 0, 0, 0, 0)), (BC_PERIODIC,) * 4, 0.0,
                   C_BOUNDARY | C_MASS, 4, phi0=sincos_2d)


def config4_rotation(k=256, seed=0, uniform_n=None):
    """2D solid-body rotation about (0.5, 0.5), omega = 2 pi, inflow ghost 0, Gaussian hill.

    Per-element node counts n = N + 1 with N drawn uniformly from {3..15} (seeded)."""
    orders = None
    n = uniform_n if uniform_n is not None else 16
    if uniform_n is None:
        orders = p_adaptive_orders(k, k, seed)
    return Problem(f"2d_rotation_K{k}x{k}", 2, k, k, (0.0, 1.0, 0.0, 1.0), n, GAUSS_LEGENDRE,
                   Velocity(VEL_ROTATION, (2.0 * np.pi, 0.5, 0.5, 0, 0, 0)), (BC_INFLOW,) * 4, 0.0,
                   C_BOUNDARY | C_MASS, 4, phi0=hill_2d, orders=orders, dt_rule="half_paper")


def config5_swirl(n=8, k=2048, T=5.0):
    """2D swirling deformation flow with period T = 5, cosine bell, mass + energy (+ boundary)."""
    return Problem(f"2d_swirl_K{k}x{k}_n{n}", 2, k, k, (0.0, 1.0, 0.0, 1.0), n, GAUSS_LEGENDRE,
                   Velocity(VEL_SWIRL, (T, 0, 0, 0, 0, 0)), (BC_INFLOW,) * 4, 0.0,
                   C_BOUNDARY | C_MASS | C_ENERGY, 4, phi0=cosine_bell_2d, dt_rule="half_paper")


def p_adaptive_orders(kx, ky, seed):
    """Per-element node counts n = N + 1, N ~ U{3..15}, drawn with numpy's default_rng(seed)."""
    return np.random.default_rng(seed).integers(3, 16, (ky, kx)).astype(np.int32) + 1


def batch_sizes(nprob=64, seed=1):
    """Side lengths (elements per direction) of the independent problems in the batched workload."""
    return np.random.default_rng(seed).integers(32, 257, nprob)


def batch_orders(i, k):
    """Per-element node counts of problem i of the batched workload (k x k elements)."""
    return np.random.default_rng(100 + i).integers(3, 16, (k, k)).astype(np.int32) + 1


def config4_batch(nprob=64):
    """The batched rotation workload: nprob independent p-adaptive problems of config 4's kind,
    side lengths from batch_sizes, node counts from batch_orders."""
    probs = []
    for i, k in enumerate(batch_sizes(nprob)):
        p = config4_rotation(int(k), seed=0)
        p.orders = batch_orders(i, int(k))
        probs.append(p)
    return probs


# ----------------------------------------------------------------------------- random states


def random_state(shape, seed, smooth=None):
    """Seeded random node values for parity tests (uniform in [-1, 1])."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=shape)


def random_velocity_const(seed, dim):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.3, 1.0) * rng.choice([-1.0, 1.0])
    b = rng.uniform(0.3, 1.0) * rng.choice([-1.0, 1.0]) if dim == 2 else 0.0
    return Velocity(VEL_CONST, (a, b, 0, 0, 0, 0))


def sample_elements(count, total, seed):
    """Seeded sample of distinct element indices (sorted)."""
    rng = np.random.default_rng(seed)
    count = min(count, total)
    return np.sort(rng.choice(total, size=count, replace=False))


def rule_code(prob):
    """Time-step rule of a problem as the C ABI enumeration (0: half min spacing, 1: paper,
    2: half the paper's step)."""
    return {"half_min_spacing": 0, "paper": 1, "half_paper": 2}[prob.dt_rule]


def steps_to(T, dt0):
    """Number of equal steps that lands exactly on T with dt <= dt0 (and that dt)."""
    nsteps = int(math.ceil(T / dt0 - 1e-12))
    return nsteps, T / nsteps
