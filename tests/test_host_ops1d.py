"""Host logic of the 1D shared-operator path (uniform mesh, constant velocity), on CPU: the
library's host code composes the remap (eq. 4.9), the upwinded interface values, the mass target
and the constrained fit into one linear map per element, phi_L = ref + G_self (phi - ref) +
G_up (phi_up - ref); here that map, built by the host code compiled with the host compiler (no
GPU), is applied in numpy and compared with the oracle's step.  Hard and soft fits, both bases,
both directions, periodic and inflow meshes, RK2-4."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import sl_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1910_06476_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("host compiler or CUDA headers not available")
    exe = str(tmp_path_factory.mktemp("ops1d") / "ops1d_dump")
    r = subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                        os.path.join(ROOT, "tests", "host", "ops1d_dump.cpp"), os.path.join(CSRC, "ops_mixed.cpp"),
                        os.path.join(CSRC, "tables.cpp"), "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-2000:])
    return exe


CASES = [  # n, constraints, rk, fit, a, bc, basis
    (9, 1, 4, O.FIT_HARD, 1.0, O.BC_PERIODIC, O.GAUSS_LEGENDRE),
    (9, 3, 4, O.FIT_HARD, 1.0, O.BC_PERIODIC, O.GAUSS_LEGENDRE),
    (7, 2, 3, O.FIT_HARD, -0.8, O.BC_PERIODIC, O.GAUSS_LEGENDRE),
    (5, 3, 2, O.FIT_SOFT, 0.6, O.BC_PERIODIC, O.CHEB_GAUSS),
    (6, 3, 4, O.FIT_HARD, -1.0, O.BC_INFLOW, O.GAUSS_LEGENDRE),
    (13, 3, 4, O.FIT_HARD, 1.0, O.BC_INFLOW, O.CHEB_GAUSS),
    (17, 1, 4, O.FIT_SOFT, -0.7, O.BC_PERIODIC, O.GAUSS_LEGENDRE),
]


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}c{c[1]}rk{c[2]}f{c[3]}bc{c[5]}b{c[6]}" for c in CASES])
def test_shared_operator_matches_oracle(dump, case):
    n, cons, rk, fit, a, bc, basis = case
    K = 6
    ghost = 0.2 if bc == O.BC_INFLOW else 0.0
    s = O.Setup(1, K, 1, (0.0, 1.0, 0.0, 1.0), n, basis, (bc,) * 4, ghost)
    v = O.Vel(O.VEL_CONST, (a, 0, 0, 0, 0, 0))
    dt = O.max_dt(s, v, rule="paper")
    rng = np.random.default_rng(n + cons)
    phi = O.project_1d(s, lambda x: 1.0 + 0.4 * np.sin(2 * np.pi * x)) + 0.05 * rng.uniform(-1, 1, (K, n))
    ref, _ = O.step_1d(s, phi, O.StepOpts(v, 0.0, dt, cons, rk, fit))
    out = subprocess.run([dump, str(n), str(cons), str(rk), str(fit), repr(a), str(K), repr(float(dt)), str(bc),
                          str(basis)], capture_output=True, text=True, check=True).stdout.split("\n")
    left_up, _ = map(int, out[0].split())
    Gs = np.array(out[1].split(), float).reshape(n, n)
    Gu = np.array(out[2].split(), float).reshape(n, n)
    got = np.empty_like(phi)
    for k in range(K):
        r0 = phi[k, 0]
        ku = k - 1 if left_up else k + 1
        if 0 <= ku < K or bc == O.BC_PERIODIC:
            up = phi[ku % K] - r0
        else:
            up = np.full(n, ghost - r0)
        got[k] = r0 + Gs @ (phi[k] - r0) + Gu @ up
    assert np.sqrt(np.sum((got - ref) ** 2) / np.sum(ref ** 2)) <= 1e-7
