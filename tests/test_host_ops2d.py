"""Host logic of the 2D shared-operator path (uniform mesh, constant velocity), on CPU: the
library's host code builds the operator tables (compiled here with the host compiler, no GPU),
and the structured step the kernel applies is written out in numpy from those tables:
  psihat = R_y psi R_x^T,
  inflow residuals r_x = R_y (psi_X r_ox - psi xi_x) (+ ghost), r_y = R_x (r_oy . psi_Y) (+ ghost)
  - l_in,y . psihat, mass residual from the three functionals,
  s = (C C^T)^+ r over the kept rows, phi_L = psihat + C^T s in separable form.
It must agree with the oracle's step to the float rounding of the tables (the kernel adds only
float arithmetic on top, checked on the GPU by test_gpu_mixed2d.py)."""
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
    exe = str(tmp_path_factory.mktemp("ops2d") / "ops2d_dump")
    r = subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                        os.path.join(ROOT, "tests", "host", "ops2d_dump.cpp"), os.path.join(CSRC, "ops_mixed2d.cpp"),
                        os.path.join(CSRC, "tables.cpp"), "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-2000:])
    return exe


def emulate(exe, n, cons, rk, a, b, K, dt, phi, bc, ghost):
    out = subprocess.run([exe, str(n), str(cons), str(rk), repr(a), repr(b), str(K), repr(float(dt)), str(bc),
                          repr(float(ghost))], capture_output=True, text=True, check=True).stdout.split("\n")
    h = list(map(int, out[0].split()))
    f = [np.array(line.split(), float) for line in out[1:12]]
    xw, ys, mc, bnd, mass, perx, pery, oks, okx, oky, oRxT, oRyT, og, ol0, ol1, ow = h
    Rx, Ry = f[0].reshape(n, n), f[1].reshape(n, n)
    xix, rox, roy, liny, l0, l1, w, gm, tab = f[2:11]
    nd = n * n
    KsT = tab[oks:oks + nd].reshape(n, n)
    KxT = tab[okx:okx + nd].reshape(n, n)
    Ky = tab[oky:oky + nd].reshape(n, n)
    RxT = tab[oRxT:oRxT + nd].reshape(n, n)
    RyT = tab[oRyT:oRyT + nd].reshape(n, n)
    G = tab[og:og + 4 * mc * n].reshape(4, mc, n) if bnd else None
    L0, L1, W = tab[ol0:ol0 + n], tab[ol1:ol1 + n], tab[ow:ow + n]
    new = np.zeros_like(phi)

    def nb(i, d, per):
        j = i + d
        if 0 <= j < K:
            return j
        return j % K if per else None

    for ey in range(K):
        for ex in range(K):
            ref = phi[ey, ex, 0, 0]
            gval = ghost - ref
            ps = phi[ey, ex] - ref
            jx, jy = nb(ex, -1 if xw else 1, perx), nb(ey, -1 if ys else 1, pery)
            gx, gy = jx is None, jy is None
            X = np.full((n, n), gval) if gx else phi[ey, jx] - ref
            Y = np.full((n, n), gval) if gy else phi[jy, ex] - ref
            dx = (0 if gx else X @ rox) - ps @ xix
            v = np.zeros(n) if gy else roy @ Y
            rm = np.sum(KsT.T * ps) + np.sum(KxT.T * X) + np.sum(Ky * Y)
            ph = Ry @ ps @ Rx.T
            rx = RyT.T @ dx + (gval if gx else 0)
            ry = RxT.T @ v + (gval if gy else 0) - liny @ ph
            if bnd:
                r = np.concatenate([rx, ry] + ([[rm]] if mass else []))
                sW, sE, sS, sN = np.einsum("fkj,k->fj", G, r)
                sm = gm[:mc] @ r
            else:
                sW = sE = sS = sN = np.zeros(n)
                sm = gm[0] * rm
            new[ey, ex] = ref + ph + np.outer(l0, sS) + np.outer(l1, sN) + sm * np.outer(w, W) \
                + np.outer(sW, L0) + np.outer(sE, L1)
    return new


CASES = [  # n, constraints, rk, a, b, bc
    (5, 3, 4, 0.8, 0.45, 0), (4, 3, 2, -0.7, 0.5, 0), (6, 1, 4, 0.6, -0.9, 0), (5, 2, 3, -0.5, -0.8, 0),
    (5, 3, 4, 0.8, 0.45, 1), (6, 3, 4, -0.7, -0.5, 1), (9, 3, 4, 1.0, 0.5, 0), (7, 2, 4, 0.6, 0.9, 1),
    (12, 1, 4, -0.6, 0.7, 1),
]


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}c{c[1]}rk{c[2]}bc{c[5]}" for c in CASES])
def test_structured_step_matches_oracle(dump, case):
    n, cons, rk, a, b, bc = case
    K = 4
    ghost = 0.1 if bc else 0.0
    s = O.Setup(2, K, K, (0, 1, 0, 1), n, O.GAUSS_LEGENDRE, (bc,) * 4, ghost)
    v = O.Vel(O.VEL_CONST, (a, b, 0, 0, 0, 0))
    dt = O.max_dt(s, v, rule="paper")
    rng = np.random.default_rng(n + 10 * cons)
    phi = O.project_2d(s, lambda x, y: 1 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)) \
        + 0.05 * rng.uniform(-1, 1, (K, K, n, n))
    ref, _ = O.step_2d(s, phi, O.StepOpts(v, 0.0, dt, cons, rk))
    got = emulate(dump, n, cons, rk, a, b, K, dt, phi, bc, ghost)
    assert np.sqrt(np.sum((got - ref) ** 2) / np.sum(ref ** 2)) <= 1e-7
