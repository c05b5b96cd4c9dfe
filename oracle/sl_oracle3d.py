"""FP64 CPU oracle of the DSEM-SL step on a 3D tensor-product mesh (Sec. 3, eq. 3.4: the element
interpolant Q(xi, eta, zeta) = sum_ijk Q_ijk h_i(xi) h_j(eta) h_k(zeta); the step of Sec. 4 on it).

TEST INFRASTRUCTURE ONLY, like sl_oracle: only tests/ may import it; the CUDA library never
calls it.  It reuses the 1D tables, the RK tableaux, the upwind rule and the constrained fit of
sl_oracle (themselves pinned), and adds the third direction: n^3 particles per element, the
dense n^3 x n^3 collocation system (the 3D form of eq. 5.4), six faces of n^2 points each for the
interface rows, face fluxes integrated with the n x n Gauss rule, and the mass (and energy) row
with the weights w o w o w.  Readings are those of the 1D and 2D oracle (R4-R8), carried to a
third direction unchanged.

Element state layout: phi_e[k, j, i] with k along z (zeta), j along y (eta), i along x (xi);
the mesh state is (kz, ky, kx, n, n, n).  Faces: 0 W (x = x0), 1 E, 2 S (y = y0), 3 N, 4 B
(z = z0), 5 T.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .sl_oracle import (BC_PERIODIC, C_BOUNDARY, C_ENERGY, C_MASS, FIT_HARD, PICARD_CAP, PICARD_RTOL, TIE,
                        VEL_CONST, VEL_ROTATION, constrained_fit, lagrange, nodes_weights, rk_tableau,
                        upwind_value)


@dataclass
class Setup3:
    """Uniform box mesh of kx x ky x kz elements with n nodes per direction."""
    kx: int
    ky: int
    kz: int
    box: tuple                   # (x0, x1, y0, y1, z0, z1)
    n: int
    basis: int = 0
    bc: tuple = (BC_PERIODIC,) * 6
    ghost: object = 0.0          # constant, or callable ghost(x, y, z, t) at inflow faces

    @property
    def h(self):
        b = self.box
        return ((b[1] - b[0]) / self.kx, (b[3] - b[2]) / self.ky, (b[5] - b[4]) / self.kz)


@dataclass
class Vel3:
    """CONST p = (a, b, c); ROTATION p = (omega, cx, cy): solid-body rotation about the line
    x = cx, y = cy parallel to z (w = 0)."""
    kind: int
    p: tuple


@dataclass
class StepOpts3:
    vel: Vel3
    t: float
    dt: float
    constraints: int = C_BOUNDARY
    rk_order: int = 4
    fit: int = FIT_HARD
    picard_tol: float = None
    picard_cap: int = PICARD_CAP


def velocity3(vel, x, y, z, t):
    """(u, v, w) and div u at physical points (Sec. 4.2, a prescribed velocity)."""
    x = np.asarray(x, dtype=np.float64)
    zero = np.zeros_like(x)
    p = vel.p
    if vel.kind == VEL_CONST:
        return zero + p[0], zero + p[1], zero + p[2], zero
    if vel.kind == VEL_ROTATION:
        return -p[0] * (np.asarray(y) - p[2]), p[0] * (x - p[1]), zero, zero
    raise ValueError("unknown 3D velocity kind")


def rk_particles3(vel, x, y, z, phi, t, h, order):
    """One explicit RK step of dx/dt = u, dphi/dt = -phi div u (eq. 4.4a, 4.8) in 3D, size h."""
    A, b, c = rk_tableau(order)
    s = len(b)
    kx, ky, kz, kp = [], [], [], []
    for i in range(s):
        xi = x + h * sum(A[i, j] * kx[j] for j in range(i))
        yi = y + h * sum(A[i, j] * ky[j] for j in range(i))
        zi = z + h * sum(A[i, j] * kz[j] for j in range(i))
        pi = phi + h * sum(A[i, j] * kp[j] for j in range(i))
        u, v, w, dv = velocity3(vel, xi, yi, zi, t + c[i] * h)
        kx.append(u)
        ky.append(v)
        kz.append(w)
        kp.append(-pi * dv)
    return (x + h * sum(b[i] * kx[i] for i in range(s)), y + h * sum(b[i] * ky[i] for i in range(s)),
            z + h * sum(b[i] * kz[i] for i in range(s)), phi + h * sum(b[i] * kp[i] for i in range(s)))


def max_dt3(setup, vel, rule="paper"):
    """Edge-gap step (R9) per direction, the smallest over the three: the paper's rule, or half of
    it ('half_paper')."""
    xi, _ = nodes_weights(setup.n, setup.basis)
    b = setup.box
    if vel.kind == VEL_CONST:
        speeds = [abs(vel.p[0]), abs(vel.p[1]), abs(vel.p[2])]
    else:
        om, cx, cy = vel.p[0], vel.p[1], vel.p[2]
        speeds = [abs(om) * max(abs(b[2] - cy), abs(b[3] - cy)), abs(om) * max(abs(b[0] - cx), abs(b[1] - cx)), 0.0]
    lims = [h * xi[0] / s for h, s in zip(setup.h, speeds) if s > 0]
    return (1.0 if rule == "paper" else 0.5) * min(lims)


def _origin(setup, ex, ey, ez):
    hx, hy, hz = setup.h
    return setup.box[0] + ex * hx, setup.box[2] + ey * hy, setup.box[4] + ez * hz


def node_coords_3d(setup, ex, ey, ez):
    """Physical node coordinates of one element, each (n, n, n) in [k, j, i] layout."""
    xi, _ = nodes_weights(setup.n, setup.basis)
    x0, y0, z0 = _origin(setup, ex, ey, ez)
    hx, hy, hz = setup.h
    Z, Y, X = np.meshgrid(z0 + hz * xi, y0 + hy * xi, x0 + hx * xi, indexing="ij")
    return X, Y, Z


def project_3d(setup, f):
    out = np.zeros((setup.kz, setup.ky, setup.kx, setup.n, setup.n, setup.n))
    for ez in range(setup.kz):
        for ey in range(setup.ky):
            for ex in range(setup.kx):
                out[ez, ey, ex] = f(*node_coords_3d(setup, ex, ey, ez))
    return out


def poly_3d(setup, coef, ex, ey, ez, xq, yq, zq):
    """Element (ex, ey, ez)'s nodal polynomial (eq. 3.4) at physical points."""
    xi, _ = nodes_weights(setup.n, setup.basis)
    x0, y0, z0 = _origin(setup, ex, ey, ez)
    hx, hy, hz = setup.h
    Lx = lagrange(xi, (np.atleast_1d(xq) - x0) / hx)
    Ly = lagrange(xi, (np.atleast_1d(yq) - y0) / hy)
    Lz = lagrange(xi, (np.atleast_1d(zq) - z0) / hz)
    return np.einsum("qc,qb,qa,cba->q", Lz, Ly, Lx, coef)


def remap_3d(setup, phi, ex, ey, ez, o):
    """3D collocation (the 3D form of eq. 5.4): H phihat = phi* with
    H_{(k j i),(c b a)} = h_a(xi*_kji) h_b(eta*_kji) h_c(zeta*_kji), by Gaussian elimination."""
    n = setup.n
    xi, _ = nodes_weights(n, setup.basis)
    X, Y, Z = node_coords_3d(setup, ex, ey, ez)
    x0, y0, z0 = _origin(setup, ex, ey, ez)
    hx, hy, hz = setup.h
    xs, ys, zs, ps = rk_particles3(o.vel, X.ravel(), Y.ravel(), Z.ravel(), phi[ez, ey, ex].ravel().astype(np.float64),
                                   o.t, o.dt, o.rk_order)
    Lx = lagrange(xi, (xs - x0) / hx)
    Ly = lagrange(xi, (ys - y0) / hy)
    Lz = lagrange(xi, (zs - z0) / hz)
    H = (Lz[:, :, None, None] * Ly[:, None, :, None] * Lx[:, None, None, :]).reshape(n ** 3, n ** 3)
    return np.linalg.solve(H, ps).reshape(n, n, n)


_DIRS = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]


def nb_3d(setup, ex, ey, ez, face):
    """Neighbour across a face, or None at a non-periodic domain face."""
    dx, dy, dz = _DIRS[face]
    idx = [ex + dx, ey + dy, ez + dz]
    sizes = [setup.kx, setup.ky, setup.kz]
    axis = face // 2
    if 0 <= idx[axis] < sizes[axis]:
        return tuple(idx)
    if setup.bc[face] != BC_PERIODIC:
        return None
    idx[axis] %= sizes[axis]
    return tuple(idx)


def _shift_3d(setup, ex, ey, ez, face, nb):
    """Offset of a point of this element expressed in the frame of nb (non-zero across a wrap)."""
    dx, dy, dz = _DIRS[face]
    hx, hy, hz = setup.h
    return (nb[0] - (ex + dx)) * hx, (nb[1] - (ey + dy)) * hy, (nb[2] - (ez + dz)) * hz


def face_points_3d(setup, ex, ey, ez, face):
    """Face points at the tangential Gauss nodes (n x n, the first tangential index slower),
    outward normal and quadrature weights (face area element times w o w)."""
    n = setup.n
    xi, w = nodes_weights(n, setup.basis)
    x0, y0, z0 = _origin(setup, ex, ey, ez)
    hx, hy, hz = setup.h
    A, B = np.meshgrid(xi, xi, indexing="ij")      # A: slower tangential index, B: faster
    Wt = np.outer(w, w).ravel()
    axis, hi = face // 2, face % 2
    if axis == 0:     # tangential (z, y)
        x = np.full(n * n, x0 + (hx if hi else 0.0))
        y, z = y0 + hy * B.ravel(), z0 + hz * A.ravel()
        W = hy * hz * Wt
    elif axis == 1:   # tangential (z, x)
        y = np.full(n * n, y0 + (hy if hi else 0.0))
        x, z = x0 + hx * B.ravel(), z0 + hz * A.ravel()
        W = hx * hz * Wt
    else:             # tangential (y, x)
        z = np.full(n * n, z0 + (hz if hi else 0.0))
        x, y = x0 + hx * B.ravel(), y0 + hy * A.ravel()
        W = hx * hy * Wt
    nrm = [0.0, 0.0, 0.0]
    nrm[axis] = 1.0 if hi else -1.0
    return x, y, z, tuple(nrm), W


def face_rows_3d(setup, face):
    """Constraint rows of one face: the trace of the unknown polynomial at each face point, in the
    face-point order of face_points_3d ((n^2, n^3), unknowns in [k, j, i] order)."""
    n = setup.n
    xi, _ = nodes_weights(n, setup.basis)
    Lt = lagrange(xi, [1.0 if face % 2 else 0.0])[0]
    axis = face // 2
    rows = []
    for a in range(n):
        for b in range(n):
            r = np.zeros((n, n, n))
            if axis == 0:
                r[a, b, :] = Lt          # z = a, y = b, sum over x
            elif axis == 1:
                r[a, :, b] = Lt          # z = a, x = b, sum over y
            else:
                r[:, a, b] = Lt          # y = a, x = b, sum over z
            rows.append(r.ravel())
    return np.array(rows)


def _ghost3(setup, x, y, z, t):
    g = setup.ghost
    return g(x, y, z, t) if callable(g) else np.zeros_like(np.asarray(x, dtype=np.float64)) + g


def element_step_3d(setup, phi, ex, ey, ez, o, cache=None):
    """One DSEM-SL step for element (ex, ey, ez) (Sec. 4 with the 3D interpolant of eq. 3.4).
    Returns (phi_new (n, n, n), info)."""
    cache = {} if cache is None else cache

    def phihat_of(key):
        if key not in cache:
            cache[key] = remap_3d(setup, phi, *key, o)
        return cache[key]

    n = setup.n
    _, w = nodes_weights(n, setup.basis)
    hx, hy, hz = setup.h
    ph = phihat_of((ex, ey, ez))
    tn1 = o.t + o.dt
    rows, rhs = [], []
    if o.constraints & C_BOUNDARY:
        for face in range(6):
            xf, yf, zf, nrm, _ = face_points_3d(setup, ex, ey, ez, face)
            u, v, ww, _ = velocity3(o.vel, xf, yf, zf, tn1)
            un = u * nrm[0] + v * nrm[1] + ww * nrm[2]
            own = poly_3d(setup, ph, ex, ey, ez, xf, yf, zf)
            nb = nb_3d(setup, ex, ey, ez, face)
            if nb is None:
                other = _ghost3(setup, xf, yf, zf, tn1)
            else:
                sx, sy, sz = _shift_3d(setup, ex, ey, ez, face, nb)
                other = poly_3d(setup, phihat_of((nb[0], nb[1], nb[2])), nb[0], nb[1], nb[2], xf + sx, yf + sy,
                                zf + sz)
            rows.append(face_rows_3d(setup, face))
            rhs.extend(upwind_value(un[q], own[q], other[q], nb is not None) for q in range(n * n))
    phin = phi[ez, ey, ex].astype(np.float64)
    w3 = np.einsum("k,j,i->kji", w, w, w)
    vol = hx * hy * hz
    Fm = Fe = 0.0
    if o.constraints & (C_MASS | C_ENERGY):
        _, b, c = rk_tableau(o.rk_order)
        for face in range(6):
            nb = nb_3d(setup, ex, ey, ez, face)
            xf, yf, zf, nrm, Wq = face_points_3d(setup, ex, ey, ez, face)
            for s in range(len(b)):
                tau = o.t + c[s] * o.dt
                u, v, ww, _ = velocity3(o.vel, xf, yf, zf, tau)
                un = u * nrm[0] + v * nrm[1] + ww * nrm[2]
                if c[s] == 0.0:
                    fx, fy, fz, fac = xf, yf, zf, np.ones(n * n)
                else:
                    fx, fy, fz, fac = rk_particles3(o.vel, xf, yf, zf, np.ones(n * n), tau, -c[s] * o.dt, o.rk_order)
                own = poly_3d(setup, phin, ex, ey, ez, fx, fy, fz) / fac
                if nb is None:
                    other = _ghost3(setup, xf, yf, zf, tau)
                else:
                    sx, sy, sz = _shift_3d(setup, ex, ey, ez, face, nb)
                    other = poly_3d(setup, phi[nb[2], nb[1], nb[0]].astype(np.float64), nb[0], nb[1], nb[2], fx + sx,
                                    fy + sy, fz + sz) / fac
                val = np.where(un > TIE, own, np.where(un < -TIE, other, 0.0))
                unz = np.where(np.abs(un) <= TIE, 0.0, un)
                Fm += b[s] * np.sum(Wq * unz * val)
                Fe += b[s] * np.sum(Wq * unz * val ** 2)
    if o.constraints & C_MASS:
        rows.append(w3.ravel()[None, :])
        rhs.append((vol * np.sum(w3 * phin) - o.dt * Fm) / vol)
    C = np.vstack(rows) if rows else np.zeros((0, n ** 3))
    d = np.array(rhs, dtype=np.float64)
    ew, Et = None, 0.0
    if o.constraints & C_ENERGY:
        ew, Et = w3.ravel(), (vol * np.sum(w3 * phin ** 2) - o.dt * Fe) / vol
    tol = o.picard_tol if o.picard_tol is not None else PICARD_RTOL * max(np.max(np.abs(ph)), 1e-300)
    new, iters, conv = constrained_fit(ph.ravel(), C, d, ew, Et, o.fit, tol, o.picard_cap)
    return new.reshape(n, n, n), {"phihat": ph, "C": C, "d": d, "iters": iters, "converged": conv}


def step_3d(setup, phi, o, elements=None):
    """Advance a 3D state (kz, ky, kx, n, n, n) by one step; ``elements`` restricts to a sample of
    (ex, ey, ez) (the others are returned unchanged).  Returns (phi_new, infos)."""
    phi = np.asarray(phi, dtype=np.float64)
    out = phi.copy()
    infos = {}
    cache = {}
    els = elements if elements is not None else [(ex, ey, ez) for ez in range(setup.kz) for ey in range(setup.ky)
                                                 for ex in range(setup.kx)]
    for ex, ey, ez in els:
        out[ez, ey, ex], infos[(ex, ey, ez)] = element_step_3d(setup, phi, ex, ey, ez, o, cache)
    return out, infos


def mass_3d(setup, phi):
    _, w = nodes_weights(setup.n, setup.basis)
    hx, hy, hz = setup.h
    return hx * hy * hz * float(np.einsum("k,j,i,ZYXkji->", w, w, w, np.asarray(phi, dtype=np.float64)))


def rel_l2_3d(setup, a, b):
    _, w = nodes_weights(setup.n, setup.basis)
    W = np.einsum("k,j,i->kji", w, w, w)
    num = float(np.sum(W * (np.asarray(a) - np.asarray(b)) ** 2))
    den = float(np.sum(W * np.asarray(b) ** 2))
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)
