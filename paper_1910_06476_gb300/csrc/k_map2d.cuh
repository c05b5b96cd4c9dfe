#pragma once
// Element addressing of the general 2D kernels (one CTA per element): uniform meshes, p-adaptive
// meshes (per-element node counts, CSR value offsets) and batches of independent problems, see
// Map2D in sl_internal.h.
#include "sl_internal.h"

namespace sl {

// The element a CTA advances: global index g, the global index gb of its problem's first
// element, local index e (row-major (ex, ey) within its problem), first value of its state.
struct Elem {
  int64_t g, gb, base;
  int e, ex, ey;
};

// Resolves the CTA's element; copies its problem's geometry and step into P (batches).
template <int NN>
__device__ __forceinline__ Elem elem_of(StepParams& P, const Map2D& M) {
  Elem E;
  E.g = M.list ? (int64_t)M.list[blockIdx.x] : (int64_t)blockIdx.x;
  E.gb = 0;
  if (M.geo) {
    const ProbGeom& G = M.geo[M.prob[E.g]];
    P.kx = G.kx;
    P.ky = G.ky;
    for (int f = 0; f < 4; ++f) P.bc[f] = G.bc[f];
    P.x0 = G.x0;
    P.hx = G.hx;
    P.y0 = G.y0;
    P.hy = G.hy;
    P.ghost = G.ghost;
    P.t = G.t;
    P.dt = G.dt;
    E.gb = G.gbase;
  }
  E.e = (int)(E.g - E.gb);
  E.ex = E.e % P.kx;
  E.ey = E.e / P.kx;
  E.base = M.off ? M.off[E.g] : E.g * (NN * NN);
  return E;
}

// node count of the element with global index gn
template <int NN>
__device__ __forceinline__ int order_of(const Map2D& M, int64_t gn) { return M.ord ? (int)M.ord[gn] : NN; }

// Value at z of the polynomial through vals at the nodes of the nn-point rule (rules holds the
// nodes, barycentric weights and quadrature weights of every rule, NMAX apart): a neighbour's
// face trace evaluated at this element's tangential nodes across a p-nonconforming face.
template <typename R>
__device__ __forceinline__ R interp_rule(const R* rules, int nn, const R* vals, R z) {
  const R* xs = rules + (size_t)nn * 3 * NMAX;
  const R* lm = xs + NMAX;
  R d[NMAX], pre[NMAX];
  R acc = R(1);
#pragma unroll
  for (int k = 0; k < NMAX; ++k)
    if (k < nn) {
      d[k] = z - xs[k];
      pre[k] = acc;
      acc *= d[k];
    }
  R suf = R(1), v = R(0);
#pragma unroll
  for (int k = NMAX - 1; k >= 0; --k)
    if (k < nn) {
      v += lm[k] * pre[k] * suf * vals[k];
      suf *= d[k];
    }
  return v;
}

}  // namespace sl
