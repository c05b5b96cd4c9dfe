// Test helper: builds the 1D shared operator of the library's host code (uniform mesh, constant
// velocity) for one case and prints it: "left_up m", then G_self and G_up row by row.
#include <cstdio>
#include <cstdlib>

#include "sl_internal.h"

using namespace sl;

int main(int argc, char** argv) {
  if (argc < 10) return 2;
  const int n = std::atoi(argv[1]);
  const unsigned cons = (unsigned)std::atoi(argv[2]);
  const int rk = std::atoi(argv[3]);
  const int fitmode = std::atoi(argv[4]);
  const double a = std::atof(argv[5]);
  const int K = std::atoi(argv[6]);
  const double dt = std::atof(argv[7]);
  const int bc = std::atoi(argv[8]);
  const int basis = std::atoi(argv[9]);
  sl_ctx c;
  c.mesh.dim = 1;
  c.mesh.kx = K;
  c.mesh.ky = 1;
  c.mesh.x0 = 0.0;
  c.mesh.x1 = 1.0;
  for (int f = 0; f < 4; ++f) c.mesh.bc[f] = bc;
  c.n = n;
  c.basis = basis;
  c.b = make_basis(n, basis);
  FitOps fit = make_fit_1d(c.b, cons & 3u);
  finish_fit(fit, fitmode == SL_FIT_SOFT);
  Mixed1DParams P;
  std::string err;
  if (!build_mixed1d(&c, fit, a, dt, cons, rk, fitmode, P, err)) {
    std::printf("ERR %s\n", err.c_str());
    return 1;
  }
  std::printf("%d %d\n", P.left_up, P.m);
  for (int k = 0; k < n * n; ++k) std::printf("%.9g ", P.Gs[k]);
  std::printf("\n");
  for (int k = 0; k < n * n; ++k) std::printf("%.9g ", P.Gu[k]);
  std::printf("\n");
  return 0;
}
