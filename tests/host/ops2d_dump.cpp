// Test helper: builds the 2D shared-operator tables of the library's host code for one case and
// prints them (header integers, the parameter-bank arrays, then the float table), so that a test
// can apply the kernel's structured step in numpy and compare it with the oracle.
#include <cstdio>
#include <cstdlib>

#include "sl_internal.h"

using namespace sl;

static void row(const float* v, int k) {
  for (int i = 0; i < k; ++i) std::printf("%.9g ", v[i]);
  std::printf("\n");
}

int main(int argc, char** argv) {
  if (argc < 10) return 2;
  const int n = std::atoi(argv[1]);
  const unsigned cons = (unsigned)std::atoi(argv[2]);
  const int rk = std::atoi(argv[3]);
  const double a = std::atof(argv[4]), b = std::atof(argv[5]);
  const int K = std::atoi(argv[6]);
  const double dt = std::atof(argv[7]);
  const int bc = std::atoi(argv[8]);
  const double ghost = std::atof(argv[9]);
  sl_ctx c;
  c.mesh.dim = 2;
  c.mesh.kx = c.mesh.ky = K;
  c.mesh.x0 = c.mesh.y0 = 0.0;
  c.mesh.x1 = c.mesh.y1 = 1.0;
  for (int f = 0; f < 4; ++f) c.mesh.bc[f] = bc;
  c.mesh.ghost = ghost;
  c.n = n;
  c.basis = 0;
  c.b = make_basis(n, 0);
  for (unsigned m = 0; m < 4; ++m) c.fit[m][0] = make_fit_2d(c.b, m, false);
  std::vector<float> buf;
  Mixed2DConstParams P;
  std::string err;
  if (!build_mixed2d_const(&c, a, b, dt, cons, rk, buf, P, err)) {
    std::printf("ERR %s\n", err.c_str());
    return 1;
  }
  std::printf("%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", P.xw, P.ys, P.mc, P.bnd, P.mass, P.per_x, P.per_y,
              P.o_ks, P.o_kx, P.o_ky, P.o_RxT, P.o_RyT, P.o_g, P.o_l0, P.o_l1, P.o_w);
  row(P.Rx, n * n);
  row(P.Ry, n * n);
  row(P.xix, n);
  row(P.rox, n);
  row(P.roy, n);
  row(P.liny, n);
  row(P.l0, n);
  row(P.l1, n);
  row(P.w, n);
  row(P.gm, 2 * n + 1);
  row(buf.data(), (int)buf.size());
  return 0;
}
