// Internal declarations shared by the host API and the kernels of the GB300 DSEM-SL library.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sl.h"

struct sl_ctx;

namespace sl {

constexpr int NMAX = 17;                 // largest node count per direction
constexpr int MMAX1D = 3;                // linear constraint rows in 1D: left, right, mass
constexpr double TIE = 1e-13;            // |u.n| at or below this is an upwind tie
constexpr double ENERGY_SKIP_RTOL = 1e-9;   // energy row applied only beyond this relative miss

// ------------------------------------------------------------------ host tables (tables.cpp)

struct Basis1D {
  int n = 0;
  std::vector<double> xi, w, lam;        // nodes on [0,1], weights, barycentric weights
  std::vector<double> l0, l1;            // Lagrange basis values at xi = 0 and xi = 1
};

Basis1D make_basis(int n, int basis);

// Dense row-major operators of the constrained fit for one constraint set.
//   hard: phi_L = phihat + Cpinv (d - C phihat);  q = a - Cpinv (C a)
//   soft: phi_L = S phihat + SCt d;                q = S a
struct FitOps {
  int m = 0, nd = 0;                     // rows, unknowns (n or n^2)
  std::vector<double> C;                 // m x nd
  std::vector<double> Cpinv;             // nd x m (hard)
  std::vector<double> S;                 // nd x nd (soft)
  std::vector<double> SCt;               // nd x m (soft)
};

// 1D constraint rows for a mask (left face, right face, mass in the reference measure).
FitOps make_fit_1d(const Basis1D& b, unsigned mask);
// 2D constraint rows: W, E, S, N faces (n each, at the tangential nodes), then mass.
FitOps make_fit_2d(const Basis1D& b, unsigned mask, bool soft);
void finish_fit(FitOps& f, bool soft);

// ------------------------------------------------------------------ device-side parameter blocks

struct Tables1D {                         // device pointers into one table buffer
  const double* xi;
  const double* w;
  const double* lam;
  const double* l0;
  const double* l1;
  const double* Cpinv;                   // [n][m] for the active row set
  const double* S;                       // [n][n]
  const double* SCt;                     // [n][m]
};

struct StepParams {
  int K;                                 // elements (1D)
  int kx, ky;
  double x0, hx, y0, hy;
  int bc[4];
  double ghost;
  int vel_kind;
  double vp[6];
  double t, dt;
  int rk;
  unsigned cons;
  int fit;
  int bvalue;
  int m;                                 // active linear rows
  double picard_rtol;
  int picard_cap;
};

void launch_step1d_f64(int n, const StepParams& p, const Tables1D& tb, const double* in,
                       double* out, unsigned* status, cudaStream_t s);

// 2D FP64 step (two kernels); work holds nel * (n^2 + 4n + 8) doubles
void launch_step2d_f64(int n, const StepParams& p, const Tables1D& tb, const double* in, double* out, double* work,
                       unsigned* status, cudaStream_t s);
inline int64_t work2d_doubles(int64_t nel, int n) { return nel * (int64_t)(n * n + 4 * n + 8); }

// Extra parameters of the 2D mixed-precision kernels (float tables and scalars), by value
struct Mixed2DExtra {
  const float* xi;
  const float* lam;
  const float* w;
  const float* l0;
  const float* l1;
  const float* Cp;                       // [n^2][m] pseudo-inverse of the active rows (hard fit)
  int64_t plane;                         // float offset of the lo plane
  float hx, hy, ihx, ihy;
  float a, b, om, cx, cy;                // velocity parameters (constant / rotation)
  float tT, dtT;                         // t / T and dt / T (swirl)
  float dt, dt_area;                     // dt and dt / (hx hy)
};
void launch_step2d_mixed(int n, const StepParams& p, const Mixed2DExtra& x, const float* in, float* out, float* work,
                         unsigned* status, cudaStream_t s);
inline int64_t work2m_floats(int64_t nel, int n) { return nel * (int64_t)(n * n + 4 * n + 16 + 4); }

// Parameters of the 2D shared-operator kernel (uniform mesh, constant velocity).  Operators that
// every thread applies with the same entry live here (the kernel reads them from the parameter
// bank); operators read per row live in a float table at the given offsets.
struct Mixed2DConstParams {
  int n, kx, ky, xw, ys, per_x, per_y, bnd, mass, mc;
  double ghost;
  int64_t plane;
  float Rx[NMAX * NMAX], Ry[NMAX * NMAX];   // remap matrices [l][p]: l_p(xi_l - shift)
  float xix[NMAX];                          // R_x^T l_in,x: own inflow x-trace functional of a row
  float rox[NMAX], roy[NMAX];               // R^T l_out: upwind neighbour outflow-trace functionals
  float liny[NMAX];                         // l_in,y: inflow y-trace of a remapped column
  float l0[NMAX], l1[NMAX], w[NMAX];        // basis at 0 and 1, quadrature weights
  float gm[2 * NMAX + 1];                   // mass row of (C C^T)^+ over the kept residuals
  int o_ks, o_kx, o_ky;                     // mass-target functionals (own, x-, y-neighbour)
  int o_RxT, o_RyT;                         // transposed remap matrices
  int o_g;                                  // face rows of (C C^T)^+ over the kept residuals
  int o_l0, o_l1, o_w;                      // l0, l1, w again, read per thread
};
bool build_mixed2d_const(const sl_ctx* c, double a, double b, double dt, unsigned cons, int rk,
                         std::vector<float>& buf, Mixed2DConstParams& P, std::string& err);
void launch_step2d_const(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* status,
                         cudaStream_t s);

// Kernel parameter block of the 1D shared-operator (mixed precision) step; passed by value.
struct Mixed1DParams {
  int n, K, left_up, periodic, m, mass_on, energy_on, nst;
  int64_t plane;                         // float offset of the lo plane in a state buffer
  double ghost;
  float lam;                             // |a| dt / h
  float picard_rtol;
  int picard_cap;
  float Gs[NMAX * NMAX], Gu[NMAX * NMAX];  // [j][i]
  float w[NMAX];
  float fb[3];                           // merged RK weights of the distinct stage times
  float E[3][NMAX];                      // basis at the characteristic feet of the outflow face
  float C[MMAX1D * NMAX];                // linear constraint rows
  float Cp[NMAX * MMAX1D];               // their pseudo-inverse (hard fit)
};

bool build_mixed1d(const sl_ctx* c, const FitOps& fit, double a, double dt, unsigned cons, int rk, int fitmode,
                   Mixed1DParams& P, std::string& err);
void launch_step1d_mixed(const Mixed1DParams& p, const float* in, float* out, unsigned* status, cudaStream_t s);
void launch_pack(int64_t nvals, int64_t plane, const double* src, float* dst, cudaStream_t s);
void launch_unpack(int64_t nvals, int64_t plane, const float* src, double* dst, cudaStream_t s);

// float offset of the lo plane of a double-float state of nvals nodes: 256-byte aligned
inline int64_t plane_stride(int64_t nvals) { return (nvals + 63) & ~int64_t(63); }
void launch_mass_energy_f64(int64_t nelem, int nper, const double* phi, const double* w, int dim,
                            int power, double scale, double* partial, double* result, int nblocks,
                            cudaStream_t s);
void launch_mass_energy_pair(int64_t nelem, int nper, int64_t plane, const float* phi, const double* w,
                             int dim, int power, double scale, double* partial, double* result,
                             int nblocks, cudaStream_t s);

}  // namespace sl

// ------------------------------------------------------------------ context

struct sl_ctx {
  sl_mesh mesh{};
  std::vector<int32_t> orders;
  int n = 0, basis = 0, precision = 0;
  cudaStream_t stream = nullptr;
  int64_t nvals = 0;
  sl::Basis1D b;
  // fit operators per constraint mask (index = mask & 3 for linear rows) and fit mode
  sl::FitOps fit[4][2];
  double* d_tables = nullptr;            // device table buffer
  size_t table_off[4][2][3] = {};        // offsets of Cpinv, S, SCt per mask/mode
  size_t off_xi = 0, off_w = 0, off_lam = 0, off_l0 = 0, off_l1 = 0;
  unsigned* d_status = nullptr;
  double* d_partial = nullptr;           // reduction workspace
  double* d_result = nullptr;
  int red_blocks = 0;
  void* d_io = nullptr;                  // device buffers for sl_run_host
  double* d_io64 = nullptr;
  double* d_work = nullptr;              // 2D workspace between the two phases
  float* d_ftab = nullptr;               // float tables of the mixed 2D path
  // cached shared operator of the mixed 2D constant-velocity path
  bool m2c_valid = false;
  double m2c_a = 0, m2c_b = 0, m2c_dt = 0;
  unsigned m2c_cons = 0;
  int m2c_rk = 0;
  std::vector<float> m2c_host;
  float* d_m2c = nullptr;
  size_t m2c_cap = 0;
  sl::Mixed2DConstParams m2c{};
  size_t f_off[5] = {};                  // xi, lam, w, l0, l1
  size_t f_cp[4] = {};                   // float pseudo-inverse per linear-row mask
  // cached shared operator of the mixed 1D path, keyed on (a, dt, constraints, rk, fit)
  bool mix_valid = false;
  double mix_a = 0, mix_dt = 0;
  unsigned mix_cons = 0;
  int mix_rk = 0, mix_fit = 0;
  sl::Mixed1DParams mix{};
  std::string err;
};
