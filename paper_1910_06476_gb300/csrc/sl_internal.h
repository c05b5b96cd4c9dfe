// Internal declarations shared by the host API and the kernels of the GB300 DSEM-SL library.
#pragma once

#include <algorithm>
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
// SL_VEL_NODAL: a point within this of a face, relative to |x0| + |x1| (|y0| + |y1|), is on it
constexpr double FACE_RTOL = 1e-12;
// The energy row is applied only when the linear fit misses the energy target by more than this,
// relative (Sec. 4.3: the iteration starts from the linear fit and stops when iterates agree).
// FP64 paths decide one decade above the double rounding level of the energy sums.  The mixed
// paths form the mismatch from float increments, whose resolution relative to the energy is about
// eps_float (psi / phi)^2, up to 1e-10 on resolved data: they decide at 1e-9, and an element they
// skip differs from the FP64 decision by at most that relative energy miss.
constexpr double ENERGY_SKIP_RTOL = 1e-12;
constexpr double ENERGY_SKIP_RTOL_MIXED = 1e-9;

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
  const double* rules;                   // [NMAX + 1][3][NMAX] xi, lam, w of every node count
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
  const double* gtab;                    // 1D inflow record of this step (sl_set_inflow), or null
  const double* nodal;                   // SL_VEL_NODAL: [2][dim][nvals] node velocities at t, t + dt
  int64_t nvals;                         // state values (stride of the nodal components)
};

void launch_step1d_f64(int n, const StepParams& p, const Tables1D& tb, const double* in,
                       double* out, unsigned* status, cudaStream_t s);

// Geometry and step of one problem of a batch (device array); replaces the StepParams fields of
// the same names for the elements of that problem.
struct ProbGeom {
  int kx, ky;
  int bc[4];
  double x0, hx, y0, hy;
  double ghost, t, dt;
  int64_t gbase;                         // global index of the problem's first element
};

// Element map of a 2D launch of the general kernels.  A uniform single-problem mesh uses the
// null map (CTA b advances element b, values at b n^2); p-adaptive meshes (per-element node
// counts, CSR value offsets) and batches of problems launch once per node count with the list
// of elements of that count.
struct Map2D {
  const int* list;                       // global indices of the elements this launch advances
  const int64_t* off;                    // value offset of each element (null: g n^2)
  const uint8_t* ord;                    // node count of each element (null: all the launch's n)
  const uint16_t* prob;                  // problem of each element (null: the StepParams problem)
  const ProbGeom* geo;                   // per-problem geometry and step (null: StepParams)
  int tstride;                           // trace values per element in the workspace
};

struct Work2D {                          // FP64 workspace between the two phases
  double* phihat;                        // same layout as the state
  double* traces;                        // [nel][tstride]   faces W, E, S, N at the tangential nodes
  double* fluxes;                        // [nel][4][2]      outflow (mass, energy) flux per face
};

// 2D FP64 step: phase 1 (remap, traces, outflow fluxes) of every launch must run before any
// phase 2 (interface values, targets, fit); count = CTAs (elements) of the launch
void launch_step2d_f64(int phase, int n, const StepParams& p, const Tables1D& tb, const Map2D& m, int64_t count,
                       const double* in, double* out, const Work2D& w, unsigned* status, cudaStream_t s);
inline int64_t work2d_doubles(int64_t nel, int n) { return nel * (int64_t)(n * n + 4 * n + 8); }

// Extra parameters of the 2D mixed-precision kernels (float tables and scalars), by value
struct Mixed2DExtra {
  const float* xi;
  const float* lam;
  const float* w;
  const float* l0;
  const float* l1;
  const float* Cp;                       // [m][n^2] pseudo-inverse of the active rows (hard fit)
  const float* rules;                    // [NMAX + 1][3][NMAX] xi, lam, w of every node count
  const float* w2h;                      // [n^2] w_i w_j (formed in double) as float-float: hi
  const float* w2l;                      //       and lo words
  unsigned long long* counts;            // the context's work counters (SL_CNT_*), or null
  int linref;                            // 1: linear element reference (no energy row), 0: constant
  int64_t plane;                         // float offset of the lo plane
  float span;                            // 1 / (2 (xi_{n-1} - xi_0)): corner differences to slopes
  float hx, hy, ihx, ihy;
  float a, b, om, cx, cy;                // velocity parameters (constant / rotation)
  float tT, dtT;                         // t / T and dt / T (swirl)
  float dt, dt_area;                     // dt and dt / (hx hy)
  float lam_hi, lam_lo;                  // dt / (hx hy) as float-float
  double Tper;                           // swirl period T (per-problem t / T in a batch), else 0
};
struct Work2M {                          // mixed workspace between the two phases
  float* psihat;                         // same layout as the state (one plane)
  float* traces;                         // [nel][tstride]
  float* faces;                          // [nel][4][6]  G_hi, G_lo (outflow flux of phi), U_out, U_in, P1, P2
  float* elem;                           // [nel][8]     r0, gx, gy, sum w psi, sum w psi^2, M^n hi, lo, unused
};
// per_sm: resident CTAs per SM of the persistent grid (0: as many as the occupancy allows)
void launch_step2d_mixed(int phase, int n, const StepParams& p, const Mixed2DExtra& x, const Map2D& m,
                         int64_t count, const float* in, float* out, const Work2M& w, unsigned* status,
                         cudaStream_t s, int per_sm);
inline int64_t work2m_floats(int64_t nel, int n) { return nel * (int64_t)(n * n + 4 * n + 24 + 8); }
constexpr int WORK2M_FACE = 24, WORK2M_ELEM = 8;   // floats per element of the face and element records

// Parameters of the 2D shared-operator kernel (uniform mesh, constant velocity).  Operators that
// every thread applies with the same entry live here (the kernel reads them from the parameter
// bank); operators read per row live in a float table at the given offsets.
struct Mixed2DConstParams {
  int n, kx, ky, xw, ys, per_x, per_y, bnd, mass, mc;
  double ghost;
  int64_t plane;
  float Rx[NMAX * NMAX], Ry[NMAX * NMAX];   // remap matrices [l][p]: l_p(xi_l - shift)
  float2 Rxp[NMAX / 2][NMAX], Ryp[NMAX / 2][NMAX];   // rows 2q and 2q + 1 side by side
  float xix[NMAX];                          // R_x^T l_in,x: own inflow x-trace functional of a row
  float rox[NMAX], roy[NMAX];               // R^T l_out: upwind neighbour outflow-trace functionals
  float liny[NMAX];                         // l_in,y: inflow y-trace of a remapped column
  float l0[NMAX], l1[NMAX], w[NMAX];        // basis at 0 and 1, quadrature weights
  float gm[2 * NMAX + 1];                   // mass row of (C C^T)^+ over the kept residuals
  int o_ks, o_kx, o_ky;                     // mass-target functionals (own, x-, y-neighbour)
  int o_RxT, o_RyT;                         // transposed remap matrices
  int o_g;                                  // face rows of (C C^T)^+ over the kept residuals
  int o_l0, o_l1, o_w;                      // l0, l1, w again, read per thread
  // float-float mass refinement (with the mass row): lam times the outflow-flux functionals of an
  // element's own data through its x- and y-outflow faces ([i][j] tables, row j read by thread j)
  // and their sums; w_i w_j as float-float ([i][j]); the mass column of the pseudo-inverse ([k][j])
  int refine;
  float sfx, sfy;
  int o_fx, o_fy, o_wh, o_wl, o_cm;
};
bool build_mixed2d_const(const sl_ctx* c, double a, double b, double dt, unsigned cons, int rk,
                         std::vector<float>& buf, Mixed2DConstParams& P, std::string& err);
// tile: index of the compiled tile shape (0: default; k2c_tile_count candidates per node count)
void launch_step2d_const(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* status,
                         cudaStream_t s, int tile);
int k2c_tile_count(int n);
void k2c_tile_shape(int n, int tile, int* tx, int* ty);

// Kernel parameter block of the 1D shared-operator (mixed precision) step; passed by value.
struct Mixed1DParams {
  int n, K, left_up, periodic, m, mass_on, energy_on, nst;
  int64_t plane;                         // float offset of the lo plane in a state buffer
  double ghost;
  float lam;                             // |a| dt / h
  float picard_rtol;
  int picard_cap;
  float Gs[NMAX * NMAX], Gu[NMAX * NMAX];  // [j][i]
  float2 Gp[NMAX / 2][2 * NMAX];         // rows 2p and 2p + 1 side by side: [p][i] self, [p][n + i] upwind
  float w[NMAX];
  float fb[3];                           // merged RK weights of the distinct stage times
  float E[3][NMAX];                      // basis at the characteristic feet of the outflow face
  float C[MMAX1D * NMAX];                // linear constraint rows
  float Cp[NMAX * MMAX1D];               // their pseudo-inverse (hard fit)
  // float-float mass refinement (hard fit with the mass row): the outflow-flux functional
  // f = sum_s fb_s E_s, its sum, lam as float-float, the weights as float-float and the column of
  // the pseudo-inverse that belongs to the mass row
  int refine;
  float lam_lo, sumf;
  float Ff[NMAX], wh[NMAX], wl[NMAX], cmass[NMAX];
};

bool build_mixed1d(const sl_ctx* c, const FitOps& fit, double a, double dt, unsigned cons, int rk, int fitmode,
                   Mixed1DParams& P, std::string& err);
void launch_step1d_mixed(const Mixed1DParams& p, const float* in, float* out, unsigned* status, cudaStream_t s);
void launch_pack(int64_t nvals, int64_t plane, const double* src, float* dst, cudaStream_t s);
// Grid of a persistent kernel: its resident CTAs per SM on the current device (occupancy calculator,
// after raising the kernel's dynamic shared-memory limit to smem) times the SM count; cached per
// (device, kernel, threads, smem) under a lock, so host threads on several devices may launch at once.
int persistent_grid(const void* kernel, int threads, size_t smem);
// SMs of the current device (cached per device)
int sm_count();
// Raise a kernel's dynamic shared-memory allowance on the current device to bytes (once per device,
// kernel and size; needed when its static plus dynamic shared memory exceeds 48 KB).
void allow_dynamic_smem(const void* kernel, size_t bytes);
void launch_unpack(int64_t nvals, int64_t plane, const float* src, double* dst, cudaStream_t s);

// float offset of the lo plane of a double-float state of nvals nodes: 256-byte aligned
inline int64_t plane_stride(int64_t nvals) { return (nvals + 63) & ~int64_t(63); }
void launch_mass_energy_f64(int64_t nelem, int nper, const double* phi, const double* w, int dim,
                            int power, double scale, double* partial, double* result, int nblocks,
                            cudaStream_t s);
void launch_mass_energy_pair(int64_t nelem, int nper, int64_t plane, const float* phi, const double* w,
                             int dim, int power, double scale, double* partial, double* result,
                             int nblocks, cudaStream_t s);
void launch_mass_energy_csr(int64_t nel, const int64_t* off, const uint8_t* ord, const uint16_t* prob,
                            const ProbGeom* geo, double area, int precision, int64_t plane, const void* phi,
                            const double* rules, int power, double* partial, double* result, int nblocks,
                            cudaStream_t s);

}  // namespace sl

// ------------------------------------------------------------------ context

// Tables of one node count: basis, fit operators per constraint mask and mode, and their offsets
// in the context's device table buffers.
struct sl_ntab {
  bool present = false;
  sl::Basis1D b;
  sl::FitOps fit[4][2];                  // [linear-row mask][soft]
  size_t off_xi = 0, off_w = 0, off_lam = 0, off_l0 = 0, off_l1 = 0;   // doubles
  size_t table_off[4][2][3] = {};        // Cpinv, S, SCt per mask / mode (doubles)
  size_t f_off[7] = {};                  // xi, lam, w, l0, l1, w2 hi, w2 lo (floats, mixed 2D)
  size_t f_cp[4] = {};                   // float pseudo-inverse per linear-row mask
};

struct sl_ctx {
  sl_mesh mesh{};
  std::vector<int32_t> orders;
  int n = 0, basis = 0, precision = 0;
  cudaStream_t stream = nullptr;
  int64_t nvals = 0;
  sl::Basis1D b;
  // fit operators per constraint mask (index = mask & 3 for linear rows) and fit mode
  sl::FitOps fit[4][2];
  sl_ntab nt[sl::NMAX + 1];              // per node count (the context's n, or every n of a map)
  double* d_tables = nullptr;            // device table buffer
  size_t table_off[4][2][3] = {};        // offsets of Cpinv, S, SCt per mask/mode
  size_t off_xi = 0, off_w = 0, off_lam = 0, off_l0 = 0, off_l1 = 0;
  size_t off_rules = 0;                  // [NMAX + 1][3][NMAX] xi, lam, w of every node count
  unsigned* d_status = nullptr;
  unsigned long long* d_counts = nullptr;   // work counters (SL_CNT_*)
  double* d_partial = nullptr;           // reduction workspace
  double* d_result = nullptr;
  int red_blocks = 0;
  void* d_io = nullptr;                  // device buffers for sl_run_host
  double* d_io64 = nullptr;
  double* d_work = nullptr;              // 2D workspace between the two phases
  float* d_ftab = nullptr;               // float tables of the mixed 2D path
  size_t f_rules = 0;                    // float copy of the rules table
  // element map: p-adaptive meshes and batches of problems (general 2D kernels)
  bool mapped = false;
  int nprob = 1;
  int64_t nel = 0;                       // elements (all problems)
  std::vector<uint8_t> ord_host;         // node count per element
  std::vector<int64_t> off_host;         // value offset per element, then the total
  std::vector<sl_mesh> prob_mesh;        // meshes of the problems of a batch
  std::vector<sl::ProbGeom> geo_host;
  int64_t bucket_start[sl::NMAX + 1] = {}, bucket_count[sl::NMAX + 1] = {};
  int64_t* d_off = nullptr;
  uint8_t* d_ord = nullptr;
  uint16_t* d_prob = nullptr;
  sl::ProbGeom* d_geo = nullptr;
  int* d_list = nullptr;                 // element lists of the node-count buckets
  // sl_run: steps captured into a CUDA graph on an internal stream, kept for identical calls
  cudaStream_t run_stream = nullptr;
  cudaEvent_t run_ev[2] = {};
  cudaGraphExec_t run_exec = nullptr;
  bool run_valid = false;
  std::vector<double> run_key;
  sl::ProbGeom* d_geo_run = nullptr;     // per-step geometry of a batch run, [nsteps][nprob]
  size_t geo_run_cap = 0;
  const sl::ProbGeom* geo_override = nullptr;
  // cached shared operator of the mixed 2D constant-velocity path
  bool m2c_valid = false;
  double m2c_a = 0, m2c_b = 0, m2c_dt = 0;
  unsigned m2c_cons = 0;
  int m2c_rk = 0;
  std::vector<float> m2c_host;
  float* d_m2c = nullptr;
  size_t m2c_cap = 0;
  sl::Mixed2DConstParams m2c{};
  size_t f_off[7] = {};                  // xi, lam, w, l0, l1, w2 hi, w2 lo
  size_t f_cp[4] = {};                   // float pseudo-inverse per linear-row mask
  // cached shared operator of the mixed 1D path, keyed on (a, dt, constraints, rk, fit)
  bool mix_valid = false;
  double mix_a = 0, mix_dt = 0;
  unsigned mix_cons = 0;
  int mix_rk = 0, mix_fit = 0;
  sl::Mixed1DParams mix{};
  // kernel timing (sl_timing): three events per timed step (start, between the two phases, end)
  bool timing = false;
  bool capturing = false;                // sl_run is recording its graph
  std::vector<cudaEvent_t> tev;          // 3 per step, reused across timing sessions
  size_t tused = 0;                      // events of the current session
  std::vector<char> tdone;               // per timed step: its end event was recorded
  // time-dependent inflow records (sl_set_inflow); inflow_step is the record of the step being
  // enqueued
  const double* inflow = nullptr;
  int64_t inflow_stride = 0;
  const double* inflow_step = nullptr;
  // launch shapes chosen by the autotuner (sl_tune): the shared-operator kernel's tile, and the
  // resident CTAs per SM of the general mixed kernels' two phases (0: the defaults)
  int k2c_tile = 0;
  int k2m_per_sm[2] = {0, 0};
  std::string err;
};
