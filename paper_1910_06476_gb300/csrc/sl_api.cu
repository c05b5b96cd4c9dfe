// C ABI of the DSEM-SL library (declared in include/sl.h): argument checking, table upload,
// dispatch of the step kernels, deterministic diagnostics and the host-buffer run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "sl_internal.h"

using namespace sl;

namespace {

thread_local std::string g_init_err;

sl_status fail(sl_ctx* c, sl_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_init_err = msg;
  return st;
}

#define SL_CUDA(ctx, call)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(ctx, SL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// bytes of one state buffer: nvals doubles (SL_FP64), or a hi and a lo plane of floats whose
// lo plane starts at a 256-byte aligned float offset (SL_MIXED)
size_t state_bytes(const sl_ctx* c) {
  return c->precision == SL_FP64 ? (size_t)c->nvals * sizeof(double) : (size_t)2 * plane_stride(c->nvals) * sizeof(float);
}

void max_speed(const sl_ctx* c, const sl_velocity* v, double& um, double& vm) {
  const sl_mesh& M = c->mesh;
  um = vm = 0.0;
  switch (v->kind) {
    case SL_VEL_CONST: um = std::fabs(v->p[0]); vm = std::fabs(v->p[1]); break;
    case SL_VEL_ROTATION: {
      const double om = std::fabs(v->p[0]);
      um = om * std::max(std::fabs(M.y0 - v->p[2]), std::fabs(M.y1 - v->p[2]));
      vm = om * std::max(std::fabs(M.x0 - v->p[1]), std::fabs(M.x1 - v->p[1]));
      break;
    }
    case SL_VEL_SWIRL: um = vm = 1.0; break;
    case SL_VEL_SINX: um = 1.0; vm = 0.0; break;
    default: break;
  }
}

bool valid_velocity(const sl_ctx* c, const sl_velocity* v) {
  if (!v) return false;
  if (v->kind < SL_VEL_CONST || v->kind > SL_VEL_SINX) return false;
  if (c->mesh.dim == 1 && (v->kind == SL_VEL_ROTATION || v->kind == SL_VEL_SWIRL)) return false;
  if (c->mesh.dim == 2 && v->kind == SL_VEL_SINX) return false;
  if (v->kind == SL_VEL_SWIRL && !(v->p[0] != 0.0)) return false;
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(v->p[i])) return false;
  return true;
}

}  // namespace

namespace sl {
void set_global_error(const std::string& msg) { g_init_err = msg; }
}  // namespace sl

extern "C" {

sl_status sl_init(const sl_mesh* mesh, int n, int basis, int precision, void* cuda_stream, sl_ctx** out) {
  if (!out) return fail(nullptr, SL_EINVAL, "out is null");
  *out = nullptr;
  if (!mesh) return fail(nullptr, SL_EINVAL, "mesh is null");
  if (mesh->dim != 1 && mesh->dim != 2) return fail(nullptr, SL_EINVAL, "dim must be 1 or 2");
  if (mesh->kx < 1 || mesh->ky < 1 || (mesh->dim == 1 && mesh->ky != 1))
    return fail(nullptr, SL_EINVAL, "element counts must be >= 1 (ky = 1 in 1D)");
  if (!(mesh->x1 > mesh->x0) || (mesh->dim == 2 && !(mesh->y1 > mesh->y0)))
    return fail(nullptr, SL_EINVAL, "empty domain box");
  for (int f = 0; f < 4; ++f)
    if (mesh->bc[f] != SL_BC_PERIODIC && mesh->bc[f] != SL_BC_INFLOW) return fail(nullptr, SL_EINVAL, "bad bc");
  if ((mesh->bc[0] == SL_BC_PERIODIC) != (mesh->bc[1] == SL_BC_PERIODIC) ||
      (mesh->dim == 2 && (mesh->bc[2] == SL_BC_PERIODIC) != (mesh->bc[3] == SL_BC_PERIODIC)))
    return fail(nullptr, SL_EINVAL, "periodic faces must come in pairs");
  if (basis != SL_GAUSS_LEGENDRE && basis != SL_CHEB_GAUSS) return fail(nullptr, SL_EINVAL, "bad basis");
  if (precision != SL_FP64 && precision != SL_MIXED) return fail(nullptr, SL_EINVAL, "bad precision");
  if (mesh->order) return fail(nullptr, SL_EUNSUPPORTED, "p-adaptive meshes are not built yet");
  if (n < 2 || n > NMAX) return fail(nullptr, SL_EINVAL, "n must lie in [2, 17]");
  if ((int64_t)mesh->kx * mesh->ky > (int64_t)1 << 31) return fail(nullptr, SL_EINVAL, "too many elements");

  sl_ctx* c = new (std::nothrow) sl_ctx();
  if (!c) return fail(nullptr, SL_ENOMEM, "host allocation failed");
  c->mesh = *mesh;
  c->mesh.order = nullptr;
  c->n = n;
  c->basis = basis;
  c->precision = precision;
  c->stream = (cudaStream_t)cuda_stream;
  const int64_t nel = (int64_t)mesh->kx * mesh->ky;
  const int nd = mesh->dim == 1 ? n : n * n;
  c->nvals = nel * nd;
  try {
    c->b = make_basis(n, basis);
    for (unsigned mask = 0; mask < 4; ++mask)
      for (int soft = 0; soft < 2; ++soft) {
        if (mesh->dim == 1) {
          c->fit[mask][soft] = make_fit_1d(c->b, mask);
          finish_fit(c->fit[mask][soft], soft != 0);
        } else {
          c->fit[mask][soft] = make_fit_2d(c->b, mask, soft != 0);
        }
      }
  } catch (const std::exception& ex) {
    std::string msg = ex.what();
    delete c;
    return fail(nullptr, SL_EINVAL, "table construction failed: " + msg);
  }
  // one device buffer: basis tables then per (mask, mode) operators
  std::vector<double> host;
  auto put = [&](const std::vector<double>& v, size_t pad) {
    size_t off = host.size();
    host.insert(host.end(), v.begin(), v.end());
    host.resize(off + std::max(pad, v.size()), 0.0);
    host.resize((host.size() + 1) & ~size_t(1), 0.0);     // keep 16-byte alignment
    return off;
  };
  c->off_xi = put(c->b.xi, NMAX);
  c->off_w = put(c->b.w, NMAX);
  c->off_lam = put(c->b.lam, NMAX);
  c->off_l0 = put(c->b.l0, NMAX);
  c->off_l1 = put(c->b.l1, NMAX);
  for (int mask = 0; mask < 4; ++mask)
    for (int soft = 0; soft < 2; ++soft) {
      const FitOps& f = c->fit[mask][soft];
      c->table_off[mask][soft][0] = put(f.Cpinv, 1);
      c->table_off[mask][soft][1] = put(f.S, 1);
      c->table_off[mask][soft][2] = put(f.SCt, 1);
    }
  c->red_blocks = 2 * 152;
  // float copies of the tables for the mixed 2D kernels
  std::vector<float> ftab;
  auto fput = [&](const std::vector<double>& v) {
    size_t off = ftab.size();
    for (double x : v) ftab.push_back((float)x);
    ftab.resize(off + std::max<size_t>(v.size(), NMAX), 0.0f);
    ftab.resize((ftab.size() + 3) & ~size_t(3), 0.0f);
    return off;
  };
  if (mesh->dim == 2 && precision == SL_MIXED) {
    c->f_off[0] = fput(c->b.xi);
    c->f_off[1] = fput(c->b.lam);
    c->f_off[2] = fput(c->b.w);
    c->f_off[3] = fput(c->b.l0);
    c->f_off[4] = fput(c->b.l1);
    for (int mask = 0; mask < 4; ++mask) c->f_cp[mask] = fput(c->fit[mask][0].Cpinv);
  }
  const size_t work_bytes = mesh->dim != 2 ? 0
                            : precision == SL_FP64 ? work2d_doubles(nel, n) * sizeof(double)
                                                   : work2m_floats(nel, n) * sizeof(float);
  if (cudaMalloc(&c->d_tables, host.size() * sizeof(double)) != cudaSuccess ||
      (work_bytes && cudaMalloc(&c->d_work, work_bytes) != cudaSuccess) ||
      (!ftab.empty() && cudaMalloc(&c->d_ftab, ftab.size() * sizeof(float)) != cudaSuccess) ||
      cudaMalloc(&c->d_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->d_partial, c->red_blocks * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_result, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    sl_free(c);
    return fail(nullptr, SL_ENOMEM, "device allocation failed");
  }
  if (cudaMemcpy(c->d_tables, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      (!ftab.empty() &&
       cudaMemcpy(c->d_ftab, ftab.data(), ftab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
    std::string msg = cudaGetErrorString(cudaGetLastError());
    sl_free(c);
    return fail(nullptr, SL_ECUDA, "table upload failed: " + msg);
  }
  *out = c;
  return SL_OK;
}

void sl_free(sl_ctx* c) {
  if (!c) return;
  cudaFree(c->d_tables);
  cudaFree(c->d_status);
  cudaFree(c->d_partial);
  cudaFree(c->d_result);
  cudaFree(c->d_io);
  cudaFree(c->d_io64);
  cudaFree(c->d_work);
  cudaFree(c->d_ftab);
  cudaFree(c->d_m2c);
  delete c;
}

sl_status sl_step(sl_ctx* c, const void* phi_in, void* phi_out, const sl_velocity* vel, double t, double dt,
                  const sl_options* opt) {
  if (!c) return SL_EINVAL;
  if (!phi_in || !phi_out || !opt) return fail(c, SL_EINVAL, "null argument");
  if (phi_in == phi_out) return fail(c, SL_EINVAL, "phi_in and phi_out must be distinct buffers");
  if (!valid_velocity(c, vel)) return fail(c, SL_EINVAL, "bad velocity for this mesh");
  if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t)) return fail(c, SL_EINVAL, "dt must be finite and > 0");
  if (opt->rk_order < 1 || opt->rk_order > 4) return fail(c, SL_EINVAL, "rk_order must be 1..4");
  if (opt->fit != SL_FIT_HARD && opt->fit != SL_FIT_SOFT) return fail(c, SL_EINVAL, "bad fit mode");
  if (opt->bvalue != SL_BV_INTERP && opt->bvalue != SL_BV_BACKTRACK) return fail(c, SL_EINVAL, "bad bvalue");
  if (opt->constraints & ~7u) return fail(c, SL_EINVAL, "unknown constraint bits");
  if (opt->picard_rtol < 0.0 || opt->picard_cap < 0) return fail(c, SL_EINVAL, "bad energy iteration limits");
  const sl_mesh& M = c->mesh;
  const double hx = (M.x1 - M.x0) / M.kx, hy = M.dim == 2 ? (M.y1 - M.y0) / M.ky : 1.0;
  double um, vm;
  max_speed(c, vel, um, vm);
  if (um * dt > hx || (M.dim == 2 && vm * dt > hy))
    return fail(c, SL_ECFL, "displacement over the step exceeds one element width");

  StepParams P{};
  P.K = M.kx;
  P.kx = M.kx;
  P.ky = M.ky;
  P.x0 = M.x0;
  P.hx = hx;
  P.y0 = M.y0;
  P.hy = hy;
  for (int f = 0; f < 4; ++f) P.bc[f] = M.bc[f];
  P.ghost = M.ghost;
  P.vel_kind = vel->kind;
  for (int i = 0; i < 6; ++i) P.vp[i] = vel->p[i];
  P.t = t;
  P.dt = dt;
  P.rk = opt->rk_order;
  P.cons = opt->constraints;
  P.fit = opt->fit;
  P.bvalue = opt->bvalue;
  const unsigned lin = opt->constraints & 3u;
  P.m = c->fit[lin][opt->fit == SL_FIT_SOFT].m;
  P.picard_rtol = opt->picard_rtol > 0.0 ? opt->picard_rtol : 1e-13;
  P.picard_cap = opt->picard_cap > 0 ? opt->picard_cap : 60;

  const double* T = c->d_tables;
  const size_t* off = c->table_off[lin][opt->fit == SL_FIT_SOFT];
  if (M.dim == 1 && c->precision == SL_FP64) {
    Tables1D tb{T + c->off_xi, T + c->off_w, T + c->off_lam, T + c->off_l0, T + c->off_l1,
                T + off[0], T + off[1], T + off[2]};
    launch_step1d_f64(c->n, P, tb, (const double*)phi_in, (double*)phi_out, c->d_status, c->stream);
  } else if (M.dim == 1 && c->precision == SL_MIXED) {
    if (vel->kind != SL_VEL_CONST)
      return fail(c, SL_EUNSUPPORTED, "the 1D mixed path needs a constant velocity (shared operator)");
    if (opt->bvalue != SL_BV_INTERP)
      return fail(c, SL_EUNSUPPORTED, "the 1D mixed path uses interpolated interface values");
    if (!c->mix_valid || c->mix_a != vel->p[0] || c->mix_dt != dt || c->mix_cons != opt->constraints ||
        c->mix_rk != opt->rk_order || c->mix_fit != opt->fit) {
      std::string why;
      if (!build_mixed1d(c, c->fit[lin][opt->fit == SL_FIT_SOFT], vel->p[0], dt, opt->constraints, opt->rk_order,
                         opt->fit, c->mix, why))
        return fail(c, SL_EUNSUPPORTED, why);
      c->mix_valid = true;
      c->mix_a = vel->p[0];
      c->mix_dt = dt;
      c->mix_cons = opt->constraints;
      c->mix_rk = opt->rk_order;
      c->mix_fit = opt->fit;
    }
    c->mix.plane = plane_stride(c->nvals);
    c->mix.picard_rtol = (float)P.picard_rtol;
    c->mix.picard_cap = P.picard_cap;
    launch_step1d_mixed(c->mix, (const float*)phi_in, (float*)phi_out, c->d_status, c->stream);
  } else if (M.dim == 2 && c->precision == SL_FP64) {
    if (opt->bvalue != SL_BV_INTERP)
      return fail(c, SL_EUNSUPPORTED, "2D interface values are interpolated (eq. 2dx/2dy_bnd_interpolate)");
    Tables1D tb{T + c->off_xi, T + c->off_w, T + c->off_lam, T + c->off_l0, T + c->off_l1,
                T + off[0], T + off[1], T + off[2]};
    launch_step2d_f64(c->n, P, tb, (const double*)phi_in, (double*)phi_out, c->d_work, c->d_status, c->stream);
  } else if (M.dim == 2 && c->precision == SL_MIXED && vel->kind == SL_VEL_CONST && vel->p[0] != 0.0 &&
             vel->p[1] != 0.0 && opt->fit == SL_FIT_HARD && !(opt->constraints & SL_C_ENERGY) &&
             opt->bvalue == SL_BV_INTERP && (opt->constraints & 3u)) {
    // uniform mesh, constant velocity: one operator shared by all elements
    if (!c->m2c_valid || c->m2c_a != vel->p[0] || c->m2c_b != vel->p[1] || c->m2c_dt != dt ||
        c->m2c_cons != opt->constraints || c->m2c_rk != opt->rk_order) {
      std::string why;
      if (!build_mixed2d_const(c, vel->p[0], vel->p[1], dt, opt->constraints, opt->rk_order, c->m2c_host, c->m2c, why))
        return fail(c, SL_EUNSUPPORTED, why);
      if (c->m2c_host.size() > c->m2c_cap) {
        cudaFree(c->d_m2c);
        c->d_m2c = nullptr;
        c->m2c_cap = 0;
        if (cudaMalloc(&c->d_m2c, c->m2c_host.size() * sizeof(float)) != cudaSuccess) {
          cudaGetLastError();
          return fail(c, SL_ENOMEM, "device allocation of the shared operator failed");
        }
        c->m2c_cap = c->m2c_host.size();
      }
      SL_CUDA(c, cudaMemcpyAsync(c->d_m2c, c->m2c_host.data(), c->m2c_host.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, c->stream));
      c->m2c_valid = true;
      c->m2c_a = vel->p[0];
      c->m2c_b = vel->p[1];
      c->m2c_dt = dt;
      c->m2c_cons = opt->constraints;
      c->m2c_rk = opt->rk_order;
    }
    c->m2c.plane = plane_stride(c->nvals);
    launch_step2d_const(c->m2c, c->d_m2c, (const float*)phi_in, (float*)phi_out, c->d_status, c->stream);
  } else if (M.dim == 2 && c->precision == SL_MIXED) {
    if (opt->bvalue != SL_BV_INTERP)
      return fail(c, SL_EUNSUPPORTED, "2D interface values are interpolated (eq. 2dx/2dy_bnd_interpolate)");
    if (opt->fit != SL_FIT_HARD) return fail(c, SL_EUNSUPPORTED, "the 2D mixed path uses the hard fit");
    const float* F = c->d_ftab;
    Mixed2DExtra X{F + c->f_off[0], F + c->f_off[1], F + c->f_off[2], F + c->f_off[3], F + c->f_off[4],
                   F + c->f_cp[lin], plane_stride(c->nvals),
                   (float)hx, (float)hy, (float)(1.0 / hx), (float)(1.0 / hy),
                   (float)vel->p[0], (float)vel->p[1], (float)vel->p[0], (float)vel->p[1], (float)vel->p[2],
                   0.0f, 0.0f, (float)dt, (float)(dt / (hx * hy))};
    if (vel->kind == SL_VEL_SWIRL) {
      X.tT = (float)(t / vel->p[0]);
      X.dtT = (float)(dt / vel->p[0]);
    }
    launch_step2d_mixed(c->n, P, X, (const float*)phi_in, (float*)phi_out, (float*)c->d_work, c->d_status,
                        c->stream);
  } else {
    return fail(c, SL_EUNSUPPORTED, "this dimension/precision combination is not built yet");
  }
  SL_CUDA(c, cudaGetLastError());
  return SL_OK;
}

sl_status sl_run_host(sl_ctx* c, const double* host_in, double* host_out, const sl_velocity* vel, double t0,
                      double dt, int nsteps, const sl_options* opt) {
  if (!c) return SL_EINVAL;
  if (!host_in || !host_out || nsteps < 0) return fail(c, SL_EINVAL, "bad host buffers or step count");
  const size_t bytes = state_bytes(c);
  if (!c->d_io) {
    if (cudaMalloc(&c->d_io, 2 * bytes) != cudaSuccess) {
      cudaGetLastError();
      c->d_io = nullptr;
      return fail(c, SL_ENOMEM, "device allocation of the run buffers failed");
    }
    if (c->precision == SL_MIXED && cudaMalloc(&c->d_io64, (size_t)c->nvals * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->d_io);
      c->d_io = nullptr;
      c->d_io64 = nullptr;
      return fail(c, SL_ENOMEM, "device allocation of the run buffers failed");
    }
  }
  char* a = (char*)c->d_io;
  char* b = a + bytes;
  if (c->precision == SL_FP64) {
    SL_CUDA(c, cudaMemcpyAsync(a, host_in, bytes, cudaMemcpyHostToDevice, c->stream));
  } else {
    SL_CUDA(c, cudaMemcpyAsync(c->d_io64, host_in, (size_t)c->nvals * sizeof(double), cudaMemcpyHostToDevice,
                               c->stream));
    launch_pack(c->nvals, plane_stride(c->nvals), c->d_io64, (float*)a, c->stream);
  }
  for (int s = 0; s < nsteps; ++s) {
    sl_status st = sl_step(c, a, b, vel, t0 + s * dt, dt, opt);
    if (st != SL_OK) return st;
    std::swap(a, b);
  }
  if (c->precision == SL_FP64) {
    SL_CUDA(c, cudaMemcpyAsync(host_out, a, bytes, cudaMemcpyDeviceToHost, c->stream));
  } else {
    launch_unpack(c->nvals, plane_stride(c->nvals), (const float*)a, c->d_io64, c->stream);
    SL_CUDA(c, cudaMemcpyAsync(host_out, c->d_io64, (size_t)c->nvals * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  }
  SL_CUDA(c, cudaStreamSynchronize(c->stream));
  return SL_OK;
}

sl_status sl_pack(sl_ctx* c, const double* src, void* dst) {
  if (!c) return SL_EINVAL;
  if (!src || !dst) return fail(c, SL_EINVAL, "null argument");
  if (c->precision == SL_FP64)
    SL_CUDA(c, cudaMemcpyAsync(dst, src, (size_t)c->nvals * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  else
    launch_pack(c->nvals, plane_stride(c->nvals), src, (float*)dst, c->stream);
  SL_CUDA(c, cudaGetLastError());
  return SL_OK;
}

sl_status sl_unpack(sl_ctx* c, const void* src, double* dst) {
  if (!c) return SL_EINVAL;
  if (!src || !dst) return fail(c, SL_EINVAL, "null argument");
  if (c->precision == SL_FP64)
    SL_CUDA(c, cudaMemcpyAsync(dst, src, (size_t)c->nvals * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  else
    launch_unpack(c->nvals, plane_stride(c->nvals), (const float*)src, dst, c->stream);
  SL_CUDA(c, cudaGetLastError());
  return SL_OK;
}

static sl_status integral(sl_ctx* c, const void* phi, double* total, int power) {
  if (!c) return SL_EINVAL;
  if (!phi || !total) return fail(c, SL_EINVAL, "null argument");
  const sl_mesh& M = c->mesh;
  const double hx = (M.x1 - M.x0) / M.kx, hy = M.dim == 2 ? (M.y1 - M.y0) / M.ky : 1.0;
  const int64_t nel = (int64_t)M.kx * M.ky;
  if (c->precision == SL_FP64)
    launch_mass_energy_f64(nel, c->n, (const double*)phi, c->d_tables + c->off_w, M.dim, power, hx * hy,
                           c->d_partial, c->d_result, c->red_blocks, c->stream);
  else
    launch_mass_energy_pair(nel, c->n, plane_stride(c->nvals), (const float*)phi, c->d_tables + c->off_w, M.dim,
                            power, hx * hy, c->d_partial, c->d_result, c->red_blocks, c->stream);
  SL_CUDA(c, cudaGetLastError());
  SL_CUDA(c, cudaMemcpyAsync(total, c->d_result, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SL_CUDA(c, cudaStreamSynchronize(c->stream));
  return SL_OK;
}

sl_status sl_mass(sl_ctx* c, const void* phi, double* total) { return integral(c, phi, total, 1); }
sl_status sl_energy(sl_ctx* c, const void* phi, double* total) { return integral(c, phi, total, 2); }

sl_status sl_sync(sl_ctx* c, uint32_t* bits) {
  if (!c) return SL_EINVAL;
  unsigned h = 0;
  SL_CUDA(c, cudaStreamSynchronize(c->stream));
  SL_CUDA(c, cudaMemcpy(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  SL_CUDA(c, cudaMemset(c->d_status, 0, sizeof(unsigned)));
  if (bits) *bits = h;
  return h ? SL_EDEVICE : SL_OK;
}

sl_status sl_max_dt(const sl_ctx* c, const sl_velocity* vel, int rule, double* dt) {
  if (!c || !dt) return SL_EINVAL;
  if (!valid_velocity(c, vel)) return fail(const_cast<sl_ctx*>(c), SL_EINVAL, "bad velocity");
  if (rule != SL_RULE_HALF_MIN_SPACING && rule != SL_RULE_PAPER) return fail(const_cast<sl_ctx*>(c), SL_EINVAL, "bad rule");
  const std::vector<double>& xi = c->b.xi;
  double gap;
  if (rule == SL_RULE_PAPER) gap = xi[0];
  else {
    gap = 1.0;
    for (size_t i = 1; i < xi.size(); ++i) gap = std::min(gap, xi[i] - xi[i - 1]);
  }
  const double factor = rule == SL_RULE_PAPER ? 1.0 : 0.5;
  const sl_mesh& M = c->mesh;
  double um, vm;
  max_speed(c, vel, um, vm);
  double lim = INFINITY;
  if (um > 0) lim = std::min(lim, (M.x1 - M.x0) / M.kx * gap / um);
  if (M.dim == 2 && vm > 0) lim = std::min(lim, (M.y1 - M.y0) / M.ky * gap / vm);
  if (!std::isfinite(lim)) return fail(const_cast<sl_ctx*>(c), SL_EINVAL, "velocity is zero everywhere");
  *dt = factor * lim;
  return SL_OK;
}

int64_t sl_state_size(const sl_ctx* c) { return c ? c->nvals : -1; }

int64_t sl_state_bytes(const sl_ctx* c) { return c ? (int64_t)state_bytes(c) : -1; }

sl_status sl_node_coords(const sl_ctx* c, double* x, double* y) {
  if (!c || !x || (c->mesh.dim == 2 && !y)) return SL_EINVAL;
  const sl_mesh& M = c->mesh;
  const int n = c->n;
  const double hx = (M.x1 - M.x0) / M.kx, hy = M.dim == 2 ? (M.y1 - M.y0) / M.ky : 1.0;
  if (M.dim == 1) {
    for (int k = 0; k < M.kx; ++k)
      for (int i = 0; i < n; ++i) x[(int64_t)k * n + i] = M.x0 + (k + c->b.xi[i]) * hx;
    return SL_OK;
  }
  for (int ey = 0; ey < M.ky; ++ey)
    for (int ex = 0; ex < M.kx; ++ex)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const int64_t o = (((int64_t)ey * M.kx + ex) * n + j) * n + i;
          x[o] = M.x0 + (ex + c->b.xi[i]) * hx;
          y[o] = M.y0 + (ey + c->b.xi[j]) * hy;
        }
  return SL_OK;
}

sl_status sl_nodes_weights(const sl_ctx* c, int n, double* xi, double* w) {
  if (!c || !xi || !w || n < 1 || n > NMAX) return SL_EINVAL;
  Basis1D b = make_basis(n, c->basis);
  for (int i = 0; i < n; ++i) { xi[i] = b.xi[i]; w[i] = b.w[i]; }
  return SL_OK;
}

const char* sl_last_error(const sl_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }

}  // extern "C"
