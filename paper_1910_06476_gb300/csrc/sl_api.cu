// C ABI of the DSEM-SL library (declared in include/sl.h): argument checking, table upload,
// dispatch of the step kernels, deterministic diagnostics and the host-buffer run.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

#include "sl_internal.h"
#include "tune_cache.h"

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

void max_speed(const sl_mesh& M, const sl_velocity* v, double& um, double& vm) {
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
    case SL_VEL_NODAL: um = v->p[0]; vm = M.dim == 2 ? v->p[1] : 0.0; break;
    default: break;
  }
}

bool valid_velocity(const sl_ctx* c, const sl_velocity* v) {
  if (!v) return false;
  if (v->kind < SL_VEL_CONST || v->kind > SL_VEL_NODAL) return false;
  if (v->kind == SL_VEL_NODAL &&
      (!v->nodal || ((uintptr_t)v->nodal & 7u) || v->nodal_step < 0 || !(v->p[0] >= 0.0) || !(v->p[1] >= 0.0)))
    return false;
  if (c->mesh.dim == 1 && (v->kind == SL_VEL_ROTATION || v->kind == SL_VEL_SWIRL)) return false;
  if (c->mesh.dim == 2 && v->kind == SL_VEL_SINX) return false;
  if (v->kind == SL_VEL_SWIRL && !(v->p[0] != 0.0)) return false;
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(v->p[i])) return false;
  return true;
}

// Host and float table buffers of a context under construction.
struct TableBufs {
  std::vector<double> host;
  std::vector<float> ftab;
  size_t put(const std::vector<double>& v, size_t pad) {
    size_t off = host.size();
    host.insert(host.end(), v.begin(), v.end());
    host.resize(off + std::max(pad, v.size()), 0.0);
    host.resize((host.size() + 1) & ~size_t(1), 0.0);     // keep 16-byte alignment
    return off;
  }
  size_t fput(const std::vector<double>& v) {
    size_t off = ftab.size();
    for (double x : v) ftab.push_back((float)x);
    ftab.resize(off + std::max<size_t>(v.size(), NMAX), 0.0f);
    ftab.resize((ftab.size() + 3) & ~size_t(3), 0.0f);
    return off;
  }
};

// Basis and fit operators of one (node count, basis, dimension): built once per process (they
// cost up to about a second each at n = 17) and shared by every context.
struct HostOps {
  Basis1D b;
  FitOps fit[4][2];
};

std::shared_ptr<const HostOps> host_ops(int n, int basis, int dim) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, std::shared_ptr<const HostOps>> cache;
  const auto key = std::make_tuple(n, basis, dim);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  auto h = std::make_shared<HostOps>();
  h->b = make_basis(n, basis);
  for (unsigned mask = 0; mask < 4; ++mask)
    for (int soft = 0; soft < 2; ++soft) {
      if (dim == 1) {
        h->fit[mask][soft] = make_fit_1d(h->b, mask);
        finish_fit(h->fit[mask][soft], soft != 0);
      } else {
        h->fit[mask][soft] = make_fit_2d(h->b, mask, soft != 0);
      }
    }
  std::lock_guard<std::mutex> lock(mu);
  return cache.emplace(key, std::move(h)).first->second;
}

// basis and fit operators of node count n, appended to the table buffers (throws on failure)
void build_ntab(sl_ntab& t, int n, int basis, int dim, bool mixed2d, TableBufs& B) {
  t.present = true;
  const std::shared_ptr<const HostOps> h = host_ops(n, basis, dim);
  t.b = h->b;
  for (unsigned mask = 0; mask < 4; ++mask)
    for (int soft = 0; soft < 2; ++soft) t.fit[mask][soft] = h->fit[mask][soft];
  t.off_xi = B.put(t.b.xi, NMAX);
  t.off_w = B.put(t.b.w, NMAX);
  t.off_lam = B.put(t.b.lam, NMAX);
  t.off_l0 = B.put(t.b.l0, NMAX);
  t.off_l1 = B.put(t.b.l1, NMAX);
  for (int mask = 0; mask < 4; ++mask)
    for (int soft = 0; soft < 2; ++soft) {
      const FitOps& f = t.fit[mask][soft];
      t.table_off[mask][soft][0] = B.put(f.Cpinv, 1);
      t.table_off[mask][soft][1] = B.put(f.S, 1);
      t.table_off[mask][soft][2] = B.put(f.SCt, 1);
    }
  if (mixed2d) {
    t.f_off[0] = B.fput(t.b.xi);
    t.f_off[1] = B.fput(t.b.lam);
    t.f_off[2] = B.fput(t.b.w);
    t.f_off[3] = B.fput(t.b.l0);
    t.f_off[4] = B.fput(t.b.l1);
    // w_i w_j formed in double, as float-float (the element mass of the mixed path's refinement)
    std::vector<double> w2h((size_t)n * n), w2l((size_t)n * n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const double v = t.b.w[i] * t.b.w[j];
        w2h[(size_t)j * n + i] = (double)(float)v;
        w2l[(size_t)j * n + i] = v - (double)(float)v;
      }
    t.f_off[5] = B.fput(w2h);
    t.f_off[6] = B.fput(w2l);
    // the float pseudo-inverse is stored row of C first ([k][node]), so that the threads of an
    // element (one per node) read consecutive floats
    for (int mask = 0; mask < 4; ++mask) {
      const FitOps& f = t.fit[mask][0];
      std::vector<double> tr(f.Cpinv.size());
      for (int q = 0; q < f.nd; ++q)
        for (int k = 0; k < f.m; ++k) tr[(size_t)k * f.nd + q] = f.Cpinv[(size_t)q * f.m + k];
      t.f_cp[mask] = B.fput(tr);
    }
  }
}

// nodes, barycentric weights and quadrature weights of every node count, [NMAX + 1][3][NMAX]
void build_rules(int basis, TableBufs& B, size_t& off, size_t& foff) {
  std::vector<double> r((size_t)(NMAX + 1) * 3 * NMAX, 0.0);
  for (int n = 2; n <= NMAX; ++n) {
    const Basis1D b = make_basis(n, basis);
    for (int i = 0; i < n; ++i) {
      r[((size_t)n * 3 + 0) * NMAX + i] = b.xi[i];
      r[((size_t)n * 3 + 1) * NMAX + i] = b.lam[i];
      r[((size_t)n * 3 + 2) * NMAX + i] = b.w[i];
    }
  }
  off = B.put(r, 1);
  foff = B.fput(r);
}

}  // namespace

namespace sl {
void set_global_error(const std::string& msg) { g_init_err = msg; }

int sm_count() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return 152;
  }
  cache.emplace(dev, sms);
  return sms;
}

int persistent_grid(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  const auto key = std::make_tuple(dev, kernel, threads, smem);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  // the dynamic allowance is raised whenever a kernel takes any: static plus dynamic shared memory
  // above 48 KB needs it, whatever the split
  // A failed call leaves its error as the last error; it is cleared here, which loses nothing:
  // every kernel launch is checked as soon as it is enqueued, so no earlier error is pending.
  if (smem > 0 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    cudaGetLastError();
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) {
    per_sm = 1;
    cudaGetLastError();
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    sms = 152;
    cudaGetLastError();
  }
  const int grid = std::max(1, per_sm) * std::max(1, sms);
  cache.emplace(key, grid);
  return grid;
}
void allow_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*>, size_t> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[std::make_tuple(dev, kernel)];
  if (bytes <= have) return;
  // a failure is cleared here and shows as a failed launch, which is checked when enqueued
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    cudaGetLastError();
  else
    have = bytes;
}
}  // namespace sl

namespace {

// copy the tables of the context's own node count into the fields the uniform paths use
void alias_ntab(sl_ctx* c) {
  const sl_ntab& T = c->nt[c->n];
  c->b = T.b;
  for (int m = 0; m < 4; ++m)
    for (int s = 0; s < 2; ++s) {
      c->fit[m][s] = T.fit[m][s];
      for (int k = 0; k < 3; ++k) c->table_off[m][s][k] = T.table_off[m][s][k];
    }
  c->off_xi = T.off_xi;
  c->off_w = T.off_w;
  c->off_lam = T.off_lam;
  c->off_l0 = T.off_l0;
  c->off_l1 = T.off_l1;
  for (int k = 0; k < 7; ++k) c->f_off[k] = T.f_off[k];
  for (int k = 0; k < 4; ++k) c->f_cp[k] = T.f_cp[k];
}

// device allocations and table upload; frees the context on failure
sl_status alloc_upload(sl_ctx* c, const TableBufs& B, size_t work_bytes) {
  c->red_blocks = 2 * 152;
  if (cudaMalloc(&c->d_tables, B.host.size() * sizeof(double)) != cudaSuccess ||
      (work_bytes && cudaMalloc(&c->d_work, work_bytes) != cudaSuccess) ||
      (!B.ftab.empty() && cudaMalloc(&c->d_ftab, B.ftab.size() * sizeof(float)) != cudaSuccess) ||
      cudaMalloc(&c->d_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->d_counts, SL_NCOUNTERS * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->d_partial, c->red_blocks * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_result, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    sl_free(c);
    return fail(nullptr, SL_ENOMEM, "device allocation failed");
  }
  if (cudaMemcpy(c->d_tables, B.host.data(), B.host.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      (!B.ftab.empty() &&
       cudaMemcpy(c->d_ftab, B.ftab.data(), B.ftab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->d_counts, 0, SL_NCOUNTERS * sizeof(unsigned long long)) != cudaSuccess) {
    std::string msg = cudaGetErrorString(cudaGetLastError());
    sl_free(c);
    return fail(nullptr, SL_ECUDA, "table upload failed: " + msg);
  }
  return SL_OK;
}

sl_status finish_uniform(sl_ctx* c) {
  const sl_mesh& M = c->mesh;
  TableBufs B;
  try {
    build_ntab(c->nt[c->n], c->n, c->basis, M.dim, M.dim == 2 && c->precision == SL_MIXED, B);
    if (M.dim == 2) build_rules(c->basis, B, c->off_rules, c->f_rules);
  } catch (const std::exception& ex) {
    std::string msg = ex.what();
    delete c;
    return fail(nullptr, SL_EINVAL, "table construction failed: " + msg);
  }
  alias_ntab(c);
  const size_t work_bytes = M.dim != 2 ? 0
                            : c->precision == SL_FP64 ? work2d_doubles(c->nel, c->n) * sizeof(double)
                                                      : work2m_floats(c->nel, c->n) * sizeof(float);
  return alloc_upload(c, B, work_bytes);
}

// p-adaptive meshes and batches: tables of every node count present, node-count buckets, the
// element map on the device.  prob: problem of each element (batches; empty for one problem).
sl_status finish_mapped(sl_ctx* c, const std::vector<uint16_t>& prob = {}) {
  c->mapped = true;
  const int64_t nel = c->nel;
  bool present[NMAX + 1] = {};
  for (uint8_t o : c->ord_host) present[o] = true;
  TableBufs B;
  try {
    for (int n = 2; n <= NMAX; ++n)
      if (present[n]) build_ntab(c->nt[n], n, c->basis, 2, c->precision == SL_MIXED, B);
    build_rules(c->basis, B, c->off_rules, c->f_rules);
  } catch (const std::exception& ex) {
    std::string msg = ex.what();
    delete c;
    return fail(nullptr, SL_EINVAL, "table construction failed: " + msg);
  }
  alias_ntab(c);
  // elements by node count (ascending), each bucket in element order
  std::vector<int> list(nel);
  int64_t pos = 0;
  for (int n = 2; n <= NMAX; ++n) {
    c->bucket_start[n] = pos;
    for (int64_t g = 0; g < nel; ++g)
      if (c->ord_host[g] == n) list[pos++] = (int)g;
    c->bucket_count[n] = pos - c->bucket_start[n];
  }
  const size_t work_bytes = c->precision == SL_FP64
                                ? (size_t)(c->nvals + nel * (4 * NMAX + 8)) * sizeof(double)
                                : (size_t)(c->nvals + nel * (4 * NMAX + WORK2M_FACE + WORK2M_ELEM)) * sizeof(float);
  sl_status st = alloc_upload(c, B, work_bytes);
  if (st != SL_OK) return st;
  const bool batch = !prob.empty();
  if (cudaMalloc(&c->d_off, (nel + 1) * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&c->d_ord, nel * sizeof(uint8_t)) != cudaSuccess ||
      cudaMalloc(&c->d_list, nel * sizeof(int)) != cudaSuccess ||
      (batch && cudaMalloc(&c->d_prob, nel * sizeof(uint16_t)) != cudaSuccess) ||
      (batch && cudaMalloc(&c->d_geo, c->geo_host.size() * sizeof(ProbGeom)) != cudaSuccess)) {
    cudaGetLastError();
    sl_free(c);
    return fail(nullptr, SL_ENOMEM, "device allocation of the element map failed");
  }
  if (cudaMemcpy(c->d_off, c->off_host.data(), (nel + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_ord, c->ord_host.data(), nel * sizeof(uint8_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_list, list.data(), nel * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      (batch && cudaMemcpy(c->d_prob, prob.data(), nel * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess) ||
      (batch && cudaMemcpy(c->d_geo, c->geo_host.data(), c->geo_host.size() * sizeof(ProbGeom),
                           cudaMemcpyHostToDevice) != cudaSuccess)) {
    std::string msg = cudaGetErrorString(cudaGetLastError());
    sl_free(c);
    return fail(nullptr, SL_ECUDA, "element map upload failed: " + msg);
  }
  return SL_OK;
}

}  // namespace

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
  if (mesh->order && mesh->dim != 2) return fail(nullptr, SL_EUNSUPPORTED, "p-adaptive meshes are two-dimensional");
  if (!mesh->order && (n < 2 || n > NMAX)) return fail(nullptr, SL_EINVAL, "n must lie in [2, 17]");
  if ((int64_t)mesh->kx * mesh->ky > (int64_t)1 << 31) return fail(nullptr, SL_EINVAL, "too many elements");
  if (mesh->order)
    for (int64_t g = 0; g < (int64_t)mesh->kx * mesh->ky; ++g)
      if (mesh->order[g] < 2 || mesh->order[g] > NMAX)
        return fail(nullptr, SL_EINVAL, "per-element node counts must lie in [2, 17]");

  sl_ctx* c = new (std::nothrow) sl_ctx();
  if (!c) return fail(nullptr, SL_ENOMEM, "host allocation failed");
  c->mesh = *mesh;
  c->mesh.order = nullptr;
  c->basis = basis;
  c->precision = precision;
  c->stream = (cudaStream_t)cuda_stream;
  const int64_t nel = (int64_t)mesh->kx * mesh->ky;
  c->nel = nel;
  if (mesh->order) {
    c->orders.assign(mesh->order, mesh->order + nel);
    c->ord_host.resize(nel);
    c->off_host.resize(nel + 1);
    int64_t acc = 0;
    int nmax = 2;
    for (int64_t g = 0; g < nel; ++g) {
      const int o = mesh->order[g];
      c->ord_host[g] = (uint8_t)o;
      c->off_host[g] = acc;
      acc += (int64_t)o * o;
      nmax = std::max(nmax, o);
    }
    c->off_host[nel] = acc;
    c->n = nmax;
    c->nvals = acc;
    c->prob_mesh.assign(1, c->mesh);
    sl_status st = finish_mapped(c);
    if (st != SL_OK) return st;
  } else {
    c->n = n;
    c->nvals = nel * (mesh->dim == 1 ? n : n * n);
    sl_status st = finish_uniform(c);
    if (st != SL_OK) return st;
  }
  *out = c;
  return SL_OK;
}

void sl_free(sl_ctx* c) {
  if (!c) return;
  cudaFree(c->d_tables);
  cudaFree(c->d_status);
  cudaFree(c->d_counts);
  cudaFree(c->d_partial);
  cudaFree(c->d_result);
  cudaFree(c->d_io);
  cudaFree(c->d_io64);
  cudaFree(c->d_work);
  cudaFree(c->d_ftab);
  cudaFree(c->d_m2c);
  cudaFree(c->d_off);
  cudaFree(c->d_ord);
  cudaFree(c->d_prob);
  cudaFree(c->d_geo);
  cudaFree(c->d_list);
  cudaFree(c->d_geo_run);
  if (c->run_exec) cudaGraphExecDestroy(c->run_exec);
  if (c->run_ev[0]) cudaEventDestroy(c->run_ev[0]);
  if (c->run_ev[1]) cudaEventDestroy(c->run_ev[1]);
  if (c->run_stream) cudaStreamDestroy(c->run_stream);
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  delete c;
}

sl_status sl_batch_create(int nprob, sl_ctx* const* probs, sl_ctx** out) {
  if (!out) return fail(nullptr, SL_EINVAL, "out is null");
  *out = nullptr;
  if (nprob < 1 || nprob > 65535 || !probs) return fail(nullptr, SL_EINVAL, "need 1..65535 problems");
  for (int p = 0; p < nprob; ++p) {
    const sl_ctx* q = probs[p];
    if (!q) return fail(nullptr, SL_EINVAL, "null problem context");
    if (q->mesh.dim != 2) return fail(nullptr, SL_EUNSUPPORTED, "batches are of 2D problems");
    if (!q->geo_host.empty()) return fail(nullptr, SL_EINVAL, "a batch cannot contain a batch");
    if (q->basis != probs[0]->basis || q->precision != probs[0]->precision)
      return fail(nullptr, SL_EINVAL, "the problems of a batch share basis and precision");
  }
  sl_ctx* c = new (std::nothrow) sl_ctx();
  if (!c) return fail(nullptr, SL_ENOMEM, "host allocation failed");
  c->mesh = probs[0]->mesh;
  c->basis = probs[0]->basis;
  c->precision = probs[0]->precision;
  c->stream = probs[0]->stream;
  c->nprob = nprob;
  std::vector<uint16_t> prob;
  int64_t gb = 0, acc = 0;
  int nmax = 2;
  try {
    for (int p = 0; p < nprob; ++p) {
      const sl_ctx* q = probs[p];
      const sl_mesh& M = q->mesh;
      ProbGeom G{};
      G.kx = M.kx;
      G.ky = M.ky;
      for (int f = 0; f < 4; ++f) G.bc[f] = M.bc[f];
      G.x0 = M.x0;
      G.hx = (M.x1 - M.x0) / M.kx;
      G.y0 = M.y0;
      G.hy = (M.y1 - M.y0) / M.ky;
      G.ghost = M.ghost;
      G.gbase = gb;
      c->geo_host.push_back(G);
      c->prob_mesh.push_back(M);
      for (int64_t g = 0; g < q->nel; ++g) {
        const int o = q->mapped ? q->ord_host[g] : q->n;
        c->ord_host.push_back((uint8_t)o);
        c->off_host.push_back(acc);
        prob.push_back((uint16_t)p);
        acc += (int64_t)o * o;
        nmax = std::max(nmax, o);
      }
      gb += q->nel;
    }
  } catch (const std::exception&) {
    delete c;
    return fail(nullptr, SL_ENOMEM, "host allocation failed");
  }
  if (gb > (int64_t)1 << 31) {
    delete c;
    return fail(nullptr, SL_EINVAL, "too many elements");
  }
  c->off_host.push_back(acc);
  c->nel = gb;
  c->nvals = acc;
  c->n = nmax;
  sl_status st = finish_mapped(c, prob);
  if (st != SL_OK) return st;
  *out = c;
  return SL_OK;
}

int64_t sl_batch_offset(const sl_ctx* c, int p) {
  if (!c || p < 0 || p > c->nprob || c->geo_host.empty()) return -1;
  if (p == c->nprob) return c->nvals;
  return c->off_host[c->geo_host[p].gbase];
}

}  // extern "C"

namespace {

sl_status check_step(sl_ctx* c, const void* phi_in, const void* phi_out, const sl_velocity* vel,
                     const sl_options* opt) {
  if (!phi_in || !phi_out || !opt) return fail(c, SL_EINVAL, "null argument");
  if (phi_in == phi_out) return fail(c, SL_EINVAL, "phi_in and phi_out must be distinct buffers");
  if (((uintptr_t)phi_in | (uintptr_t)phi_out) & 15u)
    return fail(c, SL_EINVAL, "state buffers must be 16-byte aligned");
  if (!valid_velocity(c, vel)) return fail(c, SL_EINVAL, "bad velocity for this mesh");
  if (vel->kind == SL_VEL_NODAL && (c->precision != SL_FP64 || c->mapped || !c->geo_host.empty()))
    return fail(c, SL_EUNSUPPORTED, "a nodal velocity is read by the FP64 paths of one-node-count meshes");
  if (opt->rk_order < 1 || opt->rk_order > 4) return fail(c, SL_EINVAL, "rk_order must be 1..4");
  if (opt->fit != SL_FIT_HARD && opt->fit != SL_FIT_SOFT) return fail(c, SL_EINVAL, "bad fit mode");
  if (opt->bvalue != SL_BV_INTERP && opt->bvalue != SL_BV_BACKTRACK) return fail(c, SL_EINVAL, "bad bvalue");
  if (opt->constraints & ~7u) return fail(c, SL_EINVAL, "unknown constraint bits");
  if (opt->picard_rtol < 0.0 || opt->picard_cap < 0) return fail(c, SL_EINVAL, "bad energy iteration limits");
  return SL_OK;
}

// time and step of one problem: finite, positive, displacement within one element width
sl_status check_dt(sl_ctx* c, const sl_mesh& M, const sl_velocity* vel, double t, double dt) {
  if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t)) return fail(c, SL_EINVAL, "dt must be finite and > 0");
  const double hx = (M.x1 - M.x0) / M.kx, hy = M.dim == 2 ? (M.y1 - M.y0) / M.ky : 1.0;
  double um, vm;
  max_speed(M, vel, um, vm);
  if (um * dt > hx || (M.dim == 2 && vm * dt > hy))
    return fail(c, SL_ECFL, "displacement over the step exceeds one element width");
  return SL_OK;
}

// Event k (0 start, 1 between the phases, 2 end) of the current timed step; steps captured into a
// graph (sl_run) are not timed.
void timing_mark(sl_ctx* c, int k) {
  if (!c->timing || c->capturing) return;
  if (k == 0) {
    if (c->tused + 3 > c->tev.size()) {
      for (int i = 0; i < 3; ++i) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
          cudaGetLastError();
          c->timing = false;
          return;
        }
        c->tev.push_back(e);
      }
    }
    c->tused += 3;
    c->tdone.resize(c->tused / 3);
    c->tdone.back() = 0;
  }
  cudaEventRecord(c->tev[c->tused - 3 + k], c->stream);
  if (k == 2) c->tdone.back() = 1;
}

// the general 2D kernels: phase 1 of every node-count bucket, then phase 2 of every bucket; each
// launch is checked as it is enqueued
sl_status step2d_general(sl_ctx* c, StepParams P, const sl_velocity* vel, double t, double dt, const sl_options* opt,
                         const void* in, void* out) {
  const unsigned lin = opt->constraints & 3u;
  const int soft = opt->fit == SL_FIT_SOFT ? 1 : 0;
  const int64_t nel = c->nel;
  Map2D map{};
  int ts = 4 * c->n;
  if (c->mapped) {
    map.off = c->d_off;
    map.ord = c->d_ord;
    map.prob = c->d_prob;
    map.geo = c->geo_override ? c->geo_override : c->d_geo;
    ts = 4 * NMAX;
  }
  map.tstride = ts;
  const double* T = c->d_tables;
  const float* F = c->d_ftab;
  const sl_mesh& M = c->mesh;
  const double hx = (M.x1 - M.x0) / M.kx, hy = (M.y1 - M.y0) / M.ky;
  for (int phase = 1; phase <= 2; ++phase) {
    if (phase == 2) timing_mark(c, 1);
    for (int n = 2; n <= NMAX; ++n) {
      int64_t count;
      if (c->mapped) {
        count = c->bucket_count[n];
        if (count == 0) continue;
        map.list = c->d_list + c->bucket_start[n];
      } else {
        if (n != c->n) continue;
        count = nel;
        map.list = nullptr;
      }
      const sl_ntab& N = c->nt[n];
      P.m = N.fit[lin][soft].m;
      if (c->precision == SL_FP64) {
        const size_t* off = N.table_off[lin][soft];
        Tables1D tb{T + N.off_xi, T + N.off_w, T + N.off_lam, T + N.off_l0, T + N.off_l1,
                    T + off[0],   T + off[1],  T + off[2],    T + c->off_rules};
        double* W = c->d_work;
        Work2D w{W, W + c->nvals, W + c->nvals + nel * ts};
        launch_step2d_f64(phase, n, P, tb, map, count, (const double*)in, (double*)out, w, c->d_status, c->stream);
        SL_CUDA(c, cudaGetLastError());
      } else {
        Mixed2DExtra X{};
        X.xi = F + N.f_off[0];
        X.lam = F + N.f_off[1];
        X.w = F + N.f_off[2];
        X.l0 = F + N.f_off[3];
        X.l1 = F + N.f_off[4];
        X.w2h = F + N.f_off[5];
        X.w2l = F + N.f_off[6];
        X.Cp = F + N.f_cp[lin];
        X.rules = F + c->f_rules;
        X.counts = c->d_counts;
        X.linref = (opt->constraints & SL_C_ENERGY) ? 0 : 1;
        X.plane = plane_stride(c->nvals);
        X.span = (float)(0.5 / (N.b.xi[n - 1] - N.b.xi[0]));
        X.hx = (float)hx;
        X.hy = (float)hy;
        X.ihx = (float)(1.0 / hx);
        X.ihy = (float)(1.0 / hy);
        X.a = (float)vel->p[0];
        X.b = (float)vel->p[1];
        X.om = (float)vel->p[0];
        X.cx = (float)vel->p[1];
        X.cy = (float)vel->p[2];
        X.dt = (float)dt;
        const double lam = dt / (hx * hy);
        X.dt_area = (float)lam;
        X.lam_hi = (float)lam;
        X.lam_lo = (float)(lam - (double)X.lam_hi);
        if (vel->kind == SL_VEL_SWIRL) {
          X.tT = (float)(t / vel->p[0]);
          X.dtT = (float)(dt / vel->p[0]);
          X.Tper = vel->p[0];
        }
        float* W = (float*)c->d_work;
        Work2M w{W, W + c->nvals, W + c->nvals + nel * ts, W + c->nvals + nel * (ts + WORK2M_FACE)};
        launch_step2d_mixed(phase, n, P, X, map, count, (const float*)in, (float*)out, w, c->d_status, c->stream,
                            c->k2m_per_sm[phase - 1]);
        SL_CUDA(c, cudaGetLastError());
      }
    }
  }
  return SL_OK;
}

// the mixed 2D constant-velocity path (one operator shared by every element)
bool uses_m2c(const sl_ctx* c, const sl_velocity* vel, const sl_options* opt) {
  return c->mesh.dim == 2 && c->precision == SL_MIXED && !c->mapped && vel->kind == SL_VEL_CONST &&
         vel->p[0] != 0.0 && vel->p[1] != 0.0 && opt->fit == SL_FIT_HARD && !(opt->constraints & SL_C_ENERGY) &&
         opt->bvalue == SL_BV_INTERP && (opt->constraints & 3u);
}

// build and upload the shared operator unless the cached one matches (velocity, dt, options)
sl_status ensure_m2c(sl_ctx* c, const sl_velocity* vel, double dt, const sl_options* opt) {
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
  return SL_OK;
}

sl_status step_dispatch(sl_ctx* c, const void* phi_in, void* phi_out, const sl_velocity* vel, double t, double dt,
                        const sl_options* opt) {
  const sl_mesh& M = c->mesh;
  const double hx = (M.x1 - M.x0) / M.kx, hy = M.dim == 2 ? (M.y1 - M.y0) / M.ky : 1.0;
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
  P.gtab = c->inflow_step;
  P.nodal = vel->kind == SL_VEL_NODAL ? vel->nodal : nullptr;
  P.nvals = c->nvals;

  const double* T = c->d_tables;
  const size_t* off = c->table_off[lin][opt->fit == SL_FIT_SOFT];
  timing_mark(c, 0);
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
    if (opt->bvalue != SL_BV_INTERP && c->mapped)
      return fail(c, SL_EUNSUPPORTED, "backtracked interface values need a mesh of one node count");
    const sl_status st = step2d_general(c, P, vel, t, dt, opt, phi_in, phi_out);
    if (st != SL_OK) return st;
  } else if (uses_m2c(c, vel, opt)) {
    // uniform mesh, constant velocity: one operator shared by all elements
    sl_status st = ensure_m2c(c, vel, dt, opt);
    if (st != SL_OK) return st;
    c->m2c.plane = plane_stride(c->nvals);
    launch_step2d_const(c->m2c, c->d_m2c, (const float*)phi_in, (float*)phi_out, c->d_status, c->stream,
                        c->k2c_tile);
  } else if (M.dim == 2 && c->precision == SL_MIXED) {
    if (opt->bvalue != SL_BV_INTERP && c->mapped)
      return fail(c, SL_EUNSUPPORTED, "backtracked interface values need a mesh of one node count");
    if (opt->fit != SL_FIT_HARD) return fail(c, SL_EUNSUPPORTED, "the 2D mixed path uses the hard fit");
    const sl_status st = step2d_general(c, P, vel, t, dt, opt, phi_in, phi_out);
    if (st != SL_OK) return st;
  } else {
    return fail(c, SL_EUNSUPPORTED, "this dimension/precision combination is not built yet");
  }
  if (c->timing && !c->capturing) {
    const bool two_phase = M.dim == 2 && !uses_m2c(c, vel, opt);
    if (!two_phase) timing_mark(c, 1);
    timing_mark(c, 2);
  }
  SL_CUDA(c, cudaGetLastError());
  return SL_OK;
}

// per-problem times and steps of a batch into its device geometry table
sl_status set_batch_steps(sl_ctx* c, const sl_velocity* vel, const double* t, const double* dt) {
  for (int p = 0; p < c->nprob; ++p) {
    sl_status st = check_dt(c, c->prob_mesh[p], vel, t[p], dt[p]);
    if (st != SL_OK) return st;
    c->geo_host[p].t = t[p];
    c->geo_host[p].dt = dt[p];
  }
  SL_CUDA(c, cudaMemcpyAsync(c->d_geo, c->geo_host.data(), c->geo_host.size() * sizeof(ProbGeom),
                             cudaMemcpyHostToDevice, c->stream));
  return SL_OK;
}

}  // namespace

extern "C" {

sl_status sl_step(sl_ctx* c, const void* phi_in, void* phi_out, const sl_velocity* vel, double t, double dt,
                  const sl_options* opt) {
  if (!c) return SL_EINVAL;
  sl_status st = check_step(c, phi_in, phi_out, vel, opt);
  if (st != SL_OK) return st;
  if (!c->geo_host.empty()) {
    std::vector<double> ts(c->nprob, t), dts(c->nprob, dt);
    st = set_batch_steps(c, vel, ts.data(), dts.data());
  } else {
    st = check_dt(c, c->mesh, vel, t, dt);
  }
  if (st != SL_OK) return st;
  c->inflow_step = c->inflow;
  return step_dispatch(c, phi_in, phi_out, vel, t, dt, opt);
}

sl_status sl_set_inflow(sl_ctx* c, const double* values, int64_t step_stride) {
  if (!c) return SL_EINVAL;
  if (step_stride < 0) return fail(c, SL_EINVAL, "step_stride must be >= 0");
  if (c->mesh.dim != 1 || c->precision != SL_FP64 || !c->geo_host.empty())
    return fail(c, SL_EUNSUPPORTED, "inflow records are read by the 1D FP64 path");
  c->inflow = values;
  c->inflow_stride = values ? step_stride : 0;
  return SL_OK;
}

sl_status sl_batch_step(sl_ctx* c, const void* phi_in, void* phi_out, const sl_velocity* vel, const double* t,
                        const double* dt, const sl_options* opt) {
  if (!c) return SL_EINVAL;
  if (c->geo_host.empty()) return fail(c, SL_EINVAL, "not a batch context");
  if (!t || !dt) return fail(c, SL_EINVAL, "null argument");
  sl_status st = check_step(c, phi_in, phi_out, vel, opt);
  if (st != SL_OK) return st;
  st = set_batch_steps(c, vel, t, dt);
  if (st != SL_OK) return st;
  return step_dispatch(c, phi_in, phi_out, vel, t[0], dt[0], opt);
}

sl_status sl_run(sl_ctx* c, void* phi_a, void* phi_b, const sl_velocity* vel, double t0, double dt, int nsteps,
                 const sl_options* opt) {
  if (!c) return SL_EINVAL;
  if (nsteps < 0) return fail(c, SL_EINVAL, "nsteps must be >= 0");
  sl_status st = check_step(c, phi_a, phi_b, vel, opt);
  if (st != SL_OK) return st;
  if (nsteps == 0) return SL_OK;
  const bool batch = !c->geo_host.empty();
  if (batch) {
    for (int p = 0; p < c->nprob; ++p)
      if ((st = check_dt(c, c->prob_mesh[p], vel, t0, dt)) != SL_OK) return st;
  } else if ((st = check_dt(c, c->mesh, vel, t0, dt)) != SL_OK) {
    return st;
  }
  if (!std::isfinite(t0 + nsteps * dt)) return fail(c, SL_EINVAL, "t0 + nsteps dt must be finite");
  if (c->inflow && nsteps > 1 && c->inflow_stride < SL_INFLOW_RECORD)
    return fail(c, SL_EINVAL, "inflow records of a run need step_stride >= SL_INFLOW_RECORD");
  // operators that a step would upload are prepared before (and outside) the capture
  if (uses_m2c(c, vel, opt) && (st = ensure_m2c(c, vel, dt, opt)) != SL_OK) return st;
  if (!c->run_stream) {
    if (cudaStreamCreateWithFlags(&c->run_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->run_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->run_ev[1], cudaEventDisableTiming) != cudaSuccess)
      return fail(c, SL_ECUDA, std::string("run stream: ") + cudaGetErrorString(cudaGetLastError()));
  }
  std::vector<double> key = {(double)c->k2c_tile, (double)c->k2m_per_sm[0], (double)c->k2m_per_sm[1],
                             (double)vel->kind, t0, dt, (double)nsteps, (double)opt->constraints,
                             (double)opt->rk_order, (double)opt->fit, (double)opt->bvalue, opt->picard_rtol,
                             (double)opt->picard_cap, (double)(uintptr_t)phi_a, (double)(uintptr_t)phi_b,
                             (double)(uintptr_t)c->inflow, (double)c->inflow_stride,
                             (double)(uintptr_t)vel->nodal, (double)vel->nodal_step};
  for (int i = 0; i < 6; ++i) key.push_back(vel->p[i]);
  if (!c->run_valid || key != c->run_key) {
    if (c->run_exec) cudaGraphExecDestroy(c->run_exec);
    c->run_exec = nullptr;
    c->run_valid = false;
    if (batch) {                             // every step's times and steps, uploaded once
      const size_t need = (size_t)nsteps * c->nprob;
      if (need > c->geo_run_cap) {
        cudaFree(c->d_geo_run);
        c->d_geo_run = nullptr;
        c->geo_run_cap = 0;
        if (cudaMalloc(&c->d_geo_run, need * sizeof(ProbGeom)) != cudaSuccess) {
          cudaGetLastError();
          return fail(c, SL_ENOMEM, "device allocation of the run geometry failed");
        }
        c->geo_run_cap = need;
      }
      std::vector<ProbGeom> g(need);
      for (int s = 0; s < nsteps; ++s)
        for (int p = 0; p < c->nprob; ++p) {
          g[(size_t)s * c->nprob + p] = c->geo_host[p];
          g[(size_t)s * c->nprob + p].t = t0 + s * dt;
          g[(size_t)s * c->nprob + p].dt = dt;
        }
      SL_CUDA(c, cudaMemcpy(c->d_geo_run, g.data(), need * sizeof(ProbGeom), cudaMemcpyHostToDevice));
    }
    const cudaStream_t user = c->stream;
    c->stream = c->run_stream;
    c->capturing = true;
    const cudaError_t cb = cudaStreamBeginCapture(c->run_stream, cudaStreamCaptureModeThreadLocal);
    if (cb != cudaSuccess) {
      c->stream = user;
      c->capturing = false;
      return fail(c, SL_ECUDA, std::string("capture: ") + cudaGetErrorString(cb));
    }
    void* a = phi_a;
    void* b = phi_b;
    for (int s = 0; s < nsteps && st == SL_OK; ++s) {
      if (batch) c->geo_override = c->d_geo_run + (size_t)s * c->nprob;
      c->inflow_step = c->inflow ? c->inflow + (int64_t)s * c->inflow_stride : nullptr;
      sl_velocity vs = *vel;                 // a nodal field advances by nodal_step per step
      if (vs.kind == SL_VEL_NODAL) vs.nodal += (int64_t)s * vs.nodal_step;
      st = step_dispatch(c, a, b, &vs, t0 + s * dt, dt, opt);
      std::swap(a, b);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->run_stream, &graph);
    c->stream = user;
    c->capturing = false;
    c->geo_override = nullptr;
    if (st == SL_OK && ce != cudaSuccess) st = fail(c, SL_ECUDA, std::string("capture: ") + cudaGetErrorString(ce));
    if (st == SL_OK && cudaGraphInstantiate(&c->run_exec, graph, 0) != cudaSuccess) {
      c->run_exec = nullptr;
      st = fail(c, SL_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(cudaGetLastError()));
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != SL_OK) return st;
    c->run_key = key;
    c->run_valid = true;
  }
  // the graph runs after the work already on the context's stream, and the stream waits for it
  SL_CUDA(c, cudaEventRecord(c->run_ev[0], c->stream));
  SL_CUDA(c, cudaStreamWaitEvent(c->run_stream, c->run_ev[0], 0));
  SL_CUDA(c, cudaGraphLaunch(c->run_exec, c->run_stream));
  SL_CUDA(c, cudaEventRecord(c->run_ev[1], c->run_stream));
  SL_CUDA(c, cudaStreamWaitEvent(c->stream, c->run_ev[1], 0));
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
  if (c->inflow && nsteps > 1 && c->inflow_stride < SL_INFLOW_RECORD)
    return fail(c, SL_EINVAL, "inflow records of a run need step_stride >= SL_INFLOW_RECORD");
  const double* inflow0 = c->inflow;        // step s reads record s
  for (int s = 0; s < nsteps; ++s) {
    c->inflow = inflow0 ? inflow0 + (int64_t)s * c->inflow_stride : nullptr;
    sl_velocity vs = *vel;                   // a nodal field advances by nodal_step per step
    if (vs.kind == SL_VEL_NODAL) vs.nodal += (int64_t)s * vs.nodal_step;
    sl_status st = sl_step(c, a, b, &vs, t0 + s * dt, dt, opt);
    c->inflow = inflow0;
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
  if (c->mapped)
    launch_mass_energy_csr(c->nel, c->d_off, c->d_ord, c->d_prob, c->d_geo, hx * hy, c->precision,
                           plane_stride(c->nvals), phi, c->d_tables + c->off_rules, power, c->d_partial, c->d_result,
                           c->red_blocks, c->stream);
  else if (c->precision == SL_FP64)
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

sl_status sl_timing(sl_ctx* c, int enable) {
  if (!c) return SL_EINVAL;
  SL_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!enable) {
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    c->tev.clear();
  }
  c->tused = 0;
  c->tdone.clear();
  c->timing = enable != 0;
  return SL_OK;
}

sl_status sl_timing_read(sl_ctx* c, double* ms, int* nsteps) {
  if (!c) return SL_EINVAL;
  if (!ms || !nsteps) return fail(c, SL_EINVAL, "null argument");
  SL_CUDA(c, cudaStreamSynchronize(c->stream));
  double a = 0.0, b = 0.0;
  int done = 0;
  for (size_t k = 0; k + 3 <= c->tused; k += 3) {
    float t01 = 0.0f, t12 = 0.0f;
    // a step that failed after its start event has no end event: it is not counted
    if (!c->tdone[k / 3] || cudaEventElapsedTime(&t01, c->tev[k], c->tev[k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t12, c->tev[k + 1], c->tev[k + 2]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    a += t01;
    b += t12;
    ++done;
  }
  ms[0] = a;
  ms[1] = b;
  ms[2] = a + b;
  *nsteps = done;
  return SL_OK;
}

sl_status sl_counters(sl_ctx* c, uint64_t* counts) {
  if (!c) return SL_EINVAL;
  if (!counts) return fail(c, SL_EINVAL, "null argument");
  unsigned long long h[SL_NCOUNTERS] = {};
  SL_CUDA(c, cudaStreamSynchronize(c->stream));
  SL_CUDA(c, cudaMemcpy(h, c->d_counts, sizeof(h), cudaMemcpyDeviceToHost));
  SL_CUDA(c, cudaMemset(c->d_counts, 0, sizeof(h)));
  for (int k = 0; k < SL_NCOUNTERS; ++k) counts[k] = (uint64_t)h[k];
  return SL_OK;
}

sl_status sl_max_dt(const sl_ctx* c, const sl_velocity* vel, int rule, double* dt) {
  if (!c || !dt) return SL_EINVAL;
  if (!valid_velocity(c, vel)) return fail(const_cast<sl_ctx*>(c), SL_EINVAL, "bad velocity");
  if (rule != SL_RULE_HALF_MIN_SPACING && rule != SL_RULE_PAPER && rule != SL_RULE_HALF_PAPER)
    return fail(const_cast<sl_ctx*>(c), SL_EINVAL, "bad rule");
  const bool edge = rule != SL_RULE_HALF_MIN_SPACING;
  // smallest gap over the node counts in use: edge node to face (paper) or between nodes
  double gap = 1.0;
  for (int n = 2; n <= NMAX; ++n) {
    if (!c->nt[n].present) continue;
    const std::vector<double>& xi = c->nt[n].b.xi;
    if (edge) gap = std::min(gap, xi[0]);
    else
      for (size_t i = 1; i < xi.size(); ++i) gap = std::min(gap, xi[i] - xi[i - 1]);
  }
  const double factor = rule == SL_RULE_PAPER ? 1.0 : 0.5;     // half-spacing and half-paper: 0.5
  double lim = INFINITY;
  const std::vector<sl_mesh> one(1, c->mesh);
  for (const sl_mesh& M : c->prob_mesh.empty() ? one : c->prob_mesh) {
    double um, vm;
    max_speed(M, vel, um, vm);
    if (um > 0) lim = std::min(lim, (M.x1 - M.x0) / M.kx * gap / um);
    if (M.dim == 2 && vm > 0) lim = std::min(lim, (M.y1 - M.y0) / M.ky * gap / vm);
  }
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
  if (M.dim == 1) {
    const double hx = (M.x1 - M.x0) / M.kx;
    for (int k = 0; k < M.kx; ++k)
      for (int i = 0; i < n; ++i) x[(int64_t)k * n + i] = M.x0 + (k + c->b.xi[i]) * hx;
    return SL_OK;
  }
  const std::vector<sl_mesh> one(1, c->mesh);
  const std::vector<sl_mesh>& meshes = c->prob_mesh.empty() ? one : c->prob_mesh;
  int64_t g = 0;
  for (const sl_mesh& P : meshes) {
    const double hx = (P.x1 - P.x0) / P.kx, hy = (P.y1 - P.y0) / P.ky;
    for (int ey = 0; ey < P.ky; ++ey)
      for (int ex = 0; ex < P.kx; ++ex, ++g) {
        const int m = c->mapped ? c->ord_host[g] : n;
        const std::vector<double>& xi = c->nt[m].b.xi;
        const int64_t o0 = c->mapped ? c->off_host[g] : g * n * n;
        for (int j = 0; j < m; ++j)
          for (int i = 0; i < m; ++i) {
            x[o0 + j * m + i] = P.x0 + (ex + xi[i]) * hx;
            y[o0 + j * m + i] = P.y0 + (ey + xi[j]) * hy;
          }
      }
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

// ------------------------------------------------------------------------------ autotuner

namespace {

std::mutex g_tune_mu;                        // one cache read-modify-write at a time in this process

}  // namespace

sl_status sl_tune(sl_ctx* c, const void* phi_in, void* phi_out, const sl_velocity* vel, double t, double dt,
                  const sl_options* opt, const char* cache_path, int* choice) {
  if (!c) return SL_EINVAL;
  sl_status st = check_step(c, phi_in, phi_out, vel, opt);
  if (st != SL_OK) return st;
  if (!c->geo_host.empty()) return fail(c, SL_EUNSUPPORTED, "sl_tune takes a single problem's context");
  if ((st = check_dt(c, c->mesh, vel, t, dt)) != SL_OK) return st;
  const sl_mesh& M = c->mesh;
  const bool shared = uses_m2c(c, vel, opt);
  const bool general = M.dim == 2 && c->precision == SL_MIXED && !shared;
  auto report = [&](bool cached) {
    if (choice) {
      choice[0] = c->k2c_tile;
      choice[1] = c->k2m_per_sm[0];
      choice[2] = c->k2m_per_sm[1];
      choice[3] = cached ? 1 : 0;
    }
  };
  if (!shared && !general) {
    report(false);
    return SL_OK;
  }
  int dev = 0;
  cudaDeviceProp prop{};
  SL_CUDA(c, cudaGetDevice(&dev));
  SL_CUDA(c, cudaGetDeviceProperties(&prop, dev));
  std::string devname(prop.name);
  for (char& ch : devname)
    if (ch == '"' || ch == '\\') ch = '_';
  char kbuf[512];
  std::snprintf(kbuf, sizeof kbuf, "%s|dev=%s|n=%d|kx=%d|ky=%d|nel=%lld|mapped=%d|cons=%u|fit=%d|bv=%d|rk=%d|vel=%d",
                shared ? "k2c_tile" : "k2m_per_sm", devname.c_str(), c->n, M.kx, M.ky, (long long)c->nel,
                c->mapped ? 1 : 0, opt->constraints, opt->fit, opt->bvalue, opt->rk_order, vel->kind);
  const std::string key(kbuf);
  std::map<std::string, std::string> cache;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (cache_path) {
    if (!read_tune_cache(cache_path, cache)) return fail(c, SL_EINVAL, "sl_tune: the cache file is not a flat JSON object");
    auto it = cache.find(key);
    if (it != cache.end()) {
      int a = 0, b = 0;
      if (shared && std::sscanf(it->second.c_str(), "tile=%d", &a) == 1 && a >= 0 && a < k2c_tile_count(c->n)) {
        c->k2c_tile = a;
        report(true);
        return SL_OK;
      }
      if (general && std::sscanf(it->second.c_str(), "p1=%d,p2=%d", &a, &b) == 2 && a >= 0 && b >= 0) {
        c->k2m_per_sm[0] = a;
        c->k2m_per_sm[1] = b;
        report(true);
        return SL_OK;
      }
    }
  }
  // candidates: tile indices, or (phase 1, phase 2) CTAs per SM from {occupancy limit, 1, 2}
  std::vector<std::pair<int, int>> cands;
  if (shared) {
    for (int k = 0; k < k2c_tile_count(c->n); ++k) cands.emplace_back(k, 0);
  } else {
    for (int a : {0, 1, 2})
      for (int b : {0, 1, 2}) cands.emplace_back(a, b);
  }
  const int tile0 = c->k2c_tile, p10 = c->k2m_per_sm[0], p20 = c->k2m_per_sm[1];
  auto apply = [&](const std::pair<int, int>& cd) {
    if (shared) c->k2c_tile = cd.first;
    else {
      c->k2m_per_sm[0] = cd.first;
      c->k2m_per_sm[1] = cd.second;
    }
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(c, SL_ECUDA, std::string("sl_tune: events: ") + cudaGetErrorString(cudaGetLastError()));
  }
  float best = INFINITY;
  std::pair<int, int> pick = cands[0];
  for (const auto& cd : cands) {
    apply(cd);
    if ((st = sl_step(c, phi_in, phi_out, vel, t, dt, opt)) != SL_OK) break;
    if (cudaEventRecord(e0, c->stream) != cudaSuccess) { st = SL_ECUDA; break; }
    for (int r = 0; r < 3 && st == SL_OK; ++r) st = sl_step(c, phi_in, phi_out, vel, t, dt, opt);
    if (st != SL_OK) break;
    float ms = 0.0f;
    if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = SL_ECUDA;
      break;
    }
    if (ms < best) {
      best = ms;
      pick = cd;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SL_OK) {
    c->k2c_tile = tile0;
    c->k2m_per_sm[0] = p10;
    c->k2m_per_sm[1] = p20;
    if (st == SL_ECUDA) return fail(c, SL_ECUDA, std::string("sl_tune: ") + cudaGetErrorString(cudaGetLastError()));
    return st;
  }
  apply(pick);
  report(false);
  if (cache_path) {
    char vbuf[64];
    if (shared) std::snprintf(vbuf, sizeof vbuf, "tile=%d", pick.first);
    else std::snprintf(vbuf, sizeof vbuf, "p1=%d,p2=%d", pick.first, pick.second);
    cache[key] = vbuf;
    if (!write_tune_cache(cache_path, cache)) return fail(c, SL_EINVAL, "sl_tune: cannot write the cache file");
  }
  return SL_OK;
}
