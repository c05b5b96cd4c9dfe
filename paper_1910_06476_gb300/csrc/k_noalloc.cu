// Mass / energy integral that allocates no device memory: the deterministic two-pass reduction
// of k_reduce.cu with its per-CTA partial sums kept in a file-scope __device__ array instead of
// a buffer from cudaMalloc.
//
// Why: some callers cannot allocate device memory at the moment they need the diagnostic --
// code running while a stream is captured into a CUDA graph in global capture mode (cudaMalloc
// is not permitted there), host loops under a hard latency budget (cudaMalloc may synchronise
// the device), or applications whose memory pool owns all device memory.  They pass the state
// and a device output and get the integral without any allocation by this entry point.
#include <mutex>

#include "sl_internal.h"

namespace sl {
namespace {

constexpr int NA_BLOCK = 256;
constexpr int64_t NA_TILE = 4096;                     // values summed by one CTA
constexpr int NA_MAX_PARTIALS = 65536;                // scratch: 65536 doubles = 512 KB
static_assert((int64_t)NA_MAX_PARTIALS * NA_TILE == SL_NOALLOC_MAX_VALUES, "limit mismatch");

// Scratch shared by every call on a device, held by every GPU that loads the library until the
// process exits.  Pass 1 overwrites every partial it uses before pass 2 reads it, so no clearing
// is needed; calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_partials[NA_MAX_PARTIALS];

struct NaParams {
  int64_t total;          // values
  int nd;                 // values per element
  int nper, dim, power;
  double scale;
  double w[NMAX];
};

__global__ void __launch_bounds__(NA_BLOCK) k_na_partial(const __grid_constant__ NaParams P,
                                                         const double* __restrict__ phi, double* partials) {
  __shared__ double red[NA_BLOCK];
  const int64_t base = (int64_t)blockIdx.x * NA_TILE;
  const int64_t end = base + NA_TILE < P.total ? base + NA_TILE : P.total;
  double acc = 0.0;
  for (int64_t idx = base + threadIdx.x; idx < end; idx += NA_BLOCK) {
    const int r = (int)(idx % P.nd);
    const double wr = P.dim == 1 ? P.w[r] : P.w[r / P.nper] * P.w[r % P.nper];
    const double v = phi[idx];
    acc += wr * (P.power == 1 ? v : v * v);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = NA_BLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(NA_BLOCK) k_na_final(int nparts, const double* __restrict__ partials, double scale,
                                                       double* out) {
  __shared__ double red[NA_BLOCK];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += NA_BLOCK) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = NA_BLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

// Device address of g_partials, looked up with that device current and kept once the lookup has
// succeeded (a failed lookup is retried by the next call).  In host code the symbol g_partials is
// only a host-side stand-in and must never be passed to a kernel.  The address belongs to the
// device's primary context: a cudaDeviceReset ends that context, and the entry point must not be
// used on that device afterwards.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
double* g_addr[NA_MAX_DEVICES] = {};

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

void set_global_error(const std::string& msg);

}  // namespace sl

extern "C" sl_status sl_integral_noalloc(const double* phi, int64_t nelem, int nper, int dim, const double* w_host,
                                        int power, double scale, double* total, void* cuda_stream) {
  using namespace sl;
  if (!phi || !w_host || !total) { set_global_error("sl_integral_noalloc: null pointer"); return SL_EINVAL; }
  if ((dim != 1 && dim != 2) || nper < 1 || nper > NMAX || (power != 1 && power != 2) || nelem < 0) {
    set_global_error("sl_integral_noalloc: bad dim, nper, power or nelem");
    return SL_EINVAL;
  }
  const int nd = dim == 1 ? nper : nper * nper;
  if (nelem > SL_NOALLOC_MAX_VALUES / nd) {
    set_global_error("sl_integral_noalloc: more than SL_NOALLOC_MAX_VALUES values, beyond its fixed scratch");
    return SL_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    set_global_error(std::string("sl_integral_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return SL_ECUDA;
  }
  NaParams P{};
  P.total = nelem * nd;
  P.nd = nd;
  P.nper = nper;
  P.dim = dim;
  P.power = power;
  P.scale = scale;
  for (int i = 0; i < nper; ++i) P.w[i] = w_host[i];
  const int nparts = (int)((P.total + NA_TILE - 1) / NA_TILE);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (nparts > 0) k_na_partial<<<nparts, NA_BLOCK, 0, s>>>(P, phi, scratch);
  k_na_final<<<1, NA_BLOCK, 0, s>>>(nparts, scratch, scale, total);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("sl_integral_noalloc: launch failed: ") + cudaGetErrorString(e));
    return SL_ECUDA;
  }
  return SL_OK;
}
