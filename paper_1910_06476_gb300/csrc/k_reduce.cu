// Global mass and energy (eq. quad summed over elements; the diagnostics of Sec. 5) with a
// deterministic two-pass reduction in double: a fixed grid of CTAs each sums a fixed strided
// subset of the elements, then one CTA sums the per-CTA partials in index order.
#include "sl_internal.h"

namespace sl {
namespace {

constexpr int RBLOCK = 256;

// PAIR = true reads the double-float state (hi plane, then lo plane) of the mixed path
template <typename T, bool PAIR>
__global__ void __launch_bounds__(RBLOCK) k_partial(int64_t nelem, int nper, int64_t plane, int dim,
                                                   const T* __restrict__ phi, const double* __restrict__ w, int power,
                                                   double* partial) {
  __shared__ double red[RBLOCK];
  __shared__ double ws[NMAX * NMAX];
  const int nd = dim == 1 ? nper : nper * nper;
  for (int i = threadIdx.x; i < nd; i += RBLOCK)
    ws[i] = dim == 1 ? w[i] : w[i / nper] * w[i % nper];
  __syncthreads();
  double acc = 0.0;
  const int64_t total = nelem * nd;
  for (int64_t idx = (int64_t)blockIdx.x * RBLOCK + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * RBLOCK) {
    const double v = PAIR ? (double)phi[idx] + (double)phi[idx + plane] : (double)phi[idx];
    acc += ws[idx % nd] * (power == 1 ? v : v * v);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RBLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(RBLOCK) k_final(int nparts, const double* __restrict__ partial, double scale,
                                                 double* result) {
  __shared__ double red[RBLOCK];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += RBLOCK) acc += partial[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RBLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *result = red[0] * scale;
}

}  // namespace

void launch_mass_energy_f64(int64_t nelem, int nper, const double* phi, const double* w, int dim, int power,
                            double scale, double* partial, double* result, int nblocks, cudaStream_t s) {
  k_partial<double, false><<<nblocks, RBLOCK, 0, s>>>(nelem, nper, 0, dim, phi, w, power, partial);
  k_final<<<1, RBLOCK, 0, s>>>(nblocks, partial, scale, result);
}

void launch_mass_energy_pair(int64_t nelem, int nper, int64_t plane, const float* phi, const double* w, int dim,
                             int power, double scale, double* partial, double* result, int nblocks, cudaStream_t s) {
  k_partial<float, true><<<nblocks, RBLOCK, 0, s>>>(nelem, nper, plane, dim, phi, w, power, partial);
  k_final<<<1, RBLOCK, 0, s>>>(nblocks, partial, scale, result);
}

}  // namespace sl

namespace sl {
namespace {

// p-adaptive meshes and batches: element g has ord[g] nodes per direction starting at off[g];
// its area is its problem's hx hy (geo) or the single area given
template <typename T, bool PAIR>
__global__ void __launch_bounds__(RBLOCK) k_partial_csr(int64_t nel, const int64_t* __restrict__ off,
                                                       const uint8_t* __restrict__ ord,
                                                       const uint16_t* __restrict__ prob,
                                                       const ProbGeom* __restrict__ geo, double area, int64_t plane,
                                                       const T* __restrict__ phi, const double* __restrict__ rules,
                                                       int power, double* partial) {
  __shared__ double red[RBLOCK];
  double acc = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * RBLOCK + threadIdx.x; g < nel; g += (int64_t)gridDim.x * RBLOCK) {
    const int n = ord[g];
    const double* w = rules + (size_t)n * 3 * NMAX + 2 * NMAX;
    const double a = geo ? geo[prob[g]].hx * geo[prob[g]].hy : area;
    const int64_t b = off[g];
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      double r = 0.0;
      for (int i = 0; i < n; ++i) {
        const int64_t idx = b + j * n + i;
        const double v = PAIR ? (double)phi[idx] + (double)phi[idx + plane] : (double)phi[idx];
        r += w[i] * (power == 1 ? v : v * v);
      }
      s += w[j] * r;
    }
    acc += a * s;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RBLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace

void launch_mass_energy_csr(int64_t nel, const int64_t* off, const uint8_t* ord, const uint16_t* prob,
                            const ProbGeom* geo, double area, int precision, int64_t plane, const void* phi,
                            const double* rules, int power, double* partial, double* result, int nblocks,
                            cudaStream_t s) {
  if (precision == SL_FP64)
    k_partial_csr<double, false><<<nblocks, RBLOCK, 0, s>>>(nel, off, ord, prob, geo, area, 0, (const double*)phi,
                                                            rules, power, partial);
  else
    k_partial_csr<float, true><<<nblocks, RBLOCK, 0, s>>>(nel, off, ord, prob, geo, area, plane, (const float*)phi,
                                                          rules, power, partial);
  k_final<<<1, RBLOCK, 0, s>>>(nblocks, partial, 1.0, result);
}

}  // namespace sl
