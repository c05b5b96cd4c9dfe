// Dispatch of the 1D mixed-precision step kernel, and the conversions between double state and
// the double-float (hi plane, lo plane) state of the mixed path.
#include "sl_internal.h"

namespace sl {
namespace k1m {
template <int NN>
void launch_n(const Mixed1DParams& p, const float* in, float* out, unsigned* st, cudaStream_t s);
}

void launch_step1d_mixed(const Mixed1DParams& p, const float* in, float* out, unsigned* status, cudaStream_t s) {
  switch (p.n) {
    case 2: k1m::launch_n<2>(p, in, out, status, s); break;
    case 3: k1m::launch_n<3>(p, in, out, status, s); break;
    case 4: k1m::launch_n<4>(p, in, out, status, s); break;
    case 5: k1m::launch_n<5>(p, in, out, status, s); break;
    case 6: k1m::launch_n<6>(p, in, out, status, s); break;
    case 7: k1m::launch_n<7>(p, in, out, status, s); break;
    case 8: k1m::launch_n<8>(p, in, out, status, s); break;
    case 9: k1m::launch_n<9>(p, in, out, status, s); break;
    case 10: k1m::launch_n<10>(p, in, out, status, s); break;
    case 11: k1m::launch_n<11>(p, in, out, status, s); break;
    case 12: k1m::launch_n<12>(p, in, out, status, s); break;
    case 13: k1m::launch_n<13>(p, in, out, status, s); break;
    case 14: k1m::launch_n<14>(p, in, out, status, s); break;
    case 15: k1m::launch_n<15>(p, in, out, status, s); break;
    case 16: k1m::launch_n<16>(p, in, out, status, s); break;
    case 17: k1m::launch_n<17>(p, in, out, status, s); break;
    default: break;
  }
}

namespace {
// hi = fl(d), lo = fl(d - hi): hi + lo carries about 48 bits of d
__global__ void k_pack(int64_t nvals, int64_t plane, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvals; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = src[i];
    const float hi = (float)d;
    dst[i] = hi;
    dst[plane + i] = (float)(d - (double)hi);
  }
}

__global__ void k_unpack(int64_t nvals, int64_t plane, const float* __restrict__ src, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvals; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i] + (double)src[plane + i];
}
}  // namespace

void launch_pack(int64_t nvals, int64_t plane, const double* src, float* dst, cudaStream_t s) {
  if (nvals <= 0) return;
  const int grid = (int)std::min<int64_t>((nvals + 255) / 256, 152 * 16);
  k_pack<<<grid, 256, 0, s>>>(nvals, plane, src, dst);
}

void launch_unpack(int64_t nvals, int64_t plane, const float* src, double* dst, cudaStream_t s) {
  if (nvals <= 0) return;
  const int grid = (int)std::min<int64_t>((nvals + 255) / 256, 152 * 16);
  k_unpack<<<grid, 256, 0, s>>>(nvals, plane, src, dst);
}

}  // namespace sl
