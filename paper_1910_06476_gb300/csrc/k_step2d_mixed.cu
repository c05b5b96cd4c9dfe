// Dispatch of the 2D mixed-precision step kernels on the node count.
#include "k_step2d_mixed_impl.cuh"

namespace sl {
namespace k2m {
template <int NN>
void launch_n(const StepParams& p, const Mixed2DExtra& x, const float* in, float* out, Work2M w, unsigned* st,
              cudaStream_t s);
}

void launch_step2d_mixed(int n, const StepParams& p, const Mixed2DExtra& x, const float* in, float* out, float* work,
                         unsigned* status, cudaStream_t s) {
  const int64_t nel = (int64_t)p.kx * p.ky;
  k2m::Work2M w{work, work + nel * n * n, work + nel * (n * n + 4 * n), work + nel * (n * n + 4 * n + 16)};
  switch (n) {
    case 2: k2m::launch_n<2>(p, x, in, out, w, status, s); break;
    case 3: k2m::launch_n<3>(p, x, in, out, w, status, s); break;
    case 4: k2m::launch_n<4>(p, x, in, out, w, status, s); break;
    case 5: k2m::launch_n<5>(p, x, in, out, w, status, s); break;
    case 6: k2m::launch_n<6>(p, x, in, out, w, status, s); break;
    case 7: k2m::launch_n<7>(p, x, in, out, w, status, s); break;
    case 8: k2m::launch_n<8>(p, x, in, out, w, status, s); break;
    case 9: k2m::launch_n<9>(p, x, in, out, w, status, s); break;
    case 10: k2m::launch_n<10>(p, x, in, out, w, status, s); break;
    case 11: k2m::launch_n<11>(p, x, in, out, w, status, s); break;
    case 12: k2m::launch_n<12>(p, x, in, out, w, status, s); break;
    case 13: k2m::launch_n<13>(p, x, in, out, w, status, s); break;
    case 14: k2m::launch_n<14>(p, x, in, out, w, status, s); break;
    case 15: k2m::launch_n<15>(p, x, in, out, w, status, s); break;
    case 16: k2m::launch_n<16>(p, x, in, out, w, status, s); break;
    case 17: k2m::launch_n<17>(p, x, in, out, w, status, s); break;
    default: break;
  }
}

}  // namespace sl
