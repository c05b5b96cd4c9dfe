// Dispatch of the 2D FP64 step kernels on the node count.
#include "k_step2d_impl.cuh"

namespace sl {
namespace k2d {
template <int NN>
void launch_n(const StepParams& p, const Tables1D& tb, const double* in, double* out, Work2D w, unsigned* st,
              cudaStream_t s);
}

void launch_step2d_f64(int n, const StepParams& p, const Tables1D& tb, const double* in, double* out, double* work,
                       unsigned* status, cudaStream_t s) {
  const int64_t nel = (int64_t)p.kx * p.ky;
  k2d::Work2D w{work, work + nel * n * n, work + nel * (n * n + 4 * n)};
  switch (n) {
    case 2: k2d::launch_n<2>(p, tb, in, out, w, status, s); break;
    case 3: k2d::launch_n<3>(p, tb, in, out, w, status, s); break;
    case 4: k2d::launch_n<4>(p, tb, in, out, w, status, s); break;
    case 5: k2d::launch_n<5>(p, tb, in, out, w, status, s); break;
    case 6: k2d::launch_n<6>(p, tb, in, out, w, status, s); break;
    case 7: k2d::launch_n<7>(p, tb, in, out, w, status, s); break;
    case 8: k2d::launch_n<8>(p, tb, in, out, w, status, s); break;
    case 9: k2d::launch_n<9>(p, tb, in, out, w, status, s); break;
    case 10: k2d::launch_n<10>(p, tb, in, out, w, status, s); break;
    case 11: k2d::launch_n<11>(p, tb, in, out, w, status, s); break;
    case 12: k2d::launch_n<12>(p, tb, in, out, w, status, s); break;
    case 13: k2d::launch_n<13>(p, tb, in, out, w, status, s); break;
    case 14: k2d::launch_n<14>(p, tb, in, out, w, status, s); break;
    case 15: k2d::launch_n<15>(p, tb, in, out, w, status, s); break;
    case 16: k2d::launch_n<16>(p, tb, in, out, w, status, s); break;
    case 17: k2d::launch_n<17>(p, tb, in, out, w, status, s); break;
    default: break;
  }
}

}  // namespace sl
