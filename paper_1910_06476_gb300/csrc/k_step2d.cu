// Dispatch of the 2D FP64 step kernels on the node count.
#include "k_map2d.cuh"   // declarations only: the kernels are instantiated in k_step2d_{a..d}.cu

namespace sl {
namespace k2d {
template <int NN>
void launch_n(int phase, const StepParams& p, const Tables1D& tb, const Map2D& m, int64_t count, const double* in,
              double* out, const Work2D& w, unsigned* st, cudaStream_t s);
}

void launch_step2d_f64(int phase, int n, const StepParams& p, const Tables1D& tb, const Map2D& m, int64_t count,
                       const double* in, double* out, const Work2D& w, unsigned* status, cudaStream_t s) {
  switch (n) {
    case 2: k2d::launch_n<2>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 3: k2d::launch_n<3>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 4: k2d::launch_n<4>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 5: k2d::launch_n<5>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 6: k2d::launch_n<6>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 7: k2d::launch_n<7>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 8: k2d::launch_n<8>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 9: k2d::launch_n<9>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 10: k2d::launch_n<10>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 11: k2d::launch_n<11>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 12: k2d::launch_n<12>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 13: k2d::launch_n<13>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 14: k2d::launch_n<14>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 15: k2d::launch_n<15>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 16: k2d::launch_n<16>(phase, p, tb, m, count, in, out, w, status, s); break;
    case 17: k2d::launch_n<17>(phase, p, tb, m, count, in, out, w, status, s); break;
    default: break;
  }
}

}  // namespace sl
