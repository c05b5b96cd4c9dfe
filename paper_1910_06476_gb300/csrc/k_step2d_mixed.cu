// Dispatch of the 2D mixed-precision step kernels on the node count.
#include "k_map2d.cuh"   // declarations only: the kernels are instantiated in k_step2d_mixed_{a..c}.cu

namespace sl {
namespace k2m {
template <int NN>
void launch_n(int phase, const StepParams& p, const Mixed2DExtra& x, const Map2D& m, int64_t count, const float* in,
              float* out, const Work2M& w, unsigned* st, cudaStream_t s, int fill);
}

void launch_step2d_mixed(int phase, int n, const StepParams& p, const Mixed2DExtra& x, const Map2D& m,
                         int64_t count, const float* in, float* out, const Work2M& w, unsigned* status,
                         cudaStream_t s, int fill) {
  switch (n) {
    case 2: k2m::launch_n<2>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 3: k2m::launch_n<3>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 4: k2m::launch_n<4>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 5: k2m::launch_n<5>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 6: k2m::launch_n<6>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 7: k2m::launch_n<7>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 8: k2m::launch_n<8>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 9: k2m::launch_n<9>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 10: k2m::launch_n<10>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 11: k2m::launch_n<11>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 12: k2m::launch_n<12>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 13: k2m::launch_n<13>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 14: k2m::launch_n<14>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 15: k2m::launch_n<15>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 16: k2m::launch_n<16>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    case 17: k2m::launch_n<17>(phase, p, x, m, count, in, out, w, status, s, fill); break;
    default: break;
  }
}

}  // namespace sl
