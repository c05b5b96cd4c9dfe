// Dispatch of the 1D FP64 step kernel on the node count.
#include "sl_internal.h"

namespace sl {
namespace k1d {
template <int NN>
void launch_n(const StepParams& p, const Tables1D& tb, const double* in, double* out, unsigned* st, cudaStream_t s);
}

void launch_step1d_f64(int n, const StepParams& p, const Tables1D& tb, const double* in, double* out,
                       unsigned* status, cudaStream_t s) {
  switch (n) {
    case 2: k1d::launch_n<2>(p, tb, in, out, status, s); break;
    case 3: k1d::launch_n<3>(p, tb, in, out, status, s); break;
    case 4: k1d::launch_n<4>(p, tb, in, out, status, s); break;
    case 5: k1d::launch_n<5>(p, tb, in, out, status, s); break;
    case 6: k1d::launch_n<6>(p, tb, in, out, status, s); break;
    case 7: k1d::launch_n<7>(p, tb, in, out, status, s); break;
    case 8: k1d::launch_n<8>(p, tb, in, out, status, s); break;
    case 9: k1d::launch_n<9>(p, tb, in, out, status, s); break;
    case 10: k1d::launch_n<10>(p, tb, in, out, status, s); break;
    case 11: k1d::launch_n<11>(p, tb, in, out, status, s); break;
    case 12: k1d::launch_n<12>(p, tb, in, out, status, s); break;
    case 13: k1d::launch_n<13>(p, tb, in, out, status, s); break;
    case 14: k1d::launch_n<14>(p, tb, in, out, status, s); break;
    case 15: k1d::launch_n<15>(p, tb, in, out, status, s); break;
    case 16: k1d::launch_n<16>(p, tb, in, out, status, s); break;
    case 17: k1d::launch_n<17>(p, tb, in, out, status, s); break;
    default: break;
  }
}

}  // namespace sl
