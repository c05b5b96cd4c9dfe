// Dispatch of the 2D shared-operator kernel on the node count (tile sizes keep a CTA within
// 48 KB of shared memory and 1024 threads).
#include "sl_internal.h"

namespace sl {
namespace k2c {
template <int NN, int TX, int TY>
void launch(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* st, cudaStream_t s);
}

void launch_step2d_const(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* status,
                         cudaStream_t s) {
  switch (p.n) {
    case 2: k2c::launch<2, 8, 4>(p, tab, in, out, status, s); break;
    case 3: k2c::launch<3, 8, 4>(p, tab, in, out, status, s); break;
    case 4: k2c::launch<4, 8, 4>(p, tab, in, out, status, s); break;
    case 5: k2c::launch<5, 8, 4>(p, tab, in, out, status, s); break;
    case 6: k2c::launch<6, 8, 4>(p, tab, in, out, status, s); break;
    case 7: k2c::launch<7, 8, 4>(p, tab, in, out, status, s); break;
    case 8: k2c::launch<8, 8, 4>(p, tab, in, out, status, s); break;
    case 9: k2c::launch<9, 8, 4>(p, tab, in, out, status, s); break;
    case 10: k2c::launch<10, 4, 4>(p, tab, in, out, status, s); break;
    case 11: k2c::launch<11, 4, 4>(p, tab, in, out, status, s); break;
    case 12: k2c::launch<12, 4, 4>(p, tab, in, out, status, s); break;
    case 13: k2c::launch<13, 4, 2>(p, tab, in, out, status, s); break;
    case 14: k2c::launch<14, 4, 2>(p, tab, in, out, status, s); break;
    case 15: k2c::launch<15, 4, 2>(p, tab, in, out, status, s); break;
    case 16: k2c::launch<16, 4, 2>(p, tab, in, out, status, s); break;
    case 17: k2c::launch<17, 4, 2>(p, tab, in, out, status, s); break;
    default: break;
  }
}

}  // namespace sl
