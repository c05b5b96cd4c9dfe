// Dispatch of the 2D shared-operator kernel on the node count and the tile shape (elements per
// CTA, TX x TY).  Each node count has a few compiled shapes, all within 48 KB of static shared
// memory and 1024 threads; index 0 is the default, the others are candidates for the autotuner
// (sl_tune).  Every shape computes each element with the same arithmetic.
#include "sl_internal.h"

namespace sl {
namespace k2c {
template <int NN, int TX, int TY>
void launch(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* st, cudaStream_t s);
}

int k2c_tile_count(int n) { return n <= 12 ? 3 : 2; }

void k2c_tile_shape(int n, int tile, int* tx, int* ty) {
  static const int small[3][2] = {{8, 4}, {4, 4}, {8, 2}};     // n <= 9
  static const int mid[3][2] = {{4, 4}, {4, 2}, {2, 2}};       // n = 10..12
  static const int large[2][2] = {{4, 2}, {2, 2}};             // n = 13..17
  if (tile < 0 || tile >= k2c_tile_count(n)) tile = 0;
  const int(*t)[2] = n <= 9 ? small : n <= 12 ? mid : large;
  *tx = t[tile][0];
  *ty = t[tile][1];
}

#define SL_K2C(N, A, B) k2c::launch<N, A, B>(p, tab, in, out, status, s)
#define SL_K2C_SMALL(N)                        \
  case N:                                      \
    if (tile == 1) SL_K2C(N, 4, 4);            \
    else if (tile == 2) SL_K2C(N, 8, 2);       \
    else SL_K2C(N, 8, 4);                      \
    break;
#define SL_K2C_MID(N)                          \
  case N:                                      \
    if (tile == 1) SL_K2C(N, 4, 2);            \
    else if (tile == 2) SL_K2C(N, 2, 2);       \
    else SL_K2C(N, 4, 4);                      \
    break;
#define SL_K2C_LARGE(N)                        \
  case N:                                      \
    if (tile == 1) SL_K2C(N, 2, 2);            \
    else SL_K2C(N, 4, 2);                      \
    break;

void launch_step2d_const(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* status,
                         cudaStream_t s, int tile) {
  switch (p.n) {
    SL_K2C_SMALL(2)
    SL_K2C_SMALL(3)
    SL_K2C_SMALL(4)
    SL_K2C_SMALL(5)
    SL_K2C_SMALL(6)
    SL_K2C_SMALL(7)
    SL_K2C_SMALL(8)
    SL_K2C_SMALL(9)
    SL_K2C_MID(10)
    SL_K2C_MID(11)
    SL_K2C_MID(12)
    SL_K2C_LARGE(13)
    SL_K2C_LARGE(14)
    SL_K2C_LARGE(15)
    SL_K2C_LARGE(16)
    SL_K2C_LARGE(17)
    default: break;
  }
}

#undef SL_K2C_SMALL
#undef SL_K2C_MID
#undef SL_K2C_LARGE
#undef SL_K2C

}  // namespace sl
