// Instantiations of the 2D shared-operator (constant velocity) kernel for n = 2..9, tiles 8 x 4 (default), 4 x 4, 8 x 2.
#include "k_step2d_const_impl.cuh"

namespace sl {
namespace k2c {
template void launch<2, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<2, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<2, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<3, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<3, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<3, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<4, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<4, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<4, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<5, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<5, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<5, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<6, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<6, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<6, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<7, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<7, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<7, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<8, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<8, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<8, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<9, 8, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<9, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<9, 8, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
}  // namespace k2c
}  // namespace sl
