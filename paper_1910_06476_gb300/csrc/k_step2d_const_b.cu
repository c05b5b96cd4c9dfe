// Instantiations of the 2D shared-operator (constant velocity) kernel for n = 10..17: tiles 4 x 4 (default), 4 x 2,
// 2 x 2 for n <= 12; 4 x 2 (default), 2 x 2 above.
#include "k_step2d_const_impl.cuh"

namespace sl {
namespace k2c {
template void launch<10, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<10, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<10, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<11, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<11, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<11, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<12, 4, 4>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<12, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<12, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<13, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<13, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<14, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<14, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<15, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<15, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<16, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<16, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<17, 4, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
template void launch<17, 2, 2>(const Mixed2DConstParams&, const float*, const float*, float*, unsigned*, cudaStream_t);
}  // namespace k2c
}  // namespace sl
