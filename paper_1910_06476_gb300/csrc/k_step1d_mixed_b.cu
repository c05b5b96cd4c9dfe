// Instantiations of the 1D mixed-precision step kernel for n = 10, 11, 12, 13, 14, 15, 16, 17.
#include "k_step1d_mixed_impl.cuh"

namespace sl {
namespace k1m {
template void launch_n<10>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<11>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<12>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<13>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<14>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<15>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<16>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<17>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
}  // namespace k1m
}  // namespace sl
