// Instantiations of the 1D mixed-precision step kernel for n = 2, 3, 4, 5, 6, 7, 8, 9.
#include "k_step1d_mixed_impl.cuh"

namespace sl {
namespace k1m {
template void launch_n<2>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<3>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<4>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<5>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<6>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<7>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<8>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
template void launch_n<9>(const Mixed1DParams&, const float*, float*, unsigned*, cudaStream_t);
}  // namespace k1m
}  // namespace sl
