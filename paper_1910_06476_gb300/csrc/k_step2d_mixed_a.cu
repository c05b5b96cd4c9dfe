// Instantiations of the 2D mixed-precision step kernels for n = 2, 3, 4, 5, 6, 7, 8.
#include "k_step2d_mixed_impl.cuh"

namespace sl {
namespace k2m {
template void launch_n<2>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<3>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<4>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<5>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<6>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<7>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<8>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
}  // namespace k2m
}  // namespace sl
