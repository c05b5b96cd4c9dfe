// Instantiations of the 2D mixed-precision step kernels for n = 13, 14, 15, 16, 17.
#include "k_step2d_mixed_impl.cuh"

namespace sl {
namespace k2m {
template void launch_n<13>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<14>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<15>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<16>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<17>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
}  // namespace k2m
}  // namespace sl
