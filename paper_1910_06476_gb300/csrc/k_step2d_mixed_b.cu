// Instantiations of the 2D mixed-precision step kernels for n = 9, 10, 11, 12.
#include "k_step2d_mixed_impl.cuh"

namespace sl {
namespace k2m {
template void launch_n<9>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<10>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<11>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
template void launch_n<12>(const StepParams&, const Mixed2DExtra&, const float*, float*, Work2M, unsigned*, cudaStream_t);
}  // namespace k2m
}  // namespace sl
