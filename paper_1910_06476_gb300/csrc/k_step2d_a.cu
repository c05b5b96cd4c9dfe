// Instantiations of the 2D FP64 step kernels for n = 2, 3, 4, 5, 6.
#include "k_step2d_impl.cuh"

namespace sl {
namespace k2d {
template void launch_n<2>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<3>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<4>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<5>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<6>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
}  // namespace k2d
}  // namespace sl
