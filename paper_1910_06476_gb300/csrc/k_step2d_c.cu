// Instantiations of the 2D FP64 step kernels for n = 11, 12, 13.
#include "k_step2d_impl.cuh"

namespace sl {
namespace k2d {
template void launch_n<11>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<12>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<13>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
}  // namespace k2d
}  // namespace sl
