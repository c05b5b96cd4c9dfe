// Instantiations of the 2D FP64 step kernels for n = 14, 15, 16, 17.
#include "k_step2d_impl.cuh"

namespace sl {
namespace k2d {
template void launch_n<14>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<15>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<16>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
template void launch_n<17>(const StepParams&, const Tables1D&, const double*, double*, Work2D, unsigned*, cudaStream_t);
}  // namespace k2d
}  // namespace sl
