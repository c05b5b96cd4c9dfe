// Instantiations of the 1D FP64 step kernel for n = 2, 3, 4, 5.
#include "k_step1d_impl.cuh"

namespace sl {
namespace k1d {
template void launch_n<2>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<3>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<4>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<5>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
}  // namespace k1d
}  // namespace sl
