// Instantiations of the 1D FP64 step kernel for n = 6, 7, 8, 9.
#include "k_step1d_impl.cuh"

namespace sl {
namespace k1d {
template void launch_n<6>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<7>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<8>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<9>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
}  // namespace k1d
}  // namespace sl
