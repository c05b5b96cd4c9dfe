// Instantiations of the 1D FP64 step kernel for n = 10, 11, 12, 13.
#include "k_step1d_impl.cuh"

namespace sl {
namespace k1d {
template void launch_n<10>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<11>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<12>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<13>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
}  // namespace k1d
}  // namespace sl
