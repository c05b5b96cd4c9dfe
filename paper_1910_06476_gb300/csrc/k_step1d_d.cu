// Instantiations of the 1D FP64 step kernel for n = 14, 15, 16, 17.
#include "k_step1d_impl.cuh"

namespace sl {
namespace k1d {
template void launch_n<14>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<15>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<16>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
template void launch_n<17>(const StepParams&, const Tables1D&, const double*, double*, unsigned*, cudaStream_t);
}  // namespace k1d
}  // namespace sl
