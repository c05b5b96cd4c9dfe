// Instantiations of the 2D FP64 step kernels for n = 14, 15, 16, 17.
#include "k_step2d_impl.cuh"

namespace sl {
namespace k2d {
template void launch_n<14>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<15>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<16>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<17>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
}  // namespace k2d
}  // namespace sl
