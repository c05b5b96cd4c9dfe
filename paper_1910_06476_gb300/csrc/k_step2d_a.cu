// Instantiations of the 2D FP64 step kernels for n = 2, 3, 4, 5, 6.
#include "k_step2d_impl.cuh"

namespace sl {
namespace k2d {
template void launch_n<2>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<3>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<4>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<5>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<6>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
}  // namespace k2d
}  // namespace sl
