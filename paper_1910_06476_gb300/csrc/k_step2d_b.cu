// Instantiations of the 2D FP64 step kernels for n = 7, 8, 9, 10.
#include "k_step2d_impl.cuh"

namespace sl {
namespace k2d {
template void launch_n<7>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<8>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<9>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
template void launch_n<10>(int, const StepParams&, const Tables1D&, const Map2D&, int64_t, const double*, double*,
                            const Work2D&, unsigned*, cudaStream_t);
}  // namespace k2d
}  // namespace sl
