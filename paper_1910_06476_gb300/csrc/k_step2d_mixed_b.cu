// Instantiations of the 2D mixed-precision step kernels for n = 9, 10, 11, 12.
#include "k_step2d_mixed_impl.cuh"

namespace sl {
namespace k2m {
template void launch_n<9>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<10>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<11>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<12>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
}  // namespace k2m
}  // namespace sl
