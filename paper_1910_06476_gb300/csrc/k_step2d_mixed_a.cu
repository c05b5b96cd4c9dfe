// Instantiations of the 2D mixed-precision step kernels for n = 2, 3, 4, 5, 6, 7, 8.
#include "k_step2d_mixed_impl.cuh"

namespace sl {
namespace k2m {
template void launch_n<2>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<3>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<4>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<5>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<6>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<7>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<8>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
}  // namespace k2m
}  // namespace sl
