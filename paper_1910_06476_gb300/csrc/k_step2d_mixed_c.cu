// Instantiations of the 2D mixed-precision step kernels for n = 13, 14, 15, 16, 17.
#include "k_step2d_mixed_impl.cuh"

namespace sl {
namespace k2m {
template void launch_n<13>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<14>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<15>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<16>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
template void launch_n<17>(int, const StepParams&, const Mixed2DExtra&, const Map2D&, int64_t, const float*, float*,
                            const Work2M&, unsigned*, cudaStream_t, int);
}  // namespace k2m
}  // namespace sl
