// Spreading / interpolation kernels instantiated for float, 2D.
#include "spread_interp.cuh"

namespace nufft {
NUFFT_INSTANTIATE_SI(float, 2, f32_2d)
}  // namespace nufft
