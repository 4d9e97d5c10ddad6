// Spreading / interpolation kernels instantiated for float, 3D.
#include "spread_interp.cuh"

namespace nufft {
NUFFT_INSTANTIATE_SI(float, 3, f32_3d)
}  // namespace nufft
