// Spreading / interpolation kernels instantiated for double, 3D.
#include "spread_interp.cuh"

namespace nufft {
NUFFT_INSTANTIATE_SI(double, 3, f64_3d)
}  // namespace nufft
