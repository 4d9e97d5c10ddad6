// Spreading / interpolation kernels instantiated for double, 2D.
#include "spread_interp.cuh"

namespace nufft {
NUFFT_INSTANTIATE_SI(double, 2, f64_2d)
}  // namespace nufft
