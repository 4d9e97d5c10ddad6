// Spreading / interpolation kernels instantiated for float, 1D.
#include "spread_interp_1d.cuh"

namespace nufft {
NUFFT_INSTANTIATE_SI_1D(float, f32_1d)
}  // namespace nufft
