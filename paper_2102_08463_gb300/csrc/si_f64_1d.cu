// Spreading / interpolation kernels instantiated for double, 1D.
#include "spread_interp_1d.cuh"

namespace nufft {
NUFFT_INSTANTIATE_SI_1D(double, f64_1d)
}  // namespace nufft
