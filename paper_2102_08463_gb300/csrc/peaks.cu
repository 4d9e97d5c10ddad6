// peaks.cu -- measured arithmetic peak of the GPU's FMA pipes, the denominator
// the benchmark's roofline uses for kernels bound by plain FP32 / FP64
// arithmetic (spreading and interpolation at large widths).  Not part of the
// transform.
#include "nufft_internal.cuh"

namespace nufft {
namespace {

constexpr int kChains = 8;          // independent FMA chains per thread
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads)
fma_loop_kernel(T *out, int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = a[i] * b + c;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    // never true for the inputs used; keeps the loop from being removed
    if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(int iters, double *tflops, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NUFFT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NUFFT_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_loop_kernel<T>, kPeakThreads, 0) !=
        cudaSuccess)
        return NUFFT_ERR_CUDA;
    const int blocks = sms * (per_sm < 1 ? 1 : per_sm);
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = NUFFT_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = NUFFT_ERR_CUDA;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == NUFFT_OK; ++rep) {      // the first launch warms up
        count_launch();
        cudaEventRecord(a, st);
        fma_loop_kernel<T><<<blocks, kPeakThreads, 0, st>>>(nullptr, iters, (T)0.999, (T)1e-4);
        cudaEventRecord(b, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
            rc = NUFFT_ERR_CUDA;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (rc != NUFFT_OK) return rc;
    const double fmas = (double)blocks * kPeakThreads * iters * kChains;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return NUFFT_OK;
}

}  // namespace
}  // namespace nufft

extern "C" int nufft_fma_peak(int prec, double *tflops, void *stream)
{
    if ((prec != 0 && prec != 1) || !tflops) return NUFFT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    return prec == 0 ? nufft::measure<float>(1024, tflops, st)
                     : nufft::measure<double>(256, tflops, st);
}
