// correct.cu -- the correction steps (type 1 step 3 "truncate and scale",
// type 2 step 1 "pre-correct and zero-pad", Sec. 3.1 / 3.2), the plan-time
// computation of the correction factors p_k, and a fine-grid clear.
//
// Correction factors (Sec. 3.1 step 3): p_k = prod_i (2/w) / phihat(alpha_i k_i),
// alpha_i = w pi / n_i, times (-1)^{k_i} because fine-grid point l sits at
// -pi + l h (the origin implied by the bin rule of Sec. 4.1).  phihat is the
// kernel's Fourier transform, int_{-1}^{1} phi(z) cos(xi z) dz; with
// z = sin(t) the integrand exp(beta (cos t - 1)) cos(xi sin t) cos t is analytic
// on [-pi/2, pi/2], so Gauss-Legendre nodes in t (computed on the host by
// Newton's method on the Legendre recurrence) converge geometrically.
#include "nufft_internal.cuh"

namespace nufft {

namespace {

constexpr int kPerThread = 4;   // row elements per thread in the correction kernels

// One thread per mode: rows of N1 along threadIdx/blockIdx.x, one grid row
// (k2, k3, transform) per blockIdx.y/z slot.
template <typename T>
__global__ void deconvolve_kernel(const typename cplx<T>::type *__restrict__ grid,
                                  typename cplx<T>::type *__restrict__ f,
                                  const T *__restrict__ p0, const T *__restrict__ p1,
                                  const T *__restrict__ p2, int N0, int N1, int N2, int n0,
                                  int n1, int n2, int64_t nftot, int64_t Ntot, int64_t rows)
{
    using C = typename cplx<T>::type;
    const int h0 = N0 / 2, h1 = N1 / 2, h2 = N2 / 2;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const int i1 = (int)(row % N1);
        const int64_t r2 = row / N1;
        const int i2 = (int)(r2 % N2);
        const int tr = (int)(r2 / N2);
        int l1 = i1 - h1;
        if (l1 < 0) l1 += n1;
        int l2 = i2 - h2;
        if (l2 < 0) l2 += n2;
        const T s = p1[i1] * p2[i2];
        const C *src = grid + (int64_t)tr * nftot + ((int64_t)l2 * n1 + l1) * n0;
        C *dst = f + (int64_t)tr * Ntot + ((int64_t)i2 * N1 + i1) * N0;
        // kPerThread modes per thread, consecutive across the lanes of each step
        for (int b0 = blockIdx.x * blockDim.x * kPerThread; b0 < N0;
             b0 += gridDim.x * blockDim.x * kPerThread) {
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                const int i0 = b0 + u * (int)blockDim.x + threadIdx.x;
                if (i0 < N0) {
                    int l0 = i0 - h0;
                    if (l0 < 0) l0 += n0;
                    const C v = src[l0];
                    const T sc = s * p0[i0];
                    C o;
                    o.x = v.x * sc;
                    o.y = v.y * sc;
                    dst[i0] = o;
                }
            }
        }
    }
}

// One thread per fine-grid cell of a row: mode value scaled by p_k, or zero.
template <typename T>
__global__ void precorrect_kernel(const typename cplx<T>::type *__restrict__ f,
                                  typename cplx<T>::type *__restrict__ grid,
                                  const T *__restrict__ p0, const T *__restrict__ p1,
                                  const T *__restrict__ p2, int N0, int N1, int N2, int n0,
                                  int n1, int n2, int64_t nftot, int64_t Ntot, int64_t rows)
{
    using C = typename cplx<T>::type;
    const int h0 = N0 / 2, h1 = N1 / 2, h2 = N2 / 2;
    const int c0 = N0 - h0, c1 = N1 - h1, c2 = N2 - h2;     // ceil(N/2)
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const int l1 = (int)(row % n1);
        const int64_t r2 = row / n1;
        const int l2 = (int)(r2 % n2);
        const int tr = (int)(r2 / n2);
        // mode index along y / z, or -1 for a zero-padding row
        int i1 = l1 < c1 ? l1 + h1 : (l1 >= n1 - h1 ? l1 - n1 + h1 : -1);
        int i2 = l2 < c2 ? l2 + h2 : (l2 >= n2 - h2 ? l2 - n2 + h2 : -1);
        C *dst = grid + (int64_t)tr * nftot + ((int64_t)l2 * n1 + l1) * n0;
        if (i1 < 0 || i2 < 0) {
            C zero;
            zero.x = 0;
            zero.y = 0;
            for (int b0 = blockIdx.x * blockDim.x * kPerThread; b0 < n0;
                 b0 += gridDim.x * blockDim.x * kPerThread) {
#pragma unroll
                for (int u = 0; u < kPerThread; ++u) {
                    const int l0 = b0 + u * (int)blockDim.x + threadIdx.x;
                    if (l0 < n0) dst[l0] = zero;
                }
            }
            continue;
        }
        const T s = p1[i1] * p2[i2];
        const C *src = f + (int64_t)tr * Ntot + ((int64_t)i2 * N1 + i1) * N0;
        for (int b0 = blockIdx.x * blockDim.x * kPerThread; b0 < n0;
             b0 += gridDim.x * blockDim.x * kPerThread) {
#pragma unroll
            for (int u = 0; u < kPerThread; ++u) {
                const int l0 = b0 + u * (int)blockDim.x + threadIdx.x;
                if (l0 >= n0) continue;
                const int i0 = l0 < c0 ? l0 + h0 : (l0 >= n0 - h0 ? l0 - n0 + h0 : -1);
                C o;
                if (i0 >= 0) {
                    const C v = src[i0];
                    const T sc = s * p0[i0];
                    o.x = v.x * sc;
                    o.y = v.y * sc;
                } else {
                    o.x = 0;
                    o.y = 0;
                }
                dst[l0] = o;
            }
        }
    }
}

__global__ void zero_kernel(uint4 *__restrict__ p, size_t n16)
{
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = z;
}

__global__ void set_int_kernel(int32_t *dst, int32_t v)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *dst = v;
}

// p(k) for k = -floor(N/2) .. ceil(N/2)-1 along one axis, from the quadrature
// nodes t_q and weights v_q = (pi/2) w_q exp(beta (cos t_q - 1)) cos t_q.
template <typename T>
__global__ void correction_kernel(T *__restrict__ out, int N, int n, int w,
                                  const double *__restrict__ st, const double *__restrict__ v,
                                  int nq)
{
    const double PI = 3.14159265358979323846;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int k = i - N / 2;
        const double xi = (double)w * PI * (double)k / (double)n;
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += v[q] * cos(xi * st[q]);
        const double sgn = (k & 1) ? -1.0 : 1.0;
        out[i] = (T)(sgn * (2.0 / (double)w) / s);
    }
}

// Threads per block for rows of rowlen elements: enough warps to give every
// thread kPerThread elements, at most 256.
inline int row_threads(int rowlen)
{
    int t = (rowlen + kPerThread - 1) / kPerThread;
    t = (t + 31) / 32 * 32;
    return t < 32 ? 32 : (t > 256 ? 256 : t);
}

inline dim3 row_grid(int64_t rows, int rowlen, int threads)
{
    int bx = (rowlen + threads * kPerThread - 1) / (threads * kPerThread);
    if (bx < 1) bx = 1;
    int64_t by = rows < 65535 ? rows : 65535;
    return dim3(bx, (unsigned)(by < 1 ? 1 : by), 1);
}

template <typename T>
cudaError_t deconvolve_impl(Plan &p, void *f)
{
    const int64_t rows = p.N[1] * p.N[2] * p.ntransf;
    const int threads = row_threads((int)p.N[0]);
    count_launch();
    deconvolve_kernel<T><<<row_grid(rows, (int)p.N[0], threads), threads, 0, p.stream>>>(
        reinterpret_cast<const typename cplx<T>::type *>(p.fine),
        reinterpret_cast<typename cplx<T>::type *>(f), (const T *)p.corr[0], (const T *)p.corr[1],
        (const T *)p.corr[2], (int)p.N[0], (int)p.N[1], (int)p.N[2], (int)p.nf[0], (int)p.nf[1],
        (int)p.nf[2], p.nftot, p.Ntot, rows);
    return cudaGetLastError();
}

template <typename T>
cudaError_t precorrect_impl(Plan &p, const void *f)
{
    const int64_t rows = p.nf[1] * p.nf[2] * p.ntransf;
    const int threads = row_threads((int)p.nf[0]);
    count_launch();
    precorrect_kernel<T><<<row_grid(rows, (int)p.nf[0], threads), threads, 0, p.stream>>>(
        reinterpret_cast<const typename cplx<T>::type *>(f),
        reinterpret_cast<typename cplx<T>::type *>(p.fine), (const T *)p.corr[0],
        (const T *)p.corr[1], (const T *)p.corr[2], (int)p.N[0], (int)p.N[1], (int)p.N[2],
        (int)p.nf[0], (int)p.nf[1], (int)p.nf[2], p.nftot, p.Ntot, rows);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_deconvolve(Plan &p, void *f)
{
    return p.prec == 0 ? deconvolve_impl<float>(p, f) : deconvolve_impl<double>(p, f);
}

cudaError_t launch_precorrect(Plan &p, const void *f)
{
    return p.prec == 0 ? precorrect_impl<float>(p, f) : precorrect_impl<double>(p, f);
}

cudaError_t launch_zero(Plan &p, void *ptr, size_t bytes)
{
    // every buffer cleared here is a multiple of 16 bytes (complex float pairs or wider)
    const size_t n16 = bytes / 16;
    if (n16 == 0) return cudaSuccess;
    size_t blocks = (n16 + 255) / 256;
    const size_t cap = (size_t)p.num_sms * 8;
    if (blocks > cap) blocks = cap;
    count_launch();
    zero_kernel<<<(unsigned)blocks, 256, 0, p.stream>>>(reinterpret_cast<uint4 *>(ptr), n16);
    return cudaGetLastError();
}

cudaError_t launch_set_int(Plan &p, int32_t *dst, int32_t value)
{
    count_launch();
    set_int_kernel<<<1, 32, 0, p.stream>>>(dst, value);   // the value travels as a kernel argument
    return cudaGetLastError();
}

cudaError_t launch_correction(Plan &p, const double *st, const double *v, int nq)
{
    for (int d = 0; d < p.dim; ++d) {
        const int N = (int)p.N[d];
        const int blocks = (N + 127) / 128;
        count_launch();
        if (p.prec == 0)
            correction_kernel<float><<<blocks, 128, 0, p.stream>>>((float *)p.corr[d], N,
                                                                   (int)p.nf[d], p.w, st, v, nq);
        else
            correction_kernel<double><<<blocks, 128, 0, p.stream>>>((double *)p.corr[d], N,
                                                                    (int)p.nf[d], p.w, st, v, nq);
    }
    return cudaGetLastError();
}

}  // namespace nufft
