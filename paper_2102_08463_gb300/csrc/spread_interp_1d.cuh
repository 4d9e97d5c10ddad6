// spread_interp_1d.cuh -- 1D spreading (type 1 step 1, Sec. 3.1) and
// interpolation (type 2 step 3, Sec. 3.2), the d = 1 case of the method, which
// the paper lists as future work.  The same three methods as 2D / 3D:
//
//   SM       one CTA per (subproblem, transform): the padded bin (m0 + w
//            cells) in shared memory, one thread per point adding its w
//            values with shared atomics, then the bin added to the fine grid
//            with reductions (Sec. 4.1 SM steps 1-3); interpolation stages the
//            padded bin the same way and sums each point's w cells from it.
//   GM-sort  the same walk over bin-sorted records, straight to / from the
//            fine grid.
//   GM       one thread per (transform, point) in user order, positions from
//            the coordinates.
//
// Records are those of setpts: r.x = delta (kernel offset), r.z = the point's
// index (bits), r.w = window start relative to the padded bin origin.
#pragma once

#include "spread_interp.cuh"

namespace nufft {

template <typename T, int W, bool SM>
__device__ __forceinline__ void spread1_item(const KArgs<T> &a, int sp, int tr, T *sbuf)
{
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    const int4 sub = a.subprob[sp];
    const int o0 = (sub.x % a.nb0) * a.m0;
    const int P = pad_lo(W);
    const C *cin = a.cin + (int64_t)tr * a.M;
    C *grid = a.grid + (int64_t)tr * a.nftot;
    if (SM) {
        for (int i = threadIdx.x; i < 2 * a.p0; i += blockDim.x) sbuf[i] = (T)0;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < sub.z; k += blockDim.x) {
        const R r = a.recs[sub.y + k];
        const C cv = cin[(int)unpack_word<T>(r.z)];
        const int sx = (int)(unpack_word<T>(r.w) & 1023u);
        T v[W];
        kernel_row<T, W>(a, r.x, v);
#pragma unroll
        for (int i = 0; i < W; ++i) {
            if (SM) {
                atomicAdd(&sbuf[2 * (sx + i)], cv.x * v[i]);
                atomicAdd(&sbuf[2 * (sx + i) + 1], cv.y * v[i]);
            } else {
                atomic_add_cplx(&grid[wrap_any(o0 - P + sx + i, a.n0)], cv.x * v[i], cv.y * v[i]);
            }
        }
    }
    if (SM) {
        __syncthreads();
        // Sec. 4.1 SM step 3: the padded bin into the fine grid, l = (s + Delta) mod n
        for (int rx = threadIdx.x; rx < a.p0; rx += blockDim.x) {
            const T re = sbuf[2 * rx], im = sbuf[2 * rx + 1];
            if (re != (T)0 || im != (T)0)
                atomic_add_cplx(&grid[wrap_any(o0 - P + rx, a.n0)], re, im);
        }
        __syncthreads();
    }
}

template <typename T, int W, bool SM>
__device__ __forceinline__ void interp1_item(const KArgs<T> &a, int sp, int tr, T *sbuf)
{
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    const int4 sub = a.subprob[sp];
    const int o0 = (sub.x % a.nb0) * a.m0;
    const int P = pad_lo(W);
    const C *grid = a.grid + (int64_t)tr * a.nftot;
    C *cout = a.cout + (int64_t)tr * a.M;
    C *tile = reinterpret_cast<C *>(sbuf);
    if (SM) {
        for (int rx = threadIdx.x; rx < a.p0; rx += blockDim.x)
            tile[rx] = grid[wrap_any(o0 - P + rx, a.n0)];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < sub.z; k += blockDim.x) {
        const R r = a.recs[sub.y + k];
        const int sx = (int)(unpack_word<T>(r.w) & 1023u);
        T v[W];
        kernel_row<T, W>(a, r.x, v);
        T sr = 0, si = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const C g = SM ? tile[sx + i] : grid[wrap_any(o0 - P + sx + i, a.n0)];
            sr += v[i] * g.x;
            si += v[i] * g.y;
        }
        C o;
        o.x = sr;
        o.y = si;
        cout[(int)unpack_word<T>(r.z)] = o;
    }
    if (SM) __syncthreads();
}

template <typename T, int W, bool SPREAD, bool SM>
__global__ void __launch_bounds__(256)
sub1_kernel(KArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sbuf = reinterpret_cast<T *>(smem_raw);
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        if (SPREAD) spread1_item<T, W, SM>(a, (int)(wi % nsp), (int)(wi / nsp), sbuf);
        else interp1_item<T, W, SM>(a, (int)(wi % nsp), (int)(wi / nsp), sbuf);
    }
}

template <typename T, int W, bool SPREAD, bool SM>
__global__ void __launch_bounds__(256)
sub1_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                  int nplans)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sbuf = reinterpret_cast<T *>(smem_raw);
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        const KArgs<T> &a = args[pl];
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        if (SPREAD) spread1_item<T, W, SM>(a, (int)(local % nsp), (int)(local / nsp), sbuf);
        else interp1_item<T, W, SM>(a, (int)(local % nsp), (int)(local / nsp), sbuf);
    }
}

// GM: items [base, end) of the flattened (transform, point) range, user order.
template <typename T, int W, bool SPREAD>
__device__ __forceinline__ void gm1_range(const KArgs<T> &a, int64_t base, int64_t end, int64_t stride)
{
    using C = typename cplx<T>::type;
    for (int64_t item = base; item < end; item += stride) {
        const int tr = (int)(item / a.M);
        const int64_t j = item - (int64_t)tr * a.M;
        const AxisPos<T> px = axis_position<T>(period_fraction(a.xyz0[j]), a.n0, W);
        T v[W];
        kernel_row<T, W>(a, px.delta, v);
        if (SPREAD) {
            C *grid = a.grid + (int64_t)tr * a.nftot;
            const C cv = a.cin[item];
#pragma unroll
            for (int i = 0; i < W; ++i)
                atomic_add_cplx(&grid[wrap_any(px.l0 + i, a.n0)], cv.x * v[i], cv.y * v[i]);
        } else {
            const C *grid = a.grid + (int64_t)tr * a.nftot;
            T sr = 0, si = 0;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const C g = grid[wrap_any(px.l0 + i, a.n0)];
                sr += v[i] * g.x;
                si += v[i] * g.y;
            }
            C o;
            o.x = sr;
            o.y = si;
            a.cout[item] = o;
        }
    }
}

template <typename T, int W, bool SPREAD>
__global__ void __launch_bounds__(256)
gm1_kernel(KArgs<T> a)
{
    const int64_t total = a.M * a.ntransf;
    gm1_range<T, W, SPREAD>(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, total,
                            (int64_t)gridDim.x * blockDim.x);
}

// Batched GM: work item = a chunk of kGmChunk items of one plan.
template <typename T, int W, bool SPREAD>
__global__ void __launch_bounds__(256)
gm1_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff, int nplans)
{
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        const KArgs<T> &a = args[pl];
        const int64_t local = wi - workoff[pl];
        const int64_t chunks = *a.nsub;
        const int tr = (int)(local / chunks);
        const int64_t c0 = (local - (int64_t)tr * chunks) * kGmChunk;
        const int64_t end = min(c0 + kGmChunk, a.M);
        gm1_range<T, W, SPREAD>(a, (int64_t)tr * a.M + c0 + threadIdx.x, (int64_t)tr * a.M + end,
                                blockDim.x);
    }
}

template <typename T, int DIM, int W, bool SPREAD>
cudaError_t run1_w(Plan &p, const void *cin, void *cout)
{
    static_assert(DIM == 1, "1D kernels");
    KArgs<T> a = make_args<T>(p);
    a.cin = reinterpret_cast<const typename cplx<T>::type *>(cin);
    a.cout = reinterpret_cast<typename cplx<T>::type *>(cout);
    const int threads = p.threads;
    count_launch();
    if (p.method == NUFFT_METHOD_GM) {
        auto k = gm1_kernel<T, W, SPREAD>;
        int64_t blocks = (p.M * p.ntransf + threads - 1) / threads;
        const int64_t cap = (int64_t)p.num_sms * 32;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        k<<<(int)blocks, threads, 0, p.stream>>>(a);
    } else if (p.method == NUFFT_METHOD_SM) {
        const size_t smem = 2 * sizeof(T) * (size_t)a.p0;
        auto k = sub1_kernel<T, W, SPREAD, true>;
        if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
        k<<<persistent_grid(p, k, threads, smem), threads, smem, p.stream>>>(a);
    } else {
        auto k = sub1_kernel<T, W, SPREAD, false>;
        k<<<persistent_grid(p, k, threads, 0), threads, 0, p.stream>>>(a);
    }
    return cudaGetLastError();
}

template <typename T, int DIM, int W>
cudaError_t spread1_w(Plan &p, const void *c) { return run1_w<T, DIM, W, true>(p, c, nullptr); }
template <typename T, int DIM, int W>
cudaError_t interp1_w(Plan &p, void *c) { return run1_w<T, DIM, W, false>(p, nullptr, c); }

template <typename T, int DIM, int W, bool SPREAD>
cudaError_t multi1_w(const MultiLaunch &ml)
{
    const auto *args = reinterpret_cast<const KArgs<T> *>(ml.args);
    count_launch();
    if (ml.method == NUFFT_METHOD_GM) {
        auto k = gm1_multi_kernel<T, W, SPREAD>;
        k<<<multi_grid(k, ml.threads, 0, ml.num_sms), ml.threads, 0, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    } else if (ml.method == NUFFT_METHOD_SM) {
        const size_t smem = 2 * sizeof(T) * (size_t)ml.tile;
        auto k = sub1_multi_kernel<T, W, SPREAD, true>;
        if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
        k<<<multi_grid(k, ml.threads, smem, ml.num_sms), ml.threads, smem, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    } else {
        auto k = sub1_multi_kernel<T, W, SPREAD, false>;
        k<<<multi_grid(k, ml.threads, 0, ml.num_sms), ml.threads, 0, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    }
    return cudaGetLastError();
}

template <typename T, int DIM, int W>
cudaError_t spread1_multi_w(const MultiLaunch &ml) { return multi1_w<T, DIM, W, true>(ml); }
template <typename T, int DIM, int W>
cudaError_t interp1_multi_w(const MultiLaunch &ml) { return multi1_w<T, DIM, W, false>(ml); }

#define NUFFT_INSTANTIATE_SI_1D(T, TAG)                                       \
    cudaError_t spread_##TAG(Plan &p, const void *c)                          \
    {                                                                         \
        NUFFT_W_SWITCH(spread1_w, T, 1, p, c)                                 \
    }                                                                         \
    cudaError_t interp_##TAG(Plan &p, void *c)                                \
    {                                                                         \
        NUFFT_W_SWITCH(interp1_w, T, 1, p, c)                                 \
    }                                                                         \
    cudaError_t spread_multi_##TAG(const MultiLaunch &ml)                     \
    {                                                                         \
        NUFFT_W_SWITCH_ON(ml.w, spread1_multi_w, T, 1, ml)                    \
    }                                                                         \
    cudaError_t interp_multi_##TAG(const MultiLaunch &ml)                     \
    {                                                                         \
        NUFFT_W_SWITCH_ON(ml.w, interp1_multi_w, T, 1, ml)                    \
    }

}  // namespace nufft
