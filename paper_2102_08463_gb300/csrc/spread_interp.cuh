// spread_interp.cuh -- spreading (type 1 step 1, Sec. 3.1 / Sec. 4.1) and
// interpolation (type 2 step 3, Sec. 3.2 / Sec. 4.2) kernels, templated on the
// precision T, the dimension DIM and the kernel width W.
//
// Thread mapping shared by every kernel here: a warp is cut into G = 32 / W
// lane groups of W lanes; group g works on one point, lane dx of the group owns
// window column dx.  Each lane evaluates the ES kernel only for its own column
// in x, y (and z) -- d evaluations per lane instead of d*W per thread -- and
// the y / z weights of the other columns come from the group by warp shuffles.
// The W lanes of a group touch W consecutive cells of a grid row, so their
// shared-memory atomics fall in distinct banks and their global accesses
// coalesce.
//
//   SM       one CTA per subproblem (Sec. 4.1 SM steps 1-3): points accumulate
//            into a shared-memory copy of the padded bin, p_i = m_i + 2 ceil(w/2)
//            cells per axis, then the padded bin is atomically added to the
//            fine grid with periodic wrap.  Persistent CTAs stride over the
//            (subproblem, transform) pairs.
//   GM-sort  the same bin-ordered points, atomics straight into the fine grid.
//   GM       user order, positions recomputed from the coordinates.
//   interp   the transpose: each group gathers its point's w^d cells (from the
//            fine grid, or from a padded bin staged in shared memory) and the
//            W column sums are combined with shuffles.
#pragma once

#include "nufft_internal.cuh"

namespace nufft {

constexpr unsigned kFullMask = 0xffffffffu;

template <typename T>
struct KArgs {
    const typename rec4<T>::type *recs;
    const int32_t *perm;
    const int4 *subprob;
    const int32_t *nsub;
    const T *xyz0, *xyz1, *xyz2;                 // coordinates (GM kernels)
    typename cplx<T>::type *grid;                // fine grid [ntransf][n3][n2][n1]
    const typename cplx<T>::type *cin;           // spread input  [ntransf][M]
    typename cplx<T>::type *cout;                // interp output [ntransf][M]
    int64_t M;
    int64_t nftot;
    int ntransf;
    int n0, n1, n2;                              // fine grid
    int m0, m1, m2;                              // bin size
    int nb0, nb1;                                // bins along x, y
    int p0, p1, p2;                              // padded bin
    T beta;
    T hw;                                        // 2 / w
};

template <typename T> __device__ __forceinline__ uint32_t unpack_word(T v);
template <> __device__ __forceinline__ uint32_t unpack_word<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ uint32_t unpack_word<double>(double v)
{
    return (uint32_t)__double_as_longlong(v);
}

__device__ __forceinline__ int wrap_any(int v, int n)
{
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// Bin origin (first cell) of bin index b along each axis.
__device__ __forceinline__ void bin_origin(int b, int nb0, int nb1, int m0, int m1, int m2,
                                           int &o0, int &o1, int &o2)
{
    int bx = b % nb0;
    int r = b / nb0;
    int by = r % nb1;
    int bz = r / nb1;
    o0 = bx * m0;
    o1 = by * m1;
    o2 = bz * m2;
}

// ---------------------------------------------------------------------------
// SM spreading.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_sm_kernel(KArgs<T> a)
{
    using C = typename cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ptot = a.p0 * a.p1 * (DIM == 3 ? a.p2 : 1);
    T *sre = reinterpret_cast<T *>(smem_raw);
    T *sim = sre + ptot;
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int P = (W + 1) / 2;
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int sp = (int)(wi % nsp);
        const int tr = (int)(wi / nsp);
        const int4 sub = a.subprob[sp];
        for (int i = threadIdx.x; i < ptot; i += blockDim.x) {
            sre[i] = (T)0;
            sim[i] = (T)0;
        }
        __syncthreads();
        const C *cin = a.cin + (int64_t)tr * a.M;
        for (int q0 = warp * G; q0 < sub.z; q0 += nwarps * G) {
            const int q = q0 + g;
            const bool act = gact && q < sub.z;
            T wx = 0, wy = 0, wz = 0, cre = 0, cim = 0;
            int sx = 0, sy = 0, sz = 0;
            if (act) {
                const auto r = a.recs[sub.y + q];
                const C cv = cin[a.perm[sub.y + q]];
                cre = cv.x;
                cim = cv.y;
                wx = es_kernel(((T)dx - r.x) * a.hw, a.beta);
                wy = es_kernel(((T)dx - r.y) * a.hw, a.beta);
                if (DIM == 3) wz = es_kernel(((T)dx - r.z) * a.hw, a.beta);
                const uint32_t pk = unpack_word<T>(r.w);
                sx = pk & 1023u;
                sy = (pk >> 10) & 1023u;
                sz = pk >> 20;
            }
            if (DIM == 2) {
#pragma unroll
                for (int iy = 0; iy < W; ++iy) {
                    const T vy = __shfl_sync(kFullMask, wy, src0 + iy);
                    if (act) {
                        const T v = wx * vy;
                        const int idx = (sy + iy) * a.p0 + sx + dx;
                        atomicAdd(&sre[idx], v * cre);
                        atomicAdd(&sim[idx], v * cim);
                    }
                }
            } else {
#pragma unroll 1
                for (int iz = 0; iz < W; ++iz) {
                    const T vz = __shfl_sync(kFullMask, wz, src0 + iz);
                    const T zr = cre * vz, zi = cim * vz;
                    const int zoff = (sz + iz) * a.p1;
#pragma unroll
                    for (int iy = 0; iy < W; ++iy) {
                        const T vy = __shfl_sync(kFullMask, wy, src0 + iy);
                        if (act) {
                            const T v = wx * vy;
                            const int idx = (zoff + sy + iy) * a.p0 + sx + dx;
                            atomicAdd(&sre[idx], v * zr);
                            atomicAdd(&sim[idx], v * zi);
                        }
                    }
                }
            }
        }
        __syncthreads();
        // Step 3: add the padded bin back to the fine grid, l = (s + Delta) mod n.
        int o0, o1, o2;
        bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
        C *grid = a.grid + (int64_t)tr * a.nftot;
        const int rows = a.p1 * (DIM == 3 ? a.p2 : 1);
        for (int r = warp; r < rows; r += nwarps) {
            const int ry = r % a.p1, rz = r / a.p1;
            const int gy = wrap_any(o1 - P + ry, a.n1);
            const int gz = DIM == 3 ? wrap_any(o2 - P + rz, a.n2) : 0;
            const int64_t rowbase = ((int64_t)gz * a.n1 + gy) * a.n0;
            for (int rx = lane; rx < a.p0; rx += 32) {
                const T re = sre[r * a.p0 + rx], im = sim[r * a.p0 + rx];
                if (re != (T)0 || im != (T)0) {
                    const int gx = wrap_any(o0 - P + rx, a.n0);
                    atomic_add_cplx(&grid[rowbase + gx], re, im);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// GM-sort spreading: bin-ordered points, global atomics.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_gmsort_kernel(KArgs<T> a)
{
    using C = typename cplx<T>::type;
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int P = (W + 1) / 2;
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int sp = (int)(wi % nsp);
        const int tr = (int)(wi / nsp);
        const int4 sub = a.subprob[sp];
        int o0, o1, o2;
        bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
        const C *cin = a.cin + (int64_t)tr * a.M;
        C *grid = a.grid + (int64_t)tr * a.nftot;
        for (int q0 = warp * G; q0 < sub.z; q0 += nwarps * G) {
            const int q = q0 + g;
            const bool act = gact && q < sub.z;
            T wx = 0, wy = 0, wz = 0, cre = 0, cim = 0;
            int gx = 0, ly0 = 0, lz0 = 0;
            if (act) {
                const auto r = a.recs[sub.y + q];
                const C cv = cin[a.perm[sub.y + q]];
                cre = cv.x;
                cim = cv.y;
                wx = es_kernel(((T)dx - r.x) * a.hw, a.beta);
                wy = es_kernel(((T)dx - r.y) * a.hw, a.beta);
                if (DIM == 3) wz = es_kernel(((T)dx - r.z) * a.hw, a.beta);
                const uint32_t pk = unpack_word<T>(r.w);
                gx = wrap_any(o0 - P + (int)(pk & 1023u) + dx, a.n0);
                ly0 = o1 - P + (int)((pk >> 10) & 1023u);
                lz0 = o2 - P + (int)(pk >> 20);
            }
            const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
            for (int iz = 0; iz < nz; ++iz) {
                T zr = cre, zi = cim;
                int gz = 0;
                if (DIM == 3) {
                    const T vz = __shfl_sync(kFullMask, wz, src0 + iz);
                    zr *= vz;
                    zi *= vz;
                    gz = wrap_any(lz0 + iz, a.n2);
                }
#pragma unroll
                for (int iy = 0; iy < W; ++iy) {
                    const T vy = __shfl_sync(kFullMask, wy, src0 + iy);
                    if (act) {
                        const T v = wx * vy;
                        const int gy = wrap_any(ly0 + iy, a.n1);
                        atomic_add_cplx(&grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx], v * zr, v * zi);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// GM spreading: user order, positions from the coordinates.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_gm_kernel(KArgs<T> a)
{
    using C = typename cplx<T>::type;
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = a.M * a.ntransf;
    for (int64_t base = gwarp * G; base < total; base += nwarps_total * G) {
        const int64_t item = base + g;
        const bool act = gact && item < total;
        T wx = 0, wy = 0, wz = 0, cre = 0, cim = 0;
        int gx = 0, ly0 = 0, lz0 = 0, tr = 0;
        if (act) {
            tr = (int)(item / a.M);
            const int64_t j = item - (int64_t)tr * a.M;
            const AxisPos<T> px = axis_position<T>(period_fraction(a.xyz0[j]), a.n0, W);
            const AxisPos<T> py = axis_position<T>(period_fraction(a.xyz1[j]), a.n1, W);
            wx = es_kernel(((T)dx - px.delta) * a.hw, a.beta);
            wy = es_kernel(((T)dx - py.delta) * a.hw, a.beta);
            gx = wrap_any(px.l0 + dx, a.n0);
            ly0 = py.l0;
            if (DIM == 3) {
                const AxisPos<T> pz = axis_position<T>(period_fraction(a.xyz2[j]), a.n2, W);
                wz = es_kernel(((T)dx - pz.delta) * a.hw, a.beta);
                lz0 = pz.l0;
            }
            const C cv = a.cin[item];
            cre = cv.x;
            cim = cv.y;
        }
        C *grid = a.grid + (int64_t)tr * a.nftot;
        const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
        for (int iz = 0; iz < nz; ++iz) {
            T zr = cre, zi = cim;
            int gz = 0;
            if (DIM == 3) {
                const T vz = __shfl_sync(kFullMask, wz, src0 + iz);
                zr *= vz;
                zi *= vz;
                gz = wrap_any(lz0 + iz, a.n2);
            }
#pragma unroll
            for (int iy = 0; iy < W; ++iy) {
                const T vy = __shfl_sync(kFullMask, wy, src0 + iy);
                if (act) {
                    const T v = wx * vy;
                    const int gy = wrap_any(ly0 + iy, a.n1);
                    atomic_add_cplx(&grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx], v * zr, v * zi);
                }
            }
        }
    }
}

// Sum of a value over the W lanes of each group; lane dx == 0 gets the total.
template <typename T, int W>
__device__ __forceinline__ T group_sum(T v, int dx)
{
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        const T t = __shfl_down_sync(kFullMask, v, o);
        if (dx + o < W) v += t;
    }
    return v;
}

// ---------------------------------------------------------------------------
// Sorted interpolation (GM-sort, Sec. 4.2) and its shared-memory staged form
// (STAGED = true): the padded bin of the subproblem is first copied into
// shared memory with coalesced row loads, then every gather reads it there.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W, bool STAGED>
__global__ void __launch_bounds__(256)
interp_sorted_kernel(KArgs<T> a)
{
    using C = typename cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int P = (W + 1) / 2;
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int sp = (int)(wi % nsp);
        const int tr = (int)(wi / nsp);
        const int4 sub = a.subprob[sp];
        int o0, o1, o2;
        bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
        const C *grid = a.grid + (int64_t)tr * a.nftot;
        C *cout = a.cout + (int64_t)tr * a.M;
        if (STAGED) {
            const int rows = a.p1 * (DIM == 3 ? a.p2 : 1);
            for (int r = warp; r < rows; r += nwarps) {
                const int ry = r % a.p1, rz = r / a.p1;
                const int gy = wrap_any(o1 - P + ry, a.n1);
                const int gz = DIM == 3 ? wrap_any(o2 - P + rz, a.n2) : 0;
                const int64_t rowbase = ((int64_t)gz * a.n1 + gy) * a.n0;
                for (int rx = lane; rx < a.p0; rx += 32)
                    tile[r * a.p0 + rx] = grid[rowbase + wrap_any(o0 - P + rx, a.n0)];
            }
            __syncthreads();
        }
        for (int q0 = warp * G; q0 < sub.z; q0 += nwarps * G) {
            const int q = q0 + g;
            const bool act = gact && q < sub.z;
            T wx = 0, wy = 0, wz = 0;
            int sx = 0, sy = 0, sz = 0;
            if (act) {
                const auto r = a.recs[sub.y + q];
                wx = es_kernel(((T)dx - r.x) * a.hw, a.beta);
                wy = es_kernel(((T)dx - r.y) * a.hw, a.beta);
                if (DIM == 3) wz = es_kernel(((T)dx - r.z) * a.hw, a.beta);
                const uint32_t pk = unpack_word<T>(r.w);
                sx = pk & 1023u;
                sy = (pk >> 10) & 1023u;
                sz = pk >> 20;
            }
            const int gx = STAGED ? 0 : wrap_any(o0 - P + sx + dx, a.n0);
            T ar = 0, ai = 0;
            const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
            for (int iz = 0; iz < nz; ++iz) {
                T vz = (T)1;
                if (DIM == 3) vz = __shfl_sync(kFullMask, wz, src0 + iz);
                T zr = 0, zi = 0;
#pragma unroll
                for (int iy = 0; iy < W; ++iy) {
                    const T vy = __shfl_sync(kFullMask, wy, src0 + iy);
                    if (act) {
                        C v;
                        if (STAGED) {
                            v = tile[((sz + iz) * a.p1 + sy + iy) * a.p0 + sx + dx];
                        } else {
                            const int gy = wrap_any(o1 - P + sy + iy, a.n1);
                            const int gz = DIM == 3 ? wrap_any(o2 - P + sz + iz, a.n2) : 0;
                            v = grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx];
                        }
                        zr += vy * v.x;
                        zi += vy * v.y;
                    }
                }
                ar += vz * zr;
                ai += vz * zi;
            }
            ar = group_sum<T, W>(ar * wx, dx);
            ai = group_sum<T, W>(ai * wx, dx);
            if (act && dx == 0) {
                C o;
                o.x = ar;
                o.y = ai;
                cout[a.perm[sub.y + q]] = o;
            }
        }
        if (STAGED) __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// GM interpolation: user order.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
interp_gm_kernel(KArgs<T> a)
{
    using C = typename cplx<T>::type;
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = a.M * a.ntransf;
    for (int64_t base = gwarp * G; base < total; base += nwarps_total * G) {
        const int64_t item = base + g;
        const bool act = gact && item < total;
        T wx = 0, wy = 0, wz = 0;
        int gx = 0, ly0 = 0, lz0 = 0, tr = 0;
        if (act) {
            tr = (int)(item / a.M);
            const int64_t j = item - (int64_t)tr * a.M;
            const AxisPos<T> px = axis_position<T>(period_fraction(a.xyz0[j]), a.n0, W);
            const AxisPos<T> py = axis_position<T>(period_fraction(a.xyz1[j]), a.n1, W);
            wx = es_kernel(((T)dx - px.delta) * a.hw, a.beta);
            wy = es_kernel(((T)dx - py.delta) * a.hw, a.beta);
            gx = wrap_any(px.l0 + dx, a.n0);
            ly0 = py.l0;
            if (DIM == 3) {
                const AxisPos<T> pz = axis_position<T>(period_fraction(a.xyz2[j]), a.n2, W);
                wz = es_kernel(((T)dx - pz.delta) * a.hw, a.beta);
                lz0 = pz.l0;
            }
        }
        const C *grid = a.grid + (int64_t)tr * a.nftot;
        T ar = 0, ai = 0;
        const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
        for (int iz = 0; iz < nz; ++iz) {
            T vz = (T)1;
            int gz = 0;
            if (DIM == 3) {
                vz = __shfl_sync(kFullMask, wz, src0 + iz);
                gz = wrap_any(lz0 + iz, a.n2);
            }
            T zr = 0, zi = 0;
#pragma unroll
            for (int iy = 0; iy < W; ++iy) {
                const T vy = __shfl_sync(kFullMask, wy, src0 + iy);
                if (act) {
                    const int gy = wrap_any(ly0 + iy, a.n1);
                    const C v = grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx];
                    zr += vy * v.x;
                    zi += vy * v.y;
                }
            }
            ar += vz * zr;
            ai += vz * zi;
        }
        ar = group_sum<T, W>(ar * wx, dx);
        ai = group_sum<T, W>(ai * wx, dx);
        if (act && dx == 0) {
            C o;
            o.x = ar;
            o.y = ai;
            a.cout[item] = o;
        }
    }
}

// ---------------------------------------------------------------------------
// Host-side launch for one (T, DIM): picks the kernel for p.method and p.w.
// ---------------------------------------------------------------------------
template <typename T>
KArgs<T> make_args(const Plan &p)
{
    KArgs<T> a;
    a.recs = reinterpret_cast<const typename rec4<T>::type *>(p.recs);
    a.perm = p.perm;
    a.subprob = p.subprob;
    a.nsub = p.nsub;
    a.xyz0 = reinterpret_cast<const T *>(p.xyz_copy[0]);
    a.xyz1 = reinterpret_cast<const T *>(p.xyz_copy[1]);
    a.xyz2 = reinterpret_cast<const T *>(p.xyz_copy[2]);
    a.grid = reinterpret_cast<typename cplx<T>::type *>(p.fine);
    a.cin = nullptr;
    a.cout = nullptr;
    a.M = p.M;
    a.nftot = p.nftot;
    a.ntransf = p.ntransf;
    a.n0 = (int)p.nf[0];
    a.n1 = (int)p.nf[1];
    a.n2 = (int)p.nf[2];
    a.m0 = p.m[0];
    a.m1 = p.m[1];
    a.m2 = p.m[2];
    a.nb0 = p.nb[0];
    a.nb1 = p.nb[1];
    const int P = (p.w + 1) / 2;
    a.p0 = p.m[0] + 2 * P;
    a.p1 = p.m[1] + 2 * P;
    a.p2 = p.dim == 3 ? p.m[2] + 2 * P : 1;
    a.beta = (T)p.beta;
    a.hw = (T)(2.0 / p.w);
    return a;
}

template <typename K>
inline int persistent_grid(const Plan &p, K kernel, int threads, size_t smem)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    if (p.ctas_per_sm > 0 && p.ctas_per_sm < per_sm) per_sm = p.ctas_per_sm;
    return p.num_sms * per_sm;
}

template <typename T, int DIM, int W>
cudaError_t spread_w(Plan &p, const void *c)
{
    KArgs<T> a = make_args<T>(p);
    a.cin = reinterpret_cast<const typename cplx<T>::type *>(c);
    const int threads = p.threads;
    if (p.method == NUFFT_METHOD_SM) {
        const size_t smem = (size_t)2 * sizeof(T) * a.p0 * a.p1 * a.p2;
        auto k = spread_sm_kernel<T, DIM, W>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = persistent_grid(p, k, threads, smem);
        count_launch();
        k<<<grid, threads, smem, p.stream>>>(a);
    } else if (p.method == NUFFT_METHOD_GM_SORT) {
        auto k = spread_gmsort_kernel<T, DIM, W>;
        count_launch();
        k<<<persistent_grid(p, k, threads, 0), threads, 0, p.stream>>>(a);
    } else {
        auto k = spread_gm_kernel<T, DIM, W>;
        const int64_t warps = (p.M * p.ntransf + (32 / W) - 1) / (32 / W);
        int64_t blocks = (warps * 32 + threads - 1) / threads;
        const int64_t cap = (int64_t)p.num_sms * 32;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        count_launch();
        k<<<(int)blocks, threads, 0, p.stream>>>(a);
    }
    return cudaGetLastError();
}

template <typename T, int DIM, int W>
cudaError_t interp_w(Plan &p, void *c)
{
    KArgs<T> a = make_args<T>(p);
    a.cout = reinterpret_cast<typename cplx<T>::type *>(c);
    const int threads = p.threads;
    if (p.method == NUFFT_METHOD_SM) {
        const size_t smem = sizeof(typename cplx<T>::type) * a.p0 * a.p1 * a.p2;
        auto k = interp_sorted_kernel<T, DIM, W, true>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        count_launch();
        k<<<persistent_grid(p, k, threads, smem), threads, smem, p.stream>>>(a);
    } else if (p.method == NUFFT_METHOD_GM_SORT) {
        auto k = interp_sorted_kernel<T, DIM, W, false>;
        count_launch();
        k<<<persistent_grid(p, k, threads, 0), threads, 0, p.stream>>>(a);
    } else {
        auto k = interp_gm_kernel<T, DIM, W>;
        const int64_t warps = (p.M * p.ntransf + (32 / W) - 1) / (32 / W);
        int64_t blocks = (warps * 32 + threads - 1) / threads;
        const int64_t cap = (int64_t)p.num_sms * 32;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        count_launch();
        k<<<(int)blocks, threads, 0, p.stream>>>(a);
    }
    return cudaGetLastError();
}

#define NUFFT_W_SWITCH(FN, T, DIM, ...)                                       \
    switch (p.w) {                                                            \
    case 2: return FN<T, DIM, 2>(__VA_ARGS__);                                \
    case 3: return FN<T, DIM, 3>(__VA_ARGS__);                                \
    case 4: return FN<T, DIM, 4>(__VA_ARGS__);                                \
    case 5: return FN<T, DIM, 5>(__VA_ARGS__);                                \
    case 6: return FN<T, DIM, 6>(__VA_ARGS__);                                \
    case 7: return FN<T, DIM, 7>(__VA_ARGS__);                                \
    case 8: return FN<T, DIM, 8>(__VA_ARGS__);                                \
    case 9: return FN<T, DIM, 9>(__VA_ARGS__);                                \
    case 10: return FN<T, DIM, 10>(__VA_ARGS__);                              \
    case 11: return FN<T, DIM, 11>(__VA_ARGS__);                              \
    case 12: return FN<T, DIM, 12>(__VA_ARGS__);                              \
    case 13: return FN<T, DIM, 13>(__VA_ARGS__);                              \
    case 14: return FN<T, DIM, 14>(__VA_ARGS__);                              \
    case 15: return FN<T, DIM, 15>(__VA_ARGS__);                              \
    case 16: return FN<T, DIM, 16>(__VA_ARGS__);                              \
    default: return cudaErrorInvalidValue;                                    \
    }

// One translation unit per (T, DIM) defines spread_<tag> and interp_<tag>.
#define NUFFT_INSTANTIATE_SI(T, DIM, TAG)                                     \
    cudaError_t spread_##TAG(Plan &p, const void *c)                          \
    {                                                                         \
        NUFFT_W_SWITCH(spread_w, T, DIM, p, c)                                \
    }                                                                         \
    cudaError_t interp_##TAG(Plan &p, void *c)                                \
    {                                                                         \
        NUFFT_W_SWITCH(interp_w, T, DIM, p, c)                                \
    }

}  // namespace nufft
