// spread_interp.cuh -- spreading (type 1 step 1, Sec. 3.1 / Sec. 4.1) and
// interpolation (type 2 step 3, Sec. 3.2 / Sec. 4.2) kernels, templated on the
// precision T, the dimension DIM and the kernel width W.
//
//   SM spreading   the row sweeps (spread_sweep2 / spread_sweep3): one warp per
//                  subproblem, lanes own the columns of the padded bin, the rows a
//                  window reaches are registers, finished rows are reduced into
//                  the fine grid -- no shared-memory atomics.  Bins too wide for 32
//                  lanes (and 3D double precision) use spread_sm_kernel: the padded
//                  bin in shared memory with shared atomics, then added to the fine
//                  grid (Sec. 4.1 SM steps 1-3).
//   GM-sort / GM   bin-ordered / user-order points, reductions straight into the
//                  fine grid; a warp is cut into G = 32 / W lane groups, group g
//                  works on one point, lane dx owns window column dx.
//   interpolation  one thread per point: the padded bin is staged in shared memory
//                  (SM; one warp per subproblem in 2D) or read from the fine grid
//                  (GM-sort), each lane sums its own point's W^d window; GM
//                  interpolation uses the lane groups.
// Kernel values come from kernel_row: piecewise polynomials for the interior
// window cells, the ES formula for the two edge cells.
#pragma once

#include "nufft_internal.cuh"

namespace nufft {

constexpr unsigned kFullMask = 0xffffffffu;

template <typename T>
struct alignas(16) KArgs {
    const typename rec4<T>::type *recs;          // packed records, in t order
    const int32_t *order;                        // t: sorted position -> point index
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
    int p0, p1, p2;                              // padded bin (m + w)
    T beta;
    T hw;                                        // 2 / w
    int poly;                                    // use coef for interior cells
    T coef[kMaxW][kPolyTerms];                   // kernel polynomials (Plan::poly)
};

template <typename T> __device__ __forceinline__ uint32_t unpack_word(T v);
template <> __device__ __forceinline__ uint32_t unpack_word<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ uint32_t unpack_word<double>(double v)
{
    return (uint32_t)__double_as_longlong(v);
}

// Original index of the point at execution position pos with record r: in 2D
// the record's z slot, in 3D the order array.
template <typename T, int DIM>
__device__ __forceinline__ int point_of(const KArgs<T> &a, const typename rec4<T>::type &r,
                                        int64_t pos)
{
    return DIM == 2 ? (int)unpack_word<T>(r.z) : a.order[pos];
}

// Packed single-precision pairs: the f32x2 arithmetic of sm_100-class GPUs
// (one instruction for both halves of a float2), through the compiler's
// builtins so that it allocates the register pairs itself.
// acc += a * b, half by half
__device__ __forceinline__ void fma2(float2 &acc, float2 a, float2 b) { acc = __ffma2_rn(a, b, acc); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

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
    const int bx = b % nb0;
    const int r = b / nb0;
    const int by = r % nb1;
    const int bz = r / nb1;
    o0 = bx * m0;
    o1 = by * m1;
    o2 = bz * m2;
}

// Shuffle helpers for the batch hand-off.
__device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(kFullMask, v, src); }
__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(kFullMask, v, src); }

// One point of a 32-point batch, as seen by its lane group.
template <typename T>
struct PointView {
    T dx, dy, dz;      // kernel offsets delta
    uint32_t pk;       // packed window start in the padded bin
    T cr, ci;          // strength (spread only)
};

template <typename T, bool WITH_C>
__device__ __forceinline__ PointView<T> take_point(const typename rec4<T>::type &r,
                                                   const typename cplx<T>::type &cv, int src)
{
    PointView<T> v;
    v.dx = shfl(r.x, src);
    v.dy = shfl(r.y, src);
    v.dz = shfl(r.z, src);
    v.pk = __shfl_sync(kFullMask, unpack_word<T>(r.w), src);
    if (WITH_C) {
        v.cr = shfl(cv.x, src);
        v.ci = shfl(cv.y, src);
    } else {
        v.cr = v.ci = (T)0;
    }
    return v;
}

// ---------------------------------------------------------------------------
// SM spreading.  One work item = one (subproblem, transform) pair, run by the
// whole CTA; the single-plan kernel and the multi-plan (batched) kernel below
// both stride over work items.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__device__ __forceinline__ void spread_sm_item(const KArgs<T> &a, int sp, int tr, T *sre)
{
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    constexpr int G = 32 / W;
    const int ptot = a.p0 * a.p1 * (DIM == 3 ? a.p2 : 1);
    const int p01 = a.p0 * a.p1;
    T *sim = sre + ptot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int P = pad_lo(W);
    {
        const int4 sub = a.subprob[sp];
        for (int i = threadIdx.x; i < 2 * ptot; i += blockDim.x) sre[i] = (T)0;
        __syncthreads();
        const C *cin = a.cin + (int64_t)tr * a.M;
        for (int base = warp * 32; base < sub.z; base += nwarps * 32) {
            R r;
            r.x = r.y = r.z = r.w = (T)0;
            C cv;
            cv.x = cv.y = (T)0;
            if (base + lane < sub.z) {
                const int64_t pos = sub.y + base + lane;
                r = a.recs[pos];
                cv = cin[point_of<T, DIM>(a, r, pos)];
            }
            const int np = min(32, sub.z - base);
            for (int i0 = 0; i0 < np; i0 += G) {
                const int p = i0 + g;
                const bool act = gact && p < np;
                const PointView<T> pv = take_point<T, true>(r, cv, p < 32 ? p : 31);
                const T wx = es_kernel(((T)dx - pv.dx) * a.hw, a.beta);
                const T myy = es_kernel(((T)dx - pv.dy) * a.hw, a.beta);
                const T myz = DIM == 3 ? es_kernel(((T)dx - pv.dz) * a.hw, a.beta) : (T)0;
                T wy[W];
#pragma unroll
                for (int i = 0; i < W; ++i) wy[i] = shfl(myy, src0 + i);
                const int sx = pv.pk & 1023u, sy = (pv.pk >> 10) & 1023u, sz = pv.pk >> 20;
                const T zr0 = pv.cr * wx, zi0 = pv.ci * wx;
                const int baddr = (sz * a.p1 + sy) * a.p0 + sx + dx;
                const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
                for (int iz = 0; iz < nz; ++iz) {
                    const T vz = DIM == 3 ? shfl(myz, src0 + iz) : (T)1;
                    const T zr = zr0 * vz, zi = zi0 * vz;
                    int addr = baddr + iz * p01;
#pragma unroll
                    for (int iy = 0; iy < W; ++iy) {
                        if (act) {
                            atomicAdd(&sre[addr], wy[iy] * zr);
                            atomicAdd(&sim[addr], wy[iy] * zi);
                        }
                        addr += a.p0;
                    }
                }
            }
        }
        __syncthreads();
        // Step 3: accumulate the padded bin into the fine grid, l = (s + Delta) mod n.
        int o0, o1, o2;
        bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
        C *grid = a.grid + (int64_t)tr * a.nftot;
        const int rows = a.p1 * (DIM == 3 ? a.p2 : 1);
        for (int rr = warp; rr < rows; rr += nwarps) {
            const int ry = rr % a.p1, rz = rr / a.p1;
            const int gy = wrap_any(o1 - P + ry, a.n1);
            const int gz = DIM == 3 ? wrap_any(o2 - P + rz, a.n2) : 0;
            const int64_t rowbase = ((int64_t)gz * a.n1 + gy) * a.n0;
            for (int rx = lane; rx < a.p0; rx += 32) {
                const T re = sre[rr * a.p0 + rx], im = sim[rr * a.p0 + rx];
                if (re != (T)0 || im != (T)0)
                    atomic_add_cplx(&grid[rowbase + wrap_any(o0 - P + rx, a.n0)], re, im);
            }
        }
        __syncthreads();
    }
}

template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_sm_kernel(KArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sre = reinterpret_cast<T *>(smem_raw);
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x)
        spread_sm_item<T, DIM, W>(a, (int)(wi % nsp), (int)(wi / nsp), sre);
}

// Plan of global work item wi in a batch: workoff[p] <= wi < workoff[p + 1].
__device__ __forceinline__ int batch_plan_of(const int64_t *workoff, int nplans, int64_t wi)
{
    int lo = 0, hi = nplans - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (workoff[mid] <= wi) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_sm_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                       int nplans)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sre = reinterpret_cast<T *>(smem_raw);
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        const KArgs<T> &a = args[pl];
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        spread_sm_item<T, DIM, W>(a, (int)(local % nsp), (int)(local / nsp), sre);
    }
}

// ---------------------------------------------------------------------------
// Row-sweep SM spreading, 2D (Sec. 4.1 SM with the accumulation moved from
// shared-memory atomics into registers).  One warp per work item, cut into
// S = 32 / L sub-warps of L lanes; lane q of every sub-warp owns column q of the
// padded bin (p0 = m0 + W <= L) and holds, in registers, the W rows that a
// window starting at the current row can reach.
//
//  1. The subproblem's records (one contiguous run in t order) are ordered by
//     the first row of their window: a stable counting sort in shared memory
//     (warp-aggregated integer atomics), whose counters then mark where each
//     start row's points end; the records are read in that order, 32 at a
//     time, with the strengths c gathered by index.
//  2. Lane i evaluates point i's 2W kernel values and stores w_y and c w_x in a
//     staging slot.  The W window rows live in register slots indexed by row
//     mod W; w_y is stored rotated the same way.
//  3. The warp walks the padded rows in blocks of W (row rb + k in slot k, a
//     compile-time index): the points starting at the row are dealt to the
//     sub-warps -- every lane adds (c w_x[q - s_x]) w_y to its W slots, a plain
//     register update, since within a sub-warp no two lanes own the same cell;
//     in single precision one f32x2 FMA per slot -- and then the row is
//     complete: the sub-warps' copies are summed by shuffles, added to the
//     fine grid (periodic wrap) and the slot cleared.
//
// Shared memory per warp (sweep_bytes): the sorted positions, the row counters
// and 32 staging slots.
// ---------------------------------------------------------------------------
// Staging slots are built from 16-byte quads (4 floats or 2 doubles), with an
// odd quad count so that the 8 lanes of a quarter-warp storing their slots with
// 128-bit stores hit 8 different bank quads.
template <typename T> __host__ __device__ constexpr int quad_vec() { return 16 / (int)sizeof(T); }
template <typename T, int W> __host__ __device__ constexpr int quad_row()
{
    return (W + quad_vec<T>() - 1) / quad_vec<T>();
}
// 2D slot: the W row weights (single precision: W duplicated pairs (w_y, w_y),
// (W + 1) / 2 quads; double: W values), then c w_x scattered into an L-wide
// complex row (zeros outside the window), so lane q reads entry q at a fixed
// address.
template <typename T, int W> __host__ __device__ constexpr int sweep2_wy_quads()
{
    return sizeof(T) == 4 ? (W + 1) / 2 : quad_row<T, W>();
}
template <typename T, int W, int L> __host__ __device__ constexpr int sweep2_slot()
{
    return ((sweep2_wy_quads<T, W>() + 2 * L * (int)sizeof(T) / 16) | 1) * quad_vec<T>();
}
// 3D slot (single precision): w_y and w_z as duplicated pairs ((W + 1) / 2
// quads each), then the L-wide c w_x row.
template <typename T, int W, int L> __host__ __device__ constexpr int sweep3_slot()
{
    return ((2 * ((W + 1) / 2) + 2 * L / quad_vec<T>()) | 1) * quad_vec<T>();
}

__device__ __forceinline__ void store_zero_quad(float *dst)
{
    *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void store_zero_quad(double *dst)
{
    *reinterpret_cast<double2 *>(dst) = make_double2(0.0, 0.0);
}

// Stores a W-value row as quad_row<T, W>() 16-byte quads, zero-padded.
template <int W>
__device__ __forceinline__ void store_row(float *dst, const float (&v)[W])
{
#pragma unroll
    for (int k = 0; k < W; k += 4) {
        float4 t;
        t.x = v[k];
        t.y = k + 1 < W ? v[k + 1 < W ? k + 1 : k] : 0.f;
        t.z = k + 2 < W ? v[k + 2 < W ? k + 2 : k] : 0.f;
        t.w = k + 3 < W ? v[k + 3 < W ? k + 3 : k] : 0.f;
        *reinterpret_cast<float4 *>(dst + k) = t;
    }
}
template <int W>
__device__ __forceinline__ void store_row(double *dst, const double (&v)[W])
{
#pragma unroll
    for (int k = 0; k < W; k += 2) {
        double2 t;
        t.x = v[k];
        t.y = k + 1 < W ? v[k + 1 < W ? k + 1 : k] : 0.0;
        *reinterpret_cast<double2 *>(dst + k) = t;
    }
}
// Stores the W values as duplicated pairs (v, v), two pairs per quad.
template <int W>
__device__ __forceinline__ void store_dup_row(float *dst, const float (&v)[W])
{
#pragma unroll
    for (int k = 0; k < W; k += 2) {
        const float b = k + 1 < W ? v[k + 1 < W ? k + 1 : k] : 0.f;
        *reinterpret_cast<float4 *>(dst + 2 * k) = make_float4(v[k], v[k], b, b);
    }
}

// The row sweeps order a subproblem's points by window start row themselves,
// in pieces of at most kSweepCap points (each piece swept on its own): warp
// shared memory holds the piece's sorted positions (u16), the key counters and
// the 32 staging slots.
constexpr int kSweepCap = 1024;

__host__ __device__ inline size_t sweep_head(int nkeys)
{
    return ((size_t)2 * kSweepCap + (size_t)4 * (nkeys + 1) + 15) & ~(size_t)15;
}

template <typename T, int W, int L>
__host__ __device__ inline size_t sweep_bytes(int m1)
{
    return sweep_head(m1 + 1) + sizeof(T) * (size_t)32 * sweep2_slot<T, W, L>();
}

// Stable counting sort (one warp) of the n records of a piece by key_of(record
// packed word) in [0, nkeys): idx[] receives the positions grouped by key,
// increasing inside a key; afterwards cnt[k] is the end of key k's run.  cnt[]
// holds nkeys + 1 ints.  The packed words are read from the records (coalesced).
template <typename T, typename KeyOf>
__device__ __forceinline__ void warp_sort_records(const typename rec4<T>::type *recs, int n,
                                                  int nkeys, uint16_t *idx, int *cnt, KeyOf key_of)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = lane; i <= nkeys; i += 32) cnt[i] = 0;
    __syncwarp();
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const int key = i < n ? key_of(unpack_word<T>(recs[i].w)) : 0x7fffffff;
        const unsigned peers = __match_any_sync(kFullMask, key);
        if (i < n && (peers & lt) == 0) atomicAdd(&cnt[key + 1], __popc(peers));
    }
    __syncwarp();
    int running = 0;
    for (int i0 = 0; i0 <= nkeys; i0 += 32) {
        const int i = i0 + lane;
        int v = i <= nkeys ? cnt[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFullMask, v, o);
            if (lane >= o) v += t;
        }
        if (i <= nkeys) cnt[i] = running + v;
        running += __shfl_sync(kFullMask, v, 31);
    }
    __syncwarp();
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const int key = i < n ? key_of(unpack_word<T>(recs[i].w)) : 0x7fffffff;
        const unsigned peers = __match_any_sync(kFullMask, key);
        const int leader = __ffs(peers) - 1;
        int pos = 0;
        if (i < n && lane == leader) pos = atomicAdd(&cnt[key], __popc(peers));
        pos = __shfl_sync(kFullMask, pos, leader);
        if (i < n) idx[pos + __popc(peers & lt)] = (uint16_t)i;
    }
    __syncwarp();
}

// By window start row (ZMUL = 0) or row * ZMUL + start plane (3D).
template <typename T, int ZMUL>
__device__ __forceinline__ void sweep_row_order(const typename rec4<T>::type *recs, int n,
                                                int nkeys, uint16_t *idx, int *cnt)
{
    warp_sort_records<T>(recs, n, nkeys, idx, cnt, [](uint32_t pk) {
        const int row = (int)((pk >> 10) & 1023u);
        return ZMUL == 0 ? row : row * ZMUL + (int)(pk >> 20);
    });
}

// Single-precision ES kernel for the staging step, written without the
// cancellation of sqrt(1 - z^2) - 1 near z = 0:
//   beta (sqrt(1 - z^2) - 1) = -beta z^2 / (1 + sqrt(1 - z^2)),
// so the hardware reciprocal square root, reciprocal and fast exponential
// (each ~1e-7 relative) give phi to ~1e-7 relative everywhere.  Double keeps
// the correctly rounded es_kernel.
__device__ __forceinline__ float es_kernel_stage(float z, float beta)
{
    const float z2 = z * z;
    const float s = 1.0f - z2;
    const float r = s > 0.0f ? s * rsqrtf(s) : 0.0f;
    return s >= 0.0f ? __expf(__fdividef(-beta * z2, 1.0f + r)) : 0.0f;
}
__device__ __forceinline__ double es_kernel_stage(double z, double beta)
{
    return es_kernel(z, beta);
}

// The W kernel weights phi((i - delta) 2 / W), i < W, of one axis: interior
// cells by Horner's rule on the plan's polynomials (constant-bank operands),
// the two edge cells -- where sqrt(1 - z^2) is not smooth -- directly.
template <typename T, int W>
__device__ __forceinline__ void kernel_row(const KArgs<T> &a, T delta, T (&v)[W])
{
    constexpr int D = poly_degree(W, sizeof(T) == 4 ? 0 : 1);
    if (a.poly) {
        const T s = (T)2 * (delta - (T)(0.5 * W - 1)) - (T)1;
#pragma unroll
        for (int i = 1; i + 1 < W; ++i) {
            T acc = a.coef[i][D];
#pragma unroll
            for (int d = D - 1; d >= 0; --d) acc = acc * s + a.coef[i][d];
            v[i] = acc;
        }
        v[0] = es_kernel_stage(((T)0 - delta) * a.hw, a.beta);
        v[W - 1] = es_kernel_stage(((T)(W - 1) - delta) * a.hw, a.beta);
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) v[i] = es_kernel_stage(((T)i - delta) * a.hw, a.beta);
    }
}

// One weight phi((i - delta) 2 / W) with a run-time cell index.
template <typename T, int W>
__device__ __forceinline__ T kernel_cell(const KArgs<T> &a, T delta, int i)
{
    constexpr int D = poly_degree(W, sizeof(T) == 4 ? 0 : 1);
    if (a.poly && i > 0 && i < W - 1) {
        const T s = (T)2 * (delta - (T)(0.5 * W - 1)) - (T)1;
        T acc = a.coef[i][D];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) acc = acc * s + a.coef[i][d];
        return acc;
    }
    return es_kernel_stage(((T)i - delta) * a.hw, a.beta);
}

// A W-value row stored by store_row: whole 16-byte quads (the padding is read
// and dropped).
template <int W>
__device__ __forceinline__ void load_row(const float *s, float (&v)[W])
{
#pragma unroll
    for (int k = 0; k < W; k += 4) {
        const float4 t = *reinterpret_cast<const float4 *>(s + k);
        v[k] = t.x;
        if (k + 1 < W) v[k + 1 < W ? k + 1 : k] = t.y;
        if (k + 2 < W) v[k + 2 < W ? k + 2 : k] = t.z;
        if (k + 3 < W) v[k + 3 < W ? k + 3 : k] = t.w;
    }
}
template <int W>
__device__ __forceinline__ void load_row(const double *s, double (&v)[W])
{
#pragma unroll
    for (int k = 0; k < W; k += 2) {
        const double2 t = *reinterpret_cast<const double2 *>(s + k);
        v[k] = t.x;
        if (k + 1 < W) v[k + 1 < W ? k + 1 : k] = t.y;
    }
}

template <typename T, int W, int L>
__device__ __forceinline__ void spread_sweep2_sub(const KArgs<T> &a, int4 sub, int tr,
                                                  unsigned char *sm)
{
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int S = 32 / L;
    constexpr int SLOT = sweep2_slot<T, W, L>();
    constexpr int OCX = sweep2_wy_quads<T, W>() * quad_vec<T>();
    const int lane = threadIdx.x & 31, h = lane / L, q = lane % L;
    const int n = sub.z;
    uint16_t *idx = reinterpret_cast<uint16_t *>(sm);
    int *cnt = reinterpret_cast<int *>(sm + 2 * kSweepCap);
    T *stg = reinterpret_cast<T *>(sm + sweep_head(a.m1 + 1));
    int o0, o1, o2;
    bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
    const int P = pad_lo(W);
    const C *cin = a.cin + (int64_t)tr * a.M;
    C *grid = a.grid + (int64_t)tr * a.nftot;
    const bool writer = h == 0 && q < a.p0;
    const int gx = wrap_any(o0 - P + (q < a.p0 ? q : 0), a.n0);
    const int grow0 = wrap_any(o1 - P, a.n1);            // fine-grid row of padded row 0
    // Window slot s holds the padded row r with r mod W = s: (re, im) as a float2
    // (single) or accr / acci (double).  A staged point's w_y is stored rotated
    // the same way, so every update touches the slots in a fixed order.
    float2 accp[F32 ? W : 1];
    T accr[F32 ? 1 : W], acci[F32 ? 1 : W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        if constexpr (F32) accp[k] = make_float2(0.f, 0.f);
        else accr[k] = acci[k] = (T)0;
    }
    // add slot k to fine-grid row g (sub-warp copies summed by shuffles) and clear it
    auto flush = [&](int k, int g) {
        T vr, vi;
        if constexpr (F32) {
            vr = accp[k < W ? k : 0].x;
            vi = accp[k < W ? k : 0].y;
            accp[k < W ? k : 0] = make_float2(0.f, 0.f);
        } else {
            vr = accr[k < W ? k : 0];
            vi = acci[k < W ? k : 0];
            accr[k < W ? k : 0] = acci[k < W ? k : 0] = (T)0;
        }
#pragma unroll
        for (int o = L; o < 32; o <<= 1) {
            vr += __shfl_xor_sync(kFullMask, vr, o);
            vi += __shfl_xor_sync(kFullMask, vi, o);
        }
        if (writer && (vr != (T)0 || vi != (T)0))
            atomic_add_cplx(&grid[(int64_t)g * a.n0 + gx], vr, vi);
    };
    // one staged point: lane q adds (c w_x)[q] w_y to the W window rows
    auto step = [&](int i) {
        const T *s = stg + i * SLOT;
        if constexpr (F32) {
            const float2 cx = *reinterpret_cast<const float2 *>(s + OCX + 2 * q);
#pragma unroll
            for (int k = 0; k < W; k += 2) {
                const float4 wp = *reinterpret_cast<const float4 *>(s + 2 * k);
                fma2(accp[k], cx, make_float2(wp.x, wp.y));
                if (k + 1 < W) fma2(accp[k + 1 < W ? k + 1 : k], cx, make_float2(wp.z, wp.w));
            }
        } else {
            const C cx = *reinterpret_cast<const C *>(s + OCX + 2 * q);
            T wy[W];
            load_row<W>(s, wy);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                accr[k] += cx.x * wy[k];
                acci[k] += cx.y * wy[k];
            }
        }
    };

    const R *recs = a.recs + sub.y;
    for (int piece = 0; piece < n; piece += kSweepCap) {
        const int np = min(kSweepCap, n - piece);
        // points by window start row; afterwards cnt[r] = end of start row r
        sweep_row_order<T, 0>(recs + piece, np, a.m1 + 1, idx, cnt);
        R rc;
        C cv;
        if (lane < np) {
            rc = recs[piece + idx[lane]];
            cv = cin[unpack_word<T>(rc.z)];
        }
        int bbase = -32, bend = 0;                         // staged positions [bbase, bend)
        auto stage_next = [&]() {
            __syncwarp();                                  // the old slots are consumed
            bbase += 32;
            const int c = min(32, np - bbase);
            if (lane < c) {
                const uint32_t pk = unpack_word<T>(rc.w);
                T *s = stg + lane * SLOT;
                const int sy = (int)((pk >> 10) & 1023u);
                const int sx = (int)(pk & 1023u);
                T vx[W], vy[W];
                kernel_row<T, W>(a, rc.x, vx);
                kernel_row<T, W>(a, rc.y, vy);
#pragma unroll
                for (int k = 0; k < 2 * L; k += quad_vec<T>()) store_zero_quad(s + OCX + k);
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    C v;
                    v.x = cv.x * vx[i];
                    v.y = cv.y * vx[i];
                    *reinterpret_cast<C *>(s + OCX + 2 * (sx + i)) = v;
                }
                int slot = sy % W;                         // w_y[k] goes to slot (sy + k) mod W
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    if constexpr (F32)
                        *reinterpret_cast<float2 *>(s + 2 * slot) = make_float2(vy[k], vy[k]);
                    else
                        s[slot] = vy[k];
                    slot = slot + 1 == W ? 0 : slot + 1;
                }
            }
            const int nb = bbase + 32;                     // prefetch the next batch
            if (nb + lane < np) {
                rc = recs[piece + idx[nb + lane]];
                cv = cin[unpack_word<T>(rc.z)];
            }
            bend = bbase + c;
            __syncwarp();
        };
        // Walk the padded rows in blocks of W, so that row r = rb + k lives in the
        // static slot k: process the points starting at r, then r is complete.
        int pos = 0;
        int g = grow0;
        int k = 0;                                         // slot of row r = r mod W
#pragma unroll 1
        for (int r = 0; r < a.p1; ++r) {
            const int end = r <= a.m1 ? cnt[r] : pos;
            while (pos < end) {
                if (pos == bend) stage_next();
                const int e = min(end, bend);
                const int ie = e - bbase;
                int i = pos - bbase + h;
                for (; i + S < ie; i += 2 * S) {
                    step(i);
                    step(i + S);
                }
                if (i < ie) step(i);
                pos = e;
            }
#pragma unroll
            for (int kk = 0; kk < W; ++kk)                 // row r is complete: flush slot k
                if (kk == k) flush(kk, g);
            g = g + 1 == a.n1 ? 0 : g + 1;
            k = k + 1 == W ? 0 : k + 1;
        }
        __syncwarp();                                      // idx / cnt reused by the next piece
    }
}

// ---------------------------------------------------------------------------
// Row-sweep SM spreading, 3D (single precision, W <= 8, bins m2 = M2 in {1, 2}).
// As the 2D sweep: S = 32 / L sub-warps, lane q owns x column q of the padded
// bin (p0 <= L) and holds the W y rows in reach times all M2 + W z planes in
// registers.  The points are ordered by (window start row, start plane) as in
// 2D; the points of one (row, plane) group are dealt to the sub-warps, so the first
// plane s_z is the same for the whole warp and selects one of M2 + 1 unrolled
// updates  acc[j][s_z + k] += (c w_x[q - s_x] w_y[j]) w_z[k],  j, k < W.
// A finished row is summed over the sub-warps and added to the fine grid plane
// by plane.
// ---------------------------------------------------------------------------
template <typename T, int W, int M2, int L>
__host__ __device__ inline size_t sweep3_bytes(int m1)
{
    return sweep_head((m1 + 1) * (M2 + 1)) + sizeof(T) * (size_t)32 * sweep3_slot<T, W, L>();
}

// acc[j][O + k] += tu[j] * wzz[k], (re, im) pairs
template <int W, int PZ, int O>
__device__ __forceinline__ void sweep3_add(float2 (&acc)[W][PZ], const float2 (&tu)[W],
                                           const float2 (&wzz)[W])
{
#pragma unroll
    for (int j = 0; j < W; ++j) {
#pragma unroll
        for (int k = 0; k < W; ++k) fma2(acc[j][O + k], tu[j], wzz[k]);
    }
}

template <typename T, int W, int M2, int L>
__device__ __forceinline__ void spread_sweep3_sub(const KArgs<T> &a, int4 sub, int tr,
                                                  unsigned char *sm)
{
    static_assert(sizeof(T) == 4, "the 3D row sweep is single precision");
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    constexpr int S = 32 / L;
    constexpr int PZ = M2 + W;
    constexpr int SLOT = sweep3_slot<T, W, L>();
    constexpr int OWY = 0, OWZ = 4 * ((W + 1) / 2), OCX = 2 * OWZ;
    const int lane = threadIdx.x & 31, h = lane / L, q = lane % L;
    const int n = sub.z;
    const int nkeys = (a.m1 + 1) * (M2 + 1);
    uint16_t *idx = reinterpret_cast<uint16_t *>(sm);
    int *cnt = reinterpret_cast<int *>(sm + 2 * kSweepCap);
    T *stg = reinterpret_cast<T *>(sm + sweep_head(nkeys));

    int o0, o1, o2;
    bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
    const int P = pad_lo(W);
    const C *cin = a.cin + (int64_t)tr * a.M;
    C *grid = a.grid + (int64_t)tr * a.nftot;
    const bool writer = h == 0 && q < a.p0;
    const int gx = wrap_any(o0 - P + (q < a.p0 ? q : 0), a.n0);
    const int row0 = o1 - P, plane0 = o2 - P;
    float2 acc[W][PZ];                                     // (re, im) of row j, plane k
#pragma unroll
    for (int j = 0; j < W; ++j)
#pragma unroll
        for (int k = 0; k < PZ; ++k) acc[j][k] = make_float2(0.f, 0.f);
    int row = 0;

    auto flush_row = [&](int r_rel, const float2 (&v)[PZ]) {
        float vr[PZ], vi[PZ];
#pragma unroll
        for (int k = 0; k < PZ; ++k) {
            vr[k] = v[k].x;
            vi[k] = v[k].y;
#pragma unroll
            for (int o = L; o < 32; o <<= 1) {
                vr[k] += __shfl_xor_sync(kFullMask, vr[k], o);
                vi[k] += __shfl_xor_sync(kFullMask, vi[k], o);
            }
        }
        if (!writer) return;
        const int gy = wrap_any(row0 + r_rel, a.n1);
#pragma unroll
        for (int k = 0; k < PZ; ++k) {
            if (vr[k] != 0.f || vi[k] != 0.f) {
                const int gz = wrap_any(plane0 + k, a.n2);
                atomic_add_cplx(&grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx], vr[k], vi[k]);
            }
        }
    };

    R rc;
    C cv;
    int piece = 0, np = 0;
    auto fetch = [&](int base) {
        if (base + lane < np) {
            const int64_t pos = sub.y + piece + idx[base + lane];
            rc = a.recs[pos];
            cv = cin[a.order[pos]];
        }
    };
    for (piece = 0; piece < n; piece += kSweepCap) {
    np = min(kSweepCap, n - piece);
    sweep_row_order<T, M2 + 1>(a.recs + sub.y + piece, np, nkeys, idx, cnt);
    fetch(0);
    for (int base = 0; base < np; base += 32) {
        const int cnt = min(32, np - base);
        int mykey = 0x7fffffff;
        if (lane < cnt) {
            const uint32_t pk = unpack_word<T>(rc.w);
            T *s = stg + lane * SLOT;
            mykey = (int)((pk >> 10) & 1023u) * (M2 + 1) + (int)(pk >> 20);
            const int sx = (int)(pk & 1023u);
            T vx[W], vy[W], vz[W];
            kernel_row<T, W>(a, rc.x, vx);
            kernel_row<T, W>(a, rc.y, vy);
            kernel_row<T, W>(a, rc.z, vz);
#pragma unroll
            for (int k = 0; k < 2 * L; k += quad_vec<T>()) store_zero_quad(s + OCX + k);
#pragma unroll
            for (int i = 0; i < W; ++i) {
                C v;
                v.x = cv.x * vx[i];
                v.y = cv.y * vx[i];
                *reinterpret_cast<C *>(s + OCX + 2 * (sx + i)) = v;
            }
            store_dup_row<W>(s + OWY, vy);
            store_dup_row<W>(s + OWZ, vz);
        }
        if (base == 0 && piece == 0) row = __shfl_sync(kFullMask, mykey, 0) / (M2 + 1);
        fetch(base + 32);
        __syncwarp();
        int i0 = 0;
        while (i0 < cnt) {
            const int r = __shfl_sync(kFullMask, mykey, i0);
            const int rrow = r / (M2 + 1);
            if (rrow < row || rrow >= row + W) {      // new ordering piece, or a jump
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    flush_row(row + j, acc[j]);
#pragma unroll
                    for (int k = 0; k < PZ; ++k) acc[j][k] = make_float2(0.f, 0.f);
                }
                row = rrow;
            }
            while (row < rrow) {
                flush_row(row, acc[0]);
#pragma unroll
                for (int j = 0; j + 1 < W; ++j)
#pragma unroll
                    for (int k = 0; k < PZ; ++k) acc[j][k] = acc[j + 1][k];
#pragma unroll
                for (int k = 0; k < PZ; ++k) acc[W - 1][k] = make_float2(0.f, 0.f);
                ++row;
            }
            const unsigned later = __ballot_sync(kFullMask, mykey != r) & ~((2u << i0) - 1u);
            const int i1 = later ? __ffs(later) - 1 : cnt;
            const int sz = r - rrow * (M2 + 1);             // the group's first plane
            for (int i = i0 + h; i < i1; i += S) {
                const T *s = stg + i * SLOT;
                const float2 cx = *reinterpret_cast<const float2 *>(s + OCX + 2 * q);
                float2 tu[W], wzz[W];
#pragma unroll
                for (int k = 0; k < W; k += 2) {
                    const float4 y2 = *reinterpret_cast<const float4 *>(s + OWY + 2 * k);
                    const float4 z2 = *reinterpret_cast<const float4 *>(s + OWZ + 2 * k);
                    tu[k] = mul2(cx, make_float2(y2.x, y2.y));
                    wzz[k] = make_float2(z2.x, z2.y);
                    if (k + 1 < W) {
                        tu[k + 1 < W ? k + 1 : k] = mul2(cx, make_float2(y2.z, y2.w));
                        wzz[k + 1 < W ? k + 1 : k] = make_float2(z2.z, z2.w);
                    }
                }
                if (sz == 0)
                    sweep3_add<W, PZ, 0>(acc, tu, wzz);
                else if (M2 == 1 || sz == 1)
                    sweep3_add<W, PZ, 1>(acc, tu, wzz);
                else
                    sweep3_add<W, PZ, (M2 >= 2 ? 2 : 1)>(acc, tu, wzz);
            }
            i0 = i1;
        }
        __syncwarp();
    }
    }
#pragma unroll
    for (int j = 0; j < W; ++j) flush_row(row + j, acc[j]);
}

// ---------------------------------------------------------------------------
// Plane-split row sweep, 3D (single precision, padded width p0 <= 16, W <= 8).
// The warp is two halves of 16 lanes; lane (h, q) owns x column q of the padded
// bin and the KZ = (M2 + W + 1) / 2 planes h KZ .. h KZ + KZ - 1, each with its
// W window rows in registers (slot s = padded row mod W, as in 2D).  Every lane
// takes part in every point: the point's c w_x row (zero outside the window)
// and its z weights (zero outside the window) are staged, so the update
//   acc[i][s] += (c w_x[q] w_z[h KZ + i]) w_y[s],  i < KZ, s < W
// has no branch on the point's start plane.  The two halves hold different
// planes, so a finished row goes to the fine grid without any reduction: each
// lane adds its KZ cells of that row.  Points are ordered by window start row
// only (Sec. 4.1 SM step 2 with the subproblem's accumulators in registers).
template <int W, int M2> __host__ __device__ constexpr int planes3_kz() { return (M2 + W + 1) / 2; }
// slot: W rotated w_y dup pairs, 2 KZ w_z dup pairs, the 16-wide c w_x row
template <int W, int M2> __host__ __device__ constexpr int planes3_owz() { return 4 * ((W + 1) / 2); }
template <int W, int M2> __host__ __device__ constexpr int planes3_ocx()
{
    return planes3_owz<W, M2>() + 4 * planes3_kz<W, M2>();
}
template <int W, int M2> __host__ __device__ constexpr int planes3_slot()
{
    return ((planes3_ocx<W, M2>() + 32) / 4 | 1) * 4;
}
template <int W, int M2>
__host__ __device__ inline size_t planes3_bytes(int m1)
{
    (void)m1;
    return sizeof(float) * (size_t)32 * planes3_slot<W, M2>();
}

template <typename T, int W, int M2>
__device__ __forceinline__ void spread_planes3_sub(const KArgs<T> &a, int4 sub, int tr,
                                                   unsigned char *sm)
{
    static_assert(sizeof(T) == 4, "the 3D row sweep is single precision");
    using C = float2;
    using R = typename rec4<T>::type;
    constexpr int KZ = planes3_kz<W, M2>();
    constexpr int PZ = M2 + W;
    constexpr int SLOT = planes3_slot<W, M2>();
    constexpr int OWZ = planes3_owz<W, M2>(), OCX = planes3_ocx<W, M2>();
    const int lane = threadIdx.x & 31, h = lane >> 4, q = lane & 15;
    const int n = sub.z;
    float *stg = reinterpret_cast<float *>(sm);
    int o0, o1, o2;
    bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
    const int P = pad_lo(W);
    const C *cin = a.cin + (int64_t)tr * a.M;
    const bool xok = q < a.p0;
    const int gx = wrap_any(o0 - P + (xok ? q : 0), a.n0);
    const int grow0 = wrap_any(o1 - P, a.n1);
    C *grid = a.grid + (int64_t)tr * a.nftot + gx;
    int gz[KZ];                                            // fine-grid plane of each owned plane
#pragma unroll
    for (int i = 0; i < KZ; ++i)
        gz[i] = xok && h * KZ + i < PZ ? wrap_any(o2 - P + h * KZ + i, a.n2) : -1;
    float2 acc[KZ][W];
#pragma unroll
    for (int i = 0; i < KZ; ++i)
#pragma unroll
        for (int k = 0; k < W; ++k) acc[i][k] = make_float2(0.f, 0.f);
    // add window slot k of every owned plane to fine-grid row g and clear it
    auto flush = [&](int k, int g) {
#pragma unroll
        for (int i = 0; i < KZ; ++i) {
            const float2 v = acc[i][k < W ? k : 0];
            acc[i][k < W ? k : 0] = make_float2(0.f, 0.f);
            if (gz[i] >= 0 && (v.x != 0.f || v.y != 0.f))
                atomic_add_cplx(grid + ((int64_t)gz[i] * a.n1 + g) * a.n0, v.x, v.y);
        }
    };
    auto step = [&](int i) {
        const float *s = stg + i * SLOT;
        const float2 cx = *reinterpret_cast<const float2 *>(s + OCX + 2 * q);
        float2 t[KZ];
        if constexpr (KZ % 2 == 0) {
#pragma unroll
            for (int j = 0; j < KZ; j += 2) {
                const float4 z2 = *reinterpret_cast<const float4 *>(s + OWZ + 2 * (h * KZ + j));
                t[j] = mul2(cx, make_float2(z2.x, z2.y));
                t[j + 1] = mul2(cx, make_float2(z2.z, z2.w));
            }
        } else {
#pragma unroll
            for (int j = 0; j < KZ; ++j)
                t[j] = mul2(cx, *reinterpret_cast<const float2 *>(s + OWZ + 2 * (h * KZ + j)));
        }
#pragma unroll
        for (int k = 0; k < W; k += 2) {
            const float4 wp = *reinterpret_cast<const float4 *>(s + 2 * k);
#pragma unroll
            for (int j = 0; j < KZ; ++j) {
                fma2(acc[j][k], t[j], make_float2(wp.x, wp.y));
                if (k + 1 < W) fma2(acc[j][k + 1 < W ? k + 1 : k], t[j], make_float2(wp.z, wp.w));
            }
        }
    };

    // The records come ordered by start row (setpts).  row is the oldest padded
    // row held (slot k, fine-grid row g); a point starting at row r needs rows
    // r .. r + W - 1: the rows below r are complete and are flushed first; a row
    // W or more above (or, defensively, below) the held ones flushes all W slots,
    // and so does the end of the subproblem (one past the last point).
    const R *recs = a.recs + sub.y;
    const int32_t *ord = a.order + sub.y;
    int row = 0, k = 0, g = grow0;
    R rc;
    C cv;
    if (lane < n) {
        rc = recs[lane];
        cv = cin[ord[lane]];
    }
    for (int base = 0; base < n; base += 32) {
        const int c = min(32, n - base);
        int myrow = 0x7fffffff;
        __syncwarp();                                      // the old slots are consumed
        if (lane < c) {
            const uint32_t pk = unpack_word<T>(rc.w);
            float *s = stg + lane * SLOT;
            const int sx = (int)(pk & 1023u);
            const int sy = (int)((pk >> 10) & 1023u);
            const int sz = (int)(pk >> 20);
            myrow = sy;
            float vx[W], vy[W], vz[W];
            kernel_row<T, W>(a, rc.x, vx);
            kernel_row<T, W>(a, rc.y, vy);
            kernel_row<T, W>(a, rc.z, vz);
#pragma unroll
            for (int kk = 0; kk < 32; kk += 4) store_zero_quad(s + OCX + kk);
#pragma unroll
            for (int kk = 0; kk < 4 * KZ; kk += 4) store_zero_quad(s + OWZ + kk);
#pragma unroll
            for (int i = 0; i < W; ++i) {
                *reinterpret_cast<C *>(s + OCX + 2 * (sx + i)) = make_float2(cv.x * vx[i], cv.y * vx[i]);
                *reinterpret_cast<float2 *>(s + OWZ + 2 * (sz + i)) = make_float2(vz[i], vz[i]);
            }
            int slot = sy % W;                             // w_y[i] goes to slot (sy + i) mod W
#pragma unroll
            for (int i = 0; i < W; ++i) {
                *reinterpret_cast<float2 *>(s + 2 * slot) = make_float2(vy[i], vy[i]);
                slot = slot + 1 == W ? 0 : slot + 1;
            }
        }
        if (base + 32 + lane < n) {                        // the next batch in flight
            rc = recs[base + 32 + lane];
            cv = cin[ord[base + 32 + lane]];
        }
        if (base == 0) {
            row = __shfl_sync(kFullMask, myrow, 0);
            k = row % W;
            g = wrap_any(grow0 + row, a.n1);
        }
        __syncwarp();
        // the batch as segments of equal start row: one ballot, then per segment
        // the rows below it are flushed and its points run back to back
        const int prev = __shfl_up_sync(kFullMask, myrow, 1);
        unsigned starts = __ballot_sync(kFullMask, lane < c && (lane == 0 || myrow != prev));
        const bool last = base + 32 >= n;
        while (starts != 0u || last) {
            const int i0 = starts ? __ffs(starts) - 1 : c;     // c: the end of the subproblem
            if (starts) starts &= starts - 1;
            const int i1 = starts ? __ffs(starts) - 1 : c;
            const int r = i0 < c ? __shfl_sync(kFullMask, myrow, i0) : 0x7fffffff;
            if (r != row) {
                const bool all = r < row || r - row >= W;
                const int nf = all ? W : r - row;
#pragma unroll 1
                for (int f = 0; f < nf; ++f) {             // rows row .. row + nf - 1 are complete
                    switch (k) {                           // W <= 8 slots
                    case 0: flush(0, g); break;
                    case 1: if constexpr (W > 1) flush(1, g); break;
                    case 2: if constexpr (W > 2) flush(2, g); break;
                    case 3: if constexpr (W > 3) flush(3, g); break;
                    case 4: if constexpr (W > 4) flush(4, g); break;
                    case 5: if constexpr (W > 5) flush(5, g); break;
                    case 6: if constexpr (W > 6) flush(6, g); break;
                    default: if constexpr (W > 7) flush(7, g); break;
                    }
                    k = k + 1 == W ? 0 : k + 1;
                    g = g + 1 == a.n1 ? 0 : g + 1;
                }
                if (i0 < c) {
                    if (all) {
                        k = r % W;
                        g = wrap_any(grow0 + r, a.n1);
                    }
                    row = r;
                }
            }
            if (i0 >= c) break;
#pragma unroll 1
            for (int i = i0; i < i1; ++i) step(i);
        }
    }
}

template <typename T, int W, int M2, int L>
__device__ __forceinline__ void spread_sweep3_item(const KArgs<T> &a, int sp, int tr,
                                                   unsigned char *sm)
{
    if constexpr (L == 16)
        spread_planes3_sub<T, W, M2>(a, a.subprob[sp], tr, sm);
    else
        spread_sweep3_sub<T, W, M2, L>(a, a.subprob[sp], tr, sm);
}

// Four warps per CTA; the plane-split form (L = 16) fits three CTAs per SM.
template <int L> __host__ __device__ constexpr int sweep3_threads() { return 128; }

template <typename T, int W, int M2, int L>
__global__ void __launch_bounds__(sweep3_threads<L>(), L == 16 ? 3 : 1)
spread_sweep3_kernel(KArgs<T> a, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    unsigned char *sm = smem_raw + (size_t)warp * warp_bytes;
    const int per_cta = blockDim.x >> 5;
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = (int64_t)blockIdx.x * per_cta + warp; wi < nwork;
         wi += (int64_t)gridDim.x * per_cta)
        spread_sweep3_item<T, W, M2, L>(a, (int)(wi % nsp), (int)(wi / nsp), sm);
}

template <typename T, int W, int L>
__device__ __forceinline__ void spread_sweep2_item(const KArgs<T> &a, int sp, int tr,
                                                   unsigned char *sm)
{
    spread_sweep2_sub<T, W, L>(a, a.subprob[sp], tr, sm);
}

template <typename T, int W, int L>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
spread_sweep2_kernel(KArgs<T> a, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    unsigned char *sm = smem_raw + (size_t)warp * warp_bytes;
    const int per_cta = blockDim.x >> 5;
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = (int64_t)blockIdx.x * per_cta + warp; wi < nwork;
         wi += (int64_t)gridDim.x * per_cta)
        spread_sweep2_item<T, W, L>(a, (int)(wi % nsp), (int)(wi / nsp), sm);
}

// ---------------------------------------------------------------------------
// GM-sort spreading: bin-ordered points, global atomics.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__device__ __forceinline__ void spread_gmsort_item(const KArgs<T> &a, int sp, int tr)
{
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int P = pad_lo(W);
    {
        const int4 sub = a.subprob[sp];
        int o0, o1, o2;
        bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
        const C *cin = a.cin + (int64_t)tr * a.M;
        C *grid = a.grid + (int64_t)tr * a.nftot;
        for (int base = warp * 32; base < sub.z; base += nwarps * 32) {
            R r;
            r.x = r.y = r.z = r.w = (T)0;
            C cv;
            cv.x = cv.y = (T)0;
            if (base + lane < sub.z) {
                const int64_t pos = sub.y + base + lane;
                r = a.recs[pos];
                cv = cin[point_of<T, DIM>(a, r, pos)];
            }
            const int np = min(32, sub.z - base);
            for (int i0 = 0; i0 < np; i0 += G) {
                const int p = i0 + g;
                const bool act = gact && p < np;
                const PointView<T> pv = take_point<T, true>(r, cv, p < 32 ? p : 31);
                const T wx = es_kernel(((T)dx - pv.dx) * a.hw, a.beta);
                const T myy = es_kernel(((T)dx - pv.dy) * a.hw, a.beta);
                const T myz = DIM == 3 ? es_kernel(((T)dx - pv.dz) * a.hw, a.beta) : (T)0;
                T wy[W];
#pragma unroll
                for (int i = 0; i < W; ++i) wy[i] = shfl(myy, src0 + i);
                const int gx = wrap_any(o0 - P + (int)(pv.pk & 1023u) + dx, a.n0);
                const int ly0 = o1 - P + (int)((pv.pk >> 10) & 1023u);
                const int lz0 = o2 - P + (int)(pv.pk >> 20);
                const T zr0 = pv.cr * wx, zi0 = pv.ci * wx;
                const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
                for (int iz = 0; iz < nz; ++iz) {
                    const T vz = DIM == 3 ? shfl(myz, src0 + iz) : (T)1;
                    const T zr = zr0 * vz, zi = zi0 * vz;
                    const int gz = DIM == 3 ? wrap_any(lz0 + iz, a.n2) : 0;
#pragma unroll
                    for (int iy = 0; iy < W; ++iy) {
                        if (act) {
                            const int gy = wrap_any(ly0 + iy, a.n1);
                            atomic_add_cplx(&grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx],
                                            wy[iy] * zr, wy[iy] * zi);
                        }
                    }
                }
            }
        }
    }
}

template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_gmsort_kernel(KArgs<T> a)
{
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x)
        spread_gmsort_item<T, DIM, W>(a, (int)(wi % nsp), (int)(wi / nsp));
}

template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_gmsort_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                           int nplans)
{
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        const KArgs<T> &a = args[pl];
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        spread_gmsort_item<T, DIM, W>(a, (int)(local % nsp), (int)(local / nsp));
    }
}

// ---------------------------------------------------------------------------
// GM spreading: user order, positions from the coordinates.  A warp takes
// G = 32 / W consecutive (transform, point) items at a time, item = tr * M + j;
// lane group g works on item base + g.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__device__ __forceinline__ void spread_gm_step(const KArgs<T> &a, int64_t base, int64_t end)
{
    using C = typename cplx<T>::type;
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int64_t item = base + g;
    const bool act = gact && item < end;
    T wx = 0, myy = 0, myz = 0, cre = 0, cim = 0;
    int gx = 0, ly0 = 0, lz0 = 0, tr = 0;
    if (act) {
        tr = (int)(item / a.M);
        const int64_t j = item - (int64_t)tr * a.M;
        const AxisPos<T> px = axis_position<T>(period_fraction(a.xyz0[j]), a.n0, W);
        const AxisPos<T> py = axis_position<T>(period_fraction(a.xyz1[j]), a.n1, W);
        wx = es_kernel(((T)dx - px.delta) * a.hw, a.beta);
        myy = es_kernel(((T)dx - py.delta) * a.hw, a.beta);
        gx = wrap_any(px.l0 + dx, a.n0);
        ly0 = py.l0;
        if (DIM == 3) {
            const AxisPos<T> pz = axis_position<T>(period_fraction(a.xyz2[j]), a.n2, W);
            myz = es_kernel(((T)dx - pz.delta) * a.hw, a.beta);
            lz0 = pz.l0;
        }
        const C cv = a.cin[item];
        cre = cv.x;
        cim = cv.y;
    }
    T wy[W];
#pragma unroll
    for (int i = 0; i < W; ++i) wy[i] = shfl(myy, src0 + i);
    C *grid = a.grid + (int64_t)tr * a.nftot;
    const T zr0 = cre * wx, zi0 = cim * wx;
    const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
    for (int iz = 0; iz < nz; ++iz) {
        const T vz = DIM == 3 ? shfl(myz, src0 + iz) : (T)1;
        const T zr = zr0 * vz, zi = zi0 * vz;
        const int gz = DIM == 3 ? wrap_any(lz0 + iz, a.n2) : 0;
#pragma unroll
        for (int iy = 0; iy < W; ++iy) {
            if (act) {
                const int gy = wrap_any(ly0 + iy, a.n1);
                atomic_add_cplx(&grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx], wy[iy] * zr,
                                wy[iy] * zi);
            }
        }
    }
}

template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
spread_gm_kernel(KArgs<T> a)
{
    constexpr int G = 32 / W;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = a.M * a.ntransf;
    for (int64_t base = gwarp * G; base < total; base += nwarps_total * G)
        spread_gm_step<T, DIM, W>(a, base, total);
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
// Sorted interpolation with one thread per point (Sec. 4.2).  The CTA stages
// the subproblem's padded bin in shared memory (STAGED; coalesced row loads
// with periodic wrap) or reads the fine grid directly (GM-sort), then every
// thread takes points of the subproblem: it evaluates its point's d W kernel
// values and accumulates the W^d window as sum_z w_z sum_y w_y sum_x w_x g --
// no shuffles and no cross-lane sums, every lane busy with its own point.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W, bool STAGED>
__device__ __forceinline__ void interp_lane_item(const KArgs<T> &a, int sp, int tr,
                                                 typename cplx<T>::type *tile)
{
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    const int P = pad_lo(W);
    const int4 sub = a.subprob[sp];
    int o0, o1, o2;
    bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
    const C *grid = a.grid + (int64_t)tr * a.nftot;
    C *cout = a.cout + (int64_t)tr * a.M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    if (STAGED) {
        const int rows = a.p1 * (DIM == 3 ? a.p2 : 1);
        for (int rr = warp; rr < rows; rr += nwarps) {
            const int ry = rr % a.p1, rz = rr / a.p1;
            const int gy = wrap_any(o1 - P + ry, a.n1);
            const int gz = DIM == 3 ? wrap_any(o2 - P + rz, a.n2) : 0;
            const C *src = grid + ((int64_t)gz * a.n1 + gy) * a.n0;
            for (int rx = lane; rx < a.p0; rx += 32)
                tile[rr * a.p0 + rx] = src[wrap_any(o0 - P + rx, a.n0)];
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < sub.z; k += blockDim.x) {
        const R rc = a.recs[sub.y + k];
        const int j = point_of<T, DIM>(a, rc, sub.y + k);
        const uint32_t pk = unpack_word<T>(rc.w);
        const int sx = pk & 1023u, sy = (pk >> 10) & 1023u, sz = pk >> 20;
        T wx[W], wy[W];
        kernel_row<T, W>(a, rc.x, wx);
        kernel_row<T, W>(a, rc.y, wy);
        int gxs[STAGED ? 1 : W];
        if (!STAGED) {
#pragma unroll
            for (int i = 0; i < W; ++i) gxs[STAGED ? 0 : i] = wrap_any(o0 - P + sx + i, a.n0);
        }
        T ar = 0, ai = 0;
        const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
        for (int iz = 0; iz < nz; ++iz) {
            T zr = 0, zi = 0;
            const int gz = DIM == 3 && !STAGED ? wrap_any(o2 - P + sz + iz, a.n2) : 0;
#pragma unroll
            for (int iy = 0; iy < W; ++iy) {
                T yr = 0, yi = 0;
                if (STAGED) {
                    const C *t = tile + ((sz + iz) * a.p1 + sy + iy) * a.p0 + sx;
#pragma unroll
                    for (int ix = 0; ix < W; ++ix) {
                        const C g = t[ix];
                        yr += wx[ix] * g.x;
                        yi += wx[ix] * g.y;
                    }
                } else {
                    const int gy = wrap_any(o1 - P + sy + iy, a.n1);
                    const C *row = grid + ((int64_t)gz * a.n1 + gy) * a.n0;
#pragma unroll
                    for (int ix = 0; ix < W; ++ix) {
                        const C g = row[gxs[STAGED ? 0 : ix]];
                        yr += wx[ix] * g.x;
                        yi += wx[ix] * g.y;
                    }
                }
                zr += wy[iy] * yr;
                zi += wy[iy] * yi;
            }
            const T vz = DIM == 3 ? kernel_cell<T, W>(a, rc.z, iz) : (T)1;
            ar += vz * zr;
            ai += vz * zi;
        }
        C o;
        o.x = ar;
        o.y = ai;
        cout[j] = o;
    }
    if (STAGED) __syncthreads();
}

// ---------------------------------------------------------------------------
// Plane-split row sweep for 3D interpolation (single precision, p0 <= 16,
// W <= 8; Sec. 4.2 with the padded bin held in registers instead of shared
// memory).  Lane (h, q) owns x column q and planes h KZ .. h KZ + KZ - 1 of
// the padded bin, as in the spreading sweep, and holds the W padded rows that
// a window starting at the current row reads (slot = row mod W), loaded from
// the fine grid one row ahead of their first use.  The points, ordered by
// window start row, are staged 32 at a time (w_x as a 16-wide row, w_z as a
// PZ-wide row, both zero outside the window; w_y rotated to the row slots);
// for each point every lane forms
//   sum_i (w_x[q] w_z[h KZ + i]) sum_s g[i][s] w_y[s]
// and stores it in a per-batch table of partial sums (one row per point, pitch
// 33); after the batch the lane that staged point i sums row i and stores the
// point's value -- 2 operations per point instead of a 5-level butterfly.
template <int W, int M2> __host__ __device__ constexpr int iplanes3_owz() { return 4 * ((W + 1) / 2); }
template <int W, int M2> __host__ __device__ constexpr int iplanes3_owx()
{
    return iplanes3_owz<W, M2>() + 4 * ((2 * planes3_kz<W, M2>() + 3) / 4);
}
template <int W, int M2> __host__ __device__ constexpr int iplanes3_slot()
{
    return ((iplanes3_owx<W, M2>() + 16) / 4 | 1) * 4;
}
template <int W, int M2>
__host__ __device__ inline size_t iplanes3_bytes(int m1)
{
    (void)m1;
    // 32 staging slots, then the 32 x 33 partial sums of a batch (float2)
    return sizeof(float) * (size_t)32 * iplanes3_slot<W, M2>() + sizeof(float2) * 32 * 33;
}

template <typename T, int W, int M2>
__device__ __forceinline__ void interp_planes3_sub(const KArgs<T> &a, int4 sub, int tr,
                                                   unsigned char *sm)
{
    static_assert(sizeof(T) == 4, "the 3D row sweep is single precision");
    using C = float2;
    using R = typename rec4<T>::type;
    constexpr int KZ = planes3_kz<W, M2>();
    constexpr int PZ = M2 + W;
    constexpr int SLOT = iplanes3_slot<W, M2>();
    constexpr int OWZ = iplanes3_owz<W, M2>(), OWX = iplanes3_owx<W, M2>();
    const int lane = threadIdx.x & 31, h = lane >> 4, q = lane & 15;
    const int n = sub.z;
    float *stg = reinterpret_cast<float *>(sm);
    float2 *part = reinterpret_cast<float2 *>(sm + sizeof(float) * 32 * SLOT);   // [point][lane], pitch 33
    int o0, o1, o2;
    bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
    const int P = pad_lo(W);
    const C *grid = a.grid + (int64_t)tr * a.nftot;
    C *cout = a.cout + (int64_t)tr * a.M;
    const bool xok = q < a.p0;
    const int gx = wrap_any(o0 - P + (xok ? q : 0), a.n0);
    const int grow0 = wrap_any(o1 - P, a.n1);
    const C *gcol = grid + gx;
    int gz[KZ];                                            // fine-grid plane of each owned plane
#pragma unroll
    for (int i = 0; i < KZ; ++i)
        gz[i] = xok && h * KZ + i < PZ ? wrap_any(o2 - P + h * KZ + i, a.n2) : -1;
    // padded row rr (fine-grid row gg) of every owned plane, zero past the padded bin
    auto load_row = [&](int rr, int gg, float2 (&dst)[KZ]) {
#pragma unroll
        for (int i = 0; i < KZ; ++i)
            dst[i] = gz[i] >= 0 && rr < a.p1 ? __ldg(gcol + ((int64_t)gz[i] * a.n1 + gg) * a.n0)
                                             : make_float2(0.f, 0.f);
    };
    float2 g[KZ][W];                                       // g[i][slot]: padded row = slot mod W
    float2 nxt[KZ];                                        // row + W, in flight
    auto put_slot = [&](int k, const float2 (&v)[KZ]) {
#pragma unroll
        for (int kk = 0; kk < W; ++kk)
            if (kk == k) {
#pragma unroll
                for (int i = 0; i < KZ; ++i) g[i][kk] = v[i];
            }
    };
    // rows r .. r + W - 1 into their slots, row r + W in flight
    auto load_window = [&](int r) {
        int gg = wrap_any(grow0 + r, a.n1);
        int k = r % W;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            float2 v[KZ];
            load_row(r + j, gg, v);
            put_slot(k, v);
            k = k + 1 == W ? 0 : k + 1;
            gg = gg + 1 == a.n1 ? 0 : gg + 1;
        }
        load_row(r + W, gg, nxt);
    };

    // Records ordered by start row (setpts); row is the lowest padded row held.  Moving up one row puts the row in flight into the freed slot
    // and starts the load of the next; any other change of row (the next run,
    // or a gap) reloads the whole window.
    const R *recs = a.recs + sub.y;
    const int32_t *ord = a.order + sub.y;
    int row = 0, k = 0, gnext = 0;                         // gnext: fine-grid row of nxt
    R rc;
    int jn = 0;
    if (lane < n) {
        rc = recs[lane];
        jn = ord[lane];
    }
    for (int base = 0; base < n; base += 32) {
        const int c = min(32, n - base);
        int myrow = 0x7fffffff, jout = 0;
        __syncwarp();
        if (lane < c) {
            const uint32_t pk = unpack_word<T>(rc.w);
            float *s = stg + lane * SLOT;
            const int sx = (int)(pk & 1023u);
            const int sy = (int)((pk >> 10) & 1023u);
            const int sz = (int)(pk >> 20);
            myrow = sy;
            jout = jn;
            float vx[W], vy[W], vz[W];
            kernel_row<T, W>(a, rc.x, vx);
            kernel_row<T, W>(a, rc.y, vy);
            kernel_row<T, W>(a, rc.z, vz);
#pragma unroll
            for (int kk = 0; kk < 16; kk += 4) store_zero_quad(s + OWX + kk);
#pragma unroll
            for (int kk = 0; kk < OWX - OWZ; kk += 4) store_zero_quad(s + OWZ + kk);
#pragma unroll
            for (int i = 0; i < W; ++i) {
                s[OWX + sx + i] = vx[i];
                s[OWZ + sz + i] = vz[i];
            }
            int slot = sy % W;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                *reinterpret_cast<float2 *>(s + 2 * slot) = make_float2(vy[i], vy[i]);
                slot = slot + 1 == W ? 0 : slot + 1;
            }
        }
        if (base + 32 + lane < n) {
            rc = recs[base + 32 + lane];
            jn = ord[base + 32 + lane];
        }
        if (base == 0) {
            row = __shfl_sync(kFullMask, myrow, 0);
            k = row % W;
            load_window(row);
            gnext = wrap_any(grow0 + row + W, a.n1);
        }
        __syncwarp();
        const int prev = __shfl_up_sync(kFullMask, myrow, 1);
        unsigned starts = __ballot_sync(kFullMask, lane < c && (lane == 0 || myrow != prev));
        while (starts) {                                   // segments of equal start row
            const int i0 = __ffs(starts) - 1;
            starts &= starts - 1;
            const int i1 = starts ? __ffs(starts) - 1 : c;
            const int r = __shfl_sync(kFullMask, myrow, i0);
            if (r == row + 1) {                            // slot k (row) takes row + W
                put_slot(k, nxt);
                k = k + 1 == W ? 0 : k + 1;
                gnext = gnext + 1 == a.n1 ? 0 : gnext + 1;
                row = r;
                load_row(row + W, gnext, nxt);
            } else if (r != row) {                         // a new run or a gap
                row = r;
                k = r % W;
                load_window(r);
                gnext = wrap_any(grow0 + r + W, a.n1);
            }
#pragma unroll 1
            for (int i = i0; i < i1; ++i) {
                const float *s = stg + i * SLOT;
                const float wx = s[OWX + q];
                float wz[KZ];
                if constexpr (KZ % 4 == 0) {
#pragma unroll
                    for (int j = 0; j < KZ; j += 4) {
                        const float4 z4 = *reinterpret_cast<const float4 *>(s + OWZ + h * KZ + j);
                        wz[j] = z4.x;
                        wz[j + 1] = z4.y;
                        wz[j + 2] = z4.z;
                        wz[j + 3] = z4.w;
                    }
                } else if constexpr (KZ % 2 == 0) {
#pragma unroll
                    for (int j = 0; j < KZ; j += 2) {
                        const float2 z2 = *reinterpret_cast<const float2 *>(s + OWZ + h * KZ + j);
                        wz[j] = z2.x;
                        wz[j + 1 < KZ ? j + 1 : j] = z2.y;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < KZ; ++j) wz[j] = s[OWZ + h * KZ + j];
                }
                float2 u[KZ];
#pragma unroll
                for (int kk = 0; kk < W; kk += 2) {
                    const float4 wp = *reinterpret_cast<const float4 *>(s + 2 * kk);
#pragma unroll
                    for (int j = 0; j < KZ; ++j) {
                        if (kk == 0) u[j] = mul2(g[j][0], make_float2(wp.x, wp.y));
                        else fma2(u[j], g[j][kk], make_float2(wp.x, wp.y));
                        if (kk + 1 < W) fma2(u[j], g[j][kk + 1 < W ? kk + 1 : kk], make_float2(wp.z, wp.w));
                    }
                }
                float2 v = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < KZ; ++j) {
                    const float tw = wx * wz[j];
                    fma2(v, u[j], make_float2(tw, tw));
                }
                part[i * 33 + lane] = v;                   // summed over the lanes per batch
            }
        }
        __syncwarp();
        if (lane < c) {                                    // lane i sums point i's 32 partials
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int l = 0; l < 32; ++l) acc = __fadd2_rn(acc, part[lane * 33 + l]);
            cout[jout] = acc;
        }
    }
}

template <typename T, int W, int M2>
__global__ void __launch_bounds__(128, 3)
interp_planes3_kernel(KArgs<T> a, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    unsigned char *sm = smem_raw + (size_t)warp * warp_bytes;
    const int per_cta = blockDim.x >> 5;
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = (int64_t)blockIdx.x * per_cta + warp; wi < nwork;
         wi += (int64_t)gridDim.x * per_cta) {
        const int sp = (int)(wi % nsp);
        interp_planes3_sub<T, W, M2>(a, a.subprob[sp], (int)(wi / nsp), sm);
    }
}

// Asynchronous global -> shared copies (cp.async, sm_80+): the data land in
// shared memory without passing through registers, and a warp can compute on
// one buffer while the next one is in flight.
__device__ __forceinline__ void cp_async_cplx(float2 *dst, const float2 *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_cplx(double2 *dst, const double2 *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 2D interpolation, one warp per work item (no CTA barriers, so many
// subproblems are in flight per SM).  interp2_stage issues the copies of the
// work item's padded bin into a warp-private tile (row by row, periodic wrap);
// interp2_points then has every lane take points of the subproblem as above:
// the 2D records carry their point's index, and the next record is loaded
// while the current point is computed.
template <typename T, int W>
__device__ __forceinline__ void interp2_stage(const KArgs<T> &a, int sp, int tr,
                                              typename cplx<T>::type *tile)
{
    using C = typename cplx<T>::type;
    const int P = pad_lo(W);
    const int lane = threadIdx.x & 31;
    const int4 sub = a.subprob[sp];
    int o0, o1, o2;
    bin_origin(sub.x, a.nb0, a.nb1, a.m0, a.m1, a.m2, o0, o1, o2);
    const C *grid = a.grid + (int64_t)tr * a.nftot;
    for (int rx = lane; rx < a.p0; rx += 32) {
        const C *src = grid + wrap_any(o0 - P + rx, a.n0);
        int gy = wrap_any(o1 - P, a.n1);
        for (int ry = 0; ry < a.p1; ++ry) {
            cp_async_cplx(tile + ry * a.p0 + rx, src + (int64_t)gy * a.n0);
            gy = gy + 1 == a.n1 ? 0 : gy + 1;
        }
    }
}

template <typename T, int W>
__device__ __forceinline__ void interp2_points(const KArgs<T> &a, int sp, int tr,
                                               const typename cplx<T>::type *tile)
{
    using C = typename cplx<T>::type;
    using R = typename rec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int4 sub = a.subprob[sp];
    C *cout = a.cout + (int64_t)tr * a.M;
    const R *recs = a.recs + sub.y;
    const int np = sub.z;
    R rn;
    if (lane < np) rn = recs[lane];
    for (int k = lane; k < np; k += 32) {
        const R rc = rn;
        if (k + 32 < np) rn = recs[k + 32];
        const int j = (int)unpack_word<T>(rc.z);
        const uint32_t pk = unpack_word<T>(rc.w);
        const int sx = pk & 1023u, sy = (pk >> 10) & 1023u;
        T wx[W], wy[W];
        kernel_row<T, W>(a, rc.x, wx);
        kernel_row<T, W>(a, rc.y, wy);
        C o;
        if constexpr (sizeof(T) == 4) {
            // (re, im) sums: one f32x2 FMA per cell
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int iy = 0; iy < W; ++iy) {
                const float2 *t = reinterpret_cast<const float2 *>(tile + (sy + iy) * a.p0 + sx);
                float2 yv = make_float2(0.f, 0.f);
#pragma unroll
                for (int ix = 0; ix < W; ++ix) fma2(yv, t[ix], make_float2(wx[ix], wx[ix]));
                fma2(acc, yv, make_float2(wy[iy], wy[iy]));
            }
            o.x = acc.x;
            o.y = acc.y;
        } else {
            T ar = 0, ai = 0;
#pragma unroll
            for (int iy = 0; iy < W; ++iy) {
                const C *t = tile + (sy + iy) * a.p0 + sx;
                T yr = 0, yi = 0;
#pragma unroll
                for (int ix = 0; ix < W; ++ix) {
                    const C g = t[ix];
                    yr += wx[ix] * g.x;
                    yi += wx[ix] * g.y;
                }
                ar += wy[iy] * yr;
                ai += wy[iy] * yi;
            }
            o.x = ar;
            o.y = ai;
        }
        cout[j] = o;
    }
}

// One work item with its own (not overlapped) staging: the batched form.
template <typename T, int W>
__device__ __forceinline__ void interp_warp2_item(const KArgs<T> &a, int sp, int tr,
                                                  unsigned char *sm)
{
    auto *tile = reinterpret_cast<typename cplx<T>::type *>(sm);
    __syncwarp();
    interp2_stage<T, W>(a, sp, tr, tile);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    interp2_points<T, W>(a, sp, tr, tile);
}

// Shared memory of one warp of the 2D interpolation: `buffers` padded bins of
// tile_elems cells.
template <typename T>
__host__ __device__ inline size_t interp2_warp_bytes(int tile_elems, int buffers)
{
    return sizeof(typename cplx<T>::type) * (size_t)tile_elems * buffers;
}

// Single plan: each warp walks its work items with two tiles, copying the next
// item's padded bin while it interpolates at the current one's points.
template <typename T, int W>
__global__ void __launch_bounds__(256)
interp_warp2_kernel(KArgs<T> a, int tile_elems)
{
    using C = typename cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    C *buf = reinterpret_cast<C *>(smem_raw) + (size_t)warp * 2 * tile_elems;
    const int per_cta = blockDim.x >> 5;
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    const int64_t stride = (int64_t)gridDim.x * per_cta;
    int64_t wi = (int64_t)blockIdx.x * per_cta + warp;
    if (wi < nwork) interp2_stage<T, W>(a, (int)(wi % nsp), (int)(wi / nsp), buf);
    cp_async_commit();
    int cur = 0;
    for (; wi < nwork; wi += stride) {
        const int64_t nx = wi + stride;
        if (nx < nwork)
            interp2_stage<T, W>(a, (int)(nx % nsp), (int)(nx / nsp), buf + (cur ^ 1) * tile_elems);
        cp_async_commit();
        cp_async_wait<1>();                                // the current tile has landed
        __syncwarp();
        interp2_points<T, W>(a, (int)(wi % nsp), (int)(wi / nsp), buf + cur * tile_elems);
        __syncwarp();                                      // before the tile is refilled
        cur ^= 1;
    }
    cp_async_wait<0>();
}

template <typename T, int DIM, int W, bool STAGED>
__global__ void __launch_bounds__(256)
interp_lane_kernel(KArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto *tile = reinterpret_cast<typename cplx<T>::type *>(smem_raw);
    const int nsp = *a.nsub;
    const int64_t nwork = (int64_t)nsp * a.ntransf;
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x)
        interp_lane_item<T, DIM, W, STAGED>(a, (int)(wi % nsp), (int)(wi / nsp), tile);
}

// ---------------------------------------------------------------------------
// GM interpolation: user order, G items per warp as in GM spreading.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int W>
__device__ __forceinline__ void interp_gm_step(const KArgs<T> &a, int64_t base, int64_t end)
{
    using C = typename cplx<T>::type;
    constexpr int G = 32 / W;
    const int lane = threadIdx.x & 31;
    const int g = lane / W, dx = lane - (lane / W) * W;
    const bool gact = g < G;
    const int src0 = (gact ? g : G - 1) * W;
    const int64_t item = base + g;
    const bool act = gact && item < end;
    T wx = 0, myy = 0, myz = 0;
    int gx = 0, ly0 = 0, lz0 = 0, tr = 0;
    if (act) {
        tr = (int)(item / a.M);
        const int64_t j = item - (int64_t)tr * a.M;
        const AxisPos<T> px = axis_position<T>(period_fraction(a.xyz0[j]), a.n0, W);
        const AxisPos<T> py = axis_position<T>(period_fraction(a.xyz1[j]), a.n1, W);
        wx = es_kernel(((T)dx - px.delta) * a.hw, a.beta);
        myy = es_kernel(((T)dx - py.delta) * a.hw, a.beta);
        gx = wrap_any(px.l0 + dx, a.n0);
        ly0 = py.l0;
        if (DIM == 3) {
            const AxisPos<T> pz = axis_position<T>(period_fraction(a.xyz2[j]), a.n2, W);
            myz = es_kernel(((T)dx - pz.delta) * a.hw, a.beta);
            lz0 = pz.l0;
        }
    }
    T wy[W];
#pragma unroll
    for (int i = 0; i < W; ++i) wy[i] = shfl(myy, src0 + i);
    const C *grid = a.grid + (int64_t)tr * a.nftot;
    T ar = 0, ai = 0;
    const int nz = DIM == 3 ? W : 1;
#pragma unroll 1
    for (int iz = 0; iz < nz; ++iz) {
        const T vz = DIM == 3 ? shfl(myz, src0 + iz) : (T)1;
        const int gz = DIM == 3 ? wrap_any(lz0 + iz, a.n2) : 0;
        T zr = 0, zi = 0;
#pragma unroll
        for (int iy = 0; iy < W; ++iy) {
            if (act) {
                const int gy = wrap_any(ly0 + iy, a.n1);
                const C v = grid[((int64_t)gz * a.n1 + gy) * a.n0 + gx];
                zr += wy[iy] * v.x;
                zi += wy[iy] * v.y;
            }
        }
        ar += vz * zr;
        ai += vz * zi;
    }
    ar = group_sum<T, W>(act ? ar * wx : (T)0, dx);
    ai = group_sum<T, W>(act ? ai * wx : (T)0, dx);
    if (act && dx == 0) {
        C o;
        o.x = ar;
        o.y = ai;
        a.cout[item] = o;
    }
}

template <typename T, int DIM, int W>
__global__ void __launch_bounds__(256)
interp_gm_kernel(KArgs<T> a)
{
    constexpr int G = 32 / W;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps_total = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = a.M * a.ntransf;
    for (int64_t base = gwarp * G; base < total; base += nwarps_total * G)
        interp_gm_step<T, DIM, W>(a, base, total);
}

// ---------------------------------------------------------------------------
// Multi-plan (batched) forms of the row sweeps and the one-thread-per-point
// interpolation.  Work items of all plans of a group are numbered by workoff;
// a warp (or CTA) copies the KArgs of the plan it is working on into shared
// memory when the plan changes, so parameter reads -- the kernel polynomial
// coefficients above all -- are shared-memory broadcasts.  Single-precision
// groups evaluate the kernel directly (cheaper than coefficients read from
// shared memory); double precision keeps the polynomials.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void warp_load_args(const KArgs<T> *args, int pl, KArgs<T> *cache,
                                               int &cached)
{
    if (pl == cached) return;
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const int4 *src = reinterpret_cast<const int4 *>(args + pl);
    int4 *dst = reinterpret_cast<int4 *>(cache);
    for (int i = lane; i < (int)(sizeof(KArgs<T>) / 16); i += 32) dst[i] = src[i];
    __syncwarp();
    if (sizeof(T) == 4 && lane == 0) cache->poly = 0;
    __syncwarp();
    cached = pl;
}

template <typename T>
__host__ __device__ constexpr size_t args_slot() { return (sizeof(KArgs<T>) + 15) & ~(size_t)15; }

template <typename T, int W, int L>
__global__ void __launch_bounds__(256)
spread_sweep2_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                           int nplans, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    unsigned char *base = smem_raw + (size_t)warp * (args_slot<T>() + warp_bytes);
    KArgs<T> *cache = reinterpret_cast<KArgs<T> *>(base);
    unsigned char *sm = base + args_slot<T>();
    const int per_cta = blockDim.x >> 5;
    int cached = -1;
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = (int64_t)blockIdx.x * per_cta + warp; wi < nwork;
         wi += (int64_t)gridDim.x * per_cta) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        warp_load_args(args, pl, cache, cached);
        const KArgs<T> &a = *cache;
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        spread_sweep2_item<T, W, L>(a, (int)(local % nsp), (int)(local / nsp), sm);
    }
}

template <typename T, int W, int M2>
__global__ void __launch_bounds__(128, 3)
interp_planes3_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                            int nplans, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    unsigned char *base = smem_raw + (size_t)warp * (args_slot<T>() + warp_bytes);
    KArgs<T> *cache = reinterpret_cast<KArgs<T> *>(base);
    unsigned char *sm = base + args_slot<T>();
    const int per_cta = blockDim.x >> 5;
    int cached = -1;
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = (int64_t)blockIdx.x * per_cta + warp; wi < nwork;
         wi += (int64_t)gridDim.x * per_cta) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        warp_load_args(args, pl, cache, cached);
        const KArgs<T> &a = *cache;
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        interp_planes3_sub<T, W, M2>(a, a.subprob[(int)(local % nsp)], (int)(local / nsp), sm);
    }
}

template <typename T, int W, int M2, int L>
__global__ void __launch_bounds__(sweep3_threads<L>(), L == 16 ? 3 : 1)
spread_sweep3_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                           int nplans, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    unsigned char *base = smem_raw + (size_t)warp * (args_slot<T>() + warp_bytes);
    KArgs<T> *cache = reinterpret_cast<KArgs<T> *>(base);
    unsigned char *sm = base + args_slot<T>();
    const int per_cta = blockDim.x >> 5;
    int cached = -1;
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = (int64_t)blockIdx.x * per_cta + warp; wi < nwork;
         wi += (int64_t)gridDim.x * per_cta) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        warp_load_args(args, pl, cache, cached);
        const KArgs<T> &a = *cache;
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        spread_sweep3_item<T, W, M2, L>(a, (int)(local % nsp), (int)(local / nsp), sm);
    }
}

template <typename T, int W>
__global__ void __launch_bounds__(256)
interp_warp2_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                          int nplans, int warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const size_t slot = args_slot<T>() + (size_t)warp_bytes;
    unsigned char *base = smem_raw + (size_t)warp * slot;
    KArgs<T> *cache = reinterpret_cast<KArgs<T> *>(base);
    unsigned char *sm = base + args_slot<T>();
    const int per_cta = blockDim.x >> 5;
    int cached = -1;
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = (int64_t)blockIdx.x * per_cta + warp; wi < nwork;
         wi += (int64_t)gridDim.x * per_cta) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        warp_load_args(args, pl, cache, cached);
        const KArgs<T> &a = *cache;
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        interp_warp2_item<T, W>(a, (int)(local % nsp), (int)(local / nsp), sm);
    }
}

// One CTA per work item (3D staged tile, or unstaged GM-sort); the CTA shares
// one KArgs copy.
template <typename T, int DIM, int W, bool STAGED>
__global__ void __launch_bounds__(256)
interp_lane_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff,
                         int nplans)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KArgs<T> *cache = reinterpret_cast<KArgs<T> *>(smem_raw);
    auto *tile = reinterpret_cast<typename cplx<T>::type *>(smem_raw + args_slot<T>());
    int cached = -1;
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        if (pl != cached) {
            __syncthreads();
            const int4 *src = reinterpret_cast<const int4 *>(args + pl);
            int4 *dst = reinterpret_cast<int4 *>(cache);
            for (int i = threadIdx.x; i < (int)(sizeof(KArgs<T>) / 16); i += blockDim.x)
                dst[i] = src[i];
            __syncthreads();
            if (sizeof(T) == 4 && threadIdx.x == 0) cache->poly = 0;
            __syncthreads();
            cached = pl;
        }
        const KArgs<T> &a = *cache;
        const int64_t local = wi - workoff[pl];
        const int nsp = *a.nsub;
        interp_lane_item<T, DIM, W, STAGED>(a, (int)(local % nsp), (int)(local / nsp), tile);
    }
}

// GM plans in a batch: a work item is a chunk of kGmChunk consecutive points of
// one transform (the plan's nsub holds its chunk count, set at setpts), run by
// one CTA whose warps take G = 32 / W points at a time.
template <typename T, int DIM, int W, bool SPREAD>
__global__ void __launch_bounds__(256)
gm_multi_kernel(const KArgs<T> *__restrict__ args, const int64_t *__restrict__ workoff, int nplans)
{
    __shared__ __align__(16) unsigned char cache_raw[sizeof(KArgs<T>)];
    KArgs<T> *cache = reinterpret_cast<KArgs<T> *>(cache_raw);
    constexpr int G = 32 / W;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int cached = -1;
    const int64_t nwork = workoff[nplans];
    for (int64_t wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int pl = batch_plan_of(workoff, nplans, wi);
        if (pl != cached) {
            __syncthreads();
            const int4 *src = reinterpret_cast<const int4 *>(args + pl);
            int4 *dst = reinterpret_cast<int4 *>(cache);
            for (int i = threadIdx.x; i < (int)(sizeof(KArgs<T>) / 16); i += blockDim.x)
                dst[i] = src[i];
            __syncthreads();
            cached = pl;
        }
        const KArgs<T> &a = *cache;
        const int64_t local = wi - workoff[pl];
        const int nchunk = *a.nsub;
        const int64_t tr = local / nchunk;
        const int64_t beg = tr * a.M + (local - tr * nchunk) * (int64_t)kGmChunk;
        const int64_t end = min(beg + (int64_t)kGmChunk, (tr + 1) * a.M);
        for (int64_t base = beg + (int64_t)warp * G; base < end; base += (int64_t)nwarps * G) {
            if (SPREAD) spread_gm_step<T, DIM, W>(a, base, end);
            else interp_gm_step<T, DIM, W>(a, base, end);
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
    // index of the point at each record position: t, or its copy reordered with
    // the records by start row (3D plane-split plans)
    a.order = p.row_ordered ? p.rorder : p.perm;
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
    a.p0 = padded(p.m[0], p.w);
    a.p1 = padded(p.m[1], p.w);
    a.p2 = p.dim == 3 ? padded(p.m[2], p.w) : 1;
    a.beta = (T)p.beta;
    a.hw = (T)(2.0 / p.w);
    a.poly = p.poly_ok ? 1 : 0;
    for (int i = 0; i < kMaxW; ++i)
        for (int d = 0; d < kPolyTerms; ++d) a.coef[i][d] = (T)p.poly[i][d];
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

// Launches the row-sweep kernel with as many warps per CTA as the shared memory
// allows (at most threads / 32); returns false, launching nothing, when fewer
// than two fit.
template <typename T, int W, int L>
bool launch_sweep2(Plan &p, const KArgs<T> &a, int threads, cudaError_t *err)
{
    const size_t warp_bytes = sweep_bytes<T, W, L>(a.m1);
    int nw = threads / 32;
    while (nw > 0 && (size_t)nw * warp_bytes > (size_t)p.smem_optin) --nw;
    if (nw < 2) return false;
    const size_t smem = warp_bytes * nw;
    auto k = spread_sweep2_kernel<T, W, L>;
    if (cudaError_t ea = allow_max_smem((const void *)k)) {
        *err = ea;
        return true;
    }
    k<<<persistent_grid(p, k, nw * 32, smem), nw * 32, smem, p.stream>>>(a, (int)warp_bytes);
    *err = cudaGetLastError();
    return true;
}

template <typename T, int W, int M2, int L>
bool launch_sweep3(Plan &p, const KArgs<T> &a, cudaError_t *err)
{
    size_t warp_bytes;
    if constexpr (L == 16) warp_bytes = planes3_bytes<W, M2>(a.m1);
    else warp_bytes = sweep3_bytes<T, W, M2, L>(a.m1);
    int nw = sweep3_threads<L>() / 32;
    while (nw > 0 && (size_t)nw * warp_bytes > (size_t)p.smem_optin) --nw;
    if (nw < 2) return false;
    const size_t smem = warp_bytes * nw;
    auto k = spread_sweep3_kernel<T, W, M2, L>;
    if (cudaError_t ea = allow_max_smem((const void *)k)) {
        *err = ea;
        return true;
    }
    k<<<persistent_grid(p, k, nw * 32, smem), nw * 32, smem, p.stream>>>(a, (int)warp_bytes);
    *err = cudaGetLastError();
    return true;
}

template <typename T, int W, int M2>
bool launch_iplanes3(Plan &p, const KArgs<T> &a, cudaError_t *err)
{
    const size_t warp_bytes = iplanes3_bytes<W, M2>(a.m1);
    int nw = 4;
    while (nw > 0 && (size_t)nw * warp_bytes > (size_t)p.smem_optin) --nw;
    if (nw < 2) return false;
    const size_t smem = warp_bytes * nw;
    auto k = interp_planes3_kernel<T, W, M2>;
    if (cudaError_t ea = allow_max_smem((const void *)k)) {
        *err = ea;
        return true;
    }
    k<<<persistent_grid(p, k, nw * 32, smem), nw * 32, smem, p.stream>>>(a, (int)warp_bytes);
    *err = cudaGetLastError();
    return true;
}

template <typename T, int DIM, int W>
cudaError_t spread_w(Plan &p, const void *c)
{
    KArgs<T> a = make_args<T>(p);
    a.cin = reinterpret_cast<const typename cplx<T>::type *>(c);
    const int threads = p.threads;
    count_launch();
    const int variant = sweep_variant(p);
    if constexpr (DIM == 3 && sizeof(T) == 4 && W <= 8) {
        if (variant > 0) {
            cudaError_t e = cudaSuccess;
            // variant: m2 (1 or 2), plus 4 when the padded width fits 16 lanes
            const bool ok = variant == 1   ? launch_sweep3<T, W, 1, 32>(p, a, &e)
                            : variant == 2 ? launch_sweep3<T, W, 2, 32>(p, a, &e)
                            : variant == 5 ? launch_sweep3<T, W, 1, 16>(p, a, &e)
                                           : launch_sweep3<T, W, 2, 16>(p, a, &e);
            if (ok) return e;
        }
    }
    if (DIM == 2 && variant > 0) {
        cudaError_t e = cudaSuccess;
        if (variant == 8 ? launch_sweep2<T, W, 8>(p, a, threads, &e)
                         : variant == 16 ? launch_sweep2<T, W, 16>(p, a, threads, &e)
                                         : launch_sweep2<T, W, 32>(p, a, threads, &e))
            return e;
    }
    if (p.method == NUFFT_METHOD_SM) {
        const size_t smem = (size_t)2 * sizeof(T) * a.p0 * a.p1 * a.p2;
        auto k = spread_sm_kernel<T, DIM, W>;
        if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
        const int grid = persistent_grid(p, k, threads, smem);
        k<<<grid, threads, smem, p.stream>>>(a);
    } else if (p.method == NUFFT_METHOD_GM_SORT) {
        auto k = spread_gmsort_kernel<T, DIM, W>;
        k<<<persistent_grid(p, k, threads, 0), threads, 0, p.stream>>>(a);
    } else {
        auto k = spread_gm_kernel<T, DIM, W>;
        const int64_t warps = (p.M * p.ntransf + (32 / W) - 1) / (32 / W);
        int64_t blocks = (warps * 32 + threads - 1) / threads;
        const int64_t cap = (int64_t)p.num_sms * 32;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
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
    count_launch();
    if constexpr (DIM == 3 && sizeof(T) == 4 && W <= 8) {
        const int variant = sweep_variant(p);
        if (variant == 5 || variant == 6) {
            cudaError_t e = cudaSuccess;
            if (variant == 5 ? launch_iplanes3<T, W, 1>(p, a, &e) : launch_iplanes3<T, W, 2>(p, a, &e))
                return e;
        }
    }
    if (p.method == NUFFT_METHOD_SM && DIM == 2) {
        // one padded bin per warp, as many warps per CTA as shared memory allows
        const int tile = a.p0 * a.p1;
        const size_t per_warp = interp2_warp_bytes<T>(tile, 2);
        int nw = threads / 32;
        while (nw > 1 && (size_t)nw * per_warp > (size_t)p.smem_optin) --nw;
        if ((size_t)nw * per_warp <= (size_t)p.smem_optin) {
            const size_t smem = per_warp * nw;
            auto k = interp_warp2_kernel<T, W>;
            if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
            k<<<persistent_grid(p, k, nw * 32, smem), nw * 32, smem, p.stream>>>(a, tile);
            return cudaGetLastError();
        }
    }
    if (p.method == NUFFT_METHOD_SM) {
        const size_t smem = sizeof(typename cplx<T>::type) * a.p0 * a.p1 * a.p2;
        auto k = interp_lane_kernel<T, DIM, W, true>;
        if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
        k<<<persistent_grid(p, k, threads, smem), threads, smem, p.stream>>>(a);
    } else if (p.method == NUFFT_METHOD_GM_SORT) {
        auto k = interp_lane_kernel<T, DIM, W, false>;
        k<<<persistent_grid(p, k, threads, 0), threads, 0, p.stream>>>(a);
    } else {
        auto k = interp_gm_kernel<T, DIM, W>;
        const int64_t warps = (p.M * p.ntransf + (32 / W) - 1) / (32 / W);
        int64_t blocks = (warps * 32 + threads - 1) / threads;
        const int64_t cap = (int64_t)p.num_sms * 32;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        k<<<(int)blocks, threads, 0, p.stream>>>(a);
    }
    return cudaGetLastError();
}

template <typename K>
inline int multi_grid(K kernel, int threads, size_t smem, int num_sms)
{
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    return num_sms * (per < 1 ? 1 : per);
}

template <typename T, int DIM, int W>
cudaError_t spread_multi_w(const MultiLaunch &ml)
{
    const auto *args = reinterpret_cast<const KArgs<T> *>(ml.args);
    count_launch();
    if (ml.method == NUFFT_METHOD_SM && ml.variant > 0) {
        if constexpr (DIM == 2) {
            const size_t wb = sweep_bytes<T, W, 32>(ml.m1max);
            const size_t per = args_slot<T>() + wb;
            int nw = 8;
            while (nw > 1 && (size_t)nw * per > ml.smem_optin) --nw;
            const size_t smem = per * nw;
            auto launch = [&](auto k, int lanes_wb) -> cudaError_t {
                if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
                k<<<multi_grid(k, nw * 32, smem, ml.num_sms), nw * 32, smem, ml.stream>>>(
                    args, ml.workoff, ml.nplans, lanes_wb);
                return cudaGetLastError();
            };
            // the staging slots of the widest sub-warp form bound the narrower ones
            if (ml.variant == 8) return launch(spread_sweep2_multi_kernel<T, W, 8>, (int)wb);
            if (ml.variant == 16) return launch(spread_sweep2_multi_kernel<T, W, 16>, (int)wb);
            return launch(spread_sweep2_multi_kernel<T, W, 32>, (int)wb);
        } else if constexpr (sizeof(T) == 4 && W <= 8) {
            // the group's widest row range bounds every member's staging
            auto launch = [&](auto k, size_t wb, int threads) -> cudaError_t {
                const size_t per = args_slot<T>() + wb;
                int nw = threads / 32;
                while (nw > 1 && (size_t)nw * per > ml.smem_optin) --nw;
                const size_t smem = per * nw;
                if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
                k<<<multi_grid(k, nw * 32, smem, ml.num_sms), nw * 32, smem, ml.stream>>>(
                    args, ml.workoff, ml.nplans, (int)wb);
                return cudaGetLastError();
            };
            if (ml.variant == 1)
                return launch(spread_sweep3_multi_kernel<T, W, 1, 32>, sweep3_bytes<T, W, 1, 32>(ml.m1max), 128);
            if (ml.variant == 2)
                return launch(spread_sweep3_multi_kernel<T, W, 2, 32>, sweep3_bytes<T, W, 2, 32>(ml.m1max), 128);
            if (ml.variant == 5)
                return launch(spread_sweep3_multi_kernel<T, W, 1, 16>, planes3_bytes<W, 1>(ml.m1max), 128);
            return launch(spread_sweep3_multi_kernel<T, W, 2, 16>, planes3_bytes<W, 2>(ml.m1max), 128);
        }
    }
    if (ml.method == NUFFT_METHOD_GM) {
        auto k = gm_multi_kernel<T, DIM, W, true>;
        k<<<multi_grid(k, ml.threads, 0, ml.num_sms), ml.threads, 0, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    } else if (ml.method == NUFFT_METHOD_SM) {
        auto k = spread_sm_multi_kernel<T, DIM, W>;
        if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
        k<<<multi_grid(k, ml.threads, ml.smem, ml.num_sms), ml.threads, ml.smem, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    } else {
        auto k = spread_gmsort_multi_kernel<T, DIM, W>;
        k<<<multi_grid(k, ml.threads, 0, ml.num_sms), ml.threads, 0, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    }
    return cudaGetLastError();
}

template <typename T, int DIM, int W>
cudaError_t interp_multi_w(const MultiLaunch &ml)
{
    using C = typename cplx<T>::type;
    const auto *args = reinterpret_cast<const KArgs<T> *>(ml.args);
    count_launch();
    if constexpr (DIM == 3 && sizeof(T) == 4 && W <= 8) {
        if (ml.method == NUFFT_METHOD_SM && (ml.variant == 5 || ml.variant == 6)) {
            const size_t wb = ml.variant == 5 ? iplanes3_bytes<W, 1>(ml.m1max)
                                              : iplanes3_bytes<W, 2>(ml.m1max);
            const size_t per = args_slot<T>() + wb;
            int nw = 4;
            while (nw > 1 && (size_t)nw * per > ml.smem_optin) --nw;
            const size_t smem = per * nw;
            auto launch = [&](auto k) -> cudaError_t {
                if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
                k<<<multi_grid(k, nw * 32, smem, ml.num_sms), nw * 32, smem, ml.stream>>>(
                    args, ml.workoff, ml.nplans, (int)wb);
                return cudaGetLastError();
            };
            return ml.variant == 5 ? launch(interp_planes3_multi_kernel<T, W, 1>)
                                   : launch(interp_planes3_multi_kernel<T, W, 2>);
        }
    }
    if (ml.method == NUFFT_METHOD_SM && DIM == 2) {
        const size_t wb = interp2_warp_bytes<T>(ml.tile, 1);
        const size_t per = args_slot<T>() + wb;
        int nw = 8;
        while (nw > 1 && (size_t)nw * per > ml.smem_optin) --nw;
        if ((size_t)nw * per <= ml.smem_optin) {
            const size_t smem = per * nw;
            auto k = interp_warp2_multi_kernel<T, W>;
            if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
            k<<<multi_grid(k, nw * 32, smem, ml.num_sms), nw * 32, smem, ml.stream>>>(
                args, ml.workoff, ml.nplans, (int)wb);
            return cudaGetLastError();
        }
    }
    if (ml.method == NUFFT_METHOD_GM) {
        auto k = gm_multi_kernel<T, DIM, W, false>;
        k<<<multi_grid(k, ml.threads, 0, ml.num_sms), ml.threads, 0, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    } else if (ml.method == NUFFT_METHOD_SM) {
        const size_t smem = args_slot<T>() + sizeof(C) * (size_t)ml.tile;
        auto k = interp_lane_multi_kernel<T, DIM, W, true>;
        if (cudaError_t ea = allow_max_smem((const void *)k)) return ea;
        k<<<multi_grid(k, ml.threads, smem, ml.num_sms), ml.threads, smem, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    } else {
        const size_t smem = args_slot<T>();
        auto k = interp_lane_multi_kernel<T, DIM, W, false>;
        k<<<multi_grid(k, ml.threads, smem, ml.num_sms), ml.threads, smem, ml.stream>>>(
            args, ml.workoff, ml.nplans);
    }
    return cudaGetLastError();
}

#define NUFFT_W_SWITCH_ON(WV, FN, T, DIM, ...)                                \
    switch (WV) {                                                             \
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

// One translation unit per (T, DIM) defines spread_<tag>, interp_<tag> and
// their multi-plan (batched) forms.
#define NUFFT_INSTANTIATE_SI(T, DIM, TAG)                                     \
    cudaError_t spread_##TAG(Plan &p, const void *c)                          \
    {                                                                         \
        NUFFT_W_SWITCH(spread_w, T, DIM, p, c)                                \
    }                                                                         \
    cudaError_t interp_##TAG(Plan &p, void *c)                                \
    {                                                                         \
        NUFFT_W_SWITCH(interp_w, T, DIM, p, c)                                \
    }                                                                         \
    cudaError_t spread_multi_##TAG(const MultiLaunch &ml)                     \
    {                                                                         \
        NUFFT_W_SWITCH_ON(ml.w, spread_multi_w, T, DIM, ml)                   \
    }                                                                         \
    cudaError_t interp_multi_##TAG(const MultiLaunch &ml)                     \
    {                                                                         \
        NUFFT_W_SWITCH_ON(ml.w, interp_multi_w, T, DIM, ml)                   \
    }

}  // namespace nufft
