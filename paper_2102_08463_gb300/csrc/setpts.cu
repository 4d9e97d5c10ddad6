// setpts.cu -- bin-sort of the nonuniform points (Sec. 4.1, GM-sort and SM
// step 1): the bin of every point, per-bin counts, a permutation t listing the
// points bin by bin (increasing original index inside a bin, unless the plan
// asks for shared-atomic order), the subproblem list (runs of at most M_sub
// points of one bin) and a packed record of each point's kernel offsets.
//
// Two sort paths, both giving the same t in index order:
//   counting sort (bins fit in shared memory): each CTA owns a contiguous chunk
//     of points and histograms its bins in shared memory into row b of a
//     CTAs x bins matrix; a prefix over the CTAs of each bin (which also sums
//     groups of 32 bins) and one offsets kernel (bin starts from those sums and
//     a block scan, plus the subproblem list) give every CTA the first output
//     slot of each of its bins; the CTA's points then claim slots in index
//     order (or, on request, in shared-atomic order).
//   LSD radix sort (many bins): 8-bit digits, per-CTA digit histograms, a scan
//     of the digit x CTA matrix, ranked scatter; every pass is stable.
// A last pass writes every point's packed record in t order (coordinates
// gathered through t), so that the spreading and interpolation kernels read
// the records of a subproblem as one contiguous run.
#include "nufft_internal.cuh"

namespace nufft {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanSeg = kScanThreads * kScanItems;   // elements per scan block

// ---------------------------------------------------------------------------
// Multi-block exclusive scan of int32 (three kernels: reduce, scan of block
// sums, rescan with offsets).  in may equal out.  *total gets the sum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int &block_total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) warp_sums[warp] = s;
    __syncthreads();
    if (warp == 0) {
        int ws = lane < nwarps ? warp_sums[lane] : 0;
        int wsc = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(kFull, wsc, o);
            if (lane >= o) wsc += t;
        }
        if (lane < nwarps) warp_sums[lane] = wsc - ws;
        if (lane == nwarps - 1) warp_sums[32] = wsc;
    }
    __syncthreads();
    int excl = warp_sums[warp] + s - v;
    block_total = warp_sums[32];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const int32_t *__restrict__ in, int64_t L, int32_t *__restrict__ part)
{
    __shared__ int red[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanSeg;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < L) s += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// One block scans the block sums in rounds of blockDim.
__global__ void __launch_bounds__(kScanThreads)
scan_partials_kernel(int32_t *part, int64_t nparts, int32_t *total)
{
    __shared__ int ws[33];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nparts; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int v = i < nparts ? part[i] : 0;
        int bt;
        int e = block_exclusive_scan(v, ws, bt);
        if (i < nparts) part[i] = carry + e;
        __syncthreads();
        if (threadIdx.x == 0) carry += bt;
        __syncthreads();
    }
    if (total != nullptr && threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_down_kernel(const int32_t *in, int32_t *out, int64_t L, const int32_t *__restrict__ part)
{
    __shared__ int ws[33];
    const int64_t base = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < L) ? in[base + k] : 0;
        tsum += v[k];
    }
    int bt;
    int run = part[blockIdx.x] + block_exclusive_scan(tsum, ws, bt);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < L) out[base + k] = run;
        run += v[k];
    }
}

// ---------------------------------------------------------------------------
// Bin of a point (Sec. 4.1 bin rule, integer position rule of nufft_internal.cuh).
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__device__ __forceinline__ int bin_of_v(T xv, T yv, T zv, int3 n, int3 m, int3 nb)
{
    int lx = (int)__umul64hi(period_fraction(xv), (uint64_t)n.x);
    int ly = DIM >= 2 ? (int)__umul64hi(period_fraction(yv), (uint64_t)n.y) : 0;
    int bz = 0;
    if (DIM == 3) bz = (int)__umul64hi(period_fraction(zv), (uint64_t)n.z) / m.z;
    return lx / m.x + nb.x * (ly / m.y + nb.y * bz);
}

template <typename T, int DIM>
__device__ __forceinline__ int bin_of(const T *x, const T *y, const T *z, int64_t j, int3 n,
                                      int3 m, int3 nb)
{
    return bin_of_v<T, DIM>(x[j], DIM >= 2 ? y[j] : (T)0, DIM == 3 ? z[j] : (T)0, n, m, nb);
}

template <typename T> __device__ __forceinline__ uint32_t unpack_word_t(T v);
template <> __device__ __forceinline__ uint32_t unpack_word_t<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ uint32_t unpack_word_t<double>(double v)
{
    return (uint32_t)__double_as_longlong(v);
}
template <typename T> __device__ __forceinline__ T packed_word(uint32_t v);
template <> __device__ __forceinline__ float packed_word<float>(uint32_t v) { return __uint_as_float(v); }
template <> __device__ __forceinline__ double packed_word<double>(uint32_t v)
{
    return __longlong_as_double((long long)v);
}

// Packed record of a point at (xv, yv, zv): kernel offsets and the window start
// relative to the padded origin of the point's own bin (bin origin - floor(w/2)),
// 10 bits per axis.
template <typename T, int DIM>
__device__ __forceinline__ typename rec4<T>::type make_record_v(T xv, T yv, T zv, int3 n, int3 m,
                                                                int w)
{
    const int P = pad_lo(w);
    AxisPos<T> px = axis_position<T>(period_fraction(xv), n.x, w);
    uint32_t sx = (uint32_t)(px.l0 - ((px.l / m.x) * m.x - P));
    uint32_t sy = 0;
    T dy = 0, dz = 0;
    if (DIM >= 2) {
        AxisPos<T> py = axis_position<T>(period_fraction(yv), n.y, w);
        sy = (uint32_t)(py.l0 - ((py.l / m.y) * m.y - P));
        dy = py.delta;
    }
    uint32_t sz = 0;
    if (DIM == 3) {
        AxisPos<T> pz = axis_position<T>(period_fraction(zv), n.z, w);
        sz = (uint32_t)(pz.l0 - ((pz.l / m.z) * m.z - P));
        dz = pz.delta;
    }
    typename rec4<T>::type r;
    r.x = px.delta;
    r.y = dy;
    r.z = dz;
    r.w = packed_word<T>(sx | (sy << 10) | (sz << 20));
    return r;
}

// ---------------------------------------------------------------------------
// Counting sort, pass 1: keys and per-CTA bin histograms, stored CTA-major
// (mat[cta * nbins + bin], coalesced).  Four points per thread per round keep
// several loads in flight.
// ---------------------------------------------------------------------------
constexpr int kCountThreads = 1024;
constexpr int kCountUnroll = 4;

template <typename T, int DIM>
__global__ void __launch_bounds__(kCountThreads)
count_kernel(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z, int64_t M,
             int64_t chunk, int3 n, int3 m, int3 nb, int nbins, int32_t *__restrict__ keys,
             int32_t *__restrict__ mat)
{
    extern __shared__ int hist[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(beg + chunk, M);
    const int64_t step = (int64_t)blockDim.x * kCountUnroll;
    for (int64_t j0 = beg + threadIdx.x; j0 < end; j0 += step) {
        int key[kCountUnroll];
        T xv[kCountUnroll], yv[kCountUnroll], zv[kCountUnroll];
#pragma unroll
        for (int k = 0; k < kCountUnroll; ++k) {
            const int64_t j = j0 + (int64_t)k * blockDim.x;
            key[k] = -1;
            xv[k] = yv[k] = zv[k] = (T)0;
            if (j < end) {
                xv[k] = x[j];
                if (DIM >= 2) yv[k] = y[j];
                if (DIM == 3) zv[k] = z[j];
                key[k] = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < kCountUnroll; ++k) {
            if (key[k] >= 0) {
                const int64_t j = j0 + (int64_t)k * blockDim.x;
                const int b = bin_of_v<T, DIM>(xv[k], yv[k], zv[k], n, m, nb);
                keys[j] = b;
                atomicAdd(&hist[b], 1);
            }
        }
    }
    __syncthreads();
    int32_t *col = mat + (int64_t)blockIdx.x * nbins;
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) col[i] = hist[i];
}

// Counting sort, pass 2: per bin, exclusive prefix over the CTAs (in place) and
// the bin total; per group of 32 bins, the sums of the counts and of the
// subproblem counts ceil(count / msub) (agg, skipped when null).
constexpr int kColWarps = 8;

// 32 bins per CTA (lane = bin, coalesced rows); each warp owns a slice of the
// CTA rows: slice sums, exclusive prefix over slices, then a rescan of the slice.
__global__ void __launch_bounds__(kColWarps * 32)
column_scan_kernel(int32_t *__restrict__ mat, int nbins, int nblk, int32_t *__restrict__ bincount,
                   int msub, int2 *__restrict__ agg)
{
    __shared__ int part[kColWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    const bool ok = b < nbins;
    const int r0 = (int)((int64_t)nblk * warp / kColWarps);
    const int r1 = (int)((int64_t)nblk * (warp + 1) / kColWarps);
    int s = 0;
    if (ok) {
#pragma unroll 4
        for (int r = r0; r < r1; ++r) s += mat[(int64_t)r * nbins + b];
    }
    part[warp][lane] = s;
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += part[w][lane];
    if (warp == kColWarps - 1) {
        const int cnt = ok ? off + s : 0;
        if (ok) bincount[b] = cnt;
        if (agg != nullptr) {
            int sc = cnt, sn = cnt / msub + (cnt % msub != 0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sc += __shfl_xor_sync(kFull, sc, o);
                sn += __shfl_xor_sync(kFull, sn, o);
            }
            if (lane == 0) agg[blockIdx.x] = make_int2(sc, sn);
        }
    }
    if (ok) {
        for (int r = r0; r < r1; ++r) {
            const int64_t i = (int64_t)r * nbins + b;
            const int v = mat[i];
            mat[i] = off;
            off += v;
        }
    }
}

// Counting sort, pass 2b: one thread per bin.  The exclusive prefix of the
// column-scan groups before the CTA (agg) plus a block scan of (count,
// subproblems) give each bin its first sorted slot (binstart) and its first
// subproblem; the bin writes its ceil(count / msub) subproblems (Sec. 4.1 SM
// step 1) and the last bin the total.
constexpr int kOffThreads = 256;
constexpr int kOffGroups = kOffThreads / 32;   // column-scan groups per CTA

__global__ void __launch_bounds__(kOffThreads)
bin_offsets_kernel(const int32_t *__restrict__ bincount, const int2 *__restrict__ agg, int nbins,
                   int msub, int32_t *__restrict__ binstart, int4 *__restrict__ subprob,
                   int32_t *__restrict__ nsub_total)
{
    __shared__ int2 red[kOffThreads / 32];
    __shared__ int2 wtot[kOffThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g0 = blockIdx.x * kOffGroups;
    const int b = blockIdx.x * kOffThreads + threadIdx.x;
    const int cnt = b < nbins ? bincount[b] : 0;
    const int ns = cnt / msub + (cnt % msub != 0);
    int pc = 0, pn = 0;
    for (int i = threadIdx.x; i < g0; i += kOffThreads) {
        const int2 a = agg[i];
        pc += a.x;
        pn += a.y;
    }
    int ic = cnt, in = ns;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pc += __shfl_xor_sync(kFull, pc, o);
        pn += __shfl_xor_sync(kFull, pn, o);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int tc = __shfl_up_sync(kFull, ic, o);
        const int tn = __shfl_up_sync(kFull, in, o);
        if (lane >= o) {
            ic += tc;
            in += tn;
        }
    }
    if (lane == 0) red[warp] = make_int2(pc, pn);
    if (lane == 31) wtot[warp] = make_int2(ic, in);
    __syncthreads();
    int sc = 0, sn = 0;
#pragma unroll
    for (int w = 0; w < kOffThreads / 32; ++w) {
        sc += red[w].x;
        sn += red[w].y;
        if (w < warp) {
            sc += wtot[w].x;
            sn += wtot[w].y;
        }
    }
    if (b < nbins) {
        const int start = sc + ic - cnt;
        const int first = sn + in - ns;
        binstart[b] = start;
        for (int k = 0; k < ns; ++k)
            subprob[first + k] = make_int4(b, start + k * msub, min(msub, cnt - k * msub), 0);
        if (b == nbins - 1) *nsub_total = first + ns;
    }
}

// Counting sort, pass 3: ranked scatter of t.  Each CTA loads its first output
// slot of every bin (prefix over the CTAs before it + bin start) into shared
// memory; its points then claim the next slots of their bins.  A tile is
// kRankU x 32 consecutive points per warp (warp w owns the w-th run of
// kRankU * 32); the keys of the next tile are loaded before the current tile's
// claims.
//   kOrdered (default): t lists every bin's points in increasing index.  Lanes
//     of a chunk of 32 with equal keys are grouped with __match_any_sync; one
//     leader per group claims the group's slots with one shared atomicAdd, and
//     the lanes take them in lane order.  Chunks claim in order (__syncwarp
//     between them) and warps take turns in warp order (one barrier per warp
//     per tile), so equal keys keep their index order.
//   kFilter (with kOrdered): match costs about one step per distinct key of
//     the chunk, and uniform points over many bins give 32 distinct keys.  So
//     each warp first hashes its keys into 256 byte buckets of its own (512
//     bytes of shared memory after the bin table: bucket owner, collision
//     mark): a lane alone in its bucket holds a key no other lane holds and is
//     its own group; only lanes in shared buckets (equal keys or hash
//     collisions) run match among themselves.
//   otherwise: every point claims its own slot with a shared atomicAdd, no
//     turns; a CTA's points of one bin fill its run of slots in atomic order.
constexpr int kRankU = 4;
constexpr size_t kFilterBytes = (size_t)(kCountThreads / 32) * 512;

template <bool kOrdered, bool kFilter = false>
__global__ void __launch_bounds__(kCountThreads)
rank_scatter_kernel(int64_t M, int64_t chunk, int nbins, const int32_t *__restrict__ keys,
                    const int32_t *__restrict__ mat, const int32_t *__restrict__ binstart,
                    int32_t *__restrict__ perm)
{
    extern __shared__ int run[];   // next output slot per bin for this CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int32_t *col = mat + (int64_t)blockIdx.x * nbins;
    uint8_t *owner = reinterpret_cast<uint8_t *>(run + nbins) + warp * 512;
    uint8_t *clash = owner + 256;
#pragma unroll 4
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) run[i] = col[i] + binstart[i];
    if (kFilter)
        for (int i = lane; i < 256; i += 32) clash[i] = 0;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(beg + chunk, M);
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t tile = (int64_t)nwarps * 32 * kRankU;
    const int64_t mine0 = (int64_t)warp * 32 * kRankU + lane;
    int key[kRankU], keyn[kRankU];
#pragma unroll
    for (int u = 0; u < kRankU; ++u) {
        const int64_t j = beg + mine0 + u * 32;
        key[u] = j < end ? keys[j] : -1;
    }
    for (int64_t t0 = beg; t0 < end; t0 += tile) {
#pragma unroll
        for (int u = 0; u < kRankU; ++u) {
            const int64_t j = t0 + tile + mine0 + u * 32;
            keyn[u] = j < end ? keys[j] : -1;
        }
        if (kOrdered) {
            unsigned peers[kRankU];
            int base[kRankU];
#pragma unroll
            for (int u = 0; u < kRankU; ++u) {
                base[u] = 0;
                if (kFilter) {
                    const unsigned h = ((unsigned)key[u] * 2654435761u) >> 24;   // 0..255
                    owner[h] = (uint8_t)lane;
                    __syncwarp();
                    const bool lost = owner[h] != (uint8_t)lane;
                    if (lost) clash[h] = 1;
                    __syncwarp();
                    const bool shared_bucket = clash[h] != 0;
                    __syncwarp();
                    if (lost) clash[h] = 0;                // the marks are clear again
                    __syncwarp();
                    const unsigned sm = __ballot_sync(kFull, shared_bucket);
                    peers[u] = shared_bucket ? __match_any_sync(sm, key[u]) : (1u << lane);
                } else {
                    peers[u] = __match_any_sync(kFull, key[u]);
                }
            }
            for (int wv = 0; wv < nwarps; ++wv) {
                if (warp == wv) {
#pragma unroll
                    for (int u = 0; u < kRankU; ++u) {
                        if (key[u] >= 0 && (peers[u] & lt_mask) == 0)
                            base[u] = atomicAdd(&run[key[u]], __popc(peers[u]));
                        __syncwarp();
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int u = 0; u < kRankU; ++u) {
                const int b = __shfl_sync(kFull, base[u], __ffs(peers[u]) - 1);
                if (key[u] >= 0)
                    perm[b + __popc(peers[u] & lt_mask)] = (int32_t)(t0 + mine0 + u * 32);
            }
        } else {
            int slot[kRankU];
#pragma unroll
            for (int u = 0; u < kRankU; ++u)
                slot[u] = key[u] >= 0 ? atomicAdd(&run[key[u]], 1) : 0;
#pragma unroll
            for (int u = 0; u < kRankU; ++u)
                if (key[u] >= 0) perm[slot[u]] = (int32_t)(t0 + mine0 + u * 32);
        }
#pragma unroll
        for (int u = 0; u < kRankU; ++u) key[u] = keyn[u];
    }
}

// Packed records in t order: recs[i] = record of point perm[i] (gathered
// coordinates); in 2D the z slot carries the point's index.
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
records_from_perm_kernel(const int32_t *__restrict__ perm, int64_t M, const T *__restrict__ x,
                         const T *__restrict__ y, const T *__restrict__ z, int3 n, int3 m, int w,
                         typename rec4<T>::type *__restrict__ recs)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = perm[i];
        typename rec4<T>::type r =
            make_record_v<T, DIM>(x[j], DIM >= 2 ? y[j] : (T)0, DIM == 3 ? z[j] : (T)0, n, m, w);
        if (DIM != 3) r.z = packed_word<T>((uint32_t)j);
        recs[i] = r;
    }
}

// 3D plane-split sweeps: the records of every subproblem put in order of window
// start row (stable: t order inside a row), out of place from the t-ordered
// records into the plan's second record buffer, with the point indices moved
// alike into rorder.  One warp per subproblem: the start rows are counted
// (warp-aggregated shared atomics), prefix-summed, and every record is copied to
// its position.  The records are read in order (coalesced) twice; t itself is
// not touched.
constexpr int kRowWarps = 8;

template <typename T>
__global__ void __launch_bounds__(kRowWarps * 32)
row_order_kernel(const typename rec4<T>::type *__restrict__ recs_in,
                 const int32_t *__restrict__ perm, const int4 *__restrict__ subprob,
                 const int32_t *__restrict__ nsub, int nkeys,
                 typename rec4<T>::type *__restrict__ recs_out, int32_t *__restrict__ rorder)
{
    extern __shared__ int cnt_all[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *cnt = cnt_all + warp * (nkeys + 1);
    const unsigned lt = (1u << lane) - 1u;
    const int ns = *nsub;
    for (int sp = blockIdx.x * kRowWarps + warp; sp < ns; sp += gridDim.x * kRowWarps) {
        const int4 sub = subprob[sp];
        const typename rec4<T>::type *in = recs_in + sub.y;
        for (int i = lane; i <= nkeys; i += 32) cnt[i] = 0;
        __syncwarp();
        for (int b = 0; b < sub.z; b += 32) {
            const int i = b + lane;
            const int key = i < sub.z ? (int)((unpack_word_t<T>(in[i].w) >> 10) & 1023u) : 0x7fffffff;
            const unsigned peers = __match_any_sync(kFull, key);
            if (i < sub.z && (peers & lt) == 0) atomicAdd(&cnt[key + 1], __popc(peers));
        }
        __syncwarp();
        int running = 0;
        for (int i0 = 0; i0 <= nkeys; i0 += 32) {
            const int i = i0 + lane;
            int v = i <= nkeys ? cnt[i] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, v, o);
                if (lane >= o) v += t;
            }
            if (i <= nkeys) cnt[i] = running + v;
            running += __shfl_sync(kFull, v, 31);
        }
        __syncwarp();
        for (int b = 0; b < sub.z; b += 32) {
            const int i = b + lane;
            typename rec4<T>::type r;
            int key = 0x7fffffff, j = 0;
            if (i < sub.z) {
                r = in[i];
                j = perm[sub.y + i];
                key = (int)((unpack_word_t<T>(r.w) >> 10) & 1023u);
            }
            const unsigned peers = __match_any_sync(kFull, key);
            const int leader = __ffs(peers) - 1;
            int pos = 0;
            if (i < sub.z && lane == leader) pos = atomicAdd(&cnt[key], __popc(peers));
            pos = __shfl_sync(kFull, pos, leader) + __popc(peers & lt);
            if (i < sub.z) {
                recs_out[sub.y + pos] = r;
                rorder[sub.y + pos] = j;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// LSD radix path (bins too many for shared memory).
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void keys_kernel(const T *__restrict__ x, const T *__restrict__ y,
                            const T *__restrict__ z, int64_t M, int3 n, int3 m, int3 nb,
                            int32_t *__restrict__ keys)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const T xv = x[j], yv = DIM >= 2 ? y[j] : (T)0, zv = DIM == 3 ? z[j] : (T)0;
        keys[j] = bin_of_v<T, DIM>(xv, yv, zv, n, m, nb);
    }
}

__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const int32_t *__restrict__ keys, int64_t M, int64_t chunk, int shift,
                  int32_t *__restrict__ mat)
{
    __shared__ int h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(beg + chunk, M);
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x)
        mat[(int64_t)i * gridDim.x + blockIdx.x] = h[i];
}

__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const int32_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in,
                     int64_t M, int64_t chunk, int shift, const int32_t *__restrict__ mat,
                     int32_t *__restrict__ keys_out, int32_t *__restrict__ vals_out)
{
    constexpr int NW = kSortThreads / 32;
    __shared__ int run[kRadix];
    __shared__ int wcount[NW][kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = mat[(int64_t)tid * gridDim.x + blockIdx.x];   // blockDim == kRadix
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(beg + chunk, M);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t tile = beg; tile < end; tile += kSortThreads) {
#pragma unroll
        for (int w = 0; w < NW; ++w) wcount[w][tid] = 0;
        __syncthreads();
        const int64_t i = tile + tid;
        int key = 0, val = 0, d = -1;
        if (i < end) {
            key = keys_in[i];
            val = vals_in ? vals_in[i] : (int)i;
            d = (key >> shift) & (kRadix - 1);
        }
        const unsigned peers = __match_any_sync(kFull, d);
        const int lrank = __popc(peers & lt_mask);
        if (d >= 0 && lrank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        int s = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int cnt = wcount[w][tid];
            wcount[w][tid] = s;
            s += cnt;
        }
        __syncthreads();
        if (d >= 0) {
            const int pos = run[d] + wcount[warp][d] + lrank;
            if (keys_out) keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        run[tid] += s;
        __syncthreads();
    }
}

__global__ void iota_kernel(int32_t *out, int64_t M)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

__global__ void bin_histogram_kernel(const int32_t *__restrict__ keys, int64_t M,
                                     int32_t *__restrict__ bincount)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&bincount[keys[i]], 1);
}

// ---------------------------------------------------------------------------
// Subproblems (Sec. 4.1 SM step 1): bin b gets ceil(count_b / msub) runs.
// ---------------------------------------------------------------------------
__global__ void subs_per_bin_kernel(const int32_t *__restrict__ bincount, int64_t nbins, int msub,
                                    int32_t *__restrict__ nsubs)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
         b += (int64_t)gridDim.x * blockDim.x)
        nsubs[b] = bincount[b] / msub + (bincount[b] % msub != 0);
}

__global__ void write_subs_kernel(const int32_t *__restrict__ bincount,
                                  const int32_t *__restrict__ binstart,
                                  const int32_t *__restrict__ suboff, int64_t nbins, int msub,
                                  int4 *__restrict__ subprob)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int cnt = bincount[b], st = binstart[b], so = suboff[b];
        for (int off = 0, k = 0; off < cnt; off += msub, ++k)
            subprob[so + k] = make_int4((int)b, st + off, min(msub, cnt - off), 0);
    }
}

inline int grid_for(int64_t work, int threads, int num_sms)
{
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

namespace {

// debug_checks: every coordinate finite and inside [-3 pi, 3 pi] (NaN fails the
// comparison), and t a permutation of 0 .. M-1 (each index seen once: seen[]
// holds a count per index).  Failures set bit 0 (coordinates) or bit 1 (t) of
// *status; nothing traps.
template <typename T>
__global__ void check_coords_kernel(const T *__restrict__ x, const T *__restrict__ y,
                                    const T *__restrict__ z, int64_t M, int32_t *status)
{
    const T lim = (T)(3.0 * 3.14159265358979323846);
    bool bad = false;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        bad |= !(x[j] >= -lim && x[j] <= lim) || (y != nullptr && !(y[j] >= -lim && y[j] <= lim)) ||
               (z != nullptr && !(z[j] >= -lim && z[j] <= lim));
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(status, 1);
}

__global__ void check_perm_kernel(const int32_t *__restrict__ perm, int64_t M,
                                  int32_t *__restrict__ seen, int32_t *status)
{
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = perm[i];
        if (v < 0 || v >= M) bad = true;
        else if (atomicAdd(&seen[v], 1) != 0) bad = true;
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(status, 2);
}

}  // namespace

cudaError_t launch_checks(Plan &p, const void *x, const void *y, const void *z)
{
    if (!p.dstatus || p.M == 0) return cudaSuccess;
    const int g = grid_for(p.M, 256, p.num_sms);
    count_launch(2);
    if (p.prec == 0)
        check_coords_kernel<float><<<g, 256, 0, p.stream>>>(
            (const float *)x, p.dim >= 2 ? (const float *)y : nullptr,
            p.dim == 3 ? (const float *)z : nullptr, p.M,
            p.dstatus);
    else
        check_coords_kernel<double><<<g, 256, 0, p.stream>>>(
            (const double *)x, p.dim >= 2 ? (const double *)y : nullptr,
            p.dim == 3 ? (const double *)z : nullptr, p.M,
            p.dstatus);
    if (p.method == NUFFT_METHOD_GM) return cudaGetLastError();   // GM sorts nothing
    cudaError_t e = cudaMemsetAsync(p.keys_alt, 0, sizeof(int32_t) * p.M, p.stream);
    if (e != cudaSuccess) return e;
    check_perm_kernel<<<g, 256, 0, p.stream>>>(p.perm, p.M, p.keys_alt, p.dstatus);
    return cudaGetLastError();
}

// Exclusive scan of L int32 (in may equal out); p.scan_part holds the block sums.
cudaError_t launch_scan(Plan &p, const int32_t *in, int32_t *out, int64_t L, int32_t *total)
{
    if (L <= 0) return cudaSuccess;
    const int64_t nb = (L + kScanSeg - 1) / kScanSeg;
    count_launch(3);
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, p.stream>>>(in, L, p.scan_part);
    scan_partials_kernel<<<1, kScanThreads, 0, p.stream>>>(p.scan_part, nb, total);
    scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, p.stream>>>(in, out, L, p.scan_part);
    return cudaGetLastError();
}

int64_t scan_parts_needed(int64_t L) { return (L + kScanSeg - 1) / kScanSeg + 1; }

// Blocks of the counting sort for M points and nbins bins (0 = use the radix
// path): one CTA of kCountThreads per SM, fewer for small M (at least 8192
// points a CTA).  One full-size CTA per SM keeps the CTAs x bins matrix (written
// by the count, read and rewritten by the column scan, read by the scatter) and
// each CTA's per-bin setup small against its chunk of points: measured on 2D
// 2048^2 with 10 x 16 bins, M = 4.2M, setpts 0.103 ms with two 512-thread CTAs
// per SM against 0.090 ms with one of 1024.
int counting_sort_blocks(const Plan &p, int64_t M)
{
    const size_t smem = (size_t)p.nbins * sizeof(int32_t);
    if (smem > (size_t)p.smem_optin) return 0;
    int64_t blocks = p.num_sms;
    const int64_t by_size = (M + 8191) / 8192;
    if (blocks > by_size) blocks = by_size;
    return (int)(blocks < 1 ? 1 : blocks);
}

int radix_sort_blocks(const Plan &p, int64_t M)
{
    int64_t blocks = (M + 4095) / 4096;
    if (blocks > (int64_t)p.num_sms * 2) blocks = (int64_t)p.num_sms * 2;
    return (int)(blocks < 1 ? 1 : blocks);
}

namespace {

// Packed records in t order: recs[i] = record of point t[i] (coordinates
// gathered through t: they were read moments before by the counting pass and
// sit in L2), written in order so that the spreading and interpolation kernels
// read every subproblem's records as one contiguous run.
template <typename T>
cudaError_t launch_records(Plan &p, const T *x, const T *y, const T *z,
                           typename rec4<T>::type *recs)
{
    const int3 n = make_int3((int)p.nf[0], (int)p.nf[1], (int)p.nf[2]);
    const int3 m = make_int3(p.m[0], p.m[1], p.m[2]);
    int64_t g = (p.M + 255) / 256;
    const int64_t cap = (int64_t)p.num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    count_launch();
    auto k = p.dim == 1 ? records_from_perm_kernel<T, 1>
             : p.dim == 2 ? records_from_perm_kernel<T, 2> : records_from_perm_kernel<T, 3>;
    k<<<(unsigned)g, 256, 0, p.stream>>>(p.perm, p.M, x, y, z, n, m, p.w, recs);
    return cudaGetLastError();
}

// Records in t order; for the 3D plane-split sweeps then ordered by start row
// inside every subproblem (row_order_kernel, into the second record buffer,
// which becomes the plan's records).
template <typename T>
cudaError_t finish_records(Plan &p, const T *x, const T *y, const T *z,
                           typename rec4<T>::type *recs)
{
    p.row_ordered = false;
    cudaError_t e = launch_records<T>(p, x, y, z, recs);
    if (e != cudaSuccess || p.dim != 3 || sizeof(T) != 4 || planes3_form(p) == 0) return e;
    const int nkeys = p.m[1] + 1;
    const size_t smem = sizeof(int) * (size_t)(nkeys + 1) * kRowWarps;
    auto k = row_order_kernel<T>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRowWarps * 32, smem);
    const int grid = p.num_sms * (per_sm < 1 ? 1 : per_sm);
    auto *out = reinterpret_cast<typename rec4<T>::type *>(p.recs2);
    count_launch();
    k<<<grid, kRowWarps * 32, smem, p.stream>>>(recs, p.perm, p.subprob, p.nsub, nkeys, out,
                                                 p.rorder);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void *tmp = p.recs;                            // the ordered records become the plan's
    p.recs = p.recs2;
    p.recs2 = tmp;
    p.row_ordered = true;
    return cudaSuccess;
}

template <typename T>
cudaError_t setpts_impl(Plan &p, const T *x, const T *y, const T *z)
{
    cudaStream_t st = p.stream;
    const int64_t M = p.M;
    const int3 n = make_int3((int)p.nf[0], (int)p.nf[1], (int)p.nf[2]);
    const int3 m = make_int3(p.m[0], p.m[1], p.m[2]);
    const int3 nb = make_int3(p.nb[0], p.nb[1], p.nb[2]);
    const int nbins = (int)p.nbins;
    auto *recs = reinterpret_cast<typename rec4<T>::type *>(p.recs);
    cudaError_t e = cudaSuccess;
    if (M == 0) {
        e = cudaMemsetAsync(p.bincount, 0, sizeof(int32_t) * p.nbins, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(p.nsub, 0, sizeof(int32_t), st);
        return e;
    }
    const int cblk = counting_sort_blocks(p, M);
    if (cblk > 0) {
        const int64_t chunk = (M + cblk - 1) / cblk;
        const size_t smem = (size_t)nbins * sizeof(int32_t);
        auto kc = p.dim == 1 ? count_kernel<T, 1> : p.dim == 2 ? count_kernel<T, 2> : count_kernel<T, 3>;
        const bool filter = !p.unordered_bins && smem + kFilterBytes <= (size_t)p.smem_optin;
        auto ks = p.unordered_bins ? rank_scatter_kernel<false>
                                   : filter ? rank_scatter_kernel<true, true> : rank_scatter_kernel<true>;
        e = allow_max_smem((const void *)kc);
        if (e == cudaSuccess) e = allow_max_smem((const void *)ks);
        if (e != cudaSuccess) return e;
        int2 *agg = reinterpret_cast<int2 *>(p.scan_part);   // (nbins + 31) / 32 groups
        count_launch(4);
        kc<<<cblk, kCountThreads, smem, st>>>(x, y, z, M, chunk, n, m, nb, nbins, p.keys, p.mat);
        column_scan_kernel<<<(nbins + 31) / 32, kColWarps * 32, 0, st>>>(p.mat, nbins, cblk,
                                                                         p.bincount, p.msub, agg);
        bin_offsets_kernel<<<(nbins + kOffThreads - 1) / kOffThreads, kOffThreads, 0, st>>>(
            p.bincount, agg, nbins, p.msub, p.binstart, p.subprob, p.nsub);
        ks<<<cblk, kCountThreads, smem + (filter ? kFilterBytes : 0), st>>>(M, chunk, nbins, p.keys,
                                                                           p.mat, p.binstart, p.vals);
        p.perm = p.vals;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return finish_records<T>(p, x, y, z, recs);
    } else {
        const int g = grid_for(M, 256, p.num_sms);
        count_launch();
        auto kk = p.dim == 1 ? keys_kernel<T, 1> : p.dim == 2 ? keys_kernel<T, 2> : keys_kernel<T, 3>;
        kk<<<g, 256, 0, st>>>(x, y, z, M, n, m, nb, p.keys);
        e = cudaMemsetAsync(p.bincount, 0, sizeof(int32_t) * p.nbins, st);
        if (e != cudaSuccess) return e;
        count_launch();
        bin_histogram_kernel<<<g, 256, 0, st>>>(p.keys, M, p.bincount);
        int bits = 0;
        while (bits < 31 && ((int64_t)1 << bits) < p.nbins) ++bits;
        const int passes = (bits + kRadixBits - 1) / kRadixBits;
        int32_t *kbuf[2] = {p.keys, p.keys_alt};
        int32_t *vbuf[2] = {p.vals, p.vals_alt};
        const int rblk = radix_sort_blocks(p, M);
        const int64_t chunk = (M + rblk - 1) / rblk;
        int cur = 0;
        if (passes == 0) {
            count_launch();
            iota_kernel<<<g, 256, 0, st>>>(p.vals, M);
        }
        for (int ps = 0; ps < passes; ++ps) {
            const int shift = ps * kRadixBits;
            const bool last = ps == passes - 1;
            count_launch();
            radix_hist_kernel<<<rblk, kSortThreads, 0, st>>>(kbuf[cur], M, chunk, shift, p.mat);
            e = launch_scan(p, p.mat, p.mat, (int64_t)kRadix * rblk, nullptr);
            if (e != cudaSuccess) return e;
            count_launch();
            radix_scatter_kernel<<<rblk, kSortThreads, 0, st>>>(
                kbuf[cur], ps == 0 ? nullptr : vbuf[cur], M, chunk, shift, p.mat,
                last ? nullptr : kbuf[cur ^ 1], vbuf[cur ^ 1]);
            cur ^= 1;
        }
        p.perm = vbuf[cur];
        e = launch_scan(p, p.bincount, p.binstart, nbins, nullptr);
        if (e != cudaSuccess) return e;
        count_launch();
        subs_per_bin_kernel<<<grid_for(nbins, 256, p.num_sms), 256, 0, st>>>(p.bincount, nbins,
                                                                           p.msub, p.scan_tmp);
    }
    e = launch_scan(p, p.scan_tmp, p.scan_tmp, nbins, p.nsub);
    if (e != cudaSuccess) return e;
    count_launch();
    write_subs_kernel<<<grid_for(nbins, 256, p.num_sms), 256, 0, st>>>(
        p.bincount, p.binstart, p.scan_tmp, nbins, p.msub, p.subprob);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return finish_records<T>(p, x, y, z, recs);
}

}  // namespace

cudaError_t launch_setpts(Plan &p, const void *x, const void *y, const void *z)
{
    if (p.prec == 0)
        return setpts_impl<float>(p, (const float *)x, (const float *)y, (const float *)z);
    return setpts_impl<double>(p, (const double *)x, (const double *)y, (const double *)z);
}

// ---------------------------------------------------------------------------
// Bin-sort into caller-provided scratch (used by the allocation-free entry
// point): the counting-sort path above without the packed records.
// ---------------------------------------------------------------------------
namespace {

template <typename T, int DIM>
__global__ void __launch_bounds__(kCountThreads)
count_keys_kernel(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z,
                  int64_t M, int64_t chunk, int3 n, int3 m, int3 nb, int nbins,
                  int32_t *__restrict__ keys, int32_t *__restrict__ mat)
{
    extern __shared__ int hist[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(beg + chunk, M);
    for (int64_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
        const int b = bin_of<T, DIM>(x, y, z, j, n, m, nb);
        keys[j] = b;
        atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    int32_t *col = mat + (int64_t)blockIdx.x * nbins;
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) col[i] = hist[i];
}

template <typename T>
cudaError_t binsort_into_impl(const BinsortScratch &s, int dim, int64_t M, const T *x, const T *y,
                              const T *z, const int64_t *nf, const int *bins, int32_t *perm,
                              int32_t *bincount, cudaStream_t st)
{
    int3 n = make_int3((int)nf[0], (int)nf[1], dim == 3 ? (int)nf[2] : 1);
    int3 m = make_int3(bins[0], bins[1], dim == 3 ? bins[2] : 1);
    int3 nb = make_int3((n.x + m.x - 1) / m.x, (n.y + m.y - 1) / m.y, (n.z + m.z - 1) / m.z);
    const int nbins = nb.x * nb.y * nb.z;
    const int64_t chunk = (M + s.nblk - 1) / s.nblk;
    const size_t smem = (size_t)nbins * sizeof(int32_t);
    auto kc = dim == 2 ? count_keys_kernel<T, 2> : count_keys_kernel<T, 3>;
    cudaError_t e = allow_max_smem((const void *)kc);
    if (e != cudaSuccess) return e;
    e = allow_max_smem((const void *)rank_scatter_kernel<true>);
    if (e != cudaSuccess) return e;
    count_launch(3);
    kc<<<s.nblk, kCountThreads, smem, st>>>(x, y, z, M, chunk, n, m, nb, nbins, s.keys, s.mat);
    column_scan_kernel<<<(nbins + 31) / 32, kColWarps * 32, 0, st>>>(s.mat, nbins, s.nblk, bincount,
                                                                     1, nullptr);
    Plan scan_plan;                 // only scan_part and stream are used by launch_scan
    scan_plan.stream = st;
    scan_plan.scan_part = s.scan_part;
    e = launch_scan(scan_plan, bincount, s.binstart, nbins, nullptr);
    if (e != cudaSuccess) return e;
    rank_scatter_kernel<true><<<s.nblk, kCountThreads, smem, st>>>(M, chunk, nbins, s.keys, s.mat,
                                                                   s.binstart, perm);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_binsort_into(const BinsortScratch &s, int prec, int dim, int64_t M,
                                const void *x, const void *y, const void *z, const int64_t *nf,
                                const int *bins, int32_t *perm, int32_t *bincount,
                                cudaStream_t st)
{
    if (prec == 0)
        return binsort_into_impl<float>(s, dim, M, (const float *)x, (const float *)y,
                                        (const float *)z, nf, bins, perm, bincount, st);
    return binsort_into_impl<double>(s, dim, M, (const double *)x, (const double *)y,
                                     (const double *)z, nf, bins, perm, bincount, st);
}

}  // namespace nufft
