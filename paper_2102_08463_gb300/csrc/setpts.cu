// setpts.cu -- bin-sort of the nonuniform points (Sec. 4.1, GM-sort and SM
// step 1): bin index per point, per-bin counts, a stable permutation t listing
// the points bin by bin, the subproblem list (runs of at most M_sub points of
// one bin) and a packed bin-ordered record of each point's kernel offsets.
//
// The permutation is a stable LSD radix sort of the bin keys written here:
// 8-bit digits, one histogram pass and one ranked scatter pass per digit.
// Within a tile the scatter ranks equal digits by (warp, lane) order using
// __match_any_sync, so equal keys keep their original order and t is unique.
#include "nufft_internal.cuh"

namespace nufft {

namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;          // one digit per thread in the scans below
constexpr int kScanThreads = 1024;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Bin key of every point (user order) and per-bin counts.
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void prep_keys_kernel(const T *__restrict__ x, const T *__restrict__ y,
                                 const T *__restrict__ z, int64_t M, int3 n, int3 m, int3 nb,
                                 int32_t *__restrict__ keys, int32_t *__restrict__ bincount)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // Warp-uniform loop: every lane of a warp runs the same iterations.
    const int64_t warp_base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (int64_t b = warp_base; b < M; b += stride) {
        int64_t j = b + lane;
        int key = -1;
        if (j < M) {
            int lx = (int)__umul64hi(period_fraction(x[j]), (uint64_t)n.x);
            int ly = (int)__umul64hi(period_fraction(y[j]), (uint64_t)n.y);
            int bz = 0;
            if (DIM == 3) {
                int lz = (int)__umul64hi(period_fraction(z[j]), (uint64_t)n.z);
                bz = lz / m.z;
            }
            key = lx / m.x + nb.x * (ly / m.y + nb.y * bz);
            keys[j] = key;
        }
        unsigned peers = __match_any_sync(kFull, key);
        if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&bincount[key], __popc(peers));
    }
}

// ---------------------------------------------------------------------------
// Radix pass, step 1: digit histogram of each block's contiguous chunk.
// hist is digit-major: hist[d * nblocks + block].
// ---------------------------------------------------------------------------
__global__ void radix_hist_kernel(const int32_t *__restrict__ keys, int64_t M, int64_t chunk,
                                  int shift, int32_t *__restrict__ hist)
{
    __shared__ int h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int64_t beg = (int64_t)blockIdx.x * chunk;
    int64_t end = min(beg + chunk, M);
    for (int64_t b = beg + (threadIdx.x & ~31); b < end; b += blockDim.x) {
        int64_t i = b + lane;
        int d = i < end ? ((keys[i] >> shift) & (kRadix - 1)) : -1;
        unsigned peers = __match_any_sync(kFull, d);
        if (d >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x)
        hist[(int64_t)i * gridDim.x + blockIdx.x] = h[i];
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum of L int32 values by one block (in may equal out);
// the grand total goes to *total when total is not null.  Each thread takes
// kScanItems consecutive values per round.
// ---------------------------------------------------------------------------
constexpr int kScanItems = 8;

__global__ void __launch_bounds__(kScanThreads)
scan_exclusive_kernel(const int32_t *in, int32_t *out, int64_t L, int32_t *total)
{
    __shared__ int warp_sums[kScanThreads / 32];
    __shared__ int carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int64_t per_round = (int64_t)blockDim.x * kScanItems;
    for (int64_t base = 0; base < L; base += per_round) {
        int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
        int v[kScanItems];
        int tsum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = (i0 + k < L) ? in[i0 + k] : 0;
            tsum += v[k];
        }
        int s = tsum;                             // inclusive warp scan of thread sums
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
            if (lane < nwarps) warp_sums[lane] = wsc - ws;   // exclusive over warps
        }
        __syncthreads();
        const int carry = carry_s;
        int run = carry + warp_sums[warp] + s - tsum;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (i0 + k < L) out[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = run;
        __syncthreads();
    }
    if (total != nullptr && threadIdx.x == 0) *total = carry_s;
}

// ---------------------------------------------------------------------------
// Radix pass, step 2: stable scatter.  Each block walks its chunk in tiles of
// blockDim keys (key index = tile base + threadIdx.x), ranks equal digits by
// (warp, lane) inside the tile and by tile order across tiles.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const int32_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in,
                     int64_t M, int64_t chunk, int shift, const int32_t *__restrict__ offsets,
                     int32_t *__restrict__ keys_out, int32_t *__restrict__ vals_out)
{
    constexpr int NW = kSortThreads / 32;
    __shared__ int run[kRadix];               // next output slot per digit for this block
    __shared__ int wcount[NW][kRadix];        // per-warp digit counts, then warp prefixes
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offsets[(int64_t)tid * gridDim.x + blockIdx.x];   // blockDim == kRadix
    int64_t beg = (int64_t)blockIdx.x * chunk;
    int64_t end = min(beg + chunk, M);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t tile = beg; tile < end; tile += kSortThreads) {
#pragma unroll
        for (int w = 0; w < NW; ++w) wcount[w][tid] = 0;
        __syncthreads();
        int64_t i = tile + tid;
        int key = 0, val = 0, d = -1;
        if (i < end) {
            key = keys_in[i];
            val = vals_in ? vals_in[i] : (int)i;
            d = (key >> shift) & (kRadix - 1);
        }
        unsigned peers = __match_any_sync(kFull, d);
        int lrank = __popc(peers & lt_mask);
        if (d >= 0 && lrank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        {   // thread tid owns digit tid: exclusive prefix over warps
            int s = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                int cnt = wcount[w][tid];
                wcount[w][tid] = s;
                s += cnt;
            }
            __syncthreads();
            if (d >= 0) {
                int pos = run[d] + wcount[warp][d] + lrank;
                if (keys_out) keys_out[pos] = key;
                vals_out[pos] = val;
            }
            __syncthreads();
            run[tid] += s;
        }
        __syncthreads();
    }
}

__global__ void iota_kernel(int32_t *out, int64_t M)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

// Subproblems per bin: ceil(count / msub).
__global__ void count_subs_kernel(const int32_t *__restrict__ bincount, int64_t nbins, int msub,
                                  int32_t *__restrict__ nsubs)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
         b += (int64_t)gridDim.x * blockDim.x)
        nsubs[b] = (bincount[b] + msub - 1) / msub;
}

__global__ void write_subs_kernel(const int32_t *__restrict__ bincount,
                                  const int32_t *__restrict__ binstart,
                                  const int32_t *__restrict__ suboff, int64_t nbins, int msub,
                                  int4 *__restrict__ subprob)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
         b += (int64_t)gridDim.x * blockDim.x) {
        int cnt = bincount[b], st = binstart[b], so = suboff[b];
        for (int off = 0, k = 0; off < cnt; off += msub, ++k)
            subprob[so + k] = make_int4((int)b, st + off, min(msub, cnt - off), 0);
    }
}

// ---------------------------------------------------------------------------
// Packed records in bin order: kernel offsets and window start relative to
// the padded bin origin (bin origin - ceil(w/2)).
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T packed_word(uint32_t v);
template <> __device__ __forceinline__ float packed_word<float>(uint32_t v) { return __uint_as_float(v); }
template <> __device__ __forceinline__ double packed_word<double>(uint32_t v)
{
    return __longlong_as_double((long long)v);
}

template <typename T, int DIM>
__global__ void pack_records_kernel(const T *__restrict__ x, const T *__restrict__ y,
                                    const T *__restrict__ z, const int32_t *__restrict__ perm,
                                    int64_t M, int3 n, int3 m, int w,
                                    typename rec4<T>::type *__restrict__ recs)
{
    const int P = (w + 1) / 2;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < M;
         s += (int64_t)gridDim.x * blockDim.x) {
        int j = perm[s];
        AxisPos<T> px = axis_position<T>(period_fraction(x[j]), n.x, w);
        AxisPos<T> py = axis_position<T>(period_fraction(y[j]), n.y, w);
        uint32_t sx = (uint32_t)(px.l0 - ((px.l / m.x) * m.x - P));
        uint32_t sy = (uint32_t)(py.l0 - ((py.l / m.y) * m.y - P));
        uint32_t sz = 0;
        T dz = 0;
        if (DIM == 3) {
            AxisPos<T> pz = axis_position<T>(period_fraction(z[j]), n.z, w);
            sz = (uint32_t)(pz.l0 - ((pz.l / m.z) * m.z - P));
            dz = pz.delta;
        }
        typename rec4<T>::type r;
        r.x = px.delta;
        r.y = py.delta;
        r.z = dz;
        r.w = packed_word<T>(sx | (sy << 10) | (sz << 20));
        recs[s] = r;
    }
}

inline int grid_for(int64_t work, int threads, int num_sms)
{
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t setpts_impl(Plan &p, const T *x, const T *y, const T *z)
{
    cudaStream_t st = p.stream;
    const int64_t M = p.M;
    const int3 n = make_int3((int)p.nf[0], (int)p.nf[1], (int)p.nf[2]);
    const int3 m = make_int3(p.m[0], p.m[1], p.m[2]);
    const int3 nb = make_int3(p.nb[0], p.nb[1], p.nb[2]);
    cudaError_t e = cudaMemsetAsync(p.bincount, 0, sizeof(int32_t) * p.nbins, st);
    if (e != cudaSuccess) return e;
    if (M > 0) {
        int g = grid_for(M, 256, p.num_sms);
        if (p.dim == 2) {
            count_launch();
            prep_keys_kernel<T, 2><<<g, 256, 0, st>>>(x, y, z, M, n, m, nb, p.keys, p.bincount);
        }
        else {
            count_launch();
            prep_keys_kernel<T, 3><<<g, 256, 0, st>>>(x, y, z, M, n, m, nb, p.keys, p.bincount);
        }
        // stable LSD radix sort of (key, index)
        int bits = 0;
        while (bits < 31 && ((int64_t)1 << bits) < p.nbins) ++bits;
        int passes = (bits + kRadixBits - 1) / kRadixBits;
        int32_t *kbuf[2] = {p.keys, p.keys_alt};
        int32_t *vbuf[2] = {p.vals, p.vals_alt};
        const int nblk = p.hist_blocks;
        const int64_t chunk = (M + nblk - 1) / nblk;
        if (passes == 0) {
            count_launch();
            iota_kernel<<<grid_for(M, 256, p.num_sms), 256, 0, st>>>(p.vals, M);
            p.perm = p.vals;
        }
        int cur = 0;
        for (int ps = 0; ps < passes; ++ps) {
            const int shift = ps * kRadixBits;
            const bool last = ps == passes - 1;
            count_launch();
            radix_hist_kernel<<<nblk, kSortThreads, 0, st>>>(kbuf[cur], M, chunk, shift, p.hist);
            count_launch();
            scan_exclusive_kernel<<<1, kScanThreads, 0, st>>>(p.hist, p.hist,
                                                              (int64_t)kRadix * nblk, nullptr);
            count_launch();
            radix_scatter_kernel<<<nblk, kSortThreads, 0, st>>>(
                kbuf[cur], ps == 0 ? nullptr : vbuf[cur], M, chunk, shift, p.hist,
                last ? nullptr : kbuf[cur ^ 1], vbuf[cur ^ 1]);
            cur ^= 1;
        }
        if (passes > 0) p.perm = vbuf[cur];
    }
    // subproblems
    const int64_t nbins = p.nbins;
    int gb = grid_for(nbins, 256, p.num_sms);
    count_launch();
    scan_exclusive_kernel<<<1, kScanThreads, 0, st>>>(p.bincount, p.binstart, nbins, nullptr);
    count_launch();
    count_subs_kernel<<<gb, 256, 0, st>>>(p.bincount, nbins, p.msub, p.scan_tmp);
    count_launch();
    scan_exclusive_kernel<<<1, kScanThreads, 0, st>>>(p.scan_tmp, p.scan_tmp, nbins, p.nsub);
    count_launch();
    write_subs_kernel<<<gb, 256, 0, st>>>(p.bincount, p.binstart, p.scan_tmp, nbins, p.msub,
                                          p.subprob);
    if (M > 0) {
        int g = grid_for(M, 256, p.num_sms);
        auto *recs = reinterpret_cast<typename rec4<T>::type *>(p.recs);
        if (p.dim == 2) {
            count_launch();
            pack_records_kernel<T, 2><<<g, 256, 0, st>>>(x, y, z, p.perm, M, n, m, p.w, recs);
        }
        else {
            count_launch();
            pack_records_kernel<T, 3><<<g, 256, 0, st>>>(x, y, z, p.perm, M, n, m, p.w, recs);
        }
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_setpts(Plan &p, const void *x, const void *y, const void *z)
{
    if (p.prec == 0)
        return setpts_impl<float>(p, (const float *)x, (const float *)y, (const float *)z);
    return setpts_impl<double>(p, (const double *)x, (const double *)y, (const double *)z);
}

}  // namespace nufft
