// picker.cu -- learned choice of spreading / interpolation tiles.
//
// The paper fixes its method and tiles by hand-tuned rules (Sec. 4.1 remark:
// 32 x 32 and 16 x 16 x 2 bins, M_sub = 1024; method advice of Sec. 5.4).  Here
// a ReLU perceptron 12 -> 64 -> 64 -> 1 predicts log2 of a plan's execute time
// under one candidate tiling, trained on the autotuner's measured trials, and
// plans made with opts.use_picker take the argmin of its predictions over the
// candidate list.  Everything runs in single precision in these kernels:
//
//   mlp_fwd_kernel<false>  prediction, one thread per sample, weights in smem;
//   mlp_fwd_kernel<true>   forward plus the per-sample deltas of the mean
//                          squared error (dL/dz of every layer), stored
//                          feature-major for coalesced reads below;
//   mlp_wgrad_kernel       dL/dW = sum over samples of delta x activation, one
//                          CTA per weight row, fixed-order (deterministic) sums;
//   mlp_adam_kernel        Adam update with bias correction;
//   sq_loss_kernel         mean squared error in one CTA;
//   coarse_hist_kernel     the point-skew feature: counts in 4096 boxes.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "nufft_internal.cuh"

using namespace nufft;

namespace {

constexpr int kFeat = NUFFT_PICKER_NFEAT;
constexpr int kHid = NUFFT_PICKER_HIDDEN;
constexpr int kParam = NUFFT_PICKER_NPARAM;
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kHid * kFeat;
constexpr int oW2 = oB1 + kHid;
constexpr int oB2 = oW2 + kHid * kHid;
constexpr int oW3 = oB2 + kHid;
constexpr int oB3 = oW3 + kHid;
static_assert(oB3 + 1 == kParam, "parameter layout");

constexpr int kFwdThreads = 128;
constexpr int kTrainThreads = 64;
constexpr int kGradThreads = 256;
constexpr int kBoxes = 4096;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// One thread per sample b (row idx[b] of X, or b).  TRAIN also writes, for
// the minibatch of B samples, feature-major ([unit][b]): A0 = inputs, H1, H2 =
// activations, D1, D2 = dL/dz1, dL/dz2, and G[b] = dL/dy, sq[b] = (y - t)^2.
// h1 and the dL/dz1 sums stay in registers; the second layer's values pass
// through a shared-memory column per thread.
template <bool TRAIN>
__global__ void __launch_bounds__(TRAIN ? kTrainThreads : kFwdThreads)
mlp_fwd_kernel(const float *__restrict__ theta, const float *__restrict__ X,
               const int32_t *__restrict__ idx, int64_t B, const float *__restrict__ T,
               float two_over_b, float *__restrict__ y, float *__restrict__ A0,
               float *__restrict__ H1, float *__restrict__ H2, float *__restrict__ D1,
               float *__restrict__ D2, float *__restrict__ G, float *__restrict__ sq)
{
    __shared__ float s[kParam];
    __shared__ float col[TRAIN ? kHid : 1][TRAIN ? kTrainThreads : 1];
    for (int i = threadIdx.x; i < kParam; i += blockDim.x) s[i] = theta[i];
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int64_t r = idx ? (int64_t)idx[b] : b;
    const int t = TRAIN ? threadIdx.x : 0;
    float x[kFeat];
#pragma unroll
    for (int k = 0; k < kFeat; ++k) x[k] = X[r * kFeat + k];
    float h1[kHid];
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        float a = s[oB1 + i];
#pragma unroll
        for (int k = 0; k < kFeat; ++k) a = fmaf(s[oW1 + i * kFeat + k], x[k], a);
        h1[i] = fmaxf(a, 0.f);
    }
    float out = s[oB3];
#pragma unroll 1
    for (int j = 0; j < kHid; ++j) {
        float a = s[oB2 + j];
#pragma unroll
        for (int i = 0; i < kHid; ++i) a = fmaf(s[oW2 + j * kHid + i], h1[i], a);
        const float h = fmaxf(a, 0.f);
        out = fmaf(s[oW3 + j], h, out);
        if (TRAIN) col[TRAIN ? j : 0][t] = h;
    }
    if (!TRAIN) {
        y[b] = out;
        return;
    }
    const float err = out - T[r];
    const float g = two_over_b * err;
    G[b] = g;
    sq[b] = err * err;
#pragma unroll
    for (int k = 0; k < kFeat; ++k) A0[k * B + b] = x[k];
#pragma unroll 4
    for (int j = 0; j < kHid; ++j) {
        const float h = col[TRAIN ? j : 0][t];
        H2[j * B + b] = h;
        const float d = h > 0.f ? g * s[oW3 + j] : 0.f;
        D2[j * B + b] = d;
        col[TRAIN ? j : 0][t] = d;                    // the column now holds dL/dz2
    }
    float a[kHid];
#pragma unroll
    for (int i = 0; i < kHid; ++i) a[i] = 0.f;
#pragma unroll 1
    for (int j = 0; j < kHid; ++j) {
        const float d = col[TRAIN ? j : 0][t];
#pragma unroll
        for (int i = 0; i < kHid; ++i) a[i] = fmaf(s[oW2 + j * kHid + i], d, a[i]);
    }
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        H1[i * B + b] = h1[i];
        D1[i * B + b] = h1[i] > 0.f ? a[i] : 0.f;
    }
}

// Sums over the B samples of delta[b] * act[k][b] (K weights) and delta[b]
// (the bias) for one weight row: per-thread partial sums over a fixed stride,
// then warp shuffles and a fixed-order sum over warps, so the result does not
// depend on scheduling.
template <int K>
__device__ void row_grad(int64_t B, const float *__restrict__ delta, const float *__restrict__ act,
                         float *__restrict__ gw, float *__restrict__ gb, float scale_b)
{
    __shared__ float red[kGradThreads / 32][kHid + 1];
    float acc[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) acc[k] = 0.f;
    for (int64_t b = threadIdx.x; b < B; b += kGradThreads) {
        const float d = delta[b];
        acc[K] += d;
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = fmaf(d, act[k * B + b], acc[k]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k <= K; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x <= K) {
        float v = 0.f;
        for (int w = 0; w < kGradThreads / 32; ++w) v += red[w][threadIdx.x];
        if ((int)threadIdx.x < K)
            gw[threadIdx.x] = v;
        else
            *gb = v * scale_b;
    }
}

// CTAs 0..63: rows of W1 / b1; 64..127: rows of W2 / b2; 128: w3 / b3;
// 129 (when loss != NULL): loss = mean of sq.
__global__ void __launch_bounds__(kGradThreads)
mlp_wgrad_kernel(int64_t B, const float *__restrict__ A0, const float *__restrict__ H1,
                 const float *__restrict__ H2, const float *__restrict__ D1,
                 const float *__restrict__ D2, const float *__restrict__ G,
                 const float *__restrict__ sq, float *__restrict__ grad, float *__restrict__ loss)
{
    const int blk = blockIdx.x;
    if (blk < kHid)
        row_grad<kFeat>(B, D1 + blk * B, A0, grad + oW1 + blk * kFeat, grad + oB1 + blk, 1.f);
    else if (blk < 2 * kHid)
        row_grad<kHid>(B, D2 + (blk - kHid) * B, H1, grad + oW2 + (blk - kHid) * kHid,
                       grad + oB2 + (blk - kHid), 1.f);
    else if (blk == 2 * kHid)
        row_grad<kHid>(B, G, H2, grad + oW3, grad + oB3, 1.f);
    else
        row_grad<0>(B, sq, nullptr, nullptr, loss, 1.f / (float)B);
}

__global__ void mlp_adam_kernel(float *__restrict__ theta, const float *__restrict__ g,
                                float *__restrict__ m, float *__restrict__ v, int n, float lr,
                                float beta1, float beta2, float c1, float c2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// loss = (1/n) sum_b (y[b] - T[b])^2 in one CTA, fixed order.
__global__ void __launch_bounds__(1024)
sq_loss_kernel(int64_t n, const float *__restrict__ y, const float *__restrict__ T,
               float *__restrict__ loss)
{
    __shared__ float red[32];
    float acc = 0.f;
    for (int64_t b = threadIdx.x; b < n; b += blockDim.x) {
        const float e = y[b] - T[b];
        acc = fmaf(e, e, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        *loss = v / (float)n;
    }
}

// Box index of one coordinate along an axis cut into g equal boxes over the
// period [-pi, pi); any finite input folds into [0, g), and the integer
// conversion of NaN or huge values still lands in range after the fold.
template <typename T>
__device__ __forceinline__ int box_of(T x, int g)
{
    const float u = ((float)x + 3.14159265f) * ((float)g * 0.159154943f);
    int c = (int)floorf(u) % g;
    return c < 0 ? c + g : c;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256)
coarse_hist_kernel(int64_t M, const T *__restrict__ x, const T *__restrict__ y,
                   const T *__restrict__ z, int32_t *__restrict__ hist)
{
    constexpr int g = DIM == 2 ? 64 : 16;
    __shared__ int32_t h[kBoxes];
    for (int i = threadIdx.x; i < kBoxes; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count, so the whole warp takes part in every match
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < M; base += stride) {
        const int64_t j = base + threadIdx.x;
        const bool valid = j < M;
        int box = -1;
        if (valid) {
            box = box_of(x[j], g) + g * box_of(y[j], g);
            if (DIM == 3) box += g * g * box_of(z[j], g);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, box);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[box], __popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBoxes; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void __launch_bounds__(1024) hist_max_kernel(const int32_t *__restrict__ hist,
                                                        int32_t *__restrict__ out)
{
    __shared__ int32_t red[32];
    int32_t m = 0;
    for (int i = threadIdx.x; i < kBoxes; i += blockDim.x) m = max(m, hist[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = max(v, red[w]);
        *out = v;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

uint64_t splitmix64(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t &state) { return (double)(splitmix64(state) >> 11) * 0x1.0p-53; }

int rc_of(cudaError_t e)
{
    if (e == cudaSuccess) return NUFFT_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NUFFT_ERR_ALLOC : NUFFT_ERR_CUDA;
}

template <typename P>
int grow(P **ptr, int64_t &cap, int64_t want)
{
    if (want <= cap) return NUFFT_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    cap = 0;
    void *v = nullptr;
    if (cudaMalloc(&v, sizeof(P) * (size_t)want) != cudaSuccess) {
        cudaGetLastError();
        return NUFFT_ERR_ALLOC;
    }
    *ptr = (P *)v;
    cap = want;
    return NUFFT_OK;
}

std::mutex g_install_mutex;
nufft_picker g_installed = nullptr;

}  // namespace

struct nufft_picker_s {
    int device = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    int64_t step = 0;
    // minibatch scratch, grown on demand: 12 + 4 * 64 rows of cap floats, then G, sq, y
    float *scr = nullptr;
    int64_t scr_cap = 0;
    int32_t *idx = nullptr;
    int64_t idx_cap = 0;
    float *feat = nullptr;           // candidate features / predictions for picker_choose
    int64_t feat_cap = 0;
    int32_t *hist = nullptr;         // 4096 boxes + 1 max
};

namespace {

constexpr int kScrRows = kFeat + 4 * kHid + 3;

struct Scratch {
    float *A0, *H1, *H2, *D1, *D2, *G, *sq, *y;
};

Scratch carve(nufft_picker h, int64_t B)
{
    Scratch s;
    float *p = h->scr;
    s.A0 = p;
    p += kFeat * B;
    s.H1 = p;
    p += kHid * B;
    s.H2 = p;
    p += kHid * B;
    s.D1 = p;
    p += kHid * B;
    s.D2 = p;
    p += kHid * B;
    s.G = p;
    p += B;
    s.sq = p;
    p += B;
    s.y = p;
    return s;
}

int fwd_grad(nufft_picker h, int64_t B, const float *X, const int32_t *idx, const float *T,
             float *grad, float *loss, cudaStream_t st)
{
    int rc = grow(&h->scr, h->scr_cap, kScrRows * B);
    if (rc != NUFFT_OK) return rc;
    Scratch s = carve(h, B);
    const unsigned nb = (unsigned)((B + kTrainThreads - 1) / kTrainThreads);
    mlp_fwd_kernel<true><<<nb, kTrainThreads, 0, st>>>(h->theta, X, idx, B, T, 2.f / (float)B,
                                                       nullptr, s.A0, s.H1, s.H2, s.D1, s.D2, s.G,
                                                       s.sq);
    count_launch();
    mlp_wgrad_kernel<<<2 * kHid + 1 + (loss ? 1 : 0), kGradThreads, 0, st>>>(
        B, s.A0, s.H1, s.H2, s.D1, s.D2, s.G, s.sq, grad, loss);
    count_launch();
    return rc_of(cudaGetLastError());
}

int adam(nufft_picker h, float lr, cudaStream_t st)
{
    const double b1 = 0.9, b2 = 0.999;
    ++h->step;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)h->step)));
    const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)h->step)));
    mlp_adam_kernel<<<(kParam + 255) / 256, 256, 0, st>>>(h->theta, h->grad, h->m, h->v, kParam,
                                                           lr, (float)b1, (float)b2, c1, c2, 1e-8f);
    count_launch();
    return rc_of(cudaGetLastError());
}

int predict(nufft_picker h, int64_t B, const float *X, float *y, cudaStream_t st)
{
    if (B == 0) return NUFFT_OK;
    const unsigned nb = (unsigned)((B + kFwdThreads - 1) / kFwdThreads);
    mlp_fwd_kernel<false><<<nb, kFwdThreads, 0, st>>>(h->theta, X, nullptr, B, nullptr, 0.f, y,
                                                        nullptr, nullptr, nullptr, nullptr,
                                                        nullptr, nullptr, nullptr);
    count_launch();
    return rc_of(cudaGetLastError());
}

int point_skew(int dim, int prec, int64_t M, const void *x, const void *y, const void *z,
               int32_t *hist, double *skew, cudaStream_t st)
{
    *skew = 0.0;
    if (M == 0) return NUFFT_OK;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (kBoxes + 1), st);
    if (e != cudaSuccess) return rc_of(e);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (M + 256 * 32 - 1) / (256 * 32);
    const int nb = (int)(want < 4 * sms ? (want < 1 ? 1 : want) : 4 * sms);
    if (prec == 0) {
        if (dim == 2)
            coarse_hist_kernel<float, 2><<<nb, 256, 0, st>>>(M, (const float *)x, (const float *)y,
                                                             nullptr, hist);
        else
            coarse_hist_kernel<float, 3><<<nb, 256, 0, st>>>(M, (const float *)x, (const float *)y,
                                                             (const float *)z, hist);
    } else {
        if (dim == 2)
            coarse_hist_kernel<double, 2><<<nb, 256, 0, st>>>(M, (const double *)x,
                                                              (const double *)y, nullptr, hist);
        else
            coarse_hist_kernel<double, 3><<<nb, 256, 0, st>>>(M, (const double *)x,
                                                              (const double *)y,
                                                              (const double *)z, hist);
    }
    count_launch();
    hist_max_kernel<<<1, 1024, 0, st>>>(hist, hist + kBoxes);
    count_launch();
    int32_t mx = 0;
    e = cudaMemcpyAsync(&mx, hist + kBoxes, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return rc_of(e);
    const double s = log2((double)mx * kBoxes / (double)M);
    *skew = s > 0.0 ? s : 0.0;
    return NUFFT_OK;
}

void features(int type, int dim, int prec, int w, double nftot, double M, double skew,
              const Tiles &t, float *out)
{
    const double mm = M > 1.0 ? M : 1.0;
    double cells = 1.0;
    for (int d = 0; d < dim; ++d) cells *= t.bin[d];
    out[0] = type == 2 ? 1.f : 0.f;
    out[1] = dim == 3 ? 1.f : 0.f;
    out[2] = prec == 1 ? 1.f : 0.f;
    out[3] = (float)(w / 16.0);
    out[4] = (float)(log2(nftot) / 32.0);
    out[5] = (float)(log2(mm / nftot) / 8.0);
    out[6] = (float)(skew / 16.0);
    out[7] = t.method == NUFFT_METHOD_SM ? 1.f : 0.f;
    out[8] = t.method == NUFFT_METHOD_GM ? 1.f : 0.f;
    out[9] = (float)(log2(cells) / 12.0);
    out[10] = (float)(log2((double)t.msub) / 12.0);
    out[11] = (float)(t.threads / 256.0);
}

}  // namespace

int nufft::picker_choose(Plan &p, int64_t M, const void *x, const void *y, const void *z,
                         Tiles *out, bool *chosen)
{
    *chosen = false;
    std::lock_guard<std::mutex> lock(g_install_mutex);
    nufft_picker h = g_installed;
    if (!h) return NUFFT_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) return NUFFT_OK;          // the picker lives on another device
    double skew = 0.0;
    int rc = point_skew(p.dim, p.prec, M, x, y, z, h->hist, &skew, p.stream);
    if (rc != NUFFT_OK) return rc;
    std::vector<Tiles> cand;
    for (const Tiles &t : tile_candidates(p))
        if (tiles_feasible(p, t)) cand.push_back(t);
    if (cand.empty()) return NUFFT_OK;
    const int64_t nc = (int64_t)cand.size();
    rc = grow(&h->feat, h->feat_cap, nc * (kFeat + 1));
    if (rc != NUFFT_OK) return rc;
    std::vector<float> X((size_t)nc * kFeat), yv((size_t)nc);
    for (int64_t i = 0; i < nc; ++i)
        features(p.type, p.dim, p.prec, p.w, (double)p.nftot, (double)M, skew, cand[i],
                 &X[(size_t)i * kFeat]);
    cudaError_t e = cudaMemcpyAsync(h->feat, X.data(), sizeof(float) * X.size(),
                                    cudaMemcpyHostToDevice, p.stream);
    if (e != cudaSuccess) return rc_of(e);
    rc = predict(h, nc, h->feat, h->feat + nc * kFeat, p.stream);
    if (rc != NUFFT_OK) return rc;
    e = cudaMemcpyAsync(yv.data(), h->feat + nc * kFeat, sizeof(float) * nc,
                        cudaMemcpyDeviceToHost, p.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return rc_of(e);
    int64_t best = 0;
    for (int64_t i = 1; i < nc; ++i)
        if (yv[i] < yv[best]) best = i;
    *out = cand[best];
    *chosen = true;
    return NUFFT_OK;
}

extern "C" {

int nufft_picker_create(uint64_t seed, nufft_picker *out)
{
    if (!out) return NUFFT_ERR_ARG;
    *out = nullptr;
    nufft_picker h = new (std::nothrow) nufft_picker_s;
    if (!h) return NUFFT_ERR_ALLOC;
    cudaGetDevice(&h->device);
    float *bufs[4] = {nullptr, nullptr, nullptr, nullptr};
    bool ok = true;
    for (auto &b : bufs) ok = ok && cudaMalloc(&b, sizeof(float) * kParam) == cudaSuccess;
    ok = ok && cudaMalloc(&h->loss, sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->hist, sizeof(int32_t) * (kBoxes + 1)) == cudaSuccess;
    h->theta = bufs[0];
    h->m = bufs[1];
    h->v = bufs[2];
    h->grad = bufs[3];
    if (!ok) {
        cudaGetLastError();
        nufft_picker_destroy(h);
        return NUFFT_ERR_ALLOC;
    }
    // He-uniform: W ~ U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)), biases 0
    std::vector<float> th(kParam, 0.f);
    uint64_t st = seed;
    const double a1 = sqrt(6.0 / kFeat), a2 = sqrt(6.0 / kHid);
    for (int i = 0; i < kHid * kFeat; ++i) th[oW1 + i] = (float)((2.0 * uniform01(st) - 1.0) * a1);
    for (int i = 0; i < kHid * kHid; ++i) th[oW2 + i] = (float)((2.0 * uniform01(st) - 1.0) * a2);
    for (int i = 0; i < kHid; ++i) th[oW3 + i] = (float)((2.0 * uniform01(st) - 1.0) * a2);
    const int rc = nufft_picker_set_params(h, th.data());
    if (rc != NUFFT_OK) {
        nufft_picker_destroy(h);
        return rc;
    }
    *out = h;
    return NUFFT_OK;
}

int nufft_picker_destroy(nufft_picker h)
{
    if (!h) return NUFFT_ERR_ARG;
    {
        std::lock_guard<std::mutex> lock(g_install_mutex);
        if (g_installed == h) g_installed = nullptr;
    }
    for (void *p : {(void *)h->theta, (void *)h->m, (void *)h->v, (void *)h->grad,
                    (void *)h->loss, (void *)h->scr, (void *)h->idx, (void *)h->feat,
                    (void *)h->hist})
        if (p) cudaFree(p);
    delete h;
    return NUFFT_OK;
}

int nufft_picker_set_params(nufft_picker h, const float *params)
{
    if (!h || !params) return NUFFT_ERR_ARG;
    cudaError_t e = cudaMemcpy(h->theta, params, sizeof(float) * kParam, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->m, 0, sizeof(float) * kParam);
    if (e == cudaSuccess) e = cudaMemset(h->v, 0, sizeof(float) * kParam);
    h->step = 0;
    return rc_of(e);
}

int nufft_picker_get_params(nufft_picker h, float *params)
{
    if (!h || !params) return NUFFT_ERR_ARG;
    return rc_of(cudaMemcpy(params, h->theta, sizeof(float) * kParam, cudaMemcpyDeviceToHost));
}

int nufft_picker_save(nufft_picker h, const char *path)
{
    if (!h || !path) return NUFFT_ERR_ARG;
    std::vector<float> th(kParam);
    int rc = nufft_picker_get_params(h, th.data());
    if (rc != NUFFT_OK) return rc;
    FILE *fp = fopen(path, "w");
    if (!fp) return NUFFT_ERR_ARG;
    fprintf(fp, "# nufft_gb300 tile picker v1: %d parameters (W1 b1 W2 b2 w3 b3)\n", kParam);
    for (float v : th) fprintf(fp, "%.9g\n", v);
    fclose(fp);
    return NUFFT_OK;
}

int nufft_picker_load(nufft_picker h, const char *path)
{
    if (!h || !path) return NUFFT_ERR_ARG;
    FILE *fp = fopen(path, "r");
    if (!fp) return NUFFT_ERR_ARG;
    std::vector<float> th;
    th.reserve(kParam);
    char line[256];
    while (fgets(line, sizeof(line), fp)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        float v;
        if (sscanf(line, "%f", &v) != 1) break;
        th.push_back(v);
    }
    fclose(fp);
    if ((int)th.size() != kParam) return NUFFT_ERR_ARG;
    return nufft_picker_set_params(h, th.data());
}

int nufft_picker_predict(nufft_picker h, int64_t B, const float *X, float *y, void *stream)
{
    if (!h || B < 0 || (B > 0 && (!X || !y))) return NUFFT_ERR_ARG;
    return predict(h, B, X, y, (cudaStream_t)stream);
}

int nufft_picker_grad(nufft_picker h, int64_t B, const float *X, const float *T, float *grad,
                      float *loss, void *stream)
{
    if (!h || B < 1 || !X || !T || !grad || !loss) return NUFFT_ERR_ARG;
    return fwd_grad(h, B, X, nullptr, T, grad, loss, (cudaStream_t)stream);
}

int nufft_picker_step(nufft_picker h, int64_t B, const float *X, const float *T, float lr,
                      float *loss, void *stream)
{
    if (!h || B < 1 || !X || !T || !(lr > 0.f)) return NUFFT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = fwd_grad(h, B, X, nullptr, T, h->grad, loss ? loss : h->loss, st);
    return rc == NUFFT_OK ? adam(h, lr, st) : rc;
}

int nufft_picker_loss(nufft_picker h, int64_t n, const float *X, const float *T, float *loss,
                      void *stream)
{
    if (!h || n < 1 || !X || !T || !loss) return NUFFT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = grow(&h->scr, h->scr_cap, kScrRows * n);
    if (rc != NUFFT_OK) return rc;
    float *y = carve(h, n).y;
    rc = predict(h, n, X, y, st);
    if (rc != NUFFT_OK) return rc;
    sq_loss_kernel<<<1, 1024, 0, st>>>(n, y, T, loss);
    count_launch();
    return rc_of(cudaGetLastError());
}

int nufft_picker_train(nufft_picker h, int64_t n, const float *X, const float *T, int epochs,
                       int batch, float lr, uint64_t seed, float *final_loss, void *stream)
{
    if (!h || n < 1 || !X || !T || epochs < 0 || batch < 1 || !(lr > 0.f) ||
        n > ((int64_t)1 << 30))
        return NUFFT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = grow(&h->idx, h->idx_cap, n);
    if (rc != NUFFT_OK) return rc;
    const int64_t bs = batch < n ? batch : n;
    rc = grow(&h->scr, h->scr_cap, kScrRows * (bs > n ? bs : n));
    if (rc != NUFFT_OK) return rc;
    std::vector<int32_t> perm((size_t)n);
    uint64_t state = seed;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (int32_t)i;
        for (int64_t i = n - 1; i > 0; --i) {                  // Fisher-Yates
            const int64_t j = (int64_t)(uniform01(state) * (double)(i + 1));
            std::swap(perm[(size_t)i], perm[(size_t)(j > i ? i : j)]);
        }
        // the previous epoch's kernels read idx: wait before overwriting it
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->idx, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                                st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return rc_of(e);
        for (int64_t off = 0; off < n; off += bs) {
            const int64_t B = off + bs <= n ? bs : n - off;
            rc = fwd_grad(h, B, X, h->idx + off, T, h->grad, h->loss, st);
            if (rc == NUFFT_OK) rc = adam(h, lr, st);
            if (rc != NUFFT_OK) return rc;
        }
    }
    if (final_loss) {
        rc = nufft_picker_loss(h, n, X, T, h->loss, stream);
        if (rc != NUFFT_OK) return rc;
        cudaError_t e = cudaMemcpyAsync(final_loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost,
                                        st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return rc_of(e);
    }
    return rc_of(cudaStreamSynchronize(st));
}

int nufft_picker_install(nufft_picker h)
{
    std::lock_guard<std::mutex> lock(g_install_mutex);
    g_installed = h;
    return NUFFT_OK;
}

int nufft_picker_features(int type, int dim, const int64_t *nmodes, double eps, int prec,
                          double upsampfac, int64_t M, double skew, const nufft_opts *tiles,
                          float *out)
{
    if ((type != 1 && type != 2) || (dim != 2 && dim != 3) || !nmodes || !tiles || !out ||
        !(eps > 0.0) || M < 0 || prec < -1 || prec > 1)
        return NUFFT_ERR_ARG;
    const double sigma = upsampfac == 0.0 ? 2.0 : upsampfac;
    if (sigma != 2.0 && sigma != 1.25) return NUFFT_ERR_ARG;
    const double fp32_floor = sigma == 2.0 ? 1e-6 : 1e-4;
    if (prec == -1) prec = eps >= fp32_floor ? 0 : 1;
    if (prec == 0 && eps < fp32_floor) return NUFFT_ERR_EPS;
    const int w = kernel_width(eps, sigma);
    if (w > kMaxW) return NUFFT_ERR_EPS;
    if (tiles->method < NUFFT_METHOD_GM || tiles->method > NUFFT_METHOD_SM) return NUFFT_ERR_ARG;
    double nftot = 1.0;
    Tiles t;
    t.method = tiles->method;
    for (int d = 0; d < dim; ++d) {
        if (nmodes[d] < 1) return NUFFT_ERR_ARG;
        int64_t want = (int64_t)ceil(sigma * (double)nmodes[d] - 1e-9);
        if (want < 2 * w) want = 2 * w;
        const int64_t nf = next235(want);
        nftot *= (double)nf;
        int defb[3];
        default_bins(type, dim, prec, w, defb);            // as makeplan
        const int mdef = defb[d];
        int m = tiles->bin[d] > 0 ? tiles->bin[d] : mdef;
        if (m > nf) m = (int)nf;
        t.bin[d] = m;
    }
    t.msub = tiles->msub > 0 ? tiles->msub : 1024;
    t.threads = tiles->threads > 0 ? tiles->threads : kDefaultThreads;
    features(type, dim, prec, w, nftot, (double)M, skew < 0.0 ? 0.0 : skew, t, out);
    return NUFFT_OK;
}

int nufft_pick(int type, int dim, const int64_t *nmodes, double eps, int prec, int64_t M,
               const void *x, const void *y, const void *z, void *stream, nufft_opts *opts)
{
    if ((type != 1 && type != 2) || (dim != 2 && dim != 3) || !nmodes || !opts ||
        !(eps > 0.0) || (prec != 0 && prec != 1) || M < 0)
        return NUFFT_ERR_ARG;
    if (M > 0 && (!x || !y || (dim == 3 && !z))) return NUFFT_ERR_ARG;
    for (int d = 0; d < dim; ++d)
        if (nmodes[d] < 1 || nmodes[d] > (1 << 26)) return NUFFT_ERR_SIZE;
    // one light plan per upsampling factor whose plan at this precision reaches
    // eps (the grid rule of makeplan); nothing is allocated
    std::vector<Plan> grids;
    for (double sigma : {2.0, 1.25}) {
        const double fp32_floor = sigma == 2.0 ? 1e-6 : 1e-4;
        if (prec == 0 && eps < fp32_floor) continue;
        const int w = kernel_width(eps, sigma);
        if (w > kMaxW) continue;
        Plan q;
        q.type = type;
        q.dim = dim;
        q.prec = prec;
        q.eps = eps;
        q.sigma = sigma;
        q.w = w;
        q.nftot = 1;
        for (int d = 0; d < dim; ++d) {
            q.N[d] = nmodes[d];
            int64_t want = (int64_t)ceil(sigma * (double)nmodes[d] - 1e-9);
            if (want < 2 * w) want = 2 * w;
            q.nf[d] = next235(want);
            q.nftot *= q.nf[d];
        }
        grids.push_back(q);
    }
    if (grids.empty()) return NUFFT_ERR_EPS;
    // no picker: sigma = 2 (listed first; it reaches every eps 1.25 reaches), tiles automatic
    opts->upsampfac = grids[0].sigma;
    opts->method = NUFFT_METHOD_AUTO;
    opts->bin[0] = opts->bin[1] = opts->bin[2] = 0;
    opts->msub = 0;
    opts->threads = 0;
    std::lock_guard<std::mutex> lock(g_install_mutex);
    nufft_picker h = g_installed;
    if (!h) return NUFFT_OK;
    int dev = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) return NUFFT_OK;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (Plan &q : grids) q.smem_optin = smem_optin;
    const cudaStream_t st = (cudaStream_t)stream;
    double skew = 0.0;
    int rc = point_skew(dim, prec, M, x, y, z, h->hist, &skew, st);
    if (rc != NUFFT_OK) return rc;
    std::vector<int> gi;
    std::vector<Tiles> cand;
    for (size_t g = 0; g < grids.size(); ++g)
        for (const Tiles &t : tile_candidates(grids[g]))
            if (tiles_feasible(grids[g], t)) {
                gi.push_back((int)g);
                cand.push_back(t);
            }
    if (cand.empty()) return NUFFT_OK;
    const int64_t nc = (int64_t)cand.size();
    rc = grow(&h->feat, h->feat_cap, nc * (kFeat + 1));
    if (rc != NUFFT_OK) return rc;
    std::vector<float> X((size_t)nc * kFeat), yv((size_t)nc);
    for (int64_t i = 0; i < nc; ++i) {
        const Plan &q = grids[(size_t)gi[(size_t)i]];
        features(type, dim, prec, q.w, (double)q.nftot, (double)M, skew, cand[(size_t)i],
                 &X[(size_t)i * kFeat]);
    }
    cudaError_t e = cudaMemcpyAsync(h->feat, X.data(), sizeof(float) * X.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return rc_of(e);
    rc = predict(h, nc, h->feat, h->feat + nc * kFeat, st);
    if (rc != NUFFT_OK) return rc;
    e = cudaMemcpyAsync(yv.data(), h->feat + nc * kFeat, sizeof(float) * nc,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return rc_of(e);
    int64_t best = 0;
    for (int64_t i = 1; i < nc; ++i)
        if (yv[(size_t)i] < yv[(size_t)best]) best = i;
    const Tiles &t = cand[(size_t)best];
    opts->upsampfac = grids[(size_t)gi[(size_t)best]].sigma;
    opts->method = t.method;
    for (int d = 0; d < 3; ++d) opts->bin[d] = d < dim ? t.bin[d] : 0;
    opts->msub = t.msub;
    opts->threads = t.threads;
    return NUFFT_OK;
}

int nufft_point_skew(int dim, int prec, int64_t M, const void *x, const void *y, const void *z,
                     double *skew, void *stream)
{
    if ((dim != 2 && dim != 3) || (prec != 0 && prec != 1) || M < 0 || !skew) return NUFFT_ERR_ARG;
    if (M > 0 && (!x || !y || (dim == 3 && !z))) return NUFFT_ERR_ARG;
    int32_t *hist = nullptr;
    if (cudaMalloc(&hist, sizeof(int32_t) * (kBoxes + 1)) != cudaSuccess) {
        cudaGetLastError();
        return NUFFT_ERR_ALLOC;
    }
    const int rc = point_skew(dim, prec, M, x, y, z, hist, skew, (cudaStream_t)stream);
    cudaFree(hist);
    return rc;
}

}  // extern "C"
