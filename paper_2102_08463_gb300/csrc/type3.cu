// type3.cu -- the type 3 transform (nonuniform points to nonuniform
// frequencies), the third NUFFT type the paper lists as future work:
//   f_k = sum_j c_j exp(i iflag s_k . x_j),  j < M, k < K, real x_j and s_k.
// Built from this library's own type 1 spreading and type 2 transform.  Per axis
// (s' = iflag s, centred: x = C + x', s' = D + s''; |x'| <= X, |s''| <= S):
//   1. pre-phase  c'_j = c_j e^{i D.x'_j};  rescale  u_j = x'_j / gamma
//   2. spread c' onto a uniform grid of n cells (spacing h = 2 pi / n, the
//      ES kernel of width w) -- the type 1 spreading step of Sec. 3.1;
//      gamma = X n / (pi (n - w - 2)) keeps every window inside one period
//   3. g(t) = sum_l b_l e^{i t u_l}, u_l = -pi + l h, at t = s'' gamma: with
//      even n this is a type 2 transform of the grid b (modes -n/2 .. n/2-1 in
//      the library's mode order are exactly b_0 .. b_{n-1}) at the points
//      tau = t h, |tau| <= pi / sigma, exponent sign +1
//   4. f_k = e^{i C.s'_k} prod_i (2 / w) / phihat(alpha_i t_i) g(t_k),
//      alpha = w h / 2 (Poisson summation of the spread kernel: the same
//      correction as Sec. 3.1 step 3, at real frequencies).
// The grid size is n = smallest even 2^a 3^b 5^c >= max(2 sigma S X / pi + w + 2, 2 w),
// so that S gamma h <= pi / sigma: the spread step then resolves the targets with
// the same upsampling factor sigma as type 1.
#include <cmath>
#include <new>
#include <vector>

#include "nufft_internal.cuh"

namespace nufft {

struct Type3 {
    nufft_opts opts;
    int64_t M = 0, K = 0, Mcap = 0, Kcap = 0;
    int64_t n[3] = {1, 1, 1};
    double C[3] = {0, 0, 0}, D[3] = {0, 0, 0}, gam[3] = {1, 1, 1}, h[3] = {1, 1, 1};
    nufft_plan spreader = nullptr;    // inner type 1 plan (fine grid = the n grid), spreading only
    nufft_plan inner = nullptr;       // inner type 2 plan: modes n, points tau
    void *u[3] = {nullptr, nullptr, nullptr};     // rescaled points [Mcap] (T)
    void *tau[3] = {nullptr, nullptr, nullptr};   // inner type 2 points [Kcap] (T)
    void *pre = nullptr;              // [Mcap] complex: e^{i D.x'}
    void *post = nullptr;             // [Kcap] complex: e^{i C.s'} prod (2/w) / phihat
    void *cbuf = nullptr;             // [ntransf Mcap] complex: pre-phased strengths
    double *stats = nullptr;          // device: per-block (min, max) partials
    double *quad = nullptr;           // device: phihat quadrature nodes and weights
    int nq = 0;
};

namespace {

constexpr int kStatBlocks = 256;
constexpr int kStatThreads = 256;

int grid_for(int64_t work, int threads, int num_sms)
{
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// Per-block minimum and maximum of a[0..n): out[2 b] = min, out[2 b + 1] = max
// (both NaN if the block saw a NaN or an infinity).
template <typename T>
__global__ void __launch_bounds__(kStatThreads)
minmax_kernel(const T *__restrict__ a, int64_t n, double *__restrict__ out)
{
    __shared__ double smin[kStatThreads], smax[kStatThreads];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double lo = INFINITY, hi = -INFINITY;
    bool nonfinite = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)a[i];
        nonfinite |= !isfinite(v);
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    if (nonfinite) bad = 1;
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {   // a non-finite value makes the block's pair NaN
        out[2 * blockIdx.x] = bad ? NAN : smin[0];
        out[2 * blockIdx.x + 1] = bad ? NAN : smax[0];
    }
}

struct Axes {
    double C[3], D[3], gam[3], h[3], alpha[3];
    double sgn;                        // iflag
    int dim;
};

// Step 1: u = (x - C) / gamma and the pre-phase e^{i D.(x - C)} (phase in FP64).
template <typename T>
__global__ void __launch_bounds__(256)
prep_points_kernel(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z,
                   int64_t M, Axes ax, T *__restrict__ u0, T *__restrict__ u1, T *__restrict__ u2,
                   typename cplx<T>::type *__restrict__ pre)
{
    const T *xs[3] = {x, y, z};
    T *us[3] = {u0, u1, u2};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        double ph = 0.0;
        for (int d = 0; d < ax.dim; ++d) {
            const double xp = (double)xs[d][j] - ax.C[d];
            us[d][j] = (T)(xp / ax.gam[d]);
            ph += ax.D[d] * xp;
        }
        double sn, cs;
        sincos(ph, &sn, &cs);
        typename cplx<T>::type v;
        v.x = (T)cs;
        v.y = (T)sn;
        pre[j] = v;
    }
}

// Steps 3-4 set-up: tau = (iflag s - D) gamma h and the post factor
// e^{i C.(iflag s)} prod (2/w) / phihat(alpha t), t = (iflag s - D) gamma, with
// phihat(xi) = sum_q v_q cos(xi s_q) (the quadrature of the correction factors).
template <typename T>
__global__ void __launch_bounds__(256)
prep_targets_kernel(const T *__restrict__ s, const T *__restrict__ t, const T *__restrict__ uu,
                    int64_t K, Axes ax, int w, const double *__restrict__ quad, int nq,
                    T *__restrict__ tau0, T *__restrict__ tau1, T *__restrict__ tau2,
                    typename cplx<T>::type *__restrict__ post)
{
    const T *ss[3] = {s, t, uu};
    T *ts[3] = {tau0, tau1, tau2};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        double ph = 0.0, amp = 1.0;
        for (int d = 0; d < ax.dim; ++d) {
            const double se = ax.sgn * (double)ss[d][k];
            const double tt = (se - ax.D[d]) * ax.gam[d];
            ts[d][k] = (T)(tt * ax.h[d]);
            ph += ax.C[d] * se;
            const double xi = ax.alpha[d] * tt;
            double phat = 0.0;
            for (int q = 0; q < nq; ++q) phat += quad[nq + q] * cos(xi * quad[q]);
            amp *= (2.0 / (double)w) / phat;
        }
        double sn, cs;
        sincos(ph, &sn, &cs);
        typename cplx<T>::type v;
        v.x = (T)(amp * cs);
        v.y = (T)(amp * sn);
        post[k] = v;
    }
}

// out[r * n + i] = a[r * n + i] * b[i] (complex), r < rows.
template <typename T>
__global__ void __launch_bounds__(256)
cmul_kernel(const typename cplx<T>::type *__restrict__ a, const typename cplx<T>::type *__restrict__ b,
            typename cplx<T>::type *__restrict__ out, int64_t n, int rows)
{
    const int64_t total = n * rows;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const typename cplx<T>::type u = a[i], v = b[i % n];
        typename cplx<T>::type o;
        o.x = u.x * v.x - u.y * v.y;
        o.y = u.x * v.y + u.y * v.x;
        out[i] = o;
    }
}

// Smallest even 2^a 3^b 5^c >= n.
int64_t next235_even(int64_t n)
{
    if (n < 2) n = 2;
    for (int64_t v = n + (n & 1);; v += 2) {
        int64_t r = v;
        while (r % 2 == 0) r /= 2;
        while (r % 3 == 0) r /= 3;
        while (r % 5 == 0) r /= 5;
        if (r == 1) return v;
    }
}

template <typename T>
int t3_stats(Plan &p, int64_t n, const void *a, double *lo, double *hi)
{
    Type3 &t = *p.t3;
    *lo = 0.0;
    *hi = 0.0;
    if (n == 0) return NUFFT_OK;
    count_launch();
    minmax_kernel<T><<<kStatBlocks, kStatThreads, 0, p.stream>>>((const T *)a, n, t.stats);
    std::vector<double> h(2 * kStatBlocks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), t.stats, sizeof(double) * 2 * kStatBlocks, cudaMemcpyDeviceToHost,
                            p.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return cuda_err(e);
    double l = INFINITY, u = -INFINITY;
    for (int b = 0; b < kStatBlocks; ++b) {
        if (std::isnan(h[2 * b]) || std::isnan(h[2 * b + 1])) return NUFFT_ERR_ARG;
        l = fmin(l, h[2 * b]);
        u = fmax(u, h[2 * b + 1]);
    }
    if (!std::isfinite(l) || !std::isfinite(u)) return NUFFT_ERR_ARG;   // NaN / inf input
    *lo = l;
    *hi = u;
    return NUFFT_OK;
}

void t3_free_inner(Type3 &t)
{
    if (t.spreader) nufft_destroy(t.spreader);
    if (t.inner) nufft_destroy(t.inner);
    t.spreader = t.inner = nullptr;
}

void t3_free_buffers(Type3 &t)
{
    for (int d = 0; d < 3; ++d) {
        dev_free(t.u[d]);
        dev_free(t.tau[d]);
        t.u[d] = t.tau[d] = nullptr;
    }
    dev_free(t.pre);
    dev_free(t.post);
    dev_free(t.cbuf);
    t.pre = t.post = t.cbuf = nullptr;
    t.Mcap = t.Kcap = 0;
}

template <typename T>
int t3_setpts(Plan &p, int64_t M, const void *const *x, int64_t K, const void *const *s)
{
    Type3 &t = *p.t3;
    const int dim = p.dim, w = p.w;
    const double PI = 3.14159265358979323846;
    // bounds of the points and of the frequencies (with the sign iflag)
    Axes ax;
    ax.dim = dim;
    ax.sgn = (double)p.iflag;
    int64_t n[3] = {1, 1, 1};
    for (int d = 0; d < 3; ++d) {
        ax.C[d] = ax.D[d] = 0.0;
        ax.gam[d] = 1.0;
        ax.h[d] = 2.0 * PI;
        ax.alpha[d] = 0.0;
    }
    for (int d = 0; d < dim; ++d) {
        double xl, xh, sl, sh;
        int rc = t3_stats<T>(p, M, x[d], &xl, &xh);
        if (rc == NUFFT_OK) rc = t3_stats<T>(p, K, s[d], &sl, &sh);
        if (rc != NUFFT_OK) return rc;
        if (p.iflag < 0) {
            const double tmp = sl;
            sl = -sh;
            sh = -tmp;
        }
        const double X = 0.5 * (xh - xl), S = 0.5 * (sh - sl);
        ax.C[d] = 0.5 * (xh + xl);
        ax.D[d] = 0.5 * (sh + sl);
        const double want = ceil(2.0 * p.sigma * S * X / PI) + w + 2;
        if (!(want < 1e9)) return NUFFT_ERR_SIZE;
        n[d] = next235_even(std::max((int64_t)want, (int64_t)2 * w));
        ax.h[d] = 2.0 * PI / (double)n[d];
        ax.gam[d] = X > 0.0 ? X * (double)n[d] / (PI * (double)(n[d] - w - 2)) : 1.0;
        ax.alpha[d] = 0.5 * w * ax.h[d];
    }
    // inner plans, made again when the grid changes
    if (!t.spreader || n[0] != t.n[0] || n[1] != t.n[1] || n[2] != t.n[2]) {
        t3_free_inner(t);
        nufft_opts o = t.opts;
        o.method = NUFFT_METHOD_AUTO;
        o.bin[0] = o.bin[1] = o.bin[2] = 0;
        o.msub = 0;
        o.use_picker = 0;
        o.upsampfac = 2.0;
        int64_t half[3], full[3];
        for (int d = 0; d < 3; ++d) {
            half[d] = n[d] / 2;
            full[d] = n[d];
        }
        int rc = nufft_makeplan(1, dim, half, 1, p.ntransf, p.eps, p.prec, &o, &t.spreader);
        if (rc == NUFFT_OK) rc = nufft_makeplan(2, dim, full, -1, p.ntransf, p.eps, p.prec, &o, &t.inner);
        if (rc != NUFFT_OK) {
            t3_free_inner(t);
            return rc;
        }
        for (int d = 0; d < dim; ++d)
            if (t.spreader->p.nf[d] != n[d] || t.spreader->p.w != w) {
                t3_free_inner(t);
                return NUFFT_ERR_SIZE;
            }
        plan_drop_fft(t.spreader->p);   // only its spreading step runs
        for (int d = 0; d < 3; ++d) t.n[d] = n[d];
    }
    // per-point and per-target buffers
    const size_t rs = sizeof(T), cs = 2 * sizeof(T);
    if (M > t.Mcap || K > t.Kcap) {
        t3_free_buffers(t);
        const int64_t mc = M > 0 ? M : 1, kc = K > 0 ? K : 1;
        int rc = NUFFT_OK;
        for (int d = 0; d < dim && rc == NUFFT_OK; ++d) rc = dev_alloc(&t.u[d], rs * mc);
        for (int d = 0; d < dim && rc == NUFFT_OK; ++d) rc = dev_alloc(&t.tau[d], rs * kc);
        if (rc == NUFFT_OK) rc = dev_alloc(&t.pre, cs * mc);
        if (rc == NUFFT_OK) rc = dev_alloc(&t.post, cs * kc);
        if (rc == NUFFT_OK) rc = dev_alloc(&t.cbuf, cs * mc * p.ntransf);
        if (rc != NUFFT_OK) {
            t3_free_buffers(t);
            return rc;
        }
        t.Mcap = mc;
        t.Kcap = kc;
    }
    for (int d = 0; d < 3; ++d) {
        t.C[d] = ax.C[d];
        t.D[d] = ax.D[d];
        t.gam[d] = ax.gam[d];
        t.h[d] = ax.h[d];
    }
    using C = typename cplx<T>::type;
    if (M > 0) {
        count_launch();
        prep_points_kernel<T><<<grid_for(M, 256, p.num_sms), 256, 0, p.stream>>>(
            (const T *)x[0], dim >= 2 ? (const T *)x[1] : nullptr, dim == 3 ? (const T *)x[2] : nullptr,
            M, ax, (T *)t.u[0], (T *)t.u[1], (T *)t.u[2], (C *)t.pre);
    }
    if (K > 0) {
        count_launch();
        prep_targets_kernel<T><<<grid_for(K, 256, p.num_sms), 256, 0, p.stream>>>(
            (const T *)s[0], dim >= 2 ? (const T *)s[1] : nullptr, dim == 3 ? (const T *)s[2] : nullptr,
            K, ax, w, t.quad, t.nq, (T *)t.tau[0], (T *)t.tau[1], (T *)t.tau[2], (C *)t.post);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e);
    int rc = nufft_setpts(t.spreader, M, t.u[0], t.u[1], t.u[2]);
    if (rc == NUFFT_OK) rc = nufft_setpts(t.inner, K, t.tau[0], t.tau[1], t.tau[2]);
    if (rc != NUFFT_OK) return rc;
    t.M = M;
    t.K = K;
    p.M = M;
    p.have_pts = true;
    return NUFFT_OK;
}

template <typename T>
int t3_execute(Plan &p, const void *c, void *f)
{
    Type3 &t = *p.t3;
    using C = typename cplx<T>::type;
    const int nt = p.ntransf;
    if ((t.K > 0 && !f) || (t.K > 0 && t.M > 0 && !c)) return NUFFT_ERR_ARG;
    if (t.K == 0) return NUFFT_OK;
    if (t.M == 0) {
        cudaError_t e = cudaMemsetAsync(f, 0, 2 * sizeof(T) * (size_t)t.K * nt, p.stream);
        return cuda_err(e);
    }
    count_launch();
    cmul_kernel<T><<<grid_for(t.M * nt, 256, p.num_sms), 256, 0, p.stream>>>(
        (const C *)c, (const C *)t.pre, (C *)t.cbuf, t.M, nt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e);
    int rc = nufft_spread(t.spreader, t.cbuf);
    if (rc == NUFFT_OK) rc = nufft_execute(t.inner, f, t.spreader->p.fine);
    if (rc != NUFFT_OK) return rc;
    count_launch();
    cmul_kernel<T><<<grid_for(t.K * nt, 256, p.num_sms), 256, 0, p.stream>>>(
        (const C *)f, (const C *)t.post, (C *)f, t.K, nt);
    return cuda_err(cudaGetLastError());
}

}  // namespace

int type3_init(Plan &p, const nufft_opts &o)
{
    Type3 *t = new (std::nothrow) Type3;
    if (!t) return NUFFT_ERR_ALLOC;
    t->opts = o;
    p.t3 = t;
    int rc = dev_alloc(&t->stats, sizeof(double) * 2 * kStatBlocks);
    // phihat(xi) = int_{-pi/2}^{pi/2} e^{beta (cos th - 1)} cos(xi sin th) cos th d th by
    // Gauss-Legendre in th, as for the correction factors of types 1 and 2
    const int nq = 64 + 4 * p.w;
    std::vector<double> gx, gw, q(2 * nq);
    gauss_legendre(nq, gx, gw);
    const double PI = 3.14159265358979323846;
    for (int i = 0; i < nq; ++i) {
        const double th = 0.5 * PI * gx[i];
        q[i] = sin(th);
        q[nq + i] = 0.5 * PI * gw[i] * exp(p.beta * (cos(th) - 1.0)) * cos(th);
    }
    if (rc == NUFFT_OK) rc = dev_alloc(&t->quad, sizeof(double) * 2 * nq);
    if (rc == NUFFT_OK &&
        cudaMemcpy(t->quad, q.data(), sizeof(double) * 2 * nq, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = NUFFT_ERR_CUDA;
    t->nq = nq;
    return rc;
}

void type3_free(Plan &p)
{
    if (!p.t3) return;
    Type3 &t = *p.t3;
    t3_free_inner(t);
    t3_free_buffers(t);
    dev_free(t.stats);
    dev_free(t.quad);
    delete p.t3;
    p.t3 = nullptr;
}

int type3_setpts(Plan &p, int64_t M, const void *const *x, int64_t K, const void *const *s)
{
    return p.prec == 0 ? t3_setpts<float>(p, M, x, K, s) : t3_setpts<double>(p, M, x, K, s);
}

int type3_execute(Plan &p, const void *c, void *f)
{
    return p.prec == 0 ? t3_execute<float>(p, c, f) : t3_execute<double>(p, c, f);
}

void type3_grid(const Plan &p, int64_t *n)
{
    for (int d = 0; d < 3; ++d) n[d] = p.t3 ? p.t3->n[d] : 1;
}

}  // namespace nufft
