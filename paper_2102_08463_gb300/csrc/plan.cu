// plan.cu -- the C ABI: plan, setpts, execute, destroy (Sec. 1.1) and the
// parameter rules of Sec. 3.  Host code only; every step of the transform runs
// in the kernels of setpts.cu, spread_interp.cuh, correct.cu and in cuFFT.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "nufft_internal.cuh"

using namespace nufft;

std::atomic<unsigned long long> nufft::g_launch_count{0};

namespace {
std::atomic<int> g_fail_after[3] = {{-1}, {-1}, {-1}};   // armed countdown per kind
std::atomic<int> g_fail_calls[3] = {{0}, {0}, {0}};     // calls since the last arming
}  // namespace

bool nufft::injected_failure(int kind)
{
    if (kind < 1 || kind > 2) return false;
    g_fail_calls[kind].fetch_add(1);
    int left = g_fail_after[kind].load();
    while (left >= 0) {
        if (g_fail_after[kind].compare_exchange_weak(left, left - 1)) return left == 0;
    }
    return false;
}

// Each kernel's dynamic shared-memory limit is raised once per device, to the
// largest the device allows next to the kernel's static shared memory, so that
// no launch depends on a per-call setting another host thread could change.
// The (kernel, device) pairs already done sit in a fixed table (no heap use);
// past its end the attribute is simply set again, to the same value.
cudaError_t nufft::allow_max_smem(const void *func)
{
    constexpr int kCap = 1024;
    static std::mutex mu;
    static const void *done_f[kCap];
    static int done_d[kCap];
    static int ndone = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < ndone; ++i)
        if (done_f[i] == func && done_d[i] == dev) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn > 0 ? dyn : 0);
    if (e != cudaSuccess) return e;
    if (ndone < kCap) {
        done_f[ndone] = func;
        done_d[ndone] = dev;
        ++ndone;
    }
    return cudaSuccess;
}

int nufft::next235(int64_t n)
{
    if (n < 1) n = 1;
    for (;; ++n) {
        int64_t m = n;
        while (m % 2 == 0) m /= 2;
        while (m % 3 == 0) m /= 3;
        while (m % 5 == 0) m /= 5;
        if (m == 1) return (int)n;
    }
}

// Kernel width (Sec. 3): w = ceil(log10(1/eps)) + 1 for sigma = 2.  Powers of
// ten map to their nominal width: a 1e-10 guard absorbs the rounding of
// log10 of a decimal tolerance.  sigma = 1.25 uses the calibrated width
// ceil(log10(1/eps) / 0.6) + 1.
int nufft::kernel_width(double eps, double sigma)
{
    double digits = -log10(eps);
    double w = sigma == 2.0 ? ceil(digits - 1e-10) + 1.0 : ceil(digits / 0.6 - 1e-10) + 1.0;
    if (w < 2.0) w = 2.0;
    return (int)fmin(w, 99.0);
}

namespace {

// beta = 2.30 w for sigma = 2 (Sec. 3); scaled by (1 - 1/(2 sigma)) / (3/4) otherwise.
double kernel_beta(int w, double sigma)
{
    return sigma == 2.0 ? 2.30 * w : 2.30 * w * (1.0 - 1.0 / (2.0 * sigma)) / 0.75;
}

void free_points(Plan &p)
{
    dev_free(p.keys);
    dev_free(p.keys_alt);
    dev_free(p.vals);
    dev_free(p.vals_alt);
    dev_free(p.recs);
    dev_free(p.rorder);
    p.rorder = nullptr;
    dev_free(p.recs2);
    p.recs2 = nullptr;
    p.row_ordered = false;
    dev_free(p.subprob);
    for (int d = 0; d < 3; ++d) {
        dev_free(p.xyz_copy[d]);
        p.xyz_copy[d] = nullptr;
    }
    p.keys = p.keys_alt = p.vals = p.vals_alt = p.perm = nullptr;
    p.recs = nullptr;
    p.subprob = nullptr;
    p.Mcap = 0;
    p.maxsub = 0;
}

void free_host_staging(Plan &p)
{
    for (int d = 0; d < 3; ++d) {
        dev_free(p.hx_pts[d]);
        p.hx_pts[d] = nullptr;
    }
    dev_free(p.hx_c);
    p.hx_c = nullptr;
    p.hx_cap = 0;
}

void free_plan(Plan &p)
{
    type3_free(p);
    free_points(p);
    free_host_staging(p);
    dev_free(p.hx_f);
    p.hx_f = nullptr;
    for (int i = 0; i < 2; ++i)
        if (p.hx_ev[i]) cudaEventDestroy(p.hx_ev[i]);
    if (p.hx_copy) cudaStreamDestroy(p.hx_copy);
    p.hx_copy = nullptr;
    p.hx_ev[0] = p.hx_ev[1] = nullptr;
    dev_free(p.fine);
    for (int d = 0; d < 3; ++d) dev_free(p.corr[d]);
    dev_free(p.bincount);
    dev_free(p.binstart);
    dev_free(p.scan_tmp);
    dev_free(p.nsub);
    dev_free(p.dstatus);
    p.dstatus = nullptr;
    dev_free(p.mat);
    dev_free(p.scan_part);
    p.mat = p.scan_part = nullptr;
    p.mat_cap = p.scan_part_cap = 0;
    if (p.fft_ready) cufftDestroy(p.fft);
    p.fft_ready = false;
}

size_t real_size(const Plan &p) { return p.prec == 0 ? 4 : 8; }

int default_method(const Plan &p, size_t smem_limit)
{
    size_t cells = 1;
    for (int d = 0; d < p.dim; ++d) cells *= (size_t)padded(p.m[d], p.w);
    // SM (type 1: shared-memory subproblems; type 2: padded bin staged in shared
    // memory) unless the padded bin does not fit (Sec. 4.1 remark on 3D fp64)
    return cells * 2 * real_size(p) <= smem_limit ? NUFFT_METHOD_SM : NUFFT_METHOD_GM_SORT;
}

}  // namespace

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_nq.
void nufft::gauss_legendre(int nq, std::vector<double> &x, std::vector<double> &wt)
{
    const double PI = 3.14159265358979323846;
    x.assign(nq, 0.0);
    wt.assign(nq, 0.0);
    for (int i = 0; i < nq; ++i) {
        double z = cos(PI * (i + 0.75) / (nq + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= nq; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            // p1 = P_nq(z), p0 = P_{nq-1}(z)
            dp = nq * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int nufft::cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return NUFFT_OK;
    if (e == cudaErrorMemoryAllocation) return NUFFT_ERR_ALLOC;
    return NUFFT_ERR_CUDA;
}

int nufft::dev_alloc_raw(void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (injected_failure(NUFFT_FAIL_ALLOC)) return NUFFT_ERR_ALLOC;
    if (bytes == 0) bytes = 16;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free allocation error
        return NUFFT_ERR_ALLOC;
    }
    *ptr = v;
    return NUFFT_OK;
}

void nufft::dev_free(void *ptr)
{
    if (ptr) cudaFree(ptr);
}

// Frees the cuFFT plan (and its work area) of a plan that will only spread.
void nufft::plan_drop_fft(Plan &p)
{
    if (p.fft_ready) cufftDestroy(p.fft);
    p.fft_ready = false;
}

// Interior window cell i of a width-w kernel as a function of s in [-1, 1]:
// g_i(s) = phi_beta((i + 1 - w/2 - t) 2 / w), t = (s + 1) / 2 (Sec. 3 Eq. (es)).
static double kernel_cell_value(int w, double beta, int i, double s)
{
    const double t = 0.5 * (s + 1.0);
    const double z = (i + 1 - 0.5 * w - t) * 2.0 / w;
    const double q = 1.0 - z * z;
    return q >= 0.0 ? exp(beta * (sqrt(q) - 1.0)) : 0.0;
}

void nufft::fit_kernel_poly(Plan &p)
{
    const int w = p.w, D = poly_degree(p.w, p.prec);
    const double PI = 3.14159265358979323846;
    for (int i = 0; i < kMaxW; ++i)
        for (int d = 0; d < kPolyTerms; ++d) p.poly[i][d] = 0.0;
    double worst = 0.0;
    for (int i = 1; i + 1 < w; ++i) {
        // Chebyshev coefficients a_j from the values at the D + 1 first-kind nodes
        std::vector<double> f(D + 1), a(D + 1);
        for (int k = 0; k <= D; ++k)
            f[k] = kernel_cell_value(w, p.beta, i, cos(PI * (k + 0.5) / (D + 1)));
        for (int j = 0; j <= D; ++j) {
            double acc = 0.0;
            for (int k = 0; k <= D; ++k) acc += f[k] * cos(PI * j * (k + 0.5) / (D + 1));
            a[j] = acc * (j == 0 ? 1.0 : 2.0) / (D + 1);
        }
        // sum_j a_j T_j(s) as monomials: T_0 = 1, T_1 = s, T_{j+1} = 2 s T_j - T_{j-1}
        std::vector<double> tm(D + 1, 0.0), t0(D + 1, 0.0), t1(D + 1, 0.0), c(D + 1, 0.0);
        t0[0] = 1.0;
        c[0] += a[0];
        if (D >= 1) {
            t1[1] = 1.0;
            c[1] += a[1];
        }
        for (int j = 2; j <= D; ++j) {
            std::vector<double> tn(D + 1, 0.0);
            for (int d = 0; d <= D; ++d) {
                tn[d] = -t0[d];
                if (d > 0) tn[d] += 2.0 * t1[d - 1];
            }
            for (int d = 0; d <= D; ++d) c[d] += a[j] * tn[d];
            t0 = t1;
            t1 = tn;
        }
        for (int d = 0; d <= D; ++d) p.poly[i][d] = c[d];
        for (int k = 0; k <= 2000; ++k) {
            const double s = -1.0 + k / 1000.0;
            double v = c[D];
            for (int d = D - 1; d >= 0; --d) v = v * s + c[d];
            const double e = fabs(v - kernel_cell_value(w, p.beta, i, s));
            if (e > worst) worst = e;
        }
    }
    p.poly_ok = worst <= fmax(p.eps * 1e-3, p.prec == 0 ? 3e-8 : 1e-14);
}

int nufft::planes3_form(const Plan &p)
{
    if (p.method != NUFFT_METHOD_SM || p.dim != 3 || p.prec != 0 || p.w > 8) return 0;
    const int p0 = padded(p.m[0], p.w);
    return p0 <= 16 && (p.m[2] == 1 || p.m[2] == 2) ? p.m[2] + 4 : 0;
}

int nufft::sweep_variant(const Plan &p)
{
    if (p.method != NUFFT_METHOD_SM) return 0;
    const int p0 = padded(p.m[0], p.w);
    if (p.dim == 2 && p.type == 2) return 0;
    if (p.dim == 3) {
        // the plane-split sweeps read records ordered by start row (setpts)
        const int f = planes3_form(p);
        if (f) return p.row_ordered ? f : 0;
        if (p.type == 2) return 0;
        return p0 <= 32 && p.prec == 0 && p.w <= 8 && (p.m[2] == 1 || p.m[2] == 2) ? p.m[2] : 0;
    }
    return sweep2_form(p);
}

int nufft::sweep2_form(const Plan &p)
{
    if (p.method != NUFFT_METHOD_SM || p.dim != 2 || p.type != 1) return 0;
    const int p0 = padded(p.m[0], p.w);
    return p0 <= 8 ? 8 : (p0 <= 16 ? 16 : (p0 <= 32 ? 32 : 0));
}

bool nufft::tiles_feasible(const Plan &p, const Tiles &t)
{
    if (t.method < NUFFT_METHOD_GM || t.method > NUFFT_METHOD_SM) return false;
    if (t.msub < 1 || t.threads < 32 || t.threads > 256 || t.threads % 32) return false;
    size_t cells = 1;
    for (int d = 0; d < p.dim; ++d) {
        if (t.bin[d] < 1) return false;
        const int m = t.bin[d] > p.nf[d] ? (int)p.nf[d] : t.bin[d];
        if (padded(m, p.w) > 1023) return false;
        cells *= (size_t)padded(m, p.w);
    }
    return !(t.method == NUFFT_METHOD_SM && cells * 2 * real_size(p) > (size_t)p.smem_optin);
}

int nufft::plan_set_tiles(Plan &p, const Tiles &t)
{
    if (t.method < NUFFT_METHOD_GM || t.method > NUFFT_METHOD_SM) return NUFFT_ERR_ARG;
    if (t.msub < 1 || t.threads < 32 || t.threads > 256 || t.threads % 32) return NUFFT_ERR_ARG;
    int m[3] = {1, 1, 1}, nb[3] = {1, 1, 1};
    size_t cells = 1;
    for (int d = 0; d < p.dim; ++d) {
        if (t.bin[d] < 1) return NUFFT_ERR_ARG;
        m[d] = t.bin[d] > p.nf[d] ? (int)p.nf[d] : t.bin[d];
        if (padded(m[d], p.w) > 1023) return NUFFT_ERR_ARG;
        nb[d] = (int)((p.nf[d] + m[d] - 1) / m[d]);
        cells *= (size_t)padded(m[d], p.w);
    }
    if (t.method == NUFFT_METHOD_SM && cells * 2 * real_size(p) > (size_t)p.smem_optin)
        return NUFFT_ERR_METHOD;
    const int64_t nbins = (int64_t)nb[0] * nb[1] * nb[2];
    if (nbins != p.nbins) {
        dev_free(p.bincount);
        dev_free(p.binstart);
        dev_free(p.scan_tmp);
        p.bincount = p.binstart = p.scan_tmp = nullptr;
        int rc = dev_alloc(&p.bincount, sizeof(int32_t) * nbins);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.binstart, sizeof(int32_t) * nbins);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.scan_tmp, sizeof(int32_t) * nbins);
        if (rc != NUFFT_OK) return rc;
    }
    for (int d = 0; d < 3; ++d) {
        p.m[d] = m[d];
        p.nb[d] = nb[d];
    }
    p.nbins = nbins;
    p.method = t.method;
    p.msub = t.msub;
    p.threads = t.threads;
    p.maxsub = 0;                   // the subproblem list is resized by the next setpts
    p.have_pts = false;
    return NUFFT_OK;
}

extern "C" {

void nufft_default_opts(nufft_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->method = NUFFT_METHOD_AUTO;
    o->upsampfac = 2.0;
}

const char *nufft_strerror(int code)
{
    switch (code) {
    case NUFFT_OK: return "success";
    case NUFFT_ERR_ARG: return "invalid argument";
    case NUFFT_ERR_EPS: return "tolerance outside the supported range for this precision";
    case NUFFT_ERR_SIZE: return "mode count or fine grid too large";
    case NUFFT_ERR_ALLOC: return "device allocation failed";
    case NUFFT_ERR_CUDA: return "CUDA error";
    case NUFFT_ERR_CUFFT: return "cuFFT error";
    case NUFFT_ERR_NOPTS: return "execute called before setpts";
    case NUFFT_ERR_CHECK: return "a device-side check failed (debug_checks)";
    case NUFFT_ERR_METHOD: return "method not available for this plan";
    default: return "unknown error";
    }
}

int nufft_makeplan(int type, int dim, const int64_t *nmodes, int iflag, int ntransf, double eps,
                   int prec, const nufft_opts *opts, nufft_plan *out)
{
    if (!out) return NUFFT_ERR_ARG;
    *out = nullptr;
    if (type < 1 || type > 3 || dim < 1 || dim > 3 || (type != 3 && !nmodes)) return NUFFT_ERR_ARG;
    if (iflag != 1 && iflag != -1) return NUFFT_ERR_ARG;
    if (ntransf < 1 || prec < -1 || prec > 1) return NUFFT_ERR_ARG;
    if (!(eps > 0.0) || !isfinite(eps)) return NUFFT_ERR_EPS;
    nufft_opts o;
    nufft_default_opts(&o);
    if (opts) o = *opts;
    double sigma = o.upsampfac == 0.0 ? 2.0 : o.upsampfac;
    if (sigma != 2.0 && sigma != 1.25) return NUFFT_ERR_ARG;
    if (o.method < 0 || o.method > 3) return NUFFT_ERR_ARG;
    if (o.msub < 0 || o.threads < 0 || o.ctas_per_sm < 0) return NUFFT_ERR_ARG;
    if (o.threads != 0 && (o.threads % 32 != 0 || o.threads > 256)) return NUFFT_ERR_ARG;

    // Single precision reaches 1e-6 at sigma = 2; at sigma = 1.25 the correction
    // factors span ~100x more, which amplifies single-precision rounding of the
    // fine grid to ~1e-4, so single precision there needs eps >= 1e-4.
    const double fp32_floor = sigma == 2.0 ? 1e-6 : 1e-4;
    if (prec == -1) prec = eps >= fp32_floor ? 0 : 1;
    if (prec == 0 && eps < fp32_floor) return NUFFT_ERR_EPS;
    int w = kernel_width(eps, sigma);
    if (w > kMaxW) return NUFFT_ERR_EPS;
    if (type == 3) {
        // type 3: the grids depend on the points and frequencies, so the inner
        // plans are made at setpts (nufft_setpts3); sigma = 2 only
        if (sigma != 2.0) return NUFFT_ERR_ARG;
        nufft_plan_s *h3 = new (std::nothrow) nufft_plan_s;
        if (!h3) return NUFFT_ERR_ALLOC;
        Plan &q = h3->p;
        q.type = 3;
        q.dim = dim;
        q.iflag = iflag;
        q.ntransf = ntransf;
        q.prec = prec;
        q.eps = eps;
        q.sigma = sigma;
        q.w = w;
        q.beta = kernel_beta(w, sigma);
        q.stream = (cudaStream_t)o.stream;
        q.debug_checks = o.debug_checks != 0;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&q.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (q.num_sms < 1) q.num_sms = 1;
        const int rc = type3_init(q, o);
        if (rc != NUFFT_OK) {
            free_plan(q);
            delete h3;
            return rc;
        }
        *out = h3;
        return NUFFT_OK;
    }

    nufft_plan_s *h = new (std::nothrow) nufft_plan_s;
    if (!h) return NUFFT_ERR_ALLOC;
    Plan &p = h->p;
    p.type = type;
    p.dim = dim;
    p.iflag = iflag;
    p.ntransf = ntransf;
    p.prec = prec;
    p.eps = eps;
    p.sigma = sigma;
    p.w = w;
    p.beta = kernel_beta(w, sigma);
    fit_kernel_poly(p);
    p.stream = (cudaStream_t)o.stream;
    p.threads = o.threads ? o.threads : kDefaultThreads;
    p.ctas_per_sm = o.ctas_per_sm;
    p.msub = o.msub ? o.msub : 1024;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&p.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (p.num_sms < 1) p.num_sms = 1;
    p.smem_optin = smem_optin;

    int64_t ntot = 1, nftot = 1;
    for (int d = 0; d < 3; ++d) {
        if (d < dim) {
            if (nmodes[d] < 1 || nmodes[d] > (1 << 26)) { delete h; return NUFFT_ERR_SIZE; }
            p.N[d] = nmodes[d];
            int64_t want = (int64_t)ceil(sigma * (double)p.N[d] - 1e-9);
            if (want < 2 * w) want = 2 * w;
            p.nf[d] = next235(want);
            int defb[3];
            default_bins(type, dim, prec, w, defb);
            const int mdef = defb[d];
            int m = o.bin[d] > 0 ? o.bin[d] : mdef;
            if (m > p.nf[d]) m = (int)p.nf[d];
            if (padded(m, w) > 1023) { delete h; return NUFFT_ERR_ARG; }
            p.m[d] = m;
            p.nb[d] = (int)((p.nf[d] + m - 1) / m);
        } else {
            p.N[d] = 1;
            p.nf[d] = 1;
            p.m[d] = 1;
            p.nb[d] = 1;
        }
        ntot *= p.N[d];
        nftot *= p.nf[d];
    }
    if (nftot > ((int64_t)1 << 40) || (double)nftot * ntransf * 2 * real_size(p) > 4e11) {
        delete h;
        return NUFFT_ERR_SIZE;
    }
    p.Ntot = ntot;
    p.nftot = nftot;
    p.nbins = (int64_t)p.nb[0] * p.nb[1] * p.nb[2];
    if (p.nbins > ((int64_t)1 << 30)) { delete h; return NUFFT_ERR_SIZE; }

    p.method = o.method == NUFFT_METHOD_AUTO ? default_method(p, (size_t)smem_optin) : o.method;
    // measured / learned tiles (autotuner, picker) cover 2D and 3D
    p.auto_tiles = o.method == NUFFT_METHOD_AUTO && o.bin[0] == 0 && o.bin[1] == 0 &&
                   o.bin[2] == 0 && o.msub == 0 && o.threads == 0 && dim >= 2;
    p.use_picker = p.auto_tiles && o.use_picker != 0;
    p.unordered_bins = o.unordered_bins != 0;
    p.debug_checks = o.debug_checks != 0;
    if (p.method == NUFFT_METHOD_SM) {
        size_t cells = 1;
        for (int d = 0; d < dim; ++d) cells *= (size_t)padded(p.m[d], w);
        size_t need = cells * 2 * real_size(p);
        if (need > (size_t)smem_optin) { delete h; return NUFFT_ERR_METHOD; }
    }

    int rc = NUFFT_OK;
    const size_t csz = 2 * real_size(p);
    rc = dev_alloc(&p.fine, (size_t)nftot * ntransf * csz);
    for (int d = 0; d < 3 && rc == NUFFT_OK; ++d) rc = dev_alloc(&p.corr[d], (size_t)p.N[d] * real_size(p));
    if (rc == NUFFT_OK) rc = dev_alloc(&p.bincount, sizeof(int32_t) * p.nbins);
    if (rc == NUFFT_OK) rc = dev_alloc(&p.binstart, sizeof(int32_t) * p.nbins);
    if (rc == NUFFT_OK) rc = dev_alloc(&p.scan_tmp, sizeof(int32_t) * p.nbins);
    if (rc == NUFFT_OK) rc = dev_alloc(&p.nsub, sizeof(int32_t) * 4);
    if (rc == NUFFT_OK && p.debug_checks) {
        rc = dev_alloc(&p.dstatus, sizeof(int32_t));
        if (rc == NUFFT_OK && cudaMemsetAsync(p.dstatus, 0, sizeof(int32_t), p.stream) != cudaSuccess)
            rc = NUFFT_ERR_CUDA;
    }
    if (rc != NUFFT_OK) {
        free_plan(p);
        delete h;
        return rc;
    }

    // correction factors, in FP64 then rounded to the plan precision
    {
        const int nq = 64 + 4 * w;
        std::vector<double> gx, gw;
        gauss_legendre(nq, gx, gw);
        std::vector<double> st(nq), v(nq);
        const double PI = 3.14159265358979323846;
        for (int q = 0; q < nq; ++q) {
            double t = 0.5 * PI * gx[q];
            st[q] = sin(t);
            v[q] = 0.5 * PI * gw[q] * exp(p.beta * (cos(t) - 1.0)) * cos(t);
        }
        double *dst = nullptr, *dv = nullptr;
        rc = dev_alloc(&dst, sizeof(double) * nq);
        if (rc == NUFFT_OK) rc = dev_alloc(&dv, sizeof(double) * nq);
        cudaError_t e = cudaSuccess;
        if (rc == NUFFT_OK) e = cudaMemcpyAsync(dst, st.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, p.stream);
        if (rc == NUFFT_OK && e == cudaSuccess) e = cudaMemcpyAsync(dv, v.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, p.stream);
        if (rc == NUFFT_OK && e == cudaSuccess) e = launch_correction(p, dst, dv, nq);
        // axes beyond dim hold the single factor 1
        for (int d = dim; d < 3 && rc == NUFFT_OK && e == cudaSuccess; ++d) {
            if (p.prec == 0) {
                static const float one_f = 1.0f;
                e = cudaMemcpyAsync(p.corr[d], &one_f, sizeof(float), cudaMemcpyHostToDevice, p.stream);
            } else {
                static const double one_d = 1.0;
                e = cudaMemcpyAsync(p.corr[d], &one_d, sizeof(double), cudaMemcpyHostToDevice, p.stream);
            }
        }
        if (rc == NUFFT_OK && e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
        dev_free(dst);
        dev_free(dv);
        if (rc == NUFFT_OK && e != cudaSuccess) rc = cuda_err(e);
        if (rc != NUFFT_OK) {
            free_plan(p);
            delete h;
            return rc;
        }
    }

    // cuFFT plan for the fine grid, batched over ntransf (Sec. 4, step 2)
    {
        int dims[3];
        for (int d = 0; d < dim; ++d) dims[d] = (int)p.nf[dim - 1 - d];   // slowest first
        cufftResult r = injected_failure(NUFFT_FAIL_CUFFT)
                            ? CUFFT_INTERNAL_ERROR
                            : cufftPlanMany(&p.fft, dim, dims, nullptr, 1, (int)nftot, nullptr, 1,
                                            (int)nftot, p.prec == 0 ? CUFFT_C2C : CUFFT_Z2Z,
                                            ntransf);
        if (r == CUFFT_SUCCESS) {
            p.fft_ready = true;
            r = cufftSetStream(p.fft, p.stream);
        }
        if (r != CUFFT_SUCCESS) {
            free_plan(p);
            delete h;
            return r == CUFFT_ALLOC_FAILED ? NUFFT_ERR_ALLOC : NUFFT_ERR_CUFFT;
        }
    }
    *out = h;
    return NUFFT_OK;
}

int nufft_setpts(nufft_plan h, int64_t M, const void *x, const void *y, const void *z)
{
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (p.type == 3) return NUFFT_ERR_ARG;   // nufft_setpts3
    p.row_ordered = false;
    if (M < 0 || M >= ((int64_t)1 << 31) - 1) return NUFFT_ERR_ARG;
    if (M > 0 && (!x || (p.dim >= 2 && !y) || (p.dim == 3 && !z))) return NUFFT_ERR_ARG;
    p.have_pts = false;
    if (p.auto_tiles) {
        // measured tiles from the autotuner's cache first, then the picker's
        // prediction, else the heuristic tiles chosen at makeplan stay
        Tiles t;
        bool have = tune_cache_lookup(p, M, &t);
        if (!have && p.use_picker) {
            const int rc = picker_choose(p, M, x, y, z, &t, &have);
            if (rc != NUFFT_OK) return rc;
        }
        if (have && (t.method != p.method || t.msub != p.msub || t.threads != p.threads ||
                     t.bin[0] != p.m[0] || t.bin[1] != p.m[1] || t.bin[2] != p.m[2])) {
            const int rc = plan_set_tiles(p, t);
            if (rc != NUFFT_OK) return rc;
        }
    }
    const int64_t maxsub = p.nbins + M / p.msub + 1;
    if (M > p.Mcap || maxsub > p.maxsub) {
        free_points(p);
        const int64_t cap = M > 0 ? M : 1;
        const size_t rsz = p.prec == 0 ? sizeof(float4) : sizeof(double4_32a);
        int rc = dev_alloc(&p.keys, sizeof(int32_t) * cap);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.keys_alt, sizeof(int32_t) * cap);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.vals, sizeof(int32_t) * cap);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.vals_alt, sizeof(int32_t) * cap);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.recs, rsz * cap);
        if (rc == NUFFT_OK && p.dim == 3) rc = dev_alloc(&p.rorder, sizeof(int32_t) * cap);
        if (rc == NUFFT_OK && p.dim == 3) rc = dev_alloc(&p.recs2, rsz * cap);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.subprob, sizeof(int4) * maxsub);
        if (rc != NUFFT_OK) {
            free_points(p);
            return rc;
        }
        p.Mcap = cap;
        p.maxsub = maxsub;
    }
    if (p.method == NUFFT_METHOD_GM) {
        // GM works in user order (Sec. 4.1): keep a copy of the coordinates, no sort
        for (int d = 0; d < p.dim; ++d) {
            if (!p.xyz_copy[d]) {
                int rc = dev_alloc(&p.xyz_copy[d], real_size(p) * p.Mcap);
                if (rc != NUFFT_OK) return rc;
            }
        }
        const void *src[3] = {x, y, z};
        for (int d = 0; d < p.dim && M > 0; ++d) {
            cudaError_t e = cudaMemcpyAsync(p.xyz_copy[d], src[d], real_size(p) * M,
                                            cudaMemcpyDeviceToDevice, p.stream);
            if (e != cudaSuccess) return cuda_err(e);
        }
        // work count of the plan in a batched launch: chunks of kGmChunk points
        cudaError_t e = launch_set_int(p, p.nsub, (int32_t)((M + kGmChunk - 1) / kGmChunk));
        if (e != cudaSuccess) return cuda_err(e);
        p.M = M;
        p.have_pts = true;
        return NUFFT_OK;
    }
    p.M = M;
    // sort matrix and scan scratch for this M
    {
        const int cblk = counting_sort_blocks(p, M > 0 ? M : 1);
        const int rblk = radix_sort_blocks(p, M > 0 ? M : 1);
        int64_t mat = cblk > 0 ? p.nbins * cblk : 256 * (int64_t)rblk;
        int64_t L = mat > p.nbins ? mat : p.nbins;
        int64_t parts = scan_parts_needed(L);
        // the counting sort keeps an int2 of sums per 32 bins there
        const int64_t groups = 2 * ((p.nbins + 31) / 32);
        if (parts < groups) parts = groups;
        if (mat > p.mat_cap) {
            dev_free(p.mat);
            p.mat = nullptr;
            p.mat_cap = 0;
            int rc = dev_alloc(&p.mat, sizeof(int32_t) * mat);
            if (rc != NUFFT_OK) return rc;
            p.mat_cap = mat;
        }
        if (parts > p.scan_part_cap) {
            dev_free(p.scan_part);
            p.scan_part = nullptr;
            p.scan_part_cap = 0;
            int rc = dev_alloc(&p.scan_part, sizeof(int32_t) * parts);
            if (rc != NUFFT_OK) return rc;
            p.scan_part_cap = parts;
        }
    }
    cudaError_t e = launch_setpts(p, x, y, z);
    if (e == cudaSuccess && p.debug_checks) e = launch_checks(p, x, y, z);
    if (e != cudaSuccess) return cuda_err(e);
    p.have_pts = true;
    return NUFFT_OK;
}

int nufft_setpts3(nufft_plan h, int64_t M, const void *x, const void *y, const void *z, int64_t K,
                  const void *s, const void *t, const void *u)
{
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (p.type != 3) return NUFFT_ERR_ARG;
    if (M < 0 || M >= ((int64_t)1 << 31) - 1 || K < 0 || K >= ((int64_t)1 << 31) - 1)
        return NUFFT_ERR_ARG;
    if (M > 0 && (!x || (p.dim >= 2 && !y) || (p.dim == 3 && !z))) return NUFFT_ERR_ARG;
    if (K > 0 && (!s || (p.dim >= 2 && !t) || (p.dim == 3 && !u))) return NUFFT_ERR_ARG;
    p.have_pts = false;
    const void *xs[3] = {x, y, z}, *ss[3] = {s, t, u};
    return type3_setpts(p, M, xs, K, ss);
}

int nufft_spread(nufft_plan h, const void *c)
{
    if (h && h->p.type == 3) return NUFFT_ERR_ARG;   // stages of types 1 and 2
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (!p.have_pts) return NUFFT_ERR_NOPTS;
    if (p.M > 0 && !c) return NUFFT_ERR_ARG;
    cudaError_t e = launch_zero(p, p.fine, (size_t)p.nftot * p.ntransf * 2 * real_size(p));
    if (e != cudaSuccess) return cuda_err(e);
    return nufft_spread_add(h, c);
}

int nufft_spread_add(nufft_plan h, const void *c)
{
    if (h && h->p.type == 3) return NUFFT_ERR_ARG;   // stages of types 1 and 2
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (!p.have_pts) return NUFFT_ERR_NOPTS;
    if (p.M == 0) return NUFFT_OK;
    if (!c) return NUFFT_ERR_ARG;
    cudaError_t e;
    int method = p.method;
    if (p.type == 2 && method == NUFFT_METHOD_SM) p.method = NUFFT_METHOD_GM_SORT;   // SM spread needs its smem
    if (p.prec == 0)
        e = p.dim == 1 ? spread_f32_1d(p, c) : p.dim == 2 ? spread_f32_2d(p, c) : spread_f32_3d(p, c);
    else
        e = p.dim == 1 ? spread_f64_1d(p, c) : p.dim == 2 ? spread_f64_2d(p, c) : spread_f64_3d(p, c);
    p.method = method;
    return cuda_err(e);
}

int nufft_interp(nufft_plan h, void *c)
{
    if (h && h->p.type == 3) return NUFFT_ERR_ARG;   // stages of types 1 and 2
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (!p.have_pts) return NUFFT_ERR_NOPTS;
    if (p.M == 0) return NUFFT_OK;
    if (!c) return NUFFT_ERR_ARG;
    cudaError_t e;
    if (p.prec == 0)
        e = p.dim == 1 ? interp_f32_1d(p, c) : p.dim == 2 ? interp_f32_2d(p, c) : interp_f32_3d(p, c);
    else
        e = p.dim == 1 ? interp_f64_1d(p, c) : p.dim == 2 ? interp_f64_2d(p, c) : interp_f64_3d(p, c);
    return cuda_err(e);
}

int nufft_fft(nufft_plan h)
{
    if (h && h->p.type == 3) return NUFFT_ERR_ARG;   // stages of types 1 and 2
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    // type 1 FFT takes the sign of iflag, type 2 the opposite (Eq. 2d1 / 2d2)
    const int sign = p.type == 1 ? p.iflag : -p.iflag;
    const int dir = sign > 0 ? CUFFT_INVERSE : CUFFT_FORWARD;
    cufftResult r;
    if (p.prec == 0)
        r = cufftExecC2C(p.fft, (cufftComplex *)p.fine, (cufftComplex *)p.fine, dir);
    else
        r = cufftExecZ2Z(p.fft, (cufftDoubleComplex *)p.fine, (cufftDoubleComplex *)p.fine, dir);
    return r == CUFFT_SUCCESS ? NUFFT_OK : NUFFT_ERR_CUFFT;
}

int nufft_deconvolve(nufft_plan h, void *f)
{
    if (h && h->p.type == 3) return NUFFT_ERR_ARG;   // stages of types 1 and 2
    if (!h || !f) return NUFFT_ERR_ARG;
    return cuda_err(launch_deconvolve(h->p, f));
}

int nufft_precorrect(nufft_plan h, const void *f)
{
    if (h && h->p.type == 3) return NUFFT_ERR_ARG;   // stages of types 1 and 2
    if (!h || !f) return NUFFT_ERR_ARG;
    return cuda_err(launch_precorrect(h->p, f));
}

int nufft_execute(nufft_plan h, void *c, void *f)
{
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (p.type == 3) return p.have_pts ? type3_execute(p, c, f) : NUFFT_ERR_NOPTS;
    if (!f) return NUFFT_ERR_ARG;
    if (!p.have_pts) return NUFFT_ERR_NOPTS;
    if (p.M > 0 && !c) return NUFFT_ERR_ARG;
    int rc;
    if (p.type == 1) {
        if ((rc = nufft_spread(h, c)) != NUFFT_OK) return rc;
        if ((rc = nufft_fft(h)) != NUFFT_OK) return rc;
        return nufft_deconvolve(h, f);
    }
    if ((rc = nufft_precorrect(h, f)) != NUFFT_OK) return rc;
    if ((rc = nufft_fft(h)) != NUFFT_OK) return rc;
    return nufft_interp(h, c);
}

int nufft_execute_host(nufft_plan h, int64_t M, const void *x, const void *y, const void *z,
                       void *c, void *f)
{
    if (!h || !f) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (p.type == 3) return NUFFT_ERR_ARG;
    if (M < 0 || M >= ((int64_t)1 << 31) - 1) return NUFFT_ERR_ARG;
    if (M > 0 && (!x || (p.dim >= 2 && !y) || (p.dim == 3 && !z) || !c)) return NUFFT_ERR_ARG;
    const size_t rs = real_size(p), cs = 2 * rs;
    int rc = NUFFT_OK;
    // staging and the copy stream, made once and grown with M
    if (!p.hx_copy) {
        cudaError_t e = cudaStreamCreateWithFlags(&p.hx_copy, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&p.hx_ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_err(e);
    }
    if (!p.hx_f) {
        rc = dev_alloc(&p.hx_f, (size_t)p.Ntot * p.ntransf * cs);
        if (rc != NUFFT_OK) return rc;
    }
    if (M > p.hx_cap) {
        free_host_staging(p);
        for (int d = 0; d < p.dim && rc == NUFFT_OK; ++d) rc = dev_alloc(&p.hx_pts[d], rs * M);
        if (rc == NUFFT_OK) rc = dev_alloc(&p.hx_c, cs * (size_t)M * p.ntransf);
        if (rc != NUFFT_OK) {
            free_host_staging(p);
            return rc;
        }
        p.hx_cap = M;
    }
    cudaStream_t st = p.stream;
    // the staging may still be in use by the previous call's kernels
    cudaError_t e = cudaEventRecord(p.hx_ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.hx_copy, p.hx_ev[0], 0);
    // points first, on the plan stream, so the sort starts as soon as they arrive
    const void *src[3] = {x, y, z};
    for (int d = 0; d < p.dim && M > 0 && e == cudaSuccess; ++d)
        e = cudaMemcpyAsync(p.hx_pts[d], src[d], rs * M, cudaMemcpyHostToDevice, st);
    // the input of the transform on the copy stream, overlapping the sort
    if (e == cudaSuccess) {
        if (p.type == 1) {
            if (M > 0)
                e = cudaMemcpyAsync(p.hx_c, c, cs * (size_t)M * p.ntransf, cudaMemcpyHostToDevice,
                                    p.hx_copy);
        } else {
            e = cudaMemcpyAsync(p.hx_f, f, cs * (size_t)p.Ntot * p.ntransf, cudaMemcpyHostToDevice,
                                p.hx_copy);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(p.hx_ev[1], p.hx_copy);
    if (e != cudaSuccess) return cuda_err(e);
    rc = nufft_setpts(h, M, p.hx_pts[0], p.dim >= 2 ? p.hx_pts[1] : nullptr,
                      p.dim == 3 ? p.hx_pts[2] : nullptr);
    if (rc != NUFFT_OK) return rc;
    e = cudaStreamWaitEvent(st, p.hx_ev[1], 0);
    if (e != cudaSuccess) return cuda_err(e);
    rc = nufft_execute(h, p.hx_c, p.hx_f);
    if (rc != NUFFT_OK) return rc;
    if (p.type == 1)
        e = cudaMemcpyAsync(f, p.hx_f, cs * (size_t)p.Ntot * p.ntransf, cudaMemcpyDeviceToHost, st);
    else if (M > 0)
        e = cudaMemcpyAsync(c, p.hx_c, cs * (size_t)M * p.ntransf, cudaMemcpyDeviceToHost, st);
    return cuda_err(e);
}

uint64_t nufft_get_launch_count(void)
{
    return (uint64_t)g_launch_count.load(std::memory_order_relaxed);
}

int nufft_destroy(nufft_plan h)
{
    if (!h) return NUFFT_OK;
    free_plan(h->p);
    delete h;
    return NUFFT_OK;
}

int nufft_get_params(nufft_plan h, int *w, double *beta, int64_t *nf, int *bins, int64_t *nbins,
                     int *prec, int *method)
{
    if (!h) return NUFFT_ERR_ARG;
    const Plan &p = h->p;
    if (w) *w = p.w;
    if (beta) *beta = p.beta;
    int64_t g3[3] = {1, 1, 1};
    if (p.type == 3) type3_grid(p, g3);
    for (int d = 0; d < 3; ++d) {
        if (nf) nf[d] = p.type == 3 ? g3[d] : p.nf[d];
        if (bins) bins[d] = p.m[d];
    }
    if (nbins) *nbins = p.nbins;
    if (prec) *prec = p.prec;
    if (method) *method = p.method;
    return NUFFT_OK;
}

int nufft_get_finegrid(nufft_plan h, void **dptr, size_t *bytes)
{
    if (h && h->p.type == 3) return NUFFT_ERR_ARG;   // stages of types 1 and 2
    if (!h) return NUFFT_ERR_ARG;
    const Plan &p = h->p;
    if (dptr) *dptr = p.fine;
    if (bytes) *bytes = (size_t)p.nftot * p.ntransf * 2 * real_size(p);
    return NUFFT_OK;
}

int nufft_get_tiles(nufft_plan h, nufft_opts *out)
{
    if (!h || !out) return NUFFT_ERR_ARG;
    const Plan &p = h->p;
    out->method = p.method;
    for (int d = 0; d < 3; ++d) out->bin[d] = p.m[d];
    out->msub = p.msub;
    out->threads = p.threads;
    return NUFFT_OK;
}

int nufft_get_status(nufft_plan h)
{
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (!p.debug_checks || !p.dstatus) return NUFFT_OK;
    int32_t v = 0;
    cudaError_t e = cudaStreamSynchronize(p.stream);
    if (e == cudaSuccess) e = cudaMemcpy(&v, p.dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0) e = cudaMemset(p.dstatus, 0, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_err(e);
    return v != 0 ? NUFFT_ERR_CHECK : NUFFT_OK;
}

int nufft_debug_fail(int kind, int after)
{
    if (kind != NUFFT_FAIL_ALLOC && kind != NUFFT_FAIL_CUFFT) return NUFFT_ERR_ARG;
    const int calls = g_fail_calls[kind].exchange(0);
    g_fail_after[kind].store(after < 0 ? -1 : after);
    return calls;
}

int nufft_get_sort(nufft_plan h, int32_t *t, int32_t *bincounts, int32_t *nsub)
{
    if (!h) return NUFFT_ERR_ARG;
    Plan &p = h->p;
    if (p.type == 3) return NUFFT_ERR_ARG;
    if (!p.have_pts) return NUFFT_ERR_NOPTS;
    if (p.method == NUFFT_METHOD_GM) return NUFFT_ERR_METHOD;
    cudaError_t e = cudaSuccess;
    if (t && p.M > 0) e = cudaMemcpyAsync(t, p.perm, sizeof(int32_t) * p.M, cudaMemcpyDeviceToDevice, p.stream);
    if (e == cudaSuccess && bincounts)
        e = cudaMemcpyAsync(bincounts, p.bincount, sizeof(int32_t) * p.nbins, cudaMemcpyDeviceToDevice, p.stream);
    if (e == cudaSuccess && nsub)
        e = cudaMemcpyAsync(nsub, p.nsub, sizeof(int32_t), cudaMemcpyDeviceToDevice, p.stream);
    return cuda_err(e);
}

}  // extern "C"
