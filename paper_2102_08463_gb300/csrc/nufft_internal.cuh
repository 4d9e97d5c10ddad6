// nufft_internal.cuh -- plan object and device helpers shared by the library's
// translation units.  See include/nufft_gb300.h for the public contract.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/nufft_gb300.h"

namespace nufft {

constexpr int kMaxW = 16;

// Raises a kernel's dynamic shared-memory limit to the device's maximum, once
// per (kernel, current device); thread-safe.
cudaError_t allow_max_smem(const void *func);

// Fault injection (nufft_debug_fail): true if the armed failure of this kind
// fires now; counts the calls of each kind.
bool injected_failure(int kind);

// Process-wide count of kernel launches made by this library.
extern std::atomic<unsigned long long> g_launch_count;
inline void count_launch(unsigned n = 1) { g_launch_count.fetch_add(n, std::memory_order_relaxed); }
constexpr int kDefaultThreads = 256;
constexpr int kPolyTerms = 17;     // polynomial degree <= 16
// Points per work item of a GM plan in a batched launch.
constexpr int kGmChunk = 2048;
// Default 2D type 1 bins, sized for the row-sweep spreader: the padded width
// m0 + w fills 8 lanes (w <= 3, single precision) or 16 lanes, so a warp
// sweeps 4 or 2 points per step; taller bins in double precision and at
// small w amortise the row flushes.
inline int default_bin_2d_type1(int axis, int prec, int w)
{
    if (prec == 0 && w <= 3) return axis == 0 ? 8 - w : 32;
    if (axis == 0) return w <= 15 ? 16 - w : 32 - w;
    return prec == 0 ? 16 : 32;
}
// Default bin sizes of a plan (1 on unused axes): 512 (1D), 16 x 16 (2D) and
// 16 x 16 x 2 (3D), with the row-sweep sizes above for 2D type 1 and, for 3D single
// precision at w <= 8 (both types), the plane-split sizes (16 - w) x 64 x 1
// (w odd) or (16 - w) x 32 x 2 (w even): the padded width fills 16 lanes and
// the padded depth m2 + w is even, so the two half-warps own equal plane sets;
// the tall bins amortise the row flushes and loads (29 x 4 x 256 bins on a
// 256^3 grid at w = 7, within the shared-memory counting sort).
inline void default_bins(int type, int dim, int prec, int w, int out[3])
{
    for (int d = 0; d < 3; ++d) out[d] = d < dim ? (dim == 2 ? 16 : (d < 2 ? 16 : 2)) : 1;
    if (dim == 1) out[0] = 512;
    if (dim == 2 && type == 1)
        for (int d = 0; d < 2; ++d) out[d] = default_bin_2d_type1(d, prec, w);
    if (dim == 3 && prec == 0 && w <= 8) {
        out[0] = 16 - w;
        out[1] = w % 2 ? 64 : 32;
        out[2] = w % 2 ? 1 : 2;
    }
}
// Degree of the kernel polynomials of width w: the fits of the interior window
// cells reach eps / 1000 of the smallest tolerance that gives width w (floor
// 3e-8 single / 1e-14 double): single 6 (w <= 3), 7 (w = 4), 8; double w + 2.
// Every plan checks its own fit (fit_kernel_poly) and evaluates the kernel
// directly if the fit misses that bound.
__host__ __device__ constexpr int poly_degree(int w, int prec)
{
    return prec == 0 ? (w <= 3 ? 6 : (w == 4 ? 7 : 8)) : (w + 2 < kPolyTerms - 1 ? w + 2 : kPolyTerms - 1);
}

// Complex storage types matching cuFFT's interleaved layout.
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };

// Packed per-point record: kernel offsets delta_i = u_i - l0_i
// (u_i the fine-grid coordinate, l0_i the first window cell) and the window
// start relative to the padded bin, three 10-bit fields in one 32-bit word
// stored in the last slot.  In 2D the z slot holds the point's original index
// (as the bits of a 32-bit word).
template <typename T> struct rec4;
template <> struct rec4<float> { using type = float4; };
template <> struct rec4<double> { using type = double4_32a; };

struct Plan;

// ---------------------------------------------------------------------------
// Position rule shared by setpts and the unsorted (GM) kernels.
//
// A coordinate x is turned into a 64-bit fraction Phi of the period,
// Phi / 2^64 = (x + pi) / (2 pi) mod 1, in exact integer arithmetic:
//   X   = round-half-even(clamp(x, -1024, 1024) * 2^52)
//   Q   = floor(|X| * K / 2^64) mod 2^64, K = round(2^76 / (2 pi))
//   Phi = 2^63 + sign(X) Q mod 2^64
// and along an axis with n cells: cell l = floor(Phi n / 2^64), fraction
// F = Phi n mod 2^64.  Integer-only, so the bin of every point is the same on
// any machine (the paper's floor((x+pi)/h), Sec. 4.1, with the rounding fixed).
// ---------------------------------------------------------------------------
constexpr uint64_t kKHi = 651ULL;
constexpr uint64_t kKLo = 0xe60db9391054a7f1ULL;

__device__ __forceinline__ long long coord_fixed(float x)
{
    float xc = x;
    if (!(xc >= -1024.0f)) xc = -1024.0f;
    if (xc > 1024.0f) xc = 1024.0f;
    return __float2ll_rn(xc * 0x1p52f);        // exact scaling, then round-half-even
}
__device__ __forceinline__ long long coord_fixed(double x)
{
    double xc = x;
    if (!(xc >= -1024.0)) xc = -1024.0;
    if (xc > 1024.0) xc = 1024.0;
    return __double2ll_rn(xc * 0x1p52);
}

__device__ __forceinline__ uint64_t period_fraction_fx(long long X)
{
    uint64_t A = X < 0 ? (uint64_t)(-X) : (uint64_t)X;
    uint64_t Q = A * kKHi + __umul64hi(A, kKLo);
    return (1ULL << 63) + (X < 0 ? (0ULL - Q) : Q);
}

template <typename T>
__device__ __forceinline__ uint64_t period_fraction(T x)
{
    return period_fraction_fx(coord_fixed(x));
}

// Cell, window start and kernel offset along one axis.
//   l     = floor(u), u the fine-grid coordinate (Sec. 4.1 bin rule)
//   l0    = ceil(u - w/2), first of the w window cells (unwrapped, may be < 0)
//   delta = u - l0, so the kernel argument of window cell i is (i - delta) * 2/w
template <typename T>
struct AxisPos { int l; int l0; T delta; };

template <typename T>
__device__ __forceinline__ AxisPos<T> axis_position(uint64_t phi, int n, int w)
{
    AxisPos<T> r;
    uint64_t F = phi * (uint64_t)n;
    r.l = (int)__umul64hi(phi, (uint64_t)n);
    int e;                                       // l - l0
    if (w & 1) e = (w - 1) / 2 - (F > (1ULL << 63) ? 1 : 0);
    else       e = w / 2 - (F != 0 ? 1 : 0);
    r.l0 = r.l - e;
    T f;
    if (sizeof(T) == 4) f = (T)(float)(F >> 40) * (T)0x1p-24;
    else                f = (T)(double)(F >> 11) * (T)0x1p-53;
    r.delta = (T)e + f;
    return r;
}

// Padded bin of Sec. 4.1 SM step 2: a point whose cell lies in a bin of m
// cells has its w-cell window inside the m + w cells starting floor(w/2) before
// the bin origin (the paper's p_i = m_i + 2 ceil(w/2) is one cell larger for
// odd w; the window never reaches that cell).
__host__ __device__ __forceinline__ int pad_lo(int w) { return w / 2; }
__host__ __device__ __forceinline__ int padded(int m, int w) { return m + w; }

// ES kernel, Sec. 3 Eq. (es): phi_beta(z) = exp(beta (sqrt(1 - z^2) - 1)), |z| <= 1.
__device__ __forceinline__ float es_kernel(float z, float beta)
{
    float s = 1.0f - z * z;
    return s >= 0.0f ? expf(beta * (sqrtf(s) - 1.0f)) : 0.0f;
}
__device__ __forceinline__ double es_kernel(double z, double beta)
{
    double s = 1.0 - z * z;
    return s >= 0.0 ? exp(beta * (sqrt(s) - 1.0)) : 0.0;
}

__device__ __forceinline__ int wrap_index(int l, int n)
{
    // l within (-n, 2n): one conditional correction
    return l < 0 ? l + n : (l >= n ? l - n : l);
}

// Atomic complex add into global memory as reductions (no value returned, so
// the issuing warp does not wait for the L2 round trip): one 8-byte vector
// reduction for single precision (sm_90+), two 8-byte ones for double.
// No memory clobber: no kernel reads the grid it reduces into, so the compiler
// may schedule other loads and stores around the reductions.
__device__ __forceinline__ void atomic_add_cplx(float2 *p, float re, float im)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(re), "f"(im));
}
__device__ __forceinline__ void atomic_add_cplx(double2 *p, double re, double im)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(&p->x), "d"(re));
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(&p->y), "d"(im));
}

// ---------------------------------------------------------------------------
// Plan object (Sec. 1.1 plan / setup / execute / destroy).
// ---------------------------------------------------------------------------
struct Type3;   // type 3 state (type3.cu)

struct Plan {
    int type = 1, dim = 2, iflag = 1, ntransf = 1, prec = 0;
    double eps = 1e-6, sigma = 2.0, beta = 0.0;
    int w = 0;
    int64_t N[3] = {1, 1, 1};
    int64_t nf[3] = {1, 1, 1};
    int64_t Ntot = 1, nftot = 1;
    int method = NUFFT_METHOD_SM;
    int m[3] = {1, 1, 1};
    int nb[3] = {1, 1, 1};
    int64_t nbins = 1;
    int msub = 1024;
    int threads = kDefaultThreads;
    int ctas_per_sm = 0;
    int num_sms = 152;
    cudaStream_t stream = nullptr;

    bool fft_ready = false;
    cufftHandle fft = 0;

    void *fine = nullptr;          // ntransf * nftot complex
    void *corr[3] = {nullptr, nullptr, nullptr};   // per-axis correction factors (T), N_i each

    // setpts state
    bool have_pts = false;
    int64_t M = 0, Mcap = 0;
    const void *xyz[3] = {nullptr, nullptr, nullptr};   // caller's arrays (GM only)
    int32_t *keys = nullptr;       // [Mcap] bin per point, user order
    int32_t *keys_alt = nullptr;   // [Mcap] radix ping-pong
    int32_t *vals = nullptr;       // [Mcap]
    int32_t *vals_alt = nullptr;   // [Mcap]
    int32_t *perm = nullptr;       // [Mcap] t: sorted position -> original index
    int32_t *rorder = nullptr;     // [Mcap] 3D: record position -> original index
    bool row_ordered = false;      // records ordered by start row inside each subproblem
    void *recs = nullptr;          // [Mcap] rec4<T> per point, in t order (see setpts.cu)
    void *recs2 = nullptr;         // [Mcap] 3D: the other record buffer of the row ordering
    void *xyz_copy[3] = {nullptr, nullptr, nullptr};  // coordinate copies for GM
    int32_t *bincount = nullptr;   // [nbins]
    int32_t *binstart = nullptr;   // [nbins]
    int4 *subprob = nullptr;       // [maxsub] (bin, start, count, 0)
    int64_t maxsub = 0;
    int32_t *nsub = nullptr;       // [1] device scalar: subproblems (GM: kGmChunk chunks)
    int32_t *mat = nullptr;        // sort histogram matrix (bins or digits) x CTAs
    int64_t mat_cap = 0;
    int32_t *scan_part = nullptr;  // block sums of the multi-block scan
    int64_t scan_part_cap = 0;
    int32_t *scan_tmp = nullptr;   // [nbins] subproblem offsets per bin
    int smem_optin = 0;            // max dynamic shared memory per CTA (bytes)
    int smem_per_sm = 0;           // shared memory per SM (bytes)
    bool auto_tiles = false;       // method, bins and msub left to the library
    // Piecewise polynomial form of the kernel: for interior window cell i
    // (1 <= i <= w - 2), phi((i - delta) 2 / w) = sum_d poly[i][d] s^d with
    // s = 2 (delta - w/2 + 1) - 1 in (-1, 1]; poly_ok when the fit met its bound.
    double poly[kMaxW][kPolyTerms] = {};
    bool poly_ok = false;
    bool use_picker = false;       // consult the installed tile picker at setpts
    bool unordered_bins = false;   // counting-sort scatter in shared-atomic order
    bool debug_checks = false;     // device-side checks at setpts (status word)
    int32_t *dstatus = nullptr;    // [1] device status of the checks (0 = passed)

    // host-buffer execute (nufft_execute_host): device staging, grown on demand
    void *hx_pts[3] = {nullptr, nullptr, nullptr};   // coordinates [hx_cap]
    void *hx_c = nullptr;          // ntransf * M complex
    void *hx_f = nullptr;          // ntransf * Ntot complex
    int64_t hx_cap = 0;            // points the staging holds
    cudaStream_t hx_copy = nullptr;   // stream of the input copy
    cudaEvent_t hx_ev[2] = {nullptr, nullptr};   // entry, input copied

    Type3 *t3 = nullptr;           // type 3 plans: inner plans and per-point factors
};

// Tile settings of a plan (method, bin sizes, subproblem cap, threads per CTA).
struct Tiles {
    int method = NUFFT_METHOD_SM;
    int bin[3] = {1, 1, 1};
    int msub = 1024;
    int threads = 256;
};
// Fits plan.poly (Chebyshev interpolation of each interior cell, converted to
// monomials in s) and sets plan.poly_ok if the fit is within its bound on a fine
// sampling of s.
void fit_kernel_poly(Plan &p);
// Re-tile an existing plan (keeps its cuFFT plan and fine grid); the points
// must be set again afterwards.  Returns an NUFFT_ERR_* code.
int plan_set_tiles(Plan &p, const Tiles &t);
// Whether plan_set_tiles would accept t for this plan (no state is changed).
bool tiles_feasible(const Plan &p, const Tiles &t);
// Tuned tiles for this plan and M from the autotuner's cache, if any.
bool tune_cache_lookup(const Plan &p, int64_t M, Tiles *out);
// The candidate tilings the autotuner times and the picker ranks, in a fixed
// order: a grid of bins x M_sub x threads for SM and GM-sort, one GM entry, and
// the plan's default tiling when the grid does not contain it.
std::vector<Tiles> tile_candidates(const Plan &p);
// Tiles chosen by the installed picker for this plan and these points.  Sets
// *chosen = false (and returns NUFFT_OK) when no picker is installed.
// Synchronizes p.stream.
int picker_choose(Plan &p, int64_t M, const void *x, const void *y, const void *z, Tiles *out,
                  bool *chosen);
// Parameter rules of Sec. 3 shared by makeplan and the picker's features.
int next235(int64_t n);
// Device allocation (NUFFT_ERR_ALLOC on failure, honouring nufft_debug_fail) and
// the CUDA-to-NUFFT error mapping shared by the host code.
int cuda_err(cudaError_t e);
int dev_alloc_raw(void **ptr, size_t bytes);
template <typename Ptr>
inline int dev_alloc(Ptr **ptr, size_t bytes)
{
    void *v = nullptr;
    const int rc = dev_alloc_raw(&v, bytes);
    *ptr = reinterpret_cast<Ptr *>(v);
    return rc;
}
void dev_free(void *ptr);
// Gauss-Legendre nodes and weights on [-1, 1].
void gauss_legendre(int nq, std::vector<double> &x, std::vector<double> &wt);
// Frees the cuFFT plan of a plan used for spreading only.
void plan_drop_fft(Plan &p);
// Type 3 (type3.cu): state set-up at makeplan, points and frequencies, execute,
// release, and the size of its spreading grid.
int type3_init(Plan &p, const nufft_opts &o);
void type3_free(Plan &p);
int type3_setpts(Plan &p, int64_t M, const void *const *x, int64_t K, const void *const *s);
int type3_execute(Plan &p, const void *c, void *f);
void type3_grid(const Plan &p, int64_t *n);
int kernel_width(double eps, double sigma);

// Launchers implemented in the .cu files.  All enqueue on p.stream and return a
// cudaError_t from the last launch.
cudaError_t launch_setpts(Plan &p, const void *x, const void *y, const void *z);
cudaError_t launch_scan(Plan &p, const int32_t *in, int32_t *out, int64_t L, int32_t *total);
// debug_checks: coordinates finite and in [-3 pi, 3 pi]; t a permutation of 0..M-1.
cudaError_t launch_checks(Plan &p, const void *x, const void *y, const void *z);

// Scratch of the bin-sort when the caller supplies it (allocation-free entry point).
struct BinsortScratch {
    int32_t *keys;        // [M]
    int32_t *mat;         // [nblk * nbins]
    int32_t *binstart;    // [nbins]
    int32_t *scan_part;   // scan block sums
    int nblk;             // CTAs of the counting sort
};
cudaError_t launch_binsort_into(const BinsortScratch &s, int prec, int dim, int64_t M,
                                const void *x, const void *y, const void *z, const int64_t *nf,
                                const int *bins, int32_t *perm, int32_t *bincount,
                                cudaStream_t st);
int64_t scan_parts_needed(int64_t L);
int counting_sort_blocks(const Plan &p, int64_t M);
int radix_sort_blocks(const Plan &p, int64_t M);
cudaError_t spread_f32_1d(Plan &p, const void *c);
cudaError_t spread_f32_2d(Plan &p, const void *c);
cudaError_t spread_f32_3d(Plan &p, const void *c);
cudaError_t spread_f64_1d(Plan &p, const void *c);
cudaError_t spread_f64_2d(Plan &p, const void *c);
cudaError_t spread_f64_3d(Plan &p, const void *c);
cudaError_t interp_f32_1d(Plan &p, void *c);
cudaError_t interp_f32_2d(Plan &p, void *c);
cudaError_t interp_f32_3d(Plan &p, void *c);
cudaError_t interp_f64_1d(Plan &p, void *c);
cudaError_t interp_f64_2d(Plan &p, void *c);
cudaError_t interp_f64_3d(Plan &p, void *c);

// One grouped launch over several plans of equal type, dimension, precision,
// width and method (batched execution): per-plan kernel arguments in device
// memory, workoff[p] = first global work item of plan p (workoff[nplans] = total).
struct MultiLaunch {
    const void *args;          // device array of KArgs<T>, one per plan
    const int64_t *workoff;    // device [nplans + 1]
    int nplans;
    int w, method, threads, num_sms;
    size_t smem;               // shared memory per CTA (max over the plans)
    size_t smem_optin;         // largest dynamic shared memory per CTA
    int variant;               // row sweep: 2D lanes (8/16/32), 3D m2 (1/2); 0 = none
    int m0max, m1max;          // largest bin width and height over the plans
    int tile;                  // largest padded bin (cells) over the plans
    cudaStream_t stream;
};
// Row-sweep form of an SM plan (the batch's grouping key).  Type 1: 2D sub-warp
// lanes 8, 16 or 32; 3D: bin depth m2 (1 or 2), plus 4 for the plane-split form
// (padded width <= 16).  Type 2: m2 + 4 for the 3D plane-split interpolation.
// 0 if the plan uses the shared-memory kernels.
int sweep_variant(const Plan &p);
// m2 + 4 if the plan's shape suits the 3D plane-split sweeps (single precision,
// SM, w <= 8, padded width <= 16, m2 in {1, 2}), else 0; setpts orders such a
// plan's records by start row and sweep_variant then reports the form.
int planes3_form(const Plan &p);
// 8, 16 or 32 (sub-warp lanes) if a 2D type 1 SM plan suits the spreading row
// sweep (padded width <= 32), else 0.
int sweep2_form(const Plan &p);
cudaError_t spread_multi_f32_1d(const MultiLaunch &ml);
cudaError_t spread_multi_f64_1d(const MultiLaunch &ml);
cudaError_t interp_multi_f32_1d(const MultiLaunch &ml);
cudaError_t interp_multi_f64_1d(const MultiLaunch &ml);
cudaError_t spread_multi_f32_2d(const MultiLaunch &ml);
cudaError_t spread_multi_f32_3d(const MultiLaunch &ml);
cudaError_t spread_multi_f64_2d(const MultiLaunch &ml);
cudaError_t spread_multi_f64_3d(const MultiLaunch &ml);
cudaError_t interp_multi_f32_2d(const MultiLaunch &ml);
cudaError_t interp_multi_f32_3d(const MultiLaunch &ml);
cudaError_t interp_multi_f64_2d(const MultiLaunch &ml);
cudaError_t interp_multi_f64_3d(const MultiLaunch &ml);
cudaError_t launch_deconvolve(Plan &p, void *f);
cudaError_t launch_precorrect(Plan &p, const void *f);
cudaError_t launch_zero(Plan &p, void *ptr, size_t bytes);
// Stores value in the device int *dst on the plan's stream.
cudaError_t launch_set_int(Plan &p, int32_t *dst, int32_t value);
cudaError_t launch_correction(Plan &p, const double *gl_t, const double *gl_w, int nq);

}  // namespace nufft

// The opaque handle of the C ABI.
struct nufft_plan_s {
    nufft::Plan p;
};
