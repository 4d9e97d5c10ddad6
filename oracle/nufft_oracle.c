/*
 * nufft_oracle.c -- plain, slow FP64 CPU reference for the 1D/2D/3D type 1,
 * type 2 (and exact type 3) NUFFT of Shih et al., "cuFINUFFT: a load-balanced GPU library for
 * general-purpose nonuniform FFTs" (arXiv 2102.08463).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, includes or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header or
 * constant generator with the CUDA path.
 *
 * Contents (each function cites the passage it follows):
 *   orc_es_kernel      ES kernel phi_beta (Sec. 3, Eq. "es").
 *   orc_direct_type1   exact type 1 sum (Eq. 2d1, extended to 3D as Sec. 1 says).
 *   orc_direct_type2   exact type 2 sum (Eq. 2d2).
 *   orc_direct_type3   exact type 3 sum (nonuniform to nonuniform; the third
 *                      type, which the paper lists as future work).
 *   orc_spread         type 1 step 1, spreading with the periodised kernel (Sec. 3.1).
 *   orc_interp         type 2 step 3, interpolation (Sec. 3.2).
 *   orc_cells          fixed-point bin rule for the bin-sort (Sec. 4.1, GM-sort).
 *   orc_binsort        stable counting sort giving the permutation t (Sec. 4.1).
 *
 * Conventions (readings of the paper where it leaves a choice open):
 *   - complex arrays are interleaved (re, im) doubles;
 *   - mode arrays are [N3][N2][N1] with k1 fastest and k_i running from
 *     -floor(N_i/2) upwards (Eq. "I");
 *   - fine grid point l sits at position -pi + l*h, h = 2 pi / n (the shift
 *     implied by the bin rule floor((x+pi)/h) of Sec. 4.1);
 *   - the kernel window of a point at fine-grid coordinate u = (x+pi)/h is the
 *     w cells l0 .. l0+w-1 with l0 = ceil(u - w/2), indices taken mod n.
 *   - iflag is the sign of the exponent of type 1; type 2 uses -iflag.
 *
 * Compile with -ffp-contract=off so that every floating-point operation is a
 * separately rounded IEEE operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846;

/* ES kernel, Sec. 3 Eq. (es): exp(beta*(sqrt(1-z^2)-1)) for |z| <= 1, else 0. */
double orc_es_kernel(double z, double beta)
{
    if (fabs(z) > 1.0) return 0.0;
    return exp(beta * (sqrt(1.0 - z * z) - 1.0));
}

/* ---------------------------------------------------------------------------
 * Accurate phase e^{i s theta} with theta = sum_i k_i * x_i.
 * Each product k_i*x_i is split exactly into p + e (p = fl(k x), e = fma(k,x,-p)),
 * the high parts are summed with an exact two-sum, and the tiny tail is applied
 * to first order: e^{i(a + t)} = e^{ia} (1 + i t) + O(t^2), |t| < 1e-12.
 * This keeps the phase error near 1e-16 even when |k x| is in the thousands.
 * ------------------------------------------------------------------------- */
static void two_sum(double a, double b, double *s, double *err)
{
    double ss = a + b;
    double bb = ss - a;
    *err = (a - (ss - bb)) + (b - bb);
    *s = ss;
}

static void phase_exp(int dim, const double *k, const double *x, double sgn,
                      double *re, double *im)
{
    double hi = 0.0, lo = 0.0;
    for (int i = 0; i < dim; ++i) {
        double p = k[i] * x[i];
        double e = fma(k[i], x[i], -p);
        double s, t;
        two_sum(hi, p, &s, &t);
        hi = s;
        lo += t + e;
    }
    double a = sgn * hi, tail = sgn * lo;
    double ca = cos(a), sa = sin(a);
    /* (ca + i sa)(1 + i tail) */
    *re = ca - sa * tail;
    *im = sa + ca * tail;
}

/* Neumaier (Kahan-Babuska) compensated accumulator. */
typedef struct { double s, c; } acc_t;
static void acc_add(acc_t *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double acc_val(const acc_t *a) { return a->s + a->c; }

static void mode_of_flat(int dim, const int64_t *N, int64_t flat, double *k)
{
    for (int i = 0; i < dim; ++i) {
        int64_t idx = flat % N[i];
        flat /= N[i];
        k[i] = (double)(idx - N[i] / 2);
    }
}

/*
 * Exact type 1 sum, Eq. (2d1) with the exponent sign iflag:
 *   f_k = sum_j c_j exp(i*iflag*(k . x_j)),  k in I_{N1} x I_{N2} (x I_{N3}).
 * nk modes are evaluated: the flat mode indices kflat[0..nk) (k1 fastest), or
 * all N1*N2*N3 modes in order if kflat is NULL.  f receives nk complex values.
 */
void orc_direct_type1(int dim, int64_t M, const double *x, const double *y,
                      const double *z, const double *c, int iflag,
                      const int64_t *N, int64_t nk, const int64_t *kflat,
                      double *f)
{
    const double *xs[3] = {x, y, z};
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nk; ++q) {
        double k[3] = {0, 0, 0};
        mode_of_flat(dim, N, kflat ? kflat[q] : q, k);
        acc_t ar = {0, 0}, ai = {0, 0};
        for (int64_t j = 0; j < M; ++j) {
            double xv[3];
            for (int i = 0; i < dim; ++i) xv[i] = xs[i][j];
            double er, ei;
            phase_exp(dim, k, xv, (double)iflag, &er, &ei);
            double cr = c[2 * j], ci = c[2 * j + 1];
            acc_add(&ar, cr * er - ci * ei);
            acc_add(&ai, cr * ei + ci * er);
        }
        f[2 * q] = acc_val(&ar);
        f[2 * q + 1] = acc_val(&ai);
    }
}

/*
 * Exact type 2 sum, Eq. (2d2) with exponent sign -iflag:
 *   c_j = sum_k f_k exp(-i*iflag*(k . x_j)).
 * Evaluated at the nt targets jlist[0..nt) (or all M in order if jlist is NULL).
 */
void orc_direct_type2(int dim, int64_t M, const double *x, const double *y,
                      const double *z, const double *f, int iflag,
                      const int64_t *N, int64_t nt, const int64_t *jlist,
                      double *c)
{
    const double *xs[3] = {x, y, z};
    int64_t Ntot = 1;
    for (int i = 0; i < dim; ++i) Ntot *= N[i];
    (void)M;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nt; ++q) {
        int64_t j = jlist ? jlist[q] : q;
        double xv[3];
        for (int i = 0; i < dim; ++i) xv[i] = xs[i][j];
        acc_t ar = {0, 0}, ai = {0, 0};
        for (int64_t m = 0; m < Ntot; ++m) {
            double k[3] = {0, 0, 0};
            mode_of_flat(dim, N, m, k);
            double er, ei;
            phase_exp(dim, k, xv, -(double)iflag, &er, &ei);
            double fr = f[2 * m], fi = f[2 * m + 1];
            acc_add(&ar, fr * er - fi * ei);
            acc_add(&ai, fr * ei + fi * er);
        }
        c[2 * q] = acc_val(&ar);
        c[2 * q + 1] = acc_val(&ai);
    }
}

/*
 * Exact type 3 sum with exponent sign iflag, at real frequencies (s_k, t_k, u_k):
 *   f_k = sum_j c_j exp(i*iflag*(s_k x_j + t_k y_j + u_k z_j)),  k < nk.
 * The same compensated phase and sum as type 1, with non-integer frequencies.
 */
void orc_direct_type3(int dim, int64_t M, const double *x, const double *y,
                      const double *z, const double *c, int iflag, int64_t nk,
                      const double *s, const double *t, const double *u, double *f)
{
    const double *xs[3] = {x, y, z};
    const double *ks[3] = {s, t, u};
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nk; ++q) {
        double k[3] = {0, 0, 0};
        for (int i = 0; i < dim; ++i) k[i] = ks[i][q];
        acc_t ar = {0, 0}, ai = {0, 0};
        for (int64_t j = 0; j < M; ++j) {
            double xv[3];
            for (int i = 0; i < dim; ++i) xv[i] = xs[i][j];
            double er, ei;
            phase_exp(dim, k, xv, (double)iflag, &er, &ei);
            double cr = c[2 * j], ci = c[2 * j + 1];
            acc_add(&ar, cr * er - ci * ei);
            acc_add(&ai, cr * ei + ci * er);
        }
        f[2 * q] = acc_val(&ar);
        f[2 * q + 1] = acc_val(&ai);
    }
}

/* ---------------------------------------------------------------------------
 * Spreading and interpolation, Sec. 3.1 step 1 and Sec. 3.2 step 3.
 * psi(x) = prod_i phi_beta(x_i / alpha_i), alpha_i = w pi / n_i, periodised.
 * In fine-grid units u_i = (x_i + pi)/h_i the kernel argument of cell l is
 * (l - u_i) * 2 / w, so only the w cells l0..l0+w-1, l0 = ceil(u - w/2), see it.
 * ------------------------------------------------------------------------- */
static void window_1d(double xv, int64_t n, int w, double beta,
                      int64_t *l0, double *wt)
{
    double h = 2.0 * ORC_PI / (double)n;
    double u = (xv + ORC_PI) / h;
    double s = ceil(u - 0.5 * (double)w);
    *l0 = (int64_t)s;
    for (int i = 0; i < w; ++i)
        wt[i] = orc_es_kernel((s + (double)i - u) * 2.0 / (double)w, beta);
}

static int64_t wrap(int64_t l, int64_t n)
{
    int64_t r = l % n;
    return r < 0 ? r + n : r;
}

/*
 * Type 1 step 1:  b_l = sum_j c_j psi_per(l h - pi - x_j), Sec. 3.1.
 * b is the fine grid [n3][n2][n1] complex, overwritten.  The slowest grid axis
 * is split into one slab per OpenMP thread; every thread walks all points and
 * adds only the rows of its own slab, so no two threads write the same cell.
 */
void orc_spread(int dim, int64_t M, const double *x, const double *y,
                const double *z, const double *c, const int64_t *n, int w,
                double beta, double *b)
{
    const double *xs[3] = {x, y, z};
    int64_t nn[3] = {n[0], dim >= 2 ? n[1] : 1, dim == 3 ? n[2] : 1};
    int64_t ntot = nn[0] * nn[1] * nn[2];
    memset(b, 0, sizeof(double) * 2 * (size_t)ntot);
    int slow = dim - 1;
    int64_t nslow = nn[slow];
    #pragma omp parallel
    {
        int nth = 1, tid = 0;
#ifdef _OPENMP
        nth = omp_get_num_threads();
        tid = omp_get_thread_num();
#endif
        int64_t r0 = nslow * tid / nth, r1 = nslow * (tid + 1) / nth;
        double *wt = (double *)malloc(sizeof(double) * 3 * (size_t)w);
        for (int64_t j = 0; j < M; ++j) {
            int64_t l0[3] = {0, 0, 0};
            double *wx = wt, *wy = wt + w, *wz = wt + 2 * w;
            window_1d(xs[slow][j], nn[slow], w, beta, &l0[slow], wt + slow * w);
            int any = 0;
            for (int i = 0; i < w; ++i) {
                int64_t r = wrap(l0[slow] + i, nslow);
                if (r >= r0 && r < r1) { any = 1; break; }
            }
            if (!any) continue;
            for (int d = 0; d < slow; ++d)
                window_1d(xs[d][j], nn[d], w, beta, &l0[d], wt + d * w);
            double cr = c[2 * j], ci = c[2 * j + 1];
            int wzn = dim == 3 ? w : 1, wyn = dim >= 2 ? w : 1;
            for (int iz = 0; iz < wzn; ++iz) {
                int64_t lz = dim == 3 ? wrap(l0[2] + iz, nn[2]) : 0;
                double vz = dim == 3 ? wz[iz] : 1.0;
                if (dim == 3 && !(lz >= r0 && lz < r1)) continue;
                for (int iy = 0; iy < wyn; ++iy) {
                    int64_t ly = dim >= 2 ? wrap(l0[1] + iy, nn[1]) : 0;
                    if (dim == 2 && !(ly >= r0 && ly < r1)) continue;
                    double vyz = dim >= 2 ? vz * wy[iy] : vz;
                    for (int ix = 0; ix < w; ++ix) {
                        int64_t lx = wrap(l0[0] + ix, nn[0]);
                        if (dim == 1 && !(lx >= r0 && lx < r1)) continue;
                        double v = vyz * wx[ix];
                        int64_t cell = lx + nn[0] * (ly + nn[1] * lz);
                        b[2 * cell] += v * cr;
                        b[2 * cell + 1] += v * ci;
                    }
                }
            }
        }
        free(wt);
    }
}

/*
 * Type 2 step 3:  c_j = sum_l b_l psi_per(l h - pi - x_j), Sec. 3.2.
 * b is the fine grid [n3][n2][n1] complex; c receives M complex values.
 */
void orc_interp(int dim, int64_t M, const double *x, const double *y,
                const double *z, const double *b, const int64_t *n, int w,
                double beta, double *c)
{
    const double *xs[3] = {x, y, z};
    int64_t nn[3] = {n[0], dim >= 2 ? n[1] : 1, dim == 3 ? n[2] : 1};
    #pragma omp parallel
    {
        double *wt = (double *)malloc(sizeof(double) * 3 * (size_t)w);
        #pragma omp for schedule(static)
        for (int64_t j = 0; j < M; ++j) {
            int64_t l0[3] = {0, 0, 0};
            for (int d = 0; d < dim; ++d)
                window_1d(xs[d][j], nn[d], w, beta, &l0[d], wt + d * w);
            double sr = 0.0, si = 0.0;
            int wzn = dim == 3 ? w : 1, wyn = dim >= 2 ? w : 1;
            for (int iz = 0; iz < wzn; ++iz) {
                int64_t lz = dim == 3 ? wrap(l0[2] + iz, nn[2]) : 0;
                double vz = dim == 3 ? wt[2 * w + iz] : 1.0;
                for (int iy = 0; iy < wyn; ++iy) {
                    int64_t ly = dim >= 2 ? wrap(l0[1] + iy, nn[1]) : 0;
                    double vyz = dim >= 2 ? vz * wt[w + iy] : vz;
                    for (int ix = 0; ix < w; ++ix) {
                        int64_t lx = wrap(l0[0] + ix, nn[0]);
                        double v = vyz * wt[ix];
                        int64_t cell = lx + nn[0] * (ly + nn[1] * lz);
                        sr += v * b[2 * cell];
                        si += v * b[2 * cell + 1];
                    }
                }
            }
            c[2 * j] = sr;
            c[2 * j + 1] = si;
        }
        free(wt);
    }
}

/* ---------------------------------------------------------------------------
 * Bin-sort, Sec. 4.1 (GM-sort): point j is "inside" the bin that holds its
 * fine-grid cell l_i = floor((x_i + pi)/h_i); bins are m1 x m2 (x m3) blocks of
 * cells, x fastest, the last bin on an axis possibly smaller.  The permutation t
 * lists the points bin by bin.
 *
 * The paper does not say in which arithmetic floor((x+pi)/h) is taken.  Reading
 * (exact, integer): the position is carried as a 64-bit fraction of the period,
 *   X   = round-half-even(clamp(x, -1024, 1024) * 2^52)        (int64)
 *   Q   = floor(|X| * K / 2^64) mod 2^64,  K = round(2^76 / (2 pi))
 *   Phi = 2^63 + sign(X) Q  mod 2^64       (Phi / 2^64 = (x+pi)/(2 pi) mod 1)
 *   l   = floor(Phi * n / 2^64),  F = Phi * n mod 2^64.
 * K = 651 * 2^64 + 0xe60db9391054a7f1.  This takes x anywhere in [-1024, 1024]
 * into its periodic image and is reproducible bit for bit on any machine.
 * ------------------------------------------------------------------------- */
static const uint64_t ORC_K_HI = 651ULL;
static const uint64_t ORC_K_LO = 0xe60db9391054a7f1ULL;

static uint64_t mulhi_u64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

static uint64_t period_fraction(double xv)
{
    double xc = xv;
    if (!(xc >= -1024.0)) xc = -1024.0;       /* also catches NaN */
    if (xc > 1024.0) xc = 1024.0;
    int64_t X = (int64_t)nearbyint(xc * 4503599627370496.0);   /* 2^52, exact */
    uint64_t A = X < 0 ? (uint64_t)(-X) : (uint64_t)X;
    uint64_t Q = A * ORC_K_HI + mulhi_u64(A, ORC_K_LO);
    return (1ULL << 63) + (X < 0 ? (0ULL - Q) : Q);
}

/*
 * Cell index l and cell fraction F (as F / 2^64) of each point along one axis.
 * cell[j] in [0, n), frac[j] in [0, 1).
 */
void orc_cells(int64_t M, const double *x, int64_t n, int64_t *cell, double *frac)
{
    for (int64_t j = 0; j < M; ++j) {
        uint64_t phi = period_fraction(x[j]);
        cell[j] = (int64_t)mulhi_u64(phi, (uint64_t)n);
        uint64_t F = phi * (uint64_t)n;
        frac[j] = (double)(F >> 11) * 0x1p-53;
    }
}

/*
 * Stable bin-sort, Sec. 4.1: bin index per point (x fastest), per-bin counts,
 * and the permutation t listing points bin by bin, in increasing original index
 * within a bin.  n, m: fine-grid and bin sizes per axis (dim entries).
 * Outputs: binidx[M], counts[nbins], t[M].  Returns nbins.
 */
int64_t orc_binsort(int dim, int64_t M, const double *x, const double *y,
                    const double *z, const int64_t *n, const int64_t *m,
                    int64_t *binidx, int64_t *counts, int64_t *t)
{
    const double *xs[3] = {x, y, z};
    int64_t nb[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) nb[d] = (n[d] + m[d] - 1) / m[d];
    int64_t nbins = nb[0] * nb[1] * nb[2];
    for (int64_t j = 0; j < M; ++j) {
        int64_t bi[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            uint64_t phi = period_fraction(xs[d][j]);
            int64_t l = (int64_t)mulhi_u64(phi, (uint64_t)n[d]);
            bi[d] = l / m[d];
        }
        binidx[j] = bi[0] + nb[0] * (bi[1] + nb[1] * bi[2]);
    }
    memset(counts, 0, sizeof(int64_t) * (size_t)nbins);
    for (int64_t j = 0; j < M; ++j) counts[binidx[j]]++;
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nbins > 0 ? nbins : 1));
    int64_t run = 0;
    for (int64_t b = 0; b < nbins; ++b) { next[b] = run; run += counts[b]; }
    for (int64_t j = 0; j < M; ++j) t[next[binidx[j]]++] = j;   /* index order: stable */
    free(next);
    return nbins;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int nth)
{
#ifdef _OPENMP
    if (nth > 0) omp_set_num_threads(nth);
#else
    (void)nth;
#endif
}
