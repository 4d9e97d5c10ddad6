/*
 * nufft_gb300.h -- C ABI of the GB300 (sm_103a) nonuniform FFT library.
 *
 * Computes the 2D and 3D type 1 and type 2 NUFFT of Shih et al., "cuFINUFFT:
 * a load-balanced GPU library for general-purpose nonuniform FFTs"
 * (arXiv 2102.08463), with the paper's "plan, setup, execute, destroy"
 * interface (Sec. 1.1).
 *
 *   type 1 (Eq. 2d1):  f_k = sum_{j<M} c_j exp( i*iflag*(k . x_j) ),   k in I_N1 x I_N2 (x I_N3)
 *   type 2 (Eq. 2d2):  c_j = sum_k    f_k exp(-i*iflag*(k . x_j) ),   j < M
 *
 * with I_N = { -floor(N/2), ..., ceil(N/2)-1 } (Eq. I).  The paper writes type 1
 * with exponent -i and type 2 with +i; that is iflag = -1 here.  The result is
 * approximated to a relative l2 tolerance near eps by the three-step algorithm
 * of Sec. 3 (spread / FFT / correct, and its transpose).
 *
 * Memory layout and ownership
 *   - All array arguments are DEVICE pointers on the current CUDA device, in
 *     the plan's precision (prec 0: float / interleaved complex float,
 *     prec 1: double / interleaved complex double).
 *   - Nonuniform points: three separate arrays x, y, z of M reals (z is NULL
 *     in 2D).  Coordinates are periodic with period 2 pi; accuracy is as stated
 *     for x in [-3 pi, 3 pi); values beyond +-1024 are clamped.
 *   - Strengths / targets c: ntransf vectors of M complex values, c[t*M + j].
 *   - Modes f: ntransf arrays of N1*N2(*N3) complex values, f[t][k3][k2][k1],
 *     k1 fastest, each axis ordered from -floor(N_i/2) upwards.
 *   - The plan owns every buffer it allocates (fine grid, sort arrays, cuFFT
 *     plan).  setpts copies what it needs: the caller may free x, y, z after
 *     setpts returns and the stream has passed it.
 *   - Calls are asynchronous on opts.stream; they enqueue work and return.
 *
 * Errors: every function returns 0 on success or a negative NUFFT_ERR_* code;
 * none aborts, traps or prints.  After any error the plan can still be passed
 * to nufft_destroy.
 */
#ifndef NUFFT_GB300_H
#define NUFFT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define NUFFT_OK               0
#define NUFFT_ERR_ARG         -1   /* invalid argument (type, dim, sizes, null pointer, option) */
#define NUFFT_ERR_EPS         -2   /* tolerance outside the supported range for the precision */
#define NUFFT_ERR_SIZE        -3   /* mode count or fine grid too large */
#define NUFFT_ERR_ALLOC       -4   /* device allocation failed */
#define NUFFT_ERR_CUDA        -5   /* CUDA runtime error while enqueueing work */
#define NUFFT_ERR_CUFFT       -6   /* cuFFT plan or execution error */
#define NUFFT_ERR_NOPTS       -7   /* execute before setpts */
#define NUFFT_ERR_CHECK       -8   /* a device-side check of opts.debug_checks failed */
#define NUFFT_ERR_METHOD      -9   /* requested method not available for this plan */

/* Spreading / interpolation methods (Sec. 4.1, 4.2). */
#define NUFFT_METHOD_AUTO      0   /* the library's heuristic */
#define NUFFT_METHOD_GM        1   /* one thread group per point, user order, global atomics */
#define NUFFT_METHOD_GM_SORT   2   /* the same in bin-sorted order */
#define NUFFT_METHOD_SM        3   /* type 1: shared-memory subproblems (Sec. 4.1 SM);
                                      type 2: padded bin staged in shared memory, sorted gather */

typedef struct nufft_plan_s *nufft_plan;   /* opaque, library-owned */

typedef struct {
    int    method;        /* NUFFT_METHOD_*; 0 = auto */
    int    bin[3];        /* bin size m_i in fine-grid cells; 0 = default: 16x16x2 in 3D
                             ((16 - w) x 16 x 2 for single-precision type 1 at w <= 4),
                             16x16 in 2D type 2; 2D type 1: (16 - w) x 16 single precision
                             ((8 - w) x 32 for w <= 3), (16 - w) x 32 double */
    int    msub;          /* max points per subproblem M_sub; 0 = default 1024 (Sec. 4.1 remark) */
    double upsampfac;     /* sigma; 0 or 2.0 = the paper's 2; 1.25 = the lower-memory variant */
    void  *stream;        /* cudaStream_t to enqueue on; NULL = legacy default stream */
    int    threads;       /* threads per block for spread / interp; 0 = default 256 */
    int    ctas_per_sm;   /* persistent CTAs per SM for the subproblem kernels; 0 = auto */
    int    use_picker;    /* 1 = with method, bin, msub and threads all automatic, let the
                             installed tile picker (nufft_picker_install) choose them at
                             setpts, after the autotuner's cache; 0 = off */
    int    unordered_bins; /* 0 = t lists the points of every bin in increasing original
                             index (unique t; the default); 1 = in the order the sort's
                             shared-memory atomics claim slots (faster setpts, t may differ
                             between calls; bins, counts and subproblems unchanged).  Plans
                             whose bins exceed shared memory sort stably either way. */
    int    debug_checks;  /* 1 = setpts also checks on the device that every coordinate is
                             finite and inside [-3 pi, 3 pi] and that t is a permutation,
                             and records a failure in a device status word instead of
                             trapping; nufft_get_status reads it.  0 = off (the default). */
} nufft_opts;

/* Fill opts with the defaults listed above. */
void nufft_default_opts(nufft_opts *opts);

/*
 * Create a plan (Sec. 1.1 "plan"; parameters of Sec. 3).
 *   type    1 or 2; 3 for nonuniform-to-nonuniform (see nufft_setpts3).
 *   dim     1, 2 or 3 (1D is the d = 1 case of Sec. 3, which the paper lists as
 *           future work: bins of m1 cells, the same three methods).
 *   nmodes  dim entries N1 (, N2 (, N3)), each >= 1 (ignored, may be NULL, for type 3).
 *   iflag   +1 or -1: sign of the type 1 exponent (type 2 uses the opposite).
 *   ntransf number of strength / coefficient vectors per execute (>= 1).
 *   eps     requested relative tolerance; kernel width w = ceil(log10(1/eps)) + 1
 *           (clamped to [2, 16]), beta = 2.30 w, fine grid n_i = smallest
 *           2^a 3^b 5^c >= max(sigma N_i, 2w).
 *   prec    0 = single, 1 = double, -1 = by tolerance (single if eps >= 1e-6;
 *           with upsampfac 1.25, single if eps >= 1e-4).  Single precision
 *           requires those tolerances (NUFFT_ERR_EPS otherwise).
 *   opts    NULL for defaults.
 *   out     receives the plan handle (NULL on failure).
 * Allocates the fine grid (ntransf * n1*n2(*n3) complex), the correction factors
 * and the cuFFT plan on the current device.
 */
int nufft_makeplan(int type, int dim, const int64_t *nmodes, int iflag, int ntransf,
                   double eps, int prec, const nufft_opts *opts, nufft_plan *out);

/*
 * Set the nonuniform points (Sec. 1.1 "setup"; bin-sort of Sec. 4.1).
 * Computes each point's fine-grid cell, bins of m1 (x m2 (x m3)) cells with x
 * fastest, the permutation t listing points bin by bin (increasing original
 * index inside a bin, unless the plan was made with opts.unordered_bins), the
 * subproblem list (runs of at most M_sub points of one bin) and packed
 * per-point kernel offsets.
 * M = 0 is allowed.  x, y, z: device arrays of M reals (z NULL in 2D; y and z
 * NULL in 1D).
 */
int nufft_setpts(nufft_plan plan, int64_t M, const void *x, const void *y, const void *z);

/*
 * Type 3 points and frequencies (the nonuniform-to-nonuniform transform the
 * paper lists as future work):
 *   f_k = sum_j c_j exp(i iflag s_k . x_j),  j < M, k < K,
 * x_j = (x, y, z)_j and s_k = (s, t, u)_k real and of any range (device arrays
 * of the plan precision; y / t NULL in 1D, z / u NULL in 1D and 2D).  The call
 * reads the extents of both sets (X_i and S_i, the half-widths about their
 * centres; it synchronizes the plan's stream for that), sizes a spreading grid
 * of n_i = smallest even 2^a 3^b 5^c >= max(4 S_i X_i / pi + w + 2, 2w) cells,
 * and sets up two inner plans of this library: the type 1 spreading step on
 * that grid for the rescaled points, and a type 2 transform of the grid at the
 * rescaled frequencies.  Only for plans made with type 3; upsampfac 2.
 * Errors: NUFFT_ERR_ARG (wrong plan type, null arrays, non-finite coordinates),
 * NUFFT_ERR_SIZE (S_i X_i too large), NUFFT_ERR_ALLOC.
 */
int nufft_setpts3(nufft_plan plan, int64_t M, const void *x, const void *y, const void *z,
                  int64_t K, const void *s, const void *t, const void *u);

/*
 * Execute (Sec. 1.1 "execute"; Sec. 3.1 for type 1, Sec. 3.2 for type 2).
 *   type 1: reads c (ntransf*M complex), overwrites f (ntransf*N complex).
 *   type 2: reads f, overwrites c.
 *   type 3: reads c (ntransf*M complex), overwrites f (ntransf*K complex).
 * The stage entry points below, nufft_execute_host, nufft_get_finegrid,
 * nufft_get_sort and batches take type 1 and type 2 plans only.
 */
int nufft_execute(nufft_plan plan, void *c, void *f);

/*
 * Set points and execute from HOST memory ("total+mem" of Sec. 5: the timing
 * that includes the host-device transfers).  x, y, z (M reals each), c
 * (ntransf*M complex) and f (ntransf*N complex) are host arrays with the same
 * layouts and roles as in nufft_setpts / nufft_execute: type 1 reads c and
 * writes f, type 2 reads f and writes c.  On the plan's stream the points are
 * copied in and sorted while the input array is copied on an internal stream;
 * the execute waits for that copy, then the output is copied back.  The call is
 * asynchronous: the output is valid, and the host arrays may be reused, once the
 * plan's stream has passed the call.  Page-locked (pinned) host arrays let the
 * copies overlap the kernels; pageable arrays work but their copies are staged
 * synchronously by the CUDA runtime.  Device staging for the points, c and f is
 * allocated on first use (and when M grows) and held by the plan.
 * Errors as nufft_setpts / nufft_execute (NUFFT_ERR_ALLOC for the staging).
 */
int nufft_execute_host(nufft_plan plan, int64_t M, const void *x, const void *y, const void *z,
                       void *c, void *f);

/* Free everything the plan owns (Sec. 1.1 "destroy").  NULL is accepted. */
int nufft_destroy(nufft_plan plan);

/* Static message for an error code. */
const char *nufft_strerror(int code);

/* ---- stage entry points (the same kernels execute runs, one step at a time) ---- */

/* Type 1 step 1 (Sec. 3.1): zero the fine grid and spread c into it. */
int nufft_spread(nufft_plan plan, const void *c);
/* The spreading kernel alone: adds the spread of c into the fine grid as it is. */
int nufft_spread_add(nufft_plan plan, const void *c);
/* Type 2 step 3 (Sec. 3.2): interpolate the fine grid at the points into c. */
int nufft_interp(nufft_plan plan, void *c);
/* Step 2 of either type: in-place cuFFT of the fine grid, direction from type and iflag. */
int nufft_fft(nufft_plan plan);
/* Type 1 step 3: truncate the transformed fine grid to the N modes and scale by p_k into f. */
int nufft_deconvolve(nufft_plan plan, void *f);
/* Type 2 step 1: scale f by p_k and zero-pad into the fine grid. */
int nufft_precorrect(nufft_plan plan, const void *f);

/* ---- introspection, for tests and benchmarks ---- */

/* Kernel width, beta, fine grid sizes (3 entries, 1 for unused axes), bin sizes
   (3 entries), number of bins, precision (0/1) and method actually used. */
int nufft_get_params(nufft_plan plan, int *w, double *beta, int64_t *nf, int *bins,
                     int64_t *nbins, int *prec, int *method);
/* Device pointer and byte size of the fine grid (ntransf * n complex). */
int nufft_get_finegrid(nufft_plan plan, void **dptr, size_t *bytes);
/* Copy (device to device, on the plan stream) the permutation t (int32[M]),
   the per-bin counts (int32[nbins]) and the subproblem count (int32[1]);
   any destination may be NULL. */
int nufft_get_sort(nufft_plan plan, int32_t *t, int32_t *bincounts, int32_t *nsub);
/* The plan's current tiles: fills method, bin[3] (1 on unused axes), msub and
   threads of *out and leaves the other fields alone. */
int nufft_get_tiles(nufft_plan plan, nufft_opts *out);

/* Result of the device-side checks of a plan made with opts.debug_checks = 1:
   waits for the plan's stream, then returns NUFFT_OK if every setpts since the
   plan was made (or since the last call) passed, NUFFT_ERR_CHECK if one did not
   (a coordinate NaN, infinite or outside [-3 pi, 3 pi], or t not a permutation),
   and clears the status.  Plans without debug_checks return NUFFT_OK. */
int nufft_get_status(nufft_plan plan);

/* ---- fault injection, for tests of the error paths (host side only) ----
 * nufft_debug_fail(kind, after) arms a process-wide failure: the (after + 1)-th
 * next device allocation made by this library (kind NUFFT_FAIL_ALLOC) or cuFFT
 * plan creation (NUFFT_FAIL_CUFFT) fails as an out-of-memory or cuFFT error would,
 * without touching the device; after < 0 disarms.  Returns the number of
 * allocations (or cuFFT plans) made since the last call, so a test can count the
 * failure points of an entry point.  Not part of the transform. */
#define NUFFT_FAIL_ALLOC 1
#define NUFFT_FAIL_CUFFT 2
int nufft_debug_fail(int kind, int after);

/* Number of CUDA kernels this library has launched in this process (all plans,
   all threads).  cuFFT's own kernels are not counted. */
uint64_t nufft_get_launch_count(void);

/* Measured FMA throughput of the current device in TFLOP/s (an FMA counts as two
   operations): a kernel of independent FMA chains over all SMs, timed with CUDA
   events on stream (NULL = legacy default stream); prec 0 = float, 1 = double.
   The benchmark's roofline denominator for arithmetic-bound kernels; not part of
   the transform (the paper has no counterpart).  Synchronizes stream.
   Errors: NUFFT_ERR_ARG, NUFFT_ERR_CUDA. */
int nufft_fma_peak(int prec, double *tflops, void *stream);

/* ---- autotuner ----
 * The paper hand-tunes its tiles for its own GPU (Sec. 4.1 remark).  This times
 * candidate tiles -- method (SM, GM-sort, GM), bin sizes, M_sub and threads per
 * CTA -- for one problem on the caller's data and returns the fastest execute.
 *   type ... prec, base   as nufft_makeplan (base may be NULL; its stream is used);
 *                         dim 2 or 3 (1D plans keep their default tiles).
 *   M, x, y, z            points (device), M >= 1.
 *   c, f                  device arrays of the plan's shapes; overwritten.
 *   reps                  timed executes per candidate (median taken), >= 1.
 *   best                  receives base with the winning method / bin / msub / threads.
 *   best_ms               receives the winner's execute time (may be NULL).
 *   trials, max_trials    optional per-candidate records; ntrials receives their count.
 * The winner is also stored in a process-wide cache under the problem class
 * (type, dim, precision, w, sigma, log2 fine-grid size, half-octave of M / n_tot);
 * plans made with all tile options left automatic adopt cached tiles at setpts.
 * Blocks the host until the timing is done. */
typedef struct {
    int    method;
    int    bin[3];
    int    msub;
    int    threads;
    double exec_ms;      /* median execute time */
    double setpts_ms;    /* one setpts */
} nufft_tune_trial;
int nufft_autotune(int type, int dim, const int64_t *nmodes, int iflag, int ntransf, double eps,
                   int prec, const nufft_opts *base, int64_t M, const void *x, const void *y,
                   const void *z, void *c, void *f, int reps, nufft_opts *best, double *best_ms,
                   nufft_tune_trial *trials, int max_trials, int *ntrials);
/* Save / load the tuning cache as text (one class per line); clear it. */
int nufft_tune_cache_save(const char *path);
int nufft_tune_cache_load(const char *path);
int nufft_tune_cache_clear(void);

/* ---- batched execution of many plans ----
 * Not in the paper (its interface runs one plan at a time); for workloads of
 * many independent transforms of uneven N and M.  Plans that share type,
 * dimension, precision, kernel width and method are grouped, and each group's
 * spreading / interpolation runs as one persistent launch over the subproblems
 * (GM: chunks of points) of all its plans; clears, corrections and cuFFT stay
 * per plan.
 *
 * nufft_batch_create: plans[0..nplans) must be distinct type 1 / 2 plans, set up (setpts)
 *   before each execute; while the batch exists they run on `stream` (their cuFFT
 *   plans are re-bound to it) and must not be used on their own.  Destroying the
 *   batch hands them back their own streams.
 * nufft_batch_execute: c[k], f[k] are the plan-k arrays of nufft_execute.  Calls
 *   may follow one another without a host synchronization; each call's arguments
 *   are staged in host buffers of their own until its copies have run.
 * nufft_batch_capture: records the execute of these c / f arrays into a CUDA
 *   graph (stream must not be NULL); nufft_batch_launch replays it.  Re-running
 *   setpts on a member with the same M keeps the graph valid; a larger M or a new
 *   subproblem capacity reallocates and needs a new capture.  The graph keeps the
 *   arguments of its capture: later nufft_batch_execute calls with other arrays
 *   do not change what it replays.  Capturing waits for the stream to drain.
 * Errors as nufft_execute; NUFFT_ERR_NOPTS from launch when nothing was captured. */
typedef struct nufft_batch_s *nufft_batch;
int nufft_batch_create(const nufft_plan *plans, int nplans, void *stream, nufft_batch *out);
int nufft_batch_execute(nufft_batch batch, void *const *c, void *const *f);
int nufft_batch_capture(nufft_batch batch, void *const *c, void *const *f);
int nufft_batch_launch(nufft_batch batch);
int nufft_batch_destroy(nufft_batch batch);

/* ---- allocation-free bin-sort ----
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory (code running inside another allocator's callbacks,
 * real-time or embedded callers with a memory budget fixed at start-up, host
 * paths that must not take the driver's allocation locks).  It computes the
 * bin-sort of nufft_setpts with default options -- the permutation t listing
 * the points bin by bin (increasing original index inside a bin) and the
 * number of points per bin -- without calling cudaMalloc, cudaFree or any
 * allocating library routine.
 *
 *   dim, prec   2 or 3; 0 = float coordinates, 1 = double.
 *   M           number of points, 0 <= M <= 1048576 (else NUFFT_ERR_SIZE).
 *   x, y, z     device arrays of M coordinates (z NULL in 2D).
 *   nf          dim fine-grid sizes n_i (as nufft_get_params reports them).
 *   bins        dim bin sizes m_i, 1 <= m_i <= n_i; at most 16384 bins in all
 *               (else NUFFT_ERR_SIZE).
 *   perm        device int32[M], receives t.
 *   bincount    device int32[number of bins], receives the counts (x fastest).
 *   stream      cudaStream_t (NULL = legacy default stream); asynchronous.
 * Scratch: one fixed device array of about 8.1 MB inside the library, resident
 * on every device that loads it until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and raises
 * the kernels' shared-memory limits; with CUDA's lazy module loading (the
 * default) that first call, or the library's first kernel use on the device, is
 * also when the driver loads the module and places the array, which may
 * allocate device memory.  Callers that must not allocate later should make one
 * call per device at start-up (M = 0 is enough) and before any stream capture;
 * later calls allocate nothing.  Every call overwrites all scratch it uses, but
 * all calls on a device share the one array: calls whose GPU work could overlap
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Errors: NUFFT_ERR_ARG, NUFFT_ERR_SIZE, NUFFT_ERR_CUDA; nothing is
 * written on an argument error. */
int nufft_binsort_noalloc(int dim, int prec, int64_t M, const void *x, const void *y,
                          const void *z, const int64_t *nf, const int *bins, int32_t *perm,
                          int32_t *bincount, void *stream);

/* ---- learned tile picker ----
 * Not in the paper, which fixes the method and tiles by hand-tuned rules (Sec.
 * 4.1 remark; method advice of Sec. 5.4).  A perceptron 12 -> 64 -> 64 -> 1 with
 * ReLU predicts log2 of the execute time (ms) of a plan under one candidate
 * tiling from NUFFT_PICKER_NFEAT features (nufft_picker_features); a plan made
 * with opts.use_picker = 1 evaluates it over the autotuner's candidate list at
 * setpts and takes the argmin (first in list order on ties) among the tilings
 * the plan can run.  With no picker installed such plans keep the heuristic
 * tiles.  Forward, backward, loss and Adam run in the library's kernels in
 * single precision on the device the picker was created on.
 *
 * Parameters: NUFFT_PICKER_NPARAM floats, in the order W1[64][12] (row = unit),
 * b1[64], W2[64][64], b2[64], w3[64], b3.  Training data: X[n][12] features
 * (row-major) and T[n] targets = log2(exec ms), device arrays.
 *
 * nufft_picker_create   He-uniform weights from SplitMix64(seed), zero biases.
 * nufft_picker_set_params / get_params   host arrays of NPARAM floats; setting
 *                       also zeroes the Adam moments and step count.
 * nufft_picker_save / load   the parameters as text (one value per line).
 * nufft_picker_predict  y[B] = network(X[B][12]); asynchronous on stream.
 * nufft_picker_grad     grad[NPARAM] = dL/dtheta and loss[0] = L for the mean
 *                       squared error L over the B samples; device outputs.
 * nufft_picker_step     one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, rate lr)
 *                       on the B samples; loss[0] (device, may be NULL) = L before.
 * nufft_picker_train    epochs of Adam over shuffled minibatches of `batch`
 *                       samples (order from SplitMix64(seed)); *final_loss (host)
 *                       = L over all n afterwards.  Synchronizes stream.
 * nufft_picker_loss     L over n samples into loss[0] (device).
 * nufft_picker_install  make `picker` the process-wide picker (NULL = none); the
 *                       caller keeps it alive until it is uninstalled or
 *                       destroyed (destroy uninstalls it).
 * nufft_picker_features the 12 features of a problem and candidate tiling:
 *     [0] type == 2  [1] dim == 3  [2] double precision  [3] w / 16
 *     [4] log2(n_tot) / 32  [5] log2(M / n_tot) / 8  [6] skew / 16
 *     [7] method == SM  [8] method == GM  [9] log2(bin cells) / 12
 *     [10] log2(M_sub) / 12  [11] threads / 256
 *   prec -1 resolves as in makeplan; tiles->bin / msub / threads 0 mean the
 *   defaults; tiles->method must not be AUTO.
 * nufft_point_skew      skew = log2(max count * 4096 / M) of the points in a fixed
 *                       grid of 4096 equal boxes (64 x 64 in 2D, 16^3 in 3D) over
 *                       the period, at least 0 (0 for M = 0); synchronizes stream.
 * Errors: NUFFT_ERR_ARG, NUFFT_ERR_ALLOC, NUFFT_ERR_CUDA, NUFFT_ERR_EPS. */
#define NUFFT_PICKER_NFEAT  12
#define NUFFT_PICKER_HIDDEN 64
#define NUFFT_PICKER_NPARAM 5057
typedef struct nufft_picker_s *nufft_picker;
int nufft_picker_create(uint64_t seed, nufft_picker *out);
int nufft_picker_destroy(nufft_picker picker);
int nufft_picker_set_params(nufft_picker picker, const float *params);
int nufft_picker_get_params(nufft_picker picker, float *params);
int nufft_picker_save(nufft_picker picker, const char *path);
int nufft_picker_load(nufft_picker picker, const char *path);
int nufft_picker_predict(nufft_picker picker, int64_t B, const float *X, float *y, void *stream);
int nufft_picker_grad(nufft_picker picker, int64_t B, const float *X, const float *T, float *grad,
                      float *loss, void *stream);
int nufft_picker_step(nufft_picker picker, int64_t B, const float *X, const float *T, float lr,
                      float *loss, void *stream);
int nufft_picker_train(nufft_picker picker, int64_t n, const float *X, const float *T, int epochs,
                       int batch, float lr, uint64_t seed, float *final_loss, void *stream);
int nufft_picker_loss(nufft_picker picker, int64_t n, const float *X, const float *T, float *loss,
                      void *stream);
int nufft_picker_install(nufft_picker picker);
int nufft_picker_features(int type, int dim, const int64_t *nmodes, double eps, int prec,
                          double upsampfac, int64_t M, double skew, const nufft_opts *tiles,
                          float *out);
int nufft_point_skew(int dim, int prec, int64_t M, const void *x, const void *y, const void *z,
                     double *skew, void *stream);

/* nufft_pick: the upsampling factor sigma and the tiles for a plan that is yet
 * to be made, chosen by the installed picker from the points themselves.  The
 * paper fixes sigma = 2 and names sigma = 1.25 as the choice that trades a
 * wider kernel (more spreading work, Sec. 3) for a smaller fine grid (a cheaper
 * FFT); sigma shapes the fine grid, the kernel and the cuFFT plan, so it is
 * chosen here, before nufft_makeplan, not at setpts.
 *   type, dim (2 or 3), nmodes, eps   as nufft_makeplan;
 *   prec                0 or 1: the precision of x / y / z and of the plan to be
 *                       made (sigma = 1.25 is a candidate in single precision
 *                       only for eps >= 1e-4, as in makeplan);
 *   M, x, y, z          the points (device arrays of prec; z NULL in 2D);
 *   stream              the stream of the skew histogram and the prediction;
 *   opts                in / out: on return upsampfac, method, bin[], msub and
 *                       threads hold the candidate of least predicted execute
 *                       time over sigma in {2, 1.25} and the autotuner's tile
 *                       candidates; its other fields are left as given.  Pass it
 *                       to nufft_makeplan unchanged.
 * With no picker installed on this device: upsampfac = 2 (it reaches every eps
 * that 1.25 reaches) and the tile fields automatic (0).  Synchronizes stream; the
 * picker's scratch is shared as for plans with use_picker.
 * Errors: NUFFT_ERR_ARG, NUFFT_ERR_SIZE, NUFFT_ERR_EPS (no sigma reaches eps at
 * this precision), NUFFT_ERR_ALLOC, NUFFT_ERR_CUDA; opts is unchanged on an
 * argument error. */
int nufft_pick(int type, int dim, const int64_t *nmodes, double eps, int prec, int64_t M,
               const void *x, const void *y, const void *z, void *stream, nufft_opts *opts);

#ifdef __cplusplus
}
#endif

#endif /* NUFFT_GB300_H */
