// autotune.cu -- measured choice of the spreading / interpolation tiles (method,
// bin sizes, subproblem cap M_sub, threads per CTA) for a problem, and a cache of
// the winners that plans created with automatic settings consult at setpts.
//
// The paper fixes its tiles by hand for its own GPU (Sec. 4.1 remark: 32 x 32
// and 16 x 16 x 2 bins, M_sub = 1024).  Here the candidates are timed on the
// caller's own points with CUDA events: one plan is made, re-tiled for every
// candidate (its cuFFT plan and fine grid are kept), its points set, and its
// execute timed.  The winner is stored under a problem class (type, dimension,
// precision, kernel width, sigma, log2 of the fine-grid size, half-octave of the
// density M / n_tot) and can be saved to / loaded from a text file.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "nufft_internal.cuh"

using namespace nufft;

namespace {

struct Key {
    int type, dim, prec, w, sig, lgn, lgrho;
    bool operator<(const Key &o) const
    {
        return std::tie(type, dim, prec, w, sig, lgn, lgrho) <
               std::tie(o.type, o.dim, o.prec, o.w, o.sig, o.lgn, o.lgrho);
    }
};

struct Entry {
    Tiles tiles;
    double ms = 0.0;
};

std::mutex g_cache_mutex;
std::map<Key, Entry> g_cache;

Key key_of(const Plan &p, int64_t M)
{
    Key k;
    k.type = p.type;
    k.dim = p.dim;
    k.prec = p.prec;
    k.w = p.w;
    k.sig = p.sigma == 2.0 ? 200 : (int)lround(p.sigma * 100);
    k.lgn = (int)lround(log2((double)p.nftot));
    const double rho = M > 0 ? (double)M / (double)p.nftot : 1e-9;
    k.lgrho = (int)lround(2.0 * log2(rho));
    return k;
}

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return NUFFT_OK;
    cudaGetLastError();
    return NUFFT_ERR_CUDA;
}

}  // namespace

std::vector<Tiles> nufft::tile_candidates(const Plan &p)
{
    const int dim = p.dim;
    std::vector<std::vector<int>> bins;
    if (dim == 2)
        bins = {{8, 8, 1}, {16, 16, 1}, {32, 16, 1}, {32, 32, 1}, {64, 32, 1}};
    else
        bins = {{8, 8, 4}, {8, 8, 8}, {16, 16, 2}, {16, 16, 4}, {16, 8, 4}, {32, 32, 2}, {32, 16, 4}};
    const int msubs[] = {256, 1024, 4096};
    const int threads[] = {128, 256};
    std::vector<Tiles> out;
    for (int method : {NUFFT_METHOD_SM, NUFFT_METHOD_GM_SORT})
        for (const auto &b : bins)
            for (int ms : msubs)
                for (int th : threads) {
                    Tiles t;
                    t.method = method;
                    t.bin[0] = b[0];
                    t.bin[1] = b[1];
                    t.bin[2] = b[2];
                    t.msub = ms;
                    t.threads = th;
                    out.push_back(t);
                }
    Tiles gm;
    gm.method = NUFFT_METHOD_GM;
    gm.bin[0] = gm.bin[1] = 16;
    gm.bin[2] = dim == 3 ? 2 : 1;
    out.push_back(gm);
    // the plan's default (heuristic) tiling, when not already listed
    Tiles h;
    h.method = NUFFT_METHOD_SM;
    default_bins(p.type, dim, p.prec, p.w, h.bin);
    h.msub = 1024;
    h.threads = kDefaultThreads;
    bool listed = false;
    for (const Tiles &t : out)
        listed = listed || (t.method == h.method && t.bin[0] == h.bin[0] && t.bin[1] == h.bin[1] &&
                            t.bin[2] == h.bin[2] && t.msub == h.msub && t.threads == h.threads);
    if (!listed) out.push_back(h);
    return out;
}

bool nufft::tune_cache_lookup(const Plan &p, int64_t M, Tiles *out)
{
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto it = g_cache.find(key_of(p, M));
    if (it == g_cache.end()) return false;
    *out = it->second.tiles;
    return true;
}

extern "C" {

int nufft_autotune(int type, int dim, const int64_t *nmodes, int iflag, int ntransf, double eps,
                   int prec, const nufft_opts *base, int64_t M, const void *x, const void *y,
                   const void *z, void *c, void *f, int reps, nufft_opts *best, double *best_ms,
                   nufft_tune_trial *trials, int max_trials, int *ntrials)
{
    if (!best || reps < 1 || M < 1 || !c || !f || dim < 2) return NUFFT_ERR_ARG;   // 2D and 3D tiles
    nufft_opts o;
    nufft_default_opts(&o);
    if (base) o = *base;
    o.method = NUFFT_METHOD_SM;
    nufft_plan h = nullptr;
    int rc = nufft_makeplan(type, dim, nmodes, iflag, ntransf, eps, prec, &o, &h);
    if (rc != NUFFT_OK) {
        o.method = NUFFT_METHOD_GM_SORT;
        rc = nufft_makeplan(type, dim, nmodes, iflag, ntransf, eps, prec, &o, &h);
        if (rc != NUFFT_OK) return rc;
    }
    Plan &p = h->p;
    p.auto_tiles = false;
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    double best_time = 1e300;
    Tiles best_t;
    int n = 0;
    for (const Tiles &t : tile_candidates(p)) {
        if (plan_set_tiles(p, t) != NUFFT_OK) continue;
        cudaEventRecord(e0, p.stream);
        if (nufft_setpts(h, M, x, y, z) != NUFFT_OK) continue;
        cudaEventRecord(e1, p.stream);
        if (nufft_execute(h, c, f) != NUFFT_OK) continue;     // warm-up
        std::vector<float> times;
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r) {
            cudaEventRecord(e1, p.stream);
            ok = nufft_execute(h, c, f) == NUFFT_OK;
            cudaEventRecord(e2, p.stream);
            if (cudaEventSynchronize(e2) != cudaSuccess) ok = false;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e1, e2);
            times.push_back(ms);
        }
        if (!ok) {
            cudaGetLastError();
            continue;
        }
        float setpts_ms = 0.f;
        // e0 -> first e1 brackets setpts; re-measure it once on its own
        cudaEventRecord(e0, p.stream);
        nufft_setpts(h, M, x, y, z);
        cudaEventRecord(e1, p.stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&setpts_ms, e0, e1);
        std::sort(times.begin(), times.end());
        const double med = times[times.size() / 2];
        if (trials && n < max_trials) {
            nufft_tune_trial &tr = trials[n];
            tr.method = t.method;
            tr.bin[0] = t.bin[0];
            tr.bin[1] = t.bin[1];
            tr.bin[2] = t.bin[2];
            tr.msub = t.msub;
            tr.threads = t.threads;
            tr.exec_ms = med;
            tr.setpts_ms = setpts_ms;
        }
        ++n;
        if (med < best_time) {
            best_time = med;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (ntrials) *ntrials = n;
    if (n == 0) {
        nufft_destroy(h);
        return NUFFT_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        Entry &en = g_cache[key_of(p, M)];
        en.tiles = best_t;
        en.ms = best_time;
    }
    nufft_destroy(h);
    *best = o;
    best->method = best_t.method;
    best->bin[0] = best_t.bin[0];
    best->bin[1] = best_t.bin[1];
    best->bin[2] = best_t.bin[2];
    best->msub = best_t.msub;
    best->threads = best_t.threads;
    if (best_ms) *best_ms = best_time;
    return cuda_rc(cudaGetLastError());
}

int nufft_tune_cache_save(const char *path)
{
    if (!path) return NUFFT_ERR_ARG;
    FILE *fp = fopen(path, "w");
    if (!fp) return NUFFT_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    fprintf(fp, "# nufft_gb300 tuning cache v1: type dim prec w sigma100 lg2n lg2rho*2 "
                "method b0 b1 b2 msub threads ms\n");
    for (const auto &kv : g_cache) {
        const Key &k = kv.first;
        const Entry &e = kv.second;
        fprintf(fp, "%d %d %d %d %d %d %d %d %d %d %d %d %d %.6f\n", k.type, k.dim, k.prec, k.w,
                k.sig, k.lgn, k.lgrho, e.tiles.method, e.tiles.bin[0], e.tiles.bin[1],
                e.tiles.bin[2], e.tiles.msub, e.tiles.threads, e.ms);
    }
    fclose(fp);
    return NUFFT_OK;
}

int nufft_tune_cache_load(const char *path)
{
    if (!path) return NUFFT_ERR_ARG;
    FILE *fp = fopen(path, "r");
    if (!fp) return NUFFT_ERR_ARG;
    char line[512];
    int rc = NUFFT_OK;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    while (fgets(line, sizeof(line), fp)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        Key k;
        Entry e;
        const int got = sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d %d %lf", &k.type, &k.dim,
                               &k.prec, &k.w, &k.sig, &k.lgn, &k.lgrho, &e.tiles.method,
                               &e.tiles.bin[0], &e.tiles.bin[1], &e.tiles.bin[2], &e.tiles.msub,
                               &e.tiles.threads, &e.ms);
        if (got != 14) {
            rc = NUFFT_ERR_ARG;
            continue;
        }
        g_cache[k] = e;
    }
    fclose(fp);
    return rc;
}

int nufft_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    g_cache.clear();
    return NUFFT_OK;
}

}  // extern "C"
