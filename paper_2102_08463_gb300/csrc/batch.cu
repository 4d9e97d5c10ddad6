// batch.cu -- many plans executed together (batched execution of independent
// transforms of uneven N and M; not in the paper, whose interface runs one plan
// at a time).
//
// Plans that share type, dimension, precision, kernel width and method form a
// group; each group's spreading or interpolation runs as ONE persistent launch
// over the work items of all its plans ((plan, subproblem, transform) triples,
// or (plan, chunk of kGmChunk points, transform) for GM plans, located by a
// binary search over device-side work offsets computed from each plan's
// subproblem or chunk count).  The fine-grid clear, the
// correction steps and cuFFT stay one call per plan.  The whole sequence can be
// captured once into a CUDA graph and replayed with one launch.
#include <algorithm>
#include <new>
#include <vector>

#include "spread_interp.cuh"

using namespace nufft;

namespace {

__global__ void batch_workoff_kernel(const int32_t *const *__restrict__ nsub,
                                     const int *__restrict__ ntransf, int nplans,
                                     int64_t *__restrict__ workoff)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t s = 0;
    for (int p = 0; p < nplans; ++p) {
        workoff[p] = s;
        s += (int64_t)(*nsub[p]) * ntransf[p];
    }
    workoff[nplans] = s;
}

// Host staging of the kernel arguments: a direct execute fills the next of
// kRing pinned slots, after waiting for the event that marks the end of that
// slot's previous copy, so back-to-back executes never overwrite arguments that
// an earlier copy has yet to read.  A captured graph copies from a slot of its
// own (graph_h_args) into a device array of its own (graph_d_args), written
// only when the graph is captured; executes never touch either.
constexpr int kRing = 4;

struct Group {
    int type = 1, dim = 2, prec = 0, w = 0, method = NUFFT_METHOD_SM;
    int variant = 0;                   // row-sweep form (sweep_variant), part of the key
    int m0max = 1, m1max = 1, tile = 1, smem_optin = 0;
    std::vector<int> members;          // indices into the batch's plans
    size_t smem = 0;                   // max padded-bin bytes over the members
    size_t args_bytes = 0;             // one KArgs<T> per member
    void *d_args = nullptr;            // device KArgs array (direct executes)
    void *h_ring[kRing] = {};          // pinned staging slots (direct executes)
    cudaEvent_t ev_ring[kRing] = {};   // end of each slot's last copy
    int ring_next = 0;
    void *graph_d_args = nullptr;      // device KArgs array read by the captured graph
    void *graph_h_args = nullptr;      // pinned source of the graph's copy
    int64_t *d_workoff = nullptr;      // device [members + 1]
    const int32_t **d_nsub = nullptr;  // device array of the members' nsub pointers
    int *d_ntransf = nullptr;
};

size_t real_bytes(int prec) { return prec == 0 ? 4 : 8; }

template <typename T>
void fill_args(const std::vector<nufft_plan> &plans, const Group &g, void *const *c, void *host)
{
    KArgs<T> *dst = reinterpret_cast<KArgs<T> *>(host);
    for (size_t i = 0; i < g.members.size(); ++i) {
        const int k = g.members[i];
        const Plan &p = plans[k]->p;
        KArgs<T> a = make_args<T>(p);
        if (p.type == 1)
            a.cin = reinterpret_cast<const typename cplx<T>::type *>(c[k]);
        else
            a.cout = reinterpret_cast<typename cplx<T>::type *>(c[k]);
        dst[i] = a;
    }
}

cudaError_t multi_launch(const Group &g, const MultiLaunch &ml)
{
    const bool t1 = g.type == 1;
    if (g.prec == 0) {
        if (g.dim == 1) return t1 ? spread_multi_f32_1d(ml) : interp_multi_f32_1d(ml);
        if (g.dim == 2) return t1 ? spread_multi_f32_2d(ml) : interp_multi_f32_2d(ml);
        return t1 ? spread_multi_f32_3d(ml) : interp_multi_f32_3d(ml);
    }
    if (g.dim == 1) return t1 ? spread_multi_f64_1d(ml) : interp_multi_f64_1d(ml);
    if (g.dim == 2) return t1 ? spread_multi_f64_2d(ml) : interp_multi_f64_2d(ml);
    return t1 ? spread_multi_f64_3d(ml) : interp_multi_f64_3d(ml);
}

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return NUFFT_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NUFFT_ERR_ALLOC : NUFFT_ERR_CUDA;
}

}  // namespace

struct nufft_batch_s {
    std::vector<nufft_plan> plans;
    std::vector<cudaStream_t> saved_streams;
    std::vector<Group> groups;
    cudaStream_t stream = nullptr;
    int num_sms = 152;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
};

namespace {

void free_batch(nufft_batch_s *b)
{
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (Group &g : b->groups) {
        if (g.d_args) cudaFree(g.d_args);
        for (int i = 0; i < kRing; ++i) {
            if (g.h_ring[i]) cudaFreeHost(g.h_ring[i]);
            if (g.ev_ring[i]) cudaEventDestroy(g.ev_ring[i]);
        }
        if (g.graph_d_args) cudaFree(g.graph_d_args);
        if (g.graph_h_args) cudaFreeHost(g.graph_h_args);
        if (g.d_workoff) cudaFree(g.d_workoff);
        if (g.d_nsub) cudaFree(g.d_nsub);
        if (g.d_ntransf) cudaFree(g.d_ntransf);
    }
    // hand the plans back their own streams
    for (size_t i = 0; i < b->plans.size() && i < b->saved_streams.size(); ++i) {
        Plan &p = b->plans[i]->p;
        p.stream = b->saved_streams[i];
        if (p.fft_ready) cufftSetStream(p.fft, p.stream);
    }
    delete b;
}

// One batched execute.  for_graph: the call is being captured; the arguments
// go through the graph's own staging (see kRing).
int run_batch(nufft_batch_s *b, void *const *c, void *const *f, bool for_graph)
{
    cudaStream_t st = b->stream;
    for (size_t k = 0; k < b->plans.size(); ++k) {
        const Plan &p = b->plans[k]->p;
        if (!p.have_pts) return NUFFT_ERR_NOPTS;
        if (!f[k] || (p.M > 0 && !c[k])) return NUFFT_ERR_ARG;
    }
    // per-plan pre-steps: clear the fine grid (type 1) / precorrect (type 2)
    for (Group &g : b->groups) {
        for (int k : g.members) {
            Plan &p = b->plans[k]->p;
            cudaError_t e = g.type == 1
                                ? launch_zero(p, p.fine, (size_t)p.nftot * p.ntransf * 2 * real_bytes(p.prec))
                                : launch_precorrect(p, f[k]);
            if (e != cudaSuccess) return cuda_rc(e);
            if (g.type == 2) {
                int rc = nufft_fft(b->plans[k]);
                if (rc != NUFFT_OK) return rc;
            }
        }
    }
    // grouped spreading / interpolation
    for (Group &g : b->groups) {
        void *host = g.graph_h_args, *dev = g.graph_d_args;
        int slot = -1;
        if (!for_graph) {
            slot = g.ring_next;
            g.ring_next = (g.ring_next + 1) % kRing;
            cudaError_t e = cudaEventSynchronize(g.ev_ring[slot]);   // slot's last copy done
            if (e != cudaSuccess) return cuda_rc(e);
            host = g.h_ring[slot];
            dev = g.d_args;
        }
        if (g.prec == 0) fill_args<float>(b->plans, g, c, host);
        else fill_args<double>(b->plans, g, c, host);
        cudaError_t e = cudaMemcpyAsync(dev, host, g.args_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_rc(e);
        if (slot >= 0) {
            e = cudaEventRecord(g.ev_ring[slot], st);
            if (e != cudaSuccess) return cuda_rc(e);
        }
        count_launch();
        batch_workoff_kernel<<<1, 32, 0, st>>>(g.d_nsub, g.d_ntransf, (int)g.members.size(),
                                               g.d_workoff);
        MultiLaunch ml;
        ml.args = dev;
        ml.workoff = g.d_workoff;
        ml.nplans = (int)g.members.size();
        ml.w = g.w;
        ml.method = g.method;
        ml.threads = kDefaultThreads;
        ml.num_sms = b->num_sms;
        ml.smem = g.method == NUFFT_METHOD_SM ? g.smem : 0;
        ml.smem_optin = (size_t)g.smem_optin;
        ml.variant = g.variant;
        ml.m0max = g.m0max;
        ml.m1max = g.m1max;
        ml.tile = g.tile;
        ml.stream = st;
        e = multi_launch(g, ml);
        if (e != cudaSuccess) return cuda_rc(e);
    }
    // type 1 post-steps: cuFFT and correction per plan
    for (Group &g : b->groups) {
        if (g.type != 1) continue;
        for (int k : g.members) {
            int rc = nufft_fft(b->plans[k]);
            if (rc != NUFFT_OK) return rc;
            rc = nufft_deconvolve(b->plans[k], f[k]);
            if (rc != NUFFT_OK) return rc;
        }
    }
    return NUFFT_OK;
}

}  // namespace

extern "C" {

int nufft_batch_create(const nufft_plan *plans, int nplans, void *stream, nufft_batch *out)
{
    if (!out) return NUFFT_ERR_ARG;
    *out = nullptr;
    if (!plans || nplans < 1) return NUFFT_ERR_ARG;
    for (int k = 0; k < nplans; ++k) {
        if (!plans[k] || plans[k]->p.type == 3) return NUFFT_ERR_ARG;   // types 1 and 2
        for (int j = 0; j < k; ++j)
            if (plans[j] == plans[k]) return NUFFT_ERR_ARG;
    }
    nufft_batch_s *b = new (std::nothrow) nufft_batch_s;
    if (!b) return NUFFT_ERR_ALLOC;
    b->stream = (cudaStream_t)stream;
    b->plans.assign(plans, plans + nplans);
    b->num_sms = plans[0]->p.num_sms;
    for (int k = 0; k < nplans; ++k) {
        Plan &p = plans[k]->p;
        b->saved_streams.push_back(p.stream);
        p.stream = b->stream;
        if (p.fft_ready && cufftSetStream(p.fft, p.stream) != CUFFT_SUCCESS) {
            free_batch(b);
            return NUFFT_ERR_CUFFT;
        }
        const int variant = sweep_variant(p);
        Group *g = nullptr;
        for (Group &cand : b->groups)
            if (cand.type == p.type && cand.dim == p.dim && cand.prec == p.prec && cand.w == p.w &&
                cand.method == p.method && cand.variant == variant)
                g = &cand;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->type = p.type;
            g->dim = p.dim;
            g->prec = p.prec;
            g->w = p.w;
            g->method = p.method;
            g->variant = variant;
            g->smem_optin = p.smem_optin;
        }
        g->members.push_back(k);
        size_t cells = 1;
        for (int d = 0; d < p.dim; ++d) cells *= (size_t)padded(p.m[d], p.w);
        g->smem = std::max(g->smem, cells * 2 * real_bytes(p.prec));
        g->tile = std::max(g->tile, (int)cells);
        g->m0max = std::max(g->m0max, p.m[0]);
        g->m1max = std::max(g->m1max, p.m[1]);
    }
    for (Group &g : b->groups) {
        const size_t n = g.members.size();
        g.args_bytes = n * (g.prec == 0 ? sizeof(KArgs<float>) : sizeof(KArgs<double>));
        std::vector<const int32_t *> nsub(n);
        std::vector<int> nt(n);
        for (size_t i = 0; i < n; ++i) {
            nsub[i] = b->plans[g.members[i]]->p.nsub;
            nt[i] = b->plans[g.members[i]]->p.ntransf;
        }
        cudaError_t e = cudaMalloc(&g.d_args, g.args_bytes);
        for (int i = 0; i < kRing && e == cudaSuccess; ++i) {
            e = cudaMallocHost(&g.h_ring[i], g.args_bytes);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.ev_ring[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaMalloc(&g.graph_d_args, g.args_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&g.graph_h_args, g.args_bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g.d_workoff, sizeof(int64_t) * (n + 1));
        if (e == cudaSuccess) e = cudaMalloc((void **)&g.d_nsub, sizeof(int32_t *) * n);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g.d_ntransf, sizeof(int) * n);
        if (e == cudaSuccess)
            e = cudaMemcpy(g.d_nsub, nsub.data(), sizeof(int32_t *) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(g.d_ntransf, nt.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_batch(b);
            return cuda_rc(e);
        }
    }
    *out = b;
    return NUFFT_OK;
}

int nufft_batch_execute(nufft_batch b, void *const *c, void *const *f)
{
    if (!b || !c || !f) return NUFFT_ERR_ARG;
    return run_batch(b, c, f, false);
}

int nufft_batch_capture(nufft_batch b, void *const *c, void *const *f)
{
    if (!b || !c || !f) return NUFFT_ERR_ARG;
    if (b->stream == nullptr) return NUFFT_ERR_ARG;   // the legacy stream cannot be captured
    if (b->graph_exec) {
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    // a replay of the previous graph may still be reading its staging
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_rc(e);
    const int rc = run_batch(b, c, f, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->stream, &g);
    if (rc != NUFFT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_rc(e);
    b->graph = g;
    e = cudaGraphInstantiate(&b->graph_exec, g, 0);
    return cuda_rc(e);
}

int nufft_batch_launch(nufft_batch b)
{
    if (!b) return NUFFT_ERR_ARG;
    if (!b->graph_exec) return NUFFT_ERR_NOPTS;
    return cuda_rc(cudaGraphLaunch(b->graph_exec, b->stream));
}

int nufft_batch_destroy(nufft_batch b)
{
    if (b) free_batch(b);
    return NUFFT_OK;
}

}  // extern "C"
