// noalloc.cu -- allocation-free bin-sort entry point (nufft_binsort_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while memory is being
// handed out by another allocator, real-time or embedded callers with a fixed
// memory budget decided at start-up, and host paths that must not take the
// driver's allocation locks.  For them this file provides the stable bin-sort
// of the points (the permutation t and the per-bin counts) with all of its
// scratch in one file-scope device array of a fixed size, so a call allocates
// nothing: the caller passes the points and the two output arrays.
//
// Limits: at most kMaxPoints points and kMaxBins bins per call.  The array is
// about 8.1 MB and is resident on every device that loads this library, for the
// life of the process.  Under CUDA's lazy module loading the driver places it
// (and loads the kernels) at the library's first use on a device, which may
// allocate; a warm-up call per device at start-up (M = 0 suffices) moves that
// cost out of the caller's allocation-free section.  Every call writes all the
// scratch it later reads, so nothing in it has to start at zero; but all calls
// on one device share it, so calls whose GPU work overlaps (different streams,
// or host threads) race and must be serialised by the caller.
#include <mutex>

#include "nufft_internal.cuh"

using namespace nufft;

namespace {

constexpr int64_t kMaxPoints = (int64_t)1 << 20;
constexpr int kMaxBins = 1 << 14;
constexpr int kMaxCtas = 64;
constexpr int64_t kPartInts = 1024;

constexpr size_t kKeysBytes = sizeof(int32_t) * (size_t)kMaxPoints;
constexpr size_t kMatBytes = sizeof(int32_t) * (size_t)kMaxBins * kMaxCtas;
constexpr size_t kBinBytes = sizeof(int32_t) * (size_t)kMaxBins;
constexpr size_t kPartBytes = sizeof(int32_t) * (size_t)kPartInts;
constexpr size_t kScratchBytes = kKeysBytes + kMatBytes + kBinBytes + kPartBytes;

static __device__ __align__(256) unsigned char g_binsort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name of a
// __device__ array in host code is only a host-side handle, so the address is
// looked up once per device with cudaGetSymbolAddress and cached.
int scratch_on_current_device(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NUFFT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return NUFFT_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_binsort_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return NUFFT_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return NUFFT_OK;
}

}  // namespace

extern "C" int nufft_binsort_noalloc(int dim, int prec, int64_t M, const void *x, const void *y,
                                     const void *z, const int64_t *nf, const int *bins,
                                     int32_t *perm, int32_t *bincount, void *stream)
{
    if ((dim != 2 && dim != 3) || (prec != 0 && prec != 1) || !nf || !bins || !bincount)
        return NUFFT_ERR_ARG;
    if (M < 0) return NUFFT_ERR_ARG;
    if (M > kMaxPoints) return NUFFT_ERR_SIZE;
    if (M > 0 && (!x || !y || (dim == 3 && !z) || !perm)) return NUFFT_ERR_ARG;
    int64_t nbins = 1;
    for (int d = 0; d < dim; ++d) {
        if (nf[d] < 1 || nf[d] > (1 << 20) || bins[d] < 1 || bins[d] > nf[d]) return NUFFT_ERR_ARG;
        nbins *= (nf[d] + bins[d] - 1) / bins[d];
        if (nbins > kMaxBins) return NUFFT_ERR_SIZE;
    }
    unsigned char *base = nullptr;
    int rc = scratch_on_current_device(&base);
    if (rc != NUFFT_OK) return rc;
    int64_t nblk = (M + 8191) / 8192;
    if (nblk > kMaxCtas) nblk = kMaxCtas;
    if (nblk < 1) nblk = 1;
    BinsortScratch s;
    s.keys = reinterpret_cast<int32_t *>(base);
    s.mat = reinterpret_cast<int32_t *>(base + kKeysBytes);
    s.binstart = reinterpret_cast<int32_t *>(base + kKeysBytes + kMatBytes);
    s.scan_part = reinterpret_cast<int32_t *>(base + kKeysBytes + kMatBytes + kBinBytes);
    s.nblk = (int)nblk;
    cudaError_t e = launch_binsort_into(s, prec, dim, M, x, y, z, nf, bins, perm, bincount,
                                        (cudaStream_t)stream);
    if (e == cudaErrorMemoryAllocation) return NUFFT_ERR_ALLOC;
    return e == cudaSuccess ? NUFFT_OK : NUFFT_ERR_CUDA;
}
