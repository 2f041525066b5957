// ld_static.cu -- ld_hough_peaks_static: the peak search of ld_hough_peaks
// for callers that may not allocate device memory.
//
// Who needs it: a camera loop with a fixed per-frame deadline, or a host
// thread that must never block on the GPU, cannot call cudaMalloc once it is
// running (cudaMalloc may synchronise the device and its latency is
// unbounded), and a process whose device memory budget is fixed when it starts
// may not grow it later.  ld_hough_peaks keeps its candidate buffer in the
// context and grows it with cudaMalloc on first use; this variant needs no
// context and allocates nothing: its candidates live in a file-scope
// __device__ array of fixed size that is part of the loaded library.
//
// The array holds kStaticCandKeys 8-byte keys (1 MiB) on every GPU that loads
// the library, for the life of the process.  Its device address is looked up
// once per device and kept, so the entry point must not be used on a device
// after cudaDeviceReset (or any other teardown of its primary context) in the
// same process: the kept address would then be stale.  Every call on a device
// shares the array and it keeps the last call's contents; the kernels write
// every slot they later read, so nothing has to be cleared between calls.  Two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on the array: serialise them.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ld_internal.cuh"

namespace ld {
namespace {

constexpr int64_t kStaticCandKeys = 131072;   // 1 MiB of uint64 candidate keys
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint64_t g_static_cand[kStaticCandKeys];

std::mutex g_setup_mu;
void *g_cand_addr[kMaxDevices] = {};   // device address of g_static_cand, per device

// Host code cannot use &g_static_cand (that is a host-side stand-in); the
// device address comes from cudaGetSymbolAddress, once per device, with that
// device current.
cudaError_t static_cand(int dev, uint64_t **out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_cand_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_cand);
        if (e != cudaSuccess) return e;
        g_cand_addr[dev] = p;
    }
    *out = static_cast<uint64_t *>(g_cand_addr[dev]);
    return cudaSuccess;
}

}  // namespace
}  // namespace ld

using namespace ld;

extern "C" ld_status ld_hough_peaks_static(const int32_t *d_acc, int32_t n_theta, int32_t n_rho,
                                          const ld_params *pp, ld_peak *d_peaks, int32_t *d_n_peaks,
                                          void *stream) {
    char msg[256];
    ld_params q;
    const ld_status st = peak_params(pp, n_theta, &q);   // NULL: the defaults, as ld_hough_peaks
    if (st != LD_OK) return st;
    const ld_params *p = &q;
    if (!d_acc || !d_peaks || !d_n_peaks) {
        set_last_error("ld_hough_peaks_static: NULL buffer");
        return LD_ERR_INVALID;
    }
    if (n_theta < 1 || n_theta > kMaxTheta || n_rho < 1 || n_rho > 65535) {
        snprintf(msg, sizeof msg, "ld_hough_peaks_static: accumulator %d x %d: need 1 <= n_theta <= %d, "
                                  "1 <= n_rho <= 65535", n_theta, n_rho, kMaxTheta);
        set_last_error(msg);
        return LD_ERR_INVALID;
    }
    const int M = p->nms_theta * p->nms_rho * (p->top_k - 1) + 1;
    const int64_t cells = (int64_t)n_theta * n_rho;
    const int64_t n_chunks = (cells + kSelectChunk - 1) / kSelectChunk;
    if (n_chunks * M > kStaticCandKeys) {
        snprintf(msg, sizeof msg, "ld_hough_peaks_static: %lld cells with M = %d need %lld candidate slots, "
                                  "the static buffer holds %lld (use ld_hough_peaks)",
                 (long long)cells, M, (long long)(n_chunks * M), (long long)kStaticCandKeys);
        set_last_error(msg);
        return LD_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_last_error("ld_hough_peaks_static: no usable current device");
        return LD_ERR_CUDA;
    }
    uint64_t *cand = nullptr;
    e = static_cand(dev, &cand);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "ld_hough_peaks_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return LD_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SelectLaunch SL;
    std::memset(&SL, 0, sizeof SL);
    SL.n = 1;
    SL.cand_m = M;
    SL.min_votes = p->min_votes;
    SL.j[0].acc = d_acc;
    SL.j[0].cand = cand;
    SL.j[0].cells = cells;
    SL.j[0].n_rho = n_rho;
    SL.j[0].n_chunks = (int32_t)n_chunks;
    SL.j[0].chunk_begin = 0;
    e = launch_select(SL, (int)n_chunks, s);
    if (e == cudaSuccess) {
        MergeLaunch ML;
        std::memset(&ML, 0, sizeof ML);
        ML.n = 1;
        ML.top_k = p->top_k;
        ML.nms_theta = p->nms_theta;
        ML.nms_rho = p->nms_rho;
        ML.j[0].cand = cand;
        ML.j[0].n_cand = n_chunks * M;
        ML.j[0].peaks = d_peaks;
        ML.j[0].n_peaks = d_n_peaks;
        e = launch_merge(ML, s);
    }
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "ld_hough_peaks_static: launch: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return LD_ERR_CUDA;
    }
    return LD_OK;
}
