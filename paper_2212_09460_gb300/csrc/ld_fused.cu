// ld_fused.cu -- Steps 1-3 without an edge list: each CTA takes a square
// block of a frame (64 x 64 pixels when the block's accumulator fits shared
// memory, else 32 x 32), finds its edge pixels (Sobel |Gx|+|Gy| on the
// zero-padded image, Eq. 1, saturated and thresholded, Sec. 2.2) and votes
// them straight into a shared-memory accumulator that covers every theta bin
// but only the rho cells the block can reach (Eq. 3 with the Q16 table of
// Eqs. 4-5), then adds its non-zero cells into the frame's int32 accumulator
// in global memory.
//
// This is the paper's FPGA dataflow (Sec. 3.3: pixels stream through one
// processing element per theta, no list of edge coordinates in between) laid
// out for a GPU: the pixel stream is cut into blocks so that a block's rho
// range is short.  For a block of side B, rho over the block spans at most
// floor((B - 1)(|cos| + |sin|) + 1) cells per theta (45 for B = 32, 90 for
// B = 64), so the block's accumulator is at most 48 or 96 rows x n_theta
// counters.  The votes are the same integers as the two-stage path's, so the
// accumulator (and the peaks taken from it) are identical.
#include "ld_internal.cuh"

namespace ld {
namespace {

constexpr int kFThreads = 1024;

__device__ __forceinline__ int32_t floor_q16_i64(int64_t v) {
    return (int32_t)(v >= 0 ? v / 65536 : -((-v + 65535) / 65536));
}

// Rows of a theta's counters in a block of side B: rho over the block spans at
// most floor((B - 1)(|cos| + |sin|) + 1) <= 45 (B = 32) or 90 (B = 64) cells;
// the row stride is odd so that lanes of consecutive thetas fall on different
// banks.
template <int B>
struct FusedGeom {
    static constexpr int kRows = B == 32 ? 48 : 96;
    static constexpr int kRS = kRows + 1;
    static constexpr int kPPT = B * B / kFThreads;   // pixels per thread
};

template <int B>
__global__ void __launch_bounds__(kFThreads, 1) fused_vote_kernel(const __grid_constant__ FusedLaunch L) {
    constexpr int kRows = FusedGeom<B>::kRows, kRS = FusedGeom<B>::kRS, kPPT = FusedGeom<B>::kPPT;
    extern __shared__ __align__(16) int32_t fsm[];
    const int n_theta = L.n_theta;
    int32_t *acc_s = fsm;                                   // [n_theta][kRS]
    int32_t *rmin_s = acc_s + kRS * n_theta;                // [n_theta] rho of row 0
    int32_t *cs_s = rmin_s + n_theta;                       // [n_theta][2] Q16 (c, s)
    uint32_t *edges_s = reinterpret_cast<uint32_t *>(cs_s + 2 * n_theta);   // [B * B]
    __shared__ uint8_t patch[B + 2][B + 2];
    __shared__ int n_edges;
    const int tid = threadIdx.x, lane = tid & 31;

    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.f[mid].tile_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const FusedFrame &F = L.f[lo];
    const int local = blockIdx.x - F.tile_begin;
    const int x0 = (local % F.tiles_x) * B, y0 = (local / F.tiles_x) * B;
    const int w = F.w, h = F.h;
    if (local == 0 && tid == 0) {   // until the merge writes the frame's peaks
        if (F.status_init) *F.status_init = LD_ERR_TIMEOUT;
        if (F.npeaks_init) *F.npeaks_init = 0;
    }

    // the block's pixels with a 1-pixel halo, zero outside the image
    for (int i = tid; i < (B + 2) * (B + 2); i += kFThreads) {
        const int r = i / (B + 2), c = i % (B + 2);
        const int y = y0 - 1 + r, x = x0 - 1 + c;
        patch[r][c] = (x >= 0 && y >= 0 && x < w && y < h) ? F.img[(size_t)y * F.pitch + x] : 0;
    }
    // per theta: Q16 (c, s) (Eqs. 4-5) and the smallest rho over the block's corners
    const int half = n_theta / 2;
    const int bx1 = min(x0 + B, w) - 1, by1 = min(y0 + B, h) - 1;
    for (int k = tid; k < n_theta; k += kFThreads) {
        const int kk = k <= half ? k : n_theta - k;
        const int32_t c = k <= half ? L.trig[2 * kk] : -L.trig[2 * kk];
        const int32_t s = L.trig[2 * kk + 1];
        cs_s[2 * k] = c;
        cs_s[2 * k + 1] = s;
        const int64_t xm = c < 0 ? (int64_t)bx1 * c : (int64_t)x0 * c;
        const int64_t ym = s < 0 ? (int64_t)by1 * s : (int64_t)y0 * s;
        rmin_s[k] = floor_q16_i64(xm + ym + 32768);
    }
    for (int i = tid; i < kRS * n_theta; i += kFThreads) acc_s[i] = 0;
    if (tid == 0) n_edges = 0;
    __syncthreads();

    // Steps 1-2 for this thread's pixels
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
        const int pix = tid + k * kFThreads;
        const int px = pix % B, py = pix / B;
        const int x = x0 + px, y = y0 + py;
        bool edge = false;
        if (x < w && y < h) {
            const uint8_t *a = patch[py] + px, *b = patch[py + 1] + px, *d = patch[py + 2] + px;
            const int gx = (a[2] + 2 * b[2] + d[2]) - (a[0] + 2 * b[0] + d[0]);
            const int gy = (d[0] + 2 * d[1] + d[2]) - (a[0] + 2 * a[1] + a[2]);
            int m = abs(gx) + abs(gy);
            m = m > 255 ? 255 : m;
            edge = m >= L.threshold;
            if (L.border == LD_BORDER_CLEAR && (x == 0 || y == 0 || x == w - 1 || y == h - 1)) edge = false;
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, edge);
        if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&n_edges, __popc(bal));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (edge) edges_s[base + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)y << 16) | (uint32_t)x;
        }
    }
    __syncthreads();

    // Step 3 into the block's accumulator: thread t votes theta t % n_theta for
    // the edges t / n_theta, + G, + 2G, ... (G = the thread groups that fit)
    const int ne = n_edges;
    const int G = kFThreads / n_theta;   // >= 1 (n_theta <= 1024)
    if (tid < G * n_theta) {
        const int k = tid % n_theta;
        const int32_t c = cs_s[2 * k], s = cs_s[2 * k + 1], r0 = rmin_s[k];
        int32_t *col = acc_s + k * kRS;
        for (int e = tid / n_theta; e < ne; e += G) {
            const uint32_t ev = edges_s[e];
            const int32_t rho = (int32_t)(((int)(ev & 0xFFFFu) * c + (int)(ev >> 16) * s + 32768) >> 16);   // floor
            const int row = rho - r0;   // 0 .. kRows - 1 by the corner bound
            if ((unsigned)row < (unsigned)kRows) atomicAdd(col + row, 1);
        }
    }
    __syncthreads();

    // the block's non-zero cells into the frame's accumulator: consecutive
    // threads take consecutive rho cells of one theta (contiguous addresses)
    if (ne > 0) {
        for (int i = tid; i < kRS * n_theta; i += kFThreads) {
            const int v = acc_s[i];
            if (v) {
                const int k = i / kRS, row = i - k * kRS;
                atomicAdd(F.acc + (size_t)k * F.n_rho + (rmin_s[k] + row + F.D), v);
            }
        }
    }
}

template <int B>
size_t fused_smem(int n_theta) {
    return (size_t)(FusedGeom<B>::kRS * n_theta + 3 * n_theta) * 4 + (size_t)B * B * 4;
}

}  // namespace

// Blocks of 64 x 64 pixels can be used when their accumulator fits shared
// memory (four times the pixels per flush of the block's cells).
int fused_side(int n_theta) { return fused_smem<64>(n_theta) <= (size_t)kSmemLimit - 8192 ? 64 : 32; }

size_t fused_smem_bytes(int n_theta) { return fused_smem<32>(n_theta); }

int fused_blocks(int w, int h) { return ((w + kFusedBlock - 1) / kFusedBlock) * ((h + kFusedBlock - 1) / kFusedBlock); }

cudaError_t launch_fused_vote(const FusedLaunch &L0, int /*n_blocks*/, cudaStream_t s) {
    if (L0.n <= 0) return cudaSuccess;
    auto count = [&](int side) {
        int64_t b = 0;
        for (int k = 0; k < L0.n; ++k) b += (int64_t)((L0.f[k].w + side - 1) / side) * ((L0.f[k].h + side - 1) / side);
        return b;
    };
    // large blocks only when they still give every SM two of them (small
    // launches keep the smaller blocks' parallelism)
    int dev = 0, sms = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) return e0;
    const int side = fused_side(L0.n_theta) == 64 && count(64) >= 2 * (int64_t)sms ? 64 : 32;
    if (count(side) > 0x7FFFFFFF) return cudaErrorInvalidValue;
    FusedLaunch L = L0;   // block layout of the chosen side
    int blocks = 0;
    for (int k = 0; k < L.n; ++k) {
        L.f[k].tile_begin = blocks;
        L.f[k].tiles_x = (L.f[k].w + side - 1) / side;
        blocks += L.f[k].tiles_x * ((L.f[k].h + side - 1) / side);
    }
    const size_t smem = side == 64 ? fused_smem<64>(L.n_theta) : fused_smem<32>(L.n_theta);
    // the dynamic limit leaves room for the kernels' static shared memory (the patch)
    if (smem > (size_t)kSmemLimit - 8192) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> attr_done{0};
    const cudaError_t e = once_per_device(attr_done, [](int) {
        cudaError_t r = cudaFuncSetAttribute(fused_vote_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemLimit - 8192);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(fused_vote_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kSmemLimit - 8192);
        return r;
    });
    if (e != cudaSuccess) return e;
    if (side == 64) fused_vote_kernel<64><<<blocks, kFThreads, smem, s>>>(L);
    else fused_vote_kernel<32><<<blocks, kFThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace ld
