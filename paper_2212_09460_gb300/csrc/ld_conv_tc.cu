// ld_conv_tc.cu -- forward 3x3 convolutions of the proposal network (16->32
// and 32->32 channels, stride 1 or 2) on the fifth-generation tensor cores:
// tcgen05.mma with bf16 operands from shared memory and an fp32 accumulator
// in tensor memory.  The paper has no learned stage; this is the project's
// proposal network (see ld_cnn.cu).
//
// Implicit GEMM per CTA tile: D[128 pixels][32 channels] = sum over the 9
// taps of A_tap[128][Cin] B_tap[32][Cin]^T, B being the weights
// [Cout][3][3][Cin] (K = 9 * Cin ordered (tap, channel)).  A tile is 16
// output rows x 8 output columns of one image.  All 128 threads copy the
// tile's input patch (zero-filled at the image border) and the weights with
// cp.async into shared memory in the unswizzled K-major core-matrix layout
// the tensor core reads (a core matrix = 8 rows of 16 bytes, contiguous); the
// patch is split by column parity so that every tap's A operand is a plain
// matrix descriptor into it (see Patch below) and no im2col copy is made.
// One thread issues the 9 * Cin/16 MMAs (M = 128, N = 32, K = 16 each) and
// commits them to an mbarrier; after a bounded wait each warp reads its 32
// accumulator lanes (one output pixel per thread, 32 fp32 channels) with
// tcgen05.ld, adds the bias, applies the ReLU and stores bf16 NHWC.  CTAs are
// persistent (as many as fit the SMs) with two shared-memory stages, so the
// copies of the next tile overlap the current tile's MMAs and epilogue.  A
// CTA holds 32 tensor-memory columns and at most 16 CTAs are placed on an SM,
// so allocation never waits.  A wait that gives up records a fault
// (ld_conv_faults) and the CTA frees its tensor memory and leaves.
#include <cuda_bf16.h>

#include "ld_internal.cuh"

namespace ld {

__device__ int32_t g_conv_faults;

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTcM = 128, kTcN = 32, kTcThreads = 128, kTmemCols = 32;
constexpr uint32_t kTcSpinLimit = 1u << 24;
// instruction descriptor (kind::f16): D fp32, A and B bf16, both K-major,
// N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (16-byte units), fixed version bit 46, no swizzle
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int nbytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const uint32_t a = saddr(bar);
    for (uint32_t i = 0; i < kTcSpinLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Tile geometry: 16 output rows x 8 output columns (m = 8 * row + column).
// The input patch of a tile, PR x PC pixels from (S*oy0 - 1, S*ox0 - 1), is
// stored as [PR][QPP][S][HC] chunks of 16 bytes (8 channels), the pixel of
// patch column pc in parity plane pc % S at index pc / S.  For tap (ky, kx)
// and channel chunks (q, q+1), the A operand of output pixel m = 8 r + c is
// the chunk at patch row S r + ky, column S c + kx: 8 consecutive c are 8
// consecutive 16-byte chunks of one parity plane (one core matrix), the next
// 8 pixels (r + 1) are S patch rows further (stride byte offset), and chunk
// q + 1 is S * HC chunks further (leading byte offset).  So every MMA reads
// its operands straight from the patch; no im2col copy is made.
constexpr int kTileH = 16, kTileW = 8;
template <int S>
struct Patch {
    static constexpr int PR = (kTileH - 1) * S + 3, PC = (kTileW - 1) * S + 3, HC = (PC + S - 1) / S;
};

// Start the copies of tile `tile`'s patch into one stage (and of the weights
// B when with_b); one commit group.
template <int CIN, int S>
__device__ __forceinline__ void load_tile(const bf16 *x, const ConvTcGeom &G, const bf16 *wt, int tile,
                                          int tiles_per_img, int tiles_x, uint8_t *Ps, uint8_t *Bs, bool with_b) {
    constexpr int K = 9 * CIN, KC = K / 8, QPP = CIN / 8;
    constexpr int PR = Patch<S>::PR, PC = Patch<S>::PC, HC = Patch<S>::HC;
    const int tid = threadIdx.x;
    const int img = tile / tiles_per_img, t = tile - img * tiles_per_img;
    const int iy0 = (t / tiles_x) * kTileH * S - 1, ix0 = (t % tiles_x) * kTileW * S - 1;
    const bf16 *xi = x + (int64_t)img * G.h * G.w * CIN;
    for (int i = tid; i < PR * PC * QPP; i += kTcThreads) {
        const int q = i % QPP, rest = i / QPP, pc = rest % PC, pr = rest / PC;
        const int iy = iy0 + pr, ix = ix0 + pc;
        const bool ok = iy >= 0 && iy < G.h && ix >= 0 && ix < G.w;
        const bf16 *src = ok ? xi + ((int64_t)iy * G.w + ix) * CIN + q * 8 : x;
        cp_async16(saddr(Ps + (((pr * QPP + q) * S + pc % S) * HC + pc / S) * 16), src, ok ? 16 : 0);
    }
    // B: chunk kc of output channel n (the same for every tile: loaded once)
    if (with_b)
        for (int i = tid; i < kTcN * KC; i += kTcThreads) {
            const int kc = i % KC, n = i / KC;
            cp_async16(saddr(Bs + ((kc * (kTcN / 8) + (n >> 3)) * 8 + (n & 7)) * 16), wt + (int64_t)n * K + kc * 8,
                       16);
        }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Fused first layer (inference): the input patch of a 16->32 stride-2 tile
// is conv1's output, computed here from the uint8 edge-count map x0 [h][w]
// (one image) exactly as the separate conv1 layer computes it (same fp32
// fused multiply-adds in the same order, same rounding to bf16), and zero
// outside the image (conv2's padding).  xs stages the counts / 64 of the
// (PR + 2) x (PC + 2) region under the patch.
struct Conv1Params {
    const uint8_t *x0;
    const bf16 *w1;   // [16][3][3][1]
    const float *b1;  // [16]
};

constexpr int kXsN = (Patch<2>::PR + 2) * (Patch<2>::PC + 2);   // staged counts per tile
constexpr int kXsPer = (kXsN + kTcThreads - 1) / kTcThreads;       // per thread

// Issue the loads of this thread's share of tile `tile`'s edge counts (/ 64,
// zero outside the map) into registers; they land while other work runs.
__device__ __forceinline__ void load_counts(const Conv1Params &C1, const ConvTcGeom &G, int tile, int tiles_per_img,
                                            int tiles_x, float (&xr)[kXsPer]) {
    constexpr int S = 2, XW = Patch<2>::PC + 2;
    const int img = tile / tiles_per_img, t = tile - img * tiles_per_img;
    const int iy0 = (t / tiles_x) * kTileH * S - 1, ix0 = (t % tiles_x) * kTileW * S - 1;
    const uint8_t *xi = C1.x0 + (int64_t)img * G.h * G.w;
#pragma unroll
    for (int j = 0; j < kXsPer; ++j) {
        const int i = threadIdx.x + j * kTcThreads;
        const int yy = iy0 - 1 + i / XW, xx = ix0 - 1 + i % XW;
        xr[j] = (i < kXsN && yy >= 0 && yy < G.h && xx >= 0 && xx < G.w) ? (float)__ldg(xi + yy * G.w + xx) * (1.f / 64.f)
                                                                          : 0.f;
    }
}

// Stage the counts and compute the tile's patch: conv1 for channels
// 4w .. 4w+3 in warp w, of patch pixels lane, lane + 32, ...; 8 bytes into
// chunk w / 2 at byte offset (w % 2) * 8.  All threads of the CTA call this.
__device__ __forceinline__ void compute_patch(const ConvTcGeom &G, int tile, int tiles_per_img, int tiles_x,
                                              uint8_t *Ps, float *xs, const float (&xr)[kXsPer],
                                              const float (&w4)[36], const float (&b4)[4]) {
    constexpr int S = 2, QPP = 2, PR = Patch<2>::PR, PC = Patch<2>::PC, HC = Patch<2>::HC;
    constexpr int XW = PC + 2;
    const int tid = threadIdx.x, lane = tid & 31, cg = tid >> 5;
    const int img = tile / tiles_per_img, t = tile - img * tiles_per_img;
    const int iy0 = (t / tiles_x) * kTileH * S - 1, ix0 = (t % tiles_x) * kTileW * S - 1;
    (void)img;
    __syncthreads();   // xs is free (the previous patch is written)
#pragma unroll
    for (int j = 0; j < kXsPer; ++j) {
        const int i = tid + j * kTcThreads;
        if (i < kXsN) xs[i] = xr[j];
    }
    __syncthreads();
    for (int p = lane; p < PR * PC; p += 32) {
        const int pr = p / PC, pc = p - pr * PC;
        const int yy = iy0 + pr, xx = ix0 + pc;
        uint32_t o0 = 0u, o1 = 0u;
        if (yy >= 0 && yy < G.h && xx >= 0 && xx < G.w) {
            float v[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] = xs[(pr + k / 3) * XW + pc + k % 3];
            float a[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float acc = b4[c];
#pragma unroll
                for (int k = 0; k < 9; ++k) acc = __fmaf_rn(w4[c * 9 + k], v[k], acc);
                a[c] = fmaxf(acc, 0.f);
            }
            o0 = to_bf16x2(a[0], a[1]);
            o1 = to_bf16x2(a[2], a[3]);
        }
        *reinterpret_cast<uint2 *>(Ps + (((pr * QPP + (cg >> 1)) * S + pc % S) * HC + pc / S) * 16 + (cg & 1) * 8) =
            make_uint2(o0, o1);
    }
}

// Persistent: CTA c takes tiles c, c + gridDim.x, ...; the next tile's
// operands are prepared (copied, or with FUSE1 computed) while the current
// one is multiplied and written (2 stages).
template <int CIN, int S, bool FUSE1>
__global__ void __launch_bounds__(kTcThreads, 4) conv_fwd_tc_kernel(const bf16 *x, ConvTcGeom G, const bf16 *wt,
                                                                const float *bias, bf16 *y, Conv1Params C1) {
    constexpr int K = 9 * CIN, QPP = CIN / 8;
    constexpr int HC = Patch<S>::HC;
    constexpr int P_BYTES = (Patch<S>::PR * QPP * S * HC * 16 + 1023) / 1024 * 1024;
    constexpr int B_BYTES = (kTcN * K * 2 + 1023) / 1024 * 1024, STAGE = P_BYTES;
    constexpr uint32_t ROW = QPP * S * HC * 16;   // bytes per patch row
    extern __shared__ __align__(1024) uint8_t smem[];   // B (the weights), then 2 patch stages
    uint8_t *const Bs = smem, *const stages = smem + B_BYTES;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_s;
    __shared__ float bias_s[kTcN];
    __shared__ float xs[FUSE1 ? kXsN : 1];
    float w4[36], b4[4];   // FUSE1: conv1 weights and biases of this warp's 4 channels
    float xr[kXsPer];      // FUSE1: the next tile's counts in flight
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (G.ow + kTileW - 1) / kTileW;
    const int tiles_per_img = ((G.oh + kTileH - 1) / kTileH) * tiles_x;
    const int n_tiles = G.n * tiles_per_img;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < kTcN) bias_s[tid] = bias[tid];

    int tile = blockIdx.x;
    if (FUSE1) {
#pragma unroll
        for (int i = 0; i < 36; ++i) w4[i] = __bfloat162float(C1.w1[(warp * 4) * 9 + i]);
#pragma unroll
        for (int c = 0; c < 4; ++c) b4[c] = C1.b1[warp * 4 + c];
        // the weights, then the first tile's patch
        constexpr int KC = K / 8;
        for (int i = tid; i < kTcN * KC; i += kTcThreads) {
            const int kc = i % KC, n = i / KC;
            cp_async16(saddr(Bs + ((kc * (kTcN / 8) + (n >> 3)) * 8 + (n & 7)) * 16), wt + (int64_t)n * K + kc * 8,
                       16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (tile < n_tiles) {
            load_counts(C1, G, tile, tiles_per_img, tiles_x, xr);
            compute_patch(G, tile, tiles_per_img, tiles_x, stages, xs, xr, w4, b4);
        }
    } else if (tile < n_tiles) {
        load_tile<CIN, S>(x, G, wt, tile, tiles_per_img, tiles_x, stages, Bs, true);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    bool fault = false;
    for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {   // block-uniform
        const int st = it & 1;
        uint8_t *Ps = stages + st * STAGE;
        const int next = tile + gridDim.x;
        if (!FUSE1) {
            if (next < n_tiles) {
                uint8_t *Pn = stages + (st ^ 1) * STAGE;
                load_tile<CIN, S>(x, G, wt, next, tiles_per_img, tiles_x, Pn, Bs, false);
                asm volatile("cp.async.wait_group 1;" ::: "memory");   // this tile's copies are done
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // smem writes -> tensor core (async proxy)
        __syncthreads();
        if (tid == 0) {
            const uint32_t p0 = saddr(Ps), b0 = saddr(Bs);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap % 3;
#pragma unroll
                for (int qq = 0; qq < QPP; qq += 2) {
                    const uint32_t a_off = (uint32_t)((((ky * QPP + qq) * S + kx % S) * HC + kx / S) * 16);
                    const uint64_t da = mat_desc(p0 + a_off, S * HC * 16, S * ROW);
                    const uint64_t db = mat_desc(b0 + (uint32_t)(tap * QPP + qq) * (kTcN * 16), kTcN * 16, 128);
                    const uint32_t accumulate = (tap > 0 || qq > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr(&bar))
                         : "memory");
        }
        // the next tile's counts are fetched while the tensor core works on
        // this one (its patch is computed after the epilogue)
        if (FUSE1 && next < n_tiles) load_counts(C1, G, next, tiles_per_img, tiles_x, xr);
        const bool done = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
        const bool all_done = __syncthreads_and(done ? 1 : 0) != 0;   // block-uniform
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!all_done) {
            fault = true;
            break;
        }
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int img = tile / tiles_per_img, t = tile - img * tiles_per_img;
        const int m = warp * 32 + lane;
        const int oy = (t / tiles_x) * kTileH + (m >> 3), ox = (t % tiles_x) * kTileW + (m & 7);
        if (oy < G.oh && ox < G.ow) {
            uint32_t o[16];
#pragma unroll
            for (int c = 0; c < 16; ++c)
                o[c] = to_bf16x2(fmaxf(__uint_as_float(r[2 * c]) + bias_s[2 * c], 0.f),
                                 fmaxf(__uint_as_float(r[2 * c + 1]) + bias_s[2 * c + 1], 0.f));
            uint4 *dst = reinterpret_cast<uint4 *>(y + (((int64_t)img * G.oh + oy) * G.ow + ox) * kTcN);
            dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
            dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
            dst[2] = make_uint4(o[8], o[9], o[10], o[11]);
            dst[3] = make_uint4(o[12], o[13], o[14], o[15]);
        }
        if (FUSE1 && next < n_tiles)   // block-uniform
            compute_patch(G, next, tiles_per_img, tiles_x, stages + (st ^ 1) * STAGE, xs, xr, w4, b4);
        // the accumulator is read and this stage's operands are used before
        // the next MMA or the next copies into this stage
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (fault) {
        if (tid == 0) atomicOr(&g_conv_faults, 1);
        asm volatile("cp.async.wait_group 0;" ::: "memory");   // own copies in flight
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int CIN, int S, bool FUSE1>
cudaError_t launch_tc(const bf16 *x, const ConvTcGeom &G, const bf16 *w, const float *b, bf16 *y,
                      const Conv1Params &C1, cudaStream_t s) {
    constexpr int QPP = CIN / 8;
    constexpr int P_BYTES = (Patch<S>::PR * QPP * S * Patch<S>::HC * 16 + 1023) / 1024 * 1024;
    constexpr int smem = (kTcN * 9 * CIN * 2 + 1023) / 1024 * 1024 + 2 * P_BYTES;
    auto kern = conv_fwd_tc_kernel<CIN, S, FUSE1>;
    // once per device: the attributes, and the grid limit (SMs x CTAs per SM)
    static std::atomic<uint64_t> done{0};
    static std::atomic<int> grid_max[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int limit = dev < 64 ? grid_max[dev].load(std::memory_order_acquire) : 0;
    e = once_per_device(done, [&](int d) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (r == cudaSuccess)   // as much shared memory as possible: several CTAs per SM
            r = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        int sms = 0, sm_smem = 0, reserved = 0;
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, d);
        // CTAs per SM by shared memory (dynamic + static + the per-block
        // reservation) and by registers, at most 512 / 32 by tensor memory
        cudaFuncAttributes fa;
        if (r == cudaSuccess) r = cudaFuncGetAttributes(&fa, kern);
        if (r != cudaSuccess) return r;
        int per_sm = sm_smem / (smem + (int)fa.sharedSizeBytes + reserved);
        const int per_sm_regs = 65536 / (kTcThreads * ((fa.numRegs + 7) / 8 * 8));
        if (per_sm_regs < per_sm) per_sm = per_sm_regs;
        if (per_sm < 1) per_sm = 1;
        if (per_sm * kTmemCols > 512) per_sm = 512 / kTmemCols;
        limit = sms * per_sm;
        if (d < 64) grid_max[d].store(limit, std::memory_order_release);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    if (limit <= 0 && dev < 64) limit = grid_max[dev].load(std::memory_order_acquire);
    if (limit <= 0) return cudaErrorInvalidValue;
    const int tiles = G.n * ((G.oh + kTileH - 1) / kTileH) * ((G.ow + kTileW - 1) / kTileW);
    const int grid = tiles < limit ? tiles : limit;
    kern<<<grid, kTcThreads, smem, s>>>(x, G, w, b, y, C1);
    return cudaGetLastError();
}


// ------------------------------------------------------------------ backward

// Instruction descriptor (kind::f16) for M = 128 and N columns: D fp32, A and
// B bf16, both K-major.
__host__ __device__ constexpr uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// Offset of the 16-byte chunk (K chunk kc, row r) in a K-major operand of
// `rows` rows (unswizzled core matrices of 8 rows x 16 bytes: the rows of a
// core matrix 16 bytes apart, row groups 128 bytes apart (SBO), K chunks
// rows * 16 bytes apart (LBO)).
__device__ __forceinline__ uint32_t kmaj(int kc, int r, int rows) {
    return (uint32_t)(((kc * (rows >> 3) + (r >> 3)) * 8 + (r & 7)) * 16);
}

// ReLU gradient mask of 8 bf16 gradients by the stored outputs (> 0: bits != 0).
__device__ __forceinline__ uint4 relu_mask8(uint4 d, uint4 o) {
    auto m2 = [](uint32_t dw, uint32_t ow) {
        return dw & (((ow & 0xFFFFu) ? 0xFFFFu : 0u) | ((ow >> 16) ? 0xFFFF0000u : 0u));
    };
    return make_uint4(m2(d.x, o.x), m2(d.y, o.y), m2(d.z, o.z), m2(d.w, o.w));
}

// Transpose of an 8 x 8 block of bf16: W[i] holds 8 channels of pixel i;
// returns in out[c] the 8 pixels of channel c (pixel 2k in the low half of
// word k).
__device__ __forceinline__ void transpose8(const uint4 (&W)[8], uint4 (&out)[8]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t sel = (c & 1) ? 0x7632u : 0x5410u;
        uint32_t v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint4 &q = W[i];
            v[i] = (c >> 1) == 0 ? q.x : (c >> 1) == 1 ? q.y : (c >> 1) == 2 ? q.z : q.w;
        }
        out[c] = make_uint4(__byte_perm(v[0], v[1], sel), __byte_perm(v[2], v[3], sel), __byte_perm(v[4], v[5], sel),
                            __byte_perm(v[6], v[7], sel));
    }
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Weight gradient, per CTA a chunk of one image's output pixels (K = pixels):
//   D[(tap, ci)][co] = sum_p x[pix(p, tap)][ci] dz[p][co],  dz = dy masked by
// the ReLU, i.e. dw transposed, plus a row of ones whose D row is the bias
// gradient sum_p dz[p][co].  M = 9 CIN + 1 rows in tiles of 128 (2 or 3
// tensor-memory accumulators of 32 columns), N = 32, K blocks of 64 pixels:
// the block's x values per tap and its dz are transposed into K-major
// operands (8 x 8 blocks through registers), then one thread issues the
// tiles' MMAs and commits; the next block is staged after a bounded wait.
// The CTA's partial sums go to part[cta][co * 9 CIN + (tap, ci)] and
// part_b[cta][co], summed over CTAs in a fixed order (reduce_parts).
constexpr int kWgKB = 64;
template <int CIN>
__global__ void __launch_bounds__(kTcThreads, 1) conv_wgrad_tc_kernel(const bf16 *x, const bf16 *y, const bf16 *dy,
                                                                   ConvTcGeom G, int chunk, float *part,
                                                                   float *part_b) {
    constexpr int KW = 9 * CIN, QPP = CIN / 8;
    constexpr int MT = (KW + 1 + kTcM - 1) / kTcM;
    constexpr int A_TILE = kTcM * kWgKB * 2;
    constexpr uint32_t IDESC = idesc_n(32);
    extern __shared__ __align__(1024) uint8_t smem[];   // MT A tiles, then B
    uint8_t *const As = smem, *const Bs = smem + MT * A_TILE;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_s;
    __shared__ int pix_s[kWgKB];   // (oy << 16 | ox) of the block's pixels, -1 past the chunk
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_s)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // rows past the ones row stay zero; the ones row (bf16 1.0) is written once
    for (int i = tid; i < MT * A_TILE / 16; i += kTcThreads) reinterpret_cast<uint4 *>(As)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (tid < kWgKB / 8)
        *reinterpret_cast<uint4 *>(As + (KW / kTcM) * A_TILE + kmaj(tid, KW % kTcM, kTcM)) =
            make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    const int Mi = G.oh * G.ow, img = blockIdx.y;
    const int p_begin = blockIdx.x * chunk, p_end = min(Mi, p_begin + chunk);
    const bf16 *xi = x + (int64_t)img * G.h * G.w * CIN;
    const int64_t zbase = (int64_t)img * Mi * 32;
    bool fault = false;
    int it = 0;
    for (int k0 = p_begin; k0 < p_end; k0 += kWgKB, ++it) {   // block-uniform
        if (tid < kWgKB) {
            const int p = k0 + tid;
            pix_s[tid] = p < p_end ? ((p / G.ow) << 16 | (p % G.ow)) : -1;
        }
        __syncthreads();
        // B: dz of the block, 8 pixels x 8 channels per thread
        if (tid < 32) {
            const int pg = tid >> 2, cg = tid & 3;
            uint4 W[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                W[i] = make_uint4(0u, 0u, 0u, 0u);
                if (pix_s[pg * 8 + i] >= 0) {
                    const int64_t off = zbase + (int64_t)(k0 + pg * 8 + i) * 32 + cg * 8;
                    W[i] = relu_mask8(__ldg(reinterpret_cast<const uint4 *>(dy + off)),
                                      __ldg(reinterpret_cast<const uint4 *>(y + off)));
                }
            }
            uint4 T[8];
            transpose8(W, T);
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4 *>(Bs + kmaj(pg, cg * 8 + c, 32)) = T[c];
        }
        // A: x of the block per tap, 8 pixels x 8 channels per thread and step
        for (int b = tid; b < 9 * QPP * 8; b += kTcThreads) {
            const int pg = b & 7, rest = b >> 3, cg = rest % QPP, tap = rest / QPP;
            const int ky = tap / 3, kx = tap % 3;
            uint4 W[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                W[i] = make_uint4(0u, 0u, 0u, 0u);
                const int pp = pix_s[pg * 8 + i];
                if (pp >= 0) {
                    const int iy = G.stride * (pp >> 16) + ky - 1, ix = G.stride * (pp & 0xFFFF) + kx - 1;
                    if (iy >= 0 && iy < G.h && ix >= 0 && ix < G.w)
                        W[i] = __ldg(reinterpret_cast<const uint4 *>(xi + ((int64_t)iy * G.w + ix) * CIN + cg * 8));
                }
            }
            uint4 T[8];
            transpose8(W, T);
            const int m0 = tap * CIN + cg * 8;   // 8 rows of one core matrix
#pragma unroll
            for (int c = 0; c < 8; ++c)
                *reinterpret_cast<uint4 *>(As + (m0 / kTcM) * A_TILE + kmaj(pg, (m0 % kTcM) + c, kTcM)) = T[c];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // smem writes -> tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = saddr(As), b0 = saddr(Bs);
#pragma unroll
            for (int t = 0; t < MT; ++t)
#pragma unroll
                for (int j = 0; j < kWgKB / 16; ++j)
                    mma_f16(tmem + (uint32_t)(t * 32), mat_desc(a0 + t * A_TILE + (2 * j) * (kTcM * 16), kTcM * 16, 128),
                            mat_desc(b0 + (2 * j) * (32 * 16), 32 * 16, 128), IDESC, (it > 0 || j > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr(&bar))
                         : "memory");
        }
        const bool done = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
        const bool all_done = __syncthreads_and(done ? 1 : 0) != 0;   // block-uniform
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!all_done) {
            fault = true;
            break;
        }
    }
    if (!fault && it > 0) {
        const int cta = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll 1
        for (int t = 0; t < MT; ++t) {
            uint32_t r[32];
            tmem_ld32(tmem + (uint32_t)(t * 32) + ((uint32_t)(warp * 32) << 16), r);
            const int m = t * kTcM + warp * 32 + lane;
            if (m < KW) {
                float *pc = part + (int64_t)cta * (32 * KW) + m;
#pragma unroll
                for (int co = 0; co < 32; ++co) pc[co * KW] = __uint_as_float(r[co]);
            } else if (m == KW) {
#pragma unroll
                for (int co = 0; co < 32; ++co) part_b[(int64_t)cta * 32 + co] = __uint_as_float(r[co]);
            }
        }
    }
    if (fault && tid == 0) atomicOr(&g_conv_faults, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
}

// Input gradient:
//   dx[q][ci] = sum over (tap, co) of dz[o(q, tap)][co] w[co][tap][ci],
// o(q, tap) the output pixel whose tap reads input pixel q.  With stride 2 a
// tap reads q only if it matches q's parity: ky = 1 for even rows, ky = 0 or
// 2 for odd ones (and so for x), so the input pixels fall into 4 parity
// classes with 1, 2, 2 and 4 taps (stride 1: one class, 9 taps).  A CTA tile
// is 128 input pixels of one class of one image (persistent CTAs), so K =
// taps x 32 only: M = 128, N = CIN, 2 MMAs of K = 16 per tap.  A is dz
// gathered per (pixel, tap) in K-major chunks of 8 channels (no transpose:
// channels are contiguous); B is the weights transposed once per CTA for all
// 9 taps, and each MMA points at its tap's chunks.  The accumulator is read
// with tcgen05.ld and stored as bf16 NHWC.
struct DgClass {
    int py, px, ny, nx, ntap, tiles;
};

// Tap (ky * 3 + kx) of slot `slot` of a class: stride 1, every tap in order;
// stride 2, ky = 1 (even rows) or 0, 2 (odd rows), and so for x.
__device__ __forceinline__ int dg_tap(const DgClass &k, int slot, int stride) {
    if (stride != 2) return slot;
    const int nkx = k.px ? 2 : 1, a = slot / nkx, b = slot - a * nkx;
    return (k.py ? 2 * a : 1) * 3 + (k.px ? 2 * b : 1);
}

__device__ __forceinline__ DgClass dg_class(const ConvTcGeom &G, int c) {
    DgClass k;
    const int S = G.stride;
    k.py = S == 2 ? c >> 1 : 0;
    k.px = S == 2 ? c & 1 : 0;
    k.ny = S == 2 ? (G.h - k.py + 1) >> 1 : G.h;
    k.nx = S == 2 ? (G.w - k.px + 1) >> 1 : G.w;
    k.tiles = (k.ny * k.nx + kTcM - 1) / kTcM;
    k.ntap = S == 2 ? (k.py ? 2 : 1) * (k.px ? 2 : 1) : 9;
    return k;
}

template <int CIN>
__global__ void __launch_bounds__(kTcThreads, 1) conv_dgrad_tc_kernel(const bf16 *y, const bf16 *dy, ConvTcGeom G,
                                                                   const bf16 *wt, bf16 *dx) {
    constexpr int KCH = 9 * 32 / 8;   // K chunks (tap, 8 output channels) of all taps
    constexpr int B_BYTES = CIN * KCH * 16;
    constexpr uint32_t IDESC = idesc_n(CIN);
    extern __shared__ __align__(1024) uint8_t smem[];   // B, then A (at most 9 taps)
    uint8_t *const Bs = smem, *const As = smem + (B_BYTES + 1023) / 1024 * 1024;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B[ci][(tap, co)] = w[co][tap][ci]
    for (int b = tid; b < KCH * CIN; b += kTcThreads) {
        const int ci = b % CIN, kc = b / CIN, tap = kc >> 2, cg = kc & 3;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t lo = *reinterpret_cast<const unsigned short *>(wt + ((cg * 8 + 2 * k) * 9 + tap) * CIN + ci);
            const uint32_t hi =
                *reinterpret_cast<const unsigned short *>(wt + ((cg * 8 + 2 * k + 1) * 9 + tap) * CIN + ci);
            v[k] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4 *>(Bs + kmaj(kc, ci, CIN)) = make_uint4(v[0], v[1], v[2], v[3]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    const int n_cls = G.stride == 2 ? 4 : 1;
    int tiles_img = 0;
    for (int c = 0; c < n_cls; ++c) tiles_img += dg_class(G, c).tiles;
    const int n_tiles = G.n * tiles_img;
    bool fault = false;
    int it = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {   // block-uniform
        const int img = tile / tiles_img;
        int r = tile - img * tiles_img, c = 0;
        DgClass K = dg_class(G, 0);
        while (r >= K.tiles) {
            r -= K.tiles;
            K = dg_class(G, ++c);
        }
        const int s0 = r * kTcM, npts = K.ny * K.nx;
        const int64_t zbase = (int64_t)img * G.oh * G.ow * 32;
        // A[q][(slot, co)]: thread b takes chunk (slot, row q, 8 channels cg); 4 threads per pixel
        for (int b = tid; b < K.ntap * 4 * kTcM; b += kTcThreads) {
            const int cg = b & 3, q = (b >> 2) & (kTcM - 1), slot = b >> 9;
            const int tap = dg_tap(K, slot, G.stride);
            const int sidx = s0 + q;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (sidx < npts) {
                const int i = sidx / K.nx, j = sidx - i * K.nx;
                const int qy = K.py + G.stride * i, qx = K.px + G.stride * j;
                const int ny = qy + 1 - tap / 3, nx = qx + 1 - tap % 3;   // divisible by the stride (class)
                if (ny >= 0 && nx >= 0) {
                    const int oy = ny / G.stride, ox = nx / G.stride;
                    if (oy < G.oh && ox < G.ow) {
                        const int64_t off = zbase + ((int64_t)oy * G.ow + ox) * 32 + cg * 8;
                        v = relu_mask8(__ldg(reinterpret_cast<const uint4 *>(dy + off)),
                                       __ldg(reinterpret_cast<const uint4 *>(y + off)));
                    }
                }
            }
            *reinterpret_cast<uint4 *>(As + kmaj(slot * 4 + cg, q, kTcM)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = saddr(As), b0 = saddr(Bs);
            for (int slot = 0; slot < K.ntap; ++slot) {
                const int tap = dg_tap(K, slot, G.stride);
#pragma unroll
                for (int m = 0; m < 2; ++m)
                    mma_f16(tmem, mat_desc(a0 + (slot * 4 + 2 * m) * (kTcM * 16), kTcM * 16, 128),
                            mat_desc(b0 + (tap * 4 + 2 * m) * (CIN * 16), CIN * 16, 128), IDESC,
                            (slot > 0 || m > 0) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             saddr(&bar))
                         : "memory");
        }
        const bool done = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
        const bool all_done = __syncthreads_and(done ? 1 : 0) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!all_done) {
            fault = true;
            break;
        }
        uint32_t rr[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), rr);   // CIN < 32: the upper columns are unused
        const int sidx = s0 + warp * 32 + lane;
        if (sidx < npts) {
            const int i = sidx / K.nx, j = sidx - i * K.nx;
            const int qy = K.py + G.stride * i, qx = K.px + G.stride * j;
            uint4 *dst = reinterpret_cast<uint4 *>(dx + (((int64_t)img * G.h + qy) * G.w + qx) * CIN);
#pragma unroll
            for (int c8 = 0; c8 < CIN / 8; ++c8)
                dst[c8] = make_uint4(to_bf16x2(__uint_as_float(rr[8 * c8]), __uint_as_float(rr[8 * c8 + 1])),
                                     to_bf16x2(__uint_as_float(rr[8 * c8 + 2]), __uint_as_float(rr[8 * c8 + 3])),
                                     to_bf16x2(__uint_as_float(rr[8 * c8 + 4]), __uint_as_float(rr[8 * c8 + 5])),
                                     to_bf16x2(__uint_as_float(rr[8 * c8 + 6]), __uint_as_float(rr[8 * c8 + 7])));
        }
        // the accumulator is read and A is consumed before the next tile's staging and MMAs
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (fault && tid == 0) atomicOr(&g_conv_faults, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int CIN>
int wgrad_smem() {
    constexpr int MT = (9 * CIN + 1 + kTcM - 1) / kTcM;
    constexpr int need = MT * kTcM * kWgKB * 2 + 32 * kWgKB * 2;
    return need > 56 * 1024 ? need : 56 * 1024;
}
template <int CIN>
int dgrad_smem() {
    return (CIN * 36 * 16 + 1023) / 1024 * 1024 + kTcM * 36 * 16;
}

}  // namespace

cudaError_t launch_conv_fwd_tc(const void *x, const ConvTcGeom &G, int cin, const void *w, const float *b, void *y,
                               cudaStream_t s) {
    const Conv1Params none{nullptr, nullptr, nullptr};
    if (G.stride == 2) {
        if (cin == 16) return launch_tc<16, 2, false>((const bf16 *)x, G, (const bf16 *)w, b, (bf16 *)y, none, s);
        if (cin == 32) return launch_tc<32, 2, false>((const bf16 *)x, G, (const bf16 *)w, b, (bf16 *)y, none, s);
    } else if (G.stride == 1) {
        if (cin == 16) return launch_tc<16, 1, false>((const bf16 *)x, G, (const bf16 *)w, b, (bf16 *)y, none, s);
        if (cin == 32) return launch_tc<32, 1, false>((const bf16 *)x, G, (const bf16 *)w, b, (bf16 *)y, none, s);
    }
    return cudaErrorInvalidValue;
}

// Grid limit of a kernel: SMs x CTAs per SM by shared memory (and the
// per-block reservation) and by tensor-memory columns.
static cudaError_t grid_limit(const void *kern, int smem, int tmem_cols, int *limit) {
    int dev = 0, sms = 0, sm_smem = 0, reserved = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa;
    if (r == cudaSuccess) r = cudaFuncGetAttributes(&fa, kern);
    if (r != cudaSuccess) return r;
    int per_sm = sm_smem / (smem + (int)fa.sharedSizeBytes + reserved);
    if (per_sm * tmem_cols > 512) per_sm = 512 / tmem_cols;
    if (per_sm < 1) per_sm = 1;
    *limit = sms * per_sm;
    return cudaSuccess;
}

cudaError_t launch_conv_wgrad_tc(const void *x, const void *y, const void *dy, const ConvTcGeom &G, int cin,
                                 int chunk, float *part, float *part_b, cudaStream_t s) {
    if ((cin != 16 && cin != 32) || chunk < 1) return cudaErrorInvalidValue;
    const dim3 grid((G.oh * G.ow + chunk - 1) / chunk, G.n);
    static std::atomic<uint64_t> done16{0}, done32{0};
    if (cin == 16) {
        auto kern = conv_wgrad_tc_kernel<16>;
        const int smem = wgrad_smem<16>();
        cudaError_t e = once_per_device(done16, [&](int) {
            return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        });
        if (e != cudaSuccess) return e;
        kern<<<grid, kTcThreads, smem, s>>>((const bf16 *)x, (const bf16 *)y, (const bf16 *)dy, G, chunk, part, part_b);
    } else {
        auto kern = conv_wgrad_tc_kernel<32>;
        const int smem = wgrad_smem<32>();
        cudaError_t e = once_per_device(done32, [&](int) {
            return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        });
        if (e != cudaSuccess) return e;
        kern<<<grid, kTcThreads, smem, s>>>((const bf16 *)x, (const bf16 *)y, (const bf16 *)dy, G, chunk, part, part_b);
    }
    return cudaGetLastError();
}

cudaError_t launch_conv_dgrad_tc(const void *y, const void *dy, const ConvTcGeom &G, int cin, const void *w, void *dx,
                                 cudaStream_t s) {
    if (cin != 16 && cin != 32) return cudaErrorInvalidValue;
    int tiles = 0;   // per image: the parity classes' tiles (stride 2), else ceil(h w / 128)
    if (G.stride == 2) {
        for (int c = 0; c < 4; ++c) {
            const int ny = (G.h - (c >> 1) + 1) >> 1, nx = (G.w - (c & 1) + 1) >> 1;
            tiles += (ny * nx + kTcM - 1) / kTcM;
        }
    } else {
        tiles = (G.h * G.w + kTcM - 1) / kTcM;
    }
    tiles *= G.n;
    static std::atomic<uint64_t> done16{0}, done32{0};
    static std::atomic<int> lim16[64], lim32[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidValue;
    if (cin == 16) {
        auto kern = conv_dgrad_tc_kernel<16>;
        const int smem = dgrad_smem<16>();
        e = once_per_device(done16, [&](int d) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            int lim = 0;
            if (r == cudaSuccess) r = grid_limit((const void *)kern, smem, kTmemCols, &lim);
            if (r == cudaSuccess) lim16[d].store(lim, std::memory_order_release);
            return r;
        });
        if (e != cudaSuccess) return e;
        const int lim = lim16[dev].load(std::memory_order_acquire);
        if (lim <= 0) return cudaErrorInvalidValue;
        kern<<<tiles < lim ? tiles : lim, kTcThreads, smem, s>>>((const bf16 *)y, (const bf16 *)dy, G,
                                                                  (const bf16 *)w, (bf16 *)dx);
    } else {
        auto kern = conv_dgrad_tc_kernel<32>;
        const int smem = dgrad_smem<32>();
        e = once_per_device(done32, [&](int d) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            int lim = 0;
            if (r == cudaSuccess) r = grid_limit((const void *)kern, smem, kTmemCols, &lim);
            if (r == cudaSuccess) lim32[d].store(lim, std::memory_order_release);
            return r;
        });
        if (e != cudaSuccess) return e;
        const int lim = lim32[dev].load(std::memory_order_acquire);
        if (lim <= 0) return cudaErrorInvalidValue;
        kern<<<tiles < lim ? tiles : lim, kTcThreads, smem, s>>>((const bf16 *)y, (const bf16 *)dy, G,
                                                                  (const bf16 *)w, (bf16 *)dx);
    }
    return cudaGetLastError();
}

cudaError_t launch_conv12_fused_tc(const uint8_t *x0, const ConvTcGeom &G, const void *w1, const float *b1,
                                   const void *w2, const float *b2, void *y2, cudaStream_t s) {
    if (G.stride != 2) return cudaErrorInvalidValue;
    const Conv1Params C1{x0, (const bf16 *)w1, b1};
    return launch_tc<16, 2, true>((const bf16 *)w2, G, (const bf16 *)w2, b2, (bf16 *)y2, C1, s);
}

}  // namespace ld

extern "C" ld_status ld_conv_faults(int32_t device, int32_t *flags) {
    if (!flags) {
        ld::set_last_error("ld_conv_faults: NULL flags");
        return LD_ERR_INVALID;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    int32_t v = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, ld::g_conv_faults, sizeof v);
    const int32_t zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(ld::g_conv_faults, &zero, sizeof zero);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        ld::set_last_error(cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    *flags = v;
    return LD_OK;
}
