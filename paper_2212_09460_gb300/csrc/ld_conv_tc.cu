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
