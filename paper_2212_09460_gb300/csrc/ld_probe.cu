// ld_probe.cu -- the measured ceiling of Step 3's voting: the rate at which
// one GPU performs 32-lane shared-memory reductions (red.shared.add.u32),
// with every lane of a warp on its own bank (the bank roofline the voting
// kernels are reported against) and with random words (what 32 unrelated
// votes cost).  Not part of the lane-detection path.
#include "ld_internal.cuh"

namespace ld {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeWords = 4096;   // 16 KB of counters per CTA

// pattern 0: lane l of warp w adds to word w * 32 + l (+ a stride of 1024
// words per step), so the 32 lanes of an instruction hit 32 distinct banks.
// pattern 1: each lane adds to a pseudo-random word (xorshift32) of the
// 4096-word array.  `iters` reductions per thread; the sum of the array goes
// to sink[blockIdx.x] so that the work is observable.
__global__ void __launch_bounds__(kProbeThreads) smem_red_probe_kernel(int iters, int pattern, uint32_t *sink) {
    __shared__ uint32_t buf[kProbeWords];
    const int tid = threadIdx.x;
    for (int i = tid; i < kProbeWords; i += kProbeThreads) buf[i] = 0u;
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    if (pattern == 0) {
        const uint32_t a0 = base + (uint32_t)tid * 4u;   // warp w, lane l: word 32 w + l
#pragma unroll 1
        for (int i = 0; i < iters; i += 8) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t a = a0 + (uint32_t)(((i + k) & 3) * kProbeThreads * 4) % (kProbeWords * 4);
                asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(1u) : "memory");
            }
        }
    } else {
        uint32_t x = 0x9E3779B9u * (uint32_t)(blockIdx.x * kProbeThreads + tid + 1);
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
            x ^= x << 13;
            x ^= x >> 17;
            x ^= x << 5;
            const uint32_t a = base + (x & (kProbeWords - 1)) * 4u;
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(1u) : "memory");
        }
    }
    __syncthreads();
    if (tid < 32) {
        uint32_t s = 0;
        for (int i = tid; i < kProbeWords; i += 32) s += buf[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (tid == 0) sink[blockIdx.x] = s;
    }
}

}  // namespace
}  // namespace ld

extern "C" ld_status ld_probe_smem_red(int32_t n_ctas, int32_t iters, int32_t pattern, uint32_t *d_sink,
                                       void *stream) {
    if (n_ctas < 1 || iters < 8 || (iters & 7) || (pattern != 0 && pattern != 1) || !d_sink) {
        ld::set_last_error("ld_probe_smem_red: need n_ctas >= 1, iters a positive multiple of 8, pattern 0 or 1");
        return LD_ERR_INVALID;
    }
    ld::smem_red_probe_kernel<<<n_ctas, ld::kProbeThreads, 0, (cudaStream_t)stream>>>(iters, pattern, d_sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ld::set_last_error(cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    return LD_OK;
}
