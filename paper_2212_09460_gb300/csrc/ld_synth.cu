// ld_synth.cu -- device-side generator of the seeded synthetic road frames
// (the stand-in workload for the paper's missing test image), producing the
// same bytes as the host generator in synth.py: every pixel is an integer
// function of the frame's descriptor and (x, y).  No step of the detection
// method is computed here; this only draws inputs (training frames for the
// proposal network, camera frames for the serving loop).
//
// Per pixel: background 40 + 80*y/(h-1); each stripe whose exact integer test
// |x*nx + y*ny - c| < 3*65536 (and dash phase) holds sets the stripe value;
// noise = floor(((sum of eight 16-bit fields of two SplitMix64 outputs) -
// 262140) * K / 2^32 + 1/2) with K the row's Q32 std scale; clamp to [0, 255];
// salt sets 255 where the low 32 bits of a third output are below the salt
// threshold.
#include "ld_internal.cuh"

namespace ld {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__global__ void __launch_bounds__(256) synth_kernel(const ld_synth_frame *fr, int n_frames) {
    const ld_synth_frame &F = fr[blockIdx.y];
    const int64_t npx = (int64_t)F.w * F.h;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / F.w, x = i - y * F.w;
        int64_t v = 40 + (80 * y) / (F.h > 1 ? F.h - 1 : 1);
        for (int k = 0; k < F.n_stripes; ++k) {
            const ld_synth_stripe &S = F.stripes[k];
            const int64_t d = x * S.nx + y * S.ny - S.c;
            bool in = (d < 0 ? -d : d) < 3 * 65536;
            if (in && S.dash > 0) {
                const int64_t t = (x * S.tx + y * S.ty - S.t0) >> 16;   // floor division by 65536
                const int64_t per = S.dash + S.gap;
                int64_t m = t % per;
                if (m < 0) m += per;
                in = m < S.dash;
            }
            if (in) v = S.value;
        }
        const uint64_t idx1 = (uint64_t)i + 1ull;
        const uint64_t a = mix64(F.base[0] + idx1 * kGamma);
        const uint64_t b = mix64(F.base[1] + idx1 * kGamma);
        int64_t s8 = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) s8 += (int64_t)((a >> (16 * k)) & 0xFFFFu) + (int64_t)((b >> (16 * k)) & 0xFFFFu);
        const int64_t nz = s8 - 262140;
        const int64_t kk = (y >= F.h / 2) ? F.k_road : F.k_top;
        v += (nz * kk + (1ll << 31)) >> 32;
        v = v < 0 ? 0 : (v > 255 ? 255 : v);
        if (F.salt_thr > 0) {
            const uint64_t c = mix64(F.base[2] + idx1 * kGamma);
            if ((c & 0xFFFFFFFFull) < F.salt_thr) v = 255;
        }
        F.img[y * F.pitch + x] = (uint8_t)v;
    }
}

}  // namespace
}  // namespace ld

extern "C" ld_status ld_synth_frames(const ld_synth_frame *d_frames, int32_t n, void *stream) {
    if (!d_frames || n < 1 || n > 65535) {
        ld::set_last_error("ld_synth_frames: need a device descriptor array and 1 <= n <= 65535");
        return LD_ERR_INVALID;
    }
    dim3 grid(148 * 4, n);
    ld::synth_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_frames, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ld::set_last_error(cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    return LD_OK;
}
