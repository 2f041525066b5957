// ld_cnn.cu -- kernels of the learned theta-band proposal network (the paper
// has no learned stage; this one predicts which 5-degree theta bands hold the
// top Hough peaks so that voting can skip the others).
//
// Network (NHWC activations, bf16 storage, fp32 accumulation):
//   conv1 3x3 s1 1->16 | conv2 3x3 s2 16->32 | conv3 3x3 s2 32->32 |
//   conv4 3x3 s2 32->32, each + bias + ReLU | adaptive average pool to 4x8 |
//   linear 1024 -> 44 logits (36 theta bands + 8 row bands) | BCE loss.
//
// conv2..4 are implicit GEMMs on the fifth-generation tensor cores (tcgen05,
// bf16 operands in shared memory, fp32 accumulators in tensor memory;
// ld_conv_tc.cu): the forward pass (M = output pixels, N = Cout, K = 9*Cin),
// the input gradient (M = input pixels, N = Cin, K = 9*Cout over the taps
// that read each pixel) and the weight gradient (M = (tap, Cin) plus a row
// of ones for the bias, N = Cout, K = pixels, split over CTAs into partial
// sums added in a fixed order).  conv1 has a single input channel (K = 9)
// and runs on the CUDA cores.  Every output of the
// forward pass depends only on its own sample, in a fixed summation order,
// so a frame's logits are the same alone and in any batch.
#include <cmath>
#include <cstdio>

#include <cuda_bf16.h>

#include "ld_internal.cuh"

namespace ld {
namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t bits16(const bf16 *p) {
    return (uint32_t) * reinterpret_cast<const unsigned short *>(p);
}
__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
// dy masked by the ReLU: keep the gradient where the stored output is > 0
// (ReLU outputs are +0 or positive, so "bits != 0" is "> 0").
__device__ __forceinline__ uint32_t relu_mask1(uint32_t dyb, uint32_t yb) { return yb ? dyb : 0u; }

// ------------------------------------------------------------------ conv1 (Cin = 1)

// y[p][16] = relu(b + sum_tap w[co][tap] * x[pix(p, tap)] / 64), x uint8 edge counts [n][h][w].
// Block 32 x 8 pixels of one image (grid x, y over the image, z = image).
__global__ void __launch_bounds__(256) conv1_fwd_kernel(const uint8_t *x, int h, int w, const bf16 *wt,
                                                       const float *b, bf16 *y) {
    __shared__ float ws[16 * 9], bs[16];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int i = tid; i < 16 * 9; i += 256) ws[i] = __bfloat162float(wt[i]);
    if (tid < 16) bs[tid] = b[tid];
    __syncthreads();
    const int ox = blockIdx.x * 32 + threadIdx.x, oy = blockIdx.y * 8 + threadIdx.y, img = blockIdx.z;
    if (ox >= w || oy >= h) return;
    const uint8_t *xi = x + (int64_t)img * h * w;
    float v[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int iy = oy + t / 3 - 1, ix = ox + t % 3 - 1;
        v[t] = (iy >= 0 && iy < h && ix >= 0 && ix < w) ? (float)xi[iy * w + ix] * (1.f / 64.f) : 0.f;
    }
    uint32_t out[8];
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
        float s0 = bs[c], s1 = bs[c + 1];
#pragma unroll
        for (int t = 0; t < 9; ++t) {   // explicit fused multiply-adds: the fused inference path repeats them
            s0 = __fmaf_rn(ws[c * 9 + t], v[t], s0);
            s1 = __fmaf_rn(ws[(c + 1) * 9 + t], v[t], s1);
        }
        out[c / 2] = to_bf16x2(fmaxf(s0, 0.f), fmaxf(s1, 0.f));
    }
    uint4 *dst = reinterpret_cast<uint4 *>(y + (((int64_t)img * h + oy) * w + ox) * 16);
    dst[0] = make_uint4(out[0], out[1], out[2], out[3]);
    dst[1] = make_uint4(out[4], out[5], out[6], out[7]);
}

// Partial sums of dw1[co][tap] = sum_p dy_pre[p][co] * x[pix(p, tap)] and
// db1[co] = sum_p dy_pre[p][co] over this block's pixels: part[block][co * 10
// + tap] (tap 9 = bias).  Block: 16 channels x 16 pixel lanes.
__global__ void __launch_bounds__(256) conv1_wgrad_kernel(const uint8_t *x, const bf16 *y, const bf16 *dy, int n,
                                                         int h, int w, float *part) {
    const int co = threadIdx.x & 15, lane = threadIdx.x >> 4;
    float acc[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) acc[t] = 0.f;
    const int64_t P = (int64_t)n * h * w;
    for (int64_t p = (int64_t)blockIdx.x * 16 + lane; p < P; p += (int64_t)gridDim.x * 16) {
        const float g = __uint_as_float(relu_mask1(bits16(dy + p * 16 + co), bits16(y + p * 16 + co)) << 16);
        if (g == 0.f) continue;
        const int img = (int)(p / ((int64_t)h * w));
        const int rem = (int)(p - (int64_t)img * h * w);
        const int oy = rem / w, ox = rem - (rem / w) * w;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int iy = oy + t / 3 - 1, ix = ox + t % 3 - 1;
            if (iy >= 0 && iy < h && ix >= 0 && ix < w)
                acc[t] += g * ((float)x[((int64_t)img * h + iy) * w + ix] * (1.f / 64.f));
        }
        acc[9] += g;
    }
    __shared__ float red[16][16][10];
#pragma unroll
    for (int t = 0; t < 10; ++t) red[lane][co][t] = acc[t];
    __syncthreads();
    if (threadIdx.x < 160) {
        const int c = threadIdx.x / 10, t = threadIdx.x % 10;
        float s = 0.f;
        for (int l = 0; l < 16; ++l) s += red[l][c][t];
        part[(int64_t)blockIdx.x * 160 + c * 10 + t] = s;
    }
}

// ------------------------------------------------------------------ conv2..4 on tensor cores

// Geometry of one layer (the forward and backward kernels are in ld_conv_tc.cu).
struct ConvGeom {
    int n, h, w, oh, ow, stride;
};

// out[i] += sum over r < rows of part[r][i], in order (one thread per i).
__global__ void __launch_bounds__(256) reduce_parts(const float *part, int rows, int cols, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += part[(int64_t)r * cols + i];
    out[i] += s;
}
// out[c * 9 + t] += ..., outb[c] += ... from conv1's [rows][16 * 10] partials.
__global__ void __launch_bounds__(160) reduce_parts1(const float *part, int rows, float *dw, float *db) {
    const int i = threadIdx.x, c = i / 10, t = i % 10;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += part[(int64_t)r * 160 + i];
    if (t < 9) dw[c * 9 + t] += s;
    else db[c] += s;
}

// ------------------------------------------------------------------ pool + head

constexpr int kPH = 4, kPW = 8, kC4 = 32, kFeat = kPH * kPW * kC4, kOut = 44;

__device__ __forceinline__ int bin_lo(int i, int n_in, int n_out) { return i * n_in / n_out; }
__device__ __forceinline__ int bin_hi(int i, int n_in, int n_out) { return ((i + 1) * n_in + n_out - 1) / n_out; }

// One CTA per sample: feat[1024] (adaptive average pool, (bin row, bin col,
// channel) order), logits[44] = wh . feat + bh.
__global__ void __launch_bounds__(1024) pool_head_fwd_kernel(const bf16 *y4, int h4, int w4, const float *wh,
                                                            const float *bh, float *feat, float *logits) {
    __shared__ float f[kFeat];
    const int s = blockIdx.x;
    const bf16 *src = y4 + (int64_t)s * h4 * w4 * kC4;
    for (int q = threadIdx.x; q < kFeat; q += blockDim.x) {
        const int c = q % kC4, bin = q / kC4, bi = bin / kPW, bj = bin % kPW;
        const int y0 = bin_lo(bi, h4, kPH), y1 = bin_hi(bi, h4, kPH);
        const int x0 = bin_lo(bj, w4, kPW), x1 = bin_hi(bj, w4, kPW);
        float acc = 0.f;
        for (int yy = y0; yy < y1; ++yy)
            for (int xx = x0; xx < x1; ++xx) acc += __bfloat162float(src[((int64_t)yy * w4 + xx) * kC4 + c]);
        f[q] = acc / (float)((y1 - y0) * (x1 - x0));
        feat[(int64_t)s * kFeat + q] = f[q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = warp; o < kOut; o += blockDim.x >> 5) {
        float acc = 0.f;
        for (int q = lane; q < kFeat; q += 32) acc += wh[o * kFeat + q] * f[q];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, d);
        if (lane == 0) logits[(int64_t)s * kOut + o] = acc + bh[o];
    }
}

// One CTA per sample: dfeat = wh^T dlogits, then dy4 (each conv4 output pixel
// collects dfeat / bin area from every bin that covers it).
__global__ void __launch_bounds__(256) pool_head_bwd_kernel(const float *dlogits, const float *wh, int h4, int w4,
                                                           bf16 *dy4) {
    __shared__ float df[kFeat], dl[kOut];
    const int s = blockIdx.x;
    for (int o = threadIdx.x; o < kOut; o += blockDim.x) dl[o] = dlogits[(int64_t)s * kOut + o];
    __syncthreads();
    for (int q = threadIdx.x; q < kFeat; q += blockDim.x) {
        float acc = 0.f;
        for (int o = 0; o < kOut; ++o) acc += wh[o * kFeat + q] * dl[o];
        const int bin = q / kC4, bi = bin / kPW, bj = bin % kPW;
        const int area = (bin_hi(bi, h4, kPH) - bin_lo(bi, h4, kPH)) * (bin_hi(bj, w4, kPW) - bin_lo(bj, w4, kPW));
        df[q] = acc / (float)area;
    }
    __syncthreads();
    bf16 *dst = dy4 + (int64_t)s * h4 * w4 * kC4;
    for (int q = threadIdx.x; q < h4 * w4 * kC4; q += blockDim.x) {
        const int c = q % kC4, pix = q / kC4, yy = pix / w4, xx = pix % w4;
        float acc = 0.f;
        for (int bi = 0; bi < kPH; ++bi) {
            if (yy < bin_lo(bi, h4, kPH) || yy >= bin_hi(bi, h4, kPH)) continue;
            for (int bj = 0; bj < kPW; ++bj)
                if (xx >= bin_lo(bj, w4, kPW) && xx < bin_hi(bj, w4, kPW)) acc += df[(bi * kPW + bj) * kC4 + c];
        }
        dst[q] = __float2bfloat16_rn(acc);
    }
}

// dwh[o][q] += sum_s dlogits[s][o] * feat[s][q]; dbh[o] += sum_s dlogits[s][o].
__global__ void __launch_bounds__(256) head_wgrad_kernel(const float *dlogits, const float *feat, int n, float *dwh,
                                                        float *dbh) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < kOut * kFeat) {
        const int o = idx / kFeat, q = idx % kFeat;
        float acc = 0.f;
        for (int s = 0; s < n; ++s) acc += dlogits[(int64_t)s * kOut + o] * feat[(int64_t)s * kFeat + q];
        dwh[idx] += acc;
    }
    if (idx < kOut) {
        float acc = 0.f;
        for (int s = 0; s < n; ++s) acc += dlogits[(int64_t)s * kOut + idx];
        dbh[idx] += acc;
    }
}

// ------------------------------------------------------------------ loss, optimiser

// Mean binary cross-entropy with logits over n*k outputs and its gradient.
__global__ void __launch_bounds__(256) bce_kernel(const float *z, const float *tgt, int64_t nk, float *loss,
                                                 float *dz) {
    __shared__ float red[8];
    float part = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = z[i], t = tgt[i];
        part += fmaxf(x, 0.f) - x * t + log1pf(expf(-fabsf(x)));
        dz[i] = (1.f / (1.f + expf(-x)) - t) / (float)nk;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *loss = s / (float)nk;   // one block: the sum is in a fixed order
    }
}

__global__ void __launch_bounds__(256) adam_kernel(float *p, const float *g, float *m, float *v, int64_t count,
                                                  float lr, float b1, float b2, float eps, float c1, float c2,
                                                  bf16 *p16) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (p16) p16[i] = __float2bfloat16_rn(pi);
    }
}

int blocks_for(int64_t work, int per_block, int cap = 4096) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace
}  // namespace ld

using namespace ld;

namespace {
ld_status launch_status(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return LD_OK;
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    set_last_error(msg);
    return LD_ERR_CUDA;
}
ld_status bad(const char *msg) {
    set_last_error(msg);
    return LD_ERR_INVALID;
}
bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
bool shape_ok(int cin, int cout) {
    return (cin == 1 && cout == 16) || (cin == 16 && cout == 32) || (cin == 32 && cout == 32);
}
// pixel indices of one image stay below 2^31, and w >= 2 (3x3 windows)
bool size_ok(int h, int w) { return w >= 2 && (uint64_t)h * (uint64_t)w * (uint64_t)w < ((uint64_t)1 << 32); }
ConvGeom geom(int n, int h, int w, int stride) {
    return ConvGeom{n, h, w, (h + 2 - 3) / stride + 1, (w + 2 - 3) / stride + 1, stride};
}
}  // namespace

extern "C" {

ld_status ld_conv3x3_forward(const void *d_x, int32_t n, int32_t h, int32_t w, int32_t cin, int32_t cout,
                             int32_t stride, const void *d_w, const float *d_b, void *d_y, void *stream) {
    if (!d_x || !d_w || !d_b || !d_y || n < 1 || h < 1 || !size_ok(h, w) || (stride != 1 && stride != 2) ||
        !shape_ok(cin, cout))
        return bad("ld_conv3x3_forward: bad argument (supported: 1->16, 16->32, 32->32; stride 1 or 2)");
    cudaStream_t s = (cudaStream_t)stream;
    if (cin == 1) {
        if (stride != 1) return bad("ld_conv3x3_forward: the 1-channel layer has stride 1");
        conv1_fwd_kernel<<<dim3((w + 31) / 32, (h + 7) / 8, n), dim3(32, 8), 0, s>>>(
            (const uint8_t *)d_x, h, w, (const bf16 *)d_w, d_b, (bf16 *)d_y);
        return launch_status("conv1_fwd");
    }
    const ConvGeom G = geom(n, h, w, stride);
    const ConvTcGeom T{n, h, w, G.oh, G.ow, stride};
    const cudaError_t e = launch_conv_fwd_tc(d_x, T, cin, d_w, d_b, d_y, s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    return launch_status("conv_fwd_tc");
}

ld_status ld_conv3x3_backward(const void *d_x, int32_t n, int32_t h, int32_t w, int32_t cin, int32_t cout,
                              int32_t stride, const void *d_w, const void *d_y, const void *d_dy, void *d_dx,
                              float *d_dw, float *d_db, void *stream) {
    if (!d_x || !d_w || !d_y || !d_dy || !d_dw || !d_db || n < 1 || h < 1 || !size_ok(h, w) ||
        (stride != 1 && stride != 2) || !shape_ok(cin, cout))
        return bad("ld_conv3x3_backward: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (cin == 1) {
        if (stride != 1 || d_dx) return bad("ld_conv3x3_backward: the 1-channel layer: stride 1, no dx");
        const int blocks = blocks_for((int64_t)n * h * w, 16 * 64, 1024);
        float *part = nullptr;
        if (cudaMallocAsync((void **)&part, (size_t)blocks * 160 * sizeof(float), s) != cudaSuccess)
            return launch_status("conv1_wgrad workspace");
        conv1_wgrad_kernel<<<blocks, 256, 0, s>>>((const uint8_t *)d_x, (const bf16 *)d_y, (const bf16 *)d_dy, n,
                                                 h, w, part);
        reduce_parts1<<<1, 160, 0, s>>>(part, blocks, d_dw, d_db);
        cudaFreeAsync(part, s);
        return launch_status("conv1_wgrad");
    }
    if (h > 65535 || w > 65535 || !aligned16(d_x) || !aligned16(d_y) || !aligned16(d_dy) || !aligned16(d_w) ||
        (d_dx && !aligned16(d_dx)))
        return bad("ld_conv3x3_backward: h, w <= 65535 and 16-byte aligned tensors required");
    const ConvGeom G = geom(n, h, w, stride);
    const ConvTcGeom T{n, h, w, G.oh, G.ow, stride};
    const int chunk = 2048;
    const int ctas = ((G.oh * G.ow + chunk - 1) / chunk) * n, nw = cout * 9 * cin;
    float *part = nullptr;   // per-CTA partial sums (weights, then biases), stream-ordered
    if (cudaMallocAsync((void **)&part, (size_t)ctas * (nw + cout) * sizeof(float), s) != cudaSuccess)
        return launch_status("conv_wgrad workspace");
    float *part_b = part + (size_t)ctas * nw;
    cudaError_t e = launch_conv_wgrad_tc(d_x, d_y, d_dy, T, cin, chunk, part, part_b, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(part, s);
        set_last_error(cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    reduce_parts<<<(nw + 255) / 256, 256, 0, s>>>(part, ctas, nw, d_dw);
    reduce_parts<<<1, 256, 0, s>>>(part_b, ctas, cout, d_db);
    cudaFreeAsync(part, s);
    ld_status st = launch_status("conv_wgrad_tc");
    if (st != LD_OK || !d_dx) return st;
    e = launch_conv_dgrad_tc(d_y, d_dy, T, cin, d_w, d_dx, s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    return launch_status("conv_dgrad_tc");
}

ld_status ld_pool_head_forward(const void *d_y4, int32_t n, int32_t h4, int32_t w4, const float *d_wh,
                               const float *d_bh, float *d_feat, float *d_logits, void *stream) {
    if (!d_y4 || !d_wh || !d_bh || !d_feat || !d_logits || n < 1 || h4 < kPH || w4 < kPW)
        return bad("ld_pool_head_forward: bad argument");
    pool_head_fwd_kernel<<<n, 1024, 0, (cudaStream_t)stream>>>((const bf16 *)d_y4, h4, w4, d_wh, d_bh, d_feat,
                                                               d_logits);
    return launch_status("pool_head_fwd");
}

ld_status ld_pool_head_backward(const float *d_feat, const float *d_dlogits, const float *d_wh, int32_t n,
                                int32_t h4, int32_t w4, float *d_dwh, float *d_dbh, void *d_dy4, void *stream) {
    if (!d_feat || !d_dlogits || !d_wh || !d_dwh || !d_dbh || !d_dy4 || n < 1 || h4 < kPH || w4 < kPW)
        return bad("ld_pool_head_backward: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    head_wgrad_kernel<<<(kOut * kFeat + 255) / 256, 256, 0, s>>>(d_dlogits, d_feat, n, d_dwh, d_dbh);
    ld_status st = launch_status("head_wgrad");
    if (st != LD_OK) return st;
    pool_head_bwd_kernel<<<n, 256, 0, s>>>(d_dlogits, d_wh, h4, w4, (bf16 *)d_dy4);
    return launch_status("pool_head_bwd");
}

ld_status ld_bce_loss(const float *d_logits, const float *d_target, int32_t n, int32_t k, float *d_loss,
                      float *d_dlogits, void *stream) {
    if (!d_logits || !d_target || !d_loss || !d_dlogits || n < 1 || k < 1) return bad("ld_bce_loss: bad argument");
    const int64_t nk = (int64_t)n * k;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return launch_status("ld_bce_loss memset");
    bce_kernel<<<1, 256, 0, s>>>(d_logits, d_target, nk, d_loss, d_dlogits);
    return launch_status("bce");
}

ld_status ld_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v, int64_t count, float lr,
                       float beta1, float beta2, float eps, int32_t step, void *d_param_bf16, void *stream) {
    if (!d_param || !d_grad || !d_m || !d_v || count < 1 || step < 1) return bad("ld_adam_step: bad argument");
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<blocks_for(count, 256), 256, 0, (cudaStream_t)stream>>>(d_param, d_grad, d_m, d_v, count, lr,
                                                                         beta1, beta2, eps, c1, c2,
                                                                         (bf16 *)d_param_bf16);
    return launch_status("adam");
}

}  // extern "C"
