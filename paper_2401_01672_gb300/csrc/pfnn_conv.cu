// Kernels of the learned warm start: a 3D convolutional encoder-decoder trained and run with BF16
// activations and weights, FP32 accumulation, FP32 master weights and gradients.  The forward and
// backward-data convolutions and the weight gradient run on tcgen05 (pfnn_umma.cu); this file holds the
// data-movement, head and optimiser kernels.
//
// Layout: activations N x D x H x W x C (channels last), bf16; a tensor may be a channel slice
// [off, off + C) of a wider buffer with ld channels per voxel (skip concatenation is free).
// Convolutions are 3x3x3 with zero padding 1 and stride 1; weights are [27][Cout][Cin] bf16 with
// tap t = (dz+1)*9 + (dy+1)*3 + (dx+1).
//
// Implicit GEMM (forward): D[v][co] = sum over (t, ci) of X[v + off(t)][ci] W[t][co][ci].
// Backward data is the same GEMM on dY with flipped taps and transposed weights [27][Cin][Cout]:
//   dX[v][ci] = sum over (t, co) of dY[v - off(t)][co] W[t][co][ci].
// Backward weight, per tap: dW[t][co][ci] = sum over v of dY[v][co] X[v + off(t)][ci] (pfnn_umma.cu).
#include "../../include/pfnn.h"
#include "pf_internal.cuh"

#include <cuda_bf16.h>
#include <cstdint>

namespace {

// voxel index -> coordinates
__device__ __forceinline__ void vox_coord(long long v, int D, int H, int W, int& b, int& z, int& y, int& x) {
    x = (int)(v % W);
    long long r = v / W;
    y = (int)(r % H);
    r /= H;
    z = (int)(r % D);
    b = (int)(r / D);
}


__global__ void k_bias_grad(const float* __restrict__ dz, int ld, int off, int c, long long nvox, float* db) {
    // one block per channel group of 32 channels x 8 voxel lanes
    const int ch = blockIdx.y * 32 + (threadIdx.x & 31);
    float s = 0.f;
    if (ch < c)
        for (long long v = blockIdx.x * 8 + (threadIdx.x >> 5); v < nvox; v += (long long)gridDim.x * 8)
            s += dz[v * ld + off + ch];
    __shared__ float sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < 32 && ch < c) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += sh[q * 32 + threadIdx.x];
        atomicAdd(&db[ch], t);
    }
}

// dz = dy * (y > 0) cast to bf16 (ReLU backward), or plain cast when y is NULL
__global__ void k_relu_bwd_cast(const float* __restrict__ dy, int lddy, int dyoff, const __nv_bfloat16* __restrict__ y,
                                int ldy, int yoff, int c, long long nvox, float* __restrict__ dzf,
                                __nv_bfloat16* __restrict__ dzb) {
    const long long n = nvox * c;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long v = q / c;
        const int ch = (int)(q % c);
        float gr = dy[v * lddy + dyoff + ch];
        if (y && !(__bfloat162float(y[v * ldy + yoff + ch]) > 0.f)) gr = 0.f;
        if (dzf) dzf[v * c + ch] = gr;
        dzb[v * c + ch] = __float2bfloat16_rn(gr);
    }
}

// [27][Cout][Cin] -> [27][Cin][Cout]
__global__ void k_wtranspose(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt, int cout, int cin) {
    const long long n = 27LL * cout * cin;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(q % cin);
        const int co = (int)((q / cin) % cout);
        const int t = (int)(q / ((long long)cin * cout));
        wt[((long long)t * cin + ci) * cout + co] = w[q];
    }
}

// 2x2x2 average pooling of a channel slice (even sizes), and its adjoint
__global__ void k_avgpool(const __nv_bfloat16* __restrict__ x, int ldx, int xoff, __nv_bfloat16* __restrict__ y, int ldy,
                          int yoff, int c, int N, int D, int H, int W) {
    const int d2 = D / 2, h2 = H / 2, w2 = W / 2;
    const long long n = (long long)N * d2 * h2 * w2 * c;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(q % c);
        long long v = q / c;
        int b, z, yy, xx;
        vox_coord(v, d2, h2, w2, b, z, yy, xx);
        float s = 0.f;
        for (int o = 0; o < 8; ++o) {
            const long long sv = (((long long)b * D + 2 * z + (o >> 2)) * H + 2 * yy + ((o >> 1) & 1)) * W + 2 * xx + (o & 1);
            s += __bfloat162float(x[sv * ldx + xoff + ch]);
        }
        y[v * ldy + yoff + ch] = __float2bfloat16_rn(0.125f * s);
    }
}

__global__ void k_avgpool_bwd(const float* __restrict__ dy, int c, float* __restrict__ dx, int lddx, int dxoff, int N,
                              int D, int H, int W) {
    const long long n = (long long)N * D * H * W * c;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(q % c);
        const long long v = q / c;
        int b, z, yy, xx;
        vox_coord(v, D, H, W, b, z, yy, xx);
        const long long pv = (((long long)b * (D / 2) + z / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2;
        dx[v * lddx + dxoff + ch] += 0.125f * dy[pv * c + ch];
    }
}

// x2 nearest-neighbour upsampling of a channel slice, and its adjoint (sum of the 8 children)
__global__ void k_upsample(const __nv_bfloat16* __restrict__ x, int c, __nv_bfloat16* __restrict__ y, int ldy, int yoff,
                           int N, int D, int H, int W) {  // D, H, W of the output
    const long long n = (long long)N * D * H * W * c;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(q % c);
        const long long v = q / c;
        int b, z, yy, xx;
        vox_coord(v, D, H, W, b, z, yy, xx);
        const long long pv = (((long long)b * (D / 2) + z / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2;
        y[v * ldy + yoff + ch] = x[pv * c + ch];
    }
}

__global__ void k_upsample_bwd(const float* __restrict__ dy, int lddy, int dyoff, int c, float* __restrict__ dx, int N,
                               int D, int H, int W) {  // D, H, W of the (coarse) input
    const long long n = (long long)N * D * H * W * c;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(q % c);
        const long long v = q / c;
        int b, z, yy, xx;
        vox_coord(v, D, H, W, b, z, yy, xx);
        float s = 0.f;
        for (int o = 0; o < 8; ++o) {
            const long long sv = (((long long)b * 2 * D + 2 * z + (o >> 2)) * 2 * H + 2 * yy + ((o >> 1) & 1)) * 2 * W +
                                 2 * xx + (o & 1);
            s += dy[sv * lddy + dyoff + ch];
        }
        dx[v * c + ch] += s;
    }
}

// 1x1x1 head: logit[v] = sum_c x[v][c] w[c] + b; loss = mean of BCE(sigmoid(logit), target) or its
// sum of squares; dlogit = (sigmoid - target) / nvox (BCE) written for the backward pass.
__global__ void k_head_fwd_loss(const __nv_bfloat16* __restrict__ x, int c, const float* __restrict__ w, const float* __restrict__ bp,
                                const float* __restrict__ target, long long nvox, float* __restrict__ prob,
                                float* __restrict__ dlogit, double* loss) {
    double l = 0.0;
    const float b = bp[0];
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        float s = b;
        for (int ch = 0; ch < c; ++ch) s += __bfloat162float(x[v * c + ch]) * w[ch];
        const float p = 1.f / (1.f + expf(-s));
        if (prob) prob[v] = p;
        if (target) {
            const double t = target[v];
            // cross-entropy of the clipped probability, evaluated in binary64 from the logit
            const double pd = 1.0 / (1.0 + exp(-(double)s));
            const double pc = fmin(fmax(pd, 1e-7), 1.0 - 1e-7);
            const double qc = fmin(fmax(1.0 / (1.0 + exp((double)s)), 1e-7), 1.0 - 1e-7);  // 1 - p without cancellation
            l += -(t * log(pc) + (1.0 - t) * log(qc));
            if (dlogit) dlogit[v] = (p - (float)t) / (float)nvox;
        }
    }
    if (target && loss) {
        __shared__ double sh[256];
        sh[threadIdx.x] = l;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(loss, sh[0] / (double)nvox);
    }
}

// head backward: dx[v][c] = dlogit[v] w[c]; dw[c] += sum_v dlogit[v] x[v][c]; db += sum_v dlogit[v]
__global__ void k_head_bwd(const __nv_bfloat16* __restrict__ x, int c, const float* __restrict__ w,
                           const float* __restrict__ dlogit, long long nvox, float* __restrict__ dx, float* dw, float* db) {
    float accw[32];
    for (int ch = 0; ch < 32; ++ch) accw[ch] = 0.f;
    float accb = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const float gl = dlogit[v];
        accb += gl;
        for (int ch = 0; ch < c && ch < 32; ++ch) {
            dx[v * c + ch] = gl * w[ch];
            accw[ch] += gl * __bfloat162float(x[v * c + ch]);
        }
    }
    for (int ch = 0; ch < c && ch < 32; ++ch) atomicAdd(&dw[ch], accw[ch]);
    atomicAdd(db, accb);
}

// Adam with bias correction on FP32 master weights; writes the bf16 working copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float gq = gr[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        const float pq = p[q] - lr * (mq * c1) / (sqrtf(vq * c2) + eps);
        p[q] = pq;
        if (pb) pb[q] = __float2bfloat16_rn(pq);
    }
}

// network input: channel 0 = glass field G, 1..2 = per-sample features, 3..15 = 0
__global__ void k_pack_input(const float* __restrict__ G, const float* __restrict__ feat, int nfeat, long long vps,
                             long long nvox, __nv_bfloat16* __restrict__ out) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const long long smp = v / vps;
        __nv_bfloat16* o = out + v * 16;
        o[0] = __float2bfloat16_rn(G[v]);
        for (int f = 0; f < 15; ++f) o[1 + f] = __float2bfloat16_rn(f < nfeat ? feat[smp * nfeat + f] : 0.f);
    }
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    return (int)(b < 1 ? 1 : b);
}

bool aligned8(int a) { return (a % 8) == 0; }

}  // namespace

using bf16 = __nv_bfloat16;

extern "C" {


pf_status pfnn_bias_grad(const float* dz, int ld, int off, int c, long long nvox, float* db, void* stream) {
    if (!dz || !db || c < 1) return PF_E_INVALID;
    dim3 grid(152 * 4, (c + 31) / 32);
    k_bias_grad<<<grid, 256, 0, (cudaStream_t)stream>>>(dz, ld, off, c, nvox, db);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_relu_bwd_cast(const float* dy, int lddy, int dyoff, const void* y, int ldy, int yoff, int c,
                             long long nvox, float* dz_f32, void* dz_bf16, void* stream) {
    if (!dy || !dz_bf16 || c < 1) return PF_E_INVALID;
    k_relu_bwd_cast<<<grid_for(nvox * c), 256, 0, (cudaStream_t)stream>>>(dy, lddy, dyoff, (const bf16*)y, ldy, yoff, c,
                                                                         nvox, dz_f32, (bf16*)dz_bf16);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_weight_transpose(const void* w, void* wt, int cout, int cin, void* stream) {
    if (!w || !wt) return PF_E_INVALID;
    k_wtranspose<<<grid_for(27LL * cout * cin), 256, 0, (cudaStream_t)stream>>>((const bf16*)w, (bf16*)wt, cout, cin);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_avgpool(const void* x, int ldx, int xoff, void* y, int ldy, int yoff, int c, int n, int d, int h, int wd,
                       void* stream) {
    if (!x || !y || d % 2 || h % 2 || wd % 2) return PF_E_INVALID;
    k_avgpool<<<grid_for((long long)n * d * h * wd / 8 * c), 256, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, ldx, xoff, (bf16*)y, ldy, yoff, c, n, d, h, wd);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_avgpool_bwd(const float* dy, int c, float* dx, int lddx, int dxoff, int n, int d, int h, int wd,
                           void* stream) {
    if (!dy || !dx || d % 2 || h % 2 || wd % 2) return PF_E_INVALID;
    k_avgpool_bwd<<<grid_for((long long)n * d * h * wd * c), 256, 0, (cudaStream_t)stream>>>(dy, c, dx, lddx, dxoff, n, d,
                                                                                             h, wd);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_upsample(const void* x, int c, void* y, int ldy, int yoff, int n, int d, int h, int wd, void* stream) {
    if (!x || !y || d % 2 || h % 2 || wd % 2) return PF_E_INVALID;
    k_upsample<<<grid_for((long long)n * d * h * wd * c), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, c, (bf16*)y,
                                                                                          ldy, yoff, n, d, h, wd);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_upsample_bwd(const float* dy, int lddy, int dyoff, int c, float* dx, int n, int d, int h, int wd,
                            void* stream) {
    if (!dy || !dx) return PF_E_INVALID;
    k_upsample_bwd<<<grid_for((long long)n * d * h * wd * c), 256, 0, (cudaStream_t)stream>>>(dy, lddy, dyoff, c, dx, n,
                                                                                              d, h, wd);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_head_forward(const void* x, int c, const float* w, const float* b, const float* target, long long nvox,
                            float* prob, float* dlogit, double* loss, void* stream) {
    if (!x || !w || !b || c < 1 || c > 32) return PF_E_INVALID;
    k_head_fwd_loss<<<grid_for(nvox), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, c, w, b, target, nvox, prob,
                                                                       dlogit, loss);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_head_backward(const void* x, int c, const float* w, const float* dlogit, long long nvox, float* dx,
                             float* dw, float* db, void* stream) {
    if (!x || !w || !dlogit || !dx || !dw || !db || c < 1 || c > 32) return PF_E_INVALID;
    k_head_bwd<<<152 * 4, 256, 0, (cudaStream_t)stream>>>((const bf16*)x, c, w, dlogit, nvox, dx, dw, db);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_pack_input(const float* G, const float* feat, int nfeat, long long vox_per_sample, long long nvox,
                          void* out, void* stream) {
    if (!G || !out || nfeat < 0 || nfeat > 15 || (nfeat && !feat) || vox_per_sample < 1) return PF_E_INVALID;
    k_pack_input<<<grid_for(nvox), 256, 0, (cudaStream_t)stream>>>(G, feat, nfeat, vox_per_sample, nvox, (bf16*)out);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_adam(float* p, const float* g, float* m, float* v, void* p_bf16, long long n, float lr, float b1,
                    float b2, float eps, int step, void* stream) {
    if (!p || !g || !m || !v || step < 1) return PF_E_INVALID;
    const float c1 = 1.f / (1.f - powf(b1, (float)step));
    const float c2 = 1.f / (1.f - powf(b2, (float)step));
    k_adam<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, (bf16*)p_bf16, n, lr, b1, b2, eps, c1, c2);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

}  // extern "C"
