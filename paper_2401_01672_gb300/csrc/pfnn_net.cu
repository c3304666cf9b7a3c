// Network-level C ABI of the learned warm start: the 3D convolutional encoder-decoder (4 levels,
// 16/32/64/128 channels) assembled from the layer kernels of include/pfnn.h, with its parameters, FP32
// master weights, BF16 working copies, gradients, Adam moments and activation buffers owned by the
// library.  Forward, backward and the optimiser step are sequences of the library's own kernels on the
// network's stream; nothing runs on the host but the sequencing.
//
// Architecture (two 3x3x3 convolutions + ReLU per level, 2x2x2 average-pool down, x2 nearest up + 3x3x3
// convolution, skip concatenation through channel slices of shared buffers, 1x1x1 sigmoid head):
//   in(16) -> e1a(16) -> e1b(16)=cat1[0:16] -> pool -> e2a(32) -> e2b(32)=cat2[0:32] -> pool
//          -> e3a(64) -> e3b(64)=cat3[0:64] -> pool -> e4a(128) -> e4b(128)
//          -> up -> u3(64)=cat3[64:128] -> d3a(64) -> d3b(64) -> up -> u2(32)=cat2[32:64] -> d2a(32) -> d2b(32)
//          -> up -> u1(16)=cat1[16:32] -> d1a(16) -> d1b(16) -> head(1) -> sigmoid
#include "../../include/pfnn.h"
#include "pf_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace {

enum Buf { IN0, E1A, CAT1, P1, E2A, CAT2, P2, E3A, CAT3, P3, E4A, E4B, UP3, D3A, D3B, UP2, D2A, D2B, UP1, D1A, D1B, NBUF };
// channels and level (side S >> level) of each buffer
const int kBufC[NBUF] = {16, 16, 32, 16, 32, 64, 32, 64, 128, 64, 128, 128, 128, 64, 64, 64, 32, 32, 32, 16, 16};
const int kBufL[NBUF] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0};

// what happens before a convolution: 0 none, 1 pool (src buffer, level, channels, dst buffer), 2 upsample
struct Layer {
    const char* name;
    int src, soff, cin, dst, doff, cout, lev;
    int pre;          // 0 none, 1 pool, 2 upsample
    int pre_src, pre_c, pre_dst, pre_lev;
};
const Layer kLayers[] = {
    {"e1a", IN0, 0, 16, E1A, 0, 16, 0, 0, 0, 0, 0, 0},
    {"e1b", E1A, 0, 16, CAT1, 0, 16, 0, 0, 0, 0, 0, 0},
    {"e2a", P1, 0, 16, E2A, 0, 32, 1, 1, CAT1, 16, P1, 0},
    {"e2b", E2A, 0, 32, CAT2, 0, 32, 1, 0, 0, 0, 0, 0},
    {"e3a", P2, 0, 32, E3A, 0, 64, 2, 1, CAT2, 32, P2, 1},
    {"e3b", E3A, 0, 64, CAT3, 0, 64, 2, 0, 0, 0, 0, 0},
    {"e4a", P3, 0, 64, E4A, 0, 128, 3, 1, CAT3, 64, P3, 2},
    {"e4b", E4A, 0, 128, E4B, 0, 128, 3, 0, 0, 0, 0, 0},
    {"u3", UP3, 0, 128, CAT3, 64, 64, 2, 2, E4B, 128, UP3, 2},
    {"d3a", CAT3, 0, 128, D3A, 0, 64, 2, 0, 0, 0, 0, 0},
    {"d3b", D3A, 0, 64, D3B, 0, 64, 2, 0, 0, 0, 0, 0},
    {"u2", UP2, 0, 64, CAT2, 32, 32, 1, 2, D3B, 64, UP2, 1},
    {"d2a", CAT2, 0, 64, D2A, 0, 32, 1, 0, 0, 0, 0, 0},
    {"d2b", D2A, 0, 32, D2B, 0, 32, 1, 0, 0, 0, 0, 0},
    {"u1", UP1, 0, 32, CAT1, 16, 16, 0, 2, D2B, 32, UP1, 0},
    {"d1a", CAT1, 0, 32, D1A, 0, 16, 0, 0, 0, 0, 0, 0},
    {"d1b", D1A, 0, 16, D1B, 0, 16, 0, 0, 0, 0, 0, 0},
};
constexpr int NCONV = sizeof(kLayers) / sizeof(kLayers[0]);
constexpr int NPARAM = NCONV + 1;   // + the 1x1x1 head (16 weights, 1 bias)
constexpr int NFEAT = 2;            // supercooling and surface-tension features

struct Param {
    long long nw = 0, nb = 0;
    float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    void* wb = nullptr;   // bf16 working copy [27][cout][cin]
    void* wt = nullptr;   // bf16 transposed copy [27][cin][cout] (backward data)
};

// splitmix64 (Steele, Lea, Flood 2014) and Box-Muller: the He-normal initial weights
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double normal(uint64_t& s) {
    const double u1 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = __float2bfloat16_rn(in[q]);
}

}  // namespace

struct pfnn_net {
    Param p[NPARAM];
    cudaStream_t stream = nullptr;
    int step = 0;
    int n = 0, S = 0;                      // batch and side of the allocated activation buffers
    void* act[NBUF] = {};                  // bf16 activations
    float* grad[NBUF] = {};                // fp32 gradients of the activations
    float *dz_f = nullptr, *logit_grad = nullptr, *prob = nullptr;
    void* dz_b = nullptr;
    void* wg_work = nullptr;               // scratch of the weight gradients
    long long wg_bytes = 0;
    double* loss = nullptr;
    bool have_target = false;
    std::vector<void*> allocs, act_allocs;
    std::string err;
};

namespace {

pf_status nfail(pfnn_net* net, pf_status s, const std::string& m) {
    if (net) net->err = m;
    return s;
}

void* nalloc(std::vector<void*>& v, size_t bytes) {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    v.push_back(q);
    return q;
}

void free_acts(pfnn_net* net) {
    for (void* q : net->act_allocs) cudaFree(q);
    net->act_allocs.clear();
    for (int b = 0; b < NBUF; ++b) {
        net->act[b] = nullptr;
        net->grad[b] = nullptr;
    }
    net->dz_f = net->logit_grad = net->prob = nullptr;
    net->dz_b = nullptr;
    net->wg_work = nullptr;
    net->wg_bytes = 0;
    net->n = net->S = 0;
}

pf_status ensure_acts(pfnn_net* net, int n, int S) {
    if (net->n == n && net->S == S) return PF_OK;
    free_acts(net);
    for (int b = 0; b < NBUF; ++b) {
        const long long s = S >> kBufL[b];
        const long long cells = (long long)n * s * s * s * kBufC[b];
        net->act[b] = nalloc(net->act_allocs, 2 * cells);
        net->grad[b] = (float*)nalloc(net->act_allocs, 4 * cells);
        if (!net->act[b] || !net->grad[b]) return nfail(net, PF_E_OOM, "activation buffers");
        if (cudaMemsetAsync(net->act[b], 0, 2 * cells, net->stream) != cudaSuccess)
            return nfail(net, PF_E_CUDA, "activation buffers");
    }
    const long long nvox = (long long)n * S * S * S;
    net->dz_f = (float*)nalloc(net->act_allocs, 4 * nvox * 128);
    net->dz_b = nalloc(net->act_allocs, 2 * nvox * 128);
    net->logit_grad = (float*)nalloc(net->act_allocs, 4 * nvox);
    net->prob = (float*)nalloc(net->act_allocs, 4 * nvox);
    long long wg = 0;
    for (int q = 0; q < NCONV; ++q) {
        const int sd = S >> kLayers[q].lev;
        const long long b = pfnn_conv3d_wgrad_work_bytes(kLayers[q].cout, kLayers[q].cin, n, sd, sd, sd);
        wg = b > wg ? b : wg;
    }
    net->wg_work = nalloc(net->act_allocs, (size_t)wg);
    net->wg_bytes = wg;
    if (!net->dz_f || !net->dz_b || !net->logit_grad || !net->prob || !net->wg_work)
        return nfail(net, PF_E_OOM, "work buffers");
    net->n = n;
    net->S = S;
    return PF_OK;
}

#define NN_CK(net, call, what)                                                 \
    do {                                                                       \
        pf_status s_ = (call);                                                 \
        if (s_ != PF_OK) return nfail((net), s_, std::string(what) + " failed"); \
    } while (0)

}  // namespace

extern "C" {

int pfnn_net_params(void) { return NPARAM; }

pf_status pfnn_net_param_shape(int q, int* cin, int* cout) {
    if (q < 0 || q >= NPARAM) return PF_E_INVALID;
    if (cin) *cin = q < NCONV ? kLayers[q].cin : 16;
    if (cout) *cout = q < NCONV ? kLayers[q].cout : 1;
    return PF_OK;
}

const char* pfnn_net_param_name(int q) { return q >= 0 && q < NCONV ? kLayers[q].name : (q == NCONV ? "head" : ""); }

const char* pfnn_net_last_error(const pfnn_net* net) { return net ? net->err.c_str() : ""; }

int pfnn_net_buffers(void) { return NBUF; }

// layer q's wiring: input buffer and channel offset, cin, output buffer and offset, cout, level, and what
// runs before it (0 none, 1 pool of pre_c channels of buffer pre_src into pre_dst, 2 upsample)
pf_status pfnn_net_layer(int q, int* wiring) {
    if (q < 0 || q >= NCONV || !wiring) return PF_E_INVALID;
    const Layer& L = kLayers[q];
    const int v[12] = {L.src, L.soff, L.cin, L.dst, L.doff, L.cout, L.lev, L.pre, L.pre_src, L.pre_c, L.pre_dst, L.pre_lev};
    for (int k = 0; k < 12; ++k) wiring[k] = v[k];
    return PF_OK;
}

// buffer b: channels per voxel and level (side >> level)
pf_status pfnn_net_buffer(int b, int* channels, int* level) {
    if (b < 0 || b >= NBUF) return PF_E_INVALID;
    if (channels) *channels = kBufC[b];
    if (level) *level = kBufL[b];
    return PF_OK;
}

// copy buffer b of the last forward / backward to host arrays (bf16 activations, fp32 gradients; either
// may be NULL) of n (side >> level)^3 channels values; synchronous
pf_status pfnn_net_read_buffer(pfnn_net* net, int b, void* act, float* grad) {
    if (!net || b < 0 || b >= NBUF) return PF_E_INVALID;
    if (!net->S) return nfail(net, PF_E_STATE, "no forward yet");
    const long long s = net->S >> kBufL[b];
    const long long cells = (long long)net->n * s * s * s * kBufC[b];
    if ((act && cudaMemcpyAsync(act, net->act[b], 2 * cells, cudaMemcpyDeviceToHost, net->stream) != cudaSuccess) ||
        (grad && cudaMemcpyAsync(grad, net->grad[b], 4 * cells, cudaMemcpyDeviceToHost, net->stream) != cudaSuccess) ||
        cudaStreamSynchronize(net->stream) != cudaSuccess)
        return nfail(net, PF_E_CUDA, "read_buffer");
    return PF_OK;
}

pf_status pfnn_net_destroy(pfnn_net* net) {
    if (!net) return PF_OK;
    if (net->stream) cudaStreamSynchronize(net->stream);
    free_acts(net);
    for (void* q : net->allocs) cudaFree(q);
    delete net;
    return PF_OK;
}

pf_status pfnn_net_create(unsigned long long seed, void* stream, pfnn_net** out) {
    if (!out) return PF_E_INVALID;
    *out = nullptr;
    pfnn_net* net = new pfnn_net();
    net->stream = (cudaStream_t)stream;
    uint64_t rs = seed;
    for (int q = 0; q < NPARAM; ++q) {
        Param& P = net->p[q];
        const int cin = q < NCONV ? kLayers[q].cin : 16, cout = q < NCONV ? kLayers[q].cout : 1;
        P.nw = q < NCONV ? 27LL * cout * cin : 16;
        P.nb = cout;
        float** f32s[] = {&P.w, &P.gw, &P.mw, &P.vw};
        for (float** f : f32s) *f = (float*)nalloc(net->allocs, 4 * P.nw);
        float** f32b[] = {&P.b, &P.gb, &P.mb, &P.vb};
        for (float** f : f32b) *f = (float*)nalloc(net->allocs, 4 * P.nb);
        if (q < NCONV) {
            P.wb = nalloc(net->allocs, 2 * P.nw);
            P.wt = nalloc(net->allocs, 2 * P.nw);
        }
        if (!P.w || !P.gw || !P.mw || !P.vw || !P.b || !P.gb || !P.mb || !P.vb || (q < NCONV && (!P.wb || !P.wt))) {
            pfnn_net_destroy(net);
            return PF_E_OOM;
        }
        // He-normal weights for the ReLU layers (std sqrt(2 / fan_in)), sqrt(1/16) for the head; zero biases
        std::vector<float> w(P.nw), z(P.nb, 0.f);
        const double sd = q < NCONV ? std::sqrt(2.0 / (27.0 * cin)) : std::sqrt(1.0 / 16.0);
        for (long long k = 0; k < P.nw; ++k) w[k] = (float)(normal(rs) * sd);
        cudaError_t e = cudaMemcpy(P.w, w.data(), 4 * P.nw, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(P.b, z.data(), 4 * P.nb, cudaMemcpyHostToDevice);
        for (float* f : {P.gw, P.mw, P.vw})
            if (e == cudaSuccess) e = cudaMemset(f, 0, 4 * P.nw);
        for (float* f : {P.gb, P.mb, P.vb})
            if (e == cudaSuccess) e = cudaMemset(f, 0, 4 * P.nb);
        if (e == cudaSuccess && P.wb) {
            k_f32_to_bf16<<<(unsigned)((P.nw + 255) / 256), 256>>>(P.w, (__nv_bfloat16*)P.wb, P.nw);
            pfgb::count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            pfnn_net_destroy(net);
            return PF_E_CUDA;
        }
    }
    net->loss = (double*)nalloc(net->allocs, sizeof(double));
    if (!net->loss) {
        pfnn_net_destroy(net);
        return PF_E_OOM;
    }
    *out = net;
    return PF_OK;
}

// parameter q's FP32 master weights and biases from / to host arrays (w: [27][cout][cin], head: [16])
pf_status pfnn_net_set_params(pfnn_net* net, int q, const float* w, const float* b) {
    if (!net || q < 0 || q >= NPARAM || !w || !b) return PF_E_INVALID;
    Param& P = net->p[q];
    if (cudaMemcpyAsync(P.w, w, 4 * P.nw, cudaMemcpyHostToDevice, net->stream) != cudaSuccess ||
        cudaMemcpyAsync(P.b, b, 4 * P.nb, cudaMemcpyHostToDevice, net->stream) != cudaSuccess)
        return nfail(net, PF_E_CUDA, "set_params");
    if (P.wb) {
        k_f32_to_bf16<<<(unsigned)((P.nw + 255) / 256), 256, 0, net->stream>>>(P.w, (__nv_bfloat16*)P.wb, P.nw);
        pfgb::count_launch();
    }
    if (cudaStreamSynchronize(net->stream) != cudaSuccess) return nfail(net, PF_E_CUDA, "set_params");
    return PF_OK;
}

pf_status pfnn_net_get_params(pfnn_net* net, int q, float* w, float* b) {
    if (!net || q < 0 || q >= NPARAM) return PF_E_INVALID;
    const Param& P = net->p[q];
    if ((w && cudaMemcpyAsync(w, P.w, 4 * P.nw, cudaMemcpyDeviceToHost, net->stream) != cudaSuccess) ||
        (b && cudaMemcpyAsync(b, P.b, 4 * P.nb, cudaMemcpyDeviceToHost, net->stream) != cudaSuccess) ||
        cudaStreamSynchronize(net->stream) != cudaSuccess)
        return nfail(net, PF_E_CUDA, "get_params");
    return PF_OK;
}

pf_status pfnn_net_get_grads(pfnn_net* net, int q, float* gw, float* gb) {
    if (!net || q < 0 || q >= NPARAM) return PF_E_INVALID;
    const Param& P = net->p[q];
    if ((gw && cudaMemcpyAsync(gw, P.gw, 4 * P.nw, cudaMemcpyDeviceToHost, net->stream) != cudaSuccess) ||
        (gb && cudaMemcpyAsync(gb, P.gb, 4 * P.nb, cudaMemcpyDeviceToHost, net->stream) != cudaSuccess) ||
        cudaStreamSynchronize(net->stream) != cudaSuccess)
        return nfail(net, PF_E_CUDA, "get_grads");
    return PF_OK;
}

pf_status pfnn_net_forward(pfnn_net* net, const float* G, const float* feat, int n, int side, const float* target,
                           float* prob) {
    if (!net || !G || !feat || n < 1 || side < 8 || side % 8) return PF_E_INVALID;
    pf_status st = ensure_acts(net, n, side);
    if (st != PF_OK) return st;
    cudaStream_t s = net->stream;
    const long long vps = (long long)side * side * side, nvox = (long long)n * vps;
    auto dims = [&](int lev, int* d) { const int sd = side >> lev; d[0] = n; d[1] = d[2] = d[3] = sd; };
    NN_CK(net, pfnn_pack_input(G, feat, NFEAT, vps, nvox, net->act[IN0], s), "pack");
    for (int q = 0; q < NCONV; ++q) {
        const Layer& L = kLayers[q];
        int d[4];
        if (L.pre == 1) {
            dims(L.pre_lev, d);
            NN_CK(net, pfnn_avgpool(net->act[L.pre_src], kBufC[L.pre_src], 0, net->act[L.pre_dst], kBufC[L.pre_dst], 0,
                                    L.pre_c, d[0], d[1], d[2], d[3], s), "pool");
        } else if (L.pre == 2) {
            dims(L.pre_lev, d);
            NN_CK(net, pfnn_upsample(net->act[L.pre_src], L.pre_c, net->act[L.pre_dst], kBufC[L.pre_dst], 0, d[0], d[1],
                                     d[2], d[3], s), "upsample");
        }
        dims(L.lev, d);
        const Param& P = net->p[q];
        NN_CK(net, pfnn_conv3d(net->act[L.src], kBufC[L.src], L.soff, P.wb, L.cin, L.cout, P.b, 1, 0, net->act[L.dst],
                               nullptr, kBufC[L.dst], L.doff, 0, d[0], d[1], d[2], d[3], s), L.name);
    }
    if (cudaMemsetAsync(net->loss, 0, sizeof(double), s) != cudaSuccess) return nfail(net, PF_E_CUDA, "loss");
    const Param& H = net->p[NCONV];
    net->have_target = target != nullptr;
    NN_CK(net, pfnn_head_forward(net->act[D1B], 16, H.w, H.b, target, nvox, prob ? prob : net->prob,
                                 target ? net->logit_grad : nullptr, target ? net->loss : nullptr, s), "head");
    return PF_OK;
}

pf_status pfnn_net_infer(pfnn_net* net, const float* G, const float* feat, int n, int side, float* prob) {
    if (!prob) return PF_E_INVALID;
    return pfnn_net_forward(net, G, feat, n, side, nullptr, prob);
}

pf_status pfnn_net_loss(pfnn_net* net, double* loss) {
    if (!net || !loss) return PF_E_INVALID;
    if (cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, net->stream) != cudaSuccess ||
        cudaStreamSynchronize(net->stream) != cudaSuccess)
        return nfail(net, PF_E_CUDA, "loss");
    return PF_OK;
}

pf_status pfnn_net_backward(pfnn_net* net) {
    if (!net) return PF_E_INVALID;
    if (!net->have_target || !net->S) return nfail(net, PF_E_STATE, "backward needs a forward with a target");
    cudaStream_t s = net->stream;
    const int n = net->n, side = net->S;
    auto dims = [&](int lev, int* d) { const int sd = side >> lev; d[0] = n; d[1] = d[2] = d[3] = sd; };
    for (int b = 0; b < NBUF; ++b) {
        const long long sd = side >> kBufL[b];
        if (cudaMemsetAsync(net->grad[b], 0, 4LL * n * sd * sd * sd * kBufC[b], s) != cudaSuccess)
            return nfail(net, PF_E_CUDA, "zero gradients");
    }
    for (int q = 0; q < NPARAM; ++q) {
        if (cudaMemsetAsync(net->p[q].gw, 0, 4 * net->p[q].nw, s) != cudaSuccess ||
            cudaMemsetAsync(net->p[q].gb, 0, 4 * net->p[q].nb, s) != cudaSuccess)
            return nfail(net, PF_E_CUDA, "zero gradients");
    }
    const long long nvox0 = (long long)n * side * side * side;
    const Param& H = net->p[NCONV];
    NN_CK(net, pfnn_head_backward(net->act[D1B], 16, H.w, net->logit_grad, nvox0, net->grad[D1B], H.gw, H.gb, s),
          "head backward");
    for (int q = NCONV - 1; q >= 0; --q) {
        const Layer& L = kLayers[q];
        Param& P = net->p[q];
        int d[4];
        dims(L.lev, d);
        const long long nvox = (long long)d[0] * d[1] * d[2] * d[3];
        const int ldy = kBufC[L.dst];
        // ReLU backward on this layer's output slice, then the three products of the convolution
        NN_CK(net, pfnn_relu_bwd_cast(net->grad[L.dst], ldy, L.doff, net->act[L.dst], ldy, L.doff, L.cout, nvox,
                                      net->dz_f, net->dz_b, s), "relu backward");
        NN_CK(net, pfnn_bias_grad(net->dz_f, L.cout, 0, L.cout, nvox, P.gb, s), "bias gradient");
        NN_CK(net, pfnn_conv3d_wgrad(net->dz_b, L.cout, 0, L.cout, net->act[L.src], kBufC[L.src], L.soff, L.cin, P.gw,
                                     d[0], d[1], d[2], d[3], net->wg_work, net->wg_bytes, s), "weight gradient");
        if (L.src != IN0) {
            NN_CK(net, pfnn_weight_transpose(P.wb, P.wt, L.cout, L.cin, s), "weight transpose");
            NN_CK(net, pfnn_conv3d(net->dz_b, L.cout, 0, P.wt, L.cout, L.cin, nullptr, 0, 1, nullptr, net->grad[L.src],
                                   kBufC[L.src], L.soff, 1, d[0], d[1], d[2], d[3], s), "data gradient");
        }
        // adjoint of the data movement that produced this layer's input
        if (L.pre == 1) {
            int e[4];
            dims(L.pre_lev, e);
            NN_CK(net, pfnn_avgpool_bwd(net->grad[L.pre_dst], L.pre_c, net->grad[L.pre_src], kBufC[L.pre_src], 0, e[0],
                                        e[1], e[2], e[3], s), "pool backward");
        } else if (L.pre == 2) {
            int e[4];
            dims(L.pre_lev + 1, e);  // the coarse side
            NN_CK(net, pfnn_upsample_bwd(net->grad[L.pre_dst], kBufC[L.pre_dst], 0, L.pre_c, net->grad[L.pre_src],
                                         e[0], e[1], e[2], e[3], s), "upsample backward");
        }
    }
    return PF_OK;
}

pf_status pfnn_net_adam_step(pfnn_net* net, float lr, float b1, float b2, float eps) {
    if (!net || !(lr > 0.f)) return PF_E_INVALID;
    net->step += 1;
    for (int q = 0; q < NPARAM; ++q) {
        Param& P = net->p[q];
        NN_CK(net, pfnn_adam(P.w, P.gw, P.mw, P.vw, P.wb, P.nw, lr, b1, b2, eps, net->step, net->stream), "adam");
        NN_CK(net, pfnn_adam(P.b, P.gb, P.mb, P.vb, nullptr, P.nb, lr, b1, b2, eps, net->step, net->stream), "adam");
    }
    return PF_OK;
}

}  // extern "C"
