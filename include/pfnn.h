/*
 * pfnn.h -- C ABI of the learned warm start's kernels (BF16 tensor-core 3D convolutions and the
 * encoder-decoder glue), used to train and run a network that predicts the micro-scale equilibrium
 * phase field from the bead mask, the supercooling and the surface-tension scale.  Its prediction is
 * the initial state of the Runge-Kutta-Merson relaxation of Secs. 2.4-2.5 (the integration stays the
 * judge of the result); the network itself is not part of the paper.
 *
 * Conventions
 *   - Activations: N x D x H x W voxels, channels last (NDHWC), bfloat16.  A tensor may be the channel
 *     slice [off, off + C) of a buffer with ld channels per voxel.  FP32 gradient buffers use the
 *     same layout.
 *   - Convolutions: 3x3x3 taps, zero padding 1, stride 1.  Weights [27][Cout][Cin] bfloat16, tap
 *     t = (dz+1)*9 + (dy+1)*3 + (dx+1).  Forward and backward-data products on the fifth-generation
 *     tensor cores (TMA-staged operands, tcgen05.mma with fp32 accumulators in tensor memory), weight
 *     gradients too (over a packed copy of the operands).
 *   - All pointers are DEVICE pointers borrowed for the call (caller-owned, e.g. torch tensors);
 *     16-byte alignment of every bf16 row is required (ld, off multiples of 8).  Work is enqueued on
 *     `stream` (cudaStream_t, NULL = legacy default stream); nothing synchronises.
 *   - Return PF_OK, PF_E_INVALID for unsupported sizes/alignments (nothing launched) or PF_E_CUDA.
 */
#ifndef PFNN_H
#define PFNN_H
#include "pf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Forward (flip = 0): y[v][co] = act(bias[co] + sum_{t,ci} x[v + off(t)][ci] w[t][co][ci]).
 * (16 or 32 channels in and out on grids of at least 8 x 16 x 4 cells: one shared-memory tile per
 * 8 x 16 x 4 brick, the three taps along z of each lateral offset in one MMA; else one TMA box per tap.)
 * Backward data (flip = 1, w = transposed weights [27][Cin][Cout], cin/cout swapped):
 *   dx[v][ci] = sum_{t,co} dy[v - off(t)][co] w[t][co][ci].
 * cin a multiple of 16; cout a multiple of 16 up to 256; act = ReLU when relu != 0.  ldx, xoff, ldy and
 * yoff multiples of 8, x, w and the output 16-byte aligned.  Output either bf16 (y_bf16) or fp32 (y_f32;
 * accumulate != 0 adds to it).  A kernel whose pipeline wait gives up (bounded; it does not happen in
 * normal operation) finishes without storing and raises the flag that pfnn_status reports. */
pf_status pfnn_conv3d(const void* x, int ldx, int xoff, const void* w, int cin, int cout, const float* bias, int relu,
                      int flip, void* y_bf16, float* y_f32, int ldy, int yoff, int accumulate, int n, int d, int h,
                      int wd, void* stream);

/* Reads and clears the device flag of the tensor-core convolutions (1 = a pipeline wait gave up since
 * the last call, so some output was not written).  Returns PF_E_TIMEOUT when the flag was set, PF_OK
 * when not (PF_E_CUDA if it cannot be read).  Synchronous: waits for the device. */
pf_status pfnn_status(int* failed);

/* Test of the failure path (no counterpart in the paper): the NEXT pfnn_conv3d call withholds the TMA
 * loads of pipeline stage `stage` (0 <= stage < 27 * cin / ck) and bounds every pipeline wait by `tries`
 * (1 <= tries <= 2^24) instead of 2^24.  The waits for that stage then give up: the call finishes
 * without storing its output, TMEM freed after every issued MMA has retired, and pfnn_status reports
 * it.  The setting applies to one call only.  Nothing faults: the withheld stage is an empty wait.
 * Layers of 16 or 32 channels in and out on grids of at least 8 x 16 x 4 (W x H x D) run the halo-tile
 * kernel, which loads one tile per block: there any stage >= 0 withholds that tile. */
pf_status pfnn_test_withhold_stage(int stage, long long tries);

/* Weight gradient: dw[t][co][ci] += sum_v dy[v][co] x[v + off(t)][ci], on the fifth-generation tensor cores:
 * dy and x are packed channel-major over the zero-padded grid (dy three times, shifted by dx = -1, 0, 1) in
 * the caller-owned device scratch `work` (16-byte aligned, at least pfnn_conv3d_wgrad_work_bytes bytes,
 * overwritten), then a GEMM over the packed voxels with rows (tap, co) -- 128 / cout taps per MMA tile --
 * and columns ci accumulates in TMEM; each CTA adds its voxel chunk's partial sums into dw with FP32
 * atomics.  cout in {16, 32, 64, 128}, cin a multiple of 16 up to 256. */
long long pfnn_conv3d_wgrad_work_bytes(int cout, int cin, int n, int d, int h, int wd);
pf_status pfnn_conv3d_wgrad(const void* dy, int lddy, int dyoff, int cout, const void* x, int ldx, int xoff, int cin,
                            float* dw, int n, int d, int h, int wd, void* work, long long work_bytes, void* stream);

/* db[c] += sum_v dz[v][off + c]  (dz fp32 with ld channels per voxel). */
pf_status pfnn_bias_grad(const float* dz, int ld, int off, int c, long long nvox, float* db, void* stream);

/* ReLU backward and cast: dz[v][c] = dy[v][off + c] * (y[v][yoff + c] > 0) (y may be NULL: no mask);
 * dz_f32 (may be NULL) and dz_bf16 are compact [nvox][c]. */
pf_status pfnn_relu_bwd_cast(const float* dy, int lddy, int dyoff, const void* y, int ldy, int yoff, int c,
                             long long nvox, float* dz_f32, void* dz_bf16, void* stream);

/* [27][Cout][Cin] -> [27][Cin][Cout] (weights for the backward-data convolution). */
pf_status pfnn_weight_transpose(const void* w, void* wt, int cout, int cin, void* stream);

/* 2x2x2 average pooling (even D, H, W of the input) and its adjoint (dy compact, dx += strided). */
pf_status pfnn_avgpool(const void* x, int ldx, int xoff, void* y, int ldy, int yoff, int c, int n, int d, int h, int wd,
                       void* stream);
pf_status pfnn_avgpool_bwd(const float* dy, int c, float* dx, int lddx, int dxoff, int n, int d, int h, int wd,
                           void* stream);

/* x2 nearest-neighbour upsampling (d, h, wd = OUTPUT size) and its adjoint (d, h, wd = coarse size,
 * dx compact +=). */
pf_status pfnn_upsample(const void* x, int c, void* y, int ldy, int yoff, int n, int d, int h, int wd, void* stream);
pf_status pfnn_upsample_bwd(const float* dy, int lddy, int dyoff, int c, float* dx, int n, int d, int h, int wd,
                            void* stream);

/* 1x1x1 head: logit[v] = b[0] + sum_c x[v][c] w[c] (c <= 32), prob = sigmoid(logit) (may be NULL).  With a
 * target (fp32, may be NULL): *loss += mean binary cross-entropy, dlogit[v] = (prob - target)/nvox. */
pf_status pfnn_head_forward(const void* x, int c, const float* w, const float* b, const float* target, long long nvox,
                            float* prob, float* dlogit, double* loss, void* stream);
/* dx[v][c] = dlogit[v] w[c] (compact), dw[c] += sum_v dlogit[v] x[v][c], db[0] += sum_v dlogit[v]. */
pf_status pfnn_head_backward(const void* x, int c, const float* w, const float* dlogit, long long nvox, float* dx,
                             float* dw, float* db, void* stream);

/* Network input (16 channels, compact): channel 0 = G[v] (fp32 glass field), channels 1..nfeat =
 * feat[sample][f] (fp32, sample = v / vox_per_sample), the rest 0. */
pf_status pfnn_pack_input(const float* G, const float* feat, int nfeat, long long vox_per_sample, long long nvox,
                          void* out, void* stream);

/* Adam step (bias-corrected, step >= 1) on fp32 master weights p with gradient g and moments m, v;
 * p_bf16 (may be NULL) receives the rounded working copy. */
pf_status pfnn_adam(float* p, const float* g, float* m, float* v, void* p_bf16, long long n, float lr, float b1,
                    float b2, float eps, int step, void* stream);

/* Warm-start constraint (the micro-scale model of Sec. 2.4 has no nucleation term: ice only exists where
 * it grew from the seed through the pore space).  From the network output prob (device fp32, n1 n2 n3,
 * x fastest), the seed phase field phi_seed and the glass field G (device binary64): the cells that may
 * carry ice are those with prob > 1/2 and a water indicator 1 - zeta G above zero, eroded by `erode` cells
 * (0..64; throats narrower than about twice that are cut); the ones connected to the seed (phi_seed > 1/2)
 * through face neighbours, grown back by `erode` cells inside the predicted ice and by `halo` cells (0..64)
 * beyond it to keep the diffuse interface, take max(prob clamped to [0, 1], phi_seed); every other cell
 * takes phi_seed (cells with a zero water indicator never change).  work: caller-owned device scratch of
 * at least 16 * ceil(n / 16) + 4 bytes.  The flood fill sweeps in place until a sweep reaches no new cell
 * (checked every 16 sweeps; bounded by the cell count); *sweeps (may be NULL) receives the sweeps run.
 * Synchronises `stream`. */
pf_status pfnn_seed_connect(const float* prob, const double* phi_seed, const double* G, int n1, int n2, int n3,
                            double zeta, int erode, int halo, unsigned char* work, double* phi_out, void* stream,
                            long long* sweeps);

/* ---- The warm-start network as one object (pfnn_net): the 3D convolutional encoder-decoder of 4 levels
 * (16/32/64/128 channels; two 3x3x3 convolutions + ReLU per level, 2x2x2 average pooling down, x2 nearest
 * upsampling + 3x3x3 convolution up, skip concatenation, 1x1x1 sigmoid head) that predicts the micro-scale
 * equilibrium phase field from the glass field and two features (supercooling, surface-tension scale).
 * The library owns the FP32 master weights, their BF16 working copies, the gradients, the Adam moments and
 * the activation buffers (allocated with cudaMalloc at creation and on the first forward of a new batch
 * shape); forward, backward and the Adam step are sequences of the kernels above on the net's stream.
 * Parameters are numbered 0 .. pfnn_net_params() - 1 in forward order (the last is the head);
 * convolution weights are [27][cout][cin], the head's [16] with one bias.
 *   create  : He-normal weights (std sqrt(2 / (27 cin)); the head sqrt(1/16)) from a splitmix64/Box-Muller
 *             stream seeded by `seed`, zero biases; stream = cudaStream_t (NULL = legacy default stream).
 *   forward : G fp32 [n][side^3] (glass field, x fastest), feat fp32 [n][2], DEVICE pointers; side a
 *             multiple of 8, >= 8; prob (device, n side^3 fp32) receives the sigmoid output.  With a target
 *             (device fp32, NULL = none) it also forms the mean binary cross-entropy (pfnn_net_loss) and
 *             keeps what pfnn_net_backward needs.  pfnn_net_infer = forward without a target.
 *   backward: gradients of that loss into every parameter (PF_E_STATE without a forward with a target).
 *   set/get : host arrays, synchronous.  Errors: PF_E_INVALID, PF_E_OOM, PF_E_CUDA, PF_E_STATE; the failing
 *             step is named by pfnn_net_last_error. */
typedef struct pfnn_net pfnn_net;
int pfnn_net_params(void);
const char* pfnn_net_param_name(int q);
pf_status pfnn_net_param_shape(int q, int* cin, int* cout);
pf_status pfnn_net_create(unsigned long long seed, void* stream, pfnn_net** out);
pf_status pfnn_net_destroy(pfnn_net* net);
pf_status pfnn_net_set_params(pfnn_net* net, int q, const float* w, const float* b);
pf_status pfnn_net_get_params(pfnn_net* net, int q, float* w, float* b);
pf_status pfnn_net_get_grads(pfnn_net* net, int q, float* gw, float* gb);
pf_status pfnn_net_forward(pfnn_net* net, const float* G, const float* feat, int n, int side, const float* target,
                           float* prob);
pf_status pfnn_net_infer(pfnn_net* net, const float* G, const float* feat, int n, int side, float* prob);
pf_status pfnn_net_loss(pfnn_net* net, double* loss);
pf_status pfnn_net_backward(pfnn_net* net);
pf_status pfnn_net_adam_step(pfnn_net* net, float lr, float b1, float b2, float eps);
const char* pfnn_net_last_error(const pfnn_net* net);
/* Inspection of the wiring and of the buffers of the last forward / backward: pfnn_net_layer fills
 * wiring[12] = {input buffer, input channel offset, cin, output buffer, output offset, cout, level, pre (0
 * none, 1 pooling, 2 upsampling), pre input buffer, pre channels, pre output buffer, pre level} for
 * convolution q < pfnn_net_params() - 1; buffer b (0 <= b < pfnn_net_buffers()) holds bf16 activations and
 * fp32 gradients with `channels` per voxel at side >> level; pfnn_net_read_buffer copies them to host
 * arrays of n (side >> level)^3 channels values (PF_E_STATE before the first forward). */
int pfnn_net_buffers(void);
pf_status pfnn_net_layer(int q, int* wiring);
pf_status pfnn_net_buffer(int b, int* channels, int* level);
pf_status pfnn_net_read_buffer(pfnn_net* net, int b, void* act_bf16, float* grad);

#ifdef __cplusplus
}
#endif
#endif /* PFNN_H */
