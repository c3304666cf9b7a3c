// 3x3x3 convolution (forward and backward-data) of the learned warm start as an implicit GEMM on
// the fifth-generation tensor cores of sm_103a: TMA brings the operand tiles into shared memory,
// tcgen05.mma accumulates in tensor memory (TMEM), tcgen05.ld reads the accumulator back for the
// epilogue.
//
// GEMM view (forward): D[v][co] = sum over taps t and input channels ci of X[v + off(t)][ci] W[t][co][ci]
//   M = 128 voxels of one brick (wb x hb x db cells of one sample), N = cout, K = 27 taps x cin.
// Backward data is the same GEMM on dY with flipped taps and the transposed weights [27][cin][cout].
//
// A operand: one TMA box of the channels-last activation tensor per (tap, channel block): the brick
// shifted by the tap offset, ck channels deep.  Cells outside the grid (the convolution's zero
// padding) are filled with zeros by the TMA unit itself.  The box lands in shared memory as 128 rows
// (voxels, x fastest) of ck bf16 channels, swizzled with the pattern whose span equals the row length
// (32, 64 or 128 bytes), which is the K-major layout the MMA descriptors name.
// B operand: the [cout][ck] weight slice of the same tap and channel block (K-major, same swizzle).
//
// Roles (4 warps): thread 0 issues the TMA loads into a ring of shared-memory stages, thread 32 issues
// the MMAs (one per 16 channels) and commits each stage back to the producer, warp 2 owns the TMEM
// allocation; all four warps then read the 128 x cout fp32 accumulator (warp w owns TMEM lanes
// 32w..32w+31 = voxels 32w..32w+31 of the brick) and apply bias, ReLU and the bf16 or fp32 store.
// Every wait on an mbarrier gives up after a bounded number of tries, records the failure in a device
// flag (read by pfnn_status) and lets the block finish: no wait can hang the GPU.
#include "../../include/pfnn.h"
#include "pf_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

namespace {

using bf16 = __nv_bfloat16;

constexpr int UM = 128;     // MMA M: voxels per tile
constexpr int UTHR = 128;   // threads per block (4 warps)
constexpr long long WAIT_TRIES = 1LL << 24;

// Test-only setting of the failure-path test, consumed by the next pfnn_conv3d call: the producer
// withholds the TMA loads of one stage and every wait gives up after g_test_tries tries.
static int g_test_withhold = -1;
static long long g_test_tries = 0;

__device__ int g_umma_status = 0;  // 0 = ok; 1 = an mbarrier wait gave up

struct UmmaArgs {
    int cin, cout, ck, nkb;       // channels in/out, channels per k block, k blocks per tap
    int wb, hb, db;               // brick (wb * hb * db = 128)
    int D, H, W;                  // grid of one sample
    int tx, ty, tz;               // bricks per sample along x, y, z
    int flip, relu, accumulate;
    int stages;
    int withhold;                 // stage whose loads are withheld (test of the failure path), -1 = none
    long long tries;              // bound of every mbarrier wait
    unsigned a_bytes, stage_bytes;  // shared-memory footprint of the A tile and of one stage (1024-byte units)
    unsigned tx_bytes;              // bytes the two TMA loads of one stage deliver
    unsigned idesc;               // MMA instruction descriptor
    unsigned long long desc_hi;   // constant high bits of the shared-memory descriptors
    int tmem_cols;
    const float* bias;
    bf16* y;
    float* yf;
    int ldy, yoff;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait for the phase of the given parity to complete; false (and the device flag set) after WAIT_TRIES.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long tries) {
    for (long long it = 0; it < tries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    atomicExch(&g_umma_status, 1);
    return false;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6, %7}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

// Shared-memory matrix descriptor: start address (bits 0-13, in 16-byte units) over the constant
// part (stride between 8-row groups, descriptor version, swizzle mode).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, unsigned long long hi) {
    return hi | (uint64_t)((addr >> 4) & 0x3FFFu);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__global__ void __launch_bounds__(UTHR)
k_conv_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const UmmaArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // stage tiles start on 1024-byte boundaries of the shared window (the swizzle patterns repeat there)
    unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int S = p.stages;
    unsigned char* ctl = sm + (size_t)S * p.stage_bytes;  // barriers and the TMEM address slot
    const uint32_t full0 = smem_u32(ctl);                  // full[s]  at full0  + 8 s
    const uint32_t empty0 = full0 + 8u * S;                // empty[s] at empty0 + 8 s
    const uint32_t accum = empty0 + 8u * S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctl + 16 * S + 8);
    __shared__ int s_fail;  // the MMA issuer gave up a wait: the accumulator is incomplete

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // brick of this block
    long long b = blockIdx.x;
    const int bx = (int)(b % p.tx);
    b /= p.tx;
    const int by = (int)(b % p.ty);
    b /= p.ty;
    const int bz = (int)(b % p.tz);
    const int bn = (int)(b / p.tz);
    const int x0 = bx * p.wb, y0 = by * p.hb, z0 = bz * p.db;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8u * s, 1);
            mbar_init(empty0 + 8u * s, 1);
        }
        mbar_init(accum, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int KB = 27 * p.nkb;
    const uint32_t sm0 = smem_u32(sm);

    int issued = 0;  // TMA stages issued (thread 0)
    if (threadIdx.x == 0) {
        // ---- producer: one stage = the A box and the B slice of one (tap, channel block)
        for (int kb = 0; kb < KB; ++kb, ++issued) {
            const int s = kb % S;
            const uint32_t use = (uint32_t)(kb / S);
            if (kb >= S && !mbar_wait(empty0 + 8u * s, (use & 1u) ^ 1u, p.tries)) break;
            const uint32_t fb = full0 + 8u * s;
            mbar_expect_tx(fb, p.tx_bytes);
            if (kb == p.withhold) continue;  // test of the failure path: this stage never fills
            const int tap = kb / p.nkb, cb = kb - tap * p.nkb;
            int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            if (p.flip) { dz = -dz; dy = -dy; dx = -dx; }
            const uint32_t a_dst = sm0 + (uint32_t)s * p.stage_bytes;
            tma_load_5d(a_dst, &tmA, fb, cb * p.ck, x0 + dx, y0 + dy, z0 + dz, bn);
            tma_load_2d(a_dst + p.a_bytes, &tmB, fb, cb * p.ck, tap * p.cout);
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer: ck / 16 MMAs (K = 16 each) per stage, accumulating into TMEM
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            const int s = kb % S;
            const uint32_t use = (uint32_t)(kb / S);
            ok = mbar_wait(full0 + 8u * s, use & 1u, p.tries);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_addr = sm0 + (uint32_t)s * p.stage_bytes;
            const uint32_t b_addr = a_addr + p.a_bytes;
            for (int k = 0; k < p.ck / 16; ++k) {
                // K step k starts 32 bytes further along the (swizzled) rows
                umma_f16(tmem, sdesc(a_addr + 32u * k, p.desc_hi), sdesc(b_addr + 32u * k, p.desc_hi), p.idesc,
                         (kb > 0 || k > 0) ? 1u : 0u);
            }
            umma_commit(empty0 + 8u * s);
        }
        // the accumulator barrier completes once every MMA issued above has retired, also after a
        // failed wait: TMEM and the stages are not released while an MMA may still use them
        if (!ok) s_fail = 1;
        umma_commit(accum);
    }
    __syncwarp();
    __syncthreads();  // s_fail is visible to every thread

    // ---- epilogue: warp w reads TMEM lanes 32w..32w+31 (voxels of the brick), 16 columns at a time
    const bool ready = mbar_wait(accum, 0u, p.tries) && !s_fail;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = warp * 32 + lane;
    const int dx = m % p.wb, dy = (m / p.wb) % p.hb, dz = m / (p.wb * p.hb);
    const int x = x0 + dx, y = y0 + dy, z = z0 + dz;
    const bool inside = ready && x < p.W && y < p.H && z < p.D;
    const long long v = (((long long)bn * p.D + z) * p.H + y) * p.W + x;
    for (int c0 = 0; c0 < p.cout; c0 += 16) {
        float o[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, o);  // whole warp, always
        if (!inside) continue;
        if (p.bias) {
#pragma unroll
            for (int q = 0; q < 16; ++q) o[q] += p.bias[c0 + q];
        }
        if (p.relu) {
#pragma unroll
            for (int q = 0; q < 16; ++q) o[q] = fmaxf(o[q], 0.f);
        }
        if (p.yf) {
            float4* dst = reinterpret_cast<float4*>(p.yf + v * p.ldy + p.yoff + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 w = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
                if (p.accumulate) {
                    const float4 r = dst[q];
                    w.x += r.x; w.y += r.y; w.z += r.z; w.w += r.w;
                }
                dst[q] = w;
            }
        } else {
            uint4 pk[2];
            uint32_t* u = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(o[2 * q], o[2 * q + 1]);
                u[q] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            uint4* dst = reinterpret_cast<uint4*>(p.y + v * p.ldy + p.yoff + c0);
            dst[0] = pk[0];
            dst[1] = pk[1];
        }
    }

    // after a failed wait, the TMA loads still in flight must land before the block's shared memory
    // is released (bounded as well); on success the completed accumulation implies that they have
    if (threadIdx.x == 0 && !ready) {
        for (int kb = issued - S < 0 ? 0 : issued - S; kb < issued; ++kb)
            mbar_wait(full0 + 8u * (kb % S), (uint32_t)(kb / S) & 1u, p.tries);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------- narrow layers: one halo tile per brick
// For 16 or 32 channels the per-tap boxes of k_conv_umma are 32- or 64-byte rows and the 27 boxes of a
// 128-voxel tile move 27 times its input through TMA.  Here a block loads the input of its whole brick
// (8 x 16 x DZ cells, x fastest) once, with a one-cell halo: a (DZ + 2) x 18 x 10 tile per 8-channel
// chunk, unswizzled, so that every cell is a 16-byte row and a row of 10 cells is 160 contiguous bytes.
// The A operand is a window of that tile: for tile plane z' and lateral offset (dy, dx), the 128 rows
// (8 x by 16 y) start at cell (dx + 1, dy + 1, z'); 8 consecutive x cells are one 8 x 16-byte core
// matrix, consecutive y rows are 160 bytes apart (the stride between core matrices along M) and
// consecutive 8-channel chunks one chunk apart (the stride along K); the start is a multiple of 16 bytes,
// as the unswizzled layout requires.  One window serves the three taps (dz = -1, 0, +1) of its (dy, dx):
// tile plane z' feeds output planes o = z' - 1 - dz.  The B operand stacks the three taps' weights along
// N (3 cout rows: dz = -1, 0, +1), and the accumulators of the output planes lie in TMEM at decreasing
// columns, plane o at (DZ + 1 - o) cout, so the three column groups of one MMA are the accumulators of
// planes z', z' - 1 and z' - 2 (planes -2, -1, DZ and DZ + 1 are scratch).  Per brick: (DZ + 2) x 9 x
// cin/16 MMAs of M = 128, N = 3 cout, K = 16 (a third of the A reads from shared memory of one MMA per
// tap); the accumulators start from zero written by tcgen05.st.  The weights of all taps stay in shared
// memory as [dy, dx][chunk][dz, cout][8 channels]; backward data (flipped taps) copies tap 26 - t there.
struct HaloArgs {
    int cin, cout, dz_planes;     // channels in/out, output planes per brick
    int D, H, W;                  // grid of one sample
    int tx, ty, tz;               // bricks per sample
    int flip, relu, accumulate;
    int withhold;                 // >= 0: the tile loads are withheld (failure-path test)
    long long tries;
    unsigned chunk_bytes;         // shared bytes of one 8-channel chunk of the tile (1024-byte multiple)
    unsigned tile_bytes;          // all chunks
    unsigned w_bytes;             // weights of all taps
    unsigned tx_bytes;            // bytes the tile loads deliver
    unsigned idesc;
    int tmem_cols;
    const float* bias;
    const bf16* w;
    bf16* y;
    float* yf;
    int ldy, yoff;
};

constexpr int HB_X = 8, HB_Y = 16;            // brick extent along x and y (one plane = 128 voxels)
constexpr int HT_X = HB_X + 2, HT_Y = HB_Y + 2;
constexpr unsigned HT_ROW = HT_X * 16;        // bytes of one tile row of 8 channels

// unswizzled K-major descriptor: start, stride along K (LBO) and along M/N (SBO), version 1
__device__ __forceinline__ uint64_t desc_plain(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ULL << 46);
}

// tcgen05.mma with the descriptors given as 32-bit words (the issue loop advances the low words only)
__device__ __forceinline__ void umma_f16_w(uint32_t tmem_d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "mov.b64 da, {%1, %2};\n\t"
        "mov.b64 db, {%3, %4};\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}" ::"r"(tmem_d),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The MMAs of one brick.  a_lo / b_lo: low descriptor words of the tile and weight bases; the start field
// (bits 0-13, 16-byte units) is advanced by adding to the low word (the shared window lies below 256 KB,
// so it never carries out).
template <int NKB>
__device__ __forceinline__ void halo_issue(uint32_t tmem, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t b_hi,
                                           uint32_t idesc, int planes, int cout, uint32_t chunk16) {
    for (int zt = 0; zt < planes + 2; ++zt) {
        const uint32_t d = tmem + (uint32_t)((planes + 1 - zt) * cout);  // accumulator of output plane zt
        const uint32_t a_z = a_lo + (uint32_t)(zt * HT_Y * HT_X);
#pragma unroll
        for (int l = 0; l < 9; ++l) {  // l = 3 (dy + 1) + (dx + 1)
            const uint32_t off = (uint32_t)((l / 3) * HT_X + l % 3);
#pragma unroll
            for (int kb = 0; kb < NKB; ++kb)
                umma_f16_w(d, a_z + off + (uint32_t)(2 * kb) * chunk16, a_hi,
                           b_lo + (uint32_t)((l * 2 * NKB + 2 * kb) * 3 * cout), b_hi, idesc, 1u);
        }
    }
}

// Weights of all taps into shared memory as [dy, dx][chunk][dz, cout][8] (tap t = 9 (dz + 1) + l,
// l = 3 (dy + 1) + (dx + 1); flipped: the tap 26 - t), in rounds of 7 16-byte vectors per thread: each
// round loads all of its vectors (read-only path) before storing them, so the copy costs one round trip
// to L2 per 14 KB (one for 16 x 16 channels, four for 32 x 32).
__device__ __forceinline__ void halo_weights(const bf16* __restrict__ w, unsigned char* dst, int cout, int nkc,
                                             int flip) {
    constexpr int CAP = 7;
    const int nvec = 27 * cout * nkc;
    const uint4* src = reinterpret_cast<const uint4*>(w);
    for (int base = 0; base < nvec; base += CAP * UTHR) {
        uint4 v[CAP];
#pragma unroll
        for (int j = 0; j < CAP; ++j) {
            const int q = base + threadIdx.x + j * UTHR;
            if (q < nvec) v[j] = __ldg(src + q);
        }
#pragma unroll
        for (int j = 0; j < CAP; ++j) {
            const int q = base + threadIdx.x + j * UTHR;
            if (q < nvec) {
                const int kc = q % nkc;
                const int co = (q / nkc) % cout;
                int t = q / (nkc * cout);
                if (flip) t = 26 - t;
                const int dzi = t / 9, l = t % 9;
                *reinterpret_cast<uint4*>(dst + ((size_t)(l * nkc + kc) * 3 * cout + dzi * cout + co) * 16) = v[j];
            }
        }
    }
}

// zero the accumulator columns [0, cols) of this warp's TMEM lane quadrant
__device__ __forceinline__ void tmem_zero(uint32_t taddr, int cols) {
    const uint32_t z = 0u;
    for (int c = 0; c < cols; c += 16)
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1, %1};" ::"r"(taddr + (uint32_t)c), "r"(z)
            : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// One block per brick: thread 0 issues the tile's TMA loads (one box per 8-channel chunk, zero fill
// outside the grid) while all threads copy the weights; thread 32 issues the MMAs once the tile has
// landed and commits them to one barrier; all four warps read the accumulators (bias and ReLU applied
// from registers).  Three or two blocks share an SM (shared memory), so one block's loads overlap
// another's MMAs and epilogue.  Both waits are bounded.
__global__ void __launch_bounds__(UTHR)
k_conv_halo(const __grid_constant__ CUtensorMap tmX, const HaloArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* ctl = sm + p.tile_bytes + p.w_bytes;
    const uint32_t full = smem_u32(ctl);
    const uint32_t accum = full + 8u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctl + 16);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkc = p.cin / 8;
    long long b = blockIdx.x;
    const int bx = (int)(b % p.tx);
    b /= p.tx;
    const int by = (int)(b % p.ty);
    b /= p.ty;
    const int bz = (int)(b % p.tz);
    const int bn = (int)(b / p.tz);
    const int x0 = bx * HB_X, y0 = by * HB_Y, z0 = bz * p.dz_planes;
    const uint32_t tile0 = smem_u32(sm);
    const uint32_t w0 = tile0 + p.tile_bytes;

    if (threadIdx.x == 0) {
        mbar_init(full, 1);
        mbar_init(accum, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(full, p.tx_bytes);
        if (p.withhold < 0) {  // failure-path test: the tile never arrives
            for (int kc = 0; kc < nkc; ++kc)
                tma_load_5d(tile0 + (uint32_t)kc * p.chunk_bytes, &tmX, full, kc * 8, x0 - 1, y0 - 1, z0 - 1, bn);
        }
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    halo_weights(p.w, sm + p.tile_bytes, p.cout, nkc, p.flip);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the TMEM address is in shared memory
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem_zero(*tmem_slot + ((uint32_t)(warp * 32) << 16), (p.dz_planes + 4) * p.cout);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 32) {
        const bool ok = mbar_wait(full, 0u, p.tries);
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = desc_plain(tile0, p.chunk_bytes, HT_ROW);
            const uint64_t db = desc_plain(w0, 3u * (uint32_t)p.cout * 16u, 128u);
            const uint32_t alo = (uint32_t)da, ahi = (uint32_t)(da >> 32), blo = (uint32_t)db, bhi = (uint32_t)(db >> 32);
            const uint32_t c16 = p.chunk_bytes >> 4;
            if (nkc == 2) halo_issue<1>(tmem, alo, ahi, blo, bhi, p.idesc, p.dz_planes, p.cout, c16);
            else halo_issue<2>(tmem, alo, ahi, blo, bhi, p.idesc, p.dz_planes, p.cout, c16);
        } else {
            s_fail = 1;
        }
        umma_commit(accum);  // also after a failed wait: every issued MMA has retired when it completes
    }
    __syncwarp();
    __syncthreads();

    const bool ready = mbar_wait(accum, 0u, p.tries) && !s_fail;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = warp * 32 + lane;           // accumulator row: x = m % 8, y = m / 8
    const int x = x0 + (m % HB_X), y = y0 + m / HB_X;
    const bool inxy = ready && x < p.W && y < p.H;
    for (int c0 = 0; c0 < p.cout; c0 += 16) {
        float bias[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) bias[q] = p.bias ? __ldg(p.bias + c0 + q) : 0.f;
        for (int zo = 0; zo < p.dz_planes; ++zo) {
            const int z = z0 + zo;
            const bool inside = inxy && z < p.D;
            const long long v = (((long long)bn * p.D + z) * p.H + y) * p.W + x;
            float o[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((p.dz_planes + 1 - zo) * p.cout + c0), o);
            if (!inside) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) o[q] += bias[q];
            if (p.relu) {
#pragma unroll
                for (int q = 0; q < 16; ++q) o[q] = fmaxf(o[q], 0.f);
            }
            if (p.yf) {
                float4* dst = reinterpret_cast<float4*>(p.yf + v * p.ldy + p.yoff + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 w = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
                    if (p.accumulate) {
                        const float4 r = dst[q];
                        w.x += r.x; w.y += r.y; w.z += r.z; w.w += r.w;
                    }
                    dst[q] = w;
                }
            } else {
                uint4 pk[2];
                uint32_t* u = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(o[2 * q], o[2 * q + 1]);
                    u[q] = *reinterpret_cast<const uint32_t*>(&h2);
                }
                uint4* dst = reinterpret_cast<uint4*>(p.y + v * p.ldy + p.yoff + c0);
                dst[0] = pk[0];
                dst[1] = pk[1];
            }
        }
    }
    // a tile load still in flight after a failed wait lands before the shared memory is released
    if (threadIdx.x == 0 && !ready && p.withhold < 0) mbar_wait(full, 0u, p.tries);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------- weight gradient on tcgen05
// dW[t][co][ci] = sum over voxels v of dY[v][co] X[v + off(t)][ci] (zero padding) is, with u = v + off(t),
// sum over u of dY[u - off(t)][co] X[u][ci]: a GEMM whose reduction runs over voxels.  Both tensors are
// first packed channel-major over a zero-padded grid (rows of W' = W + 2 rounded up to 8 cells, planes of
// (H + 2) W', samples of (D + 2) planes), so that a tap's offset is a constant shift of the packed voxel
// index; dY is packed three times, shifted by dx = -1, 0, +1, so that the remaining shift
// dz (H + 2) W' + dy W' keeps the TMA coordinate a multiple of 8 elements (16 bytes).
//   A (M = 128 rows): 128 / cout taps x cout output channels; tap j's rows are one TMA box of the dx-copy,
//                     64 voxels wide, shifted by the tap's offset (out-of-range voxels filled with zeros);
//   B (N = cin):      one TMA box of the packed X, 64 voxels wide;
//   K:                the packed voxels of the CTA's chunk, 64 per pipeline stage (4 MMAs of K = 16).
// Both operands are K-major with 128-byte rows (the 128-byte swizzle), as in k_conv_umma.  Each CTA adds
// its chunk's partial products into dW with FP32 atomics (split over voxel chunks).
struct WgArgs {
    int cout, cin, taps_per_tile;
    int kb_per_cta;               // k blocks (of 64 packed voxels) per CTA
    long long nkb;                // k blocks in total
    int plane_p, row_p;           // packed plane and row lengths
    int stages;
    unsigned a_bytes, stage_bytes;
    unsigned idesc;
    unsigned long long desc_hi;
    int tmem_cols;
    long long tries;
    float* dw;
};

__global__ void __launch_bounds__(UTHR)
k_wgrad_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const WgArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int S = p.stages;
    unsigned char* ctl = sm + (size_t)S * p.stage_bytes;
    const uint32_t full0 = smem_u32(ctl);
    const uint32_t empty0 = full0 + 8u * S;
    const uint32_t accum = empty0 + 8u * S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctl + 16 * S + 8);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t0 = blockIdx.x * p.taps_per_tile;
    const int ntap = min(p.taps_per_tile, 27 - t0);
    const long long kb0 = (long long)blockIdx.y * p.kb_per_cta;
    const int KB = (int)min((long long)p.kb_per_cta, p.nkb - kb0);
    const unsigned tx_bytes = (unsigned)(ntap * p.cout * 128 + p.cin * 128);

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8u * s, 1);
            mbar_init(empty0 + 8u * s, 1);
        }
        mbar_init(accum, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t sm0 = smem_u32(sm);

    int issued = 0;
    if (threadIdx.x == 0) {
        // ---- producer: one stage = the ntap shifted dY boxes and the X box of 64 packed voxels
        for (int kb = 0; kb < KB; ++kb, ++issued) {
            const int s = kb % S;
            const uint32_t use = (uint32_t)(kb / S);
            if (kb >= S && !mbar_wait(empty0 + 8u * s, (use & 1u) ^ 1u, p.tries)) break;
            const uint32_t fb = full0 + 8u * s;
            mbar_expect_tx(fb, tx_bytes);
            const int k0 = (int)((kb0 + kb) * 64);
            const uint32_t a_dst = sm0 + (uint32_t)s * p.stage_bytes;
            for (int j = 0; j < ntap; ++j) {
                const int t = t0 + j;
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                tma_load_2d(a_dst + (uint32_t)(j * p.cout * 128), &tmA, fb, k0 - (dz * p.plane_p + dy * p.row_p),
                            (dx + 1) * p.cout);
            }
            tma_load_2d(a_dst + p.a_bytes, &tmB, fb, k0, 0);
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer: 4 MMAs (K = 16 packed voxels each) per stage into the TMEM accumulator
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            const int s = kb % S;
            const uint32_t use = (uint32_t)(kb / S);
            ok = mbar_wait(full0 + 8u * s, use & 1u, p.tries);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_addr = sm0 + (uint32_t)s * p.stage_bytes;
            const uint32_t b_addr = a_addr + p.a_bytes;
            for (int k = 0; k < 4; ++k)
                umma_f16(tmem, sdesc(a_addr + 32u * k, p.desc_hi), sdesc(b_addr + 32u * k, p.desc_hi), p.idesc,
                         (kb > 0 || k > 0) ? 1u : 0u);
            umma_commit(empty0 + 8u * s);
        }
        if (!ok) s_fail = 1;
        umma_commit(accum);
    }
    __syncwarp();
    __syncthreads();

    // ---- epilogue: TMEM lane r = row (tap t0 + r / cout, channel r % cout), columns = input channels
    const bool ready = mbar_wait(accum, 0u, p.tries) && !s_fail && KB > 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int r = warp * 32 + lane;
    const int j = r / p.cout, co = r - j * p.cout;
    const bool live = ready && j < ntap;
    for (int c0 = 0; c0 < p.cin; c0 += 16) {
        float o[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, o);  // whole warp, always
        if (!live) continue;
        float* dst = p.dw + ((long long)(t0 + j) * p.cout + co) * p.cin + c0;
#pragma unroll
        for (int q = 0; q < 16; ++q) atomicAdd(dst + q, o[q]);
    }

    if (threadIdx.x == 0 && !ready) {
        for (int kb = issued - S < 0 ? 0 : issued - S; kb < issued; ++kb)
            mbar_wait(full0 + 8u * (kb % S), (uint32_t)(kb / S) & 1u, p.tries);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
    }
}

// Packing for the weight gradient: X and the three dx-shifted copies of dY, channel-major over the padded
// grid (see k_wgrad_umma); the buffers are zeroed before, so the padding stays zero.
__global__ void k_wgrad_pack(const __nv_bfloat16* __restrict__ dy, int lddy, int dyoff, int cout,
                             const __nv_bfloat16* __restrict__ x, int ldx, int xoff, int cin, int D, int H, int W,
                             int Wp, long long nvox, long long vp64, __nv_bfloat16* __restrict__ A3,
                             __nv_bfloat16* __restrict__ XB) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const int xx = (int)(v % W);
        long long q = v / W;
        const int yy = (int)(q % H);
        q /= H;
        const int zz = (int)(q % D);
        const long long b = q / D;
        const long long vp = ((b * (D + 2) + zz + 1) * (H + 2) + yy + 1) * (long long)Wp + xx + 1;
        for (int c = 0; c < cout; ++c) {
            const __nv_bfloat16 val = dy[v * lddy + dyoff + c];
            for (int d = 0; d < 3; ++d) A3[((long long)d * cout + c) * vp64 + vp + (d - 1)] = val;
        }
        for (int c = 0; c < cin; ++c) XB[(long long)c * vp64 + vp] = x[v * ldx + xoff + c];
    }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// swizzle span = row length of a k block (ck bf16 = 32, 64 or 128 bytes)
CUtensorMapSwizzle tma_swizzle(int ck) {
    return ck == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : (ck == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
}
// the matching layout code of the MMA shared-memory descriptor (bits 61-63)
unsigned long long umma_layout(int ck) { return ck == 16 ? 6ULL : (ck == 32 ? 4ULL : 2ULL); }

unsigned round1024(unsigned v) { return (v + 1023u) & ~1023u; }

// the narrow-layer kernel takes 16 or 32 channels in and out on grids at least one brick across
bool halo_shape(int cin, int cout, int d, int h, int wd) {
    return (cin == 16 || cin == 32) && (cout == 16 || cout == 32) && wd >= HB_X && h >= HB_Y && d >= 4;
}

pf_status conv_halo(const void* x, int ldx, int xoff, const void* w, int cin, int cout, const float* bias, int relu,
                    int flip, void* y_bf16, float* y_f32, int ldy, int yoff, int accumulate, int n, int d, int h,
                    int wd, cudaStream_t stream, PFN_cuTensorMapEncodeTiled_v12000 enc) {
    HaloArgs a{};
    a.cin = cin;
    a.cout = cout;
    a.D = d;
    a.H = h;
    a.W = wd;
    a.flip = flip;
    a.relu = relu;
    a.accumulate = accumulate;
    a.withhold = g_test_withhold;
    a.tries = g_test_tries > 0 ? g_test_tries : WAIT_TRIES;
    g_test_withhold = -1;
    g_test_tries = 0;
    a.w_bytes = (unsigned)(27 * cout * cin * 2);
    // 4 output planes per brick: 16 -> 16 channels then fit four blocks per SM (48.6 KB of shared memory,
    // 8 x 16 TMEM columns each), the wider layers two (32 x 32: one)
    const int dzp = 4;
    auto chunk = [](int dz) { return round1024((unsigned)(HT_ROW * HT_Y * (dz + 2))); };
    a.dz_planes = dzp;
    a.chunk_bytes = chunk(dzp);
    a.tile_bytes = (unsigned)(cin / 8) * a.chunk_bytes;
    a.tx_bytes = (unsigned)(cin / 8) * (HT_ROW * HT_Y * (dzp + 2));
    a.tx = (wd + HB_X - 1) / HB_X;
    a.ty = (h + HB_Y - 1) / HB_Y;
    a.tz = (d + dzp - 1) / dzp;
    // MMA N = 3 cout: the taps dz = -1, 0, +1 of one lateral offset
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(3 * cout >> 3) << 17) | ((unsigned)(UM >> 4) << 24);
    const int cols = (dzp + 4) * cout;
    a.tmem_cols = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : 256));
    a.bias = bias;
    a.w = (const bf16*)w;
    a.y = (bf16*)y_bf16;
    a.yf = y_f32;
    a.ldy = ldy;
    a.yoff = yoff;
    alignas(64) CUtensorMap mX;
    const cuuint64_t dims[5] = {(cuuint64_t)cin, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)d, (cuuint64_t)n};
    const cuuint64_t row = (cuuint64_t)ldx * 2;
    const cuuint64_t strides[4] = {row, row * wd, row * wd * h, row * wd * h * d};
    const cuuint32_t box[5] = {8, (cuuint32_t)HT_X, (cuuint32_t)HT_Y, (cuuint32_t)(dzp + 2), 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    if (enc(&mX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)((const bf16*)x + xoff), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return PF_E_INVALID;
    const size_t smem = 1024 + (size_t)a.tile_bytes + a.w_bytes + 32;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(k_conv_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (attr_err != cudaSuccess || smem > 200u * 1024u) return PF_E_CUDA;
    const long long blocks = (long long)a.tx * a.ty * a.tz * n;
    if (blocks > 0x7FFFFFFFLL) return PF_E_RANGE;
    k_conv_halo<<<(unsigned)blocks, UTHR, smem, stream>>>(mX, a);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

}  // namespace

extern "C" {

pf_status pfnn_conv3d(const void* x, int ldx, int xoff, const void* w, int cin, int cout, const float* bias, int relu,
                      int flip, void* y_bf16, float* y_f32, int ldy, int yoff, int accumulate, int n, int d, int h,
                      int wd, void* stream) {
    if (!x || !w || (!y_bf16 && !y_f32) || n < 1 || d < 1 || h < 1 || wd < 1) return PF_E_INVALID;
    if (cin < 16 || cin % 16 || cout < 16 || cout % 16 || cout > 256 || ldx % 8 || xoff % 8 || ldx < xoff + cin ||
        ldy % 8 || yoff % 8 || ldy < yoff + cout)
        return PF_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(y_bf16) |
         reinterpret_cast<uintptr_t>(y_f32)) % 16)
        return PF_E_INVALID;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return PF_E_CUDA;
    if (halo_shape(cin, cout, d, h, wd))
        return conv_halo(x, ldx, xoff, w, cin, cout, bias, relu, flip, y_bf16, y_f32, ldy, yoff, accumulate, n, d, h,
                         wd, (cudaStream_t)stream, enc);

    UmmaArgs a{};
    a.cin = cin;
    a.cout = cout;
    a.ck = cin % 64 == 0 ? 64 : (cin % 32 == 0 ? 32 : 16);
    a.nkb = cin / a.ck;
    // brick of 128 cells: 32 x 4 x 1, 16 x 8 x 1 or 8 x 8 x 2 (x fastest), the widest that the grid fills
    a.wb = wd >= 32 ? 32 : (wd >= 16 ? 16 : 8);
    a.hb = a.wb == 32 ? 4 : 8;
    a.db = UM / (a.wb * a.hb);
    a.D = d;
    a.H = h;
    a.W = wd;
    a.tx = (wd + a.wb - 1) / a.wb;
    a.ty = (h + a.hb - 1) / a.hb;
    a.tz = (d + a.db - 1) / a.db;
    a.flip = flip;
    a.relu = relu;
    a.withhold = g_test_withhold;
    a.tries = g_test_tries > 0 ? g_test_tries : WAIT_TRIES;
    g_test_withhold = -1;
    g_test_tries = 0;
    a.accumulate = accumulate;
    a.a_bytes = round1024((unsigned)(UM * a.ck * 2));
    a.stage_bytes = a.a_bytes + round1024((unsigned)(cout * a.ck * 2));
    a.tx_bytes = (unsigned)((UM + cout) * a.ck * 2);
    int stages = (int)(98304u / a.stage_bytes);
    a.stages = stages < 2 ? 2 : (stages > 8 ? 8 : stages);
    // instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
    // both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(cout >> 3) << 17) | ((unsigned)(UM >> 4) << 24);
    // descriptor: leading offset 16 B (unused for swizzled K-major), stride between 8-row groups = 8 rows x
    // row bytes, version 1 (bit 46), swizzle layout code at bits 61-63
    const unsigned long long sbo = (unsigned long long)(8 * a.ck * 2);
    a.desc_hi = (1ULL << 16) | ((sbo >> 4) << 32) | (1ULL << 46) | (umma_layout(a.ck) << 61);
    a.tmem_cols = cout <= 32 ? 32 : (cout <= 64 ? 64 : (cout <= 128 ? 128 : 256));
    a.bias = bias;
    a.y = (bf16*)y_bf16;
    a.yf = y_f32;
    a.ldy = ldy;
    a.yoff = yoff;

    alignas(64) CUtensorMap mA, mB;
    {
        const cuuint64_t dims[5] = {(cuuint64_t)cin, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)d, (cuuint64_t)n};
        const cuuint64_t row = (cuuint64_t)ldx * 2;
        const cuuint64_t strides[4] = {row, row * wd, row * wd * h, row * wd * h * d};
        const cuuint32_t box[5] = {(cuuint32_t)a.ck, (cuuint32_t)a.wb, (cuuint32_t)a.hb, (cuuint32_t)a.db, 1};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)((const bf16*)x + xoff), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, tma_swizzle(a.ck), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return PF_E_INVALID;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)cin, (cuuint64_t)(27 * cout)};
        const cuuint64_t strides[1] = {(cuuint64_t)cin * 2};
        const cuuint32_t box[2] = {(cuuint32_t)a.ck, (cuuint32_t)cout};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(w), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, tma_swizzle(a.ck), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return PF_E_INVALID;
    }
    const size_t smem = (size_t)a.stages * a.stage_bytes + 1024 + 16 * a.stages + 16;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(k_conv_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024 + 2048);
    });
    if (attr_err != cudaSuccess) return PF_E_CUDA;
    const long long blocks = (long long)a.tx * a.ty * a.tz * n;
    if (blocks > 0x7FFFFFFFLL) return PF_E_RANGE;
    k_conv_umma<<<(unsigned)blocks, UTHR, smem, (cudaStream_t)stream>>>(mA, mB, a);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

// packed layout of the weight gradient: padded row W' = W + 2 rounded up to 8, packed voxels rounded to 64
static void wgrad_layout(int n, int d, int h, int wd, int* wp, long long* vp64) {
    *wp = (wd + 2 + 7) / 8 * 8;
    const long long vp = (long long)n * (d + 2) * (h + 2) * (*wp);
    *vp64 = (vp + 63) / 64 * 64;
}

long long pfnn_conv3d_wgrad_work_bytes(int cout, int cin, int n, int d, int h, int wd) {
    if (cout < 1 || cin < 1 || n < 1 || d < 1 || h < 1 || wd < 1) return -1;
    int wp;
    long long vp64;
    wgrad_layout(n, d, h, wd, &wp, &vp64);
    return 2LL * (3LL * cout + cin) * vp64;
}

pf_status pfnn_conv3d_wgrad(const void* dy, int lddy, int dyoff, int cout, const void* x, int ldx, int xoff, int cin,
                            float* dw, int n, int d, int h, int wd, void* work, long long work_bytes, void* stream) {
    if (!dy || !x || !dw || !work || n < 1 || d < 1 || h < 1 || wd < 1) return PF_E_INVALID;
    if ((cout != 16 && cout != 32 && cout != 64 && cout != 128) || cin < 16 || cin % 16 || cin > 256 ||
        lddy < dyoff + cout || ldx < xoff + cin || dyoff < 0 || xoff < 0)
        return PF_E_INVALID;
    if (work_bytes < pfnn_conv3d_wgrad_work_bytes(cout, cin, n, d, h, wd) || reinterpret_cast<uintptr_t>(work) % 16)
        return PF_E_INVALID;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return PF_E_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int wp;
    long long vp64;
    wgrad_layout(n, d, h, wd, &wp, &vp64);
    bf16* A3 = (bf16*)work;
    bf16* XB = A3 + 3LL * cout * vp64;
    if (cudaMemsetAsync(work, 0, (size_t)pfnn_conv3d_wgrad_work_bytes(cout, cin, n, d, h, wd), st) != cudaSuccess)
        return PF_E_CUDA;
    const long long nvox = (long long)n * d * h * wd;
    long long pb = (nvox + 255) / 256;
    if (pb > 152LL * 32) pb = 152LL * 32;
    k_wgrad_pack<<<(unsigned)pb, 256, 0, st>>>((const bf16*)dy, lddy, dyoff, cout, (const bf16*)x, ldx, xoff, cin, d, h,
                                                wd, wp, nvox, vp64, A3, XB);
    pfgb::count_launch();

    alignas(64) CUtensorMap mA, mB;
    {
        const cuuint64_t dims[2] = {(cuuint64_t)vp64, (cuuint64_t)(3 * cout)};
        const cuuint64_t strides[1] = {(cuuint64_t)vp64 * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)cout};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A3, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return PF_E_INVALID;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)vp64, (cuuint64_t)cin};
        const cuuint64_t strides[1] = {(cuuint64_t)vp64 * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)cin};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, XB, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return PF_E_INVALID;
    }
    WgArgs a{};
    a.cout = cout;
    a.cin = cin;
    a.taps_per_tile = UM / cout;
    const int ntiles = (27 + a.taps_per_tile - 1) / a.taps_per_tile;
    a.nkb = vp64 / 64;
    // about four waves of CTAs over the 152 SMs
    long long chunks = (4LL * 152 + ntiles - 1) / ntiles;
    if (chunks > a.nkb) chunks = a.nkb;
    a.kb_per_cta = (int)((a.nkb + chunks - 1) / chunks);
    chunks = (a.nkb + a.kb_per_cta - 1) / a.kb_per_cta;
    a.plane_p = (h + 2) * wp;
    a.row_p = wp;
    a.a_bytes = (unsigned)(UM * 128);
    a.stage_bytes = a.a_bytes + round1024((unsigned)(cin * 128));
    int stages = (int)(98304u / a.stage_bytes);
    a.stages = stages < 2 ? 2 : (stages > 8 ? 8 : stages);
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(cin >> 3) << 17) | ((unsigned)(UM >> 4) << 24);
    a.desc_hi = (1ULL << 16) | ((1024ULL >> 4) << 32) | (1ULL << 46) | (umma_layout(64) << 61);
    a.tmem_cols = cin <= 32 ? 32 : (cin <= 64 ? 64 : (cin <= 128 ? 128 : 256));
    a.tries = WAIT_TRIES;
    a.dw = dw;
    const size_t smem = (size_t)a.stages * a.stage_bytes + 1024 + 16 * a.stages + 16;
    static std::once_flag wg_once;
    static cudaError_t wg_err = cudaSuccess;
    std::call_once(wg_once, [] {
        wg_err = cudaFuncSetAttribute(k_wgrad_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024 + 2048);
    });
    if (wg_err != cudaSuccess) return PF_E_CUDA;
    k_wgrad_umma<<<dim3((unsigned)ntiles, (unsigned)chunks), UTHR, smem, st>>>(mA, mB, a);
    pfgb::count_launch();
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_E_CUDA;
}

pf_status pfnn_status(int* failed) {
    if (!failed) return PF_E_INVALID;
    int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_umma_status, sizeof(int)) != cudaSuccess) return PF_E_CUDA;
    if (v && cudaMemcpyToSymbol(g_umma_status, &zero, sizeof(int)) != cudaSuccess) return PF_E_CUDA;
    *failed = v;
    return v ? PF_E_TIMEOUT : PF_OK;
}

pf_status pfnn_test_withhold_stage(int stage, long long tries) {
    if (stage < 0 || tries < 1 || tries > WAIT_TRIES) return PF_E_INVALID;
    g_test_withhold = stage;
    g_test_tries = tries;
    return PF_OK;
}

}  // extern "C"
