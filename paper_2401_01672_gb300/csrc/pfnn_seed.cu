// Warm-start constraint from the micro-scale model: it has no nucleation term, so ice can only exist
// where it grew from the seed through the pore space (Sec. 2.4: constant supercooling, the phase field
// of every ice region is connected to the initial ice).  The network's prediction is kept only in the
// predicted-ice region that is connected to the seed (and within `halo` cells of it, which keeps the
// diffuse interface profile), and never below the seed's own phase field; everywhere else, and in the
// cells whose water indicator is zero (they never change, eq. water-indicator), the initial phase field
// is kept.
//
// The predicted-ice mask is first eroded by `erode` cells (so that throats narrower than about twice
// that are cut: behind them the prediction may hold ice the seed does not reach through the throat, a
// different equilibrium of the same equations), the connected region is found by flood fill through the
// eroded mask: reached = seed, then repeatedly reached |= mask & (a face neighbour is reached), in place
// (the flags only go from 0 to 1, so the order in which threads see each other's updates changes only how
// many sweeps it takes), until a sweep changes nothing; it is then grown back by `erode` cells inside the
// original mask and by `halo` cells without it.
#include "../../include/pfnn.h"
#include "pf_internal.cuh"

#include <cuda_runtime.h>

namespace {

constexpr int SF_THREADS = 256;
constexpr int SWEEPS_PER_CHECK = 16;

int sf_blocks(long long n) {
    long long b = (n + SF_THREADS - 1) / SF_THREADS;
    if (b > 152LL * 16) b = 152LL * 16;
    return (int)(b < 1 ? 1 : b);
}

// flags: bit 0 = may carry ice (eroded), bit 1 = reached, bit 2 = marked in the current growth sweep,
// bit 3 = predicted ice (predicted phi > 1/2 and a water indicator above zero), bit 4 = marked for erosion
__global__ void k_sf_init(const float* __restrict__ prob, const double* __restrict__ seed, const double* __restrict__ G,
                          double zeta, long long n, unsigned char* __restrict__ fl) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const bool water = 1.0 - zeta * G[q] > 0.0;
        const bool ice = prob[q] > 0.5f && water;
        fl[q] = (unsigned char)((ice ? 9 : 0) | (seed[q] > 0.5 ? 2 : 0));
    }
}

// one erosion sweep: a cell of the mask with a face neighbour outside it (inside the grid) leaves it
__global__ void k_sf_erode(unsigned char* fl, int n1, int n2, int n3) {
    const long long plane = (long long)n1 * n2, n = plane * n3;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        if (!(fl[q] & 1)) continue;
        const int i = (int)(q % n1), j = (int)((q / n1) % n2), k = (int)(q / plane);
        const bool edge = (i > 0 && !(fl[q - 1] & 1)) || (i < n1 - 1 && !(fl[q + 1] & 1)) ||
                          (j > 0 && !(fl[q - n1] & 1)) || (j < n2 - 1 && !(fl[q + n1] & 1)) ||
                          (k > 0 && !(fl[q - plane] & 1)) || (k < n3 - 1 && !(fl[q + plane] & 1));
        if (edge) fl[q] |= 16;
    }
}

__global__ void k_sf_erode_commit(unsigned char* fl, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        if (fl[q] & 16) fl[q] = (unsigned char)(fl[q] & ~17);
}

__device__ __forceinline__ bool any_reached(const unsigned char* fl, long long q, int i, int j, int k, int n1, int n2,
                                            int n3, long long plane) {
    return (i > 0 && (fl[q - 1] & 2)) || (i < n1 - 1 && (fl[q + 1] & 2)) || (j > 0 && (fl[q - n1] & 2)) ||
           (j < n2 - 1 && (fl[q + n1] & 2)) || (k > 0 && (fl[q - plane] & 2)) || (k < n3 - 1 && (fl[q + plane] & 2));
}

// one flood-fill sweep (grow = 0: only through cells that may carry ice), one dilation sweep inside the
// predicted ice (grow = 2) or one dilation sweep everywhere (grow = 1)
__global__ void k_sf_sweep(unsigned char* fl, int n1, int n2, int n3, int grow, int* changed) {
    const long long plane = (long long)n1 * n2, n = plane * n3;
    int local = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const unsigned char f = ((volatile unsigned char*)fl)[q];
        if ((f & 2) || (grow == 0 && !(f & 1)) || (grow == 2 && !(f & 8))) continue;
        const int i = (int)(q % n1), j = (int)((q / n1) % n2), k = (int)(q / plane);
        if (any_reached(fl, q, i, j, k, n1, n2, n3, plane)) {
            ((volatile unsigned char*)fl)[q] = (unsigned char)(f | (grow ? 4 : 2));
            local = 1;
        }
    }
    if (local) atomicOr(changed, 1);
}

// dilation marks (bit 2) become reached (bit 1) between dilation sweeps, so each sweep grows one cell
__global__ void k_sf_commit(unsigned char* fl, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        if (fl[q] & 4) fl[q] = (unsigned char)((fl[q] & ~4) | 2);
}

__global__ void k_sf_apply(const float* __restrict__ prob, const double* __restrict__ seed, const double* __restrict__ G,
                           double zeta, long long n, const unsigned char* __restrict__ fl, double* __restrict__ out) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const bool water = 1.0 - zeta * G[q] > 0.0;
        const double p = fminf(fmaxf(prob[q], 0.f), 1.f);
        // the seed itself stays ice where the prediction has less
        out[q] = (water && (fl[q] & 2)) ? fmax(p, seed[q]) : seed[q];
    }
}

}  // namespace

extern "C" pf_status pfnn_seed_connect(const float* prob, const double* phi_seed, const double* G, int n1, int n2,
                                       int n3, double zeta, int erode, int halo, unsigned char* work, double* phi_out,
                                       void* stream, long long* sweeps) {
    if (!prob || !phi_seed || !G || !work || !phi_out || n1 < 1 || n2 < 1 || n3 < 1 || halo < 0 || halo > 64 ||
        erode < 0 || erode > 64 || !(zeta >= 0.0))
        return PF_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = (long long)n1 * n2 * n3;
    unsigned char* fl = work;
    int* changed = reinterpret_cast<int*>(work + ((n + 15) / 16) * 16);
    const int nb = sf_blocks(n);
    k_sf_init<<<nb, SF_THREADS, 0, s>>>(prob, phi_seed, G, zeta, n, fl);
    pfgb::count_launch();
    for (int r = 0; r < erode; ++r) {
        k_sf_erode<<<nb, SF_THREADS, 0, s>>>(fl, n1, n2, n3);
        k_sf_erode_commit<<<nb, SF_THREADS, 0, s>>>(fl, n);
        pfgb::count_launch(2);
    }
    long long done_sweeps = 0;
    // every sweep that changes something reaches at least one more cell: at most n sweeps
    for (;;) {
        if (cudaMemsetAsync(changed, 0, sizeof(int), s) != cudaSuccess) return PF_E_CUDA;
        for (int r = 0; r < SWEEPS_PER_CHECK; ++r) {
            k_sf_sweep<<<nb, SF_THREADS, 0, s>>>(fl, n1, n2, n3, 0, changed);
            pfgb::count_launch();
        }
        done_sweeps += SWEEPS_PER_CHECK;
        int h = 0;
        if (cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return PF_E_CUDA;
        if (!h || done_sweeps > n) break;
    }
    for (int r = 0; r < erode + halo; ++r) {
        k_sf_sweep<<<nb, SF_THREADS, 0, s>>>(fl, n1, n2, n3, r < erode ? 2 : 1, changed);
        k_sf_commit<<<nb, SF_THREADS, 0, s>>>(fl, n);
        pfgb::count_launch(2);
    }
    k_sf_apply<<<nb, SF_THREADS, 0, s>>>(prob, phi_seed, G, zeta, n, fl, phi_out);
    pfgb::count_launch();
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return PF_E_CUDA;
    if (sweeps) *sweeps = done_sweeps;
    return PF_OK;
}
