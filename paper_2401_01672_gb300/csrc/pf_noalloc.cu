// Unfrozen-water counts without any device allocation.
//
// Some callers cannot call cudaMalloc: a plug-in running inside a host
// application that owns all device memory through its own pool, a control
// loop that cannot afford the implicit synchronisation of an allocation, or
// a process whose GPU memory budget is fixed in advance.  They hand in the
// glass field and the phase field they already own and receive the counts
// back; the reduction's block partials live in the file-scope array below.
//
// The array is a module global: every GPU that loads this library holds it
// (PF_NOALLOC_MAX_PARTIALS + 1 slots of 32 bytes, about 512 KiB) until the
// process exits.  All calls share it, so calls that overlap on the GPU (on
// different streams, or from different host threads) race on it.
#include "../../include/pf.h"
#include "pf_internal.cuh"

#include <cfloat>
#include <cmath>
#include <mutex>

namespace {

struct NaPart {
    unsigned long long nw, ni;  // #{G < 1/2}, #{phi > 1/2 and G < 1/2}
    double sn, sd;              // sum (1 - G) phi, sum (1 - G)
};

constexpr int NA_THREADS = 256;
constexpr long long NA_CELLS_PER_PART = 64LL * NA_THREADS;

// Block partials [0, PF_NOALLOC_MAX_PARTIALS) and the final result [PF_NOALLOC_MAX_PARTIALS].
// Every slot a call reads is written earlier in the same call, so nothing has to be cleared.
static __device__ __align__(256) NaPart g_na_scratch[PF_NOALLOC_MAX_PARTIALS + 1];

// Device address of g_na_scratch per device (host code may not use the symbol itself:
// its host-side name is a stand-in, not a device address).
constexpr int NA_MAX_DEVICES = 64;
static NaPart* g_na_addr[NA_MAX_DEVICES] = {nullptr};
static std::mutex g_na_mutex;

// Counts over the half-open box [i0,i1) x [j0,j1) x [k0,k1); one partial per block (grid-stride).
__global__ void __launch_bounds__(NA_THREADS)
k_na_uwc_partial(const double* __restrict__ G, const double* __restrict__ ph, int n1, int n2, int i0, int i1,
                 int j0, int j1, int k0, int k1, NaPart* parts) {
    const long long bx = i1 - i0, byy = j1 - j0, bz = k1 - k0;
    const long long n = bx * byy * bz;
    unsigned long long nw = 0, ni = 0;
    double sn = 0.0, sd = 0.0;
    for (long long q = blockIdx.x * (long long)NA_THREADS + threadIdx.x; q < n; q += (long long)gridDim.x * NA_THREADS) {
        const int i = i0 + (int)(q % bx), j = j0 + (int)((q / bx) % byy), k = k0 + (int)(q / (bx * byy));
        const long long id = i + (long long)n1 * (j + (long long)n2 * k);
        const double g = G[id];
        const double p = ph[id];
        if (g < 0.5) {
            ++nw;
            if (p > 0.5) ++ni;
        }
        sn += (1.0 - g) * p;
        sd += (1.0 - g);
    }
    __shared__ NaPart s[NA_THREADS];
    s[threadIdx.x] = {nw, ni, sn, sd};
    __syncthreads();
    for (int h = NA_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[threadIdx.x].nw += s[threadIdx.x + h].nw;
            s[threadIdx.x].ni += s[threadIdx.x + h].ni;
            s[threadIdx.x].sn += s[threadIdx.x + h].sn;
            s[threadIdx.x].sd += s[threadIdx.x + h].sd;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = s[0];
}

// Fixed-order sum of the partials into the result slot.
__global__ void k_na_uwc_final(NaPart* parts, int nparts) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    NaPart acc = {0, 0, 0.0, 0.0};
    for (int b = 0; b < nparts; ++b) {
        acc.nw += parts[b].nw;
        acc.ni += parts[b].ni;
        acc.sn += parts[b].sn;
        acc.sd += parts[b].sd;
    }
    parts[PF_NOALLOC_MAX_PARTIALS] = acc;
}

// Set-up, once per device, with that device current: look up the array's device address.
static cudaError_t na_scratch_address(NaPart** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        NaPart* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" pf_status pf_unfrozen_fraction_noalloc(const double* G, const double* phi, int n1, int n2, int n3,
                                                  const int* region, void* stream, double* uwc, long long* n_ice,
                                                  long long* n_water, double* smooth) {
    if (!G || !phi) return PF_E_INVALID;
    if (n1 < 1 || n2 < 1 || n3 < 1) return PF_E_INVALID;
    int r[6] = {0, n1, 0, n2, 0, n3};
    if (region) {
        for (int q = 0; q < 6; ++q) r[q] = region[q];
        if (r[0] < 0 || r[1] > n1 || r[2] < 0 || r[3] > n2 || r[4] < 0 || r[5] > n3 || r[0] > r[1] || r[2] > r[3] ||
            r[4] > r[5])
            return PF_E_INVALID;
    }
    const long long n = (long long)(r[1] - r[0]) * (r[3] - r[2]) * (r[5] - r[4]);
    const long long nb = n > 0 ? (n + NA_CELLS_PER_PART - 1) / NA_CELLS_PER_PART : 1;
    // the fixed scratch holds PF_NOALLOC_MAX_PARTIALS partials of NA_CELLS_PER_PART cells each
    if (nb > PF_NOALLOC_MAX_PARTIALS) return PF_E_RANGE;
    // both arrays must be device memory of the current device (cudaPointerGetAttributes allocates nothing)
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PF_E_CUDA;
    for (const double* ptr : {G, phi}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return PF_E_INVALID;
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return PF_E_INVALID;
    }
    NaPart* parts = nullptr;
    cudaError_t e = na_scratch_address(&parts);
    if (e != cudaSuccess) return PF_E_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    k_na_uwc_partial<<<(unsigned)nb, NA_THREADS, 0, s>>>(G, phi, n1, n2, r[0], r[1], r[2], r[3], r[4], r[5], parts);
    k_na_uwc_final<<<1, 32, 0, s>>>(parts, (int)nb);
    pfgb::count_launch(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return PF_E_CUDA;
    NaPart res;
    e = cudaMemcpyAsync(&res, parts + PF_NOALLOC_MAX_PARTIALS, sizeof(NaPart), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return PF_E_CUDA;
    if (n_ice) *n_ice = (long long)res.ni;
    if (n_water) *n_water = (long long)res.nw;
    if (uwc) *uwc = res.nw ? 1.0 - (double)res.ni / (double)res.nw : NAN;
    if (smooth) *smooth = res.sd != 0.0 ? 1.0 - res.sn / res.sd : NAN;
    return PF_OK;
}
