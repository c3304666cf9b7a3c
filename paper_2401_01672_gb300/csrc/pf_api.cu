// C ABI of the GB300 phase-field library: grid lifecycle, geometry, state,
// Runge-Kutta-Merson driving, unfrozen-water reductions (arXiv 2401.01672).
#include "../../include/pf.h"
#include "pf_internal.cuh"

#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <array>
#include <vector>

using namespace pfgb;

namespace pfgb {
static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace pfgb

static thread_local std::string t_create_err;

struct pf_grid {
    int n1 = 0, n2 = 0, n3 = 0;
    long long N = 0;
    // z-slab of a multi-domain group: ghost planes below / above (filled by the neighbour slab),
    // global index of local plane 0, cells allocated per ghosted array (N plus the ghost planes)
    int zg_lo = 0, zg_hi = 0, k_off = 0;
    long long NA = 0;
    bool own_ctrl = true;
    double h = 0;
    int model = 0, rx = 0, prec = 0;
    pf_params p{};
    Coefs cf{};
    CoefT<double> k64{};
    CoefT<float> k32{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int by = 8, zc = 32;
    double* y_th[2] = {nullptr, nullptr};
    double* y_ph[2] = {nullptr, nullptr};
    void* ua_th = nullptr; void* ua_ph = nullptr;
    void* ub_th = nullptr; void* ub_ph = nullptr;
    void* k1_th = nullptr; void* k1_ph = nullptr;
    void* k3_th = nullptr; void* k3_ph = nullptr;
    void* k4_th = nullptr; void* k4_ph = nullptr;
    // binary32 form of the full model: binary32 copies of the two state buffers (the stage inputs are
    // increments over the current one); set with the state, written by stage 5 beside the candidate state
    void* y32_th[2] = {nullptr, nullptr};
    void* y32_ph[2] = {nullptr, nullptr};
    double* G64 = nullptr;
    float* G32 = nullptr;
    double* statics = nullptr;  // full model, binary64: NSTATIC per-cell coefficient arrays (see StageArgs)
    double* scratch64 = nullptr;
    void* red = nullptr;
    size_t red_bytes = 0;
    Ctrl* dctrl = nullptr;
    Ctrl* hctrl = nullptr;  // pinned mirror
    double** ptab = nullptr;  // device table {y_ph[0], y_ph[1], y_th[0], y_th[1]}
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    long long launches = 0;
    std::vector<void*> allocs;
    std::string err;
};

// ------------------------------------------------------------------ helpers
#define PF_CUDA(g, call)                                                              \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return fail((g), PF_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static pf_status fail(pf_grid* g, pf_status s, const std::string& msg) {
    if (g) g->err = msg;
    else t_create_err = msg;
    return s;
}

static bool is_f32(const pf_grid* g) { return g->prec == PF_PREC_FP32_FIELDS; }
extern "C" {
static pf_status refresh_g32(pf_grid* g);
static pf_status refresh_y32(pf_grid* g, int b);
}
static size_t fbytes(const pf_grid* g) { return is_f32(g) ? sizeof(float) : sizeof(double); }
static bool has_th(const pf_grid* g) { return g->model != PF_MODEL_MICRO; }
static bool has_ph(const pf_grid* g) { return g->model != PF_MODEL_TEMP; }
// binary32 form of the full model: stage inputs are increments over a binary32 copy of the state
static bool has_y32(const pf_grid* g) { return is_f32(g) && g->model == PF_MODEL_FULL; }

static int blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 16) b = 152LL * 16;
    return (int)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------ kernels
__global__ void k_fill(double* p, long long n, double v) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        p[q] = v;
}

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = (float)in[q];
}

// Sec. 2.1, G_balls: one block per sphere scatters 1/2 (1 - tanh((|x - x_s| - r_s)/(2 xi_G))) into the
// cells within r_s + 40 xi_G of its centre by atomicMax on the bit pattern (G >= 0).  Beyond that radius
// the term is below e^-40 and is skipped.  The array holds global planes kofs .. kofs + n3 - 1 (a z-slab
// with its ghost planes; kofs = 0 for a whole grid); cell centres use the global indices.
__global__ void k_glass_spheres(const double* __restrict__ sp, long long ns, double* G, int n1, int n2, int n3,
                                int kofs, double h, double xi_G) {
    const long long s = blockIdx.x;
    if (s >= ns) return;
    const double cx = sp[4 * s], cy = sp[4 * s + 1], cz = sp[4 * s + 2], r = sp[4 * s + 3];
    const double rc = r + 40.0 * xi_G;
    int lo[3], hi[3];
    const double cc[3] = {cx, cy, cz};
    const int nlo[3] = {0, 0, kofs};
    const int nhi[3] = {n1 - 1, n2 - 1, kofs + n3 - 1};
    for (int d = 0; d < 3; ++d) {
        double a = floor((cc[d] - rc) / h - 0.5), b = ceil((cc[d] + rc) / h - 0.5);
        lo[d] = (int)fmax((double)nlo[d], a);
        hi[d] = (int)fmin((double)nhi[d], b);
    }
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]) return;
    const long long bx = hi[0] - lo[0] + 1, byy = hi[1] - lo[1] + 1, bz = hi[2] - lo[2] + 1;
    const long long nb = bx * byy * bz;
    const double inv2x = 1.0 / (2.0 * xi_G);
    unsigned long long* Gb = reinterpret_cast<unsigned long long*>(G);
    for (long long q = threadIdx.x; q < nb; q += blockDim.x) {
        const int i = lo[0] + (int)(q % bx);
        const int j = lo[1] + (int)((q / bx) % byy);
        const int k = lo[2] + (int)(q / (bx * byy));
        const double dx = (i + 0.5) * h - cx, dy = (j + 0.5) * h - cy, dz = (k + 0.5) * h - cz;
        const double dist = sqrt(dx * dx + dy * dy + dz * dz);
        if (dist - r > 40.0 * xi_G) continue;
        const double g = 0.5 * (1.0 - tanh((dist - r) * inv2x));
        if (g > 0.0)
            atomicMax(&Gb[i + (long long)n1 * (j + (long long)n2 * (k - kofs))], (unsigned long long)__double_as_longlong(g));
    }
}

// Sec. 2.1: G = max(G_balls, 1/2 (1 + tanh((x3 - x3cap)/(2 xi_G))))  (array plane 0 = global plane kofs)
__global__ void k_glass_cap(double* G, int n1, int n2, int n3, int kofs, double h, double xi_G, double x3cap) {
    const long long n = (long long)n1 * n2 * n3;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q / ((long long)n1 * n2)) + kofs;
        const double z = (k + 0.5) * h;
        const double g = 0.5 * (1.0 + tanh((z - x3cap) / (2.0 * xi_G)));
        if (g > G[q]) G[q] = g;
    }
}

// Per-cell coefficients of the full model from G (eq. material-properties-blending-formula): with
// w(phi) = A_w + B_w phi, A_w = w_L + G (w_G - w_L), B_w = (1 - G)(w_I - w_L):
//   lambda' = A_lam + B_lam phi (scaled by 1/(2h^2)), W = 2 (1 - zeta G)/(alpha xi^2),
//   rho c = A_rho A_c + (A_rho B_c + B_rho A_c) phi + B_rho B_c phi^2,  rho L = L A_rho + L B_rho phi,
//   and 1/(rho c) at phi = 0 and at phi = 1 (IEEE division), used where phi and its six neighbours
//   are all exactly 0 or all exactly 1 (there dphi/dt = 0 and dtheta/dt = div / (rho c)).
__global__ void k_full_statics(const double* __restrict__ G, double* __restrict__ S, long long n, CoefT<double> k) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double g = G[q];
        const double ar = fma(g, k.dRG, k.rhoL), br = fma(-g, k.dRI, k.dRI);
        const double ac = fma(g, k.dCG, k.capL), bc = fma(-g, k.dCI, k.dCI);
        S[q] = fma(g, k.dLG, k.lamL);
        S[n + q] = fma(-g, k.dLI, k.dLI);
        S[2 * n + q] = fma(k.wb, g, k.wa);
        S[3 * n + q] = ar * ac;
        S[4 * n + q] = fma(ar, bc, br * ac);
        S[5 * n + q] = br * bc;
        S[6 * n + q] = k.latent * ar;
        S[7 * n + q] = k.latent * br;
        const double c0 = ar * ac;
        const double c1 = c0 + fma(ar, bc, br * ac) + br * bc;
        S[8 * n + q] = 1.0 / c0;
        S[9 * n + q] = 1.0 / c1;
    }
}

// Temp model phase field, eq. (explicit-p-dependence-on-T)
__global__ void k_temp_phi(const double* __restrict__ th, const double* __restrict__ G, double* __restrict__ ph,
                           long long n, double gamma, double zeta) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        double iw = 1.0 - zeta * G[q];
        iw = iw > 0.0 ? iw : 0.0;
        ph[q] = 0.5 * iw * (1.0 - tanh(gamma * th[q]));
    }
}

// Step control after stage 5 (one thread per grid).  Accept iff E <= tol (or fixed mode); proposal
// dt * min(5, 0.8 (tol/E)^(1/5)) capped at dt_max; the next step is shortened to land on t_freeze or
// t_end.  With eq_window > 0 the run stops, before accepting, once the pore-bulk ice count of the
// current state (measured in stage 1) has stayed within eq_rel_tol x (pore-bulk cells) of a reference
// value for eq_window seconds and, when eq_rate > 0, the largest |dphi/dt| over the pore-bulk cells of
// that state is at most eq_rate (the state is then the one at t_eq = t).
__device__ void controller_step(Ctrl* c) {
    if (c->done) return;
    const double E = __longlong_as_double((long long)c->err_bits);
    const long long cnt = (long long)c->ice_count;
    const double tolc = c->eq_rel_tol * (double)c->pore_count;
    const double rate = __longlong_as_double((long long)c->rate_bits);
    c->err_bits = 0ULL;
    c->ice_count = 0ULL;
    c->pore_count = 0ULL;
    c->rate_bits = 0ULL;
    c->last_err = E;
    c->last_rate = rate;
    if (c->eq_window > 0.0) {
        if (c->prev_count < 0 || fabs((double)(cnt - c->prev_count)) > tolc) {
            c->prev_count = cnt;
            c->last_change_t = c->t;
        } else if (c->t - c->last_change_t >= c->eq_window && (c->eq_rate <= 0.0 || rate <= c->eq_rate)) {
            c->equilibrium = 1;
            c->t_eq = c->t;
            c->accepted = 0;
            c->done = 1;
            return;
        }
    }
    const bool finite = E <= DBL_MAX;
    const bool accept = c->fixed || (finite && E <= c->tol);
    c->accepted = accept;
    if (!finite && !c->fixed) {
        c->status = PF_E_NONFINITE;
        c->done = 1;
        return;
    }
    if (accept) {
        c->t = c->land ? c->target : c->t + c->dt_step;
        c->cur ^= 1;
        c->n_acc++;
    } else {
        c->n_rej++;
    }
    if (!c->fixed || c->single) {
        double fac;
        if (E == 0.0) {
            fac = 5.0;
        } else {
            fac = 0.8 * pow(c->tol / E, 0.2);
            if (fac > 5.0) fac = 5.0;
        }
        double dn = c->dt_step * fac;
        if (dn > c->dt_max) dn = c->dt_max;
        c->dt = dn;
        if (!c->fixed && dn < c->dt_min) {
            c->status = PF_E_DT_UNDERFLOW;
            c->done = 1;
            return;
        }
    }
    if (c->single) return;
    if (c->t >= c->t_end || c->n_acc + c->n_rej >= c->max_attempts) {
        c->done = 1;
        return;
    }
    double target = c->t_end;
    if (c->t < c->t_freeze && c->t_freeze < target) target = c->t_freeze;
    if (c->t + c->dt >= target) {
        c->dt_step = target - c->t;
        c->land = 1;
        c->target = target;
    } else {
        c->dt_step = c->dt;
        c->land = 0;
    }
    prepare_step(c);
}

__global__ void k_controller(Ctrl* c) {
    if (threadIdx.x == 0 && blockIdx.x == 0) controller_step(c);
}

// Batched step control: one thread per active instance.
__global__ void k_batch_controller(Ctrl* const* ctrls, const BatchPlan* plan) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < plan->nactive) controller_step(ctrls[plan->inst[s]]);
}

// Rebuild the batched work list from the instances' done flags and decide whether the device-side
// loop runs another step (at most max_iter steps, so the loop always ends).
__global__ void k_batch_plan(Ctrl* const* ctrls, const int4* tilegrid, int n, BatchPlan* plan,
                             cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int nt = 0, na = 0;
    for (int q = 0; q < n; ++q) {
        if (!ctrls[q]->done) {
            plan->inst[na] = q;
            plan->tile_start[na] = nt;
            nt += tilegrid[q].w;
            ++na;
        }
    }
    plan->tile_start[na] = nt;
    plan->ntiles = nt;
    plan->nactive = na;
    plan->iter += 1;
    cudaGraphSetConditional(cond, (na > 0 && plan->iter <= plan->max_iter) ? 1u : 0u);
}

// UWC partial sums over a half-open box; one slot of 4 words per block:
// [n_water, n_ice] as unsigned 64-bit, [sum (1-G) phi, sum (1-G)] as binary64.
struct UwcPart { unsigned long long nw, ni; double sn, sd; };

template <int BS>
__global__ void __launch_bounds__(BS) k_uwc_partial(const double* __restrict__ G, const double* const* yph,
                                                    const double* const* yth, const Ctrl* ctrl, int temp,
                                                    double gamma, double zeta, int n1, int n2, int i0, int i1,
                                                    int j0, int j1, int k0, int k1, UwcPart* parts) {
    const int cur = ctrl->cur;
    const double* ph = temp ? nullptr : yph[cur];
    const double* th = temp ? yth[cur] : nullptr;
    const long long bx = i1 - i0, byy = j1 - j0, bz = k1 - k0;
    const long long n = bx * byy * bz;
    unsigned long long nw = 0, ni = 0;
    double sn = 0.0, sd = 0.0;
    for (long long q = blockIdx.x * (long long)BS + threadIdx.x; q < n; q += (long long)gridDim.x * BS) {
        const int i = i0 + (int)(q % bx), j = j0 + (int)((q / bx) % byy), k = k0 + (int)(q / (bx * byy));
        const long long id = i + (long long)n1 * (j + (long long)n2 * k);
        const double g = G[id];
        double p;
        if (temp) {
            double iw = 1.0 - zeta * g;
            iw = iw > 0.0 ? iw : 0.0;
            p = 0.5 * iw * (1.0 - tanh(gamma * th[id]));
        } else {
            p = ph[id];
        }
        if (g < 0.5) {
            ++nw;
            if (p > 0.5) ++ni;
        }
        sn += (1.0 - g) * p;
        sd += (1.0 - g);
    }
    __shared__ UwcPart sp[BS];
    sp[threadIdx.x] = {nw, ni, sn, sd};
    __syncthreads();
    for (int s = BS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sp[threadIdx.x].nw += sp[threadIdx.x + s].nw;
            sp[threadIdx.x].ni += sp[threadIdx.x + s].ni;
            sp[threadIdx.x].sn += sp[threadIdx.x + s].sn;
            sp[threadIdx.x].sd += sp[threadIdx.x + s].sd;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = sp[0];
}

// Fixed-order final sum of the per-block partials (deterministic binary64 result): thread t sums
// partials t, t+256, ... in order, then a fixed tree combines the 256 thread sums.
__global__ void __launch_bounds__(256) k_uwc_final(UwcPart* parts, int nparts, UwcPart* out) {
    __shared__ UwcPart s[256];
    UwcPart acc = {0, 0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nparts; b += 256) {
        acc.nw += parts[b].nw;
        acc.ni += parts[b].ni;
        acc.sn += parts[b].sn;
        acc.sd += parts[b].sd;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[threadIdx.x].nw += s[threadIdx.x + h].nw;
            s[threadIdx.x].ni += s[threadIdx.x + h].ni;
            s[threadIdx.x].sn += s[threadIdx.x + h].sn;
            s[threadIdx.x].sd += s[threadIdx.x + h].sd;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// max |v| over n values of type T -> per-block partial maxima (binary64), then a final pass.
template <typename T, int BS>
__global__ void __launch_bounds__(BS) k_maxabs_partial(const T* __restrict__ v, long long n, double* parts) {
    double m = 0.0;
    for (long long q = blockIdx.x * (long long)BS + threadIdx.x; q < n; q += (long long)gridDim.x * BS) {
        double a = fabs((double)v[q]);
        if (!(a <= DBL_MAX)) a = INFINITY;
        m = a > m ? a : m;
    }
    __shared__ double s[BS];
    s[threadIdx.x] = m;
    __syncthreads();
    for (int k = BS / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = s[0];
}

__global__ void k_max_final(const double* parts, int n, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = 0.0;
    for (int b = 0; b < n; ++b) m = parts[b] > m ? parts[b] : m;
    *out = m;
}

// Model constants in the stage kernels' form, computed in binary64 (see CoefT).
template <typename T>
static void fill_coefs(CoefT<T>& k, const pf_params& p, double h) {
    const double s = 0.5 / (h * h);
    k.lamL = T(p.lambda[0] * s);
    k.dLG = T((p.lambda[2] - p.lambda[0]) * s);
    k.dLI = T((p.lambda[1] - p.lambda[0]) * s);
    k.rhoL = T(p.rho[0]); k.dRG = T(p.rho[2] - p.rho[0]); k.dRI = T(p.rho[1] - p.rho[0]);
    k.capL = T(p.c[0]); k.dCG = T(p.c[2] - p.c[0]); k.dCI = T(p.c[1] - p.c[0]);
    k.latent = T(p.latent);
    const double w = (p.alpha > 0 && p.xi > 0) ? 2.0 / (p.alpha * p.xi * p.xi) : 0.0;
    k.wa = T(w);
    k.wb = T(-p.zeta * w);
    k.g_pore = T(p.zeta > 0 ? 0.5 / p.zeta : 1.0);
    k.wa_half = T(0.5 * w);
    k.klap = T(p.xi * p.xi * s);
    k.ksig = T(0.5 * p.xi * p.b * p.mu * p.alpha);
    k.kgrad = T(p.xi * p.xi * p.mu * p.alpha / (4.0 * h));
    k.eps0 = T(p.eps0); k.eps1 = T(p.eps1);
    k.inv_de = T(p.eps1 > p.eps0 ? 1.0 / (p.eps1 - p.eps0) : 0.0);
    k.gamma = T(p.gamma); k.zeta = T(p.zeta);
    k.theta_micro = T(p.theta_micro);
}

// ------------------------------------------------------------------ stage dispatch
template <typename T>
static StageArgs<T> make_args(pf_grid* g) {
    StageArgs<T> a{};
    a.cf = g->cf;
    if constexpr (std::is_same<T, float>::value) a.k = g->k32;
    else a.k = g->k64;
    a.ctrl = g->dctrl;
    for (int b = 0; b < 2; ++b) {
        a.y_th[b] = g->y_th[b];
        a.y_ph[b] = g->y_ph[b];
        a.yo_th[b] = g->y_th[b];
        a.yo_ph[b] = g->y_ph[b];
    }
    a.ua_th = (T*)g->ua_th; a.ua_ph = (T*)g->ua_ph;
    a.ub_th = (T*)g->ub_th; a.ub_ph = (T*)g->ub_ph;
    a.k1_th = (T*)g->k1_th; a.k1_ph = (T*)g->k1_ph;
    a.k3_th = (T*)g->k3_th; a.k3_ph = (T*)g->k3_ph;
    a.k4_th = (T*)g->k4_th; a.k4_ph = (T*)g->k4_ph;
    for (int b = 0; b < 2; ++b) {
        a.y32_th[b] = (T*)g->y32_th[b];
        a.y32_ph[b] = (T*)g->y32_ph[b];
    }
    if constexpr (std::is_same<T, float>::value) a.G = g->G32;
    else a.G = g->G64;
    a.zc = g->zc;
    a.statics = g->statics;
    a.ncell = g->NA;
    return a;
}

static cudaError_t launch_stage(pf_grid* g, int stage, cudaStream_t s) {
    g->launches++;
    if (is_f32(g)) return launch_stage_f32(g->model, g->rx, stage, make_args<float>(g), g->by, s);
    return launch_stage_f64(g->model, g->rx, stage, make_args<double>(g), g->by, s);
}

// S1..S5 + controller on stream s
static cudaError_t enqueue_attempt(pf_grid* g, cudaStream_t s) {
    for (int st = 1; st <= 5; ++st) {
        cudaError_t e = launch_stage(g, st, s);
        if (e != cudaSuccess) return e;
    }
    k_controller<<<1, 32, 0, s>>>(g->dctrl);
    count_launch();
    g->launches++;
    return cudaGetLastError();
}

static void free_graph(pf_grid* g) {
    if (g->graph) cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
    g->graph_steps = 0;
}

// Capture `steps` attempts into one executable graph (replayed by pf_run_to / pf_run_fixed).
static pf_status build_graph(pf_grid* g, int steps) {
    free_graph(g);
    cudaGraph_t graph = nullptr;
    PF_CUDA(g, cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    long long before = g->launches;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < steps && e == cudaSuccess; ++s) e = enqueue_attempt(g, g->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
    // launches made during capture are only recorded, not executed
    g->launches = before;
    pfgb::g_launches.fetch_sub((long long)steps * 6, std::memory_order_relaxed);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(g, PF_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&g->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        g->graph = nullptr;
        return fail(g, PF_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
    }
    g->graph_steps = steps;
    return PF_OK;
}

static pf_status sync_ctrl_to_host(pf_grid* g) {
    PF_CUDA(g, cudaMemcpyAsync(g->hctrl, g->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, g->stream));
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    return PF_OK;
}

static pf_status push_ctrl(pf_grid* g) {
    PF_CUDA(g, cudaMemcpyAsync(g->dctrl, g->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, g->stream));
    return PF_OK;
}

// ------------------------------------------------------------------ ABI
extern "C" {

const char* pf_last_error(const pf_grid* g) { return g ? g->err.c_str() : t_create_err.c_str(); }

long long pf_kernel_launches(void) { return pfgb::g_launches.load(); }

static void destroy_impl(pf_grid* g) {
    free_graph(g);
    for (void* p : g->allocs) cudaFree(p);
    if (g->hctrl) cudaFreeHost(g->hctrl);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
}

pf_status pf_destroy_grid(pf_grid* g) {
    if (!g) return PF_OK;
    cudaStreamSynchronize(g->stream);
    destroy_impl(g);
    return PF_OK;
}

// Options of a grid that is one z-slab of a multi-domain group (all zero for a whole grid).
struct SlabOpts {
    int zg_lo = 0, zg_hi = 0;  // ghost plane below / above
    int k_off = 0;             // global index of local plane 0
    pf_grid* ctrl_owner = nullptr;  // shares this grid's control block (step control of the group)
};

static pf_status create_impl(int n1, int n2, int n3, double h, int model, int reaction, int precision,
                             const pf_params* p, void* stream, const SlabOpts& so, pf_grid** out) {
    if (!out) return fail(nullptr, PF_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, PF_E_INVALID, "params is NULL");
    if (n1 < 1 || n2 < 1 || n3 < 1) return fail(nullptr, PF_E_INVALID, "grid sizes must be >= 1");
    // the stage kernels index cells with 32-bit integers (ghost planes of a slab included)
    if ((long long)n1 * n2 * ((long long)n3 + 2) >= (1LL << 31)) return fail(nullptr, PF_E_INVALID, "grid too large");
    if (!(h > 0.0)) return fail(nullptr, PF_E_INVALID, "h must be > 0");
    if (model < 0 || model > 2) return fail(nullptr, PF_E_INVALID, "unknown model");
    if (reaction < 0 || reaction > 1) return fail(nullptr, PF_E_INVALID, "unknown reaction");
    if (precision < 0 || precision > 1) return fail(nullptr, PF_E_INVALID, "unknown precision");
    if (model != PF_MODEL_TEMP && (!(p->alpha > 0) || !(p->xi > 0) || !(p->eps1 > p->eps0)))
        return fail(nullptr, PF_E_INVALID, "alpha, xi must be > 0 and eps1 > eps0");
    if (!(p->zeta >= 0)) return fail(nullptr, PF_E_INVALID, "zeta must be >= 0");
    if (model != PF_MODEL_MICRO)
        for (int m = 0; m < 3; ++m)
            if (!(p->rho[m] > 0) || !(p->c[m] > 0) || !(p->lambda[m] >= 0))
                return fail(nullptr, PF_E_INVALID, "rho, c must be > 0 and lambda >= 0");

    pf_grid* g = new pf_grid();
    g->n1 = n1; g->n2 = n2; g->n3 = n3;
    g->N = (long long)n1 * n2 * n3;
    g->zg_lo = so.zg_lo; g->zg_hi = so.zg_hi; g->k_off = so.k_off;
    const long long plane = (long long)n1 * n2;
    g->NA = g->N + (long long)(so.zg_lo + so.zg_hi) * plane;
    g->h = h;
    g->model = model; g->rx = reaction; g->prec = precision;
    g->p = *p;
    g->stream = (cudaStream_t)stream;
    Coefs& c = g->cf;
    c.n1 = n1; c.n2 = n2; c.n3 = n3;
    c.zlo = so.zg_lo ? -1 : 0;
    c.zhi = so.zg_hi ? n3 : n3 - 1;
    c.dirichlet = (model == PF_MODEL_MICRO) ? 0 : (p->dirichlet_faces & 63);
    // a face shared with a neighbour slab is interior to the domain: no boundary condition there
    if (so.zg_lo) c.dirichlet &= ~PF_FACE_ZM;
    if (so.zg_hi) c.dirichlet &= ~PF_FACE_ZP;
    c.harmonic = p->harmonic_mean ? 1 : 0;
    c.theta_freeze = p->theta_freeze; c.theta_thaw = p->theta_thaw; c.t_freeze = p->t_freeze;
    fill_coefs(g->k64, *p, h);
    fill_coefs(g->k32, *p, h);
    auto alloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
        g->allocs.push_back(q);
        return q;
    };
    const size_t nd = sizeof(double) * g->N, nf = fbytes(g) * g->N;
    bool ok = true;
    auto A = [&](size_t b) { void* q = alloc(b); ok = ok && q; return q; };
    // arrays read at the z neighbours get the ghost planes; the pointer kept is that of local plane 0
    auto AG = [&](size_t esz) -> void* {
        char* q = (char*)alloc(esz * (size_t)g->NA);
        ok = ok && q;
        return q ? q + esz * (size_t)(so.zg_lo * plane) : nullptr;
    };
    if (has_th(g)) {
        g->y_th[0] = (double*)AG(8); g->y_th[1] = (double*)AG(8);
        g->ua_th = AG(fbytes(g)); g->ub_th = AG(fbytes(g)); g->k1_th = A(nf); g->k3_th = A(nf); g->k4_th = A(nf);
    }
    if (has_ph(g)) {
        g->y_ph[0] = (double*)AG(8); g->y_ph[1] = (double*)AG(8);
        g->ua_ph = AG(fbytes(g)); g->ub_ph = AG(fbytes(g)); g->k1_ph = A(nf); g->k3_ph = A(nf); g->k4_ph = A(nf);
    }
    if (is_f32(g) && model == PF_MODEL_FULL) {
        for (int b = 0; b < 2; ++b) {
            g->y32_th[b] = AG(4);
            g->y32_ph[b] = AG(4);
        }
    }
    g->G64 = (double*)AG(8);
    if (is_f32(g)) g->G32 = (float*)AG(4);
    if (!is_f32(g) && model == PF_MODEL_FULL) {
        // NSTATIC arrays of NA cells each, ghost planes included (stride NA between arrays)
        char* q = (char*)A(NSTATIC * sizeof(double) * (size_t)g->NA);
        g->statics = q ? (double*)(q + sizeof(double) * (size_t)(so.zg_lo * plane)) : nullptr;
    }
    g->scratch64 = (double*)A(nd);
    g->red_bytes = sizeof(UwcPart) * (152 * 16 + 2);
    g->red = A(g->red_bytes);
    if (so.ctrl_owner) {
        g->own_ctrl = false;
        g->dctrl = so.ctrl_owner->dctrl;
    } else {
        g->dctrl = (Ctrl*)A(sizeof(Ctrl));
    }
    g->ptab = (double**)A(4 * sizeof(double*));
    cudaGetLastError();
    if (!ok) {
        destroy_impl(g);
        return fail(nullptr, PF_E_OOM, "device allocation failed");
    }
    if (cudaMallocHost((void**)&g->hctrl, sizeof(Ctrl)) != cudaSuccess) {
        cudaGetLastError();
        destroy_impl(g);
        return fail(nullptr, PF_E_OOM, "pinned allocation failed");
    }
    if (cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        destroy_impl(g);
        return fail(nullptr, PF_E_CUDA, "stream creation failed");
    }
    // default state: all water, theta = 0, phi = 0, t = 0 (ghost planes included)
    const size_t gbytes = sizeof(double) * (size_t)(so.zg_lo * plane);
    double* h_tab[4] = {g->y_ph[0], g->y_ph[1], g->y_th[0], g->y_th[1]};
    cudaError_t e = cudaMemcpy(g->ptab, h_tab, sizeof(h_tab), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && g->own_ctrl) e = cudaMemsetAsync(g->dctrl, 0, sizeof(Ctrl), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync((char*)g->G64 - gbytes, 0, 8 * (size_t)g->NA, g->stream);
    if (e == cudaSuccess && g->G32)
        e = cudaMemsetAsync((char*)g->G32 - gbytes / 2, 0, 4 * (size_t)g->NA, g->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        if (g->y_th[b]) e = cudaMemsetAsync((char*)g->y_th[b] - gbytes, 0, 8 * (size_t)g->NA, g->stream);
        if (e == cudaSuccess && g->y_ph[b]) e = cudaMemsetAsync((char*)g->y_ph[b] - gbytes, 0, 8 * (size_t)g->NA, g->stream);
        if (e == cudaSuccess && g->y32_th[b])
            e = cudaMemsetAsync((char*)g->y32_th[b] - gbytes / 2, 0, 4 * (size_t)g->NA, g->stream);
        if (e == cudaSuccess && g->y32_ph[b])
            e = cudaMemsetAsync((char*)g->y32_ph[b] - gbytes / 2, 0, 4 * (size_t)g->NA, g->stream);
    }
    if (e != cudaSuccess) {
        destroy_impl(g);
        return fail(nullptr, PF_E_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
    }
    if (refresh_g32(g) != PF_OK) {
        cudaGetLastError();
        destroy_impl(g);
        return fail(nullptr, PF_E_CUDA, "initialisation of the glass-field coefficients failed");
    }
    std::memset(g->hctrl, 0, sizeof(Ctrl));
    g->hctrl->dt = std::isfinite(p->dt_max) ? p->dt_max : 1e-3;
    g->hctrl->t_freeze = p->t_freeze;
    g->hctrl->theta_freeze = p->theta_freeze;
    g->hctrl->theta_thaw = p->theta_thaw;
    g->hctrl->dt_min = p->dt_min;
    g->hctrl->dt_max = p->dt_max;
    if ((g->own_ctrl && push_ctrl(g) != PF_OK) || cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        destroy_impl(g);
        return fail(nullptr, PF_E_CUDA, "initialisation failed");
    }
    *out = g;
    return PF_OK;
}

pf_status pf_create_grid(int n1, int n2, int n3, double h, int model, int reaction, int precision,
                         const pf_params* p, void* stream, pf_grid** out) {
    return create_impl(n1, n2, n3, h, model, reaction, precision, p, stream, SlabOpts{}, out);
}

// Derived copies of the glass field: binary32 copy (binary32 form), per-cell coefficients (full model, binary64).
static pf_status refresh_g32(pf_grid* g) {
    // over every allocated cell, ghost planes included
    const long long go = (long long)g->zg_lo * g->n1 * g->n2;
    if (g->statics) {
        k_full_statics<<<blocks_for(g->NA, 256), 256, 0, g->stream>>>(g->G64 - go, g->statics - go, g->NA, g->k64);
        count_launch();
        PF_CUDA(g, cudaGetLastError());
    }
    if (!g->G32) return PF_OK;
    k_to_f32<<<blocks_for(g->NA, 256), 256, 0, g->stream>>>(g->G64 - go, g->G32 - go, g->NA);
    count_launch();
    PF_CUDA(g, cudaGetLastError());
    return PF_OK;
}

// Binary32 copy of state buffer b (binary32 form of the full model), every allocated cell (ghost planes
// included), rounded to nearest like the stage kernels' conversion.
static pf_status refresh_y32(pf_grid* g, int b) {
    if (!has_y32(g)) return PF_OK;
    const long long go = (long long)g->zg_lo * g->n1 * g->n2;
    k_to_f32<<<blocks_for(g->NA, 256), 256, 0, g->stream>>>(g->y_th[b] - go, (float*)g->y32_th[b] - go, g->NA);
    k_to_f32<<<blocks_for(g->NA, 256), 256, 0, g->stream>>>(g->y_ph[b] - go, (float*)g->y32_ph[b] - go, g->NA);
    count_launch(2);
    PF_CUDA(g, cudaGetLastError());
    return PF_OK;
}

pf_status pf_set_geometry(pf_grid* g, const double* spheres, long long n, double x3_cap) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (n < 0 || (n > 0 && !spheres)) return fail(g, PF_E_INVALID, "bad sphere list");
    if (!(g->p.xi_G > 0)) return fail(g, PF_E_INVALID, "xi_G must be > 0");
    for (long long s = 0; s < n; ++s) {
        for (int d = 0; d < 4; ++d)
            if (!std::isfinite(spheres[4 * s + d])) return fail(g, PF_E_INVALID, "non-finite sphere");
        if (!(spheres[4 * s + 3] > 0)) return fail(g, PF_E_INVALID, "sphere radius must be > 0");
    }
    // a z-slab computes its ghost planes too (global plane indices: k_off - zg_lo ...)
    const long long go = (long long)g->zg_lo * g->n1 * g->n2;
    const int n3a = g->n3 + g->zg_lo + g->zg_hi, kofs = g->k_off - g->zg_lo;
    PF_CUDA(g, cudaMemsetAsync(g->G64 - go, 0, sizeof(double) * g->NA, g->stream));
    if (n > 0) {
        double* dsp = nullptr;
        PF_CUDA(g, cudaMalloc(&dsp, sizeof(double) * 4 * n));
        cudaError_t e = cudaMemcpyAsync(dsp, spheres, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) {
            const long long chunk = 1LL << 30;
            for (long long s0 = 0; s0 < n && e == cudaSuccess; s0 += chunk) {
                long long cnt = n - s0 < chunk ? n - s0 : chunk;
                k_glass_spheres<<<(unsigned)cnt, 256, 0, g->stream>>>(dsp + 4 * s0, cnt, g->G64 - go, g->n1, g->n2,
                                                                     n3a, kofs, g->h, g->p.xi_G);
                count_launch();
                e = cudaGetLastError();
            }
        }
        cudaError_t e2 = cudaStreamSynchronize(g->stream);
        cudaFree(dsp);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(g, PF_E_CUDA, std::string("glass field: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    if (!std::isnan(x3_cap)) {
        k_glass_cap<<<blocks_for(g->NA, 256), 256, 0, g->stream>>>(g->G64 - go, g->n1, g->n2, n3a, kofs, g->h,
                                                                   g->p.xi_G, x3_cap);
        count_launch();
        PF_CUDA(g, cudaGetLastError());
    }
    pf_status s = refresh_g32(g);
    if (s != PF_OK) return s;
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    return PF_OK;
}

pf_status pf_set_glass(pf_grid* g, const double* G) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (!G) return fail(g, PF_E_INVALID, "G is NULL");
    PF_CUDA(g, cudaMemcpyAsync(g->G64, G, sizeof(double) * g->N, cudaMemcpyHostToDevice, g->stream));
    pf_status s = refresh_g32(g);
    if (s != PF_OK) return s;
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    return PF_OK;
}

pf_status pf_get_glass(pf_grid* g, double* G) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (!G) return fail(g, PF_E_INVALID, "G is NULL");
    PF_CUDA(g, cudaMemcpyAsync(G, g->G64, sizeof(double) * g->N, cudaMemcpyDeviceToHost, g->stream));
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    return PF_OK;
}

pf_status pf_set_state(pf_grid* g, const double* theta, const double* phi, double t, double dt) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (has_th(g) && !theta) return fail(g, PF_E_INVALID, "theta is NULL");
    if (has_ph(g) && !phi) return fail(g, PF_E_INVALID, "phi is NULL");
    if (!std::isfinite(t) || !(dt > 0)) return fail(g, PF_E_INVALID, "t must be finite and dt > 0");
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    if (has_th(g)) PF_CUDA(g, cudaMemcpyAsync(g->y_th[0], theta, sizeof(double) * g->N, cudaMemcpyHostToDevice, g->stream));
    if (has_ph(g)) PF_CUDA(g, cudaMemcpyAsync(g->y_ph[0], phi, sizeof(double) * g->N, cudaMemcpyHostToDevice, g->stream));
    Ctrl* c = g->hctrl;
    c->t = t;
    c->dt = dt;
    c->cur = 0;
    c->err_bits = 0;
    c->ice_count = 0;
    c->pore_count = 0;
    c->rate_bits = 0;
    c->prev_count = -1;
    c->done = 0;
    c->status = 0;
    c->last_err = 0;
    c->equilibrium = 0;
    c->eq_window = 0.0;
    pf_status s = push_ctrl(g);
    if (s != PF_OK) return s;
    s = refresh_y32(g, 0);
    if (s != PF_OK) return s;
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    return PF_OK;
}

pf_status pf_get_state(pf_grid* g, double* theta, double* phi, double* t, double* dt) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    pf_status s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    const int cur = g->hctrl->cur;
    if (theta) {
        if (has_th(g)) {
            PF_CUDA(g, cudaMemcpyAsync(theta, g->y_th[cur], sizeof(double) * g->N, cudaMemcpyDeviceToHost, g->stream));
        } else {
            for (long long q = 0; q < g->N; ++q) theta[q] = g->p.theta_micro;
        }
    }
    if (phi) {
        if (has_ph(g)) {
            PF_CUDA(g, cudaMemcpyAsync(phi, g->y_ph[cur], sizeof(double) * g->N, cudaMemcpyDeviceToHost, g->stream));
        } else {
            k_temp_phi<<<blocks_for(g->N, 256), 256, 0, g->stream>>>(g->y_th[cur], g->G64, g->scratch64, g->N,
                                                                      g->p.gamma, g->p.zeta);
            count_launch();
            PF_CUDA(g, cudaGetLastError());
            PF_CUDA(g, cudaMemcpyAsync(phi, g->scratch64, sizeof(double) * g->N, cudaMemcpyDeviceToHost, g->stream));
        }
    }
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    if (t) *t = g->hctrl->t;
    if (dt) *dt = g->hctrl->dt;
    return PF_OK;
}

pf_status pf_rhs(pf_grid* g, double t, const void* theta_in, const void* phi_in, void* dtheta_out, void* dphi_out) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (has_th(g) && !theta_in) return fail(g, PF_E_INVALID, "theta_in is NULL");
    if (has_ph(g) && !phi_in) return fail(g, PF_E_INVALID, "phi_in is NULL");
    if (!std::isfinite(t)) return fail(g, PF_E_INVALID, "t must be finite");
    cudaError_t e;
    if (is_f32(g)) {
        StageArgs<float> a = make_args<float>(g);
        a.in_th = (const float*)theta_in; a.in_ph = (const float*)phi_in;
        a.out_th = (float*)dtheta_out; a.out_ph = (float*)dphi_out;
        a.t_rhs = t;
        e = launch_stage_f32(g->model, g->rx, 0, a, g->by, g->stream);
    } else {
        StageArgs<double> a = make_args<double>(g);
        a.in_th = (const double*)theta_in; a.in_ph = (const double*)phi_in;
        a.out_th = (double*)dtheta_out; a.out_ph = (double*)dphi_out;
        a.t_rhs = t;
        e = launch_stage_f64(g->model, g->rx, 0, a, g->by, g->stream);
    }
    g->launches++;
    if (e != cudaSuccess) return fail(g, PF_E_CUDA, std::string("rhs launch: ") + cudaGetErrorString(e));
    // the micro model integrates no temperature: dtheta = 0; Temp has dphi from the kernel
    if (!has_th(g) && dtheta_out) PF_CUDA(g, cudaMemsetAsync(dtheta_out, 0, fbytes(g) * g->N, g->stream));
    return PF_OK;
}

pf_status pf_rkm_step(pf_grid* g, double* dt_inout, double tol, int force_accept, int* accepted, double* err) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (!dt_inout || !(*dt_inout > 0) || !std::isfinite(*dt_inout)) return fail(g, PF_E_INVALID, "dt must be > 0");
    if (!force_accept && !(tol > 0)) return fail(g, PF_E_INVALID, "tol must be > 0");
    pf_status s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    Ctrl* c = g->hctrl;
    c->dt_step = *dt_inout;
    c->dt = *dt_inout;
    c->eq_window = 0.0;
    c->equilibrium = 0;
    c->land = 0;
    prepare_step(c);
    c->done = 0;
    c->status = 0;
    c->fixed = force_accept ? 1 : 0;
    c->single = 1;
    c->tol = tol;
    c->n_acc = c->n_rej = 0;
    c->err_bits = 0;
    s = push_ctrl(g);
    if (s != PF_OK) return s;
    PF_CUDA(g, enqueue_attempt(g, g->stream));
    s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    if (accepted) *accepted = c->accepted;
    if (err) *err = c->last_err;
    *dt_inout = c->dt;
    if (c->status == PF_E_NONFINITE) return fail(g, PF_E_NONFINITE, "non-finite error estimate");
    return PF_OK;
}

static pf_status run_loop(pf_grid* g, pf_run_stats* stats) {
    const long long want = g->hctrl->max_attempts;
    const int steps_per_graph = want >= 16 ? 16 : (want >= 4 ? 4 : 1);
    if (!g->graph || g->graph_steps != steps_per_graph) {
        pf_status s = build_graph(g, steps_per_graph);
        if (s != PF_OK) return s;
    }
    long long launched = 0;
    pf_status s = push_ctrl(g);
    if (s != PF_OK) return s;
    for (;;) {
        PF_CUDA(g, cudaGraphLaunch(g->graph, g->stream));
        launched += 6LL * steps_per_graph;
        s = sync_ctrl_to_host(g);
        if (s != PF_OK) return s;
        if (g->hctrl->done) break;
    }
    count_launch(launched);
    g->launches += launched;
    const Ctrl* c = g->hctrl;
    if (stats) {
        stats->n_accepted = c->n_acc;
        stats->n_rejected = c->n_rej;
        stats->t = c->t;
        stats->dt = c->dt;
        stats->last_err = c->last_err;
        stats->launches = launched;
    }
    if (c->status == PF_E_DT_UNDERFLOW) return fail(g, PF_E_DT_UNDERFLOW, "step size fell below dt_min");
    if (c->status == PF_E_NONFINITE) return fail(g, PF_E_NONFINITE, "non-finite error estimate");
    return PF_OK;
}

static void first_step(Ctrl* c) {
    double target = c->t_end;
    if (c->t < c->t_freeze && c->t_freeze < target) target = c->t_freeze;
    if (c->t + c->dt >= target) {
        c->dt_step = target - c->t;
        c->land = 1;
        c->target = target;
    } else {
        c->dt_step = c->dt;
        c->land = 0;
    }
    prepare_step(c);
}

pf_status pf_run_to(pf_grid* g, double t_end, double tol, long long max_steps, pf_run_stats* stats) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (!(tol > 0) || std::isnan(t_end)) return fail(g, PF_E_INVALID, "tol must be > 0 and t_end a number");
    pf_status s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    Ctrl* c = g->hctrl;
    c->t_end = t_end;
    c->tol = tol;
    c->fixed = 0;
    c->eq_window = 0.0;
    c->equilibrium = 0;
    c->single = 0;
    c->max_attempts = max_steps;
    c->n_acc = c->n_rej = 0;
    c->status = 0;
    c->err_bits = 0;
    if (!(c->t < t_end) || max_steps <= 0) {
        if (stats) *stats = {0, 0, c->t, c->dt, c->last_err, 0};
        return PF_OK;
    }
    c->done = 0;
    first_step(c);
    return run_loop(g, stats);
}

pf_status pf_run_fixed(pf_grid* g, long long n_steps, double dt, pf_run_stats* stats) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(g, PF_E_INVALID, "dt must be > 0");
    pf_status s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    Ctrl* c = g->hctrl;
    c->t_end = INFINITY;
    c->tol = 0.0;
    c->fixed = 1;
    c->eq_window = 0.0;
    c->equilibrium = 0;
    c->single = 0;
    c->max_attempts = n_steps;
    c->n_acc = c->n_rej = 0;
    c->status = 0;
    c->err_bits = 0;
    c->dt = dt;
    if (n_steps <= 0) {
        if (stats) *stats = {0, 0, c->t, c->dt, c->last_err, 0};
        return PF_OK;
    }
    c->done = 0;
    first_step(c);
    return run_loop(g, stats);
}

pf_status pf_unfrozen_fraction(pf_grid* g, const int* region, double* uwc, long long* n_ice, long long* n_water,
                               double* smooth) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    int r[6] = {0, g->n1, 0, g->n2, 0, g->n3};
    if (region) {
        std::memcpy(r, region, sizeof(r));
        if (r[0] < 0 || r[1] > g->n1 || r[2] < 0 || r[3] > g->n2 || r[4] < 0 || r[5] > g->n3 || r[0] > r[1] ||
            r[2] > r[3] || r[4] > r[5])
            return fail(g, PF_E_INVALID, "region outside the grid");
    }
    const long long n = (long long)(r[1] - r[0]) * (r[3] - r[2]) * (r[5] - r[4]);
    const int nb = n > 0 ? blocks_for(n, 256) : 1;
    UwcPart* parts = (UwcPart*)g->red;
    UwcPart* res = parts + (152 * 16);
    double** tab = g->ptab;  // the kernel picks the current state buffer from ctrl->cur
    k_uwc_partial<256><<<nb, 256, 0, g->stream>>>(g->G64, (const double* const*)tab, (const double* const*)(tab + 2),
                                                  g->dctrl, g->model == PF_MODEL_TEMP, g->p.gamma, g->p.zeta, g->n1,
                                                  g->n2, r[0], r[1], r[2], r[3], r[4], r[5], parts);
    k_uwc_final<<<1, 256, 0, g->stream>>>(parts, nb, res);
    count_launch(2);
    g->launches += 2;
    PF_CUDA(g, cudaGetLastError());
    UwcPart hres;
    PF_CUDA(g, cudaMemcpyAsync(&hres, res, sizeof(UwcPart), cudaMemcpyDeviceToHost, g->stream));
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    if (n_ice) *n_ice = (long long)hres.ni;
    if (n_water) *n_water = (long long)hres.nw;
    if (uwc) *uwc = hres.nw ? 1.0 - (double)hres.ni / (double)hres.nw : NAN;
    if (smooth) *smooth = hres.sd != 0.0 ? 1.0 - hres.sn / hres.sd : NAN;
    return PF_OK;
}

pf_status pf_profile_stages(pf_grid* g, int n_attempts, double* stage_ms) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (n_attempts < 1 || !stage_ms) return fail(g, PF_E_INVALID, "n_attempts >= 1 and stage_ms required");
    pf_status s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    Ctrl* c = g->hctrl;
    c->fixed = 1;
    c->single = 1;
    c->dt_step = c->dt;
    c->eq_window = 0.0;
    c->equilibrium = 0;
    c->land = 0;
    prepare_step(c);
    c->done = 0;
    c->status = 0;
    c->err_bits = 0;
    s = push_ctrl(g);
    if (s != PF_OK) return s;
    cudaEvent_t ev[7];
    for (int q = 0; q < 7; ++q) PF_CUDA(g, cudaEventCreate(&ev[q]));
    double acc[6] = {0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < n_attempts && e == cudaSuccess; ++a) {
        e = cudaEventRecord(ev[0], g->stream);
        for (int st = 1; st <= 5 && e == cudaSuccess; ++st) {
            e = launch_stage(g, st, g->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev[st], g->stream);
        }
        if (e == cudaSuccess) {
            k_controller<<<1, 32, 0, g->stream>>>(g->dctrl);
            count_launch();
            g->launches++;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[6], g->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[6]);
        for (int q = 0; q < 6 && e == cudaSuccess; ++q) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
            acc[q] += ms;
        }
    }
    for (int q = 0; q < 7; ++q) cudaEventDestroy(ev[q]);
    if (e != cudaSuccess) return fail(g, PF_E_CUDA, std::string("profile: ") + cudaGetErrorString(e));
    for (int q = 0; q < 6; ++q) stage_ms[q] = acc[q] / n_attempts;
    return sync_ctrl_to_host(g);
}

pf_status pf_max_phase_rate(pf_grid* g, double* max_rate) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (!max_rate) return fail(g, PF_E_INVALID, "max_rate is NULL");
    pf_status s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    const int cur = g->hctrl->cur;
    const double t = g->hctrl->t;
    cudaError_t e;
    const int nb = blocks_for(g->N, 256);
    double* parts = (double*)g->red;
    double* res = parts + 152 * 16;
    if (is_f32(g)) {
        // binary32 copies of the binary64 state feed the binary32 right-hand side
        if (has_th(g)) { k_to_f32<<<nb, 256, 0, g->stream>>>(g->y_th[cur], (float*)g->ua_th, g->N); count_launch(); }
        if (has_ph(g)) { k_to_f32<<<nb, 256, 0, g->stream>>>(g->y_ph[cur], (float*)g->ua_ph, g->N); count_launch(); }
        StageArgs<float> a = make_args<float>(g);
        a.in_th = (const float*)g->ua_th; a.in_ph = (const float*)g->ua_ph;
        a.out_th = nullptr; a.out_ph = (float*)g->k1_ph;
        if (!has_ph(g)) a.out_ph = (float*)g->k1_th;  // Temp: dphi goes to the theta slot
        a.t_rhs = t;
        e = launch_stage_f32(g->model, g->rx, 0, a, g->by, g->stream);
        if (e == cudaSuccess) {
            k_maxabs_partial<float, 256><<<nb, 256, 0, g->stream>>>((const float*)a.out_ph, g->N, parts);
            count_launch();
        }
    } else {
        StageArgs<double> a = make_args<double>(g);
        a.in_th = g->y_th[cur]; a.in_ph = g->y_ph[cur];
        a.out_th = nullptr; a.out_ph = g->scratch64;
        a.t_rhs = t;
        e = launch_stage_f64(g->model, g->rx, 0, a, g->by, g->stream);
        if (e == cudaSuccess) {
            k_maxabs_partial<double, 256><<<nb, 256, 0, g->stream>>>(g->scratch64, g->N, parts);
            count_launch();
        }
    }
    if (e != cudaSuccess) return fail(g, PF_E_CUDA, std::string("max rate: ") + cudaGetErrorString(e));
    k_max_final<<<1, 32, 0, g->stream>>>(parts, nb, res);
    count_launch();
    PF_CUDA(g, cudaGetLastError());
    PF_CUDA(g, cudaMemcpyAsync(max_rate, res, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    return PF_OK;
}


// ------------------------------------------------------------------ tiles and autotuning

static pf_status set_tiles_impl(pf_grid* g, int by, int zc) {
    if (by != 4 && by != 8 && by != 16) return fail(g, PF_E_INVALID, "by must be 4, 8 or 16");
    if (zc < 1) return fail(g, PF_E_INVALID, "zc must be >= 1");
    if (by != g->by || zc != g->zc) free_graph(g);
    g->by = by;
    g->zc = zc;
    return PF_OK;
}

pf_status pf_set_tiles(pf_grid* g, int by, int zc) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    return set_tiles_impl(g, by, zc);
}

pf_status pf_get_tiles(pf_grid* g, int* by, int* zc) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    if (by) *by = g->by;
    if (zc) *zc = g->zc;
    return PF_OK;
}

static const int kTuneBY[3] = {4, 8, 16};
// z chunks: powers of two plus the values between them that let small grids fill the SMs in about one
// wave of blocks (a 50 x 50 x 100 grid in 32 x 4 columns: zc = 5 gives 520 blocks, zc = 4 gives 650)
constexpr int NZC = 12;
static const int kTuneZC[NZC] = {2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 64};

// Time the plain right-hand side (the stage kernels' common body) for every (by, zc) candidate on the
// grid itself; ms[b][z] = best of 3 launches (infinity for skipped candidates).
// Device time of one Merson attempt's five stage kernels for every tile shape (best of three after
// a warm-up).  The controller is not launched: the state, the time and the step counters stay as
// they are (stage 5 writes only the spare state buffer), and the control block is restored after.
static pf_status tune_table(pf_grid* g, double ms[3][NZC]) {
    pf_status s = sync_ctrl_to_host(g);
    if (s != PF_OK) return s;
    const Ctrl saved = *g->hctrl;
    Ctrl* c = g->hctrl;
    c->dt_step = c->dt;
    prepare_step(c);
    c->done = 0;
    c->status = 0;
    c->fixed = 1;
    c->single = 1;
    s = push_ctrl(g);
    if (s != PF_OK) return s;
    cudaEvent_t e0, e1;
    PF_CUDA(g, cudaEventCreate(&e0));
    PF_CUDA(g, cudaEventCreate(&e1));
    cudaError_t e = cudaSuccess;
    const int by0 = g->by, zc0 = g->zc;
    for (int b = 0; b < 3; ++b)
        for (int z = 0; z < NZC; ++z) {
            ms[b][z] = INFINITY;
            if (e != cudaSuccess) continue;
            if (kTuneZC[z] > 2 * g->n3 && z > 0) continue;
            g->by = kTuneBY[b];
            g->zc = kTuneZC[z];
            double best = INFINITY;
            for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
                e = cudaEventRecord(e0, g->stream);
                for (int st = 1; st <= 5 && e == cudaSuccess; ++st) e = launch_stage(g, st, g->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (r > 0 && t < best) best = t;  // first launch is a warm-up
            }
            ms[b][z] = best;
        }
    g->by = by0;
    g->zc = zc0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(g, PF_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    *g->hctrl = saved;
    s = push_ctrl(g);
    if (s != PF_OK) return s;
    PF_CUDA(g, cudaStreamSynchronize(g->stream));
    return PF_OK;
}

static std::string tune_key(const pf_grid* g) {
    char k[128];
    snprintf(k, sizeof(k), "%dx%dx%d/m%d/r%d/p%d", g->n1, g->n2, g->n3, g->model, g->rx, g->prec);
    return k;
}

// cache file: one line per grid shape "key by zc ms"
static bool cache_lookup(const char* path, const std::string& key, int* by, int* zc, double* ms) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char k[128];
    int b, z;
    double m;
    bool found = false;
    while (fscanf(f, "%127s %d %d %lf", k, &b, &z, &m) == 4)
        if (key == k) { *by = b; *zc = z; *ms = m; found = true; }
    fclose(f);
    return found;
}

static void cache_store(const char* path, const std::string& key, int by, int zc, double ms) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %.6f\n", key.c_str(), by, zc, ms);
    fclose(f);
}

pf_status pf_autotune(pf_grid* g, const char* cache_path, int* by_out, int* zc_out, double* ms_out) {
    if (!g) return fail(nullptr, PF_E_INVALID, "grid is NULL");
    int by = 8, zc = 32;
    double best = INFINITY;
    const std::string key = tune_key(g);
    if (!cache_lookup(cache_path, key, &by, &zc, &best)) {
        double ms[3][NZC];
        pf_status s = tune_table(g, ms);
        if (s != PF_OK) return s;
        for (int b = 0; b < 3; ++b)
            for (int z = 0; z < NZC; ++z)
                if (ms[b][z] < best) { best = ms[b][z]; by = kTuneBY[b]; zc = kTuneZC[z]; }
        cache_store(cache_path, key, by, zc, best);
    }
    pf_status s = set_tiles_impl(g, by, zc);
    if (s != PF_OK) return s;
    if (by_out) *by_out = by;
    if (zc_out) *zc_out = zc;
    if (ms_out) *ms_out = best;
    return PF_OK;
}

// ------------------------------------------------------------------ batched persistent runs

struct pf_batch {
    int n = 0;
    std::vector<pf_grid*> g;
    int model = 0, rx = 0, prec = 0, by = 8;
    cudaStream_t stream = nullptr, cap = nullptr;
    void* d_args = nullptr;
    Ctrl** d_ctrls = nullptr;
    int4* d_tiles = nullptr;
    BatchPlan* d_plan = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long iters = 0;
    std::string err;
};

static pf_status bfail(pf_batch* b, pf_status s, const std::string& m) {
    if (b) b->err = m;
    else t_create_err = m;
    return s;
}

#define PF_BCUDA(b, call)                                                                              \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return bfail((b), PF_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void batch_free_graph(pf_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// per-instance stage arguments and tile lattices on the device
static pf_status batch_upload(pf_batch* b) {
    std::vector<int4> tiles(b->n);
    for (int q = 0; q < b->n; ++q) {
        pf_grid* g = b->g[q];
        g->by = b->by;
        const int nbx = (g->n1 + TX - 1) / TX, nby = (g->n2 + b->by - 1) / b->by, nbz = (g->n3 + g->zc - 1) / g->zc;
        tiles[q] = make_int4(nbx, nby, nbz, nbx * nby * nbz);
    }
    PF_BCUDA(b, cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int4) * b->n, cudaMemcpyHostToDevice));
    if (b->prec == PF_PREC_FP32_FIELDS) {
        std::vector<StageArgs<float>> a(b->n);
        for (int q = 0; q < b->n; ++q) a[q] = make_args<float>(b->g[q]);
        PF_BCUDA(b, cudaMemcpy(b->d_args, a.data(), sizeof(StageArgs<float>) * b->n, cudaMemcpyHostToDevice));
    } else {
        std::vector<StageArgs<double>> a(b->n);
        for (int q = 0; q < b->n; ++q) a[q] = make_args<double>(b->g[q]);
        PF_BCUDA(b, cudaMemcpy(b->d_args, a.data(), sizeof(StageArgs<double>) * b->n, cudaMemcpyHostToDevice));
    }
    return PF_OK;
}

static cudaError_t batch_enqueue_step(pf_batch* b, cudaStream_t s, int blocks, cudaGraphConditionalHandle h) {
    cudaError_t e = cudaSuccess;
    for (int st = 1; st <= 5 && e == cudaSuccess; ++st) {
        if (b->prec == PF_PREC_FP32_FIELDS)
            e = launch_batch_stage_f32(b->model, b->rx, st, (const StageArgs<float>*)b->d_args, b->d_plan, b->d_tiles,
                                       b->by, blocks, s);
        else
            e = launch_batch_stage_f64(b->model, b->rx, st, (const StageArgs<double>*)b->d_args, b->d_plan, b->d_tiles,
                                       b->by, blocks, s);
    }
    if (e != cudaSuccess) return e;
    k_batch_controller<<<(BATCH_MAX + 127) / 128, 128, 0, s>>>(b->d_ctrls, b->d_plan);
    k_batch_plan<<<1, 32, 0, s>>>(b->d_ctrls, b->d_tiles, b->n, b->d_plan, h);
    count_launch(2);
    return cudaGetLastError();
}

// Graph: plan -> WHILE(any instance active and iter <= max_iter) { stages 1..5, controller, plan }.
static pf_status batch_build_graph(pf_batch* b) {
    batch_free_graph(b);
    const long long before = pfgb::g_launches.load();
    cudaGraph_t graph = nullptr;
    PF_BCUDA(b, cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    // persistent stage grid: enough blocks to fill every SM (the blocks loop over tiles)
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * (2048 / (TX * b->by)) / 2;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(b->cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        k_batch_plan<<<1, 32, 0, b->cap>>>(b->d_ctrls, b->d_tiles, b->n, b->d_plan, h);
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = e2;
    }
    cudaGraphNode_t first = nullptr;
    size_t nn = 1;
    if (e == cudaSuccess) e = cudaGraphGetNodes(graph, &first, &nn);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, graph, &first, nullptr, 1, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = batch_enqueue_step(b, b->cap, blocks, h);
            cudaError_t e2 = cudaStreamEndCapture(b->cap, &body);
            e = e1 != cudaSuccess ? e1 : e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    // launches made during capture are recorded, not executed
    pfgb::g_launches.store(before);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        cudaGetLastError();
        return bfail(b, PF_E_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    return PF_OK;
}

const char* pf_batch_last_error(const pf_batch* b) { return b ? b->err.c_str() : t_create_err.c_str(); }

pf_status pf_batch_destroy(pf_batch* b) {
    if (!b) return PF_OK;
    cudaStreamSynchronize(b->stream);
    batch_free_graph(b);
    for (pf_grid* g : b->g) pf_destroy_grid(g);
    if (b->d_args) cudaFree(b->d_args);
    if (b->d_ctrls) cudaFree(b->d_ctrls);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_plan) cudaFree(b->d_plan);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return PF_OK;
}

pf_status pf_batch_create(int n, pf_grid* const* grids, pf_batch** out) {
    if (!out) return bfail(nullptr, PF_E_INVALID, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > BATCH_MAX || !grids) return bfail(nullptr, PF_E_INVALID, "need 1..256 grids");
    for (int q = 0; q < n; ++q) {
        if (!grids[q]) return bfail(nullptr, PF_E_INVALID, "NULL grid");
        for (int r = 0; r < q; ++r)
            if (grids[r] == grids[q]) return bfail(nullptr, PF_E_INVALID, "a grid appears twice");
        if (grids[q]->model != grids[0]->model || grids[q]->rx != grids[0]->rx || grids[q]->prec != grids[0]->prec)
            return bfail(nullptr, PF_E_INVALID, "all grids of a batch share model, reaction and precision");
    }
    pf_batch* b = new pf_batch();
    b->n = n;
    b->g.assign(grids, grids + n);
    b->model = grids[0]->model;
    b->rx = grids[0]->rx;
    b->prec = grids[0]->prec;
    b->by = grids[0]->by;
    b->stream = grids[0]->stream;
    const size_t asz = b->prec == PF_PREC_FP32_FIELDS ? sizeof(StageArgs<float>) : sizeof(StageArgs<double>);
    bool ok = cudaMalloc(&b->d_args, asz * n) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_ctrls, sizeof(Ctrl*) * n) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_tiles, sizeof(int4) * n) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_plan, sizeof(BatchPlan)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        b->g.clear();
        pf_batch_destroy(b);
        return bfail(nullptr, PF_E_OOM, "batch allocation failed");
    }
    std::vector<Ctrl*> c(n);
    for (int q = 0; q < n; ++q) c[q] = grids[q]->dctrl;
    if (cudaMemcpy(b->d_ctrls, c.data(), sizeof(Ctrl*) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        b->g.clear();
        pf_batch_destroy(b);
        return bfail(nullptr, PF_E_CUDA, "batch initialisation failed");
    }
    for (int q = 0; q < n; ++q) cudaStreamSynchronize(grids[q]->stream);
    pf_status s = batch_upload(b);
    if (s != PF_OK) {
        std::string m = b->err;
        b->g.clear();
        pf_batch_destroy(b);
        return bfail(nullptr, s, m);
    }
    *out = b;
    return PF_OK;
}

pf_grid* pf_batch_grid(pf_batch* b, int i) { return (b && i >= 0 && i < b->n) ? b->g[i] : nullptr; }

pf_status pf_batch_autotune(pf_batch* b, const char* cache_path) {
    if (!b) return bfail(nullptr, PF_E_INVALID, "batch is NULL");
    // a common block height for the batched kernels, then the best z chunk per instance
    std::vector<std::array<std::array<double, NZC>, 3>> t(b->n);
    double sum[3] = {0, 0, 0};
    for (int q = 0; q < b->n; ++q) {
        double ms[3][NZC];
        pf_status s = tune_table(b->g[q], ms);
        if (s != PF_OK) return bfail(b, s, b->g[q]->err);
        for (int bb = 0; bb < 3; ++bb) {
            double m = INFINITY;
            for (int z = 0; z < NZC; ++z) { t[q][bb][z] = ms[bb][z]; m = fmin(m, ms[bb][z]); }
            sum[bb] += m;
        }
    }
    int bb = 0;
    for (int k = 1; k < 3; ++k) if (sum[k] < sum[bb]) bb = k;
    b->by = kTuneBY[bb];
    for (int q = 0; q < b->n; ++q) {
        int z = 0;
        for (int k = 1; k < NZC; ++k) if (t[q][bb][k] < t[q][bb][z]) z = k;
        set_tiles_impl(b->g[q], b->by, kTuneZC[z]);
        cache_store(cache_path, tune_key(b->g[q]), b->by, kTuneZC[z], t[q][bb][z]);
    }
    batch_free_graph(b);
    return batch_upload(b);
}

pf_status pf_batch_run_to(pf_batch* b, const double* t_end, const double* eq_window, double eq_rel_tol,
                          const double* eq_rate, double tol, long long max_steps, pf_batch_result* res) {
    if (!b) return bfail(nullptr, PF_E_INVALID, "batch is NULL");
    if (!(eq_rel_tol >= 0.0)) return bfail(b, PF_E_INVALID, "eq_rel_tol must be >= 0");
    if (!t_end || !(tol > 0) || max_steps < 1) return bfail(b, PF_E_INVALID, "t_end, tol > 0, max_steps >= 1 required");
    if (max_steps > (1LL << 30)) max_steps = 1LL << 30;
    for (int q = 0; q < b->n; ++q) {
        pf_grid* g = b->g[q];
        PF_BCUDA(b, cudaMemcpy(g->hctrl, g->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
        Ctrl* c = g->hctrl;
        c->t_end = t_end[q];
        c->tol = tol;
        c->fixed = 0;
        c->single = 0;
        c->max_attempts = max_steps;
        c->n_acc = c->n_rej = 0;
        c->status = 0;
        c->err_bits = 0;
        c->ice_count = 0;
        c->pore_count = 0;
        c->rate_bits = 0;
        c->prev_count = -1;
        c->eq_window = eq_window ? eq_window[q] : 0.0;
        c->eq_rel_tol = eq_rel_tol;
        c->eq_rate = eq_rate ? eq_rate[q] : 0.0;
        c->equilibrium = 0;
        c->t_eq = NAN;
        c->done = (c->t < t_end[q]) ? 0 : 1;
        if (!c->done) first_step(c);
        PF_BCUDA(b, cudaMemcpy(g->dctrl, c, sizeof(Ctrl), cudaMemcpyHostToDevice));
    }
    BatchPlan hp = {};
    hp.iter = 0;
    hp.max_iter = (int)max_steps + 1;
    PF_BCUDA(b, cudaMemcpyAsync(b->d_plan, &hp, 4 * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    if (!b->exec) {
        pf_status s = batch_build_graph(b);
        if (s != PF_OK) return s;
    }
    PF_BCUDA(b, cudaGraphLaunch(b->exec, b->stream));
    PF_BCUDA(b, cudaMemcpyAsync(&hp, b->d_plan, 4 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    PF_BCUDA(b, cudaStreamSynchronize(b->stream));
    b->iters = hp.iter;
    count_launch(1 + 7LL * (hp.iter - 1));  // plan, then 5 stages + controller + plan per iteration
    for (int q = 0; q < b->n; ++q) {
        pf_grid* g = b->g[q];
        PF_BCUDA(b, cudaMemcpy(g->hctrl, g->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
        const Ctrl* c = g->hctrl;
        if (res) {
            res[q].stats.n_accepted = c->n_acc;
            res[q].stats.n_rejected = c->n_rej;
            res[q].stats.t = c->t;
            res[q].stats.dt = c->dt;
            res[q].stats.last_err = c->last_err;
            res[q].stats.launches = 0;
            res[q].t_eq = c->equilibrium ? c->t_eq : NAN;
            res[q].rate = c->last_rate;
            res[q].equilibrium = c->equilibrium;
            res[q].status = c->status;
        }
    }
    return PF_OK;
}

long long pf_batch_iterations(const pf_batch* b) { return b ? b->iters : -1; }

}  // extern "C"

// ------------------------------------------------------------------ z-slab multi-domain mode
// The paper's parallel layer (Sec. 2.5): the domain is cut along x3 into slabs, each stage's input
// planes next to a cut are exchanged with the neighbour slab, and the step control uses the error
// maximum over all slabs.  Here every slab is a grid with ghost planes in one process on one GPU:
// the exchange is a copy kernel after each stage, the slabs share one control block (so the
// error maximum and the pore counts accumulate over all slabs and one controller decides).

namespace {
// Pointers (local plane 0) of one slab's exchanged buffers: [theta, phi][y0, y1, ua, ub, y32_0, y32_1].
struct SlabTab {
    void* f[2][6];
    int n3;
    int pad;
};

// which: 0 = ua, 1 = ub (stage inputs written by the stage just run), 2 = y[cur ^ 1] (the step's
// candidate state), 3 = y[cur] (the state), 4 = y32[cur ^ 1] (the binary32 copy of the candidate state
// that stage 5 writes in the binary32 form of the full model).  blockIdx.y = cut * 4 + direction * 2 + field.
template <typename TF>
__global__ void k_halo(const SlabTab* __restrict__ tab, long long plane, int which, int fields,
                       const Ctrl* __restrict__ c) {
    const int r = blockIdx.y;
    const int cut = r >> 2, dir = (r >> 1) & 1, f = r & 1;
    if (!((fields >> f) & 1)) return;
    const int slot = which < 2 ? 2 + which : (which == 2 ? (c->cur ^ 1) : (which == 3 ? c->cur : 4 + (c->cur ^ 1)));
    const SlabTab& lo = tab[cut];
    const SlabTab& hi = tab[cut + 1];
    const TF* src;
    TF* dst;
    if (dir == 0) {  // top plane of the lower slab -> ghost plane below the upper slab
        src = (const TF*)lo.f[f][slot] + (long long)(lo.n3 - 1) * plane;
        dst = (TF*)hi.f[f][slot] - plane;
    } else {         // bottom plane of the upper slab -> ghost plane above the lower slab
        src = (const TF*)hi.f[f][slot];
        dst = (TF*)lo.f[f][slot] + (long long)lo.n3 * plane;
    }
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < plane; q += (long long)gridDim.x * blockDim.x)
        dst[q] = src[q];
}
}  // namespace

struct pf_slabs {
    int P = 0;
    int n1 = 0, n2 = 0, n3 = 0;
    std::vector<int> kb;            // plane boundaries, P + 1 values from 0 to n3
    std::vector<pf_grid*> s;        // slab 0 owns the shared control block
    SlabTab* d_tab = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    long long halo_bytes = 0;       // bytes the halo exchanges of the last run moved
    std::string err;
};

static pf_status sfail(pf_slabs* S, pf_status st, const std::string& m) {
    if (S) S->err = m;
    else t_create_err = m;
    return st;
}

#define PF_SCUDA(S, call)                                                                              \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return sfail((S), PF_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// bytes one exchange moves (every cut, both directions, integrated fields)
static long long halo_exchange_bytes(const pf_slabs* S, int which) {
    const pf_grid* g = S->s[0];
    const int nf = (has_th(g) ? 1 : 0) + (has_ph(g) ? 1 : 0);
    const size_t esz = (which == 2 || which == 3) ? sizeof(double) : fbytes(g);
    return (long long)(S->P - 1) * 2 * nf * (long long)esz * S->n1 * S->n2;
}

static cudaError_t halo(pf_slabs* S, int which, cudaStream_t st) {
    if (S->P < 2) return cudaSuccess;
    const pf_grid* g = S->s[0];
    const long long plane = (long long)S->n1 * S->n2;
    const int fields = (has_th(g) ? 1 : 0) | (has_ph(g) ? 2 : 0);
    dim3 grid((unsigned)std::min<long long>((plane + 255) / 256, 1024), (unsigned)(4 * (S->P - 1)));
    if (which == 2 || which == 3 || !is_f32(g))
        k_halo<double><<<grid, 256, 0, st>>>(S->d_tab, plane, which, fields, g->dctrl);
    else
        k_halo<float><<<grid, 256, 0, st>>>(S->d_tab, plane, which, fields, g->dctrl);
    count_launch();
    return cudaGetLastError();
}

// One Merson attempt over all slabs: each stage on every slab, then the exchange of the planes the
// next stage reads at the cuts; the controller once (shared control block).
static cudaError_t slabs_enqueue_attempt(pf_slabs* S, cudaStream_t st) {
    for (int stage = 1; stage <= 5; ++stage) {
        for (pf_grid* g : S->s) {
            cudaError_t e = launch_stage(g, stage, st);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = halo(S, stage == 5 ? 2 : (stage % 2 == 1 ? 0 : 1), st);
        if (e == cudaSuccess && stage == 5 && has_y32(S->s[0])) e = halo(S, 4, st);
        if (e != cudaSuccess) return e;
    }
    k_controller<<<1, 32, 0, st>>>(S->s[0]->dctrl);
    count_launch();
    return cudaGetLastError();
}

static long long slabs_attempt_launches(const pf_slabs* S) {
    const int extra = (S->P > 1 && has_y32(S->s[0])) ? 1 : 0;
    return 5LL * (S->P + (S->P > 1 ? 1 : 0)) + extra + 1;
}

static void slabs_free_graph(pf_slabs* S) {
    if (S->graph) cudaGraphExecDestroy(S->graph);
    S->graph = nullptr;
    S->graph_steps = 0;
}

static pf_status slabs_build_graph(pf_slabs* S, int steps) {
    slabs_free_graph(S);
    pf_grid* g0 = S->s[0];
    cudaGraph_t graph = nullptr;
    PF_SCUDA(S, cudaStreamBeginCapture(g0->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < steps && e == cudaSuccess; ++q) e = slabs_enqueue_attempt(S, g0->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(g0->cap_stream, &graph);
    // launches made during capture are only recorded, not executed
    pfgb::g_launches.fetch_sub((long long)steps * slabs_attempt_launches(S), std::memory_order_relaxed);
    for (pf_grid* g : S->s) g->launches -= (long long)steps * 5;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return sfail(S, PF_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&S->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        S->graph = nullptr;
        return sfail(S, PF_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
    }
    S->graph_steps = steps;
    return PF_OK;
}

static void slabs_destroy_impl(pf_slabs* S) {
    slabs_free_graph(S);
    // slabs other than 0 borrow slab 0's control block: destroy them first
    for (int q = (int)S->s.size() - 1; q >= 0; --q)
        if (S->s[q]) destroy_impl(S->s[q]);
    if (S->d_tab) cudaFree(S->d_tab);
    delete S;
}

extern "C" {

const char* pf_slabs_last_error(const pf_slabs* S) { return S ? S->err.c_str() : t_create_err.c_str(); }

pf_status pf_slabs_create(int n1, int n2, int n3, double h, int model, int reaction, int precision,
                          const pf_params* p, int nslabs, const int* planes, void* stream, pf_slabs** out) {
    if (!out) return sfail(nullptr, PF_E_INVALID, "out is NULL");
    *out = nullptr;
    if (nslabs < 1 || nslabs > 1024 || n3 < nslabs) return sfail(nullptr, PF_E_INVALID, "need 1 <= nslabs <= n3");
    std::vector<int> kb(nslabs + 1);
    for (int q = 0; q <= nslabs; ++q) kb[q] = planes ? planes[q] : (int)((long long)n3 * q / nslabs);
    if (kb[0] != 0 || kb[nslabs] != n3) return sfail(nullptr, PF_E_INVALID, "planes must run from 0 to n3");
    for (int q = 0; q < nslabs; ++q)
        if (kb[q + 1] <= kb[q]) return sfail(nullptr, PF_E_INVALID, "every slab needs at least one plane");
    pf_slabs* S = new pf_slabs();
    S->P = nslabs;
    S->n1 = n1; S->n2 = n2; S->n3 = n3;
    S->kb = kb;
    S->s.assign(nslabs, nullptr);
    for (int q = 0; q < nslabs; ++q) {
        SlabOpts so;
        so.zg_lo = q > 0 ? 1 : 0;
        so.zg_hi = q < nslabs - 1 ? 1 : 0;
        so.k_off = kb[q];
        so.ctrl_owner = q > 0 ? S->s[0] : nullptr;
        pf_status st = create_impl(n1, n2, kb[q + 1] - kb[q], h, model, reaction, precision, p, stream, so, &S->s[q]);
        if (st != PF_OK) {
            const std::string m = t_create_err;
            slabs_destroy_impl(S);
            return sfail(nullptr, st, "slab " + std::to_string(q) + ": " + m);
        }
    }
    std::vector<SlabTab> tab(nslabs);
    for (int q = 0; q < nslabs; ++q) {
        pf_grid* g = S->s[q];
        SlabTab& t = tab[q];
        t.f[0][0] = g->y_th[0]; t.f[0][1] = g->y_th[1]; t.f[0][2] = g->ua_th; t.f[0][3] = g->ub_th;
        t.f[1][0] = g->y_ph[0]; t.f[1][1] = g->y_ph[1]; t.f[1][2] = g->ua_ph; t.f[1][3] = g->ub_ph;
        t.f[0][4] = g->y32_th[0]; t.f[0][5] = g->y32_th[1];
        t.f[1][4] = g->y32_ph[0]; t.f[1][5] = g->y32_ph[1];
        t.n3 = g->n3;
        t.pad = 0;
    }
    if (cudaMalloc(&S->d_tab, sizeof(SlabTab) * nslabs) != cudaSuccess ||
        cudaMemcpy(S->d_tab, tab.data(), sizeof(SlabTab) * nslabs, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        slabs_destroy_impl(S);
        return sfail(nullptr, PF_E_OOM, "slab table allocation failed");
    }
    *out = S;
    return PF_OK;
}

pf_status pf_slabs_destroy(pf_slabs* S) {
    if (!S) return PF_OK;
    cudaStreamSynchronize(S->s[0]->stream);
    slabs_destroy_impl(S);
    return PF_OK;
}

pf_grid* pf_slabs_grid(pf_slabs* S, int q) {
    if (!S || q < 0 || q >= S->P) return nullptr;
    return S->s[q];
}

pf_status pf_slabs_set_geometry(pf_slabs* S, const double* spheres, long long n, double x3_cap) {
    if (!S) return sfail(nullptr, PF_E_INVALID, "slabs is NULL");
    for (pf_grid* g : S->s) {
        pf_status st = pf_set_geometry(g, spheres, n, x3_cap);
        if (st != PF_OK) return sfail(S, st, g->err);
    }
    return PF_OK;
}

pf_status pf_slabs_set_tiles(pf_slabs* S, int by, int zc) {
    if (!S) return sfail(nullptr, PF_E_INVALID, "slabs is NULL");
    for (pf_grid* g : S->s) {
        pf_status st = set_tiles_impl(g, by, zc);
        if (st != PF_OK) return sfail(S, st, g->err);
    }
    slabs_free_graph(S);
    return PF_OK;
}

pf_status pf_slabs_set_state(pf_slabs* S, const double* theta, const double* phi, double t, double dt) {
    if (!S) return sfail(nullptr, PF_E_INVALID, "slabs is NULL");
    pf_grid* g0 = S->s[0];
    if (has_th(g0) && !theta) return sfail(S, PF_E_INVALID, "theta is NULL");
    if (has_ph(g0) && !phi) return sfail(S, PF_E_INVALID, "phi is NULL");
    const long long plane = (long long)S->n1 * S->n2;
    for (int q = S->P - 1; q >= 0; --q) {  // slab 0 last: its pf_set_state resets the shared control block
        pf_grid* g = S->s[q];
        const long long off = (long long)S->kb[q] * plane;
        if (q == 0) {
            pf_status st = pf_set_state(g, theta ? theta + off : nullptr, phi ? phi + off : nullptr, t, dt);
            if (st != PF_OK) return sfail(S, st, g->err);
        } else {
            if (has_th(g)) PF_SCUDA(S, cudaMemcpyAsync(g->y_th[0], theta + off, sizeof(double) * g->N, cudaMemcpyHostToDevice, g->stream));
            if (has_ph(g)) PF_SCUDA(S, cudaMemcpyAsync(g->y_ph[0], phi + off, sizeof(double) * g->N, cudaMemcpyHostToDevice, g->stream));
        }
    }
    PF_SCUDA(S, halo(S, 3, g0->stream));
    // the binary32 copies again, now that the ghost planes of the state are filled
    for (pf_grid* g : S->s) {
        pf_status st = refresh_y32(g, 0);
        if (st != PF_OK) return sfail(S, st, g->err);
    }
    PF_SCUDA(S, cudaStreamSynchronize(g0->stream));
    return PF_OK;
}

pf_status pf_slabs_get_state(pf_slabs* S, double* theta, double* phi, double* t, double* dt) {
    if (!S) return sfail(nullptr, PF_E_INVALID, "slabs is NULL");
    pf_grid* g0 = S->s[0];
    pf_status st = sync_ctrl_to_host(g0);
    if (st != PF_OK) return sfail(S, st, g0->err);
    const int cur = g0->hctrl->cur;
    const long long plane = (long long)S->n1 * S->n2;
    for (int q = 0; q < S->P; ++q) {
        pf_grid* g = S->s[q];
        const long long off = (long long)S->kb[q] * plane;
        if (theta && has_th(g))
            PF_SCUDA(S, cudaMemcpyAsync(theta + off, g->y_th[cur], sizeof(double) * g->N, cudaMemcpyDeviceToHost, g->stream));
        if (phi && has_ph(g))
            PF_SCUDA(S, cudaMemcpyAsync(phi + off, g->y_ph[cur], sizeof(double) * g->N, cudaMemcpyDeviceToHost, g->stream));
    }
    PF_SCUDA(S, cudaStreamSynchronize(g0->stream));
    if (theta && !has_th(g0)) for (long long q = 0; q < (long long)S->n3 * plane; ++q) theta[q] = g0->p.theta_micro;
    if (t) *t = g0->hctrl->t;
    if (dt) *dt = g0->hctrl->dt;
    return PF_OK;
}

pf_status pf_slabs_run_to(pf_slabs* S, double t_end, double tol, long long max_steps, pf_run_stats* stats) {
    if (!S) return sfail(nullptr, PF_E_INVALID, "slabs is NULL");
    if (!(tol > 0) || std::isnan(t_end)) return sfail(S, PF_E_INVALID, "tol must be > 0 and t_end a number");
    pf_grid* g0 = S->s[0];
    pf_status st = sync_ctrl_to_host(g0);
    if (st != PF_OK) return sfail(S, st, g0->err);
    Ctrl* c = g0->hctrl;
    c->t_end = t_end;
    c->tol = tol;
    c->fixed = 0;
    c->eq_window = 0.0;
    c->equilibrium = 0;
    c->single = 0;
    c->max_attempts = max_steps;
    c->n_acc = c->n_rej = 0;
    c->status = 0;
    c->err_bits = 0;
    S->halo_bytes = 0;
    if (!(c->t < t_end) || max_steps <= 0) {
        if (stats) *stats = {0, 0, c->t, c->dt, c->last_err, 0};
        return PF_OK;
    }
    c->done = 0;
    first_step(c);
    const int steps_per_graph = max_steps >= 16 ? 16 : (max_steps >= 4 ? 4 : 1);
    if (!S->graph || S->graph_steps != steps_per_graph) {
        st = slabs_build_graph(S, steps_per_graph);
        if (st != PF_OK) return st;
    }
    st = push_ctrl(g0);
    if (st != PF_OK) return sfail(S, st, g0->err);
    long long launched = 0, replays = 0;
    for (;;) {
        PF_SCUDA(S, cudaGraphLaunch(S->graph, g0->stream));
        launched += steps_per_graph * slabs_attempt_launches(S);
        ++replays;
        st = sync_ctrl_to_host(g0);
        if (st != PF_OK) return sfail(S, st, g0->err);
        if (c->done) break;
    }
    count_launch(launched);
    // every replayed attempt exchanges the five stages' planes (attempts after the run ended copy
    // unchanged planes)
    long long per_attempt = 0;
    for (int w : {0, 1, 0, 1, 2}) per_attempt += halo_exchange_bytes(S, w);
    if (has_y32(S->s[0])) per_attempt += halo_exchange_bytes(S, 4);
    S->halo_bytes = replays * steps_per_graph * per_attempt;
    if (stats) {
        stats->n_accepted = c->n_acc;
        stats->n_rejected = c->n_rej;
        stats->t = c->t;
        stats->dt = c->dt;
        stats->last_err = c->last_err;
        stats->launches = launched;
    }
    if (c->status == PF_E_DT_UNDERFLOW) return sfail(S, PF_E_DT_UNDERFLOW, "step size fell below dt_min");
    if (c->status == PF_E_NONFINITE) return sfail(S, PF_E_NONFINITE, "non-finite error estimate");
    return PF_OK;
}

pf_status pf_slabs_unfrozen_fraction(pf_slabs* S, double* uwc, long long* n_ice, long long* n_water) {
    if (!S) return sfail(nullptr, PF_E_INVALID, "slabs is NULL");
    long long ni = 0, nw = 0;
    for (pf_grid* g : S->s) {
        long long a = 0, b = 0;
        pf_status st = pf_unfrozen_fraction(g, nullptr, nullptr, &a, &b, nullptr);
        if (st != PF_OK) return sfail(S, st, g->err);
        ni += a;
        nw += b;
    }
    if (n_ice) *n_ice = ni;
    if (n_water) *n_water = nw;
    if (uwc) *uwc = nw ? 1.0 - (double)ni / (double)nw : NAN;
    return PF_OK;
}

long long pf_slabs_halo_bytes(const pf_slabs* S) { return S ? S->halo_bytes : -1; }

}  // extern "C"
