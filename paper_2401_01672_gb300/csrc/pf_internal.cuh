// Internal types of the GB300 phase-field library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace pfgb {

enum { M_FULL = 0, M_TEMP = 1, M_MICRO = 2 };
enum { R_SIGMA = 0, R_GRADP = 1 };

// Tile of a stage kernel: one warp spans 32 cells along x, BY warps span y,
// each thread marches along z over a chunk of ZC planes.
constexpr int TX = 32;

// per-cell coefficient arrays of the binary64 full model (see StageArgs::statics)
constexpr int NSTATIC = 10;

// Model constants in the form the stage kernels use them, filled on the host
// (binary64 arithmetic) for each field type, so kernels convert nothing.
//   lambda = lamL + G dLG + (1 - G) phi dLI, scaled by 1/(2 h^2)  (eq. material-properties-blending-formula)
//   rho, c : same blend, unscaled
//   2 I_W/(alpha xi^2) = max(0, wa + wb G)                         (eqs. water-indicator, Allen-Cahn-equation)
template <typename T>
struct CoefT {
    T lamL, dLG, dLI;
    T rhoL, dRG, dRI;
    T capL, dCG, dCI;
    T latent;
    T wa, wb;
    T g_pore;    // 1/(2 zeta): cells with G below it have I_W > 1/2 (pore bulk, used by the equilibrium count)
    T wa_half;   // wa / 2: the same test on W = 2 I_W / (alpha xi^2)
    T klap;      // xi^2 / (2 h^2)
    T ksig;      // xi b mu alpha / 2                (SigmaP1-P)
    T kgrad;     // xi^2 mu alpha / (4 h)            (GradP, central differences)
    T eps0, eps1, inv_de;
    T gamma, zeta;
    T theta_micro;
};

// Grid-wide integer constants.
struct Coefs {
    int n1, n2, n3;
    int dirichlet;      // PF_FACE_* bits
    int harmonic;       // face conductivity: harmonic mean
    int zlo, zhi;       // planes the z neighbours are clamped to: 0 and n3 - 1 (mirror ghosts at both ends);
                        // -1 / n3 where a z-slab has a ghost plane filled by its neighbour
    int pad0;
    double theta_freeze, theta_thaw, t_freeze;
};

// Merson stage coefficients of the step being taken (dt = dt_step):
// [0] dt/3 [1] dt/6 [2] dt/8 [3] 3dt/8 [4] dt/2 [5] 3dt/2 [6] 2dt [7] dt/30 [8] 5dt/24 [9] 15dt/8
constexpr int NSC = 10;

// Device-resident step control (one per grid).  All per-step scalars live
// here so that a captured CUDA graph can be replayed without host updates.
struct Ctrl {
    double t;          // time of the current state
    double dt;         // next step-size proposal
    double dt_step;    // size of the step being taken (shortened to land on target)
    double target;     // landing time when land != 0
    double tol, t_end, t_freeze, dt_min, dt_max;
    double theta_freeze, theta_thaw;
    double last_err;
    double theta_b;    // Dirichlet value of the step being taken
    double sc[NSC];    // stage coefficients, binary64
    float scf[NSC];    // stage coefficients, binary32
    float theta_bf;
    int pad1;
    unsigned long long err_bits;  // max of the error estimate over cells (bit pattern of a double >= 0)
    unsigned long long ice_count; // stage 1: #{phi > 1/2 and G < 1/(2 zeta)} of the current state (pore bulk)
    unsigned long long pore_count; // stage 1: #{G < 1/(2 zeta)} (pore-bulk cells)
    unsigned long long rate_bits;  // stage 1: max |dphi/dt| over the pore-bulk cells (bit pattern of a double)
    double eq_rate;               // equilibrium also needs that maximum <= eq_rate (0 = no residual test)
    double last_rate;             // the maximum of the last attempt
    long long prev_count;         // ice count when it last changed by more than the tolerance (-1: none yet)
    double eq_rel_tol;            // tolerated change of the ice count, relative to the pore-bulk cells
    double last_change_t;         // time of that change
    double eq_window;  // equilibrium: ice count unchanged for this long (0 = no test)
    double t_eq;       // time at which the equilibrium test held
    int equilibrium;   // the equilibrium test stopped the run
    int pad2;
    long long n_acc, n_rej, max_attempts;
    int cur;           // state buffer holding y
    int land;
    int done;
    int status;
    int fixed;         // accept every attempt, keep dt
    int single;        // one attempt: no landing, no termination test
    int accepted;
    int pad;
};

// Stage coefficients and the boundary value for the step (t, dt_step): the
// Dirichlet value of the interval the step lies in (t < t_freeze -> freeze value).
__host__ __device__ inline void prepare_step(Ctrl* c) {
    const double dt = c->dt_step;
    const double v[NSC] = {dt / 3.0, dt / 6.0, dt / 8.0, 3.0 * dt / 8.0, dt / 2.0,
                           1.5 * dt, 2.0 * dt, dt / 30.0, 5.0 * dt / 24.0, 15.0 * dt / 8.0};
    for (int q = 0; q < NSC; ++q) {
        c->sc[q] = v[q];
        c->scf[q] = (float)v[q];
    }
    c->theta_b = (c->t < c->t_freeze) ? c->theta_freeze : c->theta_thaw;
    c->theta_bf = (float)c->theta_b;
}

// Work list of the batched persistent stage kernels, rebuilt on the device after every step:
// active instance s covers tiles [tile_start[s], tile_start[s+1]) of the flattened tile list.
constexpr int BATCH_MAX = 256;
struct BatchPlan {
    int ntiles;
    int nactive;
    int iter;
    int max_iter;
    int inst[BATCH_MAX];
    int tile_start[BATCH_MAX + 1];
};

template <typename T>
struct StageArgs {
    Coefs cf;
    CoefT<T> k;
    Ctrl* ctrl;
    const double* y_th[2];   // state double buffer (binary64 in both precisions)
    const double* y_ph[2];
    double* yo_th[2];        // same buffers, writable view
    double* yo_ph[2];
    T* ua_th; T* ua_ph;      // stage-input buffers
    T* ub_th; T* ub_ph;
    T* k1_th; T* k1_ph;
    T* k3_th; T* k3_ph;
    T* k4_th; T* k4_ph;
    T* y32_th[2];            // binary32 form of the full model: binary32 copies of the state buffers (set with
    T* y32_ph[2];            // the state; stage 5 writes that of the candidate state beside it)
    const T* G;              // glass field
    // full model, binary64: per-cell coefficients precomputed from G (SoA, NSTATIC arrays of n cells):
    // [0] A_lam [1] B_lam (lambda' = A + B phi)  [2] W = 2 I_W/(alpha xi^2) before the max
    // [3..5] C0, C1, C2 (rho c = C0 + phi (C1 + phi C2))  [6..7] D0, D1 (rho L = D0 + D1 phi)
    // [8..9] 1/(rho c) at phi = 0 and at phi = 1
    const double* statics;
    long long ncell;
    // plain right-hand side (stage 0)
    const T* in_th; const T* in_ph;
    T* out_th; T* out_ph;
    double t_rhs;
    int zc;                  // planes per block along z
};

// Launch one stage (0 = plain RHS, 1..5 = Merson stages) of the given model.
// Returns the CUDA error of the launch.
cudaError_t launch_stage_f64(int model, int rx, int stage, const StageArgs<double>& a, int by,
                             cudaStream_t s);
cudaError_t launch_stage_f32(int model, int rx, int stage, const StageArgs<float>& a, int by,
                             cudaStream_t s);

cudaError_t launch_batch_stage_f64(int model, int rx, int stage, const StageArgs<double>* args,
                                   const BatchPlan* plan, const int4* tilegrid, int by, int blocks,
                                   cudaStream_t s);
cudaError_t launch_batch_stage_f32(int model, int rx, int stage, const StageArgs<float>* args,
                                   const BatchPlan* plan, const int4* tilegrid, int by, int blocks,
                                   cudaStream_t s);

// Launch accounting (process-wide).
void count_launch(long long n = 1);

}  // namespace pfgb
