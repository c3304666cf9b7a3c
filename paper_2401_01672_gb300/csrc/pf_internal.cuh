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

// Model constants, precomputed on the host in binary64 (Secs. 2.1-2.5).
struct Coefs {
    int n1, n2, n3;
    int dirichlet;      // PF_FACE_* bits
    int harmonic;       // face conductivity: harmonic mean
    int pad0;
    double inv_h2;      // 1/h^2
    double half_inv_h2; // 1/(2 h^2): arithmetic-mean face conductivity folded in
    double lam[3], rho[3], cap[3]; // liquid, ice, glass
    double latent;
    double xi2;         // xi^2
    double inv_axi2;    // 1/(alpha xi^2)
    double ksig;        // 1/2 xi b mu alpha      (SigmaP1-P)
    double kgrad;       // xi^2 mu alpha / (2h)   (GradP, central differences)
    double eps0, eps1, inv_de;
    double gamma, zeta;
    double theta_micro, theta_freeze, theta_thaw, t_freeze;
};

// Device-resident step control (one per grid).  All per-step scalars live
// here so that a captured CUDA graph can be replayed without host updates.
struct Ctrl {
    double t;          // time of the current state
    double dt;         // next step-size proposal
    double dt_step;    // size of the step being taken (shortened to land on target)
    double target;     // landing time when land != 0
    double tol, t_end, t_freeze, dt_min, dt_max;
    double last_err;
    unsigned long long err_bits;  // max of the error estimate over cells (bit pattern of a double >= 0)
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

template <typename T>
struct StageArgs {
    Coefs cf;
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
    const T* G;              // glass field
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

// Launch accounting (process-wide).
void count_launch(long long n = 1);

}  // namespace pfgb
