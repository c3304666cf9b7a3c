/*
 * pf.h -- C ABI of the GB300 phase-field freezing/thawing solver.
 *
 * Method: Strachota, "Three-dimensional phase-field simulations of water
 * freezing and thawing at pore-scale" (arXiv 2401.01672).  The library
 * integrates, on one NVIDIA GB300 (sm_103a), the semi-discrete finite-volume
 * system of Sec. 2.5 with the Runge-Kutta-Merson method:
 *   full model  : heat equation (eq. heat-equation) + Allen-Cahn (eq. Allen-Cahn-equation)
 *                 with the GradP (eq. reaction-term-GradP) or SigmaP1-P
 *                 (eq. reaction-term-SigmaP1-P) reaction term, Sec. 2.2;
 *   Temp model  : eqs. (explicit-p-dependence-on-T), (combined-heat-xfer-phase-transition), Sec. 2.3;
 *   micro model : constant supercooling, lambda = 0, L = 0 (Sec. 2.4).
 *
 * Conventions shared by every call
 *   - Every call returns pf_status; nothing is thrown across the ABI.  On an
 *     error pf_last_error(grid) returns a message (pf_last_error(NULL) for
 *     failures of pf_create_grid).
 *   - Grid layout: n1 x n2 x n3 cells of edge h (metres), cell (i,j,k) at
 *     linear index i + n1*(j + n2*k) (x fastest), centre ((i+1/2)h, (j+1/2)h, (k+1/2)h).
 *   - Temperatures are offsets theta = T - T* in kelvin (T* = bulk melting point).
 *   - Host arrays are copied; the caller keeps ownership.  Device arrays
 *     passed in are borrowed for the duration of the call.
 *   - All GPU work is enqueued on the stream given at creation; calls that
 *     return host data synchronise that stream.
 *   - A grid may be used by one host thread at a time.
 *   - Device buffers are owned by the grid (allocated at creation, freed by
 *     pf_destroy_grid).  Out of memory -> PF_E_OOM, nothing leaks.
 */
#ifndef PF_H
#define PF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_grid pf_grid;

typedef enum {
    PF_OK = 0,
    PF_E_INVALID = -1,      /* bad argument (NULL, size, enum, inconsistent parameters) */
    PF_E_CUDA = -2,         /* a CUDA runtime call failed; message has the CUDA error */
    PF_E_OOM = -3,          /* device or pinned-host allocation failed */
    PF_E_DT_UNDERFLOW = -4, /* the step-size controller proposed dt < dt_min */
    PF_E_NONFINITE = -5,    /* the error estimate was NaN or Inf: the state is left at the last accepted step */
    PF_E_RANGE = -6,        /* a value is outside its admissible range */
    PF_E_TIMEOUT = -7,      /* a bounded device-side wait ran out (batched persistent runs) */
    PF_E_STATE = -8         /* call not valid in the grid's current state (e.g. no geometry) */
} pf_status;

typedef enum { PF_MODEL_FULL = 0, PF_MODEL_TEMP = 1, PF_MODEL_MICRO = 2 } pf_model;      /* Secs. 2.2-2.4 */
typedef enum { PF_REACT_SIGMAP1P = 0, PF_REACT_GRADP = 1 } pf_reaction;                 /* Sec. 2.2 */
/* PF_PREC_FP64: every field, stage buffer and operation in IEEE binary64.
 * PF_PREC_FP32_FIELDS: stage inputs u_s, stage slopes k_s and the glass field in
 * binary32 (right-hand side evaluated in binary32); the state y, its update
 * y + dt/6 (k1 + 4 k4 + k5), the error-norm reduction, the step control and the
 * unfrozen-water integrals stay binary64. */
typedef enum { PF_PREC_FP64 = 0, PF_PREC_FP32_FIELDS = 1 } pf_precision;

/* Dirichlet face bits (eq. BC-temperature-cap); faces without a bit are insulated
 * (eq. BC-temperature-wall).  phi has zero normal flux on every face (eq. BC-PF). */
enum { PF_FACE_XM = 1, PF_FACE_XP = 2, PF_FACE_YM = 4, PF_FACE_YP = 8, PF_FACE_ZM = 16, PF_FACE_ZP = 32 };

/* Model parameters, SI units (Table 1, Table 2).  Index 0 = liquid water (L), 1 = ice (I), 2 = glass (G). */
typedef struct pf_params {
    double rho[3];        /* density [kg m^-3] */
    double c[3];          /* specific heat capacity [J kg^-1 K^-1] */
    double lambda[3];     /* heat conductivity [W m^-1 K^-1] */
    double latent;        /* specific latent heat L [J kg^-1] */
    double mu;            /* interface mobility [m s^-1 K^-1] */
    double alpha;         /* attachment-kinetics coefficient [s m^-2] (eq. attachment-kinetics-coeff) */
    double xi;            /* ice-liquid diffuse-interface thickness [m] */
    double xi_G;          /* glass-water diffuse-interface thickness [m] (Sec. 2.1) */
    double eps0, eps1;    /* Sigma-limiter corners (eq. Sigma-limiter), 0 <= eps0 < eps1 <= 1/2 */
    double b;             /* b(eps0, eps1) of eq. (reaction-term-SigmaP1-P); the paper uses 1 */
    double gamma;         /* Temp model transition rate [K^-1] (eq. explicit-p-dependence-on-T) */
    double zeta;          /* water indicator parameter, >= 1 (eq. water-indicator) */
    double theta_micro;   /* micro model: constant T - T* (= -supercooling) [K] */
    double theta_freeze;  /* Dirichlet value T_freeze - T* for t < t_freeze [K] */
    double theta_thaw;    /* Dirichlet value T_thaw - T* for t >= t_freeze [K] */
    double t_freeze;      /* switching time [s]; +inf = never */
    double dt_min;        /* adaptive control fails with PF_E_DT_UNDERFLOW below this [s] */
    double dt_max;        /* proposals are capped here [s]; +inf = no cap */
    int dirichlet_faces;  /* PF_FACE_* bit mask */
    int harmonic_mean;    /* face conductivity: 0 = arithmetic mean of the two cells, 1 = harmonic mean */
} pf_params;

/* Statistics of one pf_run_to / pf_run_fixed call. */
typedef struct pf_run_stats {
    long long n_accepted;   /* accepted steps in this call */
    long long n_rejected;   /* rejected attempts in this call */
    double t;               /* time reached */
    double dt;              /* next step-size proposal */
    double last_err;        /* error estimate E of the last attempt */
    long long launches;     /* GPU kernels issued by this call (early-exiting ones included) */
} pf_run_stats;

/* Create a grid and allocate its device buffers.
 * n1, n2, n3 >= 1 with n1 n2 (n3 + 2) < 2^31 (cells are indexed with 32-bit integers); h > 0 [m]; model/reaction/precision from the enums above; p copied;
 * stream: a cudaStream_t (NULL = legacy default stream).  Geometry defaults to G = 0
 * (all water), state to theta = 0, phi = 0, t = 0, dt = dt_max (or 1e-3 s when dt_max is inf).
 * Sec. 2.5: uniform N1 x N2 x N3 finite-volume mesh. */
pf_status pf_create_grid(int n1, int n2, int n3, double h, int model, int reaction, int precision,
                         const pf_params* p, void* stream, pf_grid** out);

/* Free every buffer of the grid (synchronises its stream).  NULL is a no-op. */
pf_status pf_destroy_grid(pf_grid* g);

/* Glass field G from spheres (Sec. 2.1, G_balls and the cap formula), computed on the GPU.
 * spheres: host array of n rows (x, y, z, r) in metres (n >= 0, radii > 0);
 * x3_cap: elevation of the bottom of the glass cap in metres, NaN = no cap.
 * Terms below 1e-17 (beyond r + 40 xi_G from a sphere's centre) are skipped. */
pf_status pf_set_geometry(pf_grid* g, const double* spheres, long long n, double x3_cap);

/* Upload / download the glass field G directly (host arrays of n1*n2*n3 values in [0, 1]). */
pf_status pf_set_glass(pf_grid* g, const double* G);
pf_status pf_get_glass(pf_grid* g, double* G);

/* Set the state (host arrays of n1*n2*n3 doubles), the time t and the next step size dt > 0.
 * theta is ignored (may be NULL) for the micro model; phi is ignored (may be NULL) for Temp. */
pf_status pf_set_state(pf_grid* g, const double* theta, const double* phi, double t, double dt);

/* Copy the state to host arrays (either may be NULL).  For Temp, phi = phi(theta) of
 * eq. (explicit-p-dependence-on-T); for micro, theta = theta_micro everywhere.  t, dt may be NULL. */
pf_status pf_get_state(pf_grid* g, double* theta, double* phi, double* t, double* dt);

/* Right-hand side F(t, y) of the semi-discrete system (Secs. 2.2-2.5) on caller-owned DEVICE arrays of
 * n1*n2*n3 elements in the grid's field type (double for PF_PREC_FP64, float for PF_PREC_FP32_FIELDS).
 * t selects the Dirichlet value (t < t_freeze -> theta_freeze).  theta_in may be NULL (micro),
 * phi_in may be NULL (Temp); dtheta_out / dphi_out may be NULL to skip.  For Temp, dphi = phi'(T) dtheta;
 * for micro, dtheta = 0.  Inputs and outputs must not overlap.  Enqueued on the grid's stream. */
pf_status pf_rhs(pf_grid* g, double t, const void* theta_in, const void* phi_in, void* dtheta_out,
                 void* dphi_out);

/* One Runge-Kutta-Merson attempt of size *dt_inout from the current state (Sec. 2.5):
 * k1..k5 by the Merson tableau, y' = y + dt/6 (k1 + 4 k4 + k5), E = max |dt/30 (2k1 - 9k3 + 8k4 - k5)|
 * over cells and integrated fields.  Accepted iff force_accept or E <= tol; an accepted attempt
 * replaces the state and advances t.  On return *dt_inout holds the controller's proposal
 * dt * min(5, 0.8 (tol/E)^(1/5)) capped at dt_max (the step is not shortened to t_freeze here).
 * accepted / err may be NULL.  Synchronises. */
pf_status pf_rkm_step(pf_grid* g, double* dt_inout, double tol, int force_accept, int* accepted, double* err);

/* Adaptive integration from the current time to t_end with tolerance tol > 0, at most max_steps
 * attempts.  Steps are shortened to land exactly on t_freeze and t_end.  The step loop runs on the
 * device (CUDA graph replays, no host round trip per step).  stats may be NULL.
 * PF_E_DT_UNDERFLOW / PF_E_NONFINITE stop the run with the state at the last accepted step. */
pf_status pf_run_to(pf_grid* g, double t_end, double tol, long long max_steps, pf_run_stats* stats);

/* n_steps steps of size dt (each shortened only to land on t_freeze), every one accepted. */
pf_status pf_run_fixed(pf_grid* g, long long n_steps, double dt, pf_run_stats* stats);

/* Unfrozen water (Sec. 3.1 eqs. water-occupied-subdomain, frozen-subdomain; Sec. 3.3 eq. UWC-formula)
 * over the half-open cell box region = {i0, i1, j0, j1, k0, k1} (NULL = whole grid):
 *   n_water = #{G < 1/2}, n_ice = #{phi > 1/2 and G < 1/2}, uwc = 1 - n_ice / n_water (NaN if no water),
 *   smooth = 1 - sum (1-G) phi / sum (1-G) (binary64 sums in a fixed order).
 * Any output pointer may be NULL.  Synchronises. */
pf_status pf_unfrozen_fraction(pf_grid* g, const int* region, double* uwc, long long* n_ice,
                               long long* n_water, double* smooth);

/* Largest |dphi/dt| (binary64) over the grid at the current state, for the equilibrium test
 * 4 xi max|dphi/dt| <= tol_v (speed of a tanh front, Sec. 2.2).  Synchronises. */
pf_status pf_max_phase_rate(pf_grid* g, double* max_rate);

/* Timing aid: n_attempts forced (accepted) Merson steps of the current dt, launched one kernel at a
 * time with CUDA events around each launch on the grid's stream.  stage_ms[0..4] = mean duration of
 * stages 1..5, stage_ms[5] = mean duration of the step-control kernel, in milliseconds.  The state
 * advances by n_attempts steps.  Synchronises. */
pf_status pf_profile_stages(pf_grid* g, int n_attempts, double* stage_ms);

/* Tile shape of the stage kernels: blocks of 32 x by threads (by = 4, 8 or 16) marching along z over
 * zc >= 1 planes.  Any shape gives the same results; only speed changes.  Default 8 x 32. */
pf_status pf_set_tiles(pf_grid* g, int by, int zc);
pf_status pf_get_tiles(pf_grid* g, int* by, int* zc);

/* Tile autotuner: times the five stage kernels of one Merson attempt for by in {4, 8, 16} x zc in
 * {2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 64} on the grid itself and keeps the fastest.  The step controller is not run, so the
 * state, time, step size and counters are unchanged (stage 5 writes only the spare state buffer).  cache_path (NULL = none) is a text file of
 * lines "n1xn2xn3/model/reaction/precision by zc ms"; a cached shape is reused without timing and new
 * results are appended.  Outputs may be NULL. */
pf_status pf_autotune(pf_grid* g, const char* cache_path, int* by, int* zc, double* ms);

/* ---- Batched persistent runs (independent instances, each with its own adaptive step).
 * Equilibrium test (Sec. 3.3: the unfrozen water content no longer changes): stage 1 counts the ice
 * cells of the pore bulk, #{phi > 1/2 and I_W(G) > 1/2}, of the current state and takes the largest
 * |dphi/dt| over those pore-bulk cells; an instance is in equilibrium at the first state whose count has
 * stayed within eq_rel_tol x (pore-bulk cells) of a reference value for eq_window seconds
 * (eq_rel_tol = 0: no change at all) and, when eq_rate is given and eq_rate[i] > 0, whose largest
 * |dphi/dt| is at most eq_rate[i] (a residual test: 4 xi |dphi/dt| is the speed of a tanh interface,
 * Sec. 2.2, so eq_rate = v / (4 xi) bounds the speed of every pore interface by v).  (The thin glass
 * layer with I_W -> 0 keeps relaxing on the slow time scale alpha xi^2 / I_W without moving any pore
 * interface; it is left out of the test but not out of pf_unfrozen_fraction.)
 * A batch takes ownership of n grids (1 <= n <= 256) that share model, reaction and precision but may
 * differ in size, parameters, geometry and state; pf_batch_destroy destroys them.  All work goes to
 * the first grid's stream.  pf_batch_run_to advances every instance to its own t_end[i] (or until the
 * equilibrium test holds, when eq_window is not NULL and eq_window[i] > 0, or until max_steps attempts)
 * in ONE launch of a CUDA graph whose WHILE node repeats, on the device, five
 * batched persistent stage kernels (a fixed grid of blocks walking the tiles of all active instances),
 * the per-instance step control and the rebuild of the active-tile list; the loop stops when no
 * instance is active (at most max_steps + 1 iterations).  Per-instance results in res[n] (may be NULL).
 * Use pf_batch_grid to read an instance's state afterwards. */
typedef struct pf_batch pf_batch;
typedef struct pf_batch_result {
    pf_run_stats stats;
    double t_eq;       /* time at which the equilibrium test held (NaN if it did not) */
    double rate;       /* largest |dphi/dt| over the pore-bulk cells at the last attempt */
    int equilibrium;   /* 1 if the run stopped on the equilibrium test */
    int status;        /* PF_OK, PF_E_DT_UNDERFLOW or PF_E_NONFINITE for this instance */
} pf_batch_result;
pf_status pf_batch_create(int n, pf_grid* const* grids, pf_batch** out);
pf_status pf_batch_destroy(pf_batch* b);
pf_grid* pf_batch_grid(pf_batch* b, int i);
/* One block height for all instances (minimising the summed best times), then the best zc per instance. */
pf_status pf_batch_autotune(pf_batch* b, const char* cache_path);
pf_status pf_batch_run_to(pf_batch* b, const double* t_end, const double* eq_window, double eq_rel_tol,
                          const double* eq_rate, double tol, long long max_steps, pf_batch_result* res);
/* Device-side loop iterations of the last pf_batch_run_to (steps of the slowest instance + 1). */
long long pf_batch_iterations(const pf_batch* b);
const char* pf_batch_last_error(const pf_batch* b);

/* ---- z-slab multi-domain mode (Sec. 2.5: the domain cut along x3 into slabs; the planes next to a cut
 * are exchanged between neighbour slabs before every stage that reads them, and the step control uses
 * the error maximum over all slabs).  Here all slabs live in one process on one GPU: each slab is a grid
 * with a ghost plane at every cut, the exchange is a copy kernel after each stage (and after setting the
 * state), and the slabs share one device-side control block, so the error maximum and the pore counts
 * accumulate over all slabs and one step controller decides.  Results are bit-identical to the
 * single-domain grid of the same size: every cell sees the same neighbour values and arithmetic.
 *   nslabs : 1 <= nslabs <= min(n3, 1024);
 *   planes : nslabs + 1 increasing plane indices from 0 to n3 (slab q holds planes [planes[q],
 *            planes[q+1])), or NULL for an even split;
 *   other arguments as pf_create_grid; Dirichlet z faces apply only at the two ends of the domain.
 * Host arrays of set_state / get_state hold the whole n1 x n2 x n3 grid.  pf_slabs_grid returns slab q's
 * grid (owned by the group; use it only for reads such as pf_get_glass).  pf_slabs_halo_bytes: bytes the
 * exchanges of the last pf_slabs_run_to moved.  Errors as for the single-grid calls; messages from
 * pf_slabs_last_error. */
typedef struct pf_slabs pf_slabs;
pf_status pf_slabs_create(int n1, int n2, int n3, double h, int model, int reaction, int precision,
                          const pf_params* p, int nslabs, const int* planes, void* stream, pf_slabs** out);
pf_status pf_slabs_destroy(pf_slabs* s);
pf_grid* pf_slabs_grid(pf_slabs* s, int q);
pf_status pf_slabs_set_geometry(pf_slabs* s, const double* spheres, long long n, double x3_cap);
pf_status pf_slabs_set_tiles(pf_slabs* s, int by, int zc);
pf_status pf_slabs_set_state(pf_slabs* s, const double* theta, const double* phi, double t, double dt);
pf_status pf_slabs_get_state(pf_slabs* s, double* theta, double* phi, double* t, double* dt);
pf_status pf_slabs_run_to(pf_slabs* s, double t_end, double tol, long long max_steps, pf_run_stats* stats);
pf_status pf_slabs_unfrozen_fraction(pf_slabs* s, double* uwc, long long* n_ice, long long* n_water);
long long pf_slabs_halo_bytes(const pf_slabs* s);
const char* pf_slabs_last_error(const pf_slabs* s);

/* Throughput probes of the current device: binary64 and binary32 FMA rates (TFLOP/s, FMA = 2 flops,
 * 8 independent chains per thread, 8 blocks of 256 threads per SM) and device-memory copy bandwidth
 * (GB/s, read + write bytes of a 2 x 2 GiB copy, best of 5).  Any pointer may be NULL to skip a probe.
 * They give the roofline denominators of the stage kernels.  Allocates and frees its own buffers. */
pf_status pf_measure_peaks(double* fp64_tflops, double* fp32_tflops, double* copy_gbs);

/* Unfrozen-water counts that allocate nothing (no counterpart in the paper; a service for callers).
 *
 * Some callers cannot call cudaMalloc: a plug-in inside a host application that owns all device
 * memory through its own pool, a control loop that cannot afford the implicit synchronisation of an
 * allocation, or a process with a fixed GPU memory budget.  This entry point computes what
 * pf_unfrozen_fraction computes, on caller-owned device arrays, without creating a grid:
 *   G, phi : DEVICE arrays of n1*n2*n3 binary64 values (x fastest), borrowed for the call;
 *   region : host array {i0, i1, j0, j1, k0, k1} (half-open box) or NULL for the whole grid;
 *   stream : cudaStream_t to enqueue on (NULL = legacy default stream); the call synchronises it;
 *   outputs: host pointers, any may be NULL (same meaning as in pf_unfrozen_fraction).
 * Scratch: a file-scope __device__ array of PF_NOALLOC_MAX_PARTIALS + 1 slots of 32 bytes (about
 * 512 KiB) that every GPU loading the library holds until the process exits.  Each block of the
 * reduction covers 16384 cells, so a region may hold at most PF_NOALLOC_MAX_PARTIALS * 16384 =
 * 2^28 cells; larger regions return PF_E_RANGE before any launch.  Bad sizes or regions, and G or phi
 * that is not device memory of the current device (checked with cudaPointerGetAttributes), return
 * PF_E_INVALID; CUDA failures PF_E_CUDA.  The arrays' lengths cannot be checked here: each must hold
 * n1*n2*n3 values.  No cudaMalloc, cudaFree or allocating library call is
 * made.  The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All calls share the array
 * and every slot a call reads is written earlier in the same call; calls that overlap on the GPU
 * (other streams, other host threads) race on it. */
#define PF_NOALLOC_MAX_PARTIALS 16384
pf_status pf_unfrozen_fraction_noalloc(const double* G, const double* phi, int n1, int n2, int n3,
                                       const int* region, void* stream, double* uwc, long long* n_ice,
                                       long long* n_water, double* smooth);

/* Message of the last failed call on g (or of the last failed pf_create_grid when g is NULL). */
const char* pf_last_error(const pf_grid* g);

/* Total GPU kernels this library has enqueued in the process (for launch accounting). */
long long pf_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
