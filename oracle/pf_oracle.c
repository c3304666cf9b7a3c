/*
 * pf_oracle.c -- plain, slow FP64 CPU oracle of the phase-field freezing model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  The product
 * path never calls it and shares no code, header or constant with it.
 *
 * It follows Strachota, "Three-dimensional phase-field simulations of water
 * freezing and thawing at pore-scale" (arXiv 2401.01672):
 *   - glass field G of spheres and cap ............ Sec. 2.1 (G_balls, G formulas)
 *   - material blending ............................ Sec. 2.1, eq. (material-properties-blending-formula)
 *   - heat equation ................................ Sec. 2.2, eq. (heat-equation)
 *   - Allen-Cahn equation, water indicator ......... Sec. 2.2, eqs. (Allen-Cahn-equation), (water-indicator)
 *   - GradP and SigmaP1-P reaction terms, limiter .. Sec. 2.2, eqs. (reaction-term-GradP),
 *                                                    (reaction-term-SigmaP1-P), (Sigma-limiter)
 *   - boundary conditions .......................... Sec. 2.2, eqs. (BC-temperature-cap), (BC-temperature-wall), (BC-PF)
 *   - Temp model ................................... Sec. 2.3, eqs. (explicit-p-dependence-on-T),
 *                                                    (combined-heat-xfer-phase-transition)
 *   - micro-scale model (lambda = 0, L = 0) ........ Sec. 2.4
 *   - finite volumes + Runge-Kutta-Merson .......... Sec. 2.5
 *   - water / ice subdomains, UWC .................. Sec. 3.1 eqs. (water-occupied-subdomain), (frozen-subdomain);
 *                                                    Sec. 3.3 eq. (UWC-formula)
 *
 * Readings where the paper is silent (cited papers not available):
 *   - unknowns: theta = T - T* (K) and phi on cell centres x = (i+1/2)h, x fastest;
 *   - face conductivity = arithmetic mean of the two cell-blended values
 *     (harmonic mean selectable);
 *   - Dirichlet face: the boundary value sits on the face, half a cell from the
 *     centre: flux 2 lambda_i (theta_b - theta_i) / h^2;
 *   - zero normal flux of phi on every face, zero heat flux on non-Dirichlet faces;
 *   - |grad phi| by central differences with mirror ghosts;
 *   - rho c = (blended rho) * (blended c); the rho multiplying L dphi/dt is the blended rho;
 *   - Merson tableau and error estimate as published by Merson (1957);
 *     step control: accept iff E <= tol, dt <- dt min(5, 0.8 (tol/E)^(1/5)), capped by dt_max;
 *     a step never crosses t_freeze or t_end (it is shortened to land on them);
 *   - the Dirichlet value of a step is the one of the interval the step lies in
 *     (decided by the step's start time: t < t_freeze -> freeze value);
 *   - E = max over cells and integrated fields of |dt/30 (2k1 - 9k3 + 8k4 - k5)|.
 *
 * Built with -O2 -ffp-contract=off so each operation rounds as written.  With -fopenmp the loops
 * over cells are shared among threads (every cell is computed by the same arithmetic whatever the
 * thread; the error maximum does not depend on the order in which cells are visited; the UWC sums
 * stay serial and in a fixed order), so results are identical for any thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by the loops over cells: n > 0 sets the count; returns the count in use (1 when
 * built without OpenMP). */
int or_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

enum { OR_FULL = 0, OR_TEMP = 1, OR_MICRO = 2 };
enum { OR_SIGMAP1P = 0, OR_GRADP = 1 };
enum { LQ = 0, IC = 1, GL = 2 };

typedef struct {
    int n1, n2, n3;
    double h;
    int model;
    int reaction;
    double rho[3], c[3], lam[3]; /* liquid, ice, glass (Table 1) */
    double L, mu, alpha, xi, eps0, eps1, b, gamma, zeta;
    double theta_micro;
    double theta_freeze, theta_thaw, t_freeze;
    double dt_min, dt_max;
    int dirichlet; /* bit f set -> face f has a Dirichlet temperature; f = x-,x+,y-,y+,z-,z+ */
    int harmonic;
} or_model;

/* ---------------------------------------------------------------- geometry */

/* Sec. 2.1: G_balls(x) = max_i 1/2 (1 - tanh((|x - x_i| - r_i) / (2 xi_G))),
 * then G = max(G_balls, 1/2 (1 + tanh((x3 - x3cap)/(2 xi_G)))) when a cap is present.
 * Spheres are rows (x, y, z, r) in metres; every sphere is visited for every cell.
 * cells == NULL: all cells, G_out[n1*n2*n3]; else G_out[k] for linear cell index cells[k]. */
void or_glass(const or_model* m, const double* spheres, long long n_spheres, double xi_G,
              double x3_cap, int has_cap, const long long* cells, long long n_cells, double* G_out)
{
    long long N = (long long)m->n1 * m->n2 * m->n3;
    long long count = cells ? n_cells : N;
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < count; ++q) {
        long long id = cells ? cells[q] : q;
        long long i = id % m->n1;
        long long j = (id / m->n1) % m->n2;
        long long k = id / ((long long)m->n1 * m->n2);
        double x = (i + 0.5) * m->h, y = (j + 0.5) * m->h, z = (k + 0.5) * m->h;
        double G = 0.0;
        for (long long s = 0; s < n_spheres; ++s) {
            double dx = x - spheres[4 * s + 0];
            double dy = y - spheres[4 * s + 1];
            double dz = z - spheres[4 * s + 2];
            double dist = sqrt(dx * dx + dy * dy + dz * dz);
            double g = 0.5 * (1.0 - tanh((dist - spheres[4 * s + 3]) / (2.0 * xi_G)));
            if (g > G) G = g;
        }
        if (has_cap) {
            double g = 0.5 * (1.0 + tanh((z - x3_cap) / (2.0 * xi_G)));
            if (g > G) G = g;
        }
        G_out[q] = G;
    }
}

/* ------------------------------------------------------------ local terms */

/* eq. (material-properties-blending-formula): w = G w_G + (1 - G)[phi w_I + (1 - phi) w_L] */
static double blend(double G, double phi, const double w[3])
{
    return G * w[GL] + (1.0 - G) * (phi * w[IC] + (1.0 - phi) * w[LQ]);
}

/* eq. (water-indicator): I_W(G) = max(0, 1 - zeta G) */
static double water_indicator(double G, double zeta)
{
    double v = 1.0 - zeta * G;
    return v > 0.0 ? v : 0.0;
}

/* eq. (Sigma-limiter) */
static double sigma_limiter(double w, double e0, double e1)
{
    if (w <= e0) return 0.0;
    if (w >= e1) return 1.0;
    double d = e1 - e0;
    double a = w - e0;
    return 3.0 * (a * a) / (d * d) - 2.0 * (a * a * a) / (d * d * d);
}

/* eq. (explicit-p-dependence-on-T): phi = 1/2 I_W (1 - tanh(gamma (T - T*))), and its T-derivative */
static double temp_phi(double G, double theta, const or_model* m)
{
    return 0.5 * water_indicator(G, m->zeta) * (1.0 - tanh(m->gamma * theta));
}
static double temp_dphi(double G, double theta, const or_model* m)
{
    double th = tanh(m->gamma * theta);
    return -0.5 * water_indicator(G, m->zeta) * m->gamma * (1.0 - th * th);
}

void or_temp_phi(const or_model* m, const double* G, const double* theta, double* phi_out)
{
    long long N = (long long)m->n1 * m->n2 * m->n3;
    for (long long q = 0; q < N; ++q) phi_out[q] = temp_phi(G[q], theta[q], m);
}

/* Dirichlet value of the interval containing time t (eq. BC-temperature-cap). */
static double boundary_theta(const or_model* m, double t)
{
    return (t < m->t_freeze) ? m->theta_freeze : m->theta_thaw;
}

/* phi at a cell as seen by the heat equation's blends */
static double phase_at(const or_model* m, const double* G, const double* theta, const double* phi, long long id)
{
    if (m->model == OR_TEMP) return temp_phi(G[id], theta[id], m);
    return phi[id];
}

/* ------------------------------------------------------------------ RHS */

/*
 * Right-hand side of the semi-discrete system at the listed cells (all cells if cells == NULL).
 *   full  : dphi from eq. (Allen-Cahn-equation), dtheta from eq. (heat-equation)
 *   Temp  : dtheta from eq. (combined-heat-xfer-phase-transition); dphi = phi'(T) dtheta
 *   micro : theta = theta_micro constant, lambda = L = 0 -> dtheta = 0 (Sec. 2.4)
 * theta may be NULL for micro, phi may be NULL for Temp.  Outputs are indexed like the
 * grid when cells == NULL, else by list position.
 */
void or_rhs(const or_model* m, const double* G, double t, const double* theta, const double* phi,
            const long long* cells, long long n_cells, double* dtheta, double* dphi)
{
    const int n1 = m->n1, n2 = m->n2, n3 = m->n3;
    const long long N = (long long)n1 * n2 * n3;
    const long long count = cells ? n_cells : N;
    const double h = m->h, h2 = h * h;
    const double th_b = boundary_theta(m, t);
    const long long stride[3] = {1, n1, (long long)n1 * n2};
    const int dims[3] = {n1, n2, n3};

#pragma omp parallel for schedule(static)
    for (long long q = 0; q < count; ++q) {
        long long id = cells ? cells[q] : q;
        int idx[3];
        idx[0] = (int)(id % n1);
        idx[1] = (int)((id / n1) % n2);
        idx[2] = (int)(id / ((long long)n1 * n2));

        double Gi = G[id];
        double th_i = (m->model == OR_MICRO) ? m->theta_micro : theta[id];
        double ph_i = phase_at(m, G, theta, phi, id);

        /* heat flux divergence div(lambda grad T) by finite volumes */
        double div = 0.0;
        if (m->model != OR_MICRO) {
            double lam_i = blend(Gi, ph_i, m->lam);
            for (int d = 0; d < 3; ++d) {
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    int nb = idx[d] + sgn;
                    int face = 2 * d + (sgn > 0 ? 1 : 0);
                    if (nb >= 0 && nb < dims[d]) {
                        long long jd = id + sgn * stride[d];
                        double lam_j = blend(G[jd], phase_at(m, G, theta, phi, jd), m->lam);
                        double lam_f;
                        if (m->harmonic)
                            lam_f = (lam_i + lam_j > 0.0) ? 2.0 * lam_i * lam_j / (lam_i + lam_j) : 0.0;
                        else
                            lam_f = 0.5 * (lam_i + lam_j);
                        div += lam_f * (theta[jd] - th_i) / h2;
                    } else if (m->dirichlet & (1 << face)) {
                        div += 2.0 * lam_i * (th_b - th_i) / h2;
                    }
                    /* else: insulated wall, zero flux */
                }
            }
        }

        double dph = 0.0;
        if (m->model != OR_TEMP) {
            /* Laplacian of phi with zero normal flux on the boundary (eq. BC-PF) */
            double lap = 0.0;
            double grad2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                double lo = ph_i, hi = ph_i;
                if (idx[d] - 1 >= 0) lo = phi[id - stride[d]];
                if (idx[d] + 1 < dims[d]) hi = phi[id + stride[d]];
                lap += (lo - ph_i) / h2 + (hi - ph_i) / h2;
                double g = (hi - lo) / (2.0 * h);
                grad2 += g * g;
            }
            double under = -th_i; /* T* - T */
            double f;
            if (m->reaction == OR_GRADP) {
                /* eq. (reaction-term-GradP) */
                f = 2.0 * ph_i * (1.0 - ph_i) * (ph_i - 0.5) + m->xi * m->xi * m->mu * m->alpha * sqrt(grad2) * under;
            } else {
                /* eq. (reaction-term-SigmaP1-P) */
                double S = sigma_limiter(ph_i, m->eps0, m->eps1) * sigma_limiter(1.0 - ph_i, m->eps0, m->eps1);
                f = 2.0 * ph_i * (1.0 - ph_i) * (ph_i - 0.5 + 0.5 * m->xi * m->b * m->mu * m->alpha * S * under);
            }
            /* eq. (Allen-Cahn-equation): alpha xi^2 dphi/dt = I_W(G) [xi^2 lap phi + f] */
            dph = water_indicator(Gi, m->zeta) * (m->xi * m->xi * lap + f) / (m->alpha * m->xi * m->xi);
        }

        double dth = 0.0;
        if (m->model == OR_FULL) {
            /* eq. (heat-equation): rho c dT/dt = div(lambda grad T) + rho L dphi/dt */
            double rho = blend(Gi, ph_i, m->rho);
            double c = blend(Gi, ph_i, m->c);
            dth = (div + rho * m->L * dph) / (rho * c);
        } else if (m->model == OR_TEMP) {
            /* eq. (combined-heat-xfer-phase-transition): rho [c - L phi'(T)] dT/dt = div(lambda grad T) */
            double rho = blend(Gi, ph_i, m->rho);
            double c = blend(Gi, ph_i, m->c);
            double dp = temp_dphi(Gi, th_i, m);
            dth = div / (rho * (c - m->L * dp));
            dph = dp * dth;
        }
        if (dtheta) dtheta[q] = dth;
        if (dphi) dphi[q] = dph;
    }
}

/* ------------------------------------------------------- Runge-Kutta-Merson */

/* which fields are integrated: full {theta, phi}, Temp {theta}, micro {phi} */
static int has_theta(const or_model* m) { return m->model != OR_MICRO; }
static int has_phi(const or_model* m) { return m->model != OR_TEMP; }

/*
 * One Merson step of size dt from (t, y) (Sec. 2.5; Merson 1957 tableau):
 *   k1 = F(y)
 *   k2 = F(y + dt/3 k1)
 *   k3 = F(y + dt/6 k1 + dt/6 k2)
 *   k4 = F(y + dt/8 k1 + 3dt/8 k3)
 *   k5 = F(y + dt/2 k1 - 3dt/2 k3 + 2dt k4)
 *   y' = y + dt/6 (k1 + 4 k4 + k5)
 *   E  = max |dt/30 (2 k1 - 9 k3 + 8 k4 - k5)|
 * The boundary value of every stage is the one of the step's interval.
 * y_out may not alias y.  Returns E in *err.
 */
void or_rkm_step(const or_model* m, const double* G, double t, double dt,
                 const double* y_th, const double* y_ph, double* out_th, double* out_ph, double* err)
{
    const long long N = (long long)m->n1 * m->n2 * m->n3;
    const int ht = has_theta(m), hp = has_phi(m);
    double* k[6][2];
    for (int s = 1; s <= 5; ++s)
        for (int f = 0; f < 2; ++f) k[s][f] = (double*)calloc((size_t)N, sizeof(double));
    double* u_th = (double*)calloc((size_t)N, sizeof(double));
    double* u_ph = (double*)calloc((size_t)N, sizeof(double));
    const double* yt = ht ? y_th : NULL;
    const double* yp = hp ? y_ph : NULL;

    /* stage 1 */
    or_rhs(m, G, t, yt, yp, NULL, 0, k[1][0], k[1][1]);
    /* stage 2 */
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < N; ++q) {
        if (ht) u_th[q] = y_th[q] + dt / 3.0 * k[1][0][q];
        if (hp) u_ph[q] = y_ph[q] + dt / 3.0 * k[1][1][q];
    }
    or_rhs(m, G, t, ht ? u_th : NULL, hp ? u_ph : NULL, NULL, 0, k[2][0], k[2][1]);
    /* stage 3 */
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < N; ++q) {
        if (ht) u_th[q] = y_th[q] + dt / 6.0 * k[1][0][q] + dt / 6.0 * k[2][0][q];
        if (hp) u_ph[q] = y_ph[q] + dt / 6.0 * k[1][1][q] + dt / 6.0 * k[2][1][q];
    }
    or_rhs(m, G, t, ht ? u_th : NULL, hp ? u_ph : NULL, NULL, 0, k[3][0], k[3][1]);
    /* stage 4 */
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < N; ++q) {
        if (ht) u_th[q] = y_th[q] + dt / 8.0 * k[1][0][q] + 3.0 * dt / 8.0 * k[3][0][q];
        if (hp) u_ph[q] = y_ph[q] + dt / 8.0 * k[1][1][q] + 3.0 * dt / 8.0 * k[3][1][q];
    }
    or_rhs(m, G, t, ht ? u_th : NULL, hp ? u_ph : NULL, NULL, 0, k[4][0], k[4][1]);
    /* stage 5 */
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < N; ++q) {
        if (ht) u_th[q] = y_th[q] + dt / 2.0 * k[1][0][q] - 3.0 * dt / 2.0 * k[3][0][q] + 2.0 * dt * k[4][0][q];
        if (hp) u_ph[q] = y_ph[q] + dt / 2.0 * k[1][1][q] - 3.0 * dt / 2.0 * k[3][1][q] + 2.0 * dt * k[4][1][q];
    }
    or_rhs(m, G, t, ht ? u_th : NULL, hp ? u_ph : NULL, NULL, 0, k[5][0], k[5][1]);

    double E = 0.0;
#pragma omp parallel
    {
        double Et = 0.0; /* maximum over this thread's cells; once a NaN is seen it stays */
#pragma omp for schedule(static)
        for (long long q = 0; q < N; ++q) {
            for (int f = 0; f < 2; ++f) {
                if ((f == 0 && !ht) || (f == 1 && !hp)) continue;
                const double* y = f == 0 ? y_th : y_ph;
                double* o = f == 0 ? out_th : out_ph;
                o[q] = y[q] + dt / 6.0 * (k[1][f][q] + 4.0 * k[4][f][q] + k[5][f][q]);
                double e = fabs(dt / 30.0 * (2.0 * k[1][f][q] - 9.0 * k[3][f][q] + 8.0 * k[4][f][q] - k[5][f][q]));
                if (Et == Et && !(e <= Et)) Et = e;
            }
        }
#pragma omp critical
        {
            if (E == E && !(Et <= E)) E = Et;
        }
    }
    if (!ht && out_th && y_th) memcpy(out_th, y_th, (size_t)N * sizeof(double));
    if (!hp && out_ph && y_ph) memcpy(out_ph, y_ph, (size_t)N * sizeof(double));
    *err = E;

    for (int s = 1; s <= 5; ++s)
        for (int f = 0; f < 2; ++f) free(k[s][f]);
    free(u_th);
    free(u_ph);
}

/* Step-size proposal after a step of size dt with error E (reading of the adaptive Merson control). */
double or_controller(double E, double tol, double dt, double dt_max)
{
    double fac;
    if (E == 0.0) {
        fac = 5.0;
    } else {
        fac = 0.8 * pow(tol / E, 0.2);
        if (fac > 5.0) fac = 5.0;
    }
    double dn = dt * fac;
    if (dn > dt_max) dn = dt_max;
    return dn;
}

enum { OR_OK = 0, OR_E_DT_UNDERFLOW = -4, OR_E_NONFINITE = -5 };

/*
 * Integrate from *t to t_end.  fixed != 0: every step has size *dt (shortened only to land on
 * t_freeze / t_end) and is accepted.  Otherwise adaptive with tolerance tol.
 * Stops after max_steps attempts.  State is updated in place.  Per-attempt records
 * (t_start, dt, E, accepted) go to trace[4*a..] when trace != NULL (capacity max_steps).
 */
int or_run(const or_model* m, const double* G, double* theta, double* phi, double* t, double* dt,
           double t_end, double tol, long long max_steps, int fixed,
           long long* n_acc, long long* n_rej, double* last_err, double* trace)
{
    const long long N = (long long)m->n1 * m->n2 * m->n3;
    double* o_th = (double*)calloc((size_t)N, sizeof(double));
    double* o_ph = (double*)calloc((size_t)N, sizeof(double));
    int status = OR_OK;
    long long att = 0;
    *n_acc = 0;
    *n_rej = 0;
    while (*t < t_end && att < max_steps) {
        /* shorten the step so it lands on the next switching time */
        double target = t_end;
        if (*t < m->t_freeze && m->t_freeze < target) target = m->t_freeze;
        double h = *dt;
        int land = 0;
        if (*t + h >= target) {
            h = target - *t;
            land = 1;
        }
        double E;
        or_rkm_step(m, G, *t, h, theta, phi, o_th, o_ph, &E);
        int accept = fixed || (E <= tol);
        if (trace) {
            trace[4 * att + 0] = *t;
            trace[4 * att + 1] = h;
            trace[4 * att + 2] = E;
            trace[4 * att + 3] = accept;
        }
        ++att;
        *last_err = E;
        if (!(E <= 1.79e308) && !fixed) {
            status = OR_E_NONFINITE;
            break;
        }
        if (accept) {
            *t = land ? target : *t + h;
            if (has_theta(m)) memcpy(theta, o_th, (size_t)N * sizeof(double));
            if (has_phi(m)) memcpy(phi, o_ph, (size_t)N * sizeof(double));
            ++*n_acc;
        } else {
            ++*n_rej;
        }
        if (!fixed) {
            double dn = or_controller(E, tol, h, m->dt_max);
            if (dn < m->dt_min) {
                *dt = dn;
                status = OR_E_DT_UNDERFLOW;
                break;
            }
            *dt = dn;
        }
    }
    free(o_th);
    free(o_ph);
    return status;
}

/* ---------------------------------------------------------------- observables */

/*
 * eqs. (water-occupied-subdomain), (frozen-subdomain), (UWC-formula) over the half-open box
 * region = {i0, i1, j0, j1, k0, k1} (NULL = whole grid):
 *   n_water = #{G < 1/2}, n_ice = #{phi > 1/2 and G < 1/2},
 *   smooth = (sum (1 - G) phi, sum (1 - G)).
 */
void or_uwc(const or_model* m, const double* G, const double* phi, const int* region,
            long long* n_water, long long* n_ice, double* smooth_num, double* smooth_den)
{
    int r[6] = {0, m->n1, 0, m->n2, 0, m->n3};
    if (region) memcpy(r, region, sizeof(r));
    long long nw = 0, ni = 0;
    double sn = 0.0, sd = 0.0;
    for (int k = r[4]; k < r[5]; ++k)
        for (int j = r[2]; j < r[3]; ++j)
            for (int i = r[0]; i < r[1]; ++i) {
                long long id = i + (long long)m->n1 * (j + (long long)m->n2 * k);
                if (G[id] < 0.5) {
                    ++nw;
                    if (phi[id] > 0.5) ++ni;
                }
                sn += (1.0 - G[id]) * phi[id];
                sd += (1.0 - G[id]);
            }
    *n_water = nw;
    *n_ice = ni;
    *smooth_num = sn;
    *smooth_den = sd;
}
