// Stage kernels of the Runge-Kutta-Merson integration of the semi-discrete
// phase-field system (Strachota, arXiv 2401.01672, Secs. 2.2-2.5).
//
// One kernel evaluates the right-hand side F at every cell of its tile and
// fuses the stage combination of the Merson tableau into the same pass:
//   stage 1: k1 = F(y),  u2 = y + dt/3 k1
//   stage 2: k2 = F(u2), u3 = y + dt/6 (k1 + k2)
//   stage 3: k3 = F(u3), u4 = y + dt/8 k1 + 3dt/8 k3
//   stage 4: k4 = F(u4), u5 = y + dt/2 k1 - 3dt/2 k3 + 2dt k4
//   stage 5: k5 = F(u5), y' = y + dt/6 (k1 + 4k4 + k5), E = max |dt/30 (2k1 - 9k3 + 8k4 - k5)|
// k2 and k5 are never stored.  Stage 0 is the plain right-hand side.
//
// Tiling: a block of 32 x BY threads owns a 32 x BY column of cells and
// marches along z over ZC planes.  Plane k (with a one-cell lateral halo)
// sits in shared memory together with the blended conductivity of every
// cell, so each cell's lambda is evaluated once per plane visit; the z
// neighbours of a thread's own column stay in registers.  Cells outside
// the grid are replaced by the nearest boundary cell (mirror ghost), which
// makes the interior formula give zero flux on every face; Dirichlet faces
// add their half-cell flux separately.
//
// Binary32 form (T = float): stage inputs chain from one stage input to the
// next (u3 = u2 + dt/6 (k2 - k1), u4 = u2 - 5dt/24 k1 + 3dt/8 k3,
// u5 = u4 + 3dt/8 k1 - 15dt/8 k3 + 2dt k4 -- algebraically the tableau rows)
// so that only stages 1 and 5 touch the binary64 state; the state update
// y' = y + (dt/6 (k1 + 4k4 + k5)) adds a binary32 increment to binary64 y.
#pragma once
#include "pf_internal.cuh"
#include <cfloat>
#include <type_traits>

namespace pfgb {

__device__ __forceinline__ double dtanh(double x) { return tanh(x); }
__device__ __forceinline__ float dtanh(float x) { return tanhf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }

// eq. (Sigma-limiter)
template <typename T>
__device__ __forceinline__ T sigma_lim(T w, T e0, T e1, T inv_de) {
    if (w <= e0) return T(0);
    if (w >= e1) return T(1);
    T s = (w - e0) * inv_de;
    return s * s * (T(3) - T(2) * s);
}

// eq. (material-properties-blending-formula)
template <typename T>
__device__ __forceinline__ T blend(T G, T ph, T wL, T wI, T wG) {
    return G * wG + (T(1) - G) * (ph * wI + (T(1) - ph) * wL);
}

// eq. (water-indicator)
template <typename T>
__device__ __forceinline__ T water_ind(T G, T zeta) {
    T v = T(1) - zeta * G;
    return v > T(0) ? v : T(0);
}

template <typename T>
struct CoefT {
    T inv_h2, half_inv_h2;
    T lamL, lamI, lamG, rhoL, rhoI, rhoG, cL, cI, cG;
    T latent, xi2, inv_axi2, ksig, kgrad, eps0, eps1, inv_de, gamma, zeta;
    T theta_micro;
    __device__ __forceinline__ explicit CoefT(const Coefs& c)
        : inv_h2(T(c.inv_h2)), half_inv_h2(T(c.half_inv_h2)),
          lamL(T(c.lam[0])), lamI(T(c.lam[1])), lamG(T(c.lam[2])),
          rhoL(T(c.rho[0])), rhoI(T(c.rho[1])), rhoG(T(c.rho[2])),
          cL(T(c.cap[0])), cI(T(c.cap[1])), cG(T(c.cap[2])),
          latent(T(c.latent)), xi2(T(c.xi2)), inv_axi2(T(c.inv_axi2)), ksig(T(c.ksig)),
          kgrad(T(c.kgrad)), eps0(T(c.eps0)), eps1(T(c.eps1)), inv_de(T(c.inv_de)),
          gamma(T(c.gamma)), zeta(T(c.zeta)), theta_micro(T(c.theta_micro)) {}
};

// Load one cell of the stage input: theta, phi (the Temp model's phi(theta),
// eq. explicit-p-dependence-on-T), blended conductivity and G.
template <int MODEL, typename T, typename TIN>
__device__ __forceinline__ void load_cell(const CoefT<T>& c, const TIN* __restrict__ in_th,
                                          const TIN* __restrict__ in_ph, const T* __restrict__ Gf,
                                          long long id, T& th, T& ph, T& lam, T& G) {
    G = Gf[id];
    if constexpr (MODEL == M_MICRO) th = c.theta_micro;
    else th = T(in_th[id]);
    if constexpr (MODEL == M_TEMP) ph = T(0.5) * water_ind(G, c.zeta) * (T(1) - dtanh(c.gamma * th));
    else ph = T(in_ph[id]);
    if constexpr (MODEL == M_MICRO) lam = T(0);
    else lam = blend(G, ph, c.lamL, c.lamI, c.lamG);
}

template <int MODEL, int RX, typename T, typename TIN, int STAGE, int BY>
__global__ void __launch_bounds__(TX * BY)
stage_kernel(const StageArgs<T> a) {
    static_assert(STAGE == 1 ? std::is_same<TIN, double>::value : std::is_same<TIN, T>::value,
                  "stage 1 reads the binary64 state; other stages read stage buffers");
    constexpr bool HAS_TH = (MODEL != M_MICRO);  // theta integrated
    constexpr bool HAS_PH = (MODEL != M_TEMP);   // phi integrated
    constexpr bool F32 = std::is_same<T, float>::value;

    Ctrl* ctrl = a.ctrl;
    int cur = 0;
    double dt = 0.0, tstart = a.t_rhs;
    if constexpr (STAGE != 0) {
        if (ctrl->done) return;  // uniform across the grid
        cur = ctrl->cur;
        dt = ctrl->dt_step;
        tstart = ctrl->t;
    }
    const Coefs& cf = a.cf;
    const CoefT<T> c(cf);
    const int n1 = cf.n1, n2 = cf.n2, n3 = cf.n3;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * TX + tx, j = blockIdx.y * BY + ty;
    const int kb = blockIdx.z * a.zc;
    const int ke = min(kb + a.zc, n3);
    const int ic = min(i, n1 - 1), jc = min(j, n2 - 1);
    const bool inside = (i < n1) && (j < n2);
    const long long plane = (long long)n1 * n2;
    const int ixm = min(max(i - 1, 0), n1 - 1), ixp = min(i + 1, n1 - 1);
    const int jym = min(max(j - 1, 0), n2 - 1), jyp = min(j + 1, n2 - 1);

    const TIN* in_th = nullptr;
    const TIN* in_ph = nullptr;
    if constexpr (STAGE == 0) {
        in_th = reinterpret_cast<const TIN*>(a.in_th);
        in_ph = reinterpret_cast<const TIN*>(a.in_ph);
    } else if constexpr (STAGE == 1) {
        in_th = reinterpret_cast<const TIN*>(a.y_th[cur]);
        in_ph = reinterpret_cast<const TIN*>(a.y_ph[cur]);
    } else if constexpr (STAGE == 2 || STAGE == 4) {
        in_th = reinterpret_cast<const TIN*>(a.ua_th);
        in_ph = reinterpret_cast<const TIN*>(a.ua_ph);
    } else {
        in_th = reinterpret_cast<const TIN*>(a.ub_th);
        in_ph = reinterpret_cast<const TIN*>(a.ub_ph);
    }

    constexpr int SX = TX + 2, SY = BY + 2;
    __shared__ T s_th[2][SY][SX];
    __shared__ T s_ph[2][SY][SX];
    __shared__ T s_lam[2][SY][SX];

    const T* __restrict__ Gf = a.G;
    auto load_plane = [&](int kk, int b, T& th, T& ph, T& lam, T& G) {
        const int kc = min(max(kk, 0), n3 - 1);
        const long long base = (long long)kc * plane;
        load_cell<MODEL, T, TIN>(c, in_th, in_ph, Gf, base + (long long)jc * n1 + ic, th, ph, lam, G);
        s_th[b][ty + 1][tx + 1] = th;
        s_ph[b][ty + 1][tx + 1] = ph;
        s_lam[b][ty + 1][tx + 1] = lam;
        T h_th, h_ph, h_lam, h_G;
        if (tx == 0) {
            load_cell<MODEL, T, TIN>(c, in_th, in_ph, Gf, base + (long long)jc * n1 + ixm, h_th, h_ph, h_lam, h_G);
            s_th[b][ty + 1][0] = h_th; s_ph[b][ty + 1][0] = h_ph; s_lam[b][ty + 1][0] = h_lam;
        }
        if (tx == TX - 1) {
            load_cell<MODEL, T, TIN>(c, in_th, in_ph, Gf, base + (long long)jc * n1 + ixp, h_th, h_ph, h_lam, h_G);
            s_th[b][ty + 1][TX + 1] = h_th; s_ph[b][ty + 1][TX + 1] = h_ph; s_lam[b][ty + 1][TX + 1] = h_lam;
        }
        if (ty == 0) {
            load_cell<MODEL, T, TIN>(c, in_th, in_ph, Gf, base + (long long)jym * n1 + ic, h_th, h_ph, h_lam, h_G);
            s_th[b][0][tx + 1] = h_th; s_ph[b][0][tx + 1] = h_ph; s_lam[b][0][tx + 1] = h_lam;
        }
        if (ty == BY - 1) {
            load_cell<MODEL, T, TIN>(c, in_th, in_ph, Gf, base + (long long)jyp * n1 + ic, h_th, h_ph, h_lam, h_G);
            s_th[b][BY + 1][tx + 1] = h_th; s_ph[b][BY + 1][tx + 1] = h_ph; s_lam[b][BY + 1][tx + 1] = h_lam;
        }
    };

    // Dirichlet faces of this column (x and y faces are fixed along the march)
    const double t_b = (tstart < cf.t_freeze) ? cf.theta_freeze : cf.theta_thaw;
    const T th_b = T(t_b);
    int nd_xy = 0;
    if (cf.dirichlet) {
        nd_xy += ((cf.dirichlet & 1) && i == 0) + ((cf.dirichlet & 2) && i == n1 - 1);
        nd_xy += ((cf.dirichlet & 4) && j == 0) + ((cf.dirichlet & 8) && j == n2 - 1);
    }

    // stage coefficients
    const T c13 = T(dt / 3.0), c16 = T(dt / 6.0), c18 = T(dt / 8.0), c38 = T(3.0 * dt / 8.0);
    const T c12 = T(dt / 2.0), c32 = T(1.5 * dt), c2 = T(2.0 * dt), c30 = T(dt / 30.0);
    const T c524 = T(5.0 * dt / 24.0), c158 = T(15.0 * dt / 8.0);

    T thm, phm, lamm, Gm, thc, phc, lamc, Gc, thp, php, lamp, Gp;
    {
        const int km = min(max(kb - 1, 0), n3 - 1);
        load_cell<MODEL, T, TIN>(c, in_th, in_ph, Gf, (long long)km * plane + (long long)jc * n1 + ic, thm, phm,
                                 lamm, Gm);
    }
    load_plane(kb, 0, thc, phc, lamc, Gc);
    __syncthreads();

    T emax = T(0);
    bool nonfinite = false;

    for (int k = kb; k < ke; ++k) {
        const int b = (k - kb) & 1;
        load_plane(k + 1, b ^ 1, thp, php, lamp, Gp);
        if (inside) {
            const long long id = (long long)k * plane + (long long)j * n1 + i;
            // ---- heat flux divergence (eq. heat-equation), per-face conductivity
            T div = T(0);
            if constexpr (MODEL != M_MICRO) {
                const T t_xm = s_th[b][ty + 1][tx], t_xp = s_th[b][ty + 1][tx + 2];
                const T t_ym = s_th[b][ty][tx + 1], t_yp = s_th[b][ty + 2][tx + 1];
                const T l_xm = s_lam[b][ty + 1][tx], l_xp = s_lam[b][ty + 1][tx + 2];
                const T l_ym = s_lam[b][ty][tx + 1], l_yp = s_lam[b][ty + 2][tx + 1];
                if (!cf.harmonic) {
                    div = (lamc + l_xm) * (t_xm - thc) + (lamc + l_xp) * (t_xp - thc) +
                          (lamc + l_ym) * (t_ym - thc) + (lamc + l_yp) * (t_yp - thc) +
                          (lamc + lamm) * (thm - thc) + (lamc + lamp) * (thp - thc);
                    div *= c.half_inv_h2;
                } else {
                    auto hm = [&](T lj) { T s = lamc + lj; return s > T(0) ? T(2) * lamc * lj / s : T(0); };
                    div = hm(l_xm) * (t_xm - thc) + hm(l_xp) * (t_xp - thc) + hm(l_ym) * (t_ym - thc) +
                          hm(l_yp) * (t_yp - thc) + hm(lamm) * (thm - thc) + hm(lamp) * (thp - thc);
                    div *= c.inv_h2;
                }
                int nd = nd_xy;
                if (cf.dirichlet) nd += ((cf.dirichlet & 16) && k == 0) + ((cf.dirichlet & 32) && k == n3 - 1);
                if (nd) div += T(nd) * (T(2) * lamc * (th_b - thc) * c.inv_h2);
            }
            // ---- Allen-Cahn rate (eq. Allen-Cahn-equation)
            T dph = T(0);
            if constexpr (MODEL != M_TEMP) {
                const T IW = water_ind(Gc, c.zeta);
                if (IW > T(0)) {
                    const T p_xm = s_ph[b][ty + 1][tx], p_xp = s_ph[b][ty + 1][tx + 2];
                    const T p_ym = s_ph[b][ty][tx + 1], p_yp = s_ph[b][ty + 2][tx + 1];
                    const T lap = ((p_xm - phc) + (p_xp - phc) + (p_ym - phc) + (p_yp - phc) + (phm - phc) +
                                   (php - phc)) * c.inv_h2;
                    const T under = -thc;  // T* - T
                    T f;
                    if constexpr (RX == R_GRADP) {
                        const T gx = p_xp - p_xm, gy = p_yp - p_ym, gz = php - phm;
                        f = T(2) * phc * (T(1) - phc) * (phc - T(0.5)) +
                            c.kgrad * dsqrt(gx * gx + gy * gy + gz * gz) * under;
                    } else {
                        const T S = sigma_lim(phc, c.eps0, c.eps1, c.inv_de) *
                                    sigma_lim(T(1) - phc, c.eps0, c.eps1, c.inv_de);
                        f = T(2) * phc * (T(1) - phc) * (phc - T(0.5) + c.ksig * S * under);
                    }
                    dph = IW * (c.xi2 * lap + f) * c.inv_axi2;
                }
            }
            // ---- latent-heat coupling
            T dth = T(0);
            if constexpr (MODEL == M_FULL) {
                const T rho = blend(Gc, phc, c.rhoL, c.rhoI, c.rhoG);
                const T cp = blend(Gc, phc, c.cL, c.cI, c.cG);
                dth = (div + rho * c.latent * dph) / (rho * cp);
            } else if constexpr (MODEL == M_TEMP) {
                const T rho = blend(Gc, phc, c.rhoL, c.rhoI, c.rhoG);
                const T cp = blend(Gc, phc, c.cL, c.cI, c.cG);
                const T tg = dtanh(c.gamma * thc);
                const T dp = T(-0.5) * water_ind(Gc, c.zeta) * c.gamma * (T(1) - tg * tg);
                dth = div / (rho * (cp - c.latent * dp));
                dph = dp * dth;  // eq. after (combined-heat-xfer-phase-transition)
            }

            // ---- fused stage combination
            if constexpr (STAGE == 0) {
                if (a.out_th) a.out_th[id] = dth;
                if (a.out_ph) a.out_ph[id] = dph;
            } else if constexpr (STAGE == 1) {
                if constexpr (HAS_TH) { a.k1_th[id] = dth; a.ua_th[id] = thc + c13 * dth; }
                if constexpr (HAS_PH) { a.k1_ph[id] = dph; a.ua_ph[id] = phc + c13 * dph; }
            } else if constexpr (STAGE == 2) {
                if constexpr (F32) {
                    if constexpr (HAS_TH) a.ub_th[id] = thc + c16 * (dth - a.k1_th[id]);
                    if constexpr (HAS_PH) a.ub_ph[id] = phc + c16 * (dph - a.k1_ph[id]);
                } else {
                    if constexpr (HAS_TH) a.ub_th[id] = T(a.y_th[cur][id]) + c16 * (a.k1_th[id] + dth);
                    if constexpr (HAS_PH) a.ub_ph[id] = T(a.y_ph[cur][id]) + c16 * (a.k1_ph[id] + dph);
                }
            } else if constexpr (STAGE == 3) {
                if constexpr (F32) {
                    if constexpr (HAS_TH) { a.k3_th[id] = dth; a.ua_th[id] = a.ua_th[id] - c524 * a.k1_th[id] + c38 * dth; }
                    if constexpr (HAS_PH) { a.k3_ph[id] = dph; a.ua_ph[id] = a.ua_ph[id] - c524 * a.k1_ph[id] + c38 * dph; }
                } else {
                    if constexpr (HAS_TH) { a.k3_th[id] = dth; a.ua_th[id] = T(a.y_th[cur][id]) + c18 * a.k1_th[id] + c38 * dth; }
                    if constexpr (HAS_PH) { a.k3_ph[id] = dph; a.ua_ph[id] = T(a.y_ph[cur][id]) + c18 * a.k1_ph[id] + c38 * dph; }
                }
            } else if constexpr (STAGE == 4) {
                if constexpr (F32) {
                    if constexpr (HAS_TH) { a.k4_th[id] = dth; a.ub_th[id] = thc + c38 * a.k1_th[id] - c158 * a.k3_th[id] + c2 * dth; }
                    if constexpr (HAS_PH) { a.k4_ph[id] = dph; a.ub_ph[id] = phc + c38 * a.k1_ph[id] - c158 * a.k3_ph[id] + c2 * dph; }
                } else {
                    if constexpr (HAS_TH) { a.k4_th[id] = dth; a.ub_th[id] = T(a.y_th[cur][id]) + c12 * a.k1_th[id] - c32 * a.k3_th[id] + c2 * dth; }
                    if constexpr (HAS_PH) { a.k4_ph[id] = dph; a.ub_ph[id] = T(a.y_ph[cur][id]) + c12 * a.k1_ph[id] - c32 * a.k3_ph[id] + c2 * dph; }
                }
            } else {  // STAGE 5
                if constexpr (HAS_TH) {
                    const T k1 = a.k1_th[id], k3 = a.k3_th[id], k4 = a.k4_th[id];
                    if constexpr (F32) a.yo_th[cur ^ 1][id] = a.y_th[cur][id] + double(c16 * (k1 + T(4) * k4 + dth));
                    else a.yo_th[cur ^ 1][id] = a.y_th[cur][id] + c16 * (k1 + T(4) * k4 + dth);
                    const T e = fabs(c30 * (T(2) * k1 - T(9) * k3 + T(8) * k4 - dth));
                    if (!(e < T(INFINITY))) nonfinite = true; else emax = e > emax ? e : emax;
                }
                if constexpr (HAS_PH) {
                    const T k1 = a.k1_ph[id], k3 = a.k3_ph[id], k4 = a.k4_ph[id];
                    if constexpr (F32) a.yo_ph[cur ^ 1][id] = a.y_ph[cur][id] + double(c16 * (k1 + T(4) * k4 + dph));
                    else a.yo_ph[cur ^ 1][id] = a.y_ph[cur][id] + c16 * (k1 + T(4) * k4 + dph);
                    const T e = fabs(c30 * (T(2) * k1 - T(9) * k3 + T(8) * k4 - dph));
                    if (!(e < T(INFINITY))) nonfinite = true; else emax = e > emax ? e : emax;
                }
            }
        }
        thm = thc; phm = phc; lamm = lamc; Gm = Gc;
        thc = thp; phc = php; lamc = lamp; Gc = Gp;
        __syncthreads();
    }

    if constexpr (STAGE == 5) {
        // block max of the error estimate -> one atomicMax on the bit pattern (valid for E >= 0)
        double e = nonfinite ? double(INFINITY) : double(emax);
        for (int o = 16; o > 0; o >>= 1) {
            double v = __shfl_xor_sync(0xffffffffu, e, o);
            e = v > e ? v : e;
        }
        __shared__ double s_red[BY];
        if (tx == 0) s_red[ty] = e;
        __syncthreads();
        if (ty == 0) {
            double v = tx < BY ? s_red[tx] : 0.0;
            for (int o = 16; o > 0; o >>= 1) {
                double w = __shfl_xor_sync(0xffffffffu, v, o);
                v = w > v ? w : v;
            }
            if (tx == 0 && v > 0.0)
                atomicMax(&ctrl->err_bits, (unsigned long long)__double_as_longlong(v));
        }
    }
    (void)Gm;
}

}  // namespace pfgb
