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
// Tiling: a block of 32 x BY threads owns a 32 x BY column of cells and marches
// along z over ZC planes.  Plane k (with a one-cell lateral halo) sits in shared
// memory together with the blended conductivity of every cell, so each cell's
// lambda is evaluated once per plane visit; the z neighbours of a thread's own
// column stay in registers.  The raw values of plane k+2 are loaded while plane
// k is computed (three-plane shared-memory ring, one barrier per plane), and the
// stage-combination operands are loaded before the right-hand-side arithmetic
// (binary32 stages 2-4: one plane ahead), so memory latency overlaps computation.
// Cells outside the grid are replaced by the nearest boundary cell (mirror ghost),
// which makes the interior formula give zero flux on every face; Dirichlet faces
// add their half-cell flux separately.  A z-slab of a multi-domain run instead reads
// the ghost plane its neighbour slab fills (Coefs::zlo, zhi).
//
// Binary64 operation count: the binary64 pipe of sm_103a issues two FMAs per clock
// per SM, a sixtieth of the binary32 rate, so the binary64 kernels keep every
// comparison, absolute value and maximum in integer instructions on the IEEE bit
// patterns, take blends as three FMAs, and divide with one third-order reciprocal step
// seeded by the binary32 reciprocal.
//
// Binary32 form (T = float): stage inputs chain from one stage input to the next
// (u3 = u2 + dt/6 (k2 - k1), u4 = u2 - 5dt/24 k1 + 3dt/8 k3,
// u5 = u4 + 3dt/8 k1 - 15dt/8 k3 + 2dt k4 -- algebraically the tableau rows) so that
// only stages 1 and 5 touch the binary64 state; the state update y' = y + (dt/6 (k1 +
// 4k4 + k5)) adds a binary32 increment to binary64 y.  For the full model the chained quantities are
// the increments d_s = u_s - y32 over a binary32 copy y32 of the state (set with the state, written by
// stage 5 beside the candidate state, so stage 1 reads it instead of the binary64 state), and the
// stiff terms (heat flux, Laplacian) are formed from differences of y32 and of d_s separately: the
// rounding of y to binary32 is then the same in every stage and drops out of the error estimate
// (2 - 9 + 8 - 1 = 0), where rounding each u_s separately left a noise floor in E that the latent
// heat (L/c ~ 160 K) lifts above usual tolerances, and the controller took several times more steps.
#pragma once
#include "pf_internal.cuh"
#include <cfloat>
#include <type_traits>

namespace pfgb {

// tanh in binary64; for |x| >= 20 the result is +-1 exactly (1 - tanh|x| < 2 e^-40 is below half an
// ulp of 1, 2^-54), decided on the bit pattern, so cells far from the melting point skip the call
__device__ __forceinline__ double dtanh(double x) {
    const long long b = __double_as_longlong(x);
    const long long a = b & 0x7FFFFFFFFFFFFFFFLL;
    if (a >= 0x4034000000000000LL) {                 // |x| >= 20, infinities and NaN
        if (a > 0x7FF0000000000000LL) return x;      // NaN
        return __longlong_as_double((b & (1LL << 63)) | 0x3FF0000000000000LL);
    }
    return tanh(x);
}
__device__ __forceinline__ float dtanh(float x) { return tanhf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double FMA(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float FMA(float a, float b, float c) { return fmaf(a, b, c); }

// Comparisons against a non-negative constant y through the IEEE bit pattern
// (signed-integer order equals numeric order for x >= -0 and puts negatives first).
__device__ __forceinline__ bool le_nonneg(double x, double y) { return __double_as_longlong(x) <= __double_as_longlong(y); }
__device__ __forceinline__ bool le_nonneg(float x, float y) { return x <= y; }
__device__ __forceinline__ bool ge_nonneg(double x, double y) { return __double_as_longlong(x) >= __double_as_longlong(y); }
__device__ __forceinline__ bool ge_nonneg(float x, float y) { return x >= y; }
__device__ __forceinline__ bool lt_nonneg(double x, double y) { return __double_as_longlong(x) < __double_as_longlong(y); }
__device__ __forceinline__ bool lt_nonneg(float x, float y) { return x < y; }
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool positive(float x) { return x > 0.f; }

// 1/x for x > 0: from the binary32 reciprocal r of x's leading 20 mantissa bits (r = (1 + u)/x with
// |u| < 2^-19.9), one third-order step r <- r + r (d + d^2), d = 1 - x r = -u: r (1 - u + u^2) =
// (1 + u^3)/x, |u^3| < 2^-59, so the step's single final rounding leaves it within about half an ulp
// (three binary64 FMAs where two Newton steps take four).  The binary32 seed is built from the bit
// pattern with integer instructions.
__device__ __forceinline__ double recip_pos(double x) {
    const long long b = __double_as_longlong(x);
    const int hi = (int)(b >> 32);
    const int e = ((hi >> 20) & 0x7FF) - 1023 + 127;
    if (b <= 0 || e < 2 || e > 252) return 1.0 / x;
    const float xf = __int_as_float((e << 23) | ((hi & 0xFFFFF) << 3));
    const int bf = __float_as_int(__frcp_rn(xf));
    const long long er = (long long)(((bf >> 23) & 0xFF) - 127 + 1023);
    double r = __longlong_as_double((er << 52) | ((long long)(bf & 0x7FFFFF) << 29));
    const double d = fma(-x, r, 1.0);
    return fma(r, fma(d, d, d), r);
}
__device__ __forceinline__ float recip_pos(float x) { return __frcp_rn(x); }

// Conversions between binary64 and binary32 in 32-bit integer instructions on the two halves of the
// binary64 bit pattern.  The binary64 pipe of sm_103a (two operations per clock per SM) executes the
// conversion instructions and 64-bit integer arithmetic too, which would make them a large part of
// the binary32 kernels that touch the binary64 state (stages 1 and 5).  Both follow the IEEE 754
// formats: the exponent is rebiased by 1023 - 127 = 896 and the significand is shifted by
// 52 - 23 = 29 bits.  Values outside the range of binary32 normal numbers (except zero) take the
// conversion instruction.

// binary32 -> binary64 (exact)
__device__ __forceinline__ double widen(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned a = b & 0x7FFFFFFFu;
    if (a - 0x00800000u < 0x7F000000u)  // exponent field in [1, 254]: normal
        return __hiloint2double((int)(((a >> 3) + (896u << 20)) | (b & 0x80000000u)), (int)(a << 29));
    if (a == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)x;
}

// binary64 -> binary32, round to nearest, ties to even: the 29 dropped significand bits (the low 29
// bits of the low word) are rounded by adding 2^28 - 1 plus the lowest kept bit; a carry out of the
// significand increments the exponent (up to infinity, as rounding to nearest requires).  The shift
// of the high word drops the top exponent bits; the rebias is exact modulo 2^32.
__device__ __forceinline__ float narrow(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned a = hi & 0x7FFFFFFFu;
    if ((a >> 20) - 897u < 254u) {  // exponent field in [897, 1150]: binary32 normal
        unsigned f = ((a << 3) | (lo >> 29)) - (896u << 23);
        f += ((lo & 0x1FFFFFFFu) + 0x0FFFFFFFu + (f & 1u)) >> 29;
        return __uint_as_float(f | (hi & 0x80000000u));
    }
    if ((a | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return (float)x;
}

template <typename T> __device__ __forceinline__ T to_T(double x) { return T(x); }
template <> __device__ __forceinline__ float to_T<float>(double x) { return narrow(x); }
template <typename T> __device__ __forceinline__ T to_T(float x) { return T(x); }

// eq. (Sigma-limiter)
template <typename T>
__device__ __forceinline__ T sigma_lim(T w, const CoefT<T>& k) {
    if (le_nonneg(w, k.eps0)) return T(0);
    if (ge_nonneg(w, k.eps1)) return T(1);
    const T s = (w - k.eps0) * k.inv_de;
    return s * s * FMA(T(-2), s, T(3));
}

// eq. (material-properties-blending-formula): w0 + G dG + (1 - G) phi dI
template <typename T>
__device__ __forceinline__ T blend3(T G, T ph, T w0, T dG, T dI) {
    return FMA(ph, FMA(-G, dI, dI), FMA(G, dG, w0));
}

// eq. (water-indicator)
template <typename T>
__device__ __forceinline__ T water_ind(T G, T zeta) {
    const T v = FMA(-zeta, G, T(1));
    return positive(v) ? v : T(0);
}

// phi of a cell and of its six neighbours all exactly +0 or all exactly 1 (IEEE bit patterns, integer
// instructions only).  There the Laplacian is 0 and the reaction term 2 phi (1 - phi)(...) is 0, so
// dphi/dt = 0 exactly (eq. Allen-Cahn-equation): the bulk of the water and of the ice.
__device__ __forceinline__ bool uniform_01(double c, double a0, double a1, double a2, double a3, double a4,
                                           double a5) {
    const long long cb = __double_as_longlong(c);
    bool r = (cb == 0LL) | (cb == 0x3FF0000000000000LL);
    r &= (__double_as_longlong(a0) == cb) & (__double_as_longlong(a1) == cb) & (__double_as_longlong(a2) == cb);
    r &= (__double_as_longlong(a3) == cb) & (__double_as_longlong(a4) == cb) & (__double_as_longlong(a5) == cb);
    return r;
}
__device__ __forceinline__ bool uniform_01(float c, float a0, float a1, float a2, float a3, float a4, float a5) {
    const int cb = __float_as_int(c);
    bool r = (cb == 0) | (cb == 0x3F800000);
    r &= (__float_as_int(a0) == cb) & (__float_as_int(a1) == cb) & (__float_as_int(a2) == cb);
    r &= (__float_as_int(a3) == cb) & (__float_as_int(a4) == cb) & (__float_as_int(a5) == cb);
    return r;
}
__device__ __forceinline__ bool is_one(double v) { return __double_as_longlong(v) == 0x3FF0000000000000LL; }
__device__ __forceinline__ bool is_01(double v) {
    const long long b = __double_as_longlong(v);
    return b == 0LL || b == 0x3FF0000000000000LL;
}
__device__ __forceinline__ bool is_one(float v) { return __float_as_int(v) == 0x3F800000; }

template <typename T>
__device__ __forceinline__ unsigned long long abs_bits(T v) {
    if constexpr (std::is_same<T, double>::value) {
        return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
    } else {
        return (unsigned long long)((unsigned)__float_as_int(v) & 0x7FFFFFFFu);
    }
}

// Allen-Cahn rate of one cell from phi, its six neighbours, theta and W = 2 I_W / (alpha xi^2) > 0
// (eqs. Allen-Cahn-equation, reaction-term-GradP, reaction-term-SigmaP1-P, Sigma-limiter)
template <int RX, typename T>
__device__ __forceinline__ T allen_cahn_rate(const CoefT<T>& K, T pc, T pxm, T pxp, T pym, T pyp, T pzm, T pzp, T th,
                                             T W) {
    const T lsum = ((pxm + pxp) + (pym + pyp)) + (pzm + pzp);
    const T lap = FMA(T(-6), pc, lsum);
    const T om = T(1) - pc;
    const T q = pc * om;
    T inner = pc - T(0.5);
    T fh;
    if constexpr (RX == R_GRADP) {
        const T gx = pxp - pxm, gy = pyp - pym, gz = pzp - pzm;
        const T gn = dsqrt(FMA(gx, gx, FMA(gy, gy, gz * gz)));
        fh = FMA(q, inner, K.kgrad * gn * (-th));          // eq. (reaction-term-GradP) / 2
    } else {
        if (!le_nonneg(pc, K.eps0) && !le_nonneg(om, K.eps0)) {
            const T S = sigma_lim(pc, K) * sigma_lim(om, K);
            inner = FMA(K.ksig * S, -th, inner);            // eq. (reaction-term-SigmaP1-P) / 2
        }
        fh = q * inner;
    }
    return W * FMA(K.klap, lap, fh);
}

// The same rate at phi = a + d, where a is the cell's value in the binary32 copy of the state (common to
// every stage of the step) and d the stage's increment, with the neighbours split the same way.  The
// Laplacian, the gradient and the factor phi (1 - phi) are formed from differences of a and of d
// separately: the rounding of a + d then enters only the limiter and the temperature factor, so the
// stages' rates carry the same rounding of a (it cancels in the error estimate) instead of each its own.
template <int RX, typename T>
__device__ __forceinline__ T allen_cahn_rate_inc(const CoefT<T>& K, T a, T d, T axm, T axp, T aym, T ayp, T azm,
                                                 T azp, T dxm, T dxp, T dym, T dyp, T dzm, T dzp, T th, T W) {
    const T lap = FMA(T(-6), a, ((axm + axp) + (aym + ayp)) + (azm + azp)) +
                  FMA(T(-6), d, ((dxm + dxp) + (dym + dyp)) + (dzm + dzp));
    const T pc = a + d;
    const T om = T(1) - pc;
    // (a + d)(1 - a - d) = a (1 - a) + d (1 - 2a - d)
    const T q = FMA(d, (T(1) - T(2) * a) - d, a * (T(1) - a));
    T inner = (a - T(0.5)) + d;
    T fh;
    if constexpr (RX == R_GRADP) {
        const T gx = (axp - axm) + (dxp - dxm), gy = (ayp - aym) + (dyp - dym), gz = (azp - azm) + (dzp - dzm);
        const T gn = dsqrt(FMA(gx, gx, FMA(gy, gy, gz * gz)));
        fh = FMA(q, inner, K.kgrad * gn * (-th));
    } else {
        if (!le_nonneg(pc, K.eps0) && !le_nonneg(om, K.eps0)) {
            const T S = sigma_lim(pc, K) * sigma_lim(om, K);
            inner = FMA(K.ksig * S, -th, inner);
        }
        fh = q * inner;
    }
    return W * FMA(K.klap, lap, fh);
}

// End of a tile: stage 5 folds the block's largest |2k1 - 9k3 + 8k4 - k5| into the error maximum (one
// atomicMax on the binary64 bit pattern, scaled by dt/30); stage 1 adds the block's pore-bulk counts and
// folds its largest |dphi/dt| (warp shuffles, then shared memory across the block's warps).
template <int STAGE, bool HAS_PH, bool F32, int BY>
__device__ __forceinline__ void publish_block(Ctrl* ctrl, unsigned long long ebits, unsigned int icount,
                                              unsigned int pcount, unsigned long long rbits) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    if constexpr (STAGE == 5) {
        // block max of |E| -> one atomicMax on the binary64 bit pattern (valid for E >= 0; NaN/Inf
        // patterns sort above every finite value)
        unsigned long long e = ebits;
        if constexpr (F32) {
            const unsigned fb = (unsigned)e;
            e = (fb >= 0x7F800000u) ? 0x7FF0000000000000ULL
                                    : (unsigned long long)__double_as_longlong((double)__uint_as_float(fb));
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, e, o);
            e = v > e ? v : e;
        }
        __shared__ unsigned long long s_red[BY];
        if (tx == 0) s_red[ty] = e;
        __syncthreads();
        if (ty == 0) {
            unsigned long long v = tx < BY ? s_red[tx] : 0ULL;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
                v = w > v ? w : v;
            }
            if (tx == 0 && v > 0ULL) {
                if (v < 0x7FF0000000000000ULL)  // finite: scale by dt/30 (binary64)
                    v = (unsigned long long)__double_as_longlong(__longlong_as_double((long long)v) * ctrl->sc[7]);
                atomicMax(&ctrl->err_bits, v);
            }
        }
    }
    if constexpr (STAGE == 1 && HAS_PH) {
        // block sums of the two counts -> one atomicAdd each; block max of |dphi/dt| -> one atomicMax
        unsigned int ci = icount, cp = pcount;
        unsigned long long r = rbits;
        if constexpr (F32) {
            const unsigned fb = (unsigned)r;
            r = (fb >= 0x7F800000u) ? 0x7FF0000000000000ULL
                                    : (unsigned long long)__double_as_longlong((double)__uint_as_float(fb));
        }
        for (int o = 16; o > 0; o >>= 1) {
            ci += __shfl_xor_sync(0xffffffffu, ci, o);
            cp += __shfl_xor_sync(0xffffffffu, cp, o);
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, r, o);
            r = v > r ? v : r;
        }
        __shared__ unsigned int s_cnt[2][BY];
        __shared__ unsigned long long s_rate[BY];
        if (tx == 0) { s_cnt[0][ty] = ci; s_cnt[1][ty] = cp; s_rate[ty] = r; }
        __syncthreads();
        if (ty == 0) {
            unsigned int v = tx < BY ? s_cnt[0][tx] : 0u, w = tx < BY ? s_cnt[1][tx] : 0u;
            unsigned long long m = tx < BY ? s_rate[tx] : 0ULL;
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
                const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
                m = x > m ? x : m;
            }
            if (tx == 0 && v > 0u) atomicAdd(&ctrl->ice_count, (unsigned long long)v);
            if (tx == 0 && w > 0u) atomicAdd(&ctrl->pore_count, (unsigned long long)w);
            if (tx == 0 && m > 0ULL) atomicMax(&ctrl->rate_bits, m);
        }
    }
}

// One tile (32 x BY columns, one z chunk) of one stage.  (bxi, byi, bzi) is the tile's position in
// the grid's tile lattice.  Called by the single-grid kernel (one block per tile) and by the batched
// persistent kernel (blocks loop over the tiles of all active instances).
template <int MODEL, int RX, typename T, typename TIN, int STAGE, int BY>
__device__ __forceinline__ void stage_tile(const StageArgs<T>& a, const int bxi, const int byi, const int bzi) {
    static_assert((STAGE == 1 && !(std::is_same<T, float>::value && MODEL == M_FULL))
                      ? std::is_same<TIN, double>::value : std::is_same<TIN, T>::value,
                  "stage 1 reads the binary64 state (the binary32 form of the full model: its binary32 copy); "
                  "other stages read stage buffers");
    constexpr bool HAS_TH = (MODEL != M_MICRO);  // theta integrated
    constexpr bool HAS_PH = (MODEL != M_TEMP);   // phi integrated
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr bool TEMP = (MODEL == M_TEMP);
    // full model in binary64: blends from precomputed per-cell coefficients (fewer binary64 operations)
    constexpr bool STATIC = (!F32 && MODEL == M_FULL);
    // full model in binary32: the inputs of stages 2-5 are increments d = u - y32 over the binary32 copy
    // y32 of the state (stage 1 reads it as its input); the heat flux, the Laplacian and phi (1 - phi)
    // take the differences of y32 and of d separately (see allen_cahn_rate_inc)
    constexpr bool INC = (F32 && MODEL == M_FULL);
    constexpr bool DIN = (INC && STAGE >= 2);

    Ctrl* ctrl = a.ctrl;
    int cur = 0;
    T th_b;
    T sc[NSC];
    if constexpr (STAGE != 0) {
        if (ctrl->done) return;  // uniform across the grid
        cur = ctrl->cur;
        if constexpr (F32) {
            th_b = ctrl->theta_bf;
#pragma unroll
            for (int q = 0; q < NSC; ++q) sc[q] = ctrl->scf[q];
        } else {
            th_b = ctrl->theta_b;
#pragma unroll
            for (int q = 0; q < NSC; ++q) sc[q] = ctrl->sc[q];
        }
    } else {
        th_b = T((a.t_rhs < a.cf.t_freeze) ? a.cf.theta_freeze : a.cf.theta_thaw);
#pragma unroll
        for (int q = 0; q < NSC; ++q) sc[q] = T(0);
    }
    const CoefT<T>& K = a.k;
    const int n1 = a.cf.n1, n2 = a.cf.n2, n3 = a.cf.n3;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = bxi * TX, j0 = byi * BY;
    const int i = i0 + tx, j = j0 + ty;
    const int kb = bzi * a.zc;
    const int ke = min(kb + a.zc, n3);
    const bool inside = (i < n1) && (j < n2);
    // 32-bit cell indices (grids are limited to fewer than 2^31 cells, ghost planes included, at creation)
    const int plane = n1 * n2;
    const int ooff = min(j, n2 - 1) * n1 + min(i, n1 - 1);

    // one halo cell per thread for the first 2 TX + 2 BY threads: y rows, then x columns
    const int tid = ty * TX + tx;
    bool hal = false;
    int hx = 0, hy = 0;
    if (tid < 2 * TX) {
        hal = true;
        hx = tid % TX;
        hy = (tid < TX) ? -1 : BY;
    } else if (tid < 2 * TX + 2 * BY) {
        hal = true;
        const int r = tid - 2 * TX;
        hy = r % BY;
        hx = (r < BY) ? -1 : TX;
    }
    const int hoff = min(max(j0 + hy, 0), n2 - 1) * n1 + min(max(i0 + hx, 0), n1 - 1);

    const TIN* in_th = nullptr;
    const TIN* in_ph = nullptr;
    if constexpr (STAGE == 0) {
        in_th = reinterpret_cast<const TIN*>(a.in_th);
        in_ph = reinterpret_cast<const TIN*>(a.in_ph);
    } else if constexpr (STAGE == 1 && INC) {
        in_th = reinterpret_cast<const TIN*>(a.y32_th[cur]);
        in_ph = reinterpret_cast<const TIN*>(a.y32_ph[cur]);
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
    // increments: the stage buffer holds d, the values are read from y32
    const T* in_dth = nullptr;
    const T* in_dph = nullptr;
    if constexpr (DIN) {
        in_dth = reinterpret_cast<const T*>(in_th);
        in_dph = reinterpret_cast<const T*>(in_ph);
        in_th = reinterpret_cast<const TIN*>(a.y32_th[cur]);
        in_ph = reinterpret_cast<const TIN*>(a.y32_ph[cur]);
    }
    const T* __restrict__ Gf = a.G;

    constexpr int SX = TX + 2, SY = BY + 2;
    // with increments, each cell's (y32, d) pair of a field sits in one 8-byte entry (one shared load)
    constexpr bool TH1 = HAS_TH && !DIN;
    __shared__ T s_th[TH1 ? 3 : 1][TH1 ? SY : 1][TH1 ? SX : 1];
    __shared__ T s_ph[DIN ? 1 : 3][DIN ? 1 : SY][DIN ? 1 : SX];
    __shared__ T s_lam[HAS_TH ? 3 : 1][SY][SX];
    __shared__ float2 s_th2[DIN ? 3 : 1][DIN ? SY : 1][DIN ? SX : 1];
    __shared__ float2 s_ph2[DIN ? 3 : 1][DIN ? SY : 1][DIN ? SX : 1];

    // the per-cell coefficient arrays (64-bit offsets between arrays, computed once)
    const double* __restrict__ St = a.statics;
    const double* __restrict__ St_B = St + a.ncell;
    const double* __restrict__ St_W = St + 2 * a.ncell;
    const double* __restrict__ St_C = St + 3 * a.ncell;
    const double* __restrict__ St_D = St + 6 * a.ncell;
    const double* __restrict__ St_I = St + 8 * a.ncell;
    const long long NC = a.ncell;
    // raw loads of one cell of plane kk (clamped: mirror ghosts); G holds A_lam and B B_lam when STATIC
    // (theta and phi stay in the input type until `cvt`, so that a conversion does not wait for its
    // load where the load is issued)
    auto fetch = [&](int kk, int off, TIN& th, TIN& ph, T& G, T& B, T& dt, T& dp) {
        const int id = min(max(kk, a.cf.zlo), a.cf.zhi) * plane + off;
        if constexpr (DIN) {
            dt = in_dth[id];
            dp = in_dph[id];
        } else {
            dt = T(0);
            dp = T(0);
        }
        if constexpr (STATIC) {
            G = T(St[id]);
            B = T(St_B[id]);
        } else {
            G = Gf[id];
            B = T(0);
        }
        if constexpr (HAS_TH) th = in_th[id];
        else th = TIN(0);
        if constexpr (HAS_PH) ph = in_ph[id];
        else ph = TIN(0);
    };
    auto cvt = [&](TIN rth, TIN rph, T& th, T& ph) {
        if constexpr (HAS_TH) th = to_T<T>(rth);
        else th = K.theta_micro;
        if constexpr (HAS_PH) ph = to_T<T>(rph);
        else ph = T(0);
    };
    auto fetch_cvt = [&](int kk, int off, T& th, T& ph, T& G, T& B, T& dt, T& dp) {
        TIN rth, rph;
        fetch(kk, off, rth, rph, G, B, dt, dp);
        cvt(rth, rph, th, ph);
    };
    // derived values: Temp phase field (eq. explicit-p-dependence-on-T) and blended conductivity (at
    // phi = y32 + d with increments)
    auto finish = [&](T th, T& ph, T G, T B, T& lam, T& tg, T dp) {
        if constexpr (TEMP) {
            tg = dtanh(K.gamma * th);
            ph = T(0.5) * water_ind(G, K.zeta) * (T(1) - tg);
        }
        if constexpr (STATIC) lam = FMA(ph, B, G);
        else if constexpr (DIN) lam = blend3(G, ph + dp, K.lamL, K.dLG, K.dLI);
        else if constexpr (HAS_TH) lam = blend3(G, ph, K.lamL, K.dLG, K.dLI);
        else lam = T(0);
    };
    auto put = [&](int b, int y, int x, T th, T ph, T lam, T dt, T dp) {
        if constexpr (DIN) {
            s_th2[b][y][x] = make_float2(th, dt);
            s_ph2[b][y][x] = make_float2(ph, dp);
            s_lam[b][y][x] = lam;
        } else {
            if constexpr (HAS_TH) {
                s_th[b][y][x] = th;
                s_lam[b][y][x] = lam;
            }
            s_ph[b][y][x] = ph;
        }
    };
    // a lateral neighbour of plane b: value and (with increments) increment
    auto nb_th = [&](int bb, int yy, int xx, T& v, T& d) {
        if constexpr (DIN) {
            const float2 q = s_th2[bb][yy][xx];
            v = q.x;
            d = q.y;
        } else {
            v = s_th[bb][yy][xx];
            d = T(0);
        }
    };
    auto nb_ph = [&](int bb, int yy, int xx, T& v, T& d) {
        if constexpr (DIN) {
            const float2 q = s_ph2[bb][yy][xx];
            v = q.x;
            d = q.y;
        } else {
            v = s_ph[bb][yy][xx];
            d = T(0);
        }
    };

    auto ac_rate = [&](T pc, T pxm, T pxp, T pym, T pyp, T pzm, T pzp, T th, T W) -> T {
        return allen_cahn_rate<RX>(K, pc, pxm, pxp, pym, pyp, pzm, pzp, th, W);
    };
    // binary64 (full and micro models): the Allen-Cahn arithmetic runs on compacted slots (not for the
    // 16-row blocks, whose planes already fill most of the 48 KiB of static shared memory)
    constexpr bool COMPACT = !F32 && !TEMP && BY <= 8;
    __shared__ int s_wcnt[BY];
    __shared__ int s_slot_xy[COMPACT ? TX * BY : 1];
    // per slot: phi's z neighbours, theta, W; full model also the heat flux divergence and the cell's
    // coefficients of rho c and rho L, so the latent coupling runs on the slots too
    constexpr int NSLOT = COMPACT ? (STATIC ? 10 : 4) : 1;
    __shared__ T s_slot[NSLOT][COMPACT ? TX * BY : 1];

    // Dirichlet faces of this column (x and y faces are fixed along the march)
    const int dmask = a.cf.dirichlet;
    int nd_xy = 0;
    if (dmask) {
        nd_xy += ((dmask & 1) && i == 0) + ((dmask & 2) && i == n1 - 1);
        nd_xy += ((dmask & 4) && j == 0) + ((dmask & 8) && j == n2 - 1);
    }

    // Binary32 stages 2-4 move few bytes and do little arithmetic per cell, so memory latency
    // bounds them: their stage-combination operands are loaded one plane ahead.  (Binary64 kernels
    // are bound by the binary64 pipe, and binary32 stage 5 by its register budget: both load
    // their operands within the plane.)
    constexpr bool PF = F32 && STAGE >= 2 && STAGE <= 4;
    T n_k1t = T(0), n_k1p = T(0), n_k3t = T(0), n_k3p = T(0), n_uat = T(0), n_uap = T(0);
    if constexpr (PF) {
        if (inside && kb < ke) {
            const int q = kb * plane + j * n1 + i;
            if constexpr (HAS_TH) n_k1t = a.k1_th[q];
            if constexpr (HAS_PH) n_k1p = a.k1_ph[q];
            if constexpr (STAGE == 3) {
                if constexpr (HAS_TH) n_uat = a.ua_th[q];
                if constexpr (HAS_PH) n_uap = a.ua_ph[q];
            }
            if constexpr (STAGE == 4) {
                if constexpr (HAS_TH) n_k3t = a.k3_th[q];
                if constexpr (HAS_PH) n_k3p = a.k3_ph[q];
            }
        }
    }

    // ---- prologue: own column at kb-1, kb, kb+1; planes kb, kb+1 into the ring
    T thm, phm, lamm, tgm = T(0), dtm, dpm;
    T thc, phc, lamc, Gc, tgc = T(0), dtc, dpc;
    T thp, php, lamp, Gp, tgp = T(0), dtp, dpp;
    {
        T Gm, Bm, Bc, Bp;
        fetch_cvt(kb - 1, ooff, thm, phm, Gm, Bm, dtm, dpm);
        finish(thm, phm, Gm, Bm, lamm, tgm, dpm);
        fetch_cvt(kb, ooff, thc, phc, Gc, Bc, dtc, dpc);
        finish(thc, phc, Gc, Bc, lamc, tgc, dpc);
        put(0, ty + 1, tx + 1, thc, phc, lamc, dtc, dpc);
        fetch_cvt(kb + 1, ooff, thp, php, Gp, Bp, dtp, dpp);
        finish(thp, php, Gp, Bp, lamp, tgp, dpp);
        put(1, ty + 1, tx + 1, thp, php, lamp, dtp, dpp);
        if (hal) {
            T h_th, h_ph, h_G, h_B, h_lam, h_tg, h_dt, h_dp;
            fetch_cvt(kb, hoff, h_th, h_ph, h_G, h_B, h_dt, h_dp);
            finish(h_th, h_ph, h_G, h_B, h_lam, h_tg, h_dp);
            put(0, hy + 1, hx + 1, h_th, h_ph, h_lam, h_dt, h_dp);
            fetch_cvt(kb + 1, hoff, h_th, h_ph, h_G, h_B, h_dt, h_dp);
            finish(h_th, h_ph, h_G, h_B, h_lam, h_tg, h_dp);
            put(1, hy + 1, hx + 1, h_th, h_ph, h_lam, h_dt, h_dp);
        }
    }
    __syncthreads();

    unsigned long long ebits = 0ULL;  // max |E| as a bit pattern (NaN/Inf sort above every finite value)
    unsigned int icount = 0, pcount = 0;  // stage 1: pore-bulk ice cells and pore-bulk cells of this thread
    unsigned long long rbits = 0ULL;      // stage 1: max |dphi/dt| over this thread's pore-bulk cells
    int b = 0;

#pragma unroll 3
    for (int k = kb; k < ke; ++k) {
        // 1. raw values of plane k+2 (consumed after the arithmetic of plane k)
        TIN rth, rph, qth, qph;
        T rG, rB, qG, qB, rdt, rdp, qdt, qdp;
        fetch(k + 2, ooff, rth, rph, rG, rB, rdt, rdp);
        if (hal) fetch(k + 2, hoff, qth, qph, qG, qB, qdt, qdp);

        const int id = k * plane + j * n1 + i;
        // phase field of the lateral neighbours (Laplacian, gradient) and the bulk test
        // (binary64 only: its integer test is free next to the binary64 arithmetic it can save, while
        // the binary32 kernels are bound by memory and instruction issue, where the test costs more)
        T p_xm = T(0), p_xp = T(0), p_ym = T(0), p_yp = T(0);
        bool bulk = false;
        if constexpr (!TEMP && !F32) {
            p_xm = s_ph[b][ty + 1][tx]; p_xp = s_ph[b][ty + 1][tx + 2];
            p_ym = s_ph[b][ty][tx + 1]; p_yp = s_ph[b][ty + 2][tx + 1];
            bulk = uniform_01(phc, p_xm, p_xp, p_ym, p_yp, phm, php);
        }
        // 2. stage-combination operands of this cell
        T y_t = T(0), y_p = T(0), k1t = T(0), k1p = T(0), k3t = T(0), k3p = T(0), k4t = T(0), k4p = T(0);
        double y_t64 = 0.0, y_p64 = 0.0;
        T ua_t = T(0), ua_p = T(0);
        T sW = T(0), sC0 = T(0), sC1 = T(0), sC2 = T(0), sD0 = T(0), sD1 = T(0), sIR = T(0);
        if constexpr (PF) {
            // take the operands loaded during the previous plane, then load those of plane k+1
            k1t = n_k1t; k1p = n_k1p; k3t = n_k3t; k3p = n_k3p; ua_t = n_uat; ua_p = n_uap;
            if (inside && k + 1 < ke) {
                const int q = id + plane;
                if constexpr (HAS_TH) n_k1t = a.k1_th[q];
                if constexpr (HAS_PH) n_k1p = a.k1_ph[q];
                if constexpr (STAGE == 3) {
                    if constexpr (HAS_TH) n_uat = a.ua_th[q];
                    if constexpr (HAS_PH) n_uap = a.ua_ph[q];
                }
                if constexpr (STAGE == 4) {
                    if constexpr (HAS_TH) n_k3t = a.k3_th[q];
                    if constexpr (HAS_PH) n_k3p = a.k3_ph[q];
                }
            }
        } else if (inside) {
            if constexpr (STAGE >= 2) {
                if constexpr (HAS_TH) k1t = a.k1_th[id];
                if constexpr (HAS_PH) k1p = a.k1_ph[id];
            }
            if constexpr (STAGE >= 4) {
                if constexpr (HAS_TH) k3t = a.k3_th[id];
                if constexpr (HAS_PH) k3p = a.k3_ph[id];
            }
            if constexpr (STAGE == 5) {
                if constexpr (HAS_TH) { k4t = a.k4_th[id]; y_t64 = a.y_th[cur][id]; }
                if constexpr (HAS_PH) { k4p = a.k4_ph[id]; y_p64 = a.y_ph[cur][id]; }
            }
            if constexpr (!F32 && STAGE >= 2 && STAGE <= 4) {
                if constexpr (HAS_TH) y_t = a.y_th[cur][id];
                if constexpr (HAS_PH) y_p = a.y_ph[cur][id];
            }
            if constexpr (F32 && STAGE == 3) {
                if constexpr (HAS_TH) ua_t = a.ua_th[id];
                if constexpr (HAS_PH) ua_p = a.ua_ph[id];
            }
            if constexpr (STATIC) {
                // a cell whose dphi is exactly 0 with phi exactly 0 or 1 (bulk, or no water) needs only
                // 1/(rho c) at its phi; stage 1 also counts the pore cells (W)
                if (STAGE == 1 || !bulk) sW = St_W[id];
                if (bulk || is_01(phc)) sIR = St_I[(is_one(phc) ? NC : 0) + id];
                if (!bulk) {
                    sC0 = St_C[id]; sC1 = St_C[NC + id]; sC2 = St_C[2 * NC + id];
                    sD0 = St_D[id]; sD1 = St_D[NC + id];
                }
            }
        }

        // ---- heat flux divergence (eq. heat-equation), per-face conductivity, lambda pre-scaled by 1/(2h^2)
        T div = T(0);
        if (inside) {
            if constexpr (MODEL != M_MICRO) {
                T t_xm, t_xp, t_ym, t_yp, d_xm, d_xp, d_ym, d_yp;
                nb_th(b, ty + 1, tx, t_xm, d_xm);
                nb_th(b, ty + 1, tx + 2, t_xp, d_xp);
                nb_th(b, ty, tx + 1, t_ym, d_ym);
                nb_th(b, ty + 2, tx + 1, t_yp, d_yp);
                const T l_xm = s_lam[b][ty + 1][tx], l_xp = s_lam[b][ty + 1][tx + 2];
                const T l_ym = s_lam[b][ty][tx + 1], l_yp = s_lam[b][ty + 2][tx + 1];
                // theta_j - theta_c; with increments (y32_j - y32_c) + (d_j - d_c)
                T g_xm = t_xm - thc, g_xp = t_xp - thc, g_ym = t_ym - thc, g_yp = t_yp - thc;
                T g_zm = thm - thc, g_zp = thp - thc, g_b = th_b - thc;
                if constexpr (DIN) {
                    g_xm += d_xm - dtc;
                    g_xp += d_xp - dtc;
                    g_ym += d_ym - dtc;
                    g_yp += d_yp - dtc;
                    g_zm += dtm - dtc;
                    g_zp += dtp - dtc;
                    g_b -= dtc;
                }
                if (!a.cf.harmonic) {
                    div = (lamc + l_xm) * g_xm;
                    div = FMA(lamc + l_xp, g_xp, div);
                    div = FMA(lamc + l_ym, g_ym, div);
                    div = FMA(lamc + l_yp, g_yp, div);
                    div = FMA(lamc + lamm, g_zm, div);
                    div = FMA(lamc + lamp, g_zp, div);
                } else {
                    auto hm = [&](T lj) {
                        const T s = lamc + lj;
                        return positive(s) ? T(4) * lamc * lj / s : T(0);
                    };
                    div = hm(l_xm) * g_xm;
                    div = FMA(hm(l_xp), g_xp, div);
                    div = FMA(hm(l_ym), g_ym, div);
                    div = FMA(hm(l_yp), g_yp, div);
                    div = FMA(hm(lamm), g_zm, div);
                    div = FMA(hm(lamp), g_zp, div);
                }
                if (dmask) {
                    const int nd = nd_xy + ((dmask & 16) && k == 0) + ((dmask & 32) && k == n3 - 1);
                    // Dirichlet face: 2 lambda (theta_b - theta)/h^2 = 4 lambda' (theta_b - theta)
                    if (nd) div = FMA(T(4 * nd) * lamc, g_b, div);
                }
            }
        }
        // ---- Allen-Cahn rate (eq. Allen-Cahn-equation): dphi = W (klap lap + f/2), W = 2 I_W/(alpha xi^2)
        T dph = T(0);
        bool need = false;  // the Allen-Cahn arithmetic runs (W > 0, not bulk)
        T dth_slot = T(0);  // full model, compacted: the latent coupling's result from the slot
        if constexpr (!TEMP) {
            T W = T(0);
            if (inside && !bulk) {  // bulk cells: dphi = 0 without arithmetic
                if constexpr (STATIC) W = sW;
                else W = FMA(K.wb, Gc, K.wa);
            }
            need = positive(W);
            if constexpr (COMPACT) {
                // Binary64: the cells of the block that need the Allen-Cahn arithmetic are packed into
                // consecutive slots (warp ballots and a prefix over the block's warps), so each warp runs
                // it on full lanes; a row of 32 cells mixing glass, bulk and interface cells would run it
                // on all lanes.  Owners leave their z neighbours, theta and W in the slot; the lateral
                // neighbours are read from the plane in shared memory.  (Ordering the slots so that the
                // cells taking the Sigma limiter come first was measured: no gain.)
                const unsigned m = __ballot_sync(0xffffffffu, need);
                if (tx == 0) s_wcnt[ty] = __popc(m);
                __syncthreads();
                int base = 0, total = 0;
#pragma unroll
                for (int w = 0; w < BY; ++w) {
                    const int c = s_wcnt[w];
                    base += (w < ty) ? c : 0;
                    total += c;
                }
                const int slot = base + __popc(m & ((1u << tx) - 1u));
                if (need) {
                    s_slot_xy[slot] = tx | (ty << 8);
                    s_slot[0][slot] = phm;
                    s_slot[1][slot] = php;
                    s_slot[2][slot] = thc;
                    s_slot[3][slot] = W;
                    if constexpr (STATIC) {
                        s_slot[4][slot] = div;
                        s_slot[5][slot] = sC0;
                        s_slot[6][slot] = sC1;
                        s_slot[7][slot] = sC2;
                        s_slot[8][slot] = sD0;
                        s_slot[9][slot] = sD1;
                    }
                }
                __syncthreads();
                for (int q = tid; q < total; q += TX * BY) {
                    const int xy = s_slot_xy[q];
                    const int qx = xy & 255, qy = xy >> 8;
                    const T pc = s_ph[b][qy + 1][qx + 1];
                    const T r = ac_rate(pc, s_ph[b][qy + 1][qx], s_ph[b][qy + 1][qx + 2], s_ph[b][qy][qx + 1],
                                        s_ph[b][qy + 2][qx + 1], s_slot[0][q], s_slot[1][q], s_slot[2][q], s_slot[3][q]);
                    // the rate goes back into the slot's first entry, the coupling's result into the second
                    // (both read above by this thread only)
                    if constexpr (STATIC) {
                        const T rhoc = FMA(pc, FMA(pc, s_slot[7][q], s_slot[6][q]), s_slot[5][q]);
                        s_slot[1][q] = FMA(FMA(pc, s_slot[9][q], s_slot[8][q]), r, s_slot[4][q]) * recip_pos(rhoc);
                    }
                    s_slot[0][q] = r;
                }
                __syncthreads();
                if (need) {
                    dph = s_slot[0][slot];
                    if constexpr (STATIC) dth_slot = s_slot[1][slot];
                }
            } else if (need) {
                T q_xm = T(0), q_xp = T(0), q_ym = T(0), q_yp = T(0);
                if constexpr (F32) {
                    nb_ph(b, ty + 1, tx, p_xm, q_xm);
                    nb_ph(b, ty + 1, tx + 2, p_xp, q_xp);
                    nb_ph(b, ty, tx + 1, p_ym, q_ym);
                    nb_ph(b, ty + 2, tx + 1, p_yp, q_yp);
                }
                if constexpr (DIN)
                    dph = allen_cahn_rate_inc<RX>(K, phc, dpc, p_xm, p_xp, p_ym, p_yp, phm, php, q_xm, q_xp, q_ym, q_yp,
                                                  dpm, dpp, thc + dtc, W);
                else
                    dph = ac_rate(phc, p_xm, p_xp, p_ym, p_yp, phm, php, thc, W);
            }
        }
        if (inside) {
            // ---- latent-heat coupling
            T dth = T(0);
            if constexpr (STATIC) {
                if (COMPACT && need) {
                    dth = dth_slot;
                } else if (!need && (bulk || is_01(phc))) {
                    dth = div * sIR;  // dphi = 0 and phi exactly 0 or 1
                } else {
                    const T rhoc = FMA(phc, FMA(phc, sC2, sC1), sC0);
                    dth = FMA(FMA(phc, sD1, sD0), dph, div) * recip_pos(rhoc);
                }
            } else if constexpr (MODEL == M_FULL) {
                const T phu = DIN ? phc + dpc : phc;
                const T rho = blend3(Gc, phu, K.rhoL, K.dRG, K.dRI);
                const T cp = blend3(Gc, phu, K.capL, K.dCG, K.dCI);
                dth = FMA(rho * K.latent, dph, div) * recip_pos(rho * cp);
            } else if constexpr (TEMP) {
                const T rho = blend3(Gc, phc, K.rhoL, K.dRG, K.dRI);
                const T cp = blend3(Gc, phc, K.capL, K.dCG, K.dCI);
                const T dp = T(-0.5) * water_ind(Gc, K.zeta) * K.gamma * FMA(-tgc, tgc, T(1));
                dth = div * recip_pos(rho * FMA(-K.latent, dp, cp));  // eq. (combined-heat-xfer-phase-transition)
                dph = dp * dth;
            }

            // ---- fused stage combination (binary32 stages 2 and 4 continue from their own input: the
            // increment with increments, else the stage value)
            const T bth = DIN ? dtc : thc, bph = DIN ? dpc : phc;
            if constexpr (STAGE == 0) {
                if (a.out_th) a.out_th[id] = dth;
                if (a.out_ph) a.out_ph[id] = dph;
            } else if constexpr (STAGE == 1) {
                if constexpr (INC) {
                    a.k1_th[id] = dth;
                    a.ua_th[id] = sc[0] * dth;
                    a.k1_ph[id] = dph;
                    a.ua_ph[id] = sc[0] * dph;
                } else {
                    if constexpr (HAS_TH) { a.k1_th[id] = dth; a.ua_th[id] = FMA(sc[0], dth, thc); }
                    if constexpr (HAS_PH) { a.k1_ph[id] = dph; a.ua_ph[id] = FMA(sc[0], dph, phc); }
                }
                if constexpr (HAS_PH) {
                    // ice and cell counts of the pore bulk (I_W > 1/2) for the equilibrium test
                    bool in_pore;
                    if constexpr (STATIC) in_pore = ge_nonneg(sW, K.wa_half) && sW != K.wa_half;
                    else in_pore = lt_nonneg(Gc, K.g_pore);
                    if (in_pore) {
                        ++pcount;
                        if (!le_nonneg(phc, T(0.5))) ++icount;
                        const unsigned long long rb = abs_bits(dph);
                        rbits = rb > rbits ? rb : rbits;
                    }
                }
            } else if constexpr (STAGE == 2) {
                if constexpr (F32) {
                    if constexpr (HAS_TH) a.ub_th[id] = FMA(sc[1], dth - k1t, bth);
                    if constexpr (HAS_PH) a.ub_ph[id] = FMA(sc[1], dph - k1p, bph);
                } else {
                    if constexpr (HAS_TH) a.ub_th[id] = FMA(sc[1], k1t + dth, y_t);
                    if constexpr (HAS_PH) a.ub_ph[id] = FMA(sc[1], k1p + dph, y_p);
                }
            } else if constexpr (STAGE == 3) {
                if constexpr (F32) {
                    if constexpr (HAS_TH) { a.k3_th[id] = dth; a.ua_th[id] = FMA(sc[3], dth, FMA(-sc[8], k1t, ua_t)); }
                    if constexpr (HAS_PH) { a.k3_ph[id] = dph; a.ua_ph[id] = FMA(sc[3], dph, FMA(-sc[8], k1p, ua_p)); }
                } else {
                    if constexpr (HAS_TH) { a.k3_th[id] = dth; a.ua_th[id] = FMA(sc[3], dth, FMA(sc[2], k1t, y_t)); }
                    if constexpr (HAS_PH) { a.k3_ph[id] = dph; a.ua_ph[id] = FMA(sc[3], dph, FMA(sc[2], k1p, y_p)); }
                }
            } else if constexpr (STAGE == 4) {
                if constexpr (F32) {
                    if constexpr (HAS_TH) { a.k4_th[id] = dth; a.ub_th[id] = FMA(sc[6], dth, FMA(-sc[9], k3t, FMA(sc[3], k1t, bth))); }
                    if constexpr (HAS_PH) { a.k4_ph[id] = dph; a.ub_ph[id] = FMA(sc[6], dph, FMA(-sc[9], k3p, FMA(sc[3], k1p, bph))); }
                } else {
                    if constexpr (HAS_TH) { a.k4_th[id] = dth; a.ub_th[id] = FMA(sc[6], dth, FMA(-sc[5], k3t, FMA(sc[4], k1t, y_t))); }
                    if constexpr (HAS_PH) { a.k4_ph[id] = dph; a.ub_ph[id] = FMA(sc[6], dph, FMA(-sc[5], k3p, FMA(sc[4], k1p, y_p))); }
                }
            } else {  // STAGE 5
                // |2k1 - 9k3 + 8k4 - k5| here; the factor dt/30 is applied to the block maximum
                // (rounding is monotone, so max(dt/30 |x|) = dt/30 max |x| exactly)
                if constexpr (HAS_TH) {
                    if constexpr (F32) {
                        const double yn = y_t64 + widen(sc[1] * (k1t + FMA(T(4), k4t, dth)));
                        a.yo_th[cur ^ 1][id] = yn;
                        if constexpr (INC) a.y32_th[cur ^ 1][id] = narrow(yn);
                    }
                    else a.yo_th[cur ^ 1][id] = FMA(sc[1], k1t + FMA(T(4), k4t, dth), y_t64);
                    const unsigned long long eb = abs_bits(FMA(T(2), k1t, FMA(T(-9), k3t, FMA(T(8), k4t, -dth))));
                    ebits = eb > ebits ? eb : ebits;
                }
                if constexpr (HAS_PH) {
                    if constexpr (F32) {
                        const double yn = y_p64 + widen(sc[1] * (k1p + FMA(T(4), k4p, dph)));
                        a.yo_ph[cur ^ 1][id] = yn;
                        if constexpr (INC) a.y32_ph[cur ^ 1][id] = narrow(yn);
                    }
                    else a.yo_ph[cur ^ 1][id] = FMA(sc[1], k1p + FMA(T(4), k4p, dph), y_p64);
                    const unsigned long long eb = abs_bits(FMA(T(2), k1p, FMA(T(-9), k3p, FMA(T(8), k4p, -dph))));
                    ebits = eb > ebits ? eb : ebits;
                }
            }
        }

        // 3. finish plane k+2 into the ring slot of plane k-1; rotate the own column
        const int b2 = (b + 2) % 3;
        {
            T cth, cph, lam2, tg2 = T(0);
            cvt(rth, rph, cth, cph);
            finish(cth, cph, rG, rB, lam2, tg2, rdp);
            put(b2, ty + 1, tx + 1, cth, cph, lam2, rdt, rdp);
            thm = thc; phm = phc; lamm = lamc; tgm = tgc; dtm = dtc; dpm = dpc;
            thc = thp; phc = php; lamc = lamp; Gc = Gp; tgc = tgp; dtc = dtp; dpc = dpp;
            thp = cth; php = cph; lamp = lam2; Gp = rG; tgp = tg2; dtp = rdt; dpp = rdp;
        }
        if (hal) {
            T h_th, h_ph, h_lam, h_tg;
            cvt(qth, qph, h_th, h_ph);
            finish(h_th, h_ph, qG, qB, h_lam, h_tg, qdp);
            put(b2, hy + 1, hx + 1, h_th, h_ph, h_lam, qdt, qdp);
        }
        b = (b + 1) % 3;
        __syncthreads();
    }

    publish_block<STAGE, HAS_PH, F32, BY>(ctrl, ebits, icount, pcount, rbits);
    __syncthreads();  // the block may start another tile: shared memory is reused
    (void)tgm;
}

template <int MODEL, int RX, typename T, typename TIN, int STAGE, int BY>
__global__ void __launch_bounds__(TX * BY)
stage_kernel(const StageArgs<T> a) {
    stage_tile<MODEL, RX, T, TIN, STAGE, BY>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Binary64 form: resident blocks per SM the register bound is set for: 24 warps for blocks of 32 x 4 and
// 32 x 8 (at most 85 registers per thread, some spilled; measured over the five stages at 256^3: 2.3 %
// faster than 16 warps at 128 registers with 32 x 4, 3.5 % with 32 x 8; 28 and 32 warps slower), one
// block of 32 x 16 (16 warps at 128 registers; one 8-warp block at 136 registers was slower).  The
// binary32 kernels keep the compiler's own register choice (an explicit bound, even of one block, made
// it take more registers).
constexpr int f64_min_blocks(int by) { return by <= 8 ? 24 / by : 1; }

template <int MODEL, int RX, typename T, typename TIN, int STAGE, int BY>
__global__ void __launch_bounds__(TX * BY, f64_min_blocks(BY))
stage_kernel_r128(const StageArgs<T> a) {
    stage_tile<MODEL, RX, T, TIN, STAGE, BY>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Batched persistent form: a fixed grid of blocks walks, in order, the tiles of the instances
// listed in the plan (instances that are finished are not listed).
template <int MODEL, int RX, typename T, typename TIN, int STAGE, int BY>
__device__ __forceinline__ void batch_tiles(const StageArgs<T>* __restrict__ args, const BatchPlan* __restrict__ plan,
                                            const int4* __restrict__ tilegrid) {
    const int nt = plan->ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        int s = 0;
        while (t >= plan->tile_start[s + 1]) ++s;
        const int inst = plan->inst[s];
        const int local = t - plan->tile_start[s];
        const int4 tg = tilegrid[inst];
        stage_tile<MODEL, RX, T, TIN, STAGE, BY>(args[inst], local % tg.x, (local / tg.x) % tg.y,
                                                  local / (tg.x * tg.y));
    }
}

template <int MODEL, int RX, typename T, typename TIN, int STAGE, int BY>
__global__ void __launch_bounds__(TX * BY)
batch_stage_kernel(const StageArgs<T>* __restrict__ args, const BatchPlan* __restrict__ plan,
                   const int4* __restrict__ tilegrid) {
    batch_tiles<MODEL, RX, T, TIN, STAGE, BY>(args, plan, tilegrid);
}

template <int MODEL, int RX, typename T, typename TIN, int STAGE, int BY>
__global__ void __launch_bounds__(TX * BY, f64_min_blocks(BY))
batch_stage_kernel_r128(const StageArgs<T>* __restrict__ args, const BatchPlan* __restrict__ plan,
                        const int4* __restrict__ tilegrid) {
    batch_tiles<MODEL, RX, T, TIN, STAGE, BY>(args, plan, tilegrid);
}

// ---------------------------------------------------------------- launchers (one per field type)
template <typename T, int MODEL, int RX, int STAGE, int BY>
void launch_one(const StageArgs<T>& a, dim3 grid, cudaStream_t s) {
    using TIN = typename std::conditional<STAGE == 1 && !(std::is_same<T, float>::value && MODEL == M_FULL), double,
                                          T>::type;
    if constexpr (std::is_same<T, double>::value)
        stage_kernel_r128<MODEL, RX, T, TIN, STAGE, BY><<<grid, dim3(TX, BY), 0, s>>>(a);
    else
        stage_kernel<MODEL, RX, T, TIN, STAGE, BY><<<grid, dim3(TX, BY), 0, s>>>(a);
}

template <typename T, int MODEL, int RX, int BY>
cudaError_t launch_by(int stage, const StageArgs<T>& a, cudaStream_t s) {
    const int n1 = a.cf.n1, n2 = a.cf.n2, n3 = a.cf.n3;
    dim3 grid((n1 + TX - 1) / TX, (n2 + BY - 1) / BY, (n3 + a.zc - 1) / a.zc);
    switch (stage) {
        case 0: launch_one<T, MODEL, RX, 0, BY>(a, grid, s); break;
        case 1: launch_one<T, MODEL, RX, 1, BY>(a, grid, s); break;
        case 2: launch_one<T, MODEL, RX, 2, BY>(a, grid, s); break;
        case 3: launch_one<T, MODEL, RX, 3, BY>(a, grid, s); break;
        case 4: launch_one<T, MODEL, RX, 4, BY>(a, grid, s); break;
        case 5: launch_one<T, MODEL, RX, 5, BY>(a, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

template <typename T, int MODEL, int RX, int STAGE, int BY>
void batch_one(const StageArgs<T>* args, const BatchPlan* plan, const int4* tg, int blocks, cudaStream_t s) {
    using TIN = typename std::conditional<STAGE == 1 && !(std::is_same<T, float>::value && MODEL == M_FULL), double,
                                          T>::type;
    if constexpr (std::is_same<T, double>::value)
        batch_stage_kernel_r128<MODEL, RX, T, TIN, STAGE, BY><<<blocks, dim3(TX, BY), 0, s>>>(args, plan, tg);
    else
        batch_stage_kernel<MODEL, RX, T, TIN, STAGE, BY><<<blocks, dim3(TX, BY), 0, s>>>(args, plan, tg);
}

template <typename T, int MODEL, int RX, int BY>
cudaError_t batch_by(int stage, const StageArgs<T>* args, const BatchPlan* plan, const int4* tg, int blocks,
                     cudaStream_t s) {
    switch (stage) {
        case 1: batch_one<T, MODEL, RX, 1, BY>(args, plan, tg, blocks, s); break;
        case 2: batch_one<T, MODEL, RX, 2, BY>(args, plan, tg, blocks, s); break;
        case 3: batch_one<T, MODEL, RX, 3, BY>(args, plan, tg, blocks, s); break;
        case 4: batch_one<T, MODEL, RX, 4, BY>(args, plan, tg, blocks, s); break;
        case 5: batch_one<T, MODEL, RX, 5, BY>(args, plan, tg, blocks, s); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

// model, reaction term and block height chosen at run time
template <typename T>
cudaError_t launch_stage_t(int model, int rx, int stage, const StageArgs<T>& a, int by, cudaStream_t s) {
    if (a.zc <= 0) return cudaErrorInvalidValue;
    auto m = [&](auto M, auto R) -> cudaError_t {
        constexpr int MO = decltype(M)::value, RO = decltype(R)::value;
        switch (by) {
            case 4: return launch_by<T, MO, RO, 4>(stage, a, s);
            case 8: return launch_by<T, MO, RO, 8>(stage, a, s);
            case 16: return launch_by<T, MO, RO, 16>(stage, a, s);
            default: return cudaErrorInvalidValue;
        }
    };
    using F = std::integral_constant<int, M_FULL>;
    using Tm = std::integral_constant<int, M_TEMP>;
    using Mi = std::integral_constant<int, M_MICRO>;
    using Sg = std::integral_constant<int, R_SIGMA>;
    using Gp = std::integral_constant<int, R_GRADP>;
    if (model == M_FULL) return rx == R_GRADP ? m(F{}, Gp{}) : m(F{}, Sg{});
    if (model == M_TEMP) return m(Tm{}, Sg{});
    if (model == M_MICRO) return rx == R_GRADP ? m(Mi{}, Gp{}) : m(Mi{}, Sg{});
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_batch_stage_t(int model, int rx, int stage, const StageArgs<T>* args, const BatchPlan* plan,
                                 const int4* tg, int by, int blocks, cudaStream_t s) {
    auto m = [&](auto M, auto R) -> cudaError_t {
        constexpr int MO = decltype(M)::value, RO = decltype(R)::value;
        switch (by) {
            case 4: return batch_by<T, MO, RO, 4>(stage, args, plan, tg, blocks, s);
            case 8: return batch_by<T, MO, RO, 8>(stage, args, plan, tg, blocks, s);
            case 16: return batch_by<T, MO, RO, 16>(stage, args, plan, tg, blocks, s);
            default: return cudaErrorInvalidValue;
        }
    };
    using F = std::integral_constant<int, M_FULL>;
    using Tm = std::integral_constant<int, M_TEMP>;
    using Mi = std::integral_constant<int, M_MICRO>;
    using Sg = std::integral_constant<int, R_SIGMA>;
    using Gp = std::integral_constant<int, R_GRADP>;
    if (model == M_FULL) return rx == R_GRADP ? m(F{}, Gp{}) : m(F{}, Sg{});
    if (model == M_TEMP) return m(Tm{}, Sg{});
    if (model == M_MICRO) return rx == R_GRADP ? m(Mi{}, Gp{}) : m(Mi{}, Sg{});
    return cudaErrorInvalidValue;
}

}  // namespace pfgb
