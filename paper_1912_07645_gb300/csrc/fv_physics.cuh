// Device-side physics of the finite-volume step (Sec. 2.1, eq. (2.1)): state conversions,
// per-face reconstruction and numerical fluxes, templated on the arithmetic type R.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "alsv_internal.h"

namespace alsv {

// FP64 evaluates every formula with the same operations in the same order as the plain CPU
// restatement of the scheme (true divisions; the FP64 translation units are compiled without FMA
// contraction), so FP64 runs are reproducible across both. FP32 uses reciprocal multiplications
// and FMA, within its 2e-5 relative L1 budget.
template <class R> struct IsExact { static constexpr bool value = false; };
template <> struct IsExact<double> { static constexpr bool value = true; };

template <class R> __device__ __forceinline__ R rcp(R x) { return R(1) / x; }

// The divergence accumulation acc - dF f and the RK combination a U^n + b (U^(s) + dt L) with a
// fixed rounding in FP32 (explicit fused multiply-adds, which the compiler neither splits nor
// re-associates), so every FP32 schedule that accumulates in the same order is bitwise equal;
// FP64 evaluates them as written (its translation units do not contract).
template <class R> __device__ __forceinline__ R acc_sub(R acc, R dF, R f) {
    if constexpr (IsExact<R>::value) return acc - dF * f;
    else return __fmaf_rn(-dF, f, acc);
}
template <class R> __device__ __forceinline__ R rk_combine(R us, R dt, R L, bool has_un, R ca, R un, R cb) {
    if constexpr (IsExact<R>::value) {
        R o = us + dt * L;
        if (has_un) o = ca * un + cb * o;
        return o;
    } else {
        R o = __fmaf_rn(dt, L, us);
        if (has_un) o = __fmaf_rn(ca, un, __fmul_rn(cb, o));
        return o;
    }
}

// Grid and stage constants in the kernel's precision: FP64 reads the doubles, FP32 the float copies
// made on the host (or by the time control for dt), so no thread converts a double to float.
template <class R> __device__ __forceinline__ R c_gamma(const GridArgs& g) {
    if constexpr (IsExact<R>::value) return g.gamma;
    else return g.gamma_f;
}
template <class R> __device__ __forceinline__ R c_inv_dx(const LevelInfo& L, int k) {
    if constexpr (IsExact<R>::value) return L.inv_dx[k];
    else return L.inv_dx_f[k];
}
template <class R> __device__ __forceinline__ R c_eps(const GridArgs& g, const LevelInfo& L, int k) {
    if constexpr (IsExact<R>::value) return g.weno_eps_dx2 ? L.dx[k] * L.dx[k] : g.weno_eps;
    else return L.eps_f[k];
}
template <class R> __device__ __forceinline__ R c_dt(const StageArgs& p, int s) {
    if constexpr (IsExact<R>::value) return p.dt[s];
    else return p.dt_f[s];
}
template <class R> __device__ __forceinline__ R c_a(const StageArgs& p) {
    if constexpr (IsExact<R>::value) return p.a;
    else return p.a_f;
}
template <class R> __device__ __forceinline__ R c_b(const StageArgs& p) {
    if constexpr (IsExact<R>::value) return p.b;
    else return p.b_f;
}

// FP32 fast forms (MUFU reciprocal / reciprocal square root, about 2 ulp)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// sound speed sqrt(gamma p / rho): FP64 as written; FP32 as (gamma p) * rsqrt(gamma p rho)
template <class R> __device__ __forceinline__ R sound_speed(R gamma, R p, R rho);
template <> __device__ __forceinline__ double sound_speed(double gamma, double p, double rho) {
    return sqrt(gamma * p / rho);
}
template <> __device__ __forceinline__ float sound_speed(float gamma, float p, float rho) {
    const float gp = gamma * p;
    return gp * rsqrt_approx(gp * rho);
}
template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }
// FP64: |x|, max, min as the CPU restatement writes them (ties keep the first argument);
// FP32: the native single-instruction forms (equal values are interchangeable there).
template <class R> __device__ __forceinline__ R fabs_(R x) { return x < R(0) ? -x : x; }
template <class R> __device__ __forceinline__ R fmax_(R a, R b) { return b > a ? b : a; }
template <class R> __device__ __forceinline__ R fmin_(R a, R b) { return b < a ? b : a; }
template <> __device__ __forceinline__ float fabs_(float x) { return fabsf(x); }
template <> __device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
template <> __device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }

// ---------------------------------------------------------------------------------------------
// Ideal gas: p = (gamma - 1) (E - |m|^2 / (2 rho)); E = p / (gamma - 1) + rho |u|^2 / 2.
// Primitive layout: [rho, u_0 .. u_{ND-1}, p].
// ---------------------------------------------------------------------------------------------
template <class R, int ND>
__device__ __forceinline__ void cons_to_prim(const R* U, R* W, R gm1) {
    const R rho = U[0];
    R m2 = U[1] * U[1];
#pragma unroll
    for (int k = 1; k < ND; ++k) m2 = m2 + U[1 + k] * U[1 + k];
    W[0] = rho;
    if constexpr (IsExact<R>::value) {
#pragma unroll
        for (int k = 0; k < ND; ++k) W[1 + k] = U[1 + k] / rho;
        W[ND + 1] = gm1 * (U[ND + 1] - R(0.5) * m2 / rho);
    } else {
        const R inv = rcp_approx(rho);
#pragma unroll
        for (int k = 0; k < ND; ++k) W[1 + k] = U[1 + k] * inv;
        W[ND + 1] = gm1 * (U[ND + 1] - R(0.5) * m2 * inv);
    }
}

// gm1 = gamma - 1 and its reciprocal: FP64 divides by gm1, FP32 multiplies by inv_gm1
template <class R>
__device__ __forceinline__ R div_gm1(R x, R gm1, R inv_gm1) {
    if constexpr (IsExact<R>::value) return x / gm1;
    else return x * inv_gm1;
}

template <class R, int ND>
__device__ __forceinline__ void prim_to_cons(const R* W, R* U, R gm1, R inv_gm1) {
    const R rho = W[0];
    R u2 = W[1] * W[1];
#pragma unroll
    for (int k = 1; k < ND; ++k) u2 = u2 + W[1 + k] * W[1 + k];
    U[0] = rho;
#pragma unroll
    for (int k = 0; k < ND; ++k) U[1 + k] = rho * W[1 + k];
    U[ND + 1] = div_gm1(W[ND + 1], gm1, inv_gm1) + R(0.5) * rho * u2;
}

// ---------------------------------------------------------------------------------------------
// Reconstruction (Sec. 2.1: WENO after Shu 1999; MC-limited linear; piecewise constant).
// face_r: value at i+1/2 from cell i; face_l: value at i-1/2 from cell i. Stencil (wm, w0, wp).
// ---------------------------------------------------------------------------------------------
template <class R> __device__ __forceinline__ R minmod3(R a, R b, R c) {
    if (a > R(0) && b > R(0) && c > R(0)) return fmin_(fmin_(a, b), c);
    if (a < R(0) && b < R(0) && c < R(0)) return fmax_(fmax_(a, b), c);
    return R(0);
}
// FP32: the same value from the extremes (all positive <=> min > 0; all negative <=> max < 0)
template <> __device__ __forceinline__ float minmod3(float a, float b, float c) {
    const float mn = fminf(fminf(a, b), c), mx = fmaxf(fmaxf(a, b), c);
    return mn > 0.0f ? mn : (mx < 0.0f ? mx : 0.0f);
}

template <class R> __device__ __forceinline__ R mc_slope(R wm, R w0, R wp) {
    const R dm = w0 - wm, dp = wp - w0;
    return minmod3(R(2) * dm, R(0.5) * (dm + dp), R(2) * dp);
}

// Jiang-Shu WENO3 face value from candidates p0 (stencil {far, 0}) and p1 ({0, near}) with
// linear weights 1/3, 2/3 and alpha_r = d_r / (eps + beta_r)^2. FP64 evaluates
// (alpha_0 p0 + alpha_1 p1) / (alpha_0 + alpha_1) as written; FP32 uses the equivalent one-division
// form (d0 q1 p0 + d1 q0 p1) / (d0 q1 + d1 q0) with q_r = (eps + beta_r)^2.
template <class R> __device__ __forceinline__ R weno3_face(R wfar, R w0, R wnear, R eps) {
    const R p0 = R(-0.5) * wfar + R(1.5) * w0;
    const R p1 = R(0.5) * w0 + R(0.5) * wnear;
    const R b0 = (w0 - wfar) * (w0 - wfar);
    const R b1 = (wnear - w0) * (wnear - w0);
    const R e0 = eps + b0, e1 = eps + b1;
    const R q0 = e0 * e0, q1 = e1 * e1;
    if constexpr (IsExact<R>::value) {
        const R a0 = R(1.0 / 3.0) / q0;
        const R a1 = R(2.0 / 3.0) / q1;
        return (a0 * p0 + a1 * p1) / (a0 + a1);
    } else {
        const R t0 = R(2) * q0;
        return (q1 * p0 + t0 * p1) * rcp_approx(q1 + t0);
    }
}

// Both face states of interface i+1/2 from (w_{i-1}, w_i, w_{i+1}, w_{i+2}): fr = right face of
// cell i, fl = left face of cell i+1. The two share p1 = (w_i + w_{i+1})/2 and the smoothness
// indicator of (w_i, w_{i+1}); FP32 form (q1 p0 + 2 q0 p1) / (q1 + 2 q0), q = (eps + beta)^2.
__device__ __forceinline__ void weno3_pair(float wm, float w0, float w1, float w2, float eps, float& fr, float& fl) {
    const float p1 = 0.5f * (w0 + w1);
    const float d1 = w1 - w0;
    const float e1 = eps + d1 * d1;
    const float q1 = e1 * e1;
    const float dm = w0 - wm, dp = w1 - w2;
    const float em = eps + dm * dm, ep = eps + dp * dp;
    const float tm = 2.0f * (em * em), tp = 2.0f * (ep * ep);
    const float p0r = 1.5f * w0 - 0.5f * wm;
    const float p0l = 1.5f * w1 - 0.5f * w2;
    fr = (q1 * p0r + tm * p1) * rcp_approx(q1 + tm);
    fl = (q1 * p0l + tp * p1) * rcp_approx(q1 + tp);
}

// The same for two variables at once with packed FP32x2 arithmetic (one instruction per pair).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ void weno3_pair2(float2 wm, float2 w0, float2 w1, float2 w2, float2 e, float2& fr,
                                            float2& fl) {
    const float2 half = f2(0.5f), m1 = f2(-1.0f), two = f2(2.0f);
    const float2 p1 = __fmul2_rn(half, __fadd2_rn(w0, w1));
    const float2 d1 = __ffma2_rn(w0, m1, w1);
    const float2 e1 = __ffma2_rn(d1, d1, e);
    const float2 q1 = __fmul2_rn(e1, e1);
    const float2 dm = __ffma2_rn(wm, m1, w0);
    const float2 dp = __ffma2_rn(w2, m1, w1);
    const float2 em = __ffma2_rn(dm, dm, e);
    const float2 ep = __ffma2_rn(dp, dp, e);
    const float2 sm = __fmul2_rn(em, em), sp = __fmul2_rn(ep, ep);
    const float2 p0r = __ffma2_rn(f2(1.5f), w0, __fmul2_rn(f2(-0.5f), wm));
    const float2 p0l = __ffma2_rn(f2(1.5f), w1, __fmul2_rn(f2(-0.5f), w2));
    const float2 nr = __ffma2_rn(two, __fmul2_rn(sm, p1), __fmul2_rn(q1, p0r));
    const float2 nl = __ffma2_rn(two, __fmul2_rn(sp, p1), __fmul2_rn(q1, p0l));
    const float2 dr = __ffma2_rn(two, sm, q1);
    const float2 dl = __ffma2_rn(two, sp, q1);
    fr = __fmul2_rn(nr, make_float2(rcp_approx(dr.x), rcp_approx(dr.y)));
    fl = __fmul2_rn(nl, make_float2(rcp_approx(dl.x), rcp_approx(dl.y)));
}

template <class R, int RECON>
__device__ __forceinline__ void recon_faces(R wm, R w0, R wp, R eps, R& fl, R& fr) {
    if (RECON == REC_PC) {
        fl = w0;
        fr = w0;
    } else if (RECON == REC_MC) {
        const R s = mc_slope(wm, w0, wp);
        fl = w0 - R(0.5) * s;
        fr = w0 + R(0.5) * s;
    } else {
        fr = weno3_face(wm, w0, wp, eps);
        fl = weno3_face(wp, w0, wm, eps);
    }
}

// second-order ENO (Sec. 2.1 names ENO): the one-sided difference of smaller magnitude (ties: the
// backward one), i.e. the smoother of the two linear candidates
template <class R> __device__ __forceinline__ R eno2_slope(R wm, R w0, R wp) {
    const R dm = w0 - wm, dp = wp - w0;
    return fabs_(dp) < fabs_(dm) ? dp : dm;
}

template <class R, int RECON> __device__ __forceinline__ R recon_right(R wm, R w0, R wp, R eps) {
    if (RECON == REC_PC) return w0;
    if (RECON == REC_MC) return w0 + R(0.5) * mc_slope(wm, w0, wp);
    if (RECON == REC_ENO2) return w0 + R(0.5) * eno2_slope(wm, w0, wp);
    return weno3_face(wm, w0, wp, eps);
}
template <class R, int RECON> __device__ __forceinline__ R recon_left(R wm, R w0, R wp, R eps) {
    if (RECON == REC_PC) return w0;
    if (RECON == REC_MC) return w0 - R(0.5) * mc_slope(wm, w0, wp);
    if (RECON == REC_ENO2) return w0 - R(0.5) * eno2_slope(wm, w0, wp);
    return weno3_face(wp, w0, wm, eps);
}

// ---------------------------------------------------------------------------------------------
// Numerical fluxes through a face normal to direction D (Sec. 2.1: HLLC, Rusanov; plus HLL).
// Inputs are primitive face states; output is the conserved flux. Wave speeds (Davis):
// S_L = min(uL - cL, uR - cR), S_R = max(uL + cL, uR + cR); Rusanov a = max(|uL|+cL, |uR|+cR).
// ---------------------------------------------------------------------------------------------
// FP32 HLLC with the same case rules: the upwind side K is L when S_L >= 0 or S* >= 0, else R;
// only K's physical flux and conserved state are formed, and the star state uses one reciprocal:
// U*_E = ((S_K - u_K) E_K + (S* - u_K) p_K) / (S_K - S*) + fac (S* - u_K) S*,
// fac = rho_K (S_K - u_K) / (S_K - S*) (algebraically equal to the textbook form).
template <class R, int ND, int D>
__device__ __forceinline__ void hllc_fast(const R* WL, const R* WR, R* F, R gamma, R gm1, R inv_gm1) {
    constexpr int NV = ND + 2, IP = ND + 1;
    const R rL = WL[0], rR = WR[0], uL = WL[1 + D], uR = WR[1 + D], pL = WL[IP], pR = WR[IP];
    const R cL = sound_speed<R>(gamma, pL, rL), cR = sound_speed<R>(gamma, pR, rR);
    const R SL = fmin_(uL - cL, uR - cR), SR = fmax_(uL + cL, uR + cR);
    const R mL = rL * (SL - uL), mR = rR * (SR - uR);
    const R Ss = (pR - pL + uL * mL - uR * mR) * rcp_approx(mL - mR);
    const bool leftK = (SL >= R(0)) || (Ss >= R(0));
    const bool star = !(SL >= R(0)) && (leftK || (SR > R(0)));
    R WK[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) WK[v] = leftK ? WL[v] : WR[v];
    const R SK = leftK ? SL : SR;
    const R rK = WK[0], uK = WK[1 + D], pK = WK[IP];
    R UK[NV], FK[NV];
    prim_to_cons<R, ND>(WK, UK, gm1, inv_gm1);
#pragma unroll
    for (int v = 0; v < NV; ++v) FK[v] = UK[v] * uK;
    FK[1 + D] = FK[1 + D] + pK;
    FK[IP] = uK * (UK[IP] + pK);
    const R A = SK - uK;
    const R invB = rcp_approx(SK - Ss);
    const R fac = rK * A * invB;
    const R dS = Ss - uK;
    R Us[NV];
    Us[0] = fac;
#pragma unroll
    for (int j = 0; j < ND; ++j) Us[1 + j] = fac * WK[1 + j];
    Us[1 + D] = fac * Ss;
    Us[IP] = (A * UK[IP] + dS * pK) * invB + fac * dS * Ss;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = star ? FK[v] + SK * (Us[v] - UK[v]) : FK[v];
}

// Harten's smoothing of |lambda| on an acoustic field, width from the Harten-Hyman estimate
// delta = max(0, lambda - lambda_L, lambda_R - lambda) of the one-sided eigenvalues.
template <class R> __device__ __forceinline__ R harten_abs(R lam, R lamL, R lamR) {
    const R del = fmax_(R(0), fmax_(lam - lamL, lamR - lam));
    if (fabs_(lam) < del) return (lam * lam + del * del) / (R(2) * del);
    return fabs_(lam);
}

// Roe's flux (Sec. 2.1 names it) with the entropy fix above on the two acoustic fields: F = (F_L +
// F_R)/2 - (1/2) sum |lambda| alpha r over the waves of the Roe-averaged Jacobian along D (acoustic
// u_n -/+ a, entropy and shear waves at u_n); Roe averages weighted by sqrt(rho). Operations in
// the same order as the CPU restatement of the scheme.
template <class R, int ND, int D>
__device__ __forceinline__ void roe_flux(const R* WL, const R* WR, R* F, R gamma, R gm1, R inv_gm1) {
    constexpr int NV = ND + 2, IP = ND + 1;
    R UL[NV], UR[NV], FL[NV], FR[NV];
    prim_to_cons<R, ND>(WL, UL, gm1, inv_gm1);
    prim_to_cons<R, ND>(WR, UR, gm1, inv_gm1);
#pragma unroll
    for (int v = 0; v < NV; ++v) { FL[v] = UL[v] * WL[1 + D]; FR[v] = UR[v] * WR[1 + D]; }
    FL[1 + D] = FL[1 + D] + WL[IP];
    FR[1 + D] = FR[1 + D] + WR[IP];
    FL[IP] = WL[1 + D] * (UL[IP] + WL[IP]);
    FR[IP] = WR[1 + D] * (UR[IP] + WR[IP]);
    const R rL = WL[0], rR = WR[0], pL = WL[IP], pR = WR[IP];
    const R sL = sqrt(rL), sR = sqrt(rR);
    const R HL = (UL[IP] + pL) / rL, HR = (UR[IP] + pR) / rR;
    R ut[ND];
    R q2 = R(0);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        ut[j] = (sL * WL[1 + j] + sR * WR[1 + j]) / (sL + sR);
        q2 = q2 + ut[j] * ut[j];
    }
    const R H = (sL * HL + sR * HR) / (sL + sR);
    const R a2 = gm1 * (H - R(0.5) * q2);
    const R a = sqrt(a2);
    const R rt = sL * sR;
    const R un = ut[D];
    const R dr = rR - rL, dp = pR - pL, dun = WR[1 + D] - WL[1 + D];
    const R al1 = (dp - rt * a * dun) / (R(2) * a2);
    const R al3 = (dp + rt * a * dun) / (R(2) * a2);
    const R al2 = dr - dp / a2;
    const R cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
    const R l1 = harten_abs(un - a, WL[1 + D] - cL, WR[1 + D] - cR);
    const R l3 = harten_abs(un + a, WL[1 + D] + cL, WR[1 + D] + cR);
    const R l2 = fabs_(un);
    R Dv[NV];
    Dv[0] = l1 * al1 + l2 * al2 + l3 * al3;
#pragma unroll
    for (int j = 0; j < ND; ++j) Dv[1 + j] = l1 * al1 * ut[j] + l2 * al2 * ut[j] + l3 * al3 * ut[j];
    Dv[1 + D] = Dv[1 + D] - l1 * al1 * a + l3 * al3 * a;
    Dv[IP] = l1 * al1 * (H - un * a) + l2 * al2 * (R(0.5) * q2) + l3 * al3 * (H + un * a);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        if (j == D) continue;
        const R alt = rt * (WR[1 + j] - WL[1 + j]);
        Dv[1 + j] = Dv[1 + j] + l2 * alt;
        Dv[IP] = Dv[IP] + l2 * alt * ut[j];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * Dv[v];
}

// Godunov's flux (Sec. 2.1 names it): the physical flux of the exact Riemann solution at x/t = 0.
// The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0 (shock: Rankine-Hugoniot branch,
// rarefaction: isentropic branch) by Newton's method from the linearised guess, to a relative step
// of 1e-15 (FP64) or 1e-7 (FP32), at most 60 steps; then the solution is sampled at x/t = 0 and the
// tangential velocities come from the side of the contact it lies on.
template <class R> __device__ __forceinline__ R pressure_branch(R g, R p, R rK, R pK, R cK, R& df) {
    if (p > pK) {
        const R A = R(2) / ((g + R(1)) * rK);
        const R B = (g - R(1)) / (g + R(1)) * pK;
        const R s = sqrt(A / (p + B));
        df = s * (R(1) - (p - pK) / (R(2) * (B + p)));
        return (p - pK) * s;
    }
    const R q = p / pK;
    df = pow(q, -(g + R(1)) / (R(2) * g)) / (rK * cK);
    return R(2) * cK / (g - R(1)) * (pow(q, (g - R(1)) / (R(2) * g)) - R(1));
}
template <class R, int ND, int D>
__device__ __forceinline__ void godunov_flux(const R* WL, const R* WR, R* F, R gamma, R gm1, R inv_gm1) {
    constexpr int IP = ND + 1, NV = ND + 2;
    const R g = gamma;
    const R rL = WL[0], uL = WL[1 + D], pL = WL[IP], rR = WR[0], uR = WR[1 + D], pR = WR[IP];
    const R cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    const R ppv = R(0.5) * (pL + pR) - R(0.125) * (uR - uL) * (rL + rR) * (cL + cR);
    const R pfloor = R(1e-10) * fmin_(pL, pR);
    R p = fmax_(ppv, pfloor);
    const R tol = IsExact<R>::value ? R(1e-15) : R(1e-7);
    R dL, dR;
#pragma unroll 1
    for (int it = 0; it < 60; ++it) {
        const R fL = pressure_branch(g, p, rL, pL, cL, dL);
        const R fR = pressure_branch(g, p, rR, pR, cR, dR);
        R pn = p - (fL + fR + uR - uL) / (dL + dR);
        if (pn <= R(0)) pn = R(0.5) * p;
        const R step = pn - p;
        p = pn;
        if (fabs_(step) <= tol * p) break;
    }
    const R fL = pressure_branch(g, p, rL, pL, cL, dL);
    const R fR = pressure_branch(g, p, rR, pR, cR, dR);
    const R us = R(0.5) * (uL + uR) + R(0.5) * (fR - fL);
    const R gr = (g - R(1)) / (g + R(1));
    const bool left = us >= R(0);
    R r0, u0, p0;
    if (left) {
        if (p > pL) {
            const R SL = uL - cL * sqrt((g + R(1)) / (R(2) * g) * p / pL + (g - R(1)) / (R(2) * g));
            if (SL >= R(0)) { r0 = rL; u0 = uL; p0 = pL; }
            else { r0 = rL * (p / pL + gr) / (gr * p / pL + R(1)); u0 = us; p0 = p; }
        } else if (uL - cL >= R(0)) {
            r0 = rL; u0 = uL; p0 = pL;
        } else if (us - cL * pow(p / pL, (g - R(1)) / (R(2) * g)) < R(0)) {
            r0 = rL * pow(p / pL, R(1) / g); u0 = us; p0 = p;
        } else {
            const R c = R(2) / (g + R(1)) * (cL + R(0.5) * (g - R(1)) * uL);
            u0 = c;
            r0 = rL * pow(c / cL, R(2) / (g - R(1)));
            p0 = pL * pow(c / cL, R(2) * g / (g - R(1)));
        }
    } else {
        if (p > pR) {
            const R SR = uR + cR * sqrt((g + R(1)) / (R(2) * g) * p / pR + (g - R(1)) / (R(2) * g));
            if (SR <= R(0)) { r0 = rR; u0 = uR; p0 = pR; }
            else { r0 = rR * (p / pR + gr) / (gr * p / pR + R(1)); u0 = us; p0 = p; }
        } else if (uR + cR <= R(0)) {
            r0 = rR; u0 = uR; p0 = pR;
        } else if (us + cR * pow(p / pR, (g - R(1)) / (R(2) * g)) > R(0)) {
            r0 = rR * pow(p / pR, R(1) / g); u0 = us; p0 = p;
        } else {
            const R c = R(2) / (g + R(1)) * (cR - R(0.5) * (g - R(1)) * uR);
            u0 = -c;
            r0 = rR * pow(c / cR, R(2) / (g - R(1)));
            p0 = pR * pow(c / cR, R(2) * g / (g - R(1)));
        }
    }
    R W[NV], U[NV];
#pragma unroll
    for (int j = 0; j < ND; ++j) W[1 + j] = left ? WL[1 + j] : WR[1 + j];
    W[0] = r0;
    W[1 + D] = u0;
    W[IP] = p0;
    prim_to_cons<R, ND>(W, U, gm1, inv_gm1);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = U[v] * u0;
    F[1 + D] = F[1 + D] + p0;
    F[IP] = u0 * (U[IP] + p0);
}

// Logarithmic mean (a - b)/(ln a - ln b); for nearly equal arguments the series of artanh(f)/f,
// f = (a - b)/(a + b), to f^8 when f^2 < 1e-4.
template <class R> __device__ __forceinline__ R log_mean(R a, R b) {
    const R f = (a - b) / (a + b);
    const R u = f * f;
    if (u < R(1e-4)) {
        const R s = R(1) + u * (R(1.0 / 3.0) + u * (R(1.0 / 5.0) + u * (R(1.0 / 7.0) + u * R(1.0 / 9.0))));
        return (a + b) / (R(2) * s);
    }
    return (a - b) / log(a / b);
}

// Two-point entropy-conservative flux for the entropy -rho s/(gamma-1) (Ismail-Roe): satisfies
// Tadmor's condition (v_R - v_L) . F = psi_R - psi_L. The fourth-order entropy-conservative flux
// of LeFloch-Mercier-Rohde combines three of them over four cells (in the stage kernels).
template <class R, int ND, int D>
__device__ __forceinline__ void ec_flux(const R* WL, const R* WR, R* F, R gamma) {
    constexpr int IP = ND + 1;
    const R g = gamma;
    const R z1L = sqrt(WL[0] / WL[IP]), z1R = sqrt(WR[0] / WR[IP]);
    const R z3L = sqrt(WL[0] * WL[IP]), z3R = sqrt(WR[0] * WR[IP]);
    const R z1m = R(0.5) * (z1L + z1R), z3m = R(0.5) * (z3L + z3R);
    const R z1l = log_mean(z1L, z1R), z3l = log_mean(z3L, z3R);
    const R rho = z1m * z3l;
    R u[ND];
    R q2 = R(0);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        u[j] = R(0.5) * (z1L * WL[1 + j] + z1R * WR[1 + j]) / z1m;
        q2 = q2 + u[j] * u[j];
    }
    const R p1 = z3m / z1m;
    const R p2 = (g + R(1)) / (R(2) * g) * z3l / z1l + (g - R(1)) / (R(2) * g) * z3m / z1m;
    const R H = g * p2 / ((g - R(1)) * rho) + R(0.5) * q2;
    const R mf = rho * u[D];
    F[0] = mf;
#pragma unroll
    for (int j = 0; j < ND; ++j) F[1 + j] = mf * u[j];
    F[1 + D] = F[1 + D] + p1;
    F[IP] = mf * H;
}

// Entropy variables of the entropy -rho s/(gamma-1), s = ln p - gamma ln rho, from a primitive
// state: ((gamma - s)/(gamma - 1) - rho |u|^2/(2p), rho u/p, -rho/p).
template <class R, int ND>
__device__ __forceinline__ void entropy_vars(const R* W, R* v, R gamma) {
    constexpr int IP = ND + 1;
    const R s = log(W[IP]) - gamma * log(W[0]);
    const R beta = W[0] / W[IP];
    R q2 = R(0);
#pragma unroll
    for (int j = 0; j < ND; ++j) q2 = q2 + W[1 + j] * W[1 + j];
    v[0] = (gamma - s) / (gamma - R(1)) - R(0.5) * beta * q2;
#pragma unroll
    for (int j = 0; j < ND; ++j) v[1 + j] = beta * W[1 + j];
    v[IP] = -beta;
}

// Jump <<w>> = w_{i+1}^- - w_i^+ of the second-order ENO faces of one component at interface
// i+1/2 from the values at cells i-1 .. i+2 (per face the one-sided difference of smaller
// magnitude, ties to the backward one). It has the sign of w_{i+1} - w_i (ENO's sign property).
template <class R>
__device__ __forceinline__ R eno2_jump(R w0, R w1, R w2, R w3) {
    const R dm = w1 - w0, d1 = w2 - w1, d2 = w3 - w2;
    const R si = fabs_(d1) < fabs_(dm) ? d1 : dm;
    const R sj = fabs_(d2) < fabs_(d1) ? d2 : d1;
    return (w2 - R(0.5) * sj) - (w1 + R(0.5) * si);
}

// TECNO2 flux along D from the primitive states of cells i-1 .. i+2 (Fjordholm-Mishra-Tadmor's
// entropy-stable ENO scheme, second order): F = F_ec(W_i, W_{i+1}) - 1/2 Rs Lambda <<w>>, where Rs
// holds the eigenvectors of the flux Jacobian scaled so that Rs Rs^T = dU/dv (acoustic columns by
// sqrt(rho/(2 gamma)), the entropy column by sqrt((gamma-1) rho/gamma), shear columns by sqrt(p)),
// Rs and Lambda = |eigenvalues| at the arithmetic mean of the two cells' rho, u, p, w_j = Rs^T v_j
// the scaled entropy variables and <<w>> their ENO2 jump. The sum over components runs in the
// order of the column layout (u - c, entropy, shear in increasing direction, u + c).
template <class R, int ND, int D>
__device__ __forceinline__ void tecno2_flux(const R* W0, const R* W1, const R* W2, const R* W3, R* F, R gamma) {
    constexpr int NV = ND + 2, IP = ND + 1;
    ec_flux<R, ND, D>(W1, W2, F, gamma);
    const R g = gamma;
    const R r = R(0.5) * (W1[0] + W2[0]), p = R(0.5) * (W1[IP] + W2[IP]);
    R u[ND];
    R q2 = R(0);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        u[j] = R(0.5) * (W1[1 + j] + W2[1 + j]);
        q2 = q2 + u[j] * u[j];
    }
    const R c = sqrt(g * p / r);
    const R H = c * c / (g - R(1)) + R(0.5) * q2;
    const R un = u[D];
    const R sac = sqrt(r / (R(2) * g)), sen = sqrt((g - R(1)) * r / g), ssh = sqrt(p);
    R Rs[NV][NV], lam[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = 0; b < NV; ++b) Rs[a][b] = R(0);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int col = side == 0 ? 0 : NV - 1;
        const R sg = side == 0 ? R(-1) : R(1);
        Rs[0][col] = sac;
#pragma unroll
        for (int j = 0; j < ND; ++j) Rs[1 + j][col] = sac * u[j];
        Rs[1 + D][col] = sac * (un + sg * c);
        Rs[IP][col] = sac * (H + sg * un * c);
        lam[col] = fabs_(un + sg * c);
    }
    Rs[0][1] = sen;
#pragma unroll
    for (int j = 0; j < ND; ++j) Rs[1 + j][1] = sen * u[j];
    Rs[IP][1] = sen * R(0.5) * q2;
    lam[1] = fabs_(un);
    {
        int col = 2;
#pragma unroll
        for (int t = 0; t < ND; ++t) {
            if (t == D) continue;
            Rs[1 + t][col] = ssh;
            Rs[IP][col] = ssh * u[t];
            lam[col] = fabs_(un);
            ++col;
        }
    }
    const R* Wc[4] = {W0, W1, W2, W3};
    R w[4][NV];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        R v[NV];
        entropy_vars<R, ND>(Wc[j], v, g);
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            R acc = R(0);
#pragma unroll
            for (int q = 0; q < NV; ++q) acc = acc + Rs[q][m] * v[q];
            w[j][m] = acc;
        }
    }
    R dl[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) dl[m] = lam[m] * eno2_jump<R>(w[0][m], w[1][m], w[2][m], w[3][m]);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        R acc = R(0);
#pragma unroll
        for (int m = 0; m < NV; ++m) acc = acc + Rs[q][m] * dl[m];
        F[q] = F[q] - R(0.5) * acc;
    }
}

// TECNO2 for Burgers (entropy u^2/2): v = u, Rs = 1, Lambda = max(|u_i|, |u_{i+1}|).
template <class R>
__device__ __forceinline__ R tecno2_burgers(R u0, R u1, R u2, R u3) {
    const R Fec = (u1 * u1 + u1 * u2 + u2 * u2) / R(6);
    const R lam = fmax_(fabs_(u1), fabs_(u2));
    return Fec - R(0.5) * (R(1) * (lam * eno2_jump<R>(u0, u1, u2, u3)));
}

template <class R, int ND, int D, int FLUX>
__device__ __forceinline__ void euler_flux(const R* WL, const R* WR, R* F, R gamma, R gm1, R inv_gm1) {
    if constexpr (FLUX == FLX_ROE) {
        roe_flux<R, ND, D>(WL, WR, F, gamma, gm1, inv_gm1);
        return;
    }
    if constexpr (FLUX == FLX_GODUNOV) {
        godunov_flux<R, ND, D>(WL, WR, F, gamma, gm1, inv_gm1);
        return;
    }
    if constexpr (FLUX == FLX_EC || FLUX == FLX_EC4) {
        ec_flux<R, ND, D>(WL, WR, F, gamma);
        return;
    }
    if constexpr (FLUX == FLX_HLLC && !IsExact<R>::value) {
        hllc_fast<R, ND, D>(WL, WR, F, gamma, gm1, inv_gm1);
        return;
    }
    constexpr int NV = ND + 2, IP = ND + 1;
    R UL[NV], UR[NV], FL[NV], FR[NV];
    prim_to_cons<R, ND>(WL, UL, gm1, inv_gm1);
    prim_to_cons<R, ND>(WR, UR, gm1, inv_gm1);
    const R rL = WL[0], rR = WR[0], uL = WL[1 + D], uR = WR[1 + D], pL = WL[IP], pR = WR[IP];
    // physical fluxes
#pragma unroll
    for (int v = 0; v < NV; ++v) { FL[v] = UL[v] * uL; FR[v] = UR[v] * uR; }
    FL[1 + D] = FL[1 + D] + pL;
    FR[1 + D] = FR[1 + D] + pR;
    FL[IP] = uL * (UL[IP] + pL);
    FR[IP] = uR * (UR[IP] + pR);
    const R cL = sound_speed<R>(gamma, pL, rL);
    const R cR = sound_speed<R>(gamma, pR, rR);
    if (FLUX == FLX_RUSANOV) {
        const R a = fmax_(fabs_(uL) + cL, fabs_(uR) + cR);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * a * (UR[v] - UL[v]);
        return;
    }
    const R SL = fmin_(uL - cL, uR - cR);
    const R SR = fmax_(uL + cL, uR + cR);
    if (FLUX == FLX_HLL) {
        if (SL >= R(0)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = FL[v];
        } else if (SR <= R(0)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = FR[v];
        } else if constexpr (IsExact<R>::value) {
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
        } else {
            const R inv = rcp_approx(SR - SL);
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * inv;
        }
        return;
    }
    // HLLC: F_L if 0 <= S_L; F*_L if S_L < 0 <= S*; F*_R if S* < 0 < S_R; F_R otherwise.
    if (SL >= R(0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = FL[v];
        return;
    }
    const R Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    const bool left = Ss >= R(0);
    if (!left && !(SR > R(0))) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = FR[v];
        return;
    }
    const R SK = left ? SL : SR;
    const R rK = left ? rL : rR, uK = left ? uL : uR, pK = left ? pL : pR;
    const R EK = left ? UL[IP] : UR[IP];
    const R fac = rK * (SK - uK) / (SK - Ss);
    R Us[NV];
    Us[0] = fac;
#pragma unroll
    for (int j = 0; j < ND; ++j) Us[1 + j] = fac * (left ? WL[1 + j] : WR[1 + j]);
    Us[1 + D] = fac * Ss;
    Us[IP] = fac * (EK / rK + (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const R fk = left ? FL[v] : FR[v];
        const R uk = left ? UL[v] : UR[v];
        F[v] = fk + SK * (Us[v] - uk);
    }
}

// Scalar Burgers flux f(u) = u^2/2: Rusanov or HLL (HLLC coincides with HLL for a scalar law).
template <class R, int FLUX> __device__ __forceinline__ R burgers_flux(R uL, R uR) {
    if (FLUX == FLX_EC || FLUX == FLX_EC4) return (uL * uL + uL * uR + uR * uR) / R(6);   // entropy u^2/2
    const R fL = R(0.5) * uL * uL, fR = R(0.5) * uR * uR;
    if (FLUX == FLX_ROE) {
        const R a = R(0.5) * (uL + uR);   // Roe speed, Harten's fix on the transonic rarefaction
        return R(0.5) * (fL + fR) - R(0.5) * harten_abs(a, uL, uR) * (uR - uL);
    }
    if (FLUX == FLX_GODUNOV) {            // exact solution at x/t = 0
        if (uL > uR) return uL + uR >= R(0) ? fL : fR;
        if (uL >= R(0)) return fL;
        if (uR <= R(0)) return fR;
        return R(0);
    }
    if (FLUX == FLX_RUSANOV) {
        const R a = fmax_(fabs_(uL), fabs_(uR));
        return R(0.5) * (fL + fR) - R(0.5) * a * (uR - uL);
    }
    const R SL = fmin_(uL, uR), SR = fmax_(uL, uR);
    if (SL >= R(0)) return fL;
    if (SR <= R(0)) return fR;
    return (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL);
}

// ---------------------------------------------------------------------------------------------
// Ghost cells (paper silent; reading): periodic wraps, outflow copies the nearest interior cell,
// reflective mirrors interior cell -1-j for ghost j and negates the normal velocity. Indices far
// outside the grid (padding of partial tiles) are clamped so every read stays in bounds.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int map_ghost(int i, int n, int bc_lo, int bc_hi, bool& flip) {
    if (i >= 0 && i < n) return i;
    if (i < 0) {
        if (bc_lo == BC_PERIODIC) { i %= n; return i < 0 ? i + n : i; }
        if (bc_lo == BC_OUTFLOW) return 0;
        flip = !flip;
        i = -1 - i;
        return i < n ? i : n - 1;
    }
    if (bc_hi == BC_PERIODIC) return i % n;
    if (bc_hi == BC_OUTFLOW) return n - 1;
    flip = !flip;
    i = 2 * n - 1 - i;
    return i >= 0 ? i : 0;
}

// Locate the level and local sample of a global work item / sample.
__device__ __forceinline__ int level_of_work(const GridArgs& g, uint32_t w) {
    int l = 0;
#pragma unroll 1
    for (int k = 1; k < g.nlev; ++k)
        if ((long long)w >= g.lev[k].work0) l = k;
    return l;
}
__device__ __forceinline__ int level_of_sample(const GridArgs& g, int s) {
    int l = 0;
#pragma unroll 1
    for (int k = 1; k < g.nlev; ++k)
        if (s >= g.lev[k].sample0) l = k;
    return l;
}

}  // namespace alsv
