// Packed FP32x2 building blocks: two independent evaluations per instruction (two interfaces of one
// cell in the column schedule, or the same interface of two Monte Carlo samples in the pair
// schedule). States are (density, normal velocity, tangential velocity, pressure).
#pragma once

#include "fv_physics.cuh"

namespace alsv {

struct F2x4 {
    float2 r, n, t, p;  // density, normal velocity, tangential velocity, pressure (or flux components)
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b) {
    return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}
__device__ __forceinline__ float2 min2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// sound speed sqrt(gamma p / rho) per lane, as gamma p * rsqrt(gamma p rho)
__device__ __forceinline__ float2 sound2(float gamma, float2 p, float2 r) {
    const float2 gp = mul2(f2(gamma), p);
    const float2 q = mul2(gp, r);
    return mul2(gp, make_float2(rsqrt_approx(q.x), rsqrt_approx(q.y)));
}

// conserved state and physical flux of a primitive state in (normal, tangential) coordinates
__device__ __forceinline__ void cons_flux2(const F2x4& W, float inv_gm1, F2x4& U, F2x4& F) {
    const float2 u2 = fma2(W.n, W.n, mul2(W.t, W.t));
    U.r = W.r;
    U.n = mul2(W.r, W.n);
    U.t = mul2(W.r, W.t);
    U.p = fma2(mul2(f2(0.5f), W.r), u2, mul2(W.p, f2(inv_gm1)));  // E
    F.r = U.n;
    F.n = fma2(U.n, W.n, W.p);
    F.t = mul2(U.t, W.n);
    F.p = mul2(W.n, add2(U.p, W.p));
}

// Rusanov flux, two interfaces at once
__device__ __forceinline__ F2x4 rusanov2(const F2x4& L, const F2x4& R, float gamma, float inv_gm1) {
    F2x4 UL, FL, UR, FR, F;
    cons_flux2(L, inv_gm1, UL, FL);
    cons_flux2(R, inv_gm1, UR, FR);
    const float2 cL = sound2(gamma, L.p, L.r), cR = sound2(gamma, R.p, R.r);
    const float2 a = max2(add2(abs2(L.n), cL), add2(abs2(R.n), cR));
    const float2 ha = mul2(f2(-0.5f), a);
    const float2 h = f2(0.5f);
    F.r = fma2(ha, sub2(UR.r, UL.r), mul2(h, add2(FL.r, FR.r)));
    F.n = fma2(ha, sub2(UR.n, UL.n), mul2(h, add2(FL.n, FR.n)));
    F.t = fma2(ha, sub2(UR.t, UL.t), mul2(h, add2(FL.t, FR.t)));
    F.p = fma2(ha, sub2(UR.p, UL.p), mul2(h, add2(FL.p, FR.p)));
    return F;
}

// HLLC flux, two interfaces at once: the same case rules and one-sided form as hllc_fast
__device__ __forceinline__ F2x4 hllc2(const F2x4& L, const F2x4& R, float gamma, float inv_gm1) {
    const float2 cL = sound2(gamma, L.p, L.r), cR = sound2(gamma, R.p, R.r);
    const float2 SL = min2(sub2(L.n, cL), sub2(R.n, cR));
    const float2 SR = max2(add2(L.n, cL), add2(R.n, cR));
    const float2 mL = mul2(L.r, sub2(SL, L.n)), mR = mul2(R.r, sub2(SR, R.n));
    const float2 num = fma2(neg2(R.n), mR, fma2(L.n, mL, sub2(R.p, L.p)));
    const float2 Ss = mul2(num, rcp2(sub2(mL, mR)));
    const bool lx = SL.x >= 0.f || Ss.x >= 0.f, ly = SL.y >= 0.f || Ss.y >= 0.f;
    const bool sx = !(SL.x >= 0.f) && (lx || SR.x > 0.f), sy = !(SL.y >= 0.f) && (ly || SR.y > 0.f);
    F2x4 K;
    K.r = sel2(lx, ly, L.r, R.r);
    K.n = sel2(lx, ly, L.n, R.n);
    K.t = sel2(lx, ly, L.t, R.t);
    K.p = sel2(lx, ly, L.p, R.p);
    const float2 SK = sel2(lx, ly, SL, SR);
    F2x4 UK, FK;
    cons_flux2(K, inv_gm1, UK, FK);
    const float2 A = sub2(SK, K.n);
    const float2 invB = rcp2(sub2(SK, Ss));
    const float2 fac = mul2(mul2(K.r, A), invB);
    const float2 dS = sub2(Ss, K.n);
    F2x4 Us;
    Us.r = fac;
    Us.n = mul2(fac, Ss);
    Us.t = mul2(fac, K.t);
    Us.p = fma2(mul2(fac, dS), Ss, mul2(fma2(A, UK.p, mul2(dS, K.p)), invB));
    F2x4 F;
    F.r = sel2(sx, sy, fma2(SK, sub2(Us.r, UK.r), FK.r), FK.r);
    F.n = sel2(sx, sy, fma2(SK, sub2(Us.n, UK.n), FK.n), FK.n);
    F.t = sel2(sx, sy, fma2(SK, sub2(Us.t, UK.t), FK.t), FK.t);
    F.p = sel2(sx, sy, fma2(SK, sub2(Us.p, UK.p), FK.p), FK.p);
    return F;
}

// both face values of one variable at an interface, for the two packed evaluations
template <int RECON>
__device__ __forceinline__ void faces2(float2 wm, float2 w0, float2 w1, float2 w2, float2 eps, float2& fr, float2& fl) {
    if (RECON == REC_WENO3) {
        weno3_pair2(wm, w0, w1, w2, eps, fr, fl);
    } else if (RECON == REC_PC) {
        fr = w0;
        fl = w1;
    } else {
        fr = make_float2(w0.x + 0.5f * mc_slope(wm.x, w0.x, w1.x), w0.y + 0.5f * mc_slope(wm.y, w0.y, w1.y));
        fl = make_float2(w1.x - 0.5f * mc_slope(w0.x, w1.x, w2.x), w1.y - 0.5f * mc_slope(w0.y, w1.y, w2.y));
    }
}

}  // namespace alsv
