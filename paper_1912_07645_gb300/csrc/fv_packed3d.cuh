// Packed FP32x2 flux building blocks for 3D Euler: two independent interface evaluations per
// instruction (an x- and a y-interface of one plane in the packed z-march). States are (density,
// normal velocity, two tangential velocities, pressure); the same rules and one-sided HLLC form
// as hllc_fast.
#pragma once

#include "fv_pair2.cuh"

namespace alsv {

// ---- 3D states: (density, normal velocity, two tangential velocities, pressure)
struct F2x5 {
    float2 r, n, t, w, p;
};

__device__ __forceinline__ void cons_flux2_5(const F2x5& W, float inv_gm1, F2x5& U, F2x5& F) {
    const float2 u2 = fma2(W.n, W.n, fma2(W.t, W.t, mul2(W.w, W.w)));
    U.r = W.r;
    U.n = mul2(W.r, W.n);
    U.t = mul2(W.r, W.t);
    U.w = mul2(W.r, W.w);
    U.p = fma2(mul2(f2(0.5f), W.r), u2, mul2(W.p, f2(inv_gm1)));  // E
    F.r = U.n;
    F.n = fma2(U.n, W.n, W.p);
    F.t = mul2(U.t, W.n);
    F.w = mul2(U.w, W.n);
    F.p = mul2(W.n, add2(U.p, W.p));
}

__device__ __forceinline__ F2x5 rusanov2_5(const F2x5& L, const F2x5& R, float gamma, float inv_gm1) {
    F2x5 UL, FL, UR, FR, F;
    cons_flux2_5(L, inv_gm1, UL, FL);
    cons_flux2_5(R, inv_gm1, UR, FR);
    const float2 cL = sound2(gamma, L.p, L.r), cR = sound2(gamma, R.p, R.r);
    const float2 a = max2(add2(abs2(L.n), cL), add2(abs2(R.n), cR));
    const float2 ha = mul2(f2(-0.5f), a);
    const float2 h = f2(0.5f);
    F.r = fma2(ha, sub2(UR.r, UL.r), mul2(h, add2(FL.r, FR.r)));
    F.n = fma2(ha, sub2(UR.n, UL.n), mul2(h, add2(FL.n, FR.n)));
    F.t = fma2(ha, sub2(UR.t, UL.t), mul2(h, add2(FL.t, FR.t)));
    F.w = fma2(ha, sub2(UR.w, UL.w), mul2(h, add2(FL.w, FR.w)));
    F.p = fma2(ha, sub2(UR.p, UL.p), mul2(h, add2(FL.p, FR.p)));
    return F;
}

// HLLC in 3D, two interfaces at once: the case rules and one-sided form of hllc_fast
__device__ __forceinline__ F2x5 hllc2_5(const F2x5& L, const F2x5& R, float gamma, float inv_gm1) {
    const float2 cL = sound2(gamma, L.p, L.r), cR = sound2(gamma, R.p, R.r);
    const float2 SL = min2(sub2(L.n, cL), sub2(R.n, cR));
    const float2 SR = max2(add2(L.n, cL), add2(R.n, cR));
    const float2 mL = mul2(L.r, sub2(SL, L.n)), mR = mul2(R.r, sub2(SR, R.n));
    const float2 num = fma2(neg2(R.n), mR, fma2(L.n, mL, sub2(R.p, L.p)));
    const float2 Ss = mul2(num, rcp2(sub2(mL, mR)));
    const bool lx = SL.x >= 0.f || Ss.x >= 0.f, ly = SL.y >= 0.f || Ss.y >= 0.f;
    const bool sx = !(SL.x >= 0.f) && (lx || SR.x > 0.f), sy = !(SL.y >= 0.f) && (ly || SR.y > 0.f);
    F2x5 K;
    K.r = sel2(lx, ly, L.r, R.r);
    K.n = sel2(lx, ly, L.n, R.n);
    K.t = sel2(lx, ly, L.t, R.t);
    K.w = sel2(lx, ly, L.w, R.w);
    K.p = sel2(lx, ly, L.p, R.p);
    const float2 SK = sel2(lx, ly, SL, SR);
    F2x5 UK, FK;
    cons_flux2_5(K, inv_gm1, UK, FK);
    const float2 A = sub2(SK, K.n);
    const float2 invB = rcp2(sub2(SK, Ss));
    const float2 fac = mul2(mul2(K.r, A), invB);
    const float2 dS = sub2(Ss, K.n);
    F2x5 Us;
    Us.r = fac;
    Us.n = mul2(fac, Ss);
    Us.t = mul2(fac, K.t);
    Us.w = mul2(fac, K.w);
    Us.p = fma2(mul2(fac, dS), Ss, mul2(fma2(A, UK.p, mul2(dS, K.p)), invB));
    F2x5 F;
    F.r = sel2(sx, sy, fma2(SK, sub2(Us.r, UK.r), FK.r), FK.r);
    F.n = sel2(sx, sy, fma2(SK, sub2(Us.n, UK.n), FK.n), FK.n);
    F.t = sel2(sx, sy, fma2(SK, sub2(Us.t, UK.t), FK.t), FK.t);
    F.w = sel2(sx, sy, fma2(SK, sub2(Us.w, UK.w), FK.w), FK.w);
    F.p = sel2(sx, sy, fma2(SK, sub2(Us.p, UK.p), FK.p), FK.p);
    return F;
}

// HLLC in 3D as hllc2_5 (same wave speeds, contact speed and upwind side K), with the star
// correction F = F_K + S_K (U*_K - U_K) applied through s = S_K in the star cases and 0 otherwise,
// as hllc2_lean does in 2D (the star state has a finite denominator in every case).
__device__ __forceinline__ F2x5 hllc2_5_lean(const F2x5& L, const F2x5& R, float gamma, float inv_gm1) {
    const float2 cL = sound2(gamma, L.p, L.r), cR = sound2(gamma, R.p, R.r);
    const float2 SL = min2(sub2(L.n, cL), sub2(R.n, cR));
    const float2 SR = max2(add2(L.n, cL), add2(R.n, cR));
    const float2 mL = mul2(L.r, sub2(SL, L.n)), mR = mul2(R.r, sub2(SR, R.n));
    const float2 num = fma2(neg2(R.n), mR, fma2(L.n, mL, sub2(R.p, L.p)));
    const float2 Ss = mul2(num, rcp2(sub2(mL, mR)));
    const bool lx = SL.x >= 0.f || Ss.x >= 0.f, ly = SL.y >= 0.f || Ss.y >= 0.f;
    const bool sx = !(SL.x >= 0.f) && (lx || SR.x > 0.f), sy = !(SL.y >= 0.f) && (ly || SR.y > 0.f);
    F2x5 K;
    K.r = sel2(lx, ly, L.r, R.r);
    K.n = sel2(lx, ly, L.n, R.n);
    K.t = sel2(lx, ly, L.t, R.t);
    K.w = sel2(lx, ly, L.w, R.w);
    K.p = sel2(lx, ly, L.p, R.p);
    const float2 SK = sel2(lx, ly, SL, SR);
    F2x5 UK, FK;
    cons_flux2_5(K, inv_gm1, UK, FK);
    const float2 A = sub2(SK, K.n);
    const float2 B = sub2(SK, Ss);
    const float2 invB = rcp2(make_float2(sx ? B.x : 1.0f, sy ? B.y : 1.0f));
    const float2 sk = make_float2(sx ? SK.x : 0.0f, sy ? SK.y : 0.0f);
    const float2 fac = mul2(mul2(K.r, A), invB);
    const float2 dS = sub2(Ss, K.n);
    F2x5 Us;
    Us.r = fac;
    Us.n = mul2(fac, Ss);
    Us.t = mul2(fac, K.t);
    Us.w = mul2(fac, K.w);
    Us.p = fma2(mul2(fac, dS), Ss, mul2(fma2(A, UK.p, mul2(dS, K.p)), invB));
    F2x5 F;
    F.r = fma2(sk, sub2(Us.r, UK.r), FK.r);
    F.n = fma2(sk, sub2(Us.n, UK.n), FK.n);
    F.t = fma2(sk, sub2(Us.t, UK.t), FK.t);
    F.w = fma2(sk, sub2(Us.w, UK.w), FK.w);
    F.p = fma2(sk, sub2(Us.p, UK.p), FK.p);
    return F;
}

// Both face values of the five variables at an interface from the stencil cells c[0..3] (the
// cell pair is c[1], c[2]): differences, WENO3 weights and faces as faces_d, then the positivity
// fallback (a face with rho <= 0 or p <= 0 takes its cell's own state, per lane) only when a lane
// of the warp needs it (mask = the warp's active lanes).
template <int RECON>
__device__ __forceinline__ void faces2_5_lean(const F2x5 c[4], float2 eps, unsigned mask, F2x5& WL, F2x5& WR) {
    auto one = [&](float2 wm, float2 w0, float2 w1, float2 w2, float2& fr, float2& fl) {
        float2 dm = f2(0.f), d1 = f2(0.f), d2 = f2(0.f), qm = f2(0.f), q1 = f2(0.f), q2 = f2(0.f);
        if (RECON != REC_PC) {
            dm = sub2(w0, wm);
            d1 = sub2(w1, w0);
            d2 = sub2(w2, w1);
        }
        if (RECON == REC_WENO3) {
            qm = wq2(dm, eps);
            q1 = wq2(d1, eps);
            q2 = wq2(d2, eps);
        }
        faces_d<RECON>(w0, w1, dm, d1, d2, qm, q1, q2, fr, fl);
    };
    one(c[0].r, c[1].r, c[2].r, c[3].r, WL.r, WR.r);
    one(c[0].n, c[1].n, c[2].n, c[3].n, WL.n, WR.n);
    one(c[0].t, c[1].t, c[2].t, c[3].t, WL.t, WR.t);
    one(c[0].w, c[1].w, c[2].w, c[3].w, WL.w, WR.w);
    one(c[0].p, c[1].p, c[2].p, c[3].p, WL.p, WR.p);
    if (RECON != REC_PC) {
        const bool okLx = WL.r.x > 0.f && WL.p.x > 0.f, okLy = WL.r.y > 0.f && WL.p.y > 0.f;
        const bool okRx = WR.r.x > 0.f && WR.p.x > 0.f, okRy = WR.r.y > 0.f && WR.p.y > 0.f;
        if (!__all_sync(mask, okLx && okLy && okRx && okRy)) {
            WL.r = sel2(okLx, okLy, WL.r, c[1].r);
            WL.n = sel2(okLx, okLy, WL.n, c[1].n);
            WL.t = sel2(okLx, okLy, WL.t, c[1].t);
            WL.w = sel2(okLx, okLy, WL.w, c[1].w);
            WL.p = sel2(okLx, okLy, WL.p, c[1].p);
            WR.r = sel2(okRx, okRy, WR.r, c[2].r);
            WR.n = sel2(okRx, okRy, WR.n, c[2].n);
            WR.t = sel2(okRx, okRy, WR.t, c[2].t);
            WR.w = sel2(okRx, okRy, WR.w, c[2].w);
            WR.p = sel2(okRx, okRy, WR.p, c[2].p);
        }
    }
}

}  // namespace alsv
