// Packed FP32x2 flux building blocks for 3D Euler: two independent interface evaluations per
// instruction (an x- and a y-interface of one plane in the packed z-march). States are (density,
// normal velocity, two tangential velocities, pressure); the same rules and one-sided HLLC form
// as hllc_fast.
#pragma once

#include "fv_packed.cuh"

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

}  // namespace alsv
