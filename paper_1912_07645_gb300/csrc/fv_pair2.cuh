// Two-sample SSP-RK stage for 2D Euler in FP32, lean schedule: the same eq. (2.1) stage and the
// same pair-interleaved shared-memory tile as k_stage2d_pair (lane .x = sample A, lane .y = sample
// B, or the two halves of one y-periodic sample), arranged to issue fewer instructions per cell:
//
// * fixed thread-to-cell maps (lane = column, warp = row group): no division or remainder by the
//   halo width or the interface count in any loop;
// * WENO3 faces from the three differences around an interface, fr = p1 + q1 (dm - d1) / (2 (q1 +
//   2 qm)), fl = p1 + q1 (d1 - d2) / (2 (q1 + 2 q2)), q = (eps + d^2)^2 - the Jiang-Shu weights
//   with p0 - p1 written as half a difference of differences (fewer operations than forming both
//   candidates);
// * the positivity fallback (a face with rho <= 0 or p <= 0 takes its cell's own state, per face
//   and per sample) runs only when a lane of the warp needs it;
// * HLLC applies its star correction through the upwind speed, zeroed outside the star cases,
//   instead of selecting each flux component.
#pragma once

#include "fv_packed.cuh"

namespace alsv {

template <int RECON, int TY, int XSHFL = 0>
constexpr size_t pair2_smem_bytes() {
    constexpr int TX = 32;
    constexpr int G = RECON == REC_PC ? 1 : 2;
    constexpr int NS = (TX + 2 * G) * (TY + 2 * G);
    constexpr int NIX = (TX + 1) * TY, NIY = TX * (TY + 1);
    constexpr int NI = NIX > NIY ? NIX : NIY;
    // XSHFL: the right-edge x-fluxes and lane 31's left-face x-fluxes, two float4 per row each
    return (size_t)32 * (NS + NI) + (XSHFL ? (size_t)64 * TY : 0);
}

__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }

// MC slope minmod(2 dm, (dm + dp) / 2, 2 dp) from the two one-sided differences (as mc_slope)
__device__ __forceinline__ float mc_slope_d(float dm, float dp) {
    return minmod3(2.0f * dm, 0.5f * (dm + dp), 2.0f * dp);
}

// WENO3 smoothness weight (eps + d^2)^2 of one difference
__device__ __forceinline__ float2 wq2(float2 d, float2 eps) {
    const float2 e = fma2(d, d, eps);
    return mul2(e, e);
}

// Both face values of one variable at interface i+1/2 from the cell values w0 = w_i, w1 = w_{i+1},
// the differences dm = w_i - w_{i-1}, d1 = w_{i+1} - w_i, d2 = w_{i+2} - w_{i+1} and (WENO3) their
// weights qm, q1, q2. fr is the right face of cell i, fl the left face of cell i+1.
template <int RECON>
__device__ __forceinline__ void faces_d(float2 w0, float2 w1, float2 dm, float2 d1, float2 d2, float2 qm, float2 q1,
                                        float2 q2, float2& fr, float2& fl) {
    if (RECON == REC_WENO3) {
        const float2 p1 = fma2(f2(0.5f), d1, w0);
        const float2 hq = mul2(f2(0.5f), q1);
        const float2 dr = fma2(f2(2.0f), qm, q1), dl = fma2(f2(2.0f), q2, q1);
        fr = fma2(mul2(hq, sub2(dm, d1)), rcp2(dr), p1);
        fl = fma2(mul2(hq, sub2(d1, d2)), rcp2(dl), p1);
    } else if (RECON == REC_MC) {
        // MC slope minmod(2 d-, (d- + d+)/2, 2 d+) per lane, half of it to each face
        const float2 sr = make_float2(mc_slope_d(dm.x, d1.x), mc_slope_d(dm.y, d1.y));
        const float2 sl = make_float2(mc_slope_d(d1.x, d2.x), mc_slope_d(d1.y, d2.y));
        fr = fma2(f2(0.5f), sr, w0);
        fl = fma2(f2(-0.5f), sl, w1);
    } else {
        fr = w0;
        fl = w1;
    }
}

// HLLC as hllc2 (same wave speeds, contact speed and upwind side K), with the star correction
// F = F_K + S_K (U*_K - U_K) applied through s = S_K in the star cases and 0 otherwise (the star
// state is formed from a finite denominator in every case, so the product is always finite).
__device__ __forceinline__ F2x4 hllc2_lean(const F2x4& L, const F2x4& R, float gamma, float inv_gm1) {
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
    const float2 B = sub2(SK, Ss);
    const float2 invB = rcp2(make_float2(sx ? B.x : 1.0f, sy ? B.y : 1.0f));
    const float2 s = make_float2(sx ? SK.x : 0.0f, sy ? SK.y : 0.0f);
    const float2 fac = mul2(mul2(K.r, A), invB);
    const float2 dS = sub2(Ss, K.n);
    F2x4 Us;
    Us.r = fac;
    Us.n = mul2(fac, Ss);
    Us.t = mul2(fac, K.t);
    Us.p = fma2(mul2(fac, dS), Ss, mul2(fma2(A, UK.p, mul2(dS, K.p)), invB));
    F2x4 F;
    F.r = fma2(s, sub2(Us.r, UK.r), FK.r);
    F.n = fma2(s, sub2(Us.n, UK.n), FK.n);
    F.t = fma2(s, sub2(Us.t, UK.t), FK.t);
    F.p = fma2(s, sub2(Us.p, UK.p), FK.p);
    return F;
}

// Stencil of one interface for the four variables (rho, normal, tangential, p) of both lanes.
struct Sten2 {
    float2 w0[4], w1[4], dm[4], d1[4], d2[4], qm[4], q1[4], q2[4];
};

// Interface flux from a filled stencil: faces, positivity fallback (only when some lane of the
// warp needs it; mask = the warp's active lanes), flux.
template <int RECON, int FLUX>
__device__ __forceinline__ F2x4 interface_flux2(const Sten2& S, float gamma, float inv_gm1, unsigned mask) {
    F2x4 WL, WR;
    faces_d<RECON>(S.w0[0], S.w1[0], S.dm[0], S.d1[0], S.d2[0], S.qm[0], S.q1[0], S.q2[0], WL.r, WR.r);
    faces_d<RECON>(S.w0[1], S.w1[1], S.dm[1], S.d1[1], S.d2[1], S.qm[1], S.q1[1], S.q2[1], WL.n, WR.n);
    faces_d<RECON>(S.w0[2], S.w1[2], S.dm[2], S.d1[2], S.d2[2], S.qm[2], S.q1[2], S.q2[2], WL.t, WR.t);
    faces_d<RECON>(S.w0[3], S.w1[3], S.dm[3], S.d1[3], S.d2[3], S.qm[3], S.q1[3], S.q2[3], WL.p, WR.p);
    if (RECON != REC_PC) {
        const bool okLx = WL.r.x > 0.f && WL.p.x > 0.f, okLy = WL.r.y > 0.f && WL.p.y > 0.f;
        const bool okRx = WR.r.x > 0.f && WR.p.x > 0.f, okRy = WR.r.y > 0.f && WR.p.y > 0.f;
        if (!__all_sync(mask, okLx && okLy && okRx && okRy)) {
            WL.r = sel2(okLx, okLy, WL.r, S.w0[0]);
            WL.n = sel2(okLx, okLy, WL.n, S.w0[1]);
            WL.t = sel2(okLx, okLy, WL.t, S.w0[2]);
            WL.p = sel2(okLx, okLy, WL.p, S.w0[3]);
            WR.r = sel2(okRx, okRy, WR.r, S.w1[0]);
            WR.n = sel2(okRx, okRy, WR.n, S.w1[1]);
            WR.t = sel2(okRx, okRy, WR.t, S.w1[2]);
            WR.p = sel2(okRx, okRy, WR.p, S.w1[3]);
        }
    }
    return FLUX == FLX_HLLC ? hllc2_lean(WL, WR, gamma, inv_gm1) : rusanov2(WL, WR, gamma, inv_gm1);
}

// the four variables of a shared-memory cell in (rho, normal, tangential, p) order of direction D
template <int D>
__device__ __forceinline__ void cell_vars(const float4* sW0, const float4* sW1, int idx, float2 v[4]) {
    const float4 a = sW0[idx], b = sW1[idx];
    v[0] = lo2(a);
    v[1] = D == 0 ? hi2(a) : lo2(b);
    v[2] = D == 0 ? lo2(b) : hi2(a);
    v[3] = hi2(b);
}

// Fill a stencil around the interface whose left/lower cell has shared-memory index i0 (cells
// i0 - step .. i0 + 2 step; PC reads only i0 and i0 + step).
template <int RECON, int D>
__device__ __forceinline__ void load_sten(const float4* sW0, const float4* sW1, int i0, int step, float2 eps,
                                          Sten2& S) {
    float2 wm[4], w2[4];
    cell_vars<D>(sW0, sW1, i0, S.w0);
    cell_vars<D>(sW0, sW1, i0 + step, S.w1);
    if (RECON != REC_PC) {
        cell_vars<D>(sW0, sW1, i0 - step, wm);
        cell_vars<D>(sW0, sW1, i0 + 2 * step, w2);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        if (RECON != REC_PC) {
            S.dm[v] = sub2(S.w0[v], wm[v]);
            S.d1[v] = sub2(S.w1[v], S.w0[v]);
            S.d2[v] = sub2(w2[v], S.w1[v]);
        }
        if (RECON == REC_WENO3) {
            S.qm[v] = wq2(S.dm[v], eps);
            S.q1[v] = wq2(S.d1[v], eps);
            S.q2[v] = wq2(S.d2[v], eps);
        }
    }
}

// TY rows per tile (16: 4 CTAs per SM with 64 registers; 32: 3 CTAs with 80); 256 threads = 8
// warps; lane = column, warp = row group. HALVES as in k_stage2d_pair. PREF: every global read of
// the tile load in flight at once (one round trip instead of two), and the epilogue's reads of
// all the thread's cells issued before its first store. XSHFL: each lane evaluates the x-interface
// at the left face of its cells and takes the right face's flux from lane + 1 by a warp shuffle,
// so the x-fluxes never pass through shared memory; the tile's right-edge x-interfaces (evaluated
// by one half-warp) and lane 31's own left-face fluxes go through two small shared arrays, and
// lane 31 adds its x part after the one barrier that also completes the y-fluxes. Both directions
// thus share one phase between two barriers (instead of four barriers), with the same operations
// per cell in the same order (bitwise equal to XSHFL = 0).
template <int RECON, int FLUX, int TY, int HALVES = 0, int PREF = 0, int XSHFL = 0>
__global__ void __launch_bounds__(256, TY >= 32 ? 3 : 4) k_stage2d_pair2(const StageArgs p) {
    constexpr int TX = 32, NT = 256, NW = 8;
    constexpr int G = RECON == REC_PC ? 1 : 2;
    constexpr int SX = TX + 2 * G, SY = TY + 2 * G, NS = SX * SY;
    constexpr int NIX = (TX + 1) * TY, NIY = TX * (TY + 1);
    constexpr int NI = NIX > NIY ? NIX : NIY;
    constexpr int CPT = TY / NW;   // cells per thread (and y-interfaces per thread run)
    static_assert(TY % NW == 0, "tile height must be a multiple of the warp count");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* sW0 = reinterpret_cast<float4*>(smem_raw);  // [NS] (rho, u) of both lanes
    float4* sW1 = sW0 + NS;                              // [NS] (v, p)
    float4* sF0 = sW1 + NS;                              // [NI] (mass, x-momentum) fluxes
    float4* sF1 = sF0 + NI;                              // [NI] (y-momentum, energy)
    float4* sXL = sF1 + NI;                              // XSHFL: [2][TY] lane 31's left-face x-fluxes
    float4* sXE = sXL + 2 * TY;                          // XSHFL: [2][TY] right-edge x-fluxes

    const GridArgs& g = p.g;
    const uint32_t w = blockIdx.x;
    int l = 0;
#pragma unroll 1
    for (int k = 1; k < g.nlev; ++k)
        if ((long long)w >= g.lev[k].pwork0) l = k;
    const LevelInfo& L = g.lev[l];
    const uint32_t wl = w - (uint32_t)L.pwork0;
    const uint32_t htiles = (uint32_t)L.tiles / 2u;
    const uint32_t q = HALVES ? wl / htiles : fdiv(wl, L.fd_tiles);
    const uint32_t tile = wl - q * (HALVES ? htiles : (uint32_t)L.tiles);
    const int sA = HALVES ? (int)q : 2 * (int)q;
    const bool hasB = HALVES ? true : sA + 1 < L.samples;
    const int sB = HALVES ? sA : (hasB ? sA + 1 : sA);
    // While no sample has finished (the host sets done_first from its done-flag polls) the done
    // flags are read now but acted on after the tile load, so that their round trip overlaps the
    // halo loads instead of preceding them. Once samples finish (and on grids of several levels,
    // whose coarse levels finish after a fraction of the finest level's steps), a finished pair
    // returns before any load, as its tile reads would otherwise repeat in every later stage.
    const bool doneA = p.done[L.sample0 + sA] != 0;
    const bool doneB = hasB ? p.done[L.sample0 + sB] != 0 : true;
    if ((g.nlev > 1 || p.done_first) && doneA && doneB) return;   // uniform over the CTA, before any barrier

    const int nx = L.n[0], ny = L.n[1];
    const uint32_t trow = fdiv(tile, L.fd_nt0);
    const int tx0 = (int)(tile - trow * (uint32_t)L.ntile[0]) * TX;
    const int ty0 = (int)trow * TY;
    const int plane = nx * ny;
    const int hs = HALVES ? ny / 2 : 0;
    const long long bA = L.elem0 + (long long)sA * 4 * plane, bB = L.elem0 + (long long)sB * 4 * plane;
    const float* UsA = reinterpret_cast<const float*>(p.Us) + bA;
    const float* UsB = reinterpret_cast<const float*>(p.Us) + bB;
    const float gamma = g.gamma_f, gm1 = g.gm1_f, inv_gm1 = g.inv_gm1_f;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- 1. tile + halo load: the TX core columns by (lane, row group), the 2G side columns by
    // the first 2G SY threads; boundary fill on edge tiles; primitive conversion.
    const bool interior = tx0 >= G && tx0 + SX - G <= nx && ty0 >= G && ty0 + SY - G <= ny;
    constexpr int CORE_IT = (SY + NW - 1) / NW;          // row groups of the core columns
    constexpr int NSIDE = 2 * G * SY;                    // side-column cells
    static_assert(NSIDE <= NT, "side columns in one pass");
    constexpr int NLOAD = CORE_IT + 1;
    constexpr int LG = PREF ? NLOAD : 2;
#pragma unroll
    for (int it0 = 0; it0 < NLOAD; it0 += LG) {
        float2 r[LG], mx[LG], my[LG], E[LG];
        bool fxs[LG], fys[LG], act[LG];
        int sidx[LG];
#pragma unroll
        for (int j = 0; j < LG; ++j) {
            const int it = it0 + j;
            int sx, sy;
            if (it < CORE_IT) {
                sx = G + lane;
                sy = warp + NW * it;
                act[j] = sy < SY;
            } else {
                const int c = tid;
                const int side = c % (2 * G);   // compile-time power-of-two divisor for G = 1, 2
                sx = side < G ? side : TX + side;
                sy = c / (2 * G);
                act[j] = it < NLOAD && c < NSIDE;
            }
            sidx[j] = sy * SX + sx;
            fxs[j] = false;
            fys[j] = false;
            if (act[j]) {
                int ix = tx0 + sx - G, iy = ty0 + sy - G;
                if (!interior) {
                    ix = map_ghost(ix, nx, g.bc[0][0], g.bc[0][1], fxs[j]);
                    iy = map_ghost(iy, ny, g.bc[1][0], g.bc[1][1], fys[j]);
                }
                const int off = iy * nx + ix;
                int offB = off;
                if (HALVES) {
                    const int iyB = iy + hs < ny ? iy + hs : iy + hs - ny;
                    offB = iyB * nx + ix;
                }
                r[j] = make_float2(UsA[off], UsB[offB]);
                mx[j] = make_float2(UsA[plane + off], UsB[plane + offB]);
                my[j] = make_float2(UsA[2 * plane + off], UsB[2 * plane + offB]);
                E[j] = make_float2(UsA[3 * plane + off], UsB[3 * plane + offB]);
            }
        }
#pragma unroll
        for (int j = 0; j < LG; ++j) {
            if (!act[j]) continue;
            float2 mxj = mx[j], myj = my[j];
            if (fxs[j]) mxj = neg2(mxj);
            if (fys[j]) myj = neg2(myj);
            const float2 inv = rcp2(r[j]);
            const float2 u = mul2(mxj, inv), v = mul2(myj, inv);
            const float2 m2 = fma2(mxj, mxj, mul2(myj, myj));
            const float2 pr = mul2(f2(gm1), fma2(mul2(f2(-0.5f), m2), inv, E[j]));
            sW0[sidx[j]] = make_float4(r[j].x, r[j].y, u.x, u.y);
            sW1[sidx[j]] = make_float4(v.x, v.y, pr.x, pr.y);
        }
    }

    if (doneA && doneB) return;   // uniform over the CTA, before its first barrier

    float2 acc[CPT][4];
#pragma unroll
    for (int m = 0; m < CPT; ++m)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[m][v] = f2(0.f);

    // ---- 2. interfaces of direction D: (fx, fy) with fx = lane and fy = warp + 8 m over the tile,
    // plus the extra column (D = 0: fx = TX, fy < TY, the first TY threads) or row (D = 1: fy = TY,
    // the first warp). The left / lower cell of an interface is tile column fx - 1 / row fy - 1.
    // Fluxes go to shared memory; each thread then adds the divergence of its own cells.
    // interfaces of direction D into their flux buffer; the extra column / row goes to the last
    // warp (x) or, merged, the one before it (y), so that no warp takes both
    auto flux_pass = [&](const int D) {
        const float2 eps = f2(L.eps_f[D]);
        const int EX = D == 0 ? TX + 1 : TX;
        const int step = D == 0 ? 1 : SX;
        const int xwarp = NW - 1, ywarp = NW - 1;
        float4* F0 = sF0;
        float4* F1 = sF1;
#pragma unroll 1
        for (int m = 0; m <= CPT; ++m) {
            int fx = lane, fy = warp + NW * m;
            unsigned mask = 0xffffffffu;
            if (m == CPT) {
                if (D == 0) {
                    if (warp != xwarp || lane >= TY) break;
                    fx = TX;
                    fy = lane;
                    mask = TY >= 32 ? 0xffffffffu : ((1u << TY) - 1u);
                } else {
                    if (warp != ywarp) break;
                    fy = TY;
                }
            }
            const int i0 = (fy - (D == 1) + G) * SX + fx - (D == 0) + G;
            Sten2 S;
            if (D == 0) load_sten<RECON, 0>(sW0, sW1, i0, step, eps, S);
            else load_sten<RECON, 1>(sW0, sW1, i0, step, eps, S);
            const F2x4 F = interface_flux2<RECON, FLUX>(S, gamma, inv_gm1, mask);
            const float2 fxm = D == 0 ? F.n : F.t, fym = D == 0 ? F.t : F.n;   // x-, y-momentum
            const int f = fy * EX + fx;
            F0[f] = make_float4(F.r.x, F.r.y, fxm.x, fxm.y);
            F1[f] = make_float4(fym.x, fym.y, F.p.x, F.p.y);
        }
    };
    // each thread adds -(F_{+1/2} - F_{-1/2}) / dx_D of its own cells, x before y
    auto divergence = [&](const int D) {
        const float2 nid = f2(-L.inv_dx_f[D]);
        const int EX = D == 0 ? TX + 1 : TX;
        const int fstep = D == 0 ? 1 : TX;
        const float4* F0 = sF0;
        const float4* F1 = sF1;
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const int fidx = (warp + NW * m) * EX + lane;
            const float4 am = F0[fidx], bm = F1[fidx];
            const float4 ap = F0[fidx + fstep], bp = F1[fidx + fstep];
            acc[m][0] = fma2(sub2(lo2(ap), lo2(am)), nid, acc[m][0]);
            acc[m][1] = fma2(sub2(hi2(ap), hi2(am)), nid, acc[m][1]);
            acc[m][2] = fma2(sub2(lo2(bp), lo2(bm)), nid, acc[m][2]);
            acc[m][3] = fma2(sub2(hi2(bp), hi2(bm)), nid, acc[m][3]);
        }
    };
    if constexpr (XSHFL) {
        static_assert(!XSHFL || TY <= 32, "edge rows fit one warp");
        __syncthreads();
        // y first (its fluxes go to shared memory), so that the x part of acc, which the x pass
        // forms directly, is live only from the x pass on
        flux_pass(1);
        // x: the left-face interface of each of the thread's cells; the right face from lane + 1
        {
            const float2 eps = f2(L.eps_f[0]);
            const float2 nid = f2(-L.inv_dx_f[0]);
#pragma unroll   // acc[m] is written here: a runtime m would move acc to local memory
            for (int m = 0; m < CPT; ++m) {
                const int fy = warp + NW * m;
                const int i0 = (fy + G) * SX + lane - 1 + G;
                Sten2 S;
                load_sten<RECON, 0>(sW0, sW1, i0, 1, eps, S);
                const F2x4 F = interface_flux2<RECON, FLUX>(S, gamma, inv_gm1, 0xffffffffu);
                // variables (mass, x-momentum, y-momentum, energy) = (r, n, t, p) along x
                auto down = [](float2 a) {
                    return make_float2(__shfl_down_sync(0xffffffffu, a.x, 1), __shfl_down_sync(0xffffffffu, a.y, 1));
                };
                const float2 nr = down(F.r), nn = down(F.n), nt = down(F.t), np = down(F.p);
                if (lane < 31) {
                    acc[m][0] = fma2(sub2(nr, F.r), nid, acc[m][0]);
                    acc[m][1] = fma2(sub2(nn, F.n), nid, acc[m][1]);
                    acc[m][2] = fma2(sub2(nt, F.t), nid, acc[m][2]);
                    acc[m][3] = fma2(sub2(np, F.p), nid, acc[m][3]);
                } else {
                    sXL[fy] = make_float4(F.r.x, F.r.y, F.n.x, F.n.y);
                    sXL[TY + fy] = make_float4(F.t.x, F.t.y, F.p.x, F.p.y);
                }
            }
            // the tile's right-edge x-interfaces: warp NW - 2, lane = row
            if (warp == NW - 2 && lane < TY) {
                const int i0 = (lane + G) * SX + TX - 1 + G;
                Sten2 S;
                load_sten<RECON, 0>(sW0, sW1, i0, 1, eps, S);
                const unsigned mask = TY >= 32 ? 0xffffffffu : ((1u << TY) - 1u);
                const F2x4 F = interface_flux2<RECON, FLUX>(S, gamma, inv_gm1, mask);
                sXE[lane] = make_float4(F.r.x, F.r.y, F.n.x, F.n.y);
                sXE[TY + lane] = make_float4(F.t.x, F.t.y, F.p.x, F.p.y);
            }
        }
        __syncthreads();
        if (lane == 31) {
            const float2 nid = f2(-L.inv_dx_f[0]);
#pragma unroll
            for (int m = 0; m < CPT; ++m) {
                const int fy = warp + NW * m;
                const float4 am = sXL[fy], bm = sXL[TY + fy], ap = sXE[fy], bp = sXE[TY + fy];
                acc[m][0] = fma2(sub2(lo2(ap), lo2(am)), nid, acc[m][0]);
                acc[m][1] = fma2(sub2(hi2(ap), hi2(am)), nid, acc[m][1]);
                acc[m][2] = fma2(sub2(lo2(bp), lo2(bm)), nid, acc[m][2]);
                acc[m][3] = fma2(sub2(hi2(bp), hi2(bm)), nid, acc[m][3]);
            }
        }
        divergence(1);
    } else {
#pragma unroll
        for (int D = 0; D < 2; ++D) {
            __syncthreads();
            flux_pass(D);
            __syncthreads();
            divergence(D);
        }
    }

    // ---- 3. RK combination, store per sample, CFL speed of the new states
    const float2 dt = make_float2(p.dt_f[L.sample0 + sA], p.dt_f[L.sample0 + sB]);
    const float2 ca = f2(p.a_f), cb = f2(p.b_f);
    const bool has_un = p.has_un != 0, want_speed = p.want_speed != 0;
    const float* UnA = reinterpret_cast<const float*>(p.Un) + bA;
    const float* UnB = reinterpret_cast<const float*>(p.Un) + bB;
    float* UoA = reinterpret_cast<float*>(p.Uout) + bA;
    float* UoB = reinterpret_cast<float*>(p.Uout) + bB;
    const float idx = L.inv_dx_f[0], idy = L.inv_dx_f[1];
    float2 smax = f2(0.f);
    bool badA = false, badB = false;
    const int x = tx0 + lane;
    // PREF: all reads of the thread's cells before the first write (the last stage writes over U^n
    // in place, so a later cell's read may not pass an earlier cell's write otherwise)
    constexpr int NPRE = PREF ? CPT : 1;
    float2 us_p[NPRE][4], un_p[NPRE][4];
    if (PREF) {
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const int y = ty0 + warp + NW * m;
            if (x >= nx || y >= ny) continue;
            const int off = y * nx + x;
            const int offB = off + hs * nx;
#pragma unroll
            for (int v = 0; v < 4; ++v) us_p[m % NPRE][v] = make_float2(UsA[v * plane + off], UsB[v * plane + offB]);
            if (has_un) {
#pragma unroll
                for (int v = 0; v < 4; ++v) un_p[m % NPRE][v] = make_float2(UnA[v * plane + off], UnB[v * plane + offB]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int y = ty0 + warp + NW * m;
        if (x >= nx || y >= ny) continue;
        const int off = y * nx + x;
        const int offB = off + hs * nx;
        float2 us[4], un[4];
        if (PREF) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                us[v] = us_p[m % NPRE][v];
                un[v] = un_p[m % NPRE][v];
            }
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) us[v] = make_float2(UsA[v * plane + off], UsB[v * plane + offB]);
            if (has_un) {
#pragma unroll
                for (int v = 0; v < 4; ++v) un[v] = make_float2(UnA[v * plane + off], UnB[v * plane + offB]);
            }
        }
        float2 o[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            o[v] = fma2(dt, acc[m][v], us[v]);
            if (has_un) o[v] = fma2(ca, un[v], mul2(cb, o[v]));
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (!doneA) UoA[v * plane + off] = o[v].x;
            if (!doneB) UoB[v * plane + offB] = o[v].y;
        }
        if (want_speed) {
            const float2 inv = rcp2(o[0]);
            const float2 u = mul2(o[1], inv), vv = mul2(o[2], inv);
            const float2 m2 = fma2(o[1], o[1], mul2(o[2], o[2]));
            const float2 pr = mul2(f2(gm1), fma2(mul2(f2(-0.5f), m2), inv, o[3]));
            const bool okx = o[0].x > 0.f && pr.x > 0.f && !isinf(o[0].x) && !isinf(pr.x);
            const bool oky = o[0].y > 0.f && pr.y > 0.f && !isinf(o[0].y) && !isinf(pr.y);
            badA |= !okx;
            badB |= !oky;
            const float2 cs = sound2(gamma, pr, o[0]);
            const float2 s = max2(mul2(add2(abs2(u), cs), f2(idx)), mul2(add2(abs2(vv), cs), f2(idy)));
            smax = make_float2(okx ? fmaxf(smax.x, s.x) : smax.x, oky ? fmaxf(smax.y, s.y) : smax.y);
        }
    }
    if (want_speed) {
        __shared__ float red[NW][2];
        __shared__ int redbad[NW][2];
        float sa = smax.x, sb = smax.y;
        int ba = badA ? 1 : 0, bb = badB ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa = fmaxf(sa, __shfl_xor_sync(0xffffffffu, sa, o));
            sb = fmaxf(sb, __shfl_xor_sync(0xffffffffu, sb, o));
            ba |= __shfl_xor_sync(0xffffffffu, ba, o);
            bb |= __shfl_xor_sync(0xffffffffu, bb, o);
        }
        if (lane == 0) {
            red[warp][0] = sa;
            red[warp][1] = sb;
            redbad[warp][0] = ba;
            redbad[warp][1] = bb;
        }
        __syncthreads();
        if (tid == 0) {
            float ra = red[0][0], rb = red[0][1];
            int xa = redbad[0][0], xb = redbad[0][1];
            for (int k = 1; k < NW; ++k) {
                ra = fmaxf(ra, red[k][0]);
                rb = fmaxf(rb, red[k][1]);
                xa |= redbad[k][0];
                xb |= redbad[k][1];
            }
            const double nanv = __longlong_as_double(0x7fffffffffffffffLL);
            if (!doneA) p.speed_part[L.work0 + (long long)sA * L.tiles + tile] = xa ? nanv : (double)ra;
            const uint32_t tileB = HALVES ? tile + htiles : tile;
            if (!doneB) p.speed_part[L.work0 + (long long)sB * L.tiles + tileB] = xb ? nanv : (double)rb;
        }
    }
}

}  // namespace alsv
