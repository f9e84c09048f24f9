// Two-sample SSP-RK stage for 2D Euler in FP32 (primitive reconstruction PC/MC/WENO3, HLLC or
// Rusanov, any boundary conditions): the same eq. (2.1) stage as k_stage, with two Monte Carlo
// samples of the batch advanced together by every thread. Lane .x of each packed FP32x2 value is
// sample A, lane .y sample B, so every arithmetic instruction serves both samples and all index
// and address arithmetic is shared. Shared memory interleaves the pair: one cell is two float4,
// (rho_A, rho_B, u_A, u_B) and (v_A, v_B, p_A, p_B), which load straight into register pairs; the
// two halves live in separate arrays so neighbouring cells are 16 bytes apart (conflict-free).
// Tile structure as k_stage: halo load with boundary fill, per-direction interface fluxes in shared
// memory (each evaluated once), divergence in registers, RK combination, CFL partials per sample.
#pragma once

#include "fv_packed.cuh"

namespace alsv {

template <int RECON, int TX, int TY>
constexpr size_t pair_smem_bytes() {
    constexpr int G = RECON == REC_PC ? 1 : 2;
    constexpr int NS = (TX + 2 * G) * (TY + 2 * G);
    constexpr int NIX = (TX + 1) * TY, NIY = TX * (TY + 1);
    constexpr int NI = NIX > NIY ? NIX : NIY;
    return (size_t)32 * (NS + NI);
}

// HALVES = 1: the pair is one sample's tile in the lower half of a y-periodic grid (lane .x) and
// the tile ny/2 rows above it (lane .y); every level needs ny divisible by 2 TY.
// 32x16 tiles run 4 CTAs per SM with up to 64 registers (no spills with the loads hoisted);
// 32x8 tiles 5 CTAs (measured best for each)
template <int RECON, int FLUX, int TX, int TY, int NT, int HALVES = 0>
__global__ void __launch_bounds__(NT, TY >= 16 ? 4 : 5) k_stage2d_pair(const StageArgs p) {
    constexpr int G = RECON == REC_PC ? 1 : 2;
    constexpr int SX = TX + 2 * G, SY = TY + 2 * G, NS = SX * SY;
    constexpr int NIX = (TX + 1) * TY, NIY = TX * (TY + 1);
    constexpr int NI = NIX > NIY ? NIX : NIY;
    constexpr int CELLS = TX * TY;
    static_assert(CELLS % NT == 0, "tile cells must be a multiple of the CTA size");
    constexpr int CPT = CELLS / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* sW0 = reinterpret_cast<float4*>(smem_raw);  // [NS] (rho, u) of both samples
    float4* sW1 = sW0 + NS;                              // [NS] (v, p)
    float4* sF0 = sW1 + NS;                              // [NI] (mass, x-momentum) fluxes
    float4* sF1 = sF0 + NI;                              // [NI] (y-momentum, energy)

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
    const bool doneA = p.done[L.sample0 + sA] != 0;
    const bool doneB = hasB ? p.done[L.sample0 + sB] != 0 : true;
    if (doneA && doneB) return;

    const int nx = L.n[0], ny = L.n[1];
    const uint32_t trow = fdiv(tile, L.fd_nt0);
    const int tx0 = (int)(tile - trow * (uint32_t)L.ntile[0]) * TX;
    const int ty0 = (int)trow * TY;
    const int plane = nx * ny;
    const int hs = HALVES ? ny / 2 : 0;   // row shift of lane .y (halves)
    const long long bA = L.elem0 + (long long)sA * 4 * plane, bB = L.elem0 + (long long)sB * 4 * plane;
    const float* UsA = reinterpret_cast<const float*>(p.Us) + bA;
    const float* UsB = reinterpret_cast<const float*>(p.Us) + bB;
    const float gamma = g.gamma_f, gm1 = g.gm1_f, inv_gm1 = g.inv_gm1_f;
    const int tid = threadIdx.x;

    // ---- 1. tile + halo load (both samples), boundary fill, primitive conversion. The loads of
    // a group of LG halo cells are all issued before the first is used, so they are in flight
    // together instead of one cell's round trip at a time.
    const bool interior = tx0 >= G && tx0 + SX - G <= nx && ty0 >= G && ty0 + SY - G <= ny;
    constexpr int ITER = (NS + NT - 1) / NT;
    constexpr int LG = ITER < 2 ? ITER : 2;
#pragma unroll 1
    for (int it0 = 0; it0 < ITER; it0 += LG) {
        float2 r[LG], mx[LG], my[LG], E[LG];
        bool fxs[LG], fys[LG];
#pragma unroll
        for (int j = 0; j < LG; ++j) {
            const int s = tid + (it0 + j) * NT;
            fxs[j] = false;
            fys[j] = false;
            if (s < NS) {
                const int sx = s % SX, sy = s / SX;
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
            const int s = tid + (it0 + j) * NT;
            if (s >= NS) continue;
            float2 mxj = mx[j], myj = my[j];
            if (fxs[j]) mxj = neg2(mxj);
            if (fys[j]) myj = neg2(myj);
            const float2 inv = rcp2(r[j]);
            const float2 u = mul2(mxj, inv), v = mul2(myj, inv);
            const float2 m2 = fma2(mxj, mxj, mul2(myj, myj));
            const float2 pr = mul2(f2(gm1), fma2(mul2(f2(-0.5f), m2), inv, E[j]));
            sW0[s] = make_float4(r[j].x, r[j].y, u.x, u.y);
            sW1[s] = make_float4(v.x, v.y, pr.x, pr.y);
        }
    }

    float2 acc[CPT][4];
#pragma unroll
    for (int m = 0; m < CPT; ++m)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[m][v] = f2(0.f);

#pragma unroll
    for (int D = 0; D < 2; ++D) {
        __syncthreads();
        const int EX = TX + (D == 0), EY = TY + (D == 1);
        const int NID = EX * EY;
        const int step = D == 0 ? 1 : SX;
        const float epsD = L.eps_f[D];
        const float2 eps = f2(epsD);
#pragma unroll 1
        for (int f = tid; f < NID; f += NT) {
            const int fx = f % EX, fy = f / EX;
            const int cx = fx + G - (D == 0 ? 1 : 0), cy = fy + G - (D == 1 ? 1 : 0);
            const int i0 = cy * SX + cx;   // left cell of the interface
            // stencil cells i-1, i, i+1, i+2 (PC: i, i+1); rho, u, v, p for both samples
            float2 Rk[4], Uk[4], Vk[4], Pk[4];
#pragma unroll
            for (int k = (G == 1 ? 1 : 0); k < (G == 1 ? 3 : 4); ++k) {
                const int idx = i0 + (k - 1) * step;
                const float4 a = sW0[idx], b = sW1[idx];
                Rk[k] = make_float2(a.x, a.y);
                Uk[k] = make_float2(a.z, a.w);
                Vk[k] = make_float2(b.x, b.y);
                Pk[k] = make_float2(b.z, b.w);
            }
            if (G == 1) {
                Rk[0] = Rk[1]; Uk[0] = Uk[1]; Vk[0] = Vk[1]; Pk[0] = Pk[1];
                Rk[3] = Rk[2]; Uk[3] = Uk[2]; Vk[3] = Vk[2]; Pk[3] = Pk[2];
            }
            F2x4 fr, fl;
            faces2<RECON>(Rk[0], Rk[1], Rk[2], Rk[3], eps, fr.r, fl.r);
            // normal / tangential velocity of this direction
            faces2<RECON>(D == 0 ? Uk[0] : Vk[0], D == 0 ? Uk[1] : Vk[1], D == 0 ? Uk[2] : Vk[2], D == 0 ? Uk[3] : Vk[3],
                          eps, fr.n, fl.n);
            faces2<RECON>(D == 0 ? Vk[0] : Uk[0], D == 0 ? Vk[1] : Uk[1], D == 0 ? Vk[2] : Uk[2], D == 0 ? Vk[3] : Uk[3],
                          eps, fr.t, fl.t);
            faces2<RECON>(Pk[0], Pk[1], Pk[2], Pk[3], eps, fr.p, fl.p);
            F2x4 WL, WR;
            if (G == 1) {
                WL = fr;
                WR = fl;
            } else {
                // positivity fallback per face and per sample: revert to the cell's own state
                const bool okLx = fr.r.x > 0.f && fr.p.x > 0.f, okLy = fr.r.y > 0.f && fr.p.y > 0.f;
                const bool okRx = fl.r.x > 0.f && fl.p.x > 0.f, okRy = fl.r.y > 0.f && fl.p.y > 0.f;
                WL.r = sel2(okLx, okLy, fr.r, Rk[1]);
                WL.n = sel2(okLx, okLy, fr.n, D == 0 ? Uk[1] : Vk[1]);
                WL.t = sel2(okLx, okLy, fr.t, D == 0 ? Vk[1] : Uk[1]);
                WL.p = sel2(okLx, okLy, fr.p, Pk[1]);
                WR.r = sel2(okRx, okRy, fl.r, Rk[2]);
                WR.n = sel2(okRx, okRy, fl.n, D == 0 ? Uk[2] : Vk[2]);
                WR.t = sel2(okRx, okRy, fl.t, D == 0 ? Vk[2] : Uk[2]);
                WR.p = sel2(okRx, okRy, fl.p, Pk[2]);
            }
            const F2x4 F = FLUX == FLX_HLLC ? hllc2(WL, WR, gamma, inv_gm1) : rusanov2(WL, WR, gamma, inv_gm1);
            const float2 fxm = D == 0 ? F.n : F.t, fym = D == 0 ? F.t : F.n;
            sF0[f] = make_float4(F.r.x, F.r.y, fxm.x, fxm.y);
            sF1[f] = make_float4(fym.x, fym.y, F.p.x, F.p.y);
        }
        __syncthreads();
        const float2 nidx = f2(-L.inv_dx_f[D]);
        const int fstep = D == 0 ? 1 : TX;
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const int c = tid + m * NT;
            const int x = c % TX, y = c / TX;
            const int fidx = y * EX + x;
            const float4 am = sF0[fidx], bm = sF1[fidx];
            const float4 ap = sF0[fidx + fstep], bp = sF1[fidx + fstep];
            acc[m][0] = fma2(sub2(make_float2(ap.x, ap.y), make_float2(am.x, am.y)), nidx, acc[m][0]);
            acc[m][1] = fma2(sub2(make_float2(ap.z, ap.w), make_float2(am.z, am.w)), nidx, acc[m][1]);
            acc[m][2] = fma2(sub2(make_float2(bp.x, bp.y), make_float2(bm.x, bm.y)), nidx, acc[m][2]);
            acc[m][3] = fma2(sub2(make_float2(bp.z, bp.w), make_float2(bm.z, bm.w)), nidx, acc[m][3]);
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
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int c = tid + m * NT;
        const int x = tx0 + c % TX, y = ty0 + c / TX;
        if (x >= nx || y >= ny) continue;
        const int off = y * nx + x;
        const int offB = off + hs * nx;   // lower-half rows: y + ny/2 < ny
        // all reads of the cell first (the last stage writes in place over U^n: each element is
        // read by the thread that writes it, before the write)
        float2 us[4], un[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) us[v] = make_float2(UsA[v * plane + off], UsB[v * plane + offB]);
        if (has_un) {
#pragma unroll
            for (int v = 0; v < 4; ++v) un[v] = make_float2(UnA[v * plane + off], UnB[v * plane + offB]);
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
        __shared__ float red[NT / 32][2];
        __shared__ int redbad[NT / 32][2];
        float sa = smax.x, sb = smax.y;
        int ba = badA ? 1 : 0, bb = badB ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa = fmaxf(sa, __shfl_xor_sync(0xffffffffu, sa, o));
            sb = fmaxf(sb, __shfl_xor_sync(0xffffffffu, sb, o));
            ba |= __shfl_xor_sync(0xffffffffu, ba, o);
            bb |= __shfl_xor_sync(0xffffffffu, bb, o);
        }
        if ((tid & 31) == 0) {
            red[tid >> 5][0] = sa;
            red[tid >> 5][1] = sb;
            redbad[tid >> 5][0] = ba;
            redbad[tid >> 5][1] = bb;
        }
        __syncthreads();
        if (tid == 0) {
            float ra = red[0][0], rb = red[0][1];
            int xa = redbad[0][0], xb = redbad[0][1];
            for (int k = 1; k < NT / 32; ++k) {
                ra = fmaxf(ra, red[k][0]);
                rb = fmaxf(rb, red[k][1]);
                xa |= redbad[k][0];
                xb |= redbad[k][1];
            }
            const double nanv = __longlong_as_double(0x7fffffffffffffffLL);
            if (!doneA) p.speed_part[L.work0 + (long long)sA * L.tiles + tile] = xa ? nanv : (double)ra;
            const uint32_t tileB = HALVES ? tile + htiles : tile;   // the tile ny/2 rows above
            if (!doneB) p.speed_part[L.work0 + (long long)sB * L.tiles + tileB] = xb ? nanv : (double)rb;
        }
    }
}

}  // namespace alsv
