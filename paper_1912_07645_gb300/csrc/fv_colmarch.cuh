// Column-marching SSP-RK stage for 2D Euler in FP32 on periodic grids (primitive reconstruction,
// WENO3 or MC, HLLC or Rusanov): the same eq. (2.1) stage as k_stage, scheduled differently.
//
// One warp owns a strip of 31 columns of one sample and marches down all rows. Lane l holds column
// x0 + l (lanes 0..30 own their cells; lane 31 only supplies the right face of lane 30's cell).
// A per-warp ring of four rows (plus two halo columns on the left and one on the right) in shared
// memory holds primitive states. At row j every lane evaluates two interfaces at once with packed
// FP32x2 arithmetic: lane.x = its x-interface x-1/2 (stencil along the row) and lane.y = its
// y-interface j+1/2 (stencil down the column), both in (normal, tangential) coordinates, so one
// flux evaluation serves both directions. The right x-face of a cell is the left face of the next
// lane (one shuffle); the lower y-face is the upper face of the previous row (kept in registers).
// Only __syncwarp orders the ring; warps never wait for each other.
#pragma once

#include "fv_packed.cuh"

namespace alsv {

constexpr int kColOwned = 31;       // owned columns per strip
constexpr int kColWarps = 4;        // strips per CTA
constexpr int kColRing = 35;        // ring row width: columns x0-2 .. x0+32

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

template <int RECON, int FLUX>
__global__ void __launch_bounds__(32 * kColWarps) k_stage2d_col(const StageArgs p) {
    __shared__ __align__(16) float ring[kColWarps][4][kColRing][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GridArgs& g = p.g;
    const uint32_t w = blockIdx.x * kColWarps + warp;
    if ((long long)w >= g.total_work) return;  // whole warp
    const int l = level_of_work(g, w);
    const LevelInfo& Lv = g.lev[l];
    const uint32_t wl = w - (uint32_t)Lv.work0;
    const uint32_t b_local = fdiv(wl, Lv.fd_tiles);
    const uint32_t strip = wl - b_local * (uint32_t)Lv.tiles;
    const int sample = Lv.sample0 + (int)b_local;
    if (p.done[sample]) return;  // whole warp
    const int nx = Lv.n[0], ny = Lv.n[1];
    const int plane = nx * ny;
    const long long sbase = Lv.elem0 + (long long)b_local * 4 * plane;
    const float* Us = reinterpret_cast<const float*>(p.Us) + sbase;
    const float* Un = reinterpret_cast<const float*>(p.Un) + sbase;
    float* Uo = reinterpret_cast<float*>(p.Uout) + sbase;
    const float gamma = g.gamma_f, gm1 = g.gm1_f, inv_gm1 = g.inv_gm1_f;
    const float2 eps = make_float2(Lv.eps_f[0], Lv.eps_f[1]);
    const float idx = Lv.inv_dx_f[0], idy = Lv.inv_dx_f[1];
    const float dt = p.dt_f[sample], ca = p.a_f, cb = p.b_f;
    const bool has_un = p.has_un != 0, want_speed = p.want_speed != 0;

    const int x0 = (int)strip * kColOwned;
    const int xs = x0 + lane;                  // this lane's column (>= nx on a partial last strip)
    const bool owns = lane < kColOwned && xs < nx;
    const int xc = xs % nx;                    // periodic
    // halo columns carried by lanes 0, 1, 2: x0-2, x0-1, x0+32 (periodic)
    const int xh_raw = lane == 0 ? x0 - 2 : (lane == 1 ? x0 - 1 : x0 + 32);
    const int xh = ((xh_raw % nx) + nx) % nx;
    const bool has_halo = lane < 3;
    const int rc = lane + 2;                   // ring column of this lane
    const int rh = lane == 0 ? 0 : (lane == 1 ? 1 : 34);
    float (*rg)[kColRing][4] = ring[warp];

    auto wrap_row = [&](int j) {
        int jr = j % ny;
        return jr < 0 ? jr + ny : jr;
    };
    // raw conserved loads of one row (own column, and the halo column on lanes 0..2)
    auto fetch = [&](int j, float4& own, float4& halo) {
        const int jr = wrap_row(j);
        const int o = jr * nx + xc;
        own = make_float4(Us[o], Us[plane + o], Us[2 * plane + o], Us[3 * plane + o]);
        if (has_halo) {
            const int oh = jr * nx + xh;
            halo = make_float4(Us[oh], Us[plane + oh], Us[2 * plane + oh], Us[3 * plane + oh]);
        }
    };
    auto insert = [&](int j, const float4& own, const float4& halo) {
        float u[4] = {own.x, own.y, own.z, own.w}, wv[4];
        cons_to_prim<float, 2>(u, wv, gm1);
        *reinterpret_cast<float4*>(rg[j & 3][rc]) = make_float4(wv[0], wv[1], wv[2], wv[3]);
        if (has_halo) {
            float uh[4] = {halo.x, halo.y, halo.z, halo.w};
            cons_to_prim<float, 2>(uh, wv, gm1);
            *reinterpret_cast<float4*>(rg[j & 3][rh]) = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
    };

    // interface pair at row j: x-interface (xs-1/2, j) and y-interface (xs, j+1/2)
    auto fluxes = [&](int j, float4& Fx, float4& Gy) {
        const float4 a0 = lds4(rg[j & 3][rc - 2]), a1 = lds4(rg[j & 3][rc - 1]);
        const float4 a2 = lds4(rg[j & 3][rc]), a3 = lds4(rg[j & 3][rc + 1]);
        const float4 b0 = lds4(rg[(j - 1) & 3][rc]), b1 = a2;
        const float4 b2 = lds4(rg[(j + 1) & 3][rc]), b3 = lds4(rg[(j + 2) & 3][rc]);
        // packed (row stencil, column stencil) in (rho, normal, tangential, p)
        F2x4 fr, fl;
        faces2<RECON>(make_float2(a0.x, b0.x), make_float2(a1.x, b1.x), make_float2(a2.x, b2.x), make_float2(a3.x, b3.x),
                      eps, fr.r, fl.r);
        faces2<RECON>(make_float2(a0.y, b0.z), make_float2(a1.y, b1.z), make_float2(a2.y, b2.z), make_float2(a3.y, b3.z),
                      eps, fr.n, fl.n);
        faces2<RECON>(make_float2(a0.z, b0.y), make_float2(a1.z, b1.y), make_float2(a2.z, b2.y), make_float2(a3.z, b3.y),
                      eps, fr.t, fl.t);
        faces2<RECON>(make_float2(a0.w, b0.w), make_float2(a1.w, b1.w), make_float2(a2.w, b2.w), make_float2(a3.w, b3.w),
                      eps, fr.p, fl.p);
        // positivity fallback per face: revert to the cell's own state
        const bool okLx = fr.r.x > 0.f && fr.p.x > 0.f, okLy = fr.r.y > 0.f && fr.p.y > 0.f;
        const bool okRx = fl.r.x > 0.f && fl.p.x > 0.f, okRy = fl.r.y > 0.f && fl.p.y > 0.f;
        F2x4 WL, WR;
        WL.r = sel2(okLx, okLy, fr.r, make_float2(a1.x, b1.x));
        WL.n = sel2(okLx, okLy, fr.n, make_float2(a1.y, b1.z));
        WL.t = sel2(okLx, okLy, fr.t, make_float2(a1.z, b1.y));
        WL.p = sel2(okLx, okLy, fr.p, make_float2(a1.w, b1.w));
        WR.r = sel2(okRx, okRy, fl.r, make_float2(a2.x, b2.x));
        WR.n = sel2(okRx, okRy, fl.n, make_float2(a2.y, b2.z));
        WR.t = sel2(okRx, okRy, fl.t, make_float2(a2.z, b2.y));
        WR.p = sel2(okRx, okRy, fl.p, make_float2(a2.w, b2.w));
        const F2x4 F = FLUX == FLX_HLLC ? hllc2(WL, WR, gamma, inv_gm1) : rusanov2(WL, WR, gamma, inv_gm1);
        Fx = make_float4(F.r.x, F.n.x, F.t.x, F.p.x);   // (mass, x-momentum, y-momentum, energy)
        Gy = make_float4(F.r.y, F.t.y, F.n.y, F.p.y);
    };

    // prologue: rows -2 .. 1 in the ring, row 2 in flight, lower y-face of row 0
    float4 own, halo = make_float4(0.f, 0.f, 0.f, 0.f), cq0, cq1;
    fetch(-2, own, halo);
    insert(-2, own, halo);
    fetch(-1, own, halo);
    insert(-1, own, halo);
    fetch(0, own, halo);
    insert(0, own, halo);
    cq0 = own;
    fetch(1, own, halo);
    insert(1, own, halo);
    cq1 = own;
    float4 pend_own, pend_halo = halo;
    fetch(2, pend_own, pend_halo);
    __syncwarp();
    float4 Fx, Gprev;
    {
        float4 unused;
        fluxes(-1, unused, Gprev);
    }
    float smax = 0.0f;
    bool bad = false;
    for (int j = 0; j < ny; ++j) {
        __syncwarp();                      // every lane finished reading row j-2's slot
        insert(j + 2, pend_own, pend_halo);
        const float4 cq2 = pend_own;
        __syncwarp();
        if (j + 3 <= ny + 1) fetch(j + 3, pend_own, pend_halo);   // in flight during this row
        float4 G;
        fluxes(j, Fx, G);
        float4 Fr;
        Fr.x = __shfl_down_sync(0xffffffffu, Fx.x, 1);
        Fr.y = __shfl_down_sync(0xffffffffu, Fx.y, 1);
        Fr.z = __shfl_down_sync(0xffffffffu, Fx.z, 1);
        Fr.w = __shfl_down_sync(0xffffffffu, Fx.w, 1);
        if (owns) {
            const float Lq[4] = {-(Fr.x - Fx.x) * idx - (G.x - Gprev.x) * idy, -(Fr.y - Fx.y) * idx - (G.y - Gprev.y) * idy,
                                 -(Fr.z - Fx.z) * idx - (G.z - Gprev.z) * idy, -(Fr.w - Fx.w) * idx - (G.w - Gprev.w) * idy};
            const float us[4] = {cq0.x, cq0.y, cq0.z, cq0.w};
            const int o = j * nx + xs;
            float out[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                float q = us[v] + dt * Lq[v];
                if (has_un) q = ca * Un[v * plane + o] + cb * q;
                out[v] = q;
                Uo[v * plane + o] = q;
            }
            if (want_speed) {
                float wv[4];
                cons_to_prim<float, 2>(out, wv, gm1);
                if (!(wv[0] > 0.f && wv[3] > 0.f) || isinf(wv[0]) || isinf(wv[3])) {
                    bad = true;
                } else {
                    const float c = sound_speed<float>(gamma, wv[3], wv[0]);
                    smax = fmaxf(smax, fmaxf((fabsf(wv[1]) + c) * idx, (fabsf(wv[2]) + c) * idy));
                }
            }
        }
        Gprev = G;
        cq0 = cq1;
        cq1 = cq2;
    }
    if (want_speed) {
        float sm = smax;
        int bd = bad ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
            bd |= __shfl_xor_sync(0xffffffffu, bd, o);
        }
        if (lane == 0) p.speed_part[w] = bd ? __longlong_as_double(0x7fffffffffffffffLL) : (double)sm;
    }
}

// Initial wave-speed partials with the column tiling (one warp per strip).
__global__ void __launch_bounds__(32 * kColWarps) k_speed2d_col(const GridArgs g, const void* Uv, double* part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t w = blockIdx.x * kColWarps + warp;
    if ((long long)w >= g.total_work) return;
    const int l = level_of_work(g, w);
    const LevelInfo& Lv = g.lev[l];
    const uint32_t wl = w - (uint32_t)Lv.work0;
    const uint32_t b_local = fdiv(wl, Lv.fd_tiles);
    const uint32_t strip = wl - b_local * (uint32_t)Lv.tiles;
    const int nx = Lv.n[0], ny = Lv.n[1];
    const int plane = nx * ny;
    const float* U = reinterpret_cast<const float*>(Uv) + Lv.elem0 + (long long)b_local * 4 * plane;
    const float gamma = (float)g.gamma, gm1 = gamma - 1.0f;
    const float idx = (float)Lv.inv_dx[0], idy = (float)Lv.inv_dx[1];
    const int xs = (int)strip * kColOwned + lane;
    const bool owns = lane < kColOwned && xs < nx;
    float smax = 0.0f;
    bool bad = false;
    if (owns) {
        for (int j = 0; j < ny; ++j) {
            const int o = j * nx + xs;
            float u[4] = {U[o], U[plane + o], U[2 * plane + o], U[3 * plane + o]};
            float wv[4];
            cons_to_prim<float, 2>(u, wv, gm1);
            if (!(wv[0] > 0.f && wv[3] > 0.f) || isinf(wv[0]) || isinf(wv[3])) {
                bad = true;
            } else {
                const float c = sound_speed<float>(gamma, wv[3], wv[0]);
                smax = fmaxf(smax, fmaxf((fabsf(wv[1]) + c) * idx, (fabsf(wv[2]) + c) * idy));
            }
        }
    }
    float sm = smax;
    int bd = bad ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
        bd |= __shfl_xor_sync(0xffffffffu, bd, o);
    }
    if (lane == 0) part[w] = bd ? __longlong_as_double(0x7fffffffffffffffLL) : (double)sm;
}

}  // namespace alsv
