// z-marching SSP-RK stage for 3D Euler (eq. (2.1), Sec. 2.1), FP32.
//
// One CTA owns an x-y tile of TX x TY columns (one thread per column) and a chunk of LZ cells in z.
// It marches up the chunk with a ring of five z-planes of reconstruction variables in shared
// memory, each plane carrying a g = 2 halo in x and y. Per output plane z:
//   1. load plane z + 2 (boundary fill and primitive conversion at load; the ring slot of plane
//      z - 3, whose last reader was two iterations ago);
//   2. the x- and y-interface fluxes of plane z into shared memory (each interface once);
//   3. the z-interface flux at z + 1/2 of the thread's own column from planes z - 1 .. z + 2 (the
//      flux at z - 1/2 is kept in registers from the previous plane);
//   4. divergence, RK combination, coalesced store and (last stage) the CFL speed.
// Every halo cell is loaded and converted 1.7 times per cell (36 x 12 halo plane for 32 x 8 cells)
// instead of 3.4 times for an 8^3 tile, and each interface flux is still evaluated once.
#pragma once

#include "fv_packed3d.cuh"
#include "fv_stage.cuh"

namespace alsv {

// PACK = 1 (primitive reconstruction, HLLC or Rusanov): each thread evaluates the k-th x-interface
// and the k-th y-interface of the plane together in packed FP32x2 arithmetic (lane .x the
// x-interface with normal velocity u, lane .y the y-interface with normal velocity v).
// PACK = 2: as 1 with fewer instructions per interface pair: the ring planes split into a float4
// (rho, u, v, w) and a float (p) array (two shared-memory loads per stencil cell and lane instead
// of five), the x-interfaces mapped as the TX x TY left faces then the right edge column (no
// division by TX + 1), WENO3 faces from the three differences around an interface (faces_d), the
// positivity fallback only when a lane of the warp needs it, and HLLC's star correction through
// the upwind speed. Its x- and y-fluxes round differently from PACK 1 (not bitwise equal to it).
// NTH threads (default: one per column); more threads than columns lets a plane's interface pairs
// fit in one pass (32 x 7 columns: 256 pairs for 256 threads), the threads past the columns only
// take part in the loads and the interfaces.
template <int RECON, int FLUX, int TX, int TY, int LZ, int PACK = 0, int NTH = TX * TY>
__global__ void __launch_bounds__(NTH, 4) k_stage3d_zm(const StageArgs p) {
    using R = float;
    constexpr int ND = 3, NV = 5, G = (RECON == REC_PC) ? 1 : 2;
    constexpr int NT = NTH;
    static_assert(NT >= TX * TY && NT % 32 == 0 && NT / TX <= TY + 2 * G, "threads cover the columns");
    constexpr int SX = TX + 2 * G, SY = TY + 2 * G, PS = SX * SY;   // halo plane
    constexpr int NP = 2 * G + 1;                                    // ring planes
    constexpr int NIX = (TX + 1) * TY, NIY = TX * (TY + 1);
    constexpr int CS = NV;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sW = reinterpret_cast<R*>(smem_raw);      // [NP][PS][CS] (PACK 2: [NP][PS] float4 + [NP][PS] p)
    float4* sW4 = reinterpret_cast<float4*>(smem_raw);
    float* sWp = reinterpret_cast<float*>(sW4 + NP * PS);
    R* sFx = sW + NP * PS * CS;                  // [NIX][CS]
    R* sFy = sFx + NIX * CS;                     // [NIY][CS]
    static_assert(PACK != 2 || CS == 5, "PACK 2 splits five variables as 4 + 1");

    const uint32_t w = blockIdx.x;
    const GridArgs& g = p.g;
    const int l = level_of_work(g, w);
    const LevelInfo& L = g.lev[l];
    const uint32_t wl = w - (uint32_t)L.work0;
    const uint32_t b_local = fdiv(wl, L.fd_tiles);
    const uint32_t tile = wl - b_local * (uint32_t)L.tiles;
    const int sample = L.sample0 + (int)b_local;
    if (p.done[sample]) return;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const uint32_t trow = fdiv(tile, L.fd_nt0);
    const int tx0 = (int)(tile - trow * (uint32_t)L.ntile[0]) * TX;
    const uint32_t tplane = fdiv(trow, L.fd_nt1);
    const int ty0 = (int)(trow - tplane * (uint32_t)L.ntile[1]) * TY;
    const int z0 = (int)tplane * LZ;
    const int z1 = min(z0 + LZ, nz);
    {
        const int c0[3] = {tx0, ty0, z0}, c1[3] = {tx0 + TX, ty0 + TY, z1}, nn[3] = {nx, ny, nz};
        if (!tile_in_part<3>(g, p.part, c0, c1, nn, G)) return;   // uniform per CTA
    }
    const int plane = nx * ny * nz;
    const long long sbase = L.elem0 + (long long)b_local * NV * plane;
    const R* Us = reinterpret_cast<const R*>(p.Us) + sbase;
    const R* Un = reinterpret_cast<const R*>(p.Un) + sbase;
    R* Uo = reinterpret_cast<R*>(p.Uout) + sbase;

    const R gamma = c_gamma<R>(g), gm1 = IsExact<R>::value ? gamma - R(1) : R(g.gm1_f);
    const R inv_gm1 = IsExact<R>::value ? R(1) / gm1 : R(g.inv_gm1_f);
    const int tid = threadIdx.x;
    const int cx = tid % TX, cy = tid / TX;
    const int X = tx0 + cx, Y = ty0 + cy;
    const bool own = cy < TY && X < nx && Y < ny;
    const bool xy_interior = tx0 >= G && tx0 + TX + G <= nx && ty0 >= G && ty0 + TY + G <= ny;
    const int rv = g.rvars;

    // load plane zz (any integer; ghost-mapped in z) into its ring slot
    auto load_plane = [&](int zz) {
        bool fz = false;
        // a plane beyond a halo face of a block comes from that face's halo buffer
        const bool zhalo = (zz < 0 && g.bc[2][0] == BC_HALO) || (zz >= nz && g.bc[2][1] == BC_HALO);
        const int iz = zhalo ? zz : map_ghost(zz, nz, g.bc[2][0], g.bc[2][1], fz);
        const int slot = (zz % NP + NP) % NP;
        R* dst = sW + slot * PS * CS;
#pragma unroll 1
        for (int s = tid; s < PS; s += NT) {
            const int sx = s % SX, sy = s / SX;
            bool flip[3] = {false, false, fz};
            int ix = tx0 + sx - G, iy = ty0 + sy - G;
            const R* src = Us;
            int off = 0, vstride = plane, hf = -1;
            if (!xy_interior || zhalo) {
                hf = halo_cell<3, G>(g, ix, iy, iz, nx, ny, nz, off, vstride);
                if (hf >= 0) {
                    src = reinterpret_cast<const R*>(p.halo[hf]) + (long long)b_local * NV * vstride;
                } else if (!xy_interior) {
                    ix = map_ghost(ix, nx, g.bc[0][0], g.bc[0][1], flip[0]);
                    iy = map_ghost(iy, ny, g.bc[1][0], g.bc[1][1], flip[1]);
                }
            }
            if (hf < 0) off = (iz * ny + iy) * nx + ix;
            R u[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = src[v * vstride + off];
#pragma unroll
            for (int k = 0; k < ND; ++k)
                if (flip[k]) u[1 + k] = -u[1 + k];
            if (PACK == 2) {
                R wv[NV];
                cons_to_prim<R, ND>(u, wv, gm1);
                sW4[slot * PS + s] = make_float4(wv[0], wv[1], wv[2], wv[3]);
                sWp[slot * PS + s] = wv[4];
            } else if (rv == RV_PRIM) {
                R wv[NV];
                cons_to_prim<R, ND>(u, wv, gm1);
#pragma unroll
                for (int v = 0; v < NV; ++v) dst[s * CS + v] = wv[v];
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) dst[s * CS + v] = u[v];
            }
        }
    };
    auto cell_at = [&](int zz, int off, R* out) {
        if (PACK == 2) {
            const int i = ((zz % NP + NP) % NP) * PS + off;
            const float4 a = sW4[i];
            out[0] = a.x;
            out[1] = a.y;
            out[2] = a.z;
            out[3] = a.w;
            out[4] = sWp[i];
            return;
        }
        const R* src = sW + (((zz % NP + NP) % NP) * PS + off) * CS;
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = src[v];
    };
    const int own_off = (cy + G) * SX + cx + G;
    const R epsz = c_eps<R>(g, L, 2), epsx = c_eps<R>(g, L, 0), epsy = c_eps<R>(g, L, 1);
    auto zflux = [&](int zl, R* F) {   // flux at the interface between planes zl and zl + 1
        R cm[NV], cl[NV], cr[NV], c2[NV], WL[NV], WR[NV];
        cell_at(zl, own_off, cl);
        cell_at(zl + 1, own_off, cr);
        if (G == 2) {
            cell_at(zl - 1, own_off, cm);
            cell_at(zl + 2, own_off, c2);
        }
        face_states<R, EQ_EULER, ND, RECON>(cm, cl, cr, c2, rv, gm1, epsz, WL, WR);
        euler_flux<R, ND, 2, FLUX>(WL, WR, F, gamma, gm1, inv_gm1);
    };

    // prologue: planes z0 - G .. z0 + G - 1 and the flux at z0 - 1/2
    for (int zz = z0 - G; zz < z0 + G; ++zz) load_plane(zz);
    __syncthreads();
    R Fzm[NV];
    zflux(z0 - 1, Fzm);

    const R dt = c_dt<R>(p, sample);
    const R ca = c_a<R>(p), cb = c_b<R>(p);
    const bool has_un = p.has_un != 0;
    const bool want_speed = p.want_speed != 0;
    const R idx = c_inv_dx<R>(L, 0), idy = c_inv_dx<R>(L, 1), idz = c_inv_dx<R>(L, 2);
    R smax = R(0);
    bool bad = false;

#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
        load_plane(z + G);
        __syncthreads();
        const int pz = ((z % NP) + NP) % NP;
        const R* sp = sW + pz * PS * CS;
        if constexpr (PACK == 2) {
            static_assert(NIY >= NIX && (TX & (TX - 1)) == 0, "y interfaces outnumber x; TX a power of two");
            const float2 eps2 = make_float2(epsx, epsy);
            const float4* p4 = sW4 + pz * PS;
            const float* pp = sWp + pz * PS;
#pragma unroll 1
            for (int k = tid; k < NIY; k += NT) {
                // x lane: left faces of the TX x TY cells, then the right edge column; past NIX it
                // repeats interface 0 unused
                int fxx = k & (TX - 1), fyx = k / TX;
                if (k >= TX * TY) {
                    fxx = TX;
                    fyx = k - TX * TY;
                }
                const bool hx = fyx < TY;
                if (!hx) fxx = fyx = 0;
                const int i0x = (fyx + G) * SX + fxx + G - 1;
                const int i0y = (k / TX + G - 1) * SX + (k & (TX - 1)) + G;
                F2x5 c[4];
#pragma unroll
                for (int q = (G == 1 ? 1 : 0); q < (G == 1 ? 3 : 4); ++q) {
                    const int ix = i0x + (q - 1), iy = i0y + (q - 1) * SX;
                    const float4 a = p4[ix], b = p4[iy];
                    c[q].r = make_float2(a.x, b.x);
                    c[q].n = make_float2(a.y, b.z);   // normal: u (x-interface), v (y-interface)
                    c[q].t = make_float2(a.z, b.y);   // tangential: v, u
                    c[q].w = make_float2(a.w, b.w);
                    c[q].p = make_float2(pp[ix], pp[iy]);
                }
                if (G == 1) {
                    c[0] = c[1];
                    c[3] = c[2];
                }
                F2x5 WL, WR;
                faces2_5_lean<RECON>(c, eps2, 0xffffffffu, WL, WR);   // whole warps: NIY, NT multiples of 32
                const F2x5 F = FLUX == FLX_HLLC ? hllc2_5_lean(WL, WR, gamma, inv_gm1) : rusanov2_5(WL, WR, gamma, inv_gm1);
                if (hx) {
                    float* o = sFx + (fyx * (TX + 1) + fxx) * CS;
                    o[0] = F.r.x; o[1] = F.n.x; o[2] = F.t.x; o[3] = F.w.x; o[4] = F.p.x;
                }
                float* o = sFy + k * CS;
                o[0] = F.r.y; o[1] = F.t.y; o[2] = F.n.y; o[3] = F.w.y; o[4] = F.p.y;
            }
        } else if constexpr (PACK) {
            static_assert(NIY >= NIX, "the y interfaces outnumber the x interfaces");
            const float2 eps2 = make_float2(epsx, epsy);
#pragma unroll 1
            for (int k = tid; k < NIY; k += NT) {
                const bool hx = k < NIX;            // past NIX the x lane repeats interface 0 unused
                const int kx = hx ? k : 0;
                const int i0x = (kx / (TX + 1) + G) * SX + kx % (TX + 1) + G - 1;
                const int i0y = (k / TX + G - 1) * SX + k % TX + G;
                float2 Rk[4], Nk[4], Tk[4], Wk[4], Pk[4];
#pragma unroll
                for (int q = (G == 1 ? 1 : 0); q < (G == 1 ? 3 : 4); ++q) {
                    const float* ax = sp + (i0x + (q - 1)) * CS;
                    const float* ay = sp + (i0y + (q - 1) * SX) * CS;
                    Rk[q] = make_float2(ax[0], ay[0]);
                    Nk[q] = make_float2(ax[1], ay[2]);   // normal: u (x-interface), v (y-interface)
                    Tk[q] = make_float2(ax[2], ay[1]);   // tangential: v, u
                    Wk[q] = make_float2(ax[3], ay[3]);
                    Pk[q] = make_float2(ax[4], ay[4]);
                }
                if (G == 1) {
                    Rk[0] = Rk[1]; Nk[0] = Nk[1]; Tk[0] = Tk[1]; Wk[0] = Wk[1]; Pk[0] = Pk[1];
                    Rk[3] = Rk[2]; Nk[3] = Nk[2]; Tk[3] = Tk[2]; Wk[3] = Wk[2]; Pk[3] = Pk[2];
                }
                F2x5 fr, fl;
                faces2<RECON>(Rk[0], Rk[1], Rk[2], Rk[3], eps2, fr.r, fl.r);
                faces2<RECON>(Nk[0], Nk[1], Nk[2], Nk[3], eps2, fr.n, fl.n);
                faces2<RECON>(Tk[0], Tk[1], Tk[2], Tk[3], eps2, fr.t, fl.t);
                faces2<RECON>(Wk[0], Wk[1], Wk[2], Wk[3], eps2, fr.w, fl.w);
                faces2<RECON>(Pk[0], Pk[1], Pk[2], Pk[3], eps2, fr.p, fl.p);
                F2x5 WL, WR;
                if (G == 1) {
                    WL = fr;
                    WR = fl;
                } else {
                    // positivity fallback per face and lane: revert to the cell's own state
                    const bool okLx = fr.r.x > 0.f && fr.p.x > 0.f, okLy = fr.r.y > 0.f && fr.p.y > 0.f;
                    const bool okRx = fl.r.x > 0.f && fl.p.x > 0.f, okRy = fl.r.y > 0.f && fl.p.y > 0.f;
                    WL.r = sel2(okLx, okLy, fr.r, Rk[1]);
                    WL.n = sel2(okLx, okLy, fr.n, Nk[1]);
                    WL.t = sel2(okLx, okLy, fr.t, Tk[1]);
                    WL.w = sel2(okLx, okLy, fr.w, Wk[1]);
                    WL.p = sel2(okLx, okLy, fr.p, Pk[1]);
                    WR.r = sel2(okRx, okRy, fl.r, Rk[2]);
                    WR.n = sel2(okRx, okRy, fl.n, Nk[2]);
                    WR.t = sel2(okRx, okRy, fl.t, Tk[2]);
                    WR.w = sel2(okRx, okRy, fl.w, Wk[2]);
                    WR.p = sel2(okRx, okRy, fl.p, Pk[2]);
                }
                const F2x5 F = FLUX == FLX_HLLC ? hllc2_5(WL, WR, gamma, inv_gm1) : rusanov2_5(WL, WR, gamma, inv_gm1);
                if (hx) {
                    float* o = sFx + kx * CS;
                    o[0] = F.r.x; o[1] = F.n.x; o[2] = F.t.x; o[3] = F.w.x; o[4] = F.p.x;
                }
                float* o = sFy + k * CS;
                o[0] = F.r.y; o[1] = F.t.y; o[2] = F.n.y; o[3] = F.w.y; o[4] = F.p.y;
            }
        } else {
        // x interfaces of plane z ((TX + 1) x TY), then its y interfaces (TX x (TY + 1)), as one
        // loop so that only its last pass leaves threads idle before the barrier
#pragma unroll 1
        for (int f = tid; f < NIX + NIY; f += NT) {
            R WL[NV], WR[NV], F[NV];
            if (f < NIX) {
                const int fx = f % (TX + 1), fy = f / (TX + 1);
                const int i0 = (fy + G) * SX + fx + G - 1;
                interface_states<R, EQ_EULER, ND, RECON, CS>(sp, i0, 1, rv, gm1, epsx, WL, WR);
                euler_flux<R, ND, 0, FLUX>(WL, WR, F, gamma, gm1, inv_gm1);
#pragma unroll
                for (int v = 0; v < NV; ++v) sFx[f * CS + v] = F[v];
            } else {
                const int fi = f - NIX;
                const int fx = fi % TX, fy = fi / TX;
                const int i0 = (fy + G - 1) * SX + fx + G;
                interface_states<R, EQ_EULER, ND, RECON, CS>(sp, i0, SX, rv, gm1, epsy, WL, WR);
                euler_flux<R, ND, 1, FLUX>(WL, WR, F, gamma, gm1, inv_gm1);
#pragma unroll
                for (int v = 0; v < NV; ++v) sFy[fi * CS + v] = F[v];
            }
        }
        }
        R Fzp[NV];
        zflux(z, Fzp);
        __syncthreads();
        if (own) {
            const int fxm = cy * (TX + 1) + cx, fym = cy * TX + cx;
            const int off = (z * ny + Y) * nx + X;
            // all reads of the cell first (the last stage writes in place over U^n: each element
            // is read by the thread that writes it, before the write)
            R us[NV], un[NV], out[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) us[v] = Us[v * plane + off];
            if (has_un) {
#pragma unroll
                for (int v = 0; v < NV; ++v) un[v] = Un[v * plane + off];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                // directions accumulated x, y, z as in the tile kernel (same rounding)
                R Lv = R(0);
                Lv = acc_sub<R>(Lv, sFx[(fxm + 1) * CS + v] - sFx[fxm * CS + v], idx);
                Lv = acc_sub<R>(Lv, sFy[(fym + TX) * CS + v] - sFy[fym * CS + v], idy);
                Lv = acc_sub<R>(Lv, Fzp[v] - Fzm[v], idz);
                out[v] = rk_combine<R>(us[v], dt, Lv, has_un, ca, has_un ? un[v] : R(0), cb);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) Uo[v * plane + off] = out[v];
            if (want_speed) {
                R wv[NV];
                cons_to_prim<R, ND>(out, wv, gm1);
                const R rho = wv[0], pr = wv[ND + 1];
                if (!(rho > R(0) && pr > R(0)) || isinf(rho) || isinf(pr)) {
                    bad = true;
                } else {
                    const R c = sound_speed<R>(gamma, pr, rho);
                    smax = fmax_(smax, (fabs_(wv[1]) + c) * idx);
                    smax = fmax_(smax, (fabs_(wv[2]) + c) * idy);
                    smax = fmax_(smax, (fabs_(wv[3]) + c) * idz);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Fzm[v] = Fzp[v];
    }

    if (want_speed) {
        // in R: the maximum of FP32 values converted to double equals the converted maximum, so
        // FP32 kernels keep this reduction off the FP64 pipe
        __shared__ R red[NT / 32];
        __shared__ int redbad[NT / 32];
        R sm = smax;
        int bd = bad ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const R other = __shfl_xor_sync(0xffffffffu, sm, o);
            sm = other > sm ? other : sm;
            bd |= __shfl_xor_sync(0xffffffffu, bd, o);
        }
        if ((tid & 31) == 0) { red[tid >> 5] = sm; redbad[tid >> 5] = bd; }
        __syncthreads();
        if (tid == 0) {
            R r = red[0];
            int rb = redbad[0];
            for (int k = 1; k < NT / 32; ++k) { r = red[k] > r ? red[k] : r; rb |= redbad[k]; }
            p.speed_part[w] = rb ? __longlong_as_double(0x7fffffffffffffffLL) : r;
        }
    }
}

template <int RECON, int TX, int TY, int LZ>
constexpr size_t zm_smem_bytes() {
    constexpr int G = (RECON == REC_PC) ? 1 : 2;
    return sizeof(float) * 5 * ((size_t)(2 * G + 1) * (TX + 2 * G) * (TY + 2 * G) + (TX + 1) * TY + TX * (TY + 1));
}

template <int RECON, int FLUX, int TX, int TY, int LZ, int PACK = 0, int NTH = TX * TY>
static cudaError_t launch_zm_one(const StageArgs& a, cudaStream_t s) {
    auto k = k_stage3d_zm<RECON, FLUX, TX, TY, LZ, PACK, NTH>;
    constexpr size_t sm = zm_smem_bytes<RECON, TX, TY, LZ>();
    static unsigned long long smem_devices = 0;   // devices on which the opt-in is done
    {
        const cudaError_t e = ensure_dynamic_smem(k, sm, smem_devices);
        if (e != cudaSuccess) return e;
    }
    if (a.g.total_work <= 0) return cudaSuccess;
    k<<<(unsigned)a.g.total_work, NTH, sm, s>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY, int LZ>
static cudaError_t launch_stage_zm(int recon, int flux, const StageArgs& a, cudaStream_t s) {
#define ALSV_ZM_FLUX(RC)                                                                     \
    switch (flux) {                                                                          \
        case FLX_RUSANOV: return launch_zm_one<RC, FLX_RUSANOV, TX, TY, LZ>(a, s);           \
        case FLX_HLL: return launch_zm_one<RC, FLX_HLL, TX, TY, LZ>(a, s);                   \
        default: return launch_zm_one<RC, FLX_HLLC, TX, TY, LZ>(a, s);                       \
    }
    switch (recon) {
        case REC_PC: ALSV_ZM_FLUX(REC_PC)
        case REC_MC: ALSV_ZM_FLUX(REC_MC)
        default: ALSV_ZM_FLUX(REC_WENO3)
    }
#undef ALSV_ZM_FLUX
}

// packed x/y interfaces (primitive reconstruction, HLLC or Rusanov); PK 1 or 2 as PACK above
template <int TX, int TY, int LZ, int NTH = TX * TY, int PK = 1>
static cudaError_t launch_stage_zm_packed(int recon, int flux, const StageArgs& a, cudaStream_t s) {
    if (a.g.rvars != RV_PRIM || (flux != FLX_HLLC && flux != FLX_RUSANOV)) return cudaErrorNotSupported;
    if (flux == FLX_HLLC) {
        if (recon == REC_WENO3) return launch_zm_one<REC_WENO3, FLX_HLLC, TX, TY, LZ, PK, NTH>(a, s);
        if (recon == REC_MC) return launch_zm_one<REC_MC, FLX_HLLC, TX, TY, LZ, PK, NTH>(a, s);
        return launch_zm_one<REC_PC, FLX_HLLC, TX, TY, LZ, PK, NTH>(a, s);
    }
    if (recon == REC_WENO3) return launch_zm_one<REC_WENO3, FLX_RUSANOV, TX, TY, LZ, PK, NTH>(a, s);
    if (recon == REC_MC) return launch_zm_one<REC_MC, FLX_RUSANOV, TX, TY, LZ, PK, NTH>(a, s);
    return launch_zm_one<REC_PC, FLX_RUSANOV, TX, TY, LZ, PK, NTH>(a, s);
}

}  // namespace alsv
