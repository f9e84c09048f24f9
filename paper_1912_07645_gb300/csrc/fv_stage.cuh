// Fused SSP-RK stage kernel for eq. (2.1) (Sec. 2.1), one CTA per (sample, tile):
//   1. load the tile plus a ghost halo of g cells (g = 1 for PC, 2 for MC/WENO3) into shared
//      memory, filling ghosts from the boundary conditions and converting to the reconstruction
//      variables (primitive or conserved);
//   2. per direction (x, then y, then z): each thread computes whole interfaces - both face
//      states by reconstruction, positivity fallback, one numerical flux - into a shared flux
//      buffer; every flux is evaluated once per tile and shared by its two cells; each owned cell
//      then accumulates -(F_{i+1/2} - F_{i-1/2}) / dx_k in registers;
//   3. epilogue: Uout = a Un + b (Us + dt L) with coalesced stores, and (last stage) the tile's
//      maximum CFL wave speed of the new state into a fixed per-tile slot.
// Face values and fluxes never touch HBM: per stage the kernel reads Us once (the halo comes from
// L2), Un point-wise, and writes Uout once.
#pragma once

#include "fv_physics.cuh"

namespace alsv {

template <int ND, int TX, int TY, int TZ> struct TileGeom {
    static constexpr int CELLS = TX * TY * TZ;
};

// CFL wave speed (|u_k| + c) / dx_k of one direction
template <class R> __device__ __forceinline__ R speed_over_dx(R s, const LevelInfo& L, int k) {
    if constexpr (IsExact<R>::value) return s / R(L.dx[k]);
    else return s * L.inv_dx_f[k];
}
// the same with the per-direction factor already converted: dx_k (FP64) or 1/dx_k (FP32)
template <class R> __device__ __forceinline__ R speed_dx(R s, R f) {
    if constexpr (IsExact<R>::value) return s / f;
    else return s * f;
}

template <class R> struct RealTraits;
template <> struct RealTraits<float> { static __device__ __forceinline__ float nan() { return __int_as_float(0x7fffffff); } };
template <> struct RealTraits<double> { static __device__ __forceinline__ double nan() { return __longlong_as_double(0x7fffffffffffffffLL); } };

template <class R, int EQ, int ND, int RECON>
struct StageSmem {
    static constexpr int NV = (EQ == EQ_BURGERS) ? 1 : ND + 2;
    static constexpr int G = (RECON == REC_PC) ? 1 : 2;
};

// Shared memory holds one record per cell (all variables of the cell together), padded to 16 bytes
// when that costs at most one element per cell, so a cell moves in 128-bit accesses.
template <class R, int NV> __host__ __device__ constexpr int cell_stride() {
    constexpr int bytes = NV * (int)sizeof(R);
    constexpr int padded = (bytes + 15) / 16 * 16 / (int)sizeof(R);
    return (NV == 1 || bytes % 16 == 0) ? NV : (padded - NV <= 1 ? padded : NV);
}

template <class R, int NV, int CS> __device__ __forceinline__ void lds_cell(const R* p, R* out) {
    if constexpr ((CS * sizeof(R)) % 16 == 0) {
        constexpr int NCH = CS * (int)sizeof(R) / 16;
        R tmp[CS];
#pragma unroll
        for (int c = 0; c < NCH; ++c) reinterpret_cast<uint4*>(tmp)[c] = reinterpret_cast<const uint4*>(p)[c];
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = tmp[v];
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = p[v];
    }
}

template <class R, int NV, int CS> __device__ __forceinline__ void sts_cell(R* p, const R* in) {
    if constexpr ((CS * sizeof(R)) % 16 == 0) {
        constexpr int NCH = CS * (int)sizeof(R) / 16;
        R tmp[CS];
#pragma unroll
        for (int v = 0; v < CS; ++v) tmp[v] = v < NV ? in[v < NV ? v : 0] : R(0);
#pragma unroll
        for (int c = 0; c < NCH; ++c) reinterpret_cast<uint4*>(p)[c] = reinterpret_cast<const uint4*>(tmp)[c];
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) p[v] = in[v];
    }
}

template <class R, int EQ, int ND, int RECON, int TX, int TY, int TZ, int FLUX = FLX_HLLC>
constexpr size_t stage_smem_bytes() {
    constexpr int NV = (EQ == EQ_BURGERS) ? 1 : ND + 2;
    constexpr int CS = cell_stride<R, NV>();
    constexpr int G = ghost_width(RECON, FLUX);
    constexpr int SX = TX + 2 * G, SY = ND >= 2 ? TY + 2 * G : 1, SZ = ND >= 3 ? TZ + 2 * G : 1;
    constexpr int NIX = (TX + 1) * TY * TZ;
    constexpr int NIY = ND >= 2 ? TX * (TY + 1) * TZ : 0;
    constexpr int NIZ = ND >= 3 ? TX * TY * (TZ + 1) : 0;
    constexpr int NI = NIX > NIY ? (NIX > NIZ ? NIX : NIZ) : (NIY > NIZ ? NIY : NIZ);
    return sizeof(R) * (size_t)CS * (size_t)(SX * SY * SZ + NI);
}

// Reconstruct the two face states of interface (left cell i, right cell i+1) from the cell values
// cm = i-1, cl = i, cr = i+1, c2 = i+2 (cm and c2 unused for PC) along one direction, apply the
// positivity fallback, and return primitive states for the flux.
template <class R, int EQ, int ND, int RECON>
__device__ __forceinline__ void face_states(const R* cm, const R* cl, const R* cr, const R* c2, int rvars, R gm1, R eps,
                                            R* WL, R* WR) {
    constexpr int NV = (EQ == EQ_BURGERS) ? 1 : ND + 2;
    constexpr int G = (RECON == REC_PC) ? 1 : 2;
    R fl[NV], fr[NV];
    if (G == 1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { fr[v] = cl[v]; fl[v] = cr[v]; }
    } else {
        if constexpr (RECON == REC_WENO3 && !IsExact<R>::value) {
#pragma unroll
            for (int v = 0; v + 1 < NV; v += 2) {
                float2 a, b;
                weno3_pair2(make_float2(cm[v], cm[v + 1]), make_float2(cl[v], cl[v + 1]),
                            make_float2(cr[v], cr[v + 1]), make_float2(c2[v], c2[v + 1]), f2(eps), a, b);
                fr[v] = a.x; fr[v + 1] = a.y;
                fl[v] = b.x; fl[v + 1] = b.y;
            }
            if constexpr (NV % 2 == 1) weno3_pair(cm[NV - 1], cl[NV - 1], cr[NV - 1], c2[NV - 1], eps, fr[NV - 1], fl[NV - 1]);
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                fr[v] = recon_right<R, RECON>(cm[v], cl[v], cr[v], eps);  // cell i, face i+1/2
                fl[v] = recon_left<R, RECON>(cl[v], cr[v], c2[v], eps);   // cell i+1, face i+1/2
            }
        }
    }
    if (EQ == EQ_BURGERS) {
        WL[0] = fr[0];
        WR[0] = fl[0];
        return;
    }
    constexpr int IP = ND + 1;
    if (G == 1) {  // PC: a face is its cell's value, so the fallback would return the same state
        if (rvars == RV_PRIM) {
#pragma unroll
            for (int v = 0; v < NV; ++v) { WL[v] = cl[v]; WR[v] = cr[v]; }
        } else {
            cons_to_prim<R, ND>(cl, WL, gm1);
            cons_to_prim<R, ND>(cr, WR, gm1);
        }
        return;
    }
    if (rvars == RV_PRIM) {
        const bool okL = fr[0] > R(0) && fr[IP] > R(0);
        const bool okR = fl[0] > R(0) && fl[IP] > R(0);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            WL[v] = okL ? fr[v] : cl[v];
            WR[v] = okR ? fl[v] : cr[v];
        }
    } else {
        R a[NV], b[NV];
        cons_to_prim<R, ND>(fr, a, gm1);
        cons_to_prim<R, ND>(fl, b, gm1);
        const bool okL = a[0] > R(0) && a[IP] > R(0);
        const bool okR = b[0] > R(0) && b[IP] > R(0);
        R ca[NV], cb[NV];
        if (!okL) cons_to_prim<R, ND>(cl, ca, gm1);
        if (!okR) cons_to_prim<R, ND>(cr, cb, gm1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            WL[v] = okL ? a[v] : ca[v];
            WR[v] = okR ? b[v] : cb[v];
        }
    }
}

// The same from shared-memory cell records: i0 = record index of cell i, step = records between
// neighbours along the direction.
template <class R, int EQ, int ND, int RECON, int CS>
__device__ __forceinline__ void interface_states(const R* sw, int i0, int step, int rvars, R gm1, R eps, R* WL,
                                                 R* WR) {
    constexpr int NV = (EQ == EQ_BURGERS) ? 1 : ND + 2;
    constexpr int G = (RECON == REC_PC) ? 1 : 2;
    R cm[NV], cl[NV], cr[NV], c2[NV];
    lds_cell<R, NV, CS>(sw + i0 * CS, cl);
    lds_cell<R, NV, CS>(sw + (i0 + step) * CS, cr);
    if (G == 2) {
        lds_cell<R, NV, CS>(sw + (i0 - step) * CS, cm);
        lds_cell<R, NV, CS>(sw + (i0 + 2 * step) * CS, c2);
    }
    face_states<R, EQ, ND, RECON>(cm, cl, cr, c2, rvars, gm1, eps, WL, WR);
}

// Ghost cell of a block of a decomposed grid (Sec. 2.1, last paragraph; Sec. 3.1): a cell beyond
// a face of kind BC_HALO is read from that face's halo buffer [sample][var][layer][cross], layer l
// of the low face holding index -G + l along the face's direction and of the high face n + l,
// cross = the other directions' cells in (z, y, x) order. Returns the face 2k + side (-1: not a
// halo cell) with the cell's offset and the stride between variables in the buffer. The other
// coordinates are clamped into the block: only tile corners reach outside it there, and the
// direction-by-direction stencils never read tile corners.
template <int ND, int G>
__device__ __forceinline__ int halo_cell(const GridArgs& g, int ix, int iy, int iz, int nx, int ny, int nz, int& off,
                                         int& vstride) {
    const int c[3] = {ix, iy, iz};
    const int n[3] = {nx, ny, nz};
    int f = -1, layer = 0;
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        if (f >= 0) break;
        if (c[k] < 0 && g.bc[k][0] == BC_HALO) {
            f = 2 * k;
            layer = c[k] + G > 0 ? c[k] + G : 0;
        } else if (c[k] >= n[k] && g.bc[k][1] == BC_HALO) {
            f = 2 * k + 1;
            layer = c[k] - n[k] < G - 1 ? c[k] - n[k] : G - 1;
        }
    }
    if (f < 0) return -1;
    int cross = 0, csize = 1;
#pragma unroll
    for (int j = ND - 1; j >= 0; --j) {
        if (j == (f >> 1)) continue;
        const int cj = c[j] < 0 ? 0 : (c[j] >= n[j] ? n[j] - 1 : c[j]);
        cross = cross * n[j] + cj;
        csize *= n[j];
    }
    off = layer * csize + cross;
    vstride = G * csize;
    return f;
}

// entropy-conservative two-point flux along a runtime direction (unrolled loops make D a constant)
template <class R, int ND>
__device__ __forceinline__ void ec_flux_dir(int D, const R* WL, const R* WR, R* F, R gamma) {
    if (D == 0) ec_flux<R, ND, 0>(WL, WR, F, gamma);
    if (D == 1) ec_flux<R, ND, (ND >= 2 ? 1 : 0)>(WL, WR, F, gamma);
    if (D == 2) ec_flux<R, ND, (ND >= 3 ? 2 : 0)>(WL, WR, F, gamma);
}

// RV: reconstruction variables (primitive or conserved) as a compile-time choice, so that each
// instantiation carries only its own conversion path
template <class R, int EQ, int ND, int RECON, int FLUX, int TX, int TY, int TZ, int NT, int RV = RV_PRIM>
__global__ void __launch_bounds__(NT) k_stage(const StageArgs p) {
    constexpr int NV = (EQ == EQ_BURGERS) ? 1 : ND + 2;
    constexpr int G = ghost_width(RECON, FLUX);
    constexpr bool EC = FLUX == FLX_EC || FLUX == FLX_EC4 || FLUX == FLX_TECNO2;   // cell values, no reconstruction
    static_assert(!EC || RV == RV_PRIM, "entropy-conservative fluxes read primitive cell values");
    constexpr int SX = TX + 2 * G, SY = ND >= 2 ? TY + 2 * G : 1, SZ = ND >= 3 ? TZ + 2 * G : 1;
    constexpr int NS = SX * SY * SZ;
    constexpr int NIX = (TX + 1) * TY * TZ;
    constexpr int NIY = ND >= 2 ? TX * (TY + 1) * TZ : 0;
    constexpr int NIZ = ND >= 3 ? TX * TY * (TZ + 1) : 0;
    constexpr int NI = NIX > NIY ? (NIX > NIZ ? NIX : NIZ) : (NIY > NIZ ? NIY : NIZ);
    constexpr int CELLS = TX * TY * TZ;
    static_assert(CELLS % NT == 0, "tile cells must be a multiple of the CTA size");
    constexpr int CPT = CELLS / NT;
    constexpr int CS = cell_stride<R, NV>();

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sW = reinterpret_cast<R*>(smem_raw);   // [NS][CS] reconstruction variables per cell
    R* sF = sW + CS * NS;                      // [NI][CS] interface fluxes

    const uint32_t w = blockIdx.x;  // < 2^31 work items (host-checked)
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
    const uint32_t tplane = ND >= 2 ? fdiv(trow, L.fd_nt1) : 0u;
    const int ty0 = ND >= 2 ? (int)(trow - tplane * (uint32_t)L.ntile[1]) * TY : 0;
    const int tz0 = ND >= 3 ? (int)tplane * TZ : 0;
    {
        const int c0[3] = {tx0, ty0, tz0}, c1[3] = {tx0 + TX, ty0 + TY, tz0 + TZ}, nn[3] = {nx, ny, nz};
        if (!tile_in_part<ND>(g, p.part, c0, c1, nn, G)) return;   // uniform per CTA
    }
    const int plane = nx * ny * nz;  // one sample holds < 2^31 elements (host-checked)
    const long long sbase = L.elem0 + (long long)b_local * NV * plane;
    const R* Us = reinterpret_cast<const R*>(p.Us) + sbase;

    const R gamma = c_gamma<R>(g);
    const R gm1 = IsExact<R>::value ? gamma - R(1) : R(g.gm1_f);
    const R inv_gm1 = IsExact<R>::value ? R(1) / gm1 : R(g.inv_gm1_f);
    const int tid = threadIdx.x;

    // ---- 1. tile + halo load with boundary fill and variable conversion
    // (tiles whose halo lies inside the grid skip the ghost mapping; uniform per CTA)
    const bool interior = tx0 >= G && tx0 + SX - G <= nx && (ND < 2 || (ty0 >= G && ty0 + SY - G <= ny)) &&
                          (ND < 3 || (tz0 >= G && tz0 + SZ - G <= nz));
#pragma unroll 1
    for (int s = tid; s < NS; s += NT) {
        const int sx = s % SX;
        const int sy = ND >= 2 ? (s / SX) % SY : 0;
        const int sz = ND >= 3 ? s / (SX * SY) : 0;
        bool flip[3] = {false, false, false};
        int ix = tx0 + sx - G, iy = ND >= 2 ? ty0 + sy - G : 0, iz = ND >= 3 ? tz0 + sz - G : 0;
        const R* src = Us;
        int off = 0, vstride = plane, hf = -1;
        if (!interior) {
            hf = halo_cell<ND, G>(g, ix, iy, iz, nx, ny, nz, off, vstride);
            if (hf >= 0) {
                src = reinterpret_cast<const R*>(p.halo[hf]) + (long long)b_local * NV * vstride;
            } else {
                ix = map_ghost(ix, nx, g.bc[0][0], g.bc[0][1], flip[0]);
                if (ND >= 2) iy = map_ghost(iy, ny, g.bc[1][0], g.bc[1][1], flip[1]);
                if (ND >= 3) iz = map_ghost(iz, nz, g.bc[2][0], g.bc[2][1], flip[2]);
            }
        }
        if (hf < 0) off = (iz * ny + iy) * nx + ix;
        R u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = src[v * vstride + off];
        if (EQ == EQ_BURGERS) {
            if (flip[0] ^ flip[1] ^ flip[2]) u[0] = -u[0];
            sW[s] = u[0];
        } else {
#pragma unroll
            for (int k = 0; k < ND; ++k)
                if (flip[k]) u[1 + k] = -u[1 + k];
            if (RV == RV_PRIM) {
                R wv[NV];
                cons_to_prim<R, ND>(u, wv, gm1);
                sts_cell<R, NV, CS>(sW + s * CS, wv);
            } else {
                sts_cell<R, NV, CS>(sW + s * CS, u);
            }
        }
    }

    R acc[CPT][NV];
#pragma unroll
    for (int m = 0; m < CPT; ++m)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[m][v] = R(0);

    // ---- 2. per direction: interface fluxes into smem, then divergence into registers
#pragma unroll
    for (int D = 0; D < ND; ++D) {
        __syncthreads();
        const int EX = TX + (D == 0), EY = TY + (D == 1), EZ = TZ + (D == 2);
        const int NID = EX * EY * EZ;
        const int step = D == 0 ? 1 : (D == 1 ? SX : SX * SY);
        const R eps = c_eps<R>(g, L, D);
#pragma unroll 1
        for (int f = tid; f < NID; f += NT) {
            const int fx = f % EX;
            const int fy = ND >= 2 ? (f / EX) % EY : 0;
            const int fz = ND >= 3 ? f / (EX * EY) : 0;
            // left cell of the interface in tile coordinates = (fx,fy,fz) - e_D; smem offset +G
            int cx = fx + G, cy = ND >= 2 ? fy + G : 0, cz = ND >= 3 ? fz + G : 0;
            if (D == 0) cx -= 1;
            if (D == 1) cy -= 1;
            if (D == 2) cz -= 1;
            const int i0 = (cz * SY + cy) * SX + cx;
            R WL[NV], WR[NV], F[NV];
            if constexpr (EC) {
                // entropy-conservative: the two-point flux of the interface's cells; EC4 (fourth
                // order, LeFloch-Mercier-Rohde) 4/3 F(w_i, w_{i+1}) - 1/6 (F(w_{i-1}, w_{i+1}) +
                // F(w_i, w_{i+2}))
                R cl[NV], cr[NV];
                lds_cell<R, NV, CS>(sW + i0 * CS, cl);
                lds_cell<R, NV, CS>(sW + (i0 + step) * CS, cr);
                if constexpr (FLUX == FLX_TECNO2) {
                    // TECNO2: the two-point entropy-conservative flux plus the entropy-stable
                    // diffusion of the ENO2 jump of the scaled entropy variables over four cells
                    R cm[NV], c2[NV];
                    lds_cell<R, NV, CS>(sW + (i0 - step) * CS, cm);
                    lds_cell<R, NV, CS>(sW + (i0 + 2 * step) * CS, c2);
                    if (EQ == EQ_BURGERS) {
                        F[0] = tecno2_burgers<R>(cm[0], cl[0], cr[0], c2[0]);
                    } else {
                        if (D == 0) tecno2_flux<R, ND, 0>(cm, cl, cr, c2, F, gamma);
                        if (D == 1) tecno2_flux<R, ND, (ND >= 2 ? 1 : 0)>(cm, cl, cr, c2, F, gamma);
                        if (D == 2) tecno2_flux<R, ND, (ND >= 3 ? 2 : 0)>(cm, cl, cr, c2, F, gamma);
                    }
                    sts_cell<R, NV, CS>(sF + f * CS, F);
                    continue;
                }
                if (EQ == EQ_BURGERS) F[0] = burgers_flux<R, FLUX>(cl[0], cr[0]);
                else ec_flux_dir<R, ND>(D, cl, cr, F, gamma);
                if constexpr (FLUX == FLX_EC4) {
                    R cm[NV], c2[NV], Fb[NV], Fc[NV];
                    lds_cell<R, NV, CS>(sW + (i0 - step) * CS, cm);
                    lds_cell<R, NV, CS>(sW + (i0 + 2 * step) * CS, c2);
                    if (EQ == EQ_BURGERS) {
                        Fb[0] = burgers_flux<R, FLUX>(cm[0], cr[0]);
                        Fc[0] = burgers_flux<R, FLUX>(cl[0], c2[0]);
                    } else {
                        ec_flux_dir<R, ND>(D, cm, cr, Fb, gamma);
                        ec_flux_dir<R, ND>(D, cl, c2, Fc, gamma);
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v) F[v] = R(4.0 / 3.0) * F[v] - R(1.0 / 6.0) * (Fb[v] + Fc[v]);
                }
                sts_cell<R, NV, CS>(sF + f * CS, F);
                continue;
            }
            interface_states<R, EQ, ND, RECON, CS>(sW, i0, step, RV, gm1, eps, WL, WR);
            if (EQ == EQ_BURGERS) {
                F[0] = burgers_flux<R, FLUX>(WL[0], WR[0]);
            } else {
                if (D == 0) euler_flux<R, ND, 0, FLUX>(WL, WR, F, gamma, gm1, inv_gm1);
                if (D == 1) euler_flux<R, ND, (ND >= 2 ? 1 : 0), FLUX>(WL, WR, F, gamma, gm1, inv_gm1);
                if (D == 2) euler_flux<R, ND, (ND >= 3 ? 2 : 0), FLUX>(WL, WR, F, gamma, gm1, inv_gm1);
            }
            sts_cell<R, NV, CS>(sF + f * CS, F);
        }
        __syncthreads();
        const R inv_dx = c_inv_dx<R>(L, D);
        const R hD = IsExact<R>::value ? R(L.dx[D]) : R(0);
        const int fstep = D == 0 ? 1 : (D == 1 ? TX : TX * TY);
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const int c = tid + m * NT;
            const int x = c % TX;
            const int y = ND >= 2 ? (c / TX) % TY : 0;
            const int z = ND >= 3 ? c / (TX * TY) : 0;
            const int fidx = (z * EY + y) * EX + x;
            R Fm[NV], Fp[NV];
            lds_cell<R, NV, CS>(sF + fidx * CS, Fm);
            lds_cell<R, NV, CS>(sF + (fidx + fstep) * CS, Fp);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const R dF = Fp[v] - Fm[v];
                if constexpr (IsExact<R>::value) acc[m][v] = acc[m][v] - dF / hD;
                else acc[m][v] = acc_sub<R>(acc[m][v], dF, inv_dx);
            }
        }
    }

    // ---- 3. RK combination and store; wave speed of the new state
    const R dt = c_dt<R>(p, sample);
    const R ca = c_a<R>(p), cb = c_b<R>(p);
    const bool has_un = p.has_un != 0;        // loop invariants
    const bool want_speed = p.want_speed != 0;
    R sdx[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) sdx[k] = IsExact<R>::value ? R(L.dx[k]) : c_inv_dx<R>(L, k);
    const R* Un = reinterpret_cast<const R*>(p.Un) + sbase;
    R* Uo = reinterpret_cast<R*>(p.Uout) + sbase;
    R smax = R(0);
    bool bad = false;
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int c = tid + m * NT;
        const int x = tx0 + c % TX;
        const int y = ty0 + (ND >= 2 ? (c / TX) % TY : 0);
        const int z = tz0 + (ND >= 3 ? c / (TX * TY) : 0);
        if (x >= nx || y >= ny || z >= nz) continue;
        const int off = (z * ny + y) * nx + x;
        // all reads of the cell first (the last stage writes in place over U^n: each element is
        // read by the thread that writes it, before the write)
        R us[NV], un[NV], out[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) us[v] = Us[v * plane + off];
        if (has_un) {
#pragma unroll
            for (int v = 0; v < NV; ++v) un[v] = Un[v * plane + off];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            out[v] = rk_combine<R>(us[v], dt, acc[m][v], has_un, ca, has_un ? un[v] : R(0), cb);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Uo[v * plane + off] = out[v];
        if (want_speed) {
            if (EQ == EQ_BURGERS) {
                const R au = fabs_(out[0]);
                if (!(au == au) || isinf(au)) bad = true;
#pragma unroll
                for (int k = 0; k < ND; ++k) smax = fmax_(smax, speed_dx<R>(au, sdx[k]));
            } else {
                R wv[NV];
                cons_to_prim<R, ND>(out, wv, gm1);
                const R rho = wv[0], pr = wv[ND + 1];
                if (!(rho > R(0) && pr > R(0)) || isinf(rho) || isinf(pr)) {
                    bad = true;
                } else {
                    const R c = sound_speed<R>(gamma, pr, rho);
#pragma unroll
                    for (int k = 0; k < ND; ++k) smax = fmax_(smax, speed_dx<R>(fabs_(wv[1 + k]) + c, sdx[k]));
                }
            }
        }
    }
    if (want_speed) {
        // fixed-pattern CTA reduction (max is exact; the pattern is fixed anyway)
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

// Initial wave-speed partials of a state (same tiling as the stage kernel).
template <class R, int EQ, int ND, int TX, int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT) k_speed(const GridArgs g, const void* Uv, double* part) {
    constexpr int NV = (EQ == EQ_BURGERS) ? 1 : ND + 2;
    constexpr int CELLS = TX * TY * TZ;
    constexpr int CPT = CELLS / NT;
    const uint32_t w = blockIdx.x;
    const int l = level_of_work(g, w);
    const LevelInfo& L = g.lev[l];
    const uint32_t wl = w - (uint32_t)L.work0;
    const uint32_t b_local = fdiv(wl, L.fd_tiles);
    const uint32_t tile = wl - b_local * (uint32_t)L.tiles;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const uint32_t trow = fdiv(tile, L.fd_nt0);
    const int tx0 = (int)(tile - trow * (uint32_t)L.ntile[0]) * TX;
    const uint32_t tplane = ND >= 2 ? fdiv(trow, L.fd_nt1) : 0u;
    const int ty0 = ND >= 2 ? (int)(trow - tplane * (uint32_t)L.ntile[1]) * TY : 0;
    const int tz0 = ND >= 3 ? (int)tplane * TZ : 0;
    const int plane = nx * ny * nz;
    const R* U = reinterpret_cast<const R*>(Uv) + L.elem0 + (long long)b_local * NV * plane;
    const R gamma = R(g.gamma), gm1 = gamma - R(1);
    const int tid = threadIdx.x;
    R smax = R(0);
    bool bad = false;
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int c = tid + m * NT;
        const int x = tx0 + c % TX;
        const int y = ty0 + (ND >= 2 ? (c / TX) % TY : 0);
        const int z = tz0 + (ND >= 3 ? c / (TX * TY) : 0);
        if (x >= nx || y >= ny || z >= nz) continue;
        const int off = (z * ny + y) * nx + x;
        R u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = U[v * plane + off];
        if (EQ == EQ_BURGERS) {
            const R au = fabs_(u[0]);
            if (!(au == au) || isinf(au)) bad = true;
#pragma unroll
            for (int k = 0; k < ND; ++k) smax = fmax_(smax, speed_over_dx<R>(au, L, k));
        } else {
            R wv[NV];
            cons_to_prim<R, ND>(u, wv, gm1);
            const R rho = wv[0], pr = wv[ND + 1];
            if (!(rho > R(0) && pr > R(0)) || isinf(rho) || isinf(pr)) {
                bad = true;
            } else {
                const R c = sound_speed<R>(gamma, pr, rho);
#pragma unroll
                for (int k = 0; k < ND; ++k) smax = fmax_(smax, speed_over_dx<R>(fabs_(wv[1 + k]) + c, L, k));
            }
        }
    }
    __shared__ R red[NT / 32];   // in R: see k_stage's reduction
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
        part[w] = rb ? __longlong_as_double(0x7fffffffffffffffLL) : r;
    }
}

}  // namespace alsv
