// Discrete adjoint of the fixed-dt SSP-RK finite-volume scheme (eq. (2.1), Sec. 2.1) for 2D
// Euler on a periodic grid with PC or MC reconstruction and the Rusanov flux, giving the gradient
// of the kinetic energy at T with respect to the Kelvin-Helmholtz perturbation parameters.
// (The paper has no adjoint; this is the differentiation path of the method's forward map.)
//
// Reverse mode is written by hand, statement by statement against the forward code, with the
// active-branch rule at kinks (limiter selection, max of the Rusanov wave speeds, |u|, clamp of
// the volume fractions, positivity fallback). J_L^T lambda is formed as a gather: each interface
// writes its contributions to the cells of its stencil into shared memory, then every cell sums
// the contributions of the interfaces that touch it in a fixed order - no atomics.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "alsv_ctx.h"
#include "fv_physics.cuh"

namespace alsv {

// ---------------------------------------------------------------------------------------------
// Device VJP helpers (2D Euler, 4 variables: rho, m_x, m_y, E / rho, u, v, p)
// ---------------------------------------------------------------------------------------------
// W = prim(U): Ubar += (dW/dU)^T Wbar
template <class R> __device__ __forceinline__ void prim_vjp(const R* U, const R* Wb, R* Ub, R gm1) {
    R inv;
    if constexpr (IsExact<R>::value) inv = R(1) / U[0];
    else inv = rcp_approx(U[0]);   // FP32: the forward's own fast reciprocal
    const R u = U[1] * inv, v = U[2] * inv;
    Ub[0] += Wb[0] - Wb[1] * u * inv - Wb[2] * v * inv + Wb[3] * gm1 * R(0.5) * (u * u + v * v);
    Ub[1] += Wb[1] * inv - Wb[3] * gm1 * u;
    Ub[2] += Wb[2] * inv - Wb[3] * gm1 * v;
    Ub[3] += Wb[3] * gm1;
}

// U = cons(W): Wbar += (dU/dW)^T Ubar
template <class R> __device__ __forceinline__ void cons_vjp(const R* W, const R* Ub, R* Wb, R inv_gm1) {
    Wb[0] += Ub[0] + Ub[1] * W[1] + Ub[2] * W[2] + Ub[3] * R(0.5) * (W[1] * W[1] + W[2] * W[2]);
    Wb[1] += Ub[1] * W[0] + Ub[3] * W[0] * W[1];
    Wb[2] += Ub[2] * W[0] + Ub[3] * W[0] * W[2];
    Wb[3] += Ub[3] * inv_gm1;
}

// physical flux along D (normal N = 1 + D, tangential T = 2 - D): Wbar += (dF/dW)^T Fbar
template <class R, int D>
__device__ __forceinline__ void phys_flux_vjp(const R* W, const R* Fb, R* Wb, R inv_gm1) {
    constexpr int N = 1 + D, T = 2 - D;
    const R rho = W[0], un = W[N], ut = W[T], p = W[3];
    const R q2 = un * un + ut * ut;
    const R E = p * inv_gm1 + R(0.5) * rho * q2;
    Wb[0] += Fb[0] * un + Fb[N] * un * un + Fb[T] * ut * un + Fb[3] * un * R(0.5) * q2;
    Wb[N] += Fb[0] * rho + Fb[N] * R(2) * rho * un + Fb[T] * rho * ut + Fb[3] * (E + p + rho * un * un);
    Wb[T] += Fb[T] * rho * un + Fb[3] * un * rho * ut;
    Wb[3] += Fb[N] + Fb[3] * un * (inv_gm1 + R(1));
}

// Rusanov flux F = (F(UL) + F(UR))/2 - a (UR - UL)/2, a = max(|uL|+cL, |uR|+cR) (ties pick L)
template <class R, int D>
__device__ __forceinline__ void rusanov_vjp(const R* WL, const R* WR, const R* Fb, R* WLb, R* WRb, R gamma,
                                            R inv_gm1) {
    constexpr int N = 1 + D;
    R UL[4], UR[4];
    prim_to_cons<R, 2>(WL, UL, R(1) / inv_gm1, inv_gm1);
    prim_to_cons<R, 2>(WR, UR, R(1) / inv_gm1, inv_gm1);
    const R cL = sound_speed<R>(gamma, WL[3], WL[0]);
    const R cR = sound_speed<R>(gamma, WR[3], WR[0]);
    const R sL = fabs_(WL[N]) + cL, sR = fabs_(WR[N]) + cR;
    const bool pickR = sR > sL;
    const R a = pickR ? sR : sL;
    R ab = R(0);
    R FLb[4], FRb[4], ULb[4], URb[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        ab += R(-0.5) * Fb[v] * (UR[v] - UL[v]);
        FLb[v] = R(0.5) * Fb[v];
        FRb[v] = R(0.5) * Fb[v];
        ULb[v] = R(0.5) * a * Fb[v];
        URb[v] = R(-0.5) * a * Fb[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) { WLb[v] = R(0); WRb[v] = R(0); }
    phys_flux_vjp<R, D>(WL, FLb, WLb, inv_gm1);
    phys_flux_vjp<R, D>(WR, FRb, WRb, inv_gm1);
    cons_vjp<R>(WL, ULb, WLb, inv_gm1);
    cons_vjp<R>(WR, URb, WRb, inv_gm1);
    // a -> |u_K| + c_K of the selected side; c = sqrt(gamma p / rho)
    const R* W = pickR ? WR : WL;
    R* Wb = pickR ? WRb : WLb;
    const R c = pickR ? cR : cL;
    Wb[N] += ab * (W[N] < R(0) ? R(-1) : R(1));
    if constexpr (IsExact<R>::value) {
        Wb[3] += ab * gamma / (R(2) * W[0] * c);
        Wb[0] += ab * (-c / (R(2) * W[0]));
    } else {   // FP32: reciprocals instead of two divisions
        const R i2w = rcp_approx(R(2) * W[0]);
        Wb[3] += ab * gamma * i2w * rcp_approx(c);
        Wb[0] += ab * (-c * i2w);
    }
}

// The MC slope of the forward face (the value of mc_slope, bit for bit: the same operations) and
// the candidate it took: 0 -> zero, 1 -> 2 D-, 2 -> (D- + D+)/2, 3 -> 2 D+. minmod returns one of
// its arguments unchanged, and among equal candidates the first, so the first candidate equal to
// a nonzero slope is the one taken (minmod's tie rules).
template <class R> __device__ __forceinline__ R mc_slope_sel(R wm, R w0, R wp, unsigned& sel) {
    const R dm = w0 - wm, dp = wp - w0;
    const R A = R(2) * dm, B = R(0.5) * (dm + dp), C = R(2) * dp;
    const R s = minmod3(A, B, C);
    sel = s == R(0) ? 0u : (s == A ? 1u : (s == B ? 2u : 3u));
    return s;
}
// d(slope)/d(wm, w0, wp) of the candidate sel
template <class R> __device__ __forceinline__ void mc_sel_grad(unsigned sel, R* g) {
    g[0] = sel == 1u ? R(-2) : (sel == 2u ? R(-0.5) : R(0));
    g[1] = sel == 1u ? R(2) : (sel == 3u ? R(-2) : R(0));
    g[2] = sel == 2u ? R(0.5) : (sel == 3u ? R(2) : R(0));
}

struct AdjStageArgs {
    GridArgs g;
    const void* Us;    // forward stage input U^(s) (stencil)
    const void* Ls;    // adjoint of the stage output (stencil)
    const void* X1;    // optional point-wise terms
    const void* X2;
    void* out;         // out = c1 X1 + c2 X2 + b (Ls + dt J_L(Us)^T Ls)
    double c1, c2, b, dt;
    float c1_f, c2_f, b_f, dt_f;   // FP32 copies (no per-thread double->float conversion)
};
template <class R> __device__ __forceinline__ R adj_c(double d, float f) {
    if constexpr (IsExact<R>::value) return d;
    else return f;
}

// One CTA per (sample, TX x TY tile), one cell per thread; RV: reconstruction variables (the
// conserved-variable path is compiled only where it runs).
// FP32: 4 CTAs per SM (the shared-memory limit; measured faster than 2 CTAs without spills);
// FP64: 2 CTAs per SM
template <class R, int RECON, int RV, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 2) k_stage_adj(const AdjStageArgs p) {
    static_assert(TX * TY == NT, "one cell per thread");
    constexpr int NV = 4;
    constexpr bool PC = RECON == REC_PC;
    constexpr int HU = PC ? 1 : 3;        // halo of U: stencil of the outermost interface
    constexpr int HL = PC ? 1 : 2;        // halo of lambda: both cells of each interface
    constexpr int NSL = PC ? 2 : 4;       // stencil cells per interface
    constexpr int OFF = PC ? 1 : 2;       // first interface j = x0 - OFF (interface j+1/2)
    constexpr int NIF = TX + (PC ? 1 : 3);// interfaces per row along x
    constexpr int NIFY = TY + (PC ? 1 : 3);
    constexpr int SUX = TX + 2 * HU, SUY = TY + 2 * HU;
    constexpr int SLX = TX + 2 * HL, SLY = TY + 2 * HL;
    constexpr int NIMAX = (NIF * TY > TX * NIFY) ? NIF * TY : TX * NIFY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sU = reinterpret_cast<R*>(smem_raw);     // [NV][SUY][SUX] conserved
    R* sW = sU + NV * SUX * SUY;                // [NV][SUY][SUX] reconstruction variables
    R* sL = sW + NV * SUX * SUY;                // [NV][SLY][SLX] lambda
    R* sC = sL + NV * SLX * SLY;                // [NSL][NV][NIMAX] interface contributions

    const GridArgs& g = p.g;
    const LevelInfo& L = g.lev[0];
    const uint32_t w = blockIdx.x;
    const uint32_t b_local = fdiv(w, L.fd_tiles);
    const uint32_t tile = w - b_local * (uint32_t)L.tiles;
    const int nx = L.n[0], ny = L.n[1];
    const uint32_t trow = fdiv(tile, L.fd_nt0);
    const int x0 = (int)(tile - trow * (uint32_t)L.ntile[0]) * TX, y0 = (int)trow * TY;
    const long long plane = (long long)nx * ny;
    const long long sbase = (long long)b_local * NV * plane;
    const R* Us = reinterpret_cast<const R*>(p.Us) + sbase;
    const R* Ls = reinterpret_cast<const R*>(p.Ls) + sbase;
    const R gamma = c_gamma<R>(g);
    const R gm1 = IsExact<R>::value ? gamma - R(1) : R(g.gm1_f);
    const R inv_gm1 = IsExact<R>::value ? R(1) / gm1 : R(g.inv_gm1_f);
    constexpr bool prim = RV == RV_PRIM;
    const int tid = threadIdx.x;

    // periodic tile loads
    for (int s = tid; s < SUX * SUY; s += NT) {
        const int sx = s % SUX, sy = s / SUX;
        int ix = (x0 + sx - HU) % nx; if (ix < 0) ix += nx;
        int iy = (y0 + sy - HU) % ny; if (iy < 0) iy += ny;
        const long long off = (long long)iy * nx + ix;
        R u[NV], wv[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = Us[v * plane + off];
        if (prim) cons_to_prim<R, 2>(u, wv, gm1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            sU[v * SUX * SUY + s] = u[v];
            sW[v * SUX * SUY + s] = prim ? wv[v] : u[v];
        }
    }
    for (int s = tid; s < SLX * SLY; s += NT) {
        const int sx = s % SLX, sy = s / SLX;
        int ix = (x0 + sx - HL) % nx; if (ix < 0) ix += nx;
        int iy = (y0 + sy - HL) % ny; if (iy < 0) iy += ny;
        const long long off = (long long)iy * nx + ix;
#pragma unroll
        for (int v = 0; v < NV; ++v) sL[v * SLX * SLY + s] = Ls[v * plane + off];
    }

    R acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = R(0);
    const int cx = tid % TX, cy = tid / TX;

#pragma unroll
    for (int D = 0; D < 2; ++D) {
        __syncthreads();
        const int EX = D == 0 ? NIF : TX, EY = D == 0 ? TY : NIFY;
        const int ustep = D == 0 ? 1 : SUX, lstep = D == 0 ? 1 : SLX;
        const R inv_dx = c_inv_dx<R>(L, D);
        for (int f = tid; f < EX * EY; f += NT) {
            const int fx = f % EX, fy = f / EX;
            // interface j+1/2 along D; left cell j in tile coordinates
            const int jx = D == 0 ? fx - OFF : fx;
            const int jy = D == 0 ? fy : fy - OFF;
            // smem index of the first stencil cell (j - 1 for MC, j for PC)
            const int first = PC ? 0 : 1;
            const int ui = ((jy - (D == 1 ? first : 0)) + HU) * SUX + (jx - (D == 0 ? first : 0)) + HU;
            const int li = (jy + HL) * SLX + jx + HL;
            R w[NSL][NV], cu[NSL][NV];
#pragma unroll
            for (int k = 0; k < NSL; ++k)
#pragma unroll
                for (int v = 0; v < NV; ++v) w[k][v] = sW[v * SUX * SUY + ui + k * ustep];
            if (!prim) {   // conserved stencil values: only the conserved-variable path reads them
#pragma unroll
                for (int k = 0; k < NSL; ++k)
#pragma unroll
                    for (int v = 0; v < NV; ++v) cu[k][v] = sU[v * SUX * SUY + ui + k * ustep];
            }
            constexpr int KL = PC ? 0 : 1, KR = PC ? 1 : 2;   // stencil slots of cells j, j+1
            // forward face states
            R fL[NV], fR[NV];
            unsigned selbits = 0;   // the MC candidate of each face, 2 bits per (variable, face)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (PC) { fL[v] = w[0][v]; fR[v] = w[1][v]; }
                else {
                    unsigned sl, sr;
                    fL[v] = w[1][v] + R(0.5) * mc_slope_sel(w[0][v], w[1][v], w[2][v], sl);
                    fR[v] = w[2][v] - R(0.5) * mc_slope_sel(w[1][v], w[2][v], w[3][v], sr);
                    selbits |= (sl | (sr << 2)) << (4 * v);
                }
            }
            R WL[NV], WR[NV], cw[2][NV];
            bool okL, okR;
            if (prim) {
                okL = fL[0] > R(0) && fL[3] > R(0);
                okR = fR[0] > R(0) && fR[3] > R(0);
#pragma unroll
                for (int v = 0; v < NV; ++v) { WL[v] = okL ? fL[v] : w[KL][v]; WR[v] = okR ? fR[v] : w[KR][v]; }
            } else {
                R a[NV], bb[NV];
                cons_to_prim<R, 2>(fL, a, gm1);
                cons_to_prim<R, 2>(fR, bb, gm1);
                okL = a[0] > R(0) && a[3] > R(0);
                okR = bb[0] > R(0) && bb[3] > R(0);
                cons_to_prim<R, 2>(cu[KL], cw[0], gm1);
                cons_to_prim<R, 2>(cu[KR], cw[1], gm1);
#pragma unroll
                for (int v = 0; v < NV; ++v) { WL[v] = okL ? a[v] : cw[0][v]; WR[v] = okR ? bb[v] : cw[1][v]; }
            }
            // adjoint of the flux: mu = (lambda_{j+1} - lambda_j) / dx
            R mu[NV], WLb[NV], WRb[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) mu[v] = (sL[v * SLX * SLY + li + lstep] - sL[v * SLX * SLY + li]) * inv_dx;
            if (D == 0) rusanov_vjp<R, 0>(WL, WR, mu, WLb, WRb, gamma, inv_gm1);
            else rusanov_vjp<R, 1>(WL, WR, mu, WLb, WRb, gamma, inv_gm1);
            // back through positivity fallback, primitive map of cons faces, reconstruction
            R cb[NSL][NV];
#pragma unroll
            for (int k = 0; k < NSL; ++k)
#pragma unroll
                for (int v = 0; v < NV; ++v) cb[k][v] = R(0);
            R gL[NV], gR[NV];   // adjoints of the reconstructed faces (in reconstruction variables)
            if (prim) {
#pragma unroll
                for (int v = 0; v < NV; ++v) { gL[v] = okL ? WLb[v] : R(0); gR[v] = okR ? WRb[v] : R(0); }
                if (!okL) for (int v = 0; v < NV; ++v) cb[KL][v] += WLb[v];
                if (!okR) for (int v = 0; v < NV; ++v) cb[KR][v] += WRb[v];
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) { gL[v] = R(0); gR[v] = R(0); }
                if (okL) prim_vjp<R>(fL, WLb, gL, gm1);
                else prim_vjp<R>(cu[KL], WLb, cb[KL], gm1);
                if (okR) prim_vjp<R>(fR, WRb, gR, gm1);
                else prim_vjp<R>(cu[KR], WRb, cb[KR], gm1);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (PC) {
                    cb[0][v] += gL[v];
                    cb[1][v] += gR[v];
                } else {
                    R sg[3];
                    mc_sel_grad<R>((selbits >> (4 * v)) & 3u, sg);        // fL = w1 + s/2
                    cb[0][v] += gL[v] * R(0.5) * sg[0];
                    cb[1][v] += gL[v] * (R(1) + R(0.5) * sg[1]);
                    cb[2][v] += gL[v] * R(0.5) * sg[2];
                    mc_sel_grad<R>((selbits >> (4 * v + 2)) & 3u, sg);    // fR = w2 - s/2
                    cb[1][v] += gR[v] * R(-0.5) * sg[0];
                    cb[2][v] += gR[v] * (R(1) - R(0.5) * sg[1]);
                    cb[3][v] += gR[v] * R(-0.5) * sg[2];
                }
            }
#pragma unroll
            for (int k = 0; k < NSL; ++k)
#pragma unroll
                for (int v = 0; v < NV; ++v) sC[(k * NV + v) * NIMAX + f] = cb[k][v];
        }
        __syncthreads();
        // gather: the cell is slot NSL-1 of the first interface touching it ... slot 0 of the last
        const int EXg = D == 0 ? NIF : TX;
#pragma unroll
        for (int k = 0; k < NSL; ++k) {
            const int slot = NSL - 1 - k;
            const int fidx = D == 0 ? cy * EXg + (cx + k) : (cy + k) * EXg + cx;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += sC[(slot * NV + v) * NIMAX + fidx];
        }
    }

    // epilogue: adjoint in conserved variables, RK combination
    const int x = x0 + cx, y = y0 + cy;
    if (x >= nx || y >= ny) return;
    const int ci = (cy + HU) * SUX + cx + HU;
    R Ub[NV];
    if (prim) {
        R cc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { cc[v] = sU[v * SUX * SUY + ci]; Ub[v] = R(0); }
        prim_vjp<R>(cc, acc, Ub, gm1);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) Ub[v] = acc[v];
    }
    const long long off = (long long)y * nx + x;
    const R dt = adj_c<R>(p.dt, p.dt_f), cb_ = adj_c<R>(p.b, p.b_f), c1 = adj_c<R>(p.c1, p.c1_f),
            c2 = adj_c<R>(p.c2, p.c2_f);
    const R* X1 = reinterpret_cast<const R*>(p.X1) + sbase;
    const R* X2 = reinterpret_cast<const R*>(p.X2) + sbase;
    R* out = reinterpret_cast<R*>(p.out) + sbase;
    const int li = (cy + HL) * SLX + cx + HL;
    R x1[NV], x2[NV], o[NV];
    if (p.X1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) x1[v] = X1[v * plane + off];
    }
    if (p.X2) {
#pragma unroll
        for (int v = 0; v < NV; ++v) x2[v] = X2[v * plane + off];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        o[v] = cb_ * (sL[v * SLX * SLY + li] + dt * Ub[v]);
        if (p.X1) o[v] = c1 * x1[v] + o[v];
        if (p.X2) o[v] = c2 * x2[v] + o[v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * plane + off] = o[v];
}

template <class R, int RECON, int TX, int TY, int NT>
constexpr size_t adj_smem_bytes() {
    constexpr bool PC = RECON == REC_PC;
    constexpr int HU = PC ? 1 : 3, HL = PC ? 1 : 2, NSL = PC ? 2 : 4;
    constexpr int NIF = TX + (PC ? 1 : 3), NIFY = TY + (PC ? 1 : 3);
    constexpr int NIMAX = (NIF * TY > TX * NIFY) ? NIF * TY : TX * NIFY;
    return sizeof(R) * (size_t)(4 * 2 * (TX + 2 * HU) * (TY + 2 * HU) + 4 * (TX + 2 * HL) * (TY + 2 * HL) +
                                NSL * 4 * NIMAX);
}

constexpr int kAdjTX = 32, kAdjTY = 8, kAdjNT = 256;

template <class R, int RECON, int RV>
static cudaError_t launch_adj_t(const AdjStageArgs& a, cudaStream_t s) {
    auto k = k_stage_adj<R, RECON, RV, kAdjTX, kAdjTY, kAdjNT>;
    constexpr size_t sm = adj_smem_bytes<R, RECON, kAdjTX, kAdjTY, kAdjNT>();
    static unsigned long long smem_devices = 0;   // devices on which the opt-in is done
    {
        const cudaError_t e = ensure_dynamic_smem(k, sm, smem_devices);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)a.g.total_work, kAdjNT, sm, s>>>(a);
    return cudaGetLastError();
}

template <class R>
static cudaError_t launch_adj_r(int recon, const AdjStageArgs& a, cudaStream_t s) {
    const bool prim = a.g.rvars == RV_PRIM;
    if (recon == REC_PC) return prim ? launch_adj_t<R, REC_PC, RV_PRIM>(a, s) : launch_adj_t<R, REC_PC, RV_CONS>(a, s);
    return prim ? launch_adj_t<R, REC_MC, RV_PRIM>(a, s) : launch_adj_t<R, REC_MC, RV_CONS>(a, s);
}

static cudaError_t launch_adj(int fp64, int recon, const AdjStageArgs& a, cudaStream_t s) {
    return fp64 ? launch_adj_r<double>(recon, a, s) : launch_adj_r<float>(recon, a, s);
}

// lambda^n = d KE / d U^n, KE = sum |m|^2 / (2 rho) dV
template <class R>
__global__ void k_ke_seed(const GridArgs g, const void* Uv, void* Lv) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= C) return;
    const R* U = reinterpret_cast<const R*>(Uv) + (long long)b * 4 * C;
    R* Lm = reinterpret_cast<R*>(Lv) + (long long)b * 4 * C;
    const double dV = L.dx[0] * L.dx[1];
    const double rho = (double)U[i], mx = (double)U[C + i], my = (double)U[2 * C + i];
    const double inv = 1.0 / rho;
    Lm[i] = R(-0.5 * (mx * mx + my * my) * inv * inv * dV);
    Lm[C + i] = R(mx * inv * dV);
    Lm[2 * C + i] = R(my * inv * dV);
    Lm[3 * C + i] = R(0);
}

// lambda^n = d W / d U^n, W = sum 4 (rho - 1)(2 - rho) dV (mixing-layer width): only rho enters
template <class R>
__global__ void k_mix_seed(const GridArgs g, const void* Uv, void* Lv) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= C) return;
    const R* U = reinterpret_cast<const R*>(Uv) + (long long)b * 4 * C;
    R* Lm = reinterpret_cast<R*>(Lv) + (long long)b * 4 * C;
    const double dV = L.dx[0] * L.dx[1];
    const double rho = (double)U[i];
    Lm[i] = R(4.0 * (3.0 - 2.0 * rho) * dV);
    Lm[C + i] = R(0);
    Lm[2 * C + i] = R(0);
    Lm[3 * C + i] = R(0);
}

// KH initial data adjoint, part 1: per (sample, column) G(x) = dJ/dY(x), with
//   U = f Uin + (1-f) Uout, f = clamp01((0.75+Y-ylo)/hy) - clamp01((0.25+Y-ylo)/hy)
// (clamp01 has derivative 1 on [0, 1], the branch the forward takes there).
template <class R>
__global__ void k_kh_adj_column2(const GridArgs g, const void* Lv, const double* theta, double* G) {
    const LevelInfo& L = g.lev[0];
    const int nx = L.n[0], ny = L.n[1];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (x >= nx) return;
    const long long C = (long long)nx * ny;
    const R* Lm = reinterpret_cast<const R*>(Lv) + (long long)b * 4 * C;
    const double PI = 3.14159265358979323846;
    const double* th = theta + (long long)b * 20;
    const double hx = L.dx[0], hy = L.dx[1];
    const double xc = g.lo[0] + (x + 0.5) * hx;
    double Y = 0.0;
    for (int n = 1; n <= 10; ++n) Y = Y + th[n - 1] * sin(2.0 * PI * n * xc + th[10 + n - 1]);
    Y = 0.01 * Y;
    const double gmm = g.gamma;
    const double dU0 = 2.0 - 1.0;
    const double dU1 = 2.0 * -0.5 - 1.0 * 0.5;
    const double dU3 = (2.5 / (gmm - 1.0) + 0.5 * 2.0 * (-0.5 * -0.5)) - (2.5 / (gmm - 1.0) + 0.5 * 1.0 * (0.5 * 0.5));
    double acc = 0.0;
    for (int y = 0; y < ny; ++y) {
        const double ylo = g.lo[1] + y * hy;
        const double alo = (0.25 + Y - ylo) / hy;
        const double ahi = (0.75 + Y - ylo) / hy;
        const double dlo = (alo >= 0.0 && alo <= 1.0) ? 1.0 / hy : 0.0;
        const double dhi = (ahi >= 0.0 && ahi <= 1.0) ? 1.0 / hy : 0.0;
        const double dfdY = dhi - dlo;
        if (dfdY == 0.0) continue;
        const long long off = (long long)y * nx + x;
        const double lu = (double)Lm[off] * dU0 + (double)Lm[C + off] * dU1 + (double)Lm[3 * C + off] * dU3;
        acc += lu * dfdY;
    }
    G[(long long)b * nx + x] = acc;
}

// part 2: grad_j = sum_x G(x) dY(x)/dtheta_j with dY/da_n = 0.01 sin(2 pi n x + b_n),
// dY/db_n = 0.01 a_n cos(2 pi n x + b_n); fixed-order reduction over x.
__global__ void k_kh_adj_params(const GridArgs g, const double* G, const double* theta, double* grad) {
    __shared__ double sh[8];
    const LevelInfo& L = g.lev[0];
    const int nx = L.n[0];
    const int b = blockIdx.y, j = blockIdx.x;
    const double PI = 3.14159265358979323846;
    const double* th = theta + (long long)b * 20;
    const int n = (j % 10) + 1;
    const double hx = L.dx[0];
    double acc = 0.0;
    for (int x = threadIdx.x; x < nx; x += 256) {
        const double xc = g.lo[0] + (x + 0.5) * hx;
        const double arg = 2.0 * PI * n * xc + th[10 + n - 1];
        const double d = j < 10 ? 0.01 * sin(arg) : 0.01 * th[n - 1] * cos(arg);
        acc += G[(long long)b * nx + x] * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int k = 1; k < 8; ++k) r += sh[k];
        grad[(long long)b * 20 + j] = r;
    }
}

}  // namespace alsv

using namespace alsv;

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AdjPlan {
    long long n = 0, c = 0, nck = 0, n_cap = 0;
    double dt = 0.0;
};

// Workspace allowance: the fastest signal may grow by this factor over the run before the
// checkpoint storage sized from the initial data runs out (see the re-planning in the sweep).
constexpr double kAdjGrowth = 1.5;
constexpr int kAdjMaxPasses = 3;

AdjPlan adj_plan(const alsv_ctx* c, double T) {
    AdjPlan p;
    // fixed step (reading): the fastest signal of the two unperturbed KH states
    const double smax = 0.5 + std::sqrt(c->d.gamma * 2.5 / 1.0);
    const double dxm = std::min(c->g.lev[0].dx[0], c->g.lev[0].dx[1]);
    p.n = (long long)std::ceil(T * smax / (c->d.cfl * dxm));
    if (p.n < 1) p.n = 1;
    p.dt = T / (double)p.n;
    // storage: ceil(sqrt(n_cap)) steps per segment, enough checkpoints for any n <= n_cap
    p.n_cap = (long long)std::ceil(kAdjGrowth * (double)p.n);
    p.c = (long long)std::ceil(std::sqrt((double)p.n_cap));
    p.nck = (p.n_cap + p.c - 1) / p.c;
    return p;
}

alsv_status adj_validate(alsv_ctx* c) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (c->eq != ALSV_EQ_EULER || c->ndim != 2) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint: 2D Euler only");
    if (c->g.nlev != 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint: single-level contexts only");
    if (ctx_has_halo(c)) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint: no halo faces (whole grids only)");
    if (c->d.flux != ALSV_FLUX_RUSANOV) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint: Rusanov flux only");
    if (c->d.recon != ALSV_RECON_PC && c->d.recon != ALSV_RECON_MC)
        return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint: PC or MC reconstruction only");
    for (int k = 0; k < 2; ++k)
        for (int s = 0; s < 2; ++s)
            if (c->d.bc[k][s] != ALSV_BC_PERIODIC) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint: periodic boundaries only");
    if (!(c->d.cfl > 0.0)) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint: cfl must be > 0");
    return ALSV_OK;
}

size_t adj_bytes(const alsv_ctx* c, const AdjPlan& p) {
    const size_t S = a256(c->state_bytes);
    return (size_t)(p.nck + (p.c - 1) + 3) * S + a256((size_t)c->total_samples * c->g.lev[0].n[0] * 8);
}

// grid args with the adjoint tile decomposition (32 x 8)
GridArgs adj_grid(const alsv_ctx* c) {
    GridArgs g = c->g;
    LevelInfo& L = g.lev[0];
    L.ntile[0] = (L.n[0] + kAdjTX - 1) / kAdjTX;
    L.ntile[1] = (L.n[1] + kAdjTY - 1) / kAdjTY;
    L.ntile[2] = 1;
    L.tiles = L.ntile[0] * L.ntile[1];
    L.fd_tiles = make_fastdiv((uint32_t)L.tiles);
    L.fd_nt0 = make_fastdiv((uint32_t)L.ntile[0]);
    L.fd_nt1 = make_fastdiv((uint32_t)L.ntile[1]);
    L.work0 = 0;
    g.total_work = (long long)L.samples * L.tiles;
    return g;
}

}  // namespace

extern "C" {

alsv_status alsv_adjoint_workspace_bytes(alsv_ctx* c, double T, size_t* bytes) {
    alsv_status st = adj_validate(c);
    if (st != ALSV_OK) return st;
    if (!bytes) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null output");
    if (!(T > 0.0) || !std::isfinite(T)) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "T must be finite and > 0");
    *bytes = adj_bytes(c, adj_plan(c, T));
    return ALSV_OK;
}

alsv_status alsv_bind_adjoint_workspace(alsv_ctx* c, void* dev, size_t bytes) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (!dev) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null adjoint workspace");
    if (((uintptr_t)dev & 255) != 0) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "adjoint workspace must be 256-byte aligned");
    c->adj_ws = (char*)dev;
    c->adj_bytes = bytes;
    return ALSV_OK;
}

alsv_status alsv_adjoint_evolve(alsv_ctx* c, double T, int observable, const double* theta_dev, double* grad_theta_dev,
                                double* J_dev) {
    alsv_status st = adj_validate(c);
    if (st != ALSV_OK) return st;
    if (observable != ALSV_OBS_KINETIC_ENERGY && observable != ALSV_OBS_MIXING_WIDTH)
        return ctx_fail(c, ALSV_ERR_INVALID_ARG, "unknown observable");
    if (!theta_dev || !grad_theta_dev || !J_dev) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null theta/grad/J pointer");
    if (!c->ws) return ctx_fail(c, ALSV_ERR_NOT_READY, "workspace not bound");
    if (!c->U) return ctx_fail(c, ALSV_ERR_NOT_READY, "no state buffer bound (call alsv_set_initial_data once)");
    if (!(T > 0.0) || !std::isfinite(T)) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "T must be finite and > 0");
    AdjPlan P = adj_plan(c, T);
    if (!c->adj_ws || c->adj_bytes < adj_bytes(c, P))
        return ctx_fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "adjoint workspace missing or smaller than alsv_adjoint_workspace_bytes");
    cudaStream_t s = c->stream;
    const size_t SB = a256(c->state_bytes);
    char* base = c->adj_ws;
    auto ckpt = [&](long long k) { return (void*)(base + (size_t)k * SB); };
    auto seg = [&](long long j) { return (void*)(base + (size_t)(P.nck + j - 1) * SB); };  // j >= 1
    void* Lam = base + (size_t)(P.nck + P.c - 1) * SB;
    void* L1 = base + (size_t)(P.nck + P.c) * SB;
    void* L2 = base + (size_t)(P.nck + P.c + 1) * SB;
    double* G = (double*)(base + (size_t)(P.nck + P.c + 2) * SB);
    const int S = c->total_samples;
    cudaError_t e;
#define CKA(x)                                                        \
    do {                                                              \
        e = (x);                                                      \
        if (e != cudaSuccess) return ctx_cuda_fail(c, e, #x);         \
    } while (0)

    // ---- forward sweep with checkpoints every c steps, from initial data of theta. The first
    // pass uses the step planned from the initial data; if the wave speeds grow so far that the
    // realised CFL number passes the guard, the sweep is repeated with n re-planned from the
    // fastest signal the pass saw (same CFL target), within the workspace's step allowance.
    InitArgs ia;
    ia.g = c->g;
    ia.U = c->U;
    ia.kind = 0;
    ia.theta = theta_dev;
    ia.P = 20;
    const double third = 1.0 / 3.0, two_third = 2.0 / 3.0;
    const int ns = c->nstages;
    auto fwd_step = [&](const void* Uin, void* Uout, bool finish) -> cudaError_t {
        // Uin -> Uout (may alias for the in-context state), stage buffers A, B of the context
        cudaError_t ee;
        if (ns == 2) {
            StageArgs a1 = ctx_stage_args(c, Uin, nullptr, c->A, 0.0, 1.0, false);
            ee = launch_stage(c->fp64, 2, c->eq, c->d.recon, c->d.flux, c->variant, a1, s);
            if (ee != cudaSuccess) return ee;
            StageArgs a2 = ctx_stage_args(c, c->A, Uin, Uout, 0.5, 0.5, finish);
            ee = launch_stage(c->fp64, 2, c->eq, c->d.recon, c->d.flux, c->variant, a2, s);
        } else {
            StageArgs a1 = ctx_stage_args(c, Uin, nullptr, c->A, 0.0, 1.0, false);
            ee = launch_stage(c->fp64, 2, c->eq, c->d.recon, c->d.flux, c->variant, a1, s);
            if (ee != cudaSuccess) return ee;
            StageArgs a2 = ctx_stage_args(c, c->A, Uin, c->Bb, 0.75, 0.25, false);
            ee = launch_stage(c->fp64, 2, c->eq, c->d.recon, c->d.flux, c->variant, a2, s);
            if (ee != cudaSuccess) return ee;
            StageArgs a3 = ctx_stage_args(c, c->Bb, Uin, Uout, third, two_third, finish);
            ee = launch_stage(c->fp64, 2, c->eq, c->d.recon, c->d.flux, c->variant, a3, s);
        }
        c->launches += ns;
        if (ee != cudaSuccess || !finish) return ee;
        FinishArgs f = ctx_finish_args(c, 1);
        f.fixed_dt = P.dt;
        f.cfl_max = c->cfl_max;
        c->launches++;
        return launch_finish(f, s);
    };
    c->adj_passes = 0;
    c->adj_n = 0;
    NvtxRange fwd_range("alsv: adjoint forward sweep and reverse sweep");
    for (;;) {
        ++c->adj_passes;
        CKA(launch_init(c->fp64, 2, ia, s));
        CKA(cudaMemsetAsync(c->t, 0, (size_t)S * 8, s));
        CKA(cudaMemsetAsync(c->nstep, 0, (size_t)S * 8, s));
        CKA(cudaMemsetAsync(c->done, 0, (size_t)S * 4, s));
        CKA(cudaMemsetAsync(c->last, 0, (size_t)S * 4, s));
        CKA(cudaMemsetAsync(c->status, 0, 4, s));
        CKA(cudaMemsetAsync(c->cfl_max, 0, 8, s));
        {
            double hv[2] = {T, 0.0};
            long long nt = P.n;
            std::memcpy(&hv[1], &nt, 8);
            CKA(cudaMemcpyAsync(c->T_end, hv, 16, cudaMemcpyHostToDevice, s));
            CKA(cudaStreamSynchronize(s));
        }
        FinishArgs fa = ctx_finish_args(c, 0);
        fa.fixed_dt = P.dt;
        fa.cfl_max = c->cfl_max;
        CKA(launch_speed(c->fp64, 2, c->eq, c->variant, c->g, c->U, c->part, s));
        CKA(launch_finish(fa, s));
        c->launches += 3;
        for (long long m = 0; m < P.n; ++m) {
            if (m % P.c == 0) CKA(cudaMemcpyAsync(ckpt(m / P.c), c->U, c->state_bytes, cudaMemcpyDeviceToDevice, s));
            CKA(fwd_step(c->U, c->U, true));
        }
        int hs = 0;
        double cfl_seen = 0.0;
        CKA(cudaMemcpyAsync(&hs, c->status, 4, cudaMemcpyDeviceToHost, s));
        CKA(cudaMemcpyAsync(&cfl_seen, c->cfl_max, 8, cudaMemcpyDeviceToHost, s));
        CKA(cudaStreamSynchronize(s));
        if (hs & ST_NONPHYSICAL) return ctx_fail(c, ALSV_ERR_NONPHYSICAL, "adjoint: non-physical state in the forward sweep");
        if (!(hs & ST_CFL)) break;
        // fastest signal over the pass, then the step count that puts it at the target CFL
        const double s_seen = cfl_seen / P.dt;
        long long n1 = (long long)std::ceil(T * s_seen / c->d.cfl);
        if (n1 <= P.n) n1 = P.n + 1;
        if (c->adj_passes >= kAdjMaxPasses || n1 > P.n_cap) {
            char msg[192];
            std::snprintf(msg, sizeof msg,
                          "adjoint: realised CFL number %.4f above the guard 0.5 with %lld steps; the re-planned %lld "
                          "steps exceed the allowance of %lld (or %d passes)", cfl_seen, P.n, n1, P.n_cap, kAdjMaxPasses);
            return ctx_fail(c, ALSV_ERR_CFL, msg);
        }
        P.n = n1;
        P.dt = T / (double)n1;
    }
    c->adj_n = P.n;
    c->adj_dt = P.dt;
    const long long nseg = (P.n + P.c - 1) / P.c;
    // ---- observable and its seed
    const bool mix = observable == ALSV_OBS_MIXING_WIDTH;
    CKA(launch_reduce(c->fp64, mix ? 2 : 1, c->g, c->U, c->red, J_dev, s));
    const long long C = (long long)c->g.lev[0].n[0] * c->g.lev[0].n[1];
    {
        dim3 grid((unsigned)((C + 255) / 256), S);
        if (mix) {
            if (c->fp64) k_mix_seed<double><<<grid, 256, 0, s>>>(c->g, c->U, Lam);
            else k_mix_seed<float><<<grid, 256, 0, s>>>(c->g, c->U, Lam);
        } else {
            if (c->fp64) k_ke_seed<double><<<grid, 256, 0, s>>>(c->g, c->U, Lam);
            else k_ke_seed<float><<<grid, 256, 0, s>>>(c->g, c->U, Lam);
        }
        CKA(cudaGetLastError());
        c->launches += 3;
    }
    // recomputation runs the stage kernels on every sample
    CKA(cudaMemsetAsync(c->done, 0, (size_t)S * 4, s));
    AdjStageArgs aa;
    aa.g = adj_grid(c);
    aa.dt = P.dt;
    aa.dt_f = (float)P.dt;
    auto adj_stage = [&](const void* Us, const void* Ls, const void* X1, double c1, const void* X2, double c2, double b,
                         void* out) -> cudaError_t {
        aa.Us = Us;
        aa.Ls = Ls;
        aa.X1 = X1;
        aa.c1 = c1;
        aa.X2 = X2;
        aa.c2 = c2;
        aa.b = b;
        aa.c1_f = (float)c1;
        aa.c2_f = (float)c2;
        aa.b_f = (float)b;
        aa.out = out;
        c->launches++;
        return launch_adj(c->fp64, c->d.recon, aa, s);
    };
    // ---- reverse sweep, segment by segment
    for (long long k = nseg - 1; k >= 0; --k) {
        const long long m0 = k * P.c, m1 = std::min(P.n, m0 + P.c);
        auto state = [&](long long m) -> void* { return m == m0 ? ckpt(k) : seg(m - m0); };
        for (long long m = m0; m + 1 < m1; ++m) CKA(fwd_step(state(m), state(m + 1), false));
        for (long long m = m1 - 1; m >= m0; --m) {
            void* Um = state(m);
            // stage states of step m
            StageArgs a1 = ctx_stage_args(c, Um, nullptr, c->A, 0.0, 1.0, false);
            CKA(launch_stage(c->fp64, 2, c->eq, c->d.recon, c->d.flux, c->variant, a1, s));
            c->launches++;
            if (ns == 2) {
                // U2 = U/2 + (U1 + dt L(U1))/2 ; U1 = U + dt L(U)
                CKA(adj_stage(c->A, Lam, nullptr, 0.0, nullptr, 0.0, 0.5, L1));
                CKA(adj_stage(Um, L1, Lam, 0.5, nullptr, 0.0, 1.0, Lam));
            } else {
                StageArgs a2 = ctx_stage_args(c, c->A, Um, c->Bb, 0.75, 0.25, false);
                CKA(launch_stage(c->fp64, 2, c->eq, c->d.recon, c->d.flux, c->variant, a2, s));
                c->launches++;
                CKA(adj_stage(c->Bb, Lam, nullptr, 0.0, nullptr, 0.0, two_third, L1));   // lambda_2
                CKA(adj_stage(c->A, L1, nullptr, 0.0, nullptr, 0.0, 0.25, L2));          // lambda_1
                CKA(adj_stage(Um, L2, Lam, third, L1, 0.75, 1.0, Lam));                    // lambda^m
            }
        }
    }
    // ---- initial-data adjoint: d J / d theta
    {
        const int nx = c->g.lev[0].n[0];
        dim3 g1((nx + 127) / 128, S);
        if (c->fp64) k_kh_adj_column2<double><<<g1, 128, 0, s>>>(c->g, Lam, theta_dev, G);
        else k_kh_adj_column2<float><<<g1, 128, 0, s>>>(c->g, Lam, theta_dev, G);
        CKA(cudaGetLastError());
        dim3 g2(20, S);
        k_kh_adj_params<<<g2, 256, 0, s>>>(c->g, G, theta_dev, grad_theta_dev);
        CKA(cudaGetLastError());
        c->launches += 2;
    }
    CKA(cudaStreamSynchronize(s));
    c->time_ready = false;  // the state now holds U^n of the adjoint's forward sweep
#undef CKA
    return ALSV_OK;
}

alsv_status alsv_adjoint_get_plan(alsv_ctx* c, int64_t* n_steps, double* dt, int32_t* passes) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (!n_steps || !dt || !passes) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null output");
    if (c->adj_passes == 0 || c->adj_n == 0) return ctx_fail(c, ALSV_ERR_NOT_READY, "no completed adjoint call");
    *n_steps = c->adj_n;
    *dt = c->adj_dt;
    *passes = c->adj_passes;
    return ALSV_OK;
}

}  // extern "C"
