// Sample-resident time loop for 2D Euler in FP32: every SSP-RK step of one Monte Carlo sample runs
// inside one thread-block cluster, with the whole sample held in the cluster's distributed shared
// memory from the first step to the last (the state touches HBM once on entry and once on exit).
//
// The sample's rows are split over the CS CTAs of the cluster (CTA r owns rows [r R, (r+1) R),
// R = ny / CS); a CTA has one thread per column. Per CTA, shared memory holds U^n and the stage
// state in conserved variables and a primitive copy of its rows with two ghost rows on each side.
// Per RK stage:
//   (a) convert the CTA's own rows of the stage state to primitive variables;
//   (b) after a cluster barrier, read the two boundary rows of each neighbouring CTA's primitive
//       copy into the ghost rows with plain distributed-shared-memory loads (periodic in y: the
//       first and last CTA are neighbours), then a second cluster barrier;
//   (c) march down the rows: each thread evaluates the x-interface to the left of its cell (the
//       right one is the next thread's, through a double-buffered shared row; periodic in x) and
//       the y-interface above it (the one below is carried from the previous row), adds the flux
//       divergence and writes a U^n + b (U^(s) + dt L) into the stage state in place.
// Each interface is evaluated once (plus one y-interface per CTA at its lower edge), with the
// same device functions and the same order of operations as the tile schedule (tile variant 0),
// so the result is bitwise that of alsv_evolve_to_T with variant 0 for MC and WENO3 faces (with PC
// faces the compiler contracts the scalar flux arithmetic of the two instantiations differently,
// a few ulp apart). After the last stage each CTA
// reduces the CFL speed of its new rows, the cluster takes the maximum over its CTAs (distributed
// loads again), and every thread computes the next dt in FP64 exactly as the time control does.
// Cluster barriers are hardware barriers; no thread spins on a flag.
#pragma once

#include <cooperative_groups.h>

#include "fv_stage.cuh"

namespace alsv {

template <int RECON, int FLUX>
__global__ void __launch_bounds__(1024) k_resident2d(const ResidentArgs a) {
    namespace cg = cooperative_groups;
    constexpr int G = 2;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int cs = a.cs;
    const int sample = blockIdx.x / cs;
    const LevelInfo& L = a.g.lev[0];
    const int nx = L.n[0], ny = L.n[1];
    const int R = ny / cs;
    const int x = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* A = reinterpret_cast<float4*>(smem_raw);     // [R][nx] U^n
    float4* B = A + R * nx;                              // [R][nx] stage state
    float4* P = B + R * nx;                              // [R + 4][nx] primitive, ghost rows 0, 1, R+2, R+3
    float4* Fx = P + (R + 4) * nx;                       // [2][nx] x-fluxes of a row
    float* red = reinterpret_cast<float*>(Fx + 2 * nx);  // [32] per-warp maxima
    int* redbad = reinterpret_cast<int*>(red + 32);      // [32] per-warp flags
    float* slot = red + 64;                              // the CTA's maximum, read by the cluster
    int* slotb = reinterpret_cast<int*>(red + 65);

    const float gamma = a.g.gamma_f, gm1 = a.g.gm1_f, inv_gm1 = a.g.inv_gm1_f;
    const float inv_dx = L.inv_dx_f[0], inv_dy = L.inv_dx_f[1];
    const float epsx = L.eps_f[0], epsy = L.eps_f[1];
    const long long plane = (long long)nx * ny;
    float* Ug = a.U + L.elem0 + (long long)sample * 4 * plane;
    const int y0 = rank * R;

    // ---- entry: the CTA's rows from HBM into A and B
    for (int j = 0; j < R; ++j) {
        const long long o = (long long)(y0 + j) * nx + x;
        const float4 u = make_float4(Ug[o], Ug[plane + o], Ug[2 * plane + o], Ug[3 * plane + o]);
        A[j * nx + x] = u;
        B[j * nx + x] = u;
    }

    // CFL speed of the CTA's rows of B (as the stage epilogue forms it), maximum over the cluster
    auto cluster_speed = [&](float smax, bool bad, double& smax_out, bool& bad_out) {
        float s = smax;
        int b = bad ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s = fmaxf(s, __shfl_xor_sync(0xffffffffu, s, o));
            b |= __shfl_xor_sync(0xffffffffu, b, o);
        }
        __syncthreads();   // the slots of the previous reduction are read by everyone
        if ((x & 31) == 0) {
            red[x >> 5] = s;
            redbad[x >> 5] = b;
        }
        __syncthreads();
        if (x == 0) {
            float r = red[0];
            int rb = redbad[0];
            for (int w = 1; w < (nx + 31) / 32; ++w) {
                r = fmaxf(r, red[w]);
                rb |= redbad[w];
            }
            *slot = r;                   // this CTA's slot, read by the whole cluster
            *slotb = rb;
        }
        cluster.sync();
        double m = 0.0;
        int anybad = 0;
        for (int k = 0; k < cs; ++k) {
            const double v = (double)*cluster.map_shared_rank(slot, k);
            m = v > m ? v : m;
            anybad |= *cluster.map_shared_rank(slotb, k);
        }
        cluster.sync();   // every CTA has read every slot before any is rewritten
        smax_out = m;
        bad_out = anybad != 0;
    };
    auto cell_speed = [&](const float4& u, float& smax, bool& bad) {
        const float uu[4] = {u.x, u.y, u.z, u.w};
        float wv[4];
        cons_to_prim<float, 2>(uu, wv, gm1);
        const float rho = wv[0], pr = wv[3];
        if (!(rho > 0.0f && pr > 0.0f) || isinf(rho) || isinf(pr)) {
            bad = true;
        } else {
            const float c = sound_speed<float>(gamma, pr, rho);
            smax = fmax_(smax, speed_dx<float>(fabs_(wv[1]) + c, inv_dx));
            smax = fmax_(smax, speed_dx<float>(fabs_(wv[2]) + c, inv_dy));
        }
    };

    double t = a.t[sample];
    long long n = a.nstep[sample];
    double smax;
    bool bad;
    {
        float s = 0.0f;
        bool b = false;
        for (int j = 0; j < R; ++j) cell_speed(B[j * nx + x], s, b);
        cluster_speed(s, b, smax, bad);
    }
    const int nst = a.rk == 3 ? 3 : 2;
    const float third = (float)(1.0 / 3.0), two_third = (float)(2.0 / 3.0);
    const int up = (rank + 1) % cs, down = (rank + cs - 1) % cs;
    const float4* Pup = cluster.map_shared_rank(P, up);
    const float4* Pdown = cluster.map_shared_rank(P, down);
    int done = 0, last = 0;
    double dt = 0.0;
    long long taken = 0;
    for (;;) {
        if (bad) break;
        if (!(t < a.T)) {
            done = 1;
            break;
        }
        // next step (the time control's adaptive rule: cfl / smax, clipped to land on T)
        dt = a.cfl / smax;
        last = 0;
        if (!(dt < a.T - t)) {
            dt = a.T - t;
            last = 1;
        }
        if (isinf(dt)) dt = 0.0;
        if (taken >= a.max_steps || dt == 0.0) break;
        const float dtf = (float)dt;
        float s_new = 0.0f;
        bool b_new = false;
        for (int st = 0; st < nst; ++st) {
            // stage coefficients as the host's stage schedule: U_out = ca U^n + cb (U^(s) + dt L)
            float ca = 0.0f, cb = 1.0f;
            if (st == 1) { ca = nst == 3 ? 0.75f : 0.5f; cb = nst == 3 ? 0.25f : 0.5f; }
            if (st == 2) { ca = third; cb = two_third; }
            const bool has_un = st > 0;
            // (a) primitive copy of the own rows
            __syncthreads();
            for (int j = 0; j < R; ++j) {
                const float4 u = B[j * nx + x];
                const float uu[4] = {u.x, u.y, u.z, u.w};
                float wv[4];
                cons_to_prim<float, 2>(uu, wv, gm1);
                P[(j + G) * nx + x] = make_float4(wv[0], wv[1], wv[2], wv[3]);
            }
            cluster.sync();
            // (b) ghost rows from the neighbours' primitive copies (distributed shared memory)
            P[0 * nx + x] = Pdown[(R + 0) * nx + x];
            P[1 * nx + x] = Pdown[(R + 1) * nx + x];
            P[(R + 2) * nx + x] = Pup[2 * nx + x];
            P[(R + 3) * nx + x] = Pup[3 * nx + x];
            cluster.sync();
            // (c) march down the rows
            const int xm2 = (x + nx - 2) % nx, xm1 = (x + nx - 1) % nx, xp1 = (x + 1) % nx;
            auto cell = [&](int prow, int cx, float* out) {
                const float4 w = P[prow * nx + cx];
                out[0] = w.x; out[1] = w.y; out[2] = w.z; out[3] = w.w;
            };
            float Glo[4];
            {   // y-interface below row 0: cells rows -2 .. 1 = P rows 0 .. 3
                float cm[4], cl[4], cr[4], c2[4], WL[4], WR[4];
                cell(0, x, cm); cell(1, x, cl); cell(2, x, cr); cell(3, x, c2);
                face_states<float, EQ_EULER, 2, RECON>(cm, cl, cr, c2, RV_PRIM, gm1, epsy, WL, WR);
                euler_flux<float, 2, 1, FLUX>(WL, WR, Glo, gamma, gm1, inv_gm1);
            }
            for (int j = 0; j < R; ++j) {
                const int pr = j + G;
                float Flx[4], Gup[4];
                {   // x-interface to the left of (x, j)
                    float cm[4], cl[4], cr[4], c2[4], WL[4], WR[4];
                    cell(pr, xm2, cm); cell(pr, xm1, cl); cell(pr, x, cr); cell(pr, xp1, c2);
                    face_states<float, EQ_EULER, 2, RECON>(cm, cl, cr, c2, RV_PRIM, gm1, epsx, WL, WR);
                    euler_flux<float, 2, 0, FLUX>(WL, WR, Flx, gamma, gm1, inv_gm1);
                }
                {   // y-interface above (x, j): cells rows j-1 .. j+2
                    float cm[4], cl[4], cr[4], c2[4], WL[4], WR[4];
                    cell(pr - 1, x, cm); cell(pr, x, cl); cell(pr + 1, x, cr); cell(pr + 2, x, c2);
                    face_states<float, EQ_EULER, 2, RECON>(cm, cl, cr, c2, RV_PRIM, gm1, epsy, WL, WR);
                    euler_flux<float, 2, 1, FLUX>(WL, WR, Gup, gamma, gm1, inv_gm1);
                }
                float4* Frow = Fx + (j & 1) * nx;
                Frow[x] = make_float4(Flx[0], Flx[1], Flx[2], Flx[3]);
                __syncthreads();
                const float4 fr = Frow[xp1];
                const float Frt[4] = {fr.x, fr.y, fr.z, fr.w};
                const float4 us4 = B[j * nx + x], un4 = A[j * nx + x];
                const float us[4] = {us4.x, us4.y, us4.z, us4.w}, un[4] = {un4.x, un4.y, un4.z, un4.w};
                float out[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    float acc = 0.0f;
                    acc = acc_sub<float>(acc, Frt[v] - Flx[v], inv_dx);
                    acc = acc_sub<float>(acc, Gup[v] - Glo[v], inv_dy);
                    out[v] = rk_combine<float>(us[v], dtf, acc, has_un, ca, un[v], cb);
                    Glo[v] = Gup[v];
                }
                const float4 o4 = make_float4(out[0], out[1], out[2], out[3]);
                B[j * nx + x] = o4;
                if (st == nst - 1) cell_speed(o4, s_new, b_new);
            }
        }
        // the step is complete: U^{n+1} is in B; it becomes U^n of the next step
        for (int j = 0; j < R; ++j) A[j * nx + x] = B[j * nx + x];
        t = last ? a.T : t + dt;
        ++n;
        ++taken;
        cluster_speed(s_new, b_new, smax, bad);
    }
    // ---- exit: the rows back to HBM, and the sample's time state
    for (int j = 0; j < R; ++j) {
        const long long o = (long long)(y0 + j) * nx + x;
        const float4 u = B[j * nx + x];
        Ug[o] = u.x;
        Ug[plane + o] = u.y;
        Ug[2 * plane + o] = u.z;
        Ug[3 * plane + o] = u.w;
    }
    if (rank == 0 && x == 0) {
        a.t[sample] = t;
        a.nstep[sample] = n;
        if (bad) {
            atomicOr(a.status, ST_NONPHYSICAL);
            a.done[sample] = 1;
        } else {
            a.done[sample] = done;
            // the time control's state for a later step: dt from the current maximum
            double d = a.cfl / smax;
            int l = 0;
            if (!(d < a.T - t)) {
                d = a.T - t;
                l = 1;
            }
            if (isinf(d)) d = 0.0;
            if (!done) {
                a.dt[sample] = d;
                a.dt_f[sample] = (float)d;
                a.last[sample] = l;
            }
        }
    }
}

}  // namespace alsv
