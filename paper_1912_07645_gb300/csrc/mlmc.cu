// Multilevel Monte Carlo estimator (Sec. 2.2, multilevel form of the sampling display):
//   E[G(u)] ~ sum_l (1/M_l) sum_k (G(u^l_k) - G(u^{l-1}_k)),  G(u^{-1}) = 0,
// for G = q and G = q^2 per cell, q the primitive variables. Level l's coarse companion group runs
// the same KH parameters on a coarser grid; its values are prolongated piecewise constantly (each
// fine cell reads the coarse cell containing it). Per level and cell the accumulator keeps an FP64
// Welford mean and M2 of Y = q^l - P q^{l-1} (samples in ascending order) and the running mean of
// Z = (q^l)^2 - (P q^{l-1})^2; the estimate sums the levels in table order on the finest grid.
#include <cstdint>
#include <cstring>

#include "alsv_ctx.h"
#include "fv_physics.cuh"
#include "fv_quantities.cuh"

namespace alsv {
namespace {

constexpr int kMlmcNT = 128;

// the levels of the estimator (table groups with level_fine == 0) and their companions
struct MlmcLevels {
    int n = 0;                    // number of levels
    int grp[kMaxLevels];          // level -> table group
    int comp[kMaxLevels];         // level -> companion group or -1
    long long off[kMaxLevels];    // byte offset of the level's block in the accumulator
    long long cells[kMaxLevels];  // cells of the level's grid
    int finest = 0;               // level with the most cells
};

MlmcLevels mlmc_levels(const alsv_ctx* c) {
    MlmcLevels m;
    const GridArgs& g = c->g;
    const int nq = c->nv;
    long long off = 256;
    for (int k = 0; k < g.nlev; ++k) {
        if (c->d.level_fine[k] != 0) continue;
        const int l = m.n++;
        m.grp[l] = k;
        m.comp[l] = -1;
        for (int j = 0; j < g.nlev; ++j)
            if (c->d.level_fine[j] == k + 1) m.comp[l] = j;
        const LevelInfo& L = g.lev[k];
        m.cells[l] = (long long)L.n[0] * L.n[1] * L.n[2];
        m.off[l] = off;
        off += ((3LL * nq * m.cells[l] * 8 + 255) / 256) * 256;
        if (m.cells[l] > m.cells[m.finest]) m.finest = l;
    }
    return m;
}

size_t mlmc_total_bytes(const alsv_ctx* c) {
    if (c->g.nlev < 2) return 0;
    const MlmcLevels m = mlmc_levels(c);
    const int l = m.n - 1;
    return (size_t)(m.off[l] + ((3LL * c->nv * m.cells[l] * 8 + 255) / 256) * 256);
}

// one thread per cell of level l's grid, samples in ascending order
template <class R, int NV, int EULER>
__global__ void __launch_bounds__(kMlmcNT) k_mlmc_welford(const GridArgs g, const void* Uv, int gf, int gc,
                                                          char* acc, long long off, int level) {
    const LevelInfo& F = g.lev[gf];
    const long long C = (long long)F.n[0] * F.n[1] * F.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const long long n0 = reinterpret_cast<const long long*>(acc)[level];
    double* mY = reinterpret_cast<double*>(acc + off);
    double* M2 = mY + NV * C;
    double* mZ = M2 + NV * C;
    const R* U = reinterpret_cast<const R*>(Uv);
    const double gm1 = g.gamma - 1.0;
    // parent cell on the companion's grid
    long long Cc = 1, pc = 0;
    if (gc >= 0) {
        const LevelInfo& Q = g.lev[gc];
        Cc = (long long)Q.n[0] * Q.n[1] * Q.n[2];
        const int x = (int)(i % F.n[0]);
        const int y = (int)((i / F.n[0]) % F.n[1]);
        const int z = (int)(i / ((long long)F.n[0] * F.n[1]));
        const int px = x / (F.n[0] / Q.n[0]), py = y / (F.n[1] / Q.n[1]), pz = z / (F.n[2] / Q.n[2]);
        pc = ((long long)pz * Q.n[1] + py) * Q.n[0] + px;
    }
    double my[NV], m2[NV], mz[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        my[q] = mY[q * C + i];
        m2[q] = M2[q * C + i];
        mz[q] = mZ[q * C + i];
    }
    const int B = F.samples;
#pragma unroll 1
    for (int b = 0; b < B; ++b) {
        double xf[NV], xc[NV];
        prim_quantities<R, NV, EULER>(U + F.elem0 + (long long)b * NV * C, C, i, gm1, xf);
        if (gc >= 0) {
            prim_quantities<R, NV, EULER>(U + g.lev[gc].elem0 + (long long)b * NV * Cc, Cc, pc, gm1, xc);
        } else {
#pragma unroll
            for (int q = 0; q < NV; ++q) xc[q] = 0.0;
        }
        const double n = (double)(n0 + b + 1);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double Y = xf[q] - xc[q];
            const double Z = xf[q] * xf[q] - xc[q] * xc[q];
            const double d = Y - my[q];
            my[q] = my[q] + d / n;
            m2[q] = m2[q] + d * (Y - my[q]);
            mz[q] = mz[q] + (Z - mz[q]) / n;
        }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        mY[q * C + i] = my[q];
        M2[q * C + i] = m2[q];
        mZ[q * C + i] = mz[q];
    }
}

__global__ void k_mlmc_count(char* acc, MlmcLevels m, const GridArgs g) {
    long long* cnt = reinterpret_cast<long long*>(acc);
    for (int l = 0; l < m.n; ++l) cnt[l] += g.lev[m.grp[l]].samples;
}

// estimate on the finest grid: levels summed in table order
__global__ void __launch_bounds__(kMlmcNT) k_mlmc_read(const GridArgs g, MlmcLevels m, int nq, const char* acc,
                                                       double* mean_out, double* var_out) {
    const LevelInfo& L = g.lev[m.grp[m.finest]];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const int x = (int)(i % L.n[0]);
    const int y = (int)((i / L.n[0]) % L.n[1]);
    const int z = (int)(i / ((long long)L.n[0] * L.n[1]));
    for (int q = 0; q < nq; ++q) {
        double mean = 0.0, sec = 0.0;
        for (int l = 0; l < m.n; ++l) {
            const LevelInfo& Q = g.lev[m.grp[l]];
            const long long Cl = m.cells[l];
            const int px = x / (L.n[0] / Q.n[0]), py = y / (L.n[1] / Q.n[1]), pz = z / (L.n[2] / Q.n[2]);
            const long long p = ((long long)pz * Q.n[1] + py) * Q.n[0] + px;
            const double* mY = reinterpret_cast<const double*>(acc + m.off[l]);
            mean = mean + mY[q * Cl + p];
            sec = sec + mY[2 * nq * Cl + q * Cl + p];
        }
        if (mean_out) mean_out[q * C + i] = mean;
        if (var_out) var_out[q * C + i] = sec - mean * mean;
    }
}

// per (level, q): sums over the level's cells of mean_Y dV, |mean_Y| dV and var_Y dV; each
// thread sums a strided subset in ascending order, then a fixed shared-memory tree
__global__ void __launch_bounds__(256) k_mlmc_level_stats(const GridArgs g, MlmcLevels m, int nq, const char* acc,
                                                          double* out) {
    const int l = blockIdx.x / nq, q = blockIdx.x % nq;
    const LevelInfo& Q = g.lev[m.grp[l]];
    const long long C = m.cells[l];
    const long long n = reinterpret_cast<const long long*>(acc)[l];
    const double* mY = reinterpret_cast<const double*>(acc + m.off[l]) + q * C;
    const double* M2 = mY + nq * C;
    double dV = 1.0;
    for (int k = 0; k < g.ndim; ++k) dV *= Q.dx[k];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long long i = threadIdx.x; i < C; i += 256) {
        s0 = s0 + mY[i];
        s1 = s1 + fabs(mY[i]);
        s2 = s2 + (n > 1 ? M2[i] / (double)(n - 1) : 0.0);
    }
    __shared__ double sh[3][256];
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = sh[k][threadIdx.x] + sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[(l * nq + q) * 3 + k] = sh[k][0] * dV;
}

template <class R>
cudaError_t launch_mlmc_welford_t(const GridArgs& g, const MlmcLevels& m, int nv, int eq_euler, const void* U,
                                  char* acc, cudaStream_t s) {
    for (int l = 0; l < m.n; ++l) {
        const unsigned grid = (unsigned)((m.cells[l] + kMlmcNT - 1) / kMlmcNT);
        const int gf = m.grp[l], gc = m.comp[l];
        if (!eq_euler) k_mlmc_welford<R, 1, 0><<<grid, kMlmcNT, 0, s>>>(g, U, gf, gc, acc, m.off[l], l);
        else if (nv == 3) k_mlmc_welford<R, 3, 1><<<grid, kMlmcNT, 0, s>>>(g, U, gf, gc, acc, m.off[l], l);
        else if (nv == 4) k_mlmc_welford<R, 4, 1><<<grid, kMlmcNT, 0, s>>>(g, U, gf, gc, acc, m.off[l], l);
        else k_mlmc_welford<R, 5, 1><<<grid, kMlmcNT, 0, s>>>(g, U, gf, gc, acc, m.off[l], l);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_mlmc_count<<<1, 1, 0, s>>>(acc, m, g);
    return cudaGetLastError();
}

alsv_status check_acc(alsv_ctx* c, const void* acc, size_t bytes) {
    if (c->g.nlev < 2) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "the MLMC estimator needs a level table");
    if (!acc) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null MLMC accumulator");
    if (((uintptr_t)acc & 255) != 0) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "MLMC accumulator must be 256-byte aligned");
    if (bytes < mlmc_total_bytes(c)) return ctx_fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "MLMC accumulator smaller than alsv_mlmc_bytes");
    return ALSV_OK;
}

}  // namespace
}  // namespace alsv

using namespace alsv;

extern "C" {

size_t alsv_mlmc_bytes(const alsv_ctx* c) { return c ? mlmc_total_bytes(c) : 0; }

alsv_status alsv_mlmc_reset(alsv_ctx* c, void* acc, size_t bytes) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    alsv_status st = check_acc(c, acc, bytes);
    if (st != ALSV_OK) return st;
    cudaError_t e = cudaMemsetAsync(acc, 0, mlmc_total_bytes(c), c->stream);
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "cudaMemsetAsync");
    return ALSV_OK;
}

alsv_status alsv_mlmc_accumulate(alsv_ctx* c, void* acc, size_t bytes) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    alsv_status st = check_acc(c, acc, bytes);
    if (st != ALSV_OK) return st;
    if (!c->U) return ctx_fail(c, ALSV_ERR_NOT_READY, "no state bound (alsv_set_initial_data)");
    const MlmcLevels m = mlmc_levels(c);
    const int euler = c->eq == ALSV_EQ_EULER;
    cudaError_t e = c->fp64 ? launch_mlmc_welford_t<double>(c->g, m, c->nv, euler, c->U, (char*)acc, c->stream)
                            : launch_mlmc_welford_t<float>(c->g, m, c->nv, euler, c->U, (char*)acc, c->stream);
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "MLMC Welford kernel");
    c->launches += m.n + 1;
    return ALSV_OK;
}

alsv_status alsv_mlmc_read(alsv_ctx* c, const void* acc, size_t bytes, double* mean_dev, double* var_dev,
                           double* level_dev, int64_t* counts_host) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    alsv_status st = check_acc(c, acc, bytes);
    if (st != ALSV_OK) return st;
    const MlmcLevels m = mlmc_levels(c);
    const LevelInfo& L = c->g.lev[m.grp[m.finest]];
    for (int l = 0; l < m.n; ++l) {
        const LevelInfo& Q = c->g.lev[m.grp[l]];
        for (int k = 0; k < 3; ++k)
            if (L.n[k] % Q.n[k] != 0)
                return ctx_fail(c, ALSV_ERR_INVALID_ARG, "every level's grid must divide the finest level's grid");
    }
    cudaError_t e;
    if (mean_dev || var_dev) {
        const long long C = m.cells[m.finest];
        k_mlmc_read<<<(unsigned)((C + kMlmcNT - 1) / kMlmcNT), kMlmcNT, 0, c->stream>>>(c->g, m, c->nv, (const char*)acc,
                                                                                      mean_dev, var_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda_fail(c, e, "MLMC read kernel");
        c->launches++;
    }
    if (level_dev) {
        k_mlmc_level_stats<<<m.n * c->nv, 256, 0, c->stream>>>(c->g, m, c->nv, (const char*)acc, level_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda_fail(c, e, "MLMC level statistics kernel");
        c->launches++;
    }
    if (counts_host) {
        if ((e = cudaMemcpyAsync(counts_host, acc, (size_t)m.n * 8, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return ctx_cuda_fail(c, e, "cudaMemcpyAsync");
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return ctx_cuda_fail(c, e, "cudaStreamSynchronize");
    }
    return ALSV_OK;
}

}  // extern "C"
