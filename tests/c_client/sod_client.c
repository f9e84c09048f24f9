/*
 * A plain C client of the C ABI (include/alsv.h): no Python, no torch. It allocates the caller-owned
 * device buffers with the CUDA runtime, runs the Sod shock tube (Sec. 3's 1D configuration: 1024
 * cells, MC + HLLC + SSP-RK2, CFL 0.45, outflow, FP64) to T = 0.2 on a stream of its own, folds the
 * final state into the Welford accumulator, and writes
 *   line 1: steps taken, sample count of the statistics
 *   line 2: the conservation totals (rho, rho u, E)
 *   then the final state, one "rho m E" line per cell (%.17g).
 * Usage: sod_client OUT_FILE. Exit status 0 on success, otherwise the failing call's status.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "alsv.h"

#define CHECK(call)                                                                   \
    do {                                                                              \
        alsv_status st_ = (call);                                                     \
        if (st_ != ALSV_OK) {                                                         \
            fprintf(stderr, "%s: status %d: %s\n", #call, st_, alsv_last_error(ctx)); \
            return st_;                                                               \
        }                                                                             \
    } while (0)

int main(int argc, char** argv) {
    if (argc < 2) {
        fprintf(stderr, "usage: %s OUT_FILE\n", argv[0]);
        return 1;
    }
    alsv_grid_desc d;
    memset(&d, 0, sizeof(d));
    d.ndim = 1;
    d.n[0] = 1024; d.n[1] = 1; d.n[2] = 1;
    d.lo[0] = 0.0; d.hi[0] = 1.0; d.hi[1] = 1.0; d.hi[2] = 1.0;
    d.batch = 1;
    d.eq = ALSV_EQ_EULER;
    d.gamma = 1.4;
    d.recon = ALSV_RECON_MC;
    d.recon_vars = ALSV_VARS_PRIM;
    d.flux = ALSV_FLUX_HLLC;
    d.rk = ALSV_RK_SSP2;
    for (int k = 0; k < 3; ++k) d.bc[k][0] = d.bc[k][1] = ALSV_BC_OUTFLOW;
    d.cfl = 0.45;
    d.precision = ALSV_FP64;
    d.weno_eps = 1e-6;

    cudaStream_t stream;
    if (cudaStreamCreate(&stream) != cudaSuccess) return 2;
    alsv_ctx* ctx = NULL;
    size_t ws_bytes = 0;
    CHECK(alsv_init_grid(&d, (void*)stream, &ctx, &ws_bytes));
    void *ws = NULL, *U = NULL, *stats = NULL;
    double* totals = NULL;
    const size_t u_bytes = alsv_state_bytes(ctx), s_bytes = alsv_stats_bytes(ctx);
    if (cudaMalloc(&ws, ws_bytes) != cudaSuccess || cudaMalloc(&U, u_bytes) != cudaSuccess ||
        cudaMalloc(&stats, s_bytes) != cudaSuccess || cudaMalloc((void**)&totals, 3 * sizeof(double)) != cudaSuccess)
        return 2;
    CHECK(alsv_bind_workspace(ctx, ws, ws_bytes));
    CHECK(alsv_set_initial_data(ctx, ALSV_INIT_SOD, NULL, 0, U, u_bytes));
    int64_t steps = 0;
    CHECK(alsv_evolve_to_T(ctx, 0.2, &steps));
    CHECK(alsv_stats_reset(ctx, stats, s_bytes));
    CHECK(alsv_stats_accumulate(ctx, stats, s_bytes));
    int64_t count = 0;
    CHECK(alsv_stats_read(ctx, stats, NULL, NULL, &count));
    CHECK(alsv_conservation_totals(ctx, totals));
    CHECK(alsv_sync(ctx));

    const size_t n = u_bytes / sizeof(double);
    double* h = (double*)malloc(u_bytes);
    double ht[3];
    if (!h || cudaMemcpy(h, U, u_bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ht, totals, sizeof(ht), cudaMemcpyDeviceToHost) != cudaSuccess)
        return 2;
    FILE* f = fopen(argv[1], "w");
    if (!f) return 3;
    fprintf(f, "%lld %lld\n", (long long)steps, (long long)count);
    fprintf(f, "%.17g %.17g %.17g\n", ht[0], ht[1], ht[2]);
    const size_t cells = n / 3;
    for (size_t i = 0; i < cells; ++i) fprintf(f, "%.17g %.17g %.17g\n", h[i], h[cells + i], h[2 * cells + i]);
    fclose(f);
    free(h);
    CHECK(alsv_destroy(ctx));
    cudaFree(ws);
    cudaFree(U);
    cudaFree(stats);
    cudaFree(totals);
    cudaStreamDestroy(stream);
    return 0;
}
