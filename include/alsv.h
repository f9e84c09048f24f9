/*
 * alsv.h - C ABI of the GB300 (sm_103a) finite-volume Monte Carlo solver.
 *
 * The library advances many samples of a hyperbolic conservation law u_t + div F(u) = 0
 * (eq. (1.1), Sec. 1 of "Alsvinn: A Fast multi-GPGPU finite volume solver with a strong emphasis
 * on reproducibility", arXiv:1912.07645) with the semi-discrete finite-volume update of eq. (2.1)
 * (Sec. 2.1), a numerical flux (HLLC, Rusanov, HLL), a reconstruction (piecewise constant,
 * MC-limited linear, WENO3) and SSP Runge-Kutta time stepping, and keeps the Monte Carlo mean and
 * variance of every cell on the device (Sec. 2.2).
 *
 * Conventions for every entry point:
 *   - Every call returns an alsv_status; nothing throws across the ABI. alsv_last_error(ctx)
 *     gives a message owned by the context (valid until the next call on that context).
 *   - All device memory is CALLER-OWNED: the caller allocates it (e.g. torch tensors) and passes
 *     raw device pointers with their sizes in bytes. A context only borrows pointers; it never
 *     allocates or frees device memory.
 *   - All GPU work is enqueued on the stream given to alsv_init_grid (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream). Calls are asynchronous unless documented as
 *     synchronous.
 *   - A context is not thread-safe: use one context per stream and per host thread.
 *   - State layout ("SoA"): U[sample][var][z][y][x], x fastest, interior cells only, no ghost
 *     cells in memory. Elements are float (ALSV_FP32) or double (ALSV_FP64). Variables: Burgers
 *     u; Euler rho, rho*u_0 .. rho*u_{ndim-1}, E. Samples of an MLMC level table are stored level
 *     after level, each level contiguous.
 *   - Determinism: no floating-point atomics; every reduction has a fixed order, so repeated runs
 *     with the same inputs are bitwise identical.
 */
#ifndef ALSV_H
#define ALSV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int alsv_status;
enum {
    ALSV_OK = 0,
    ALSV_ERR_INVALID_ARG = 1,       /* bad descriptor, pointer, size or call order */
    ALSV_ERR_CUDA = 2,              /* a CUDA runtime call failed (message names it) */
    ALSV_ERR_NONPHYSICAL = 3,       /* a sample reached rho <= 0, p <= 0 or a non-finite value */
    ALSV_ERR_CFL = 4,               /* fixed-dt mode: realised CFL number above the guard */
    ALSV_ERR_TIMEOUT = 5,           /* a bounded device wait gave up */
    ALSV_ERR_BUFFER_TOO_SMALL = 6,  /* a caller buffer is smaller than required */
    ALSV_ERR_NOT_READY = 7          /* workspace / state not bound yet */
};

enum { ALSV_EQ_BURGERS = 0, ALSV_EQ_EULER = 1 };
/* Reconstruction (Sec. 2.1 names ENO and WENO): PC piecewise constant; MC monotonized-central
 * limited linear; WENO3 Jiang-Shu third order; ENO2 second-order ENO (of the two linear
 * candidates, the one with the smaller one-sided difference). */
enum { ALSV_RECON_PC = 0, ALSV_RECON_MC = 1, ALSV_RECON_WENO3 = 2, ALSV_RECON_ENO2 = 3 };
enum { ALSV_VARS_CONS = 0, ALSV_VARS_PRIM = 1 };
/* Numerical flux (Sec. 2.1 names HLLC, Godunov, Rusanov, Roe and high-order entropy-conservative
 * fluxes): RUSANOV, HLL, HLLC (Davis wave speeds); ROE with Harten's entropy fix on the acoustic
 * fields (Harten-Hyman width); GODUNOV the flux of the exact Riemann solution at x/t = 0; EC the
 * two-point entropy-conservative flux (Ismail-Roe for Euler, (uL^2 + uL uR + uR^2)/6 for Burgers)
 * and EC4 its fourth-order combination over four cells (LeFloch-Mercier-Rohde); TECNO2 the EC
 * flux made entropy stable (Fjordholm-Mishra-Tadmor): minus half the scaled eigenvector matrix
 * times |eigenvalues| times the jump of the ENO2 faces of the scaled entropy variables, over four
 * cells (Burgers: diffusion coefficient max(|uL|, |uR|)). EC, EC4 and TECNO2 take cell values:
 * recon and recon_vars are ignored for them. ENO2, ROE, GODUNOV, EC, EC4 and TECNO2 run on the
 * default stage schedule (tile variant 0); with ENO2, ROE or GODUNOV Euler needs recon_vars PRIM,
 * and Burgers is served in 1D only (INVALID_ARG at alsv_init_grid otherwise). */
enum { ALSV_FLUX_RUSANOV = 0, ALSV_FLUX_HLL = 1, ALSV_FLUX_HLLC = 2, ALSV_FLUX_ROE = 3, ALSV_FLUX_GODUNOV = 4,
       ALSV_FLUX_EC = 5, ALSV_FLUX_EC4 = 6, ALSV_FLUX_TECNO2 = 7 };
enum { ALSV_RK_SSP2 = 2, ALSV_RK_SSP3 = 3 };
/* ALSV_BC_HALO: a face of a block of a decomposed grid whose ghost layers are filled by the caller
 * (alsv_bind_halo; see "Domain decomposition" below). */
enum { ALSV_BC_PERIODIC = 0, ALSV_BC_OUTFLOW = 1, ALSV_BC_REFLECTIVE = 2, ALSV_BC_HALO = 3 };
enum { ALSV_FP32 = 0, ALSV_FP64 = 1 };
enum {
    ALSV_INIT_KH = 0,           /* Kelvin-Helmholtz shear layer (Sec. 3), 2D (20 params) or 3D (128) */
    ALSV_INIT_SOD = 1,          /* Sod tube, split at x = 0.5 */
    ALSV_INIT_LAX = 2,          /* Lax tube, split at x = 0.5 */
    ALSV_INIT_BURGERS_SINE = 3, /* u0 = sin(2 pi x), exact cell averages */
    ALSV_INIT_VORTEX = 4,       /* isentropic vortex, 5x5 Gauss cell averages */
    ALSV_INIT_RAW = 5           /* U_dev already holds the initial state */
};
/* Observables of the adjoint: kinetic energy sum |m|^2 / (2 rho) dV; mixing-layer width
 * sum 4 c (1 - c) dV with c = rho - 1 the inner-band fraction of the KH densities 1 and 2. */
enum { ALSV_OBS_KINETIC_ENERGY = 0, ALSV_OBS_MIXING_WIDTH = 1 };
/* Sampling of the KH parameters theta_{b,j} (Sec. 2.2: Monte Carlo or Quasi Monte Carlo), from the
 * sample's global counter index g (sample_offset + b, or its level's index for an MLMC companion),
 * hi_j = 1 for amplitudes (first half of theta) and 2 pi for phases:
 *   MC              hi_j (splitmix64(seed ^ (g P + j)) >> 11) 2^-53
 *   HALTON          hi_j phi_{p_j}(g + 1): radical inverse of g + 1 in base p_j, the (j+1)-th prime,
 *                   evaluated as an integer fraction num / p_j^K (exact) and one FP64 division
 *   HALTON_SHIFTED  hi_j frac(phi_{p_j}(g + 1) + s_j), s_j = (splitmix64(seed ^ (2^63 + j)) >> 11)
 *                   2^-53 (a Cranley-Patterson rotation; one shift per run and parameter) */
enum { ALSV_SAMPLER_MC = 0, ALSV_SAMPLER_HALTON = 1, ALSV_SAMPLER_HALTON_SHIFTED = 2 };

#define ALSV_MAX_LEVELS 8

/* Problem descriptor. Unused trailing dimensions must have n = 1. */
typedef struct alsv_grid_desc {
    int32_t ndim;          /* 1, 2 or 3 */
    int32_t n[3];          /* cells per direction (level 0 when n_levels > 1 ignores this) */
    double lo[3], hi[3];   /* domain box; dx_k = (hi_k - lo_k) / n_k (one dx per direction), with
                              n_k = global_n[k] for a block of a decomposed grid */
    int32_t batch;         /* samples B (single-level) */
    int32_t eq;            /* ALSV_EQ_* */
    double gamma;          /* ideal-gas ratio of specific heats (Euler) */
    int32_t recon;         /* ALSV_RECON_* */
    int32_t recon_vars;    /* ALSV_VARS_* (Euler only) */
    int32_t flux;          /* ALSV_FLUX_* (Burgers: HLLC behaves as HLL) */
    int32_t rk;            /* ALSV_RK_* */
    int32_t bc[3][2];      /* ALSV_BC_* per direction and side; periodic must pair with periodic;
                              HALO: single grid (n_levels <= 1) only */
    double cfl;            /* CFL number for the adaptive step */
    double fixed_dt;       /* > 0: fixed step (adjoint mode); 0: adaptive CFL step */
    int32_t precision;     /* ALSV_FP32 or ALSV_FP64: state and stencil arithmetic */
    uint64_t seed;         /* master seed for counter-based KH parameters */
    double weno_eps;       /* WENO3 epsilon (default 1e-6) */
    int32_t weno_eps_dx2;  /* 1: epsilon = dx_k^2 per direction */
    int32_t n_levels;      /* 0 or 1: single grid; 2..8: MLMC level table below */
    int32_t level_n[ALSV_MAX_LEVELS][3];
    int32_t level_batch[ALSV_MAX_LEVELS];
    double vortex_center[2];
    int64_t sample_offset; /* global index of this context's first sample: counter-based KH
                              parameters of local sample b use global index sample_offset + b
                              (shards of one Monte Carlo ensemble across GPUs) */
    int32_t level_fine[ALSV_MAX_LEVELS];
                           /* MLMC coupling (n_levels >= 2): 0 = group l of the level table is a
                              level of the estimator; j > 0 = group l is the coarse companion of
                              group j - 1: same batch, and its sample b takes the KH parameters of
                              group j - 1's sample b (the counter index of that sample); its grid
                              must divide group j - 1's grid, which must be a level. At most one
                              companion per level. */
    int32_t sampler;       /* ALSV_SAMPLER_* for counter-generated KH parameters (default MC) */
    int32_t global_n[3];   /* block of a decomposed grid (single grid only): 0 = direction not
                              decomposed (global_n = n); else the whole grid's cells along k, of
                              which this context holds [offset[k], offset[k] + n[k]). lo / hi stay
                              the whole domain's, so dx and every cell centre equal the whole
                              grid's bitwise. */
    int32_t offset[3];     /* first global cell index of the block along k (0 if not decomposed) */
    int32_t reserved[4];   /* must be zero */
} alsv_grid_desc;

typedef struct alsv_ctx alsv_ctx;

/* Library version string (static storage). */
const char* alsv_version(void);

/* Message of the last failed call on ctx (or of the last failed alsv_init_grid when ctx is
 * NULL). Owned by the library. */
const char* alsv_last_error(const alsv_ctx* ctx);

/*
 * alsv_init_grid - validate a descriptor and create a context bound to `stream`.
 *   d                 descriptor (host, read during the call only)
 *   stream            cudaStream_t as void*; all later work of this context goes there
 *   out               receives the new context (host pointer)
 *   workspace_bytes   receives the device workspace size the context needs: RK stage buffers,
 *                     per-tile wave-speed partials, per-sample time state, parameters, status.
 * Errors: ALSV_ERR_INVALID_ARG (bad field; message names it). Synchronous; no GPU work.
 * Defines the discretisation of eq. (2.1) (Sec. 2.1) on the given grid(s).
 */
alsv_status alsv_init_grid(const alsv_grid_desc* d, void* stream, alsv_ctx** out, size_t* workspace_bytes);

/* Bind caller-allocated device workspace (>= workspace_bytes, 256-byte aligned). The context
 * borrows it until alsv_destroy or the next bind. ALSV_ERR_BUFFER_TOO_SMALL if short. */
alsv_status alsv_bind_workspace(alsv_ctx* ctx, void* dev, size_t bytes);

/* Bytes of the full state U for all samples (and levels) of this context. */
size_t alsv_state_bytes(const alsv_ctx* ctx);

/* Copy the context's KH parameters (generated from the seed or passed to alsv_set_initial_data)
 * into theta_dev (device FP64 [samples][n_params]). Asynchronous. */
alsv_status alsv_get_parameters(alsv_ctx* ctx, double* theta_dev);

/* Total number of samples (sum over levels) and conserved variables per cell. */
int32_t alsv_num_samples(const alsv_ctx* ctx);
int32_t alsv_num_vars(const alsv_ctx* ctx);

/*
 * alsv_set_initial_data - write u0 into U_dev and reset every sample's time to 0.
 *   kind        ALSV_INIT_*; KH follows Sec. 3 (two-state shear flow with perturbed interfaces);
 *               the perturbation reading is: interfaces at y = 0.25 + Y and 0.75 + Y with
 *               Y = 0.01 sum a_n sin(2 pi n x + b_n) (2D, 10 modes) or a 2D Fourier sum with 8x8
 *               modes in (x,z) (3D), cell values blended by the band's volume fraction in y.
 *   theta_dev   device FP64 [samples][n_params] parameters (a_n then b_n); NULL: expand them
 *               from d->seed with SplitMix64 (theta_{b,j} = hi_j * (splitmix64(seed ^ (b P + j))
 *               >> 11) * 2^-53, hi = 1 for amplitudes, 2 pi for phases).
 *   n_params    20 (2D KH) or 128 (3D KH); ignored by other kinds
 *   U_dev       device state buffer (layout above) of U_bytes >= alsv_state_bytes(ctx); the
 *               context keeps the pointer and evolves it in place.
 * Asynchronous. Errors: INVALID_ARG, BUFFER_TOO_SMALL, NOT_READY (no workspace).
 */
alsv_status alsv_set_initial_data(alsv_ctx* ctx, int kind, const double* theta_dev, int n_params, void* U_dev,
                                  size_t U_bytes);

/*
 * alsv_step - advance every sample that is not done by n_steps full SSP-RK steps of eq. (2.1)
 * (Sec. 2.1). Adaptive mode: dt_b = min(cfl / s_b, T - t_b) with s_b the largest
 * (|u_k| + c)/dx_k of sample b (Burgers |u|/dx_k); T is +infinity unless set by
 * alsv_evolve_to_T. Fixed mode: dt = d->fixed_dt. Asynchronous; status errors raised by the
 * kernels are reported by the next synchronous call (alsv_sync or alsv_evolve_to_T).
 */
alsv_status alsv_step(alsv_ctx* ctx, int n_steps);

/*
 * alsv_evolve_to_T - advance every sample to t = T (last step clipped to land on T), replaying a
 * captured CUDA graph of step chunks and polling the per-sample done flags between chunks.
 * SYNCHRONOUS. steps_taken_host (may be NULL) receives the largest step count of any sample.
 * Returns the first status error any sample raised (NONPHYSICAL, CFL) or OK.
 */
alsv_status alsv_evolve_to_T(alsv_ctx* ctx, double T, int64_t* steps_taken_host);

/*
 * alsv_evolve_resident - the same evolution to T in ONE launch, each sample resident in the
 * distributed shared memory of one thread-block cluster (the smallest cluster of 1 .. 16 CTAs whose
 * shared memory holds U^n, the stage state and a primitive copy: 256^2 takes 16 CTAs); the state
 * is read from HBM once and written back once, the boundary rows of neighbouring CTAs are read by
 * distributed-shared-memory loads, and each sample takes its own CFL steps. The step counts and
 * times of alsv_evolve_to_T with tile variant 0, and (MC, WENO3) bitwise its state; with PC faces
 * the state agrees to a few ulp (the compiler contracts the two instantiations' scalar flux
 * arithmetic differently). Serves FP32
 * 2D Euler on one grid, periodic in x and y, primitive PC / MC / WENO3 with HLLC or Rusanov, CFL
 * steps, nx a multiple of 32 up to 1024 (INVALID_ARG otherwise, or when the sample does not fit 16
 * CTAs). SYNCHRONOUS; t, steps, done and the next dt are left as alsv_evolve_to_T leaves them.
 * Not in the paper: a schedule of the same scheme (Sec. 2.1) for single-GPU batches.
 */
alsv_status alsv_evolve_resident(alsv_ctx* ctx, double T, int64_t* steps_taken_host);

/*
 * alsv_set_time - resume: set every sample's time t_host[b] and step count steps_host[b] (host
 * arrays of alsv_num_samples entries; steps may be NULL for 0) for the state currently bound, and
 * recompute the CFL partials and time steps from that state. A run checkpointed as (U, t, steps)
 * and resumed with alsv_set_initial_data(ALSV_INIT_RAW) + alsv_set_time continues bitwise as if it
 * had not stopped. Synchronous with respect to the host arrays.
 */
alsv_status alsv_set_time(alsv_ctx* ctx, const double* t_host, const int64_t* steps_host);

/* Synchronise the stream and report the device status word (OK or the first error raised). */
alsv_status alsv_sync(alsv_ctx* ctx);

/* Per-sample time and step count (host arrays of alsv_num_samples entries, may be NULL).
 * SYNCHRONOUS. */
alsv_status alsv_get_time(alsv_ctx* ctx, double* t_host, int64_t* steps_host);

/*
 * Monte Carlo statistics (Sec. 2.2: mean and variance per cell, computed on the GPU).
 * Accumulator layout (caller-owned device buffer of alsv_stats_bytes): int64 count, padding to
 * 256 bytes, then FP64 mean[q][cells] and FP64 M2[q][cells] with q = rho, u_0.., p (Euler,
 * primitive) or u (Burgers). Single-level contexts only.
 *   alsv_stats_reset       zero the accumulator (asynchronous)
 *   alsv_stats_accumulate  fold the current samples in ascending sample order with Welford's
 *                          update (n += 1; delta = x - mean; mean += delta/n; M2 += delta*(x-mean)),
 *                          in FP64; may be called once per batch to stream many batches
 *   alsv_stats_read        mean[q][cells] and unbiased var = M2/(n-1) (0 when n = 1) into
 *                          caller device buffers; count (host, may be NULL) makes it synchronous
 */
size_t alsv_stats_bytes(const alsv_ctx* ctx);
alsv_status alsv_stats_reset(alsv_ctx* ctx, void* stats_dev, size_t bytes);
alsv_status alsv_stats_accumulate(alsv_ctx* ctx, void* stats_dev, size_t bytes);
alsv_status alsv_stats_read(alsv_ctx* ctx, const void* stats_dev, double* mean_dev, double* var_dev,
                            int64_t* count_host);

/*
 * alsv_stats_merge - fold the accumulator other_dev into stats_dev (both laid out as above, same
 * grid), with the pairwise update of Chan, Golub and LeVeque: n = nA + nB, d = meanB - meanA,
 * mean = meanA + d nB / n, M2 = M2A + M2B + d^2 nA nB / n, in FP64. Merging per-GPU shards in rank
 * order gives the ensemble statistics of Sec. 2.2 independently of timing. Asynchronous.
 */
alsv_status alsv_stats_merge(alsv_ctx* ctx, void* stats_dev, const void* other_dev, size_t bytes);

/* Conservation totals sum_i U_{v,i} dV in FP64 with a fixed-order tree, into the caller's device
 * buffer totals_dev[samples][vars] (eq. (2.1) conserves them on periodic grids). Asynchronous. */
alsv_status alsv_conservation_totals(alsv_ctx* ctx, double* totals_dev);

/*
 * alsv_conservation_totals_noalloc - the totals of alsv_conservation_totals for callers that
 * cannot allocate device memory (a plugin whose host framework owns all device buffers and gives
 * it no allocator; a service under a fixed device-memory budget where an allocation could fail or
 * synchronise the device). It needs no context and no workspace: the kernels' per-chunk partial
 * sums live in a static device array of 2^20 doubles (8 MiB) that every GPU loading this library
 * holds until the process exits. The paper has no counterpart; it is an execution variant.
 *   d            descriptor of the state (only ndim, n / level table, lo, hi, batch, eq,
 *                precision and, for a block of a decomposed grid, global_n and offset are read;
 *                they are checked by alsv_init_grid's rules)
 *   U_dev        device state, layout as above, U_bytes >= the descriptor's state size
 *   totals_dev   device FP64 [samples][vars], written
 *   stream       cudaStream_t as void*
 * Calls no cudaMalloc / cudaFree or allocating library routine. Every call looks up the array's
 * device address with cudaGetSymbolAddress (with the calling device current), so a device reset
 * between calls leaves no stale address; the first call on a device also loads the library's
 * device code there, so make that first call before any stream capture. All calls share the
 * array: calls that overlap on the GPU (other streams, other threads) race. Every partial slot is
 * written before it is read, so no clearing is needed. Errors: INVALID_ARG (bad descriptor, a
 * sample of more than 65535 x 4096 cells, or samples x vars x ceil(cells / 4096) above 2^20: the
 * message says so), BUFFER_TOO_SMALL, CUDA; the message is read with alsv_last_error(NULL).
 * Asynchronous.
 */
alsv_status alsv_conservation_totals_noalloc(const alsv_grid_desc* d, const void* U_dev, size_t U_bytes,
                                             double* totals_dev, void* stream);

/* Kinetic energy sum_i |m_i|^2 / (2 rho_i) dV per sample in FP64 (Euler), into ke_dev[samples]. */
alsv_status alsv_kinetic_energy(alsv_ctx* ctx, double* ke_dev);

/* Mixing-layer width sum_i 4 (rho_i - 1)(2 - rho_i) dV per sample in FP64 (Euler; the KH densities
 * 1 and 2 are the two pure states), into w_dev[samples]. Fixed-order sum; asynchronous. */
alsv_status alsv_mixing_width(alsv_ctx* ctx, double* w_dev);

/*
 * Discrete adjoint (not in the paper; gradient of an observable at time T with respect to the
 * KH parameters). Fixed step dt = T / n with n = ceil(T s_max / (cfl dx)), s_max the fastest
 * signal of the two unperturbed KH states; checkpoints every ceil(sqrt(n_cap)) steps with
 * recomputation, n_cap = ceil(1.5 n). When the flow speeds up so far that the realised CFL number
 * dt (|u_k| + c)/dx_k of some step exceeds 0.5, the forward sweep is repeated with
 * n = ceil(T s_seen / cfl), s_seen the fastest signal of the previous pass (at most 3 passes,
 * n <= n_cap); all samples of the batch share n.
 *   alsv_adjoint_workspace_bytes  device bytes the adjoint needs for T (checkpoints for n_cap
 *                                 steps + segment buffers + adjoint states)
 *   alsv_bind_adjoint_workspace   bind it (caller-owned, 256-byte aligned)
 *   alsv_adjoint_evolve           initial data from theta_dev (FP64 [samples][20]), forward with
 *                                 checkpoints, reverse sweep for the observable ALSV_OBS_* at T;
 *                                 writes J_dev[samples] and grad_theta_dev[samples][20] (FP64).
 *                                 SYNCHRONOUS. Supported:
 *                                 2D Euler KH, periodic, PC or MC reconstruction, Rusanov flux,
 *                                 SSP-RK2 or RK3. ALSV_ERR_CFL when re-planning cannot bring the
 *                                 realised CFL under 0.5 within n_cap steps or 3 passes.
 *   alsv_adjoint_get_plan         the last successful alsv_adjoint_evolve's step count n, step dt
 *                                 and number of forward passes (host outputs);
 *                                 ALSV_ERR_NOT_READY before one.
 */
alsv_status alsv_adjoint_workspace_bytes(alsv_ctx* ctx, double T, size_t* bytes);
alsv_status alsv_bind_adjoint_workspace(alsv_ctx* ctx, void* dev, size_t bytes);
alsv_status alsv_adjoint_evolve(alsv_ctx* ctx, double T, int observable, const double* theta_dev,
                                double* grad_theta_dev, double* J_dev);
alsv_status alsv_adjoint_get_plan(alsv_ctx* ctx, int64_t* n_steps, double* dt, int32_t* passes);

/*
 * Multilevel Monte Carlo estimator (Sec. 2.2, the multilevel sum of the sampling display):
 *   E[G(u)] ~ sum_l (1/M_l) sum_k (G(u^l_k) - G(u^{l-1}_k)),   G(u^{-1}) = 0,
 * for G(u) = q and G(u) = q^2, q the primitive variables (rho, u_k, p) (Burgers: u) per cell.
 * The levels l are the level-table groups with level_fine == 0, in table order; u^{l-1}_k is
 * group l's coarse companion (level_fine, same KH parameters), and a level without companion has
 * G(u^{l-1}) = 0. The companion's cell values are prolongated piecewise constantly to level l's grid
 * (each level-l cell takes the value of the coarse cell that contains it).
 *   alsv_mlmc_bytes       accumulator size: a 256-byte header of int64 sample counts per level,
 *                         then per level (256-byte aligned) FP64 arrays [q][cells_l]: Welford mean
 *                         and M2 of Y = q^l - P q^{l-1}, and the running mean of
 *                         Z = (q^l)^2 - (P q^{l-1})^2. 0 for contexts without a level table.
 *   alsv_mlmc_reset       zero it (asynchronous).
 *   alsv_mlmc_accumulate  fold every level's current samples into it, samples in ascending order
 *                         (may be repeated over batches with other seeds or sample_offset:
 *                         streaming M_l). Asynchronous.
 *   alsv_mlmc_read        estimates on the grid of the finest level (the level with the most
 *                         cells; every level's grid must divide it): mean_dev[q][cells] =
 *                         sum_l P mean_Y_l, var_dev[q][cells] = sum_l P mean_Z_l - mean^2 (the
 *                         telescoped second moment minus the squared telescoped mean; it is not
 *                         clipped at zero). level_dev (nullable), FP64 [levels][q][3]:
 *                         (sum_cells mean_Y_l dV_l, sum_cells |mean_Y_l| dV_l,
 *                         sum_cells var_Y_l dV_l) with var_Y = M2/(M_l - 1) (0 for M_l = 1).
 *                         counts_host (nullable): int64 [levels] samples per level (synchronises
 *                         the stream). Device outputs are written asynchronously.
 * Errors: ALSV_ERR_INVALID_ARG without a level table or for a null/unaligned (256 B) buffer,
 * ALSV_ERR_BUFFER_TOO_SMALL below alsv_mlmc_bytes, ALSV_ERR_NOT_READY without a state.
 */
size_t alsv_mlmc_bytes(const alsv_ctx* ctx);
alsv_status alsv_mlmc_reset(alsv_ctx* ctx, void* acc_dev, size_t bytes);
alsv_status alsv_mlmc_accumulate(alsv_ctx* ctx, void* acc_dev, size_t bytes);
alsv_status alsv_mlmc_read(alsv_ctx* ctx, const void* acc_dev, size_t bytes, double* mean_dev, double* var_dev,
                           double* level_dev, int64_t* counts_host);

/*
 * Statistical functionals over the current batch (Sec. 2.2: point PDFs, two-point structure
 * functions, joint PDFs and multi-point correlators among the on-device statistics). Single-level contexts. quantity_index selects a
 * primitive quantity (rho, u_k, p) (Burgers: u), computed in FP64 from the stored state.
 *   alsv_point_pdf_accumulate  for each of n_points cells (cells_dev: int64 flat indices
 *       z*ny*nx + y*nx + x, device) adds every sample's value to counts_dev (int64
 *       [n_points][n_bins + 2], device, caller-zeroed): bin 0 for x < lo, bin 1 + k for
 *       lo + k w <= x < lo + (k+1) w (w = (hi - lo) / n_bins, k = floor((x - lo) / (hi - lo) n_bins)
 *       in FP64, at most n_bins - 1), bin n_bins + 1 for x >= hi or NaN. Asynchronous; streams.
 *   alsv_structure_function_bytes   accumulator bytes for radius R (256-byte header of FP64
 *       acc[0..R] plus per-sample partial sums)
 *   alsv_structure_function_accumulate  order p (1 or 2), radius R in cells (1..16 in 1D and
 *       2D, 1..4 in 3D): acc[0] += samples, acc[r] += sum over samples (ascending) of
 *       sum_x sum_{k in Z^d, r-1 < |k|_2 <= r} |q(x + k) - q(x)|^p dV^2; periodic directions
 *       wrap (they need >= 2R + 1 cells), pairs leaving a non-periodic domain are skipped.
 *       acc_dev is caller-owned, 256-byte aligned, zeroed before the first call. Asynchronous.
 *   alsv_structure_function_read  S_dev[r-1] = (sum_{r' <= r} acc[r'] / acc[0])^(1/p), r = 1..R
 *       (the ball form E[ sum_x sum_{0 < |k| <= r} |dq|^p dV^2 ]^(1/p)). Asynchronous.
 * Errors: ALSV_ERR_INVALID_ARG (level table, index, p, R, bins or null pointers),
 * ALSV_ERR_BUFFER_TOO_SMALL, ALSV_ERR_NOT_READY without a state.
 */
alsv_status alsv_point_pdf_accumulate(alsv_ctx* ctx, int quantity_index, const int64_t* cells_dev, int n_points,
                                      double lo, double hi, int n_bins, int64_t* counts_dev);
/*   alsv_joint_pdf_accumulate  the joint histogram of quantities q1 and q2 at each cell: counts_dev
 *       int64 [n_points][n_bins1 + 2][n_bins2 + 2], bins of each quantity as in the point PDF.
 *   alsv_correlator_accumulate  multi-point correlator E[prod_{j<k} q(x_j)] (the paper's
 *       multi-point correlators, read as raw moments): cells_dev int64 [n_sets][k] (1 <= k <= 8),
 *       acc_dev FP64 [1 + n_sets], caller-zeroed: acc[0] += samples, acc[1 + s] += sum over samples
 *       (ascending) of the product over set s. Asynchronous; streams over batches. */
alsv_status alsv_joint_pdf_accumulate(alsv_ctx* ctx, int q1, int q2, const int64_t* cells_dev, int n_points, double lo1,
                                      double hi1, int n_bins1, double lo2, double hi2, int n_bins2, int64_t* counts_dev);
alsv_status alsv_correlator_accumulate(alsv_ctx* ctx, int quantity_index, const int64_t* cells_dev, int n_sets, int k,
                                       double* acc_dev);
size_t alsv_structure_function_bytes(const alsv_ctx* ctx, int radius);
alsv_status alsv_structure_function_accumulate(alsv_ctx* ctx, int quantity_index, int p, int radius, void* acc_dev,
                                               size_t bytes);
alsv_status alsv_structure_function_read(alsv_ctx* ctx, const void* acc_dev, int p, int radius, double* S_dev);

/*
 * Domain decomposition (Sec. 2.1, last paragraph, and Sec. 3.1: one sample split over several
 * devices, each advancing a block of the grid and exchanging the halo cells its stencil reads
 * from the neighbouring blocks; the paper decomposes in x, y or both). A block is a context whose
 * descriptor sets global_n / offset and marks each face that borders another block
 * ALSV_BC_HALO. Its ghost cells on such a face are read from a caller-bound halo buffer instead
 * of being derived from a boundary condition; everything else (physical faces, arithmetic,
 * statistics, totals) is the single-grid path. The caller drives each step stage by stage and
 * fills the halo buffers between stages (from the neighbours' alsv_halo_pack output, by device
 * copies, NCCL send/recv or any other transport), and takes the CFL maximum over all blocks:
 *
 *   alsv_set_end_time(T);  alsv_speed_max(smax);  MAX over blocks;  alsv_finish_step(smax, 0)
 *   per step: for s = 0 .. stages-1:
 *                 alsv_halo_pack(s, ...) on every block;  deliver into the neighbours' halos;
 *                 alsv_stage(s)
 *             alsv_speed_max(smax);  MAX over blocks;  alsv_finish_step(smax, 1)
 *
 * With every block fed its neighbours' layers of the same stage state and the same maximum, each
 * cell sees exactly the inputs it sees on the whole grid, so the blocks together reproduce the
 * whole-grid run bitwise under the same stage schedule. Every schedule reads halo faces except the
 * FP32 2D column march and two-sample schedules (variants 3-13), which reject them.
 *
 * Halo buffer of face (k, side): [samples][vars][layers][cross], layers = alsv_halo_info's g (1
 * for PC, 2 otherwise), cross = the block's cells across k in (z, y, x) order without k. Layer l
 * of the low face holds the cells at index -g + l along k, of the high face n_k + l. Elements are
 * the state's precision.
 *
 *   alsv_halo_info     layers g and the element count of each face's buffer (host outputs;
 *                      elems[2k + side], 0 for faces that are not HALO)
 *   alsv_bind_halo     device pointers of the six face buffers (NULL for faces that are not
 *                      HALO) and their byte sizes bytes[6] (each >= that face's elems * element
 *                      size). The context borrows them; they are read by every later stage launch.
 *   alsv_halo_pack     write the block's own g boundary layers of the state that stage s reads
 *                      (s = 0: U; RK2 s = 1: the stage buffer; RK3 s = 1, 2: the two stage
 *                      buffers) into send[2k + side] of bytes[2k + side] bytes (same layout; low
 *                      face = indices 0 .. g-1, high face = n_k - g .. n_k - 1), for every face
 *                      whose pointer is not NULL. A neighbour's halo buffer may be passed
 *                      directly. Asynchronous.
 *   alsv_stage         enqueue RK stage s of the current step for every sample that is not done;
 *                      stages must come in order 0, 1, ... (INVALID_ARG otherwise). The last stage
 *                      also writes the per-tile CFL partials. Asynchronous.
 *   alsv_stage_part    stage s split around the halo exchange: ALSV_PART_INTERIOR runs the tiles
 *                      whose stencil reads no halo buffer, so it may be enqueued before the
 *                      neighbours' layers for stage s are delivered (the paper's overlap of the
 *                      exchange with the inner-domain computation, Sec. 2.1, last paragraph; Sec.
 *                      3.1); ALSV_PART_BOUNDARY runs the rest and needs the halos delivered. Both
 *                      parts, in either order, make up alsv_stage(s) (each tile is computed by
 *                      exactly one of them, so the result is bitwise the same); a context with no
 *                      HALO face runs everything in the interior part. Asynchronous.
 *   alsv_speed_max     smax_dev[samples] (device FP64) = each sample's largest (|u_k|+c)/dx_k over
 *                      the block, from the partials of the last stage (or of set_initial_data /
 *                      set_time), +infinity for a sample with a non-finite partial. Allowed before
 *                      the first stage of a step or after the last. Asynchronous.
 *   alsv_speed_max_combine  out_dev[s] = the maximum over i < n of smax_dev[i][s] for s <
 *                      samples (device FP64 vectors; smax_dev is a HOST array of n <= 64 device
 *                      pointers), NaN-propagating: the "MAX over blocks" of the protocol above for
 *                      blocks on one GPU. Needs no context (the blocks are separate contexts);
 *                      errors go to alsv_last_error(NULL). Asynchronous on stream.
 *   alsv_finish_step   time control from an external maximum (the MAX of every block's
 *                      smax; +infinity or NaN marks the sample non-physical): advance = 1 after
 *                      the last stage (t += dt, step count, done flags, next dt), 0 to only
 *                      recompute dt (after set_initial_data, set_time or set_end_time).
 *                      Asynchronous; status errors are reported by alsv_sync.
 *   alsv_set_end_time  set the end time T of the run driven by alsv_finish_step (fixed-dt mode:
 *                      the step target ceil(T / fixed_dt)). SYNCHRONOUS.
 * alsv_step, alsv_evolve_to_T, the adjoint and the structure functions return INVALID_ARG on a
 * context with HALO faces (they would read halo buffers nobody refills).
 */
alsv_status alsv_halo_info(const alsv_ctx* ctx, int32_t* layers, int64_t* elems);
alsv_status alsv_bind_halo(alsv_ctx* ctx, const void* const* halo_dev, const size_t* bytes);
alsv_status alsv_halo_pack(alsv_ctx* ctx, int stage, void* const* send_dev, const size_t* bytes);
alsv_status alsv_stage(alsv_ctx* ctx, int stage);
enum { ALSV_PART_INTERIOR = 1, ALSV_PART_BOUNDARY = 2 };
alsv_status alsv_stage_part(alsv_ctx* ctx, int stage, int part);
alsv_status alsv_speed_max(alsv_ctx* ctx, double* smax_dev);
alsv_status alsv_speed_max_combine(const double* const* smax_dev, int n, int samples, double* out_dev, void* stream);
alsv_status alsv_finish_step(alsv_ctx* ctx, const double* smax_dev, int advance);
alsv_status alsv_set_end_time(alsv_ctx* ctx, double T);

/* Destroy the context (host memory and CUDA graphs only; caller buffers are untouched). */
alsv_status alsv_destroy(alsv_ctx* ctx);

/*
 * Execution controls (no counterpart in the paper; they choose how the same scheme is scheduled
 * on the GPU: FP64 results and FP32 results of schedules with the same arithmetic are bitwise
 * equal, other FP32 schedules agree to FP32 rounding).
 *   alsv_num_tile_variants  number of stage-kernel schedules for this (precision, ndim). FP32 2D:
 *                           0-2 tiles of 32x16, 32x8, 32x32; 3 column march (periodic, primitive
 *                           WENO3/MC, HLLC/Rusanov); 4, 5 two samples per thread in packed FP32x2
 *                           (32x16, 32x8 tiles; primitive, HLLC/Rusanov); 6, 7 the two halves of
 *                           each sample per thread (as 4, 5, with y periodic and ny divisible by
 *                           32, 16); 8, 9 the two-sample schedule with fewer instructions per
 *                           cell (WENO3 from the differences around an interface, fixed thread
 *                           maps, positivity fallback only where needed; 32x16 tiles; 9 with
 *                           every global read of a phase in flight at once); 10, 11 as 8, 9 on
 *                           the two halves of each sample (ny divisible by 32); 12, 13 as 9, 11
 *                           with the x-fluxes passed between lanes by warp shuffles, both
 *                           directions between one pair of barriers (bitwise equal to 8-11).
 *                           FP32 3D: 0, 1 tiles of 16x8x8, 8x8x8; 2, 3 z-marching 32x8 column
 *                           chunks of 64 / 128 planes (Euler); 4 as 2 with the x and y interfaces
 *                           of a plane packed in FP32x2 (primitive, HLLC/Rusanov); 5 as 4 with
 *                           32x7 columns on 256 threads (a plane's 256 interface pairs in one
 *                           pass); 6, 7 as 4, 5 with fewer instructions per interface pair (WENO3
 *                           from the differences around an interface, positivity fallback only
 *                           where needed, split shared-memory planes). FP64 2D / 3D:
 *                           0, 1 tiles. 1D: tiles of 256, 64, 32 cells.
 *   alsv_set_tile_variant   select one (recomputes the wave-speed partials; asynchronous;
 *                           ALSV_ERR_INVALID_ARG if the variant does not support the scheme)
 *   alsv_get_tile           current tile shape, variant and (sample, tile) work items per launch
 *   alsv_autotune           time `reps` pairs of launches per variant - a first stage and a
 *                           last-stage-like launch (U^n read, CFL partials), both writing only the
 *                           stage buffer, so the state is unchanged - with CUDA events on the
 *                           context stream and keep the fastest (a later variant must beat an
 *                           earlier one by more than 1 %); ms_per_variant (host, may be NULL)
 *                           receives the times (-1 for unsupported variants). SYNCHRONOUS.
 *   alsv_set_graphs         1 (default): alsv_evolve_to_T replays captured CUDA graphs of
 *                           16-step chunks; 0: direct launches
 *   alsv_set_profiling      1: record CUDA events around every stage / time-control launch of
 *                           later steps (direct launches, no graphs) and accumulate their device
 *                           time; alsv_get_profile reads the sums (SYNCHRONOUS)
 *   alsv_get_launch_count   kernels this context has launched (graph replays included)
 */
int alsv_num_tile_variants(const alsv_ctx* ctx);
alsv_status alsv_set_tile_variant(alsv_ctx* ctx, int variant);
alsv_status alsv_get_tile(const alsv_ctx* ctx, int* tx, int* ty, int* tz, int* variant, int64_t* work_items);
alsv_status alsv_autotune(alsv_ctx* ctx, int reps, int* chosen, float* ms_per_variant);
alsv_status alsv_set_graphs(alsv_ctx* ctx, int on);
alsv_status alsv_set_profiling(alsv_ctx* ctx, int on);
alsv_status alsv_get_profile(alsv_ctx* ctx, double* stage_ms, int64_t* stage_launches, double* finish_ms,
                             int64_t* finish_launches);
alsv_status alsv_get_launch_count(const alsv_ctx* ctx, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* ALSV_H */
