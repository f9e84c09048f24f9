// Internal declarations shared by the host API (alsv_api.cu) and the kernel translation units.
// Not part of the public ABI (include/alsv.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace alsv {

enum { EQ_BURGERS = 0, EQ_EULER = 1 };
enum { REC_PC = 0, REC_MC = 1, REC_WENO3 = 2, REC_ENO2 = 3 };
enum { RV_CONS = 0, RV_PRIM = 1 };
enum { FLX_RUSANOV = 0, FLX_HLL = 1, FLX_HLLC = 2, FLX_ROE = 3, FLX_GODUNOV = 4, FLX_EC = 5, FLX_EC4 = 6, FLX_TECNO2 = 7 };

// Schemes served by the default tile schedule only (ENO2 reconstruction; Roe, Godunov, the
// entropy-conservative fluxes and TECNO2).
inline bool ext_scheme(int recon, int flux) { return recon == REC_ENO2 || flux >= FLX_ROE; }
// Ghost layers a scheme reads: the entropy-conservative fluxes take cell values (EC: the two cells
// of an interface, EC4 and TECNO2: four); the others one (PC) or two layers.
inline constexpr int ghost_width(int recon, int flux) {
    return (flux == FLX_EC4 || flux == FLX_TECNO2) ? 2 : (flux == FLX_EC ? 1 : (recon == REC_PC ? 1 : 2));
}
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECTIVE = 2, BC_HALO = 3 };

// Device status bits (OR-ed into the status word by kernels; kernels never trap).
enum { ST_NONPHYSICAL = 1, ST_CFL = 2, ST_TIMEOUT = 4 };

constexpr int kMaxLevels = 8;

// Division by a runtime constant d (1 <= d < 2^31) for 0 <= n < 2^31 without a divide
// instruction sequence (Granlund-Montgomery): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l.
struct FastDiv {
    uint32_t d, m, l;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    f.l = 0;
    while ((1ull << f.l) < d) ++f.l;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << f.l) - d)) / d + 1);
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) { return (__umulhi(n, f.m) + n) >> f.l; }
#endif

// One grid of an MLMC level table (a single-grid context has one level).
struct LevelInfo {
    int n[3];          // cells per direction
    int ntile[3];      // tiles per direction for the launched tile shape
    int tiles;         // tiles per sample
    int samples;       // samples on this level
    int sample0;       // global index of the level's first sample
    long long elem0;   // element offset of the level's first sample in U
    long long work0;   // first (sample, tile) work item of the level
    double dx[3];
    double inv_dx[3];
    float inv_dx_f[3]; // FP32 copies for the single-precision kernels (a double->float conversion
    float eps_f[3];    // runs on the FP64 pipe, very narrow on this GPU): 1/dx, WENO epsilon
    FastDiv fd_tiles;  // divisors for the (sample, tile) decomposition of a work item
    FastDiv fd_nt0;    // tiles along x
    FastDiv fd_nt1;    // tiles along y
    long long pwork0;  // first (sample pair, tile) work item of the level (two-sample schedule)
};

struct GridArgs {
    int ndim;
    double lo[3];      // domain origin (all levels share the domain box)
    int nlev;
    LevelInfo lev[kMaxLevels];
    long long total_work;  // sum over levels of samples * tiles
    long long total_pwork; // sum over levels of ceil(samples / 2) * tiles
    int total_samples;
    int nv;
    double gamma;
    float gamma_f, gm1_f, inv_gm1_f;  // FP32 copies: gamma, gamma - 1, 1 / (gamma - 1)
    int rvars;
    int bc[3][2];
    double weno_eps;
    int weno_eps_dx2;
    int off[3];        // block of a decomposed grid: global index of the first cell per direction
};

#ifdef __CUDACC__
// Whether a tile whose cells span [c0[k], c1[k]) reads a halo buffer: its stencil (G layers
// beyond the tile) crosses a face of kind BC_HALO. A stage part skips the tiles of the other kind.
template <int ND>
__device__ __forceinline__ bool tile_in_part(const GridArgs& g, int part, const int c0[3], const int c1[3],
                                             const int n[3], int G) {
    if (part == 0) return true;
    bool halo = false;
#pragma unroll
    for (int k = 0; k < ND; ++k)
        halo |= (c0[k] - G < 0 && g.bc[k][0] == BC_HALO) || (c1[k] + G > n[k] && g.bc[k][1] == BC_HALO);
    return part == 1 ? !halo : halo;
}
#endif

// The sample-resident time loop (FP32 2D Euler, one thread-block cluster per sample; stage_f32_2d_resident.cu).
struct ResidentArgs {
    GridArgs g;           // single level, periodic in x and y
    float* U;             // [samples][4][ny][nx], in: state at t, out: state at T
    double* t;            // per-sample time (in/out)
    double* dt;           // per-sample next step (out)
    float* dt_f;
    int64_t* nstep;       // per-sample step count (in/out)
    int* done;            // out: 1 once t >= T
    int* last;
    int* status;          // OR-ed ST_NONPHYSICAL
    double T;
    double cfl;
    long long max_steps;  // per call
    int rk;               // 2 or 3
    int cs;               // CTAs per sample (cluster size)
};

inline size_t resident_smem_bytes(int nx, int R) {
    // A, B [R][nx], P [R + 4][nx], two x-flux rows [nx], all float4; 32 per-warp maxima and flags,
    // the CTA's slot read by the cluster
    return (size_t)16 * nx * (3 * R + 4 + 2) + 66 * 4;
}

cudaError_t launch_resident(const ResidentArgs& a, int recon, int flux, int nx, int R, int samples, cudaStream_t s);

// FP32 copies of the grid's constants (computed once on the host; the stage kernels read them
// instead of converting the doubles in every thread).
inline void fill_float_consts(GridArgs& g) {
    g.gamma_f = (float)g.gamma;
    g.gm1_f = g.gamma_f - 1.0f;
    g.inv_gm1_f = 1.0f / g.gm1_f;
    for (int l = 0; l < kMaxLevels; ++l)
        for (int k = 0; k < 3; ++k) {
            g.lev[l].inv_dx_f[k] = (float)g.lev[l].inv_dx[k];
            g.lev[l].eps_f[k] = g.weno_eps_dx2 ? (float)(g.lev[l].dx[k] * g.lev[l].dx[k]) : (float)g.weno_eps;
        }
}

// One SSP-RK stage: Uout = a * Un + b * (Us + dt * L(Us)); a == 0 means Un is not read.
struct StageArgs {
    GridArgs g;
    const void* Us;
    const void* Un;
    void* Uout;
    double a, b;
    float a_f, b_f;       // FP32 copies of a, b
    int has_un;           // a != 0
    const double* dt;     // [samples]
    const float* dt_f;    // [samples] FP32 copy of dt (written with it)
    const int* done;      // [samples]; nonzero: the sample is skipped
    double* speed_part;   // [work items]; written when want_speed
    int want_speed;
    const void* halo[6];  // face 2k + side with bc HALO: [samples][NV][G][cross] ghost layers
    int part;             // tiles to run: 0 all, 1 those whose stencil reads no halo buffer,
                          // 2 the others (a block's stage split around the halo exchange)
    int done_first;       // nonzero: some sample has finished; the two-sample schedules then test
                          // the done flags before the tile load (otherwise under it)
};

// Tile shape used for a given (precision, ndim); the host derives the tiling from it.
struct TileShape {
    int tx, ty, tz, threads;
};
TileShape stage_tile(int fp64, int ndim, int variant);
int stage_num_variants(int fp64, int ndim);
// whether a variant pairs the two halves of each sample (work items: samples x tiles / 2)
bool stage_variant_halves(int fp64, int ndim, int variant);
// whether a variant supports a configuration (the column-marching variant is specialised)
bool stage_variant_supported(int fp64, int ndim, int eq, int recon, int rvars, int flux, const int bc[3][2], int variant);

// Launchers (return cudaGetLastError of the launch).
cudaError_t launch_stage(int fp64, int ndim, int eq, int recon, int flux, int variant, const StageArgs& a,
                         cudaStream_t s);
// the default tile schedule for the schemes of ext_scheme (stage_ext_*.cu)
cudaError_t launch_stage_ext_f32_1d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ext_f32_2d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ext_f32_3d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ext_f64_1d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ext_f64_2d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_ext_f64_3d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_speed(int fp64, int ndim, int eq, int variant, const GridArgs& g, const void* U,
                         double* speed_part, cudaStream_t s);

struct FinishArgs {
    GridArgs g;
    const double* speed_part;
    double* t;
    double* dt;
    float* dt_f;           // FP32 copy of dt, for the single-precision stage kernels
    int64_t* nstep;
    int* done;
    int* last;
    int* status;
    const double* T_end;   // device scalar: end time of the current run
    const long long* n_target;  // device scalar: fixed mode, steps to take from the start
    double cfl;
    double fixed_dt;       // > 0: fixed mode
    double cfl_guard;      // fixed mode: realised CFL limit
    double* cfl_max;       // fixed mode, nullable: running maximum of the realised CFL number
    int advance;           // 1: the step just finished (advance t); 0: only prepare dt
    const double* smax_in; // nullable: per-sample maximum speed from outside (decomposed grids)
    double* smax_out;      // nullable: only write each sample's maximum speed (+inf if non-finite)
};
cudaError_t launch_finish(const FinishArgs& a, cudaStream_t s);

// Initial data. theta: [samples][P] FP64 (device) or NULL.
struct InitArgs {
    GridArgs g;
    void* U;
    int kind;
    const double* theta;
    int P;
    double vortex_center[2];
};
cudaError_t launch_init(int fp64, int ndim, const InitArgs& a, cudaStream_t s);
// Boundary layers of a block for its neighbours' halos: for each face f with dst[f] != NULL,
// dst[f][b][v][l][cross] = U[b][v][...] at index l (low face) or n_k - G + l (high face) along k.
constexpr int kSpeedCombineMax = 64;   // blocks per alsv_speed_max_combine call
struct SpeedCombineArgs {
    const double* in[kSpeedCombineMax];
    int n;
};
cudaError_t launch_speed_max_combine(const SpeedCombineArgs& a, int samples, double* out, cudaStream_t s);
cudaError_t launch_halo_pack(int fp64, const GridArgs& g, int G, const void* U, void* const dst[6], cudaStream_t s);
// Counter index of each sample's KH parameters: sample s of group l uses src0[l] + (s - sample0[l])
// (an MLMC companion group takes its level's indices, every other group its own).
struct ThetaMap {
    int nlev;
    int sample0[kMaxLevels];
    int src0[kMaxLevels];
};
cudaError_t launch_theta(uint64_t seed, long long sample_offset, int sampler, const ThetaMap& map, int samples, int P,
                         double* theta, cudaStream_t s);

// Monte Carlo statistics (single level).
cudaError_t launch_welford(int fp64, const GridArgs& g, const void* U, void* stats, cudaStream_t s);
cudaError_t launch_stats_read(const GridArgs& g, const void* stats, double* mean, double* var, cudaStream_t s);
cudaError_t launch_stats_merge(const GridArgs& g, void* stats, const void* other, cudaStream_t s);

// Fixed-order FP64 reductions: out[sample][var] totals (kind 0) or out[sample] KE (kind 1).
// partial: scratch of reduce_partial_count(g) doubles.
long long reduce_partial_count(const GridArgs& g);
cudaError_t launch_reduce(int fp64, int kind, const GridArgs& g, const void* U, double* partial, double* out,
                          cudaStream_t s);

// Opt a kernel into `bytes` of dynamic shared memory on the current device, once per device (the
// attribute is per device; `done_mask` is the caller's per-kernel bit set of devices 0..63).
template <class K>
inline cudaError_t ensure_dynamic_smem(K kernel, size_t bytes, unsigned long long& done_mask) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done_mask & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done_mask |= bit;
    return e;
}

// Profiler timeline range for the enclosing scope (NVTX; no cost without an attached tool).
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace alsv
