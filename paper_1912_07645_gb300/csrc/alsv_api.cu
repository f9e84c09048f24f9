// Host side of the C ABI declared in include/alsv.h: descriptor validation, workspace layout,
// the step sequence of eq. (2.1) with SSP-RK stages (Sec. 2.1), CUDA-graph step chunks, Monte
// Carlo statistics (Sec. 2.2) and fixed-order reductions. Device memory is caller-owned; this file
// never allocates device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/alsv.h"
#include <nvtx3/nvToolsExt.h>

#include "alsv_ctx.h"
#include "alsv_internal.h"

using namespace alsv;

namespace {
thread_local std::string g_init_error;
}  // namespace

namespace {

alsv_status fail(alsv_ctx* c, alsv_status st, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return st;
}

alsv_status cuda_fail(alsv_ctx* c, cudaError_t e, const char* what) {
    return fail(c, ALSV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                                           \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return cuda_fail(c, _e, #expr);             \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool variant_ok(const alsv_ctx* c, int v) {
    if (!stage_variant_supported(c->fp64, c->ndim, c->eq, c->d.recon, c->g.rvars, c->d.flux, c->g.bc, v)) return false;
    // halo faces are read by the tile kernels and the 3D z-march (every variant but the FP32 2D
    // column march and two-sample schedules, 3-13)
    if (ctx_has_halo(c) && !c->fp64 && c->ndim == 2 && v >= 3) return false;
    if (stage_variant_halves(c->fp64, c->ndim, v)) {
        // the halves must align with whole tiles: ny divisible by twice the tile height
        const TileShape ts = stage_tile(c->fp64, c->ndim, v);
        for (int l = 0; l < c->g.nlev; ++l)
            if (c->g.lev[l].n[1] % (2 * ts.ty) != 0) return false;
    }
    return true;
}

// Build the per-level tiling for one tile variant.
long long build_levels(const alsv_ctx* c, int variant, GridArgs& g) {
    TileShape ts = stage_tile(c->fp64, c->ndim, variant);
    long long work = 0, elem = 0, pwork = 0;
    int s0 = 0;
    for (int l = 0; l < g.nlev; ++l) {
        LevelInfo& L = g.lev[l];
        const int t[3] = {ts.tx, ts.ty, ts.tz};
        L.tiles = 1;
        for (int k = 0; k < 3; ++k) {
            L.ntile[k] = k < c->ndim ? (L.n[k] + t[k] - 1) / t[k] : 1;
            L.tiles *= L.ntile[k];
        }
        L.fd_tiles = make_fastdiv((uint32_t)L.tiles);
        L.fd_nt0 = make_fastdiv((uint32_t)L.ntile[0]);
        L.fd_nt1 = make_fastdiv((uint32_t)L.ntile[1]);
        L.sample0 = s0;
        L.elem0 = elem;
        L.work0 = work;
        L.pwork0 = pwork;
        // two-sample schedules: one work item per sample pair and tile, or per sample and tile of
        // the lower half (halves pairing)
        pwork += stage_variant_halves(c->fp64, c->ndim, variant) ? (long long)L.samples * (L.tiles / 2)
                                                                 : (long long)((L.samples + 1) / 2) * L.tiles;
        s0 += L.samples;
        elem += (long long)L.samples * c->nv * L.n[0] * L.n[1] * L.n[2];
        work += (long long)L.samples * L.tiles;
    }
    g.total_work = work;
    g.total_pwork = pwork;
    return work;
}

alsv_status require_ready(alsv_ctx* c, bool need_state = true) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    if (!c->ws) return fail(c, ALSV_ERR_NOT_READY, "workspace not bound (alsv_bind_workspace)");
    if (need_state && !c->U) return fail(c, ALSV_ERR_NOT_READY, "no state bound (alsv_set_initial_data)");
    return ALSV_OK;
}

// The level table of the live levels only, for the two-sample schedules (their CTAs map to work
// items through the levels' pwork0 offsets; sample, element and wave-speed slot offsets stay
// absolute, so a finished level's work items are simply not launched).
GridArgs live_level_grid(const GridArgs& g, unsigned live) {
    GridArgs r = g;
    int j = 0;
    long long pw = 0;
    for (int l = 0; l < g.nlev; ++l) {
        const long long items = (l + 1 < g.nlev ? g.lev[l + 1].pwork0 : g.total_pwork) - g.lev[l].pwork0;
        if (!(live & (1u << l))) continue;
        r.lev[j] = g.lev[l];
        r.lev[j].pwork0 = pw;
        pw += items;
        ++j;
    }
    if (j == 0) {   // nothing live: launch nothing
        r.nlev = 1;
        r.lev[0] = g.lev[0];
        r.total_pwork = 0;
        return r;
    }
    r.nlev = j;
    r.total_pwork = pw;
    return r;
}

bool pair_schedule(const alsv_ctx* c) { return !c->fp64 && c->ndim == 2 && c->variant >= 4 && c->variant <= 13; }

StageArgs stage_args(alsv_ctx* c, const void* Us, const void* Un, void* Uout, double a, double b, bool want_speed) {
    StageArgs s;
    s.g = c->g;
    if (c->live_levels != ~0u && pair_schedule(c)) s.g = live_level_grid(c->g, c->live_levels);
    s.Us = Us;
    s.Un = Un;
    s.Uout = Uout;
    s.a = a;
    s.b = b;
    s.a_f = (float)a;
    s.b_f = (float)b;
    s.has_un = a != 0.0 ? 1 : 0;
    s.dt = c->dt;
    s.dt_f = c->dt_f;
    s.done = c->done;
    s.speed_part = c->part;
    s.want_speed = want_speed ? 1 : 0;
    for (int f = 0; f < 6; ++f) s.halo[f] = c->halo[f];
    s.part = 0;
    s.done_first = c->any_done;
    return s;
}

FinishArgs finish_args(alsv_ctx* c, int advance) {
    FinishArgs f;
    f.g = c->g;
    f.speed_part = c->part;
    f.t = c->t;
    f.dt = c->dt;
    f.dt_f = c->dt_f;
    f.nstep = c->nstep;
    f.done = c->done;
    f.last = c->last;
    f.status = c->status;
    f.T_end = c->T_end;
    f.n_target = c->n_target;
    f.cfl = c->d.cfl;
    f.fixed_dt = c->d.fixed_dt;
    f.cfl_guard = 0.5;
    f.cfl_max = nullptr;
    f.advance = advance;
    f.smax_in = nullptr;
    f.smax_out = nullptr;
    return f;
}

void prof_mark(alsv_ctx* c, int kind_next) {
    if (!c->prof.on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, c->stream);
    c->prof.ev.push_back(e);
    if (kind_next >= 0) c->prof.kinds.push_back(kind_next);
}

void prof_collect(alsv_ctx* c) {
    Profile& p = c->prof;
    if (p.ev.empty()) return;
    cudaEventSynchronize(p.ev.back());
    for (size_t i = 0; i + 1 < p.ev.size() && i < p.kinds.size(); ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.ev[i], p.ev[i + 1]);
        if (p.kinds[i] == 0) { p.stage_ms += ms; p.stage_launches++; }
        else { p.finish_ms += ms; p.finish_launches++; }
    }
    for (auto e : p.ev) cudaEventDestroy(e);
    p.ev.clear();
    p.kinds.clear();
}

// Buffers and coefficients of SSP-RK stage k: Uout = a U^n + b (U^(k) + dt L(U^(k))).
struct StageIO { const void* Us; const void* Un; void* Uo; double a, b; };
StageIO stage_io(const alsv_ctx* c, int k) {
    if (c->nstages == 2) {
        if (k == 0) return {c->U, nullptr, c->A, 0.0, 1.0};
        return {c->A, c->U, c->U, 0.5, 0.5};
    }
    if (k == 0) return {c->U, nullptr, c->A, 0.0, 1.0};
    if (k == 1) return {c->A, c->U, c->Bb, 0.75, 0.25};
    return {c->Bb, c->U, c->U, 1.0 / 3.0, 2.0 / 3.0};
}

alsv_status enqueue_stage(alsv_ctx* c, int k, int part = 0) {
    const StageIO io = stage_io(c, k);
    StageArgs a = stage_args(c, io.Us, io.Un, io.Uo, io.a, io.b, k == c->nstages - 1);
    if (part != 0 && !ctx_has_halo(c)) {
        // no tile reads a halo buffer: the interior part is the whole stage, the boundary part empty
        if (part == 2) return ALSV_OK;
        part = 0;
    }
    a.part = part;
    if (c->prof.on && c->prof.ev.empty()) prof_mark(c, -1);
    if (c->prof.on) c->prof.kinds.push_back(0);
    cudaError_t e = launch_stage(c->fp64, c->ndim, c->eq, c->d.recon, c->d.flux, c->variant, a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel launch");
    prof_mark(c, -1);
    c->launches++;
    return ALSV_OK;
}

// Enqueue one full SSP-RK step: stages + per-sample time control.
alsv_status enqueue_step(alsv_ctx* c) {
    for (int k = 0; k < c->nstages; ++k) {
        alsv_status st = enqueue_stage(c, k);
        if (st != ALSV_OK) return st;
    }
    FinishArgs f = finish_args(c, 1);
    if (c->prof.on) c->prof.kinds.push_back(1);
    cudaError_t e = launch_finish(f, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finish kernel launch");
    prof_mark(c, -1);
    c->launches++;
    return ALSV_OK;
}

alsv_status enqueue_speed_and_prepare(alsv_ctx* c) {
    cudaError_t e = launch_speed(c->fp64, c->ndim, c->eq, c->variant, c->g, c->U, c->part, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "speed kernel launch");
    FinishArgs f = finish_args(c, 0);
    e = launch_finish(f, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finish kernel launch");
    c->launches += 2;
    return ALSV_OK;
}

alsv_status read_status(alsv_ctx* c, int* st_host) {
    CK(cudaMemcpyAsync(st_host, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ALSV_OK;
}

alsv_status status_to_code(alsv_ctx* c, int st) {
    if (st & ST_NONPHYSICAL) return fail(c, ALSV_ERR_NONPHYSICAL, "a sample reached a non-physical state (rho<=0, p<=0 or non-finite)");
    if (st & ST_CFL) return fail(c, ALSV_ERR_CFL, "fixed-dt mode: realised CFL number above the guard 0.5");
    if (st & ST_TIMEOUT) return fail(c, ALSV_ERR_TIMEOUT, "a bounded device wait timed out");
    return ALSV_OK;
}

void drop_graph(alsv_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->g_U = nullptr;
    c->g_variant = -1;
    c->g_steps = 0;
}

// Make sure the dynamic shared-memory attribute of the selected stage kernel is set before a
// capture (the launcher sets it on first use; total_work = 0 launches nothing).
void touch_kernels(alsv_ctx* c) {
    StageArgs a = stage_args(c, c->U, c->U, c->A, 0.0, 1.0, false);
    a.g.total_work = 0;
    launch_stage(c->fp64, c->ndim, c->eq, c->d.recon, c->d.flux, c->variant, a, c->stream);
}

alsv_status capture_chunk(alsv_ctx* c, int steps) {
    drop_graph(c);
    touch_kernels(c);
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->graphs_enabled = false;  // e.g. the legacy default stream cannot be captured
        return ALSV_OK;
    }
    long long l0 = c->launches;
    alsv_status st = ALSV_OK;
    for (int i = 0; i < steps && st == ALSV_OK; ++i) st = enqueue_step(c);
    e = cudaStreamEndCapture(c->stream, &graph);
    c->launches = l0;
    if (st != ALSV_OK) return st;
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->g_U = c->U;
    c->g_variant = c->variant;
    c->g_steps = steps;
    return ALSV_OK;
}

alsv_status run_chunk(alsv_ctx* c, int steps) {
    if (c->graphs_enabled && !c->prof.on) {
        if (!c->gexec || c->g_U != c->U || c->g_variant != c->variant || c->g_steps != steps) {
            alsv_status st = capture_chunk(c, steps);
            if (st != ALSV_OK) return st;
        }
        if (c->gexec) {
            CK(cudaGraphLaunch(c->gexec, c->stream));
            c->launches += (long long)steps * (c->nstages + 1);
            return ALSV_OK;
        }
    }
    for (int i = 0; i < steps; ++i) {
        alsv_status st = enqueue_step(c);
        if (st != ALSV_OK) return st;
    }
    return ALSV_OK;
}

}  // namespace

namespace alsv {
NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }
void set_global_error(const std::string& msg) { g_init_error = msg; }
alsv_status ctx_fail(alsv_ctx* c, alsv_status st, const std::string& msg) { return fail(c, st, msg); }
alsv_status ctx_cuda_fail(alsv_ctx* c, cudaError_t e, const char* what) { return cuda_fail(c, e, what); }
FinishArgs ctx_finish_args(alsv_ctx* c, int advance) { return finish_args(c, advance); }
StageArgs ctx_stage_args(alsv_ctx* c, const void* Us, const void* Un, void* Uout, double a, double b, bool want_speed) {
    return stage_args(c, Us, Un, Uout, a, b, want_speed);
}
bool ctx_has_halo(const alsv_ctx* c) {
    for (int k = 0; k < 3; ++k)
        if (c->g.bc[k][0] == BC_HALO || c->g.bc[k][1] == BC_HALO) return true;
    return false;
}
}  // namespace alsv

// =============================================================================================
// Tile table
// =============================================================================================
namespace alsv {
TileShape stage_tile(int fp64, int ndim, int variant) {
    if (ndim == 1) {
        // short tiles spread a small grid over more SMs (FP64 arithmetic is slow per SM)
        if (variant == 1) return {64, 1, 1, 64};
        if (variant == 2) return {32, 1, 1, 32};
        return {256, 1, 1, 256};
    }
    if (ndim == 2) {
        if (variant == 1) return TileShape{32, 8, 1, 256};
        if (variant == 2 && !fp64) return TileShape{32, 32, 1, 256};
        if (variant == 3 && !fp64) return TileShape{31, 1 << 20, 1, 128};  // column strips, whole height
        if (variant == 5 && !fp64) return TileShape{32, 8, 1, 256};        // two-sample tiles
        if (variant == 6 && !fp64) return TileShape{32, 16, 1, 256};       // two halves of a sample
        if (variant == 7 && !fp64) return TileShape{32, 8, 1, 256};

        return TileShape{32, 16, 1, 256};                                   // variants 0, 4, 8-13
    }
    if (fp64) return variant == 1 ? TileShape{8, 8, 4, 256} : TileShape{8, 8, 8, 256};
    if (variant == 2) return TileShape{32, 8, 64, 256};    // z-marching column chunks
    if (variant == 3) return TileShape{32, 8, 128, 256};
    if (variant == 4) return TileShape{32, 8, 64, 256};     // z-march, packed x/y interfaces
    if (variant == 5) return TileShape{32, 7, 64, 256};     // as 4 with 32 x 7 columns, 256 threads
    if (variant == 6) return TileShape{32, 8, 64, 256};     // lean packed z-march
    if (variant == 7) return TileShape{32, 7, 64, 256};
    return variant == 1 ? TileShape{8, 8, 8, 256} : TileShape{16, 8, 8, 256};
}
bool stage_variant_halves(int fp64, int ndim, int variant) {
    return ndim == 2 && !fp64 && (variant == 6 || variant == 7 || variant == 10 || variant == 11 || variant == 13);
}
int stage_num_variants(int fp64, int ndim) {
    if (ndim == 1) return 3;
    if (ndim == 2 && !fp64) return 14;
    if (ndim == 3 && !fp64) return 8;
    return 2;
}
bool stage_variant_supported(int fp64, int ndim, int eq, int recon, int rvars, int flux, const int bc[3][2], int variant) {
    if (variant < 0 || variant >= stage_num_variants(fp64, ndim)) return false;
    // ENO2 and the Roe / Godunov / entropy-conservative fluxes: the default tile schedule
    if (ext_scheme(recon, flux))
        return variant == 0 && (eq == EQ_EULER ? rvars == RV_PRIM : ndim == 1);
    if (ndim == 2 && !fp64 && (variant == 4 || variant == 5 || variant == 8 || variant == 9 || variant == 12))
        return eq == EQ_EULER && rvars == RV_PRIM && (flux == FLX_HLLC || flux == FLX_RUSANOV);
    if (ndim == 2 && !fp64 && (variant == 6 || variant == 7 || variant == 10 || variant == 11 || variant == 13))
        return eq == EQ_EULER && rvars == RV_PRIM && (flux == FLX_HLLC || flux == FLX_RUSANOV) &&
               bc[1][0] == BC_PERIODIC && bc[1][1] == BC_PERIODIC;
    if (ndim == 3 && !fp64 && (variant == 4 || variant == 5 || variant == 6 || variant == 7))
        return eq == EQ_EULER && rvars == RV_PRIM && (flux == FLX_HLLC || flux == FLX_RUSANOV);
    if (ndim == 3 && !fp64 && variant >= 2) return eq == EQ_EULER;
    if (!(ndim == 2 && !fp64 && variant == 3)) return true;
    const bool periodic = bc[0][0] == BC_PERIODIC && bc[0][1] == BC_PERIODIC && bc[1][0] == BC_PERIODIC &&
                          bc[1][1] == BC_PERIODIC;
    return eq == EQ_EULER && rvars == RV_PRIM && periodic && (recon == REC_WENO3 || recon == REC_MC) &&
           (flux == FLX_HLLC || flux == FLX_RUSANOV);
}
}  // namespace alsv

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

const char* alsv_version(void) { return "alsv 0.2 (sm_103a finite-volume MC solver)"; }

const char* alsv_last_error(const alsv_ctx* c) {
    if (!c) return g_init_error.c_str();
    return c->err.c_str();
}

alsv_status alsv_init_grid(const alsv_grid_desc* d_in, void* stream, alsv_ctx** out, size_t* workspace_bytes) {
    if (!d_in || !out) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null descriptor or output pointer");
    *out = nullptr;
    alsv_grid_desc d = *d_in;
    auto bad = [](const std::string& m) { return fail(nullptr, ALSV_ERR_INVALID_ARG, m); };
    if (d.ndim < 1 || d.ndim > 3) return bad("ndim must be 1, 2 or 3");
    if (d.eq != ALSV_EQ_BURGERS && d.eq != ALSV_EQ_EULER) return bad("eq must be BURGERS or EULER");
    if (d.recon < 0 || d.recon > 3) return bad("recon must be PC, MC, WENO3 or ENO2");
    if (d.recon_vars != ALSV_VARS_CONS && d.recon_vars != ALSV_VARS_PRIM) return bad("recon_vars must be CONS or PRIM");
    if (d.flux < 0 || d.flux > 7) return bad("flux must be RUSANOV, HLL, HLLC, ROE, GODUNOV, EC, EC4 or TECNO2");
    if (ext_scheme(d.recon, d.flux)) {
        if (d.eq == ALSV_EQ_BURGERS && d.ndim != 1)
            return bad("ENO2 reconstruction and the ROE, GODUNOV, EC, EC4, TECNO2 fluxes serve Burgers in 1D only");
        if (d.eq == ALSV_EQ_EULER && d.recon_vars != ALSV_VARS_PRIM && d.flux != ALSV_FLUX_EC && d.flux != ALSV_FLUX_EC4 &&
            d.flux != ALSV_FLUX_TECNO2)
            return bad("ENO2 reconstruction and the ROE, GODUNOV fluxes reconstruct primitive variables (recon_vars PRIM)");
    }
    if (d.rk != ALSV_RK_SSP2 && d.rk != ALSV_RK_SSP3) return bad("rk must be SSP2 or SSP3");
    if (d.precision != ALSV_FP32 && d.precision != ALSV_FP64) return bad("precision must be FP32 or FP64");
    if (d.eq == ALSV_EQ_EULER && !(d.gamma > 1.0)) return bad("gamma must be > 1");
    if (!(d.cfl > 0.0) && !(d.fixed_dt > 0.0)) return bad("cfl must be > 0 (or fixed_dt > 0)");
    if (d.fixed_dt < 0.0 || !std::isfinite(d.fixed_dt)) return bad("fixed_dt must be >= 0 and finite");
    if (d.weno_eps == 0.0) d.weno_eps = 1e-6;
    if (!(d.weno_eps > 0.0)) return bad("weno_eps must be > 0");
    for (int k = 0; k < 4; ++k)
        if (d.reserved[k] != 0) return bad("reserved fields must be zero");
    if (d.sampler < ALSV_SAMPLER_MC || d.sampler > ALSV_SAMPLER_HALTON_SHIFTED) return bad("unknown sampler");
    if (d.sample_offset < 0) return bad("sample_offset must be >= 0");
    for (int k = 0; k < d.ndim; ++k)
        if (!(d.hi[k] > d.lo[k])) return bad("hi must exceed lo in every active direction");
    const int G = ghost_width(d.recon, d.flux);
    for (int k = 0; k < 3; ++k)
        for (int s = 0; s < 2; ++s)
            if (d.bc[k][s] < 0 || d.bc[k][s] > 3) return bad("bc must be PERIODIC, OUTFLOW, REFLECTIVE or HALO");
    for (int k = 0; k < d.ndim; ++k)
        if ((d.bc[k][0] == ALSV_BC_PERIODIC) != (d.bc[k][1] == ALSV_BC_PERIODIC))
            return bad("a periodic side must be paired with a periodic side");
    // block of a decomposed grid
    bool block = false, halo = false;
    for (int k = 0; k < 3; ++k) {
        if (d.global_n[k] != 0 || d.offset[k] != 0) block = true;
        if (k < d.ndim && (d.bc[k][0] == ALSV_BC_HALO || d.bc[k][1] == ALSV_BC_HALO)) halo = true;
        if (k >= d.ndim && (d.global_n[k] > 1 || d.offset[k] != 0))
            return bad("global_n / offset of an inactive direction must be 0");
        if (k < d.ndim && d.global_n[k] == 0 && d.offset[k] != 0) return bad("offset needs global_n");
        if (k < d.ndim && d.global_n[k] != 0 &&
            (d.offset[k] < 0 || (long long)d.offset[k] + d.n[k] > d.global_n[k]))
            return bad("a block must lie inside the whole grid: 0 <= offset and offset + n <= global_n");
    }
    if ((block || halo) && d.n_levels > 1) return bad("decomposed grids and halo faces need a single grid (n_levels <= 1)");
    for (int k = 0; k < d.ndim; ++k)
        if ((d.bc[k][0] == ALSV_BC_HALO || d.bc[k][1] == ALSV_BC_HALO) && d.n[k] < G)
            return bad("a block with a halo face needs at least as many cells as ghost layers across it");

    auto* c = new alsv_ctx();
    c->d = d;
    c->stream = (cudaStream_t)stream;
    c->fp64 = d.precision == ALSV_FP64;
    c->ndim = d.ndim;
    c->eq = d.eq;
    c->nv = d.eq == ALSV_EQ_BURGERS ? 1 : d.ndim + 2;
    c->G = G;
    c->nstages = d.rk == ALSV_RK_SSP3 ? 3 : 2;
    GridArgs& g = c->g;
    std::memset(&g, 0, sizeof(g));
    g.ndim = d.ndim;
    for (int k = 0; k < 3; ++k) g.lo[k] = d.lo[k];
    const int nlev = d.n_levels <= 1 ? 1 : d.n_levels;
    if (nlev > ALSV_MAX_LEVELS) { delete c; return bad("n_levels must be <= 8"); }
    g.nlev = nlev;
    long long samples = 0;
    for (int l = 0; l < nlev; ++l) {
        LevelInfo& L = g.lev[l];
        const int* n = d.n_levels <= 1 ? d.n : d.level_n[l];
        L.samples = d.n_levels <= 1 ? d.batch : d.level_batch[l];
        if (L.samples < 1) { delete c; return bad("batch (samples per level) must be >= 1"); }
        for (int k = 0; k < 3; ++k) {
            L.n[k] = k < d.ndim ? n[k] : 1;
            if (L.n[k] < 1) { delete c; return bad("every active direction needs n >= 1"); }
            if (k < d.ndim && (d.bc[k][0] == ALSV_BC_REFLECTIVE || d.bc[k][1] == ALSV_BC_REFLECTIVE) && L.n[k] < G) {
                delete c;
                return bad("reflective boundaries need at least as many cells as ghost layers");
            }
            const int ng = k < d.ndim && d.global_n[k] != 0 ? d.global_n[k] : L.n[k];  // whole grid
            L.dx[k] = k < d.ndim ? (d.hi[k] - d.lo[k]) / ng : 1.0;
            L.inv_dx[k] = 1.0 / L.dx[k];
        }
        samples += L.samples;
        if ((long long)c->nv * L.n[0] * L.n[1] * L.n[2] >= (1LL << 31)) {
            delete c;
            return bad("one sample must hold fewer than 2^31 elements");
        }
    }
    if (samples > 65535) { delete c; return bad("at most 65535 samples per context"); }
    // MLMC coupling: companion groups point at the level they pair with
    {
        int comp_of[ALSV_MAX_LEVELS];
        for (int l = 0; l < ALSV_MAX_LEVELS; ++l) comp_of[l] = -1;
        for (int l = 0; l < ALSV_MAX_LEVELS; ++l) {
            const int j = d.level_fine[l];
            if (j == 0) continue;
            if (nlev < 2 || l >= nlev || j < 0 || j > nlev || j - 1 == l) {
                delete c;
                return bad("level_fine: 0, or 1 + the index of another group of the level table");
            }
            const int f = j - 1;
            if (d.level_fine[f] != 0) { delete c; return bad("level_fine: a companion must pair with a level"); }
            if (comp_of[f] >= 0) { delete c; return bad("level_fine: at most one companion per level"); }
            comp_of[f] = l;
            if (g.lev[f].samples != g.lev[l].samples) { delete c; return bad("level_fine: a companion needs its level's batch"); }
            for (int k = 0; k < d.ndim; ++k)
                if (g.lev[f].n[k] % g.lev[l].n[k] != 0) {
                    delete c;
                    return bad("level_fine: a companion's grid must divide its level's grid");
                }
        }
    }
    if (d.sampler != ALSV_SAMPLER_MC && d.sample_offset + samples >= (1LL << 31)) {
        delete c;
        return bad("Halton sampling needs sample indices below 2^31");
    }
    c->total_samples = (int)samples;
    g.total_samples = (int)samples;
    g.nv = c->nv;
    g.gamma = d.gamma;
    // the entropy-conservative fluxes read primitive cell values whatever recon_vars says
    g.rvars = d.eq == ALSV_EQ_EULER ? ((d.flux == ALSV_FLUX_EC || d.flux == ALSV_FLUX_EC4 || d.flux == ALSV_FLUX_TECNO2)
                                           ? ALSV_VARS_PRIM : d.recon_vars)
                                    : ALSV_VARS_CONS;
    for (int k = 0; k < 3; ++k) {
        g.bc[k][0] = d.bc[k][0];
        g.bc[k][1] = d.bc[k][1];
    }
    g.weno_eps = d.weno_eps;
    g.weno_eps_dx2 = d.weno_eps_dx2;
    fill_float_consts(g);
    for (int k = 0; k < 3; ++k) g.off[k] = d.offset[k];
    // tiling: keep the largest work count over variants for the partials buffer
    long long mx = 0;
    for (int v = 0; v < stage_num_variants(c->fp64, c->ndim); ++v) {
        GridArgs tmp = g;
        mx = std::max(mx, build_levels(c, v, tmp));
    }
    build_levels(c, 0, g);
    if (mx > INT_MAX) { delete c; return bad("too many tiles for one launch"); }
    c->max_work = mx;
    const size_t esz = c->fp64 ? 8 : 4;
    long long elems = 0;
    for (int l = 0; l < nlev; ++l) elems += (long long)g.lev[l].samples * c->nv * g.lev[l].n[0] * g.lev[l].n[1] * g.lev[l].n[2];
    c->state_bytes = (size_t)elems * esz;
    c->P = d.eq == ALSV_EQ_EULER ? (d.ndim == 3 ? 128 : (d.ndim == 2 ? 20 : 0)) : 0;
    size_t ws = 0;
    ws += align256(c->state_bytes);                               // A
    if (c->nstages == 3) ws += align256(c->state_bytes);          // B
    ws += align256((size_t)mx * 8);                               // partials
    ws += 3 * align256((size_t)samples * 8);                      // t, dt, nstep
    ws += 3 * align256((size_t)samples * 4);                      // done, last, FP32 dt
    ws += 256;                                                    // status
    ws += 256;                                                    // T_end, n_target, cfl_max
    ws += align256((size_t)samples * std::max(c->P, 1) * 8);      // theta
    ws += align256((size_t)reduce_partial_count(g) * 8);          // reduction partials
    c->ws_bytes = ws;
    c->h_done.resize(samples);
    if (workspace_bytes) *workspace_bytes = ws;
    *out = c;
    return ALSV_OK;
}

alsv_status alsv_bind_workspace(alsv_ctx* c, void* dev, size_t bytes) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    if (!dev) return fail(c, ALSV_ERR_INVALID_ARG, "null workspace pointer");
    if (((uintptr_t)dev & 255) != 0) return fail(c, ALSV_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (bytes < c->ws_bytes) return fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "workspace smaller than alsv_init_grid reported");
    drop_graph(c);
    char* p = (char*)dev;
    const size_t S = c->total_samples;
    c->ws = p;
    c->A = p; p += align256(c->state_bytes);
    if (c->nstages == 3) { c->Bb = p; p += align256(c->state_bytes); }
    c->part = (double*)p; p += align256((size_t)c->max_work * 8);
    c->t = (double*)p; p += align256(S * 8);
    c->dt = (double*)p; p += align256(S * 8);
    c->nstep = (int64_t*)p; p += align256(S * 8);
    c->done = (int*)p; p += align256(S * 4);
    c->last = (int*)p; p += align256(S * 4);
    c->dt_f = (float*)p; p += align256(S * 4);
    c->status = (int*)p; p += 256;
    c->T_end = (double*)p;
    c->n_target = (long long*)(p + 8);
    c->cfl_max = (double*)(p + 16); p += 256;
    c->theta = (double*)p; p += align256(S * std::max(c->P, 1) * 8);
    c->red = (double*)p;
    c->time_ready = false;
    return ALSV_OK;
}

size_t alsv_state_bytes(const alsv_ctx* c) { return c ? c->state_bytes : 0; }

alsv_status alsv_get_parameters(alsv_ctx* c, double* theta_dev) {
    alsv_status st = require_ready(c, false);
    if (st != ALSV_OK) return st;
    if (!theta_dev) return fail(c, ALSV_ERR_INVALID_ARG, "null output buffer");
    if (!c->have_theta || c->P == 0) return fail(c, ALSV_ERR_NOT_READY, "no KH parameters set");
    CK(cudaMemcpyAsync(theta_dev, c->theta, (size_t)c->total_samples * c->P * 8, cudaMemcpyDeviceToDevice, c->stream));
    return ALSV_OK;
}
int32_t alsv_num_samples(const alsv_ctx* c) { return c ? c->total_samples : 0; }
int32_t alsv_num_vars(const alsv_ctx* c) { return c ? c->nv : 0; }

static alsv_status set_run_params(alsv_ctx* c, double T, long long n_target) {
    double hv[2];
    hv[0] = T;
    std::memcpy(&hv[1], &n_target, 8);
    CK(cudaMemcpyAsync(c->T_end, hv, 16, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // hv lives on this stack frame
    return ALSV_OK;
}

alsv_status alsv_set_initial_data(alsv_ctx* c, int kind, const double* theta_dev, int n_params, void* U_dev,
                                  size_t U_bytes) {
    alsv_status st = require_ready(c, false);
    if (st != ALSV_OK) return st;
    if (!U_dev) return fail(c, ALSV_ERR_INVALID_ARG, "null state pointer");
    if (((uintptr_t)U_dev & 15) != 0) return fail(c, ALSV_ERR_INVALID_ARG, "state must be 16-byte aligned");
    if (U_bytes < c->state_bytes) return fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "state buffer smaller than alsv_state_bytes");
    if (kind < ALSV_INIT_KH || kind > ALSV_INIT_RAW) return fail(c, ALSV_ERR_INVALID_ARG, "unknown initial-data kind");
    if (kind == ALSV_INIT_KH && (c->eq != ALSV_EQ_EULER || c->ndim < 2))
        return fail(c, ALSV_ERR_INVALID_ARG, "KH initial data needs 2D or 3D Euler");
    if ((kind == ALSV_INIT_SOD || kind == ALSV_INIT_LAX) && c->eq != ALSV_EQ_EULER)
        return fail(c, ALSV_ERR_INVALID_ARG, "shock tubes need Euler");
    if (kind == ALSV_INIT_BURGERS_SINE && c->eq != ALSV_EQ_BURGERS)
        return fail(c, ALSV_ERR_INVALID_ARG, "sine initial data needs Burgers");
    if (kind == ALSV_INIT_VORTEX && (c->eq != ALSV_EQ_EULER || c->ndim != 2))
        return fail(c, ALSV_ERR_INVALID_ARG, "the vortex needs 2D Euler");
    c->U = U_dev;
    if (kind == ALSV_INIT_KH) {
        const double* th = theta_dev;
        if (!th) {
            ThetaMap tm;
            tm.nlev = c->g.nlev;
            for (int l = 0; l < c->g.nlev; ++l) {
                tm.sample0[l] = c->g.lev[l].sample0;
                const int f = c->d.n_levels > 1 ? c->d.level_fine[l] - 1 : -1;
                tm.src0[l] = f >= 0 ? c->g.lev[f].sample0 : c->g.lev[l].sample0;
            }
            cudaError_t e = launch_theta(c->d.seed, c->d.sample_offset, c->d.sampler, tm, c->total_samples, c->P,
                                         c->theta, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "theta kernel");
            th = c->theta;
        } else if (n_params != c->P) {
            return fail(c, ALSV_ERR_INVALID_ARG, "n_params must be 20 (2D KH) or 128 (3D KH)");
        }
        InitArgs a;
        a.g = c->g;
        a.U = U_dev;
        a.kind = 0;
        a.theta = th;
        a.P = c->P;
        cudaError_t e = launch_init(c->fp64, c->ndim, a, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
        if (th != c->theta)
            CK(cudaMemcpyAsync(c->theta, th, (size_t)c->total_samples * c->P * 8, cudaMemcpyDeviceToDevice, c->stream));
        c->have_theta = true;
    } else if (kind != ALSV_INIT_RAW) {
        InitArgs a;
        a.g = c->g;
        a.U = U_dev;
        a.kind = kind;
        a.theta = nullptr;
        a.P = 0;
        a.vortex_center[0] = c->d.vortex_center[0];
        a.vortex_center[1] = c->d.vortex_center[1];
        cudaError_t e = launch_init(c->fp64, c->ndim, a, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    }
    const size_t S = c->total_samples;
    CK(cudaMemsetAsync(c->t, 0, S * 8, c->stream));
    CK(cudaMemsetAsync(c->nstep, 0, S * 8, c->stream));
    CK(cudaMemsetAsync(c->done, 0, S * 4, c->stream));
    CK(cudaMemsetAsync(c->last, 0, S * 4, c->stream));
    CK(cudaMemsetAsync(c->status, 0, 4, c->stream));
    st = set_run_params(c, INFINITY, LLONG_MAX);
    if (st != ALSV_OK) return st;
    st = enqueue_speed_and_prepare(c);
    if (st != ALSV_OK) return st;
    c->time_ready = true;
    c->stage_next = 0;
    c->stage_parts = 0;
    return ALSV_OK;
}

alsv_status alsv_set_time(alsv_ctx* c, const double* t_host, const int64_t* steps_host) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!t_host) return fail(c, ALSV_ERR_INVALID_ARG, "null time array");
    const size_t S = c->total_samples;
    for (size_t i = 0; i < S; ++i)
        if (!std::isfinite(t_host[i]) || t_host[i] < 0.0) return fail(c, ALSV_ERR_INVALID_ARG, "times must be finite and >= 0");
    CK(cudaMemcpyAsync(c->t, t_host, S * 8, cudaMemcpyHostToDevice, c->stream));
    if (steps_host) CK(cudaMemcpyAsync(c->nstep, steps_host, S * 8, cudaMemcpyHostToDevice, c->stream));
    else CK(cudaMemsetAsync(c->nstep, 0, S * 8, c->stream));
    CK(cudaMemsetAsync(c->done, 0, S * 4, c->stream));
    CK(cudaMemsetAsync(c->last, 0, S * 4, c->stream));
    CK(cudaStreamSynchronize(c->stream));   // the host arrays may be released after return
    st = enqueue_speed_and_prepare(c);
    if (st != ALSV_OK) return st;
    c->time_ready = true;
    c->stage_next = 0;
    c->stage_parts = 0;
    return ALSV_OK;
}

alsv_status alsv_step(alsv_ctx* c, int n_steps) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (n_steps < 0) return fail(c, ALSV_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (ctx_has_halo(c)) return fail(c, ALSV_ERR_INVALID_ARG, "halo faces: step with alsv_stage / alsv_finish_step");
    NvtxRange range("alsv: steps");
    for (int i = 0; i < n_steps; ++i) {
        st = enqueue_step(c);
        if (st != ALSV_OK) return st;
    }
    return ALSV_OK;
}

alsv_status alsv_sync(alsv_ctx* c) {
    alsv_status st = require_ready(c, false);
    if (st != ALSV_OK) return st;
    int hs = 0;
    st = read_status(c, &hs);
    if (st != ALSV_OK) return st;
    prof_collect(c);
    return status_to_code(c, hs);
}

alsv_status alsv_evolve_to_T(alsv_ctx* c, double T, int64_t* steps_taken_host) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!std::isfinite(T) || T < 0.0) return fail(c, ALSV_ERR_INVALID_ARG, "T must be finite and >= 0");
    if (ctx_has_halo(c)) return fail(c, ALSV_ERR_INVALID_ARG, "halo faces: step with alsv_stage / alsv_finish_step");
    long long n_target = LLONG_MAX;
    if (c->d.fixed_dt > 0.0) n_target = (long long)std::ceil(T / c->d.fixed_dt * (1.0 - 1e-12));
    st = set_run_params(c, T, n_target);
    if (st != ALSV_OK) return st;
    FinishArgs f = finish_args(c, 0);
    cudaError_t e = launch_finish(f, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finish kernel launch");
    c->launches++;
    const int chunk = 16;
    const size_t S = c->total_samples;
    // Two polls in flight: the next chunk is enqueued before the host reads the done flags and
    // status of the previous one (pinned slots), so the GPU does not idle during the round trip.
    // A chunk that runs after every sample is done changes nothing (stages and time control skip
    // done samples).
    const size_t slot_bytes = (S * 4 + 16 + 255) / 256 * 256;
    if (!c->h_poll) {
        CK(cudaHostAlloc(reinterpret_cast<void**>(&c->h_poll), 2 * slot_bytes, cudaHostAllocDefault));
        for (int k = 0; k < 2; ++k) CK(cudaEventCreateWithFlags(&c->poll_ev[k], cudaEventDisableTiming));
    }
    auto slot_done = [&](int k) { return reinterpret_cast<int*>(c->h_poll + k * slot_bytes); };
    auto slot_status = [&](int k) { return reinterpret_cast<int*>(c->h_poll + k * slot_bytes + S * 4); };
    auto post = [&](int k) -> cudaError_t {
        cudaError_t ee = cudaMemcpyAsync(slot_done(k), c->done, S * 4, cudaMemcpyDeviceToHost, c->stream);
        if (ee == cudaSuccess) ee = cudaMemcpyAsync(slot_status(k), c->status, 4, cudaMemcpyDeviceToHost, c->stream);
        if (ee == cudaSuccess) ee = cudaEventRecord(c->poll_ev[k], c->stream);
        return ee;
    };
    CK(post(0));
    int cur = 0;
    long long chunks = 0;
    // every exit restores the full level table (and drops a chunk captured with a reduced one)
    struct LiveReset {
        alsv_ctx* c;
        ~LiveReset() {
            if (c->live_levels != ~0u || c->any_done) {
                c->live_levels = ~0u;
                c->any_done = 0;
                drop_graph(c);
            }
        }
    } live_reset{c};
    for (;;) {
        if (++chunks > (1LL << 26)) return fail(c, ALSV_ERR_TIMEOUT, "evolve_to_T: step limit reached");
        {
            NvtxRange range("alsv: step chunk");
            st = run_chunk(c, chunk);
        }
        if (st != ALSV_OK) return st;
        CK(post(cur ^ 1));
        CK(cudaEventSynchronize(c->poll_ev[cur]));
        const int hs = *slot_status(cur);
        if (hs & (ST_NONPHYSICAL | ST_CFL)) {
            st = status_to_code(c, hs);
            break;
        }
        const int* dn = slot_done(cur);
        bool all = true;
        for (size_t i = 0; i < S && all; ++i) all = dn[i] != 0;
        if (all) break;
        if (!c->any_done && pair_schedule(c)) {
            // from the first finished sample on, finished pairs skip their tile load
            bool any = false;
            for (size_t i = 0; i < S && !any; ++i) any = dn[i] != 0;
            if (any) {
                c->any_done = 1;
                drop_graph(c);
            }
        }
        if (c->g.nlev > 1 && pair_schedule(c)) {
            // leave out levels whose samples have all finished (done flags never clear during a
            // run); the captured chunk holds the level table, so a change re-captures it
            unsigned live = 0;
            for (int l = 0; l < c->g.nlev; ++l) {
                const LevelInfo& L = c->g.lev[l];
                bool any = false;
                for (int i = 0; i < L.samples && !any; ++i) any = dn[L.sample0 + i] == 0;
                if (any) live |= 1u << l;
            }
            if (live != (c->live_levels & ((1u << c->g.nlev) - 1u))) {
                c->live_levels = live;
                drop_graph(c);
            }
        }
        cur ^= 1;
    }
    prof_collect(c);
    if (steps_taken_host) {
        std::vector<int64_t> ns(S);
        CK(cudaMemcpyAsync(ns.data(), c->nstep, S * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        int64_t mx = 0;
        for (auto v : ns) mx = std::max(mx, v);
        *steps_taken_host = mx;
    }
    return st;
}

alsv_status alsv_evolve_resident(alsv_ctx* c, double T, int64_t* steps_taken_host) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!std::isfinite(T) || T < 0.0) return fail(c, ALSV_ERR_INVALID_ARG, "T must be finite and >= 0");
    if (c->fp64 || c->ndim != 2 || c->eq != ALSV_EQ_EULER || c->g.nlev != 1 || c->g.rvars != RV_PRIM)
        return fail(c, ALSV_ERR_INVALID_ARG, "the resident schedule serves FP32 2D Euler, one grid, primitive reconstruction");
    if (c->d.recon > REC_WENO3 || (c->d.flux != FLX_HLLC && c->d.flux != FLX_RUSANOV))
        return fail(c, ALSV_ERR_INVALID_ARG, "the resident schedule serves PC / MC / WENO3 with HLLC or Rusanov");
    for (int k = 0; k < 2; ++k)
        if (c->g.bc[k][0] != BC_PERIODIC || c->g.bc[k][1] != BC_PERIODIC)
            return fail(c, ALSV_ERR_INVALID_ARG, "the resident schedule needs periodic boundaries in x and y");
    if (c->d.fixed_dt > 0.0) return fail(c, ALSV_ERR_INVALID_ARG, "the resident schedule takes CFL steps (fixed_dt = 0)");
    const int nx = c->g.lev[0].n[0], ny = c->g.lev[0].n[1];
    if (nx % 32 != 0 || nx > 1024) return fail(c, ALSV_ERR_INVALID_ARG, "the resident schedule needs nx a multiple of 32, at most 1024");
    // the smallest cluster whose shared memory holds the sample (each CTA at least two rows)
    int cs = 0;
    for (int k = 1; k <= 16; k *= 2) {
        if (ny % k != 0 || ny / k < 2) continue;
        if (resident_smem_bytes(nx, ny / k) <= 227 * 1024) {
            cs = k;
            break;
        }
    }
    if (cs == 0) return fail(c, ALSV_ERR_INVALID_ARG, "the sample does not fit one cluster's shared memory (at most 16 CTAs)");
    st = set_run_params(c, T, LLONG_MAX);
    if (st != ALSV_OK) return st;
    ResidentArgs a;
    a.g = c->g;
    a.U = static_cast<float*>(c->U);
    a.t = c->t;
    a.dt = c->dt;
    a.dt_f = c->dt_f;
    a.nstep = c->nstep;
    a.done = c->done;
    a.last = c->last;
    a.status = c->status;
    a.T = T;
    a.cfl = c->d.cfl;
    a.max_steps = 1LL << 40;
    a.rk = c->nstages;
    a.cs = cs;
    cudaError_t e = launch_resident(a, c->d.recon, c->d.flux, nx, ny / cs, c->total_samples, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "resident kernel launch");
    c->launches++;
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, c->status, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hs & (ST_NONPHYSICAL | ST_CFL)) return status_to_code(c, hs);
    if (steps_taken_host) {
        const size_t S = c->total_samples;
        std::vector<int64_t> ns(S);
        CK(cudaMemcpyAsync(ns.data(), c->nstep, S * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        int64_t mx = 0;
        for (auto v : ns) mx = std::max(mx, v);
        *steps_taken_host = mx;
    }
    return ALSV_OK;
}

alsv_status alsv_get_time(alsv_ctx* c, double* t_host, int64_t* steps_host) {
    alsv_status st = require_ready(c, false);
    if (st != ALSV_OK) return st;
    const size_t S = c->total_samples;
    if (t_host) CK(cudaMemcpyAsync(t_host, c->t, S * 8, cudaMemcpyDeviceToHost, c->stream));
    if (steps_host) CK(cudaMemcpyAsync(steps_host, c->nstep, S * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ALSV_OK;
}

size_t alsv_stats_bytes(const alsv_ctx* c) {
    if (!c) return 0;
    const LevelInfo& L = c->g.lev[0];
    const size_t C = (size_t)L.n[0] * L.n[1] * L.n[2];
    return 256 + 2 * (size_t)c->nv * C * 8;
}

static alsv_status check_stats(alsv_ctx* c, const void* stats, size_t bytes) {
    if (!stats) return fail(c, ALSV_ERR_INVALID_ARG, "null statistics buffer");
    if (((uintptr_t)stats & 255) != 0) return fail(c, ALSV_ERR_INVALID_ARG, "statistics buffer must be 256-byte aligned");
    if (bytes < alsv_stats_bytes(c)) return fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "statistics buffer smaller than alsv_stats_bytes");
    if (c->g.nlev != 1) return fail(c, ALSV_ERR_INVALID_ARG, "statistics need a single-level context");
    return ALSV_OK;
}

alsv_status alsv_stats_reset(alsv_ctx* c, void* stats_dev, size_t bytes) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    alsv_status st = check_stats(c, stats_dev, bytes);
    if (st != ALSV_OK) return st;
    CK(cudaMemsetAsync(stats_dev, 0, alsv_stats_bytes(c), c->stream));
    return ALSV_OK;
}

alsv_status alsv_stats_accumulate(alsv_ctx* c, void* stats_dev, size_t bytes) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    st = check_stats(c, stats_dev, bytes);
    if (st != ALSV_OK) return st;
    cudaError_t e = launch_welford(c->fp64, c->g, c->U, stats_dev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "welford kernel");
    c->launches += 2;
    return ALSV_OK;
}

alsv_status alsv_stats_read(alsv_ctx* c, const void* stats_dev, double* mean_dev, double* var_dev, int64_t* count_host) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    alsv_status st = check_stats(c, stats_dev, alsv_stats_bytes(c));
    if (st != ALSV_OK) return st;
    if (mean_dev || var_dev) {
        cudaError_t e = launch_stats_read(c->g, stats_dev, mean_dev, var_dev, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "stats read kernel");
        c->launches++;
    }
    if (count_host) {
        CK(cudaMemcpyAsync(count_host, stats_dev, 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return ALSV_OK;
}

alsv_status alsv_stats_merge(alsv_ctx* c, void* stats_dev, const void* other_dev, size_t bytes) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    alsv_status st = check_stats(c, stats_dev, bytes);
    if (st != ALSV_OK) return st;
    st = check_stats(c, other_dev, bytes);
    if (st != ALSV_OK) return st;
    if (stats_dev == other_dev) return fail(c, ALSV_ERR_INVALID_ARG, "stats and other must differ");
    cudaError_t e = launch_stats_merge(c->g, stats_dev, other_dev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stats merge kernel");
    c->launches += 2;
    return ALSV_OK;
}

alsv_status alsv_conservation_totals(alsv_ctx* c, double* totals_dev) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!totals_dev) return fail(c, ALSV_ERR_INVALID_ARG, "null totals buffer");
    cudaError_t e = launch_reduce(c->fp64, 0, c->g, c->U, c->red, totals_dev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduction kernel");
    c->launches += 2;
    return ALSV_OK;
}

alsv_status alsv_mixing_width(alsv_ctx* c, double* w_dev) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!w_dev) return fail(c, ALSV_ERR_INVALID_ARG, "null output");
    if (c->eq != ALSV_EQ_EULER) return fail(c, ALSV_ERR_INVALID_ARG, "the mixing-layer width needs Euler");
    cudaError_t e = launch_reduce(c->fp64, 2, c->g, c->U, c->red, w_dev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduction kernel launch");
    c->launches += 2;
    return ALSV_OK;
}

alsv_status alsv_kinetic_energy(alsv_ctx* c, double* ke_dev) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!ke_dev) return fail(c, ALSV_ERR_INVALID_ARG, "null output buffer");
    if (c->eq != ALSV_EQ_EULER) return fail(c, ALSV_ERR_INVALID_ARG, "kinetic energy needs Euler");
    cudaError_t e = launch_reduce(c->fp64, 1, c->g, c->U, c->red, ke_dev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduction kernel");
    c->launches += 2;
    return ALSV_OK;
}

alsv_status alsv_destroy(alsv_ctx* c) {
    if (!c) return ALSV_OK;
    drop_graph(c);
    if (c->h_poll) {
        cudaStreamSynchronize(c->stream);
        for (int k = 0; k < 2; ++k) cudaEventDestroy(c->poll_ev[k]);
        cudaFreeHost(c->h_poll);
    }
    for (auto e : c->prof.ev) cudaEventDestroy(e);
    delete c;
    return ALSV_OK;
}

// ---------------------------------------------------------------------------------------------
// Execution controls (declared in alsv.h): tile-shape selection/autotuning, launch counting, profiling
// ---------------------------------------------------------------------------------------------
alsv_status alsv_set_tile_variant(alsv_ctx* c, int variant) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    if (variant < 0 || variant >= stage_num_variants(c->fp64, c->ndim))
        return fail(c, ALSV_ERR_INVALID_ARG, "tile variant out of range");
    if (!variant_ok(c, variant)) return fail(c, ALSV_ERR_INVALID_ARG, "tile variant does not support this scheme");
    if (variant == c->variant) return ALSV_OK;
    c->variant = variant;
    build_levels(c, variant, c->g);
    drop_graph(c);
    if (c->U && c->ws && c->time_ready) {
        // partials follow the tiling: recompute them for the current state
        cudaError_t e = launch_speed(c->fp64, c->ndim, c->eq, c->variant, c->g, c->U, c->part, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "speed kernel launch");
        c->launches++;
    }
    return ALSV_OK;
}

int alsv_num_tile_variants(const alsv_ctx* c) { return c ? stage_num_variants(c->fp64, c->ndim) : 0; }

alsv_status alsv_autotune(alsv_ctx* c, int reps, int* chosen, float* ms_per_variant) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (ctx_has_halo(c) && !c->halo_bound) return fail(c, ALSV_ERR_NOT_READY, "halo buffers not bound (alsv_bind_halo)");
    if (reps < 1) reps = 1;
    const int nvar = stage_num_variants(c->fp64, c->ndim);
    int best = c->variant;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int v = 0; v < nvar; ++v) {
        if (!variant_ok(c, v)) {
            if (ms_per_variant) ms_per_variant[v] = -1.0f;
            continue;
        }
        GridArgs g = c->g;
        const int saved = c->variant;
        c->variant = v;
        build_levels(c, v, c->g);
        // timed: a first-stage launch (reads U, writes the stage buffer A) and a last-stage-like
        // launch (also reads U^n point-wise and forms the CFL partials), both writing only scratch,
        // so the state is unchanged; the partials are recomputed below
        StageArgs a = stage_args(c, c->U, nullptr, c->A, 0.0, 1.0, false);
        StageArgs a3 = stage_args(c, c->U, c->U, c->A, 1.0 / 3.0, 2.0 / 3.0, true);
        cudaError_t e = launch_stage(c->fp64, c->ndim, c->eq, c->d.recon, c->d.flux, v, a, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = launch_stage(c->fp64, c->ndim, c->eq, c->d.recon, c->d.flux, v, a, c->stream);
            if (e == cudaSuccess) e = launch_stage(c->fp64, c->ndim, c->eq, c->d.recon, c->d.flux, v, a3, c->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        c->launches += 2 * reps + 1;
        c->variant = saved;
        c->g = g;
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(c, e, "autotune launch");
        }
        ms /= reps;
        if (ms_per_variant) ms_per_variant[v] = ms;
        // a later variant must be faster by more than 1 % to replace an earlier one, so that
        // schedules of equal speed do not trade places from run to run
        if (ms < best_ms * 0.99f) { best_ms = ms; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosen) *chosen = best;
    st = alsv_set_tile_variant(c, best);
    if (st != ALSV_OK) return st;
    // partials of the current state for the chosen tiling (the timing launches overwrote them)
    cudaError_t e = launch_speed(c->fp64, c->ndim, c->eq, c->variant, c->g, c->U, c->part, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "speed kernel launch");
    c->launches++;
    return ALSV_OK;
}

alsv_status alsv_get_launch_count(const alsv_ctx* c, int64_t* launches) {
    if (!c || !launches) return ALSV_ERR_INVALID_ARG;
    *launches = c->launches;
    return ALSV_OK;
}

alsv_status alsv_set_profiling(alsv_ctx* c, int on) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    prof_collect(c);
    c->prof.on = on != 0;
    c->prof.stage_ms = c->prof.finish_ms = 0.0;
    c->prof.stage_launches = c->prof.finish_launches = 0;
    return ALSV_OK;
}

alsv_status alsv_get_profile(alsv_ctx* c, double* stage_ms, int64_t* stage_launches, double* finish_ms,
                             int64_t* finish_launches) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    prof_collect(c);
    if (stage_ms) *stage_ms = c->prof.stage_ms;
    if (stage_launches) *stage_launches = c->prof.stage_launches;
    if (finish_ms) *finish_ms = c->prof.finish_ms;
    if (finish_launches) *finish_launches = c->prof.finish_launches;
    return ALSV_OK;
}

alsv_status alsv_set_graphs(alsv_ctx* c, int on) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    c->graphs_enabled = on != 0;
    drop_graph(c);
    return ALSV_OK;
}

alsv_status alsv_get_tile(const alsv_ctx* c, int* tx, int* ty, int* tz, int* variant, int64_t* work_items) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    TileShape t = stage_tile(c->fp64, c->ndim, c->variant);
    if (tx) *tx = t.tx;
    if (ty) *ty = t.ty;
    if (tz) *tz = t.tz;
    if (variant) *variant = c->variant;
    if (work_items) *work_items = c->g.total_work;
    return ALSV_OK;
}

// ---------------------------------------------------------------------------------------------
// Domain decomposition (Sec. 2.1, last paragraph; Sec. 3.1): a block of a decomposed grid steps
// stage by stage; the caller refills its halo buffers between stages and takes the CFL maximum
// over every block.
// ---------------------------------------------------------------------------------------------
static long long halo_elems(const alsv_ctx* c, int f) {
    const int k = f >> 1;
    if (k >= c->ndim || c->g.bc[k][f & 1] != BC_HALO) return 0;
    const LevelInfo& L = c->g.lev[0];
    const long long cross = (long long)L.n[0] * L.n[1] * L.n[2] / L.n[k];
    return (long long)L.samples * c->nv * c->G * cross;
}

alsv_status alsv_halo_info(const alsv_ctx* c, int32_t* layers, int64_t* elems) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    if (layers) *layers = c->G;
    if (elems)
        for (int f = 0; f < 6; ++f) elems[f] = halo_elems(c, f);
    return ALSV_OK;
}

alsv_status alsv_bind_halo(alsv_ctx* c, const void* const* halo_dev, const size_t* bytes) {
    if (!c) return fail(nullptr, ALSV_ERR_INVALID_ARG, "null context");
    if (!halo_dev || !bytes) return fail(c, ALSV_ERR_INVALID_ARG, "null halo pointer or size array");
    const size_t esz = c->fp64 ? 8 : 4;
    for (int f = 0; f < 6; ++f) {
        const long long n = halo_elems(c, f);
        if (n == 0) continue;
        if (!halo_dev[f]) return fail(c, ALSV_ERR_INVALID_ARG, "a halo face needs a buffer");
        if (((uintptr_t)halo_dev[f] & 15) != 0) return fail(c, ALSV_ERR_INVALID_ARG, "halo buffers must be 16-byte aligned");
        if (bytes[f] < (size_t)n * esz) return fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "halo buffer smaller than alsv_halo_info's size");
    }
    for (int f = 0; f < 6; ++f) c->halo[f] = halo_elems(c, f) ? halo_dev[f] : nullptr;
    c->halo_bound = true;
    return ALSV_OK;
}

alsv_status alsv_halo_pack(alsv_ctx* c, int stage, void* const* send_dev, const size_t* bytes) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (c->g.nlev != 1) return fail(c, ALSV_ERR_INVALID_ARG, "halo layers need a single grid");
    if (stage < 0 || stage >= c->nstages) return fail(c, ALSV_ERR_INVALID_ARG, "stage out of range");
    if (!send_dev || !bytes) return fail(c, ALSV_ERR_INVALID_ARG, "null send pointer or size array");
    const size_t esz = c->fp64 ? 8 : 4;
    void* dst[6];
    for (int f = 0; f < 6; ++f) {
        dst[f] = send_dev[f];
        if (!dst[f]) continue;
        const int k = f >> 1;
        if (k >= c->ndim) return fail(c, ALSV_ERR_INVALID_ARG, "send buffer for an inactive direction");
        if (c->g.lev[0].n[k] < c->G) return fail(c, ALSV_ERR_INVALID_ARG, "fewer cells than ghost layers across a face");
        const LevelInfo& L = c->g.lev[0];
        const long long n = (long long)L.samples * c->nv * c->G * ((long long)L.n[0] * L.n[1] * L.n[2] / L.n[k]);
        if (bytes[f] < (size_t)n * esz) return fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "send buffer smaller than a face's layers");
    }
    const void* src = stage_io(c, stage).Us;
    cudaError_t e = launch_halo_pack(c->fp64, c->g, c->G, src, dst, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "halo pack kernel");
    for (int f = 0; f < 6; ++f) c->launches += dst[f] ? 1 : 0;
    return ALSV_OK;
}

alsv_status alsv_stage(alsv_ctx* c, int stage) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!c->time_ready) return fail(c, ALSV_ERR_NOT_READY, "no time state (alsv_set_initial_data)");
    if (ctx_has_halo(c) && !c->halo_bound) return fail(c, ALSV_ERR_NOT_READY, "halo buffers not bound (alsv_bind_halo)");
    if (stage != c->stage_next || stage >= c->nstages)
        return fail(c, ALSV_ERR_INVALID_ARG, "stages run in order 0 .. stages-1, then alsv_finish_step");
    if (c->stage_parts != 0) return fail(c, ALSV_ERR_INVALID_ARG, "stage already started in parts (alsv_stage_part)");
    st = enqueue_stage(c, stage);
    if (st != ALSV_OK) return st;
    c->stage_next = stage + 1;
    return ALSV_OK;
}

alsv_status alsv_stage_part(alsv_ctx* c, int stage, int part) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!c->time_ready) return fail(c, ALSV_ERR_NOT_READY, "no time state (alsv_set_initial_data)");
    if (part != ALSV_PART_INTERIOR && part != ALSV_PART_BOUNDARY)
        return fail(c, ALSV_ERR_INVALID_ARG, "part must be ALSV_PART_INTERIOR or ALSV_PART_BOUNDARY");
    if (stage != c->stage_next || stage >= c->nstages)
        return fail(c, ALSV_ERR_INVALID_ARG, "stages run in order 0 .. stages-1, then alsv_finish_step");
    const int bit = part == ALSV_PART_INTERIOR ? 1 : 2;
    if (c->stage_parts & bit) return fail(c, ALSV_ERR_INVALID_ARG, "this part of the stage already ran");
    // the boundary part reads the halo buffers: they must be bound (the interior part reads none)
    if (part == ALSV_PART_BOUNDARY && ctx_has_halo(c) && !c->halo_bound)
        return fail(c, ALSV_ERR_NOT_READY, "halo buffers not bound (alsv_bind_halo)");
    st = enqueue_stage(c, stage, part == ALSV_PART_INTERIOR ? 1 : 2);
    if (st != ALSV_OK) return st;
    c->stage_parts |= bit;
    if (c->stage_parts == 3) {
        c->stage_parts = 0;
        c->stage_next = stage + 1;
    }
    return ALSV_OK;
}

alsv_status alsv_speed_max(alsv_ctx* c, double* smax_dev) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!smax_dev) return fail(c, ALSV_ERR_INVALID_ARG, "null output");
    if ((c->stage_next != 0 && c->stage_next != c->nstages) || c->stage_parts != 0)
        return fail(c, ALSV_ERR_INVALID_ARG, "the maximum speed is defined before the first or after the last stage");
    FinishArgs f = finish_args(c, 0);
    f.smax_out = smax_dev;
    cudaError_t e = launch_finish(f, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finish kernel launch");
    c->launches++;
    return ALSV_OK;
}

alsv_status alsv_speed_max_combine(const double* const* smax_dev, int n, int samples, double* out_dev, void* stream) {
    auto bad = [](alsv_status st, const std::string& m) {
        set_global_error("alsv_speed_max_combine: " + m);
        return st;
    };
    if (!smax_dev || !out_dev) return bad(ALSV_ERR_INVALID_ARG, "null input array or output");
    if (n < 1 || n > kSpeedCombineMax)
        return bad(ALSV_ERR_INVALID_ARG, "n must be 1 .. " + std::to_string(kSpeedCombineMax));
    if (samples < 0) return bad(ALSV_ERR_INVALID_ARG, "samples must be >= 0");
    SpeedCombineArgs a{};
    a.n = n;
    for (int i = 0; i < n; ++i) {
        if (!smax_dev[i]) return bad(ALSV_ERR_INVALID_ARG, "null input " + std::to_string(i));
        a.in[i] = smax_dev[i];
    }
    const cudaError_t e = launch_speed_max_combine(a, samples, out_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return bad(ALSV_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return ALSV_OK;
}

alsv_status alsv_finish_step(alsv_ctx* c, const double* smax_dev, int advance) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!smax_dev) return fail(c, ALSV_ERR_INVALID_ARG, "null maximum");
    if ((advance ? c->stage_next != c->nstages : c->stage_next != 0) || c->stage_parts != 0)
        return fail(c, ALSV_ERR_INVALID_ARG, advance ? "advance = 1 follows the last stage" : "advance = 0 comes before the first stage");
    FinishArgs f = finish_args(c, advance ? 1 : 0);
    f.smax_in = smax_dev;
    cudaError_t e = launch_finish(f, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finish kernel launch");
    c->launches++;
    c->stage_next = 0;
    c->stage_parts = 0;
    return ALSV_OK;
}

alsv_status alsv_set_end_time(alsv_ctx* c, double T) {
    alsv_status st = require_ready(c);
    if (st != ALSV_OK) return st;
    if (!std::isfinite(T) || T < 0.0) return fail(c, ALSV_ERR_INVALID_ARG, "T must be finite and >= 0");
    long long n_target = LLONG_MAX;
    if (c->d.fixed_dt > 0.0) n_target = (long long)std::ceil(T / c->d.fixed_dt * (1.0 - 1e-12));
    return set_run_params(c, T, n_target);
}

}  // extern "C"

// Launch dispatch over (precision, ndim) to the per-TU launchers.
namespace alsv {
cudaError_t launch_stage_f32_1d(int, int, int, int, const StageArgs&, cudaStream_t);
cudaError_t launch_stage_f64_1d(int, int, int, int, const StageArgs&, cudaStream_t);
cudaError_t launch_stage_f32_2d(int, int, int, int, const StageArgs&, cudaStream_t);
cudaError_t launch_stage_f64_2d(int, int, int, int, const StageArgs&, cudaStream_t);
cudaError_t launch_stage_f32_3d(int, int, int, int, const StageArgs&, cudaStream_t);
cudaError_t launch_stage_f64_3d(int, int, int, int, const StageArgs&, cudaStream_t);
cudaError_t launch_speed_f32_1d(int, int, const GridArgs&, const void*, double*, cudaStream_t);
cudaError_t launch_speed_f64_1d(int, int, const GridArgs&, const void*, double*, cudaStream_t);
cudaError_t launch_speed_f32_2d(int, int, const GridArgs&, const void*, double*, cudaStream_t);
cudaError_t launch_speed_f64_2d(int, int, const GridArgs&, const void*, double*, cudaStream_t);
cudaError_t launch_speed_f32_3d(int, int, const GridArgs&, const void*, double*, cudaStream_t);
cudaError_t launch_speed_f64_3d(int, int, const GridArgs&, const void*, double*, cudaStream_t);

cudaError_t launch_stage(int fp64, int ndim, int eq, int recon, int flux, int variant, const StageArgs& a,
                         cudaStream_t s) {
    if (ext_scheme(recon, flux)) {
        if (variant != 0) return cudaErrorNotSupported;
        if (ndim == 1) return fp64 ? launch_stage_ext_f64_1d(eq, recon, flux, a, s) : launch_stage_ext_f32_1d(eq, recon, flux, a, s);
        if (ndim == 2) return fp64 ? launch_stage_ext_f64_2d(eq, recon, flux, a, s) : launch_stage_ext_f32_2d(eq, recon, flux, a, s);
        return fp64 ? launch_stage_ext_f64_3d(eq, recon, flux, a, s) : launch_stage_ext_f32_3d(eq, recon, flux, a, s);
    }
    if (ndim == 1) return fp64 ? launch_stage_f64_1d(variant, eq, recon, flux, a, s) : launch_stage_f32_1d(variant, eq, recon, flux, a, s);
    if (ndim == 2) return fp64 ? launch_stage_f64_2d(variant, eq, recon, flux, a, s) : launch_stage_f32_2d(variant, eq, recon, flux, a, s);
    return fp64 ? launch_stage_f64_3d(variant, eq, recon, flux, a, s) : launch_stage_f32_3d(variant, eq, recon, flux, a, s);
}

cudaError_t launch_speed(int fp64, int ndim, int eq, int variant, const GridArgs& g, const void* U, double* part,
                         cudaStream_t s) {
    if (ndim == 1) return fp64 ? launch_speed_f64_1d(variant, eq, g, U, part, s) : launch_speed_f32_1d(variant, eq, g, U, part, s);
    if (ndim == 2) return fp64 ? launch_speed_f64_2d(variant, eq, g, U, part, s) : launch_speed_f32_2d(variant, eq, g, U, part, s);
    return fp64 ? launch_speed_f64_3d(variant, eq, g, U, part, s) : launch_speed_f32_3d(variant, eq, g, U, part, s);
}
}  // namespace alsv
