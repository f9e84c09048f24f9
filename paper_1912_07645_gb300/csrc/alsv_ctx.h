// Host-side context of the C ABI (internal; shared by alsv_api.cu and adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/alsv.h"
#include "alsv_internal.h"

namespace alsv {
struct Profile {
    bool on = false;
    double stage_ms = 0.0, finish_ms = 0.0;
    long long stage_launches = 0, finish_launches = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<int> kinds;  // 0 stage, 1 finish; kinds[i] is the kernel between ev[i] and ev[i+1]
};
}  // namespace alsv

struct alsv_ctx {
    alsv_grid_desc d;
    cudaStream_t stream = nullptr;
    int fp64 = 0, ndim = 1, nv = 1, eq = 1, G = 2, nstages = 2;
    int variant = 0;
    alsv::GridArgs g;
    int total_samples = 0;
    long long max_work = 0;  // largest work-item count over the tile variants
    size_t state_bytes = 0, ws_bytes = 0;
    int P = 0;               // KH parameters per sample
    // workspace regions
    char* ws = nullptr;
    void* A = nullptr;
    void* Bb = nullptr;
    double* part = nullptr;
    double* t = nullptr;
    double* dt = nullptr;
    float* dt_f = nullptr;
    int64_t* nstep = nullptr;
    int* done = nullptr;
    int* last = nullptr;
    int* status = nullptr;
    double* T_end = nullptr;
    long long* n_target = nullptr;
    double* cfl_max = nullptr;   // fixed mode: running maximum of the realised CFL number
    double* theta = nullptr;
    double* red = nullptr;
    // state
    void* U = nullptr;
    bool time_ready = false;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    void* g_U = nullptr;
    int g_variant = -1;
    int g_steps = 0;
    // levels whose stage work is launched (bit l = level l; all set outside alsv_evolve_to_T): the
    // two-sample schedules leave out levels whose samples have all finished
    unsigned live_levels = ~0u;
    int any_done = 0;   // some sample finished (set from the done-flag polls of alsv_evolve_to_T)
    bool graphs_enabled = true;
    // host staging
    std::vector<int> h_done;
    char* h_poll = nullptr;          // pinned: done flags + status of two polls in flight
    cudaEvent_t poll_ev[2] = {nullptr, nullptr};
    long long launches = 0;
    alsv::Profile prof;
    std::string err;
    // adjoint workspace (caller-owned)
    char* adj_ws = nullptr;
    size_t adj_bytes = 0;
    long long adj_n = 0;         // plan of the last adjoint call: steps, step, forward passes
    double adj_dt = 0.0;
    int adj_passes = 0;
    bool have_theta = false;
    // block of a decomposed grid: caller-bound halo buffers per face, next stage of the
    // stage-by-stage protocol (alsv_stage / alsv_finish_step)
    const void* halo[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool halo_bound = false;
    int stage_next = 0;
    int stage_parts = 0;   // parts of stage stage_next already enqueued (1 interior, 2 boundary)
};

namespace alsv {
// shared helpers implemented in alsv_api.cu
alsv_status ctx_fail(alsv_ctx* c, alsv_status st, const std::string& msg);
alsv_status ctx_cuda_fail(alsv_ctx* c, cudaError_t e, const char* what);
FinishArgs ctx_finish_args(alsv_ctx* c, int advance);
StageArgs ctx_stage_args(alsv_ctx* c, const void* Us, const void* Un, void* Uout, double a, double b, bool want_speed);
// whether any face of the context is a halo face of a decomposed grid
bool ctx_has_halo(const alsv_ctx* c);
}  // namespace alsv
