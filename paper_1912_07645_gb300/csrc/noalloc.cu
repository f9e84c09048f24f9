// Allocation-free variant of the conservation-totals reduction.
//
// Some callers cannot allocate device memory at all: a plugin inside a host framework that owns
// every device buffer and hands its plugins no allocator, or a service running under a fixed
// device-memory budget where a cudaMalloc (or torch's caching allocator) could fail under memory
// pressure or synchronise the device in the middle of its work. They cannot provide the workspace
// a context needs. For them alsv_conservation_totals_noalloc computes the same FP64 totals with
// the same two kernels as alsv_conservation_totals, but keeps the per-chunk partial sums in the
// file-scope device array below instead of in a caller workspace.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/alsv.h"
#include "alsv_internal.h"

namespace alsv {
void set_global_error(const std::string& msg);  // alsv_last_error(NULL) reports it
}

namespace {

// Scratch for the per-chunk partial sums: at most kNoallocPartials doubles (8 MiB). Every GPU that
// loads this library holds it until the process exits. All calls share it.
constexpr long long kNoallocPartials = 1LL << 20;
static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

alsv_status bad(alsv_status st, const std::string& m) {
    alsv::set_global_error("alsv_conservation_totals_noalloc: " + m);
    return st;
}

}  // namespace

extern "C" alsv_status alsv_conservation_totals_noalloc(const alsv_grid_desc* d, const void* U_dev, size_t U_bytes,
                                                        double* totals_dev, void* stream) {
    using namespace alsv;
    if (!d || !U_dev || !totals_dev) return bad(ALSV_ERR_INVALID_ARG, "null descriptor, state or output pointer");
    if (d->ndim < 1 || d->ndim > 3) return bad(ALSV_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
    if (d->eq != ALSV_EQ_BURGERS && d->eq != ALSV_EQ_EULER) return bad(ALSV_ERR_INVALID_ARG, "eq must be BURGERS or EULER");
    if (d->precision != ALSV_FP32 && d->precision != ALSV_FP64) return bad(ALSV_ERR_INVALID_ARG, "precision must be FP32 or FP64");
    if (d->n_levels > ALSV_MAX_LEVELS) return bad(ALSV_ERR_INVALID_ARG, "n_levels must be <= 8");
    // a block of a decomposed grid: the same rules as alsv_init_grid
    bool block = false;
    for (int k = 0; k < 3; ++k) {
        if (d->global_n[k] != 0 || d->offset[k] != 0) block = true;
        if (k >= d->ndim && (d->global_n[k] > 1 || d->offset[k] != 0))
            return bad(ALSV_ERR_INVALID_ARG, "global_n / offset of an inactive direction must be 0");
        if (k < d->ndim && d->global_n[k] == 0 && d->offset[k] != 0)
            return bad(ALSV_ERR_INVALID_ARG, "offset needs global_n");
        if (k < d->ndim && d->global_n[k] != 0 &&
            (d->offset[k] < 0 || (long long)d->offset[k] + d->n[k] > d->global_n[k]))
            return bad(ALSV_ERR_INVALID_ARG, "a block must lie inside the whole grid: 0 <= offset and offset + n <= global_n");
    }
    if (block && d->n_levels > 1) return bad(ALSV_ERR_INVALID_ARG, "a decomposed grid needs a single grid (n_levels <= 1)");
    GridArgs g{};
    g.ndim = d->ndim;
    for (int k = 0; k < 3; ++k) g.lo[k] = d->lo[k];
    g.nv = d->eq == ALSV_EQ_BURGERS ? 1 : d->ndim + 2;
    g.nlev = d->n_levels <= 1 ? 1 : d->n_levels;
    long long samples = 0, elems = 0;
    for (int l = 0; l < g.nlev; ++l) {
        LevelInfo& L = g.lev[l];
        const int* n = d->n_levels <= 1 ? d->n : d->level_n[l];
        L.samples = d->n_levels <= 1 ? d->batch : d->level_batch[l];
        if (L.samples < 1) return bad(ALSV_ERR_INVALID_ARG, "batch (samples per level) must be >= 1");
        for (int k = 0; k < 3; ++k) {
            L.n[k] = k < d->ndim ? n[k] : 1;
            if (L.n[k] < 1) return bad(ALSV_ERR_INVALID_ARG, "every active direction needs n >= 1");
            if (k < d->ndim && !(d->hi[k] > d->lo[k])) return bad(ALSV_ERR_INVALID_ARG, "hi must exceed lo");
            // a block of a decomposed grid has the whole grid's dx
            const int ng = k < d->ndim && d->global_n[k] > 0 ? d->global_n[k] : L.n[k];
            L.dx[k] = k < d->ndim ? (d->hi[k] - d->lo[k]) / ng : 1.0;
            L.inv_dx[k] = 1.0 / L.dx[k];
        }
        L.sample0 = (int)samples;
        L.elem0 = elems;
        samples += L.samples;
        elems += (long long)L.samples * g.nv * L.n[0] * L.n[1] * L.n[2];
    }
    if (samples > 65535) return bad(ALSV_ERR_INVALID_ARG, "at most 65535 samples");
    fill_float_consts(g);
    g.total_samples = (int)samples;
    long long maxchunks = 0;
    for (int l = 0; l < g.nlev; ++l) {
        const long long c = ((long long)g.lev[l].n[0] * g.lev[l].n[1] * g.lev[l].n[2] + 4095) / 4096;
        maxchunks = c > maxchunks ? c : maxchunks;
    }
    if (maxchunks > 65535)
        return bad(ALSV_ERR_INVALID_ARG, "a sample of " + std::to_string(maxchunks) +
                                             " chunks of 4096 cells exceeds the reduction's 65535 chunks per sample");
    const long long parts = reduce_partial_count(g);
    if (parts > kNoallocPartials)
        return bad(ALSV_ERR_INVALID_ARG, "samples x variables x ceil(cells/4096) = " + std::to_string(parts) +
                                             " exceeds the static scratch of " + std::to_string(kNoallocPartials) +
                                             " partial sums");
    const size_t need = (size_t)elems * (d->precision == ALSV_FP64 ? 8 : 4);
    if (U_bytes < need) return bad(ALSV_ERR_BUFFER_TOO_SMALL, "state buffer smaller than the descriptor's state");
    // Set-up, with the calling device current: the device address of the scratch array. (In host
    // code the array's name is only a host-side stand-in, not a device address.) It is looked up on
    // every call, which allocates nothing, so a device reset between calls (which reloads the module
    // at another address) cannot leave a stale address behind. The first call on a device loads the
    // module there.
    void* sym = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&sym, g_noalloc_partials);
    if (e != cudaSuccess) return bad(ALSV_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    double* scratch = static_cast<double*>(sym);
    // The reduction writes every partial slot before reading it, so nothing needs clearing.
    e = launch_reduce(d->precision == ALSV_FP64, 0, g, U_dev, scratch, totals_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return bad(ALSV_ERR_CUDA, std::string("reduction launch: ") + cudaGetErrorString(e));
    return ALSV_OK;
}
