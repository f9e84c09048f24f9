// Runtime (eq, recon, flux) -> template instantiation of the fused stage kernel for one tile shape.
#pragma once

#include "fv_stage.cuh"

namespace alsv {

template <class R, int EQ, int ND, int RECON, int FLUX, int TX, int TY, int TZ, int NT, int RV>
static cudaError_t launch_stage_rv(const StageArgs& a, cudaStream_t s) {
    auto k = k_stage<R, EQ, ND, RECON, FLUX, TX, TY, TZ, NT, RV>;
    constexpr size_t sm = stage_smem_bytes<R, EQ, ND, RECON, TX, TY, TZ>();
    static unsigned long long smem_devices = 0;   // devices on which the opt-in is done
    {
        const cudaError_t e = ensure_dynamic_smem(k, sm, smem_devices);
        if (e != cudaSuccess) return e;
    }
    if (a.g.total_work <= 0) return cudaSuccess;
    k<<<(unsigned)a.g.total_work, NT, sm, s>>>(a);
    return cudaGetLastError();
}

// reconstruction variables: Euler primitive or conserved; a scalar law has only its own variable
template <class R, int EQ, int ND, int RECON, int FLUX, int TX, int TY, int TZ, int NT>
static cudaError_t launch_stage_one(const StageArgs& a, cudaStream_t s) {
    if (EQ == EQ_EULER && a.g.rvars == RV_CONS) return launch_stage_rv<R, EQ, ND, RECON, FLUX, TX, TY, TZ, NT, RV_CONS>(a, s);
    return launch_stage_rv<R, EQ, ND, RECON, FLUX, TX, TY, TZ, NT, RV_PRIM>(a, s);
}

template <class R, int EQ, int ND, int RECON, int TX, int TY, int TZ, int NT>
static cudaError_t launch_stage_flux(int flux, const StageArgs& a, cudaStream_t s) {
    if (EQ == EQ_BURGERS) {
        // for a scalar law HLLC coincides with HLL
        if (flux == FLX_RUSANOV) return launch_stage_one<R, EQ, ND, RECON, FLX_RUSANOV, TX, TY, TZ, NT>(a, s);
        return launch_stage_one<R, EQ, ND, RECON, FLX_HLL, TX, TY, TZ, NT>(a, s);
    }
    switch (flux) {
        case FLX_RUSANOV: return launch_stage_one<R, EQ, ND, RECON, FLX_RUSANOV, TX, TY, TZ, NT>(a, s);
        case FLX_HLL: return launch_stage_one<R, EQ, ND, RECON, FLX_HLL, TX, TY, TZ, NT>(a, s);
        default: return launch_stage_one<R, EQ, ND, RECON, FLX_HLLC, TX, TY, TZ, NT>(a, s);
    }
}

template <class R, int EQ, int ND, int TX, int TY, int TZ, int NT>
static cudaError_t launch_stage_recon(int recon, int flux, const StageArgs& a, cudaStream_t s) {
    switch (recon) {
        case REC_PC: return launch_stage_flux<R, EQ, ND, REC_PC, TX, TY, TZ, NT>(flux, a, s);
        case REC_MC: return launch_stage_flux<R, EQ, ND, REC_MC, TX, TY, TZ, NT>(flux, a, s);
        default: return launch_stage_flux<R, EQ, ND, REC_WENO3, TX, TY, TZ, NT>(flux, a, s);
    }
}

template <class R, int ND, int TX, int TY, int TZ, int NT>
static cudaError_t launch_stage_tile(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    if (eq == EQ_BURGERS) return launch_stage_recon<R, EQ_BURGERS, ND, TX, TY, TZ, NT>(recon, flux, a, s);
    return launch_stage_recon<R, EQ_EULER, ND, TX, TY, TZ, NT>(recon, flux, a, s);
}

template <class R, int ND, int TX, int TY, int TZ, int NT>
static cudaError_t launch_speed_tile(int eq, const GridArgs& g, const void* U, double* part, cudaStream_t s) {
    if (g.total_work <= 0) return cudaSuccess;
    if (eq == EQ_BURGERS)
        k_speed<R, EQ_BURGERS, ND, TX, TY, TZ, NT><<<(unsigned)g.total_work, NT, 0, s>>>(g, U, part);
    else
        k_speed<R, EQ_EULER, ND, TX, TY, TZ, NT><<<(unsigned)g.total_work, NT, 0, s>>>(g, U, part);
    return cudaGetLastError();
}

}  // namespace alsv
