// Dispatch of the schemes served by the default tile schedule only: ENO2 reconstruction and the
// Roe, Godunov and entropy-conservative fluxes (Sec. 2.1). Euler reconstructs primitive variables
// for them; the entropy-conservative fluxes take cell values (reconstruction ignored, the ghost
// width is the flux's own). Burgers is instantiated in 1D only.
#pragma once

#include "stage_dispatch.cuh"

namespace alsv {

template <class R, int EQ, int ND, int RECON, int FLUX, int TX, int TY, int TZ, int NT>
static cudaError_t launch_ext_one(const StageArgs& a, cudaStream_t s) {
    auto k = k_stage<R, EQ, ND, RECON, FLUX, TX, TY, TZ, NT, RV_PRIM>;
    constexpr size_t sm = stage_smem_bytes<R, EQ, ND, RECON, TX, TY, TZ, FLUX>();
    static unsigned long long smem_devices = 0;
    {
        const cudaError_t e = ensure_dynamic_smem(k, sm, smem_devices);
        if (e != cudaSuccess) return e;
    }
    if (a.g.total_work <= 0) return cudaSuccess;
    k<<<(unsigned)a.g.total_work, NT, sm, s>>>(a);
    return cudaGetLastError();
}

template <class R, int EQ, int ND, int FLUX, int TX, int TY, int TZ, int NT>
static cudaError_t launch_ext_recon(int recon, const StageArgs& a, cudaStream_t s) {
    switch (recon) {
        case REC_PC: return launch_ext_one<R, EQ, ND, REC_PC, FLUX, TX, TY, TZ, NT>(a, s);
        case REC_MC: return launch_ext_one<R, EQ, ND, REC_MC, FLUX, TX, TY, TZ, NT>(a, s);
        case REC_WENO3: return launch_ext_one<R, EQ, ND, REC_WENO3, FLUX, TX, TY, TZ, NT>(a, s);
        default: return launch_ext_one<R, EQ, ND, REC_ENO2, FLUX, TX, TY, TZ, NT>(a, s);
    }
}

template <class R, int EQ, int ND, int TX, int TY, int TZ, int NT>
static cudaError_t launch_ext_eq(int recon, int flux, const StageArgs& a, cudaStream_t s) {
    switch (flux) {
        case FLX_ROE: return launch_ext_recon<R, EQ, ND, FLX_ROE, TX, TY, TZ, NT>(recon, a, s);
        case FLX_GODUNOV: return launch_ext_recon<R, EQ, ND, FLX_GODUNOV, TX, TY, TZ, NT>(recon, a, s);
        case FLX_EC: return launch_ext_one<R, EQ, ND, REC_PC, FLX_EC, TX, TY, TZ, NT>(a, s);
        case FLX_EC4: return launch_ext_one<R, EQ, ND, REC_PC, FLX_EC4, TX, TY, TZ, NT>(a, s);
        case FLX_TECNO2: return launch_ext_one<R, EQ, ND, REC_PC, FLX_TECNO2, TX, TY, TZ, NT>(a, s);
        case FLX_RUSANOV: return launch_ext_one<R, EQ, ND, REC_ENO2, FLX_RUSANOV, TX, TY, TZ, NT>(a, s);
        case FLX_HLL: return launch_ext_one<R, EQ, ND, REC_ENO2, FLX_HLL, TX, TY, TZ, NT>(a, s);
        default:   // HLLC with ENO2 (Burgers: HLLC is HLL)
            if constexpr (EQ == EQ_BURGERS) return launch_ext_one<R, EQ, ND, REC_ENO2, FLX_HLL, TX, TY, TZ, NT>(a, s);
            else return launch_ext_one<R, EQ, ND, REC_ENO2, FLX_HLLC, TX, TY, TZ, NT>(a, s);
    }
}

template <class R, int ND, int TX, int TY, int TZ, int NT>
static cudaError_t launch_stage_ext(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    if (eq == EQ_BURGERS) {
        if constexpr (ND == 1) return launch_ext_eq<R, EQ_BURGERS, ND, TX, TY, TZ, NT>(recon, flux, a, s);
        else return cudaErrorNotSupported;
    }
    return launch_ext_eq<R, EQ_EULER, ND, TX, TY, TZ, NT>(recon, flux, a, s);
}

}  // namespace alsv
