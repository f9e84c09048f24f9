// Stage kernels for float, 2D: the lean two-sample schedules (variants 8-13; 9, 11, 12 and 13 keep
// every global read of a phase in flight at once; 12 and 13 take the x-fluxes by warp shuffles and
// evaluate both directions between one pair of barriers).
#include "fv_pair2.cuh"
#include "stage_dispatch.cuh"
namespace alsv {
template <int RECON, int FLUX, int TY, int HALVES, int PREF, int XS>
static cudaError_t launch_pair2_one(const StageArgs& a, cudaStream_t s) {
    auto k = k_stage2d_pair2<RECON, FLUX, TY, HALVES, PREF, XS>;
    constexpr size_t sm = pair2_smem_bytes<RECON, TY, XS>();
    static unsigned long long smem_devices = 0;   // devices on which the opt-in is done
    {
        const cudaError_t e = ensure_dynamic_smem(k, sm, smem_devices);
        if (e != cudaSuccess) return e;
    }
    if (a.g.total_pwork <= 0) return cudaSuccess;
    k<<<(unsigned)a.g.total_pwork, 256, sm, s>>>(a);
    return cudaGetLastError();
}

template <int TY, int HALVES, int PREF = 0, int XS = 0>
static cudaError_t launch_pair2(int recon, int flux, int eq, const StageArgs& a, cudaStream_t s) {
    if (eq != EQ_EULER || a.g.rvars != RV_PRIM) return cudaErrorNotSupported;
    if (flux == FLX_HLLC) {
        if (recon == REC_WENO3) return launch_pair2_one<REC_WENO3, FLX_HLLC, TY, HALVES, PREF, XS>(a, s);
        if (recon == REC_MC) return launch_pair2_one<REC_MC, FLX_HLLC, TY, HALVES, PREF, XS>(a, s);
        return launch_pair2_one<REC_PC, FLX_HLLC, TY, HALVES, PREF, XS>(a, s);
    }
    if (flux == FLX_RUSANOV) {
        if (recon == REC_WENO3) return launch_pair2_one<REC_WENO3, FLX_RUSANOV, TY, HALVES, PREF, XS>(a, s);
        if (recon == REC_MC) return launch_pair2_one<REC_MC, FLX_RUSANOV, TY, HALVES, PREF, XS>(a, s);
        return launch_pair2_one<REC_PC, FLX_RUSANOV, TY, HALVES, PREF, XS>(a, s);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_stage_f32_2d_lean(int variant, int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    switch (variant) {
        case 8: return launch_pair2<16, 0>(recon, flux, eq, a, s);
        case 9: return launch_pair2<16, 0, 1>(recon, flux, eq, a, s);
        case 10: return launch_pair2<16, 1>(recon, flux, eq, a, s);
        case 11: return launch_pair2<16, 1, 1>(recon, flux, eq, a, s);
        case 12: return launch_pair2<16, 0, 1, 1>(recon, flux, eq, a, s);
        case 13: return launch_pair2<16, 1, 1, 1>(recon, flux, eq, a, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace alsv
