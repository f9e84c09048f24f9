// Stage and speed kernels for float, 2D (explicit tile-shape variants).
#include "fv_colmarch.cuh"
#include "fv_pair.cuh"
#include "stage_dispatch.cuh"
namespace alsv {
template <int RECON, int FLUX, int TX, int TY, int NT, int HALVES>
static cudaError_t launch_pair_one(const StageArgs& a, cudaStream_t s) {
    auto k = k_stage2d_pair<RECON, FLUX, TX, TY, NT, HALVES>;
    constexpr size_t sm = pair_smem_bytes<RECON, TX, TY>();
    static unsigned long long smem_devices = 0;   // devices on which the opt-in is done
    {
        const cudaError_t e = ensure_dynamic_smem(k, sm, smem_devices);
        if (e != cudaSuccess) return e;
    }
    if (a.g.total_pwork <= 0) return cudaSuccess;
    k<<<(unsigned)a.g.total_pwork, NT, sm, s>>>(a);
    return cudaGetLastError();
}

// two-sample schedule (FP32 2D Euler, primitive reconstruction, HLLC or Rusanov); HALVES pairs the
// two halves of one y-periodic sample instead of two samples
template <int TX, int TY, int NT, int HALVES = 0>
static cudaError_t launch_pair(int recon, int flux, int eq, const StageArgs& a, cudaStream_t s) {
    if (eq != EQ_EULER || a.g.rvars != RV_PRIM) return cudaErrorNotSupported;
    if (flux == FLX_HLLC) {
        if (recon == REC_WENO3) return launch_pair_one<REC_WENO3, FLX_HLLC, TX, TY, NT, HALVES>(a, s);
        if (recon == REC_MC) return launch_pair_one<REC_MC, FLX_HLLC, TX, TY, NT, HALVES>(a, s);
        return launch_pair_one<REC_PC, FLX_HLLC, TX, TY, NT, HALVES>(a, s);
    }
    if (flux == FLX_RUSANOV) {
        if (recon == REC_WENO3) return launch_pair_one<REC_WENO3, FLX_RUSANOV, TX, TY, NT, HALVES>(a, s);
        if (recon == REC_MC) return launch_pair_one<REC_MC, FLX_RUSANOV, TX, TY, NT, HALVES>(a, s);
        return launch_pair_one<REC_PC, FLX_RUSANOV, TX, TY, NT, HALVES>(a, s);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_stage_f32_2d_lean(int variant, int eq, int recon, int flux, const StageArgs& a, cudaStream_t s);

cudaError_t launch_stage_f32_2d(int variant, int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    if (variant >= 8) return launch_stage_f32_2d_lean(variant, eq, recon, flux, a, s);
    switch (variant) {
        case 0: return launch_stage_tile<float, 2, 32, 16, 1, 256>(eq, recon, flux, a, s);
        case 1: return launch_stage_tile<float, 2, 32, 8, 1, 256>(eq, recon, flux, a, s);
        case 2: return launch_stage_tile<float, 2, 32, 32, 1, 256>(eq, recon, flux, a, s);
        case 3: {
            // column-marching variant (FP32 2D Euler, periodic, primitive; WENO3/MC x HLLC/Rusanov)
            if (eq != EQ_EULER || a.g.rvars != RV_PRIM) return cudaErrorNotSupported;
            if (a.g.total_work <= 0) return cudaSuccess;
            const unsigned blocks = (unsigned)((a.g.total_work + kColWarps - 1) / kColWarps);
            if (recon == REC_WENO3 && flux == FLX_HLLC) k_stage2d_col<REC_WENO3, FLX_HLLC><<<blocks, 32 * kColWarps, 0, s>>>(a);
            else if (recon == REC_WENO3 && flux == FLX_RUSANOV) k_stage2d_col<REC_WENO3, FLX_RUSANOV><<<blocks, 32 * kColWarps, 0, s>>>(a);
            else if (recon == REC_MC && flux == FLX_HLLC) k_stage2d_col<REC_MC, FLX_HLLC><<<blocks, 32 * kColWarps, 0, s>>>(a);
            else if (recon == REC_MC && flux == FLX_RUSANOV) k_stage2d_col<REC_MC, FLX_RUSANOV><<<blocks, 32 * kColWarps, 0, s>>>(a);
            else return cudaErrorNotSupported;
            return cudaGetLastError();
        }
        case 4: return launch_pair<32, 16, 256>(recon, flux, eq, a, s);
        case 5: return launch_pair<32, 8, 256>(recon, flux, eq, a, s);
        case 6: return launch_pair<32, 16, 256, 1>(recon, flux, eq, a, s);
        case 7: return launch_pair<32, 8, 256, 1>(recon, flux, eq, a, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_speed_f32_2d(int variant, int eq, const GridArgs& g, const void* U, double* part, cudaStream_t s) {
    switch (variant) {
        case 0: return launch_speed_tile<float, 2, 32, 16, 1, 256>(eq, g, U, part, s);
        case 1: return launch_speed_tile<float, 2, 32, 8, 1, 256>(eq, g, U, part, s);
        case 2: return launch_speed_tile<float, 2, 32, 32, 1, 256>(eq, g, U, part, s);
        case 3: {
            if (eq != EQ_EULER) return cudaErrorNotSupported;
            if (g.total_work <= 0) return cudaSuccess;
            k_speed2d_col<<<(unsigned)((g.total_work + kColWarps - 1) / kColWarps), 32 * kColWarps, 0, s>>>(g, U, part);
            return cudaGetLastError();
        }
        case 4: return launch_speed_tile<float, 2, 32, 16, 1, 256>(eq, g, U, part, s);
        case 5: return launch_speed_tile<float, 2, 32, 8, 1, 256>(eq, g, U, part, s);
        case 6: return launch_speed_tile<float, 2, 32, 16, 1, 256>(eq, g, U, part, s);
        case 7: return launch_speed_tile<float, 2, 32, 8, 1, 256>(eq, g, U, part, s);
        case 8: case 9: case 10: case 11: case 12: case 13: return launch_speed_tile<float, 2, 32, 16, 1, 256>(eq, g, U, part, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace alsv
