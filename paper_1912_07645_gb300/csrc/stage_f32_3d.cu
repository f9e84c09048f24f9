// Stage and speed kernels for float, 3D (explicit tile-shape variants).
#include "stage_dispatch.cuh"
#include "fv_zmarch.cuh"
namespace alsv {
cudaError_t launch_stage_f32_3d_lean(int variant, int recon, int flux, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_f32_3d(int variant, int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    switch (variant) {
        case 0: return launch_stage_tile<float, 3, 16, 8, 8, 256>(eq, recon, flux, a, s);
        case 1: return launch_stage_tile<float, 3, 8, 8, 8, 256>(eq, recon, flux, a, s);
        case 2: return eq == EQ_EULER ? launch_stage_zm<32, 8, 64>(recon, flux, a, s) : cudaErrorInvalidValue;
        case 3: return eq == EQ_EULER ? launch_stage_zm<32, 8, 128>(recon, flux, a, s) : cudaErrorInvalidValue;
        case 4: return eq == EQ_EULER ? launch_stage_zm_packed<32, 8, 64>(recon, flux, a, s) : cudaErrorInvalidValue;
        case 5: return eq == EQ_EULER ? launch_stage_zm_packed<32, 7, 64, 256>(recon, flux, a, s) : cudaErrorInvalidValue;
        case 6: case 7: return eq == EQ_EULER ? launch_stage_f32_3d_lean(variant, recon, flux, a, s) : cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_speed_f32_3d(int variant, int eq, const GridArgs& g, const void* U, double* part, cudaStream_t s) {
    switch (variant) {
        case 0: return launch_speed_tile<float, 3, 16, 8, 8, 256>(eq, g, U, part, s);
        case 1: return launch_speed_tile<float, 3, 8, 8, 8, 256>(eq, g, U, part, s);
        case 2: return launch_speed_tile<float, 3, 32, 8, 64, 256>(eq, g, U, part, s);
        case 3: return launch_speed_tile<float, 3, 32, 8, 128, 256>(eq, g, U, part, s);
        case 4: return launch_speed_tile<float, 3, 32, 8, 64, 256>(eq, g, U, part, s);
        case 5: case 7: return launch_speed_tile<float, 3, 32, 7, 64, 256>(eq, g, U, part, s);
        case 6: return launch_speed_tile<float, 3, 32, 8, 64, 256>(eq, g, U, part, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace alsv
