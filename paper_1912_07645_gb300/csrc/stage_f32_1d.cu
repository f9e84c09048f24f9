// Stage and speed kernels for float, 1D (explicit tile-shape variants).
#include "stage_dispatch.cuh"
namespace alsv {
cudaError_t launch_stage_f32_1d(int variant, int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    switch (variant) {
        case 0: return launch_stage_tile<float, 1, 256, 1, 1, 256>(eq, recon, flux, a, s);
        case 1: return launch_stage_tile<float, 1, 64, 1, 1, 64>(eq, recon, flux, a, s);
        case 2: return launch_stage_tile<float, 1, 32, 1, 1, 32>(eq, recon, flux, a, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_speed_f32_1d(int variant, int eq, const GridArgs& g, const void* U, double* part, cudaStream_t s) {
    switch (variant) {
        case 0: return launch_speed_tile<float, 1, 256, 1, 1, 256>(eq, g, U, part, s);
        case 1: return launch_speed_tile<float, 1, 64, 1, 1, 64>(eq, g, U, part, s);
        case 2: return launch_speed_tile<float, 1, 32, 1, 1, 32>(eq, g, U, part, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace alsv
