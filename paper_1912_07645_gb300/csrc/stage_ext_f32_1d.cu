// Default-schedule stage kernels for float, 1D: ENO2 and the Roe, Godunov, entropy-conservative fluxes.
#include "stage_ext.cuh"
namespace alsv {
cudaError_t launch_stage_ext_f32_1d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    return launch_stage_ext<float, 1, 256, 1, 1, 256>(eq, recon, flux, a, s);
}
}  // namespace alsv
