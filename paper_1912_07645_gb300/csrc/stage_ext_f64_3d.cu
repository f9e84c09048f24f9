// Default-schedule stage kernels for double, 3D: ENO2 and the Roe, Godunov, entropy-conservative fluxes.
#include "stage_ext.cuh"
namespace alsv {
cudaError_t launch_stage_ext_f64_3d(int eq, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    return launch_stage_ext<double, 3, 8, 8, 8, 256>(eq, recon, flux, a, s);
}
}  // namespace alsv
