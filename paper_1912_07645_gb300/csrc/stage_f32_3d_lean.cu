// Stage kernels for float, 3D: the lean packed z-march (variants 6 and 7: 32 x 8 columns on 256
// threads, 32 x 7 columns on 256 threads), in a translation unit of their own.
#include "fv_zmarch.cuh"
namespace alsv {
cudaError_t launch_stage_f32_3d_lean(int variant, int recon, int flux, const StageArgs& a, cudaStream_t s) {
    switch (variant) {
        case 6: return launch_stage_zm_packed<32, 8, 64, 256, 2>(recon, flux, a, s);
        case 7: return launch_stage_zm_packed<32, 7, 64, 256, 2>(recon, flux, a, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace alsv
