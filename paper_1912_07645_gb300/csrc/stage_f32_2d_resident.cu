// The sample-resident cluster kernel (FP32 2D Euler): launch with cluster dimensions.
#include "fv_resident.cuh"

namespace alsv {

template <int RECON, int FLUX>
static cudaError_t launch_resident_one(const ResidentArgs& a, int nx, int R, int samples, cudaStream_t s) {
    auto k = k_resident2d<RECON, FLUX>;
    const size_t sm = resident_smem_bytes(nx, R);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (a.cs > 8) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(samples * a.cs), 1, 1);
    cfg.blockDim = dim3((unsigned)nx, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, k, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;   // no SM group holds one cluster
    return cudaLaunchKernelEx(&cfg, k, a);
}

cudaError_t launch_resident(const ResidentArgs& a, int recon, int flux, int nx, int R, int samples, cudaStream_t s) {
    if (flux == FLX_HLLC) {
        if (recon == REC_WENO3) return launch_resident_one<REC_WENO3, FLX_HLLC>(a, nx, R, samples, s);
        if (recon == REC_MC) return launch_resident_one<REC_MC, FLX_HLLC>(a, nx, R, samples, s);
        return launch_resident_one<REC_PC, FLX_HLLC>(a, nx, R, samples, s);
    }
    if (flux == FLX_RUSANOV) {
        if (recon == REC_WENO3) return launch_resident_one<REC_WENO3, FLX_RUSANOV>(a, nx, R, samples, s);
        if (recon == REC_MC) return launch_resident_one<REC_MC, FLX_RUSANOV>(a, nx, R, samples, s);
        return launch_resident_one<REC_PC, FLX_RUSANOV>(a, nx, R, samples, s);
    }
    return cudaErrorNotSupported;
}

}  // namespace alsv
