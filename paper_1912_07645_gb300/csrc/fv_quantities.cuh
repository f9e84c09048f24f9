// Primitive quantities of one cell in FP64, read from the stored conserved state (float or
// double): (rho, u_k, p) for Euler with u_k = m_k / rho and p = (gamma - 1) (E - |m|^2 / (2 rho)),
// u itself for Burgers. Shared by the statistics (Welford, MLMC) and the functionals, which all
// evaluate them with the same operations (translation units built without FMA contraction).
#pragma once

namespace alsv {

// all quantities of cell i; U points at the sample's first variable, C = cells per variable
template <class R, int NV, int EULER>
__device__ __forceinline__ void prim_quantities(const R* U, long long C, long long i, double gm1, double* x) {
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = (double)U[v * C + i];
    if (EULER) {
        double mm = u[1] * u[1];
#pragma unroll
        for (int k = 2; k < NV - 1; ++k) mm = mm + u[k] * u[k];
        x[0] = u[0];
#pragma unroll
        for (int k = 1; k < NV - 1; ++k) x[k] = u[k] / u[0];
        x[NV - 1] = gm1 * (u[NV - 1] - 0.5 * mm / u[0]);
    } else {
        x[0] = u[0];
    }
}

// quantity q of cell i (nv variables; euler = 0 for Burgers), the same operations as above
template <class R>
__device__ __forceinline__ double prim_quantity(const R* U, long long C, long long i, int q, int nv, int euler,
                                                double gm1) {
    if (!euler) return (double)U[i];
    const double rho = (double)U[i];
    if (q == 0) return rho;
    if (q < nv - 1) return (double)U[q * C + i] / rho;
    const double m1 = (double)U[C + i];
    double mm = m1 * m1;
    for (int k = 2; k < nv - 1; ++k) {
        const double m = (double)U[k * C + i];
        mm = mm + m * m;
    }
    return gm1 * ((double)U[(nv - 1) * C + i] - 0.5 * mm / rho);
}

}  // namespace alsv
