// Statistical functionals over the samples of a batch (Sec. 2.2 lists point PDFs, two-point
// structure functions, joint PDFs and multi-point correlators among the on-device statistics).
// Quantities are the primitive variables (rho, u_k, p) (Burgers: u), computed in FP64 from the
// stored state.
//
// Point PDF: histogram counts of one quantity at given cells over the samples; bin 0 takes values
// below lo, bins 1..n_bins the equal-width bins of [lo, hi), bin n_bins + 1 the values >= hi (and
// NaN). Integer counts (exact in any order). Joint PDF: the same bins for two quantities at one
// cell. Multi-point correlator: E[prod_j q(x_j)] over a set of k cells, an FP64 sum over samples
// in ascending order.
//
// Structure function of order p (p = 1 or 2) at radius r, reading of the ball form:
//   S_p(r) = ( E[ sum_x sum_{k in Z^d, 0 < |k| <= r} |q(x + k dx) - q(x)|^p dV^2 ] )^(1/p),
// periodic directions wrap, pairs leaving a non-periodic domain are skipped. The kernel sums each
// sample's shells r - 1 < |k| <= r in FP64 in a fixed order; the expectation is the sample mean.
#include <cstdint>
#include <cstring>

#include "alsv_ctx.h"
#include "fv_physics.cuh"
#include "fv_quantities.cuh"

namespace alsv {
namespace {

constexpr int kSfMaxR2 = 16;   // largest radius (cells) in 1D and 2D
constexpr int kSfMaxR3 = 4;    // in 3D
constexpr int kSfNT = 256;

// ------------------------------------------------------------------------------ point PDF
__device__ __forceinline__ int pdf_bin(double x, double lo, double hi, int n_bins) {
    if (x < lo) return 0;
    if (x < hi) {
        int k = (int)floor((x - lo) / (hi - lo) * (double)n_bins);
        if (k > n_bins - 1) k = n_bins - 1;
        return 1 + k;
    }
    return n_bins + 1;   // >= hi or NaN
}

template <class R>
__global__ void k_point_pdf(const GridArgs g, const void* Uv, int q, const int64_t* cells, int n_points, double lo,
                            double hi, int n_bins, unsigned long long* counts) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_points * L.samples) return;
    const int pt = (int)(t % n_points);
    const int b = (int)(t / n_points);
    const R* U = reinterpret_cast<const R*>(Uv) + (long long)b * g.nv * C;
    const double x = prim_quantity<R>(U, C, cells[pt], q, g.nv, g.nv > 1, g.gamma - 1.0);
    atomicAdd(counts + (long long)pt * (n_bins + 2) + pdf_bin(x, lo, hi, n_bins), 1ull);
}

// ------------------------------------------------------------------------------ joint PDF
template <class R>
__global__ void k_joint_pdf(const GridArgs g, const void* Uv, int q1, int q2, const int64_t* cells, int n_points,
                            double lo1, double hi1, int nb1, double lo2, double hi2, int nb2,
                            unsigned long long* counts) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_points * L.samples) return;
    const int pt = (int)(t % n_points);
    const int b = (int)(t / n_points);
    const R* U = reinterpret_cast<const R*>(Uv) + (long long)b * g.nv * C;
    const double x1 = prim_quantity<R>(U, C, cells[pt], q1, g.nv, g.nv > 1, g.gamma - 1.0);
    const double x2 = prim_quantity<R>(U, C, cells[pt], q2, g.nv, g.nv > 1, g.gamma - 1.0);
    const int k1 = pdf_bin(x1, lo1, hi1, nb1), k2 = pdf_bin(x2, lo2, hi2, nb2);
    atomicAdd(counts + ((long long)pt * (nb1 + 2) + k1) * (nb2 + 2) + k2, 1ull);
}

// ------------------------------------------------------------------------------ correlators
// acc[0] += samples; acc[1 + s] += sum over samples (ascending) of prod_j q(cells[s][j]) (FP64)
template <class R>
__global__ void k_correlator(const GridArgs g, const void* Uv, int q, const int64_t* cells, int n_sets, int k,
                             double* acc) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0 && threadIdx.x == 0 && blockIdx.x == 0) acc[0] = acc[0] + (double)L.samples;
    if (s >= n_sets) return;
    double sum = 0.0;
    for (int b = 0; b < L.samples; ++b) {
        const R* U = reinterpret_cast<const R*>(Uv) + (long long)b * g.nv * C;
        double prod = 1.0;
        for (int j = 0; j < k; ++j)
            prod = prod * prim_quantity<R>(U, C, cells[(long long)s * k + j], q, g.nv, g.nv > 1, g.gamma - 1.0);
        sum = sum + prod;
    }
    acc[1 + s] = acc[1 + s] + sum;
}

// ------------------------------------------------------------------------------ structure functions
__device__ __forceinline__ int isqrt_floor(int a) {
    int s = (int)sqrt((double)a);
    while (s * s > a) --s;
    while ((s + 1) * (s + 1) <= a) ++s;
    return s;
}

// One CTA per (sample, split): tiles split0..split1 of the sample. Each thread owns one cell of
// the tile; per radius shell it sums |dq|^p over the shell's offsets, warps reduce with shuffles,
// and each warp adds its sums to its own slot in tile order. part[(sample * splits + split) * R + r-1].
template <int ND, int TX, int TY, int TZ>
__global__ void __launch_bounds__(kSfNT) k_sf_partial(const GridArgs g, const void* Uv, int fp64, int q, int p, int Rr,
                                                      int splits, double* part) {
    extern __shared__ double sm[];
    constexpr int NW = kSfNT / 32;
    const LevelInfo& L = g.lev[0];
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const long long C = (long long)nx * ny * nz;
    const int b = blockIdx.x / splits, sp = blockIdx.x % splits;
    const int ntx = (nx + TX - 1) / TX, nty = ND >= 2 ? (ny + TY - 1) / TY : 1, ntz = ND >= 3 ? (nz + TZ - 1) / TZ : 1;
    const int tiles = ntx * nty * ntz;
    const int t0 = (int)((long long)tiles * sp / splits), t1 = (int)((long long)tiles * (sp + 1) / splits);
    const int HX = TX + 2 * Rr, HY = ND >= 2 ? TY + 2 * Rr : 1, HZ = ND >= 3 ? TZ + 2 * Rr : 1;
    double* sq = sm;                      // [HZ][HY][HX]
    double* wsum = sm + HX * HY * HZ;     // [R][NW]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < Rr * NW; i += kSfNT) wsum[i] = 0.0;
    const bool per[3] = {g.bc[0][0] == BC_PERIODIC, g.bc[1][0] == BC_PERIODIC, g.bc[2][0] == BC_PERIODIC};
    const int gx = Rr, gy = ND >= 2 ? Rr : 0, gz = ND >= 3 ? Rr : 0;
    const double gm1 = g.gamma - 1.0;
    const int euler = g.nv > 1;
    double dV = 1.0;
    for (int k = 0; k < ND; ++k) dV *= L.dx[k];
    const double w2 = dV * dV;
    for (int tile = t0; tile < t1; ++tile) {
        const int tx0 = (tile % ntx) * TX;
        const int ty0 = ND >= 2 ? ((tile / ntx) % nty) * TY : 0;
        const int tz0 = ND >= 3 ? (tile / (ntx * nty)) * TZ : 0;
        __syncthreads();   // previous tile's reads done
        for (int h = tid; h < HX * HY * HZ; h += kSfNT) {
            const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
            int x = tx0 - gx + hx, y = ty0 - gy + hy, z = tz0 - gz + hz;
            bool in = true;
            if (per[0]) x = ((x % nx) + nx) % nx; else in = in && x >= 0 && x < nx;
            if (ND >= 2) { if (per[1]) y = ((y % ny) + ny) % ny; else in = in && y >= 0 && y < ny; }
            if (ND >= 3) { if (per[2]) z = ((z % nz) + nz) % nz; else in = in && z >= 0 && z < nz; }
            double v = 0.0;
            if (in) {
                const long long i = ((long long)z * ny + y) * nx + x;
                v = fp64 ? prim_quantity<double>(reinterpret_cast<const double*>(Uv) + (long long)b * g.nv * C, C, i, q,
                                            g.nv, euler, gm1)
                         : prim_quantity<float>(reinterpret_cast<const float*>(Uv) + (long long)b * g.nv * C, C, i, q,
                                           g.nv, euler, gm1);
            }
            sq[h] = v;
        }
        __syncthreads();
        const int cx = tid % TX, cy = ND >= 2 ? (tid / TX) % TY : 0, cz = ND >= 3 ? tid / (TX * TY) : 0;
        const int X = tx0 + cx, Y = ty0 + cy, Z = tz0 + cz;
        const bool own = X < nx && Y < ny && Z < nz;
        const int hc = ((cz + gz) * HY + (cy + gy)) * HX + (cx + gx);
        const double q0 = sq[hc];
        for (int r = 1; r <= Rr; ++r) {
            double s = 0.0;
            const int r2 = r * r, rm2 = (r - 1) * (r - 1);
            const int zr = ND >= 3 ? r : 0, yr = ND >= 2 ? r : 0;
            for (int dz = -zr; dz <= zr; ++dz) {
                for (int dy = -yr; dy <= yr; ++dy) {
                    const int a = r2 - dz * dz - dy * dy;
                    if (a < 0) continue;
                    const int bb = rm2 - dz * dz - dy * dy;
                    const int hi = isqrt_floor(a);
                    const int lo = bb < 0 ? 0 : isqrt_floor(bb) + 1;
                    if (lo > hi) continue;
                    const bool yz_in = (ND < 2 || per[1] || (Y + dy >= 0 && Y + dy < ny)) &&
                                       (ND < 3 || per[2] || (Z + dz >= 0 && Z + dz < nz));
                    if (!yz_in) continue;
                    const int row = ((cz + gz + dz) * HY + (cy + gy + dy)) * HX + cx + gx;
                    for (int sgn = -1; sgn <= 1; sgn += 2) {
                        if (sgn == 1 && lo == 0) break;     // [-hi, hi] done in one sweep
                        const int d0 = lo == 0 ? -hi : (sgn < 0 ? -hi : lo);
                        const int d1 = lo == 0 ? hi : (sgn < 0 ? -lo : hi);
                        for (int dx = d0; dx <= d1; ++dx) {
                            if (!per[0] && (X + dx < 0 || X + dx >= nx)) continue;
                            const double d = sq[row + dx] - q0;
                            s = s + (p == 1 ? fabs(d) : d * d);
                        }
                    }
                }
            }
            if (!own) s = 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = s + __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) wsum[(r - 1) * NW + warp] = wsum[(r - 1) * NW + warp] + s;
        }
    }
    __syncthreads();
    for (int r = tid; r < Rr; r += kSfNT) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s = s + wsum[r * NW + w];
        part[((long long)b * splits + sp) * Rr + r] = s * w2;
    }
}

// acc[0] += samples; acc[r] += sum over samples (ascending) of the sample's shell-r sum (splits in order)
__global__ void k_sf_reduce(const double* part, int samples, int splits, int Rr, double* acc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > Rr) return;
    if (r == 0) {
        acc[0] = acc[0] + (double)samples;
        return;
    }
    double s = 0.0;
    for (int b = 0; b < samples; ++b) {
        double sb = 0.0;
        for (int k = 0; k < splits; ++k) sb = sb + part[((long long)b * splits + k) * Rr + (r - 1)];
        s = s + sb;
    }
    acc[r] = acc[r] + s;
}

// S_p(r) = (sum_{r' <= r} acc[r'] / acc[0])^(1/p)
__global__ void k_sf_read(const double* acc, int p, int Rr, double* S) {
    if (threadIdx.x != 0) return;
    double cum = 0.0;
    for (int r = 1; r <= Rr; ++r) {
        cum = cum + acc[r];
        const double m = acc[0] > 0.0 ? cum / acc[0] : 0.0;
        S[r - 1] = p == 1 ? m : sqrt(m);
    }
}

int sf_splits(const alsv_ctx* c) {
    const LevelInfo& L = c->g.lev[0];
    const int S = L.samples;
    const long long want = 4LL * 152;   // CTAs to fill the GPU
    long long sp = (want + S - 1) / S;
    const long long tiles_max = ((long long)L.n[0] * L.n[1] * L.n[2] + 255) / 256;
    if (sp > tiles_max) sp = tiles_max;
    return (int)(sp < 1 ? 1 : sp);
}

alsv_status sf_check(alsv_ctx* c, int q, int p, int Rr) {
    if (c->g.nlev != 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "structure functions need a single-level context");
    if (ctx_has_halo(c))
        return ctx_fail(c, ALSV_ERR_INVALID_ARG, "structure functions need the whole grid (pairs cross halo faces)");
    if (q < 0 || q >= c->nv) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "quantity index out of range");
    if (p != 1 && p != 2) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "order p must be 1 or 2");
    const int rmax = c->ndim == 3 ? kSfMaxR3 : kSfMaxR2;
    if (Rr < 1 || Rr > rmax) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "radius out of range (1..16 in 1D/2D, 1..4 in 3D)");
    for (int k = 0; k < c->ndim; ++k)
        if (c->g.bc[k][0] == BC_PERIODIC && c->g.lev[0].n[k] < 2 * Rr + 1)
            return ctx_fail(c, ALSV_ERR_INVALID_ARG, "a periodic direction needs at least 2 R + 1 cells");
    return ALSV_OK;
}

size_t sf_part_bytes(const alsv_ctx* c, int Rr) {
    return (((size_t)c->g.lev[0].samples * sf_splits(c) * Rr * 8) + 255) / 256 * 256;
}

}  // namespace
}  // namespace alsv

using namespace alsv;

extern "C" {

alsv_status alsv_point_pdf_accumulate(alsv_ctx* c, int quantity_index, const int64_t* cells_dev, int n_points,
                                      double lo, double hi, int n_bins, int64_t* counts_dev) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (!c->U) return ctx_fail(c, ALSV_ERR_NOT_READY, "no state bound (alsv_set_initial_data)");
    if (c->g.nlev != 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "point PDFs need a single-level context");
    if (quantity_index < 0 || quantity_index >= c->nv) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "quantity index out of range");
    if (!cells_dev || !counts_dev || n_points < 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null cells/counts or no points");
    if (n_bins < 1 || !(hi > lo)) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "need n_bins >= 1 and hi > lo");
    const long long n = (long long)n_points * c->g.lev[0].samples;
    const unsigned grid = (unsigned)((n + 255) / 256);
    auto* cnt = reinterpret_cast<unsigned long long*>(counts_dev);
    if (c->fp64) k_point_pdf<double><<<grid, 256, 0, c->stream>>>(c->g, c->U, quantity_index, cells_dev, n_points, lo, hi, n_bins, cnt);
    else k_point_pdf<float><<<grid, 256, 0, c->stream>>>(c->g, c->U, quantity_index, cells_dev, n_points, lo, hi, n_bins, cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "point PDF kernel");
    c->launches++;
    return ALSV_OK;
}

alsv_status alsv_joint_pdf_accumulate(alsv_ctx* c, int q1, int q2, const int64_t* cells_dev, int n_points, double lo1,
                                      double hi1, int n_bins1, double lo2, double hi2, int n_bins2, int64_t* counts_dev) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (!c->U) return ctx_fail(c, ALSV_ERR_NOT_READY, "no state bound (alsv_set_initial_data)");
    if (c->g.nlev != 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "joint PDFs need a single-level context");
    if (q1 < 0 || q1 >= c->nv || q2 < 0 || q2 >= c->nv) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "quantity index out of range");
    if (!cells_dev || !counts_dev || n_points < 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null cells/counts or no points");
    if (n_bins1 < 1 || n_bins2 < 1 || !(hi1 > lo1) || !(hi2 > lo2))
        return ctx_fail(c, ALSV_ERR_INVALID_ARG, "need n_bins >= 1 and hi > lo for both quantities");
    const long long n = (long long)n_points * c->g.lev[0].samples;
    const unsigned grid = (unsigned)((n + 255) / 256);
    auto* cnt = reinterpret_cast<unsigned long long*>(counts_dev);
    if (c->fp64)
        k_joint_pdf<double><<<grid, 256, 0, c->stream>>>(c->g, c->U, q1, q2, cells_dev, n_points, lo1, hi1, n_bins1, lo2, hi2,
                                                        n_bins2, cnt);
    else
        k_joint_pdf<float><<<grid, 256, 0, c->stream>>>(c->g, c->U, q1, q2, cells_dev, n_points, lo1, hi1, n_bins1, lo2, hi2,
                                                       n_bins2, cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "joint PDF kernel");
    c->launches++;
    return ALSV_OK;
}

alsv_status alsv_correlator_accumulate(alsv_ctx* c, int quantity_index, const int64_t* cells_dev, int n_sets, int k,
                                       double* acc_dev) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (!c->U) return ctx_fail(c, ALSV_ERR_NOT_READY, "no state bound (alsv_set_initial_data)");
    if (c->g.nlev != 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "correlators need a single-level context");
    if (quantity_index < 0 || quantity_index >= c->nv) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "quantity index out of range");
    if (!cells_dev || !acc_dev || n_sets < 1 || k < 1 || k > 8)
        return ctx_fail(c, ALSV_ERR_INVALID_ARG, "need cells, an accumulator, n_sets >= 1 and 1 <= k <= 8");
    const unsigned grid = (unsigned)((n_sets + 127) / 128);
    if (c->fp64) k_correlator<double><<<grid, 128, 0, c->stream>>>(c->g, c->U, quantity_index, cells_dev, n_sets, k, acc_dev);
    else k_correlator<float><<<grid, 128, 0, c->stream>>>(c->g, c->U, quantity_index, cells_dev, n_sets, k, acc_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "correlator kernel");
    c->launches++;
    return ALSV_OK;
}

size_t alsv_structure_function_bytes(const alsv_ctx* c, int radius) {
    if (!c || radius < 1) return 0;
    return 256 + sf_part_bytes(c, radius);
}

alsv_status alsv_structure_function_accumulate(alsv_ctx* c, int quantity_index, int p, int radius, void* acc_dev,
                                               size_t bytes) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (!c->U) return ctx_fail(c, ALSV_ERR_NOT_READY, "no state bound (alsv_set_initial_data)");
    alsv_status st = sf_check(c, quantity_index, p, radius);
    if (st != ALSV_OK) return st;
    if (!acc_dev || ((uintptr_t)acc_dev & 255) != 0)
        return ctx_fail(c, ALSV_ERR_INVALID_ARG, "accumulator must be non-null and 256-byte aligned");
    if (bytes < alsv_structure_function_bytes(c, radius))
        return ctx_fail(c, ALSV_ERR_BUFFER_TOO_SMALL, "accumulator smaller than alsv_structure_function_bytes");
    double* acc = reinterpret_cast<double*>(acc_dev);
    double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(acc_dev) + 256);
    const int splits = sf_splits(c);
    const int S = c->g.lev[0].samples;
    const int Rr = radius;
    const unsigned grid = (unsigned)(S * splits);
    cudaError_t e;
    if (c->ndim == 1) {
        const size_t sm = ((256 + 2 * Rr) + Rr * (kSfNT / 32)) * 8;
        k_sf_partial<1, 256, 1, 1><<<grid, kSfNT, sm, c->stream>>>(c->g, c->U, c->fp64, quantity_index, p, Rr, splits, part);
    } else if (c->ndim == 2) {
        const size_t sm = ((32 + 2 * Rr) * (8 + 2 * Rr) + Rr * (kSfNT / 32)) * 8;
        k_sf_partial<2, 32, 8, 1><<<grid, kSfNT, sm, c->stream>>>(c->g, c->U, c->fp64, quantity_index, p, Rr, splits, part);
    } else {
        const size_t sm = ((8 + 2 * Rr) * (8 + 2 * Rr) * (4 + 2 * Rr) + Rr * (kSfNT / 32)) * 8;
        k_sf_partial<3, 8, 8, 4><<<grid, kSfNT, sm, c->stream>>>(c->g, c->U, c->fp64, quantity_index, p, Rr, splits, part);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda_fail(c, e, "structure function kernel");
    k_sf_reduce<<<1, 64, 0, c->stream>>>(part, S, splits, Rr, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda_fail(c, e, "structure function reduction");
    c->launches += 2;
    return ALSV_OK;
}

alsv_status alsv_structure_function_read(alsv_ctx* c, const void* acc_dev, int p, int radius, double* S_dev) {
    if (!c) return ALSV_ERR_INVALID_ARG;
    if (!acc_dev || !S_dev) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "null accumulator or output");
    if (p != 1 && p != 2) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "order p must be 1 or 2");
    if (radius < 1) return ctx_fail(c, ALSV_ERR_INVALID_ARG, "radius must be >= 1");
    k_sf_read<<<1, 32, 0, c->stream>>>(reinterpret_cast<const double*>(acc_dev), p, radius, S_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "structure function read kernel");
    c->launches++;
    return ALSV_OK;
}

}  // extern "C"
