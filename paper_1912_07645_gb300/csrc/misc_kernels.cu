// Per-sample time control (CFL step), initial data, counter-based parameters, Monte Carlo
// statistics (Sec. 2.2) and fixed-order FP64 reductions.
#include <algorithm>

#include "fv_physics.cuh"
#include "fv_quantities.cuh"

namespace alsv {

// ---------------------------------------------------------------------------------------------
// Time control per sample. Adaptive mode (reading; the paper gives no CFL rule): s_b = max over
// tiles of the per-tile partials (the largest (|u_k| + c) / dx_k), dt_b = cfl / s_b, clipped to
// T - t_b (then the sample lands exactly on T and is done). Fixed mode: dt = fixed_dt until
// n_target steps; the realised CFL number dt * s_b is checked against a guard. A NaN partial marks
// a non-physical sample: it stops and the status word records it.
// One block per sample: the block's threads stride over the sample's tile partials and combine
// them with a shuffle tree. The maximum of non-negative doubles is exact in any order, so the
// result is bitwise independent of the block size. A decomposed grid splits this in two: the
// maximum of each block (smax_out), then the time control from the maximum over all blocks
// (smax_in).
// ---------------------------------------------------------------------------------------------
constexpr int FINISH_NT = 256;

__device__ void finish_sample(const FinishArgs& a, int s, double smax, int bad);

__global__ void __launch_bounds__(FINISH_NT) k_finish(const FinishArgs a) {
    const int s = blockIdx.x;
    const int l = level_of_sample(a.g, s);
    const LevelInfo& L = a.g.lev[l];
    const int b = s - L.sample0;
    if (a.advance && a.done[s]) return;  // skipped by this step's stages (uniform over the block)
    if (a.smax_in) {
        // decomposed grid: the maximum over every block, taken by the caller
        if (threadIdx.x != 0) return;
        const double v = a.smax_in[s];
        finish_sample(a, s, v, !(v < INFINITY));
        return;
    }
    const double* part = a.speed_part + L.work0 + (long long)b * L.tiles;
    double smax = 0.0;
    int bad = 0;
    for (int k = threadIdx.x; k < L.tiles; k += FINISH_NT) {
        const double v = part[k];
        if (v != v) bad = 1;
        else smax = v > smax ? v : smax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, smax, o);
        smax = v > smax ? v : smax;
    }
    __shared__ double wmax[FINISH_NT / 32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = smax;
    bad = __syncthreads_or(bad);   // also orders every thread's read of done[s] before the writes below
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int w = 1; w < FINISH_NT / 32; ++w) smax = wmax[w] > smax ? wmax[w] : smax;
    if (a.smax_out) {
        a.smax_out[s] = bad ? INFINITY : smax;
        return;
    }
    finish_sample(a, s, smax, bad);
}

// Time control of sample s from its maximum speed: advance t and the step count after a step,
// then the next dt (CFL or fixed), the last-step and done flags and the status bits.
__device__ void finish_sample(const FinishArgs& a, int s, double smax, int bad) {
    if (a.advance) {
        double t = a.t[s];
        const long long n = a.nstep[s] + 1;
        if (a.fixed_dt > 0.0) t = (double)n * a.fixed_dt;
        else t = a.last[s] ? *a.T_end : t + a.dt[s];
        a.t[s] = t;
        a.nstep[s] = n;
    }
    if (bad) {
        atomicOr(a.status, ST_NONPHYSICAL);
        a.done[s] = 1;
        return;
    }
    const double t = a.t[s];
    if (a.fixed_dt > 0.0) {
        a.dt[s] = a.fixed_dt;
        a.dt_f[s] = (float)a.fixed_dt;
        a.last[s] = 0;
        const bool fin = a.nstep[s] >= *a.n_target;
        a.done[s] = fin ? 1 : 0;
        if (!fin && a.cfl_max) atomicMax(reinterpret_cast<unsigned long long*>(a.cfl_max),
                                         (unsigned long long)__double_as_longlong(a.fixed_dt * smax));
        if (!fin && a.fixed_dt * smax > a.cfl_guard) atomicOr(a.status, ST_CFL);
        return;
    }
    const double T = *a.T_end;
    if (!(t < T)) {
        a.done[s] = 1;
        return;
    }
    double dt = a.cfl / smax;
    int last = 0;
    if (!(dt < T - t)) {
        dt = T - t;
        last = 1;
    }
    if (isinf(dt)) dt = 0.0;  // no wave motion and no end time: nothing to advance
    a.dt[s] = dt;
    a.dt_f[s] = (float)dt;
    a.last[s] = last;
    a.done[s] = 0;
}

cudaError_t launch_finish(const FinishArgs& a, cudaStream_t s) {
    const int n = a.g.total_samples;
    if (n <= 0) return cudaSuccess;
    k_finish<<<n, FINISH_NT, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator of the KH parameters:
// theta_{b,j} = hi_j * (splitmix64(seed ^ (b P + j)) >> 11) * 2^-53, hi = 1 (amplitudes, first
// half) or 2 pi (phases, second half); splitmix64(x) = mix(x + golden gamma).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sm64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// (j+1)-th prime by trial division (j < 128 here: primes up to 719)
__device__ uint32_t nth_prime(int j) {
    uint32_t p = 1;
    for (int found = -1; found < j;) {
        ++p;
        bool prime = p >= 2;
        for (uint32_t d = 2; d * d <= p; ++d)
            if (p % d == 0) { prime = false; break; }
        if (prime) ++found;
    }
    return p;
}

// Halton radical inverse phi_p(n) = sum_k d_k p^(-k-1) for n = sum_k d_k p^k, formed as the exact
// integer fraction num / p^K (both below 2^53 for n < 2^31, p < 1024) and one rounded division
__device__ double radical_inverse(uint64_t n, uint32_t p) {
    uint64_t num = 0, den = 1;
    while (n > 0) {
        num = num * p + n % p;
        den *= p;
        n /= p;
    }
    return (double)num / (double)den;
}

__global__ void k_theta(uint64_t seed, long long sample_offset, int sampler, const ThetaMap map, int samples, int P,
                        double* theta) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)samples * P) return;
    const int b = (int)(i / P), j = (int)(i - (long long)b * P);
    int l = 0;
    for (int k = 1; k < map.nlev; ++k)
        if (b >= map.sample0[k]) l = k;
    const uint64_t gb = (uint64_t)(sample_offset + map.src0[l] + (b - map.sample0[l]));
    const double hi = j < P / 2 ? 1.0 : 2.0 * 3.14159265358979323846;
    double u01;
    if (sampler == 0) {
        const uint64_t r = sm64(seed ^ (gb * (uint64_t)P + (uint64_t)j));
        u01 = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    } else {
        u01 = radical_inverse(gb + 1, nth_prime(j));
        if (sampler == 2) {
            const uint64_t r = sm64(seed ^ ((1ull << 63) + (uint64_t)j));
            u01 = u01 + (double)(r >> 11) * (1.0 / 9007199254740992.0);
            if (u01 >= 1.0) u01 = u01 - 1.0;
        }
    }
    theta[i] = hi * u01;
}

cudaError_t launch_theta(uint64_t seed, long long sample_offset, int sampler, const ThetaMap& map, int samples, int P,
                         double* theta, cudaStream_t s) {
    const long long n = (long long)samples * P;
    if (n <= 0) return cudaSuccess;
    k_theta<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, sample_offset, sampler, map, samples, P, theta);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Initial data (cell averages of conserved variables), computed in FP64, stored as R.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

__device__ __forceinline__ void kh_states(int nd, double gamma, double* Uin, double* Uout) {
    // inner band rho = 2, u = -0.5; outer rho = 1, u = 0.5; v = w = 0; p = 2.5 (Sec. 3, reading)
    for (int v = 0; v < 5; ++v) { Uin[v] = 0.0; Uout[v] = 0.0; }
    Uin[0] = 2.0;
    Uin[1] = 2.0 * -0.5;
    Uin[nd + 1] = 2.5 / (gamma - 1.0) + 0.5 * 2.0 * (-0.5 * -0.5);
    Uout[0] = 1.0;
    Uout[1] = 1.0 * 0.5;
    Uout[nd + 1] = 2.5 / (gamma - 1.0) + 0.5 * 1.0 * (0.5 * 0.5);
}

// One thread per (column, sample): the interface displacement Y is evaluated once per column
// (x for 2D, (x,z) for 3D), then the column is filled with the band's volume fraction in y.
template <class R, int ND>
__global__ void k_init_kh(const InitArgs a) {
    constexpr int NV = ND + 2;
    const int s = blockIdx.y;
    const int l = level_of_sample(a.g, s);
    const LevelInfo& L = a.g.lev[l];
    const int b = s - L.sample0;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    if (col >= nx * nz) return;
    const int x = col % nx, z = col / nx;
    const double PI = 3.14159265358979323846;
    const double* th = a.theta + (long long)s * a.P;
    const double hx = L.dx[0], hy = L.dx[1];
    // cell centres from the whole grid's indices (a block of a decomposed grid is offset by off)
    const double xc = a.g.lo[0] + (x + a.g.off[0] + 0.5) * hx;
    double Y = 0.0;
    if (ND == 2) {
        for (int n = 1; n <= 10; ++n) Y = Y + th[n - 1] * sin(2.0 * PI * n * xc + th[10 + n - 1]);
    } else {
        const double zc = a.g.lo[2] + (z + a.g.off[2] + 0.5) * L.dx[2];
        for (int n = 1; n <= 8; ++n)
            for (int m = 1; m <= 8; ++m) {
                const int j = (n - 1) * 8 + (m - 1);
                Y = Y + th[j] * sin(2.0 * PI * (n * xc + m * zc) + th[64 + j]);
            }
    }
    Y = 0.01 * Y;
    double Uin[5], Uout[5];
    kh_states(ND, a.g.gamma, Uin, Uout);
    const long long plane = (long long)nx * ny * nz;
    R* U = reinterpret_cast<R*>(a.U) + L.elem0 + (long long)b * NV * plane;
    for (int y = 0; y < ny; ++y) {
        const double ylo = a.g.lo[1] + (y + a.g.off[1]) * hy;
        const double f_lo = clamp01((0.25 + Y - ylo) / hy);
        const double f_hi = clamp01((0.75 + Y - ylo) / hy);
        const double f = f_hi - f_lo;
        const long long off = ((long long)z * ny + y) * nx + x;
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v * plane + off] = R(f * Uin[v] + (1.0 - f) * Uout[v]);
    }
}

__device__ void vortex_point(double g, double xc, double yc, double x, double y, double* Uc) {
    const double PI = 3.14159265358979323846, beta = 5.0;
    const double rx = x - xc, ry = y - yc, r2 = rx * rx + ry * ry;
    const double e = exp(0.5 * (1.0 - r2));
    const double u = 1.0 - beta / (2.0 * PI) * e * ry;
    const double v = 1.0 + beta / (2.0 * PI) * e * rx;
    const double Tm = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * PI * PI) * e * e;
    const double rho = pow(Tm, 1.0 / (g - 1.0));
    const double p = rho * Tm;
    Uc[0] = rho;
    Uc[1] = rho * u;
    Uc[2] = rho * v;
    Uc[3] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
}

// Tubes (split at x = 0.5 with exact volume fraction), Burgers sine (exact averages) and the
// isentropic vortex (5x5 Gauss-Legendre averages); one thread per cell.
template <class R, int ND>
__global__ void k_init_cell(const InitArgs a) {
    const int s = blockIdx.y;
    const int l = level_of_sample(a.g, s);
    const LevelInfo& L = a.g.lev[l];
    const int b = s - L.sample0;
    const int nv = a.g.nv;
    const long long plane = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= plane) return;
    const int x = (int)(i % L.n[0]) + a.g.off[0];          // whole-grid indices
    const int y = (int)((i / L.n[0]) % L.n[1]) + a.g.off[1];
    R* U = reinterpret_cast<R*>(a.U) + L.elem0 + (long long)b * nv * plane;
    const double g = a.g.gamma;
    const double PI = 3.14159265358979323846;
    double out[5] = {0, 0, 0, 0, 0};
    if (a.kind == 1 || a.kind == 2) {
        double WL[5] = {0, 0, 0, 0, 0}, WR[5] = {0, 0, 0, 0, 0};
        const int ip = ND + 1;
        if (a.kind == 1) { WL[0] = 1.0; WL[ip] = 1.0; WR[0] = 0.125; WR[ip] = 0.1; }
        else { WL[0] = 0.445; WL[1] = 0.698; WL[ip] = 3.528; WR[0] = 0.5; WR[ip] = 0.571; }
        double UL[5], UR[5];
        for (int k = 0; k < 2; ++k) {
            const double* W = k == 0 ? WL : WR;
            double* Uc = k == 0 ? UL : UR;
            double u2 = 0.0;
            for (int d = 0; d < ND; ++d) u2 = u2 + W[1 + d] * W[1 + d];
            Uc[0] = W[0];
            for (int d = 0; d < ND; ++d) Uc[1 + d] = W[0] * W[1 + d];
            Uc[ip] = W[ip] / (g - 1.0) + 0.5 * W[0] * u2;
        }
        const double h = L.dx[0];
        const double xl = a.g.lo[0] + x * h;
        const double f = fmin(1.0, fmax(0.0, (0.5 - xl) / h));
        for (int v = 0; v < nv; ++v) out[v] = f * UL[v] + (1.0 - f) * UR[v];
    } else if (a.kind == 3) {
        const double h = L.dx[0];
        const double xl = a.g.lo[0] + x * h, xr = xl + h;
        out[0] = (cos(2.0 * PI * xl) - cos(2.0 * PI * xr)) / (2.0 * PI * h);
    } else if (a.kind == 4) {
        const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831, 0.9061798459386640};
        const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                              0.2369268850561891};
        const double hx = L.dx[0], hy = L.dx[1];
        const double lo0 = a.g.lo[0], lo1 = a.g.lo[1];
        const double cx = lo0 + (x + 0.5) * hx, cy = lo1 + (y + 0.5) * hy;
        for (int p = 0; p < 5; ++p)
            for (int q = 0; q < 5; ++q) {
                double Uc[4];
                vortex_point(g, a.vortex_center[0], a.vortex_center[1], cx + 0.5 * hx * gx[p], cy + 0.5 * hy * gx[q], Uc);
                for (int v = 0; v < 4; ++v) out[v] += 0.25 * gw[p] * gw[q] * Uc[v];
            }
    }
    for (int v = 0; v < nv; ++v) U[v * plane + i] = R(out[v]);
}

template <class R>
static cudaError_t launch_init_t(int ndim, const InitArgs& a, cudaStream_t s) {
    int maxcols = 0;
    long long maxcells = 0;
    for (int l = 0; l < a.g.nlev; ++l) {
        const LevelInfo& L = a.g.lev[l];
        maxcols = max(maxcols, L.n[0] * L.n[2]);
        maxcells = maxcells > (long long)L.n[0] * L.n[1] * L.n[2] ? maxcells : (long long)L.n[0] * L.n[1] * L.n[2];
    }
    if (a.g.total_samples <= 0) return cudaSuccess;
    if (a.kind == 0) {
        dim3 grid((maxcols + 127) / 128, a.g.total_samples);
        if (ndim == 2) k_init_kh<R, 2><<<grid, 128, 0, s>>>(a);
        else k_init_kh<R, 3><<<grid, 128, 0, s>>>(a);
    } else {
        dim3 grid((unsigned)((maxcells + 255) / 256), a.g.total_samples);
        if (ndim == 1) k_init_cell<R, 1><<<grid, 256, 0, s>>>(a);
        else if (ndim == 2) k_init_cell<R, 2><<<grid, 256, 0, s>>>(a);
        else k_init_cell<R, 3><<<grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_init(int fp64, int ndim, const InitArgs& a, cudaStream_t s) {
    return fp64 ? launch_init_t<double>(ndim, a, s) : launch_init_t<float>(ndim, a, s);
}

// ---------------------------------------------------------------------------------------------
// Halo layers of a block of a decomposed grid (Sec. 2.1, last paragraph; Sec. 3.1): the G cells
// next to face f = 2k + side, gathered as [sample][var][layer][cross] for the neighbouring block,
// cross = the other directions' cells in (z, y, x) order (x fastest). Layer l is index l along k
// on the low face and n_k - G + l on the high face. A plain copy.
// ---------------------------------------------------------------------------------------------
template <class R>
__global__ void k_halo_pack(const GridArgs g, int G, int face, int rows, const R* __restrict__ U, R* __restrict__ dst) {
    // blockIdx.x (with x-threads) covers the cross-section, blockIdx.y strides over the rows
    // (sample, var, layer); 32-bit index arithmetic within a sample (< 2^31 elements)
    const LevelInfo& L = g.lev[0];
    const int k = face >> 1;
    const int n[3] = {L.n[0], L.n[1], L.n[2]};
    const int csize = n[0] * n[1] * n[2] / n[k];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= csize) return;
    // the cell of this cross-section index (x fastest, the face direction left out)
    int c[3];
    int rem = q;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j == k) continue;
        c[j] = rem % n[j];
        rem /= n[j];
    }
    const int plane = n[0] * n[1] * n[2];
    const int stride_k = k == 0 ? 1 : (k == 1 ? n[0] : n[0] * n[1]);
    c[k] = 0;
    const int base = (c[2] * n[1] + c[1]) * n[0] + c[0];
    const int first = (face & 1) ? n[k] - G : 0;
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        const int layer = r % G;
        const long long bv = r / G;  // sample * nv + var
        dst[(long long)r * csize + q] = U[bv * plane + base + (first + layer) * stride_k];
    }
}

// Maximum wave speed over the blocks of a decomposed grid, per sample (step a8 across blocks): the
// elementwise maximum of n per-block vectors, NaN-propagating (a NaN or +infinity in any block
// marks the sample non-physical for alsv_finish_step). The maximum is exact, so the order of the
// blocks does not matter; it is the blocks' order anyway.
__global__ void k_speed_max_combine(const SpeedCombineArgs a, int samples, double* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= samples) return;
    double m = a.in[0][s];
    for (int i = 1; i < a.n; ++i) {
        const double v = a.in[i][s];
        if (v != v || v > m) m = v;   // once m is NaN, neither test replaces it
    }
    out[s] = m;
}

cudaError_t launch_speed_max_combine(const SpeedCombineArgs& a, int samples, double* out, cudaStream_t s) {
    if (samples <= 0) return cudaSuccess;
    k_speed_max_combine<<<(unsigned)((samples + 255) / 256), 256, 0, s>>>(a, samples, out);
    return cudaGetLastError();
}

cudaError_t launch_halo_pack(int fp64, const GridArgs& g, int G, const void* U, void* const dst[6], cudaStream_t s) {
    const LevelInfo& L = g.lev[0];
    for (int f = 0; f < 6; ++f) {
        if (!dst[f]) continue;
        const long long csize = (long long)L.n[0] * L.n[1] * L.n[2] / L.n[f >> 1];
        const int rows = L.samples * g.nv * G;   // < 2^16 samples x 5 vars x 2 layers
        if (csize <= 0 || rows <= 0) continue;
        const unsigned bx = (unsigned)((csize + 255) / 256);
        // about 16 resident blocks per SM in all, rows strided by gridDim.y
        const unsigned by = (unsigned)std::max<long long>(1, std::min<long long>(rows, (152LL * 16 + bx - 1) / bx));
        const dim3 grid(bx, std::min(by, 65535u));
        if (fp64)
            k_halo_pack<double><<<grid, 256, 0, s>>>(g, G, f, rows, static_cast<const double*>(U), static_cast<double*>(dst[f]));
        else
            k_halo_pack<float><<<grid, 256, 0, s>>>(g, G, f, rows, static_cast<const float*>(U), static_cast<float*>(dst[f]));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------------------------
// Monte Carlo mean/variance (Sec. 2.2), FP64 Welford over samples in ascending order, one thread
// per cell; quantities are primitive (rho, u_k, p) for Euler and u for Burgers.
// Accumulator: int64 count at byte 0, mean[q][cells] at byte 256, then M2[q][cells].
// ---------------------------------------------------------------------------------------------
template <class R, int NV, int EULER>
__global__ void k_welford(const GridArgs g, const void* Uv, void* stats) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const long long n0 = *reinterpret_cast<const long long*>(stats);
    double* mean = reinterpret_cast<double*>(reinterpret_cast<char*>(stats) + 256);
    double* M2 = mean + NV * C;
    const R* U = reinterpret_cast<const R*>(Uv);
    double mu[NV], m2[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) { mu[q] = mean[q * C + i]; m2[q] = M2[q * C + i]; }
    const int B = L.samples;
    const double gm1 = g.gamma - 1.0;
#pragma unroll 4
    for (int b = 0; b < B; ++b) {
        double x[NV];
        prim_quantities<R, NV, EULER>(U + (long long)b * NV * C, C, i, gm1, x);
        const double n = (double)(n0 + b + 1);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double delta = x[q] - mu[q];
            mu[q] = mu[q] + delta / n;
            m2[q] = m2[q] + delta * (x[q] - mu[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) { mean[q * C + i] = mu[q]; M2[q * C + i] = m2[q]; }
}

__global__ void k_welford_count(void* stats, int B) { *reinterpret_cast<long long*>(stats) += B; }

template <class R>
static cudaError_t launch_welford_t(const GridArgs& g, const void* U, void* stats, cudaStream_t s) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const unsigned grid = (unsigned)((C + 127) / 128);
    switch (g.nv) {
        case 1: k_welford<R, 1, 0><<<grid, 128, 0, s>>>(g, U, stats); break;
        case 3: k_welford<R, 3, 1><<<grid, 128, 0, s>>>(g, U, stats); break;
        case 4: k_welford<R, 4, 1><<<grid, 128, 0, s>>>(g, U, stats); break;
        default: k_welford<R, 5, 1><<<grid, 128, 0, s>>>(g, U, stats); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_welford_count<<<1, 1, 0, s>>>(stats, L.samples);
    return cudaGetLastError();
}

cudaError_t launch_welford(int fp64, const GridArgs& g, const void* U, void* stats, cudaStream_t s) {
    return fp64 ? launch_welford_t<double>(g, U, stats, s) : launch_welford_t<float>(g, U, stats, s);
}

__global__ void k_stats_read(long long C, int nq, const void* stats, double* mean_out, double* var_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C * nq) return;
    const long long n = *reinterpret_cast<const long long*>(stats);
    const double* mean = reinterpret_cast<const double*>(reinterpret_cast<const char*>(stats) + 256);
    const double* M2 = mean + nq * C;
    if (mean_out) mean_out[i] = mean[i];
    if (var_out) var_out[i] = n > 1 ? M2[i] / (double)(n - 1) : 0.0;
}

cudaError_t launch_stats_read(const GridArgs& g, const void* stats, double* mean, double* var, cudaStream_t s) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long n = C * g.nv;
    k_stats_read<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C, g.nv, stats, mean, var);
    return cudaGetLastError();
}

// Chan-Golub-LeVeque pairwise merge of two Welford accumulators, one thread per (q, cell):
// n = nA + nB, d = mB - mA, m = mA + d nB / n, M2 = M2A + M2B + d^2 nA nB / n. The count is
// updated by a one-thread kernel afterwards (every thread reads the counts first).
__global__ void k_stats_merge(long long C, int nq, void* stats, const void* other) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C * nq) return;
    const long long na = *reinterpret_cast<const long long*>(stats);
    const long long nb = *reinterpret_cast<const long long*>(other);
    double* mA = reinterpret_cast<double*>(reinterpret_cast<char*>(stats) + 256);
    double* MA = mA + nq * C;
    const double* mB = reinterpret_cast<const double*>(reinterpret_cast<const char*>(other) + 256);
    const double* MB = mB + nq * C;
    if (nb == 0) return;
    if (na == 0) {
        mA[i] = mB[i];
        MA[i] = MB[i];
        return;
    }
    const double n = (double)(na + nb);
    const double d = mB[i] - mA[i];
    mA[i] = mA[i] + d * (double)nb / n;
    MA[i] = MA[i] + MB[i] + d * d * (double)na * (double)nb / n;
}

__global__ void k_stats_merge_count(void* stats, const void* other) {
    *reinterpret_cast<long long*>(stats) += *reinterpret_cast<const long long*>(other);
}

cudaError_t launch_stats_merge(const GridArgs& g, void* stats, const void* other, cudaStream_t s) {
    const LevelInfo& L = g.lev[0];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long n = C * g.nv;
    k_stats_merge<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C, g.nv, stats, other);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_stats_merge_count<<<1, 1, 0, s>>>(stats, other);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Fixed-order FP64 reductions (conservation totals per sample and variable; kinetic energy per
// sample). Pass 1: each CTA reduces one chunk of kChunk cells of one (sample, var) - thread t
// sums cells t, t+256, ... sequentially, then a fixed shuffle tree and a fixed tree over warps -
// into a per-chunk partial. Pass 2: one CTA per (sample, var) reduces the partials in the same
// pattern and multiplies by the cell volume. The result depends only on the data.
// ---------------------------------------------------------------------------------------------
constexpr int kChunk = 4096;
constexpr int kRT = 256;

__device__ __forceinline__ double block_sum_fixed(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x;
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid == 0) {
        r = sh[0];
        for (int k = 1; k < kRT / 32; ++k) r += sh[k];
    }
    __syncthreads();
    return r;
}

static long long chunks_of(const LevelInfo& L) {
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    return (C + kChunk - 1) / kChunk;
}

long long reduce_partial_count(const GridArgs& g) {
    long long mx = 0;
    for (int l = 0; l < g.nlev; ++l) mx = mx > chunks_of(g.lev[l]) ? mx : chunks_of(g.lev[l]);
    return mx * (long long)g.total_samples * g.nv;
}

template <class R>
__global__ void __launch_bounds__(kRT) k_reduce1(const GridArgs g, int kind, const void* Uv, double* partial,
                                                 long long maxchunks) {
    __shared__ double sh[kRT / 32];
    const int nvr = kind == 0 ? g.nv : 1;
    const int sv = blockIdx.x;
    const int s = sv / nvr, v = sv - s * nvr;
    const int l = level_of_sample(g, s);
    const LevelInfo& L = g.lev[l];
    const int b = s - L.sample0;
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long chunk = blockIdx.y;
    if (chunk * kChunk >= C) return;  // uniform per CTA
    const R* U = reinterpret_cast<const R*>(Uv) + L.elem0 + (long long)b * g.nv * C;
    const long long c0 = chunk * kChunk;
    const long long c1 = c0 + kChunk < C ? c0 + kChunk : C;
    double acc = 0.0;
    for (long long i = c0 + threadIdx.x; i < c1; i += kRT) {
        if (kind == 0) {
            acc += (double)U[v * C + i];
        } else if (kind == 2) {
            // mixing-layer width: 4 c (1 - c), c = rho - 1 the inner-band fraction of the KH
            // densities 1 and 2
            const double rho = (double)U[i];
            acc += 4.0 * (rho - 1.0) * (2.0 - rho);
        } else {
            const double rho = (double)U[i];
            double mm = 0.0;
            for (int k = 1; k < g.nv - 1; ++k) {
                const double m = (double)U[k * C + i];
                mm += m * m;
            }
            acc += 0.5 * mm / rho;
        }
    }
    const double r = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0) partial[(long long)sv * maxchunks + chunk] = r;
}

__device__ __forceinline__ double cell_volume(const GridArgs& g, const LevelInfo& L) {
    double dV = 1.0;
    for (int k = 0; k < g.ndim; ++k) dV *= L.dx[k];
    return dV;
}

__global__ void __launch_bounds__(kRT) k_reduce2(const GridArgs g, int kind, const double* partial, long long maxchunks,
                                                 double* out) {
    __shared__ double sh[kRT / 32];
    const int nvr = kind == 0 ? g.nv : 1;
    const int sv = blockIdx.x;
    const int s = sv / nvr;
    const int l = level_of_sample(g, s);
    const LevelInfo& L = g.lev[l];
    const long long C = (long long)L.n[0] * L.n[1] * L.n[2];
    const long long nch = (C + kChunk - 1) / kChunk;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < nch; i += kRT) acc += partial[(long long)sv * maxchunks + i];
    const double r = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0) out[sv] = r * cell_volume(g, L);
}

cudaError_t launch_reduce(int fp64, int kind, const GridArgs& g, const void* U, double* partial, double* out,
                          cudaStream_t s) {
    long long maxchunks = 0;
    for (int l = 0; l < g.nlev; ++l) maxchunks = maxchunks > chunks_of(g.lev[l]) ? maxchunks : chunks_of(g.lev[l]);
    const int nvr = kind == 0 ? g.nv : 1;
    const long long rows = (long long)g.total_samples * nvr;
    if (rows <= 0 || maxchunks <= 0) return cudaSuccess;
    if (maxchunks > 65535) return cudaErrorInvalidConfiguration;  // 2.7e8 cells per sample
    dim3 grid1((unsigned)rows, (unsigned)maxchunks);
    if (fp64) k_reduce1<double><<<grid1, kRT, 0, s>>>(g, kind, U, partial, maxchunks);
    else k_reduce1<float><<<grid1, kRT, 0, s>>>(g, kind, U, partial, maxchunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce2<<<(unsigned)rows, kRT, 0, s>>>(g, kind, partial, maxchunks, out);
    return cudaGetLastError();
}

}  // namespace alsv
