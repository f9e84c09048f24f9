// Plain FP64 CPU oracle for the finite-volume hot path of Alsvinn (arXiv:1912.07645).
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or calls this file;
// only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / --impl reference legs load it.
// It shares no code, header, table or constant generator with the CUDA path.
//
// What it computes (each function cites the passage it follows):
//   * eq. (1.1), Sec. 1: u_t + div F(u) = 0 for the compressible Euler equations (ideal gas) and,
//     as the scalar case, multi-dimensional Burgers u_t + sum_k (u^2/2)_{x_k} = 0.
//   * eq. (2.1), Sec. 2.1: the semi-discrete update d/dt u_i = -sum_k (F_{i+e_k/2} - F_{i-e_k/2})/dx_k,
//     with one dx per direction (the paper prints a single Delta).
//   * Sec. 2.1 names the components: HLLC, Rusanov numerical fluxes (plus HLL, the HLLC family
//     without the contact wave), SSP Runge-Kutta time stepping (Gottlieb-Shu-Tadmor), WENO
//     reconstruction (Shu 1999) and, as simpler reconstructions, piecewise constant and the
//     MC-limited linear one.
//   * Sec. 2.2: the Monte Carlo estimator of mean and variance per cell (Welford, samples in
//     ascending order).
//   * Sec. 3: Kelvin-Helmholtz shear-flow initial data (two states, perturbed interfaces).
// Readings where the paper is silent (wave speeds, CFL rule, HLLC form, WENO3 epsilon, KH
// perturbation, positivity fallback, boundary ghosts, RNG) are listed beside each function.
//
// Style: one cell at a time, directions summed in the order x, y, z, every interface flux
// recomputed for each adjacent cell, no tiling, no fusion. Compiled with -O2 -ffp-contract=off.
//
// The scalar type is a template parameter so the same code runs on double and on forward-mode
// dual numbers; the dual run gives the exact derivative of the discrete map (active branch at
// kinks), which is the oracle for the discrete adjoint.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ------------------------------------------------------------------------------------------
// Enumerations (values are part of the oracle's own ctypes interface)
// ------------------------------------------------------------------------------------------
enum { EQ_BURGERS = 0, EQ_EULER = 1 };
enum { REC_PC = 0, REC_MC = 1, REC_WENO3 = 2, REC_ENO2 = 3 };
enum { RV_CONS = 0, RV_PRIM = 1 };
enum { FLUX_RUSANOV = 0, FLUX_HLL = 1, FLUX_HLLC = 2, FLUX_ROE = 3, FLUX_GODUNOV = 4, FLUX_EC = 5, FLUX_EC4 = 6, FLUX_TECNO2 = 7 };
enum { RK_SSP2 = 2, RK_SSP3 = 3 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECTIVE = 2 };
enum { INIT_KH = 0, INIT_SOD = 1, INIT_LAX = 2, INIT_BURGERS_SINE = 3, INIT_VORTEX = 4 };

struct Desc {
    int32_t ndim;
    int32_t n[3];
    double lo[3];
    double hi[3];
    int32_t eq;
    double gamma;
    int32_t recon;
    int32_t rvars;
    int32_t flux;
    int32_t rk;
    int32_t bc[3][2];
    double cfl;
    double weno_eps;      // used when weno_eps_dx2 == 0
    int32_t weno_eps_dx2; // 1: epsilon = dx_k^2 per direction
};

// ------------------------------------------------------------------------------------------
// Forward-mode dual numbers. Derivatives of max/min/abs/clamp follow the branch taken.
// ------------------------------------------------------------------------------------------
template <int N> struct Dual {
    double v;
    double d[N];
    Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
    Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v / b.v;
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
    return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
    Dual<N> r; r.v = std::sqrt(a.v);
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
    return r;
}
template <int N> inline Dual<N> sin(const Dual<N>& a) {
    Dual<N> r; r.v = std::sin(a.v); double c = std::cos(a.v);
    for (int i = 0; i < N; ++i) r.d[i] = c * a.d[i];
    return r;
}

// ------------------------------------------------------------------------------------------
// Flop-counting scalar: a double whose arithmetic (+, -, *, /, sqrt, sin) adds one to a counter.
// Only used to count the algorithmic floating-point operations of the scheme's pieces.
// ------------------------------------------------------------------------------------------
static thread_local long long g_flops = 0;
struct Cnt {
    double v;
    Cnt() : v(0.0) {}
    Cnt(double x) : v(x) {}
};
inline Cnt operator+(const Cnt& a, const Cnt& b) { ++g_flops; return Cnt(a.v + b.v); }
inline Cnt operator-(const Cnt& a, const Cnt& b) { ++g_flops; return Cnt(a.v - b.v); }
inline Cnt operator*(const Cnt& a, const Cnt& b) { ++g_flops; return Cnt(a.v * b.v); }
inline Cnt operator/(const Cnt& a, const Cnt& b) { ++g_flops; return Cnt(a.v / b.v); }
inline Cnt operator-(const Cnt& a) { return Cnt(-a.v); }
inline Cnt operator+(const Cnt& a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, const Cnt& b) { return Cnt(a) + b; }
inline Cnt operator-(const Cnt& a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, const Cnt& b) { return Cnt(a) - b; }
inline Cnt operator*(const Cnt& a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, const Cnt& b) { return Cnt(a) * b; }
inline Cnt operator/(const Cnt& a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, const Cnt& b) { return Cnt(a) / b; }

inline double val(double x) { return x; }
inline double val(const Cnt& x) { return x.v; }
inline Cnt sqrt_(const Cnt& x) { ++g_flops; return Cnt(std::sqrt(x.v)); }
inline Cnt sin_(const Cnt& x) { ++g_flops; return Cnt(std::sin(x.v)); }
template <int N> inline double val(const Dual<N>& x) { return x.v; }
inline double sqrt_(double x) { return std::sqrt(x); }
template <int N> inline Dual<N> sqrt_(const Dual<N>& x) { return sqrt(x); }
inline double sin_(double x) { return std::sin(x); }
template <int N> inline Dual<N> sin_(const Dual<N>& x) { return sin(x); }
inline double pow_(double x, double e) { return std::pow(x, e); }
inline Cnt pow_(const Cnt& x, double e) { ++g_flops; return Cnt(std::pow(x.v, e)); }
template <int N> inline Dual<N> pow_(const Dual<N>& x, double e) {
    Dual<N> r; r.v = std::pow(x.v, e); double dv = e * std::pow(x.v, e - 1.0);
    for (int i = 0; i < N; ++i) r.d[i] = dv * x.d[i];
    return r;
}
inline double log_(double x) { return std::log(x); }
inline Cnt log_(const Cnt& x) { ++g_flops; return Cnt(std::log(x.v)); }
template <int N> inline Dual<N> log_(const Dual<N>& x) {
    Dual<N> r; r.v = std::log(x.v);
    for (int i = 0; i < N; ++i) r.d[i] = x.d[i] / x.v;
    return r;
}
template <class T> inline T abs_(const T& x) { return val(x) < 0.0 ? T(-x) : x; }
// ties pick the first argument
template <class T> inline T max_(const T& a, const T& b) { return val(b) > val(a) ? b : a; }
template <class T> inline T min_(const T& a, const T& b) { return val(b) < val(a) ? b : a; }

// ------------------------------------------------------------------------------------------
// Grid geometry and ghost cells
// ------------------------------------------------------------------------------------------
inline int nvars(const Desc& d) { return d.eq == EQ_BURGERS ? 1 : d.ndim + 2; }
inline double dx(const Desc& d, int k) { return (d.hi[k] - d.lo[k]) / d.n[k]; }
inline int64_t ncells(const Desc& d) { return (int64_t)d.n[0] * d.n[1] * d.n[2]; }
inline int64_t lin(const Desc& d, int v, int x, int y, int z) {
    return (((int64_t)v * d.n[2] + z) * d.n[1] + y) * d.n[0] + x;
}

// Boundary reading (paper silent): periodic wraps; outflow copies the nearest interior cell;
// reflective mirrors interior cell -1-j for ghost j and negates the velocity normal to the wall.
// Returns the interior index and sets *flip when the mirrored value must be negated.
inline int ghost_map(int i, int n, int bc_lo, int bc_hi, bool* flip) {
    *flip = false;
    if (i < 0) {
        if (bc_lo == BC_PERIODIC) return ((i % n) + n) % n;
        if (bc_lo == BC_OUTFLOW) return 0;
        *flip = true;
        return -1 - i;
    }
    if (i >= n) {
        if (bc_hi == BC_PERIODIC) return i % n;
        if (bc_hi == BC_OUTFLOW) return n - 1;
        *flip = true;
        return 2 * n - 1 - i;
    }
    return i;
}

// Conserved state of the cell at position c (x,y,z) shifted to index i along direction k.
template <class T>
inline void cell_cons(const Desc& d, const T* U, const int c[3], int k, int i, T* out) {
    int p[3] = {c[0], c[1], c[2]};
    bool flip;
    p[k] = ghost_map(i, d.n[k], d.bc[k][0], d.bc[k][1], &flip);
    int nv = nvars(d);
    for (int v = 0; v < nv; ++v) out[v] = U[lin(d, v, p[0], p[1], p[2])];
    if (flip) {
        if (d.eq == EQ_BURGERS) out[0] = -out[0];
        else out[1 + k] = -out[1 + k];
    }
}

// ------------------------------------------------------------------------------------------
// Ideal-gas Euler relations: p = (gamma-1)(E - |m|^2/(2 rho)), E = p/(gamma-1) + rho|u|^2/2
// ------------------------------------------------------------------------------------------
// prim layout: [rho, u_0..u_{ndim-1}, p]
template <class T> inline void cons_to_prim(const Desc& d, const T* U, T* W) {
    int nd = d.ndim;
    T rho = U[0];
    T m2 = T(0.0);
    for (int k = 0; k < nd; ++k) m2 = m2 + U[1 + k] * U[1 + k];
    W[0] = rho;
    for (int k = 0; k < nd; ++k) W[1 + k] = U[1 + k] / rho;
    W[1 + nd] = (d.gamma - 1.0) * (U[1 + nd] - 0.5 * m2 / rho);
}
template <class T> inline void prim_to_cons(const Desc& d, const T* W, T* U) {
    int nd = d.ndim;
    T rho = W[0];
    T u2 = T(0.0);
    for (int k = 0; k < nd; ++k) u2 = u2 + W[1 + k] * W[1 + k];
    U[0] = rho;
    for (int k = 0; k < nd; ++k) U[1 + k] = rho * W[1 + k];
    U[1 + nd] = W[1 + nd] / (d.gamma - 1.0) + 0.5 * rho * u2;
}

// ------------------------------------------------------------------------------------------
// Reconstruction of one cell's two face values from (w_{i-1}, w_i, w_{i+1}) along a direction
// (Sec. 2.1 names ENO/WENO after Shu 1999). fl = value at i-1/2, fr = value at i+1/2.
// ------------------------------------------------------------------------------------------
// minmod of three: the common-sign minimum magnitude, 0 if signs differ or any is 0.
template <class T> inline T minmod3(const T& a, const T& b, const T& c) {
    if (val(a) > 0.0 && val(b) > 0.0 && val(c) > 0.0) return min_(min_(a, b), c);
    if (val(a) < 0.0 && val(b) < 0.0 && val(c) < 0.0) return max_(max_(a, b), c);
    return T(0.0);
}

template <class T>
inline void recon_scalar(int recon, double eps, const T& wm, const T& w0, const T& wp, T* fl, T* fr) {
    if (recon == REC_PC) {
        *fl = w0;
        *fr = w0;
    } else if (recon == REC_MC) {
        // monotonized-central slope: minmod(2 D-, (D- + D+)/2, 2 D+)
        T dm = w0 - wm;
        T dp = wp - w0;
        T s = minmod3(T(2.0 * dm), T(0.5 * (dm + dp)), T(2.0 * dp));
        *fl = w0 - 0.5 * s;
        *fr = w0 + 0.5 * s;
    } else if (recon == REC_ENO2) {
        // second-order ENO (Harten-Engquist-Osher-Chakravarthy; Sec. 2.1 names ENO): of the two
        // linear candidates through {i-1, i} and {i, i+1}, take the smoother one, i.e. the
        // one-sided difference of smaller magnitude (ties take the backward difference)
        T dm = w0 - wm;
        T dp = wp - w0;
        T s = val(abs_(dp)) < val(abs_(dm)) ? dp : dm;
        *fl = w0 - 0.5 * s;
        *fr = w0 + 0.5 * s;
    } else {
        // Jiang-Shu WENO3: candidates on {i-1,i} and {i,i+1}, linear weights 1/3, 2/3,
        // smoothness (differences)^2, alpha_r = d_r / (eps + beta_r)^2.
        const double d0 = 1.0 / 3.0, d1 = 2.0 / 3.0;
        {   // face i+1/2
            T p0 = -0.5 * wm + 1.5 * w0;
            T p1 = 0.5 * w0 + 0.5 * wp;
            T b0 = (w0 - wm) * (w0 - wm);
            T b1 = (wp - w0) * (wp - w0);
            T a0 = d0 / ((eps + b0) * (eps + b0));
            T a1 = d1 / ((eps + b1) * (eps + b1));
            *fr = (a0 * p0 + a1 * p1) / (a0 + a1);
        }
        {   // face i-1/2 (mirror image)
            T p0 = -0.5 * wp + 1.5 * w0;
            T p1 = 0.5 * w0 + 0.5 * wm;
            T b0 = (wp - w0) * (wp - w0);
            T b1 = (w0 - wm) * (w0 - wm);
            T a0 = d0 / ((eps + b0) * (eps + b0));
            T a1 = d1 / ((eps + b1) * (eps + b1));
            *fl = (a0 * p0 + a1 * p1) / (a0 + a1);
        }
    }
}

// Face states of the cell at c shifted to index i along k, returned as PRIMITIVE variables
// (Burgers: the scalar u). Reconstruction is done on conserved or primitive variables per
// d.rvars. Positivity reading: a face state whose density or pressure is not positive reverts
// to the cell's own value in all variables (first order at that face only).
template <class T>
void cell_faces(const Desc& d, const T* U, const int c[3], int k, int i, T* Wl, T* Wr) {
    const int nv = nvars(d);
    T Um[8], U0[8], Up[8];
    cell_cons(d, U, c, k, i - 1, Um);
    cell_cons(d, U, c, k, i, U0);
    cell_cons(d, U, c, k, i + 1, Up);
    double eps = d.weno_eps_dx2 ? dx(d, k) * dx(d, k) : d.weno_eps;
    if (d.eq == EQ_BURGERS) {
        recon_scalar(d.recon, eps, Um[0], U0[0], Up[0], &Wl[0], &Wr[0]);
        return;
    }
    T wm[8], w0[8], wp[8], fl[8], fr[8];
    if (d.rvars == RV_PRIM) {
        cons_to_prim(d, Um, wm);
        cons_to_prim(d, U0, w0);
        cons_to_prim(d, Up, wp);
    } else {
        for (int v = 0; v < nv; ++v) { wm[v] = Um[v]; w0[v] = U0[v]; wp[v] = Up[v]; }
    }
    for (int v = 0; v < nv; ++v) recon_scalar(d.recon, eps, wm[v], w0[v], wp[v], &fl[v], &fr[v]);
    T Wc[8];
    if (d.rvars == RV_PRIM) {
        for (int v = 0; v < nv; ++v) { Wl[v] = fl[v]; Wr[v] = fr[v]; Wc[v] = w0[v]; }
    } else {
        cons_to_prim(d, fl, Wl);
        cons_to_prim(d, fr, Wr);
        cons_to_prim(d, U0, Wc);
    }
    const int ip = d.ndim + 1;
    if (!(val(Wl[0]) > 0.0 && val(Wl[ip]) > 0.0))
        for (int v = 0; v < nv; ++v) Wl[v] = Wc[v];
    if (!(val(Wr[0]) > 0.0 && val(Wr[ip]) > 0.0))
        for (int v = 0; v < nv; ++v) Wr[v] = Wc[v];
}

// ------------------------------------------------------------------------------------------
// Numerical fluxes (Sec. 2.1 names HLLC and Rusanov). Inputs are primitive states; k is the
// sweep direction; output is the conserved flux vector.
// Wave-speed reading (Davis): S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R);
// Rusanov a = max(|u_L| + c_L, |u_R| + c_R); c = sqrt(gamma p / rho).
// ------------------------------------------------------------------------------------------
template <class T> inline void euler_phys_flux(const Desc& d, const T* W, int k, T* F) {
    int nd = d.ndim;
    T U[8];
    prim_to_cons(d, W, U);
    T un = W[1 + k];
    T p = W[1 + nd];
    F[0] = U[0] * un;
    for (int j = 0; j < nd; ++j) F[1 + j] = U[1 + j] * un;
    F[1 + k] = F[1 + k] + p;
    F[1 + nd] = un * (U[1 + nd] + p);
}

// Roe's flux (Roe 1981; Sec. 2.1 names it) for the Euler equations: F = (F_L + F_R)/2
// - (1/2) sum_w |lambda_w| alpha_w r_w over the waves of the Roe-averaged Jacobian along k
// (acoustic waves u_n -/+ a, the entropy wave and one shear wave per tangential direction, all at
// u_n). Roe averages with weights sqrt(rho): u~, H~; a~^2 = (gamma-1)(H~ - |u~|^2/2), rho~ =
// sqrt(rho_L rho_R). Wave strengths from the jumps: alpha_{1,3} = (dp -/+ rho~ a~ du_n)/(2 a~^2),
// alpha_2 = drho - dp/a~^2, alpha_t = rho~ du_t. Entropy fix (reading; the paper names the flux
// only): Harten's smoothing |lambda| -> (lambda^2 + delta^2)/(2 delta) when |lambda| < delta on the
// two acoustic fields, with the Harten-Hyman width delta = max(0, lambda~ - lambda(W_L),
// lambda(W_R) - lambda~) from the one-sided eigenvalues u_n -/+ c.
template <class T> inline T harten_abs(const T& lam, const T& lamL, const T& lamR) {
    T del = max_(T(0.0), max_(T(lam - lamL), T(lamR - lam)));
    if (val(abs_(lam)) < val(del)) return (lam * lam + del * del) / (2.0 * del);
    return abs_(lam);
}
template <class T> void roe_flux_euler(const Desc& d, int k, const T* WL, const T* WR, T* F) {
    const int nd = d.ndim, nv = nd + 2, ip = nd + 1;
    const double g = d.gamma;
    T UL[8], UR[8], FL[8], FR[8];
    prim_to_cons(d, WL, UL);
    prim_to_cons(d, WR, UR);
    euler_phys_flux(d, WL, k, FL);
    euler_phys_flux(d, WR, k, FR);
    T rL = WL[0], rR = WR[0], pL = WL[ip], pR = WR[ip];
    T sL = sqrt_(rL), sR = sqrt_(rR);
    T HL = (UL[ip] + pL) / rL, HR = (UR[ip] + pR) / rR;
    T ut[8];
    T q2 = T(0.0);
    for (int j = 0; j < nd; ++j) {
        ut[j] = (sL * WL[1 + j] + sR * WR[1 + j]) / (sL + sR);
        q2 = q2 + ut[j] * ut[j];
    }
    T H = (sL * HL + sR * HR) / (sL + sR);
    T a2 = (g - 1.0) * (H - 0.5 * q2);
    T a = sqrt_(a2);
    T rt = sL * sR;
    T un = ut[k];
    T dr = rR - rL, dp = pR - pL, dun = WR[1 + k] - WL[1 + k];
    T al1 = (dp - rt * a * dun) / (2.0 * a2);
    T al3 = (dp + rt * a * dun) / (2.0 * a2);
    T al2 = dr - dp / a2;
    T cL = sqrt_(g * pL / rL), cR = sqrt_(g * pR / rR);
    T l1 = harten_abs(T(un - a), T(WL[1 + k] - cL), T(WR[1 + k] - cR));
    T l3 = harten_abs(T(un + a), T(WL[1 + k] + cL), T(WR[1 + k] + cR));
    T l2 = abs_(un);
    T D[8];
    // acoustic waves r_{1,3} = (1, u~ -/+ a e_k, H~ -/+ u_n a), entropy wave r_2 = (1, u~, |u~|^2/2)
    D[0] = l1 * al1 + l2 * al2 + l3 * al3;
    for (int j = 0; j < nd; ++j) D[1 + j] = l1 * al1 * ut[j] + l2 * al2 * ut[j] + l3 * al3 * ut[j];
    D[1 + k] = D[1 + k] - l1 * al1 * a + l3 * al3 * a;
    D[ip] = l1 * al1 * (H - un * a) + l2 * al2 * (0.5 * q2) + l3 * al3 * (H + un * a);
    // shear waves r_t = (0, e_t, u~_t) with strength rho~ du_t, speed u_n
    for (int j = 0; j < nd; ++j) {
        if (j == k) continue;
        T alt = rt * (WR[1 + j] - WL[1 + j]);
        D[1 + j] = D[1 + j] + l2 * alt;
        D[ip] = D[ip] + l2 * alt * ut[j];
    }
    for (int v = 0; v < nv; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * D[v];
}

// Godunov's flux (Sec. 2.1 names it): the physical flux of the exact Riemann solution at x/t = 0.
// Star pressure: root of f_L(p) + f_R(p) + (u_R - u_L) = 0, f_K the shock (Rankine-Hugoniot) or
// rarefaction (isentropic) branch (Toro, ch. 4), by Newton from the linearised (PVRS) guess until
// the relative step is below 1e-15 (at most 60 steps). Tangential velocities are those of the side
// of the contact that x/t = 0 lies on (left when u* >= 0).
template <class T> inline T pressure_branch(double g, const T& p, const T& rK, const T& pK, const T& cK, T* df) {
    if (val(p) > val(pK)) {   // shock
        T A = 2.0 / ((g + 1.0) * rK);
        T B = (g - 1.0) / (g + 1.0) * pK;
        T s = sqrt_(A / (p + B));
        *df = s * (1.0 - (p - pK) / (2.0 * (B + p)));
        return (p - pK) * s;
    }
    T q = p / pK;             // rarefaction
    *df = pow_(q, -(g + 1.0) / (2.0 * g)) / (rK * cK);
    return 2.0 * cK / (g - 1.0) * (pow_(q, (g - 1.0) / (2.0 * g)) - 1.0);
}
template <class T> void godunov_state_euler(double g, const T& rL, const T& uL, const T& pL, const T& rR, const T& uR,
                                            const T& pR, T* r0, T* u0, T* p0, bool* left_of_contact) {
    T cL = sqrt_(g * pL / rL), cR = sqrt_(g * pR / rR);
    T ppv = 0.5 * (pL + pR) - 0.125 * (uR - uL) * (rL + rR) * (cL + cR);
    T p = max_(ppv, T(1e-10 * val(min_(pL, pR))));
    for (int it = 0; it < 60; ++it) {
        T dL, dR;
        T fL = pressure_branch(g, p, rL, pL, cL, &dL);
        T fR = pressure_branch(g, p, rR, pR, cR, &dR);
        T pn = p - (fL + fR + uR - uL) / (dL + dR);
        if (val(pn) <= 0.0) pn = T(0.5 * val(p));
        T step = pn - p;
        p = pn;
        if (std::fabs(val(step)) <= 1e-15 * val(p)) break;
    }
    T dL, dR;
    T fL = pressure_branch(g, p, rL, pL, cL, &dL);
    T fR = pressure_branch(g, p, rR, pR, cR, &dR);
    T us = 0.5 * (uL + uR) + 0.5 * (fR - fL);
    const double gr = (g - 1.0) / (g + 1.0);
    *left_of_contact = val(us) >= 0.0;
    if (*left_of_contact) {
        if (val(p) > val(pL)) {   // left shock, speed S_L
            T SL = uL - cL * sqrt_((g + 1.0) / (2.0 * g) * p / pL + (g - 1.0) / (2.0 * g));
            if (val(SL) >= 0.0) { *r0 = rL; *u0 = uL; *p0 = pL; return; }
            *r0 = rL * (p / pL + gr) / (gr * p / pL + 1.0); *u0 = us; *p0 = p; return;
        }
        T head = uL - cL;         // left rarefaction
        if (val(head) >= 0.0) { *r0 = rL; *u0 = uL; *p0 = pL; return; }
        T tail = us - cL * pow_(T(p / pL), (g - 1.0) / (2.0 * g));
        if (val(tail) < 0.0) { *r0 = rL * pow_(T(p / pL), 1.0 / g); *u0 = us; *p0 = p; return; }
        T c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL);   // inside the fan at x/t = 0
        *u0 = c;
        *r0 = rL * pow_(T(c / cL), 2.0 / (g - 1.0));
        *p0 = pL * pow_(T(c / cL), 2.0 * g / (g - 1.0));
        return;
    }
    if (val(p) > val(pR)) {       // right shock
        T SR = uR + cR * sqrt_((g + 1.0) / (2.0 * g) * p / pR + (g - 1.0) / (2.0 * g));
        if (val(SR) <= 0.0) { *r0 = rR; *u0 = uR; *p0 = pR; return; }
        *r0 = rR * (p / pR + gr) / (gr * p / pR + 1.0); *u0 = us; *p0 = p; return;
    }
    T head = uR + cR;             // right rarefaction
    if (val(head) <= 0.0) { *r0 = rR; *u0 = uR; *p0 = pR; return; }
    T tail = us + cR * pow_(T(p / pR), (g - 1.0) / (2.0 * g));
    if (val(tail) > 0.0) { *r0 = rR * pow_(T(p / pR), 1.0 / g); *u0 = us; *p0 = p; return; }
    T c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * uR);
    *u0 = -c;
    *r0 = rR * pow_(T(c / cR), 2.0 / (g - 1.0));
    *p0 = pR * pow_(T(c / cR), 2.0 * g / (g - 1.0));
}
template <class T> void godunov_flux_euler(const Desc& d, int k, const T* WL, const T* WR, T* F) {
    const int nd = d.ndim, ip = nd + 1;
    T r0, u0, p0;
    bool left;
    godunov_state_euler(d.gamma, WL[0], WL[1 + k], WL[ip], WR[0], WR[1 + k], WR[ip], &r0, &u0, &p0, &left);
    T W[8];
    const T* side = left ? WL : WR;
    for (int j = 0; j < nd; ++j) W[1 + j] = side[1 + j];
    W[0] = r0;
    W[1 + k] = u0;
    W[ip] = p0;
    euler_phys_flux(d, W, k, F);
}

// Logarithmic mean (a - b)/(ln a - ln b) of two positive numbers; for nearly equal arguments from
// ln(a/b) = 2 artanh(f), f = (a - b)/(a + b): (a + b) / (2 artanh(f)/f) with the series
// artanh(f)/f = 1 + f^2/3 + f^4/5 + f^6/7 + f^8/9 when f^2 < 1e-4 (Ismail-Roe's device, more terms).
template <class T> inline T log_mean(const T& a, const T& b) {
    T f = (a - b) / (a + b);
    T u = f * f;
    if (val(u) < 1e-4) {
        T s = 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0 + u * (1.0 / 9.0))));
        return (a + b) / (2.0 * s);
    }
    return (a - b) / log_(T(a / b));
}

// Two-point entropy-conservative flux (Sec. 2.1 cites LeFloch-Mercier-Rohde's entropy-conservative
// schemes, built from two-point fluxes that satisfy Tadmor's condition
// (v_R - v_L) . F = psi_R - psi_L for an entropy pair). Euler: Ismail-Roe's flux for the entropy
// -rho s/(gamma - 1), s = ln(p rho^-gamma), from z = sqrt(rho/p) (1, u, p):
// rho^ = z1_mean z3_ln, u^ = zu_mean / z1_mean, p1^ = z3_mean / z1_mean,
// p2^ = (gamma+1)/(2 gamma) z3_ln / z1_ln + (gamma-1)/(2 gamma) z3_mean / z1_mean,
// H^ = gamma p2^ / ((gamma-1) rho^) + |u^|^2/2; F = (rho^ u^_k, rho^ u^_k u^ + p1^ e_k, rho^ u^_k H^).
// Burgers: the flux (u_L^2 + u_L u_R + u_R^2)/6 of the square entropy u^2/2.
template <class T> void ec_flux(const Desc& d, int k, const T* WL, const T* WR, T* F) {
    if (d.eq == EQ_BURGERS) {
        F[0] = (WL[0] * WL[0] + WL[0] * WR[0] + WR[0] * WR[0]) / 6.0;
        return;
    }
    const int nd = d.ndim, ip = nd + 1;
    const double g = d.gamma;
    T z1L = sqrt_(WL[0] / WL[ip]), z1R = sqrt_(WR[0] / WR[ip]);
    T z3L = sqrt_(WL[0] * WL[ip]), z3R = sqrt_(WR[0] * WR[ip]);
    T z1m = 0.5 * (z1L + z1R), z3m = 0.5 * (z3L + z3R);
    T z1l = log_mean(z1L, z1R), z3l = log_mean(z3L, z3R);
    T rho = z1m * z3l;
    T u[8];
    T q2 = T(0.0);
    for (int j = 0; j < nd; ++j) {
        u[j] = 0.5 * (z1L * WL[1 + j] + z1R * WR[1 + j]) / z1m;
        q2 = q2 + u[j] * u[j];
    }
    T p1 = z3m / z1m;
    T p2 = (g + 1.0) / (2.0 * g) * z3l / z1l + (g - 1.0) / (2.0 * g) * z3m / z1m;
    T H = g * p2 / ((g - 1.0) * rho) + 0.5 * q2;
    T mf = rho * u[k];
    F[0] = mf;
    for (int j = 0; j < nd; ++j) F[1 + j] = mf * u[j];
    F[1 + k] = F[1 + k] + p1;
    F[ip] = mf * H;
}

// Entropy variables v = dU/du of the entropy used by the entropy-conservative fluxes. Euler: U =
// -rho s/(gamma - 1), s = ln p - gamma ln rho, so v = ((gamma - s)/(gamma - 1) - rho |u|^2/(2p),
// rho u/p, -rho/p); Burgers: U = u^2/2, v = u. W is the primitive state.
template <class T> void entropy_vars(const Desc& d, const T* W, T* v) {
    if (d.eq == EQ_BURGERS) {
        v[0] = W[0];
        return;
    }
    const int nd = d.ndim, ip = nd + 1;
    const double g = d.gamma;
    T s = log_(W[ip]) - g * log_(W[0]);
    T beta = W[0] / W[ip];
    T q2 = T(0.0);
    for (int j = 0; j < nd; ++j) q2 = q2 + W[1 + j] * W[1 + j];
    v[0] = (g - s) / (g - 1.0) - 0.5 * beta * q2;
    for (int j = 0; j < nd; ++j) v[1 + j] = beta * W[1 + j];
    v[ip] = -beta;
}

// Eigenvectors of the Euler flux Jacobian along k, scaled so that Rs Rs^T = dU/dv (Barth's
// scaling), and the absolute eigenvalues, at the state with the arithmetic means of WL and WR's
// density, velocity and pressure. Columns: the u_k - c acoustic wave, the entropy wave, one shear
// wave per tangential direction (in increasing order), the u_k + c acoustic wave. Rs[row][col].
template <class T> void tecno_matrix(const Desc& d, int k, const T* WL, const T* WR, T Rs[8][8], T* lam) {
    const int nd = d.ndim, ip = nd + 1, nv = nd + 2;
    const double g = d.gamma;
    T r = 0.5 * (WL[0] + WR[0]), p = 0.5 * (WL[ip] + WR[ip]);
    T u[3];
    T q2 = T(0.0);
    for (int j = 0; j < nd; ++j) {
        u[j] = 0.5 * (WL[1 + j] + WR[1 + j]);
        q2 = q2 + u[j] * u[j];
    }
    T c = sqrt_(g * p / r);
    T H = c * c / (g - 1.0) + 0.5 * q2;
    T un = u[k];
    T sac = sqrt_(r / (2.0 * g)), sen = sqrt_((g - 1.0) * r / g), ssh = sqrt_(p);
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) Rs[a][b] = T(0.0);
    // acoustic waves u_k -/+ c: (1, u -/+ c e_k, H -/+ u_k c)
    for (int side = 0; side < 2; ++side) {
        const int col = side == 0 ? 0 : nv - 1;
        const double sg = side == 0 ? -1.0 : 1.0;
        Rs[0][col] = sac;
        for (int j = 0; j < nd; ++j) Rs[1 + j][col] = sac * u[j];
        Rs[1 + k][col] = sac * (un + sg * c);
        Rs[ip][col] = sac * (H + sg * un * c);
        lam[col] = abs_(T(un + sg * c));
    }
    // entropy wave: (1, u, |u|^2/2)
    Rs[0][1] = sen;
    for (int j = 0; j < nd; ++j) Rs[1 + j][1] = sen * u[j];
    Rs[ip][1] = sen * 0.5 * q2;
    lam[1] = abs_(un);
    // shear waves: (0, e_t, u_t)
    int col = 2;
    for (int t = 0; t < nd; ++t) {
        if (t == k) continue;
        Rs[1 + t][col] = ssh;
        Rs[ip][col] = ssh * u[t];
        lam[col] = abs_(un);
        ++col;
    }
}

// TECNO2 (Fjordholm-Mishra-Tadmor's entropy-stable ENO scheme, second order): the two-point
// entropy-conservative flux of the interface's cells plus an entropy-stable diffusion,
//   F = F_ec(W_i, W_{i+1}) - 1/2 Rs Lambda <<w>>,
// with w_j = Rs^T v_j the scaled entropy variables of the cells i-1 .. i+2 (Rs, Lambda at the
// interface, v_j the entropy variables) and <<w>> = w_{i+1}^- - w_i^+ the jump of their
// second-order ENO reconstructions at the interface (per component, the one-sided difference of
// smaller magnitude, ties taking the backward one). ENO's sign property makes <<w>> carry the sign
// of w_{i+1} - w_i per component, so each interface produces entropy -1/2 [[w]]^T Lambda <<w>> <= 0.
// Burgers: v = u, Rs = 1, Lambda = max(|u_i|, |u_{i+1}|) (a Roe speed would vanish on a
// transonic rarefaction and keep an expansion shock).
template <class T> void tecno_flux(const Desc& d, int k, T W[4][8], T* F) {
    const int nv = nvars(d);
    ec_flux(d, k, W[1], W[2], F);
    T Rs[8][8], lam[8], v[4][8], w[4][8];
    if (d.eq == EQ_BURGERS) {
        Rs[0][0] = T(1.0);
        lam[0] = max_(abs_(W[1][0]), abs_(W[2][0]));
    } else {
        tecno_matrix(d, k, W[1], W[2], Rs, lam);
    }
    for (int j = 0; j < 4; ++j) {
        entropy_vars(d, W[j], v[j]);
        for (int m = 0; m < nv; ++m) {
            T acc = T(0.0);
            for (int r = 0; r < nv; ++r) acc = acc + Rs[r][m] * v[j][r];
            w[j][m] = acc;
        }
    }
    T jump[8];
    for (int m = 0; m < nv; ++m) {
        T dm = w[1][m] - w[0][m], d1 = w[2][m] - w[1][m], d2 = w[3][m] - w[2][m];
        T si = val(abs_(d1)) < val(abs_(dm)) ? d1 : dm;   // cell i, right face
        T sj = val(abs_(d2)) < val(abs_(d1)) ? d2 : d1;   // cell i + 1, left face
        jump[m] = (w[2][m] - 0.5 * sj) - (w[1][m] + 0.5 * si);
    }
    for (int r = 0; r < nv; ++r) {
        T acc = T(0.0);
        for (int m = 0; m < nv; ++m) acc = acc + Rs[r][m] * (lam[m] * jump[m]);
        F[r] = F[r] - 0.5 * acc;
    }
}

template <class T> void flux(const Desc& d, int k, const T* WL, const T* WR, T* F) {
    const int nv = nvars(d);
    if (d.flux == FLUX_EC || d.flux == FLUX_EC4 || d.flux == FLUX_TECNO2) { ec_flux(d, k, WL, WR, F); return; }
    if (d.eq == EQ_BURGERS) {
        T uL = WL[0], uR = WR[0];
        T fL = 0.5 * uL * uL, fR = 0.5 * uR * uR;
        if (d.flux == FLUX_ROE) {
            // Roe speed (u_L + u_R)/2 with Harten's fix of width max(0, a - u_L, u_R - a)
            T a = 0.5 * (uL + uR);
            F[0] = 0.5 * (fL + fR) - 0.5 * harten_abs(a, uL, uR) * (uR - uL);
            return;
        }
        if (d.flux == FLUX_GODUNOV) {
            // exact Riemann solution at x/t = 0: shock (u_L > u_R) moving with (u_L + u_R)/2, or
            // rarefaction (u_L <= u_R), whose fan holds u = 0 when it straddles x/t = 0
            if (val(uL) > val(uR)) F[0] = val(uL + uR) >= 0.0 ? fL : fR;
            else if (val(uL) >= 0.0) F[0] = fL;
            else if (val(uR) <= 0.0) F[0] = fR;
            else F[0] = T(0.0);
            return;
        }
        if (d.flux == FLUX_RUSANOV) {
            T a = max_(abs_(uL), abs_(uR));
            F[0] = 0.5 * (fL + fR) - 0.5 * a * (uR - uL);
        } else {  // HLL; for a scalar law HLLC coincides with HLL
            T SL = min_(uL, uR), SR = max_(uL, uR);
            if (val(SL) >= 0.0) F[0] = fL;
            else if (val(SR) <= 0.0) F[0] = fR;
            else F[0] = (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL);
        }
        return;
    }
    if (d.flux == FLUX_ROE) { roe_flux_euler(d, k, WL, WR, F); return; }
    if (d.flux == FLUX_GODUNOV) { godunov_flux_euler(d, k, WL, WR, F); return; }
    const int nd = d.ndim;
    const int ip = nd + 1;
    T UL[8], UR[8], FL[8], FR[8];
    prim_to_cons(d, WL, UL);
    prim_to_cons(d, WR, UR);
    euler_phys_flux(d, WL, k, FL);
    euler_phys_flux(d, WR, k, FR);
    T rL = WL[0], rR = WR[0], uL = WL[1 + k], uR = WR[1 + k], pL = WL[ip], pR = WR[ip];
    T cL = sqrt_(d.gamma * pL / rL);
    T cR = sqrt_(d.gamma * pR / rR);
    if (d.flux == FLUX_RUSANOV) {
        T a = max_(T(abs_(uL) + cL), T(abs_(uR) + cR));
        for (int v = 0; v < nv; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * a * (UR[v] - UL[v]);
        return;
    }
    T SL = min_(T(uL - cL), T(uR - cR));
    T SR = max_(T(uL + cL), T(uR + cR));
    if (d.flux == FLUX_HLL) {
        if (val(SL) >= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; }
        else if (val(SR) <= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; }
        else {
            for (int v = 0; v < nv; ++v)
                F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
        }
        return;
    }
    // HLLC (Toro-Spruce-Speares) with the contact speed S* and star states U*_K. Cases in order:
    // F_L if 0 <= S_L; F*_L if S_L < 0 <= S*; F*_R if S* < 0 < S_R; F_R otherwise.
    if (val(SL) >= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; return; }
    T Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    const bool left = val(Ss) >= 0.0;
    if (!left && !(val(SR) > 0.0)) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; return; }
    const T* WK = left ? WL : WR;
    const T* UK = left ? UL : UR;
    const T* FK = left ? FL : FR;
    T SK = left ? SL : SR;
    T rK = WK[0], uK = WK[1 + k], pK = WK[ip];
    T fac = rK * (SK - uK) / (SK - Ss);
    T Us[8];
    Us[0] = fac;
    for (int j = 0; j < nd; ++j) Us[1 + j] = fac * WK[1 + j];
    Us[1 + k] = fac * Ss;
    Us[ip] = fac * (UK[ip] / rK + (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
    for (int v = 0; v < nv; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

// Flux through the interface i+1/2 (between cell i and i+1) along k at cell position c.
template <class T> void interface_flux(const Desc& d, const T* U, const int c[3], int k, int i, T* F) {
    if (d.flux == FLUX_EC || d.flux == FLUX_EC4 || d.flux == FLUX_TECNO2) {
        // entropy-conservative fluxes (and TECNO2) take the cell values (primitive), no reconstruction
        const int nv = nvars(d);
        T W[4][8];
        for (int s = 0; s < 4; ++s) {
            if (d.flux == FLUX_EC && (s == 0 || s == 3)) continue;
            T Uc[8];
            cell_cons(d, U, c, k, i - 1 + s, Uc);
            if (d.eq == EQ_BURGERS) W[s][0] = Uc[0];
            else cons_to_prim(d, Uc, W[s]);
        }
        if (d.flux == FLUX_EC) { ec_flux(d, k, W[1], W[2], F); return; }
        if (d.flux == FLUX_TECNO2) { tecno_flux(d, k, W, F); return; }
        // fourth order (LeFloch-Mercier-Rohde): 4/3 F(w_i, w_{i+1}) - 1/6 (F(w_{i-1}, w_{i+1}) + F(w_i, w_{i+2}))
        T Fa[8], Fb[8], Fc[8];
        ec_flux(d, k, W[1], W[2], Fa);
        ec_flux(d, k, W[0], W[2], Fb);
        ec_flux(d, k, W[1], W[3], Fc);
        for (int v = 0; v < nv; ++v) F[v] = (4.0 / 3.0) * Fa[v] - (1.0 / 6.0) * (Fb[v] + Fc[v]);
        return;
    }
    T Wl_i[8], Wr_i[8], Wl_j[8], Wr_j[8];
    cell_faces(d, U, c, k, i, Wl_i, Wr_i);
    cell_faces(d, U, c, k, i + 1, Wl_j, Wr_j);
    flux(d, k, Wr_i, Wl_j, F);
}

// ------------------------------------------------------------------------------------------
// eq. (2.1): L(U)_i = -sum_k (F_{i+1/2 e_k} - F_{i-1/2 e_k}) / dx_k, directions in order x,y,z.
// ------------------------------------------------------------------------------------------
template <class T> void rhs(const Desc& d, const T* U, T* L) {
    const int nv = nvars(d);
    const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c[3] = {x, y, z};
                T acc[8];
                for (int v = 0; v < nv; ++v) acc[v] = T(0.0);
                for (int k = 0; k < d.ndim; ++k) {
                    T Fm[8], Fp[8];
                    interface_flux(d, U, c, k, c[k] - 1, Fm);
                    interface_flux(d, U, c, k, c[k], Fp);
                    double h = dx(d, k);
                    for (int v = 0; v < nv; ++v) acc[v] = acc[v] - (Fp[v] - Fm[v]) / h;
                }
                for (int v = 0; v < nv; ++v) L[lin(d, v, x, y, z)] = acc[v];
            }
}

// ------------------------------------------------------------------------------------------
// SSP Runge-Kutta (Gottlieb-Shu-Tadmor), Sec. 2.1:
//   RK2: U1 = U + dt L(U);  U^{n+1} = 1/2 U + 1/2 (U1 + dt L(U1))
//   RK3: U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));  U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2))
// ------------------------------------------------------------------------------------------
template <class T> void rk_step(const Desc& d, T* U, T dt) {
    const int64_t N = (int64_t)nvars(d) * ncells(d);
    std::vector<T> L(N), U1(N), U2(N);
    rhs(d, U, L.data());
    for (int64_t q = 0; q < N; ++q) U1[q] = U[q] + dt * L[q];
    rhs(d, U1.data(), L.data());
    if (d.rk == RK_SSP2) {
        for (int64_t q = 0; q < N; ++q) U[q] = 0.5 * U[q] + 0.5 * (U1[q] + dt * L[q]);
        return;
    }
    for (int64_t q = 0; q < N; ++q) U2[q] = 0.75 * U[q] + 0.25 * (U1[q] + dt * L[q]);
    rhs(d, U2.data(), L.data());
    const double third = 1.0 / 3.0, two_third = 2.0 / 3.0;
    for (int64_t q = 0; q < N; ++q) U[q] = third * U[q] + two_third * (U2[q] + dt * L[q]);
}

// CFL reading: s = max over cells and directions of (|u_k| + c)/dx_k (Burgers: |u|/dx_k).
// Returns NaN if a cell is non-physical (rho <= 0 or p <= 0) or non-finite.
double max_speed(const Desc& d, const double* U) {
    const int nv = nvars(d);
    double s = 0.0;
    bool bad = false;
    for (int z = 0; z < d.n[2]; ++z)
        for (int y = 0; y < d.n[1]; ++y)
            for (int x = 0; x < d.n[0]; ++x) {
                double Uc[8], W[8];
                for (int v = 0; v < nv; ++v) Uc[v] = U[lin(d, v, x, y, z)];
                if (d.eq == EQ_BURGERS) {
                    if (!std::isfinite(Uc[0])) bad = true;
                    for (int k = 0; k < d.ndim; ++k) s = std::max(s, std::fabs(Uc[0]) / dx(d, k));
                    continue;
                }
                cons_to_prim(d, Uc, W);
                double rho = W[0], p = W[d.ndim + 1];
                if (!(rho > 0.0 && p > 0.0) || !std::isfinite(rho) || !std::isfinite(p)) { bad = true; continue; }
                double c = std::sqrt(d.gamma * p / rho);
                for (int k = 0; k < d.ndim; ++k) s = std::max(s, (std::fabs(W[1 + k]) + c) / dx(d, k));
            }
    return bad ? NAN : s;
}

// ------------------------------------------------------------------------------------------
// Initial data. Cell values are cell averages of conserved variables.
// ------------------------------------------------------------------------------------------
// Kelvin-Helmholtz (Sec. 3 defers to Fjordholm-Kappeli-Mishra-Tadmor; reading):
//   2D: inner band (rho=2, u=-0.5) between y = 0.25 + Y(x) and y = 0.75 + Y(x), outer rho=1,
//   u=0.5, v=0, p=2.5; Y(x) = 0.01 sum_{n=1}^{10} a_n sin(2 pi n x + b_n), theta = [a_1..a_10,
//   b_1..b_10]. The cell value blends the two states in conserved variables by the fraction of
//   the cell (in y, interfaces evaluated at the cell-centre x) that lies inside the band.
//   3D slab: the same in (x,z) with Y(x,z) = 0.01 sum_{n,m=1}^{8} a_nm sin(2 pi (n x + m z) + b_nm),
//   theta = [a (n-major, 64), b (64)], momentum along x, v = w = 0.
template <class T> inline T clamp01(const T& x) {
    if (val(x) < 0.0) return T(0.0);
    if (val(x) > 1.0) return T(1.0);
    return x;
}

template <class T> void init_kh(const Desc& d, const T* theta, T* U) {
    const double PI = 3.14159265358979323846;
    const int nd = d.ndim;
    double Win[8] = {0}, Wout[8] = {0};
    Win[0] = 2.0; Win[1] = -0.5; Win[nd + 1] = 2.5;
    Wout[0] = 1.0; Wout[1] = 0.5; Wout[nd + 1] = 2.5;
    double Uin[8], Uout[8];
    prim_to_cons(d, Win, Uin);
    prim_to_cons(d, Wout, Uout);
    const double hx = dx(d, 0), hy = dx(d, 1), hz = nd == 3 ? dx(d, 2) : 0.0;
    for (int z = 0; z < d.n[2]; ++z)
        for (int x = 0; x < d.n[0]; ++x) {
            double xc = d.lo[0] + (x + 0.5) * hx;
            T Y = T(0.0);
            if (nd == 2) {
                for (int n = 1; n <= 10; ++n) Y = Y + theta[n - 1] * sin_(2.0 * PI * n * xc + theta[10 + n - 1]);
            } else {
                double zc = d.lo[2] + (z + 0.5) * hz;
                for (int n = 1; n <= 8; ++n)
                    for (int m = 1; m <= 8; ++m) {
                        int j = (n - 1) * 8 + (m - 1);
                        Y = Y + theta[j] * sin_(2.0 * PI * (n * xc + m * zc) + theta[64 + j]);
                    }
            }
            Y = 0.01 * Y;
            for (int y = 0; y < d.n[1]; ++y) {
                double ylo = d.lo[1] + y * hy;
                T f_lo = clamp01(T((0.25 + Y - ylo) / hy));  // fraction of the cell below interface 1
                T f_hi = clamp01(T((0.75 + Y - ylo) / hy));  // fraction of the cell below interface 2
                T f = f_hi - f_lo;                           // fraction inside the band
                for (int v = 0; v < nvars(d); ++v) U[lin(d, v, x, y, z)] = f * Uin[v] + (1.0 - f) * Uout[v];
            }
        }
}

// Two-state shock tube split at x = 0.5 (exact volume fraction when a cell straddles it).
void init_tube(const Desc& d, const double* WLp, const double* WRp, double* U) {
    double UL[8], UR[8];
    prim_to_cons(d, WLp, UL);
    prim_to_cons(d, WRp, UR);
    const double h = dx(d, 0);
    for (int z = 0; z < d.n[2]; ++z)
        for (int y = 0; y < d.n[1]; ++y)
            for (int x = 0; x < d.n[0]; ++x) {
                double xl = d.lo[0] + x * h;
                double f = std::min(1.0, std::max(0.0, (0.5 - xl) / h));  // left-state fraction
                for (int v = 0; v < nvars(d); ++v) U[lin(d, v, x, y, z)] = f * UL[v] + (1.0 - f) * UR[v];
            }
}

// Burgers u0 = sin(2 pi x): exact cell averages (cos(2 pi x_l) - cos(2 pi x_r)) / (2 pi dx).
void init_burgers_sine(const Desc& d, double* U) {
    const double PI = 3.14159265358979323846;
    const double h = dx(d, 0);
    for (int z = 0; z < d.n[2]; ++z)
        for (int y = 0; y < d.n[1]; ++y)
            for (int x = 0; x < d.n[0]; ++x) {
                double xl = d.lo[0] + x * h, xr = xl + h;
                U[lin(d, 0, x, y, z)] = (std::cos(2.0 * PI * xl) - std::cos(2.0 * PI * xr)) / (2.0 * PI * h);
            }
}

// Isentropic vortex (Shu's standard test): ambient (rho,u,v,p) = (1,1,1,1), strength beta = 5,
// centre (xc, yc); perturbations du = -beta/(2pi) e^{(1-r^2)/2} (y-yc), dv = beta/(2pi) e^{(1-r^2)/2}
// (x-xc), dT = -(gamma-1) beta^2/(8 gamma pi^2) e^{1-r^2}; T = 1 + dT, rho = T^{1/(gamma-1)},
// p = rho T. Cell averages of conserved variables by 5x5 Gauss-Legendre quadrature.
void vortex_point(double g, double xc, double yc, double x, double y, double* Uc) {
    const double PI = 3.14159265358979323846, beta = 5.0;
    double rx = x - xc, ry = y - yc, r2 = rx * rx + ry * ry;
    double e = std::exp(0.5 * (1.0 - r2));
    double u = 1.0 - beta / (2.0 * PI) * e * ry;
    double v = 1.0 + beta / (2.0 * PI) * e * rx;
    double Tm = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * PI * PI) * e * e;
    double rho = std::pow(Tm, 1.0 / (g - 1.0));
    double p = rho * Tm;
    Uc[0] = rho;
    Uc[1] = rho * u;
    Uc[2] = rho * v;
    Uc[3] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
}

void init_vortex(const Desc& d, double xc, double yc, double* U) {
    // 5-point Gauss-Legendre nodes/weights on [-1,1]
    const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831, 0.9061798459386640};
    const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                          0.2369268850561891};
    const double hx = dx(d, 0), hy = dx(d, 1);
    for (int y = 0; y < d.n[1]; ++y)
        for (int x = 0; x < d.n[0]; ++x) {
            double acc[4] = {0, 0, 0, 0};
            double cx = d.lo[0] + (x + 0.5) * hx, cy = d.lo[1] + (y + 0.5) * hy;
            for (int a = 0; a < 5; ++a)
                for (int b = 0; b < 5; ++b) {
                    double Uc[4];
                    vortex_point(d.gamma, xc, yc, cx + 0.5 * hx * gx[a], cy + 0.5 * hy * gx[b], Uc);
                    for (int v = 0; v < 4; ++v) acc[v] += 0.25 * gw[a] * gw[b] * Uc[v];
                }
            for (int v = 0; v < 4; ++v) U[lin(d, v, x, y, 0)] = acc[v];
        }
}

// ------------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based generator for KH parameters:
//   theta_{b,j} = lo_j + (hi_j - lo_j) * (splitmix64(seed XOR (b*P + j)) >> 11) * 2^-53,
//   splitmix64(x) = mix(x + 0x9E3779B97F4A7C15) with the published finaliser.
// ------------------------------------------------------------------------------------------
inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace orc

using namespace orc;

// ==========================================================================================
// ctypes interface. All arrays are host FP64, layout [sample][var][z][y][x], x fastest.
// Return codes: 0 ok, 1 invalid argument, 3 non-physical state / non-finite wave speed.
// ==========================================================================================
extern "C" {

int orc_num_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_nvars(const Desc* d) { return nvars(*d); }

// One numerical flux on primitive states (for unit pins).
void orc_flux(const Desc* d, int k, const double* WL, const double* WR, double* F) { flux(*d, k, WL, WR, F); }

// TECNO2 pieces (tests): entropy variables of a primitive state; the scaled eigenvectors (row-major
// nv x nv) and absolute eigenvalues at the mean of two states; the flux of four consecutive cells'
// primitive states W4[4][nv].
void orc_entropy_vars(const Desc* d, const double* W, double* v) { entropy_vars(*d, W, v); }
void orc_tecno_matrix(const Desc* d, int k, const double* WL, const double* WR, double* Rs, double* lam) {
    double R8[8][8];
    tecno_matrix(*d, k, WL, WR, R8, lam);
    const int nv = nvars(*d);
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) Rs[a * nv + b] = R8[a][b];
}
void orc_tecno_flux(const Desc* d, int k, const double* W4, double* F) {
    const int nv = nvars(*d);
    double W[4][8];
    for (int j = 0; j < 4; ++j)
        for (int v = 0; v < nv; ++v) W[j][v] = W4[j * nv + v];
    tecno_flux(*d, k, W, F);
}

// Reconstruction of a single cell's faces from three scalars.
void orc_recon(int recon, double eps, double wm, double w0, double wp, double* fl, double* fr) {
    recon_scalar(recon, eps, wm, w0, wp, fl, fr);
}

void orc_cons_to_prim(const Desc* d, const double* U, double* W) { cons_to_prim(*d, U, W); }
// The two face states (primitive; Burgers: u) of cell (cx, cy, cz) along direction k of one sample
// U, after reconstruction and the positivity fallback: what every interface flux of the scheme
// receives from that cell.
void orc_face_states(const Desc* d, const double* U, int cx, int cy, int cz, int k, double* Wl, double* Wr) {
    const int c[3] = {cx, cy, cz};
    cell_faces(*d, U, c, k, c[k], Wl, Wr);
}
void orc_prim_to_cons(const Desc* d, const double* W, double* U) { prim_to_cons(*d, W, U); }

// L(U) for B samples.
void orc_rhs(const Desc* d, int B, const double* U, double* L) {
    const int64_t S = (int64_t)nvars(*d) * ncells(*d);
    for (int b = 0; b < B; ++b) rhs(*d, U + b * S, L + b * S);
}

// Maximum CFL wave speed of each sample (NaN if non-physical).
void orc_max_speed(const Desc* d, int B, const double* U, double* s) {
    const int64_t S = (int64_t)nvars(*d) * ncells(*d);
    for (int b = 0; b < B; ++b) s[b] = max_speed(*d, U + b * S);
}

// Advance B samples in place.
//   fixed_dt > 0: exactly n_steps steps of fixed_dt (T ignored).
//   fixed_dt == 0: CFL steps dt = cfl / s until t = T (last step clipped to land on T), at most
//                  max_steps steps (max_steps <= 0: unlimited).
// steps[b], t[b] receive the step count and final time.
int orc_evolve(const Desc* d, int B, double* U, double T, double fixed_dt, int64_t n_steps, int64_t max_steps,
               int64_t* steps, double* t_out) {
    const int64_t S = (int64_t)nvars(*d) * ncells(*d);
    int status = 0;
    for (int b = 0; b < B; ++b) {
        double* Ub = U + b * S;
        double t = 0.0;
        int64_t k = 0;
        if (fixed_dt > 0.0) {
            for (k = 0; k < n_steps; ++k) rk_step(*d, Ub, fixed_dt);
            t = fixed_dt * (double)n_steps;
        } else {
            while (t < T && (max_steps <= 0 || k < max_steps)) {
                double s = max_speed(*d, Ub);
                if (!std::isfinite(s)) { status = 3; break; }
                double dt = d->cfl / s;
                bool last = false;
                if (!(dt < T - t)) { dt = T - t; last = true; }
                rk_step(*d, Ub, dt);
                t = last ? T : t + dt;
                ++k;
            }
        }
        if (steps) steps[b] = k;
        if (t_out) t_out[b] = t;
    }
    return status;
}

// KH parameters from SplitMix64: B x P, amplitudes U(0,1) for j < P/2, phases U(0, 2 pi) after.
void orc_theta(uint64_t seed, int B, int P, double* theta) {
    const double PI = 3.14159265358979323846;
    for (int b = 0; b < B; ++b)
        for (int j = 0; j < P; ++j) {
            uint64_t r = splitmix64(seed ^ ((uint64_t)b * (uint64_t)P + (uint64_t)j));
            double u01 = (double)(r >> 11) * (1.0 / 9007199254740992.0);
            double hi = j < P / 2 ? 1.0 : 2.0 * PI;
            theta[(int64_t)b * P + j] = 0.0 + (hi - 0.0) * u01;
        }
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

// Initial data for B samples; theta is B x P (KH only). Vortex: centre (param0, param1).
int orc_init(const Desc* d, int kind, int B, const double* theta, int P, double param0, double param1, double* U) {
    const int64_t S = (int64_t)nvars(*d) * ncells(*d);
    for (int b = 0; b < B; ++b) {
        double* Ub = U + b * S;
        if (kind == INIT_KH) {
            if (d->eq != EQ_EULER || d->ndim < 2) return 1;
            init_kh(*d, theta + (int64_t)b * P, Ub);
        } else if (kind == INIT_SOD || kind == INIT_LAX) {
            if (d->eq != EQ_EULER) return 1;
            double WL[8] = {0}, WR[8] = {0};
            int ip = d->ndim + 1;
            if (kind == INIT_SOD) { WL[0] = 1.0; WL[ip] = 1.0; WR[0] = 0.125; WR[ip] = 0.1; }
            else { WL[0] = 0.445; WL[1] = 0.698; WL[ip] = 3.528; WR[0] = 0.5; WR[ip] = 0.571; }
            init_tube(*d, WL, WR, Ub);
        } else if (kind == INIT_BURGERS_SINE) {
            if (d->eq != EQ_BURGERS) return 1;
            init_burgers_sine(*d, Ub);
        } else if (kind == INIT_VORTEX) {
            if (d->eq != EQ_EULER || d->ndim != 2) return 1;
            init_vortex(*d, param0, param1, Ub);
        } else {
            return 1;
        }
    }
    return 0;
}

// Welford update of per-cell mean/M2 of the primitive quantities (Burgers: u; Euler: rho,
// velocities, p) over B samples in ascending order (Sec. 2.2: mean and variance on device).
// count is shared by all cells; mean, M2 are [q][cells].
// Algorithmic floating-point operations of the scheme of d, counted by running its pieces on the
// counting scalar with a representative smooth, subsonic pair of states (MC central slope, HLLC
// left star state): out = {reconstruction of one variable (both faces of a cell), cons->prim of a
// cell, one interface flux, divergence + RK combination of one cell and stage, per cell-stage,
// per cell-update}. A cell-stage takes its cell's conversion (primitive reconstruction) and per
// direction one cell's reconstruction and one interface flux (each interface belongs to one cell).
void orc_count_flops(const Desc* d, double* out) {
    const int nv = nvars(*d), nd = d->ndim;
    const bool euler = d->eq != EQ_BURGERS;
    Cnt wm(1.0), w0(1.1), wp(1.3), fl, fr;
    g_flops = 0;
    recon_scalar(d->recon, d->weno_eps_dx2 ? 1e-4 : d->weno_eps, wm, w0, wp, &fl, &fr);
    const double f_rec = (double)g_flops;
    Cnt U[8], W[8];
    const double Wl0[5] = {1.0, 0.3, 0.1, 0.05, 2.5}, Wr0[5] = {1.1, 0.25, 0.05, 0.0, 2.4};
    Cnt WL[8], WR[8], F[8];
    for (int v = 0; v < nv; ++v) {
        const int src = v <= nd ? v : 4;      // rho, velocities of the active directions, p
        WL[v] = Cnt(euler ? Wl0[src] : 0.3);
        WR[v] = Cnt(euler ? Wr0[src] : 0.25);
    }
    double f_c2p = 0.0;
    if (euler) {
        prim_to_cons(*d, WL, U);
        g_flops = 0;
        cons_to_prim(*d, U, W);
        f_c2p = (double)g_flops;
    }
    g_flops = 0;
    flux(*d, 0, WL, WR, F);
    const double f_flux = (double)g_flops;
    // divergence over the directions and the RK combination averaged over the stages
    g_flops = 0;
    Cnt acc(0.0), Fm(0.1), Fp(0.2), dt(1e-3), us(1.0), un(1.0);
    for (int k = 0; k < nd; ++k) acc = acc - (Fp - Fm) / dx(*d, k);
    const double f_div = (double)g_flops * nv;
    g_flops = 0;
    Cnt o1 = us + dt * acc;
    Cnt o2 = 0.75 * un + 0.25 * (us + dt * acc);
    Cnt o3 = (1.0 / 3.0) * un + (2.0 / 3.0) * (us + dt * acc);
    (void)o1; (void)o2; (void)o3;
    const int stages = d->rk == RK_SSP2 ? 2 : 3;
    const double f_rk = (stages == 2 ? (2.0 + 5.0) / 2.0 : (double)g_flops / 3.0) * nv;
    double per_stage = nd * (nv * f_rec + f_flux) + f_div + f_rk;
    if (euler && d->rvars == RV_PRIM) per_stage += f_c2p;          // each cell converted once
    if (euler && d->rvars == RV_CONS) per_stage += nd * 2 * f_c2p; // both faces converted
    out[0] = f_rec;
    out[1] = f_c2p;
    out[2] = f_flux;
    out[3] = f_div + f_rk;
    out[4] = per_stage;
    out[5] = per_stage * stages;
}

void orc_welford(const Desc* d, int B, const double* U, int64_t* count, double* mean, double* M2) {
    const int nv = nvars(*d);
    const int64_t C = ncells(*d);
    const int64_t S = (int64_t)nv * C;
    int64_t n0 = *count;
    for (int64_t i = 0; i < C; ++i) {
        int64_t n = n0;
        for (int b = 0; b < B; ++b) {
            double Uc[8], W[8];
            for (int v = 0; v < nv; ++v) Uc[v] = U[b * S + v * C + i];
            if (d->eq == EQ_BURGERS) W[0] = Uc[0];
            else cons_to_prim(*d, Uc, W);
            n += 1;
            for (int q = 0; q < nv; ++q) {
                double x = W[q];
                double delta = x - mean[q * C + i];
                mean[q * C + i] += delta / (double)n;
                M2[q * C + i] += delta * (x - mean[q * C + i]);
            }
        }
    }
    *count = n0 + B;
}

// Pairwise merge of two Welford accumulators (Chan, Golub, LeVeque): n = nA + nB, d = mB - mA,
// mean = mA + d nB / n, M2 = M2A + M2B + d^2 nA nB / n; folds (B) into (A) in place.
void orc_stats_merge(const Desc* d, int64_t* countA, double* meanA, double* M2A, int64_t countB,
                     const double* meanB, const double* M2B) {
    const int64_t C = ncells(*d);
    const int nq = nvars(*d);
    const int64_t na = *countA, nb = countB;
    if (nb == 0) return;
    for (int64_t i = 0; i < nq * C; ++i) {
        if (na == 0) { meanA[i] = meanB[i]; M2A[i] = M2B[i]; continue; }
        const double n = (double)(na + nb);
        const double dl = meanB[i] - meanA[i];
        meanA[i] = meanA[i] + dl * (double)nb / n;
        M2A[i] = M2A[i] + M2B[i] + dl * dl * (double)na * (double)nb / n;
    }
    *countA = na + nb;
}

// Totals sum_i U_{v,i} dV per sample and variable (pairwise summation).
static double pairwise(const double* x, int64_t n) {
    if (n <= 8) { double s = 0.0; for (int64_t i = 0; i < n; ++i) s += x[i]; return s; }
    int64_t h = n / 2;
    return pairwise(x, h) + pairwise(x + h, n - h);
}
void orc_totals(const Desc* d, int B, const double* U, double* tot) {
    const int nv = nvars(*d);
    const int64_t C = ncells(*d);
    double dV = 1.0;
    for (int k = 0; k < d->ndim; ++k) dV *= dx(*d, k);
    for (int b = 0; b < B; ++b)
        for (int v = 0; v < nv; ++v) tot[b * nv + v] = pairwise(U + ((int64_t)b * nv + v) * C, C) * dV;
}

// Kinetic energy KE = sum_i |m_i|^2 / (2 rho_i) dV per sample (Euler).
void orc_kinetic_energy(const Desc* d, int B, const double* U, double* ke) {
    const int nv = nvars(*d);
    const int64_t C = ncells(*d);
    double dV = 1.0;
    for (int k = 0; k < d->ndim; ++k) dV *= dx(*d, k);
    std::vector<double> e(C);
    for (int b = 0; b < B; ++b) {
        const double* Ub = U + (int64_t)b * nv * C;
        for (int64_t i = 0; i < C; ++i) {
            double m2 = 0.0;
            for (int k = 0; k < d->ndim; ++k) m2 += Ub[(1 + k) * C + i] * Ub[(1 + k) * C + i];
            e[i] = 0.5 * m2 / Ub[i];
        }
        ke[b] = pairwise(e.data(), C) * dV;
    }
}

// Mixing-layer width of the KH shear layer (reading; the paper names no observable): the
// inner-band fraction c = (rho - 1) / (2 - 1) of the two KH densities (1 outside, 2 inside) gives
// W = sum_i 4 c_i (1 - c_i) dV, i.e. 4 (rho_i - 1) (2 - rho_i) dV per cell: 0 in either pure state,
// the cell's area where the two are mixed half and half. Pairwise sum per sample (2D Euler).
void orc_mixing_width(const Desc* d, int B, const double* U, double* out) {
    const int nv = nvars(*d);
    const int64_t C = ncells(*d);
    double dV = 1.0;
    for (int k = 0; k < d->ndim; ++k) dV *= dx(*d, k);
    std::vector<double> e(C);
    for (int b = 0; b < B; ++b) {
        const double* Ub = U + (int64_t)b * nv * C;
        for (int64_t i = 0; i < C; ++i) e[i] = 4.0 * (Ub[i] - 1.0) * (2.0 - Ub[i]);
        out[b] = pairwise(e.data(), C) * dV;
    }
}

// Exact gradient of an observable at time n_steps*dt with respect to the 20 2D KH parameters of
// ONE sample, by forward-mode dual numbers through init + n fixed-dt steps: observable 0 = the
// kinetic energy sum |m|^2 / (2 rho) dV, 1 = the mixing-layer width sum 4 (rho - 1)(2 - rho) dV
// (cells summed in order). Returns J in *J and dJ/dtheta in grad[20].
int orc_obs_grad_kh2d(const Desc* d, const double* theta, double dt, int64_t n_steps, int observable, double* J,
                      double* grad) {
    if (d->eq != EQ_EULER || d->ndim != 2 || observable < 0 || observable > 1) return 1;
    typedef Dual<20> D;
    const int64_t N = (int64_t)nvars(*d) * ncells(*d);
    std::vector<D> th(20), U(N);
    for (int j = 0; j < 20; ++j) { th[j] = D(theta[j]); th[j].d[j] = 1.0; }
    init_kh(*d, th.data(), U.data());
    for (int64_t s = 0; s < n_steps; ++s) rk_step(*d, U.data(), D(dt));
    const int64_t C = ncells(*d);
    const double dV = dx(*d, 0) * dx(*d, 1);
    D acc(0.0);
    for (int64_t i = 0; i < C; ++i) {
        if (observable == 0) {
            D m2 = U[C + i] * U[C + i] + U[2 * C + i] * U[2 * C + i];
            acc = acc + 0.5 * m2 / U[i];
        } else {
            acc = acc + 4.0 * (U[i] - 1.0) * (2.0 - U[i]);
        }
    }
    acc = acc * dV;
    *J = acc.v;
    for (int j = 0; j < 20; ++j) grad[j] = acc.d[j];
    return 0;
}

// The kinetic-energy case of orc_obs_grad_kh2d.
int orc_ke_grad_kh2d(const Desc* d, const double* theta, double dt, int64_t n_steps, double* J, double* grad) {
    return orc_obs_grad_kh2d(d, theta, dt, n_steps, 0, J, grad);
}

// Directional derivative dJ/dtheta . vdir via a single-direction dual run (dot-product pin).
int orc_ke_dir_kh2d(const Desc* d, const double* theta, const double* vdir, double dt, int64_t n_steps, double* J,
                    double* dJ) {
    if (d->eq != EQ_EULER || d->ndim != 2) return 1;
    typedef Dual<1> D;
    const int64_t N = (int64_t)nvars(*d) * ncells(*d);
    std::vector<D> th(20), U(N);
    for (int j = 0; j < 20; ++j) { th[j] = D(theta[j]); th[j].d[0] = vdir[j]; }
    init_kh(*d, th.data(), U.data());
    for (int64_t s = 0; s < n_steps; ++s) rk_step(*d, U.data(), D(dt));
    const int64_t C = ncells(*d);
    const double dV = dx(*d, 0) * dx(*d, 1);
    D acc(0.0);
    for (int64_t i = 0; i < C; ++i) {
        D m2 = U[C + i] * U[C + i] + U[2 * C + i] * U[2 * C + i];
        acc = acc + 0.5 * m2 / U[i];
    }
    acc = acc * dV;
    *J = acc.v;
    *dJ = acc.d[0];
    return 0;
}

}  // extern "C"
