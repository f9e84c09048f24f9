"""Plain FP64 CPU oracle for the Alsvinn finite-volume hot path (arXiv:1912.07645).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``, never by the product package.
It shares no code with the CUDA library; the C++ source is ``alsv_oracle.cpp`` (one cell at a
time, FP64, ``-ffp-contract=off``), and this module only builds it and marshals numpy arrays.

Every function here is a thin wrapper over the C++ entry point of the same name; the C++ file
cites the passage of the paper (or the reading of it) that each computes. The exception is the
multilevel Monte Carlo estimator (``mlmc_estimate`` and its helpers), written here in numpy
directly from the estimator's definition.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alsv_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EQ = {"burgers": 0, "euler": 1}
RECON = {"pc": 0, "mc": 1, "weno3": 2, "eno2": 3}
RVARS = {"cons": 0, "prim": 1}
FLUX = {"rusanov": 0, "hll": 1, "hllc": 2, "roe": 3, "godunov": 4, "ec": 5, "ec4": 6, "tecno2": 7}
RK = {"ssprk2": 2, "ssprk3": 3}
BC = {"periodic": 0, "outflow": 1, "reflective": 2}
INIT = {"kh": 0, "sod": 1, "lax": 2, "burgers_sine": 3, "vortex": 4}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with g++ (OpenMP when available). Returns the library path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", _SRC]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base + extra + ["-o", tmp], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB_PATH)
            return _LIB_PATH
    raise RuntimeError("oracle build failed:\n" + r.stderr)


class Desc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("eq", C.c_int32), ("gamma", C.c_double), ("recon", C.c_int32), ("rvars", C.c_int32),
        ("flux", C.c_int32), ("rk", C.c_int32), ("bc", (C.c_int32 * 2) * 3), ("cfl", C.c_double),
        ("weno_eps", C.c_double), ("weno_eps_dx2", C.c_int32),
    ]


def make_desc(ndim=1, n=(8, 1, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), eq="euler", gamma=1.4,
              recon="mc", rvars="prim", flux="hllc", rk="ssprk2", bc="periodic", cfl=0.45,
              weno_eps=1e-6, weno_eps_dx2=False, **_ignored) -> Desc:
    """Build the oracle's descriptor from plain keyword values.

    ``bc`` is a name for all sides, or a list of ``(lo, hi)`` names per direction.
    """
    d = Desc()
    d.ndim = ndim
    nn = list(n) + [1] * (3 - len(n))
    for k in range(3):
        d.n[k] = int(nn[k]) if k < ndim else 1
        d.lo[k] = float(lo[k]) if k < len(lo) else 0.0
        d.hi[k] = float(hi[k]) if k < len(hi) else 1.0
    d.eq = EQ[eq]
    d.gamma = gamma
    d.recon = RECON[recon]
    d.rvars = RVARS[rvars]
    d.flux = FLUX[flux]
    d.rk = RK[rk]
    for k in range(3):
        if isinstance(bc, str):
            pair = (bc, bc)
        else:
            pair = bc[k] if k < len(bc) else ("periodic", "periodic")
        d.bc[k][0] = BC[pair[0]]
        d.bc[k][1] = BC[pair[1]]
    d.cfl = cfl
    d.weno_eps = weno_eps
    d.weno_eps_dx2 = 1 if weno_eps_dx2 else 0
    return d


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER
            dp = P(C.c_double)
            i64p = P(C.c_int64)
            dsc = P(Desc)
            L.orc_num_threads.restype = C.c_int
            L.orc_nvars.argtypes = [dsc]
            L.orc_flux.argtypes = [dsc, C.c_int, dp, dp, dp]
            L.orc_entropy_vars.argtypes = [dsc, dp, dp]
            L.orc_tecno_matrix.argtypes = [dsc, C.c_int, dp, dp, dp, dp]
            L.orc_tecno_flux.argtypes = [dsc, C.c_int, dp, dp]
            L.orc_recon.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
            L.orc_cons_to_prim.argtypes = [dsc, dp, dp]
            L.orc_prim_to_cons.argtypes = [dsc, dp, dp]
            L.orc_rhs.argtypes = [dsc, C.c_int, dp, dp]
            L.orc_max_speed.argtypes = [dsc, C.c_int, dp, dp]
            L.orc_evolve.argtypes = [dsc, C.c_int, dp, C.c_double, C.c_double, C.c_int64, C.c_int64,
                                     i64p, dp]
            L.orc_evolve.restype = C.c_int
            L.orc_theta.argtypes = [C.c_uint64, C.c_int, C.c_int, dp]
            L.orc_splitmix64.argtypes = [C.c_uint64]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_init.argtypes = [dsc, C.c_int, C.c_int, dp, C.c_int, C.c_double, C.c_double, dp]
            L.orc_init.restype = C.c_int
            L.orc_welford.argtypes = [dsc, C.c_int, dp, i64p, dp, dp]
            L.orc_totals.argtypes = [dsc, C.c_int, dp, dp]
            L.orc_stats_merge.argtypes = [dsc, i64p, dp, dp, C.c_int64, dp, dp]
            L.orc_kinetic_energy.argtypes = [dsc, C.c_int, dp, dp]
            L.orc_ke_grad_kh2d.argtypes = [dsc, dp, C.c_double, C.c_int64, dp, dp]
            L.orc_ke_grad_kh2d.restype = C.c_int
            L.orc_obs_grad_kh2d.argtypes = [dsc, dp, C.c_double, C.c_int64, C.c_int, dp, dp]
            L.orc_obs_grad_kh2d.restype = C.c_int
            L.orc_mixing_width.argtypes = [dsc, C.c_int, dp, dp]
            L.orc_face_states.argtypes = [dsc, dp, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
            L.orc_ke_dir_kh2d.argtypes = [dsc, dp, dp, C.c_double, C.c_int64, dp, dp]
            L.orc_ke_dir_kh2d.restype = C.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def nvars(d: Desc) -> int:
    return int(lib().orc_nvars(C.byref(d)))


def state_shape(d: Desc, B: int):
    return (B, nvars(d), d.n[2], d.n[1], d.n[0])


def flux(d: Desc, k: int, WL, WR) -> np.ndarray:
    WL, WR = _f64(WL), _f64(WR)
    F = np.zeros(nvars(d))
    lib().orc_flux(C.byref(d), k, _dp(WL), _dp(WR), _dp(F))
    return F


def entropy_vars(d: Desc, W) -> np.ndarray:
    """Entropy variables of a primitive state (Euler: entropy -rho s/(gamma - 1); Burgers: u^2/2)."""
    W = _f64(W)
    v = np.zeros(nvars(d))
    lib().orc_entropy_vars(C.byref(d), _dp(W), _dp(v))
    return v


def tecno_matrix(d: Desc, k: int, WL, WR):
    """Scaled eigenvectors Rs (Rs Rs^T = dU/dv) and absolute eigenvalues along k at the mean of
    two primitive states (TECNO2's diffusion operator)."""
    WL, WR = _f64(WL), _f64(WR)
    nv = nvars(d)
    Rs = np.zeros(nv * nv)
    lam = np.zeros(nv)
    lib().orc_tecno_matrix(C.byref(d), k, _dp(WL), _dp(WR), _dp(Rs), _dp(lam))
    return Rs.reshape(nv, nv), lam


def tecno_flux(d: Desc, k: int, W4) -> np.ndarray:
    """TECNO2 flux at the interface between the middle two of four consecutive primitive states."""
    W4 = _f64(W4).reshape(4, nvars(d))
    F = np.zeros(nvars(d))
    lib().orc_tecno_flux(C.byref(d), k, _dp(np.ascontiguousarray(W4)), _dp(F))
    return F


def recon(kind: str, wm: float, w0: float, wp: float, eps: float = 1e-6):
    fl, fr = C.c_double(), C.c_double()
    lib().orc_recon(RECON[kind], eps, wm, w0, wp, C.byref(fl), C.byref(fr))
    return fl.value, fr.value


def cons_to_prim(d: Desc, U) -> np.ndarray:
    U = _f64(U)
    W = np.zeros_like(U)
    lib().orc_cons_to_prim(C.byref(d), _dp(U), _dp(W))
    return W


def face_states(d: Desc, U, cell, k: int):
    """(left face, right face) primitive states of one cell (x, y, z) along direction k of a single
    sample U [nv, nz, ny, nx], after reconstruction and the positivity fallback."""
    U = _f64(U)
    nv = nvars(d)
    Wl, Wr = np.zeros(nv), np.zeros(nv)
    c = list(cell) + [0] * (3 - len(cell))
    lib().orc_face_states(C.byref(d), _dp(U), c[0], c[1], c[2], k, _dp(Wl), _dp(Wr))
    return Wl, Wr


def prim_to_cons(d: Desc, W) -> np.ndarray:
    W = _f64(W)
    U = np.zeros_like(W)
    lib().orc_prim_to_cons(C.byref(d), _dp(W), _dp(U))
    return U


def rhs(d: Desc, U) -> np.ndarray:
    U = _f64(U)
    L = np.zeros_like(U)
    lib().orc_rhs(C.byref(d), U.shape[0], _dp(U), _dp(L))
    return L


def max_speed(d: Desc, U) -> np.ndarray:
    U = _f64(U)
    s = np.zeros(U.shape[0])
    lib().orc_max_speed(C.byref(d), U.shape[0], _dp(U), _dp(s))
    return s


def evolve(d: Desc, U, T: float = 0.0, fixed_dt: float = 0.0, n_steps: int = 0, max_steps: int = 0):
    """Advance a copy of U ([B, nv, nz, ny, nx]); returns (U_new, steps[B], t[B])."""
    U = _f64(U).copy()
    B = U.shape[0]
    steps = np.zeros(B, dtype=np.int64)
    t = np.zeros(B)
    st = lib().orc_evolve(C.byref(d), B, _dp(U), T, fixed_dt, n_steps, max_steps,
                          steps.ctypes.data_as(C.POINTER(C.c_int64)), _dp(t))
    if st != 0:
        raise FloatingPointError(f"oracle evolve: non-physical state (status {st})")
    return U, steps, t


def theta_splitmix(seed: int, B: int, P: int) -> np.ndarray:
    th = np.zeros((B, P))
    lib().orc_theta(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), B, P, _dp(th))
    return th


def primes(k: int) -> list:
    """The first k primes by trial division."""
    out = []
    p = 1
    while len(out) < k:
        p += 1
        if all(p % d for d in range(2, int(p ** 0.5) + 1)):
            out.append(p)
    return out


def radical_inverse(n: int, p: int) -> float:
    """Halton's radical inverse phi_p(n) = sum_k d_k p^(-k-1), n = sum_k d_k p^k (exact rational,
    rounded once)."""
    num, den = 0, 1
    while n > 0:
        n, d = divmod(n, p)
        num = num * p + d
        den *= p
    return num / den


def theta_halton(B: int, P: int, seed: int = 0, shifted: bool = False, first_index: int = 0) -> np.ndarray:
    """Quasi Monte Carlo KH parameters (Sec. 2.2 QMC): theta_{b,j} = hi_j phi_{p_j}(g + 1) with g the
    sample's global index, p_j the (j+1)-th prime, hi = 1 (amplitudes) or 2 pi (phases); the
    shifted form adds the Cranley-Patterson rotation s_j = u01(splitmix64(seed ^ (2^63 + j))) mod 1."""
    ps = primes(P)
    th = np.zeros((B, P))
    for b in range(B):
        for j in range(P):
            u = radical_inverse(first_index + b + 1, ps[j])
            if shifted:
                u = u + (splitmix64(seed ^ ((1 << 63) + j)) >> 11) * (1.0 / 9007199254740992.0)
                if u >= 1.0:
                    u = u - 1.0
            th[b, j] = (1.0 if j < P // 2 else 2.0 * math.pi) * u
    return th


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def init(d: Desc, kind: str, B: int = 1, theta=None, center=(5.0, 5.0)) -> np.ndarray:
    U = np.zeros(state_shape(d, B))
    if theta is None:
        th = np.zeros((B, 1))
    else:
        th = _f64(theta).reshape(B, -1)
    st = lib().orc_init(C.byref(d), INIT[kind], B, _dp(th), th.shape[1], center[0], center[1], _dp(U))
    if st != 0:
        raise ValueError(f"oracle init {kind}: invalid for this descriptor")
    return U


def welford(d: Desc, U, count: int = 0, mean=None, M2=None):
    """Fold B samples into (count, mean[q, cells], M2[q, cells]); returns the updated triple."""
    U = _f64(U)
    B = U.shape[0]
    nq = nvars(d)
    cells = d.n[0] * d.n[1] * d.n[2]
    mean = np.zeros((nq, cells)) if mean is None else _f64(mean).copy()
    M2 = np.zeros((nq, cells)) if M2 is None else _f64(M2).copy()
    cnt = C.c_int64(count)
    lib().orc_welford(C.byref(d), B, _dp(U), C.byref(cnt), _dp(mean), _dp(M2))
    return cnt.value, mean, M2


def stats_merge(d: Desc, a, b):
    """Fold accumulator b = (count, mean, M2) into a copy of a; returns the merged triple."""
    ca, ma, Ma = a
    cb, mb, Mb = b
    ma, Ma = _f64(ma).copy(), _f64(Ma).copy()
    mb, Mb = _f64(mb), _f64(Mb)
    cnt = C.c_int64(ca)
    lib().orc_stats_merge(C.byref(d), C.byref(cnt), _dp(ma), _dp(Ma), cb, _dp(mb), _dp(Mb))
    return cnt.value, ma, Ma


def totals(d: Desc, U) -> np.ndarray:
    U = _f64(U)
    out = np.zeros((U.shape[0], nvars(d)))
    lib().orc_totals(C.byref(d), U.shape[0], _dp(U), _dp(out))
    return out


def kinetic_energy(d: Desc, U) -> np.ndarray:
    U = _f64(U)
    out = np.zeros(U.shape[0])
    lib().orc_kinetic_energy(C.byref(d), U.shape[0], _dp(U), _dp(out))
    return out


def ke_grad_kh2d(d: Desc, theta, dt: float, n_steps: int):
    """(J, dJ/dtheta[20]) of one 2D KH sample after n fixed steps, by forward-mode duals."""
    th = _f64(theta).reshape(20)
    J = C.c_double()
    g = np.zeros(20)
    st = lib().orc_ke_grad_kh2d(C.byref(d), _dp(th), dt, n_steps, C.byref(J), _dp(g))
    if st != 0:
        raise ValueError("ke_grad_kh2d needs a 2D Euler descriptor")
    return J.value, g


def mixing_width(d: Desc, U) -> np.ndarray:
    """Mixing-layer width sum_i 4 (rho_i - 1)(2 - rho_i) dV per sample (KH densities 1 and 2)."""
    U = _f64(U)
    out = np.zeros(U.shape[0])
    lib().orc_mixing_width(C.byref(d), U.shape[0], _dp(U), _dp(out))
    return out


OBSERVABLES = {"ke": 0, "mixing": 1}


def obs_grad_kh2d(d: Desc, theta, dt: float, n_steps: int, observable: str = "ke"):
    """(J, dJ/dtheta[20]) of one 2D KH sample after n fixed steps for the kinetic energy ("ke") or
    the mixing-layer width ("mixing"), by forward-mode duals."""
    th = _f64(theta).reshape(20)
    J = C.c_double()
    g = np.zeros(20)
    st = lib().orc_obs_grad_kh2d(C.byref(d), _dp(th), dt, n_steps, OBSERVABLES[observable], C.byref(J), _dp(g))
    if st != 0:
        raise ValueError("obs_grad_kh2d needs a 2D Euler descriptor")
    return J.value, g


def ke_dir_kh2d(d: Desc, theta, vdir, dt: float, n_steps: int):
    th = _f64(theta).reshape(20)
    v = _f64(vdir).reshape(20)
    J, dJ = C.c_double(), C.c_double()
    st = lib().orc_ke_dir_kh2d(C.byref(d), _dp(th), _dp(v), dt, n_steps, C.byref(J), C.byref(dJ))
    if st != 0:
        raise ValueError("ke_dir_kh2d needs a 2D Euler descriptor")
    return J.value, dJ.value


def count_flops(d: Desc) -> dict:
    """Algorithmic floating-point operations of the scheme, counted on the oracle's counting
    scalar: per reconstruction (one variable, both faces), cons->prim, interface flux,
    divergence + RK per cell-stage, per cell-stage and per cell-update."""
    out = np.zeros(6)
    lib().orc_count_flops(C.byref(d), _dp(out))
    keys = ("recon", "cons_to_prim", "flux", "div_rk", "per_cell_stage", "per_cell_update")
    return dict(zip(keys, out.tolist()))


def fixed_dt_kh(n: int, T: float, cfl: float, gamma: float = 1.4, length: float = 1.0):
    """Fixed step for the adjoint (reading): s_max from the two unperturbed KH states,
    n_steps = ceil(T s_max / (cfl dx)), dt = T / n_steps."""
    import math
    s_max = 0.5 + math.sqrt(gamma * 2.5 / 1.0)
    dxh = length / n
    n_steps = int(math.ceil(T * s_max / (cfl * dxh)))
    return T / n_steps, n_steps


# ---------------------------------------------------------------------------------------------
# Multilevel Monte Carlo estimator (Sec. 2.2, the multilevel form of the sampling display):
#   E[G(u)] ~ sum_l (1/M_l) sum_k (G(u^l_k) - G(u^{l-1}_k)),  G(u^{-1}) = 0,
# for G = q and G = q^2, q = primitive variables per cell. The coarse member u^{l-1}_k of a pair
# is the same sample (same KH parameters) on level l-1's grid, prolongated piecewise constantly
# to level l's grid. Mean = telescoped first moment; variance = telescoped second moment minus
# the squared mean (reading). Per-level sums: (sum mean_Y dV, sum |mean_Y| dV, sum var_Y dV),
# var_Y the unbiased sample variance of Y = q^l - P q^{l-1}.
# ---------------------------------------------------------------------------------------------
def primitive_quantities(U, gamma: float = 1.4, euler: bool = True) -> np.ndarray:
    """q = (rho, u_k, p) from conserved U [M, nv, nz, ny, nx] (Burgers: u itself)."""
    U = _f64(U)
    if not euler:
        return U.copy()
    rho = U[:, 0]
    m = U[:, 1:-1]
    q = np.empty_like(U)
    q[:, 0] = rho
    q[:, 1:-1] = m / rho[:, None]
    q[:, -1] = (gamma - 1.0) * (U[:, -1] - 0.5 * (m * m).sum(axis=1) / rho)
    return q


def prolongate(x, shape) -> np.ndarray:
    """Piecewise-constant prolongation of x [..., nz, ny, nx] to the grid shape (nz', ny', nx'):
    each fine cell takes the value of the coarse cell that contains it."""
    x = _f64(x)
    for ax, n_fine in zip((-3, -2, -1), shape):
        n_coarse = x.shape[ax]
        if n_fine % n_coarse:
            raise ValueError("the coarse grid must divide the fine grid")
        x = np.repeat(x, n_fine // n_coarse, axis=ax)
    return x


def mlmc_estimate(levels, gamma: float = 1.4, euler: bool = True):
    """levels: list of (U_fine [M_l, nv, ...], U_coarse [M_l, nv, ...] or None, dV_l) in level
    order. Returns (mean [nq, ...], var [nq, ...], level_sums [L, nq, 3]) on the finest grid."""
    fine_shape = max((lv[0].shape[-3:] for lv in levels), key=lambda s: s[0] * s[1] * s[2])
    mean = 0.0
    second = 0.0
    sums = []
    for Uf, Uc, dV in levels:
        qf = primitive_quantities(Uf, gamma, euler)
        qc = 0.0 if Uc is None else prolongate(primitive_quantities(Uc, gamma, euler), qf.shape[-3:])
        Y = qf - qc
        Z = qf * qf - qc * qc
        M = Y.shape[0]
        mY = Y.mean(axis=0)
        vY = Y.var(axis=0, ddof=1) if M > 1 else np.zeros_like(mY)
        mean = mean + prolongate(mY, fine_shape)
        second = second + prolongate(Z.mean(axis=0), fine_shape)
        nq = mY.shape[0]
        sums.append([[mY[q].sum() * dV, np.abs(mY[q]).sum() * dV, vY[q].sum() * dV] for q in range(nq)])
    return mean, second - mean * mean, np.array(sums)


# ---------------------------------------------------------------------------------------------
# Statistical functionals (Sec. 2.2: point PDFs and two-point structure functions), numpy.
# ---------------------------------------------------------------------------------------------
def point_pdf(U, q: int, cells, lo: float, hi: float, n_bins: int, gamma: float = 1.4, euler: bool = True):
    """Counts [points, n_bins + 2] of quantity q at flat cell indices over the samples of U:
    bin 0 below lo, 1 + floor((x - lo) / (hi - lo) * n_bins) (at most n_bins) inside, n_bins + 1
    at or above hi (and NaN)."""
    Q = primitive_quantities(U, gamma, euler)[:, q].reshape(U.shape[0], -1)
    counts = np.zeros((len(cells), n_bins + 2), dtype=np.int64)
    for i, c in enumerate(cells):
        for x in Q[:, c]:
            counts[i, _bin(x, lo, hi, n_bins)] += 1
    return counts


def _bin(x: float, lo: float, hi: float, n_bins: int) -> int:
    if x < lo:
        return 0
    if x < hi:
        return 1 + min(int(math.floor((x - lo) / (hi - lo) * n_bins)), n_bins - 1)
    return n_bins + 1


def joint_pdf(U, q1: int, q2: int, cells, lo1, hi1, nb1, lo2, hi2, nb2, gamma: float = 1.4, euler: bool = True):
    """Joint counts [points, nb1 + 2, nb2 + 2] of quantities q1, q2 at each cell over the samples,
    each binned as in point_pdf."""
    Q = primitive_quantities(U, gamma, euler).reshape(U.shape[0], U.shape[1], -1)
    counts = np.zeros((len(cells), nb1 + 2, nb2 + 2), dtype=np.int64)
    for i, c in enumerate(cells):
        for b in range(U.shape[0]):
            counts[i, _bin(Q[b, q1, c], lo1, hi1, nb1), _bin(Q[b, q2, c], lo2, hi2, nb2)] += 1
    return counts


def correlator(U, q: int, cell_sets, gamma: float = 1.4, euler: bool = True):
    """Multi-point correlator sums: (samples, [sum over samples of prod_j q(x_j)] per set)."""
    Q = primitive_quantities(U, gamma, euler)[:, q].reshape(U.shape[0], -1)
    sums = np.zeros(len(cell_sets))
    for s, cs in enumerate(cell_sets):
        for b in range(U.shape[0]):
            prod = 1.0
            for c in cs:
                prod = prod * Q[b, c]
            sums[s] += prod
    return U.shape[0], sums


def structure_function_sums(U, q: int, p: int, R: int, dx, periodic, gamma: float = 1.4, euler: bool = True):
    """Per radius shell r = 1..R, the sum over samples of
    sum_x sum_{k in Z^d, r-1 < |k| <= r} |q(x + k) - q(x)|^p dV^2 (periodic directions wrap; pairs
    leaving a non-periodic domain are dropped). Returns (number of samples, shell sums [R])."""
    Q = primitive_quantities(U, gamma, euler)[:, q]        # [M, nz, ny, nx]
    nd = len(dx)
    dV = float(np.prod(dx))
    sums = np.zeros(R)
    rng = [range(-R, R + 1) if k < nd else range(0, 1) for k in range(3)]
    for kz in rng[2]:
        for ky in rng[1]:
            for kx in rng[0]:
                d2 = kx * kx + ky * ky + kz * kz
                if d2 == 0 or d2 > R * R:
                    continue
                r = math.isqrt(d2)
                if r * r < d2:
                    r += 1                                  # smallest r with r^2 >= |k|^2
                A, B = Q, Q
                for ax, (k, per) in zip((-1, -2, -3), ((kx, periodic[0]), (ky, periodic[1] if nd > 1 else True),
                                                      (kz, periodic[2] if nd > 2 else True))):
                    if k == 0:
                        continue
                    if per:
                        B = np.roll(B, -k, axis=ax)         # B[x] = Q[x + k]
                    else:
                        n = Q.shape[ax]
                        sl_a = [slice(None)] * 4
                        sl_b = [slice(None)] * 4
                        sl_a[ax] = slice(max(0, -k), n - max(0, k))
                        sl_b[ax] = slice(max(0, k), n - max(0, -k))
                        A, B = A[tuple(sl_a)], B[tuple(sl_b)]
                diff = np.abs(B - A)
                sums[r - 1] += (diff ** p).sum() * dV * dV
    return Q.shape[0], sums


def structure_function(count: int, sums, p: int):
    """S_p(r) = (sum_{r' <= r} sums[r'] / count)^(1/p)."""
    return (np.cumsum(sums) / count) ** (1.0 / p)
