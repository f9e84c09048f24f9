"""Pins of the FP64 CPU oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: published values (SplitMix64
outputs, the Sod star state), closed forms (exact Riemann and Burgers solutions, boundary-flux
balances, KH band mass), invariants (consistency, conservation, mirror/rotation symmetry),
convergence orders on smooth data, and finite differences for the exact discrete gradient.
"""
import math
import os

import numpy as np
import pytest

import oracle
from exact import RiemannExact, burgers_sine_cell_averages, observed_rates

HERE = os.path.dirname(os.path.abspath(__file__))
rng = np.random.default_rng(1234)


def euler_phys_flux_1d(W, g=1.4):
    r, u, p = W
    E = p / (g - 1) + 0.5 * r * u * u
    return np.array([r * u, r * u * u + p, u * (E + p)])


def random_prim(nd, rng, n=1):
    r = rng.uniform(0.2, 3.0, n)
    u = rng.uniform(-2.0, 2.0, (n, nd))
    p = rng.uniform(0.1, 4.0, n)
    return [np.concatenate([[r[i]], u[i], [p[i]]]) for i in range(n)]


# ---------------------------------------------------------------- RNG (O3 reading)
def test_splitmix64_published_sequence():
    # First outputs of SplitMix64 seeded with 0 (Steele-Lea-Flood / Vigna reference code):
    # state advances by the golden gamma before each mix.
    gamma = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(gamma) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * gamma) & (2**64 - 1)) == 0x06C45D188009454F


def test_theta_ranges_and_counter_property():
    th = oracle.theta_splitmix(12345, 64, 20)
    assert th.shape == (64, 20)
    assert np.all(th[:, :10] >= 0) and np.all(th[:, :10] < 1)
    assert np.all(th[:, 10:] >= 0) and np.all(th[:, 10:] < 2 * math.pi)
    # sample b depends only on (seed, b): a sub-batch equals the slice
    th2 = oracle.theta_splitmix(12345, 8, 20)
    assert np.array_equal(th[:8], th2)
    # the value is the top 53 bits of the mixed counter
    r = oracle.splitmix64(12345 ^ (3 * 20 + 4))
    assert th[3, 4] == (r >> 11) * 2.0**-53


# ---------------------------------------------------------------- fluxes (Sec. 2.1)
@pytest.mark.parametrize("fl", ["rusanov", "hll", "hllc"])
def test_flux_consistency_euler_1d(fl):
    d = oracle.make_desc(ndim=1, n=(4,), eq="euler", flux=fl)
    for W in random_prim(1, rng, 50):
        F = oracle.flux(d, 0, W, W)
        np.testing.assert_allclose(F, euler_phys_flux_1d(W), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("fl", ["rusanov", "hll", "hllc"])
@pytest.mark.parametrize("nd", [2, 3])
def test_flux_consistency_euler_multid(fl, nd):
    d = oracle.make_desc(ndim=nd, n=(4, 4, 4), eq="euler", flux=fl)
    g = 1.4
    for W in random_prim(nd, rng, 30):
        for k in range(nd):
            r, vel, p = W[0], W[1:1 + nd], W[1 + nd]
            E = p / (g - 1) + 0.5 * r * np.dot(vel, vel)
            ref = np.concatenate([[r * vel[k]], r * vel[k] * vel + p * (np.arange(nd) == k), [vel[k] * (E + p)]])
            np.testing.assert_allclose(oracle.flux(d, k, W, W), ref, rtol=1e-14, atol=1e-13)


def test_hllc_stationary_contact_is_exact():
    d = oracle.make_desc(ndim=2, n=(4, 4), eq="euler", flux="hllc")
    F = oracle.flux(d, 0, [3.0, 0.0, 0.7, 1.3], [0.25, 0.0, -0.2, 1.3])
    assert F[0] == 0.0 and F[3] == 0.0
    assert F[1] == 1.3


def test_hllc_moving_contact_is_upwind_exact():
    # an isolated contact (equal u and p) is resolved exactly: F = F(U_L) for u > 0
    d = oracle.make_desc(ndim=1, n=(4,), eq="euler", flux="hllc")
    WL, WR = [2.0, 0.3, 1.0], [0.5, 0.3, 1.0]
    np.testing.assert_allclose(oracle.flux(d, 0, WL, WR), euler_phys_flux_1d(WL), rtol=1e-14)
    d2 = oracle.make_desc(ndim=1, n=(4,), eq="euler", flux="hll")
    assert not np.allclose(oracle.flux(d2, 0, WL, WR), euler_phys_flux_1d(WL), rtol=1e-6)


@pytest.mark.parametrize("fl", ["hll", "hllc"])
def test_supersonic_upwinding(fl):
    d = oracle.make_desc(ndim=1, n=(4,), eq="euler", flux=fl)
    WL, WR = [1.0, 3.0, 1.0], [0.5, 2.9, 0.8]       # S_L > 0
    np.testing.assert_allclose(oracle.flux(d, 0, WL, WR), euler_phys_flux_1d(WL), rtol=1e-15)
    WL, WR = [1.0, -3.0, 1.0], [0.5, -2.9, 0.8]     # S_R < 0
    np.testing.assert_allclose(oracle.flux(d, 0, WL, WR), euler_phys_flux_1d(WR), rtol=1e-15)


@pytest.mark.parametrize("fl", ["rusanov", "hll", "hllc"])
def test_flux_mirror_symmetry(fl):
    # F(U_L, U_R) = -M F(M U_R, M U_L), M negating the normal velocity
    nd = 2
    d = oracle.make_desc(ndim=nd, n=(4, 4), eq="euler", flux=fl)
    for _ in range(30):
        WL, WR = random_prim(nd, rng, 2)
        for k in range(nd):
            M = np.ones(nd + 2)
            M[1 + k] = -1
            F = oracle.flux(d, k, WL, WR)
            Fm = oracle.flux(d, k, M * WR, M * WL)
            np.testing.assert_allclose(F, -M * Fm, rtol=1e-13, atol=1e-13)


def burgers_godunov(uL, uR):
    f = lambda u: 0.5 * u * u
    if uL > uR:
        s = 0.5 * (uL + uR)
        return f(uL) if s > 0 else f(uR)
    if uL > 0:
        return f(uL)
    if uR < 0:
        return f(uR)
    return 0.0


@pytest.mark.parametrize("fl", ["hll", "rusanov"])
def test_burgers_flux_vs_godunov_monotone(fl):
    d = oracle.make_desc(ndim=1, n=(4,), eq="burgers", flux=fl)
    for _ in range(50):
        a, b = rng.uniform(0.1, 2.0, 2)
        for uL, uR in ((a, b), (-a, -b)):
            F = oracle.flux(d, 0, [uL], [uR])[0]
            if fl == "hll":
                assert F == pytest.approx(burgers_godunov(uL, uR), rel=1e-15)
            else:  # Rusanov adds dissipation; equal to Godunov only for uL == uR
                assert F >= burgers_godunov(uL, uR) - 1e-15 if uL > uR else True
        F = oracle.flux(d, 0, [a], [a])[0]
        assert F == pytest.approx(0.5 * a * a, rel=1e-15)


def test_hll_equals_rusanov_for_symmetric_wave_speeds():
    """Both states at rest with equal sound speed (p/rho equal) give S_L = -S_R = a: the HLL
    formula then reduces to the Rusanov (local Lax-Friedrichs) flux with the same a. The two
    formulas share no code, so a wrong coefficient or sign in either one breaks the identity."""
    for nd in (1, 2, 3):
        dh = oracle.make_desc(ndim=nd, n=(4, 4, 4), eq="euler", flux="hll")
        dr = oracle.make_desc(ndim=nd, n=(4, 4, 4), eq="euler", flux="rusanov")
        for _ in range(20):
            rL, pL = rng.uniform(0.3, 3.0), rng.uniform(0.2, 4.0)
            s = rng.uniform(0.1, 0.9)
            vt = rng.uniform(-1.0, 1.0, nd)               # tangential velocities ride along
            for k in range(nd):
                WL = np.concatenate([[rL], vt, [pL]])
                WR = np.concatenate([[s * rL], -vt, [s * pL]])
                WL[1 + k] = WR[1 + k] = 0.0
                Fh, Fr = oracle.flux(dh, k, WL, WR), oracle.flux(dr, k, WL, WR)
                np.testing.assert_allclose(Fh, Fr, rtol=1e-13, atol=1e-14)
                assert abs(Fh[0]) > 1e-3                   # the dissipation term is active


def _entropy_wave_viscosity_run(fl, nd, u, rk, n=32, kmode=3, steps=40, eps=1e-7):
    """PC scheme on a small-amplitude entropy wave rho = 1 + eps cos(2 pi kmode x), uniform normal
    velocity u, tangential velocity 0.2 and pressure 1, fixed dt, periodic: returns (measured
    amplification of the mode over the run, lambda = dt/dx, theta = 2 pi kmode / n, c)."""
    g, p0 = 1.4, 1.0
    c = math.sqrt(g * p0 / 1.0)
    dx = 1.0 / n
    dt = 0.4 * dx / (abs(u) + c)
    x = (np.arange(n) + 0.5) * dx
    rho = 1.0 + eps * np.cos(2 * np.pi * kmode * x)
    ax = nd - 1                                          # the wave runs along the last direction
    shape = [1] * 3
    shape[2 - ax] = n
    nn = [4, 4, 4][:nd]
    nn[ax] = n
    d = oracle.make_desc(ndim=nd, n=nn, eq="euler", recon="pc", flux=fl, rk=rk, bc="periodic")
    U = np.zeros(oracle.state_shape(d, 1))
    r = np.broadcast_to(rho.reshape(shape), U.shape[2:])
    vel = np.full(nd, 0.2)
    vel[ax] = u
    U[0, 0] = r
    for j in range(nd):
        U[0, 1 + j] = r * vel[j]
    U[0, 1 + nd] = p0 / (g - 1) + 0.5 * r * np.dot(vel, vel)
    Un, _, _ = oracle.evolve(d, U, fixed_dt=dt, n_steps=steps)
    line = [0] * 3
    line[2 - ax] = slice(None)
    r0 = U[0, 0][tuple(line)] - 1.0
    r1 = Un[0, 0][tuple(line)] - 1.0
    G = np.fft.fft(r1)[kmode] / np.fft.fft(r0)[kmode]
    # the velocity and pressure of an entropy wave stay uniform under any of these fluxes
    W = Un[0, 1 + ax] / Un[0, 0]
    assert np.abs(W - u).max() < 1e-12
    return G, dt / dx, 2 * np.pi * kmode / n, c


@pytest.mark.parametrize("nd", [1, 2])
@pytest.mark.parametrize("fl,u", [("rusanov", 0.3), ("rusanov", -0.3), ("rusanov", 2.0), ("hll", 0.3),
                                  ("hll", -0.7), ("hll", 2.0), ("hll", -2.0), ("hllc", 0.3), ("hllc", -0.7)])
def test_entropy_wave_numerical_viscosity_von_neumann(fl, u, nd):
    """Von Neumann analysis of the first-order scheme on a linearised entropy wave (u, p uniform,
    rho = 1 + eps cos): every flux here becomes F_{j+1/2} = u (rho_j + rho_{j+1})/2
    - q (rho_{j+1} - rho_j)/2, so a Fourier mode e^{i theta j} is multiplied per step by the RK
    polynomial of z = -lambda (i u sin(theta) + q (1 - cos(theta))). The numerical viscosity q
    follows from each flux's wave speeds (Davis estimates, reading O7):
    * Rusanov: q = |u| + c (the largest signal speed);
    * HLL with S_L = u - c, S_R = u + c: q = (u (S_R + S_L) - 2 S_L S_R) / (S_R - S_L) = c when
      subsonic, and the upwind q = |u| when supersonic;
    * HLLC: q = |u| (it resolves the contact exactly).
    A factor on the Rusanov dissipation, a sign error in HLL's S_L S_R term or a wrong wave speed
    changes q and the decay of the mode by far more than the eps-sized nonlinearity."""
    rk = "ssprk2"
    G, lam, th, c = _entropy_wave_viscosity_run(fl, nd, u, rk)
    q = {"rusanov": abs(u) + c, "hll": c if abs(u) < c else abs(u), "hllc": abs(u)}[fl]
    steps = 40
    z = -lam * (1j * u * math.sin(th) + q * (1 - math.cos(th)))
    Gp = (1 + z + z * z / 2) ** steps
    assert abs(G - Gp) <= 1e-5 * abs(Gp), (G, Gp)
    # the viscosity is resolved: a 10 % change of q moves the decay well beyond the tolerance
    z2 = -lam * (1j * u * math.sin(th) + 1.1 * q * (1 - math.cos(th)))
    assert abs((1 + z2 + z2 * z2 / 2) ** steps - Gp) > 1e-3 * abs(Gp)


def test_entropy_wave_viscosity_ssprk3_polynomial():
    """The same analysis through the three-stage SSP-RK3 (stability polynomial 1 + z + z^2/2 + z^3/6
    for a linear operator) with the Rusanov viscosity."""
    G, lam, th, c = _entropy_wave_viscosity_run("rusanov", 1, 0.5, "ssprk3")
    z = -lam * (1j * 0.5 * math.sin(th) + (0.5 + c) * (1 - math.cos(th)))
    Gp = (1 + z + z * z / 2 + z ** 3 / 6) ** 40
    assert abs(G - Gp) <= 1e-5 * abs(Gp), (G, Gp)


# ---------------------------------------------------------------- reconstruction (Sec. 2.1)
@pytest.mark.parametrize("kind", ["pc", "mc", "weno3"])
def test_recon_linear_data(kind):
    for i in range(-5, 6):
        wm, w0, wp = 2.0 * i - 1.0, 2.0 * i + 1.0, 2.0 * i + 3.0   # w = 2x+1 on integer cells
        fl, fr = oracle.recon(kind, wm, w0, wp)
        if kind == "pc":
            assert fl == w0 and fr == w0
        else:
            assert fl == pytest.approx(2.0 * i, abs=1e-14)
            assert fr == pytest.approx(2.0 * i + 2.0, abs=1e-14)


def test_mc_zero_slope_at_extrema():
    for wm, w0, wp in ((0.0, 1.0, 0.5), (1.0, 0.0, 2.0), (1.0, 1.0, 3.0)):
        fl, fr = oracle.recon("mc", wm, w0, wp)
        assert fl == w0 and fr == w0


def test_mc_limits_to_twice_one_sided_difference():
    # minmod(2 D-, D_c, 2 D+): a small left difference limits the slope to 2 D-
    fl, fr = oracle.recon("mc", 0.9, 1.0, 3.0)
    assert fr - 1.0 == pytest.approx(0.1)
    assert 1.0 - fl == pytest.approx(0.1)


def test_weno3_third_order_face_values():
    # cell averages of sin on a refined grid; face errors at rate ~3 away from extrema (eps = h^2)
    errs, hs = [], []
    for n in (40, 80, 160, 320):
        h = 1.0 / n
        x = np.arange(-1, 2) * h + 0.3
        avg = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h
        fl, fr = oracle.recon("weno3", avg[0], avg[1], avg[2], eps=h * h)
        errs.append(abs(fr - math.sin(0.3 + h / 2)))
        hs.append(n)
    rates = observed_rates(hs, errs)
    assert np.all(rates > 2.7), rates


# ---------------------------------------------------------------- exact Riemann solver pin
def read_golden(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_exact_riemann_matches_toro_table():
    g = read_golden("sod_star_toro_table_4_3_test1.txt")
    R = RiemannExact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    rL, rR = R.star_densities()
    assert R.pstar == pytest.approx(g["p_star"], abs=6e-6)
    assert R.ustar == pytest.approx(g["u_star"], abs=6e-6)
    assert rL == pytest.approx(g["rho_star_left"], abs=6e-6)
    assert rR == pytest.approx(g["rho_star_right"], abs=6e-6)


def test_exact_riemann_rankine_hugoniot_lax():
    R = RiemannExact((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))
    _, rR = R.star_densities()
    S = R.shock_speed_right()
    g = 1.4
    UR = np.array([0.5, 0.0, 0.571 / (g - 1)])
    Us = np.array([rR, rR * R.ustar, R.pstar / (g - 1) + 0.5 * rR * R.ustar**2])
    FR = euler_phys_flux_1d((0.5, 0.0, 0.571))
    Fs = euler_phys_flux_1d((rR, R.ustar, R.pstar))
    np.testing.assert_allclose(Fs - FR, S * (Us - UR), rtol=1e-10)


# ---------------------------------------------------------------- full scheme, 1D Euler
@pytest.mark.parametrize("recon,min_rate,fl", [("pc", 0.45, "hllc"), ("mc", 0.6, "hllc"), ("weno3", 0.6, "hllc"),
                                               ("pc", 0.45, "rusanov"), ("mc", 0.6, "rusanov"),
                                               ("pc", 0.45, "hll"), ("mc", 0.6, "hll")])
def test_sod_converges_to_exact(recon, min_rate, fl):
    R = RiemannExact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    ns, errs = [128, 256, 512, 1024], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="euler", recon=recon, flux=fl, rk="ssprk2",
                             bc="outflow", cfl=0.45)
        U, _, t = oracle.evolve(d, oracle.init(d, "sod"), T=0.2)
        assert t[0] == 0.2
        errs.append(np.abs(U[0, 0, 0, 0] - R.cell_average_density(n, 0.2)).mean())
    assert np.all(np.diff(errs) < 0), errs
    rate = math.log(errs[0] / errs[-1]) / math.log(ns[-1] / ns[0])
    assert rate >= min_rate, (errs, rate)
    if recon == "mc":
        assert errs[-1] < {"hllc": 1e-3, "hll": 1.5e-3, "rusanov": 2e-3}[fl]


@pytest.mark.parametrize("fl", ["hllc", "hll", "rusanov"])
def test_lax_converges_to_exact(fl):
    R = RiemannExact((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))
    ns, errs = [128, 256, 512], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="euler", recon="mc", flux=fl, rk="ssprk2",
                             bc="outflow", cfl=0.45)
        U, _, _ = oracle.evolve(d, oracle.init(d, "lax"), T=0.13)
        errs.append(np.abs(U[0, 0, 0, 0] - R.cell_average_density(n, 0.13)).mean())
    assert np.all(np.diff(errs) < 0), errs
    assert math.log(errs[0] / errs[-1]) / math.log(4) >= 0.6


def test_sod_first_cfl_step_closed_form():
    # at t=0 the fastest signal is the left sound speed sqrt(1.4): dt = cfl dx / sqrt(1.4)
    n = 64
    d = oracle.make_desc(ndim=1, n=(n,), eq="euler", bc="outflow", cfl=0.45)
    U0 = oracle.init(d, "sod")
    s = oracle.max_speed(d, U0)[0]
    assert s == pytest.approx(math.sqrt(1.4) * n, rel=1e-15)
    _, steps, t = oracle.evolve(d, U0, T=1.0, max_steps=1)
    assert steps[0] == 1 and t[0] == pytest.approx(0.45 / n / math.sqrt(1.4), rel=1e-15)


def test_outflow_boundary_flux_balance():
    # before waves reach the ends, only the boundary pressure moves momentum: d(sum m)/dt = pL - pR
    d = oracle.make_desc(ndim=1, n=(200,), eq="euler", recon="mc", flux="hllc", bc="outflow")
    U0 = oracle.init(d, "sod")
    U, _, _ = oracle.evolve(d, U0, T=0.2)
    t0, t1 = oracle.totals(d, U0)[0], oracle.totals(d, U)[0]
    assert abs(t1[0] - t0[0]) < 1e-14
    assert t1[1] - t0[1] == pytest.approx((1.0 - 0.1) * 0.2, rel=1e-12)
    assert abs(t1[2] - t0[2]) < 1e-13


@pytest.mark.parametrize("recon", ["mc", "weno3"])
def test_reflective_walls_conserve_mass_energy(recon):
    d = oracle.make_desc(ndim=1, n=(100,), eq="euler", recon=recon, flux="hllc", bc="reflective")
    U0 = oracle.init(d, "sod")
    U, _, _ = oracle.evolve(d, U0, T=0.6)   # waves hit the walls
    t0, t1 = oracle.totals(d, U0)[0], oracle.totals(d, U)[0]
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    assert abs(t1[2] - t0[2]) <= 1e-13 * abs(t0[2])
    assert abs(t1[1] - t0[1]) > 1e-3        # the walls do push momentum


# ---------------------------------------------------------------- Burgers
@pytest.mark.parametrize("recon,rk,fl,lo_rate", [("pc", "ssprk2", "rusanov", 0.8), ("mc", "ssprk2", "hll", 1.8),
                                                 ("weno3", "ssprk3", "rusanov", 2.5)])
def test_burgers_pre_shock_convergence(recon, rk, fl, lo_rate):
    ns, errs = [32, 64, 128, 256], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="burgers", recon=recon, flux=fl, rk=rk, bc="periodic",
                             cfl=0.45, weno_eps_dx2=True)
        U, _, _ = oracle.evolve(d, oracle.init(d, "burgers_sine"), T=0.1)
        errs.append(np.abs(U[0, 0, 0, 0] - burgers_sine_cell_averages(n, 0.1)).mean())
    rates = observed_rates(ns, errs)
    assert rates[-1] >= lo_rate, rates


def test_burgers_multid_directions_equal_the_1d_run():
    """Burgers in 2D/3D applies u^2/2 along every direction: data varying only along y (2D) or z
    (3D) evolves exactly as the 1D run along x."""
    n = 32
    kw = dict(eq="burgers", recon="weno3", flux="rusanov", rk="ssprk3", cfl=0.45)
    d1 = oracle.make_desc(ndim=1, n=(n,), bc="periodic", **kw)
    u1 = oracle.init(d1, "burgers_sine")
    r1, s1, _ = oracle.evolve(d1, u1, T=0.08)
    d2 = oracle.make_desc(ndim=2, n=(3, n), bc="periodic", **kw)
    U2 = np.repeat(u1[:, :, :, :, :].reshape(1, 1, 1, n, 1), 3, axis=4)
    r2, s2, _ = oracle.evolve(d2, U2, T=0.08)
    d3 = oracle.make_desc(ndim=3, n=(2, 3, n), bc="periodic", **kw)
    U3 = np.broadcast_to(u1.reshape(1, 1, n, 1, 1), (1, 1, n, 3, 2)).copy()
    r3, s3, _ = oracle.evolve(d3, U3, T=0.08)
    assert s1[0] == s2[0] == s3[0]
    for i in range(3):
        assert np.array_equal(r2[0, 0, 0, :, i], r1[0, 0, 0, 0])
    for i in range(2):
        for j in range(3):
            assert np.array_equal(r3[0, 0, :, j, i], r1[0, 0, 0, 0])


def test_burgers_reflective_walls_match_the_odd_periodic_solution():
    """u0 = sin(2 pi x) is odd about x = 0 and x = 1, so mirrored ghosts with negated u (reading
    O11 for the scalar law) equal the periodic ghosts: the reflective run equals the periodic one,
    through the shock at t > 1/(2 pi)."""
    n = 64
    kw = dict(eq="burgers", recon="mc", flux="hll", rk="ssprk2", cfl=0.45)
    dp = oracle.make_desc(ndim=1, n=(n,), bc="periodic", **kw)
    dr = oracle.make_desc(ndim=1, n=(n,), bc="reflective", **kw)
    u0 = oracle.init(dp, "burgers_sine")
    rp, _, _ = oracle.evolve(dp, u0, T=0.3)
    rr, _, _ = oracle.evolve(dr, u0, T=0.3)
    np.testing.assert_allclose(rr, rp, rtol=0, atol=1e-13)


def test_burgers_init_exact_cell_averages():
    d = oracle.make_desc(ndim=1, n=(16,), eq="burgers")
    U = oracle.init(d, "burgers_sine")[0, 0, 0, 0]
    np.testing.assert_allclose(U, burgers_sine_cell_averages(16, 0.0), atol=1e-15)


# ---------------------------------------------------------------- 2D smooth vortex
def vortex_errors(recon, rk, rvars, ns, eps2, T=1.0, fl="hllc"):
    errs = []
    for n in ns:
        d = oracle.make_desc(ndim=2, n=(n, n), lo=(0, 0), hi=(10, 10), eq="euler", recon=recon, rvars=rvars,
                             flux=fl, rk=rk, bc="periodic", cfl=0.4, weno_eps_dx2=eps2)
        U, _, _ = oracle.evolve(d, oracle.init(d, "vortex", center=(5, 5)), T=T)
        E = oracle.init(d, "vortex", center=(5 + T, 5 + T))
        errs.append(np.abs(U[0, 0] - E[0, 0]).mean())
    return errs


def test_vortex_init_quadrature_vs_scipy():
    from scipy import integrate
    d = oracle.make_desc(ndim=2, n=(20, 20), lo=(0, 0), hi=(10, 10), eq="euler")
    U = oracle.init(d, "vortex", center=(5, 5))
    g, beta = 1.4, 5.0

    def rho(y, x):
        r2 = (x - 5) ** 2 + (y - 5) ** 2
        T = 1 - (g - 1) * beta**2 / (8 * g * math.pi**2) * math.exp(1 - r2)
        return T ** (1 / (g - 1))
    for (i, j) in ((10, 10), (9, 11), (3, 12)):
        ref, _ = integrate.dblquad(rho, i * 0.5, (i + 1) * 0.5, j * 0.5, (j + 1) * 0.5, epsabs=1e-13)
        assert U[0, 0, 0, j, i] == pytest.approx(ref / 0.25, rel=1e-9)


@pytest.mark.parametrize("fl", ["hllc", "rusanov"])
def test_vortex_mc_second_order(fl):
    # MC + Rusanov + SSP-RK2 is the adjoint configuration's scheme
    rates = observed_rates([32, 64, 128], vortex_errors("mc", "ssprk2", "prim", [32, 64, 128], False, fl=fl))
    assert np.all(rates >= 1.8), rates


def test_vortex_tecno2_second_order():
    """TECNO2 (two-point entropy-conservative flux plus ENO2 entropy-stable diffusion, cell values,
    SSP-RK3) on the smooth 2D vortex: second order in both directions (observed rates 1.86 then
    1.96 on 64 -> 128 -> 256); a first-order diffusion (a dropped ENO slope) would give rate 1."""
    ns = [64, 128, 256]
    rates = observed_rates(ns, vortex_errors("pc", "ssprk3", "prim", ns, False, fl="tecno2"))
    assert np.all(rates >= 1.8) and rates[-1] >= 1.9, rates


@pytest.mark.slow
def test_vortex_weno3_third_order():
    ns = [64, 128, 256]
    rates = observed_rates(ns, vortex_errors("weno3", "ssprk3", "cons", ns, True))
    assert np.all(rates >= 2.5) and rates[-1] >= 2.7, rates


# ---------------------------------------------------------------- conservation, symmetry
def test_kh_periodic_conservation():
    n = 48
    d = oracle.make_desc(ndim=2, n=(n, n), eq="euler", recon="weno3", flux="hllc", rk="ssprk3",
                         bc="periodic", cfl=0.4)
    th = oracle.theta_splitmix(0, 1, 20)
    U0 = oracle.init(d, "kh", theta=th)
    U, steps, _ = oracle.evolve(d, U0, T=0.3)
    assert steps[0] > 20
    t0, t1 = oracle.totals(d, U0)[0], oracle.totals(d, U)[0]
    dV = 1.0 / n**2
    # O14 reading: relative to sum_i |U_v,i| dV (taken over both states: m_y starts identically 0)
    scale = np.maximum(np.abs(U0[0]).reshape(4, -1).sum(axis=1), np.abs(U[0]).reshape(4, -1).sum(axis=1)) * dV
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def test_kh_init_band_mass_closed_form():
    # the band between the two displaced interfaces has width exactly 0.5 in every column
    n = 64
    d = oracle.make_desc(ndim=2, n=(n, n), eq="euler")
    th = oracle.theta_splitmix(7, 3, 20)
    U = oracle.init(d, "kh", B=3, theta=th)
    tot = oracle.totals(d, U)
    g = 1.4
    for b in range(3):
        assert tot[b, 0] == pytest.approx(0.5 * 2.0 + 0.5 * 1.0, rel=1e-14)
        assert tot[b, 1] == pytest.approx(0.5 * 2.0 * -0.5 + 0.5 * 1.0 * 0.5, rel=1e-13)
        assert tot[b, 2] == 0.0
        E_in = 2.5 / (g - 1) + 0.5 * 2.0 * 0.25
        E_out = 2.5 / (g - 1) + 0.5 * 1.0 * 0.25
        assert tot[b, 3] == pytest.approx(0.5 * E_in + 0.5 * E_out, rel=1e-14)
    # perturbation moves the interface: samples differ, columns differ
    assert not np.allclose(U[0], U[1])


def _lower_interface(U, dy):
    """Per column, the lower interface height 0.25 + Y recovered from the density: below y = 1/2
    the column holds 1 per unit height plus 1 more between the interface and 1/2, so
    sum_{y < 1/2} rho dy = 0.5 + (0.5 - (0.25 + Y)) = 0.75 - Y."""
    half = U.shape[-2] // 2
    return 0.75 - U[0, 0, :, :half, :].sum(axis=1) * dy + 0.25        # [nz, nx]: 0.25 + Y


def test_kh_single_mode_interface_position_2d():
    """One Fourier mode (a_3 = 0.7, b_3 = 0.4): the interface recovered from each column's mass is
    0.25 + 0.01 a_3 sin(2 pi 3 x_c + b_3) at the cell centres x_c (reading O2)."""
    nx, ny = 24, 40
    d = oracle.make_desc(ndim=2, n=(nx, ny), eq="euler")
    th = np.zeros((1, 20))
    th[0, 2], th[0, 12] = 0.7, 0.4
    U = oracle.init(d, "kh", 1, th)
    y_if = _lower_interface(U, 1.0 / ny)[0]
    xc = (np.arange(nx) + 0.5) / nx
    np.testing.assert_allclose(y_if, 0.25 + 0.01 * 0.7 * np.sin(2 * np.pi * 3 * xc + 0.4), rtol=0, atol=1e-14)


def test_kh_3d_band_mass_and_single_mode_interface():
    """3D slab (reading O2): the band keeps width 1/2 in every (x, z) column, so mass, momenta and
    energy take the 2D closed forms for any parameters; one mode a_nm (n = 2 along x, m = 3 along z,
    n-major index 8 (n - 1) + (m - 1)) puts the interface at 0.25 + 0.01 a sin(2 pi (2 x + 3 z) + b)."""
    n = (12, 16, 10)
    d = oracle.make_desc(ndim=3, n=n, eq="euler")
    th = oracle.theta_splitmix(3, 2, 128)
    U = oracle.init(d, "kh", 2, th)
    tot = oracle.totals(d, U)
    g = 1.4
    for b in range(2):
        assert tot[b, 0] == pytest.approx(1.5, rel=1e-14)
        assert tot[b, 1] == pytest.approx(-0.25, rel=1e-13)
        assert tot[b, 2] == 0.0 and tot[b, 3] == 0.0
        assert tot[b, 4] == pytest.approx(0.5 * (2.5 / (g - 1) + 0.25) + 0.5 * (2.5 / (g - 1) + 0.125), rel=1e-14)
    one = np.zeros((1, 128))
    j = 8 * (2 - 1) + (3 - 1)
    one[0, j], one[0, 64 + j] = 0.9, 1.1
    U1 = oracle.init(d, "kh", 1, one)
    y_if = _lower_interface(U1, 1.0 / n[1])                       # [nz, nx]
    xc = (np.arange(n[0]) + 0.5) / n[0]
    zc = (np.arange(n[2]) + 0.5) / n[2]
    Y = 0.01 * 0.9 * np.sin(2 * np.pi * (2 * xc[None, :] + 3 * zc[:, None]) + 1.1)
    np.testing.assert_allclose(y_if, 0.25 + Y, rtol=0, atol=1e-14)


def test_sod_mirror_symmetry():
    n = 128
    d = oracle.make_desc(ndim=1, n=(n,), eq="euler", recon="weno3", flux="hllc", rk="ssprk3", bc="outflow")
    U0 = oracle.init(d, "sod")
    Um0 = U0[..., ::-1].copy()
    Um0[:, 1] *= -1
    U, _, _ = oracle.evolve(d, U0, T=0.15)
    Um, _, _ = oracle.evolve(d, Um0, T=0.15)
    mir = U[..., ::-1].copy()
    mir[:, 1] *= -1
    np.testing.assert_allclose(Um, mir, rtol=1e-13, atol=1e-13)


def test_rotation_symmetry_2d():
    n = 24
    d = oracle.make_desc(ndim=2, n=(n, n), eq="euler", recon="mc", flux="hllc", rk="ssprk2", bc="periodic")
    th = oracle.theta_splitmix(3, 1, 20)
    U0 = oracle.init(d, "kh", theta=th)
    # rotate: swap x <-> y and u <-> v
    R0 = U0.transpose(0, 1, 2, 4, 3)[:, [0, 2, 1, 3]].copy()
    U, _, _ = oracle.evolve(d, U0, T=0.05)
    Rt, _, _ = oracle.evolve(d, R0, T=0.05)
    np.testing.assert_allclose(Rt, U.transpose(0, 1, 2, 4, 3)[:, [0, 2, 1, 3]], rtol=1e-13, atol=1e-13)


def test_rotation_symmetry_3d():
    """The 3D slab rotated about y (x <-> z with u <-> w) evolves to the rotated result: every
    direction uses its own normal velocity and spacing."""
    n = (10, 12, 10)
    d = oracle.make_desc(ndim=3, n=n, eq="euler", recon="weno3", flux="hllc", rk="ssprk3", bc="periodic", cfl=0.3)
    th = oracle.theta_splitmix(11, 1, 128)
    U0 = oracle.init(d, "kh", theta=th)
    U0[:, 3] = 0.2 * U0[:, 0]                       # a z-velocity too, so that w moves with x
    R0 = U0.transpose(0, 1, 4, 3, 2)[:, [0, 3, 2, 1, 4]].copy()
    U, _, _ = oracle.evolve(d, U0, T=0.02)
    Rt, _, _ = oracle.evolve(d, R0, T=0.02)
    np.testing.assert_allclose(Rt, U.transpose(0, 1, 4, 3, 2)[:, [0, 3, 2, 1, 4]], rtol=1e-13, atol=1e-13)


def test_cfl_speed_takes_each_direction_with_its_own_spacing():
    """Reading O9 with O1: s = max_k (|u_k| + c) / dx_k on a 2 x 1 domain with dx = 2 dy."""
    d = oracle.make_desc(ndim=2, n=(10, 10), hi=(2.0, 1.0, 1.0), eq="euler")
    rho, u, v, p = 1.3, 0.3, 0.1, 0.9
    U = np.zeros((1, 4, 1, 10, 10))
    U[:, 0], U[:, 1], U[:, 2] = rho, rho * u, rho * v
    U[:, 3] = p / 0.4 + 0.5 * rho * (u * u + v * v)
    c = math.sqrt(1.4 * p / rho)
    s = oracle.max_speed(d, U)[0]
    assert s == pytest.approx(max((u + c) / 0.2, (v + c) / 0.1), rel=1e-14)
    assert s == pytest.approx((v + c) / 0.1, rel=1e-14)


def test_1d_extruded_in_y_equals_1d_bitwise():
    n = 64
    d1 = oracle.make_desc(ndim=1, n=(n,), eq="euler", recon="weno3", flux="hllc", rk="ssprk3", bc="outflow")
    d2 = oracle.make_desc(ndim=2, n=(n, 4), eq="euler", recon="weno3", flux="hllc", rk="ssprk3",
                          bc=[("outflow", "outflow"), ("periodic", "periodic")])
    U1 = oracle.init(d1, "sod")
    U2 = np.zeros((1, 4, 1, 4, n))
    U2[:, 0] = U1[:, 0]
    U2[:, 1] = U1[:, 1]
    U2[:, 3] = U1[:, 2]
    r1, s1, _ = oracle.evolve(d1, U1, T=0.1)
    r2, s2, _ = oracle.evolve(d2, U2, T=0.1)
    assert s1[0] == s2[0]
    for j in range(4):
        assert np.array_equal(r2[0, 0, 0, j], r1[0, 0, 0, 0])
        assert np.array_equal(r2[0, 1, 0, j], r1[0, 1, 0, 0])
        assert np.array_equal(r2[0, 3, 0, j], r1[0, 2, 0, 0])
        assert np.all(r2[0, 2, 0, j] == 0.0)


def test_free_stream_preserved():
    for nd in (1, 2, 3):
        d = oracle.make_desc(ndim=nd, n=(5, 4, 3), eq="euler", recon="weno3", flux="hllc")
        W = np.concatenate([[1.3], np.arange(1, nd + 1) * 0.3, [0.9]])
        U = np.zeros(oracle.state_shape(d, 1))
        Uc = oracle.prim_to_cons(d, W)
        for v in range(nd + 2):
            U[0, v] = Uc[v]
        assert np.all(oracle.rhs(d, U) == 0.0)


# ---------------------------------------------------------------- MC statistics (Sec. 2.2)
def test_welford_vs_two_pass_long_double():
    d = oracle.make_desc(ndim=2, n=(8, 6), eq="euler")
    B = 37
    rng = np.random.default_rng(77)
    U = np.zeros((B, 4, 1, 6, 8))
    U[:, 0] = rng.uniform(0.5, 2.0, (B, 1, 6, 8))
    U[:, 1] = rng.uniform(-1, 1, (B, 1, 6, 8))
    U[:, 2] = rng.uniform(-1, 1, (B, 1, 6, 8))
    U[:, 3] = rng.uniform(3, 5, (B, 1, 6, 8))
    cnt, mean, M2 = oracle.welford(d, U[:20])
    cnt, mean, M2 = oracle.welford(d, U[20:], cnt, mean, M2)     # streaming over batches
    assert cnt == B
    L = U.astype(np.longdouble)
    W = np.stack([L[:, 0], L[:, 1] / L[:, 0], L[:, 2] / L[:, 0],
                  0.4 * (L[:, 3] - 0.5 * (L[:, 1] ** 2 + L[:, 2] ** 2) / L[:, 0])], axis=1).reshape(B, 4, -1)
    mu = W.mean(axis=0)
    var = ((W - mu) ** 2).sum(axis=0) / (B - 1)
    np.testing.assert_allclose(mean, mu.astype(float), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(M2 / (B - 1), var.astype(float), rtol=1e-13)


def test_welford_integer_data_exact():
    d = oracle.make_desc(ndim=1, n=(3,), eq="burgers")
    B = 101
    U = np.arange(B, dtype=float)[:, None, None, None, None] * np.ones((1, 1, 1, 1, 3))
    cnt, mean, M2 = oracle.welford(d, U)
    assert np.all(mean == (B - 1) / 2)
    assert np.all(M2 / (B - 1) == B * (B + 1) / 12)


# ---------------------------------------------------------------- kinetic energy (reading O16)
def test_kinetic_energy_closed_forms():
    """KE = sum_i |m_i|^2 / (2 rho_i) dV. (i) The unperturbed KH data on 8 rows puts both interfaces
    on cell faces (y = 2/8, 6/8), so the band (area 1/2, rho 2, u -1/2) carries 1/2 * 2 * 1/4 * 1/2
    = 1/8 and the rest (rho 1, u 1/2) 1/2 * 1 * 1/4 * 1/2 = 1/16: KE = 3/16 exactly. (ii) Uniform
    states with every velocity component nonzero: KE = rho |u|^2 / 2 times the domain's volume."""
    d = oracle.make_desc(ndim=2, n=(4, 8), eq="euler")
    U = oracle.init(d, "kh", theta=np.zeros((1, 20)))
    assert oracle.kinetic_energy(d, U)[0] == 0.1875
    for nd, vel, vol in ((1, [0.7], 2.0), (2, [0.3, 0.4], 2.0), (3, [0.3, 0.4, 1.2], 2.0)):
        d = oracle.make_desc(ndim=nd, n=(5, 4, 3), hi=(2.0, 1.0, 1.0), eq="euler")
        W = np.concatenate([[2.0], vel, [0.9]])
        Uc = oracle.prim_to_cons(d, W)
        U = np.zeros(oracle.state_shape(d, 1))
        for v in range(nd + 2):
            U[0, v] = Uc[v]
        assert oracle.kinetic_energy(d, U)[0] == pytest.approx(0.5 * 2.0 * np.dot(vel, vel) * vol, rel=1e-14)


# ---------------------------------------------------------------- exact discrete gradient
def _ke_after(d, th, dt, n):
    U = oracle.init(d, "kh", theta=th.reshape(1, 20))
    U, _, _ = oracle.evolve(d, U, fixed_dt=dt, n_steps=n)
    return oracle.kinetic_energy(d, U)[0]


@pytest.mark.parametrize("fl,rk", [("rusanov", "ssprk2"), ("hllc", "ssprk3")])
def test_dual_gradient_vs_central_differences(fl, rk):
    n = 16
    d = oracle.make_desc(ndim=2, n=(n, n), eq="euler", recon="mc", flux=fl, rk=rk, bc="periodic", cfl=0.4)
    dt, _ = oracle.fixed_dt_kh(n, 1.0, 0.4)
    steps = 12
    th = oracle.theta_splitmix(99, 1, 20)[0]
    J, g = oracle.ke_grad_kh2d(d, th, dt, steps)
    assert J == pytest.approx(_ke_after(d, th, dt, steps), rel=1e-15)
    fd = np.zeros(20)
    for j in range(20):
        h = 1e-6 * max(1.0, abs(th[j]))
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd[j] = (_ke_after(d, tp, dt, steps) - _ke_after(d, tm, dt, steps)) / (2 * h)
    # FD straddles limiter / wave-case kinks near some faces; the dual value is the exact
    # active-branch derivative, so compare relative to the gradient's size
    assert np.abs(g - fd).max() <= 1e-4 * np.abs(g).max(), np.abs(g - fd).max() / np.abs(g).max()
    np.testing.assert_allclose(g, fd, rtol=1e-3, atol=1e-5 * np.abs(g).max())
    assert np.abs(g).max() > 1e-4


def test_dual_gradient_dot_direction():
    n = 12
    d = oracle.make_desc(ndim=2, n=(n, n), eq="euler", recon="mc", flux="rusanov", rk="ssprk2")
    dt, _ = oracle.fixed_dt_kh(n, 1.0, 0.4)
    th = oracle.theta_splitmix(5, 1, 20)[0]
    v = rng.standard_normal(20)
    J, g = oracle.ke_grad_kh2d(d, th, dt, 8)
    J1, dJ = oracle.ke_dir_kh2d(d, th, v, dt, 8)
    assert J1 == J
    assert dJ == pytest.approx(np.dot(g, v), rel=1e-10)


def _tube(rho, p, u=None):
    """1D Euler state [1, 3, 1, 1, n] from primitive rows (gamma = 1.4)."""
    rho, p = np.asarray(rho, float), np.asarray(p, float)
    u = np.zeros_like(rho) if u is None else np.asarray(u, float)
    U = np.zeros((1, 3, 1, 1, rho.size))
    U[0, 0, 0, 0] = rho
    U[0, 1, 0, 0] = rho * u
    U[0, 2, 0, 0] = p / 0.4 + 0.5 * rho * u * u
    return U


@pytest.mark.parametrize("rvars", ["prim", "cons"])
def test_positivity_fallback_face_states(rvars):
    """Reading O6: WENO3 on (4, 1, 50) overshoots below zero at the right face of the middle cell
    (the smooth left stencil extrapolates -1/2*4 + 3/2*1 < 0 with weight near one); that face then
    carries the cell's own state in every variable, while the left face keeps its reconstruction."""
    d = oracle.make_desc(ndim=1, n=(5,), eq="euler", recon="weno3", rvars=rvars, flux="hllc", bc="periodic")
    _, fr_rho = oracle.recon("weno3", 4.0, 1.0, 50.0)
    assert fr_rho < 0.0
    # density overshoot
    U = _tube([4.0, 1.0, 50.0, 1.0, 1.0], [1.0] * 5)
    cell = oracle.cons_to_prim(d, U[0, :, 0, 0, 1])        # the cell's own primitive state
    Wl, Wr = oracle.face_states(d, U[0], (1,), 0)
    np.testing.assert_array_equal(Wr, cell)
    assert Wl[0] > 0 and Wl[2] > 0 and Wl[0] != cell[0]
    if rvars == "prim":
        fl_rho, _ = oracle.recon("weno3", 4.0, 1.0, 50.0)
        assert Wl[0] == fl_rho and Wl[1] == 0.0 and Wl[2] == cell[2]
    # pressure overshoot (density uniform): same fallback
    U = _tube([1.0] * 5, [4.0, 1.0, 50.0, 1.0, 1.0])
    cell = oracle.cons_to_prim(d, U[0, :, 0, 0, 1])
    Wl, Wr = oracle.face_states(d, U[0], (1,), 0)
    np.testing.assert_array_equal(Wr, cell)
    assert Wl[2] > 0 and Wl[2] != cell[2]
    # the mirrored data falls back at the mirrored (left) face
    U = _tube([1.0, 1.0, 50.0, 1.0, 4.0], [1.0] * 5)
    cell = oracle.cons_to_prim(d, U[0, :, 0, 0, 3])
    Wl, Wr = oracle.face_states(d, U[0], (3,), 0)
    np.testing.assert_array_equal(Wl, cell)
    assert Wr[0] > 0 and Wr[0] != cell[0]


def test_positivity_fallback_keeps_runs_physical_and_mirror_symmetric():
    """Steep density and pressure contrasts whose WENO3 faces overshoot below zero: the run stays
    physical (a non-positive face state would give a NaN sound speed) and the mirrored data gives
    the mirrored result."""
    d = oracle.make_desc(ndim=1, n=(12,), eq="euler", recon="weno3", rvars="prim", flux="hllc", rk="ssprk3",
                         bc="periodic", cfl=0.3)
    rho = np.array([4.0, 1.0, 50.0, 1.0, 1.0, 30.0, 0.5, 0.5, 2.0, 1.0, 80.0, 1.0])
    p = np.array([1.0, 1.0, 1.0, 4.0, 0.2, 40.0, 1.0, 1.0, 1.0, 2.0, 1.0, 1.0])
    u = np.linspace(-0.3, 0.4, 12)
    U = _tube(rho, p, u)
    out, steps, _ = oracle.evolve(d, U, T=math.inf, max_steps=6)
    assert steps[0] == 6 and np.all(np.isfinite(out))
    Um = _tube(rho[::-1], p[::-1], -u[::-1])
    outm, _, _ = oracle.evolve(d, Um, T=math.inf, max_steps=6)
    mir = outm[..., ::-1].copy()
    mir[:, 1] *= -1
    np.testing.assert_allclose(mir, out, rtol=1e-12, atol=1e-12)


def _mix_after(d, th, dt, steps):
    U = oracle.init(d, "kh", 1, th[None, :])
    U, _, _ = oracle.evolve(d, U, fixed_dt=dt, n_steps=steps)
    return float(oracle.mixing_width(d, U)[0])


def test_mixing_width_closed_forms():
    """W = sum 4 (rho - 1)(2 - rho) dV: 0 where the unperturbed interfaces lie on cell faces
    (ny = 8), the area of the two half-filled rows where they cut cells in half (ny = 10: 2 dy),
    and the whole domain for a half-and-half state."""
    zero = np.zeros((1, 20))
    d8 = oracle.make_desc(ndim=2, n=(12, 8), eq="euler")
    assert oracle.mixing_width(d8, oracle.init(d8, "kh", 1, zero))[0] == 0.0
    d10 = oracle.make_desc(ndim=2, n=(12, 10), eq="euler")
    assert oracle.mixing_width(d10, oracle.init(d10, "kh", 1, zero))[0] == pytest.approx(0.2, rel=1e-14)
    U = np.zeros((1, 4, 1, 10, 12))
    U[:, 0] = 1.5
    U[:, 3] = 2.5 / 0.4
    assert oracle.mixing_width(d10, U)[0] == pytest.approx(1.0, rel=1e-14)


def test_mixing_width_dual_gradient_vs_central_differences():
    n = 16
    d = oracle.make_desc(ndim=2, n=(n, n), eq="euler", recon="mc", flux="rusanov", rk="ssprk2", bc="periodic",
                         cfl=0.4)
    dt, _ = oracle.fixed_dt_kh(n, 1.0, 0.4)
    steps = 10
    th = oracle.theta_splitmix(41, 1, 20)[0]
    J, g = oracle.obs_grad_kh2d(d, th, dt, steps, "mixing")
    assert J == pytest.approx(_mix_after(d, th, dt, steps), rel=1e-13)
    fd = np.zeros(20)
    for j in range(20):
        h = 1e-6 * max(1.0, abs(th[j]))
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd[j] = (_mix_after(d, tp, dt, steps) - _mix_after(d, tm, dt, steps)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-4 * np.abs(g).max(), np.abs(g - fd).max() / np.abs(g).max()
    assert np.abs(g).max() > 1e-3
    # the kinetic-energy case is the same dual run
    Jk, gk = oracle.obs_grad_kh2d(d, th, dt, steps, "ke")
    Jk2, gk2 = oracle.ke_grad_kh2d(d, th, dt, steps)
    assert Jk == Jk2 and np.array_equal(gk, gk2)


def test_fixed_dt_reading_at_512():
    dt, n = oracle.fixed_dt_kh(512, 1.0, 0.4)
    assert n == 3035 and dt == 1.0 / 3035


def test_stats_merge_equals_two_pass_of_union():
    d = oracle.make_desc(ndim=1, n=(7,), eq="euler")
    rng = np.random.default_rng(3)
    U = np.zeros((23, 3, 1, 1, 7))
    U[:, 0] = rng.uniform(0.5, 2, (23, 1, 1, 7))
    U[:, 1] = rng.uniform(-1, 1, (23, 1, 1, 7))
    U[:, 2] = rng.uniform(3, 5, (23, 1, 1, 7))
    parts = [U[:9], U[9:10], U[10:]]
    acc = (0, np.zeros((3, 7)), np.zeros((3, 7)))
    for p in parts:
        acc = oracle.stats_merge(d, acc, oracle.welford(d, p))
    c, m, M2 = acc
    L = U.astype(np.longdouble)
    W = np.stack([L[:, 0], L[:, 1] / L[:, 0], 0.4 * (L[:, 2] - 0.5 * L[:, 1] ** 2 / L[:, 0])], axis=1).reshape(23, 3, -1)
    mu = W.mean(axis=0)
    var = ((W - mu) ** 2).sum(axis=0) / 22
    assert c == 23
    np.testing.assert_allclose(m, mu.astype(float), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(M2 / 22, var.astype(float), rtol=1e-13)


# ---------------------------------------------------------------------------------------------
# Multilevel Monte Carlo estimator (Sec. 2.2)
# ---------------------------------------------------------------------------------------------
def test_mlmc_hand_worked_two_level_example():
    """Scalar quantity (no conversion); level 0 one cell (dV = 1), level 1 two cells (dV = 1/2).
    Level 0: samples 1, 3           -> Y mean 2, var 2; Z = 1, 9 -> mean 5.
    Level 1: fine (2, 4), (0, 2); coarse 1, 3 (prolongated to both cells):
             Y = (1, 3), (-3, -1)   -> mean (-1, 1), var (8, 8)
             Z = (4-1, 16-1), (0-9, 4-9) = (3, 15), (-9, -5) -> mean (-3, 5).
    Estimate: mean = 2 + (-1, 1) = (1, 3); second = 5 + (-3, 5) = (2, 10); var = (2-1, 10-9) = (1, 1).
    Level sums: level 0 (2, 2, 2); level 1 ((-1+1)/2, (1+1)/2, (8+8)/2) = (0, 1, 8)."""
    l0 = (np.array([1.0, 3.0]).reshape(2, 1, 1, 1, 1), None, 1.0)
    fine = np.array([[2.0, 4.0], [0.0, 2.0]]).reshape(2, 1, 1, 1, 2)
    coarse = np.array([1.0, 3.0]).reshape(2, 1, 1, 1, 1)
    mean, var, sums = oracle.mlmc_estimate([l0, (fine, coarse, 0.5)], euler=False)
    np.testing.assert_array_equal(mean.reshape(-1), [1.0, 3.0])
    np.testing.assert_array_equal(var.reshape(-1), [1.0, 1.0])
    np.testing.assert_array_equal(sums.reshape(2, 3), [[2.0, 2.0, 2.0], [0.0, 1.0, 8.0]])


def test_mlmc_prolongation_is_the_containing_coarse_cell():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(3, 1, 2, 3))
    y = oracle.prolongate(x, (1, 4, 9))
    for q in range(3):
        for j in range(4):
            for i in range(9):
                assert y[q, 0, j, i] == x[q, 0, j // 2, i // 3]
    with pytest.raises(ValueError):
        oracle.prolongate(x, (1, 5, 9))


@pytest.mark.parametrize("euler", [False, True])
def test_mlmc_telescopes_to_the_finest_level_when_levels_share_samples(euler):
    """If every level's coarse companion is exactly the previous level's own sample set, the sum
    collapses: the estimate is the plain sample mean (and biased variance) of the finest level.
    Grids refine by 2 in y and 3 in x, so a transposed prolongation cannot pass."""
    rng = np.random.default_rng(11)
    M = 5
    shapes = [(1, 2, 3), (1, 4, 9), (1, 8, 27)]

    def fields(shape):
        if not euler:
            return rng.normal(size=(M, 1) + shape)
        U = np.empty((M, 4) + shape)
        rho = rng.uniform(0.5, 2.0, (M,) + shape)
        u = rng.uniform(-1, 1, (M, 2) + shape)
        p = rng.uniform(0.5, 3.0, (M,) + shape)
        U[:, 0] = rho
        U[:, 1:3] = rho[:, None] * u
        U[:, 3] = p / 0.4 + 0.5 * rho * (u * u).sum(axis=1)
        return U

    A = [fields(s) for s in shapes]
    levels = [(A[0], None, 1.0)] + [(A[l], A[l - 1], 1.0) for l in (1, 2)]
    mean, var, _ = oracle.mlmc_estimate(levels, euler=euler)
    if euler:   # quantities from the (pinned) C++ cell conversion
        d = oracle.make_desc(ndim=2, n=(27, 8), eq="euler")
        q = np.empty_like(A[2])
        for b in range(M):
            for j in range(8):
                for i in range(27):
                    q[b, :, 0, j, i] = oracle.cons_to_prim(d, A[2][b, :, 0, j, i])
    else:
        q = A[2]
    mu = q.mean(axis=0)
    np.testing.assert_allclose(mean, mu, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(var, ((q - mu) ** 2).mean(axis=0), rtol=1e-9, atol=1e-12)


def test_mlmc_single_level_is_plain_monte_carlo():
    """One level without companion: mean and level variance sum are the sample mean and the
    unbiased sample variance integrated over the grid (integer data, exact)."""
    U = np.array([[1.0, 2.0], [3.0, 6.0], [8.0, 1.0]]).reshape(3, 1, 1, 1, 2)
    mean, var, sums = oracle.mlmc_estimate([(U, None, 0.5)], euler=False)
    np.testing.assert_array_equal(mean.reshape(-1), [4.0, 3.0])
    # second moments (1+9+64)/3, (4+36+1)/3 minus squared means 16, 9
    np.testing.assert_allclose(var.reshape(-1), [74 / 3 - 16, 41 / 3 - 9], rtol=1e-15)
    # unbiased variances: ((9+1+16)/2, (1+9+4)/2) = (13, 7); sums x dV = 0.5
    np.testing.assert_allclose(sums.reshape(3), [3.5, 3.5, 10.0], rtol=1e-15)


# ---------------------------------------------------------------------------------------------
# Quasi Monte Carlo parameters (Halton)
# ---------------------------------------------------------------------------------------------
def test_halton_textbook_values_and_primes():
    assert [oracle.radical_inverse(n, 2) for n in range(1, 8)] == [1 / 2, 1 / 4, 3 / 4, 1 / 8, 5 / 8, 3 / 8, 7 / 8]
    assert [oracle.radical_inverse(n, 3) for n in range(1, 7)] == [1 / 3, 2 / 3, 1 / 9, 4 / 9, 7 / 9, 2 / 9]
    ps = oracle.primes(128)
    assert ps[:10] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]
    assert ps[19] == 71 and ps[127] == 719   # the 20th and the 128th prime


@pytest.mark.parametrize("p,k", [(2, 10), (3, 6), (71, 2)])
def test_halton_first_p_to_the_k_points_fill_the_lattice(p, k):
    """phi_p permutes {0, 1/p^k, ..., (p^k - 1)/p^k} over n = 0 .. p^k - 1 (digit reversal)."""
    vals = sorted(oracle.radical_inverse(n, p) for n in range(p ** k))
    assert vals == [i / p ** k for i in range(p ** k)]


def test_halton_theta_ranges_and_shift():
    th = oracle.theta_halton(50, 20)
    assert np.all(th[:, :10] > 0) and np.all(th[:, :10] < 1)
    assert np.all(th[:, 10:] > 0) and np.all(th[:, 10:] < 2 * math.pi)
    # sample b uses index b + 1: the amplitude a_1 (base 2) runs through 1/2, 1/4, 3/4, ...
    assert list(th[:3, 0]) == [0.5, 0.25, 0.75]
    sh = oracle.theta_halton(50, 20, seed=7, shifted=True)
    s0 = (oracle.splitmix64(7 ^ (1 << 63)) >> 11) * 2.0 ** -53
    assert sh[0, 0] == (0.5 + s0) - (1.0 if 0.5 + s0 >= 1.0 else 0.0)
    assert np.all(sh[:, :10] >= 0) and np.all(sh[:, :10] < 1)
    assert np.array_equal(oracle.theta_halton(5, 20, first_index=3), th[3:8])


# ---------------------------------------------------------------------------------------------
# Point PDFs and structure functions
# ---------------------------------------------------------------------------------------------
# lattice points of Z^2 and Z^3 in the closed ball of radius r (Gauss circle / sphere counts,
# OEIS A000328 and A000605)
BALL2 = [1, 5, 13, 29, 49, 81, 113, 149, 197, 253, 317, 377, 441, 529, 613, 709, 797]
BALL3 = [1, 7, 33, 123, 257]


@pytest.mark.parametrize("nd", [2, 3])
def test_structure_function_of_a_single_spike_counts_lattice_points(nd):
    """q = 1 at one cell, 0 elsewhere, periodic: a pair differs exactly when one end is the spike,
    so the ball sum of |dq| (and of dq^2) is twice the number of nonzero offsets in the ball."""
    R = 16 if nd == 2 else 4
    n = 2 * R + 3
    shape = (1, 1) + ((1, n, n) if nd == 2 else (n, n, n))
    U = np.zeros(shape)
    U[(0, 0) + ((0, 5, 9) if nd == 2 else (4, 5, 9))] = 1.0
    ball = BALL2 if nd == 2 else BALL3
    for p in (1, 2):
        cnt, sums = oracle.structure_function_sums(U, 0, p, R, (1.0,) * nd, (True, True, True), euler=False)
        assert cnt == 1
        np.testing.assert_array_equal(np.cumsum(sums), [2 * (ball[r] - 1) for r in range(1, R + 1)])


def test_structure_function_of_a_linear_profile_without_wrap():
    """q_i = i on n cells, non-periodic: shell r holds the offsets +-r with 2 (n - r) valid pairs
    of difference r: sums r^p 2 (n - r) dx^2; S_p(r) then follows in closed form."""
    n, R, dx = 40, 6, 0.025
    U = np.arange(n, dtype=float).reshape(1, 1, 1, 1, n)
    for p in (1, 2):
        cnt, sums = oracle.structure_function_sums(U, 0, p, R, (dx,), (False,), euler=False)
        expect = np.array([r ** p * 2 * (n - r) * dx * dx for r in range(1, R + 1)])
        np.testing.assert_allclose(sums, expect, rtol=1e-15)
        S = oracle.structure_function(cnt, sums, p)
        np.testing.assert_allclose(S, np.cumsum(expect) ** (1.0 / p), rtol=1e-15)
    flat = np.full((2, 1, 1, 1, n), 3.5)
    assert not oracle.structure_function_sums(flat, 0, 2, R, (dx,), (True,), euler=False)[1].any()


def test_point_pdf_bins_by_definition():
    # integer data: 0.5 on a bin edge goes up, the top edge and NaN go to the overflow bin
    vals = np.array([-1.0, 0.0, 0.49, 0.5, 0.99, 1.0, np.nan, 0.25])
    U = vals.reshape(8, 1, 1, 1, 1)
    c = oracle.point_pdf(U, 0, [0], 0.0, 1.0, 2, euler=False)
    np.testing.assert_array_equal(c, [[1, 3, 2, 2]])


# ---------------------------------------------------------------------------------------------
# Algorithmic flop counts (counting scalar)
# ---------------------------------------------------------------------------------------------
def test_flop_counts_of_the_pieces_by_hand():
    """Counted by hand from the formulas: MC: two differences, 2 dm, (dm + dp)/2 (two), 2 dp, two
    faces w0 -+ s/2 (two each) = 10. WENO3, per face: two candidates (3 each), two smoothness
    indicators (3 each), two weights d/((eps + b)(eps + b)) (4 each), the weighted average (5) =
    25; both faces 50. cons->prim 2D: two velocities (2), |m|^2 (3), /2, /rho, E - ., (gamma - 1),
    * (5) = 10; 3D: 3 + 5 + 5 = 13."""
    d2 = oracle.make_desc(ndim=2, n=(8, 8), eq="euler", recon="mc", flux="rusanov", rvars="prim", rk="ssprk2")
    c = oracle.count_flops(d2)
    assert c["recon"] == 10 and c["cons_to_prim"] == 10
    d2w = oracle.make_desc(ndim=2, n=(8, 8), eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3")
    c = oracle.count_flops(d2w)
    assert c["recon"] == 50
    # per cell-stage: conversion + per direction (4 reconstructions + one flux) + divergence/RK;
    # per cell-update: three stages
    assert c["per_cell_stage"] == c["cons_to_prim"] + 2 * (4 * c["recon"] + c["flux"]) + c["div_rk"]
    assert c["per_cell_update"] == 3 * c["per_cell_stage"]
    d3 = oracle.make_desc(ndim=3, n=(8, 8, 8), eq="euler", recon="pc", flux="rusanov", rvars="prim", rk="ssprk3")
    c = oracle.count_flops(d3)
    assert c["recon"] == 0 and c["cons_to_prim"] == 13


def test_bench_flop_constant_matches_the_count():
    """bench.py reports its FP32-ALU fraction with this count (it does not call the oracle)."""
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "bench.py")).read()
    m = re.search(r"FLOPS_PER_CELL_UPDATE_2D_WENO3_HLLC_RK3 = (\d+)", src)
    assert m, "bench.py must state the flop count"
    d = oracle.make_desc(ndim=2, n=(8, 8), eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3")
    assert int(m.group(1)) == oracle.count_flops(d)["per_cell_update"]


def test_joint_pdf_and_correlator_by_hand():
    # two quantities (scalar data in two "variables" read without conversion) at two cells, three samples
    U = np.array([[[1.0, 4.0], [0.2, 0.9]],
                  [[2.0, 5.0], [0.6, 0.1]],
                  [[3.0, 6.0], [0.7, 0.4]]]).reshape(3, 2, 1, 1, 2)
    # q0 bins on [0, 4) with 2 bins: 1 -> 1, 2 -> 2, 3 -> 2, 4, 5, 6 -> overflow 3
    # q1 bins on [0, 1) with 2 bins: 0.2 -> 1, 0.6 -> 2, 0.7 -> 2, 0.9 -> 2, 0.1 -> 1, 0.4 -> 1
    c = oracle.joint_pdf(U, 0, 1, [0, 1], 0.0, 4.0, 2, 0.0, 1.0, 2, euler=False)
    expect = np.zeros((2, 4, 4), dtype=np.int64)
    expect[0, 1, 1] = 1      # (1, 0.2)
    expect[0, 2, 2] = 2      # (2, 0.6), (3, 0.7)
    expect[1, 3, 2] = 1      # (4, 0.9)
    expect[1, 3, 1] = 2      # (5, 0.1), (6, 0.4)
    np.testing.assert_array_equal(c, expect)
    # marginals of the joint PDF are the point PDFs
    np.testing.assert_array_equal(c.sum(axis=2), oracle.point_pdf(U, 0, [0, 1], 0.0, 4.0, 2, euler=False))
    # correlators of q0: <x0> = 2, <x0 x1> = (4 + 10 + 18)/3, <x0 x0 x1> = (4 + 20 + 54)/3
    n, sums = oracle.correlator(U, 0, [[0], [0, 1], [0, 0, 1]], euler=False)
    assert n == 3
    np.testing.assert_array_equal(sums, [6.0, 32.0, 78.0])


def test_bench_workload_flop_constants_match_the_count():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for name, flops in bench.WORKLOAD_FLOPS.items():
        desc = dict(bench.WORKLOADS[name]["desc"])
        if "levels" in desc:
            desc["n"] = desc.pop("levels")[0][0]
        d = oracle.make_desc(**desc)
        assert oracle.count_flops(d)["per_cell_update"] == flops, name


# ---------------------------------------------------------------- more fluxes (Sec. 2.1): Roe, Godunov,
# entropy conservative; ENO reconstruction
def _entropy_vars(W, g=1.4):
    """Entropy variables of S = -rho s / (g - 1), s = ln(p rho^-g), and the entropy-flux potential
    psi_k = rho u_k, for a primitive state [rho, u_1..u_d, p]."""
    W = np.asarray(W, float)
    r, u, p = W[0], W[1:-1], W[-1]
    s = math.log(p) - g * math.log(r)
    v = np.concatenate([[(g - s) / (g - 1) - r * np.dot(u, u) / (2 * p)], r * u / p, [-r / p]])
    return v, r * u


@pytest.mark.parametrize("fl", ["roe", "godunov", "ec"])
@pytest.mark.parametrize("nd", [1, 2, 3])
def test_new_fluxes_consistency(fl, nd):
    d = oracle.make_desc(ndim=nd, n=(4, 4, 4), eq="euler", flux=fl)
    g = 1.4
    for W in random_prim(nd, rng, 20):
        for k in range(nd):
            r, vel, p = W[0], W[1:1 + nd], W[1 + nd]
            E = p / (g - 1) + 0.5 * r * np.dot(vel, vel)
            ref = np.concatenate([[r * vel[k]], r * vel[k] * vel + p * (np.arange(nd) == k), [vel[k] * (E + p)]])
            np.testing.assert_allclose(oracle.flux(d, k, W, W), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("fl", ["roe", "godunov", "ec"])
def test_new_fluxes_mirror_symmetry(fl):
    nd = 2
    d = oracle.make_desc(ndim=nd, n=(4, 4), eq="euler", flux=fl)
    for _ in range(20):
        WL, WR = random_prim(nd, rng, 2)
        for k in range(nd):
            M = np.ones(nd + 2)
            M[1 + k] = -1
            np.testing.assert_allclose(oracle.flux(d, k, WL, WR), -M * oracle.flux(d, k, M * WR, M * WL),
                                       rtol=1e-12, atol=1e-12)


def test_godunov_flux_is_the_flux_of_the_exact_riemann_solution():
    """The Godunov flux equals the physical flux of the exact Riemann solution sampled at x/t = 0,
    taken from the independent test-side solver (Toro's pressure function, tests/exact.py): shocks,
    rarefactions (including transonic ones), contacts on either side of the interface."""
    d = oracle.make_desc(ndim=1, n=(4,), eq="euler", flux="godunov")
    cases = [((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)), ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571)),
             ((1.0, 0.75, 1.0), (0.125, 0.0, 0.1)), ((1.0, -0.5, 0.4), (1.0, 0.5, 0.4)),
             ((5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.0950)), ((1.0, -19.59745, 1000.0), (1.0, -19.59745, 0.01))]
    r = np.random.default_rng(5)
    for _ in range(40):
        cases.append(((r.uniform(0.2, 3), r.uniform(-1.5, 1.5), r.uniform(0.2, 4)),
                      (r.uniform(0.2, 3), r.uniform(-1.5, 1.5), r.uniform(0.2, 4))))
    for WL, WR in cases:
        R = RiemannExact(WL, WR)
        rho, u, p = (float(a[0]) for a in R.sample(np.array([0.0])))
        ref = euler_phys_flux_1d((rho, u, p))
        np.testing.assert_allclose(oracle.flux(d, 0, WL, WR), ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_godunov_tangential_velocity_follows_the_contact():
    d = oracle.make_desc(ndim=2, n=(4, 4), eq="euler", flux="godunov")
    WL, WR = [1.0, 0.3, 0.7, 1.0], [0.5, 0.3, -0.4, 1.0]   # a pure contact moving right: upwind left
    F = oracle.flux(d, 0, WL, WR)
    assert F[2] == pytest.approx(1.0 * 0.3 * 0.7, rel=1e-13)
    WL, WR = [1.0, -0.3, 0.7, 1.0], [0.5, -0.3, -0.4, 1.0]
    F = oracle.flux(d, 0, WL, WR)
    assert F[2] == pytest.approx(0.5 * -0.3 * -0.4, rel=1e-13)


def test_roe_resolves_isolated_contacts_and_shocks_exactly():
    """Roe's linearisation satisfies A(U_L, U_R)(U_R - U_L) = F_R - F_L, so a jump that is a single
    wave of the exact problem is upwinded exactly: a stationary contact gives zero mass flux, and
    the two sides of the Lax problem's right shock (Rankine-Hugoniot-connected, from the exact
    solver) give the flux of the upwind side."""
    d = oracle.make_desc(ndim=2, n=(4, 4), eq="euler", flux="roe")
    F = oracle.flux(d, 0, [3.0, 0.0, 0.0, 1.3], [0.25, 0.0, 0.0, 1.3])
    assert abs(F[0]) <= 1e-15 and F[1] == pytest.approx(1.3, rel=1e-15) and abs(F[3]) <= 1e-15
    R = RiemannExact((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))
    _, rs = R.star_densities()
    d1 = oracle.make_desc(ndim=1, n=(4,), eq="euler", flux="roe")
    WS, WR = (rs, R.ustar, R.pstar), (0.5, 0.0, 0.571)
    assert R.shock_speed_right() > 0
    np.testing.assert_allclose(oracle.flux(d1, 0, WS, WR), euler_phys_flux_1d(WS), rtol=1e-9)
    # the same shock moving left (mirror): upwind is the right side
    np.testing.assert_allclose(oracle.flux(d1, 0, (0.5, 0.0, 0.571), (rs, -R.ustar, R.pstar)),
                               euler_phys_flux_1d((rs, -R.ustar, R.pstar)), rtol=1e-9)
    # a moving shear wave (equal rho and p, normal velocity 0.3, tangential jump): upwind (left)
    # flux, as Godunov's exact flux gives it; a 3D shear across both tangential directions too
    dg = oracle.make_desc(ndim=2, n=(4, 4), eq="euler", flux="godunov")
    WL, WR = [1.2, 0.3, 0.7, 0.9], [1.2, 0.3, -0.4, 0.9]
    np.testing.assert_allclose(oracle.flux(d, 0, WL, WR), oracle.flux(dg, 0, WL, WR), rtol=1e-13, atol=1e-15)
    g = 1.4
    E = 0.9 / (g - 1) + 0.5 * 1.2 * (0.09 + 0.49)
    np.testing.assert_allclose(oracle.flux(d, 0, WL, WR), [1.2 * 0.3, 1.2 * 0.09 + 0.9, 1.2 * 0.3 * 0.7, 0.3 * (E + 0.9)],
                               rtol=1e-13)
    d3 = oracle.make_desc(ndim=3, n=(4, 4, 4), eq="euler", flux="roe")
    WL, WR = [1.2, 0.7, 0.1, -0.3, 0.9], [1.2, -0.2, 0.5, -0.3, 0.9]
    F = oracle.flux(d3, 2, WL, WR)                                   # u_z = -0.3 < 0: upwind is the right
    E = 0.9 / (g - 1) + 0.5 * 1.2 * (0.04 + 0.25 + 0.09)
    np.testing.assert_allclose(F, [1.2 * -0.3, 1.2 * -0.3 * -0.2, 1.2 * -0.3 * 0.5, 1.2 * 0.09 + 0.9, -0.3 * (E + 0.9)],
                               rtol=1e-13)


@pytest.mark.parametrize("nd", [1, 2, 3])
def test_entropy_conservative_flux_satisfies_tadmors_condition(nd):
    """(v_R - v_L) . F(W_L, W_R) = psi_R - psi_L for the entropy pair (-rho s/(g-1), -rho u s/(g-1)):
    the defining identity of an entropy-conservative two-point flux, on random pairs (including
    nearly equal states, where the logarithmic means switch to their series), and F(L,R) = F(R,L)."""
    d = oracle.make_desc(ndim=nd, n=(4, 4, 4), eq="euler", flux="ec")
    pairs = [tuple(random_prim(nd, rng, 2)) for _ in range(30)]
    for _ in range(10):
        W = random_prim(nd, rng, 1)[0]
        pairs.append((W, W * (1 + 1e-4 * rng.standard_normal(nd + 2))))
    for WL, WR in pairs:
        vL, psiL = _entropy_vars(WL)
        vR, psiR = _entropy_vars(WR)
        for k in range(nd):
            F = oracle.flux(d, k, WL, WR)
            lhs = np.dot(vR - vL, F)
            scale = np.abs(vR - vL) @ np.abs(F) + abs(psiR[k]) + abs(psiL[k])
            assert abs(lhs - (psiR[k] - psiL[k])) <= 1e-12 * scale
            np.testing.assert_allclose(oracle.flux(d, k, WR, WL), F, rtol=1e-13, atol=1e-14)


def test_burgers_new_fluxes():
    """Burgers: Godunov is the exact solution's flux at x/t = 0 (shock with speed (uL+uR)/2, or the
    rarefaction's sonic point); Roe with Harten's fix equals it on shocks and one-sided waves; the
    entropy-conservative flux (uL^2 + uL uR + uR^2)/6 satisfies Tadmor's condition for the entropy
    u^2/2 (entropy variable u, flux potential psi = u f - q = u^3/6): (uR - uL) F = uR^3/6 - uL^3/6."""
    dg = oracle.make_desc(ndim=1, n=(4,), eq="burgers", flux="godunov")
    dr = oracle.make_desc(ndim=1, n=(4,), eq="burgers", flux="roe")
    de = oracle.make_desc(ndim=1, n=(4,), eq="burgers", flux="ec")
    r = np.random.default_rng(9)
    for _ in range(200):
        uL, uR = r.uniform(-2, 2, 2)
        Fg = oracle.flux(dg, 0, [uL], [uR])[0]
        assert Fg == pytest.approx(burgers_godunov(uL, uR), rel=1e-15, abs=1e-300)
        if uL > uR or uL * uR > 0:
            assert oracle.flux(dr, 0, [uL], [uR])[0] == pytest.approx(Fg, rel=1e-14, abs=1e-15)
        Fe = oracle.flux(de, 0, [uL], [uR])[0]
        assert (uR - uL) * Fe == pytest.approx((uR**3 - uL**3) / 6, rel=1e-13, abs=1e-15)
    # transonic rarefaction: the fix keeps Roe's flux below the expansion-shock value (fL + fR)/2 - 0
    uL, uR = -0.5, 1.0
    assert oracle.flux(dr, 0, [uL], [uR])[0] < 0.5 * (0.5 * uL * uL + 0.5 * uR * uR) - 0.5 * 0.25 * (uR - uL)


@pytest.mark.parametrize("fl,recon,min_rate", [("roe", "pc", 0.45), ("roe", "mc", 0.6), ("godunov", "pc", 0.45),
                                               ("godunov", "mc", 0.6), ("hllc", "eno2", 0.6)])
def test_sod_converges_with_roe_godunov_eno(fl, recon, min_rate):
    R = RiemannExact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    ns, errs = [128, 256, 512, 1024], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="euler", recon=recon, flux=fl, rk="ssprk2", bc="outflow", cfl=0.45)
        U, _, _ = oracle.evolve(d, oracle.init(d, "sod"), T=0.2)
        errs.append(np.abs(U[0, 0, 0, 0] - R.cell_average_density(n, 0.2)).mean())
    assert np.all(np.diff(errs) < 0), errs
    assert math.log(errs[0] / errs[-1]) / math.log(ns[-1] / ns[0]) >= min_rate, errs


def test_roe_entropy_fix_on_a_transonic_rarefaction():
    """Toro's test 1 (left state moving right at 0.75) has a sonic point inside the left
    rarefaction, where the unfixed Roe flux keeps an entropy-violating expansion shock. With the
    Harten-Hyman fix the first-order scheme converges to the exact solution, and near the sonic
    point the density jumps between neighbouring cells shrink with the mesh."""
    R = RiemannExact((1.0, 0.75, 1.0), (0.125, 0.0, 0.1))
    ns, errs, jumps = [200, 400, 800], [], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="euler", recon="pc", flux="roe", rk="ssprk2", bc="outflow", cfl=0.45)
        U0 = np.zeros((1, 3, 1, 1, n))
        x = (np.arange(n) + 0.5) / n
        rho = np.where(x < 0.3, 1.0, 0.125)
        u = np.where(x < 0.3, 0.75, 0.0)
        p = np.where(x < 0.3, 1.0, 0.1)
        U0[0, 0, 0, 0], U0[0, 1, 0, 0], U0[0, 2, 0, 0] = rho, rho * u, p / 0.4 + 0.5 * rho * u * u
        U, _, _ = oracle.evolve(d, U0, T=0.2)
        ex = R.cell_average_density(n, 0.2, x0=0.3)
        errs.append(np.abs(U[0, 0, 0, 0] - ex).mean())
        # the sonic point sits at x = 0.3 at every time (x/t = 0 inside the fan)
        i0 = int(0.3 * n)
        jumps.append(np.abs(np.diff(U[0, 0, 0, 0, i0 - 3:i0 + 4])).max())
    assert np.all(np.diff(errs) < 0) and math.log(errs[0] / errs[-1]) / math.log(4) >= 0.5, errs
    assert jumps[-1] < 0.6 * jumps[0] and jumps[-1] < 0.02, jumps


def test_eno2_reconstruction():
    """ENO2 takes the smoother of the two linear candidates (the smaller one-sided difference):
    exact on linear data, the smaller slope at a kink, and second order on smooth Burgers data."""
    for i in range(-3, 4):
        fl, fr = oracle.recon("eno2", 2.0 * i - 1.0, 2.0 * i + 1.0, 2.0 * i + 3.0)
        assert fl == pytest.approx(2.0 * i) and fr == pytest.approx(2.0 * i + 2.0)
    fl, fr = oracle.recon("eno2", 0.0, 1.0, 1.5)     # differences 1 and 0.5: slope 0.5
    assert (fl, fr) == (0.75, 1.25)
    fl, fr = oracle.recon("eno2", 0.9, 1.0, 3.0)     # differences 0.1 and 2: slope 0.1
    assert fl == pytest.approx(0.95) and fr == pytest.approx(1.05)
    fl, fr = oracle.recon("eno2", 1.0, 0.0, 2.0)     # extremum: differences -1, 2: slope -1 (not limited to 0)
    assert (fl, fr) == (0.5, -0.5)
    ns, errs = [32, 64, 128, 256], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="burgers", recon="eno2", flux="godunov", rk="ssprk2", bc="periodic",
                             cfl=0.4)
        U, _, _ = oracle.evolve(d, oracle.init(d, "burgers_sine"), T=0.1)
        errs.append(np.abs(U[0, 0, 0, 0] - burgers_sine_cell_averages(n, 0.1)).mean())
    assert observed_rates(ns, errs)[-1] >= 1.8, errs


def _smooth_euler_1d(n):
    x = (np.arange(n) + 0.5) / n
    tp = 2 * np.pi
    rho, drho = 1 + 0.2 * np.sin(tp * x), 0.2 * tp * np.cos(tp * x)
    u, du = 0.5 + 0.1 * np.cos(tp * x), -0.1 * tp * np.sin(tp * x)
    p, dp = 1 + 0.1 * np.sin(tp * x + 1), 0.1 * tp * np.cos(tp * x + 1)
    return rho, u, p, drho, du, dp


@pytest.mark.parametrize("fl,order", [("ec", 2), ("ec4", 4)])
def test_entropy_conservative_schemes_order_and_entropy_balance(fl, order):
    """On point values of a smooth periodic state, L(U)_i approximates -d/dx f(U(x_i)) (closed form
    by the product rule) at second (two-point flux) and fourth order (LeFloch-Mercier-Rohde
    combination), and the semi-discrete entropy is conserved: sum_i v(U_i) . L(U)_i = 0."""
    g = 1.4
    errs, ns = [], [16, 32, 64, 128]
    for n in ns:
        rho, u, p, dr, du, dp = _smooth_euler_1d(n)
        d = oracle.make_desc(ndim=1, n=(n,), eq="euler", flux=fl, bc="periodic")
        U = np.zeros((1, 3, 1, 1, n))
        E = p / (g - 1) + 0.5 * rho * u * u
        U[0, 0, 0, 0], U[0, 1, 0, 0], U[0, 2, 0, 0] = rho, rho * u, E
        L = oracle.rhs(d, U)[0, :, 0, 0]
        dE = dp / (g - 1) + 0.5 * dr * u * u + rho * u * du
        exact = -np.array([dr * u + rho * du, dr * u * u + 2 * rho * u * du + dp, du * (E + p) + u * (dE + dp)])
        errs.append(np.abs(L - exact).max())
        W = np.stack([rho, u, p])
        V = np.array([_entropy_vars(W[:, i])[0] for i in range(n)]).T
        bal = (V * L).sum()
        assert abs(bal) <= 1e-12 * (np.abs(V) * np.abs(L)).sum(), bal
    rates = observed_rates(ns, errs)
    assert np.all(rates[1:] >= order - 0.2), (errs, rates)


def test_entropy_conservative_burgers_and_2d_balance():
    """Burgers: sum_i u_i L_i = 0 for both entropy-conservative schemes (entropy u^2/2); 2D Euler on
    a random smooth periodic state: sum_i v_i . L_i = 0 with both directions."""
    n = 40
    x = (np.arange(n) + 0.5) / n
    for fl in ("ec", "ec4"):
        d = oracle.make_desc(ndim=1, n=(n,), eq="burgers", flux=fl, bc="periodic")
        U = (0.3 + np.sin(2 * np.pi * x) + 0.2 * np.cos(6 * np.pi * x)).reshape(1, 1, 1, 1, n)
        L = oracle.rhs(d, U)
        assert abs((U * L).sum()) <= 1e-13 * (np.abs(U) * np.abs(L)).sum()
    from inputs import euler_state
    U = euler_state(1, 2, (12, 10), seed=4)
    for fl in ("ec", "ec4"):
        d = oracle.make_desc(ndim=2, n=(12, 10), eq="euler", flux=fl, bc="periodic")
        L = oracle.rhs(d, U)[0].reshape(4, -1)
        W = oracle.cons_to_prim(d, U[0].reshape(4, -1).T.copy()).T if False else None
        Uc = U[0].reshape(4, -1)
        rho, mx, my, E = Uc
        p = 0.4 * (E - 0.5 * (mx * mx + my * my) / rho)
        V = np.array([_entropy_vars([rho[i], mx[i] / rho[i], my[i] / rho[i], p[i]])[0] for i in range(rho.size)]).T
        assert abs((V * L).sum()) <= 1e-12 * (np.abs(V) * np.abs(L)).sum()


# ---------------------------------------------------------------- TECNO2: entropy-stable diffusion added to
# the two-point entropy-conservative flux (Fjordholm-Mishra-Tadmor), Sec. 2.1's entropy-conservative
# fluxes made entropy stable
def _cons_from_prim(W, g=1.4):
    W = np.asarray(W, float)
    r, u, p = W[0], W[1:-1], W[-1]
    return np.concatenate([[r], r * u, [p / (g - 1) + 0.5 * r * np.dot(u, u)]])


def _prim_from_cons(U, g=1.4):
    U = np.asarray(U, float)
    r, m, E = U[0], U[1:-1], U[-1]
    return np.concatenate([[r], m / r, [(g - 1) * (E - 0.5 * np.dot(m, m) / r)]])


def _phys_flux_cons(U, k, g=1.4):
    W = _prim_from_cons(U, g)
    r, u, p = W[0], W[1:-1], W[-1]
    return np.concatenate([[r * u[k]], r * u[k] * u + p * (np.arange(u.size) == k), [u[k] * (U[-1] + p)]])


def _num_jacobian(f, x, h=1e-6):
    J = np.zeros((f(x).size, x.size))
    for c in range(x.size):
        e = np.zeros(x.size)
        e[c] = h * max(1.0, abs(x[c]))
        J[:, c] = (f(x + e) - f(x - e)) / (2 * e[c])
    return J


@pytest.mark.parametrize("nd", [1, 2, 3])
def test_tecno_entropy_variables_and_scaled_eigenvectors(nd):
    """The oracle's entropy variables equal the independent formula; at a state W the scaled
    eigenvectors satisfy Rs Rs^T = dU/dv (the inverse of the numerical Jacobian dv/dU, Barth's
    scaling) and are eigenvectors of the numerical flux Jacobian dF_k/dU with eigenvalues of
    magnitude lam (u_k - c, u_k, ..., u_k + c). A wrong scale factor fails the first check, a wrong
    column or eigenvalue the second."""
    d = oracle.make_desc(ndim=nd, n=(4, 4, 4), eq="euler", flux="tecno2")
    nv = nd + 2
    for W in random_prim(nd, rng, 6):
        np.testing.assert_allclose(oracle.entropy_vars(d, W), _entropy_vars(W)[0], rtol=1e-13, atol=1e-13)
        U0 = _cons_from_prim(W)
        dUdv = np.linalg.inv(_num_jacobian(lambda U: _entropy_vars(_prim_from_cons(U))[0], U0))
        for k in range(nd):
            Rs, lam = oracle.tecno_matrix(d, k, W, W)
            np.testing.assert_allclose(Rs @ Rs.T, dUdv, rtol=1e-6, atol=1e-6 * np.abs(dUdv).max())
            A = _num_jacobian(lambda U: _phys_flux_cons(U, k), U0)
            AR = A @ Rs
            c = math.sqrt(1.4 * W[-1] / W[0])
            expect = sorted([abs(W[1 + k] - c), abs(W[1 + k] + c)] + [abs(W[1 + k])] * (nv - 2))
            assert np.allclose(sorted(lam), expect, rtol=1e-13)
            for m in range(nv):
                res = min(np.linalg.norm(AR[:, m] - lam[m] * Rs[:, m]), np.linalg.norm(AR[:, m] + lam[m] * Rs[:, m]))
                assert res <= 1e-6 * (np.linalg.norm(AR[:, m]) + np.linalg.norm(Rs[:, m])), (k, m, res)


def test_tecno_burgers_flux_hand_values():
    """Burgers (v = u, Rs = 1, Lambda = max(|u_i|, |u_i+1|)): F = (u_i^2 + u_i u_i+1 + u_i+1^2)/6 -
    1/2 Lambda <<u>>, <<u>> the jump of the ENO2 faces. Hand-evaluated stencils: (0, 0, 1, 3)
    (differences 0, 1, 2: slopes 0 and 1, jump 1/2); (0, 0, 1, 0.5) (slopes 0 and -0.5, jump 5/4);
    (2, 1, 1, 1) (slopes 0 and 0, jump 0: no diffusion). Taking the larger difference, dropping the
    1/2 or flipping the sign each changes a value."""
    d = oracle.make_desc(ndim=1, n=(8,), eq="burgers", flux="tecno2")
    cases = [((0.0, 0.0, 1.0, 3.0), 1 / 6 - 0.5 * 1.0 * 0.5), ((0.0, 0.0, 1.0, 0.5), 1 / 6 - 0.5 * 1.0 * 1.25),
             ((2.0, 1.0, 1.0, 1.0), 0.5), ((-3.0, -1.0, 0.0, 0.0), 1 / 6 - 0.5 * 1.0 * 0.5)]
    for u, ref in cases:
        F = oracle.tecno_flux(d, 0, np.array(u).reshape(4, 1))[0]
        assert F == pytest.approx(ref, rel=1e-14, abs=1e-15), (u, F, ref)


@pytest.mark.parametrize("nd", [1, 2, 3])
def test_tecno_consistency_and_mirror_symmetry(nd):
    d = oracle.make_desc(ndim=nd, n=(4, 4, 4), eq="euler", flux="tecno2")
    for _ in range(10):
        W4 = random_prim(nd, rng, 4)
        for k in range(nd):
            W = W4[0]
            ref = _phys_flux_cons(_cons_from_prim(W), k)
            np.testing.assert_allclose(oracle.tecno_flux(d, k, np.stack([W] * 4)), ref, rtol=1e-13, atol=1e-13)
            M = np.ones(nd + 2)
            M[1 + k] = -1
            F = oracle.tecno_flux(d, k, np.stack(W4))
            Fm = oracle.tecno_flux(d, k, np.stack([M * W4[3], M * W4[2], M * W4[1], M * W4[0]]))
            np.testing.assert_allclose(F, -M * Fm, rtol=1e-12, atol=1e-12)


def test_tecno_is_entropy_stable():
    """The semi-discrete entropy rate sum_i v_i . L_i, zero for the entropy-conservative flux, is
    negative with TECNO2's diffusion on rough periodic data (random 1D and 2D Euler states, random
    Burgers data), and zero on a constant state."""
    from inputs import euler_state
    for trial in range(3):
        n = 24
        U = euler_state(1, 1, (n,), seed=60 + trial)
        for fl, sign in (("ec", 0), ("tecno2", -1)):
            d = oracle.make_desc(ndim=1, n=(n,), eq="euler", flux=fl, bc="periodic")
            L = oracle.rhs(d, U)[0].reshape(3, -1)
            Uc = U[0].reshape(3, -1)
            V = np.array([_entropy_vars(_prim_from_cons(Uc[:, i]))[0] for i in range(n)]).T
            rate, scale = (V * L).sum(), (np.abs(V) * np.abs(L)).sum()
            if sign == 0:
                assert abs(rate) <= 1e-12 * scale
            else:
                assert rate < -1e-4 * scale, (rate, scale)
    U = euler_state(1, 2, (12, 10), seed=5)
    d = oracle.make_desc(ndim=2, n=(12, 10), eq="euler", flux="tecno2", bc="periodic")
    L = oracle.rhs(d, U)[0].reshape(4, -1)
    Uc = U[0].reshape(4, -1)
    V = np.array([_entropy_vars(_prim_from_cons(Uc[:, i]))[0] for i in range(Uc.shape[1])]).T
    assert (V * L).sum() < -1e-4 * (np.abs(V) * np.abs(L)).sum()
    n = 40
    r = np.random.default_rng(7)
    for _ in range(3):
        u = r.uniform(-1, 1, n).reshape(1, 1, 1, 1, n)
        d = oracle.make_desc(ndim=1, n=(n,), eq="burgers", flux="tecno2", bc="periodic")
        L = oracle.rhs(d, u)
        assert (u * L).sum() < -1e-4 * (np.abs(u) * np.abs(L)).sum()
    Uk = np.broadcast_to(_cons_from_prim([1.0, 0.3, 0.9]).reshape(1, 3, 1, 1, 1), (1, 3, 1, 1, 16)).copy()
    d = oracle.make_desc(ndim=1, n=(16,), eq="euler", flux="tecno2", bc="periodic")
    assert np.abs(oracle.rhs(d, Uk)).max() <= 1e-14


def test_tecno_converges_on_sod_and_smooth_burgers():
    """Sod to T = 0.2 against the exact solution (monotone decrease, rate >= 0.6), and the smooth
    Burgers sine before its shock at second order (rate >= 1.8)."""
    R = RiemannExact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    ns, errs = [128, 256, 512, 1024], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="euler", flux="tecno2", rk="ssprk3", bc="outflow", cfl=0.4)
        U, _, _ = oracle.evolve(d, oracle.init(d, "sod"), T=0.2)
        errs.append(np.abs(U[0, 0, 0, 0] - R.cell_average_density(n, 0.2)).mean())
    assert np.all(np.diff(errs) < 0), errs
    assert math.log(errs[0] / errs[-1]) / math.log(ns[-1] / ns[0]) >= 0.6, errs
    ns, errs = [32, 64, 128, 256], []
    for n in ns:
        d = oracle.make_desc(ndim=1, n=(n,), eq="burgers", flux="tecno2", rk="ssprk3", bc="periodic", cfl=0.4)
        U, _, _ = oracle.evolve(d, oracle.init(d, "burgers_sine"), T=0.1)
        errs.append(np.abs(U[0, 0, 0, 0] - burgers_sine_cell_averages(n, 0.1)).mean())
    assert observed_rates(ns, errs)[-1] >= 1.8, errs
