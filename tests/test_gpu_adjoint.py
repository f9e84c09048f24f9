"""Discrete adjoint on the GPU vs the oracle's exact forward-mode (dual number) gradient of the
same discrete map, vs central finite differences, and through torch.autograd."""
import math

import numpy as np
import pytest

import oracle
from harness import gpu_solver, host, need_gpu
from inputs import kh_theta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    from paper_1912_07645_gb300 import build
    build.build()


def gpu_adjoint(cfg, th, T, variant=0, observable="ke"):
    import torch
    import paper_1912_07645_gb300 as alsv
    S = gpu_solver(**cfg)
    alsv.alsv_set_tile_variant(S.ctx, variant)
    S.set_initial_data("kh", theta=torch.from_numpy(th).cuda())
    J, g = S.adjoint(torch.from_numpy(th), T, observable)
    out = host(J), host(g)
    S.close()
    return out


@pytest.mark.parametrize("recon,rvars,rk", [("mc", "prim", "ssprk2"), ("pc", "cons", "ssprk3"),
                                            ("mc", "cons", "ssprk3"), ("pc", "prim", "ssprk2")])
def test_adjoint_fp64_matches_oracle_dual_gradient(recon, rvars, rk):
    n = 32
    cfg = dict(ndim=2, n=(n, n), batch=3, eq="euler", recon=recon, rvars=rvars, flux="rusanov", rk=rk,
               bc="periodic", cfl=0.4, precision="fp64")
    T = 0.1
    dt, nsteps = oracle.fixed_dt_kh(n, T, 0.4)
    assert nsteps == 19      # ragged: 19 steps in checkpoint segments of ceil(sqrt(ceil(1.5 * 19))) = 6
    th = kh_theta(3, 31)
    J, g = gpu_adjoint(cfg, th, T)
    d = oracle.make_desc(**cfg)
    for b in range(3):
        Jo, go = oracle.ke_grad_kh2d(d, th[b], dt, nsteps)
        assert J[b] == pytest.approx(Jo, rel=1e-13)
        assert np.abs(g[b] - go).max() <= 1e-10 * np.abs(go).max(), (g[b], go)


def test_adjoint_replans_when_the_realised_cfl_passes_the_guard():
    """CFL 0.495 from the initial data: the start-up transient pushes the realised CFL number over
    0.5 within the first steps, so the sweep is repeated with n = ceil(T s_seen / cfl); the result
    is the oracle's gradient of the re-planned discrete map."""
    import torch
    import paper_1912_07645_gb300 as alsv
    n, T, cfl = 32, 0.2, 0.495
    cfg = dict(ndim=2, n=(n, n), batch=2, eq="euler", recon="mc", rvars="prim", flux="rusanov", rk="ssprk2",
               bc="periodic", cfl=cfl, precision="fp64")
    th = oracle.theta_splitmix(7, 2, 20)
    d = oracle.make_desc(**cfg)
    dt0, n0 = oracle.fixed_dt_kh(n, T, cfl)
    U = oracle.init(d, "kh", 2, th)
    seen = 0.0
    for _ in range(n0):
        seen = max(seen, float(oracle.max_speed(d, U).max()) * dt0)
        U, _, _ = oracle.evolve(d, U, fixed_dt=dt0, n_steps=1)
    assert seen > 0.5
    n1 = math.ceil(T * (seen / dt0) / cfl)
    S = gpu_solver(**cfg)
    S.set_initial_data("kh", theta=torch.from_numpy(th).cuda())
    J, g = S.adjoint(torch.from_numpy(th), T)
    J, g = host(J), host(g)
    n_gpu, dt_gpu, passes = alsv.alsv_adjoint_get_plan(S.ctx)
    S.close()
    assert (n_gpu, passes) == (n1, 2) and dt_gpu == T / n1
    for b in range(2):
        Jo, go = oracle.ke_grad_kh2d(d, th[b], T / n1, n1)
        assert J[b] == pytest.approx(Jo, rel=1e-13)
        assert np.abs(g[b] - go).max() <= 1e-10 * np.abs(go).max(), (g[b], go)


def test_adjoint_fp64_vs_central_differences():
    import torch
    n = 24
    cfg = dict(ndim=2, n=(n, n), batch=1, eq="euler", recon="mc", rvars="prim", flux="rusanov", rk="ssprk2",
               bc="periodic", cfl=0.4, precision="fp64")
    T = 0.2
    th = kh_theta(1, 5)
    J, g = gpu_adjoint(cfg, th, T)
    S = gpu_solver(**dict(cfg, batch=2))
    fd = np.zeros(20)
    for j in range(20):
        h = 1e-6 * max(1.0, abs(th[0, j]))
        pm = np.concatenate([th, th])
        pm[0, j] += h
        pm[1, j] -= h
        S.set_initial_data("kh", theta=torch.from_numpy(pm).cuda())
        Jpm, _ = S.adjoint(torch.from_numpy(pm), T)
        Jpm = host(Jpm)
        fd[j] = (Jpm[0] - Jpm[1]) / (2 * h)
    S.close()
    assert np.abs(g[0] - fd).max() <= 1e-4 * np.abs(g[0]).max(), (g[0], fd)


@pytest.mark.parametrize("variant", [0, 4])
def test_adjoint_fp32_close_to_fp64_oracle(variant):
    """variant 4: the forward sweeps run the two-sample schedule (the benchmark autotunes it)."""
    n = 32
    cfg = dict(ndim=2, n=(n, n), batch=2, eq="euler", recon="mc", rvars="prim", flux="rusanov", rk="ssprk2",
               bc="periodic", cfl=0.4, precision="fp32")
    T = 0.1
    dt, nsteps = oracle.fixed_dt_kh(n, T, 0.4)
    th = kh_theta(2, 77)
    J, g = gpu_adjoint(cfg, th, T, variant=variant)
    d = oracle.make_desc(**cfg)
    for b in range(2):
        Jo, go = oracle.ke_grad_kh2d(d, th[b], dt, nsteps)
        assert J[b] == pytest.approx(Jo, rel=1e-5)
        assert np.abs(g[b] - go).max() <= 2e-3 * np.abs(go).max()


def test_autograd_function_backward():
    import torch
    from paper_1912_07645_gb300.autograd import kinetic_energy
    n = 16
    cfg = dict(ndim=2, n=(n, n), batch=2, eq="euler", recon="mc", rvars="prim", flux="rusanov", rk="ssprk2",
               bc="periodic", cfl=0.4, precision="fp64")
    th = torch.from_numpy(kh_theta(2, 3)).requires_grad_(True)
    S = gpu_solver(**cfg)
    S.set_initial_data("kh", theta=th.detach().cuda())
    J = kinetic_energy(th, S, 0.1)
    w = torch.tensor([2.0, -0.5], dtype=torch.float64)
    (J * w).sum().backward()
    _, g = S.adjoint(th.detach(), 0.1)
    g = host(g)
    np.testing.assert_allclose(th.grad.numpy(), w.numpy()[:, None] * g, rtol=1e-14)
    S.close()


def test_adjoint_rejects_unsupported_schemes():
    import paper_1912_07645_gb300 as alsv
    S = gpu_solver(ndim=2, n=(16, 16), batch=1, recon="weno3", flux="hllc", precision="fp64")
    with pytest.raises(alsv.AlsvError, match="Rusanov"):
        alsv.alsv_adjoint_workspace_bytes(S.ctx, 0.1)
    S.close()


# ------------------------------------------------------------------ mixing-layer width observable
@pytest.mark.parametrize("recon,rvars,rk,precision", [("mc", "prim", "ssprk2", "fp64"), ("pc", "cons", "ssprk3", "fp64"),
                                                      ("mc", "prim", "ssprk2", "fp32")])
def test_mixing_width_adjoint_matches_oracle_dual_gradient(recon, rvars, rk, precision):
    """W = sum 4 (rho - 1)(2 - rho) dV at T: the adjoint with the mixing-width seed against the
    oracle's dual-number gradient of the same discrete map (FP64 1e-10, FP32 2e-3 of |g|)."""
    n = 32
    cfg = dict(ndim=2, n=(n, n), batch=3, eq="euler", recon=recon, rvars=rvars, flux="rusanov", rk=rk,
               bc="periodic", cfl=0.4, precision=precision)
    T = 0.1
    dt, nsteps = oracle.fixed_dt_kh(n, T, 0.4)
    th = kh_theta(3, 57)
    J, g = gpu_adjoint(cfg, th, T, observable="mixing")
    d = oracle.make_desc(**cfg)
    fp64 = precision == "fp64"
    for b in range(3):
        Jo, go = oracle.obs_grad_kh2d(d, th[b], dt, nsteps, "mixing")
        assert J[b] == pytest.approx(Jo, rel=1e-12 if fp64 else 1e-5)
        assert np.abs(g[b] - go).max() <= (1e-10 if fp64 else 2e-3) * np.abs(go).max(), (g[b], go)
        assert np.abs(go).max() > 1e-3


def test_mixing_width_adjoint_vs_central_differences_and_autograd():
    import torch
    from paper_1912_07645_gb300.autograd import mixing_width
    n = 24
    cfg = dict(ndim=2, n=(n, n), batch=2, eq="euler", recon="mc", rvars="prim", flux="rusanov", rk="ssprk2",
               bc="periodic", cfl=0.4, precision="fp64")
    T = 0.2
    th = kh_theta(1, 8)
    J, g = gpu_adjoint(dict(cfg, batch=1), th, T, observable="mixing")
    S = gpu_solver(**cfg)
    fd = np.zeros(20)
    for j in range(20):
        h = 1e-6 * max(1.0, abs(th[0, j]))
        pm = np.concatenate([th, th])
        pm[0, j] += h
        pm[1, j] -= h
        S.set_initial_data("kh", theta=torch.from_numpy(pm).cuda())
        Jpm, _ = S.adjoint(torch.from_numpy(pm), T, "mixing")
        Jpm = host(Jpm)
        fd[j] = (Jpm[0] - Jpm[1]) / (2 * h)
    assert np.abs(g[0] - fd).max() <= 1e-4 * np.abs(g[0]).max(), (g[0], fd)
    # autograd scales the same gradient; the forward value equals alsv_mixing_width of the state at
    # T that the forward sweep leaves in the context
    thb = torch.from_numpy(np.concatenate([th, th])).requires_grad_(True)
    Jb = mixing_width(thb, S, T)
    Jb.sum().backward()
    np.testing.assert_allclose(thb.grad.numpy()[0], g[0], rtol=1e-12)
    np.testing.assert_allclose(host(S.mixing_width()), host(Jb.detach()), rtol=1e-13)
    S.close()
