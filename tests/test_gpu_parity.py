"""GPU (libalsv.so through the C ABI) vs the FP64 CPU oracle, element by element.

FP64: per cell within 1e-12 relative (cells whose value is below 1e-3 of the variable's largest
magnitude are measured against that magnitude), FMA contraction and reciprocal-multiplication
being the only differences. FP32: within 2e-5 relative L1. Sizes are
small enough for the oracle but span several tiles and ragged tails; the full-size batched
configuration is checked on sampled outputs.
"""
import math

import numpy as np
import pytest

import oracle
from harness import gpu_solver, host, need_gpu, p1_check, p2_check
from inputs import burgers_state, euler_state, kh_theta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    from paper_1912_07645_gb300 import build
    build.build()


def torch_():
    import torch
    return torch


def run_gpu(cfg, init=None, theta=None, U0=None, steps=None, T=None):
    torch = torch_()
    S = gpu_solver(**cfg)
    if U0 is not None:
        S.set_state(torch.from_numpy(np.ascontiguousarray(U0)))
    else:
        th = None if theta is None else torch.from_numpy(np.ascontiguousarray(theta)).cuda()
        S.set_initial_data(init, theta=th)
    nsteps = None
    if steps is not None:
        S.step(steps)
        S.sync()
    if T is not None:
        nsteps = S.evolve_to(T)
    out = host(S.U).reshape(S.level_shape(0)) if S.desc.n_levels <= 1 else None
    t, st = S.time()
    S.close()
    return out, t, st, nsteps


def run_oracle(cfg, init=None, theta=None, U0=None, steps=None, T=None):
    d = oracle.make_desc(**cfg)
    B = cfg.get("batch", 1)
    U = U0.copy() if U0 is not None else oracle.init(d, init, B, theta, center=cfg.get("vortex_center", (5, 5)))
    if steps is not None:
        return oracle.evolve(d, U, T=math.inf, max_steps=steps)
    return oracle.evolve(d, U, T=T)


# ------------------------------------------------------------------ parameters and initial data
def test_theta_splitmix_bitwise():
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    S = gpu_solver(ndim=2, n=(16, 16), batch=64, seed=12345, precision="fp64")
    S.set_initial_data("kh")
    th = torch.empty((64, 20), dtype=torch.float64, device="cuda")
    alsv.alsv_get_parameters(S.ctx, th)
    S.sync()
    assert np.array_equal(host(th), oracle.theta_splitmix(12345, 64, 20))
    S3 = gpu_solver(ndim=3, n=(8, 8, 8), batch=3, seed=77, precision="fp32")
    S3.set_initial_data("kh")
    th3 = torch.empty((3, 128), dtype=torch.float64, device="cuda")
    alsv.alsv_get_parameters(S3.ctx, th3)
    S3.sync()
    assert np.array_equal(host(th3), oracle.theta_splitmix(77, 3, 128))


@pytest.mark.parametrize("sampler", ["halton", "halton_shifted"])
def test_theta_halton_bitwise(sampler):
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    shifted = sampler == "halton_shifted"
    for ndim, n, B, P, off in ((2, (16, 16), 40, 20, 0), (3, (8, 8, 8), 3, 128, 1000)):
        S = gpu_solver(ndim=ndim, n=n, batch=B, seed=99, sampler=sampler, sample_offset=off, precision="fp32")
        S.set_initial_data("kh")
        th = torch.empty((B, P), dtype=torch.float64, device="cuda")
        alsv.alsv_get_parameters(S.ctx, th)
        S.sync()
        ref = oracle.theta_halton(B, P, seed=99, shifted=shifted, first_index=off)
        assert np.array_equal(host(th), ref)
        S.close()


def test_sample_offset_draws_global_parameters():
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    S = gpu_solver(ndim=2, n=(16, 16), batch=8, seed=555, sample_offset=100, precision="fp32")
    S.set_initial_data("kh")
    th = torch.empty((8, 20), dtype=torch.float64, device="cuda")
    alsv.alsv_get_parameters(S.ctx, th)
    assert np.array_equal(host(th), oracle.theta_splitmix(555, 108, 20)[100:])
    S.close()


def test_stats_merge_matches_oracle_and_sharded_ensemble():
    """Two shards of one ensemble (sample_offset), merged in order, equal the whole ensemble."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    from paper_1912_07645_gb300.parallel import merge_in_rank_order
    cfg = dict(ndim=2, n=(40, 36), eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2", bc="periodic",
               cfl=0.4, precision="fp64", seed=8)
    accs, states = [], []
    for off, B in ((0, 5), (5, 7)):
        S = gpu_solver(**dict(cfg, batch=B, sample_offset=off))
        S.set_initial_data("kh")
        S.step(4)
        S.stats_init()
        S.stats_accumulate()
        states.append(host(S.U).reshape(S.level_shape(0)))
        accs.append(S.stats.clone())
        S.sync()
        keep = S if off == 0 else keep
        if off:
            S.close()
    merged = merge_in_rank_order(keep, accs)
    keep.sync()
    d = oracle.make_desc(**cfg)
    a = oracle.welford(d, states[0])
    b = oracle.welford(d, states[1])
    c, m, M2 = oracle.stats_merge(d, a, b)
    raw = host(merged.view(torch.float64))
    cells = 40 * 36
    assert int(host(merged[:8].view(torch.int64))[0]) == c == 12
    np.testing.assert_array_equal(raw[32:32 + 4 * cells].reshape(4, -1), m)
    np.testing.assert_array_equal(raw[32 + 4 * cells:32 + 8 * cells].reshape(4, -1), M2)
    # and the sharded ensemble equals the single ensemble of 12 samples
    S12 = gpu_solver(**dict(cfg, batch=12))
    S12.set_initial_data("kh")
    S12.step(4)
    all12 = host(S12.U).reshape(S12.level_shape(0))
    assert np.array_equal(np.concatenate(states), all12)
    c2, m2, M22 = oracle.welford(d, all12)
    np.testing.assert_allclose(m, m2, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(M2, M22, rtol=1e-11, atol=1e-14)
    S12.close()
    keep.close()


@pytest.mark.parametrize("case", ["kh2", "kh3", "sod", "lax", "burgers", "vortex"])
def test_initial_data_fp64(case):
    if case == "kh2":
        cfg = dict(ndim=2, n=(70, 45), batch=3, eq="euler")
        th = kh_theta(3, 1)
        init = "kh"
    elif case == "kh3":
        cfg = dict(ndim=3, n=(12, 10, 9), batch=2, eq="euler")
        th = kh_theta(2, 2, P=128)
        init = "kh"
    elif case in ("sod", "lax"):
        cfg = dict(ndim=1, n=(301,), eq="euler")
        th, init = None, case
    elif case == "burgers":
        cfg = dict(ndim=1, n=(97,), eq="burgers")
        th, init = None, "burgers_sine"
    else:
        cfg = dict(ndim=2, n=(24, 20), lo=(0, 0), hi=(10, 10), eq="euler", vortex_center=(5.0, 4.5))
        th, init = None, "vortex"
    cfg["precision"] = "fp64"
    g, *_ = run_gpu(cfg, init, th, steps=0)
    d = oracle.make_desc(**cfg)
    o = oracle.init(d, init, cfg.get("batch", 1), th, center=cfg.get("vortex_center", (5, 5)))
    if init != "kh":
        p1_check(g, o, rel=1e-13, what=case)
        return
    # KH: the interface height Y = 0.01 sum a sin(...) comes from CUDA's sin on the GPU and the C
    # library's on the host, each within an ulp of the exact value but not always the same double.
    # A height that differs by d moves the band's volume fraction in the cut cell by d / dy, so the
    # cell's value moves by |U_in - U_out| d / dy: near zero where the blend of the two states
    # passes through zero (the x-momentum 0.5 - 1.5 f), where per-cell relative error means little.
    # The interface height 0.25 + Y (0.75 + Y) is then rounded to the ulp of 0.75 either way.
    # Bound: 1e-13 |o| + |U_in - U_out| (2 ulp(0.75) + 4 ulp(sum_n |0.01 a_n|)) / dy, per variable.
    g_ = 1.4
    U_in = np.array([2.0, -1.0, 0.0, 0.0, 2.5 / (g_ - 1) + 0.25])
    U_out = np.array([1.0, 0.5, 0.0, 0.0, 2.5 / (g_ - 1) + 0.125])
    nv = o.shape[1]
    jump = np.abs(U_in - U_out)[[0, 1] + list(range(2, nv - 1)) + [4]][:nv]
    dy = 1.0 / cfg["n"][1]
    P = th.shape[1] // 2
    for b in range(o.shape[0]):
        dY = 2 * np.spacing(0.75) + 4 * np.spacing(0.01 * np.abs(th[b, :P]).sum())
        for v in range(nv):
            tol = 1e-13 * np.abs(o[b, v]) + jump[v] * dY / dy
            bad = np.abs(g[b, v] - o[b, v]) > tol
            assert not bad.any(), (case, b, v, np.abs(g[b, v] - o[b, v])[bad][:5], tol[bad][:5])
    # and the cut cells do carry the sin difference: elsewhere the values are bitwise equal
    far = (np.abs(o[:, 0] - 1.0) < 1e-300) | (np.abs(o[:, 0] - 2.0) < 1e-300)
    assert np.array_equal(g[:, 0][far], o[:, 0][far])


# ------------------------------------------------------------------ one and ten steps, FP64
CASES_1D = [(r, f, v) for r in ("pc", "mc", "weno3") for f in ("rusanov", "hll", "hllc") for v in ("prim", "cons")]


@pytest.mark.parametrize("recon,flux,rvars", CASES_1D)
@pytest.mark.parametrize("steps", [1, 10])
def test_euler_1d_steps_fp64(recon, flux, rvars, steps):
    cfg = dict(ndim=1, n=(300,), eq="euler", recon=recon, flux=flux, rvars=rvars, rk="ssprk2",
               bc="outflow", cfl=0.45, precision="fp64")
    g, t, st, _ = run_gpu(cfg, "sod", steps=steps)
    o, ost, ot = run_oracle(cfg, "sod", steps=steps)
    assert st[0] == ost[0] == steps
    assert t[0] == pytest.approx(ot[0], rel=1e-13)
    p1_check(g, o, what=f"sod {recon} {flux} {rvars}")


@pytest.mark.parametrize("bc,init,rk", [("reflective", "sod", "ssprk3"), ("outflow", "lax", "ssprk3"),
                                        ("periodic", "raw", "ssprk3"), ("reflective", "raw", "ssprk2")])
def test_euler_1d_boundaries_fp64(bc, init, rk):
    cfg = dict(ndim=1, n=(257,), batch=2, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk=rk, bc=bc,
               cfl=0.45, precision="fp64")
    U0 = euler_state(2, 1, (257,), seed=5) if init == "raw" else None
    g, *_ = run_gpu(cfg, None if init == "raw" else init, U0=U0, steps=10)
    o, *_ = run_oracle(cfg, None if init == "raw" else init, U0=U0, steps=10)
    p1_check(g, o, what=f"{bc} {init}")


@pytest.mark.parametrize("recon", ["pc", "mc", "weno3"])
@pytest.mark.parametrize("flux", ["rusanov", "hll", "hllc"])
def test_burgers_1d_steps_fp64(recon, flux):
    cfg = dict(ndim=1, n=(200,), batch=3, eq="burgers", recon=recon, flux=flux, rk="ssprk3", bc="periodic",
               cfl=0.45, precision="fp64")
    U0 = burgers_state(3, 200, seed=9)
    g, *_ = run_gpu(cfg, U0=U0, steps=10)
    o, *_ = run_oracle(cfg, U0=U0, steps=10)
    p1_check(g, o, what=f"burgers {recon} {flux}")


CASES_2D = [("weno3", "hllc", "prim", "ssprk3"), ("mc", "rusanov", "cons", "ssprk2"), ("pc", "hll", "prim", "ssprk2"),
            ("weno3", "hll", "cons", "ssprk3"), ("mc", "hllc", "prim", "ssprk3"), ("weno3", "rusanov", "prim", "ssprk2")]


@pytest.mark.parametrize("recon,flux,rvars,rk", CASES_2D)
def test_kh_2d_steps_fp64(recon, flux, rvars, rk):
    cfg = dict(ndim=2, n=(70, 45), batch=2, eq="euler", recon=recon, flux=flux, rvars=rvars, rk=rk,
               bc="periodic", cfl=0.4, precision="fp64")
    th = kh_theta(2, 11)
    g, t, st, _ = run_gpu(cfg, "kh", th, steps=10)
    o, ost, ot = run_oracle(cfg, "kh", th, steps=10)
    np.testing.assert_allclose(t, ot, rtol=1e-13)
    p1_check(g, o, what=f"kh2d {recon} {flux} {rvars} {rk}")


def test_2d_mixed_boundaries_fp64():
    cfg = dict(ndim=2, n=(37, 50), batch=2, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc=[("outflow", "reflective"), ("reflective", "outflow")], cfl=0.4, precision="fp64")
    U0 = euler_state(2, 2, (37, 50), seed=3)
    g, *_ = run_gpu(cfg, U0=U0, steps=8)
    o, *_ = run_oracle(cfg, U0=U0, steps=8)
    p1_check(g, o, what="2d mixed bc")


def test_burgers_2d_fp64():
    cfg = dict(ndim=2, n=(40, 33), batch=1, eq="burgers", recon="mc", flux="hll", rk="ssprk2", bc="periodic",
               cfl=0.4, precision="fp64")
    x = np.arange(40) / 40
    y = np.arange(33) / 33
    U0 = (np.sin(2 * np.pi * x)[None, :] * 0.5 + np.cos(2 * np.pi * y)[:, None] * 0.3)[None, None, None]
    g, *_ = run_gpu(cfg, U0=U0, steps=10)
    o, *_ = run_oracle(cfg, U0=U0, steps=10)
    p1_check(g, o, what="burgers 2d")


@pytest.mark.parametrize("recon,flux,rvars,bc", [("weno3", "hllc", "prim", "periodic"),
                                                 ("mc", "rusanov", "cons", [("periodic", "periodic"), ("outflow", "outflow"), ("reflective", "reflective")])])
def test_kh_3d_steps_fp64(recon, flux, rvars, bc):
    cfg = dict(ndim=3, n=(20, 18, 17), batch=1, eq="euler", recon=recon, flux=flux, rvars=rvars, rk="ssprk3",
               bc=bc, cfl=0.3, precision="fp64")
    th = kh_theta(1, 4, P=128)
    g, *_ = run_gpu(cfg, "kh", th, steps=4)
    o, *_ = run_oracle(cfg, "kh", th, steps=4)
    p1_check(g, o, what=f"kh3d {recon} {flux}")


# ------------------------------------------------------------------ tiny and odd grids
@pytest.mark.parametrize("n,recon,bc", [
    ((1,), "pc", "periodic"), ((2,), "mc", "periodic"), ((3,), "weno3", "outflow"), ((5,), "mc", "reflective"),
    ((7,), "weno3", "periodic"), ((1, 3), "weno3", "periodic"), ((3, 2), "mc", "reflective"),
    ((5, 7), "weno3", [("outflow", "reflective"), ("periodic", "periodic")]), ((2, 3, 5), "mc", "periodic"),
    ((3, 1, 2), "pc", "outflow")])
def test_tiny_and_odd_grids_fp64(n, recon, bc):
    """Grids of 1 to 7 cells per direction, far below one tile: every ghost, halo and tile-edge
    path against the oracle per cell (FP64, 5 steps)."""
    nd = len(n)
    cfg = dict(ndim=nd, n=n, batch=2, eq="euler", recon=recon, flux="hllc", rvars="prim",
               rk="ssprk3", bc=bc, cfl=0.3, precision="fp64")
    U0 = euler_state(2, nd, n, seed=sum(n) + nd)
    g, *_ = run_gpu(cfg, U0=U0, steps=5)
    o, *_ = run_oracle(cfg, U0=U0, steps=5)
    p1_check(g, o, what=f"tiny {n} {recon} {bc}")


# ------------------------------------------------------------------ full runs to T (non-chaotic)
def test_sod_config_full_run_fp64():
    cfg = dict(ndim=1, n=(1024,), eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2", bc="outflow",
               cfl=0.45, precision="fp64")
    g, t, st, n = run_gpu(cfg, "sod", T=0.2)
    o, ost, ot = run_oracle(cfg, "sod", T=0.2)
    assert n == ost[0] and t[0] == 0.2 and ot[0] == 0.2
    p1_check(g, o, what="sod full")


@pytest.mark.parametrize("variant,precision", [(1, "fp64"), (2, "fp64"), (2, "fp32")])
def test_short_1d_tiles_bitwise_equal_to_default_tile(variant, precision):
    """1D tiles of 64 and 32 cells (ragged: 1000 cells) compute every interface with the same
    arithmetic as the 256-cell tile, so whole runs agree bitwise."""
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=1, n=(1000,), batch=2, eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2",
               bc="outflow", cfl=0.45, precision=precision)
    outs = []
    for v in (0, variant):
        S = gpu_solver(**cfg)
        alsv.alsv_set_tile_variant(S.ctx, v)
        S.set_initial_data("sod")
        S.evolve_to(0.2)
        outs.append(host(S.U))
        S.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("init,recon,flux,rvars", [("sod", "weno3", "hllc", "prim"), ("lax", "mc", "hll", "cons"),
                                                   ("sod", "pc", "rusanov", "prim")])
def test_fp64_tubes_bitwise_equal_to_oracle(init, recon, flux, rvars):
    """The FP64 path evaluates every formula with the oracle's operations in the oracle's order
    (no FMA contraction, true divisions); initial data without transcendental functions makes the
    whole run bitwise reproducible across the two."""
    T = 0.2 if init == "sod" else 0.13
    cfg = dict(ndim=1, n=(400,), eq="euler", recon=recon, flux=flux, rvars=rvars, rk="ssprk3", bc="outflow",
               cfl=0.45, precision="fp64")
    g, t, st, n = run_gpu(cfg, init, T=T)
    o, ost, ot = run_oracle(cfg, init, T=T)
    assert n == ost[0]
    assert np.array_equal(g, o)


def test_burgers_full_run_fp64():
    cfg = dict(ndim=1, n=(512,), eq="burgers", recon="weno3", flux="rusanov", rk="ssprk3", bc="periodic",
               cfl=0.45, precision="fp64")
    g, t, st, n = run_gpu(cfg, "burgers_sine", T=0.1)
    o, ost, _ = run_oracle(cfg, "burgers_sine", T=0.1)
    assert n == ost[0]
    p1_check(g, o, what="burgers full")


def test_vortex_full_run_fp64():
    cfg = dict(ndim=2, n=(32, 32), lo=(0, 0), hi=(10, 10), eq="euler", recon="weno3", flux="hllc", rvars="cons",
               rk="ssprk3", bc="periodic", cfl=0.4, precision="fp64", weno_eps_dx2=True)
    g, t, st, n = run_gpu(cfg, "vortex", T=1.0)
    o, ost, _ = run_oracle(cfg, "vortex", T=1.0)
    assert n == ost[0]
    p1_check(g, o, what="vortex full")


# ------------------------------------------------------------------ FP32
def test_kh_2d_fp32_ten_steps():
    cfg = dict(ndim=2, n=(64, 64), batch=2, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32")
    th = kh_theta(2, 21)
    g, *_ = run_gpu(cfg, "kh", th, steps=10)
    o, *_ = run_oracle(cfg, "kh", th, steps=10)
    p2_check(g, o, what="kh fp32")


def test_sod_fp32_full_run():
    cfg = dict(ndim=1, n=(1024,), eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2", bc="outflow",
               cfl=0.45, precision="fp32")
    g, *_ = run_gpu(cfg, "sod", T=0.2)
    o, *_ = run_oracle(cfg, "sod", T=0.2)
    p2_check(g, o, what="sod fp32")


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("recon,flux,rvars,bc", [("weno3", "hllc", "prim", "periodic"),
                                                  ("mc", "hll", "cons", "periodic"),
                                                  ("pc", "rusanov", "prim", "periodic"),
                                                  ("weno3", "rusanov", "prim",
                                                   [("periodic", "periodic"), ("reflective", "outflow"),
                                                    ("outflow", "reflective")])])
def test_kh_3d_zmarch_bitwise_equal_to_tiles(variant, recon, flux, rvars, bc):
    """The z-marching schedule evaluates every interface and the divergence with the tile kernel's
    arithmetic (ragged: 70 cells in z = one chunk of 64 plus 6, or one partial chunk of 128)."""
    import paper_1912_07645_gb300 as alsv
    torch = torch_()
    cfg = dict(ndim=3, n=(40, 20, 70), batch=2, eq="euler", recon=recon, flux=flux, rvars=rvars, rk="ssprk3",
               bc=bc, cfl=0.3, precision="fp32")
    th = torch.from_numpy(kh_theta(2, 21, P=128)).cuda()
    outs = []
    for v in (0, variant):
        S = gpu_solver(**cfg)
        alsv.alsv_set_tile_variant(S.ctx, v)
        S.set_initial_data("kh", theta=th)
        S.step(3)
        S.sync()
        outs.append((host(S.U), S.time()))
        S.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1][0], outs[1][1][0])


@pytest.mark.parametrize("pair", [(4, 5), (6, 7)])
@pytest.mark.parametrize("recon,flux,bc", [("weno3", "hllc", "periodic"),
                                           ("mc", "rusanov", [("periodic", "periodic"), ("reflective", "outflow"),
                                                              ("outflow", "reflective")]),
                                           ("pc", "hllc", [("outflow", "outflow"), ("reflective", "reflective"),
                                                           ("periodic", "periodic")])])
def test_kh_3d_packed_zmarch_32x7_bitwise_equal_to_32x8(pair, recon, flux, bc):
    """Variants 5 and 7 run the packed z-marches of 4 and 6 on 32 x 7 columns with 256 threads: the
    same packed arithmetic per interface, so bitwise equal (ragged: ny = 20 is 2 x 7 + 6)."""
    import paper_1912_07645_gb300 as alsv
    torch = torch_()
    cfg = dict(ndim=3, n=(40, 20, 70), batch=2, eq="euler", recon=recon, flux=flux, rvars="prim", rk="ssprk3",
               bc=bc, cfl=0.3, precision="fp32")
    th = torch.from_numpy(kh_theta(2, 23, P=128)).cuda()
    outs = []
    for v in pair:
        S = gpu_solver(**cfg)
        alsv.alsv_set_tile_variant(S.ctx, v)
        S.set_initial_data("kh", theta=th)
        S.step(3)
        S.sync()
        outs.append((host(S.U), S.time()))
        S.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1][0], outs[1][1][0])


@pytest.mark.parametrize("variant,recon,flux,bc", [
    (2, "weno3", "hllc", "periodic"),
    (4, "weno3", "hllc", "periodic"),
    (4, "mc", "rusanov", [("reflective", "outflow"), ("periodic", "periodic"), ("outflow", "reflective")]),
    (4, "pc", "hllc", [("outflow", "outflow"), ("reflective", "reflective"), ("periodic", "periodic")]),
    (5, "weno3", "hllc", [("periodic", "periodic"), ("reflective", "outflow"), ("periodic", "periodic")]),
    (6, "weno3", "hllc", "periodic"),
    (6, "mc", "rusanov", [("reflective", "outflow"), ("periodic", "periodic"), ("outflow", "reflective")]),
    (7, "weno3", "hllc", [("periodic", "periodic"), ("reflective", "outflow"), ("periodic", "periodic")]),
    (7, "pc", "rusanov", [("outflow", "outflow"), ("reflective", "reflective"), ("periodic", "periodic")])])
def test_kh_3d_zmarch_fp32_vs_oracle(variant, recon, flux, bc):
    """z-march schedules against the oracle (ragged: 70 planes); variants 4-7 pack an x- and a
    y-interface into the two FP32x2 lanes, 6 and 7 with the lean interface arithmetic."""
    import paper_1912_07645_gb300 as alsv
    torch = torch_()
    cfg = dict(ndim=3, n=(24, 20, 70), batch=1, eq="euler", recon=recon, flux=flux, rvars="prim", rk="ssprk3",
               bc=bc, cfl=0.3, precision="fp32")
    th = kh_theta(1, 8, P=128)
    S = gpu_solver(**cfg)
    alsv.alsv_set_tile_variant(S.ctx, variant)
    S.set_initial_data("kh", theta=torch.from_numpy(th).cuda())
    S.step(3)
    S.sync()
    g = host(S.U).reshape(S.level_shape(0))
    S.close()
    o, *_ = run_oracle(cfg, "kh", th, steps=3)
    p2_check(g, o, what=f"kh3d z-march v{variant} {recon} {flux} fp32")


def test_kh_3d_fp32():
    cfg = dict(ndim=3, n=(24, 20, 16), batch=1, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.3, precision="fp32")
    th = kh_theta(1, 8, P=128)
    g, *_ = run_gpu(cfg, "kh", th, steps=3)
    o, *_ = run_oracle(cfg, "kh", th, steps=3)
    p2_check(g, o, what="kh3d fp32")


# ------------------------------------------------------------------ determinism and invariances
def test_determinism_graphs_variants_and_batch_independence():
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=(64, 64), batch=6, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=42)
    outs = []
    for graphs, variant in ((True, 0), (True, 0), (False, 0), (True, 1)):
        S = gpu_solver(**cfg)
        alsv.alsv_set_graphs(S.ctx, graphs)
        alsv.alsv_set_tile_variant(S.ctx, variant)
        S.set_initial_data("kh")
        S.evolve_to(0.05)
        outs.append(host(S.U))
        S.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    # sample 3 of the batch equals a single-sample run on the same parameters
    th = torch.from_numpy(oracle.theta_splitmix(42, 6, 20)[3:4].copy()).cuda()
    S1 = gpu_solver(**dict(cfg, batch=1))
    S1.set_initial_data("kh", theta=th)
    S1.evolve_to(0.05)
    one = host(S1.U)
    assert np.array_equal(outs[0].reshape(6, -1)[3], one.reshape(-1))


def test_totals_and_kinetic_energy_fp64():
    cfg = dict(ndim=2, n=(70, 45), batch=3, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp64")
    th = kh_theta(3, 13)
    torch = torch_()
    S = gpu_solver(**cfg)
    S.set_initial_data("kh", theta=torch.from_numpy(th).cuda())
    tot0 = host(S.totals())
    S.step(20)
    tot1 = host(S.totals())
    ke = host(S.kinetic_energy())
    U = host(S.U).reshape(S.level_shape(0))
    S.sync()
    d = oracle.make_desc(**cfg)
    scale = np.abs(U).reshape(3, 4, -1).sum(axis=2) / (70 * 45)
    np.testing.assert_allclose(tot1, oracle.totals(d, U), rtol=0, atol=1e-14 * scale.max())
    np.testing.assert_allclose(ke, oracle.kinetic_energy(d, U), rtol=1e-13)
    # eq. (2.1) on a periodic grid conserves every total
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.maximum(scale, 1e-300))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_welford_statistics_match_oracle(precision):
    torch = torch_()
    cfg = dict(ndim=2, n=(40, 36), batch=16, eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2",
               bc="periodic", cfl=0.4, precision=precision, seed=5)
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    S.step(3)
    S.stats_init()
    S.stats_accumulate()
    U1 = host(S.U).reshape(S.level_shape(0))
    S.step(2)
    S.stats_accumulate()          # streaming: a second batch folds in after the first
    U2 = host(S.U).reshape(S.level_shape(0))
    cnt, mean, var = S.stats_read()
    mean, var = host(mean), host(var)
    d = oracle.make_desc(**cfg)
    c, m, M2 = oracle.welford(d, U1)
    c, m, M2 = oracle.welford(d, U2, c, m, M2)
    assert cnt == c == 32
    np.testing.assert_allclose(mean.reshape(4, -1), m, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(var.reshape(4, -1), M2 / (c - 1), rtol=1e-11, atol=1e-15)


# ------------------------------------------------------------------ full-size batched configuration, sampled
@pytest.mark.parametrize("variant", [4, 8, 9, 13])
def test_full_size_batched_kh_sampled(variant):
    """256^2 x 4096 samples, FP32 WENO3 + HLLC + SSP-RK3 (the benchmark workload), in the launch
    geometry of each two-sample schedule the autotuner picks from for it; three sampled samples
    against the oracle after two CFL steps."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=(256, 256), batch=4096, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=12345)
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    alsv.alsv_set_tile_variant(S.ctx, variant)
    S.step(2)
    S.sync()
    V = S.state()
    picks = [0, 1234, 4095]
    g = np.stack([host(V[b]) for b in picks])
    t, st = S.time()
    S.close()
    del V
    torch.cuda.empty_cache()
    th = oracle.theta_splitmix(12345, 4096, 20)[picks]
    ocfg = dict(cfg, batch=3)
    o, ost, ot = run_oracle(ocfg, "kh", th, steps=2)
    np.testing.assert_allclose(t[picks], ot, rtol=1e-6)
    p2_check(g, o, what="full-size sampled")


def test_mlmc_levels_one_launch_fp32():
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    lv = [((32, 32), 6), ((64, 64), 3), ((96, 96), 2)]
    cfg = dict(ndim=2, levels=lv, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=99)
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    S.step(3)
    S.sync()
    th_all = oracle.theta_splitmix(99, 11, 20)
    s0 = 0
    for l, (n, B) in enumerate(lv):
        g = host(S.state(l))
        ocfg = dict(cfg, n=n, batch=B)
        ocfg.pop("levels")
        o, *_ = run_oracle(ocfg, "kh", th_all[s0:s0 + B], steps=3)
        p2_check(g, o, what=f"level {l}")
        s0 += B
    S.close()


# ------------------------------------------------------------------ failure reporting (host-side injection)
def test_nonphysical_state_is_reported_and_gpu_stays_usable():
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=1, n=(64,), batch=2, eq="euler", recon="mc", flux="hllc", rk="ssprk2", bc="outflow",
               precision="fp64")
    U0 = euler_state(2, 1, (64,), seed=1)
    U0[1, 2, 0, 0, 10] = -5.0            # negative pressure in sample 1
    S = gpu_solver(**cfg)
    S.set_state(torch.from_numpy(U0))
    with pytest.raises(alsv.AlsvError) as ei:
        S.evolve_to(0.1)
    assert ei.value.status_name == "ERR_NONPHYSICAL"
    S.close()
    g, *_ = run_gpu(cfg, "sod", steps=2)
    assert np.isfinite(g).all()


def test_fixed_dt_cfl_guard():
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=1, n=(64,), eq="euler", recon="mc", flux="rusanov", rk="ssprk2", bc="outflow",
               precision="fp64", fixed_dt=0.02)     # CFL = 0.02 * 1.18 * 64 > 0.5
    S = gpu_solver(**cfg)
    S.set_initial_data("sod")
    with pytest.raises(alsv.AlsvError) as ei:
        S.evolve_to(0.1)
    assert ei.value.status_name == "ERR_CFL"
    S.close()


def test_checkpoint_resume_is_bitwise():
    """Evolve 0 -> T/2, checkpoint (U, t, steps), resume in a new context, evolve to T: bitwise
    equal to one uninterrupted evolve to T (checkpoint and resume)."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=(64, 48), batch=3, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=21)
    A = gpu_solver(**cfg)
    A.set_initial_data("kh")
    A.evolve_to(0.05)
    U_ck = host(A.U).copy()
    t_ck, s_ck = A.time()
    A.evolve_to(0.1)
    ref = host(A.U)
    _, s_ref = A.time()
    A.close()
    B = gpu_solver(**cfg)
    B.set_state(torch.from_numpy(U_ck))
    alsv.alsv_set_time(B.ctx, t_ck, s_ck)
    B.evolve_to(0.1)
    out = host(B.U)
    t_b, s_b = B.time()
    B.close()
    assert np.array_equal(out, ref)
    assert np.array_equal(s_b, s_ref) and np.all(t_b == 0.1)


@pytest.mark.parametrize("recon,flux,n", [("weno3", "hllc", (70, 45)), ("mc", "rusanov", (64, 33)),
                                          ("weno3", "rusanov", (31, 40)), ("mc", "hllc", (93, 62))])
def test_column_variant_fp32_vs_oracle(recon, flux, n):
    """The column-marching schedule (variant 3) computes the same FP32 stage: 2e-5 relative L1 vs
    the oracle, on strips with ragged widths."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=n, batch=3, eq="euler", recon=recon, flux=flux, rvars="prim", rk="ssprk3", bc="periodic",
               cfl=0.4, precision="fp32")
    th = kh_theta(3, 61)
    outs = []
    for _ in range(2):
        S = gpu_solver(**cfg)
        alsv.alsv_set_tile_variant(S.ctx, 3)
        S.set_initial_data("kh", theta=torch.from_numpy(th).cuda())
        S.step(10)
        S.sync()
        outs.append(host(S.U).reshape(S.level_shape(0)))
        t, _ = S.time()
        S.close()
    assert np.array_equal(outs[0], outs[1])          # deterministic
    o, _, ot = run_oracle(cfg, "kh", th, steps=10)
    np.testing.assert_allclose(t, ot, rtol=1e-5)
    p2_check(outs[0], o, what=f"column {recon} {flux}")


def test_column_variant_mlmc_levels_and_rejection():
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    lv = [((32, 32), 4), ((64, 64), 2), ((100, 100), 1)]
    cfg = dict(ndim=2, levels=lv, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=5)
    S = gpu_solver(**cfg)
    alsv.alsv_set_tile_variant(S.ctx, 3)
    S.set_initial_data("kh")
    S.step(4)
    S.sync()
    th_all = oracle.theta_splitmix(5, 7, 20)
    s0 = 0
    for l, (n, B) in enumerate(lv):
        ocfg = dict(cfg, n=n, batch=B)
        ocfg.pop("levels")
        o, *_ = run_oracle(ocfg, "kh", th_all[s0:s0 + B], steps=4)
        p2_check(host(S.state(l)), o, what=f"column level {l}")
        s0 += B
    S.close()
    S2 = gpu_solver(ndim=2, n=(32, 32), batch=1, recon="weno3", flux="hllc", rvars="prim", bc="outflow",
                    precision="fp32")
    with pytest.raises(alsv.AlsvError, match="variant"):
        alsv.alsv_set_tile_variant(S2.ctx, 3)
    S2.close()


@pytest.mark.parametrize("variant", [4, 5, 8, 9, 12])
@pytest.mark.parametrize("recon,flux,bc", [("weno3", "hllc", "periodic"), ("mc", "rusanov", "periodic"),
                                           ("pc", "hllc", [("outflow", "reflective"), ("reflective", "outflow")]),
                                           ("weno3", "rusanov", "reflective")])
def test_pair_variant_fp32_vs_oracle(variant, recon, flux, bc):
    """Two-sample schedules (variants 4, 5 and the lean 8, 9, 12): each sample within 2e-5 relative L1
    of the oracle, with an odd batch (the last sample has no partner), ragged tiles and boundary
    fill."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=(70, 45), batch=3, eq="euler", recon=recon, flux=flux, rvars="prim", rk="ssprk3", bc=bc,
               cfl=0.4, precision="fp32")
    U0 = euler_state(3, 2, (70, 45), seed=71)
    S = gpu_solver(**cfg)
    alsv.alsv_set_tile_variant(S.ctx, variant)
    S.set_state(torch.from_numpy(U0))
    S.step(10)
    S.sync()
    g = host(S.U).reshape(S.level_shape(0))
    S.close()
    o, *_ = run_oracle(cfg, U0=U0, steps=10)
    for b in range(3):
        p2_check(g[b:b + 1], o[b:b + 1], what=f"pair v{variant} {recon} {flux} sample {b}")


@pytest.mark.parametrize("recon,flux,bcx", [("weno3", "hllc", "periodic"), ("mc", "rusanov", "outflow"),
                                            ("pc", "hllc", "reflective")])
def test_halves_variant_fp32_vs_oracle_and_bitwise_with_sample_pairs(recon, flux, bcx):
    """Variant 6 pairs the two halves of each y-periodic sample (ragged x: 70 cells, ny = 64): within
    2e-5 relative L1 of the oracle, and bitwise equal to the two-sample schedule (every packed lane
    performs the same operations on its own data)."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    bc = [(bcx, bcx), ("periodic", "periodic")]
    cfg = dict(ndim=2, n=(70, 64), batch=3, eq="euler", recon=recon, flux=flux, rvars="prim", rk="ssprk3", bc=bc,
               cfl=0.4, precision="fp32")
    U0 = euler_state(3, 2, (70, 64), seed=73)
    out = {}
    for v in (4, 6, 7):
        S = gpu_solver(**cfg)
        alsv.alsv_set_tile_variant(S.ctx, v)
        S.set_state(torch.from_numpy(U0))
        S.step(10)
        S.sync()
        out[v] = (host(S.U).reshape(S.level_shape(0)), S.time())
        S.close()
    assert np.array_equal(out[4][0], out[6][0]) and np.array_equal(out[4][0], out[7][0])
    np.testing.assert_array_equal(out[4][1][0], out[6][1][0])
    o, *_ = run_oracle(cfg, U0=U0, steps=10)
    for b in range(3):
        p2_check(out[6][0][b:b + 1], o[b:b + 1], what=f"halves {recon} {flux} sample {b}")


@pytest.mark.parametrize("recon,flux,bcx", [("weno3", "hllc", "periodic"), ("mc", "rusanov", "outflow"),
                                            ("pc", "hllc", "reflective"), ("weno3", "rusanov", "reflective")])
def test_lean_pair_variants_bitwise_equal_and_vs_oracle(recon, flux, bcx):
    """The lean two-sample schedules evaluate every interface with the same operations whatever
    the order of the reads, the barrier structure or the pairing: sample pairs (8, 9, 12) and the
    two halves of each sample (10, 11, 13; 12 and 13 pass the x-fluxes by warp shuffles) are
    bitwise equal (ragged x: 70 cells, ny = 64, odd batch), and within 2e-5 relative L1 of the
    oracle."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    bc = [(bcx, bcx), ("periodic", "periodic")]
    cfg = dict(ndim=2, n=(70, 64), batch=3, eq="euler", recon=recon, flux=flux, rvars="prim", rk="ssprk3", bc=bc,
               cfl=0.4, precision="fp32")
    U0 = euler_state(3, 2, (70, 64), seed=74)
    out = {}
    for v in (8, 9, 10, 11, 12, 13):
        S = gpu_solver(**cfg)
        alsv.alsv_set_tile_variant(S.ctx, v)
        S.set_state(torch.from_numpy(U0))
        S.step(10)
        S.sync()
        out[v] = (host(S.U).reshape(S.level_shape(0)), S.time())
        S.close()
    for v in (9, 10, 11, 12, 13):
        assert np.array_equal(out[8][0], out[v][0]), v
        np.testing.assert_array_equal(out[8][1][0], out[v][1][0])
    o, *_ = run_oracle(cfg, U0=U0, steps=10)
    for b in range(3):
        p2_check(out[8][0][b:b + 1], o[b:b + 1], what=f"lean {recon} {flux} sample {b}")


def test_halves_variant_needs_aligned_periodic_y():
    torch_()
    import paper_1912_07645_gb300 as alsv
    for n, bc in (((64, 40), "periodic"), ((64, 64), [("periodic", "periodic"), ("outflow", "outflow")])):
        S = gpu_solver(ndim=2, n=n, batch=1, eq="euler", recon="weno3", flux="hllc", rvars="prim", precision="fp32",
                       bc=bc)
        for v in (6, 7, 10, 11, 13):
            with pytest.raises(alsv.AlsvError, match="does not support"):
                alsv.alsv_set_tile_variant(S.ctx, v)
        S.close()
    S = gpu_solver(ndim=2, n=(64, 48), batch=1, eq="euler", recon="weno3", flux="hllc", rvars="prim",
                   precision="fp32", bc="periodic")
    alsv.alsv_set_tile_variant(S.ctx, 7)      # 48 = 3 x 16: 32x8 halves align
    for v in (10, 11, 13):                    # 32x16 halves need ny divisible by 32
        with pytest.raises(alsv.AlsvError, match="does not support"):
            alsv.alsv_set_tile_variant(S.ctx, v)
    S.close()


@pytest.mark.parametrize("variant", [4, 8])
def test_pair_variant_samples_finishing_at_different_steps(variant):
    """Samples of one pair reach T after different step counts: the finished lane must stay
    untouched while its partner continues."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=(48, 40), batch=5, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32")
    U0 = euler_state(5, 2, (48, 40), seed=72)
    U0[1, 3] *= 1.6          # hotter sample: larger sound speed, more steps to the same T
    S = gpu_solver(**cfg)
    alsv.alsv_set_tile_variant(S.ctx, variant)
    S.set_state(torch.from_numpy(U0))
    S.evolve_to(0.04)
    g = host(S.U).reshape(S.level_shape(0))
    t, st = S.time()
    S.close()
    o, ost, ot = run_oracle(cfg, U0=U0, T=0.04)
    assert len(set(ost.tolist())) > 1            # the pairs really finish at different steps
    assert np.array_equal(st, ost) and np.all(t == 0.04)
    for b in range(5):
        p2_check(g[b:b + 1], o[b:b + 1], what=f"pair finish sample {b}")


@pytest.mark.parametrize("variant", [4, 8, 9])
def test_pair_variant_mlmc_levels_odd_counts(variant):
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    lv = [((32, 32), 3), ((64, 48), 1), ((40, 40), 4)]
    cfg = dict(ndim=2, levels=lv, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=9)
    S = gpu_solver(**cfg)
    alsv.alsv_set_tile_variant(S.ctx, variant)
    S.set_initial_data("kh")
    S.step(3)
    S.sync()
    th_all = oracle.theta_splitmix(9, 8, 20)
    s0 = 0
    for l, (n, B) in enumerate(lv):
        ocfg = dict(cfg, n=n, batch=B)
        ocfg.pop("levels")
        o, *_ = run_oracle(ocfg, "kh", th_all[s0:s0 + B], steps=3)
        p2_check(host(S.state(l)), o, what=f"pair level {l}")
        s0 += B
    S.close()


@pytest.mark.parametrize("variant", [8, 11, 13])
def test_pair_schedule_levels_finishing_apart_equal_single_level_runs(variant):
    """Levels of one launch finish at different step counts (coarser grids take fewer CFL steps), so
    alsv_evolve_to_T leaves the finished levels out of the later two-sample stage launches. Each
    level's samples equal, bitwise and in step count, the same samples evolved alone on a one-level
    grid."""
    torch = torch_()
    import paper_1912_07645_gb300 as alsv
    lv = [((32, 32), 3), ((64, 64), 2), ((32, 64), 4)]
    T = 0.3
    cfg = dict(ndim=2, levels=lv, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=9)
    S = gpu_solver(**cfg)
    alsv.alsv_set_tile_variant(S.ctx, variant)
    S.set_initial_data("kh")
    S.evolve_to(T)
    t_all, n_all = S.time()
    th_all = oracle.theta_splitmix(9, 9, 20)
    s0, last = 0, []
    for l, (n, B) in enumerate(lv):
        one = dict(cfg, n=n, batch=B)
        one.pop("levels")
        S1 = gpu_solver(**one)
        alsv.alsv_set_tile_variant(S1.ctx, variant)
        S1.set_initial_data("kh", theta=torch.from_numpy(th_all[s0:s0 + B]).cuda())
        S1.evolve_to(T)
        t1, n1 = S1.time()
        assert np.array_equal(host(S.state(l)), host(S1.U).reshape(host(S.state(l)).shape)), f"level {l}"
        assert np.array_equal(n_all[s0:s0 + B], n1) and np.all(t1 == T)
        last.append(int(n1.max()))
        S1.close()
        s0 += B
    S.close()
    assert max(last) > min(last) + 32, last   # levels finish more than two 16-step chunks apart


# ------------------------------------------------------------------ seeded random configurations
def _random_configs(count, seed=2026):
    """Seeded draws over the descriptor: dimension, odd and ragged sizes, scheme, variables, RK
    order, boundary kinds per face, precision and batch."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        nd = int(rng.integers(1, 4))
        hi_n = {1: 300, 2: 70, 3: 19}[nd]
        n = tuple(int(v) for v in rng.integers(3, hi_n, nd))
        recon = str(rng.choice(["pc", "mc", "weno3"]))
        g = 1 if recon == "pc" else 2
        bc = []
        for k in range(nd):
            kind = str(rng.choice(["periodic", "outflow", "reflective"]))
            if kind == "periodic":
                bc.append(("periodic", "periodic"))
            else:
                other = str(rng.choice(["outflow", "reflective"]))
                bc.append((kind, other))
            if "reflective" in bc[-1] and n[k] < g:
                bc[-1] = ("outflow", "outflow")
        out.append(dict(ndim=nd, n=n, batch=int(rng.integers(1, 4)), eq="euler", recon=recon,
                        rvars=str(rng.choice(["prim", "cons"])), flux=str(rng.choice(["rusanov", "hll", "hllc"])),
                        rk=str(rng.choice(["ssprk2", "ssprk3"])), bc=bc, cfl=0.3,
                        precision=str(rng.choice(["fp64", "fp32"]))))
    return out


@pytest.mark.parametrize("k,cfg", list(enumerate(_random_configs(24))), ids=[f"r{k}" for k in range(24)])
def test_seeded_random_configurations_vs_oracle(k, cfg):
    """Four CFL steps of smooth random states on seeded random descriptors against the oracle:
    FP64 per cell (P1), FP32 relative L1 (P2)."""
    U0 = euler_state(cfg["batch"], cfg["ndim"], cfg["n"], seed=100 + k)
    g, _, st, _ = run_gpu(cfg, U0=U0, steps=4)
    o, ost, _ = run_oracle(cfg, U0=U0, steps=4)
    assert np.array_equal(st, ost)
    if cfg["precision"] == "fp64":
        p1_check(g, o, what=f"random {cfg}")
    else:
        p2_check(g, o, what=f"random {cfg}")


def test_batched_fp32_statistics_within_mc_error_of_fp64():
    """The batched FP32 run's per-cell mean and variance against the FP64 path's on the same 256
    samples (KH 64^2 to T = 0.5): the mean differs by far less than the Monte Carlo standard error
    sigma / sqrt(M) in L1 (the precision change is invisible next to the sampling error)."""
    M = 256
    out = {}
    for prec in ("fp32", "fp64"):
        S = gpu_solver(ndim=2, n=(64, 64), batch=M, eq="euler", recon="weno3", flux="hllc", rvars="prim",
                       rk="ssprk3", bc="periodic", cfl=0.4, precision=prec, seed=99)
        S.set_initial_data("kh")
        S.evolve_to(0.5)
        S.stats_init()
        S.stats_accumulate()
        cnt, mean, var = S.stats_read()
        out[prec] = (cnt, host(mean), host(var))
        S.close()
    assert out["fp32"][0] == out["fp64"][0] == M
    m32, v32 = out["fp32"][1], out["fp32"][2]
    m64, v64 = out["fp64"][1], out["fp64"][2]
    se = np.sqrt(v64 / M)                                   # MC standard error per cell and quantity
    for q in range(4):
        d = np.abs(m32[q] - m64[q]).sum()
        assert d <= 3 * se[q].sum(), (q, d, se[q].sum())
        assert d <= 0.05 * se[q].sum(), (q, d / se[q].sum())  # in fact far below it
    np.testing.assert_allclose(v32.sum(axis=(1, 2, 3)), v64.sum(axis=(1, 2, 3)), rtol=1e-2)
