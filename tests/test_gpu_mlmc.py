"""Multilevel Monte Carlo estimator on the GPU (Sec. 2.2) against the oracle's estimator.

The coupled batch holds every level and, for each level above the coarsest, a companion group that
runs the same KH parameters on the next coarser grid; everything advances in one launch per stage.
"""
import numpy as np
import pytest

import oracle
from harness import gpu_solver, host, need_gpu, p1_check, p2_check

pytestmark = pytest.mark.gpu

# (grid (nx, ny), samples, fine partner): levels 16x8 / 32x16 / 64x32 with companions
LEVELS = [((16, 8), 6), ((32, 16), 4), ((16, 8), 4, 1), ((64, 32), 3), ((32, 16), 3, 3)]
PAIRS = [(0, None), (1, 2), (3, 4)]   # (level group, companion group)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    from paper_1912_07645_gb300 import build
    build.build()


def cfg_for(precision, seed=21):
    return dict(ndim=2, levels=LEVELS, eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2",
                bc="periodic", cfl=0.4, precision=precision, seed=seed)


def group_cfg(cfg, l):
    c = dict(cfg, n=LEVELS[l][0], batch=LEVELS[l][1])
    c.pop("levels")
    return c


def sample0(l):
    return sum(e[1] for e in LEVELS[:l])


def run_gpu(cfg, T, accumulate_twice_with=None):
    import paper_1912_07645_gb300 as alsv
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    S.evolve_to(T)
    S.mlmc_accumulate()
    states = [host(S.state(l)) for l in range(len(LEVELS))]
    th = host(_params(S, alsv))
    if accumulate_twice_with is not None:
        S2 = gpu_solver(**dict(cfg, seed=accumulate_twice_with))
        S2.set_initial_data("kh")
        S2.evolve_to(T)
        states2 = [host(S2.state(l)) for l in range(len(LEVELS))]
        # fold the second batch into the first accumulator
        alsv.alsv_mlmc_accumulate(S2.ctx, S.mlmc_acc)
        S2.sync()
        S2.close()
        states = [np.concatenate([a, b]) for a, b in zip(states, states2)]
    cnt, mean, var, lev = S.mlmc_read()
    out = (cnt, host(mean), host(var), host(lev), states, th)
    S.close()
    return out


def _params(S, alsv):
    th = S.torch.empty((S.samples, 20), dtype=S.torch.float64, device="cuda")
    alsv.alsv_get_parameters(S.ctx, th)
    S.sync()
    return th


def oracle_levels(states, dxs):
    return [(states[f], None if c is None else states[c], dxs[f]) for f, c in PAIRS]


def dV(l):
    nx, ny = LEVELS[l][0]
    return (1.0 / nx) * (1.0 / ny)


def test_companions_share_their_levels_parameters():
    import paper_1912_07645_gb300 as alsv
    S = gpu_solver(**cfg_for("fp64"))
    S.set_initial_data("kh")
    th = host(_params(S, alsv))
    S.close()
    ref = oracle.theta_splitmix(21, sum(e[1] for e in LEVELS), 20)
    for f, c in PAIRS:
        s, B = sample0(f), LEVELS[f][1]
        np.testing.assert_array_equal(th[s:s + B], ref[s:s + B])
        if c is not None:
            np.testing.assert_array_equal(th[sample0(c):sample0(c) + B], ref[s:s + B])


def test_estimator_fp64_against_oracle_runs():
    T = 0.05
    cfg = cfg_for("fp64")
    cnt, mean, var, lev, states, th = run_gpu(cfg, T)
    assert cnt == [6, 4, 3]
    # every group against the oracle run of the same parameters
    ostates = []
    for l in range(len(LEVELS)):
        oc = oracle.make_desc(**group_cfg(cfg, l))
        s, B = sample0(l), LEVELS[l][1]
        o, *_ = oracle.evolve(oc, oracle.init(oc, "kh", B, th[s:s + B]), T=T)
        p1_check(states[l], o, what=f"group {l}")
        ostates.append(o)
    dxs = [dV(l) for l in range(len(LEVELS))]
    # the estimator kernels on the GPU's own states: same numbers up to summation rounding
    m_g, v_g, s_g = oracle.mlmc_estimate(oracle_levels(states, dxs))
    np.testing.assert_allclose(mean, m_g, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(var, v_g, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(lev, s_g, rtol=1e-12, atol=1e-14)
    # and against the estimate of the oracle's runs
    m_o, v_o, s_o = oracle.mlmc_estimate(oracle_levels(ostates, dxs))
    scale = np.abs(m_o).max(axis=(1, 2, 3), keepdims=True)
    assert np.all(np.abs(mean - m_o) <= 1e-12 * scale)
    assert np.all(np.abs(var - v_o) <= 1e-12 * np.abs(m_o * m_o).max(axis=(1, 2, 3), keepdims=True))


def test_estimator_streams_over_batches():
    T = 0.02
    cnt, mean, var, lev, states, _ = run_gpu(cfg_for("fp64", seed=5), T, accumulate_twice_with=6)
    assert cnt == [12, 8, 6]
    dxs = [dV(l) for l in range(len(LEVELS))]
    m_g, v_g, s_g = oracle.mlmc_estimate(oracle_levels(states, dxs))
    np.testing.assert_allclose(mean, m_g, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(var, v_g, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(lev, s_g, rtol=1e-12, atol=1e-14)


def test_estimator_fp32_states():
    T = 0.05
    cfg = cfg_for("fp32", seed=8)
    cnt, mean, var, lev, states, th = run_gpu(cfg, T)
    dxs = [dV(l) for l in range(len(LEVELS))]
    m_g, v_g, _ = oracle.mlmc_estimate(oracle_levels(states, dxs))
    np.testing.assert_allclose(mean, m_g, rtol=1e-12, atol=1e-13)
    ostates = []
    for l in range(len(LEVELS)):
        oc = oracle.make_desc(**group_cfg(cfg, l))
        s, B = sample0(l), LEVELS[l][1]
        o, *_ = oracle.evolve(oc, oracle.init(oc, "kh", B, th[s:s + B]), T=T)
        p2_check(states[l], o, what=f"group {l}")
        ostates.append(o)
    m_o, _, _ = oracle.mlmc_estimate(oracle_levels(ostates, dxs))
    p2_check(mean[None], m_o[None], what="MLMC mean")


def test_estimator_is_deterministic():
    a = run_gpu(cfg_for("fp32", seed=3), 0.03)
    b = run_gpu(cfg_for("fp32", seed=3), 0.03)
    for x, y in zip(a[1:4], b[1:4]):
        np.testing.assert_array_equal(x, y)


def test_estimator_3d_levels_and_halton_companions():
    """3D slab levels 8^3 / 16^3 with a companion, parameters from the Halton sequence: the
    companion carries its level's parameters and the estimate matches the oracle's on the GPU's
    states."""
    import paper_1912_07645_gb300 as alsv
    lv = [((8, 8, 8), 3), ((16, 16, 16), 2), ((8, 8, 8), 2, 1)]
    cfg = dict(ndim=3, levels=lv, eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2", bc="periodic",
               cfl=0.3, precision="fp64", seed=4, sampler="halton")
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    th = S.torch.empty((S.samples, 128), dtype=S.torch.float64, device="cuda")
    alsv.alsv_get_parameters(S.ctx, th)
    S.step(3)
    S.mlmc_accumulate()
    states = [host(S.state(l)) for l in range(3)]
    th = host(th)
    cnt, mean, var, lev = S.mlmc_read()
    mean, var, lev = host(mean), host(var), host(lev)
    S.close()
    ref = oracle.theta_halton(7, 128)
    np.testing.assert_array_equal(th[:5], ref[:5])
    np.testing.assert_array_equal(th[5:7], ref[3:5])      # the companion takes level 1's indices
    assert cnt == [3, 2]
    levels = [(states[0], None, 1 / 512), (states[1], states[2], 1 / 4096)]
    m_g, v_g, s_g = oracle.mlmc_estimate(levels)
    np.testing.assert_allclose(mean, m_g, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(var, v_g, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(lev, s_g, rtol=1e-12, atol=1e-14)
