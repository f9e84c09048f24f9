"""Spatial domain decomposition on the GPU (Sec. 2.1, last paragraph; Sec. 3.1): a grid advanced
as blocks that exchange halo layers between RK stages and share the CFL maximum must reproduce
the undivided context bitwise - FP64 and FP32, 1D/2D/3D, periodic wraps, physical faces and
ragged block sizes - through the C ABI's stage-by-stage protocol (all blocks in one process, one
GPU, one stream; the torch.distributed transport is covered by the gloo tests on CPUs)."""
import numpy as np
import pytest

import oracle
from harness import gpu_solver, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    from paper_1912_07645_gb300 import build
    build.build()


CASES = [
    ("kh2d_fp64_x2", dict(ndim=2, n=(64, 48), batch=3, eq="euler", recon="mc", rvars="prim", flux="hllc",
                          rk="ssprk2", bc="periodic", cfl=0.4, precision="fp64", seed=3), "kh", (2, 1), 0.05),
    ("kh2d_fp64_y2", dict(ndim=2, n=(64, 48), batch=3, eq="euler", recon="mc", rvars="prim", flux="hllc",
                          rk="ssprk2", bc="periodic", cfl=0.4, precision="fp64", seed=3), "kh", (1, 2), 0.05),
    ("kh2d_fp64_3x2_mixed", dict(ndim=2, n=(64, 48), batch=2, eq="euler", recon="weno3", rvars="prim", flux="hllc",
                                 rk="ssprk3", bc=[("periodic", "periodic"), ("reflective", "outflow")], cfl=0.4,
                                 precision="fp64", seed=4), "kh", (3, 2), 0.04),
    ("kh2d_fp32_2x2", dict(ndim=2, n=(64, 64), batch=4, eq="euler", recon="weno3", rvars="prim", flux="hllc",
                           rk="ssprk3", bc="periodic", cfl=0.4, precision="fp32", seed=5), "kh", (2, 2), 0.1),
    ("kh2d_fp32_cons_y3", dict(ndim=2, n=(40, 70), batch=2, eq="euler", recon="mc", rvars="cons", flux="rusanov",
                               rk="ssprk2", bc="periodic", cfl=0.4, precision="fp32", seed=6), "kh", (1, 3), 0.05),
    ("sod_fp64_x4", dict(ndim=1, n=(200,), batch=1, eq="euler", recon="weno3", rvars="prim", flux="hllc",
                         rk="ssprk3", bc="outflow", cfl=0.45, precision="fp64"), "sod", (4,), 0.2),
    ("burgers_fp32_x3", dict(ndim=1, n=(96,), batch=2, eq="burgers", recon="pc", flux="hll", rk="ssprk2",
                             bc="periodic", cfl=0.45, precision="fp32"), "burgers_sine", (3,), 0.1),
    ("kh3d_fp64_2x1x2", dict(ndim=3, n=(16, 12, 20), batch=2, eq="euler", recon="mc", rvars="prim", flux="hllc",
                             rk="ssprk2", bc="periodic", cfl=0.3, precision="fp64", seed=7), "kh", (2, 1, 2), 0.06),
    ("kh3d_fp32_1x2x2", dict(ndim=3, n=(16, 16, 16), batch=2, eq="euler", recon="weno3", rvars="prim",
                             flux="hllc", rk="ssprk3", bc=[("periodic", "periodic"), ("outflow", "outflow"),
                                                           ("periodic", "periodic")], cfl=0.3,
                             precision="fp32", seed=8), "kh", (1, 2, 2), 0.06),
    # cell-value fluxes over four cells (ghost width 2) through the halo faces
    ("kh2d_fp64_tecno2_2x2", dict(ndim=2, n=(48, 40), batch=2, eq="euler", flux="tecno2", rvars="prim",
                                  rk="ssprk3", bc=[("periodic", "periodic"), ("reflective", "outflow")], cfl=0.4,
                                  precision="fp64", seed=10), "kh", (2, 2), 0.03),
    ("kh2d_fp32_ec4_x3", dict(ndim=2, n=(60, 32), batch=2, eq="euler", flux="ec4", rvars="prim", rk="ssprk3",
                              bc="periodic", cfl=0.4, precision="fp32", seed=11), "kh", (3, 1), 0.02),
    ("burgers_fp64_tecno2_x3", dict(ndim=1, n=(90,), batch=2, eq="burgers", flux="tecno2", rk="ssprk2",
                                    bc="periodic", cfl=0.45, precision="fp64"), "burgers_sine", (3,), 0.1),
]


@pytest.mark.parametrize("name,cfg,kind,parts,T", CASES, ids=[c[0] for c in CASES])
def test_blocks_reproduce_the_whole_grid_bitwise(name, cfg, kind, parts, T):
    from paper_1912_07645_gb300.decomp import Decomposition
    whole = gpu_solver(**cfg)
    whole.set_initial_data(kind)
    n_whole = whole.evolve_to(T)
    U_whole = host(whole.state())
    t_whole, _ = whole.time()
    whole.close()
    dec = Decomposition(parts=parts, **cfg)
    dec.set_initial_data(kind)
    n_dec = dec.evolve_to(T, check_every=5)
    U_dec = host(dec.state())
    t_dec, _ = dec.time()
    dec.close()
    assert n_dec == n_whole > 5
    assert np.array_equal(t_dec, t_whole) and np.all(t_dec == T)
    assert np.array_equal(U_dec, U_whole), f"{name}: {int((U_dec != U_whole).sum())} elements differ"


@pytest.mark.parametrize("variant,parts", [(2, (1, 1, 2)), (4, (1, 1, 3)), (4, (2, 2, 1)), (3, (2, 1, 2)),
                                           (7, (1, 1, 3))])
def test_z_march_blocks_reproduce_the_whole_grid(variant, parts):
    from paper_1912_07645_gb300.decomp import Decomposition
    # z chunks of 64 / 128 planes over blocks of 53-80 planes (ragged chunks), x/y halos as well
    cfg = dict(ndim=3, n=(48, 24, 160), batch=2, eq="euler", recon="weno3", rvars="prim", flux="hllc",
               rk="ssprk3", bc=[("periodic", "periodic"), ("outflow", "reflective"), ("periodic", "periodic")],
               cfl=0.3, precision="fp32", seed=9)
    whole = gpu_solver(**cfg)
    whole.set_tile_variant(variant)
    whole.set_initial_data("kh")
    n_whole = whole.evolve_to(0.02)
    U_whole = host(whole.state())
    whole.close()
    dec = Decomposition(parts=parts, tile_variant=variant, **cfg)
    dec.set_initial_data("kh")
    n_dec = dec.evolve_to(0.02)
    U_dec = host(dec.state())
    dec.close()
    assert n_dec == n_whole > 5
    assert np.array_equal(U_dec, U_whole), f"{int((U_dec != U_whole).sum())} elements differ"


def test_decomposed_sod_matches_the_oracle_bitwise():
    from paper_1912_07645_gb300.decomp import Decomposition
    cfg = dict(ndim=1, n=(256,), batch=1, eq="euler", recon="mc", rvars="prim", flux="hllc", rk="ssprk2",
               bc=[("outflow", "reflective")], cfl=0.45, precision="fp64")
    dec = Decomposition(parts=(5,), **cfg)
    dec.set_initial_data("sod")
    dec.evolve_to(0.2)
    U = host(dec.state())
    dec.close()
    d = oracle.make_desc(**cfg)
    ref, _, _ = oracle.evolve(d, oracle.init(d, "sod", 1), T=0.2)
    assert np.array_equal(U, ref)


def test_block_statistics_and_totals():
    from paper_1912_07645_gb300.decomp import Decomposition
    cfg = CASES[3][1]
    whole = gpu_solver(**cfg)
    whole.set_initial_data("kh")
    whole.evolve_to(0.05)
    whole.stats_init()
    whole.stats_accumulate()
    _, mean_w, var_w = whole.stats_read()
    mean_w, var_w = host(mean_w), host(var_w)
    tot_w = host(whole.totals())
    whole.close()
    dec = Decomposition(parts=(2, 2), **cfg)
    dec.set_initial_data("kh")
    dec.evolve_to(0.05)
    tot = host(dec.totals())
    nx, ny = cfg["n"]
    for (bx, by, _), b in zip(dec.coords, dec.blocks):
        b.stats_init()
        b.stats_accumulate()
        _, m, v = b.stats_read()
        m = host(m).reshape(4, ny // 2, nx // 2)
        v = host(v).reshape(4, ny // 2, nx // 2)
        sl = (slice(None), slice(by * ny // 2, (by + 1) * ny // 2), slice(bx * nx // 2, (bx + 1) * nx // 2))
        assert np.array_equal(m, mean_w.reshape(4, ny, nx)[sl])
        assert np.array_equal(v, var_w.reshape(4, ny, nx)[sl])
    # the same statistics through the driver, assembled into the whole grid
    for b in dec.blocks:
        b.stats_init()                  # fresh accumulators
    dec.stats_accumulate()
    cnt, mean_d, var_d = dec.stats_read()
    assert cnt == cfg["batch"]
    assert np.array_equal(host(mean_d).reshape(4, ny, nx), mean_w.reshape(4, ny, nx))
    assert np.array_equal(host(var_d).reshape(4, ny, nx), var_w.reshape(4, ny, nx))
    dec.close()
    # totals are sums in another order: equal to FP64 rounding
    np.testing.assert_allclose(tot, tot_w, rtol=1e-13, atol=1e-13 * np.abs(tot_w).max())


def test_protocol_errors_are_reported():
    import paper_1912_07645_gb300 as alsv
    from paper_1912_07645_gb300.decomp import Decomposition
    cfg = CASES[0][1]
    dec = Decomposition(parts=(2, 1), **cfg)
    dec.set_initial_data("kh")
    b = dec.blocks[0]

    def status(fn):
        with pytest.raises(alsv.AlsvError) as ei:
            fn()
        return ei.value.status_name

    assert status(lambda: b.step(1)) == "ERR_INVALID_ARG"           # whole steps would skip the exchange
    assert status(lambda: b.evolve_to(0.1)) == "ERR_INVALID_ARG"
    assert status(lambda: b.stage(1)) == "ERR_INVALID_ARG"          # out of order
    b.stage(0)
    assert status(lambda: b.speed_max(dec.smax[0])) == "ERR_INVALID_ARG"   # mid-step
    assert status(lambda: b.finish_step(dec.smax[0], True)) == "ERR_INVALID_ARG"
    assert status(lambda: b.structure_function(0, 2, 2)) == "ERR_INVALID_ARG"
    dec.close()
    # a halo face without bound buffers
    from paper_1912_07645_gb300.decomp import block_config
    s = gpu_solver(**block_config(CASES[3][1], (2, 1, 1), (0, 0, 0)))     # FP32 2D: every schedule
    s.set_initial_data("kh")
    assert status(lambda: s.stage(0)) == "ERR_NOT_READY"
    assert status(lambda: s.autotune()) == "ERR_NOT_READY"
    s.bind_halo()
    # tile schedules without halo reads are not offered to a block
    ch, ms = alsv.alsv_autotune(s.ctx, 1)
    assert len(ms) == alsv.alsv_num_tile_variants(s.ctx) and ch in (0, 1, 2)
    assert all(m > 0 for m in ms[:3]) and all(m < 0 for m in ms[3:])
    s.close()


def test_speed_max_combine_is_the_nan_propagating_maximum():
    """The cross-block CFL maximum runs in the library: per sample the largest value over the
    blocks, with a NaN or +infinity in any block (a non-physical sample) kept."""
    import torch
    import paper_1912_07645_gb300 as alsv
    rng = np.random.default_rng(8)
    n_blocks, samples = 5, 1000
    vals = rng.uniform(0.0, 10.0, (n_blocks, samples))
    vals[2, 7] = np.nan
    vals[0, 9] = np.nan            # NaN in the first input too
    vals[4, 11] = np.inf
    ins = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in vals]
    out = torch.full((samples,), -1.0, dtype=torch.float64, device="cuda")
    alsv.alsv_speed_max_combine(ins, out)
    o = host(out)
    ref = vals.max(axis=0)          # numpy's max propagates NaN
    assert np.array_equal(np.isnan(o), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.array_equal(o[ok], ref[ok]) and o[11] == np.inf
    with pytest.raises(alsv.AlsvError, match="n must be"):
        alsv.alsv_speed_max_combine(ins * 13, out)   # 65 inputs


@pytest.mark.parametrize("case,variant", [("kh2d_fp64_3x2_mixed", None), ("kh3d_fp32_1x2x2", None),
                                          ("kh3d_fp32_1x2x2", 5), ("sod_fp64_x4", None)])
def test_overlapped_stage_parts_equal_whole_stages(case, variant):
    """Each stage run as two parts around the exchange (the tiles that read no halo buffer first,
    then the others: the paper's overlap of the exchange with the inner-domain computation, the
    distributed transport's default) gives bitwise the state of whole stages run after the
    exchange, and of the undivided grid."""
    import torch
    _, cfg, init, parts, T = [c for c in CASES if c[0] == case][0]
    from paper_1912_07645_gb300.decomp import Decomposition
    out = []
    for overlap in (True, False):
        D = Decomposition(parts=parts, overlap=overlap, tile_variant=variant, **cfg)
        D.set_initial_data(init)
        D.step(4)
        D.sync()
        out.append(host(D.state()))
        D.close()
    assert np.array_equal(out[0], out[1])
    S = gpu_solver(**cfg)
    if variant is not None:
        S.set_tile_variant(variant)
    S.set_initial_data(init)
    S.step(4)
    assert np.array_equal(out[0], host(S.state()))
    S.close()


def test_stage_part_protocol():
    import paper_1912_07645_gb300 as alsv
    from paper_1912_07645_gb300.decomp import Decomposition
    _, cfg, init, parts, _ = CASES[0]
    D = Decomposition(parts=parts, **cfg)
    D.set_initial_data(init)
    b = D.blocks[0]

    def status(fn):
        with pytest.raises(alsv.AlsvError) as ei:
            fn()
        return ei.value.status_name

    b.stage_part(0, "boundary")                      # either order
    assert status(lambda: b.stage_part(0, "boundary")) == "ERR_INVALID_ARG"    # twice
    assert status(lambda: b.stage(0)) == "ERR_INVALID_ARG"                     # mixed with a whole stage
    assert status(lambda: b.speed_max(D.smax[0])) == "ERR_INVALID_ARG"         # mid-stage
    assert status(lambda: b.stage_part(1, "interior")) == "ERR_INVALID_ARG"    # out of order
    b.stage_part(0, "interior")
    b.stage_part(1, "interior")                      # stage 0 complete: stage 1 may start
    D.close()
