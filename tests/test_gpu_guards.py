"""Guard-zone memory checks (compute-sanitizer is not available on the GPU pool): every caller-owned
buffer is carved from an allocation with 1 MiB guard zones before and after it, all bytes set to
0xFF (a NaN for every float and double), and the workspace and state start as that NaN pattern
too. After the calls, the guards must be untouched (no write outside a buffer), the device status
must be OK and every output finite (a read outside a buffer, or of workspace that was never
written, brings a NaN in). Covers tiny, odd and ragged grids in 1D/2D/3D, every stage schedule
that supports the scheme, statistics, totals, functionals, the MLMC estimator, the adjoint and
the halo exchange of decomposed grids."""
import numpy as np
import pytest

from harness import need_gpu

pytestmark = pytest.mark.gpu
GUARD = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()
    from paper_1912_07645_gb300 import build
    build.build()


class Arena:
    def __init__(self):
        import torch
        self.torch = torch
        self.parts = []

    def buf(self, nbytes, dtype=None, zero=False):
        torch = self.torch
        dtype = dtype or torch.uint8
        nbytes = max(int(nbytes), 8)
        raw = torch.full((GUARD + nbytes + GUARD,), 0xFF, dtype=torch.uint8, device="cuda")
        inner = raw[GUARD:GUARD + nbytes]
        if zero:
            inner.zero_()
        self.parts.append((raw, nbytes))
        esz = torch.empty((), dtype=dtype).element_size()
        return inner[:nbytes - nbytes % esz].view(dtype)

    def check(self, what=""):
        torch = self.torch
        torch.cuda.synchronize()
        for raw, n in self.parts:
            assert bool((raw[:GUARD] == 0xFF).all()), f"{what}: write below a buffer"
            assert bool((raw[GUARD + n:] == 0xFF).all()), f"{what}: write above a buffer"


def finite(t, what):
    import torch
    torch.cuda.synchronize()
    assert bool(torch.isfinite(t).all()), f"{what}: non-finite output"


def run_context(arena, cfg, kind, steps, tag):
    """One context on guarded buffers: init, steps under every supported schedule, statistics,
    totals. Returns (ctx, U)."""
    import torch

    import paper_1912_07645_gb300 as alsv
    d = alsv.make_desc(**cfg)
    stream = torch.cuda.current_stream().cuda_stream
    ctx, wsb = alsv.alsv_init_grid(d, stream)
    ws = arena.buf(wsb)
    alsv.alsv_bind_workspace(ctx, ws)
    fp64 = cfg.get("precision") == "fp64"
    dt = torch.float64 if fp64 else torch.float32
    U = arena.buf(alsv.alsv_state_bytes(ctx), dt)
    alsv.alsv_set_initial_data(ctx, kind, None, 0, U)
    for v in range(alsv.alsv_num_tile_variants(ctx)):
        try:
            alsv.alsv_set_tile_variant(ctx, v)
        except alsv.AlsvError:
            continue
        alsv.alsv_step(ctx, steps)
        alsv.alsv_sync(ctx)
    finite(U, tag)
    S, nv = alsv.alsv_num_samples(ctx), alsv.alsv_num_vars(ctx)
    if d.n_levels <= 1:
        st = arena.buf(alsv.alsv_stats_bytes(ctx))
        alsv.alsv_stats_reset(ctx, st)
        alsv.alsv_stats_accumulate(ctx, st)
        cells = int(np.prod(list(d.n)))
        mean = arena.buf(nv * cells * 8, torch.float64)
        var = arena.buf(nv * cells * 8, torch.float64)
        assert alsv.alsv_stats_read(ctx, st, mean, var) == S
        finite(mean, tag)
        finite(var, tag)
    tot = arena.buf(S * nv * 8, torch.float64)
    alsv.alsv_conservation_totals(ctx, tot)
    finite(tot, tag)
    if cfg.get("eq", "euler") == "euler":
        ke = arena.buf(S * 8, torch.float64)
        alsv.alsv_kinetic_energy(ctx, ke)
        finite(ke, tag)
    alsv.alsv_sync(ctx)
    arena.check(tag)
    return ctx, U


GRIDS = [
    dict(ndim=1, n=(1,), recon="pc", bc="periodic"), dict(ndim=1, n=(2,), recon="mc", bc="outflow"),
    dict(ndim=1, n=(3,), recon="weno3", bc="periodic"), dict(ndim=1, n=(7,), recon="weno3", bc="reflective"),
    dict(ndim=1, n=(257,), recon="mc", bc=[("outflow", "reflective")]),
    dict(ndim=2, n=(1, 1), recon="pc", bc="periodic"), dict(ndim=2, n=(3, 5), recon="mc", bc="outflow"),
    dict(ndim=2, n=(17, 9), recon="weno3", bc=[("periodic", "periodic"), ("reflective", "outflow")]),
    dict(ndim=2, n=(70, 45), recon="weno3", bc="periodic"), dict(ndim=2, n=(33, 64), recon="mc", bc="periodic"),
    dict(ndim=3, n=(3, 4, 5), recon="mc", bc="periodic"), dict(ndim=3, n=(9, 7, 5), recon="weno3", bc="reflective"),
    dict(ndim=3, n=(17, 9, 70), recon="weno3", bc=[("periodic", "periodic"), ("outflow", "outflow"),
                                                    ("periodic", "periodic")]),
]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("grid", GRIDS, ids=[f"{g['ndim']}d_{'x'.join(map(str, g['n']))}_{g['recon']}" for g in GRIDS])
def test_contexts_stay_inside_their_buffers(grid, precision):
    arena = Arena()
    import paper_1912_07645_gb300 as alsv
    kind = "sod" if grid["ndim"] == 1 else "kh"
    rk = "ssprk3" if grid["recon"] == "weno3" else "ssprk2"
    cfg = dict(grid, batch=3, eq="euler", rvars="prim", flux="hllc", rk=rk, cfl=0.3, precision=precision, seed=1)
    ctx, _ = run_context(arena, cfg, kind, 2, f"{grid} {precision}")
    alsv.alsv_destroy(ctx)
    # Burgers and conserved-variable reconstruction on the same grid
    ctx, _ = run_context(arena, dict(cfg, eq="burgers", flux="hll"), "burgers_sine", 2, f"{grid} {precision} burgers")
    alsv.alsv_destroy(ctx)
    cfg_c = dict(cfg, rvars="cons", flux="rusanov")
    ctx, _ = run_context(arena, cfg_c, kind, 2, f"{grid} {precision} cons")
    alsv.alsv_destroy(ctx)


def test_functionals_mlmc_and_adjoint_stay_inside_their_buffers():
    import torch

    import paper_1912_07645_gb300 as alsv
    arena = Arena()
    cfg = dict(ndim=2, n=(37, 29), batch=5, eq="euler", recon="mc", rvars="prim", flux="hllc", rk="ssprk2",
               bc="periodic", cfl=0.4, precision="fp32", seed=3)
    ctx, U = run_context(arena, cfg, "kh", 3, "functionals")
    cells = arena.buf(4 * 8, torch.int64)
    cells.copy_(torch.tensor([0, 100, 37 * 29 - 1, 500], device="cuda"))
    counts = arena.buf(4 * 9 * 8, torch.int64, zero=True)          # [points][bins + 2]
    alsv.alsv_point_pdf_accumulate(ctx, 0, cells, 0.5, 2.5, 7, counts)
    jc = arena.buf(4 * 6 * 5 * 8, torch.int64, zero=True)          # [points][4 + 2][3 + 2]
    alsv.alsv_joint_pdf_accumulate(ctx, 0, 3, cells, 0.5, 2.5, 4, 2.0, 3.0, 3, jc)
    sets = arena.buf(2 * 3 * 8, torch.int64)
    sets.copy_(torch.tensor([0, 1, 2, 30, 31, 32], device="cuda"))
    corr = arena.buf(3 * 8, torch.float64, zero=True)
    alsv.alsv_correlator_accumulate(ctx, 1, sets.view(2, 3), corr)
    finite(corr, "correlator")
    R = 4
    acc = arena.buf(alsv.alsv_structure_function_bytes(ctx, R), zero=True)
    alsv.alsv_structure_function_accumulate(ctx, 0, 2, R, acc)
    Sp = arena.buf(R * 8, torch.float64)                          # S_p(r), r = 1..R
    alsv.alsv_structure_function_read(ctx, acc, 2, R, Sp)
    finite(Sp, "structure function")
    alsv.alsv_sync(ctx)
    assert int(counts.sum()) == 4 * 5 and int(jc.sum()) == 4 * 5
    alsv.alsv_destroy(ctx)
    arena.check("functionals")

    # MLMC level table with companions
    lv = [((16, 16), 8), ((32, 32), 4), ((16, 16), 4, 1), ((64, 64), 2), ((32, 32), 2, 3)]
    cfg_m = dict(cfg, levels=lv)
    del cfg_m["n"]
    ctx, U = run_context(arena, dict(cfg_m, n=(16, 16)), "kh", 2, "mlmc")
    acc = arena.buf(alsv.alsv_mlmc_bytes(ctx))
    alsv.alsv_mlmc_reset(ctx, acc)
    alsv.alsv_mlmc_accumulate(ctx, acc)
    mean = arena.buf(4 * 64 * 64 * 8, torch.float64)
    var = arena.buf(4 * 64 * 64 * 8, torch.float64)
    lev = arena.buf(3 * 4 * 3 * 8, torch.float64)
    counts = alsv.alsv_mlmc_read(ctx, acc, mean, var, lev, 3)
    assert counts == [8, 4, 2]
    finite(mean, "mlmc mean")
    finite(var, "mlmc var")
    alsv.alsv_destroy(ctx)
    arena.check("mlmc")

    # adjoint (FP64 and FP32), workspace and outputs guarded
    for prec in ("fp64", "fp32"):
        cfg_a = dict(ndim=2, n=(24, 20), batch=3, eq="euler", recon="mc", rvars="prim", flux="rusanov",
                     rk="ssprk2", bc="periodic", cfl=0.4, precision=prec, seed=4)
        ctx, U = run_context(arena, cfg_a, "kh", 1, "adjoint")
        th = arena.buf(3 * 20 * 8, torch.float64)
        alsv.alsv_get_parameters(ctx, th)
        T = 0.02
        aws = arena.buf(alsv.alsv_adjoint_workspace_bytes(ctx, T))
        alsv.alsv_bind_adjoint_workspace(ctx, aws)
        grad = arena.buf(3 * 20 * 8, torch.float64)
        J = arena.buf(3 * 8, torch.float64)
        alsv.alsv_adjoint_evolve(ctx, T, 0, th, grad, J)
        alsv.alsv_sync(ctx)
        finite(grad, "adjoint gradient")
        finite(J, "adjoint J")
        alsv.alsv_destroy(ctx)
        arena.check(f"adjoint {prec}")


@pytest.mark.parametrize("ndim,n,parts", [(2, (37, 30), (3, 2, 1)), (3, (12, 10, 70), (2, 1, 3)), (1, (50,), (4, 1, 1))])
def test_halo_exchange_stays_inside_its_buffers(ndim, n, parts):
    import torch

    import paper_1912_07645_gb300 as alsv
    from paper_1912_07645_gb300.decomp import Decomposition
    arena = Arena()
    cfg = dict(ndim=ndim, n=n, batch=2, eq="euler", recon="weno3", rvars="prim", flux="hllc", rk="ssprk3",
               bc="periodic" if ndim > 1 else "outflow", cfl=0.3, precision="fp32", seed=6)
    D = Decomposition(parts=parts, **cfg)
    for b in D.blocks:                     # guarded halo buffers, NaN until the first exchange
        _, elems = b.halo_info()
        b.halos = [arena.buf(e * 4, torch.float32) if e else None for e in elems]
        alsv.alsv_bind_halo(b.ctx, b.halos)
    D.set_initial_data("kh" if ndim > 1 else "sod")
    D.step(4)
    D.sync()
    finite(D.state(), "blocks")
    arena.check("halo exchange")
    D.close()
