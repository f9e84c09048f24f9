"""Spatial domain decomposition on the CPU (no GPU): the host logic (block ranges, neighbours,
halo faces), the C ABI's validation of block descriptors, and the stage-by-stage protocol with
both transports - in one process, and as gloo ranks (world size 2 and 4) through
torch.distributed - driving oracle-backed host blocks. The blocks must reproduce the undivided
grid bitwise, and the undivided protocol run must match the oracle's own time loop."""
import os
import socket

import numpy as np
import pytest

import oracle
from host_block import OracleBlock
from inputs import kh_theta
from paper_1912_07645_gb300.decomp import Decomposition, block_config, block_coords, neighbour, split

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_neighbours_and_block_faces():
    assert split(10, 3) == [(0, 4), (4, 3), (7, 3)]
    assert split(8, 1) == [(0, 8)]
    with pytest.raises(ValueError):
        split(2, 3)
    parts = (3, 2, 1)
    coords = block_coords(parts)
    assert coords[0] == (0, 0, 0) and coords[1] == (1, 0, 0) and coords[3] == (0, 1, 0)
    per = [True, False, False]
    assert neighbour((0, 0, 0), 0, parts, per) == (2, 0, 0)       # periodic wrap in x
    assert neighbour((2, 0, 0), 1, parts, per) == (0, 0, 0)
    assert neighbour((0, 0, 0), 2, parts, per) is None           # physical face in y
    assert neighbour((0, 0, 0), 3, parts, per) == (0, 1, 0)
    assert neighbour((0, 0, 0), 4, parts, per) is None           # z not decomposed
    cfg = dict(ndim=2, n=(30, 20), bc=[("periodic", "periodic"), ("reflective", "outflow")])
    kw = block_config(cfg, parts, (1, 1, 0))
    assert kw["n"] == (10, 10) and kw["global_n"] == (30, 20) and kw["offset"] == (10, 10)
    assert kw["bc"][0] == ("halo", "halo") and kw["bc"][1] == ("halo", "outflow")
    kw = block_config(cfg, parts, (0, 0, 0))
    assert kw["bc"][1] == ("reflective", "halo")
    # a direction that is not decomposed keeps its conditions
    kw = block_config(cfg, (1, 2, 1), (0, 0, 0))
    assert kw["bc"][0] == ("periodic", "periodic")


def test_split_and_neighbours_edge_cases():
    assert split(5, 5) == [(i, 1) for i in range(5)]
    assert split(7, 2) == [(0, 4), (4, 3)]
    # two blocks on a periodic direction: the same neighbour on both sides
    per = [True, True, True]
    assert neighbour((0, 0, 0), 0, (2, 1, 1), per) == (1, 0, 0)
    assert neighbour((0, 0, 0), 1, (2, 1, 1), per) == (1, 0, 0)
    # 3D block: faces only along the decomposed direction, offsets and the whole grid's counts
    cfg = dict(ndim=3, n=(8, 6, 10), bc=[("periodic", "periodic"), ("outflow", "outflow"), ("reflective", "outflow")])
    kw = block_config(cfg, (1, 1, 3), (0, 0, 2))
    assert kw["n"] == (8, 6, 3) and kw["offset"] == (0, 0, 7) and kw["global_n"] == (8, 6, 10)
    assert kw["bc"][0] == ("periodic", "periodic") and kw["bc"][1] == ("outflow", "outflow")
    assert kw["bc"][2] == ("halo", "outflow")
    kw = block_config(cfg, (1, 1, 3), (0, 0, 0))
    assert kw["bc"][2] == ("reflective", "halo")


def test_decomposition_rejects_bad_layouts():
    cfg, _, _, _ = CASES["sod1d_x4"]
    _, U0 = initial("sod1d_x4")
    with pytest.raises(ValueError):
        Decomposition(parts=(2, 2, 1), make_block=lambda **kw: OracleBlock(U0, **kw), **cfg)   # y in 1D
    with pytest.raises(ValueError):
        Decomposition(parts=(2,), transport="carrier pigeon", make_block=lambda **kw: OracleBlock(U0, **kw), **cfg)
    with pytest.raises(ValueError):
        split(3, 4)


@pytest.fixture(scope="module")
def alsv():
    from paper_1912_07645_gb300 import build
    build.build()
    import paper_1912_07645_gb300 as a
    a.load()
    return a


def test_block_descriptor_validation(alsv):
    def init(**kw):
        ctx, _ = alsv.alsv_init_grid(alsv.make_desc(**kw), 0)
        return ctx

    base = dict(ndim=2, n=(16, 8), batch=3, recon="weno3")
    ctx = init(global_n=(16, 32), offset=(0, 8), bc=[("periodic", "periodic"), ("halo", "halo")], **base)
    g, elems = alsv.alsv_halo_info(ctx)
    assert g == 2 and elems == [0, 0, 3 * 4 * 2 * 16, 3 * 4 * 2 * 16, 0, 0]
    alsv.alsv_destroy(ctx)
    ctx = init(ndim=3, n=(6, 5, 4), recon="pc", bc=[("halo", "outflow"), ("periodic", "periodic"), ("outflow", "halo")],
               global_n=(12, 5, 9), offset=(6, 0, 5))
    g, elems = alsv.alsv_halo_info(ctx)
    assert g == 1 and elems == [5 * 4 * 5, 0, 0, 0, 0, 6 * 5 * 5]
    alsv.alsv_destroy(ctx)
    bad = [
        dict(global_n=(16, 12), offset=(0, 8), **base),                       # block leaves the grid
        dict(global_n=(16, 16), offset=(0, -1), **base),                      # negative offset
        dict(offset=(0, 4), **base),                                          # offset without global_n
        dict(bc=[("periodic", "periodic"), ("halo", "periodic")], **base),    # periodic pairs with periodic
        dict(ndim=2, n=(16, 1), batch=1, recon="mc", bc=[("periodic", "periodic"), ("halo", "halo")]),  # n < g
        dict(ndim=2, levels=[((8, 8), 2), ((16, 16), 2)], bc=[("periodic", "periodic"), ("halo", "halo")]),
        dict(ndim=2, levels=[((8, 8), 2), ((16, 16), 2)], global_n=(16, 16)),
    ]
    for kw in bad:
        with pytest.raises(alsv.AlsvError) as ei:
            init(**kw)
        assert ei.value.status_name == "ERR_INVALID_ARG", kw
    d = alsv.make_desc(ndim=1, n=(8,))
    d.global_n[1] = 4                                                          # inactive direction
    with pytest.raises(alsv.AlsvError, match="inactive"):
        alsv.alsv_init_grid(d, 0)


# (whole-grid config, initial data, parts, end time)
CASES = {
    "kh2d_x2": (dict(ndim=2, n=(32, 32), eq="euler", recon="mc", rvars="prim", flux="hllc", rk="ssprk2",
                     bc="periodic", cfl=0.4), "kh", (2, 1, 1), 0.03),
    "kh2d_y2": (dict(ndim=2, n=(32, 32), eq="euler", recon="weno3", rvars="prim", flux="hllc", rk="ssprk3",
                     bc="periodic", cfl=0.4), "kh", (1, 2, 1), 0.03),
    "kh2d_2x2": (dict(ndim=2, n=(32, 32), eq="euler", recon="mc", rvars="cons", flux="rusanov", rk="ssprk3",
                      bc=[("periodic", "periodic"), ("reflective", "outflow")], cfl=0.4), "kh", (2, 2, 1), 0.03),
    "kh2d_3x2_ragged": (dict(ndim=2, n=(32, 32), eq="euler", recon="weno3", rvars="prim", flux="hllc",
                             rk="ssprk2", bc="periodic", cfl=0.4), "kh", (3, 2, 1), 0.03),
    "sod1d_x4": (dict(ndim=1, n=(64,), eq="euler", recon="weno3", rvars="prim", flux="hllc", rk="ssprk3",
                      bc="outflow", cfl=0.45), "sod", (4, 1, 1), 0.05),
    "burgers1d_x3": (dict(ndim=1, n=(64,), eq="burgers", recon="pc", flux="hll", rk="ssprk2", bc="periodic",
                          cfl=0.45), "burgers_sine", (3, 1, 1), 0.05),
    "kh3d_z2": (dict(ndim=3, n=(8, 16, 16), eq="euler", recon="mc", rvars="prim", flux="hllc", rk="ssprk2",
                     bc="periodic", cfl=0.3), "kh", (1, 1, 2), 0.06),
}


def initial(case, B=2):
    cfg, kind, _, _ = CASES[case]
    d = oracle.make_desc(**cfg)
    theta = kh_theta(B, 5, P=128 if cfg["ndim"] == 3 else 20) if kind == "kh" else None
    return d, oracle.init(d, kind, B, theta)


def run(case, parts, transport="local", group=None):
    cfg, _, _, T = CASES[case]
    _, U0 = initial(case)
    dec = Decomposition(parts=parts, transport=transport, group=group,
                        make_block=lambda **kw: OracleBlock(U0, **kw), **cfg)
    dec.set_initial_data()
    steps = dec.evolve_to(T, check_every=3)
    return dec, steps


@pytest.mark.parametrize("case", list(CASES))
def test_local_blocks_reproduce_the_whole_grid(case):
    cfg, _, parts, T = CASES[case]
    whole, n_whole = run(case, (1, 1, 1))
    U_whole = whole.state().numpy().copy()
    dec, n_dec = run(case, parts)
    assert n_dec == n_whole > 3
    np.testing.assert_array_equal(dec.state().numpy(), U_whole)
    t, _ = dec.time()
    assert np.all(t == T)
    # the undivided protocol run against the oracle's own time loop
    d, U0 = initial(case)
    U_ref, steps, _ = oracle.evolve(d, U0, T=T)
    assert int(steps.max()) == n_whole
    np.testing.assert_allclose(U_whole, U_ref, rtol=1e-12, atol=1e-12 * np.abs(U_ref).max())


def _dist_worker(rank, world, port, case, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    _, _, parts, _ = CASES[case]
    dec, steps = run(case, parts, transport="dist")
    mine = (dec.coords[0], dec.state().numpy().copy(), steps)
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        np.savez(out_path, **{f"b{c[0]}_{c[1]}_{c[2]}": U for c, U, _ in got},
                 steps=np.array([s for _, _, s in got]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("case,world", [("kh2d_x2", 2), ("kh2d_2x2", 4), ("kh2d_3x2_ragged", 6)])
def test_gloo_ranks_reproduce_the_whole_grid(tmp_path, case, world):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "blocks.npz")
    mp.start_processes(_dist_worker, args=(world, port, case, out), nprocs=world, join=True, start_method="spawn")
    r = np.load(out)
    whole, n_whole = run(case, (1, 1, 1))
    U = whole.state().numpy()
    cfg, _, parts, _ = CASES[case]
    n = list(cfg["n"]) + [1] * (3 - cfg["ndim"])
    rng = [split(n[k], parts[k]) for k in range(3)]
    for c in block_coords(parts):
        (ox, nx), (oy, ny), (oz, nz) = rng[0][c[0]], rng[1][c[1]], rng[2][c[2]]
        np.testing.assert_array_equal(r[f"b{c[0]}_{c[1]}_{c[2]}"], U[:, :, oz:oz + nz, oy:oy + ny, ox:ox + nx])
    assert list(r["steps"]) == [n_whole] * world
