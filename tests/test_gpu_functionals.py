"""Point and joint PDFs, multi-point correlators and structure functions (Sec. 2.2) on the GPU
against the oracle's definitions, evaluated on the GPU's own states (the quantities are FP64 on
both sides)."""
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


def kh_run(n, batch, precision, steps, bc="periodic", seed=4, ndim=2):
    cfg = dict(ndim=ndim, n=n, batch=batch, eq="euler", recon="mc", flux="hllc", rvars="prim", rk="ssprk2", bc=bc,
               cfl=0.4, precision=precision, seed=seed)
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    S.step(steps)
    S.sync()
    return S


def test_point_pdf_counts_are_exact_and_stream():
    S = kh_run((48, 40), 16, "fp32", 5)
    nx, ny = 48, 40
    cells = [0, 7 * nx + 3, 10 * nx + 20, 30 * nx + 47, nx * ny - 1]
    c = S.point_pdf(0, cells, 0.8, 2.2, 7)
    U1 = host(S.U).reshape(S.level_shape(0))
    S.close()
    S2 = kh_run((48, 40), 16, "fp32", 5, seed=5)
    c = S2.point_pdf(0, cells, 0.8, 2.2, 7, counts=c)
    U2 = host(S2.U).reshape(S2.level_shape(0))
    got = host(c).astype(np.int64)
    S2.close()
    ref = oracle.point_pdf(np.concatenate([U1, U2]), 0, cells, 0.8, 2.2, 7)
    np.testing.assert_array_equal(got, ref)
    assert got.sum() == 32 * len(cells)


@pytest.mark.parametrize("precision,q,p,R", [("fp32", 0, 1, 16), ("fp32", 3, 2, 7), ("fp64", 1, 2, 3)])
def test_structure_function_2d_periodic(precision, q, p, R):
    import paper_1912_07645_gb300 as alsv
    S = kh_run((48, 40), 6, precision, 4)
    acc, Sp = S.structure_function(q, p, R)
    U = host(S.U).reshape(S.level_shape(0))
    head = host(acc[:8 * (R + 1)].view(S.torch.float64))
    Sp = host(Sp)
    S.close()
    cnt, sums = oracle.structure_function_sums(U, q, p, R, (1 / 48, 1 / 40), (True, True, True))
    assert head[0] == cnt == 6
    np.testing.assert_allclose(head[1:], sums, rtol=1e-12, atol=0)
    np.testing.assert_allclose(Sp, oracle.structure_function(cnt, sums, p), rtol=1e-12)


def test_structure_function_outflow_and_streaming():
    S = kh_run((40, 36), 4, "fp64", 3, bc="outflow")
    acc, _ = S.structure_function(3, 1, 5)
    U1 = host(S.U).reshape(S.level_shape(0))
    S.close()
    S2 = kh_run((40, 36), 4, "fp64", 3, bc="outflow", seed=9)
    acc, Sp = S2.structure_function(3, 1, 5, acc=acc)
    U2 = host(S2.U).reshape(S2.level_shape(0))
    head = host(acc[:48].view(S2.torch.float64))
    Sp = host(Sp)
    S2.close()
    cnt, sums = oracle.structure_function_sums(np.concatenate([U1, U2]), 3, 1, 5, (1 / 40, 1 / 36), (False, False))
    assert head[0] == cnt == 8
    np.testing.assert_allclose(head[1:6], sums, rtol=1e-12)
    np.testing.assert_allclose(Sp, oracle.structure_function(cnt, sums, 1), rtol=1e-12)


def test_structure_function_1d_3d_and_one_large_sample():
    import torch
    # 1D Sod, outflow, R = 16
    S = gpu_solver(ndim=1, n=(300,), batch=2, eq="euler", recon="mc", flux="hllc", rk="ssprk2", bc="outflow",
                   cfl=0.45, precision="fp64")
    S.set_initial_data("sod")
    S.step(40)
    acc, _ = S.structure_function(0, 2, 16)
    U = host(S.U).reshape(S.level_shape(0))
    head = host(acc[:8 * 17].view(torch.float64))
    S.close()
    cnt, sums = oracle.structure_function_sums(U, 0, 2, 16, (1 / 300,), (False,))
    np.testing.assert_allclose(head[1:], sums, rtol=1e-12)
    # 3D slab, periodic, R = 4
    S = kh_run((10, 12, 9), 2, "fp32", 2, ndim=3)
    acc, _ = S.structure_function(4, 1, 4)
    U = host(S.U).reshape(S.level_shape(0))
    head = host(acc[:40].view(torch.float64))
    S.close()
    cnt, sums = oracle.structure_function_sums(U, 4, 1, 4, (0.1, 1 / 12, 1 / 9), (True, True, True))
    np.testing.assert_allclose(head[1:], sums, rtol=1e-12)
    # one 256^2 sample: the sample's tiles are split over many CTAs
    S = kh_run((256, 256), 1, "fp32", 3)
    acc, _ = S.structure_function(0, 2, 4)
    U = host(S.U).reshape(S.level_shape(0))
    head = host(acc[:40].view(torch.float64))
    S.close()
    cnt, sums = oracle.structure_function_sums(U, 0, 2, 4, (1 / 256, 1 / 256), (True, True, True))
    np.testing.assert_allclose(head[1:], sums, rtol=1e-12)


def test_functionals_reject_bad_arguments():
    import paper_1912_07645_gb300 as alsv
    S = kh_run((20, 20), 1, "fp32", 1)
    for q, p, R in ((0, 3, 4), (7, 1, 4), (0, 1, 17), (0, 1, 10)):   # R = 10 needs 21 periodic cells
        with pytest.raises(alsv.AlsvError) as ei:
            S.structure_function(q, p, R, acc=S.torch.zeros(1 << 16, dtype=S.torch.uint8, device="cuda"))
        assert ei.value.status_name == "ERR_INVALID_ARG"
    with pytest.raises(alsv.AlsvError):
        S.point_pdf(0, [0], 1.0, 1.0, 4)
    S.close()


def test_joint_pdf_and_correlators():
    S = kh_run((48, 40), 16, "fp32", 5)
    nx = 48
    cells = [0, 9 * nx + 3, 20 * nx + 30]
    c = S.joint_pdf(0, 3, cells, 0.8, 2.2, 6, 2.3, 2.7, 5)
    # one call per set size k (a call takes sets of one size)
    sets2 = [[9 * nx + 3, 9 * nx + 4], [5, 5], [0, 39 * nx + 47]]
    sets3 = [[0, 20 * nx + 30, 39 * nx + 47], [7 * nx, 7 * nx + 1, 7 * nx + 2]]
    acc2 = S.correlator(1, sets2)
    acc3 = S.correlator(3, sets3)
    U = host(S.U).reshape(S.level_shape(0))
    got, a2, a3 = host(c).astype(np.int64), host(acc2), host(acc3)
    S.close()
    np.testing.assert_array_equal(got, oracle.joint_pdf(U, 0, 3, cells, 0.8, 2.2, 6, 2.3, 2.7, 5))
    for acc, q, sets in ((a2, 1, sets2), (a3, 3, sets3)):
        n, sums = oracle.correlator(U, q, sets)
        assert acc[0] == n == 16
        np.testing.assert_allclose(acc[1:], sums, rtol=1e-13, atol=1e-15)
