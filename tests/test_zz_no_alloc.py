"""The allocation-free totals entry point (static device scratch, no context, no workspace) must
give the same totals as the context-based alsv_conservation_totals, call after call.

It serves callers that cannot allocate device memory (a plugin without an allocator, a service
under a fixed device-memory budget). The file name sorts last so that a run stopping at the first
failure has already run every other test; the test also passes alone in a fresh process.
"""
import numpy as np
import pytest

from harness import gpu_solver, host, need_gpu

pytestmark = pytest.mark.gpu


def _check_twice(cfg, nsamples, nv, cells):
    torch = need_gpu()
    import paper_1912_07645_gb300 as alsv
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    desc = alsv.make_desc(**cfg)
    for call in range(2):
        S.step(3)                               # a different state for each call
        ref = S.totals()
        with torch.cuda.stream(S.stream):
            out = torch.full((nsamples, nv), float("nan"), dtype=torch.float64, device="cuda")
        alsv.alsv_conservation_totals_noalloc(desc, S.U, out, S.stream.cuda_stream)
        r, o = host(ref), host(out)
        # the same kernels in the same order: equal up to the last bits of the FP64 sums
        scale = np.abs(r) + 1e-300
        assert np.all(np.isfinite(o)), (call, o)
        assert np.all(np.abs(o - r) <= 1e-14 * np.maximum(scale, 1.0)), (call, o - r)
    return S, out


def test_noalloc_totals_match_context_totals_twice():
    from paper_1912_07645_gb300 import build
    build.build()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=(96, 80), batch=5, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=314)
    S, out = _check_twice(cfg, 5, 4, 96 * 80)
    # sizes beyond the static scratch are rejected with a clear message
    big = alsv.make_desc(ndim=2, n=(1024, 1024), batch=4096, precision="fp32")
    with pytest.raises(alsv.AlsvError, match="static scratch"):
        alsv.alsv_conservation_totals_noalloc(big, S.U, out, S.stream.cuda_stream)
    # so is a single sample with more chunks than the reduction's grid holds
    huge = alsv.make_desc(ndim=1, n=(65536 * 4096 + 1,), batch=1, eq="burgers", precision="fp32")
    with pytest.raises(alsv.AlsvError, match="65535 chunks"):
        alsv.alsv_conservation_totals_noalloc(huge, S.U, out, S.stream.cuda_stream)
    # and a block descriptor that does not lie inside its whole grid
    blk = alsv.make_desc(ndim=2, n=(96, 80), batch=5, precision="fp32")
    blk.global_n[0], blk.offset[0] = 100, 10
    with pytest.raises(alsv.AlsvError, match="inside the whole grid"):
        alsv.alsv_conservation_totals_noalloc(blk, S.U, out, S.stream.cuda_stream)
    S.close()


def test_noalloc_totals_fp64_and_levels():
    cfg = dict(ndim=2, n=(70, 45), batch=3, eq="euler", recon="mc", flux="rusanov", rvars="prim", rk="ssprk2",
               bc="periodic", cfl=0.4, precision="fp64", seed=9)
    S, _ = _check_twice(cfg, 3, 4, 70 * 45)
    S.close()
    lv = [((32, 32), 4), ((64, 64), 2), ((96, 96), 1)]
    cfg = dict(ndim=2, levels=lv, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=5)
    S, _ = _check_twice(cfg, 7, 4, None)
    S.close()
