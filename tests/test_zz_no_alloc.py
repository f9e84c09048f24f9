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


def test_noalloc_totals_match_context_totals_twice():
    torch = need_gpu()
    from paper_1912_07645_gb300 import build
    build.build()
    import paper_1912_07645_gb300 as alsv
    cfg = dict(ndim=2, n=(96, 80), batch=5, eq="euler", recon="weno3", flux="hllc", rvars="prim", rk="ssprk3",
               bc="periodic", cfl=0.4, precision="fp32", seed=314)
    S = gpu_solver(**cfg)
    S.set_initial_data("kh")
    desc = alsv.make_desc(**cfg)
    for call in range(2):
        S.step(3)                               # a different state for each call
        ref = S.totals()
        with torch.cuda.stream(S.stream):
            out = torch.full((5, 4), float("nan"), dtype=torch.float64, device="cuda")
        alsv.alsv_conservation_totals_noalloc(desc, S.U, out, S.stream.cuda_stream)
        r, o = host(ref), host(out)
        scale = np.abs(host(S.U)).reshape(5, 4, -1).sum(axis=2) / (96 * 80)
        assert np.all(np.abs(o - r) <= 1e-14 * np.maximum(scale, 1.0)), (call, o - r)
    # sizes beyond the static scratch are rejected with a clear message
    big = alsv.make_desc(ndim=2, n=(1024, 1024), batch=4096, precision="fp32")
    with pytest.raises(alsv.AlsvError, match="static scratch"):
        alsv.alsv_conservation_totals_noalloc(big, S.U, out, S.stream.cuda_stream)
    S.close()
