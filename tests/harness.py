"""Helpers for GPU-vs-oracle parity tests: build one configuration for both sides, run, compare."""
import numpy as np
import pytest

import oracle


def both_descs(**cfg):
    import paper_1912_07645_gb300 as alsv
    return alsv.make_desc(**cfg), oracle.make_desc(**cfg)


def gpu_solver(**cfg):
    import paper_1912_07645_gb300 as alsv
    return alsv.Solver(alsv.make_desc(**cfg))


def host(t) -> np.ndarray:
    """Copy a device tensor to host after all streams finished (the solver works on its own
    non-blocking stream, so a plain .cpu() on the default stream could race with it)."""
    import torch
    torch.cuda.synchronize()
    return t.detach().to("cpu").double().numpy()


P1_NEAR_ZERO = 1e-3


def p1_scale(ov: np.ndarray) -> np.ndarray:
    """Per-cell scale of the FP64 rule for one variable: |o| itself, except for near-zero values
    (|o| < 1e-3 max|o_v|), which are measured against the variable's maximum magnitude instead."""
    vmax = float(np.abs(ov).max())
    if vmax == 0.0:
        return np.ones_like(ov)
    a = np.abs(ov)
    return np.where(a >= P1_NEAR_ZERO * vmax, a, vmax)


def p1_check(g: np.ndarray, o: np.ndarray, rel: float = 1e-12, what: str = ""):
    """FP64 parity, per cell: |g - o| <= rel |o|, with the floor rel * max|o_v| only for cells whose
    value is near zero (|o| < 1e-3 max|o_v|, variable by variable)."""
    assert g.shape == o.shape, (g.shape, o.shape)
    nv = o.shape[1]
    bad_total = 0
    worst = 0.0
    for v in range(nv):
        ov, gv = o[:, v], g[:, v]
        err = np.abs(gv - ov) / p1_scale(ov)
        bad_total += int((err > rel).sum())
        worst = max(worst, float(err.max()))
    assert bad_total == 0, f"{what}: {bad_total} cells differ by more than {rel} (worst {worst:.3e})"
    return worst


def p2_check(g: np.ndarray, o: np.ndarray, rel: float = 2e-5, what: str = ""):
    """FP32 parity: relative L1 per variable, sum|g - o| / sum|o| <= rel (floor for zero fields)."""
    nv = o.shape[1]
    worst = 0.0
    for v in range(nv):
        num = np.abs(g[:, v] - o[:, v]).sum()
        den = np.abs(o[:, v]).sum()
        if den == 0:
            den = o[:, v].size * max(1.0, np.abs(o).max())
        worst = max(worst, num / den)
    assert worst <= rel, f"{what}: relative L1 {worst:.3e} > {rel}"
    return worst


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch
