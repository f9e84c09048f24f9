"""The C ABI from plain C: tests/c_client/sod_client.c includes only include/alsv.h and the CUDA
runtime, allocates its own device buffers and runs the Sod tube (Sec. 3, 1D configuration) to
T = 0.2. On the CPU the client must compile and link against libalsv.so; on the GPU its output must
equal the oracle's Sod run bitwise (the FP64 path evaluates the oracle's operations)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1912_07645_gb300")


def cuda_home():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return cand
    pytest.skip("CUDA toolkit headers not found")


def build_client(tmp_path):
    from paper_1912_07645_gb300 import build
    build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    cuda = cuda_home()
    exe = str(tmp_path / "sod_client")
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-O2", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_client", "sod_client.c"),
           "-o", exe, "-L" + PKG, "-lalsv", "-L" + os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + PKG + ":" + os.path.join(cuda, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(build_client(tmp_path))


@pytest.mark.gpu
def test_c_client_sod_equals_the_oracle(tmp_path):
    from harness import need_gpu
    need_gpu()
    import oracle
    exe = build_client(tmp_path)
    out = str(tmp_path / "sod.txt")
    r = subprocess.run([exe, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = open(out).read().split("\n")
    steps, count = (int(v) for v in lines[0].split())
    totals = np.array([float(v) for v in lines[1].split()])
    U = np.array([[float(v) for v in l.split()] for l in lines[2:] if l.strip()])   # [cells, 3]
    d = oracle.make_desc(ndim=1, n=(1024,), eq="euler", recon="mc", rvars="prim", flux="hllc", rk="ssprk2",
                         bc="outflow", cfl=0.45)
    ref, ref_steps, _ = oracle.evolve(d, oracle.init(d, "sod", 1), T=0.2)
    assert count == 1 and steps == int(ref_steps[0])
    assert np.array_equal(U.T, ref[0, :, 0, 0, :])
    np.testing.assert_allclose(totals, oracle.totals(d, ref)[0], rtol=1e-13)
