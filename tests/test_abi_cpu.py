"""Host-side checks of the C ABI (no GPU): the library loads, exports every entry point that
include/alsv.h declares, and validates descriptors without touching the device."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def alsv():
    from paper_1912_07645_gb300 import build
    build.build()
    import paper_1912_07645_gb300 as a
    a.load()
    return a


def declared_functions():
    text = open(os.path.join(ROOT, "include", "alsv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(alsv_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["alsv_init_grid", "alsv_set_initial_data", "alsv_step", "alsv_evolve_to_T",
                     "alsv_stats_accumulate", "alsv_stats_read", "alsv_adjoint_evolve",
                     "alsv_conservation_totals", "alsv_destroy", "alsv_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(alsv):
    lib = alsv.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(alsv):
    from paper_1912_07645_gb300 import _abi
    assert set(declared_functions()) == set(_abi.SIGNATURES)
    for n in declared_functions():
        assert hasattr(_abi, n)


def test_descriptor_mirror_matches_the_header():
    """The ctypes mirror of alsv_grid_desc lists the header's fields in the header's order, with the
    same scalar types and array extents (a stale mirror would shift every later field)."""
    from paper_1912_07645_gb300 import _abi
    import ctypes as C
    text = open(os.path.join(ROOT, "include", "alsv.h")).read()
    body = re.search(r"typedef struct alsv_grid_desc \{(.*?)\} alsv_grid_desc;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    ctype = {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "double": C.c_double}
    header = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = decl.split(None, 1)
        for name in (v.strip() for v in rest.split(",")):
            dims = [int(x) if x.isdigit() else {"ALSV_MAX_LEVELS": _abi.MAX_LEVELS}[x]
                    for x in re.findall(r"\[(\w+)\]", name)]
            header.append((re.match(r"\w+", name).group(0), ctype[typ], dims))
    mirror = _abi.alsv_grid_desc._fields_
    assert [h[0] for h in header] == [m[0] for m in mirror]
    for (name, typ, dims), (_, mt) in zip(header, mirror):
        for n in dims:
            assert issubclass(mt, C.Array) and mt._length_ == n, name
            mt = mt._type_
        assert mt == typ, name


def test_binding_argument_counts_match_the_prototypes():
    from paper_1912_07645_gb300 import _abi
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "alsv.h")).read(), flags=re.S)
    protos = dict(re.findall(r"\b(alsv_\w+)\s*\(([^)]*)\)\s*;", text))
    assert len(protos) == len(_abi.SIGNATURES)
    for name, params in protos.items():
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(_abi.SIGNATURES[name][1]) == n, name


def test_version(alsv):
    assert "alsv" in alsv.alsv_version()


def test_workspace_and_state_sizes(alsv):
    d = alsv.make_desc(ndim=2, n=(256, 256), batch=4096, precision="fp32", recon="weno3", rk="ssprk3")
    ctx, ws = alsv.alsv_init_grid(d, 0)
    try:
        assert alsv.alsv_state_bytes(ctx) == 4096 * 4 * 256 * 256 * 4
        assert ws >= 2 * alsv.alsv_state_bytes(ctx)      # RK3 keeps two stage buffers
        assert alsv.alsv_num_samples(ctx) == 4096 and alsv.alsv_num_vars(ctx) == 4
        (tx, ty, tz), v, work = alsv.alsv_get_tile(ctx)
        assert work == 4096 * ((256 + tx - 1) // tx) * ((256 + ty - 1) // ty)
        assert alsv.alsv_stats_bytes(ctx) == 256 + 2 * 4 * 256 * 256 * 8
    finally:
        alsv.alsv_destroy(ctx)
    d2 = alsv.make_desc(ndim=2, n=(256, 256), batch=4096, precision="fp32", rk="ssprk2")
    ctx, ws2 = alsv.alsv_init_grid(d2, 0)
    alsv.alsv_destroy(ctx)
    assert ws2 < ws                                      # RK2 needs one stage buffer


def test_mlmc_level_table_sizes(alsv):
    lv = [((64, 64), 4096), ((128, 128), 1024), ((256, 256), 256), ((512, 512), 64)]
    d = alsv.make_desc(ndim=2, levels=lv, precision="fp32", recon="weno3", rk="ssprk3")
    ctx, _ = alsv.alsv_init_grid(d, 0)
    try:
        assert alsv.alsv_num_samples(ctx) == 4096 + 1024 + 256 + 64
        assert alsv.alsv_state_bytes(ctx) == sum(b * 4 * n[0] * n[1] * 4 for n, b in lv)
    finally:
        alsv.alsv_destroy(ctx)


@pytest.mark.parametrize("field,value,msg", [
    ("ndim", 0, "ndim"), ("ndim", 4, "ndim"), ("eq", 7, "eq"), ("recon", 4, "recon"), ("flux", 9, "flux"), ("flux", 8, "flux"),
    ("rk", 4, "rk"), ("precision", 2, "precision"), ("gamma", 1.0, "gamma"), ("batch", 0, "batch"),
    ("cfl", 0.0, "cfl"), ("weno_eps", -1.0, "weno_eps"),
])
def test_descriptor_validation(alsv, field, value, msg):
    d = alsv.make_desc(ndim=2, n=(16, 16), batch=2)
    setattr(d, field, value)
    with pytest.raises(alsv.AlsvError) as ei:
        alsv.alsv_init_grid(d, 0)
    assert ei.value.status_name == "ERR_INVALID_ARG"
    assert msg in str(ei.value)


def test_validation_of_boundaries_and_sizes(alsv):
    d = alsv.make_desc(ndim=1, n=(16,), bc=[("periodic", "outflow")])
    with pytest.raises(alsv.AlsvError, match="periodic"):
        alsv.alsv_init_grid(d, 0)
    d = alsv.make_desc(ndim=1, n=(1,), recon="weno3", bc="reflective")
    with pytest.raises(alsv.AlsvError, match="reflective"):
        alsv.alsv_init_grid(d, 0)
    d = alsv.make_desc(ndim=2, n=(0, 4))
    with pytest.raises(alsv.AlsvError, match="n >= 1"):
        alsv.alsv_init_grid(d, 0)
    d = alsv.make_desc(ndim=1, n=(8,))
    d.reserved[3] = 1
    with pytest.raises(alsv.AlsvError, match="reserved"):
        alsv.alsv_init_grid(d, 0)
    # tiny and ragged grids are valid
    for n in (1, 2, 3, 7, 257):
        ctx, _ = alsv.alsv_init_grid(alsv.make_desc(ndim=1, n=(n,), recon="pc", bc="periodic"), 0)
        alsv.alsv_destroy(ctx)


def test_calls_before_binding_report_not_ready(alsv):
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(ndim=1, n=(8,)), 0)
    try:
        with pytest.raises(alsv.AlsvError) as ei:
            alsv.alsv_step(ctx, 1)
        assert ei.value.status_name == "ERR_NOT_READY"
        with pytest.raises(alsv.AlsvError) as ei:
            alsv.alsv_bind_workspace(ctx, 0x1000, 16)
        assert ei.value.status_name == "ERR_BUFFER_TOO_SMALL"
        with pytest.raises(alsv.AlsvError, match="aligned"):
            alsv.alsv_bind_workspace(ctx, 0x1001, 1 << 30)
    finally:
        alsv.alsv_destroy(ctx)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1912_07645_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "alsv_oracle" not in src, f


def test_adjoint_validation_without_gpu(alsv):
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(ndim=2, n=(16, 16), recon="weno3", flux="hllc"), 0)
    try:
        with pytest.raises(alsv.AlsvError, match="Rusanov"):
            alsv.alsv_adjoint_workspace_bytes(ctx, 0.1)
    finally:
        alsv.alsv_destroy(ctx)
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(ndim=2, n=(512, 512), batch=64, recon="mc", flux="rusanov",
                                                rk="ssprk2", precision="fp64", cfl=0.4), 0)
    try:
        b = alsv.alsv_adjoint_workspace_bytes(ctx, 1.0)
        state = 64 * 4 * 512 * 512 * 8
        # n = 3035 steps, allowance n_cap = ceil(1.5 n) = 4553, segments of ceil(sqrt(n_cap)) = 68
        # steps: 67 checkpoints + 67 segment states + 3 adjoint buffers
        assert b >= (67 + 67 + 3) * state and b < (67 + 67 + 3) * state + (1 << 24)
        with pytest.raises(alsv.AlsvError, match="no completed adjoint call"):
            alsv.alsv_adjoint_get_plan(ctx)
    finally:
        alsv.alsv_destroy(ctx)


def test_provenance_record(alsv, tmp_path):
    import json
    d = alsv.make_desc(ndim=2, n=(32, 16), batch=3, seed=77)
    rec = alsv.provenance(d, initial_data="kh")
    assert rec["library"].startswith("alsv") and rec["descriptor"]["n"][:2] == [32, 16]
    assert rec["descriptor"]["seed"] == 77 and rec["initial_data"] == "kh"
    p = alsv.save_result(str(tmp_path / "r"), {"x": [1.0, 2.0]}, d, note="test")
    assert json.load(open(p))["note"] == "test"


def test_fast_division_formula():
    """The work-item decomposition divides by runtime constants with the Granlund-Montgomery
    multiply-high form n / d = (umulhi(n, m) + n) >> l, l = ceil(log2 d),
    m = floor(2^32 (2^l - d) / d) + 1, valid for 0 <= n < 2^31; checked here exhaustively on
    edge cases and randomly elsewhere."""
    import random
    rnd = random.Random(1)

    def mk(d):
        l = 0
        while (1 << l) < d:
            l += 1
        return ((1 << 32) * ((1 << l) - d)) // d + 1, l

    ds = list(range(1, 600)) + [rnd.randrange(1, 2**31) for _ in range(3000)] + [2**k for k in range(31)] + \
        [2**k - 1 for k in range(1, 31)] + [2**k + 1 for k in range(1, 30)]
    for d in ds:
        m, l = mk(d)
        assert m < 2**32
        ns = [0, 1, d - 1, d, d + 1, 2**31 - 1] + [rnd.randrange(0, 2**31) for _ in range(20)]
        for n in ns:
            if 0 <= n < 2**31:
                assert ((((n * m) >> 32) + n) >> l) == n // d


def test_mlmc_coupling_validation(alsv):
    base = dict(ndim=2, recon="mc", flux="hllc", precision="fp64")
    good = [((16, 8), 6), ((32, 16), 4), ((16, 8), 4, 1)]
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(levels=good, **base), 0)
    try:
        # one 256-byte header, then per level 3 arrays of 4 quantities (256-byte aligned blocks)
        assert alsv.alsv_mlmc_bytes(ctx) == 256 + 3 * 4 * 128 * 8 + 3 * 4 * 512 * 8
    finally:
        alsv.alsv_destroy(ctx)
    bad = {
        "batch": [((16, 8), 6), ((32, 16), 4), ((16, 8), 3, 1)],
        "divide": [((16, 8), 6), ((32, 16), 4), ((12, 8), 4, 1)],
        "level": [((16, 8), 6), ((32, 16), 4, 0), ((16, 8), 4, 1)],
        "one companion": [((32, 16), 4), ((16, 8), 4, 0), ((16, 8), 4, 0)],
        "another group": [((32, 16), 4), ((16, 8), 4, 1)],
    }
    for what, levels in bad.items():
        with pytest.raises(alsv.AlsvError, match="level_fine"):
            alsv.alsv_init_grid(alsv.make_desc(levels=levels, **base), 0)
    d = alsv.make_desc(n=(16, 8), **base)
    d.level_fine[0] = 1
    with pytest.raises(alsv.AlsvError, match="level_fine"):
        alsv.alsv_init_grid(d, 0)
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(n=(16, 8), **base), 0)
    try:
        assert alsv.alsv_mlmc_bytes(ctx) == 0
    finally:
        alsv.alsv_destroy(ctx)


def test_size_limits_and_sampler_validation(alsv):
    # the largest batch a context holds, one past it, and a sample of 2^31 or more elements
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(ndim=1, n=(4,), batch=65535, recon="pc"), 0)
    alsv.alsv_destroy(ctx)
    with pytest.raises(alsv.AlsvError, match="65535"):
        alsv.alsv_init_grid(alsv.make_desc(ndim=1, n=(4,), batch=65536, recon="pc"), 0)
    with pytest.raises(alsv.AlsvError, match="2\\^31"):
        alsv.alsv_init_grid(alsv.make_desc(ndim=3, n=(1024, 1024, 1024), precision="fp32"), 0)
    d = alsv.make_desc(ndim=2, n=(8, 8))
    d.sampler = 3
    with pytest.raises(alsv.AlsvError, match="sampler"):
        alsv.alsv_init_grid(d, 0)
    with pytest.raises(alsv.AlsvError, match="Halton"):
        alsv.alsv_init_grid(alsv.make_desc(ndim=2, n=(8, 8), batch=4, sampler="halton",
                                           sample_offset=(1 << 31) - 2), 0)
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(ndim=2, n=(8, 8), batch=4, sampler="halton_shifted",
                                                sample_offset=(1 << 31) - 5), 0)
    alsv.alsv_destroy(ctx)


def test_statistics_calls_without_a_state_report_not_ready(alsv):
    import torch
    ctx, _ = alsv.alsv_init_grid(alsv.make_desc(ndim=2, n=(16, 16), batch=2), 0)
    buf = torch.zeros(1 << 16, dtype=torch.uint8)   # never touched: the calls fail first
    try:
        for call in (lambda: alsv.alsv_structure_function_accumulate(ctx, 0, 1, 2, buf),
                     lambda: alsv.alsv_mlmc_accumulate(ctx, buf)):
            with pytest.raises(alsv.AlsvError) as ei:
                call()
            assert ei.value.status_name in ("ERR_NOT_READY", "ERR_INVALID_ARG")
    finally:
        alsv.alsv_destroy(ctx)


def test_python_name_maps_match_the_header_enums():
    """Every name the binding maps to an integer (equation, reconstruction, variables, flux, RK
    order, boundary, precision, initial data, observable, sampler, stage part) has the value of the
    header's enum constant of that name."""
    from paper_1912_07645_gb300 import _abi
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "alsv.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(ALSV_[A-Z0-9_]+)\s*=\s*(-?\d+)", hdr)}
    groups = [(_abi.EQ, "ALSV_EQ_"), (_abi.RECON, "ALSV_RECON_"), (_abi.RVARS, "ALSV_VARS_"), (_abi.FLUX, "ALSV_FLUX_"),
              (_abi.BC, "ALSV_BC_"), (_abi.SAMPLER, "ALSV_SAMPLER_"), (_abi.PART, "ALSV_PART_")]
    for table, prefix in groups:
        for name, value in table.items():
            assert consts[prefix + name.upper()] == value, (prefix, name)
    assert {"ssprk2": consts["ALSV_RK_SSP2"], "ssprk3": consts["ALSV_RK_SSP3"]} == _abi.RK
    assert {"fp32": consts["ALSV_FP32"], "fp64": consts["ALSV_FP64"]} == _abi.PRECISION
    assert {"ke": consts["ALSV_OBS_KINETIC_ENERGY"], "mixing": consts["ALSV_OBS_MIXING_WIDTH"]} == _abi.OBSERVABLE
    for name, value in _abi.INIT.items():
        assert consts["ALSV_INIT_" + name.upper()] == value, name
    # every header flux and reconstruction has a name in the binding (and the oracle)
    for prefix, table in (("ALSV_FLUX_", _abi.FLUX), ("ALSV_RECON_", _abi.RECON)):
        assert sorted(v for k, v in consts.items() if k.startswith(prefix)) == sorted(table.values()), prefix
    import oracle
    assert oracle.FLUX == _abi.FLUX and oracle.RECON == _abi.RECON
