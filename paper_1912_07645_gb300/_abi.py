"""ctypes declarations of the C ABI in include/alsv.h and thin wrappers with the same names.

Argument marshalling only: every step of the method runs in libalsv.so's CUDA kernels. A missing
or unloadable library raises at import of the first call; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libalsv.so")

OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID_ARG", 2: "ERR_CUDA", 3: "ERR_NONPHYSICAL", 4: "ERR_CFL",
                5: "ERR_TIMEOUT", 6: "ERR_BUFFER_TOO_SMALL", 7: "ERR_NOT_READY"}
EQ = {"burgers": 0, "euler": 1}
RECON = {"pc": 0, "mc": 1, "weno3": 2, "eno2": 3}
RVARS = {"cons": 0, "prim": 1}
FLUX = {"rusanov": 0, "hll": 1, "hllc": 2, "roe": 3, "godunov": 4, "ec": 5, "ec4": 6, "tecno2": 7}
RK = {"ssprk2": 2, "ssprk3": 3}
BC = {"periodic": 0, "outflow": 1, "reflective": 2, "halo": 3}
PRECISION = {"fp32": 0, "fp64": 1}
INIT = {"kh": 0, "sod": 1, "lax": 2, "burgers_sine": 3, "vortex": 4, "raw": 5}
OBSERVABLE = {"ke": 0, "mixing": 1}
MAX_LEVELS = 8


class AlsvError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.status_name}: {message}")


SAMPLER = {"mc": 0, "halton": 1, "halton_shifted": 2}


class alsv_grid_desc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("batch", C.c_int32), ("eq", C.c_int32), ("gamma", C.c_double), ("recon", C.c_int32),
        ("recon_vars", C.c_int32), ("flux", C.c_int32), ("rk", C.c_int32), ("bc", (C.c_int32 * 2) * 3),
        ("cfl", C.c_double), ("fixed_dt", C.c_double), ("precision", C.c_int32), ("seed", C.c_uint64),
        ("weno_eps", C.c_double), ("weno_eps_dx2", C.c_int32), ("n_levels", C.c_int32),
        ("level_n", (C.c_int32 * 3) * MAX_LEVELS), ("level_batch", C.c_int32 * MAX_LEVELS),
        ("vortex_center", C.c_double * 2), ("sample_offset", C.c_int64),
        ("level_fine", C.c_int32 * MAX_LEVELS), ("sampler", C.c_int32), ("global_n", C.c_int32 * 3),
        ("offset", C.c_int32 * 3), ("reserved", C.c_int32 * 4),
    ]


# name -> (restype, argtypes)
_vp, _sz, _i64p, _dp = C.c_void_p, C.c_size_t, C.POINTER(C.c_int64), C.POINTER(C.c_double)
_ctx = C.c_void_p
SIGNATURES = {
    "alsv_version": (C.c_char_p, []),
    "alsv_last_error": (C.c_char_p, [_ctx]),
    "alsv_init_grid": (C.c_int, [C.POINTER(alsv_grid_desc), _vp, C.POINTER(_ctx), C.POINTER(_sz)]),
    "alsv_bind_workspace": (C.c_int, [_ctx, _vp, _sz]),
    "alsv_state_bytes": (_sz, [_ctx]),
    "alsv_get_parameters": (C.c_int, [_ctx, _vp]),
    "alsv_num_samples": (C.c_int32, [_ctx]),
    "alsv_num_vars": (C.c_int32, [_ctx]),
    "alsv_set_initial_data": (C.c_int, [_ctx, C.c_int, _vp, C.c_int, _vp, _sz]),
    "alsv_step": (C.c_int, [_ctx, C.c_int]),
    "alsv_evolve_to_T": (C.c_int, [_ctx, C.c_double, _i64p]),
    "alsv_evolve_resident": (C.c_int, [_ctx, C.c_double, _i64p]),
    "alsv_sync": (C.c_int, [_ctx]),
    "alsv_set_time": (C.c_int, [_ctx, _dp, _i64p]),
    "alsv_get_time": (C.c_int, [_ctx, _dp, _i64p]),
    "alsv_stats_bytes": (_sz, [_ctx]),
    "alsv_stats_reset": (C.c_int, [_ctx, _vp, _sz]),
    "alsv_stats_accumulate": (C.c_int, [_ctx, _vp, _sz]),
    "alsv_stats_read": (C.c_int, [_ctx, _vp, _vp, _vp, _i64p]),
    "alsv_stats_merge": (C.c_int, [_ctx, _vp, _vp, _sz]),
    "alsv_conservation_totals": (C.c_int, [_ctx, _vp]),
    "alsv_point_pdf_accumulate": (C.c_int, [_ctx, C.c_int, _vp, C.c_int, C.c_double, C.c_double, C.c_int, _vp]),
    "alsv_joint_pdf_accumulate": (C.c_int, [_ctx, C.c_int, C.c_int, _vp, C.c_int, C.c_double, C.c_double, C.c_int,
                                            C.c_double, C.c_double, C.c_int, _vp]),
    "alsv_correlator_accumulate": (C.c_int, [_ctx, C.c_int, _vp, C.c_int, C.c_int, _vp]),
    "alsv_structure_function_bytes": (_sz, [_ctx, C.c_int]),
    "alsv_structure_function_accumulate": (C.c_int, [_ctx, C.c_int, C.c_int, C.c_int, _vp, _sz]),
    "alsv_structure_function_read": (C.c_int, [_ctx, _vp, C.c_int, C.c_int, _vp]),
    "alsv_mlmc_bytes": (_sz, [_ctx]),
    "alsv_mlmc_reset": (C.c_int, [_ctx, _vp, _sz]),
    "alsv_mlmc_accumulate": (C.c_int, [_ctx, _vp, _sz]),
    "alsv_mlmc_read": (C.c_int, [_ctx, _vp, _sz, _vp, _vp, _vp, _i64p]),
    "alsv_kinetic_energy": (C.c_int, [_ctx, _vp]),
    "alsv_mixing_width": (C.c_int, [_ctx, _vp]),
    "alsv_conservation_totals_noalloc": (C.c_int, [C.POINTER(alsv_grid_desc), _vp, _sz, _vp, _vp]),
    "alsv_adjoint_workspace_bytes": (C.c_int, [_ctx, C.c_double, C.POINTER(_sz)]),
    "alsv_bind_adjoint_workspace": (C.c_int, [_ctx, _vp, _sz]),
    "alsv_adjoint_evolve": (C.c_int, [_ctx, C.c_double, C.c_int, _vp, _vp, _vp]),
    "alsv_adjoint_get_plan": (C.c_int, [_ctx, _i64p, _dp, C.POINTER(C.c_int32)]),
    "alsv_destroy": (C.c_int, [_ctx]),
    "alsv_num_tile_variants": (C.c_int, [_ctx]),
    "alsv_set_tile_variant": (C.c_int, [_ctx, C.c_int]),
    "alsv_get_tile": (C.c_int, [_ctx, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int), _i64p]),
    "alsv_autotune": (C.c_int, [_ctx, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "alsv_set_graphs": (C.c_int, [_ctx, C.c_int]),
    "alsv_set_profiling": (C.c_int, [_ctx, C.c_int]),
    "alsv_get_profile": (C.c_int, [_ctx, _dp, _i64p, _dp, _i64p]),
    "alsv_get_launch_count": (C.c_int, [_ctx, _i64p]),
    "alsv_halo_info": (C.c_int, [_ctx, C.POINTER(C.c_int32), _i64p]),
    "alsv_bind_halo": (C.c_int, [_ctx, C.POINTER(_vp), C.POINTER(_sz)]),
    "alsv_halo_pack": (C.c_int, [_ctx, C.c_int, C.POINTER(_vp), C.POINTER(_sz)]),
    "alsv_stage": (C.c_int, [_ctx, C.c_int]),
    "alsv_speed_max": (C.c_int, [_ctx, _vp]),
    "alsv_speed_max_combine": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, _vp, _vp]),
    "alsv_stage_part": (C.c_int, [_ctx, C.c_int, C.c_int]),
    "alsv_finish_step": (C.c_int, [_ctx, _vp, C.c_int]),
    "alsv_set_end_time": (C.c_int, [_ctx, C.c_double]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libalsv.so (building it first is the caller's job: paper_1912_07645_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libalsv.so not found at {p}: run paper_1912_07645_gb300.build.build() "
                                   "(the CUDA library is required; there is no CPU fallback)")
            lib = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st: int, where: str, ctx=None):
    if st != OK:
        msg = load().alsv_last_error(ctx)
        raise AlsvError(st, where, msg.decode() if msg else "")


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _nbytes(x) -> int:
    return x.numel() * x.element_size()


# ---------------------------------------------------------------- wrappers (same names as the C ABI)
def alsv_version() -> str:
    return load().alsv_version().decode()


def alsv_last_error(ctx) -> str:
    m = load().alsv_last_error(ctx)
    return m.decode() if m else ""


def alsv_init_grid(desc: alsv_grid_desc, stream: int = 0):
    """Returns (ctx, workspace_bytes)."""
    ctx = C.c_void_p()
    ws = C.c_size_t()
    _check(load().alsv_init_grid(C.byref(desc), C.c_void_p(stream or None), C.byref(ctx), C.byref(ws)),
           "alsv_init_grid", None)
    return ctx.value, ws.value


def alsv_bind_workspace(ctx, ws, nbytes: int | None = None):
    _check(load().alsv_bind_workspace(ctx, _ptr(ws), nbytes if nbytes is not None else _nbytes(ws)),
           "alsv_bind_workspace", ctx)


def alsv_state_bytes(ctx) -> int:
    return int(load().alsv_state_bytes(ctx))


def alsv_get_parameters(ctx, theta):
    _check(load().alsv_get_parameters(ctx, _ptr(theta)), "alsv_get_parameters", ctx)


def alsv_num_samples(ctx) -> int:
    return int(load().alsv_num_samples(ctx))


def alsv_num_vars(ctx) -> int:
    return int(load().alsv_num_vars(ctx))


def alsv_set_initial_data(ctx, kind, theta, n_params: int, U, U_bytes: int | None = None):
    k = INIT[kind] if isinstance(kind, str) else int(kind)
    _check(load().alsv_set_initial_data(ctx, k, _ptr(theta), n_params, _ptr(U),
                                        U_bytes if U_bytes is not None else _nbytes(U)),
           "alsv_set_initial_data", ctx)


def alsv_step(ctx, n_steps: int):
    _check(load().alsv_step(ctx, n_steps), "alsv_step", ctx)


def alsv_evolve_to_T(ctx, T: float) -> int:
    steps = C.c_int64()
    _check(load().alsv_evolve_to_T(ctx, T, C.byref(steps)), "alsv_evolve_to_T", ctx)
    return steps.value


def alsv_set_time(ctx, t, steps=None):
    """t, steps: host sequences of alsv_num_samples entries."""
    import numpy as np
    tt = np.ascontiguousarray(t, dtype=np.float64)
    ss = None if steps is None else np.ascontiguousarray(steps, dtype=np.int64)
    _check(load().alsv_set_time(ctx, tt.ctypes.data_as(_dp), None if ss is None else ss.ctypes.data_as(_i64p)),
           "alsv_set_time", ctx)


def alsv_sync(ctx):
    _check(load().alsv_sync(ctx), "alsv_sync", ctx)


def alsv_get_time(ctx):
    import numpy as np
    n = alsv_num_samples(ctx)
    t = np.zeros(n)
    s = np.zeros(n, dtype=np.int64)
    _check(load().alsv_get_time(ctx, t.ctypes.data_as(_dp), s.ctypes.data_as(_i64p)), "alsv_get_time", ctx)
    return t, s


def alsv_stats_bytes(ctx) -> int:
    return int(load().alsv_stats_bytes(ctx))


def alsv_stats_reset(ctx, stats):
    _check(load().alsv_stats_reset(ctx, _ptr(stats), _nbytes(stats)), "alsv_stats_reset", ctx)


def alsv_stats_accumulate(ctx, stats):
    _check(load().alsv_stats_accumulate(ctx, _ptr(stats), _nbytes(stats)), "alsv_stats_accumulate", ctx)


def alsv_stats_read(ctx, stats, mean=None, var=None) -> int:
    cnt = C.c_int64()
    _check(load().alsv_stats_read(ctx, _ptr(stats), _ptr(mean), _ptr(var), C.byref(cnt)), "alsv_stats_read", ctx)
    return cnt.value


def alsv_stats_merge(ctx, stats, other):
    _check(load().alsv_stats_merge(ctx, _ptr(stats), _ptr(other), _nbytes(stats)), "alsv_stats_merge", ctx)


def alsv_point_pdf_accumulate(ctx, quantity: int, cells, lo: float, hi: float, n_bins: int, counts):
    _check(load().alsv_point_pdf_accumulate(ctx, quantity, _ptr(cells), int(cells.numel()), lo, hi, n_bins,
                                            _ptr(counts)), "alsv_point_pdf_accumulate", ctx)


def alsv_joint_pdf_accumulate(ctx, q1: int, q2: int, cells, lo1: float, hi1: float, n_bins1: int, lo2: float,
                              hi2: float, n_bins2: int, counts):
    _check(load().alsv_joint_pdf_accumulate(ctx, q1, q2, _ptr(cells), int(cells.numel()), lo1, hi1, n_bins1, lo2, hi2,
                                            n_bins2, _ptr(counts)), "alsv_joint_pdf_accumulate", ctx)


def alsv_correlator_accumulate(ctx, quantity: int, cells, acc):
    """cells: int64 [n_sets, k] device tensor; acc: FP64 [1 + n_sets]."""
    n_sets, k = int(cells.shape[0]), int(cells.shape[1])
    _check(load().alsv_correlator_accumulate(ctx, quantity, _ptr(cells), n_sets, k, _ptr(acc)),
           "alsv_correlator_accumulate", ctx)


def alsv_structure_function_bytes(ctx, radius: int) -> int:
    return int(load().alsv_structure_function_bytes(ctx, radius))


def alsv_structure_function_accumulate(ctx, quantity: int, p: int, radius: int, acc):
    _check(load().alsv_structure_function_accumulate(ctx, quantity, p, radius, _ptr(acc), _nbytes(acc)),
           "alsv_structure_function_accumulate", ctx)


def alsv_structure_function_read(ctx, acc, p: int, radius: int, S):
    _check(load().alsv_structure_function_read(ctx, _ptr(acc), p, radius, _ptr(S)), "alsv_structure_function_read", ctx)


def alsv_mlmc_bytes(ctx) -> int:
    return int(load().alsv_mlmc_bytes(ctx))


def alsv_mlmc_reset(ctx, acc):
    _check(load().alsv_mlmc_reset(ctx, _ptr(acc), _nbytes(acc)), "alsv_mlmc_reset", ctx)


def alsv_mlmc_accumulate(ctx, acc):
    _check(load().alsv_mlmc_accumulate(ctx, _ptr(acc), _nbytes(acc)), "alsv_mlmc_accumulate", ctx)


def alsv_mlmc_read(ctx, acc, mean=None, var=None, level=None, n_levels: int = 0):
    """Writes the estimate (and per-level sums) to the device buffers given; returns the per-level
    sample counts when n_levels > 0 (synchronises the stream)."""
    cnt = (C.c_int64 * max(n_levels, 1))()
    _check(load().alsv_mlmc_read(ctx, _ptr(acc), _nbytes(acc), _ptr(mean), _ptr(var), _ptr(level),
                                 cnt if n_levels > 0 else None), "alsv_mlmc_read", ctx)
    return [int(v) for v in cnt][:n_levels]


def alsv_conservation_totals(ctx, totals):
    _check(load().alsv_conservation_totals(ctx, _ptr(totals)), "alsv_conservation_totals", ctx)


def alsv_conservation_totals_noalloc(desc: alsv_grid_desc, U, totals, stream: int = 0):
    """Totals without a context or workspace (static device scratch); see include/alsv.h."""
    _check(load().alsv_conservation_totals_noalloc(C.byref(desc), _ptr(U), _nbytes(U), _ptr(totals),
                                                   C.c_void_p(stream or None)),
           "alsv_conservation_totals_noalloc", None)


def alsv_kinetic_energy(ctx, ke):
    _check(load().alsv_kinetic_energy(ctx, _ptr(ke)), "alsv_kinetic_energy", ctx)


def alsv_mixing_width(ctx, w):
    _check(load().alsv_mixing_width(ctx, _ptr(w)), "alsv_mixing_width", ctx)


def alsv_adjoint_workspace_bytes(ctx, T: float) -> int:
    b = C.c_size_t()
    _check(load().alsv_adjoint_workspace_bytes(ctx, T, C.byref(b)), "alsv_adjoint_workspace_bytes", ctx)
    return b.value


def alsv_bind_adjoint_workspace(ctx, ws, nbytes: int | None = None):
    _check(load().alsv_bind_adjoint_workspace(ctx, _ptr(ws), nbytes if nbytes is not None else _nbytes(ws)),
           "alsv_bind_adjoint_workspace", ctx)


def alsv_adjoint_evolve(ctx, T: float, observable, theta, grad_theta, J):
    """observable: ALSV_OBS_* (int) or a name of OBSERVABLE ("ke", "mixing")."""
    observable = OBSERVABLE[observable] if isinstance(observable, str) else int(observable)
    _check(load().alsv_adjoint_evolve(ctx, T, observable, _ptr(theta), _ptr(grad_theta), _ptr(J)),
           "alsv_adjoint_evolve", ctx)


def alsv_adjoint_get_plan(ctx):
    """(n_steps, dt, forward passes) of the last successful alsv_adjoint_evolve."""
    n, dt, p = C.c_int64(0), C.c_double(0.0), C.c_int32(0)
    _check(load().alsv_adjoint_get_plan(ctx, C.byref(n), C.byref(dt), C.byref(p)), "alsv_adjoint_get_plan", ctx)
    return int(n.value), float(dt.value), int(p.value)


def alsv_halo_info(ctx):
    """(ghost layers g, [elements of the halo buffer of face 2k + side] * 6)."""
    g, n = C.c_int32(0), (C.c_int64 * 6)()
    _check(load().alsv_halo_info(ctx, C.byref(g), n), "alsv_halo_info", ctx)
    return int(g.value), [int(v) for v in n]


def _faces(bufs):
    arr = (C.c_void_p * 6)()
    for f in range(6):
        arr[f] = _ptr(bufs[f]) if f < len(bufs) else None
    return arr


def _sizes(bufs, nbytes=None):
    arr = (C.c_size_t * 6)()
    for f in range(6):
        b = bufs[f] if f < len(bufs) else None
        if nbytes is not None:
            arr[f] = int(nbytes[f])
        elif b is not None and not isinstance(b, int):
            arr[f] = _nbytes(b)
    return arr


def alsv_bind_halo(ctx, halos, nbytes=None):
    """halos: six device buffers (None for faces that are not HALO), face 2k + side; nbytes: their
    byte sizes (default: the tensors' sizes)."""
    _check(load().alsv_bind_halo(ctx, _faces(halos), _sizes(halos, nbytes)), "alsv_bind_halo", ctx)


def alsv_halo_pack(ctx, stage: int, sends, nbytes=None):
    """sends: six device buffers (None to skip a face) that receive the block's boundary layers."""
    _check(load().alsv_halo_pack(ctx, stage, _faces(sends), _sizes(sends, nbytes)), "alsv_halo_pack", ctx)


def alsv_stage(ctx, stage: int):
    _check(load().alsv_stage(ctx, stage), "alsv_stage", ctx)


PART = {"interior": 1, "boundary": 2}


def alsv_stage_part(ctx, stage: int, part: str):
    """One part of stage s (interior tiles, or the tiles that read halo buffers); see include/alsv.h."""
    _check(load().alsv_stage_part(ctx, stage, PART[part]), "alsv_stage_part", ctx)


def alsv_evolve_resident(ctx, T: float) -> int:
    """Evolve to T with every sample resident in one thread-block cluster; see include/alsv.h."""
    n = C.c_int64(0)
    _check(load().alsv_evolve_resident(ctx, T, C.byref(n)), "alsv_evolve_resident", ctx)
    return int(n.value)


def alsv_speed_max(ctx, smax):
    _check(load().alsv_speed_max(ctx, _ptr(smax)), "alsv_speed_max", ctx)


def alsv_speed_max_combine(smax_list, out, stream: int = 0):
    """out[s] = max over the blocks' device FP64 vectors smax_list[i][s] (NaN-propagating), on
    stream; see include/alsv.h."""
    n = len(smax_list)
    arr = (_vp * max(n, 1))(*[_ptr(x) for x in smax_list])
    samples = int(out.numel()) if hasattr(out, "numel") else 0
    _check(load().alsv_speed_max_combine(arr, n, samples, _ptr(out), C.c_void_p(stream or None)),
           "alsv_speed_max_combine", None)


def alsv_finish_step(ctx, smax, advance: bool):
    _check(load().alsv_finish_step(ctx, _ptr(smax), 1 if advance else 0), "alsv_finish_step", ctx)


def alsv_set_end_time(ctx, T: float):
    _check(load().alsv_set_end_time(ctx, T), "alsv_set_end_time", ctx)


def alsv_destroy(ctx):
    if ctx:
        load().alsv_destroy(ctx)


def alsv_num_tile_variants(ctx) -> int:
    return int(load().alsv_num_tile_variants(ctx))


def alsv_set_tile_variant(ctx, v: int):
    _check(load().alsv_set_tile_variant(ctx, v), "alsv_set_tile_variant", ctx)


def alsv_get_tile(ctx):
    tx, ty, tz, v = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    w = C.c_int64()
    _check(load().alsv_get_tile(ctx, C.byref(tx), C.byref(ty), C.byref(tz), C.byref(v), C.byref(w)),
           "alsv_get_tile", ctx)
    return (tx.value, ty.value, tz.value), v.value, w.value


def alsv_autotune(ctx, reps: int = 3):
    n = alsv_num_tile_variants(ctx)
    ms = (C.c_float * max(n, 1))()
    ch = C.c_int()
    _check(load().alsv_autotune(ctx, reps, C.byref(ch), ms), "alsv_autotune", ctx)
    return ch.value, [ms[i] for i in range(n)]


def alsv_set_graphs(ctx, on: bool):
    _check(load().alsv_set_graphs(ctx, 1 if on else 0), "alsv_set_graphs", ctx)


def alsv_set_profiling(ctx, on: bool):
    _check(load().alsv_set_profiling(ctx, 1 if on else 0), "alsv_set_profiling", ctx)


def alsv_get_profile(ctx):
    sm, fm = C.c_double(), C.c_double()
    sl, fl = C.c_int64(), C.c_int64()
    _check(load().alsv_get_profile(ctx, C.byref(sm), C.byref(sl), C.byref(fm), C.byref(fl)), "alsv_get_profile", ctx)
    return {"stage_ms": sm.value, "stage_launches": sl.value, "finish_ms": fm.value, "finish_launches": fl.value}


def alsv_get_launch_count(ctx) -> int:
    n = C.c_int64()
    _check(load().alsv_get_launch_count(ctx, C.byref(n)), "alsv_get_launch_count", ctx)
    return n.value
