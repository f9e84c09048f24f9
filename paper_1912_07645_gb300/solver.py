"""Descriptor construction and a context wrapper that owns torch-allocated device buffers.

The wrapper only allocates memory and forwards to the C ABI; it performs no arithmetic.
"""
from __future__ import annotations

from . import _abi as A


def make_desc(ndim=1, n=(8, 1, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), batch=1, eq="euler", gamma=1.4,
              recon="mc", rvars="prim", flux="hllc", rk="ssprk2", bc="periodic", cfl=0.45, fixed_dt=0.0,
              precision="fp64", seed=0, weno_eps=1e-6, weno_eps_dx2=False, levels=None,
              vortex_center=(5.0, 5.0), sample_offset=0, sampler="mc", global_n=None, offset=None,
              **_ignored) -> A.alsv_grid_desc:
    """Build an ``alsv_grid_desc`` from plain values.

    ``bc``: one name for every side or a list of (lo, hi) names per direction.
    ``levels``: optional level table, a list of (n_tuple, samples) or (n_tuple, samples, fine):
    ``fine`` = index of the table entry this group is the MLMC coarse companion of (same samples
    and KH parameters on a coarser grid).
    ``global_n`` / ``offset``: a block of a decomposed grid (whole grid's cells per direction, the
    block's first cell); ``bc`` may then name "halo" faces (see ``decomp``).
    """
    d = A.alsv_grid_desc()
    d.ndim = ndim
    nn = list(n) + [1] * (3 - len(n))
    for k in range(3):
        d.n[k] = int(nn[k]) if k < ndim else 1
        d.lo[k] = float(lo[k]) if k < len(lo) else 0.0
        d.hi[k] = float(hi[k]) if k < len(hi) else 1.0
    d.batch = batch
    d.eq = A.EQ[eq]
    d.gamma = gamma
    d.recon = A.RECON[recon]
    d.recon_vars = A.RVARS[rvars]
    d.flux = A.FLUX[flux]
    d.rk = A.RK[rk]
    for k in range(3):
        pair = (bc, bc) if isinstance(bc, str) else (bc[k] if k < len(bc) else ("periodic", "periodic"))
        d.bc[k][0] = A.BC[pair[0]]
        d.bc[k][1] = A.BC[pair[1]]
    d.cfl = cfl
    d.fixed_dt = fixed_dt
    d.precision = A.PRECISION[precision]
    d.seed = seed & 0xFFFFFFFFFFFFFFFF
    d.weno_eps = weno_eps
    d.weno_eps_dx2 = 1 if weno_eps_dx2 else 0
    if levels:
        d.n_levels = len(levels)
        for l, entry in enumerate(levels):
            ln, lb = entry[0], entry[1]
            ln = list(ln) + [1] * (3 - len(ln))
            for k in range(3):
                d.level_n[l][k] = int(ln[k]) if k < ndim else 1
            d.level_batch[l] = lb
            d.level_fine[l] = int(entry[2]) + 1 if len(entry) > 2 and entry[2] is not None else 0
    d.vortex_center[0], d.vortex_center[1] = vortex_center
    d.sample_offset = int(sample_offset)
    d.sampler = A.SAMPLER[sampler]
    if global_n is not None:
        for k, v in enumerate(global_n):
            d.global_n[k] = int(v) if k < ndim else 0
    if offset is not None:
        for k, v in enumerate(offset):
            d.offset[k] = int(v) if k < ndim else 0
    return d


class Solver:
    """One context with its workspace and state held as torch CUDA tensors.

    ``stream``: a torch.cuda.Stream (default: a new stream, so step chunks can be captured in CUDA
    graphs). All calls enqueue work on that stream; tensors returned by the methods are written on
    it, so synchronise (``sync()``) before reading them from another stream or the host.
    """

    def __init__(self, desc: A.alsv_grid_desc | None = None, stream=None, device="cuda", **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the solver has no CPU path)")
        self.torch = torch
        self.desc = desc if desc is not None else make_desc(**kw)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.ctx, ws_bytes = A.alsv_init_grid(self.desc, self.stream.cuda_stream)
        with torch.cuda.stream(self.stream):
            self.ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=self.device)
        A.alsv_bind_workspace(self.ctx, self.ws)
        self.nv = A.alsv_num_vars(self.ctx)
        self.samples = A.alsv_num_samples(self.ctx)
        self.dtype = torch.float64 if self.desc.precision == 1 else torch.float32
        nbytes = A.alsv_state_bytes(self.ctx)
        with torch.cuda.stream(self.stream):
            self.U = torch.empty(nbytes // (8 if self.desc.precision == 1 else 4), dtype=self.dtype, device=self.device)
        self.stats = None
        self.adj_ws = None

    # ---- shapes
    def level_shape(self, level=0):
        d = self.desc
        if d.n_levels > 1:
            n = list(d.level_n[level])
            b = d.level_batch[level]
        else:
            n = list(d.n)
            b = d.batch
        return (b, self.nv, n[2], n[1], n[0])

    def state(self, level=0):
        """View of the state of one level as [B, nv, nz, ny, nx]."""
        off = 0
        for l in range(level):
            sh = self.level_shape(l)
            off += sh[0] * sh[1] * sh[2] * sh[3] * sh[4]
        sh = self.level_shape(level)
        cnt = sh[0] * sh[1] * sh[2] * sh[3] * sh[4]
        return self.U[off:off + cnt].view(sh)

    # ---- calls
    def set_initial_data(self, kind="kh", theta=None):
        n_params = 0 if theta is None else int(theta.shape[-1])
        A.alsv_set_initial_data(self.ctx, kind, theta, n_params, self.U)

    def set_state(self, U_host_or_dev):
        """Copy a full state into the bound buffer and initialise time (RAW initial data)."""
        src = U_host_or_dev.reshape(-1).to(device=self.device, dtype=self.dtype)
        with self.torch.cuda.stream(self.stream):
            self.U.copy_(src, non_blocking=False)
        A.alsv_set_initial_data(self.ctx, "raw", None, 0, self.U)

    def step(self, n=1):
        A.alsv_step(self.ctx, n)

    def evolve_to(self, T):
        return A.alsv_evolve_to_T(self.ctx, T)

    def evolve_resident(self, T):
        """evolve_to with every sample resident in one thread-block cluster (FP32 2D Euler)."""
        return A.alsv_evolve_resident(self.ctx, T)

    def sync(self):
        A.alsv_sync(self.ctx)

    def to_host(self, t):
        """Copy a tensor produced on this solver's stream to the host (waits for the stream)."""
        self.stream.synchronize()
        return t.detach().cpu()

    def time(self):
        return A.alsv_get_time(self.ctx)

    def stats_init(self):
        nb = A.alsv_stats_bytes(self.ctx)
        with self.torch.cuda.stream(self.stream):
            self.stats = self.torch.empty(nb, dtype=self.torch.uint8, device=self.device)
        A.alsv_stats_reset(self.ctx, self.stats)

    def stats_accumulate(self):
        if self.stats is None:
            self.stats_init()
        A.alsv_stats_accumulate(self.ctx, self.stats)

    def stats_read(self):
        b, nv, nz, ny, nx = self.level_shape(0)
        with self.torch.cuda.stream(self.stream):
            mean = self.torch.empty((nv, nz, ny, nx), dtype=self.torch.float64, device=self.device)
            var = self.torch.empty_like(mean)
        cnt = A.alsv_stats_read(self.ctx, self.stats, mean, var)
        return cnt, mean, var

    def mlmc_levels(self):
        """Table indices of the estimator's levels (groups that are not coarse companions)."""
        return [l for l in range(self.desc.n_levels) if self.desc.level_fine[l] == 0]

    def mlmc_init(self):
        nb = A.alsv_mlmc_bytes(self.ctx)
        with self.torch.cuda.stream(self.stream):
            self.mlmc_acc = self.torch.empty(nb, dtype=self.torch.uint8, device=self.device)
        A.alsv_mlmc_reset(self.ctx, self.mlmc_acc)

    def mlmc_accumulate(self):
        if getattr(self, "mlmc_acc", None) is None:
            self.mlmc_init()
        A.alsv_mlmc_accumulate(self.ctx, self.mlmc_acc)

    def mlmc_read(self):
        """(counts per level, mean [q, nz, ny, nx], variance, per-level sums [levels, q, 3]) on the
        finest level's grid; synchronous."""
        lv = self.mlmc_levels()
        fine = max(lv, key=lambda l: self.level_shape(l)[2] * self.level_shape(l)[3] * self.level_shape(l)[4])
        _, nv, nz, ny, nx = self.level_shape(fine)
        with self.torch.cuda.stream(self.stream):
            mean = self.torch.empty((nv, nz, ny, nx), dtype=self.torch.float64, device=self.device)
            var = self.torch.empty_like(mean)
            lev = self.torch.empty((len(lv), nv, 3), dtype=self.torch.float64, device=self.device)
        cnt = A.alsv_mlmc_read(self.ctx, self.mlmc_acc, mean, var, lev, n_levels=len(lv))
        return cnt, mean, var, lev

    def point_pdf(self, quantity, cells, lo, hi, n_bins, counts=None):
        """Add this batch to the counts (int64 [points, n_bins + 2], zeros when None) of the
        quantity's values at the given flat cell indices; returns the counts tensor."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            cells = torch.as_tensor(cells, dtype=torch.int64).to(self.device)
            if counts is None:
                counts = torch.zeros((cells.numel(), n_bins + 2), dtype=torch.int64, device=self.device)
        A.alsv_point_pdf_accumulate(self.ctx, quantity, cells, lo, hi, n_bins, counts)
        return counts

    def joint_pdf(self, q1, q2, cells, lo1, hi1, n_bins1, lo2, hi2, n_bins2, counts=None):
        """Add this batch to the joint counts (int64 [points, n_bins1 + 2, n_bins2 + 2])."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            cells = torch.as_tensor(cells, dtype=torch.int64).to(self.device)
            if counts is None:
                counts = torch.zeros((cells.numel(), n_bins1 + 2, n_bins2 + 2), dtype=torch.int64, device=self.device)
        A.alsv_joint_pdf_accumulate(self.ctx, q1, q2, cells, lo1, hi1, n_bins1, lo2, hi2, n_bins2, counts)
        return counts

    def correlator(self, quantity, cell_sets, acc=None):
        """Add this batch to acc (FP64 [1 + sets]: sample count, then sums of prod_j q(x_j))."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            cells = torch.as_tensor(cell_sets, dtype=torch.int64).to(self.device)
            if acc is None:
                acc = torch.zeros(1 + cells.shape[0], dtype=torch.float64, device=self.device)
        A.alsv_correlator_accumulate(self.ctx, quantity, cells, acc)
        return acc

    def structure_function(self, quantity, p, radius, acc=None):
        """Fold this batch into the accumulator (new when None) and return (acc, S_p(1..radius))."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            if acc is None:
                acc = torch.zeros(A.alsv_structure_function_bytes(self.ctx, radius), dtype=torch.uint8,
                                  device=self.device)
            S = torch.empty(radius, dtype=torch.float64, device=self.device)
        A.alsv_structure_function_accumulate(self.ctx, quantity, p, radius, acc)
        A.alsv_structure_function_read(self.ctx, acc, p, radius, S)
        return acc, S

    def totals(self):
        with self.torch.cuda.stream(self.stream):
            out = self.torch.empty((self.samples, self.nv), dtype=self.torch.float64, device=self.device)
        A.alsv_conservation_totals(self.ctx, out)
        return out

    def mixing_width(self):
        with self.torch.cuda.stream(self.stream):
            out = self.torch.empty(self.samples, dtype=self.torch.float64, device=self.device)
        A.alsv_mixing_width(self.ctx, out)
        return out

    def kinetic_energy(self):
        with self.torch.cuda.stream(self.stream):
            out = self.torch.empty(self.samples, dtype=self.torch.float64, device=self.device)
        A.alsv_kinetic_energy(self.ctx, out)
        return out

    def adjoint(self, theta, T, observable="ke"):
        """Observable J at T ("ke": kinetic energy, "mixing": mixing-layer width) and dJ/dtheta for
        every sample (theta: [samples, 20] FP64 on the device). Allocates the adjoint workspace on
        first use; synchronous."""
        torch = self.torch
        need = A.alsv_adjoint_workspace_bytes(self.ctx, T)
        if self.adj_ws is None or self.adj_ws.numel() < need:
            self.adj_ws = None
            with torch.cuda.stream(self.stream):
                self.adj_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        A.alsv_bind_adjoint_workspace(self.ctx, self.adj_ws)
        with torch.cuda.stream(self.stream):
            th = theta.to(device=self.device, dtype=torch.float64).contiguous()
            J = torch.empty(self.samples, dtype=torch.float64, device=self.device)
            g = torch.empty((self.samples, 20), dtype=torch.float64, device=self.device)
        A.alsv_adjoint_evolve(self.ctx, T, observable, th, g, J)
        return J, g

    # ---- block of a decomposed grid: the stage-by-stage protocol driven by decomp.Decomposition
    @property
    def stages(self):
        return 3 if self.desc.rk == 3 else 2

    def halo_info(self):
        """(ghost layers, element count of each face's halo buffer, 0 for faces that are not halo)."""
        return A.alsv_halo_info(self.ctx)

    def bind_halo(self):
        """Allocate and bind this block's halo buffers (one per halo face); returns them."""
        _, elems = self.halo_info()
        with self.torch.cuda.stream(self.stream):
            self.halos = [self.torch.zeros(n, dtype=self.dtype, device=self.device) if n else None for n in elems]
        if any(elems):
            A.alsv_bind_halo(self.ctx, self.halos)
        return self.halos

    def halo_pack(self, stage, sends):
        """Write the block's boundary layers of stage ``stage``'s input into ``sends`` (six device
        buffers or None, e.g. the neighbours' halo buffers)."""
        A.alsv_halo_pack(self.ctx, stage, sends)

    def stage(self, s):
        A.alsv_stage(self.ctx, s)

    def stage_part(self, s, part):
        A.alsv_stage_part(self.ctx, s, part)

    def speed_max(self, out):
        A.alsv_speed_max(self.ctx, out)

    def finish_step(self, smax, advance):
        A.alsv_finish_step(self.ctx, smax, advance)

    def set_end_time(self, T):
        A.alsv_set_end_time(self.ctx, T)

    def autotune(self, reps=3):
        return A.alsv_autotune(self.ctx, reps)

    def set_tile_variant(self, v):
        A.alsv_set_tile_variant(self.ctx, v)

    def close(self):
        if getattr(self, "ctx", None):
            A.alsv_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
