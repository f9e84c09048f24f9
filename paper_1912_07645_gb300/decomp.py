"""Spatial domain decomposition: one grid advanced as blocks with halo exchange (Sec. 2.1, last
paragraph; Sec. 3.1, where the paper splits a single sample over many GPUs in x, y or both).

The whole grid is cut into px x py x pz blocks of contiguous cells (``split``). Each block is a
context whose descriptor carries the whole grid's cell counts and the block's offset, so its dx
and every cell centre are the whole grid's bitwise, and whose faces that border another block are
halo faces: the stage kernels read the ghost cells there from halo buffers instead of a boundary
condition. A step then runs stage by stage:

  for every stage s:  each block writes the boundary layers of the state stage s reads into its
                      neighbours' halo buffers (the exchange), then runs stage s - across ranks
                      in two parts: the tiles whose stencil reads no halo buffer while the layers
                      travel, the others once they have arrived
  after the last:     the per-sample maximum wave speed is reduced over all blocks (MAX) and each
                      block finishes the step with it (t, dt, done flags)

so every cell sees exactly the inputs it has on the whole grid, and the blocks reproduce the
whole-grid run bitwise (the GPU tests check this against an undivided context).

Two transports carry the exchange and the maximum:
  ``LocalExchange``  every block in this process on one device, each on its own CUDA stream: a
                     block writes straight into its neighbours' halo buffers (no copies), CUDA
                     events order each pack after the neighbour's previous stage and each stage
                     after its neighbours' packs, so the blocks' launches overlap on the GPU; the
                     maximum is taken over the blocks' device arrays. Useful on its own: a block
                     holds fewer than 2^31 elements per sample, so a grid above one context's
                     limit still runs on one GPU.
  ``DistExchange``   one block per rank of a torch.distributed group (NCCL on GPUs, gloo on CPUs):
                     packs go to send buffers, batch_isend_irecv delivers them into the
                     neighbours' halo buffers, all_reduce(MAX) takes the maximum.
"""
from __future__ import annotations

import contextlib
import math

from . import _abi as A


def split(n: int, parts: int):
    """Contiguous ranges (offset, count) of ``parts`` blocks over ``n`` cells, sizes within one."""
    if parts < 1 or n < parts:
        raise ValueError("need 1 <= parts <= n")
    base, extra = divmod(n, parts)
    out, off = [], 0
    for p in range(parts):
        c = base + (1 if p < extra else 0)
        out.append((off, c))
        off += c
    return out


def block_coords(parts):
    """Block coordinates in rank order: rank = bx + px (by + py bz)."""
    px, py, pz = parts
    return [(bx, by, bz) for bz in range(pz) for by in range(py) for bx in range(px)]


def rank_of(coord, parts) -> int:
    return coord[0] + parts[0] * (coord[1] + parts[1] * coord[2])


def bc_pairs(bc, ndim):
    """Boundary conditions as (lo, hi) names per direction."""
    out = []
    for k in range(3):
        if isinstance(bc, str):
            out.append((bc, bc))
        else:
            out.append(tuple(bc[k]) if k < len(bc) else ("periodic", "periodic"))
    return out


def neighbour(coord, face: int, parts, periodic):
    """Coordinate of the block across face 2k + side, or None at a physical boundary."""
    k, side = face >> 1, face & 1
    if parts[k] == 1:
        return None
    c = coord[k] + (1 if side else -1)
    if not 0 <= c < parts[k]:
        if not periodic[k]:
            return None
        c %= parts[k]
    nb = list(coord)
    nb[k] = c
    return tuple(nb)


def block_config(cfg: dict, parts, coord) -> dict:
    """make_desc keywords of one block: its cells, the whole grid's counts, its offset, and halo
    faces where it borders another block (physical faces keep the grid's conditions)."""
    ndim = cfg.get("ndim", 1)
    n = list(cfg["n"]) + [1] * (3 - len(cfg["n"]))
    pairs = bc_pairs(cfg.get("bc", "periodic"), ndim)
    periodic = [pairs[k][0] == "periodic" for k in range(3)]
    local_n, offset, bcs = [], [], []
    for k in range(3):
        if k >= ndim:
            local_n.append(1)
            offset.append(0)
            bcs.append(pairs[k])
            continue
        off, cnt = split(n[k], parts[k])[coord[k]]
        local_n.append(cnt)
        offset.append(off)
        lo = "halo" if neighbour(coord, 2 * k, parts, periodic) is not None else pairs[k][0]
        hi = "halo" if neighbour(coord, 2 * k + 1, parts, periodic) is not None else pairs[k][1]
        bcs.append((lo, hi))
    kw = dict(cfg)
    kw.update(n=tuple(local_n[:ndim]), global_n=tuple(n[:ndim]), offset=tuple(offset[:ndim]), bc=bcs)
    return kw


def _on(block):
    """Stream context of a block (its own CUDA stream; nothing for host blocks)."""
    stream = getattr(block, "stream", None)
    if stream is None:
        return contextlib.nullcontext()
    import torch
    return torch.cuda.stream(stream)


class LocalExchange:
    """Every block in this process. Blocks with CUDA streams run concurrently, ordered by events: a
    block packs into a neighbour's halo only after the neighbour's previous stage (the last reader
    of that halo) has ended, and starts a stage only after its neighbours' packs for it have ended;
    the maximum runs on a stream of its own after every block's speed_max, and every block's
    time control waits for it. Host blocks (no stream) run in call order."""

    def __init__(self, blocks, coords, parts, periodic):
        self.blocks = blocks
        index = {c: i for i, c in enumerate(coords)}
        self.nbr = [[index.get(neighbour(c, f, parts, periodic)) for f in range(6)] for c in coords]
        self.peers = [sorted({j for j in row if j is not None}) for row in self.nbr]
        self.events = all(getattr(b, "stream", None) is not None for b in blocks)
        if self.events:
            import torch
            dev = blocks[0].device
            self.main = torch.cuda.Stream(device=dev)
            self.ev_stage = [torch.cuda.Event() for _ in blocks]
            self.ev_pack = [torch.cuda.Event() for _ in blocks]
            self.ev_speed = [torch.cuda.Event() for _ in blocks]
            self.ev_max = torch.cuda.Event()
            with torch.cuda.stream(self.main):
                self.gmax = torch.zeros(blocks[0].samples, dtype=torch.float64, device=dev)

    # the interior part of a stage goes before the packs: on one device the packs wait for the
    # neighbours' previous stage, and a block's own stream would hold its interior tiles behind them
    pack_first = False

    def start(self, stage: int):
        """Pack every block's boundary layers of the state stage s reads into its neighbours' halo
        buffers, each after the neighbour's previous stage (the last reader of that halo)."""
        for i, b in enumerate(self.blocks):
            # my low face's layers are the low neighbour's high-face halo, and so on
            sends = [self.blocks[j].halos[f ^ 1] if j is not None else None for f, j in enumerate(self.nbr[i])]
            if any(s is not None for s in sends):
                if self.events:
                    for j in self.peers[i]:
                        self.ev_stage[j].wait(b.stream)
                b.halo_pack(stage, sends)
            if self.events:
                self.ev_pack[i].record(b.stream)

    def finish(self, stage: int):
        """Make every block wait for its neighbours' packs of stage s (its halos are then filled)."""
        if self.events:
            for i, b in enumerate(self.blocks):
                for j in self.peers[i]:
                    self.ev_pack[j].wait(b.stream)

    def exchange(self, stage: int):
        self.start(stage)
        self.finish(stage)

    def after_stage(self, i: int):
        if self.events:
            self.ev_stage[i].record(self.blocks[i].stream)

    def join(self):
        """Make the exchange's own stream wait for every block's work so far; returns it (None for
        host blocks)."""
        if not self.events:
            return None
        for i, b in enumerate(self.blocks):
            self.ev_speed[i].record(b.stream)
            self.ev_speed[i].wait(self.main)
        return self.main

    def max(self, smax):
        import torch
        if len(smax) == 1:
            return smax[0]
        if not self.events:
            with _on(self.blocks[0]):
                return torch.stack(smax).amax(0)
        self.join()
        A.alsv_speed_max_combine(smax, self.gmax, self.main.cuda_stream)
        self.ev_max.record(self.main)
        for b in self.blocks:
            self.ev_max.wait(b.stream)
        return self.gmax


class DistExchange:
    """One block per rank of a torch.distributed group."""

    def __init__(self, block, coord, parts, periodic, group=None):
        import torch
        self.block, self.group = block, group
        self._works = []
        self.peer = []
        for f in range(6):
            nb = neighbour(coord, f, parts, periodic)
            self.peer.append(None if nb is None else self._global_rank(rank_of(nb, parts)))
        with _on(block):
            self.sends = [torch.empty_like(h) if h is not None else None for h in block.halos]

    def _global_rank(self, group_rank: int) -> int:
        import torch.distributed as dist
        if self.group is None:
            return group_rank
        return dist.get_global_rank(self.group, group_rank)

    # pack and post the transfers first, so that they travel while the interior tiles compute
    pack_first = True

    def exchange(self, stage: int):
        self.start(stage)
        self.finish(stage)

    def finish(self, stage: int):
        b = self.block
        with _on(b):
            for w in self._works:
                w.wait()
        self._works = []

    def start(self, stage: int):
        import torch.distributed as dist
        b = self.block
        b.halo_pack(stage, [s if p is not None else None for s, p in zip(self.sends, self.peer)])
        ops = []
        # sends in face order; receives in the order the neighbour sends them (its face f ^ 1 is my
        # face f), so that two messages between the same pair match also where tags are ignored
        for f in range(6):
            if self.peer[f] is not None:
                ops.append(dist.P2POp(dist.isend, self.sends[f], self.peer[f], self.group, tag=f))
        for f in (1, 0, 3, 2, 5, 4):
            if self.peer[f] is not None:
                ops.append(dist.P2POp(dist.irecv, b.halos[f], self.peer[f], self.group, tag=f ^ 1))
        self._works = []
        if ops:
            with _on(b):
                self._works = list(dist.batch_isend_irecv(ops))

    def after_stage(self, i: int):
        pass

    def join(self):
        return getattr(self.block, "stream", None)

    def max(self, smax):
        import torch.distributed as dist
        with _on(self.block):
            dist.all_reduce(smax[0], op=dist.ReduceOp.MAX, group=self.group)
        return smax[0]


class Decomposition:
    """One grid (``cfg``: the make_desc keywords of the whole grid) advanced as ``parts`` blocks.

    ``transport``: "local" (every block in this process on one device, each on its own stream) or
    "dist" (this rank's block of a torch.distributed group whose size is the number of blocks).
    ``make_block``: factory of a block from make_desc keywords (default: a Solver on ``device``).
    ``tile_variant``: stage schedule of every block (include/alsv.h, execution controls; None keeps
    the default).
    ``overlap``: run each stage as two parts around the exchange - the tiles whose stencil reads no
    halo buffer while the layers travel, the rest after they arrive (the paper overlaps its
    exchange with the inner-domain computation); False runs whole stages after the exchange. Both
    give bitwise the same result. Default (None): on for the distributed transport, off for blocks
    on one device, where nothing travels and the split only doubles the stage launches (measured
    6 % slower at 256^3 in four blocks).
    """

    def __init__(self, parts=(2, 1, 1), transport="local", group=None, make_block=None, device="cuda",
                 tile_variant=None, overlap=None, **cfg):
        import torch
        self.torch = torch
        parts = tuple(int(p) for p in parts) + (1,) * (3 - len(parts))
        ndim = cfg.get("ndim", 1)
        if any(parts[k] != 1 for k in range(ndim, 3)):
            raise ValueError("parts beyond ndim must be 1")
        self.parts, self.cfg = parts, dict(cfg)
        self.overlap = (transport == "dist") if overlap is None else bool(overlap)
        pairs = bc_pairs(cfg.get("bc", "periodic"), ndim)
        periodic = [pairs[k][0] == "periodic" for k in range(3)]
        coords = block_coords(parts)
        if make_block is None:
            from .solver import Solver

            def make_block(**kw):
                return Solver(device=device, **kw)     # each block on a stream of its own
        if transport == "local":
            self.coords = coords
            self.blocks = [make_block(**block_config(cfg, parts, c)) for c in coords]
            for b in self.blocks:
                b.bind_halo()
            self.xch = LocalExchange(self.blocks, coords, parts, periodic)
        elif transport == "dist":
            import torch.distributed as dist
            world, rank = dist.get_world_size(group), dist.get_rank(group)
            if world != len(coords):
                raise ValueError(f"{len(coords)} blocks need a group of {len(coords)} ranks, not {world}")
            self.coords = [coords[rank]]
            self.blocks = [make_block(**block_config(cfg, parts, coords[rank]))]
            self.blocks[0].bind_halo()
            self.xch = DistExchange(self.blocks[0], coords[rank], parts, periodic, group)
        else:
            raise ValueError("transport must be 'local' or 'dist'")
        if tile_variant is not None:
            for b in self.blocks:
                b.set_tile_variant(tile_variant)
        self._prof = None
        b0 = self.blocks[0]
        self.stages = b0.stages
        self.smax = []
        for b in self.blocks:
            with _on(b):
                self.smax.append(torch.zeros(b.samples, dtype=torch.float64, device=b.device))

    # ---- the protocol
    def _prepare(self):
        for b, m in zip(self.blocks, self.smax):
            b.speed_max(m)
        g = self.xch.max(self.smax)
        for b in self.blocks:
            b.finish_step(g, False)

    def set_initial_data(self, kind="kh", theta=None):
        for b in self.blocks:
            b.set_initial_data(kind, theta)
        self._prepare()

    def set_profiling(self, on: bool):
        """Record CUDA events around every stage launch of later steps (stage_ms reads their sum)."""
        self._prof = [] if on else None

    def stage_ms(self):
        """Device time of the stage launches recorded since set_profiling(True), and their count."""
        if not self._prof:
            return 0.0, 0
        for _, e1 in self._prof:      # the blocks' streams finish in any order
            e1.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in self._prof), len(self._prof)

    def _stage(self, b, s, part=None):
        run = (lambda: b.stage(s)) if part is None else (lambda: b.stage_part(s, part))
        if self._prof is None:
            run()
            return
        torch = self.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        run()
        e1.record(b.stream)
        self._prof.append((e0, e1))

    def step(self, n: int = 1):
        for _ in range(n):
            for s in range(self.stages):
                if self.overlap:
                    if self.xch.pack_first:
                        self.xch.start(s)
                    for b in self.blocks:
                        self._stage(b, s, "interior")
                    if not self.xch.pack_first:
                        self.xch.start(s)
                    self.xch.finish(s)
                    for i, b in enumerate(self.blocks):
                        self._stage(b, s, "boundary")
                        self.xch.after_stage(i)
                    continue
                self.xch.exchange(s)
                for i, b in enumerate(self.blocks):
                    self._stage(b, s)
                    self.xch.after_stage(i)
            for b, m in zip(self.blocks, self.smax):
                b.speed_max(m)
            g = self.xch.max(self.smax)
            for b in self.blocks:
                b.finish_step(g, True)

    def evolve_to(self, T: float, check_every: int = 8, max_steps: int = 1 << 26) -> int:
        """Advance every sample to T; returns the largest step count. Synchronous."""
        for b in self.blocks:
            b.set_end_time(T)
        self._prepare()
        fixed = float(self.cfg.get("fixed_dt", 0.0) or 0.0)
        target = math.ceil(T / fixed * (1.0 - 1e-12)) if fixed > 0 else None
        taken = 0
        while True:
            t, steps = self.blocks[0].time()
            done = all(int(v) >= target for v in steps) if target is not None else all(float(v) >= T for v in t)
            if done:
                break
            if taken >= max_steps:
                raise RuntimeError("evolve_to: step limit reached")
            self.step(check_every)
            taken += check_every
            for b in self.blocks:
                b.sync()
        for b in self.blocks:
            b.sync()
        return int(max(int(v) for v in self.blocks[0].time()[1]))

    # ---- results
    def time(self):
        return self.blocks[0].time()

    def sync(self):
        for b in self.blocks:
            b.sync()

    def _hand_over(self, stream):
        """Order the caller's current stream after ``stream`` (results are then usable there)."""
        if stream is not None:
            self.torch.cuda.current_stream(stream.device).wait_stream(stream)

    def state(self):
        """The whole grid's state [B, nv, nz, ny, nx] assembled from the blocks (local transport;
        with "dist", this rank's block), ready on the caller's current stream."""
        torch = self.torch
        main = self.xch.join()
        if len(self.blocks) == 1:
            self._hand_over(main)
            return self.blocks[0].state()
        px, py, pz = self.parts
        at = {c: b for c, b in zip(self.coords, self.blocks)}
        with (torch.cuda.stream(main) if main is not None else contextlib.nullcontext()):
            planes = []
            for bz in range(pz):
                rows = []
                for by in range(py):
                    rows.append(torch.cat([at[(bx, by, bz)].state() for bx in range(px)], dim=4))
                planes.append(torch.cat(rows, dim=3))
            out = torch.cat(planes, dim=2)
        self._hand_over(main)
        return out

    def _assemble(self, parts, axis_z, axis_y, axis_x):
        """Concatenate per-block tensors (block order) into the whole grid along the given axes."""
        torch = self.torch
        px, py, pz = self.parts
        at = dict(zip(self.coords, parts))
        planes = []
        for bz in range(pz):
            rows = [torch.cat([at[(bx, by, bz)] for bx in range(px)], dim=axis_x) for by in range(py)]
            planes.append(torch.cat(rows, dim=axis_y))
        return torch.cat(planes, dim=axis_z)

    def stats_accumulate(self):
        """Fold the current samples into every block's FP64 Welford accumulator (the cells of the
        blocks are disjoint, so no merge is needed)."""
        for b in self.blocks:
            b.stats_accumulate()

    def stats_read(self):
        """(count, mean [q, nz, ny, nx], unbiased variance) of the whole grid assembled from the
        blocks (local transport; with "dist", this rank's block), ready on the caller's stream."""
        torch = self.torch
        reads = [b.stats_read() for b in self.blocks]
        counts = {int(c) for c, _, _ in reads}
        assert len(counts) == 1, "blocks folded different sample counts"
        main = self.xch.join()
        with (torch.cuda.stream(main) if main is not None else contextlib.nullcontext()):
            if len(self.blocks) == 1:
                mean, var = reads[0][1], reads[0][2]
            else:
                mean = self._assemble([m for _, m, _ in reads], 1, 2, 3)
                var = self._assemble([v for _, _, v in reads], 1, 2, 3)
        self._hand_over(main)
        return counts.pop(), mean, var

    def totals(self):
        """FP64 conservation totals [B][nv] summed over the blocks (block order), ready on the
        caller's current stream."""
        torch = self.torch
        parts = [b.totals() for b in self.blocks]
        main = self.xch.join()
        with (torch.cuda.stream(main) if main is not None else contextlib.nullcontext()):
            tot = parts[0].clone()
            for t in parts[1:]:
                tot += t
        self._hand_over(main)
        return tot

    def close(self):
        # the blocks' buffers are written from their neighbours' streams too: let every stream
        # drain before the contexts and tensors go
        main = self.xch.join()
        if main is not None:
            main.synchronize()
        for b in self.blocks:
            b.close()
