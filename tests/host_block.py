"""A host block of the stage-by-stage decomposition protocol that computes with the oracle: the
test double that lets the decomposition driver and its transports (in-process and
torch.distributed over gloo) run on CPUs. Its spatial operator is the oracle's; the SSP-RK stage
combination and the per-sample time control follow the rules include/alsv.h documents for
alsv_stage and alsv_finish_step (adaptive CFL mode).

A block's halo faces are handled by extending its state with the received ghost layers and
evaluating the oracle's operator on the extended grid (outflow beyond it, which reaches only the
ghost cells' own updates). Grid sizes in the tests are powers of two on [0, 1], so the extended
grid's dx is the whole grid's exactly and the blocks reproduce the whole-grid run bitwise.
"""
import numpy as np
import torch

import oracle


def _pad3(v, fill):
    v = list(v)
    return v + [fill] * (3 - len(v))


class OracleBlock:
    def __init__(self, U0_whole, **kw):
        self.kw = kw
        ndim = self.ndim = kw["ndim"]
        assert not kw.get("fixed_dt"), "the host block implements the adaptive CFL mode"
        self.n = _pad3(kw["n"], 1)
        self.gn = _pad3(kw.get("global_n") or kw["n"], 1)
        self.off = _pad3(kw.get("offset") or (0,) * ndim, 0)
        self.bc = [tuple(p) for p in kw["bc"]] if not isinstance(kw["bc"], str) else [(kw["bc"], kw["bc"])] * 3
        self.G = 1 if kw.get("recon", "mc") == "pc" else 2
        self.stages = 3 if kw.get("rk", "ssprk2") == "ssprk3" else 2
        self.cfl = kw.get("cfl", 0.45)
        self.device = torch.device("cpu")
        self.stream = None
        n, off = self.n, self.off
        self.U0 = np.ascontiguousarray(U0_whole[:, :, off[2]:off[2] + n[2], off[1]:off[1] + n[1], off[0]:off[0] + n[0]],
                                       dtype=np.float64)
        self.samples, self.nv = self.U0.shape[0], self.U0.shape[1]
        lo = _pad3(kw.get("lo", (0.0,) * 3), 0.0)
        hi = _pad3(kw.get("hi", (1.0,) * 3), 1.0)
        dx = [(hi[k] - lo[k]) / self.gn[k] for k in range(3)]
        self.ext = [(self.G if k < ndim and self.bc[k][0] == "halo" else 0,
                     self.G if k < ndim and self.bc[k][1] == "halo" else 0) for k in range(3)]
        en = [n[k] + self.ext[k][0] + self.ext[k][1] for k in range(3)]
        elo = [lo[k] + (off[k] - self.ext[k][0]) * dx[k] for k in range(3)]
        ehi = [elo[k] + en[k] * dx[k] for k in range(3)]
        for k in range(ndim):
            assert (ehi[k] - elo[k]) / en[k] == dx[k], "test grids must keep dx exact (powers of two)"
        ebc = [tuple("outflow" if s == "halo" else s for s in self.bc[k]) for k in range(3)]
        common = {key: kw[key] for key in ("eq", "gamma", "recon", "rvars", "flux", "rk", "cfl", "weno_eps",
                                           "weno_eps_dx2") if key in kw}
        self.d_ext = oracle.make_desc(ndim=ndim, n=en[:ndim], lo=elo, hi=ehi, bc=ebc, **common)
        blo = [lo[k] + off[k] * dx[k] for k in range(3)]
        bhi = [blo[k] + n[k] * dx[k] for k in range(3)]
        self.d_blk = oracle.make_desc(ndim=ndim, n=n[:ndim], lo=blo, hi=bhi, bc=ebc, **common)
        self.halos = [None] * 6
        self.set_initial_data()

    # ---- the block interface the decomposition driver uses
    def set_initial_data(self, kind=None, theta=None):
        B = self.samples
        self.U = self.U0.copy()
        self.A = np.zeros_like(self.U)
        self.Bb = np.zeros_like(self.U)
        self.t = np.zeros(B)
        self.steps = np.zeros(B, dtype=np.int64)
        self.dt = np.zeros(B)
        self.last = np.zeros(B, dtype=bool)
        self.done = np.zeros(B, dtype=bool)
        self.T = np.inf
        self.status = 0

    def halo_info(self):
        elems = []
        for f in range(6):
            k, side = f >> 1, f & 1
            if k < self.ndim and self.bc[k][side] == "halo":
                cross = int(np.prod(self.n)) // self.n[k]
                elems.append(self.samples * self.nv * self.G * cross)
            else:
                elems.append(0)
        return self.G, elems

    def bind_halo(self):
        _, elems = self.halo_info()
        self.halos = [torch.zeros(e, dtype=torch.float64) if e else None for e in elems]
        return self.halos

    def _state(self, s):
        return (self.U, self.A, self.Bb)[s]

    def _coef(self, s):
        if self.stages == 2:
            return ((0.0, 1.0, None, self.A), (0.5, 0.5, self.U, self.U))[s]
        return ((0.0, 1.0, None, self.A), (0.75, 0.25, self.U, self.Bb), (1.0 / 3.0, 2.0 / 3.0, self.U, self.U))[s]

    def halo_pack(self, stage, sends):
        X = self._state(stage)
        G = self.G
        for f, dst in enumerate(sends):
            if dst is None:
                continue
            k, side = f >> 1, f & 1
            ax = 4 - k
            idx = np.arange(G) if side == 0 else np.arange(self.n[k] - G, self.n[k])
            lay = np.moveaxis(np.take(X, idx, axis=ax), ax, 2)    # [B, nv, G, cross (z, y, x)]
            flat = np.ascontiguousarray(lay).reshape(-1)
            dst[:flat.size] = torch.from_numpy(flat)

    def _extended(self, X):
        pad = [(0, 0), (0, 0)] + [self.ext[k] for k in (2, 1, 0)]
        E = np.pad(X, pad, mode="edge")   # corners keep edge copies: the stencils never read them
        G = self.G
        for f in range(6):
            k, side = f >> 1, f & 1
            if self.ext[k][side] == 0:
                continue
            ax = 4 - k
            shape = [self.samples, self.nv, G] + [self.n[j] for j in (2, 1, 0) if j != k]
            lay = self.halos[f][:int(np.prod(shape))].numpy().reshape(shape)
            lay = np.moveaxis(lay, 2, ax)
            sl = [slice(None), slice(None)]
            for j in (2, 1, 0):
                lo_j = self.ext[j][0]
                if j == k:
                    start = 0 if side == 0 else lo_j + self.n[j]
                    sl.append(slice(start, start + G))
                else:
                    sl.append(slice(lo_j, lo_j + self.n[j]))
            E[tuple(sl)] = lay
        return E

    def _interior(self, E):
        sl = [slice(None), slice(None)]
        for j in (2, 1, 0):
            sl.append(slice(self.ext[j][0], self.ext[j][0] + self.n[j]))
        return E[tuple(sl)]

    def stage(self, s):
        Us = self._state(s)
        a, b, Un, out = self._coef(s)
        L = self._interior(oracle.rhs(self.d_ext, self._extended(Us)))
        dt = self.dt[:, None, None, None, None]
        new = b * (Us + dt * L) if Un is None else a * Un + b * (Us + dt * L)
        live = ~self.done
        out[live] = new[live]

    def stage_part(self, s, part):
        """The interior part computes nothing here; the boundary part (after the exchange) runs the
        whole stage - the same result as the device's split."""
        if part == "boundary":
            self.stage(s)

    def speed_max(self, m):
        s = oracle.max_speed(self.d_blk, self.U)
        m[:] = torch.from_numpy(np.where(np.isfinite(s), s, np.inf))

    def finish_step(self, smax, advance):
        g = smax.numpy()
        for b in range(self.samples):
            if advance and self.done[b]:
                continue
            if advance:
                self.steps[b] += 1
                self.t[b] = self.T if self.last[b] else self.t[b] + self.dt[b]
            if not g[b] < np.inf:
                self.status |= 1
                self.done[b] = True
                continue
            t = self.t[b]
            if not t < self.T:
                self.done[b] = True
                continue
            dt = self.cfl / g[b]
            last = False
            if not dt < self.T - t:
                dt = self.T - t
                last = True
            if np.isinf(dt):
                dt = 0.0
            self.dt[b], self.last[b], self.done[b] = dt, last, False

    def set_end_time(self, T):
        self.T = T

    def time(self):
        return self.t.copy(), self.steps.copy()

    def sync(self):
        if self.status:
            raise FloatingPointError("non-physical state")

    def state(self):
        return torch.from_numpy(self.U)

    def totals(self):
        return torch.from_numpy(oracle.totals(self.d_blk, self.U))

    def close(self):
        pass
