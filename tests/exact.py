"""Exact solutions used to pin the oracle (test-only, numpy).

* Exact Riemann solver for the 1D Euler equations of an ideal gas: the star pressure is the root
  of f_L(p) + f_R(p) + u_R - u_L = 0 (shock branch from the Rankine-Hugoniot conditions,
  rarefaction branch from the isentropic Riemann invariants), solved by Newton's method; the
  solution is then sampled along x/t. Written from the gas-dynamics relations (Toro, Riemann
  Solvers and Numerical Methods for Fluid Dynamics, ch. 4).
* Burgers u_t + (u^2/2)_x = 0 with u0 = sin(2 pi x) before the shock time 1/(2 pi): foot points
  xi solve xi + t u0(xi) = x, and the exact cell average of u over [x_a, x_b] is
  [U0(xi) + t u0(xi)^2 / 2]_{xi_a}^{xi_b} / (x_b - x_a) with U0' = u0.
"""
from __future__ import annotations

import math

import numpy as np


class RiemannExact:
    def __init__(self, WL, WR, gamma=1.4):
        self.g = gamma
        self.rL, self.uL, self.pL = map(float, WL)
        self.rR, self.uR, self.pR = map(float, WR)
        self.cL = math.sqrt(gamma * self.pL / self.rL)
        self.cR = math.sqrt(gamma * self.pR / self.rR)
        self.pstar, self.ustar = self._solve()

    def _fK(self, p, rK, pK, cK):
        g = self.g
        if p > pK:  # shock
            A = 2.0 / ((g + 1.0) * rK)
            Bk = (g - 1.0) / (g + 1.0) * pK
            f = (p - pK) * math.sqrt(A / (p + Bk))
            df = math.sqrt(A / (Bk + p)) * (1.0 - 0.5 * (p - pK) / (Bk + p))
        else:  # rarefaction
            f = 2.0 * cK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
            df = 1.0 / (rK * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
        return f, df

    def _solve(self):
        du = self.uR - self.uL
        p = max(1e-8, 0.5 * (self.pL + self.pR))
        for _ in range(100):
            fL, dL = self._fK(p, self.rL, self.pL, self.cL)
            fR, dR = self._fK(p, self.rR, self.pR, self.cR)
            pn = p - (fL + fR + du) / (dL + dR)
            pn = max(pn, 1e-12)
            if abs(pn - p) <= 1e-15 * (pn + p):
                p = pn
                break
            p = pn
        fL, _ = self._fK(p, self.rL, self.pL, self.cL)
        fR, _ = self._fK(p, self.rR, self.pR, self.cR)
        u = 0.5 * (self.uL + self.uR) + 0.5 * (fR - fL)
        return p, u

    def star_densities(self):
        g = self.g
        out = []
        for (rK, pK) in ((self.rL, self.pL), (self.rR, self.pR)):
            q = self.pstar / pK
            if q > 1.0:
                out.append(rK * (q + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * q + 1.0))
            else:
                out.append(rK * q ** (1.0 / g))
        return tuple(out)

    def shock_speed_right(self):
        g = self.g
        q = self.pstar / self.pR
        return self.uR + self.cR * math.sqrt((g + 1) / (2 * g) * q + (g - 1) / (2 * g))

    def shock_speed_left(self):
        g = self.g
        q = self.pstar / self.pL
        return self.uL - self.cL * math.sqrt((g + 1) / (2 * g) * q + (g - 1) / (2 * g))

    def sample(self, xi):
        """Primitive (rho, u, p) at similarity coordinate xi = (x - x0)/t (array)."""
        xi = np.asarray(xi, dtype=np.float64)
        g = self.g
        rho = np.empty_like(xi)
        u = np.empty_like(xi)
        p = np.empty_like(xi)
        rsL, rsR = self.star_densities()
        ps, us = self.pstar, self.ustar
        for idx, s in np.ndenumerate(xi):
            if s <= us:  # left of contact
                if ps > self.pL:
                    SL = self.shock_speed_left()
                    W = (self.rL, self.uL, self.pL) if s <= SL else (rsL, us, ps)
                else:
                    SH = self.uL - self.cL
                    cs = self.cL * (ps / self.pL) ** ((g - 1) / (2 * g))
                    ST = us - cs
                    if s <= SH:
                        W = (self.rL, self.uL, self.pL)
                    elif s >= ST:
                        W = (rsL, us, ps)
                    else:
                        base = 2 / (g + 1) + (g - 1) / ((g + 1) * self.cL) * (self.uL - s)
                        W = (self.rL * base ** (2 / (g - 1)),
                             2 / (g + 1) * (self.cL + (g - 1) / 2 * self.uL + s),
                             self.pL * base ** (2 * g / (g - 1)))
            else:  # right of contact
                if ps > self.pR:
                    SR = self.shock_speed_right()
                    W = (self.rR, self.uR, self.pR) if s >= SR else (rsR, us, ps)
                else:
                    SH = self.uR + self.cR
                    cs = self.cR * (ps / self.pR) ** ((g - 1) / (2 * g))
                    ST = us + cs
                    if s >= SH:
                        W = (self.rR, self.uR, self.pR)
                    elif s <= ST:
                        W = (rsR, us, ps)
                    else:
                        base = 2 / (g + 1) - (g - 1) / ((g + 1) * self.cR) * (self.uR - s)
                        W = (self.rR * base ** (2 / (g - 1)),
                             2 / (g + 1) * (-self.cR + (g - 1) / 2 * self.uR + s),
                             self.pR * base ** (2 * g / (g - 1)))
            rho[idx], u[idx], p[idx] = W
        return rho, u, p

    def cell_average_density(self, n, t, x0=0.5, sub=64):
        """Cell averages of rho on n uniform cells of [0,1] at time t (midpoint sub-sampling)."""
        h = 1.0 / n
        offs = (np.arange(sub) + 0.5) / sub
        x = (np.arange(n)[:, None] + offs[None, :]) * h
        rho, _, _ = self.sample((x - x0) / t)
        return rho.mean(axis=1)


def burgers_sine_cell_averages(n, t):
    """Exact cell averages of the Burgers solution with u0 = sin(2 pi x) on [0,1] periodic."""
    two_pi = 2.0 * math.pi
    xe = np.arange(n + 1) / n

    def foot(x):
        xi = x.copy()
        for _ in range(100):
            g = xi + t * np.sin(two_pi * xi) - x
            dg = 1.0 + t * two_pi * np.cos(two_pi * xi)
            step = g / dg
            xi = xi - step
            if np.max(np.abs(step)) < 1e-16:
                break
        return xi

    xi = foot(xe)
    prim = -np.cos(two_pi * xi) / two_pi + 0.5 * t * np.sin(two_pi * xi) ** 2
    return np.diff(prim) * n


def observed_rates(ns, errs):
    ns = np.asarray(ns, dtype=float)
    errs = np.asarray(errs, dtype=float)
    return np.log(errs[:-1] / errs[1:]) / np.log(ns[1:] / ns[:-1])
