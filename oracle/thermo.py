"""Thermodynamics predicted by the model's pressure tensor (oracle side).

TEST INFRASTRUCTURE ONLY: used by tests/, ``__graft_entry__.smoke()`` and
bench.py's CPU baseline, never by the product path.

Everything here follows the paper's definitions literally and leans on
library primitives (``scipy.integrate.quad``, ``scipy.optimize.brentq``):

* EOS: van der Waals ``p = rho R T/(1 - b rho) - a rho^2`` and
  Carnahan-Starling (Eq. 20), both scaled by ``K_EOS``.
* Maxwell construction (from the free energy below Eq. 19): coexistence
  densities with ``p(rho_g) = p(rho_l) = p*`` and
  ``int_{rho_g}^{rho_l} (p(s) - p*)/s^2 ds = 0``.
* Flat interface from the pressure tensor of Eq. 17 with
  ``kappa = G^2 dx^4 / 4`` and ``G = K_INT sqrt(2 K_EOS a)`` (Eq. 21):
  ``kappa/2 rho'^2 = w(rho)`` with ``w(rho) = rho int_{rho_g}^{rho} (p - p*)/s^2 ds``,
  so ``sigma = int sqrt(2 kappa w) drho`` and the interface thickness ``W``
  (measured from ``0.95 rho_g + 0.05 rho_l`` to ``0.05 rho_g + 0.95 rho_l``,
  supplement Sec. V) is ``int sqrt(kappa / (2 w)) drho`` between those levels.
"""
from __future__ import annotations

import math
import warnings
from dataclasses import dataclass

from scipy.integrate import IntegrationWarning, quad
from scipy.optimize import brentq

# Carnahan-Starling constants of Eq. 20: a = 0.496388 R^2 Tc^2/pc, b = 0.187295 R Tc/pc.
CS_A = 0.496388
CS_B = 0.187295

_QUAD = dict(epsabs=0.0, epsrel=1e-13, limit=400)
# quad reports round-off when it reaches the double-precision floor of these
# smooth integrands; the results are then accurate to that floor.
warnings.filterwarnings("ignore", category=IntegrationWarning)


@dataclass(frozen=True)
class EOS:
    kind: str          # "vdw" or "cs"
    a: float
    b: float
    R: float
    T: float
    K_eos: float = 1.0

    def p_rep(self, rho: float) -> float:
        """Repulsive (short-range) part of p_EOS per unit K_EOS."""
        if self.kind == "vdw":
            return rho * self.R * self.T / (1.0 - self.b * rho)
        t = self.b * rho / 4.0
        return rho * self.R * self.T * (1 + t + t * t - t ** 3) / (1 - t) ** 3

    def dp_rep(self, rho: float) -> float:
        """d p_rep / d rho.  vdW: R T/(1 - b rho)^2.  CS: R T (1 + 4t + 4t^2 - 4t^3 + t^4)/(1 - t)^4."""
        if self.kind == "vdw":
            return self.R * self.T / (1.0 - self.b * rho) ** 2
        t = self.b * rho / 4.0
        return self.R * self.T * (1 + 4 * t + 4 * t * t - 4 * t ** 3 + t ** 4) / (1 - t) ** 4

    def p(self, rho: float) -> float:
        return self.K_eos * (self.p_rep(rho) - self.a * rho * rho)

    def rho_max(self) -> float:
        return 1.0 / self.b if self.kind == "vdw" else 4.0 / self.b


def critical_temperature(kind: str, a: float, b: float, R: float) -> float:
    """vdW: Tc = 8a/(27 R b).  CS: from the two definitions under Eq. 20,
    Tc = (a/b) (0.187295/0.496388) / R."""
    if kind == "vdw":
        return 8.0 * a / (27.0 * R * b)
    return (a / b) * (CS_B / CS_A) / R


def make_eos(kind: str, a: float, b: float, R: float, Tr: float, K_eos: float = 1.0) -> EOS:
    return EOS(kind, a, b, R, Tr * critical_temperature(kind, a, b, R), K_eos)


def _spinodals(e: EOS) -> tuple[float, float]:
    """Local maximum and minimum of p(rho) below the critical temperature."""
    rmax = e.rho_max()
    n = 4000
    grid = [rmax * (i + 0.5) / n for i in range(n)]
    vals = [e.p(r) for r in grid]
    imax = next(i for i in range(1, n - 1) if vals[i] >= vals[i - 1] and vals[i] > vals[i + 1])
    imin = next(i for i in range(imax + 1, n - 1) if vals[i] <= vals[i - 1] and vals[i] < vals[i + 1])
    dp = lambda r: e.K_eos * (e.dp_rep(r) - 2.0 * e.a * r)
    s1 = brentq(dp, grid[imax - 1], grid[imax + 1], xtol=1e-15, rtol=1e-15)
    s2 = brentq(dp, grid[imin - 1], grid[imin + 1], xtol=1e-15, rtol=1e-15)
    return s1, s2


def maxwell(e: EOS) -> tuple[float, float, float]:
    """Coexistence densities (rho_g, rho_l) and pressure p* by the Maxwell
    construction (equal area in specific volume)."""
    s1, s2 = _spinodals(e)
    rmax = e.rho_max()

    def branches(ps):
        rg = brentq(lambda r: e.p(r) - ps, 1e-300, s1, xtol=1e-300, rtol=1e-15, maxiter=500)
        rl = brentq(lambda r: e.p(r) - ps, s2, rmax * (1 - 1e-15), xtol=1e-15, rtol=1e-15, maxiter=500)
        return rg, rl

    def area(ps):
        rg, rl = branches(ps)
        return quad(lambda s: (e.p(s) - ps) / (s * s), rg, rl, **_QUAD)[0]

    p_hi = e.p(s1)
    p_lo = max(e.p(s2), 0.0)
    span = p_hi - p_lo
    ps = brentq(area, p_lo + 1e-12 * span, p_hi - 1e-12 * span, xtol=1e-16 * span, rtol=1e-15,
                maxiter=500)
    rg, rl = branches(ps)
    return rg, rl, ps


def w_profile(e: EOS, rho_g: float, p_star: float, rho: float) -> float:
    """w(rho) = rho int_{rho_g}^{rho} (p(s) - p*)/s^2 ds  (>= 0 between the phases)."""
    return rho * quad(lambda s: (e.p(s) - p_star) / (s * s), rho_g, rho, **_QUAD)[0]


def kappa(e: EOS, K_int: float) -> float:
    """kappa = G^2 dx^4 / 4 with G^2 = 2 K_INT^2 K_EOS a (Eq. 21), dx = 1."""
    return K_int * K_int * e.K_eos * e.a / 2.0


def interface(e: EOS, K_int: float = 1.0) -> dict:
    """Flat-interface predictions of the pressure tensor: coexistence densities,
    surface tension sigma and interface thickness W (5%..95% levels)."""
    rg, rl, ps = maxwell(e)
    kap = kappa(e, K_int)
    w = lambda r: w_profile(e, rg, ps, r)
    sigma = quad(lambda r: math.sqrt(max(2.0 * kap * w(r), 0.0)), rg, rl, epsabs=0.0, epsrel=1e-11,
                 limit=200)[0]
    r5 = 0.95 * rg + 0.05 * rl
    r95 = 0.05 * rg + 0.95 * rl
    W = quad(lambda r: math.sqrt(kap / (2.0 * w(r))), r5, r95, epsabs=0.0, epsrel=1e-11, limit=200)[0]
    return {"rho_g": rg, "rho_l": rl, "p_star": ps, "sigma": sigma, "W": W, "kappa": kap}


def flat_profile(e: EOS, K_int: float, z: "list[float]") -> "list[float]":
    """Analytic flat-interface density profile rho(z) (z = 0 at the mid density,
    liquid towards +z), by inverting z(rho) = int_{rho_mid}^{rho} sqrt(kappa/(2w)) drho."""
    rg, rl, ps = maxwell(e)
    kap = kappa(e, K_int)
    rmid = 0.5 * (rg + rl)
    zof = lambda r: quad(lambda s: math.sqrt(kap / (2.0 * w_profile(e, rg, ps, s))), rmid, r,
                         epsabs=0.0, epsrel=1e-10, limit=200)[0]
    out = []
    for zz in z:
        lo, hi = rg + 1e-9 * (rl - rg), rl - 1e-9 * (rl - rg)
        if zz <= zof(lo):
            out.append(lo)
        elif zz >= zof(hi):
            out.append(hi)
        else:
            out.append(brentq(lambda r: zof(r) - zz, lo, hi, xtol=1e-13))
    return out
