"""Physical -> lattice-unit parameters for the oracle (test infrastructure only).

The paper fixes (main text, after Eq. 20):
  * G = K_INT sqrt(2 K_EOS a / dx^2)                              (Eq. 21)
  * c_s = K_INT sqrt(d/drho (p_EOS + K_EOS a rho^2)) at rho_l       (Eq. 22)
  * c = sqrt(3) c_s, dt = dx / c                                    (below Eq. 9)
and the relaxation-rate constraint tau_p tau_q = (k+1) tau_e tau_q = 1/12
with tau = 1/s - 1/2 (Eq. 16).  The oracle runs with c = 1, so the pressure is
carried as p/c^2: lam = K_EOS / c^2 multiplies the EOS and G2 = G^2 / c^2.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Pins (tests/test_oracle_physics.py): relaxation_rates by hand-worked values and
by the flat-interface tests whose outcome depends on Eq. 16; the c^2 rule (Eq. 22)
and G (Eq. 21) by what they say about the recovered pressure p_LBE = p_EOS +
G^2 rho^2 / 2, with slopes of the EOS pressure taken by central differences: in
lattice units K_INT^2 lam d(p + a rho^2)/drho = 1/3 at rho_l, the attraction left
in p_LBE is (K_INT^2 - 1) K_EOS a rho^2, and at K_INT = 1 the liquid's sound speed
equals the lattice sound speed (four planted mistakes each fail it).
"""
from __future__ import annotations

from dataclasses import asdict, dataclass

from . import thermo

EOS_CODE = {"vdw": 0, "cs": 1, "ideal": 2}


@dataclass
class LatticeParams:
    eos: int
    form: int
    eos_a: float
    eos_b: float
    R_gas: float
    T: float
    lam: float
    G2: float
    varpi: float
    s0: float
    se: float
    seps: float
    sj: float
    sq: float
    sp: float
    # Bookkeeping (not used by the step): coexistence densities of the EOS.
    rho_g: float = float("nan")
    rho_l: float = float("nan")
    Tc: float = float("nan")

    def as_dict(self) -> dict:
        return asdict(self)


def relaxation_rates(s_p: float, varpi: float) -> tuple[float, float]:
    """(s_q, s_e) from tau_p tau_q = (k + 1) tau_e tau_q = 1/12, k = 1 - varpi (Eq. 16)."""
    tau_p = 1.0 / s_p - 0.5
    tau_q = 1.0 / (12.0 * tau_p)
    k = 1.0 - varpi
    tau_e = 1.0 / (12.0 * (k + 1.0) * tau_q)
    return 1.0 / (tau_q + 0.5), 1.0 / (tau_e + 0.5)


def from_physical(eos: str = "vdw", a: float = 9.0 / 49.0, b: float = 2.0 / 21.0, R: float = 1.0,
                  Tr: float = 0.85, K_eos: float = 1.0, K_int: float = 1.0, G2: float | None = None,
                  varpi: float = 1.0 / 6.0, s_p: float = 1.0, s_q: float | None = None,
                  s_e: float | None = None, s_eps: float | None = None, s0: float = 1.0,
                  sj: float = 1.0, form: int = 13) -> LatticeParams:
    """Lattice parameters for a two-phase run at reduced temperature Tr."""
    e = thermo.make_eos(eos, a, b, R, Tr, K_eos)
    rg, rl, _ = thermo.maxwell(e)
    c2 = 3.0 * K_int * K_int * K_eos * e.dp_rep(rl)       # c^2 = 3 c_s^2
    lam = K_eos / c2
    g2 = 2.0 * K_int * K_int * K_eos * a / c2 if G2 is None else G2
    sq_d, se_d = relaxation_rates(s_p, varpi)
    se = se_d if s_e is None else s_e
    return LatticeParams(eos=EOS_CODE[eos], form=form, eos_a=a, eos_b=b, R_gas=R, T=e.T, lam=lam,
                         G2=g2, varpi=varpi, s0=s0, se=se, seps=se if s_eps is None else s_eps,
                         sj=sj, sq=sq_d if s_q is None else s_q, sp=s_p, rho_g=rg, rho_l=rl,
                         Tc=thermo.critical_temperature(eos, a, b, R))
