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


# --- D3Q19 form of the model (lbm3d_oracle.cpp) ---------------------------------

def k_3d(varpi: float) -> float:
    """k of the 3-D collision matrix: the bulk viscosity (1 - 11 k / 38) (2/3) c_s^2 tau_e
    is varpi times the plain lattice's, so k = 38 (1 - varpi) / 11."""
    return 38.0 * (1.0 - varpi) / 11.0


def relaxation_rates_3d(s_p: float, varpi: float) -> tuple[float, float]:
    """(s_q, s_e) from the D3Q19 closure tau_p tau_q = (1 + 5 k / 19) tau_e tau_q = 1/12,
    the 3-D counterpart of Eq. 16 (the isotropic error term of the steady third-order
    analysis is proportional to (1 + 5k/19) tau_e tau_q - tau_p tau_q, the anisotropic
    one to 12 tau_p tau_q - 1, as on D2Q9 with k + 1 in place of 1 + 5k/19)."""
    tau_p = 1.0 / s_p - 0.5
    tau_q = 1.0 / (12.0 * tau_p)
    tau_e = 1.0 / (12.0 * (1.0 + 5.0 * k_3d(varpi) / 19.0) * tau_q)
    return 1.0 / (tau_q + 0.5), 1.0 / (tau_e + 0.5)


@dataclass
class LatticeParams3(LatticeParams):
    """D3Q19 parameters: the D2Q9 set plus the rates of the third-order m moments
    (s_m) and the anisotropic fourth-order pi moments (s_pi)."""
    sm: float = 1.0
    spi: float = 1.0


S_EPS_3D = 1.75


def from_physical_3d(s_m: float | None = None, s_pi: float | None = None, **kw) -> LatticeParams3:
    """As from_physical (same EOS, G, c^2 and coexistence densities: the recovered
    pressure tensor of the 3-D model is that of Eq. 17), with the 3-D rate closure.
    Unless given, s_eps = 1.75, s_m = s_q (all third-order moments at one rate) and
    s_pi = s_eps (all fourth-order moments at one rate).  None of the three enters
    the Navier-Stokes stress or the steady third-order terms; s_eps = s_e (the 2-D
    default) leaves the checkerboard mode k = (pi, pi, pi) of the e-eps block
    unstable in the gas (|lambda| = 1.26 per step at Tr = 0.8), s_eps = s_pi in
    [1.7, 1.8] makes the uniform gas and liquid linearly stable at every wave vector."""
    s_p = kw.get("s_p", 1.0)
    varpi = kw.get("varpi", 1.0 / 6.0)
    sq, se = relaxation_rates_3d(s_p, varpi)
    kw.setdefault("s_q", sq)
    kw.setdefault("s_e", se)
    kw.setdefault("s_eps", S_EPS_3D)
    base = from_physical(**kw)
    d = base.as_dict()
    d["sm"] = base.sq if s_m is None else s_m
    d["spi"] = base.seps if s_pi is None else s_pi
    return LatticeParams3(**d)
