"""Pins of the oracle's thermodynamics (Maxwell construction, pressure-tensor
sigma and W) against the numbers the paper prints and against closed forms."""
import math
import os

import numpy as np
import pytest

from oracle import thermo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _rows("cs_interface_constants.txt"), ids=lambda r: "Tr%.1f" % r[0])
def test_cs_pressure_tensor_constants(row):
    """W/K_INT and sigma/K_INT for the CS EOS (a=1, b=4, R=1, K_EOS=K_INT=1) to the printed digits."""
    Tr, W_an, s_an, W_sim, s_sim = row
    r = thermo.interface(thermo.make_eos("cs", 1.0, 4.0, 1.0, Tr), 1.0)
    assert round(r["W"], 4) == pytest.approx(W_an, abs=1.01e-4)
    digits = 6 if s_an < 0.01 else 5
    assert round(r["sigma"], digits) == pytest.approx(s_an, abs=1.01 * 10 ** -digits)
    # The paper's simulated slopes agree with the analytic values within 0.7%.
    assert W_sim == pytest.approx(r["W"], rel=7e-3)
    assert s_sim == pytest.approx(r["sigma"], rel=7e-3)


def test_cs_kint_for_width_10():
    r = thermo.interface(thermo.make_eos("cs", 1.0, 4.0, 1.0, 0.8), 1.0)
    assert round(10.0 / r["W"], 4) == 2.2949


@pytest.mark.parametrize("row", _rows("cs_fixed_width_sigma.txt"), ids=lambda r: "Tr%.1f" % r[0])
def test_cs_sigma_at_fixed_width(row):
    """sigma ~ K_EOS K_INT and W ~ K_INT: at fixed W, sigma/K_EOS = sigma_1 W / W_1,
    which matches the paper's simulated slopes (supplement Fig. 4) within 1%."""
    Tr, W, slope = row
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, Tr)
    r1 = thermo.interface(e, 1.0)
    K_int = W / r1["W"]
    r = thermo.interface(thermo.make_eos("cs", 1.0, 4.0, 1.0, Tr, K_eos=3.0), K_int)
    assert r["W"] == pytest.approx(W, rel=1e-9)                       # W independent of K_EOS
    assert r["sigma"] / 3.0 == pytest.approx(r1["sigma"] * K_int, rel=1e-9)
    assert r["sigma"] / 3.0 == pytest.approx(slope, rel=1e-2)


def _vdw_mu(e, rho):
    """Chemical potential from the closed-form vdW free energy
    psi = rho R T ln(rho/(1 - b rho)) - a rho^2."""
    return e.R * e.T * (math.log(rho / (1 - e.b * rho)) + 1 / (1 - e.b * rho)) - 2 * e.a * rho


def _cs_mu(e, rho):
    """Chemical potential from the closed-form CS free energy
    psi = rho R T [ln rho + (4t - 3t^2)/(1 - t)^2] - a rho^2, t = b rho / 4."""
    t = e.b * rho / 4
    g = (4 * t - 3 * t * t) / (1 - t) ** 2
    dg = (4 - 2 * t) / (1 - t) ** 3 * e.b / 4
    return e.R * e.T * (math.log(rho) + 1 + g + rho * dg) - 2 * e.a * rho


@pytest.mark.parametrize("kind,a,b,Tr", [("vdw", 9 / 49, 2 / 21, 0.85), ("vdw", 9 / 49, 2 / 21, 0.65),
                                         ("cs", 1.0, 4.0, 0.7), ("cs", 1.0, 4.0, 0.95)])
def test_maxwell_equals_common_tangent(kind, a, b, Tr):
    """Equal-area coexistence = equal pressure and chemical potential of the closed-form free energy."""
    e = thermo.make_eos(kind, a, b, 1.0, Tr)
    rg, rl, ps = thermo.maxwell(e)
    mu = _vdw_mu if kind == "vdw" else _cs_mu
    assert e.p(rg) == pytest.approx(ps, rel=1e-12) and e.p(rl) == pytest.approx(ps, rel=1e-12)
    assert mu(e, rg) == pytest.approx(mu(e, rl), rel=1e-11, abs=1e-13)
    assert rg < rl


def test_vdw_reduced_coexistence_is_universal():
    """The vdW law of corresponding states: reduced coexistence densities depend on Tr only."""
    out = []
    for a, b in [(9 / 49, 2 / 21), (1.0, 0.5), (3.0, 0.1)]:
        e = thermo.make_eos("vdw", a, b, 1.0, 0.8)
        rg, rl, _ = thermo.maxwell(e)
        out.append((rg * 3 * b, rl * 3 * b))
    assert np.allclose(out, out[0], rtol=1e-11)
