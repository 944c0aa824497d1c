"""Symbolic Chapman-Enskog pins of the collision coefficients (oracle/chapman_enskog.py):
the expansion of the discrete scheme reproduces the paper's D2Q9 statements (Eq. 7
gives a Newtonian stress with bulk viscosity varpi c_s^2 tau_e; the steady
third-order residual is the lattice term plus the paper's R_iso-bar and
R_aniso-bar), and with the D3Q19 coefficients of the 3-D oracle every O(Ma)
non-Newtonian term and every third-order eta term vanish.  Planted mistakes in the
coefficients leave terms that do not vanish."""
import pytest

sp = pytest.importorskip("sympy")

from oracle import chapman_enskog as ce  # noqa: E402


def _all_zero(res):
    return all(sp.simplify(v) == 0 for comp in res.values() for v in comp.values())


@pytest.mark.parametrize("mistake", [None, "b", "k"])
def test_d2q9_coefficients_give_the_newtonian_stress(mistake):
    w = sp.Symbol("varpi")
    kw = {None: {}, "b": dict(b=1 / (1 - 3 * w)), "k": dict(k=1 - w / 2)}[mistake]
    res = ce.d2q9_ns(w, **kw)
    assert _all_zero(res) == (mistake is None)


@pytest.mark.parametrize("varpi", [sp.Rational(1, 6), sp.Rational(3, 10)])
@pytest.mark.parametrize("mistake", [None, "h", "beta2"])
def test_d3q19_coefficients_give_the_newtonian_stress(varpi, mistake):
    w = varpi
    k = 38 * (1 - w) / 11
    co = dict(k=k, beta2=-19 / k, b=21 * (1 - w) / (5 * (7 - 18 * w)), h=798 * w * (1 - w) / (5 * (7 - 18 * w)))
    if mistake == "h":
        co["h"] = 0
    elif mistake == "beta2":
        co["beta2"] = -2 / (1 - w)  # the 2-D beta_2
    res = ce.d3q19_ns(w, **co)
    assert _all_zero(res) == (mistake is None)


def test_d2q9_steady_residual_is_the_papers():
    """The steady eta terms are -(R_iso-bar + R_aniso-bar) of the paper with
    p-bar = (3 + beta_2) c_s^2 eta (as the residual, momentum balance minus F);
    no term in rho beyond the lattice one."""
    w = sp.Rational(1, 6)
    te, tq, tp = sp.symbols("tau_e tau_q tau_p", positive=True)
    s = lambda t: 1 / (t + sp.Rational(1, 2))
    eta_parts, rho_parts, d = ce.d2q9_steady(w, s(te), sp.Rational(3, 2), s(tq), s(tp))
    k, beta2 = 1 - w, -2 / (1 - w)
    pbar = (3 + beta2) * ce.CS2
    lap = d[0] ** 2 + d[1] ** 2
    for a in range(2):
        R_iso = -sp.Rational(1, 6) * ((k + 1) * te * tq - tp * tq) * lap * d[a] * pbar
        R_ani = -sp.Rational(1, 12) * (12 * tp * tq - 1) * [d[1] ** 2 * d[0], d[0] ** 2 * d[1]][a] * pbar
        assert sp.simplify(eta_parts[a] + R_iso + R_ani) == 0
        assert rho_parts[a] == 0


def _rates(kind):
    """Rational rates at s_p = 1, varpi = 1/6: the 3-D closure, or a planted mistake."""
    k = sp.Rational(95, 33)
    tp, tq = sp.Rational(1, 2), sp.Rational(1, 6)
    te = 1 / (12 * (1 + 5 * k / 19) * tq)
    if kind == "2d_closure":
        te = 1 / (12 * (sp.Rational(5, 6) + 1) * tq)
    elif kind == "sixth":
        tq = 1 / (6 * tp)
    s = lambda t: 1 / (t + sp.Rational(1, 2))
    return k, s(te), s(tq), s(tp)


@pytest.mark.parametrize("kind", [None, "2d_closure", "sixth"])
def test_d3q19_rate_closure_removes_the_steady_eta_terms(kind):
    """With tau_p tau_q = (1 + 5k/19) tau_e tau_q = 1/12 the steady third-order eta
    terms vanish whatever s_eps, s_m, s_pi are; with the 2-D closure or
    tau_p tau_q = 1/6 they do not."""
    k, se, sq, sp_ = _rates(kind)
    eta_parts, rho_parts, _ = ce.d3q19_steady(k, se, sp.Rational(7, 4), sq, sp_, sp.Rational(13, 10), sp.Rational(7, 4))
    assert all(r == 0 for r in rho_parts)
    assert all(e == 0 for e in eta_parts) == (kind is None)


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19"])
def test_q_m_enters_the_steady_balance_through_its_second_order_tensor(lattice):
    """At third order the term S Q_m (Eq. 13) adds div Pi(M^-1 Q_m) to the steady
    momentum balance and nothing else, whatever its fourth-order components are:
    the paper's R_add is -div of (2 F~F~ + |F~|^2 I)/24, the second-order tensor of
    its Q_m, and a 3-D Q_m with that tensor gives the same pressure tensor (the
    reading of the 3-D Q_m)."""
    if lattice == "d2q9":
        w = sp.Rational(1, 6)
        res = ce.d2q9_steady(w, sp.Rational(22, 17), sp.Rational(3, 2), sp.Rational(3, 2), sp.Integer(1),
                             q_rows=("e", "eps", "pxx", "pxy"))
    else:
        k, se, sq, sp_ = _rates(None)
        res = ce.d3q19_steady(k, se, sp.Rational(7, 4), sq, sp_, sp.Rational(13, 10), sp.Rational(7, 4),
                              q_rows=("e", "eps", "pxx3", "pww", "pxy", "pyz", "pxz", "pixx3", "piww"))
    _, _, _, q_parts, q_div = res
    for qp, qd in zip(q_parts, q_div):
        assert sp.simplify(qp - qd) == 0
        assert qd != 0
