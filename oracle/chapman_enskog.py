"""Symbolic Chapman-Enskog checks of the collision coefficients (sympy).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Nothing here runs at run
time; tests/test_oracle_ce.py uses it to pin the coefficients of both oracles
against the conditions the paper states, by expanding the discrete scheme itself:

* Navier-Stokes level (main text Eqs. 7-9): with m1 the first-order
  non-equilibrium moments, S m1hat = -(D1 m_eq - F_m) with m1hat = m1 + F_m/2 and
  D1 = d_t1 + C . grad (C_a = M diag(c_ia) M^-1).  For rows coupled through
  S_rc = kappa_rc s_c omega_r (the form of Eq. 6) the recovered viscous stress is
  -Pi(v), v_r = -tau_r (A_r + sum_c kappa_rc A_c), A = D1 m_eq - F_m.  Terms are
  kept to first order in u and one gradient; d_t1 comes from the Euler equations.
* steady third order (main text after Eq. 14): at u = 0 the populations of a
  steady state satisfy (exp(c_i . grad) - 1) f_i = Omega_i; expanding f = f_eq + g
  in gradient order (F first order, Q_m second) and solving the non-conserved
  moments order by order leaves the momentum residual, written after replacing F
  by grad p_LBE in the third-order terms.

Gradients are commuting symbols; the fields rho, eta (with eta' = d eta / d rho)
and F are independent symbols.
"""
from __future__ import annotations

import sympy as sp

CS2 = sp.Rational(1, 3)


# --- lattices ---------------------------------------------------------------------

def d2q9():
    E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    n2 = lambda e: e[0] ** 2 + e[1] ** 2
    rows = [("rho", lambda e: 1), ("e", lambda e: 3 * n2(e) - 4),
            ("eps", lambda e: 4 - sp.Rational(21, 2) * n2(e) + sp.Rational(9, 2) * n2(e) ** 2),
            ("jx", lambda e: e[0]), ("qx", lambda e: (3 * n2(e) - 5) * e[0]),
            ("jy", lambda e: e[1]), ("qy", lambda e: (3 * n2(e) - 5) * e[1]),
            ("pxx", lambda e: e[0] ** 2 - e[1] ** 2), ("pxy", lambda e: e[0] * e[1])]
    W = [sp.Rational(4, 9)] + [sp.Rational(1, 9)] * 4 + [sp.Rational(1, 36)] * 4
    return 2, E, rows, W


def d3q19():
    E = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    E += [(a, b, 0) for a in (1, -1) for b in (1, -1)] + [(a, 0, b) for a in (1, -1) for b in (1, -1)]
    E += [(0, a, b) for a in (1, -1) for b in (1, -1)]
    n2 = lambda e: sum(c * c for c in e)
    rows = [("rho", lambda e: 1), ("e", lambda e: 19 * n2(e) - 30),
            ("eps", lambda e: (21 * n2(e) ** 2 - 53 * n2(e) + 24) / sp.Integer(2)),
            ("jx", lambda e: e[0]), ("qx", lambda e: (5 * n2(e) - 9) * e[0]),
            ("jy", lambda e: e[1]), ("qy", lambda e: (5 * n2(e) - 9) * e[1]),
            ("jz", lambda e: e[2]), ("qz", lambda e: (5 * n2(e) - 9) * e[2]),
            ("pxx3", lambda e: 3 * e[0] ** 2 - n2(e)), ("pixx3", lambda e: (3 * n2(e) - 5) * (3 * e[0] ** 2 - n2(e))),
            ("pww", lambda e: e[1] ** 2 - e[2] ** 2), ("piww", lambda e: (3 * n2(e) - 5) * (e[1] ** 2 - e[2] ** 2)),
            ("pxy", lambda e: e[0] * e[1]), ("pyz", lambda e: e[1] * e[2]), ("pxz", lambda e: e[0] * e[2]),
            ("mx", lambda e: (e[1] ** 2 - e[2] ** 2) * e[0]), ("my", lambda e: (e[2] ** 2 - e[0] ** 2) * e[1]),
            ("mz", lambda e: (e[0] ** 2 - e[1] ** 2) * e[2])]
    W = [sp.Rational(1, 3)] + [sp.Rational(1, 18)] * 6 + [sp.Rational(1, 36)] * 12
    return 3, E, rows, W


def moment_matrix(E, rows):
    return sp.Matrix([[fn(e) for e in E] for _, fn in rows])


def hermite_moments(E, W, M, rho, u, eta_row=None):
    """M f^H with the second-order Hermite equilibrium of the lattice."""
    D = len(u)
    uu = sum(x * x for x in u)
    f = []
    for e, w in zip(E, W):
        eu = sum(e[a] * u[a] for a in range(D))
        f.append(w * rho * (1 + 3 * eu + sp.Rational(9, 2) * eu ** 2 - sp.Rational(3, 2) * uu))
    return list(M * sp.Matrix(f))


def hermite_force_moments(E, W, M, u, F):
    D = len(u)
    uF = sum(u[a] * F[a] for a in range(D))
    f = []
    for e, w in zip(E, W):
        eu = sum(e[a] * u[a] for a in range(D))
        eF = sum(e[a] * F[a] for a in range(D))
        f.append(w * (3 * (eF - uF) + 9 * eu * eF))
    return list(M * sp.Matrix(f))


# --- Navier-Stokes level ----------------------------------------------------------------

def ns_residual(D, E, rows, meq_fn, fm_fn, tau, kappa, bulk):
    """Recovered viscous stress minus rho c_s^2 tau_p (grad u + grad u^T - (2/D) div u I)
    minus bulk * rho div u I, split by degree in u.  Returns {(a, b): {degree: expr}}
    for degrees 0 and 1 (the O(Ma) terms the coefficients must cancel)."""
    M = moment_matrix(E, rows)
    Minv = M.inv()
    names = [n for n, _ in rows]
    rho, eta, etap = sp.symbols("rho eta etap", positive=True)
    u = sp.symbols("ux uy uz")[:D]
    dr = sp.symbols("drx dry drz")[:D]
    F = sp.symbols("Fx Fy Fz")[:D]
    du = [[sp.Symbol("du_%s%s" % (a, b)) for b in "xyz"[:D]] for a in "xyz"[:D]]
    meq = sp.Matrix(meq_fn(rho, eta, u))
    fm = sp.Matrix(fm_fn(rho, u, F))

    def dspace(g, b):
        out = sp.diff(g, rho) * dr[b] + sp.diff(g, eta) * etap * dr[b]
        for c in range(D):
            out += sp.diff(g, u[c]) * du[c][b]
        return out

    rt = -(sum(u[a] * dr[a] for a in range(D)) + rho * sum(du[a][a] for a in range(D)))
    Pi0 = [[CS2 * (rho + eta) * (1 if a == b else 0) + rho * u[a] * u[b] for b in range(D)] for a in range(D)]
    ut = [(-sum(dspace(Pi0[a][b], b) for b in range(D)) + F[a] - u[a] * rt) / rho for a in range(D)]

    def dtime(g):
        out = sp.diff(g, rho) * rt + sp.diff(g, eta) * etap * rt
        for c in range(D):
            out += sp.diff(g, u[c]) * ut[c]
        return out

    f0 = Minv * meq
    A = []
    for k in range(len(rows)):
        val = dtime(meq[k])
        for a in range(D):
            flux = sum(M[k, i] * E[i][a] * f0[i] for i in range(len(E)))
            val += dspace(sp.expand(flux), a)
        A.append(sp.expand(val - fm[k]))
    v = [0] * len(rows)
    for r, name in enumerate(names):
        if name in tau:
            acc = A[r]
            for (rr, cc), kap in kappa.items():
                if rr == name:
                    acc += kap * A[names.index(cc)]
            v[r] = -tau[name] * acc
    vf = Minv * sp.Matrix(v)
    tp = tau["pxx3" if D == 3 else "pxx"]
    divu = sum(du[a][a] for a in range(D))
    out = {}
    for a in range(D):
        for b in range(D):
            sig = -sum(E[i][a] * E[i][b] * vf[i] for i in range(len(E)))
            newt = rho * CS2 * tp * (du[a][b] + du[b][a] - (sp.Rational(2, D) * divu if a == b else 0))
            rem = sp.expand(sig - newt - (bulk * rho * divu if a == b else 0))
            poly = sp.Poly(rem, *u)
            deg = {}
            for mon, coef in poly.terms():
                d = sum(mon)
                if d <= 1:
                    deg[d] = deg.get(d, 0) + coef * sp.prod([u[i] ** mon[i] for i in range(D)])
            out[(a, b)] = {d: sp.simplify(x) for d, x in deg.items()}
    return out, u


def d2q9_ns(varpi, k=None, h=None, b=None, beta2=None):
    """ns_residual for D2Q9 with the paper's m_eq (Eq. 3), F_m (Eq. 4) and S (Eq. 6);
    coefficients default to Eq. 7."""
    D, E, rows, W = d2q9()
    w = varpi
    k = 1 - w if k is None else k
    h = 6 * w * (1 - w) / (1 - 3 * w) if h is None else h
    b = (1 - w) / (1 - 3 * w) if b is None else b
    beta2 = -2 / (1 - w) if beta2 is None else beta2

    def meq(rho, eta, u):
        ux, uy = u
        U2 = ux ** 2 + uy ** 2
        return [rho, -2 * rho + 2 * eta + 3 * rho * U2, rho + beta2 * eta - 3 * rho * U2 + 9 * rho * ux ** 2 * uy ** 2,
                rho * ux, -rho * ux + 3 * rho * ux * uy ** 2, rho * uy, -rho * uy + 3 * rho * uy * ux ** 2,
                rho * (ux ** 2 - uy ** 2), rho * ux * uy]

    def fm(rho, u, F):
        ux, uy = u
        Fx, Fy = F
        Fu = Fx * ux + Fy * uy
        return [0, 6 * Fu, -6 * Fu + 9 * (2 * Fx * ux * uy ** 2 + 2 * Fy * uy * ux ** 2), Fx,
                -Fx + 3 * (Fx * uy ** 2 + 2 * Fy * ux * uy), Fy, -Fy + 3 * (Fy * ux ** 2 + 2 * Fx * ux * uy),
                2 * (Fx * ux - Fy * uy), Fx * uy + Fy * ux]

    te, tp = sp.symbols("tau_e tau_p")
    ux, uy = sp.symbols("ux uy")
    kappa = {("e", "eps"): k, ("e", "qx"): h * ux, ("e", "qy"): h * uy,
             ("pxx", "qx"): 2 * b * ux, ("pxx", "qy"): -2 * b * uy, ("pxy", "qx"): b * uy, ("pxy", "qy"): b * ux}
    return ns_residual(D, E, rows, meq, fm, {"e": te, "pxx": tp, "pxy": tp}, kappa, varpi * CS2 * te)[0]


def d3q19_ns(varpi, k, h, b, beta2):
    """ns_residual for the D3Q19 form: second-order Hermite m_eq with 19 eta in e and
    beta_2 eta in eps, Hermite forcing, S with the 3-D coupling pattern."""
    D, E, rows, W = d3q19()
    M = moment_matrix(E, rows)

    def meq(rho, eta, u):
        m = hermite_moments(E, W, M, rho, u)
        m[1] += 19 * eta
        m[2] += beta2 * eta
        return m

    def fm(rho, u, F):
        return hermite_force_moments(E, W, M, u, F)

    te, tp = sp.symbols("tau_e tau_p")
    ux, uy, uz = sp.symbols("ux uy uz")
    U = {"x": ux, "y": uy, "z": uz}
    q = {"x": "qx", "y": "qy", "z": "qz"}
    kappa = {("e", "eps"): k, ("e", "qx"): h * ux, ("e", "qy"): h * uy, ("e", "qz"): h * uz}

    def T(a, c):
        return {q[c]: U[a], q[a]: U[c]} if a != c else {q[a]: 2 * U[a]}

    def add(row, coeffs, scale):
        for col, val in coeffs.items():
            kappa[(row, col)] = kappa.get((row, col), 0) + scale * val

    add("pxx3", T("x", "x"), 2 * b); add("pxx3", T("y", "y"), -b); add("pxx3", T("z", "z"), -b)
    add("pww", T("y", "y"), b); add("pww", T("z", "z"), -b)
    add("pxy", T("x", "y"), b); add("pyz", T("y", "z"), b); add("pxz", T("x", "z"), b)
    tau = {"e": te, "pxx3": tp, "pww": tp, "pxy": tp, "pyz": tp, "pxz": tp}
    return ns_residual(D, E, rows, meq, fm, tau, kappa, varpi * sp.Rational(2, 3) * CS2 * te)[0]


# --- steady third order -----------------------------------------------------------------

def steady_eta_residual(D, E, rows, meq0, fm0, S, order=3, q_rows=()):
    """Momentum residual of a steady state at u = 0 through third order in the
    gradients, with F replaced by grad p_LBE (p_LBE = c_s^2 (rho + eta)) in the
    third-order terms, minus the lattice term -(1/12) c_s^2 lap grad(rho + eta).
    Returns the list of its eta parts (one per component) and of its rho parts.
    q_rows: moments that carry an independent second-order term Q_r of the collision's
    + S Q_m (symbol 'Q_<row>'); with them a third list holds the part linear in the
    Q symbols, and a fourth the divergence of the second-order tensor of Q_m,
    div Pi(M^-1 Q), for comparison."""
    lam = sp.Symbol("lam")
    n = len(E)
    d = sp.symbols("dx dy dz")[:D]
    M = moment_matrix(E, rows)
    Minv = M.inv()
    names = [nm for nm, _ in rows]
    js = ("jx", "jy", "jz")[:D]
    cons = [names.index("rho")] + [names.index(j) for j in js]
    noncons = [i for i in range(n) if i not in cons]

    def trunc(x):
        x = sp.expand(x)
        return sum(x.coeff(lam, k) * lam ** k for k in range(order + 1))

    shift = [sum((lam * sum(e[a] * d[a] for a in range(D))) ** p / sp.factorial(p) for p in range(1, order + 1))
             for e in E]
    F = sp.symbols("Fx Fy Fz")[:D]
    rho, eta = sp.symbols("rho eta")
    meq = sp.Matrix(meq0(rho, eta))
    fm = sp.Matrix([lam * x for x in fm0(F)])
    G = sp.zeros(n, 1)
    for a, j in enumerate(js):
        G[names.index(j)] = -lam * F[a] / 2
    Snn_inv = S.extract(noncons, noncons).inv()
    half = (sp.eye(n) - S / 2) * fm
    Qsym = {r: sp.Symbol("Q_" + r) for r in q_rows}
    Qm = sp.Matrix([lam ** 2 * Qsym[nm] if nm in Qsym else 0 for nm in names])
    SQ = S * Qm
    for _ in range(order + 1):
        fpop = Minv * (meq + G)
        mD = M * sp.Matrix([trunc(shift[i] * fpop[i]) for i in range(n)])
        Gn = Snn_inv * sp.Matrix([-mD[i] + half[i] + SQ[i] for i in noncons])
        for k, i in enumerate(noncons):
            G[i] = trunc(Gn[k])
    fpop = Minv * (meq + G)
    mD = M * sp.Matrix([trunc(shift[i] * fpop[i]) for i in range(n)])
    p0 = CS2 * (rho + eta)
    lap = sum(x * x for x in d)
    eta_parts, rho_parts, q_parts, q_div = [], [], [], []
    qv = Minv * sp.Matrix([Qsym[nm] if nm in Qsym else 0 for nm in names])  # M^-1 Q in velocity space
    Pi_Q = [[sum(E[i][a] * E[i][b] * qv[i] for i in range(n)) for b in range(D)] for a in range(D)]
    for a, j in enumerate(js):
        r3 = sp.expand(mD[names.index(j)]).coeff(lam, 3)
        canon = sp.expand(r3.subs({F[b]: d[b] * p0 for b in range(D)}) + sp.Rational(1, 12) * lap * d[a] * p0)
        eta_parts.append(sp.factor(canon.coeff(eta)))
        rho_parts.append(sp.factor(canon.coeff(rho)))
        if Qsym:
            q_parts.append(sp.expand(sum(canon.coeff(q) * q for q in Qsym.values())))
            q_div.append(sp.expand(sum(d[b] * Pi_Q[a][b] for b in range(D))))
    if Qsym:
        return eta_parts, rho_parts, d, q_parts, q_div
    return eta_parts, rho_parts, d


def d2q9_steady(varpi, se, seps, sq, sp_, q_rows=()):
    D, E, rows, W = d2q9()
    k = 1 - varpi
    beta2 = -2 / (1 - varpi)
    S = sp.diag(1, se, seps, 1, sq, 1, sq, sp_, sp_)
    S[1, 2] = k * seps * (se / 2 - 1)
    meq0 = lambda rho, eta: [rho, -2 * rho + 2 * eta, rho + beta2 * eta, 0, 0, 0, 0, 0, 0]
    fm0 = lambda F: [0, 0, 0, F[0], -F[0], F[1], -F[1], 0, 0]
    return steady_eta_residual(D, E, rows, meq0, fm0, S, q_rows=q_rows)


def d3q19_steady(k, se, seps, sq, sp_, sm, spi, q_rows=()):
    D, E, rows, W = d3q19()
    names = [nm for nm, _ in rows]
    beta2 = -19 / k
    rate = {"rho": 1, "e": se, "eps": seps, "jx": 1, "jy": 1, "jz": 1, "qx": sq, "qy": sq, "qz": sq,
            "pxx3": sp_, "pww": sp_, "pxy": sp_, "pyz": sp_, "pxz": sp_, "pixx3": spi, "piww": spi,
            "mx": sm, "my": sm, "mz": sm}
    S = sp.diag(*[rate[nm] for nm in names])
    S[1, 2] = k * seps * (se / 2 - 1)

    def meq0(rho, eta):
        m = [0] * 19
        m[0], m[1], m[2] = rho, -11 * rho + 19 * eta, 3 * rho + beta2 * eta
        return m

    def fm0(F):
        m = [0] * 19
        for a, (j, q) in enumerate((("jx", "qx"), ("jy", "qy"), ("jz", "qz"))):
            m[names.index(j)] = F[a]
            m[names.index(q)] = -sp.Rational(2, 3) * F[a]
        return m

    return steady_eta_residual(D, E, rows, meq0, fm0, S, q_rows=q_rows)
