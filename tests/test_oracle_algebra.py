"""Pins of the oracle's transcribed algebra against what the paper and the
mathematics fix independently of the oracle (CPU only)."""
import math

import numpy as np
import pytest

from oracle import params as op

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

RNG = np.random.default_rng(1234)


def lattice_velocities():
    """Supplement Eq. 3 evaluated from its trigonometric definition (c = 1)."""
    e = [(0.0, 0.0)]
    for i in range(1, 5):
        e.append((math.cos((i - 1) * math.pi / 2), math.sin((i - 1) * math.pi / 2)))
    for i in range(5, 9):
        a = (2 * i - 1) * math.pi / 4
        e.append((math.sqrt(2) * math.cos(a), math.sqrt(2) * math.sin(a)))
    return np.rint(np.array(e)).astype(int)


def test_velocity_set_matches_eq3(orc):
    ex, ey = orc.velocities()
    e = lattice_velocities()
    assert np.array_equal(ex, e[:, 0]) and np.array_equal(ey, e[:, 1])


def test_moment_matrix_from_polynomials(orc):
    """Rows of M are the Lallemand-Luo moments 1, -4+3|e|^2, 4-21/2|e|^2+9/2|e|^4,
    e_x, (-5+3|e|^2)e_x, e_y, (-5+3|e|^2)e_y, e_x^2-e_y^2, e_x e_y."""
    e = lattice_velocities().astype(float)
    ex, ey = e[:, 0], e[:, 1]
    e2 = ex ** 2 + ey ** 2
    rows = [np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, ex, (-5 + 3 * e2) * ex, ey,
            (-5 + 3 * e2) * ey, ex ** 2 - ey ** 2, ex * ey]
    assert np.array_equal(orc.matrix_M(), np.array(rows))


def test_moment_matrix_orthogonal_and_inverse(orc):
    M, Mi = orc.matrix_M(), orc.matrix_Minv()
    assert np.array_equal(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))
    assert np.abs(Mi @ M - np.eye(9)).max() < 1e-15
    # M^-1 = M^T diag(1/9, 1/36, ...) follows from the orthogonality.
    assert np.abs(Mi - M.T @ np.diag(1 / np.diag(M @ M.T))).max() < 1e-16


def _par(varpi=1.0 / 6.0, **kw):
    p = op.from_physical(varpi=varpi, **kw).as_dict()
    return p


@pytest.mark.parametrize("varpi", [1.0 / 6.0, 0.1, 0.25, 0.5, 0.8])
def test_collision_matrix_times_printed_inverse(orc, varpi):
    """S (Eq. 6) times the inverse printed in supplement Eq. 46 is the identity."""
    p = _par(varpi=varpi)
    k = 1 - varpi
    h = 6 * varpi * (1 - varpi) / (1 - 3 * varpi)
    b = (1 - varpi) / (1 - 3 * varpi)
    se, seps, sq, sp, s0, sj = p["se"], 1.17, p["sq"], p["sp"], 0.9, 1.1
    p.update(seps=seps, s0=s0, sj=sj)
    for ux, uy in [(0.1, -0.07), (-0.03, 0.2), (0.0, 0.0)]:
        S, _, _, _ = orc.matrices(p, ux, uy)
        Si = np.diag([1 / s0, 1 / se, 1 / seps, 1 / sj, 1 / sq, 1 / sj, 1 / sq, 1 / sp, 1 / sp])
        Si[1, 2] = k * (1 / se - 0.5)
        Si[1, 4] = h * ux * (1 / se - 0.5)
        Si[1, 6] = h * uy * (1 / se - 0.5)
        Si[7, 4] = 2 * b * ux * (1 / sp - 0.5)
        Si[7, 6] = -2 * b * uy * (1 / sp - 0.5)
        Si[8, 4] = b * uy * (1 / sp - 0.5)
        Si[8, 6] = b * ux * (1 / sp - 0.5)
        assert np.abs(S @ Si - np.eye(9)).max() < 1e-14


@pytest.mark.parametrize("varpi", [1.0 / 6.0, 0.1, 0.25, 0.5, 0.8])
def test_coefficients_satisfy_ce_constraints(orc, varpi):
    """k, h, b (read back from S) and alpha_2, beta_2 (read back from m_eq) satisfy the
    Chapman-Enskog constraints of supplement Eqs. 24, 27 and 30."""
    p = _par(varpi=varpi)
    ux, uy = 0.13, -0.21
    S, _, _, _ = orc.matrices(p, ux, uy)
    om_e, om_p = p["se"] / 2 - 1, p["sp"] / 2 - 1
    k = S[1, 2] / (p["seps"] * om_e)
    h = S[1, 4] / (ux * p["sq"] * om_e)
    b = S[8, 4] / (uy * p["sq"] * om_p)
    assert S[1, 6] == pytest.approx(h * uy * p["sq"] * om_e, rel=1e-14)
    assert S[7, 4] == pytest.approx(2 * b * ux * p["sq"] * om_p, rel=1e-14)
    assert S[7, 6] == pytest.approx(-2 * b * uy * p["sq"] * om_p, rel=1e-14)
    assert S[8, 6] == pytest.approx(b * ux * p["sq"] * om_p, rel=1e-14)
    a1 = orc.moments_eq(p, 1.0, 0.0, 0.0, 0.0)[1] / 2
    b1 = orc.moments_eq(p, 0.0, 1.0, 0.0, 0.0)[1] / 2
    a2 = orc.moments_eq(p, 1.0, 0.0, 0.0, 0.0)[2]
    b2 = orc.moments_eq(p, 0.0, 1.0, 0.0, 0.0)[2]
    assert (a1, b1) == (-1.0, 1.0)
    w = varpi
    # Eq. 24
    assert 2 * a1 + k * a2 + k == pytest.approx(-2 * w, abs=1e-14)
    assert h * ((a2 - 4) * b1 - (a1 + 2) * b2) / (3 * b1) == pytest.approx(-2 * w, abs=1e-13)
    assert (h * (3 * b1 + b2) - 6 * b1 * (1 - k)) / b1 == pytest.approx(0, abs=1e-13)
    assert 2 * b1 + k * b2 == pytest.approx(0, abs=1e-14)
    # Eq. 27 and Eq. 30
    assert b * ((a2 - 4) * b1 - (a1 + 2) * b2) / b1 == pytest.approx(-1, abs=1e-13)
    assert ((6 * b - 2) * b1 + 2 * b * b2) / b1 == pytest.approx(0, abs=1e-13)
    assert ((3 * b - 1) * b1 + b * b2) / b1 == pytest.approx(0, abs=1e-13)


def test_equilibrium_is_product_maxwellian_for_ideal_gas(orc):
    """With eta = 0 the equilibrium moments of Eq. 3 are M applied to the D2Q9
    product-form equilibrium rho w(e_x, u_x) w(e_y, u_y), w(0,u) = 2/3 - u^2,
    w(+-1,u) = (1 +- 3u + 3u^2)/6 (the discrete Maxwellian with full Hermite terms)."""
    p = _par()
    e = lattice_velocities()
    M = orc.matrix_M()

    def w(c, u):
        return 2 / 3 - u * u if c == 0 else (1 + 3 * c * u + 3 * u * u) / 6

    for rho, ux, uy in [(1.3, 0.1, -0.2), (0.7, -0.05, 0.03), (2.0, 0.0, 0.15)]:
        feq = np.array([rho * w(e[i, 0], ux) * w(e[i, 1], uy) for i in range(9)])
        assert np.abs(orc.moments_eq(p, rho, 0.0, ux, uy) - M @ feq).max() < 1e-14


def test_force_moments_are_hermite_derivative_of_equilibrium(orc):
    """F_m of Eq. 4 with the bracket read as the sum over the force's positions
    equals the derivative of m_eq along the momentum change F (rho, eta fixed)."""
    p = _par()
    for _ in range(20):
        rho, eta = RNG.uniform(0.5, 3), RNG.uniform(-1, 1)
        ux, uy, Fx, Fy = RNG.uniform(-0.2, 0.2, 4)
        h = 1e-5
        dm = (orc.moments_eq(p, rho, eta, ux + h * Fx / rho, uy + h * Fy / rho)
              - orc.moments_eq(p, rho, eta, ux - h * Fx / rho, uy - h * Fy / rho)) / (2 * h)
        assert np.abs(orc.moments_force(Fx, Fy, ux, uy) - dm).max() < 1e-9


def _sequence_collision(orc, p, f, Sx, Sy):
    """Collision by the execution sequence (1)-(6) of supplement Sec. IV, written
    independently of the matrix form the oracle evaluates."""
    M, Mi = orc.matrix_M(), orc.matrix_Minv()
    ex, ey = orc.velocities()
    rho = f.sum()
    Fx, Fy = p["G2"] * rho * Sx, p["G2"] * rho * Sy
    ux = (ex @ f + Fx / 2) / rho
    uy = (ey @ f + Fy / 2) / rho
    pe, dpe = orc.eos(p, rho)
    eta = 3 * (pe + p["G2"] * rho * rho / 2) - rho
    gp = (dpe + p["G2"] * rho) * np.array([Sx, Sy])
    grho = np.array([Sx, Sy])
    w = p["varpi"]
    k, h, b = 1 - w, 6 * w * (1 - w) / (1 - 3 * w), (1 - w) / (1 - 3 * w)
    se, seps, sq, sp = p["se"], p["seps"], p["sq"], p["sp"]
    diagS = np.array([p["s0"], se, seps, p["sj"], sq, p["sj"], sq, sp, sp])
    meq = orc.moments_eq(p, rho, eta, ux, uy)
    Fm = orc.moments_force(Fx, Fy, ux, uy)
    Q = orc.moments_Q(p, Sx, Sy)
    _, Rm, T, X = orc.matrices(p, ux, uy)
    m = M @ f
    # (1)
    mb = m.copy()
    m = m - meq
    mb = mb - 2 * m
    m = m + Fm / 2
    # (2)
    m1 = m[1] + 0.5 * k * seps * m[2] + 0.5 * h * sq * (ux * m[4] + uy * m[6])
    m7 = m[7] + b * sq * (ux * m[4] - uy * m[6])
    m8 = m[8] + 0.5 * b * sq * (uy * m[4] + ux * m[6])
    m[1], m[7], m[8] = m1, m7, m8
    # (3)
    m = (1 - diagS / 2) * m
    # (4)
    for r in (1, 7, 8):
        mb[r] -= Rm[r, 1] * m[1] + Rm[r, 7] * m[7] + Rm[r, 8] * m[8] + T[r] @ grho + X[r] @ gp
    # (5)
    mb = mb + 2 * m
    # (6)
    mb[1] += se * Q[1] + k * (0.5 * se - 1) * seps * Q[2]
    mb[2] += seps * Q[2]
    mb[7] += sp * Q[7]
    mb[8] += sp * Q[8]
    return Mi @ mb


@pytest.mark.parametrize("varpi", [1.0 / 6.0, 0.25])
def test_matrix_form_equals_execution_sequence(orc, varpi):
    p = _par(varpi=varpi)
    p.update(seps=1.1, s0=0.8, sj=1.2)
    for _ in range(30):
        rho = RNG.uniform(1.0, 6.0)
        f = rho * np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4) * (1 + 0.2 * RNG.uniform(-1, 1, 9))
        Sx, Sy = RNG.uniform(-0.3, 0.3, 2)
        ref = _sequence_collision(orc, p, f, Sx, Sy)
        out = orc.collide_node(p, f, Sx, Sy)
        assert np.abs(out - ref).max() < 1e-13 * np.abs(ref).max()


def test_cubic_correction_entries_cancel_their_targets(orc):
    """R, T, X rows reproduce the cubic velocity terms they must cancel
    (supplement Eqs. 33, 36, 39 with the leading order of Eq. 32): e.g. row 1's
    R-part equals the decomposition of the u-u-grad(u) terms of Eq. 33."""
    p = _par()
    w = p["varpi"]
    k, h, b = 1 - w, 6 * w * (1 - w) / (1 - 3 * w), (1 - w) / (1 - 3 * w)
    se, sp = p["se"], p["sp"]
    for ux, uy in [(0.1, 0.05), (-0.07, 0.12)]:
        _, Rm, T, X = orc.matrices(p, ux, uy)
        # Linear map: (div u, dxux - dyuy, dxuy + dyux) -> G-hat (Eq. 32, dt = 1, rho = 1).
        g1 = lambda d: -d * (2 - se) / (2 * se) * 2 * w
        g7 = lambda d: -d * (2 - sp) / (2 * sp) * 2 / 3
        g8 = lambda d: -d * (2 - sp) / (2 * sp) / 3
        # Random velocity-gradient tensor.
        A = RNG.uniform(-1, 1, (2, 2))
        dxux, dxuy, dyux, dyuy = A[0, 0], A[0, 1], A[1, 0], A[1, 1]
        G1, G7, G8 = g1(dxux + dyuy), g7(dxux - dyuy), g8(dxuy + dyux)
        # Row 1 (Eq. 33): 2/(2-se) (R11 G1 + R17 G7 + R18 G8) must equal the cubic terms.
        cub1 = ((9 * (1 - k) * ux ** 2 - 2 * (3 * k + h) * uy ** 2) * dxux
                + (9 * (1 - k) * uy ** 2 - 2 * (3 * k + h) * ux ** 2) * dyuy
                - 4 * (3 * k + h) * ux * uy * (dxuy + dyux))
        assert 2 / (2 - se) * (Rm[1, 1] * G1 + Rm[1, 7] * G7 + Rm[1, 8] * G8) == pytest.approx(cub1, rel=1e-12)
        # Row 7 (Eq. 36)
        cub7 = (3 * ux ** 2 + 4 * b * uy ** 2) * dxux - (3 * uy ** 2 + 4 * b * ux ** 2) * dyuy
        assert 2 / (2 - sp) * (Rm[7, 1] * G1 + Rm[7, 7] * G7 + Rm[7, 8] * G8) == pytest.approx(cub7, rel=1e-12)
        # Row 8 (Eq. 39)
        cub8 = -(2 * b * ux * uy * (dxux + dyuy) + 2 * b * (ux ** 2 + uy ** 2) * (dxuy + dyux))
        assert 2 / (2 - sp) * (Rm[8, 1] * G1 + Rm[8, 7] * G7 + Rm[8, 8] * G8) == pytest.approx(cub8, rel=1e-12)
        # Gradient rows: 2/(2-s) (T . grad rho + X . grad p) equals the grad rho / grad p terms.
        gr, gp = RNG.uniform(-1, 1, 2), RNG.uniform(-1, 1, 2)
        t1 = (3 * ((1 - k) * ux ** 3 - (2 * k + h) * ux * uy ** 2) * gr[0]
              + 3 * ((1 - k) * uy ** 3 - (2 * k + h) * ux ** 2 * uy) * gr[1]
              + 9 * (2 * k + h) * (ux * uy ** 2 * gp[0] + ux ** 2 * uy * gp[1]))
        assert 2 / (2 - se) * (T[1] @ gr + X[1] @ gp) == pytest.approx(t1, rel=1e-12)
        t7 = ((ux ** 3 + 2 * b * ux * uy ** 2) * gr[0] - (uy ** 3 + 2 * b * ux ** 2 * uy) * gr[1]
              - 6 * b * ux * uy ** 2 * gp[0] + 6 * b * ux ** 2 * uy * gp[1])
        assert 2 / (2 - sp) * (T[7] @ gr + X[7] @ gp) == pytest.approx(t7, rel=1e-12)
        t8 = (-b * (uy ** 3 + 2 * ux ** 2 * uy) * gr[0] - b * (ux ** 3 + 2 * ux * uy ** 2) * gr[1]
              + 3 * b * (uy ** 3 + 2 * ux ** 2 * uy) * gp[0] + 3 * b * (ux ** 3 + 2 * ux * uy ** 2) * gp[1])
        assert 2 / (2 - sp) * (T[8] @ gr + X[8] @ gp) == pytest.approx(t8, rel=1e-12)
        # Rows that must stay zero (conserved moments and the non-corrected ones).
        for r in (0, 2, 3, 4, 5, 6):
            assert not Rm[r].any() and not T[r].any() and not X[r].any()


def test_force_stencil_closed_form(orc):
    """Eq. 12's stencil on rho = cos(k.x): S_x = -2 sin(phi) [sin(kx)/3 + sin(kx) cos(ky)/6]."""
    nx, ny = 24, 18
    kx, ky = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    y, x = np.mgrid[0:ny, 0:nx]
    phi = kx * x + ky * y
    sx, sy = orc.force_stencil(np.cos(phi))
    ex = -2 * np.sin(phi) * (np.sin(kx) / 3 + np.sin(kx) * np.cos(ky) / 6)
    ey = -2 * np.sin(phi) * (np.sin(ky) / 3 + np.sin(ky) * np.cos(kx) / 6)
    assert np.abs(sx - ex).max() < 1e-14 and np.abs(sy - ey).max() < 1e-14
    # Isotropy: sum_i w_i e_i e_i = I, so a long wave gives grad(rho) to O(k^3).
    k = 2 * np.pi / 400
    sx, _ = orc.force_stencil(np.cos(k * np.mgrid[0:4, 0:400][1]))
    assert np.abs(sx[0] + k * np.sin(k * np.arange(400))).max() < k ** 3


@pytest.mark.parametrize("kind,code", [("vdw", 0), ("cs", 1)])
def test_eos_derivative_and_critical_point(orc, kind, code):
    """dp/drho of the oracle's EOS matches a central difference of its p, and at
    T = Tc the isotherm has an inflection with zero slope (critical point)."""
    from oracle import thermo

    a, b = (9 / 49, 2 / 21) if kind == "vdw" else (1.0, 4.0)
    Tc = thermo.critical_temperature(kind, a, b, 1.0)
    p = dict(_par(), eos=code, eos_a=a, eos_b=b, R_gas=1.0, T=Tc, lam=1.0)
    rmax = 1 / b if kind == "vdw" else 4 / b
    for rho in np.linspace(0.05, 0.8, 7) * rmax:
        hh = 1e-6 * rho
        dfd = (orc.eos(p, rho + hh)[0] - orc.eos(p, rho - hh)[0]) / (2 * hh)
        assert orc.eos(p, rho)[1] == pytest.approx(dfd, rel=1e-7)
    grid = np.linspace(0.05, 0.9, 20001) * rmax
    d = np.array([orc.eos(p, r)[1] for r in grid])
    if kind == "vdw":
        # Exact: rho_c = 1/(3b), p_c = a/(27 b^2).
        assert orc.eos(p, 1 / (3 * b))[1] == pytest.approx(0.0, abs=1e-14)
        assert orc.eos(p, 1 / (3 * b))[0] == pytest.approx(a / (27 * b * b), rel=1e-14)
    # Zero minimum slope on the critical isotherm; the six-digit constants of
    # Eq. 20 make the CS critical point exact to ~1e-5 of R Tc.
    assert abs(d.min()) < 2e-5 * Tc
