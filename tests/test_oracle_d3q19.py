"""Pins of the D3Q19 oracle (the three-dimensional form of the model): the lattice
and its moments, the equilibrium, force and Q_m moments against their defining
sums, invariants, the BGK special case, and the physics the 3-D coefficients are
derived to give (Newtonian viscous stress with the bulk viscosity of Eq. 7, the
pressure tensor of Eq. 17, Galilean invariance of the interface stresses).  Each
physics pin is paired with a planted mistake that it detects."""
import numpy as np
import pytest

from oracle import params as op
from oracle import thermo
from paper_1809_02390_gb300 import inputs

RNG = np.random.default_rng(11)
VDW = dict(eos="vdw", a=9 / 49, b=2 / 21)


@pytest.fixture(scope="module")
def o3():
    from oracle import d3q19

    d3q19.build()
    return d3q19


def test_lattice_weights_and_isotropy(o3):
    """D3Q19 weights and velocity moments: sum w = 1, sum w e e = I/3 and the fourth
    moment is (1/9)(d d + d d + d d) (the isotropy the force weights and the
    pressure-tensor derivation rely on)."""
    e, w = o3.velocities(), o3.weights()
    assert e.shape == (3, 19) and sorted(map(tuple, e.T)) == sorted(set(map(tuple, e.T)))
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    d = np.eye(3)
    assert np.allclose(np.einsum("i,ai,bi->ab", w, e, e), d / 3, atol=1e-15)
    m4 = np.einsum("i,ai,bi,ci,di->abcd", w, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-15)
    assert np.allclose(np.einsum("i,ai,bi,ci->abc", w, e, e, e), 0.0)


def test_moment_matrix_is_orthogonal(o3):
    """Orthogonal moments without weights (as in Eq. 2): M M^T is diagonal with the
    row norms of the D3Q19 polynomial set, and M^-1 M = I."""
    M, Mi = o3.matrix_M(), o3.matrix_Minv()
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0
    assert np.allclose(np.diag(G), [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8])
    assert np.abs(Mi @ M - np.eye(19)).max() < 1e-15
    e = o3.velocities()
    assert np.array_equal(M[3], e[0]) and np.array_equal(M[5], e[1]) and np.array_equal(M[7], e[2])


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.05, -0.03, 0.02)])
def test_equilibrium_carries_the_self_tuning_pressure(o3, u):
    """f_eq = M^-1 m_eq(rho, eta, u) has mass rho, momentum rho u and second moment
    c_s^2 (rho + eta) I + rho u u: p_LBE = c_s^2 (rho + eta) (Eq. 9 with alpha_1 = -1,
    beta_1 = 1) in 3-D."""
    p = op.from_physical_3d(Tr=0.8)
    rho, eta = 2.3, -0.71
    f = o3.matrix_Minv() @ o3.moments_eq(p, rho, eta, u)
    e = o3.velocities()
    u = np.array(u)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    assert np.allclose(e @ f, rho * u, atol=1e-14)
    Pi = np.einsum("ai,bi,i->ab", e, e, f)
    assert np.allclose(Pi, (rho + eta) / 3 * np.eye(3) + rho * np.outer(u, u), atol=1e-13)


def test_force_and_q_moments_are_what_they_define(o3):
    """F_m = M F_v with zeroth, first and second moments 0, F and u F + F u; Q_m = M g
    with no mass and the second-order tensor (2 F~F~ + |F~|^2 I)/24 of Eq. 14
    (F~ = G s, c = 1)."""
    p = op.from_physical_3d(Tr=0.8)
    e, Mi = o3.velocities(), o3.matrix_Minv()
    F, u = np.array([0.013, -0.007, 0.004]), np.array([0.04, 0.01, -0.02])
    fv = Mi @ o3.moments_force(F, u)
    assert abs(fv.sum()) < 1e-16 and np.allclose(e @ fv, F, atol=1e-16)
    assert np.allclose(np.einsum("ai,bi,i->ab", e, e, fv), np.outer(u, F) + np.outer(F, u), atol=1e-16)
    s = np.array([0.21, -0.09, 0.05])
    g = Mi @ o3.moments_Q(p, s)
    Ft = np.sqrt(p.G2) * s
    assert abs(g.sum()) < 1e-16 and np.allclose(e @ g, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("ai,bi,i->ab", e, e, g), (2 * np.outer(Ft, Ft) + Ft @ Ft * np.eye(3)) / 24,
                       atol=1e-16)


def test_coefficients_and_rates_by_hand(o3):
    """The 3-D counterparts of Eq. 7 and Eq. 16 worked by hand at varpi = 1/6, s_p = 1:
    k = 38 (5/6)/11 = 95/33, beta_2 = -19/k = -33/5, b = 21 (5/6)/(5 * 4) = 7/8,
    h = 798 (1/6)(5/6)/(5 * 4) = 133/24; tau_p = 1/2, tau_q = 1/6, 1 + 5k/19 = 58/33,
    tau_e = 1/(12 (58/33)(1/6)) = 33/116, so s_q = 3/2 and s_e = 116/91."""
    p = op.from_physical_3d(Tr=0.8)
    c = o3.coefficients(p)
    assert c["k"] == pytest.approx(95 / 33, rel=1e-15) and c["beta2"] == pytest.approx(-33 / 5, rel=1e-15)
    assert c["b"] == pytest.approx(7 / 8, rel=1e-15) and c["h"] == pytest.approx(133 / 24, rel=1e-15)
    assert p.sq == pytest.approx(3 / 2, rel=1e-15) and p.se == pytest.approx(116 / 91, rel=1e-15)
    assert p.sm == p.sq and p.spi == p.seps == op.S_EPS_3D


def _amplification(o3, p, rho0, k):
    """Largest |eigenvalue| of the one-step map of a small perturbation
    exp(i k.x) of the uniform fluid at rest (Jacobians of the node collision by
    central differences, pull streaming as the phase exp(-i k.e_i), the force
    stencil as i sum_j omega_j sin(k.e_j) e_j times the density perturbation)."""
    e = o3.velocities()
    n2 = (e ** 2).sum(0)
    om = np.where(n2 == 1, 1 / 6, np.where(n2 == 2, 1 / 12, 0.0))
    f0 = o3.init_eq(p, np.full((1, 1, 1), rho0))[:, 0, 0, 0]
    h, s0, I19, I3 = 1e-7, np.zeros(3), np.eye(19), np.eye(3)
    C = lambda f, s: o3.collide_node(p, f, s)
    Jf = np.stack([(C(f0 + h * I19[i], s0) - C(f0 - h * I19[i], s0)) / (2 * h) for i in range(19)], 1)
    Js = np.stack([(C(f0, s0 + h * I3[a]) - C(f0, s0 - h * I3[a])) / (2 * h) for a in range(3)], 1)
    P = np.diag(np.exp(-1j * (k @ e)))
    g = 1j * (om * np.sin(k @ e) * e).sum(1)
    A = Jf @ P + np.outer(Js @ g, np.ones(19)) @ P
    return np.abs(np.linalg.eigvals(A)).max()


@pytest.mark.parametrize("s_eps", [None, "s_e"])
def test_checkerboard_mode_of_the_uniform_gas(o3, s_eps):
    """The free rates s_eps and s_pi decide the linear stability of the e-eps block at
    k = (pi, pi, pi), a mode that only a lattice varying in all three directions has.
    With s_eps = s_pi = 1.75 the uniform gas and liquid (Tr = 0.8) do not amplify it,
    nor any other sampled wave vector; with s_eps = s_e, the 2-D choice, the gas
    amplifies it by 1.26 per step (a 3-D droplet or spinodal run then diverges within
    100 steps)."""
    kw = {} if s_eps is None else dict(s_eps=op.relaxation_rates_3d(1.0, 1 / 6)[1])
    p = op.from_physical_3d(Tr=0.8, **kw)
    corner = np.pi * np.ones(3)
    if s_eps is None:
        ks = [corner] + [t * corner for t in (0.3, 0.6)] + [RNG.uniform(-np.pi, np.pi, 3) for _ in range(25)]
        for rho0 in (p.rho_g, p.rho_l):
            assert max(_amplification(o3, p, rho0, k) for k in ks) < 1.0
    else:
        assert _amplification(o3, p, p.rho_g, corner) > 1.2


def test_rest_state_is_a_fixed_point(o3):
    p = op.from_physical_3d(Tr=0.8)
    f0 = o3.init_eq(p, np.full((4, 5, 6), p.rho_l))
    assert np.abs(o3.step(p, f0, 500) - f0).max() <= 1e-13 * np.abs(f0).max()


def test_mass_and_momentum_conservation(o3):
    """Collision rows rho and j act on zero and the pairwise force sums to zero on a
    periodic lattice: total mass and total momentum are invariants."""
    p = op.from_physical_3d(Tr=0.8)
    nz, ny, nx = 8, 10, 12
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    r = np.sqrt((x - 5.3) ** 2 + (y - 4.6) ** 2 + (z - 3.9) ** 2)
    rho = 0.5 * (p.rho_g + p.rho_l) - 0.5 * (p.rho_l - p.rho_g) * np.tanh(2 * (r - 3.5) / 4.0)
    u = [RNG.uniform(-0.02, 0.02, rho.shape) for _ in range(3)]
    f = o3.init_eq(p, rho, *u)
    e = o3.velocities()
    mass0, j0 = f.sum(), np.tensordot(e, f, 1).sum(axis=(1, 2, 3))
    f = o3.step(p, f, 150)
    assert abs(f.sum() - mass0) <= 1e-13 * mass0
    assert np.abs(np.tensordot(e, f, 1).sum(axis=(1, 2, 3)) - j0).max() <= 1e-12 * mass0
    assert np.abs(j0).max() > 1e-3


def test_classical_limit_is_d3q19_bgk(o3):
    """varpi = 1 (k = h = b = beta_2 = 0) with eta = 0 (ideal gas), no force and one
    relaxation rate: the model is D3Q19 BGK with the second-order Hermite equilibrium,
    written out here with numpy rolls."""
    om = 1.3
    p = dict(eos=2, form=2, eos_a=0.0, eos_b=0.0, R_gas=1.0, T=1.0, lam=1.0, G2=0.0, varpi=1.0,
             s0=om, se=om, seps=om, sj=om, sq=om, sp=om, sm=om, spi=om)
    e, w = o3.velocities(), o3.weights()
    nz, ny, nx = 4, 5, 6
    f = w[:, None, None, None] * (1 + 0.1 * RNG.uniform(-1, 1, (19, nz, ny, nx)))
    ref = f.copy()
    for _ in range(12):
        g = np.stack([np.roll(ref[i], (e[2, i], e[1, i], e[0, i]), (0, 1, 2)) for i in range(19)])
        rho = g.sum(0)
        u = np.tensordot(e, g, 1) / rho
        uu = (u * u).sum(0)
        eu = np.tensordot(e.T, u, 1)
        feq = w[:, None, None, None] * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * uu)
        ref = g - om * (g - feq)
    assert np.abs(o3.step(p, f, 12) - ref).max() < 1e-14


def _shear_nu(o3, p, U, along, L=32, amp=1e-3, n=200):
    """Decay rate of the shear wave u_y = amp sin(k x) on a background U along x
    (the wave vector) or z (across it), lattice L x 2 x 1."""
    k = 2 * np.pi / L
    x = np.arange(L)[None, None, :] * np.ones((1, 2, 1))
    ux = np.full(x.shape, U if along else 0.0)
    uz = np.full(x.shape, 0.0 if along else U)
    f = o3.init_eq(p, np.full(x.shape, p.rho_l), ux, amp * np.sin(k * x), uz)
    phase = np.exp(-2j * np.pi * x / L)
    amp_of = lambda f: abs(np.sum(o3.macro(p, f)[2] * phase))
    f = o3.step(p, f, 20)
    a1 = amp_of(f)
    return -np.log(amp_of(o3.step(p, f, n)) / a1) / (k * k * n)


def test_shear_viscosity_and_its_galilean_shift(o3):
    """nu = c_s^2 (1/s_p - 1/2) (Eq. 9; finite-k correction < 1%).  A background flow
    across the wave vector leaves it unchanged; along the wave vector it shifts it by
    O(U^2) (the 3-D model has no cubic correction R, T, X: measured 0.5% at U = 0.06)."""
    p = op.from_physical_3d(Tr=0.85)
    nu0 = _shear_nu(o3, p, 0.0, True)
    assert nu0 == pytest.approx((1 / p.sp - 0.5) / 3, rel=1e-2)
    assert abs(_shear_nu(o3, p, 0.06, False) / nu0 - 1) < 1e-6
    shift = _shear_nu(o3, p, 0.06, True) / nu0 - 1
    assert 0 < shift < 1e-2
    assert _shear_nu(o3, p, 0.03, True) / nu0 - 1 == pytest.approx(shift / 4, rel=0.1)


def _sound(o3, p, L=64, amp=1e-5, n=1500, every=5):
    """(damping rate / k^2, phase speed) of a standing sound wave in the liquid."""
    from scipy.optimize import curve_fit

    x = np.arange(L)[None, None, :]
    k = 2 * np.pi / L
    f = o3.init_eq(p, p.rho_l * (1 + amp * np.cos(k * x)))
    A = []
    for _ in range(0, n, every):
        A.append((o3.macro(p, f)[0][0, 0] * np.cos(k * x[0, 0])).sum())
        f = o3.step(p, f, every)
    t = np.arange(len(A)) * every
    fn = lambda t, a, G, w, ph: a * np.exp(-G * t) * np.cos(w * t + ph)
    popt, _ = curve_fit(fn, t, np.array(A), p0=(A[0], 1e-3, k / np.sqrt(3), 0.0))
    return popt[1] / k ** 2, popt[2] / k


@pytest.mark.parametrize("varpi", [1 / 6, 0.3])
def test_bulk_viscosity_and_sound_speed(o3, orc, varpi):
    """Sound in the non-ideal liquid: the damping 2 Gamma / k^2 = (4/3) nu + zeta with
    the 3-D bulk viscosity zeta = varpi (2/3) c_s^2 (1/s_e - 1/2), and the speed
    sqrt(dp_EOS/drho) (the interaction force turns p_LBE into p_EOS, Eq. 18).  The
    eta' terms of the recovered stress cancel only for k beta_2 = -19; with the
    coefficients of the 2-D model (bulk viscosity varpi c_s^2 tau_e) zeta would be 50%
    larger, a 2.3% change of the damping (measured agreement: 0.4% of zeta)."""
    p = op.from_physical_3d(Tr=0.8, varpi=varpi)
    G, c = _sound(o3, p)
    nu, zeta = (1 / p.sp - 0.5) / 3, varpi * (2 / 3) * (1 / p.se - 0.5) / 3
    assert 2 * G - 4 * nu / 3 == pytest.approx(zeta, rel=1e-2)
    h = 1e-6 * p.rho_l
    c2 = (orc.eos(p, p.rho_l + h)[0] - orc.eos(p, p.rho_l - h)[0]) / (2 * h)
    assert c == pytest.approx(np.sqrt(c2), rel=5e-3)


def _flat(o3, p, W, L=128, steps=8000, axis=2):
    """Relaxed slab with interfaces normal to x (axis 2) or z (axis 0):
    (gas density, liquid density, 5%-95% thickness)."""
    prof = inputs.slab(L, 2, L // 2, W, p.rho_g, p.rho_l)[0]
    rho0 = prof[None, None, :] if axis == 2 else prof[:, None, None] * np.ones((1, 1, 1))
    rho = o3.macro(p, o3.step(p, o3.init_eq(p, rho0), steps))[0]
    r = rho[0, 0, :] if axis == 2 else rho[:, 0, 0]
    return r[0], r[L // 2], _thickness(r[:L // 2], r[0], r[L // 2])


def _thickness(profile, rg, rl):
    lo, hi = rg + 0.05 * (rl - rg), rg + 0.95 * (rl - rg)
    x = np.arange(len(profile))
    return np.interp(hi, profile, x) - np.interp(lo, profile, x)


def _planted_rates(kind):
    """(s_q, s_e) at s_p = 1, varpi = 1/6 from a mis-read 3-D closure (planted
    mistakes): 'k' puts k where the closure has 1 + 5k/19; 'sixth' sets
    tau_p tau_q = 1/6 instead of 1/12."""
    tau_p, k = 0.5, op.k_3d(1 / 6)
    if kind == "k":
        tau_q = 1 / (12 * tau_p)
        tau_e = 1 / (12 * k * tau_q)
    else:
        tau_q = 1 / (6 * tau_p)
        tau_e = 1 / (12 * (1 + 5 * k / 19) * tau_q)
    return dict(s_q=1 / (tau_q + 0.5), s_e=1 / (tau_e + 0.5))


@pytest.mark.parametrize("mistake", [None, "k", "sixth", "no_Q"])
def test_flat_interface_is_on_the_maxwell_construction(o3, mistake):
    """The recovered pressure tensor of the 3-D model is that of Eq. 17, so a flat
    interface (vdW, Tr = 0.8, K_INT = 1.5) has the Maxwell-construction densities and
    the pressure-tensor thickness: measured gas -0.22%, liquid -0.01%, W -0.37%.
    Planted mistakes move the gas density: k for 1 + 5k/19 in the closure +1.6%,
    no S Q_m -34%; tau_p tau_q = 1/6 (+4.7% at s_eps = s_e) diverges with the 3-D
    s_eps, which counts as detected (a NaN never passes the tolerance)."""
    Tr, K_int = 0.8, 1.5
    W = thermo.interface(thermo.make_eos("vdw", 9 / 49, 2 / 21, 1.0, Tr), K_int)["W"]
    kw = {"no_Q": dict(form=2), None: {}}.get(mistake) if mistake in (None, "no_Q") else _planted_rates(mistake)
    p = op.from_physical_3d(Tr=Tr, K_int=K_int, **kw)
    rg, rl, w = _flat(o3, p, W)
    if mistake is None:
        assert rg == pytest.approx(p.rho_g, rel=5e-3)
        assert rl == pytest.approx(p.rho_l, rel=5e-4)
        assert w == pytest.approx(W, rel=1e-2)
    else:
        assert not abs(rg / p.rho_g - 1) <= 1.2e-2


def test_interface_normal_to_z_is_the_interface_normal_to_x(o3):
    """Cubic symmetry of the lattice, the moment set and S: a slab normal to z relaxes
    to the same profile as one normal to x."""
    p = op.from_physical_3d(Tr=0.85, K_int=1.0)
    W = thermo.interface(thermo.make_eos("vdw", 9 / 49, 2 / 21, 1.0, 0.85), 1.0)["W"]
    a = _flat(o3, p, W, L=32, steps=600, axis=2)
    b = _flat(o3, p, W, L=32, steps=600, axis=0)
    assert np.allclose(a, b, rtol=1e-12)


def _diagonal(o3, p, W, N=48, steps=3000):
    """Slab normal to (1, 1, 0) on an N x N x 1 lattice (rho depends on (x + y) mod N):
    (gas density, liquid density, thickness along the normal)."""
    y, x = np.mgrid[0:N, 0:N]
    s = ((x + y) % N) / np.sqrt(2.0)
    d = np.abs(s - N / np.sqrt(2.0) / 2) - N / np.sqrt(2.0) / 4
    mid, half = 0.5 * (p.rho_g + p.rho_l), 0.5 * (p.rho_l - p.rho_g)
    rho0 = (mid - half * np.tanh(2.0 * np.arctanh(0.9) * d / W))[None]
    rho = o3.macro(p, o3.step(p, o3.init_eq(p, rho0), steps))[0][0, 0]
    return rho[0], rho[N // 2], _thickness(rho[:N // 2], rho[0], rho[N // 2]) / np.sqrt(2.0)


@pytest.mark.parametrize("mistake", [None, "sixth"])
def test_diagonal_interface_matches_the_axis_aligned_one(o3, mistake):
    """The anisotropic error term of the 3-D third-order analysis is proportional to
    12 tau_p tau_q - 1 (as on D2Q9) and acts on mixed third derivatives: zero on an
    axis-aligned interface, largest on one normal to (1, 1, 0).  With the closure the
    two agree (measured: gas -0.5%, liquid -0.1%, W -0.7%); with tau_p tau_q = 1/6 the
    diagonal gas density is 9.5% off and W 6% at s_eps = s_e, and the run diverges at
    the 3-D s_eps (detected either way)."""
    Tr, K_int = 0.8, 1.5
    W = thermo.interface(thermo.make_eos("vdw", 9 / 49, 2 / 21, 1.0, Tr), K_int)["W"]
    p = op.from_physical_3d(Tr=Tr, K_int=K_int, **({} if mistake is None else _planted_rates(mistake)))
    ga, la, wa = _flat(o3, p, W, L=48, steps=3000)
    gd, ld, wd = _diagonal(o3, p, W)
    if mistake is None:
        assert gd == pytest.approx(ga, rel=1.5e-2)
        assert ld == pytest.approx(la, rel=2e-3)
        assert wd == pytest.approx(wa, rel=1.5e-2)
    else:
        assert not (abs(gd / ga - 1) <= 5e-2 and abs(wd / wa - 1) <= 3e-2)


@pytest.mark.parametrize("form", [13, 6])
def test_flow_along_an_interface_needs_the_velocity_dependent_s(o3, form):
    """A flat interface (normal y) in a uniform flow U = 0.05 along x.  Without h and b
    the recovered stress keeps -c_s^2 (u grad eta + grad eta u), which shears the gas
    against the liquid (measured slip 0.12 after 3000 steps); with them (Eq. 6 in 3-D)
    the slip is 1.5e-3, the level of the 2-D model with its cubic correction
    (2.3e-3 on the same case)."""
    Tr, K_int, L, U = 0.8, 1.0, 64, 0.05
    W = thermo.interface(thermo.make_eos("vdw", 9 / 49, 2 / 21, 1.0, Tr), K_int)["W"]
    p = op.from_physical_3d(Tr=Tr, K_int=K_int, form=form)
    prof = inputs.slab(L, 2, L // 2, W, p.rho_g, p.rho_l)[0]
    rho0 = prof[None, :, None] * np.ones((1, 1, 2))
    rho, ux, _, _ = o3.macro(p, o3.step(p, o3.init_eq(p, rho0, np.full(rho0.shape, U)), 3000))
    slip = ux[0, L // 2, 0] - ux[0, 0, 0]
    if form == 13:
        assert abs(slip) < 3e-3
    else:
        assert abs(slip) > 5e-2


def test_laplace_law_of_a_liquid_column(o3, orc):
    """A liquid column (radius 10, W = 5, 48 x 48 x 1) obeys dp = sigma / R with sigma
    from the pressure tensor (Eq. 17), as the 2-D model does on the same lattice:
    dp R / sigma = 0.977 for both (curvature corrections at R / W = 2), and the two
    agree to 0.5%."""
    N, R = 48, 10.0
    e = thermo.make_eos("vdw", 9 / 49, 2 / 21, 1.0, 0.85)
    sigma = thermo.interface(e, 1.0)["sigma"]
    out = []
    for dim in (3, 2):
        p = (op.from_physical_3d if dim == 3 else op.from_physical)(Tr=0.85, K_int=1.0)
        rho0 = inputs.droplet(N, N, R, 5.0, p.rho_g, p.rho_l)
        if dim == 3:
            rho = o3.macro(p, o3.step(p, o3.init_eq(p, rho0[None]), 2500))[0][0]
        else:
            rho = orc.macro(p, orc.step(p, orc.init_feq(p, rho0), 2500))[0]
        dp = orc.eos(p, rho[N // 2, N // 2])[0] - orc.eos(p, rho[0, 0])[0]
        radius = np.sqrt((rho > 0.5 * (p.rho_g + p.rho_l)).sum() / np.pi)
        out.append(dp * radius / (sigma * p.lam))
    assert out[0] == pytest.approx(1.0, rel=4e-2)
    assert out[0] == pytest.approx(out[1], rel=5e-3)


def test_carnahan_starling_interface_at_the_papers_setting(o3, orc):
    """The paper's EOS and setting of supplement Fig. 2 (Carnahan-Starling, a = 1,
    b = 4, Tr = 0.8, K_INT = 2.2949, so W = 10): a flat 3-D interface has the Maxwell
    densities and the pressure-tensor thickness (measured: gas -0.03%, liquid +0.14%,
    W +1.0%), and the same densities as the D2Q9 oracle on the same slab."""
    Tr, K, L = 0.8, 2.2949, 160
    e = thermo.make_eos("cs", 1.0, 4.0, 1.0, Tr)
    W = thermo.interface(e, K)["W"]
    p3 = op.from_physical_3d(eos="cs", a=1.0, b=4.0, Tr=Tr, K_int=K)
    p2 = op.from_physical(eos="cs", a=1.0, b=4.0, Tr=Tr, K_int=K)
    slab = inputs.slab(L, 2, L // 2, W, p3.rho_g, p3.rho_l)
    r3 = o3.macro(p3, o3.step(p3, o3.init_eq(p3, slab[0][None, None, :]), 10000))[0][0, 0]
    r2 = orc.macro(p2, orc.step(p2, orc.init_feq(p2, slab), 10000))[0][0]
    assert r3[0] == pytest.approx(p3.rho_g, rel=3e-3)
    assert r3[L // 2] == pytest.approx(p3.rho_l, rel=3e-3)
    assert _thickness(r3[: L // 2], r3[0], r3[L // 2]) == pytest.approx(W, rel=2e-2)
    assert r3[0] == pytest.approx(r2[0], rel=3e-3) and r3[L // 2] == pytest.approx(r2[L // 2], rel=1e-3)


def _transform(o3, f, R):
    """The state f[i, z, y, x] of an N^3 periodic lattice carried by the integer
    rotation / reflection R: population i at r goes to population j (e_j = R e_i) at
    R r (mod N)."""
    e = o3.velocities().T
    perm = [next(j for j in range(19) if np.array_equal(e[j], R @ e[i])) for i in range(19)]
    n = f.shape[1]
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    r = np.stack([x, y, z])                       # (3, n, n, n): coordinates as (x, y, z)
    rr = np.tensordot(R, r, 1) % n
    out = np.empty_like(f)
    for i in range(19):
        out[perm[i], rr[2], rr[1], rr[0]] = f[i]
    return out


@pytest.mark.parametrize("name,R", [
    ("z90", [[0, -1, 0], [1, 0, 0], [0, 0, 1]]), ("x90", [[1, 0, 0], [0, 0, -1], [0, 1, 0]]),
    ("y90", [[0, 0, 1], [0, 1, 0], [-1, 0, 0]]), ("mirror_x", [[-1, 0, 0], [0, 1, 0], [0, 0, 1]]),
    ("diagonal", [[0, 1, 0], [1, 0, 0], [0, 0, 1]])])
def test_the_step_commutes_with_the_cubic_symmetries(o3, name, R):
    """The D3Q19 lattice, its moment set, the 3-D S (whose velocity-dependent entries
    couple the five traceless second-order moments to q through the traceless part
    of u qhat + qhat u), the forcing and Q_m are invariant under the cubic group:
    stepping a rotated (or reflected) state equals rotating the stepped state.  A
    state with a droplet and random velocities exercises every coupling; a sign
    slip in one entry of S breaks the symmetry (planted in a copy of the oracle:
    S(p_xz, q_x) with the wrong sign fails the 90-degree rotations about z and x
    and the diagonal reflection)."""
    R = np.array(R)
    p = op.from_physical_3d(Tr=0.8)
    n = 8
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    r = np.sqrt((x - 3.3) ** 2 + (y - 4.1) ** 2 + (z - 3.7) ** 2)
    rho = 0.5 * (p.rho_g + p.rho_l) - 0.5 * (p.rho_l - p.rho_g) * np.tanh(2 * (r - 2.5) / 3.0)
    u = [RNG.uniform(-0.03, 0.03, rho.shape) for _ in range(3)]
    f = o3.init_eq(p, rho, *u)
    a = o3.step(p, _transform(o3, f, R), 3)
    b = _transform(o3, o3.step(p, f, 3), R)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
