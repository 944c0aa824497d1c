"""Parity of the CUDA time step (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 GPU path <= 1e-12 relative on f after 2,000 steps; FP32 path
<= 2e-5 relative on rho; FP16 storage (FP32 arithmetic) <= 8e-3 relative on rho
after 500 steps: each step rounds every stored deviation to half precision
(relative 2^-12), the nine roundings of a node add to its density, and the
mass they move performs a random walk, so the bound is
2^-12 * sqrt(500) * (sum_i |f_i - w_i rho_ref| / max rho ~ 1.4) ~ 8e-3.
Relative error = max|diff| / max|reference|."""
import numpy as np
import pytest

from gpu_util import W_REST, gpu_populations, lattice, oracle_params, rel_inf, set_state_fp64
from paper_1809_02390_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_02390_gb300 import build

    build.build()


def droplet64():
    p = oracle_params(Tr=0.85, K_int=1.0)
    return p, inputs.droplet(64, 64, 16, 5, p.rho_g, p.rho_l)


@pytest.mark.parametrize("variant", ["fused", "two_pass"])
def test_fp64_droplet_2000_steps(orc, variant):
    """64x64 periodic vdW droplet, R = 16, tanh width 5, Tr = 0.85, tau = 1, 2,000 steps."""
    p, rho0 = droplet64()
    ref = orc.step(p, orc.init_feq(p, rho0), 2000)
    lat = lattice(rho0, "fp64", variant, Tr=0.85, K_int=1.0)
    lat.step(2000)
    torch.cuda.synchronize()
    assert rel_inf(gpu_populations(lat), ref) <= 1e-12


def test_fp64_init_matches_oracle(orc):
    p, rho0 = droplet64()
    lat = lattice(rho0, "fp64")
    assert rel_inf(gpu_populations(lat), orc.init_feq(p, rho0)) <= 1e-15


@pytest.mark.parametrize("precision,tol,steps", [("fp32", 2e-5, 2000), ("fp16s", 8e-3, 500)])
@pytest.mark.parametrize("variant", ["fused", "two_pass"])
def test_reduced_precision_droplet(orc, precision, tol, steps, variant):
    p, rho0 = droplet64()
    ref = orc.macro(p, orc.step(p, orc.init_feq(p, rho0), steps))[0]
    lat = lattice(rho0, precision, variant, Tr=0.85, K_int=1.0)
    lat.step(steps)
    rho = lat.moments(velocity=False).double().cpu().numpy()
    assert rel_inf(rho, ref) <= tol


RAGGED = [(37, 29), (70, 45), (33, 31), (32, 32), (3, 3), (5, 7), (4, 100), (100, 4), (65, 9)]


@pytest.mark.parametrize("nx,ny", RAGGED)
@pytest.mark.parametrize("variant", ["fused", "two_pass"])
def test_fp64_ragged_with_flow(orc, nx, ny, variant):
    """Arbitrary sizes (several strips, ragged tails, lattices narrower than a warp)
    from a state with a random velocity field, so that the velocity-dependent
    terms (S off-diagonals, R, T, X, the cubic F_m terms) are all exercised."""
    p = oracle_params(Tr=0.85, K_int=1.0)
    rng = np.random.default_rng(nx * 1000 + ny)
    rho = inputs.droplet(nx, ny, min(nx, ny) / 4, 3, p.rho_g, p.rho_l) * (1 + 0.01 * rng.uniform(-1, 1, (ny, nx)))
    f0 = orc.init_eq(p, rho, 0.05 * rng.uniform(-1, 1, (ny, nx)), 0.05 * rng.uniform(-1, 1, (ny, nx)))
    ref = orc.step(p, f0, 20)
    lat = lattice(rho, "fp64", variant, Tr=0.85, K_int=1.0)
    set_state_fp64(lat, f0)
    lat.step(20)
    torch.cuda.synchronize()
    assert rel_inf(gpu_populations(lat), ref) <= 1e-13


def test_fp64_carnahan_starling(orc):
    """The paper's own EOS (Eq. 20, a = 1, b = 4, R = 1) at Tr = 0.8 with W = 10 (K_INT = 2.2949)."""
    p = oracle_params(eos="cs", a=1.0, b=4.0, Tr=0.8, K_int=2.2949)
    rho0 = inputs.slab(48, 16, 24, 10, p.rho_g, p.rho_l)
    ref = orc.step(p, orc.init_feq(p, rho0), 300)
    lat = lattice(rho0, "fp64", eos="cs", eos_a=1.0, eos_b=4.0, Tr=0.8, K_int=2.2949)
    lat.step(300)
    torch.cuda.synchronize()
    assert rel_inf(gpu_populations(lat), ref) <= 1e-12


def test_moments_and_reduce(orc):
    p, rho0 = droplet64()
    f = orc.step(p, orc.init_feq(p, rho0), 50)
    rho_o, ux_o, uy_o = orc.macro(p, f)
    lat = lattice(rho0, "fp64", Tr=0.85, K_int=1.0)
    lat.step(50)
    rho, ux, uy = (t.cpu().numpy() for t in lat.moments())
    assert rel_inf(rho, rho_o) <= 1e-13
    assert np.abs(ux - ux_o).max() <= 1e-13 and np.abs(uy - uy_o).max() <= 1e-13
    r = lat.reduce()
    assert r["mass"] == pytest.approx(rho_o.sum(), rel=1e-13)
    assert r["mom_x"] == pytest.approx((rho_o * ux_o).sum(), abs=1e-11)
    assert r["n_liquid"] == (rho_o > 0.5 * (p.rho_g + p.rho_l)).sum()
    assert r["rho_min"] == pytest.approx(rho_o.min(), rel=1e-13)
    assert r["rho_max"] == pytest.approx(rho_o.max(), rel=1e-13)
    assert r["p_center"] == pytest.approx(orc.eos(p, rho_o[32, 32])[0], rel=1e-12)


@pytest.mark.parametrize("static", [False, True])
def test_reduce_carnahan_starling_against_the_oracle(orc, static):
    """lb_reduce and lb_reduce_static on a Carnahan-Starling droplet (a = 1, b = 4,
    Tr = 0.7, K_INT = 2, K_EOS = 0.5; 80 x 60, 40 FP64 steps): the sums against the
    oracle's fields, and both probe pressures against the oracle's EOS (Eq. 20) at
    the oracle's densities of the probe nodes."""
    from paper_1809_02390_gb300 import capi

    kw = dict(eos="cs", a=1.0, b=4.0, R=1.0, Tr=0.7, K_int=2.0, K_eos=0.5)
    p = oracle_params(**kw)
    rho0 = inputs.droplet(80, 60, 14.0, 8.0, p.rho_g, p.rho_l)
    rho_o, ux_o, uy_o = orc.macro(p, orc.step(p, orc.init_feq(p, rho0), 40))
    lat = lattice(rho0, "fp64", eos="cs", eos_a=1.0, eos_b=4.0, R_gas=1.0, Tr=0.7, K_int=2.0, K_eos=0.5)
    lat.step(40)
    v = capi.lb_reduce_static(lat.h) if static else capi.lb_reduce(lat.h)
    mass, mx, my, p_c, p_0, n_liq, r_min, r_max = v
    assert mass == pytest.approx(rho_o.sum(), rel=1e-13)
    assert mx == pytest.approx((rho_o * ux_o).sum(), abs=1e-11)
    assert my == pytest.approx((rho_o * uy_o).sum(), abs=1e-11)
    assert p_c == pytest.approx(orc.eos(p, rho_o[30, 40])[0], rel=1e-12)
    assert p_0 == pytest.approx(orc.eos(p, rho_o[0, 0])[0], rel=1e-12)
    assert n_liq == (rho_o > 0.5 * (p.rho_g + p.rho_l)).sum()
    assert r_min == pytest.approx(rho_o.min(), rel=1e-13) and r_max == pytest.approx(rho_o.max(), rel=1e-13)
    lat.close()


def test_deterministic():
    p, rho0 = droplet64()
    a = lattice(rho0, "fp32")
    b = lattice(rho0, "fp32")
    a.step(100)
    b.step(100)
    torch.cuda.synchronize()
    assert torch.equal(a.state(), b.state())


def _patch(f, x, y, r):
    ny, nx = f.shape[1:]
    ys = [(y + d) % ny for d in range(-r, r + 1)]
    xs = [(x + d) % nx for d in range(-r, r + 1)]
    return f[:, ys][:, :, xs]


def test_full_size_spinodal_sampled(orc):
    """4096 x 4096 FP32 spinodal decomposition in the benchmark's launch
    configuration: two steps from the seeded initial state, checked at sampled
    nodes, each computed by the oracle from its own initial state on the 9x9
    neighbourhood that determines it (periodic wrap of the patch is never reached)."""
    p = oracle_params(Tr=0.8, K_int=1.0)
    n = 4096
    rho0 = inputs.spinodal(n, n, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=0)
    lat = lattice(rho0, "fp32", Tr=0.8, K_int=1.0, layout="rows")
    from paper_1809_02390_gb300 import capi

    assert capi.lb_uses_tma(lat.h) and capi.lb_tile_dispatch(lat.h)  # the benchmark's kernel
    steps = 2
    lat.step(steps)
    torch.cuda.synchronize()
    st = lat.state()
    rng = np.random.default_rng(3)
    pts = [(0, 0), (n - 1, n - 1), (31, 32), (32, 4095), (4064, 17)] + [tuple(v) for v in rng.integers(0, n, (27, 2))]
    worst = 0.0
    for x, y in pts:
        patch_rho = _patch(rho0[None], x, y, 2 * steps + 2)[0]
        ref = orc.step(p, orc.init_feq(p, patch_rho), steps)[:, 2 * steps + 2, 2 * steps + 2]
        got = st[:, y, x].double().cpu().numpy() + lat.rho_ref * W_REST
        worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    assert worst <= 2e-6


def test_full_size_mass_conservation():
    p = oracle_params(Tr=0.8, K_int=1.0)
    n = 4096
    rho0 = inputs.spinodal(n, n, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=0)
    lat = lattice(rho0, "fp32", Tr=0.8, K_int=1.0)
    m0 = lat.reduce()["mass"]
    lat.step(200)
    r = lat.reduce()
    assert r["mass"] == pytest.approx(m0, rel=2e-6)
    assert rho0.sum() == pytest.approx(m0, rel=1e-6)


def test_fp32_tma_path(orc):
    """The FP32 fused step with tensor-copy staging (interior tiles) and the plain
    path (tiles whose windows wrap) on one lattice, against the oracle, with many
    tiles per block and with one; no bounded wait gave up."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(160, 96, 30, 5, p.rho_g, p.rho_l, center=(70.3, 50.6))
    lat = lattice(rho0, "fp32", Tr=0.85, K_int=1.0)
    assert capi.lb_uses_tma(lat.h)
    capi.lb_set_step_blocks(lat.h, 4)  # 30 tiles: each block steps 7 or 8, interior and wrapping mixed
    lat.step(150)
    capi.lb_set_step_blocks(lat.h, 0)
    lat.step(150)
    ref = orc.macro(p, orc.step(p, orc.init_feq(p, rho0), 300))[0]
    rho = lat.moments(velocity=False).double().cpu().numpy()
    assert rel_inf(rho, ref) <= 2e-5
    capi.lb_status(lat.h)
    assert not capi.lb_uses_tma(lattice(rho0[:, :150], "fp32", Tr=0.85, K_int=1.0).h)  # nx % 4 != 0


def test_fp16_tma_path(orc):
    """FP16 storage with tensor-copy staging (48-half windows; interior tiles) and
    plain loads (wrapping tiles) on one lattice, many tiles per block and one,
    against the oracle within the FP16 tolerance of 500 steps; no wait gave up."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(160, 96, 30, 5, p.rho_g, p.rho_l, center=(70.3, 50.6))
    lat = lattice(rho0, "fp16s", Tr=0.85, K_int=1.0)
    assert capi.lb_uses_tma(lat.h)
    capi.lb_set_step_blocks(lat.h, 4)
    lat.step(250)
    capi.lb_set_step_blocks(lat.h, 0)
    lat.step(250)
    ref = orc.macro(p, orc.step(p, orc.init_feq(p, rho0), 500))[0]
    rho = lat.moments(velocity=False).double().cpu().numpy()
    assert rel_inf(rho, ref) <= 8e-3
    capi.lb_status(lat.h)
    assert not capi.lb_uses_tma(lattice(rho0[:, :156], "fp16s", Tr=0.85, K_int=1.0).h)  # nx % 8 != 0


# (oracle keywords, library keywords): relaxation rates other than s_p = 1 (so
# s_q, s_e and every R, T, X, Q_m coefficient move), another varpi, and the
# Carnahan-Starling EOS with the paper's a = 1, b = 4 and K_EOS, K_INT != 1.
PARAM_SETS = [
    (dict(Tr=0.85, K_int=1.0, s_p=1.5), dict(Tr=0.85, K_int=1.0, s_p=1.5)),
    (dict(Tr=0.75, K_int=1.3, s_p=0.8), dict(Tr=0.75, K_int=1.3, s_p=0.8)),
    (dict(Tr=0.85, K_int=1.0, varpi=0.3, s_p=1.1), dict(Tr=0.85, K_int=1.0, varpi=0.3, s_p=1.1)),
    (dict(eos="cs", a=1.0, b=4.0, R=1.0, Tr=0.7, K_eos=0.2, K_int=2.0, s_p=1.3),
     dict(eos="cs", eos_a=1.0, eos_b=4.0, R_gas=1.0, Tr=0.7, K_eos=0.2, K_int=2.0, s_p=1.3)),
]


@pytest.mark.parametrize("okw,lkw", PARAM_SETS, ids=["sp1.5", "sp0.8", "varpi0.3", "cs"])
def test_fp64_parameters_with_flow(orc, okw, lkw):
    """FP64 step against the oracle for 100 steps from a state with a random
    velocity field, away from the default rates, varpi and EOS."""
    p = oracle_params(**okw)
    nx, ny = 70, 45
    rng = np.random.default_rng(7)
    rho = inputs.droplet(nx, ny, 12, 6, p.rho_g, p.rho_l) * (1 + 0.01 * rng.uniform(-1, 1, (ny, nx)))
    f0 = orc.init_eq(p, rho, 0.03 * rng.uniform(-1, 1, (ny, nx)), 0.03 * rng.uniform(-1, 1, (ny, nx)))
    ref = orc.step(p, f0, 100)
    lat = lattice(rho, "fp64", **lkw)
    set_state_fp64(lat, f0)
    lat.step(100)
    torch.cuda.synchronize()
    assert rel_inf(gpu_populations(lat), ref) <= 1e-12


def test_fp16_stochastic_rounding_keeps_mass():
    """A stationary flat interface (Tr = 0.9, 256 x 32, 5,000 steps) in FP16 storage:
    round-to-nearest repeats the same rounding errors every step, so the mass drifts
    steadily (by how much depends on the rounding of the arithmetic before the
    store); stochastic rounding (the default) makes the errors zero-mean, leaving a
    random walk of order 2^-11 sqrt(steps / nodes) ~ 2e-4."""
    from paper_1809_02390_gb300 import derive

    d = derive(256, 32, Tr=0.9)
    rho0 = inputs.slab(256, 32, 128, d["W1"], d["rho_g"], d["rho_l"])
    drift = {}
    for name, rounding in (("stochastic", 0), ("nearest", 1)):
        lat = lattice(rho0, "fp16s", Tr=0.9, rounding=rounding)
        lat.step(5000)
        drift[name] = abs(lat.reduce()["mass"] / rho0.sum() - 1)
        lat.close()
    assert drift["stochastic"] < 1e-3
    assert drift["nearest"] > 2 * drift["stochastic"]


@pytest.mark.parametrize("layout", ["rows", "planes"])
def test_fp16_pair_and_single_node_stores_round_alike(layout):
    """FP16 stores round with random words drawn per pair of x-neighbours: the fused
    step writes each pair with one packed conversion, the two-pass step one node at
    a time, taking the pair's word and its half of it.  One step of each from the
    same state (160 x 96: tensor-copy tiles, wrapping tiles, both nodes of every
    pair) gives the same halves, except where the two steps' FP32 arithmetic
    already differs in the last bit (about 0.3% of the values) and that difference
    crosses a rounding boundary (chance about 2^-13 each); random words used
    inconsistently would change about half of all halves."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(160, 96, 30, 5, p.rho_g, p.rho_l, center=(70.3, 50.6))
    a = lattice(rho0, "fp16s", "fused", layout=layout, Tr=0.85, K_int=1.0)
    b = lattice(rho0, "fp16s", "two_pass", layout=layout, Tr=0.85, K_int=1.0)
    assert capi.lb_uses_tma(a.h) and not capi.lb_uses_tma(b.h)
    for lat in (a, b):
        lat.step(1)
    torch.cuda.synchronize()
    def ordered(lat):  # halves as integers in value order (sign-magnitude to two's complement; -0 = +0)
        h = lat.state().view(torch.int16).to(torch.int32)
        return torch.where(h < 0, -(h & 0x7FFF), h)

    diff = (ordered(a) - ordered(b)).abs()
    assert int((diff != 0).sum()) <= 20
    assert int(diff.max()) <= 1
    for lat in (a, b):
        capi.lb_status(lat.h)
        lat.close()


@pytest.mark.parametrize("precision,layout,on_device", [("fp32", "rows", False), ("fp16s", "planes", False),
                                                       ("fp32", "planes", True)])
def test_storage_shift_defaults_to_the_mean_density(precision, layout, on_device):
    """Without rho_ref the binding passes NaN and lb_init takes the mean initial
    density (FP64 sum on the device, rounded to float); the lattice then steps bit
    for bit like one given that value explicitly, and a batch takes the same value
    for the same density."""
    from paper_1809_02390_gb300 import Batch, capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(160, 96, 30, 5, p.rho_g, p.rho_l, center=(70.3, 50.6))
    src = torch.from_numpy(rho0).cuda() if on_device else rho0
    a = lattice(src, precision, layout=layout, Tr=0.85, K_int=1.0)
    want = float(np.float32(rho0.mean()))
    assert abs(a.rho_ref - want) <= abs(want) * 2.0 ** -23
    assert a.rho_ref == float(np.float32(a.rho_ref))
    b = lattice(rho0, precision, layout=layout, Tr=0.85, K_int=1.0, rho_ref=a.rho_ref)
    for lat in (a, b):
        lat.step(40)
    torch.cuda.synchronize()
    assert torch.equal(a.buffer(), b.buffer())
    if precision == "fp32":
        bt = Batch([rho0, rho0[:64, :80]], [dict(Tr=0.85, K_int=1.0, layout=layout)] * 2)
        assert bt.rho_refs[0] == a.rho_ref
        assert abs(bt.rho_refs[1] - float(np.float32(rho0[:64, :80].mean()))) <= 2.0 ** -22
        bt.close()
    for lat in (a, b):
        lat.close()


def test_bounded_wait_gives_up_and_is_reported(orc):
    """A wait that nothing completes (lb_wait_selftest) ends after its poll budget,
    is reported as LB_ETIMEOUT once (the flag is then clear), and the context stays
    usable: the tensor-copy step still matches the oracle afterwards."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(160, 96, 30, 5, p.rho_g, p.rho_l)
    lat = lattice(rho0, "fp32", Tr=0.85, K_int=1.0)
    assert capi.lb_wait_selftest(lat.h, 2000) == capi.LB_ETIMEOUT
    capi.lb_status(lat.h)  # cleared: no error now
    lat.step(100)
    ref = orc.macro(p, orc.step(p, orc.init_feq(p, rho0), 100))[0]
    assert rel_inf(lat.moments(velocity=False).double().cpu().numpy(), ref) <= 2e-5
    capi.lb_status(lat.h)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_stream_copy_leaves_the_state(precision):
    """lb_stream_copy (the step's memory traffic without its arithmetic) moves the
    state to the other buffer bit for bit; the lattice then steps as before."""
    from paper_1809_02390_gb300 import capi, derive

    d = derive(130, 70, Tr=0.8)
    rho0 = inputs.droplet(130, 70, 15, 4, d["rho_g"], d["rho_l"])
    a = lattice(rho0, precision, Tr=0.8)
    b = lattice(rho0, precision, Tr=0.8)
    a.step(3)
    b.step(3)
    before = a.state().clone()
    capi.lb_stream_copy(a.h)
    assert torch.equal(a.state(), before)
    a.step(5)
    b.step(5)
    assert torch.equal(a.state(), b.state())


@pytest.mark.parametrize("layout", ["planes", "rows"])
def test_set_equilibrium_matches_oracle(orc, layout):
    """lb_set_equilibrium (equilibrium of Eq. 3 for a density and velocity field)
    against the oracle's equilibrium, then 100 FP64 steps from it; the FP32 state
    is the FP64 one rounded once."""
    import torch

    p = oracle_params(Tr=0.85, K_int=1.0)
    nx, ny = 70, 45
    rng = np.random.default_rng(11)
    rho = inputs.droplet(nx, ny, 12, 6, p.rho_g, p.rho_l) * (1 + 0.01 * rng.uniform(-1, 1, (ny, nx)))
    ux, uy = 0.05 * rng.uniform(-1, 1, (ny, nx)), 0.05 * rng.uniform(-1, 1, (ny, nx))
    f0 = orc.init_eq(p, rho, ux, uy)
    lat = lattice(rho, "fp64", layout=layout, Tr=0.85, K_int=1.0)
    lat.set_equilibrium(rho, ux, uy)
    assert rel_inf(gpu_populations(lat), f0) <= 1e-15
    lat.step(100)
    torch.cuda.synchronize()
    assert rel_inf(gpu_populations(lat), orc.step(p, f0, 100)) <= 1e-12
    l32 = lattice(rho, "fp32", layout=layout, Tr=0.85, K_int=1.0)
    l32.set_equilibrium(rho, ux, None)
    ref = orc.init_eq(p, rho, ux, None)
    assert rel_inf(gpu_populations(l32), ref) <= 2e-7


def test_host_and_device_initial_densities_agree():
    """lb_init from host densities (copied and checked on the device, the end-to-end
    path of the benchmark) and from the same densities already on the device give
    the same state, bit for bit, in every storage precision."""
    from paper_1809_02390_gb300 import Lattice

    p = oracle_params(Tr=0.8, K_int=1.0)
    rho0 = inputs.spinodal(160, 96, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=4)
    shift = float(np.float32(rho0.mean()))  # the same storage shift for both (the default is a mean)
    for precision in ("fp64", "fp32", "fp16s"):
        a = Lattice(rho0, precision=precision, Tr=0.8, layout="rows", rho_ref=shift)
        b = Lattice(torch.from_numpy(rho0).cuda(), precision=precision, Tr=0.8, layout="rows", rho_ref=shift)
        torch.cuda.synchronize()
        assert torch.equal(a.buffer(), b.buffer()), precision
        a.step(10)
        b.step(10)
        torch.cuda.synchronize()
        assert torch.equal(a.buffer(), b.buffer()), precision
        a.close()
        b.close()


def test_largest_lattice_sampled(orc):
    """The largest lattice the library accepts (9 nx ny just below 2^31, the limit of
    its 32-bit population offsets): 16384 x 14563 FP32 in the rows layout of the
    benchmark (8.6 GB per population buffer; 14563 rows leave a ragged last tile
    row).  Two steps from a seeded spinodal field, checked at sampled nodes against
    the oracle on each node's own 9 x 9 neighbourhood, including the last node of
    the buffer, the four corners (periodic wrap) and the last ragged tile row."""
    p = oracle_params(Tr=0.8, K_int=1.0)
    nx, ny = 16384, 14563
    assert 9 * nx * ny < 2 ** 31 <= 9 * nx * (ny + 1)
    rho0 = inputs.spinodal(nx, ny, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=5)
    lat = lattice(rho0, "fp32", Tr=0.8, K_int=1.0, layout="rows")
    steps = 2
    lat.step(steps)
    torch.cuda.synchronize()
    st = lat.state()
    rng = np.random.default_rng(9)
    pts = [(0, 0), (nx - 1, ny - 1), (nx - 1, 0), (0, ny - 1), (8191, 14560), (31, ny - 3)]
    pts += [(int(x), int(y)) for x, y in zip(rng.integers(0, nx, 12), rng.integers(0, ny, 12))]
    worst = 0.0
    for x, y in pts:
        patch_rho = _patch(rho0[None], x, y, 2 * steps + 2)[0]
        ref = orc.step(p, orc.init_feq(p, patch_rho), steps)[:, 2 * steps + 2, 2 * steps + 2]
        got = st[:, y, x].double().cpu().numpy() + lat.rho_ref * W_REST
        worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    assert worst <= 2e-6
    lat.close()
    del st
    torch.cuda.empty_cache()
