"""The rows layout f[ny][9][nx] against the oracle and against the planes layout.

Both layouts run the same arithmetic on every node (only the addresses of the
loads and stores differ, and the random words of the FP16 stores' stochastic
rounding are keyed by the node's coordinates, not the address), so after any
number of steps the two states
agree bit for bit, and so do the densities, pressures and reductions computed from
them.  The FP64 rows path is also checked against the oracle directly."""
import numpy as np
import pytest

from gpu_util import W_REST, lattice, oracle_params, rel_inf
from paper_1809_02390_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_02390_gb300 import build

    build.build()


def _pair(rho0, precision, variant="fused", **kw):
    a = lattice(rho0, precision, variant, **kw)
    b = lattice(rho0, precision, variant, layout="rows", **kw)
    return a, b


def _same(a, b):
    torch.cuda.synchronize()
    assert (a.layout, b.layout) == ("planes", "rows") and b.buffer().shape == (a.ny, 9, a.nx)
    assert torch.equal(a.state(), b.state())
    ra, ua, va = a.moments()
    rb, ub, vb = b.moments()
    assert torch.equal(ra, rb) and torch.equal(ua, ub) and torch.equal(va, vb)
    assert torch.equal(a.pressure(), b.pressure())
    assert a.reduce() == b.reduce()


@pytest.mark.parametrize("variant", ["fused", "two_pass"])
@pytest.mark.parametrize("nx,ny", [(70, 45), (33, 17)])
def test_rows_fp64_matches_oracle(orc, variant, nx, ny):
    """FP64, ragged lattices (partial tiles in x and y), 300 steps from a droplet."""
    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(nx, ny, min(nx, ny) / 4, 4, p.rho_g, p.rho_l, center=(0.45 * nx, 0.55 * ny))
    lat = lattice(rho0, "fp64", variant, layout="rows", Tr=0.85, K_int=1.0)
    assert rel_inf(lat.populations().cpu().numpy(), orc.init_feq(p, rho0)) <= 1e-15
    lat.step(300)
    torch.cuda.synchronize()
    ref = orc.step(p, orc.init_feq(p, rho0), 300)
    assert rel_inf(lat.populations().cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("variant", ["fused", "two_pass"])
def test_rows_bit_identical_to_planes(precision, variant):
    """160 x 96 (the FP32 and FP16 fused steps take the tensor-copy kernel: interior
    tiles by tensor copies through the (x, plane, y) map, wrapping tiles by plain
    loads), 60 steps with a block stepping many tiles, 60 with the default grid."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(160, 96, 30, 5, p.rho_g, p.rho_l, center=(70.3, 50.6))
    a, b = _pair(rho0, precision, variant, Tr=0.85, K_int=1.0)
    tma = precision != "fp64" and variant == "fused"
    assert capi.lb_uses_tma(a.h) == capi.lb_uses_tma(b.h) == int(tma)
    for lat in (a, b):
        capi.lb_set_step_blocks(lat.h, 4)
        lat.step(60)
        capi.lb_set_step_blocks(lat.h, 0)
        lat.step(60)
    _same(a, b)
    capi.lb_status(b.h)


@pytest.mark.parametrize("precision,nx", [("fp32", 150), ("fp16s", 156), ("fp32", 40)])
def test_rows_plain_fused_bit_identical(precision, nx):
    """Lattices the tensor-copy kernel does not take (nx not a multiple of 16 bytes,
    or too narrow): the plain fused kernel in both layouts."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(nx, 60, 12, 4, p.rho_g, p.rho_l)
    a, b = _pair(rho0, precision, Tr=0.85, K_int=1.0)
    assert not capi.lb_uses_tma(b.h)
    a.step(80)
    b.step(80)
    _same(a, b)


def test_rows_full_size_bit_identical():
    """4096 x 4096 FP32 spinodal lattice in the benchmark's launch configuration:
    the rows layout equals the planes layout bit for bit after 3 steps."""
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.8, K_int=1.0)
    n = 4096
    rho0 = inputs.spinodal(n, n, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=0)
    a, b = _pair(rho0, "fp32", Tr=0.8, K_int=1.0)
    assert capi.lb_uses_tma(b.h)
    a.step(3)
    b.step(3)
    torch.cuda.synchronize()
    assert torch.equal(a.state(), b.state())
    assert a.reduce() == b.reduce()
    capi.lb_status(b.h)


def test_rows_full_size_sampled(orc):
    """The same lattice in the rows layout against the oracle at sampled nodes
    (each from its own 13 x 13 neighbourhood of the initial state), 2 steps."""
    p = oracle_params(Tr=0.8, K_int=1.0)
    n = 4096
    rho0 = inputs.spinodal(n, n, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=0)
    lat = lattice(rho0, "fp32", layout="rows", Tr=0.8, K_int=1.0)
    lat.step(2)
    torch.cuda.synchronize()
    st = lat.state()
    rng = np.random.default_rng(5)
    pts = [(0, 0), (n - 1, n - 1), (31, 32), (4095, 16), (17, 4064)] + [tuple(v) for v in rng.integers(0, n, (20, 2))]
    r = 6
    for x, y in pts:
        ys = [(y + d) % n for d in range(-r, r + 1)]
        xs = [(x + d) % n for d in range(-r, r + 1)]
        ref = orc.step(p, orc.init_feq(p, rho0[ys][:, xs]), 2)[:, r, r]
        got = st[:, y, x].double().cpu().numpy() + lat.rho_ref * W_REST
        assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 2e-6, (x, y)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_rows_stream_copy_leaves_the_state(precision):
    from paper_1809_02390_gb300 import capi, derive

    d = derive(130, 70, Tr=0.8)
    rho0 = inputs.droplet(130, 70, 15, 4, d["rho_g"], d["rho_l"])
    a = lattice(rho0, precision, layout="rows", Tr=0.8)
    a.step(3)
    before = a.buffer().clone()
    capi.lb_stream_copy(a.h)
    assert torch.equal(a.buffer(), before)


def test_rows_rejected_by_the_adjoint():
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(64, 64, 16, 5, p.rho_g, p.rho_l)
    lat = lattice(rho0, "fp64", layout="rows", Tr=0.85, K_int=1.0)
    f = lat.buffer().clone()
    lam_in, lam_out = torch.zeros_like(f), torch.zeros_like(f)
    nscr = capi.lib().lb_adjoint_scratch_bytes(capi.ctypes.byref(lat.p))
    scr = torch.empty(nscr, dtype=torch.uint8, device=f.device)
    rc = capi.lib().lb_adjoint_step(lat.h, f.data_ptr(), lam_in.data_ptr(), lam_out.data_ptr(), None,
                                    scr.data_ptr(), nscr)
    assert rc == capi.LB_ENOTSUP and "planes layout" in capi.lb_last_error(lat.h)
