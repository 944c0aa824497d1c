"""Dynamic tile dispatch of the tensor-copy step (tiles handed out by ticket, two
windows in flight per block) against the static walk (block b steps tiles b,
b + grid, ...): the same tiles with the same arithmetic, so the states agree bit
for bit after any number of launches.  A launch that skipped or repeated a tile
(a ticket counter not reset between launches) would show as a difference."""
import pytest

from gpu_util import lattice, oracle_params, rel_inf
from paper_1809_02390_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_02390_gb300 import build

    build.build()


def _pair(rho0, precision, layout, **kw):
    from paper_1809_02390_gb300 import capi

    dyn = lattice(rho0, precision, layout=layout, **kw)
    sta = lattice(rho0, precision, layout=layout, **kw)
    assert capi.lb_uses_tma(dyn.h) and capi.lb_tile_dispatch(dyn.h)
    capi.lb_set_tile_dispatch(sta.h, False)
    assert not capi.lb_tile_dispatch(sta.h)
    return dyn, sta


@pytest.mark.parametrize("layout", ["planes", "rows"])
@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
@pytest.mark.parametrize("nx,ny", [(160, 96), (208, 83), (512, 100)])
def test_dynamic_dispatch_bit_identical(precision, layout, nx, ny):
    """Interior tiles by tensor copies, wrapping and ragged tiles by plain loads;
    default grids, then 4 and 1 blocks (each block takes many tiles), 101 steps."""
    from paper_1809_02390_gb300 import capi

    if precision == "fp16s":
        nx -= nx % 8
    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(nx, ny, min(nx, ny) / 4, 5, p.rho_g, p.rho_l, center=(0.41 * nx, 0.53 * ny))
    dyn, sta = _pair(rho0, precision, layout, Tr=0.85, K_int=1.0)
    for blocks, steps in ((0, 40), (4, 30), (1, 11), (0, 20)):
        for lat in (dyn, sta):
            capi.lb_set_step_blocks(lat.h, blocks)
            lat.step(steps)
        torch.cuda.synchronize()
        assert torch.equal(dyn.state(), sta.state()), (blocks, steps)
    capi.lb_status(dyn.h)
    capi.lb_set_tile_dispatch(sta.h, True)  # and back


def test_dynamic_dispatch_matches_oracle(orc):
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(208, 83, 20, 5, p.rho_g, p.rho_l, center=(100.3, 40.6))
    lat = lattice(rho0, "fp32", layout="rows", Tr=0.85, K_int=1.0)
    assert capi.lb_tile_dispatch(lat.h)
    lat.step(300)
    ref = orc.macro(p, orc.step(p, orc.init_feq(p, rho0), 300))[0]
    assert rel_inf(lat.moments(velocity=False).double().cpu().numpy(), ref) <= 2e-5
    capi.lb_status(lat.h)


def test_dynamic_dispatch_full_size_bit_identical():
    """4096 x 4096 FP32 spinodal lattice, rows layout (the benchmark's workload and
    launch configuration): 6 launches of each form agree bit for bit."""
    p = oracle_params(Tr=0.8, K_int=1.0)
    n = 4096
    rho0 = inputs.spinodal(n, n, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=0)
    dyn, sta = _pair(rho0, "fp32", "rows", Tr=0.8, K_int=1.0)
    dyn.step(6)
    sta.step(6)
    torch.cuda.synchronize()
    assert torch.equal(dyn.state(), sta.state())
    assert dyn.reduce() == sta.reduce()


def test_dispatch_not_available_without_tensor_copies():
    from paper_1809_02390_gb300 import capi

    p = oracle_params(Tr=0.85, K_int=1.0)
    rho0 = inputs.droplet(150, 96, 20, 5, p.rho_g, p.rho_l)  # nx % 4 != 0: plain fused kernel
    lat = lattice(rho0, "fp32", Tr=0.85, K_int=1.0)
    assert not capi.lb_uses_tma(lat.h) and not capi.lb_tile_dispatch(lat.h)
    with pytest.raises(capi.LBError) as ei:
        capi.lb_set_tile_dispatch(lat.h, True)
    assert ei.value.code == capi.LB_ENOTSUP


@pytest.mark.parametrize("precision,variant,layout,shape", [("fp32", "fused", "rows", (160, 96)),
                                                            ("fp32", "fused", "planes", (70, 45)),
                                                            ("fp64", "fused", "planes", (64, 64)),
                                                            ("fp32", "two_pass", "planes", (64, 48)),
                                                            ("fp16s", "fused", "rows", (160, 96)),
                                                            ("fp16s", "two_pass", "planes", (64, 48))])
def test_graph_replayed_steps_equal_direct_launches(precision, variant, layout, shape):
    """lb_step replays runs of 64 steps from a captured graph on the handle's own
    stream (FP16 stores seed from the step count, which the replayed steps read from
    a device word set before each replay); the result is bit-identical to launching
    the steps one call at a time, including after the launch configuration changes
    (the graph is captured again)."""
    from paper_1809_02390_gb300 import Lattice, capi, derive

    nx, ny = shape
    d = derive(nx, ny, Tr=0.85)
    rho0 = inputs.droplet(nx, ny, min(nx, ny) / 4, 5, d["rho_g"], d["rho_l"])
    a = Lattice(rho0, precision=precision, variant=variant, layout=layout, Tr=0.85)
    b = Lattice(rho0, precision=precision, variant=variant, layout=layout, Tr=0.85)
    a.step(2 * 64 + 7)
    for _ in range(2 * 64 + 7):
        b.step(1)
    torch.cuda.synchronize()
    assert torch.equal(a.buffer(), b.buffer())
    if capi.lb_uses_tma(a.h):
        capi.lb_set_step_blocks(a.h, 40)
        capi.lb_set_step_blocks(b.h, 40)
    a.step(64)
    for _ in range(64):
        b.step(1)
    torch.cuda.synchronize()
    assert torch.equal(a.buffer(), b.buffer())
    assert a.steps_done == b.steps_done == 2 * 64 + 7 + 64
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_graph_replay_follows_buffer_flips_and_new_states(precision):
    """The step graphs are captured per starting buffer: a run after lb_stream_copy
    (same state, the other buffer current) and after lb_set_state (a new state in
    the current buffer) equals single launches bit for bit."""
    from paper_1809_02390_gb300 import Lattice, capi, derive

    d = derive(160, 96, Tr=0.85)
    rho0 = inputs.droplet(160, 96, 24, 5, d["rho_g"], d["rho_l"])
    a = Lattice(rho0, precision=precision, layout="rows", Tr=0.85)
    b = Lattice(rho0, precision=precision, layout="rows", Tr=0.85)

    def same_run(n):
        a.step(n)
        for _ in range(n):
            b.step(1)
        torch.cuda.synchronize()
        assert torch.equal(a.state(), b.state())

    same_run(64)
    for lat in (a, b):
        capi.lb_stream_copy(lat.h)
    same_run(64 + 5)
    other = a.buffer().clone()  # an earlier state, in the lattices' own layout
    same_run(64)
    for lat in (a, b):
        capi.lb_set_state(lat.h, other.data_ptr())
    same_run(128)
    a.close()
    b.close()


def test_steps_inside_a_callers_graph_capture():
    """A caller that captures its own stream into a CUDA graph (here torch's
    CUDAGraph) gets plain launches from lb_step, which the graph records: one
    replay of 70 captured steps equals 70 steps run directly, bit for bit."""
    from paper_1809_02390_gb300 import Lattice, derive

    d = derive(160, 96, Tr=0.85)
    rho0 = inputs.droplet(160, 96, 24, 5, d["rho_g"], d["rho_l"])
    s = torch.cuda.Stream()
    a = Lattice(rho0, precision="fp32", layout="rows", Tr=0.85, stream=s)
    b = Lattice(rho0, precision="fp32", layout="rows", Tr=0.85)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        a.step(70)
    g.replay()
    b.step(70)
    torch.cuda.synchronize()
    assert torch.equal(a.state(), b.state())
    a.close()
    b.close()
