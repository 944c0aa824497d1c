"""The batched solver (one persistent launch per step over the tiles of many
lattices, CUDA-graph replay, autotuned launch shape) gives every lattice exactly
the trajectory the single-lattice step gives it."""
import numpy as np
import pytest

from gpu_util import oracle_params, rel_inf
from paper_1809_02390_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_02390_gb300 import build

    build.build()


CASES = [((64, 64), 0.85, 1.0, "droplet"), ((100, 70), 0.7, 1.6, "slab"), ((33, 45), 0.9, 1.0, "droplet"),
         ((130, 96), 0.8, 1.3, "slab"), ((40, 40), 0.75, 1.2, "droplet"), ((17, 23), 0.85, 1.0, "slab")]


def _inputs():
    from paper_1809_02390_gb300 import derive

    rhos, kws = [], []
    for (nx, ny), tr, kint, shape in CASES:
        d = derive(nx, ny, Tr=tr, K_int=kint)
        if shape == "droplet":
            r = inputs.droplet(nx, ny, min(nx, ny) / 4, 4, d["rho_g"], d["rho_l"])
        else:
            r = inputs.slab(nx, ny, nx / 2, 4, d["rho_g"], d["rho_l"])
        rhos.append(r)
        kws.append(dict(Tr=tr, K_int=kint))
    return rhos, kws


def _singles(rhos, kws, steps):
    from paper_1809_02390_gb300 import Lattice

    out = []
    for r, kw in zip(rhos, kws):
        lat = Lattice(r, precision="fp32", **kw)
        lat.step(steps)
        out.append(lat.state().clone())
        lat.close()
    return out


@pytest.mark.parametrize("steps", [37, 64 * 2 + 5])
def test_batch_equals_single_lattices(steps):
    from paper_1809_02390_gb300 import Batch

    rhos, kws = _inputs()
    b = Batch(rhos, [dict(k) for k in kws])
    b.run(steps)
    ref = _singles(rhos, kws, steps)
    for i in range(len(rhos)):
        assert torch.equal(b.state(i), ref[i]), i
    b.close()


def test_autotune_keeps_the_trajectory():
    from paper_1809_02390_gb300 import Batch

    rhos, kws = _inputs()
    b = Batch(rhos, [dict(k) for k in kws])
    ms = b.tune(4)
    cfg = b.config()
    assert ms > 0 and cfg["tile_y"] in (16, 32) and cfg["blocks_per_sm"] >= 0  # 0: one block per tile
    b.run(70)
    ref = _singles(rhos, kws, b.steps_done)
    for i in range(len(rhos)):
        assert torch.equal(b.state(i), ref[i]), i
    b.close()


def test_batch_lattice_matches_oracle(orc):
    from paper_1809_02390_gb300 import Batch

    p = oracle_params(Tr=0.85, K_int=1.0)
    r = inputs.droplet(48, 40, 10, 4, p.rho_g, p.rho_l)
    other = inputs.slab(70, 30, 35, 4, p.rho_g, p.rho_l)
    b = Batch([other, r], [dict(Tr=0.8), dict(Tr=0.85, K_int=1.0)])
    b.run(100)
    ref = orc.macro(p, orc.step(p, orc.init_feq(p, r), 100))[0]
    assert rel_inf(b.density(1).cpu().numpy(), ref) <= 2e-5
    b.close()


@pytest.mark.parametrize("shape,bps", [(0, 0), (0, 2), (1, 1), (2, 0), (3, 1), (3, 3), (4, 1), (4, 2), (5, 1), (5, 3),
                                       (6, 1), (6, 2)])
def test_every_launch_form_equals_single_lattices(shape, bps):
    """Each launch form by hand (plain loads one block per tile or persistent,
    tensor copies persistent at both register budgets, walking the tile list
    statically or taking tiles by ticket; the ticket counter must be reset between
    launches for the replayed steps to match), with a 512 x 256 lattice
    added so that persistent blocks walk several tiles (mixed interior and wrapping
    tiles, lattices with and without a padded row stride), in graph replay and
    single launches: bit-identical to the single-lattice step; no wait gave up."""
    from paper_1809_02390_gb300 import Batch, derive

    rhos, kws = _inputs()
    d = derive(512, 256, Tr=0.8)
    rhos.append(inputs.spinodal(512, 256, 0.5 * (d["rho_g"] + d["rho_l"]), 0.01, 3))
    kws.append(dict(Tr=0.8))
    b = Batch(rhos, [dict(k) for k in kws])
    b.set_config(shape, bps)
    assert b.config()["tensor_copies"] == (shape >= 3)
    b.run(64 + 7)
    b.status()
    ref = _singles(rhos, kws, 64 + 7)
    for i in range(len(rhos)):
        assert torch.equal(b.state(i), ref[i]), i
    b.close()


def test_set_config_rejects_bad_forms():
    from paper_1809_02390_gb300 import Batch, capi

    rhos, kws = _inputs()
    b = Batch(rhos, [dict(k) for k in kws])
    for shape, bps in [(7, 1), (-1, 0), (3, 0), (5, 0), (0, 1000)]:
        with pytest.raises(capi.LBError):
            b.set_config(shape, bps)
    b.close()


@pytest.mark.parametrize("shape,bps", [(0, 0), (1, 1), (3, 1), (5, 1), (6, 2)])
def test_rows_layout_batch_equals_single_lattices(shape, bps):
    """Pools in the rows layout f[ny][9][sx] (padded rows; tensor maps with dimensions
    (x, plane, y)): every launch form gives each lattice the single-lattice
    trajectory bit for bit (the layouts share the arithmetic), in graph replay and
    single launches."""
    from paper_1809_02390_gb300 import Batch, derive

    rhos, kws = _inputs()
    d = derive(512, 256, Tr=0.8)
    rhos.append(inputs.spinodal(512, 256, 0.5 * (d["rho_g"] + d["rho_l"]), 0.01, 3))
    kws.append(dict(Tr=0.8))
    b = Batch(rhos, [dict(k, layout="rows") for k in kws])
    b.set_config(shape, bps)
    b.run(64 + 7)
    b.status()
    ref = _singles(rhos, kws, 64 + 7)
    for i in range(len(rhos)):
        assert torch.equal(b.state(i), ref[i]), i
    b.close()


def test_status_names_the_lattices_that_go_non_finite(orc):
    """Lattice 125 of the 256-lattice benchmark set (side 133, vdW, Tr = 0.6642,
    W = 3.29 droplet) is past the method's stability limit: the FP64 oracle itself
    goes non-finite within 60 steps.  In a batch next to two stable lattices,
    lb_batch_status reports LB_ENONFINITE naming it, lb_batch_nonfinite counts its
    nodes, and the stable lattices stay finite and equal to their single runs."""
    from oracle import params as op
    from oracle import thermo
    from paper_1809_02390_gb300 import Batch, capi, derive

    sp = inputs.batch_specs(256, 0)[125]
    assert sp["nx"] == 133 and sp["shape"] == "droplet"
    e = thermo.make_eos("vdw", 9 / 49, 2 / 21, 1.0, sp["Tr"])
    k_int = sp["W"] / thermo.interface(e, 1.0)["W"]
    p = op.from_physical(Tr=sp["Tr"], K_int=k_int)
    bad_rho = inputs.droplet(133, 133, 133 / 4, sp["W"], p.rho_g, p.rho_l)
    assert not np.isfinite(orc.step(p, orc.init_feq(p, bad_rho), 60)).all()

    rhos, kws = _inputs()
    rhos = [rhos[0], bad_rho, rhos[3]]
    kws = [kws[0], dict(Tr=sp["Tr"], K_int=k_int), kws[3]]
    b = Batch(rhos, kws)
    b.run(100)
    with pytest.raises(capi.LBError) as ei:
        b.status()
    assert ei.value.code == capi.LB_ENONFINITE and "non-finite densities: 1" in str(ei.value)
    n_bad, counts = capi.lb_batch_nonfinite(b.b, 3)
    assert n_bad == 1 and b.nonfinite() == [1]
    assert counts[0] == 0 and counts[2] == 0 and 0 < counts[1] <= 133 * 133
    singles = _singles([rhos[0], rhos[2]], [kws[0], kws[2]], 100)
    for i, ref in zip((0, 2), singles):
        assert torch.equal(b.state(i), ref)
    b.close()


def test_batch_steps_inside_a_callers_graph_capture():
    """A batch whose stream the caller captures into its own CUDA graph records
    plain launches: one replay of 70 captured steps equals 70 single-lattice steps."""
    from paper_1809_02390_gb300 import Batch

    rhos, kws = _inputs()
    s = torch.cuda.Stream()
    b = Batch(rhos, kws, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(70)
    g.replay()
    torch.cuda.synchronize()
    ref = _singles(rhos, kws, 70)
    for i in range(len(rhos)):
        assert torch.equal(b.state(i), ref[i]), i
    b.close()
