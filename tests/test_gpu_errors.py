"""Error paths of the library on the GPU: rejected initial densities, non-finite
states reported by the reductions, and bounded waits reported per handle.  No
kernel here faults or hangs: bad values are made on the host and loaded through
the C ABI, and the give-up comes from a wait that nothing completes."""
import ctypes

import numpy as np
import pytest

from paper_1809_02390_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_02390_gb300 import build

    build.build()


def _init_raw(rho_host, **kw):
    """lb_init from a host density array; returns (rc, message, handle, buffers)."""
    from paper_1809_02390_gb300 import capi, params

    ny, nx = rho_host.shape
    p = params(nx, ny, precision="fp32", **kw)
    f_a = torch.empty((9, ny, nx), dtype=torch.float32, device="cuda")
    f_b = torch.empty_like(f_a)
    rho = np.ascontiguousarray(rho_host, dtype=np.float64)
    h = ctypes.c_void_p()
    rc = capi.lib().lb_init(ctypes.byref(h), ctypes.byref(p), ctypes.c_void_p(f_a.data_ptr()),
                            ctypes.c_void_p(f_b.data_ptr()), None, 0, rho.ctypes.data_as(ctypes.c_void_p), 0,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, capi.lb_last_error(None), h, (f_a, f_b)


@pytest.mark.parametrize("bad,needle", [(-1.0, "not positive and finite"), (float("nan"), "not positive and finite"),
                                        (float("inf"), "not positive and finite"), (0.0, "not positive and finite"),
                                        (10.5, "exceeds 1/b")])
def test_init_rejects_bad_host_densities_with_the_first_node(bad, needle):
    """Host densities are checked on the device after the copy: the smallest bad
    node index is reported, positivity before the vdW bound 1 - b rho > 0."""
    from paper_1809_02390_gb300 import capi

    rho = np.full((20, 24), 3.0)
    rho[7, 5] = bad            # node 173
    rho[15, 2] = 11.0          # above 1/b = 10.5 as well, later node
    rc, msg, h, _ = _init_raw(rho, Tr=0.85)
    assert rc == capi.LB_EINVAL and not h.value
    assert "node 173" in msg and needle in msg
    # A good field initialises, and the handle works.
    rho[7, 5] = 3.0
    rho[15, 2] = 3.0
    rc, msg, h, bufs = _init_raw(rho, Tr=0.85)
    assert rc == capi.LB_OK, msg
    assert capi.lib().lb_step(h, 3) == capi.LB_OK
    capi.lib().lb_free(h)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_reductions_report_a_non_finite_state(precision):
    """A state with one NaN population, made on the host and loaded by lb_set_state:
    lb_reduce and lb_reduce_static both return LB_ENONFINITE (the sums are still
    written), and a clean state reduces without error again."""
    from paper_1809_02390_gb300 import Lattice, capi, derive

    d = derive(64, 48, Tr=0.85)
    lat = Lattice(inputs.droplet(64, 48, 12, 5, d["rho_g"], d["rho_l"]), precision=precision, Tr=0.85)
    lat.step(5)
    good = lat.buffer().clone()
    bad = good.clone()
    bad[3, 20, 30] = float("nan")
    capi.lb_set_state(lat.h, bad.data_ptr())
    for fn in (capi.lb_reduce, capi.lb_reduce_static):
        with pytest.raises(capi.LBError) as ei:
            fn(lat.h)
        assert ei.value.code == capi.LB_ENONFINITE and "non-finite" in str(ei.value)
    capi.lb_set_state(lat.h, good.data_ptr())
    a, b = capi.lb_reduce(lat.h), capi.lb_reduce_static(lat.h)
    assert a == b and np.isfinite(a).all()
    lat.close()


def test_wait_give_up_is_reported_on_its_own_handle():
    """Each handle has its own wait flag: a give-up on one handle is reported by
    lb_status on that handle (and cleared), while another handle on the same
    device stays clean and keeps stepping."""
    from paper_1809_02390_gb300 import Lattice, capi, derive

    d = derive(128, 64, Tr=0.85)
    rho = inputs.droplet(128, 64, 16, 5, d["rho_g"], d["rho_l"])
    a, b = Lattice(rho, precision="fp32", Tr=0.85), Lattice(rho, precision="fp32", Tr=0.85)
    rc = capi.lib().lb_wait_selftest(a.h, 1000)
    assert rc == capi.LB_ETIMEOUT
    capi.lb_status(b.h)          # raises if b saw a's give-up
    capi.lb_status(a.h)          # cleared by the read
    a.step(10)
    b.step(10)
    torch.cuda.synchronize()
    assert torch.equal(a.buffer(), b.buffer())
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_zero_steps_change_nothing_and_negative_counts_are_rejected(precision):
    """lb_step(h, 0) and lb_batch_run(b, 0) leave the state and the step count as
    they are; a negative count is LB_EINVAL and launches nothing."""
    from paper_1809_02390_gb300 import Batch, Lattice, capi, derive

    d = derive(96, 64, Tr=0.85)
    rho0 = inputs.droplet(96, 64, 16, 5, d["rho_g"], d["rho_l"])
    lat = Lattice(rho0, precision=precision, Tr=0.85)
    lat.step(3)
    torch.cuda.synchronize()
    before = lat.buffer().clone()
    lat.step(0)
    with pytest.raises(capi.LBError) as ei:
        lat.step(-1)
    assert ei.value.code == capi.LB_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(lat.buffer(), before) and lat.steps_done == 3
    lat.close()
    if precision == "fp32":
        b = Batch([rho0, rho0[:40, :50]], [dict(Tr=0.85)] * 2)
        b.run(2)
        s0 = b.state(1).clone()
        b.run(0)
        with pytest.raises(capi.LBError):
            b.run(-5)
        assert torch.equal(b.state(1), s0) and b.steps_done == 2
        b.close()
