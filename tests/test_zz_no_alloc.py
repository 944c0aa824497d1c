"""lb_reduce_static: the lattice diagnostics of lb_reduce without any device allocation.

Some programs cannot call cudaMalloc: a host whose own allocator has taken
every byte of the GPU, or a plugin running inside such a host, which gets its
lattice from the host and has no allocator of its own.  They can still get the
reductions (mass, momentum, probe pressures, liquid count, density range) from
lb_reduce_static, which keeps its scratch in a static device array inside the
library, committed when the handle is created.  These tests call it through the
C ABI and check that it returns exactly what lb_reduce returns, call after call,
that a call changes neither the device's free memory nor torch's pool, and that
it still works once the GPU's memory has been filled.

This file is collected last on purpose: it runs after every other test, and
it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1809_02390_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("mass", "mom_x", "mom_y", "p_center", "p_corner", "n_liquid", "rho_min", "rho_max")
TOL = 1e-13  # the FP64 tolerance of the other reduction tests; both paths run the same kernels


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_02390_gb300 import build

    build.build()


def _droplet(nx, ny):
    from paper_1809_02390_gb300 import derive

    d = derive(nx, ny, Tr=0.85)
    rng = np.random.default_rng(11)
    rho = inputs.droplet(nx, ny, min(nx, ny) / 4, 5, d["rho_g"], d["rho_l"])
    return rho * (1 + 0.002 * rng.uniform(-1, 1, rho.shape))


def _same(a, b):
    for k, x, y in zip(KEYS, a, b):
        assert x == pytest.approx(y, rel=TOL, abs=1e-12), k


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_matches_lb_reduce_on_consecutive_calls(precision):
    from paper_1809_02390_gb300 import Lattice, capi

    lat = Lattice(_droplet(96, 80), precision=precision, Tr=0.85)
    lat.step(37)
    first = capi.lb_reduce_static(lat.h)
    _same(first, capi.lb_reduce(lat.h))
    lat.step(23)
    second = capi.lb_reduce_static(lat.h)
    _same(second, capi.lb_reduce(lat.h))
    # The second call reflects the new state, not what the first call left behind.
    assert second[6] != first[6] or second[7] != first[7]
    lat.close()


def test_works_on_a_handle_created_without_scratch():
    """A caller that allocated no scratch at all: lb_reduce must refuse, the
    static variant must give the same numbers as a lattice that has scratch."""
    from paper_1809_02390_gb300 import Lattice, capi, params

    rho = _droplet(64, 72)
    ref = Lattice(rho, precision="fp64", Tr=0.85)
    p = params(64, 72, precision="fp64", Tr=0.85)
    f_a = torch.empty((9, 72, 64), dtype=torch.float64, device="cuda")
    f_b = torch.empty_like(f_a)
    rho_dev = torch.from_numpy(rho).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    h = capi.lb_init(p, f_a.data_ptr(), f_b.data_ptr(), 0, 0, rho_dev.data_ptr(), True, stream)
    try:
        for n in (5, 40):
            capi.lb_step(h, n)
            ref.step(n)
            with pytest.raises(capi.LBError) as ei:
                capi.lb_reduce(h)
            assert ei.value.code == capi.LB_ENOMEM
            _same(capi.lb_reduce_static(h), capi.lb_reduce(ref.h))
    finally:
        capi.lb_free(h)
        ref.close()


def test_rejects_lattices_above_its_limit():
    from paper_1809_02390_gb300 import Lattice, capi

    nx, ny = 1100, 1000  # 1.1 M nodes > LB_REDUCE_STATIC_MAX_NODES
    lat = Lattice(np.full((ny, nx), 3.0), precision="fp32", Tr=0.85)
    out = (ctypes.c_double * 8)()
    rc = capi.lib().lb_reduce_static(lat.h, out)
    assert rc == capi.LB_ENOMEM
    assert "static scratch" in capi.lb_last_error(lat.h)
    lat.close()


def test_calls_allocate_nothing():
    """Free device memory (cudaMemGetInfo) and torch's reserved pool are the same
    before and after a run of calls (after one warm-up call)."""
    from paper_1809_02390_gb300 import Lattice, capi

    lat = Lattice(_droplet(128, 96), precision="fp32", Tr=0.85)
    lat.step(10)
    first = capi.lb_reduce_static(lat.h)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(5):
        _same(capi.lb_reduce_static(lat.h), first)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    lat.close()


def test_works_after_the_gpu_memory_is_filled():
    """The caller this entry point is for: after the handle exists, another
    allocator takes (nearly) all free device memory; lb_reduce_static still
    returns the reductions, because its array was committed by lb_init."""
    from paper_1809_02390_gb300 import Lattice, capi

    lat = Lattice(_droplet(96, 96), precision="fp64", Tr=0.85)
    lat.step(15)
    want = capi.lb_reduce(lat.h)
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    hog = torch.empty(max(free - (96 << 20), 0), dtype=torch.uint8, device="cuda")
    try:
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after < (256 << 20)
        _same(capi.lb_reduce_static(lat.h), want)
        _same(capi.lb_reduce_static(lat.h), want)
    finally:
        del hog
        torch.cuda.empty_cache()
    lat.close()
