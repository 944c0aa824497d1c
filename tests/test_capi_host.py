"""CPU tests of the C ABI: the library loads, exports every declared entry
point, derives the same lattice parameters as the oracle (host-only code),
and rejects invalid input with clear errors before touching a GPU."""
import ctypes
import os
import re

import pytest

from oracle import params as op
from oracle import thermo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1809_02390_gb300 import build as b

    b.build()
    from paper_1809_02390_gb300 import capi as c

    return c


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(lb_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(capi):
    lib = capi.lib()
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names |= _declared(h)
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    bound = {n for n, _, _ in capi.SIGNATURES}
    assert names <= bound | {n for n in names if n.startswith("lb_batch") or n.startswith("lb_adjoint")}


def test_abi_struct_sizes(capi):
    assert ctypes.sizeof(capi.lb_params) == 8 * 4 + 16 * 8
    assert capi.lb_params.layout.offset == 6 * 4 + 16 * 8
    assert ctypes.sizeof(capi.lb_derived) == 20 * 8
    assert capi.lib().lb_abi_version() == 2


@pytest.mark.parametrize("eos,a,b,Tr,K_int", [("vdw", 9 / 49, 2 / 21, 0.85, 1.0), ("vdw", 9 / 49, 2 / 21, 0.7, 1.7),
                                              ("cs", 1.0, 4.0, 0.8, 2.2949), ("cs", 1.0, 4.0, 0.6, 1.0)])
def test_derived_parameters_match_oracle(capi, eos, a, b, Tr, K_int):
    p = capi.make_params(64, 64, eos=capi.LB_EOS_VDW if eos == "vdw" else capi.LB_EOS_CS, eos_a=a, eos_b=b,
                         Tr=Tr, K_int=K_int, K_eos=2.0)
    d = capi.lb_derive(p)
    o = op.from_physical(eos=eos, a=a, b=b, Tr=Tr, K_int=K_int, K_eos=2.0)
    for k_lib, k_or in [("rho_g", "rho_g"), ("rho_l", "rho_l"), ("lam", "lam"), ("G2", "G2"), ("s_e", "se"),
                        ("s_q", "sq"), ("s_eps", "seps"), ("s_p", "sp"), ("T", "T"), ("Tc", "Tc")]:
        assert d[k_lib] == pytest.approx(getattr(o, k_or), rel=1e-12), k_lib
    it = thermo.interface(thermo.make_eos(eos, a, b, 1.0, Tr, K_eos=2.0), 1.0)
    assert d["W1"] == pytest.approx(it["W"], rel=1e-9)
    assert d["sigma1"] == pytest.approx(it["sigma"], rel=1e-9)
    assert d["k"] == pytest.approx(5 / 6) and d["b"] == pytest.approx(5 / 3) and d["h"] == pytest.approx(5 / 3)
    assert d["beta2"] == pytest.approx(-2.4)


@pytest.mark.parametrize("field,value,needle", [
    ("nx", 2, "nx and ny"), ("varpi", 1.0, "varpi"), ("varpi", 1 / 3, "varpi"), ("s_p", 2.0, "s_p"),
    ("s_p", 0.0, "s_p"), ("eos", 7, "eos"), ("precision", 5, "precision"), ("Tr", 1.2, "coexistence"),
    ("eos_b", -1.0, "eos_a"), ("s_q", 2.5, "rates"), ("layout", 2, "layout"), ("reserved1", 1, "reserved")])
def test_invalid_parameters_are_rejected(capi, field, value, needle):
    p = capi.make_params(64, 64)
    setattr(p, field, value)
    with pytest.raises(capi.LBError) as ei:
        capi.lb_derive(p)
    assert ei.value.code == capi.LB_EINVAL and needle in str(ei.value)


def test_init_rejects_bad_input_before_any_gpu_work(capi):
    import numpy as np

    p = capi.make_params(8, 8)
    rho = np.full(64, 2.0)
    rho[5] = -1.0
    h = ctypes.c_void_p()
    buf = (ctypes.c_char * 16)()
    rc = capi.lib().lb_init(ctypes.byref(h), ctypes.byref(p), ctypes.addressof(buf), ctypes.addressof(buf),
                            None, 0, rho.ctypes.data, 0, None)
    assert rc == capi.LB_EINVAL  # identical f buffers
    # (A density that is not positive is rejected on the device, after the copy:
    # tests/test_gpu_errors.py.)
    p.variant = capi.LB_TWO_PASS
    rho[5] = 2.0
    rc = capi.lib().lb_init(ctypes.byref(h), ctypes.byref(p), 1 << 40, 2 << 40, None, 0, rho.ctypes.data, 0, None)
    assert rc == capi.LB_ENOMEM


def test_sizes(capi):
    p = capi.make_params(100, 30, precision=capi.LB_FP16S)
    assert capi.lb_state_bytes(p) == 9 * 100 * 30 * 2
    p.precision = capi.LB_FP64
    assert capi.lb_state_bytes(p) == 9 * 100 * 30 * 8
    assert capi.lb_scratch_bytes(p) >= 100 * 30 * 8


def test_batch_rejects_mixed_layouts_before_any_gpu_work(capi):
    """The lattices of one batch share the layout of its pools: a batch mixing planes
    and rows is refused with LB_ENOTSUP on the host (the buffers are never touched)."""
    import numpy as np

    ps = (capi.lb_params * 2)(capi.make_params(64, 64), capi.make_params(64, 64, layout=capi.LB_LAYOUT_ROWS))
    rho = np.full(2 * 64 * 64, 2.0)
    b = ctypes.c_void_p()
    meta = capi.lib().lb_batch_meta_bytes(ps, 2)
    rc = capi.lib().lb_batch_init(ctypes.byref(b), ps, 2, 1 << 40, 2 << 40, 3 << 40, meta, rho.ctypes.data, 0, None)
    assert rc == capi.LB_ENOTSUP and "share the layout" in capi.lb_last_error(None)


def test_batch_with_automatic_shifts_validates_before_any_gpu_work(capi):
    """rho_ref = NaN makes lb_batch_init sum densities on the device, but only after
    every lattice's parameters are checked: a batch whose second lattice has no two
    phases (Tr > 1) is refused with LB_EINVAL on the host (on a machine without a
    GPU, any device work would have failed with LB_ECUDA instead)."""
    import numpy as np

    a = capi.make_params(64, 64)
    bad = capi.make_params(64, 64, Tr=1.2)
    for q in (a, bad):
        q.rho_ref = float("nan")
    ps = (capi.lb_params * 2)(a, bad)
    rho = np.full(2 * 64 * 64, 2.0)
    b = ctypes.c_void_p()
    meta = capi.lib().lb_batch_meta_bytes(ps, 2)
    rc = capi.lib().lb_batch_init(ctypes.byref(b), ps, 2, 1 << 40, 2 << 40, 3 << 40, meta, rho.ctypes.data, 0, None)
    assert rc == capi.LB_EINVAL and not b.value


def test_new_entry_points_reject_null_handles(capi):
    """The equilibrium, dispatch and tuning calls check their handle
    before any GPU work."""
    lib = capi.lib()
    assert lib.lb_set_equilibrium(None, None, None, None) == capi.LB_EINVAL
    assert lib.lb_set_tile_dispatch(None, 1) == capi.LB_EINVAL
    assert lib.lb_tile_dispatch(None) == 0
    assert lib.lb_set_step_blocks(None, 0) == capi.LB_EINVAL
    assert lib.lb_uses_tma(None) == 0


def test_scratch_holds_the_tile_tickets(capi):
    """Scratch = one density plane (rounded to 256 bytes) + the reduction workspace
    + 256 bytes of tile tickets; FP16 and FP32 planes are float, FP64 double."""
    p = capi.make_params(100, 30, precision=capi.LB_FP32)
    q = capi.make_params(100, 30, precision=capi.LB_FP64)
    plane32 = (100 * 30 * 4 + 255) // 256 * 256
    plane64 = (100 * 30 * 8 + 255) // 256 * 256
    assert capi.lb_scratch_bytes(q) - capi.lb_scratch_bytes(p) == plane64 - plane32
    assert capi.lb_scratch_bytes(p) >= plane32 + 256


def test_size_limit_of_32_bit_offsets(capi):
    """The kernels index populations with 32-bit offsets: 9 nx ny must stay below
    2^31.  15446^2 and 16384 x 14563 are accepted, one node row more is not."""
    ok = capi.lb_derive(capi.make_params(15446, 15446))
    assert ok["rho_l"] > ok["rho_g"]
    capi.lb_derive(capi.make_params(16384, 14563))
    for nx, ny in ((15447, 15447), (16384, 14564)):
        with pytest.raises(capi.LBError) as ei:
            capi.lb_derive(capi.make_params(nx, ny))
        assert ei.value.code == capi.LB_EINVAL and "too large" in str(ei.value)


def test_storage_shift_nan_means_the_mean_density(capi):
    """rho_ref = NaN asks lb_init / lb_batch_init for the mean initial density, so
    lb_derive accepts it; an infinite shift is rejected."""
    p = capi.make_params(64, 64)
    p.rho_ref = float("nan")
    assert capi.lb_derive(p)["rho_l"] > 0
    for bad in (float("inf"), float("-inf")):
        p.rho_ref = bad
        with pytest.raises(capi.LBError) as ei:
            capi.lb_derive(p)
        assert ei.value.code == capi.LB_EINVAL and "rho_ref" in str(ei.value)


def test_null_and_empty_arguments_are_rejected_without_a_gpu(capi):
    """Calls on a null handle or an empty batch return LB_EINVAL before any CUDA
    work: lb_step, lb_moments, lb_reduce, lb_batch_init with n = 0."""
    lib = capi.lib()
    assert lib.lb_step(None, 1) == capi.LB_EINVAL
    assert lib.lb_step(None, -1) == capi.LB_EINVAL
    out = (ctypes.c_double * 8)()
    assert lib.lb_reduce(None, out) == capi.LB_EINVAL
    b = ctypes.c_void_p()
    ps = (capi.lb_params * 1)(capi.make_params(8, 8))
    rc = lib.lb_batch_init(ctypes.byref(b), ps, 0, 1 << 40, 2 << 40, 3 << 40, 1 << 20, None, 0, None)
    assert rc == capi.LB_EINVAL and not b.value


def test_d3_velocities_are_the_d3q19_set(capi):
    e = capi.lb_d3_velocities()
    assert len(set(e)) == 19 and e[0] == (0, 0, 0)
    assert sorted(sum(c * c for c in v) for v in e) == [0] + [1] * 6 + [2] * 12
    assert all(e[2 * P + 2] == tuple(-c for c in e[2 * P + 1]) for P in range(9))


@pytest.mark.parametrize("varpi,s_p", [(1 / 6, 1.0), (0.3, 1.25), (0.05, 0.8)])
def test_d3_derived_parameters_match_the_3d_oracle(capi, varpi, s_p):
    """The library's 3-D coefficients and closure against the D3Q19 oracle's (host
    code on both sides; the oracle's are pinned in tests/test_oracle_d3q19.py)."""
    from oracle import d3q19

    d3q19.build()
    p = capi.make_params(40, 20, Tr=0.8, K_int=1.5, varpi=varpi, s_p=s_p)
    d = capi.lb_d3_derive(p, 10)
    o = op.from_physical_3d(Tr=0.8, K_int=1.5, varpi=varpi, s_p=s_p)
    c = d3q19.coefficients(o)
    for k_lib, v in (("s_e", o.se), ("s_q", o.sq), ("s_eps", o.seps), ("lam", o.lam), ("G2", o.G2),
                     ("rho_g", o.rho_g), ("rho_l", o.rho_l), ("k", c["k"]), ("h", c["h"]), ("b", c["b"]),
                     ("beta2", c["beta2"])):
        assert d[k_lib] == pytest.approx(v, rel=1e-12), k_lib


@pytest.mark.parametrize("field,value,nz,code,needle", [
    ("precision", 2, 4, "ENOTSUP", "FP64 or FP32"), ("layout", 1, 4, "ENOTSUP", "planes"),
    ("variant", 2, 4, "ENOTSUP", "fused"), ("varpi", 7 / 18, 4, "EINVAL", "7/18"), ("varpi", 1.0, 4, "EINVAL", "varpi"),
    ("nx", 0, 4, "EINVAL", ">= 1"), ("nx", 40, 0, "EINVAL", ">= 1"), ("nx", 2048, 512, "EINVAL", "too large"),
    ("s_p", 2.0, 4, "EINVAL", "s_p"), ("Tr", 1.2, 4, "EINVAL", "coexistence")])
def test_d3_invalid_parameters_are_rejected(capi, field, value, nz, code, needle):
    p = capi.make_params(40, 20)
    setattr(p, field, value)
    if field == "nx" and value == 2048:
        p.ny = 2048  # 2048^2 x 512 = 2^31 nodes
    with pytest.raises(capi.LBError) as ei:
        capi.lb_d3_derive(p, nz)
    assert ei.value.code == getattr(capi, "LB_" + code) and needle in str(ei.value)


def test_d3_varpi_one_third_is_regular_in_3d(capi):
    """varpi = 1/3 is singular for the D2Q9 coefficients (h, b of Eq. 7) but not for
    the D3Q19 ones (singular at 7/18)."""
    p = capi.make_params(16, 16, varpi=1 / 3)
    with pytest.raises(capi.LBError):
        capi.lb_derive(p)
    d = capi.lb_d3_derive(p, 16)
    assert d["b"] == pytest.approx(21 * (2 / 3) / (5 * (7 - 6)))


def test_d3_init_rejects_bad_arguments_before_any_gpu_work(capi):
    import numpy as np

    lib = capi.lib()
    p = capi.make_params(8, 8)
    rho = np.full(8 * 8 * 4, 2.0)
    h = ctypes.c_void_p()
    buf = (ctypes.c_char * 16)()
    assert lib.lb_d3_init(ctypes.byref(h), ctypes.byref(p), 4, ctypes.addressof(buf), ctypes.addressof(buf),
                          rho.ctypes.data, 0, None) == capi.LB_EINVAL
    assert lib.lb_d3_init(ctypes.byref(h), ctypes.byref(p), 4, 1 << 40, 2 << 40, None, 0, None) == capi.LB_EINVAL
    assert not h.value
    assert lib.lb_d3_step(None, 1) == capi.LB_EINVAL and lib.lb_d3_moments(None, None, None, None, None) == capi.LB_EINVAL
    assert capi.lb_d3_state_bytes(p, 4) == 19 * 8 * 8 * 4 * 4
    p.precision = capi.LB_FP64
    assert capi.lb_d3_state_bytes(p, 4) == 19 * 8 * 8 * 4 * 8
