"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every function here has the name of the C entry point it calls; device
buffers are torch CUDA tensors (PyTorch provides device memory and streams),
passed as raw pointers.  There is no CPU fallback: loading fails loudly if the
compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

LB_OK, LB_EINVAL, LB_ECUDA, LB_ENOMEM, LB_ENONFINITE, LB_ETIMEOUT, LB_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
LB_FP64, LB_FP32, LB_FP16S = 0, 1, 2
LB_EOS_VDW, LB_EOS_CS = 0, 1
LB_AUTO, LB_FUSED, LB_TWO_PASS = 0, 1, 2
LB_LAYOUT_PLANES, LB_LAYOUT_ROWS = 0, 1


class lb_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("eos", ctypes.c_int32), ("variant", ctypes.c_int32), ("rounding", ctypes.c_int32),
                ("eos_a", ctypes.c_double), ("eos_b", ctypes.c_double), ("R_gas", ctypes.c_double),
                ("Tr", ctypes.c_double), ("K_eos", ctypes.c_double), ("K_int", ctypes.c_double),
                ("G2", ctypes.c_double), ("lam", ctypes.c_double), ("varpi", ctypes.c_double),
                ("s_p", ctypes.c_double), ("s_q", ctypes.c_double), ("s_e", ctypes.c_double),
                ("s_eps", ctypes.c_double), ("s_0", ctypes.c_double), ("s_j", ctypes.c_double),
                ("rho_ref", ctypes.c_double), ("layout", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class lb_derived(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "Tc", "T", "rho_g", "rho_l", "p_star", "lam", "G2", "c2", "s_0", "s_e", "s_eps", "s_j", "s_q", "s_p",
        "k", "h", "b", "beta2", "W1", "sigma1")]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("lbm error %d: %s" % (code, msg))
        self.code = code


_lib = None

# (name, restype, argtypes) of every entry point declared in include/lbm.h.
_P, _V, _D = ctypes.POINTER(lb_params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
SIGNATURES = [
    ("lb_abi_version", ctypes.c_int, []),
    ("lb_derive", ctypes.c_int, [_P, ctypes.POINTER(lb_derived)]),
    ("lb_state_bytes", ctypes.c_size_t, [_P]),
    ("lb_scratch_bytes", ctypes.c_size_t, [_P]),
    ("lb_init", ctypes.c_int, [ctypes.POINTER(_V), _P, _V, _V, _V, ctypes.c_size_t, _V, ctypes.c_int, _V]),
    ("lb_step", ctypes.c_int, [_V, ctypes.c_int64]),
    ("lb_state", _V, [_V]),
    ("lb_steps_done", ctypes.c_int64, [_V]),
    ("lb_moments", ctypes.c_int, [_V, _V, _V, _V]),
    ("lb_reduce", ctypes.c_int, [_V, _D]),
    ("lb_reduce_static", ctypes.c_int, [_V, _D]),
    ("lb_adjoint_scratch_bytes", ctypes.c_size_t, [_P]),
    ("lb_adjoint_step", ctypes.c_int, [_V, _V, _V, _V, _V, _V, ctypes.c_size_t]),
    ("lb_adjoint_steps_scratch_bytes", ctypes.c_size_t, [_P]),
    ("lb_adjoint_steps", ctypes.c_int, [_V, ctypes.POINTER(_V), ctypes.c_int, _V, _V, _V, ctypes.c_size_t]),
    ("lb_batch_pool_bytes", ctypes.c_size_t, [_P, ctypes.c_int]),
    ("lb_batch_meta_bytes", ctypes.c_size_t, [_P, ctypes.c_int]),
    ("lb_batch_init", ctypes.c_int, [ctypes.POINTER(_V), _P, ctypes.c_int, _V, _V, _V, ctypes.c_size_t, _V,
                                     ctypes.c_int, _V]),
    ("lb_batch_run", ctypes.c_int, [_V, ctypes.c_int64]),
    ("lb_batch_tune", ctypes.c_int, [_V, ctypes.c_int, _D]),
    ("lb_batch_config", ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    ("lb_batch_nonfinite", ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_uint32)]),
    ("lb_batch_state", _V, [_V]),
    ("lb_batch_steps_done", ctypes.c_int64, [_V]),
    ("lb_batch_offset", ctypes.c_int64, [_V, ctypes.c_int]),
    ("lb_batch_row_stride", ctypes.c_int, [_V, ctypes.c_int]),
    ("lb_batch_density", ctypes.c_int, [_V, ctypes.c_int, _V]),
    ("lb_batch_uses_tma", ctypes.c_int, [_V]),
    ("lb_batch_set_config", ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int]),
    ("lb_batch_status", ctypes.c_int, [_V]),
    ("lb_batch_derived", ctypes.c_int, [_V, ctypes.c_int, ctypes.POINTER(lb_derived)]),
    ("lb_batch_params", ctypes.c_int, [_V, ctypes.c_int, ctypes.POINTER(lb_params)]),
    ("lb_batch_last_error", ctypes.c_char_p, [_V]),
    ("lb_batch_free", None, [_V]),
    ("lb_get_state", ctypes.c_int, [_V, _V]),
    ("lb_set_state", ctypes.c_int, [_V, _V]),
    ("lb_get_derived", ctypes.c_int, [_V, ctypes.POINTER(lb_derived)]),
    ("lb_get_params", ctypes.c_int, [_V, ctypes.POINTER(lb_params)]),
    ("lb_status", ctypes.c_int, [_V]),
    ("lb_wait_selftest", ctypes.c_int, [_V, ctypes.c_longlong]),
    ("lb_stream_copy", ctypes.c_int, [_V]),
    ("lb_pressure", ctypes.c_int, [_V, _V]),
    ("lb_uses_tma", ctypes.c_int, [_V]),
    ("lb_set_equilibrium", ctypes.c_int, [_V, _V, _V, _V]),
    ("lb_set_tile_dispatch", ctypes.c_int, [_V, ctypes.c_int]),
    ("lb_tile_dispatch", ctypes.c_int, [_V]),
    ("lb_set_step_blocks", ctypes.c_int, [_V, ctypes.c_int]),
    ("lb_last_error", ctypes.c_char_p, [_V]),
    ("lb_free", None, [_V]),
    # D3Q19 form of the step (include/lbm3d.h)
    ("lb_d3_velocities", None, [ctypes.POINTER(ctypes.c_int)] * 3),
    ("lb_d3_derive", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lb_derived)]),
    ("lb_d3_state_bytes", ctypes.c_size_t, [_P, ctypes.c_int32]),
    ("lb_d3_init", ctypes.c_int, [ctypes.POINTER(_V), _P, ctypes.c_int32, _V, _V, _V, ctypes.c_int, _V]),
    ("lb_d3_step", ctypes.c_int, [_V, ctypes.c_int64]),
    ("lb_d3_moments", ctypes.c_int, [_V, _V, _V, _V, _V]),
    ("lb_d3_reduce", ctypes.c_int, [_V, _D]),
    ("lb_d3_state", _V, [_V]),
    ("lb_d3_get_state", ctypes.c_int, [_V, _V]),
    ("lb_d3_set_state", ctypes.c_int, [_V, _V]),
    ("lb_d3_get_params", ctypes.c_int, [_V, ctypes.POINTER(lb_params), ctypes.POINTER(lb_derived)]),
    ("lb_d3_last_error", ctypes.c_char_p, [_V]),
    ("lb_d3_free", None, [_V]),
]


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it was not built: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("the CUDA library %s is not built; run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int, handle=None) -> int:
    if rc != LB_OK:
        msg = lib().lb_last_error(handle)
        raise LBError(rc, msg.decode() if msg else "")
    return rc


def make_params(nx: int, ny: int, precision: int = LB_FP32, eos: int = LB_EOS_VDW, variant: int = LB_FUSED,
                eos_a: float = 9.0 / 49.0, eos_b: float = 2.0 / 21.0, R_gas: float = 1.0, Tr: float = 0.85,
                K_eos: float = 1.0, K_int: float = 1.0, G2: float = 0.0, lam: float = 0.0,
                varpi: float = 1.0 / 6.0, s_p: float = 1.0, s_q: float = 0.0, s_e: float = 0.0,
                s_eps: float = 0.0, s_0: float = 0.0, s_j: float = 0.0, rho_ref: float = 0.0,
                rounding: int = 0, layout: int = LB_LAYOUT_PLANES) -> lb_params:
    return lb_params(nx=nx, ny=ny, precision=precision, eos=eos, variant=variant, rounding=rounding, eos_a=eos_a,
                     eos_b=eos_b, R_gas=R_gas, Tr=Tr, K_eos=K_eos, K_int=K_int, G2=G2, lam=lam, varpi=varpi,
                     s_p=s_p, s_q=s_q, s_e=s_e, s_eps=s_eps, s_0=s_0, s_j=s_j, rho_ref=rho_ref, layout=layout)


def lb_derive(p: lb_params) -> dict:
    d = lb_derived()
    check(lib().lb_derive(ctypes.byref(p), ctypes.byref(d)))
    return d.as_dict()


def lb_state_bytes(p: lb_params) -> int:
    return lib().lb_state_bytes(ctypes.byref(p))


def lb_scratch_bytes(p: lb_params) -> int:
    return lib().lb_scratch_bytes(ctypes.byref(p))


def lb_init(p: lb_params, f_a: int, f_b: int, scratch: int, scratch_bytes: int, rho0: int,
            rho0_on_device: bool, stream: int) -> int:
    h = ctypes.c_void_p()
    check(lib().lb_init(ctypes.byref(h), ctypes.byref(p), f_a, f_b, scratch or None, scratch_bytes, rho0,
                        int(bool(rho0_on_device)), stream or None))
    return h.value


def lb_step(h: int, nsteps: int) -> None:
    check(lib().lb_step(h, int(nsteps)), h)


def lb_state(h: int) -> int:
    return lib().lb_state(h)


def lb_steps_done(h: int) -> int:
    return lib().lb_steps_done(h)


def lb_moments(h: int, rho: int, ux: int | None, uy: int | None) -> None:
    check(lib().lb_moments(h, rho, ux, uy), h)


def lb_reduce(h: int) -> list[float]:
    out = (ctypes.c_double * 8)()
    rc = lib().lb_reduce(h, out)
    vals = list(out)
    if rc not in (LB_OK, LB_ENONFINITE):
        check(rc, h)
    return vals if rc == LB_OK else check(rc, h)


def lb_reduce_static(h: int) -> list[float]:
    """lb_reduce with the library's static device scratch (no allocation anywhere)."""
    out = (ctypes.c_double * 8)()
    rc = lib().lb_reduce_static(h, out)
    if rc not in (LB_OK, LB_ENONFINITE):
        check(rc, h)
    return list(out) if rc == LB_OK else check(rc, h)


def lb_adjoint_scratch_bytes(p: lb_params) -> int:
    return lib().lb_adjoint_scratch_bytes(ctypes.byref(p))


def lb_adjoint_step(h: int, f_state: int, lam_in: int, lam_out: int, dtheta: int | None, scratch: int,
                    scratch_bytes: int) -> None:
    check(lib().lb_adjoint_step(h, f_state, lam_in, lam_out, dtheta, scratch, scratch_bytes), h)


def lb_adjoint_steps_scratch_bytes(p: lb_params) -> int:
    return lib().lb_adjoint_steps_scratch_bytes(ctypes.byref(p))


def lb_adjoint_steps(h: int, states: list[int], lam: int, dtheta: int | None, scratch: int,
                     scratch_bytes: int) -> None:
    arr = (ctypes.c_void_p * len(states))(*states)
    check(lib().lb_adjoint_steps(h, arr, len(states), lam, dtheta, scratch, scratch_bytes), h)


def lb_get_state(h: int, dst: int) -> None:
    check(lib().lb_get_state(h, dst), h)


def lb_set_state(h: int, src: int) -> None:
    check(lib().lb_set_state(h, src), h)


def lb_get_derived(h: int) -> dict:
    d = lb_derived()
    check(lib().lb_get_derived(h, ctypes.byref(d)), h)
    return d.as_dict()


def lb_get_params(h: int) -> lb_params:
    p = lb_params()
    check(lib().lb_get_params(h, ctypes.byref(p)), h)
    return p


def check_batch(rc: int, b=None) -> int:
    if rc != LB_OK:
        msg = lib().lb_batch_last_error(b)
        raise LBError(rc, msg.decode() if msg else "")
    return rc


def lb_batch_pool_bytes(ps) -> int:
    return lib().lb_batch_pool_bytes(ps, len(ps))


def lb_batch_meta_bytes(ps) -> int:
    return lib().lb_batch_meta_bytes(ps, len(ps))


def lb_batch_init(ps, pool_a: int, pool_b: int, meta: int, meta_bytes: int, rho0: int, rho0_on_device: bool,
                  stream: int) -> int:
    b = ctypes.c_void_p()
    check_batch(lib().lb_batch_init(ctypes.byref(b), ps, len(ps), pool_a, pool_b, meta, meta_bytes, rho0,
                                    int(bool(rho0_on_device)), stream or None))
    return b.value


def lb_batch_run(b: int, nsteps: int) -> None:
    check_batch(lib().lb_batch_run(b, int(nsteps)), b)


def lb_batch_tune(b: int, trial_steps: int) -> float:
    ms = ctypes.c_double()
    check_batch(lib().lb_batch_tune(b, int(trial_steps), ctypes.byref(ms)), b)
    return ms.value


def lb_batch_config(b: int) -> dict:
    ty, bps, grid = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check_batch(lib().lb_batch_config(b, ctypes.byref(ty), ctypes.byref(bps), ctypes.byref(grid)), b)
    return {"tile_y": ty.value, "blocks_per_sm": bps.value, "grid": grid.value,
            "tensor_copies": bool(lib().lb_batch_uses_tma(b))}


def lb_batch_set_config(b: int, shape: int, blocks_per_sm: int) -> None:
    check_batch(lib().lb_batch_set_config(b, shape, blocks_per_sm), b)


def lb_batch_status(b: int) -> None:
    check_batch(lib().lb_batch_status(b), b)


def lb_batch_nonfinite(b: int, n: int) -> tuple[int, list[int]]:
    """(number of lattices with a non-finite density, per-lattice node counts)."""
    counts = (ctypes.c_uint32 * n)()
    rc = lib().lb_batch_nonfinite(b, counts)
    if rc < 0:
        check_batch(rc, b)
    return rc, list(counts)


def lb_batch_density(b: int, i: int, rho: int) -> None:
    check_batch(lib().lb_batch_density(b, i, rho), b)


def lb_batch_state(b: int) -> int:
    return lib().lb_batch_state(b)


def lb_batch_steps_done(b: int) -> int:
    return lib().lb_batch_steps_done(b)


def lb_batch_offset(b: int, i: int) -> int:
    return lib().lb_batch_offset(b, i)


def lb_batch_row_stride(b: int, i: int) -> int:
    return lib().lb_batch_row_stride(b, i)


def lb_batch_derived(b: int, i: int) -> dict:
    d = lb_derived()
    check_batch(lib().lb_batch_derived(b, i, ctypes.byref(d)), b)
    return d.as_dict()


def lb_batch_params(b: int, i: int) -> lb_params:
    p = lb_params()
    check_batch(lib().lb_batch_params(b, i, ctypes.byref(p)), b)
    return p


def lb_batch_free(b: int) -> None:
    lib().lb_batch_free(b)


def lb_pressure(h: int, p: int) -> None:
    check(lib().lb_pressure(h, p), h)


def lb_wait_selftest(h: int, polls: int) -> int:
    """Return code of lb_wait_selftest (LB_ETIMEOUT = -5 when the give-up is reported)."""
    return lib().lb_wait_selftest(h, polls)


def lb_stream_copy(h: int) -> None:
    check(lib().lb_stream_copy(h), h)


def lb_status(h: int) -> None:
    check(lib().lb_status(h), h)


def lb_uses_tma(h: int) -> bool:
    return bool(lib().lb_uses_tma(h))


def lb_set_equilibrium(h: int, rho: int, ux: int | None, uy: int | None) -> None:
    check(lib().lb_set_equilibrium(h, rho, ux, uy), h)


def lb_set_tile_dispatch(h: int, dynamic: bool) -> None:
    check(lib().lb_set_tile_dispatch(h, int(dynamic)), h)


def lb_tile_dispatch(h: int) -> bool:
    return bool(lib().lb_tile_dispatch(h))


def lb_set_step_blocks(h: int, blocks: int) -> None:
    check(lib().lb_set_step_blocks(h, blocks), h)


def lb_last_error(h: int | None = None) -> str:
    return lib().lb_last_error(h).decode()


def lb_free(h: int) -> None:
    lib().lb_free(h)


# --- D3Q19 step ------------------------------------------------------------------

def check_d3(rc: int, h=None) -> int:
    if rc != LB_OK:
        msg = lib().lb_d3_last_error(h)
        raise LBError(rc, msg.decode() if msg else "")
    return rc


def lb_d3_velocities() -> list[tuple[int, int, int]]:
    e = [(ctypes.c_int * 19)() for _ in range(3)]
    lib().lb_d3_velocities(*e)
    return list(zip(*[list(a) for a in e]))


def lb_d3_derive(p: lb_params, nz: int) -> dict:
    d = lb_derived()
    check_d3(lib().lb_d3_derive(ctypes.byref(p), int(nz), ctypes.byref(d)))
    return d.as_dict()


def lb_d3_state_bytes(p: lb_params, nz: int) -> int:
    return lib().lb_d3_state_bytes(ctypes.byref(p), int(nz))


def lb_d3_init(p: lb_params, nz: int, f_a: int, f_b: int, rho0: int, rho0_on_device: bool, stream: int) -> int:
    h = ctypes.c_void_p()
    check_d3(lib().lb_d3_init(ctypes.byref(h), ctypes.byref(p), int(nz), f_a, f_b, rho0, int(bool(rho0_on_device)),
                              stream or None))
    return h.value


def lb_d3_step(h: int, nsteps: int) -> None:
    check_d3(lib().lb_d3_step(h, int(nsteps)), h)


def lb_d3_moments(h: int, rho: int, ux: int | None, uy: int | None, uz: int | None) -> None:
    check_d3(lib().lb_d3_moments(h, rho, ux, uy, uz), h)


def lb_d3_reduce(h: int) -> list[float]:
    out = (ctypes.c_double * 8)()
    check_d3(lib().lb_d3_reduce(h, out), h)
    return list(out)


def lb_d3_state(h: int) -> int:
    return lib().lb_d3_state(h)


def lb_d3_get_state(h: int, dst: int) -> None:
    check_d3(lib().lb_d3_get_state(h, dst), h)


def lb_d3_set_state(h: int, src: int) -> None:
    check_d3(lib().lb_d3_set_state(h, src), h)


def lb_d3_get_params(h: int) -> tuple[lb_params, dict]:
    p, d = lb_params(), lb_derived()
    check_d3(lib().lb_d3_get_params(h, ctypes.byref(p), ctypes.byref(d)), h)
    return p, d.as_dict()


def lb_d3_free(h: int) -> None:
    lib().lb_d3_free(h)
