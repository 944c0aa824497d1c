"""FP64 CPU oracle of the D3Q19 form of the self-tuning-EOS model (ctypes
binding of ``lbm3d_oracle.cpp``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are
[19][nz][ny][nx] (populations) and [nz][ny][nx] (fields).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import params

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm3d_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle3d.so")
Q = 19


def build(force: bool = False) -> str:
    """Compile with g++ (-O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("eos", ctypes.c_int32), ("form", ctypes.c_int32),
                ("eos_a", ctypes.c_double), ("eos_b", ctypes.c_double),
                ("R_gas", ctypes.c_double), ("T", ctypes.c_double),
                ("lam", ctypes.c_double), ("G2", ctypes.c_double), ("varpi", ctypes.c_double),
                ("s0", ctypes.c_double), ("se", ctypes.c_double), ("seps", ctypes.c_double),
                ("sj", ctypes.c_double), ("sq", ctypes.c_double), ("sp", ctypes.c_double),
                ("sm", ctypes.c_double), ("spi", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i = ctypes.POINTER(ctypes.c_double), ctypes.c_int
        P = ctypes.POINTER(_Params)
        _lib.or3_step.argtypes = [P, i, i, i, d, d, i]
        _lib.or3_init_eq.argtypes = [P, i, i, i, d, d, d, d, d]
        _lib.or3_force_stencil.argtypes = [i, i, i, d, d, d, d]
        _lib.or3_macro.argtypes = [P, i, i, i, d, d, d, d, d]
        _lib.or3_moments_eq.argtypes = [P, ctypes.c_double, ctypes.c_double, d, d]
        _lib.or3_moments_force.argtypes = [d, d, d]
        _lib.or3_moments_Q.argtypes = [P, d, d]
        _lib.or3_matrix_S.argtypes = [P, d, d]
        _lib.or3_collide_node.argtypes = [P, d, d, d]
        _lib.or3_coefficients.argtypes = [P, d]
        _lib.or3_matrix_M.argtypes = [d]
        _lib.or3_matrix_Minv.argtypes = [d]
        _lib.or3_weights.argtypes = [d]
        _lib.or3_velocities.argtypes = [ctypes.POINTER(ctypes.c_int)] * 3
    return _lib


def _cparams(p) -> _Params:
    if isinstance(p, params.LatticeParams):
        p = p.as_dict()
    return _Params(**{k: p[k] for k, _ in _Params._fields_})


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def velocities() -> np.ndarray:
    e = [(ctypes.c_int * Q)() for _ in range(3)]
    lib().or3_velocities(*e)
    return np.array([list(x) for x in e])          # (3, 19)


def weights() -> np.ndarray:
    out = np.empty(Q)
    lib().or3_weights(_dp(out))
    return out


def matrix_M() -> np.ndarray:
    out = np.empty((Q, Q))
    lib().or3_matrix_M(_dp(out))
    return out


def matrix_Minv() -> np.ndarray:
    out = np.empty((Q, Q))
    lib().or3_matrix_Minv(_dp(out))
    return out


def coefficients(p) -> dict:
    out = np.empty(4)
    lib().or3_coefficients(ctypes.byref(_cparams(p)), _dp(out))
    return dict(zip(("beta2", "k", "h", "b"), out))


def moments_eq(p, rho, eta, u) -> np.ndarray:
    out = np.empty(Q)
    lib().or3_moments_eq(ctypes.byref(_cparams(p)), float(rho), float(eta), _dp(_f64(u)), _dp(out))
    return out


def moments_force(F, u) -> np.ndarray:
    out = np.empty(Q)
    lib().or3_moments_force(_dp(_f64(F)), _dp(_f64(u)), _dp(out))
    return out


def moments_Q(p, s) -> np.ndarray:
    out = np.empty(Q)
    lib().or3_moments_Q(ctypes.byref(_cparams(p)), _dp(_f64(s)), _dp(out))
    return out


def matrix_S(p, u) -> np.ndarray:
    out = np.empty((Q, Q))
    lib().or3_matrix_S(ctypes.byref(_cparams(p)), _dp(_f64(u)), _dp(out))
    return out


def collide_node(p, f19, s) -> np.ndarray:
    out = np.empty(Q)
    lib().or3_collide_node(ctypes.byref(_cparams(p)), _dp(_f64(f19)), _dp(_f64(s)), _dp(out))
    return out


def init_eq(p, rho, ux=None, uy=None, uz=None) -> np.ndarray:
    """Equilibrium populations for given fields (rest where a component is None)."""
    rho = _f64(rho)
    nz, ny, nx = rho.shape
    comps = [None if c is None else _f64(np.broadcast_to(c, rho.shape)) for c in (ux, uy, uz)]
    f = np.empty((Q, nz, ny, nx))
    lib().or3_init_eq(ctypes.byref(_cparams(p)), nx, ny, nz, _dp(rho),
                      *[None if c is None else _dp(c) for c in comps], _dp(f))
    return f


def force_stencil(rho):
    rho = _f64(rho)
    nz, ny, nx = rho.shape
    s = [np.empty(rho.shape) for _ in range(3)]
    lib().or3_force_stencil(nx, ny, nz, _dp(rho), *[_dp(a) for a in s])
    return tuple(s)


def step(p, f, nsteps: int = 1) -> np.ndarray:
    f = _f64(f)
    _, nz, ny, nx = f.shape
    out = np.empty_like(f)
    if lib().or3_step(ctypes.byref(_cparams(p)), nx, ny, nz, _dp(f), _dp(out), int(nsteps)) != 0:
        raise ValueError("or3_step failed")
    return out


def macro(p, f):
    """(rho, ux, uy, uz) at the time level of the last collision held in ``f``."""
    f = _f64(f)
    _, nz, ny, nx = f.shape
    out = [np.empty((nz, ny, nx)) for _ in range(4)]
    lib().or3_macro(ctypes.byref(_cparams(p)), nx, ny, nz, _dp(f), *[_dp(a) for a in out])
    return tuple(out)
