"""FP64 CPU oracle of the self-tuning-EOS multiphase LB time step.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and
bench.py's CPU-baseline / reference leg may import this package.  It shares
no code with the CUDA library and never imports it.

The per-node step lives in ``lbm_oracle.cpp`` (plain C++, FP64, no FMA
contraction), loaded here through ctypes; thermodynamics (Maxwell
construction, sigma, W) in ``thermo.py``; the physical -> lattice parameter
derivation in ``params.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import params, thermo  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no fast-math, no FMA contraction)."""
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
                ("lam", ctypes.c_double), ("G2", ctypes.c_double),
                ("varpi", ctypes.c_double),
                ("s0", ctypes.c_double), ("se", ctypes.c_double), ("seps", ctypes.c_double),
                ("sj", ctypes.c_double), ("sq", ctypes.c_double), ("sp", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i = ctypes.POINTER(ctypes.c_double), ctypes.c_int
        P = ctypes.POINTER(_Params)
        _lib.or_step.argtypes = [P, i, i, d, d, i]
        _lib.or_step_cs.argtypes = [P, d, i, i, d, d, d, d, i]
        _lib.or_init_feq.argtypes = [P, i, i, d, d]
        _lib.or_init_eq.argtypes = [P, i, i, d, d, d, d]
        _lib.or_force_stencil.argtypes = [i, i, d, d, d]
        _lib.or_macro.argtypes = [P, i, i, d, d, d, d]
        _lib.or_eos.argtypes = [P, ctypes.c_double, d, d]
        _lib.or_moments_eq.argtypes = [P] + [ctypes.c_double] * 4 + [d]
        _lib.or_moments_force.argtypes = [ctypes.c_double] * 4 + [d]
        _lib.or_moments_Q.argtypes = [P, ctypes.c_double, ctypes.c_double, d]
        _lib.or_matrices.argtypes = [P, ctypes.c_double, ctypes.c_double, d, d, d, d]
        _lib.or_collide_node.argtypes = [P, d, ctypes.c_double, ctypes.c_double, d]
        _lib.or_matrix_M.argtypes = [d]
        _lib.or_matrix_Minv.argtypes = [d]
        _lib.or_velocities.argtypes = [ctypes.POINTER(ctypes.c_int)] * 2
    return _lib


def _cparams(p) -> _Params:
    if isinstance(p, params.LatticeParams):
        p = p.as_dict()
    return _Params(**{k: p[k] for k, _ in _Params._fields_})


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def init_feq(p, rho0: np.ndarray) -> np.ndarray:
    """Rest equilibrium populations f_i = (M^-1 m_eq(rho0, u=0))_i, shape (9, ny, nx)."""
    rho0 = _f64(rho0)
    ny, nx = rho0.shape
    f = np.empty((9, ny, nx))
    lib().or_init_feq(ctypes.byref(_cparams(p)), nx, ny, _dp(rho0), _dp(f))
    return f


def init_eq(p, rho: np.ndarray, ux: np.ndarray | None = None, uy: np.ndarray | None = None) -> np.ndarray:
    """Equilibrium populations (M^-1 m_eq(rho, u))_i for given fields, shape (9, ny, nx)."""
    rho = _f64(rho)
    ny, nx = rho.shape
    f = np.empty((9, ny, nx))
    ux = None if ux is None else _f64(np.broadcast_to(ux, rho.shape))
    uy = None if uy is None else _f64(np.broadcast_to(uy, rho.shape))
    lib().or_init_eq(ctypes.byref(_cparams(p)), nx, ny, _dp(rho), None if ux is None else _dp(ux),
                     None if uy is None else _dp(uy), _dp(f))
    return f


def force_stencil(rho: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """S = sum_i omega_i rho(x + e_i) e_i on a periodic lattice (Eq. 12)."""
    rho = _f64(rho)
    ny, nx = rho.shape
    sx, sy = np.empty((ny, nx)), np.empty((ny, nx))
    lib().or_force_stencil(nx, ny, _dp(rho), _dp(sx), _dp(sy))
    return sx, sy


def step(p, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """``nsteps`` time steps (pull streaming + collision) of post-collision populations."""
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    rc = lib().or_step(ctypes.byref(_cparams(p)), nx, ny, _dp(f), _dp(out), int(nsteps))
    if rc != 0:
        raise ValueError("or_step failed")
    return out


def step_cs(p, f: np.ndarray, f_im: np.ndarray | None, dtheta_im=(0.0, 0.0, 0.0),
            nsteps: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Complex-step run: returns (Re, Im) of the state after ``nsteps`` steps when
    the input carries imaginary part ``f_im`` and the parameters (T, G2, lam)
    carry imaginary parts ``dtheta_im``."""
    f = _f64(f)
    _, ny, nx = f.shape
    fi = np.zeros_like(f) if f_im is None else _f64(f_im)
    th = _f64(np.asarray(dtheta_im, dtype=np.float64))
    re, im = np.empty_like(f), np.empty_like(f)
    rc = lib().or_step_cs(ctypes.byref(_cparams(p)), _dp(th), nx, ny, _dp(f), _dp(fi), _dp(re),
                          _dp(im), int(nsteps))
    if rc != 0:
        raise ValueError("or_step_cs failed")
    return re, im


def macro(p, f: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(rho, ux, uy) at the time level of the last collision held in ``f``."""
    f = _f64(f)
    _, ny, nx = f.shape
    rho, ux, uy = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
    lib().or_macro(ctypes.byref(_cparams(p)), nx, ny, _dp(f), _dp(rho), _dp(ux), _dp(uy))
    return rho, ux, uy


def eos(p, rho: float) -> tuple[float, float]:
    pe, dpe = ctypes.c_double(), ctypes.c_double()
    lib().or_eos(ctypes.byref(_cparams(p)), float(rho), ctypes.byref(pe), ctypes.byref(dpe))
    return pe.value, dpe.value


def moments_eq(p, rho, eta, ux, uy) -> np.ndarray:
    out = np.empty(9)
    lib().or_moments_eq(ctypes.byref(_cparams(p)), rho, eta, ux, uy, _dp(out))
    return out


def moments_force(Fx, Fy, ux, uy) -> np.ndarray:
    out = np.empty(9)
    lib().or_moments_force(Fx, Fy, ux, uy, _dp(out))
    return out


def moments_Q(p, Sx, Sy) -> np.ndarray:
    out = np.empty(9)
    lib().or_moments_Q(ctypes.byref(_cparams(p)), Sx, Sy, _dp(out))
    return out


def matrices(p, ux, uy):
    S, Rm = np.empty((9, 9)), np.empty((9, 9))
    T, X = np.empty((9, 2)), np.empty((9, 2))
    lib().or_matrices(ctypes.byref(_cparams(p)), ux, uy, _dp(S), _dp(Rm), _dp(T), _dp(X))
    return S, Rm, T, X


def collide_node(p, f9, Sx, Sy) -> np.ndarray:
    f9 = _f64(f9)
    out = np.empty(9)
    lib().or_collide_node(ctypes.byref(_cparams(p)), _dp(f9), Sx, Sy, _dp(out))
    return out


def matrix_M() -> np.ndarray:
    out = np.empty((9, 9))
    lib().or_matrix_M(_dp(out))
    return out


def matrix_Minv() -> np.ndarray:
    out = np.empty((9, 9))
    lib().or_matrix_Minv(_dp(out))
    return out


def velocities() -> tuple[np.ndarray, np.ndarray]:
    ex, ey = (ctypes.c_int * 9)(), (ctypes.c_int * 9)()
    lib().or_velocities(ex, ey)
    return np.array(ex[:]), np.array(ey[:])
