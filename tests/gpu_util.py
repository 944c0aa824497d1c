"""Helpers shared by the GPU tests (imported by test modules only)."""
import numpy as np

W_REST = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def oracle_params(**kw):
    from oracle import params as op

    return op.from_physical(**kw)


def lattice(rho0, precision="fp64", variant="fused", **kw):
    from paper_1809_02390_gb300 import Lattice

    return Lattice(rho0, precision=precision, variant=variant, **kw)


def gpu_populations(lat):
    """Post-collision populations of a lattice as FP64 numpy (shift added back)."""
    return lat.populations().cpu().numpy()


def rel_inf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def set_state_fp64(lat, f):
    """Loads an FP64 population array (9, ny, nx) into an FP64 lattice (rho_ref = 0)."""
    import torch

    from paper_1809_02390_gb300 import capi

    assert lat.precision == "fp64" and lat.rho_ref == 0.0
    t = torch.from_numpy(np.ascontiguousarray(f)).to(lat.f_a.device)
    capi.lb_set_state(lat.h, t.data_ptr())
    torch.cuda.synchronize()
