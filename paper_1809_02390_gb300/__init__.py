"""GB300-native (sm_103a) multiphase lattice Boltzmann with self-tuning EOS.

Implements the per-node time step of Huang, Wu & Adams, "Lattice Boltzmann
model with self-tuning equation of state for multiphase flows"
(arXiv:1809.02390) as hand-written CUDA behind the C ABI of include/lbm.h,
and its D3Q19 form behind include/lbm3d.h (Lattice3).
PyTorch only provides device memory and streams.

    lat = Lattice(rho0, precision="fp32", Tr=0.85)
    lat.step(1000)
    rho, ux, uy = lat.moments()
"""
from __future__ import annotations

import numpy as np

from . import capi
from .capi import LB_FP16S, LB_FP32, LB_FP64, LB_FUSED, LB_TWO_PASS, LBError  # noqa: F401

PRECISIONS = {"fp64": capi.LB_FP64, "fp32": capi.LB_FP32, "fp16s": capi.LB_FP16S}
VARIANTS = {"fused": capi.LB_FUSED, "two_pass": capi.LB_TWO_PASS}
EOS = {"vdw": capi.LB_EOS_VDW, "cs": capi.LB_EOS_CS}
# Population layouts of the state buffers: f[9][ny][nx], or f[ny][9][nx].
LAYOUTS = {"planes": capi.LB_LAYOUT_PLANES, "rows": capi.LB_LAYOUT_ROWS}
# Rest-state weights w_i of the storage shift, in the velocity order of the ABI.
W_REST = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (the library has no CPU path)")
    return torch


def derive(nx: int = 64, ny: int = 64, **kw) -> dict:
    """Host-side derived parameters (lb_derive): coexistence densities, lattice
    pressure scale, G^2/c^2, relaxation rates, pressure-tensor W1 and sigma1."""
    return capi.lb_derive(params(nx, ny, **kw))


def params(nx: int, ny: int, precision: str = "fp32", eos: str = "vdw", variant: str = "fused",
           layout: str = "planes", **kw) -> capi.lb_params:
    return capi.make_params(nx, ny, precision=PRECISIONS[precision], eos=EOS[eos], variant=VARIANTS[variant],
                            layout=LAYOUTS[layout], **kw)


class Lattice:
    """One periodic lattice on the current CUDA device and stream.

    rho0: initial density [ny, nx] (numpy array on the host, or a float64 CUDA
    tensor).  Keyword arguments are the fields of ``lb_params`` (Tr, K_int,
    s_p, rho_ref, ...).  ``rho_ref=None`` stores deviations from the rest state
    at the mean initial density for reduced-precision storage.  ``layout``:
    "planes" stores f[9][ny][nx], "rows" f[ny][9][nx] (same results; the adjoint
    and the batched solver take "planes")."""

    def __init__(self, rho0, precision: str = "fp32", eos: str = "vdw", variant: str = "fused",
                 rho_ref: float | None = None, stream=None, layout: str = "planes", **kw):
        torch = _torch()
        if isinstance(rho0, np.ndarray):
            rho_host = np.ascontiguousarray(rho0, dtype=np.float64)
            ny, nx = rho_host.shape
            rho_t = torch.from_numpy(rho_host).pin_memory()
            on_device = False
        else:
            rho_t = rho0.to(dtype=torch.float64).contiguous()
            ny, nx = rho_t.shape
            on_device = rho_t.is_cuda
            if not on_device:
                rho_t = rho_t.pin_memory()
        if rho_ref is None:  # FP32 / FP16: NaN asks lb_init for the mean initial density
            rho_ref = 0.0 if precision == "fp64" else float("nan")
        elif precision != "fp64":
            rho_ref = float(np.float32(rho_ref))  # the library stores the shift in float
        self.p = params(nx, ny, precision=precision, eos=eos, variant=variant, rho_ref=rho_ref, layout=layout,
                        **kw)
        self.nx, self.ny, self.precision, self.layout = nx, ny, precision, layout
        self.rho_ref = rho_ref
        self.dtype = {"fp64": torch.float64, "fp32": torch.float32, "fp16s": torch.float16}[precision]
        self.real = torch.float64 if precision == "fp64" else torch.float32
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        shape = (9, ny, nx) if layout == "planes" else (ny, 9, nx)
        self.f_a = torch.empty(shape, dtype=self.dtype, device=dev)
        self.f_b = torch.empty(shape, dtype=self.dtype, device=dev)
        nscr = capi.lb_scratch_bytes(self.p)
        self.scratch = torch.empty(nscr, dtype=torch.uint8, device=dev)
        self._rho0_keep = rho_t
        self.h = capi.lb_init(self.p, self.f_a.data_ptr(), self.f_b.data_ptr(), self.scratch.data_ptr(), nscr,
                              rho_t.data_ptr(), on_device, self.stream.cuda_stream)
        self.p = capi.lb_get_params(self.h)
        self.rho_ref = self.p.rho_ref
        self.derived = capi.lb_get_derived(self.h)

    def step(self, nsteps: int = 1) -> None:
        capi.lb_step(self.h, nsteps)

    @property
    def steps_done(self) -> int:
        return capi.lb_steps_done(self.h)

    def set_equilibrium(self, rho, ux=None, uy=None) -> None:
        """Sets the state to the equilibrium of a density and velocity field ([ny, nx]
        arrays or tensors; ux, uy default 0; u is the velocity before the half-force
        shift), through lb_set_equilibrium."""
        torch = _torch()
        dev = self.f_a.device

        def dev64(a):
            t = torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()
            if tuple(t.shape) != (self.ny, self.nx):
                raise ValueError("fields must be [ny, nx]")
            return t

        keep = [dev64(rho)] + [dev64(a) if a is not None else None for a in (ux, uy)]
        capi.lb_set_equilibrium(self.h, keep[0].data_ptr(), *[t.data_ptr() if t is not None else None
                                                               for t in keep[1:]])
        self.stream.synchronize()

    def buffer(self):
        """The current (post-collision) state buffer in its storage layout."""
        return self.f_a if capi.lb_state(self.h) == self.f_a.data_ptr() else self.f_b

    def state(self):
        """The current state as a [9, ny, nx] view of the buffer (a permuted view in
        the rows layout), stored as deviations f_i - w_i rho_ref."""
        b = self.buffer()
        return b if self.layout == "planes" else b.permute(1, 0, 2)

    def populations(self):
        """Post-collision populations in FP64 (storage shift added back)."""
        torch = _torch()
        w = torch.tensor(W_REST, dtype=torch.float64, device=self.f_a.device)
        return self.state().double() + self.rho_ref * w[:, None, None]

    def moments(self, velocity: bool = True):
        torch = _torch()
        rho = torch.empty((self.ny, self.nx), dtype=self.real, device=self.f_a.device)
        ux = torch.empty_like(rho) if velocity else None
        uy = torch.empty_like(rho) if velocity else None
        capi.lb_moments(self.h, rho.data_ptr(), ux.data_ptr() if velocity else None,
                        uy.data_ptr() if velocity else None)
        return (rho, ux, uy) if velocity else rho

    def pressure(self):
        """p_EOS / c^2 at every node ([ny, nx] tensor of the compute type)."""
        torch = _torch()
        p = torch.empty((self.ny, self.nx), dtype=self.real, device=self.f_a.device)
        capi.lb_pressure(self.h, p.data_ptr())
        return p

    def reduce(self) -> dict:
        v = capi.lb_reduce(self.h)
        keys = ("mass", "mom_x", "mom_y", "p_center", "p_corner", "n_liquid", "rho_min", "rho_max")
        return dict(zip(keys, v))

    def close(self) -> None:
        if getattr(self, "h", None):
            capi.lb_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class Lattice3:
    """One periodic D3Q19 lattice (the 3-D form of the model, include/lbm3d.h) on
    the current CUDA device and stream.

    rho0: initial density [nz, ny, nx] (numpy array, or a float64 tensor).
    precision "fp32" or "fp64"; keyword arguments are the fields of ``lb_params``.
    ``rho_ref=None`` stores deviations from the rest state at the mean initial
    density (FP32) or at 0 (FP64)."""

    def __init__(self, rho0, precision: str = "fp32", eos: str = "vdw", rho_ref: float | None = None, stream=None,
                 **kw):
        torch = _torch()
        if isinstance(rho0, np.ndarray):
            rho_t = torch.from_numpy(np.ascontiguousarray(rho0, dtype=np.float64)).pin_memory()
            on_device = False
        else:
            rho_t = rho0.to(dtype=torch.float64).contiguous()
            on_device = rho_t.is_cuda
            if not on_device:
                rho_t = rho_t.pin_memory()
        nz, ny, nx = rho_t.shape
        if rho_ref is None:
            rho_ref = 0.0 if precision == "fp64" else float("nan")
        self.p = params(nx, ny, precision=precision, eos=eos, rho_ref=rho_ref, **kw)
        self.nx, self.ny, self.nz, self.precision = nx, ny, nz, precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.f_a = torch.empty((19, nz, ny, nx), dtype=self.dtype, device=dev)
        self.f_b = torch.empty_like(self.f_a)
        self._rho0_keep = rho_t
        self.h = capi.lb_d3_init(self.p, nz, self.f_a.data_ptr(), self.f_b.data_ptr(), rho_t.data_ptr(), on_device,
                                 self.stream.cuda_stream)
        self.p, self.derived = capi.lb_d3_get_params(self.h)
        self.rho_ref = self.p.rho_ref
        self.velocities = capi.lb_d3_velocities()

    def step(self, nsteps: int = 1) -> None:
        capi.lb_d3_step(self.h, nsteps)

    def state(self):
        """The current state [19, nz, ny, nx], stored as deviations f_i - w_i rho_ref."""
        return self.f_a if capi.lb_d3_state(self.h) == self.f_a.data_ptr() else self.f_b

    def populations(self):
        """Post-collision populations in FP64 (storage shift added back)."""
        torch = _torch()
        w = torch.tensor([1 / 3 if sum(c * c for c in e) == 0 else (1 / 18 if sum(c * c for c in e) == 1 else 1 / 36)
                          for e in self.velocities], dtype=torch.float64, device=self.f_a.device)
        return self.state().double() + self.rho_ref * w[:, None, None, None]

    def set_state(self, f) -> None:
        """Loads a [19, nz, ny, nx] state (deviations, the storage type) from the device."""
        f = f.to(device=self.f_a.device, dtype=self.dtype).contiguous()
        capi.lb_d3_set_state(self.h, f.data_ptr())
        self.stream.synchronize()

    def moments(self, velocity: bool = True):
        """(rho, ux, uy, uz) as FP64 [nz, ny, nx] tensors (rho only if not velocity)."""
        torch = _torch()
        shape = (self.nz, self.ny, self.nx)
        rho = torch.empty(shape, dtype=torch.float64, device=self.f_a.device)
        u = [torch.empty_like(rho) for _ in range(3)] if velocity else [None] * 3
        capi.lb_d3_moments(self.h, rho.data_ptr(), *[t.data_ptr() if t is not None else None for t in u])
        return (rho, *u) if velocity else rho

    def reduce(self) -> dict:
        """FP64 diagnostics of the current state (lb_d3_reduce)."""
        v = capi.lb_d3_reduce(self.h)
        keys = ("mass", "mom_x", "mom_y", "mom_z", "n_liquid", "rho_min", "rho_max")
        return dict(zip(keys, v))

    def close(self) -> None:
        if getattr(self, "h", None):
            capi.lb_d3_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

class Batch:
    """Independent FP32 lattices advanced together (lb_batch_*).

    rho0s: list of initial densities [ny, nx] (numpy); kws: list of dicts of
    lb_params fields per lattice (Tr, K_int, ..., and layout="rows" for pools of
    f[ny][9][sx], the same for every lattice).  Runs on its own CUDA stream (graphs
    cannot be captured on the legacy default stream)."""

    def __init__(self, rho0s, kws, stream=None):
        torch = _torch()
        n = len(rho0s)
        self.n = n
        self.shapes = [np.asarray(r).shape for r in rho0s]
        self.layout = kws[0].get("layout", "planes")
        kws = [dict(kw) for kw in kws]
        # No rho_ref: NaN asks lb_batch_init for the lattice's mean initial density.
        refs = [float(np.float32(kw.pop("rho_ref"))) if "rho_ref" in kw else float("nan") for kw in kws]
        ps = (capi.lb_params * n)(*[params(s[1], s[0], precision="fp32", rho_ref=rr, **kw)
                                    for s, rr, kw in zip(self.shapes, refs, kws)])
        self._ps = ps
        self.stream = stream if stream is not None else torch.cuda.Stream()
        dev = torch.device("cuda", torch.cuda.current_device())
        pb, mb = capi.lb_batch_pool_bytes(ps), capi.lb_batch_meta_bytes(ps)
        self.pool_a = torch.empty(pb // 4, dtype=torch.float32, device=dev)
        self.pool_b = torch.empty(pb // 4, dtype=torch.float32, device=dev)
        self.meta = torch.empty(mb, dtype=torch.uint8, device=dev)
        rho = np.concatenate([np.ascontiguousarray(r, dtype=np.float64).ravel() for r in rho0s])
        self._rho_host = torch.from_numpy(rho).pin_memory()
        torch.cuda.current_stream().synchronize()
        self.b = capi.lb_batch_init(ps, self.pool_a.data_ptr(), self.pool_b.data_ptr(), self.meta.data_ptr(), mb,
                                    self._rho_host.data_ptr(), False, self.stream.cuda_stream)
        self.rho_refs = [capi.lb_batch_params(self.b, i).rho_ref for i in range(n)]

    def run(self, nsteps: int) -> None:
        capi.lb_batch_run(self.b, nsteps)

    def tune(self, trial_steps: int = 10) -> float:
        return capi.lb_batch_tune(self.b, trial_steps)

    def config(self) -> dict:
        return capi.lb_batch_config(self.b)

    def set_config(self, shape: int, blocks_per_sm: int) -> None:
        """Launch form by hand (lb_batch_set_config): shapes 0-2 plain loads, 3-4 tensor
        copies with a static tile walk, 5-6 tensor copies with tiles taken by ticket."""
        capi.lb_batch_set_config(self.b, shape, blocks_per_sm)

    @property
    def steps_done(self) -> int:
        return capi.lb_batch_steps_done(self.b)

    def state(self, i: int):
        """Current state of lattice i: [9, ny, nx] view of the current pool (deviations;
        rows are strided by nx rounded up to a multiple of 4; a permuted view in the
        rows layout)."""
        self.stream.synchronize()
        pool = self.pool_a if capi.lb_batch_state(self.b) == self.pool_a.data_ptr() else self.pool_b
        off = capi.lb_batch_offset(self.b, i)
        sx = capi.lb_batch_row_stride(self.b, i)
        ny, nx = self.shapes[i]
        if self.layout == "rows":
            return pool[off:off + 9 * sx * ny].view(ny, 9, sx)[:, :, :nx].permute(1, 0, 2)
        return pool[off:off + 9 * sx * ny].view(9, ny, sx)[:, :, :nx]

    def status(self) -> None:
        """Raises LBError if a bounded wait of the tensor-copy kernel gave up
        (LB_ETIMEOUT) or a lattice has a non-finite density (LB_ENONFINITE)."""
        capi.lb_batch_status(self.b)

    def nonfinite(self) -> list[int]:
        """Indices of the lattices whose current state has a non-finite density."""
        _, counts = capi.lb_batch_nonfinite(self.b, self.n)
        return [i for i, c in enumerate(counts) if c]

    def density(self, i: int):
        """Density of lattice i ([ny, nx] float32 tensor on the device, lb_batch_density)."""
        torch = _torch()
        ny, nx = self.shapes[i]
        rho = torch.empty((ny, nx), dtype=torch.float32, device=self.pool_a.device)
        capi.lb_batch_density(self.b, i, rho.data_ptr())
        self.stream.synchronize()
        return rho

    def derived(self, i: int) -> dict:
        return capi.lb_batch_derived(self.b, i)

    def close(self) -> None:
        if getattr(self, "b", None):
            self.stream.synchronize()
            capi.lb_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
