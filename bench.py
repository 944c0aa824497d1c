"""Benchmark of the D2Q9 self-tuning-EOS multiphase LB time step on GB300.

Workload: FP32 spinodal decomposition on a 4096 x 4096 periodic lattice,
mean density at the midpoint of the coexistence densities with seeded uniform
+-1% noise, van der Waals EOS (a = 9/49, b = 2/21, R = 1) at T/Tc = 0.8, fluid
at rest, tau = 1.  One benchmark step = one full time step of the lattice
(pull streaming, density, interaction force, moment-space collision of Eq. 13,
inverse transform) = 16.8 M lattice updates.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent lattice (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D2Q9 multiphase MLUPS & % of GB300 HBM peak (FP32 vs FP64); adjoint/forward cost"
N_SIDE = 4096
TR = 0.8
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal
BYTES_PER_LU = {"fp64": 144, "fp32": 72, "fp16s": 36}  # read 9 + write 9 populations
BYTES_PER_LU_D3Q19 = {"fp64": 304, "fp32": 152}  # read 19 + write 19 populations
# DRAM bytes per launch of the dominant kernel from one ncu capture, valid only
# for the kernel code they were measured on (sha256 of the files below with
# comments and blank lines removed).
KERNEL_SOURCES = ["paper_1809_02390_gb300/csrc/lbm_kernels.cuh", "paper_1809_02390_gb300/csrc/lbm_device.cuh",
                  "paper_1809_02390_gb300/csrc/lbm_tma.cuh"]
# DRAM bytes per launch of the timed kernel from one ncu capture, keyed by kernel,
# layout and the hash of its sources (a changed kernel has no figure until recaptured).
NCU_TRAFFIC = {
    # 2048^2 capture (profiles/k_step_tma_dyn_fp32_rows_2048_full.md) scaled x4 to 4096^2.
    ("k_step_tma_dyn<f2>", "rows", "6ce1a8b1aef1d2b0"): 1021228032,
}
# The same for the D3Q19 step, keyed by the hash of its step code (csrc/lbm3d_step.cuh):
# the 192^3 capture (profiles/k_d3_step_fp32_192cubed_full.md) scaled by the node
# count to 256^3.
KERNEL_SOURCES_D3Q19 = ["paper_1809_02390_gb300/csrc/lbm3d_step.cuh"]
NCU_TRAFFIC_D3Q19 = {
    ("k_d3_step<float, true>", "a1c9912d3353d741"): 2512434821,
}


def code_only(text: str) -> str:
    """C++ source without comments, trailing blanks and empty lines (string literals
    of these files hold no comment markers), so that edits to comments leave the
    hash of the code unchanged."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES if sources is None else sources:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_rho(n: int, seed: int):
    from paper_1809_02390_gb300 import derive, inputs

    d = derive(n, n, Tr=TR)
    return inputs.spinodal(n, n, 0.5 * (d["rho_g"] + d["rho_l"]), 0.01, seed=seed), d


def time_steps(lat, steps: int, torch) -> float:
    """Milliseconds for `steps` time steps, CUDA events on the lattice's stream (runs
    of 64 steps replay a graph on the handle's own stream, which lb_step orders
    between the work before and after it on this one)."""
    s = lat.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    lat.step(steps)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def max_over_ranks(v: float, torch, world: int) -> float:
    """Largest value over the ranks (the slowest rank's time): one all_reduce, on
    the GPU under NCCL, on the host under gloo."""
    if world == 1:
        return v
    import torch.distributed as dist

    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(world: int, nodes: int, steps: int, ms: float) -> float:
    """Whole-job throughput: every rank advances its own lattice of `nodes` nodes by
    `steps` steps; `ms` is the slowest rank's time (weak scaling)."""
    return world * nodes * steps / (ms * 1e-3) / 1e6


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def cpu_baseline(rho0, seconds: float = 12.0) -> dict:
    """The FP64 oracle as it stands (single-threaded C++), on a 256 x 256 periodic
    crop of the same initial field, stepped until ~`seconds` of CPU time."""
    import oracle
    from oracle import params as op

    p = op.from_physical(Tr=TR)
    crop = rho0[:256, :256].copy()
    f = oracle.init_feq(p, crop)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        f = oracle.step(p, f, 10)
        steps += 10
    dt = time.perf_counter() - t0
    out = {"value": round(256 * 256 * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": "%d steps of the FP64 oracle on a 256x256 periodic crop of the workload" % steps}
    out["all_cores"] = cpu_baseline_all_cores(rho0, seconds=0.75 * seconds)
    out["host"] = {"cpu": host_cpu(), "nproc": os.cpu_count()}
    return out


def host_cpu() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_rate(job):
    """One oracle process: steps its crop for about `seconds`; returns
    (node updates, seconds).  Module-level so that spawned workers can import it."""
    crop, seconds = job
    import oracle
    from oracle import params as op

    p = op.from_physical(Tr=TR)
    f = oracle.init_feq(p, crop)
    f = oracle.step(p, f, 2)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        f = oracle.step(p, f, 10)
        steps += 10
    return crop.size * steps, time.perf_counter() - t0


def cpu_baseline_all_cores(rho0, seconds: float = 9.0) -> dict:
    """The same oracle on every host core at once: one process per core (spawned:
    CUDA is initialised in this process), each on its own 256 x 256 crop of the
    workload; the throughput is the sum of the processes' rates over overlapping
    windows of about `seconds`."""
    import multiprocessing as mp

    import numpy as np

    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    gy, gx = max(1, rho0.shape[0] // 256), max(1, rho0.shape[1] // 256)
    crops = [np.ascontiguousarray(rho0[256 * ((k // gx) % gy):][:256, 256 * (k % gx):][:, :256]) for k in range(n)]
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map_async(_oracle_rate, [(c, seconds) for c in crops]).get(timeout=120 + 4 * seconds)
    rate = sum(u / t for u, t in res) / 1e6
    return {"value": round(rate, 3), "unit": "MLUPS", "cores": n, "kind": "oracle",
            "sample": "%d single-threaded oracle processes, one per core, each ~%.0f s on its own 256x256 crop"
                      % (n, seconds)}


def measure_adjoint(n: int, torch) -> dict:
    """Adjoint (lb_adjoint_steps, a 45-step checkpoint segment) against the forward step, FP32."""
    from paper_1809_02390_gb300 import Lattice, capi

    rho0, _ = workload_rho(n, seed=0)
    lat = Lattice(rho0, precision="fp32", Tr=TR)
    lat.step(5)
    st = lat.state().clone()
    lam = torch.randn((9, n, n), dtype=torch.float32, device="cuda")
    dth = torch.zeros(3, dtype=torch.float64, device="cuda")
    nscr = capi.lb_adjoint_steps_scratch_bytes(lat.p)
    scr = torch.empty(nscr, dtype=torch.uint8, device="cuda")
    k = 45
    states = [st.data_ptr()] * k
    capi.lb_adjoint_steps(lat.h, states, lam.data_ptr(), dth.data_ptr(), scr.data_ptr(), nscr)
    s = lat.stream
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(s)
    lat.step(k)
    e[1].record(s)
    capi.lb_adjoint_steps(lat.h, states, lam.data_ptr(), dth.data_ptr(), scr.data_ptr(), nscr)
    e[2].record(s)
    torch.cuda.synchronize()
    fw, ad = e[0].elapsed_time(e[1]) / k, e[1].elapsed_time(e[2]) / k
    lat.close()
    return {"lattice": [n, n], "dtype": "f32", "steps": k, "forward_ms_per_step": round(fw, 5),
            "adjoint_ms_per_step": round(ad, 5), "adjoint_over_forward": round(ad / fw, 3),
            "adjoint_bytes_per_node": 124, "adjoint_GBps_algorithmic": round(124 * n * n / (ad * 1e-3) / 1e9, 1)}


def batch_workload(n_lattices: int = 256, seed: int = 0):
    """256 lattices: side log-uniform in [64, 1024], Tr uniform in [0.65, 0.95],
    interface width W uniform in [3, 8] (K_int = W / W1(Tr)), droplet (R = L/4)
    or slab (thickness L/2) by a seeded coin."""
    from paper_1809_02390_gb300 import derive, inputs

    rhos, kws, meta = [], [], []
    for sp in inputs.batch_specs(n_lattices, seed=seed):
        nx, ny = sp["nx"], sp["ny"]
        d = derive(nx, ny, Tr=sp["Tr"])
        rg, rl = d["rho_g"], d["rho_l"]
        if sp["shape"] == "droplet":
            r = inputs.droplet(nx, ny, nx / 4, sp["W"], rg, rl)
        else:
            r = inputs.slab(nx, ny, nx / 2, sp["W"], rg, rl)
        rhos.append(r)
        kws.append(dict(Tr=sp["Tr"], K_int=sp["W"] / d["W1"]))
        meta.append(dict(sp, rho_g=rg, rho_l=rl))
    return rhos, kws, meta


def measure_batch(torch, single_mlups: float, steps: int, layout: str = "rows") -> dict:
    from paper_1809_02390_gb300 import Batch

    rhos, kws, meta = batch_workload()
    nodes = sum(r.size for r in rhos)
    b = Batch(rhos, [dict(k, layout=layout) for k in kws])
    b.tune(4)
    cfg = b.config()
    s = b.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.run(64)
    s.synchronize()
    e0.record(s)
    b.run(steps)
    e1.record(s)
    s.synchronize()
    ms = e0.elapsed_time(e1)
    mlups = nodes * steps / (ms * 1e-3) / 1e6
    # Coexistence curve: bulk densities (centre = liquid, corner / edge column = gas) against Maxwell.
    import numpy as np

    eg, el, curve, unstable = [], [], [], []
    bad = set(b.nonfinite())  # lb_batch_nonfinite: lattices with a non-finite density
    for i, m in enumerate(meta):
        if i in bad:
            unstable.append({"index": i, "side": m["nx"], "Tr": round(m["Tr"], 4), "W": round(m["W"], 3),
                             "shape": m["shape"]})
            continue
        rho = b.density(i).cpu().numpy()
        ny, nx = rho.shape
        liq, gas = float(rho[ny // 2, nx // 2]), float(rho[0, 0])
        eg.append(abs(gas / m["rho_g"] - 1))
        el.append(abs(liq / m["rho_l"] - 1))
        curve.append([round(m["Tr"], 4), round(gas, 5), round(liq, 5), round(m["rho_g"], 5), round(m["rho_l"], 5)])
    b.close()

    return {"lattices": len(rhos), "layout": layout, "nodes": nodes, "steps": steps, "ms": round(ms, 2), "MLUPS": round(mlups, 1),
            "ratio_vs_single_lattice": round(mlups / single_mlups, 4) if single_mlups else None, "tuned": cfg,
            "launch": "one multi-lattice kernel per step (blocks_per_sm 0: one block per tile, else persistent), "
                      "graph replay of 64 steps",
            "unstable_lattices": unstable,
            "coexistence_vs_maxwell": {"lattices": len(eg),"gas_rel_err_median": round(float(np.median(eg)), 5),
                                       "gas_rel_err_max": round(float(np.max(eg)), 5),
                                       "liquid_rel_err_median": round(float(np.median(el)), 5),
                                       "liquid_rel_err_max": round(float(np.max(el)), 5),
                                       "columns": ["Tr", "rho_gas", "rho_liquid", "maxwell_gas", "maxwell_liquid"],
                                       "first_8": curve[:8]}}


def measure_precision(torch, steps: int = 20000) -> dict:
    """FP64 / FP32 / FP16-storage on 512 x 512 equilibria: flat slabs (liquid band
    256 thick, two interfaces) at Tr = 0.7, 0.8, 0.9 and droplets of radius 20, 40,
    80 at Tr = 0.8, all with a tanh start of the pressure-tensor width W1, run for
    `steps` steps.  Per case: max |rho - rho_FP64| / max rho_FP64 of the reduced
    precisions, the bulk densities against the Maxwell construction (slabs), and
    Laplace's dp R against the pressure-tensor sigma (droplets).  FP16 storage runs
    with stochastic rounding (the default) and with round-to-nearest."""
    import numpy as np

    from paper_1809_02390_gb300 import Lattice, derive, inputs

    n = 512
    cases = [("slab", tr, None) for tr in (0.7, 0.8, 0.9)] + [("droplet", 0.8, r) for r in (20, 40, 80)]
    out = []
    t0 = time.perf_counter()
    for shape, tr, radius in cases:
        d = derive(n, n, Tr=tr)
        rg, rl = d["rho_g"], d["rho_l"]
        if shape == "slab":
            rho0 = inputs.slab(n, n, n / 2, d["W1"], rg, rl)
        else:
            rho0 = inputs.droplet(n, n, radius, d["W1"], rg, rl)
        res = {"shape": shape, "Tr": tr}
        if radius:
            res["R0"] = radius
        rho64 = None
        for prec in ("fp64", "fp32", "fp16s", "fp16s_nearest"):
            extra = {"rounding": 1} if prec == "fp16s_nearest" else {}
            lat = Lattice(rho0, precision=prec.split("_")[0], Tr=tr, **extra)
            lat.step(steps)
            rho = lat.moments(velocity=False).double().cpu().numpy()
            r = lat.reduce()
            lat.close()
            entry = {"mass_rel_drift": float(r["mass"] / rho0.sum() - 1.0)}
            if rho64 is None:
                rho64 = rho
            else:
                entry["rel_err_vs_fp64"] = float(np.abs(rho - rho64).max() / np.abs(rho64).max())
            if shape == "slab":
                entry["rho_liquid_rel_err"] = float(rho[n // 2, n // 2] / rl - 1.0)
                entry["rho_gas_rel_err"] = float(rho[n // 2, 0] / rg - 1.0)
            else:
                radius_eq = float(np.sqrt(r["n_liquid"] / np.pi))
                entry["R"] = round(radius_eq, 3)
                entry["laplace_dpR_over_sigma"] = (r["p_center"] - r["p_corner"]) * radius_eq / (d["sigma1"] * d["lam"])
            res[prec] = {k: (round(v, 8) if isinstance(v, float) else v) for k, v in entry.items()}
        out.append(res)
        torch.cuda.empty_cache()
    return {"lattice": [n, n], "steps": steps, "seconds": round(time.perf_counter() - t0, 1), "cases": out}


def measure_oscillation(torch, steps: int = 60000) -> dict:
    """The paper's dynamic test (elliptic droplet, 512 x 512, CS EOS, Tr = 0.6,
    sigma = 0.01, W = 10; main text after Fig. 2) in FP32 with tau = 1: fitted
    damped and undamped periods against the inviscid n = 2 period.  The paper
    prints 18346 steps measured and 18628 from theory, at a viscosity it does not
    state; tau = 1 is the reading used here."""
    from paper_1809_02390_gb300.validation import elliptic_oscillation

    t0 = time.perf_counter()
    r = elliptic_oscillation("fp32", steps=steps)
    r["seconds"] = round(time.perf_counter() - t0, 1)
    r["paper_T_measured"], r["paper_T_analytic"] = 18346, 18628.0
    return {k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()}


def measure_translation(torch) -> dict:
    """Galilean check: a droplet restarted with a uniform velocity U against the same
    droplet at rest, compared in the co-moving frame after 2,000 steps (FP32)."""
    from paper_1809_02390_gb300.validation import translating_droplet

    t0 = time.perf_counter()
    rows = [translating_droplet(U=u, steps=2000) for u in (0.025, 0.05, 0.1)]
    out = {"rows": [{k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()} for r in rows],
           "seconds": round(time.perf_counter() - t0, 1)}
    return out


def measure_sweeps(torch) -> dict:
    """Interface thickness and surface tension against K_INT (CS EOS, a = 1, b = 4),
    fitted slopes next to the simulated and analytic slopes printed in supplement
    Sec. V (Figs. 1 and 3): W from 1024 x 4 flat interfaces after 40,000 steps,
    sigma from Laplace's law on 512 x 512 droplets of radius 128 (100,000 steps,
    then averaged over 20,000)."""
    from paper_1809_02390_gb300 import validation as v

    paper = {0.9: (6.3682, 6.3711, 0.003157, 0.003146), 0.8: (4.3490, 4.3574, 0.009115, 0.009081),
             0.7: (3.4403, 3.4423, 0.01716, 0.01710), 0.6: (2.8787, 2.8875, 0.02725, 0.02716),
             0.5: (2.5178, 2.5052, 0.03979, 0.03954)}
    t0 = time.perf_counter()
    ws, ss = v.thickness_slopes(), v.sigma_slopes()
    rows = []
    for Tr in sorted(paper, reverse=True):
        row = {"Tr": Tr, "W_slope": round(ws[Tr]["slope"], 5), "W_slope_paper_sim": paper[Tr][0],
               "W_slope_analytic": paper[Tr][1]}
        if Tr in ss:
            row.update({"sigma_slope": round(ss[Tr]["slope"], 7), "sigma_slope_paper_sim": paper[Tr][2],
                        "sigma_slope_analytic": paper[Tr][3],
                        "sigma_slope_with_intercept": round(ss[Tr]["slope_with_intercept"], 7)})
        rows.append(row)
    return {"seconds": round(time.perf_counter() - t0, 1), "rows": rows,
            "K_int": {"W": {str(k): list(v_) for k, v_ in v.W_SWEEP.items()},
                      "sigma": {str(k): list(v_[0]) for k, v_ in v.SIGMA_SWEEP.items()}},
            "sigma_setup": {str(k): {"lattice": v_[1], "radius": v_[2], "relax_steps": v_[3], "avg_steps": v_[4]}
                            for k, v_ in v.SIGMA_SWEEP.items()}}


def measure_calibration(torch, iterations: int = 50) -> dict:
    """256 x 256 FP32, perturbed ellipse (axis ratio 1.5, area of an R = 40 disk),
    2,000 steps, checkpoints every 45; target made at (Tr, G2, K_int) = (0.8, G2_ref, 1);
    loss = squared L2 distance of the final density.  L-BFGS (the library's default)
    and, for comparison, Adam, each for at most `iterations` loss-and-gradient
    evaluations from the same perturbed start."""
    from paper_1809_02390_gb300 import inputs
    from paper_1809_02390_gb300.adjoint import RolloutSpec, calibrate, density, initial_state, rollout

    n, steps = 256, 2000
    spec = RolloutSpec(n, n, precision="fp32", Tr_ref=TR, K_int_ref=1.0)
    ref = torch.tensor([TR, spec.G2_ref, 1.0], dtype=torch.float64)
    a = 40 * 1.5 ** 0.5
    rho0 = inputs.ellipse(n, n, a, 40 * 40 / a, 5.0, spec.rho_g, spec.rho_l, noise=0.01, seed=0)
    f0 = initial_state(spec, rho0, ref)
    with torch.no_grad():
        target = density(rollout(ref, f0, spec, steps, 45), spec).detach()
    start = ref * torch.tensor([0.97, 1.05, 1.08], dtype=torch.float64)
    rel = lambda t: [round(float(v), 5) for v in ((t - ref) / ref)]
    out = {"lattice": [n, n], "steps_per_rollout": steps, "checkpoint_every": 45, "params": ["Tr", "G2", "K_int"],
           "rel_error_start": rel(start)}
    for method, lr in (("lbfgs", 1.0), ("adam", 0.01)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        theta, losses = calibrate(spec, f0, target, start, steps, iterations=iterations, lr=lr, checkpoint_every=45,
                                  method=method)
        torch.cuda.synchronize()
        out[method] = {"evaluations": len(losses), "seconds": round(time.perf_counter() - t0, 2),
                       "loss_first": losses[0], "loss_last": losses[-1], "rel_error_fit": rel(theta)}
    return out


def workload_config(n: int, layout: str, world: int) -> dict:
    """The benchmark's workload description (the same dict on both arms)."""
    return {"workload": "spinodal-%dx%d-fp32-vdw-Tr0.8" % (n, n), "lattice": [n, n], "eos": "vdw",
            "Tr": TR, "storage": "fp32 (deviation from w_i rho_ref)", "variant": "fused",
            "layout": {"planes": "f[9][ny][nx]", "rows": "f[ny][9][nx]"}[layout],
            "l2": "inputs larger than L2 (2 x 604 MB population buffers)",
            "parallelism": "independent lattice per GPU" if world > 1 else "single GPU"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores; each step is one
    oracle time step on a 128 x 128 periodic crop of the workload."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from oracle import params as op
    from paper_1809_02390_gb300 import inputs

    p = op.from_physical(Tr=TR)
    rho0 = inputs.spinodal(N_SIDE, N_SIDE, 0.5 * (p.rho_g + p.rho_l), 0.01, seed=0)
    crop = np.ascontiguousarray(rho0[:128, :128])
    f = oracle.init_feq(p, crop)
    f = oracle.step(p, f, args.warmup)
    t0 = time.perf_counter()
    f = oracle.step(p, f, args.steps)
    dt = time.perf_counter() - t0
    value = 128 * 128 * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(N_SIDE, args.layout, world),
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": "each step: one FP64 oracle time step on a 128 x 128 periodic crop of the "
                                       "4096 x 4096 workload's initial field (%d timed steps after %d warm-up "
                                       "steps; rate = crop nodes x steps / time)" % (args.steps, args.warmup)},
            "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    from paper_1809_02390_gb300 import Lattice, capi
    from paper_1809_02390_gb300 import build as lbuild

    lbuild.build()
    n = args.size
    if args.only_adjoint or args.only_batch or args.only_precision or args.only_validation:  # one measurement
        if args.only_validation:
            part = {"oscillation": measure_oscillation(torch), "translation": measure_translation(torch),
                    "interface_sweeps": measure_sweeps(torch)}
        elif args.only_precision:
            part = measure_precision(torch, args.precision_steps)
        else:
            part = measure_adjoint(n, torch) if args.only_adjoint else measure_batch(torch, None, args.batch_steps, args.layout)
        print(json.dumps(part), flush=True)
        return
    rho0, d = workload_rho(n, seed=rank)
    nodes = n * n
    pk = peaks()

    # --- main measurement: FP32 fused, inputs resident in HBM -----------------
    main_prec = args.main_precision if args.only_main else "fp32"
    main_var = args.main_variant if args.only_main else "fused"
    lat = Lattice(rho0, precision=main_prec, variant=main_var, Tr=TR, layout=args.layout)
    if args.dispatch == "static" and capi.lb_tile_dispatch(lat.h):
        capi.lb_set_tile_dispatch(lat.h, False)
    kernel = ("k_step_tma_dyn<f2>" if capi.lb_tile_dispatch(lat.h) else "k_step_tma<f2>") if capi.lb_uses_tma(lat.h) \
        else ("k_step_fused<f2,float>" if main_var == "fused" else "k_density + k_collide_rho")
    lat.step(args.warmup)
    barrier(world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = time_steps(lat, args.steps, torch)
    ms = max_over_ranks(ms, torch, world)
    ms_step = ms / args.steps
    value = aggregate_mlups(world, nodes, args.steps, ms)
    achieved = BYTES_PER_LU[main_prec] * nodes / (ms_step * 1e-3) / 1e9
    sane = lat.reduce()
    # Ceiling of the access pattern: the same nine read and nine write streams with
    # no arithmetic (lb_stream_copy), timed like the step.
    for _ in range(5):
        capi.lb_stream_copy(lat.h)
    s_ = lat.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s_)
    for _ in range(50):
        capi.lb_stream_copy(lat.h)
    e1.record(s_)
    torch.cuda.synchronize()
    pattern_gbs = BYTES_PER_LU[main_prec] * nodes * 50 / (e0.elapsed_time(e1) * 1e-3) / 1e9
    lat.close()
    del lat
    torch.cuda.empty_cache()
    if args.only_main:
        if rank == 0:
            print(json.dumps({"only_main": True, "size": n, "layout": args.layout, "kernel": kernel,
                              "precision": main_prec, "variant": main_var, "MLUPS": round(value, 1),
                              "ms_per_step": ms_step, "algorithmic_GBps": round(achieved, 1),
                              "pattern_GBps": round(pattern_gbs, 1)}))
        return

    # --- other variants / precisions (shorter runs, same workload) -------------
    variants = {}
    other = "planes" if args.layout == "rows" else "rows"
    quarter = max(50, args.steps // 4)
    for prec, var, lay, k, static in (("fp32", "fused", other, quarter, False),
                                      ("fp32", "fused", args.layout, quarter, True),
                                      ("fp32", "two_pass", args.layout, quarter, False),
                                      ("fp16s", "fused", args.layout, quarter, False),
                                      ("fp16s", "fused", other, quarter, False), ("fp64", "fused", args.layout, 30, False)):
        lt = Lattice(rho0, precision=prec, variant=var, Tr=TR, layout=lay)
        if static:  # the static tile walk of the tensor-copy step, for comparison
            capi.lb_set_tile_dispatch(lt.h, False)
        lt.step(3)
        m = time_steps(lt, k, torch) / k
        variants["%s_%s_%s%s" % (prec, var, lay, "_static_tiles" if static else "")] = {
            "MLUPS": round(nodes / (m * 1e-3) / 1e6, 1), "ms_per_step": round(m, 4),
            "algorithmic_GBps": round(BYTES_PER_LU[prec] * nodes / (m * 1e-3) / 1e9, 1)}
        lt.close()
        del lt
        torch.cuda.empty_cache()

    # Carnahan-Starling EOS (Eq. 20 with the paper's a = 1, b = 4): the same spinodal
    # recipe between its own coexistence densities, FP32 and FP64 (rows as above).
    from paper_1809_02390_gb300 import derive as lderive, inputs as linputs

    cs = dict(eos="cs", eos_a=1.0, eos_b=4.0, Tr=TR)
    dcs = lderive(n, n, **cs)
    rho_cs = linputs.spinodal(n, n, 0.5 * (dcs["rho_g"] + dcs["rho_l"]), 0.01, seed=rank)
    for prec, k in (("fp32", quarter), ("fp64", 30)):
        lt = Lattice(rho_cs, precision=prec, layout=args.layout, **cs)
        lt.step(3)
        m = time_steps(lt, k, torch) / k
        variants["%s_fused_%s_carnahan_starling" % (prec, args.layout)] = {
            "MLUPS": round(nodes / (m * 1e-3) / 1e6, 1), "ms_per_step": round(m, 4),
            "algorithmic_GBps": round(BYTES_PER_LU[prec] * nodes / (m * 1e-3) / 1e9, 1)}
        lt.close()
        del lt
        torch.cuda.empty_cache()
    del rho_cs

    # D3Q19 form of the step (include/lbm3d.h): a 256^3 spinodal decomposition at the
    # same Tr (16.8M nodes, as many as the 4096^2 lattice), FP32 and FP64; the fused
    # step reads and writes 19 populations per node (152 / 304 bytes).
    import numpy as np

    from paper_1809_02390_gb300 import Lattice3

    n3 = 256
    d3 = lderive(n, n, Tr=TR)
    rho3 = 0.5 * (d3["rho_g"] + d3["rho_l"]) * (1 + 0.01 * np.random.default_rng(rank).uniform(-1, 1, (n3,) * 3))
    for prec, k in (("fp32", quarter), ("fp64", 30)):
        lt = Lattice3(rho3, precision=prec, Tr=TR)
        lt.step(3)
        m = time_steps(lt, k, torch) / k
        gbs = BYTES_PER_LU_D3Q19[prec] * n3 ** 3 / (m * 1e-3) / 1e9
        kern = "k_d3_step<%s>" % ("float, true" if prec == "fp32" else "double, false")
        sha3 = kernel_source_hash(KERNEL_SOURCES_D3Q19)
        tr3 = NCU_TRAFFIC_D3Q19.get((kern, sha3))
        variants["d3q19_%s_256cubed" % prec] = {
            "MLUPS": round(n3 ** 3 / (m * 1e-3) / 1e6, 1), "ms_per_step": round(m, 4),
            "algorithmic_GBps": round(gbs, 1), "frac_of_measured_hbm": round(gbs / pk["hbm_gbs"], 4),
            "algorithmic_bytes_per_launch": BYTES_PER_LU_D3Q19[prec] * n3 ** 3, "traffic": tr3,
            "traffic_note": "ncu dram bytes read + written, 192^3 capture scaled by nodes" if tr3 else None,
            "kernel": kern, "kernel_source_sha": sha3}
        lt.close()
        del lt
        torch.cuda.empty_cache()
    del rho3
    # The same recipe at 512^3 (134 M nodes, 10.2 GB per FP32 buffer): the step
    # addresses its population planes with 64-bit offsets above 19 nx ny nz = 2^31.
    n5 = 512
    rho5 = torch.from_numpy(0.5 * (d3["rho_g"] + d3["rho_l"])
                            * (1 + 0.01 * np.random.default_rng(rank).uniform(-1, 1, (n5,) * 3))).cuda()
    lt = Lattice3(rho5, precision="fp32", Tr=TR)
    del rho5
    lt.step(3)
    k5 = max(10, quarter // 8)
    m = time_steps(lt, k5, torch) / k5
    gbs = BYTES_PER_LU_D3Q19["fp32"] * n5 ** 3 / (m * 1e-3) / 1e9
    variants["d3q19_fp32_512cubed"] = {
        "MLUPS": round(n5 ** 3 / (m * 1e-3) / 1e6, 1), "ms_per_step": round(m, 4), "steps": k5,
        "algorithmic_GBps": round(gbs, 1), "frac_of_measured_hbm": round(gbs / pk["hbm_gbs"], 4),
        "kernel": "k_d3_step<float, true, long long> (64-bit plane offsets)"}
    lt.close()
    del lt
    torch.cuda.empty_cache()

    # --- end to end through the public API with host buffers -------------------
    rho_host = torch.from_numpy(np.ascontiguousarray(rho0)).pin_memory()
    out_host = torch.empty((n, n), dtype=torch.float32).pin_memory()

    def end_to_end(steps):
        lt = Lattice(rho_host, precision="fp32", variant="fused", Tr=TR, layout=args.layout)
        lt.step(steps)
        rho_dev = lt.moments(velocity=False)
        out_host.copy_(rho_dev, non_blocking=True)
        torch.cuda.synchronize()
        lt.close()

    end_to_end(args.warmup)  # warm-up pass: first-use costs of the allocator and the library
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    end_to_end(args.steps)
    e2e_s = max_over_ranks(time.perf_counter() - t0, torch, world)
    e2e = {"value": round(world * nodes * args.steps / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": round(nodes * 8 / args.steps, 1),
           "d2h_bytes_per_step": round(nodes * 4 / args.steps, 1),
           "note": "lb_init from pinned host densities (checked on the device), K steps, lb_moments, density "
                   "read back; after one untimed pass of W steps; bytes amortised per step"}

    extras = {}
    if world == 1 and not args.no_extras:
        extras["adjoint"] = measure_adjoint(n, torch)
        extras["adjoint_256"] = measure_adjoint(256, torch)  # the calibration lattice
        torch.cuda.empty_cache()
        extras["batch"] = measure_batch(torch, value, args.batch_steps, args.layout)
        torch.cuda.empty_cache()
        extras["calibration"] = measure_calibration(torch)
        extras["precision"] = measure_precision(torch, args.precision_steps)
        extras["oscillation"] = measure_oscillation(torch)
        extras["translation"] = measure_translation(torch)
        extras["interface_sweeps"] = measure_sweeps(torch)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    src_hash = kernel_source_hash()
    traffic = NCU_TRAFFIC.get((kernel, args.layout, src_hash))
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": traffic,
            "frac_of_nominal": round(achieved / HBM_NOMINAL_GBS, 4),
            "frac_note": "frac divides by the measured copy bandwidth (the roofline peak); frac_of_nominal by "
                         "GB300's nominal HBM3e bandwidth of %.0f GB/s" % HBM_NOMINAL_GBS,
            "kernel": kernel, "algorithmic_bytes_per_launch": BYTES_PER_LU["fp32"] * nodes,
            "traffic_GBps": round(traffic / (ms_step * 1e-3) / 1e9, 1) if traffic else None,
            "peak_source": pk["source"] + " (MEASURED_PEAKS.json hbm_gbs, copy burst)",
            "kernel_source_sha": src_hash,
            "pattern_ceiling": {"GBps": round(pattern_gbs, 1), "frac": round(achieved / pattern_gbs, 4),
                                "what": "lb_stream_copy: the step's 9 reads + 9 writes per node, same layout "
                                        "and 32x16 tiles, one block per tile, no arithmetic"}}
    cpu = cpu_baseline(rho0) if world == 1 else None
    line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(n, args.layout, world),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clk.summary(), "variants": variants, **extras,
            "check": {"mass": sane["mass"], "rho_min": sane["rho_min"], "rho_max": sane["rho_max"]}}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_d3q19(args):
    """The D3Q19 step alone: an N^3 spinodal lattice at Tr = 0.8 (mean density plus 1%
    uniform noise, seed 0), W untimed steps, K timed steps (CUDA events), one JSON line."""
    import numpy as np
    import torch

    from paper_1809_02390_gb300 import Lattice3, derive

    n = args.only_d3q19
    d = derive(64, 64, Tr=TR)
    rho = 0.5 * (d["rho_g"] + d["rho_l"]) * (1 + 0.01 * np.random.default_rng(0).uniform(-1, 1, (n,) * 3))
    lat = Lattice3(rho, precision=args.d3q19_precision, Tr=TR)
    lat.step(args.warmup)
    ms = time_steps(lat, args.steps, torch) / args.steps
    ok = bool(torch.isfinite(lat.moments(velocity=False)).all())
    b = BYTES_PER_LU_D3Q19[args.d3q19_precision]
    print(json.dumps({"only_d3q19": True, "size": n, "precision": args.d3q19_precision, "steps": args.steps,
                      "ms_per_step": round(ms, 5), "MLUPS": round(n ** 3 / (ms * 1e-3) / 1e6, 1),
                      "algorithmic_GBps": round(b * n ** 3 / (ms * 1e-3) / 1e9, 1), "finite": ok}))
    lat.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=N_SIDE, help="lattice side (profiling runs use smaller cases)")
    ap.add_argument("--only-main", action="store_true", help="time the FP32 fused step only (profiling)")
    ap.add_argument("--main-precision", choices=["fp32", "fp16s", "fp64"], default="fp32",
                    help="with --only-main: storage precision of the timed step (profiling)")
    ap.add_argument("--main-variant", choices=["fused", "two_pass"], default="fused",
                    help="with --only-main: fused step or the two-pass variant (profiling)")
    ap.add_argument("--only-adjoint", action="store_true", help="time the FP32 adjoint at --size only (profiling)")
    ap.add_argument("--only-d3q19", type=int, default=0, metavar="N",
                    help="time the D3Q19 step on an N^3 spinodal lattice only (profiling)")
    ap.add_argument("--d3q19-precision", choices=["fp32", "fp64"], default="fp32",
                    help="with --only-d3q19: storage precision")
    ap.add_argument("--only-batch", action="store_true", help="time the 256-lattice batch only (profiling)")
    ap.add_argument("--only-precision", action="store_true", help="run the FP64/FP32/FP16 study only")
    ap.add_argument("--only-validation", action="store_true", help="run the oscillation and W/sigma sweeps only")
    ap.add_argument("--precision-steps", type=int, default=20000, help="steps of the precision study")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjoint, batch and calibration runs")
    ap.add_argument("--batch-steps", type=int, default=5000, help="steps of the 256-lattice batch run")
    ap.add_argument("--dispatch", choices=["dynamic", "static"], default="dynamic",
                    help="tile dispatch of the tensor-copy step (tickets, or the static walk)")
    ap.add_argument("--layout", choices=["planes", "rows"], default="rows",
                    help="population layout of the timed lattice (the other one is timed as a variant)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.only_d3q19:
        run_d3q19(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
