"""Throughput of the free-space convolution u = U * rho plus energy (Algorithm 1) on one GB300.

One step = one full evaluation (type-2 NUFFT, multiply by W_j, type-1 NUFFT, energy) of the
3D Coulomb workload on a 256^3 grid over [-16,16]^3 (rho = 16 seeded Gaussians, 160x160x320
spherical nodes, FP32 path with FP64 nodes/weights and a compensated FP64 energy).  The metric
is grid points per second per potential evaluation.  Beside it the line reports the same
workload on the FP64 GPU path (speedup, and the FP32 result's error against it), the
end-to-end rate through the host-buffer entry point, the roofline of the dominant kernel and
the FP64 CPU oracle timed on this machine's host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only.  Each rank evaluates its own copy of the workload (independent
densities; no collective on the data path); value = all ranks' points / max-over-ranks time.
``--impl reference`` times the FP64 CPU oracle instead (rank 0 only), on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "grid points/s per potential eval (FP32 & batched vs FP64 GPU) at stated rel L-inf err"
UNIT = "grid points/s"
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2: written between timed steps
TOL = 1e-5                          # stated relative L-inf tolerance of the FP32 path

# DRAM bytes per launch from an ncu capture of the kernel (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by stage name, with the hash of the kernel source the capture
# was taken on: a changed source reports traffic null until it is captured again.
# Measured with ncu on the 256^3 FP32 workload (one launch of each kernel, one pass of
# dram__bytes_read.sum and dram__bytes_write.sum).
TRAFFIC = {
    "interp": {"bytes": 460.9e6, "src": "53af5c4351994734"},
    "spread": {"bytes": 659.0e6, "src": "53af5c4351994734"},
    "fwd_fft_z": {"bytes": 155.2e6, "src": "13173716e1349e52"},
    "fwd_fft_y": {"bytes": 341.2e6, "src": "13173716e1349e52"},
    "fwd_fft_x": {"bytes": 481.6e6, "src": "13173716e1349e52"},
    "inv_fft_x": {"bytes": 530.2e6, "src": "13173716e1349e52"},
    "inv_fft_y": {"bytes": 370.4e6, "src": "13173716e1349e52"},
    "inv_fft_z": {"bytes": 254.8e6, "src": "13173716e1349e52"},
}


def _src_hash(stage: str) -> str:
    fname = "node_kernels.cuh" if stage in ("interp", "spread") else "fft_kernels.cuh"
    with open(os.path.join(ROOT, "paper_1311_4120_gb300", "csrc", fname), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank times over all ranks of the default process group (the
    values themselves when there is no process group): the whole job finishes with its
    slowest rank."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_rate(units_per_rank, world, t_max):
    """Whole-job throughput of replicas: every rank's units over the slowest rank's time."""
    return units_per_rank * world / t_max


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (FileNotFoundError, OSError):
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
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self._t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- byte model
def stage_bytes(info: dict, stage: str) -> float:
    """Algorithmic DRAM bytes of one launch of a stage (3D, sigma = 2 Hermitian layout).

    s = real size, b = 2 s complex size, N grid, n fine grid, nh = n/2 + 1 stored planes,
    M = half node count.  FFT passes read their input once and write their output once.  The
    node kernels follow the whole-path model s (51.4 N^3 + 2 N_f): each touches the ball
    |t| < pi of the half grid once ((pi/12) n^3 cells) and carries half of the node stream of
    four values per node (2 N_f s over the path, i.e. two values, M b, per kernel).
    """
    s = 4.0 if info["precision"] == 0 else 8.0
    b = 2 * s
    N, n, M = info["n"], info["n_fine"], info["n_half_nodes"]
    nh = n // 2 + 1
    ball = (np.pi / 12.0) * n ** 3 * b
    table = {
        "fwd_fft_z": N ** 3 * s + nh * N * N * b,
        "fwd_fft_y": nh * N * N * b + nh * n * N * b,
        "fwd_fft_x": nh * n * N * b + nh * n * n * b,
        "interp": ball + M * b,
        "spread": ball + M * b,
        "inv_fft_x": nh * n * n * b + nh * n * N * b,
        "inv_fft_y": nh * n * N * b + nh * N * N * b,
        "inv_fft_z": nh * N * N * b + 2 * N ** 3 * s,
        "energy": 0.0,
    }
    return float(table[stage])


def layout_bytes(info: dict, stage: str) -> float:
    """DRAM bytes of one launch as the kernels store their data: the ball once plus the node
    records each node kernel reads and writes (FP32 plans: a 16-byte record of the packed
    stencil origin and three offsets; FP64 plans: the packed origin and the d w stencil values
    the plan precomputes), W and c.  Reported beside the algorithmic model, which ``frac``
    divides by."""
    s = 4.0 if info["precision"] == 0 else 8.0
    b = 2 * s
    n, M = info["n_fine"], info["n_half_nodes"]
    ball = (np.pi / 12.0) * n ** 3 * b
    rec = 16.0 if info["precision"] == 0 else 4.0 + 3 * info["w"] * s
    if stage == "interp":
        return float(ball + M * (rec + s + b))
    if stage == "spread":
        return float(ball + M * (rec + b))
    return stage_bytes(info, stage)


def run_alg2(pkg, torch, dev, wl, rho32, flush, stream, args, ms_step, ms64=None, u64=None):
    """Algorithm 2 (eq. 3.9) on the benchmark workload in FP32 and FP64: time per evaluation
    (L2 flushed), the FP32 result against the FP64 one (same operator), and the FP64 result
    against the FP64 Algorithm 1 result in the interior |x| < 8 (both resolve it; Algorithm 1's
    node set does not resolve the box corners to 1e-5)."""
    res, us = {}, {}
    for prec in ("fp32", "fp64"):
        if prec == "fp64" and args.no_fp64:
            continue
        torch.cuda.nvtx.range_push(f"alg2_{prec}")  # ncu --nvtx-include selects a leg
        p2 = pkg.Plan(wl.d, wl.n, wl.L, wl.kernel, precision=prec,
                      eps=1e-6 if prec == "fp32" else 1e-12, algorithm=2, device=dev.index)
        r = rho32 if prec == "fp32" else torch.from_numpy(wl.rho()).to(dev)
        uu = torch.empty_like(r)
        EE = torch.empty((), dtype=torch.float64, device=dev)
        for _ in range(max(2, args.warmup)):
            p2.eval_energy(r, lam=wl.lam, out=uu, E_out=EE)
        k2 = args.steps if prec == "fp32" else max(2, min(args.steps, 5))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * k2)]
        for k in range(k2):
            flush.fill_(float(k))
            ev[2 * k].record(stream)
            p2.eval_energy(r, lam=wl.lam, out=uu, E_out=EE)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        ms = statistics.median(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(k2))
        inf = p2.info
        res[prec] = {"value": wl.n_points / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "energy": float(EE.item()), "w": inf["w"], "I2_nodes": inf["n_nodes"],
                     "a": inf["pu_a"], "P2": inf["P2"]}
        us[prec] = uu.double()
        p2.close()
        torch.cuda.nvtx.range_pop()
    out = {"workload": "same as the headline (3D Coulomb 256^3, 16-Gaussian mixture); "
                       "I_1 by the 2x zero-padded FFT, I_2 by the NUFFT on 32x32x64 (FP32) / "
                       "40x40x80 (FP64) nodes of radius P2 = 6.1 sqrt(a), a = (11.8/L)^2",
           "fp32": res["fp32"], "fp64": res.get("fp64"),
           "speedup_vs_algorithm1_fp32": ms_step / res["fp32"]["ms_per_step"]}
    if "fp64" in res:
        out["rel_linf_fp32_vs_fp64"] = float((us["fp32"] - us["fp64"]).abs().max() / us["fp64"].abs().max())
        out["speedup_fp32_vs_fp64"] = res["fp64"]["ms_per_step"] / res["fp32"]["ms_per_step"]
        if ms64:
            out["speedup_vs_algorithm1_fp64"] = ms64 / res["fp64"]["ms_per_step"]
        if u64 is not None:
            z, y, x = synth.grid_coords(3, wl.n, wl.L)
            inner = torch.from_numpy((x * x + y * y + z * z) < 64.0).to(dev)
            d = (us["fp64"] - u64).abs()
            out["rel_linf_vs_algorithm1_fp64_interior"] = float(d[inner].max() / u64.abs().max())
            out["rel_linf_vs_algorithm1_fp64_whole_box"] = float(d.max() / u64.abs().max())
    return out


FP64_TFLOPS = 1.25   # nominal dense FP64 rate of a GB300 (FP64 vector units)
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def node_flops(info: dict) -> float:
    """Algorithmic flops of one interpolation plus one spreading over the half node set: per
    stencil cell a complex-by-real multiply-add in each (8 w^d flops per node)."""
    return 8.0 * info["w"] ** info["d"] * info["n_half_nodes"]


def run_configs(pkg, torch, dev, flush, stream, reps=5):
    """The other single-density configurations (3D Coulomb 32^3, 2.5D Coulomb 512^2, 3D dipole
    128^3) in FP32 and FP64: time per evaluation (L2 flushed), throughput, and the FP32 result's
    error against the FP64 GPU result (u: relative L-inf; E: relative to the FP64 energy's
    magnitude)."""
    out = {}
    for name in ("c1", "c2", "c3"):
        wl = synth.CONFIGS[name]()
        rho64 = torch.from_numpy(wl.rho()).to(dev)
        res, us, Es = {}, {}, {}
        for prec in ("fp32", "fp64"):
            plan = pkg.Plan(wl.d, wl.n, wl.L, wl.kernel, axis=wl.axis, nodes=wl.nodes, precision=prec,
                            eps=1e-6 if prec == "fp32" else 1e-12, device=dev.index)
            r = rho64 if prec == "fp64" else rho64.float()
            u = torch.empty_like(r)
            E = torch.empty((), dtype=torch.float64, device=dev)
            for _ in range(3):
                plan.eval_energy(r, lam=wl.lam, out=u, E_out=E)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
            for k in range(reps):
                flush.fill_(float(k))
                ev[2 * k].record(stream)
                plan.eval_energy(r, lam=wl.lam, out=u, E_out=E)
                ev[2 * k + 1].record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps))
            res[prec] = {"ms_per_step": ms, "value": wl.n_points / (ms / 1e3), "w": plan.info["w"]}
            us[prec], Es[prec] = u.double(), float(E.item())
            plan.close()
        out[name] = {"workload": wl.desc, "unit": UNIT, "fp32": res["fp32"], "fp64": res["fp64"],
                     "speedup_fp32_vs_fp64_gpu": res["fp64"]["ms_per_step"] / res["fp32"]["ms_per_step"],
                     "rel_linf_fp32_vs_fp64": float((us["fp32"] - us["fp64"]).abs().max()
                                                    / us["fp64"].abs().max()),
                     "rel_energy_fp32_vs_fp64": abs(Es["fp32"] - Es["fp64"]) / abs(Es["fp64"])}
    return out


def fft_yardstick(torch, dev, wl, n_fine, flush, stream, stages, reps=5):
    """cuFFT (torch.fft) on the same oversampled grid, as a timing yardstick only (never on the
    path): the full real-to-complex transform of the zero-padded n_fine^3 density and the
    complex-to-real transform back, against the path's three forward and three inverse passes
    (which also deconvolve, prune to the stored modes and window, and fold)."""
    x = torch.zeros((n_fine,) * 3, dtype=torch.float32, device=dev)
    x[: wl.n, : wl.n, : wl.n] = torch.from_numpy(wl.rho()).to(dev, torch.float32)
    X = torch.fft.rfftn(x)
    y = torch.fft.irfftn(X, s=x.shape)
    ms = {"rfftn": [], "irfftn": []}
    for k in range(reps + 1):
        for name in ms:
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if name == "rfftn":
                X = torch.fft.rfftn(x)
            else:
                y = torch.fft.irfftn(X, s=x.shape)
            b.record(stream)
            torch.cuda.synchronize()
            if k > 0:
                ms[name].append(a.elapsed_time(b))
    del x, X, y
    ours_f = sum(stages.get(k, 0.0) for k in ("fwd_fft_z", "fwd_fft_y", "fwd_fft_x"))
    ours_i = sum(stages.get(k, 0.0) for k in ("inv_fft_x", "inv_fft_y", "inv_fft_z"))
    return {"what": f"cuFFT via torch.fft on the {n_fine}^3 FP32 zero-padded grid (yardstick, not "
                    "on the path) vs the path's pruned passes with their fused deconvolution",
            "cufft_rfftn_ms": statistics.median(ms["rfftn"]),
            "cufft_irfftn_ms": statistics.median(ms["irfftn"]),
            "ours_forward_passes_ms": ours_f, "ours_inverse_passes_ms": ours_i}


def path_bytes(info: dict) -> float:
    """Whole-path algorithmic bytes per evaluation: s (51.4 N^3 + 2 N_f) in 3D."""
    s = 4.0 if info["precision"] == 0 else 8.0
    return s * (51.4 * info["n"] ** 3 + 2 * info["n_nodes"])


# ----------------------------------------------------------------------------- oracle arm
def cpu_model() -> str:
    """The host CPU's model name: /proc/cpuinfo on x86, lscpu's "Model name" on Arm (whose
    /proc/cpuinfo has part numbers only), else the machine type."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def time_oracle_eval(rho, L, nodes, setting, node_stride=1, node_offset=0):
    """Seconds for one FP64 oracle evaluation (Algorithm 1 by the Gaussian-gridding NUFFT of
    Section 2 at `setting`: type 2, multiply, type 1, energy) of the 3D Coulomb operator on
    rho, over every node_stride-th node of the spherical node set (starting at node_offset)."""
    from oracle import nufft, pipeline, quadrature
    n = rho.shape[0]
    t0 = time.perf_counter()
    k, W = quadrature.nodes_weights(3, n, L, nodes, "coulomb")
    k, W = k[node_offset::node_stride], W[node_offset::node_stride]
    rh = pipeline.type2(rho, L, k, "nufft", setting)
    u = pipeline.type1(W * rh, 3, n, L, k, "nufft", setting).real
    pipeline.energy(u, rho, L)
    return time.perf_counter() - t0, nufft.threads()


def cpu_baseline_obj():
    """The FP64 CPU oracle on this machine's host cores, on the benchmark workload itself (the
    256^3 grid, its 16-Gaussian density and its 160x160x320 node set): one full evaluation at
    the paper's 6-digit setting (Section 2: oversampling 2, tau = 6/N^2, 12 points), which is
    the line's value, and the parity setting (sigma = 3, w = 28) on every 64th node of the same
    node set (a full parity evaluation takes minutes)."""
    wl = synth.config4()
    rho = wl.rho()
    dt, cores = time_oracle_eval(rho, wl.L, wl.nodes, "paper6")
    dtp, _ = time_oracle_eval(rho, wl.L, wl.nodes, "parity", node_stride=64)
    return {"value": rho.size / dt, "unit": UNIT, "cores": cores, "cpu": cpu_model(),
            "kind": "oracle",
            "sample": (f"one FP64 oracle evaluation of the benchmark workload (256^3, 16 Gaussians, "
                       f"160x160x320 nodes) at the paper's 6-digit setting (sigma=2, tau=6/N^2, "
                       f"12 points): {dt:.1f} s"),
            "settings": {"paper6": {"seconds": dt, "nodes": "all", "runs": 1},
                         "parity": {"seconds": dtp, "nodes": "every 64th",
                                    "what": "sigma=3, w=28 on 1/64 of the node set (FFTs full)"}}}


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle (the paper ships no code) on the benchmark
    workload's grid and density.  A full evaluation takes about 15 s on 16 cores, so each step,
    warm-up or timed, is one evaluation over a quarter of the node set (every 4th node, the
    offset rotating with the step): the FFTs are full, the node work a quarter."""
    if rank != 0:
        return 0
    wl = synth.config4()
    rho = wl.rho()
    for k in range(args.warmup):
        time_oracle_eval(rho, wl.L, wl.nodes, "paper6", node_stride=4, node_offset=k % 4)
    times, cores = [], 1
    for k in range(args.steps):
        dt, cores = time_oracle_eval(rho, wl.L, wl.nodes, "paper6", node_stride=4, node_offset=k % 4)
        times.append(dt)
    tot = sum(times)
    value = rho.size * args.steps / tot
    sample = ("per step one FP64 oracle evaluation at the paper's 6-digit setting (sigma=2, "
              "tau=6/N^2, 12 points) of the benchmark workload's 256^3 grid and 16-Gaussian "
              "density over every 4th node of its 160x160x320 node set (rotating offset)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "3D Coulomb 256^3 over [-16,16]^3, 16 seeded Gaussians, "
                                   "160x160x320 nodes (CPU oracle, a quarter of the nodes per step)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": cpu_model(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- batched form
def tuned_member_params(pkg, members, precision, dev):
    """Autotuned parameters for every member of the batch (nlint_autotune_batch): one tuning per
    (grid size, kernel) class (width for the tolerance, bin shape, subproblem size), then the
    whole batch timed with the classes' own fastest decompositions and with the default one, the
    faster kept.  Returns the member parameters (each with its own dipole axis) and the report."""
    tol = TOL if precision == "fp32" else 1e-10
    cache = os.environ.get("NLINT_TUNE_CACHE")
    prm = [pkg.make_params(3, m.n, m.L, m.kernel, axis=m.axis, nodes=m.nodes, precision=precision,
                           device=dev.index) for m in members]
    out, reps, brep = pkg.autotune_batch(prm, tol, cache)
    classes = {}
    for m, r in zip(members, reps):
        classes.setdefault(f"{m.n}^3 {m.kernel}", {k: r[k] for k in ("w", "bin_shape", "max_sub", "err",
                                                                       "w_alt", "err_alt", "fft_sched")})
    kinds = ("each class's own fastest decomposition and width", "the default decomposition",
             "the default decomposition at each class's other width")
    batch = {"kept": kinds[brep["choice"]], "ms": {k: t for k, t in zip(kinds, brep["ms"]) if t > 0}}
    return out, {"classes": classes, "batch": batch}


def run_batched(pkg, torch, dev, precision, reps, flush, stream, loop_too=False, tune=False):
    """64 seeded densities on uneven grids {32,48,64,96,128}^3 (box [-12,12]^3, 16-Gaussian
    mixtures, half Coulomb and half dipolar with seeded axes), one plan each, evaluated by one
    captured CUDA graph.  Returns throughput (total grid points per second) and, optionally, the
    same plans evaluated one after another on one stream.  tune=True builds every plan from
    autotuned parameters (tuned_member_params) instead of the width rule of eps."""
    members = synth.config5(precision)
    eps = 1e-6 if precision == "fp32" else 1e-12
    dt = torch.float32 if precision == "fp32" else torch.float64
    tune_rep = None
    if tune:
        t0 = time.perf_counter()
        prms, tune_rep = tuned_member_params(pkg, members, precision, dev)
        tune_rep["seconds"] = time.perf_counter() - t0
        plans = [pkg.Plan(3, m.n, m.L, params=q, device=dev.index) for m, q in zip(members, prms)]
    else:
        plans = [pkg.Plan(3, m.n, m.L, m.kernel, axis=m.axis, nodes=m.nodes, precision=precision,
                          eps=eps, device=dev.index) for m in members]
    rhos = [torch.from_numpy(m.rho()).to(dev, dt) for m in members]
    points = sum(m.n_points for m in members)
    batch = pkg.Batch(plans)
    for _ in range(3):
        batch.eval(rhos)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    for k in range(reps):
        flush.fill_(float(k))
        ev[2 * k].record(stream)
        batch.eval(rhos)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps))
    info = batch.info()
    out = {"value": points / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "densities": len(members),
           "grid_points": points, "kernels_per_eval": info["kernels_per_eval"],
           "branches": info["branches"], "sizes": sorted({m.n for m in members}),
           "autotuned": tune_rep}
    if loop_too:
        us = [torch.empty_like(r) for r in rhos]
        Es = torch.empty(len(rhos), dtype=torch.float64, device=dev)
        for k in range(reps + 1):
            flush.fill_(float(k))
            ev[0].record(stream)
            for i, (p, r) in enumerate(zip(plans, rhos)):
                p.eval_energy(r, out=us[i], E_out=Es[i])
            ev[1].record(stream)
            torch.cuda.synchronize()
            if k == 0:
                continue
            ms_loop = ev[0].elapsed_time(ev[1])
        out["one_by_one_ms"] = ms_loop
        out["speedup_vs_one_by_one"] = ms_loop / ms
    batch.close()
    # the same batch with every plan's Toeplitz kernel precomputed: the graph then runs the FFT
    # passes only (the same operators to the NUFFT tolerance); precompute time reported apart
    t0 = time.perf_counter()
    for p in plans:
        p.toeplitz()
    t_pre = time.perf_counter() - t0
    batch = pkg.Batch(plans)
    for _ in range(3):
        batch.eval(rhos)
    torch.cuda.synchronize()
    for k in range(reps):
        flush.fill_(float(k))
        ev[2 * k].record(stream)
        batch.eval(rhos)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    ms_t = statistics.median(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps))
    out["toeplitz_form"] = {"value": points / (ms_t / 1e3), "unit": UNIT, "ms_per_step": ms_t,
                            "precompute_s": t_pre,
                            "kernels_per_eval": batch.info()["kernels_per_eval"]}
    batch.close()
    for p in plans:
        p.close()
    return out


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1311_4120_gb300 as pkg
    from paper_1311_4120_gb300 import build as nb

    if rank == 0 or not os.path.exists(nb.LIB):
        nb.build()
    if world > 1:
        torch.distributed.barrier()
    pkg.load_library()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    wl = synth.config4()
    rho_np = wl.rho().astype(np.float32)
    # the FP32 plan for the stated tolerance: the autotuner measures the stencil width that
    # meets TOL/2 against an FP64 plan and the fastest subproblem size (NLINT_TUNE_CACHE reuses it)
    prm = pkg.make_params(wl.d, wl.n, wl.L, wl.kernel, nodes=wl.nodes, precision="fp32",
                          device=local_rank)
    t0 = time.perf_counter()
    tuned, tune_rep = pkg.autotune(prm, TOL, os.environ.get("NLINT_TUNE_CACHE"))
    tune_rep["seconds"] = time.perf_counter() - t0
    plan = pkg.Plan(wl.d, wl.n, wl.L, params=tuned, device=local_rank)
    info = plan.info
    rho = torch.from_numpy(rho_np).to(dev)
    u = torch.empty_like(rho)
    E = torch.empty((), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        plan.eval_energy(rho, lam=wl.lam, out=u, E_out=E)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each, per-step CUDA events on the stream; no
    # events between the stages of an evaluation (they would serialise its dependent launches)
    # and no host synchronisation inside the loop
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = plan.launch_count()
    barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("headline")
    with ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else
                      int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank])) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            plan.eval_energy(rho, lam=wl.lam, out=u, E_out=E)
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall0
    torch.cuda.nvtx.range_pop()
    launches = plan.launch_count() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]

    # ---- the same K steps again with CUDA events between the stages (on the evaluation stream),
    # for the per-kernel durations of the stage split and the roofline
    plan.set_stage_timing(True)
    stage_ms = {}
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        plan.eval_energy(rho, lam=wl.lam, out=u, E_out=E)
        for name, ms in plan.stage_times():
            stage_ms.setdefault(name, []).append(ms)
    torch.cuda.synchronize()
    plan.set_stage_timing(False)
    t_dev = sum(step_ms) / 1e3
    (t_max,) = max_over_ranks([t_dev], dev)
    points = wl.n_points * args.steps * world
    value = job_rate(wl.n_points * args.steps, world, t_max)
    E32 = float(E.item())
    u32 = u.clone()

    # ---- end to end through the host-buffer entry points (pinned host memory): the streaming
    # entry point (copies of step k+1's density and step k-1's u overlapped with step k's
    # evaluation) is the e2e value; one synchronous call per step is reported beside it
    rho_h = [torch.from_numpy(rho_np).pin_memory() for _ in range(2)]
    u_h = [torch.empty(rho_h[0].shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    rhos_k = [rho_h[k % 2] for k in range(args.steps)]
    us_k = [u_h[k % 2] for k in range(args.steps)]
    plan.eval_host_many(rhos_k[:2], lam=wl.lam, us_host=us_k[:2])
    for _ in range(2):
        plan.eval_host(rho_h[0], lam=wl.lam, u_host=u_h[0])
    barrier()
    t0 = time.perf_counter()
    plan.eval_host_many(rhos_k, lam=wl.lam, us_host=us_k)
    t_e2e = time.perf_counter() - t0
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.eval_host(rho_h[0], lam=wl.lam, u_host=u_h[0])
    t_sync = time.perf_counter() - t0
    t_e2e, t_sync = max_over_ranks([t_e2e, t_sync], dev)
    e2e = {"value": points / t_e2e, "unit": UNIT, "h2d_bytes_per_step": rho_np.nbytes,
           "d2h_bytes_per_step": rho_np.nbytes + 8,
           "api": "nlint_eval_host_many: K steps in one call, copies overlapped with evaluations",
           "one_call_per_step": {"api": "nlint_eval_host (synchronous)", "value": points / t_sync}}

    # ---- the same operator in its precomputed Toeplitz form (FFT passes only per evaluation)
    toep = None
    if not args.no_toeplitz:
        t0 = time.perf_counter()
        plan.toeplitz()
        t_pre = time.perf_counter() - t0
        ut = torch.empty_like(u)
        Et = torch.empty((), dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            plan.eval_toeplitz(rho, lam=wl.lam, out=ut, E_out=Et)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[2 * k].record(stream)
            plan.eval_toeplitz(rho, lam=wl.lam, out=ut, E_out=Et)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        ms_t = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)) / args.steps
        toep = {"value": wl.n_points / (ms_t / 1e3), "unit": UNIT, "ms_per_step": ms_t,
                "precompute_s": t_pre,
                "rel_linf_vs_nufft_path": float((ut.double() - u32.double()).abs().max()
                                                / u32.double().abs().max()),
                "energy": float(Et.item())}

    # ---- the same workload on the FP64 GPU path: speedup and the FP32 result's error
    fp64 = None
    if not args.no_fp64:
        plan64 = pkg.Plan(wl.d, wl.n, wl.L, wl.kernel, nodes=wl.nodes, eps=1e-12, precision="fp64",
                          device=local_rank)
        rho64 = torch.from_numpy(wl.rho()).to(dev)
        u64 = torch.empty_like(rho64)
        E64 = torch.empty((), dtype=torch.float64, device=dev)
        for _ in range(2):
            plan64.eval_energy(rho64, lam=wl.lam, out=u64, E_out=E64)
        k64 = max(2, min(args.steps, 5))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * k64)]
        for k in range(k64):
            flush.fill_(float(k))
            ev[2 * k].record(stream)
            plan64.eval_energy(rho64, lam=wl.lam, out=u64, E_out=E64)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        ms64 = statistics.median(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(k64))
        # FP64 ALU roofline of the node kernels: one more evaluation with the stage events
        plan64.set_stage_timing(True)
        plan64.eval_energy(rho64, lam=wl.lam, out=u64, E_out=E64)
        torch.cuda.synchronize()
        st64 = dict(plan64.stage_times())
        plan64.set_stage_timing(False)
        i64 = plan64.info
        fl = node_flops(i64)
        t_nodes = (st64["interp"] + st64["spread"]) / 1e3
        fp64 = {"value": wl.n_points / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "w": i64["w"], "energy": float(E64.item()),
                "rel_linf_fp32_vs_fp64": float((u32.double() - u64).abs().max() / u64.abs().max()),
                "rel_energy_fp32_vs_fp64": abs(E32 - float(E64.item())) / abs(float(E64.item())),
                "stages_ms": {k: round(v, 3) for k, v in st64.items()},
                "roofline": {"bound": "alu", "kernel": "interp+spread", "unit": "TFLOP/s",
                             "algorithmic_flops": fl, "achieved": fl / t_nodes / 1e12,
                             "peak": FP64_TFLOPS, "peak_kind": "nominal FP64 (no measured figure)",
                             "frac": fl / t_nodes / 1e12 / FP64_TFLOPS}}
        plan64.close()
        del rho64

    # ---- Algorithm 2 (partition of unity, eq. 3.9) on the same workload
    alg2 = None
    if not args.no_alg2:
        alg2 = run_alg2(pkg, torch, dev, wl, rho, flush, stream, args, ms_step=1e3 * t_max / args.steps,
                        ms64=fp64["ms_per_step"] if fp64 else None, u64=u64 if fp64 else None)
    if fp64:
        del u64

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel (stage events on the launch stream)
    mean_stage = {k: sum(v) / len(v) for k, v in stage_ms.items()}
    dom = max(mean_stage, key=mean_stage.get)
    peak, peak_kind = peaks()
    roof = {"bound": "hbm"}
    ach = stage_bytes(info, dom) / (mean_stage[dom] / 1e3) / 1e9
    tr = TRAFFIC.get(dom)
    traffic = tr["bytes"] if (tr and tr.get("src") == _src_hash(dom)) else None
    roof.update({"kernel": dom, "achieved": ach, "peak": peak, "peak_kind": peak_kind,
                 "unit": "GB/s", "frac": ach / peak, "traffic": traffic,
                 "algorithmic_bytes": stage_bytes(info, dom),
                 "model": "ball (pi/12) n^3 b + half node stream M b (whole path s (51.4 N^3 + 2 N_f))",
                 "layout_bytes": layout_bytes(info, dom),
                 "mean_ms": mean_stage[dom]})
    # the node kernels against the FP32 ALU rate as well (they are issue-bound, not flop-bound)
    t_nodes32 = (mean_stage.get("interp", 0.0) + mean_stage.get("spread", 0.0)) / 1e3
    if t_nodes32 > 0:
        roof["alu_view"] = {"kernel": "interp+spread", "unit": "TFLOP/s",
                            "achieved": node_flops(info) / t_nodes32 / 1e12,
                            "peak": FP32_TFLOPS, "peak_kind": "nominal FP32 (SM count x lanes x clock)",
                            "frac": node_flops(info) / t_nodes32 / 1e12 / FP32_TFLOPS}
    ms_step = 1e3 * t_max / args.steps
    path_gbs = path_bytes(info) / (ms_step / 1e3) / 1e9

    batched = None
    if not args.no_batch:
        b32 = run_batched(pkg, torch, dev, "fp32", 5, flush, stream, loop_too=True, tune=True)
        b32_untuned = run_batched(pkg, torch, dev, "fp32", 5, flush, stream)
        b32["untuned"] = {"value": b32_untuned["value"], "ms_per_step": b32_untuned["ms_per_step"],
                          "what": "every plan at the width rule of eps = 1e-6 and default bins"}
        b64 = run_batched(pkg, torch, dev, "fp64", 3, flush, stream)
        batched = {"workload": "64 seeded densities on {32,48,64,96,128}^3 grids over [-12,12]^3, "
                               "half Coulomb, half dipole, one CUDA graph",
                   "fp32": b32, "fp64": b64,
                   "speedup_fp32_vs_fp64_gpu": b64["ms_per_step"] / b32["ms_per_step"]}
    configs = None if args.no_configs else run_configs(pkg, torch, dev, flush, stream)
    yard = None if args.no_yardstick else fft_yardstick(torch, dev, wl, info["n_fine"], flush,
                                                         stream, mean_stage)
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline_obj()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3D Coulomb 256^3 over [-16,16]^3, rho = 16 seeded Gaussians, "
                               "160x160x320 spherical nodes, FP32 path (FP64 nodes/weights, "
                               "compensated FP64 energy)",
                   "w": info["w"], "sigma": info["sigma"], "n_fine": info["n_fine"],
                   "max_sub": tuned.max_sub, "bin_shape": tuned.bin_shape,
                   "fft_sched": tuned.fft_sched, "tolerance": TOL,
                   "autotune": tune_rep,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "energy": E32,
        "fp64_gpu": fp64,
        "speedup_fp32_vs_fp64_gpu": (fp64["ms_per_step"] / ms_step) if fp64 else None,
        "batched": batched,
        "toeplitz_form": toep,
        "algorithm2": alg2,
        "other_configs": configs,
        "fft_yardstick": yard,
        "stages_ms": {k: round(v, 4) for k, v in mean_stage.items()},
        "path_bytes_per_step": path_bytes(info),
        "path_frac_of_hbm": path_gbs / peak,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s_timed_region": t_wall,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-density batched form")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-toeplitz", action="store_true", help="skip the precomputed-kernel form")
    ap.add_argument("--no-alg2", action="store_true", help="skip the Algorithm 2 leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the other single-density configs")
    ap.add_argument("--no-yardstick", action="store_true", help="skip the cuFFT timing yardstick")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
