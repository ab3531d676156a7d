"""Throughput of the G1-G2 RK4 propagation on GB300.

One bench "step" is one RK4 step of each of the two workloads the metric names,
back to back: the general-basis SOA system at nb = 96 and the general-basis GW
system at nb = 64 (seeded h, w = Σ_P L^P ⊗ L^P, gauss-sine pulse; the
`inputs` module).  Together they run every stage of the right-hand side (HF
build, collision integral, two-particle commutator, source term, GW
quasi-Hamiltonian and polarisation, assembly + RK4, observables).
value = bench steps per second = 1 / (t_SOA96 + t_GW64).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x4|tf32x3|fp64]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

With N > 1 (torchrun) every rank runs an independent replica of the same
propagation on its own GPU (the method has no data-parallel split without an
exchange step that is not built); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
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

from paper_2002_12717_gb300 import inputs  # noqa: E402

METRIC = "G1-G2 RK4 steps/s (one step = SOA nb=96 + GW nb=64)"
WORKLOADS = ("general-soa-nb96", "general-gw-nb64")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 (DFMA) throughput of one GB300 (profiles/fp64_dfma_peak.md: the FP64 GEMM sustains
# 1.212 TFLOP/s; `--fp64-peak` runs the committed probe, a lower bound); used as the ALU
# roofline of the FP64 form.
FP64_PEAK_TFLOPS = 1.200
FP64_PEAK_NOTE = "profiles/fp64_dfma_peak.md"
# nominal dense tensor ratio TF32 / BF16 (1.1 / 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25
# DRAM bytes (read + write) per launch of the dominant kernel, keyed by (kernel tag,
# workload), from one ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum, profiles/); missing entries report null.
TRAFFIC = {("tc_gemm_pi", "general-gw-nb64"): 1875060000 + 123198464}   # profiles/tc_pi_gemm_gw64.md
# sm__pipe_tensor_cycles_active (percent of peak, sustained over active cycles) of the
# dominant kernel from the same capture; missing entries report null.
TENSOR_PIPE = {("tc_gemm_pi", "general-gw-nb64"): 89.2}


def load_peaks():
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# algorithmic work per launch of each kernel family
# ---------------------------------------------------------------------------

def algorithmic_flops(nb, se, stage_launches=None):
    """Paper-level work of one RK4 step: 8 real flops per complex MAC.

    Per right-hand side: collision integral nb^5, commutator 4 nb^5, source
    term 4 nb^5 (successive contractions), GW: quasi-Hamiltonian 2 nb^5 and
    polarisation nb^6.  Four right-hand sides per step.
    """
    n5 = nb ** 5
    per_rhs = 9 * n5 + (2 * n5 + nb ** 6 if se == "GW" else 0)
    return 8.0 * per_rhs * 4


# tensor products issued per real multiply-add: TF32 hi/lo (3) or BF16 slices (10 in the
# nb^5 passes, 6 in the nb^2 x nb^2 x nb^2 products of tc_pi_gemm_kernel)
SPLIT_PRODUCTS = {"tf32x3": 3, "bf16x4": 10}
SPLIT_PRODUCTS_PI = {"tf32x3": 3, "bf16x4": 6}


def kernel_work(tag, nb, se, precision="tf32x3"):
    """(bound, algorithmic work per launch, issued work per launch) of the dominant-kernel
    candidates.

    Algorithmic work is the contraction the launch evaluates at 8 real flops per
    complex multiply-add (4 per real-by-complex one): the polarisation and the
    ladder products nb^6 complex MACs, a complex nb^5 pass nb^5, a pass with the
    real w as A (source pass 1, quasi-Hamiltonian, collision) nb^5 real-by-complex
    MACs.  Issued work counts the split-precision products the kernel runs on the
    realified problem (three TF32 products, or ten BF16 slice products in the nb^5
    passes and six in the nb^2 x nb^2 x nb^2 products, per real multiply-add, 2 flops
    each): issued / algorithmic is the cost of the emulated
    FP32-class accuracy.  The assembly counts its algorithmic HBM bytes averaged over
    the four RK4 stages: the FP32 intermediates Z and Q (and Pi for GW), the FP32
    state copy (stages 0-2) or the FP64 state (last stage), the FP32 accumulator
    (read at stages 1-3), and the stores (accumulator and stage input at stages 0-2,
    FP64 state and its FP32 copy at the last).
    """
    n = float(nb)
    split = SPLIT_PRODUCTS.get(precision, 3) * 2
    if tag in ("tc_gemm_pi", "tc_gemm_ladder"):
        return "tensor", 8 * n ** 6, SPLIT_PRODUCTS_PI.get(precision, 3) * 2 * n * n * (2 * n * n) * (2 * n * n)
    if tag in ("tc_gemm_commutator", "tc_gemm_psi2", "tc_gemm_psi3", "tc_gemm_psi4"):
        return "tensor", 8 * n ** 5, split * n ** 3 * (2 * n) * (2 * n)
    if tag in ("tc_gemm_psi1", "tc_gemm_hcorr"):
        return "tensor", 4 * n ** 5, split * n ** 3 * (2 * n) * n
    if tag == "tc_gemm_collision":
        return "tensor", 4 * n ** 5, split * (2 * n) * n * n ** 3
    if tag == "tc_orbit_assemble_rk4":
        per_elem = 8 + 8 + (3 * 8 + 16) / 4 + 0.75 * 8 + (3 * 16 + 24) / 4 + (8 if se == "GW" else 0)
        return "hbm", per_elem * n ** 4, per_elem * n ** 4
    if tag in ("fp64_zgemm", "fp64_zgemm_splitk"):
        return "alu", None, None
    return None, None, None


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def max_over_ranks(values_ms, dist):
    """Per-entry maximum over the ranks of per-rank times (the slowest replica sets the job's rate)."""
    if dist is None:
        return [float(v) for v in values_ms]
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_rate(world, ms_per_step):
    """Whole-job steps/s of `world` independent replicas that each take at most ms_per_step per step."""
    return world * 1e3 / ms_per_step


def run_ours(args, rank, world, dist):
    import torch

    from paper_2002_12717_gb300.g1g2 import from_workload

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    peaks, peak_kind = load_peaks()

    def barrier():
        if dist is not None:
            dist.barrier()

    per = {}
    prof_all = {}
    per_kernel = {}
    launches_total = 0
    clocks = ClockSampler(dev)
    for name in args.workloads:
        d = inputs.workload(name)
        prop = from_workload(d, precision=args.precision)
        dt = d["dt"]
        prop.propagate(dt, args.warmup)          # warm-up steps (untimed)
        torch.cuda.synchronize()
        barrier()
        c0 = prop.launch_count
        if not per:
            clocks.start()
        # the library launches on the default stream, where these events are recorded
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record()
        for _ in range(args.steps):
            prop.step(dt)
        end.record()
        torch.cuda.synchronize()
        ms = start.elapsed_time(end) / args.steps
        launches = prop.launch_count - c0
        launches_total += launches
        # per-kernel device time from a separate pass of the same number of steps, with a
        # CUDA-event pair around every launch (kept out of the timed region above)
        prop.profile(True)
        for _ in range(args.steps):
            prop.step(dt)
        rep = prop.profile_report()
        prop.profile(False)
        for k, (n_l, t_ms) in rep.items():
            a = prof_all.setdefault(k, [0, 0.0, 0.0])
            a[0] += n_l
            a[1] += t_ms
        per_kernel[name] = rep
        # algorithmic flops of the contraction kernels of this workload
        per[name] = {"nb": d["nb"], "selfenergy": d["selfenergy"], "ms_per_step": ms, "launches": launches,
                     "flops_per_step": algorithmic_flops(d["nb"], d["selfenergy"], None), "dt": dt}
        # end-to-end through the public API: state from pinned host memory, K steps,
        # observables (energies + density) copied back after every step
        n0 = torch.from_numpy(np.ascontiguousarray(d["n0"])).pin_memory().numpy()
        g0 = torch.zeros((d["nb"],) * 4, dtype=torch.complex128).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prop.set_state(0.0, n0, g0)
        obs, _ = prop.propagate(dt, args.steps, 1)
        e2e_s = time.perf_counter() - t0
        per[name]["e2e_ms_per_step"] = 1e3 * e2e_s / args.steps
        per[name]["h2d_bytes"] = n0.nbytes + g0.nbytes
        per[name]["d2h_bytes_per_step"] = 56 + 16 * d["nb"]
        per[name]["energy_drift_rel"] = abs(obs[-1]["e_total"] - obs[0]["e_total"] - obs[-1]["pulse_work"]) / abs(
            obs[0]["e_total"])
        if args.compare_steps > 0 and args.precision != "fp64":
            # same steps from the same initial state in the FP64 form: speed-up and error
            c = args.compare_steps
            prop.set_state(0.0, d["n0"], None)
            obs_m, _ = prop.propagate(dt, c, c)
            _, n_m, g_m = prop.get_state()
            ref = from_workload(d, precision="fp64")
            ref.propagate(dt, 1)
            ref.set_state(0.0, d["n0"], None)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            obs_r, _ = ref.propagate(dt, c, c)
            e1.record()
            torch.cuda.synchronize()
            _, n_r, g_r = ref.get_state()
            ref.close()
            del ref
            per[name]["fp64_ms_per_step"] = e0.elapsed_time(e1) / c
            per[name]["vs_fp64"] = {
                "steps": c, "max_abs_dG1": float(np.abs(n_m - n_r).max()),
                "max_abs_dG2": float(np.abs(g_m - g_r).max()),
                "rel_dE": abs(obs_m[-1]["e_total"] - obs_r[-1]["e_total"]) / abs(obs_r[-1]["e_total"])}
        prop.close()
        del prop
        torch.cuda.empty_cache()
        barrier()
    clk = clocks.stop()

    step_ms, e2e_ms = max_over_ranks([sum(p["ms_per_step"] for p in per.values()),
                                      sum(p["e2e_ms_per_step"] for p in per.values())], dist)
    value = job_rate(world, step_ms)
    e2e_value = job_rate(world, e2e_ms)

    # roofline of the dominant kernel: the (kernel, workload) pair with the largest device time
    total_ms = sum(v[1] for v in prof_all.values())
    cands = [(t_ms, tag, name, n_l) for name, rep in per_kernel.items() for tag, (n_l, t_ms) in rep.items()
             if kernel_work(tag, per[name]["nb"], per[name]["selfenergy"], args.precision)[0] is not None]
    cands.sort(reverse=True)
    if not cands:
        cands = [(0.0, "none", next(iter(per)), 1)]
    t_ms, dom_tag, dom_wl, dom_n = cands[0]
    d_nb, d_se = per[dom_wl]["nb"], per[dom_wl]["selfenergy"]
    bound, work, issued = kernel_work(dom_tag, d_nb, d_se, args.precision)
    avg_s = t_ms * 1e-3 / dom_n
    if bound == "tensor":
        if args.precision == "bf16x4":
            peak = peaks["bf16_tflops_sustained"]
            src = f"{peak_kind} bf16 sustained (cuBLAS loop), of {peak_kind}"
        else:
            peak = peaks["bf16_tflops_sustained"] * TF32_OVER_BF16
            src = f"{peak_kind} bf16 sustained x TF32/BF16 nominal ratio (1.1/2.25), of {peak_kind}"
        achieved = work / avg_s / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "work": "algorithmic: 8 flop per complex MAC of the contraction the launch evaluates",
                "issued_achieved": issued / avg_s / 1e12, "issued_frac": issued / avg_s / 1e12 / peak,
                "issued_over_algorithmic": issued / work, "peak_source": src}
    elif bound == "hbm":
        peak = peaks["hbm_gbs"]
        achieved = work / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} copy bandwidth, of {peak_kind}"}
    else:
        fl = sum(p["flops_per_step"] * args.steps for p in per.values())
        zg = sum(v[1] for k, v in prof_all.items() if "zgemm" in k)
        achieved = fl / (zg * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": FP64_PEAK_NOTE + " (measured DFMA)"}
        dom_tag = "fp64_zgemm (+ split-K): every complex contraction"
    roof.update({"traffic": TRAFFIC.get((dom_tag, dom_wl)) if args.precision == "bf16x4" else None,
                 "tensor_pipe_active_pct": TENSOR_PIPE.get((dom_tag, dom_wl)) if args.precision == "bf16x4" else None,
                 "kernel": dom_tag, "workload": dom_wl,
                 "avg_launch_ms": avg_s * 1e3, "launches": dom_n, "share": t_ms / total_ms})

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else args.precision + "+f64",
        "data": "synthetic (seeded general basis: h Hermitian Gaussian, w = sum_P L^P x L^P, gauss-sine pulse)",
        "config": {"workload": "+".join(args.workloads), "precision": args.precision,
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (G2 state 1.36 GB at nb=96, 268 MB at nb=64)",
                   "parts": {k: {kk: vv for kk, vv in v.items()} for k, v in per.items()}},
        "e2e": {"value": e2e_value, "unit": "steps/s",
                "h2d_bytes_per_step": sum(p["h2d_bytes"] for p in per.values()) / args.steps,
                "d2h_bytes_per_step": sum(p["d2h_bytes_per_step"] for p in per.values()),
                "how": "g1g2_set_state from pinned host + g1g2_propagate(K, observables every step)"},
        "gpu_launches": launches_total,
        "fp64_form": ({"ms_per_step": sum(p["fp64_ms_per_step"] for p in per.values()),
                       "steps_per_s": 1e3 / sum(p["fp64_ms_per_step"] for p in per.values()),
                       "speedup_of_value": value / world / (1e3 / sum(p["fp64_ms_per_step"] for p in per.values())),
                       "vs_fp64_error": {k: p["vs_fp64"] for k, p in per.items()}}
                      if all("fp64_ms_per_step" in p for p in per.values()) else None),
        "roofline": roof,
        "clocks": clk,
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1][1])},
    }
    return line


def adjoint_sample(args):
    """Discrete adjoint on the 2D Hubbard cluster (4x4 sites, 32 spin-orbitals, 64 pulse
    controls, dt = 0.01): gradient of the final double occupancy with respect to the
    controls and U over the first `adjoint_steps` steps with checkpoints every 32 steps,
    timed against the FP64 forward propagation of the same steps, with a central
    finite-difference check (eps = 1e-5) of dJ/dU."""
    from paper_2002_12717_gb300.g1g2 import Propagator

    d = inputs.workload("hubbard-2d-4x4")
    steps, dt, k = args.adjoint_steps, d["dt"], 32
    M = len(d["drive"].values)

    def make(w):
        p = Propagator(d["h"], w, d["n0"], None, "SOA", "fp64")
        p.set_drive(d["D"], d["drive"])
        return p

    def forward(w):
        with make(w) as p:
            t0 = time.perf_counter()
            p.propagate(dt, steps)
            J = float(p.observables(double_occ=True)["double_occ"].mean())
            return J, time.perf_counter() - t0

    forward(d["w"])  # warm-up
    with make(d["w"]) as p:
        t0 = time.perf_counter()
        J, gd, gws, gh = p.adjoint(dt, steps, objective=0, ckpt_every=k, n_drive_params=M)
        t_adj = time.perf_counter() - t0
    J_f, t_fwd = forward(d["w"])
    eps = 1e-5
    fd = (forward(d["w"] * (1 + eps))[0] - forward(d["w"] * (1 - eps))[0]) / (2 * eps)
    U = 2.0
    return {"workload": f"hubbard-2d-4x4 (32 spin-orbitals, {M} controls), first {steps} of {d['nsteps']} steps",
            "objective": "mean double occupancy at the final time", "ckpt_every": k, "precision": "fp64",
            "ms_per_step": 1e3 * t_adj / steps, "forward_ms_per_step": 1e3 * t_fwd / steps,
            "adjoint_over_forward": t_adj / t_fwd, "J": J, "J_forward": J_f,
            "dJ_dU": gws / U, "fd_dJ_dU": fd / U, "rel_diff_dJ_dU": abs(gws - fd) / abs(fd),
            "grad_controls_norm": float(np.linalg.norm(gd))}


def adjoint_run(eps=1e-5):
    """The discrete adjoint over the whole 4x4 Hubbard workload (32 spin-orbitals, U = 2,
    64 piecewise-linear controls on [0, 10], 1000 steps of dt = 0.01, checkpoints every
    32 steps), FP64 form: the gradient of the final mean double occupancy with respect to
    the controls, the w scale (U dJ/dU), h and the entries of w, timed against the
    forward propagation, and checked by central differences (eps) on three controls, on
    U and on two perturbations of w with its symmetries (the on-site U of one site, and
    a random dense one)."""
    from paper_2002_12717_gb300.g1g2 import Propagator

    d = inputs.workload("hubbard-2d-4x4")
    steps, dt, k = d["nsteps"], d["dt"], 32
    M = len(d["drive"].values)
    nb = d["nb"]

    def J_of(w=None, controls=None):
        drv = d["drive"] if controls is None else inputs.PiecewiseLinear(controls, d["drive"].ta, d["drive"].tb)
        with Propagator(d["h"], d["w"] if w is None else w, d["n0"], None, "SOA", "fp64") as p:
            p.set_drive(d["D"], drv)
            t0 = time.perf_counter()
            p.propagate(dt, steps)
            J = float(p.observables(double_occ=True)["double_occ"].mean())
            return J, time.perf_counter() - t0

    J_of()  # warm-up
    J_f, t_fwd = J_of()
    with Propagator(d["h"], d["w"], d["n0"], None, "SOA", "fp64") as p:
        p.set_drive(d["D"], d["drive"])
        t0 = time.perf_counter()
        J, gd, gws, gh, gw = p.adjoint(dt, steps, objective=0, ckpt_every=k, n_drive_params=M, grad_w=True)
        t_adj = time.perf_counter() - t0
    rel = lambda a, b: abs(a - b) / max(abs(b), 1e-300)
    checks = {}
    vals = d["drive"].values
    for m in (5, 31, 50):
        vp, vm = vals.copy(), vals.copy()
        vp[m] += eps
        vm[m] -= eps
        fd = (J_of(controls=vp)[0] - J_of(controls=vm)[0]) / (2 * eps)
        checks[f"control_{m}"] = {"adjoint": float(gd[m]), "fd": fd, "rel_diff": rel(float(gd[m]), fd)}
    fd = (J_of(w=d["w"] * (1 + eps))[0] - J_of(w=d["w"] * (1 - eps))[0]) / (2 * eps)
    checks["wscale"] = {"adjoint": gws, "fd": fd, "rel_diff": rel(gws, fd)}
    E1 = np.zeros((nb,) * 4)
    for a in ((0, 1, 0, 1), (1, 0, 1, 0)):        # the on-site U of site 0 (spin-orbitals 0, 1)
        E1[a] = 1.0
    rng = np.random.default_rng(9)
    E2 = rng.standard_normal((nb,) * 4)
    E2 = E2 + E2.transpose(1, 0, 3, 2)
    E2 = 0.01 * (E2 + E2.transpose(2, 3, 0, 1)) / 4
    for name, E in (("w_onsite_site0", E1), ("w_random_symmetric", E2)):
        fd = (J_of(w=d["w"] + eps * E)[0] - J_of(w=d["w"] - eps * E)[0]) / (2 * eps)
        want = float((np.conj(gw) * E).real.sum())
        checks[name] = {"adjoint": want, "fd": fd, "rel_diff": rel(want, fd)}
    return {"workload": f"hubbard-2d-4x4 ({nb} spin-orbitals, U = 2, {M} controls, {steps} steps of dt = {dt})",
            "objective": "mean double occupancy at t = 10", "ckpt_every": k, "precision": "fp64",
            "J": J, "J_forward": J_f, "adjoint_s": t_adj, "forward_s": t_fwd, "adjoint_over_forward": t_adj / t_fwd,
            "grad_controls_norm": float(np.linalg.norm(gd)), "grad_w_norm": float(np.linalg.norm(gw)),
            "checks": checks, "max_rel_diff": max(c["rel_diff"] for c in checks.values())}


def hubbard_scaling(sizes, steps=3, selfenergy="SOA"):
    """ms per RK4 step of the spin-restricted Hubbard chain (J = 1, U = 2, half filling,
    quench) on the O(nb^4) Hubbard path and, for SOA, on the general O(nb^5) FP64 path
    (spin-restricted GW exists only in the Hubbard form)."""
    import torch

    from paper_2002_12717_gb300.g1g2 import from_workload

    out = []
    for nb in sizes:
        d = dict(inputs.hubbard_chain_restricted(L=nb, U=2.0), selfenergy=selfenergy)
        row = {"nb": nb, "selfenergy": selfenergy}
        for hub in ((True, False) if selfenergy == "SOA" else (True,)):
            with from_workload(d, precision="fp64") as p:
                p.hubbard_path = hub
                p.propagate(0.02, 2)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(steps):
                    p.step(0.02)
                e1.record()
                torch.cuda.synchronize()
                row["hubbard_ms" if hub else "general_ms"] = e0.elapsed_time(e1) / steps
        out.append(row)
    return out


def nt_scaling(nts, dt=0.02, L=8):
    """Wall time of the memory-integral HF-GKBA (Sec. III.B, O(N_t^2)) against the G1-G2
    equations (O(N_t)) for N_t time steps: spin-restricted Hubbard chain (J = 1, U = 1,
    half filling, quench), SOA, FP64 form.  The G1-G2 runs take RK4 steps, on the
    general O(nb^5) path and on the Hubbard O(nb^4) path.  Per-kernel time of
    the longest HF-GKBA run comes from the library's CUDA-event profile."""
    import torch

    from paper_2002_12717_gb300.g1g2 import from_workload

    d = inputs.hubbard_chain_restricted(L=L, U=1.0)
    nb = d["nb"]
    rows, prof = [], None
    for nt in nts:
        row = {"N_t": nt}
        with from_workload(d) as p:
            p.propagate_hfgkba(dt, 2)                     # warm-up (kernels loaded)
        with from_workload(d) as p:
            last = nt == max(nts)
            if last:
                p.profile(True)
            t0 = time.perf_counter()
            p.propagate_hfgkba(dt, nt)
            row["hfgkba_s"] = time.perf_counter() - t0
            if last:
                prof = p.profile_report()
        for hub in (False, True):
            with from_workload(d) as p:
                p.hubbard_path = hub
                p.propagate(dt, 2)
                p.set_state(0.0, d["n0"], None)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                p.propagate(dt, nt)
                torch.cuda.synchronize()
                row["g1g2_hubbard_s" if hub else "g1g2_general_s"] = time.perf_counter() - t0
        rows.append(row)
    ntm = max(nts)
    points = ntm * (ntm - 1) + 4 * ntm                    # history points summed over all evaluations
    rot = prof.get("hfgkba_mode_rotate", (0, 0.0))
    flops = 4 * 8 * nb ** 5 * points                      # four mode products of nb^5 complex MACs each
    summary = {"workload": f"hubbard-chain-restricted-nb{nb}", "dt": dt,
               "kernels_at_max_N_t": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items()},
               "mode_rotate_gflops": round(flops / (rot[1] * 1e-3) / 1e9, 1) if rot[1] else None}
    if len(rows) >= 2:
        a, b = rows[-2], rows[-1]
        for key in ("hfgkba_s", "g1g2_general_s", "g1g2_hubbard_s"):
            summary["exponent_" + key[:-2]] = round(float(np.log(b[key] / a[key]) / np.log(b["N_t"] / a["N_t"])), 2)
    return rows, summary


# complex multiply-adds per right-hand side of the FP64 form, by selfenergy: commutator
# 4 nb^5, source 4 nb^5, collision nb^5; GW quasi-Hamiltonian 2 nb^5 and polarisation
# nb^6; each T-matrix quasi-Hamiltonian 4 nb^5 and ladder product nb^6
FP64_CMAC = {
    "SOA": lambda n: 9 * n ** 5,
    "GW": lambda n: 11 * n ** 5 + n ** 6,
    "GWX": lambda n: 11 * n ** 5 + n ** 6,
    "TPP": lambda n: 13 * n ** 5 + n ** 6,
    "TPH": lambda n: 13 * n ** 5 + n ** 6,
    "DSL": lambda n: 19 * n ** 5 + 3 * n ** 6,
}


def factorised_compare(sizes, steps=3, selfenergies=("SOA", "GWX")):
    """ms per RK4 step of the FP64 form on the seeded general basis (rank 2 nb, nb/2 occupied,
    gauss-sine pulse) with w given as the nb^4 tensor and as its 2 nb factors (the factorised
    source term), and the largest difference of the two states after the timed steps."""
    import torch

    from paper_2002_12717_gb300.g1g2 import Propagator

    out = []
    for nb, se in ((nb, se) for nb in sizes for se in selfenergies):
        d = inputs.general_basis(nb, 2 * nb, nb // 2, seed=nb, selfenergy=se, pulse=True)
        row, states = {"nb": nb, "selfenergy": se, "nfac": 2 * nb}, []
        for key in ("w", "factors"):
            kw = {"factors": d["factors"]} if key == "factors" else {}
            with Propagator(d["h"], d["w"] if key == "w" else None, d["n0"], None, se, "fp64", **kw) as p:
                p.set_drive(d["D"], d["drive"])
                p.step(0.01)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(steps):
                    p.step(0.01)
                e1.record()
                torch.cuda.synchronize()
                row[f"{key}_ms"] = round(e0.elapsed_time(e1) / steps, 3)
                states.append(p.get_state()[1:])
        row["max_dG1"] = float(np.abs(states[0][0] - states[1][0]).max())
        row["max_dG2"] = float(np.abs(states[0][1] - states[1][1]).max())
        out.append(row)
    return out


def selfenergy_sweep(sizes, precisions=("fp64",), steps=2):
    """ms per RK4 step of every selfenergy on the seeded general basis (rank 2 nb, nb/2
    occupied, gauss-sine pulse).  FP64 form: the algorithmic FLOP rate against the
    measured DFMA rate; BF16-slice form: the rate of its nb^2 x nb^2 x nb^2 products
    (polarisation, ladder), algorithmic and in issued slice products, against the measured
    sustained BF16 rate."""
    import torch

    from paper_2002_12717_gb300.g1g2 import from_workload

    peaks, _ = load_peaks()
    out = []
    for prec, nb, se in ((pr, nb, se) for pr in precisions for nb in sizes
                         for se in ("SOA", "GW", "GWX", "TPP", "TPH", "DSL")):
        d = inputs.general_basis(nb, 2 * nb, nb // 2, seed=nb, selfenergy=se, pulse=True)
        with from_workload(d, precision=prec) as p:
            p.step(0.01)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                p.step(0.01)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            p.profile(True)
            p.step(0.01)
            prof = p.profile_report()
            p.profile(False)
        tot = sum(v[1] for v in prof.values())
        top = max(prof.items(), key=lambda kv: kv[1][1])
        row = {"precision": prec, "nb": nb, "selfenergy": se, "ms_per_step": round(ms, 3),
               "top_kernel": top[0], "top_share": round(top[1][1] / tot, 3)}
        if prec == "fp64":
            tflops = 4 * 8 * FP64_CMAC[se](nb) / (ms * 1e-3) / 1e12
            row.update(algorithmic_tflops=round(tflops, 4), frac_of_dfma=round(tflops / FP64_PEAK_TFLOPS, 3))
        else:
            for tag in ("tc_gemm_pi", "tc_gemm_ladder"):
                if tag in prof:
                    launches, tms = prof[tag]
                    _, work, issued = kernel_work(tag, nb, se, prec)
                    tf = work * launches / (tms * 1e-3) / 1e12
                    tfi = issued * launches / (tms * 1e-3) / 1e12
                    row[tag] = {"ms_per_launch": round(tms / launches, 3), "algorithmic_tflops": round(tf, 1),
                                "frac_of_bf16_sustained": round(tf / peaks["bf16_tflops_sustained"], 3),
                                "issued_tflops": round(tfi, 1),
                                "issued_frac_of_bf16_sustained": round(tfi / peaks["bf16_tflops_sustained"], 3)}
        out.append(row)
    return out


def oracle_rhs_seconds(names):
    """Wall seconds of one oracle right-hand side of each named workload (the oracle as it
    stands, on whatever BLAS threads the process has)."""
    from oracle import g1g2_oracle as O

    times = {}
    for name in names:
        d = inputs.workload(name)
        prob = O.Problem(d["h"], d["w"], d["selfenergy"], d["restricted"], d["D"], d["drive"].f)
        g0 = np.zeros((d["nb"],) * 4, dtype=np.complex128)
        t0 = time.perf_counter()
        O.rhs(prob, 0.0, d["n0"], g0)
        times[name] = time.perf_counter() - t0
    return times


SINGLE_THREAD_ENV = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                      "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS")}


def oracle_rhs_seconds_single_thread(names, timeout=300):
    """oracle_rhs_seconds in a child process whose BLAS runs one thread (the thread
    count of numpy's BLAS is fixed when it loads, hence the separate process)."""
    env = dict(os.environ, **SINGLE_THREAD_ENV)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rhs-times", ",".join(names)],
                       env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(args):
    """The CPU oracle as it stands (a bounded sample): one right-hand side of each workload
    on all host cores, and one right-hand side of the GW workload on one thread."""
    times = oracle_rhs_seconds(args.workloads)
    step_s = 4 * sum(times.values())   # an RK4 step is four right-hand sides
    out = {"value": 1.0 / step_s, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "one right-hand side per workload on all cores (" +
                     ", ".join(f"{k}: {v:.1f} s" for k, v in times.items()) + "); RK4 step = 4 x the sum"}
    one = [w for w in args.workloads if "gw" in w][:1] or args.workloads[:1]
    try:
        st = oracle_rhs_seconds_single_thread(one)
        out["single_thread"] = {"cores": 1, "rhs_s": st, "all_cores_rhs_s": {k: times[k] for k in st},
                                "all_core_speedup": {k: st[k] / times[k] for k in st},
                                "sample": "one right-hand side of " + ", ".join(st) + " with BLAS on one thread"}
    except (RuntimeError, subprocess.TimeoutExpired, ValueError) as e:
        out["single_thread"] = {"unavailable": str(e)[-200:]}
    return out


def run_reference(args):
    """--impl reference: the CPU oracle, as it stands, on the host cores.

    Each timed step is a bounded sample: one oracle right-hand side, alternating
    between the workloads, so ms_per_step is the measured wall time of one such
    sample.  value converts to the metric's unit: one bench step (one RK4 step of
    each workload) is four right-hand sides of each workload.
    """
    from oracle import g1g2_oracle as O

    probs = []
    for name in args.workloads:
        d = inputs.workload(name)
        probs.append((name, O.Problem(d["h"], d["w"], d["selfenergy"], d["restricted"], d["D"], d["drive"].f),
                      d["n0"], np.zeros((d["nb"],) * 4, dtype=np.complex128)))
    times = {name: [] for name, *_ in probs}
    warm = min(args.warmup, 1)   # the oracle has no caches to warm; one untimed call
    samples = []
    for i in range(warm + args.steps):
        name, prob, n0, g0 = probs[i % len(probs)]
        t0 = time.perf_counter()
        O.rhs(prob, 0.0, n0, g0)
        if i >= warm:
            dt = time.perf_counter() - t0
            times[name].append(dt)
            samples.append(dt)
    for name, *_ in probs:
        if not times[name]:   # K too small to visit every workload: time one call
            _, prob, n0, g0 = next(p for p in probs if p[0] == name)
            t0 = time.perf_counter()
            O.rhs(prob, 0.0, n0, g0)
            times[name].append(time.perf_counter() - t0)
    bench_step_s = 4 * sum(statistics.mean(v) for v in times.values())
    value = 1.0 / bench_step_s
    sample = ("per timed step one oracle right-hand side, alternating " + " / ".join(times) +
              "; one bench step = 4 right-hand sides of each workload = " +
              " + ".join(f"4 x {statistics.mean(v):.2f} s" for v in times.values()))
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": warm, "ms_per_step": 1e3 * statistics.mean(samples) if samples else None,
        "step": "one oracle right-hand side (a bounded sample); value converts it to RK4 bench steps",
        "ms_per_bench_step": 1e3 * bench_step_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "+".join(args.workloads), "precision": "fp64-oracle"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def accuracy_run(names, every, out_path, max_steps=0):
    """Accuracy over whole runs: each named workload propagated for its full
    length (or its first max_steps steps) in the BF16-slice tensor-core form and in the FP64 GPU form from the same
    initial state, recorded every `every` steps: max|dG1| and max|dG2| between the two,
    each form's energy drift |E(t) - E(0) - W(t)| / |E(0)| (W the drive work), and the
    relative energy difference between the forms.  One JSON line per record, appended to
    out_path as it is taken."""
    import torch

    from paper_2002_12717_gb300.g1g2 import from_workload

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    summary = []
    for name in names:
        d = inputs.workload(name)
        dt, nsteps = d["dt"], d["nsteps"]
        if max_steps > 0:
            nsteps = min(nsteps, max_steps)
        forms = {"bf16x4": from_workload(d, precision="bf16x4"), "fp64": from_workload(d, precision="fp64")}
        o0 = {k: p.observables() for k, p in forms.items()}
        secs = {k: 0.0 for k in forms}
        worst = {"max_abs_dG1": 0.0, "max_abs_dG2": 0.0, "rel_dE": 0.0}
        step = 0
        while step < nsteps:
            m = min(every, nsteps - step)
            for k, p in forms.items():
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                p.propagate(dt, m)
                torch.cuda.synchronize()
                secs[k] += time.perf_counter() - t0
            step += m
            st = {k: p.get_state() for k, p in forms.items()}
            ob = {k: p.observables() for k, p in forms.items()}
            (_, n_m, g_m), (_, n_r, g_r) = st["bf16x4"], st["fp64"]
            e0 = abs(o0["fp64"]["e_total"])
            row = {"workload": name, "step": step, "t": ob["fp64"]["t"],
                   "max_abs_dG1": float(np.abs(n_m - n_r).max()),
                   "max_abs_dG2": float(np.abs(g_m - g_r).max()), "max_abs_G2": float(np.abs(g_r).max()),
                   "rel_dE": abs(ob["bf16x4"]["e_total"] - ob["fp64"]["e_total"]) / e0,
                   "drift": {k: abs(ob[k]["e_total"] - o0[k]["e_total"] - ob[k]["pulse_work"]) / abs(o0[k]["e_total"])
                             for k in forms},
                   "pulse_work": ob["fp64"]["pulse_work"], "seconds": dict(secs)}
            del st, g_m, g_r
            for key in worst:
                worst[key] = max(worst[key], row[key])
            with open(out_path, "a") as f:
                f.write(json.dumps(row) + "\n")
            print(json.dumps(row), flush=True)
        for p in forms.values():
            p.close()
        summary.append({"workload": name, "steps": nsteps, "dt": dt, "record_every": every, **worst,
                        "final_drift": row["drift"], "ms_per_step": {k: 1e3 * v / nsteps for k, v in secs.items()},
                        "speedup": secs["fp64"] / secs["bf16x4"],
                        "meets_target": worst["max_abs_dG1"] <= 1e-6 and worst["rel_dE"] <= 1e-7})
        torch.cuda.empty_cache()
    return summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp64", "tf32x3", "bf16x4"])
    ap.add_argument("--workloads", default=",".join(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-steps", type=int, default=3,
                    help="steps run in both forms from the initial state (speed-up and error vs FP64)")
    ap.add_argument("--hubbard-scaling", default="",
                    help="comma-separated nb: time the Hubbard O(nb^4) path against the general path and exit")
    ap.add_argument("--hubbard-selfenergy", default="SOA", choices=["SOA", "GW"],
                    help="selfenergy of --hubbard-scaling")
    ap.add_argument("--nt-scaling", default="",
                    help="comma-separated N_t: time the memory-integral HF-GKBA against the G1-G2 equations and exit")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="measure the FP64 FMA rate of the GPU (the FP64 roofline) and exit")
    ap.add_argument("--selfenergy-sweep", default="",
                    help="comma-separated nb: time every selfenergy and exit (forms: --sweep-precisions)")
    ap.add_argument("--sweep-precisions", default="fp64", help="comma-separated forms of --selfenergy-sweep")
    ap.add_argument("--factorised-compare", default="",
                    help="comma-separated nb: time the FP64 form with w as a tensor and as its factors, and exit")
    ap.add_argument("--accuracy-run", default="",
                    help="comma-separated workloads: propagate each for its full length in the BF16-slice and "
                         "FP64 forms side by side, record the differences and energy drifts, and exit")
    ap.add_argument("--accuracy-every", type=int, default=50, help="record interval of --accuracy-run")
    ap.add_argument("--accuracy-steps", type=int, default=0,
                    help="--accuracy-run: stop after this many steps (0: the workload's full length)")
    ap.add_argument("--accuracy-out", default="accuracy.jsonl", help="JSON-lines file of --accuracy-run")
    ap.add_argument("--oracle-rhs-times", default="", help=argparse.SUPPRESS)
    ap.add_argument("--adjoint-run", action="store_true",
                    help="the discrete adjoint over the whole 4x4 Hubbard workload with finite-difference checks, "
                         "and exit")
    ap.add_argument("--adjoint-steps", type=int, default=100,
                    help="steps of the discrete-adjoint sample on the 4x4 Hubbard cluster (0: skip)")
    args = ap.parse_args()
    args.workloads = args.workloads.split(",")
    if args.precision is None:
        args.precision = os.environ.get("G1G2_BENCH_PRECISION", "bf16x4")
    if args.steps is None:
        args.steps = 3 if args.precision == "fp64" else 20
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.oracle_rhs_times:
        print(json.dumps(oracle_rhs_seconds(args.oracle_rhs_times.split(","))), flush=True)
        return
    if args.adjoint_run:
        if rank == 0:
            print(json.dumps({"adjoint_run": adjoint_run()}), flush=True)
        return
    if args.accuracy_run:
        if rank == 0:
            os.makedirs(os.path.dirname(os.path.abspath(args.accuracy_out)), exist_ok=True)
            summary = accuracy_run(args.accuracy_run.split(","), args.accuracy_every, args.accuracy_out,
                                   args.accuracy_steps)
            print(json.dumps({"accuracy_run": summary}), flush=True)
        return
    if args.hubbard_scaling:
        if rank == 0:
            sizes = [int(x) for x in args.hubbard_scaling.split(",")]
            print(json.dumps({"hubbard_scaling": hubbard_scaling(sizes, selfenergy=args.hubbard_selfenergy)}),
                  flush=True)
        return
    if args.fp64_peak:
        if rank == 0:
            from paper_2002_12717_gb300.g1g2 import fp64_rate
            sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
            sampler.start()
            rate = fp64_rate()
            print(json.dumps({"fp64_fma_tflops": round(rate, 4), "clocks": sampler.stop()}), flush=True)
        return
    if args.selfenergy_sweep:
        if rank == 0:
            sweep = selfenergy_sweep([int(x) for x in args.selfenergy_sweep.split(",")],
                                     args.sweep_precisions.split(","))
            print(json.dumps({"selfenergy_sweep": sweep}), flush=True)
        return
    if args.factorised_compare:
        if rank == 0:
            rows = factorised_compare([int(x) for x in args.factorised_compare.split(",")])
            print(json.dumps({"factorised_compare": rows}), flush=True)
        return
    if args.nt_scaling:
        if rank == 0:
            rows, summary = nt_scaling([int(x) for x in args.nt_scaling.split(",")])
            print(json.dumps({"nt_scaling": rows, "summary": summary}), flush=True)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)), flush=True)
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        if args.adjoint_steps > 0:
            line["adjoint"] = adjoint_sample(args)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
