"""Throughput of the GB300 DG Euler time step (DOF-updates/s), one JSON line.

Workload (the ~200k-element p=3 ball): the Kuhn lattice n=32 on [-1,1]^3
mapped onto the unit ball (196,608 tetrahedra, jittered interior vertices,
seed 0), order p=3 (20 nodes per element, 1.97e7 DOF), SI air at rest with a
10% p0 Gaussian pressure pulse of width 0.15 at the centre, characteristic
pass-through boundary on the sphere, CFL 0.5 time step. One step = one full
five-stage low-storage RK4 time step of the whole mesh.

  value      device-resident state, K steps timed with CUDA events on the
             solver's stream; max over ranks; DOF-updates/s = 5 Np K_elem steps / s
  e2e        same metric through the C ABI with host buffers: dg_set_state
             from pinned host memory, dg_step, sensor read-back and
             dg_get_state to host, all inside the timed region (wall clock)
  roofline   stage kernel of the headline form: algorithmic flops (float32
             and float64 forms, ALU bound) or bytes (tensor-core form, HBM
             bound) per launch / average launch time (CUDA event pairs around
             every stage launch on the solver's stream)
  forms      every arithmetic form (float32 perturbation, its tensor-core
             variant, float64, the paper's modal form, and the one-pass
             tensor-core variant) timed the same way, with the float32 forms'
             error against float64 after the timed steps
  learned_bc the learned boundary closure: traces recorded, network trained
             and reflected energies measured on the GPU, and the closure timed on
             the bench workload
  paper_configuration  p = 1 with RK2 on the bench mesh (the paper's own setting)
             in the paper's discretisation and the nodal forms, with device
             memory per element
  order4     both float32 forms at p = 4 (the production configuration's order)
             on the bench mesh, timed the same way
  locality   the float32 form on the bench mesh in lattice, Morton and random
             element order (how far tiles' gathers reach)
  horn       the horn-in-room workload (1,489,704 tets, p=3: a flared horn with
             slip walls, the inflow pulse at its mouthpiece, a pass-through
             room in front of the bell), both float32 forms timed the same way
  cpu_baseline  the float64 CPU oracle on a bounded sample of the workload

``--impl reference`` times the CPU oracle itself on that sample instead.
Multi-GPU (torchrun): independent replicas, one per GPU (the method has no
data exchange on one mesh); value = all ranks' DOF-updates / max time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "DOF-updates/s (p=3 3D Euler DG, 1 GB300); mixed/learned-BC vs FP64 at error"
UNIT = "DOF-updates/s"
WORKLOAD = dict(n=32, radius=1.0, jitter=0.1, seed=0, order=3, amplitude=0.1, width=0.15, cfl=0.5)
WORKLOAD_NAME = ("ball r=1: Kuhn lattice n=32 radially mapped, 196608 tets (Morton order), jitter "
                 "0.1h seed 0; p=3 nodal DG (Np=20); SI air, 10% p0 Gaussian pulse w=0.15; "
                 "characteristic BC")
# CPU sample: the elements of the same mesh whose centroid lies within this radius
CPU_SAMPLE_RADIUS = 0.25


def stage_flops_per_element(p):
    """Algorithmic float64 flops of one stage per element (1 FMA = 2 flops).

    node:      Euler flux + metric fold (103) + RK update (25)   per node
    volume:    3 derivative matrices x 5 variables x Np^2 FMAs
    face node: two normal fluxes + wave speeds, LLF, jump (101)   per face node
    lift:      5 variables x Np x 4 Nfp FMAs
    """
    Np = (p + 1) * (p + 2) * (p + 3) // 6
    Nfp = (p + 1) * (p + 2) // 2
    return Np * (103 + 25) + 30 * Np * Np + 4 * Nfp * 101 + 40 * Np * Nfp


def modal_stage_flops_per_element(p):
    """Algorithmic float64 flops of one stage of the paper's discretisation
    (Gauss rules of degree 2p and 2p+1: Nq = (p+1)^3 volume and Nfq = (p+1)^2
    points per face) per element (1 FMA = 2 flops).

    volume point: state from the nodes (5 x Np FMAs), Euler flux + metric fold (103)
    volume sums:  3 directions x 5 variables x Np x Nq FMAs
    face point:   own and neighbour trace (2 x 5 x Nfp FMAs), LLF (101),
                  surface sum (5 x Np FMAs)
    node:         RK update (25)
    """
    Np = (p + 1) * (p + 2) * (p + 3) // 6
    Nfp = (p + 1) * (p + 2) // 2
    Nq, Nfq = (p + 1) ** 3, (p + 1) ** 2
    return Nq * (10 * Np + 103) + 30 * Np * Nq + 4 * Nfq * (20 * Nfp + 101 + 10 * Np) + 25 * Np


def fp64_peak_gflops(sm_mhz=2070.0):
    """Nominal GB300 float64 rate: 1.25 TFLOP/s at the 2070 MHz boost clock over
    152 SMs, i.e. 4 flops per SM per clock; scaled to the given clock."""
    return 152 * 4 * sm_mhz * 1e-3


def fp32_peak_tflops(sm_mhz=2070.0):
    """GB300 float32 FMA rate: 152 SMs x 128 lanes x 2 flop per clock."""
    return 152 * 128 * 2 * sm_mhz * 1e-6


def profiled_traffic(summary, source):
    """DRAM bytes per full-size launch from an ncu summary under profiles/, or
    None when the kernel source changed after the counters were taken."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        src = open(os.path.join(ROOT, "paper_1710_03887_gb300", "csrc", source), "rb").read()
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("source_sha256_16:", "bytes_per_launch_full:")))
    if fields.get("source_sha256_16", "").strip() != hashlib.sha256(src).hexdigest()[:16]:
        return None
    try:
        return float(fields["bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index          # < 0: do not sample
        self.proc = None
        self.lines = []
        self.skip = 0

    def __enter__(self):
        if self.index < 0:
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once the sampler runs; its first lines
            # (before the region) are kept apart
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.skip = len(self.lines)
        except OSError:
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

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.skip:]
        before = 0
        if not lines and self.skip:
            # a region shorter than the polling interval: the last sample
            # before it stands in, and the record says so
            lines, before = self.lines[self.skip - 1:self.skip], 1
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
               "reasons": sorted(reasons), "samples": len(sm), "interval_ms": 50}
        if before:
            out["note"] = "no sample fell inside the timed region; the last one before it"
        return out


def build_workload():
    """The bench ball with its elements in Morton order of their centroids
    (consecutive elements close in space, as the stage kernels' tiles want)."""
    from paper_1710_03887_gb300 import workloads as W
    w = WORKLOAD
    xyz, EToV = W.ball(w["n"], w["radius"], jitter=w["jitter"], seed=w["seed"])
    return xyz, EToV[W.morton_order(xyz, EToV)]


def cpu_sample_run(steps, warmup, xyz, EToV):
    """Time the float64 CPU oracle on the sample of the workload; DOF-updates/s."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.euler_dg import Gas, Solver
    from oracle.geometry import Geometry
    from oracle.reference_element import ReferenceElement
    from paper_1710_03887_gb300 import workloads as W
    w = WORKLOAD
    cen = W.element_centroids(xyz, EToV)
    keep = np.linalg.norm(cen, axis=1) < CPU_SAMPLE_RADIUS
    sx, sE = W.submesh(xyz, EToV, keep)
    ref = ReferenceElement(w["order"])
    geom = Geometry(ref, sx, sE)
    gas = Gas(W.GAMMA, W.RHO0_SI, W.P0_SI)
    S = Solver(geom, gas)
    q = W.gaussian_pulse_state(geom.x, W.GAMMA, W.RHO0_SI, W.P0_SI, w["amplitude"], w["width"])
    dt = S.stable_dt(q, w["cfl"])
    res = np.zeros_like(q)
    led = (np.zeros(5), np.zeros(5))
    t = 0.0
    for _ in range(warmup):
        q, t, res, led = S.step(q, t, dt, res, led)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        q, t, res, led = S.step(q, t, dt, res, led)
        times.append(time.perf_counter() - t0)
    dof = 5 * ref.Np * geom.K
    total = sum(times)
    sample = (f"{geom.K} elements of the workload mesh (centroid radius < {CPU_SAMPLE_RADIUS}), "
              f"p=3, {steps} full RK4 steps, numpy float64 oracle")
    return dof * steps / total, sample, geom.K


def reduce_max(x, dist, device):
    """Max of a scalar over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, dof_per_rank, steps, seconds):
    """Whole-job DOF-updates/s: every replica advanced dof_per_rank DOF by steps."""
    return world * dof_per_rank * steps / seconds


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    workload: every number is what was measured on that sample (nothing is
    scaled to the full mesh)."""
    if rank != 0:
        return
    xyz, EToV = build_workload()
    value, sample, K = cpu_sample_run(args.steps, args.warmup, xyz, EToV)
    Np = (WORKLOAD["order"] + 1) * (WORKLOAD["order"] + 2) * (WORKLOAD["order"] + 3) // 6
    dof_sample = 5 * Np * K
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dof_sample / value,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "sample of: " + WORKLOAD_NAME, "sample": sample, "elements": K,
                   "dof": dof_sample,
                   "ms_per_step": "measured on the sample (the oracle's time per step of its elements)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def timed_repeats(args, S, q0_dev, dt, dev, stream, dist, sample_clocks, repeats):
    """``repeats`` timed regions of ``args.steps`` steps, each from the same
    initial state, with CUDA events on the solver's stream (synchronised and,
    under torchrun, barriered on both sides; max over ranks). Per-launch
    stage timing is on for all of them and the clock sampler runs across
    all of them. Returns (ms per region list, summed stage-kernel ms, stage
    launches, sampler)."""
    import torch
    S.set_kernel_timing(True)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")) if sample_clocks else -1)
    reps = []
    target = repeats if repeats > 0 else 5
    with clk:
        while len(reps) < target:
            S.set_state(q0_dev)
            if dist:
                dist.barrier()
            torch.cuda.synchronize(dev)
            start.record(stream)
            S.step(args.steps, dt)
            stop.record(stream)
            torch.cuda.synchronize(dev)
            if dist:
                dist.barrier()
            reps.append(reduce_max(start.elapsed_time(stop), dist, dev))
            if repeats <= 0 and len(reps) == 1:
                # automatic count: at least 5 regions, and enough of them for
                # the regions to span ~0.5 s (ten clock samples at 50 ms)
                target = int(min(200, max(5, np.ceil(500.0 / max(reps[0], 1e-3)))))
    kms, klaunch = S.read_kernel_timing()
    S.set_kernel_timing(False)
    S.read_probes()
    return reps, kms, klaunch, clk


def repeat_stats(reps, steps, sm_mhz=None):
    """Median, spread and per-step times of the repeated timed regions."""
    med = statistics.median(reps)
    out = {"n": len(reps), "ms_per_step": [r / steps for r in reps],
           "median_ms_per_step": med / steps, "min_ms_per_step": min(reps) / steps,
           "max_ms_per_step": max(reps) / steps,
           "spread_rel": (max(reps) - min(reps)) / med}
    if sm_mhz:
        # clock-normalised time: a run at a lower clock shows a larger
        # product only if it was slowed by more than the clock
        out["median_ms_per_step_x_sm_mhz"] = med / steps * sm_mhz
    return out


def measure_form(args, precision, xyz, EToV, dev, stream, dist, world, sample_clocks, mlp=None,
                 order=None):
    """Time one arithmetic form on the bench workload; returns a dict. With
    ``mlp`` = (weights, radius) the sphere takes the learned closure;
    ``order`` replaces the workload's polynomial order."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    w = WORKLOAD
    prec = {"f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC, "fp64": B.DG_PREC_FP64,
            "modal": B.DG_PREC_MODAL, "f32_tc1": B.DG_PREC_F32_TC1}[precision]
    S = B.Solver(order or w["order"], W.GAMMA, W.RHO0_SI, W.P0_SI, precision=prec)
    S.set_stream(stream.cuda_stream)
    S.upload_mesh(xyz, EToV)
    if mlp is not None:
        S.set_bc(0, B.DG_BC_LEARNED)
        S.set_bc_mlp(*mlp)
    nodes = S.node_coords()
    q0 = W.gaussian_pulse_state(nodes, W.GAMMA, W.RHO0_SI, W.P0_SI, w["amplitude"], w["width"])
    dt = S.stable_dt(q0, w["cfl"])
    dof = 5 * S.Np * S.K
    probes = np.array([[0.5 * np.cos(a), 0.5 * np.sin(a), 0.1] for a in np.linspace(0, 6, 32)])
    S.set_probes(probes, capacity=max(args.steps, 1))
    q0_dev = torch.from_numpy(q0).to(dev)
    # device-resident timing
    S.set_state(q0_dev)
    S.step(args.warmup, dt)
    torch.cuda.synchronize(dev)
    S.read_probes()
    reps, kms, klaunch, clk = timed_repeats(args, S, q0_dev, dt, dev, stream, dist,
                                            sample_clocks, args.repeats)
    ms = statistics.median(reps)
    S.sync()
    q_end = torch.empty_like(q0_dev)
    S.get_state(q_end)
    # end to end through the C ABI with host buffers (median of three runs)
    q0_host = torch.from_numpy(q0).pin_memory()
    q_out = torch.empty_like(q0_host).pin_memory()
    nprobe = probes.shape[0]
    psamples = np.zeros((args.steps, nprobe, 5))
    e2e_runs = []
    for _ in range(3):
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        S.set_state(q0_host)
        S.step(args.steps, dt)
        S.read_probes(args.steps, out=psamples)
        S.get_state(q_out)
        e2e_runs.append(reduce_max(time.perf_counter() - t0, dist, dev))
    e2e_s = statistics.median(e2e_runs)
    S.close()
    return dict(precision=precision, ms=ms, reps=reps, kms=kms, klaunch=klaunch, dof=dof,
                K=len(EToV), dt=dt, q0=q0, q_end=q_end.cpu().numpy(), e2e_s=e2e_s, nprobe=nprobe,
                clocks=clk.summary() if sample_clocks else None,
                value=aggregate_value(world, dof, args.steps, ms * 1e-3),
                e2e=aggregate_value(world, dof, args.steps, e2e_s))


def measure_partitioned(args, xyz, EToV, dev, stream, dist, world, rank):
    """The bench workload split across the ranks (Morton slabs; the face
    traces of cut faces exchanged before every stage over NCCL), timed like
    measure_form: ``repeats`` regions of ``steps`` steps, max over ranks.
    value = DOF of the whole mesh x steps / time (strong scaling)."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import partition as PT
    from paper_1710_03887_gb300 import workloads as W
    w = WORKLOAD
    prec = {"f32": B.DG_PREC_F32, "f32_tc": B.DG_PREC_F32_TC, "fp64": B.DG_PREC_FP64}[args.precision]
    part = PT.partition_elements(xyz, EToV, world)
    L = PT.local_mesh(xyz, EToV, part, rank)
    PS = PT.PartitionedSolver(w["order"], L, W.GAMMA, W.RHO0_SI, W.P0_SI, prec, dev)
    S = PS.S
    q0 = W.gaussian_pulse_state(S.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, w["amplitude"],
                                w["width"])
    dt = reduce_max(-S.stable_dt(q0, w["cfl"]), dist, dev) * -1.0      # the smallest over ranks
    q0_dev = torch.from_numpy(q0).to(dev)
    PS.set_state(q0_dev)
    PS.step(args.warmup, dt)
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    reps = []
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    with clk:
        for _ in range(max(args.repeats, 5)):
            PS.set_state(q0_dev)
            dist.barrier()
            torch.cuda.synchronize(dev)
            start.record(stream)
            PS.step(args.steps, dt)
            stop.record(stream)
            torch.cuda.synchronize(dev)
            dist.barrier()
            reps.append(reduce_max(start.elapsed_time(stop), dist, dev))
    ms = statistics.median(reps)
    dof_total = 5 * S.Np * len(EToV)
    out = dict(ms=ms, reps=reps, value=dof_total * args.steps / (ms * 1e-3), dof=dof_total,
               K=len(EToV), K_own=L.K_own, cut_faces=int(L.send_elem.size), dt=dt,
               clocks=clk.summary(), peers=L.peers)
    S.close()
    return out


def roofline_for(m, order):
    """Roofline object of the stage kernel of one measured form."""
    K = m["K"]
    avg_launch_s = (m["kms"] * 1e-3) / max(m["klaunch"], 1)
    if m["precision"] == "modal":
        achieved = modal_stage_flops_per_element(order) * K / avg_launch_s * 1e-12
        peak = fp64_peak_gflops(2070.0) * 1e-3
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic("stage_modal_p3_ball.md", "stage_modal.cu"),
                "traffic_note": "ncu capture of a first (a = 0) stage: no residual read",
                "kernel": "stage_modal_kernel<3>",
                "note": ("the paper's discretisation (Gauss rules of degree 2p, 2p+1; two Heun "
                         "stages per step); algorithmic float64 flops per stage; float64 pipe "
                         "peak as for the float64 nodal form"),
                "avg_launch_ms": avg_launch_s * 1e3, "launches": m["klaunch"]}
    if m["precision"] == "fp64":
        achieved = stage_flops_per_element(order) * K / avg_launch_s * 1e-12
        peak = fp64_peak_gflops(2070.0) * 1e-3
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic("stage_fp64_p3_ball.md", "stage_fp64.cu"),
                "kernel": "stage_fp64_kernel<3>",
                "note": ("float64 pipe; peak = nominal 1.25 TFLOP/s = 152 SMs x 4 flop/clk x "
                         "2070 MHz (recipe; ncu peak_sustained DFMA = 2/SM/clk)"),
                "avg_launch_ms": avg_launch_s * 1e3, "launches": m["klaunch"]}
    peaks = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "of measured (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks else "of fallback"
    bytes_per_elem = stage_bytes_per_element(order, 4)
    hbm_achieved = bytes_per_elem * K / avg_launch_s * 1e-9
    flops = stage_flops_per_element(order) * K / avg_launch_s * 1e-12
    if m["precision"] == "f32":
        # 26,600 flop / 1,744 B = 15 flop/B at p=3, above the float32 ridge
        # (80.5 TFLOP/s / 6.78 TB/s = 12 flop/B): bound by the float32 ALUs
        peak = fp32_peak_tflops(2070.0)
        return {"bound": "alu", "achieved": flops, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / peak,
                "traffic": profiled_traffic("stage_f32_p3_ball.md", "stage_f32.cu"),
                "kernel": "stage_f32_kernel<3>",
                "note": ("algorithmic float32 flops per stage (1 FMA = 2); peak = 152 SMs x 128 "
                         "FMA lanes x 2 flop x 2070 MHz (recipe's unit counts and clock)"),
                "hbm": {"achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                        "frac": hbm_achieved / hbm, "peak_source": hbm_src},
                "avg_launch_ms": avg_launch_s * 1e3, "launches": m["klaunch"]}
    # tensor-core form: the contractions leave the ALUs; the rest (6.6 kflop /
    # 1,744 B per element) is below the ridge: bound by HBM
    return {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
            "frac": hbm_achieved / hbm,
            "traffic": (profiled_traffic("stage_tc_p3_ball.md", "stage_tc.cu")
                        if m["precision"] == "f32_tc" else None),
            "kernel": "stage_tc_kernel<3>" + (" (one pass)" if m["precision"] == "f32_tc1" else ""),
            "note": ("algorithmic bytes per stage: q, res read + q, res written (float32), "
                     "geometry record 128 B, connections 16 B; peak " + hbm_src),
            "flops_frac_fp32": flops / fp32_peak_tflops(2070.0),
            "avg_launch_ms": avg_launch_s * 1e3, "launches": m["klaunch"]}


def stage_bytes_per_element(p, word):
    """Algorithmic HBM bytes of one stage per element (word = 4 or 8 bytes)."""
    Np = (p + 1) * (p + 2) * (p + 3) // 6
    return 4 * 5 * Np * word + 32 * word + 16


LEARNED_AMPLITUDES = (0.001, 0.005, 0.02, 0.1)


def learned_bc_section(args, xyz, EToV, dev, stream, dist, world):
    """The learned closure end to end on the GPU: seeded reference runs on the
    radius-2 ball record traces at r = 1, the library trains the network,
    the large ball is the reference for the reflected energy of the free-stream,
    characteristic and learned conditions on the truncated ball, and the
    trained closure is timed on the bench workload."""
    from paper_1710_03887_gb300 import learned_bc as L
    n, runs, centred, every, iters = args.learned_n, 8, 48, args.learned_every, 1200
    t0 = time.perf_counter()
    nested = L.nested_ball(n)
    X, Y = L.record(WORKLOAD["order"], nested, L.run_seeds(0, runs, centred), every=every, device=dev,
                    width_scale=2.0, node_fraction=args.learned_fraction)
    t_rec = time.perf_counter() - t0
    w, hist = L.train(X, Y, iters=iters, lr=3e-3, seed=0, radius=nested.radius,
                      order=WORKLOAD["order"])
    t_train = time.perf_counter() - t0 - t_rec
    table = {}
    for amp in LEARNED_AMPLITUDES:
        table[f"{100 * amp:g}% p0"] = L.reflection_table(WORKLOAD["order"], nested, amp, 0.3,
                                                         (0.0, 0.0, 0.0), w)
    # sources off the centre, where the spherical memory is no longer exact
    table["2% p0 off-centre (0.3,0.1,-0.2)"] = L.reflection_table(
        WORKLOAD["order"], nested, 0.02, 0.25, (0.3, 0.1, -0.2), w)
    table["2% p0 off-centre (-0.2,0.35,0.1)"] = L.reflection_table(
        WORKLOAD["order"], nested, 0.02, 0.25, (-0.2, 0.35, 0.1), w)
    # plain float64 DG on the same pulse: the float32 form's reflected energy
    # and state against it (at 2 % p0)
    from paper_1710_03887_gb300 import binding as B
    centre = (0.0, 0.0, 0.0)
    small = nested if n <= 16 else L.nested_ball(16)      # float64 runs stay small
    r64, d64 = L.reflected_energy(WORKLOAD["order"], small, 0.02, 0.3, centre,
                                  B.DG_BC_CHARACTERISTIC, precision=B.DG_PREC_FP64)
    r32, d32 = L.reflected_energy(WORKLOAD["order"], small, 0.02, 0.3, centre,
                                  B.DG_BC_CHARACTERISTIC, precision=B.DG_PREC_F32)
    fp64_check = {
        "pulse": ("2% p0, width 0.3, centred; characteristic condition on the truncated ball "
                  f"of the n={min(n, 16)} lattice"),
        "reflected_energy_fp64": r64, "reflected_energy_f32": r32,
        "f32_minus_fp64_rel": (r32 - r64) / r64,
        "max_state_diff_rel_to_pulse_amplitude": L.max_state_difference(d32, d64, 0.02),
    }
    t_eval = time.perf_counter() - t0 - t_rec - t_train
    m = measure_form(args, "f32", xyz, EToV, dev, stream, dist, world, sample_clocks=False,
                     mlp=(w, WORKLOAD["radius"]))
    return ({
        "config": (f"radius-2 ball on the n={n} lattice ({len(nested.big[1])} tets), truncated at "
                   f"r=1 ({len(nested.small[1])} tets); p=3 float32; {runs} seeded pulse runs "
                   f"(centre |x|<0.5) and {centred} centred ones (width 0.2-0.4, amplitude "
                   f"0.1-10% p0) sampled every "
                   f"{every} steps at r=1 (fraction {args.learned_fraction:g} of the trace nodes); "
                   "measured with centred pulses of width 0.3 and two "
                   "off-centre pulses of width 0.25; 'spherical' is the memory closure w_in = psi "
                   "(the untrained network: its output layer starts at zero and its output "
                   "corrects psi)"),
        "samples": int(X.shape[0]), "iters": iters, "loss_first": float(hist[0]),
        "loss_last": float(hist[-1]),
        "reflected_energy_rel": table,
        "gain_vs_characteristic": {k: v["characteristic"] / v["learned"] for k, v in table.items()},
        "gain_vs_spherical": {k: v["spherical"] / v["learned"] for k, v in table.items()},
        "vs_plain_fp64": fp64_check,
        "seconds": {"record": t_rec, "train": t_train, "evaluate": t_eval},
        "bench_workload_learned_bc": {"value": m["value"], "unit": UNIT,
                                      "ms_per_step": m["ms"] / args.steps,
                                      "avg_stage_launch_ms": m["kms"] / max(m["klaunch"], 1)},
    }, w)


def rest_cfl_dt(xyz, EToV, order, p_fast, rho_fast, cfl=0.5):
    """The library's CFL step, cfl r_in / ((p+1)^2 max(|u| + c)), for a gas at
    rest whose fastest sound speed is sqrt(gamma p_fast / rho_fast), with the
    smallest inscribed radius 3V / (face areas) computed in chunks: no
    state-sized array on the host."""
    from paper_1710_03887_gb300 import workloads as W
    rin = np.inf
    for k0 in range(0, len(EToV), 1 << 20):
        v = xyz[EToV[k0:k0 + (1 << 20)]]
        vol = np.abs(np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]),
                               v[:, 3] - v[:, 0])) / 6.0
        area = sum(0.5 * np.linalg.norm(np.cross(v[:, b] - v[:, a], v[:, c] - v[:, a]), axis=1)
                   for a, b, c in ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)))
        rin = min(rin, float((3.0 * vol / area).min()))
    return cfl * rin / ((order + 1) ** 2 * np.sqrt(W.GAMMA * p_fast / rho_fast))


def horn_section(args, dev, stream):
    """Both float32 forms on the horn-in-room workload: the mixed-precision
    configuration's geometry (a flared horn with slip walls inside a room in
    front of its bell, ~1.5 M tets, p = 3, the inflow pulse of 10 % p0 at the
    mouthpiece), timed like the bench workload (device-resident state, CUDA
    events on the solver's stream), with the sensor analogues recorded."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    t0 = time.perf_counter()
    xyz, EToV, tag, info = W.horn_in_room()
    t_mesh = time.perf_counter() - t0
    out = {"workload": ("horn in a box room: bore 0.006, Bessel flare 0.006 (1.05 - x)^-0.7 to "
                        "x = 1, room 1.02 x 2 x 2 in front of the bell; %d tets (horn %d, room %d); "
                        "p=3; slip walls, inflow pulse A = 0.05 (peak 10%% p0), alpha = 565 /s, "
                        "characteristic BC on the room" % (len(EToV), info["n_horn"], info["n_room"])),
           "elements": int(len(EToV)), "mesh_seconds": t_mesh}
    for precision, code in (("f32", B.DG_PREC_F32), ("f32_tc", B.DG_PREC_F32_TC)):
        S = B.Solver(3, W.GAMMA, W.RHO0_SI, W.P0_SI, precision=code)
        S.set_stream(stream.cuda_stream)
        S.upload_mesh(xyz, EToV, face_tag=tag)
        S.set_bc(W.HORN_OUTER, B.DG_BC_CHARACTERISTIC)
        S.set_bc(W.HORN_WALL, B.DG_BC_SLIP_WALL)
        S.set_bc(W.HORN_MOUTHPIECE, B.DG_BC_INFLOW_PULSE)
        S.set_inflow(0.05, 565.0)
        q0 = torch.empty((S.K, 5, S.Np), dtype=torch.float64, device=dev)
        base = W.uniform_state(1, S.Np, W.RHO0_SI, (0, 0, 0), W.P0_SI, W.GAMMA)
        q0[:] = torch.from_numpy(base).to(dev)
        dt = rest_cfl_dt(xyz, EToV, 3, W.P0_SI, W.RHO0_SI)
        S.set_probes(info["sensors"], capacity=max(args.horn_steps, 1))
        S.set_state(q0)
        S.step(args.warmup, dt)
        S.read_probes()
        S.set_state(q0)
        torch.cuda.synchronize(dev)
        S.set_kernel_timing(True)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        S.step(args.horn_steps, dt)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        ms = start.elapsed_time(stop)
        kms, klaunch = S.read_kernel_timing()
        S.set_kernel_timing(False)
        series = S.read_probes(args.horn_steps)
        S.sync()
        dof = 5 * S.Np * S.K
        avg = kms / max(klaunch, 1)
        out[precision] = {
            "value": dof * args.horn_steps / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / args.horn_steps, "steps": args.horn_steps, "dt": dt,
            "avg_stage_launch_ms": avg,
            "stage_tflops": stage_flops_per_element(3) * S.K / (avg * 1e-3) / 1e12,
            "sensor_max_abs_dp_rel_p0": float(np.abs(series[..., 4] - series[:1, :, 4]).max()
                                              * (W.GAMMA - 1.0) / W.P0_SI)}
        S.close()
    return out


# the outer domains of section 1.2 (Table 1) at ~1.5 M elements: type B with
# the default lattice, type A (the room reaches 1.02 behind the mouthpiece)
# with a coarser one
HORN_DOMAINS = {
    "B-half-cube": dict(shape="box"),
    "B-half-sphere": dict(shape="sphere"),
    "B-half-cone": dict(shape="cone"),
    "A-cube": dict(shape="box", behind=1.02, m1=3, growth=1.3, aspect=4.0),
    "A-sphere": dict(shape="sphere", behind=1.02, m1=3, growth=1.3, aspect=4.0),
    "A-cone": dict(shape="cone", behind=1.02, m1=3, growth=1.3, aspect=4.0),
    "A-scone": dict(shape="scone", behind=1.02, m1=3, growth=1.3, aspect=4.0),
}


def domains_section(args, dev, stream):
    """The float32 form on full-size outer domains of Table 1 (slip-walled
    horn, the inflow pulse of 10 % p0 at the mouthpiece, characteristic
    condition on the outer surface), timed like the bench workload, with the
    Table 2 sensor analogues recorded every step."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    out = {"steps": args.horn_steps, "precision": "f32"}
    for name in [n for n in args.domains.split(",") if n]:
        kw = HORN_DOMAINS[name]
        t0 = time.perf_counter()
        xyz, EToV, tag, info = W.horn_in_room(**kw)
        t_mesh = time.perf_counter() - t0
        S = B.Solver(3, W.GAMMA, W.RHO0_SI, W.P0_SI, precision=B.DG_PREC_F32)
        S.set_stream(stream.cuda_stream)
        S.upload_mesh(xyz, EToV, face_tag=tag)
        S.set_bc(W.HORN_OUTER, B.DG_BC_CHARACTERISTIC)
        S.set_bc(W.HORN_WALL, B.DG_BC_SLIP_WALL)
        S.set_bc(W.HORN_MOUTHPIECE, B.DG_BC_INFLOW_PULSE)
        S.set_inflow(0.05, 565.0)
        q0 = torch.empty((S.K, 5, S.Np), dtype=torch.float64, device=dev)
        q0[:] = torch.from_numpy(W.uniform_state(1, S.Np, W.RHO0_SI, (0, 0, 0), W.P0_SI,
                                                 W.GAMMA)).to(dev)
        dt = rest_cfl_dt(xyz, EToV, 3, W.P0_SI, W.RHO0_SI)
        S.set_probes(info["sensors"], capacity=max(args.horn_steps, 1))
        S.set_state(q0)
        S.step(args.warmup, dt)
        S.read_probes()
        S.set_state(q0)
        torch.cuda.synchronize(dev)
        S.set_kernel_timing(True)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        S.step(args.horn_steps, dt)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        ms = start.elapsed_time(stop)
        kms, kl = S.read_kernel_timing()
        S.set_kernel_timing(False)
        series = S.read_probes(args.horn_steps)
        led = S.boundary_flux()
        S.sync()
        dof = 5 * S.Np * S.K
        avg = kms / max(kl, 1)
        out[name] = {
            "elements": int(S.K), "horn_elements": info["n_horn"], "mesh_seconds": t_mesh,
            "lattice": {k: v for k, v in kw.items() if k != "shape"},
            "value": dof * args.horn_steps / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / args.horn_steps, "dt": dt, "avg_stage_launch_ms": avg,
            "stage_tflops": stage_flops_per_element(3) * S.K / (avg * 1e-3) / 1e12,
            "mass_in_through_mouthpiece": float(-led[0]),
            "sensor_max_abs_dp_rel_p0": float(np.abs(series[..., 4] - series[:1, :, 4]).max()
                                              * (W.GAMMA - 1.0) / W.P0_SI)}
        S.close()
        del q0
    return out


def order4_section(args, xyz, EToV, dev, stream):
    """Both float32 forms at p = 4 (Np = 35, the production configuration's
    order) on the bench mesh, timed like the headline (median of repeated
    regions), with the tensor-core form's difference from the SIMT form after
    the same steps, relative to the perturbation."""
    from paper_1710_03887_gb300 import workloads as W
    sub = argparse.Namespace(**vars(args))
    sub.steps = args.order4_steps
    out = {"order": 4, "steps": sub.steps, "elements": int(len(EToV))}
    res = {}
    for f in ("f32", "f32_tc"):
        m = measure_form(sub, f, xyz, EToV, dev, stream, None, 1, False, order=4)
        res[f] = m
        out[f] = {"value": m["value"], "unit": UNIT, "ms_per_step": m["ms"] / sub.steps,
                  "avg_stage_launch_ms": m["kms"] / max(m["klaunch"], 1),
                  "repeats": repeat_stats(m["reps"], sub.steps),
                  "stage_tflops": stage_flops_per_element(4) * m["K"]
                  / (m["kms"] / max(m["klaunch"], 1) * 1e-3) / 1e12}
    a, b = res["f32_tc"], res["f32"]
    base = W.uniform_state(a["q0"].shape[0], a["q0"].shape[2], W.RHO0_SI, (0, 0, 0), W.P0_SI,
                           W.GAMMA)
    num = np.abs(a["q_end"] - b["q_end"]).max(axis=(0, 2))
    den = np.abs(b["q_end"] - base).max(axis=(0, 2))
    out["f32_tc_vs_f32_max_diff_rel_to_perturbation"] = (num / den).tolist()
    out["tc_speedup"] = a["value"] / b["value"]
    return out


def locality_section(args, xyz, EToV, dev, stream):
    """The float32 form on the bench mesh with its elements in three orders:
    as built (lattice order), sorted along a Morton curve, and randomly
    permuted (a mesh generator's order, at its worst). Tiles are runs of
    consecutive elements, so the order decides how many faces a tile shares
    internally and how far its gathers reach."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    w = WORKLOAD
    ET = 32
    out = {"steps": args.locality_steps, "tile_elements": ET}
    # the ball as the lattice generator numbers it (the bench itself runs it
    # in Morton order)
    xyz, EToV = W.ball(w["n"], w["radius"], jitter=w["jitter"], seed=w["seed"])
    for name, perm in (("lattice", None), ("morton", W.morton_order(xyz, EToV)),
                       ("random", W.random_order(len(EToV), 1))):
        E = EToV if perm is None else EToV[perm]
        S = B.Solver(w["order"], W.GAMMA, W.RHO0_SI, W.P0_SI, precision=B.DG_PREC_F32)
        S.set_stream(stream.cuda_stream)
        S.upload_mesh(xyz, E)
        EToE = S.geometry()["EToE"]
        own = np.arange(len(E))[:, None] // ET
        interior = EToE >= 0
        intra = float(np.count_nonzero(interior & (EToE // ET == own)) / np.count_nonzero(interior))
        q0 = W.gaussian_pulse_state(S.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, w["amplitude"],
                                    w["width"])
        dt = S.stable_dt(q0, w["cfl"])
        q0d = torch.from_numpy(q0).to(dev)
        S.set_state(q0d)
        S.step(args.warmup, dt)
        S.set_state(q0d)
        torch.cuda.synchronize(dev)
        S.set_kernel_timing(True)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        S.step(args.locality_steps, dt)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        ms = start.elapsed_time(stop)
        kms, kl = S.read_kernel_timing()
        S.set_kernel_timing(False)
        S.sync()
        dof = 5 * S.Np * S.K
        out[name] = {"value": dof * args.locality_steps / (ms * 1e-3), "unit": UNIT,
                     "ms_per_step": ms / args.locality_steps,
                     "avg_stage_launch_ms": kms / max(kl, 1),
                     "interior_faces_inside_a_tile": intra}
        S.close()
    return out


def paper_config_section(args, xyz, EToV, dev, stream):
    """The paper's own configuration (section 1.1, Appendix A; Tables 1 and 3):
    linear elements (p = 1) and RK2 on a ~200k-element mesh, in the paper's
    discretisation (Gauss quadrature, Heun) and, beside it, the nodal float64
    and float32 forms at p = 1; each with the device memory its context
    holds per element (the paper's Table 3 gives ~1000 B per element)."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    w = WORKLOAD
    out = {"order": 1, "elements": int(len(EToV)), "steps": args.paper_steps,
           "paper_bytes_per_element": "998-1111 (Tables 1 and 3, GTX 750 Ti, precision not stated)"}
    for name, code in (("modal", B.DG_PREC_MODAL), ("fp64", B.DG_PREC_FP64), ("f32", B.DG_PREC_F32)):
        S = B.Solver(1, W.GAMMA, W.RHO0_SI, W.P0_SI, precision=code)
        S.set_stream(stream.cuda_stream)
        S.upload_mesh(xyz, EToV)                      # host only: no device memory yet
        q0 = W.gaussian_pulse_state(S.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, w["amplitude"],
                                    w["width"])
        dt = S.stable_dt(q0, w["cfl"])
        q0d = torch.from_numpy(q0).to(dev)
        torch.cuda.synchronize(dev)
        free0 = torch.cuda.mem_get_info(dev)[0]
        S.set_state(q0d)                              # the context allocates here
        S.step(args.warmup, dt)
        S.set_state(q0d)
        torch.cuda.synchronize(dev)
        held = free0 - torch.cuda.mem_get_info(dev)[0]
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        S.step(args.paper_steps, dt)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        ms = start.elapsed_time(stop)
        S.sync()
        dof = 5 * S.Np * S.K
        out[name] = {"value": dof * args.paper_steps / (ms * 1e-3), "unit": UNIT,
                     "ms_per_step": ms / args.paper_steps,
                     "stages_per_step": 2 if name == "modal" else 5,
                     "device_bytes_per_element": held / S.K}
        S.close()
        del q0d
    return out


def far_field_probes(n=32, radius=2.5):
    """n points on the half-sphere of the given radius in front of the bell
    (x > 0 about the bell's centre), spread by a Fibonacci spiral."""
    k = np.arange(n) + 0.5
    z = k / n                                     # cos of the angle from the axis, in (0, 1)
    phi = np.pi * (1.0 + 5.0 ** 0.5) * k
    r = np.sqrt(1.0 - z * z)
    return radius * np.column_stack([z, r * np.cos(phi), r * np.sin(phi)])


def production_section(args, dev, stream, weights=None):
    """The production configuration: the horn in a sphere of radius 3 about
    its bell's centre, with the region behind the bell kept (type A, ~8M
    tets) and truncated (type B half-ball), p = 4, both float32 perturbation
    forms (SIMT and tensor-core contractions), slip walls, the 10 % p0 inflow
    pulse at the mouthpiece, the learned closure on the outer sphere
    (``weights``: the network trained by the learned-closure section, else
    the spherical-wave memory alone) and 32 far-field pressure probes at
    radius 2.5; coordinates are shifted so the bell's centre is the origin,
    the centre of the closure's spherical memory. Timed like the bench
    workload."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import learned_bc as LB
    from paper_1710_03887_gb300 import workloads as W
    w_net = LB.spherical_weights() if weights is None else np.asarray(weights, dtype=np.float32)
    probes = far_field_probes()
    out = {"order": 4, "steps": args.production_steps, "precisions": ["f32", "f32_tc"],
           "closure": "trained network" if weights is not None else "spherical-wave memory",
           "probes": "32 points at radius 2.5 about the bell's centre (Fibonacci half-sphere)"}
    for name, kw in (("kept", dict(shape="sphere", room_length=3.0, behind=2.0, m1=3, growth=1.16,
                                   aspect=2.5)),
                     ("truncated", dict(shape="sphere", room_length=3.0))):
        t0 = time.perf_counter()
        xyz, EToV, tag, info = W.horn_in_room(**kw)
        xyz = xyz - np.array([info["bell_x"], 0.0, 0.0])        # bell centre at the origin
        mesh_s = time.perf_counter() - t0
        out[name] = {"elements": int(len(EToV)), "horn_elements": info["n_horn"],
                     "lattice": {k: v for k, v in kw.items() if k != "shape"},
                     "mesh_seconds": mesh_s}
        for prec_name, prec in (("f32", B.DG_PREC_F32), ("f32_tc", B.DG_PREC_F32_TC)):
            out[name][prec_name] = _production_run(args, dev, stream, xyz, EToV, tag, prec, w_net,
                                                   probes)
    return out


def _production_run(args, dev, stream, xyz, EToV, tag, prec, w_net, probes):
    """One float32 form on one production mesh, timed like the bench."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    t0 = time.perf_counter()
    S = B.Solver(4, W.GAMMA, W.RHO0_SI, W.P0_SI, precision=prec)
    S.set_stream(stream.cuda_stream)
    S.upload_mesh(xyz, EToV, face_tag=tag)
    S.set_bc(W.HORN_OUTER, B.DG_BC_LEARNED)
    S.set_bc(W.HORN_WALL, B.DG_BC_SLIP_WALL)
    S.set_bc(W.HORN_MOUTHPIECE, B.DG_BC_INFLOW_PULSE)
    S.set_inflow(0.05, 565.0)
    S.set_bc_mlp(w_net, 3.0)
    S.set_probes(probes, capacity=max(args.production_steps, 1))
    q0 = torch.empty((S.K, 5, S.Np), dtype=torch.float64, device=dev)
    q0[:] = torch.from_numpy(W.uniform_state(1, S.Np, W.RHO0_SI, (0, 0, 0), W.P0_SI,
                                             W.GAMMA)).to(dev)
    # the fastest state of the run: the inflow pulse's peak, at rest
    dt = rest_cfl_dt(xyz, EToV, 4, 1.1 * W.P0_SI, W.RHO0_SI * 1.1 ** (1.0 / W.GAMMA))
    setup = time.perf_counter() - t0
    S.set_state(q0)
    S.step(1, dt)
    S.set_state(q0)
    S.read_probes()
    torch.cuda.synchronize(dev)
    S.set_kernel_timing(True)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    S.step(args.production_steps, dt)
    stop.record(stream)
    torch.cuda.synchronize(dev)
    ms = start.elapsed_time(stop)
    kms, kl = S.read_kernel_timing()
    S.set_kernel_timing(False)
    series = S.read_probes(args.production_steps)
    led = S.boundary_flux()
    S.sync()
    dof = 5 * S.Np * S.K
    avg = kms / max(kl, 1)
    res = {
        "dof": int(dof),
        "value": dof * args.production_steps / (ms * 1e-3), "unit": UNIT,
        "ms_per_step": ms / args.production_steps, "dt": dt,
        "avg_stage_launch_ms_with_closure": avg,
        "stage_tflops": stage_flops_per_element(4) * S.K / (avg * 1e-3) / 1e12,
        "mass_in_through_mouthpiece": float(-led[0]),
        "probe_max_abs_dp_rel_p0": float(np.abs(series[..., 4] - series[:1, :, 4]).max()
                                         * (W.GAMMA - 1.0) / W.P0_SI),
        "setup_seconds": setup}
    S.close()
    del q0
    torch.cuda.empty_cache()
    return res


# six probes near the axes at r = 0.5: images of one point inside an element
# under reflections and axis swaps of the lattice, so a centred pulse gives
# them equal values (exactly on an unjittered lattice ball)
_A, _B, _C = 0.5, 0.013, 0.007
AXIS_PROBES = np.array([[_A, _B, _C], [-_A, _B, _C], [_B, _A, _C], [_B, -_A, _C], [_C, _B, _A],
                        [_C, _B, -_A]], dtype=np.float64)


def acoustic_energy(q_rel, J, M, gamma, rho0, p0):
    """Acoustic energy  sum_e J_e (p'^T M p' / (2 rho0 c0^2) + m'^T M m' / (2 rho0))  of a
    perturbation given as (rho', m', p') on the nodes: q_rel[K, 5, Np] holds
    rho', m_x, m_y, m_z and p' (pressure perturbation, not energy)."""
    c2 = gamma * p0 / rho0
    pm = np.einsum("ki,ij,kj->k", q_rel[:, 4], M, q_rel[:, 4]) / (2.0 * rho0 * c2)
    mm = sum(np.einsum("ki,ij,kj->k", q_rel[:, v], M, q_rel[:, v]) for v in (1, 2, 3)) / (2.0 * rho0)
    return float(np.sum(J * (pm + mm)))


def pressure(q, gamma):
    """p = (gamma - 1)(E - |m|^2 / (2 rho)) of conserved states q[..., 5, ...] (axis -2)."""
    rho, E = q[..., 0, :], q[..., 4, :]
    m2 = q[..., 1, :] ** 2 + q[..., 2, :] ** 2 + q[..., 3, :] ** 2
    return (gamma - 1.0) * (E - 0.5 * m2 / rho)


def precision_comparison(run32, run64, amplitude, M, gamma, rho0, p0):
    """The float32 perturbation form against plain float64 DG after the same
    steps from the same pulse. Each run: q0, q (end states [K, 5, Np]),
    probes [steps, 6, 5] (the axis probes), tot0, tot, led (conserved totals
    at start and end, boundary ledger), J. Returns the comparison's figures,
    every one relative to a stated scale."""
    q0, q32, q64 = run64["q0"], run32["q"], run64["q"]
    K, _, Np = q0.shape
    base = np.zeros((1, 5, 1))
    base[0, 0, 0] = rho0
    base[0, 4, 0] = p0 / (gamma - 1.0)
    num = np.abs(q32 - q64).max(axis=(0, 2))
    den = np.abs(q64 - base).max(axis=(0, 2))
    p32, p64 = pressure(q32, gamma), pressure(q64, gamma)
    apulse = amplitude * p0
    diff = np.empty_like(q64)
    diff[:, 0:4] = q32[:, 0:4] - q64[:, 0:4]
    diff[:, 4] = p32 - p64
    init = np.zeros_like(q0)
    init[:, 0:4] = q0[:, 0:4] - base[:, 0:4]
    init[:, 4] = pressure(q0, gamma) - p0
    e_init = acoustic_energy(init, run64["J"], M, gamma, rho0, p0)
    e_diff = acoustic_energy(diff, run64["J"], M, gamma, rho0, p0)
    pr32 = pressure(np.swapaxes(run32["probes"], 1, 2), gamma)       # [steps, 6]
    pr64 = pressure(np.swapaxes(run64["probes"], 1, 2), gamma)
    out = {
        "max_err_per_var_rel_to_perturbation": (num / np.where(den > 0, den, 1.0)).tolist(),
        "pressure_max_diff_rel_to_pulse_amplitude": float(np.abs(p32 - p64).max() / apulse),
        "energy_of_difference_rel_to_initial_acoustic_energy": e_diff / e_init,
        "axis_probes_f32_minus_fp64_max_rel_to_pulse_amplitude": float(np.abs(pr32 - pr64).max() / apulse),
        "axis_probes_spread_rel_to_pulse_amplitude": {
            "f32": float((pr32.max(axis=1) - pr32.min(axis=1)).max() / apulse),
            "fp64": float((pr64.max(axis=1) - pr64.min(axis=1)).max() / apulse)},
        "axis_probes_peak_rel_to_pulse_amplitude": float(np.abs(pr64 - p0).max() / apulse),
    }
    # scale of each total: its own size, and for the momentum components
    # (zero at rest) the total mass times c0
    scale = np.abs(run64["tot0"]).astype(np.float64)
    scale[1:4] = np.maximum(scale[1:4], abs(run64["tot0"][0]) * np.sqrt(gamma * p0 / rho0))
    scale = scale.clip(min=1e-300)
    for name, r in (("f32", run32), ("fp64", run64)):
        bal = r["tot"] - r["tot0"] + r["led"]
        out["balance_rel_" + name] = (np.abs(bal) / scale).tolist()
    out["ledger_f32_minus_fp64_rel_to_totals"] = (np.abs(run32["led"] - run64["led"]) / scale).tolist()
    return out


def precision_run(order, xyz, EToV, precision, steps, amplitude, width, cfl, dev, stream):
    """One run of the C2 comparison: the pulse at the centre, the six axis
    probes sampled every step. Returns the dict precision_comparison reads."""
    import torch
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    S = B.Solver(order, W.GAMMA, W.RHO0_SI, W.P0_SI, precision=precision)
    S.set_stream(stream.cuda_stream)
    S.upload_mesh(xyz, EToV)
    q0 = W.gaussian_pulse_state(S.node_coords(), W.GAMMA, W.RHO0_SI, W.P0_SI, amplitude, width)
    dt = S.stable_dt(q0, cfl)
    S.set_probes(AXIS_PROBES, capacity=max(steps, 1))
    S.set_state(torch.from_numpy(q0).to(dev))
    tot0 = S.totals()
    t0 = time.perf_counter()
    S.step(steps, dt)
    S.sync()
    secs = time.perf_counter() - t0
    q, _ = S.get_state()
    out = dict(q0=q0, q=q, probes=S.read_probes(steps), tot0=tot0, tot=S.totals(),
               led=S.boundary_flux(), J=S.geometry()["J"], dt=dt, seconds=secs)
    S.close()
    return out


def c2_section(args, xyz, EToV, dev, stream):
    """Configuration C2 at its full length: plain float64 DG and the float32
    perturbation form, from the same 10 % p0 pulse at the centre of the bench
    ball, for --c2-steps steps; element-wise, probe, energy and balance
    comparison (precision_comparison)."""
    from paper_1710_03887_gb300 import binding as B
    from paper_1710_03887_gb300 import workloads as W
    w = WORKLOAD
    r64 = precision_run(w["order"], xyz, EToV, B.DG_PREC_FP64, args.c2_steps, w["amplitude"],
                        w["width"], w["cfl"], dev, stream)
    r32 = precision_run(w["order"], xyz, EToV, B.DG_PREC_F32, args.c2_steps, w["amplitude"],
                        w["width"], w["cfl"], dev, stream)
    out = precision_comparison(r32, r64, w["amplitude"], B.reference_mass(w["order"]), W.GAMMA,
                               W.RHO0_SI, W.P0_SI)
    c0 = float(np.sqrt(W.GAMMA * W.P0_SI / W.RHO0_SI))
    out.update({"steps": args.c2_steps, "dt": r64["dt"],
                "distance_travelled_c0_t": c0 * r64["dt"] * args.c2_steps,
                "seconds": {"fp64": r64["seconds"], "f32": r32["seconds"]},
                "workload": WORKLOAD_NAME + "; axis probes at r = 0.5"})
    return out


def run_gpu(args, rank, world):
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    xyz, EToV = build_workload()
    if args.partition and world > 1:
        m = measure_partitioned(args, xyz, EToV, dev, stream, dist, world, rank)
        if rank == 0:
            line = {
                "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"] / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": args.precision, "data": "synthetic",
                "config": {"workload": WORKLOAD_NAME, "elements": m["K"], "order": w["order"],
                           "dof": m["dof"], "dt": m["dt"], "precision": args.precision,
                           "parallelism": f"element partition x{world} (Morton slabs; halo "
                                          "exchange of cut-face traces before every stage, NCCL)",
                           "rank0_elements": m["K_own"], "rank0_cut_faces": m["cut_faces"]},
                "repeats": repeat_stats(m["reps"], args.steps),
                "gpu_launches": args.steps * 5 * (3 if m["peers"] else 1),
                "clocks": m["clocks"],
            }
            print(json.dumps(line), flush=True)
        return
    forms = [args.precision] + [f for f in ("f32_tc", "f32", "fp64", "modal", "f32_tc1")
                                if f != args.precision and not args.one_form]
    res = {f: measure_form(args, f, xyz, EToV, dev, stream, dist, world, sample_clocks=(f == args.precision))
           for f in forms}
    if rank != 0:
        return
    head = res[args.precision]
    state_bytes = head["dof"] * 8
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head["precision"], "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "elements": head["K"], "order": w["order"],
                   "dof": head["dof"], "dt": head["dt"], "precision": head["precision"],
                   "parallelism": f"replicas x{world}",
                   "l2": ("inputs larger than L2 (four state-sized streams per stage, "
                          f"{state_bytes / (2 if head['precision'] == 'f32' else 1) / 1e6:.0f} MB each); no flush")},
        "e2e": {"value": head["e2e"], "unit": UNIT, "h2d_bytes_per_step": state_bytes / args.steps,
                "d2h_bytes_per_step": (state_bytes + head["nprobe"] * 5 * 8 * args.steps) / args.steps},
        # 5 stage kernels (ledger inside) + 1 probe kernel per step; 2 + 1 for Heun's RK2
        "gpu_launches": args.steps * (3 if head["precision"] == "modal" else 6),
        "roofline": roofline_for(head, w["order"]),
        "clocks": head["clocks"],
        "repeats": repeat_stats(head["reps"], args.steps, (head["clocks"] or {}).get("sm_mhz")),
    }
    forms_out = {}
    for f, m in res.items():
        forms_out[f] = {"value": m["value"], "ms_per_step": m["ms"] / args.steps, "e2e": m["e2e"],
                        "repeats": repeat_stats(m["reps"], args.steps),
                        "roofline": roofline_for(m, w["order"])}
    from paper_1710_03887_gb300 import workloads as W
    for f in ("f32", "f32_tc", "f32_tc1"):
        if f in res and "fp64" in res:
            a, b = res[f], res["fp64"]
            base = W.uniform_state(a["q0"].shape[0], a["q0"].shape[2], W.RHO0_SI, (0, 0, 0),
                                   W.P0_SI, W.GAMMA)
            num = np.abs(a["q_end"] - b["q_end"]).max(axis=(0, 2))
            den = np.abs(b["q_end"] - base).max(axis=(0, 2))
            forms_out[f + "_vs_fp64"] = {
                "max_err_per_var_rel_to_perturbation": (num / den).tolist(),
                "after_steps": args.steps,
                "speedup": a["value"] / b["value"]}
    if "modal" in res and "fp64" in res:
        # the two discretisations side by side (same pulse, same dt, same steps):
        # their difference is the discretisation difference (quadrature vs
        # collocation, RK2 vs RK4), measured against the perturbation
        a, b = res["modal"], res["fp64"]
        base = W.uniform_state(a["q0"].shape[0], a["q0"].shape[2], W.RHO0_SI, (0, 0, 0),
                               W.P0_SI, W.GAMMA)
        num = np.abs(a["q_end"] - b["q_end"]).max(axis=(0, 2))
        den = np.abs(b["q_end"] - base).max(axis=(0, 2))
        forms_out["modal_vs_nodal_fp64"] = {
            "max_diff_per_var_rel_to_perturbation": (num / den).tolist(), "after_steps": args.steps,
            "speedup_per_step": a["value"] / b["value"]}
    line["forms"] = forms_out
    if args.c2_steps > 0:
        line["f32_vs_fp64_%d" % args.c2_steps] = c2_section(args, xyz, EToV, dev, stream)
    if args.learned_n > 0:
        # rank 0 only, after the replicas' timed regions: no barrier inside
        lb, trained = learned_bc_section(args, xyz, EToV, dev, stream, None, 1)
        lb["bench_workload_learned_bc"]["vs_characteristic"] = (
            lb["bench_workload_learned_bc"]["value"] / res["f32"]["value"] if "f32" in res else None)
        line["learned_bc"] = lb
    if args.closure_timing:
        # the closure's cost alone: the untrained network (the spherical
        # memory) does the same work per stage as a trained one
        from paper_1710_03887_gb300 import learned_bc as L
        m = measure_form(args, "f32", xyz, EToV, dev, stream, None, 1, False,
                         mlp=(L.spherical_weights(), WORKLOAD["radius"]))
        line["closure_timing"] = {
            "value": m["value"], "unit": UNIT, "ms_per_step": m["ms"] / args.steps,
            "avg_stage_launch_ms": m["kms"] / max(m["klaunch"], 1),
            "vs_characteristic": m["value"] / res["f32"]["value"] if "f32" in res else None}
    if args.horn_steps > 0:
        line["horn"] = horn_section(args, dev, stream)
        if args.domains:
            line["domains"] = domains_section(args, dev, stream)
    if args.order4_steps > 0:
        line["order4"] = order4_section(args, xyz, EToV, dev, stream)
    if args.locality_steps > 0:
        line["locality"] = locality_section(args, xyz, EToV, dev, stream)
    if args.paper_steps > 0:
        line["paper_configuration"] = paper_config_section(args, xyz, EToV, dev, stream)
    if args.production_steps > 0:
        line["production"] = production_section(args, dev, stream,
                                                 trained if args.learned_n > 0 else None)
    if not args.no_cpu_baseline:
        v, sample, _ = cpu_sample_run(args.cpu_steps, 1, xyz, EToV)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--repeats", type=int, default=0,
                    help="timed regions of --steps steps per form (median reported, spread beside "
                         "it); 0 = at least 5 and enough to span ~0.5 s")
    ap.add_argument("--c2-steps", type=int, default=2000,
                    help="steps of the float32-against-float64 run on the bench workload (0: skip it)")
    ap.add_argument("--cpu-steps", type=int, default=50,
                    help="oracle steps on the CPU sample (about 10-20 s of one core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="f32", choices=["f32", "f32_tc", "fp64", "modal", "f32_tc1"],
                    help="arithmetic form of the headline number (the other is measured beside it)")
    ap.add_argument("--one-form", action="store_true", help="measure only --precision")
    ap.add_argument("--partition", action="store_true",
                    help="under torchrun: split the one mesh across the ranks (halo exchange per "
                         "stage, strong scaling) instead of running independent replicas")
    ap.add_argument("--learned-n", type=int, default=16,
                    help="lattice of the learned-closure experiment's radius-2 ball (0 = skip; "
                         "64 gives the ~200k-element truncated ball of the configuration)")
    ap.add_argument("--closure-timing", action="store_true",
                    help="time the bench workload with the learned closure on the untrained "
                         "network, without the training experiment")
    ap.add_argument("--production-steps", type=int, default=0,
                    help="steps timed on the production configuration: p=4, the horn in a "
                         "radius-3 sphere with the region behind the bell kept (~8M tets) and "
                         "truncated, learned closure, 32 far-field probes (0: skip it; it builds "
                         "the meshes on the host first, a few minutes)")
    ap.add_argument("--paper-steps", type=int, default=50,
                    help="steps timed per form in the paper-configuration section (0: skip it)")
    ap.add_argument("--order4-steps", type=int, default=20,
                    help="steps timed per float32 form at p = 4 on the bench mesh (0: skip it)")
    ap.add_argument("--locality-steps", type=int, default=20,
                    help="steps timed per element order in the locality section (0: skip it)")
    ap.add_argument("--horn-steps", type=int, default=20,
                    help="steps timed on the horn-in-room workload (0: skip it)")
    ap.add_argument("--domains", default="B-half-sphere,A-sphere",
                    help="comma-separated outer domains of Table 1 timed at full size after the "
                         "horn section (names of bench.HORN_DOMAINS; empty: none)")
    ap.add_argument("--learned-every", type=int, default=10, help="steps between trace samples")
    ap.add_argument("--learned-fraction", type=float, default=0.125,
                    help="fraction of trace nodes kept per sample (seeded)")
    ap.add_argument("--mesh-n", type=int, default=WORKLOAD["n"],
                    help="lattice size of the ball (32 = the benchmark; smaller for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.repeats < 0:
        ap.error("--repeats must be >= 0")
    WORKLOAD["n"] = args.mesh_n
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if args.impl != "reference":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
