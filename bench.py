"""Benchmark: device-timed MLUPS of the fused N-phase lattice Boltzmann step
and its fraction of the HBM roofline.

Workload (one GPU): the 2048x2048 periodic five-phase disk suspension
(200 disks, radii U[10, 40], densities {1, 2, 5, 10, 1}, eps = 4, mobility
0.1, Model B unless --model A).  One step = every phase set and the flow set
advanced one time step = one launch of the fused step kernel.  The
population buffers (604 MB each) are larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--model A|B] [--storage f32|bf16|f16]
                    [--impl reference] [--no-forms] [--no-cpu-baseline]

Beside the headline the line carries "forms": the same workload with
bfloat16 / binary16 population storage (throughput, roofline fraction and
distance to the FP32 fields after the same steps), the other model (Model A
with n = 1 beside the Model B headline), the error of every storage against
the FP64 oracle on the 256x256 cut of the workload (short and 2000-step
horizons, both unit-vector readings), the 64-member lens ensemble advanced in
one persistent launch per step (against one launch per member), the ternary
Rayleigh-Taylor instability (gravity and walls) and the differentiated run
(forward and reverse sweep of the adjoint).

Under torchrun (N > 1) every rank runs an independent replica of the
workload (weak scaling, no collective on the data path); rank 0 prints one
JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (rank 0
only), on a 256x256 cut of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N-phase LBM MLUPS & % HBM roofline: plain FP32 vs BF16/batched/adjoint forms"
WORKLOAD = "2048x2048 periodic, N=5, 200 disks (seed 2306), eps=4, M=0.1"
# GB300 HBM3e nominal bandwidth (GB/s); the roofline fraction is taken
# against the measured copy bandwidth, this one is reported beside it
NOMINAL_HBM_GBS = 8000.0


def bytes_per_lup(N: int, storage: str = "f32") -> int:
    """Algorithmic HBM bytes of one lattice update: each stored value read
    once and written once.  FP32 storage: 9(N-1) phase + 8 flow populations
    and (N-1) phi + 2 u + 2 m_phi of the previous step, 4 bytes each.
    16-bit storage: 8(N-1) phase + 8 flow deviations of 2 bytes, (N-1) FP32
    rest populations, and (N-1) phi + 2 u + 2 m_phi + 1 P of 4 bytes."""
    if storage == "f32":
        return 8 * (9 * (N - 1) + 8 + (N - 1) + 4)
    return 2 * (2 * (8 * (N - 1) + 8) + 4 * (N - 1) + 4 * ((N - 1) + 5))


def adjoint_bytes_per_lup(N: int) -> dict:
    """Algorithmic HBM bytes of one differentiated lattice update (Model B,
    FP32; NS = N - 1 solved phases, NP = N(N-1)/2 tension pairs), each field
    a pass reads or writes counted once per pass:
    forward step 8(10N + 2); reverse step = the taping rebuild (a forward
    step that also writes 8 NS + 13 tape floats) and four passes:
    1 collision: 8 NS + 12 tape, NS + 4 state and 10 NS + 12 seed floats
      read, 9 NS + 16 adjoint floats written, NP + 1 FP64 sums updated;
    2 source: 10 NS + 10 floats read, 3 NS + 2 written, one FP64 sum updated;
    3 stencil: 4 NS read, NS written;
    4 pull: 3 NS + 8 read, 9 NS + 8 written."""
    NS, NP = N - 1, N * (N - 1) // 2
    fwd = 8 * (10 * N + 2)
    tape = fwd + 4 * (8 * NS + 13)
    collide = 4 * ((8 * NS + 12) + (NS + 4) + (10 * NS + 12) + (9 * NS + 16)) + 16 * (NP + 1)
    source = 4 * ((10 * NS + 10) + (3 * NS + 2)) + 16
    stencil = 4 * (4 * NS + NS)
    pull = 4 * ((3 * NS + 8) + (9 * NS + 8))
    return {"forward": fwd, "reverse": tape + collide + source + stencil + pull,
            "reverse_parts": {"taping_rebuild": tape, "collision": collide, "source": source,
                              "stencil": stencil, "pull": pull}}


def kernel_sources_digest() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_06983_gb300", "csrc")
    for name in ("step_kernel.cuh", "nlbm_internal.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(model: str, storage: str = "f32"):
    """DRAM bytes per lattice update of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    suffix = "" if storage == "f32" else f"_{storage}"
    path = os.path.join(ROOT, "profiles", f"step_kernel_model{model}{suffix}_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.lstrip().startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_digest") != kernel_sources_digest():
        return None
    try:
        return float(kv["dram_bytes_per_lup"])
    except (KeyError, ValueError):
        return None


def reduce_max_over_ranks(values):
    """Max over ranks of a list of floats (identity without a process group).
    Uses the process group's own backend: gloo on CPU tensors, NCCL on CUDA."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_mlups(world: int, lups_per_step: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas, each advancing lups_per_step
    lattice updates per step, over the slowest rank's time."""
    return world * lups_per_step * steps / seconds / 1e6


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v == "Active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows),
                "samples": len(rows), "reasons": reasons}


def oracle_sample(model: str, steps: int, warmup: int, cut: int = 512):
    """FP64 oracle on a cut x cut corner of the workload; returns (MLUPS, cores, seconds)."""
    from oracle.oracle import OracleSim, max_threads
    from paper_2306_06983_gb300 import workloads as W
    p, phi0 = W.disks_2048(model)
    q = dict(p, nx=cut, ny=cut)
    o = OracleSim(q, np.ascontiguousarray(phi0[:, :cut, :cut]))
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return cut * cut * steps / dt / 1e6, max_threads(), dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.oracle import build_oracle
    build_oracle()
    steps = max(1, args.steps)
    cut = 256
    mlups, cores, dt = oracle_sample(args.model, steps, args.warmup, cut)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": round(dt / steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + f", Model {args.model}; {cut}x{cut} cut on host cores",
                   "nx": cut, "ny": cut, "n_phases": 5, "model": args.model},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{steps} time steps of a {cut}x{cut} cut of the 2048x2048 "
                                   f"N=5 workload, FP64 oracle, OpenMP"},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_forms(args, p, phi0, ref_fields, lups, peak):
    """The other forms of the method, each timed with CUDA events over
    args.steps steps after args.warmup, beside the headline (FP32) run:
    16-bit population storage on the same workload (with its distance to the
    FP32 fields after the same steps), the 64-member lens ensemble in one
    persistent launch per step (autotuned tile shape, graph replays) against
    one launch per member, the ternary Rayleigh-Taylor instability (gravity,
    walls) and the adjoint."""
    import torch
    from paper_2306_06983_gb300 import workloads as W
    from paper_2306_06983_gb300.nlbm import Batch, Simulation

    def timed(stream, fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    forms = {}
    N = p["n_phases"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for st in ("bf16", "f16"):
            if st == args.storage:
                continue
            sim = Simulation(dict(p, storage=st), stream=stream)
            sim.set_phi(phi0.astype(np.float32))
            m0 = sim.phase_mass()
            tile = sim.autotune(20)[:2]
            sim.step(args.warmup)
            ms = timed(stream, sim.step, args.steps)
            phi, u = (t.cpu().numpy() for t in sim.moments()[:2])
            m1 = sim.phase_mass(allow_diverged=True)
            sim.close()
            del sim
            torch.cuda.empty_cache()
            bpl = bytes_per_lup(N, st)
            fphi, fu = ref_fields
            forms[st] = {
                "value": round(lups / ms / 1e3, 2), "unit": "MLUPS", "ms_per_step": round(ms, 5),
                "algorithmic_bytes_per_lup": bpl,
                "roofline_frac": round(bpl * lups / (ms / 1e3) / 1e9 / peak, 4),
                # the minimum for 16-bit populations with every population
                # (the rest one too) in 16 bits and N + 3 FP32 fields
                "roofline_frac_at_min_bytes": round((44 * N + 20) * lups / (ms / 1e3) / 1e9 / peak, 4),
                "min_bytes_per_lup": 44 * N + 20, "tile": list(tile),
                "of_f32_headline": None,
                "vs_f32_after_same_steps": {
                    "steps": args.warmup + args.steps,
                    "max_abs_dphi": float(np.abs(phi - fphi).max()),
                    "u_rel_l2": float(np.sqrt(((u - fu) ** 2).sum() / max((fu ** 2).sum(), 1e-300)))},
                "mass_drift_rel": float((np.abs(m1 - m0) / np.abs(m0)).max()),
            }

        # the other model on the same workload (Model A with n = 1 beside the
        # Model B headline, or B beside A), FP32
        other = "A" if args.model == "B" else "B"
        q = dict(p, model=other, model_a_n=1.0, storage="f32")
        sim = Simulation(q, stream=stream)
        sim.set_phi(phi0.astype(np.float32))
        m0 = sim.phase_mass()
        tile = sim.autotune(20)[:2]
        sim.step(args.warmup)
        ms = timed(stream, sim.step, args.steps)
        m1 = sim.phase_mass(allow_diverged=True)
        sim.close()
        del sim
        torch.cuda.empty_cache()
        bpl = bytes_per_lup(N)
        forms[f"model_{other}"] = {
            "workload": WORKLOAD + f", Model {other}" + (" (n = 1)" if other == "A" else ""),
            "value": round(lups / ms / 1e3, 2), "unit": "MLUPS", "ms_per_step": round(ms, 5), "tile": list(tile),
            "algorithmic_bytes_per_lup": bpl,
            "roofline_frac": round(bpl * lups / (ms / 1e3) / 1e9 / peak, 4),
            "mass_drift_rel": float((np.abs(m1 - m0) / np.abs(m0)).max()),
        }
        if not args.no_oracle_accuracy:
            forms["accuracy_256"] = measure_accuracy_256(args, stream)

        mem = W.lens_ensemble(64)
        nodes = sum(q["nx"] * q["ny"] for q, _ in mem)
        b = Batch([q for q, _ in mem], stream=stream)
        for k, (_, f0) in enumerate(mem):
            b.set_phi(k, f0.astype(np.float32))
        m0 = [b.phase_mass(k) for k in range(len(mem))]
        b.step(args.warmup)
        tx, ty, _ = b.autotune(5)
        l0 = b.kernel_launches
        ms = timed(stream, b.step, args.steps)
        launches = b.kernel_launches - l0
        drift = max(float((np.abs(b.phase_mass(k) - m0[k]) / m0[k]).max()) for k in range(len(mem)))
        ntiles = b.get_tile()[2]
        b.close()
        sims = [Simulation(q, stream=stream) for q, _ in mem]
        for s_, (_, f0) in zip(sims, mem):
            s_.set_phi(f0.astype(np.float32))
            s_.step(args.warmup)
        n_single = max(10, args.steps // 20)
        ms1 = timed(stream, lambda n: [s_.step(1) for _ in range(n) for s_ in sims], n_single)
        for s_ in sims:
            s_.close()
        bpl = bytes_per_lup(3)
        forms["batched"] = {
            "workload": "64 three-phase lens problems (sizes 128x64, 256x128, 512x256 drawn with seed "
                        "2306; lens R = 0.2 height on the 1|2 interface; walls top and bottom; sigma_12 = "
                        "0.01, sigma_13, sigma_23 ~ U[0.005, 0.015]; 32 Model B, 32 Model A with n in "
                        "0.5..4), FP32",
            "nodes": nodes, "value": round(nodes / ms / 1e3, 2), "unit": "MLUPS",
            "ms_per_step": round(ms, 5), "algorithmic_bytes_per_lup": bpl,
            "roofline_frac": round(bpl * nodes / (ms / 1e3) / 1e9 / peak, 4),
            "tile": [tx, ty], "tiles_per_step": ntiles, "gpu_launches": launches,
            "one_launch_per_member_mlups": round(nodes / ms1 / 1e3, 2),
            "mass_drift_rel_max": drift,
        }
        del sims
        torch.cuda.empty_cache()
        forms["rti"] = measure_rti(args, timed, stream, peak)
        forms["adjoint"] = measure_adjoint(timed, 256, peak)
        forms["adjoint_1024"] = measure_adjoint(timed, 1024, peak)
        forms["adjoint_model_A"] = measure_adjoint(timed, 256, peak, model="A")
    return forms


def measure_accuracy_256(args, stream):
    """Error of every population storage against the FP64 oracle on the
    256x256 N = 5 cut of the workload (25 disks, radii U[6, 12], same
    parameter draws, Model B): max |dphi| over all N phases, relative L2
    error of u and the largest per-phase volume drift of the GPU run, after
    a short horizon and after args.accuracy_steps steps, under both
    unit-vector readings (delta = 0, the paper's v/|v| with 0 at v = 0, and
    the smooth v/sqrt(|v|^2 + delta^2) with delta = 1e-3).  The oracle runs
    on the host cores (OpenMP); the GPU runs are untimed."""
    from oracle.oracle import OracleSim, build_oracle, max_threads
    from paper_2306_06983_gb300 import workloads as W
    from paper_2306_06983_gb300.nlbm import Simulation
    build_oracle()
    p, phi0 = W.disks_256(args.model)
    phi0 = phi0.astype(np.float32).astype(np.float64)
    horizons = (25, args.accuracy_steps)
    out = {"workload": "256x256 periodic, N=5, 25 disks radii U[6, 12] (seed 2306), eps=4, M=0.1, "
                       f"Model {args.model}; FP64 oracle on {max_threads()} host threads",
           "steps": list(horizons), "readings": {}}
    t0 = time.perf_counter()
    for delta in (0.0, 1e-3):
        q = dict(p, unit_delta=delta)
        o = OracleSim(q, phi0)
        ref = {}
        done = 0
        for h in horizons:
            o.step(h - done)
            done = h
            ref[h] = o.moments()[:2]
        res = {}
        for st in ("f32", "bf16", "f16"):
            with torch_stream(stream):
                sim = Simulation(dict(q, storage=st), stream=stream)
                sim.set_phi(phi0)
                m0 = sim.phase_mass()
                rows = {}
                done = 0
                for h in horizons:
                    sim.step(h - done)
                    done = h
                    phi, u = (t.cpu().numpy().astype(np.float64) for t in sim.moments()[:2])
                    m = sim.phase_mass(allow_diverged=True)
                    ophi, ou = ref[h]
                    rows[str(h)] = {
                        "max_abs_dphi": float(np.abs(phi - ophi).max()),
                        "u_rel_l2": float(np.sqrt(((u - ou) ** 2).sum() / max((ou ** 2).sum(), 1e-300))),
                        "mass_drift_rel": float((np.abs(m - m0) / np.abs(m0)).max()),
                    }
                sim.close()
            res[st] = rows
        out["readings"][f"unit_delta={delta:g}"] = res
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def torch_stream(stream):
    import torch
    return torch.cuda.stream(stream)


def measure_rti(args, timed, stream, peak):
    """Gravity and walls: the ternary Rayleigh-Taylor instability (Sec. 4.4,
    256 x 1024, rho 3:2:1, F_g = rho g), FP32, one launch per step, timed with
    CUDA events like the headline; with the volume drift over the run."""
    from paper_2306_06983_gb300 import workloads as W
    from paper_2306_06983_gb300.nlbm import Simulation
    p, phi0 = W.rayleigh_taylor(d=256)
    sim = Simulation(p, stream=stream)
    sim.set_phi(phi0.astype(np.float32))
    m0 = sim.phase_mass()
    tile = sim.autotune(20)[:2]
    sim.step(args.warmup)
    l0 = sim.kernel_launches
    ms = timed(stream, sim.step, args.steps)
    launches = sim.kernel_launches - l0
    drift = float((np.abs(sim.phase_mass() - m0) / np.abs(m0)).max())
    sim.close()
    nodes = p["nx"] * p["ny"]
    bpl = bytes_per_lup(3)
    return {
        "workload": "ternary Rayleigh-Taylor instability 256x1024, rho 3:2:1, At 0.5, Re 1000, Ca 0.28, "
                    "sqrt(g d) = 0.04, walls top and bottom, Model B, FP32",
        "nodes": nodes, "value": round(nodes / ms / 1e3, 2), "unit": "MLUPS", "ms_per_step": round(ms, 5),
        "algorithmic_bytes_per_lup": bpl, "roofline_frac": round(bpl * nodes / (ms / 1e3) / 1e9 / peak, 4),
        "gpu_launches": launches, "mass_drift_rel": drift, "tile": list(tile),
    }


def measure_adjoint(timed, n=256, peak=None, model="B"):
    """Gradient study (n x n periodic, 256 by default, N = 3, Model B or A with
    n = 1, 500 steps, a
    checkpoint every 50, smooth unit vectors delta = 1e-3): L = 1/2 |phi(T) -
    phi_hat|^2 with phi_hat from sigma = (0.012, 0.008, 0.010); gradients with
    respect to the three tensions, the mobility and the initial fields from
    sigma = (0.01, 0.01, 0.01).  Forward (with checkpoints) and reverse sweep
    timed with CUDA events (median of three calls after two warm-up calls);
    a plain forward of the same steps beside them."""
    import torch
    from paper_2306_06983_gb300 import workloads as W
    from paper_2306_06983_gb300.nlbm import AdjointRun, Simulation, pair_list
    T, every = 500, 50
    p, phi0 = W.adjoint_problem(n, n)
    p = dict(p, model=model, model_a_n=1.0)
    phi0 = phi0.astype(np.float32)
    N = p["n_phases"]

    def sig(s):
        m = np.zeros((N, N))
        for (a, b), v in zip(pair_list(N), s):
            m[a, b] = m[b, a] = v
        return m.tolist()
    stream = torch.cuda.current_stream()
    ref = Simulation(dict(p, sigma=sig((0.012, 0.008, 0.010))))
    ref.set_phi(phi0)
    ref.step(T)
    tgt = ref.moments()[0]
    ref.close()
    q = dict(p, sigma=sig((0.01, 0.01, 0.01)))
    plain = Simulation(q)
    plain.set_phi(phi0)
    plain.step(3)
    ms_plain = timed(stream, plain.step, T) * T
    plain.close()
    run = AdjointRun(q, T, every)
    # warm-up: the first reverse sweep of a handle loads the kernels and
    # captures the sweep into a CUDA graph (about 0.5 s), and the seed's
    # subtraction loads torch's own kernel; time replays
    for _ in range(2):
        phiT = run.forward(phi0)
        run.backward((phiT - tgt).contiguous())
    l0 = run.kernel_launches
    fwds, bwds = [], []
    for _ in range(3):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(stream)
        phiT = run.forward(phi0)
        e[1].record(stream)
        seed = (phiT - tgt).contiguous()
        g0, gs, gm = run.backward(seed)
        e[2].record(stream)
        torch.cuda.synchronize()
        fwds.append(e[0].elapsed_time(e[1]))
        bwds.append(e[1].elapsed_time(e[2]))
    launches = (run.kernel_launches - l0) // 3
    graph = run.uses_graph
    run.close()
    fwd, bwd = float(np.median(fwds)), float(np.median(bwds))
    nodes = n * n
    ab = adjoint_bytes_per_lup(N)
    roof = None
    if peak:
        gbs = (ab["forward"] + ab["reverse"]) * nodes * T / ((fwd + bwd) / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs / peak, 4), "algorithmic_bytes_per_lup": ab,
                "forward_frac": round(ab["forward"] * nodes * T / (fwd / 1e3) / 1e9 / peak, 4),
                "backward_frac": round(ab["reverse"] * nodes * T / (bwd / 1e3) / 1e9 / peak, 4),
                "note": ("the step's fields (%.0f MB) fit the 129 MB L2: bound by launch and dependency latency, "
                         "not by HBM" % (nodes * 4 * (10 * N + 2) / 1e6)) if nodes * 4 * (10 * N + 2) < 129e6
                else "fields larger than L2"}
    return {
        "workload": f"{n}x{n} periodic N=3 Model {model}{' (n = 1)' if model == 'A' else ''} disks, 500 steps, "
                    "checkpoint every 50, unit vectors "
                    "v/sqrt(|v|^2+1e-6); L2 mismatch of phi(T) against the sigma=(0.012,0.008,0.010) run",
        "value": round(nodes * T / ((fwd + bwd) / 1e3) / 1e6, 2), "unit": "MLUPS (differentiated)",
        "forward_ms": round(fwd, 3), "backward_ms": round(bwd, 3), "backward_over_forward": round(bwd / fwd, 2),
        "plain_forward_ms": round(ms_plain, 3), "gpu_launches": launches,
        "backward_ms_calls": [round(v, 3) for v in bwds], "reverse_sweep_graph": graph,
        "loss": float(0.5 * ((phiT.double() - tgt.double()) ** 2).sum()),
        "grad_sigma_pairs": [float(gs[a, b]) for a, b in pair_list(N)], "grad_mobility": float(gm),
        "grad_phi0_max_abs": float(g0.abs().max()),
        "roofline": roof,
    }


def run_forms_only(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2306_06983_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.lattice:
        lx, ly = args.lattice
        p, phi0 = W.random_disks(lx, ly, 5, max(1, int(round(200 * lx * ly / 2048 ** 2))), 10.0, 40.0,
                                 model=args.model)
    else:
        p, phi0 = W.disks_2048(args.model)
    N = p["n_phases"]
    shape = (N, p["ny"], p["nx"])
    ref = [np.zeros(shape, np.float32), np.zeros((2,) + shape[1:], np.float32)]
    peak, _ = peak_hbm()
    forms = measure_forms(args, p, phi0, ref, p["nx"] * p["ny"], peak)
    for f in forms.values():
        f.pop("vs_f32_after_same_steps", None)
    print(json.dumps({"metric": METRIC, "forms": forms}), flush=True)


def run_adjoint_only(args):
    """Profiling aid: the adjoint form alone on an n x n lattice."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))

    def timed(stream, fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps
    peak, _ = peak_hbm()
    print(json.dumps({"metric": METRIC, "forms": {"adjoint": measure_adjoint(timed, args.only_adjoint, peak)}}),
          flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2306_06983_gb300 import workloads as W
    from paper_2306_06983_gb300.nlbm import Simulation

    if args.lattice:
        lx, ly = args.lattice
        n_disks = max(1, int(round(200 * lx * ly / 2048 ** 2)))
        p, phi0 = W.random_disks(lx, ly, 5, n_disks, 10.0, 40.0, model=args.model)
        workload = f"{lx}x{ly} periodic, N=5, {n_disks} disks (seed 2306), eps=4, M=0.1"
    else:
        p, phi0 = W.disks_2048(args.model)
        workload = WORKLOAD
    p = dict(p, storage=args.storage)
    N, nx, ny = p["n_phases"], p["nx"], p["ny"]
    lups = nx * ny
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = Simulation(p, stream=stream)
        sim.set_phi(phi0.astype(np.float32))
        # tile shape: the library's autotuner (before the warm-up steps; the
        # result of a step does not depend on it), unless --tile fixes it
        if args.tile:
            sim.set_tile(*args.tile)
        else:
            sim.autotune(20)
        stream.synchronize()

        # ---------------------------------------------- device-timed region
        # the K steps are one nlbm_step call: K launches of the fused step
        # kernel back to back on the stream, between two events; every step
        # is one launch, so the region's time / K is the kernel's average
        # launch duration (an event between launches would stop each launch
        # from overlapping the tail of the one before)
        # the clock sampler starts (and waits for nvidia-smi) before the W
        # warm-up steps, so that the GPU is busy right up to the timed region
        e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clocks:
            sim.step(args.warmup)
            launches0 = sim.kernel_launches
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            e_start.record(stream)
            sim.step(args.steps)
            e_end.record(stream)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
        launches = sim.kernel_launches - launches0
        total_ms = e_start.elapsed_time(e_end)
        mass = sim.phase_mass(allow_diverged=True)
        tile = list(sim.get_tile())
        ref_fields = [t.cpu().numpy() for t in sim.moments()[:2]]
        sim.close()

        # ------------------------------------------- end to end, host buffers
        phi_host = torch.from_numpy(phi0.astype(np.float32)).pin_memory()
        out_phi = torch.empty((N, ny, nx), dtype=torch.float32).pin_memory()
        out_u = torch.empty((2, ny, nx), dtype=torch.float32).pin_memory()
        out_p = torch.empty((ny, nx), dtype=torch.float32).pin_memory()
        sim2 = Simulation(p, stream=stream)
        sim2.set_tile(*tile)
        stream.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_l0 = sim2.kernel_launches
        t0 = time.perf_counter()
        e0.record(stream)
        sim2.set_phi_host(phi_host)
        sim2.step(args.steps)
        sim2.moments_host(out_phi, out_u, out_p)
        e2e_mass = sim2.phase_mass(allow_diverged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_launches = sim2.kernel_launches - e2e_l0
        sim2.close()

    total_s = total_ms / 1e3
    total_s, e2e_s = reduce_max_over_ranks([total_s, e2e_s])
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    mlups = whole_job_mlups(world, lups, args.steps, total_s)
    avg_launch_s = total_ms / 1e3 / max(launches, 1)
    bpl = bytes_per_lup(N, args.storage)
    achieved = bpl * lups / avg_launch_s / 1e9
    peak, peak_kind = peak_hbm()
    traffic_bpl = measured_traffic(args.model, args.storage)
    line = {
        "metric": METRIC, "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload + f", Model {args.model}", "nx": nx, "ny": ny,
                   "n_phases": N, "model": args.model, "tile": tile,
                   "population_storage": args.storage,
                   "l2": f"inputs larger than L2 ({bytes_per_lup(N, args.storage) / 2 * nx * ny / 1e6:.0f} MB "
                         f"of state per step vs 129 MB L2); no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": (round(traffic_bpl * lups) if traffic_bpl else None),
                     "kernel": f"step_kernel<NS={N - 1}, MODEL={args.model}, storage={args.storage}>",
                     "algorithmic_bytes_per_lup": bpl,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth",
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "avg_launch_ms": round(avg_launch_s * 1e3, 5)},
        "e2e": {"value": round(whole_job_mlups(world, lups, args.steps, e2e_s), 2), "unit": "MLUPS",
                "h2d_bytes_per_step": round(4 * (N - 1) * lups / args.steps),
                "d2h_bytes_per_step": round((4 * (N + 3) * lups + 8 * N) / args.steps),
                "seconds": round(e2e_s, 4), "gpu_launches": e2e_launches,
                "path": "nlbm_set_phi_host (pinned) + nlbm_step + nlbm_get_moments_host + "
                        "nlbm_phase_mass"},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "mass_after": [float(v) for v in mass],
    }
    if not args.no_forms and world == 1:
        line["forms"] = measure_forms(args, p, phi0, ref_fields, lups, peak)
        for st in ("bf16", "f16", "f32"):
            f = line["forms"].get(st)
            if f is not None and "of_f32_headline" in f:
                f["of_f32_headline"] = round(f["value"] / line["value"], 4) if args.storage == "f32" else None
    if not args.no_cpu_baseline and world == 1:
        from oracle.oracle import build_oracle
        build_oracle()
        mlups_cpu, cores, dt = oracle_sample(args.model, args.cpu_steps, 1)
        line["cpu_baseline"] = {
            "value": round(mlups_cpu, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{args.cpu_steps} time steps of a 512x512 cut of the workload, FP64 "
                      f"oracle, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--model", choices=["A", "B"], default="B")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32",
                    help="population storage: FP32, or 16-bit deviations (FP32 arithmetic)")
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--tile", type=int, nargs=2, default=None, metavar=("TX", "TY"))
    ap.add_argument("--lattice", type=int, nargs=2, default=None, metavar=("NX", "NY"),
                    help="profiling aid: a disk suspension of this size instead of 2048x2048")
    ap.add_argument("--cpu-steps", type=int, default=500,
                    help="oracle steps of the CPU baseline (about 10 s on 16 cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--accuracy-steps", type=int, default=2000,
                    help="long horizon of the 256x256 comparison of every storage with the FP64 oracle")
    ap.add_argument("--no-oracle-accuracy", action="store_true",
                    help="skip the 256x256 comparison with the FP64 oracle among the forms")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the 16-bit storage and ensemble forms measured beside the headline")
    ap.add_argument("--only-forms", action="store_true",
                    help="profiling aid: time only the forms (on --lattice if given), print them")
    ap.add_argument("--only-adjoint", type=int, default=0, metavar="N",
                    help="profiling aid: time only the adjoint form on an N x N lattice, print it")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.only_adjoint:
        run_adjoint_only(args)
    elif args.only_forms:
        run_forms_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
