"""Benchmark of the coupled phi-mu LBM step on one GB300 (or N independent replicas).

Workload: 256^3 synthetic porous medium (Gaussian random field, porosity 0.35,
W = 3, D_l = 0.1, D_s = 0 with anti-trapping, counter term on), D3Q19, FP32
storage and arithmetic.  One "step" is one coupled time step n -> n+1 (the phi
kernel and the composition kernel).  The state (2.6 GB) is far larger than L2.

Prints ONE JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle
on the host cores instead (a deliberately slow baseline, not the target).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled phi-mu LBM MLUPS on 1 GB300, % of HBM roofline; FP32/adjoint vs FP64 fwd"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="side of the cubic domain")
    ap.add_argument("--nz", type=int, default=0, help="planes along z (0: n, a cube); for small profiling cases")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16dev", "bf16dev"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=20, help="steps of the FP64 comparison run")
    ap.add_argument("--dev16-steps", type=int, default=50, help="timed steps of each 16-bit storage run (0 = skip)")
    ap.add_argument("--hvar-steps", type=int, default=100,
                    help="timed steps of each variant of the composition scheme (h on D3Q7, h^eq,alt; 0 = skip)")
    ap.add_argument("--e4-steps", type=int, default=10000,
                    help="steps of the paper's 1024^2 porous experiment, timed in FP64 and FP32 (0 = skip)")
    ap.add_argument("--adj-steps", type=int, default=2000, help="steps of the 128^3 adjoint run (0 = skip)")
    ap.add_argument("--adj-every", type=int, default=100, help="checkpoint interval of the adjoint run")
    ap.add_argument("--batch-steps", type=int, default=40,
                    help="timed steps of the 384-instance 2-D batch (0 = skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int) -> float:
    """The maximum of a per-rank time over all ranks (the job's time): an
    all-reduce over the default process group (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: int, steps: int, world: int, job_ms: float) -> float:
    """Replicas: every rank advances its own copy of the workload, so the job's
    throughput is all ranks' node updates over the slowest rank's time."""
    return world * nodes_per_rank * steps / (job_ms * 1e-3) / 1e6


def dram_throughput(traffic_bytes, kernel_ms, peak_gbs):
    """Actual DRAM throughput of a kernel: its ncu bytes per launch over its mean
    event-timed duration, in GB/s and as a fraction of the peak (None when the
    committed capture does not match the current kernel sources)."""
    if not traffic_bytes or not kernel_ms or kernel_ms <= 0:
        return None
    gbs = traffic_bytes / (kernel_ms * 1e-3) / 1e9
    return {"gbs": gbs, "frac": gbs / peak_gbs}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# sources that define the 3-D step kernels, and the lines of lbpf.cu that fix
# their FP32 tile shape
STEP_SOURCES = ("lattice.cuh", "step_kernels.cuh")
STEP_TILE_MACROS = ("LBPF_BY3", "LBPF_ZCH3", "LBPF_MINB3")


def kernel_source_hash(files=STEP_SOURCES, macros=STEP_TILE_MACROS) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2111_05960_gb300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "lbpf.cu")) as fh:
        for line in fh:
            if line.startswith("#define") and line.split()[1] in macros:
                h.update(line.encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload][kernel]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


def fp64_roofline(stream, nodes, ms_per_step, workload):
    """The FP64 step against the FP64 pipe of this GPU.  Every FP64 add, multiply
    or FMA occupies one FP64 issue slot, so the step's FP64 instructions per
    node (committed ncu count, profiles/fp64_flops.json, while the step-kernel
    sources match) are counted as FMAs (2 flops each) and compared with the FMA
    rate lbpf_fp64_fma_rate measures; arithmetic flops are reported beside."""
    from paper_2111_05960_gb300 import lbpf as L
    peak = L.lbpf_fp64_fma_rate(stream.cuda_stream)
    out = {"bound": "alu", "peak": peak, "unit": "TFLOP/s", "peak_source": "measured (lbpf_fp64_fma_rate)",
           "counting": "FP64 pipe instructions x 2 (FMA-equivalent)", "achieved": None, "frac": None}
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_flops.json")) as f:
            d = json.load(f)
        if d.get("source_hash") == kernel_source_hash(STEP_SOURCES, ("LBPF_BY3_F64", "LBPF_ZCH3_F64", "LBPF_MINB3_F64")):
            ipn = float(d["fp64_instructions_per_node"])
            ach = 2.0 * ipn * nodes / (ms_per_step * 1e-3) / 1e12
            out.update({"achieved": ach, "frac": ach / peak, "fp64_instructions_per_node": ipn,
                        "arithmetic_tflops": float(d["flops_per_node"]) * nodes / (ms_per_step * 1e-3) / 1e12})
    except Exception:
        pass
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for n, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(n, nz=0):
    from paper_2111_05960_gb300 import workloads as WL
    return WL.porous_3d(n=n, nz=nz or None)


def workload_config(model):
    """The workload both arms run, by what it is (the same dict for the GPU arm
    and the oracle arm; the arithmetic type is the line's dtype)."""
    size = "%d" % model.nx if model.nz == model.nx else "%dx%dx%d" % (model.nx, model.ny, model.nz)
    return {"workload": "porous_3d_%s_d3q19" % size, "nodes": model.nodes, "lattice": "D3Q19",
            "porosity": 0.35, "W": model.W, "D_l": model.D_l, "D_s": model.D_s,
            "counter_term": model.counter_term, "anti_trapping": model.anti_trapping,
            "boundaries": "periodic", "inputs": "seeded Gaussian-random-field medium (PCG64 seed 0)"}


def algorithmic_bytes(q: int, real: int, store: int):
    """Bytes per node of each kernel: populations read once and written once, phi^n
    read and phi^{n+1} written by the phi kernel (mu is recomputed from c and phi)."""
    phi_kernel = 2 * q * store + 2 * real
    c_kernel = 2 * q * store
    return phi_kernel, c_kernel


def batch_measurement(args, stream, hbm):
    """The 384-instance 2-D sweep (sizes 64..768, 1-8 discs, random D_l and
    M_phi/D_l, counter term on or off), FP32, stepped as one batch: one
    persistent launch per kernel phase over row-marched tiles whose shape the
    library's autotuner picked at creation, two steps per replayed CUDA graph."""
    import torch
    from paper_2111_05960_gb300 import lbpf as L
    from paper_2111_05960_gb300 import workloads as WL
    inst = WL.batch_2d(count=384, seed=1)
    b = L.BatchSimulation([x.params for x in inst], [x.phi for x in inst], [x.c for x in inst],
                          precision="fp32", stream=stream.cuda_stream)
    nodes = b.nodes
    b.step(6)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.batch_steps
    k_phi, k_c, _ = b.step_timed(10)
    tile, tune_ms = b.tile()
    b.close()
    bytes_node = 2 * 9 * 4 + 2 * 4 + 2 * 9 * 4     # phi kernel 80 B, composition kernel 72 B
    gbs = bytes_node * nodes / (ms * 1e-3) / 1e9
    return {"workload": "batch_2d_384_d2q9_fp32", "instances": 384, "nodes": nodes, "steps": args.batch_steps,
            "tile": {"shape": list(tile), "autotune_ms_per_step": dict(zip(["%dx%d" % t for t in L.BATCH_TILES], [float(v) for v in tune_ms]))},
            "ms_per_step": ms, "mlups": nodes / (ms * 1e-3) / 1e6, "bytes_per_node": bytes_node,
            "achieved_gbs": gbs, "frac": gbs / hbm, "launch": "2 persistent launches per step (all 384 instances are periodic; walled instances would add 2), CUDA graph",
            "kernel_ms": {"k_batch_phi": k_phi / 10, "k_batch_c": k_c / 10}}


# Algorithmic bytes per node of one reversed step (FP32, D3Q19): k_adj_h reads h,
# gathers hb and writes hb (3 x 76), reads phi, c, phi^{n+1}, cb, phib (20) and
# writes seven work values (28); k_adj_g reads g, gathers gb, writes gb (228),
# reads phi, c and five work values (28), updates the grad adjoint (24) and
# writes the phi and c adjoints (8); k_adj_finish reads the grad adjoint (12)
# and updates the phi adjoint (8).
ADJ_BYTES_PER_NODE_FP32 = 276 + 288 + 20


def adjoint_measurement(args, stream, hbm, fwd_bytes_per_node):
    """The differentiable 3-D workload: 128^3 porous medium (porosity 0.4), FP32
    with the FP64 mass correction, T steps recorded every k, the slab
    solid-fraction loss (workloads.slab_loss).  Times the forward steps and the whole reverse sweep
    (checkpoint restores, segment replays and three adjoint kernels per step)
    with CUDA events on the context's stream; seed and outputs stay on the GPU."""
    import torch
    from paper_2111_05960_gb300 import lbpf as L
    from paper_2111_05960_gb300 import workloads as WL
    m, phi0, c0, target = WL.differentiable_3d(128)
    N, T, K = m.nodes, args.adj_steps, args.adj_every
    sim = L.Simulation(m, phi0, c0, precision="fp32", stream=stream.cuda_stream, mass_every=1,
                       checkpoint_every=K)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    sim.step(T)
    ev[1].record(stream)
    phi = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    L.lbpf_get_fields(sim.ctx, phi, None, None, 1)
    with torch.cuda.stream(stream):
        loss, seed = WL.slab_loss(phi, torch.tensor(target, dtype=torch.float64, device="cuda"))
        dphi0 = torch.empty_like(phi)
        dc0 = torch.empty_like(phi)
    torch.cuda.synchronize()
    ev[2].record(stream)
    pv = L.lbpf_adjoint_step(sim.ctx, seed, None, dphi0, dc0, 1)
    ev[3].record(stream)
    torch.cuda.synchronize()
    sim.close()
    fwd_ms = ev[0].elapsed_time(ev[1]) / T
    sweep_ms = ev[2].elapsed_time(ev[3]) / T
    rev_ms = max(sweep_ms - fwd_ms, 1e-9)        # the replay runs the forward kernels again
    gbs = ADJ_BYTES_PER_NODE_FP32 * N / (rev_ms * 1e-3) / 1e9
    return {"workload": "differentiable_3d_128_d3q19_fp32", "nodes": N, "steps": T, "checkpoint_every": K,
            "loss": loss, "forward_ms_per_step": fwd_ms, "adjoint_sweep_ms_per_step": sweep_ms,
            "adjoint_to_forward": sweep_ms / fwd_ms,
            "reverse_kernels_ms_per_step": rev_ms,
            "reverse_bytes_per_node": ADJ_BYTES_PER_NODE_FP32,
            "reverse_achieved_gbs": gbs, "reverse_frac": gbs / hbm,
            "ideal_adjoint_to_forward": (ADJ_BYTES_PER_NODE_FP32 + fwd_bytes_per_node) / fwd_bytes_per_node,
            "dL_dparams": dict(zip(L.ADJ_PARAM_NAMES, [float(v) for v in pv])),
            "dL_dM_phi": 3.0 * float(pv[1]),
            "max_abs_dL_dphi0": float(dphi0.abs().max()),
            "note": "sweep = checkpoint restores + replay of every segment + reverse kernels; "
                    "reverse kernels = sweep - forward (the replay is the forward's kernels)"}


PAPER_E4_V100_SECONDS = 70.0     # Sec. 5: 10^4 steps of the 1024^2 experiment on one V100


def paper_e4_measurement(args, stream):
    """The dissolution experiment of Sec. 5 (1024^2 D2Q9, W ~ 20 nodes,
    lambda* = 230, anti-trapping, zero-flux walls) on a synthetic porous slice,
    with and without the counter term: seconds for the paper's 10^4 steps in
    FP64 and in FP32 (with the mass correction), CUDA events around the steps,
    fields resident on the GPU.  The paper's code took 70 s on a V100 (context:
    another GPU, another code, an unknown precision)."""
    import torch
    from paper_2111_05960_gb300 import lbpf as L
    from paper_2111_05960_gb300 import workloads as WL
    out = {"workload": "paper_e4_2d_1024_d2q9", "steps": args.e4_steps, "paper_v100_seconds": PAPER_E4_V100_SECONDS}
    for prec in ("fp64", "fp32"):
        for ct in (1, 0):
            m, phi0, c0 = WL.paper_e4_2d(counter_term=ct)
            sim = L.Simulation(m, phi0, c0, precision=prec, stream=stream.cuda_stream,
                               mass_every=1 if prec == "fp32" else 0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(args.e4_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            sim.close()
            key = "%s_%s" % (prec, "counter_term" if ct else "no_counter_term")
            out[key] = {"seconds": sec, "mlups": m.nodes * args.e4_steps / sec / 1e6,
                        "speedup_vs_paper": PAPER_E4_V100_SECONDS * args.e4_steps / 1e4 / sec}
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
        import platform
        return platform.machine()
    except Exception:
        return "unknown"


def cpu_baseline(model, phi0, c0, budget_s=12.0, single_s=3.0):
    """The FP64 oracle, as it stands, on a z-slab of the same medium (periodic):
    on all host cores (OpenMP) for ~budget_s, and on one core for ~single_s."""
    import oracle as O
    names = O.OracleParams.__dataclass_fields__
    nz = 16
    sub_phi = np.ascontiguousarray(phi0[:nz])
    sub_c = np.ascontiguousarray(c0[:nz])
    p = O.OracleParams(**{k: getattr(model, k) for k in names})
    p.nz = nz
    nodes = p.nx * p.ny * nz

    def timed(budget):
        o = O.Oracle(p, sub_phi, sub_c)
        t = time.perf_counter()
        o.step(1)
        one = time.perf_counter() - t
        steps = max(1, int(budget / max(one, 1e-3)))
        t = time.perf_counter()
        o.step(steps)
        return steps, time.perf_counter() - t

    threads = O.Oracle.threads()
    steps, el = timed(budget_s)
    O.Oracle.set_threads(1)
    steps1, el1 = timed(single_s)
    O.Oracle.set_threads(threads)
    try:
        other = oracle_other_configs()
    except Exception as ex:   # context only: never sinks the main baseline
        O.Oracle.set_threads(threads)
        other = {"error": str(ex)}
    return {"value": nodes * steps / el / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": "%dx%dx%d z-slab of the 256^3 medium, %d FP64 steps, %.1f s" % (p.nx, p.ny, nz, steps, el),
            "single_core_value": nodes * steps1 / el1 / 1e6, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "other_configs": other}


def oracle_other_configs(budget_s=1.5):
    """The oracle, as it stands, on the other workloads, on all host cores and on
    one: the 512^2 disc (counter term on) and, for the batch sweep, its smallest,
    median and largest instance (each timed alone, ~budget_s)."""
    import oracle as O
    from paper_2111_05960_gb300 import workloads as WL
    names = O.OracleParams.__dataclass_fields__

    def rate(model, phi0, c0, budget):
        o = O.Oracle(O.OracleParams(**{k: getattr(model, k) for k in names}), phi0, c0)
        t = time.perf_counter()
        o.step(1)
        steps = max(1, int(budget / max(time.perf_counter() - t, 1e-3)))
        t = time.perf_counter()
        o.step(steps)
        return model.nodes * steps / (time.perf_counter() - t) / 1e6

    threads = O.Oracle.threads()
    out = {}
    m, phi0, c0 = WL.disc_2d(n=512, counter_term=1)
    out["disc_2d_512"] = {"mlups": rate(m, phi0, c0, budget_s)}
    O.Oracle.set_threads(1)
    out["disc_2d_512"]["single_core_mlups"] = rate(m, phi0, c0, budget_s)
    O.Oracle.set_threads(threads)
    inst = WL.batch_2d(count=384, seed=1)
    order = sorted(range(len(inst)), key=lambda i: inst[i].params.nodes)
    sweep = {}
    for i in (order[0], order[len(order) // 2], order[-1]):
        x = inst[i]
        sweep["%dx%d" % (x.params.nx, x.params.ny)] = rate(x.params, x.phi, x.c, budget_s / 2)
    out["batch_2d_instance_sweep_mlups"] = sweep
    out["cores"] = threads
    return out


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on the same workload and the full grid,
    on the host cores: W untimed warm-up steps, then K timed steps; value and
    ms_per_step are those of the timed steps on the whole grid."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    model, phi0, c0 = make_workload(args.n, args.nz)
    import oracle as O
    O.build()
    names = O.OracleParams.__dataclass_fields__
    p = O.OracleParams(**{k: getattr(model, k) for k in names})
    o = O.Oracle(p, phi0, c0)
    if args.warmup > 0:
        o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t
    nodes = model.nodes
    mlups = nodes * args.steps / el / 1e6
    cores = O.Oracle.threads()
    out = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(model), "parallelism": "%d host threads (OpenMP)" % cores,
           "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                            "sample": "the whole %dx%dx%d grid, %d FP64 steps after %d warm-up steps, %.1f s"
                                      % (p.nx, p.ny, p.nz, args.steps, args.warmup, el),
                            "cpu_model": cpu_model()},
           "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def compact_legs(out):
    """The headline numbers of each optional leg, rounded, in one small dict."""
    def g(d, *path):
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return round(d, 4) if isinstance(d, float) else d
    r = out.get("roofline") or {}
    legs = {"step_glups": g(out, "value") and round(out["value"] / 1e3, 3),
            "k_c_step_frac": g(r, "frac") if r.get("kernel") == "k_c_step" else None,
            "kernel_ms": {k: round(v, 4) for k, v in (r.get("kernel_ms") or {}).items()},
            "step_frac": g(r, "step", "frac"),
            "fp64_glups": g(out, "fp64_forward", "mlups") and round(out["fp64_forward"]["mlups"] / 1e3, 3),
            "fp32_over_fp64": g(out, "fp64_forward", "fp32_speedup"),
            "fp64_alu_frac": g(out, "fp64_forward", "roofline", "frac"),
            "batch_2d_glups": g(out, "batch_2d", "mlups") and round(out["batch_2d"]["mlups"] / 1e3, 3),
            "batch_2d_frac": g(out, "batch_2d", "frac"),
            "adjoint_to_forward": g(out, "adjoint", "adjoint_to_forward"),
            "adjoint_reverse_frac": g(out, "adjoint", "reverse_frac"),
            "e2e_glups": g(out, "e2e", "value") and round(out["e2e"]["value"] / 1e3, 3),
            "paper_e4_fp32_seconds": g(out, "paper_e4", "fp32_counter_term", "seconds")}
    for p16 in ("fp16dev", "bf16dev"):
        legs[p16 + "_glups"] = g(out, "dev16", p16, "mlups") and round(out["dev16"][p16]["mlups"] / 1e3, 3)
        legs[p16 + "_step_frac"] = g(out, "dev16", p16, "step_frac")
    for hv in ("h_d3q7", "h_eq_alt"):
        legs[hv + "_glups"] = g(out, "h_variants", hv, "mlups") and round(out["h_variants"][hv]["mlups"] / 1e3, 3)
    legs["h_d3q7_k_c_step_frac"] = g(out, "h_variants", "h_d3q7", "k_c_step_frac")
    return legs


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2111_05960_gb300 import build as B
    from paper_2111_05960_gb300 import lbpf as L
    B.build()
    L.load()

    model, phi0, c0 = make_workload(args.n, args.nz)
    N = model.nodes
    stream = torch.cuda.Stream()
    prec = args.precision
    # FP32 and 16-bit storage hold the solute mass with the FP64 correction every step
    mass_every = 0 if prec == "fp64" else 1
    sim = L.Simulation(model, phi0, c0, precision=prec, stream=stream.cuda_stream, lattice=L.LBPF_D3Q19,
                       mass_every=mass_every)
    q = 19
    real = 8 if prec == "fp64" else 4
    store = {"fp64": 8, "fp32": 4, "fp16dev": 2, "bf16dev": 2}[prec]

    sim.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m_before, m_target = sim.solute_mass()
    barrier()
    # the timed region: the product call, lbpf_step (K steps queued on the
    # library's stream, replayed from the captured two-step graph), bracketed by
    # two events on that stream
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    # the per-kernel split of the same steps (events around every launch,
    # lbpf_step_timed), taken right after the timed region for the roofline
    k_phi_ms, k_c_ms, k_corr_ms = sim.step_timed(args.steps)
    m_c, m_phi = sim.mass()
    m_after, _ = sim.solute_mass()
    sim.close()

    ms_per_step = ms / args.steps
    mlups = whole_job_mlups(N, args.steps, world, ms)
    hbm, hbm_src = peaks()
    b_phi, b_c = algorithmic_bytes(q, real, store)
    avg_phi = k_phi_ms / args.steps
    avg_c = k_c_ms / args.steps
    dom = ("k_phi_step", avg_phi, b_phi) if avg_phi >= avg_c else ("k_c_step", avg_c, b_c)
    achieved = dom[2] * N / (dom[1] * 1e-3) / 1e9
    step_bytes = (b_phi + b_c) * N
    wl = "porous_3d_%d_d3q19_%s" % (args.n, prec)
    roof = {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback",
            "traffic": ncu_traffic(dom[0], wl),
            "traffic_throughput": dram_throughput(ncu_traffic(dom[0], wl), dom[1], hbm),
            "bytes_per_node": dom[2],
            "step": {"achieved": step_bytes / (ms_per_step * 1e-3) / 1e9,
                     "frac": step_bytes / (ms_per_step * 1e-3) / 1e9 / hbm, "bytes_per_node": b_phi + b_c},
            "kernel_ms": {"k_phi_step": avg_phi, "k_c_step": avg_c,
                          "mass_correction": k_corr_ms / args.steps},
            "kernel_timing": "CUDA events around each launch on the library's stream (lbpf_step_timed), "
                             "%d steps right after the timed region" % args.steps}

    extra = {}
    # FP64 forward on the same GPU, for the FP32/FP64 ratio the metric asks for
    if prec == "fp32" and args.fp64_steps > 0:
        try:
            sim64 = L.Simulation(model, phi0, c0, precision="fp64", stream=stream.cuda_stream, lattice=L.LBPF_D3Q19)
            sim64.step(2)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim64.step(args.fp64_steps)
            b.record(stream)
            torch.cuda.synchronize()
            ms64 = a.elapsed_time(b) / args.fp64_steps
            sim64.close()
            extra["fp64_forward"] = {"ms_per_step": ms64, "mlups": N / (ms64 * 1e-3) / 1e6,
                                     "fp32_speedup": ms64 / ms_per_step,
                                     "roofline": fp64_roofline(stream, N, ms64, wl.replace("_fp32", "_fp64"))}
        except Exception as ex:   # reported, never silently dropped
            extra["fp64_forward"] = {"error": str(ex)}

    # the 16-bit deviation-storage variants of the same step, for context
    if prec == "fp32" and args.dev16_steps > 0:
        try:
            dev = {}
            for p16 in ("fp16dev", "bf16dev"):
                s16 = L.Simulation(model, phi0, c0, precision=p16, stream=stream.cuda_stream, lattice=L.LBPF_D3Q19,
                                   mass_every=1)
                s16.step(3)
                torch.cuda.synchronize()
                a16, b16 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a16.record(stream)
                kp, kc, kr = s16.step_timed(args.dev16_steps)
                b16.record(stream)
                torch.cuda.synchronize()
                ms16 = a16.elapsed_time(b16) / args.dev16_steps
                m0, tgt = s16.solute_mass()
                s16.close()
                bp, bc = algorithmic_bytes(q, 4, 2)
                dev[p16] = {"ms_per_step": ms16, "mlups": N / (ms16 * 1e-3) / 1e6,
                            "step_frac": (bp + bc) * N / (ms16 * 1e-3) / 1e9 / hbm, "bytes_per_node": bp + bc,
                            "kernel_ms": {"k_phi_step": kp / args.dev16_steps, "k_c_step": kc / args.dev16_steps},
                            "mass_drift": (m0 - tgt) / tgt}
            extra["dev16"] = dev
        except Exception as ex:   # reported, never silently dropped
            extra["dev16"] = {"error": str(ex)}

    # the two variants of the composition scheme of Sec. 3 on the same workload:
    # h on D3Q7 (fewer bytes per node) and the alternative equilibrium h^eq,alt
    if prec == "fp32" and args.hvar_steps > 0:
        try:
            import dataclasses
            hv = {}
            for name, hl, alt in (("h_d3q7", 1, 0), ("h_eq_alt", 0, 1), ("h_d3q7_eq_alt", 1, 1)):
                mv = dataclasses.replace(model, h_lattice=hl, h_eq_alt=alt)
                sv = L.Simulation(mv, phi0, c0, precision="fp32", stream=stream.cuda_stream, lattice=L.LBPF_D3Q19,
                                  mass_every=1)
                sv.step(3)
                torch.cuda.synchronize()
                av, bv = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                av.record(stream)
                kp, kc, kr = sv.step_timed(args.hvar_steps)
                bv.record(stream)
                torch.cuda.synchronize()
                msv = av.elapsed_time(bv) / args.hvar_steps
                m0, tgt = sv.solute_mass()
                sv.close()
                qh = 7 if hl else 19
                bp, bc = 2 * q * 4 + 2 * 4, 2 * qh * 4
                kcm = kc / args.hvar_steps
                hv[name] = {"h_lattice": "D3Q7" if hl else "D3Q19", "h_eq_alt": alt,
                            "ms_per_step": msv, "mlups": N / (msv * 1e-3) / 1e6,
                            "bytes_per_node": bp + bc, "step_frac": (bp + bc) * N / (msv * 1e-3) / 1e9 / hbm,
                            "k_c_step_frac": bc * N / (kcm * 1e-3) / 1e9 / hbm,
                            "kernel_ms": {"k_phi_step": kp / args.hvar_steps, "k_c_step": kcm},
                            "speedup_vs_main": ms_per_step / msv, "mass_drift": (m0 - tgt) / tgt}
            extra["h_variants"] = hv
        except Exception as ex:   # reported, never silently dropped
            extra["h_variants"] = {"error": str(ex)}

    e4 = None
    if args.e4_steps > 0 and prec == "fp32":
        try:
            e4 = paper_e4_measurement(args, stream)
        except Exception as ex:   # reported, never silently dropped
            e4 = {"error": str(ex)}

    batch = None
    if args.batch_steps > 0 and prec == "fp32":
        try:
            batch = batch_measurement(args, stream, hbm)
        except Exception as ex:   # reported, never silently dropped
            batch = {"error": str(ex)}

    adj = None
    if args.adj_steps > 0 and prec == "fp32":
        try:
            adj = adjoint_measurement(args, stream, hbm, b_phi + b_c)
            if "ms_per_step" in extra.get("fp64_forward", {}):
                # per node: the sweep runs on 128^3, the FP64 forward on the main grid
                adj["adjoint_to_fp64_forward_per_node"] = (adj["adjoint_sweep_ms_per_step"] / adj["nodes"]) / \
                    (extra["fp64_forward"]["ms_per_step"] / N)
        except Exception as ex:   # reported, never silently dropped
            adj = {"error": str(ex)}

    e2e = None
    if not args.no_e2e:
        # end to end through the public API with host buffers: create from pinned host
        # fields (H2D inside), K steps each followed by the FP64 mass read (D2H), and the
        # final fields read back to pinned host memory
        hphi = torch.from_numpy(np.ascontiguousarray(phi0)).pin_memory().numpy()
        hc = torch.from_numpy(np.ascontiguousarray(c0)).pin_memory().numpy()
        out_phi = torch.empty(phi0.shape, dtype=torch.float64).pin_memory().numpy()
        out_c = torch.empty(phi0.shape, dtype=torch.float64).pin_memory().numpy()
        barrier()
        t0 = time.perf_counter()
        s2 = L.Simulation(model, hphi, hc, precision=prec, stream=stream.cuda_stream, lattice=L.LBPF_D3Q19,
                          mass_every=mass_every)
        for _ in range(args.steps):
            s2.step(1)
            s2.mass()
        L.lbpf_get_fields(s2.ctx, out_phi, out_c, None, 0)
        barrier()
        el = time.perf_counter() - t0
        s2.close()
        el = max_over_ranks(el, world)
        e2e = {"value": whole_job_mlups(N, args.steps, world, el * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": 2 * N * 8 / args.steps,
               "d2h_bytes_per_step": (2 * N * 8) / args.steps + 16,
               "includes": "create from host fields, K x (step + FP64 mass read), final phi and c read"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(model, phi0, c0)
        except Exception as ex:  # the baseline must not sink the GPU line
            cpu = {"value": None, "error": str(ex)}

    if rank == 0:
        out = {"metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f32 (f16 deviation storage)",
                         "bf16dev": "f32 (bf16 deviation storage)"}[prec],
               "data": "synthetic",
               "config": workload_config(model),
               "parallelism": "replicas" if world > 1 else "single GPU",
               "l2": "state %.1f GB per buffer set, larger than L2 (no flush needed)"
                     % (N * (2 * q * store + 2 * real) / 1e9),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "batch_2d": batch, "adjoint": adj, "paper_e4": e4,
               "gpu_launches": (4 if mass_every else 2) * args.steps, "clocks": clk,
               "mass": {"solute_before": m_before, "solute_after": m_after,
                        "relative_drift": (m_after - m_before) / m_before,
                        "correction": "FP64, every step" if mass_every else "off",
                        "sum_c_field": m_c, "sum_phi": m_phi}}
        out.update(extra)
        # compact figures of every leg, last on the line so that a reader that
        # keeps only the end of the output still has them
        out["legs"] = compact_legs(out)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
