#!/usr/bin/env python3
"""Benchmark of the fused lattice Boltzmann warm-plasma step on GB300.

Default workload: 2D Cartesian (z, x) LB at 1024 x 512 nodes (dx = 0.05
k_p^-1), local-equilibrium closure (D = 3, k_B T / m c^2 = 1e-2), Gaussian
driver n_b/n_0 = 0.1, sigma_z = 1, sigma_r = 0.5 k_p^-1, C = 0.1, tau = 0.53,
FP32 population storage.  One step = one launch of the fused
collide-stream-field kernel over the whole grid.  The metric is MLUPS (node
updates per second, all population sets plus the field update) and the
fraction of the measured HBM copy bandwidth that the step kernel's
algorithmic bytes reach.

Timing: W untimed steps, then K steps, each bracketed by CUDA events on the
stream the kernel is launched on; L2 is flushed between timed steps (a 256 MiB
write, then a 256 MiB read, so no dirty lines drain inside the timed step),
outside the events.  Under torchrun every rank runs its own replica of
the workload; value = all ranks' node updates / the slowest rank's time.

--impl reference times the FP64 CPU oracle on the host cores on the same
workload (bounded sample) and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline per closure/precision; adjoint cost ratio vs forward"

WORKLOAD_2D = dict(dim=2, n=(1024, 512), dx=0.05, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-2,
                   alpha=0.1, sigma_z=1.0, sigma_r=0.5, z0=4.0, boundary="open", init_fields=True)
WORKLOAD_NAME = "2d_lec_1024x512_fp32"
# step kernel of each lbpwfa_info kernel_variant
KERNEL_NAMES = {1: "lb_step_kernel", 2: "lb_step_tma2d_kernel", 3: "lb_step_persist2d_kernel",
                4: "lb_step_march3d_kernel", 5: "lb_step_axi_kernel"}

# the 1D configuration (launch-bound, 0.2 MB of state: reported as steps/s)
CONFIG_1D = dict(dim=1, n=(2048,), dx=40 / 2048, courant=0.5, tau=0.52, closure="lec", dv=1, mu=1e-3,
                 alpha=0.01, sigma_z=1.0, z0=-5.0, boundary="open")
# the 3D configuration: 512 (z) x 256 x 256, warm-plasma closure
CONFIG_3D = dict(dim=3, n=(512, 256, 256), dx=0.05, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=1e-2,
                 alpha=1.0, sigma_z=0.7, sigma_r=0.3, z0=2.8, boundary="open", init_fields=True)
# the adjoint configuration: 2D 512 (z) x 256 (x) WARMC, 1000 steps, J = E_z on
# axis at 4 k_p^-1 behind the driver centre at the end
CONFIG_ADJ = dict(dim=2, n=(512, 256), dx=0.05, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=5e-3,
                  alpha=0.1, sigma_z=1.0, sigma_r=0.5, z0=4.0, boundary="open", init_fields=True)
ADJ_STEPS = 1000
# the 3D3V axisymmetric configuration of Sec. 6 (Fig. 4): L_z = 30, L_r = 6 at
# dz = dr = 0.01 (3000 x 600 nodes), dt = 0.001, tau = 0.53, mu = 0.04 (20 keV),
# sigma_z = sigma_r = 25 um at n_i = 1e16 cm^-3 (0.47 k_p^-1), Q~ = 0.5
# (alpha = Q~ / ((2 pi)^{3/2} sigma_z sigma_r^2))
CONFIG_AXI = dict(dim=2, n=(3000, 600), dx=0.01, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=0.04,
                  alpha=0.5 / ((2 * np.pi) ** 1.5 * 0.47 ** 3), sigma_z=0.47, sigma_r=0.47, z0=4.0,
                  boundary="open", init_fields=True, geometry="axisymmetric")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp32c", "fp16s"])
    ap.add_argument("--workload", default="2d_lec",
                    choices=["2d_lec", "2d_warmc", "3d_warmc", "3d_warmc_128", "3d_warmc_64", "adjoint_2d_warmc",
                             "batch_2d", "axi_warmc", "axi_lec"],
                    help="2d_lec: 1024 x 512 LEC (default); 2d_warmc: the same grid with the warm-plasma "
                         "closure; 3d_warmc: 512 x 256 x 256 WARMC; "
                         "3d_warmc_128, 3d_warmc_64: 128^3 and 64^3 WARMC (small cases for profiling); "
                         "adjoint_2d_warmc: "
                         "forward + reverse sweep of the 512 x 256 WARMC adjoint case over --steps steps "
                         "(whole tape kept), for profiling; batch_2d: the first --batch-runs runs of the batched "
                         "sweep over --steps steps, for profiling; axi_warmc, axi_lec: the 3000 x 600 "
                         "axisymmetric (z, r) grid of the paper's 3D3V runs")
    ap.add_argument("--batch-runs", type=int, default=64, help="batch_2d: runs of the sweep (1..64)")
    ap.add_argument("--no-tune", action="store_true", help="batch_2d: skip the tile autotuner")
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="0: automatic (2D LEC: persistent TMA CTAs in FP32 and FP16S, a TMA box per CTA "
                         "in FP64; 3D: marching columns), 1: plain global-memory pull kernel (3D: 32 x 4 x 4 "
                         "tiles), 2: TMA box per CTA, 3: persistent CTAs that refill their TMA box after the "
                         "decode phase, 4: 3D marching columns")
    ap.add_argument("--no-modes", action="store_true", help="skip the per-precision mode table")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 1D and 3D configuration measurements")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint cost and gradient check")
    return ap.parse_args()


def _config_block(cfg, precision, extra=None):
    grid = "x".join(str(v) for v in cfg["n"])
    kind = "axi" if cfg.get("geometry") == "axisymmetric" else f"{cfg['dim']}d"
    d = {"workload": f"{kind}_{cfg['closure']}_{grid}_{precision}",
         "grid": list(cfg["n"]), "dx": cfg["dx"], "courant": cfg["courant"], "tau": cfg["tau"],
         "closure": cfg["closure"], "D": cfg["dv"], "mu": cfg["mu"], "alpha": cfg["alpha"],
         "sigma_z": cfg["sigma_z"], "sigma_r": cfg["sigma_r"], "precision": precision,
         "l2": "flushed between timed steps (256 MiB write, then 256 MiB read)", "parallelism": "replicas"}
    if extra:
        d.update(extra)
    return d


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.device), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        time.sleep(0.15)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        load = [r for r in rows if r["util"] >= 50] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(load)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _time_steps(run, stream, steps, warmup, flush):
    """Per-step CUDA events on the launch stream.  Between timed steps L2 is
    flushed by writing one 256 MiB buffer and then reading another, so the
    timed step finds its inputs in HBM and no dirty flush lines left in L2."""
    import torch
    wbuf, rbuf, sink = flush
    # the flush kernels once before the warm-up steps: their first use loads
    # them, and inside the timed loop that host delay would leave the GPU idle
    # between a step's start event and its launch
    with torch.cuda.stream(stream):
        wbuf.fill_(0)
        torch.amax(rbuf, dim=0, out=sink)
    torch.cuda.synchronize()
    for _ in range(warmup):
        run.step(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        with torch.cuda.stream(stream):
            wbuf.fill_(k & 0xFF)
            torch.amax(rbuf, dim=0, out=sink)
        ev[k][0].record(stream)
        run.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]  # ms


def _traffic_for(kernel_key):
    """Per-launch DRAM bytes of the step kernel from a committed ncu summary
    (a `traffic <kernel:workload> <bytes> sources_sha256=<digest>` line under
    profiles/), valid only while the kernel sources are unchanged."""
    import glob
    import re
    try:
        from paper_2309_04872_gb300 import build as B
        digest = B.step_kernel_digest()
        for fn in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
            for m in re.finditer(r"traffic (\S+) (\d+) sources_sha256=([0-9a-f]+)", open(fn).read()):
                if m.group(1) == kernel_key and m.group(3) == digest:
                    return int(m.group(2))
    except OSError:
        pass
    return None


def _oracle_sample(cfg, budget_s=15.0):
    import oracle as O
    o = O.Oracle(cfg)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    nsteps = max(1, int(budget_s / max(t1, 1e-6)))
    nsteps = min(nsteps, 200)
    t0 = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t0
    ncell = 1
    for v in cfg["n"]:
        ncell *= v
    return ncell * nsteps / dt / 1e6, nsteps, dt


def _slowest_rank_seconds(local_s, world, device):
    """The timed region's length over all ranks: a barrier, then the maximum
    of the ranks' times (the only collective; none on the data path)."""
    if world <= 1:
        return local_s
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_s], device=device, dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _aggregate_mlups(ncell_per_rank, steps, world, seconds):
    """Whole-job node updates per second (MLUPS): every rank advances its own
    replica (or shard) by `steps` steps of ncell_per_rank nodes."""
    return ncell_per_rank * steps * world / seconds / 1e6


def _batch_shard(nruns, rank, world):
    """Indices of the batched sweep's runs that rank `rank` of `world` owns:
    whole runs, round-robin, so the ranks exchange nothing."""
    return list(range(rank, nruns, world))


def _batch_cfgs(nruns):
    """The first nruns of the batched sweep's 64 seeded draws, as run
    configurations."""
    from tests import inputs
    draws = inputs.batch_draws(64, seed=2309)[:nruns]
    cfgs = [dict(dim=2, n=(d["nz"], d["nx"]), dx=0.05, courant=0.1, tau=0.53, closure=d["closure"], dv=3,
                 mu=d["mu"], alpha=d["alpha"], sigma_z=d["sigma_z"], sigma_r=0.5, z0=4.0 * d["sigma_z"],
                 boundary="open", init_fields=True) for d in draws]
    return draws, cfgs


def run_batch_case(a):
    """--warmup then --steps batched steps of the sweep's first --batch-runs
    runs (FP32); prints the timing as one JSON line.  Under torchrun each
    rank advances its own shard of whole runs (no data-path collective) and
    rank 0 reports the whole job."""
    import torch
    import torch.distributed as dist

    from paper_2309_04872_gb300 import lbpwfa as lb
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    lb.load_library()
    draws, cfgs = _batch_cfgs(max(1, min(64, a.batch_runs)))
    mine = _batch_shard(len(cfgs), rank, world)
    draws = [draws[i] for i in mine]
    cfgs = [cfgs[i] for i in mine]
    stream = torch.cuda.Stream()
    with lb.Batch(cfgs, "fp32", stream=stream.cuda_stream, tune=not a.no_tune) as b:
        info = b.info()
        b.step(a.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(a.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        seconds = e0.elapsed_time(e1) * 1e-3
    seconds = _slowest_rank_seconds(seconds, world, torch.device("cuda", local))
    nodes = torch.tensor([float(info.ncell)], dtype=torch.float64, device=torch.device("cuda", local))
    if world > 1:
        dist.all_reduce(nodes)
    if rank == 0:
        total_runs = max(1, min(64, a.batch_runs))
        ms = seconds * 1e3 / max(1, a.steps)
        print(json.dumps({"metric": "batched step timing", "workload": f"batch_2d_{total_runs}runs_fp32",
                          "runs": total_runs, "n_gpus": world, "runs_on_rank0": len(cfgs),
                          "nodes": int(nodes.item()), "steps": a.steps, "ms_per_step": round(ms, 4),
                          "mlups": round(_aggregate_mlups(float(nodes.item()) / world, a.steps, world, seconds), 2),
                          "tile_rank0": {"lec": list(info.tile[0]), "warmc": list(info.tile[1])}}), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_adjoint_case(a):
    """Forward steps with recording and the reverse sweep of the adjoint
    configuration, --steps steps (after --warmup forward steps), whole tape
    kept; prints the timings as one JSON line."""
    import torch

    from paper_2309_04872_gb300 import lbpwfa as lb
    cfg = dict(CONFIG_ADJ)
    N = a.steps
    stream = torch.cuda.Stream()
    with lb.Run(cfg, a.precision, stream=stream.cuda_stream, variant=a.variant) as run:
        run.step(a.warmup)
        wit = _adj_witness(cfg, a.warmup + N, run.info().dt)
        run.record(N, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run.step(N)
        run.synchronize()
        t1 = time.perf_counter()
        J, g, _ = run.adjoint(wit)
        t2 = time.perf_counter()
    print(json.dumps({"metric": "adjoint sweep timing", "workload": "adjoint_2d_warmc_512x256", "steps": N,
                      "precision": a.precision, "variant": a.variant, "forward_recording_ms": round((t1 - t0) * 1e3, 3),
                      "reverse_ms": round((t2 - t1) * 1e3, 3), "J": J, "grad": [float(v) for v in g]}),
          flush=True)


def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_2309_04872_gb300 import lbpwfa as lb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lb.load_library()
    cfg = {"2d_lec": WORKLOAD_2D, "2d_warmc": dict(WORKLOAD_2D, closure="warmc"), "3d_warmc": CONFIG_3D,
           "3d_warmc_128": dict(CONFIG_3D, n=(128, 128, 128), z0=2.0),
           "3d_warmc_64": dict(CONFIG_3D, n=(64, 64, 64), z0=1.2), "axi_warmc": CONFIG_AXI,
           "axi_lec": dict(CONFIG_AXI, closure="lec")}[a.workload]
    cfg = dict(cfg)
    stream = torch.cuda.Stream(device=dev)
    flush = (torch.empty(256 << 20, dtype=torch.uint8, device=dev),
             torch.zeros((1024, 64 << 10), dtype=torch.float32, device=dev),
             torch.empty(64 << 10, dtype=torch.float32, device=dev))
    peaks, peak_kind = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    def measure(prec, steps, warmup, mu=None, variant=None, closure=None):
        c = dict(cfg)
        if mu is not None:
            c["mu"] = mu
        if closure is not None:
            c["closure"] = closure
        v = a.variant if variant is None else variant
        with lb.Run(c, prec, stream=stream.cuda_stream, variant=v) as run:
            info = run.info()
            times = _time_steps(run, stream, steps, warmup, flush)
            bad = run.reduce()[2]
        mean_ms = sum(times) / len(times)
        mlups = info.ncell / (mean_ms * 1e-3) / 1e6
        gbs = info.algorithmic_bytes_per_update * info.ncell / (mean_ms * 1e-3) / 1e9
        stored = info.bytes_per_update * info.ncell / (mean_ms * 1e-3) / 1e9
        return dict(mlups=mlups, ms=mean_ms, gbs=gbs, frac=gbs / hbm,
                    bytes_per_update=info.algorithmic_bytes_per_update,
                    stored_bytes_per_update=info.bytes_per_update, stored_gbs=stored,
                    ncell=info.ncell, total_ms=sum(times), nonfinite=bad, times=times,
                    kernel=KERNEL_NAMES[info.kernel_variant])

    with ClockSampler(local) as clk:
        main = measure(a.precision, a.steps, a.warmup)
    clocks = clk.summary()

    total_s = _slowest_rank_seconds(main["total_ms"] * 1e-3, world, dev)
    value = _aggregate_mlups(main["ncell"], a.steps, world, total_s)

    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": round(total_s * 1e3 / a.steps, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if a.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": _config_block(cfg, a.precision, {"kernel": main["kernel"]}),
        "roofline": {
            "bound": "hbm", "achieved": round(main["gbs"], 2), "peak": hbm, "unit": "GB/s",
            "frac": round(main["frac"], 4),
            "traffic": _traffic_for(f"{main['kernel']}:{_config_block(cfg, a.precision)['workload']}"),
            "bytes_per_update": main["bytes_per_update"], "peak_source": f"{peak_kind} hbm_gbs",
            "bytes_note": "algorithmic bytes per node update (2 K Q s populations + 2 x 3 field components "
                          "x 4 B); achieved = bytes_per_update x nodes / mean CUDA-event step time",
            "stored_bytes_per_update": main["stored_bytes_per_update"],
            "stored_frac": round(main["stored_gbs"] / hbm, 4),
        },
        "clocks": clocks,
        "gpu_launches": a.steps,
    }
    if main["nonfinite"]:
        out["warning"] = "non-finite populations at the end of the timed run"

    fp64_peak = None
    if rank == 0 and (not a.no_modes or not a.no_configs):
        fp64_peak = lb.measure_fp64_rate()
        out["fp64_peak"] = {"value_tflops": round(fp64_peak / 1e12, 4), "source":
                            "lbpwfa_measure_fp64_rate (independent DFMA chains, CUDA events, this GPU)"}

    def mode_entry(r, steps, workload):
        e = {"mlups": round(r["mlups"], 2), "ms_per_step": round(r["ms"], 5),
             "achieved_gbs": round(r["gbs"], 1), "frac_of_measured_hbm": round(r["frac"], 4),
             "bytes_per_update": r["bytes_per_update"], "stored_bytes_per_update": r["stored_bytes_per_update"],
             "steps": steps, "kernel": r["kernel"]}
        if workload.endswith("fp64"):
            # FP64 storage is bound by FP64 arithmetic on this GPU: FP64 operations per update
            # (2 DFMA + DADD + DMUL, counted by ncu on the same kernel) over the measured rate
            alu = _fp64_alu(r["kernel"], workload, r["mlups"], fp64_peak)
            if alu:
                e["fp64_alu"] = alu
        return e

    if rank == 0 and not a.no_modes and a.workload == "2d_lec":
        modes = {}
        for prec in ("fp64", "fp32", "fp16s"):
            for mu in (1e-3, 1e-2):
                for variant in (0, 1, 2, 3):
                    steps = 300 if prec == "fp64" else 1000
                    r = measure(prec, steps, 5, mu=mu, variant=variant)
                    key = f"lec_{prec}_mu{mu:g}" + {0: "", 1: "_plain", 2: "_box", 3: "_persistent"}[variant]
                    modes[key] = mode_entry(r, steps, f"2d_lec_1024x512_{prec}")
        # FP32 storage with exact set sums (the automatic kernel)
        for mu in (1e-3, 1e-2):
            r = measure("fp32c", 1000, 5, mu=mu, variant=0)
            modes[f"lec_fp32c_mu{mu:g}"] = mode_entry(r, 1000, "2d_lec_1024x512_fp32c")
        for prec in ("fp64", "fp32", "fp32c", "fp16s"):
            steps = 200 if prec == "fp64" else 600
            r = measure(prec, steps, 5, mu=1e-2, variant=0, closure="warmc")
            modes[f"warmc_{prec}_mu0.01"] = mode_entry(r, steps, f"2d_warmc_1024x512_{prec}")
        out["modes"] = modes
        out["precision_vs_fp64"] = _precision_table(cfg, stream)
        # the 2D configuration's second temperature (k_B T / m c^2 = 1e-3)
        out["precision_vs_fp64_mu1e-3"] = _precision_table(dict(cfg, mu=1e-3), stream)
        # the same check on the axisymmetric path (600 x 120 nodes of the 3D3V configuration's spacing 0.05)
        out["precision_vs_fp64_axisymmetric"] = _precision_table(
            dict(CONFIG_AXI, n=(600, 120), dx=0.05, z0=3.0), stream)
        out["precision_vs_fp64_3d"] = _precision_3d(stream)

    if rank == 0 and not a.no_configs and a.workload == "2d_lec":
        out["configs_measured"] = _configs(stream, flush, hbm, fp64_peak)

    if rank == 0 and not a.no_adjoint and a.workload == "2d_lec":
        out["adjoint"] = _adjoint(stream)

    if rank == 0 and not a.no_e2e:
        out["e2e"] = _e2e(cfg, a, world)

    if rank == 0 and world == 1 and not a.no_cpu:
        mlups, ns, dt = _oracle_sample(cfg)
        one = _oracle_one_thread(cfg)
        out["cpu_baseline"] = {"value": round(mlups, 4), "unit": "MLUPS", "cores": os.cpu_count(),
                               "kind": "oracle", "cpu_model": _cpu_model(),
                               "sample": f"{ns} FP64 oracle steps of the full 1024x512 grid ({dt:.1f} s)",
                               "one_thread": one}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        out["summary"] = _summary(out)
        print(json.dumps(out), flush=True)


def _summary(out):
    """A compact digest of the line's measurements, placed last so that a
    reader who sees only the end of the line still finds every workload:
    [MLUPS, fraction of the measured HBM by the algorithmic bytes] per
    workload, the FP64 ALU fractions, the reduced-precision errors of n - 1
    after 2000 steps, and the adjoint's cost ratios."""
    s = {"headline": [out["value"], out["roofline"]["frac"]]}
    for k, v in (out.get("modes") or {}).items():
        if not k.endswith(("_plain", "_box", "_persistent")):
            s[k] = [round(v["mlups"]), round(v["frac_of_measured_hbm"], 3)] + \
                ([round(v["fp64_alu"]["frac"], 3)] if v.get("fp64_alu") else [])
    for k, v in (out.get("configs_measured") or {}).items():
        frac = v.get("frac_of_measured_hbm")
        s[k] = [round(v["mlups"]), round(frac, 3) if frac is not None else None] + \
            ([round(v["fp64_alu"]["frac"], 3)] if v.get("fp64_alu") else [])
    for key, tag in (("precision_vs_fp64", "mu1e-2"), ("precision_vs_fp64_mu1e-3", "mu1e-3"),
                     ("precision_vs_fp64_axisymmetric", "axi")):
        for k, v in (out.get(key) or {}).items():
            if isinstance(v, dict) and "rel_err_n_minus_1" in v:
                s[f"err_n-1_{tag}_{k}"] = float(f"{v['rel_err_n_minus_1']:.2e}")
    p3 = out.get("precision_vs_fp64_3d") or {}
    for prec in ("fp32", "fp16s"):
        if prec in p3:
            s[f"err_3d_{prec}"] = {k: float(f"{p3[prec][k]:.2e}") for k in ("n-1", "E_z")}
    adj = out.get("adjoint") or {}
    if "cost_ratio_whole_tape" in adj:
        s["adjoint_cost_ratio"] = {"whole_tape": adj["cost_ratio_whole_tape"], "checkpoint50": adj["cost_ratio_checkpoint50"]}
    return s


def _flops64_for(kernel_key):
    """FP64 operations per node update of a kernel on a workload (2 x DFMA +
    DADD + DMUL of one launch over its nodes, from a committed ncu summary's
    `flops64 <kernel:workload> <count> sources_sha256=<digest>` line), valid
    only while the kernel sources are unchanged."""
    import glob
    import re
    try:
        from paper_2309_04872_gb300 import build as B
        digest = B.step_kernel_digest()
        for fn in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
            for m in re.finditer(r"flops64 (\S+) ([0-9.]+) sources_sha256=([0-9a-f]+)", open(fn).read()):
                if m.group(1) == kernel_key and m.group(3) == digest:
                    return float(m.group(2))
    except OSError:
        pass
    return None


def _cpu_model():
    """The host CPU's model name (lscpu), for the CPU baseline."""
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in txt.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def _oracle_one_thread(cfg, budget_s=8.0):
    """The oracle on one host thread (a child process with OMP_NUM_THREADS=1,
    so the parent's thread pool is untouched): MLUPS on the same grid."""
    code = ("import json,sys,time; sys.path.insert(0, %r); import oracle as O; o=O.Oracle(%r); o.step(1); "
            "t=time.perf_counter(); o.step(1); one=time.perf_counter()-t; n=max(1,min(50,int(%r/max(one,1e-6)))); "
            "t=time.perf_counter(); o.step(n); dt=time.perf_counter()-t; "
            "print(json.dumps({'steps': n, 'seconds': dt}))") % (ROOT, dict(cfg), budget_s)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None
    ncell = 1
    for v in cfg["n"]:
        ncell *= v
    return {"value": round(ncell * d["steps"] / d["seconds"] / 1e6, 4), "unit": "MLUPS", "cores": 1,
            "sample": f"{d['steps']} FP64 oracle steps of the full grid on one thread ({d['seconds']:.1f} s)"}


def _precision_3d(stream, nsteps=2000):
    """The 3D configuration's accuracy statement: WARMC D = 3, mu = 1e-2,
    alpha = 1, sigma_z = 0.7, sigma_r = 0.3 on a 250 x 70 x 72 grid (ragged
    against the marching kernel's 32 x 8 columns and 32-plane chunks), FP32
    and FP16S storage against the FP64 path after nsteps: relative L2 error
    per field (n - 1, u_z, u_x, gamma - 1, lambda - lambda_0, theta_zz -
    theta_rest, theta_xx - theta_rest, theta_zx, E_z, E_x)."""
    from paper_2309_04872_gb300 import lbpwfa as lb
    cfg = dict(CONFIG_3D, n=(250, 70, 72), z0=1.4)
    names = ["n-1", "u_z", "u_x", "gamma-1", "lambda-lambda0", "theta_zz", "theta_xx", "theta_zx"]
    mask = lb.M_N | lb.M_UZ | lb.M_UX | lb.M_GAMMA | lb.M_LAMBDA | lb.M_TH_ZZ | lb.M_TH_XX | lb.M_TH_ZX
    with lb.Run(dict(cfg, alpha=0.0, init_fields=False), "fp64", stream=stream.cuda_stream) as r0:
        rest = r0.moments(mask)[:, :1]
    out = {}
    for prec in ("fp64", "fp32", "fp16s"):
        with lb.Run(cfg, prec, stream=stream.cuda_stream) as run:
            run.step(nsteps)
            out[prec] = (run.moments(mask) - rest, run.fields(lb.F_EZ | lb.F_EX), run.reduce()[2])
    m64, f64, _ = out["fp64"]
    res = {"grid": list(cfg["n"]), "steps": nsteps, "alpha": cfg["alpha"], "mu": cfg["mu"]}
    for prec in ("fp32", "fp16s"):
        m, f, bad = out[prec]
        d = {nm: float(np.linalg.norm(m[j] - m64[j]) / np.linalg.norm(m64[j])) for j, nm in enumerate(names)}
        d["E_z"] = float(np.linalg.norm(f[1] - f64[1]) / np.linalg.norm(f64[1]))
        d["E_x"] = float(np.linalg.norm(f[0] - f64[0]) / np.linalg.norm(f64[0]))
        d["nonfinite"] = int(bad)
        res[prec] = d
    return res


def _precision_table(cfg, stream, nsteps=2000):
    """Reduced-precision storage against the FP64 GPU path on the same
    workload after nsteps: relative L2 error of E_z and of n - 1."""
    from paper_2309_04872_gb300 import lbpwfa as lb
    res = {}
    for closure in ("lec", "warmc"):
        c = dict(cfg, closure=closure)
        out = {}
        for prec in ("fp64", "fp32", "fp32c", "fp16s"):
            with lb.Run(c, prec, stream=stream.cuda_stream) as run:
                run.step(nsteps)
                out[prec] = (run.moments(lb.M_N)[0] - 1.0, run.fields(lb.F_EZ)[0])
        ref_n, ref_e = out["fp64"]
        for prec in ("fp32", "fp32c", "fp16s"):
            n1, ez = out[prec]
            res[f"{closure}_{prec}"] = {
                "rel_err_n_minus_1": float(np.linalg.norm(n1 - ref_n) / np.linalg.norm(ref_n)),
                "rel_err_Ez": float(np.linalg.norm(ez - ref_e) / np.linalg.norm(ref_e)),
                "steps": nsteps}
    return res


def _fp64_alu(kernel, workload, mlups, fp64_peak):
    """FP64 ALU roofline entry of an FP64-storage measurement, or None."""
    fl = _flops64_for(f"{kernel}:{workload}") if fp64_peak else None
    if fl is None:
        return None
    rate = fl * mlups * 1e6
    return {"bound": "alu", "flops_per_update": fl, "achieved_tflops": round(rate / 1e12, 4),
            "peak_tflops": round(fp64_peak / 1e12, 4), "frac": round(rate / fp64_peak, 4)}


def _configs(stream, flush, hbm, fp64_peak=None):
    """The 1D configuration as a whole run (4000 steps, FP64), the batched
    sweep, the axisymmetric grid and the 3D configuration over a few timed
    steps."""
    import torch

    from paper_2309_04872_gb300 import lbpwfa as lb
    res = {}
    with lb.Run(CONFIG_1D, "fp64", stream=stream.cuda_stream) as run:
        run.step(10)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run.step(4000)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res["1d_lec_fp64_2048"] = {"steps": 4000, "ms_total": round(ms, 3), "steps_per_s": round(4000 / ms * 1e3, 1),
                                   "mlups": round(2048 * 4000 / ms / 1e3, 2),
                                   "note": "state is L2-resident and launch-bound; no flush"}
    # the batched sweep: 64 uneven 2D runs, both closures, one launch per closure and step
    draws, cfgs = _batch_cfgs(64)
    for bprec in ("fp32", "fp16s"):
        with lb.Batch(cfgs, bprec, stream=stream.cuda_stream, tune=True) as b:
            info = b.info()
            b.step(32)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(96)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 96
            gbs = info.algorithmic_bytes_per_step / (ms * 1e-3) / 1e9
            nlec = sum(1 for d in draws if d["closure"] == "lec")
            res[f"batch_64x2d_{bprec}"] = {
                "mlups": round(info.ncell / (ms * 1e-3) / 1e6, 2), "ms_per_step": round(ms, 4),
                "achieved_gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
                "nodes": int(info.ncell), "runs": 64, "lec_runs": nlec, "warmc_runs": 64 - nlec,
                "tile": {"lec": list(info.tile[0]), "warmc": list(info.tile[1])},
                "tuned_ms": {"lec": [round(v, 4) for v in info.tuned_ms[0] if v > 0],
                             "warmc": [round(v, 4) for v in info.tuned_ms[1] if v > 0]},
                "graph_steps": info.graph_steps, "steps": 96, "kernel": "lb_step_batch_kernel",
                "l2": "state larger than L2 (no flush)"}
    # the axisymmetric 3D3V grid, both closures
    for closure in ("warmc", "lec"):
        for prec in ("fp32", "fp16s", "fp64"):
            c = dict(CONFIG_AXI, closure=closure)
            with lb.Run(c, prec, stream=stream.cuda_stream) as run:
                info = run.info()
                times = _time_steps(run, stream, 100 if prec == "fp64" else 300, 5, flush)
            mean = sum(times) / len(times)
            gbs = info.algorithmic_bytes_per_update * info.ncell / (mean * 1e-3) / 1e9
            res[f"axi_{closure}_{prec}_3000x600"] = {
                "mlups": round(info.ncell / (mean * 1e-3) / 1e6, 2), "ms_per_step": round(mean, 4),
                "achieved_gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
                "bytes_per_update": info.algorithmic_bytes_per_update,
                "stored_bytes_per_update": info.bytes_per_update, "steps": len(times),
                "kernel": KERNEL_NAMES[info.kernel_variant], "geometry": "axisymmetric (z, r)"}
            if prec == "fp64":
                alu = _fp64_alu(KERNEL_NAMES[info.kernel_variant], f"axi_{closure}_3000x600_fp64",
                                info.ncell / (mean * 1e-3) / 1e6, fp64_peak)
                if alu:
                    res[f"axi_{closure}_{prec}_3000x600"]["fp64_alu"] = alu
    for prec in ("fp32", "fp64"):
        try:
            with lb.Run(CONFIG_3D, prec, stream=stream.cuda_stream) as run:
                info = run.info()
                times = _time_steps(run, stream, 6 if prec == "fp64" else 10, 3, flush)
        except lb.LbpwfaError as err:
            res[f"3d_warmc_{prec}_512x256x256"] = {"error": str(err)}
            continue
        mean = sum(times) / len(times)
        gbs = info.algorithmic_bytes_per_update * info.ncell / (mean * 1e-3) / 1e9
        res[f"3d_warmc_{prec}_512x256x256"] = {
            "mlups": round(info.ncell / (mean * 1e-3) / 1e6, 2), "ms_per_step": round(mean, 3),
            "achieved_gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
            "bytes_per_update": info.algorithmic_bytes_per_update,
            "stored_bytes_per_update": info.bytes_per_update, "steps": len(times),
            "kernel": KERNEL_NAMES[info.kernel_variant],
            "device_gb": round(info.device_bytes / 1e9, 2)}
        if prec == "fp64":
            alu = _fp64_alu(KERNEL_NAMES[info.kernel_variant], "3d_warmc_512x256x256_fp64",
                            info.ncell / (mean * 1e-3) / 1e6, fp64_peak)
            if alu:
                res[f"3d_warmc_{prec}_512x256x256"]["fp64_alu"] = alu
    return res


def _adj_witness(cfg, nsteps, dt):
    """On-axis E_z slot 4 k_p^-1 behind the driver centre at t_{N-1/2}
    (the time of the stored E)."""
    zc = cfg["z0"] + (nsteps - 0.5) * dt
    return (int(round((zc - 4.0) / cfg["dx"])), cfg["n"][1] // 2 - 1)


def _adjoint(stream):
    """Cost of forward + reverse sweep against the forward alone (FP32
    storage), with checkpoints every 50 steps and with the whole tape kept,
    and the gradient against central differences of the FP64 path."""
    import torch

    from paper_2309_04872_gb300 import lbpwfa as lb
    cfg = dict(CONFIG_ADJ)
    N = ADJ_STEPS
    sc = stream.cuda_stream
    res = {"config": "2d_warmc_512x256_fp32_1000steps", "steps": N}

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    with lb.Run(cfg, "fp32", stream=sc) as run:
        dt = run.info().dt
    wit = _adj_witness(cfg, N, dt)
    res["witness"] = list(wit)

    def fwd():
        with lb.Run(cfg, "fp32", stream=sc) as run:
            run.step(N)
            run.synchronize()

    def fwd_adj(C):
        with lb.Run(cfg, "fp32", stream=sc) as run:
            run.record(N, C)
            run.step(N)
            return run.adjoint(wit)

    fwd()
    fwd_adj(50)  # warm-up (allocations, module load)
    t_f = min(wall(fwd)[0] for _ in range(3))
    t_c, (J32, g32, _) = min((wall(lambda: fwd_adj(50)) for _ in range(3)), key=lambda r: r[0])
    t_t, (J32t, g32t, _) = min((wall(lambda: fwd_adj(0)) for _ in range(3)), key=lambda r: r[0])
    res["forward_ms"] = round(t_f * 1e3, 2)
    res["forward_plus_adjoint_ms_checkpoint50"] = round(t_c * 1e3, 2)
    res["forward_plus_adjoint_ms_whole_tape"] = round(t_t * 1e3, 2)
    res["cost_ratio_checkpoint50"] = round(t_c / t_f, 3)
    res["cost_ratio_whole_tape"] = round(t_t / t_f, 3)
    res["target_ratio"] = 3.0
    res["note"] = ("wall time of (forward steps + recording + reverse sweep) / wall time of the same forward "
                   "steps alone; run creation included in both")
    res["J_fp32"] = J32
    res["grad_fp32"] = [float(v) for v in g32]
    res["checkpoint_equals_tape"] = bool(J32 == J32t and np.array_equal(g32, g32t))

    def J64(c):
        with lb.Run(c, "fp64", stream=sc) as run:
            run.step(N)
            ez = run.fields(lb.F_EZ)[0]
        return float(ez[wit[0] + c["n"][0] * wit[1]])

    with lb.Run(cfg, "fp64", stream=sc) as run:
        run.record(N, 50)
        run.step(N)
        J64v, g64, _ = run.adjoint(wit)
    fd = []
    for k, name in enumerate(["alpha", "sigma_z", "sigma_r"]):
        h = 1e-4 * cfg[name]
        fd.append((J64(dict(cfg, **{name: cfg[name] + h})) - J64(dict(cfg, **{name: cfg[name] - h}))) / (2 * h))
    fd = np.array(fd)
    res["J_fp64"] = J64v
    res["grad_fp64"] = [float(v) for v in g64]
    res["fd_fp64_h1e-4"] = [float(v) for v in fd]
    res["rel_err_fp32_adjoint_vs_fd"] = [float(v) for v in np.abs(g32 - fd) / np.abs(fd)]
    res["rel_err_fp64_adjoint_vs_fd"] = [float(v) for v in np.abs(g64 - fd) / np.abs(fd)]
    # the 256-sample profile (dz = 0.05, the Gaussian), FP32 adjoint vs FP64
    # central differences on four samples around the peak
    zs = (np.arange(256) - 127.5) * 0.05
    prof = cfg["alpha"] * np.exp(-zs ** 2 / (2 * cfg["sigma_z"] ** 2))
    cp = dict(cfg, profile=prof, profile_dz=0.05)
    with lb.Run(cp, "fp32", stream=sc) as run:
        run.record(N, 50)
        run.step(N)
        _, gsr, gp = run.adjoint(wit)
    errs = []
    scale = float(np.abs(gp).max())
    for j in (112, 124, 128, 140):
        h = 1e-4 * cfg["alpha"]
        pp, pm = prof.copy(), prof.copy()
        pp[j] += h
        pm[j] -= h
        fdj = (J64(dict(cp, profile=pp)) - J64(dict(cp, profile=pm))) / (2 * h)
        errs.append({"sample": j, "adjoint_fp32": float(gp[j]), "fd_fp64": fdj,
                     "rel_err_of_max": abs(gp[j] - fdj) / scale})
    res["profile_samples"] = errs
    return res


def _e2e(cfg, a, world):
    """Same metric through the public C ABI with host buffers: upload of the
    initial state from pinned host memory, K steps, read-back of n and E_z."""
    import torch

    from paper_2309_04872_gb300 import lbpwfa as lb
    steps = a.steps
    with lb.Run(cfg, a.precision) as run:
        f0, E0, B0 = run.get_state()
        nc, K, Q = run.ncell, run.K, run.Q
    pin = lambda x: torch.from_numpy(x).pin_memory()  # noqa: E731
    f0p, E0p, B0p = pin(f0), pin(E0), pin(B0)
    n_out = torch.empty((1, nc), dtype=torch.float64).pin_memory()
    e_out = torch.empty((1, nc), dtype=torch.float64).pin_memory()
    with lb.Run(cfg, a.precision) as run:
        run.set_state(f0p, E0p, B0p)  # first call allocates the staging buffer
        run.step(2)
        run.moments(lb.M_N, out=n_out)
        run.synchronize()
        t0 = time.perf_counter()
        run.set_state(f0p, E0p, B0p)
        run.step(steps)
        run.moments(lb.M_N, out=n_out)
        run.fields(lb.F_EZ, out=e_out)
        t1 = time.perf_counter()
    h2d = (f0.nbytes + E0.nbytes + B0.nbytes) / steps
    d2h = (n_out.numel() + e_out.numel()) * 8 / steps
    return {"value": round(nc * steps * world / (t1 - t0) / 1e6, 3), "unit": "MLUPS",
            "h2d_bytes_per_step": round(h2d, 1), "d2h_bytes_per_step": round(d2h, 1),
            "note": "lbpwfa_set_state from pinned host + lbpwfa_step(K) + lbpwfa_moments/fields to host"}


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    cfg = dict(WORKLOAD_2D)
    o = O.Oracle(cfg)
    for _ in range(max(0, min(a.warmup, 3))):
        o.step(1)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    budget = 120.0
    nsteps = max(1, min(a.steps, int(budget / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t0
    ncell = cfg["n"][0] * cfg["n"][1]
    value = ncell * nsteps / dt / 1e6
    sample = f"{nsteps} FP64 oracle steps of the full 1024x512 grid ({dt:.1f} s)"
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": round(dt * 1e3 / nsteps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config_block(cfg, a.precision, {"impl": "oracle"}),
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint_2d_warmc":
        run_adjoint_case(args)
    elif args.workload == "batch_2d":
        run_batch_case(args)
    else:
        run_ours(args)
