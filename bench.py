"""Benchmark of the two-phase DUGKS step on GB300.

Default workload: the batched ensemble of 512 rising-bubble / stationary-drop
instances on square periodic meshes of uneven side (64..512, seed 1802), FP32
storage, ~3.96e7 cells.  One "step" advances every instance of the batch by
one time step (all rows of the hot path).  The metric is cell-updates/s (one
cell advancing both D2Q9 distributions f and g by one dt).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch|rt|drop|roofline] [--precision fp32|fp64]

For N > 1 (launched with torch.distributed.run) every rank advances its own
ensemble (seed 1802 + rank): weak scaling with no data-path collective.
The reference arm (--impl reference) times the CPU FP64 oracle on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
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

from paper_1802_02868_gb300 import inputs as I  # noqa: E402

METRIC = "cell-updates/s (f+g, D2Q9)"
UNIT = "cell-updates/s"

# Algorithmic floating-point operations of one cell update (FMA = 2, divide =
# 1), counted from the formulas of the step: cell macros, equilibria, sources
# and bar-plus 531; two faces x 723 (reconstruction of 18 bar distributions,
# face macros, six equilibria/sources/originals per kind, flux); update 150.
FLOP_PER_CELL_UPDATE = 2127.0
# ALU peaks from the unit counts and the maximum SM clock: 152 SMs x 128 FP32
# lanes x 2 flop x 2.07 GHz, and 152 SMs x 2 DFMA/cycle x 2 flop x 2.07 GHz.
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes per cell of one fused-step launch (uniform periodic path), per
# tile shape, from ncu captures of a 2048 x 2048 periodic drop
# (dram__bytes_read.sum + dram__bytes_write.sum over 4,194,304 cells); valid
# only for the kernel sources they were taken on.
TRAFFIC_SOURCES_SHA = "d64a9240f3552be2"
TRAFFIC_BYTES_PER_CELL_FP32 = {
    "32x8 strip16/288": (346.862080e6 + 297.274112e6) / 4194304,
}


# the headers the fused-step kernels are compiled from (not the diagnostics'
# or the adjoint's, which do not change them)
STEP_HEADERS = ("dugks_common.cuh", "dugks_kernels.cuh", "dugks_fused.cuh", "dugks_strip.cuh")


def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in STEP_HEADERS:
        h.update(open(os.path.join(ROOT, "paper_1802_02868_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def workload(name, seed):
    if name == "batch":
        cases = I.batched_ensemble(512, seed=seed)
        desc = {"workload": "batched ensemble: 512 rising-bubble/stationary-drop instances, square periodic "
                            "meshes side in {64..512}, density ratio log-uniform [2, 20], seed %d" % seed,
                "instances": 512}
    elif name == "rt":
        cases = [I.rayleigh_taylor()]
        desc = {"workload": "Rayleigh-Taylor 256x1024, At=0.5, Re=3000, walls in y", "instances": 1}
    elif name == "drop":
        cases = [I.stationary_drop()]
        desc = {"workload": "stationary drop 64x64 periodic, rho ratio 10", "instances": 1}
    elif name == "roofline":
        n = int(os.environ.get("DUGKS_ROOFLINE_N", "4096"))
        cases = [I.roofline_drop(n)]
        desc = {"workload": "roofline drop %dx%d periodic, R=%d" % (n, n, n // 4), "instances": 1}
    else:
        raise SystemExit("unknown workload %s" % name)
    desc["cells"] = int(sum(c.mesh.ncells for c in cases))
    return cases, desc


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world_size, seconds):
    """Whole-job throughput: every rank advances its own workload (weak
    scaling), so the job processes world_size times the per-rank units in the
    slowest rank's time."""
    return world_size * units_per_rank / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampler of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, tag="bench"):
        self.index = index
        self.p = None
        # raw samples: DUGKS_CLOCKS_DIR if set, else the temporary directory
        folder = os.environ.get("DUGKS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, "clocks_%s_%d.csv" % (tag, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


def measured_peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(cases, precision_name, budget_s=12.0):
    """Time the CPU FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    sample = cases[: min(len(cases), 4)]
    sims = [oracle.Oracle(c.mesh, c.params).init(c.phi0) for c in sample]
    cells = sum(c.mesh.ncells for c in sample)
    for s in sims:            # one warm step (allocates, faults pages)
        s.step(1)
    steps = 0
    t0 = time.perf_counter()
    while True:
        for s in sims:
            s.step(1, check=False)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": steps * cells / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of %d instances (%d cells), %d FP64 oracle steps, %.1f s" % (
                len(sample), len(cases), cells, steps, dt)}


def fp64_single_instance_rate(dugks, torch, cases, n_sample=16, steps=3):
    """Cell-updates/s of the plain path: instances stepped one at a time as
    single-instance FP64 simulations (a seeded sample of the workload)."""
    rng = np.random.default_rng(7)
    idx = sorted(rng.choice(len(cases), size=min(n_sample, len(cases)), replace=False).tolist())
    total_ms, cell_updates = 0.0, 0
    stream = torch.cuda.current_stream()
    for k in idx:
        c = cases[k]
        s = dugks.Sim(c.mesh, c.params, dugks.FP64, stream=stream.cuda_stream).init(c.phi0)
        s.step(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            s.step(1)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        cell_updates += steps * c.mesh.ncells
        s.close()
    return cell_updates / (total_ms * 1e-3), len(idx)


def run_adjoint(args, dugks, torch):
    """Adjoint workload: Rayleigh-Taylor 256x512, 4000 steps, FP32 forward with
    a checkpoint every 100 steps and recomputation; gradient of the squared L2
    misfit of phi against a seeded target with respect to the initial phi field,
    kappa and the mobility.  Compared with the 20 FP64 forward runs that central
    differences of the same 10 parameters (8 amplitudes, kappa, mobility) need,
    timed on one FP64 run."""
    nx, ny, nsteps, K = 256, 512, args.adjoint_steps, 100
    rng = np.random.default_rng(1803)
    amps = np.concatenate([[0.1 * nx], rng.normal(0.0, 0.01 * nx, 7)])
    c = I.rayleigh_taylor(nx=nx, ny=ny, amplitudes=list(amps))
    tgt = I.rt_field(c.mesh, float(nx), 0.5 * ny, list(amps + rng.normal(0.0, 0.01 * nx, 8)), 4.0)
    prec = dugks.FP32 if args.precision == "fp32" else dugks.FP64
    sim = dugks.Sim(c.mesh, c.params, prec).init(c.phi0)
    sim.adjoint(min(nsteps, 200), tgt, ckpt_every=K)     # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = sim.adjoint(nsteps, tgt, ckpt_every=K)
    t_adj = time.perf_counter() - t0
    s64 = dugks.Sim(c.mesh, c.params, dugks.FP64).init(c.phi0)
    s64.step(20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s64.step(nsteps)
    torch.cuda.synchronize()
    t_fwd64 = time.perf_counter() - t0
    line = {"metric": "adjoint gradient wall time (10 parameters + dL/dphi0)", "value": t_adj, "unit": "s",
            "n_gpus": 1, "steps": nsteps, "warmup": 1, "higher_is_better": False, "dtype": args.precision,
            "data": "synthetic", "config": {"workload": "adjoint: Rayleigh-Taylor %dx%d, %d steps, checkpoint every %d, "
                                                        "8 cosine amplitudes (seed 1803)" % (nx, ny, nsteps, K)},
            "loss": float(r["loss"]), "dkappa": float(r["dkappa"]), "dlambda": float(r["dlambda"]),
            "fp64_forward_s": t_fwd64, "fd20_fp64_s": 20 * t_fwd64, "speedup_vs_fd20_fp64": 20 * t_fwd64 / t_adj,
            "forward_equivalent_cell_updates_per_s": nsteps * nx * ny / t_adj}
    print(json.dumps(line))
    return 0


def run_reference(args, cases, desc):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    sample = cases[: min(len(cases), 2)]
    sims = [oracle.Oracle(c.mesh, c.params).init(c.phi0) for c in sample]
    cells = sum(c.mesh.ncells for c in sample)
    for _ in range(args.warmup):
        for s in sims:
            s.step(1, check=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in sims:
            s.step(1, check=False)
    dt = time.perf_counter() - t0
    value = args.steps * cells / dt
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(desc, sample_instances=len(sample), sample_cells=cells),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d of %d instances per step (%d cells)" % (len(sample), len(cases), cells)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_diagnostics(sim, ncells, peak_hbm, calls=5):
    """On-device diagnostics of the final state (dugks_diagnostics: k_diag_f,
    per-instance finalisation, read-back), outside the timed region:
    abi_ms_per_call times the C call into a reused array, ms_per_call the
    Python call that also builds one dict per instance."""
    from paper_1802_02868_gb300 import dugks
    buf = sim.diagnostics_array()
    t0 = time.perf_counter()
    for _ in range(calls):
        sim.diagnostics_array(buf)
    abi_ms = (time.perf_counter() - t0) * 1e3 / calls
    sim.set_timing(True)
    sim.kernel_times()
    t0 = time.perf_counter()
    for _ in range(calls):
        sim.diagnostics()
    host_ms = (time.perf_counter() - t0) * 1e3 / calls
    kt = sim.kernel_times()
    sim.set_timing(False)
    kms, kn = kt["k_diag_f"]
    avg_s = kms / max(kn, 1) * 1e-3
    bpc = sim.kernel_bytes_per_cell(dugks.kernel_name_index("k_diag_f"))
    return {"calls": calls, "ms_per_call": host_ms, "abi_ms_per_call": abi_ms,
            "kernels_ms_per_call": {k: kt[k][0] / calls for k in ("k_diag_f",)},
            "k_diag_f_hbm": {"achieved": bpc * ncells / avg_s / 1e9, "peak": peak_hbm, "unit": "GB/s",
                             "frac": bpc * ncells / avg_s / 1e9 / peak_hbm, "algorithmic_bytes_per_cell": bpc}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch", "rt", "drop", "roofline"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile-shape", type=int, default=None, help="use this fused-step shape instead of autotuning")
    ap.add_argument("--adjoint", action="store_true", help="time the adjoint workload instead")
    ap.add_argument("--adjoint-steps", type=int, default=4000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_env()
    if args.adjoint:
        import torch
        from paper_1802_02868_gb300 import dugks
        return run_adjoint(args, dugks, torch)
    cases, desc = workload(args.workload, 1802 + rank)
    if args.impl == "reference":
        return run_reference(args, cases, desc)

    import torch
    from paper_1802_02868_gb300 import dugks

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = dugks.FP32 if args.precision == "fp32" else dugks.FP64
    stream = torch.cuda.current_stream()
    sim = dugks.Sim([c.mesh for c in cases], [c.params for c in cases], prec, stream=stream.cuda_stream)
    ncells = sim.ncells
    # pinned host buffers for the end-to-end leg
    phi_h = torch.from_numpy(np.concatenate([c.phi0.reshape(-1) for c in cases])).pin_memory()
    sim.init(phi_h.numpy())
    if args.tile_shape is not None:
        sim.set_tile_shape(args.tile_shape)
        tuned = (args.tile_shape, dugks.tile_shape_name(args.tile_shape), None)
    else:
        k0 = sim.tile_shape()[0]
        tuned = sim.autotune(steps=10) if not args.no_autotune else (k0, dugks.tile_shape_name(k0), None)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- device-resident timed region
    clocks = Clocks(local)
    clocks.start()
    sim.set_timing(True)
    sim.kernel_times()            # reset the accumulators
    l0 = sim.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = sim.launch_count() - l0
    ktimes = sim.kernel_times()
    sim.set_timing(False)
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, "cuda")
    st = sim.status()
    n_finite = sum(1 for v in st if v == 0)
    # masked (non-finite) instances do no work: count only the cells advanced
    live_cells = int(sum(c.mesh.ncells for c, v in zip(cases, st) if v == 0))
    value = job_rate(args.steps * live_cells, ws, ms * 1e-3)

    # ---- end to end through the public API: host phi -> init -> steps with a
    # per-step FP64 conservation read-back -> moments to host.  The read-back
    # is pipelined: step k + 1 is enqueued before the host waits for the sums
    # of step k (dugks_conservation_async), which land in pinned buffers
    out_h = [torch.empty(ncells, dtype=torch.float64).pin_memory() for _ in range(5)]
    sums_h = [torch.empty(2 * len(cases), dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    drift = 0.0
    clocks_e2e = Clocks(local, "e2e")
    clocks_e2e.start()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.init(phi_h.numpy())   # synchronises (device-side finiteness check of phi)
    t_init = time.perf_counter()
    sim.step(1)
    sim.conservation_async(sums_h[0])
    first = None
    for k in range(1, args.steps + 1):
        if k < args.steps:
            sim.step(1)
        sim.conservation_wait()
        got = sums_h[(k - 1) % 2]
        if first is None:
            first = got[0::2].copy()
        else:   # the host consumes each step's sums: largest relative drift of sum phi
            drift = max(drift, float(np.nanmax(np.abs(got[0::2] - first) / np.maximum(np.abs(first), 1e-300))))
        if k < args.steps:
            sim.conservation_async(sums_h[k % 2])
    t_steps = time.perf_counter()   # the last sums have landed: every step is done
    sim.moments(out=[o.numpy() for o in out_h])   # straight into the pinned buffers
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    clk_e2e = clocks_e2e.stop()
    e2e_s = t_end - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    n_inst = len(cases)
    h2d = ncells * 8 / args.steps
    d2h = (2 * 8 * n_inst * args.steps + 5 * 8 * ncells) / args.steps
    e2e = {"value": job_rate(args.steps * ncells, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h,
           "phi_sum_drift": drift,
           "parts_ms": {"init": (t_init - t0) * 1e3, "steps": (t_steps - t_init) * 1e3, "moments": (t_end - t_steps) * 1e3},
           "clocks": clk_e2e,
           "note": "init from pinned host phi + K steps each followed by a conservation read-back (pipelined: "
                   "step k+1 runs while the host reads the sums of step k) + moments to host"}

    # ---- roofline of the dominant kernel: ALU bound (see FLOP_PER_CELL_UPDATE);
    # the HBM view of the same launch is reported beside it
    best = max(range(dugks.NUM_KERNELS), key=lambda k: ktimes[dugks.kernel_name(k)][0])
    kname = dugks.kernel_name(best)
    kms, kn = ktimes[kname]
    avg_s = kms / max(kn, 1) * 1e-3
    bpc = sim.kernel_bytes_per_cell(best)
    hbm_achieved = bpc * ncells / avg_s / 1e9
    peak_hbm, peak_kind = measured_peak_hbm()
    tflops = FLOP_PER_CELL_UPDATE * ncells / avg_s / 1e12
    peak_alu = PEAK_FP32_TFLOPS if prec == dugks.FP32 else PEAK_FP64_TFLOPS
    traffic = None
    if kname == "k_step" and prec == dugks.FP32 and kernel_sources_sha() == TRAFFIC_SOURCES_SHA \
            and tuned[1] in TRAFFIC_BYTES_PER_CELL_FP32:
        traffic = TRAFFIC_BYTES_PER_CELL_FP32[tuned[1]] * ncells
    # the library times the fused step under one slot, "k_step"; the kernel
    # behind it is k_strip for the strip shapes
    kernel = ("k_strip" if "strip" in tuned[1] else "k_step") if kname == "k_step" else kname
    # the same peak measured on this GPU by FMA-only kernels (scalar, packed
    # two-lane and FP64), after the timed regions
    meas = dugks.measure_alu_peaks(stream=stream.cuda_stream)
    peak_meas = max(meas["fp32"], meas["fp32x2"]) if prec == dugks.FP32 else meas["fp64"]
    roof = {"bound": "alu", "kernel": kernel, "timer": kname, "shape": tuned[1], "achieved": tflops, "peak": peak_alu,
            "unit": "TFLOP/s",
            "frac": tflops / peak_alu, "peak_source": "unit counts x 2.07 GHz max SM clock (%s)" % (
                "FP32 FMA lanes" if prec == dugks.FP32 else "FP64 DFMA rate"),
            "peak_measured": peak_meas, "frac_of_measured": tflops / peak_meas,
            "measured_fma_tflops": meas,
            "flop_per_cell": FLOP_PER_CELL_UPDATE, "traffic": traffic, "avg_launch_ms": avg_s * 1e3,
            "hbm": {"achieved": hbm_achieved, "peak": peak_hbm, "unit": "GB/s", "frac": hbm_achieved / peak_hbm,
                    "peak_source": peak_kind, "algorithmic_bytes_per_cell": bpc,
                    # the state alone: 18 tilde words read and written; the fused
                    # step also reads and writes the stored phi (a float pair in FP32)
                    "state_bytes_per_cell": 2 * 18 * (4 if prec == dugks.FP32 else 8),
                    "frac_state_bytes": (2 * 18 * (4 if prec == dugks.FP32 else 8)) * ncells / avg_s / 1e9 / peak_hbm},
            "kernel_share": {k: v[0] / max(sum(x[0] for x in ktimes.values()), 1e-12) for k, v in ktimes.items()
                             if v[1]}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == dugks.FP32 else "f64", "data": "synthetic",
            "config": dict(desc, precision=args.precision, tile_shape=tuned[1], l2="inputs larger than L2 (state %.2f GB)" % (
                ncells * 72 * (1 if prec == dugks.FP32 else 2) / 1e9) if ncells * 72 > 129e6 else
                "inputs smaller than L2: not flushed"),
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clk, "instances_finite": n_finite}
    line["diagnostics"] = time_diagnostics(sim, ncells, peak_hbm)
    if rank == 0 and ws == 1 and len(cases) > 1 and prec == dugks.FP32:
        rate64, nsamp = fp64_single_instance_rate(dugks, torch, cases)
        line["speedup_vs_fp64_single_instance"] = {
            "fp64_single_instance_value": rate64, "unit": UNIT, "ratio": (value / ws) / rate64,
            "sample": "%d instances, each its own FP64 simulation, stepped one at a time" % nsamp}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(cases, args.precision)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    sim.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
