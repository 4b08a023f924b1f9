#!/usr/bin/env python
"""Benchmark of the GB300 TCNS library: RHS cell-updates per second.

Workload (default): inviscid Taylor-Green vortex on a periodic 256^3 grid
(gamma 1.4, Roe flux, CFL 0.5), advanced by SSP-RK3 steps with the FP32
bulk path (single-precision interpolation, flux and differencing; FP64
CFL reduction and state accumulation).  One step = one RK3 step = three
RHS evaluations; value = nodes x 3 x steps x ranks / max-over-ranks time.
The FP64 plain path is timed on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload tgv256|tgv192|quad1024|sod400|rt1024|batch1d|serve|scalar]

With N > 1 (torchrun) every rank advances its own replica (weak scaling,
no data-path collective: the instances are independent).
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WCNS RHS cell-updates/s"
UNIT = "cell-updates/s"
# Unit counts of the GB300 SM: 128 FP32 lanes, 2 FP64 FMA per clock; an FMA
# is 2 flops.  The SM count and the maximum clock are read at run time.
FP32_LANES_PER_SM, FP64_FMA_PER_SM = 128, 2
DEFAULT_SMS, DEFAULT_SM_MHZ, FALLBACK_HBM_GBS = 152, 2070.0, 6800.0

# Flops per face and per node of one sweep direction of the FP32 kernel,
# counted from its arithmetic (FMA = 2, add/mul/min/max/abs = 1, one MUFU
# op = 1) with every stencil taking the no-cut branch (smooth flow).
FACE_FLOPS = {1: 520, 2: 770, 3: 1040}
NODE_FLOPS = {1: 30, 2: 40, 3: 50}
# FP64 operations per node per RHS of the scalar path (linear advection,
# TCNS weights, every stencil on the no-cut branch), one flop per add, mul,
# abs, min or divide (the fixed-order FP64 path contracts nothing into FMA):
# two interpolations of 54 (sub-stencil derivatives 30, smoothness test 7,
# Eq. 12 17), the Eq. 6 flux 6, the Eq. 3 difference and 1/h 10, and the
# SSP-RK3 stage combination 4 on average.
SCALAR_NODE_FLOPS = 2 * 54 + 6 + 10 + 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv256",
                    choices=["tgv256", "tgv192", "quad1024", "sod400", "rt1024", "batch1d", "serve", "scalar"])
    ap.add_argument("--requests", type=int, default=32, help="serve: requests replayed from the trace")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrival rate (1/s)")
    ap.add_argument("--side-lo", type=int, default=128, help="serve: smallest grid side")
    ap.add_argument("--side-hi", type=int, default=1024, help="serve: largest grid side")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving replay of the default line")
    ap.add_argument("--l1-max-side", type=int, default=1 << 30,
                    help="serve: FP32 error against FP64 only for requests up to this side (FP64 solves are slow)")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "fp64"],
                    help="single-grid workloads: the path timed (auto: the workload's default)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain-path line")
    ap.add_argument("--accuracy-steps", type=int, default=200,
                    help="CFL steps of the FP32-vs-FP64 error measurement (the 3D configuration's 200)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def workload(name):
    from paper_1810_07806_gb300 import inputs
    if name == "tgv256":
        pb = inputs.taylor_green(256)
        return pb, dict(workload="taylor_green_3d_256^3_periodic", nodes=pb.cells, nv=5,
                        precision="fp32 bulk (fp64 reductions + accumulation)", flux="roe", cfl=0.5), True
    if name == "tgv192":   # the same flow on a smaller grid (profiler captures: state still > L2)
        pb = inputs.taylor_green(192)
        return pb, dict(workload="taylor_green_3d_192^3_periodic", nodes=pb.cells, nv=5,
                        precision="fp32 bulk (fp64 reductions + accumulation)", flux="roe", cfl=0.5), True
    if name == "rt1024":
        pb = inputs.rayleigh_taylor(256)
        return pb, dict(workload="rayleigh_taylor_2d_256x1024", nodes=pb.cells, nv=4,
                        precision="fp32 bulk (fp64 reductions + accumulation)", flux="roe", cfl=0.5,
                        gamma=pb.gamma, boundaries="reflecting x walls, fixed y states, gravity (0, 1)"), True
    if name == "quad1024":
        pb = inputs.four_quadrant(1024)
        return pb, dict(workload="four_quadrant_riemann_2d_1024^2_lax_liu_3", nodes=pb.cells, nv=4,
                        precision="fp64", flux="roe", cfl=0.5), False
    pb = inputs.shock_tube(400)
    return pb, dict(workload="sod_1d_400", nodes=pb.cells, nv=3, precision="fp64", flux="roe",
                    cfl=0.5), False


def measured_peaks():
    """MEASURED_PEAKS.json at the repository root (copy bandwidth and clocks
    measured on this GPU model), or an empty dict."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def device_peaks(dev_index=0):
    """ALU peaks derived from unit counts, this device's SM count and the
    maximum SM clock, and the HBM peak: the measured copy bandwidth when
    MEASURED_PEAKS.json is present, else the fallback figure."""
    mp = measured_peaks()
    sms = DEFAULT_SMS
    try:
        import torch
        if torch.cuda.is_available():
            sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    except Exception:
        pass
    mhz = float(mp.get("sm_max_mhz", DEFAULT_SM_MHZ))
    hbm = mp.get("hbm_gbs")
    return {"sms": sms, "sm_max_mhz": mhz,
            "fp32_tflops": sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
            "fp64_tflops": sms * FP64_FMA_PER_SM * 2 * mhz * 1e6 / 1e12,
            "hbm_gbs": float(hbm) if hbm else FALLBACK_HBM_GBS,
            "hbm_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6.8 TB/s"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.dev_id = dev_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
            if self.dev_id:
                cmd += ["-i", self.dev_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        mhz = [float(r[1]) for r in rows if re.match(r"^[0-9.]+$", r[1])]
        mx = [float(r[2]) for r in rows if re.match(r"^[0-9.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- profiles
def profile_traffic(workload_name):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, or None when the kernel source changed since that capture or
    the summary covers another workload."""
    path = os.path.join(ROOT, "profiles", "sweep_fp32_tgv.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    w = re.search(r"traffic_workload:\s*(\S+)", txt)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    if not w or w.group(1) != workload_name:
        return None
    return float(m.group(1))


def kernel_source_hash():
    """Hash of the FP32 sweep's code: its source files without // comments
    and blank lines, so that a comment edit keeps a profile valid."""
    d = os.path.join(ROOT, "paper_1810_07806_gb300", "csrc")
    sha = hashlib.sha256()
    for f in ("wcns_device.cuh", "wcns_cvt.cuh", "wcns_sweep.cuh", "sweep_fp32.cu"):
        lines = (ln.split("//", 1)[0].rstrip() for ln in open(os.path.join(d, f)).read().splitlines())
        sha.update(("\n".join(ln for ln in lines if ln.strip()) + "\n").encode())
    return sha.hexdigest()[:16]


# ---------------------------------------------------------------- CPU oracle baseline
def ora_cfg_for(pb):
    """The oracle's configuration of a problem (boundary kinds, fixed states,
    body force included)."""
    from oracle import oracle as O
    oc = lambda k: k if k in (O.BC_REFLECT, O.BC_FIXED) else O.BC_AUTO
    return O.make_cfg(ndim=pb.ndim, n=pb.n, h=pb.h, periodic=pb.periodic, gamma=pb.gamma,
                      bc_lo=tuple(oc(k) for k in pb.bc_lo), bc_hi=tuple(oc(k) for k in pb.bc_hi),
                      bc_state=pb.bc_state, gravity=pb.gravity)


def cpu_oracle_rate(pb, budget_s=12.0):
    """The FP64 oracle as it stands, on whole grid lines of the same state:
    grows the sampled fraction of lines (repeating the whole grid when that
    is quicker) until about budget_s of CPU work."""
    import numpy as np
    from oracle import oracle as O
    cfg = ora_cfg_for(pb)
    U = pb.U0
    L = np.zeros_like(U)
    lines = [pb.cells // pb.n[d] for d in range(pb.ndim)]
    frac = min(1.0, 2000.0 / max(lines))
    total_t = 0.0
    total_cells = 0.0
    while True:
        t0 = time.perf_counter()
        cells = 0.0
        for d in range(pb.ndim):
            k = max(1, int(lines[d] * frac))
            O.euler_rhs_lines(cfg, U, L, d, 0, k)
            cells += k * pb.n[d] / pb.ndim   # a cell-update = all ndim directions
        dt = time.perf_counter() - t0
        total_t += dt
        total_cells += cells
        if total_t >= budget_s:
            break
        # grow the sample; a whole grid that is quicker than the budget repeats
        frac = min(1.0, frac * max(2.0, (budget_s - total_t) / max(dt, 1e-3) * 0.9))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return total_cells / total_t, cores, total_t, total_cells


# ---------------------------------------------------------------- main arms
def dist_setup(backend="nccl"):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local


def max_over_ranks(seconds, world, device):
    """The slowest rank's time (every rank gets it): the replicas are
    independent, so this timing reduction is the only collective."""
    import torch
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, evals, world, seconds):
    """Cell-updates per second of all ranks together (weak scaling: every
    rank advances its own replica of the same size)."""
    return cells_per_rank * evals * world / seconds


def reference_arm(args, world, rank):
    """The oracle (plain FP64 CPU code) timed on this host's cores on the same
    workload; each step a bounded sample of grid lines."""
    pb, cfg, _ = workload(args.workload)
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    ocfg = ora_cfg_for(pb)
    L = np.zeros_like(pb.U0)
    lines = [pb.cells // pb.n[d] for d in range(pb.ndim)]
    per_step_budget = max(0.2, 150.0 / max(1, args.steps + args.warmup))
    # calibrate the fraction of lines per step
    frac = min(1.0, 512.0 / max(lines))
    t0 = time.perf_counter()
    for d in range(pb.ndim):
        O.euler_rhs_lines(ocfg, pb.U0, L, d, 0, max(1, int(lines[d] * frac)))
    t1 = time.perf_counter() - t0
    frac = min(1.0, frac * per_step_budget / max(t1, 1e-4))
    ks = [max(1, int(lines[d] * frac)) for d in range(pb.ndim)]
    cells_per_step = sum(ks[d] * pb.n[d] for d in range(pb.ndim)) / pb.ndim
    for _ in range(args.warmup):
        for d in range(pb.ndim):
            O.euler_rhs_lines(ocfg, pb.U0, L, d, 0, ks[d])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for d in range(pb.ndim):
            O.euler_rhs_lines(ocfg, pb.U0, L, d, 0, ks[d])
    el = time.perf_counter() - t0
    value = cells_per_step * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = "%s: first %s grid lines per direction per step (%.3g cell-updates/step), FP64 oracle" % (
        cfg["workload"], "/".join(str(k) for k in ks), cells_per_step)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(cfg, precision="fp64 (CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def time_steps(torch, solver, U, steps):
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        solver.step(U)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def ours_arm(args, world, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1810_07806_gb300 import wcns

    torch.cuda.set_device(local)
    pb, cfg, fp32 = workload(args.workload)
    if args.precision != "auto":
        fp32 = args.precision == "fp32"
        cfg["precision"] = "fp32 bulk (fp64 reductions + accumulation)" if fp32 else "fp64"
    dev = torch.device("cuda", local)
    solver = wcns.Solver.for_problem(pb, precision=wcns.FP32 if fp32 else wcns.FP64, cfl=0.5)
    U = torch.from_numpy(pb.U0).to(dev)
    nodes = pb.cells
    tiles = solver.autotune(U) if fp32 else [0] * pb.ndim   # pencil-tile shapes for this grid
    for _ in range(args.warmup):
        solver.step(U)
    torch.cuda.synchronize()

    # e2e: the C-ABI call on a HOST state (wcns_step_rk3_host copies it in,
    # steps, copies it out and synchronises), one call per step
    nbytes = U.numel() * U.element_size()
    Uh = torch.from_numpy(pb.U0.copy()).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    solver.step_host(Uh)            # first call: the device copy and the step graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.step_host(Uh)
    e2e_el = time.perf_counter() - t0
    e2e_el = max_over_ranks(e2e_el, world, dev)
    e2e = {"value": whole_job_rate(nodes, 3 * e2e_steps, world, e2e_el), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": e2e_steps, "call": "wcns_step_rk3_host (pinned host state)"}
    solver.step(U)                  # the device state's step graph again, before the timed steps
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    solver.profile(True)
    if world > 1:
        dist.barrier()
    el = time_steps(torch, solver, U, args.steps)
    if world > 1:
        dist.barrier()
    sweep_ms, sweep_n = solver.profile_read()
    solver.profile(False)
    clk = clocks.stop()

    el = max_over_ranks(el, world, dev)
    evals = 3 * args.steps
    value = whole_job_rate(nodes, evals, world, el)

    # dominant kernel: the fused sweep of one direction.  Algorithmic work of
    # one launch: one face and one node difference per node (recomputed halo
    # faces are implementation work, not counted), and 1/ndim of an RHS
    # evaluation's bytes (read U once, write L once: 2 nv w per cell).
    nd = pb.ndim
    pk = device_peaks(local)
    avg_ms = sweep_ms / max(1, sweep_n)
    flops_launch = nodes * (FACE_FLOPS[nd] + NODE_FLOPS[nd])
    achieved_tflops = flops_launch / (avg_ms / 1e3) / 1e12
    peak = pk["fp32_tflops"] if fp32 else pk["fp64_tflops"]
    traffic = profile_traffic(cfg["workload"]) if fp32 else None
    w = 4 if fp32 else 8
    bytes_launch = nodes * pb.nv * w * 2 / nd
    # measured FMA-chain throughput of this GPU, beside the derived peak
    probe = {"fp32": wcns.alu_probe(0), "fp32_packed": wcns.alu_probe(1), "fp64": wcns.alu_probe(2)}
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak, "traffic": traffic,
                "kernel": "sweep_kernel (fused interpolation+flux+MD, one direction)",
                "peak_source": "derived: %d SMs x %s x 2 flops x %.0f MHz" % (
                    pk["sms"], "128 FP32 lanes" if fp32 else "2 FP64 FMA/clk", pk["sm_max_mhz"]),
                "flops_per_launch": flops_launch, "avg_launch_ms": avg_ms, "launches": sweep_n,
                "alu_probe_tflops": probe,
                "hbm": {"algorithmic_bytes_per_launch": bytes_launch,
                        "achieved_gbs": bytes_launch / (avg_ms / 1e3) / 1e9,
                        "peak_gbs": pk["hbm_gbs"], "peak_source": pk["hbm_source"],
                        "frac": bytes_launch / (avg_ms / 1e3) / 1e9 / pk["hbm_gbs"]}}

    # the FP64 plain path on the same workload
    fp64_line = None
    if fp32 and not args.no_fp64:
        s64 = wcns.Solver.for_problem(pb, precision=wcns.FP64, cfl=0.5)
        U64 = torch.from_numpy(pb.U0).to(dev)
        s64.step(U64)
        k64 = max(1, min(3, args.steps))
        el64 = time_steps(torch, s64, U64, k64)
        fp64_line = {"value": nodes * 3 * k64 / el64, "unit": UNIT, "ms_per_step": el64 / k64 * 1e3,
                     "steps": k64, "dtype": "f64"}
        # FP32 bulk vs FP64 (which reproduces the FP64 oracle bit for bit,
        # tests/test_gpu_parity.py): the FP64 path takes CFL steps, the FP32
        # path the same step sizes; relative L1 per variable (momenta against
        # the largest momentum total), the largest over the variables
        Ua = torch.from_numpy(pb.U0).to(dev)
        Ub = torch.from_numpy(pb.U0).to(dev)
        errs = {}
        marks = sorted({3, 20, args.accuracy_steps})
        for k in range(1, args.accuracy_steps + 1):
            dt = s64.step(Ua, 0.0, want_dt=True)
            solver.step(Ub, dt)
            if k in marks:
                d = (Ub - Ua).abs().reshape(pb.nv, -1).sum(dim=1)
                tot = Ua.abs().reshape(pb.nv, -1).sum(dim=1)
                tot[1:-1] = tot[1:-1].max()
                errs[str(k)] = float((d / tot).max())
        fp64_line["fp32_l1_rel_error_vs_fp64_after_steps"] = errs
        fp64_line["fp32_l1_rel_error_3_steps"] = errs.get("3")
        del U64, Ua, Ub
        s64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores, secs, cells = cpu_oracle_rate(pb)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%s: %.3g cell-updates as whole grid lines of every direction, %.1f s" % (
                   cfg["workload"], cells, secs)}

    # the whole run of the paper's finer Rayleigh-Taylor grid, t = 1.95
    rt_run = None
    if args.workload == "rt1024" and rank == 0:
        Ur = torch.from_numpy(pb.U0).to(dev)
        solver.fallback_count(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_reached, nsteps = solver.advance(Ur, pb.t_end, check_every=256)
        secs = time.perf_counter() - t0
        rho = Ur[0].double()
        rt_run = {"t_end": t_reached, "rk3_steps": nsteps, "seconds": secs,
                  "fallback_faces": solver.fallback_count(),
                  "density_range": [float(rho.min()), float(rho.max())],
                  "mirror_asymmetry_max": float((rho - rho.flip(1)).abs().max())}
        del Ur

    # a short bounded replay of the serving configuration (four-quadrant
    # requests, Poisson arrivals at 200/s, half FP32), smaller sides than the
    # full trace so that it takes seconds: served vs the plain path
    serving = None
    if rank == 0 and world == 1 and not args.no_serve and args.workload == "tgv256":
        from paper_1810_07806_gb300 import inputs
        trace = inputs.serving_trace(SERVE_SHORT["requests"], rate=SERVE_SHORT["rate"],
                                     side_lo=SERVE_SHORT["side_lo"], side_hi=SERVE_SHORT["side_hi"])
        served = serve_replay(trace)
        plain = plain_replay(trace)
        serving = {"workload": "serving_four_quadrant_2d_trace (bounded sample: %d requests, side log-uniform "
                               "%d..%d, t_end U[0.1,0.3], 200 req/s, seed 7806, half FP32)" % (
                                   SERVE_SHORT["requests"], SERVE_SHORT["side_lo"], SERVE_SHORT["side_hi"]),
                   **serving_summary(trace, served, plain)}

    launches = solver.launches_per_step(True) * args.steps
    if rank == 0:
        cfg.update({"global_batch": world, "parallelism": "replicas x%d" % world, "tile_configs": tiles,
                    "l2": "inputs larger than L2 (state %.0f MB)" % (nbytes / 1e6)})
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
            "data": "synthetic", "config": cfg, "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "fp64_plain": fp64_line,
            **({"rt_run": rt_run} if rt_run else {}),
            **({"serving": serving} if serving else {}),
        }))
    solver.close()


def batch_arm(args):
    """Batched 1D Euler: 4096 Shu-Osher-type instances (N log-uniform in
    [200, 4000]); one step = one SSP-RK3 step of every instance."""
    import torch
    from paper_1810_07806_gb300 import inputs, wcns
    pbs = inputs.shu_osher_batch(4096)
    nodes = sum(p.cells for p in pbs)
    out = {}
    for name, prec, k in (("fp32", wcns.FP32, args.steps), ("fp64", wcns.FP64, max(1, min(args.steps, 5)))):
        b = wcns.Batch(1, max_nodes=nodes, max_instances=len(pbs), precision=prec)
        for pb in pbs:
            b.add(pb)
        b.step(max(1, args.warmup))
        # launch form (tile table or persistent CTAs) picked by timing both
        mode, ms_modes = b.autotune(steps=3 if prec == wcns.FP64 else 10)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(k)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        out[name] = {"value": nodes * 3 / ms * 1e3, "ms_per_step": ms, "steps": k,
                     "launch_form": ["tile table", "persistent"][mode],
                     "autotune_ms_per_step": {"tile_table": ms_modes[0], "persistent": ms_modes[1]}}
        b.close()
    # the plain path: one instance per launch sequence, FP64, on a subset
    sub = pbs[:64]
    sol = [wcns.Solver.for_problem(pb) for pb in sub]
    Us = [torch.from_numpy(pb.U0.copy()).cuda() for pb in sub]
    for s_, U in zip(sol, Us):
        s_.step(U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        for s_, U in zip(sol, Us):
            s_.step(U)
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / 3
    out["plain_fp64"] = {"value": sum(p.cells for p in sub) * 3 / el, "ms_per_step_64_instances": el * 1e3}
    # FP32 vs FP64 (= the oracle bit for bit) for 64 instances run to t = 0.2
    import numpy as np
    sub = pbs[:64]
    res = {}
    for prec in (wcns.FP32, wcns.FP64):
        b = wcns.Batch(1, max_nodes=sum(p.cells for p in sub), max_instances=len(sub), precision=prec)
        sl = [b.add(pb, t_end=0.2) for pb in sub]
        b.run(check_every=64)
        res[prec] = [b.read(k)[0] for k in sl]
        b.close()
    def rel(a, c):
        tot = np.sum(np.abs(c), axis=1)
        tot[1:-1] = tot[1:-1].max()
        return float(np.max(np.sum(np.abs(a - c), axis=1) / tot))
    errs32 = [rel(a, c) for a, c in zip(res[wcns.FP32], res[wcns.FP64])]
    out["fp32"]["l1_rel_error_vs_fp64_t0.2_64_instances"] = max(errs32)
    # the problem's own sensitivity: the FP64 path (= the oracle) from the
    # initial states perturbed by relative noise of FP32 rounding size
    # (2^-24): where this is as large as the FP32 error, that error is the
    # conditioning of the cut decisions (Eq. 18) at the shocks, not FP32 loss
    rng = np.random.default_rng(24)
    b = wcns.Batch(1, max_nodes=sum(p.cells for p in sub), max_instances=len(sub), precision=wcns.FP64)
    sl = [b.add(pb, U0=pb.U0 * (1.0 + rng.uniform(-1.0, 1.0, pb.U0.shape) * 2.0 ** -24), t_end=0.2) for pb in sub]
    b.run(check_every=64)
    pert = [b.read(k)[0] for k in sl]
    b.close()
    sens = [rel(a, c) for a, c in zip(pert, res[wcns.FP64])]
    out["fp32"]["fp64_response_to_2^-24_input_noise"] = {"max": max(sens), "median": float(np.median(sens))}
    out["fp32"]["fp32_error_median"] = float(np.median(errs32))
    # the smooth counterpart: 4096 density waves (N log-uniform 200..4000),
    # FP32 batch against the FP64 batch (= the oracle) and the plain path
    smooth = inputs.density_wave_batch(4096)
    snodes = sum(p.cells for p in smooth)
    b = wcns.Batch(1, max_nodes=snodes, max_instances=len(smooth), precision=wcns.FP32)
    for pb in smooth:
        b.add(pb, t_end=10.0)       # every instance still running in the timed steps
    b.step(max(1, args.warmup))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    sms = e0.elapsed_time(e1) / args.steps
    b.close()
    ssub = smooth[:64]
    sres = {}
    for prec in (wcns.FP32, wcns.FP64):
        b = wcns.Batch(1, max_nodes=sum(p.cells for p in ssub), max_instances=len(ssub), precision=prec)
        sl = [b.add(pb) for pb in ssub]
        b.run(check_every=64)
        sres[prec] = [b.read(k)[0] for k in sl]
        b.close()
    serr = [rel(a, c) for a, c in zip(sres[wcns.FP32], sres[wcns.FP64])]
    sol = [wcns.Solver.for_problem(pb) for pb in ssub]
    Us = [torch.from_numpy(pb.U0.copy()).cuda() for pb in ssub]
    for s_, U in zip(sol, Us):
        s_.step(U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        for s_, U in zip(sol, Us):
            s_.step(U)
    torch.cuda.synchronize()
    plain_rate = sum(p.cells for p in ssub) * 3 * 3 / (time.perf_counter() - t0)
    smooth_line = {"workload": "4096 periodic density waves, N log-uniform 200..4000, seed 1811",
                   "fp32_batch": {"value": snodes * 3 / sms * 1e3, "ms_per_step": sms},
                   "fp32_l1_rel_error_vs_fp64_t0.2_64_instances": {"max": max(serr),
                                                                  "median": float(np.median(serr))},
                   "plain_fp64_one_instance_per_launch": {"value": plain_rate}}
    # the FP64 oracle on the same instances (all host cores over each
    # instance's lines: one line each in 1D), a bounded sample of RK3 steps
    cpu = None
    if not args.no_cpu:
        from oracle import oracle as O
        t0 = time.perf_counter()
        cells = 0.0
        k = 0
        while time.perf_counter() - t0 < 10.0 and k < len(pbs):
            pb = pbs[k]
            cfg = O.make_cfg(ndim=1, n=pb.n, h=pb.h)
            U = pb.U0.copy()
            for _ in range(5):
                O.rk3_step(cfg, U, O.cfl_dt(cfg, U, 0.5))
            cells += pb.cells * 3 * 5
            k += 1
        secs = time.perf_counter() - t0
        cpu = {"value": cells / secs, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
               "kind": "oracle", "sample": "first %d instances, 5 RK3 steps each, %.1f s" % (k, secs)}
    print(json.dumps({
        "metric": METRIC, "value": out["fp32"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": out["fp32"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched_shu_osher_1d_4096_instances", "nodes": nodes, "seed": 1810,
                   "precision": "fp32 bulk", "launch": "one graph per RK3 step; sweep launch form %s (autotuned)" % (
                       out["fp32"]["launch_form"])},
        "fp32_launch_forms_ms_per_step": out["fp32"]["autotune_ms_per_step"],
        "fp32_l1_rel_error_vs_fp64": out["fp32"]["l1_rel_error_vs_fp64_t0.2_64_instances"],
        "fp32_l1_rel_error_median": out["fp32"]["fp32_error_median"],
        "fp64_response_to_fp32_sized_input_noise": out["fp32"]["fp64_response_to_2^-24_input_noise"],
        "batched_fp64": out["fp64"], "plain_fp64_one_instance_per_launch": out["plain_fp64"],
        "smooth_batch": smooth_line, "cpu_baseline": cpu}))


def serve_replay(trace, steps_per_tick=16):
    """Replays a serving trace in real time against one server: each request
    is submitted at its arrival time, results are polled as they finish.
    Returns per-request results (state, steps, status, latency = result
    ready - arrival), the wall time, queue depths and server statistics."""
    from paper_1810_07806_gb300 import wcns
    sv = wcns.Server(hbm_budget_bytes=64 << 30, max_instances_per_class=64, steps_per_tick=steps_per_tick)
    t0 = time.perf_counter()
    arrivals, work, got, qdepth = {}, {}, {}, []
    k = 0
    while len(got) < len(trace):
        now = time.perf_counter() - t0
        while k < len(trace) and trace[k].arrival_s <= now:
            r = trace[k]
            pb = r.problem()
            sv.submit(pb, tag=k, precision=wcns.FP32 if r.fp32 else wcns.FP64)
            arrivals[k] = time.perf_counter() - t0
            work[k] = pb.cells
            k += 1
        for res in sv.poll(64, timeout_us=2000):
            res["ready"] = time.perf_counter() - t0
            res["latency"] = res["ready"] - arrivals[res["tag"]]
            got[res["tag"]] = res
        qdepth.append(sv.stats()["queued"])
    total = time.perf_counter() - t0
    st = sv.stats()
    sv.close()
    cells = sum(work[i] * 3 * got[i]["steps"] for i in range(len(trace)))
    return {"results": [got[i] for i in range(len(trace))], "wall_s": total, "cell_updates": cells,
            "max_queue": int(max(qdepth) if qdepth else 0), "stats": st}


def plain_replay(trace, fp64_reference=True, ref_max_side=1 << 30):
    """The plain baseline on the same trace: one request at a time, in arrival
    order, each solved alone by the single-grid path in its own precision
    (host state in, wcns_advance, host state out).  Latencies are those of a
    first-come first-served queue in front of it: finish_i = max(arrival_i,
    finish_(i-1)) + solve_i, with the measured solve times.  With
    fp64_reference, the FP64 solution of every FP32 request (the FP64 path
    equals the oracle bit for bit) is computed too, for the FP32 error."""
    import torch
    from paper_1810_07806_gb300 import wcns
    out, ref, ref_time = [], {}, {}
    finish = 0.0
    cells = 0
    busy = 0.0
    for k, r in enumerate(trace):
        pb = r.problem()
        t0 = time.perf_counter()
        s = wcns.Solver.for_problem(pb, precision=wcns.FP32 if r.fp32 else wcns.FP64, cfl=0.5)
        U = torch.from_numpy(pb.U0.copy()).cuda()
        _, steps = s.advance(U, r.t_end, check_every=64)
        Uh = U.cpu().numpy()
        solve = time.perf_counter() - t0
        s.close()
        finish = max(r.arrival_s, finish) + solve
        busy += solve
        cells += pb.cells * 3 * steps
        out.append({"U": Uh, "steps": steps, "latency": finish - r.arrival_s, "solve_s": solve})
        if fp64_reference and r.fp32 and r.side <= ref_max_side:
            t0 = time.perf_counter()
            s = wcns.Solver.for_problem(pb, precision=wcns.FP64, cfl=0.5)
            U = torch.from_numpy(pb.U0.copy()).cuda()
            _, steps64 = s.advance(U, r.t_end, check_every=64)
            ref[k] = U.cpu().numpy()
            ref_time[k] = (time.perf_counter() - t0, pb.cells * 3 * steps64)
            s.close()
    return {"results": out, "busy_s": busy, "cell_updates": cells, "fp64_of_fp32": ref, "fp64_time": ref_time}


def rel_l1(a, c):
    """Relative L1 difference per variable of a against c, the momenta against
    the largest momentum total; the largest over the variables."""
    import numpy as np
    a = a.reshape(a.shape[0], -1)
    c = c.reshape(c.shape[0], -1)
    tot = np.sum(np.abs(c), axis=1)
    tot[1:-1] = tot[1:-1].max()
    return float(np.max(np.sum(np.abs(a - c), axis=1) / tot))


def serving_summary(trace, served, plain):
    """p50/p99 latency and throughput of the served trace beside the plain
    baseline, the FP32 error of served results against the FP64 solution, and
    whether the served FP64 results equal the plain FP64 path (= the oracle)."""
    import numpy as np
    sl = np.array([r["latency"] for r in served["results"]])
    pl = np.array([r["latency"] for r in plain["results"]])
    # requests whose solution left the physical range entirely (non-finite
    # values, in the oracle's arithmetic as well: the FP64 path is the
    # oracle's bit for bit) are counted, not averaged
    finite = {k: bool(np.all(np.isfinite(served["results"][k]["U"]))) for k in range(len(trace))}
    fp32_err = [rel_l1(served["results"][k]["U"], plain["fp64_of_fp32"][k]) for k in plain["fp64_of_fp32"]
                if finite[k] and np.all(np.isfinite(plain["fp64_of_fp32"][k]))]
    fp64_same = all(np.array_equal(served["results"][k]["U"], plain["results"][k]["U"], equal_nan=True)
                    for k, r in enumerate(trace) if not r.fp32)
    fp32_same = all(np.array_equal(served["results"][k]["U"], plain["results"][k]["U"], equal_nan=True)
                    for k, r in enumerate(trace) if r.fp32)
    plain_wall = max(max(r.arrival_s for r in trace), 0.0)
    finish = 0.0
    for r, res in zip(trace, plain["results"]):
        finish = max(r.arrival_s, finish) + res["solve_s"]
    statuses = [r["status"] for r in served["results"]]
    # the FP32 requests that have an FP64 solution: their served share of the
    # wall time is not separable, so the comparison is the plain FP32 path
    # and the plain FP64 path on the same requests, one at a time
    ks = sorted(plain["fp64_time"])
    fp32_vs_fp64 = None
    if ks:
        t32 = sum(plain["results"][k]["solve_s"] for k in ks)
        c32 = sum(trace[k].problem().cells * 3 * plain["results"][k]["steps"] for k in ks)
        t64 = sum(plain["fp64_time"][k][0] for k in ks)
        c64 = sum(plain["fp64_time"][k][1] for k in ks)
        fp32_vs_fp64 = {"requests": len(ks), "plain_fp32_rate": c32 / t32, "plain_fp64_rate": c64 / t64,
                        "speedup": (c32 / t32) / (c64 / t64)}
    return {
        "served": {"value": served["cell_updates"] / served["wall_s"], "unit": UNIT,
                   "latency_s": {"p50": float(np.percentile(sl, 50)), "p99": float(np.percentile(sl, 99)),
                                 "max": float(sl.max())},
                   "wall_s": served["wall_s"], "max_queue": served["max_queue"],
                   "max_running": served["stats"]["max_running"],
                   "status_counts": {str(v): statuses.count(v) for v in sorted(set(statuses))},
                   "non_finite_results": sum(1 for k in finite if not finite[k])},
        "plain_one_at_a_time": {"value": plain["cell_updates"] / finish, "unit": UNIT,
                                "latency_s": {"p50": float(np.percentile(pl, 50)),
                                              "p99": float(np.percentile(pl, 99)), "max": float(pl.max())},
                                "wall_s": finish, "busy_s": plain["busy_s"],
                                "latency_rule": "FCFS queue over measured solve times"},
        "speedup_served_vs_plain": (served["cell_updates"] / served["wall_s"]) / (plain["cell_updates"] / finish),
        "fp32_l1_rel_error_vs_fp64": {"max": max(fp32_err) if fp32_err else None,
                                      "median": float(np.median(fp32_err)) if fp32_err else None,
                                      "requests": len(fp32_err),
                                      "reference": "FP64 path, equal to the FP64 oracle bit for bit"},
        "fp32_requests_fp32_vs_fp64_plain": fp32_vs_fp64,
        "fp64_served_equal_plain_fp64": fp64_same,
        "fp32_served_equal_plain_fp32": fp32_same,
    }


def serve_arm(args):
    """Serving: a seeded Poisson trace of four-quadrant Riemann requests (side
    log-uniform 128..1024, t_end U[0.1, 0.3], half FP32 / half FP64) replayed
    in real time against one server; latency = result ready - arrival.  The
    plain one-request-at-a-time path runs the same trace for comparison."""
    from paper_1810_07806_gb300 import inputs
    trace = inputs.serving_trace(args.requests, rate=args.rate, side_lo=args.side_lo, side_hi=args.side_hi)
    served = serve_replay(trace)
    plain = plain_replay(trace, ref_max_side=args.l1_max_side)
    summ = serving_summary(trace, served, plain)
    print(json.dumps({
        "metric": METRIC, "value": summ["served"]["value"], "unit": UNIT, "n_gpus": 1,
        "steps": int(served["stats"]["steps"]), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serving_four_quadrant_2d_trace", "requests": len(trace), "rate_per_s": args.rate,
                   "seed": 7806, "side": "log-uniform %d..%d" % (args.side_lo, args.side_hi),
                   "t_end": "U[0.1,0.3]", "fp32_share": 0.5,
                   "fp32_error_for_sides_up_to": min(args.l1_max_side, args.side_hi)},
        **summ}))


SCALAR_N, SCALAR_LINES, SCALAR_STEPS_PER_CALL = 1600, 152 * 8, 100
# the serving sample of the default line
SERVE_SHORT = {"requests": 24, "rate": 200.0, "side_lo": 64, "side_hi": 192}


def scalar_lines():
    """Gaussian pulses exp(-300 (x - c)^2) of Table 2's finest grid (N = 1601,
    1600 unique periodic nodes on [0, 1)), centres c ~ U[0.3, 0.7] (seed 1810)."""
    import numpy as np
    h = 1.0 / SCALAR_N
    x = h * np.arange(SCALAR_N)
    c = np.random.default_rng(1810).uniform(0.3, 0.7, (SCALAR_LINES, 1))
    return np.exp(-300.0 * (x[None, :] - c) ** 2), h


def scalar_oracle_rate(h, u, budget_s):
    """The FP64 oracle's scalar solver on one line, steps doubled until about
    budget_s of CPU work; returns node-RHS evaluations per second."""
    from oracle import oracle as O
    cfg = O.make_cfg()
    steps, total_t, total = 8, 0.0, 0.0
    while total_t < budget_s:
        t0 = time.perf_counter()
        O.scalar_run(cfg, 0, u, h, steps * 0.01 * h, steps)
        dt = time.perf_counter() - t0
        total_t += dt
        total += u.size * 3 * steps
        steps *= 2
    return total / total_t, total_t, total


def scalar_arm(args):
    """Scalar path (linear advection, TCNS, FP64): 1216 independent lines of
    Table 2's finest grid; one bench step = 100 SSP-RK3 steps of every line
    in one launch (dt = 0.01 h).  Also the time to reproduce Table 2's
    N = 1601 TCNS entry (t = 1, 160000 steps) on one line."""
    import numpy as np
    import torch
    from paper_1810_07806_gb300 import wcns
    U0, h = scalar_lines()
    nodes = U0.size
    k = SCALAR_STEPS_PER_CALL
    t_call = k * 0.01 * h
    dev = torch.device("cuda", 0)
    U = torch.from_numpy(U0).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        wcns.scalar_run(wcns.SCALAR_ADVECTION, U, h, t_call, k)
    torch.cuda.synchronize()
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0])
    clocks.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        wcns.scalar_run(wcns.SCALAR_ADVECTION, U, h, t_call, k)
        e1.record()
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = total_ms / args.steps
    value = nodes * 3 * k / ms * 1e3
    # end to end: host state in, k steps, host state out, every bench step
    host = torch.from_numpy(U0.copy()).pin_memory()
    out = torch.empty_like(host).pin_memory()
    Ud = torch.empty_like(U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Ud.copy_(host, non_blocking=True)
        wcns.scalar_run(wcns.SCALAR_ADVECTION, Ud, h, t_call, k)
        out.copy_(Ud, non_blocking=True)
        torch.cuda.synchronize()
    e2e = nodes * 3 * k * args.steps / (time.perf_counter() - t0)
    nbytes = U0.size * 8
    # Table 2, N = 1601, TCNS, t = 1 on one line
    x = h * np.arange(SCALAR_N)
    u0 = np.exp(-300.0 * (x - 0.5) ** 2)
    one = torch.from_numpy(u0.copy()).to(dev)
    nsteps = int(math.ceil(1.0 / (0.01 * h)))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    wcns.scalar_run(wcns.SCALAR_ADVECTION, one, h, 1.0, nsteps)
    e1.record()
    torch.cuda.synchronize()
    t2_ms = e0.elapsed_time(e1)
    t2_err = float(np.max(np.abs(one.cpu().numpy() - u0)))
    achieved = value * SCALAR_NODE_FLOPS / 1e12
    pk = device_peaks(0)
    cpu = None
    if not args.no_cpu:
        rate, secs, work = scalar_oracle_rate(h, u0, 10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one 1600-node line, %.3g node-RHS evaluations in %.1f s (the scalar oracle "
                         "is single-threaded)" % (work, secs)}
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gaussian_advection_1d_periodic_%dx%d_lines" % (SCALAR_LINES, SCALAR_N),
                   "weights": "tcns", "rk3_steps_per_bench_step": k, "dt": "0.01 h",
                   "l2": "flushed (256 MiB write) between timed steps",
                   "launch": "one cluster launch per bench step (16-CTA clusters, line resident in DSMEM)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / pk["fp64_tflops"], "traffic": None,
                     "kernel": "scalar_kernel (whole run on chip)",
                     "flops_per_node_rhs": SCALAR_NODE_FLOPS,
                     "peak_note": "FP64 FMA peak derived from %d SMs x 2 FP64 FMA/clk x 2 flops x %.0f MHz; "
                                  "the fixed-order path issues no FMA, so 0.5 is its ceiling" % (
                                      pk["sms"], pk["sm_max_mhz"])},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": args.steps, "clocks": clk,
        "table2_n1601_tcns": {"ms": t2_ms, "rk3_steps": nsteps, "linf_error": t2_err,
                              "printed": 3.64e-9},
    }))


def scalar_reference_arm(args):
    """The oracle's scalar solver on this host, each bench step a bounded
    sample (one line, a few RK3 steps) of the same workload."""
    U0, h = scalar_lines()
    from oracle import oracle as O
    cfg = O.make_cfg()
    budget = max(0.2, 150.0 / max(1, args.steps + args.warmup))
    steps = 4
    t0 = time.perf_counter()
    O.scalar_run(cfg, 0, U0[0], h, steps * 0.01 * h, steps)
    steps = max(1, int(steps * budget / max(time.perf_counter() - t0, 1e-4)))
    for _ in range(args.warmup):
        O.scalar_run(cfg, 0, U0[0], h, steps * 0.01 * h, steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.scalar_run(cfg, 0, U0[0], h, steps * 0.01 * h, steps)
    el = time.perf_counter() - t0
    value = SCALAR_N * 3 * steps * args.steps / el
    sample = "one %d-node line, %d RK3 steps per bench step, FP64 oracle (single thread)" % (SCALAR_N, steps)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "gaussian_advection_1d_periodic_%dx%d_lines" % (SCALAR_LINES, SCALAR_N),
                   "weights": "tcns", "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.workload == "scalar":
        if int(os.environ.get("RANK", "0")) == 0:
            (scalar_arm if args.impl == "ours" else scalar_reference_arm)(args)
        return
    if args.workload == "batch1d" and args.impl == "ours":
        return batch_arm(args)
    if args.workload == "serve" and args.impl == "ours":
        return serve_arm(args)
    if args.impl == "reference":
        # the reference arm runs on rank 0's host cores only; other ranks exit
        rank = int(os.environ.get("RANK", "0"))
        if rank == 0:
            reference_arm(args, int(os.environ.get("WORLD_SIZE", "1")), 0)
        return
    world, rank, local = dist_setup()
    ours_arm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
