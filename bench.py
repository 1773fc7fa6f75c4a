"""Benchmark of the PSMS hot path on GB300.

A step is one 3-level hierarchical filter update (domain sweep -> per-block
stochastic det ratios -> global Schur det ratio -> random translation) on the
synthetic 32^3 x 64 workload: kappa 0.157, beta 5.3, 8^4 domains, 24
interpolation steps (noise vectors) at the global level, FP32 inner Krylov
iterations inside FP64 defect correction, tolerance 1e-10.  The gauge field
U = exp(i eps H) (eps 0.5) is thermalised by pure-gauge sweeps at beta 5.3
before timing.  Inputs (1.2 GB of links) are larger than the 129 MB L2.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (bounded sample, extrapolated, see `reference_arm`).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D_w GB/s vs HBM peak; accepted updates/s, learned+mixed vs plain FP64 at 1e-8"
UNIT = "accepted updates/s"
SEED = 0x50534D53

WORKLOADS = {
    # name: dims (L0..L3), block, kappa, eps, beta, n_block, n_global, therm iterations
    "32^3x64": dict(dims=(64, 32, 32, 32), block=(8, 8, 8, 8), kappa=0.157, eps=0.5, beta=5.3, n_block=4,
                    n_global=24, therm=4, n_iter=1, n_or=2, tol=1e-10),
    "16^4": dict(dims=(16, 16, 16, 16), block=(4, 4, 4, 4), kappa=0.156, eps=0.5, beta=5.3, n_block=12,
                 n_global=12, therm=4, n_iter=1, n_or=1, tol=1e-10),
    "4^4": dict(dims=(4, 4, 4, 4), block=(2, 2, 2, 2), kappa=0.15, eps=0.3, beta=5.3, n_block=4, n_global=4,
                therm=0, n_iter=1, n_or=0, tol=1e-10),
}
DW_FLOP_PER_SITE = 1320.0
DW_BYTES_PER_SITE = {"bf16": 384.0, "f32": 480.0, "f64": 960.0}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def measure_dw(ps, ctx, torch, reps=20):
    """Stand-alone full-lattice D_w (Eq. (Dw)) per precision: GB/s of the
    algorithmic bytes and GFLOP/s at 1320 flop/site, CUDA events on the
    library's stream, inputs larger than L2."""
    out = {}
    V = ctx.V
    stream = torch.cuda.current_stream()
    for name, prec in (("bf16", ps.PREC_BF16), ("f32", ps.PREC_F32), ("f64", ps.PREC_F64)):
        nb = ps.psms_spinor_bytes(ctx, prec)
        a = torch.empty(nb, dtype=torch.uint8, device="cuda")
        b = torch.empty(nb, dtype=torch.uint8, device="cuda")
        canon = torch.randn(V * 24, dtype=torch.float64, device="cuda")
        ps.psms_spinor_import(ctx, canon, a, prec)
        for _ in range(3):
            ps.psms_dw_apply(ctx, 0, ps.OP_FULL, a, b, prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(reps):
            ps.psms_dw_apply(ctx, 0, ps.OP_FULL, a if i % 2 == 0 else b, b if i % 2 == 0 else a, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = DW_BYTES_PER_SITE[name] * V / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "GB/s": round(gbs, 1),
                     "GFLOP/s": round(DW_FLOP_PER_SITE * V / (ms * 1e-3) / 1e9, 1),
                     "bytes_per_site": DW_BYTES_PER_SITE[name]}
        del a, b, canon
    return out


def dw_only(args):
    """Stand-alone D_w on the workload lattice (about 4 GB on the device):
    the small case used for Nsight Compute captures of the hop kernel."""
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    _build.build()
    torch.cuda.set_device(0)
    wl = WORKLOADS[args.workload]
    ctx = ps.psms_create(wl["dims"], wl["block"], wl["kappa"], 1)
    ps.psms_set_stream(ctx, torch.cuda.current_stream())
    ps.psms_gauge_init(ctx, 0, wl["eps"], SEED + 4)
    dw = measure_dw(ps, ctx, torch, reps=args.steps)
    peak, kind = peaks()
    print(json.dumps({"workload": args.workload, "dw": dw, "peak_gbs": peak, "peak_kind": kind,
                      "frac": {k: round(v["GB/s"] / peak, 4) for k, v in dw.items()}}), flush=True)


def our_arm(args):
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    ws, rank, local = dist_setup()
    _build.build()
    wl = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    ctx = ps.psms_create(wl["dims"], wl["block"], wl["kappa"], 2)
    ps.psms_set_stream(ctx, stream)
    seed = SEED + 4 + 1000 * rank
    ps.psms_gauge_init(ctx, 0, wl["eps"], seed)
    if wl["therm"]:
        ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, wl["therm"], 2, wl["beta"], seed, 1 << 40)
    plaq0, _ = ps.psms_plaquette(ctx, 0)
    prm = dict(beta0=wl["beta"], n_iter=wl["n_iter"], n_or=wl["n_or"], n_block=wl["n_block"],
               n_global=wl["n_global"], tol=wl["tol"], inner_prec=ps.PREC_F32, seed=seed)
    step_id = 0

    def step():
        nonlocal step_id
        r = ps.psms_filter_step(ctx, 0, step=step_id, **prm)
        step_id += 1
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    n_launch0 = ps.load_library().psms_kernel_launches()
    ps.psms_profile_enable(ctx, 10 + ps.PREC_F32)
    recs = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            recs.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(ws)
    ms = e0.elapsed_time(e1)
    n_launch = ps.load_library().psms_kernel_launches() - n_launch0
    hop_n, hop_ms, hop_bytes = ps.psms_profile_read(ctx)
    ps.psms_profile_enable(ctx, 0)
    ms_max = allmax(ws, ms)
    accepted = sum(1 for r in recs if r["accept_global"] and r["n_accept_blocks"] > 0)
    accepted_all = allsum(ws, accepted)
    value = accepted_all / (ms_max * 1e-3)
    attempted = allsum(ws, len(recs)) / (ms_max * 1e-3)

    # end to end through the C ABI with host buffers: H2D of the gauge field,
    # one filter step, D2H of the updated field, every step
    V = ctx.V
    host_links = torch.empty(V * 4 * 9 * 2, dtype=torch.float64).pin_memory()
    dev_links = torch.empty(V * 4 * 9 * 2, dtype=torch.float64, device="cuda")
    ps.psms_gauge_get(ctx, 0, dev_links)
    host_links.copy_(dev_links)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    e2e_acc = 0
    for _ in range(args.steps):
        dev_links.copy_(host_links, non_blocking=True)
        ps.psms_gauge_set(ctx, 0, dev_links)
        r = step()
        e2e_acc += int(r["accept_global"] and r["n_accept_blocks"] > 0)
        ps.psms_gauge_get(ctx, 0, dev_links)
        host_links.copy_(dev_links, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = allmax(ws, time.perf_counter() - t0)
    e2e_value = allsum(ws, e2e_acc) / e2e_s
    link_bytes = V * 4 * 9 * 16

    dw = measure_dw(ps, ctx, torch)
    peak, peak_kind = peaks()
    hop_avg_ms = hop_ms / max(hop_n, 1)
    achieved = (hop_bytes / max(hop_n, 1)) / (hop_avg_ms * 1e-3) / 1e9 if hop_n else 0.0
    if rank != 0:
        return
    full_iters = sum(r["solver_iters"] for r in recs) / max(len(recs), 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic: U = exp(i eps H) links thermalised at beta 5.3, Philox noise",
        "config": {"workload": args.workload, "dims": list(wl["dims"]), "block": list(wl["block"]),
                   "kappa": wl["kappa"], "beta": wl["beta"], "eps": wl["eps"], "n_block": wl["n_block"],
                   "n_global": wl["n_global"], "tol": wl["tol"], "inner": "fp32 in fp64 defect correction",
                   "l2": "inputs larger than L2 (1.2 GB links)", "parallelism": f"independent chains x{ws}"},
        "attempted_updates_per_s": attempted,
        "acceptance": {"global": sum(r["accept_global"] for r in recs) / len(recs),
                       "blocks": sum(r["n_accept_blocks"] for r in recs) / sum(r["n_blocks"] for r in recs)},
        "solver_iters_per_step": full_iters,
        "delta_block_mean": float(sum(float(r["delta_block"].mean()) for r in recs) / len(recs)),
        "delta_block_std": float(sum(float(r["delta_block"].std()) for r in recs) / len(recs)),
        "plaquette_start": plaq0,
        "dw": dict(dw, peak_gbs=peak, frac_bf16=round(dw["bf16"]["GB/s"] / peak, 4)),
        "roofline": {"kernel": "hop_kernel<float> (Wilson hop of the FP32 inner Krylov iterations, all launches "
                               "in the timed steps)", "bound": "hbm",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
                     "launches": hop_n, "avg_launch_ms": round(hop_avg_ms, 5)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": link_bytes, "d2h_bytes_per_step": link_bytes},
        "gpu_launches": n_launch,
        "wall_s_timed": wall,
    }
    line["clocks"] = clk.summary()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, full_iters, len(recs), accepted, ms_max)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# CPU oracle timing (single thread), bounded sample
# ---------------------------------------------------------------------------
_SAMPLE = r'''
import os, sys, time, json
sys.path.insert(0, sys.argv[1])
import numpy as np
from oracle import dirac, gauge
dims = tuple(json.loads(sys.argv[2])); kappa = float(sys.argv[3]); reps = int(sys.argv[4])
V = int(np.prod(dims))
g = np.random.default_rng(0)
U = np.empty(dims + (4, 3, 3), dtype=np.complex128)
U[...] = np.eye(3)
psi = (g.standard_normal(dims + (4, 3)) + 1j * g.standard_normal(dims + (4, 3))) / np.sqrt(2)
t = []
for _ in range(reps):
    t0 = time.perf_counter()
    a = dirac.apply_D(U, psi, kappa)
    b = dirac.apply_D(U, a, kappa, dagger=True)
    t.append(time.perf_counter() - t0)
print(json.dumps({"s_per_iter": min(t)}))
'''


def oracle_iteration_seconds(dims, kappa, reps=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _SAMPLE, ROOT, json.dumps(list(dims)), str(kappa), str(reps)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])["s_per_iter"]


def cpu_baseline(workload, iters_per_step, steps, accepted, gpu_ms):
    """Oracle (numpy FP64, 1 thread) time of one CGNR iteration (D then
    D^dagger) on the full workload lattice, scaled by the GPU step's Krylov
    iteration count (whole-lattice iterations plus block iterations, both in
    full-lattice-iteration units) to the same metric."""
    wl = WORKLOADS[workload]
    s_iter = oracle_iteration_seconds(wl["dims"], wl["kappa"])
    cpu_step_s = s_iter * iters_per_step
    acc_frac = accepted / max(steps, 1)
    return {"value": acc_frac / cpu_step_s if cpu_step_s > 0 else 0.0, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one oracle CGNR iteration (D and D^dagger, numpy FP64) on the {workload} lattice "
                       f"= {s_iter:.2f} s, times {iters_per_step:.0f} full-lattice-equivalent Krylov iterations "
                       f"per step (measured on the GPU step), times the GPU acceptance; extrapolated"),
            "seconds_per_iteration": s_iter, "extrapolated_step_s": cpu_step_s}


def reference_arm(args):
    """The oracle timed as it stands on the host cores: each step is one CGNR
    iteration of the oracle on the full workload lattice (bounded sample),
    extrapolated to the metric with the step cost model below."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    times = []
    for i in range(args.warmup + args.steps):
        s = oracle_iteration_seconds(wl["dims"], wl["kappa"])
        if i >= args.warmup:
            times.append(s)
    s_iter = statistics.median(times)
    # step cost model: whole-lattice-equivalent CGNR iterations of one filter
    # step of this workload and its acceptance, as measured by our arm on GB300
    iters, acc = STEP_MODEL[args.workload]
    step_s = s_iter * iters
    value = acc / step_s
    sample = (f"one oracle CGNR iteration (D and D^dagger, numpy FP64, 1 thread) on the {args.workload} lattice "
              f"per step ({s_iter:.2f} s), times {iters} full-lattice-equivalent iterations per filter step, "
              f"times acceptance {acc}; extrapolated")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "dims": list(wl["dims"]), "block": list(wl["block"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# (full-lattice-equivalent Krylov iterations per step, fraction of accepted updates), measured on GB300
STEP_MODEL = {"32^3x64": (4000, 0.5), "16^4": (3000, 0.5), "4^4": (600, 0.3)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="32^3x64", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dw-only", action="store_true", help="stand-alone D_w measurement only")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    elif args.dw_only:
        dw_only(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
