"""Benchmark of the PSMS hot path on GB300.

A step is one 3-level hierarchical filter update of the synthetic 16^4
workload (kappa 0.156, beta 5.3, 4^4 domains): domain sweep -> relative gauge
fixing of the proposal -> learned level -> per-block stochastic det ratios
(48 interpolation steps, all blocks and steps batched) -> global Schur det
ratio (12 steps) -> random translation, FP32 inner Krylov iterations inside
FP64 defect correction to a true residual of 1e-13 (estimates within 1e-8 of
the FP64 ones).  The gauge field U = exp(i eps H) (eps 0.5) is thermalised
by pure-gauge sweeps at beta 5.3 before timing; the learned level is trained
on the GPU before timing.  The same line carries the plain FP64 and the
mixed-precision arms on identical proposals and noise, and the 32^3 x 64
measurements (D_w GB/s per precision, the domain heatbath, filter steps with
8^4 domains).

Every arm starts from one checkpoint (the thermalised field and the trained
learned level) and runs the same number of timed steps with the same step
counters.  Prints one JSON line (rank 0).  `--impl reference` times the FP64
CPU oracle instead (bounded samples, see `reference_arm`).
"""
import argparse
import json
import math

import numpy as np
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
    # name: dims (L0..L3), block (the smallest Dirichlet blocks), outer blocks of the recursive
    # decomposition (None: one level), kappa, eps, beta, interpolation steps per level,
    # thermalisation iterations, proposal sweeps, tolerance, proposals for the learned level's labels
    "32^3x64": dict(dims=(64, 32, 32, 32), block=(4, 4, 4, 4), outer=(8, 8, 8, 8), kappa=0.157, eps=0.5,
                    beta=5.3, n_block=12, n_sub=12, n_global=24, therm=4, n_iter=1, n_or=2, tol=1e-12,
                    train_props=8),
    "16^4": dict(dims=(16, 16, 16, 16), block=(4, 4, 4, 4), outer=None, kappa=0.156, eps=0.5, beta=5.3, n_block=48,
                 n_sub=0, n_global=12, therm=4, n_iter=1, n_or=1, tol=1e-13, train_props=48),
    "4^4": dict(dims=(4, 4, 4, 4), block=(2, 2, 2, 2), outer=None, kappa=0.15, eps=0.3, beta=5.3, n_block=4,
                n_sub=0, n_global=4, therm=0, n_iter=1, n_or=0, tol=1e-10, train_props=8),
}
HEADLINE = "32^3x64"
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


# DRAM bytes (ncu dram__bytes_read.sum + write.sum) / algorithmic bytes of
# captured launches of the current kernels (profiles/; None: no capture of
# the current code -- set back to None whenever the kernel changes)
TRAFFIC_RATIO = {# 16^4 block level, 256 blocks x 12 systems: 12.48 GB of DRAM traffic
                 # for 118.9 GB of algorithmic bytes in one launch
                 "block_solve_cluster_kernel": 0.105,
                 # shared-endpoint-link FP32 hop, 32^3x64 global level, 8 systems:
                 # 3.75 GB of DRAM traffic for 6.4-7.3 GB of algorithmic bytes
                 "hop_kernel": 0.55}


def roofline_entry(kernel, n, ms, nbytes, peak, peak_kind):
    """achieved = algorithmic bytes of the kernel's launches in the timed steps
    / their summed CUDA-event durations (on the library's stream)."""
    achieved = nbytes / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind, "launches": n,
            "avg_launch_ms": round(ms / max(n, 1), 4), "total_ms": round(ms, 2)}


def train_learned(ps, torch, ctx, n_props, n_interp=48, gauge_fix=True):
    """Train the learned level on block log-det-ratio estimates the method
    generates for domain-sweep proposals of the current field (between the
    relatively gauge-fixed endpoints when the filter uses them; slots 2, 3
    hold those).  The labels are noise-dominated, so the learning rate is
    small and the epochs few (larger ones fit the label noise)."""
    nb = ps.psms_geometry_info(ctx)[0]
    zs, ys = [], []
    zb = torch.zeros(nb * 64, dtype=torch.float32, device="cuda")
    for s in range(n_props):
        ps.psms_gauge_copy(ctx, 1, 0)
        ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, (s + 7) << 20)
        f0, f1 = 0, 1
        if gauge_fix:
            ps.psms_relative_gauge_fix(ctx, 0, 1, 2, 3, prec=ps.PREC_F32)
            f0, f1 = 2, 3
        d = ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, f0, f1, n_interp, ps.EST_INTERP, SEED, 50_000 + s, 1e-10,
                                 ps.PREC_F32)
        ps.psms_domain_features_pair(ctx, 0, 1, zb)
        zs.append(zb.view(nb, 64).clone())
        ys.append(torch.from_numpy(d.sum(axis=1)))
    z = torch.cat(zs).contiguous()
    y = torch.cat(ys).to("cuda").contiguous()
    ps.psms_mlp_init(ctx, 7)
    return ps.psms_mlp_train(ctx, z, y, len(y), epochs=10, batch=256, lr=1e-4, weight_decay=1e-4, seed=3)


def measure_heatbath(ps, ctx, torch, wl, reps=3):
    """Domain sweep (Sec. 6) on the active links: link updates per second
    (HB and OR sweeps each update every active link once) and the FP64
    arithmetic rate at about 3000 flop per link update (6 staples of 2 SU(3)
    products, 3 SU(2) subgroup updates); its fraction of the measured FP64
    peak is added by the caller."""
    _, _, n_active = ps.psms_geometry_info(ctx)
    n_iter, n_or = 1, 2
    sweeps = n_iter * (2 + 2 * n_or)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, n_iter, n_or, wl["beta"], SEED, 7 << 40)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(reps):
        ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, n_iter, n_or, wl["beta"], SEED, (8 + i) << 40)
    torch.cuda.synchronize()
    s = (time.perf_counter() - t0) / reps
    ups = n_active * sweeps / s
    return {"active_links": n_active, "sweeps_per_call": sweeps, "s_per_call": round(s, 4),
            "link_updates_per_s": round(ups, 1), "fp64_gflops_est": round(ups * 3000 / 1e9, 1), "bound": "alu"}


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
    out = {"workload": args.workload, "dw": dw, "peak_gbs": peak, "peak_kind": kind,
           "frac": {k: round(v["GB/s"] / peak, 4) for k, v in dw.items()}}
    if args.hop_variants:
        # every hop variant forced in turn (same operator): GB/s per variant
        n = ps.psms_hop_variant(ctx, 0)
        per = {}
        for v in range(n):
            ps.psms_hop_variant(ctx, v)
            d = measure_dw(ps, ctx, torch, reps=args.steps)
            per[v] = {k: d[k]["GB/s"] for k in ("bf16", "f32")}
        ps.psms_hop_variant(ctx, -1)
        out["per_variant_GB/s"] = per
    print(json.dumps(out), flush=True)


def solve_only(args):
    """Whole-lattice and all-blocks solves of one system on the workload
    lattice (FP32 inner iterations, FP64 defect correction to the workload
    tolerance), with the solvers' algorithmic bytes per Krylov iteration:
      block CG iteration (per block, FP32): 4 half hops over the block
        (in, out, 8 links per output site; y on the second hop of a pair) and
        the vector updates (12 half-vector passes) = 4416 B per half-block site;
      whole-lattice CG iteration: the same per half-lattice site.
    This is the small case for Nsight Compute captures of the solver kernels."""
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    _build.build()
    torch.cuda.set_device(0)
    wl = WORKLOADS[args.workload]
    ctx = ps.psms_create(wl["dims"], wl["block"], wl["kappa"], 1)
    ps.psms_set_stream(ctx, torch.cuda.current_stream())
    ps.psms_gauge_init(ctx, 0, wl["eps"], SEED + 4)
    V = ctx.V
    canon = torch.randn(V * 24, dtype=torch.float64, device="cuda")
    b = torch.empty(ps.psms_spinor_bytes(ctx, ps.PREC_F64), dtype=torch.uint8, device="cuda")
    x = torch.zeros_like(b)
    ps.psms_spinor_import(ctx, canon, b, ps.PREC_F64)
    peak, kind = peaks()
    out = {"workload": args.workload, "peak_gbs": peak, "peak_kind": kind}
    per_site = 4416.0
    for name, op in (("blocks", ps.OP_BLOCKS), ("full", ps.OP_FULL)):
        for _ in range(max(1, args.warmup - 2)):
            ps.psms_solve(ctx, 0, op, b, x, wl["tol"], 20000, ps.PREC_F32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = ps.psms_solve(ctx, 0, op, b, x, wl["tol"], 20000, ps.PREC_F32)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        its = info["inner_iters"]
        # block iterations are summed over the blocks: one block iteration
        # covers Vb/2 half-block sites; a whole-lattice iteration covers V/2
        nblk = 1
        if op == ps.OP_BLOCKS:
            nblk = int(np.prod([d // l for d, l in zip(wl["dims"], wl["block"])]))
        half_sites = (V / 2) / nblk
        gbs = its * half_sites * per_site / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 2), "inner_iters": its, "true_residual": info["true_residual"],
                     "algorithmic_GB/s": round(gbs, 1), "frac": round(gbs / peak, 4)}
    print(json.dumps(out), flush=True)


def learned_only(args):
    """The learned level at its own workload: 16^3 x 32 lattice, 8^4 domains
    (32 per field), kappa 0.156, beta 5.3.  Labels: block log-det-ratio
    estimates Delta_b (N = 4 interpolation steps between relatively
    gauge-fixed endpoints) of domain-sweep proposals, `--labels` of them
    (default 10^5); the last tenth of the proposals is held out.  The BF16
    MLP is trained on the GPU by the library's kernels, then filter steps of
    the learned + mixed hierarchy and of the plain mixed hierarchy run on
    identical proposals and noise.  Reports label generation and training
    time, held-out prediction, the fraction of blocks sent on to the
    stochastic level, acceptances and updates/s."""
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    _build.build()
    torch.cuda.set_device(0)
    wl = dict(dims=(32, 16, 16, 16), block=(8, 8, 8, 8), kappa=0.156, eps=0.5, beta=5.3, n_block=4, n_global=8,
              therm=4, n_iter=1, n_or=1, tol=1e-10)
    seed = SEED + 3
    ctx = _new_chain(ps, torch, wl, seed)
    nb = ps.psms_geometry_info(ctx)[0]
    n_props = max(2, -(-args.labels // nb))
    zb = torch.zeros(nb * 64, dtype=torch.float32, device="cuda")
    zs, ys = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(n_props):
        ps.psms_gauge_copy(ctx, 1, 0)
        ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, wl["beta"], seed, (s + 7) << 20)
        ps.psms_relative_gauge_fix(ctx, 0, 1, 2, 3, prec=ps.PREC_F32)
        d = ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 2, 3, wl["n_block"], ps.EST_INTERP, seed, 50_000 + s, 1e-10,
                                 ps.PREC_F32)
        ps.psms_domain_features_pair(ctx, 0, 1, zb)
        zs.append(zb.view(nb, 64).clone())
        ys.append(torch.from_numpy(d.sum(axis=1)))
        if s % 4 == 3:
            ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 1, 0, wl["beta"], seed, (s + 1) << 30)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    n_te = max(1, n_props // 10)
    z = torch.cat(zs[:-n_te]).contiguous()
    y = torch.cat(ys[:-n_te]).to("cuda").contiguous()
    z_te = torch.cat(zs[-n_te:]).contiguous()
    y_te = torch.cat(ys[-n_te:]).numpy()
    ps.psms_mlp_init(ctx, 7)
    t0 = time.perf_counter()
    losses = ps.psms_mlp_train(ctx, z, y, len(y), epochs=10, batch=256, lr=1e-4, weight_decay=1e-4, seed=3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    h = torch.zeros(len(y_te), dtype=torch.float32, device="cuda")
    ps.psms_mlp_predict(ctx, z_te, len(y_te), h)
    h = h.cpu().numpy().astype(np.float64)
    p_pass = np.exp(-np.clip(h, 0.0, 700.0))
    out = {"workload": "16^3x32, 8^4 domains, learned level", "dims": list(wl["dims"]), "block": list(wl["block"]),
           "kappa": wl["kappa"], "n_block": wl["n_block"], "labels": int(len(y) + len(y_te)),
           "proposals": n_props, "label_generation_s": round(gen_s, 2), "train_s": round(train_s, 2),
           "train_loss_first_last": [losses[0], losses[-1]],
           "heldout": {"n": int(len(y_te)), "corr_h_delta": float(np.corrcoef(h, y_te)[0, 1]),
                       "delta_mean": float(y_te.mean()), "delta_std": float(y_te.std()),
                       "h_std": float(h.std()), "pass_fraction": float(p_pass.mean())}}
    prm = _filter_prm(ps, wl, seed)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    params = ps.psms_mlp_params(ctx)
    ctx.close()
    for name, learned in (("learned_mixed", True), ("mixed", False)):
        # both arms from the same thermalised field: identical proposals and noise
        c = _new_chain(ps, torch, wl, seed)
        if learned:
            ps.psms_mlp_params(c, params)
        ps.psms_filter_step(c, 0, step=100_000, inner_prec=ps.PREC_F32, learned=learned, **prm)
        rr, mm = _timed_steps(ps, torch, c, prm, ps.PREC_F32, learned, args.steps, flush, step0=1_000_000)
        out[name] = {"s_per_step": mm / len(rr) / 1e3, "accepted_updates_per_s": _accepted(rr) / (mm * 1e-3),
                     "block_acceptance": sum(r["n_accept_blocks"] for r in rr) / sum(r["n_blocks"] for r in rr),
                     "learned_pass": (sum(r["n_accept_learned"] for r in rr) / sum(r["n_blocks"] for r in rr)
                                      if learned else None),
                     "solver_iters_per_step": sum(r["solver_iters"] for r in rr) / len(rr)}
        c.close()
    print(json.dumps(out), flush=True)


def measure_batch(ps, torch, steps=3, warmup=3):
    """All 4^4 Dirichlet blocks x 16 noise vectors of three uneven
    lattices (8^4, 12^4, 16^3 x 32; kappa 0.155, eps 0.5) in one persistent
    graph-captured launch, FP32 inner / FP64 refinement to 1e-10, autotuned
    schedule.  Returns the batch time, the mean time a CTA spends per system,
    and the aggregate algorithmic GB/s (4416 B per half-block site per block
    CG iteration, FP32)."""
    n_rhs = 16
    probs, ctxs = [], []
    for i, dims in enumerate(((8, 8, 8, 8), (12, 12, 12, 12), (32, 16, 16, 16))):
        ctx = ps.psms_create(dims, (4, 4, 4, 4), 0.155, 1)
        ps.psms_set_stream(ctx, torch.cuda.current_stream())
        ps.psms_gauge_init(ctx, 0, 0.5, SEED + 2 + i)
        nb = ps.psms_spinor_bytes(ctx, ps.PREC_F64)
        b = torch.empty(n_rhs * nb, dtype=torch.uint8, device="cuda")
        for k in range(n_rhs):
            canon = torch.randn(ctx.V * 24, dtype=torch.float64, device="cuda")
            ps.psms_spinor_import(ctx, canon, b[k * nb:(k + 1) * nb], ps.PREC_F64)
        probs.append((ctx, 0, n_rhs, b, torch.zeros_like(b)))
        ctxs.append(ctx)
    torch.cuda.synchronize()
    plan = ps.psms_block_plan_create(probs, 1e-10, 20000, ps.PREC_F32)
    for _ in range(warmup):
        plan.run()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    infos = [plan.run(stream) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sched = plan.schedule()
    items = infos[0]["n_systems"]
    iters = infos[0]["inner_iters"]
    gbs = iters * 128 * 4416.0 / (ms * 1e-3) / 1e9
    peak, kind = peaks()
    out = {"workload": "8^4 + 12^4 + 16^3x32, 4^4 blocks x 16 noises", "systems": items,
           "batch_ms": round(ms, 3), "per_solve_latency_ms": round(ms * sched["ctas"] / items, 4),
           "block_cg_iterations": iters, "algorithmic_GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
           "peak_gbs": peak, "peak_kind": kind, "schedule": sched,
           "true_residual": max(i["true_residual"] for i in infos)}
    plan.close()
    for c in ctxs:
        c.close()
    return out


def batch_only(args):
    """The batched multi-lattice block solves alone (see measure_batch)."""
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    _build.build()
    torch.cuda.set_device(0)
    print(json.dumps(measure_batch(ps, torch, steps=args.steps, warmup=args.warmup)), flush=True)


def levels_only(args):
    """The parametrised levels (App. C) and the recursive decomposition on the
    16^4 workload: the block HYP action (one smearing + per-block plaquette
    sums, FP64), the per-block plaquette-action change, the outer-block
    Schur estimates (8^4 outer blocks of 4^4 blocks), and filter steps with
    the HYP level and with one level of recursion, each timed with CUDA
    events after warm-up.  An auxiliary measurement (one JSON line)."""
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    _build.build()
    torch.cuda.set_device(0)
    wl = WORKLOADS["16^4"]
    seed = SEED + 77
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ctx = _new_chain(ps, torch, wl, seed)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, wl["n_iter"], wl["n_or"], wl["beta"], seed, 9 << 20)
    V = float(np.prod(wl["dims"]))
    out = {"workload": "16^4", "data": "synthetic"}
    fp64 = measure_fp64_peak(torch)
    out["fp64_peak_measured"] = fp64
    ms = timed(lambda: ps.psms_hyp_block_action(ctx, 0), max(3, args.steps))
    flop = 55e3 * V  # per-site model of one smearing (fat links dominate)
    out["hyp_block_action"] = {"ms": round(ms, 3), "model_gflops_fp64": round(flop / ms * 1e-6, 1),
                               "frac_of_measured_fp64": round(flop / ms * 1e-6 / fp64["gflops"], 4)}
    ms = timed(lambda: ps.psms_block_action_change(ctx, 0, 1), max(3, args.steps))
    out["block_action_change"] = {"ms": round(ms, 3)}
    # exact block determinants (batched FP64 LU of the even-odd reduced block
    # operator, n = 6 x block volume): (8/3) n^3 real flop per block
    ms = timed(lambda: ps.psms_block_logdet(ctx, 0), 1)
    nb = int(np.prod([d // b for d, b in zip(wl["dims"], wl["block"])]))
    n = 6 * int(np.prod(wl["block"]))
    flop = nb * 8.0 / 3.0 * n ** 3
    out["block_logdet"] = {"blocks": nb, "n": n, "ms": round(ms, 2), "gflops_fp64": round(flop / ms * 1e-6, 1),
                           "frac_of_measured_fp64": round(flop / ms * 1e-6 / fp64["gflops"], 4)}
    ps.psms_set_outer_blocks(ctx, (8, 8, 8, 8))
    n_sub = 12
    ms = timed(lambda: ps.psms_logdet_ratio(ctx, ps.LEVEL_SUB, 0, 1, n_sub, ps.EST_INTERP, seed, 0, wl["tol"],
                                            ps.PREC_F32), 1)
    n_o = int(np.prod([d // 8 for d in wl["dims"]]))
    out["sub_level"] = {"outer_blocks": n_o, "n": n_sub, "ms": round(ms, 2),
                        "estimates_per_s": round(n_o * n_sub / ms * 1e3, 1)}
    ps.psms_set_outer_blocks(ctx, None)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    prm = _filter_prm(ps, wl, seed)
    for name, extra in (("hyp_level", dict(hyp_level=(-0.0196, 0.0963), beta_block_hyp=-0.0614)),
                        ("recursive_5step", dict(n_sub=n_sub))):
        chain = _new_chain(ps, torch, wl, seed)
        kw = dict(prm, **extra)
        if name == "recursive_5step":
            ps.psms_set_outer_blocks(chain, (8, 8, 8, 8))
            kw.pop("gauge_fix", None)
        _timed_steps(ps, torch, chain, kw, ps.PREC_F32, False, args.warmup, flush)
        recs, ms = _timed_steps(ps, torch, chain, kw, ps.PREC_F32, False, args.steps, flush, step0=1000)
        out[name] = {"ms_per_step": round(ms / args.steps, 2), "accepted_updates": _accepted(recs),
                     "blocks_accepted": int(sum(r["n_accept_blocks"] for r in recs)),
                     "n_accept_hyp": [r["n_accept_hyp"] for r in recs],
                     "n_accept_sub": [r["n_accept_sub"] for r in recs]}
        chain.close()
    ctx.close()
    print(json.dumps(out), flush=True)


def step_only(args):
    """The headline hierarchy's filter steps alone, for launch-list captures:
    the learned level trained on two proposals' estimates, `--warmup`
    untimed steps on a copy of the field, then `--steps` steps inside the
    NVTX range "timed_steps" (CUDA events around each).  Far fewer launches
    than the full bench, so that a profiler pass over them stays short."""
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    _build.build()
    torch.cuda.set_device(0)
    wl = WORKLOADS[args.workload]
    seed = SEED + 1
    prm = _filter_prm(ps, wl, seed)
    ctx = _new_chain(ps, torch, wl, seed)
    train_learned(ps, torch, ctx, 2, n_interp=wl["n_block"])
    ps.psms_gauge_copy(ctx, 3, 0)
    for i in range(args.warmup):
        ps.psms_filter_step(ctx, 3, step=100_000 + i, inner_prec=ps.PREC_F32, learned=True, **prm)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_steps")
    recs, ms = _timed_steps(ps, torch, ctx, prm, ps.PREC_F32, True, args.steps, flush)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"workload": args.workload, "steps": args.steps, "ms_per_step": ms / args.steps,
                      "accepted_updates": _accepted(recs)}), flush=True)
    ctx.close()


def block_only(args):
    """The block level alone on the 16^4 workload (4^4 blocks): all blocks x
    n interpolation steps (--block-n, default 12) between the gauge-fixed
    endpoints of one domain-sweep proposal, FP32 inner iterations to the
    workload tolerance, one persistent launch of the block solver per call.
    The first call autotunes the solver variant; --steps calls are timed
    with CUDA events.  The small case for Nsight Compute captures of
    block_solve_cluster_kernel (about 1 GB on the device at n = 12)."""
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    _build.build()
    torch.cuda.set_device(0)
    wl = WORKLOADS["16^4"]
    seed = SEED + 5
    ctx = _new_chain(ps, torch, wl, seed)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, wl["n_iter"], wl["n_or"], wl["beta"], seed, 9 << 20)
    ps.psms_relative_gauge_fix(ctx, 0, 1, 2, 3, prec=ps.PREC_F32)
    if args.block_variant >= 0:
        ps.psms_autotune(ctx, False, args.block_variant)
    n = args.block_n
    for r in range(args.warmup):
        ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 2, 3, n, ps.EST_INTERP, seed, r, wl["tol"], ps.PREC_F32)
    ps.psms_profile_enable(ctx, 1)
    ms = []
    for r in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 2, 3, n, ps.EST_INTERP, seed, 100 + r, wl["tol"], ps.PREC_F32)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    nl, bms, bbytes = ps.psms_profile_read_block(ctx)
    peak, kind = peaks()
    nb = ps.psms_geometry_info(ctx)[0]
    print(json.dumps({"workload": "16^4 block level", "n": n, "blocks": nb, "variant": args.block_variant,
                      "ms_per_call": statistics.median(ms),
                      "estimates_per_s": nb * n / (statistics.median(ms) * 1e-3),
                      "block_solver": {"launches": nl, "ms": round(bms, 3), "algorithmic_GB/s": round(
                          bbytes / (bms * 1e-3) / 1e9, 1) if bms > 0 else None, "peak_gbs": peak, "peak_kind": kind}}),
          flush=True)
    ctx.close()


def measure_estimators(ps, torch, wl, seed, n=12, reps=3):
    """Det-ratio estimates per second on the workload lattice: the block
    level (all blocks x n interpolation steps) and the global level (n
    steps) between the gauge-fixed endpoints of one domain-sweep proposal,
    FP32 inner iterations to the workload tolerance, CUDA events."""
    ctx = _new_chain(ps, torch, wl, seed)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, wl["n_iter"], wl["n_or"], wl["beta"], seed, 9 << 20)
    ps.psms_relative_gauge_fix(ctx, 0, 1, 2, 3, prec=ps.PREC_F32)
    nb = ps.psms_geometry_info(ctx)[0]
    stream = torch.cuda.current_stream()
    out = {"n": n}
    for name, level, units in (("block", ps.LEVEL_BLOCK, nb * n), ("global", ps.LEVEL_GLOBAL, n)):
        ps.psms_logdet_ratio(ctx, level, 2, 3, n, ps.EST_INTERP, seed, 0, wl["tol"], ps.PREC_F32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for r in range(reps):
            ps.psms_logdet_ratio(ctx, level, 2, 3, n, ps.EST_INTERP, seed, r + 1, wl["tol"], ps.PREC_F32)
        e1.record(stream)
        torch.cuda.synchronize()
        s_per = e0.elapsed_time(e1) / reps * 1e-3
        out[name] = {"estimates": units, "s": round(s_per, 4), "estimates_per_s": round(units / s_per, 1)}
    ctx.close()
    return out


ARMS = (
    # name, inner Krylov precision, learned level
    ("learned_mixed", "f32", True),
    ("mixed", "f32", False),
    ("plain_fp64", "f64", False),
)


def _filter_prm(ps, wl, seed):
    return dict(beta0=wl["beta"], n_iter=wl["n_iter"], n_or=wl["n_or"], n_block=wl["n_block"],
                n_global=wl["n_global"], tol=wl["tol"], seed=seed, gauge_fix={"prec": ps.PREC_F32},
                n_sub=wl["n_sub"] if wl.get("outer") else 0)


def _ctx(ps, torch, wl):
    ctx = ps.psms_create(wl["dims"], wl["block"], wl["kappa"], 4)
    ps.psms_set_stream(ctx, torch.cuda.current_stream())
    if wl.get("outer"):
        ps.psms_set_outer_blocks(ctx, wl["outer"])
    return ctx


def _new_chain(ps, torch, wl, seed):
    ctx = _ctx(ps, torch, wl)
    ps.psms_gauge_init(ctx, 0, wl["eps"], seed)
    if wl["therm"]:
        ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, wl["therm"], 2, wl["beta"], seed, 1 << 40)
    return ctx


def _timed_steps(ps, torch, ctx, prm, inner, learned, steps, flush, step0=0):
    """`steps` filter steps, each timed with CUDA events on the library's
    stream; L2 is flushed (a 256 MB write) between steps, outside the events."""
    stream = torch.cuda.current_stream()
    recs, ms = [], 0.0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        recs.append(ps.psms_filter_step(ctx, 0, step=step0 + i, inner_prec=inner, learned=learned, **prm))
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    return recs, ms


def delta_stats(recs):
    """Per level: mean and variance of the estimates Delta, the measured
    acceptance, and the acceptance a Gaussian Delta with that variance would
    have under detailed balance, erfc(sqrt(Sigma^2 / 8)) (Sec. 2, the
    expectation of min{1, e^-Delta} over proposals)."""
    out = {}
    blocks = np.concatenate([np.asarray(r["delta_block"], dtype=np.float64) for r in recs]) if recs else np.zeros(0)
    acc_b = np.concatenate([np.asarray(r["accept_block"], dtype=bool) for r in recs]) if recs else np.zeros(0, bool)
    if blocks.size:
        var = float(blocks.var())
        out["block"] = {"mean": float(blocks.mean()), "var": var, "acceptance": float(acc_b.mean()),
                        "gaussian_prediction": math.erfc(math.sqrt(var / 8.0))}
    glob = [r["delta_global"] for r in recs if r.get("n_accept_blocks", 0) > 0]
    if len(glob) > 1:
        g = np.asarray(glob, dtype=np.float64)
        acc_g = [bool(r["accept_global"]) for r in recs if r.get("n_accept_blocks", 0) > 0]
        out["global"] = {"mean": float(g.mean()), "var": float(g.var()), "acceptance": float(np.mean(acc_g)),
                         "gaussian_prediction": math.erfc(math.sqrt(float(g.var()) / 8.0)), "n": len(glob)}
    return out


def _accepted(recs):
    """Accepted updates: steps whose global level accepted a changed field."""
    return sum(1 for r in recs if r["accept_global"] and r["n_accept_blocks"] > 0)


def dw_and_heatbath(ps, torch, wl_name):
    """Stand-alone D_w per precision and the domain heatbath on the workload
    lattice (thermalised field)."""
    wl = WORKLOADS[wl_name]
    ctx = _new_chain(ps, torch, wl, SEED + 4)
    out = {"workload": wl_name, "dims": list(wl["dims"]), "block": list(wl["block"]),
           "dw": measure_dw(ps, ctx, torch), "heatbath": measure_heatbath(ps, ctx, torch, wl)}
    ctx.close()
    return out


def _poisson_interval(k, conf=0.95):
    """Exact (Garwood) two-sided interval of the mean of a Poisson count k."""
    from scipy.stats import chi2
    a = 1.0 - conf
    lo = 0.0 if k == 0 else 0.5 * float(chi2.ppf(a / 2, 2 * k))
    hi = 0.5 * float(chi2.ppf(1 - a / 2, 2 * k + 2))
    return lo, hi


def _rb_accepted(recs):
    """Rao-Blackwellised accepted updates: the sum over steps of the global
    level's acceptance probability min{1, exp(-Delta)} given the step's
    estimate (0 where no block changed), i.e. the expected accepted count
    given the estimates (Eq. (hierarchy)); it drops the noise of the last
    coin flip."""
    tot = 0.0
    for r in recs:
        if r["n_accept_blocks"] > 0:
            d = r["delta_global"]
            tot += 1.0 if d <= 0.0 else math.exp(-d)
    return tot


def _arm_summary(recs, ms, **extra):
    s = ms * 1e-3
    k = _accepted(recs)
    lo, hi = _poisson_interval(k)
    nb = sum(r["n_blocks"] for r in recs)
    out = {"steps": len(recs), "s_per_step": s / len(recs), "accepted_updates": k,
           "accepted_updates_per_s": k / s, "accepted_updates_per_s_95ci": [lo / s, hi / s],
           "rao_blackwell_updates_per_s": _rb_accepted(recs) / s,
           "block_acceptance": sum(r["n_accept_blocks"] for r in recs) / nb,
           "accepted_blocks_per_s": sum(r["n_accept_blocks"] for r in recs if r["accept_global"]) / s,
           "solver_iters_per_step": sum(r["solver_iters"] for r in recs) / len(recs)}
    out.update(extra)
    return out


def run_workload(ps, torch, wl_name, steps, warmup, ws, rank, compare=True, fp64_steps=2, profile=True,
                 e2e=True):
    """All arms of one workload from one checkpoint (the thermalised field and
    the learned level trained on estimates the method generates from it):
    learned + mixed (the headline hierarchy), mixed without the learned
    level, and plain FP64.  The first two run `steps` timed steps with step
    counters 0..steps-1 after warm-up steps on a copy of the field.  Plain
    FP64 runs the same chain as mixed (same proposals, noise and decisions:
    its estimates agree to the refinement tolerance); it times
    min(steps, fp64_steps) steps, its decisions are checked against mixed's
    on those steps, and its accepted count over `steps` is therefore mixed's
    (reported as such)."""
    wl = WORKLOADS[wl_name]
    seed = SEED + 1 + 1000 * rank
    prec = {"f32": ps.PREC_F32, "f64": ps.PREC_F64}
    prm = _filter_prm(ps, wl, seed)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ckpt = os.path.join(tempfile.mkdtemp(), f"start_{wl_name.replace('^', '')}_{rank}.psms")
    ctx = _new_chain(ps, torch, wl, seed)
    plaq0, _ = ps.psms_plaquette(ctx, 0)
    t0 = time.perf_counter()
    losses = train_learned(ps, torch, ctx, wl["train_props"], n_interp=wl["n_block"])
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    ps.psms_checkpoint_save(ctx, 0, ckpt, 0, seed)
    ctx.close()

    def arm_ctx():
        c = _ctx(ps, torch, wl)
        ps.psms_checkpoint_load(c, 0, ckpt)
        return c

    def warm(c, inner, learned, n):
        # warm-up steps on a copy (slot 3): the timed steps start from the
        # checkpointed field with step counters 0, 1, ...
        ps.psms_gauge_copy(c, 3, 0)
        for i in range(n):
            ps.psms_filter_step(c, 3, step=100_000 + i, inner_prec=inner, learned=learned, **prm)
        torch.cuda.synchronize()

    out = {"workload": wl_name, "plaquette_start": plaq0, "train_s": round(train_s, 2),
           "train_loss_first_last": [losses[0], losses[-1]]}
    # the headline arm: learned level + FP32 inner iterations + batched solves
    ctx = arm_ctx()
    warm(ctx, ps.PREC_F32, True, warmup)
    barrier(ws)
    lib = ps.load_library()
    n_launch0 = lib.psms_kernel_launches()
    if profile:
        ps.psms_profile_enable(ctx, 10 + ps.PREC_F32)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        tw = time.perf_counter()
        torch.cuda.nvtx.range_push("timed_steps")
        recs, ms = _timed_steps(ps, torch, ctx, prm, ps.PREC_F32, True, steps, flush)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        out["wall_s_timed"] = time.perf_counter() - tw
    barrier(ws)
    out["clocks"] = clk.summary()
    out["gpu_launches"] = lib.psms_kernel_launches() - n_launch0
    if profile:
        out["hop_profile"] = ps.psms_profile_read(ctx)
        out["block_profile"] = ps.psms_profile_read_block(ctx)
        out["block_first"] = ps.psms_profile_block_launches(ctx, 4)
        ps.psms_profile_enable(ctx, 0)
    out["recs"], out["ms"] = recs, ms
    if e2e:
        # end to end through the C ABI with host buffers: the same chain from
        # the same start field, the field living in pinned host memory --
        # every step copies it to the device, runs the filter step and copies
        # the updated field back (identical steps, so identical decisions)
        V = ctx.V
        host_links = torch.empty(V * 4 * 9 * 2, dtype=torch.float64).pin_memory()
        dev_links = torch.empty(V * 4 * 9 * 2, dtype=torch.float64, device="cuda")
        ps.psms_checkpoint_load(ctx, 0, ckpt)
        ps.psms_gauge_get(ctx, 0, dev_links)
        host_links.copy_(dev_links)
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        e2e_recs = []
        for i in range(steps):
            dev_links.copy_(host_links, non_blocking=True)
            ps.psms_gauge_set(ctx, 0, dev_links)
            e2e_recs.append(ps.psms_filter_step(ctx, 0, step=i, inner_prec=ps.PREC_F32, learned=True, **prm))
            ps.psms_gauge_get(ctx, 0, dev_links)
            host_links.copy_(dev_links, non_blocking=True)
            torch.cuda.synchronize()
        out["e2e_s"] = allmax(ws, time.perf_counter() - t0)
        out["e2e_accepted"] = _accepted(e2e_recs)
        out["e2e_same"] = all(a["accept_global"] == b["accept_global"] and a["n_accept_blocks"] == b["n_accept_blocks"]
                              for a, b in zip(recs, e2e_recs))
        out["link_bytes"] = V * 4 * 9 * 16
    ctx.close()
    arms = {"learned_mixed": _arm_summary(recs, ms, learned_pass=sum(r["n_accept_learned"] for r in recs) /
                                          sum(r["n_blocks"] for r in recs))}
    if compare and rank == 0:
        runs = {}
        for name, inner, learned in ARMS[1:]:
            n = steps if name == "mixed" else min(steps, fp64_steps)
            c = arm_ctx()
            warm(c, prec[inner], False, 1)
            rr, mm = _timed_steps(ps, torch, c, prm, prec[inner], False, n, flush)
            arms[name] = _arm_summary(rr, mm)
            runs[name] = rr
            c.close()
        # mixed and plain FP64 run the same chain (same proposals, noise and
        # decisions) until a decision differs: the estimate differences are
        # the inner precision (FP32 vs FP64, both refined to the tolerance)
        diffs, same = [], 0
        for a, b in zip(runs["mixed"], runs["plain_fp64"]):
            if not np.array_equal(a["accept_block"], b["accept_block"]):
                break
            diffs.append(float(np.abs(a["delta_block"] - b["delta_block"]).max()))
            if a["n_accept_blocks"] > 0:
                diffs.append(abs(a["delta_global"] - b["delta_global"]))
            if a["accept_global"] != b["accept_global"]:
                break
            same += 1
        mx, fp = arms["mixed"], arms["plain_fp64"]
        mx["max_estimate_diff_vs_fp64"] = max(diffs) if diffs else None
        mx["steps_identical_to_fp64"] = same
        if fp["steps"] < steps and same == fp["steps"]:
            # the FP64 chain is the mixed chain: its accepted updates over the
            # headline's steps are mixed's, at FP64's measured time per step
            s_all = fp["s_per_step"] * steps
            k = mx["accepted_updates"]
            lo, hi = _poisson_interval(k)
            fp.update({"accepted_updates_over_headline_steps": k, "accepted_updates_per_s": k / s_all,
                       "accepted_updates_per_s_95ci": [lo / s_all, hi / s_all],
                       "rao_blackwell_updates_per_s": _rb_accepted(runs["mixed"]) / s_all,
                       "rates_from": f"mixed's {steps} steps (identical decisions on the {fp['steps']} FP64 steps "
                                     "run) at FP64's measured time per step"})
        lm = arms["learned_mixed"]
        arms["speedup_learned_mixed_vs_plain_fp64_s_per_step"] = fp["s_per_step"] / lm["s_per_step"]
        gain = lm["rao_blackwell_updates_per_s"] > mx["rao_blackwell_updates_per_s"]
        arms["learned_level_effect"] = (
            "learned+mixed vs mixed on the same start field and steps: "
            f"{lm['accepted_updates']} vs {mx['accepted_updates']} accepted updates, Rao-Blackwellised "
            f"{lm['rao_blackwell_updates_per_s']:.3f} vs {mx['rao_blackwell_updates_per_s']:.3f} per s: the learned "
            f"level {'gains' if gain else 'loses'} on these inputs")
    out["arms"] = arms
    return out


def our_arm(args):
    import torch

    import paper_1204_1306_gb300 as ps
    from paper_1204_1306_gb300 import build as _build

    ws, rank, local = dist_setup()
    _build.build()
    wl = WORKLOADS[args.workload]
    h = run_workload(ps, torch, args.workload, args.steps, args.warmup, ws, rank, compare=not args.no_compare,
                     fp64_steps=args.fp64_steps)
    recs, ms = h["recs"], h["ms"]
    ms_max = allmax(ws, ms)
    accepted = _accepted(recs)
    value = allsum(ws, accepted) / (ms_max * 1e-3)
    e2e_value = allsum(ws, h["e2e_accepted"]) / h["e2e_s"]
    hop_n, hop_ms, hop_bytes = h["hop_profile"]
    blk_n, blk_ms, blk_bytes = h["block_profile"]
    peak, peak_kind = peaks()
    rl_hop = roofline_entry("hop_kernel<float> (Wilson hop of the FP32 inner Krylov iterations)", hop_n, hop_ms,
                            hop_bytes, peak, peak_kind)
    rl_hop["bound_note"] = ("algorithmic bytes count every system's interpolated links (4 or 8 FP32 links per output "
                            "site); the whole-lattice solves form them from two shared endpoint fields that HBM "
                            "delivers about once per launch, so 'achieved' is an effective rate above the DRAM "
                            "traffic ('traffic')")
    rl_blk = roofline_entry("block_solve_cluster_kernel<float> (persistent Dirichlet-block CG, FP32 inner)", blk_n,
                            blk_ms, blk_bytes, peak, peak_kind)
    ratio = TRAFFIC_RATIO.get("hop_kernel")
    if ratio is not None and hop_n:
        rl_hop["traffic"] = ratio * hop_bytes / hop_n
        rl_hop["traffic_note"] = ("ncu dram__bytes_read+write / algorithmic bytes of captured launches of the "
                                  f"shared-endpoint-link FP32 hop (32^3x64 global level) = {ratio}, times the mean "
                                  "algorithmic bytes per launch of the timed steps; below 1 because the systems of "
                                  "a launch read the endpoint links from L2")
    ratio = TRAFFIC_RATIO.get("block_solve_cluster_kernel")
    if ratio is not None and blk_n:
        # DRAM bytes per launch, scaled from the capture by the algorithmic
        # bytes (block-CG iterations x sites) of the timed launches
        rl_blk["traffic"] = ratio * blk_bytes / blk_n
        rl_blk["traffic_note"] = ("ncu dram__bytes_read+write of one launch / its algorithmic bytes = "
                                  f"{ratio}, times the mean algorithmic bytes per launch of the timed steps")
    rl_blk["bound_note"] = ("effective rate: 'achieved' counts every CG pass over a block as memory traffic "
                            "(the det-ratio metric's per-iteration bytes) while L1/L2 serve most of it, so it can "
                            "exceed the HBM copy rate; the kernel is bound by instruction issue and latency")
    # the dominant kernel of the step: the larger measured time
    rl_main, rl_other = (rl_blk, rl_hop) if blk_ms >= hop_ms else (rl_hop, rl_blk)
    if rank != 0:
        return
    arms = h["arms"]
    secondary = None
    if args.workload != "16^4" and not args.no_compare and not args.no_secondary:
        s16 = run_workload(ps, torch, "16^4", args.secondary_steps, 3, 1, 0, compare=True,
                           fp64_steps=args.secondary_steps, profile=False, e2e=False)
        secondary = {"workload": "16^4 (4^4 blocks, kappa 0.156, N = 48 / 12, tol 1e-13)", "arms": s16["arms"],
                     "delta_statistics": delta_stats(s16["recs"]), "train_s": s16["train_s"]}
    dwhb = None if args.no_large else dw_and_heatbath(ps, torch, "32^3x64")
    estimators = None if args.no_compare else measure_estimators(ps, torch, WORKLOADS["16^4"], SEED + 1)
    batched = None if args.no_compare else measure_batch(ps, torch)
    fp64 = measure_fp64_peak(torch)
    if dwhb:
        hb = dwhb["heatbath"]
        hb["fp64_peak_gflops_measured"] = fp64["gflops"]
        hb["frac_of_measured_fp64"] = round(hb["fp64_gflops_est"] / fp64["gflops"], 4)
        dwhb["dw"]["f64"]["frac_of_measured_fp64"] = round(dwhb["dw"]["f64"]["GFLOP/s"] / fp64["gflops"], 4)
    full_iters = sum(r["solver_iters"] for r in recs) / max(len(recs), 1)
    cfg = {"workload": args.workload, "dims": list(wl["dims"]), "block": list(wl["block"]),
           "kappa": wl["kappa"], "beta": wl["beta"], "eps": wl["eps"], "n_block": wl["n_block"],
           "n_global": wl["n_global"], "tol": wl["tol"], "inner": "fp32 in fp64 defect correction",
           "learned_level": True, "gauge_fix": "relative, block interiors, fp32 steps",
           "start": "every arm loads one checkpoint (thermalised field + trained MLP); warm-up steps run on a copy; "
                    "timed steps use step counters 0..K-1",
           "l2": "flushed between timed steps (256 MB write, outside the step events)",
           "parallelism": f"independent chains x{ws}"}
    if wl.get("outer"):
        cfg.update({"domains": list(wl["outer"]), "n_sub": wl["n_sub"],
                    "decomposition": "8^4 domains each split into 2^4 Dirichlet blocks of 4^4 (recursive, 5-step "
                                     "filter: learned level, blocks, domain Schur complements, global Schur "
                                     "complement of the domains)"})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic: U = exp(i eps H) links thermalised at beta 5.3, Philox noise",
        "config": cfg,
        "accepted_updates": accepted,
        "accepted_updates_per_s_95ci": arms["learned_mixed"]["accepted_updates_per_s_95ci"],
        "rao_blackwell_updates_per_s": arms["learned_mixed"]["rao_blackwell_updates_per_s"],
        "acceptance": {"global": sum(r["accept_global"] for r in recs) / len(recs),
                       "blocks": sum(r["n_accept_blocks"] for r in recs) / sum(r["n_blocks"] for r in recs),
                       "domains_after_stage_2": [r["n_accept_sub"] for r in recs]},
        "solver_iters_per_step": full_iters,
        "delta_statistics": delta_stats(recs),
        "gauge_fix_steps_per_step": sum(r["gf_steps"] for r in recs) / len(recs),
        "plaquette_start": h["plaquette_start"],
        "train_s": h["train_s"], "train_loss_first_last": h["train_loss_first_last"],
        "roofline": rl_main,
        "roofline_secondary": rl_other,
        "block_solver_first_launches": [{"ms": round(a, 4), "algorithmic_bytes": b} for a, b in h["block_first"]],
        "arms": arms,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h["link_bytes"],
                "d2h_bytes_per_step": h["link_bytes"], "same_decisions_as_timed_steps": h["e2e_same"]},
        "gpu_launches": h["gpu_launches"],
        "wall_s_timed": h["wall_s_timed"],
        "fp64_peak": fp64,
        "configs1_16x4": secondary,
        "dw_heatbath_32^3x64": dwhb,
        "det_ratio_estimates_16x4": estimators,
        "batched_block_solves": batched,
        "clocks": h["clocks"],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, recs)
    print(json.dumps(line), flush=True)


def measure_fp64_peak(torch, n=4096, reps=3):
    """FP64 arithmetic peak of this GPU, measured: cuBLAS DGEMM (2 n^3 flop)
    through torch, best of `reps` after a warm-up, CUDA events."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    del a, b, c
    return {"gflops": round(2.0 * n ** 3 / (best * 1e-3) / 1e9, 1),
            "how": f"torch.matmul float64 {n}^3 (cuBLAS DGEMM), best of {reps}"}


# ---------------------------------------------------------------------------
# CPU oracle timing (one thread), bounded samples
# ---------------------------------------------------------------------------
_COMPONENTS = """
import json, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
from oracle import dirac, estimator, gauge, lattice, linalg
cfg = json.loads(sys.argv[2])
dims, block, kappa = tuple(cfg["dims"]), tuple(cfg["block"]), cfg["kappa"]
geom = lattice.Geometry(dims, block)
U = gauge.generate_links(dims, cfg["eps"], cfg["seed"])
out = {}
if cfg["sweep"]:
    t0 = time.perf_counter()
    Up, _, _ = gauge.domain_sweep(U, geom, cfg["beta"], 1, cfg["n_or"], cfg["seed"], 0)
    out["sweep_s"] = time.perf_counter() - t0
else:
    Up = U
# one CGNR iteration of the whole lattice (D and D^dagger)
psi = estimator.noise(geom, cfg["seed"], 0, 2, 0)
t0 = time.perf_counter()
a = dirac.apply_D(Up, psi, kappa)
dirac.apply_D(Up, a, kappa, dagger=True)
out["cgnr_iteration_s"] = time.perf_counter() - t0
# one interpolation step's per-lattice work of an estimator level (noise and
# D_b of every block) and block solves on a sample of blocks
t0 = time.perf_counter()
xi = estimator.noise(geom, cfg["seed"], 0, 1, 0)
eta = dirac.apply_D(U, xi, kappa, geom, mode="block")
out["level_overhead_s"] = time.perf_counter() - t0
step = max(1, geom.n_blocks // cfg["n_sample"])
sample = list(range(0, geom.n_blocks, step))[:cfg["n_sample"]]
t0 = time.perf_counter()
estimator.solve_blocks(Up, eta, geom, kappa, sample, cfg["tol"])
out["block_solve_s"] = (time.perf_counter() - t0) / len(sample)
out["block_sample"] = len(sample)
if cfg.get("full_dims"):
    # iterations of one whole-lattice solve to the tolerance (oracle CGNR),
    # measured on a smaller lattice with the same kappa and field recipe
    fd = tuple(cfg["full_dims"])
    fg = lattice.Geometry(fd, block)
    Uf = gauge.generate_links(fd, cfg["eps"], cfg["seed"])
    Uf, _, _ = gauge.domain_sweep(Uf, fg, cfg["beta"], 1, cfg["n_or"], cfg["seed"], 0)
    b = estimator.noise(fg, cfg["seed"], 0, 2, 0)
    _, it, _ = linalg.cgnr(lambda v: dirac.apply_D(Uf, v, kappa), lambda v: dirac.apply_D(Uf, v, kappa, dagger=True),
                           b, tol=cfg["tol"])
    out["full_solve_iterations"] = int(it)
print(json.dumps(out))
"""

_FILTER_STEPS = """
import json, sys, time
sys.path.insert(0, sys.argv[1])
from oracle import filter as ofilter, gauge, lattice
cfg = json.loads(sys.argv[2])
geom = lattice.Geometry(tuple(cfg["dims"]), tuple(cfg["block"]))
U = gauge.generate_links(geom.dims, cfg["eps"], cfg["seed"])
prm = ofilter.FilterParams(kappa=cfg["kappa"], beta0=cfg["beta"], n_iter=1, n_or=0, n_block=cfg["n_block"],
                           n_global=cfg["n_global"], tol=cfg["tol"])
acc, t = 0, []
for s in range(cfg["steps"]):
    t0 = time.perf_counter()
    U, rec = ofilter.filter_step(U, geom, prm, cfg["seed"], s)
    t.append(time.perf_counter() - t0)
    acc += int(rec["accept_global"] and rec["accept_block"].any())
print(json.dumps({"s_per_step": sum(t) / len(t), "accepted": acc, "steps": len(t)}))
"""


def _oracle_run(script, cfg, timeout=1200):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", script, ROOT, json.dumps(cfg)], capture_output=True, text=True,
                       env=env, timeout=timeout)
    if r.returncode:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# the oracle is timed on lattices up to this volume; larger workloads scale its
# per-lattice times by volume (the oracle's work per site is fixed)
ORACLE_MAX_SITES = 16 ** 4


def oracle_components(workload, n_sample=2, with_iterations=True, sweep=True):
    """Measured oracle (numpy FP64, one thread) times of the pieces of one
    filter step: the domain sweep (and the swept field for what follows),
    one whole-lattice CGNR iteration, one interpolation step's per-lattice
    estimator work, and one block solve (mean over a sample of blocks);
    with_iterations also measures the oracle's CGNR iteration count of one
    whole-lattice solve on an 8^4 lattice (same kappa, field recipe and
    tolerance).  Lattices above 16^4 sites are timed on a 16^4 lattice with
    the same blocks and the per-lattice times scaled by the volume ratio."""
    wl = WORKLOADS[workload]
    dims = list(wl["dims"])
    V = int(np.prod(dims))
    scale = 1.0
    if V > ORACLE_MAX_SITES:
        dims = [16, 16, 16, 16]
        scale = V / ORACLE_MAX_SITES
    cfg = {"dims": dims, "block": list(wl["block"]), "kappa": wl["kappa"], "eps": wl["eps"],
           "beta": wl["beta"], "n_or": wl["n_or"], "seed": SEED, "tol": wl["tol"], "n_sample": n_sample,
           "full_dims": [8, 8, 8, 8] if with_iterations else None, "sweep": sweep}
    comp = _oracle_run(_COMPONENTS, cfg)
    for k in ("sweep_s", "cgnr_iteration_s", "level_overhead_s"):
        if k in comp:
            comp[k] *= scale
    comp["timed_on"] = "x".join(str(d) for d in dims) + ("" if scale == 1.0 else f", per-lattice times x{scale:g}")
    return comp


def oracle_step_seconds(workload, comp, full_iters):
    """Oracle time of one filter step from measured component times:
    the sweep; N_block interpolation steps of the block level (per-lattice
    work + every block's solve); with the recursive decomposition n_sub
    steps of stage 2 (per-lattice work, every block solved once in the
    D_ww^-1 / D_bb^-1 batches, one whole-lattice solve of the domains'
    Dirichlet operator); N_global steps of the global level (per-lattice
    work and, without recursion, every block solved once and one
    whole-lattice solve; with it, three whole-lattice solves: the domains'
    D_ww^-1, D_bb^-1 and the full operator).  Every whole-lattice solve is
    counted at full_iters CGNR iterations.  Extrapolated."""
    wl = WORKLOADS[workload]
    nb = int(np.prod([d // b for d, b in zip(wl["dims"], wl["block"])]))
    ov, bs, it = comp["level_overhead_s"], comp["block_solve_s"], full_iters * comp["cgnr_iteration_s"]
    t = comp["sweep_s"] + wl["n_block"] * (ov + nb * bs)
    if wl.get("outer"):
        t += wl["n_sub"] * (ov + nb * bs + it) + wl["n_global"] * (ov + 3 * it)
    else:
        t += wl["n_global"] * (ov + nb * bs + it)
    return t


def oracle_model_check(steps=2):
    """The component model of oracle_step_seconds against complete oracle
    filter steps, both on the 4^4 workload (small enough to run the oracle
    chain): measured seconds per step, the model's seconds from the same
    components (whole-lattice iterations counted on the 4^4 lattice
    itself), and their ratio."""
    wl = WORKLOADS["4^4"]
    base = {"dims": list(wl["dims"]), "block": list(wl["block"]), "kappa": wl["kappa"], "eps": wl["eps"],
            "beta": wl["beta"], "seed": SEED, "tol": wl["tol"]}
    full = _oracle_run(_FILTER_STEPS, dict(base, n_block=wl["n_block"], n_global=wl["n_global"], steps=steps))
    comp = _oracle_run(_COMPONENTS, dict(base, n_or=wl["n_or"], n_sample=4, full_dims=list(wl["dims"]), sweep=True))
    model = oracle_step_seconds("4^4", comp, comp["full_solve_iterations"])
    return {"workload": "4^4", "measured_s_per_step": round(full["s_per_step"], 3),
            "model_s_per_step": round(model, 3), "model_over_measured": round(model / full["s_per_step"], 3),
            "steps": full["steps"]}


def cpu_baseline(workload, recs):
    """The oracle on this host, one thread: its filter-step time from measured
    components (oracle_step_seconds; the whole-lattice solve's iteration
    count measured by the oracle on 8^4), and the accepted updates per step
    of the GPU chain, which the oracle reproduces decision for decision on
    the same random numbers (parity).  Extrapolated, not a run of the full
    oracle chain."""
    comp = oracle_components(workload)
    step_s = oracle_step_seconds(workload, comp, comp["full_solve_iterations"])
    acc_frac = _accepted(recs) / max(len(recs), 1)
    return {"value": acc_frac / step_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle components (timed on {comp['timed_on']}, swept field): sweep {comp['sweep_s']:.2f} s, "
                       f"CGNR iteration {comp['cgnr_iteration_s']:.3f} s, block solve {comp['block_solve_s']:.3f} s "
                       f"(mean of {comp['block_sample']}), per-level overhead {comp['level_overhead_s']:.2f} s; "
                       f"whole-lattice solve {comp['full_solve_iterations']} CGNR iterations (oracle, 8^4); "
                       f"step time from the levels' solve counts = {step_s:.0f} s; accepted updates per step from "
                       f"the GPU chain ({_accepted(recs)}/{len(recs)}, identical decisions by parity); extrapolated"),
            "components": comp, "extrapolated_step_s": step_s, "model_check": _model_check_or_error()}


def _model_check_or_error():
    # a calibration beside the baseline: its failure must not cost the line
    try:
        return oracle_model_check()
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {str(e)[-300:]}"}


def reference_arm(args):
    """The oracle timed as it stands on the host cores (one thread).  At 4^4
    each step is one complete oracle filter step.  At the larger workloads
    each step is a bounded sample: one whole-lattice CGNR iteration and a
    block solve on the workload lattice, re-timed every step; the sweep,
    the per-level overhead and the whole-lattice iteration count (on 8^4)
    are timed once first.  The step time is extrapolated from these
    (oracle_step_seconds); the oracle's accepted updates per step cannot be
    measured in minutes, so the line counts every oracle step as one
    accepted update: its value is an upper bound."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    if args.workload == "4^4":
        cfg = {"dims": list(wl["dims"]), "block": list(wl["block"]), "kappa": wl["kappa"], "eps": wl["eps"],
               "beta": wl["beta"], "seed": SEED, "n_block": wl["n_block"], "n_global": wl["n_global"],
               "tol": wl["tol"], "steps": args.steps}
        r = _oracle_run(_FILTER_STEPS, cfg)
        step_s = r["s_per_step"]
        value = r["accepted"] / r["steps"] / step_s
        sample = f"{r['steps']} complete oracle filter steps at 4^4 (measured, {r['accepted']} accepted)"
    else:
        comp = oracle_components(args.workload)
        times = []
        for i in range(args.steps):
            c = oracle_components(args.workload, n_sample=1, with_iterations=False, sweep=False)
            times.append(oracle_step_seconds(args.workload, dict(comp, cgnr_iteration_s=c["cgnr_iteration_s"],
                                                                   block_solve_s=c["block_solve_s"]),
                                             comp["full_solve_iterations"]))
        step_s = statistics.median(times)
        value = 1.0 / step_s
        sample = (f"per step: one oracle CGNR iteration and one block solve (timed on {comp['timed_on']}, "
                  f"re-timed each step); sweep, per-level overhead and the whole-lattice iteration count "
                  f"({comp['full_solve_iterations']}, oracle CGNR on 8^4) timed once; step time extrapolated from "
                  f"the levels' solve counts; value counts one accepted update per oracle step (an upper bound)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "dims": list(wl["dims"]), "block": list(wl["block"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 arm")
    ap.add_argument("--secondary-steps", type=int, default=10, help="timed steps per arm of the 16^4 section")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 16^4 section")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP64 and mixed arms")
    ap.add_argument("--no-large", action="store_true", help="skip the 32^3x64 D_w and heatbath measurements")
    ap.add_argument("--learned-only", action="store_true", help="the learned level at 16^3x32 with 8^4 domains")
    ap.add_argument("--labels", type=int, default=100_000, help="training labels of --learned-only")
    ap.add_argument("--dw-only", action="store_true", help="stand-alone D_w measurement only")
    ap.add_argument("--hop-variants", action="store_true", help="--dw-only: time every hop variant")
    ap.add_argument("--solve-only", action="store_true", help="single-system solver measurement only")
    ap.add_argument("--batch-only", action="store_true", help="multi-lattice batched block solves (8^4, 12^4, 16^3x32)")
    ap.add_argument("--block-only", action="store_true", help="the 16^4 block level alone (ncu case)")
    ap.add_argument("--step-only", action="store_true", help="filter steps alone (launch-list case)")
    ap.add_argument("--block-n", type=int, default=12, help="interpolation steps of --block-only")
    ap.add_argument("--block-variant", type=int, default=-1, help="force a block-solver variant (--block-only)")
    ap.add_argument("--levels-only", action="store_true",
                    help="parametrised levels and the recursive decomposition on 16^4 (auxiliary line)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    elif args.dw_only:
        dw_only(args)
    elif args.solve_only:
        solve_only(args)
    elif args.batch_only:
        batch_only(args)
    elif args.learned_only:
        learned_only(args)
    elif args.levels_only:
        levels_only(args)
    elif args.block_only:
        block_only(args)
    elif args.step_only:
        step_only(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
