"""Benchmark of the phi-product hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config I] [--variant hcwy] [--precision fp64]

--config 3 selects the batched workload (512 advection-diffusion instances of
uneven size in one persistent launch per step); --config 4 the adjoint workload
(a step is one loss-and-gradient evaluation of 1/2 ||phi_1(hA(theta))v - y_t||^2
on the 256x256 Gray-Scott Jacobian: the forward phi product and lsa_phiv_vjp);
--config 5 the exponential-integrator workload (a step is one EPI4 time step,
Sect. 4, of the Gray-Scott system on the 512x512 grid: one phi-function linear
combination of the augmented operator plus the remainder evaluations), timed
beside the same run with the ioCGS baseline (the paper's runtime ratio).

A step is one phiv call -- the whole hot path (stencil matvecs, grouped
reductions, correction, projection, small exponential, output combination) over
one synthetic input.  Default workload: the Gray-Scott Jacobian on a 512x512
periodic grid (N = 524288), phi_0..phi_2 with m = 64, float64, hybrid
one-reduce Arnoldi with the compact-WY correction.

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica (the path is not sharded: one phi product fits one GPU), the time is
the max over ranks and value = all ranks' phiv calls / that time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Arnoldi steps/s and phiv calls/s at 1e-10 rel err; HBM GB/s fraction; grid syncs/step"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (recipe's unit counts and clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one launch of the dominant kernel from an ncu
# capture of the current kernel, keyed by workload, precision, variant and
# Arnoldi kernel kind (0 one-pass, 4 two-phase grid kernel, 5 flat two-phase
# kernel, 2 streaming);
# a workload without an up-to-date capture reports null.  Gray-Scott 512^2:
# profiles/k_arnoldi_grayscott2d_512_fp64.md (both step forms); the 3D line's
# capture is of the 192^3 case (same tiling), scaled by the unknowns
# ((256/192)^3) (profiles/k_arnoldi_stream_adr3d_192_fp32.md).
PROFILED_TRAFFIC = {("grayscott2d_512", "fp64", "hcwy", 0): 9.118409e9 + 0.744297e9,
                    ("grayscott2d_512", "fp64", "hcwy", 4): 13.717263e9 + 0.777655e9,
                    ("adr3d_256", "fp32", "hcwy", 2): (28.712327e9 + 2.551436e9) * (256 / 192) ** 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--variant", default="hcwy")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle leg (profiling runs)")
    ap.add_argument("--size", type=int, default=0, help="override the grid side (profiling on a smaller case)")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def aggregate_replicas(local_ms, steps, world, device=None):
    """Whole-job throughput of independent replicas: every rank timed `steps`
    phiv calls in `local_ms`; the job's time is the slowest rank's, and the
    value counts all ranks' calls.  Returns (max_ms, calls per second)."""
    t_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([t_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    return t_ms, world * steps / (t_ms / 1e3)


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload(cfg_index, size=0):
    import workloads as W

    cfg = W.config(cfg_index)
    if cfg.get("kind") == "batched":
        return cfg
    if size:
        ctor = {"advdiff2d": W.advdiff2d, "grayscott2d": W.grayscott2d, "adr3d": W.adr3d}[cfg["kind"]]
        cfg = ctor(size, h=cfg["h"], p=cfg["p"], m=cfg["m"], seed=cfg["seed"])
    return cfg


def algorithmic_counts(cfg, precision, m_eff):
    """Algorithmic bytes and FP64 flops of one Arnoldi launch (hybrid form).

    Step j (1-based) reads the j-1 previous columns and w_{j-1}, writes x_j and
    w_j (the stencil is fused, halos excluded): (j+2) N elements; the operator's
    coefficient fields add their own reads.  The final projection reads m
    columns and w_m and writes v_{m+1}: (m+2) N.  Flops: projection 2(j-1) N,
    dots 2(2(j-1)+3) N, stencil ~2*taps N per step; final 2m N."""
    import workloads as W

    N = W.n_dof(cfg)
    bs = 8 if precision == "fp64" else 4
    fb = 8 if precision == "fp64" else 4
    field_elems = {"advdiff2d": 0, "grayscott2d": N, "adr3d": N}[cfg["kind"]]
    taps = {"advdiff2d": 5, "grayscott2d": 7, "adr3d": 8}[cfg["kind"]]
    m = m_eff
    elems = sum(j + 2 for j in range(1, m + 1)) * N + (m + 2) * N
    byts = elems * bs + m * field_elems * fb
    flops = sum(2 * (j - 1) + 2 * (2 * (j - 1) + 3) + 2 * taps for j in range(1, m + 1)) * N
    flops += (2 * m + 2) * N
    return byts, flops


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def run_reference(args, world, rank):
    """The CPU oracle (float64 NumPy) timed on this host on a bounded sample."""
    if rank != 0:
        return
    import numpy as np

    import workloads as W
    from oracle import krylov as OK
    from oracle import operators as OP

    if args.config == 5:
        run_reference_integrator(args, world, integrator_workload(args.size))
        return
    cfg = workload(args.config, args.size)
    if cfg.get("kind") == "batched":
        run_reference_batched(args, world, cfg)
        return
    if args.config == 4:
        run_reference_adjoint(args, world, cfg)
        return
    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    variant = args.variant
    n_warm = min(args.warmup, 1)       # one untimed call at most: the oracle takes seconds per call
    for _ in range(n_warm):
        OK.phiv(lambda x: A @ x, inp["v"], cfg["h"], cfg["p"], cfg["m"], variant)
    t_steps = []
    t0 = time.perf_counter()
    n = 0
    while n < max(1, args.steps):
        ts = time.perf_counter()
        OK.phiv(lambda x: A @ x, inp["v"], cfg["h"], cfg["p"], cfg["m"], variant)
        t_steps.append(time.perf_counter() - ts)
        n += 1
        if time.perf_counter() - t0 > 9 * args.cpu_budget:   # keep the run within minutes
            break
    tot = sum(t_steps)
    value = n / tot
    cores = os.cpu_count()
    sample = f"{n} full phiv call(s) of {cfg['name']} (m={cfg['m']}, p={cfg['p']}, {variant})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "phiv/s",
            "n_gpus": world, "steps": n, "warmup": n_warm, "ms_per_step": 1e3 * tot / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg["name"], "N": W.n_dof(cfg), "m": cfg["m"],
                                             "p": cfg["p"], "h": cfg["h"], "variant": variant,
                                             "precision": "fp64",
                                             "parallelism": "host cores (oracle)"},
            "cpu_baseline": {"value": value, "unit": "phiv/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "phiv/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_adjoint(args, world, cfg):
    """The oracle's gradient evaluation (float64 NumPy/SciPy) on this host."""
    import workloads as W
    from oracle import adjoint as OAD

    inp = W.adjoint_inputs(cfg)
    A, dA = OAD.grayscott_parts(cfg, inp)
    t0 = time.perf_counter()
    n = 0
    while n < max(1, args.steps):
        OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], cfg["h"], cfg["m"], args.variant)
        n += 1
        if time.perf_counter() - t0 > 3 * args.cpu_budget:   # keep the run within minutes
            break
    el = time.perf_counter() - t0
    value = n / el
    sample = f"{n} full gradient evaluation(s) of {cfg['name']} (m={cfg['m']}, {args.variant})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "grad/s",
            "n_gpus": world, "steps": n, "warmup": 0, "ms_per_step": 1e3 * el / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg["name"], "m": cfg["m"], "h": cfg["h"],
                                             "variant": args.variant, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "grad/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "grad/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_batch_sample(bcfg, variant, budget, max_calls=None):
    """Time the oracle over the batch's instances in order until ~budget
    seconds have passed (bounded sample).  Returns (calls, seconds, outputs)."""
    import workloads as W
    from oracle import krylov as OK
    from oracle import operators as OP

    t0 = time.perf_counter()
    n = 0
    outs = []
    for c in bcfg["instances"]:
        inp = W.make_inputs(c)
        A = OP.from_workload(c, inp)
        ts = time.perf_counter()
        y, _ = OK.phiv(lambda x: A @ x, inp["v"], bcfg["h"], bcfg["p"], c["m"], variant)
        outs.append(y)
        n += 1
        if time.perf_counter() - t0 > budget or (max_calls and n >= max_calls):
            break
    return n, time.perf_counter() - t0, outs


def run_reference_batched(args, world, bcfg):
    n, el, _ = oracle_batch_sample(bcfg, args.variant, 9 * args.cpu_budget,
                                   max_calls=max(1, args.steps) * 8)
    value = n / el
    sample = (f"the first {n} of {len(bcfg['instances'])} instances of {bcfg['name']} "
              f"({args.variant}, float64 NumPy/SciPy)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "phiv/s",
            "n_gpus": world, "steps": n, "warmup": 0, "ms_per_step": 1e3 * el / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": bcfg["name"], "p": bcfg["p"],
                                             "variant": args.variant, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "phiv/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "phiv/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batched(args, world, rank, local, bcfg):
    """The batched workload: all instances in one persistent launch (tuned
    tiling, CUDA-graph replay) per step, beside a loop of single lsa_phiv
    calls over the same instances."""
    import numpy as np
    import torch

    import paper_2410_14917_gb300 as lsa
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    insts = bcfg["instances"]
    h, p = bcfg["h"], bcfg["p"]
    ops = [lsa.Operator.from_workload(c, {}) for c in insts]
    ms = [c["m"] for c in insts]
    vs = W.batched_inputs(bcfg)
    v_host = torch.from_numpy(np.concatenate(vs)).pin_memory()
    v = v_host.to(dev)
    b = lsa.Batch(ops, ms, h, p, variant=args.variant, precision=args.precision)
    y = torch.empty(b.y_elems, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    default_tiling = b.tiling
    t_tune = time.perf_counter()
    gs, nl, ms_tune = b.tune(v, y, reps=2)
    t_tune = time.perf_counter() - t_tune
    b.run(v, y, graph=True)
    torch.cuda.synchronize()
    st, fin, stats = b.stats()
    if st < 0 or fin != b.count:
        raise RuntimeError(f"batched run failed: status {st}, {fin}/{b.count} finished")
    m_eff = [s["m_eff"] for s in stats]
    for _ in range(args.warmup):
        b.run(v, y, graph=True)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        b.run(v, y, graph=True)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    st, fin, _ = b.stats()
    if st < 0 or fin != b.count:
        raise RuntimeError(f"batched run failed: status {st}")
    tot_ms, steps_per_s = aggregate_replicas(sum(step_ms), args.steps, world, dev)
    value = steps_per_s * b.count

    # a loop of single lsa_phiv calls over the same instances (one workspace)
    big = max(range(len(ops)), key=lambda i: lsa.workspace_bytes(ops[i], ms[i], p, args.precision))
    work = lsa.Workspace.for_call(ops[big], ms[big], p, args.precision)
    parts = b.split(y)
    ysingle = [torch.empty_like(t) for t in parts]
    vparts = [v[b.voff[i]:b.voff[i] + ops[i].N] for i in range(b.count)]

    def loop():
        for i in range(b.count):
            lsa.phiv(ops[i], vparts[i], h, p, ms[i], variant=args.variant, precision=args.precision,
                     y=ysingle[i], work=work, stats=False)
    loop()
    torch.cuda.synchronize()
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    lsteps = 2
    l0.record(stream)
    for _ in range(lsteps):
        loop()
    l1.record(stream)
    torch.cuda.synchronize()
    loop_ms = l0.elapsed_time(l1) / lsteps
    loop_diff = max(float((ysingle[i] - parts[i]).abs().max() / parts[i].abs().max().clamp_min(1e-300))
                    for i in range(b.count))

    # end to end with host buffers
    y_host = torch.empty(b.y_elems, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    vd = torch.empty_like(v)
    b.run(vd, y, graph=True)           # capture once for the (vd, y) pair
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        vd.copy_(v_host, non_blocking=True)
        b.run(vd, y, graph=True)
        y_host.copy_(y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = e2e_steps * b.count / (e0.elapsed_time(e1) / 1e3) * world

    byts = flops = 0
    for c, me in zip(insts, m_eff):
        bb, ff = algorithmic_counts(c, args.precision, me)
        byts += bb
        flops += ff
    ms_step = tot_ms / args.steps
    hbm_peak, peak_kind = load_peaks()
    gbs = byts / (ms_step / 1e3) / 1e9
    if args.precision == "fp64":
        achieved = flops / (ms_step / 1e3) / 1e12
        pk64, pk64_src = fp64_peak(lsa)
        roof = {"bound": "alu", "achieved": achieved, "peak": pk64, "unit": "TFLOP/s",
                "frac": achieved / pk64, "traffic": None,
                "kernel": "k_batched (persistent batched phi products; step time incl. its init kernel)",
                "peak_source": pk64_src,
                "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak, "algorithmic_bytes": byts,
                "algorithmic_flops": flops}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "traffic": None,
                "kernel": "k_batched (persistent batched phi products; step time incl. its init kernel)",
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes": byts,
                "algorithmic_flops": flops}
    line = {"metric": METRIC, "value": value, "unit": "phiv/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32-basis/f64", "data": "synthetic",
            "config": {"workload": bcfg["name"], "instances": b.count, "p": p, "h": h,
                       "variant": args.variant, "precision": args.precision,
                       "N_total": int(b.v_elems), "ctas": b.ctas,
                       "tiling": {"group_size": gs, "nlarge": nl, "tuned_ms": ms_tune,
                                  "tune_s": t_tune, "default": list(default_tiling),
                                  "step_form": "two-phase" if b.step_form else "one-pass"},
                       "graph": True,
                       "l2": "flushed between timed steps (256 MiB write)" if flush is not None
                       else "not flushed",
                       "parallelism": f"replicas x{world}"},
            "arnoldi_steps_per_s": steps_per_s * sum(m_eff),
            "loop_of_single_calls": {"ms_per_batch": loop_ms, "phiv_per_s": b.count / (loop_ms / 1e3),
                                     "speedup_of_batched": loop_ms / ms_step,
                                     "max_rel_diff_vs_batched": loop_diff,
                                     "launches_per_batch": 4 * b.count},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "phiv/s", "h2d_bytes_per_step": int(b.v_elems) * 8,
                    "d2h_bytes_per_step": int(b.y_elems) * 8},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu:
        n, el, outs = oracle_batch_sample(bcfg, "mgs", args.cpu_budget)
        line["cpu_baseline"] = {"value": n / el, "unit": "phiv/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"the first {n} of {b.count} instances ({'mgs'}, float64 NumPy/SciPy)"}
        errs = []
        for i in range(n):
            yi = parts[i].cpu().numpy()
            errs.append(max(float(np.linalg.norm(yi[k] - outs[i][k]) / np.linalg.norm(outs[i][k]))
                            for k in range(p + 1)))
        line["rel_err_vs_oracle"] = max(errs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def adjoint_flops(cfg, m):
    """FP64 flops of one gradient evaluation: the forward phi product and the
    product on A^T (N unknowns each) and three on the Frechet block operator
    (2N unknowns each; its stencil is counted like the Gray-Scott one; the F
    derivative is a closed form)."""
    _, f = algorithmic_counts(cfg, "fp64", m)
    return 2 * f + 3 * 2 * f


def bench_adjoint(args, world, rank, local, cfg):
    import numpy as np
    import torch

    import paper_2410_14917_gb300 as lsa
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    inp = W.adjoint_inputs(cfg)
    N = W.n_dof(cfg)
    m, h = cfg["m"], cfg["h"]
    d = {k: torch.from_numpy(v).to(dev) for k, v in inp.items()}
    op = lsa.Operator.from_workload(cfg, d)
    v, yt = d["v"], d["y_target"]
    y = torch.empty((3, N), dtype=torch.float64, device=dev)
    r = torch.empty(N, dtype=torch.float64, device=dev)
    work = lsa.Workspace.for_call(op, m, 2, "fp64")
    vwork = lsa.Workspace(lsa.vjp_workspace_bytes(op, m), device=dev)
    stream = torch.cuda.current_stream()
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def grad_eval(vv, tgt, stats=False):
        # forward with p = 2 (phi_2 feeds the closed-form F derivative), residual, gradient
        lsa.phiv(op, vv, h, 2, m, variant=args.variant, y=y, work=work, stats=False)
        lsa.axpby(1.0, y[1], -1.0, tgt, out=r)
        return lsa.phiv_vjp(op, vv, h, m, r, y, variant=args.variant, work=vwork, stats=stats)

    gv, gs, st = grad_eval(v, yt, stats=True)
    for _ in range(args.warmup):
        grad_eval(v, yt)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    fwd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        gv, gs, _ = grad_eval(v, yt)
        ev[i][1].record(stream)
    # the plain float64 forward phi product alone, for comparison
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        fwd[i][0].record(stream)
        lsa.phiv(op, v, h, 1, m, variant=args.variant, y=y[:2], work=work, stats=False)
        fwd[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    fwd_ms = statistics.mean(a.elapsed_time(b) for a, b in fwd)
    tot_ms, value = aggregate_replicas(sum(step_ms), args.steps, world, dev)

    # end to end with host buffers: v and y_t in, dL/dv and the five scalar gradients out
    v_host = torch.from_numpy(inp["v"]).pin_memory()
    t_host = torch.from_numpy(inp["y_target"]).pin_memory()
    gv_host = torch.empty(N, dtype=torch.float64).pin_memory()
    gs_host = torch.empty(5, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        vv = v_host.to(dev, non_blocking=True)
        tt = t_host.to(dev, non_blocking=True)
        g1, g2, _ = grad_eval(vv, tt)
        gv_host.copy_(g1, non_blocking=True)
        gs_host.copy_(g2, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = e2e_steps / (e0.elapsed_time(e1) / 1e3) * world

    ms_step = tot_ms / args.steps
    flops = adjoint_flops(cfg, m)
    achieved = flops / (ms_step / 1e3) / 1e12
    pk64, pk64_src = fp64_peak(lsa)
    roof = {"bound": "alu", "achieved": achieved, "peak": pk64, "unit": "TFLOP/s",
            "frac": achieved / pk64, "traffic": None,
            "kernel": "whole gradient evaluation (five k_arnoldi launches with their small kernels)",
            "peak_source": pk64_src,
            "algorithmic_flops": flops}
    line = {"metric": METRIC, "value": value, "unit": "grad/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "N": N, "m": m, "h": h, "variant": args.variant,
                       "precision": "fp64", "theta": ["Du", "Dv", "F", "k"],
                       "l2": "flushed between timed steps (256 MiB write)" if flush is not None
                       else "not flushed", "parallelism": f"replicas x{world}"},
            "phiv_per_grad": 5,
            "vs_plain_fp64_forward": {"forward_ms": fwd_ms, "gradient_ms": ms_step,
                                      "ratio": ms_step / fwd_ms},
            "grid_syncs": st["grid_syncs"],
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "grad/s", "h2d_bytes_per_step": 2 * N * 8,
                    "d2h_bytes_per_step": (N + 5) * 8},
            "gpu_launches": (5 * 4 + 10 + 1) * args.steps,
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import adjoint as OAD

        A, dA = OAD.grayscott_parts(cfg, inp)
        t0 = time.perf_counter()
        ref = OAD.grads_krylov(A, dA, inp["v"], inp["y_target"], h, m)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / el, "unit": "grad/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"one full gradient evaluation of {cfg['name']} (mgs, float64 NumPy/SciPy)"}
        g_s = gs.cpu().numpy()
        errs = [float(np.max(np.abs(gv.cpu().numpy() - ref["dv"])) / np.max(np.abs(ref["dv"]))),
                abs(g_s[0] - ref["dh"]) / abs(ref["dh"])]
        errs += [abs(g_s[1 + k] - ref["dtheta"][k]) / abs(ref["dtheta"][k]) for k in range(4)]
        line["rel_err_vs_oracle"] = max(errs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def integrator_workload(size=0):
    import workloads as W

    cfg = W.grayscott2d(size or 512, h=1.0, m=64, p=3)
    cfg.update(name=f"grayscott2d_{cfg['nx']}_epi4", method="epi4", nsub=1)
    return cfg


def bench_integrator(args, world, rank, local, cfg):
    import numpy as np
    import torch

    import paper_2410_14917_gb300 as lsa
    import workloads as W
    from paper_2410_14917_gb300.integrators import GrayScottIntegrator

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    inp = W.make_inputs(cfg)
    N = W.n_dof(cfg)
    u0 = torch.from_numpy(np.concatenate([inp["u0"], inp["v0"]])).to(dev)
    h, m, method = cfg["h"], cfg["m"], cfg["method"]
    stream = torch.cuda.current_stream()
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def make(variant):
        it = GrayScottIntegrator(cfg["nx"], cfg["ny"], cfg["dx"], cfg["diff"], cfg["diff2"], cfg["F"],
                                 cfg["k"], u0, m=m, nsub=cfg["nsub"], variant=variant)
        it.run(method, h, 2)                   # the SRERK3 start: EPI4 needs u_{n-1}, u_{n-2}
        s0 = it.stats["grid_syncs"]
        it.run(method, h, 1)                   # one EPI4 step with statistics
        it.syncs_per_step = it.stats["grid_syncs"] - s0
        it.collect_stats = False
        for _ in range(args.warmup):
            it.run(method, h, 1)
        return it

    def timed(it, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        l0 = it.stats["launches"]
        for i in range(steps):
            if flush is not None:
                flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            it.run(method, h, 1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], it.stats["launches"] - l0

    it = make(args.variant)
    syncs_step = it.syncs_per_step
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    step_ms, launches = timed(it, args.steps)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    tot_ms, value = aggregate_replicas(sum(step_ms), args.steps, world, dev)
    ms_step = tot_ms / args.steps

    # the paper's metric: the integrator with this variant over the same run with ioCGS
    io = make("iocgs")
    io_syncs = io.syncs_per_step
    io_ms = statistics.mean(timed(io, args.steps)[0])

    # end to end: the state from pinned host memory, one step, the state back
    s_host = u0.cpu().pin_memory()
    s_back = torch.empty(N, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        it.u.copy_(s_host, non_blocking=True)
        it.run(method, h, 1)
        s_back.copy_(it.u, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = e2e_steps / (e0.elapsed_time(e1) / 1e3) * world

    byts, flops = algorithmic_counts(cfg, "fp64", m)
    achieved = flops / (ms_step / 1e3) / 1e12
    pk64, pk64_src = fp64_peak(lsa)
    roof = {"bound": "alu", "achieved": achieved, "peak": pk64, "unit": "TFLOP/s",
            "frac": achieved / pk64, "traffic": None,
            "kernel": "whole EPI4 step (augmented-operator k_arnoldi with its small kernels)",
            "peak_source": pk64_src,
            "algorithmic_flops": flops}
    line = {"metric": METRIC, "value": value, "unit": "integrator steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "N": N, "method": method, "h": h, "m": m,
                       "nsub": cfg["nsub"], "variant": args.variant, "precision": "fp64",
                       "l2": "flushed between timed steps (256 MiB write)" if flush is not None
                       else "not flushed", "parallelism": f"replicas x{world}"},
            "lincomb_per_step": 1,
            "grid_syncs_per_step": syncs_step,
            "vs_iocgs": {"ms_iocgs": io_ms, "ms_variant": ms_step, "ratio": ms_step / io_ms,
                         "grid_syncs_iocgs": io_syncs,
                         "note": "integrator runtime with this variant / with ioCGS (Sect. 4's ratio)"},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "integrator steps/s", "h2d_bytes_per_step": N * 8,
                    "d2h_bytes_per_step": N * 8},
            "gpu_launches": launches,
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu:
        el, sample = oracle_integrator_sample(cfg, args.variant)
        line["cpu_baseline"] = {"value": 1.0 / el, "unit": "integrator steps/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def oracle_integrator_sample(cfg, variant):
    """One EPI4 step of the oracle (float64 NumPy/SciPy, Krylov combinations
    with the same m) from the workload's state, the history given."""
    import numpy as np

    import workloads as W
    from oracle import integrators as OI

    inp = W.make_inputs(cfg)
    u0 = np.concatenate([inp["u0"], inp["v0"]])
    F, Jf = OI.grayscott_problem(cfg)
    lc = OI.krylov_lincomb(cfg["m"], cfg["nsub"], variant)
    t0 = time.perf_counter()
    OI.epi_step(4, F, Jf, [u0, u0, u0], cfg["h"], lc)
    el = time.perf_counter() - t0
    return el, f"one EPI4 step of {cfg['name']} (history given, {variant} Krylov, float64 NumPy/SciPy)"


def run_reference_integrator(args, world, cfg):
    t_all = []
    t0 = time.perf_counter()
    while len(t_all) < max(1, args.steps):
        el, sample = oracle_integrator_sample(cfg, args.variant)
        t_all.append(el)
        if time.perf_counter() - t0 > 3 * args.cpu_budget:
            break
    n, el = len(t_all), sum(t_all)
    value = n / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "integrator steps/s",
            "n_gpus": world, "steps": n, "warmup": 0, "ms_per_step": 1e3 * el / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg["name"], "method": cfg["method"], "h": cfg["h"],
                                             "m": cfg["m"], "variant": args.variant, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "integrator steps/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": f"{n} x " + sample},
            "e2e": {"value": value, "unit": "integrator steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(cfg, variant, budget):
    """Time the oracle (as it stands) on a bounded sample: whole phiv calls on
    the full workload until ~budget seconds have passed.  Also returns the last
    oracle result for the accuracy check of the GPU result."""
    import workloads as W
    from oracle import krylov as OK
    from oracle import operators as OP

    inp = W.make_inputs(cfg)
    A = OP.from_workload(cfg, inp)
    t0 = time.perf_counter()
    n = 0
    y = None
    while True:
        y, _ = OK.phiv(lambda x: A @ x, inp["v"], cfg["h"], cfg["p"], cfg["m"], variant)
        n += 1
        if time.perf_counter() - t0 > budget or n >= 5:
            break
    el = time.perf_counter() - t0
    return {"value": n / el, "unit": "phiv/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} full phiv call(s) of {cfg['name']} ({variant}, float64 NumPy/SciPy)"}, y


def fp64_peak(lsa):
    """(TFLOP/s, source) of the float64 roofline: the FMA throughput measured
    on this GPU by lsa_probe_fp64_fma, else the nominal unit counts."""
    meas = lsa.probe_fp64_fma_tflops()
    if meas > 0:
        return meas, ("measured float64 FMA throughput (lsa_probe_fp64_fma, CUDA events, best of 10 after a warm-up; "
                      "nominal 152 SMs x 2 FMA/clk x 2.07 GHz = %.3f TFLOP/s)" % FP64_PEAK_TFLOPS)
    return FP64_PEAK_TFLOPS, "nominal unit counts (152 SMs x 2 FMA/clk x 2.07 GHz)"


def phiv_roofline(cfg, precision, variant, ms_a, m_eff, kernel_kind, fp64_peak, fp64_peak_src):
    """Roofline object of the persistent Arnoldi kernel of one phiv call."""
    byts, flops = algorithmic_counts(cfg, precision, m_eff)
    hbm_peak, peak_kind = load_peaks()
    if precision == "fp64":
        achieved = flops / (ms_a / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                "traffic": PROFILED_TRAFFIC.get((cfg["name"], precision, variant, kernel_kind)),
                "kernel": ("k_arnoldi_cluster (single thread-block cluster; the time also covers the small "
                           "exponential and the output combination fused into the launch)"
                           if kernel_kind == 3 else
                           "k_arnoldi (persistent hybrid Arnoldi, two-phase step)" if kernel_kind == 4 else
                           "k_arnoldi_flat (persistent hybrid Arnoldi, flat two-phase step)" if kernel_kind == 5 else
                           "k_arnoldi (persistent hybrid Arnoldi, one-pass step)"),
                "peak_source": fp64_peak_src,
                "hbm_gbs": byts / (ms_a / 1e3) / 1e9, "hbm_frac": byts / (ms_a / 1e3) / 1e9 / hbm_peak,
                "algorithmic_bytes": byts, "algorithmic_flops": flops}
    achieved = byts / (ms_a / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak,
            "traffic": PROFILED_TRAFFIC.get((cfg["name"], precision, variant, kernel_kind)),
            "kernel": {0: "k_arnoldi", 1: "k_arnoldi_tma", 2: "k_arnoldi_stream", 4: "k_arnoldi",
                       5: "k_arnoldi_flat"}[kernel_kind]
                      + " (persistent Arnoldi, float32 basis)",
            "peak_source": f"{peak_kind} hbm_gbs",
            "algorithmic_bytes": byts, "algorithmic_flops": flops}


def time_phiv(lsa, torch, cfg, precision, variant, steps, warmup, dev, flush, stream):
    """Inputs resident on the device, `warmup` untimed calls, then `steps`
    calls each bracketed by CUDA events on the launching stream (L2 flushed
    before each).  Returns a dict with the per-call times, the library's own
    per-kernel times, the first call's statistics and the device buffers."""
    import workloads as W

    inp = W.make_inputs(cfg)
    N = W.n_dof(cfg)
    p, m, h = cfg["p"], cfg["m"], cfg["h"]
    fields = {k: torch.from_numpy(v).to(dev) for k, v in inp.items() if k != "v"}
    v_host = torch.from_numpy(inp["v"]).pin_memory()
    v = v_host.to(dev)
    op = lsa.Operator.from_workload(cfg, fields)
    work = lsa.Workspace.for_call(op, m, p, precision)
    y = torch.empty((p + 1, N), dtype=torch.float64, device=dev)
    # the library's step-form tuner (one-pass vs two-phase hybrid step of the
    # grid kernel; a no-op for the other kernels), before anything is timed
    two, ms_one, ms_two = lsa.tune_step(op, v, m, variant=variant, precision=precision, reps=3, work=work)
    _, st0 = lsa.phiv(op, v, h, p, m, variant=variant, precision=precision, y=y, work=work)
    for _ in range(warmup):
        lsa.phiv(op, v, h, p, m, variant=variant, precision=precision, y=y, work=work, stats=False)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    k_arn, k_exp, k_cmb = [], [], []
    launches = 0
    for i in range(steps):
        if flush is not None:
            flush.fill_(i & 0xFF)           # evict L2 between timed steps
        ev[i][0].record(stream)
        _, st = lsa.phiv(op, v, h, p, m, variant=variant, precision=precision, y=y, work=work, stats=True)
        ev[i][1].record(stream)
        if st["status"] < 0:
            raise RuntimeError(f"phiv failed: {st}")
        k_arn.append(st["ms_arnoldi"])
        k_exp.append(st["ms_expm"])
        k_cmb.append(st["ms_combine"])
        launches += st["launches"]
    torch.cuda.synchronize()
    step_form = None
    if ms_one > 0:
        step_form = {"chosen": ["one-pass", "two-phase", "flat two-phase"][two], "tuner_ms_one_pass": ms_one,
                     "tuner_ms_two_phase": ms_two}
    return dict(step_ms=[a.elapsed_time(b) for a, b in ev], k_arn=k_arn, k_exp=k_exp, k_cmb=k_cmb, st0=st0,
                op=op, v=v, v_host=v_host, y=y, work=work, inp=inp, N=N, launches=launches,
                step_form=step_form)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch

    import paper_2410_14917_gb300 as lsa
    import workloads as W

    if args.config == 5:
        bench_integrator(args, world, rank, local, integrator_workload(args.size))
        return
    cfg = workload(args.config, args.size)
    if cfg.get("kind") == "batched":
        bench_batched(args, world, rank, local, cfg)
        return
    if args.config == 4:
        bench_adjoint(args, world, rank, local, cfg)
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p, m, h = cfg["p"], cfg["m"], cfg["h"]
    stream = torch.cuda.current_stream()
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    R = time_phiv(lsa, torch, cfg, args.precision, args.variant, args.steps, args.warmup, dev, flush, stream)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    # the float64 roofline's denominator: FMA throughput measured on this GPU
    # (after the timed region, on a warm GPU)
    fp64_pk, fp64_src = fp64_peak(lsa)
    op, v, v_host, y, work, N, st0 = R["op"], R["v"], R["v_host"], R["y"], R["work"], R["N"], R["st0"]

    m_eff = st0["m_eff"]
    tot_ms = sum(R["step_ms"])
    tot_ms, value = aggregate_replicas(tot_ms, args.steps, world, dev)

    # the paper's metric: runtime of the one-reduce method over the incomplete-
    # orthogonalisation baseline ioCGS (same workload, precision and GPU)
    io_ms = None
    if args.variant != "iocgs":
        _, st_io = lsa.phiv(op, v, h, p, m, variant="iocgs", precision=args.precision, y=y, work=work)
        io_t = []
        for i in range(max(3, min(args.steps, 10))):
            if flush is not None:
                flush.fill_(i & 0xFF)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            lsa.phiv(op, v, h, p, m, variant="iocgs", precision=args.precision, y=y, work=work,
                     stats=False)
            a1.record(stream)
            io_t.append((a0, a1))
        torch.cuda.synchronize()
        io_ms = statistics.mean(a.elapsed_time(b) for a, b in io_t)
        lsa.phiv(op, v, h, p, m, variant=args.variant, precision=args.precision, y=y, work=work,
                 stats=False)      # y back to the measured variant's result

    # end to end through one C-ABI call with host buffers (lsa_phiv_host): the
    # H2D copy of v, the phi product and the D2H copy of y, every step
    y_host = torch.empty((p + 1, N), dtype=torch.float64).pin_memory()
    v_dev = torch.empty(N, dtype=torch.float64, device=dev)
    y_dev = torch.empty((p + 1, N), dtype=torch.float64, device=dev)
    e2e_steps = max(3, min(args.steps, 10))
    lsa.phiv_host(op, v_host, h, p, m, y_host, v_dev, y_dev, variant=args.variant, precision=args.precision,
                  work=work)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(e2e_steps):
        lsa.phiv_host(op, v_host, h, p, m, y_host, v_dev, y_dev, variant=args.variant,
                      precision=args.precision, work=work)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = e2e_steps / (e0.elapsed_time(e1) / 1e3) * world
    e2e_match = bool(torch.equal(y_host, y.cpu()))

    ms_a = statistics.mean(R["k_arn"])
    roof = phiv_roofline(cfg, args.precision, args.variant, ms_a, m_eff, st0["arnoldi_kernel"], fp64_pk, fp64_src)
    line = {"metric": METRIC, "value": value, "unit": "phiv/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32-basis/f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "N": N, "m": m, "p": p, "h": h,
                       "variant": args.variant, "precision": args.precision,
                       "step_form": R["step_form"],
                       "l2": "flushed between timed steps (256 MiB write)" if flush is not None
                       else "not flushed; basis working set > L2",
                       "parallelism": f"replicas x{world}"},
            "arnoldi_steps_per_s": value * m_eff,
            "grid_syncs_per_step": st0["grid_syncs"] / max(m_eff, 1),
            "kernel_ms": {"arnoldi": ms_a, "expm": statistics.mean(R["k_exp"]),
                          "combine": statistics.mean(R["k_cmb"])},
            "roofline": roof,
            "vs_iocgs": None if io_ms is None else
            {"ms_iocgs": io_ms, "ms_variant": tot_ms / args.steps, "ratio": (tot_ms / args.steps) / io_ms,
             "grid_syncs_iocgs": st_io["grid_syncs"],
             "note": "runtime of this variant / incomplete-orthogonalisation ioCGS, the paper's metric; "
                     "the paper's ratios (0.55-1.28) are whole integrator runs on CPU clusters"},
            "e2e": {"value": e2e_value, "unit": "phiv/s", "h2d_bytes_per_step": N * 8,
                    "d2h_bytes_per_step": (p + 1) * N * 8,
                    "call": "lsa_phiv_host (C ABI, host buffers; copies and phi product on one stream)",
                    "y_equals_device_result": e2e_match},
            "gpu_launches": R["launches"],
            "clocks": clocks}

    # the 3D float32-basis workload, timed in the default run as a nested block
    d3 = None
    if args.config == 1 and not args.size and world == 1 and args.precision == "fp64":
        cfg3 = workload(2)
        del R
        sampler3 = ClockSampler(local)
        sampler3.start()
        time.sleep(0.3)
        steps3 = max(3, min(args.steps, 5))
        R3 = time_phiv(lsa, torch, cfg3, "fp32", "hcwy", steps3, max(3, min(args.warmup, 3)), dev, flush, stream)
        clocks3 = sampler3.stop()
        st3 = R3["st0"]
        ms3 = statistics.mean(R3["k_arn"])
        d3 = {"workload": cfg3["name"], "N": R3["N"], "m": cfg3["m"], "p": cfg3["p"], "h": cfg3["h"],
              "variant": "hcwy", "precision": "fp32 basis, float64 Hessenberg and small exponential",
              "steps": steps3, "phiv_per_s": steps3 / (sum(R3["step_ms"]) / 1e3),
              "ms_per_step": sum(R3["step_ms"]) / steps3,
              "arnoldi_steps_per_s": st3["m_eff"] / (ms3 / 1e3),
              "grid_syncs_per_step": st3["grid_syncs"] / max(st3["m_eff"], 1),
              "kernel_ms": {"arnoldi": ms3, "expm": statistics.mean(R3["k_exp"]),
                            "combine": statistics.mean(R3["k_cmb"])},
              "roofline": phiv_roofline(cfg3, "fp32", "hcwy", ms3, st3["m_eff"], st3["arnoldi_kernel"],
                                        fp64_pk, fp64_src),
              "clocks": clocks3}
        y3 = R3["y"].cpu().numpy()
        del R3
        line["adr3d_256_fp32"] = d3
    if rank == 0 and world == 1 and not args.no_cpu:
        cb, y_ref = cpu_baseline(cfg, "mgs", args.cpu_budget)
        line["cpu_baseline"] = cb
        yc = y.cpu().numpy()
        line["rel_err_vs_oracle"] = max(float(np.linalg.norm(yc[k] - y_ref[k]) / np.linalg.norm(y_ref[k]))
                                        for k in range(p + 1))
        line["max_abs_err_vs_oracle"] = max(float(np.max(np.abs(yc[k] - y_ref[k])) / np.max(np.abs(y_ref[k])))
                                            for k in range(p + 1))
        if d3 is not None:
            # the oracle's H-CWY form (pinned equal to its MGS) on the full 256^3 grid
            from oracle import krylov as OK
            from oracle import operators as OP

            inp3 = W.make_inputs(cfg3)
            A3 = OP.from_workload(cfg3, inp3)
            t0 = time.perf_counter()
            r3, _ = OK.phiv(lambda x: A3 @ x, inp3["v"], cfg3["h"], cfg3["p"], cfg3["m"], "hcwy")
            d3["rel_err_vs_oracle"] = max(float(np.linalg.norm(y3[k] - r3[k]) / np.linalg.norm(r3[k]))
                                          for k in range(cfg3["p"] + 1))
            d3["max_abs_err_vs_oracle"] = max(float(np.max(np.abs(y3[k] - r3[k])) / np.max(np.abs(r3[k])))
                                              for k in range(cfg3["p"] + 1))
            d3["oracle_s"] = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
