#!/usr/bin/env python3
"""Benchmark of the GB300 ECMG_jcg solve: -Laplace u = f on the unit cube, u = cos(pi x)
cos(pi y) cos(pi z), all-Dirichlet, Q1 elements, coarsest 8^3, 7 levels up to 512^3,
relative residual tolerance 1e-10, exact load functional; synthetic data.

One step = one complete ecmg_solve (level set-up, DSOLVE, EXP_finite / JCG / EXP_true on every
level) in MIXED precision from inputs resident in HBM. value = finest free dofs / step time
(Gdof/s). The same problem is also solved in plain FP64 (reported beside it, with both
max-norm errors against the exact solution), end to end through the C ABI from pinned host
buffers (e2e: compact separable inputs assembled on the device; e2e_dense_inputs: the dense
arrays), and by the CPU oracle on a bounded sample (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): independent replicas, one per rank, max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ECMG solve time & Gdof/s at 512^3 (mixed vs FP64, same error); stencil HBM GB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n0", type=int, default=8)
    ap.add_argument("--levels", type=int, default=7)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-levels", type=int, default=5, help="oracle sample, one thread: 8^3 -> 8*2^(L-1)")
    ap.add_argument("--cpu-levels-omp", type=int, default=6,
                    help="oracle sample, OpenMP build on every host core: 8^3 -> 8*2^(L-1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--max-iters", type=int, default=20000)
    ap.add_argument("--inner-rtol", type=float, default=1e-3,
                    help="MIXED: FP32 inner reduction between FP64 residual replacements")
    ap.add_argument("--kernels", default="0,1,2,5,6,7,11", help="kernels timed alone for the report")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 64-problem measurement")
    ap.add_argument("--batched-steps", type=int, default=3)
    ap.add_argument("--batched-form", default="two", choices=["two", "single"],
                    help="MIXED step of the batched workload: two-pass (K1 + K2, the batched default) or the "
                         "single-pass step on every level")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched 64-problem workload (one solve per step; --eager for host loop control)")
    ap.add_argument("--profile-kernel", default=None,
                    help="profiling run: one MIXED solve, then kernel W (or a comma list) of ecmg_time_kernel on "
                         "the finest level, 3 launches each inside the NVTX range kernel_profile (for ncu -k / "
                         "--nvtx-include); prints one JSON line per kernel and exits")
    ap.add_argument("--profile-batched", action="store_true",
                    help="profiling run: one batched solve of the 64-problem workload, then its last stage's K1, "
                         "K2 and FP64 residual alone (ecmg_time_kernel 0, 1, 2), 2 launches each inside the NVTX "
                         "range kernel_profile; prints one JSON line per kernel and exits")
    ap.add_argument("--profile-workload", default="cos_cube", choices=["cos_cube", "jump"],
                    help="with --profile-kernel: cos_cube (one beta, all Dirichlet: the constant-coefficient "
                         "kernels) or the coefficient-jump box (16x8x8 coarsest, beta 1 | 100, Robin face: the "
                         "general kernels)")
    ap.add_argument("--profile-tiles", default=None,
                    help="with --profile-kernel 0: the K1 tile shape ry,kz of the finest level (as autotuned in the bench)")
    ap.add_argument("--cg-form", default="auto", choices=["auto", "two", "single"],
                    help="MIXED step of the headline solve: the library default (single pass below 2^22 nodes, "
                         "two passes above), two-pass (K1 + K2) or single-pass (one kernel) on every level")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the two other paper-scale workloads (variable-beta box in FP64, jump case MIXED)")
    ap.add_argument("--no-compare-form", action="store_true",
                    help="skip timing the other MIXED step form beside the headline one")
    ap.add_argument("--eager", action="store_true",
                    help="host-driven level loops instead of one CUDA graph per solve (same kernels); "
                         "ncu cannot profile kernel nodes of graphs that hold conditional nodes")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, world, device):
    """The largest value over the ranks of the job (every rank gets it); value itself at N = 1."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), mx=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [r for r in rows if r["power"] > 200.0] or rows
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("pcap", "sw_power_cap")):
            if any(r[key].lower().startswith("active") for r in loaded):
                reasons.append(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded), "sm_max_mhz": max(r["mx"] for r in rows),
                "reasons": reasons, "samples": len(loaded)}


FALLBACK_HBM_GBS = 6800.0  # one earlier copy measurement on a GB300, used when no measured file exists


def peaks():
    """The measured peaks (MEASURED_PEAKS.json), or the fallback HBM copy rate, with its source."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if d.get("hbm_gbs"):
            d["source"] = "MEASURED_PEAKS.json hbm_gbs (copy; of measured)"
            return d
    except (OSError, ValueError):
        pass
    return {"hbm_gbs": FALLBACK_HBM_GBS, "source": "fallback 6800 GB/s (no MEASURED_PEAKS.json; of fallback)"}


def free_dofs(n):
    return (n - 1) ** 3


def host_cpu():
    """(logical cores, CPU model) of this host, from os.cpu_count and lscpu (or /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def cpu_baseline(args, levels_one=5, levels_omp=6, min_seconds=10.0, max_runs=4):
    """The oracle as it stands on the host cores, two legs on the benchmark problem cut to a
    bounded sample: the one-thread build up to 8*2^(levels_one-1) (repeated until about
    min_seconds of work), and the OpenMP build on every host core up to 8*2^(levels_omp-1) (one
    run). Each leg reports finest free dofs / wall time, and the set-up (CSR assembly, loads) and
    solve seconds apart. The headline value is the all-core leg."""
    import oracle
    from paper_1506_02983_gb300 import inputs
    oracle.build()
    oracle.build_omp()
    nproc, model = host_cpu()
    legs = []
    for levels, threads, runs_max in ((levels_one, None, max_runs), (levels_omp, nproc, 1)):
        p = inputs.cos_cube(levels=levels, n0=(args.n0,) * 3, rtol=args.rtol)
        runs, total, asm, sol, used = 0, 0.0, 0.0, 0.0, 1
        while runs < runs_max and (runs == 0 or total < min_seconds):
            t0 = time.perf_counter()
            _, st = oracle.ecmg(p, p["rtol"], threads=threads)
            total += time.perf_counter() - t0
            asm += st["seconds_assembly"]
            sol += st["seconds_solve"]
            used = st["threads"]
            runs += 1
        nf = args.n0 << (levels - 1)
        dt = total / runs
        legs.append(dict(value=free_dofs(nf) / dt / 1e9, unit="Gdof/s", cores=used, finest="%d^3" % nf,
                         levels=levels, runs=runs, seconds_per_run=dt, seconds_assembly=asm / runs,
                         seconds_solve=sol / runs, iters=st["iters"],
                         build="one thread" if threads is None else "OpenMP (CSR products, vector updates)"))
        del p
    main = legs[1]
    return dict(value=main["value"], unit="Gdof/s", cores=main["cores"], kind="oracle",
                sample="oracle ECMG_jcg FP64 (OpenMP build, %d threads) on the same problem cut to %s (%d levels), "
                       "one run of %.1f s (set-up %.1f s, solve %.1f s); finest free dofs / wall time"
                       % (main["cores"], main["finest"], main["levels"], main["seconds_per_run"],
                          main["seconds_assembly"], main["seconds_solve"]),
                host={"nproc": nproc, "cpu_model": model}, legs=legs)


def arm_config(args, world):
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    L, n0 = args.levels, args.n0
    nf = n0 << (L - 1)
    return {"workload": "cos_cube Poisson unit cube, u=cos(pi x)cos(pi y)cos(pi z), all-Dirichlet, "
                        "Q1, %d^3 -> %d^3 (%d levels), rtol %g, exact load functional" % (n0, nf, L, args.rtol),
            "precision": "MIXED (FP32 JCG, FP64 residual replacement)",
            "l2": "inputs and finest vectors (>1 GB each) larger than L2",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "loop_control": "host (eager)" if args.eager else "CUDA graph, conditional nodes",
            "mixed_step": {"single": "single-pass (one kernel per JCG step, ECMG_CG_SINGLE_PASS)",
                           "two": "two-pass (K1 + K2 per JCG step, ECMG_CG_TWO_PASS)",
                           "auto": "ECMG_CG_AUTO (the default): single-pass below 2^22 nodes, two-pass above"}[
                               args.cg_form],
            "tiles": "FP32 stencil tile shapes autotuned after the first solve (ecmg_autotune)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    steps, warm = args.steps, args.warmup
    # each step a bounded sample: the hierarchy cut at 128^3 (64^3 for long runs), so that the
    # whole run ends within a few minutes
    levels = min(args.cpu_levels, 4) if steps + warm > 30 else args.cpu_levels
    import oracle
    from paper_1506_02983_gb300 import inputs
    oracle.build_omp()
    nproc, model = host_cpu()
    p = inputs.cos_cube(levels=levels, n0=(args.n0,) * 3, rtol=args.rtol)
    for _ in range(warm):
        oracle.ecmg(p, p["rtol"], threads=nproc)
    t0 = time.perf_counter()
    asm = sol = 0.0
    used = 1
    for _ in range(steps):
        _, st = oracle.ecmg(p, p["rtol"], threads=nproc)
        asm += st["seconds_assembly"]
        sol += st["seconds_solve"]
        used = st["threads"]
    dt = (time.perf_counter() - t0) / steps
    nf = args.n0 << (levels - 1)
    v = free_dofs(nf) / dt / 1e9
    # the same workload as the GPU arm, as a bounded sample: what this arm runs is stated in
    # config (the FP64 oracle on one core, the hierarchy cut at nf^3)
    cfg = arm_config(args, world)
    for k in ("loop_control", "mixed_step", "tiles", "l2"):
        cfg.pop(k, None)
    cfg.update(precision="FP64 (the plain C oracle: CSR assembly, banded Cholesky, JCG, EXP_finite, EXP_true)",
               parallelism="OpenMP build of the oracle on %d host cores (%s)" % (used, model),
               sample="each step solves the same problem cut to %d^3 (%d levels) instead of %d^3" % (
                   nf, levels, args.n0 << (args.levels - 1)))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gdof/s", "n_gpus": args.gpus,
           "steps": steps, "warmup": warm, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": v, "unit": "Gdof/s", "cores": used, "kind": "oracle",
                            "sample": "each step: the plain C FP64 oracle (CSR assembly, banded Cholesky, JCG; OpenMP "
                                      "build) on the same cos_cube problem cut to %d^3 (%d levels), rtol %g; value = "
                                      "free dofs of that finest level / step time; set-up %.2f s and solve %.2f s "
                                      "per step" % (nf, levels, args.rtol, asm / steps, sol / steps),
                            "host": {"nproc": nproc, "cpu_model": model}},
           "e2e": {"value": v, "unit": "Gdof/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def profile_kernel(args):
    import torch
    from paper_1506_02983_gb300 import build, inputs
    build.build()
    from paper_1506_02983_gb300 import ecmg
    if args.profile_workload == "jump":
        p = inputs.jump_singular(levels=args.levels, rtol=1e-8, device="cuda")
        nfin = 16 << (args.levels - 1)
    else:
        p = inputs.cos_cube(levels=args.levels, n0=(args.n0,) * 3, rtol=args.rtol)
        nfin = args.n0 << (args.levels - 1)
    s = ecmg.solver_from_problem(p, precision=ecmg.ECMG_MIXED, max_iters=args.max_iters,
                                 cg_form={"auto": ecmg.ECMG_CG_AUTO, "two": ecmg.ECMG_CG_TWO_PASS,
                                          "single": ecmg.ECMG_CG_SINGLE_PASS}[args.cg_form])
    st, status = s.solve()
    if args.profile_tiles:
        ry, kz = (int(v) for v in args.profile_tiles.split(","))
        s.set_tiles(ry, kz, -1)
    ry, kz = s.get_tiles(-1)
    for w in [int(v) for v in str(args.profile_kernel).split(",")]:
        torch.cuda.nvtx.range_push("kernel_profile")
        ms, nb = s.time_kernel(w, -1, reps=2)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"kernel": w, "workload": args.profile_workload, "n": nfin, "ms": ms, "algorithmic_bytes": nb,
                          "GBps": nb / ms / 1e6, "tiles": [ry, kz], "solve_status": status}))
    s.close()


def profile_batched(args):
    import torch
    from paper_1506_02983_gb300 import build, inputs
    build.build()
    from paper_1506_02983_gb300 import ecmg
    dev = []
    for p in inputs.batch_problems():
        q = dict(p)
        q["beta"] = torch.as_tensor(p["beta"]).cuda()
        q["f"] = torch.as_tensor(p["f"]).cuda()
        dev.append(q)
    bs = ecmg.BatchSolver(dev, rtol=1e-8, max_iters=args.max_iters, autotune=1)
    st, status = bs.solve()
    for w in (0, 1, 2):
        torch.cuda.nvtx.range_push("kernel_profile")
        ms, nb = bs.time_kernel(w, -1, reps=2)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"batched_kernel": w, "ms": ms, "algorithmic_bytes": nb, "GBps": nb / ms / 1e6,
                          "solve_status": status}))
    bs.close()


def bench_extra():
    """The two other paper-scale single-GPU workloads, timed after a warm-up solve: the
    variable-beta box (512 x 512 x 1024 elements, Robin on z = 0) in FP64 and in MIXED, and the
    jump case (1024 x 512 x 512, beta 1 | 100, singular u, Robin on x = 0) in MIXED, with the
    general FP32 stencil kernel's own device timer for its roofline."""
    import numpy as np
    import torch
    from paper_1506_02983_gb300 import ecmg, inputs
    pk = peaks().get("hbm_gbs")
    out = {}

    def timed_solve(s, steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            st, status = s.solve()
        e1.record()
        torch.cuda.synchronize()
        assert status == 0, st
        return e0.elapsed_time(e1) / steps, st

    p = inputs.variable_box(levels=7, rtol=1e-9)
    n = inputs.finest(p["n0"], p["levels"])
    free = (n[0] - 1) * (n[1] - 1) * n[2]  # Dirichlet on five faces, Robin on z = 0
    ue = torch.from_numpy(np.ascontiguousarray(p.pop("u_exact"))).cuda()
    wl = ("box (0,1)x(0,1)x(0,2), 8x8x16 -> 512x512x1024 elements (7 levels), beta = 1 + 0.5 sin(2 pi x) "
          "cos(2 pi y) sin(pi z), Dirichlet on five faces, Robin alpha = 1 on z = 0, rtol 1e-9")
    for name, precision, steps in (("variable_box_fp64", ecmg.ECMG_FP64, 1), ("variable_box_mixed", ecmg.ECMG_MIXED, 2)):
        s = ecmg.solver_from_problem(p, precision=precision, autotune=1 if precision == ecmg.ECMG_MIXED else 0)
        u = torch.empty_like(ue)
        s.solve(u)
        ms, st = timed_solve(s, steps)
        s.solve(u)
        out[name] = {
            "workload": wl + (", FP64" if precision == ecmg.ECMG_FP64 else ", MIXED"),
            "ms_per_solve": ms, "value": free / (ms * 1e-3) / 1e9, "unit": "Gdof/s (finest free dofs / solve time)",
            "finest_free_dofs": free, "iters": st["iters"], "level_seconds": st["seconds"],
            "setup_seconds": st["setup_seconds"], "max_err": (u - ue).abs().max().item()}
        s.close()
        del u
    del p, ue

    p = inputs.jump_singular(levels=7, rtol=1e-8, device="cuda")
    n = inputs.finest(p["n0"], p["levels"])
    free = n[0] * (n[1] - 1) * (n[2] - 1)  # Robin on x = 0, Dirichlet elsewhere
    s = ecmg.solver_from_problem(p, precision=ecmg.ECMG_MIXED, autotune=1)
    s.solve()
    s.stencil_timer(-1, reset=True)
    ms, st = timed_solve(s, 2)
    k1_total, k1_n = s.stencil_timer(-1, reset=True)
    k1_ms_alone, k1_bytes = s.time_kernel(0, -1, reps=10)
    k1_live = k1_total / max(k1_n, 1)
    gbps = k1_bytes / k1_live / 1e6
    out["jump_mixed"] = {
        "workload": "box (0,2)x(0,1)x(0,1), 16x8x8 -> 1024x512x512 elements (7 levels), beta 1 for x < 1 and 100 "
                    "for x > 1, u = r^1.5, Robin alpha = 1 on x = 0, Dirichlet elsewhere, rtol 1e-8, MIXED",
        "ms_per_solve": ms, "value": free / (ms * 1e-3) / 1e9, "unit": "Gdof/s (finest free dofs / solve time)",
        "finest_free_dofs": free, "iters": st["iters"], "updates": st["updates"], "level_seconds": st["seconds"],
        "setup_seconds": st["setup_seconds"],
        "stencil_roofline": {"kernel": "K1 general path (k_pq32_tma: variable beta, a Robin face), finest level",
                             "bound": "hbm", "achieved": gbps, "peak": pk, "unit": "GB/s",
                             "frac": gbps / pk if pk else None, "algorithmic_bytes_per_launch": k1_bytes,
                             "launch_ms": k1_live, "launches_timed": k1_n, "launch_ms_alone_cuda_events": k1_ms_alone,
                             "tiles": list(s.get_tiles(-1))}}
    s.close()
    del p
    torch.cuda.empty_cache()
    return out


def bench_batched(args, steps, warmup):
    """64 independent problems (per-axis sizes from {32, 48, 64, 96, 128} cubic elements of side
    1/128, lognormal beta clipped to contrast 1e2, f ~ U[-1, 1] per node, g_D = 0), seed 1506,
    rtol 1e-8, MIXED, one batched solve per step (ecmg_solve_batched)."""
    import numpy as np
    import torch
    from paper_1506_02983_gb300 import ecmg, inputs
    probs = inputs.batch_problems()
    dev = []
    for p in probs:
        q = dict(p)
        q["beta"] = torch.as_tensor(p["beta"]).cuda()
        q["f"] = torch.as_tensor(p["f"]).cuda()
        dev.append(q)
    bs = ecmg.BatchSolver(dev, rtol=1e-8, max_iters=args.max_iters, use_graph=0 if args.eager else 1,
                          inner_rtol=args.inner_rtol, autotune=1,
                          cg_form=ecmg.ECMG_CG_TWO_PASS if args.batched_form == "two" else ecmg.ECMG_CG_SINGLE_PASS)
    for _ in range(warmup):
        st, status = bs.solve()
        assert status == 0, status
    l0 = ecmg.kernel_launches()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("ecmg_batched_timed")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        st, status = bs.solve()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1) / steps
    launches = (ecmg.kernel_launches() - l0) // steps
    # the FP32 stencil (K1) and residual (K2) launches of the last stage alone (every problem's
    # finest level), CUDA events around each launch
    two_pass = args.batched_form == "two"
    if two_pass:
        k1_ms, k1_bytes = bs.time_kernel(0, reps=10)
        k2_ms, k2_bytes = bs.time_kernel(1, reps=10)
    else:
        k1_ms, k1_bytes = bs.time_kernel(11, reps=10)
    pk = peaks()
    dofs = sum(int(np.prod([(v << (p["levels"] - 1)) - 1 for v in p["n0"]])) for p in probs)
    work = 0  # node-iterations of JCG over all problems and levels
    for p, s in zip(probs, st):
        for l in range(p["levels"]):
            work += s["iters"][l] * int(np.prod([(v << l) + 1 for v in p["n0"]]))
    bs.close()
    return {"workload": "64 problems, per-axis N from {32,48,64,96,128} (h = 1/128), lognormal beta (sigma 1, "
                        "contrast 1e2), f ~ U[-1,1], g_D = 0, rtol 1e-8, MIXED, seed 1506",
            "value": dofs / (ms * 1e-3) / 1e9, "unit": "Gdof/s", "solve_ms": ms, "finest_free_dofs": dofs,
            "steps": steps, "warmup": warmup, "gpu_launches": launches,
            "jcg_node_iterations": work, "max_iters_per_level": [max((s["iters"][l] if l < s["levels"] else 0) for s in st)
                                                                 for l in range(max(s["levels"] for s in st))],
            "worst_rel_res_finest": max(s["rel_res"][s["levels"] - 1] for s in st),
            "replacements": sum(sum(s["updates"]) for s in st), "inner_rtol": args.inner_rtol,
            "loop_control": "host (eager)" if args.eager else "CUDA graph, conditional nodes",
            "tiles": "batched FP32 stencil tile shapes autotuned at creation (per stage, per size class)",
            "mixed_step": "two-pass (K1 + K2)" if two_pass else "single-pass (one kernel per JCG step)",
            "roofline": {"kernel": ("batched K1 (bk_pq_tma: TMA-staged FP32 stencil, variable beta)" if two_pass else
                                    "batched single-pass step (bk_step_tma: TMA-staged FP32 residual update, search "
                                    "direction, stencil and dots, variable beta)") + " over the 64 finest levels, alone",
                         "bound": "hbm",
                         "achieved": k1_bytes / k1_ms / 1e6, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": k1_bytes / k1_ms / 1e6 / pk["hbm_gbs"], "algorithmic_bytes_per_launch": k1_bytes,
                         "launch_ms": k1_ms, "peak_source": pk["source"]},
            "k2_alone": ({"kernel": "batched K2 (bk_update) over the 64 finest levels", "ms": k2_ms,
                          "algorithmic_bytes": k2_bytes, "GBps": k2_bytes / k2_ms / 1e6} if two_pass else None)}


def main():
    args = parse()
    if args.batched_only:
        import torch
        from paper_1506_02983_gb300 import build
        build.build()
        r = bench_batched(args, args.steps, args.warmup)
        print(json.dumps({"metric": "batched ECMG_jcg solve, aggregate Gdof/s", **r}))
        return
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_kernel is not None:
        return profile_kernel(args)
    if args.profile_batched:
        return profile_batched(args)
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1506_02983_gb300 import build, inputs
    build.build()
    from paper_1506_02983_gb300 import ecmg

    L, n0 = args.levels, args.n0
    nf = n0 << (L - 1)
    p = inputs.cos_cube(levels=L, n0=(n0,) * 3, rtol=args.rtol)
    dev = torch.device("cuda", local)
    host = {k: torch.from_numpy(np.ascontiguousarray(p[k], dtype=np.float64)).pin_memory()
            for k in ("beta", "f", "gD")}
    d = {k: v.to(dev) for k, v in host.items()}
    u_exact = torch.from_numpy(np.ascontiguousarray(p["u_exact"])).to(dev)
    del p["beta"], p["f"], p["gD"]

    single = args.cg_form == "single"
    form = {"auto": ecmg.ECMG_CG_AUTO, "two": ecmg.ECMG_CG_TWO_PASS, "single": ecmg.ECMG_CG_SINGLE_PASS}
    other_form = "two" if args.cg_form != "two" else "auto"

    def sp_level(l):
        """Whether level l runs the single-pass step in the headline form."""
        n = (n0 << l) + 1
        return l >= 2 and (single or (args.cg_form == "auto" and n ** 3 < ecmg.ECMG_AUTO_SINGLE_PASS_NODES))

    def make(precision, cg_form=args.cg_form):
        return ecmg.Solver(p["n0"], L, p["lo"], p["hi"], p["face_bc"], p["alpha"], d["beta"], d["f"],
                           d["gD"], None, f_mode=ecmg.ECMG_F_LOAD, rtol=args.rtol, precision=precision,
                           max_iters=args.max_iters, use_graph=0 if args.eager else 1, inner_rtol=args.inner_rtol,
                           cg_form=form[cg_form] if precision == ecmg.ECMG_MIXED else ecmg.ECMG_CG_TWO_PASS)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    def timed(fn, steps):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)

    torch.cuda.synchronize()
    t_create = time.perf_counter()
    mixed = make(ecmg.ECMG_MIXED)
    torch.cuda.synchronize()
    create_ms = (time.perf_counter() - t_create) * 1e3
    # slots of the ring of search directions on the two-pass levels (ECMG_RING_AUTO resolved)
    ring_slots = mixed.ring_slots()
    u_out = torch.empty_like(u_exact)
    st_mixed, status = mixed.solve(u_out)
    assert status == 0, st_mixed
    # tile shapes timed on the set-up levels (the level flags of the set-up pick the kernels' paths)
    mixed.autotune(3)
    for _ in range(args.warmup):
        st_mixed, status = mixed.solve(u_out)
        assert status == 0, st_mixed
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ecmg.kernel_launches()
    for l in range(L):
        mixed.stencil_timer(l, reset=True)
    torch.cuda.nvtx.range_push("ecmg_mixed_timed")
    ms_mixed = timed(lambda: mixed.solve(u_out), args.steps)
    torch.cuda.nvtx.range_pop()
    launches = (ecmg.kernel_launches() - launches0) // args.steps
    clk = clocks.stop()
    # K1 launches of the finest level inside the timed solves: the kernel's own device timer
    # (earliest block start to end of last block per launch; CUDA events cannot sit inside the
    # conditional-node bodies of the solve graph)
    k1_live_total_ms, k1_live_n = mixed.stencil_timer(-1)
    # the FP32 step kernel's own device time per level and solve (K1, or the single-pass step),
    # beside the level's device time: on the small levels the rest is launch, conditional-node
    # and reduction latency
    step_kernel_ms = []
    for l in range(L):
        t_ms, n_l = mixed.stencil_timer(l, reset=True)
        step_kernel_ms.append({"ms_per_solve": t_ms / args.steps, "launches_per_solve": n_l / args.steps})
    st_mixed, status = mixed.solve(u_out)
    assert status == 0, st_mixed
    err_mixed = mixed.norms(u_out, u_exact)[0]
    # the error columns of the tables of Sec. 5 on the finest level (max and RMS norms over all
    # nodes), and r_h = ||W - U||_2 / ||U - u||_2
    e_u = mixed.norms(u_out, u_exact)
    w_fin = mixed.get(ecmg.ECMG_VEC_W)
    e_w = mixed.norms(w_fin, u_out)
    del w_fin
    ut_fin = mixed.extrapolate()
    e_t = mixed.norms(ut_fin, u_exact)
    del ut_fin
    table_norms = {"level": "%d^3" % nf, "U_minus_u": {"max": e_u[0], "rms": e_u[1]},
                   "Utilde_minus_u": {"max": e_t[0], "rms": e_t[1]}, "W_minus_U": {"max": e_w[0], "rms": e_w[1]},
                   "r_h": e_w[1] / e_u[1] if e_u[1] else None,
                   "note": "MIXED solution; Utilde = EXP_true, W = EXP_finite guess; rms = sqrt(sum e^2 / nodes)"}

    # kernels alone (finest level), for the roofline
    pk = peaks()
    hbm_peak = pk.get("hbm_gbs")
    kern = {}
    names = {0: "k_pq<float> (K1 FP32)", 1: "k_update<float> (K2 FP32)", 2: "k_res<float> (FP64 residual)",
             5: "k_res<double>", 6: "k_exp_finite", 7: "k_exp_true", 11: "k_step32 (single-pass FP32 step)"}
    step_kernel = 11 if single else 0
    for w in [int(x) for x in args.kernels.split(",") if x != ""]:
        if w in (3, 4) or (single and w in (0, 1)) or (w == 11 and not single):
            continue
        ms, nb = mixed.time_kernel(w, -1, reps=10)
        kern[names.get(w, str(w))] = {"ms": ms, "algorithmic_bytes": nb, "GBps": nb / ms / 1e6}
    k1_ms, k1_bytes = mixed.time_kernel(step_kernel, -1, reps=20)
    k1_live_ms = k1_live_total_ms / max(k1_live_n, 1)
    tiles = mixed.get_tiles(-1)
    mixed_tiles = tiles
    level_tiles = {l: mixed.get_tiles(l) for l in range(2, L)}

    # end to end through the C ABI from pinned host buffers
    u_host = torch.empty(u_exact.shape, dtype=torch.float64).pin_memory()

    def e2e_step():
        for k in ("beta", "f", "gD"):
            d[k].copy_(host[k], non_blocking=True)
        mixed.solve(u_out)
        u_host.copy_(u_out, non_blocking=True)

    ms_e2e_dense = timed(e2e_step, args.e2e_steps)
    h2d_dense = sum(v.numel() * 8 for v in host.values())
    d2h = u_host.numel() * 8
    mixed.close()

    # end to end with compact inputs: f and g_D as separable factors (Gauss samples, nodal
    # factors), beta as one constant; the load functional and the coarse levels are assembled on
    # the device inside the solve
    pc = inputs.cos_cube_compact(levels=L, n0=(n0,) * 3, rtol=args.rtol, with_exact=False)
    hostc = {k: torch.from_numpy(np.ascontiguousarray(pc[k], dtype=np.float64)).pin_memory() for k in ("f", "gD")}
    dc = {k: v.to(dev) for k, v in hostc.items()}
    compact = ecmg.Solver(pc["n0"], L, pc["lo"], pc["hi"], pc["face_bc"], pc["alpha"], None, dc["f"], dc["gD"],
                          None, f_mode=ecmg.ECMG_F_SEPARABLE, f_terms=pc["f_terms"], gD_terms=pc["gD_terms"],
                          beta_const=pc["beta_const"], rtol=args.rtol, precision=ecmg.ECMG_MIXED,
                          max_iters=args.max_iters, use_graph=0 if args.eager else 1, inner_rtol=args.inner_rtol)
    st_c, status = compact.solve(u_out)
    assert status == 0, st_c
    for l in range(2, L):  # same level sizes and kernels as the dense-input handle: its tuned shapes
        compact.set_tiles(*level_tiles[l], level=l)

    def e2e_compact():
        for k in ("f", "gD"):
            dc[k].copy_(hostc[k], non_blocking=True)
        compact.solve(u_out)
        u_host.copy_(u_out, non_blocking=True)

    for _ in range(2):
        e2e_compact()
    ms_e2e = timed(e2e_compact, args.e2e_steps)
    h2d = sum(v.numel() * 8 for v in hostc.values())
    st_c, status = compact.solve(u_out)
    assert status == 0, st_c
    err_compact = compact.norms(u_out, u_exact)[0]
    compact.close()

    # the other MIXED step form on the same problem, for comparison (same warm-up and timing)
    other = None
    if not args.no_compare_form:
        alt = make(ecmg.ECMG_MIXED, cg_form=other_form)
        st_alt, status = alt.solve(u_out)
        assert status == 0, st_alt
        alt.autotune(3)
        for _ in range(args.warmup):
            alt.solve(u_out)
        alt.stencil_timer(-1, reset=True)
        ms_alt = timed(lambda: alt.solve(u_out), args.steps)
        alt_total, alt_n = alt.stencil_timer(-1, reset=True)
        st_alt, status = alt.solve(u_out)
        assert status == 0, st_alt
        other = {"mixed_step": {"two": "two-pass", "auto": "auto"}[other_form], "ms_per_step": ms_alt,
                 "value": free_dofs(nf) * world / (ms_alt * 1e-3) / 1e9, "unit": "Gdof/s",
                 "iters": st_alt["iters"], "updates": st_alt["updates"], "rel_res": st_alt["rel_res"],
                 "max_err": alt.norms(u_out, u_exact)[0], "tiles_finest": list(alt.get_tiles(-1)),
                 "level_seconds": st_alt["seconds"], "setup_seconds": st_alt["setup_seconds"],
                 "finest_step_kernel_ms": alt_total / max(alt_n, 1),
                 "finest_step_kernels": alt_n / max(args.steps, 1)}
        alt.close()

    fp64 = make(ecmg.ECMG_FP64)
    st64, status = fp64.solve(u_out)
    assert status == 0, st64
    torch.cuda.nvtx.range_push("ecmg_fp64_timed")
    ms_fp64 = timed(lambda: fp64.solve(u_out), args.fp64_steps)
    torch.cuda.nvtx.range_pop()
    err_fp64 = fp64.norms(u_out, u_exact)[0]
    fp64.close()

    batched = None
    if not args.no_batched:
        batched = bench_batched(args, args.batched_steps, 2)
    extra = None if args.no_extra else bench_extra()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, args.cpu_levels, args.cpu_levels_omp)

    dofs = free_dofs(nf) * world
    node_its = sum(free_dofs(n0 << l) * st_mixed["iters"][l] for l in range(L))
    value = dofs / (ms_mixed * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "k_pq_float_traffic.json")
    if os.path.exists(tpath):
        try:
            tj = json.load(open(tpath))
            if (tj.get("n") == nf and list(tj.get("tiles", [])) == list(mixed_tiles)
                    and tj.get("algorithmic_bytes_per_launch") == k1_bytes):
                traffic = tj.get("dram_bytes_per_launch")
        except ValueError:
            pass
    k1_gbps = k1_bytes / k1_live_ms / 1e6
    # bytes per node-iteration of the step each level runs: 32 single-pass; two-pass 36 with the
    # correction vector (K1 24, K2 12), and with a ring of R search directions 28 (K1 16, K2 12)
    # + 4 (each direction read back once) + 8 / (R - 2) (e written and read once per full ring)
    two_pass_bytes = 36.0 if ring_slots == 0 else 32.0 + 8.0 / (ring_slots - 2)
    node_bytes = sum(free_dofs(n0 << l) * st_mixed["iters"][l] * (32.0 if sp_level(l) else two_pass_bytes)
                     for l in range(L))
    bpni = node_bytes / max(node_its, 1)
    out = {
        "metric": METRIC, "value": value, "unit": "Gdof/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": arm_config(args, world),
        "solve_ms_mixed": ms_mixed, "solve_ms_fp64": ms_fp64, "speedup_mixed_vs_fp64": ms_fp64 / ms_mixed,
        "max_err_mixed": err_mixed, "max_err_fp64": err_fp64,
        "err_ratio_mixed_over_fp64": err_mixed / err_fp64,
        "table_norms_finest": table_norms,
        "iters_mixed": st_mixed["iters"], "updates_mixed": st_mixed["updates"],
        "ring_slots_mixed": ring_slots, "iters_fp64": st64["iters"],
        "level_seconds_mixed": st_mixed["seconds"], "setup_seconds_mixed": st_mixed["setup_seconds"],
        "step_kernel_per_level_mixed": step_kernel_ms,
        "rel_res_mixed": st_mixed["rel_res"], "gdofs_fp64": dofs / (ms_fp64 * 1e-3) / 1e9,
        "roofline": {"kernel": ("single-pass step (k_step32_cc on this one-beta all-Dirichlet level: residual "
                                "update, search direction, 27-point operator and the dots in one pass)" if single else
                                "K1 (k_pq32_cc on this one-beta all-Dirichlet level: FP32 search direction + "
                                "27-point operator)") + ", finest level",
                     "bound": "hbm", "achieved": k1_gbps, "peak": hbm_peak, "unit": "GB/s",
                     "frac": (k1_gbps / hbm_peak) if hbm_peak else None, "traffic": traffic,
                     "algorithmic_bytes_per_launch": k1_bytes,
                     "launch_ms": k1_live_ms, "launches_timed": k1_live_n,
                     "timing": "device global timer per launch inside the timed solves (earliest block start to "
                               "end of last block), averaged over the launches of the finest level",
                     "launch_ms_alone_cuda_events": k1_ms, "tiles": {"ry": tiles[0], "kz": tiles[1]},
                     "peak_source": pk["source"]},
        "kernels_alone": kern,
        # the two ways of counting dofs: finest free dofs per solve (value), and free dofs times
        # JCG iterations summed over the levels; the byte model charges each node-iteration the
        # bytes the step moves on a constant-coefficient level: about 32 for K1 and K2 with the
        # ring of search directions (36 without), 32 for the single-pass kernel
        # (bytes_per_node_iteration is their iteration-weighted mean)
        "node_iterations_per_solve": node_its,
        "gdofs_node_iterations": node_its * world / (ms_mixed * 1e-3) / 1e9,
        "byte_model": {"bytes_per_node_iteration": bpni, "bytes_per_solve": bpni * node_its,
                       "fraction_of_peak": (bpni * node_its / (ms_mixed * 1e-3) / 1e9 / hbm_peak) if hbm_peak else None},
        "other_mixed_step_form": other,
        "roofline_frac_of_spec_8tbs": k1_gbps / 8000.0,
        "create_ms": create_ms,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": dofs / (ms_e2e * 1e-3) / 1e9, "unit": "Gdof/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                "inputs": "compact: f as one separable term at the 3-point Gauss nodes, g_D as one separable "
                          "term, beta_const (ECMG_F_SEPARABLE); load assembled on the device; solution read back",
                "max_err": err_compact, "iters": st_c["iters"]},
        "e2e_dense_inputs": {"value": dofs / (ms_e2e_dense * 1e-3) / 1e9, "unit": "Gdof/s",
                             "h2d_bytes_per_step": h2d_dense, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e_dense,
                             "inputs": "dense beta, load functional and g_D arrays (ECMG_F_LOAD)"},
        "cpu_baseline": cpu,
        "batched": batched,
        "paper_scale_workloads": extra,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
