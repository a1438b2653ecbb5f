"""Benchmark: 12 point-source solves of the Wilson-clover operator to a true
FP64 relative residual of 1e-10, including the adaptive setup, with the
2-level DD-alpha-AMG solver on one GB300.

Workload (synthetic, seeded): 16^4 lattice, near-unit SU(3) links
U = exp(i 0.25 H) (seed 1), m0 = -0.3, csw = 1.2, antiperiodic in time;
4^4 Schwarz blocks = aggregates, 4 SAP cycles of 4 MR iterations, n_v = 20
test vectors from 4 setup iterations; FP32 smoother / coarse GMRES / projections,
FP64 outer FGMRES; the 12 spin-colour point sources at the origin solved
one after the other.  One step = setup (clover term, test vectors, coarse
operator) + 12 solves, with the links resident in device memory.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own replica of the workload; nothing is exchanged between GPUs.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "12-RHS solves/s at 1e-10 incl. setup"
UNIT = "solves/s"
WORKLOAD = dict(L=(16, 16, 16, 16), block=(4, 4, 4, 4), eps=0.25, seed=1, m0=-0.3, csw=1.2,
                n_v=20, setup_iters=4, n_sap=4, mr_iters=4, coarse_tol=5e-2, tol=1e-10)
# algorithmic (compulsory) bytes per site of one launch of each timed kernel,
# FP32 storage with two-row links: SAP sweep reads b, x, 4 links, A, A^-1 and
# writes x on its blocks (the coarse GMRES bytes are computed below).
SAP_BYTES_PER_SITE = 4 * (24 + 24 + 24 + 48 + 72 + 72)
L2_BYTES = 129 * 2 ** 20
# DRAM bytes (read + write) per launch of each timed kernel class on this
# workload, from an ncu capture of the kernel as it is now (a single-RHS
# coarse solve); None where no capture of a single-RHS launch of the kernel
# as it is now exists
TRAFFIC_BYTES_PER_LAUNCH = {"sap_sweep": None, "coarse_gmres": 42_921_472 + 40_448}
# stencil bandwidth lattice: 32^3 x 64 (the lattice of the batched workload),
# far larger than L2, links tiled from an 8^4 field of the same generator
STENCIL = dict(L=(32, 32, 32, 64), tile=(8, 8, 8, 8), block=(4, 4, 4, 4), eps=0.2, seed=3, m0=-0.3, csw=1.5,
               n_v=24, reps=20)
# the 32^3 x 64 batched workload: 12 point sources in one lockstep batch,
# n_v 24, FP32 inner solver with FP64 refinement; m0 = -0.125 is where the
# unpreconditioned CG count of this ensemble peaks (mass_tuning.scan_mass on
# the GPU: about 2100 iterations predicted there, no mass reaches 5000)
LARGE = dict(L=(32, 32, 32, 64), block=(4, 4, 4, 4), eps=0.2, seed=3, m0=-0.125, csw=1.5, n_v=24,
             outer_restart=10, tol=1e-10)
# the 48^3 x 96 light-mass workload: eps 0.15, csw 1.6, m0 = m_c + 0.02 with
# m_c read from an 8^4 proxy (seed 5) and corrected for the proxy's
# antiperiodic lowest mode, n_v 32, FP16 storage with FP32 arithmetic and
# FP64 refinement, the 12 point sources in lockstep batches of three (outer
# restart 6), the setup's temporaries and FP64 test vectors released
# before the solves
HUGE = dict(L=(48, 48, 48, 96), block=(4, 4, 4, 4), eps=0.15, seed=5, m0=-0.034, csw=1.6, n_v=32,
            outer_restart=6, batch=3, tol=1e-10)
# compulsory bytes per site of one fine D apply: in and out spinor (24 reals
# each), four two-row links (12 reals each), packed clover A (72 reals)
D_REALS_PER_SITE = 24 + 24 + 4 * 12 + 72
WORKLOAD_NAME = ("16^4 Wilson-clover, eps 0.25, m0 -0.3, csw 1.2, 4^4 blocks and aggregates, n_v 20, "
                 "4 setup iters, 4 SAP cycles x 4 MR, 12 point sources one at a time to 1e-10; "
                 "FP32 smoother, coarse GMRES and projections, FP64 outer FGMRES")


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "of measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        for line in out.strip().splitlines():
            parts = [v.strip() for v in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def job_seconds(local_seconds, world, device):
    """The job's timed region: the maximum over ranks (replicas run
    independently; the slowest one bounds the job)."""
    if world == 1:
        return local_seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(solves_per_step, steps, world, seconds):
    """Whole-job solves/s: every rank solves its own replica each step."""
    return solves_per_step * steps * world / seconds


def workload_params(P):
    w = WORKLOAD
    return P.default_params(L=w["L"], sap_block=w["block"], n_v=w["n_v"], m0=w["m0"], csw=w["csw"],
                            setup_iters=w["setup_iters"], n_sap=w["n_sap"], mr_iters=w["mr_iters"],
                            coarse_tol=w["coarse_tol"], precision=P.FP32, seed=12345)


def sap_sweep_marginal_us(P, torch, stream, U_dev, x_dev, reps=20):
    """Live duration of one SAP colour sweep inside the smoother: CUDA events
    around `reps` back-to-back ddamg_sap calls (FP32, one right-hand side) on
    the workload with its N_SAP cycles and with half of them; the difference
    per extra sweep leaves out each call's input and output conversion."""
    w = WORKLOAD
    full, half = w["n_sap"], w["n_sap"] // 2
    if half < 1:
        raise ValueError("the marginal sweep needs at least two SAP cycles")
    t = {}
    for n_sap in (full, half):
        p = workload_params(P)
        p.n_sap = n_sap
        s = P.DDAMG(p, U_dev, stream=stream.cuda_stream)
        try:
            s.run_setup()
            for _ in range(3):
                s.sap(x_dev, P.FP32)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                s.sap(x_dev, P.FP32)
            e1.record(stream)
            torch.cuda.synchronize()
            t[n_sap] = e0.elapsed_time(e1) * 1e3 / reps
        finally:
            s.close()
    return (t[full] - t[half]) / (2 * (full - half)), {str(k): round(v, 2) for k, v in t.items()}


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_1811_00355_gb300 as P
    import synthetic as syn

    rank, local, world = env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    P.load()
    w = WORKLOAD
    L = w["L"]
    V = int(np.prod(L))
    U_host = syn.gauge_field(L, w["eps"], w["seed"] + rank)
    b_host = np.ascontiguousarray(syn.point_sources(L))
    U_dev = torch.from_numpy(U_host).cuda()
    b_dev = torch.from_numpy(b_host).cuda()
    stream = torch.cuda.current_stream()
    params = workload_params(P)
    solver = P.DDAMG(params, U_dev, stream=stream.cuda_stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        solver.run_setup()
        x, info = solver.solve(b_dev, w["tol"])
        return x, info

    for _ in range(args.warmup):
        x, info = step()
    torch.cuda.synchronize()
    bad = [i for i in info if not (i["converged"] and i["true_residual"] <= w["tol"])]
    if bad:
        raise RuntimeError(f"warm-up solves did not converge: {bad}")

    solver.reset_stats()
    times = []
    infos = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)                     # evict L2 between timed steps
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, info = step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            infos.append(info)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches = solver.stats()["kernel_launches"]
    # per-kernel device times for the roofline line come from one more step
    # with CUDA events around every timed launch (events between kernels
    # also serialise them, so this step is not part of the timed value)
    solver.reset_stats()
    solver.enable_kernel_timing(True)
    flush.fill_(1.0)
    step()
    torch.cuda.synchronize()
    st = solver.stats()
    solver.enable_kernel_timing(False)
    hist_f, hist_r = solver.history()
    flops = {"model": "theoretical real flops of the method's arithmetic (ddamg_get_history)",
             "setup_mflop_per_site": round(st["setup_flops"] / V / 1e6, 3),
             "solve_mflop_per_site": round(st["solve_flops"] / 12 / V / 1e6, 3),
             "last_solve_history": [[round(float(f), 3), float("%.3g" % r)] for f, r in zip(hist_f, hist_r)]}
    for info in infos:
        for i in info:
            if not (i["converged"] and i["true_residual"] <= w["tol"]):
                raise RuntimeError(f"a timed solve missed the tolerance: {i}")
    T = job_seconds(sum(times), world, "cuda")
    value = job_throughput(12, args.steps, world, T)
    ms_per_step = 1e3 * T / args.steps

    # roofline of the dominant timed kernel.  A SAP sweep's live duration is
    # taken at the margin of back-to-back smoother calls (events around every
    # launch would keep the next sweep's prologue from overlapping the
    # previous one); the other classes from the events around their launches
    pk, pk_kind = peaks()
    sweep_us, sap_calls = sap_sweep_marginal_us(P, torch, stream, U_dev, b_dev[:1].contiguous())
    classes = {"sap_sweep": (st["sap_ms"], st["sap_launches"]),
               "coarse_gmres": (st["coarse_ms"], st["coarse_launches"]),
               "dslash": (st["dslash_ms"], st["dslash_launches"])}
    live_ms = {k: v[0] for k, v in classes.items()}
    live_ms["sap_sweep"] = sweep_us * 1e-3 * st["sap_launches"]
    dom = max(live_ms, key=lambda k: live_ms[k])
    ms, n = live_ms[dom], classes[dom][1]
    roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": None, "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(dom), "peak_kind": pk_kind + " (burst copy)",
            "share_of_step": round(ms / (1e3 * T / args.steps) if T else 0.0, 3),
            "sap_sweep_live_us": round(sweep_us, 2), "sap_calls_us": sap_calls}
    if dom == "sap_sweep" and n:
        per_launch = (V // 2) * SAP_BYTES_PER_SITE
        achieved = per_launch / (sweep_us * 1e-6) / 1e9
        roof.update(achieved=round(achieved, 1), frac=round(achieved / pk["hbm_gbs"], 4),
                    algorithmic_bytes_per_launch=per_launch, avg_launch_us=round(sweep_us, 2),
                    timing="marginal sweep of back-to-back ddamg_sap calls (4 and 2 SAP cycles)")
    elif dom == "coarse_gmres" and n:
        nx = V // 256
        n2 = 2 * w["n_v"]
        # one iteration streams the 9 blocks of D_c of every even site and the
        # 8 premultiplied blocks A_oo^-1 D_c of every odd site (FP32 complex)
        per_iter = (nx // 2) * (9 + 8) * n2 * n2 * 8
        its = sum(i["coarse_iters"] for info in infos for i in info)
        per_launch = per_iter * its / max(1, sum(i["precond_calls"] for info in infos for i in info))
        achieved = per_launch / (ms / n * 1e-3) / 1e9
        roof.update(achieved=round(achieved, 1), frac=round(achieved / pk["hbm_gbs"], 4),
                    algorithmic_bytes_per_launch=int(per_launch), avg_launch_us=round(1e3 * ms / n, 2),
                    timing="CUDA events around every launch of one extra step")

    # end to end through the public API with host buffers: one handle kept
    # across configurations (as a production loop would); every step uploads
    # its links and right-hand sides from pinned host memory, runs the setup
    # and the 12 solves, and reads the solutions back into pinned host memory
    e2e = None
    if not args.no_e2e:
        solver.close()
        torch.cuda.synchronize()
        U_pin = torch.from_numpy(U_host).pin_memory().numpy()
        b_pin = torch.from_numpy(b_host).pin_memory().numpy()
        x_pin = torch.empty(b_host.shape, dtype=torch.complex128).pin_memory().numpy()
        s2 = P.DDAMG(params, U_pin, stream=stream.cuda_stream)
        et = []
        try:
            for k in range(max(1, min(args.steps, 3)) + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s2.set_gauge(U_pin)
                s2.run_setup()
                xh, inf = s2.solve(b_pin, w["tol"], out=x_pin)
                t1 = time.perf_counter()
                if k:
                    et.append(t1 - t0)
                if not all(i["converged"] for i in inf):
                    raise RuntimeError(f"end-to-end solve missed the tolerance: {inf}")
        finally:
            s2.close()
        e2e = {"value": round(job_throughput(12, 1, world, job_seconds(statistics.mean(et), world, "cuda")), 3),
               "unit": UNIT, "h2d_bytes_per_step": int(U_host.nbytes + b_host.nbytes),
               "d2h_bytes_per_step": int(x_pin.nbytes)}

    var = None
    if rank == 0 and world == 1 and not args.no_variants:
        var = variants(P, torch, stream, U_dev, b_dev, args.steps, flush)

    srv = None
    if rank == 0 and world == 1 and not args.no_serving:
        srv = serving(P, torch, stream)

    sten = None
    if rank == 0 and not args.no_stencils:
        sten = stencils(P, torch, stream, pk, pk_kind)

    large = None
    if rank == 0 and world == 1 and not args.no_large:
        solver.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        large = large_batched()

    three = None
    if rank == 0 and world == 1 and not args.no_three_level:
        solver.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        three = three_level()

    huge = None
    if rank == 0 and world == 1 and not args.no_huge:
        solver.close()                 # (idempotent) the child needs nearly all of the device memory
        del flush
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        huge = huge_batched()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk.summary(),
            "solve_stats": {"outer_iters_per_rhs": statistics.mean(i["outer_iters"] for i in infos[-1]),
                            "precond_calls": sum(i["precond_calls"] for i in infos[-1]),
                            "coarse_iters": sum(i["coarse_iters"] for i in infos[-1]),
                            "max_true_residual": max(i["true_residual"] for info in infos for i in info),
                            "step_seconds": [round(t, 4) for t in times]},
            "kernel_ms": {k: round(v[0], 3) for k, v in classes.items()},
            "flops": flops,
            "variants": var,
            "serving": srv,
            "stencils": sten,
            "batched_32x32x32x64": large,
            "light_mass_48x48x48x96": huge,
            "three_level_32x32x32x64": three,
            "autotune": P.tuning(),
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def variants(P, torch, stream, U_dev, b_dev, steps, flush):
    """The same 12-RHS workload (setup + 12 point sources to 1e-10) in other
    forms: the 12 sources solved together in one lockstep batch (FP32 inner
    solver), the plain single-RHS form with an FP64 inner solver, the
    single-RHS form with the test vectors of R and P stored in FP16, and the
    single-RHS form with the test vectors orthonormalised in FP32."""
    w = WORKLOAD
    out = {}
    for name, prec, batched, n in (("batched_f32", P.FP32, True, steps), ("single_f64", P.FP64, False, 1),
                                   ("single_f32_half_vectors", P.FP32, False, steps),
                                   ("single_f32_ortho_fp32", P.FP32, False, steps)):
        params = workload_params(P)
        params.precision = prec
        params.half_vectors = 1 if name.endswith("half_vectors") else 0
        params.ortho_fp32 = 1 if name.endswith("ortho_fp32") else 0
        s = P.DDAMG(params, U_dev, stream=stream.cuda_stream)
        solve = s.solve_batched if batched else s.solve
        try:
            s.run_setup()
            solve(b_dev, w["tol"])
            times, infos = [], []
            for _ in range(n):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.run_setup()
                x, info = solve(b_dev, w["tol"])
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                infos.append(info)
            for info in infos:
                for i in info:
                    if not (i["converged"] and i["true_residual"] <= w["tol"]):
                        raise RuntimeError(f"{name}: a solve missed the tolerance: {i}")
            out[name] = {"value": round(12 * n / sum(times), 3), "unit": UNIT, "steps": n,
                         "ms_per_step": round(1e3 * sum(times) / n, 2),
                         "dtype": "f32+f64" if prec == P.FP32 else "f64",
                         "outer_iters_per_rhs": statistics.mean(i["outer_iters"] for i in infos[-1]),
                         "max_true_residual": max(i["true_residual"] for info in infos for i in info)}
        finally:
            s.close()
    # the paper's second-mass use of a setup: keep the test vectors, change
    # m0 (heavier quark), rebuild the clover term and D_c, solve again
    params = workload_params(P)
    s = P.DDAMG(params, U_dev, stream=stream.cuda_stream)
    try:
        s.run_setup()
        m_new = w["m0"] + 0.1
        s.update_mass(m_new, w["csw"])
        s.solve_batched(b_dev, w["tol"])
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.update_mass(m_new, w["csw"])
        e1.record(stream)
        x, info = s.solve_batched(b_dev, w["tol"])
        e2.record(stream)
        torch.cuda.synchronize()
        for i in info:
            if not (i["converged"] and i["true_residual"] <= w["tol"]):
                raise RuntimeError(f"new-mass solve missed the tolerance: {i}")
        t_up = e0.elapsed_time(e1) / 1e3
        t_all = e0.elapsed_time(e2) / 1e3
        out["new_mass_batched_f32"] = {"value": round(12 / t_all, 3), "unit": UNIT, "m0": m_new,
                                       "update_ms": round(1e3 * t_up, 2), "ms_per_step": round(1e3 * t_all, 2),
                                       "outer_iters_per_rhs": statistics.mean(i["outer_iters"] for i in info),
                                       "max_true_residual": max(i["true_residual"] for i in info)}
    finally:
        s.close()
    return out


# serving stream: four resident gauge configurations, 8^4, 16^4, 24^3 x 48
# and 32^3 x 64 (eps, m0, csw drawn once from eps in [0.2, 0.3], m0 in
# [-0.4, -0.2], csw in [1.0, 1.5] with a fixed seed), Poisson arrivals, 1-12
# Gaussian or point-source right-hand sides per request at tol 1e-8 or
# 1e-10, two configurations served at a time, device memory admitted up to
# 250 GB (the two large configurations together fit, all four do not).  The
# arrival rate keeps the offered load (about 3 right-hand sides per second,
# a quarter of them on 32^3 x 64) below what the largest lattice can serve.
SERVING = dict(lattices=((8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 64)), requests=24,
               rate_hz=0.5, seed=2024, max_batch=12, restart=16, workers=4, budget=250 * 2 ** 30)


def serving(P, torch, stream):
    """p50 / p99 latency (submit to results on the host) and solves/s of a
    Poisson request stream through the library's serving loop."""
    import threading
    import synthetic as syn
    sv = SERVING
    gen = np.random.default_rng(sv["seed"])
    srv = P.Server(hbm_budget=sv["budget"], max_batch=sv["max_batch"], workers=sv["workers"])
    cfgs = []
    try:
        for i, L in enumerate(sv["lattices"]):
            eps, m0, csw = gen.uniform(0.2, 0.3), gen.uniform(-0.4, -0.2), gen.uniform(1.0, 1.5)
            p = P.default_params(L=L, sap_block=(4, 4, 4, 4), n_v=20, m0=m0, csw=csw, precision=P.FP32,
                                 outer_restart=sv["restart"])
            U = (syn.gauge_field(L, eps, 11 + i) if np.prod(L) <= 2 ** 20 else
                 syn.gauge_field_sliced(L, eps, 11 + i, workers=min(16, os.cpu_count() or 1)))
            cid = srv.add_config(p, U)
            del U
            cfgs.append({"L": "x".join(map(str, L)), "eps": round(eps, 3), "m0": round(m0, 3),
                         "csw": round(csw, 3), "id": cid})
        # requests drawn up front (host inputs are part of the request)
        reqs = []
        for k in range(sv["requests"]):
            c = cfgs[int(gen.integers(len(cfgs)))]
            L = tuple(int(v) for v in c["L"].split("x"))
            n = int(gen.integers(1, 13))
            tol = 1e-8 if gen.random() < 0.5 else 1e-10
            if gen.random() < 0.5:
                rhs = syn.gaussian_spinors(n, L, 1000 + k)
            else:
                rhs = np.ascontiguousarray(syn.point_sources(L)[:n])
            reqs.append((c["id"], rhs, tol, float(gen.exponential(1.0 / sv["rate_hz"]))))
        # warm: every config set up once (resident afterwards)
        for c in cfgs:
            L = tuple(int(v) for v in c["L"].split("x"))
            srv.wait(srv.submit(c["id"], syn.gaussian_spinors(1, L, 7), 1e-8))
        ids = [None] * len(reqs)
        t0 = time.perf_counter()

        def feed():
            for k, (cid, rhs, tol, gap) in enumerate(reqs):
                time.sleep(gap)
                ids[k] = srv.submit(cid, rhs, tol)

        th = threading.Thread(target=feed)
        th.start()
        lat, batch_req, nrhs = [], [], 0
        for k in range(len(reqs)):
            while ids[k] is None:
                time.sleep(0.0005)
            x, info, ri = srv.wait(ids[k])
            if not all(i["converged"] for i in info):
                raise RuntimeError(f"serving: request {k} did not converge: {info}")
            lat.append(ri["latency_seconds"])
            batch_req.append(ri["batch_requests"])
            nrhs += reqs[k][1].shape[0]
        th.join()
        wall = time.perf_counter() - t0
    finally:
        srv.close()
    lat = np.array(lat)
    per_cfg = {}
    for (cid, _, _, _), l in zip(reqs, lat):
        per_cfg.setdefault(cid, []).append(l)
    return {"p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "solves_per_s": round(nrhs / wall, 3), "requests": len(lat), "rhs": nrhs,
            "arrival_rate_hz": sv["rate_hz"], "mean_requests_per_batch": round(float(np.mean(batch_req)), 2),
            "workers": sv["workers"], "hbm_budget_GB": round(sv["budget"] / 2 ** 30),
            "configs": [dict({k: v for k, v in c.items() if k != "id"},
                             p50_latency_s=round(float(np.percentile(per_cfg.get(c["id"], [0.0]), 50)), 4),
                             requests=len(per_cfg.get(c["id"], [])))
                        for c in cfgs],
            "note": ("latency = submit to results in host memory; continuous batching (requests join a running "
                     "batch between restart cycles), up to %d configurations served at a time on their own "
                     "streams; setups done before the stream, idle configurations released by the memory budget"
                     % sv["workers"])}


def _tiled(a, small, L):
    """Periodic tiling of a per-site array of the small lattice onto L."""
    sx, sy, sz, st = small
    inner = a.shape[1:]
    a = a.reshape((st, sz, sy, sx) + inner)
    a = np.tile(a, (L[3] // st, L[2] // sz, L[1] // sy, L[0] // sx) + (1,) * len(inner))
    return np.ascontiguousarray(a.reshape((-1,) + inner))


def large_batched():
    """The 32^3 x 64 batched workload in a child process (its ~200 GB of
    device memory and any failure stay out of this process); returns its
    JSON object, or {"error": ...}."""
    import subprocess
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--large-only"], cwd=ROOT,
                           capture_output=True, text=True, timeout=1200)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode != 0 or not lines:
            return {"error": "exit %d: %s" % (r.returncode, (r.stderr or r.stdout)[-400:])}
        return json.loads(lines[-1])
    except Exception as e:                      # noqa: BLE001 - reported in the JSON line
        return {"error": repr(e)[:400]}


LARGE_RUN = dict(precisions=("f32", "bf16", "fp16"), passes=2, oracle_check=True)


def large_batched_child():
    """Setup + the 12 point sources as one batch on 32^3 x 64 in each inner
    precision (FP32, then BF16 and FP16 storage), twice each (the first pass
    allocates the batch buffers); the second is timed with CUDA events.
    Every solution's true residual is then checked with the CPU oracle's D.
    Prints one JSON object."""
    import torch
    import paper_1811_00355_gb300 as P
    import synthetic as syn
    s = LARGE
    if not torch.cuda.is_available():
        raise SystemExit("no CUDA device")
    t0 = time.perf_counter()
    U = syn.gauge_field_sliced(s["L"], s["eps"], s["seed"], workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    torch.cuda.set_device(0)
    P.load()
    stream = torch.cuda.current_stream()
    U_dev = torch.from_numpy(U).cuda()
    b_dev = torch.from_numpy(syn.point_sources(s["L"])).cuda()
    out = {"lattice": "32x32x32x64", "m0": s["m0"], "csw": s["csw"], "eps": s["eps"], "n_v": s["n_v"],
           "rhs": "12 point sources, one batch", "unit": UNIT, "gauge_generation_s": round(gen_s, 1),
           "timing": "CUDA events, second of two passes"}
    sols = {}
    precs = {"f32": P.FP32, "bf16": P.BF16, "fp16": P.FP16}
    for name in LARGE_RUN["precisions"]:
        prec = precs[name]
        params = P.default_params(L=s["L"], sap_block=s["block"], n_v=s["n_v"], m0=s["m0"], csw=s["csw"],
                                  outer_restart=s["outer_restart"], precision=prec)
        h = P.DDAMG(params, U_dev, stream=stream.cuda_stream)
        try:
            for _ in range(LARGE_RUN["passes"]):
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                ev[0].record(stream)
                h.run_setup()
                ev[1].record(stream)
                x, info = h.solve_batched(b_dev, s["tol"])
                ev[2].record(stream)
                torch.cuda.synchronize()
            setup_s = ev[0].elapsed_time(ev[1]) / 1e3
            solve_s = ev[1].elapsed_time(ev[2]) / 1e3
            sols[name] = x.cpu().numpy()
            del x
            out[name] = {"value": round(12 / (setup_s + solve_s), 3), "dtype": name + "+f64",
                         "setup_s": round(setup_s, 3), "solve_s": round(solve_s, 3),
                         "outer_iters_per_rhs": statistics.mean(i["outer_iters"] for i in info),
                         "max_true_residual": max(i["true_residual"] for i in info),
                         "all_converged": all(i["converged"] and i["true_residual"] <= s["tol"] for i in info),
                         "device_GB": round(h.stats()["device_bytes"] / 1e9, 1)}
        finally:
            h.close()
            torch.cuda.empty_cache()
    if not LARGE_RUN["oracle_check"]:
        print(json.dumps(out))
        return
    # every source's true residual once more with the CPU oracle's own D
    t_or = time.perf_counter()
    del U_dev
    torch.cuda.empty_cache()
    from oracle.dirac import WilsonClover
    op = WilsonClover(torch.from_numpy(U), s["L"], s["m0"], s["csw"])
    del U
    b_host = syn.point_sources(s["L"])
    for name, xs in sols.items():
        res = []
        for k in range(12):
            r = torch.from_numpy(b_host[k]) - op.apply(torch.from_numpy(xs[k]))
            res.append(float(torch.linalg.vector_norm(r) / np.linalg.norm(b_host[k])))
        out[name]["max_true_residual_oracle_D"] = max(res)
        out[name]["all_converged"] = out[name]["all_converged"] and max(res) <= s["tol"]
    out["oracle_check_s"] = round(time.perf_counter() - t_or, 1)
    # the line's headline for this workload: the BF16-storage batch
    out["value"] = out.get("bf16", out.get("f32", {})).get("value")
    print(json.dumps(out))


# three levels on the 32^3 x 64 lattice: level-2 blocks (= aggregates) of
# 2^4 coarse sites (a 4^3 x 8 coarsest lattice), 16 level-2 test vectors
THREE = dict(block2=(2, 2, 2, 2), n_v2=16, setup_iters2=2, sources=2,
             smoothers2=((4, 4), (2, 2), (1, 2)))      # level-2 (SAP cycles, MR iterations); the first is the default


def three_level():
    """The two- and three-level comparison on 32^3 x 64 in a child process;
    returns its JSON object, or {"error": ...}."""
    import subprocess
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--three-level-only"], cwd=ROOT,
                           capture_output=True, text=True, timeout=1200)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode != 0 or not lines:
            return {"error": "exit %d: %s" % (r.returncode, (r.stderr or r.stdout)[-400:])}
        return json.loads(lines[-1])
    except Exception as e:                      # noqa: BLE001 - reported in the JSON line
        return {"error": repr(e)[:400]}


def three_level_child():
    """32^3 x 64 (the batched workload's lattice and mass), FP32 inner
    precision: after the two-level setup, the first point sources solved
    one at a time with two levels, then with three after the level-2 setup.
    Reports per level count the outer iterations, the coarse-solve
    iterations per preconditioner call (the even-odd GMRES on D_c for two
    levels, the FGMRES on D_c preconditioned by M2 for three), the time per
    solve (CUDA events) and the level-2 setup time.  One JSON object."""
    import torch
    import paper_1811_00355_gb300 as P
    import synthetic as syn
    s, th = LARGE, THREE
    if not torch.cuda.is_available():
        raise SystemExit("no CUDA device")
    U = syn.gauge_field_sliced(s["L"], s["eps"], s["seed"], workers=min(16, os.cpu_count() or 1))
    torch.cuda.set_device(0)
    P.load()
    stream = torch.cuda.current_stream()
    U_dev = torch.from_numpy(U).cuda()
    b_dev = torch.from_numpy(syn.point_sources(s["L"])[:th["sources"]]).cuda()
    params = P.default_params(L=s["L"], sap_block=s["block"], n_v=s["n_v"], m0=s["m0"], csw=s["csw"],
                              outer_restart=s["outer_restart"], precision=P.FP32)
    h = P.DDAMG(params, U_dev, stream=stream.cuda_stream)
    out = {"lattice": "32x32x32x64", "m0": s["m0"], "csw": s["csw"], "n_v": s["n_v"],
           "level2": {"block": list(th["block2"]), "n_v": th["n_v2"], "setup_iters": th["setup_iters2"]},
           "rhs": "point sources %s, one at a time, to %g" % (list(range(th["sources"])), s["tol"]),
           "timing": "CUDA events per solve"}
    try:
        h.run_setup()
        runs = [(2, None)] + [(3, sm) for sm in th["smoothers2"]]
        for levels, sm in runs:
            rec = {}
            if levels == 3:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h.level2_init(P.level2_default_params(block=th["block2"], n_v=th["n_v2"],
                                                      setup_iters=th["setup_iters2"], n_sap=sm[0],
                                                      mr_iters=sm[1]))
                h.level2_setup()
                torch.cuda.synchronize()
                rec["level2_setup_s"] = round(time.perf_counter() - t0, 3)
                rec["level2_n_sap"], rec["level2_mr_iters"] = sm
                h.set_levels(3)
            times, infos = [], []
            for k in range(th["sources"]):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x, info = h.solve(b_dev[k:k + 1], s["tol"])
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                infos.append(info[0])
            rec.update({"solve_s": [round(v, 3) for v in times],
                        "outer_iters": [i["outer_iters"] for i in infos],
                        "precond_calls": [i["precond_calls"] for i in infos],
                        "coarse_iters_per_call": [round(i["coarse_iters"] / max(1, i["precond_calls"]), 1)
                                                  for i in infos],
                        "true_residual": [i["true_residual"] for i in infos],
                        "all_converged": all(i["converged"] and i["true_residual"] <= s["tol"] for i in infos)})
            if levels == 2 or sm == th["smoothers2"][0]:
                out["levels_%d" % levels] = rec
            else:
                out.setdefault("levels_3_other_smoothers", []).append(rec)
    finally:
        h.close()
    print(json.dumps(out))


def huge_batched():
    """The 48^3 x 96 light-mass workload in a child process; returns its
    JSON object, or {"error": ...}."""
    import subprocess
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--huge-only"], cwd=ROOT,
                           capture_output=True, text=True, timeout=2400)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode != 0 or not lines:
            return {"error": "exit %d: %s" % (r.returncode, (r.stderr or r.stdout)[-400:])}
        return json.loads(lines[-1])
    except Exception as e:                      # noqa: BLE001 - reported in the JSON line
        return {"error": repr(e)[:400]}


def huge_batched_child():
    """Setup + the 12 point sources (lockstep batches of three) on 48^3 x 96
    at the light mass, FP16 storage, one pass timed with CUDA events (host
    buffers: each batch's right-hand sides and solutions cross PCIe/NVLink-C2C
    inside its timed region).  The library reports every solution's FP64
    true residual; the first source of every batch is checked once more
    with the CPU oracle's D.  Prints one JSON object."""
    import torch
    import paper_1811_00355_gb300 as P
    import synthetic as syn
    s = HUGE
    if not torch.cuda.is_available():
        raise SystemExit("no CUDA device")
    t0 = time.perf_counter()
    U = syn.gauge_field_sliced(s["L"], s["eps"], s["seed"], workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    b = syn.point_sources(s["L"])
    torch.cuda.set_device(0)
    P.load()
    stream = torch.cuda.current_stream()
    params = P.default_params(L=s["L"], sap_block=s["block"], n_v=s["n_v"], m0=s["m0"], csw=s["csw"],
                              outer_restart=s["outer_restart"], precision=P.FP16)
    out = {"lattice": "48x48x48x96", "m0": s["m0"], "csw": s["csw"], "eps": s["eps"], "n_v": s["n_v"],
           "rhs": "12 point sources, lockstep batches of %d" % s["batch"], "unit": UNIT, "dtype": "fp16+f64",
           "gauge_generation_s": round(gen_s, 1),
           "timing": "CUDA events, one pass; solves include the host<->device copies of their fields"}
    h = P.DDAMG(params, U, stream=stream.cuda_stream)
    xs = np.empty_like(b)
    infos = []
    try:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        h.run_setup()
        ev[1].record(stream)
        torch.cuda.synchronize()
        setup_s = ev[0].elapsed_time(ev[1]) / 1e3
        setup_GB = h.stats()["device_bytes"] / 1e9
        h.trim()
        solve_s = 0.0
        for k0 in range(0, 12, s["batch"]):
            torch.cuda.synchronize()
            ev[0].record(stream)
            x, info = h.solve_batched(np.ascontiguousarray(b[k0:k0 + s["batch"]]), s["tol"])
            ev[1].record(stream)
            torch.cuda.synchronize()
            solve_s += ev[0].elapsed_time(ev[1]) / 1e3
            xs[k0:k0 + s["batch"]] = x
            infos.extend(info)
        out.update({"value": round(12 / (setup_s + solve_s), 4), "setup_s": round(setup_s, 2),
                    "solve_s": round(solve_s, 2),
                    "outer_iters_per_rhs": statistics.mean(i["outer_iters"] for i in infos),
                    "coarse_iters_per_precond": round(sum(i["coarse_iters"] for i in infos)
                                                      / max(1, sum(i["precond_calls"] for i in infos)), 1),
                    "max_true_residual": max(i["true_residual"] for i in infos),
                    "all_converged": all(i["converged"] and i["true_residual"] <= s["tol"] for i in infos),
                    "device_GB_setup": round(setup_GB, 1),
                    "device_GB_solve": round(h.stats()["device_bytes"] / 1e9, 1)})
    finally:
        h.close()
    t_or = time.perf_counter()
    from oracle.dirac import WilsonClover
    op = WilsonClover(torch.from_numpy(U), s["L"], s["m0"], s["csw"])
    del U
    res = []
    checked = list(range(0, 12, s["batch"]))       # the first source of every batch
    for k in checked:
        r = torch.from_numpy(b[k]) - op.apply(torch.from_numpy(xs[k]))
        res.append(float(torch.linalg.vector_norm(r) / np.linalg.norm(b[k])))
    out["max_true_residual_oracle_D"] = max(res)
    out["oracle_D_sources"] = checked
    out["all_converged"] = out["all_converged"] and max(res) <= s["tol"]
    out["oracle_check_s"] = round(time.perf_counter() - t_or, 1)
    print(json.dumps(out))


def stencils(P, torch, stream, pk, pk_kind):
    """Achieved HBM bandwidth of the fine D (FP32, FP64) and of the coarse
    9-point stencil (FP32) on a lattice far larger than L2, from the
    library's own per-kernel CUDA-event timing."""
    import synthetic as syn
    s = STENCIL
    L = s["L"]
    V = int(np.prod(L))
    U = torch.from_numpy(_tiled(syn.gauge_field(s["tile"], s["eps"], s["seed"]), s["tile"], L)).cuda()
    x = torch.from_numpy(_tiled(syn.gaussian_spinors(1, s["tile"], s["seed"] + 1)[0], s["tile"], L)).cuda()
    params = P.default_params(L=L, sap_block=s["block"], n_v=s["n_v"], m0=s["m0"], csw=s["csw"],
                              setup_iters=0, precision=P.FP32, seed=777)
    h = P.DDAMG(params, U, stream=stream.cuda_stream)
    out = {"lattice": "x".join(map(str, L)), "peak_gbs": pk["hbm_gbs"], "peak_kind": pk_kind + " (burst copy)",
           "timing": "CUDA events around each kernel launch, %d launches after warm-up" % s["reps"]}
    try:
        for name, prec, rs in (("dslash_f32", P.FP32, 4), ("dslash_f64", P.FP64, 8), ("dslash_bf16", P.BF16, 2),
                               ("dslash_fp16", P.FP16, 2)):
            for _ in range(3):
                h.apply_D(x, prec)
            h.reset_stats()
            h.enable_kernel_timing(True)
            for _ in range(s["reps"]):
                h.apply_D(x, prec)
            st = h.stats()
            h.enable_kernel_timing(False)
            us = 1e3 * st["dslash_ms"] / st["dslash_launches"]
            # half storage: two site norms (FP32) besides the half values
            byts = V * (D_REALS_PER_SITE * rs + (8 if rs == 2 else 0))
            gbs = byts / (us * 1e-6) / 1e9
            out[name] = {"us": round(us, 2), "bytes_per_launch": byts, "GB/s": round(gbs, 1),
                         "frac": round(gbs / pk["hbm_gbs"], 4)}
        # one SAP application (4 cycles of the two colours from a zero start,
        # single right-hand side): per sweep the sites of one colour read b,
        # x (and their neighbours' x, from L2), links, A, A^-1 and write x
        for name, prec, rs, extra in (("sap_sweep_f32", P.FP32, 4, 0), ("sap_sweep_bf16", P.BF16, 2, 12)):
            for _ in range(2):
                h.sap(x, prec)
            h.reset_stats()
            h.enable_kernel_timing(True)
            for _ in range(3):
                h.sap(x, prec)
            st = h.stats()
            h.enable_kernel_timing(False)
            us = 1e3 * st["sap_ms"] / st["sap_launches"]
            byts = (V // 2) * ((24 + 24 + 24 + 48 + 72 + 72) * rs + extra)
            gbs = byts / (us * 1e-6) / 1e9
            out[name] = {"us": round(us, 2), "bytes_per_launch": byts, "GB/s": round(gbs, 1),
                         "frac": round(gbs / pk["hbm_gbs"], 4), "sweeps_timed": st["sap_launches"]}
        del x
        h.run_setup()                      # device-drawn test vectors, SAP, orthonormalise, D_c
        n2 = 2 * s["n_v"]
        nx = h.NX
        gen = np.random.default_rng(s["seed"] + 2)
        xc = torch.from_numpy(gen.standard_normal((nx, n2)) + 1j * gen.standard_normal((nx, n2))).cuda()
        for _ in range(3):
            h.apply_coarse(xc, P.FP32)
        h.reset_stats()
        h.enable_kernel_timing(True)
        for _ in range(s["reps"]):
            h.apply_coarse(xc, P.FP32)
        st = h.stats()
        h.enable_kernel_timing(False)
        us = 1e3 * st["coarse_apply_ms"] / st["coarse_apply_launches"]
        # compulsory bytes: the self and the four forward blocks (the backward
        # blocks follow from them by G5-hermiticity) and the vectors in and out
        byts = nx * (5 * n2 * n2 + 2 * n2) * 8
        gbs = byts / (us * 1e-6) / 1e9
        out["coarse_f32"] = {"us": round(us, 2), "bytes_per_launch": byts, "GB/s": round(gbs, 1),
                             "frac": round(gbs / pk["hbm_gbs"], 4), "n_v": s["n_v"],
                             "bytes": "self + 4 forward 2n x 2n blocks per coarse site, x and y"}
        # restriction (Eq. 3) and prolongation (Eq. 4), one right-hand side:
        # per fine site the n_v test vectors (12 complex each) and one spinor
        xf = torch.from_numpy(_tiled(syn.gaussian_spinors(1, s["tile"], s["seed"] + 3)[0], s["tile"], L)).cuda()
        for name, fn, arg, key in (("restrict_f32", h.restrict, xf, "restrict"),
                                   ("prolong_f32", h.prolong, xc, "prolong")):
            for _ in range(3):
                fn(arg, P.FP32)
            h.reset_stats()
            h.enable_kernel_timing(True)
            for _ in range(s["reps"]):
                fn(arg, P.FP32)
            st = h.stats()
            h.enable_kernel_timing(False)
            us = 1e3 * st[key + "_ms"] / st[key + "_launches"]
            byts = V * (12 * s["n_v"] + 12) * 8
            gbs = byts / (us * 1e-6) / 1e9
            out[name] = {"us": round(us, 2), "bytes_per_launch": byts, "GB/s": round(gbs, 1),
                         "frac": round(gbs / pk["hbm_gbs"], 4), "n_v": s["n_v"]}
        # a batch of 12 right-hand sides (tensor-core products): the test
        # vectors once, 12 spinors, per fine site
        nb_ = 12
        xfb = xf.reshape((1,) + tuple(xf.shape)).repeat(nb_, 1, 1, 1).contiguous()
        xcb = xc.reshape((1,) + tuple(xc.shape)).repeat(nb_, 1, 1).contiguous()
        for name, fn, arg, key in (("restrict_f32_batch12", h.restrict, xfb, "restrict"),
                                   ("prolong_f32_batch12", h.prolong, xcb, "prolong")):
            for _ in range(3):
                fn(arg, P.FP32)
            h.reset_stats()
            h.enable_kernel_timing(True)
            for _ in range(s["reps"]):
                fn(arg, P.FP32)
            st = h.stats()
            h.enable_kernel_timing(False)
            us = 1e3 * st[key + "_ms"] / st[key + "_launches"]
            byts = V * (12 * s["n_v"] + 12 * nb_) * 8
            gbs = byts / (us * 1e-6) / 1e9
            out[name] = {"us": round(us, 2), "bytes_per_launch": byts, "GB/s": round(gbs, 1),
                         "frac": round(gbs / pk["hbm_gbs"], 4), "n_v": s["n_v"], "rhs": nb_,
                         "us_per_rhs": round(us / nb_, 2)}
    finally:
        h.close()
    out["coarse_gmres_8x8x8x16"] = coarse_solver_timing(P, torch, stream, pk)
    return out


# the coarse lattice of the 32^3 x 64 workload (8^3 x 16 aggregates, n_v 24),
# reached from a 16^3 x 32 fine lattice with 2^4 aggregates and the seeded
# synthetic 9-point stencil as D_c (no fine setup needed)
COARSE = dict(L=(16, 16, 16, 32), block=(2, 2, 2, 2), n_v=24, iters=20, reps=5, nrhs=(1, 8, 12))


def coarse_solver_timing(P, torch, stream, pk=None):
    """The coarse even-odd GMRES on 8^3 x 16 coarse sites, n_v 24, FP32, for
    1, 8 and 12 right-hand sides: a fixed number of iterations, timed with
    CUDA events over repeated solves; per iteration it touches the nine D_c
    blocks of every even site and the eight A_oo^-1 D_c blocks of every odd
    site (1.28 GB)."""
    import synthetic as syn
    c = COARSE
    L = c["L"]
    p = P.default_params(L=L, sap_block=c["block"], n_v=c["n_v"], precision=P.FP32, coarse_restart=30,
                         coarse_max_iter=c["iters"])
    h = P.DDAMG(p, syn.unit_gauge(L), stream=stream.cuda_stream)
    n2 = 2 * c["n_v"]
    NX = h.NX
    out = {"coarse_sites": NX, "n_v": c["n_v"], "operator": "synthetic 9-point stencil, diag 1.0, hop 0.21",
           "timing": "CUDA events over %d solves of %d iterations" % (c["reps"], c["iters"])}
    try:
        h.set_coarse_op(syn.coarse_stencil(NX, n2, 5, 1.0, 0.21))
        per_iter = (NX // 2) * (9 + 8) * n2 * n2 * 8
        for nrhs in c["nrhs"]:
            gen = np.random.default_rng(1)
            bc = torch.from_numpy(gen.standard_normal((nrhs, NX, n2)) + 1j * gen.standard_normal((nrhs, NX, n2)))
            bc = bc.cuda()
            for _ in range(2):
                h.coarse_solve(bc, 1e-30, P.FP32)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(c["reps"]):
                x, its = h.coarse_solve(bc, 1e-30, P.FP32)
            e1.record(stream)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / c["reps"]
            it = int(its.max())
            plan = h.coarse_plan(nrhs)
            passes = -(-nrhs // plan["rhs_per_pass"])
            ent = {"us_per_iter": round(us / it, 1), "plan": plan, "passes": passes}
            if pk:
                gbs = per_iter * passes / (us / it * 1e-6) / 1e9
                ent.update({"operator_GB/s": round(gbs, 1), "frac": round(gbs / pk["hbm_gbs"], 4)})
            out["nrhs_%d" % nrhs] = ent
    finally:
        h.close()
    return out


# ---------------------------------------------------------------------------
def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


class OracleRun:
    """The CPU oracle on the 16^4 workload, as it stands: its adaptive setup
    (timed as a whole), then the 12 point sources one after the other, one
    outer FGMRES iteration per call of step() (each timed)."""

    def __init__(self):
        import torch
        import synthetic as syn
        from oracle.solver import Params, TwoLevelMG
        w = WORKLOAD
        L = w["L"]
        self.mg = TwoLevelMG(torch.from_numpy(syn.gauge_field(L, w["eps"], w["seed"])),
                             Params(L, w["block"], w["block"], w["n_v"], w["m0"], w["csw"],
                                    setup_iters=w["setup_iters"], n_sap=w["n_sap"], mr_iters=w["mr_iters"],
                                    coarse_tol=w["coarse_tol"]))
        self.b = torch.from_numpy(syn.point_sources(L))
        t0 = time.perf_counter()
        self.mg.setup(torch.from_numpy(syn.gaussian_spinors(w["n_v"], L, 7)))
        self.setup_s = time.perf_counter() - t0
        self.source = 0
        self.solve_start = 0.0
        self.gen = None
        self.done = []          # (source, iterations, seconds, true residual)

    def step(self):
        """One outer iteration (starting the next source's solve when the
        previous one has finished); returns its seconds."""
        t0 = time.perf_counter()
        if self.gen is None:
            self.gen = self.mg.solve_steps(self.b[self.source], WORKLOAD["tol"])
            self.solve_start = 0.0
        try:
            next(self.gen)
        except StopIteration as fin:
            x, its, ok = fin.value
            res = self.mg.true_residual(self.b[self.source], x)
            dt = time.perf_counter() - t0
            self.done.append((self.source, its, self.solve_start + dt, res))
            self.source = (self.source + 1) % 12
            self.gen = None
            return dt + self.step()
        dt = time.perf_counter() - t0
        self.solve_start += dt
        return dt

    def finish_first_solve(self, cap=200):
        """Run (untimed) until the first source's solve is complete."""
        n = 0
        while not self.done and n < cap:
            self.step()
            n += 1


def _oracle_report(run, measured_s, timed_iters):
    """Throughput of the oracle on the whole workload (setup + 12 solves)
    from what was measured: the setup, and the solve of source 0 with its own
    iteration count (its time, or the timed iterations' mean times its count);
    the other 11 sources are taken to cost as much (the 12 point sources of
    one site differ only in spin and colour)."""
    import torch
    src, its, solve_s, res = run.done[0]
    total = run.setup_s + 12 * solve_s
    return {"value": round(12 / total, 6), "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "cpu": _cpu_model(),
            "measured": {"setup_s": round(run.setup_s, 2), "solve_s_source0": round(solve_s, 2),
                         "outer_iters_source0": its, "true_residual_source0": float("%.3g" % res),
                         "seconds": round(measured_s, 1), "timed_outer_iterations": timed_iters},
            "extrapolated_seconds": round(total, 1),
            "sample": ("the oracle's full adaptive setup and the whole solve of point source 0 (%d outer "
                       "iterations to 1e-10), both timed on the 16^4 workload; the other 11 sources "
                       "extrapolated at source 0's time" % its)}


def cpu_baseline():
    t0 = time.perf_counter()
    run = OracleRun()
    run.finish_first_solve()
    return _oracle_report(run, time.perf_counter() - t0, run.done[0][1])


def run_reference(args):
    """The reference arm: the CPU oracle as it stands.  Its setup runs once
    (timed, outside the steps); each step is then one outer FGMRES iteration
    of the 12 point-source solves, in order, so the steps are a bounded
    sample of the workload's own work.  The line's value is the whole
    workload's throughput from the measured setup and the measured solve of
    source 0 (run to the end after the steps if the steps did not finish it)."""
    rank, local, world = env_rank()
    if rank != 0:
        return
    t_all = time.perf_counter()
    run = OracleRun()
    for _ in range(args.warmup):
        run.step()
    times = [run.step() for _ in range(args.steps)]
    run.finish_first_solve()
    rep = _oracle_report(run, time.perf_counter() - t_all, args.steps)
    step_ms = 1e3 * statistics.mean(times)
    line = {"metric": METRIC, "value": rep["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(step_ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_NAME, "parallelism": "cpu",
                       "step": "one outer FGMRES iteration of the oracle (M, D, Gram-Schmidt)"},
            "cpu_baseline": rep,
            "e2e": {"value": rep["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-stencils", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 32^3 x 64 batched workload")
    ap.add_argument("--large-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-huge", action="store_true", help="skip the 48^3 x 96 light-mass workload")
    ap.add_argument("--huge-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-three-level", action="store_true", help="skip the two/three-level comparison")
    ap.add_argument("--three-level-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--large-precisions", default=None,
                    help="comma list of f32,bf16,fp16 for the 32^3 x 64 workload (default all three)")
    ap.add_argument("--large-passes", type=int, default=None, help="passes of the 32^3 x 64 workload (default 2)")
    ap.add_argument("--large-no-oracle", action="store_true", help="skip the oracle residual check (profiling)")
    ap.add_argument("--stencils-only", action="store_true",
                    help="time only the stencils (for profiler captures) and print their JSON")
    ap.add_argument("--coarse-only", action="store_true",
                    help="time only the coarse GMRES on 8^3 x 16 coarse sites (for profiler captures)")
    ap.add_argument("--stencil-lattice", default=None,
                    help="X,Y,Z,T of the stencil lattice (multiples of 8; default 32,32,32,64)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.stencil_lattice:
        L = tuple(int(v) for v in args.stencil_lattice.split(","))
        if len(L) != 4 or any(v % 8 for v in L):
            raise SystemExit("--stencil-lattice wants four multiples of 8")
        STENCIL["L"] = L
    if args.large_precisions:
        LARGE_RUN["precisions"] = tuple(v for v in args.large_precisions.split(",") if v)
    if args.large_passes:
        LARGE_RUN["passes"] = args.large_passes
    if args.large_no_oracle:
        LARGE_RUN["oracle_check"] = False
    if args.large_only:
        large_batched_child()
        return
    if args.huge_only:
        huge_batched_child()
        return
    if args.three_level_only:
        three_level_child()
        return
    if args.coarse_only:
        import torch
        import paper_1811_00355_gb300 as P
        torch.cuda.set_device(0)
        P.load()
        print(json.dumps({"coarse_gmres_8x8x8x16": coarse_solver_timing(P, torch, torch.cuda.current_stream(),
                                                                         peaks()[0]),
                          "autotune": P.tuning()}))
        return
    if args.stencils_only:
        import torch
        import paper_1811_00355_gb300 as P
        torch.cuda.set_device(0)
        P.load()
        pk, pk_kind = peaks()
        print(json.dumps({"stencils": stencils(P, torch, torch.cuda.current_stream(), pk, pk_kind),
                          "autotune": P.tuning()}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
