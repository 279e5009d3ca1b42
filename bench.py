#!/usr/bin/env python
"""Benchmark of the multigrid low-mode-averaging hot path on GB300.

A step solves one group of right-hand sides D x = b to a FP64 relative
residual of 1e-10 with the mixed-precision multigrid solver (FP64 defect
correction around FP32 flexible GCR preconditioned by T0 D1^-1 R0 with a BF16
coarse stencil, plus MR smoothing).  The default workload is the 2 fm box
shape 64x32^3 with its 96 point + Z2 noise sources; consecutive steps take
consecutive groups of those sources.  The JSON line reports:

* value       -- solves/s with sources resident in HBM (device timing);
* e2e         -- solves/s through the C ABI with pinned host buffers, the
                 host->device copy of b and device->host copy of x inside;
* fp64_plain  -- the plain FP64 CGNE solve on the GPU (bounded sample);
* roofline    -- the dominant kernel's algorithmic bytes / time against the
                 measured HBM peak, from CUDA events on its launch stream;
* cpu_baseline-- the FP64 oracle timed on the host cores (bounded sample);
* clocks      -- nvidia-smi samples taken during the timed region.

`--impl reference` runs the oracle alone as the reference arm.
`--workload c5` serves a seeded Poisson stream over the resident 64x32^3,
96x48^3 and 128x64^3 lattices; `--micro dslash32|dslash64|coarse|transfer|
contract` times one kernel class alone.
Multi-GPU (--gpus N under torchrun): independent replicas, each solving its
own sources (weak scaling); no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s @res 1e-10 mixed vs FP64; dslash GB/s vs HBM peak; p50/p99 latency"

WORKLOADS = {
    # 64x32^3, eps 0.15, kappa 0.1266, csw 1.9, 4^4 blocks, Nv 24 (FP16 basis),
    # 96 sources: 48 point (4 sites x 12 spin-colour) + 48 Z2
    "c4": dict(L=(64, 32, 32, 32), eps=0.15, kappa=0.1266, csw=1.9, block=(4, 4, 4, 4), nv=24, sub_store="fp16",
               coarse_store="bf16", n_smooth=5, n_cg=60, n_sources=96, n_point=48, group=16, cfg=4),
    # 32x16^3, eps 0.2, kappa 0.125, csw 1.7, 4^4 blocks, Nv 16: single-RHS solves
    "c2": dict(L=(32, 16, 16, 16), eps=0.2, kappa=0.125, csw=1.7, block=(4, 4, 4, 4), nv=16, sub_store="fp32",
               coarse_store="bf16", n_smooth=5, n_cg=60, n_sources=64, n_point=0, group=1, cfg=2),
}


# The serving stream of the 2, 3 and 4 fm boxes: lattices generated on the
# device, lean set-up (FP32 test vectors relaxed 4 at a time, FP16 basis, no
# FP64 basis), BF16 coarse operator with its FP64 copy released.
C5 = dict(shapes=[(128, 64, 64, 64), (96, 48, 48, 48), (64, 32, 32, 32)], eps=0.15, kappa=0.1266, csw=1.9,
          block=(4, 4, 4, 4), nv=24, n_smooth=5, n_cg=60, lean_group=4, cfg=5)


# DRAM traffic per lattice site of one launch of a kernel class at a given
# RHS count, from ncu (dram__bytes_read.sum + dram__bytes_write.sum of one
# capture divided by the captured lattice's volume; traffic grows with the
# volume).  The capture and its command are summarised under profiles/.
# 32x16^3, 16 RHS, one FGCR iteration's mix of the class: fused residual,
# fused dots, six fused MR steps (BF16 smoother fields), one plain stencil
NCU_TRAFFIC_PER_SITE = {("dslash32", 16): 5244.9}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def make_sources(m, ctx, w, first, count, out, stream=None):
    """Sources first .. first+count-1 of the workload, generated on the device
    by the library (mglma_sources): point sources first (sites drawn from the
    seed, 12 spin-colour columns each), then Z2 noise."""
    import synthetic
    L = w["L"]
    seed = 3000 + w["cfg"]
    sites = synthetic.point_source_sites(L, max(w["n_point"] // 12, 1), seed)
    i = 0
    while i < count:
        k = (first + i) % w["n_sources"]
        if k < w["n_point"]:
            n = min(count - i, w["n_point"] - k)
            ks = range(k, k + n)
            m.mglma_sources(ctx, L, m.MGLMA_SOURCE_POINT, n, 0, out[i:i + n], point_sites=[int(sites[q // 12]) for q in ks],
                            point_sc=[q % 12 for q in ks], stream=stream)
        else:
            n = min(count - i, w["n_sources"] - k)
            m.mglma_sources(ctx, L, m.MGLMA_SOURCE_Z2, n, seed, out[i:i + n], first=k - w["n_point"], stream=stream)
        i += n


class Clocks:
    """nvidia-smi sampling in the background during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s, pw in zip(sm, power) if pw > 200] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


KINDS = ("dslash64", "dslash32", "blas", "reduce", "restrict", "prolong", "coarse", "pack", "setup", "scalar", "cblas",
         "creduce", "contract")


def replica_source_base(rank, rhs_per_step, nsteps):
    """First source index of a rank: the replicas solve disjoint ranges of the
    workload's sources (weak scaling, no data-path collective)."""
    return rank * rhs_per_step * nsteps


def max_over_ranks(dist, x):
    """The slowest rank's value (the job's time); x itself on one rank."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(rhs_per_step, steps, world, seconds):
    """Whole-job solves/s: the RHS all ranks solved over the slowest rank's time."""
    return rhs_per_step * steps * world / seconds


def profile_snapshot(m, ctx):
    out = {}
    for k in KINDS:
        try:
            out[k] = m.mglma_profile_get(ctx, k)
        except Exception:
            pass
    return out


_ORACLE_JOB = None
_SLAB_JOBS = {}


def _oracle_worker_init(job):
    global _ORACLE_JOB
    _ORACLE_JOB = job


def _oracle_worker_run(iters):
    """One worker process: `iters` CGNE iterations of the oracle on its own
    copy of the slab problem; returns the seconds they took."""
    from oracle import solvers as S
    U, A, b, kappa, csw = _ORACLE_JOB
    t0 = time.perf_counter()
    S.solve_fine(U, b, kappa, csw, tol=1e-300, maxiter=iters, A=A)
    return time.perf_counter() - t0


def _oracle_all_cores(job, procs, iters):
    """Per-iteration seconds of the oracle with every core busy: `procs`
    spawned processes (one BLAS/OpenMP thread each) run the slab problem
    concurrently; the median worker time / iters."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    try:
        for k in keys:
            os.environ[k] = "1"
        with mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init, initargs=(job,)) as pool:
            times = pool.map(_oracle_worker_run, [iters] * procs, chunksize=1)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return float(np.median(times)) / iters


def cpu_baseline(w, gpu_cgne_iters, budget_slices=4, procs=None):
    """The FP64 oracle on the host cores: plain CG on the normal equations
    (the oracle's solver), timed for two iterations on a budget_slices x
    L1 x L2 x L3 slab of the same operator and extrapolated to one full
    solve: per-iteration time x (V / V_slab) x the iteration count the GPU's
    FP64 CGNE needed on this workload.  Timed in one spawned single-threaded
    process (one core), and on all host cores as `procs` concurrent such
    processes (spawned, so safe after CUDA use) whose slab throughput adds up
    as a time-slab decomposition of the full lattice would.  The clover build is set-up, untimed (as the GPU's gauge
    load is)."""
    L = (budget_slices,) + tuple(w["L"][1:])
    key = (L, w["eps"], w["kappa"], w["csw"], w["cfg"])
    if key not in _SLAB_JOBS:  # the slab problem is set-up, built once per process
        import synthetic
        from oracle import dirac as D
        U = synthetic.gauge_links(L, w["eps"], 1000 + w["cfg"])
        A = D.clover_matrix(U, w["kappa"], w["csw"])
        b = synthetic.z2_noise(L, 1, 3000 + w["cfg"])[0]
        _SLAB_JOBS[key] = (U, A, b, w["kappa"], w["csw"])
    job = _SLAB_JOBS[key]
    t_iter = _oracle_all_cores(job, 1, 2)  # one process, one thread
    scale = np.prod(w["L"]) / np.prod(L)
    one = 1.0 / (t_iter * scale * gpu_cgne_iters)
    procs = procs if procs is not None else (os.cpu_count() or 1)
    if procs > 1:
        t_busy = _oracle_all_cores(job, procs, 2)
        value = procs / (t_busy * scale * gpu_cgne_iters)
        how = (f"; all cores: {procs} spawned processes on copies of the slab, {t_busy:.2f} s/iteration each "
               f"under full load, throughput summed")
    else:
        value, how = one, ""
    return {"value": value, "unit": "solves/s", "cores": procs, "kind": "oracle",
            "one_core": {"value": one, "cores": 1, "s_per_iteration": round(t_iter, 3)},
            "sample": (f"2 FP64 CGNE iterations of the numpy oracle on a {'x'.join(map(str, L))} slab "
                       f"({t_iter:.2f} s/iteration on one core), scaled by volume x{scale:.0f} and by the "
                       f"{gpu_cgne_iters} iterations the GPU FP64 CGNE took" + how)}


def run_reference(args, w):
    """The reference arm: the oracle itself, each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    iters = 720 if args.workload == "c4" else 460  # FP64 CGNE counts measured on the GPU for these workloads
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(w, iters, budget_slices=2)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = float(np.mean(vals))
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "lattice": "x".join(map(str, w["L"]))},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}, "vs_baseline": None}
    print(json.dumps(line), flush=True)


COARSE_SOLVERS = {"gcr": 0, "minres": 1, "minres_eo": 2}


def run_serving(m, torch, ctx, g, C, w, args, dev, src_all):
    """Continuous-batching server on the resident lattice: Poisson arrivals
    (seed 4242, 20 requests/s), RHS per request uniform in 1..max, latency
    from arrival to completion.  A request of n RHS takes n consecutive
    sources of the workload's resident set (source buffers are read-only and
    may be shared); the solutions of every request go to one shared sink of
    max RHS (the server checks each RHS's FP64 residual itself), so the
    stream's memory stays bounded however many requests it has."""
    import synthetic
    n = args.serve_requests
    arrivals = synthetic.poisson_arrivals(n, 20.0, 4242)
    sizes = [int(v) for v in synthetic.uniform_ints(n, 1, args.serve_max_rhs, 4242, synthetic.TAG_GROUPS)]
    nsrc = src_all.shape[0]
    sink = torch.zeros((max(sizes), src_all.shape[1], 12), dtype=torch.complex128, device=dev)
    reqs, k = [], 0
    for i in range(n):
        q = min(sizes[i], nsrc)
        k0 = k % (nsrc - q + 1)
        reqs.append(dict(lattice=0, b=src_all[k0:k0 + q], x=sink[:q], arrival=float(arrivals[i])))
        k += q
    torch.cuda.synchronize()
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG, coarse_solver=COARSE_SOLVERS[args.coarse_solver])
    stats, res = m.mglma_serve(ctx, [(g, C)], reqs, prm, max_slots=32, hbm_fraction=0.6)
    del sink
    ok = all(r["status"] == 0 for r in res)
    resid = max(s["residual"] for r in res for s in r["stats"])
    offered_rhs = 20.0 * float(np.mean(sizes))
    return {"requests": stats["requests"], "rhs": stats["rhs"], "p50_s": round(stats["p50_s"], 3),
            "p99_s": round(stats["p99_s"], 3), "mean_s": round(stats["mean_s"], 3), "max_s": round(stats["max_s"], 3),
            "solves_per_s": round(stats["solves_per_s"], 4), "wall_s": round(stats["wall_s"], 2),
            "offered": "Poisson 20 requests/s (seed 4242), RHS per request uniform in 1.." + str(args.serve_max_rhs),
            "offered_rhs_per_s": round(offered_rhs, 1), "achieved_rhs_per_s": round(stats["solves_per_s"], 3),
            "arrival_span_s": round(float(arrivals[-1]), 2),
            "slots": stats["slots"][0], "slot_gb": round(stats["slot_bytes"][0] / 1e9, 2), "all_ok": ok,
            "residual_max": resid}


def run_c5(args):
    """Serving stream over resident 64x32^3, 96x48^3 and 128x64^3 lattices
    (eps 0.15, kappa 0.1266, csw 1.9, 4^4 blocks, Nv 24 FP16 basis, BF16
    coarse operator): Poisson arrivals (20 requests/s, seed 4242), lattice
    shape uniform over the three, RHS per request uniform in 1..max, Z2
    sources generated on the device.  Reports p50/p99 latency, solves/s and
    the sequential FP64 plain (CGNE) service time per shape, the latter from
    timed iterations times the iteration count of a full CGNE solve on the
    smallest shape (labelled extrapolated)."""
    import torch
    import paper_2412_06347_gb300 as m
    import synthetic
    w = C5
    ctx = m.Context(0)
    lats, setup = [], {}
    for i, L in enumerate(w["shapes"]):  # largest first: its set-up has the most room
        t0 = time.perf_counter()
        g = m.mglma_gauge_random(ctx, L, w["eps"], 1000 + 10 * w["cfg"] + i, w["kappa"], w["csw"])
        sub = m.mglma_subspace_create(ctx, g, w["block"], w["nv"], w["n_smooth"], 2000 + 10 * w["cfg"] + i,
                                      m.MGLMA_FP16, n_cg=w["n_cg"], cg_prec=m.MGLMA_FP32, lean_group=w["lean_group"])
        C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
        m.mglma_coarse_release_fp64(C)
        torch.cuda.synchronize()
        free, total = torch.cuda.mem_get_info()
        setup["x".join(map(str, L))] = {"setup_s": round(time.perf_counter() - t0, 1),
                                        "free_gb_after": round(free / 1e9, 1)}
        lats.append(dict(L=L, V=int(np.prod(L)), g=g, sub=sub, C=C))
    n = args.serve_requests
    arrivals = synthetic.poisson_arrivals(n, 20.0, 4242)
    shape = synthetic.uniform_ints(n, 0, len(lats) - 1, 4242, synthetic.TAG_FIELD)
    sizes = synthetic.uniform_ints(n, 1, args.serve_max_rhs, 4242, synthetic.TAG_GROUPS)
    reqs = []
    for i in range(n):
        lt = lats[int(shape[i])]
        b = torch.empty((int(sizes[i]), lt["V"], 12), dtype=torch.complex128, device="cuda")
        m.mglma_sources(ctx, lt["L"], m.MGLMA_SOURCE_Z2, int(sizes[i]), 3000 + w["cfg"], b, first=100 * i)
        reqs.append(dict(lattice=int(shape[i]), b=b, x=torch.zeros_like(b), arrival=float(arrivals[i])))
    torch.cuda.synchronize()
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG)
    stats, res = m.mglma_serve(ctx, [(lt["g"], lt["C"]) for lt in lats], reqs, prm, max_slots=8,
                               hbm_fraction=args.serve_hbm)
    per_shape = {}
    for i, r in enumerate(res):
        key = "x".join(map(str, lats[reqs[i]["lattice"]]["L"]))
        d = per_shape.setdefault(key, {"requests": 0, "rhs": 0, "latency_s": [], "residual_max": 0.0,
                                       "iterations": []})
        d["requests"] += 1
        d["rhs"] += len(r["stats"])
        d["latency_s"].append(round(r["latency"], 2))
        d["residual_max"] = max([d["residual_max"]] + [s["residual"] for s in r["stats"]])
        d["iterations"] += [s["iterations"] for s in r["stats"]]
    for lt in reqs:
        lt["b"] = lt["x"] = None
    # sequential FP64 plain service time per shape: 20 timed CGNE iterations
    # x the iteration count of a full CGNE solve on the smallest shape
    small = lats[-1]
    pc = m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE)
    b1 = torch.empty((1, small["V"], 12), dtype=torch.complex128, device="cuda")
    m.mglma_sources(ctx, small["L"], m.MGLMA_SOURCE_Z2, 1, 3000 + w["cfg"], b1)
    x1 = torch.zeros_like(b1)
    _, s1 = m.mglma_solve_batch(ctx, small["g"], None, pc, [1], b1, x1, raise_on_error=False)
    full_iters = s1[0]["iterations"]
    seq = {}
    pc.max_iter = 20
    for lt in lats:
        b1 = torch.empty((1, lt["V"], 12), dtype=torch.complex128, device="cuda")
        m.mglma_sources(ctx, lt["L"], m.MGLMA_SOURCE_Z2, 1, 3000 + w["cfg"], b1)
        x1 = torch.zeros_like(b1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.mglma_solve_batch(ctx, lt["g"], None, pc, [1], b1, x1, raise_on_error=False)
        torch.cuda.synchronize()
        t_it = (time.perf_counter() - t0) / 20
        seq["x".join(map(str, lt["L"]))] = {"s_per_iteration": round(t_it, 4),
                                            "solve_s_extrapolated": round(t_it * full_iters, 2)}
        del b1, x1
    shares = [stats["slots"][i] for i in range(len(lats))]
    mean_seq = float(np.mean([seq["x".join(map(str, lats[int(k)]["L"]))]["solve_s_extrapolated"] for k in shape]))
    line = {"workload": "c5", "metric": METRIC, "unit": "solves/s", "value": round(stats["solves_per_s"], 4),
            "p50_s": round(stats["p50_s"], 2), "p99_s": round(stats["p99_s"], 2), "wall_s": round(stats["wall_s"], 1),
            "requests": stats["requests"], "rhs": stats["rhs"], "rejected": stats["rejected"],
            "all_ok": all(r["status"] == 0 for r in res),
            "offered": f"Poisson 20 requests/s (seed 4242), shape uniform, RHS uniform in 1..{args.serve_max_rhs}",
            "slots": dict(zip(["x".join(map(str, lt["L"])) for lt in lats], shares)),
            "slot_gb": [round(b / 1e9, 1) for b in stats["slot_bytes"][:len(lats)]], "per_shape": per_shape,
            "setup": setup, "fp64_plain_sequential": seq, "cgne_iterations_smallest": full_iters,
            "fp64_plain_solves_per_s_extrapolated": round(1.0 / mean_seq, 4) if mean_seq > 0 else None,
            "dtype": "f32 inner / f64 outer / bf16 coarse / fp16 basis", "data": "synthetic (device-generated)"}
    print(json.dumps(line), flush=True)
    for lt in lats:
        m.mglma_coarse_free(lt["C"])
        m.mglma_subspace_free(lt["sub"])
        m.mglma_gauge_free(lt["g"])
    ctx.close()


def micro_dslash(m, torch, ctx, g, V, nrhs, prec, reps, stream):
    """FP32/FP64 stencil on nrhs fields, launch-level timing from the
    library's CUDA events on the launching stream."""
    kind = "dslash32" if prec == m.MGLMA_FP32 else "dslash64"
    x = torch.randn(nrhs, V, 24, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        m.mglma_dirac_apply(ctx, g, 0, nrhs, x, y, prec, stream=stream)
    torch.cuda.synchronize()
    m.mglma_profile(ctx, True, True)
    for _ in range(reps):
        m.mglma_dirac_apply(ctx, g, 0, nrhs, x, y, prec, stream=stream)
    n, ms, by, fl = m.mglma_profile_get(ctx, kind)
    m.mglma_profile(ctx, False, True)
    return {"kernel": kind, "nrhs": nrhs, "launches": n, "avg_launch_ms": ms / n,
            "achieved": round(by / (ms / 1e3) / 1e9, 1), "unit": "GB/s",
            "bytes_per_launch": by / n, "tflops": round(fl / (ms / 1e3) / 1e12, 2)}


def set_tile(m, ctx, args, nrhs):
    """--tile NR,RW fixes the FP32 stencil's tile shape for nrhs RHS."""
    if args.tile.startswith("s"):
        m.mglma_autotune_set(ctx, 0, nrhs, m.dslash32_staged_code(int(args.tile[1:])))
    elif args.tile:
        nr, rw = (int(v) for v in args.tile.split(","))
        m.mglma_autotune_set(ctx, 0, nrhs, m.dslash32_tile_code(nr, rw))


def run_micro(args, w):
    """One kernel class alone on the workload lattice (inputs larger than L2)."""
    import torch
    import paper_2412_06347_gb300 as m
    import synthetic
    hbm, _, _, peak_kind = peaks()
    L = tuple(int(v) for v in args.micro_lattice.split("x")) if args.micro_lattice else w["L"]
    V = int(np.prod(L))
    ctx = m.Context(0)
    # the seeded link recipe, generated on the device
    g = m.mglma_gauge_random(ctx, L, w["eps"], 1000 + w["cfg"], w["kappa"], w["csw"])
    set_tile(m, ctx, args, args.nrhs)
    stream = torch.cuda.current_stream()
    reps = max(args.steps, 1)
    if args.micro in ("dslash32", "dslash64"):
        prec = m.MGLMA_FP32 if args.micro == "dslash32" else m.MGLMA_FP64
        r = micro_dslash(m, torch, ctx, g, V, args.nrhs, prec, reps, stream)
    elif args.micro == "contract":
        # the estimator's time-slice contraction (Eq. C_stoch2): 4 FP64
        # canonical fields per RHS read once
        n = args.nrhs
        a = torch.randn(n, 3, V, 24, dtype=torch.float64, device="cuda")
        b = torch.randn(n, V, 24, dtype=torch.float64, device="cuda")
        out = torch.empty(n, L[0], 2, dtype=torch.float64, device="cuda")
        for _ in range(3):
            m.mglma_contract(ctx, L, n, a, b, out, stream=stream)
        torch.cuda.synchronize()
        m.mglma_profile(ctx, True, True)
        for _ in range(reps):
            m.mglma_contract(ctx, L, n, a, b, out, stream=stream)
        nl, ms, by, fl = m.mglma_profile_get(ctx, "contract")
        m.mglma_profile(ctx, False, True)
        r = {"kernel": "contract", "nrhs": n, "launches": nl, "avg_launch_ms": ms / nl,
             "achieved": round(by / (ms / 1e3) / 1e9, 1), "unit": "GB/s", "bytes_per_launch": by / nl,
             "fp64_tflops": round(fl / (ms / 1e3) / 1e12, 3)}
    else:
        prec = {"fp16": m.MGLMA_FP16, "fp32": m.MGLMA_FP32, "bf16": m.MGLMA_BF16}
        sub = m.mglma_subspace_build(ctx, g, w["block"], w["nv"], 1, 2000 + w["cfg"], prec[w["sub_store"]])
        C = m.mglma_coarse_build(ctx, g, sub, prec[w["coarse_store"]])
        nv, Lb, V1 = m.mglma_coarse_info(C)
        n = args.nrhs
        m.mglma_profile(ctx, True, True)
        if args.micro == "coarse":
            X = torch.randn(n, V1, 2 * nv, dtype=torch.complex128, device="cuda")
            Y = torch.empty_like(X)
            op = {"full": m.MGLMA_OP_D, "schur": m.MGLMA_OP_SCHUR_Q}[args.coarse_op]
            m.mglma_profile(ctx, False, True)
            m.mglma_coarse_apply(ctx, C, n, X, Y, m.MGLMA_FP32, op=op, stream=stream)  # even-odd set-up
            torch.cuda.synchronize()
            m.mglma_profile(ctx, True, True)
            for _ in range(reps):
                m.mglma_coarse_apply(ctx, C, n, X, Y, m.MGLMA_FP32, op=op, stream=stream)
            kinds = ["coarse"]
        else:
            f = torch.randn(n, V, 12, dtype=torch.complex128, device="cuda")
            c = torch.empty(n, V1, 2 * nv, dtype=torch.complex128, device="cuda")
            for _ in range(reps):
                m.mglma_restrict(ctx, sub, n, f, c, m.MGLMA_BF16 if args.restrict == "bf16" else m.MGLMA_FP32,
                                 stream=stream)
                m.mglma_prolong(ctx, sub, n, c, f, m.MGLMA_BF16 if args.restrict == "bf16" else m.MGLMA_FP32,
                                stream=stream)
            kinds = ["restrict", "prolong"]
        r = {}
        for k in kinds:
            nl, ms, by, fl = m.mglma_profile_get(ctx, k)
            r[k] = {"launches": nl, "avg_launch_ms": ms / nl, "achieved": round(by / (ms / 1e3) / 1e9, 1),
                    "unit": "GB/s", "frac": round(by / (ms / 1e3) / 1e9 / hbm, 4),
                    "tflops": round(fl / (ms / 1e3) / 1e12, 2)}
        r = {"kernels": r, "nrhs": n}
        m.mglma_coarse_free(C)
        m.mglma_subspace_free(sub)
    if "achieved" in r:
        r["frac"] = round(r["achieved"] / hbm, 4)
    r.update({"micro": args.micro, "workload": args.workload, "tile": args.tile or "default", "lattice": "x".join(map(str, L)), "peak": hbm,
              "peak_source": f"{peak_kind} hbm_gbs"})
    print(json.dumps(r), flush=True)
    m.mglma_gauge_free(g)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mglma", choices=["mglma", "reference"])
    ap.add_argument("--workload", default="c4", choices=sorted(WORKLOADS) + ["c5"],
                    help="c4: 64x32^3 solves (default); c2: 32x16^3 single-RHS; c5: serving stream over the "
                         "64x32^3, 96x48^3 and 128x64^3 lattices")
    ap.add_argument("--serve-hbm", type=float, default=0.9, help="c5: share of free HBM the serving slots take")
    ap.add_argument("--group", type=int, default=0, help="sources per step (default: the workload's)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--coarse-solver", default="minres_eo", choices=sorted(COARSE_SOLVERS),
                    help="coarse solver inside the preconditioner")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain-solver sample")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the solve's kernels one by one instead of as captured CUDA graphs")
    ap.add_argument("--micro", default="", choices=["", "dslash32", "dslash64", "coarse", "transfer", "contract"],
                    help="time one kernel class on the workload lattice instead of the solve")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides per launch in --micro mode")
    ap.add_argument("--restrict", default="fp32", choices=["fp32", "bf16"],
                    help="--micro transfer: R0 and T0 on CUDA cores (FP32) or on the tensor cores (BF16 operands)")
    ap.add_argument("--coarse-op", default="full", choices=["full", "schur"],
                    help="--micro coarse: the full coarse operator or g5hat S_ee (three tensor-core launches)")
    ap.add_argument("--tile", default="", help="FP32 stencil tile NR,RW (RHS per thread, RHS tiles per CTA) or sNRT "
                                                "(staged-tile kernel, 32 sites x NRT RHS per CTA, NRT 4, 8, 16); "
                                                "default: the library's choice")
    ap.add_argument("--micro-lattice", default="", help="lattice of --micro mode, e.g. 32x32x32x16 (default: the workload's)")
    ap.add_argument("--serve-requests", type=int, default=40,
                    help="requests of the seeded Poisson stream served after the timed solves (0: skip)")
    ap.add_argument("--serve-max-rhs", type=int, default=32, help="RHS per request drawn uniformly in 1..this")
    ap.add_argument("--prof-steps", type=int, default=2, help="profiled steps after the timed region")
    ap.add_argument("--e2e-steps", type=int, default=6, help="steps of the end-to-end (host buffer) measurement")
    ap.add_argument("--cg-batch-iters", type=int, default=40,
                    help="FP64 CGNE iterations timed on the step's batch (like-for-like plain baseline)")
    args = ap.parse_args()
    if args.workload == "c5":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "c5 has no oracle arm: the oracle cannot hold "
                                                                  "128x64^3 fields within a bounded sample"}))
            return
        run_c5(args)
        return
    w = dict(WORKLOADS[args.workload])
    if args.group:
        w["group"] = args.group
    if args.impl == "reference":
        run_reference(args, w)
        return
    if args.micro:
        run_micro(args, w)
        return

    import torch
    import paper_2412_06347_gb300 as m
    import synthetic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm, _, _, peak_kind = peaks()

    prec = {"fp16": m.MGLMA_FP16, "fp32": m.MGLMA_FP32, "fp64": m.MGLMA_FP64, "bf16": m.MGLMA_BF16}
    L = w["L"]
    V = int(np.prod(L))
    G = w["group"]
    ctx = m.Context(local)
    # the seeded link recipe, generated on the device
    g = m.mglma_gauge_random(ctx, L, w["eps"], 1000 + w["cfg"], w["kappa"], w["csw"])
    sub = m.mglma_subspace_create(ctx, g, w["block"], w["nv"], w["n_smooth"], 2000 + w["cfg"], prec[w["sub_store"]],
                                  n_cg=w["n_cg"], cg_prec=m.MGLMA_FP32)
    C = m.mglma_coarse_build(ctx, g, sub, prec[w["coarse_store"]])
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG, coarse_solver=COARSE_SOLVERS[args.coarse_solver])
    if args.no_graph:
        prm.graph = 0
    stream = torch.cuda.Stream(device=dev)
    set_tile(m, ctx, args, G)

    nsteps = args.warmup + args.steps
    # The workload's sources, resident in HBM for the whole run: n_sources /
    # G groups of G (96 / 16 = 6 at 64x32^3, 6.4 GB each); step i solves group
    # i mod ngroups.  Every rank solves its own sources (replicas).
    ngroups = max(1, w["n_sources"] // G)
    base = replica_source_base(rank, G, ngroups)
    src_all = torch.empty((ngroups * G, V, 12), dtype=torch.complex128, device=dev)
    make_sources(m, ctx, w, base, ngroups * G, src_all, stream=stream)
    dev_b = [src_all[i * G:(i + 1) * G] for i in range(ngroups)]
    dev_x = torch.zeros_like(dev_b[0])
    torch.cuda.synchronize()

    def step(i, b, x):
        st, stats = m.mglma_solve_batch(ctx, g, C, prm, [G], b, x, stream=stream, raise_on_error=False)
        if st not in (0, 5):
            raise m.MglmaError(st, m.mglma_last_error())
        return stats

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i, dev_b[i % ngroups], dev_x)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # ---- timed region: sources resident in HBM, per-launch profiling off
    clocks = Clocks(local)
    clocks.start()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    all_stats = []
    torch.cuda.synchronize()
    t_start.record(stream)
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.warmup, nsteps):
        all_stats += step(i, dev_b[i % ngroups], dev_x)
    torch.cuda.nvtx.range_pop()
    t_end.record(stream)
    torch.cuda.synchronize()
    ms = t_start.elapsed_time(t_end)
    clk = clocks.stop()
    ms = max_over_ranks(dist, ms)
    value = job_throughput(G, args.steps, world, ms / 1e3)
    resid = max(s["residual"] for s in all_stats)
    iters = [s["iterations"] for s in all_stats]
    citers = [s["coarse_iterations"] for s in all_stats]
    batch = sorted({s["batch"] for s in all_stats})

    # ---- profiled pass (after the timed region): per-launch CUDA events on
    # the launching stream give the kernel classes' times and algorithmic
    # bytes; one step with profiling on first, so the profiled coarse graphs
    # are captured before the measured steps
    m.mglma_profile(ctx, True, True)
    with torch.cuda.stream(stream):
        step(0, dev_b[0], dev_x)
    torch.cuda.synchronize()
    m.mglma_profile(ctx, True, True)
    p_start, p_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p_start.record(stream)
    for i in range(args.prof_steps):
        step(i, dev_b[(i + 1) % ngroups], dev_x)
    p_end.record(stream)
    torch.cuda.synchronize()
    prof_ms = p_start.elapsed_time(p_end)
    prof = profile_snapshot(m, ctx)
    m.mglma_profile(ctx, False, True)

    # ---- end to end: pinned host buffers, copies inside the timed region
    # (each step's sources are placed in the pinned buffer before its timing)
    e2e_steps = min(args.steps, args.e2e_steps)
    pin_b = torch.empty((G, V, 12), dtype=torch.complex128).pin_memory()
    pin_x = torch.empty_like(pin_b).pin_memory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_s = 0.0
    for i in range(e2e_steps):
        pin_b.copy_(dev_b[i % ngroups].cpu())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(0, pin_b, pin_x)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(dist, e2e_s)
    e2e = {"value": job_throughput(G, e2e_steps, world, e2e_s), "unit": "solves/s", "h2d_bytes_per_step": G * V * 24 * 8,
           "d2h_bytes_per_step": G * V * 24 * 8, "steps": e2e_steps}
    del pin_b, pin_x

    # ---- roofline of the dominant kernel class (profiled pass)
    top = max(((k, v) for k, v in prof.items() if k != "setup"), key=lambda kv: kv[1][1])
    kname, (kl, kms, kbytes, kflops) = top
    achieved = kbytes / (kms / 1e3) / 1e9
    share = {k: round(v[1] / prof_ms, 4) for k, v in prof.items() if v[0]}
    dsl = prof.get("dslash32", (0, 0, 0, 0))
    tps = NCU_TRAFFIC_PER_SITE.get((kname, batch[-1]))
    roofline = {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": round(tps * V) if tps else None,
                "bytes_per_launch": round(kbytes / max(kl, 1)),
                "peak_source": f"{peak_kind} hbm_gbs", "launches": kl, "avg_launch_ms": kms / max(kl, 1),
                "measured": f"CUDA events on the launching stream, {args.prof_steps} profiled steps after the timed region",
                "time_share": share,
                "dslash32": {"achieved": round(dsl[2] / (dsl[1] / 1e3) / 1e9, 1) if dsl[1] else None,
                             "frac": round(dsl[2] / (dsl[1] / 1e3) / 1e9 / hbm, 4) if dsl[1] else None,
                             "launches": dsl[0], "bytes_per_launch": round(dsl[2] / max(dsl[0], 1))}}
    # launches of the library's kernels in the timed region, from the
    # profiled steps' count per step: every class is one launch per record
    # except the tensor-core coarse apply, which writes the B image of X in a
    # first kernel
    per_step = (sum(v[0] for v in prof.values()) + prof.get("coarse", (0,))[0]) / max(args.prof_steps, 1)
    launches = int(round(per_step * args.steps))

    # ---- the stencil alone at N = 1 and N = G (the "dslash GB/s vs HBM peak" part of the metric)
    dslash = {}
    if rank == 0:
        for n in (1, G):
            r = micro_dslash(m, torch, ctx, g, V, n, m.MGLMA_FP32, 20, stream)
            r["frac"] = round(r["achieved"] / hbm, 4)
            dslash[f"nrhs{n}"] = r

    # ---- serving: a bounded prefix of the seeded Poisson request stream
    serving = None
    if args.serve_requests > 0 and rank == 0:
        serving = run_serving(m, torch, ctx, g, C, w, args, dev, src_all)

    # ---- plain FP64 solver on the GPU: one full solve of the first source,
    # and the same G-RHS batch as a step for a bounded number of iterations
    fp64 = None
    cg_iters = 720 if args.workload == "c4" else 460
    if not args.no_fp64 and rank == 0:
        pc = m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE)
        b1 = dev_b[0][:1].contiguous()
        x1 = torch.zeros_like(b1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, s1 = m.mglma_solve_batch(ctx, g, None, pc, [1], b1, x1, stream=stream, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t1 = e0.elapsed_time(e1) / 1e3
        cg_iters = s1[0]["iterations"]
        del b1, x1
        # like for like: FP64 CGNE on the step's G-RHS batch, cg_batch_iters
        # iterations timed, extrapolated to the full solve's iteration count
        pb = m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE, max_iter=args.cg_batch_iters,
                                          check_every=args.cg_batch_iters)
        xb = torch.zeros_like(dev_b[0])
        torch.cuda.synchronize()
        e0.record(stream)
        m.mglma_solve_batch(ctx, g, None, pb, [G], dev_b[0], xb, stream=stream, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) / 1e3
        del xb
        per_it = tb / args.cg_batch_iters
        # the plain method on the even-odd preconditioned operator, full solve
        b1 = dev_b[0][:1].contiguous()
        x1 = torch.zeros_like(b1)
        pe = m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE_EO)
        torch.cuda.synchronize()
        e0.record(stream)
        st, se = m.mglma_solve_batch(ctx, g, None, pe, [1], b1, x1, stream=stream, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        teo = e0.elapsed_time(e1) / 1e3
        del b1, x1
        fp64 = {"value": 1.0 / t1, "unit": "solves/s", "iterations": cg_iters, "residual": s1[0]["residual"],
                "sample": "first source of the workload, FP64 CG on the normal equations, full solve",
                "even_odd": {"value": 1.0 / teo, "unit": "solves/s", "iterations": se[0]["iterations"],
                             "residual": se[0]["residual"],
                             "sample": "first source, FP64 CG on the even-odd Schur system, full solve"},
                "batch": {"value": G / (per_it * cg_iters), "unit": "solves/s", "rhs": G,
                          "s_per_iteration": round(per_it, 4),
                          "sample": f"FP64 CGNE on the step's {G}-RHS batch: {args.cg_batch_iters} iterations timed "
                                    f"(CUDA events), extrapolated to the {cg_iters} iterations of the full solve"}}
    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline(w, cg_iters)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer / bf16 coarse",
            "data": "synthetic (seeded SU(3) links, point + Z2 sources generated on the device)",
            "config": {"workload": args.workload, "lattice": "x".join(map(str, L)), "eps": w["eps"],
                       "kappa": w["kappa"], "csw": w["csw"], "block": "x".join(map(str, w["block"])),
                       "Nv": w["nv"], "basis": w["sub_store"], "coarse_operator": w["coarse_store"],
                       "coarse_solver": args.coarse_solver,
                       "launch": "one by one" if args.no_graph else "CUDA graph per FGCR iteration",
                       "setup": f"{w['n_smooth']} MR + {w['n_cg']} CG relaxation steps",
                       "rhs_per_step": G, "global_batch": G * world, "tol": 1e-10,
                       "l2": "inputs larger than L2 (each source 0.4 GB)", "parallelism": f"replicas x{world}",
                       "sources_resident": f"{ngroups * G} ({ngroups} groups of {G}; step i solves group i mod {ngroups})"},
            "residual_max": resid, "fgcr_iterations": [min(iters), max(iters)],
            "coarse_iterations": [min(citers), max(citers)], "lockstep_batch": batch,
            "e2e": e2e, "roofline": roofline, "dslash_fp32": dslash, "gpu_launches": launches, "clocks": clk,
            "serving": serving,
            "fp64_plain": fp64,
            "speedup_vs_fp64": (value / world / fp64["value"]) if fp64 else None,
            "speedup_vs_fp64_batch": (value / world / fp64["batch"]["value"]) if fp64 else None,
            "speedup_vs_fp64_even_odd": (value / world / fp64["even_odd"]["value"]) if fp64 else None,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
