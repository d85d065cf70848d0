#!/usr/bin/env python
"""Benchmark: Jacobian transforms/s of the SCCSD hot path at o=21, v=200, J=663.

One step = one Davidson-style batch of right Jacobian transformations
sigma_k = A R_k (k = 1..nvec, nvec = 6) at a fixed ground state, through the
C ABI with device-resident inputs. The mixed-precision path (tensor-core
contractions) is the headline value; the FP64 GPU path is timed on the same
inputs as the comparison arm, and their outputs are compared.

`--impl reference` times the FP64 CPU oracle instead (the reference arm of
this project), on a bounded sample: one transformation of the o=10, v=90,
J=300 system per step, scaled to the o=21, v=200 workload by the ratio of the
dense flop counts of one transformation.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2403_01007_gb300 import synthetic as syn  # noqa: E402

METRIC = "Jacobian transforms/s (A R, 6-vector batch), o=21 v=200 J=663"
# The headline arm is BF16 (FP32 accumulation); the spec design makes
# it accurate by FP64 refinement in the solvers, not per transform.


def transform_flops(o, v):
    """Dense flops of one right transformation: the o^2 v^4 ladder plus the
    o^3 v^3 ring contractions (12 of them in the differentiated residual)."""
    return 2.0 * o * o * v ** 4 + 12 * 2.0 * (o * v) ** 3


def ladder_flops_dense(o, v):
    """Flops of the particle-particle ladder contraction per trial vector as
    the tensor-core kernel executes it (dense over ij and ab, cd): 2 o^2 v^4."""
    return 2.0 * o * o * v ** 4


def ladder_flops_packed(o, v):
    """Flops of the same contraction per trial vector in its minimal form: the
    amplitudes split into parts symmetric and antisymmetric under (c <-> d)
    (and correspondingly (i <-> j), (a <-> b)), each contracted over unique
    pairs only: 2 [P_o P_v^2 + o(o-1)/2 (v(v-1)/2)^2], P_x = x(x+1)/2."""
    Po, Pv = o * (o + 1) / 2, v * (v + 1) / 2
    return 2.0 * (Po * Pv ** 2 + o * (o - 1) / 2 * (v * (v - 1) / 2) ** 2)


def ladder_flops_algorithmic(o, v, J, nvec):
    """Algorithmic flops of one ladder call of nvec vectors (scope table): the
    (ac) <-> (bd) symmetric build v^2 (v^2 + 1) / 2 . 2J plus the packed
    contraction per vector."""
    vv = v * v
    return vv * (vv + 1) / 2 * 2.0 * J + nvec * ladder_flops_packed(o, v)


def ladder_flops_executed(o, v, J, nvec, precision):
    """Flops the tensor-core kernels execute for one ladder call: the build
    runs one 128-row MMA tile per half (two halves when v > 128) of N = v
    rounded up to 16 over J rounded up to 64, for every pair a <= b, with 1 or 3
    slice products; the contraction runs 128 x 256 tiles over K = v(v+1)/2
    rounded up to 64, for the + rows (nvec o(o+1)/2) and the - rows
    (nvec o(o-1)/2), with 1 or 3 slice products."""
    import math
    prod = 3 if precision == "bf16x3" else 1
    Pv = v * (v + 1) // 2
    halves = 2 if v > 128 else 1
    nb = 16 * math.ceil(v / 16)
    jp = 64 * math.ceil(J / 64)
    build = Pv * halves * 128 * nb * jp * 2.0 * prod
    kp = 64 * math.ceil(Pv / 64)
    npl, nmi = nvec * o * (o + 1) // 2, nvec * o * (o - 1) // 2
    rows = 128 * (math.ceil(npl / 128) + math.ceil(nmi / 128))
    contract = rows * 256 * math.ceil(Pv / 256) * kp * 2.0 * prod
    return build + contract


# DRAM bytes of one o=21 v=200 6-vector BF16 ladder call: the sum over its
# launches (build, contractions, packing) of dram__bytes_read.sum +
# dram__bytes_write.sum from the ncu capture summarised in
# profiles/ladder_o21_v200_bf16.md; None until that capture matches the kernels
LADDER_TRAFFIC_O21_V200 = None


def ladder_traffic(w, args):
    if (w.o, w.v, w.J) == (21, 200, 663) and args.nvec == 6 and args.precision == "bf16":
        return LADDER_TRAFFIC_O21_V200
    return None


def fp64_peak(torch):
    """Measured FP64 GEMM rate of this GPU (cuBLAS DGEMM 8192^3, best of 3):
    the ceiling of the FP64 path, whose contractions run on the CUDA cores."""
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12, "cuBLAS DGEMM 8192^3 measured in this run (best of 3)"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        # the sampler takes a moment to start: wait (at most 5 s) for its
        # first line so that the timed region is inside the sampled window
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < 5.0:
            if self.proc.poll() is not None or os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_env():
    from paper_2403_01007_gb300 import replicas
    return replicas.rank_env()


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


# host memory the oracle's o=21 v=200 transformation needs (peak RSS measured
# at 56 GB: the full vvvv integrals, their tangent and the einsum temporaries)
ORACLE_LARGE_GB = 70.0


def cpu_oracle_sample():
    """Time the FP64 CPU oracle (as it stands, all host threads) on one right
    transformation A R of the benchmark's workload, o=21 v=200 J=663; return
    (transforms/s, seconds, threads, sample text). If the host lacks the memory
    for it, one transformation of o=10 v=90 J=300 is timed instead and scaled
    by the dense-flop ratio, and the text says so."""
    import torch
    from oracle import ccsd as cc
    from oracle import response as rp
    big = (_mem_available_gb() >= ORACLE_LARGE_GB
           and os.environ.get("SCCSD_ORACLE_SAMPLE", "") != "small")
    w = syn.LARGE if big else syn.MEDIUM
    eps, L = syn.workload_system(w)
    prob = cc.Problem(eps, L, w.o)
    t = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 50), scale=1e-3)[0]
    R = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 60), normalise=True)[0]
    t0 = time.perf_counter()
    rp.jacobian_right(prob, t, R)
    sec = time.perf_counter() - t0
    threads = torch.get_num_threads()
    if big:
        return 1.0 / sec, sec, threads, (
            f"one A R of the FP64 CPU oracle at o=21 v=200 J=663 ({sec:.1f} s, {threads} threads)")
    ratio = transform_flops(syn.LARGE.o, syn.LARGE.v) / transform_flops(w.o, w.v)
    return 1.0 / (sec * ratio), sec, threads, (
        f"host memory below {ORACLE_LARGE_GB:.0f} GB: one A R of the FP64 CPU oracle at o=10 v=90 "
        f"J=300 ({sec:.2f} s, {threads} threads), scaled by the dense-flop ratio to o=21 v=200")


def run_reference(args):
    """The reference arm: the FP64 CPU oracle timed on the host cores. One step
    is one oracle transformation of the o=21 v=200 workload (a few minutes on
    16 cores), so a single step is timed whatever --steps says."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    t0 = time.perf_counter()
    val, sec, threads, sample = cpu_oracle_sample()
    wall = time.perf_counter() - t0
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "transforms/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "timed_steps": 1,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": syn.LARGE.name, "o": syn.LARGE.o, "v": syn.LARGE.v,
                   "J": syn.LARGE.J, "nvec": 1, "precision": "fp64",
                   "parallelism": "replicas1",
                   "l2": "inputs larger than L2 (the vvvv integrals alone are 12.8 GB)"},
        "cpu_baseline": {"value": val, "unit": "transforms/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "transforms/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line))
    return 0


def time_batches(ctx, R, sig, steps, stream, torch):
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(steps):
        ctx.jacobian_right(R, sigma=sig)
    s1.record(stream)
    torch.cuda.synchronize()
    return s0.elapsed_time(s1)


def kernel_case(args):
    """The particle-particle ladder as a bare contraction C = X G^T with
    X [nvec*o^2][V^2] and G [V^2][V^2] (random data), on the tensor cores."""
    import torch
    from paper_2403_01007_gb300 import binding as B
    o, V = syn.LARGE.o, args.kernel_case
    M, N, K = args.nvec * o * o, V * V, V * V
    if args.gemm:
        M, N, K = args.gemm
    g = torch.Generator(device="cuda").manual_seed(1)
    X = torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g)
    G = torch.randn(N, K, dtype=torch.float64, device="cuda", generator=g)
    C = torch.empty(M, N, dtype=torch.float64, device="cuda")
    prec = "bf16" if args.precision == "fp64" else args.precision
    for _ in range(args.warmup):
        B.gemm_tn(X, G, C, precision=prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        B.gemm_tn(X, G, C, precision=prec)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / max(1, args.steps)
    print(json.dumps({"kernel_case": "gemm" if args.gemm else "ladder", "M": M, "N": N, "K": K,
                      "precision": prec, "ms_per_call_incl_conversion": sec * 1e3,
                      "tflops_incl_conversion": 2.0 * M * N * K / sec / 1e12}))
    return 0


def batched_case(args):
    """64 uneven instances (o in [4,12], v in [30,110], J = 3(o+v), 2-5 states
    each): one batch of right transformations per instance and step, either as
    per-instance calls or as one launch of the joined CUDA graph. Under
    torchrun the instances are dealt round-robin to the ranks (no data-path
    collective); times are the slowest rank's and the rate counts all."""
    import torch
    import torch.distributed as dist
    from paper_2403_01007_gb300 import binding as B
    from paper_2403_01007_gb300 import replicas
    rank, world, local = replicas.rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    inst = syn.batch_instances()
    mine = replicas.shard(inst, rank, world)
    items = []
    t_setup = time.perf_counter()
    for x in mine:
        eps, L = syn.system(x.o, x.v, x.J, x.sd, x.seed)
        st = torch.cuda.Stream(device=dev)
        ctx = B.Context(x.o, x.v, x.J, eps, L, precision=args.precision, stream=st.cuda_stream)
        t = syn.random_vectors(x.o, x.v, 1, x.seed + 1000, scale=1e-2)[0]
        ctx.residual(t)
        R = torch.tensor(syn.random_vectors(x.o, x.v, x.nstates, x.seed + 2000, normalise=True),
                         device=dev)
        items.append((ctx, R, torch.empty_like(R), torch.empty_like(R)))
    setup_s = replicas.max_over_ranks(time.perf_counter() - t_setup, device=dev)
    ntr = sum(x.nstates for x in inst)            # all ranks together
    flops = sum(x.nstates * transform_flops(x.o, x.v) for x in inst)

    def per_instance():
        for ctx, R, W, _ in items:
            ctx.jacobian_right(R, sigma=W)

    def measure():
        """(per-instance s/step, graph s/step, graph-vs-calls difference, clocks)"""
        for _ in range(args.warmup):
            per_instance()
        torch.cuda.synchronize()
        replicas.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            per_instance()
        torch.cuda.synchronize()
        per_s = replicas.max_over_ranks((time.perf_counter() - t0) / args.steps, device=dev)
        graphs = [ctx.capture_transform(R, Wg) for ctx, R, _, Wg in items]
        batch = B.GraphBatch(graphs)
        st = torch.cuda.Stream(device=dev)
        for _ in range(args.warmup):
            batch.launch(st.cuda_stream)
        torch.cuda.synchronize()
        replicas.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            e0.record(st)
            for _ in range(args.steps):
                batch.launch(st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
        g_s = replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3 / args.steps, device=dev)
        rel = replicas.max_over_ranks(
            max(float((Wg - W).abs().max() / W.abs().max()) for _, _, W, Wg in items), device=dev)
        batch.close()
        return per_s, g_s, rel, clk.summary()

    per_s, g_s, rel, clocks = measure()
    tuned = None
    if args.autotune:
        # one uncaptured pass with tuning on records the fastest launch shape
        # of every contraction shape; the graphs captured afterwards use them
        default = (per_s, g_s)
        B.autotune_clear()
        for ctx, *_ in items:
            ctx.set_autotune(True)
        t0 = time.perf_counter()
        per_instance()
        torch.cuda.synchronize()
        tune_s = replicas.max_over_ranks(time.perf_counter() - t0, device=dev)
        for ctx, *_ in items:
            ctx.set_autotune(False)
        per_s, g_s, rel, clocks = measure()
        tuned = {"entries": B.autotune_entries(), "tune_s": tune_s,
                 "default_rule": {"graph_transforms_per_s": ntr / default[1],
                                  "calls_transforms_per_s": ntr / default[0]},
                 "tuned": {"graph_transforms_per_s": ntr / g_s,
                           "calls_transforms_per_s": ntr / per_s}}
    for ctx, *_ in items:
        ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    print(json.dumps({
        "metric": "Jacobian transforms/s, 64 uneven instances (o 4-12, v 30-110, 2-5 states)",
        "value": ntr / g_s, "unit": "transforms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": g_s * 1e3, "higher_is_better": True,
        "dtype": {"bf16x3": "bf16x3->f32->f64", "bf16": "bf16->f32->f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "batch64_o4-12_v30-110", "instances": len(inst), "transforms": ntr,
                   "precision": args.precision, "form": "one launch of the joined CUDA graph",
                   "launch_shapes": "tuned" if args.autotune else "fixed rule",
                   "parallelism": f"instances dealt round-robin to {world} rank(s)"},
        "scaling": "strong",
        "per_instance_calls": {"transforms_per_s": ntr / per_s, "ms_per_step": per_s * 1e3},
        "graph_speedup": per_s / g_s,
        "tflops_dense": flops / g_s / 1e12,
        "max_rel_diff_graph_vs_calls": rel,
        "autotune": tuned,
        "setup_s": setup_s, "clocks": clocks}))
    return 0


def row_timings(B, w, eps, L, t, Rh, prec, dev, torch, reps=2):
    """Device time of the other hot-path rows at the same workload and
    precision, on one SCCSD state (zeta = 0.1, X3 from two of the trial
    vectors): the residual (ladder, rings, X3 terms), a 6-vector left
    transformation, the transition densities d_pq and Gamma^J_pq of one
    bra/ket pair, and one application of the multiplier stationarity map
    (three reverse-over-forward state gradients plus the overlap gradient).
    Inputs are synthetic and not converged: the cost does not depend on it."""
    st = torch.cuda.Stream(device=dev)
    ctx = B.Context(w.o, w.v, w.J, torch.tensor(eps, device=dev), torch.tensor(L, device=dev),
                    precision=prec, stream=st.cuda_stream)
    td = torch.tensor(t, device=dev)
    Rd = torch.tensor(Rh, device=dev)
    Ra, Rb = Rd[0].clone(), Rd[1].clone()
    scc = (0.1, Ra, Rb)
    sig = torch.empty_like(Rd)
    n = w.o + w.v
    D1 = torch.empty(n, n, dtype=torch.float64, device=dev)
    G = torch.empty(w.J, n, n, dtype=torch.float64, device=dev)
    vecs = torch.cat([td, Rd[0], Rd[1], Rd[2], Rd[3]]).contiguous()
    scal = np.array([0.1, 0.05, -0.03, 0.4, 0.5])
    u = torch.cat([Rd[4], Rd[5], Rd[0] * 0.1, torch.tensor([0.2], dtype=torch.float64,
                                                           device=dev)]).contiguous()
    r = torch.empty_like(u)
    rows = {
        "residual": lambda: ctx.residual(td, omega=sig[0], scc=scc),
        "left_6": lambda: ctx.jacobian_left(Rd, sigma=sig),
        "densities": lambda: ctx.lib.sccsd_densities(ctx.h, 0.3, Rd[2].data_ptr(), 0.05,
                                                     Rd[0].data_ptr(), D1.data_ptr(),
                                                     G.data_ptr()),
        "multiplier_map": lambda: ctx.lib.sccsd_multiplier_residual(
            ctx.h, vecs.data_ptr(), scal.ctypes.data, 0, 0, 0, u.data_ptr(), r.data_ptr()),
    }
    out = {}
    ctx.residual(td, scc=scc)
    for name, f in rows.items():
        rc = f()
        if isinstance(rc, int) and rc != 0:
            raise RuntimeError(f"{name}: sccsd error {rc}")
        if name != "residual":
            ctx.residual(td, scc=scc)      # keep the SCC state current
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            f()
        e1.record(st)
        torch.cuda.synchronize()
        out[name + "_ms"] = e0.elapsed_time(e1) / reps
    ctx.close()
    out["note"] = ("device time per call at this workload and precision; one SCCSD state; "
                   "the multiplier map is one GMRES operator application")
    return out


def chain_case(args):
    """The whole method on one system (default o=10, v=90, J=300) in the mixed
    precision with FP64 refinement: the SCCSD state (ground state, the two
    lowest states and zeta by the secant loop, then the left vectors), and the
    multipliers plus effective densities of the gradient of state a and of the
    coupling <psi_a|d psi_b>. Each stage is timed on the host around its
    synchronous call (every call ends with a device synchronisation)."""
    import torch
    from paper_2403_01007_gb300 import binding as B
    torch.cuda.set_device(0)
    w = getattr(syn, args.workload if args.workload != "LARGE" else "MEDIUM")
    eps, L = syn.workload_system(w)
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision=args.precision)
    ctx.set_projection(args.projection)
    out = {"metric": "SCCSD gradient and coupling chain, seconds per stage", "unit": "s",
           "higher_is_better": False, "data": "synthetic",
           "config": {"workload": w.name, "o": w.o, "v": w.v, "J": w.J,
                      "precision": args.precision, "refinement": "FP64",
                      "projection": args.projection}}
    t0 = time.perf_counter()
    state = ctx.scc_state(tol=1e-9, ground_tol=1e-10, eom_tol=1e-8, left_tol=1e-7,
                          left_maxit=600)
    out["state_s"] = time.perf_counter() - t0
    out["zeta"] = state["zeta"]
    out["omega"] = [state["omega_a"], state["omega_b"]]
    out["omega_left"] = [float(x) for x in state["omega_left"]]
    out["e_corr"] = state["e_corr"]
    for name, target in [("gradient_a", ("gradient", 0)), ("coupling_ab", ("coupling", 0, 1))]:
        t1 = time.perf_counter()
        r = ctx.solve_multipliers(state, target, tol=1e-8, maxit=1500, refine_tol=1e-6)
        out[name] = {"seconds": time.perf_counter() - t1, "map_applications": r["iterations"],
                     "gbar": float(r["gbar"]), "trace_D1": float(np.trace(r["D1"])),
                     "norm_Gamma": float(np.linalg.norm(r["Gamma"]))}
    out["value"] = time.perf_counter() - t0
    ctx.close()
    print(json.dumps(out))
    return 0


def solve_case(args):
    """Converged solves at o=21 v=200 J=663 (or --workload): the ground state
    (|Omega|_2 < solve_tol) and the lowest --nstates right EOM roots
    (|A R - omega R| < state_tol), once in the mixed precision with FP64
    refinement (defect correction of the amplitudes, FP64 anchors of the
    Davidson subspace) and once in plain FP64, on the same inputs. Reports the
    wall time of each arm (host clock around the synchronous calls), the
    iteration and FP64-evaluation counts, and the differences of E_corr and of
    every omega between the arms."""
    import torch
    from paper_2403_01007_gb300 import binding as B
    torch.cuda.set_device(0)
    w = getattr(syn, args.workload)
    eps, L = syn.workload_system(w)
    dev = torch.device("cuda", 0)
    arms = [args.precision] + ([] if args.no_fp64_arm or args.precision == "fp64" else ["fp64"])
    out = {}
    for prec in arms:
        logf = tempfile.TemporaryFile(mode="w+")
        saved = os.dup(2)
        os.dup2(logf.fileno(), 2)
        os.environ["SCCSD_LOG"] = "1"
        try:
            ctx = B.Context(w.o, w.v, w.J, torch.tensor(eps, device=dev),
                            torch.tensor(L, device=dev), precision=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e, _, itg = ctx.solve_ground(tol=args.solve_tol, maxit=args.solve_maxit,
                                         refine_tol=0.0 if prec == "fp64" else 1e-5)
            t1 = time.perf_counter()
            wk, _, its = ctx.solve_states(args.nstates, "right", tol=args.state_tol,
                                          maxit=args.solve_maxit,
                                          refine_tol=0.0 if prec == "fp64" else 1e-4, vecs=False)
            t2 = time.perf_counter()
            ctx.close()
        finally:
            os.environ.pop("SCCSD_LOG", None)
            sys.stderr.flush()
            os.dup2(saved, 2)
            os.close(saved)
        logf.seek(0)
        if args.solve_log:
            with open(f"{args.solve_log}.{prec}", "w") as fo:
                fo.write(logf.read())
            logf.seek(0)
        done = {}
        for line in logf:
            if line.startswith("{") and ("_done" in line):
                try:
                    d = json.loads(line)
                    done[d["solver"]] = d
                except ValueError:
                    pass
        logf.close()
        out[prec] = {"e_corr": e, "omega": [float(x) for x in wk], "ground_iterations": itg,
                     "davidson_iterations": its, "ground_s": t1 - t0, "states_s": t2 - t1,
                     "total_s": t2 - t0, "ground_refinement": done.get("ground_done"),
                     "davidson_refinement": done.get("davidson_done")}
    mixed = out[args.precision]
    line = {"metric": f"time to converged ground state and {args.nstates} right roots, "
                      f"{w.name}: mixed vs FP64 GPU",
            "value": mixed["total_s"], "unit": "s", "higher_is_better": False,
            "data": "synthetic",
            "config": {"workload": w.name, "o": w.o, "v": w.v, "J": w.J, "nstates": args.nstates,
                       "precision": args.precision, "ground_tol": args.solve_tol,
                       "state_tol": args.state_tol, "refinement": "FP64 residuals"},
            "arms": out}
    if "fp64" in out and args.precision != "fp64":
        ref = out["fp64"]
        line["fp64_total_s"] = ref["total_s"]
        line["time_to_solution_speedup"] = ref["total_s"] / mixed["total_s"]
        line["abs_diff_e_corr"] = abs(mixed["e_corr"] - ref["e_corr"])
        line["max_abs_diff_omega"] = max(abs(a - b) for a, b in zip(mixed["omega"], ref["omega"]))
    print(json.dumps(line))
    return 0


def learned_case(args):
    """Learned guess and preconditioner, reduced form of the C5 workload: train
    on solver-generated amplitudes of n_train systems at o=8, v=60, then solve
    n_eval fresh systems with o in [8,12], v in [60,110] to 1e-8 with the plain
    MP2 start and with the network's proposal (the plain solver's result is
    kept in both cases; the proposal is used only if it starts closer)."""
    import torch
    from paper_2403_01007_gb300 import binding as B
    from paper_2403_01007_gb300 import learned as lrn
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    train_sys = [lrn.system(8, 60, k) for k in range(args.n_train)]
    X, Y = lrn.generate(train_sys, samples_per_instance=20000, tol=args.gen_tol)
    gen_s = time.perf_counter() - t0
    net = B.Mlp(seed=11)
    t1 = time.perf_counter()
    hist = lrn.train(net, X, Y, epochs=20, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    rng = np.random.Generator(np.random.PCG64(syn.seed_of(lrn.LEARN_CONFIG, 999)))
    evs = []
    for k in range(args.n_eval):
        o = int(rng.integers(8, 13))
        v = int(rng.integers(60, 111))
        evs.append(lrn.system(o, v, 1000 + k))
    rows = lrn.evaluate(net, evs, tol=1e-8)
    # the network's own throughput: forward over every doubles amplitude of an
    # o=8 v=60 system (230 400 rows), and one training step on 65 536 rows
    nrow = 8 * 8 * 60 * 60
    Xf = X[:nrow].contiguous() if X.shape[0] >= nrow else X.repeat(nrow // X.shape[0] + 1, 1)[:nrow]
    Yf = torch.empty((nrow, lrn.N_TARGETS), dtype=torch.float32, device=X.device)
    for _ in range(3):
        net.forward(Xf, Yf)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(10):
        net.forward(Xf, Yf)
    ev1.record()
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(ev1) / 10
    fwd_flops = 2.0 * nrow * (lrn.N_FEATURES * 256 + 2 * 256 * 256 + 256 * lrn.N_TARGETS)
    nb = min(65536, X.shape[0])
    Xb, Yb = X[:nb].contiguous(), Y[:nb].contiguous()
    net.train_step(Xb, Yb, 1e-6)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    for _ in range(10):
        net.train_step(Xb, Yb, 1e-6)
    torch.cuda.synchronize()
    step_ms = (time.perf_counter() - t3) * 100.0
    net.close()
    it0 = [r["plain_iters"] for r in rows]
    it1 = [r["learned_iters"] for r in rows]
    s0 = [r["plain_s"] for r in rows]
    s1 = [r["learned_s"] for r in rows]
    print(json.dumps({
        "metric": "ground-state iterations to 1e-8, learned proposal vs MP2 start",
        "value": float(np.mean(it1)), "unit": "iterations", "higher_is_better": False,
        "data": "synthetic", "dtype": "bf16 network, bf16->f32->f64 solver with FP64 refinement",
        "config": {"workload": "learned_o8_v60_train_o8-12_v60-110_eval",
                   "n_train": args.n_train, "n_eval": args.n_eval,
                   "samples_per_train_system": 20000, "epochs": 20,
                   "training_targets_tol": args.gen_tol},
        "plain_iterations_mean": float(np.mean(it0)),
        "learned_iterations_mean": float(np.mean(it1)),
        "iteration_ratio": float(np.mean(it1) / np.mean(it0)),
        "plain_seconds_mean": float(np.mean(s0)), "learned_seconds_mean": float(np.mean(s1)),
        "proposal_used": int(sum(r["used_net"] for r in rows)),
        "max_abs_energy_difference": float(max(abs(r["de"]) for r in rows)),
        "training": {"generate_s": gen_s, "train_s": train_s, "loss_first": hist[0],
                     "loss_last": hist[-1], "rows": int(X.shape[0])},
        "network": {"forward_rows": nrow, "forward_ms": fwd_ms,
                    "forward_tflops": fwd_flops / (fwd_ms * 1e-3) / 1e12,
                    "train_step_rows": nb, "train_step_ms": step_ms,
                    "train_step_tflops": 3.0 * fwd_flops * nb / nrow / (step_ms * 1e-3) / 1e12},
        "rows": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16x3", "bf16", "fp64"])
    ap.add_argument("--nvec", type=int, default=6)
    ap.add_argument("--workload", default="LARGE", choices=["SMALL", "MEDIUM", "LARGE", "LADDER_O4"],
                    help="LADDER_O4: the o=21 v=200 J=663 vvvv build with o=4, for profilers")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--no-x3-arm", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the timings of the other hot-path rows")
    ap.add_argument("--gemm", type=int, nargs=3, metavar=("M", "N", "K"), default=None,
                    help="with --kernel-case: time C[M][N] = X[M][K] G[N][K]^T instead")
    ap.add_argument("--kernel-case", type=int, default=0, metavar="V",
                    help="time only the ladder-shaped contraction (rows = nvec*21^2, "
                         "N = K = V^2) through sccsd_gemm_tn; a small case for profilers")
    ap.add_argument("--chain", action="store_true",
                    help="time the whole method (state, multipliers, densities) at o=10 v=90")
    ap.add_argument("--learned", action="store_true",
                    help="evaluate the learned guess/preconditioner on fresh systems")
    ap.add_argument("--n-train", type=int, default=24)
    ap.add_argument("--n-eval", type=int, default=12)
    ap.add_argument("--solve-log", default=None,
                    help="with --solve: write each arm's solver log to this path + '.<arm>'")
    ap.add_argument("--gen-tol", type=float, default=1e-8,
                    help="residual tolerance of the solves that make the training targets")
    ap.add_argument("--projection", default="natural", choices=["natural", "state"],
                    help="with --chain: the SCC projection, SCCSD(E) or SCCSD(K)")
    ap.add_argument("--autotune", action="store_true",
                    help="tune the launch shapes in the warm-up (with --batched: time the "
                         "fixed rule, then tune and time again)")
    ap.add_argument("--batched", action="store_true",
                    help="64 uneven instances: joined CUDA graph vs per-instance calls")
    ap.add_argument("--solve", action="store_true",
                    help="converged ground state and right roots, mixed (refined) vs FP64")
    ap.add_argument("--nstates", type=int, default=2)
    ap.add_argument("--solve-tol", type=float, default=1e-8)
    ap.add_argument("--state-tol", type=float, default=1e-5)
    ap.add_argument("--solve-maxit", type=int, default=400)
    args = ap.parse_args()
    if args.solve and args.impl == "ours":
        return solve_case(args)
    if args.batched and args.impl == "ours":
        return batched_case(args)
    if args.learned and args.impl == "ours":
        return learned_case(args)
    if args.chain and args.impl == "ours":
        return chain_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_case:
        return kernel_case(args)

    import torch
    import torch.distributed as dist
    from paper_2403_01007_gb300 import binding as B
    from paper_2403_01007_gb300 import replicas

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = getattr(syn, args.workload)
    inst = replicas.instance_of(rank)
    eps, L = syn.workload_system(w, instance=inst)
    dim = B.dim(w.o, w.v)
    t = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 50 + inst), scale=1e-3)[0]
    Rh = syn.random_vectors(w.o, w.v, args.nvec, syn.seed_of(w.config, 60 + inst), normalise=True)

    stream = torch.cuda.Stream(device=dev)
    peaks, peak_src = load_peaks()

    def make_ctx(prec):
        with torch.cuda.stream(stream):
            c = B.Context(w.o, w.v, w.J, torch.tensor(eps, device=dev), torch.tensor(L, device=dev),
                          precision=prec, stream=stream.cuda_stream)
            # with --autotune, launch shapes are tuned by the first (untimed)
            # call of each contraction shape
            c.set_autotune(args.autotune)
            td = torch.tensor(t, device=dev)
            c.residual(td)
        return c

    R = torch.tensor(Rh, device=dev)
    sig = torch.empty_like(R)
    ctx = make_ctx(args.precision)
    for _ in range(args.warmup):
        ctx.jacobian_right(R, sigma=sig)
    replicas.barrier()
    torch.cuda.synchronize()
    tuned_before = B.autotune_entries()
    ctx.profile(True)
    with Clocks(local) as clk:
        ms = time_batches(ctx, R, sig, args.steps, stream, torch)
    lad_ms, lad_calls, lad_flops, launches = ctx.profile_read()
    tuning = {"launch_shapes": "tuned in warm-up" if args.autotune else "fixed rule",
              "table_entries": tuned_before,
              "tuned_in_timed_region": B.autotune_entries() - tuned_before}
    clocks = clk.summary()
    ctx.profile(False)
    ms = replicas.max_over_ranks(ms, device=dev)
    value = replicas.whole_job_rate(args.steps * args.nvec, world, ms)
    sig_mixed = sig.cpu().numpy().copy()

    # end to end: pinned host inputs and outputs through the same public call
    e2e = None
    if not args.no_e2e:
        Rpin = torch.tensor(Rh).pin_memory()
        spin = torch.empty_like(Rpin).pin_memory()
        ctx.jacobian_right(Rpin, sigma=spin)
        torch.cuda.synchronize()
        replicas.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.jacobian_right(Rpin, sigma=spin)
        torch.cuda.synchronize()
        es = replicas.max_over_ranks(time.perf_counter() - t0, device=dev)
        e2e = {"value": replicas.whole_job_rate(args.steps * args.nvec, world, es * 1e3),
               "unit": "transforms/s",
               "h2d_bytes_per_step": int(Rpin.numel() * 8),
               "d2h_bytes_per_step": int(spin.numel() * 8)}
    ctx.close()
    del ctx

    # FP64 GPU arm on the same inputs
    fp64 = None
    if not args.no_fp64_arm and args.precision != "fp64":
        c64 = make_ctx("fp64")
        c64.jacobian_right(R, sigma=sig)       # first call builds the ladder integrals
        ms64 = time_batches(c64, R, sig, args.fp64_steps, stream, torch)
        s64 = sig.cpu().numpy()
        c64.close()
        sig_fp64 = s64
        rel = float(np.abs(sig_mixed - s64).max() / np.abs(s64).max())
        t64 = args.fp64_steps * args.nvec / (ms64 / 1e3)
        p64, p64_src = fp64_peak(torch)
        fp64 = {"transforms_per_s": t64, "ms_per_step": ms64 / args.fp64_steps,
                "warmup": 1, "steps": args.fp64_steps,
                "mixed_speedup": value / world / t64,
                "max_rel_diff_mixed_vs_fp64": rel,
                "fp64_gemm_peak_tflops": p64, "fp64_peak_source": p64_src}

    # the 3-product split arm (BF16x3) on the same inputs
    x3 = None
    if not args.no_x3_arm and args.precision == "bf16":
        cx = make_ctx("bf16x3")
        for _ in range(2):
            cx.jacobian_right(R, sigma=sig)
        msx = time_batches(cx, R, sig, max(1, args.steps), stream, torch)
        sx = sig.cpu().numpy()
        cx.close()
        x3 = {"transforms_per_s": max(1, args.steps) * args.nvec / (msx / 1e3),
              "ms_per_step": msx / max(1, args.steps)}
        if fp64 is not None:
            x3["max_rel_diff_vs_fp64"] = float(np.abs(sx - s64).max() / np.abs(s64).max())

    # the same batch through the SCCSD Jacobian (zeta = 0.1, X3 from two of the
    # trial vectors): A R including the similarity-constraint terms
    scc_arm = None
    if not args.no_rows and args.nvec >= 2:
        cs = make_ctx(args.precision)
        scc = (0.1, R[0].clone(), R[1].clone())
        with torch.cuda.stream(stream):
            cs.residual(torch.tensor(t, device=dev), scc=scc)
        for _ in range(2):
            cs.jacobian_right(R, sigma=sig)
        mss = time_batches(cs, R, sig, max(1, args.steps), stream, torch)
        cs.close()
        scc_arm = {"transforms_per_s": max(1, args.steps) * args.nvec / (mss / 1e3),
                   "ms_per_step": mss / max(1, args.steps), "zeta": 0.1}

    rows = None
    if not args.no_rows and rank == 0 and args.nvec >= 6:
        rows = row_timings(B, w, eps, L, t, Rh, args.precision, dev, torch)

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        val, sec, threads, sample = cpu_oracle_sample()
        cpu = {"value": val, "unit": "transforms/s", "cores": threads, "kind": "oracle",
               "sample": sample}

    # Roofline of the particle-particle ladder, one call = one batch of nvec
    # vectors: the algorithmic flops of the scope table (the (ac) <-> (bd)
    # symmetric build of the integrals from the Cholesky vectors plus the
    # +- packed contraction), over the device time of the whole call (build,
    # contraction, packing) from CUDA events on the context's stream, against
    # the measured BF16 burst peak (the ladder runs for milliseconds inside a
    # step of tens of milliseconds). The executed count (padded tiles, BF16x3
    # slice products) is a secondary key.
    burst = peaks.get("bf16_tflops", 1900.0)
    calls = max(lad_calls, 1)
    lad_call_ms = lad_ms / calls
    alg_call = lad_flops / calls
    exe_call = ladder_flops_executed(w.o, w.v, w.J, args.nvec, args.precision)
    achieved = alg_call / (lad_call_ms / 1e3) / 1e12 if lad_ms > 0 else None
    if args.precision == "fp64":
        p64, p64_src = fp64_peak(torch)
        roof = {"bound": "alu", "achieved": achieved, "peak": p64, "unit": "TFLOP/s",
                "frac": achieved / p64 if achieved and p64 else None, "traffic": None,
                "kernel": "ladder (FP64 build and contraction on the CUDA cores), one call",
                "peak_source": p64_src}
    else:
        roof = {"bound": "tensor", "achieved": achieved, "peak": burst, "unit": "TFLOP/s",
                "frac": achieved / burst if achieved else None,
                "traffic": ladder_traffic(w, args),
                "kernel": "ladder: k_ladder_build + k_tc_gemm contraction + pack/unpack, one call",
                "peak_source": f"bf16 burst, {peak_src}",
                "flops_per_call": {"algorithmic": alg_call, "executed": exe_call},
                "executed_tflops": exe_call / (lad_call_ms / 1e3) / 1e12 if lad_ms > 0 else None,
                "ladder_share_of_step": lad_ms / ms if ms > 0 else None}
    line = {
        "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": "bf16x3->f32->f64", "bf16": "bf16->f32->f64", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": w.name, "o": w.o, "v": w.v, "J": w.J, "nvec": args.nvec,
                   "precision": args.precision, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (ladder integrals alone exceed 129 MB)"},
        "roofline": roof,
        "autotune": tuning,
        "ladder": {"ms_per_call": lad_call_ms, "calls": lad_calls,
                   "tflops_algorithmic": achieved,
                   "tflops_executed": roof.get("executed_tflops")},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "fp64_arm": fp64,
        "bf16x3_arm": x3,
        "sccsd_arm": scc_arm,
        "rows": rows,
        "accuracy": "mixed transforms feed solvers that finish in FP64 (iterative refinement); "
                    "converged energies and roots equal the FP64 path to 1e-8 Eh "
                    "(tests/test_gpu_solvers.py)",
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
