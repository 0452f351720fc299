#!/usr/bin/env python
"""Throughput of the semi-implicit APFC amplitude step on GB300.

Workload: 2D hexagonal APFC (J = 3), 4096 x 4096 periodic grid, h = pi/2,
16 Voronoi grains (rotations uniform in [-10, 10] deg, seed 1), noise 1e-3,
dB = 0.02, Bx = 0.98, t = 0.5, v = 1/3, dt = 1.  Every Krylov solve stops at
relative residual 1e-10 ("fixed residual").  One benchmark step = one time
step of the whole hot path (explicit nonlinear right-hand side, J block solves,
state update).  The state (805 MB in FP64) is larger than L2, so no flush is
needed between steps.

Reported: amplitude DOF-steps/s (DOF = one complex eta_j at one grid point) of
the FP32-Krylov + FP64-refinement path (the headline) and of the plain FP64
path, the roofline of the dominant kernel measured live with CUDA events on
the library's stream, the end-to-end rate through the C ABI with host
buffers, and the FP64 oracle timed on the host cores as a CPU baseline.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "amplitude DOF-steps/s at fixed residual; stencil HBM GB/s vs peak; FP32-refined vs FP64"
UNIT = "DOF-steps/s"
PARAMS = (0.02, 0.98, 0.5, 1.0 / 3.0)  # dB, Bx, t, v
H = np.pi / 2
TOL = 1e-10
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=4096, help="grid points per side")
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--timed-kernel", default="fused_apinv_f32")
    ap.add_argument("--tile", type=int, default=3)
    ap.add_argument("--tile-t", type=int, default=1, help="tile variant of the t-kernel (-1: same as --tile)")
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--cheb", type=int, default=1, help="Chebyshev applications per diffusion solve")
    ap.add_argument("--tol-inner", type=float, default=1e-4, help="relative tolerance of each FP32 inner solve")
    ap.add_argument("--breakdown-steps", type=int, default=3, help="steps of the per-kernel timing pass (0: off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument(
        "--workload", choices=["voronoi", "batch", "adjoint", "bcc3d"], default="voronoi",
        help="voronoi: one n x n polycrystal (default); batch: independent runs of uneven sizes in one batch; "
        "adjoint: gradient of a rollout loss by the checkpointed adjoint",
    )
    ap.add_argument("--picard", type=int, default=1, help="Picard iterations per step (Alg. 1's K)")
    ap.add_argument("--jacobian", action="store_true", help="Picard iterations with the Jacobian in direction eta_j")
    ap.add_argument("--rollout", type=int, default=200, help="adjoint: steps per rollout")
    ap.add_argument("--every", type=int, default=20, help="adjoint: steps between checkpoints")
    ap.add_argument("--adj-size", type=int, default=1024, help="adjoint: grid points per side")
    ap.add_argument("--bcc-size", type=int, default=256, help="bcc3d: grid points per side")
    ap.add_argument("--runs", type=int, default=64, help="batch: number of independent runs")
    ap.add_argument("--no-graph", action="store_true", help="batch: launch the Krylov blocks without graphs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep --tile / --rows (batch) or the automatic segment height (single grid)")
    ap.add_argument("--alone-steps", type=int, default=4, help="batch: steps of each run alone (0: skip)")
    ap.add_argument("--guess", type=int, default=0, help="initial guess: 0 previous state, 1 extrapolated")
    ap.add_argument("--sub-steps", type=int, default=10,
                    help="default run: timed steps of the bcc3d sub-record (0: no sub-records)")
    ap.add_argument("--sub-steps-batch", type=int, default=100,
                    help="default run: timed steps of the batch sub-record (its early steps are the slow ones)")
    ap.add_argument("--oracle-workers", type=int, default=0,
                    help="host processes of the oracle legs (0: one per core, as memory allows)")
    return ap.parse_args()


def workload_config(n, steps_note=None):
    cfg = {
        "workload": f"hex2d-{n}x{n}-voronoi16",
        "lattice": "triangular, J=3",
        "grid": [n, n],
        "h": "pi/2",
        "dt": 1.0,
        "params": {"dB": PARAMS[0], "Bx": PARAMS[1], "t": PARAMS[2], "v": PARAMS[3]},
        "tol": TOL,
        "krylov": "right-preconditioned BiCGStab, Schur-complement preconditioner",
        "cheb_degree": CHEB,
        "tol_inner": TOL_INNER,
        "picard_iters": PICARD[0],
        "jacobian": PICARD[1],
        "l2": "inputs larger than L2 (FP64 state 805 MB per 4096^2 replica); no flush",
    }
    if steps_note:
        cfg["note"] = steps_note
    return cfg


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# FP64-pipe instructions per amplitude value (DOF) of the FP64-accurate kernels of the 2D
# hexagonal FP32-refined step, counted from their source: (FP64 arithmetic, FP64 <-> FP32
# conversions).  Both kernels do their arithmetic in FP32 on doubles split by integer
# operations; only the FP64 outputs cost FP64 additions.
#   residual_refine_f64 (k_resid2d_tma): r64 = f2d(hi) + f2d(lo), 4 per DOF.
#   rhs_f64 (k_rhs_resid_hex): the new right-hand side as a double, 2 per DOF.
FP64_PIPE_OPS = {"residual_refine_f64": (4.0, 0.0), "rhs_f64": (2.0, 0.0)}


def fp64_roofline(name, dof, rec, hbm_peak, alu):
    """Roofline of an FP64 kernel: the larger of its FP64-pipe time (FMA-rate and conversion-rate
    bound of its instruction count) and its HBM time, as a fraction of its measured time."""
    n_ops, n_cvt = FP64_PIPE_OPS[name]
    per_launch_ms = rec["ms"] / rec["launches"]
    alu_ms = 1e3 * dof * (n_ops / (alu["fp64_fma_tflops"] * 1e12 / 2) + n_cvt / (alu["fp64_cvt_tops"] * 1e12))
    hbm_ms = 1e3 * (rec["bytes"] / rec["launches"]) / (hbm_peak * 1e9)
    bound = "alu" if alu_ms >= hbm_ms else "hbm"
    return {"bound": bound, "fp64_ops_per_dof": n_ops, "cvt_per_dof": n_cvt, "alu_bound_ms": alu_ms,
            "hbm_bound_ms": hbm_ms, "ms_per_launch": per_launch_ms, "frac": max(alu_ms, hbm_ms) / per_launch_ms}


def kernel_source_hash(names=("fused2d.cu", "acc.cuh")):
    """Hash of the sources a kernel compiles from (default: the fused 2D pipeline's)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1902_09761_gb300", "csrc")
    for name in names:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, algorithmic_bytes_per_launch):
    """DRAM bytes per launch: the committed ncu ratio of DRAM to algorithmic bytes (taken on
    the current kernel sources) times this run's algorithmic bytes per launch; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("source_hash") != kernel_source_hash(tuple(e.get("sources", ("fused2d.cu", "acc.cuh")))):
            return None
        return float(e["dram_over_algorithmic"]) * float(algorithmic_bytes_per_launch)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    FIELDS = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL,
            )
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.file.name)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


def init_dist(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allmax(world, value, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# Reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------


# Peak resident bytes per grid point of one oracle step (measured on the GPU machine:
# 4.6 GB at 4096^2 hex, 8.5 GB at 256^3 bcc), used to size the host process pool.
ORACLE_BYTES_PER_POINT = {"hex": 300, "bcc": 550}
ORACLE_TIMEOUT_S = 1800


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _mem_available():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except Exception:
        pass
    return None


def oracle_workers(kind, n, requested=0):
    """One oracle process per host core, as many as 60% of the available memory holds."""
    w = requested if requested > 0 else host_cores()
    mem = _mem_available()
    pts = n ** (2 if kind == "hex" else 3)
    if mem:
        w = min(w, max(1, int(0.6 * mem // (ORACLE_BYTES_PER_POINT[kind] * pts))))
    return max(1, w)


def _oracle_input(kind, n):
    import oracle as O
    from paper_1902_09761_gb300 import inputs

    P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)
    if kind == "hex":
        return inputs.hex_voronoi(O.uniform_solid_hex(P), n=n), O.hex_lattice(), (H, H), P
    return inputs.bcc_sphere(O.uniform_solid_bcc(P), n=n), O.bcc_lattice(), (H, H, H), P


def _oracle_replica(idx, kind, n, steps, warmup, barrier, queue, save_dir):
    """One host process: `warmup` untimed and `steps` timed oracle steps of its own replica."""
    try:
        import oracle as O

        eta, L, h, P = _oracle_input(kind, n)
        zeta = None
        for _ in range(warmup):
            eta, zeta = O.step(eta, 1.0, P, L, h)
        barrier.wait()
        t0 = time.perf_counter()
        for _ in range(steps):
            eta, zeta = O.step(eta, 1.0, P, L, h)
        secs = time.perf_counter() - t0
        if save_dir is not None and idx == 0:
            np.save(os.path.join(save_dir, "eta.npy"), eta)
            np.save(os.path.join(save_dir, "zeta.npy"), zeta)
        queue.put((idx, secs, None))
    except Exception as e:  # reported to the parent, which raises
        try:
            barrier.abort()
        except Exception:
            pass
        queue.put((idx, None, repr(e)))


def oracle_on_host(kind, n, steps, warmup=0, workers=0, save_dir=None):
    """The oracle on the host cores: `workers` spawned processes (one per core), each stepping
    its own replica of the n^d workload; a barrier aligns the timed regions.  Returns
    (DOF-steps/s over all replicas, seconds of the slowest replica, workers).  Replica 0
    saves its final (eta, zeta) under save_dir.  Spawned (not forked) processes are safe
    after CUDA has been initialised in this one."""
    import multiprocessing as mp
    import queue as Q

    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    w = oracle_workers(kind, n, workers)
    mpc = mp.get_context("spawn")
    bar = mpc.Barrier(w)
    q = mpc.Queue()
    procs = [mpc.Process(target=_oracle_replica, args=(i, kind, n, steps, warmup, bar, q, save_dir), daemon=True)
             for i in range(w)]
    for p in procs:
        p.start()
    res = []
    try:
        for _ in range(w):
            res.append(q.get(timeout=ORACLE_TIMEOUT_S))
    except Q.Empty:
        raise RuntimeError("oracle host process timed out or died")
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    errs = [e for _, _, e in res if e]
    if errs:
        raise RuntimeError("oracle host process failed: " + errs[0])
    secs = max(t for _, t, _ in res)
    J = 3 if kind == "hex" else 6
    return w * J * n ** (2 if kind == "hex" else 3) * steps / secs, secs, w


def run_reference(args):
    world, rank, local = init_dist(args)
    if rank != 0:
        return
    n = args.size
    rate, secs, w = oracle_on_host("hex", n, args.steps, args.warmup, args.oracle_workers)
    sample = (
        f"{w} host processes (one per core), each stepping its own replica of the full {n}x{n} workload "
        f"with the FP64 oracle (numpy, exact FFT Schur solve): {args.steps} timed steps after {args.warmup} "
        f"warm-up, {secs:.1f} s for the slowest replica"
    )
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": rate,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(n),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": w, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def rel_l2_fields(eta, zeta, o_eta, o_zeta):
    """Relative L2 error per field (eta_j and zeta_j) against the oracle's result."""
    f = lambda a, b: float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))  # noqa: E731
    return {"eta": [f(eta[j], o_eta[j]) for j in range(eta.shape[0])],
            "zeta": [f(zeta[j], o_zeta[j]) for j in range(zeta.shape[0])]}


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------


def run_ours(args):
    import torch

    world, rank, local = init_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1902_09761_gb300 import apfc as A
    from paper_1902_09761_gb300 import inputs

    A.load()
    n = args.size
    J = 3
    k = inputs.hex_vectors()
    lat = A.make_lattice(k, A.APFC_LATTICE_HEX2D)
    prm = A.make_params(*PARAMS)
    phi = A.apfc_uniform_amplitude(lat, prm)
    eta0 = inputs.hex_voronoi(phi, n=n, seed=1 + rank)
    dof = J * n * n
    stream = torch.cuda.current_stream(dev)

    opts = A.apfc_default_opts(
        precision=A.APFC_FP32_REFINED, tol=TOL, cheb_degree=args.cheb, tol_inner=args.tol_inner, tile=args.tile,
        tile_rows=args.rows, picard_iters=args.picard, jacobian=int(args.jacobian), tile_t=args.tile_t,
        guess=args.guess,
    )
    ctx = A.Context(k, A.APFC_LATTICE_HEX2D, prm, (n, n), (H, H), opts, stream=stream.cuda_stream)
    eta_dev = torch.from_numpy(eta0).to(dev)

    # segment height of the fused kernels, timed on the warmed-up state (apfc_autotune;
    # outside the timed region, like a library's benchmark mode)
    tuned = None
    if args.rows == 0 and not args.no_autotune:
        ctx.set_amplitudes(eta_dev)
        ctx.step(1.0, args.warmup)
        tuned = ctx.autotune(1.0)
        opts.tile_rows, opts.tile_t = tuned["tile_rows"], tuned["tile_t"]

    def timed_steps(nsteps, sampler=None, timed_kernel=None):
        ctx.set_amplitudes(eta_dev)
        ctx.step(1.0, args.warmup)
        if timed_kernel is not None:
            ctx.profile_start(timed_kernel)
        barrier(world)
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        it0 = ctx.stats()["iters_total"]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(1.0, nsteps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        barrier(world)
        ms = e0.elapsed_time(e1)
        # Krylov iterations per timed step (of each solve, the slowest amplitude's)
        iters = (ctx.stats()["iters_total"] - it0) / max(nsteps, 1)
        return allmax(world, ms, dev), clocks, iters

    # --- headline: FP32 Krylov + FP64 refinement --------------------------------
    sampler = ClockSampler(local)
    ms, clocks, iters_mean = timed_steps(args.steps, sampler, args.timed_kernel)
    st = ctx.stats()
    prof = ctx.profile_read(args.timed_kernel)
    ctx.profile_stop()
    value = world * dof * args.steps / (ms * 1e-3)

    peak, peak_src = measured_peaks()
    avg_ms = prof["ms"] / max(prof["launches"], 1)
    bytes_per_launch = prof["bytes"] / max(prof["launches"], 1)
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
    traffic = ncu_traffic(args.timed_kernel, bytes_per_launch)

    # --- arithmetic peaks of this GPU (FP64 / FP32 FMA, FP64 <-> FP32 conversions) ----
    alu = {
        "fp64_fma_tflops": A.measure_alu_rate(A.APFC_ALU_FMA64, stream.cuda_stream) / 1e12,
        "fp32_fma_tflops": A.measure_alu_rate(A.APFC_ALU_FMA32, stream.cuda_stream) / 1e12,
        "fp64_cvt_tops": A.measure_alu_rate(A.APFC_ALU_CVT64, stream.cuda_stream) / 1e12,
        "how": "independent FMA / conversion chains, 8 blocks of 256 threads per SM, best of 3 launches "
               "(apfc_measure_alu_rate)",
    }

    # --- per-kernel breakdown: every launch bracketed by events (separate pass) ----
    breakdown = None
    if args.breakdown_steps > 0:
        ctx.set_amplitudes(eta_dev)
        ctx.step(1.0, args.warmup)
        ctx.profile_start("all")
        torch.cuda.synchronize(dev)
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        ctx.step(1.0, args.breakdown_steps)
        b1.record(stream)
        torch.cuda.synchronize(dev)
        wall = b0.elapsed_time(b1) / args.breakdown_steps
        per = {}
        for name in A.kernel_ids():
            r = ctx.profile_read(name)
            if r["launches"]:
                per[name] = {
                    "ms_per_step": r["ms"] / args.breakdown_steps,
                    "launches_per_step": r["launches"] / args.breakdown_steps,
                    "gbs": (r["bytes"] / (r["ms"] * 1e-3) / 1e9) if r["ms"] > 0 else None,
                }
                if name in FP64_PIPE_OPS and r["ms"] > 0:
                    per[name]["roofline"] = fp64_roofline(name, dof, r, peak, alu)
        ctx.profile_stop()
        breakdown = {
            "ms_per_step_wall": wall,
            "ms_per_step_kernels": sum(v["ms_per_step"] for v in per.values()),
            "kernels": dict(sorted(per.items(), key=lambda kv: -kv[1]["ms_per_step"])),
        }

    # --- plain FP64 path at the same final residual ------------------------------
    opts64 = A.apfc_default_opts(precision=A.APFC_FP64, tol=TOL, cheb_degree=args.cheb, tile_rows=args.rows,
                                 picard_iters=args.picard, jacobian=int(args.jacobian))
    ctx.set_opts(opts64)
    ms64, _, _ = timed_steps(args.fp64_steps)
    st64 = ctx.stats()
    value64 = world * dof * args.fp64_steps / (ms64 * 1e-3)

    # --- end to end through the C ABI with pinned host buffers -------------------
    # The state lives on the host: every step copies it in (host -> device), advances
    # it one step and copies the result out (device -> host), which is the next step's
    # input.  It starts from the warmed-up state of the timed region.
    ctx.set_opts(opts)
    h_state = torch.empty(eta0.shape, dtype=torch.complex128).pin_memory()
    h_np = h_state.numpy()
    ctx.set_amplitudes(eta_dev)
    ctx.step(1.0, args.warmup)
    ctx.get_amplitudes(h_np)
    barrier(world)
    torch.cuda.synchronize(dev)
    phase = [0.0, 0.0, 0.0]  # seconds in set_amplitudes, step, get_amplitudes
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ta = time.perf_counter()
        ctx.set_amplitudes(h_np)  # host -> device copy of the step's input
        tb = time.perf_counter()
        ctx.step(1.0, 1)
        torch.cuda.synchronize(dev)
        tc = time.perf_counter()
        ctx.get_amplitudes(h_np)  # device -> host copy of the step's result
        td = time.perf_counter()
        phase[0] += tb - ta
        phase[1] += tc - tb
        phase[2] += td - tc
    torch.cuda.synchronize(dev)
    e2e_s = allmax(world, time.perf_counter() - t0, dev)
    barrier(world)
    e2e = world * dof * args.e2e_steps / e2e_s
    bytes_step = eta0.nbytes
    e2e_phases = {
        "set_amplitudes_ms": 1e3 * phase[0] / args.e2e_steps,
        "step_ms": 1e3 * phase[1] / args.e2e_steps,
        "get_amplitudes_ms": 1e3 * phase[2] / args.e2e_steps,
        "h2d_gbs": bytes_step / max(phase[0] / args.e2e_steps, 1e-12) / 1e9,
        "d2h_gbs": bytes_step / max(phase[2] / args.e2e_steps, 1e-12) / 1e9,
        "note": "wall time per call; set_amplitudes also forms zeta = G_h eta on the device, and the step "
                "after it takes a stencil initial residual (a new state has no previous residual)",
    }

    # --- rotation diagnostic and adaptivity map of the final state (Sec. II.D) ------
    ctx.set_amplitudes(eta_dev)
    ctx.step(1.0, 1)
    adapt = dict(n=10.0, h_int=2.0, h_max=40.0, eps=0.02, A_min=0.05)
    ctx.rotation_field(adapt, device=dev)
    ctx.profile_start("rotation_f64")
    torch.cuda.synchronize(dev)
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    reps = 5
    for _ in range(reps):
        ctx.rotation_field(adapt, device=dev)
    r1.record(stream)
    torch.cuda.synchronize(dev)
    rot = ctx.profile_read("rotation_f64")
    ctx.profile_stop()
    rot_ms = rot["ms"] / max(rot["launches"], 1)
    rotation = {
        "ms": rot_ms,
        "gbs": (rot["bytes"] / max(rot["launches"], 1)) / (rot_ms * 1e-3) / 1e9 if rot_ms > 0 else None,
        "wall_ms_per_call": r0.elapsed_time(r1) / reps,
    }

    # --- one step from eta0 in both precisions: the error against the oracle ----------
    first = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        for name, o in (("fp32_refined", opts), ("fp64", opts64)):
            ctx.set_opts(o)
            ctx.set_amplitudes(eta_dev)
            ctx.step(1.0, 1)
            first[name] = (ctx.get_amplitudes(), ctx.get_zeta(), ctx.stats()["resid_last"])
        ctx.set_opts(opts)
    ctx.close()
    del eta_dev
    torch.cuda.empty_cache()

    # --- the other workloads, as sub-records of this line --------------------------
    subs = {}
    if args.sub_steps > 0:
        sub_args = argparse.Namespace(**vars(args))
        sub_args.steps = args.sub_steps
        sub_args.fp64_steps, sub_args.e2e_steps, sub_args.breakdown_steps = 2, 2, 1
        subs["bcc3d"] = run_bcc(sub_args, world, rank, local, sub=True)
        batch_args = argparse.Namespace(**vars(sub_args))
        batch_args.steps = args.sub_steps_batch
        subs["batch"] = run_batch(batch_args, world, rank, local, sub=True)
        adj_args = argparse.Namespace(**vars(sub_args))
        adj_args.steps = 1
        subs["adjoint"] = run_adjoint(adj_args, world, rank, local, sub=True)

    # --- CPU baseline: the oracle on this host's cores (rank 0, N = 1 only), and the
    # error of the first GPU step against the oracle's ------------------------------
    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        with tempfile.TemporaryDirectory() as tmp:
            rate, secs, w = oracle_on_host("hex", n, 1, 0, args.oracle_workers, save_dir=tmp)
            o_eta, o_zeta = np.load(os.path.join(tmp, "eta.npy")), np.load(os.path.join(tmp, "zeta.npy"))
        cpu = {
            "value": rate,
            "unit": UNIT,
            "cores": w,
            "kind": "oracle",
            "sample": f"one FP64 oracle step (numpy, exact FFT Schur solve) of the full {n}x{n} workload from "
            f"eta0 in each of {w} host processes (one per core, each its own replica), {secs:.1f} s",
        }
        err = {name: dict(rel_l2_fields(e, z, o_eta, o_zeta), resid=r) for name, (e, z, r) in first.items()}
        err["note"] = ("first step from eta0 at tol 1e-10, relative L2 per field (eta_j, zeta_j) against the "
                       "oracle's exact step; resid = the GPU solve's final relative residual")
        if "bcc3d" in subs and subs["bcc3d"] is not None and not args.no_cpu_baseline:
            bcc_oracle_leg(args, subs["bcc3d"])
    if rank != 0:
        return
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 Krylov + f64 refinement",
        "data": "synthetic",
        "config": dict(workload_config(n), **({"parallelism": f"replicas x{world}"} if world > 1 else {})),
        "iters_per_step_last": st["iters_last"],
        "iters_per_step_mean": iters_mean,
        "refine_sweeps_last": st["refine_last"],
        "resid_last": st["resid_last"],
        "fp64": {
            "value": value64,
            "unit": UNIT,
            "ms_per_step": ms64 / args.fp64_steps,
            "steps": args.fp64_steps,
            "iters_last": st64["iters_last"],
            "resid_last": st64["resid_last"],
        },
        "speedup_fp32_refined_vs_fp64": value / value64,
        "roofline": {
            "bound": "hbm",
            "kernel": args.timed_kernel,
            "achieved": achieved,
            "peak": peak,
            "peak_source": peak_src,
            "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "avg_launch_ms": avg_ms,
            "launches": prof["launches"],
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": bytes_step,
                "phases": e2e_phases},
        "autotune": tuned,
        "gpu_launches": prof["all_launches"],
        "error_vs_oracle": err,
        "alu_peaks": alu,
        "breakdown": breakdown,
        "rotation_diagnostic": rotation,
        "clocks": clocks,
    }
    for key, rec in subs.items():
        if rec is not None:
            rec.pop("_first", None)
            line[key] = rec
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Batched workload: independent hexagonal runs of uneven sizes
# ---------------------------------------------------------------------------

BATCH_SIZES = (128, 256, 512, 1024)


def batch_config(args, spec, tuned=None):
    ns = [n for n, _, _ in spec]
    cfg = {
        "workload": f"hex2d-batch{len(spec)}-N{min(BATCH_SIZES)}-{max(BATCH_SIZES)}",
        "lattice": "triangular, J=3",
        "runs": len(spec),
        "sizes": {str(n): ns.count(n) for n in BATCH_SIZES},
        "grain": "one circular grain (radius N h / 4) per run, rotation U[-10, 10] deg, in liquid",
        "h": "pi/2",
        "dt": 1.0,
        "params": {"dB": PARAMS[0], "Bx": PARAMS[1], "t": PARAMS[2], "v": PARAMS[3]},
        "tol": TOL,
        "tol_inner": TOL_INNER,
        "cheb_degree": CHEB,
        "graph": not args.no_graph,
        "l2": "inputs larger than L2 (FP64 state of all runs about 2 GB); no flush",
    }
    if tuned:
        cfg["autotuned"] = tuned
    return cfg


def batch_states(spec, phi):
    from paper_1902_09761_gb300 import inputs

    return [inputs.batch_run_state(phi, n, th, seed) for n, th, seed in spec]


def oracle_batch_rate(spec, states):
    """Oracle step time of one run of each size, summed over the batch's runs."""
    import oracle as O

    P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)
    L = O.hex_lattice()
    per_n, total_s, dof = {}, 0.0, 0
    for (n, _, _), eta in zip(spec, states):
        if n not in per_n:
            t0 = time.perf_counter()
            O.step(eta, 1.0, P, L, (H, H))
            per_n[n] = time.perf_counter() - t0
        total_s += per_n[n]
        dof += 3 * n * n
    sample = (
        "one oracle FP64 step (numpy, exact FFT Schur solve) of one run of each size "
        + ", ".join(f"{n}^2 {per_n[n]:.2f} s" for n in sorted(per_n))
        + f"; batch step estimated as the sum over its {len(spec)} runs"
    )
    return dof / total_s, total_s, sample


def run_batch_reference(args):
    world, rank, local = init_dist(args)
    if rank != 0:
        return
    import oracle as O
    from paper_1902_09761_gb300 import inputs

    P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)
    spec = inputs.batch_spec(args.runs, BATCH_SIZES, seed=7)
    states = batch_states(spec, O.uniform_solid_hex(P))
    rate, secs, sample = oracle_batch_rate(spec, states)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": rate,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * secs,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": batch_config(args, spec),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args, world=None, rank=None, local=None, sub=False):
    """The batched workload; sub: return its record (no print, no runs-alone comparison)."""
    import torch

    if world is None:
        world, rank, local = init_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1902_09761_gb300 import apfc as A
    from paper_1902_09761_gb300 import inputs

    A.load()
    k = inputs.hex_vectors()
    lat = A.make_lattice(k, A.APFC_LATTICE_HEX2D)
    prm = A.make_params(*PARAMS)
    phi = A.apfc_uniform_amplitude(lat, prm)
    spec = inputs.batch_spec(args.runs, BATCH_SIZES, seed=7 + rank)
    states = batch_states(spec, phi)
    shapes = [(n, n) for n, _, _ in spec]
    dof = 3 * sum(n * n for n, _, _ in spec)
    stream = torch.cuda.Stream(dev)  # graph capture needs a non-default stream

    opts = A.apfc_default_opts(
        precision=A.APFC_FP32_REFINED, tol=TOL, cheb_degree=args.cheb, tol_inner=args.tol_inner, tile=args.tile,
        tile_rows=args.rows,
    )
    b = A.Batch(k, A.APFC_LATTICE_HEX2D, prm, shapes, (H, H), opts, graph=not args.no_graph,
                stream=stream.cuda_stream)
    dev_states = [torch.from_numpy(e).to(dev) for e in states]

    def reset():
        for r, e in enumerate(dev_states):
            b.set_amplitudes(r, e)

    tuned = None
    reset()
    if not args.no_autotune:
        tuned = b.autotune(1.0)

    def timed(nsteps, sampler=None):
        reset()
        b.step(1.0, args.warmup)
        barrier(world)
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(1.0, nsteps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        barrier(world)
        return allmax(world, e0.elapsed_time(e1), dev), clocks

    # --- headline: all runs in one batch (graphs on, no measurement hooks) ----------
    sampler = ClockSampler(local)
    ms, clocks = timed(args.steps, sampler)
    stats = [b.stats(r) for r in range(len(spec))]
    value = world * dof * args.steps / (ms * 1e-3)
    replays = b.graph_replays()

    # --- measurement pass: dominant kernel and launch count -------------------------
    reset()
    b.step(1.0, args.warmup)
    b.profile_start(args.timed_kernel)
    torch.cuda.synchronize(dev)
    b.step(1.0, max(args.breakdown_steps, 1))
    prof = b.profile_read(args.timed_kernel)
    b.profile_stop()

    # --- per-kernel device time (every launch timed, graphs off while measuring) against
    # the graph-replayed wall time of the same steps (same start, same iterations) ------
    nb_steps = max(args.breakdown_steps, 1)
    ms_nb, _ = timed(nb_steps)
    reset()
    b.step(1.0, args.warmup)
    b.profile_start("all")
    torch.cuda.synchronize(dev)
    b.step(1.0, nb_steps)
    per = {}
    for name in A.kernel_ids():
        r = b.profile_read(name)
        if r["launches"]:
            per[name] = {"ms_per_step": r["ms"] / nb_steps, "launches_per_step": r["launches"] / nb_steps}
    b.profile_stop()
    kernels_ms = sum(v["ms_per_step"] for v in per.values())
    peak, peak_src = measured_peaks()
    avg_ms = prof["ms"] / max(prof["launches"], 1)
    bytes_per_launch = prof["bytes"] / max(prof["launches"], 1)
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
    launches_per_step = prof["all_launches"] / max(args.breakdown_steps, 1)

    # --- end to end through the C ABI with pinned host buffers ------------------------
    h_in = [torch.from_numpy(e).pin_memory() for e in states]
    h_out = [torch.empty(e.shape, dtype=torch.complex128).pin_memory().numpy() for e in states]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for r in range(len(spec)):
            b.set_amplitudes(r, h_in[r])
        b.step(1.0, 1)
        for r in range(len(spec)):
            b.get_amplitudes(r, h_out[r])
    torch.cuda.synchronize(dev)
    e2e_s = allmax(world, time.perf_counter() - t0, dev)
    e2e = world * dof * args.e2e_steps / e2e_s
    bytes_step = sum(e.nbytes for e in states)
    tuned_opts = b.opts
    b.close()

    # --- the same runs one at a time: FP32-refined and plain FP64 ---------------------
    def alone(o, nsteps):
        if nsteps <= 0:
            return None
        total = 0.0
        for r, (n, _, _) in enumerate(spec):
            with A.Context(k, A.APFC_LATTICE_HEX2D, prm, (n, n), (H, H), o, stream=stream.cuda_stream) as c:
                c.set_amplitudes(dev_states[r])
                c.step(1.0, args.warmup)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                c.step(1.0, nsteps)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                total += e0.elapsed_time(e1) / nsteps
        return total

    alone32 = alone(tuned_opts, 0 if sub else args.alone_steps)
    alone64 = alone(
        A.apfc_default_opts(precision=A.APFC_FP64, tol=TOL, cheb_degree=args.cheb),
        0 if sub else min(args.alone_steps, args.fp64_steps),
    )

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs, sample = oracle_batch_rate(spec, states)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    if rank != 0:
        return None
    ms_step = ms / args.steps
    per_n = {}
    for (n, _, _), st in zip(spec, stats):
        per_n.setdefault(str(n), []).append(st["iters_last"])
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 Krylov + f64 refinement",
        "data": "synthetic",
        "config": dict(batch_config(args, spec, tuned), **({"parallelism": f"replicas x{world}"} if world > 1 else {})),
        "per_run_ms_per_step": ms_step / len(spec),
        "iters_last_by_size": {n: max(v) for n, v in per_n.items()},
        "resid_last_max": max(st["resid_last"] for st in stats),
        "graph_replays": replays,
        "alone_fp32_refined_ms_per_step": alone32,
        "alone_fp64_ms_per_step": alone64,
        "speedup_batch_vs_alone_fp32_refined": (alone32 / ms_step) if alone32 else None,
        "speedup_batch_vs_alone_fp64": (alone64 / ms_step) if alone64 else None,
        "roofline": {
            "bound": "hbm",
            "kernel": args.timed_kernel,
            "achieved": achieved,
            "peak": peak,
            "peak_source": peak_src,
            "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": None,
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "avg_launch_ms": avg_ms,
            "launches": prof["launches"],
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": bytes_step},
        "gpu_launches_per_step": launches_per_step,
        "gpu_launches": int(launches_per_step * args.steps),
        "breakdown": {
            "steps": nb_steps,
            "ms_per_step_graph": ms_nb / nb_steps,
            "ms_per_step_kernels": kernels_ms,
            "launch_gaps_ms_per_step": ms_nb / nb_steps - kernels_ms,
            "note": "the first steps after the warm-up, twice: graph-replayed as in the timed region "
                    "(wall time), and with every launch timed (graphs off; kernel device times summed); "
                    "the difference is the time between kernels that fewer launches could save",
            "kernels": dict(sorted(per.items(), key=lambda kv: -kv[1]["ms_per_step"])),
        },
        "clocks": clocks,
    }
    if sub:
        return line
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Adjoint workload: gradient of L = misfit + F after a rollout, wrt eta0 and dB
# ---------------------------------------------------------------------------


def adjoint_config(args, tuned=None):
    return {
        "workload": f"hex2d-{args.adj_size}x{args.adj_size}-adjoint-{args.rollout}steps",
        "lattice": "triangular, J=3",
        "grid": [args.adj_size, args.adj_size],
        "initial": "8 Voronoi grains, rotations U[-10, 10] deg, noise 1e-3, seed 3",
        "loss": "1/2 h^2 sum |eta^K - target|^2 + F(eta^K), target seeded N(0, 0.1^2) complex",
        "grad": "wrt eta0 (complex128) and dB",
        "rollout_steps": args.rollout,
        "checkpoint_every": args.every,
        "h": "pi/2",
        "dt": 1.0,
        "params": {"dB": PARAMS[0], "Bx": PARAMS[1], "t": PARAMS[2], "v": PARAMS[3]},
        "tol": TOL,
        "unit_note": "one DOF-step = one amplitude DOF through one step forward and its adjoint",
        "l2": "inputs larger than L2 (states 50 MB each, checkpoints 0.55 GB); no flush",
    }


def adjoint_states(n, phi):
    from paper_1902_09761_gb300 import inputs

    eta0 = inputs.voronoi_grains(inputs.hex_vectors(), phi, (n, n), (H, H), 8, 10.0, seed=3, noise=1e-3)
    rng = np.random.default_rng(4)
    target = 0.1 * (rng.standard_normal(eta0.shape) + 1j * rng.standard_normal(eta0.shape))
    return eta0, target


def oracle_adjoint_rate(n, steps):
    import oracle as O
    from paper_1902_09761_gb300 import inputs

    P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)
    L = O.hex_lattice()
    eta0 = inputs.voronoi_grains(inputs.hex_vectors(), O.uniform_solid_hex(P), (n, n), (H, H), 8, 10.0, seed=3,
                                 noise=1e-3)
    target = np.zeros_like(eta0)
    t0 = time.perf_counter()
    O.rollout_gradient(eta0, P.dB, target, 1.0, steps, P, L, (H, H))
    secs = time.perf_counter() - t0
    return 3.0 * n * n * steps / secs, secs


def run_adjoint_reference(args):
    world, rank, local = init_dist(args)
    if rank != 0:
        return
    n = min(args.adj_size, 512)
    steps = min(args.rollout, 20)
    rate, secs = oracle_adjoint_rate(n, steps)
    sample = f"oracle rollout gradient (FFT-exact forward and adjoint solves) on {n}x{n}, {steps} steps, {secs:.1f} s"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": adjoint_config(args),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args, world=None, rank=None, local=None, sub=False):
    """The adjoint workload; sub: return its record (no print, no host baseline)."""
    import torch

    if world is None:
        world, rank, local = init_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1902_09761_gb300 import apfc as A
    from paper_1902_09761_gb300 import inputs
    from paper_1902_09761_gb300.autograd import Rollout

    A.load()
    n, K = args.adj_size, args.rollout
    phi = A.apfc_uniform_amplitude(A.make_lattice(inputs.hex_vectors(), A.APFC_LATTICE_HEX2D), A.make_params(*PARAMS))
    eta0, target = adjoint_states(n, phi)
    dof = 3 * n * n
    vol = H * H
    stream = torch.cuda.current_stream(dev)
    opts = A.apfc_default_opts(precision=A.APFC_FP32_REFINED, tol=TOL, cheb_degree=args.cheb,
                               tol_inner=args.tol_inner, tile=args.tile, tile_rows=args.rows, tile_t=args.tile_t)
    ro = Rollout(inputs.hex_vectors(), A.APFC_LATTICE_HEX2D, PARAMS, (n, n), (H, H), 1.0, K, args.every, opts,
                 device=dev)
    e0_dev = torch.from_numpy(eta0).to(dev)
    tg = torch.from_numpy(target).to(dev)
    # segment height and t-kernel variant for this grid, timed on a few steps from eta0
    tuned = None
    if args.rows == 0 and not args.no_autotune:
        ro.ctx.set_amplitudes(e0_dev)
        ro.ctx.step(1.0, 3)
        tuned = ro.ctx.autotune(1.0)

    def grad_once():
        e0 = e0_dev.clone().requires_grad_(True)
        dB = torch.tensor(PARAMS[0], dtype=torch.float64, requires_grad=True)
        etaN, F = ro(e0, dB)
        loss = 0.5 * vol * (etaN - tg).abs().pow(2).sum() + F
        loss.backward()
        return e0.grad, dB.grad

    for _ in range(args.warmup):
        grad_once()
    barrier(world)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    e0t = torch.cuda.Event(enable_timing=True)
    e1t = torch.cuda.Event(enable_timing=True)
    e0t.record(stream)
    for _ in range(args.steps):
        grad_once()
    e1t.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = allmax(world, e0t.elapsed_time(e1t), dev) / args.steps  # per gradient evaluation
    value = world * dof * K / (ms * 1e-3)

    # forward and backward separately, and the dominant kernel's roofline
    ctx = ro.ctx
    ctx.set_amplitudes(e0_dev)
    torch.cuda.synchronize(dev)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    ctx.profile_start(args.timed_kernel)
    f0.record(stream)
    ctx.rollout_forward(1.0, K, args.every)
    f1.record(stream)
    lamN = torch.zeros_like(e0_dev)
    lam0 = torch.empty_like(e0_dev)
    ctx.rollout_backward(lamN + 1e-3, lam0)
    b1.record(stream)
    torch.cuda.synchronize(dev)
    prof = ctx.profile_read(args.timed_kernel)
    ctx.profile_stop()
    fwd_ms, bwd_ms = f0.elapsed_time(f1), f1.elapsed_time(b1)
    peak, peak_src = measured_peaks()
    avg_ms = prof["ms"] / max(prof["launches"], 1)
    bpl = prof["bytes"] / max(prof["launches"], 1)
    achieved = bpl / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None

    # end to end with host buffers: the same gradient through host-resident inputs and outputs
    h_e0 = torch.from_numpy(eta0).pin_memory()
    h_tg = torch.from_numpy(target).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0 = h_e0.to(dev, non_blocking=True).requires_grad_(True)
    dB = torch.tensor(PARAMS[0], dtype=torch.float64, requires_grad=True)
    etaN, F = ro(e0, dB)
    loss = 0.5 * vol * (etaN - h_tg.to(dev, non_blocking=True)).abs().pow(2).sum() + F
    loss.backward()
    g_host = e0.grad.cpu()
    _ = float(dB.grad)
    e2e_s = allmax(world, time.perf_counter() - t0, dev)
    e2e = world * dof * K / e2e_s
    ro.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not sub:
        ns, ks = min(n, 512), min(K, 20)
        rate, secs = oracle_adjoint_rate(ns, ks)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle rollout gradient (FFT-exact solves) on {ns}x{ns}, {ks} steps, {secs:.1f} s"}
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 Krylov + f64 refinement", "data": "synthetic",
        "config": dict(adjoint_config(args), **({"parallelism": f"replicas x{world}"} if world > 1 else {})),
        "ms_per_gradient": ms,
        "autotune": tuned,
        "forward_ms_per_step": fwd_ms / K,
        "backward_ms_per_step": bwd_ms / K,
        "backward_over_forward": bwd_ms / fwd_ms,
        "roofline": {
            "bound": "hbm", "kernel": args.timed_kernel, "achieved": achieved, "peak": peak,
            "peak_source": peak_src, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "traffic": None, "algorithmic_bytes_per_launch": bpl, "avg_launch_ms": avg_ms,
            "launches": prof["launches"],
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * eta0.nbytes,
                "d2h_bytes_per_step": g_host.numel() * 16 + 8},
        "gpu_launches": prof["all_launches"],
        "clocks": clocks,
    }
    if sub:
        return line
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# 3D bcc workload: a rotated spherical grain in an unrotated matrix
# ---------------------------------------------------------------------------


def bcc_config(args):
    n = args.bcc_size
    return {
        "workload": f"bcc3d-{n}^3-sphere",
        "lattice": "bcc, J=6, k = <110>/sqrt2",
        "grid": [n, n, n],
        "initial": "sphere R = 60 rotated 8 deg about [001] in an unrotated matrix, noise 1e-3, seed 2",
        "h": "pi/2",
        "dt": 1.0,
        "params": {"dB": PARAMS[0], "Bx": PARAMS[1], "t": PARAMS[2], "v": PARAMS[3]},
        "tol": TOL,
        "tol_inner": TOL_INNER,
        "cheb_degree": CHEB,
        "kernels": "one kernel per stencil pass, z-streaming (x, y) tiles: FP32 64x8 (two points per thread), FP64 32x8",
        "l2": f"inputs larger than L2 (FP64 state {16 * 12 * n ** 3 / 1e9:.1f} GB); no flush",
    }


def run_bcc_reference(args):
    world, rank, local = init_dist(args)
    if rank != 0:
        return
    import oracle as O
    from paper_1902_09761_gb300 import inputs

    P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)
    L = O.bcc_lattice()
    ns = min(args.bcc_size, 64)
    eta = inputs.single_grain(inputs.bcc_vectors(), O.uniform_solid_bcc(P), (ns,) * 3, (H,) * 3, 0.25 * ns * H, 8.0,
                              seed=2, noise=1e-3, matrix=O.uniform_solid_bcc(P))
    t0 = time.perf_counter()
    O.step(eta, 1.0, P, L, (H,) * 3)
    secs = time.perf_counter() - t0
    rate = 6.0 * ns ** 3 / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": bcc_config(args),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"one oracle FP64 step (FFT exact solve) of a {ns}^3 bcc sphere, {secs:.2f} s"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_bcc(args, world=None, rank=None, local=None, sub=False):
    """The 3D bcc workload; sub: return its record (no print; the host-oracle leg and the
    error against the oracle are added by bcc_oracle_leg)."""
    import torch

    if world is None:
        world, rank, local = init_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1902_09761_gb300 import apfc as A
    from paper_1902_09761_gb300 import inputs

    A.load()
    n = args.bcc_size
    k = inputs.bcc_vectors()
    lat = A.make_lattice(k, A.APFC_LATTICE_BCC3D)
    prm = A.make_params(*PARAMS)
    phi = A.apfc_uniform_amplitude(lat, prm)
    eta0 = inputs.bcc_sphere(phi, n=n)
    dof = 6 * n ** 3
    stream = torch.cuda.current_stream(dev)
    opts = A.apfc_default_opts(precision=A.APFC_FP32_REFINED, tol=TOL, cheb_degree=args.cheb,
                               tol_inner=args.tol_inner)
    ctx = A.Context(k, A.APFC_LATTICE_BCC3D, prm, (n, n, n), (H, H, H), opts, stream=stream.cuda_stream)
    eta_dev = torch.from_numpy(eta0).to(dev)

    def timed(nsteps, sampler=None):
        ctx.set_amplitudes(eta_dev)
        ctx.step(1.0, args.warmup)
        barrier(world)
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(1.0, nsteps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        barrier(world)
        return allmax(world, e0.elapsed_time(e1), dev), clocks

    sampler = ClockSampler(local)
    ms, clocks = timed(args.steps, sampler)
    st = ctx.stats()
    value = world * dof * args.steps / (ms * 1e-3)

    # per-kernel breakdown (every launch bracketed by events) and the dominant kernel's roofline
    ctx.set_amplitudes(eta_dev)
    ctx.step(1.0, args.warmup)
    ctx.profile_start("all")
    torch.cuda.synchronize(dev)
    ctx.step(1.0, max(args.breakdown_steps, 1))
    per = {}
    for name in A.kernel_ids():
        r = ctx.profile_read(name)
        if r["launches"]:
            per[name] = {"ms_per_step": r["ms"] / max(args.breakdown_steps, 1),
                         "launches_per_step": r["launches"] / max(args.breakdown_steps, 1),
                         "gbs": (r["bytes"] / (r["ms"] * 1e-3) / 1e9) if r["ms"] > 0 else None,
                         "bytes": r["bytes"], "launches": r["launches"], "ms": r["ms"]}
    all_launches = ctx.profile_read("dots_f32")["all_launches"]
    ctx.profile_stop()
    top = max(per, key=lambda nm: per[nm]["ms_per_step"])
    peak, peak_src = measured_peaks()
    avg_ms = per[top]["ms"] / per[top]["launches"]
    bpl = per[top]["bytes"] / per[top]["launches"]
    achieved = bpl / (avg_ms * 1e-3) / 1e9

    # plain FP64 at the same final residual
    opts64 = A.apfc_default_opts(precision=A.APFC_FP64, tol=TOL, cheb_degree=args.cheb)
    ctx.set_opts(opts64)
    ms64, _ = timed(args.fp64_steps)
    ctx.set_opts(opts)

    # one step from eta0 in both precisions, for the error against the oracle
    first = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        for name, o in (("fp32_refined", opts), ("fp64", opts64)):
            ctx.set_opts(o)
            ctx.set_amplitudes(eta_dev)
            ctx.step(1.0, 1)
            first[name] = (ctx.get_amplitudes(), ctx.get_zeta(), ctx.stats()["resid_last"])
        ctx.set_opts(opts)

    # end to end: host-resident state copied in and out every step
    h_state = torch.empty(eta0.shape, dtype=torch.complex128).pin_memory()
    h_np = h_state.numpy()
    ctx.set_amplitudes(eta_dev)
    ctx.step(1.0, args.warmup)
    ctx.get_amplitudes(h_np)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.set_amplitudes(h_np)
        ctx.step(1.0, 1)
        ctx.get_amplitudes(h_np)
    torch.cuda.synchronize(dev)
    e2e = world * dof * args.e2e_steps / allmax(world, time.perf_counter() - t0, dev)
    ctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not sub:
        import oracle as O

        P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)
        ns = min(n, 64)
        eta_s = inputs.single_grain(k, phi, (ns,) * 3, (H,) * 3, 0.25 * ns * H, 8.0, seed=2, noise=1e-3, matrix=phi)
        t1 = time.perf_counter()
        O.step(eta_s, 1.0, P, O.bcc_lattice(), (H,) * 3)
        secs = time.perf_counter() - t1
        cpu = {"value": 6.0 * ns ** 3 / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one oracle FP64 step (FFT exact solve) of a {ns}^3 bcc sphere, {secs:.2f} s"}
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 Krylov + f64 refinement", "data": "synthetic",
        "config": dict(bcc_config(args), **({"parallelism": f"replicas x{world}"} if world > 1 else {})),
        "iters_per_step_last": st["iters_last"], "refine_sweeps_last": st["refine_last"],
        "resid_last": st["resid_last"],
        "fp64": {"value": world * dof * args.fp64_steps / (ms64 * 1e-3), "unit": UNIT,
                 "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps},
        "speedup_fp32_refined_vs_fp64": (ms64 / args.fp64_steps) / (ms / args.steps),
        "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "peak_source": peak_src,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": ncu_traffic(top, bpl),
                     "algorithmic_bytes_per_launch": bpl, "avg_launch_ms": avg_ms, "launches": per[top]["launches"]},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": eta0.nbytes, "d2h_bytes_per_step": eta0.nbytes},
        "gpu_launches": int(all_launches / max(args.breakdown_steps, 1) * args.steps),
        "breakdown": {nm: {kk: v[kk] for kk in ("ms_per_step", "launches_per_step", "gbs")}
                      for nm, v in sorted(per.items(), key=lambda kv: -kv[1]["ms_per_step"])},
        "clocks": clocks,
    }
    if sub:
        line["_first"] = first
        return line
    print(json.dumps(line), flush=True)


def bcc_oracle_leg(args, rec):
    """Host-oracle leg of the bcc3d record: one oracle step of the full sphere workload from
    eta0 in one host process per core (as memory allows); replica 0's result gives the error
    of the GPU's first step in both precisions."""
    first = rec.pop("_first", {})
    n = args.bcc_size
    with tempfile.TemporaryDirectory() as tmp:
        rate, secs, w = oracle_on_host("bcc", n, 1, 0, args.oracle_workers, save_dir=tmp)
        o_eta, o_zeta = np.load(os.path.join(tmp, "eta.npy")), np.load(os.path.join(tmp, "zeta.npy"))
    rec["cpu_baseline"] = {
        "value": rate, "unit": UNIT, "cores": w, "kind": "oracle",
        "sample": f"one FP64 oracle step (exact FFT solve) of the full {n}^3 sphere from eta0 in each of {w} host "
                  f"processes (one per core, each its own replica), {secs:.1f} s",
    }
    err = {name: dict(rel_l2_fields(e, z, o_eta, o_zeta), resid=r) for name, (e, z, r) in first.items()}
    err["note"] = "first step from eta0 at tol 1e-10, relative L2 per field against the oracle's exact step"
    rec["error_vs_oracle"] = err


CHEB = 1
TOL_INNER = 1e-4
PICARD = (1, False)


def main():
    global CHEB, TOL_INNER, PICARD
    args = parse()
    CHEB, TOL_INNER = args.cheb, args.tol_inner
    PICARD = (args.picard, bool(args.jacobian))
    if args.workload == "batch":
        run_batch_reference(args) if args.impl == "reference" else run_batch(args)
    elif args.workload == "adjoint":
        run_adjoint_reference(args) if args.impl == "reference" else run_adjoint(args)
    elif args.workload == "bcc3d":
        run_bcc_reference(args) if args.impl == "reference" else run_bcc(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
