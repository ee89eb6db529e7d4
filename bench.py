#!/usr/bin/env python3
"""Benchmark of the npFEM time step on GB300: cell-iterations per second.

Default workload: 50000 red blood cells (642-vertex Evans-Fung mesh) + 5000
platelets (162-vertex ellipsoid) in a 200^3 box, seeded Fourier + shear
forces of amplitude 0.3, BF16 tensor-core global step with FP32
accumulation and FP64-residual refinement to 1e-6, FP32 local step, K = 10
L-BFGS iterations per step, the step replayed as one CUDA graph.

One "step" = one npfem_step over all cells.  value = cells x K x steps /
time (device CUDA events on the solver's stream, max over ranks).  Inputs
(positions, forces: ~1.6 GB) are larger than L2 (129 MB), so no flush is
needed.  Also reported: the same workload in plain FP64 on the GPU, the
relative position error of both against the FP64 oracle on sampled cells,
the end-to-end number through the C ABI with host buffers, per-kernel
CUDA-event times, the roofline of the dominant kernel and the oracle timed on
the host cores.

Multi-GPU: one process per GPU (torchrun); cells are independent, each rank
steps its own suspension (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Measured DRAM traffic of k_iterate on rbc50k_plt5k (BF16 form), bytes per launch:
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture (one pass) of the
# 40 k_iterate launches of one step, averaged over the 20 launches that process all
# cells (the fallback-list launches, ~0.1 MB each, excluded like their times).
# Set to None whenever k_iterate changes until it is captured again.
ITERATE_TRAFFIC = 4.012e9
PARITY_CELLS = 16        # cells per mesh type compared with the oracle (evenly spaced)
METRIC = "cell-iterations/sec at 50k cells, mixed vs FP64 GPU at ≤1e-6 rel pos error"
UNIT = "cell-iterations/s"


# ---------------------------------------------------------------- helpers
def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes_iterate(nV, cells, K, m, b, bf16):
    """Bytes one k_iterate launch must move on average (per type, all its cells).

    Per cell and iteration k (vectors of 3 nV values of b bytes):
      read z, grad g, delta, y_rel                          4 vectors
      read the history pairs of the two L-BFGS loops       2 min(k, m) + 2 min(k+1, m) vectors
      write delta, grad g, the new pair (s, y), q            5 vectors (+ BF16 copy of q)
      last iteration instead of q and the first loop: read x_n, v_n, F_ext,
      write x_{n+1}, v_{n+1} (FP64).
    """
    n3 = 3 * nV
    tot = 0.0
    for k in range(K):
        last = k == K - 1
        vec = 4 + 2 * min(k, m) + 4
        byt = vec * n3 * b
        if last:
            byt += 5 * n3 * 8
        else:
            byt += (2 * min(k + 1, m) + 1) * n3 * b + (n3 * 2 if bf16 else 0)
        tot += byt
    return tot / K * cells


def algorithmic_gemm(nV, cells, bf16):
    """One global-step apply: read q (operand type), write z (FP32); 2 nV flops per element."""
    n = 3 * cells * nV
    return n * ((2 if bf16 else 4) + 4), 2.0 * nV * n


def with_damping(groups, alpha, beta):
    """Rayleigh damping C = alpha M + beta L on every group's mesh type (0, 0: unchanged)."""
    if alpha or beta:
        for g in groups:
            mat = dataclasses.replace(g.mtype.material, rayleigh_alpha=alpha, rayleigh_beta=beta)
            g.mtype = dataclasses.replace(g.mtype, material=mat)
    return groups


def oracle_step_sampled(groups, xn, vn, args, K=10):
    """One FP64 oracle step of sampled cells from the given state (public layout
    arrays), with the force median and, when --pik-radius is set, the particle-in-
    kernel search over each sampled cell and the cells whose bounding spheres come
    within the kernel radius of it (every vertex that can be in its kernels).
    Returns [(idx, x1)] per group."""
    from oracle import oracle as O
    shapes, offs, off = [], [], 0
    for g in groups:
        shapes.append((g.n_cells, g.mtype.nV, 3))
        offs.append(off)
        off += g.n_cells * g.mtype.nV * 3
    X = [xn[o:o + np.prod(sh)].reshape(sh) for o, sh in zip(offs, shapes)]
    V = [vn[o:o + np.prod(sh)].reshape(sh) for o, sh in zip(offs, shapes)]
    Ts = [O.OracleType.from_mesh_type(g.mtype) for g in groups]
    out = []
    if args.pik_radius > 0:
        cen = np.concatenate([x.mean(axis=1) for x in X])
        rad = np.concatenate([np.linalg.norm(x - x.mean(axis=1, keepdims=True), axis=2).max(axis=1) for x in X])
        gid = np.concatenate([np.full(g.n_cells, gi) for gi, g in enumerate(groups)])
        cid = np.concatenate([np.arange(g.n_cells) for g in groups])
        base = np.cumsum([0] + [g.n_cells for g in groups])
    for gi, g in enumerate(groups):
        idx = np.unique(np.linspace(0, g.n_cells - 1, PARITY_CELLS).astype(int))
        T = Ts[gi]
        fs = O.force_median(T, g.f_ext[idx]) if args.force_median else g.f_ext[idx]
        if args.pik_radius <= 0:
            xo, _ = T.step_cells(X[gi][idx].copy(), V[gi][idx].copy(), fs, K=K, m=5, threads=os.cpu_count() or 4)
            out.append((idx, xo))
            continue
        xo = np.empty((len(idx), g.mtype.nV, 3))
        for k, c in enumerate(idx):
            a = base[gi] + c
            near = np.flatnonzero(np.linalg.norm(cen - cen[a], axis=1) < rad + rad[a] + args.pik_radius)
            cells = [(Ts[gid[b]], X[gid[b]][cid[b]]) for b in near]          # global (public) order
            hc, _, p = O.pik(cells, args.pik_radius)[int(np.flatnonzero(near == a)[0])]
            x1, _ = T.step_cells_col(X[gi][c][None], V[gi][c][None], fs[k][None], args.collision_k,
                                     (hc >= 0).astype(np.int32)[None], p[None], K=K, m=5)
            xo[k] = x1[0]
        out.append((idx, xo))
    return out


# ---------------------------------------------------------------- peaks
def measure_peaks(local):
    """Arithmetic peaks the roofline needs beyond MEASURED_PEAKS.json: FP32 FMA and
    FP64 FMA on the SIMT pipes (libnpfem_peaks.so probes: 16 independent FMA chains
    per thread, 8 blocks of 256 threads per SM), and TF32 / BF16 dense tensor
    throughput through cuBLAS (torch.matmul, 8192^3).  Each figure is the best of
    several launches timed with CUDA events; SM clocks are sampled meanwhile."""
    import ctypes
    import torch
    from paper_1911_03062_gb300 import build as B
    B.build()
    L = ctypes.CDLL(B.PEAKS_LIB)
    L.npfem_peak_fma.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.npfem_peak_fma.restype = ctypes.c_double
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    blocks = 8 * nsm
    clocks = Clocks(local)
    clocks.start()
    out = {}

    def timed(fn, reps):
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            work = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        return work, best

    buf = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    for name, fp64, iters in (("fp32_fma_tflops", 0, 20000), ("fp64_fma_tflops", 1, 200)):
        run = lambda it: L.npfem_peak_fma(fp64, ctypes.c_void_p(stream.cuda_stream), blocks, it,
                                          ctypes.c_void_p(buf.data_ptr()))
        _, t = timed(lambda: run(iters), 2)                 # calibrate to ~0.2 s per launch
        iters = max(1, int(iters * 0.2 / t))
        flops, t = timed(lambda: run(iters), 5)
        if flops < 0:
            raise RuntimeError("peak probe launch failed")
        out[name] = flops / t / 1e12
    n = 8192
    with torch.cuda.stream(stream):
        for name, dt, tf32 in (("tf32_tensor_tflops", torch.float32, True), ("bf16_tensor_tflops", torch.bfloat16, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            c = torch.empty(n, n, device="cuda", dtype=dt)
            _, t = timed(lambda: torch.matmul(a, b, out=c), 10)
            out[name] = 2.0 * n ** 3 / t / 1e12
            del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = False
    clk = clocks.stop()
    line = {"peaks": out, "clocks": clk, "gpu": torch.cuda.get_device_name(local), "sms": nsm,
            "how": "FMA probes: 16 FMA chains/thread, 8x256 threads/SM, best of 5 (CUDA events); "
                   "tensor: torch.matmul 8192^3 (cuBLAS), best of 10"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- reference
def run_reference(args, workload):
    """The FP64 CPU oracle timed on the host cores (the reference arm)."""
    from paper_1911_03062_gb300 import inputs as I
    from oracle import oracle as O
    O.build()
    groups = with_damping(I.workload_groups(workload), args.rayleigh_alpha, args.rayleigh_beta)
    threads = os.cpu_count() or 1
    sample_rbc, sample_plt = args.ref_sample
    picks = []
    for g, n in zip(groups, (sample_rbc, sample_plt)):
        sub = I.Group(g.mtype, n, g.seed, g.amp)
        picks.append((I.materialise(sub), O.OracleType.from_mesh_type(g.mtype)))
    state = [(g.x0.copy(), g.v0.copy()) for g, _ in picks]

    def one_step():
        for i, (g, T) in enumerate(picks):
            x, v = state[i]
            state[i] = T.step_cells(x, v, g.f_ext, K=10, m=5, threads=threads)

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    cells = sample_rbc + sample_plt
    value = cells * 10 * args.steps / dt
    sample = f"{sample_rbc} RBC + {sample_plt} PLT cells of the workload per step (same seeds), K=10"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload, "cells_per_step": cells, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(workload, n_rbc=768, n_plt=96, alpha=0.0, beta=0.0):
    """Oracle on the host cores over a bounded sample (1 step, K=10)."""
    from paper_1911_03062_gb300 import inputs as I
    from oracle import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    groups = with_damping(I.workload_groups(workload), alpha, beta)
    t_total, cells = 0.0, 0
    for g, n in zip(groups, (n_rbc, n_plt)):
        sub = I.materialise(I.Group(g.mtype, n, g.seed, g.amp))
        T = O.OracleType.from_mesh_type(g.mtype)
        t0 = time.perf_counter()
        T.step_cells(sub.x0, sub.v0, sub.f_ext, K=10, m=5, threads=threads)
        t_total += time.perf_counter() - t0
        cells += n
    return {"value": cells * 10 / t_total, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_rbc} RBC + {n_plt} PLT cells of the workload, 1 step x 10 iterations, "
                      f"cells split over {threads} host threads"}


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="rbc50k_plt5k")
    ap.add_argument("--precision", default=None, help="bf16 | tf32 | fp64 (default: the workload's)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 form (0: skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-sample", type=int, nargs=2, default=[160, 16])
    ap.add_argument("--force-median", action="store_true", help="one-ring median filter of the forces before each step")
    ap.add_argument("--u-max", type=float, default=0.0, help="velocity cap after each step (0: off)")
    ap.add_argument("--pbd-kappa", type=float, default=0.0, help="PBD velocity damping after each step (0: off)")
    ap.add_argument("--rayleigh-alpha", type=float, default=0.0, help="Rayleigh damping C = alpha M + beta L")
    ap.add_argument("--rayleigh-beta", type=float, default=0.0, help="(the paper's table: alpha 0, beta 0.01)")
    ap.add_argument("--pik-radius", type=float, default=0.0, help="particle-in-kernel collision kernel radius (0: off)")
    ap.add_argument("--collision-k", type=float, default=2.0,
                    help="collision stiffness (with --pik-radius; at 200 the BF16 form misses 1e-6 in deep overlaps)")
    ap.add_argument("--ibm-cycles", type=int, default=0, help="also time the immersed-boundary forces (0: skip)")
    ap.add_argument("--peaks", action="store_true", help="measure FP32/FP64 FMA and TF32/BF16 tensor peaks, exit")
    args = ap.parse_args()
    rank, world, local = env_rank()

    if args.peaks:
        if rank == 0:
            measure_peaks(local)
        return

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, args.workload)
        return

    import torch
    from paper_1911_03062_gb300 import inputs as I
    from paper_1911_03062_gb300.npfem import Solver
    from paper_1911_03062_gb300 import build as B
    from paper_1911_03062_gb300.shard import shard_groups
    B.build()

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    wl = I.WORKLOADS[args.workload]
    precision = args.precision or wl["precision"]
    # each rank steps its own suspension (weak scaling; the partition of shard.py)
    groups = with_damping(shard_groups(args.workload, rank, world, "weak"), args.rayleigh_alpha,
                          args.rayleigh_beta)
    ncells = sum(g.n_cells for g in groups)
    K = 10
    f_host = np.concatenate([g.f_ext.ravel() for g in groups])
    stream = torch.cuda.Stream()

    def make(prec):
        s = Solver(precision=prec, stream=stream, force_median=args.force_median, u_max=args.u_max,
                   pbd_kappa=args.pbd_kappa, pik_radius=args.pik_radius, collision_k=args.collision_k)
        for g in groups:
            s.add_cells(s.create_type(g.mtype), g.x0, g.v0)
        return s

    f_dev = torch.from_numpy(f_host).to("cuda")
    s = make(precision)
    ndofs = s.num_dofs

    # ---- device-resident timed region (graph replay); the clock sampler starts
    # before the warm-up so that its start-up is not inside the timed region
    clocks = Clocks(local)
    clocks.start()
    for _ in range(args.warmup):
        s.step(f_dev)
    s.sync()
    # the state the timed steps start from: the end-to-end loop below replays the same steps
    # from it (a restored state steps bitwise like the original), so that both numbers are
    # taken on the same states (later steps of the deforming suspension cost more)
    x_start, v_start = (s.positions(), s.velocities()) if not args.no_e2e else (None, None)
    clocks.lines.clear()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.step(f_dev)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    s.sync()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    value = world * ncells * K * args.steps / t
    st = s.stats()
    launches = st["launches_per_step"] * args.steps
    ci = max(1, st["cell_iterations"])
    solver = {"backtracks_per_cell_iteration": st["backtracks"] / ci,
              "refine_sweeps_per_cell_iteration": st["refine_sweeps"] / ci,
              "max_refine_residual": st["max_refine_residual"], "fallbacks": st["fallbacks"],
              "capped_searches": st["capped_searches"], "of_step": "last timed step"}

    # ---- parity: one step from the state the timed trajectory reached (after
    # warm-up + timed steps, large deformation), on the GPU and in the FP64 oracle
    # from the same positions and velocities, sampled cells.  The step map is what
    # the implementation computes; two trajectories integrated independently drift
    # apart by rounding amplification of the dynamics (~1.16x per step on this
    # workload, the oracle against itself included), so they are not compared.
    total_steps = args.warmup + args.steps
    parity = None
    if rank == 0:
        from oracle import oracle as O
        xn, vn = s.positions(), s.velocities()
        s.step(f_dev)
        s.sync()
        x1 = s.positions()
        contacts = s.stats()["contacts"]
        errs, off = [], 0
        for g, (idx, xo) in zip(groups, oracle_step_sampled(groups, xn, vn, args, K)):
            n = g.n_cells * g.mtype.nV * 3
            shape = (g.n_cells, g.mtype.nV, 3)
            errs.append(float(np.linalg.norm(x1[off:off + n].reshape(shape)[idx] - xo, axis=2).max() / g.mtype.radius))
            off += n
        parity = {"rel_pos_err": max(errs), "sampled_cells": PARITY_CELLS * len(groups),
                  "measure": f"one step from the GPU state after {total_steps} steps, GPU vs FP64 oracle",
                  "tolerance": 1e-6 if precision != "fp64" else 1e-10}
        if args.pik_radius > 0:
            # contacts make the step map less well conditioned: the oracle against itself
            # from the same state perturbed by 1e-13 (absolute, random) shows how much
            rng = np.random.default_rng(0)
            pert = oracle_step_sampled(groups, xn + 1e-13 * rng.standard_normal(xn.shape), vn, args, K)
            base = oracle_step_sampled(groups, xn, vn, args, K)
            parity["contacts_in_step"] = contacts
            parity["oracle_self_sensitivity"] = max(
                float(np.linalg.norm(a[1] - b[1], axis=2).max() / g.mtype.radius)
                for g, a, b in zip(groups, base, pert))

    # ---- per-kernel CUDA-event times (same steps, events around every launch)
    s.profile(True)
    s.step(f_dev)                        # capture + warm
    s.profile_read(reset=True)
    for _ in range(args.steps):
        s.step(f_dev)
    prof = s.profile_read(reset=True)
    s.profile(False)

    # ---- end to end: host forces in, host positions out, through the C ABI
    e2e = None
    if not args.no_e2e:
        f_pin = torch.from_numpy(f_host).pin_memory()
        x_pin = torch.empty(ndofs, dtype=torch.float64).pin_memory()
        fnp, xnp = f_pin.numpy(), x_pin.numpy()
        s.step(fnp)                      # the pinned buffers' first use, untimed
        s.positions(out=xnp)
        s.set_state(x_start, v_start)    # back to the start of the device-timed steps
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.step(fnp)
            s.positions(out=xnp)
        te = max_over_ranks(time.perf_counter() - t0)
        barrier()
        e2e = {"value": world * ncells * K * args.steps / te, "unit": UNIT,
               "h2d_bytes_per_step": ndofs * 8, "d2h_bytes_per_step": ndofs * 8,
               "steps": "the device-timed steps again, from their start state"}

    # ---- immersed-boundary forces on every vertex (a separate measurement): a lattice of
    # spacing 0.5 over the cells' bounding box, a synthetic shear flow with a perturbation
    ibm = None
    if args.ibm_cycles > 0:
        x = s.positions().reshape(-1, 3)
        dx = 0.5
        lo, hi = x.min(axis=0) - 2 * dx, x.max(axis=0) + 2 * dx
        n = np.ceil((hi - lo) / dx).astype(int) + 1
        zz, yy, xx = (torch.arange(int(m), dtype=torch.float64, device="cuda") * dx + float(o)
                      for m, o in zip(n[::-1], lo[::-1]))
        u = torch.zeros((3, int(n[2]), int(n[1]), int(n[0])), dtype=torch.float64, device="cuda")
        u[0] += 1e-3 * (yy - yy.mean())[None, :, None]
        u[1] += 1e-3 * torch.sin(0.1 * xx)[None, None, :]
        u[2] += 1e-3 * torch.cos(0.1 * zz)[:, None, None]
        torch.cuda.synchronize()                 # u is written on torch's stream, read on the solver's
        fl, fg = s.ibm_forces(u, lo, dx, 1e-3, args.ibm_cycles)
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ea.record(stream)
        for _ in range(args.steps):
            s.ibm_forces(u, lo, dx, 1e-3, args.ibm_cycles, fl, fg)
        eb.record(stream)
        torch.cuda.synchronize()
        ti = ea.elapsed_time(eb) / 1e3 / args.steps
        npts = ndofs // 3
        ibm = {"cycles": args.ibm_cycles, "ms_per_call": ti * 1e3, "points": npts,
               "points_per_s": npts / ti, "lattice": [int(v) for v in n], "dx": dx,
               "fields_gb": 2 * 3 * int(np.prod(n)) * 8 / 1e9}
        del u, fl, fg
    s.close()
    del s
    torch.cuda.empty_cache()

    # ---- the plain FP64 GPU form on the same workload
    fp64 = None
    if args.fp64_steps > 0 and precision != "fp64":
        s64 = make("fp64")
        s64.step(f_dev)
        s64.sync()
        barrier()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(args.fp64_steps):
            s64.step(f_dev)
        eb.record(stream)
        torch.cuda.synchronize()
        t64 = max_over_ranks(ea.elapsed_time(eb) / 1e3)
        fp64 = {"value": world * ncells * K * args.fp64_steps / t64, "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": t64 / args.fp64_steps * 1e3}
        if rank == 0 and args.pik_radius > 0:
            # contacts couple the cells: the step map from the FP64 state, sampled cells
            xn, vn = s64.positions(), s64.velocities()
            s64.step(f_dev)
            x = s64.positions()
            errs, off = [], 0
            for g, (idx, xo) in zip(groups, oracle_step_sampled(groups, xn, vn, args, K)):
                n = g.n_cells * g.mtype.nV * 3
                errs.append(float(np.linalg.norm(x[off:off + n].reshape(g.n_cells, g.mtype.nV, 3)[idx] - xo,
                                                 axis=2).max() / g.mtype.radius))
                off += n
            fp64["rel_pos_err"] = max(errs)
            fp64["measure"] = f"one step from the FP64 GPU state after {args.fp64_steps} steps, sampled cells"
            fp64["mixed_over_fp64"] = value / fp64["value"]
        elif rank == 0:
            from oracle import oracle as O
            x = s64.positions()
            errs, off = [], 0
            for g in groups:
                n = g.n_cells * g.mtype.nV * 3
                xg = x[off:off + n].reshape(g.n_cells, g.mtype.nV, 3)
                off += n
                idx = np.array([0, g.n_cells - 1])
                T = O.OracleType.from_mesh_type(g.mtype)
                xo, vo = g.x0[idx].copy(), g.v0[idx].copy()
                fs = O.force_median(T, g.f_ext[idx]) if args.force_median else g.f_ext[idx]
                for _ in range(1 + args.fp64_steps):
                    xo, vo = T.step_cells(xo, vo, fs, K=K, m=5, threads=2)
                    if args.pbd_kappa > 0:
                        vo = O.pbd_damping(T, xo, vo, args.pbd_kappa)
                    if args.u_max > 0:
                        vo = O.velocity_cap(vo, args.u_max)
                errs.append(float(np.linalg.norm(xg[idx] - xo, axis=2).max() / g.mtype.radius))
            fp64["rel_pos_err"] = max(errs)
            fp64["measure"] = f"trajectory of {1 + args.fp64_steps} steps from the initial state, 2 cells per type"
            fp64["mixed_over_fp64"] = value / fp64["value"]
        s64.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (largest share of event time)
    hbm, bf_burst, bf_sust, peak_src = load_peaks()
    names = {k: v for k, v in prof.items()}
    dom = max(names, key=lambda k: names[k][0]) if names else None
    total_ms = sum(v[0] for v in names.values())
    bf16 = precision == "bf16"
    b = 8 if precision == "fp64" else 4
    roof = None
    if dom in ("iterate", "predict"):
        # bytes of one step's k_iterate launches (K per type) / launches per step
        byts = K * sum(algorithmic_bytes_iterate(g.mtype.nV, g.n_cells, K, 5, b, bf16) for g in groups)
        launches_per_step = prof[dom][1] / args.steps
        avg_ms = prof[dom][0] / prof[dom][1]
        per_launch = byts / (launches_per_step if launches_per_step else 1)
        ach = per_launch / (avg_ms / 1e3) / 1e9
        traffic = ITERATE_TRAFFIC if (args.workload == "rbc50k_plt5k" and precision == "bf16") else None
        roof = {"kernel": "k_iterate", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic, "traffic_unit": "bytes per launch",
                "peak_source": peak_src}
    elif dom in ("gemm", "gemm_refine"):
        byts = K * sum(algorithmic_gemm(g.mtype.nV, g.n_cells, bf16)[0] for g in groups)
        launches_per_step = prof[dom][1] / args.steps
        avg_ms = prof[dom][0] / prof[dom][1]
        ach = byts / launches_per_step / (avg_ms / 1e3) / 1e9
        roof = {"kernel": "k_gemm_tc", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None, "peak_source": peak_src}
    kernels = {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / total_ms if total_ms else None}
               for k, v in names.items()}
    # the global step's first apply (grouped tensor-core launch, all types): bytes of its
    # operand streams (read q, write z; P^{-1} stays in L2) and its flops, per launch
    roof_gemm = None
    if "gemm" in prof and precision != "fp64":
        byts = sum(algorithmic_gemm(g.mtype.nV, g.n_cells, bf16)[0] for g in groups)
        flops = sum(algorithmic_gemm(g.mtype.nV, g.n_cells, bf16)[1] for g in groups)
        avg_s = prof["gemm"][0] / prof["gemm"][1] / 1e3
        tpeak = bf_sust if bf16 else bf_sust / 2.0
        roof_gemm = {"kernel": "k_gemm_grouped (first apply)", "bound": "hbm",
                     "achieved_gbs": byts / avg_s / 1e9, "hbm_frac": byts / avg_s / 1e9 / hbm,
                     "achieved_tflops": flops / avg_s / 1e12, "tensor_peak_tflops": tpeak,
                     "tensor_frac": flops / avg_s / 1e12 / tpeak, "ms_per_launch": avg_s * 1e3,
                     "peak_source": peak_src + (" (BF16 sustained)" if bf16 else
                                                " (TF32 = BF16 sustained x nominal 1/2)")}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": precision if precision != "fp64" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "cells": ncells, "rbc_vertices": 642, "plt_vertices": 162,
                       "iters_per_step": K, "history": 5, "precision": precision,
                       "local_step": "fp32" if precision != "fp64" else "fp64",
                       "l2": "inputs larger than L2 (state + forces ~1.6 GB), no flush",
                       "parallelism": f"{world} independent ranks" if world > 1 else "1 GPU",
                       "force_median": bool(args.force_median), "u_max": args.u_max, "pbd_kappa": args.pbd_kappa,
                       "rayleigh_alpha": args.rayleigh_alpha, "rayleigh_beta": args.rayleigh_beta,
                       "pik_radius": args.pik_radius, "collision_k": args.collision_k if args.pik_radius > 0 else 0.0},
            "clocks": clk, "gpu_launches": launches, "parity": parity, "fp64_gpu": fp64, "e2e": e2e,
            "roofline": roof, "roofline_gemm": roof_gemm, "kernels": kernels, "solver": solver}
    if ibm:
        line["ibm"] = ibm
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.workload, alpha=args.rayleigh_alpha, beta=args.rayleigh_beta)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
