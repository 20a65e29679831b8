#!/usr/bin/env python
"""Benchmark of the CGP Poisson path on the 512x256 O-grid (525,312 fine nodes).

One step is one time step of the scale workload: a potential solve (Eq. 12:
restrict + RHS, PCG to 1e-8, prolong, grad phi and j x B) and a pressure
solve (Eq. 15: restrict + RHS, PCG to 1e-8, prolong, grad p), each warm-started
from the previous step's solution, on a synthetic advected vortex train
(B = k, N = 1).  The metric is CGP Poisson solves per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

Under torchrun every rank runs its own replica of the workload on its own GPU
(the solves are independent; there is no collective on the data path), and
rank 0 prints one JSON line with the whole-job rate (sum over ranks of the
solves / max over ranks of the time).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CGP Poisson solves/s at 526k fine nodes to 1e-8 rel resid; SpMV GB/s vs peak"
UNIT = "solves/s"
N_THETA, N_R = 512, 256
TOL = 1e-8
SEED = 1
STUART = 1.0
B_FIELD = (0.0, 0.0, 1.0)
RHO_OVER_DT = 20.0
L2_FLUSH_BYTES = 512 << 20
SPMV_MESH = (3072, 1536)       # matrix + vectors: 490 MB FP64, 320 MB FP32 (L2 is 129 MB)
KERNELS_PER_STEP = 8           # 2 x (restrict_rhs, persistent PCG, prolong, lorentz)
PERM_KERNELS_PER_SOLVE = 2     # gather and scatter around a solve in a renumbered row order


def renumbered(flags, precision):
    """Whether a solve with these tuning flags runs on renumbered rows: coordinate bisection (bit 2), or
    the O-grid tiles of the FP64 single-reduction form (bit 5, the O-grid registered as here)."""
    return bool(flags & 4) or (precision == "fp64" and bool(flags & 32) and not flags & 18)


FP64_PEAK_TFLOPS = 1.25        # nominal dense FP64 of a GB300


def workload_config(precision="fp64"):
    return {"workload": f"CGP potential+pressure step, coarse O-grid {N_THETA}x{N_R} "
                        f"(131,584 coarse / 525,312 fine nodes), advected vortex train, B=k, N=1",
            "coarse_mesh": f"{N_THETA}x{N_R}", "fine_nodes": 525312, "coarse_nodes": 131584,
            "solves_per_step": 2, "tol": TOL, "x0": "previous step", "precision": precision,
            "l2": "flushed between timed steps (512 MiB write)", "seed": SEED}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one persistent
# solver launch, from one ncu capture of `bench.py --profile-case <precision>`
# (the bench's launch shape).  They hold only for the kernel sources they were
# taken on and for the captured launch's tuning flags: when the sources' hash
# or the benchmarked flags differ the traffic is reported as null.
SOLVER_SOURCES = ("cgp_pcg.cu", "cgp_pcg_batch.cu", "cgp_pipe.cu", "cgp_solver.cuh", "cgp_sync.h", "cgp_fixed.h",
                  "cgp_internal.h")
SOLVER_TRAFFIC = {
    "sha256": "bd624dbe15e1ef9e4fd16d5f924229b690a886bbac437062f633aa27336c60dd",
    "fp64": 10377984 + 335616,
    "flags": {"fp64": 40},
}


def solver_traffic(precision, flags=None):
    import hashlib
    h = hashlib.sha256()
    for f in SOLVER_SOURCES:
        with open(os.path.join(ROOT, "paper_2003_00082_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != SOLVER_TRAFFIC["sha256"]:
        return None
    if flags is not None and SOLVER_TRAFFIC["flags"].get(precision) not in (None, flags):
        return None
    return SOLVER_TRAFFIC.get(precision)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes of the persistent PCG launch (FP64 values, int32 indices)
# ---------------------------------------------------------------------------
def spmv_bytes(n, nnz, s=8):
    """CSR y = A x: values + column indices + row pointers + x once + y."""
    return nnz * (s + 4) + 4 * (n + 1) + 2 * s * n


def pcg_iteration_bytes(n, nnz):
    """One FP64 CG iteration as the kernel performs it.

    A: read z, p; write p (24 n).  B: SpMV of p, write q (12 nnz + 4 n + 16 n).
    C: read p, q, x, r, D^-1; write x, r, z (64 n).
    """
    return 12 * nnz + 108 * n


def pcg_launch_bytes(iters, n, nnz):
    """Set-up (means, projection, r0 = b - K x0) + iterations + final projection and true residual."""
    setup = 16 * n + 32 * n + (12 * nnz + 4 * n + 8 * n) + 48 * n
    final = 24 * n + (12 * nnz + 4 * n + 8 * n) + 8 * n
    return setup + iters * pcg_iteration_bytes(n, nnz) + final


def pcg_launch_flops(iters, n, nnz):
    """FP64 flops of the FP64 launch: per iteration 2 nnz (SpMV) + 13 n (updates, D^-1 r, three dots)."""
    return iters * (2 * nnz + 13 * n) + 4 * nnz + 20 * n


def mixed_launch_bytes(inner_iters, sweeps, n, nnz):
    """Mixed launch: per inner FP32 iteration of the single-reduction CG, the FP32 SpMV
    (8 nnz + 4(n+1) + 8 n) and 15 FP32 vector streams (p, s, e, r, u updates, r/w/s published);
    per sweep the FP64 residual SpMV and 6 FP64 vector streams."""
    inner = 8 * nnz + 4 * (n + 1) + 8 * n + 60 * n
    outer = 12 * nnz + 4 * (n + 1) + 16 * n + 48 * n
    return inner_iters * inner + (sweeps + 1) * outer


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def run_mine(args, rank, world, local_rank, refs_path=None):
    import numpy as np
    import torch

    from paper_2003_00082_gb300 import build, cgp, inputs

    build.build()
    cgp.load()
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    xy, tri = inputs.ogrid(N_THETA, N_R)
    mesh = cgp.Mesh(xy, tri)
    cgp.cgp_mesh_set_ogrid(mesh.handle, N_THETA, N_R)   # the O-grid tiles are an autotuner choice
    xy_f, _, _ = mesh.fine_geometry()
    n, nnz = mesh.n_c, mesh.nnz
    W, K = args.warmup, args.steps
    total_steps = W + K
    precision = cgp.CGP_MIXED if args.precision == "mixed" else cgp.CGP_FP64

    # host inputs: one velocity field per time step (pinned for the end-to-end pass)
    U = torch.empty((total_steps, 2, mesh.n_f), dtype=torch.float64).pin_memory()
    for k in range(total_steps):
        u, v = inputs.velocity(xy_f, k, SEED, vortices=True)
        U[k, 0].copy_(torch.from_numpy(u))
        U[k, 1].copy_(torch.from_numpy(v))
    Ud = U.to(dev)

    f64 = dict(dtype=torch.float64, device=dev)
    b = torch.empty(n, **f64)
    phi_c = torch.zeros(n, **f64)
    p_c = torch.zeros(n, **f64)
    phi_f = torch.empty(mesh.n_f, **f64)
    p_f = torch.empty(mesh.n_f, **f64)
    force = torch.empty(2 * mesh.t_f, **f64)
    grad_phi = torch.empty(2 * mesh.t_f, **f64)
    grad_p = torch.empty(2 * mesh.t_f, **f64)
    n_info = 2 * total_steps + 2 * K
    infos = torch.zeros(n_info * cgp.INFO_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    info_addr = lambda slot: infos.data_ptr() + slot * cgp.INFO_BYTES  # noqa: E731

    # launch shapes for this mesh, picked by timing on the first step's potential RHS
    cgp.cgp_restrict(mesh.handle, cgp.CGP_RHS_POTENTIAL, B_FIELD, RHO_OVER_DT, Ud[0, 0], Ud[0, 1], b)
    tune_x = torch.zeros(n, **f64)
    tuned = {}
    for prec in (cgp.CGP_FP64, cgp.CGP_MIXED):
        what = cgp.CGP_TUNE_SOLVE_MIXED if prec == cgp.CGP_MIXED else cgp.CGP_TUNE_SOLVE_FP64
        if args.tuning:   # a fixed launch shape for the benchmarked precision (profiler runs), no autotuning
            if prec == precision:
                cgp.cgp_set_tuning(mesh.handle, what, *args.tuning)
                tuned["mixed" if prec else "fp64"] = dict(cgp.cgp_get_tuning(mesh.handle, what), ms=None)
            continue
        best_ms = cgp.cgp_autotune(mesh.handle, prec, b, tune_x)
        tuned["mixed" if prec else "fp64"] = dict(cgp.cgp_get_tuning(mesh.handle, what), ms=best_ms)
    del tune_x

    solve_events = []

    def step(uf, vf, warm, slot, timing=False, tol=TOL, force=force, grad_p=grad_p):
        prec = precision
        cgp.cgp_restrict(mesh.handle, cgp.CGP_RHS_POTENTIAL, B_FIELD, RHO_OVER_DT, uf, vf, b)
        e0 = torch.cuda.Event(enable_timing=True) if timing else None
        e1 = torch.cuda.Event(enable_timing=True) if timing else None
        if timing:
            e0.record(stream)
        cgp.cgp_poisson_solve_async(mesh.handle, b, phi_c, tol=tol, use_x0=warm, precision=prec,
                                    info_dev=info_addr(slot))
        if timing:
            e1.record(stream)
            solve_events.append((e0, e1))
        cgp.cgp_prolong(mesh.handle, phi_c, phi_f)
        cgp.cgp_lorentz(mesh.handle, phi_f, uf, vf, B_FIELD, STUART, grad_phi, force)
        cgp.cgp_restrict(mesh.handle, cgp.CGP_RHS_PRESSURE, B_FIELD, RHO_OVER_DT, uf, vf, b)
        e2 = torch.cuda.Event(enable_timing=True) if timing else None
        e3 = torch.cuda.Event(enable_timing=True) if timing else None
        if timing:
            e2.record(stream)
        cgp.cgp_poisson_solve_async(mesh.handle, b, p_c, tol=tol, use_x0=warm, precision=prec,
                                    info_dev=info_addr(slot + 1))
        if timing:
            e3.record(stream)
            solve_events.append((e2, e3))
        cgp.cgp_prolong(mesh.handle, p_c, p_f)
        cgp.cgp_lorentz(mesh.handle, p_f, None, None, B_FIELD, STUART, grad_p, None)

    # ---- warm-up ----
    for k in range(W):
        step(Ud[k, 0], Ud[k, 1], k > 0, 2 * k)
    torch.cuda.synchronize()
    phi_keep, p_keep = phi_c.clone(), p_c.clone()

    # ---- timed, inputs resident in HBM ----
    step_events = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clocks:
        for j in range(K):
            k = W + j
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(Ud[k, 0], Ud[k, 1], k > 0, 2 * k, timing=True)
            e1.record(stream)
            step_events.append((e0, e1))
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(c) for a, c in step_events]
    solve_ms = [a.elapsed_time(c) for a, c in solve_events]
    dev_ms = sum(step_ms)

    # ---- end to end: pinned host inputs in, fine-mesh results out, every step ----
    # One interval from the first host->device copy to the last device->host
    # copy.  Step j's velocity comes in on a copy stream while step j - 1
    # computes, and step j's force and grad p go out on another while step
    # j + 1 computes (device buffers alternate between two sets).
    phi_c.copy_(phi_keep)
    p_c.copy_(p_keep)
    out_host = torch.empty((K, 2, 2 * mesh.t_f), dtype=torch.float64).pin_memory()
    in_d = [(torch.empty(mesh.n_f, **f64), torch.empty(mesh.n_f, **f64)) for _ in range(2)]
    out_d = [(torch.empty(2 * mesh.t_f, **f64), torch.empty(2 * mesh.t_f, **f64)) for _ in range(2)]
    h2d_stream, d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()  # noqa: E731
    in_ready = [ev() for _ in range(K)]
    step_done = [ev() for _ in range(K)]
    out_done = [ev() for _ in range(K)]

    def fetch(j):   # inputs of step j into buffer set j % 2, after step j - 2 used that set
        with torch.cuda.stream(h2d_stream):
            if j >= 2:
                h2d_stream.wait_event(step_done[j - 2])
            in_d[j % 2][0].copy_(U[W + j, 0], non_blocking=True)
            in_d[j % 2][1].copy_(U[W + j, 1], non_blocking=True)
            in_ready[j].record(h2d_stream)

    torch.cuda.synchronize()
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    h2d_stream.wait_stream(stream)
    d2h_stream.wait_stream(stream)
    fetch(0)
    for j in range(K):
        k = W + j
        if j + 1 < K:
            fetch(j + 1)
        flush.zero_()
        stream.wait_event(in_ready[j])
        if j >= 2:   # output set j % 2 is free once step j - 2's results are on the host
            stream.wait_event(out_done[j - 2])
        fo, go = out_d[j % 2]
        step(in_d[j % 2][0], in_d[j % 2][1], k > 0, 2 * total_steps + 2 * j, force=fo, grad_p=go)
        step_done[j].record(stream)
        with torch.cuda.stream(d2h_stream):
            d2h_stream.wait_event(step_done[j])
            out_host[j, 0].copy_(fo, non_blocking=True)
            out_host[j, 1].copy_(go, non_blocking=True)
            out_done[j].record(d2h_stream)
    stream.wait_stream(d2h_stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t_begin.elapsed_time(t_end)
    # the last step repeats the last device-timed step from the same state: same bits on the host
    if not (torch.equal(out_host[K - 1, 0], force.cpu()) and torch.equal(out_host[K - 1, 1], grad_p.cpu())):
        raise RuntimeError("end-to-end pass: host results differ from the device-timed pass")
    h2d = 2 * mesh.n_f * 8
    d2h = 2 * 2 * mesh.t_f * 8

    # ---- outcome of every solve ----
    recs = cgp.decode_infos(bytes(infos.cpu().numpy()), n_info)
    timed = recs[2 * W: 2 * total_steps]
    bad = [r for r in recs[: 2 * total_steps] + recs[2 * total_steps:] if r["status"] != cgp.CGP_OK]
    if bad:
        raise RuntimeError(f"{len(bad)} solves did not converge: {bad[:3]}")
    its = [r["iterations"] for r in timed]

    # ---- the same timed steps in the other precision: speed and agreement ----
    other = cgp.CGP_FP64 if precision == cgp.CGP_MIXED else cgp.CGP_MIXED
    alt = {}
    if not args.no_variants:
        phi_c.copy_(phi_keep)
        p_c.copy_(p_keep)
        # fields of the first timed step: a tightly converged FP64 reference (tol 1e-13) and the main precision
        saved_prec = precision
        precision = cgp.CGP_FP64
        phi_c.copy_(phi_keep)
        p_c.copy_(p_keep)
        step(Ud[W, 0], Ud[W, 1], W > 0, 2 * W, tol=1e-13)
        torch.cuda.synchronize()
        tight = [phi_f.clone(), force.clone(), grad_p.clone()]
        precision = saved_prec
        phi_c.copy_(phi_keep)
        p_c.copy_(p_keep)
        step(Ud[W, 0], Ud[W, 1], W > 0, 2 * W)
        torch.cuda.synchronize()
        main_fields = [phi_f.clone(), force.clone(), grad_p.clone()]
        rel = lambda a, r: float(torch.linalg.norm(a - r) / torch.linalg.norm(r))  # noqa: E731
        err_main = {"phi_f": rel(main_fields[0], tight[0]), "force": rel(main_fields[1], tight[1]),
                    "grad_p": rel(main_fields[2], tight[2])}
        phi_c.copy_(phi_keep)
        p_c.copy_(p_keep)
        precision = other
        alt_events = []
        for j in range(K):
            k = W + j
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(Ud[k, 0], Ud[k, 1], k > 0, 2 * k)
            e1.record(stream)
            alt_events.append((e0, e1))
            if j == 0:
                torch.cuda.synchronize()
                alt["rel_err_vs_main"] = {"phi_f": rel(phi_f, main_fields[0]), "force": rel(force, main_fields[1]),
                                          "grad_p": rel(grad_p, main_fields[2])}
                alt["rel_err_vs_tight_fp64"] = {"phi_f": rel(phi_f, tight[0]), "force": rel(force, tight[1]),
                                                "grad_p": rel(grad_p, tight[2])}
                alt["main_rel_err_vs_tight_fp64"] = err_main
        torch.cuda.synchronize()
        alt_ms = sum(a.elapsed_time(c) for a, c in alt_events)
        alt_recs = cgp.decode_infos(bytes(infos.cpu().numpy()), n_info)[2 * W: 2 * total_steps]
        alt.update(precision="mixed" if other == cgp.CGP_MIXED else "fp64", value=2 * K / (alt_ms * 1e-3),
                   ms_per_step=alt_ms / K,
                   inner_iterations_mean=statistics.mean(r["iterations"] for r in alt_recs),
                   sweeps_mean=statistics.mean(r["outer_sweeps"] for r in alt_recs),
                   all_converged=all(r["status"] == cgp.CGP_OK for r in alt_recs),
                   rel_res_true_max=max(r["rel_res_true"] for r in alt_recs))
        precision = saved_prec


    # ---- accuracy against the CPU oracle, and speed at matched accuracy ----
    accuracy = None
    if refs_path and not args.no_variants:
        import numpy as np
        refs = np.load(refs_path)
        R = lambda key: torch.as_tensor(refs[key], **f64)  # noqa: E731
        soa = lambda key: torch.as_tensor(np.ascontiguousarray(refs[key].T).ravel(), **f64)  # noqa: E731
        relt = lambda a, r: float(torch.linalg.norm(a - r) / torch.linalg.norm(r))  # noqa: E731
        saved_prec = precision
        accuracy = {"workload": "time step 1 of the 512x256 workload (potential + pressure), step 0 from x0 = 0 at "
                                "tol 1e-8, step 1 from each side's own step-0 solution",
                    "reference": "CPU FP64 oracle (computed by the cpu_baseline leg): the same step at the same "
                                 "tolerance, and converged (tol 1e-13 from the 2e-9 solution)",
                    "gates": {"phi": 1e-8, "force": 1e-6}}
        for name, prec in (("fp64", cgp.CGP_FP64), ("mixed", cgp.CGP_MIXED)):
            precision = prec
            for tol in ACC_TOLS:
                phi_c.zero_()
                p_c.zero_()
                step(Ud[0, 0], Ud[0, 1], False, 0, tol=TOL)
                step(Ud[1, 0], Ud[1, 1], True, 0, tol=tol)
                torch.cuda.synchronize()
                e = {}
                for ref in (f"{tol:g}", "converged"):
                    e["vs_oracle_" + ("same_tol" if ref != "converged" else "converged")] = {
                        "phi_f": relt(phi_f, R(f"c2/0/{ref}/phi_f")),
                        "grad_phi": relt(grad_phi, soa(f"c2/0/{ref}/grad")),
                        "force": relt(force, soa(f"c2/0/{ref}/force")),
                        "p_f": relt(p_f, R(f"c2/1/{ref}/phi_f")),
                        "grad_p": relt(grad_p, soa(f"c2/1/{ref}/grad"))}
                c = e["vs_oracle_converged"]
                e["meets_gates_vs_converged"] = c["phi_f"] <= 1e-8 and c["p_f"] <= 1e-8 and c["force"] <= 1e-6
                accuracy.setdefault(name, {})[f"tol_{tol:g}"] = e
        # speed of both precisions at the tolerance where both meet the gates against the converged answer
        tol_acc = ACC_TOLS[-1]
        matched = {"tol": tol_acc}
        for name, prec in (("fp64", cgp.CGP_FP64), ("mixed", cgp.CGP_MIXED)):
            precision = prec
            phi_c.copy_(phi_keep)
            p_c.copy_(p_keep)
            ev_acc = []
            for j in range(K):
                k = W + j
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step(Ud[k, 0], Ud[k, 1], k > 0, 2 * k, tol=tol_acc)
                e1.record(stream)
                ev_acc.append((e0, e1))
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(c) for a, c in ev_acc)
            acc_recs = cgp.decode_infos(bytes(infos.cpu().numpy()), n_info)[2 * W: 2 * total_steps]
            matched[name] = {"solves_per_s": 2 * K / (ms * 1e-3), "ms_per_step": ms / K,
                             "iterations_mean": statistics.mean(r["iterations"] for r in acc_recs),
                             "all_converged": all(r["status"] == cgp.CGP_OK for r in acc_recs)}
        matched["speedup_mixed_over_fp64"] = matched["mixed"]["solves_per_s"] / matched["fp64"]["solves_per_s"]
        accuracy["matched_accuracy"] = matched
        accuracy["at_benchmark_tol"] = (
            "at tol 1e-8 the J x B error against the converged answer is about 2.5e-6 to 3e-6 for every "
            "solver (the oracle's own included): the 1e-6 gate holds there only between solves that follow "
            "the same Krylov path (GPU FP64 against oracle FP64); at 2e-9 both precisions meet it")
        precision = saved_prec

    # ---- roofline of the dominant kernel (the persistent PCG launch) ----
    peak, peak_kind = read_peaks()
    if precision == cgp.CGP_FP64:
        alg_bytes = [pcg_launch_bytes(r["iterations"], n, nnz) for r in timed]
    else:
        alg_bytes = [mixed_launch_bytes(r["iterations"], r["outer_sweeps"], n, nnz) for r in timed]
    fp64_flops = sum(pcg_launch_flops(r["iterations"], n, nnz) for r in timed) if precision == cgp.CGP_FP64 else 0
    pcg_total_ms = sum(solve_ms)
    achieved = sum(alg_bytes) / (pcg_total_ms * 1e-3) / 1e9

    result = dict(dev_ms=dev_ms, e2e_ms=e2e_ms, solves=2 * K, step_ms=step_ms, solve_ms=solve_ms, its=its,
                  achieved=achieved, alg_bytes_per_launch=sum(alg_bytes) / len(alg_bytes),
                  fp64_tflops=fp64_flops / (pcg_total_ms * 1e-3) / 1e12, tuned=tuned, variant=alt,
                  pcg_share=pcg_total_ms / dev_ms, clocks=clocks.summary(), peak=peak, peak_kind=peak_kind,
                  h2d=h2d, d2h=d2h, n=n, nnz=nnz, accuracy=accuracy,
                  rel_res_true_max=max(r["rel_res_true"] for r in timed))

    if rank == 0 and not args.no_spmv:
        result["spmv"] = spmv_bench(cgp, inputs, torch, dev, peak)
    if rank == 0 and not args.no_variants:
        from paper_2003_00082_gb300 import configs
        result["mixed_64x32"] = run_mixed_small(cgp, inputs, torch, dev, refs_path=refs_path)
        result["levels"] = run_levels(cgp, inputs, torch, dev, flush)
        result["far_field"] = run_far_field(cgp, inputs, torch, dev, flush)
        result["batched"] = run_batched(cgp, inputs, configs, torch, dev, flush, peak)
        result["learned_guess"] = run_learned_guess(cgp, inputs, torch)
        result["learned_guess_512x256"] = run_learned_guess_c2(cgp, inputs, torch)
    mesh.close()
    return result


def run_batched(cgp, inputs, configs, torch, dev, flush, peak, reps=5, tuning=None):
    """64 uneven CGP potential solves (n_theta in {64,...,512}), mixed precision, in the batched persistent
    solver (wave-scheduled launches or one packed launch, as its autotuner picks, or the shape `tuning` =
    (block, lanes, blocks_per_sm, flags) fixes) replayed from a CUDA graph."""
    insts = configs.batched_instances()
    meshes, bs, xs = [], [], []
    for inst in insts:
        xy, tri = inputs.ogrid(inst["n_theta"], inst["n_r"])
        m = cgp.Mesh(xy, tri)
        xy_f, _, _ = m.fine_geometry()
        u, v = inputs.velocity(xy_f, 0, inst["seed"], vortices=True)
        b = torch.empty(m.n_c, dtype=torch.float64, device=dev)
        cgp.cgp_restrict(m.handle, cgp.CGP_RHS_POTENTIAL, inst["B"], RHO_OVER_DT, torch.as_tensor(u, device=dev),
                         torch.as_tensor(v, device=dev), b)
        meshes.append(m)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    batch = cgp.Batch(meshes, bs, xs, tol=TOL, precision=cgp.CGP_MIXED, inner_tol=1e-4)
    if tuning is None:
        tune_ms = batch.autotune()
    else:
        batch.set_tuning(*tuning)
        tune_ms = None
    # capture the launch once; replays need no host work
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        batch.solve()
    times, lat, infos = [], [], None
    for r in range(reps + 1):
        for x in xs:
            x.zero_()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        infos, secs = batch.info()
        if r > 0:
            times.append(e0.elapsed_time(e1))
            lat.extend(secs)
    ms = statistics.median(times)
    lat_ms = sorted(1e3 * t for t in lat)
    pct = lambda q: lat_ms[min(len(lat_ms) - 1, int(round(q * (len(lat_ms) - 1))))]  # noqa: E731
    alg = sum(mixed_launch_bytes(i["iterations"], i["outer_sweeps"], m.n_c, m.nnz) for i, m in zip(infos, meshes))
    q = batch.query()
    out = {"workload": "64 CGP potential solves, coarse O-grids n_theta ~ U{64,128,256,512} (n_r = n_theta/2), "
                       "N ~ U[0.5,5], B = (cos a, sin a, 1), batched persistent launches (autotuned schedule) replayed from a CUDA graph",
           "instances": len(meshes), "coarse_rows_total": sum(m.n_c for m in meshes),
           "fine_nodes_total": sum(m.n_f for m in meshes), "precision": "fp32 inner + fp64 refinement",
           "tol": TOL, "value": len(meshes) / (ms * 1e-3), "unit": "solves/s", "ms_per_batch": ms,
           "latency_ms_p50": pct(0.5), "latency_ms_p99": pct(0.99),
           "all_converged": all(i["status"] == cgp.CGP_OK for i in infos),
           "rel_res_true_max": max(i["rel_res_true"] for i in infos),
           "inner_iterations_max": max(i["iterations"] for i in infos),
           "hbm": {"achieved_gb_s": alg / (ms * 1e-3) / 1e9, "frac": alg / (ms * 1e-3) / 1e9 / peak,
                   "alg_bytes": alg},
           "launch": {"grid": q["grid"], "block": q["block"], "lanes": q["lanes"], "resident": q["resident"]},
           "autotune_best_ms": tune_ms}
    batch.close()
    for m in meshes:
        m.close()
    return out


def run_levels(cgp, inputs, torch, dev, flush, steps=10, warm=3):
    """The c2 step (potential + pressure, vortex train, B = k, N = 1, tol 1e-8, previous-step x0)
    on the same 525,312-node fine mesh size reached with k = 2 and k = 3 coarsening levels
    (coarse 256x128 and 128x64 O-grids): CGP solves/s as the coarse system shrinks (Eq. 18)."""
    out = {"workload": "c2 potential+pressure steps, fine mesh 525,312 nodes from a 512/2^(k-1) x 256/2^(k-1) "
                       "coarse O-grid split k times; FP64, autotuned launch; L2 flushed between steps"}
    f64 = dict(dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for k in (2, 3):
        nt, nr = N_THETA >> (k - 1), N_R >> (k - 1)
        xy, tri = inputs.ogrid(nt, nr)
        m = cgp.Mesh(xy, tri, k)
        cgp.cgp_mesh_set_ogrid(m.handle, nt, nr)
        xy_f, _, _ = m.fine_geometry()
        n = m.n_c
        b = torch.empty(n, **f64)
        phi_c, p_c = torch.zeros(n, **f64), torch.zeros(n, **f64)
        phi_f, p_f = torch.empty(m.n_f, **f64), torch.empty(m.n_f, **f64)
        grad_phi, force, grad_p = (torch.empty(2 * m.t_f, **f64) for _ in range(3))
        U = []
        for t in range(warm + steps):
            u, v = inputs.velocity(xy_f, t, SEED, vortices=True)
            U.append((torch.as_tensor(u, device=dev), torch.as_tensor(v, device=dev)))
        cgp.cgp_restrict(m.handle, cgp.CGP_RHS_POTENTIAL, B_FIELD, RHO_OVER_DT, U[0][0], U[0][1], b)
        tune_x = torch.zeros(n, **f64)
        cgp.cgp_autotune(m.handle, cgp.CGP_FP64, b, tune_x)
        infos = torch.zeros(2 * (warm + steps) * cgp.INFO_BYTES, dtype=torch.uint8, device=dev)
        ev = []
        for t in range(warm + steps):
            uf, vf = U[t]
            if t >= warm:
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            cgp.cgp_restrict(m.handle, cgp.CGP_RHS_POTENTIAL, B_FIELD, RHO_OVER_DT, uf, vf, b)
            cgp.cgp_poisson_solve_async(m.handle, b, phi_c, tol=TOL, use_x0=t > 0,
                                        info_dev=infos.data_ptr() + 2 * t * cgp.INFO_BYTES)
            cgp.cgp_prolong(m.handle, phi_c, phi_f)
            cgp.cgp_lorentz(m.handle, phi_f, uf, vf, B_FIELD, STUART, grad_phi, force)
            cgp.cgp_restrict(m.handle, cgp.CGP_RHS_PRESSURE, B_FIELD, RHO_OVER_DT, uf, vf, b)
            cgp.cgp_poisson_solve_async(m.handle, b, p_c, tol=TOL, use_x0=t > 0,
                                        info_dev=infos.data_ptr() + (2 * t + 1) * cgp.INFO_BYTES)
            cgp.cgp_prolong(m.handle, p_c, p_f)
            cgp.cgp_lorentz(m.handle, p_f, None, None, B_FIELD, STUART, grad_p, None)
            if t >= warm:
                e1.record(stream)
                ev.append((e0, e1))
        torch.cuda.synchronize()
        recs = cgp.decode_infos(bytes(infos.cpu().numpy()), 2 * (warm + steps))[2 * warm:]
        ms = sum(a.elapsed_time(c) for a, c in ev)
        out[f"k{k}"] = {"coarse_mesh": f"{nt}x{nr}", "coarse_nodes": n, "fine_nodes": m.n_f,
                        "solves_per_s": 2 * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                        "iterations_mean": statistics.mean(r["iterations"] for r in recs),
                        "all_converged": all(r["status"] == cgp.CGP_OK for r in recs),
                        "rel_res_true_max": max(r["rel_res_true"] for r in recs),
                        "launch": cgp.cgp_last_launch(m.handle)}
        m.close()
    return out


def run_far_field(cgp, inputs, torch, dev, flush, steps=8, warm=3):
    """c2 potential solves (512x256, vortex train, B = k, tol 1e-8, previous-step x0) with the
    natural condition everywhere and with phi = 0 on the outer boundary: iterations and solves/s."""
    xy, tri = inputs.ogrid(N_THETA, N_R)
    m = cgp.Mesh(xy, tri)
    cgp.cgp_mesh_set_ogrid(m.handle, N_THETA, N_R)
    xy_f, _, _ = m.fine_geometry()
    f64 = dict(dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    U = []
    for t in range(warm + steps):
        u, v = inputs.velocity(xy_f, t, SEED, vortices=True)
        U.append((torch.as_tensor(u, device=dev), torch.as_tensor(v, device=dev)))
    B = torch.empty((warm + steps, m.n_c), **f64)
    for t in range(warm + steps):
        cgp.cgp_restrict(m.handle, cgp.CGP_RHS_POTENTIAL, B_FIELD, RHO_OVER_DT, U[t][0], U[t][1], B[t])
    out = {"workload": "512x256 potential solves, vortex train, B = k, tol 1e-8, previous-step x0"}
    for name, mode in (("natural", 0), ("dirichlet_far", 1)):
        cgp.cgp_set_far_field(m.handle, mode)
        x = torch.zeros(m.n_c, **f64)
        cgp.cgp_autotune(m.handle, cgp.CGP_FP64, B[0], x)
        x.zero_()
        infos = torch.zeros((warm + steps) * cgp.INFO_BYTES, dtype=torch.uint8, device=dev)
        ms = 0.0
        for t in range(warm + steps):
            if t >= warm:
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            cgp.cgp_poisson_solve_async(m.handle, B[t], x, tol=TOL, use_x0=t > 0,
                                        info_dev=infos.data_ptr() + t * cgp.INFO_BYTES)
            if t >= warm:
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        recs = cgp.decode_infos(bytes(infos.cpu().numpy()), warm + steps)[warm:]
        out[name] = {"solves_per_s": steps / (ms * 1e-3),
                     "iterations_mean": statistics.mean(r["iterations"] for r in recs),
                     "all_converged": all(r["status"] == cgp.CGP_OK for r in recs)}
    cgp.cgp_set_far_field(m.handle, 0)
    m.close()
    return out


def run_mixed_small(cgp, inputs, torch, dev, steps=200, check_every=10, refs_path=None):
    """Mixed precision on the 64x32 vortex-train sequence with noise (B = k, tol 1e-8, inner 1e-4,
    previous-step x0): solves/s of FP64 and mixed over the same potential steps, and the relative
    L2 errors of phi_f, grad phi and J x B of both against tightly converged FP64 (tol 1e-13)."""
    from paper_2003_00082_gb300 import configs
    wl = configs.C3_MIXED
    xy, tri = inputs.ogrid(wl.n_theta, wl.n_r)
    m = cgp.Mesh(xy, tri)
    cgp.cgp_mesh_set_ogrid(m.handle, wl.n_theta, wl.n_r)
    xy_f, _, _ = m.fine_geometry()
    f64 = dict(dtype=torch.float64, device=dev)
    n, nf, tf = m.n_c, m.n_f, m.t_f
    U = torch.empty((steps, 2, nf), **f64)
    for t in range(steps):
        u, v = inputs.velocity(xy_f, t, wl.seed, vortices=True, noise_std=wl.noise_std)
        U[t, 0].copy_(torch.as_tensor(u))
        U[t, 1].copy_(torch.as_tensor(v))
    b = torch.empty((steps, n), **f64)
    for t in range(steps):
        cgp.cgp_restrict(m.handle, cgp.CGP_RHS_POTENTIAL, wl.B, wl.rho_over_dt, U[t, 0], U[t, 1], b[t])
    stream = torch.cuda.current_stream()
    infos = torch.zeros(steps * cgp.INFO_BYTES, dtype=torch.uint8, device=dev)

    def fields(phi_c, t):
        phi_f = torch.empty(nf, **f64)
        grad = torch.empty(2 * tf, **f64)
        force = torch.empty(2 * tf, **f64)
        cgp.cgp_prolong(m.handle, phi_c, phi_f)
        cgp.cgp_lorentz(m.handle, phi_f, U[t, 0], U[t, 1], wl.B, wl.sigma, grad, force)
        return phi_f, grad, force

    out = {"workload": "64x32 O-grid potential steps, vortex train + noise 1e-3, B = k, tol 1e-8, previous-step x0",
           "steps": steps}
    sols = {}
    for name, prec in (("fp64", cgp.CGP_FP64), ("mixed", cgp.CGP_MIXED)):
        x = torch.zeros(n, **f64)
        phis = torch.empty((steps, n), **f64)
        cgp.cgp_autotune(m.handle, prec, b[0], x)   # each precision in its own best launch shape
        out.setdefault("tuned_launch", {})[name] = cgp.cgp_get_tuning(
            m.handle, cgp.CGP_TUNE_SOLVE_MIXED if prec == cgp.CGP_MIXED else cgp.CGP_TUNE_SOLVE_FP64)
        x.zero_()
        for t in range(3):   # warm-up on the first steps
            cgp.cgp_poisson_solve(m.handle, b[t], x, tol=wl.tol, precision=prec, inner_tol=wl.inner_tol,
                                  use_x0=t > 0, info=False)
        x.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(steps):
            cgp.cgp_poisson_solve_async(m.handle, b[t], x, tol=wl.tol, precision=prec, inner_tol=wl.inner_tol,
                                        use_x0=t > 0, info_dev=infos.data_ptr() + t * cgp.INFO_BYTES)
            phis[t].copy_(x)
        e1.record(stream)
        torch.cuda.synchronize()
        recs = cgp.decode_infos(bytes(infos.cpu().numpy()), steps)
        ms = e0.elapsed_time(e1)
        out[name] = {"solves_per_s": steps / (ms * 1e-3), "ms_per_solve": ms / steps,
                     "iterations_mean": statistics.mean(r["iterations"] for r in recs),
                     "all_converged": all(r["status"] == cgp.CGP_OK for r in recs),
                     "rel_res_true_max": max(r["rel_res_true"] for r in recs)}
        sols[name] = phis
    rel = lambda a, c: float(torch.linalg.norm(a - c) / torch.linalg.norm(c))  # noqa: E731
    worst = {k: {"phi_f": 0.0, "grad_phi": 0.0, "force": 0.0} for k in ("fp64", "mixed")}
    xt = torch.zeros(n, **f64)
    for t in range(0, steps, check_every):
        xt.zero_()
        cgp.cgp_poisson_solve(m.handle, b[t], xt, tol=1e-13, max_it=100000)
        ref = fields(xt, t)
        for k in ("fp64", "mixed"):
            got = fields(sols[k][t], t)
            for name, g, r in zip(("phi_f", "grad_phi", "force"), got, ref):
                worst[k][name] = max(worst[k][name], rel(g, r))
    out["rel_err_vs_tight_fp64"] = worst
    if refs_path:   # against the CPU FP64 oracle run over the same sequence (every 10th step)
        import numpy as np
        refs = np.load(refs_path)
        f64r = lambda a: torch.as_tensor(a, **f64)  # noqa: E731
        soa = lambda a: torch.as_tensor(np.ascontiguousarray(a.T).ravel(), **f64)  # noqa: E731
        for ref in ("fp64", "converged"):
            w = {k: {"phi_f": 0.0, "grad_phi": 0.0, "force": 0.0} for k in ("fp64", "mixed")}
            for t in range(0, steps, 10):
                r = (f64r(refs[f"c3/{t}/{ref}/phi_f"]), soa(refs[f"c3/{t}/{ref}/grad"]),
                     soa(refs[f"c3/{t}/{ref}/force"]))
                for k in ("fp64", "mixed"):
                    got = fields(sols[k][t], t)
                    for name, g, rr in zip(("phi_f", "grad_phi", "force"), got, r):
                        w[k][name] = max(w[k][name], rel(g, rr))
            out["rel_err_vs_oracle_" + ("same_tol" if ref == "fp64" else "converged")] = w
    out["speedup_mixed_over_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    m.close()
    return out


def run_learned_guess(cgp, inputs, torch):
    """Learned initial guess on the 64x32 mesh: train on 4 N x 5 seeds x 200 steps, test N = 3 on seeds 100-104."""
    from paper_2003_00082_gb300 import learned_guess as LG
    xy, tri = inputs.ogrid(64, 32)
    m = cgp.Mesh(xy, tri)
    xy_f, _, _ = m.fine_geometry()
    net, ev = LG.run_protocol(torch, m, xy_f)
    # both arms again with the solver launch cgp_autotune picks for this mesh (O-grid registered)
    cgp.cgp_mesh_set_ogrid(m.handle, 64, 32)
    u, v = inputs.velocity(xy_f, 0, 100, vortices=True, noise_std=1e-3)
    b = torch.empty(m.n_c, dtype=torch.float64, device="cuda")
    cgp.cgp_restrict(m.handle, cgp.CGP_RHS_POTENTIAL, (0.0, 0.0, 1.0), 20.0, torch.as_tensor(u, device="cuda"),
                     torch.as_tensor(v, device="cuda"), b)
    cgp.cgp_autotune(m.handle, cgp.CGP_FP64, b, torch.zeros_like(b))
    ev2 = LG.evaluate(torch, m, net, xy_f, (100, 101, 102, 103, 104), 200, noise_std=1e-3)
    ev["autotuned_launch"] = {k: ev2[k] for k in ("baseline_iterations_mean", "learned_iterations_mean",
                                                  "baseline_solves_per_s", "learned_solves_per_s")}
    ev["autotuned_launch"]["launch"] = cgp.cgp_get_tuning(m.handle, cgp.CGP_TUNE_SOLVE_FP64)
    net.close()
    m.close()
    ev["workload"] = ("64x32 O-grid potential solves, vortex train + noise 1e-3, tol 1e-8; train N in {0.5,1,2,5} "
                      "x seeds 0-4 x 200 steps, test N = 3 seeds 100-104 x 200 steps; both arms in the mesh's "
                      "default solver launch, and again in the launch cgp_autotune picks (autotuned_launch)")
    return ev


def run_learned_guess_c2(cgp, inputs, torch):
    """The learned guess on the benchmark's own 512x256 sequence (vortex train, no noise): trained on
    3 seeds x 100 steps of potential solves, evaluated on held-out seed 100 (40 steps) against the
    previous-step guess at the same 1e-8 tolerance, solves timed on the device."""
    from paper_2003_00082_gb300 import learned_guess as LG
    xy, tri = inputs.ogrid(N_THETA, N_R)
    m = cgp.Mesh(xy, tri)
    xy_f, _, _ = m.fine_geometry()
    net, ev = LG.run_protocol(torch, m, xy_f, train_seeds=(0, 1, 2), train_stuart=(1.0,), steps=100,
                              test_seeds=(100,), test_steps=40, iterations=(300, 150), batch=2, noise_std=0.0)
    net.close()
    m.close()
    ev["workload"] = ("512x256 O-grid potential solves, vortex train without noise, B = k, tol 1e-8; train seeds "
                      "0-2 x 100 steps, batch 2, 450 Adam steps; test seed 100 x 40 steps")
    return ev


def spmv_bench(cgp, inputs, torch, dev, peak, reps=20):
    """SpMV y = K x on a matrix several times larger than L2, every lanes-per-row choice, FP64 and FP32.

    Launches run back to back between one pair of events (the streamed matrix
    is 2.5-4x the L2, so nothing of it survives from one launch to the next);
    the figure is the mean per launch.  No L2 flush: a flush by writes leaves
    dirty lines whose write-back would be charged to the SpMV."""
    xy, tri = inputs.ogrid(*SPMV_MESH)
    m = cgp.Mesh(xy, tri)
    n, nnz = m.n_c, m.nnz
    out = {"matrix": f"P1 Laplacian of a {SPMV_MESH[0]}x{SPMV_MESH[1]} O-grid", "n": n, "nnz": nnz,
           "timing": f"mean of {reps} back-to-back launches, matrix larger than L2, no flush"}
    for prec, dt, s, what in ((cgp.CGP_FP64, torch.float64, 8, cgp.CGP_TUNE_SPMV_FP64),
                              (cgp.CGP_FP32, torch.float32, 4, cgp.CGP_TUNE_SPMV_FP32)):
        x = torch.randn(n, dtype=dt, device=dev)
        y = torch.empty(n, dtype=dt, device=dev)
        bytes_ = spmv_bytes(n, nnz, s)
        per = {}
        for lanes in (1, 2, 4, 8, 32):
            cgp.cgp_set_tuning(m.handle, what, 256, lanes, 0)
            for _ in range(3):
                cgp.cgp_spmv(m.handle, prec, x, y)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                cgp.cgp_spmv(m.handle, prec, x, y)
            e1.record()
            torch.cuda.synchronize()
            per[lanes] = e0.elapsed_time(e1) / reps
        best = min(per, key=per.get)
        cgp.cgp_set_tuning(m.handle, what, 256, best, 0)
        gbs = bytes_ / (per[best] * 1e-3) / 1e9
        key = "fp64" if prec == cgp.CGP_FP64 else "fp32"
        out[key] = {"best_lanes": best, "ms": per[best], "gb_s": gbs, "frac": gbs / peak,
                    "bytes": bytes_, "ms_by_lanes": per}
    # the O-grid stencil form of the same matrix: seven value planes, no indices (9 s n bytes)
    cgp.cgp_mesh_set_ogrid(m.handle, *SPMV_MESH)
    out["stencil"] = {"format": "7 value planes at fixed O-grid offsets, no column indices; bytes 9 s n"}
    for prec, dt, s_, what in ((cgp.CGP_FP64, torch.float64, 8, cgp.CGP_TUNE_SPMV_FP64),
                               (cgp.CGP_FP32, torch.float32, 4, cgp.CGP_TUNE_SPMV_FP32)):
        x = torch.randn(n, dtype=dt, device=dev)
        y = torch.empty(n, dtype=dt, device=dev)
        cgp.cgp_set_tuning(m.handle, what, 256, 0, 0, 1)
        for _ in range(3):
            cgp.cgp_spmv(m.handle, prec, x, y)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            cgp.cgp_spmv(m.handle, prec, x, y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        key = "fp64" if prec == cgp.CGP_FP64 else "fp32"
        bytes_ = 9 * s_ * n
        out["stencil"][key] = {"ms": ms, "gb_s": bytes_ / (ms * 1e-3) / 1e9, "frac": bytes_ / (ms * 1e-3) / 1e9 / peak,
                               "bytes": bytes_, "speedup_vs_csr": out[key]["ms"] / ms}
        cgp.cgp_set_tuning(m.handle, what, 0, 0, 0, 0)
    m.close()
    return out


# ---------------------------------------------------------------------------
# the CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def _oracle_mesh():
    from oracle import cgp_oracle as O
    from paper_2003_00082_gb300 import inputs
    xy, tri = inputs.ogrid(N_THETA, N_R)
    return O, inputs, O.OracleMesh(xy, tri)


def _oracle_time_step(O, om, u, v, x_phi, x_p, tol=TOL):
    """One time step of the workload: the potential and the pressure solve, each from its previous solution."""
    t0 = time.perf_counter()
    r1 = om.solve(u, v, O.POTENTIAL, B=B_FIELD, sigma=STUART, rho_over_dt=RHO_OVER_DT, tol=tol, x0=x_phi)
    r2 = om.solve(u, v, O.PRESSURE, B=B_FIELD, sigma=STUART, rho_over_dt=RHO_OVER_DT, tol=tol, x0=x_p)
    secs = time.perf_counter() - t0
    assert r1["status"] == O.OK and r2["status"] == O.OK
    return r1, r2, secs


def oracle_sample(refs_path=None, warm_steps=1):
    """Time the oracle as it stands on the 512x256 workload: one warm time step (2 solves) after
    `warm_steps` untimed ones.  With refs_path, afterwards (untimed) write the oracle's fields for
    the accuracy report (oracle_reference_fields)."""
    O, inputs, om = _oracle_mesh()
    x_phi = x_p = None
    for k in range(warm_steps + 1):
        u, v = inputs.velocity(om.xy_f, k, SEED, vortices=True)
        r1, r2, secs = _oracle_time_step(O, om, u, v, x_phi, x_p)
        if k < warm_steps:
            prev = (r1["phi_c"], r2["phi_c"])
        x_phi, x_p = r1["phi_c"], r2["phi_c"]
    out = {"value": 2.0 / secs, "seconds": secs, "iterations": [r1["iterations"], r2["iterations"]]}
    if refs_path:
        oracle_reference_fields(O, inputs, om, warm_steps, prev, (r1, r2), refs_path)
    return out


ACC_TOLS = (TOL, 2e-9)     # the benchmark tolerance, and one at which J x B meets 1e-6 against the converged answer


def oracle_reference_fields(O, inputs, om, step, prev, at_tol, path):
    """The oracle's fields for the accuracy report, written to an .npz (untimed).

    512x256 workload, time step `step` from the oracle's own previous-step
    solutions `prev`: phi_f, grad and (potential) the force at each tolerance
    of ACC_TOLS and converged (tol 1e-13 from the tightest, at most 3000
    iterations).  Mixed-precision workload (64x32, 200 noisy steps, previous-step
    x0): every 10th step's fields from the FP64 oracle at tol 1e-8 and converged."""
    import numpy as np
    from paper_2003_00082_gb300 import configs
    u, v = inputs.velocity(om.xy_f, step, SEED, vortices=True)
    arrays = {}

    def put(key, phi_c, kind):
        phi_f = om.prolong(phi_c)
        grad, force = O.lorentz(om.xy_f, om.tri_f, phi_f, u, v, B_FIELD, STUART)
        arrays[key + "/phi_f"] = phi_f
        arrays[key + "/grad"] = grad
        if kind == O.POTENTIAL:
            arrays[key + "/force"] = force

    for kind, x0, r in ((O.POTENTIAL, prev[0], at_tol[0]), (O.PRESSURE, prev[1], at_tol[1])):
        last = None
        for tol in ACC_TOLS:
            if tol != TOL:
                r = om.solve(u, v, kind, B=B_FIELD, sigma=STUART, rho_over_dt=RHO_OVER_DT, tol=tol, x0=x0)
            put(f"c2/{kind}/{tol:g}", r["phi_c"], kind)
            last = r
        conv = O.pcg(om.K, om.d, last["b"], x0=last["phi_c"], tol=1e-13, max_it=3000)
        put(f"c2/{kind}/converged", conv["x"], kind)
    # the mixed-precision workload on the 64x32 mesh
    wl = configs.C3_MIXED
    xy, tri = inputs.ogrid(wl.n_theta, wl.n_r)
    sm = O.OracleMesh(xy, tri)
    x = None
    for t in range(200):
        u, v = inputs.velocity(sm.xy_f, t, wl.seed, vortices=True, noise_std=wl.noise_std)
        r = sm.solve(u, v, O.POTENTIAL, B=wl.B, sigma=wl.sigma, rho_over_dt=wl.rho_over_dt, tol=wl.tol, x0=x)
        x = r["phi_c"]
        if t % 10 == 0:
            conv = O.pcg(sm.K, sm.d, r["b"], x0=x, tol=1e-13, max_it=20000)["x"]
            for key, phi_c in ((f"c3/{t}/fp64", x), (f"c3/{t}/converged", conv)):
                phi_f = sm.prolong(phi_c)
                grad, force = O.lorentz(sm.xy_f, sm.tri_f, phi_f, u, v, wl.B, wl.sigma)
                arrays[key + "/phi_f"] = phi_f
                arrays[key + "/grad"] = grad
                arrays[key + "/force"] = force
    np.savez(path, **arrays)


def _oracle_worker(idx, warm_steps, timed_steps, barrier, queue):
    """One process of the all-cores oracle timing: untimed warm steps, a barrier so that every
    process times the same interval, then `timed_steps` time steps (2 solves each)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    try:
        O, inputs, om = _oracle_mesh()
        x_phi = x_p = None
        vel = [inputs.velocity(om.xy_f, k, SEED, vortices=True) for k in range(warm_steps + timed_steps)]
        for k in range(warm_steps):
            r1, r2, _ = _oracle_time_step(O, om, vel[k][0], vel[k][1], x_phi, x_p)
            x_phi, x_p = r1["phi_c"], r2["phi_c"]
        barrier.wait(timeout=1800)
        t0 = time.perf_counter()
        for k in range(warm_steps, warm_steps + timed_steps):
            r1, r2, _ = _oracle_time_step(O, om, vel[k][0], vel[k][1], x_phi, x_p)
            x_phi, x_p = r1["phi_c"], r2["phi_c"]
        queue.put((idx, time.perf_counter() - t0, None))
    except Exception as e:   # reported by the parent
        try:
            barrier.abort()
        except Exception:
            pass
        queue.put((idx, None, repr(e)))


def oracle_all_cores(procs, warm_steps, timed_steps):
    """The oracle on `procs` host cores at once: one single-threaded process per core, each running
    the workload's time steps, all timing the same interval.  Returns (aggregate solves/s, wall s)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")   # no fork: the parent may already hold a CUDA context
    barrier = ctx.Barrier(procs)
    queue = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(i, warm_steps, timed_steps, barrier, queue), daemon=True)
          for i in range(procs)]
    for p in ps:
        p.start()
    res = [queue.get(timeout=3600) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    errs = [e for _, _, e in res if e]
    if errs:
        raise RuntimeError(f"oracle process failed: {errs[0]}")
    wall = max(t for _, t, _ in res)
    return procs * 2 * timed_steps / wall, wall


def replica_totals(dev_ms, e2e_ms, solves, world, device="cpu"):
    """N independent replicas of the workload, one per rank: the job's times are the slowest rank's
    (max over ranks of each rank's device-timed and end-to-end intervals) and its solves all ranks'.
    No data-path collective: this is the only exchange, after the timed region."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([dev_ms, e2e_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_ms, e2e_ms = float(t[0]), float(t[1])
    return dev_ms, e2e_ms, solves * world


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline_subprocess(refs_path=None):
    """The CPU oracle timed on the host: one process alone (cores_1), then one process per host
    core concurrently (the reported value).  Runs before any GPU work."""
    import platform
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample"]
    if refs_path:
        cmd += ["--oracle-refs", refs_path]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
    cores = host_cores()
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    try:
        value, wall = oracle_all_cores(cores, 1, 1)
    except Exception as e:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "error": repr(e)[-400:],
                "cores_1": {"value": d["value"], "unit": UNIT}}
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "arch": platform.machine(),
            "sample": f"one warm time step (potential + pressure solve, previous-step x0) of the 512x256 "
                      f"workload after one untimed step, in {cores} single-threaded processes at once "
                      f"(one per host core, numpy/scipy FP64), {2 * cores} solves in {wall:.1f} s",
            "cores_1": {"value": d["value"], "unit": UNIT, "seconds": d["seconds"],
                        "sample": "the same time step in one process alone"},
            "iterations": d["iterations"]}


def run_reference(args, rank):
    """The reference arm: the CPU oracle as it stands on every host core (one single-threaded
    process per core, each running the workload's time steps, potential + pressure solve)."""
    if rank != 0:
        return
    procs = args.ref_procs or host_cores()
    value, wall = oracle_all_cores(procs, args.warmup, args.steps)
    import platform
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * 2.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config("fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "arch": platform.machine(),
                             "sample": f"{args.steps} time steps (potential + pressure solve, previous-step x0) "
                                       f"of the 512x256 workload after {args.warmup} untimed ones, in each of "
                                       f"{procs} single-threaded processes at once; ms_per_step is the time "
                                       f"of one two-solve step at the aggregate rate ({wall:.1f} s timed)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def profile_case(case):
    """A short run for a profiler: the kernels of one case, no timing."""
    import torch

    from paper_2003_00082_gb300 import build, cgp, configs, inputs

    build.build()
    cgp.load()
    dev = torch.device("cuda:0")
    if case in ("fp64", "mixed"):
        xy, tri = inputs.ogrid(N_THETA, N_R)
        m = cgp.Mesh(xy, tri)
        cgp.cgp_mesh_set_ogrid(m.handle, N_THETA, N_R)
        xy_f, _, _ = m.fine_geometry()
        u, v = inputs.velocity(xy_f, 7, SEED, vortices=True)
        b = torch.empty(m.n_c, dtype=torch.float64, device=dev)
        cgp.cgp_restrict(m.handle, cgp.CGP_RHS_POTENTIAL, B_FIELD, RHO_OVER_DT, torch.as_tensor(u, device=dev),
                         torch.as_tensor(v, device=dev), b)
        x = torch.zeros(m.n_c, dtype=torch.float64, device=dev)
        prec = cgp.CGP_MIXED if case == "mixed" else cgp.CGP_FP64
        what = cgp.CGP_TUNE_SOLVE_MIXED if case == "mixed" else cgp.CGP_TUNE_SOLVE_FP64
        # the shape the autotuner picks on GB300 (FP64: O-grid tiles with the stencil product and tagged
        # reductions; mixed: tagged FP32 inner reductions)
        cgp.cgp_set_tuning(m.handle, what, 512, 1, 152, 8 if case == "mixed" else 40)
        for _ in range(2):
            x.zero_()
            info = cgp.cgp_poisson_solve(m.handle, b, x, tol=TOL, precision=prec)
        print(json.dumps({"case": case, "info": info, "launch": cgp.cgp_last_launch(m.handle, prec)}))
        m.close()
    elif case == "gnn":
        # the learned guess at the 64x32 size: 3 fused inferences, then 3 training steps of batch 16
        from paper_2003_00082_gb300 import learned_guess
        xy, tri = inputs.ogrid(64, 32)
        m = cgp.Mesh(xy, tri)
        net = cgp.GNN(m, 16, learned_guess.initial_params(0))
        g = torch.Generator(device="cpu").manual_seed(SEED)
        b, p1, p2, pt = (torch.randn((16, m.n_c), generator=g, dtype=torch.float64).to(dev) for _ in range(4))
        x0 = torch.empty(m.n_c, dtype=torch.float64, device=dev)
        for _ in range(3):
            net.predict(b[0], p1[0], p2[0], x0)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        for _ in range(3):
            net.train_step(16, b, p1, p2, pt, lr=1e-3, loss_dev=loss)
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "n": m.n_c, "loss": float(loss.item())}))
        net.close()
        m.close()
    elif case == "batched":
        # the shape the batch autotuner picks on GB300 (waves of 2048 rows a block, one 512-thread block per
        # SM, tagged FP32 inner reductions), so that a profiler sees the timed launches and no candidates;
        # two replays of the captured waves
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        out = run_batched(cgp, inputs, configs, torch, dev, flush, read_peaks()[0], reps=1, tuning=(512, 1, 1, 104))
        print(json.dumps({"case": case, "value": out["value"], "launch": out["launch"]}))
    else:
        out = spmv_bench(cgp, inputs, torch, dev, read_peaks()[0], reps=2)
        print(json.dumps({"case": case, "fp64_gb_s": out["fp64"]["gb_s"], "fp32_gb_s": out["fp32"]["gb_s"]}))


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--no-spmv", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the other-precision and batched passes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tuning", type=lambda v: tuple(int(t) for t in v.split(",")), default=None,
                    help="block,lanes,blocks,flags of the benchmarked precision's solves instead of autotuning")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-refs", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--ref-procs", type=int, default=0,
                    help="reference arm: oracle processes (default: one per host core)")
    ap.add_argument("--profile-case", choices=["fp64", "mixed", "batched", "spmv", "gnn"], default=None,
                    help="run one small case for a profiler and exit: two 512x256 potential solves, "
                         "one batched launch of the 64-instance workload, or the SpMV sweep")
    args = ap.parse_args()

    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_refs)), flush=True)
        return
    if args.profile_case:
        profile_case(args.profile_case)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")
        run_reference(args, rank)
        return

    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")

    cpu = None
    refs_path = None
    if rank == 0 and not args.no_cpu_baseline:
        import tempfile
        refs_path = os.path.join(tempfile.mkdtemp(prefix="cgp_oracle_"), "fields.npz")
        cpu = cpu_baseline_subprocess(None if args.no_variants else refs_path)   # before any GPU work
        if not os.path.exists(refs_path):
            refs_path = None

    res = run_mine(args, rank, world, local_rank, refs_path)
    if refs_path:
        import shutil
        shutil.rmtree(os.path.dirname(refs_path), ignore_errors=True)
    dev_ms, e2e_ms, total_solves = replica_totals(res["dev_ms"], res["e2e_ms"], res["solves"], world,
                                                  f"cuda:{local_rank}")
    if rank == 0:
        peak = res["peak"]
        line = {
            "metric": METRIC, "value": total_solves / (dev_ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic", "config": workload_config(args.precision),
            "roofline": {"bound": "hbm", "achieved": res["achieved"], "peak": peak, "unit": "GB/s",
                         "frac": res["achieved"] / peak, "traffic": solver_traffic(args.precision, res["tuned"][args.precision]["flags"]),
                         "kernel": "pcg_persistent_kernel",
                         "alg_bytes_per_launch": res["alg_bytes_per_launch"],
                         "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({res['peak_kind']})",
                         "kernel_share_of_step": res["pcg_share"],
                         "fp64_alu": {"achieved_tflops": res["fp64_tflops"], "peak_tflops": FP64_PEAK_TFLOPS,
                                      "frac": res["fp64_tflops"] / FP64_PEAK_TFLOPS,
                                      "peak_source": "nominal GB300 FP64 (1.25 TFLOP/s)"}},
            "cpu_baseline": cpu,
            "e2e": {"value": total_solves / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": res["h2d"],
                    "d2h_bytes_per_step": res["d2h"],
                    "timing": "one interval over all steps, from the first host-to-device copy to the last "
                              "device-to-host copy; step j+1's velocity in and step j's force and grad p out "
                              "on copy streams while steps compute (pinned host buffers)"},
            "gpu_launches": (KERNELS_PER_STEP + (2 * PERM_KERNELS_PER_SOLVE if renumbered(res["tuned"][args.precision]["flags"],
                                                                                     args.precision) else 0)) * args.steps,
            "clocks": res["clocks"],
            "iterations": {"per_solve_mean": statistics.mean(res["its"]), "min": min(res["its"]),
                           "max": max(res["its"]), "rel_res_true_max": res["rel_res_true_max"]},
        }
        if "spmv" in res:
            line["spmv"] = res["spmv"]
        if res.get("variant"):
            line["other_precision"] = res["variant"]
        if res.get("accuracy"):
            line["accuracy_vs_oracle"] = res["accuracy"]
        if "mixed_64x32" in res:
            line["mixed_64x32"] = res["mixed_64x32"]
        if "levels" in res:
            line["levels"] = res["levels"]
        if "far_field" in res:
            line["far_field"] = res["far_field"]
        if "batched" in res:
            line["batched"] = res["batched"]
        if "learned_guess" in res:
            line["learned_guess"] = res["learned_guess"]
        if "learned_guess_512x256" in res:
            line["learned_guess_512x256"] = res["learned_guess_512x256"]
        line["tuned_launch"] = res["tuned"]
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
