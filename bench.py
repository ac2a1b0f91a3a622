"""Benchmark: shifted solves per second at 1e-8 true residual on one GB300.

A step is one fks_solve of the whole workload: every frequency shift of every
source through the flexible Arnoldi basis, the per-shift least squares, the
assembly x_j = Z y_j and the true-residual check. A shifted solve counts when
its complex128 true relative residual ||b - (K + sigma_j M) x_j|| / ||b|| <= 1e-8.

Default workload (3): 3D 128^3 cell-centred aquifer (n = 2,097,152), anisotropic
lnK Gaussian field (variance 1, correlation lengths 0.2/0.2/0.05 L, mean
ln 1e-4), lognormal S_s (variance 0.25 of ln S_s), centre source, 200 shifts
(periods 5..3600 s log-spaced), 4 preconditioner shifts cycled per step,
multigrid inner solve in complex64 with complex128 defect correction, complex128
outer Arnoldi / least squares / assembly / true residual ("mixed"). Its
`comparison` times the same workload in plain complex128 on the same GPU, and
the batched workload 4 (3D 96^3, 64 well sources, 100 shifts).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload 1|2|3|4|5|6|7|8] [--precision fp64|mixed]

Workload 5 is the serving stream (request loop); workload 6 the sensitivity
matrix of workload 2's aquifer (Algorithm 6: forward solve, adjoint solves of 8
sensors, adjoint-state inner products for ln K and ln S_s), in Jacobian rows/s;
workload 7 a general sparse operator through the CSR path (K and M as CSR
arrays, BiCGSTAB inner cycles); workload 8 the mixed 2D batch (32 aquifers of
128^2 to 384^2 cells, one source each, 100 shifts) through the server's
concurrent lanes.

Under torchrun every rank solves its own copy of the workload (replicas, weak
scaling; no data-path collective). Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

# the CPU oracle legs run single-threaded unless the caller says otherwise, so
# that the reported core count is the one used (set before NumPy loads BLAS)
for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_k, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shifted solves/s at 1e-8 residual"
UNIT = "shifted solves/s"
TOL = 1e-8
INNER_EPS = 1e-10          # inner tolerance of the accuracy-gated runs (tol / 100)
# Flexible Arnoldi steps the default 512 x 512 workload takes to converge every
# shift (oracle run, multigrid inner eps 1e-10); used to extrapolate the
# bounded CPU sample to a whole solve.
WORKLOAD_STEPS = {1: 36, 2: 36, 3: 40, 4: 40}
# Inner cycles of the oracle's own complete solve of a workload (first source)
# with the relaxed rule, for extrapolating its bounded samples: workload 2 at
# l = 0.003 takes 36 steps and 307 cycles when the oracle runs to the end.
ORACLE_CYCLES = {(2, 0.003): 307}
# The same for the 3D 128^3 workload (3) at l = 0.003: (Arnoldi steps, inner
# cycles) of the oracle's complete solve of its source.
ORACLE_SOLVE = {(1, 0.003): (37, 281), (2, 0.003): (36, 307), (3, 0.003): (31, 327)}
JAC_SENSORS = 8   # sensors of the Jacobian workload (6)
FP64_PEAK_TFLOPS = 1.25    # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fks", choices=["fks", "reference"])
    ap.add_argument("--workload", type=int, default=3)
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed", "bf16"],
                    help="default: fp64 for workloads 1, 2 and 6 (complex128 throughout), mixed for 3-5")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true",
                    help="skip the all-cores oracle run beside the one-core CPU baseline (3D workloads)")
    ap.add_argument("--cpu-sample-steps", type=int, default=6,
                    help="2D workloads: Arnoldi steps of the oracle's CPU sample")
    ap.add_argument("--cpu-sample-cycles", type=int, default=4,
                    help="3D workloads: inner multigrid cycles of the oracle's CPU sample")
    ap.add_argument("--no-batched", action="store_true",
                    help="workload 3: skip timing the batched workload 4 beside the line")
    ap.add_argument("--survey", action="store_true", help="time every kernel class (stderr)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer region (very large outputs)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the plain (complex128, fixed tolerance) and mixed relaxed variants")
    ap.add_argument("--single", action="store_true",
                    help="one untimed solve (after autotuning) and exit (a short command for ncu launch lists)")
    ap.add_argument("--precond-cycles", type=int, default=0,
                    help="run this many inner cycles of one fks_precond_apply on the workload's operator (after "
                         "autotuning) and exit: the inner-solve kernels at full size with a small device footprint, "
                         "for ncu captures")
    ap.add_argument("--launch-mode", default="graph", choices=["graph", "host"],
                    help="graph: the step loop as one CUDA graph; host: the same kernels launched one by one")
    ap.add_argument("--inner-relax", type=float, default=0.003,
                    help="relaxed inner tolerance constant l (eps_k = min(1e-3, max(eps, l tol / R_k-1))); "
                         "0: the fixed eps of every step")
    ap.add_argument("--requests", type=int, default=1000, help="workload 5: requests in the stream")
    ap.add_argument("--latency-requests", type=int, default=150,
                    help="workload 5: requests of each Poisson latency run")
    ap.add_argument("--lanes", type=int, default=3, help="workload 5: concurrent server lanes")
    ap.add_argument("--mix-lanes", type=int, default=8, help="workload 8: concurrent server lanes")
    ap.add_argument("--fuse-max", type=int, default=None,
                    help="fused 2D levels up to this many cells (-1: all) instead of autotuning")
    ap.add_argument("--tile16-max", type=int, default=None,
                    help="with --fuse-max: fused levels up to this many cells on 16 x 16 tiles (-1: all)")
    ap.add_argument("--tail-max", type=int, default=None,
                    help="with --fuse-max: levels up to this many cells in the single-block tail kernel")
    ap.add_argument("--tile8-max", type=int, default=None,
                    help="with --fuse-max: fused levels up to this many cells on 8 x 8 tiles (-1: all)")
    ap.add_argument("--cluster-max", type=int, default=None,
                    help="with --fuse-max: from the first level of at most this many cells down, the cluster "
                         "V-cycle kernel (0: off)")
    ap.add_argument("--coop-max", type=int, default=None,
                    help="with --fuse-max: the cooperative lower cycle from the first level of at most this many "
                         "cells (default 0: off)")
    ap.add_argument("--variant", default="fgmres", choices=["fgmres", "ffom"])
    ap.add_argument("--precond", default="amg", choices=["amg", "jacobi"],
                    help="workload 7: preconditioner of the BiCGSTAB inner cycles")
    ap.add_argument("--restart", type=int, default=0,
                    help="restarted FFOM with cycles of this many steps (needs --variant ffom; 0: none)")
    ap.add_argument("--sensors", type=int, default=JAC_SENSORS, help="workload 6: sensors (adjoint sources)")
    ap.add_argument("--shift-stride", type=int, default=1,
                    help="workload 6: every k-th shift of the workload (a smaller case, e.g. for ncu)")
    ap.add_argument("--no-pdl", action="store_true",
                    help="launch the multigrid and defect kernels without programmatic dependent launch")
    ap.add_argument("--no-survey", action="store_true",
                    help="skip the per-class timing survey and the roofline (a short command for ncu launch lists)")
    a = ap.parse_args()
    if a.precision is None:
        a.precision = "fp64" if a.workload in (1, 2, 6, 7) else "mixed"
    return a


# The CUDA sources that define each kernel class (its translation unit and the
# headers it includes); DRAM traffic recorded for another digest of them is stale.
_GRID_SOURCES = ("grid.cu", "grid.cuh", "stencil.cuh", "common.cuh")
CLASS_SOURCES = {"smooth": _GRID_SOURCES, "restrict": _GRID_SOURCES, "prolong": _GRID_SOURCES,
                 "pre2d": _GRID_SOURCES, "post2d": _GRID_SOURCES, "tail": _GRID_SOURCES, "defect": _GRID_SOURCES,
                 "sensitivity": ("sensitivity.cu", "sensitivity.cuh", "stencil.cuh", "common.cuh")}


def source_hash(kclass=None):
    """Digest (sha256, first 16 hex digits) of the CUDA sources of a kernel
    class (CLASS_SOURCES), or of all device code but the host engine capi.cu."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1212_3660_gb300", "csrc")
    files = CLASS_SOURCES.get(kclass)
    if files is None:
        files = [f for f in os.listdir(d) if f.endswith((".cu", ".cuh")) and f != "capi.cu"]
    for f in sorted(files):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, precision, kclass, level):
    """DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum) of
    this kernel class on this level, from the table in profiles/traffic.md, if it
    was captured from the current sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None, None
    cur = source_hash(kclass)
    for line in open(path):
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) < 7 or cells[0] != workload:
            continue
        try:
            if cells[1] == precision and cells[2] == kclass and int(cells[3]) == level:
                return (float(cells[5]) if cells[6] == cur else None), cells[6]
        except ValueError:
            continue
    return None, None


# Serving stream (workload 5): x_j are delivered to the client for requests
# whose outputs (n x n_f x sources x 16 B) take at most this many bytes; larger
# ones deliver their residual certificates and statuses only (X = NULL).
SERVE_MAX_X_BYTES = 1 << 30
SERVE_WINDOW = 32          # outstanding requests of the closed-loop client


def serve_bench(args, rank, world, local, dist):
    """Request loop over the server on the serving workload: a pool of aquifers
    (2D and 3D, 64^2 to 160^3 cells) and a seeded Poisson stream of requests,
    each on one aquifer with 10-200 shifts and 1-16 sources, admitted by a
    device-memory budget onto concurrent lanes with continuous batching.
    Capacity: a closed-loop client keeps SERVE_WINDOW requests outstanding;
    latency (submit to results in host memory) at Poisson arrivals of 0.7x and
    0.9x that capacity."""
    import threading

    import torch

    from paper_1212_3660_gb300 import fks, synth
    prec = prec_of(args.precision, fks)
    count = args.requests
    aquifers, stream = synth.make_serving_stream(count, seed=3000 + rank)
    ctx = fks.fks_create(local)
    t0 = time.perf_counter()
    probs, ops = [], []
    for a in aquifers:
        p = synth.make_problem(m_max=100, **a)
        d = p.dim
        probs.append(p)
        ops.append(fks.fks_op_grid(ctx, d, [p.shape[d - 1 - q] for q in range(d)], p.h, p.cond, p.ss,
                                   p.dirichlet_mask))
    setup_ms = 1000 * (time.perf_counter() - t0)
    for p, op in zip(probs, ops):   # tiles and chunks per aquifer, as a deployment would do once
        fks.fks_op_autotune(op, prec, complex(p.tau_bar[len(p.tau_bar) // 2]))
    print(f"serving: {len(ops)} operators set up and tuned, {time.perf_counter() - t0:.1f} s", file=sys.stderr,
          flush=True)
    free, _ = torch.cuda.mem_get_info(local)
    budget = int(free * 0.7)
    srv = fks.fks_server_create(ctx, budget, lanes=args.lanes)
    sigma_of = {}

    def make_req(i):
        q = stream[i]
        p = probs[q["aquifer"]]
        key = (q["aquifer"], q["n_f"])
        if key not in sigma_of:
            sigma_of[key] = 1j * synth.log_spaced_omegas(5.0, 3600.0, q["n_f"])
        src = synth.well_cells(p.shape, q["n_rhs"], np.random.default_rng(q["src_seed"]))
        b = np.zeros((q["n_rhs"], p.n), np.complex128)
        b[np.arange(q["n_rhs"]), src] = 1.0
        opts, keep = fks.make_options(tol=TOL, m_max=p.m_max, precision=prec, inner_tol=INNER_EPS,
                                      schedule=p.schedule, inner_relax=args.inner_relax)
        with_x = p.n * q["n_f"] * q["n_rhs"] * 16 <= SERVE_MAX_X_BYTES
        return fks.ServerRequest(ops[q["aquifer"]], b, sigma_of[key], p.tau_bar, opts, keep, p.n, with_x=with_x)

    def run(idx, arrivals=None, window=None):
        out = {}
        err = []
        t_start = time.perf_counter()
        sem = threading.Semaphore(window) if window else None

        def submitter():
            try:
                for q, i in enumerate(idx):
                    if sem is not None:
                        sem.acquire()
                    if arrivals is not None:
                        dt = t_start + arrivals[q] - time.perf_counter()
                        if dt > 0:
                            time.sleep(dt)
                    r = make_req(i)
                    fks.fks_server_submit(srv, r)
                    out[q] = r
            except Exception as e:  # noqa: BLE001
                err.append(e)

        th = threading.Thread(target=submitter)
        th.start()
        lat, conv, total, ends, starts, statuses = [], 0, 0, [], [], []
        h2d = d2h = 0
        for q in range(len(idx)):
            while q not in out and not err:
                time.sleep(0.0005)
            if err:
                break
            r = out[q]
            st_r = fks.fks_server_wait(srv, r.ticket)
            statuses.append(st_r)
            if sem is not None:
                sem.release()
            ts, _, te = fks.fks_server_times(srv, r.ticket)
            lat.append(1000 * (te - ts))
            starts.append(ts)
            ends.append(te)
            if st_r >= 0:   # failed requests deliver nothing
                conv += int(np.sum(r.res_true <= TOL))
            total += r.res_true.size
            h2d += r.b.nbytes + r.sigma.nbytes + r.tau.nbytes
            d2h += (r.X.nbytes if r.X is not None else 0) + r.res_true.size * (8 * 3 + 4 * 2)
            out[q] = None   # the client drops the delivered arrays
            if (q + 1) % 50 == 0:
                print(f"serving: {q + 1}/{len(idx)} requests done, {time.perf_counter() - t_start:.1f} s",
                      file=sys.stderr, flush=True)
        th.join()
        if err:
            raise err[0]
        wall = max(ends) - min(starts)
        return {"wall_s": wall, "converged": conv, "solves": total, "solves_per_s": conv / wall,
                "requests_per_s": len(idx) / wall, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "h2d": h2d, "d2h": d2h,
                "statuses": {str(k): int(v) for k, v in zip(*np.unique(np.array(statuses), return_counts=True))}}

    # warm-up: a few requests once (graph capture, workspaces)
    for _ in range(max(args.warmup, 1)):
        run(list(range(min(4, count))), window=4)
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except ValueError:
            pass
    l0 = fks.fks_server_launches(srv)
    n_lat = min(count, args.latency_requests)
    arrival_unit = np.array([q["arrival"] for q in stream[:n_lat]])
    with ClockSampler(gpu_index) as clk:
        if world > 1:
            dist.barrier()
        cap = run(list(range(count)), window=SERVE_WINDOW)
        loads = {}
        for f in (0.7, 0.9):
            lam = f * cap["requests_per_s"]
            loads[f"{f:.1f}"] = run(list(range(n_lat)), arrivals=arrival_unit / lam)
        if world > 1:
            dist.barrier()
    launches = fks.fks_server_launches(srv) - l0

    replicas = Replicas(dist, world, torch.device("cuda", local))
    wall = replicas.max(cap["wall_s"])
    value = replicas.throughput(cap["converged"], cap["wall_s"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the stream's first request (first source), its own steps
        r0 = make_req(0)
        fks.fks_server_submit(srv, r0)
        fks.fks_server_wait(srv, r0.ticket)
        p0 = probs[stream[0]["aquifer"]]
        ws = int(r0.m_j.max())
        pr0 = synth.make_problem(m_max=100, **{**aquifers[stream[0]["aquifer"]], "n_f": stream[0]["n_f"]})
        v, dt, desc = cpu_oracle_sample(pr0, min(args.cpu_sample_steps, ws), ws, INNER_EPS, args.inner_relax)
        cpu = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": f"request 0 ({'x'.join(map(str, p0.shape[::-1]))}, {stream[0]['n_f']} shifts; "
                         f"first source): " + desc}
    fks.fks_server_destroy(srv)
    for op in ops:
        fks.fks_op_destroy(op)
    fks.fks_destroy(ctx)
    if rank == 0:
        shapes = {}
        for q in stream:
            k = "x".join(map(str, probs[q["aquifer"]].shape[::-1]))
            shapes[k] = shapes.get(k, 0) + 1
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1,
                "warmup": max(args.warmup, 1), "ms_per_step": 1000 * wall, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": dtype_of(prec, fks), "data": "synthetic",
                "config": {"workload": "serving-stream", "requests": count, "aquifers": len(aquifers),
                           "requests_per_grid": shapes, "shifts": "10..200 (multiples of 10)", "sources": "1..16",
                           "shifted_solves": cap["solves"], "lanes": args.lanes, "mem_budget_bytes": budget,
                           "precision": args.precision, "parallelism": f"replicas{world}",
                           "batching": "continuous: sources join running batches at Arnoldi-step boundaries",
                           "client": f"closed loop, {SERVE_WINDOW} requests outstanding",
                           "x_delivery": f"x_j delivered for requests with at most {SERVE_MAX_X_BYTES >> 20} MiB "
                                         "of outputs, residuals and statuses for all",
                           "step": "one pass over the stream",
                           "op_setup_ms_all_aquifers": setup_ms,
                           "l2": "aquifers up to 160^3 cells; bases and outputs exceed L2"},
                "latency_ms": {"closed_loop": {"p50": cap["p50_ms"], "p99": cap["p99_ms"]},
                               **{f"poisson_{k}x_capacity": {"p50": v_["p50_ms"], "p99": v_["p99_ms"],
                                                             "solves_per_s": v_["solves_per_s"],
                                                             "requests": n_lat,
                                                             "offered_requests_per_s": float(k) * cap["requests_per_s"]}
                                  for k, v_ in loads.items()}},
                "converged_per_step": cap["converged"], "request_statuses": cap["statuses"],
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": cap["h2d"],
                        "d2h_bytes_per_step": cap["d2h"],
                        "note": "the server API takes host buffers: every request's copies are inside the timed region"},
                "roofline": None,
                "roofline_note": "per-kernel event timing runs on fks_solve's lane; the kernels are those of the "
                                 "workload 1-4 lines",
                "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": launches}
        print(json.dumps(line), flush=True)


def mix2d_bench(args, rank, world, local, dist):
    """The mixed 2D batch: 32 aquifers of 128^2 to 384^2 cells, one centre
    source each, 100 shifts, 4 taus cycled. A step submits one request per
    aquifer to the server, whose lanes run the different operators
    concurrently, and ends when the last request's x_j are in host memory
    (page-locked output arrays, allocated once and reused, as a client would).
    Beside it, the same step on a one-lane server: one operator at a time."""
    import torch

    from paper_1212_3660_gb300 import fks, synth
    prec = prec_of(args.precision, fks)
    grids = synth.mix2d_grids()
    ctx = fks.fks_create(local)
    t0 = time.perf_counter()
    probs = [synth.make_problem(m_max=100, **g) for g in grids]
    ops = [fks.fks_op_grid(ctx, 2, [p.shape[1], p.shape[0]], p.h, p.cond, p.ss, p.dirichlet_mask) for p in probs]
    setup_ms = 1000 * (time.perf_counter() - t0)
    for p, op in zip(probs, ops):
        fks.fks_op_autotune(op, prec, complex(p.tau_bar[len(p.tau_bar) // 2]))
    outs_t = [torch.empty((1, len(p.sigma), p.n), dtype=torch.complex128, pin_memory=True) for p in probs]
    outs = [t.numpy() for t in outs_t]   # views of the page-locked tensors (kept alive in outs_t)
    rhs = [p.rhs().T.copy() for p in probs]
    free, _ = torch.cuda.mem_get_info(local)
    budget = int(free * 0.7)

    def one_pass(srv):
        t_start = time.perf_counter()
        reqs = []
        for g, p in enumerate(probs):
            opts, keep = fks.make_options(tol=TOL, m_max=p.m_max, precision=prec, inner_tol=INNER_EPS,
                                          schedule=p.schedule, inner_relax=args.inner_relax)
            r = fks.ServerRequest(ops[g], rhs[g], p.sigma, p.tau_bar, opts, keep, p.n, out=outs[g])
            fks.fks_server_submit(srv, r)
            reqs.append(r)
        conv = total = h2d = d2h = 0
        statuses = []
        for r in reqs:
            st_r = fks.fks_server_wait(srv, r.ticket)
            statuses.append(st_r)
            if st_r >= 0:
                conv += int(np.sum(r.res_true <= TOL))
            total += r.res_true.size
            h2d += r.b.nbytes + r.sigma.nbytes + r.tau.nbytes
            d2h += r.X.nbytes + r.res_true.size * (8 * 3 + 4 * 2)
        return {"wall_s": time.perf_counter() - t_start, "converged": conv, "solves": total, "h2d": h2d,
                "d2h": d2h, "steps_max": int(max(int(r.m_j.max()) for r in reqs)),
                "statuses": {str(k): int(v) for k, v in zip(*np.unique(np.array(statuses), return_counts=True))}}

    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except ValueError:
            pass
    replicas = Replicas(dist, world, torch.device("cuda", local))
    srv = fks.fks_server_create(ctx, budget, lanes=args.mix_lanes)
    for _ in range(max(args.warmup, 1)):
        one_pass(srv)
    l0 = fks.fks_server_launches(srv)
    passes = []
    with ClockSampler(gpu_index) as clk:
        replicas.barrier()
        for _ in range(args.steps):
            passes.append(one_pass(srv))
        replicas.barrier()
    launches = fks.fks_server_launches(srv) - l0
    fks.fks_server_destroy(srv)
    wall = sum(q["wall_s"] for q in passes)
    conv = sum(q["converged"] for q in passes)
    value = replicas.throughput(conv / args.steps, wall / args.steps)
    ms = 1000 * replicas.max(wall / args.steps)
    one_lane = None
    if not args.no_compare:
        srv1 = fks.fks_server_create(ctx, budget, lanes=1)
        one_pass(srv1)
        q1 = one_pass(srv1)
        fks.fks_server_destroy(srv1)
        one_lane = {"value": q1["converged"] / q1["wall_s"], "ms_per_step": 1000 * q1["wall_s"], "lanes": 1,
                    "steps_timed": 1}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = mix2d_cpu_sample(probs, args, passes[0]["steps_max"])
    for op in ops:
        fks.fks_op_destroy(op)
    fks.fks_destroy(ctx)
    if rank == 0:
        sides = {}
        for p in probs:
            k = f"{p.shape[1]}x{p.shape[0]}"
            sides[k] = sides.get(k, 0) + 1
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 1), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype_of(prec, fks), "data": "synthetic",
                "config": {"workload": "2d-mix-32x(128..384)^2-f100-p4", "aquifers": len(probs), "grids": sides,
                           "cells_total": int(sum(p.n for p in probs)), "n_f": len(probs[0].sigma), "n_p": 4,
                           "sources_per_aquifer": 1, "precision": args.precision, "lanes": args.mix_lanes,
                           "parallelism": f"replicas{world}",
                           "step": "one request per aquifer through the server, until the last x_j is in host "
                                   "memory", "op_setup_ms_all_aquifers": setup_ms,
                           "arnoldi_steps_max": passes[0]["steps_max"],
                           "l2": "bases and outputs of the 32 solves (GBs) exceed L2"},
                "solves_per_step": passes[0]["solves"], "converged_per_step": conv / args.steps,
                "request_statuses": passes[-1]["statuses"],
                "comparison": {"one_lane": one_lane},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": passes[0]["h2d"],
                        "d2h_bytes_per_step": passes[0]["d2h"],
                        "note": "the server API takes host buffers: every request's copies are inside the timed "
                                "region"},
                "roofline": None,
                "roofline_note": "per-kernel event timing runs on fks_solve's lane; the kernels are those of the "
                                 "workload 1-2 lines",
                "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": launches}
        print(json.dumps(line), flush=True)


def mix2d_cpu_sample(probs, args, steps):
    """The oracle on the mixed 2D batch: a bounded sample of its first aquifer
    (cpu_oracle_sample, scaled to `steps` Arnoldi steps), scaled to the batch by
    cell count (the oracle's time per shifted solve grows with n)."""
    p0 = probs[0]
    v, dt, desc = cpu_oracle_sample(p0, max(1, args.cpu_sample_steps // 3), max(steps, 1), INNER_EPS,
                                    args.inner_relax)
    cells = sum(p.n for p in probs)
    t_batch = len(p0.sigma) / v * cells / p0.n
    value = sum(len(p.sigma) for p in probs) / t_batch
    return {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": f"aquifer 0 ({p0.shape[1]}x{p0.shape[0]}, {len(p0.sigma)} shifts): {desc}; scaled to the "
                      f"32 aquifers by cell count ({cells} cells)"}


def jacobian_bench(args, rank, world, local, dist):
    """Sensitivity matrix of the 512 x 512 workload (Algorithm 6): the forward
    solve of the source, the adjoint solves of JAC_SENSORS sensors (one batched
    fks_solve with the right-hand sides -e_m, Eq. adjoint) and the adjoint-state
    inner products (Eq. sensitivity) for ln K and ln S_s of every cell. A step
    is one whole Jacobian; the unit is a Jacobian row, the paper's
    N_y = 2 n_f n_y real rows (real and imaginary part per sensor and
    frequency), each holding both parameter fields; a row counts when its
    forward and adjoint solves are certified at 1e-8."""
    import torch

    from paper_1212_3660_gb300 import fks, synth
    from paper_1212_3660_gb300.solver import Solver
    prec = prec_of(args.precision, fks)
    pr = synth.workload(2, m_max=100)
    pr.sigma = pr.sigma[::max(1, args.shift_stride)].copy()
    ns = args.sensors
    name = f"jacobian-512x512-f{len(pr.sigma)}-s{ns}"
    sensors = synth.well_cells(pr.shape, ns, np.random.default_rng(2006))
    solver = Solver(pr, device=local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    n, n_f = pr.n, len(pr.sigma)
    b_f = torch.from_numpy(pr.rhs().T.copy()).to(dev)
    b_a = torch.zeros((ns, n), dtype=torch.complex128, device=dev)
    for m, c in enumerate(sensors):
        b_a[m, int(c)] = -1.0
    X_f = torch.empty((1, n_f, n), dtype=torch.complex128, device=dev)
    X_a = torch.empty((ns, n_f, n), dtype=torch.complex128, device=dev)
    jk = torch.empty_like(X_a)
    js = torch.empty_like(X_a)
    sig_d = torch.from_numpy(pr.sigma.astype(np.complex128)).to(dev)
    tau_d = torch.from_numpy(pr.tau_bar.astype(np.complex128)).to(dev)
    outs = {k: (np.zeros((k, n_f)), np.zeros((k, n_f)), np.zeros((k, n_f)), np.zeros((k, n_f), np.int32),
                np.zeros((k, n_f), np.int32)) for k in (1, ns)}
    opts, keep = fks.make_options(tol=TOL, m_max=pr.m_max, precision=prec, inner_tol=INNER_EPS,
                                  schedule=pr.schedule, inner_relax=args.inner_relax)
    info1, info1_arrays = fks.make_info(1, pr.m_max)   # the arrays back the struct's pointers: keep them
    infon, infon_arrays = fks.make_info(ns, pr.m_max)
    fks.fks_op_autotune(solver.op, prec, complex(pr.tau_bar[len(pr.tau_bar) // 2]), sh)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step():
        ev[0].record(stream)
        fks.fks_solve(solver.op, b_f, 1, sig_d, n_f, tau_d, len(pr.tau_bar), opts, X_f, *outs[1], info1, sh)
        ev[1].record(stream)
        fks.fks_solve(solver.op, b_a, ns, sig_d, n_f, tau_d, len(pr.tau_bar), opts, X_a, *outs[ns], infon, sh)
        ev[2].record(stream)
        fks.fks_sensitivity(solver.op, X_f, X_a, ns, sig_d, n_f, jk, js, sh)
        ev[3].record(stream)
        ok_f = outs[1][2][0] <= TOL
        ok_a = outs[ns][2] <= TOL
        return 2 * int(np.sum(ok_a & ok_f[None, :]))

    for _ in range(args.warmup):
        step()
    replicas = Replicas(dist, world, dev)
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except ValueError:
            pass
    l0 = fks.fks_profile_read(solver.op)["all_launches"]
    parts = np.zeros(3)
    rows = 0
    with ClockSampler(gpu_index) as clk:
        replicas.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            rows += step()
            torch.cuda.synchronize()
            parts += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
        t1.record(stream)
        torch.cuda.synchronize()
        replicas.barrier()
    launches = fks.fks_profile_read(solver.op)["all_launches"] - l0 + args.steps  # + the sensitivity kernel
    ms = t0.elapsed_time(t1) / args.steps
    value = replicas.throughput(rows / args.steps, ms / 1000.0)
    parts /= args.steps
    # roofline of the inner-product kernel: algorithmic bytes and FP64 flops per
    # launch (per sensor, shift and cell: psi read, two results written; per
    # face 2 subtractions and 4 fused multiply-adds, plus one complex product;
    # per shift and cell the folded face weights)
    d = len(pr.shape)
    sens_bytes = ns * n_f * n * (16 + 2 * 16) + n_f * n * 16 + n * (8 + 8 + 8 * d) + n_f * 16
    sens_flops = ns * n_f * n * (10 * 2 * d + 6) + n_f * n * (8 * 2 * d + 6)
    hbm_peak, _, peak_src = peaks()
    sens_gbs = sens_bytes / (parts[2] / 1000.0) / 1e9
    sens_tfl = sens_flops / (parts[2] / 1000.0) / 1e12
    traffic, traffic_src = recorded_traffic(name, args.precision, "sensitivity", 0)
    if sens_tfl / FP64_PEAK_TFLOPS > sens_gbs / hbm_peak:
        roof = {"bound": "alu", "achieved": sens_tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": sens_tfl / FP64_PEAK_TFLOPS, "peak_source": "FP64 nominal: 152 SMs x 2 DFMA/clk x 2.07 GHz",
                "hbm_frac_of_" + peak_src: sens_gbs / hbm_peak}
    else:
        roof = {"bound": "hbm", "achieved": sens_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": sens_gbs / hbm_peak,
                "peak_source": peak_src}
    roof.update({"traffic": traffic, "kernel": "k_sensitivity",
            "alg_bytes_per_launch": sens_bytes, "alg_flops_per_launch": sens_flops, "launch_ms": parts[2],
            "traffic_source": ("profiles/traffic.md (ncu, sources " + traffic_src + ")") if traffic is not None
            else ("stale: kernels changed since the ncu capture" if traffic_src else "no ncu capture recorded")})
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, _, desc = jacobian_cpu_sample(pr, args, ns)
        cpu = {"value": v, "unit": "rows/s", "cores": blas_threads(), "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {"metric": "Jacobian rows/s at 1e-8 residual", "value": value, "unit": "rows/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": replicas.max(ms),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": dtype_of(prec, fks), "data": "synthetic",
                "config": {"workload": name, "grid": "x".join(map(str, pr.shape[::-1])), "n": n, "n_f": n_f,
                           "sensors": ns, "parameters": ["ln K", "ln S_s"], "precision": args.precision,
                           "inner_relax": args.inner_relax, "parallelism": f"replicas{world}",
                           "l2": "adjoint phasors and sensitivities (3 x 6.7 GB) exceed L2"},
                "breakdown_ms": {"forward": parts[0], "adjoint": parts[1], "inner_product": parts[2]},
                "shifted_solves_per_s": (1 + ns) * n_f / ((parts[0] + parts[1]) / 1000.0),
                "rows_per_step": rows / args.steps,
                "e2e": None, "e2e_note": "device-resident only: the host copies of 20 GB of phasors and "
                                         "sensitivities per step would measure the host link",
                "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    solver.close()


def csr_bench(args, rank, world, local, dist):
    """Workload 7: the general-operator path (K and M given as CSR arrays, inner
    solves by BiCGSTAB cycles preconditioned by a smoothed-aggregation AMG V-cycle,
    the paper's inner solver, or by Jacobi with --precond jacobi; complex128 defect
    correction) on a finite-element-like operator. Same timing, survey, roofline,
    end-to-end and CPU-oracle legs as the grid workloads. The AMG hierarchies of
    the taus are built once before the timed region (like the operator) and their
    host setup time is reported in config."""
    import torch

    from paper_1212_3660_gb300 import fks, synth
    from paper_1212_3660_gb300.solver import Solver
    prec = prec_of(args.precision, fks)
    pr = synth.fe_workload()
    amg = args.precond == "amg"
    solver = Solver(pr, device=local, csr=pr.csr_arrays(), amg=amg)
    amg_cfg = {}
    if amg:
        amg_ms = fks.fks_op_amg_setup(solver.op, pr.tau_bar, prec)
        sizes, _ = fks.fks_op_amg_info(solver.op)
        amg_cfg = {"amg_setup_ms": amg_ms, "amg_levels": [int(x) for x in sizes]}
    bcg_steps = 4 if amg else 8
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    n, n_f, n_rhs = pr.n, len(pr.sigma), len(pr.src_cells)
    b_d = torch.from_numpy(pr.rhs().T.copy()).to(dev)
    sig_d = torch.from_numpy(pr.sigma.astype(np.complex128)).to(dev)
    tau_d = torch.from_numpy(pr.tau_bar.astype(np.complex128)).to(dev)
    X_d = torch.empty((n_rhs, n_f, n), dtype=torch.complex128, device=dev)
    est = np.zeros((n_rhs, n_f)); bnd = np.zeros((n_rhs, n_f)); tru = np.zeros((n_rhs, n_f))
    mj = np.zeros((n_rhs, n_f), np.int32); sst = np.zeros((n_rhs, n_f), np.int32)
    opts, keep = fks.make_options(tol=TOL, m_max=pr.m_max, precision=prec, inner_tol=INNER_EPS,
                                  schedule=pr.schedule, inner_relax=args.inner_relax)
    opts_host, keep_host = fks.make_options(tol=TOL, m_max=pr.m_max, precision=prec, inner_tol=INNER_EPS,
                                            schedule=pr.schedule, launch_mode=1, inner_relax=args.inner_relax)
    info, info_arr = fks.make_info(n_rhs, pr.m_max)

    def step(b, X, o=opts):
        return fks.fks_solve(solver.op, b, n_rhs, sig_d, n_f, tau_d, len(pr.tau_bar), o, X, est, bnd, tru, mj,
                             sst, info, sh)

    for _ in range(args.warmup):
        step(b_d, X_d)
    totals = {}
    for c, name in enumerate([] if args.no_survey else fks.KERNEL_CLASSES):
        fks.fks_profile_select(solver.op, c)
        step(b_d, X_d, opts_host)
        totals[name] = fks.fks_profile_read(solver.op)
    fks.fks_profile_select(solver.op, None)
    fks.fks_profile_read(solver.op)
    dominant = max(totals, key=lambda k: totals[k]["ms"]) if totals else None
    if args.survey and rank == 0:
        tot = sum(v["ms"] for v in totals.values())
        for k, v in sorted(totals.items(), key=lambda kv: -kv[1]["ms"]):
            print(f"# {k:9s} launches {v['launches']:7d} ms {v['ms']:9.3f} ({100 * v['ms'] / max(tot, 1e-9):5.1f}%) "
                  f"GB/s {v['bytes'] / max(v['ms'], 1e-9) / 1e6:8.1f}", file=sys.stderr)
    replicas = Replicas(dist, world, dev)
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except ValueError:
            pass
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    converged = 0
    with ClockSampler(gpu_index) as clk:
        replicas.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step(b_d, X_d)
            converged += int(np.sum(tru <= TOL))
        e1.record(stream)
        torch.cuda.synchronize()
        replicas.barrier()
    launches = fks.fks_profile_read(solver.op)["all_launches"]
    ms = e0.elapsed_time(e1) / args.steps
    value = replicas.throughput(converged / args.steps, ms / 1000.0)
    main_info = {k: v.copy() for k, v in info_arr.items()}
    roof = None
    if dominant is not None:
        fks.fks_profile_select(solver.op, dominant, 0)
        for _ in range(args.steps):
            step(b_d, X_d, opts_host)
        prof = fks.fks_profile_read(solver.op)
        fks.fks_profile_select(solver.op, None)
        hbm_peak, _, peak_src = peaks()
        gbs = prof["bytes"] / max(prof["ms"], 1e-12) / 1e6
        tfl = prof["flops"] / max(prof["ms"], 1e-12) / 1e9
        f_hbm = gbs / hbm_peak
        f_alu = tfl / FP64_PEAK_TFLOPS if prec == fks.FKS_PREC_FP64 else 0.0
        common = {"traffic": None, "traffic_source": "no ncu capture recorded", "kernel": dominant,
                  "launches": prof["launches"], "avg_launch_us": 1000 * prof["ms"] / max(prof["launches"], 1),
                  "alg_bytes_per_launch": prof["bytes"] / max(prof["launches"], 1),
                  "alg_flops_per_launch": prof["flops"] / max(prof["launches"], 1)}
        if f_alu > f_hbm:
            roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": f_alu,
                    "peak_source": "FP64 nominal: 152 SMs x 2 DFMA/clk x 2.07 GHz", "hbm_frac_of_" + peak_src: f_hbm,
                    **common}
        else:
            roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": f_hbm,
                    "peak_source": peak_src, **common}
    e2e = None
    if not args.no_e2e:
        # pinned host buffers allocated as such (page-locked at allocation)
        b_h = torch.empty((n_rhs, n), dtype=torch.complex128, pin_memory=True)
        b_h.copy_(torch.from_numpy(pr.rhs().T.copy()))
        X_h = torch.empty((n_rhs, n_f, n), dtype=torch.complex128, pin_memory=True)
        step(b_h, X_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv = 0
        for _ in range(args.steps):
            step(b_h, X_h)
            conv += int(np.sum(tru <= TOL))
        t_e2e = replicas.max((time.perf_counter() - t0) / args.steps)
        e2e = {"value": replicas.sum(conv / args.steps) / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": b_h.numel() * 16 + (n_f + len(pr.tau_bar)) * 16,
               "d2h_bytes_per_step": X_h.numel() * 16 + n_rhs * n_f * (8 * 3 + 4 * 2)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, _, desc = csr_cpu_sample(pr, args, amg, int(main_info["inner_cycles"][:pr.m_max].sum()))
        cpu = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": replicas.max(ms), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype_of(prec, fks),
                "data": "synthetic",
                "config": {"workload": pr.name, "n": n, "nnz_K": int(pr.K.nnz), "n_f": n_f,
                           "n_p": len(pr.tau_bar), "schedule": "cycled", "sources_per_gpu": n_rhs,
                           "inner": f"BiCGSTAB cycles of {bcg_steps} steps ("
                                    + ("smoothed-aggregation AMG V(2,2), damped Jacobi" if amg else "Jacobi")
                                    + f"), defect correction to eps={INNER_EPS:g}"
                                    + (f", relaxed l = {args.inner_relax:g}" if args.inner_relax > 0 else ""),
                           **amg_cfg,
                           "precision": args.precision, "parallelism": f"replicas{world}",
                           "arnoldi_steps": int(main_info["steps"].max()),
                           "inner_cycles_total": int(main_info["inner_cycles"].sum())},
                "solves_per_step": n_f * n_rhs, "converged_per_step": converged / args.steps,
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    solver.close()


# inner cycles of the whole workload-7 solve (complex128, relaxed l = 0.003) on the GPU,
# by which the reference arm scales its bounded sample
CSR_CYCLES = {"amg": 114, "jacobi": 701}


def csr_cpu_sample(pr, args, amg, total_cycles):
    """The oracle on workload 7: the first Arnoldi steps of the source with the
    same inner solver (AMG- or Jacobi-preconditioned BiCGSTAB cycles, the same
    inner rule), scaled to a whole solve by its inner-cycle count. The oracle's
    AMG setup is left out, like the library's (built before the timed region).
    Returns (solves/s, seconds, description)."""
    import oracle
    from oracle.amg import AMGBiCGStabInner
    from oracle.csr import BiCGStabInner
    op = oracle.CSROperator(pr.K, pr.M)
    inner = (AMGBiCGStabInner(op, pr.tau_bar, INNER_EPS, steps=4) if amg
             else BiCGStabInner(op, pr.tau_bar, INNER_EPS, steps=8))
    c0 = time.perf_counter()
    res = oracle.shifted_solve(op, pr.rhs()[:, 0], pr.sigma, pr.tau_bar, pr.schedule, TOL,
                               max(1, args.cpu_sample_steps // 3), inner, inner_relax=args.inner_relax, eps=INNER_EPS)
    dt = time.perf_counter() - c0
    c_s = int(res.cycles.sum())
    t_full = dt * total_cycles / max(c_s, 1)
    desc = (f"first {res.steps} flexible Arnoldi steps of the source ({dt:.1f} s, {c_s} BiCGSTAB cycles), "
            f"scaled by the solve's {total_cycles} cycles")
    return len(pr.sigma) / t_full, dt, desc


def jacobian_cpu_sample(pr, args, ns):
    """The oracle on the Jacobian workload: a bounded sample of its solves
    (cpu_oracle_sample, scaled to the 1 + ns sources' shifted solves) and of its
    inner products (two (sensor, shift) pairs, scaled to all). Returns (rows/s,
    seconds spent, description)."""
    from oracle.sensitivity import sensitivities
    n_f = len(pr.sigma)
    v_s, dt_s, desc_s = cpu_oracle_sample(pr, max(1, args.cpu_sample_steps // 2), WORKLOAD_STEPS[2], INNER_EPS,
                                          args.inner_relax)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((2, pr.n)) + 1j * rng.standard_normal((2, pr.n))
    psi = rng.standard_normal((2, pr.n)) + 1j * rng.standard_normal((2, pr.n))
    c0 = time.perf_counter()
    for j in range(2):
        sensitivities(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask, pr.sigma[j], phi[j], psi[j])
    dt_ip = time.perf_counter() - c0
    t_ip = dt_ip / 2 * ns * n_f
    t_cpu = (1 + ns) * n_f / v_s + t_ip
    desc = (f"solves: {desc_s}, for 1 + {ns} sources; inner products: 2 of the {ns * n_f} (sensor, shift) "
            f"pairs timed ({dt_ip:.1f} s) and scaled")
    return 2 * ns * n_f / t_cpu, dt_s + dt_ip, desc


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Replicas:
    """N-GPU mode: every rank solves its own copy of the workload (the path does
    not shard, so there is no data-path collective). Only the bookkeeping is
    combined: a barrier around the timed region, the slowest rank's time and
    the sum of the ranks' certified solves. `device` holds the reduction
    buffers (the rank's GPU under NCCL, the CPU under gloo)."""

    def __init__(self, dist=None, world=1, device="cpu"):
        self.dist, self.world, self.device = dist, world, device

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.world == 1:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX if self.world > 1 else None)

    def sum(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM if self.world > 1 else None)

    def throughput(self, units, seconds):
        """Whole-job units per second: the units of all ranks over the slowest rank's time."""
        return self.sum(units) / self.max(seconds)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.p = None
        self.gpu = gpu_index
        # the raw samples go to FKS_CLOCKS_DIR (default: the system temp folder)
        d = os.environ.get("FKS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"fks_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(pr, sample_steps, workload_steps, eps, relax=0.0, total_cycles=None):
    """The oracle (complex128 NumPy/SciPy) on the first `sample_steps` flexible
    Arnoldi steps of the workload's first source, with the same inner-tolerance
    rule, extrapolated to a whole solve: by inner cycles when the whole solve's
    count is known (the multigrid cycles are most of the oracle's time),
    otherwise linearly in steps. Returns (solves/s, seconds, description)."""
    import oracle
    from oracle.gmg import Hierarchy, GMGInner
    t0 = time.perf_counter()
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    hier = Hierarchy(op, pr.tau_bar)
    b = pr.rhs()[:, 0]
    t_setup = time.perf_counter() - t0
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, TOL, sample_steps, GMGInner(hier, eps),
                               inner_relax=relax, eps=eps)
    dt = time.perf_counter() - t0
    c_sample = int(res.cycles.sum())
    if total_cycles and c_sample > 0:
        t_full = t_setup + (dt - t_setup) * total_cycles / c_sample
        how = f"scaled by inner cycles ({c_sample} of the solve's {total_cycles})"
    else:
        t_full = dt * workload_steps / max(res.steps, 1)
        how = f"scaled linearly to {workload_steps} steps" + (
            " (with a relaxed tolerance the first steps take the most cycles: an upper estimate)" if relax > 0 else "")
    desc = (f"oracle setup + first {res.steps} of {workload_steps} flexible Arnoldi steps of the first source "
            f"({dt:.1f} s), {how}")
    return len(pr.sigma) / t_full, dt, desc   # one source's shifted solves


class OracleModel:
    """Timed parts of the oracle's solve of a large workload, for a CPU baseline
    that a bounded sample can measure: the setup (operator and multigrid
    hierarchy), one inner cycle (defect and V-cycle on v_1 = b / ||b||), one
    flexible Arnoldi orthogonalisation (M z, then two Gram-Schmidt passes
    against k_avg basis vectors), and the final assembly x_j = Z y_j with its
    true residual (timed on a few shifts and scaled to n_f). A whole solve of S
    steps and C cycles is estimated as setup + C cycle + S orthogonalisation +
    final."""

    def __init__(self, pr, eps):
        import oracle
        from oracle.gmg import Hierarchy
        self.pr, self.eps = pr, eps
        t0 = time.perf_counter()
        self.op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
        self.hier = Hierarchy(self.op, pr.tau_bar)
        self.t_setup = time.perf_counter() - t0
        b = pr.rhs()[:, 0]
        self.b = b
        self.v1 = b / np.linalg.norm(b)
        self.calls = 0

    def cycle(self):
        """Seconds of one inner cycle (defect + V-cycle), taus in turn."""
        p = self.calls % len(self.pr.tau_bar)
        self.calls += 1
        t0 = time.perf_counter()
        self.hier.solve(self.v1, p, self.eps, 50, cycles=1)
        return time.perf_counter() - t0

    def outer(self, k_avg, k_final, shifts=4):
        """Seconds of one orthogonalisation at k_avg, and of the final assembly
        and true residual of all shifts at k_final steps (timed on `shifts`)."""
        import oracle
        rng = np.random.default_rng(0)
        n = self.op.n
        V = rng.standard_normal((n, k_avg + 1)) + 1j * rng.standard_normal((n, k_avg + 1))
        z = self.v1.copy()
        t0 = time.perf_counter()
        w = self.op.M @ z
        for _ in range(2):
            for i in range(k_avg):
                w -= np.vdot(V[:, i], w) * V[:, i]
        np.linalg.norm(w)
        t_orth = time.perf_counter() - t0
        Z = V[:, :k_final] if k_final <= k_avg + 1 else rng.standard_normal((n, k_final)) + 0j
        Y = rng.standard_normal((k_final, shifts)) + 1j * rng.standard_normal((k_final, shifts))
        sig = self.pr.sigma[:shifts]
        t0 = time.perf_counter()
        X = Z @ Y
        oracle.true_residuals(self.op, self.b, sig, X)
        t_final = (time.perf_counter() - t0) * len(self.pr.sigma) / shifts
        return t_orth, t_final

    def estimate(self, t_cycle, steps, cycles):
        t_orth, t_final = self.outer(max(1, steps // 2), steps)
        total = self.t_setup + cycles * t_cycle + steps * t_orth + t_final
        parts = {"setup_s": self.t_setup, "cycle_s": t_cycle, "orth_s_at_k_avg": t_orth, "final_s": t_final,
                 "steps": steps, "cycles": cycles}
        return total, parts


def oracle_model_sample(pr, n_cycles, steps, cycles, eps):
    """CPU baseline of a 3D workload: the oracle's timed parts (OracleModel),
    n_cycles inner cycles measured, scaled to a whole solve of `steps` Arnoldi
    steps and `cycles` inner cycles. Returns (solves/s, seconds, description)."""
    t0 = time.perf_counter()
    m = OracleModel(pr, eps)
    ts = [m.cycle() for _ in range(max(1, n_cycles))]
    t_cycle = statistics.median(ts)
    total, parts = m.estimate(t_cycle, steps, cycles)
    dt = time.perf_counter() - t0
    desc = (f"oracle setup, {len(ts)} inner multigrid cycles (median {t_cycle:.2f} s), one orthogonalisation "
            f"at k = {max(1, steps // 2)} and the final assembly + true residuals (timed on 4 shifts) of the first "
            f"source, {dt:.1f} s in all; scaled to a whole solve of {steps} steps and {cycles} cycles "
            f"(estimate {total:.1f} s)")
    return len(pr.sigma) / total, dt, desc


def _oracle_model_worker(job):
    """One process of the all-cores CPU baseline: its own oracle setup, then
    `reps` timed (cycle + outer parts) estimates; returns the best solves/s."""
    pr, steps, cycles, eps, reps = job
    m = OracleModel(pr, eps)
    best = None
    for _ in range(reps):
        total, _ = m.estimate(m.cycle(), steps, cycles)
        best = total if best is None else min(best, total)
    return len(pr.sigma) / best


def oracle_model_all_cores(pr, steps, cycles, eps, reps=3):
    """The same oracle model on every host core at once: one independent solve
    of the workload per core (spawned processes, one BLAS thread each), each the
    best of `reps` estimates; the value is their sum (throughput of a CPU that
    runs one solve per core). Cores are capped by host memory (about 5 GB per
    process at 128^3). Returns (solves/s, cores, seconds, description)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as fh:
            avail = next(int(l.split()[1]) * 1024 for l in fh if l.startswith("MemAvailable"))
        cores = max(1, min(cores, int(avail // (5 * 2 ** 30))))
    except (OSError, StopIteration, ValueError):
        pass
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        vals = pool.map(_oracle_model_worker, [(pr, steps, cycles, eps, reps)] * cores)
    dt = time.perf_counter() - t0
    desc = (f"{cores} concurrent processes (spawn, one BLAS thread each), each the oracle model of one solve "
            f"(setup, inner cycle, orthogonalisation, final assembly + true residuals as in cpu_baseline), best "
            f"of {reps}, scaled to {steps} steps and {cycles} cycles; value = sum over processes; {dt:.1f} s")
    return float(sum(vals)), cores, dt, desc


def direct_sample(pr, shifts=3):
    """The paper's "Direct" comparator (Section 6.1): a sparse LU factorisation
    and solve of K + sigma_j M per shift (SciPy SuperLU), timed on `shifts`
    shifts spread over the range and scaled to all n_f. Returns (solves/s,
    seconds, description)."""
    import oracle
    from oracle.direct import direct_solve
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    idx = np.unique(np.linspace(0, len(pr.sigma) - 1, shifts).round().astype(int))
    t0 = time.perf_counter()
    direct_solve(op, b, pr.sigma[idx])
    dt = time.perf_counter() - t0
    per = dt / len(idx)
    return 1.0 / per, dt, (f"SuperLU factorisation + solve of K + sigma_j M for {len(idx)} of {len(pr.sigma)} "
                           f"shifts ({dt:.1f} s, {per:.2f} s per shift), one source")


def blas_threads():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if k in os.environ:
            return int(os.environ[k])
    return 1


def run_reference(args):
    from paper_1212_3660_gb300 import synth
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == 6:
        pr = synth.workload(2, m_max=100)
        vals = []
        sample = None
        for i in range(args.warmup + args.steps):
            v, _, sample = jacobian_cpu_sample(pr, args, JAC_SENSORS)
            if i >= args.warmup:
                vals.append(v)
        value = statistics.median(vals)
        line = {"impl": "reference", "metric": "Jacobian rows/s at 1e-8 residual", "value": value, "unit": "rows/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * 2 * JAC_SENSORS * len(pr.sigma) / value, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
                "config": {"workload": f"jacobian-512x512-f{len(pr.sigma)}-s{JAC_SENSORS}",
                           "grid": "x".join(map(str, pr.shape[::-1])), "n_f": len(pr.sigma), "sensors": JAC_SENSORS},
                "cpu_baseline": {"value": value, "unit": "rows/s", "cores": blas_threads(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == 7:
        pr = synth.fe_workload()
        vals = []
        sample = None
        for i in range(args.warmup + args.steps):
            v, _, sample = csr_cpu_sample(pr, args, args.precond == "amg", CSR_CYCLES[args.precond])
            if i >= args.warmup:
                vals.append(v)
        value = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * len(pr.sigma) / value,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic", "config": {"workload": pr.name, "n": pr.n, "n_f": len(pr.sigma),
                                                "precond": args.precond},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload in (1, 2, 3, 4) and (args.workload, round(args.inner_relax, 6)) in ORACLE_SOLVE:
        # each step: one inner multigrid cycle of the oracle at the workload's
        # size; the value is the oracle's whole solve estimated from its timed
        # parts and its own step and cycle counts (OracleModel)
        pr = synth.workload(args.workload, m_max=100)
        steps_o, cycles_o = ORACLE_SOLVE[(args.workload, round(args.inner_relax, 6))]
        m = OracleModel(pr, INNER_EPS)
        ts = []
        for i in range(args.warmup + args.steps):
            t = m.cycle()
            if i >= args.warmup:
                ts.append(t)
        t_cycle = statistics.median(ts)
        total, parts = m.estimate(t_cycle, steps_o, cycles_o)
        n_src = len(pr.src_cells)
        value = len(pr.sigma) / total    # every source is an independent solve of the same cost
        sample = (f"one inner multigrid cycle per step (defect + V-cycle, median {t_cycle:.2f} s) of the first "
                  f"source; setup, one orthogonalisation at k = {max(1, steps_o // 2)} and the final assembly + "
                  f"true residuals timed once; whole solve estimated from the oracle's own {steps_o} steps and "
                  f"{cycles_o} cycles: {total:.1f} s")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_cycle,
                "step": "one inner multigrid cycle of the oracle (the measured unit; value is extrapolated)",
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic",
                "config": {"workload": pr.name, "grid": "x".join(map(str, pr.shape[::-1])), "n_f": len(pr.sigma),
                           "sources": n_src},
                "extrapolation": parts,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == 8:
        probs = [synth.make_problem(m_max=100, **g) for g in synth.mix2d_grids()]
        vals = []
        cpu = None
        for i in range(args.warmup + args.steps):
            cpu = mix2d_cpu_sample(probs, args, WORKLOAD_STEPS[2])
            if i >= args.warmup:
                vals.append(cpu["value"])
        value = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * sum(len(p.sigma) for p in probs) / value, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
                "config": {"workload": "2d-mix-32x(128..384)^2-f100-p4", "aquifers": len(probs),
                           "cells_total": int(sum(p.n for p in probs)), "n_f": len(probs[0].sigma)},
                "cpu_baseline": {**cpu, "value": value},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == 5:
        # the stream's first request stands for the stream
        # the stream's first request (its aquifer and shift count) stands for the stream
        aq, rq = synth.make_serving_stream(1, seed=3000)
        pr = synth.make_problem(m_max=100, **{**aq[rq[0]["aquifer"]], "n_f": rq[0]["n_f"]})
        pr.name = "serving-stream"
    else:
        pr = synth.workload(args.workload, m_max=100)
    ws = WORKLOAD_STEPS.get(args.workload, 40)
    vals, secs = [], []
    sample = None
    total_cycles = ORACLE_CYCLES.get((args.workload, round(args.inner_relax, 6)))
    for i in range(args.warmup + args.steps):
        v, dt, sample = cpu_oracle_sample(pr, max(1, args.cpu_sample_steps // 3), ws, INNER_EPS, args.inner_relax,
                                          total_cycles)
        if i >= args.warmup:
            vals.append(v)
            secs.append(dt)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * len(pr.sigma) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": pr.name, "grid": "x".join(map(str, pr.shape[::-1])), "n_f": len(pr.sigma)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def prec_of(name, fks):
    """fks precision of a --precision name."""
    return {"fp64": fks.FKS_PREC_FP64, "mixed": fks.FKS_PREC_MIXED, "bf16": fks.FKS_PREC_MIXED_BF16}[name]


def dtype_of(prec, fks):
    return {fks.FKS_PREC_FP64: "c128", fks.FKS_PREC_MIXED: "c64-inner/c128-outer",
            fks.FKS_PREC_MIXED_BF16: "c64-inner(bf16 coefficients)/c128-outer"}[prec]


def set_thresholds(fks, op, prec, args):
    """The multigrid launch thresholds given on the command line (instead of the
    autotuner's, e.g. for an ncu capture whose timings would mislead it)."""
    fks.fks_op_set_fusion(op, prec, args.fuse_max)
    if args.tile16_max is not None:
        fks.fks_op_set_tiles(op, prec, args.tile16_max)
    if args.tail_max is not None:
        fks.fks_op_set_tail(op, prec, args.tail_max)
    if args.cluster_max is not None:
        fks.fks_op_set_cluster(op, prec, args.cluster_max)
    if args.tile8_max is not None:
        fks.fks_op_set_tiles8(op, prec, args.tile8_max)
    fks.fks_op_set_coop(op, prec, args.coop_max or 0)


def batched_sample(args, local, dist, world):
    """The batched workload (3D 96^3, 64 well sources x 100 shifts, complex64
    cycles with complex128 outer work, relaxed inner tolerance): the sources
    advance in lockstep batches sized to free device memory, one CUDA graph per
    batch, tiles and z-chunks from the autotuner. Timed like the line itself
    (device-resident inputs, CUDA events on the library's stream)."""
    import torch

    from paper_1212_3660_gb300 import fks, synth
    from paper_1212_3660_gb300.solver import Solver
    pr = synth.workload(4, m_max=100)
    prec = fks.FKS_PREC_MIXED
    solver = Solver(pr, device=local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    n, n_f, n_rhs = pr.n, len(pr.sigma), len(pr.src_cells)
    b_d = torch.from_numpy(pr.rhs().T.copy()).to(dev)
    sig_d = torch.from_numpy(pr.sigma.astype(np.complex128)).to(dev)
    tau_d = torch.from_numpy(pr.tau_bar.astype(np.complex128)).to(dev)
    X_d = torch.empty((n_rhs, n_f, n), dtype=torch.complex128, device=dev)
    est = np.zeros((n_rhs, n_f)); bnd = np.zeros((n_rhs, n_f)); tru = np.zeros((n_rhs, n_f))
    mj = np.zeros((n_rhs, n_f), np.int32); sst = np.zeros((n_rhs, n_f), np.int32)
    opts, keep = fks.make_options(tol=TOL, m_max=pr.m_max, precision=prec, inner_tol=INNER_EPS,
                                  schedule=pr.schedule, inner_relax=args.inner_relax if args.inner_relax > 0 else 0.003)
    info, info_arr = fks.make_info(n_rhs, pr.m_max)
    fks.fks_op_autotune(solver.op, prec, complex(pr.tau_bar[len(pr.tau_bar) // 2]), sh)

    def step():
        return fks.fks_solve(solver.op, b_d, n_rhs, sig_d, n_f, tau_d, len(pr.tau_bar), opts, X_d, est, bnd, tru,
                             mj, sst, info, sh)

    step()
    reps = 2
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    conv = 0
    e0.record(stream)
    for _ in range(reps):
        step()
        conv += int(np.sum(tru <= TOL))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    out = {"value": conv / reps / (ms / 1000.0), "ms_per_step": ms, "precision": "mixed",
           "workload": pr.name, "sources": n_rhs, "n_f": n_f, "grid": "x".join(map(str, pr.shape[::-1])),
           "converged_per_step": conv / reps, "solves_per_step": n_f * n_rhs,
           "arnoldi_steps_max": int(info_arr["steps"].max()), "inner_cycles_total": int(info_arr["inner_cycles"].sum()),
           "steps_timed": reps, "tiling": list(fks.fks_op_tiling(solver.op, prec)),
           "coop_levels_max_cells": fks.fks_op_coop_max(solver.op, prec),
           "zchunks": fks.fks_op_zchunks(solver.op, prec)}
    del X_d
    solver.close()
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_1212_3660_gb300 import build, fks, synth
    from paper_1212_3660_gb300.solver import Solver

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()
    if args.no_pdl:
        fks.fks_set_pdl(0)
    if args.workload == 5:
        serve_bench(args, rank, world, local, dist)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == 6:
        jacobian_bench(args, rank, world, local, dist)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == 7:
        csr_bench(args, rank, world, local, dist)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == 8:
        mix2d_bench(args, rank, world, local, dist)
        if world > 1:
            dist.destroy_process_group()
        return
    pr = synth.workload(args.workload, m_max=100)
    prec = prec_of(args.precision, fks)
    t_setup0 = time.perf_counter()
    solver = Solver(pr, device=local)
    setup_ms = 1000 * (time.perf_counter() - t_setup0)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    n, n_f, n_rhs = pr.n, len(pr.sigma), len(pr.src_cells)
    if args.precond_cycles > 0:
        # the inner-solve kernels of this workload's operator, tuned as the
        # solve is (or with the thresholds given), on v = b / ||b|| (no basis,
        # no outputs on the device)
        if args.fuse_max is not None:
            set_thresholds(fks, solver.op, prec, args)
        else:
            fks.fks_op_autotune(solver.op, prec, complex(pr.tau_bar[len(pr.tau_bar) // 2]), sh)
        v = torch.from_numpy(pr.rhs()[:, 0] / np.linalg.norm(pr.rhs()[:, 0])).to(dev)
        z = torch.zeros_like(v)
        st, cyc, pn = fks.fks_precond_apply(solver.op, complex(pr.tau_bar[len(pr.tau_bar) // 2]), v, z, INNER_EPS,
                                            cycles=args.precond_cycles, precision=prec, stream=sh)
        torch.cuda.synchronize()
        print(json.dumps({"precond_cycles": cyc, "pnorm": pn, "tiling": list(fks.fks_op_tiling(solver.op, prec))}),
              flush=True)
        solver.close()
        return
    b_d = torch.from_numpy(pr.rhs().T.copy()).to(dev)
    sig_d = torch.from_numpy(pr.sigma.astype(np.complex128)).to(dev)
    tau_d = torch.from_numpy(pr.tau_bar.astype(np.complex128)).to(dev)
    X_d = torch.empty((n_rhs, n_f, n), dtype=torch.complex128, device=dev)
    est = np.zeros((n_rhs, n_f)); bnd = np.zeros((n_rhs, n_f)); tru = np.zeros((n_rhs, n_f))
    mj = np.zeros((n_rhs, n_f), np.int32); sst = np.zeros((n_rhs, n_f), np.int32)
    variant = fks.FKS_FFOM if args.variant == "ffom" else fks.FKS_FGMRES
    opts, keep = fks.make_options(tol=TOL, m_max=pr.m_max, precision=prec, inner_tol=INNER_EPS,
                                  schedule=pr.schedule, launch_mode=0 if args.launch_mode == "graph" else 1,
                                  inner_relax=args.inner_relax, variant=variant, restart_len=args.restart)
    # host-driven launches (identical kernels) for per-launch event timing
    opts_host, keep_host = fks.make_options(tol=TOL, m_max=pr.m_max, precision=prec, inner_tol=INNER_EPS,
                                            schedule=pr.schedule, launch_mode=1, inner_relax=args.inner_relax,
                                            variant=variant, restart_len=args.restart)
    info, info_arr = fks.make_info(n_rhs, pr.m_max)

    def step(b, X, o=opts):
        return fks.fks_solve(solver.op, b, n_rhs, sig_d, n_f, tau_d, len(pr.tau_bar), o, X, est, bnd, tru, mj,
                             sst, info, sh)

    replicas = Replicas(dist, world, dev)
    barrier, max_over_ranks, sum_over_ranks = replicas.barrier, replicas.max, replicas.sum

    if args.fuse_max is not None:
        set_thresholds(fks, solver.op, prec, args)
    if args.fuse_max is not None:
        tuned = args.fuse_max
    else:
        tuned = fks.fks_op_autotune(solver.op, prec, complex(pr.tau_bar[len(pr.tau_bar) // 2]), sh)
    if args.single:
        st = step(b_d, X_d)
        torch.cuda.synchronize()
        print(json.dumps({"single_solve_status": st, "converged": int(np.sum(tru <= TOL)),
                          "tiling": list(fks.fks_op_tiling(solver.op, prec))}), flush=True)
        solver.close()
        return
    for _ in range(args.warmup):
        step(b_d, X_d)
    # kernel-class survey (stderr only) and choice of the dominant class
    totals = {}
    for c, name in enumerate([] if args.no_survey else fks.KERNEL_CLASSES):
        fks.fks_profile_select(solver.op, c)
        step(b_d, X_d, opts_host)
        totals[name] = fks.fks_profile_read(solver.op)
    fks.fks_profile_select(solver.op, None)
    fks.fks_profile_read(solver.op)
    dominant = max(totals, key=lambda k: totals[k]["ms"]) if totals else None
    if args.survey and rank == 0:
        tot = sum(v["ms"] for v in totals.values())
        for k, v in sorted(totals.items(), key=lambda kv: -kv[1]["ms"]):
            print(f"# {k:9s} launches {v['launches']:7d} ms {v['ms']:9.3f} ({100 * v['ms'] / max(tot, 1e-9):5.1f}%) "
                  f"GB/s {v['bytes'] / max(v['ms'], 1e-9) / 1e6:8.1f} GFLOP/s {v['flops'] / max(v['ms'], 1e-9) / 1e6:8.1f}",
                  file=sys.stderr)

    # ---- timed region (device-resident inputs)
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except ValueError:
            pass
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    converged = 0
    with ClockSampler(gpu_index) as clk:
        barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("fks_timed")
        e0.record(stream)
        for _ in range(args.steps):
            step(b_d, X_d)
            converged += int(np.sum(tru <= TOL))
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
    launches = fks.fks_profile_read(solver.op)["all_launches"]
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms)
    conv_per_step = converged / args.steps
    value = sum_over_ranks(conv_per_step) / (ms_max / 1000.0)

    roof = None
    if dominant is not None:
        # ---- roofline of the dominant kernel class (events on the library's stream),
        # on the finest level where the class runs per level
        def timed_class(level):
            fks.fks_profile_select(solver.op, dominant, level)
            for _ in range(args.steps):
                step(b_d, X_d, opts_host)
            pr_ = fks.fks_profile_read(solver.op)
            fks.fks_profile_select(solver.op, None)
            return pr_
        roof_level = 0
        prof = timed_class(0)
        if prof["launches"] == 0:
            roof_level = -1
            prof = timed_class(-1)
        traffic, traffic_src = recorded_traffic(pr.name, args.precision, dominant, roof_level)
        hbm_peak, bf16_peak, peak_src = peaks()
        gbs = prof["bytes"] / max(prof["ms"], 1e-12) / 1e6
        tfl = prof["flops"] / max(prof["ms"], 1e-12) / 1e9
        f_hbm = gbs / hbm_peak
        f_alu = tfl / FP64_PEAK_TFLOPS if prec == fks.FKS_PREC_FP64 or dominant in ("mdot", "maxpy", "assemble",
                                                                                     "defect", "tres") else 0.0
        if f_alu > f_hbm:
            roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": f_alu,
                    "traffic": traffic, "kernel": dominant, "level": roof_level,
                    "peak_source": "FP64 nominal: 152 SMs x 2 DFMA/clk x 2.07 GHz",
                    "launches": prof["launches"], "avg_launch_us": 1000 * prof["ms"] / max(prof["launches"], 1),
                    "hbm_frac_of_" + peak_src: f_hbm}
        else:
            roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": f_hbm, "traffic": traffic,
                    "kernel": dominant, "level": roof_level, "peak_source": peak_src, "launches": prof["launches"],
                    "avg_launch_us": 1000 * prof["ms"] / max(prof["launches"], 1)}

    def end_to_end():
        # pinned host buffers allocated as such (page-locked at allocation)
        b_h = torch.empty((n_rhs, n), dtype=torch.complex128, pin_memory=True)
        b_h.copy_(torch.from_numpy(pr.rhs().T.copy()))
        X_h = torch.empty((n_rhs, n_f, n), dtype=torch.complex128, pin_memory=True)
        step(b_h, X_h)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv_e2e = 0
        for _ in range(args.steps):
            step(b_h, X_h)
            conv_e2e += int(np.sum(tru <= TOL))
        torch.cuda.synchronize()
        t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps)
        e2e_value = sum_over_ranks(conv_e2e / args.steps) / t_e2e
        h2d = b_h.numel() * 16 + (n_f + len(pr.tau_bar)) * 16
        d2h = X_h.numel() * 16 + n_rhs * n_f * (8 * 3 + 4 * 2)
        return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end()

    main_info = {k: v.copy() for k, v in info_arr.items()}   # this line's solve, before the variants

    # ---- convergence monitors (Section 3): one more solve exporting H_bar and
    # tau_k (Prop. 3's alpha comes from the Givens update at no extra launch),
    # then Prop. 1's Ritz values of every source on the GPU
    mon_info, mon_arr = fks.make_info(n_rhs, pr.m_max, n_f)
    mon_opts = opts
    if args.restart > 0:   # restarted solves export no monitors: take them from one unrestarted solve
        mon_opts, mon_keep = fks.make_options(tol=TOL, m_max=pr.m_max, precision=prec, inner_tol=INNER_EPS,
                                              schedule=pr.schedule, inner_relax=args.inner_relax, variant=variant)
    fks.fks_solve(solver.op, b_d, n_rhs, sig_d, n_f, tau_d, len(pr.tau_bar), mon_opts, X_d, est, bnd, tru, mj, sst,
                  mon_info, sh)
    theta = np.zeros((n_rhs, pr.m_max), np.complex128)
    rstat = np.zeros(n_rhs, np.int32)
    steps_m = np.ascontiguousarray(mon_arr["steps"])
    fks.fks_ritz(solver.ctx, mon_arr["hbar"], mon_arr["tau_k"], steps_m, n_rhs, pr.m_max, theta, rstat, sh)
    r0 = time.perf_counter()
    fks.fks_ritz(solver.ctx, mon_arr["hbar"], mon_arr["tau_k"], steps_m, n_rhs, pr.m_max, theta, rstat, sh)
    ritz_ms = 1000 * (time.perf_counter() - r0)
    k0 = int(steps_m[0])
    monitors = {"ritz_ms": ritz_ms, "ritz_status": rstat.tolist(), "ritz_steps": k0,
                "ritz_real_range": [float(theta[0, :k0].real.min()), float(theta[0, :k0].real.max())] if k0 else None,
                "max_gmres_alpha": float(np.max(mon_arr["gmres_alpha"])),
                "note": "Prop. 3's alpha is recorded by the Givens update; the Ritz values (sigma = 0) take one "
                        "launch of one warp per source, timed here with its host copies"}

    # ---- the same workload in the paper's plain configuration (complex128,
    # fixed inner tolerance) and in the mixed, relaxed one, on this GPU
    def variant(v_prec, v_relax, reps=3, warm=2):
        if v_prec == prec and v_relax == args.inner_relax:
            return None
        o_v, keep_v = fks.make_options(tol=TOL, m_max=pr.m_max, precision=v_prec, inner_tol=INNER_EPS,
                                       schedule=pr.schedule, inner_relax=v_relax)
        fks.fks_op_autotune(solver.op, v_prec, complex(pr.tau_bar[len(pr.tau_bar) // 2]), sh)
        for _ in range(warm):
            step(b_d, X_d, o_v)
        barrier()
        torch.cuda.synchronize()
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        conv_v = 0
        v0.record(stream)
        for _ in range(reps):
            step(b_d, X_d, o_v)
            conv_v += int(np.sum(tru <= TOL))
        v1.record(stream)
        torch.cuda.synchronize()
        ms_v = max_over_ranks(v0.elapsed_time(v1) / reps)
        return {"value": sum_over_ranks(conv_v / reps) / (ms_v / 1000.0), "ms_per_step": ms_v,
                "precision": {0: "fp64", 1: "mixed", 2: "bf16"}[v_prec], "inner_relax": v_relax,
                "inner_cycles_total": int(info_arr["inner_cycles"].sum()), "steps_timed": reps}
    comparison = None
    if args.workload in (1, 2, 3, 4) and not args.no_compare:
        comparison = {"this_line": {"value": value, "precision": args.precision, "inner_relax": args.inner_relax},
                      "plain_fp64_fixed_eps": variant(fks.FKS_PREC_FP64, 0.0),
                      "fp64_relaxed": variant(fks.FKS_PREC_FP64, args.inner_relax if args.inner_relax > 0 else 0.003),
                      "mixed_relaxed": variant(fks.FKS_PREC_MIXED, args.inner_relax if args.inner_relax > 0 else 0.003),
                      "bf16_smoother_relaxed": variant(fks.FKS_PREC_MIXED_BF16,
                                                       args.inner_relax if args.inner_relax > 0 else 0.003)}
        # restore this line's tuning for what follows
        fks.fks_op_autotune(solver.op, prec, complex(pr.tau_bar[len(pr.tau_bar) // 2]), sh)

    cpu = None
    cpu_all = None
    direct = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ws = int(main_info["steps"].max()) or WORKLOAD_STEPS.get(args.workload, 40)
        cyc0 = int(main_info["inner_cycles"][:pr.m_max].sum())
        if len(pr.shape) == 3:
            v, dt, desc = oracle_model_sample(pr, args.cpu_sample_cycles, int(main_info["steps"][0]) or ws, cyc0,
                                              INNER_EPS)
            desc += " (the GPU solve's step and cycle counts)"
            if not args.no_cpu_all_cores:
                va, ca, _, adesc = oracle_model_all_cores(pr, int(main_info["steps"][0]) or ws, cyc0, INNER_EPS)
                cpu_all = {"value": va, "unit": UNIT, "cores": ca, "kind": "oracle, one solve per core",
                           "sample": adesc}
        else:
            v, dt, desc = cpu_oracle_sample(pr, args.cpu_sample_steps, ws, INNER_EPS, args.inner_relax, cyc0)
        cpu = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle", "sample": desc}
        if len(pr.shape) == 2:
            dv, _, ddesc = direct_sample(pr)
            direct = {"value": dv, "unit": UNIT, "cores": blas_threads(), "kind": "direct (paper's comparator)",
                      "sample": ddesc}
        else:
            direct = {"value": None, "note": "not timed: a SuperLU factorisation of a 3D operator of this size "
                                             "(seven-point stencil, millions of unknowns) per shift does not fit "
                                             "a bounded sample"}

    if roof is not None:
        roof["alg_bytes_per_launch"] = prof["bytes"] / max(prof["launches"], 1)
        roof["traffic_source"] = ("profiles/traffic.md (ncu, sources " + traffic_src + ")") if traffic is not None \
            else ("stale: kernels changed since the ncu capture" if traffic_src else "no ncu capture recorded")
    tiling = fks.fks_op_tiling(solver.op, prec)
    zchunks = fks.fks_op_zchunks(solver.op, prec) if len(pr.shape) == 3 else None
    coop_max = fks.fks_op_coop_max(solver.op, prec)
    # ---- the batched workload (3D 96^3, 64 well sources) beside the 128^3 line
    batched = None
    if args.workload == 3 and not args.no_compare and not args.no_batched:
        del X_d, b_d
        solver.close()
        torch.cuda.empty_cache()
        batched = batched_sample(args, local, dist, world)
    else:
        solver.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype_of(prec, fks),
                "data": "synthetic",
                "config": {"workload": pr.name, "grid": "x".join(map(str, pr.shape[::-1])), "n": n, "n_f": n_f,
                           "n_p": len(pr.tau_bar), "schedule": "cycled", "sources_per_gpu": n_rhs,
                           "inner": (f"multigrid V(2,2) red-black GS, defect correction to eps={INNER_EPS:g}"
                                     + (f", relaxed: eps_k = min(1e-3, max(eps, {args.inner_relax:g} tol / R_k-1))"
                                        if args.inner_relax > 0 else "")),
                           "precision": args.precision, "parallelism": f"replicas{world}",
                           "l2": "working set larger than L2 (basis V, Z: 2 x 101 x n x 16 B)",
                           "arnoldi_steps": int(main_info["steps"].max()),
                           "inner_cycles_total": int(main_info["inner_cycles"].sum()),
                           "op_setup_ms": setup_ms, "fused_levels_max_cells": tuned,
                           "tile16_levels_max_cells": tiling[1], "tail_levels_max_cells": tiling[2],
                           "cluster_levels_max_cells": tiling[3], "tile8_levels_max_cells": tiling[4],
                           "zchunk_planes_per_level": zchunks,
                           "coop_levels_max_cells": coop_max,
                           "launch_mode": args.launch_mode, "variant": args.variant,
                           "restart_len": args.restart,
                           "basis_bytes_per_source": (2 * (args.restart or pr.m_max) + 1) * n * 16},
                "solves_per_step": n_f * n_rhs, "converged_per_step": conv_per_step,
                "e2e": e2e, "comparison": comparison, "monitors": monitors,
                "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "direct_baseline": direct,
                "clocks": clk.summary(),
                "gpu_launches": launches}
        if batched is not None and line["comparison"] is not None:
            line["comparison"]["batched_workload4"] = batched
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
