"""Benchmark: shifted-COCG Green's-function columns x energies per second on GB300.

Workload "sampled_columns_mixed": a 64x64x128 grid, h = 0.4 bohr, 4th-order stencil, 200 seeded
Gaussian wells, 256 unit right-hand sides sampled from the two outer planes, 128 energies in
[-0.5, 0.5] Ha with eta = 1e-3 Ha, tolerance 1e-6.  One step solves the next ``--cols-per-step``
columns of the 256-column sample to convergence for all 128 energies (steps cycle through the
sample) with one call of the library's shifted COCG (rsfd_shifted_cocg).  Every seed SpMV, seed
update, dot product, scalar recurrence, shift update and the G0_bb write-out of a step runs in the
library's kernels.

Precision: double-float Krylov vectors (``df64``, FP32 hi + lo pairs, FP64 scalars) by default.
Plain complex64 vectors (``--precision mixed``) cannot reach tol 1e-6 on this workload: at
eta = 1e-3 the FP32 SpMV rounding floors the residual near eps_32 * kappa (kappa ~ 5e4).

Output: one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead (bounded
sample, see below).  Under torchrun (N > 1) every rank solves its own columns (weak scaling,
no collective on the data path); the step time is the maximum over ranks.
"""

from __future__ import annotations

import os

# the CPU oracle leg is timed single-threaded (the "cores" it reports); pin the host BLAS pools before
# numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "sampled_columns_mixed"
METRIC = "greens_fn_columns_x_energies_per_s"
UNIT = "columns*energies/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if _cuda() else "gloo")
    return world, rank, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def rank_columns(p, rank):
    """Columns of one rank: the workload's own sample on rank 0, a rank-specific sample otherwise."""
    from workloads import sample_plane_columns
    if rank == 0:
        return p.cols
    return sample_plane_columns(p.grid, p.cols.size, seed=p.seed + 7919 * rank)


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# ---------------------------------------------------------------------------------------------
def oracle_sample(p, budget_s=15.0):
    """Time the oracle's shifted COCG (as it stands) on one column of the workload for a bounded
    number of iterations; return seconds per seed iteration and the sample description."""
    from oracle.cocg import shifted_cocg
    from oracle.operator import hamiltonian, apply_h, boundary_rows
    Hloc, P, wE = hamiltonian(p)
    rows = boundary_rows(p.grid, p.n_face)
    Z = p.energies + 1j * p.eta
    b = np.zeros(p.N, np.complex128)
    b[int(p.cols[0])] = 1.0
    f = lambda v: apply_h(Hloc, P, wE, v)
    t0 = time.perf_counter()
    shifted_cocg(f, b, Z, p.tol, rows=rows, maxit=5)
    t_probe = (time.perf_counter() - t0) / 5.0
    iters = max(10, int(budget_s / max(t_probe, 1e-6)))
    t0 = time.perf_counter()
    r = shifted_cocg(f, b, Z, p.tol, rows=rows, maxit=iters)
    dt = time.perf_counter() - t0
    return dt / max(r.iterations, 1), r.iterations, dt


def _oracle_worker(job):
    """One host core's share of the all-cores oracle sample (a spawned process): the workload rebuilt
    from its seed, one column, the same bounded sample as the single-core leg."""
    name, col_index, budget_s = job
    from workloads import make_problem
    p = make_problem(name)
    p.cols = np.asarray(p.cols)[[col_index % len(p.cols)]]
    return oracle_sample(p, budget_s)


def oracle_all_cores(p, budget_s, ncores=None):
    """The oracle as it stands on every host core at once: one spawned process per core, each timing its
    own column (columns are independent).  Returns seed iterations per second summed over the cores,
    the core count and the per-process samples."""
    import multiprocessing as mp
    n = int(ncores or os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(p.name, i, budget_s) for i in range(n)])
    return sum(1.0 / r[0] for r in res), n, res


def _oracle_iterations_per_column(p):
    """Seed iterations per column of this workload, as stored by tests/golden/make_golden.py from
    the oracle itself (None when absent)."""
    path = os.path.join(ROOT, "tests", "golden", f"{p.name}_oracle_iterations.json")
    if os.path.exists(path):
        return json.load(open(path))
    return None


def cpu_baseline_line(p, budget_s, gpu_mean_iters=None, all_cores=False):
    t_it, n_it, dt = oracle_sample(p, budget_s)
    stored = _oracle_iterations_per_column(p)
    if stored is not None:
        iters_per_col, src = float(stored["mean_iterations"]), "oracle's own iteration count (tests/golden)"
    elif gpu_mean_iters is not None:
        iters_per_col, src = float(gpu_mean_iters), "mean iteration count of this run"
    else:
        iters_per_col, src = float("nan"), "unknown"
    value = p.K / (t_it * iters_per_col)
    line = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"1 column x {p.K} energies, first {n_it} seed iterations ({dt:.1f} s, numpy/scipy "
                       f"single-threaded, host nproc={os.cpu_count()}), scaled to {iters_per_col:.0f} "
                       f"iterations per column ({src})")}
    if all_cores:
        try:
            rate, n, res = oracle_all_cores(p, budget_s)
            line["all_cores"] = {"value": p.K * rate / iters_per_col, "unit": UNIT, "cores": n, "kind": "oracle",
                                 "sample": (f"{n} spawned processes, one column each, {min(r[1] for r in res)}-"
                                            f"{max(r[1] for r in res)} seed iterations in about {budget_s:.0f} s "
                                            f"each, iteration rates summed, scaled like the single-core figure")}
        except Exception as exc:   # the single-core figure stands without it
            line["all_cores"] = {"value": None, "error": f"{type(exc).__name__}: {exc}"[:200]}
    return line


# ---------------------------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import paper_1502_00081_gb300 as rs
    from workloads import make_problem

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    rs.load_library()
    p = make_problem(args.workload)
    if args.precision:
        p.precision = args.precision
    if args.maxit:
        p.maxit = args.maxit
    if args.ncols:
        p.cols = p.cols[:args.ncols]
    all_cols = rank_columns(p, rank)
    if args.ncols:
        all_cols = all_cols[:args.ncols]
    B = min(args.cols_per_step, all_cols.size) if args.cols_per_step > 0 else all_cols.size
    batches = [np.roll(all_cols, -B * i)[:B] for i in range(max(1, all_cols.size // B))]
    cols = batches[0]
    prec = {"mixed": rs.RSFD_MIXED, "fp64": rs.RSFD_FP64, "df64": rs.RSFD_DF64}[p.precision]
    vsz = 8 if prec == rs.RSFD_MIXED else 16
    h = rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, proj=p.proj, precision=prec)
    rs.rsfd_set_solve_options(h.ptr, slots=args.slots, iters_per_sync=args.iters_per_sync, tile_y=args.tile_y,
                              z_chunk=args.z_chunk, pass_kind=args.pass_kind, prefetch=args.prefetch, profile=1,
                              reg_budget=args.reg_budget)
    tuned = None
    if not args.no_autotune:
        # launch options picked by the library's autotuner for this block width (not timed)
        topts, tus = rs.rsfd_autotune(h.ptr, p.energies, p.eta, slots=int(cols.size), iters=256)
        tuned = {"pass_kind": topts["pass_kind"], "tile_y": topts["tile_y"], "rows_per_thread": topts["rows_per_thread"],
                 "prefetch": topts["prefetch"],
                 "z_chunk": topts["z_chunk"], "iters_per_sync": topts["iters_per_sync"],
                 "reg_budget": topts["reg_budget"], "tile_x": topts["tile_x"], "us_per_slot_iteration": tus}
    G0 = torch.zeros((p.K, cols.size, h.nb), dtype=h.complex_dtype, device="cuda")
    stream = torch.cuda.current_stream()

    step_no = [0]

    def step():
        c = batches[step_no[0] % len(batches)]
        step_no[0] += 1
        st, info, res = rs.rsfd_shifted_cocg(h.ptr, c, p.energies, p.eta, p.tol, p.maxit, G0)
        return st, info

    for _ in range(args.warmup):
        st, info = step()
    # timed region
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    _barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    agg = {"ms_pass": 0.0, "ms_shift": 0.0, "slot_iterations": 0, "shift_updates": 0, "shift_slot_chunks": 0,
           "n_pass": 0, "n_shift": 0, "n_other": 0, "ms_combine": 0.0}
    statuses, iters = [], []
    for _ in range(args.steps):
        st, info = step()
        statuses.append(st)
        iters.append(float(info["iters"].mean()))
        s = rs.rsfd_get_stats(h.ptr)
        for k in agg:
            agg[k] += s[k]
        slots_used = s["slots"]
    ev1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop() if sampler else None
    ms_max = _max_over_ranks(ms, world)
    units = _sum_over_ranks(float(cols.size * p.K * args.steps), world)
    value = units / (ms_max / 1e3)

    # roofline of the dominant kernel (algorithmic bytes / summed event-timed duration)
    N, nb, K = p.N, h.nb, p.K
    # fused pass: read r_{n-1}, r_{n-2}, write r_n per slot-iteration, plus V once per launch
    kind_used = tuned["pass_kind"] if tuned else args.pass_kind
    launches_per_iter = 2 if kind_used in (3, 4) else 1   # the split passes: combine + stencil launches
    iter_launches = agg["n_pass"] / launches_per_iter     # seed iterations launched (all slots at once)
    pass_bytes = agg["slot_iterations"] * (3 * vsz * N) + iter_launches * (vsz // 2) * N
    proj_bytes_per_it = 0
    if p.proj is not None:
        # separable projectors (timed with the pass): the gather c_a = h^3 p_a^T r reads r, the value and
        # the index of every entry; the scatter reads and writes A r on the union of the supports and
        # reads every entry's value and atom index
        nnz = int(p.proj.nnz)
        n_supp = int(np.unique(p.proj.idx).size)
        s_p = vsz // 2
        proj_bytes_per_it = nnz * (vsz + s_p + 8) + n_supp * 2 * vsz + nnz * (s_p + 4)
        pass_bytes += agg["slot_iterations"] * proj_bytes_per_it
    # collapsed shift update: read and write x_b, p_b of K energies once per (slot, collapse) and read
    # the recorded boundary rows of the residuals once
    hsz = 16 if prec == rs.RSFD_FP64 else 8
    shift_bytes = agg["shift_slot_chunks"] * K * 4 * vsz * nb + agg["slot_iterations"] * hsz * nb
    peak, peak_src = _peaks()
    kern = {"pass": (pass_bytes, agg["ms_pass"]), "shift": (shift_bytes, agg["ms_shift"])}
    split = None
    if kind_used in (3, 4) and agg["ms_combine"] > 0:
        # the split pass's two launches against their own algorithmic bytes: the combine reads r_{n-1},
        # r_{n-2}, A r_{n-1} and writes r_n (4 v N); the stencil reads r_n and writes A r_n (2 v N, plus
        # the potential once per launch and the projector terms)
        cb = agg["slot_iterations"] * 4 * vsz * N
        sb = pass_bytes - agg["slot_iterations"] * 3 * vsz * N + agg["slot_iterations"] * 2 * vsz * N
        cms, sms = agg["ms_combine"], agg["ms_pass"] - agg["ms_combine"]
        split = {"combine": {"alg_bytes": cb, "ms": cms, "GBps": cb / (cms / 1e3) / 1e9,
                             "frac": cb / (cms / 1e3) / 1e9 / _peaks()[0]},
                 "stencil": {"alg_bytes": sb, "ms": sms, "GBps": sb / (sms / 1e3) / 1e9,
                             "frac": sb / (sms / 1e3) / 1e9 / _peaks()[0]}}
    dom = max(kern, key=lambda k: kern[k][1])
    dbytes, dms = kern[dom]
    achieved = dbytes / (dms / 1e3) / 1e9 if dms > 0 else None
    # measured DRAM bytes (ncu, one launch of this kernel on this workload and precision), stored per
    # slot-iteration and scaled to this run's average launch
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile) and agg["n_pass"] > 0:
        try:
            t = json.load(open(tfile)).get(dom)
            lo = tuned or {"tile_y": args.tile_y, "z_chunk": args.z_chunk}
            if (t and t.get("workload") == p.name and t.get("precision") == p.precision
                    and t.get("tile_y") == lo.get("tile_y") and t.get("z_chunk") == lo.get("z_chunk")
                    and t.get("pass_kind", 2) == (kind_used or 2)):
                traffic = t["bytes_per_slot_iteration"] * agg["slot_iterations"] / iter_launches
        except Exception:
            traffic = None

    # end to end through the public API with host buffers: V_loc from pinned host memory into a new
    # handle, the solve, and G0_bb back into pinned host memory, every step
    e2e = None
    if not args.no_e2e:
        Vh = torch.from_numpy(np.ascontiguousarray(p.V.ravel())).pin_memory()
        Gh = torch.empty(G0.shape, dtype=G0.dtype).pin_memory()
        e_steps = max(1, args.e2e_steps)
        _barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            h2 = rs.Handle(p.grid, p.h, p.fd_order, Vh.numpy(), n_face=p.n_face, proj=p.proj, precision=prec)
            rs.rsfd_set_solve_options(h2.ptr, slots=args.slots, iters_per_sync=args.iters_per_sync)
            if not args.no_autotune:
                rs.rsfd_autotune(h2.ptr, p.energies, p.eta, slots=int(cols.size), iters=256)   # cached
            G2 = torch.empty_like(G0)
            rs.rsfd_shifted_cocg(h2.ptr, cols, p.energies, p.eta, p.tol, p.maxit, G2)
            Gh.copy_(G2, non_blocking=True)
            torch.cuda.synchronize()
            h2.close()
            del G2
        dt = time.perf_counter() - t0
        dt_max = _max_over_ranks(dt, world)
        e_units = _sum_over_ranks(float(cols.size * p.K * e_steps), world)
        e2e = {"value": e_units / dt_max, "unit": UNIT, "h2d_bytes_per_step": int(Vh.numel() * 8 + cols.size * 8 + K * 8),
               "d2h_bytes_per_step": int(Gh.numel() * Gh.element_size()), "steps": e_steps}

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_line(p, args.cpu_budget, gpu_mean_iters=statistics.mean(iters),
                                all_cores=not args.no_cpu_all_cores)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {rs.RSFD_MIXED: "c64+f64", rs.RSFD_FP64: "c128", rs.RSFD_DF64: "df64(c64x2)+f64"}[prec], "data": "synthetic",
        "config": {"workload": p.name, "grid": list(p.grid), "h": p.h, "fd_order": p.fd_order,
                   "columns_per_step": int(cols.size), "columns_in_sample": int(all_cols.size),
                   "batching": "each step solves the next columns_per_step columns of the sample",
                   "energies": K, "eta": p.eta, "tol": p.tol,
                   "precision": p.precision, "boundary_rows": nb, "slots": slots_used,
                   "l2": "inputs larger than L2 (Krylov vectors of all slots: "
                         f"{3 * vsz * N * slots_used / 1e6:.0f} MB > 126 MB)",
                   "parallelism": f"columns over {world} GPU(s), no collective",
                   "launch_options": tuned if tuned else "defaults"},
        "status": [int(x) for x in statuses], "mean_iterations_per_column": statistics.mean(iters),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "alg_bytes_per_slot_iteration": 3 * vsz * N + proj_bytes_per_it,
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_source": peak_src,
                     "kernels": {k: {"alg_bytes": v[0], "ms": v[1],
                                     "GBps": (v[0] / (v[1] / 1e3) / 1e9) if v[1] > 0 else None}
                                 for k, v in kern.items()},
                     "split_launches": split},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(agg["n_pass"] + agg["n_shift"] + agg["n_other"]),
    }
    print(json.dumps(out), flush=True)
    h.close()


def run_reference(args):
    """The oracle, as it stands, on the host cores: each step is a bounded sample of the workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from workloads import make_problem
    p = make_problem(args.workload)
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(p, budget_s=min(budget, 5.0))
    vals, descr = [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        line = cpu_baseline_line(p, budget)
        vals.append(line["value"])
        descr = line
    dt = time.perf_counter() - t0
    value = statistics.mean(vals)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": p.name, "grid": list(p.grid), "h": p.h, "fd_order": p.fd_order,
                      "columns_per_step": min(args.cols_per_step, int(p.cols.size)) if args.cols_per_step > 0
                      else int(p.cols.size), "columns_in_sample": int(p.cols.size),
                      "energies": p.K, "eta": p.eta, "tol": p.tol,
                      "sample": "each step times a bounded number of seed iterations of one column"},
           "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": descr["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_shift_scaling(args):
    """Shift-scaling experiment (the GPU analogue of the paper's Fig. 2, Sec. IV): seconds and seed
    iterations of one shifted-COCG solve over K energies against K independent single-energy solves
    (K = 1 reduces shifted COCG to COCG), on the workload's grid, for --ncols columns.  One JSON line
    per (K, form)."""
    import torch
    import paper_1502_00081_gb300 as rs
    from workloads import make_problem
    torch.cuda.set_device(0)
    rs.load_library()
    p = make_problem(args.workload)
    prec = {"mixed": rs.RSFD_MIXED, "fp64": rs.RSFD_FP64, "df64": rs.RSFD_DF64}[args.precision]
    cols = p.cols[:args.ncols or 8]
    h = rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, proj=p.proj, precision=prec)
    G0 = torch.zeros((p.K, cols.size, h.nb), dtype=h.complex_dtype, device="cuda")

    def solve(E):
        G = G0[:len(E)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info, res = rs.rsfd_shifted_cocg(h.ptr, cols, np.asarray(E), p.eta, p.tol, p.maxit, G)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, st, info

    solve(p.energies[:1])   # warm-up (graph capture, workspace)
    for K in (1, 8, 32, 128):
        idx = np.linspace(0, p.K - 1, K).round().astype(int) if K > 1 else np.array([p.K // 2])
        E = p.energies[idx]
        dt, st, info = solve(E)
        print(json.dumps({"experiment": "shift_scaling", "form": "shifted", "K": K, "columns": int(cols.size),
                          "seconds": dt, "status": int(st), "mean_seed_iterations": float(info["iters"].mean()),
                          "mean_switches": float(info["switches"].mean()), "precision": args.precision}), flush=True)
        if K <= args.max_independent:
            tot, its = 0.0, []
            for e in E:
                dt1, st1, info1 = solve([e])
                tot += dt1
                its.append(float(info1["iters"].mean()))
            print(json.dumps({"experiment": "shift_scaling", "form": "independent", "K": K, "columns": int(cols.size),
                              "seconds": tot, "mean_iterations_per_energy": float(np.mean(its)),
                              "total_iterations_per_column": float(np.sum(its)), "precision": args.precision}),
                  flush=True)
    h.close()


def _golden(name):
    path = os.path.join(ROOT, "tests", "golden", f"{name}_golden.npz")
    return np.load(path) if os.path.exists(path) else None


def run_precision_speedup(args):
    """Reduced-precision forms against the plain FP64 GPU form, with errors taken against stored
    oracle values (tests/golden, written by tests/golden/make_golden.py, which calls only the oracle).

    * tiny_wire_fp64 (8x8x12, 2nd order, 3 wells, all 128 plane columns, 8 energies, eta = 1e-3): the
      full pipeline per form -- shifted COCG of every boundary column, Dyson with the closed-form lead
      self-energies, T -- every form stopped at tol 1e-6 (and the FP64 form also at the configuration's
      1e-12); G_bb and T errors against the oracle's dense (Z - H - Sigma)^{-1} and its T.
    * sampled_columns_mixed (64x64x128, 4th order, 128 energies, eta = 1e-3): the bench's first block of
      --cols-per-step columns solved by each form at tol 1e-8 (at the workload's 1e-6 every form, FP64
      included, stops about 1e-4 from the converged G0_bb, since the error is about tol / eta); G0_bb
      error on the stored oracle rows of the stored columns (oracle at tol 1e-10).  complex64 vectors stall near eps_32 * kappa here, so that
      form is capped at 40 000 iterations and reported as not converged.
    One JSON line per (workload, form); speedup_vs_fp64 is given where the form meets the mixed-mode
    tolerances (G_bb or G0_bb error <= 1e-5, |dT| <= 1e-4)."""
    import torch
    import paper_1502_00081_gb300 as rs
    from workloads import make_problem
    torch.cuda.set_device(0)
    rs.load_library()
    forms = (("fp64", rs.RSFD_FP64), ("df64", rs.RSFD_DF64), ("mixed", rs.RSFD_MIXED))

    g1 = _golden("tiny_wire_fp64")
    if g1 is not None:
        p = make_problem("tiny_wire_fp64")
        SLh, SRh = rs.rsfd_lead_sigma_uniform(p.grid[0], p.grid[1], p.h, p.fd_order, p.energies, p.eta)
        Go, To = g1["G_bb"], g1["T"]

        def run1(prec, tol_run, reps=3):
            with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=prec) as h:
                assert np.array_equal(np.asarray(h.rows), g1["rows"])
                cols = np.asarray(h.rows)
                G0 = torch.zeros((p.K, cols.size, h.nb), dtype=h.complex_dtype, device="cuda")
                SL, SR = torch.from_numpy(SLh).cuda(), torch.from_numpy(SRh).cuda()
                G = torch.empty_like(G0)
                best = None
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    st, info, res = rs.rsfd_shifted_cocg(h.ptr, cols, p.energies, p.eta, tol_run, 200000, G0)
                    torch.cuda.synchronize()
                    t1 = time.perf_counter()
                    rs.rsfd_dyson_boundary(h.ptr, G0, SL, SR, G)
                    T = rs.rsfd_transmission(h.ptr, G, SL, SR)
                    torch.cuda.synchronize()
                    t = (time.perf_counter() - t0, t1 - t0)
                    best = t if best is None or t[0] < best[0] else best
                Gm = G.cpu().numpy().astype(np.complex128).transpose(0, 2, 1)
                return best, int(st), float(info["iters"].mean()), np.asarray(T), Gm

        base = None
        for name, prec in forms:
            for tol_run in ((1e-6, 1e-12) if name == "fp64" else (1e-6,)):
                (tot, cocg), st, its, T, G = run1(prec, tol_run)
                dT = float(np.abs(T - To).max())
                gerr = float(max(np.linalg.norm(G[k] - Go[k]) / np.linalg.norm(Go[k]) for k in range(p.K)))
                ok = st == 0 and dT <= 1e-4 and gerr <= 1e-5
                if name == "fp64" and tol_run == 1e-6:
                    base = tot
                print(json.dumps({"experiment": "precision_speedup", "workload": p.name, "precision": name,
                                  "tol": tol_run, "status": st, "seconds": tot, "cocg_seconds": cocg,
                                  "columns": int(G.shape[2]), "energies": p.K, "mean_seed_iterations": its,
                                  "max_abs_dT": dT, "G_bb_rel_err_max": gerr,
                                  "reference": "oracle dense (Z - H - Sigma)^-1 and T (tests/golden)",
                                  "meets_tolerances": ok,
                                  "speedup_vs_fp64": (base / tot) if ok and base and tol_run == 1e-6 else None}),
                      flush=True)

    g2 = _golden("sampled_columns_mixed")
    if g2 is not None:
        p = make_problem("sampled_columns_mixed")
        B = args.cols_per_step if args.cols_per_step > 0 else 38
        batch = p.cols[:B]
        gcols, rows, Gref = g2["cols"], g2["rows"], g2["G0"]
        pos = [int(np.where(batch == c)[0][0]) for c in gcols]
        base = None
        for name, prec in forms:
            with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=prec) as h:
                rs.rsfd_set_solve_options(h.ptr, profile=1)
                if prec != rs.RSFD_FP64:
                    rs.rsfd_autotune(h.ptr, p.energies, p.eta, slots=int(batch.size), iters=256)
                else:
                    rs.rsfd_set_solve_options(h.ptr, slots=int(batch.size), profile=1)
                ridx = np.searchsorted(np.asarray(h.rows), rows)
                G0 = torch.zeros((p.K, batch.size, h.nb), dtype=h.complex_dtype, device="cuda")
                maxit = 40000 if prec == rs.RSFD_MIXED else 4 * p.maxit
                tol2 = 1e-8
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, info, res = rs.rsfd_shifted_cocg(h.ptr, batch, p.energies, p.eta, tol2, maxit, G0)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                G = G0.cpu().numpy()
            Gs = np.stack([G[:, j, :][:, ridx] for j in pos], axis=-1).astype(np.complex128)
            gerr = float(np.linalg.norm(Gs - Gref) / np.linalg.norm(Gref))
            ok = st == 0 and gerr <= 1e-5
            if name == "fp64":
                base = dt
            print(json.dumps({"experiment": "precision_speedup", "workload": p.name, "precision": name,
                              "tol": tol2, "status": int(st), "cocg_seconds": dt, "columns": int(batch.size),
                              "energies": p.K, "mean_seed_iterations": float(info["iters"].mean()),
                              "G0_bb_rel_err": gerr,
                              "reference": "oracle G0_bb at tol 1e-10 on the stored rows and columns (tests/golden)",
                              "meets_tolerances": ok,
                              "speedup_vs_fp64": (base / dt) if ok and base else None}), flush=True)


def run_full_boundary(args):
    """The full-boundary workload end to end on one GPU: 48x48x160 grid, h = 0.4, 4th order, 140 seeded
    wells, every one of the 2 x 2 x 48 x 48 = 9216 boundary-slab columns, 64 energies in [-0.5, 0.5]
    Ha at eta = 5e-4, tolerance 1e-6, double-float vectors.  Phases: the shifted COCG of all columns
    into a device G0_bb [64][9216][9216] (complex128, 87 GB), then, in energy chunks, the lead
    self-energies (closed form), the Dyson step (tensor-core LU, FP64 refinement of the left slab's
    columns, the block the transmission reads) and T(E).  One JSON line with the seconds per phase,
    the COCG throughput and T(E)."""
    import torch
    import paper_1502_00081_gb300 as rs
    from workloads import make_problem
    torch.cuda.set_device(0)
    rs.load_library()
    p = make_problem("full_boundary")
    if args.ncols:
        p.cols = p.cols[:args.ncols]
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_DF64) as h:
        cols = np.asarray(h.rows) if not args.ncols else np.asarray(h.rows)[:args.ncols]
        nb = h.nb
        rs.rsfd_set_solve_options(h.ptr, profile=1)
        topts, tus = rs.rsfd_autotune(h.ptr, p.energies, p.eta, slots=min(256, cols.size), iters=256)
        G0 = torch.zeros((p.K, cols.size, nb), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info, res = rs.rsfd_shifted_cocg(h.ptr, cols, p.energies, p.eta, p.tol, 4 * p.maxit, G0)
        torch.cuda.synchronize()
        t_cocg = time.perf_counter() - t0
        stats = rs.rsfd_get_stats(h.ptr)
        T_all, t_sigma, t_dyson, t_T, refres = [], 0.0, 0.0, 0.0, []
        if cols.size == nb:
            rs.rsfd_set_solve_options(h.ptr, dyson_cols=1, **{k: topts[k] for k in ("pass_kind", "tile_y", "z_chunk")})
            kc = 16
            for k0 in range(0, p.K, kc):
                E = p.energies[k0:k0 + kc]
                ta = time.perf_counter()
                SLh, SRh = rs.rsfd_lead_sigma_uniform(p.grid[0], p.grid[1], p.h, p.fd_order, E, p.eta)
                SL, SR = torch.from_numpy(SLh).cuda(), torch.from_numpy(SRh).cuda()
                torch.cuda.synchronize()
                tb = time.perf_counter()
                G = torch.empty((E.size, nb, nb), dtype=torch.complex128, device="cuda")
                refres += list(rs.rsfd_dyson_boundary(h.ptr, G0[k0:k0 + kc], SL, SR, G))
                torch.cuda.synchronize()
                tc = time.perf_counter()
                T_all += list(rs.rsfd_transmission(h.ptr, G, SL, SR))
                torch.cuda.synchronize()
                td = time.perf_counter()
                t_sigma += tb - ta
                t_dyson += tc - tb
                t_T += td - tc
                del G, SL, SR
    print(json.dumps({"experiment": "full_boundary", "workload": p.name, "grid": list(p.grid), "columns": int(cols.size),
                      "boundary_rows": int(nb), "energies": p.K, "eta": p.eta, "tol": p.tol, "precision": "df64",
                      "launch_options": {k: topts[k] for k in ("pass_kind", "tile_y", "z_chunk", "prefetch")},
                      "status": int(st), "columns_not_ok": int((info["status"] != 0).sum()),
                      "mean_seed_iterations": float(info["iters"].mean()),
                      "cocg_seconds": t_cocg, "cocg_columns_x_energies_per_s": cols.size * p.K / t_cocg,
                      "pass_ms": stats["ms_pass"], "shift_ms": stats["ms_shift"],
                      "sigma_seconds": t_sigma, "dyson_seconds": t_dyson, "transmission_seconds": t_T,
                      "dyson_form": "tensor-core LU (3xTF32), FP64 refinement, left-slab columns",
                      "dyson_refine_residual_max": float(max(refres)) if refres else None,
                      "T": [float(t) for t in T_all],
                      "T_nonnegative": bool(all(t >= -1e-6 for t in T_all)) if T_all else None}), flush=True)


def run_dyson_scaling(args):
    """The Dyson step (Eq. sec3-01a on the boundary rows) alone, tensor-core form (FP32 LU and
    triangular solves with 3xTF32 tcgen05 updates, FP64 residual refinement) against the FP64
    CUDA-core form, on seeded random complex-symmetric G0_bb and retarded Sigma of the boundary
    sizes of the workloads: nb = 1024, 2048 (both forms) and 4608, 9216 (the 48 x 48 plane and
    two-plane slab of the full-boundary workload; tensor-core form only, one energy).  One JSON
    line per (nb, form): seconds per energy, the FP64 refinement residual, and the difference
    between the two forms where both ran."""
    import torch
    import paper_1502_00081_gb300 as rs
    from workloads import random_complex_matrices
    torch.cuda.set_device(0)
    rs.load_library()

    def abi(M):
        return torch.from_numpy(np.ascontiguousarray(M.transpose(0, 2, 1))).cuda()

    for nb, K, forms in ((1024, 4, ("tc", "fp64")), (2048, 2, ("tc", "fp64")), (4608, 1, ("tc",)),
                         (9216, 1, ("tc",))):
        if args.dyson_max_nb and nb > args.dyson_max_nb:
            continue
        G0 = abi(random_complex_matrices(nb, K, seed=41, scale=0.5))
        SL = abi(random_complex_matrices(nb // 2, K, seed=42, scale=0.5, imag_sign=-1))
        SR = abi(random_complex_matrices(nb // 2, K, seed=43, scale=0.5, imag_sign=-1))
        out = {}
        for form in forms:
            kind = rs.RSFD_DYSON_TC if form == "tc" else rs.RSFD_DYSON_FP64
            with rs.Handle((nb // 2, 1, 4), 0.5, 2, np.zeros(nb // 2 * 4), n_face=1, precision=rs.RSFD_DF64) as h:
                rs.rsfd_set_solve_options(h.ptr, dyson_kind=kind, dyson_refine=1 if form == "tc" else 2)
                G = torch.empty((K, nb, nb), dtype=torch.complex128, device="cuda")
                if nb <= 2048:
                    rs.rsfd_dyson_boundary(h.ptr, G0, SL, SR, G)   # warm-up (workspace, module load)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ref = rs.rsfd_dyson_boundary(h.ptr, G0, SL, SR, G)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                out[form] = G
                nref = 1 if form == "tc" else 2
                line = {"experiment": "dyson_scaling", "form": form, "nb": nb, "energies": K,
                        "seconds_per_energy": dt / K, "refine_steps": nref,
                        "max_refine_residual": float(ref.max()),
                        "fp64_flops_per_energy": (4 + 8 * (nref + 1)) * nb ** 3 if form == "tc" else None,
                        "tf32_flops_per_energy": 3 * (8.0 / 3 + 8 * (nref + 1)) * nb ** 3 if form == "tc" else None}
                if form == "fp64" and "tc" in out:
                    d = torch.linalg.norm(out["tc"] - G) / torch.linalg.norm(G)
                    line["rel_diff_tc_vs_fp64"] = float(d)
                print(json.dumps(line), flush=True)
        del G0, SL, SR, out
        torch.cuda.empty_cache()


def run_tc_gemm(args):
    """The tensor-core GEMM of the Dyson step (rsfd_cgemm_tf32x3: complex FP32, 3xTF32 on tcgen05)
    alone, on the shapes it meets: a square 4096^3 product and the K = 64 panel updates of the
    blocked LU and triangular solves.  Reports complex FLOP/s (8 m n k per product) and the issued
    TF32 rate (three real-split products of four real GEMMs: 3 x 8 m n k)."""
    import torch
    import paper_1502_00081_gb300 as rs
    torch.cuda.set_device(0)
    rs.load_library()
    g = torch.Generator(device="cuda").manual_seed(5)
    shapes = ((1, 4096, 4096, 4096), (4, 2048, 2048, 128), (16, 1024, 1024, 64), (8, 4096, 4096, 64))
    for (b, m, n, k) in shapes:
        if args.gemm_size and m != args.gemm_size:
            continue
        A = torch.randn(b, k, m, dtype=torch.complex64, device="cuda", generator=g)
        B = torch.randn(b, n, k, dtype=torch.complex64, device="cuda", generator=g)
        C = torch.zeros(b, n, m, dtype=torch.complex64, device="cuda")
        rs.rsfd_cgemm_tf32x3(A, B, C, alpha=-1.0, beta=1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            rs.rsfd_cgemm_tf32x3(A, B, C, alpha=-1.0, beta=1.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        fl = 8.0 * b * m * n * k
        print(json.dumps({"experiment": "tc_gemm", "batch": b, "m": m, "n": n, "k": k, "ms": ms,
                          "complex_tflops": fl / ms / 1e9, "tf32_tflops_issued": 3 * fl / ms / 1e9}), flush=True)


def run_uneven_regions(args):
    """The uneven batch of six transition regions (32x32x64 ... 72x72x112, 4th order, per-region energy
    sets of 32-200 points and eta in {1e-3, 5e-4}), double-float: every region's launch options are
    chosen by the autotuner (rsfd_autotune), then the first --ncols columns of each region are solved
    (a) region after region and (b) all regions in one rsfd_shifted_cocg_regions call, whose regions
    run concurrently.  One JSON line per form with columns x energies / s over the whole batch."""
    import torch
    import paper_1502_00081_gb300 as rs
    from workloads import make_problem
    torch.cuda.set_device(0)
    rs.load_library()
    probs = make_problem("uneven_regions")
    ncols = args.ncols or 8
    prec = {"mixed": rs.RSFD_MIXED, "fp64": rs.RSFD_FP64, "df64": rs.RSFD_DF64}[args.precision]
    hs, outs, cols, tuned, topts = [], [], [], [], []
    for p in probs:
        h = rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=prec)
        # --full-columns: the configured columns (every plane point where 2 Nx Ny <= 4096, else 512 sampled)
        c = p.cols if args.full_columns else p.cols[:ncols]
        opts, us = rs.rsfd_autotune(h.ptr, p.energies, p.eta, slots=int(min(c.size, 256)), iters=128)
        topts.append(opts)
        tuned.append({"region": p.name, "grid": list(p.grid), "K": int(p.K), "eta": p.eta, "us_per_slot_iteration": us,
                      "pass_kind": opts["pass_kind"], "tile_y": opts["tile_y"], "rows_per_thread": opts["rows_per_thread"],
                      "z_chunk": opts["z_chunk"]})
        hs.append(h)
        cols.append(c)
        outs.append(torch.zeros((p.K, c.size, h.nb), dtype=h.complex_dtype, device="cuda"))
    units = float(sum(c.size * p.K for c, p in zip(cols, probs)))
    forms = []
    its = []
    if not args.full_columns:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p, h, c, o in zip(probs, hs, cols, outs):
            st, info, res = rs.rsfd_shifted_cocg(h.ptr, c, p.energies, p.eta, p.tol, p.maxit, o)
            its.append(float(info["iters"].mean()))
        torch.cuda.synchronize()
        forms.append(("region_after_region", time.perf_counter() - t0, None))
    for h, o in zip(hs, topts):   # the tuned options, with per-launch event timing
        rs.rsfd_set_solve_options(h.ptr, **dict(o, profile=1))
    jobs = [dict(h=h.ptr, cols=c, energies=p.energies, eta=p.eta, tol=p.tol, maxit=p.maxit, G0_bb=o)
            for p, h, c, o in zip(probs, hs, cols, outs)]
    t0 = time.perf_counter()
    st, per = rs.rsfd_shifted_cocg_regions(jobs)
    torch.cuda.synchronize()
    t_con = time.perf_counter() - t0
    # per region: device busy time of its passes and shift updates against its stream's span, and the
    # average host gap per iteration chunk that this leaves
    regions = []
    for p, h, c, (rst, rinfo, _) in zip(probs, hs, cols, per):
        s = rs.rsfd_get_stats(h.ptr)
        busy = s["ms_pass"] + s["ms_shift"]
        # ms_stream - ms_busy: the region's stream waiting, on the host between chunks or behind the
        # other regions' kernels on the shared SMs
        regions.append({"region": p.name, "grid": list(p.grid), "columns": int(c.size), "K": int(p.K), "eta": p.eta,
                        "slots": s["slots"], "mean_seed_iterations": s["slot_iterations"] / max(1, c.size),
                        "status": int(rst), "columns_not_converged": int((rinfo["status"] != 0).sum()),
                        "max_seed_iterations": int(rinfo["iters"].max()) if rinfo.size else 0,
                        "ms_stream": s["ms_total"], "ms_busy": busy, "chunks": s["n_shift"],
                        "ms_wait_per_chunk": (s["ms_total"] - busy) / max(1, s["n_shift"])})
    forms.append(("regions_in_one_call", t_con, regions))
    for form, t, reg in forms:
        print(json.dumps({"experiment": "uneven_regions", "form": form, "precision": args.precision,
                          "columns_per_region": [int(c.size) for c in cols], "seconds": t,
                          "columns_x_energies": units, "value": units / t, "unit": UNIT,
                          "mean_seed_iterations": its or None, "status": int(st),
                          "regions": reg, "tuned": tuned if form == "regions_in_one_call" else None}), flush=True)
    for h in hs:
        h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="df64", choices=["mixed", "fp64", "df64"])
    ap.add_argument("--cols-per-step", type=int, default=38,
                    help="columns solved per step (0 = the whole sample); 38 columns x 32 CTAs per column fill "
                         "exactly four waves of the 152 SMs x 2 resident CTAs")
    ap.add_argument("--maxit", type=int, default=0, help="iteration cap per column (profiling runs)")
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--prefetch", type=int, default=0, help="with --no-autotune: TMA planes in flight (1..7)")
    ap.add_argument("--pass-kind", type=int, default=0,
                    help="with --no-autotune: 1 fused, 2 stored-product, 3 split (combine + stencil launches), "
                         "4 split with block-floating-point leading parts (double-float)")
    ap.add_argument("--z-chunk", type=int, default=0)
    ap.add_argument("--reg-budget", type=int, default=0, help="with --no-autotune: the pass's register budget option")
    ap.add_argument("--ncols", type=int, default=0, help="use only the first n columns (quick runs)")
    ap.add_argument("--full-columns", action="store_true",
                    help="uneven_regions: every configured column of each region, the one-call form only")
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--iters-per-sync", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-option autotuner")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-all-cores", action="store_true",
                    help="skip the all-cores oracle figure (one spawned process per host core)")
    ap.add_argument("--experiment", default=None,
                    choices=[None, "shift_scaling", "precision_speedup", "dyson_scaling", "tc_gemm",
                             "uneven_regions", "full_boundary"],
                    help="run an experiment instead of the benchmark (JSON lines)")
    ap.add_argument("--dyson-max-nb", type=int, default=0, help="dyson_scaling: largest boundary size (0 = all)")
    ap.add_argument("--gemm-size", type=int, default=0, help="tc_gemm: only the shapes with this m (0 = all)")
    ap.add_argument("--max-independent", type=int, default=32,
                    help="shift_scaling: largest K also solved as K independent single-energy solves")
    args = ap.parse_args()
    if args.experiment == "shift_scaling":
        run_shift_scaling(args)
        return
    if args.experiment == "precision_speedup":
        run_precision_speedup(args)
        return
    if args.experiment == "dyson_scaling":
        run_dyson_scaling(args)
        return
    if args.experiment == "tc_gemm":
        run_tc_gemm(args)
        return
    if args.experiment == "uneven_regions":
        run_uneven_regions(args)
        return
    if args.experiment == "full_boundary":
        run_full_boundary(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
