"""Benchmark of the symmetry-adapted ED hot path on one GB300 (or N replicas).

Workload (default): Heisenberg ring N=32, J=1, sector Sz=0, momentum 0,
reflection +1, spin inversion +1 (group order 128, 4 707 969 representatives),
x0 uniform in [-1, 1] from seed 0.

One timed step = the whole hot path once: ed_basis_build (enumerate, filter,
compact, prefix table) followed by ed_lanczos with 100 steps in the fp32-matvec
mode (fp64 recurrence, fp64 refinement, fp64 Rayleigh quotient and residual).
value = matrix rows processed by H.x per second over the step
(dim x matvecs / step time).  The fp64-plain path (ed_lanczos fp64 mode) is
timed the same way and reported beside it with |dE0| between the two.

Multi-GPU: the path has one sector, which this build does not split across
GPUs; with --gpus N every rank runs an independent replica (weak scaling,
value = the sum over ranks), with a barrier and the max over ranks of the
timed region.

--impl reference times the CPU oracle (plain C, on all host cores through a
spawned process pool) on a bounded sample of the same rows and prints the
same JSON line with "impl": "reference".
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

import ed_inputs as ei  # noqa: E402

METRIC = "H·x rows/s & nonzeros/s: FP32 batched vs FP64 plain on 1 GB300 at |dE0|<1e-10"
UNIT = "rows/s"
L2_BYTES = 129 * 1024 * 1024
# INT32 ALU issue peak used for the roofline: 152 SMs x 64 lanes/clk x the
# maximum SM clock (GB300 SM: 4 sub-partitions x 16 INT32 lanes).
SMS = 152
INT_LANES_PER_SM = 64
# DRAM bytes (read + write) of one launch of the timed kernel, from one ncu
# capture of it (--set full, which starts every replay with a cold L2); keyed by
# workload.  Retake the capture and update the figure whenever the kernel
# changes (the roofline reports null traffic for workloads not listed).
KERNEL_DRAM_BYTES = {"ring32": 554_140_160 + 112_350_720}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_rows(w, n_rows, seed=1):
    """Row states for the oracle sample, found by the oracle itself: random
    states of the sector's popcount mapped to their representatives."""
    import oracle
    G = oracle.Group(w["n_sites"], w["perms"], w["chars"], w["spin_inversion"])
    rng = np.random.default_rng(seed)
    rows = []
    while len(rows) < n_rows:  # with repetition: small sectors have few rows
        bits = rng.choice(w["n_sites"], w["n_up"], replace=False)
        s = sum(1 << int(b) for b in bits)
        rep, _, norm, _ = oracle.state_info(G, s)
        if norm:
            rows.append(rep)
    return G, oracle.Operator(w["op"]), np.array(rows, np.uint64)


def time_oracle_rows(G, H, rows):
    import oracle
    t0 = time.perf_counter()
    _, nnz = oracle.rows_statex(G, H, rows, 0)
    return time.perf_counter() - t0, nnz


def _oracle_rows_worker(task):
    """One worker of the all-cores oracle run (a spawned process): the oracle's
    rows for a chunk of row states; returns the seconds it took."""
    import oracle
    n, perms, chars, z, op, rows = task
    G = oracle.Group(n, perms, chars, z)
    H = oracle.Operator(op)
    t0 = time.perf_counter()
    oracle.rows_statex(G, H, rows, 0)
    return time.perf_counter() - t0


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def time_oracle_rows_all_cores(w, rows, cores):
    """The unchanged oracle on all host cores: the rows split into one chunk per
    core, each chunk run by a process of a spawn-started pool (wall time of the
    parallel map, after a warm-up map that loads the oracle in every worker)."""
    import multiprocessing as mp
    task = (w["n_sites"], w["perms"], w["chars"], w["spin_inversion"], w["op"])
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_rows_worker, [task + (rows[:2],)] * cores)
        t0 = time.perf_counter()
        pool.map(_oracle_rows_worker, [task + (c,) for c in np.array_split(rows, cores)])
        return time.perf_counter() - t0


def cpu_baseline(w, budget_s=15.0, par_wall_s=5.0):
    G, H, rows = oracle_rows(w, 64)
    dt, _ = time_oracle_rows(G, H, rows[:8])
    per_row = max(dt / 8, 1e-6)
    n = int(min(max(budget_s / per_row, 16), 20000))
    G, H, rows = oracle_rows(w, n, seed=2)
    dt, nnz = time_oracle_rows(G, H, rows)
    single = {"value": len(rows) / dt, "cores": 1,
              "sample": f"{len(rows)} rows, single-threaded C oracle, {dt:.1f} s"}
    cores = host_cores()
    reps = max(1, int(par_wall_s * cores / (dt / len(rows)) / len(rows)))
    rows_par = np.tile(rows, reps)
    dtp = time_oracle_rows_all_cores(w, rows_par, cores)
    return {"value": len(rows_par) / dtp, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(rows_par)} rows of the {w['name']} sector ({len(rows)} distinct, each an "
                      f"H.x row with x keyed by state, no basis enumeration), the C oracle in {cores} "
                      f"spawned processes, {dtp:.1f} s wall",
            "single_core": single, "nnz_per_row": float(nnz.mean())}


def run_reference(args, w, budget_s=150.0):
    """The reference arm: the CPU oracle timed on the machine's host cores (rank 0
    only; other ranks exit without work), each step a bounded sample of rows
    sized so the whole run takes about budget_s seconds."""
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return None
    G, H, rows = oracle_rows(w, 64)
    dt, _ = time_oracle_rows(G, H, rows[:8])
    per_row = max(dt / 8, 1e-6)
    rows_per_step = int(min(max(budget_s / (args.steps + args.warmup) / per_row, 8), 20000))
    # each step: the same number of rows per core as the single-core estimate
    # allows in the budget, run by the oracle on all host cores
    cores = host_cores()
    G, H, rows = oracle_rows(w, rows_per_step, seed=3)
    step_rows = np.tile(rows, cores)
    for _ in range(args.warmup):
        time_oracle_rows_all_cores(w, step_rows[: max(cores, len(step_rows) // 8)], cores)
    total, n_done = 0.0, 0
    for _ in range(args.steps):
        total += time_oracle_rows_all_cores(w, step_rows, cores)
        n_done += len(step_rows)
    value = n_done / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "rows_per_step": rows_per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(step_rows)} rows per step of the {w['name']} sector "
                                       f"({rows_per_step} distinct), the C oracle in {cores} spawned "
                                       "processes (x keyed by state)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


# ---------------------------------------------------------------------------
# GPU measurement
# ---------------------------------------------------------------------------
def popcount64(t):
    import torch
    t = t - ((t >> 1) & 0x5555555555555555)
    t = (t & 0x3333333333333333) + ((t >> 2) & 0x3333333333333333)
    t = (t + (t >> 4)) & 0x0F0F0F0F0F0F0F0F
    return ((t * 0x0101010101010101) >> 56) & 0xFF


def generated_terms_per_row(states, n):
    """Average off-diagonal terms H|r> generates per row for the Heisenberg ring
    (one per antiparallel bond); every one of them costs a group search."""
    mask = (1 << n) - 1
    rot = ((states << 1) | (states >> (n - 1))) & mask
    return float(popcount64((states ^ rot) & mask).double().mean())


def run_matvec_only(args, w):
    """Basis build and --steps matvec launches per dtype, timed with CUDA events
    (a short program, also used for profiler captures)."""
    import torch
    from paper_2308_16712_gb300 import ed
    n = w["n_sites"]
    op = w["op"]
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    t0 = time.perf_counter()
    B = ed.basis_build(n, w["n_up"], w["spin_inversion"], w["perms"], w["chars"])
    build_ms = 1e3 * (time.perf_counter() - t0)
    dim = ed.basis_size(B)
    cplx = not ed.basis_is_real(B)
    nvec = args.nvec
    states, _ = ed.basis_states(B)
    nnz = ed.count_nnz(O, B)
    out = {"mode": "matvec", "workload": w["name"], "dim": dim, "nvec": nvec, "basis_build_ms": build_ms,
           "launches": 2 * args.steps, "nnz_per_matvec": nnz, "nnz_per_row": nnz / max(dim, 1)}
    dts = (torch.complex64, torch.complex128) if cplx else (torch.float32, torch.float64)
    y_single = None
    for dt in dts:
        x = ei.x_by_state_torch_chunked(5, states, nvec, cplx, dtype=dt)
        y = torch.empty_like(x)
        ts = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ed.matvec(O, B, x, y, nvec)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = min(ts)
        res = {"ms": ms, "rows_per_s": dim / (ms * 1e-3), "vector_rows_per_s": nvec * dim / (ms * 1e-3),
               "nonzeros_per_s": nnz / (ms * 1e-3)}
        if y_single is None:
            y_single = y  # single precision first: kept for the error against double
        else:
            # max |y_single - y_double| / max |y_double| over the whole product
            err, scale = 0.0, float(y.abs().max())
            for lo in range(0, y.shape[0], 1 << 26):
                d = y_single[lo:lo + (1 << 26)].to(y.dtype) - y[lo:lo + (1 << 26)]
                err = max(err, float(d.abs().max()))
            out["single_precision_max_rel_err"] = err / max(scale, 1e-300)
            y_single = None
        out[str(dt).replace("torch.", "")] = res
        del x, y
        torch.cuda.empty_cache()
    print(json.dumps(out))


def search_ops_per_term(n, n_perm, flip, fact, rot_L, n_cos, kinds):
    """INT32 operations of one representative search (real characters, so no
    minimiser is tracked) as the kernel runs it -- an instruction-level count of
    the algorithm, not a measurement.
    32-bit words: Benes stage = 2 shifts + 2 three-input logic ops (9 stages);
    rotation of the doubled word = 1 funnel shift (+1 mask op when n < 32);
    running min = 1 op per candidate; with spin inversion the factored search
    keeps a running max as well (1 op) and needs no per-candidate complement,
    the generic one complements (1 op) and takes a second min (1 op).
    64-bit words: shifts, logic ops, min and max cost two 32-bit operations
    each (4 for a 64-bit min or max); an incremental rotation costs 6."""
    if n <= 32:
        benes, rev = 36, (1 if n == 32 else 2)
        per_rot = (1 if n == 32 else 2) + (2 if flip else 1)
        per_perm = benes + (3 if flip else 1)
    else:
        benes, rev = 84, 4
        per_rot = 6 + (8 if flip else 4)
        per_perm = benes + (2 + 8 if flip else 4)
    if not fact:
        return n_perm * per_perm
    head = sum({0: 0, 1: rev, 2: benes}[int(k)] for k in kinds)
    return head + n_cos * rot_L * per_rot + (1 if flip else 0)


def measure_peaks(dev=None):
    """This GPU's measured ceilings (the library's peak kernels, CUDA events):
    integer op mix of the group search, fp64 and fp32 FMA, and random 32-byte
    reads over an 8 GiB buffer (far above L2)."""
    import torch
    from paper_2308_16712_gb300 import ed
    out = {}
    for kind in ("int32_mix", "fp64_fma", "fp32_fma"):
        rate, ms = ed.peak(kind)
        out[kind] = {"rate": rate, "ms": ms}
    buf = torch.empty(8 << 30, dtype=torch.uint8, device=dev or "cuda")
    buf.fill_(1)
    rate, ms = ed.peak("gather32", buf)
    out["gather32"] = {"rate": rate, "ms": ms, "span_bytes": buf.numel()}
    del buf
    torch.cuda.empty_cache()
    return out


def run_peaks(args, w):
    import torch
    sampler = ClockSampler(0)
    pk = measure_peaks()
    clocks = sampler.stop()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz", 2070.0)
    for k in ("int32_mix", "fp64_fma", "fp32_fma"):
        pk[k]["per_sm_per_clk"] = pk[k]["rate"] / sms / (mhz * 1e6)
    print(json.dumps({"mode": "peaks", "sms": sms, "clocks": clocks, **pk}), flush=True)


def run_one_step(args, w):
    import torch
    from paper_2308_16712_gb300 import ed
    n, op = w["n_sites"], w["op"]
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    x0 = None
    marks = []
    for rep in range(2):
        t0 = time.perf_counter()
        launches0 = ed.launch_count()
        B = ed.basis_build(n, w["n_up"], w["spin_inversion"], w["perms"], w["chars"])
        t1 = time.perf_counter()
        if x0 is None:
            x0 = torch.from_numpy(ei.x_by_index(0, ed.basis_size(B))[:, 0]).cuda()
        r = ed.lanczos(O, B, x0, w["lanczos_steps"], ed.ED_LANCZOS_F32_MATVEC)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        marks.append({"basis_ms": 1e3 * (t1 - t0), "lanczos_ms": 1e3 * (t2 - t1),
                      "matvec_ms": r.matvec_ms, "launches": ed.launch_count() - launches0})
        del B
    print(json.dumps({"mode": "step", "workload": w["name"], "steps": marks}))


def run_solve(args, w):
    """One ground-state solve per Lanczos mode (fp32 matvec and fp64), timed,
    for workloads too large for the benchmark loop (e.g. the N=40 ring)."""
    import torch
    from paper_2308_16712_gb300 import ed
    n, op = w["n_sites"], w["op"]
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    t0 = time.perf_counter()
    B = ed.basis_build(n, w["n_up"], w["spin_inversion"], w["perms"], w["chars"])
    build_s = time.perf_counter() - t0
    dim = ed.basis_size(B)
    cplx = not ed.basis_is_real(B)
    x0 = torch.from_numpy(ei.x_by_index(0, dim, 1, cplx)[:, 0]).cuda()
    out = {"mode": "solve", "workload": w["name"], "dim": dim, "basis_build_s": build_s,
           "lanczos_steps": w["lanczos_steps"]}
    for name, mode in (("f32_matvec", ed.ED_LANCZOS_F32_MATVEC), ("f64", ed.ED_LANCZOS_F64)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ed.lanczos(O, B, x0, w["lanczos_steps"], mode)
        torch.cuda.synchronize()
        out[name] = {"e0": r.e0, "ritz": r.ritz, "residual": r.residual, "matvecs": r.matvecs,
                     "matvec_ms": r.matvec_ms, "wall_s": time.perf_counter() - t0}
    out["dE0"] = abs(out["f32_matvec"]["e0"] - out["f64"]["e0"])
    print(json.dumps(out), flush=True)


def run_push(args, w):
    """Ablation: the pull product (default kernel choice) against the push form
    (atomic scatter into y), one vector, L2 flushed before each launch; the
    push form's run-to-run variation of y (order of the atomic adds)."""
    import torch
    from paper_2308_16712_gb300 import ed
    n = w["n_sites"]
    O = ed.operator_create(n, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    B = ed.basis_build(n, w["n_up"], w["spin_inversion"], w["perms"], w["chars"])
    dim = ed.basis_size(B)
    cplx = not ed.basis_is_real(B)
    states, _ = ed.basis_states(B)
    flush = torch.empty(L2_BYTES // 2, dtype=torch.float32, device="cuda")

    def timed(fn, reps=5):
        fn()
        best = 1e30
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    out = {"mode": "push", "workload": w["name"], "dim": dim}
    for dt in ((torch.complex64, torch.complex128) if cplx else (torch.float32, torch.float64)):
        x = ei.x_by_state_torch_chunked(5, states, 1, cplx, dtype=dt).reshape(-1)
        y_pull = torch.empty_like(x)
        y_push = torch.empty_like(x)
        ms_pull = timed(lambda: ed.matvec(O, B, x, y_pull, 1))
        ms_push = timed(lambda: ed.matvec_push(O, B, x, y_push))
        runs = []
        for _ in range(5):
            ed.matvec_push(O, B, x, y_push)
            runs.append(y_push.clone())
        scale = float(y_pull.abs().max())
        distinct = len({r.cpu().numpy().tobytes() for r in runs})
        out[str(dt).replace("torch.", "")] = {
            "pull_ms": ms_pull, "push_ms": ms_push,
            "pull_rows_per_s": dim / (ms_pull * 1e-3), "push_rows_per_s": dim / (ms_push * 1e-3),
            "push_distinct_results_of_5": distinct,
            "push_max_run_to_run_rel": max(float((r - runs[0]).abs().max()) for r in runs) / scale,
            "push_vs_pull_max_rel": float((runs[0] - y_pull).abs().max()) / scale}
        del x, y_pull, y_push, runs
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_multi(args):
    """The XXZ ring N=28 (Jxy=1, Delta=1.5) in all 140 sectors: one
    ed_matvec_multi launch over every sector against one ed_matvec per sector,
    block vectors of --nvec columns, single and double precision."""
    import torch
    from paper_2308_16712_gb300 import ed
    op = ei.xxz_ring(28, 1.0, 1.5)
    O = ed.operator_create(28, op["sites"], op["coeff"], op["local"])
    t0 = time.perf_counter()
    bases = [ed.basis_build(28, s["n_up"], s["spin_inversion"], s["perms"], s["chars"])
             for s in ei.xxz28_sectors()]
    build_s = time.perf_counter() - t0
    dims = [ed.basis_size(b) for b in bases]
    nvec = args.nvec
    out = {"mode": "multi", "workload": "xxz28: 140 sectors", "rows": sum(dims), "nvec": nvec,
           "basis_build_s": build_s, "min_dim": min(dims), "max_dim": max(dims)}
    for dt in (torch.complex64, torch.complex128):
        items = []
        for b in bases:
            st, _ = ed.basis_states(b)
            x = ei.x_by_state_torch(5, st, nvec, True, dtype=dt).contiguous()
            items.append((b, x, torch.empty_like(x)))

        def timed(fn, reps=3):
            fn()
            best = 1e30
            for _ in range(reps):
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                e.record()
                torch.cuda.synchronize()
                best = min(best, a.elapsed_time(e))
            return best

        ms_multi = timed(lambda: ed.matvec_multi(O, items, nvec))
        ms_single = timed(lambda: [ed.matvec(O, b, x, y, nvec) for b, x, y in items])
        out[str(dt).replace("torch.", "")] = {
            "multi_ms": ms_multi, "per_sector_ms": ms_single,
            "vector_rows_per_s_multi": nvec * sum(dims) / (ms_multi * 1e-3),
            "vector_rows_per_s_per_sector": nvec * sum(dims) / (ms_single * 1e-3)}
        del items
        torch.cuda.empty_cache()
    steps = args.lanczos_steps
    if steps > 0:
        # all 140 lowest energies: one batched, graph-replayed solve against
        # ed_lanczos sector by sector (fp32 matvec, fp64 recurrence + refinement)
        mode = ed.ED_LANCZOS_F32_MATVEC
        xs = []
        for b in bases:
            st, _ = ed.basis_states(b)
            xs.append(ei.x_by_state_torch(5, st, 1, True, dtype=torch.complex128).reshape(-1).contiguous())
        items = [(b, x, None) for b, x in zip(bases, xs)]
        ed.lanczos_multi(O, items, 3, mode)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ed.lanczos_multi(O, items, steps, mode)
        t_multi = time.perf_counter() - t0
        t0 = time.perf_counter()
        res1 = [ed.lanczos(O, b, x, steps, mode) for b, x in zip(bases, xs)]
        t_single = time.perf_counter() - t0
        e_sz = {}
        for s, r in zip(ei.xxz28_sectors(), res):
            e_sz[s["n_up"] - 14] = min(e_sz.get(s["n_up"] - 14, float("inf")), r.e0)
        out["lanczos"] = {
            "steps": steps, "mode": "f32_matvec", "sectors": len(items),
            "batched_s": t_multi, "per_sector_s": t_single,
            "matvecs_batched": res[0].matvecs,
            "max_rel_dE0_vs_per_sector": max(abs(a.e0 - b.e0) / abs(b.e0) for a, b in zip(res, res1)),
            "max_residual": max(r.residual for r in res),
            "e0_min_by_sz": e_sz}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ring32")
    ap.add_argument("--nvec", type=int, default=1, help="vectors per matvec in --mode matvec")
    ap.add_argument("--lanczos-steps", type=int, default=100,
                    help="Lanczos steps of the batched solve in --mode multi (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="job", choices=["job", "matvec", "step", "solve", "multi", "push",
                                                      "peaks"],
                    help="job: the benchmark; matvec: only the basis build and --steps matvec "
                         "launches per dtype; step: one untimed and one more whole step "
                         "(short programs for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = ei.workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.mode == "matvec":
        return run_matvec_only(args, w)
    if args.mode == "step":
        return run_one_step(args, w)
    if args.mode == "peaks":
        return run_peaks(args, w)
    if args.mode == "solve":
        return run_solve(args, w)
    if args.mode == "push":
        return run_push(args, ei.workload(args.workload))
    if args.mode == "multi":
        return run_multi(args)

    import torch
    from paper_2308_16712_gb300 import ed

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n, n_up, z = w["n_sites"], w["n_up"], w["spin_inversion"]
    op = w["op"]
    steps = w["lanczos_steps"]
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    B = ed.basis_build(n, n_up, z, w["perms"], w["chars"])
    dim = ed.basis_size(B)
    states, _ = ed.basis_states(B)
    t_gen = generated_terms_per_row(states, n)
    x0_host = torch.from_numpy(ei.x_by_index(0, dim)[:, 0]).pin_memory()
    x0 = x0_host.to(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def flush_l2():
        flush.fill_(1.0)

    def one_step(mode):
        b = ed.basis_build(n, n_up, z, w["perms"], w["chars"])
        r = ed.lanczos(O, b, x0, steps, mode)
        del b
        return r

    def timed_steps(mode, k, warm):
        for _ in range(warm):
            one_step(mode)
        torch.cuda.synchronize()
        barrier(world)
        total_ms, res, mv_ms, mv_n = 0.0, None, 0.0, 0
        launches0 = ed.launch_count()
        for _ in range(k):
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            res = one_step(mode)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            mv_ms += res.matvec_ms
            mv_n += res.matvecs
        launches = ed.launch_count() - launches0
        barrier(world)
        return total_ms, res, mv_ms, mv_n, launches

    sampler = ClockSampler(local) if rank == 0 else None
    ms32, r32, mv32_ms, mv32_n, launches = timed_steps(ed.ED_LANCZOS_F32_MATVEC, args.steps, args.warmup)
    clocks = sampler.stop() if sampler else None
    ms64, r64, mv64_ms, mv64_n, _ = timed_steps(ed.ED_LANCZOS_F64, max(1, args.steps), 1)
    # the same job with push-form products (opt-in, not bit-reproducible)
    msp, rp, _, _, _ = timed_steps(ed.ED_LANCZOS_F32_MATVEC | ed.ED_LANCZOS_PUSH, max(1, args.steps), 1)
    msp = max_over_ranks(msp, world)
    ms32 = max_over_ranks(ms32, world)
    ms64 = max_over_ranks(ms64, world)
    per32 = ms32 / args.steps
    per64 = ms64 / max(1, args.steps)
    rows32 = dim * r32.matvecs / (per32 * 1e-3)
    rows64 = dim * r64.matvecs / (per64 * 1e-3)
    value = sum_over_ranks(rows32, world) if world > 1 else rows32

    # where a step's time goes: basis build alone (events, L2 flushed first),
    # products (CUDA events around every product inside ed_lanczos), the rest
    build_ts = []
    for _ in range(3):
        flush_l2()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        b0.record(stream)
        bb = ed.basis_build(n, n_up, z, w["perms"], w["chars"])
        b1.record(stream)
        torch.cuda.synchronize()
        build_ts.append(b0.elapsed_time(b1))
        del bb
    build_ms = statistics.median(build_ts)
    mv_step_ms = mv32_ms / args.steps
    breakdown = {"basis_build_ms": build_ms, "products_ms": mv_step_ms,
                 "products": mv32_n // max(args.steps, 1),
                 "lanczos_vectors_and_rest_ms": per32 - build_ms - mv_step_ms}

    # single matvec launches (kernel level), L2 flushed between launches
    def matvec_rate(dtype, nvec, reps=5):
        xx = torch.from_numpy(ei.x_by_index(5, dim, nvec)).to(dev).to(dtype)
        yy = torch.empty_like(xx)
        ed.matvec(O, B, xx, yy, nvec)
        tot = 0.0
        for _ in range(reps):
            flush_l2()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ed.matvec(O, B, xx, yy, nvec)
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    mv = {}
    for name, dt, nv in [("f64", torch.float64, 1), ("f32", torch.float32, 1), ("f32_nvec8", torch.float32, 8)]:
        ms = matvec_rate(dt, nv)
        mv[name] = {"ms": ms, "rows_per_s": dim / (ms * 1e-3), "vector_rows_per_s": nv * dim / (ms * 1e-3)}

    # roofline of the dominant kernel (the matvec): integer ALU bound
    pk, pk_kind = peaks()
    n_perm = len(w["perms"])
    fact, rot_L, rot_d, n_cos = ed.basis_factored(B)
    kinds = [0, 1] if (fact and n_cos == 2) else [0] + [2] * (n_cos - 1)
    ops_term = search_ops_per_term(n, n_perm, z != 0, fact, rot_L, n_cos, kinds)
    int_ops = dim * t_gen * ops_term
    avg_ms = (mv32_ms / max(mv32_n, 1)) if mv32_n else mv["f32"]["ms"]
    achieved = int_ops / (avg_ms * 1e-3) / 1e12
    peak_int = SMS * INT_LANES_PER_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w)
    nnz_total = ed.count_nnz(O, B)  # exact, on the GPU
    nnz_row = nnz_total / dim

    # end to end through the C ABI: pinned host x0 in, ground state and E0 out
    host_out = torch.empty(dim, dtype=torch.float64).pin_memory()
    vec = torch.empty(dim, dtype=torch.float64, device=dev)
    e2e_ms = 0.0
    for i in range(1 + args.steps):
        flush_l2()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd = x0_host.to(dev, non_blocking=True)
        b = ed.basis_build(n, n_up, z, w["perms"], w["chars"])
        r = ed.lanczos(O, b, xd, steps, ed.ED_LANCZOS_F32_MATVEC, vec_out=vec)
        host_out.copy_(vec, non_blocking=True)
        torch.cuda.synchronize()
        del b
        if i:
            e2e_ms += 1e3 * (time.perf_counter() - t0)
    e2e_ms = max_over_ranks(e2e_ms / args.steps, world)
    e2e_value = dim * r.matvecs / (e2e_ms * 1e-3)
    if world > 1:
        e2e_value = sum_over_ranks(e2e_value, world)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{w['name']}: Heisenberg ring N={n}, J=1, Sz=0, k=0, p=+1, z=+1",
                   "dim": dim, "group_order": n_perm * 2, "lanczos_steps": steps,
                   "step": "basis build + Lanczos (fp32 matvec, fp64 recurrence, fp64 refinement)",
                   "l2": "flushed between timed steps", "parallelism": f"replicas x{world}"},
        "e0": r32.e0, "residual": r32.residual, "matvecs_per_step": r32.matvecs,
        "fp64_plain": {"value": rows64, "ms_per_step": per64, "e0": r64.e0, "residual": r64.residual,
                       "matvecs_per_step": r64.matvecs},
        "dE0": abs(r32.e0 - r64.e0),
        "step_breakdown": breakdown,
        "push_mode": {"value": dim * rp.matvecs / (msp / max(1, args.steps) * 1e-3),
                      "ms_per_step": msp / max(1, args.steps), "e0": rp.e0, "dE0": abs(rp.e0 - r64.e0),
                      "note": "ED_LANCZOS_PUSH: atomic scatter products, E0 varies in the last bits"},
        "speedup_fp32_vs_fp64": rows32 / rows64,
        "nonzeros_per_s": value * nnz_row,
        "nnz_per_row": nnz_row,
        "nnz_per_matvec": nnz_total,
        "generated_terms_per_row": t_gen,
        "prefix_table": dict(zip(("entries", "largest_bucket", "probe_steps"), ed.basis_table(B))),
        "hash_index": dict(zip(("present", "log2_buckets", "largest_bucket", "wide_entries"),
                               ed.basis_hash(B))),
        "matvec_kernel": mv,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_int, "unit": "TOP/s",
                     "frac": achieved / peak_int, "traffic": KERNEL_DRAM_BYTES.get(w["name"]),
                     "kernel": "k_matvec_tp (term-parallel, fp32, " + ("rotation x coset" if fact else "Benes")
                               + f" group search, {'32' if n <= 32 else '64'}-bit words)",
                     "int_ops_per_launch": int_ops, "int_ops_per_term": ops_term,
                     "peak_basis": f"{SMS} SMs x {INT_LANES_PER_SM} INT32 lanes x "
                                   f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz ({pk_kind} clock)"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": dim * 8, "d2h_bytes_per_step": dim * 8 + 8},
        "gpu_launches": launches // max(args.steps, 1) * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
