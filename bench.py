"""Benchmark of the symmetry-adapted ED hot path on one GB300 (or N replicas).

Workload (default): Heisenberg ring N=40, J=1, sector Sz=0, momentum 0,
reflection +1, spin inversion +1 (group order 160, 861 725 794
representatives -- the paper's Table 2 dimension for 40 spins).

The metric compares two forms of the product H.x on this sector:
  - FP32 batched: block Lanczos on nvec = 8 vectors, every product one
    interleaved fp32 block product (one representative search and index
    lookup per matrix element serves all 8 columns), block recurrence and
    refinement in fp64-class arithmetic (ed_lanczos_block);
  - FP64 plain: single-vector Lanczos with fp64 products (ed_lanczos).
One timed step = one block-Lanczos step (the block product plus the block
recurrence kernels; the basis is built once, before, and timed separately).
value = H.x rows per second = dim x nvec x steps / time (every basis row of a
block product counts once per vector).  fp64_plain.value is the same for the
single-vector fp64 recurrence.  dE0 is taken between two full ground-state
solves run in the same process outside the timed loops: the FP32 batched
block solve (Ritz vector by a second pass, fp64 refinement, fp64 Rayleigh
quotient) and the 150-step FP64 plain solve.

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
# DRAM bytes (read + write) per stored nonzero of one launch of the timed
# kernel (fp32 block product, keyed by kernel and nvec), from one ncu --set
# full capture of the same kernel on the ring N=36 sector with 1 230 759 430
# nonzeros (term-parallel, nvec = 8: 162.13 + 2.02 GB; row-per-lane: 161.04 +
# 2.02 GB).  A ring N=40 launch is too large for a many-pass capture, so its
# traffic is this figure times the nonzeros it processes.  Retake the capture
# and update the figure whenever the kernel changes (the roofline reports null
# traffic for kernels not listed).
KERNEL_DRAM_BYTES_PER_NNZ = {("term-parallel", 8): (162.133806e9 + 2.022193e9) / 1230759430,
                             ("row-per-lane", 8): (161.040283e9 + 2.023800e9) / 1230759430}


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


def cpu_baseline(w, budget_s=8.0, par_wall_s=4.0):
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


def workload_label(w):
    """The workload name both arms print in config.workload."""
    if w["name"] == "ring40":
        return ("ring40: Heisenberg ring N=40, J=1, Sz=0, k=0, p=+1, z=+1 "
                "(the paper's Table 2 sector for 40 spins)")
    return w["name"]


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
            "data": "synthetic",
            "config": {"workload": workload_label(w),
                       "group_order": len(w["perms"]) * (2 if w["spin_inversion"] else 1),
                       "nvec": getattr(args, "nvec", 8),
                       "rows_per_step": rows_per_step},
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
    ed.kernel_policy(args.kernel_policy)
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


def run_block_steps(args, w):
    """--steps block-Lanczos steps (fp32 block products, values only) on a
    workload: a short program for profiler captures of the block kernels."""
    import torch
    from paper_2308_16712_gb300 import ed
    n = w["n_sites"]
    O = ed.operator_create(n, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    B = ed.basis_build(n, w["n_up"], w["spin_inversion"], w["perms"], w["chars"])
    dim = ed.basis_size(B)
    states, _ = ed.basis_states(B)
    X0 = ei.x_by_state_torch_chunked(0, states, args.nvec, False, dtype=torch.float64)
    t0 = time.perf_counter()
    _, r = ed.lanczos_block(O, B, X0, args.nvec, args.steps, ed.ED_LANCZOS_F32_MATVEC | ed.ED_LANCZOS_VALUES_ONLY)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "block", "workload": w["name"], "dim": dim, "nvec": args.nvec, "steps": r.steps,
                      "ritz": r.e0, "wall_s": time.perf_counter() - t0, "product_ms": r.matvec_ms / r.matvecs}))


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
    if dim <= 1 << 30:
        x0 = torch.from_numpy(ei.x_by_index(0, dim, 1, cplx)[:, 0]).cuda()
        x0_kind = "uniform[-1,1) keyed by index, seed 0"
    else:  # billions of rows: generated on the device, keyed by state
        states, _ = ed.basis_states(B)
        x0 = ei.x_by_state_torch_chunked(0, states, 1, cplx).reshape(-1)
        del states
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # the generator's temporaries, for the solver's vectors
        ed.release_cached_memory()
        x0_kind = "uniform[-1,1) keyed by state, seed 0"
    out = {"mode": "solve", "workload": w["name"], "dim": dim, "basis_build_s": build_s,
           "lanczos_steps": w["lanczos_steps"], "x0": x0_kind,
           "index": "bucketed" if ed.basis_bucket(B)[0] else "hash"}
    modes = [m for m in (("f32_matvec", ed.ED_LANCZOS_F32_MATVEC), ("f64", ed.ED_LANCZOS_F64))
             if m[0] in args.solve_modes.split(",")]
    for name, mode in modes:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ed.lanczos(O, B, x0, w["lanczos_steps"], mode)
        torch.cuda.synchronize()
        out[name] = {"e0": r.e0, "ritz": r.ritz, "residual": r.residual, "matvecs": r.matvecs,
                     "matvec_ms": r.matvec_ms, "wall_s": time.perf_counter() - t0}
    if len(modes) == 2:
        out["dE0"] = abs(out["f32_matvec"]["e0"] - out["f64"]["e0"])
    out["device_gb_peak"] = torch.cuda.max_memory_allocated() / 1e9
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
        ed.multi_policy("batched")
        try:
            ms_batched = timed(lambda: ed.matvec_multi(O, items, nvec))
        finally:
            ed.multi_policy("auto")
        ms_single = timed(lambda: [ed.matvec(O, b, x, y, nvec) for b, x, y in items])
        out[str(dt).replace("torch.", "")] = {
            "multi_ms": ms_multi, "batched_launch_ms": ms_batched, "per_sector_ms": ms_single,
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


def pruned_search_ops(states, n):
    """INT32 operations of the pruned representative search (rotation step one
    site, identity and reversal cosets, spin inversion, 64-bit words) averaged
    over the terms that the given row states generate -- an instruction-level
    count of the algorithm the kernel runs, with its data-dependent trip counts
    (longest run of equal bits, number of candidate tops) taken from the terms:
      fixed part 39 ops (first rotation, equal-bit mask, special cases, the
      reversal's mirrored tops and image), 16 ops per run-length iteration (64-bit
      rotation by one, mask, zero test, select), 35 ops per candidate (lowest
      set bit, clear, rotation by a variable amount, complement test, 64-bit
      compare and select), candidates counted for both cosets."""
    full = np.uint64((1 << n) - 1)
    one = np.uint64(1)

    def rotl1(x):
        return ((x << one) | (x >> np.uint64(n - 1))) & full

    terms = []
    for r in states:
        r = np.uint64(r)
        rr = rotl1(r)  # bit p = bit p-1 of r: bonds (p-1, p) antiparallel where r ^ rr
        anti = int((r ^ rr) & full)
        p = 0
        while anti:
            if anti & 1:
                q = (p - 1) % n
                terms.append(int(r) ^ (1 << p) ^ (1 << q))
            anti >>= 1
            p += 1
    h = np.array(terms, dtype=np.uint64)
    x2 = ~(h ^ rotl1(h)) & full
    cur = np.full_like(h, full)
    it = np.zeros(len(h), np.int64)
    live = x2 != full
    while live.any():
        nxt = x2 & rotl1(cur)
        go = live & (nxt != 0)
        cur = np.where(go, nxt, cur)
        it += live.astype(np.int64)  # the iteration that finds nxt == 0 counts too
        live = go
    cand = np.array([bin(int(c)).count("1") for c in cur], np.int64)
    ops = 39 + 16 * it + 2 * 35 * cand
    return float(ops.mean()), float(it.mean()), float(cand.mean()), len(h)


def run_job(args, w):
    import torch
    from paper_2308_16712_gb300 import ed

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n, n_up, z = w["n_sites"], w["n_up"], w["spin_inversion"]
    nvec = args.nvec
    op = w["op"]
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    VO = ed.ED_LANCZOS_VALUES_ONLY

    def ev():
        return torch.cuda.Event(enable_timing=True)

    b0, b1 = ev(), ev()
    b0.record(stream)
    B = ed.basis_build(n, n_up, z, w["perms"], w["chars"])
    b1.record(stream)
    torch.cuda.synchronize()
    build_ms = b0.elapsed_time(b1)
    dim = ed.basis_size(B)
    states, _ = ed.basis_states(B)
    # start blocks keyed by the state (seed 0): the [dim][nvec] fp64 block of
    # the FP32 batched path and the single fp64 vector of the plain path
    X0 = ei.x_by_state_torch_chunked(0, states, nvec, False, dtype=torch.float64)
    x1 = ei.x_by_state_torch_chunked(0, states, 1, False, dtype=torch.float64).reshape(-1)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = ev(), ev()
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res

    # ---- the product variant for the batched fp32 block, chosen by the
    # library's autotuner on this GPU (the timed steps then use it) -----------
    xt = X0.to(torch.float32)
    tuning = ed.autotune(O, B, xt, torch.empty_like(xt), nvec)
    del xt
    torch.cuda.empty_cache()

    # ---- FP32 batched: block-Lanczos steps (the timed headline) --------------
    ed.lanczos_block(O, B, X0, nvec, args.warmup, ed.ED_LANCZOS_F32_MATVEC | VO)
    launches0 = ed.launch_count()
    sampler = ClockSampler(local) if rank == 0 else None
    ms_blk, (_, rb) = timed(lambda: ed.lanczos_block(O, B, X0, nvec, args.steps, ed.ED_LANCZOS_F32_MATVEC | VO))
    clocks = sampler.stop() if sampler else None
    launches = ed.launch_count() - launches0
    ms_blk = max_over_ranks(ms_blk, world)
    per_step = ms_blk / args.steps
    rows_blk = dim * nvec * args.steps / (ms_blk * 1e-3)
    value = sum_over_ranks(rows_blk, world) if world > 1 else rows_blk
    prod_ms = rb.matvec_ms / max(rb.matvecs, 1)  # the block product, CUDA events in the step

    # ---- FP64 plain: the 150-step single-vector fp64 Lanczos solve, timed
    # (CUDA events) as a whole; its lowest Ritz value is the plain E0 --------
    plain_steps = w["lanczos_steps"]
    ms_plain, rplain = timed(lambda: ed.lanczos(O, B, x1, plain_steps, ed.ED_LANCZOS_F64 | VO))
    ms_plain = max_over_ranks(ms_plain, world)
    rows_plain = dim * rplain.steps / (ms_plain * 1e-3)
    prod64_ms = rplain.matvec_ms / max(rplain.matvecs, 1)
    t_plain_solve = ms_plain * 1e-3

    # ---- dE0: the full FP32 batched solve outside the timed loop --------------
    t0 = time.perf_counter()
    _, rfull = ed.lanczos_block(O, B, X0, nvec, args.block_steps, ed.ED_LANCZOS_F32_MATVEC)
    t_blk_solve = time.perf_counter() - t0
    dE0 = abs(rfull.e0 - rplain.e0)
    del x1
    torch.cuda.empty_cache()

    # ---- nonzeros and the roofline of the dominant kernel (the block product) --
    nnz_total = ed.count_nnz(O, B)
    nnz_row = nnz_total / dim
    rng = np.random.default_rng(7)
    idx = torch.from_numpy(rng.integers(0, dim, 3000)).to(dev)
    sample = states[idx].cpu().numpy().view(np.uint64)
    ops_term, run_iters, cands, n_terms = pruned_search_ops(sample, n)
    t_gen = n_terms / len(sample)
    terms = dim * t_gen
    int_ops = terms * ops_term
    int_peak, _ = ed.peak("int32_mix")
    gather_peak = None
    pk, pk_kind = peaks()
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    alg_bytes = dim * (8 + 2 + 2 * 4 * nvec) + terms * (4 * nvec + 2)  # keys, norms, x_r, y_r; x_j, n(r')
    sector_bytes = dim * (8 + 2 * 4 * nvec) + terms * (32 + max(32, 4 * nvec))  # bucket + x row per term
    t_s = prod_ms * 1e-3
    achieved_int = int_ops / t_s / 1e12
    kern_kind = "row-per-lane" if tuning.get("kernel") == 1 else "term-parallel"
    roofline = {
        "bound": "alu", "achieved": achieved_int, "peak": int_peak / 1e12, "unit": "TOP/s",
        "frac": achieved_int / (int_peak / 1e12),
        "traffic": (KERNEL_DRAM_BYTES_PER_NNZ[(kern_kind, nvec)] * nnz_total
                    if (kern_kind, nvec) in KERNEL_DRAM_BYTES_PER_NNZ else None),
        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the ring N=36 launch, "
                          "scaled by stored nonzeros",
        "kernel": (("k_matvec (row-per-lane" if kern_kind == "row-per-lane" else "k_matvec_tp (term-parallel")
                   + f", fp32, nvec={nvec}, "
                   + ("pruned rotation search" if tuning.get("search") != 0 else "search over every rotation")
                   + ", 64-bit words, bucketed index)"),
        "peak_kind": "measured live: int32 op mix of the search (funnel shift, lop3, min, add) on every SM",
        "int_ops_per_launch": int_ops, "int_ops_per_term": ops_term,
        "run_length_iterations_per_term": run_iters, "candidate_tops_per_term_and_coset": cands,
        "generated_terms_per_row": t_gen,
        "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / t_s / 1e9, "peak_gbs": hbm_peak,
                "frac": alg_bytes / t_s / 1e9 / hbm_peak, "peak_kind": pk_kind,
                "sector_bytes": sector_bytes, "sector_gbs": sector_bytes / t_s / 1e9},
    }
    buf = torch.empty(8 << 30, dtype=torch.uint8, device=dev)
    buf.fill_(1)
    gather_peak, _ = ed.peak("gather32", buf)
    del buf
    accesses = terms * 2 + dim  # one bucket and one x row per term, one key/x/y row per basis row
    roofline["random_access"] = {"accesses_per_launch": accesses, "achieved_per_s": accesses / t_s,
                                 "peak_per_s": gather_peak, "frac": accesses / t_s / gather_peak,
                                 "peak_kind": "measured live: random 32-byte reads over 8 GiB"}
    # the slower of the algorithmic bytes at the HBM peak and the search's
    # integer ops at the integer peak, against the measured launch time
    roofline_time = max(alg_bytes / (hbm_peak * 1e9), int_ops / int_peak)
    roofline["bytes_or_ops_frac"] = roofline_time / t_s

    # ---- CPU oracle on sampled rows of the same sector ---------------------------
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w)

    # ---- end to end through the C ABI: pinned host start block in, Ritz values
    # out, the same K block steps ----------------------------------------------
    X0_host = torch.empty(X0.shape, dtype=X0.dtype, pin_memory=True)
    X0_host.copy_(X0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X0.copy_(X0_host, non_blocking=True)
    eigs, _ = ed.lanczos_block(O, B, X0, nvec, args.steps, ed.ED_LANCZOS_F32_MATVEC | VO, n_eig=nvec)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e_value = dim * nvec * args.steps / e2e_s
    if world > 1:
        e2e_value = sum_over_ranks(e2e_value, world)
    h2d = X0_host.numel() * X0_host.element_size()
    del X0_host

    # ---- secondary: ring N=32 (config 2) products, L2 flushed ----------------------
    secondary = None
    if args.workload == "ring40":
        w2 = ei.workload("ring32")
        B2 = ed.basis_build(32, 16, +1, w2["perms"], w2["chars"])
        d2 = ed.basis_size(B2)
        st2, _ = ed.basis_states(B2)
        O2 = ed.operator_create(32, w2["op"]["sites"], w2["op"]["coeff"], w2["op"]["local"])
        secondary = {"workload": "ring32: Heisenberg ring N=32, Sz=0, k=0, p=+1, z=+1", "dim": d2}
        for name, dt, nv in (("f64", torch.float64, 1), ("f32", torch.float32, 1), ("f32_nvec8", torch.float32, 8)):
            xx = ei.x_by_state_torch_chunked(5, st2, nv, False, dtype=dt)
            yy = torch.empty_like(xx)
            ed.matvec(O2, B2, xx, yy, nv)
            ms = min(timed(lambda: ed.matvec(O2, B2, xx, yy, nv))[0] for _ in range(5))
            secondary[name] = {"ms": ms, "rows_per_s": nv * d2 / (ms * 1e-3)}
        del B2

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(w),
                   "dim": dim, "group_order": len(w["perms"]) * (2 if z else 1), "nvec": nvec,
                   "step": f"one block-Lanczos step: fp32 block product of {nvec} interleaved vectors + "
                           "block recurrence (double-float arithmetic, fp64 coefficients and merges)",
                   "value_counts": "H.x rows: basis rows x vectors per second",
                   "l2": "flushed before each timed region (inputs far larger than L2)",
                   "parallelism": f"replicas x{world}", "basis_build_ms": build_ms},
        "batched_product": {"ms": prod_ms, "rows_per_s": dim / t_s, "vector_rows_per_s": nvec * dim / t_s,
                            "nonzeros_per_s": nvec * nnz_total / t_s},
        "fp64_plain": {"value": rows_plain, "unit": UNIT, "ms_per_step": ms_plain / max(rplain.steps, 1),
                       "timed": f"the {plain_steps}-step fp64 Lanczos solve (values only), CUDA events",
                       "product_ms": prod64_ms, "rows_per_s_product": dim / (prod64_ms * 1e-3),
                       "nonzeros_per_s_product": nnz_total / (prod64_ms * 1e-3)},
        "speedup_fp32_batched_vs_fp64_plain": value / sum_over_ranks(rows_plain, world) if world > 1
        else rows_blk / rows_plain,
        "nonzeros_per_s": value * nnz_row,
        "nnz_per_row": nnz_row, "nnz_per_product": nnz_total,
        "solves": {"fp32_batched": {"e0": rfull.e0, "residual": rfull.residual, "block_steps": rfull.steps,
                                    "products": rfull.matvecs, "wall_s": t_blk_solve,
                                    "form": f"block Lanczos nvec={nvec}, {args.block_steps} steps, Ritz vector "
                                            "by a second pass, 6 fp64 refinement steps, fp64 Rayleigh "
                                            "quotient"},
                   "fp64_plain": {"e0": rplain.e0, "residual_estimate": rplain.residual,
                                  "steps": rplain.steps, "wall_s": t_plain_solve,
                                  "form": f"single-vector fp64 Lanczos, {plain_steps} steps, lowest Ritz value"}},
        "dE0": dE0,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "s": e2e_s, "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": 8 * nvec / args.steps,
                "path": "pinned host start block -> device, ed_lanczos_block over the same steps, Ritz "
                        "values -> host"},
        "autotune": {"product": tuning, "kernel_names": {"0": "library rule (term-parallel for fp32 blocks of 8)",
                                                          "1": "row-per-lane", "2": "term-parallel"},
                     "search_names": {"-1": "n/a", "0": "every rotation", "1": "pruned to the longest runs"}},
        "gpu_launches": launches,
        "clocks": clocks,
        "secondary": secondary,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ring40")
    ap.add_argument("--nvec", type=int, default=8,
                    help="block size of the FP32 batched path (and vectors per product in --mode matvec)")
    ap.add_argument("--block-steps", type=int, default=40,
                    help="block steps of the full FP32 batched solve behind dE0")
    ap.add_argument("--lanczos-steps", type=int, default=100,
                    help="Lanczos steps of the batched solve in --mode multi (0: skip)")
    ap.add_argument("--kernel-policy", default="auto", choices=["auto", "rowwise", "term_parallel"],
                    help="product kernel in --mode matvec (default: the library's rule)")
    ap.add_argument("--solve-modes", default="f32_matvec,f64",
                    help="Lanczos modes of --mode solve (comma-separated: f32_matvec, f64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="job", choices=["job", "matvec", "step", "solve", "multi", "push",
                                                      "peaks", "block"],
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
    if args.mode == "block":
        return run_block_steps(args, w)
    if args.mode == "solve":
        return run_solve(args, w)
    if args.mode == "push":
        return run_push(args, ei.workload(args.workload))
    if args.mode == "multi":
        return run_multi(args)

    return run_job(args, w)

if __name__ == "__main__":
    main()
