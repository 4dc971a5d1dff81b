"""Benchmark: coupled solves/s to 1e-8 on the 3-field 3D coupled box.

Workload: 64^3 Q1 hex mesh, elasticity (3 dof/node) + heat + log-uniform
diffusion (1 dof/node each), all pairs coupled, 1,373,125 dofs; FGMRES(50)
to a 1e-8 true relative residual with the BGS(AMG) preconditioner (backward
sweep, SA-AMG, Chebyshev degree 2) computed in FP32 while the Krylov loop,
coarse LU and residuals stay FP64.  One step = one full solve from x0 = 0
with the hierarchy resident (setup excluded, timed separately).

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the same workload: each step is one whole oracle solve (all its FGMRES
iterations), the steps run concurrently in one single-threaded process per
host core, and the timed region is the wall time of the K timed steps.
"""
from __future__ import annotations

import os
import sys

if "reference" in sys.argv:
    # every oracle process computes on one core: one BLAS thread each
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[_v] = "1"

import argparse
import json
import statistics
import subprocess
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled solves/s to 1e-8 residual"
UNIT = "solves/s"
NE = 64
FALLBACK_HBM_GBS = 6800.0
# mesh edge of each workload unless --ne is given
DEFAULT_NE = {"box": 64, "cons": 64, "fsi": 48, "oseen": 48, "te2d": 32}


def solver_kw(args=None):
    """Hierarchy depth: the 2D thermo-elastic system takes 3 SA-AMG levels
    (coarsening continues to the third whatever its size), the 3D systems up
    to 5 levels with a coarsest level of at most 1000 dofs."""
    if args is not None and args.workload == "te2d":
        return dict(max_levels=3, coarse_max=0)
    return dict(max_levels=5, coarse_max=1000)
CLOCK_FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


def workload_config(args, s, extra=None):
    if args.workload == "fsi":
        what = f"4-field split-box saddle {NE}^3 Q1 ({s.ndofs} dofs: structure | mesh + PSPG Stokes u, p)"
    elif args.workload == "oseen":
        what = (f"4-field split-box saddle {NE}^3 Q1 with an Oseen velocity block, wind (0.2, 0.1, 0) ({s.ndofs} dofs), "
                f"velocity transfers {'R = P^T' if args.no_pg else 'Petrov-Galerkin'}")
    elif args.workload == "te2d":
        what = (f"2-field thermo-elastic 2D {NE}x{NE} Q1 ({s.ndofs} dofs: plane-strain elasticity + transient heat), "
                f"3 SA-AMG levels")
    elif args.workload == "cons":
        what = (f"constrained 3-field box {NE}^3 Q1 + 4 patch-mean Lagrange multipliers ({s.ndofs} dofs, "
                f"zero multiplier block)")
    else:
        what = f"3-field 3D coupled box {NE}^3 Q1 ({s.ndofs} dofs: elasticity+heat+diffusion)"
    pname = args.precond.upper()
    if args.precond == "simple" and args.simple_pred == "amg_bgs":
        pname = "SIMPLE(AMG(BGS))"
    cfg = {
        "workload": f"{what}, {pname} preconditioner in {args.precision.upper()}, FGMRES(50), rtol 1e-8",
        "ndofs": s.ndofs,
        "precond": args.precond,
        "precision": args.precision,
        "l2": "L2 flushed between timed solves (256 MB write outside each solve's event pair)",
        "parallelism": "replicas" if args.gpus > 1 else "1 GPU",
    }
    if args.precond == "simple":
        cfg["simple_pred"] = args.simple_pred
    cfg["smoother"] = "gs" if args.smoother == "gs" or args.precond == "bgs_gs" else "chebyshev"
    cfg.update(extra or {})
    return cfg


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)

        def find(o):
            if isinstance(o, dict):
                for k, v in o.items():
                    if k == "hbm_gbs" and isinstance(v, (int, float)):
                        return float(v)
                    r = find(v)
                    if r:
                        return r
            return None
        v = find(d)
        if v:
            return v, "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mfs_clocks_{os.getpid()}_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={','.join(CLOCK_FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        sm, smax, reasons = [], [], set()
        names = CLOCK_FIELDS[5:]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) != len(CLOCK_FIELDS):
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:]):
                    if v.lower() == "active":
                        reasons.add(n.split(".")[-1])
        except OSError:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_timing(elapsed, steps, world, dist=None, device=None):
    """Replicas: every rank solves its own copy of the workload; the job's
    time is the slowest rank's (all_reduce MAX) and its throughput counts
    every rank's solves.  Returns (solves per second, slowest elapsed)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    return world * steps / elapsed, elapsed


def kernel_source_digest(kernel):
    """sha256 of the device source of a kernel variant family (its __global__
    function and the row helper it calls), to tell whether stored ncu
    counters still describe the current code."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_1605_01522_gb300", "csrc", "kernels.cu")).read()
    fn = {"smooth_sell": ["sell_row", "d_smooth"], "spmv_sell": ["sell_row", "d_spmv"],
          "smooth_sell4": ["sell_row", "d_smooth"], "spmv_sell4": ["sell_row", "d_spmv"],
          "smooth_sell8": ["sell_row", "d_smooth"], "spmv_sell8": ["sell_row", "d_spmv"],
          "spmv_rows": ["d_spmv_rows"], "smooth_warp": ["bsr_warp_row", "d_smooth_warp"],
          "spmv_warp": ["bsr_warp_row", "d_spmv_warp"]}.get(kernel.split("<")[0])
    if fn:
        fn = fn + ["k_solo"]  # the single-system kernel wrapper every launch goes through
    if not fn:
        return None
    h = hashlib.sha256()
    for f in fn:
        m = re.search(r"(template <[^>]*>\s*)?(__device__|__global__)[^{;]*\b" + f + r"\(", src)
        if not m:
            return None
        depth, i = 0, src.index("{", m.end())
        for j in range(i, len(src)):
            depth += {"{": 1, "}": -1}.get(src[j], 0)
            if depth == 0:
                h.update(src[m.start():j + 1].encode())
                break
    return h.hexdigest()


def ncu_traffic(kernel, rows):
    """DRAM bytes per launch of this kernel at this size from the committed ncu
    capture table, or None if absent or captured from different kernel code."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            table = json.load(f)
    except OSError:
        return None
    for e in table.get("entries", []):
        if e["kernel"] == kernel and e["rows"] == rows:
            if e.get("source_sha256") != kernel_source_digest(kernel):
                return None
            return e["traffic_bytes_per_launch"]
    return None


def make_system(args=None):
    from paper_1605_01522_gb300 import inputs
    w = args.workload if args is not None else "box"
    if w == "fsi":
        return inputs.fsi_box(ne=NE, seed=2)
    if w == "cons":
        return inputs.constrained_box(ne=NE, nfields=3, seed=5)
    if w == "oseen":
        s = inputs.fsi_box(ne=NE, seed=2, wind=(0.2, 0.1, 0.0))
        if args.no_pg:
            s.fields[2].petrov_galerkin = False
        return s
    if w == "te2d":
        return inputs.thermo_elastic_2d(ne=NE, seed=0)
    return inputs.coupled_box_3d(ne=NE, nfields=3, seed=1)


def precond_extra(args):
    """Preconditioner options of the workload (the split box uses SIMPLE with a
    diagonal A~11 over the predictor fields S, G, Fu and the pressure as Schur field;
    --simple-pred picks SIMPLE's predictor solver)."""
    extra = {}
    if args.workload in ("fsi", "oseen") and args.precond in ("simple", "amg_simple"):
        extra = dict(simple_group=[0, 0, 0, 1], simple_approx="diag")
    if args.precond == "simple" and args.simple_pred != "bgs_amg":
        extra["simple_pred"] = args.simple_pred
    if args.smoother == "gs" or args.precond == "bgs_gs":
        extra["smoother"] = "gs"
    if getattr(args, "vcycle_tail", False):
        extra["vcycle_tail"] = 1
    if getattr(args, "pdl", -1) != -1:
        extra["pdl"] = args.pdl
    return extra


def oracle_params(args):
    """The oracle's parameter block for the library options of precond_extra."""
    from oracle import precond
    from oracle.cycles import SmootherParams
    ex = dict(precond_extra(args))
    ex.pop("vcycle_tail", None)  # launch forms of the library, not method parameters
    ex.pop("pdl", None)
    sm = SmootherParams("gs", omega=0.79, sweeps=1) if ex.pop("smoother", None) == "gs" else None
    return precond.Params(args.precond, **solver_kw(args), **ex, smoother=sm)


# ---------------------------------------------------------------------------
# The FP64 CPU oracle, timed by whole solves
# ---------------------------------------------------------------------------

_ORACLE = {}  # the forking process's operator, hierarchy and right-hand side


def oracle_prepare(args):
    """Build the workload and the oracle's own hierarchy (untimed); returns
    (system, setup seconds)."""
    from oracle import amg, precond
    s = make_system(args)
    A = s.scipy_blocks()
    D = precond.assemble(A, s.nfields)
    t0 = time.perf_counter()
    M = precond.Preconditioner(A, [amg.FieldSpec.of(f) for f in s.fields], oracle_params(args))
    _ORACLE.update(D=D, M=M, rhs=s.rhs)
    return s, time.perf_counter() - t0


def _oracle_worker(core, tasks, results):
    """Forked worker: pinned to one core, runs whole FGMRES(50) solves from
    x0 = 0 to 1e-8 on the inherited (read-only) operator and hierarchy."""
    from oracle import krylov
    try:
        os.sched_setaffinity(0, {core})
    except OSError:
        pass
    D, M, rhs = _ORACLE["D"], _ORACLE["M"], _ORACLE["rhs"]
    while True:
        cmd = tasks.get()
        if cmd is None:
            return
        count, budget, xpath = cmd
        out, t_start = [], time.perf_counter()
        while True:
            t0 = time.perf_counter()
            r = krylov.fgmres(lambda v: D @ v, M, rhs, 1e-8, 50)
            out.append((time.perf_counter() - t0, r.iters, float(r.relres)))
            if xpath and len(out) == 1:  # the oracle's solution, for the GPU arm's error against it
                np.save(xpath, r.x)
            done = len(out) >= count if count else time.perf_counter() - t_start >= budget
            if done:
                break
        results.put((core, out))


class OraclePool:
    """One single-threaded oracle process per host core, forked from the
    process that built the hierarchy (copy-on-write, never written after the
    fork; this process has made no CUDA call)."""

    def __init__(self, cores):
        import multiprocessing as mp
        ctx = mp.get_context("fork")
        self.cores = list(cores)
        self.tasks = [ctx.SimpleQueue() for _ in self.cores]
        self.results = ctx.SimpleQueue()
        self.procs = [ctx.Process(target=_oracle_worker, args=(c, q, self.results), daemon=True)
                      for c, q in zip(self.cores, self.tasks)]
        for p in self.procs:
            p.start()

    def run(self, cmds):
        """cmds[i] = (count, budget_s, xpath) for worker i, or None to leave it
        idle; a worker runs `count` solves, or (count 0) solves until budget_s
        has passed (at least one), and saves its first solution to xpath
        (.npy) unless xpath is None.  Returns (wall seconds from the first command
        to the last result, [(seconds, iters, relres) of every solve])."""
        t0 = time.perf_counter()
        busy = 0
        for q, c in zip(self.tasks, cmds):
            if c is not None:
                q.put(c)
                busy += 1
        out = []
        for _ in range(busy):
            out += self.results.get()[1]
        return time.perf_counter() - t0, out

    def close(self):
        for q in self.tasks:
            q.put(None)
        for p in self.procs:
            p.join(timeout=10)


def split_steps(total, nproc):
    return [(total // nproc + (1 if i < total % nproc else 0), 0.0, None) if i < total else None
            for i in range(nproc)]


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores.  One step = one whole
    solve; the K timed steps run concurrently, one single-threaded process
    per core (at most K processes), after W warm-up solves spread the same
    way; ms_per_step = wall time of the K timed steps / K."""
    if rank != 0:
        return
    s, setup_s = oracle_prepare(args)
    cores = sorted(os.sched_getaffinity(0))
    nproc = max(1, min(len(cores), args.steps))
    pool = OraclePool(cores[:nproc])
    if args.warmup:
        pool.run(split_steps(args.warmup, nproc))
    wall, res = pool.run(split_steps(args.steps, nproc))
    pool.close()
    value = args.steps / wall
    iters = sorted({r[1] for r in res})
    sample = (f"{args.steps} whole FGMRES(50) solves to 1e-8 of the FP64 oracle (numpy/scipy, {iters} iterations "
              f"each, true residual <= {max(r[2] for r in res):.2e}) run concurrently by {nproc} single-threaded "
              f"processes pinned one per host core (after {args.warmup} warm-up solves); the oracle's own "
              f"hierarchy built once before the processes fork ({setup_s:.1f} s, untimed)")
    cfg = workload_config(args, s, {"oracle_iters": iters, "oracle_setup_s": round(setup_s, 1),
                                    "solve_s_mean": statistics.mean(r[0] for r in res)})
    cfg["precision"] = "fp64"
    cfg["l2"] = "host cores (no GPU L2 involved); the oracle's matrices are read from host memory"
    cfg["workload"] = cfg["workload"].replace(f"in {args.precision.upper()}", "in FP64 (the CPU oracle)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_oracle_baseline(args):
    """CPU-baseline child of the GPU arm: prepares the oracle, forks one
    process per core, prints "ready", and after a line on stdin (the GPU
    arm's measurements are over) times whole solves on one core alone, then
    on every core at once; prints the result as one JSON line."""
    s, setup_s = oracle_prepare(args)
    cores = sorted(os.sched_getaffinity(0))
    pool = OraclePool(cores)
    print("ready", flush=True)
    sys.stdin.readline()
    budget = args.baseline_s
    w1, r1 = pool.run([(0, budget, args.oracle_x)] + [None] * (len(cores) - 1))
    wn, rn = pool.run([(0, budget, None)] * len(cores))
    pool.close()
    print(json.dumps({"single": {"solves": len(r1), "wall_s": w1, "value": len(r1) / w1,
                                 "iters": sorted({r[1] for r in r1}), "relres": max(r[2] for r in r1)},
                      "all": {"solves": len(rn), "wall_s": wn, "value": len(rn) / wn, "cores": len(cores),
                              "iters": sorted({r[1] for r in rn})},
                      "setup_s": setup_s}), flush=True)


class BaselineChild:
    """The oracle baseline in a separate process, started before any GPU work
    so that its preparation overlaps the GPU setup and warm-ups; the timed GPU
    solves wait until it is prepared (wait_ready), and its own timed solves
    start only when result() is called, after the GPU measurements."""

    def __init__(self, args):
        self.xpath = os.path.join(tempfile.gettempdir(), f"mfs_oracle_x_{os.getpid()}.npy")
        cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--oracle-baseline",
               "--workload", args.workload, "--ne", str(NE), "--precond", args.precond,
               "--smoother", args.smoother, "--simple-pred", args.simple_pred,
               "--baseline-s", str(args.baseline_s), "--oracle-x", self.xpath] + (["--no-pg"] if args.no_pg else [])
        self.proc = subprocess.Popen(cmd, stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True)

    def wait_ready(self):
        """Block until the child has built its hierarchy and forked its
        processes (so that no oracle work runs beside the timed GPU solves)."""
        for line in self.proc.stdout:
            if line.strip() == "ready":
                return

    def result(self):
        self.proc.stdin.write("go\n")
        self.proc.stdin.flush()
        res = None
        for line in self.proc.stdout:
            line = line.strip()
            if line.startswith("{"):
                res = json.loads(line)
        self.proc.wait()
        return res

    def solution(self):
        """The oracle's solution of the workload (x0 = 0, tol 1e-8), or None."""
        try:
            x = np.load(self.xpath)
            os.remove(self.xpath)
            return x
        except OSError:
            return None


def run_mfs(args, rank, world):
    import torch
    from paper_1605_01522_gb300 import mfs

    # the oracle baseline runs in its own process: start it before any GPU
    # work (its preparation overlaps ours; its solves wait for release)
    child = BaselineChild(args) if world == 1 and not args.no_cpu_baseline else None
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    s = make_system(args)
    stream = torch.cuda.Stream(device=dev)
    prm = mfs.default_params(precond=args.precond, precision=args.precision, profile=1,
                             cuda_stream=stream.cuda_stream, no_graphs=int(args.no_graphs), **solver_kw(args),
                             **precond_extra(args))
    t0 = time.perf_counter()
    lib = mfs.Solver(s, params=prm)
    setup_s = time.perf_counter() - t0
    n = s.ndofs
    with torch.cuda.stream(stream):
        b = torch.from_numpy(s.rhs).to(dev)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream.synchronize()
    infos = []
    # warm-up 1 times every launch to find the dominant sparse kernel and the
    # class shares; the other warm-ups and the timed region time only that
    # kernel (one event pair per launch of it), so the timed solves run at
    # full speed while its launch durations are measured live
    x.zero_()
    torch.cuda.synchronize()
    lib.solve(b, x, tol=1e-8)
    detail_all = lib.kernel_detail()
    stats_all = lib.kernel_stats(reset=True)
    dom = [r for r in detail_all if r[0].startswith(("spmv", "smooth"))][0]
    lib.profile_filter(dom[5], dom[1])
    for _ in range(max(1, args.warmup - 1)):
        x.zero_()
        torch.cuda.synchronize()
        _, info, rc = lib.solve(b, x, tol=1e-8)
    lib.kernel_stats(reset=True)
    # each timed solve is bracketed by its own event pair; between solves a
    # 256 MB write (twice the 129 MB L2) evicts the previous solve's data, so
    # every solve starts from HBM even when its matrices would fit in L2
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if child is not None:
        child.wait_ready()  # the oracle's preparation must not share the host with the timed solves
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                x.zero_()
            evs[k][0].record(stream)
            _, info, rc = lib.solve(b, x, tol=1e-8)
            evs[k][1].record(stream)
            infos.append(info)
            if rc != mfs.OK:
                raise RuntimeError(f"solve failed rc={rc} info={info}")
        torch.cuda.synchronize()
        # the FP64 FMA rate of this GPU at the clocks of the timed region
        # (the denominator of the float64 kernels' roofline)
        fp64_peak = mfs.fp64_rate(stream.cuda_stream)
    elapsed = sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3
    if dist:
        dist.barrier()
    value, elapsed = reduce_timing(elapsed, args.steps, world, dist, dev)
    detail = lib.kernel_detail()
    stats = lib.kernel_stats(reset=True)
    # true residual, recomputed through the library's FP64 matvec (device)
    r = b - lib.matvec(x)
    relres = float(torch.linalg.norm(r) / torch.linalg.norm(b))
    x_last = x.cpu().numpy()  # the last timed solve's solution (x0 = 0), compared with the oracle's below
    # end-to-end: host (pinned) vectors, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        bh = torch.from_numpy(s.rhs.copy()).pin_memory()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        e2e_times = []
        for k in range(max(2, args.steps // 2) + 1):
            xh.zero_()
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
            stream.synchronize()
            t1 = time.perf_counter()
            _, info_h, rc = lib.solve(bh.numpy(), xh.numpy(), tol=1e-8)
            dt = time.perf_counter() - t1
            if k > 0:
                e2e_times.append(dt)
        lib.kernel_stats(reset=True)
        e2e = {"value": world / statistics.mean(e2e_times), "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * n,
               "d2h_bytes_per_step": 8 * n}
    # the V-cycles timed whole: preconditioner applications through mfs_apply
    # (each one = every V-cycle kernel of one FGMRES iteration, plus the two
    # float64 <-> float32 conversions), launched back to back with no
    # per-launch events, bracketed by one event pair on the solver's stream
    with torch.cuda.stream(stream):
        v_in = b / torch.linalg.norm(b)
        z_out = torch.empty_like(v_in)
    for _ in range(3):
        lib.apply(v_in, z_out)
    n_apply = 20
    ea = torch.cuda.Event(enable_timing=True)
    eb = torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(n_apply):
        lib.apply(v_in, z_out)
    eb.record(stream)
    eb.synchronize()
    apply_ms = ea.elapsed_time(eb) / n_apply
    # roofline of the dominant kernel, timed live over the timed region.
    # float64 sparse kernels are bound by GB300's FP64 FMA rate (ncu: SM
    # throughput ~80 % while DRAM is ~50 %), float32 ones by HBM bandwidth.
    hbm_peak, peak_kind = measured_hbm_peak()
    kname, krows, launches, ms, nbytes, _, flops = detail[0]
    gbps = nbytes / (ms / 1e3) / 1e9
    tflops = flops / (ms / 1e3) / 1e12
    if kname.endswith("f64>"):
        roof = {"bound": "alu", "achieved": tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": tflops / fp64_peak,
                "peak_kind": "measured (mfs_fp64_rate: independent FP64 FMA chains on every SM, best of 5, "
                             "right after the timed region)",
                "fp64_nominal_TFLOPs": 1.25, "hbm_GBps": gbps, "hbm_frac": gbps / hbm_peak,
                "hbm_peak": hbm_peak, "hbm_peak_kind": peak_kind}
    else:
        roof = {"bound": "hbm", "achieved": gbps, "peak": hbm_peak, "unit": "GB/s", "frac": gbps / hbm_peak,
                "peak_kind": peak_kind}
    traffic = ncu_traffic(kname, krows)
    roof.update({"kernel": f"{kname} ({krows} block rows)", "traffic": traffic,
                 "algorithmic_bytes_per_launch": nbytes / launches, "flops_per_launch": flops / launches,
                 "launches": launches, "avg_launch_us": ms / launches * 1e3})
    tot_ms = sum(r[3] for r in detail_all)
    top = [{"kernel": r[0], "rows": r[1], "launches": r[2], "share": round(r[3] / tot_ms, 4),
            "GBps": round(r[4] / (r[3] / 1e3) / 1e9, 1)} for r in detail_all[:8]]
    f32 = [r for r in detail_all if r[0].endswith("f32>")]
    secondary = None
    if f32:
        r = f32[0]
        g = r[4] / (r[3] / 1e3) / 1e9
        secondary = {"kernel": f"{r[0]} ({r[1]} block rows)", "bound": "hbm", "achieved": g, "peak": hbm_peak,
                     "unit": "GB/s", "frac": g / hbm_peak, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(r[0], r[1]), "timed": "warm-up solve, every launch timed"}
    # the V-cycles as a whole: every sparse preconditioner kernel (smoothing,
    # residual, coupling, restriction, prolongation on every level; not the
    # GMRES matvec), algorithmic bytes over summed launch time, warm-up solve
    pre = [r for r in detail_all
           if r[0].startswith(("spmv", "smooth")) and "<" in r[0] and not r[0].startswith("spmv_rows")]
    vcycle = None
    if pre:
        vb, vms = sum(r[4] for r in pre), sum(r[3] for r in pre)
        by_rows = {}
        for r in pre:  # block rows identify the matrix size (fine level, coarse levels, transfers)
            e = by_rows.setdefault(r[1], [0.0, 0.0, 0])
            e[0] += r[4]
            e[1] += r[3]
            e[2] += r[2]
        groups = sorted(by_rows.items(), key=lambda kv: -kv[1][1])[:6]
        vcycle = {"GBps": vb / (vms / 1e3) / 1e9, "frac": vb / (vms / 1e3) / 1e9 / hbm_peak, "peak": hbm_peak,
                  "peak_kind": peak_kind, "share_of_solve_time": vms / tot_ms,
                  "by_block_rows": [{"rows": k, "GBps": round(v[0] / (v[1] / 1e3) / 1e9, 1),
                                     "share_of_vcycle_time": round(v[1] / vms, 4), "launches": v[2]}
                                    for k, v in groups],
                  "timed": "warm-up solve, every launch timed (algorithmic bytes / summed event time)"}
        it_w = max(1, infos[-1]["iters"])
        vcycle["wall"] = {"GBps": vb / it_w / (apply_ms / 1e3) / 1e9,
                          "frac": vb / it_w / (apply_ms / 1e3) / 1e9 / hbm_peak,
                          "ms_per_apply": apply_ms, "bytes_per_apply": vb / it_w,
                          "timed": f"{n_apply} back-to-back preconditioner applications (mfs_apply, the "
                                   "V-cycle kernels of one iteration + 2 precision conversions), one event "
                                   "pair, no per-launch events; bytes = the V-cycle kernels' algorithmic "
                                   "bytes per iteration of the warm-up solve"}
    stats = stats_all
    launches_total = sum(v[0] for v in stats_all.values()) * args.steps
    if rank != 0:
        return
    cpu = None
    vs_oracle = None
    if child is not None:
        b = child.result()
        xo = child.solution()
        if b and xo is not None:
            vs_oracle = {"x_rel_err": float(np.linalg.norm(x_last - xo) / np.linalg.norm(xo)),
                         "iters": infos[-1]["iters"], "oracle_iters": b["single"]["iters"],
                         "true_relres": relres, "oracle_relres": b["single"]["relres"],
                         "note": "||x - x_oracle|| / ||x_oracle||, same system and right-hand side, x0 = 0; "
                                 "the FP64 CPU oracle with its own hierarchy"}
        if b:
            one, alln = b["single"], b["all"]
            cpu = {"value": one["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{one['solves']} whole FGMRES(50) solve(s) to 1e-8 of the FP64 oracle (numpy/scipy, "
                             f"{one['iters']} iterations, true residual {one['relres']:.2e}) on one host core, "
                             f"{one['wall_s']:.1f} s; own hierarchy built untimed ({b['setup_s']:.1f} s); run after "
                             f"the GPU measurements",
                   "all_cores": {"value": alln["value"], "unit": UNIT, "cores": alln["cores"],
                                 "sample": f"{alln['solves']} whole solves by {alln['cores']} single-threaded "
                                           f"processes pinned one per core, started together, "
                                           f"{alln['wall_s']:.1f} s wall"}}
    shares = {c: round(v[1] / max(1e-9, sum(u[1] for u in stats.values())), 4) for c, v in stats.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32p" else "f64",
        "data": "synthetic",
        "config": workload_config(args, s, {"iters": infos[-1]["iters"], "true_relres": relres,
                                            "setup_s": round(setup_s, 2), "levels": infos[-1]["levels"],
                                            "kernel_class_share": shares, "top_kernels": top}),
        "roofline": roof,
        "roofline_top_f32": secondary,
        "vcycle": vcycle,
        "vs_oracle": vs_oracle,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches_total),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    lib.close()


def run_batch(args, rank, world):
    """Batched workload: 256 independent 2-field 3D boxes, n_e log-uniform in
    [12, 48], seeded right-hand sides, solved together by mfs_solve_batch
    (one setup per distinct mesh size, clones for the other systems).  Not
    the headline line: reported beside it."""
    import torch
    from paper_1605_01522_gb300 import inputs, mfs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    if args.batch_kind == "te2d":
        # many copies of the 3,267-dof 2D thermo-elastic system, fresh right-hand sides
        te = inputs.thermo_elastic_2d(ne=32, seed=0)
        sizes = np.full(args.nsys, 32)
        mats = {32: te}
        rhs = [inputs.system_rhs(te, 6000 + k) for k in range(args.nsys)]
        kw = dict(max_levels=3, coarse_max=0)
    else:
        sizes, mats, rhs = inputs.batch_workload(args.nsys, 12, 48, 3)
        kw = solver_kw(args)
    t1 = time.perf_counter()
    # layouts tuned for throughput (many systems on the GPU at once)
    base = {ne: mfs.Solver(sy, precond=args.precond, precision=args.precision, layout_tune=1, pdl=args.pdl, **kw)
            for ne, sy in mats.items()}
    solvers, used = [], set()
    for ne in sizes.tolist():
        solvers.append(base[ne] if ne not in used else base[ne].clone())
        used.add(ne)
    t2 = time.perf_counter()
    bs = [torch.from_numpy(b).to(dev) for b in rhs]
    xs = [torch.zeros_like(b) for b in bs]

    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)

    def batch(nthreads):
        for x in xs:
            x.zero_()
        flush.fill_(1.0)  # evict the previous step's data from L2
        torch.cuda.synchronize()
        ta = time.perf_counter()
        res = mfs.solve_batch(solvers, bs, xs, tol=1e-8, nthreads=nthreads)
        return time.perf_counter() - ta, res

    # the first fused call records, merges and captures (timed apart)
    t_plan, _ = batch(args.threads)
    for _ in range(args.warmup):
        batch(args.threads)
    times, infos = [], None
    for _ in range(args.steps):
        dt, (_, infos, status) = batch(args.threads)
        times.append(dt)
        if any(status):
            raise RuntimeError(f"batch failed: {status}")
    pool = None
    if args.threads == 0:  # the thread-pool form beside it
        batch(16)
        pool = args.nsys / batch(16)[0]
    # the same systems one after the other
    seq = []
    for sv, b, x in zip(solvers, bs, xs):
        x.zero_()
        torch.cuda.synchronize()
        ta = time.perf_counter()
        sv.solve(b, x, tol=1e-8)
        seq.append(time.perf_counter() - ta)
    value = args.nsys * args.steps / sum(times)
    iters = [i["iters"] for i in infos]
    # roofline of the whole batch: algorithmic bytes of every kernel of every
    # system's solve (per mesh size: one profiled solo solve, bytes per
    # iteration) over the batch time
    per_iter = {}
    for ne, sy in mats.items():
        with mfs.Solver(sy, precond=args.precond, precision=args.precision, layout_tune=1, profile=1, **kw) as sv:
            k = sizes.tolist().index(ne)
            _, inf, _ = sv.solve(bs[k], torch.zeros_like(bs[k]), tol=1e-8)
            per_iter[ne] = sum(v[2] for v in sv.kernel_stats(reset=True).values()) / max(1, inf["iters"])
    batch_bytes = sum(per_iter[ne] * it for ne, it in zip(sizes.tolist(), iters))
    hbm_peak, peak_kind = measured_hbm_peak()
    gbps = batch_bytes / statistics.mean(times) / 1e9
    roof = {"bound": "hbm", "achieved": gbps, "peak": hbm_peak, "unit": "GB/s", "frac": gbps / hbm_peak,
            "peak_kind": peak_kind, "traffic": None,
            "kernel": "the whole batch: algorithmic bytes of every kernel of every solve (per mesh size from a "
                      "profiled solo solve, per iteration, times each system's iterations) / mean step time",
            "bytes_per_step": batch_bytes}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32p" else "f64",
            "data": "synthetic",
            "config": {"workload": (f"batch of {args.nsys} independent 2-field 3D coupled boxes, n_e log-uniform "
                                    f"in [12,48]" if args.batch_kind == "box2" else
                                    f"batch of {args.nsys} 2-field thermo-elastic 2D systems (32x32 Q1, 3,267 dofs, "
                                    f"3 SA-AMG levels) with different right-hand sides")
                                   + f", {args.precond.upper()} {args.precision.upper()}, FGMRES(50), rtol 1e-8 each",
                       "step": "one mfs_solve_batch over all systems (host-timed, synchronous)",
                       "executor": "fused: one multi-system launch per step, one CUDA graph per FGMRES iteration"
                                   if args.threads == 0 else f"{args.threads} host threads on per-handle streams",
                       "first_call_s": round(t_plan, 3), "threadpool16_solves_per_s": pool,
                       "l2": "L2 flushed between steps (256 MB write before each step)",
                       "distinct_meshes": len(mats), "total_dofs": int(sum(b.numel() for b in bs)),
                       "iters_mean": statistics.mean(iters), "iters_max": max(iters),
                       "sequential_solves_per_s": args.nsys / sum(seq),
                       "batch_speedup_vs_sequential": value / (args.nsys / sum(seq)),
                       "generate_s": round(t1 - t0, 1), "setup_and_clone_s": round(t2 - t1, 1)},
            "roofline": roof}
    print(json.dumps(line), flush=True)
    for sv in solvers:
        sv.close()


def run_serve(args, rank, world):
    """Serving workload: Poisson arrivals of solve requests, each a 2- or
    3-field 3D box with n_e from {16,24,32,48,64}, 30 % reusing a resident
    hierarchy with a new right-hand side, admission by an HBM budget,
    concurrent solves.  Reports p50/p99 latency and solves/s."""
    import torch
    from paper_1605_01522_gb300 import inputs, serving
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    sizes = [int(v) for v in args.serve_sizes.split(",")]
    pool = {(ne, nf): inputs.coupled_box_3d(ne=ne, nfields=nf, seed=4) for ne in sizes for nf in (2, 3)}
    rhs = {key: [inputs.system_rhs(sy, 4000 + 10 * i + k) for k in range(3)] for i, (key, sy) in enumerate(pool.items())}
    rng = np.random.default_rng(4)
    keys = list(pool)
    gaps = rng.exponential(1.0 / args.rate, size=args.requests)
    picks = rng.integers(len(keys), size=args.requests)
    reuse = rng.random(args.requests) < 0.3
    workers = args.threads or 16
    srv = serving.Server(hbm_budget=int(args.hbm_gb * (1 << 30)), workers=workers, max_setups=args.max_setups,
                         fused=args.serve_fused,
                         precond=args.precond, precision=args.precision, **solver_kw(args))
    t0 = time.perf_counter()
    t = t0
    for i in range(args.requests):
        t += gaps[i]
        delay = t - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        key = keys[picks[i]]
        srv.submit(key, pool[key], rhs[key][i % 3], bool(reuse[i]))
    srv.drain()
    st = srv.stats()
    srv.close()
    line = {"metric": METRIC, "value": st["solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.requests,
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "fp32p" else "f64", "data": "synthetic",
            "config": {"workload": f"serving: {args.requests} Poisson requests at {args.rate}/s, 2- or 3-field 3D boxes, "
                                   f"n_e in {sizes}, 30 % reuse a resident hierarchy, HBM budget {args.hbm_gb} GB, "
                                   f"{workers} workers, at most {args.max_setups} setups at once, "
                                   f"{'fused batched solves' if args.serve_fused else 'one stream per request'}, "
                                   f"{args.precond.upper()} {args.precision.upper()}, rtol 1e-8",
                       **st}}
    print(json.dumps(line), flush=True)


def main():
    global NE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mfs", choices=["mfs", "reference"])
    ap.add_argument("--precond", default="bgs_amg", choices=["bgs_amg", "amg_bgs", "simple", "amg_simple", "bgs_gs"])
    ap.add_argument("--smoother", default="chebyshev", choices=["chebyshev", "gs"],
                    help="level smoother: Chebyshev degree 2, or multicolour damped Gauss-Seidel (omega 0.79)")
    ap.add_argument("--precision", default="fp32p", choices=["fp32p", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--ne", type=int, default=None,
                    help="mesh edge (default: 64 for box/cons, 48 for fsi/oseen, 32 for te2d)")
    ap.add_argument("--oracle-baseline", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-x", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--baseline-s", type=float, default=10.0,
                    help="CPU baseline: each oracle process runs whole solves for at least this long (one at least)")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--pdl", type=int, default=-1,
                    help="programmatic dependent launch of the solve-phase kernels: 1 on, 0 off, "
                         "N > 1 for launches of at most N CTAs, -1 (default) automatic")
    ap.add_argument("--vcycle-tail", action="store_true",
                    help="one-CTA V-cycle tails (the level above the coarsest and the coarse solve in one launch)")
    ap.add_argument("--no-pg", action="store_true", help="oseen workload: R = P^T on the velocity field")
    ap.add_argument("--workload", default="box", choices=["box", "fsi", "cons", "oseen", "te2d", "batch", "serve"],
                    help="box: the 64^3 three-field system (headline); fsi: the 48^3 split-box saddle; "
                         "cons: the box with 4 Lagrange-multiplier constraints (zero diagonal block); "
                         "oseen: the split box with a non-symmetric Oseen velocity block (Petrov-Galerkin AMG); "
                         "te2d: the 2-field thermo-elastic 2D system (3,267 dofs at --ne 32); "
                         "batch: 256 independent systems; serve: Poisson request stream")
    ap.add_argument("--simple-pred", default="bgs_amg", choices=["bgs_amg", "amg_bgs"],
                    help="SIMPLE's predictor solver: BGS(AMG) sweep or AMG(BGS) V-cycle")
    ap.add_argument("--nsys", type=int, default=256)
    ap.add_argument("--batch-kind", default="box2", choices=["box2", "te2d"],
                    help="batch: the 256 2-field 3D boxes, or copies of the 2D thermo-elastic system")
    ap.add_argument("--threads", type=int, default=0,
                    help="batch: 0 = fused executor, > 0 = that many host threads on per-handle streams; "
                         "serve: worker threads (0 = 16)")
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--hbm-gb", type=float, default=150.0)
    ap.add_argument("--max-setups", type=int, default=8, help="serve: setups in flight at once")
    ap.add_argument("--serve-sizes", default="16,24,32,48,64")
    ap.add_argument("--serve-fused", action="store_true",
                    help="serve: solve the ready requests together with the fused batch executor")
    args = ap.parse_args()
    NE = args.ne if args.ne is not None else DEFAULT_NE.get(args.workload, 64)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.oracle_baseline:
        run_oracle_baseline(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch":
        run_batch(args, rank, world)
    elif args.workload == "serve":
        run_serve(args, rank, world)
    else:
        run_mfs(args, rank, world)


if __name__ == "__main__":
    main()
