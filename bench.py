"""Benchmark: Newton-step solves/s of the 2D channel-with-flap FSI problem at
1e-8 relative error against the CPU oracle's solution, mixed vs FP64.

One step = one whole Newton step through the libfsi C-ABI on resident device
data: residual + exact Jacobian assembly, Galerkin coarse operators, Schwarz
block and coarse factorisation, FGMRES(30) with the multigrid V-cycle, and the
Newton update (fsi_newton_step).  Every step starts from the same seeded
linearisation state, so every step does the same work and its correction can
be compared with the oracle's x* (tests/golden/xstar_<workload>.npz).

Default workload: 6 levels (finest 512x128 quads, 1,250,308 unknowns), shear
modulus 2e6, mean inflow 1.0, 4x4-element Schwarz blocks (uneven, up to
372 unknowns).  Each path runs at the loosest FGMRES tolerance (of 1e-8, 1e-9,
1e-10, 1e-11) whose correction is within 1e-8 of x*, found first by a sweep:
the mixed path (FP32 V-cycle and Schwarz inverses, FP64 FGMRES,
true-residual products and coarse LU) gives `value`; the plain FP64 path is
reported under `fp64_path`.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
For N > 1 (torchrun) every rank runs an independent replica of the workload
(the path is not sharded; "scaling": "weak").
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1709_05660_gb300.workloads import CONFIGS, noise  # noqa: E402

METRIC = "Newton-step solves/s at 1e-8 rel. error, mixed vs FP64; served p50/p99 ms"
ERR_BAR = 1e-8
RTOL_SWEEP = (1e-8, 1e-9, 1e-10, 1e-11)
UNIT = "solves/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
FALLBACK_BF16_SUSTAINED_TFLOPS = 1700.0
# FP64 ALU peak derived from the unit counts and clocks: 152 SMs x 2.07 GHz x
# 4 FP64 flop / clock / SM (the 1.25 TFLOP/s nominal FP64 rate of the part).
FP64_ALU_PEAK_GFLOPS = 152 * 2.07 * 4.0
# FP32 CUDA-core peak: 152 SMs x 2.07 GHz x 128 FP32 FMA / clock / SM x 2 flop.
FP32_ALU_PEAK_GFLOPS = 152 * 2.07 * 256.0
HBM_BOUND = {"patch_apply", "spmv", "transfer", "krylov", "scatter"}
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return None, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region.
    The sampler is started before the warm-up (nvidia-smi takes a while to
    come up) and polls every 50 ms with a timestamp; begin() / end() mark the
    timed region, and only samples whose timestamps fall inside it count
    (the nearest one if none does)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        import datetime
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]),
                             {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"}))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return out
        t0 = self.t0 if self.t0 is not None else rows[0][0]
        t1 = self.t1 if self.t1 is not None else rows[-1][0]
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if not inside:   # region shorter than the polling interval: the sample nearest to it
            mid = 0.5 * (t0 + t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        reasons = set().union(*(r[3] for r in inside))
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside), "poll_ms": 50}


# ----------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------

class OracleSampler:
    """Times bounded samples of one Newton step of the CPU oracle on the
    benchmark workload and scales them to a full step: the residual and exact
    Jacobian of `frac` of the finest elements, the full Galerkin hierarchy,
    partial-pivot LU of `frac` of every level's Schwarz blocks plus the coarse
    LU, and one FGMRES iteration (V-cycle, product, CGS2) times `iters`
    iterations.  The operators the sample needs are built once, untimed, by
    `__init__`.  With a process pool the element assembly and the block LUs
    of the sample are spread over its workers (the oracle's own functions,
    one single-threaded process per core); the Galerkin products, the coarse
    LU and the Krylov iteration stay in this process."""

    def __init__(self, cfg: str):
        from oracle import fem, solver as osolver
        from oracle.mesh import initial_state
        self.cfg = cfg
        self.fem, self.osolver = fem, osolver
        self.prob, self.opts = CONFIGS[cfg]
        self.orc = osolver.Oracle(self.prob, self.opts)
        lev = self.orc.fine
        self.y = initial_state(self.prob, lev, noise(lev.N, 0))
        self.r, self.J = self.orc.assemble(self.y)
        self.orc.factor()

    def sample(self, frac: float, iters: int, pool=None, nworkers: int = 1):
        import scipy.linalg as sla
        fem, osolver, orc, prob, opts = self.fem, self.osolver, self.orc, self.prob, self.opts
        lev = orc.fine
        rng = np.random.default_rng(0)
        ne = max(1, int(frac * lev.n_elem))
        sel = np.sort(rng.choice(lev.n_elem, ne, replace=False))
        chunks = []
        for solid in (True, False):
            es = sel[lev.elem_solid[sel] == solid]
            step = 2048 if pool is None else max(1, -(-len(es) // (4 * nworkers)))
            chunks += [es[s0:s0 + step] for s0 in range(0, len(es), step)]
        t0 = time.perf_counter()
        if pool is None:
            for es in chunks:
                fem.element_system(prob, lev, es, self.y)
        else:
            list(pool.map(_pool_assemble, chunks))
        t_asm = (time.perf_counter() - t0) / frac
        t0 = time.perf_counter()
        Jc = self.J
        for l in range(prob.levels - 1, 0, -1):
            P, R = orc._transfers[l - 1]
            Jc = osolver.galerkin(Jc, P, R, orc.levels_mesh[l - 1])
        t_gal = time.perf_counter() - t0
        t_fac = 0.0
        for l, op in enumerate(orc.ops):
            if l == 0:
                t0 = time.perf_counter()
                sla.lu_factor(op.J.toarray())
                t_fac += time.perf_counter() - t0
                continue
            Jd = op.J.tocsr()
            npch = len(op.patches)
            k = max(1, int(frac * npch))
            blocks = [Jd[op.patches[i].dofs][:, op.patches[i].dofs].toarray() for i in range(k)]
            t0 = time.perf_counter()
            if pool is None:
                for B in blocks:
                    sla.lu_factor(B)
            else:
                list(pool.map(_pool_lu, blocks))
            t_fac += (time.perf_counter() - t0) * npch / k
        t0 = time.perf_counter()
        osolver.fgmres(self.J, -self.r, orc.precond, restart=opts.restart, rtol=opts.rtol, max_iters=1)
        t_it = time.perf_counter() - t0
        total = t_asm + t_gal + t_fac + iters * t_it
        detail = {"assemble_s": t_asm, "galerkin_s": t_gal, "factor_s": t_fac, "fgmres_iter_s": t_it,
                  "iters": iters, "frac": frac}
        return total, detail


_POOL_STATE = {}


def _pool_init(cfg):
    from oracle.mesh import build_level, initial_state
    prob, _ = CONFIGS[cfg]
    lev = build_level(prob, prob.levels - 1)
    _POOL_STATE.update(prob=prob, lev=lev, y=initial_state(prob, lev, noise(lev.N, 0)))


def _pool_assemble(elems):
    from oracle import fem
    st = _POOL_STATE
    fem.element_system(st["prob"], st["lev"], elems, st["y"])
    return len(elems)


def _pool_lu(B):
    import scipy.linalg as sla
    sla.lu_factor(B)
    return B.shape[0]


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


SINGLE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                     "OPENBLAS_MAIN_FREE": "1"}


def cpu_sample_main(cfg: str, frac: float, iters: int, out: str):
    """Child process of the cpu_baseline leg (started with one BLAS / OpenMP
    thread): builds the oracle operators of `cfg`, then times the bounded
    sample serially and with a pool of one single-threaded process per core.
    Writes a JSON dict to `out`."""
    import multiprocessing as mp
    t0 = time.perf_counter()
    smp = OracleSampler(cfg)
    setup_s = time.perf_counter() - t0
    serial, dser = smp.sample(frac, iters)
    res = {"cfg": cfg, "setup_s": setup_s, "serial": {"solve_s": serial, "detail": dser, "cores": 1}}
    n = _cores()
    if n > 1:
        ctx = mp.get_context("spawn")
        with ctx.Pool(n, initializer=_pool_init, initargs=(cfg,)) as pool:
            pool.map(_pool_lu, [np.eye(4)] * n)          # workers up before timing
            allc, dall = smp.sample(frac, iters, pool=pool, nworkers=n)
        res["all_cores"] = {"solve_s": allc, "detail": dall, "cores": n}
    with open(out, "w") as f:
        json.dump(res, f)


class CpuBaseline:
    """The cpu_baseline leg: the oracle sample in a child process started
    before the GPU measurements (its operator set-up overlaps them)."""

    def __init__(self, cfg: str, frac: float, iters: int):
        self.out = tempfile.NamedTemporaryFile(suffix=".json", delete=False).name
        env = dict(os.environ, **SINGLE_THREAD_ENV)
        env.pop("CUDA_VISIBLE_DEVICES", None)
        self.cfg, self.frac, self.iters = cfg, frac, iters
        self.proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--_cpu-sample", cfg,
                                      "--cpu-frac", str(frac), "--ref-iters", str(iters), "--_out", self.out],
                                     env=env, stdout=subprocess.DEVNULL, stderr=subprocess.PIPE)

    def result(self, timeout: float):
        try:
            self.proc.wait(timeout=timeout)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            return None, "oracle sample did not finish in time"
        try:
            d = json.load(open(self.out))
        except Exception:
            return None, "oracle sample failed: " + (self.proc.stderr.read() or b"").decode()[-300:]
        finally:
            try:
                os.unlink(self.out)
            except OSError:
                pass
        ser = d["serial"]
        out = {"value": 1.0 / ser["solve_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{self.cfg}: {self.frac:.4f} of the finest-level element assembly and of each level's "
                         f"Schwarz block LUs (times scaled by 1/{self.frac:.4f}), the full Galerkin hierarchy and "
                         f"the coarse LU, one FGMRES iteration times {self.iters} iterations; one BLAS / OpenMP "
                         f"thread", "detail": ser["detail"], "setup_s": d["setup_s"]}
        if "all_cores" in d:
            a = d["all_cores"]
            out["all_cores"] = {"value": 1.0 / a["solve_s"], "cores": a["cores"], "detail": a["detail"],
                                "how": "the sampled element assembly and block LUs spread over one "
                                       "single-threaded process per core; Galerkin, coarse LU and Krylov "
                                       "iteration serial"}
        return out, None


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------

def run_reference(args, rank, world):
    """The reference arm: the CPU oracle (there is no reference program), on
    this arm's workload, metric and unit.  Every step is a bounded sample of
    one Newton step (see OracleSampler); `ms_per_step` is the time the sample
    actually took, `value` the solves/s it scales to."""
    if rank != 0:
        return
    cfg = args.config
    iters = args.ref_iters
    smp = OracleSampler(cfg)
    spent, scaled = [], []
    detail = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t, detail = smp.sample(args.ref_frac, iters)
        if i >= args.warmup:
            spent.append(time.perf_counter() - t0)
            scaled.append(t)
    val = 1.0 / statistics.mean(scaled)
    prob, opts = CONFIGS[cfg]
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(spent) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg, "levels": prob.levels, "tile": list(opts.tile)},
        "sample_fraction": args.ref_frac,
        "scaled_s_per_solve": statistics.mean(scaled),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step: {args.ref_frac:.4f} of the finest-level element assembly and of "
                                   f"each level's Schwarz block LUs (times scaled), full Galerkin hierarchy and "
                                   f"coarse LU, one FGMRES iteration times {iters} iterations; ms_per_step is the "
                                   f"time the sample took, value the full step it scales to", "detail": detail},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, dist) -> float:
    """Largest value of x over all ranks (x itself without a process group).
    The reduction tensor lives where the backend needs it: on the GPU for
    NCCL, on the host for gloo."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, seconds: float) -> float:
    """Units per second of the whole job: every rank runs `steps` units and the
    slowest rank's time counts."""
    return world * steps / seconds


def _golden_xstar(cfg: str):
    """The oracle's x* of the workload's seeded state, or None."""
    path = os.path.join(ROOT, "tests", "golden", f"xstar_{cfg}.npz")
    if not os.path.exists(path):
        return None
    g = np.load(path)
    return {"xstar": g["xstar"], "oracle_iters": int(g["oracle_iters"]), "how": str(g["how"])}


def _rel_err(dx, xs):
    if xs is None:
        return None
    d = dx.detach().cpu().numpy() if hasattr(dx, "detach") else dx
    return float(np.linalg.norm(d - xs) / np.linalg.norm(xs))


def _measure(args, prec, stream, barrier, dist, world, local, rtol=None, steps=None, warmup=None,
             prof_steps=None, e2e=True, xs=None):
    """Times `steps` Newton steps of one precision; returns a result dict."""
    import torch
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    prof_steps = steps if prof_steps is None else prof_steps
    prob, opts = CONFIGS[args.config]
    opts = replace(opts, precision=prec, rtol=opts.rtol if rtol is None else rtol)
    s = fsi.FSI(prob, opts, stream=stream.cuda_stream)
    N = int(s.N[-1])
    nz = torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda")
    y0 = torch.empty(N, dtype=torch.float64, device="cuda")
    s.initial_state(nz, y0)
    dx = torch.empty(N, dtype=torch.float64, device="cuda")

    def step():
        s.set_state(y0)
        return s.newton_step(dx)

    clocks = ClockSampler(local)
    clocks.start()                      # up and polling by the end of the warm-up
    for _ in range(warmup):
        rel, st = step()
    # headline: `steps` Newton steps timed with CUDA events, no per-kernel events
    launches0 = s.launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters, rel_res = [], []
    for _ in range(steps):
        rel, st = step()
        iters.append(st.iters)
        rel_res.append(st.rel_res)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = s.launch_count() - launches0
    err = _rel_err(dx, xs)
    # kernel classes: the same steps timed again with CUDA events around every
    # launch group of each class on the ctx stream (fsi_set_profiling)
    s.set_profiling(True)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(prof_steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    kst = s.kernel_stats()
    s.set_profiling(False)
    ms = max_over_ranks(ms, dist)
    out = {"N": N, "ms": ms, "per_step": ms / steps, "value": whole_job_rate(world, steps, ms / 1e3),
           "steps": steps, "warmup": warmup, "rtol": opts.rtol, "error_vs_oracle": err,
           "profiled_ms_per_step": ms_prof / prof_steps, "prof_steps": prof_steps,
           "iters": iters, "rel_res": max(rel_res), "rel_step": rel, "kst": kst, "launches": launches,
           "clocks": clk, "hbm_bytes": s.hbm_bytes, "tuned": s.tuning is not None,
           "phase_ms": {"assemble": st.t_assemble_ms, "factor": st.t_factor_ms, "solve": st.t_solve_ms}}
    if e2e:
        # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
        yh = y0.cpu().pin_memory()
        dxh = torch.empty(N, dtype=torch.float64).pin_memory()
        yh_np, dxh_np = yh.numpy(), dxh.numpy()
        s.set_state(yh_np)
        s.newton_step(dxh_np)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            s.set_state(yh_np)
            s.newton_step(dxh_np)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier()
        e2e_s = max_over_ranks(e2e_s, dist)
        out["e2e"] = {"value": whole_job_rate(world, steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": N * 8,
                      "d2h_bytes_per_step": N * 8, "error_vs_oracle": _rel_err(dxh_np, xs)}
    s.close()
    return out


def _rtol_sweep(cfg, prec, stream, xs, rtols=RTOL_SWEEP):
    """One Newton step at the seeded state for each FGMRES tolerance: the
    correction's relative error against the oracle's x*, iterations and
    device time.  Returns (entries, loosest rtol meeting ERR_BAR or None)."""
    import torch
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi

    prob, opts = CONFIGS[cfg]
    out, best = [], None
    for rt in rtols:
        s = fsi.FSI(prob, replace(opts, precision=prec, rtol=rt), stream=stream.cuda_stream)
        N = int(s.N[-1])
        y0 = torch.empty(N, dtype=torch.float64, device="cuda")
        s.initial_state(torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda"), y0)
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.set_state(y0)
        s.newton_step(dx)                # warm-up (V-cycle graph)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s.set_state(y0)
        e0.record(stream)
        _, st = s.newton_step(dx)
        e1.record(stream)
        torch.cuda.synchronize()
        err = _rel_err(dx, xs)
        out.append({"rtol": rt, "error_vs_oracle": err, "fgmres_iters": st.iters, "true_rel_res": st.rel_res,
                    "ms_per_step": e0.elapsed_time(e1)})
        s.close()
        if err is not None and err <= ERR_BAR and best is None:
            best = rt
    return out, best


def _measure_config(name, prec, stream, steps=3, warmup=2, xs=None, prob_over=None, **opts_over):
    """Newton steps of another configuration at its seeded state (as the
    headline: set_state, assemble, Galerkin, factor, FGMRES, update), device
    time with CUDA events over `steps` steps after `warmup` untimed ones."""
    import torch
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi

    prob, opts = CONFIGS[name]
    opts = replace(opts, precision=prec, **opts_over)
    if prob_over:
        prob = replace(prob, **prob_over)
    s = fsi.FSI(prob, opts, stream=stream.cuda_stream)
    N = int(s.N[-1])
    y0 = torch.empty(N, dtype=torch.float64, device="cuda")
    s.initial_state(torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda"), y0)
    dx = torch.empty(N, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        s.set_state(y0)
        s.newton_step(dx)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters, rel_res = [], 0.0
    for _ in range(steps):
        s.set_state(y0)
        _, st = s.newton_step(dx)
        iters.append(st.iters)
        rel_res = max(rel_res, st.rel_res)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"unknowns": N, "levels": prob.levels, "U": prob.U, "tile": list(opts.tile), "solves_per_s": steps / (ms / 1e3),
           "ms_per_step": ms / steps, "fgmres_iters": iters, "max_true_rel_residual": rel_res,
           "rtol": opts.rtol, "error_vs_oracle": _rel_err(dx, xs),
           "phase_ms": {"assemble": st.t_assemble_ms, "factor": st.t_factor_ms, "solve": st.t_solve_ms},
           "launch_shapes": "autotuned" if s.tuning is not None else "built-in"}
    s.close()
    return out


def _measure_full_newton(args, prec, stream, U=None, max_steps=20):
    """The benchmark workload's nonlinear driver: Newton from d = 0, u = the boundary-condition
    lift, p = 0 (no noise) until ||dx|| <= 1e-8 ||y||, each step assembling
    the exact Jacobian, the Galerkin hierarchy and the Schwarz / coarse
    factors on the device and solving with FGMRES.  Device time of every
    Newton step (CUDA events on the stream); solves/s averaged over the steps."""
    import torch
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi

    prob, opts = CONFIGS[args.newton_config]
    opts = replace(opts, precision=prec)
    if U is not None:
        prob = replace(prob, U=U)
    s = fsi.FSI(prob, opts, stream=stream.cuda_stream)
    N = int(s.N[-1])
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    s.initial_state(torch.zeros(N, dtype=torch.float64, device="cuda"), y)
    s.set_state(y)
    ms, iters, rels, rel_res, status = [], [], [], 0.0, "converged"
    for _ in range(max_steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            rel, st = s.newton_step()
        except fsi.FSIError as err:
            status = str(err).split(":")[0]
            break
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        iters.append(st.iters)
        rels.append(rel)
        rel_res = max(rel_res, st.rel_res)
        if rel <= 1e-8:
            break
    else:
        status = "max_steps"
    s.close()
    tot = sum(ms)
    return {"newton_steps": len(ms), "status": status, "rel_step": rels, "fgmres_iters": iters,
            "ms_per_newton_step": tot / max(1, len(ms)), "newton_solves_per_s": len(ms) / (tot / 1e3) if tot else None,
            "ms_to_steady_state": tot, "max_true_rel_residual": rel_res}


def _measure_transient_3d(args, stream):
    """3D time-dependent workload (box channel with a plate, 27-node hexahedra,
    3 levels, 908,422 unknowns, mixed precision): args.t3d_steps BDF time steps
    of dt = 0.01 (BDF1 start-up step, then BDF2) at t = dt, 2 dt, ..., each
    solved by Newton to ||dx|| <= 1e-8 ||y|| with the pulsating inflow
    alpha(t) = (1 + sin 2 pi t) / 2, from the inflow-profile state of the
    amplitude alpha(0) (displacement noise of the seeded state).  Device time of every Newton step (CUDA
    events on the stream); the kernel-class breakdown comes from the Newton
    steps of the first time step, run with per-class events (profiled steps
    are excluded from the totals)."""
    import torch
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi

    prob, opts = CONFIGS["box3d_l3_bdf2"]
    s = fsi.FSI(prob, opts, stream=stream.cuda_stream)
    N = int(s.N[-1])
    # start at rest relative to the inflow of t = 0: the state of the inflow
    # amplitude alpha(0) = 1/2 (a plan-only instance with U alpha(0) gives it
    # on the host), so the first steps see the amplitude change smoothly
    plan = fsi.FSI(replace(prob, U=prob.U * 0.5 * (1.0 + np.sin(0.0))), opts, plan_only=True)
    yh = np.empty(N)
    plan.initial_state(noise(N, 0), yh)
    plan.close()
    y = torch.tensor(yh, dtype=torch.float64, device="cuda")
    y0 = y.clone()
    # profiled pass: the first time step's Newton steps with per-class events
    s.set_profiling(True)
    s.set_state(y0, y0, None, prob.dt)
    nprof = 0
    for _ in range(10):
        rel, _ = s.newton_step()
        nprof += 1
        if rel < 1e-8:
            break
    kst = s.kernel_stats()
    s.set_profiling(False)
    yp, ypp = y0.clone(), None
    newton, iters, rel_res, ms_tot = 0, [], 0.0, 0.0
    per_step, rels, failed = [], [], None
    for n in range(1, args.t3d_steps + 1):
        s.set_state(yp, yp, ypp, n * prob.dt)
        k = 0
        step_rels = []
        for k in range(1, 11):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            try:
                rel, st = s.newton_step()
            except fsi.FSIError as err:
                failed = {"time_step": n, "newton_step": k, "status": str(err).split(":")[0]}
                break
            e1.record(stream)
            torch.cuda.synchronize()
            ms_tot += e0.elapsed_time(e1)
            newton += 1
            iters.append(st.iters)
            step_rels.append(rel)
            rel_res = max(rel_res, st.rel_res)
            if rel < 1e-8:
                break
        rels.append(step_rels)
        if failed:
            break
        per_step.append(k)
        ynew = torch.empty_like(y)
        s.get_state(ynew)
        ypp, yp = yp, ynew
    s.close()
    _, classes = _roofline(kst, nprof, fp32_classes=("patch_factor",), traffic_key="box3d_l3_bdf2 mixed")
    return {"workload": "box3d_l3_bdf2 (3D BDF2, dt 0.01, 64x16x16 hexahedra, 3 levels, mixed)", "unknowns": N,
            "time_steps": len(per_step), "time_steps_asked": args.t3d_steps, "failed": failed,
            "newton_steps_per_time_step": per_step, "rel_steps": rels,
            "newton_solves_per_s": newton / (ms_tot / 1e3), "time_steps_per_s": len(per_step) / (ms_tot / 1e3),
            "ms_per_newton_step": ms_tot / newton, "fgmres_iters": iters, "max_true_rel_residual": rel_res,
            "kernel_classes": classes}


def _roofline(kst, steps, fp32_classes=(), traffic_key=None):
    peaks, kind = _peaks()
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) if peaks else FALLBACK_HBM_GBS
    dom = max(kst, key=lambda k: kst[k]["ms"])
    d = kst[dom]
    per_launch_ms = d["ms"] / max(1, d["launches"])
    if dom in HBM_BOUND:
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": kind}
    elif dom in fp32_classes:
        # the mixed path's Schwarz factorisation: its contraction (the rank-W
        # trailing update) runs on the tensor cores in TF32 (3xTF32 split);
        # peak = the bf16 dense peak (sustained: the kernel is timed inside a
        # long step) x the nominal TF32 / BF16 ratio 1.1 / 2.25
        bf16 = float(peaks.get("bf16_tflops_sustained", FALLBACK_BF16_SUSTAINED_TFLOPS)) if peaks else \
            FALLBACK_BF16_SUSTAINED_TFLOPS
        peak = bf16 * 1.1 / 2.25
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"{kind} bf16 sustained {bf16:.0f} TFLOP/s x nominal tf32/bf16 1.1/2.25",
                "dtype": "tf32 (3xTF32 split, FP32 accumulate)",
                "flops": "algorithmic Gauss-Jordan flops 2 n^3 per block (the tensor pipe executes 3x that)"}
    else:
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "alu", "achieved": achieved / 1e3, "peak": FP64_ALU_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": achieved / FP64_ALU_PEAK_GFLOPS,
                "peak_source": "derived FP64 ALU peak (152 SM x 2.07 GHz x 4 flop/clk)", "dtype": "f64"}
    roof.update({"kernel": dom, "traffic": _traffic(traffic_key, dom), "launches": d["launches"],
                 "avg_launch_ms": per_launch_ms})
    classes = {k: {"ms_per_step": v["ms"] / steps, "launches": v["launches"],
                   "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None,
                   "hbm_frac": (v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm_peak) if v["ms"] > 0 else None,
                   "GFLOPs": (v["flops"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None}
               for k, v in kst.items()}
    # FP64-pipe-bound classes: the Krylov product (16 FMAs per 4 x 4 block) and
    # the element and Galerkin kernels (executed FP64 operations, counted with
    # ncu per element): their fraction of the derived FP64 ALU peak
    for name in ("operator", "assemble", "galerkin"):
        op = classes.get(name)
        if op and op["GFLOPs"]:
            op["fp64_frac"] = op["GFLOPs"] / FP64_ALU_PEAK_GFLOPS
    return roof, classes


def _soft(fn, *a, **kw):
    """A secondary measurement: its failure is recorded in the line instead
    of ending the benchmark."""
    try:
        return fn(*a, **kw)
    except Exception as e:   # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def run_gpu(args, rank, world):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    cpu_leg = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_leg = CpuBaseline(args.config, args.cpu_frac, args.ref_iters)
    stream = torch.cuda.current_stream()
    prob, opts = CONFIGS[args.config]
    gold = _golden_xstar(args.config)
    xs = gold["xstar"] if gold else None
    # the loosest tolerance of each path whose correction meets ERR_BAR
    sweep = {}
    rt_mixed = rt_fp64 = opts.rtol
    if xs is not None and not args.no_sweep:
        sweep["mixed"], best = _rtol_sweep(args.config, 1, stream, xs)
        rt_mixed = best or min(RTOL_SWEEP)
        if not args.mixed_only:
            sweep["fp64"], best = _rtol_sweep(args.config, 0, stream, xs)
            rt_fp64 = best or min(RTOL_SWEEP)
    main = _measure(args, 1, stream, barrier, dist, world, local, rtol=rt_mixed, xs=xs)
    fp64 = None
    if not args.mixed_only:
        fs = min(args.steps, args.fp64_steps)
        fp64 = _measure(args, 0, stream, barrier, dist, world, local, rtol=rt_fp64, steps=fs, warmup=3,
                        prof_steps=min(fs, 2), xs=xs)
    roof, classes = _roofline(main["kst"], main["prof_steps"], fp32_classes=("patch_factor",),
                              traffic_key=f"{args.config} mixed")
    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded channel-with-flap state)",
            "config": {"workload": args.config, "unknowns": main["N"], "levels": prob.levels,
                       "tile": list(opts.tile), "mu_s": prob.mu_s, "U": prob.U, "restart": opts.restart,
                       "rtol": main["rtol"], "smoothing": [opts.n_pre, opts.n_post], "omega": opts.omega,
                       "precision": "mixed: FP32 V-cycle and Schwarz inverses, FP64 FGMRES / SpMV / coarse LU",
                       "l2": f"working set {main['hbm_bytes'] / 1e9:.2f} GB > L2 (129 MB); no flush",
                       "parallelism": "replicas" if world > 1 else "single",
                       "launch_shapes": ("autotuned (paper_1709_05660_gb300/tuning.json)" if main["tuned"]
                                         else "built-in")},
            "error_vs_oracle": main["error_vs_oracle"],
            "oracle_xstar": ({"how": gold["how"], "oracle_fgmres_iters": gold["oracle_iters"]} if gold else None),
            "rtol_sweep": sweep,
            "fgmres_iters": main["iters"], "max_true_rel_residual": main["rel_res"], "rel_step": main["rel_step"],
            "phase_ms": main["phase_ms"], "roofline": roof, "kernel_classes": classes,
            "kernel_classes_pass": "a second timed pass of the same steps with per-class CUDA events "
                                   f"({main['profiled_ms_per_step']:.2f} ms per step with the events)",
            "e2e": main["e2e"], "gpu_launches": main["launches"], "clocks": main["clocks"],
        }
        if fp64 is not None:
            r64, c64 = _roofline(fp64["kst"], fp64["prof_steps"], traffic_key=f"{args.config} fp64")
            line["fp64_path"] = {"value": fp64["value"], "ms_per_step": fp64["per_step"], "steps": fp64["steps"],
                                 "rtol": fp64["rtol"], "error_vs_oracle": fp64["error_vs_oracle"],
                                 "fgmres_iters": fp64["iters"], "max_true_rel_residual": fp64["rel_res"],
                                 "phase_ms": fp64["phase_ms"], "e2e": fp64["e2e"], "gpu_launches": fp64["launches"],
                                 "roofline": r64, "kernel_classes": c64, "clocks": fp64["clocks"]}
            line["mixed_over_fp64"] = main["value"] / fp64["value"]
        if not args.no_configs and world == 1:
            cfg = {}
            for name in args.side_configs:
                gx = _golden_xstar(name)
                cfg[name] = {"mixed": _soft(_measure_config, name, 1, stream, xs=gx["xstar"] if gx else None)}
                if not args.mixed_only:
                    cfg[name]["fp64"] = _soft(_measure_config, name, 0, stream, steps=2, warmup=1,
                                              xs=gx["xstar"] if gx else None)
                    if "error" not in cfg[name]["mixed"] and "error" not in cfg[name]["fp64"]:
                        cfg[name]["mixed_over_fp64"] = (cfg[name]["mixed"]["solves_per_s"] /
                                                        cfg[name]["fp64"]["solves_per_s"])
            line["configs"] = cfg
        if world == 1 and not args.no_configs:
            # ILU(0) local solvers for the fluid blocks (exact LU for the solid ones), the paper's
            # cheaper setting, against exact LU on the headline mesh at mean inflow 0.2: at the
            # workload's inflow 1.0 the ILU(0)-smoothed FGMRES stalls (in the oracle too)
            line["fluid_ilu"] = {
                "U": 0.2, "note": "at U = 1.0 FGMRES with ILU(0) fluid blocks stalls (oracle and device alike)",
                "ilu": _soft(_measure_config, args.config, 1, stream, prob_over={"U": 0.2}, rtol=1e-10,
                             local_solver=1),
                "lu": _soft(_measure_config, args.config, 1, stream, prob_over={"U": 0.2}, rtol=1e-10)}
        if not args.no_full_newton and world == 1:
            fn = {"workload": args.newton_config,
                  "start": "d = 0, u = boundary-condition lift, p = 0; stop at ||dx|| <= 1e-8 ||y||",
                  "note": "plain Newton (no damping or continuation); at the workload's mean inflow it diverges "
                          "from the lift in the oracle too, with direct solves, so the driver is also run at "
                          "mean inflow 0.2 on the same mesh"}
            nprob, _ = CONFIGS[args.newton_config]
            for U in (nprob.U, 0.2):
                key = f"U={U:g}"
                fn[key] = {"mixed": _soft(_measure_full_newton, args, 1, stream, U=U)}
                if not args.mixed_only:
                    fn[key]["fp64"] = _soft(_measure_full_newton, args, 0, stream, U=U)
            line["full_newton"] = fn
        if args.t3d_steps > 0 and world == 1:
            line["transient_3d"] = _soft(_measure_transient_3d, args, stream)
        if not args.no_serve and world == 1:
            line["served"] = _soft(run_serve, args, quiet=True)
        if cpu_leg is not None:
            cpu, why = cpu_leg.result(timeout=args.cpu_timeout)
            line["cpu_baseline"] = cpu if cpu else {"value": None, "unit": UNIT, "kind": "oracle", "note": why}
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# serving (continuous batching of Newton-step requests)
# ----------------------------------------------------------------------------

def serve_mix(seed: int, n_requests: int, max_levels: int, frac_3d: float = 0.25, max_levels_3d: int = 3):
    """Seeded request mix: 2D channel instances with levels uniform in
    [3, max_levels] and, with probability frac_3d, 3D box-channel instances
    with levels uniform in [2, max_levels_3d] (120,902 or 908,422 unknowns),
    shear modulus log-uniform in [1e4, 1e6], mean inflow uniform in
    [0.1, 0.3] (faster inflows make plain Newton with this smoother stall on
    the coarser meshes, in the oracle as on the GPU), 3-8 Newton steps each
    (tiles 2x2 up to 4 levels, 4x4 above, 2x2x2 in 3D)."""
    from paper_1709_05660_gb300.workloads import Problem, SolverOpts, problem_3d
    rng = np.random.Generator(np.random.PCG64(seed))
    insts, total = [], 0
    iid = 1
    while total < n_requests:
        is3d = rng.uniform() < frac_3d
        lv = int(rng.integers(2, max_levels_3d + 1)) if is3d else int(rng.integers(3, max_levels + 1))
        mu = float(10 ** rng.uniform(4, 6))
        U = float(rng.uniform(0.1, 0.3))
        steps = int(rng.integers(3, 9))
        steps = min(steps, n_requests - total)
        if is3d:
            insts.append((iid, problem_3d(levels=lv, mu_s=mu, U=U), SolverOpts(tile=(2, 2, 2)), steps))
        else:
            insts.append((iid, Problem(levels=lv, mu_s=mu, U=U), SolverOpts(tile=(2, 2) if lv <= 4 else (4, 4)),
                          steps))
        total += steps
        iid += 1
    # arrival order: interleave instances at random, keeping each instance's steps in order
    order = []
    remaining = {i[0]: i[3] for i in insts}
    while remaining:
        keys = sorted(remaining)
        k = keys[int(rng.integers(0, len(keys)))]
        order.append(k)
        remaining[k] -= 1
        if remaining[k] == 0:
            del remaining[k]
    return insts, order, rng


def _serve_once(insts, order, prec, slots, budget, arrivals=None):
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi
    spec = {i[0]: i for i in insts}
    sizes = {}
    for iid, prob, opts, _ in insts:
        plan = fsi.FSI(prob, opts, plan_only=True)
        sizes[iid] = int(plan.N[-1])
        plan.close()
    srv = fsi.Server(hbm_budget_bytes=budget, max_slots=slots)
    done_steps = {iid: 0 for iid in spec}
    tickets, rejected = [], []
    t0 = time.perf_counter()
    for r, iid in enumerate(order):
        if arrivals is not None:
            dt = arrivals[r] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
        _, prob, opts, steps = spec[iid]
        k = done_steps[iid]
        done_steps[iid] += 1
        try:
            tickets.append((iid, k, srv.submit(iid, prob, replace(opts, precision=prec),
                                               noise=noise(sizes[iid], iid) if k == 0 else None,
                                               last=(k == steps - 1))))
        except fsi.FSIError:
            rejected.append((iid, k))      # its instance was freed by an earlier failure
    srv.drain()
    wall = time.perf_counter() - t0
    res = [(iid, k, srv.poll(t)) for iid, k, t in tickets]
    evictions = srv.evictions()
    srv.close()
    good = [r for _, _, r in res if r["status"] == 0]
    lat = np.array([r["latency_ms"] for r in good]) if good else np.zeros(1)
    statuses = {}
    for _, _, r in res:
        statuses[str(r["status"])] = statuses.get(str(r["status"]), 0) + 1
    failed = sorted({iid for iid, _, r in res if r["status"] != 0})
    return {"solves_per_s": len(good) / wall, "wall_s": wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "requests": len(order), "completed": len(good),
            "statuses": statuses, "rejected": len(rejected), "evictions": evictions,
            "failed_instances": [(i, spec[i][1].dim, spec[i][1].levels, spec[i][1].mu_s, spec[i][1].U) for i in failed],
            "max_true_rel_residual": max([r["rel_res"] for r in good] or [0.0])}


def run_serve(args, n_requests=None, max_levels=None, quiet=False):
    """Mixed path: closed loop and Poisson arrivals at 0.8x the closed-loop
    capacity over the whole request stream.  FP64 path: closed loop over the
    first `serve_fp64_requests` requests of the same stream (the FP64 Schwarz
    factorisation of the 6-level and 3D instances takes seconds per step),
    compared with the mixed path on the same head of the stream."""
    n_requests = n_requests or args.serve_requests
    max_levels = max_levels or args.serve_max_levels
    insts, order, rng = serve_mix(0, n_requests, max_levels, args.serve_3d_frac, args.serve_max_levels_3d)
    budget = int(args.serve_budget_gb * 1e9)
    out = {}
    closed = _serve_once(insts, order, 1, args.serve_slots, budget)
    lam = 0.8 * closed["solves_per_s"]
    arr = np.cumsum(rng.exponential(1.0 / lam, size=len(order)))
    pois = _serve_once(insts, order, 1, args.serve_slots, budget, arrivals=arr)
    pois["arrival_rate_per_s"] = lam
    out["mixed"] = {"closed_loop": closed, "poisson": pois}
    nh = min(args.serve_fp64_requests, len(order))
    if nh > 0:
        head = order[:nh]
        used = set(head)
        hinsts = [i for i in insts if i[0] in used]
        # the head of the stream ends each of its instances at its last request in the head
        steps_in_head = {iid: head.count(iid) for iid in used}
        hinsts = [(iid, p, o, steps_in_head[iid]) for iid, p, o, _ in hinsts]
        out["head"] = {"requests": nh,
                       "mixed": _serve_once(hinsts, head, 1, args.serve_slots, budget),
                       "fp64": _serve_once(hinsts, head, 0, args.serve_slots, budget)}
        out["head"]["mixed_over_fp64"] = (out["head"]["mixed"]["solves_per_s"] /
                                          max(1e-12, out["head"]["fp64"]["solves_per_s"]))
    summary = {"requests": len(order), "instances": len(insts), "levels_2d": [3, max_levels],
               "levels_3d": [2, args.serve_max_levels_3d], "slots": args.serve_slots,
               "budget_gb": args.serve_budget_gb,
               "mix": f"2D channel (levels 3-{max_levels}) and, with probability {args.serve_3d_frac}, 3D box "
                      f"channel (levels 2-{args.serve_max_levels_3d}); mu_s log-U[1e4,1e6], U U[0.1,0.3], "
                      f"3-8 Newton steps per instance",
               "instances_3d": sum(1 for i in insts if i[1].dim == 3),
               **out}
    if not quiet:
        line = {"metric": "served Newton-step solves/s and p50/p99 latency (Poisson arrivals at 0.8x capacity)",
                "value": out["mixed"]["poisson"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
                "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic (seeded request mix)",
                "config": {"workload": "serving"}, "serving": summary}
        print(json.dumps(line), flush=True)
    return summary


def run_sweep(args):
    """The parameter studies of Sec. 4.4 on the synthetic workload, with the
    paper's solver settings (left-preconditioned GMRES(10), one classical
    Gram-Schmidt pass, rtol 1e-4 on the left-preconditioned residual,
    omega 0.7): Schwarz blocks of 4, 16, 64 and 256 elements (tiles 2x2 ...
    16x16) at 4 + 4 smoothing steps, and smoothing (pre, post) in (2,2),
    (2,4), (4,2), (4,4), (8,8) at 16-element blocks.  Per setting one Newton
    step at the seeded state after one untimed step: GMRES iterations, the
    average convergence rate rho of Sec. 4.2 and the device time of each
    phase (CUDA events)."""
    import torch
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    prob, base = CONFIGS[args.sweep_config]
    base = replace(base, krylov=1, restart=10, rtol=1e-4, gs_passes=1, omega=0.7, n_pre=4, n_post=4,
                   precision=args.sweep_precision)
    settings = [("block", t, (4, 4)) for t in ((2, 2), (4, 4), (8, 8), (16, 16))]
    settings += [("smoothing", (4, 4), sm) for sm in ((2, 2), (2, 4), (4, 2), (4, 4), (8, 8))]
    rows = []
    for kind, tile, (npre, npost) in settings:
        opts = replace(base, tile=tile, n_pre=npre, n_post=npost)
        ent = {"study": kind, "block_elements": tile[0] * tile[1], "tile": list(tile), "smoothing": [npre, npost]}
        try:
            s = fsi.FSI(prob, opts, stream=stream.cuda_stream, tuned=False)
            N = int(s.N[-1])
            y0 = torch.empty(N, dtype=torch.float64, device="cuda")
            s.initial_state(torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda"), y0)
            s.set_state(y0)
            s.newton_step()
            s.set_state(y0)
            t0 = time.perf_counter()
            _, st = s.newton_step()
            wall = time.perf_counter() - t0
            ent.update({"unknowns": N, "gmres_iters": st.iters, "rho": st.rho, "prec_rel_res": st.prec_rel_res,
                        "true_rel_res": st.rel_res, "assemble_ms": st.t_assemble_ms, "factor_ms": st.t_factor_ms,
                        "solve_ms": st.t_solve_ms, "step_wall_ms": wall * 1e3, "device_bytes": s.hbm_bytes})
            s.close()
        except Exception as e:   # noqa: BLE001
            ent["error"] = f"{type(e).__name__}: {e}"
        rows.append(ent)
        print(json.dumps(ent), file=sys.stderr, flush=True)
    line = {"metric": "paper-settings parameter studies (left GMRES(10), rtol 1e-4, omega 0.7)",
            "config": {"workload": args.sweep_config, "precision": "mixed" if args.sweep_precision else "fp64"},
            "sweep": rows}
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """A small case of one kernel for ncu captures (a few GB on the device):
    `gj` factors the 6-level channel's Schwarz blocks on the 4-level mesh
    (the same block sizes, 337 blocks in one launch) twice; `spmv` runs two
    V-cycles of the 5-level channel (residual vectors and matrices larger than
    L2); `ilu` does the same with ILU(0) fluid blocks at mean inflow 0.2;
    `krylov` solves one Newton step of the 5-level channel with FGMRES
    (Arnoldi kernels, FP64 operator products, V-cycles); `asm` assembles
    small 2D and 3D problems once in each time discretisation.  Prints the
    unknowns and the device bytes held."""
    import torch
    from dataclasses import replace
    from paper_1709_05660_gb300 import fsi

    torch.cuda.set_device(0)
    if args.profile_case == "asm":
        # one assembly (element matrices, scatter, Galerkin hierarchy) per
        # problem kind: 2D and 3D, steady, BDF and Crank-Nicolson
        from paper_1709_05660_gb300.workloads import Problem, SolverOpts, problem_3d
        out = []
        for prob, opts in [(Problem(levels=3, mu_s=5e5, U=0.2, transient=t), SolverOpts(tile=(2, 2), precision=1))
                           for t in (0, 1, 2)] + \
                          [(problem_3d(levels=2, mu_s=2e6, U=0.2, transient=t), SolverOpts(tile=(2, 2, 2), precision=1))
                           for t in (0, 1, 2)]:
            s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
            N = int(s.N[-1])
            y = torch.empty(N, dtype=torch.float64, device="cuda")
            s.initial_state(torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda"), y)
            s.set_state(y, y if prob.transient else None, y if prob.transient else None)
            s.assemble()
            torch.cuda.synchronize()
            out.append({"dim": prob.dim, "transient": prob.transient, "unknowns": N})
            s.close()
        print(json.dumps({"profile_case": "asm", "problems": out}))
        return
    prob, opts = CONFIGS[args.config]
    prob = replace(prob, levels=4 if args.profile_case == "gj" else 5)
    if args.profile_case == "ilu":   # ILU(0) fluid blocks at the inflow where they converge
        prob, opts = replace(prob, U=0.2), replace(opts, local_solver=1)
    s = fsi.FSI(prob, replace(opts, precision=1), stream=torch.cuda.current_stream().cuda_stream)
    N = int(s.N[-1])
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    s.initial_state(torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda"), y)
    s.set_state(y)
    s.assemble()
    for _ in range(2):
        s.factor()
    if args.profile_case in ("spmv", "ilu"):
        z = torch.empty(N, dtype=torch.float64, device="cuda")
        b = torch.randn(N, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        for _ in range(2):
            s.apply_vcycle(b, z)
    if args.profile_case == "krylov":
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.newton_solve_update(dx)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "workload": args.config, "levels": prob.levels,
                      "unknowns": N, "device_bytes": int(s.hbm_bytes)}))
    s.close()


_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def _traffic(key, kernel_class: str):
    """DRAM bytes per launch of the class's kernels on a workload ("<config>
    <precision>") from the committed ncu summaries, or None when none has been
    captured for the current kernel."""
    try:
        d = json.load(open(_TRAFFIC_FILE))
        return d.get(key, {}).get(kernel_class)
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="channel2d_l6")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed-only", action="store_true", help="skip the FP64-path measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the tolerance sweep (run at the workload's rtol)")
    ap.add_argument("--fp64-steps", type=int, default=5, help="timed steps of the FP64 path (at most --steps)")
    ap.add_argument("--serve", action="store_true", help="serving benchmark (request mix) instead")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-max-levels", type=int, default=6)
    ap.add_argument("--serve-max-levels-3d", type=int, default=3)
    ap.add_argument("--serve-fp64-requests", type=int, default=64,
                    help="head of the request stream served by both paths (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    ap.add_argument("--no-serve", action="store_true", help="skip the served run of the default line")
    ap.add_argument("--no-full-newton", action="store_true", help="skip the full Newton run to steady state")
    ap.add_argument("--newton-config", default="channel2d_l5", help="workload of the full Newton driver")
    ap.add_argument("--no-configs", action="store_true", help="skip the Newton-step timing of the side workloads")
    ap.add_argument("--side-configs", nargs="*", default=["channel2d_l3", "channel2d_l5"])
    ap.add_argument("--t3d-steps", type=int, default=20,
                    help="BDF time steps of the 3D transient workload in the default line (0: skip)")
    ap.add_argument("--serve-3d-frac", type=float, default=0.25, help="share of 3D instances in the request mix")
    ap.add_argument("--cpu-frac", type=float, default=1.0 / 32)
    ap.add_argument("--cpu-timeout", type=float, default=900.0)
    ap.add_argument("--ref-frac", type=float, default=1.0 / 64)
    ap.add_argument("--ref-iters", type=int, default=12)
    ap.add_argument("--sweep", action="store_true", help="paper-settings parameter studies instead")
    ap.add_argument("--sweep-config", default="channel2d_l5")
    ap.add_argument("--sweep-precision", type=int, default=1)
    ap.add_argument("--profile-case", choices=["gj", "spmv", "asm", "ilu", "krylov"], default=None,
                    help="run one small case of a kernel for an ncu capture instead")
    ap.add_argument("--_cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--_out", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args._cpu_sample:
        cpu_sample_main(args._cpu_sample, args.cpu_frac, args.ref_iters, args._out)
        return
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    elif args.sweep:
        if rank == 0:
            run_sweep(args)
    elif args.serve:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        if rank == 0:
            run_serve(args)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
