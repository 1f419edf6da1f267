"""Autotuner of the solver's launch shapes, persisted per (GPU, problem).

Tuned per multigrid level: the shape of the Schwarz apply (one thread block
per Schwarz block, or the owned rows of every block split over several
blocks, with a number of column groups per block), the thread mapping of the
V-cycle's block-sparse residual (threads per scalar row), and for the whole
instance the panel width of the tensor-core Gauss-Jordan factorisation.  The
candidates differ only in how work is mapped to threads (and so in the
rounding order of sums), never in what is computed.

``python -m paper_1709_05660_gb300.autotune --configs channel2d_l5 ...`` times
every candidate on the device with CUDA events (``fsi_time_level_kernels``;
the factorisation through the per-class counters) and writes the fastest into
``tuning.json`` beside this file, keyed by the GPU's name and by the problem's
signature (dimension, levels, coarse cells, block tile, precision: what fixes
the Schwarz block sizes and counts).  ``FSI(...)`` applies the entry of the
current GPU when there is one, so results are reproducible for a given table;
problems without an entry keep the library's built-in choice.
"""
import argparse
import json
import os
import time
from dataclasses import replace
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")

# apply shapes tried per level: (slices, column groups); slices 1 = one block per Schwarz block
APPLY_CANDIDATES = [(1, 4)] + [(s, g) for s in (2, 3, 4, 6, 8, 12, 16, 24, 32) for g in (4, 8, 16, 32)]
SPMV_CANDIDATES = (2, 4, 8)
# Gauss-Jordan variants: panel width 16, 24 or 32 (one thread block per SM), 216 = 16-column
# panels with half the tensor memory, two thread blocks per SM
PANEL_CANDIDATES = (16, 24, 32, 216)


def signature(prob, opts) -> str:
    cells = "x".join(str(len(b) - 1) for b in prob.breaks[:prob.dim])
    tile = "x".join(str(t) for t in opts.tile[:prob.dim])
    prec = "mixed" if opts.precision == 1 else "fp64"
    return f"{prob.dim}d-L{prob.levels}-c{cells}-t{tile}-{prec}"


def gpu_name() -> Optional[str]:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        pass
    return None


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except FileNotFoundError:
        return {}


def lookup(prob, opts, gpu: Optional[str] = None, table: Optional[dict] = None) -> Optional[dict]:
    table = load_table() if table is None else table
    gpu = gpu_name() if gpu is None else gpu
    if gpu is None:
        return None
    return table.get(gpu, {}).get(signature(prob, opts))


def check_entry(entry: dict, levels: int) -> None:
    """Raises ValueError unless ``entry`` holds valid launch shapes for a
    problem with ``levels`` levels (the ranges fsi_set_launch_params accepts)."""
    lv = entry.get("levels", {})
    for k, p in lv.items():
        l = int(k)
        if not 1 <= l < levels:
            raise ValueError(f"level {l} outside 1..{levels - 1}")
        if not 1 <= p["apply_slices"] <= 4096 or not 1 <= p["apply_groups"] <= 256:
            raise ValueError(f"apply shape out of range at level {l}")
        if p["spmv_sub"] not in SPMV_CANDIDATES:
            raise ValueError(f"spmv_sub out of range at level {l}")
    if entry.get("gj_panel", 0) not in (0,) + PANEL_CANDIDATES:
        raise ValueError("gj_panel out of range")


def apply_table(s, entry: Optional[dict] = None) -> Optional[dict]:
    """Sets the launch shapes of the table's entry on instance ``s``; returns
    the entry, or None (built-in shapes) when the table has none."""
    entry = lookup(s.prob, s.opts) if entry is None else entry
    if not entry:
        return None
    L = s.prob.levels
    check_entry(entry, L)
    panel = int(entry.get("gj_panel", 0))
    for l in range(1, L):
        p = entry["levels"].get(str(l), {})
        s.set_launch_params(l, apply_slices=int(p.get("apply_slices", 0)), apply_groups=int(p.get("apply_groups", 0)),
                            spmv_sub=int(p.get("spmv_sub", 0)), gj_panel=panel if l == L - 1 else 0)
    return entry


def _best(times: dict):
    return min(times.items(), key=lambda kv: kv[1])


def tune(prob, opts, stream: Optional[int] = None, reps: int = 40, trials: int = 3, log=print) -> dict:
    """Times every candidate shape on the current GPU; returns a table entry."""
    import torch
    from . import fsi
    from .workloads import noise

    s = fsi.FSI(prob, opts, stream=stream, tuned=False)
    try:
        N = int(s.N[-1])
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        s.initial_state(torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda"), y)
        if prob.transient:
            s.set_state(y, y, None, prob.dt)   # BDF1 start-up step from rest
        else:
            s.set_state(y)
        s.assemble()
        s.factor()
        L = prob.levels

        def timed(level, k):
            s.time_level_kernels(level, 2)   # warm-up
            return min(s.time_level_kernels(level, reps)[k] for _ in range(trials))

        entry = {"levels": {}}
        for l in range(1, L):
            shapes = {}
            for sl, g in APPLY_CANDIDATES:
                s.set_launch_params(l, apply_slices=sl, apply_groups=g)
                eff = s.get_launch_params(l)
                key = (eff["apply_slices"], eff["apply_groups"])
                if key not in shapes:
                    shapes[key] = timed(l, 0)
            s.set_launch_params(l)
            eff = s.get_launch_params(l)
            builtin = shapes.get((eff["apply_slices"], eff["apply_groups"]))
            (a_s, a_g), a_ms = _best(shapes)
            subs = {}
            # the thread mapping applies to the FP32 residual of 4 x 4 blocks (2D, mixed path)
            for sub in (SPMV_CANDIDATES if prob.dim == 2 and opts.precision == 1 else (4,)):
                s.set_launch_params(l, apply_slices=a_s, apply_groups=a_g, spmv_sub=sub)
                subs[sub] = timed(l, 1)
            sub, sub_ms = _best(subs)
            entry["levels"][str(l)] = dict(apply_slices=a_s, apply_groups=a_g, spmv_sub=sub,
                                           apply_ms=round(a_ms, 5), apply_builtin_ms=builtin and round(builtin, 5),
                                           spmv_ms=round(sub_ms, 5), spmv_sub4_ms=round(subs[4], 5))
            s.set_launch_params(l, apply_slices=a_s, apply_groups=a_g, spmv_sub=sub)
            log(f"  level {l}: apply {a_s}x{a_g} {a_ms * 1e3:.1f} us (built-in {builtin * 1e3 if builtin else 0:.1f}), "
                f"spmv sub {sub} {sub_ms * 1e3:.1f} us (4: {subs[4] * 1e3:.1f})")
        if opts.precision == 1:
            panels = {}
            top = entry["levels"][str(L - 1)]
            for w in PANEL_CANDIDATES:
                s.set_launch_params(L - 1, apply_slices=top["apply_slices"], apply_groups=top["apply_groups"],
                                    spmv_sub=top["spmv_sub"], gj_panel=w)
                s.set_profiling(True)
                for _ in range(trials):
                    s.factor()
                ks = s.kernel_stats()["patch_factor"]
                s.set_profiling(False)
                panels[w] = ks["ms"] / trials
            w, w_ms = _best(panels)
            entry["gj_panel"] = w
            entry["gj_panel_ms"] = {str(k): round(v, 4) for k, v in panels.items()}
            log(f"  Gauss-Jordan panel {w}: {w_ms:.3f} ms ({panels})")
        return entry
    finally:
        s.close()


def main():
    from .workloads import CONFIGS
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--configs", nargs="+", default=["channel2d_l5"])
    ap.add_argument("--precision", nargs="+", type=int, default=[1], help="1 mixed, 0 FP64")
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--reps", type=int, default=40)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    gpu = gpu_name()
    table = load_table(args.out)
    for name in args.configs:
        prob, opts = CONFIGS[name]
        for prec in args.precision:
            o = replace(opts, precision=prec)
            sig = signature(prob, o)
            print(f"{name} [{sig}] on {gpu}", flush=True)
            t0 = time.time()
            entry = tune(prob, o, stream=torch.cuda.current_stream().cuda_stream, reps=args.reps,
                         log=lambda m: print(m, flush=True))
            entry["tuned_on"] = name
            table.setdefault(gpu, {})[sig] = entry
            print(f"  {time.time() - t0:.1f} s", flush=True)
            with open(args.out, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
