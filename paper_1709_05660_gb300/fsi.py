"""Thin ctypes binding of the libfsi C-ABI (argument marshalling only).

Every step of the Newton-step solve runs in libfsi's CUDA kernels; this
module converts Python descriptors into the C structs, passes pointers
(torch tensors on the GPU or numpy arrays on the host) and turns non-zero
status codes into exceptions.  There is no CPU fallback: if ``libfsi.so`` is
missing or no CUDA device is usable, calls raise.
"""
import ctypes
import os
from typing import Optional

import numpy as np

from .workloads import Problem, SolverOpts

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsi.so")

FSI_OK = 0
ERRORS = {
    -1: "FSI_E_INVALID", -2: "FSI_E_OOM", -3: "FSI_E_CUDA", -4: "FSI_E_SINGULAR",
    -5: "FSI_E_NOT_CONVERGED", -6: "FSI_E_NONFINITE", -7: "FSI_E_MESH_TANGLED",
    -8: "FSI_E_TIMEOUT", -9: "FSI_E_CANCELLED", 1: "FSI_PENDING",
}
MAX_BREAKS = 65

# exported symbols declared in include/fsi.h
SYMBOLS = (
    "fsi_build_hierarchy", "fsi_destroy", "fsi_last_error", "fsi_get_sizes", "fsi_initial_state",
    "fsi_set_state", "fsi_get_state", "fsi_assemble_jacobian", "fsi_factor_schwarz", "fsi_solve",
    "fsi_newton_update", "fsi_newton_step", "fsi_export_csr", "fsi_export_dofmap", "fsi_export_patches",
    "fsi_apply_operator", "fsi_apply_vcycle", "fsi_apply_smoother", "fsi_restrict", "fsi_prolong",
    "fsi_launch_count", "fsi_plan_hierarchy", "fsi_export_transfer", "fsi_set_profiling",
    "fsi_kernel_stats", "fsi_server_create", "fsi_serve_submit", "fsi_serve_poll", "fsi_serve_drain",
    "fsi_server_resident_bytes", "fsi_server_destroy", "fsi_coarse_solve_static", "fsi_set_launch_params",
    "fsi_get_launch_params", "fsi_time_level_kernels", "fsi_set_stream", "fsi_import_csr",
    "fsi_set_tc_wait_limit", "fsi_fmg_newton", "fsi_newton_solve_update", "fsi_factor_schwarz_batch",
    "fsi_server_set_batching", "fsi_server_set_eviction", "fsi_server_evictions", "fsi_serve_cancel",
)

# kernel classes for fsi_kernel_stats
KERNEL_CLASSES = ("assemble", "galerkin", "scatter", "patch_factor", "coarse_factor", "patch_apply",
                  "spmv", "transfer", "krylov", "operator")


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("levels", ctypes.c_int), ("n_breaks", ctypes.c_int * 3),
        ("breaks", (ctypes.c_double * MAX_BREAKS) * 3), ("flap_lo", ctypes.c_double * 3),
        ("flap_hi", ctypes.c_double * 3), ("rho_f", ctypes.c_double), ("mu_f", ctypes.c_double),
        ("rho_s", ctypes.c_double), ("mu_s", ctypes.c_double), ("U", ctypes.c_double),
        ("transient", ctypes.c_int), ("dt", ctypes.c_double), ("ale_op", ctypes.c_int),
        ("mr_c2", ctypes.c_double),
    ]


class LaunchParams(ctypes.Structure):
    _fields_ = [("apply_slices", ctypes.c_int32), ("apply_groups", ctypes.c_int32),
                ("spmv_sub", ctypes.c_int32), ("gj_panel", ctypes.c_int32)]


class SolverOptsC(ctypes.Structure):
    _fields_ = [
        ("tile", ctypes.c_int * 3), ("n_pre", ctypes.c_int), ("n_post", ctypes.c_int),
        ("omega", ctypes.c_double), ("restart", ctypes.c_int), ("rtol", ctypes.c_double),
        ("max_iters", ctypes.c_int), ("precision", ctypes.c_int), ("krylov", ctypes.c_int),
        ("gs_passes", ctypes.c_int), ("local_solver", ctypes.c_int),
    ]


class SolveStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_res", ctypes.c_double),
        ("rho", ctypes.c_double), ("t_assemble_ms", ctypes.c_double), ("t_factor_ms", ctypes.c_double),
        ("t_solve_ms", ctypes.c_double), ("prec_rel_res", ctypes.c_double),
        ("bytes_assemble", ctypes.c_double), ("bytes_factor", ctypes.c_double), ("bytes_solve", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FMG_MAX_LEVELS = 16


class FmgStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("newton_steps", ctypes.c_int * FMG_MAX_LEVELS),
                ("krylov_iters", ctypes.c_int * FMG_MAX_LEVELS),
                ("last_rel_step", ctypes.c_double * FMG_MAX_LEVELS), ("ms", ctypes.c_double * FMG_MAX_LEVELS),
                ("status", ctypes.c_int)]

    def as_dict(self):
        L = self.levels
        return {"levels": L, "newton_steps": list(self.newton_steps[:L]), "krylov_iters": list(self.krylov_iters[:L]),
                "last_rel_step": list(self.last_rel_step[:L]), "ms": list(self.ms[:L]), "status": self.status}


class Request(ctypes.Structure):
    _fields_ = [
        ("instance", ctypes.c_uint64), ("desc", ProblemDesc), ("opts", SolverOptsC),
        ("noise", ctypes.c_void_p), ("last", ctypes.c_int), ("keep_dx", ctypes.c_int),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iters", ctypes.c_int), ("rel_step", ctypes.c_double),
        ("rel_res", ctypes.c_double), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
        ("latency_ms", ctypes.c_double), ("n", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libfsi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfsi.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    lib.fsi_build_hierarchy.argtypes = [ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolverOptsC), vp,
                                        ctypes.POINTER(vp)]
    lib.fsi_plan_hierarchy.argtypes = [ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolverOptsC),
                                       ctypes.POINTER(vp)]
    lib.fsi_export_transfer.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64p, vp, vp, vp]
    lib.fsi_destroy.argtypes = [vp]
    lib.fsi_destroy.restype = None
    lib.fsi_last_error.argtypes = [vp]
    lib.fsi_last_error.restype = ctypes.c_char_p
    lib.fsi_get_sizes.argtypes = [vp, i64p, i64p, i64p]
    lib.fsi_initial_state.argtypes = [vp, vp, vp]
    lib.fsi_set_state.argtypes = [vp, vp, vp, vp, ctypes.c_double]
    lib.fsi_get_state.argtypes = [vp, vp]
    lib.fsi_assemble_jacobian.argtypes = [vp, vp]
    lib.fsi_factor_schwarz.argtypes = [vp]
    lib.fsi_solve.argtypes = [vp, vp, vp, ctypes.POINTER(SolveStats)]
    lib.fsi_newton_update.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.fsi_newton_step.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveStats)]
    lib.fsi_export_csr.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.fsi_export_dofmap.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp]
    lib.fsi_export_patches.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, vp, vp, vp]
    lib.fsi_apply_operator.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.fsi_apply_vcycle.argtypes = [vp, vp, vp]
    lib.fsi_coarse_solve_static.argtypes = [vp, vp, vp]
    lib.fsi_set_stream.argtypes = [vp, vp]
    lib.fsi_newton_solve_update.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveStats)]
    lib.fsi_factor_schwarz_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.fsi_server_set_batching.argtypes = [vp, ctypes.c_int]
    lib.fsi_server_set_eviction.argtypes = [vp, ctypes.c_int]
    lib.fsi_serve_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.fsi_server_evictions.argtypes = [vp]
    lib.fsi_server_evictions.restype = ctypes.c_int64
    lib.fsi_fmg_newton.argtypes = [ctypes.POINTER(ProblemDesc), ctypes.POINTER(SolverOptsC), vp, ctypes.c_double,
                                   ctypes.c_int, vp, ctypes.POINTER(FmgStats)]
    lib.fsi_import_csr.argtypes = [vp, ctypes.c_int, vp]
    lib.fsi_set_tc_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.fsi_apply_smoother.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.fsi_restrict.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.fsi_prolong.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.fsi_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.fsi_kernel_stats.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), i64p,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.fsi_server_create.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(vp)]
    lib.fsi_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.fsi_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result), vp]
    lib.fsi_serve_drain.argtypes = [vp]
    lib.fsi_server_resident_bytes.argtypes = [vp]
    lib.fsi_server_resident_bytes.restype = ctypes.c_int64
    lib.fsi_server_destroy.argtypes = [vp]
    lib.fsi_launch_count.argtypes = [vp]
    lib.fsi_launch_count.restype = ctypes.c_int64
    lib.fsi_set_launch_params.argtypes = [vp, ctypes.c_int, ctypes.POINTER(LaunchParams)]
    lib.fsi_get_launch_params.argtypes = [vp, ctypes.c_int, ctypes.POINTER(LaunchParams)]
    lib.fsi_time_level_kernels.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]
    _lib = lib
    return lib


def make_desc(p: Problem) -> ProblemDesc:
    d = ProblemDesc()
    d.dim = p.dim
    d.levels = p.levels
    for a in range(p.dim):
        br = p.breaks[a]
        if len(br) > MAX_BREAKS:
            raise ValueError("too many coarse breaks")
        d.n_breaks[a] = len(br)
        for i, v in enumerate(br):
            d.breaks[a][i] = float(v)
        d.flap_lo[a] = p.flap_lo[a]
        d.flap_hi[a] = p.flap_hi[a]
    d.rho_f, d.mu_f, d.rho_s, d.mu_s, d.U = p.rho_f, p.mu_f, p.rho_s, p.mu_s, p.U
    d.transient, d.dt, d.ale_op = p.transient, p.dt, p.ale_op
    d.mr_c2 = p.mr_c2
    return d


def make_opts(o: SolverOpts) -> SolverOptsC:
    c = SolverOptsC()
    for a, t in enumerate(o.tile):
        c.tile[a] = t
    c.n_pre, c.n_post, c.omega = o.n_pre, o.n_post, o.omega
    c.restart, c.rtol, c.max_iters, c.precision = o.restart, o.rtol, o.max_iters, o.precision
    c.krylov, c.gs_passes, c.local_solver = o.krylov, o.gs_passes, o.local_solver
    return c


def _ptr(a) -> Optional[int]:
    """Raw address of a torch tensor (device or host) or numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


class FSIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class FSI:
    """One Newton-step solver instance (owns an ``fsi_ctx``)."""

    def __init__(self, prob: Problem, opts: SolverOpts, stream: Optional[int] = None, plan_only: bool = False,
                 tuned: bool = True):
        """Builds the instance on the current CUDA device (``plan_only``:
        host structures only, no GPU needed).  ``tuned``: apply the launch
        shapes of the autotuner's table for this GPU and problem, if it has
        an entry (``autotune.py``); otherwise the library's built-in choice."""
        self.lib = load_library()
        self.prob, self.opts = prob, opts
        self._desc, self._opts = make_desc(prob), make_opts(opts)
        h = ctypes.c_void_p()
        if plan_only:
            rc = self.lib.fsi_plan_hierarchy(ctypes.byref(self._desc), ctypes.byref(self._opts), ctypes.byref(h))
        else:
            rc = self.lib.fsi_build_hierarchy(ctypes.byref(self._desc), ctypes.byref(self._opts),
                                              ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if rc != FSI_OK:
            raise FSIError(rc, "fsi_build_hierarchy failed (see stderr)")
        self.h = h
        L = prob.levels
        self.N = np.zeros(L, dtype=np.int64)
        self.nnz = np.zeros(L, dtype=np.int64)
        hb = ctypes.c_int64()
        self._check(self.lib.fsi_get_sizes(self.h, self.N.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           self.nnz.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           ctypes.byref(hb)))
        self.hbm_bytes = hb.value
        self.tuning = None
        if tuned and not plan_only:
            from . import autotune
            self.tuning = autotune.apply_table(self)

    def _check(self, rc):
        if rc != FSI_OK:
            msg = self.lib.fsi_last_error(self.h).decode()
            raise FSIError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fsi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- hot path ---------------------------------------------------------
    def initial_state(self, noise, y_out):
        self._check(self.lib.fsi_initial_state(self.h, _ptr(noise), _ptr(y_out)))

    def set_state(self, y, y_prev=None, y_prev2=None, t: float = 0.0):
        """Newton state; transient problems also take the previous time
        step(s) (BDF2 with y_prev2, BDF1 without) and the new time t."""
        self._check(self.lib.fsi_set_state(self.h, _ptr(y), _ptr(y_prev), _ptr(y_prev2), float(t)))

    def get_state(self, y_out):
        self._check(self.lib.fsi_get_state(self.h, _ptr(y_out)))

    def assemble(self, residual_out=None):
        self._check(self.lib.fsi_assemble_jacobian(self.h, _ptr(residual_out)))

    def factor(self):
        self._check(self.lib.fsi_factor_schwarz(self.h))

    def solve(self, b, x) -> SolveStats:
        """FGMRES solve; on FSI_E_NOT_CONVERGED the raised FSIError carries
        the filled statistics as ``.stats``."""
        st = SolveStats()
        rc = self.lib.fsi_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(st))
        if rc != FSI_OK:
            err = FSIError(rc, self.lib.fsi_last_error(self.h).decode())
            err.stats = st
            raise err
        return st

    def newton_update(self, dx) -> float:
        rel = ctypes.c_double()
        self._check(self.lib.fsi_newton_update(self.h, _ptr(dx), ctypes.byref(rel)))
        return rel.value

    def newton_step(self, dx_out=None):
        rel = ctypes.c_double()
        st = SolveStats()
        self._check(self.lib.fsi_newton_step(self.h, _ptr(dx_out), ctypes.byref(rel), ctypes.byref(st)))
        return rel.value, st

    # -- parity / diagnostics --------------------------------------------
    def export_csr(self, level: int, values: bool = True):
        """J_level as scipy CSR (values = False: pattern only, zero data)."""
        import scipy.sparse as sp
        n = int(self.N[level])
        nnz = int(self.nnz[level])
        rowptr = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz, dtype=np.float64)
        self._check(self.lib.fsi_export_csr(self.h, level, _ptr(rowptr), _ptr(col),
                                            _ptr(val) if values else None))
        return rowptr, col, val

    def export_transfer(self, level: int, which: int):
        """(rowptr, col, val) of P (which=0) or R (which=1) between level and level-1."""
        nnz = ctypes.c_int64()
        self._check(self.lib.fsi_export_transfer(self.h, level, which, ctypes.byref(nnz), None, None, None))
        rows = int(self.N[level] if which == 0 else self.N[level - 1])
        rowptr = np.zeros(rows + 1, dtype=np.int64)
        col = np.zeros(nnz.value, dtype=np.int32)
        val = np.zeros(nnz.value, dtype=np.float64)
        self._check(self.lib.fsi_export_transfer(self.h, level, which, None, _ptr(rowptr), _ptr(col), _ptr(val)))
        return rowptr, col, val

    def export_dofmap(self, level: int, n_nodes: int, n_elem: int):
        n = int(self.N[level])
        nc = np.zeros(n_nodes, dtype=np.uint8)
        es = np.zeros(n_elem, dtype=np.uint8)
        dm = np.zeros(n, dtype=np.uint8)
        dv = np.zeros(n, dtype=np.float64)
        self._check(self.lib.fsi_export_dofmap(self.h, level, _ptr(nc), _ptr(es), _ptr(dm), _ptr(dv)))
        return nc, es, dm.astype(bool), dv

    def export_patches(self, level: int):
        npch = ctypes.c_int()
        tot = ctypes.c_int64()
        self._check(self.lib.fsi_export_patches(self.h, level, ctypes.byref(npch), ctypes.byref(tot),
                                                None, None, None))
        ptr = np.zeros(npch.value + 1, dtype=np.int64)
        dofs = np.zeros(tot.value, dtype=np.int32)
        owned = np.zeros(tot.value, dtype=np.uint8)
        self._check(self.lib.fsi_export_patches(self.h, level, None, None, _ptr(ptr), _ptr(dofs), _ptr(owned)))
        return [(dofs[ptr[k]:ptr[k + 1]], owned[ptr[k]:ptr[k + 1]].astype(bool)) for k in range(npch.value)]

    def apply_operator(self, level, x, y):
        self._check(self.lib.fsi_apply_operator(self.h, level, _ptr(x), _ptr(y)))

    def apply_vcycle(self, b, z):
        self._check(self.lib.fsi_apply_vcycle(self.h, _ptr(b), _ptr(z)))

    def newton_solve_update(self, dx_out=None):
        """Solve and update with the current factors (fsi_newton_solve_update)."""
        rel = ctypes.c_double()
        st = SolveStats()
        self._check(self.lib.fsi_newton_solve_update(self.h, _ptr(dx_out), ctypes.byref(rel), ctypes.byref(st)))
        return rel.value, st

    def import_csr(self, level: int, val):
        """Replaces J_level's values (canonical CSR order of export_csr)."""
        val = np.ascontiguousarray(val, dtype=np.float64)
        assert val.shape == (int(self.nnz[level]),)
        self._check(self.lib.fsi_import_csr(self.h, level, _ptr(val)))

    def set_tc_wait_limit(self, iters: int):
        """First tensor-core wait limit of the Schwarz factorisation (< 0: built-in)."""
        self._check(self.lib.fsi_set_tc_wait_limit(self.h, int(iters)))

    def set_stream(self, stream: int):
        """Rebinds the instance to another CUDA stream (raw cudaStream_t)."""
        self._check(self.lib.fsi_set_stream(self.h, ctypes.c_void_p(stream)))

    def coarse_solve_static(self, b, x):
        """x = J_0^{-1} b with the coarse solve's scratch in a fixed
        file-scope device array (the call allocates nothing)."""
        self._check(self.lib.fsi_coarse_solve_static(self.h, _ptr(b), _ptr(x)))

    def apply_smoother(self, level, b, x, x_out):
        self._check(self.lib.fsi_apply_smoother(self.h, level, _ptr(b), _ptr(x), _ptr(x_out)))

    def restrict(self, level, fine, coarse):
        self._check(self.lib.fsi_restrict(self.h, level, _ptr(fine), _ptr(coarse)))

    def prolong(self, level, coarse, fine):
        self._check(self.lib.fsi_prolong(self.h, level, _ptr(coarse), _ptr(fine)))

    def set_profiling(self, on: bool):
        self._check(self.lib.fsi_set_profiling(self.h, 1 if on else 0))

    def kernel_stats(self):
        """{class: dict(ms, launches, bytes, flops)} accumulated since set_profiling(True)."""
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            ms, b, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            n = ctypes.c_int64()
            self._check(self.lib.fsi_kernel_stats(self.h, k, ctypes.byref(ms), ctypes.byref(n),
                                                  ctypes.byref(b), ctypes.byref(f)))
            out[name] = dict(ms=ms.value, launches=n.value, bytes=b.value, flops=f.value)
        return out

    def launch_count(self) -> int:
        return int(self.lib.fsi_launch_count(self.h))

    def set_launch_params(self, level: int, apply_slices: int = 0, apply_groups: int = 0, spmv_sub: int = 0,
                          gj_panel: int = 0):
        p = LaunchParams(apply_slices, apply_groups, spmv_sub, gj_panel)
        self._check(self.lib.fsi_set_launch_params(self.h, level, ctypes.byref(p)))

    def get_launch_params(self, level: int) -> dict:
        p = LaunchParams()
        self._check(self.lib.fsi_get_launch_params(self.h, level, ctypes.byref(p)))
        return dict(apply_slices=p.apply_slices, apply_groups=p.apply_groups, spmv_sub=p.spmv_sub,
                    gj_panel=p.gj_panel)

    def time_level_kernels(self, level: int, reps: int):
        """(apply_ms, spmv_ms): device time of one launch of the level's
        Schwarz apply and residual product (fsi_time_level_kernels)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.fsi_time_level_kernels(self.h, level, reps, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value


def factor_batch(instances) -> None:
    """fsi_factor_schwarz_batch over FSI instances bound to one stream."""
    lib = load_library()
    arr = (ctypes.c_void_p * len(instances))(*[s.h.value if hasattr(s.h, "value") else s.h for s in instances])
    rc = lib.fsi_factor_schwarz_batch(arr, len(instances))
    if rc != FSI_OK:
        raise FSIError(rc, lib.fsi_last_error(instances[0].h).decode())


def fmg_newton(prob: Problem, opts: SolverOpts, y_out, stream: Optional[int] = None, tol: float = 1e-8,
               max_steps: int = 20) -> dict:
    """Nested-iteration (full multigrid) Newton for the steady problem
    (fsi_fmg_newton); y_out receives the finest state.  Raises FSIError
    (with .stats) on failure."""
    lib = load_library()
    d, o, st = make_desc(prob), make_opts(opts), FmgStats()
    rc = lib.fsi_fmg_newton(ctypes.byref(d), ctypes.byref(o), ctypes.c_void_p(stream or 0), float(tol),
                            int(max_steps), _ptr(y_out), ctypes.byref(st))
    if rc != FSI_OK:
        err = FSIError(rc, "fsi_fmg_newton failed (see stderr)")
        err.stats = st.as_dict()
        raise err
    return st.as_dict()


class Server:
    """Continuous-batching server of Newton-step requests (fsi_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 0, max_slots: int = 4):
        self.lib = load_library()
        h = ctypes.c_void_p()
        rc = self.lib.fsi_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h))
        if rc != FSI_OK:
            raise FSIError(rc, "fsi_server_create failed")
        self.h = h

    def submit(self, instance: int, prob: Problem, opts: SolverOpts, noise=None, last: bool = False,
               keep_dx: bool = False) -> int:
        r = Request()
        r.instance = instance
        r.desc = make_desc(prob)
        r.opts = make_opts(opts)
        if noise is not None:
            noise = np.ascontiguousarray(noise, dtype=np.float64)
            r.noise = noise.ctypes.data
        r.last = 1 if last else 0
        r.keep_dx = 1 if keep_dx else 0
        t = ctypes.c_uint64()
        rc = self.lib.fsi_serve_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if rc != FSI_OK:
            raise FSIError(rc, "fsi_serve_submit rejected the request")
        return t.value

    def poll(self, ticket: int, dx_out=None):
        """None while pending, else the result dict (dx written to dx_out)."""
        res = Result()
        rc = self.lib.fsi_serve_poll(self.h, ticket, ctypes.byref(res), _ptr(dx_out))
        if rc == 1:
            return None
        if rc != FSI_OK:
            raise FSIError(rc, "fsi_serve_poll failed")
        return res.as_dict()

    def set_batching(self, max_batch: int):
        """Requests of up to max_batch resident mixed-precision instances share
        one Schwarz factorisation launch (1: off)."""
        rc = self.lib.fsi_server_set_batching(self.h, int(max_batch))
        if rc != FSI_OK:
            raise FSIError(rc, "fsi_server_set_batching rejected the value")

    def cancel(self, ticket: int) -> bool:
        """Cancels a request that has not started (True); False if it is
        already running or done."""
        rc = self.lib.fsi_serve_cancel(self.h, ctypes.c_uint64(ticket))
        if rc == 1:
            return False
        self._check(rc)
        return True

    def set_eviction(self, on: bool):
        """Evict idle steady instances to the host when the oldest waiting
        request does not fit in the budget (on by default)."""
        self._check(self.lib.fsi_server_set_eviction(self.h, 1 if on else 0))

    def evictions(self) -> int:
        return int(self.lib.fsi_server_evictions(self.h))

    def _check(self, rc):
        if rc != FSI_OK:
            raise FSIError(rc, "server call failed")

    def drain(self):
        self.lib.fsi_serve_drain(self.h)

    def resident_bytes(self) -> int:
        return int(self.lib.fsi_server_resident_bytes(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.fsi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
