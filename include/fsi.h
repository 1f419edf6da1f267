/*
 * libfsi - GB300-native Newton-step solver for monolithic ALE fluid-structure
 * interaction (Aulisa, Bna, Bornia, arXiv 1709.05660).
 *
 * The library computes, for one Newton step of the steady Q2-P1disc FSI
 * problem, the exact Jacobian J = dr/dy of the discrete residual (Sec. 2.3,
 * 2.5, 3), the Galerkin coarse operators of the geometric multigrid hierarchy
 * (Sec. 3.2), the restricted additive Schwarz subdomain inverses of the
 * Richardson smoother (Sec. 3.3), the coarse direct solve, and the
 * right-preconditioned FGMRES solve of J dy = -r (Sec. 3, 4.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status: every call returns an int, FSI_OK (0) or a negative FSI_E_* code;
 *   fsi_last_error(ctx) gives a message for the last failure on that ctx.
 * - Vectors of unknowns use the canonical numbering of length N (finest level
 *   unless a level is given): Q2 nodes lexicographic (x fastest), node
 *   unknown = node*2n + c with c in [d_0..d_{n-1}, u_0..u_{n-1}], then the
 *   P1disc pressures, element-lexicographic, n+1 per element
 *   ({1, xi, eta(, zeta)} in reference coordinates).
 * - Vector arguments may be device pointers (e.g. torch.Tensor.data_ptr()) or
 *   ordinary host pointers; the library detects which with
 *   cudaPointerGetAttributes and stages host data through its own buffers.
 *   The caller owns every buffer it passes; the ctx owns everything else.
 * - All device work of a ctx is ordered on the cudaStream_t given at build
 *   time.  fsi_factor_schwarz forks the coarse factorisation onto a private
 *   stream of the ctx (highest priority) and makes the given stream wait for
 *   it before the call's own final work, so to the caller it is one stream.
 *   Calls return after that work has completed (they synchronise the stream
 *   whenever a host-side decision or a host output needs it).
 * - Calls on one ctx are not thread safe; distinct ctxs are independent.
 * - There is no CPU fallback: without a usable CUDA device every call that
 *   needs one returns FSI_E_CUDA.
 */
#ifndef FSI_H_
#define FSI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FSI_OK = 0,
  FSI_E_INVALID = -1,       /* bad argument or descriptor */
  FSI_E_OOM = -2,           /* device allocation failed */
  FSI_E_CUDA = -3,          /* CUDA runtime error (no device, launch failure) */
  FSI_E_SINGULAR = -4,      /* zero / non-finite pivot in a patch or coarse LU */
  FSI_E_NOT_CONVERGED = -5, /* FGMRES hit max_iters; stats still filled */
  FSI_E_NONFINITE = -6,     /* NaN / Inf in the state, residual or Krylov data */
  FSI_E_MESH_TANGLED = -7,  /* det F <= 0 at a quadrature point */
  FSI_E_TIMEOUT = -8,       /* a bounded device wait gave up */
  FSI_E_CANCELLED = -9,     /* serving: the request was cancelled before it ran */
  FSI_PENDING = 1           /* serving poll: not finished yet */
};

enum { FSI_FP64 = 0, FSI_MIXED = 1 };
enum { FSI_MAX_BREAKS = 65 };

/* Problem descriptor (Sec. 2, 4).  The solid is incompressible Neo-Hookean, or
 * Mooney-Rivlin when mr_c2 != 0 (Sec. 2.2); mu_s = 2 (C1 + C2) is the shear
 * modulus of the linearised law.  The coarse tensor grid is given by its
 * cell boundaries per axis; every finer level is one midpoint refinement
 * (Sec. 3.2).  Elements whose centroid lies inside [flap_lo, flap_hi] are
 * solid, the rest fluid.  Boundary conditions: d = 0 on the whole outer
 * boundary; u = inflow profile on x = 0 (1.5 U y(H-y)/(H/2)^2 in 2D, the
 * product parabola 36 U y(H-y) z(H-z)/H^4 in 3D), u = 0 on the other walls,
 * stress-free outflow at x = x_max. */
typedef struct {
  int dim;                              /* 2 or 3 */
  int levels;                           /* total levels incl. the coarse one (>= 1) */
  int n_breaks[3];                      /* number of cell boundaries per axis */
  double breaks[3][FSI_MAX_BREAKS];     /* coarse cell boundaries, ascending */
  double flap_lo[3], flap_hi[3];        /* solid box */
  double rho_f, mu_f, rho_s, mu_s;      /* densities, viscosity, shear modulus (C1 = mu_s/2) */
  double U;                             /* mean inflow velocity */
  int transient;                        /* 0: steady; 1: time step of the BDF form; 2: time step of the
                                           paper's Crank-Nicolson form (Sec. 2.5) */
  double dt;                            /* time step (transient only, > 0) */
  int ale_op;                           /* 0: k(grad d + grad d^T), k = 1/V_el; 1: k grad d */
  double mr_c2;                         /* Mooney-Rivlin C2 (Sec. 2.2): sigma = -p I + 2 C1 B - 2 C2 B^{-1}
                                           with C1 = mu_s/2 - C2; 0 = Neo-Hookean */
} fsi_problem_desc;

/* Solver options (Sec. 3.3, 4.1). */
typedef struct {
  int tile[3];         /* Schwarz block = aligned tile of elements per axis */
  int n_pre, n_post;   /* Richardson smoothing steps before / after the coarse correction */
  double omega;        /* Richardson damping */
  int restart;         /* Krylov restart length (<= 64) */
  double rtol;         /* krylov 0: stop when ||b - J x|| <= rtol ||b|| (true residual);
                          krylov 1: when ||P^{-1}(b - J x)|| < rtol ||P^{-1}(b - J x0)|| */
  int max_iters;       /* total Krylov iterations */
  int precision;       /* FSI_FP64, or FSI_MIXED: FP32 V-cycle and Schwarz inverses, FP64 elsewhere */
  int krylov;          /* FSI_FGMRES (0): right-preconditioned flexible GMRES, true-residual test;
                          FSI_GMRES_LEFT (1): left-preconditioned GMRES, the paper's setting (Sec. 4.1) */
  int gs_passes;       /* classical Gram-Schmidt passes per Arnoldi step: 1 or 2 (0: 2 for FGMRES,
                          1 for left GMRES, the paper's unmodified classical Gram-Schmidt) */
  int local_solver;    /* Schwarz blocks (Sec. 3.3, 4.1): 0 = exact LU of every block; 1 = ILU(0) of
                          the fluid blocks (pattern: their node / element block pairs and the diagonal;
                          blocks of at most 1024 unknowns) and exact LU of the solid ones; mixed
                          precision only */
} fsi_solver_opts;
enum { FSI_FGMRES = 0, FSI_GMRES_LEFT = 1 };

typedef struct {
  int iters;             /* FGMRES iterations (Arnoldi steps) */
  int restarts;          /* completed restart cycles */
  double rel_res;        /* final true ||b - J x|| / ||b|| */
  double rho;            /* average convergence rate (rel_res)^(1/iters) (Sec. 4.2) */
  double t_assemble_ms, t_factor_ms, t_solve_ms;  /* device time of the last calls */
  double prec_rel_res;   /* left GMRES: final ||P^{-1} r|| / ||P^{-1} r_0|| (the stopping test);
                            FGMRES: equal to rel_res */
  double bytes_assemble, bytes_factor, bytes_solve;   /* algorithmic bytes of the last calls: matrix,
                            index and vector entries their kernels must move at least once */
} fsi_solve_stats;

typedef struct fsi_ctx fsi_ctx;

/* Builds the mesh hierarchy, unknown numbering, block-sparse patterns, grid
 * transfers, Schwarz blocks and all device workspaces (Sec. 2.5, 3.2, 3.3).
 * `stream` is a cudaStream_t (NULL = legacy default stream).  On success
 * *out owns all device memory of the instance; free it with fsi_destroy.
 * Errors: FSI_E_INVALID (bad descriptor or options), FSI_E_OOM, FSI_E_CUDA. */
int fsi_build_hierarchy(const fsi_problem_desc* desc, const fsi_solver_opts* opts,
                        void* stream, fsi_ctx** out);
/* Host-only variant: builds the same hierarchy, numbering, patterns,
 * transfers and Schwarz blocks on the host without touching any GPU.  The
 * resulting ctx answers fsi_get_sizes and the structural exports
 * (fsi_export_csr with val = NULL, fsi_export_dofmap, fsi_export_patches,
 * fsi_export_transfer); compute calls on it return FSI_E_INVALID.  Used to
 * size an instance before admitting it, and to check the numbering without
 * a device. */
int fsi_plan_hierarchy(const fsi_problem_desc* desc, const fsi_solver_opts* opts, fsi_ctx** out);
/* Waits for the ctx's stream and frees everything the ctx owns (the device
 * data of the hierarchy of Sec. 3.2 and the factors of Sec. 3.3).  NULL is a
 * no-op. */
void fsi_destroy(fsi_ctx* ctx);
/* Message of the last failed call on ctx (owned by ctx, valid until its next
 * call). */
const char* fsi_last_error(const fsi_ctx* ctx);
/* Rebinds the ctx to another cudaStream_t of the same device: waits for the
 * old stream, then orders all later work of the ctx on `stream`.  Lets a
 * caller run consecutive Newton steps of one instance on whichever of its
 * streams is free (the serving loop does).  No counterpart in the paper. */
int fsi_set_stream(fsi_ctx* ctx, void* stream);

/* Sizes: N (canonical unknowns) and scalar nnz of J per level (arrays of
 * `levels` entries, level 0 = coarse) and the device bytes held by ctx (for a
 * planned ctx: the bytes fsi_build_hierarchy would allocate).  The counts are
 * those of the Q2-P1disc spaces of Sec. 2.5 on each mesh of Sec. 3.2 (the
 * unknown counts of the table in Sec. 4); any pointer may be NULL. */
int fsi_get_sizes(const fsi_ctx* ctx, int64_t* n_per_level, int64_t* nnz_per_level,
                  int64_t* hbm_bytes);

/* Benchmark linearisation state: d = 0, p = 0, u_x = inflow profile at every
 * fluid node whose u_x is free (0 at solid and interface nodes), Dirichlet
 * values at Dirichlet unknowns, then noise[i] added at every free
 * displacement unknown.  noise and y_out: N doubles (host or device; a
 * planned ctx takes host buffers).  With zero noise this is the
 * boundary-condition lift that starts a nonlinear solve. */
int fsi_initial_state(fsi_ctx* ctx, const double* noise, double* y_out);

/* Sets the Newton state y (N doubles).  Steady problems ignore y_prev,
 * y_prev2 and t.  Transient problems need the state of the previous time
 * step y_prev.  BDF form (desc.transient = 1): with y_prev2 (the one before)
 * the time derivative is BDF2, q_t = (1.5 q - 2 q_n + 0.5 q_{n-1}) / dt,
 * without it BDF1, q_t = (q - q_n) / dt (start-up step).  Crank-Nicolson form
 * (desc.transient = 2, Sec. 2.5): y_prev is the state of t_n, y_prev2 is
 * ignored; the fluid momentum uses the conservative ALE identity of Sec. 2.3
 * ((rho J u)_{n+1} - (rho J u)_n over dt with the -(div w) u terms), the
 * stresses, the convection and the solid kinematic velocity are averaged
 * over t_{n+1} and t_n, with the mesh velocity w = (d - d_n) / dt.  t is the
 * new time level: the inflow data are scaled by alpha(t) = (1 + sin 2 pi t)
 * / 2, so Dirichlet residual rows read r_i = y_i - alpha(t) g_i.  Host or
 * device buffers. */
int fsi_set_state(fsi_ctx* ctx, const double* y, const double* y_prev,
                  const double* y_prev2, double t);
int fsi_get_state(fsi_ctx* ctx, double* y_out);

/* Residual r(y) and exact Jacobian J(y) on the finest level (element-batched
 * forward-mode dual numbers, element contributions gathered into block-sparse storage),
 * Dirichlet rows replaced by identity rows with r_i = y_i - g_i, then the
 * Galerkin operators J_{l-1} = R J_l P of every coarser level (Sec. 3.2).
 * Transient problems add the BDF inertia terms, the mesh velocity in the
 * fluid convection and the BDF velocity in the solid kinematic rows, with
 * the history given to fsi_set_state (FSI_E_INVALID before the first one).
 * residual_out (N doubles) may be NULL.  Returns FSI_E_MESH_TANGLED if
 * det F <= 0 at a quadrature point and FSI_E_NONFINITE on NaN / Inf. */
int fsi_assemble_jacobian(fsi_ctx* ctx, double* residual_out);

/* Factors every Schwarz block B_k = J_l[R^delta_k, R^delta_k] of the levels
 * l >= 1 (partial-pivot Gauss-Jordan; only the owned rows of B_k^{-1} are
 * kept, as the restricted Schwarz update uses nothing else) and the coarse
 * operator J_0 (Sec. 3.3), the two concurrently (they are independent; the
 * coarse part on the ctx's private stream).  FSI_E_SINGULAR on a zero pivot. */
int fsi_factor_schwarz(fsi_ctx* ctx);

/* Krylov solve of J x = b with the multigrid V-cycle P as preconditioner
 * (Sec. 3, 4.1): right-preconditioned FGMRES(restart) with a true-residual
 * test, or (opts.krylov = FSI_GMRES_LEFT) the paper's left-preconditioned
 * GMRES(restart) with its test on the left-preconditioned residual.  x holds
 * the initial guess on entry and the solution on exit (N doubles each).
 * stats may be NULL; on FSI_E_NOT_CONVERGED they are filled and x holds the
 * last iterate. */
int fsi_solve(fsi_ctx* ctx, const double* b, double* x, fsi_solve_stats* stats);

/* Newton update y += dx (Sec. 3.1, 4.1); *rel_step_out = ||dx|| / ||y_new||. */
int fsi_newton_update(fsi_ctx* ctx, const double* dx, double* rel_step_out);

/* One whole Newton step at the current state: assemble, factor, solve
 * J dx = -r, update.  dx_out (N doubles, may be NULL) receives dx. */
int fsi_newton_step(fsi_ctx* ctx, double* dx_out, double* rel_step_out, fsi_solve_stats* stats);
/* The second half of fsi_newton_step: solve J dx = -r with the current
 * factors and the residual of the last fsi_assemble_jacobian, then y += dx
 * (Sec. 3.1).  For callers that factor several instances together
 * (fsi_factor_schwarz_batch).  FSI_E_INVALID before the first factorisation. */
int fsi_newton_solve_update(fsi_ctx* ctx, double* dx_out, double* rel_step_out, fsi_solve_stats* stats);

/* fsi_factor_schwarz for n mixed-precision instances at once (no
 * counterpart in the paper; the batched form of Sec. 3.3 for serving): the
 * Schwarz blocks of all their levels >= 1 are factored by one tensor-core
 * launch per kernel variant (instances whose largest blocks call for the
 * same panel width share a launch), and each instance's coarse LU runs on
 * its private stream beside it.  Every block is factored exactly as by the
 * instance's own fsi_factor_schwarz, so the results are bit-identical.  All
 * instances must be bound to the same stream (fsi_set_stream) and device and
 * have >= 2 levels; FSI_E_INVALID otherwise.  Errors of the factorisation
 * (FSI_E_SINGULAR, FSI_E_TIMEOUT) are reported for the first instance
 * affected. */
int fsi_factor_schwarz_batch(fsi_ctx* const* ctxs, int n);

/* ---- nested iteration (full multigrid) for the steady problem ---------- */

enum { FSI_FMG_MAX_LEVELS = 16 };
typedef struct {
  int levels;                                  /* mesh levels solved (= desc.levels) */
  int newton_steps[FSI_FMG_MAX_LEVELS];        /* Newton steps on mesh level l (0 = coarsest) */
  int krylov_iters[FSI_FMG_MAX_LEVELS];        /* Krylov iterations summed over those steps */
  double last_rel_step[FSI_FMG_MAX_LEVELS];    /* ||dy|| / ||y|| of the level's last step */
  double ms[FSI_FMG_MAX_LEVELS];               /* device time of the level's steps (assemble + factor + solve) */
  int status;                                  /* FSI_OK or the first error */
} fsi_fmg_stats;

/* Steady nonlinear problem by nested iteration, the full-multigrid driver of
 * Sec. 3: Newton (each step an fsi_newton_step: exact Jacobian, Galerkin
 * hierarchy, Schwarz and coarse factors, Krylov solve) to ||dy|| < tol ||y||
 * on the coarsest mesh from the boundary-condition lift (the state of
 * fsi_initial_state without noise), then on every finer mesh up to
 * desc->levels from the coarser solution carried over by the natural
 * injection of the nested spaces (Sec. 3.2; every unknown including its
 * boundary values, then the fine Dirichlet data).  Mesh level l is solved
 * with its own multigrid hierarchy of levels 0..l, built and freed in turn.
 * y_out receives the finest state (N doubles, host or device).  Steady
 * problems only (FSI_E_INVALID otherwise); FSI_E_NOT_CONVERGED when a level
 * needs more than max_steps steps; stats may be NULL. */
int fsi_fmg_newton(const fsi_problem_desc* desc, const fsi_solver_opts* opts, void* stream, double tol,
                   int max_steps, double* y_out, fsi_fmg_stats* stats);

/* ---- parity / diagnostics ------------------------------------------- */

/* J_level in canonical CSR (host buffers): rowptr[N+1], col[nnz], val[nnz];
 * columns ascending; the pattern is the full FE graph (explicit zeros kept),
 * i.e. the block structure of the Jacobian of Sec. 3.1.  col or val may be
 * NULL (pattern or values only; a planned ctx has no values). */
int fsi_export_csr(fsi_ctx* ctx, int level, int64_t* rowptr, int32_t* col, double* val);
/* Unknown classification of Sec. 3.1: node_class[n_nodes] (0 fluid, 1 solid,
 * 2 interface), elem_solid[n_elem], dirichlet[N] (0/1) and dir_val[N] (the
 * boundary data of Sec. 4); any pointer may be NULL; host buffers. */
int fsi_export_dofmap(fsi_ctx* ctx, int level, uint8_t* node_class, uint8_t* elem_solid,
                      uint8_t* dirichlet, double* dir_val);
/* Schwarz blocks of Sec. 3.3 on a level >= 1: the overlapping sets R^delta_k
 * and the owned sets R^0_k.  n_patches (may be NULL); ptr[n_patches+1]
 * offsets into dofs / owned; dofs ascending canonical unknowns (R^delta_k);
 * owned[i] = 1 if dofs[i] is in R^0_k.  Pass ptr = NULL to query the total
 * length through *total_len. */
int fsi_export_patches(fsi_ctx* ctx, int level, int* n_patches, int64_t* total_len,
                       int64_t* ptr, int32_t* dofs, uint8_t* owned);
/* Grid transfer matrices of Sec. 3.2 (natural injection P and the
 * interface-aware restriction R) between level and level-1 in canonical CSR
 * (host buffers): which = 0 prolongation P (N_level rows), which = 1 restriction R
 * (N_{level-1} rows); rowptr[rows+1], col[nnz], val[nnz], columns ascending.
 * Pass col = NULL to query *nnz only. */
int fsi_export_transfer(fsi_ctx* ctx, int level, int which, int64_t* nnz, int64_t* rowptr, int32_t* col,
                        double* val);
/* Replaces the values of J_level (level's pattern, canonical CSR order of
 * fsi_export_csr; val: nnz host doubles) until the next
 * fsi_assemble_jacobian.  For tests of the later steps in isolation (Sec. 3.2,
 * 3.3 on a given operator) and for injecting a defective operator, e.g. a
 * zero column that makes a Schwarz block singular (FSI_E_SINGULAR from
 * fsi_factor_schwarz).  The values are copied; on a mixed-precision instance
 * the FP32 copy of a level >= 1 is refreshed too. */
int fsi_import_csr(fsi_ctx* ctx, int level, const double* val);
/* Iteration limit of the first bounded wait of each Schwarz-block
 * factorisation on its tensor-core work (mixed precision).  When it runs out
 * the block waits (with the full limit) for the work it has already issued,
 * releases its tensor memory and reports FSI_E_TIMEOUT from
 * fsi_factor_schwarz; the ctx stays usable.  iters < 0 restores the built-in
 * limit (2^22).  A diagnostic of the time-out path; no counterpart in the
 * paper. */
int fsi_set_tc_wait_limit(fsi_ctx* ctx, long long iters);
/* y = J_level x (level's canonical numbering). */
int fsi_apply_operator(fsi_ctx* ctx, int level, const double* x, double* y);
/* z = one V-cycle applied to b on the finest level (the preconditioner). */
int fsi_apply_vcycle(fsi_ctx* ctx, const double* b, double* z);
/* x_out = x + omega sum_k (R^0_k)^T B_k^{-1} R^delta_k (b - J_level x), one
 * Richardson-Schwarz step on a level >= 1 (Sec. 3.3). */
int fsi_apply_smoother(fsi_ctx* ctx, int level, const double* b, const double* x, double* x_out);
/* Grid transfers between level and level-1: restriction (fine -> coarse) and
 * prolongation (coarse -> fine), canonical numbering of each level. */
int fsi_restrict(fsi_ctx* ctx, int level, const double* fine, double* coarse);
int fsi_prolong(fsi_ctx* ctx, int level, const double* coarse, double* fine);
/* Number of kernel launches issued by this ctx since it was built. */
int64_t fsi_launch_count(const fsi_ctx* ctx);

/* ---- coarse solve without allocation (no counterpart in the paper) ---- */

/* Largest level-0 internal length (N_0 plus the zero padding of element
 * pressure blocks) the static variant accepts, and the size in doubles of
 * its file-scope scratch array: ceil(4096 / 32) * 4096 = 2^19 (4 MiB). */
enum { FSI_STATIC_COARSE_MAX = 4096, FSI_STATIC_PART_MAX = 1 << 19 };

/* x = J_0^{-1} b on level 0 (canonical numbering, FP64; host or device
 * buffers) with the dense coarse inverse of fsi_factor_schwarz: the same
 * kernels and summation order as the FP64 coarse step of fsi_apply_vcycle,
 * so on an FP64 (precision FSI_FP64) one-level instance the result equals
 * that of fsi_apply_vcycle bit for bit.  (A mixed-precision instance's
 * V-cycle rounds its coarse input and output to FP32; this call does not.)  The GEMV partial sums live in a file-scope device array of
 * FSI_STATIC_PART_MAX doubles instead of instance scratch, and the call
 * allocates no device or pinned memory.  It is meant for callers that cannot
 * allocate at call time: a serving worker whose instances were admitted
 * against a fixed device-memory budget byte for byte, and callers driving
 * several streams at once, for whom a cudaMalloc / cudaFree could
 * synchronise the device and stall the other streams.
 * Limits: FSI_E_INVALID when the level-0 internal length exceeds
 * FSI_STATIC_COARSE_MAX, for 3D instances (slab-blocked coarse LU), before
 * the first fsi_factor_schwarz, and when the calling thread's current
 * device is not the one the ctx was built on.
 * The array is shared by every instance on a device: calls that overlap in
 * time (two threads or two streams) race on it and must be serialised by the
 * caller.  The first call on a device resolves the array's address once
 * (cudaGetSymbolAddress); make that first call before any stream capture on
 * the device.  Nothing in the array has to start at zero. */
int fsi_coarse_solve_static(fsi_ctx* ctx, const double* b, double* x);

/* Per-kernel-class timing.  With profiling on, every launch of a class is
 * bracketed by CUDA events on the ctx stream, and its algorithmic traffic
 * (bytes the operation must move at least once: matrix, index and vector
 * entries it reads or writes) and arithmetic (flops of the operation's
 * definition) are accumulated.  fsi_set_profiling(ctx, 1) clears the
 * counters; fsi_kernel_stats synchronises the stream and reports totals. */
enum {
  FSI_K_ASSEMBLE = 0,      /* element residual + Jacobian (dual numbers) */
  FSI_K_GALERKIN = 1,      /* element-wise Galerkin coarse matrices */
  FSI_K_SCATTER = 2,       /* gather of element matrices into blocks, Dirichlet rows */
  FSI_K_PATCH_FACTOR = 3,  /* Schwarz block gather + Gauss-Jordan inversion */
  FSI_K_COARSE_FACTOR = 4, /* coarse dense gather + cooperative Gauss-Jordan */
  FSI_K_PATCH_APPLY = 5,   /* restricted Schwarz update (owned inverse rows x residual) */
  FSI_K_SPMV = 6,          /* block-sparse residual of the V-cycle (FP32 on the mixed path) */
  FSI_K_TRANSFER = 7,      /* restriction / prolongation / coarse apply */
  FSI_K_KRYLOV = 8,        /* dots, Gram-Schmidt updates, norms, combinations */
  FSI_K_OPERATOR = 9,      /* the Krylov method's FP64 product J v (FP64 pipe: 16 FMAs per 4 x 4 block) */
  FSI_K_COUNT = 10
};
int fsi_set_profiling(fsi_ctx* ctx, int on);
int fsi_kernel_stats(fsi_ctx* ctx, int kind, double* device_ms, int64_t* launches, double* alg_bytes,
                     double* alg_flops);

/* ---- launch parameters and their autotuner (no counterpart in the paper) --
 *
 * Launch shapes of one level's kernels.  They change how work is mapped to
 * threads, and with it the rounding order of sums, never what is computed.
 * A zero field keeps the built-in choice.
 *   apply_slices  Schwarz apply (the smoother's restricted update): 1 = one
 *                 thread block per Schwarz block; s >= 2 = the owned rows of
 *                 every block split over s thread blocks (capped at the
 *                 number of 4-row vectors).
 *   apply_groups  with row slices: column groups per thread block (1..256,
 *                 capped so a block has at most 256 threads).
 *   spmv_sub      threads per scalar row of the level's block-sparse residual
 *                 in the V-cycle (mixed path; B = 4 blocks): 2, 4 or 8.
 *   gj_panel      variant of the tensor-core Gauss-Jordan of the Schwarz
 *                 blocks: the panel width 16, 24 or 32 (one thread block per
 *                 SM), or 216: 16-column panels with half the tensor memory,
 *                 so that two thread blocks share an SM (blocks of at most 512
 *                 unknowns).  When the asked variant does not fit the largest
 *                 block, the widest that fits is taken.  One launch factors
 *                 every level, so only the value set on the finest level counts.
 * The values are a property of the ctx; setting them waits for the ctx's
 * stream and drops the recorded V-cycle graph, which is recorded again at the
 * next solve.  FSI_E_INVALID for a bad level or out-of-range values. */
typedef struct {
  int32_t apply_slices, apply_groups, spmv_sub, gj_panel;
} fsi_launch_params;
int fsi_set_launch_params(fsi_ctx* ctx, int level, const fsi_launch_params* params);
/* The shapes in effect on `level` (the built-in choice resolved). */
int fsi_get_launch_params(fsi_ctx* ctx, int level, fsi_launch_params* out);
/* Device time (CUDA events on the ctx stream) of one launch of the level's
 * Schwarz apply and of its block-sparse residual, averaged over `reps`
 * launches each, in the ctx's V-cycle precision and launch shapes.  Runs on
 * the level's own work vectors (set to zero first; their contents are lost).
 * Needs a prior fsi_factor_schwarz; FSI_E_INVALID otherwise or for reps
 * outside [1, 10000]. */
int fsi_time_level_kernels(fsi_ctx* ctx, int level, int reps, double* apply_ms, double* spmv_ms);

/* ---- serving: continuous batching of Newton-step requests ---------------
 *
 * No counterpart in the paper (its solver runs one problem at a time, Sec.
 * 4.1): a serving form of the Newton step of Sec. 3.1 for many independent
 * instances on one GPU.
 *
 * A server owns `max_slots` worker threads, each with its own CUDA stream, and
 * a device-memory budget.  A request asks for one Newton step (assemble,
 * Galerkin, factor, FGMRES solve, update) of an instance identified by the
 * caller.  The first request of an instance builds its hierarchy (admitted
 * only when the planned device bytes fit in the budget left; otherwise it
 * waits while other requests proceed); later requests reuse the resident
 * hierarchy, state and factors; the request flagged `last` frees them.
 * Requests of one instance run in submission order; requests of different
 * instances run concurrently on different streams as slots free up.  Results
 * do not depend on what else is running: every instance computes on its own
 * buffers with a fixed reduction order. */
typedef struct fsi_server fsi_server;

typedef struct {
  uint64_t instance;          /* caller-chosen instance id */
  fsi_problem_desc desc;      /* read when the instance is first seen */
  fsi_solver_opts opts;       /* read when the instance is first seen */
  const double* noise;        /* first request: N host doubles for fsi_initial_state (copied at submit) */
  int last;                   /* 1: free the instance after this step */
  int keep_dx;                /* 1: keep the Newton update for fsi_serve_poll */
} fsi_request;

typedef struct {
  int status;                 /* FSI_OK or the step's error code */
  int iters;                  /* FGMRES iterations */
  double rel_step;            /* ||dx|| / ||y|| */
  double rel_res;             /* true relative residual of the solve */
  double queue_ms;            /* submit -> start */
  double run_ms;              /* start -> end */
  double latency_ms;          /* submit -> end */
  int64_t n;                  /* number of unknowns of the instance */
} fsi_result;

/* hbm_budget_bytes: device bytes the server may hold for instances; 0 = no
 * limit.  max_slots: concurrent requests (1..64). */
int fsi_server_create(int64_t hbm_budget_bytes, int max_slots, fsi_server** out);
/* Queues a request; *ticket identifies it.  FSI_E_INVALID if the descriptor
 * of a new instance is invalid or its planned size exceeds the whole budget. */
int fsi_serve_submit(fsi_server* srv, const fsi_request* req, uint64_t* ticket);
/* FSI_PENDING while queued or running; otherwise fills *out (and dx_out, N
 * host doubles, when the request had keep_dx) and returns FSI_OK; the ticket
 * is then released. */
int fsi_serve_poll(fsi_server* srv, uint64_t ticket, fsi_result* out, double* dx_out);
/* Blocks until every queued request has finished (results stay pollable). */
int fsi_serve_drain(fsi_server* srv);
/* Cancels a request that has not started: it completes at once with status
 * FSI_E_CANCELLED (poll it as usual; no dx) and the instance's state does not
 * advance.  A cancelled first request hands its noise to the instance's next
 * queued request, which then builds the instance.  A cancelled `last` request
 * moves the end of the instance to its latest queued request, else to the end
 * of the step that runs now, else frees the instance at once.  Returns
 * FSI_PENDING if the request is already running or done (it is not
 * cancelled), FSI_E_INVALID for an unknown or already polled ticket. */
int fsi_serve_cancel(fsi_server* srv, uint64_t ticket);
/* Device bytes currently held by resident instances. */
int64_t fsi_server_resident_bytes(const fsi_server* srv);
/* Continuous batching of the factorisation: a worker that takes a request of
 * a resident mixed-precision instance (>= 2 levels) also takes the runnable
 * requests of up to max_batch - 1 other such instances; each assembles, the
 * Schwarz blocks of all of them are factored by fsi_factor_schwarz_batch
 * (one launch per kernel variant), then each solves and updates.  Results
 * are bit-identical to unbatched steps.  1 turns it off; the default is 4.
 * FSI_E_INVALID outside [1, 64]. */
int fsi_server_set_batching(fsi_server* srv, int max_batch);
/* Eviction under memory pressure (on by default): when the oldest waiting
 * request does not fit in the budget, idle steady instances without queued
 * requests are evicted, least recently used first - the Newton state y is
 * copied to the host (fsi_get_state) and the hierarchy freed - and an evicted
 * instance is rebuilt from its descriptor and saved state (fsi_set_state)
 * when its next request is admitted.  Results do not change: every step
 * re-assembles and re-factors from the state.  0 turns it off (a request that
 * does not fit then waits for instances to finish). */
int fsi_server_set_eviction(fsi_server* srv, int on);
/* Instances evicted so far. */
int64_t fsi_server_evictions(fsi_server* srv);
/* Waits for running requests, frees every instance and the server. */
int fsi_server_destroy(fsi_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* FSI_H_ */
