// Internal data structures of libfsi (host builder, kernels, C-ABI).
//
// Device layout ("internal" numbering): a level with Nn Q2 nodes and Ne
// elements has nb = Nn + Ne blocks of B = 2*dim unknowns.  Node block a holds
// [d_0..d_{n-1}, u_0..u_{n-1}] of node a (identical to the canonical
// numbering); element block Nn + e holds the n+1 pressures of element e and
// B-(n+1) padding slots that are always zero.  The Jacobian of every level is
// a block-sparse (BSR) matrix with B x B row-major blocks on the FE graph
// (node-node blocks for nodes sharing an element, node-pressure and
// pressure-node blocks inside an element; no pressure-pressure blocks).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fsi.h"

namespace fsi {

constexpr int kFluid = 0, kSolid = 1, kIface = 2;

struct HostLevel {
  int dim = 2;
  int cells[3] = {1, 1, 1};
  int nodes_ax[3] = {1, 1, 1};
  int64_t n_nodes = 0, n_elem = 0, N = 0, nb = 0, Ni = 0;
  int B = 4, nloc = 9, ndofe = 39;
  std::vector<double> verts[3];
  std::vector<int32_t> elem_nodes;     // n_elem * nloc
  std::vector<uint8_t> elem_solid;     // n_elem
  std::vector<uint8_t> node_class;     // n_nodes
  std::vector<uint8_t> dir;            // Ni (internal), 1 = Dirichlet unknown
  std::vector<double> dir_val;         // Ni
  std::vector<int32_t> canon_of_int;   // Ni -> canonical index or -1 (padding)
  // block-sparse pattern
  std::vector<int32_t> rowptr, col;    // nb+1, nnzb
  int64_t nnzb = 0;
  std::vector<int32_t> elem_map;       // n_elem * (nloc+1)^2 block index or -1
  std::vector<int32_t> color_list;     // elements ordered by (color, material)
  std::vector<int32_t> color_ptr;      // (2^dim * 2) + 1 offsets into color_list
  std::vector<int32_t> mat_list;       // elements: the fluid ones ascending, then the solid ones
  int64_t n_fluid_elem = 0;
  // element contributions of each matrix block (nnzb + 1 offsets; entries
  // e (nloc+1)^2 + a (nloc+1) + b for local block (a, b) of element e) and of
  // each block row of the residual (nb + 1 offsets; entries e (nloc+1) + a),
  // both in the order of color_list, so that summing them in list order adds
  // the element values in the order of a coloured scatter
  std::vector<int32_t> blk_ptr, blk_src, res_ptr, res_src;
  // grid transfers from level-1 into this level (scalar CSR, internal indices)
  std::vector<int32_t> P_ptr, P_col;   // Ni rows
  std::vector<double> P_val;
  std::vector<int32_t> R_ptr, R_col;   // Ni(l-1) rows
  std::vector<double> R_val;
  // unmasked natural injection of whole states (Dirichlet values included),
  // for nested iteration: Ni rows
  std::vector<int32_t> S_ptr, S_col;
  std::vector<double> S_val;
  // Schwarz blocks (levels >= 1)
  int n_patches = 0;
  std::vector<int32_t> p_n, p_nown;            // per patch sizes (padded) / owned rows
  std::vector<int64_t> p_idx_off;              // into p_idx (sum n_k)
  std::vector<int64_t> p_own_off;              // into p_own (sum nown_k)
  std::vector<int64_t> p_dense_off;            // into dense workspace (sum n_k^2)
  std::vector<int64_t> p_inv_off;              // into owned inverse rows (sum nown_k*n_k)
  std::vector<int64_t> p_gmap_off;             // into p_gmap triples
  std::vector<int32_t> p_idx;                  // internal unknown of each patch-local unknown (-1: pad)
  std::vector<int32_t> p_own;                  // patch-local row of each owned row
  std::vector<int32_t> p_gmap;                 // (bsr block, local block row, local block col)
  std::vector<int32_t> p_padpos;               // patch-local pad positions (identity diag), flat
  std::vector<int32_t> p_boff;                 // per local block: dense offset * 8 + width (B or dim + 1)
  std::vector<int64_t> p_boff_off;             // into p_boff
  // per local block row: first p_gmap entry of the row, relative to the
  // block's first entry, plus one end entry per block (at p_boff_off[p] + p);
  // a row's entries are in ascending local column order
  std::vector<int32_t> p_gptr;
  std::vector<int64_t> p_pad_off;
  std::vector<int32_t> p_elems;                // elements of each patch (for export)
  std::vector<int64_t> p_elem_off;
  int64_t dense_total = 0, inv_total = 0, idx_total = 0, own_total = 0;
  int max_n = 0, max_nown = 0;
  // coarse level: bandwidth-reducing ordering (internal unknown -> position)
  std::vector<int32_t> coarse_perm;
  int coarse_bw = 0;
  // slab partition of the banded ordering (block-tridiagonal coarse solve):
  // slab k = positions [slab_off[k], slab_off[k+1]); the coupling of slabs k-1
  // and k runs only through the last slab_p positions of slab k-1
  std::vector<int64_t> slab_off;
  int slab_p = 0;
};

bool build_host_hierarchy(const fsi_problem_desc& d, const fsi_solver_opts& o,
                          std::vector<HostLevel>& lv, std::string& err);

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
struct DevLevel {
  int64_t n_nodes = 0, n_elem = 0, N = 0, nb = 0, Ni = 0, nnzb = 0;
  int cells[3] = {1, 1, 1};
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;          // nnzb * B*B
  double* Ke = nullptr;           // n_elem * ndofe^2 element matrices
  int32_t* elem_nodes = nullptr;
  uint8_t* elem_solid = nullptr;
  uint8_t* node_class = nullptr;
  double* elem_geo = nullptr;     // n_elem * 2*dim (lower corner, edge lengths)
  uint8_t* dir = nullptr;
  double* dir_val = nullptr;
  int32_t* dir_list = nullptr;    // internal Dirichlet unknowns
  int64_t n_dir = 0;
  int32_t* canon_of_int = nullptr;
  int32_t* int_of_canon = nullptr;
  int32_t* mat_list = nullptr;
  int64_t n_fluid_elem = 0;
  int32_t *blk_ptr = nullptr, *blk_src = nullptr, *res_ptr = nullptr, *res_src = nullptr;
  int64_t n_blk_src = 0, n_contrib = 0;   // entries of blk_src; of blk_src and res_src
  int32_t *P_ptr = nullptr, *P_col = nullptr, *R_ptr = nullptr, *R_col = nullptr;
  double *P_val = nullptr, *R_val = nullptr;
  int32_t *S_ptr = nullptr, *S_col = nullptr;   // unmasked state injection from level - 1
  double* S_val = nullptr;
  // patches
  int n_patches = 0, max_n = 0, max_nown = 0;
  // local solvers (fsi_solver_opts.local_solver = 1): blocks with an exact
  // inverse (solid, or too large for ILU) and ILU(0) blocks (fluid)
  int32_t *sel_lu = nullptr, *sel_ilu = nullptr;
  int n_lu = 0, n_ilu = 0;
  int ilu_max_n = 0, ilu_max_nb = 0;   // largest ILU(0) block: unknowns, node / element blocks
  // launch parameters (0 = built-in choice; set by fsi_set_launch_params)
  int apply_slices = 0, apply_groups = 0, spmv_sub = 0;
  int32_t *p_n = nullptr, *p_nown = nullptr;
  int64_t *p_idx_off = nullptr, *p_own_off = nullptr, *p_dense_off = nullptr, *p_inv_off = nullptr,
          *p_gmap_off = nullptr, *p_pad_off = nullptr;
  int32_t *p_idx = nullptr, *p_own = nullptr, *p_gmap = nullptr, *p_padpos = nullptr, *p_boff = nullptr;
  int64_t* p_boff_off = nullptr;
  int32_t* p_gptr = nullptr;
  double* inv = nullptr;          // owned rows of B~_k^{-1} (equilibrated block)
  double *dr = nullptr, *dc = nullptr;     // row / column scales of each block (FP64 path)
  float *dr32 = nullptr, *dc32 = nullptr;  // (mixed path)
  int64_t inv_total = 0, dense_total = 0;
  // work vectors (internal layout)
  double *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
  // mixed-precision copies (FSI_MIXED): FP32 values, inverses, vectors
  float *val32 = nullptr, *inv32 = nullptr, *x32 = nullptr, *b32 = nullptr, *r32 = nullptr;
  float *P_val32 = nullptr, *R_val32 = nullptr;
  // algorithmic traffic / arithmetic of one launch (profiling)
  double apply_bytes32 = 0, spmv_bytes32 = 0, R_bytes32 = 0, P_bytes32 = 0;
  double apply_bytes = 0, apply_flops = 0, spmv_bytes = 0, spmv_flops = 0;
  double factor_bytes = 0, factor_flops = 0, R_bytes = 0, P_bytes = 0;
};

struct Ctx {
  fsi_problem_desc desc;
  fsi_solver_opts opts;
  cudaStream_t stream = nullptr;
  std::vector<HostLevel> hl;
  std::vector<DevLevel> dl;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t est_bytes = 0;                  // planned device bytes (before building)
  std::string err;
  int64_t launches = 0;
  int dim = 2, B = 4, nloc = 9, ndofe = 39;
  int sm_count = 0;
  int device = -1;                       // CUDA device the ctx was built on
  // finest-level state and vectors (internal layout)
  double *y = nullptr, *res = nullptr;
  double *V = nullptr, *Z = nullptr;     // Krylov bases
  float* Z32 = nullptr;                  // preconditioned vectors (mixed path)
  double* zd = nullptr;                  // one of them widened to FP64 for the operator product
  double* asm_scratch = nullptr;         // 3D assembly: flux derivatives of one chunk of elements
  int asm_scratch_ne = 0;                // elements of the largest pass the scratch was sized for
  bool mixed = false;
  double *w = nullptr, *xk = nullptr, *bk = nullptr, *tmp = nullptr;
  double* partial = nullptr;              // reduction partials
  double* small = nullptr;                // device scalars
  double* host_small = nullptr;           // pinned mirror
  double *stage_a = nullptr, *stage_b = nullptr;  // canonical staging vectors
  double* dense_ws = nullptr;             // patch factorisation workspace
  int64_t dense_ws_len = 0;
  int32_t *piv_ws = nullptr;              // per-patch pivots
  // coarse dense inverse
  double *c_A = nullptr, *c_B = nullptr, *c_inv = nullptr;
  int32_t* c_piv = nullptr;
  double* c_part = nullptr;               // coarse GEMV partial sums
  int32_t* status = nullptr;              // device status flags
  double* tmp_re = nullptr;               // finest element residuals (n_elem * ndofe)
  // transient (BDF) state: yold = a1 y_n + a2 y_{n-1} (internal layout)
  double* yold = nullptr;
  double bdf_a0 = 0.0, inflow_alpha = 1.0;
  bool have_history = false;
  bool factored = false;   // fsi_factor_schwarz has run at least once
  int32_t* coarse_pad_list = nullptr;     // padding slots of the coarse dense operator
  int32_t* coarse_perm = nullptr;         // internal unknown -> banded position
  int32_t* coarse_pinv = nullptr;         // banded position -> internal unknown
  int coarse_bw = 0;
  int n_coarse_pads = 0;
  // slab-blocked coarse solve (3D): Sinv_k blocks, LU scratch, vectors
  bool coarse_slab = false;
  std::vector<int64_t> slab_off, sinv_off;
  int slab_p = 0, slab_mmax = 0;
  double *c_sinv = nullptr, *c_S = nullptr, *c_T = nullptr, *c_zb = nullptr, *c_xb = nullptr, *c_tp = nullptr;
  int32_t* c_iota = nullptr;
  float t_assemble = 0.f, t_factor = 0.f, t_solve = 0.f;
  int red_blocks = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // the V-cycle as a CUDA graph (captured once on a private stream, replayed
  // on the ctx stream; not used while per-class profiling is on)
  cudaGraph_t vc_graph = nullptr;
  cudaGraphExec_t vc_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  // the coarse factorisation runs on this higher-priority stream beside the
  // Schwarz factorisation (fork / join events on the ctx stream)
  int gj_panel = 0;   // preferred Gauss-Jordan variant on the tensor cores (0, 16, 24, 32, 216)
  long long tc_first_wait = -1;   // first tensor-core wait limit (< 0: the built-in limit)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool aux_failed = false;
  int64_t vc_launches = 0;
  double vc_bytes = 0.0;                  // algorithmic bytes of one recorded V-cycle
  double alg_bytes = 0.0;                 // running total of algorithmic bytes of all launches
  double b_assemble = 0.0, b_factor = 0.0, b_solve = 0.0;   // of the last call of each phase
  bool vc_graph_failed = false;
  // per-kernel-class profiling
  bool prof = false;
  struct KStat {
    double ms = 0.0, bytes = 0.0, flops = 0.0;
    int64_t launches = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  } kstat[FSI_K_COUNT];
  std::vector<cudaEvent_t> event_pool;
};

// status flag slots
enum { ST_SINGULAR = 0, ST_TANGLED = 1, ST_NONFINITE = 2, ST_TIMEOUT = 3, ST_COUNT = 4 };

}  // namespace fsi
