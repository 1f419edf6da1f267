// C-ABI of libfsi: context construction, device uploads, and the host-side
// orchestration of assembly, factorisation, the multigrid V-cycle and FGMRES
// (Sec. 3, 4.1).  Every arithmetic step runs in the kernels of k_*.cu; the
// host only sequences launches, reads the few scalars FGMRES needs for its
// Givens rotations and stopping test, and converts between the canonical
// numbering and the padded device layout.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fsi_internal.h"
#include "kernels.h"

using namespace fsi;

struct fsi_ctx : public Ctx {};

namespace {

struct ApiError : public std::runtime_error {
  int code;
  ApiError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw ApiError(e == cudaErrorMemoryAllocation ? FSI_E_OOM : FSI_E_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
  }
}

template <class T>
T* dalloc(Ctx& c, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  ck(cudaMalloc(&p, n * sizeof(T)), "cudaMalloc");
  c.allocs.push_back(p);
  c.bytes += (int64_t)(n * sizeof(T));
  return static_cast<T*>(p);
}

template <class T>
T* upload(Ctx& c, const std::vector<T>& v) {
  T* p = dalloc<T>(c, v.size());
  if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c.stream), "upload");
  return p;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline void sync(Ctx& c) {
  ck(cudaStreamSynchronize(c.stream), "stream sync");
  ck(cudaGetLastError(), "kernel launch");
}

inline void counted(Ctx& c, int n = 1) { c.launches += n; }

int nblk_red(const Ctx& c) { return c.red_blocks; }

cudaEvent_t get_event(Ctx& c) {
  if (!c.event_pool.empty()) {
    cudaEvent_t e = c.event_pool.back();
    c.event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  ck(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

// NVTX range of a phase (visible in Nsight timelines; no cost without a tool)
struct Nvtx {
  explicit Nvtx(const char* name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
};

// Brackets the launches of one kernel class with events (profiling only) and
// accumulates their algorithmic bytes / flops; the bytes are also counted
// without profiling, for the per-phase totals of fsi_solve_stats.
struct Prof {
  Ctx& c;
  int kind;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Prof(Ctx& c_, int k, double bytes, double flops, int launches = 1) : c(c_), kind(k) {
    c.alg_bytes += bytes;
    if (!c.prof) return;
    e0 = get_event(c);
    e1 = get_event(c);
    cudaEventRecord(e0, c.stream);
    c.kstat[k].bytes += bytes;
    c.kstat[k].flops += flops;
    c.kstat[k].launches += launches;
  }
  ~Prof() {
    if (!e0) return;
    cudaEventRecord(e1, c.stream);
    c.kstat[kind].pending.push_back({e0, e1});
  }
};

void harvest(Ctx& c) {
  sync(c);
  for (auto& ks : c.kstat) {
    for (auto& pr : ks.pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      ks.ms += ms;
      c.event_pool.push_back(pr.first);
      c.event_pool.push_back(pr.second);
    }
    ks.pending.clear();
  }
}

// ---------------------------------------------------------------------------
// canonical <-> internal vectors
// ---------------------------------------------------------------------------
// in (canonical, host or device, length N of level l) -> out (internal, device)
void to_internal(Ctx& c, int l, const double* in, double* out) {
  const DevLevel& D = c.dl[l];
  const double* src = in;
  if (!is_device_ptr(in)) {
    ck(cudaMemcpyAsync(c.stage_a, in, D.N * sizeof(double), cudaMemcpyHostToDevice, c.stream), "H2D");
    src = c.stage_a;
  }
  launch_gather(D.Ni, D.canon_of_int, src, out, c.stream);
  counted(c);
}

void to_canonical(Ctx& c, int l, const double* in, double* out) {
  const DevLevel& D = c.dl[l];
  if (is_device_ptr(out)) {
    launch_gather(D.N, D.int_of_canon, in, out, c.stream);
    counted(c);
  } else {
    launch_gather(D.N, D.int_of_canon, in, c.stage_b, c.stream);
    counted(c);
    ck(cudaMemcpyAsync(out, c.stage_b, D.N * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "D2H");
  }
}

double dev_norm(Ctx& c, int64_t n, const double* v, double* slot) {
  launch_norm_partial(n, v, c.partial, nblk_red(c), c.stream);
  launch_reduce(c.partial, 1, nblk_red(c), slot, true, c.stream);
  counted(c, 2);
  double h = 0.0;
  ck(cudaMemcpyAsync(c.host_small, slot, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "D2H");
  sync(c);
  h = c.host_small[0];
  return h;
}

void check_status(Ctx& c) {
  int32_t st[ST_COUNT];
  ck(cudaMemcpyAsync(st, c.status, sizeof(st), cudaMemcpyDeviceToHost, c.stream), "D2H status");
  sync(c);
  ck(cudaMemsetAsync(c.status, 0, sizeof(st), c.stream), "memset");
#ifdef FSI_BOUNDS_CHECK
  for (int site : {bounds_site_schwarz(), bounds_site_linalg()})
    if (site) throw ApiError(FSI_E_CUDA, "index out of range at bounds-check site " + std::to_string(site));
#endif
  if (st[ST_TIMEOUT]) throw ApiError(FSI_E_TIMEOUT, "a bounded wait on the tensor core gave up");
  if (st[ST_TANGLED]) throw ApiError(FSI_E_MESH_TANGLED, "det F <= 0 at a quadrature point");
  if (st[ST_NONFINITE]) throw ApiError(FSI_E_NONFINITE, "non-finite values");
  if (st[ST_SINGULAR]) throw ApiError(FSI_E_SINGULAR, "zero or non-finite pivot in a Schwarz block or coarse LU");
}

// ---------------------------------------------------------------------------
// build
// ---------------------------------------------------------------------------
void build_device(Ctx& c) {
  const int L = (int)c.hl.size();
  c.dl.assign(L, DevLevel());
  const int dim = c.dim, B = c.B, nloc = c.nloc, nd = c.ndofe;
  int64_t max_dense = 0;
  for (int l = 0; l < L; ++l) {
    HostLevel& H = c.hl[l];
    DevLevel& D = c.dl[l];
    D.n_nodes = H.n_nodes; D.n_elem = H.n_elem; D.N = H.N; D.nb = H.nb; D.Ni = H.Ni; D.nnzb = H.nnzb;
    for (int a = 0; a < 3; ++a) D.cells[a] = H.cells[a];
    D.rowptr = upload(c, H.rowptr);
    D.col = upload(c, H.col);
    D.val = dalloc<double>(c, (size_t)H.nnzb * B * B);
    D.Ke = dalloc<double>(c, (size_t)H.n_elem * nd * nd);
    D.elem_nodes = upload(c, H.elem_nodes);
    D.elem_solid = upload(c, H.elem_solid);
    D.node_class = upload(c, H.node_class);
    std::vector<double> geo(H.n_elem * 2 * dim);
    for (int64_t e = 0; e < H.n_elem; ++e) {
      int idx[3] = {(int)(e % H.cells[0]), (int)((e / H.cells[0]) % H.cells[1]),
                    (int)(e / ((int64_t)H.cells[0] * H.cells[1]))};
      for (int a = 0; a < dim; ++a) {
        geo[e * 2 * dim + a] = H.verts[a][idx[a]];
        geo[e * 2 * dim + dim + a] = H.verts[a][idx[a] + 1] - H.verts[a][idx[a]];
      }
    }
    D.elem_geo = upload(c, geo);
    D.dir = upload(c, H.dir);
    D.dir_val = upload(c, H.dir_val);
    std::vector<int32_t> dl;
    for (int64_t i = 0; i < H.Ni; ++i)
      if (H.dir[i]) dl.push_back((int32_t)i);
    D.n_dir = (int64_t)dl.size();
    D.dir_list = upload(c, dl);
    D.canon_of_int = upload(c, H.canon_of_int);
    std::vector<int32_t> ioc(H.N, -1);
    for (int64_t i = 0; i < H.Ni; ++i)
      if (H.canon_of_int[i] >= 0) ioc[H.canon_of_int[i]] = (int32_t)i;
    D.int_of_canon = upload(c, ioc);
    D.mat_list = upload(c, H.mat_list);
    D.n_fluid_elem = H.n_fluid_elem;
    D.blk_ptr = upload(c, H.blk_ptr); D.blk_src = upload(c, H.blk_src);
    D.res_ptr = upload(c, H.res_ptr); D.res_src = upload(c, H.res_src);
    D.n_blk_src = (int64_t)H.blk_src.size();
    D.n_contrib = (int64_t)(H.blk_src.size() + H.res_src.size());
    if (l > 0) {
      D.P_ptr = upload(c, H.P_ptr); D.P_col = upload(c, H.P_col); D.P_val = upload(c, H.P_val);
      D.R_ptr = upload(c, H.R_ptr); D.R_col = upload(c, H.R_col); D.R_val = upload(c, H.R_val);
      D.S_ptr = upload(c, H.S_ptr); D.S_col = upload(c, H.S_col); D.S_val = upload(c, H.S_val);
      D.n_patches = H.n_patches;
      D.max_n = H.max_n;
      D.max_nown = H.max_nown;
      D.p_n = upload(c, H.p_n); D.p_nown = upload(c, H.p_nown);
      D.p_idx_off = upload(c, H.p_idx_off); D.p_own_off = upload(c, H.p_own_off);
      D.p_dense_off = upload(c, H.p_dense_off); D.p_inv_off = upload(c, H.p_inv_off);
      D.p_gmap_off = upload(c, H.p_gmap_off); D.p_pad_off = upload(c, H.p_pad_off);
      D.p_idx = upload(c, H.p_idx); D.p_own = upload(c, H.p_own);
      D.p_gmap = upload(c, H.p_gmap); D.p_padpos = upload(c, H.p_padpos);
      D.p_boff = upload(c, H.p_boff); D.p_boff_off = upload(c, H.p_boff_off); D.p_gptr = upload(c, H.p_gptr);
      D.inv_total = H.inv_total;
      D.dense_total = H.dense_total;
      if (c.mixed) {
        D.dr32 = dalloc<float>(c, (size_t)H.idx_total);
        D.dc32 = dalloc<float>(c, (size_t)H.idx_total);
        D.inv32 = dalloc<float>(c, (size_t)H.inv_total);
        D.val32 = dalloc<float>(c, (size_t)H.nnzb * B * B);
        std::vector<float> pv(H.P_val.begin(), H.P_val.end()), rv(H.R_val.begin(), H.R_val.end());
        D.P_val32 = upload(c, pv);
        D.R_val32 = upload(c, rv);
      } else {
        D.dr = dalloc<double>(c, (size_t)H.idx_total);
        D.dc = dalloc<double>(c, (size_t)H.idx_total);
        D.inv = dalloc<double>(c, (size_t)H.inv_total);
      }
      max_dense = std::max(max_dense, H.dense_total);
      std::vector<char> is_ilu(H.n_patches, 0);
      if (c.opts.local_solver == 1) {
        // fluid blocks (material of the block's elements) up to the ILU size limit
        std::vector<int32_t> lu, ilu;
        for (int p = 0; p < H.n_patches; ++p) {
          const bool solid = H.elem_solid[H.p_elems[H.p_elem_off[p]]] != 0;
          is_ilu[p] = !solid && H.p_n[p] <= kIluMaxRows;
          (is_ilu[p] ? ilu : lu).push_back(p);
        }
        D.n_lu = (int)lu.size();
        D.n_ilu = (int)ilu.size();
        for (int32_t q : ilu) {
          D.ilu_max_n = std::max(D.ilu_max_n, (int)H.p_n[q]);
          D.ilu_max_nb = std::max(D.ilu_max_nb, (int)(H.p_boff_off[q + 1] - H.p_boff_off[q]));
        }
        D.sel_lu = upload(c, lu);
        D.sel_ilu = upload(c, ilu);
      }
      for (int p = 0; p < H.n_patches; ++p) {
        const double n = H.p_n[p], no = H.p_nown[p];
        if (is_ilu[p]) {
          // the pattern's B x B blocks of L and U (FP32) and their map entries, residual gather + index + row
          // scale, owned index + column scale + x read/write
          const double nz = (double)(H.p_gmap_off[p + 1] - H.p_gmap_off[p]);
          D.apply_bytes32 += nz * (B * B * 4.0 + 12.0) + n * 12.0 + no * 16.0;
          D.apply_flops += 2.0 * nz * B * B;
        } else {
          // inverse rows, residual gather + index + row scale, owned index + column scale + x read/write
          D.apply_bytes += no * n * 8.0 + n * 20.0 + no * 28.0;
          D.apply_bytes32 += no * n * 4.0 + n * 12.0 + no * 16.0;
          D.apply_flops += 2.0 * no * n;
        }
        D.factor_flops += 2.0 * n * n * n;
        D.factor_bytes += n * n * 8.0 + no * n * 8.0;
      }
      D.factor_bytes += (double)H.p_gmap.size() / 3.0 * (B * B * 8.0 + 12.0);
      D.R_bytes = (double)H.R_col.size() * 12.0 + (double)H.Ni * 8.0 + (double)c.hl[l - 1].Ni * 8.0;
      D.P_bytes = (double)H.P_col.size() * 12.0 + (double)H.Ni * 16.0 + (double)c.hl[l - 1].Ni * 8.0;
      D.R_bytes32 = (double)H.R_col.size() * 8.0 + (double)H.Ni * 4.0 + (double)c.hl[l - 1].Ni * 4.0;
      D.P_bytes32 = (double)H.P_col.size() * 8.0 + (double)H.Ni * 8.0 + (double)c.hl[l - 1].Ni * 4.0;
    }
    D.spmv_bytes = (double)H.nnzb * (B * B * 8.0 + 4.0) + (double)(H.nb + 1) * 4.0 + 3.0 * H.Ni * 8.0;
    D.spmv_flops = 2.0 * (double)H.nnzb * B * B;
    D.spmv_bytes32 = (double)H.nnzb * (B * B * 4.0 + 4.0) + (double)(H.nb + 1) * 4.0 + 3.0 * H.Ni * 4.0;
    if (c.mixed) {
      D.x32 = dalloc<float>(c, H.Ni);
      D.b32 = dalloc<float>(c, H.Ni);
      D.r32 = dalloc<float>(c, H.Ni);
      ck(cudaMemsetAsync(D.x32, 0, H.Ni * sizeof(float), c.stream), "memset");
      ck(cudaMemsetAsync(D.b32, 0, H.Ni * sizeof(float), c.stream), "memset");
      ck(cudaMemsetAsync(D.r32, 0, H.Ni * sizeof(float), c.stream), "memset");
    }
    D.x = dalloc<double>(c, H.Ni);
    D.b = dalloc<double>(c, H.Ni);
    D.r = dalloc<double>(c, H.Ni);
    ck(cudaMemsetAsync(D.x, 0, H.Ni * sizeof(double), c.stream), "memset");
    ck(cudaMemsetAsync(D.b, 0, H.Ni * sizeof(double), c.stream), "memset");
    ck(cudaMemsetAsync(D.r, 0, H.Ni * sizeof(double), c.stream), "memset");
  }
  const HostLevel& F = c.hl[L - 1];
  const int64_t Ni = F.Ni;
  const int m = c.opts.restart;
  c.y = dalloc<double>(c, Ni);
  c.res = dalloc<double>(c, Ni);
  ck(cudaMemsetAsync(c.y, 0, Ni * sizeof(double), c.stream), "memset");
  c.V = dalloc<double>(c, (size_t)(m + 1) * Ni);
  if (c.mixed) {
    c.Z32 = dalloc<float>(c, (size_t)m * Ni);
    c.zd = dalloc<double>(c, Ni);
  } else {
    c.Z = dalloc<double>(c, (size_t)m * Ni);
  }
  c.w = dalloc<double>(c, Ni);
  c.xk = dalloc<double>(c, Ni);
  c.bk = dalloc<double>(c, Ni);
  c.tmp = dalloc<double>(c, Ni);
  if (c.desc.transient != 0) {
    c.yold = dalloc<double>(c, Ni);
    ck(cudaMemsetAsync(c.yold, 0, Ni * sizeof(double), c.stream), "memset");
  }
  ck(cudaMemsetAsync(c.V, 0, (size_t)(m + 1) * Ni * sizeof(double), c.stream), "memset");
  c.red_blocks = std::max(1, c.sm_count * 2);
  c.partial = dalloc<double>(c, (size_t)c.red_blocks * 130);
  c.small = dalloc<double>(c, 512);
  ck(cudaMallocHost((void**)&c.host_small, 512 * sizeof(double)), "cudaMallocHost");
  c.stage_a = dalloc<double>(c, F.N);
  c.stage_b = dalloc<double>(c, F.N);
  // the mixed path factors the blocks of all levels in one launch: one
  // workspace region per level
  int64_t sum_dense = 0;
  for (int l = 1; l < L; ++l) sum_dense += c.hl[l].dense_total;
  c.dense_ws_len = std::max<int64_t>(c.mixed ? sum_dense : max_dense, 1);
  // patch factorisation workspace: max_dense elements of the factor precision
  c.dense_ws = dalloc<double>(c, c.mixed ? ((size_t)c.dense_ws_len + 1) / 2 : (size_t)c.dense_ws_len);
  // coarse dense operator
  const int64_t n0 = c.hl[0].Ni;
  c.c_A = dalloc<double>(c, (size_t)n0 * n0);   // banded LU in dense column-major storage
  c.c_B = dalloc<double>(c, (size_t)2 * n0);   // reciprocal pivots of the coarse LU
  c.c_piv = dalloc<int32_t>(c, n0);
  c.coarse_slab = c.dim == 3 && !c.hl[0].slab_off.empty();
  if (!c.coarse_slab) {
    c.c_inv = dalloc<double>(c, (size_t)n0 * n0);   // column-major inverse
    c.c_part = dalloc<double>(c, (size_t)((n0 + 31) / 32) * n0);   // coarse GEMV chunk partials
  } else {
    // block-tridiagonal slab factorisation: inverse Schur complements Sinv_k
    const HostLevel& H0 = c.hl[0];
    c.slab_off = H0.slab_off;
    c.slab_p = H0.slab_p;
    const int K = (int)c.slab_off.size() - 1;
    c.sinv_off.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) {
      const int64_t m = c.slab_off[k + 1] - c.slab_off[k];
      c.slab_mmax = std::max<int>(c.slab_mmax, (int)m);
      c.sinv_off[k + 1] = c.sinv_off[k] + m * m;
    }
    const int64_t mm = c.slab_mmax;
    c.c_sinv = dalloc<double>(c, (size_t)c.sinv_off[K]);
    c.c_S = dalloc<double>(c, (size_t)mm * mm);
    c.c_T = dalloc<double>(c, (size_t)c.slab_p * mm);
    c.c_zb = dalloc<double>(c, n0);
    c.c_xb = dalloc<double>(c, n0);
    c.c_tp = dalloc<double>(c, c.slab_p);
    c.c_part = dalloc<double>(c, (size_t)((mm + 31) / 32) * mm);
    std::vector<int32_t> iota(mm);
    std::iota(iota.begin(), iota.end(), 0);
    c.c_iota = upload(c, iota);
  }
  {
    const HostLevel& H0 = c.hl[0];
    std::vector<int32_t> pinv(H0.Ni);
    for (int64_t i = 0; i < H0.Ni; ++i) pinv[H0.coarse_perm[i]] = (int32_t)i;
    c.coarse_perm = upload(c, H0.coarse_perm);
    c.coarse_pinv = upload(c, pinv);
    c.coarse_bw = H0.coarse_bw;
  }
  c.status = dalloc<int32_t>(c, ST_COUNT);
  ck(cudaMemsetAsync(c.status, 0, ST_COUNT * sizeof(int32_t), c.stream), "memset");
  (void)nloc;
  ck(cudaEventCreate(&c.ev0), "event");
  ck(cudaEventCreate(&c.ev1), "event");
  sync(c);
}

// coarse pad list (internal indices of padding slots of the level-0 layout)
std::vector<int32_t> coarse_pads(const Ctx& c) {
  const HostLevel& H = c.hl[0];
  std::vector<int32_t> v;
  for (int64_t i = 0; i < H.Ni; ++i)
    if (H.canon_of_int[i] < 0) v.push_back((int32_t)i);
  return v;
}

// ---------------------------------------------------------------------------
// assembly
// ---------------------------------------------------------------------------
void assemble_impl(Ctx& c);
bool aux_stream(Ctx& c);
void assemble(Ctx& c, bool want_res) {
  Nvtx nv("fsi assemble + Galerkin");
  const double b0 = c.alg_bytes;
  assemble_impl(c);
  c.b_assemble = c.alg_bytes - b0;
  (void)want_res;
}

void assemble_impl(Ctx& c) {
  const int L = (int)c.dl.size();
  const int B = c.B;
  DevLevel& F = c.dl[L - 1];
  PhysParams pp{c.desc.rho_f, c.desc.mu_f, c.desc.rho_s, c.desc.mu_s, c.desc.ale_op, c.desc.mr_c2};
  const bool transient = c.desc.transient != 0;
  if (transient) {
    if (!c.have_history) throw ApiError(FSI_E_INVALID, "transient problem: fsi_set_state needs y_prev first");
    pp.transient = c.desc.transient == 2 ? 2 : 1;
    pp.a0 = c.bdf_a0;
    pp.idt = 1.0 / c.desc.dt;
    pp.yold = c.yold;
  }
  double* Re = c.tmp_re;
  const double nd = c.ndofe;
  {
    // element matrices: one pass over the fluid elements and one over the
    // solid ones (in 2D the small solid pass runs on the private stream beside
    // the fluid one; in 3D both share the flux scratch, so they run in turn)
    const int nf = (int)F.n_fluid_elem, ns = (int)(F.n_elem - F.n_fluid_elem);
    // bytes: element state in, element matrix + residual out; flops: executed FP64 operations
    Prof pr(c, FSI_K_ASSEMBLE, (double)F.n_elem * (nd * 8.0 + nd * nd * 8.0 + nd * 8.0),
            nf * assemble_flops_per_element(c.dim, false, pp.transient) +
                ns * assemble_flops_per_element(c.dim, true, pp.transient),
            (nf > 0) + (ns > 0));
    auto run = [&](bool solid, const int32_t* list, int ne, cudaStream_t st) {
      if (!(c.dim == 2 ? launch_assemble_2d : launch_assemble_3d)(solid, list, ne, c.y, F.elem_nodes, F.node_class,
                                                                   F.elem_geo, F.n_nodes, pp, F.Ke, Re, c.status,
                                                                   c.asm_scratch, c.asm_scratch_ne, st))
        throw ApiError(FSI_E_CUDA, "assembly: element pass larger than the flux scratch");
      counted(c, assemble_launches(c.dim, ne));
    };
    const bool fork = c.dim == 2 && nf > 0 && ns > 0 && !c.prof && aux_stream(c);
    if (fork) {
      cudaEventRecord(c.ev_fork, c.stream);
      cudaStreamWaitEvent(c.aux_stream, c.ev_fork, 0);
      run(true, F.mat_list + nf, ns, c.aux_stream);
      cudaEventRecord(c.ev_join, c.aux_stream);
    }
    run(false, F.mat_list, nf, c.stream);
    if (fork) cudaStreamWaitEvent(c.stream, c.ev_join, 0);
    else run(true, F.mat_list + nf, ns, c.stream);
  }
  {
    // element matrices in, block values out, gather lists; residual likewise
    Prof pr(c, FSI_K_SCATTER,
            (double)F.n_elem * nd * (nd + 1.0) * 8.0 + (double)F.nnzb * B * B * 8.0 + (double)F.Ni * 8.0 +
                (double)(F.nnzb + F.nb + F.n_contrib) * 4.0,
            0.0, 3);
    launch_gather_elements(c.dim, F.nnzb, F.blk_ptr, F.blk_src, F.Ke, F.val, F.nb, F.res_ptr, F.res_src, Re, c.res,
                           c.stream);
    counted(c, 2);
    launch_dirichlet(F.dir_list, F.n_dir, F.rowptr, F.col, F.val, B, c.y, F.dir_val, transient ? c.inflow_alpha : 1.0,
                     c.res, c.stream);
    counted(c);
  }
  launch_nonfinite_check(F.Ni, c.res, c.status, c.stream);
  counted(c);
  for (int l = L - 1; l >= 1; --l) {
    DevLevel& Fi = c.dl[l];
    DevLevel& Co = c.dl[l - 1];
    {
      Prof pr(c, FSI_K_GALERKIN, (double)Fi.n_elem * nd * nd * 8.0 + (double)Co.n_elem * nd * nd * 8.0,
              (double)Co.n_elem * galerkin_flops_per_coarse_element(c.dim));
      if (c.dim == 2)
        launch_galerkin_2d(Co.cells[0], Co.cells[1], Fi.Ke, Fi.elem_nodes, Fi.node_class, Fi.dir, Co.elem_nodes,
                           Co.node_class, Co.dir, Co.Ke, c.stream);
      else
        launch_galerkin_3d(Co.cells[0], Co.cells[1], Co.cells[2], Fi.Ke, Fi.elem_nodes, Fi.node_class, Fi.dir,
                           Co.elem_nodes, Co.node_class, Co.dir, Co.Ke, c.stream);
      counted(c);
    }
    Prof pr(c, FSI_K_SCATTER,
            (double)Co.n_elem * nd * nd * 8.0 + (double)Co.nnzb * B * B * 8.0 + (double)Co.nnzb * 4.0 +
                (double)Co.n_blk_src * 4.0,
            0.0, 2);
    launch_gather_elements(c.dim, Co.nnzb, Co.blk_ptr, Co.blk_src, Co.Ke, Co.val, 0, nullptr, nullptr, nullptr,
                           nullptr, c.stream);
    counted(c);
    launch_dirichlet(Co.dir_list, Co.n_dir, Co.rowptr, Co.col, Co.val, B, nullptr, nullptr, 1.0, nullptr, c.stream);
    counted(c);
  }
  if (c.mixed)
    for (int l = 1; l < L; ++l) {
      DevLevel& D = c.dl[l];
      const int64_t nv = D.nnzb * B * B;
      Prof pr(c, FSI_K_SCATTER, (double)nv * 12.0, 0.0);
      launch_to_f32(nv, D.val, D.val32, c.stream);
      counted(c);
    }
  check_status(c);
}

// ---------------------------------------------------------------------------
// slab-blocked coarse LU (3D).  In the banded (x-slab) ordering the coarse
// operator is block tridiagonal over slabs; block elimination gives the
// Schur complements S_0 = A_00, S_k = A_kk - A_{k,k-1} S_{k-1}^{-1} A_{k-1,k},
// each inverted by partial-pivot LU.  As A_{k,k-1} and A_{k-1,k} are nonzero
// only on the last x-plane P of slab k-1, the update is
// A_{k,k-1}[:,P] (S_{k-1}^{-1}[P,P] A_{k-1,k}[P,:]).
// ---------------------------------------------------------------------------
void coarse_factor_slab(Ctx& c) {
  DevLevel& C = c.dl[0];
  const int64_t n0 = C.Ni;
  const int K = (int)c.slab_off.size() - 1;
  const int p = c.slab_p;
  double flops = 0.0, bytes = (double)n0 * n0 * 8.0;
  for (int k = 0; k < K; ++k) {
    const double m = (double)(c.slab_off[k + 1] - c.slab_off[k]);
    flops += 2.0 * m * m * m * (2.0 / 3.0 + 1.0);   // LU + inverse columns
    if (k > 0) flops += 2.0 * p * (double)p * m + 2.0 * m * p * m;
    bytes += 3.0 * m * m * 8.0;
  }
  Prof pr(c, FSI_K_COARSE_FACTOR, bytes, flops, (c.n_coarse_pads > 0 ? 2 : 1) + 3 * K + 2 * (K - 1));
  launch_dense_gather(c.B, C.nb, C.rowptr, C.col, C.val, c.coarse_pad_list, c.n_coarse_pads, c.coarse_perm, n0,
                      c.c_A, c.stream);
  counted(c, c.n_coarse_pads > 0 ? 2 : 1);
  for (int k = 0; k < K; ++k) {
    const int64_t o = c.slab_off[k];
    const int m = (int)(c.slab_off[k + 1] - o);
    double* Akk = c.c_A + o * n0 + o;
    launch_copy2d(m, m, Akk, n0, c.c_S, m, c.stream);
    counted(c);
    if (k > 0) {
      const int64_t op = c.slab_off[k - 1];
      const int mp = (int)(o - op);
      const double* Sp = c.c_sinv + c.sinv_off[k - 1];
      // T = S_{k-1}^{-1}[P,P] A_{k-1,k}[P,:]   (p x m)
      launch_dgemm_nn(p, m, p, 1.0, Sp + (int64_t)(mp - p) * mp + (mp - p), mp, c.c_A + o * n0 + (o - p), n0, 0.0,
                      c.c_T, p, c.stream);
      // S -= A_{k,k-1}[:,P] T
      launch_dgemm_nn(m, m, p, -1.0, c.c_A + (o - p) * n0 + o, n0, c.c_T, p, 1.0, c.c_S, m, c.stream);
      counted(c, 2);
    }
    const int rc = launch_coarse_lu_inverse(m, m - 1, m - 1, c.c_S, c.c_B, c.c_sinv + c.sinv_off[k], c.c_piv,
                                            c.c_iota, c.c_iota, c.status, c.sm_count, c.stream);
    if (rc != 0) throw ApiError(FSI_E_CUDA, "slab LU launch failed (" + std::to_string(rc) + ")");
    counted(c, 2);
  }
}

// x = A_0^{-1} b (internal ordering, FP64): forward block elimination
// w_k = b_k - A_{k,k-1}[:,P] (S_{k-1}^{-1}[P,:] w_{k-1}), then back
// substitution x_k = S_k^{-1} (w_k - A_{k,k+1} x_{k+1}) with A_{k,k+1}
// nonzero in the rows P of slab k only.
void coarse_apply_slab(Ctx& c, const double* b, double* x) {
  const int64_t n0 = c.dl[0].Ni;
  const int K = (int)c.slab_off.size() - 1;
  const int p = c.slab_p;
  launch_gather(n0, c.coarse_pinv, b, c.c_zb, c.stream);
  counted(c);
  for (int k = 1; k < K; ++k) {
    const int64_t o = c.slab_off[k], op = c.slab_off[k - 1];
    const int m = (int)(c.slab_off[k + 1] - o), mp = (int)(o - op);
    const double* Sp = c.c_sinv + c.sinv_off[k - 1];
    launch_gemv_sub(p, mp, 1.0, Sp + (mp - p), mp, c.c_zb + op, 0.0, c.c_tp, c.c_part, c.stream);
    launch_gemv_sub(m, p, -1.0, c.c_A + (o - p) * n0 + o, n0, c.c_tp, 1.0, c.c_zb + o, c.c_part, c.stream);
    counted(c, 4);
  }
  for (int k = K - 1; k >= 0; --k) {
    const int64_t o = c.slab_off[k];
    const int m = (int)(c.slab_off[k + 1] - o);
    if (k < K - 1) {
      const int64_t on = c.slab_off[k + 1];
      const int mn = (int)(c.slab_off[k + 2] - on);
      launch_gemv_sub(p, mn, -1.0, c.c_A + on * n0 + (on - p), n0, c.c_xb + on, 1.0, c.c_zb + (on - p), c.c_part,
                      c.stream);
      counted(c, 2);
    }
    launch_gemv_sub(m, m, 1.0, c.c_sinv + c.sinv_off[k], m, c.c_zb + o, 0.0, c.c_xb + o, c.c_part, c.stream);
    counted(c, 2);
  }
  launch_gather(n0, c.coarse_perm, c.c_xb, x, c.stream);
  counted(c);
}

double coarse_slab_apply_bytes(const Ctx& c) {
  const int K = (int)c.slab_off.size() - 1;
  double b = 0.0;
  for (int k = 0; k < K; ++k) {
    const double m = (double)(c.slab_off[k + 1] - c.slab_off[k]);
    b += m * m * 8.0 + (k > 0 ? 2.0 * c.slab_p * m * 8.0 : 0.0);
  }
  return b;
}

// ---------------------------------------------------------------------------
// Schwarz factorisation (all levels >= 1) + coarse LU
// ---------------------------------------------------------------------------
// Largest Schwarz block of the instance (levels >= 1).
int max_block(const Ctx& c) {
  int m = 0;
  for (size_t l = 1; l < c.dl.size(); ++l) m = std::max(m, c.dl[l].max_n);
  return m;
}

// Mixed path: gathers the Schwarz blocks of every level >= 1 of c into the
// level's region of its FP32 workspace (on c.stream) and appends the levels
// to the tensor-core factorisation table lv (blocks numbered from *first).
// Returns false when a level has no blocks or the table is full.
bool gather_mixed(Ctx& c, GjLevels& lv, int& first, int& max_n) {
  const int L = (int)c.dl.size();
  float* ws = reinterpret_cast<float*>(c.dense_ws);
  int64_t off = 0;
  bool ok = true;
  // the gathers of all levels in one launch when the table holds them
  GatherLevels gl{};
  gl.B = c.B;
  int gblocks = 0;
  const bool one_launch = L - 1 <= kGjMaxLevels;
  for (int l = 1; l < L; ++l) {
    DevLevel& D = c.dl[l];
    if (one_launch) {
      if (D.n_patches > 0)
        gl.l[gl.nlev++] = GatherLevel{D.p_n,    D.p_dense_off, D.p_gmap_off, D.p_gmap,      D.p_boff_off,
                                      D.p_boff, D.p_pad_off,   D.p_padpos,   D.val,         ws + off,
                                      D.p_idx_off, D.dr32,     D.dc32,       gblocks};
      gblocks += D.n_patches;
    } else {
      launch_patch_gather_t<float>(D.n_patches, D.p_n, D.p_dense_off, D.p_gmap_off, D.p_gmap, D.p_boff_off,
                                   D.p_boff, D.p_pad_off, D.p_padpos, D.val, c.B, ws + off, D.p_idx_off, D.dr32,
                                   D.dc32, c.stream);
      counted(c);
    }
    off += D.dense_total;
  }
  if (one_launch && gblocks > 0) {
    launch_patch_gather_levels(gl, gblocks, c.stream);
    counted(c);
  }
  off = 0;
  for (int l = 1; l < L; ++l) {
    DevLevel& D = c.dl[l];
    const bool ilu = c.opts.local_solver == 1;
    const int nsel = ilu ? D.n_lu : D.n_patches;
    if (ilu) {   // the fluid blocks: ILU(0) in place in the workspace
      launch_patch_ilu0(D.n_ilu, D.sel_ilu, D.p_n, D.p_dense_off, D.p_gmap_off, D.p_gmap, D.p_boff_off, D.p_boff, c.B,
                        ws + off, c.status, c.stream);
      if (D.n_ilu > 0) counted(c);
    }
    if (nsel > 0 && lv.nlev < kGjMaxLevels) {
      lv.l[lv.nlev++] = GjLevel{D.p_n, D.p_nown, D.p_dense_off, D.p_own_off, D.p_own, D.p_inv_off, ws + off,
                                D.inv32, c.status, ilu ? D.sel_lu : nullptr, first};
      first += nsel;
      max_n = std::max(max_n, D.max_n);
    } else if (nsel > 0 || !ilu) {
      ok = false;
    }
    off += D.dense_total;
  }
  return ok;
}

// FP32 workspace region of level l (the mixed path keeps every level's
// gathered blocks, which the ILU(0) blocks are applied from)
float* level_ws(Ctx& c, int l) {
  int64_t off = 0;
  for (int k = 1; k < l; ++k) off += c.dl[k].dense_total;
  return reinterpret_cast<float*>(c.dense_ws) + off;
}

void schwarz_factor(Ctx& c) {
  const int L = (int)c.dl.size();
  const int B = c.B;
  if (c.mixed && L > 1) {
    // gather every level into its own workspace region, then factor the
    // blocks of all levels in one tensor-core launch (the smaller levels fill
    // the GPU beside the finest one)
    float* ws = reinterpret_cast<float*>(c.dense_ws);
    GjLevels lv{};
    lv.nlev = 0;
    lv.first_wait = c.tc_first_wait >= 0 ? c.tc_first_wait : kTcWaitIters;
    int first = 0, max_n = 0;
    double by = 0.0, fl = 0.0;
    int64_t off = 0;
    std::vector<int64_t> base(L, 0);
    for (int l = 1; l < L; ++l) {
      DevLevel& D = c.dl[l];
      base[l] = off;
      off += D.dense_total;
      by += D.factor_bytes;
      fl += D.factor_flops;
    }
    // launches: one gather for all levels (one per level past the table's
    // capacity) and the tensor-core factorisation
    Prof pr(c, FSI_K_PATCH_FACTOR, by, fl, (L - 1 <= kGjMaxLevels ? 1 : L - 1) + 1);
    const bool all = gather_mixed(c, lv, first, max_n);
    if (all && (lv.nlev == 0 || launch_patch_gj_tc_levels(lv, first, max_n, c.status, c.stream, c.gj_panel))) {
      if (lv.nlev > 0) counted(c);
    } else if (c.opts.local_solver == 1) {
      throw ApiError(FSI_E_INVALID, "ILU(0) fluid blocks: the exact blocks do not fit the tensor-core factorisation");
    } else {
      for (int l = 1; l < L; ++l) {   // blocks too large for the tensor-core kernel: level by level
        DevLevel& D = c.dl[l];
        launch_patch_gj_t<float>(D.n_patches, D.max_n, D.p_n, D.p_nown, D.p_dense_off, D.p_own_off, D.p_own,
                                 D.p_inv_off, ws + base[l], D.inv32, c.status, true, c.stream);
        counted(c);
      }
    }
  }
  for (int l = 1; l < L && !c.mixed; ++l) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_PATCH_FACTOR, D.factor_bytes, D.factor_flops, 2);
    launch_patch_gather_t<double>(D.n_patches, D.p_n, D.p_dense_off, D.p_gmap_off, D.p_gmap, D.p_boff_off,
                                  D.p_boff, D.p_pad_off, D.p_padpos, D.val, B, c.dense_ws, D.p_idx_off, D.dr, D.dc,
                                  c.stream);
    launch_patch_gj_t<double>(D.n_patches, D.max_n, D.p_n, D.p_nown, D.p_dense_off, D.p_own_off, D.p_own,
                              D.p_inv_off, c.dense_ws, D.inv, c.status, true, c.stream);
    counted(c, 2);
  }
}

void coarse_factor(Ctx& c) {
  const int B = c.B;
  DevLevel& C = c.dl[0];
  const int64_t n0 = C.Ni;
  if (c.coarse_slab) {
    coarse_factor_slab(c);
  } else {
    const double nn = (double)n0;
    // banded LU (2 n kl (kl + ku) flops) + inverse columns (~2 n^2 (kl + ku) flops, sparsity aside)
    const double bw = (double)c.coarse_bw;
    Prof pr(c, FSI_K_COARSE_FACTOR, nn * nn * 8.0 * 3.0, 2.0 * nn * bw * 2.0 * bw + 2.0 * nn * nn * 2.0 * bw, 4);
    launch_dense_gather(B, C.nb, C.rowptr, C.col, C.val, c.coarse_pad_list, c.n_coarse_pads, c.coarse_perm, n0,
                        c.c_A, c.stream);
    counted(c, c.n_coarse_pads > 0 ? 2 : 1);
    const int rc = launch_coarse_lu_inverse(n0, c.coarse_bw, c.coarse_bw, c.c_A, c.c_B, c.c_inv, c.c_piv,
                                            c.coarse_perm, c.coarse_pinv, c.status, c.sm_count, c.stream);
    if (rc != 0) throw ApiError(FSI_E_CUDA, "banded coarse LU launch failed (" + std::to_string(rc) + ")");
    counted(c, 2);
  }
}

// Private stream (highest priority) and fork / join events for the coarse
// factorisation; false if they cannot be created (then everything stays on
// the ctx stream).
bool aux_stream(Ctx& c) {
  if (c.aux_stream) return true;
  if (c.aux_failed) return false;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (cudaStreamCreateWithPriority(&c.aux_stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    c.aux_failed = true;
    return false;
  }
  return true;
}

struct StreamSwap {   // launches of the enclosing scope go to another stream
  Ctx& c;
  cudaStream_t saved;
  StreamSwap(Ctx& ctx, cudaStream_t s) : c(ctx), saved(ctx.stream) { c.stream = s; }
  ~StreamSwap() { c.stream = saved; }
};

// The coarse LU (level 0) and the Schwarz blocks (levels >= 1) depend only on
// the assembled operators, not on each other.  The coarse factorisation is a
// chain of latency-bound launches that fills a fraction of the SMs, so it runs
// on the private stream while the block factorisations take the rest of the
// GPU; the ctx stream waits for it before anything that follows.  With
// per-class profiling on (events on the ctx stream) the two run one after the
// other.
void factor(Ctx& c) {
  Nvtx nv("fsi factor (Schwarz + coarse)");
  const double b0 = c.alg_bytes;
  const bool fork = !c.prof && aux_stream(c);
  if (fork) {
    cudaEventRecord(c.ev_fork, c.stream);
    cudaStreamWaitEvent(c.aux_stream, c.ev_fork, 0);
    {
      StreamSwap sw(c, c.aux_stream);
      coarse_factor(c);
    }
    cudaEventRecord(c.ev_join, c.aux_stream);
  }
  schwarz_factor(c);
  if (fork) cudaStreamWaitEvent(c.stream, c.ev_join, 0);
  else coarse_factor(c);
  check_status(c);
  c.factored = true;
  c.b_factor = c.alg_bytes - b0;
}

// ---------------------------------------------------------------------------
// multigrid V-cycle (Sec. 3, 3.3): internal vectors of level l
// ---------------------------------------------------------------------------
void spmv(Ctx& c, int l, const double* x, const double* b, double* y, int kind = FSI_K_SPMV) {
  DevLevel& D = c.dl[l];
  Prof pr(c, kind, D.spmv_bytes - (b ? 0.0 : D.Ni * 8.0), D.spmv_flops);
  launch_bsr_residual(c.B, D.nb, D.rowptr, D.col, D.val, x, b, y, c.stream);
  counted(c);
}

// Level data of the V-cycle in precision T (double: FP64 path, float: mixed).
template <typename T> struct VC;
template <> struct VC<double> {
  static double* x(DevLevel& D) { return D.x; }
  static double* b(DevLevel& D) { return D.b; }
  static double* r(DevLevel& D) { return D.r; }
  static void residual(Ctx& c, int l, const double* x, const double* b, double* y) { spmv(c, l, x, b, y); }
  static void apply(Ctx& c, int l, const double* r, double* x) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_PATCH_APPLY, D.apply_bytes, D.apply_flops);
    launch_patch_apply_t<double>(D.n_patches, D.Ni, D.max_n, D.max_nown, D.p_n, D.p_nown, D.p_idx_off, D.p_idx,
                                 D.p_own_off, D.p_own, D.p_inv_off, D.inv, r, x, c.opts.omega, D.dr, D.dc,
                                 c.sm_count, D.apply_slices, D.apply_groups, c.stream);
    counted(c);
  }
  static void restrict_(Ctx& c, int l, const double* r, double* bc) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_TRANSFER, D.R_bytes, 2.0 * (double)c.hl[l].R_col.size());
    launch_csr_spmv(c.dl[l - 1].Ni, D.R_ptr, D.R_col, D.R_val, r, bc, false, c.stream);
    counted(c);
  }
  static void prolong_add(Ctx& c, int l, const double* xc, double* x) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_TRANSFER, D.P_bytes, 2.0 * (double)c.hl[l].P_col.size());
    launch_csr_spmv(D.Ni, D.P_ptr, D.P_col, D.P_val, xc, x, true, c.stream);
    counted(c);
  }
  static void coarse(Ctx& c, const double* b, double* x) {
    const double n0 = (double)c.dl[0].Ni;
    if (c.coarse_slab) {
      const double by = coarse_slab_apply_bytes(c);
      Prof pr(c, FSI_K_TRANSFER, by + 4.0 * n0 * 8.0, by / 4.0, 2 + 8 * ((int)c.slab_off.size() - 1));
      coarse_apply_slab(c, b, x);
      return;
    }
    Prof pr(c, FSI_K_TRANSFER, n0 * n0 * 8.0 + 2.0 * n0 * 8.0, 2.0 * n0 * n0);
    launch_gemv(c.dl[0].Ni, c.c_inv, b, x, c.c_part, c.stream);
    counted(c, 2);
  }
};
template <> struct VC<float> {
  static float* x(DevLevel& D) { return D.x32; }
  static float* b(DevLevel& D) { return D.b32; }
  static float* r(DevLevel& D) { return D.r32; }
  static void residual(Ctx& c, int l, const float* x, const float* b, float* y) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_SPMV, D.spmv_bytes32, D.spmv_flops);
    launch_bsr_residual_f32(c.B, D.nb, D.rowptr, D.col, D.val32, x, b, y, D.spmv_sub, c.stream);
    counted(c);
  }
  static void apply(Ctx& c, int l, const float* r, float* x) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_PATCH_APPLY, D.apply_bytes32, D.apply_flops);
    if (c.opts.local_solver == 1) {   // exact inverses of the solid blocks, ILU(0) solves of the fluid ones
      launch_patch_apply_t<float>(D.n_lu, D.Ni, D.max_n, D.max_nown, D.p_n, D.p_nown, D.p_idx_off, D.p_idx, D.p_own_off,
                                  D.p_own, D.p_inv_off, D.inv32, r, x, c.opts.omega, D.dr32, D.dc32, c.sm_count,
                                  D.apply_slices, D.apply_groups, c.stream, D.sel_lu);
      launch_patch_apply_ilu(D.n_ilu, D.ilu_max_n, D.ilu_max_nb, D.sel_ilu, D.p_n, D.p_nown, D.p_idx_off, D.p_idx,
                             D.p_own_off, D.p_own, D.p_dense_off, D.p_gmap_off, D.p_gmap, D.p_boff_off, D.p_boff,
                             D.p_gptr, c.B, level_ws(c, l), r, x, c.opts.omega, D.dr32, D.dc32, c.stream);
      counted(c, (D.n_lu > 0) + (D.n_ilu > 0));
      return;
    }
    launch_patch_apply_t<float>(D.n_patches, D.Ni, D.max_n, D.max_nown, D.p_n, D.p_nown, D.p_idx_off, D.p_idx,
                                D.p_own_off, D.p_own, D.p_inv_off, D.inv32, r, x, c.opts.omega, D.dr32, D.dc32,
                                c.sm_count, D.apply_slices, D.apply_groups, c.stream);
    counted(c);
  }
  static void restrict_(Ctx& c, int l, const float* r, float* bc) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_TRANSFER, D.R_bytes32, 2.0 * (double)c.hl[l].R_col.size());
    launch_csr_spmv_f32(c.dl[l - 1].Ni, D.R_ptr, D.R_col, D.R_val32, r, bc, false, c.stream);
    counted(c);
  }
  static void prolong_add(Ctx& c, int l, const float* xc, float* x) {
    DevLevel& D = c.dl[l];
    Prof pr(c, FSI_K_TRANSFER, D.P_bytes32, 2.0 * (double)c.hl[l].P_col.size());
    launch_csr_spmv_f32(D.Ni, D.P_ptr, D.P_col, D.P_val32, xc, x, true, c.stream);
    counted(c);
  }
  static void coarse(Ctx& c, const float* b, float* x) {
    // the coarsest-grid solve stays FP64 (FP64 inverse, FP64 accumulation)
    const double n0 = (double)c.dl[0].Ni;
    if (c.coarse_slab) {
      const double by = coarse_slab_apply_bytes(c);
      Prof pr(c, FSI_K_TRANSFER, by + 4.0 * n0 * 8.0 + 2.0 * n0 * 4.0, by / 4.0, 4 + 8 * ((int)c.slab_off.size() - 1));
      launch_to_f64(c.dl[0].Ni, b, c.c_xb, c.stream);
      counted(c);
      coarse_apply_slab(c, c.c_xb, c.c_zb);   // both buffers are free again when it writes its result
      launch_to_f32(c.dl[0].Ni, c.c_zb, x, c.stream);
      counted(c);
      return;
    }
    Prof pr(c, FSI_K_TRANSFER, n0 * n0 * 8.0 + 2.0 * n0 * 4.0, 2.0 * n0 * n0);
    launch_gemv_f32io(c.dl[0].Ni, c.c_inv, b, x, c.c_part, c.stream);
    counted(c, 2);
  }
};

template <typename T>
void smooth_step_t(Ctx& c, int l, const T* b, T* x, bool x_is_zero) {
  DevLevel& D = c.dl[l];
  const T* r = b;
  if (!x_is_zero) {
    VC<T>::residual(c, l, x, b, VC<T>::r(D));
    r = VC<T>::r(D);
  }
  VC<T>::apply(c, l, r, x);
}

template <typename T>
void vcycle_t(Ctx& c, int l, const T* b, T* x) {
  static const char* names[] = {"fsi V-cycle level 0", "fsi V-cycle level 1", "fsi V-cycle level 2",
                                "fsi V-cycle level 3", "fsi V-cycle level 4", "fsi V-cycle level 5",
                                "fsi V-cycle level 6", "fsi V-cycle level 7+"};
  Nvtx nv(names[l < 7 ? l : 7]);
  if (l == 0) {
    VC<T>::coarse(c, b, x);
    return;
  }
  DevLevel& D = c.dl[l];
  DevLevel& C = c.dl[l - 1];
  ck(cudaMemsetAsync(x, 0, D.Ni * sizeof(T), c.stream), "memset");
  for (int s = 0; s < c.opts.n_pre; ++s) smooth_step_t<T>(c, l, b, x, s == 0);
  VC<T>::residual(c, l, x, b, VC<T>::r(D));
  VC<T>::restrict_(c, l, VC<T>::r(D), VC<T>::b(C));
  vcycle_t<T>(c, l - 1, VC<T>::b(C), VC<T>::x(C));
  VC<T>::prolong_add(c, l, VC<T>::x(C), x);
  for (int s = 0; s < c.opts.n_post; ++s) smooth_step_t<T>(c, l, b, x, false);
}

// Records one V-cycle of the finest level, from its own b to its own x
// buffer (FP32 on the mixed path), as a CUDA graph.  The V-cycle uses the same
// buffers and launch parameters on every call, so the graph stays valid for
// the ctx's lifetime; on any capture error the direct launches are used.
void capture_vcycle(Ctx& c) {
  const int L = (int)c.dl.size();
  DevLevel& F = c.dl[L - 1];
  if (!c.cap_stream && cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    c.cap_stream = nullptr;
    c.vc_graph_failed = true;
    return;
  }
  const cudaStream_t saved = c.stream;
  const int64_t l0 = c.launches;
  const double b0 = c.alg_bytes;
  c.stream = c.cap_stream;
  bool ok = cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    try {
      if (c.mixed) vcycle_t<float>(c, L - 1, F.b32, F.x32);
      else vcycle_t<double>(c, L - 1, F.b, F.x);
    } catch (const ApiError&) {
      ok = false;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(c.cap_stream, &g) != cudaSuccess || !ok || !g) {
      ok = false;
      if (g) cudaGraphDestroy(g);
    } else {
      c.vc_graph = g;
      ok = cudaGraphInstantiate(&c.vc_exec, g, 0) == cudaSuccess;
    }
  }
  c.stream = saved;
  c.vc_launches = c.launches - l0;
  c.launches = l0;
  c.vc_bytes = c.alg_bytes - b0;   // algorithmic bytes of one V-cycle (counted per replay)
  c.alg_bytes = b0;
  if (!ok) {
    c.vc_exec = nullptr;
    c.vc_graph_failed = true;
    cudaGetLastError();
  }
}

// z = M^{-1} v on the finest level (FP64 in and out; FP32 inside on the mixed path)
void precondition(Ctx& c, const double* v, double* z64, float* z32) {
  const int L = (int)c.dl.size();
  if (!c.prof && !c.vc_graph_failed) {
    if (!c.vc_exec) capture_vcycle(c);
    if (c.vc_exec) {
      DevLevel& F = c.dl[L - 1];
      if (c.mixed) {
        launch_to_f32(F.Ni, v, F.b32, c.stream);
        counted(c);
      } else {
        ck(cudaMemcpyAsync(F.b, v, F.Ni * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "copy");
      }
      ck(cudaGraphLaunch(c.vc_exec, c.stream), "cudaGraphLaunch");
      c.launches += c.vc_launches;
      c.alg_bytes += c.vc_bytes;
      if (c.mixed) {
        if (z32 != F.x32)
          ck(cudaMemcpyAsync(z32, F.x32, F.Ni * sizeof(float), cudaMemcpyDeviceToDevice, c.stream), "copy");
      } else if (z64 != F.x) {
        ck(cudaMemcpyAsync(z64, F.x, F.Ni * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "copy");
      }
      return;
    }
  }
  if (!c.mixed) {
    vcycle_t<double>(c, L - 1, v, z64);
    return;
  }
  DevLevel& F = c.dl[L - 1];
  launch_to_f32(F.Ni, v, F.b32, c.stream);
  counted(c);
  vcycle_t<float>(c, L - 1, F.b32, z32);
}

// ---------------------------------------------------------------------------
// Arnoldi orthonormalisation of c.w against V[0..j] by classical Gram-Schmidt
// with `passes` passes (each pass's j + 1 dot products in one sweep over the
// basis), v_{j+1} = w / ||w||.  Returns the Hessenberg column h[0..j] and
// ||w|| after / before orthogonalisation (host values).
// ---------------------------------------------------------------------------
void orthonormalize(Ctx& c, int j, int passes, double* h, double* hn, double* wn0) {
  const int L = (int)c.dl.size();
  const int64_t n = c.dl[L - 1].Ni;
  const int nb = nblk_red(c);
  double* sm = c.small;
  double* hs = c.host_small;
  Prof pr(c, FSI_K_KRYLOV, (2.0 * passes * (j + 1) + 8.0) * n * 8.0, (4.0 * passes * (j + 1) + 4.0) * n,
          passes == 2 ? 8 : 5);
  // pass 1: h1 = V^T w (with ||w||^2)
  launch_arnoldi_dots(n, c.V, n, j + 1, c.w, true, c.partial, nb, c.stream);
  launch_reduce(c.partial, j + 2, nb, sm, false, c.stream);             // h1 = sm[0..j], ||w||^2 = sm[j+1]
  const double* hlast = sm;
  if (passes == 2) {
    launch_cgs_update(n, c.V, n, j + 1, sm, c.w, c.stream);
    launch_arnoldi_dots(n, c.V, n, j + 1, c.w, false, c.partial, nb, c.stream);
    launch_reduce(c.partial, j + 1, nb, sm + 128, false, c.stream);     // h2
    hlast = sm + 128;
  }
  launch_arnoldi_update_norm(n, c.V, n, j + 1, hlast, c.w, c.partial, nb, c.stream);
  launch_reduce(c.partial, 1, nb, sm + 257, true, c.stream);            // ||w|| after the passes
  launch_scale_by(n, c.w, sm + 257, c.V + (size_t)(j + 1) * n, c.stream);
  counted(c, passes == 2 ? 8 : 5);
  ck(cudaMemcpyAsync(hs, sm, 260 * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "D2H");
  sync(c);
  for (int i = 0; i <= j; ++i) h[i] = hs[i] + (passes == 2 ? hs[128 + i] : 0.0);
  *hn = hs[257];
  *wn0 = std::sqrt(hs[j + 1]);
}

// out = M^{-1} in on the finest level, FP64 in and out (FP32 V-cycle inside on
// the mixed path)
void precondition64(Ctx& c, const double* in, double* out) {
  const int L = (int)c.dl.size();
  DevLevel& F = c.dl[L - 1];
  if (c.mixed) {
    precondition(c, in, nullptr, F.x32);
    launch_to_f64(F.Ni, F.x32, out, c.stream);
    counted(c);
  } else {
    precondition(c, in, out, nullptr);
  }
}

// ---------------------------------------------------------------------------
// GMRES(m), left preconditioned (Sec. 4.1): Arnoldi on P^{-1} J with
// classical Gram-Schmidt, x += V y, convergence when the left-preconditioned
// residual ||P^{-1}(b - J x_j)|| < rtol ||P^{-1}(b - J x_0)|| (the Givens
// estimate inside a cycle, the recomputed value at every restart)
// ---------------------------------------------------------------------------
void gmres_left(Ctx& c, const double* b, double* x, fsi_solve_stats* st) {
  const int L = (int)c.dl.size();
  DevLevel& F = c.dl[L - 1];
  const int64_t n = F.Ni;
  const int m = c.opts.restart;
  const int passes = c.opts.gs_passes > 0 ? c.opts.gs_passes : 1;
  double* sm = c.small;
  const double bnorm = dev_norm(c, n, b, sm + 300);
  if (!std::isfinite(bnorm)) throw ApiError(FSI_E_NONFINITE, "non-finite right-hand side");
  auto prec_residual = [&]() {   // c.w = P^{-1}(b - J x), returns its norm
    launch_bsr_residual(c.B, F.nb, F.rowptr, F.col, F.val, x, b, c.tmp, c.stream);
    counted(c);
    precondition64(c, c.tmp, c.w);
    return dev_norm(c, n, c.w, sm + 301);
  };
  double beta = prec_residual();
  const double r0 = beta;
  int iters = 0, restarts = 0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), yv(m), hcol(m + 1);
  auto Hc = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  while (r0 > 0.0) {
    if (!std::isfinite(beta)) throw ApiError(FSI_E_NONFINITE, "non-finite residual in GMRES");
    if (beta < c.opts.rtol * r0 || iters >= c.opts.max_iters) break;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    launch_scale_by(n, c.w, sm + 301, c.V, c.stream);
    counted(c);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      const double* vj = c.V + (size_t)j * n;
      spmv(c, L - 1, vj, nullptr, c.tmp, FSI_K_OPERATOR);     // t = J v_j (FP64)
      precondition64(c, c.tmp, c.w);          // w = P^{-1} t
      double hn = 0.0, wn0 = 0.0;
      orthonormalize(c, j, passes, hcol.data(), &hn, &wn0);
      if (!std::isfinite(hn)) throw ApiError(FSI_E_NONFINITE, "non-finite Krylov vector");
      for (int i = 0; i <= j; ++i) Hc(i, j) = hcol[i];
      Hc(j + 1, j) = hn;
      const bool breakdown = hn <= 1e-14 * wn0;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
        Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
        Hc(i, j) = t;
      }
      const double den = std::hypot(Hc(j, j), Hc(j + 1, j));
      cs[j] = Hc(j, j) / den;
      sn[j] = Hc(j + 1, j) / den;
      Hc(j, j) = den;
      Hc(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      k = j + 1;
      if (std::fabs(g[j + 1]) < c.opts.rtol * r0 || breakdown || iters >= c.opts.max_iters) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= Hc(i, q) * yv[q];
      yv[i] = s / Hc(i, i);
    }
    std::memcpy(c.host_small + 384, yv.data(), k * sizeof(double));
    ck(cudaMemcpyAsync(sm + 384, c.host_small + 384, k * sizeof(double), cudaMemcpyHostToDevice, c.stream), "H2D");
    launch_combo(n, c.V, n, k, sm + 384, x, c.stream);
    counted(c);
    beta = prec_residual();
    ++restarts;
  }
  // true residual of the result, for the statistics
  launch_bsr_residual(c.B, F.nb, F.rowptr, F.col, F.val, x, b, c.tmp, c.stream);
  counted(c);
  const double rt = dev_norm(c, n, c.tmp, sm + 302);
  const double prel = r0 > 0.0 ? beta / r0 : 0.0;
  if (st) {
    st->iters = iters;
    st->restarts = restarts;
    st->rel_res = bnorm > 0.0 ? rt / bnorm : 0.0;
    st->prec_rel_res = prel;
    st->rho = iters > 0 ? std::pow(prel, 1.0 / iters) : 0.0;
  }
  if (!(prel < c.opts.rtol) && r0 > 0.0) throw ApiError(FSI_E_NOT_CONVERGED, "GMRES reached max_iters");
}

// ---------------------------------------------------------------------------
// FGMRES(m), right preconditioned, CGS2, true residual at restart / exit
// ---------------------------------------------------------------------------
void fgmres(Ctx& c, const double* b, double* x, fsi_solve_stats* st) {
  const int L = (int)c.dl.size();
  DevLevel& F = c.dl[L - 1];
  const int64_t n = F.Ni;
  const int m = c.opts.restart;
  const int nb = nblk_red(c);
  double* sm = c.small;
  double* hs = c.host_small;
  const double bnorm = dev_norm(c, n, b, sm + 300);
  int iters = 0, restarts = 0;
  double rel = 0.0;
  if (!std::isfinite(bnorm)) throw ApiError(FSI_E_NONFINITE, "non-finite right-hand side");
  if (bnorm == 0.0) {
    if (st) { st->iters = 0; st->restarts = 0; st->rel_res = 0.0; st->prec_rel_res = 0.0; st->rho = 0.0; }
    return;
  }
  launch_bsr_residual(c.B, F.nb, F.rowptr, F.col, F.val, x, b, c.w, c.stream);
  counted(c);
  double beta = dev_norm(c, n, c.w, sm + 301);
  const int passes = c.opts.gs_passes > 0 ? c.opts.gs_passes : 2;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), yv(m), hcol(m + 1);
  auto Hc = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  while (true) {
    if (!std::isfinite(beta)) throw ApiError(FSI_E_NONFINITE, "non-finite residual in FGMRES");
    if (beta <= c.opts.rtol * bnorm || iters >= c.opts.max_iters) { rel = beta / bnorm; break; }
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    launch_scale_by(n, c.w, sm + 301, c.V, c.stream);
    counted(c);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = c.V + (size_t)j * n;
      if (c.mixed) {
        float* zj = c.Z32 + (size_t)j * n;
        precondition(c, vj, nullptr, zj);
        // A z_j in FP64: z_j widened once, not once per block that reads it
        // (each widening is an FP64-pipe instruction, about 80 per entry
        // inside the block sparse product)
        Prof pr(c, FSI_K_OPERATOR, F.spmv_bytes + n * 4.0, F.spmv_flops, 2);   // no b; + widening
        launch_to_f64(n, zj, c.zd, c.stream);
        launch_bsr_residual(c.B, F.nb, F.rowptr, F.col, F.val, c.zd, nullptr, c.w, c.stream);
        counted(c, 2);
      } else {
        double* zj = c.Z + (size_t)j * n;
        precondition(c, vj, zj, nullptr);
        spmv(c, L - 1, zj, nullptr, c.w, FSI_K_OPERATOR);
      }
      // CGS (two passes by default): h = V^T w, w -= V h per pass, v_{j+1} = w / ||w||
      double hn = 0.0, wn0 = 0.0;
      orthonormalize(c, j, passes, hcol.data(), &hn, &wn0);
      for (int i = 0; i <= j; ++i) Hc(i, j) = hcol[i];
      if (!std::isfinite(hn)) throw ApiError(FSI_E_NONFINITE, "non-finite Krylov vector");
      Hc(j + 1, j) = hn;
      const bool breakdown = hn <= 1e-14 * wn0;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
        Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
        Hc(i, j) = t;
      }
      const double den = std::hypot(Hc(j, j), Hc(j + 1, j));
      cs[j] = Hc(j, j) / den;
      sn[j] = Hc(j + 1, j) / den;
      Hc(j, j) = den;
      Hc(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      k = j + 1;
      if (std::fabs(g[j + 1]) <= c.opts.rtol * bnorm || breakdown || iters >= c.opts.max_iters) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= Hc(i, q) * yv[q];
      yv[i] = s / Hc(i, i);
    }
    std::memcpy(hs + 384, yv.data(), k * sizeof(double));
    ck(cudaMemcpyAsync(sm + 384, hs + 384, k * sizeof(double), cudaMemcpyHostToDevice, c.stream), "H2D");
    if (c.mixed) launch_combo_mixed(n, c.Z32, n, k, sm + 384, x, c.stream);
    else launch_combo(n, c.Z, n, k, sm + 384, x, c.stream);
    launch_bsr_residual(c.B, F.nb, F.rowptr, F.col, F.val, x, b, c.w, c.stream);
    counted(c, 2);
    beta = dev_norm(c, n, c.w, sm + 301);
    ++restarts;
    if (beta <= c.opts.rtol * bnorm || iters >= c.opts.max_iters) { rel = beta / bnorm; break; }
  }
  if (st) {
    st->iters = iters;
    st->restarts = restarts;
    st->rel_res = rel;
    st->prec_rel_res = rel;
    st->rho = iters > 0 ? std::pow(rel, 1.0 / iters) : 0.0;
  }
  if (!(rel <= c.opts.rtol)) throw ApiError(FSI_E_NOT_CONVERGED, "FGMRES reached max_iters");
}

void krylov_solve(Ctx& c, const double* b, double* x, fsi_solve_stats* st) {
  Nvtx nv(c.opts.krylov == FSI_GMRES_LEFT ? "fsi GMRES (left)" : "fsi FGMRES");
  const double b0 = c.alg_bytes;
  struct Tally {   // also when the solve ends with an error
    Ctx& c;
    double b0;
    ~Tally() { c.b_solve = c.alg_bytes - b0; }
  } tally{c, b0};
  if (c.opts.krylov == FSI_GMRES_LEFT) gmres_left(c, b, x, st);
  else fgmres(c, b, x, st);
}

float elapsed(Ctx& c) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c.ev0, c.ev1);
  return ms;
}

template <class F>
int guard(fsi_ctx* c, F&& f) {
  if (!c) return FSI_E_INVALID;
  try {
    f();
    return FSI_OK;
  } catch (const ApiError& e) {
    c->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return FSI_E_OOM;
  } catch (const std::exception& e) {
    c->err = e.what();
    return FSI_E_INVALID;
  }
}

void need_device(const Ctx& c) {
  if (c.dl.empty()) throw ApiError(FSI_E_INVALID, "ctx was planned without a device");
}

int check_level(const Ctx& c, int level, bool need_fine_side) {
  if (level < 0 || level >= (int)c.hl.size()) throw ApiError(FSI_E_INVALID, "level out of range");
  if (need_fine_side && level < 1) throw ApiError(FSI_E_INVALID, "level must be >= 1");
  return level;
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

// Device bytes fsi_build_hierarchy will allocate for this plan (same sizes as
// build_device), used for admission by device memory.
// largest element count of one colour / material group of the finest level
// elements of the largest launch_assemble_* call: all fluid or all solid
// elements of the finest level (the 3D flux scratch holds min(this, chunk))
static int max_assembly_batch(const Ctx& c) {
  const HostLevel& F = c.hl.back();
  return (int)std::max(F.n_fluid_elem, F.n_elem - F.n_fluid_elem);
}

static int64_t estimate_device_bytes(const Ctx& c) {
  const bool mixed = c.opts.precision == FSI_MIXED;
  const double fs = mixed ? 4.0 : 8.0;
  const int B = c.B, nd = c.ndofe, m = c.opts.restart;
  double b = 0.0, max_dense = 0.0;
  const size_t L = c.hl.size();
  for (size_t l = 0; l < L; ++l) {
    const HostLevel& H = c.hl[l];
    b += (H.nb + 1) * 4.0 + H.nnzb * 4.0 + H.nnzb * B * B * 8.0 + H.n_elem * (double)nd * nd * 8.0;
    b += H.n_elem * (H.nloc * 4.0 + 1.0 + 2.0 * H.dim * 8.0 + 4.0);
    b += (H.blk_ptr.size() + H.blk_src.size() + H.res_ptr.size() + H.res_src.size()) * 4.0;
    b += H.n_nodes + H.Ni * (1.0 + 8.0 + 4.0 + 4.0) + H.N * 4.0 + H.Ni * 3.0 * 8.0;
    if (l > 0) {
      b += (H.P_ptr.size() + H.R_ptr.size() + H.S_ptr.size()) * 4.0 +
           (H.P_col.size() + H.R_col.size() + H.S_col.size()) * 12.0;
      b += H.idx_total * 4.0 + H.own_total * 4.0 + H.n_patches * 9.0 * 8.0 + H.p_gmap.size() * 4.0 +
           H.p_padpos.size() * 4.0 + (H.p_boff.size() + H.p_gptr.size()) * 4.0 + H.inv_total * fs +
           2.0 * H.idx_total * fs;
      if (mixed) b += H.nnzb * B * B * 4.0 + (H.P_col.size() + H.R_col.size()) * 4.0 + H.Ni * 3.0 * 4.0;
      max_dense = std::max(max_dense, (double)H.dense_total);
    }
  }
  const HostLevel& F = c.hl.back();
  const double n0 = (double)c.hl[0].Ni;
  b += F.Ni * 8.0 * 2 + (m + 1.0) * F.Ni * 8.0 + m * (double)F.Ni * fs + F.Ni * 8.0 * 4 + F.N * 8.0 * 2;
  if (mixed) b += F.Ni * 8.0;   // the widened preconditioned vector
  if (c.desc.transient != 0) b += F.Ni * 8.0;
  if (c.dim == 3) b += (double)assemble_3d_scratch_doubles(max_assembly_batch(c)) * 8.0;
  double sum_dense = 0.0;
  for (size_t l = 1; l < L; ++l) sum_dense += (double)c.hl[l].dense_total;
  b += (mixed ? sum_dense : max_dense) * fs + F.n_elem * (double)nd * 8.0 + 1e6;
  const std::vector<int64_t>& so = c.hl[0].slab_off;
  if (c.dim == 3 && !so.empty()) {
    // dense banded-order operator + Sinv_k blocks + LU scratch + vectors
    double mm = 0.0, sum = 0.0;
    for (size_t k = 0; k + 1 < so.size(); ++k) {
      const double m = (double)(so[k + 1] - so[k]);
      mm = std::max(mm, m);
      sum += m * m;
    }
    b += n0 * n0 * 8.0 + (sum + mm * mm + c.hl[0].slab_p * mm + mm * mm / 32.0 + mm) * 8.0 + 6.0 * n0 * 8.0;
  } else {
    b += 2.0 * n0 * n0 * 8.0 + (n0 / 32.0 + 1.0) * n0 * 8.0 + 2.0 * n0 * 8.0;
  }
  return (int64_t)b;
}

static void plan(fsi_ctx* c, const fsi_problem_desc* desc, const fsi_solver_opts* opts) {
  if (desc->transient != 0 && !(desc->dt > 0.0)) throw ApiError(FSI_E_INVALID, "transient problem needs dt > 0");
  if (desc->transient < 0 || desc->transient > 2) throw ApiError(FSI_E_INVALID, "transient must be 0, 1 or 2");
  if (opts->precision != FSI_FP64 && opts->precision != FSI_MIXED) throw ApiError(FSI_E_INVALID, "bad precision");
  if (opts->restart < 1 || opts->restart > 64) throw ApiError(FSI_E_INVALID, "restart must be in [1, 64]");
  if (opts->n_pre < 0 || opts->n_post < 0 || opts->max_iters < 1 || !(opts->rtol > 0.0))
    throw ApiError(FSI_E_INVALID, "bad solver options");
  if ((opts->krylov != FSI_FGMRES && opts->krylov != FSI_GMRES_LEFT) || opts->gs_passes < 0 || opts->gs_passes > 2)
    throw ApiError(FSI_E_INVALID, "bad Krylov options (krylov 0 or 1, gs_passes 0..2)");
  if (opts->local_solver != 0 && opts->local_solver != 1)
    throw ApiError(FSI_E_INVALID, "local_solver must be 0 (LU) or 1 (ILU(0) for fluid blocks)");
  if (opts->local_solver == 1 && opts->precision != FSI_MIXED)
    throw ApiError(FSI_E_INVALID, "ILU(0) fluid blocks are built on the mixed-precision path");
  std::string err;
  if (!build_host_hierarchy(*desc, *opts, c->hl, err)) throw ApiError(FSI_E_INVALID, err);
  c->dim = desc->dim;
  c->B = 2 * desc->dim;
  c->nloc = desc->dim == 2 ? 9 : 27;
  c->ndofe = c->B * c->nloc + desc->dim + 1;
  c->est_bytes = estimate_device_bytes(*c);
}

int fsi_plan_hierarchy(const fsi_problem_desc* desc, const fsi_solver_opts* opts, fsi_ctx** out) {
  if (!desc || !opts || !out) return FSI_E_INVALID;
  *out = nullptr;
  fsi_ctx* c = new (std::nothrow) fsi_ctx();
  if (!c) return FSI_E_OOM;
  c->desc = *desc;
  c->opts = *opts;
  int rc = guard(c, [&] { plan(c, desc, opts); });
  if (rc != FSI_OK) {
    std::fprintf(stderr, "fsi_plan_hierarchy: %s\n", c->err.c_str());
    delete c;
    return rc;
  }
  *out = c;
  return FSI_OK;
}

int fsi_build_hierarchy(const fsi_problem_desc* desc, const fsi_solver_opts* opts, void* stream, fsi_ctx** out) {
  if (!desc || !opts || !out) return FSI_E_INVALID;
  *out = nullptr;
  fsi_ctx* c = new (std::nothrow) fsi_ctx();
  if (!c) return FSI_E_OOM;
  c->desc = *desc;
  c->opts = *opts;
  c->stream = static_cast<cudaStream_t>(stream);
  int rc = guard(c, [&] {
    plan(c, desc, opts);
    c->mixed = opts->precision == FSI_MIXED;
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    c->device = dev;
    ck(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev), "attr");
    int coop = 0;
    ck(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "attr");
    if (!coop) throw ApiError(FSI_E_CUDA, "device lacks cooperative launch");
    build_device(*c);
    c->tmp_re = dalloc<double>(*c, (size_t)c->hl.back().n_elem * c->ndofe);
    if (c->dim == 3) {
      c->asm_scratch_ne = max_assembly_batch(*c);
      c->asm_scratch = dalloc<double>(*c, assemble_3d_scratch_doubles(c->asm_scratch_ne));
    }
    std::vector<int32_t> pads = coarse_pads(*c);
    c->coarse_pad_list = upload(*c, pads);
    c->n_coarse_pads = (int)pads.size();
    sync(*c);
  });
  if (rc != FSI_OK) {
    std::fprintf(stderr, "fsi_build_hierarchy: %s\n", c->err.c_str());
    fsi_destroy(c);
    return rc;
  }
  *out = c;
  return FSI_OK;
}

void fsi_destroy(fsi_ctx* c) {
  if (!c) return;
  if (c->dl.empty() && c->allocs.empty()) {   // planned ctx: no CUDA state
    delete c;
    return;
  }
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  if (c->host_small) cudaFreeHost(c->host_small);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (auto& ks : c->kstat)
    for (auto& pr : ks.pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  if (c->vc_exec) cudaGraphExecDestroy(c->vc_exec);
  if (c->vc_graph) cudaGraphDestroy(c->vc_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  cudaGetLastError();
  delete c;
}

const char* fsi_last_error(const fsi_ctx* c) { return c ? c->err.c_str() : "null ctx"; }

int64_t fsi_launch_count(const fsi_ctx* c) { return c ? c->launches : 0; }

int fsi_get_sizes(const fsi_ctx* c, int64_t* n_per_level, int64_t* nnz_per_level, int64_t* hbm_bytes) {
  if (!c) return FSI_E_INVALID;
  for (size_t l = 0; l < c->hl.size(); ++l) {
    const HostLevel& H = c->hl[l];
    if (n_per_level) n_per_level[l] = H.N;
    if (nnz_per_level) {
      int64_t nnz = 0;
      const int np = H.dim + 1;
      for (int64_t br = 0; br < H.nb; ++br) {
        const int rows = br < H.n_nodes ? H.B : np;
        for (int32_t k = H.rowptr[br]; k < H.rowptr[br + 1]; ++k) nnz += (int64_t)rows * (H.col[k] < H.n_nodes ? H.B : np);
      }
      nnz_per_level[l] = nnz;
    }
  }
  if (hbm_bytes) *hbm_bytes = c->dl.empty() ? c->est_bytes : c->bytes;
  return FSI_OK;
}

int fsi_initial_state(fsi_ctx* c, const double* noise, double* y_out) {
  return guard(c, [&] {
    // a host computation: also answers on a planned ctx (host buffers)
    if (!noise || !y_out) throw ApiError(FSI_E_INVALID, "null pointer");
    const HostLevel& H = c->hl.back();
    std::vector<double> nz(H.N), y(H.N, 0.0);
    const bool dev_in = is_device_ptr(noise), dev_out = is_device_ptr(y_out);
    if (dev_in) ck(cudaMemcpy(nz.data(), noise, H.N * sizeof(double), cudaMemcpyDeviceToHost), "copy noise");
    else std::memcpy(nz.data(), noise, H.N * sizeof(double));
    const int dim = H.dim, B = H.B;
    const double Hy = c->desc.breaks[1][c->desc.n_breaks[1] - 1];
    const double Hz = dim == 3 ? c->desc.breaks[2][c->desc.n_breaks[2] - 1] : 1.0;
    for (int64_t n = 0; n < H.n_nodes; ++n) {
      if (H.node_class[n] != kFluid) continue;
      const int iy = (int)((n / H.nodes_ax[0]) % H.nodes_ax[1]);
      const int iz = dim == 3 ? (int)(n / ((int64_t)H.nodes_ax[0] * H.nodes_ax[1])) : 0;
      const double yy = iy % 2 == 0 ? H.verts[1][iy / 2] : (H.verts[1][iy / 2] + H.verts[1][iy / 2 + 1]) / 2.0;
      double v;
      if (dim == 2) {
        v = 1.5 * c->desc.U * yy * (Hy - yy) / ((Hy / 2.0) * (Hy / 2.0));
      } else {
        const double zz = iz % 2 == 0 ? H.verts[2][iz / 2] : (H.verts[2][iz / 2] + H.verts[2][iz / 2 + 1]) / 2.0;
        v = 36.0 * c->desc.U * yy * (Hy - yy) * zz * (Hz - zz) / (Hy * Hy * Hz * Hz);
      }
      y[n * B + dim] = v;
    }
    for (int64_t i = 0; i < H.Ni; ++i) {
      const int32_t cidx = H.canon_of_int[i];
      if (cidx < 0) continue;
      if (H.dir[i]) y[cidx] = H.dir_val[i];
      else if (i < H.n_nodes * B && (i % B) < dim) y[cidx] += nz[cidx];
    }
    if (dev_out) ck(cudaMemcpy(y_out, y.data(), H.N * sizeof(double), cudaMemcpyHostToDevice), "copy state");
    else std::memcpy(y_out, y.data(), H.N * sizeof(double));
  });
}

int fsi_set_state(fsi_ctx* c, const double* y, const double* y_prev, const double* y_prev2, double t) {
  return guard(c, [&] {
    need_device(*c);
    if (!y) throw ApiError(FSI_E_INVALID, "null state");
    const int L = (int)c->dl.size();
    to_internal(*c, L - 1, y, c->y);
    if (c->desc.transient == 2) {
      // Crank-Nicolson: the state of t_n itself
      if (!y_prev) throw ApiError(FSI_E_INVALID, "transient problem: y_prev is required");
      to_internal(*c, L - 1, y_prev, c->yold);
      c->inflow_alpha = 0.5 * (1.0 + std::sin(2.0 * M_PI * t));
      c->have_history = true;
    } else if (c->desc.transient != 0) {
      if (!y_prev) throw ApiError(FSI_E_INVALID, "transient problem: y_prev is required");
      // BDF2 with two history states, BDF1 (start-up step) with one
      const double a0 = y_prev2 ? 1.5 : 1.0, a1 = y_prev2 ? -2.0 : -1.0, a2 = 0.5;
      const int64_t Ni = c->dl[L - 1].Ni;
      to_internal(*c, L - 1, y_prev, c->tmp);
      launch_axpby(Ni, a1, c->tmp, 0.0, c->yold, c->stream);
      counted(*c);
      if (y_prev2) {
        to_internal(*c, L - 1, y_prev2, c->tmp);
        launch_axpby(Ni, a2, c->tmp, 1.0, c->yold, c->stream);
        counted(*c);
      }
      c->bdf_a0 = a0;
      c->inflow_alpha = 0.5 * (1.0 + std::sin(2.0 * M_PI * t));
      c->have_history = true;
    }
    sync(*c);
  });
}

int fsi_get_state(fsi_ctx* c, double* y_out) {
  return guard(c, [&] {
    need_device(*c);
    if (!y_out) throw ApiError(FSI_E_INVALID, "null pointer");
    to_canonical(*c, (int)c->dl.size() - 1, c->y, y_out);
    sync(*c);
  });
}

int fsi_assemble_jacobian(fsi_ctx* c, double* residual_out) {
  return guard(c, [&] {
    need_device(*c);
    ck(cudaEventRecord(c->ev0, c->stream), "event");
    assemble(*c, residual_out != nullptr);
    ck(cudaEventRecord(c->ev1, c->stream), "event");
    if (residual_out) to_canonical(*c, (int)c->dl.size() - 1, c->res, residual_out);
    sync(*c);
    c->t_assemble = elapsed(*c);
  });
}

int fsi_factor_schwarz(fsi_ctx* c) {
  return guard(c, [&] {
    need_device(*c);
    ck(cudaEventRecord(c->ev0, c->stream), "event");
    factor(*c);
    ck(cudaEventRecord(c->ev1, c->stream), "event");
    sync(*c);
    c->t_factor = elapsed(*c);
  });
}

int fsi_solve(fsi_ctx* c, const double* b, double* x, fsi_solve_stats* st) {
  return guard(c, [&] {
    need_device(*c);
    if (!b || !x) throw ApiError(FSI_E_INVALID, "null pointer");
    const int L = (int)c->dl.size();
    to_internal(*c, L - 1, b, c->bk);
    to_internal(*c, L - 1, x, c->xk);
    ck(cudaEventRecord(c->ev0, c->stream), "event");
    int rc = FSI_OK;
    std::string msg;
    try {
      krylov_solve(*c, c->bk, c->xk, st);
    } catch (const ApiError& e) {
      if (e.code != FSI_E_NOT_CONVERGED) throw;
      rc = e.code;
      msg = e.what();
    }
    ck(cudaEventRecord(c->ev1, c->stream), "event");
    to_canonical(*c, L - 1, c->xk, x);
    sync(*c);
    c->t_solve = elapsed(*c);
    if (st) {
      st->t_assemble_ms = c->t_assemble; st->t_factor_ms = c->t_factor; st->t_solve_ms = c->t_solve;
      st->bytes_assemble = c->b_assemble; st->bytes_factor = c->b_factor; st->bytes_solve = c->b_solve;
    }
    if (rc != FSI_OK) throw ApiError(rc, msg);
  });
}

int fsi_newton_update(fsi_ctx* c, const double* dx, double* rel_step_out) {
  return guard(c, [&] {
    need_device(*c);
    if (!dx) throw ApiError(FSI_E_INVALID, "null pointer");
    const int L = (int)c->dl.size();
    const int64_t n = c->dl[L - 1].Ni;
    to_internal(*c, L - 1, dx, c->tmp);
    launch_axpby(n, 1.0, c->tmp, 1.0, c->y, c->stream);
    counted(*c);
    const double dn = dev_norm(*c, n, c->tmp, c->small + 310);
    const double yn = dev_norm(*c, n, c->y, c->small + 311);
    if (!std::isfinite(dn) || !std::isfinite(yn)) throw ApiError(FSI_E_NONFINITE, "non-finite Newton update");
    if (rel_step_out) *rel_step_out = yn > 0 ? dn / yn : dn;
  });
}

namespace {
// Second half of a Newton step: solve J dx = -r with the current factors and
// the residual of the last assembly, then y += dx.
void solve_update(Ctx* c, double* dx_out, double* rel_step_out, fsi_solve_stats* st);
}  // namespace

int fsi_newton_step(fsi_ctx* c, double* dx_out, double* rel_step_out, fsi_solve_stats* st) {
  return guard(c, [&] {
    need_device(*c);
    ck(cudaEventRecord(c->ev0, c->stream), "event");
    assemble(*c, true);
    ck(cudaEventRecord(c->ev1, c->stream), "event");
    sync(*c);
    c->t_assemble = elapsed(*c);
    ck(cudaEventRecord(c->ev0, c->stream), "event");
    factor(*c);
    ck(cudaEventRecord(c->ev1, c->stream), "event");
    sync(*c);
    c->t_factor = elapsed(*c);
    solve_update(c, dx_out, rel_step_out, st);
  });
}

int fsi_newton_solve_update(fsi_ctx* c, double* dx_out, double* rel_step_out, fsi_solve_stats* st) {
  return guard(c, [&] {
    need_device(*c);
    if (!c->factored) throw ApiError(FSI_E_INVALID, "fsi_newton_solve_update: assemble and factor first");
    solve_update(c, dx_out, rel_step_out, st);
  });
}

int fsi_factor_schwarz_batch(fsi_ctx* const* ctxs, int n) {
  if (!ctxs || n < 1) return FSI_E_INVALID;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return FSI_E_INVALID;
  fsi_ctx* c0 = ctxs[0];
  return guard(c0, [&] {
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctxs[i];
      need_device(c);
      if (!c.mixed || c.dl.size() < 2)
        throw ApiError(FSI_E_INVALID, "batched factorisation: mixed-precision instances with >= 2 levels only");
      if (c.stream != c0->stream || c.device != c0->device)
        throw ApiError(FSI_E_INVALID, "batched factorisation: every instance on the same stream and device");
      if (c.prof) throw ApiError(FSI_E_INVALID, "batched factorisation: per-class profiling is on");
      for (int j = 0; j < i; ++j)
        if (ctxs[j] == ctxs[i]) throw ApiError(FSI_E_INVALID, "batched factorisation: an instance appears twice");
    }
    const cudaStream_t st = c0->stream;
    ck(cudaEventRecord(c0->ev0, st), "event");
    // coarse factorisations on each instance's private stream, forked from the common stream
    std::vector<bool> forked(n, false);
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctxs[i];
      if (!aux_stream(c)) continue;
      cudaEventRecord(c.ev_fork, st);
      cudaStreamWaitEvent(c.aux_stream, c.ev_fork, 0);
      {
        StreamSwap sw(c, c.aux_stream);
        coarse_factor(c);
      }
      cudaEventRecord(c.ev_join, c.aux_stream);
      forked[i] = true;
    }
    // instances grouped by the tensor-core variant each would use alone, so
    // every block is factored exactly as in its own fsi_factor_schwarz
    std::vector<int> variant(n);
    for (int i = 0; i < n; ++i)
      variant[i] = ctxs[i]->opts.local_solver == 1 ? 0 : gj_tc_variant(max_block(*ctxs[i]), ctxs[i]->gj_panel);
    std::vector<bool> done(n, false);
    for (int i = 0; i < n; ++i) {
      if (done[i]) continue;
      if (variant[i] == 0) {   // no tensor-core variant fits: the instance's own path
        schwarz_factor(*ctxs[i]);
        done[i] = true;
        continue;
      }
      GjLevels lv{};
      lv.nlev = 0;
      lv.first_wait = kTcWaitIters;
      int first = 0, max_n = 0;
      for (int j = i; j < n; ++j) {
        if (done[j] || variant[j] != variant[i]) continue;
        Ctx& c = *ctxs[j];
        if (lv.nlev + (int)c.dl.size() - 1 > kGjMaxLevels) continue;   // next launch
        GjLevels one = lv;
        int f1 = first, m1 = max_n;
        if (!gather_mixed(c, one, f1, m1)) {   // a level without blocks: its own path
          schwarz_factor(c);
          done[j] = true;
          continue;
        }
        lv = one;
        first = f1;
        max_n = m1;
        done[j] = true;
      }
      if (lv.nlev > 0) {
        if (!launch_patch_gj_tc_levels(lv, first, max_n, c0->status, st, variant[i]))
          throw ApiError(FSI_E_CUDA, "batched factorisation: tensor-core launch refused");
        counted(*c0);
      }
    }
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctxs[i];
      if (forked[i]) cudaStreamWaitEvent(st, c.ev_join, 0);
      else coarse_factor(c);
    }
    ck(cudaEventRecord(c0->ev1, st), "event");
    sync(*c0);
    const float ms = elapsed(*c0);
    for (int i = 0; i < n; ++i) {
      Ctx& c = *ctxs[i];
      check_status(c);
      c.factored = true;
      c.t_factor = ms;
      double by = 0.0;   // the Schwarz gathers and inverses (the coarse LU is in the level-0 estimate)
      for (size_t l = 1; l < c.dl.size(); ++l) by += c.dl[l].factor_bytes;
      c.b_factor = by + (double)c.dl[0].Ni * c.dl[0].Ni * 8.0 * 3.0;
    }
  });
}

namespace {
void solve_update(Ctx* c, double* dx_out, double* rel_step_out, fsi_solve_stats* st) {
    const int L = (int)c->dl.size();
    const int64_t n = c->dl[L - 1].Ni;
    launch_axpby(n, -1.0, c->res, 0.0, c->bk, c->stream);
    ck(cudaMemsetAsync(c->xk, 0, n * sizeof(double), c->stream), "memset");
    counted(*c);
    ck(cudaEventRecord(c->ev0, c->stream), "event");
    krylov_solve(*c, c->bk, c->xk, st);
    ck(cudaEventRecord(c->ev1, c->stream), "event");
    sync(*c);
    c->t_solve = elapsed(*c);
    launch_axpby(n, 1.0, c->xk, 1.0, c->y, c->stream);
    counted(*c);
    const double dn = dev_norm(*c, n, c->xk, c->small + 310);
    const double yn = dev_norm(*c, n, c->y, c->small + 311);
    if (rel_step_out) *rel_step_out = yn > 0 ? dn / yn : dn;
    if (dx_out) to_canonical(*c, L - 1, c->xk, dx_out);
    sync(*c);
    if (st) {
      st->t_assemble_ms = c->t_assemble; st->t_factor_ms = c->t_factor; st->t_solve_ms = c->t_solve;
      st->bytes_assemble = c->b_assemble; st->bytes_factor = c->b_factor; st->bytes_solve = c->b_solve;
    }
}
}  // namespace

int fsi_export_csr(fsi_ctx* c, int level, int64_t* rowptr, int32_t* col, double* val) {
  return guard(c, [&] {
    check_level(*c, level, false);
    if (!rowptr) throw ApiError(FSI_E_INVALID, "null rowptr");
    const HostLevel& H = c->hl[level];
    const int B = H.B, np = H.dim + 1;
    std::vector<double> v;
    if (val) {
      need_device(*c);
      v.resize((size_t)H.nnzb * B * B);
      ck(cudaMemcpy(v.data(), c->dl[level].val, v.size() * sizeof(double), cudaMemcpyDeviceToHost), "D2H");
    }
    // canonical rows in order: node rows (internal order), then pressure rows
    int64_t pos = 0;
    int64_t crow = 0;
    rowptr[0] = 0;
    for (int64_t br = 0; br < H.nb; ++br) {
      const int rows = br < H.n_nodes ? B : np;
      for (int ci = 0; ci < rows; ++ci) {
        for (int32_t k = H.rowptr[br]; k < H.rowptr[br + 1]; ++k) {
          const int64_t bc = H.col[k];
          const int cols = bc < H.n_nodes ? B : np;
          for (int cj = 0; cj < cols; ++cj) {
            if (col) col[pos] = H.canon_of_int[bc * B + cj];
            if (val) val[pos] = v[(size_t)k * B * B + ci * B + cj];
            ++pos;
          }
        }
        rowptr[++crow] = pos;
      }
    }
  });
}

int fsi_export_dofmap(fsi_ctx* c, int level, uint8_t* node_class, uint8_t* elem_solid, uint8_t* dirichlet,
                      double* dir_val) {
  return guard(c, [&] {
    check_level(*c, level, false);
    const HostLevel& H = c->hl[level];
    if (node_class) std::memcpy(node_class, H.node_class.data(), H.n_nodes);
    if (elem_solid) std::memcpy(elem_solid, H.elem_solid.data(), H.n_elem);
    for (int64_t i = 0; i < H.Ni; ++i) {
      const int32_t ci = H.canon_of_int[i];
      if (ci < 0) continue;
      if (dirichlet) dirichlet[ci] = H.dir[i];
      if (dir_val) dir_val[ci] = H.dir_val[i];
    }
  });
}

int fsi_export_patches(fsi_ctx* c, int level, int* n_patches, int64_t* total_len, int64_t* ptr, int32_t* dofs,
                       uint8_t* owned) {
  return guard(c, [&] {
    check_level(*c, level, true);
    const HostLevel& H = c->hl[level];
    if (n_patches) *n_patches = H.n_patches;
    std::vector<uint8_t> own_flag(H.idx_total, 0);
    for (int p = 0; p < H.n_patches; ++p)
      for (int64_t o = H.p_own_off[p]; o < H.p_own_off[p + 1]; ++o) own_flag[H.p_idx_off[p] + H.p_own[o]] = 1;
    int64_t tot = 0;
    for (int64_t i = 0; i < H.idx_total; ++i)
      if (H.canon_of_int[H.p_idx[i]] >= 0) ++tot;
    if (total_len) *total_len = tot;
    if (!ptr) return;
    int64_t pos = 0;
    ptr[0] = 0;
    for (int p = 0; p < H.n_patches; ++p) {
      for (int64_t i = H.p_idx_off[p]; i < H.p_idx_off[p + 1]; ++i) {
        const int32_t ci = H.canon_of_int[H.p_idx[i]];
        if (ci < 0) continue;
        if (dofs) dofs[pos] = ci;
        if (owned) owned[pos] = own_flag[i];
        ++pos;
      }
      ptr[p + 1] = pos;
    }
  });
}

int fsi_export_transfer(fsi_ctx* c, int level, int which, int64_t* nnz, int64_t* rowptr, int32_t* col, double* val) {
  return guard(c, [&] {
    check_level(*c, level, true);
    if (which != 0 && which != 1) throw ApiError(FSI_E_INVALID, "which must be 0 (P) or 1 (R)");
    const HostLevel& F = c->hl[level];
    const HostLevel& C = c->hl[level - 1];
    const HostLevel& Rw = which == 0 ? F : C;     // row level
    const HostLevel& Cl = which == 0 ? C : F;     // column level
    const std::vector<int32_t>& ptr = which == 0 ? F.P_ptr : F.R_ptr;
    const std::vector<int32_t>& cols = which == 0 ? F.P_col : F.R_col;
    const std::vector<double>& vals = which == 0 ? F.P_val : F.R_val;
    if (nnz) *nnz = (int64_t)cols.size();
    if (!rowptr) return;
    // canonical row order: internal rows that map to canonical rows, ascending canonical index
    std::vector<int64_t> order(Rw.N, -1);
    for (int64_t i = 0; i < Rw.Ni; ++i)
      if (Rw.canon_of_int[i] >= 0) order[Rw.canon_of_int[i]] = i;
    int64_t pos = 0;
    rowptr[0] = 0;
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t r = 0; r < Rw.N; ++r) {
      const int64_t i = order[r];
      row.clear();
      for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) row.push_back({Cl.canon_of_int[cols[k]], vals[k]});
      std::sort(row.begin(), row.end());
      for (auto& e : row) {
        if (col) col[pos] = e.first;
        if (val) val[pos] = e.second;
        ++pos;
      }
      rowptr[r + 1] = pos;
    }
  });
}

int fsi_import_csr(fsi_ctx* c, int level, const double* val) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, false);
    if (!val) throw ApiError(FSI_E_INVALID, "null values");
    const HostLevel& H = c->hl[level];
    DevLevel& D = c->dl[level];
    const int B = H.B, np = H.dim + 1;
    // BSR storage of the level, padding entries zero; canonical CSR order as
    // in fsi_export_csr
    std::vector<double> v((size_t)H.nnzb * B * B, 0.0);
    int64_t pos = 0;
    for (int64_t br = 0; br < H.nb; ++br) {
      const int rows = br < H.n_nodes ? B : np;
      for (int ci = 0; ci < rows; ++ci)
        for (int32_t k = H.rowptr[br]; k < H.rowptr[br + 1]; ++k) {
          const int cols = H.col[k] < H.n_nodes ? B : np;
          for (int cj = 0; cj < cols; ++cj) v[(size_t)k * B * B + ci * B + cj] = val[pos++];
        }
    }
    ck(cudaMemcpyAsync(D.val, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D");
    if (c->mixed && level >= 1) {
      launch_to_f32((int64_t)v.size(), D.val, D.val32, c->stream);
      counted(*c);
    }
    sync(*c);
  });
}

int fsi_set_tc_wait_limit(fsi_ctx* c, long long iters) {
  return guard(c, [&] {
    need_device(*c);
    c->tc_first_wait = iters < 0 ? -1 : iters;
  });
}

int fsi_set_stream(fsi_ctx* c, void* stream) {
  return guard(c, [&] {
    need_device(*c);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (s == c->stream) return;
    sync(*c);   // nothing of the ctx is in flight on the old stream
    c->stream = s;
  });
}

int fsi_apply_operator(fsi_ctx* c, int level, const double* x, double* y) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, false);
    DevLevel& D = c->dl[level];
    to_internal(*c, level, x, D.x);
    launch_bsr_residual(c->B, D.nb, D.rowptr, D.col, D.val, D.x, nullptr, D.r, c->stream);
    counted(*c);
    to_canonical(*c, level, D.r, y);
    sync(*c);
  });
}

int fsi_apply_vcycle(fsi_ctx* c, const double* b, double* z) {
  return guard(c, [&] {
    need_device(*c);
    const int L = (int)c->dl.size();
    to_internal(*c, L - 1, b, c->bk);
    if (c->mixed) {
      DevLevel& F = c->dl[L - 1];
      precondition(*c, c->bk, nullptr, F.x32);
      launch_to_f64(F.Ni, F.x32, c->xk, c->stream);
      counted(*c);
    } else {
      precondition(*c, c->bk, c->xk, nullptr);
    }
    to_canonical(*c, L - 1, c->xk, z);
    sync(*c);
  });
}

// ---------------------------------------------------------------------------
// nested iteration (full multigrid) for the steady problem
// ---------------------------------------------------------------------------
namespace {
__global__ void k_set_dirichlet(const int32_t* __restrict__ list, int64_t n, const double* __restrict__ val,
                                double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[list[i]] = val[list[i]];
}
}  // namespace

int fsi_fmg_newton(const fsi_problem_desc* desc, const fsi_solver_opts* opts, void* stream, double tol,
                   int max_steps, double* y_out, fsi_fmg_stats* stats) {
  if (!desc || !opts || !y_out || desc->levels < 1 || desc->levels > FSI_FMG_MAX_LEVELS || !(tol > 0.0) ||
      max_steps < 1 || desc->transient != 0)
    return FSI_E_INVALID;
  fsi_fmg_stats st{};
  st.levels = desc->levels;
  fsi_ctx* prev = nullptr;
  int rc = FSI_OK;
  const cudaStream_t cs = static_cast<cudaStream_t>(stream);
  for (int l = 1; l <= desc->levels && rc == FSI_OK; ++l) {
    fsi_problem_desc dl = *desc;
    dl.levels = l;
    fsi_ctx* c = nullptr;
    rc = fsi_build_hierarchy(&dl, opts, stream, &c);
    if (rc != FSI_OK) break;
    rc = guard(c, [&] {
      DevLevel& F = c->dl.back();
      if (!prev) {
        // boundary-condition lift: fsi_initial_state without noise
        const int64_t N = c->hl.back().N;
        std::vector<double> zero(N, 0.0), y(N);
        const int r0 = fsi_initial_state(c, zero.data(), y.data());
        if (r0 != FSI_OK) throw ApiError(r0, c->err);
        const int r1 = fsi_set_state(c, y.data(), nullptr, nullptr, 0.0);
        if (r1 != FSI_OK) throw ApiError(r1, c->err);
      } else {
        // the coarser solution injected (every unknown, boundary values
        // included), then the Dirichlet data
        launch_csr_spmv(F.Ni, F.S_ptr, F.S_col, F.S_val, prev->y, c->y, false, cs);
        counted(*c);
        if (F.n_dir > 0) {
          k_set_dirichlet<<<(unsigned)((F.n_dir + 255) / 256), 256, 0, cs>>>(F.dir_list, F.n_dir, F.dir_val, c->y);
          counted(*c);
        }
        sync(*c);
      }
    });
    if (prev) {
      fsi_destroy(prev);
      prev = nullptr;
    }
    prev = c;
    if (rc != FSI_OK) break;
    const int li = l - 1;
    for (int k = 0; k < max_steps; ++k) {
      fsi_solve_stats s{};
      double rel = 0.0;
      rc = fsi_newton_step(c, nullptr, &rel, &s);
      if (rc != FSI_OK) break;
      st.newton_steps[li] += 1;
      st.krylov_iters[li] += s.iters;
      st.last_rel_step[li] = rel;
      st.ms[li] += s.t_assemble_ms + s.t_factor_ms + s.t_solve_ms;
      if (rel < tol) break;
    }
    if (rc == FSI_OK && !(st.last_rel_step[li] < tol)) rc = FSI_E_NOT_CONVERGED;
  }
  if (prev) {
    const int rg = fsi_get_state(prev, y_out);
    if (rc == FSI_OK) rc = rg;
    if (rc != FSI_OK) std::fprintf(stderr, "fsi_fmg_newton: %s\n", prev->err.c_str());
    fsi_destroy(prev);
  }
  st.status = rc;
  if (stats) *stats = st;
  return rc;
}

// ---------------------------------------------------------------------------
// coarse solve with file-scope scratch (allocates nothing)
// ---------------------------------------------------------------------------
// GEMV partial sums of fsi_coarse_solve_static.  Shared by every instance on
// a device; the first GEMV stage writes every partial the second stage
// reads, so nothing in it has to start at zero.
static __device__ __align__(256) double g_coarse_part[FSI_STATIC_PART_MAX];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_part_mu;
double* g_part_addr[kMaxDevices] = {};

// device address of g_coarse_part, resolved once per device
double* static_part(int dev) {
  if (dev < 0 || dev >= kMaxDevices) throw ApiError(FSI_E_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_part_mu);
  if (!g_part_addr[dev]) {
    void* p = nullptr;
    ck(cudaGetSymbolAddress(&p, g_coarse_part), "cudaGetSymbolAddress");
    g_part_addr[dev] = static_cast<double*>(p);
  }
  return g_part_addr[dev];
}
}  // namespace

int fsi_coarse_solve_static(fsi_ctx* c, const double* b, double* x) {
  return guard(c, [&] {
    need_device(*c);
    if (!b || !x) throw ApiError(FSI_E_INVALID, "null pointer");
    if (c->coarse_slab)
      throw ApiError(FSI_E_INVALID, "fsi_coarse_solve_static: the slab-blocked (3D) coarse LU is not supported");
    DevLevel& C = c->dl[0];
    const int64_t n0 = C.Ni;
    const int64_t need = ((n0 + 31) / 32) * n0;
    if (need > FSI_STATIC_PART_MAX)
      throw ApiError(FSI_E_INVALID, "fsi_coarse_solve_static: level-0 internal length " + std::to_string(n0) +
                                        " exceeds the static scratch limit of " + std::to_string(FSI_STATIC_COARSE_MAX));
    if (!c->factored) throw ApiError(FSI_E_INVALID, "fsi_coarse_solve_static: fsi_factor_schwarz first");
    // the array's address is per device: it must be the one the ctx (and its
    // stream) lives on, which must also be the calling thread's current device
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != c->device)
      throw ApiError(FSI_E_INVALID, "fsi_coarse_solve_static: the current device (" + std::to_string(dev) +
                                        ") is not the device the ctx was built on (" + std::to_string(c->device) + ")");
    double* part = static_part(dev);
    to_internal(*c, 0, b, C.b);
    launch_gemv(n0, c->c_inv, C.b, C.x, part, c->stream);
    counted(*c, 2);
    to_canonical(*c, 0, C.x, x);
    sync(*c);
  });
}

int fsi_apply_smoother(fsi_ctx* c, int level, const double* b, const double* x, double* x_out) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, true);
    DevLevel& D = c->dl[level];
    to_internal(*c, level, b, D.b);
    to_internal(*c, level, x, D.x);
    if (c->mixed) {
      launch_to_f32(D.Ni, D.b, D.b32, c->stream);
      launch_to_f32(D.Ni, D.x, D.x32, c->stream);
      smooth_step_t<float>(*c, level, D.b32, D.x32, false);
      launch_to_f64(D.Ni, D.x32, D.x, c->stream);
      counted(*c, 3);
    } else {
      smooth_step_t<double>(*c, level, D.b, D.x, false);
    }
    to_canonical(*c, level, D.x, x_out);
    sync(*c);
  });
}

int fsi_restrict(fsi_ctx* c, int level, const double* fine, double* coarse) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, true);
    DevLevel& D = c->dl[level];
    DevLevel& C = c->dl[level - 1];
    to_internal(*c, level, fine, D.r);
    launch_csr_spmv(C.Ni, D.R_ptr, D.R_col, D.R_val, D.r, C.b, false, c->stream);
    counted(*c);
    to_canonical(*c, level - 1, C.b, coarse);
    sync(*c);
  });
}

int fsi_prolong(fsi_ctx* c, int level, const double* coarse, double* fine) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, true);
    DevLevel& D = c->dl[level];
    DevLevel& C = c->dl[level - 1];
    to_internal(*c, level - 1, coarse, C.x);
    launch_csr_spmv(D.Ni, D.P_ptr, D.P_col, D.P_val, C.x, D.r, false, c->stream);
    counted(*c);
    to_canonical(*c, level, D.r, fine);
    sync(*c);
  });
}

int fsi_set_profiling(fsi_ctx* c, int on) {
  return guard(c, [&] {
    need_device(*c);
    harvest(*c);
    for (auto& ks : c->kstat) {
      ks.ms = ks.bytes = ks.flops = 0.0;
      ks.launches = 0;
    }
    c->prof = on != 0;
  });
}

// ---------------------------------------------------------------------------
// launch parameters (autotuner)
// ---------------------------------------------------------------------------
static void drop_vcycle_graph(Ctx& c) {
  if (c.vc_exec) cudaGraphExecDestroy(c.vc_exec);
  if (c.vc_graph) cudaGraphDestroy(c.vc_graph);
  c.vc_exec = nullptr;
  c.vc_graph = nullptr;
  c.vc_graph_failed = false;
}

int fsi_set_launch_params(fsi_ctx* c, int level, const fsi_launch_params* p) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, true);
    if (!p) throw ApiError(FSI_E_INVALID, "null launch parameters");
    if (p->apply_slices < 0 || p->apply_slices > 4096 || p->apply_groups < 0 || p->apply_groups > 256 ||
        (p->spmv_sub != 0 && p->spmv_sub != 2 && p->spmv_sub != 4 && p->spmv_sub != 8) ||
        (p->gj_panel != 0 && p->gj_panel != 16 && p->gj_panel != 24 && p->gj_panel != 32 &&
         p->gj_panel != kGjPanelPair))
      throw ApiError(FSI_E_INVALID, "launch parameters out of range");
    sync(*c);   // nothing in flight uses the old shapes or the graph
    DevLevel& D = c->dl[level];
    D.apply_slices = p->apply_slices;
    D.apply_groups = p->apply_groups;
    D.spmv_sub = p->spmv_sub;
    if (level == (int)c->dl.size() - 1) c->gj_panel = p->gj_panel;
    drop_vcycle_graph(*c);
  });
}

int fsi_get_launch_params(fsi_ctx* c, int level, fsi_launch_params* out) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, true);
    if (!out) throw ApiError(FSI_E_INVALID, "null output");
    const DevLevel& D = c->dl[level];
    const ApplyShape a = apply_shape(D.n_patches, D.max_nown, c->mixed ? 4 : 2, c->sm_count, D.apply_slices,
                                     D.apply_groups);
    out->apply_slices = a.kind == 0 ? 1 : a.slices;
    out->apply_groups = a.kind == 0 ? 4 : a.groups;
    out->spmv_sub = D.spmv_sub == 0 ? 4 : D.spmv_sub;
    out->gj_panel = c->gj_panel;
  });
}

int fsi_time_level_kernels(fsi_ctx* c, int level, int reps, double* apply_ms, double* spmv_ms) {
  return guard(c, [&] {
    need_device(*c);
    check_level(*c, level, true);
    if (reps < 1 || reps > 10000) throw ApiError(FSI_E_INVALID, "reps must be in [1, 10000]");
    if (!c->factored) throw ApiError(FSI_E_INVALID, "fsi_factor_schwarz first");
    DevLevel& D = c->dl[level];
    cudaEvent_t e[3];
    for (auto& ev : e) ck(cudaEventCreate(&ev), "event");
    const size_t nv = (size_t)D.Ni * (c->mixed ? sizeof(float) : sizeof(double));
    void* x = c->mixed ? (void*)D.x32 : (void*)D.x;
    void* b = c->mixed ? (void*)D.b32 : (void*)D.b;
    void* r = c->mixed ? (void*)D.r32 : (void*)D.r;
    ck(cudaMemsetAsync(x, 0, nv, c->stream), "memset");
    ck(cudaMemsetAsync(b, 0, nv, c->stream), "memset");
    ck(cudaMemsetAsync(r, 0, nv, c->stream), "memset");
    ck(cudaEventRecord(e[0], c->stream), "event");
    for (int k = 0; k < reps; ++k) {
      if (c->mixed) VC<float>::apply(*c, level, D.r32, D.x32);
      else VC<double>::apply(*c, level, D.r, D.x);
    }
    ck(cudaEventRecord(e[1], c->stream), "event");
    for (int k = 0; k < reps; ++k) {
      if (c->mixed) VC<float>::residual(*c, level, D.x32, D.b32, D.r32);
      else VC<double>::residual(*c, level, D.x, D.b, D.r);
    }
    ck(cudaEventRecord(e[2], c->stream), "event");
    sync(*c);
    float t0 = 0.f, t1 = 0.f;
    cudaEventElapsedTime(&t0, e[0], e[1]);
    cudaEventElapsedTime(&t1, e[1], e[2]);
    for (auto& ev : e) cudaEventDestroy(ev);
    if (apply_ms) *apply_ms = t0 / reps;
    if (spmv_ms) *spmv_ms = t1 / reps;
  });
}

int fsi_kernel_stats(fsi_ctx* c, int kind, double* device_ms, int64_t* launches, double* alg_bytes,
                     double* alg_flops) {
  return guard(c, [&] {
    need_device(*c);
    if (kind < 0 || kind >= FSI_K_COUNT) throw ApiError(FSI_E_INVALID, "bad kernel class");
    harvest(*c);
    const auto& ks = c->kstat[kind];
    if (device_ms) *device_ms = ks.ms;
    if (launches) *launches = ks.launches;
    if (alg_bytes) *alg_bytes = ks.bytes;
    if (alg_flops) *alg_flops = ks.flops;
  });
}

}  // extern "C"
