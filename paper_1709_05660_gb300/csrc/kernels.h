// Kernel launchers shared between the .cu translation units of libfsi.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "fsi_internal.h"

namespace fsi {

struct PhysParams {
  double rho_f, mu_f, rho_s, mu_s;
  int ale_op;
  double mr_c2;         // Mooney-Rivlin C2 (0: Neo-Hookean); 2 C1 = mu_s - 2 C2
  // transient (BDF) terms: q_t = (a0 q + yold) * idt with yold = a1 q_n + a2 q_{n-1}
  int transient;
  double a0, idt;
  const double* yold;   // internal layout, finest level (nullptr when steady)
};

// bounds-check build (-DFSI_BOUNDS_CHECK): the first failed index check of
// each translation unit's kernels since the last call (FSI_SITE code: unit *
// 100000 + line; 0: none), cleared by the read; always 0 in the normal build
int bounds_site_schwarz();
int bounds_site_linalg();

// k_assemble.cu
// scratch: 3D only, assemble_3d_scratch_doubles(scratch_ne) doubles (2D: unused); false (nothing
// launched) when one pass of ne elements needs more scratch than that
bool launch_assemble_2d(bool solid, const int32_t* elems, int ne, const double* y, const int32_t* elem_nodes,
                        const uint8_t* node_class, const double* elem_geo, int64_t n_nodes, PhysParams pp,
                        double* Ke, double* Re, int32_t* status, double* scratch, int scratch_ne, cudaStream_t st);
bool launch_assemble_3d(bool solid, const int32_t* elems, int ne, const double* y, const int32_t* elem_nodes,
                        const uint8_t* node_class, const double* elem_geo, int64_t n_nodes, PhysParams pp,
                        double* Ke, double* Re, int32_t* status, double* scratch, int scratch_ne, cudaStream_t st);
size_t assemble_3d_scratch_doubles(int max_ne);
int assemble_launches(int dim, int ne);   // kernel launches of one launch_assemble_* call
double assemble_flops_per_element(int dim, bool solid, int mode);   // executed FP64 flops (ncu count)
double galerkin_flops_per_coarse_element(int dim);
void launch_galerkin_3d(int ncx, int ncy, int ncz, const double* Kf, const int32_t* f_nodes, const uint8_t* f_class,
                        const uint8_t* f_dir, const int32_t* c_nodes, const uint8_t* c_class, const uint8_t* c_dir,
                        double* Kc, cudaStream_t st);
// element matrices -> block values (every entry written) and, with res set,
// element residuals -> residual, summed in the order of the gather lists
void launch_gather_elements(int dim, int64_t nnzb, const int32_t* blk_ptr, const int32_t* blk_src, const double* Ke,
                            double* val, int64_t nb, const int32_t* res_ptr, const int32_t* res_src,
                            const double* Re, double* res, cudaStream_t st);
void launch_dirichlet(const int32_t* dir_list, int64_t n_dir, const int32_t* rowptr, const int32_t* col, double* val,
                      int B, const double* y, const double* g, double alpha, double* res, cudaStream_t st);
void launch_galerkin_2d(int ncx, int ncy, const double* Kf, const int32_t* f_nodes, const uint8_t* f_class,
                        const uint8_t* f_dir, const int32_t* c_nodes, const uint8_t* c_class, const uint8_t* c_dir,
                        double* Kc, cudaStream_t st);

// k_linalg.cu
void launch_bsr_residual(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                         const double* x, const double* b, double* y, cudaStream_t st);
void launch_bsr_residual_f32(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const float* val,
                             const float* x, const float* b, float* y, int sub, cudaStream_t st);
void launch_csr_spmv(int64_t nrows, const int32_t* ptr, const int32_t* col, const double* val, const double* x,
                     double* y, bool add, cudaStream_t st);
void launch_gather(int64_t n, const int32_t* map, const double* in, double* out, cudaStream_t st);
void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);
void launch_scale_by(int64_t n, const double* src, const double* dev_scalar, double* dst, cudaStream_t st);
void launch_reduce(const double* partial, int nvec, int nblk, double* out, bool sqrt_out, cudaStream_t st);
// fused Arnoldi passes (nvec <= 72; partial holds (nvec + 1) * nblk doubles)
void launch_arnoldi_dots(int64_t n, const double* V, int64_t ldv, int nvec, const double* w, bool with_norm,
                         double* partial, int nblk, cudaStream_t st);
void launch_arnoldi_update_norm(int64_t n, const double* V, int64_t ldv, int nvec, const double* h, double* w,
                                double* partial, int nblk, cudaStream_t st);
void launch_cgs_update(int64_t n, const double* V, int64_t ldv, int nvec, const double* h, double* w, cudaStream_t st);
void launch_combo(int64_t n, const double* Z, int64_t ldz, int nvec, const double* coef, double* x, cudaStream_t st);
void launch_norm_partial(int64_t n, const double* w, double* partial, int nblk, cudaStream_t st);
void launch_nonfinite_check(int64_t n, const double* v, int32_t* status, cudaStream_t st);

// k_schwarz.cu (T = double: FP64 path, T = float: mixed path)
// Schwarz blocks of one level for the tensor-core factorisation; several
// levels can share one launch (blocks first .. first + n_patches - 1)
constexpr int kGjMaxLevels = 24;   // levels of one launch (several instances may share it)
struct GjLevel {
  const int32_t* p_n;
  const int32_t* p_nown;
  const int64_t* dense_off;
  const int64_t* own_off;
  const int32_t* own;
  const int64_t* inv_off;
  float* dense;
  float* invT;
  int32_t* status;   // status flags of the instance the level belongs to
  const int32_t* sel; // blocks of the level to factor (nullptr: all of them)
  int first;
};
struct GjLevels {
  int nlev;
  // iteration limit of the first bounded wait of each block on its tensor-core
  // work (the drain waits before tensor memory is released keep their full limit)
  long long first_wait;
  GjLevel l[kGjMaxLevels];
};
constexpr long long kTcWaitIters = 1LL << 22;
// Gauss-Jordan variant code: 16-column panels on 64-column tiles with 256
// tensor-memory columns, so that two blocks share an SM (blocks <= 512 unknowns)
constexpr int kGjPanelPair = 216;
// false when the blocks do not fit the tensor-core kernel (the caller then
// factors level by level)
// panel: preferred panel width (16 or 32; 0 = 32 when the blocks fit, else 16)
bool launch_patch_gj_tc_levels(const GjLevels& lv, int nblocks, int max_n, int32_t* status, cudaStream_t st,
                               int panel = 0);
// panel width of the tensor-core variant that launch_patch_gj_tc_levels picks
// for blocks up to max_n with preference `panel` (0: none fits)
int gj_tc_variant(int max_n, int panel);
// the FP32 gathers of the Schwarz levels of one instance in one launch
struct GatherLevel {
  const int32_t* p_n;
  const int64_t* dense_off;
  const int64_t* gmap_off;
  const int32_t* gmap;
  const int64_t* boff_off;
  const int32_t* boff;
  const int64_t* pad_off;
  const int32_t* padpos;
  const double* bsr_val;
  float* dense;
  const int64_t* idx_off;
  float* dr;
  float* dc;
  int first;   // first thread block of the level
};
struct GatherLevels {
  int nlev, B;
  GatherLevel l[kGjMaxLevels];
};
void launch_patch_gather_levels(const GatherLevels& lv, int nblocks, cudaStream_t st);
// boff / boff_off: per local block of a Schwarz block its dense offset * 8 + width
template <typename T>
void launch_patch_gather_t(int np, const int32_t* p_n, const int64_t* dense_off, const int64_t* gmap_off,
                           const int32_t* gmap, const int64_t* boff_off, const int32_t* boff, const int64_t* pad_off,
                           const int32_t* padpos, const double* bsr_val, int B, T* dense, const int64_t* idx_off,
                           T* dr, T* dc, cudaStream_t st);
template <typename T>
void launch_patch_gj_t(int np, int max_n, const int32_t* p_n, const int32_t* p_nown, const int64_t* dense_off,
                       const int64_t* own_off, const int32_t* own, const int64_t* inv_off, T* dense, T* invT,
                       int32_t* status, bool n_mult4, cudaStream_t st);
// sel: the np blocks to apply (nullptr: blocks 0 .. np - 1); nv: length of r and x
template <typename T>
void launch_patch_apply_t(int np, int64_t nv, int max_n, int max_nown, const int32_t* p_n, const int32_t* p_nown,
                          const int64_t* idx_off, const int32_t* idx, const int64_t* own_off, const int32_t* own,
                          const int64_t* inv_off, const T* invT, const T* r, T* x, double omega, const T* dr,
                          const T* dc, int sm_count, int want_slices, int want_groups, cudaStream_t st,
                          const int32_t* sel = nullptr);
// ILU(0) of the fluid Schwarz blocks listed in sel (Sec. 3.3, 4.1), in place
// on their gathered, equilibrated dense blocks; blocks of at most
// kIluMaxRows unknowns
constexpr int kIluMaxRows = 1024;
void launch_patch_ilu0(int nsel, const int32_t* sel, const int32_t* p_n, const int64_t* dense_off,
                       const int64_t* gmap_off, const int32_t* gmap, const int64_t* boff_off, const int32_t* boff,
                       int B, float* dense, int32_t* status, cudaStream_t st);
// x[own] += omega (R^0)^T U^{-1} L^{-1} R^delta r for the ILU(0) blocks in sel (at most max_n
// unknowns and max_nb node / element blocks each)
void launch_patch_apply_ilu(int nsel, int max_n, int max_nb, const int32_t* sel, const int32_t* p_n,
                            const int32_t* p_nown,
                            const int64_t* idx_off, const int32_t* idx, const int64_t* own_off, const int32_t* own,
                            const int64_t* dense_off, const int64_t* gmap_off, const int32_t* gmap,
                            const int64_t* boff_off, const int32_t* boff, const int32_t* gptr, int B,
                            const float* dense, const float* r, float* x, double omega, const float* dr,
                            const float* dc, cudaStream_t st);
// Launch shape of one level's Schwarz apply: kind 0 = one block per patch
// (k_patch_apply_t), kind 1 = `slices` row slices per patch of `vps` owned-row
// vectors, `groups` column groups per block (k_patch_apply_rows).
// want_slices 0 / want_groups 0 = the built-in rule; want_slices 1 = kind 0.
struct ApplyShape { int kind, slices, vps, groups; };
ApplyShape apply_shape(int np, int max_nown, int vec_width, int sm_count, int want_slices, int want_groups);

void launch_dense_gather(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                         const int32_t* pad_list, int npad, const int32_t* perm, int64_t n, double* A,
                         cudaStream_t st);
int launch_coarse_lu_inverse(int64_t n, int kl, int ku, double* M, double* rdiag, double* Ainv, int32_t* piv,
                             const int32_t* perm, const int32_t* pinv, int32_t* status, int sm_count,
                             cudaStream_t st);
// coarse apply: part holds ceil(n / 32) * n doubles of scratch
void launch_gemv(int64_t n, const double* A, const double* x, double* y, double* part, cudaStream_t st);
void launch_gemv_f32io(int64_t n, const double* A, const float* x, float* y, double* part, cudaStream_t st);
// slab-blocked coarse solve: column-major FP64 sub-matrices with leading dimensions
void launch_dgemm_nn(int m, int n, int k, double alpha, const double* A, int64_t lda, const double* Bm, int64_t ldb,
                     double beta, double* C, int64_t ldc, cudaStream_t st);
void launch_copy2d(int m, int n, const double* src, int64_t lds, double* dst, int64_t ldd, cudaStream_t st);
// y = beta y + alpha A x; part holds ceil(nc / 32) * m doubles of scratch
void launch_gemv_sub(int m, int nc, double alpha, const double* A, int64_t lda, const double* x, double beta,
                     double* y, double* part, cudaStream_t st);
void launch_csr_spmv_f32(int64_t nrows, const int32_t* ptr, const int32_t* col, const float* val, const float* x,
                         float* y, bool add, cudaStream_t st);
void launch_to_f32(int64_t n, const double* in, float* out, cudaStream_t st);
void launch_to_f64(int64_t n, const float* in, double* out, cudaStream_t st);
void launch_combo_mixed(int64_t n, const float* Z, int64_t ldz, int nvec, const double* coef, double* x,
                        cudaStream_t st);

}  // namespace fsi
