// Sparse / dense linear-algebra kernels of the Newton-step solve:
//  * BSR residual / SpMV on the block-sparse Jacobian of each level;
//  * scalar CSR SpMV for the grid transfers (Sec. 3.2);
//  * Schwarz blocks (Sec. 3.3): gather B_k from the BSR values, batched
//    partial-pivot Gauss-Jordan inversion keeping only the owned rows of
//    B_k^{-1}, and the restricted update x += omega (R^0_k)^T B_k^{-1} R^delta_k r;
//  * coarse level: dense gather, cooperative multi-block Gauss-Jordan with
//    partial pivoting (FP64), dense GEMV apply;
//  * Krylov helpers: multi-vector dot products, classical Gram-Schmidt
//    updates, norms, linear combinations (Sec. 4.1 FGMRES).
#include <cooperative_groups.h>

#include <cmath>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace fsi {

namespace {
constexpr int kWarp = 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum, result valid in thread 0
__device__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + kWarp - 1) / kWarp;
    s = lane < nw ? scratch[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// block-wide argmax of |v| (ties: lowest index); every thread gets the index
__device__ int block_argmax(double v, int idx, double* sv, int* si) {
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx && oi >= 0) || (idx < 0 && oi >= 0)) { v = ov; idx = oi; }
  }
  __syncthreads();
  if (lane == 0) { sv[wid] = v; si[wid] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + kWarp - 1) / kWarp;
    double bv = sv[0];
    int bi = si[0];
    for (int w = 1; w < nw; ++w)
      if (sv[w] > bv || (sv[w] == bv && si[w] >= 0 && (bi < 0 || si[w] < bi)) || (bi < 0 && si[w] >= 0)) {
        bv = sv[w];
        bi = si[w];
      }
    si[0] = bi;
  }
  __syncthreads();
  const int r = si[0];
  __syncthreads();
  return r;
}
}  // namespace

// ---------------------------------------------------------------------------
// BSR residual: y = b - A x  (b == nullptr: y = A x); one thread per scalar row
// ---------------------------------------------------------------------------
template <int B>
__global__ void k_bsr_residual(int64_t nb, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const double* __restrict__ x,
                               const double* __restrict__ b, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * B) return;
  const int64_t br = i / B;
  const int ci = (int)(i % B);
  double acc = 0.0;
  const int32_t k1 = rowptr[br + 1];
  for (int32_t k = rowptr[br]; k < k1; ++k) {
    const int64_t bc = col[k];
    const double* v = val + (int64_t)k * B * B + ci * B;
    if (B == 4) {
      const double2 a0 = *reinterpret_cast<const double2*>(v);
      const double2 a1 = *reinterpret_cast<const double2*>(v + 2);
      const double2 x0 = *reinterpret_cast<const double2*>(x + bc * 4);
      const double2 x1 = *reinterpret_cast<const double2*>(x + bc * 4 + 2);
      acc += a0.x * x0.x + a0.y * x0.y + a1.x * x1.x + a1.y * x1.y;
    } else {
#pragma unroll
      for (int c = 0; c < B; ++c) acc += v[c] * x[bc * B + c];
    }
  }
  y[i] = b ? b[i] - acc : acc;
}

void launch_bsr_residual(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                         const double* x, const double* b, double* y, cudaStream_t st) {
  const int64_t n = nb * B;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (B == 4) k_bsr_residual<4><<<grid, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
  else k_bsr_residual<6><<<grid, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
}

__global__ void k_csr_spmv(int64_t nrows, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                           int add) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  double acc = 0.0;
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) acc += val[k] * x[col[k]];
  y[i] = add ? y[i] + acc : acc;
}

void launch_csr_spmv(int64_t nrows, const int32_t* ptr, const int32_t* col, const double* val, const double* x,
                     double* y, bool add, cudaStream_t st) {
  k_csr_spmv<<<(unsigned)((nrows + 255) / 256), 256, 0, st>>>(nrows, ptr, col, val, x, y, add ? 1 : 0);
}

__global__ void k_gather(int64_t n, const int32_t* __restrict__ map, const double* __restrict__ in,
                         double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t m = map[i];
  out[i] = m >= 0 ? in[m] : 0.0;
}

void launch_gather(int64_t n, const int32_t* map, const double* in, double* out, cudaStream_t st) {
  k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, map, in, out);
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, b, y);
}

__global__ void k_scale_by(int64_t n, const double* __restrict__ src, const double* __restrict__ s,
                           double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double inv = 1.0 / s[0];
  if (i < n) dst[i] = src[i] * inv;
}

void launch_scale_by(int64_t n, const double* src, const double* dev_scalar, double* dst, cudaStream_t st) {
  k_scale_by<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, src, dev_scalar, dst);
}

// partial[v * nblk + bx] = sum over block bx's chunk of V[v] . w
__global__ void k_dots(int64_t n, const double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                       double* __restrict__ partial) {
  __shared__ double scratch[32];
  const int v = blockIdx.y;
  const double* Vv = V + (int64_t)v * ldv;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += Vv[i] * w[i];
  const double s = block_sum(acc, scratch);
  if (threadIdx.x == 0) partial[(int64_t)v * gridDim.x + blockIdx.x] = s;
}

void launch_dots(int64_t n, const double* V, int64_t ldv, int nvec, const double* w, double* partial, int nblk,
                 cudaStream_t st) {
  k_dots<<<dim3(nblk, nvec), 256, 0, st>>>(n, V, ldv, w, partial);
}

__global__ void k_norm_partial(int64_t n, const double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double scratch[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += w[i] * w[i];
  const double s = block_sum(acc, scratch);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

void launch_norm_partial(int64_t n, const double* w, double* partial, int nblk, cudaStream_t st) {
  k_norm_partial<<<nblk, 256, 0, st>>>(n, w, partial);
}

// out[v] = sum_b partial[v * nblk + b] (fixed order), optionally sqrt
__global__ void k_reduce(const double* __restrict__ partial, int nblk, double* __restrict__ out, int sqrt_out) {
  __shared__ double scratch[32];
  const int v = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partial[(int64_t)v * nblk + b];
  const double s = block_sum(acc, scratch);
  if (threadIdx.x == 0) out[v] = sqrt_out ? sqrt(s) : s;
}

void launch_reduce(const double* partial, int nvec, int nblk, double* out, bool sqrt_out, cudaStream_t st) {
  k_reduce<<<nvec, 256, 0, st>>>(partial, nblk, out, sqrt_out ? 1 : 0);
}

// w -= sum_v V[v] h[v]
__global__ void k_cgs_update(int64_t n, const double* __restrict__ V, int64_t ldv, int nvec,
                             const double* __restrict__ h, double* __restrict__ w) {
  __shared__ double sh[64];
  if (threadIdx.x < nvec) sh[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int v = 0; v < nvec; ++v) acc -= V[(int64_t)v * ldv + i] * sh[v];
    w[i] = acc;
  }
}

void launch_cgs_update(int64_t n, const double* V, int64_t ldv, int nvec, const double* h, double* w,
                       cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_cgs_update<<<grid, 256, 0, st>>>(n, V, ldv, nvec, h, w);
}

// x += sum_v Z[v] coef[v]
__global__ void k_combo(int64_t n, const double* __restrict__ Z, int64_t ldz, int nvec, const double* __restrict__ c,
                        double* __restrict__ x) {
  __shared__ double sc[64];
  if (threadIdx.x < nvec) sc[threadIdx.x] = c[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int v = 0; v < nvec; ++v) acc += Z[(int64_t)v * ldz + i] * sc[v];
    x[i] = acc;
  }
}

void launch_combo(int64_t n, const double* Z, int64_t ldz, int nvec, const double* coef, double* x, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_combo<<<grid, 256, 0, st>>>(n, Z, ldz, nvec, coef, x);
}

__global__ void k_nonfinite(int64_t n, const double* __restrict__ v, int32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(v[i])) atomicExch(&status[ST_NONFINITE], 1);
}

void launch_nonfinite_check(int64_t n, const double* v, int32_t* status, cudaStream_t st) {
  k_nonfinite<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, v, status);
}

// ---------------------------------------------------------------------------
// Schwarz blocks
// ---------------------------------------------------------------------------
__global__ void k_patch_gather(const int32_t* __restrict__ p_n, const int64_t* __restrict__ dense_off,
                               const int64_t* __restrict__ gmap_off, const int32_t* __restrict__ gmap,
                               const int64_t* __restrict__ pad_off, const int32_t* __restrict__ padpos,
                               const double* __restrict__ bsr_val, int B, double* __restrict__ dense) {
  const int p = blockIdx.x;
  const int n = p_n[p];
  double* D = dense + dense_off[p];
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) D[t] = 0.0;
  __syncthreads();
  const int BB = B * B;
  const int64_t g0 = gmap_off[p], g1 = gmap_off[p + 1];
  for (int64_t t = threadIdx.x; t < (g1 - g0) * BB; t += blockDim.x) {
    const int64_t g = g0 + t / BB;
    const int e = (int)(t % BB), ci = e / B, cj = e % B;
    const int32_t blk = gmap[3 * g], lr = gmap[3 * g + 1], lc = gmap[3 * g + 2];
    D[(int64_t)(lr * B + ci) * n + lc * B + cj] = bsr_val[(int64_t)blk * BB + e];
  }
  __syncthreads();
  for (int64_t t = pad_off[p] + threadIdx.x; t < pad_off[p + 1]; t += blockDim.x) {
    const int q = padpos[t];
    D[(int64_t)q * n + q] = 1.0;
  }
}

void launch_patch_gather(int np, const int32_t* p_n, const int64_t* dense_off, const int64_t* gmap_off,
                         const int32_t* gmap, const int64_t* pad_off, const int32_t* padpos, const double* bsr_val,
                         int B, double* dense, cudaStream_t st) {
  if (np <= 0) return;
  k_patch_gather<<<np, 256, 0, st>>>(p_n, dense_off, gmap_off, gmap, pad_off, padpos, bsr_val, B, dense);
}

// In-place Gauss-Jordan with partial (row) pivoting on one Schwarz block per
// thread block.  Step k pivots on the unused row p with the largest |M[p][k]|;
// every row is updated from copies of row p and column k, so no row is read
// while it is written.  At the end M[p_k][q_c] = (B^{-1})[k][c] with q the
// inverse pivot permutation; only the owned rows k are written out.
template <bool SMEM>
__global__ void __launch_bounds__(512)
k_patch_gj(const int32_t* __restrict__ p_n, const int32_t* __restrict__ p_nown,
           const int64_t* __restrict__ dense_off, const int64_t* __restrict__ own_off,
           const int32_t* __restrict__ own, const int64_t* __restrict__ inv_off, double* __restrict__ dense,
           double* __restrict__ inv, int32_t* __restrict__ status) {
  extern __shared__ double smem[];
  const int p = blockIdx.x;
  const int n = p_n[p];
  double* prow = smem;
  double* pcol = prow + n;
  int* piv = reinterpret_cast<int*>(pcol + n);
  int* qinv = piv + n;
  uint8_t* used = reinterpret_cast<uint8_t*>(qinv + n);
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_sing;
  double* Mg = dense + dense_off[p];
  double* M = Mg;
  if (SMEM) {
    M = reinterpret_cast<double*>(used + ((n + 15) / 16) * 16);
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) M[t] = Mg[t];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) used[i] = 0;
  if (threadIdx.x == 0) s_sing = 0;
  __syncthreads();
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = -1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (used[i]) continue;
      double a = fabs(M[(int64_t)i * n + k]);
      if (!(a >= 0.0)) a = 0.0;   // NaN never wins, but an unused row always exists
      if (a > best) { best = a; bi = i; }
    }
    const int pr = block_argmax(best, bi, sv, si);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      prow[j] = M[(int64_t)pr * n + j];
      pcol[j] = M[(int64_t)j * n + k];
    }
    if (threadIdx.x == 0) { used[pr] = 1; piv[k] = pr; }
    __syncthreads();
    double pv = prow[k];
    if (!(fabs(pv) > 0.0) || !isfinite(pv)) {
      if (threadIdx.x == 0) s_sing = 1;
      pv = 1.0;
    }
    const double rp = 1.0 / pv;
    for (int i = wid; i < n; i += nw) {
      double* Mi = M + (int64_t)i * n;
      if (i == pr) {
        for (int j = lane; j < n; j += kWarp) Mi[j] = (j == k) ? rp : prow[j] * rp;
      } else {
        const double f = pcol[i] * rp;
        if (f != 0.0)
          for (int j = lane; j < n; j += kWarp) Mi[j] = (j == k) ? -f : Mi[j] - f * prow[j];
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) qinv[piv[k]] = k;
  __syncthreads();
  const int nown = p_nown[p];
  const int32_t* ow = own + own_off[p];
  double* out = inv + inv_off[p];
  for (int o = wid; o < nown; o += nw) {
    const double* Mr = M + (int64_t)piv[ow[o]] * n;
    for (int c = lane; c < n; c += kWarp) out[(int64_t)o * n + c] = Mr[qinv[c]];
  }
  if (threadIdx.x == 0 && s_sing) atomicExch(&status[ST_SINGULAR], 1);
}

void launch_patch_gj(int np, int max_n, const int32_t* p_n, const int32_t* p_nown, const int64_t* dense_off,
                     const int64_t* own_off, const int32_t* own, const int64_t* inv_off, double* dense, double* inv,
                     int32_t* status, cudaStream_t st) {
  if (np <= 0) return;
  const size_t base = (size_t)max_n * (2 * sizeof(double) + 2 * sizeof(int)) + ((max_n + 15) / 16) * 16;
  const size_t with_m = base + (size_t)max_n * max_n * sizeof(double);
  if (with_m <= 200 * 1024) {
    cudaFuncSetAttribute(k_patch_gj<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)with_m);
    k_patch_gj<true><<<np, 512, with_m, st>>>(p_n, p_nown, dense_off, own_off, own, inv_off, dense, inv, status);
  } else {
    cudaFuncSetAttribute(k_patch_gj<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base);
    k_patch_gj<false><<<np, 512, base, st>>>(p_n, p_nown, dense_off, own_off, own, inv_off, dense, inv, status);
  }
}

// x[idx[own[o]]] += omega * (B_k^{-1} r[idx])[own[o]] for every owned row o
__global__ void __launch_bounds__(256)
k_patch_apply(const int32_t* __restrict__ p_n, const int32_t* __restrict__ p_nown,
              const int64_t* __restrict__ idx_off, const int32_t* __restrict__ idx,
              const int64_t* __restrict__ own_off, const int32_t* __restrict__ own,
              const int64_t* __restrict__ inv_off, const double* __restrict__ inv,
              const double* __restrict__ r, double* __restrict__ x, double omega) {
  extern __shared__ double rs[];
  const int p = blockIdx.x;
  const int n = p_n[p];
  const int32_t* id = idx + idx_off[p];
  for (int i = threadIdx.x; i < n; i += blockDim.x) rs[i] = r[id[i]];
  __syncthreads();
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
  const int nown = p_nown[p];
  const int32_t* ow = own + own_off[p];
  const double* Bi = inv + inv_off[p];
  for (int o = wid; o < nown; o += nw) {
    const double2* row = reinterpret_cast<const double2*>(Bi + (int64_t)o * n);
    double acc = 0.0;
    for (int c = lane; c < n / 2; c += kWarp) {
      const double2 a = row[c];
      acc += a.x * rs[2 * c] + a.y * rs[2 * c + 1];
    }
    acc = warp_sum(acc);
    if (lane == 0) x[id[ow[o]]] += omega * acc;
  }
}

void launch_patch_apply(int np, int max_n, const int32_t* p_n, const int32_t* p_nown, const int64_t* idx_off,
                        const int32_t* idx, const int64_t* own_off, const int32_t* own, const int64_t* inv_off,
                        const double* inv, const double* r, double* x, double omega, cudaStream_t st) {
  if (np <= 0) return;
  k_patch_apply<<<np, 256, (size_t)max_n * sizeof(double), st>>>(p_n, p_nown, idx_off, idx, own_off, own, inv_off,
                                                                 inv, r, x, omega);
}

// ---------------------------------------------------------------------------
// coarse level
// ---------------------------------------------------------------------------
__global__ void k_dense_gather(int B, int64_t nb, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, int64_t n, double* __restrict__ A) {
  const int64_t br = blockIdx.x;
  if (br >= nb) return;
  const int BB = B * B;
  for (int32_t k = rowptr[br]; k < rowptr[br + 1]; ++k)
    for (int e = threadIdx.x; e < BB; e += blockDim.x) {
      const int ci = e / B, cj = e % B;
      A[(br * B + ci) * n + (int64_t)col[k] * B + cj] = val[(int64_t)k * BB + e];
    }
}

__global__ void k_set_diag(const int32_t* __restrict__ list, int cnt, int64_t n, double* __restrict__ A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cnt) A[(int64_t)list[t] * n + list[t]] = 1.0;
}

void launch_dense_gather(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                         const int32_t* pad_list, int npad, int64_t n, double* A, cudaStream_t st) {
  cudaMemsetAsync(A, 0, (size_t)n * n * sizeof(double), st);
  k_dense_gather<<<(unsigned)nb, 64, 0, st>>>(B, nb, rowptr, col, val, n, A);
  if (npad > 0) k_set_diag<<<(npad + 255) / 256, 256, 0, st>>>(pad_list, npad, n, A);
}

// Cooperative Gauss-Jordan with partial pivoting on the coarse operator.
// Step k reads matrix M_k and writes M_{k+1} (ping-pong between A and Bm) so
// that the pivot row and column are never read while being written; one grid
// barrier per step.  Every block finds the pivot itself (same deterministic
// rule), so no extra barrier is needed for it.
__global__ void __launch_bounds__(256) k_coarse_gj(int64_t n, double* A, double* Bm, int32_t* __restrict__ piv,
                                                   int32_t* __restrict__ status) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ uint8_t used[];
  __shared__ double sv[32];
  __shared__ int si[32];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) used[i] = 0;
  __syncthreads();
  for (int64_t k = 0; k < n; ++k) {
    const double* M = (k & 1) ? Bm : A;
    double* O = (k & 1) ? A : Bm;
    double best = -1.0;
    int bi = -1;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      if (used[i]) continue;
      double a = fabs(M[i * n + k]);
      if (!(a >= 0.0)) a = 0.0;
      if (a > best) { best = a; bi = (int)i; }
    }
    const int pr = block_argmax(best, bi, sv, si);
    if (threadIdx.x == 0) used[pr] = 1;
    double pv = M[(int64_t)pr * n + k];
    if (!(fabs(pv) > 0.0) || !isfinite(pv)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&status[ST_SINGULAR], 1);
      pv = 1.0;
    }
    const double rp = 1.0 / pv;
    const double* Mp = M + (int64_t)pr * n;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
      const double* Mi = M + i * n;
      double* Oi = O + i * n;
      if (i == pr) {
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) Oi[j] = (j == k) ? rp : Mp[j] * rp;
      } else {
        const double f = Mi[k] * rp;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) Oi[j] = (j == k) ? -f : Mi[j] - f * Mp[j];
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) piv[k] = pr;
    __syncthreads();
    grid.sync();
  }
}

__global__ void k_coarse_permute(int64_t n, const double* __restrict__ M, const int32_t* __restrict__ piv,
                                 double* __restrict__ inv) {
  extern __shared__ int qinv_s[];
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) qinv_s[piv[k]] = (int)k;
  __syncthreads();
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
    const double* Mr = M + (int64_t)piv[k] * n;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) inv[k * n + c] = Mr[qinv_s[c]];
  }
}

int launch_coarse_gj(int64_t n, double* A, double* Bm, double* inv, int32_t* piv, int32_t* status, int sm_count,
                     cudaStream_t st) {
  int per_sm = 0;
  const size_t smem = (size_t)n;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_gj, 256, smem);
  if (per_sm < 1) return -1;
  int grid = std::min<int64_t>((int64_t)per_sm * sm_count, n);
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&n, (void*)&A, (void*)&Bm, (void*)&piv, (void*)&status};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_coarse_gj, grid, 256, args, smem, st);
  if (e != cudaSuccess) return -2;
  const double* M = (n & 1) ? Bm : A;   // after n steps the result sits here
  k_coarse_permute<<<std::min<int64_t>(n, 1024), 256, (size_t)n * sizeof(int), st>>>(n, M, piv, inv);
  return 0;
}

// y = A x, one warp per row (A row-major, n x n)
__global__ void k_gemv(int64_t n, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x % kWarp;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  if (row >= n) return;
  const double* Ar = A + row * n;
  double acc = 0.0;
  for (int64_t c = lane; c < n; c += kWarp) acc += Ar[c] * x[c];
  acc = warp_sum(acc);
  if (lane == 0) y[row] = acc;
}

void launch_gemv(int64_t n, const double* A, const double* x, double* y, cudaStream_t st) {
  const int64_t threads = n * kWarp;
  k_gemv<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, A, x, y);
}

}  // namespace fsi
