// Sparse / dense linear-algebra kernels of the Newton-step solve:
//  * BSR residual / SpMV on the block-sparse Jacobian of each level;
//  * scalar CSR SpMV for the grid transfers (Sec. 3.2);
//  * coarse level (FP64): dense gather in the banded x-slab ordering, blocked
//    banded LU with partial pivoting (cooperative), inverse columns by
//    triangular solves, dense GEMV apply; for the slab-blocked 3D solve also
//    dense GEMM / GEMV on column-major sub-matrices;
//  * Krylov helpers: multi-vector dot products, classical Gram-Schmidt
//    updates, norms, linear combinations (Sec. 4.1 FGMRES).
#include <cooperative_groups.h>

#include <cmath>

#include "bounds.cuh"
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

// Block-wide argmax of |a| (largest wins, ties to the lower index; threads
// without a candidate pass idx = -1) on integer keys: the bit pattern of a
// non-negative double orders like its value, so |a| compared as a 64-bit
// integer (NaN mapped to 0) picks the row a floating-point comparison would,
// while keeping the comparisons off the FP64 pipe, which on GB300 retires two
// operations per SM and cycle.
// a != 0.0 (either sign of zero fails) as an integer test, off the FP64 pipe
__device__ __forceinline__ bool nonzero(double a) {
  return ((unsigned long long)__double_as_longlong(a) << 1) != 0ull;
}
__device__ __forceinline__ unsigned long long abs_key(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
  return b > 0x7FF0000000000000ull ? 0ull : b;   // NaN -> 0; +inf stays the largest
}
__device__ __forceinline__ bool key_wins(unsigned long long ok, int oi, unsigned long long k, int i) {
  return (oi >= 0 && i < 0) || (oi >= 0 && (ok > k || (ok == k && oi < i)));
}
__device__ int block_argmax_key(unsigned long long v, int idx, unsigned long long* sv, int* si) {
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (key_wins(ov, oi, v, idx)) { v = ov; idx = oi; }
  }
  __syncthreads();
  if (lane == 0) { sv[wid] = v; si[wid] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + kWarp - 1) / kWarp;
    unsigned long long bv = sv[0];
    int bi = si[0];
    for (int w = 1; w < nw; ++w)
      if (key_wins(sv[w], si[w], bv, bi)) {
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
// BSR residual: y = b - A x  (b == nullptr: y = A x); one thread per scalar
// row, two blocks per iteration with independent accumulators.  TV: matrix
// values, TX: input vector, TY: output (and accumulation) type.
// ---------------------------------------------------------------------------
namespace {
template <int B, typename TV, typename TX, typename TA>
__device__ __forceinline__ TA block_row_dot(const TV* __restrict__ v, const TX* __restrict__ xb) {
  TA acc = TA(0);
#pragma unroll
  for (int c = 0; c < B; ++c) acc += TA(v[c]) * TA(xb[c]);
  return acc;
}
}  // namespace

template <int B, typename TV, typename TX, typename TY>
__global__ void k_bsr_residual(int64_t nb, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const TV* __restrict__ val, const TX* __restrict__ x, const TY* __restrict__ b,
                               TY* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * B) return;
  const int64_t br = i / B;
  const int ci = (int)(i % B);
  TY acc0 = TY(0), acc1 = TY(0);
  const int32_t k1 = rowptr[br + 1];
  int32_t k = rowptr[br];
  for (; k + 1 < k1; k += 2) {
    const int64_t c0 = __ldg(col + k), c1 = __ldg(col + k + 1);
    if (FSI_IN(c0, nb, FSI_SITE(2))) acc0 += block_row_dot<B, TV, TX, TY>(val + (int64_t)k * B * B + ci * B, x + c0 * B);
    if (FSI_IN(c1, nb, FSI_SITE(2)))
      acc1 += block_row_dot<B, TV, TX, TY>(val + (int64_t)(k + 1) * B * B + ci * B, x + c1 * B);
  }
  if (k < k1 && FSI_IN(__ldg(col + k), nb, FSI_SITE(2)))
    acc0 += block_row_dot<B, TV, TX, TY>(val + (int64_t)k * B * B + ci * B, x + (int64_t)__ldg(col + k) * B);
  const TY acc = acc0 + acc1;
  y[i] = b ? b[i] - acc : acc;
}

// B = 4 variant with SUB threads per scalar row: thread sub takes blocks
// rowptr + sub, rowptr + sub + SUB, ... in rounds of four; a round issues the
// column, value and vector loads of its four blocks before any product, so
// one thread keeps up to 12 loads in flight instead of a dependent chain per
// block.  The partial sums are combined with warp shuffles (sub is the
// fastest index, so a row's threads are adjacent lanes); a warp reads
// consecutive blocks of two block-rows (coalesced).
template <typename TV> struct BlkRow;
template <> struct BlkRow<double> {   // one row of a 4 x 4 FP64 block
  double2 a, b;
  __device__ __forceinline__ void load(const double* p) {
    a = __ldg(reinterpret_cast<const double2*>(p));
    b = __ldg(reinterpret_cast<const double2*>(p + 2));
  }
  __device__ __forceinline__ void zero() { a = make_double2(0.0, 0.0); b = a; }
  template <typename TY> __device__ __forceinline__ void fma_into(TY& acc, const TY (&x)[4]) const {
    acc = fma(TY(a.x), x[0], acc);
    acc = fma(TY(a.y), x[1], acc);
    acc = fma(TY(b.x), x[2], acc);
    acc = fma(TY(b.y), x[3], acc);
  }
};
template <> struct BlkRow<float> {
  float4 a;
  __device__ __forceinline__ void load(const float* p) { a = __ldg(reinterpret_cast<const float4*>(p)); }
  __device__ __forceinline__ void zero() { a = make_float4(0.f, 0.f, 0.f, 0.f); }
  template <typename TY> __device__ __forceinline__ void fma_into(TY& acc, const TY (&x)[4]) const {
    acc = fma(TY(a.x), x[0], acc);
    acc = fma(TY(a.y), x[1], acc);
    acc = fma(TY(a.z), x[2], acc);
    acc = fma(TY(a.w), x[3], acc);
  }
};
template <typename TX, typename TY>
__device__ __forceinline__ void load_x4(const TX* p, TY (&x)[4]) {
  if constexpr (sizeof(TX) == 8) {
    const double2 u = __ldg(reinterpret_cast<const double2*>(p)), v = __ldg(reinterpret_cast<const double2*>(p + 2));
    x[0] = TY(u.x); x[1] = TY(u.y); x[2] = TY(v.x); x[3] = TY(v.y);
  } else {
    const float4 u = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = TY(u.x); x[1] = TY(u.y); x[2] = TY(u.z); x[3] = TY(u.w);
  }
}

// FP32: 8 blocks of 256 threads per SM (32 registers a thread): full
// occupancy, as the finest levels' residual is bound by the loads in flight.
// FP64: 4 blocks (64 registers), so that a thread's four blocks of values and
// x entries (64 registers of doubles) are loaded together
template <int SUB, typename TV, typename TX, typename TY>
__global__ void __launch_bounds__(256, sizeof(TV) == 8 ? 4 : 8) k_bsr4_residual_sub(int64_t nb, const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col, const TV* __restrict__ val,
                                                          const TX* __restrict__ x, const TY* __restrict__ b,
                                                          TY* __restrict__ y) {
  constexpr int B = 4, R = 4;   // blocks per thread and round
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / SUB;
  const int sub = (int)(t % SUB);
  TY acc = TY(0);
  if (i < nb * B) {
    const int64_t br = i / B;
    const int ci = (int)(i % B);
    const int32_t k0 = rowptr[br], k1 = rowptr[br + 1];
    for (int32_t kb = k0 + sub; kb < k1; kb += R * SUB) {
      int32_t c[R];
      BlkRow<TV> v[R];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const int32_t k = kb + u * SUB;
        c[u] = k < k1 ? __ldg(col + k) : -1;
        if (c[u] >= 0 && !FSI_IN(c[u], nb, FSI_SITE(2))) c[u] = -1;
        if (k < k1) v[u].load(val + (int64_t)k * B * B + ci * B);
        else v[u].zero();
      }
      TY xv[R][4];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        if (c[u] >= 0) load_x4<TX, TY>(x + (int64_t)c[u] * B, xv[u]);
        else xv[u][0] = xv[u][1] = xv[u][2] = xv[u][3] = TY(0);
      }
      // four fused multiply-adds per block (FP64: the pipe that bounds this
      // kernel on GB300); slots past the row's last block are skipped, which
      // a warp does as a whole when both of its block-rows have ended
#pragma unroll
      for (int u = 0; u < R; ++u)
        if (c[u] >= 0) v[u].template fma_into<TY>(acc, xv[u]);
    }
  }
#pragma unroll
  for (int o = SUB / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (sub == 0 && i < nb * B) y[i] = b ? b[i] - acc : acc;
}

void launch_bsr_residual(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                         const double* x, const double* b, double* y, cudaStream_t st) {
  const int64_t n = nb * B;
  const unsigned grid = (unsigned)((n + 255) / 256);
  const unsigned grid4 = (unsigned)((n * 4 + 255) / 256);
  if (B == 4) k_bsr4_residual_sub<4, double, double, double><<<grid4, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
  else k_bsr_residual<6, double, double, double><<<grid, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
}

void launch_bsr_residual_f32(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const float* val,
                             const float* x, const float* b, float* y, int sub, cudaStream_t st) {
  const int64_t n = nb * B;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (B == 4) {
    // threads per scalar row: 4 unless a tuned mapping says 2 or 8
    const int S = (sub == 2 || sub == 8) ? sub : 4;
    const unsigned gs = (unsigned)((n * S + 255) / 256);
    if (S == 2) k_bsr4_residual_sub<2, float, float, float><<<gs, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
    else if (S == 8) k_bsr4_residual_sub<8, float, float, float><<<gs, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
    else k_bsr4_residual_sub<4, float, float, float><<<gs, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
  } else {
    k_bsr_residual<6, float, float, float><<<grid, 256, 0, st>>>(nb, rowptr, col, val, x, b, y);
  }
}

template <typename TV, typename TX, typename TY>
__global__ void k_csr_spmv(int64_t nrows, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const TV* __restrict__ val, const TX* __restrict__ x, TY* __restrict__ y, int add) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  TY acc = TY(0);
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) acc += TY(val[k]) * TY(x[col[k]]);
  y[i] = add ? y[i] + acc : acc;
}

void launch_csr_spmv(int64_t nrows, const int32_t* ptr, const int32_t* col, const double* val, const double* x,
                     double* y, bool add, cudaStream_t st) {
  k_csr_spmv<double, double, double><<<(unsigned)((nrows + 255) / 256), 256, 0, st>>>(nrows, ptr, col, val, x, y,
                                                                                      add ? 1 : 0);
}

void launch_csr_spmv_f32(int64_t nrows, const int32_t* ptr, const int32_t* col, const float* val, const float* x,
                         float* y, bool add, cudaStream_t st) {
  k_csr_spmv<float, float, float><<<(unsigned)((nrows + 255) / 256), 256, 0, st>>>(nrows, ptr, col, val, x, y,
                                                                                   add ? 1 : 0);
}

template <typename TI, typename TO>
__global__ void k_convert(int64_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = TO(in[i]);
}

void launch_to_f32(int64_t n, const double* in, float* out, cudaStream_t st) {
  k_convert<double, float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, in, out);
}

void launch_to_f64(int64_t n, const float* in, double* out, cudaStream_t st) {
  k_convert<float, double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, in, out);
}

// x += sum_v Z[v] coef[v] with FP32 basis vectors and FP64 coefficients / result
__global__ void k_combo_mixed(int64_t n, const float* __restrict__ Z, int64_t ldz, int nvec,
                              const double* __restrict__ c, double* __restrict__ x) {
  __shared__ double sc[64];
  if (threadIdx.x < nvec) sc[threadIdx.x] = c[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int v = 0; v < nvec; ++v) acc += (double)Z[(int64_t)v * ldz + i] * sc[v];
    x[i] = acc;
  }
}

void launch_combo_mixed(int64_t n, const float* Z, int64_t ldz, int nvec, const double* coef, double* x,
                        cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_combo_mixed<<<grid, 256, 0, st>>>(n, Z, ldz, nvec, coef, x);
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

// ---------------------------------------------------------------------------
// Fused Arnoldi (CGS2) passes.  One pass over the rows i of a block's chunk
// forms all nvec partial dot products V[v] . w at once (one accumulator per
// vector, NV >= nvec, so w and every V[v][i] are read once); the Gram-Schmidt
// updates w -= sum_v V[v] h[v] are fused with the partial sums the next step
// needs (the second pass's dots, or ||w||^2).  Partial sums are reduced within
// a warp by shuffles, then across the block's warps in a fixed order, and
// k_reduce adds the blocks' partials in a fixed order: the result does not
// depend on scheduling.
// ---------------------------------------------------------------------------
// out[v * out_stride] (v < nacc) = the block's sums of acc[v]; with has_extra,
// out[nacc * out_stride] = the block's sum of `extra`.  red: 8 * (NV + 1) doubles.
template <int NV>
__device__ __forceinline__ void block_partials(double (&acc)[NV], int nacc, double extra, bool has_extra,
                                               double* red, double* out, int64_t out_stride) {
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v < nacc) {   // warp-uniform; no early exit, so acc stays in registers
      double a = acc[v];
#pragma unroll
      for (int o = kWarp / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red[wid * (NV + 1) + v] = a;
    }
  }
  if (has_extra) {
#pragma unroll
    for (int o = kWarp / 2; o > 0; o >>= 1) extra += __shfl_xor_sync(0xffffffffu, extra, o);
    if (lane == 0) red[wid * (NV + 1) + nacc] = extra;
  }
  __syncthreads();
  const int nout = nacc + (has_extra ? 1 : 0);
  for (int v = threadIdx.x; v < nout; v += blockDim.x) {
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a += red[k * (NV + 1) + v];
    out[(int64_t)v * out_stride] = a;
  }
}

// partial[v * nblk + b] = V[v] . w over block b's rows (v < nvec); with
// with_norm, partial[nvec * nblk + b] = w . w
template <int NV>
__global__ void __launch_bounds__(256) k_arnoldi_dots(int64_t n, const double* __restrict__ V, int64_t ldv, int nvec,
                                                      const double* __restrict__ w, int with_norm,
                                                      double* __restrict__ partial) {
  __shared__ double red[8 * (NV + 1)];
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  double nn = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
    nn += wi * wi;
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (v < nvec) acc[v] += V[(int64_t)v * ldv + i] * wi;
  }
  block_partials<NV>(acc, nvec, nn, with_norm != 0, red, partial + blockIdx.x, gridDim.x);
}

// w -= sum_v V[v] h[v], fused with the partial sums of the new w . w
template <int NV>
__global__ void __launch_bounds__(256) k_arnoldi_update_norm(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                             int nvec, const double* __restrict__ h,
                                                             double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double red[8 * 2];
  __shared__ double sh[NV];
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) sh[v] = h[v];
  __syncthreads();
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double wi = w[i];
    for (int v = 0; v < nvec; ++v) wi -= V[(int64_t)v * ldv + i] * sh[v];
    w[i] = wi;
    acc[0] += wi * wi;
  }
  block_partials<1>(acc, 1, 0.0, false, red, partial + blockIdx.x, gridDim.x);
}

template <int NV>
static bool arnoldi_go_dots(int64_t n, const double* V, int64_t ldv, int nvec, const double* w, bool with_norm,
                            double* partial, int nblk, cudaStream_t st) {
  if (nvec > NV) return false;
  k_arnoldi_dots<NV><<<nblk, 256, 0, st>>>(n, V, ldv, nvec, w, with_norm ? 1 : 0, partial);
  return true;
}

void launch_arnoldi_dots(int64_t n, const double* V, int64_t ldv, int nvec, const double* w, bool with_norm,
                         double* partial, int nblk, cudaStream_t st) {
  if (arnoldi_go_dots<8>(n, V, ldv, nvec, w, with_norm, partial, nblk, st)) return;
  if (arnoldi_go_dots<16>(n, V, ldv, nvec, w, with_norm, partial, nblk, st)) return;
  if (arnoldi_go_dots<32>(n, V, ldv, nvec, w, with_norm, partial, nblk, st)) return;
  arnoldi_go_dots<72>(n, V, ldv, nvec, w, with_norm, partial, nblk, st);   // restart <= 64: nvec <= 65
}

void launch_arnoldi_update_norm(int64_t n, const double* V, int64_t ldv, int nvec, const double* h, double* w,
                                double* partial, int nblk, cudaStream_t st) {
  if (nvec <= 64) k_arnoldi_update_norm<64><<<nblk, 256, 0, st>>>(n, V, ldv, nvec, h, w, partial);
  else k_arnoldi_update_norm<128><<<nblk, 256, 0, st>>>(n, V, ldv, nvec, h, w, partial);
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
// coarse level
// ---------------------------------------------------------------------------
// Dense coarse operator in the banded ordering, column-major:
// A[perm[col] * n + perm[row]] (padding slots get 1 on the diagonal).
__global__ void k_dense_gather(int B, int64_t nb, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const int32_t* __restrict__ perm, int64_t n,
                               double* __restrict__ A) {
  const int64_t br = blockIdx.x;
  if (br >= nb) return;
  const int BB = B * B;
  for (int32_t k = rowptr[br]; k < rowptr[br + 1]; ++k)
    for (int e = threadIdx.x; e < BB; e += blockDim.x) {
      const int ci = e / B, cj = e % B;
      if (!FSI_IN(col[k], nb, FSI_SITE(2))) continue;
      const int64_t r = perm[br * B + ci], c = perm[(int64_t)col[k] * B + cj];
      if (FSI_IN(r, n, FSI_SITE(2)) && FSI_IN(c, n, FSI_SITE(2))) A[c * n + r] = val[(int64_t)k * BB + e];
    }
}

__global__ void k_set_diag(const int32_t* __restrict__ list, int cnt, const int32_t* __restrict__ perm, int64_t n,
                           double* __restrict__ A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < cnt) {
    const int64_t q = perm[list[t]];
    if (FSI_IN(q, n, FSI_SITE(2))) A[q * n + q] = 1.0;
  }
}

void launch_dense_gather(int B, int64_t nb, const int32_t* rowptr, const int32_t* col, const double* val,
                         const int32_t* pad_list, int npad, const int32_t* perm, int64_t n, double* A,
                         cudaStream_t st) {
  cudaMemsetAsync(A, 0, (size_t)n * n * sizeof(double), st);
  k_dense_gather<<<(unsigned)nb, 64, 0, st>>>(B, nb, rowptr, col, val, perm, n, A);
  if (npad > 0) k_set_diag<<<(npad + 255) / 256, 256, 0, st>>>(pad_list, npad, perm, n, A);
}


// Blocked banded LU with partial pivoting of a matrix stored column-major in
// dense form (lower half-bandwidth kl, upper ku; row interchanges widen U to
// kl + ku).  Factors as in the unblocked band algorithm: multipliers of step j
// in column j rows j+1..j+kl in the row order of step j (later interchanges are
// not applied to them), U up to kl + ku above the diagonal, piv[j] the row
// swapped with j, rdiag[j] = 1 / U_jj (the reciprocal the step scales its
// multipliers with; 1 where the pivot is zero, which also flags the status).  Panels of NB columns; per panel two grid barriers instead of NB:
//  A. block 0 factors the panel (rows k0 .. k0+nb-1+kl) in shared memory with
//     the unblocked steps, row swaps applied to the panel's columns right of
//     the step only, and writes panel and pivots back;
//  B. every block stages the panel's multipliers and pivots, and each warp
//     applies the panel's NB steps (swap, then the multiplier update) to one
//     trailing column in shared memory: columns k0+nb .. k0+nb-1+kl+ku.

// y[r] += a x[r] for r = base + lane, base + lane + 32, ... <= rhi (a warp-wide
// update in shared memory): whole rounds of 128 rows (four per lane, all loads
// issued before the stores: x and y are different columns, which the compiler
// cannot prove), then the last partial round the same way with the rows past
// rhi masked, so a short range (a narrow band) costs one round trip, not one
// per 32 rows.
__device__ __forceinline__ void axpy_rows(double* y, const double* x, double a, int base, int rhi) {
  int r = base + threadIdx.x % kWarp;
  const int rounds = (rhi - base + 1) / (4 * kWarp);
  for (int q = 0; q < rounds; ++q, r += 4 * kWarp) {
    const double x0 = x[r], x1 = x[r + kWarp], x2 = x[r + 2 * kWarp], x3 = x[r + 3 * kWarp];
    const double y0 = y[r], y1 = y[r + kWarp], y2 = y[r + 2 * kWarp], y3 = y[r + 3 * kWarp];
    y[r] = fma(a, x0, y0);
    y[r + kWarp] = fma(a, x1, y1);
    y[r + 2 * kWarp] = fma(a, x2, y2);
    y[r + 3 * kWarp] = fma(a, x3, y3);
  }
  double xv[4], yv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int rk = r + k * kWarp;
    xv[k] = rk <= rhi ? x[rk] : 0.0;
    yv[k] = rk <= rhi ? y[rk] : 0.0;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (r + k * kWarp <= rhi) y[r + k * kWarp] = fma(a, xv[k], yv[k]);
}

// the same with x a column of the factor in global memory (y in shared memory)
__device__ __forceinline__ void axpy_rows_g(double* y, const double* __restrict__ x, double a, int base, int rhi) {
  int r = base + threadIdx.x % kWarp;
  const int rounds = (rhi - base + 1) / (4 * kWarp);
  for (int q = 0; q < rounds; ++q, r += 4 * kWarp) {
    const double x0 = __ldg(x + r), x1 = __ldg(x + r + kWarp), x2 = __ldg(x + r + 2 * kWarp),
                 x3 = __ldg(x + r + 3 * kWarp);
    const double y0 = y[r], y1 = y[r + kWarp], y2 = y[r + 2 * kWarp], y3 = y[r + 3 * kWarp];
    y[r] = fma(a, x0, y0);
    y[r + kWarp] = fma(a, x1, y1);
    y[r + 2 * kWarp] = fma(a, x2, y2);
    y[r + 3 * kWarp] = fma(a, x3, y3);
  }
  for (; r <= rhi; r += kWarp) y[r] = fma(a, __ldg(x + r), y[r]);
}

// panel columns k0 .. k0 + nb - 1, rows k0 .. k0 + nr - 1 of M into P (R rows
// a column): four loads in flight per thread
__device__ __forceinline__ void load_panel(double* P, int R, const double* __restrict__ M, int64_t n, int64_t k0,
                                           int nb, int nr) {
  const int tot = nb * nr, step = blockDim.x;
  for (int t0 = threadIdx.x; t0 < tot; t0 += 4 * step) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * step, j = t / nr, r = t - j * nr;
      v[u] = t < tot ? M[(k0 + j) * n + k0 + r] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * step, j = t / nr, r = t - j * nr;
      if (t < tot) P[j * R + r] = v[u];
    }
  }
}

template <int NB>
__global__ void __launch_bounds__(512) k_band_lu_blk(int64_t n, int kl, int ku, double* __restrict__ M,
                                                    int32_t* __restrict__ piv, double* __restrict__ rdiag,
                                                    int32_t* __restrict__ status, int col_warps) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = NB + kl;                                  // panel rows (at most)
  double* P = reinterpret_cast<double*>(smem_raw);        // R x NB, column-major
  double* S = P + (size_t)R * NB;                         // per warp: R entries of one trailing column
  __shared__ int s_piv[NB];
  __shared__ unsigned long long skey[32];
  __shared__ int si[32];
  __shared__ double s_rp;
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
  // the trailing update of phase B uses col_warps warps per block (one
  // shared-memory column buffer each); all warps work in phase A
  const int nwb = min(nw, col_warps);
  const int64_t wmax = (int64_t)kl + ku;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nb = (int)min((int64_t)NB, n - k0);
    const int nr = (int)(min(n, k0 + nb + kl) - k0);
    if (blockIdx.x == 0) {
      load_panel(P, R, M, n, k0, nb, nr);
      __syncthreads();
      for (int j = 0; j < nb; ++j) {
        const int rhi = min(j + kl, nr - 1);
        unsigned long long best = 0ull;
        int bi = -1;
        for (int r = j + threadIdx.x; r <= rhi; r += blockDim.x) {
          const unsigned long long a = abs_key(P[j * R + r]);
          if (bi < 0 || a > best) { best = a; bi = r; }
        }
        int pr = block_argmax_key(best, bi, skey, si);
        if (pr < 0) pr = j;
        if (pr != j)
          for (int c = j + threadIdx.x; c < nb; c += blockDim.x) {
            const double t0 = P[c * R + j];
            P[c * R + j] = P[c * R + pr];
            P[c * R + pr] = t0;
          }
        // the reciprocal pivot by one thread (it swapped column j itself):
        // a division on every thread would occupy each SM sub-partition's
        // FP64 pipe for the whole warp
        if (threadIdx.x == 0) {
          double pv = P[j * R + j];
          if (!(fabs(pv) > 0.0) || !isfinite(pv)) {
            atomicExch(&status[ST_SINGULAR], 1);
            pv = 1.0;
          }
          s_rp = 1.0 / pv;
          rdiag[k0 + j] = s_rp;
        }
        __syncthreads();
        const double rp = s_rp;
        for (int r = j + 1 + threadIdx.x; r <= rhi; r += blockDim.x) P[j * R + r] *= rp;
        __syncthreads();
        // rank-1 update of the panel's columns right of j: a warp per column,
        // lanes over rows (the column's multiplier is warp-uniform)
        for (int c = j + 1 + wid; c < nb; c += nw) {
          const double pc = P[c * R + j];
          if (nonzero(pc)) axpy_rows(P + c * R, P + j * R, -pc, j + 1, rhi);
        }
        if (threadIdx.x == 0) s_piv[j] = pr;
        __syncthreads();
      }
      for (int t = threadIdx.x; t < nb * nr; t += blockDim.x) {
        const int j = t / nr, r = t - j * nr;
        M[(k0 + j) * n + k0 + r] = P[j * R + r];
      }
      for (int j = threadIdx.x; j < nb; j += blockDim.x) piv[k0 + j] = (int32_t)(k0 + s_piv[j]);
    }
    grid.sync();
    const int64_t c_lo = k0 + nb, c_hi = min(n - 1, k0 + nb - 1 + wmax);
    if (c_lo <= c_hi) {
      // stage multipliers and pivots (every block)
      load_panel(P, R, M, n, k0, nb, nr);
      for (int j = threadIdx.x; j < nb; j += blockDim.x) s_piv[j] = (int)(piv[k0 + j] - k0);
      __syncthreads();
      double* Sw = S + (size_t)wid * R;
      for (int64_t c = c_lo + (int64_t)blockIdx.x * nwb + wid; wid < nwb && c <= c_hi;
           c += (int64_t)gridDim.x * nwb) {
        double* Mc = M + c * n + k0;
        for (int r0 = lane; r0 < nr; r0 += 4 * kWarp) {   // four loads in flight per lane
          double v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = r0 + u * kWarp < nr ? Mc[r0 + u * kWarp] : 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (r0 + u * kWarp < nr) Sw[r0 + u * kWarp] = v[u];
        }
        __syncwarp();
        for (int j = 0; j < nb; ++j) {
          const int pr = s_piv[j];
          if (pr != j && lane == 0) {
            const double t0 = Sw[j];
            Sw[j] = Sw[pr];
            Sw[pr] = t0;
          }
          __syncwarp();
          const double t = Sw[j];
          if (nonzero(t)) axpy_rows(Sw, P + j * R, -t, j + 1, min(j + kl, nr - 1));
          __syncwarp();
        }
        for (int r = lane; r < nr; r += kWarp) Mc[r] = Sw[r];
        __syncwarp();
      }
    }
    grid.sync();
  }
}

template <int NB>
size_t band_lu_blk_smem(int kl, int col_warps) {
  return ((size_t)(NB + kl) * NB + (size_t)col_warps * (NB + kl)) * sizeof(double);
}

// Narrow-band variant of k_band_inv (kl + ku <= 32 MR): each lane holds at
// most MR rows of a factor column, and the column of step k + 1 is loaded
// into registers before the updates of step k, so a step waits on shared
// memory only, not on a fresh global load.
template <int MR>
__global__ void __launch_bounds__(128) k_band_inv_pf(int64_t n, int kl, int ku, const double* __restrict__ M,
                                                     const int32_t* __restrict__ piv,
                                                     const double* __restrict__ rdiag,
                                                     const int32_t* __restrict__ perm,
                                                     const int32_t* __restrict__ pinv, double* __restrict__ Ainv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / kWarp) + wid;
  if (c >= n) return;
  double* x = reinterpret_cast<double*>(smem_raw) + (int64_t)wid * n;
  for (int64_t i = lane; i < n; i += kWarp) x[i] = (i == c) ? 1.0 : 0.0;
  __syncwarp();
  // forward: rows k+1 .. k+kl of column k; lane's m-th row is k + 1 + lane + 32 m
  const int64_t k_start = max((int64_t)0, c - (int64_t)kl);
  double cur[MR], nxt[MR];
  auto load_l = [&](int64_t k, double (&v)[MR]) {
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      if (32 * m >= kl) { v[m] = 0.0; continue; }
      const int64_t r = k + 1 + lane + 32 * m;
      v[m] = (k < n && r <= min(n - 1, k + (int64_t)kl)) ? M[k * n + r] : 0.0;
    }
  };
  load_l(k_start, cur);
  int64_t pcur = piv[k_start];
  for (int64_t k = k_start; k < n; ++k) {
    load_l(k + 1, nxt);
    const int64_t pnxt = k + 1 < n ? piv[k + 1] : 0;
    const int64_t p = pcur;
    if (p != k) {
      if (lane == 0) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
      __syncwarp();
    }
    const double xk = x[k];
    if (nonzero(xk)) {
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        if (32 * m >= kl) break;   // warp-uniform: no issue slots for rows beyond the band
        const int64_t r = k + 1 + lane + 32 * m;
        if (r <= min(n - 1, k + (int64_t)kl)) x[r] -= cur[m] * xk;
      }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < MR; ++m) cur[m] = nxt[m];
    pcur = pnxt;
  }
  // backward: rows k - w .. k - 1 of column k (w = kl + ku); lane's m-th row is k - 1 - lane - 32 m
  const int64_t w = (int64_t)kl + ku;
  auto load_u = [&](int64_t k, double (&v)[MR], double& d) {
    d = k >= 0 ? rdiag[k] : 1.0;
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      if (32 * m >= w) { v[m] = 0.0; continue; }
      const int64_t r = k - 1 - lane - 32 * m;
      v[m] = (k >= 0 && r >= 0 && r >= k - w) ? M[k * n + r] : 0.0;
    }
  };
  double dcur, dnxt;
  load_u(n - 1, cur, dcur);
  for (int64_t k = n - 1; k >= 0; --k) {
    load_u(k - 1, nxt, dnxt);
    // reciprocal pivot (no FP64 division on the critical chain), formed by
    // lane 0 and broadcast, so the warp spends one lane's FP64 multiply on it
    double xk = 0.0;
    if (lane == 0) {
      xk = x[k] * dcur;
      x[k] = xk;
    }
    xk = __shfl_sync(0xffffffffu, xk, 0);
    if (nonzero(xk)) {
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        if (32 * m >= w) break;
        const int64_t r = k - 1 - lane - 32 * m;
        if (r >= 0 && r >= k - w) x[r] -= cur[m] * xk;
      }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < MR; ++m) cur[m] = nxt[m];
    dcur = dnxt;
  }
  double* out = Ainv + (int64_t)pinv[c] * n;
  for (int64_t i = lane; i < n; i += kWarp) out[i] = x[perm[i]];
}

// Columns of the inverse from the banded LU: one warp per right-hand side
// e_c (banded ordering), forward substitution with the row interchanges and
// unit L, back substitution with U; the column is written to the inverse in
// the original internal ordering, column-major:
// Ainv[pinv(c) * n + i] = x[perm[i]].
__global__ void __launch_bounds__(128) k_band_inv(int64_t n, int kl, int ku, const double* __restrict__ M,
                                                  const int32_t* __restrict__ piv, const double* __restrict__ rdiag,
                                                  const int32_t* __restrict__ perm,
                                                  const int32_t* __restrict__ pinv, double* __restrict__ Ainv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / kWarp) + wid;
  if (c >= n) return;
  double* x = reinterpret_cast<double*>(smem_raw) + (int64_t)wid * n;
  for (int64_t i = lane; i < n; i += kWarp) x[i] = (i == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int64_t k = 0; k < n; ++k) {
    const int64_t p = piv[k];
    if (p != k) {
      if (lane == 0) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
      __syncwarp();
    }
    const double xk = x[k];
    if (nonzero(xk)) {
      const int64_t r_hi = min(n - 1, k + (int64_t)kl);
      axpy_rows_g(x + k, M + k * n + k, -xk, 1, (int)(r_hi - k));
    }
    __syncwarp();
  }
  const int64_t w = (int64_t)kl + ku;
  for (int64_t k = n - 1; k >= 0; --k) {
    const double* Uk = M + k * n;
    if (lane == 0) x[k] *= rdiag[k];
    __syncwarp();
    const double xk = x[k];
    if (nonzero(xk)) {
      const int64_t r_lo = max((int64_t)0, k - w);
      axpy_rows_g(x + r_lo, Uk + r_lo, -xk, 0, (int)(k - 1 - r_lo));
    }
    __syncwarp();
  }
  double* out = Ainv + (int64_t)pinv[c] * n;
  for (int64_t i = lane; i < n; i += kWarp) out[i] = x[perm[i]];
}

int launch_coarse_lu_inverse(int64_t n, int kl, int ku, double* M, double* rdiag, double* Ainv, int32_t* piv,
                             const int32_t* perm, const int32_t* pinv, int32_t* status, int sm_count,
                             cudaStream_t st) {
  // blocked LU: 16-column panels when they fit in shared memory, else 8.
  // The kl + ku trailing columns of a panel are spread at about three per
  // warp: more blocks only add grid-barrier cost and take SMs from the work
  // that runs beside the coarse factorisation.
  // wide bands (the dense 3D slab complements): 16 warps, so the panel
  // factorisation of block 0, which every other block waits for, has four
  // times the threads; narrow bands (2D): 4 warps
  const int threads = kl >= 256 ? 512 : 128;
  int grid = (int)std::min(std::min((int64_t)sm_count, n), std::max<int64_t>(8, ((int64_t)kl + ku + 11) / 12));
  if (grid < 1) grid = 1;
  // trailing-update warps per block: 8 when their column buffers fit beside
  // the panel (wide bands), else 4
  int cw = threads >= 512 ? 8 : 4;
  void* args[] = {(void*)&n,     (void*)&kl,     (void*)&ku, (void*)&M, (void*)&piv, (void*)&rdiag,
                  (void*)&status, (void*)&cw};
  auto go = [&](auto kern, size_t smem) -> int {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) return -1;
    if (cudaLaunchCooperativeKernel((const void*)kern, grid, threads, args, smem, st) != cudaSuccess) return -2;
    return 0;
  };
  int rc;
  const size_t cap = 222 * 1024;   // dynamic shared memory per block (227 KB minus the static arrays)
  if (band_lu_blk_smem<16>(kl, cw) > cap) cw = 4;
  if (band_lu_blk_smem<16>(kl, cw) <= cap) rc = go(k_band_lu_blk<16>, band_lu_blk_smem<16>(kl, cw));
  else if (band_lu_blk_smem<8>(kl, cw) <= cap) rc = go(k_band_lu_blk<8>, band_lu_blk_smem<8>(kl, cw));
  else return -3;
  if (rc != 0) return rc;
  // inverse columns: 4 warps (right-hand sides) per block, x in shared memory
  const int wpb = 4;
  const size_t ismem = (size_t)wpb * n * sizeof(double);
  if (ismem > 200 * 1024) return -4;
  const unsigned nblk = (unsigned)((n + wpb - 1) / wpb);
  if ((int64_t)kl + ku <= 32 * 8) {   // narrow band: register prefetch of the next factor column
    cudaFuncSetAttribute(k_band_inv_pf<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem);
    k_band_inv_pf<8><<<nblk, wpb * kWarp, ismem, st>>>(n, kl, ku, M, piv, rdiag, perm, pinv, Ainv);
  } else {
    cudaFuncSetAttribute(k_band_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem);
    k_band_inv<<<nblk, wpb * kWarp, ismem, st>>>(n, kl, ku, M, piv, rdiag, perm, pinv, Ainv);
  }
  return 0;
}

// y = A x with A column-major FP64 (n x n).  Stage 1: block (rb, cb) forms
// the partial product of rows [256 rb, 256 rb + 256) over the column chunk
// cb (kGemvChunk columns), one thread per row, coalesced column reads;
// stage 2 adds the chunk partials in a fixed order.
constexpr int kGemvChunk = 32;

template <typename TX>
__global__ void __launch_bounds__(256) k_gemv_cm_part(int64_t n, const double* __restrict__ A,
                                                      const TX* __restrict__ x, double* __restrict__ part) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * kGemvChunk;
  const int64_t c1 = min(n, c0 + kGemvChunk);
  if (i >= n) return;
  double a0 = 0.0, a1 = 0.0;
  int64_t c = c0;
  for (; c + 1 < c1; c += 2) {
    a0 += A[c * n + i] * (double)x[c];
    a1 += A[(c + 1) * n + i] * (double)x[c + 1];
  }
  if (c < c1) a0 += A[c * n + i] * (double)x[c];
  part[(int64_t)blockIdx.y * n + i] = a0 + a1;
}

template <typename TY>
__global__ void k_gemv_cm_sum(int64_t n, int nchunk, const double* __restrict__ part, TY* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int q = 0; q < nchunk; ++q) s += part[(int64_t)q * n + i];
  y[i] = TY(s);
}

void launch_gemv(int64_t n, const double* A, const double* x, double* y, double* part, cudaStream_t st) {
  const int nchunk = (int)((n + kGemvChunk - 1) / kGemvChunk);
  k_gemv_cm_part<double><<<dim3((unsigned)((n + 255) / 256), nchunk), 256, 0, st>>>(n, A, x, part);
  k_gemv_cm_sum<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, nchunk, part, y);
}

void launch_gemv_f32io(int64_t n, const double* A, const float* x, float* y, double* part, cudaStream_t st) {
  const int nchunk = (int)((n + kGemvChunk - 1) / kGemvChunk);
  k_gemv_cm_part<float><<<dim3((unsigned)((n + 255) / 256), nchunk), 256, 0, st>>>(n, A, x, part);
  k_gemv_cm_sum<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, nchunk, part, y);
}

// ---------------------------------------------------------------------------
// slab-blocked coarse solve (3D): dense FP64 building blocks on column-major
// sub-matrices with explicit leading dimensions
// ---------------------------------------------------------------------------

// C (m x n, ldc) = beta C + alpha A (m x k, lda) B (k x n, ldb).  64 x 64
// output tile per block, k in steps of 16 staged in shared memory, 4 x 4
// outputs per thread (rows tx + 16 i, columns ty + 16 j).
__global__ void __launch_bounds__(256) k_dgemm_nn(int m, int n, int k, double alpha, const double* __restrict__ A,
                                                 int64_t lda, const double* __restrict__ Bm, int64_t ldb, double beta,
                                                 double* __restrict__ C, int64_t ldc) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < k; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int r = e % 64, kk = e / 64;            // A tile: rows fastest (coalesced columns)
      const int gr = r0 + r, gk = k0 + kk;
      As[kk][r] = (gr < m && gk < k) ? A[(int64_t)gk * lda + gr] : 0.0;
      const int kb = e % 16, cb = e / 16;           // B tile: k fastest (coalesced columns)
      const int gkb = k0 + kb, gc = c0 + cb;
      Bs[kb][cb] = (gkb < k && gc < n) ? Bm[(int64_t)gc * ldb + gkb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gr = r0 + tx + 16 * i, gc = c0 + ty + 16 * j;
      if (gr < m && gc < n) {
        double* cp = C + (int64_t)gc * ldc + gr;
        *cp = (beta == 0.0 ? 0.0 : beta * *cp) + alpha * acc[i][j];
      }
    }
}

void launch_dgemm_nn(int m, int n, int k, double alpha, const double* A, int64_t lda, const double* Bm, int64_t ldb,
                     double beta, double* C, int64_t ldc, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  k_dgemm_nn<<<dim3((unsigned)((m + 63) / 64), (unsigned)((n + 63) / 64)), 256, 0, st>>>(m, n, k, alpha, A, lda, Bm,
                                                                                          ldb, beta, C, ldc);
}

// dst (m x n, ldd) = src (m x n, lds), column-major
__global__ void k_copy2d(int m, int n, const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                         int64_t ldd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * n) return;
  const int64_t c = t / m, r = t % m;
  dst[c * ldd + r] = src[c * lds + r];
}

void launch_copy2d(int m, int n, const double* src, int64_t lds, double* dst, int64_t ldd, cudaStream_t st) {
  const int64_t t = (int64_t)m * n;
  if (t <= 0) return;
  k_copy2d<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(m, n, src, lds, dst, ldd);
}

// y (m) = beta y + alpha A (m x nc, lda) x, A column-major.  Stage 1: block
// (rb, cb) forms the partial product of rows [256 rb, 256 rb + 256) over the
// column chunk cb; stage 2 adds the chunk partials in a fixed order.  x and y
// must not overlap.
__global__ void __launch_bounds__(256) k_gemv_sub_part(int m, int nc, const double* __restrict__ A, int64_t lda,
                                                       const double* __restrict__ x, double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c0 = blockIdx.y * kGemvChunk;
  const int c1 = min(nc, c0 + kGemvChunk);
  if (i >= m) return;
  double a0 = 0.0, a1 = 0.0;
  int c = c0;
  for (; c + 1 < c1; c += 2) {
    a0 += A[(int64_t)c * lda + i] * x[c];
    a1 += A[(int64_t)(c + 1) * lda + i] * x[c + 1];
  }
  if (c < c1) a0 += A[(int64_t)c * lda + i] * x[c];
  part[(int64_t)blockIdx.y * m + i] = a0 + a1;
}

__global__ void k_gemv_sub_sum(int m, int nchunk, const double* __restrict__ part, double alpha, double beta,
                               double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int q = 0; q < nchunk; ++q) s += part[(int64_t)q * m + i];
  y[i] = (beta == 0.0 ? 0.0 : beta * y[i]) + alpha * s;
}

void launch_gemv_sub(int m, int nc, double alpha, const double* A, int64_t lda, const double* x, double beta,
                     double* y, double* part, cudaStream_t st) {
  if (m <= 0) return;
  const int nchunk = (nc + kGemvChunk - 1) / kGemvChunk;
  if (nchunk > 0)
    k_gemv_sub_part<<<dim3((unsigned)((m + 255) / 256), (unsigned)nchunk), 256, 0, st>>>(m, nc, A, lda, x, part);
  k_gemv_sub_sum<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, nchunk, part, alpha, beta, y);
}

// the bounds-check build's recorded site of this translation unit (0: none)
FSI_BOUNDS_READER(bounds_site_linalg)

}  // namespace fsi
