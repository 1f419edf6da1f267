// Restricted additive Schwarz blocks of the Richardson smoother (Sec. 3.3),
// templated on the storage precision T (double: FP64 path, float: mixed path).
//
//  * k_patch_gather: B_k = J_l[R^delta_k, R^delta_k] copied from the BSR values
//    of level l into a dense n_k x n_k workspace (padding slots get 1 on the
//    diagonal so every block stays invertible), then equilibrated with exact
//    power-of-two row and column scales; the blocks mix rows scaled by the
//    shear modulus, the ALE stiffness 1/V_el and the kinematic mass matrix,
//    and without scaling an FP32 inverse loses its small entries.
//  * k_patch_gj: in-place Gauss-Jordan with partial (row) pivoting, one thread
//    block per Schwarz block.  Only the rows of B_k^{-1} that belong to R^0_k
//    are written out, transposed (column-major in the owned row index) so the
//    smoother's batched product reads them with coalesced loads.
//  * k_patch_apply: x[own] += omega * (B_k^{-1} r[R^delta_k])[own]; one thread
//    per owned row, the block residual broadcast from shared memory.
#include <cmath>
#include <type_traits>

#include "bounds.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace fsi {

namespace {
constexpr int kWarp = 32;

// Owned inverse rows are stored column-major with the owned count padded to a
// multiple of 4 (pad rows are zero), so each thread of the apply streams 4
// (FP32) or 2 (FP64) rows with one vector load.
__host__ __device__ __forceinline__ int own_pad(int nown) { return (nown + 3) & ~3; }

__device__ int block_argmax_abs(double v, int idx, double* sv, int* si) {
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) { v = ov; idx = oi; }
  }
  __syncthreads();
  if (lane == 0) { sv[wid] = v; si[wid] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + kWarp - 1) / kWarp;
    double bv = sv[0];
    int bi = si[0];
    for (int w = 1; w < nw; ++w)
      if (sv[w] > bv || (sv[w] == bv && si[w] >= 0 && (bi < 0 || si[w] < bi))) { bv = sv[w]; bi = si[w]; }
    si[0] = bi;
  }
  __syncthreads();
  const int r = si[0];
  __syncthreads();
  return r;
}
}  // namespace

// power of two closest (from below) to 1 / m, so scaling is exact; 1 for m == 0
constexpr int kGatherMaxN = 1024;   // blocks up to this size take the sparse-pass gather

__device__ __forceinline__ double pow2_inv(double m) {
  if (!(m > 0.0) || !isfinite(m)) return 1.0;
  int e;
  frexp(m, &e);           // m = f * 2^e, f in [0.5, 1)
  return ldexp(1.0, 1 - e);
}

// Gather B_k and equilibrate it: B~ = D_r B D_c with power-of-two row scales
// (row maxima -> [1, 2)) and then column scales.  The scales are stored so
// that B^{-1} r = D_c B~^{-1} (D_r r).
// Entry e of the B x B matrix block of gmap entry g: its dense row i and
// column j, or false for a padding component of an element block (left out
// of the dense block).
__device__ __forceinline__ bool gather_pos(const int32_t* __restrict__ gmap, const int32_t* __restrict__ bo,
                                           int64_t g, int e, int B, int& i, int& j) {
  const int ci = e / B, cj = e % B;
  const int32_t r = __ldg(bo + gmap[3 * g + 1]), c = __ldg(bo + gmap[3 * g + 2]);
  i = (r >> 3) + ci;
  j = (c >> 3) + cj;
  return ci < (r & 7) && cj < (c & 7);
}

template <typename T>
__device__ __forceinline__ void gather_block(int p, const int32_t* __restrict__ p_n,
                                             const int64_t* __restrict__ dense_off,
                                             const int64_t* __restrict__ gmap_off, const int32_t* __restrict__ gmap,
                                             const int64_t* __restrict__ boff_off, const int32_t* __restrict__ boff,
                                             const int64_t* __restrict__ pad_off, const int32_t* __restrict__ padpos,
                                             const double* __restrict__ bsr_val, int B, T* __restrict__ dense,
                                             const int64_t* __restrict__ idx_off, T* __restrict__ dr,
                                             T* __restrict__ dc) {
  const int n = p_n[p];
  T* D = dense + dense_off[p];
  const int32_t* bo = boff + boff_off[p];
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) D[t] = T(0);
  __syncthreads();
  const int BB = B * B;
  const int64_t g0 = gmap_off[p], g1 = gmap_off[p + 1];
  if (n <= kGatherMaxN) {
    // scales from the block-sparse entries (row and column maxima by integer
    // max on the bits of non-negative values, 32-bit for FP32 blocks), then one
    // scattered write of the equilibrated entries: the dense block is written
    // once.  Each pass takes kU entries per thread at a time, their loads
    // issued together (the passes are bound by the latency of these loads).
    using Key = typename std::conditional<sizeof(T) == 4, unsigned int, unsigned long long>::type;
    auto key = [](T a) -> Key {
      if constexpr (sizeof(T) == 4) return __float_as_uint(fabsf(a));
      else return (Key)__double_as_longlong(fabs(a));
    };
    auto val = [](Key k) -> double {
      if constexpr (sizeof(T) == 4) return (double)__uint_as_float(k);
      else return __longlong_as_double((long long)k);
    };
    __shared__ Key rmx[kGatherMaxN], cmx[kGatherMaxN];
    __shared__ T srw[kGatherMaxN], scl[kGatherMaxN];
    constexpr int kU = 8;
    const int64_t tot = (g1 - g0) * BB;
    // entries t0, t0 + blockDim, ... (kU of them): value, dense position, kept?
    auto fetch = [&](int64_t t0, T (&v)[kU], int (&ii)[kU], int (&jj)[kU], bool (&ok)[kU]) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t t = t0 + (int64_t)u * blockDim.x;
        ok[u] = false;
        v[u] = T(0);
        ii[u] = jj[u] = 0;
        if (t < tot) {
          const int64_t g = g0 + t / BB;
          const int e = (int)(t % BB);
          ok[u] = gather_pos(gmap, bo, g, e, B, ii[u], jj[u]);
          ok[u] = ok[u] && FSI_IN(ii[u], n, FSI_SITE(1)) && FSI_IN(jj[u], n, FSI_SITE(1));
          v[u] = T(bsr_val[(int64_t)gmap[3 * g] * BB + e]);
        }
      }
    };
    for (int i = threadIdx.x; i < n; i += blockDim.x) { rmx[i] = 0; cmx[i] = 0; }
    __syncthreads();
    for (int64_t t0 = threadIdx.x; t0 < tot; t0 += (int64_t)kU * blockDim.x) {
      T v[kU];
      int ii[kU], jj[kU];
      bool ok[kU];
      fetch(t0, v, ii, jj, ok);
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) atomicMax(&rmx[ii[u]], key(v[u]));
    }
    for (int64_t t = pad_off[p] + threadIdx.x; t < pad_off[p + 1]; t += blockDim.x)
      if (FSI_IN(padpos[t], n, FSI_SITE(1))) atomicMax(&rmx[padpos[t]], key(T(1)));
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) srw[i] = T(pow2_inv(val(rmx[i])));
    __syncthreads();
    for (int64_t t0 = threadIdx.x; t0 < tot; t0 += (int64_t)kU * blockDim.x) {
      T v[kU];
      int ii[kU], jj[kU];
      bool ok[kU];
      fetch(t0, v, ii, jj, ok);
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) atomicMax(&cmx[jj[u]], key(T(v[u] * srw[ii[u]])));
    }
    for (int64_t t = pad_off[p] + threadIdx.x; t < pad_off[p + 1]; t += blockDim.x) {
      const int q = padpos[t];
      if (FSI_IN(q, n, FSI_SITE(1))) atomicMax(&cmx[q], key(T(T(1) * srw[q])));
    }
    __syncthreads();
    T* Dr = dr + idx_off[p];
    T* Dc = dc + idx_off[p];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      scl[i] = T(pow2_inv(val(cmx[i])));
      Dr[i] = srw[i];
      Dc[i] = scl[i];
    }
    __syncthreads();
    for (int64_t t0 = threadIdx.x; t0 < tot; t0 += (int64_t)kU * blockDim.x) {
      T v[kU];
      int ii[kU], jj[kU];
      bool ok[kU];
      fetch(t0, v, ii, jj, ok);
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) D[(int64_t)ii[u] * n + jj[u]] = T(v[u] * srw[ii[u]]) * scl[jj[u]];
    }
    __syncthreads();   // padding rows / columns of the block matrix hold zeros: the diagonal goes last
    for (int64_t t = pad_off[p] + threadIdx.x; t < pad_off[p + 1]; t += blockDim.x) {
      const int q = padpos[t];
      if (FSI_IN(q, n, FSI_SITE(1))) D[(int64_t)q * n + q] = T(T(1) * srw[q]) * scl[q];
    }
    return;
  }
  for (int64_t t = threadIdx.x; t < (g1 - g0) * BB; t += blockDim.x) {
    const int64_t g = g0 + t / BB;
    const int e = (int)(t % BB);
    int i, j;
    if (!gather_pos(gmap, bo, g, e, B, i, j)) continue;
    if (!FSI_IN(i, n, FSI_SITE(1)) || !FSI_IN(j, n, FSI_SITE(1))) continue;
    D[(int64_t)i * n + j] = T(bsr_val[(int64_t)gmap[3 * g] * BB + e]);
  }
  __syncthreads();
  for (int64_t t = pad_off[p] + threadIdx.x; t < pad_off[p + 1]; t += blockDim.x) {
    const int q = padpos[t];
    if (FSI_IN(q, n, FSI_SITE(1))) D[(int64_t)q * n + q] = T(1);
  }
  __syncthreads();
  T* Dr = dr + idx_off[p];
  T* Dc = dc + idx_off[p];
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
  for (int i = wid; i < n; i += nw) {
    double m = 0.0;
    for (int j = lane; j < n; j += kWarp) m = fmax(m, fabs((double)D[(int64_t)i * n + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const T s = T(pow2_inv(m));
    for (int j = lane; j < n; j += kWarp) D[(int64_t)i * n + j] *= s;
    if (lane == 0) Dr[i] = s;
  }
  __syncthreads();
  // column maxima: 32-column chunks, warps stride over rows (coalesced), then
  // a shared-memory reduction over the warps
  __shared__ double cmax[32][33];
  for (int c0 = 0; c0 < n; c0 += kWarp) {
    const int j = c0 + lane;
    double m = 0.0;
    if (j < n)
      for (int i = wid; i < n; i += nw) m = fmax(m, fabs((double)D[(int64_t)i * n + j]));
    cmax[wid][lane] = m;
    __syncthreads();
    if (wid == 0) {
      double mm = 0.0;
      for (int w = 0; w < nw; ++w) mm = fmax(mm, cmax[w][lane]);
      if (j < n) Dc[j] = T(pow2_inv(mm));
    }
    __syncthreads();
  }
  for (int i = wid; i < n; i += nw)
    for (int j = lane; j < n; j += kWarp) D[(int64_t)i * n + j] *= Dc[j];
}

// Step k pivots on the unused row p with the largest |M[p][k]|; all rows are
// updated from shared-memory copies of row p and column k, so no element is
// read after it was overwritten in the same step.  Rows whose multiplier is
// exactly zero are skipped (most of a Schwarz block is zero early on).  At the
// end M[p_k][q_c] = (B^{-1})[k][c], q the inverse pivot permutation.
template <typename T, bool SMEM>
__global__ void __launch_bounds__(512)
k_patch_gj_t(const int32_t* __restrict__ p_n, const int32_t* __restrict__ p_nown,
             const int64_t* __restrict__ dense_off, const int64_t* __restrict__ own_off,
             const int32_t* __restrict__ own, const int64_t* __restrict__ inv_off, T* __restrict__ dense,
             T* __restrict__ invT, int32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x;
  const int n = p_n[p];
  T* prow = reinterpret_cast<T*>(smem_raw);
  T* pcol = prow + n;
  int* piv = reinterpret_cast<int*>(pcol + n);
  int* qinv = piv + n;
  uint8_t* used = reinterpret_cast<uint8_t*>(qinv + n);
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_sing;
  __shared__ T tile[32][33];
  T* Mg = dense + dense_off[p];
  T* M = Mg;
  if (SMEM) {
    M = reinterpret_cast<T*>(used + ((n + 15) / 16) * 16);
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
      double a = fabs((double)M[(int64_t)i * n + k]);
      if (!(a >= 0.0)) a = 0.0;   // NaN never wins, but an unused row always exists
      if (a > best) { best = a; bi = i; }
    }
    const int pr = block_argmax_abs(best, bi, sv, si);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      prow[j] = M[(int64_t)pr * n + j];
      pcol[j] = M[(int64_t)j * n + k];
    }
    if (threadIdx.x == 0) { used[pr] = 1; piv[k] = pr; }
    __syncthreads();
    T pv = prow[k];
    if (!(fabs((double)pv) > 0.0) || !isfinite((double)pv)) {
      if (threadIdx.x == 0) s_sing = 1;
      pv = T(1);
    }
    const T rp = T(1) / pv;
    for (int i = wid; i < n; i += nw) {
      T* Mi = M + (int64_t)i * n;
      if (i == pr) {
        for (int j = lane; j < n; j += kWarp) Mi[j] = (j == k) ? rp : prow[j] * rp;
      } else {
        const T f = pcol[i] * rp;
        if (f != T(0))
          for (int j = lane; j < n; j += kWarp) Mi[j] = (j == k) ? -f : Mi[j] - f * prow[j];
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (FSI_IN(piv[k], n, FSI_SITE(1))) qinv[piv[k]] = k;
  __syncthreads();
  // owned rows of the inverse, written transposed through a shared tile
  const int nown = p_nown[p];
  const int32_t* ow = own + own_off[p];
  T* out = invT + inv_off[p];
  for (int o0 = 0; o0 < own_pad(nown); o0 += 32) {
    for (int c0 = 0; c0 < n; c0 += 32) {
      for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int oo = t / 32, cc = t % 32;
        const int o = o0 + oo, c = c0 + cc;
        if (o < nown && c < n && FSI_IN(ow[o], n, FSI_SITE(1))) tile[oo][cc] = M[(int64_t)piv[ow[o]] * n + qinv[c]];
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int cc = t / 32, oo = t % 32;
        const int o = o0 + oo, c = c0 + cc;
        if (o < own_pad(nown) && c < n) out[(int64_t)c * own_pad(nown) + o] = o < nown ? tile[oo][cc] : T(0);
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && s_sing) atomicExch(&status[ST_SINGULAR], 1);
}

// Panel-blocked form of the same in-place Gauss-Jordan sweep.  For a panel of
// W columns K = [k0, k0+W): (1) the n x W panel G = M[:, K] is swept in shared
// memory (pivot search and rank-1 updates touch only panel columns); (2) the
// pivot rows P of the panel are read from M (old values) into R; (3) the
// panel is written back; (4) every other column is updated at once by the
// composite transform of the W steps, M[:, rest] += (G - E_P) R[:, rest],
// with E_P the identity columns at the pivot rows - a rank-W update that reads
// and writes each block once per panel instead of once per pivot step.
template <typename T, int W>
__global__ void __launch_bounds__(512)
k_patch_gj_blk(const int32_t* __restrict__ p_n, const int32_t* __restrict__ p_nown,
               const int64_t* __restrict__ dense_off, const int64_t* __restrict__ own_off,
               const int32_t* __restrict__ own, const int64_t* __restrict__ inv_off, T* __restrict__ dense,
               T* __restrict__ invT, int32_t* __restrict__ status, int max_n) {
  constexpr int GS = W + 1;   // padded panel row stride (bank conflicts)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x;
  const int n = p_n[p];
  // regions sized for the largest block of the launch (max_n), so the output
  // tile (32 x 33, placed in G; the host checks max_n * GS >= 32 * 33) never
  // overlaps the pivot arrays, whatever this block's n
  T* G = reinterpret_cast<T*>(smem_raw);              // max_n * GS
  T* R = G + (size_t)max_n * GS;                      // W * max_n
  T* pcol = R + (size_t)W * max_n;                    // max_n
  T* prow = pcol + max_n;                             // W
  int* piv = reinterpret_cast<int*>(prow + W);        // max_n
  int* qinv = piv + max_n;                            // max_n
  uint8_t* used = reinterpret_cast<uint8_t*>(qinv + max_n);   // max_n
  uint8_t* live = used + max_n;                       // max_n: row touched by this panel
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_sing;
  T* M = dense + dense_off[p];
  for (int i = threadIdx.x; i < n; i += blockDim.x) used[i] = 0;
  if (threadIdx.x == 0) s_sing = 0;
  __syncthreads();
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
  for (int k0 = 0; k0 < n; k0 += W) {
    const int wp = min(W, n - k0);
    for (int i = wid; i < n; i += nw)
      for (int m = lane; m < W; m += kWarp) G[i * GS + m] = m < wp ? M[(int64_t)i * n + k0 + m] : T(0);
    __syncthreads();
    for (int m = 0; m < wp; ++m) {
      double best = -1.0;
      int bi = -1;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (used[i]) continue;
        double a = fabs((double)G[i * GS + m]);
        if (!(a >= 0.0)) a = 0.0;
        if (a > best) { best = a; bi = i; }
      }
      const int pr = block_argmax_abs(best, bi, sv, si);
      for (int i = threadIdx.x; i < n; i += blockDim.x) pcol[i] = G[i * GS + m];
      if (threadIdx.x < W) prow[threadIdx.x] = G[pr * GS + threadIdx.x];
      if (threadIdx.x == 0) { used[pr] = 1; piv[k0 + m] = pr; }
      __syncthreads();
      T pv = prow[m];
      if (!(fabs((double)pv) > 0.0) || !isfinite((double)pv)) {
        if (threadIdx.x == 0) s_sing = 1;
        pv = T(1);
      }
      const T rp = T(1) / pv;
      for (int i = wid; i < n; i += nw) {
        if (lane >= wp) continue;
        T* Gi = G + i * GS;
        if (i == pr) {
          Gi[lane] = (lane == m) ? rp : prow[lane] * rp;
        } else {
          const T f = pcol[i] * rp;
          if (f != T(0)) Gi[lane] = (lane == m) ? -f : Gi[lane] - f * prow[lane];
        }
      }
      __syncthreads();
    }
    // old pivot rows, panel write-back, G - E_P, live rows
    for (int m = wid; m < wp; m += nw) {
      const T* Mp = M + (int64_t)piv[k0 + m] * n;
      for (int j = lane; j < n; j += kWarp) R[m * n + j] = Mp[j];
    }
    for (int i = wid; i < n; i += nw)
      if (lane < wp) M[(int64_t)i * n + k0 + lane] = G[i * GS + lane];
    __syncthreads();
    if (threadIdx.x < wp) G[piv[k0 + threadIdx.x] * GS + threadIdx.x] -= T(1);
    __syncthreads();
    for (int i = wid; i < n; i += nw) {
      const bool nz = lane < wp && G[i * GS + lane] != T(0);
      const unsigned any = __ballot_sync(0xffffffffu, nz);
      if (lane == 0) live[i] = any != 0u;
    }
    __syncthreads();
    // trailing rank-wp update, 4 rows per warp pass sharing each R load
    // (the FP64 pipe, not shared memory, bounds this loop on this part)
    for (int g = wid; 4 * g < n; g += nw) {
      const int i0 = 4 * g;
      bool any = false;
#pragma unroll
      for (int r = 0; r < 4; ++r) any |= (i0 + r < n) && live[i0 + r];
      if (!any) continue;
      for (int j = lane; j < n; j += kWarp) {
        if (j >= k0 && j < k0 + wp) continue;
        T acc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = T(0);
        for (int m = 0; m < wp; ++m) {
          const T rv = R[m * n + j];
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (i0 + r < n) acc[r] += G[(i0 + r) * GS + m] * rv;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (i0 + r < n && live[i0 + r]) M[(int64_t)(i0 + r) * n + j] += acc[r];
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (FSI_IN(piv[k], n, FSI_SITE(1))) qinv[piv[k]] = k;
  __syncthreads();
  // owned rows of the inverse, transposed through a shared tile (reuses G)
  T* tile = G;   // 32 x 33
  const int nown = p_nown[p];
  const int32_t* ow = own + own_off[p];
  T* out = invT + inv_off[p];
  for (int o0 = 0; o0 < own_pad(nown); o0 += 32) {
    for (int c0 = 0; c0 < n; c0 += 32) {
      for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int oo = t / 32, cc = t % 32;
        const int o = o0 + oo, c = c0 + cc;
        if (o < nown && c < n && FSI_IN(ow[o], n, FSI_SITE(1)))
          tile[oo * 33 + cc] = M[(int64_t)piv[ow[o]] * n + qinv[c]];
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int cc = t / 32, oo = t % 32;
        const int o = o0 + oo, c = c0 + cc;
        if (o < own_pad(nown) && c < n) out[(int64_t)c * own_pad(nown) + o] = o < nown ? tile[oo * 33 + cc] : T(0);
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && s_sing) atomicExch(&status[ST_SINGULAR], 1);
}

// FP32 panel-blocked Gauss-Jordan, same sweep as k_patch_gj_blk with:
//  * ping-pong panel buffers: step m reads buffer m&1 and writes the other, so
//    a step needs a single barrier; each warp updates its own rows (i = warp
//    mod nw) and, in the same pass, finds its pivot candidate for the next
//    column, published per warp in shared memory;
//  * the trailing rank-32 update reads the transposed panel G'^T and the old
//    pivot rows R with float4 shared-memory loads: 4 rows x 4 columns per
//    thread, 16 FMAs per 2 loads, the global tile prefetched before the loop.
// Requires n % 4 == 0 (true for the 2D block layout, B = 4).
// Panel width W = 32 (one lane per panel column) or 16 for large blocks.
template <int W>
__global__ void __launch_bounds__(1024, 1)
k_patch_gj_f32(const int32_t* __restrict__ p_n, const int32_t* __restrict__ p_nown,
               const int64_t* __restrict__ dense_off, const int64_t* __restrict__ own_off,
               const int32_t* __restrict__ own, const int64_t* __restrict__ inv_off, float* __restrict__ dense,
               float* __restrict__ invT, int32_t* __restrict__ status, int max_n) {
  constexpr int GS = W + 1;
  static_assert(W == 16 || W == 32, "panel width");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x;
  const int n = p_n[p];
  float* Gbuf0 = reinterpret_cast<float*>(smem_raw);          // max_n * GS
  float* Gbuf1 = Gbuf0 + (size_t)max_n * GS;                   // max_n * GS
  float* R = Gbuf1 + (size_t)max_n * GS;                       // W * max_n
  float* cand_v = R + (size_t)W * max_n;                       // 2 * 32
  int* cand_i = reinterpret_cast<int*>(cand_v + 64);           // 2 * 32
  int* piv = cand_i + 64;                                      // max_n
  int* qinv = piv + max_n;                                     // max_n
  uint8_t* used = reinterpret_cast<uint8_t*>(qinv + max_n);   // max_n
  uint8_t* live = used + max_n;                                // max_n
  __shared__ int s_sing;
  float* M = dense + dense_off[p];
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
  for (int i = threadIdx.x; i < n; i += blockDim.x) used[i] = 0;
  if (threadIdx.x == 0) s_sing = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += W) {
    const int wp = min(W, n - k0);
    // panel load (and candidates for its first column)
    float best = -1.f;
    int bi = -1;
    for (int i = wid; i < n; i += nw) {
      const float v = lane < wp ? M[(int64_t)i * n + k0 + lane] : 0.f;
      if (lane < W) Gbuf0[i * GS + lane] = v;
      const float c0 = __shfl_sync(0xffffffffu, v, 0);
      if (!used[i]) {
        float a = fabsf(c0);
        if (!(a >= 0.f)) a = 0.f;
        if (a > best) { best = a; bi = i; }
      }
    }
    if (lane == 0) { cand_v[wid] = best; cand_i[wid] = bi; }
    __syncthreads();
    for (int m = 0; m < wp; ++m) {
      const float* src = (m & 1) ? Gbuf1 : Gbuf0;
      float* dst = (m & 1) ? Gbuf0 : Gbuf1;
      const float* cv = cand_v + (m & 1) * 32;
      const int* ci = cand_i + (m & 1) * 32;
      // final pivot choice: every warp reduces the nw (= 32) warp candidates
      // with shuffles (lane l holds candidate l); same result in every warp
      float bv = lane < nw ? cv[lane] : -1.f;
      int pr = lane < nw ? ci[lane] : -1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, pr, o);
        if (oi >= 0 && (pr < 0 || ov > bv || (ov == bv && oi < pr))) { bv = ov; pr = oi; }
      }
      float pv = src[pr * GS + m];
      if (!(fabsf(pv) > 0.f) || !isfinite(pv)) {
        if (threadIdx.x == 0) s_sing = 1;
        pv = 1.f;
      }
      const float rp = 1.f / pv;
      const float prl = lane < W ? src[pr * GS + lane] : 0.f;
      best = -1.f;
      bi = -1;
      for (int i = wid; i < n; i += nw) {
        const float g = lane < W ? src[i * GS + lane] : 0.f;
        const float f = __shfl_sync(0xffffffffu, g, m) * rp;
        float val;
        if (i == pr) val = (lane == m) ? rp : prl * rp;
        else val = (lane == m) ? -f : g - f * prl;
        if (lane >= wp) val = 0.f;
        if (lane < W) dst[i * GS + lane] = val;
        if (i == pr && lane == 0) used[i] = 1;
        if (m + 1 < wp && i != pr && !used[i]) {
          float a = fabsf(__shfl_sync(0xffffffffu, val, m + 1));
          if (!(a >= 0.f)) a = 0.f;
          if (a > best) { best = a; bi = i; }
        } else {
          __shfl_sync(0xffffffffu, val, 0);   // keep the warp converged on the shuffle
        }
      }
      if (lane == 0) { cand_v[((m + 1) & 1) * 32 + wid] = best; cand_i[((m + 1) & 1) * 32 + wid] = bi; }
      if (threadIdx.x == 0) piv[k0 + m] = pr;
      __syncthreads();
    }
    float* G = (wp & 1) ? Gbuf1 : Gbuf0;     // final panel
    float* Gt = (wp & 1) ? Gbuf0 : Gbuf1;    // (G - E_P)^T, row stride n
    // old pivot rows, panel write-back, transposed G - E_P, live rows
    for (int m = wid; m < wp; m += nw) {
      const float4* Mp = reinterpret_cast<const float4*>(M + (int64_t)piv[k0 + m] * n);
      float4* Rm = reinterpret_cast<float4*>(R + m * n);
      for (int j = lane; j < n / 4; j += kWarp) Rm[j] = Mp[j];
    }
    for (int i = wid; i < n; i += nw) {
      const float g = lane < W ? G[i * GS + lane] : 0.f;
      if (lane < wp) M[(int64_t)i * n + k0 + lane] = g;
      const float gm = (lane < wp && piv[k0 + lane] == i) ? g - 1.f : g;
      if (lane < W) Gt[lane * n + i] = lane < wp ? gm : 0.f;
      const unsigned any = __ballot_sync(0xffffffffu, lane < wp && gm != 0.f);
      if (lane == 0) live[i] = any != 0u;
    }
    __syncthreads();
    // trailing update: rows i0..i0+3 (one float4 of G'^T), columns j..j+3
    const int ngr = n / 4, ncg = n / 4;
    const float inv_ncg = 1.f / (float)ncg;
    for (int t = threadIdx.x; t < ngr * ncg; t += blockDim.x) {
      // t = gr * ncg + cgp without an integer division (exact for t < 2^22)
      const int gr = __float2int_rz(((float)t + 0.5f) * inv_ncg);
      const int cgp = t - gr * ncg;
      const int i0 = 4 * gr, j = 4 * cgp;
      if (!(live[i0] | live[i0 + 1] | live[i0 + 2] | live[i0 + 3])) continue;
      if (j >= k0 && j + 3 < k0 + wp) continue;   // fully inside the panel
      float4 old[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) old[r] = *reinterpret_cast<const float4*>(M + (int64_t)(i0 + r) * n + j);
      float acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
#pragma unroll 8
      for (int m = 0; m < wp; ++m) {
        const float4 gv = *reinterpret_cast<const float4*>(Gt + m * n + i0);   // broadcast in the warp
        const float4 rv = *reinterpret_cast<const float4*>(R + m * n + j);
        const float g4[4] = {gv.x, gv.y, gv.z, gv.w};
        const float r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] += g4[r] * r4[q];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (!live[i0 + r]) continue;
        float4 o = old[r];
        float* ov = reinterpret_cast<float*>(&o);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (!(j + q >= k0 && j + q < k0 + wp)) ov[q] += acc[r][q];
        *reinterpret_cast<float4*>(M + (int64_t)(i0 + r) * n + j) = o;
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (FSI_IN(piv[k], n, FSI_SITE(1))) qinv[piv[k]] = k;
  __syncthreads();
  float* tile = Gbuf0;   // 32 x 33
  const int nown = p_nown[p];
  const int32_t* ow = own + own_off[p];
  float* out = invT + inv_off[p];
  for (int o0 = 0; o0 < own_pad(nown); o0 += 32) {
    for (int c0 = 0; c0 < n; c0 += 32) {
      for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int oo = t / 32, cc = t % 32;
        const int o = o0 + oo, c = c0 + cc;
        if (o < nown && c < n && FSI_IN(ow[o], n, FSI_SITE(1)))
          tile[oo * 33 + cc] = M[(int64_t)piv[ow[o]] * n + qinv[c]];
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int cc = t / 32, oo = t % 32;
        const int o = o0 + oo, c = c0 + cc;
        if (o < own_pad(nown) && c < n) out[(int64_t)c * own_pad(nown) + o] = o < nown ? tile[oo * 33 + cc] : 0.f;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && s_sing) atomicExch(&status[ST_SINGULAR], 1);
}

size_t gj_f32_smem(int max_n, int W) {
  return ((size_t)2 * max_n * (W + 1) + (size_t)W * max_n + 64) * sizeof(float) + 64 * sizeof(int) +
         2 * (size_t)max_n * sizeof(int) + 2 * (size_t)max_n + 64;
}

template <int W>
bool try_gj_f32(int np, int max_n, const int32_t* p_n, const int32_t* p_nown, const int64_t* dense_off,
                const int64_t* own_off, const int32_t* own, const int64_t* inv_off, float* dense, float* invT,
                int32_t* status, cudaStream_t st) {
  const size_t smem = gj_f32_smem(max_n, W);
  if (smem > 225 * 1024 || max_n % 4 != 0 || (size_t)max_n * (W + 1) < 32 * 33) return false;
  cudaFuncSetAttribute(k_patch_gj_f32<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_patch_gj_f32<W><<<np, 1024, smem, st>>>(p_n, p_nown, dense_off, own_off, own, inv_off, dense, invT, status,
                                            max_n);
  return true;
}

// ---------------------------------------------------------------------------
// FP32 Gauss-Jordan with the trailing update on the tensor cores (tcgen05).
//
// Thread i owns row i of the block (n <= 1024).  A panel of W columns is
// factored in registers.  Pivot choice per step: every warp holding rows
// offers its best unused row as a 32-bit key (|entry| with the 10 low
// mantissa bits replaced by 1023 - row, so one integer max-reduction picks
// the largest magnitude, ties to the lowest row) and stores that row's panel
// values in shared memory; every thread reduces the 32 keys to the same
// pivot and updates its own row (one block barrier per step).
// The rank-W update of the whole matrix, M += (G - E_P) R with R the old
// pivot rows, runs as UMMAs on 128 x 128 tiles: A = G - E_P is written by its
// row owners straight into tensor memory (TF32 high and low parts), B = R
// sits in shared memory in K-major layout (high and low parts), and
// D = A_lo B_hi + A_hi B_lo + A_hi B_hi (products at FP32 accuracy) goes to
// one of two accumulators, so the UMMAs of tile t + 1 run while tile t is
// added to M: D is staged through shared memory and each warp adds whole
// rows of it to M with coalesced loads and stores (panel columns excluded).
// Tiles are 128 rows x TN columns.  Tensor memory: the two accumulators in
// columns [0, 2 TN), the A parts of row tile t at 2 TN + 2 W t.  The panel
// width W is what the 512 columns leave room for: W = 32 with TN = 128 up to
// n = 512, W = 16 with TN = 128 or W = 24 with TN = 64 (a third fewer passes
// over M, but half the loads in flight per tile) up to n = 1024.  Requires
// n % 4 == 0.  The waits on the tensor core are bounded; on time-out the
// block records ST_TIMEOUT, stops issuing work and releases its tensor memory.
// ---------------------------------------------------------------------------
// NC: tensor-memory columns of a block (512: one block per SM; 256: two)
template <int W, int TN, int NC = 512>
__host__ __device__ constexpr int gj_tc_max_n() {
  // row tiles whose A parts (2 W columns each) fit beside the accumulators
  return (NC - 2 * TN) / (2 * W) * 128 < 1024 ? (NC - 2 * TN) / (2 * W) * 128 : 1024;
}
template <int W, int TN, int NC = 512>
__host__ __device__ constexpr int gj_tc_threads() { return gj_tc_max_n<W, TN, NC>(); }   // one thread per row
template <int TN>
__host__ __device__ constexpr int gj_stage() { return TN + 4; }   // row stride of the staged tile
// (rows 16-byte aligned for 4-wide accesses; eight consecutive rows start in
// distinct groups of four banks, so a quarter-warp's 4-wide stores of eight
// rows do not conflict)

template <int W, int TN, int NC = 512>
size_t gj_tc_smem(int max_n) {
  const size_t n16 = ((size_t)max_n + 15) / 16 * 16;
  return (2 * n16 * W + 2 * 32 * (size_t)W + 128 * (size_t)gj_stage<TN>()) * sizeof(float) +
         2 * 32 * sizeof(uint32_t) + 2 * (size_t)max_n * sizeof(int) + (size_t)max_n + 64;
}

// pivot key: larger |a| wins, ties to the lower row; 0 = no candidate
__device__ __forceinline__ uint32_t piv_key(float a, int row) {
  uint32_t b = __float_as_uint(fabsf(a));
  if (!(fabsf(a) <= 3.402823466e38f)) b = 0u;   // NaN / Inf never win
  return (b & ~0x3FFu) | (uint32_t)(1023 - row);
}

template <int W, int TN, int NC>
__global__ void __launch_bounds__(gj_tc_threads<W, TN, NC>(), 512 / NC)
k_patch_gj_tc(const GjLevels lv, int32_t* __restrict__ status, int max_n) {
  static_assert(W % 8 == 0 && W >= 16 && W <= 32, "panel width");
  static_assert(TN == 64 || TN == 128, "tile width");
  static_assert(NC == 512 || NC == 256, "tensor-memory columns");
  constexpr int NWARP = gj_tc_threads<W, TN, NC>() / kWarp;   // 16 or 32 warps
  constexpr int CGN = NWARP / 4;                           // column-chunk slots of a tile per lane quarter
  constexpr int CW = TN / CGN > 16 ? TN / CGN : 16;        // chunk width (multiple of 16)
  constexpr int kStage = gj_stage<TN>();
  constexpr int LPR = TN / 4;                              // epilogue lanes per tile row (4 columns each)
  constexpr int RPI = kWarp / LPR;                         // tile rows per warp instruction (1 or 2)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n16 = (max_n + 15) / 16 * 16;
  float* Bhi = reinterpret_cast<float*>(smem_raw);          // n16 x W, K-major
  float* Blo = Bhi + (size_t)n16 * W;
  float* offer_row = Blo + (size_t)n16 * W;                 // [2][32][W] panel values of each warp's offer
  float* stage = offer_row + 2 * 32 * W;                    // 128 x kStage staged accumulator tile
  uint32_t* offer_key = reinterpret_cast<uint32_t*>(stage + 128 * kStage);   // [2][32]
  int* piv = reinterpret_cast<int*>(offer_key + 64);        // max_n
  int* qinv = piv + max_n;                                  // max_n
  uint8_t* live = reinterpret_cast<uint8_t*>(qinv + max_n);  // max_n
  __shared__ __align__(8) uint64_t mbar2[2];
  __shared__ uint32_t tslot;
  __shared__ int s_sing, s_abort;
  // the blocks of several levels share one launch: find this block's level
  int lvl = 0;
  while (lvl + 1 < lv.nlev && (int)blockIdx.x >= lv.l[lvl + 1].first) ++lvl;
  const GjLevel& L = lv.l[lvl];
  const int p = L.sel ? L.sel[(int)blockIdx.x - L.first] : (int)blockIdx.x - L.first;
  const int n = L.p_n[p];
  float* M = L.dense + L.dense_off[p];
  const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
  const int me = threadIdx.x;
  const bool has_row = me < n;
  const bool warp_rows = wid * kWarp < n;     // this warp owns at least one row
  constexpr uint32_t kCols = NC, kD = 2 * TN;
  if (wid == 0) tc::tmem_alloc(&tslot, kCols);
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar2[0], 1);
    tc::mbar_init(&mbar2[1], 1);
    s_sing = 0;
    s_abort = 0;
  }
  if (lane == 0 && !warp_rows) { offer_key[wid] = 0u; offer_key[32 + wid] = 0u; }
  for (int w = NWARP + threadIdx.x; w < 32; w += blockDim.x) { offer_key[w] = 0u; offer_key[32 + w] = 0u; }
  // B rows (matrix columns) beyond n stay zero
  for (int e = threadIdx.x; e < (n16 - n) * W; e += blockDim.x) {
    const int r = n + e / W, k = e % W;
    Bhi[tc::kmajor_off<W>(r, k)] = 0.f;
    Blo[tc::kmajor_off<W>(r, k)] = 0.f;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tslot;
  uint32_t bphase = 0;   // bit b: phase of accumulator b's barrier
  bool used = false;
  const int q = wid % 4, cgi = wid / 4;   // TMEM lane quarter, first column chunk of a tile
  for (int k0 = 0; k0 < n; k0 += W) {
    const int wp = min(W, n - k0);
    float row[W];
#pragma unroll
    for (int c4 = 0; c4 < W / 4; ++c4) {
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (has_row && 4 * c4 < wp) x = *reinterpret_cast<const float4*>(M + (int64_t)me * n + k0 + 4 * c4);
      row[4 * c4] = x.x; row[4 * c4 + 1] = x.y; row[4 * c4 + 2] = x.z; row[4 * c4 + 3] = x.w;
    }
    int my_step = -1;
    if (warp_rows) {   // offers for column 0 of the panel
      const uint32_t key = (has_row && !used) ? piv_key(row[0], me) : 0u;
      const uint32_t best = __reduce_max_sync(0xffffffffu, key);
      if (lane == 0) offer_key[wid] = best;
      if (best != 0u && key == best) {
        float4* dst = reinterpret_cast<float4*>(offer_row + wid * W);
#pragma unroll
        for (int c4 = 0; c4 < W / 4; ++c4)
          dst[c4] = make_float4(row[4 * c4], row[4 * c4 + 1], row[4 * c4 + 2], row[4 * c4 + 3]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < W; ++m) {
      if (m >= wp) break;
      const int par = m & 1;
      if (warp_rows) {
        // the same pivot in every warp: the largest of the 32 offered keys
        const uint32_t best = __reduce_max_sync(0xffffffffu, offer_key[par * 32 + lane]);
        const int bi = best != 0u ? 1023 - (int)(best & 0x3FFu) : 0;   // a row of warp bi / 32
        const float* prow_s = offer_row + (par * 32 + bi / kWarp) * W;
        const float4* src = reinterpret_cast<const float4*>(prow_s);
        float pv = prow_s[m];
        if (best == 0u || !(fabsf(pv) > 0.f) || !isfinite(pv)) {
          if (lane == 0) s_sing = 1;
          pv = 1.f;
        }
        const float rp = 1.f / pv;
        if (has_row) {
          if (me == bi) {
#pragma unroll
            for (int c4 = 0; c4 < W / 4; ++c4) {
              const float4 x = src[c4];
              const float pr4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) row[4 * c4 + e] = (4 * c4 + e == m) ? rp : pr4[e] * rp;
            }
            used = true;
            my_step = m;
          } else {
            const float f = row[m] * rp;
#pragma unroll
            for (int c4 = 0; c4 < W / 4; ++c4) {
              const float4 x = src[c4];
              const float pr4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) row[4 * c4 + e] = (4 * c4 + e == m) ? -f : row[4 * c4 + e] - f * pr4[e];
            }
          }
        }
        if (threadIdx.x == 0) piv[k0 + m] = bi;
        if (m + 1 < wp) {
          const uint32_t key = (has_row && !used) ? piv_key(row[m + 1], me) : 0u;
          const uint32_t wbest = __reduce_max_sync(0xffffffffu, key);
          if (lane == 0) offer_key[(par ^ 1) * 32 + wid] = wbest;
          if (wbest != 0u && key == wbest) {
            float4* dst = reinterpret_cast<float4*>(offer_row + ((par ^ 1) * 32 + wid) * W);
#pragma unroll
            for (int c4 = 0; c4 < W / 4; ++c4)
              dst[c4] = make_float4(row[4 * c4], row[4 * c4 + 1], row[4 * c4 + 2], row[4 * c4 + 3]);
          }
        }
      }
      __syncthreads();
    }
    // B = old pivot rows (k = panel column, row index = matrix column j)
    for (int m = wid; m < W; m += NWARP) {
      const float* Mp = m < wp ? M + (int64_t)piv[k0 + m] * n : nullptr;
      for (int j0 = 0; j0 < n; j0 += 4 * kWarp) {   // four loads in flight per lane
        float b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * kWarp + lane;
          b[u] = (Mp && j < n) ? Mp[j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * kWarp + lane;
          if (j < n) {
            const float hi = tc::to_tf32(b[u]);
            Bhi[tc::kmajor_off<W>(j, m)] = hi;
            Blo[tc::kmajor_off<W>(j, m)] = b[u] - hi;
          }
        }
      }
    }
    // A = G - E_P from the thread's own row into tensor memory; live rows
    const int n128 = (n + 127) / 128 * 128;
    if (wid * kWarp < n128) {
      bool any = false;
      const uint32_t col = kD + 2u * W * (uint32_t)(me / 128);
#pragma unroll
      for (int h = 0; h < W / 8; ++h) {   // 8 columns at a time: hi part, then lo part
        float ahi[8], alo[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int cc = 8 * h + c;
          const float a = (has_row && cc < wp) ? (cc == my_step ? row[cc] - 1.f : row[cc]) : 0.f;
          any |= a != 0.f;
          ahi[c] = tc::to_tf32(a);
          alo[c] = a - ahi[c];
        }
        tc::tmem_st8(tc::taddr(tbase, 32 * q, col + 8 * h), ahi);
        tc::tmem_st8(tc::taddr(tbase, 32 * q, col + W + 8 * h), alo);
      }
      tc::tmem_wait_st();
      if (has_row) live[me] = any;
    }
    __syncthreads();   // every B read of the old pivot rows precedes the write-back
    if (has_row) {
#pragma unroll
      for (int c4 = 0; c4 < W / 4; ++c4)
        if (4 * c4 < wp)
          *reinterpret_cast<float4*>(M + (int64_t)me * n + k0 + 4 * c4) =
              make_float4(row[4 * c4], row[4 * c4 + 1], row[4 * c4 + 2], row[4 * c4 + 3]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // trailing update: tile t's UMMAs into accumulator t % 2, issued one tile
    // ahead of the epilogue that adds the previous tile to M
    {
      const int ntr = (n + 127) / 128, ntcc = (n + TN - 1) / TN, ntiles = ntr * ntcc;
      auto issue = [&](int t) {
        const int i0 = (t / ntcc) * 128, j0 = (t % ntcc) * TN, b = t & 1;
        const int nt = min(TN, (n - j0 + 15) / 16 * 16);
        const uint32_t id = tc::idesc_tf32(128, nt);
        const uint32_t lbo = tc::kmajor_lbo<W>(), sbo = tc::kmajor_sbo<W>();
        const uint32_t ahi = tbase + kD + 2u * W * (uint32_t)(i0 / 128), alo = ahi + W;
        const uint32_t b0 = tc::smem_u32(Bhi) + (uint32_t)(j0 / 8) * sbo;
        const uint32_t b1 = tc::smem_u32(Blo) + (uint32_t)(j0 / 8) * sbo;
        const uint32_t d = tbase + (uint32_t)TN * b;
#pragma unroll
        for (int s8 = 0; s8 < W / 8; ++s8) {
          const uint32_t ko = 256u * s8;   // two core matrices (8 k-values) of B per UMMA
          tc::mma_tf32_ts(d, alo + 8 * s8, tc::smem_desc(b0 + ko, lbo, sbo), id, s8 > 0);
          tc::mma_tf32_ts(d, ahi + 8 * s8, tc::smem_desc(b1 + ko, lbo, sbo), id, 1);
          tc::mma_tf32_ts(d, ahi + 8 * s8, tc::smem_desc(b0 + ko, lbo, sbo), id, 1);
        }
        tc::commit(&mbar2[b]);
      };
      if (threadIdx.x == 0) issue(0);
      constexpr int RPW = 128 / NWARP;   // epilogue rows per warp
      constexpr int NK = RPW / RPI;      // 4-wide accesses per lane and tile
      static_assert(RPW % RPI == 0, "epilogue rows per warp");
      const int c4 = lane % LPR, rsub = lane / LPR;   // the lane's 4 columns and row of an instruction
      for (int t = 0; t < ntiles; ++t) {
        const int i0 = (t / ntcc) * 128, j0 = (t % ntcc) * TN, b = t & 1;
        const int nt = min(TN, (n - j0 + 15) / 16 * 16);
        // the tile's old values (lane l: columns 4 (l % LPR) .. + 3 of a row
        // of its warp) are loaded before waiting for the tile's UMMAs, so
        // their L2 round trip overlaps the tensor-core work and the staging;
        // n, j0 and the panel bounds are multiples of 4, so a 4-wide chunk is
        // wholly inside or outside the matrix and the panel
        const int jc = j0 + 4 * c4;
        const bool col_ok = 4 * c4 < nt && jc < n && !(jc >= k0 && jc < k0 + wp);
        float4 old[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
          const int r = i0 + wid + NWARP * (RPI * k + rsub);
          const bool ok = col_ok && r < n && live[r];
          old[k] = ok ? *reinterpret_cast<const float4*>(M + (int64_t)r * n + jc) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (threadIdx.x == 0) {
          tc::fence_after_sync();
          if (t + 1 < ntiles) issue(t + 1);   // its accumulator was drained in iteration t - 1
          if (!tc::mbar_wait(&mbar2[b], (bphase >> b) & 1u, lv.first_wait)) {
            // one more bounded wait (full limit) for tile t and for tile t + 1
            // before the tensor memory is released
            tc::mbar_wait(&mbar2[b], (bphase >> b) & 1u, kTcWaitIters);
            if (t + 1 < ntiles) tc::mbar_wait(&mbar2[b ^ 1], (bphase >> (b ^ 1)) & 1u, kTcWaitIters);
            s_abort = 1;
          }
        }
        bphase ^= 1u << b;
        __syncthreads();
        if (s_abort) goto done;
        tc::fence_after_sync();
        // accumulator -> shared memory (thread = tile row), 16 columns at a time
        if (i0 + 32 * q < n) {
          for (int cg = cgi; cg * CW < nt; cg += CGN) {
#pragma unroll
            for (int h = 0; h < CW / 16; ++h) {
              float v[16];
              tc::tmem_ld<16>(tc::taddr(tbase, 32 * q, (uint32_t)TN * b + cg * CW + 16 * h), v);
              tc::tmem_wait_ld();
              float4* srow = reinterpret_cast<float4*>(stage + (32 * q + lane) * kStage + cg * CW + 16 * h);
#pragma unroll
              for (int c = 0; c < 4; ++c) srow[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
            }
          }
        }
        tc::fence_before_sync();
        __syncthreads();
        // M += D for live rows, panel columns excluded: 4-wide, a warp
        // instruction covers whole rows (coalesced)
        if (col_ok) {
#pragma unroll
          for (int k = 0; k < NK; ++k) {
            const int rr = wid + NWARP * (RPI * k + rsub), r = i0 + rr;
            if (!(r < n && live[r])) continue;
            const float4 d = *reinterpret_cast<const float4*>(stage + rr * kStage + 4 * c4);
            *reinterpret_cast<float4*>(M + (int64_t)r * n + jc) =
                make_float4(old[k].x + d.x, old[k].y + d.y, old[k].z + d.z, old[k].w + d.w);
          }
        }
      }
    }
    __syncthreads();
  }
  // qinv starts at 0 so that it stays a valid column even if a singular
  // block repeated a pivot row (ST_SINGULAR is reported; the values are void)
  for (int k = threadIdx.x; k < n; k += blockDim.x) qinv[k] = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (FSI_IN(piv[k], n, FSI_SITE(1))) qinv[piv[k]] = k;
  __syncthreads();
  {
    // owned rows of the inverse, transposed: out[c][o] = Binv[own[o]][c]; o is
    // the fastest index (coalesced writes), reads hit rows of M just written
    const int nown = L.p_nown[p], opad = own_pad(nown);
    const int32_t* ow = L.own + L.own_off[p];
    float* out = L.invT + L.inv_off[p];
    int* roff = reinterpret_cast<int*>(stage);   // row offset of B^{-1} row own[o] in M
    for (int o = threadIdx.x; o < nown; o += blockDim.x)
      roff[o] = FSI_IN(ow[o], n, FSI_SITE(1)) ? piv[ow[o]] * n : 0;
    __syncthreads();
    const int tot = n * opad;
    for (int t0 = threadIdx.x; t0 < tot; t0 += 4 * (int)blockDim.x) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + u * blockDim.x;
        const int c = t / opad, o = t - c * opad;
        v[u] = (t < tot && o < nown) ? M[roff[o] + qinv[c]] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < tot) out[t] = v[u];
      }
    }
  }
done:
  tc::fence_before_sync();
  __syncthreads();
  int32_t* const stat = L.status ? L.status : status;   // the block's own instance
  if (s_abort && threadIdx.x == 0) atomicExch(&stat[ST_TIMEOUT], 1);
  tc::fence_after_sync();
  if (wid == 0) tc::tmem_dealloc(tbase, kCols);
  if (threadIdx.x == 0 && s_sing) atomicExch(&stat[ST_SINGULAR], 1);
}

template <int W, int TN, int NC = 512>
bool fits_gj_tc(int max_n) {
  // two blocks per SM (NC = 256) share the SM's 228 KB of shared memory
  const size_t smem = gj_tc_smem<W, TN, NC>(max_n), cap = NC == 512 ? 225 * 1024 : 112 * 1024;
  return !(smem > cap || max_n % 4 != 0 || max_n > gj_tc_max_n<W, TN, NC>() || max_n < 64);
}

template <int W, int TN, int NC = 512>
void run_gj_tc(const GjLevels& lv, int nblocks, int max_n, int32_t* status, cudaStream_t st) {
  const size_t smem = gj_tc_smem<W, TN, NC>(max_n);
  cudaFuncSetAttribute(k_patch_gj_tc<W, TN, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_patch_gj_tc<W, TN, NC><<<nblocks, gj_tc_threads<W, TN, NC>(), smem, st>>>(lv, status, max_n);
}

// 32-column panels where they fit (n <= 512), else 16-column ones on
// 128-column tiles; the 24-column panel on 64-column tiles only when asked
// for: measured on GB300 it is slower (146 against 132 ms for the 6-level
// channel's blocks of 784 unknowns), as the narrower tiles halve the loads
// in flight of the tile epilogue that bounds this kernel
int gj_tc_variant(int max_n, int panel) {
  if (panel == kGjPanelPair && fits_gj_tc<16, 64, 256>(max_n)) return kGjPanelPair;
  if (panel == 16 && fits_gj_tc<16, 128>(max_n)) return 16;
  if (panel == 24 && fits_gj_tc<24, 64>(max_n)) return 24;
  if (fits_gj_tc<32, 128>(max_n)) return 32;
  if (fits_gj_tc<16, 128>(max_n)) return 16;
  if (fits_gj_tc<24, 64>(max_n)) return 24;
  return 0;
}

bool launch_patch_gj_tc_levels(const GjLevels& lv, int nblocks, int max_n, int32_t* status, cudaStream_t st,
                               int panel) {
  if (nblocks <= 0 || lv.nlev < 1 || lv.nlev > kGjMaxLevels) return false;
  switch (gj_tc_variant(max_n, panel)) {
    case 32: run_gj_tc<32, 128>(lv, nblocks, max_n, status, st); return true;
    case 24: run_gj_tc<24, 64>(lv, nblocks, max_n, status, st); return true;
    case 16: run_gj_tc<16, 128>(lv, nblocks, max_n, status, st); return true;
    case kGjPanelPair: run_gj_tc<16, 64, 256>(lv, nblocks, max_n, status, st); return true;
    default: return false;
  }
}

template <typename T, int W>
size_t gj_blk_smem(int n) {
  return (size_t)n * (W + 1) * sizeof(T) + (size_t)W * n * sizeof(T) + (size_t)n * sizeof(T) + W * sizeof(T) +
         2 * (size_t)n * sizeof(int) + 2 * (size_t)n + 64;
}

// owned-row vectors of the apply: 4 rows per thread in FP32, 2 in FP64
template <typename T> struct VecT;
template <> struct VecT<float> {
  using V = float4;
  static constexpr int W = 4;
  static __device__ __forceinline__ void fma(float (&a)[4], const V& v, float r) {
    a[0] += v.x * r; a[1] += v.y * r; a[2] += v.z * r; a[3] += v.w * r;
  }
};
template <> struct VecT<double> {
  using V = double2;
  static constexpr int W = 2;
  static __device__ __forceinline__ void fma(double (&a)[2], const V& v, double r) {
    a[0] += v.x * r; a[1] += v.y * r;
  }
};


// Thread (v, g): owned-row vector v, column group g of CG; the CG partial
// sums of each owned row are combined in shared memory.
template <typename T, int CG>
__global__ void __launch_bounds__(512)
k_patch_apply_t(const int32_t* __restrict__ p_n, const int32_t* __restrict__ p_nown,
                const int64_t* __restrict__ idx_off, const int32_t* __restrict__ idx,
                const int64_t* __restrict__ own_off, const int32_t* __restrict__ own,
                const int64_t* __restrict__ inv_off, const T* __restrict__ invT, const T* __restrict__ r,
                T* __restrict__ x, T omega, const T* __restrict__ dr, const T* __restrict__ dc, int vstride,
                const int32_t* __restrict__ sel, int64_t nv) {
  using VT = VecT<T>;
  constexpr int W = VT::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = sel ? sel[blockIdx.x] : (int)blockIdx.x;
  const int n = p_n[p];
  T* rs = reinterpret_cast<T*>(smem_raw);              // n (padded to 4)
  const int32_t* id = idx + idx_off[p];
  const T* Dr = dr + idx_off[p];
  const T* Dc = dc + idx_off[p];
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    rs[i] = FSI_IN(id[i], nv, FSI_SITE(1)) ? r[id[i]] * Dr[i] : T(0);
  const int nown = p_nown[p];
  const int nvec = own_pad(nown) / W;
  const int32_t* ow = own + own_off[p];
  const typename VT::V* Bi = reinterpret_cast<const typename VT::V*>(invT + inv_off[p]);
  T* partial = rs + ((n + 3) & ~3);                    // CG * vstride * W partial sums
  __syncthreads();
  const int g = threadIdx.x / vstride;                 // column group
  const int vt = threadIdx.x % vstride;
  const int c_lo = (int)(((int64_t)n * g) / CG), c_hi = (int)(((int64_t)n * (g + 1)) / CG);
  for (int v0 = 0; v0 < nvec; v0 += vstride) {
    const int v = v0 + vt;
    T a0[W], a1[W];
#pragma unroll
    for (int q = 0; q < W; ++q) { a0[q] = T(0); a1[q] = T(0); }
    if (v < nvec) {
      int c = c_lo;
      for (; c + 8 <= c_hi; c += 8) {   // eight column loads in flight per thread
        typename VT::V bb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) bb[u] = __ldg(Bi + (int64_t)(c + u) * nvec + v);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          VT::fma(a0, bb[u], rs[c + u]);
          VT::fma(a1, bb[u + 1], rs[c + u + 1]);
        }
      }
      for (; c + 4 <= c_hi; c += 4) {
        const typename VT::V b0 = __ldg(Bi + (int64_t)c * nvec + v);
        const typename VT::V b1 = __ldg(Bi + (int64_t)(c + 1) * nvec + v);
        const typename VT::V b2 = __ldg(Bi + (int64_t)(c + 2) * nvec + v);
        const typename VT::V b3 = __ldg(Bi + (int64_t)(c + 3) * nvec + v);
        VT::fma(a0, b0, rs[c]);
        VT::fma(a1, b1, rs[c + 1]);
        VT::fma(a0, b2, rs[c + 2]);
        VT::fma(a1, b3, rs[c + 3]);
      }
      for (; c < c_hi; ++c) VT::fma(a0, __ldg(Bi + (int64_t)c * nvec + v), rs[c]);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) partial[(g * vstride + vt) * W + q] = a0[q] + a1[q];
    __syncthreads();
    for (int t = threadIdx.x; t < vstride * W; t += blockDim.x) {
      const int o = v0 * W + t;
      if (o < nown) {
        T sum = T(0);
#pragma unroll
        for (int gg = 0; gg < CG; ++gg) sum += partial[gg * vstride * W + t];
        const int k = ow[o];
        if (FSI_IN(k, n, FSI_SITE(1)) && FSI_IN(id[k], nv, FSI_SITE(1))) x[id[k]] += omega * Dc[k] * sum;
      }
    }
    __syncthreads();
  }
}

// one Schwarz block per thread block (the level's own launch)
template <typename T>
__global__ void k_patch_gather_t(const int32_t* __restrict__ p_n, const int64_t* __restrict__ dense_off,
                                 const int64_t* __restrict__ gmap_off, const int32_t* __restrict__ gmap,
                                 const int64_t* __restrict__ boff_off, const int32_t* __restrict__ boff,
                                 const int64_t* __restrict__ pad_off, const int32_t* __restrict__ padpos,
                                 const double* __restrict__ bsr_val, int B, T* __restrict__ dense,
                                 const int64_t* __restrict__ idx_off, T* __restrict__ dr, T* __restrict__ dc) {
  gather_block<T>(blockIdx.x, p_n, dense_off, gmap_off, gmap, boff_off, boff, pad_off, padpos, bsr_val, B, dense,
                  idx_off, dr, dc);
}

// the FP32 gathers of several levels in one launch (thread block i gathers
// block i - first of the level whose range holds i), so that the coarse
// levels' few blocks run beside the finest level's instead of each paying a
// launch of their own
__global__ void __launch_bounds__(512) k_patch_gather_levels(const GatherLevels lv) {
  int l = 0;
  while (l + 1 < lv.nlev && (int)blockIdx.x >= lv.l[l + 1].first) ++l;
  const GatherLevel& G = lv.l[l];
  gather_block<float>((int)blockIdx.x - G.first, G.p_n, G.dense_off, G.gmap_off, G.gmap, G.boff_off, G.boff,
                      G.pad_off, G.padpos, G.bsr_val, lv.B, G.dense, G.idx_off, G.dr, G.dc);
}

void launch_patch_gather_levels(const GatherLevels& lv, int nblocks, cudaStream_t st) {
  if (nblocks <= 0 || lv.nlev < 1) return;
  k_patch_gather_levels<<<nblocks, 512, 0, st>>>(lv);
}


// ---------------------------------------------------------------------------
template <typename T>
void launch_patch_gather_t(int np, const int32_t* p_n, const int64_t* dense_off, const int64_t* gmap_off,
                           const int32_t* gmap, const int64_t* boff_off, const int32_t* boff, const int64_t* pad_off,
                           const int32_t* padpos, const double* bsr_val, int B, T* dense, const int64_t* idx_off,
                           T* dr, T* dc, cudaStream_t st) {
  if (np <= 0) return;
  k_patch_gather_t<T><<<np, 512, 0, st>>>(p_n, dense_off, gmap_off, gmap, boff_off, boff, pad_off, padpos, bsr_val,
                                          B, dense, idx_off, dr, dc);
}

template <typename T, int W>
bool try_gj_blk(int np, int max_n, const int32_t* p_n, const int32_t* p_nown, const int64_t* dense_off,
                const int64_t* own_off, const int32_t* own, const int64_t* inv_off, T* dense, T* invT,
                int32_t* status, cudaStream_t st) {
  const size_t smem = gj_blk_smem<T, W>(max_n);
  if (smem > 220 * 1024 || (size_t)32 * 33 > (size_t)max_n * (W + 1)) return false;
  cudaFuncSetAttribute(k_patch_gj_blk<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_patch_gj_blk<T, W><<<np, 512, smem, st>>>(p_n, p_nown, dense_off, own_off, own, inv_off, dense, invT, status,
                                               max_n);
  return true;
}

template <typename T>
void launch_patch_gj_t(int np, int max_n, const int32_t* p_n, const int32_t* p_nown, const int64_t* dense_off,
                       const int64_t* own_off, const int32_t* own, const int64_t* inv_off, T* dense, T* invT,
                       int32_t* status, bool n_mult4, cudaStream_t st) {
  if (np <= 0) return;
  // small blocks: the whole matrix fits in shared memory (unblocked sweep)
  const size_t base = (size_t)max_n * (2 * sizeof(T) + 2 * sizeof(int)) + ((max_n + 15) / 16) * 16;
  const size_t with_m = base + (size_t)max_n * max_n * sizeof(T);
  if (with_m <= 190 * 1024) {
    cudaFuncSetAttribute(k_patch_gj_t<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)with_m);
    k_patch_gj_t<T, true><<<np, 512, with_m, st>>>(p_n, p_nown, dense_off, own_off, own, inv_off, dense, invT,
                                                   status);
    return;
  }
  // larger blocks: panel-blocked sweep with the widest panel that fits
  if (std::is_same<T, float>::value && n_mult4) {
    float* d = reinterpret_cast<float*>(dense);
    float* o = reinterpret_cast<float*>(invT);
    GjLevels lv{};
    lv.nlev = 1;
    lv.first_wait = kTcWaitIters;
    lv.l[0] = GjLevel{p_n, p_nown, dense_off, own_off, own, inv_off, d, o, status, nullptr, 0};
    if (launch_patch_gj_tc_levels(lv, np, max_n, status, st)) return;
    if (try_gj_f32<32>(np, max_n, p_n, p_nown, dense_off, own_off, own, inv_off, d, o, status, st)) return;
    if (try_gj_f32<16>(np, max_n, p_n, p_nown, dense_off, own_off, own, inv_off, d, o, status, st)) return;
  }
  if (try_gj_blk<T, 32>(np, max_n, p_n, p_nown, dense_off, own_off, own, inv_off, dense, invT, status, st)) return;
  if (try_gj_blk<T, 16>(np, max_n, p_n, p_nown, dense_off, own_off, own, inv_off, dense, invT, status, st)) return;
  if (try_gj_blk<T, 8>(np, max_n, p_n, p_nown, dense_off, own_off, own, inv_off, dense, invT, status, st)) return;
  cudaFuncSetAttribute(k_patch_gj_t<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base);
  k_patch_gj_t<T, false><<<np, 512, base, st>>>(p_n, p_nown, dense_off, own_off, own, inv_off, dense, invT,
                                                status);
}

// Row-sliced variant for levels with few patches, where one block per patch
// leaves most SMs idle and each block streams its inverse alone at the
// latency of one block: block b applies the owned-row vectors
// [s vps, (s + 1) vps) of patch b / S (s = b % S) over all n columns.  Its
// threads form cg column groups of vps lanes; the cg partial sums of each row
// are added in a fixed order, and the slices write disjoint rows of x, so the
// result does not depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(256)
k_patch_apply_rows(const int32_t* __restrict__ p_n, const int32_t* __restrict__ p_nown,
                   const int64_t* __restrict__ idx_off, const int32_t* __restrict__ idx,
                   const int64_t* __restrict__ own_off, const int32_t* __restrict__ own,
                   const int64_t* __restrict__ inv_off, const T* __restrict__ invT, const T* __restrict__ r,
                   T* __restrict__ x, T omega, const T* __restrict__ dr, const T* __restrict__ dc, int S, int vps,
                   int cg, const int32_t* __restrict__ sel, int64_t nv) {
  using VT = VecT<T>;
  constexpr int W = VT::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = sel ? sel[blockIdx.x / S] : (int)(blockIdx.x / S), s = blockIdx.x % S;
  const int nown = p_nown[p];
  const int nvec = own_pad(nown) / W;
  const int v_lo = s * vps;
  if (v_lo >= nvec) return;                            // whole block: before any barrier
  const int v_hi = min(nvec, v_lo + vps);
  const int n = p_n[p];
  T* rs = reinterpret_cast<T*>(smem_raw);              // n (padded to 4)
  const int32_t* id = idx + idx_off[p];
  const T* Dr = dr + idx_off[p];
  const T* Dc = dc + idx_off[p];
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    rs[i] = FSI_IN(id[i], nv, FSI_SITE(1)) ? r[id[i]] * Dr[i] : T(0);
  const int32_t* ow = own + own_off[p];
  const typename VT::V* Bi = reinterpret_cast<const typename VT::V*>(invT + inv_off[p]);
  T* partial = rs + ((n + 3) & ~3);                    // cg * vps * W partial sums
  __syncthreads();
  const int g = threadIdx.x / vps;
  const int vt = threadIdx.x % vps;
  const int v = v_lo + vt;
  T a0[W], a1[W];
#pragma unroll
  for (int q = 0; q < W; ++q) { a0[q] = T(0); a1[q] = T(0); }
  if (g < cg && v < v_hi) {
    const int c_lo = (int)(((int64_t)n * g) / cg), c_hi = (int)(((int64_t)n * (g + 1)) / cg);
    int c = c_lo;
    for (; c + 8 <= c_hi; c += 8) {
      typename VT::V bb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) bb[u] = __ldg(Bi + (int64_t)(c + u) * nvec + v);
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        VT::fma(a0, bb[u], rs[c + u]);
        VT::fma(a1, bb[u + 1], rs[c + u + 1]);
      }
    }
    for (; c < c_hi; ++c) VT::fma(a0, __ldg(Bi + (int64_t)c * nvec + v), rs[c]);
  }
  if (g < cg) {
#pragma unroll
    for (int q = 0; q < W; ++q) partial[(g * vps + vt) * W + q] = a0[q] + a1[q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < (v_hi - v_lo) * W; t += blockDim.x) {
    const int o = v_lo * W + t;
    if (o < nown) {
      T sum = T(0);
      for (int gg = 0; gg < cg; ++gg) sum += partial[gg * vps * W + t];
      const int k = ow[o];
      if (FSI_IN(k, n, FSI_SITE(1)) && FSI_IN(id[k], nv, FSI_SITE(1))) x[id[k]] += omega * Dc[k] * sum;
    }
  }
}

ApplyShape apply_shape(int np, int max_nown, int vec_width, int sm_count, int want_slices, int want_groups) {
  ApplyShape a{0, 1, 0, 4};
  const int nvec = own_pad(max_nown) / vec_width;
  if (np <= 0 || nvec < 2 || want_slices == 1) return a;
  int S;
  if (want_slices >= 2) {
    S = std::min(want_slices, nvec);
  } else {
    // built-in rule: row slices when one block per patch fills less than half
    // of about one wave (four blocks per SM) of the one-block kernel
    const int target = 4 * sm_count;
    if (2 * np >= target) return a;
    S = std::max(1, std::min(nvec, (target + np - 1) / np));
  }
  const int vps = (nvec + S - 1) / S;
  if (S < 2 || vps > 256) return a;
  a.kind = 1;
  a.vps = vps;
  a.slices = (nvec + vps - 1) / vps;
  const int cap = std::max(1, 256 / vps);
  a.groups = want_groups > 0 ? std::min(want_groups, cap) : std::min(32, cap);
  return a;
}

template <typename T>
void launch_patch_apply_t(int np, int64_t nv, int max_n, int max_nown, const int32_t* p_n, const int32_t* p_nown,
                          const int64_t* idx_off, const int32_t* idx, const int64_t* own_off, const int32_t* own,
                          const int64_t* inv_off, const T* invT, const T* r, T* x, double omega, const T* dr,
                          const T* dc, int sm_count, int want_slices, int want_groups, cudaStream_t st,
                          const int32_t* sel) {
  if (np <= 0) return;
  const ApplyShape a = apply_shape(np, max_nown, VecT<T>::W, sm_count, want_slices, want_groups);
  if (a.kind == 1) {
    const int threads = a.vps * a.groups;
    const size_t smem = ((size_t)((max_n + 3) & ~3) + (size_t)a.groups * a.vps * VecT<T>::W) * sizeof(T);
    if (smem > 48 * 1024)   // large blocks (e.g. 16 x 16 elements): opt in to more shared memory
      cudaFuncSetAttribute(k_patch_apply_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_patch_apply_rows<T><<<(unsigned)((int64_t)np * a.slices), threads, smem, st>>>(
        p_n, p_nown, idx_off, idx, own_off, own, inv_off, invT, r, x, T(omega), dr, dc, a.slices, a.vps, a.groups,
        sel, nv);
    return;
  }
  constexpr int CG = 4;                       // column groups per block
  const int nvec = own_pad(max_nown) / VecT<T>::W;
  int vstride = ((nvec + 31) / 32) * 32;      // threads per column group
  if (vstride > 128) vstride = 128;
  const int threads = vstride * CG;
  const size_t smem = ((size_t)((max_n + 3) & ~3) + (size_t)CG * vstride * VecT<T>::W) * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_patch_apply_t<T, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_patch_apply_t<T, CG><<<np, threads, smem, st>>>(p_n, p_nown, idx_off, idx, own_off, own, inv_off, invT, r, x,
                                                    T(omega), dr, dc, vstride, sel, nv);
}

// ---------------------------------------------------------------------------
// ILU(0) of the fluid Schwarz blocks (Sec. 3.3, 4.1: the approximate local
// solver that suffices for fluid subdomains).  The pattern of a block is its
// node / element block pairs (the block-sparse entries gathered from the
// level's Jacobian) plus the diagonal; elimination without pivoting keeps
// every entry outside it at zero.  The gathered block is equilibrated by
// power-of-two row and column scales; ILU(0) commutes with them, so
// B^{-1} r is applied as D_c U~^{-1} L~^{-1} D_r r as for the exact inverses.
// ---------------------------------------------------------------------------
namespace {
constexpr int kIluMaxNb = 352;   // node / element blocks of a Schwarz block: <= 1024 / 3
constexpr int kIluWords = kIluMaxNb / 32;

// pattern bits of block pairs (local block row, local block column)
__device__ __forceinline__ bool ilu_bit(const uint32_t* bm, int bi, int bj) {
  return (bm[bi * kIluWords + (bj >> 5)] >> (bj & 31)) & 1u;
}

__device__ void ilu_mask(uint32_t* bm, int nb, int64_t g0, int64_t g1, const int32_t* __restrict__ gmap) {
  for (int t = threadIdx.x; t < nb * kIluWords; t += blockDim.x) bm[t] = 0u;
  __syncthreads();
  for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const int lr = gmap[3 * g + 1], lc = gmap[3 * g + 2];
    atomicOr(&bm[lr * kIluWords + (lc >> 5)], 1u << (lc & 31));
  }
  __syncthreads();
}
}  // namespace

// the dense offsets and widths of a Schwarz block's node / element blocks
__device__ void ilu_blocks(int16_t* off, int8_t* w, int nb, const int32_t* __restrict__ bo, int n) {
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int32_t v = bo[b];
    const bool ok = FSI_IN((v >> 3) + (v & 7) - 1, n, FSI_SITE(1));
    off[b] = (int16_t)(ok ? v >> 3 : 0);
    w[b] = (int8_t)(ok ? v & 7 : 0);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256)
k_patch_ilu0(const int32_t* __restrict__ sel, const int32_t* __restrict__ p_n, const int64_t* __restrict__ dense_off,
             const int64_t* __restrict__ gmap_off, const int32_t* __restrict__ gmap,
             const int64_t* __restrict__ boff_off, const int32_t* __restrict__ boff, int B,
             float* __restrict__ dense, int32_t* __restrict__ status) {
  __shared__ uint32_t bm[kIluMaxNb * kIluWords];
  __shared__ int16_t rb[kIluMaxNb], cb[kIluMaxNb];   // block rows / columns touching block bk
  __shared__ int16_t s_off[kIluMaxNb];
  __shared__ int8_t s_w[kIluMaxNb];
  __shared__ int nrb, ncb, s_sing;
  const int p = sel[blockIdx.x];
  const int n = p_n[p], nb = (int)(boff_off[p + 1] - boff_off[p]);
  float* D = dense + dense_off[p];
  if (threadIdx.x == 0) s_sing = 0;
  ilu_mask(bm, nb, gmap_off[p], gmap_off[p + 1], gmap);
  ilu_blocks(s_off, s_w, nb, boff + boff_off[p], n);
  for (int bk = 0; bk < nb; ++bk) {
    // candidate block rows (i > k) and columns (j > k): bk itself and the
    // blocks coupled to it in the pattern
    if (threadIdx.x == 0) {
      int a = 0, c = 0;
      rb[a++] = (int16_t)bk;
      cb[c++] = (int16_t)bk;
      for (int b = bk + 1; b < nb; ++b) {
        if (ilu_bit(bm, b, bk)) rb[a++] = (int16_t)b;
        if (ilu_bit(bm, bk, b)) cb[c++] = (int16_t)b;
      }
      nrb = a;
      ncb = c;
    }
    __syncthreads();
    const bool self = ilu_bit(bm, bk, bk);   // a full diagonal block (node block)
    const int nr = nrb * B, nc = ncb * B;
    for (int kk = 0; kk < s_w[bk]; ++kk) {
      const int k = s_off[bk] + kk;
      float* Dk = D + (int64_t)k * n;
      float akk = Dk[k];
      if (!(fabsf(akk) > 0.f) || !isfinite(akk)) {
        if (threadIdx.x == 0) s_sing = 1;
        akk = 1.f;
      }
      const float rk = 1.f / akk;
      // l_ik = a_ik / u_kk
      for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        const int bi = rb[t / B], cr = t % B;
        if (cr >= s_w[bi]) continue;
        const int i = s_off[bi] + cr;
        if (i <= k || (bi == bk && !self)) continue;
        D[(int64_t)i * n + k] *= rk;
      }
      __syncthreads();
      // a_ij -= l_ik u_kj on the pattern
      for (int t = threadIdx.x; t < nr * nc; t += blockDim.x) {
        const int ri = t / nc, ci = t % nc;
        const int bi = rb[ri / B], cr = ri % B, bj = cb[ci / B], cc = ci % B;
        if (cr >= s_w[bi] || cc >= s_w[bj]) continue;
        const int i = s_off[bi] + cr, j = s_off[bj] + cc;
        if (i <= k || j <= k) continue;
        if ((bi == bk || bj == bk) && !self) continue;
        if (!(ilu_bit(bm, bi, bj) || i == j)) continue;
        D[(int64_t)i * n + j] -= D[(int64_t)i * n + k] * Dk[j];
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && s_sing) atomicExch(&status[ST_SINGULAR], 1);
}

// One warp per block: y = D_r r, forward sweep with the unit lower factor and
// backward sweep with the upper factor over node / element block rows, then
// x[own] += omega D_c y.  A block row's entries come from the block's pattern
// (row pointers built on the host, columns ascending): the lower part is the
// entries left of the diagonal block, the upper part those right of it.  The
// factor entries of the next block row (its first 32 coupled blocks, one per
// lane, and its diagonal block) are loaded while the current row is reduced
// and solved, so a row waits on shared memory rather than on a fresh load.
template <int B>
__global__ void __launch_bounds__(32)
k_patch_apply_ilu(const int32_t* __restrict__ sel, const int32_t* __restrict__ p_n,
                  const int32_t* __restrict__ p_nown, const int64_t* __restrict__ idx_off,
                  const int32_t* __restrict__ idx, const int64_t* __restrict__ own_off,
                  const int32_t* __restrict__ own, const int64_t* __restrict__ dense_off,
                  const int64_t* __restrict__ gmap_off, const int32_t* __restrict__ gmap,
                  const int64_t* __restrict__ boff_off, const int32_t* __restrict__ boff,
                  const int32_t* __restrict__ gptr, int max_n, const float* __restrict__ dense,
                  const float* __restrict__ r, float* __restrict__ x, float omega, const float* __restrict__ dr,
                  const float* __restrict__ dc) {
  extern __shared__ __align__(16) unsigned char ilu_smem[];
  const int p = sel[blockIdx.x];
  const int lane = threadIdx.x;
  const int n = p_n[p], nb = (int)(boff_off[p + 1] - boff_off[p]);
  float* y = reinterpret_cast<float*>(ilu_smem);              // max_n
  float* dg = y + max_n;                                       // B x B: the diagonal block
  int16_t* s_off = reinterpret_cast<int16_t*>(dg + B * B);
  int8_t* s_w = reinterpret_cast<int8_t*>(s_off + nb);
  const float* D = dense + dense_off[p];
  const int32_t* id = idx + idx_off[p];
  const float* Dr = dr + idx_off[p];
  const float* Dc = dc + idx_off[p];
  const int32_t* gp = gptr + boff_off[p] + p;                  // nb + 1 row pointers
  const int32_t* gm = gmap + 3 * gmap_off[p];
  const int32_t* bo = boff + boff_off[p];
  for (int b = lane; b < nb; b += 32) {
    const int32_t v = bo[b];
    const bool ok = FSI_IN((v >> 3) + (v & 7) - 1, n, FSI_SITE(1));
    s_off[b] = (int16_t)(ok ? v >> 3 : 0);
    s_w[b] = (int8_t)(ok ? v & 7 : 0);
  }
  for (int i = lane; i < n; i += 32) y[i] = id[i] >= 0 ? Dr[i] * r[id[i]] : 0.f;
  __syncwarp();
  // entry t of block row bi on the given side of the diagonal: its column
  // block (-1: none) and factor values (row-major wi x wk, zero-padded to B x B)
  auto fetch = [&](int bi, int t, bool lower, int& bk, bool& diag, float (&v)[B * B]) {
    bk = -1;
    diag = false;
    const int e0 = gp[bi], e1 = gp[bi + 1];
    if (e0 + t < e1) {
      const int c = gm[3 * (e0 + t) + 2];
      if (FSI_IN(c, nb, FSI_SITE(1))) {
        if (lower ? c < bi : c > bi) bk = c;
        diag = c == bi;
      }
    }
    const int oi = s_off[bi], wi = s_w[bi];
    const int ok = bk >= 0 ? s_off[bk] : 0, wk = bk >= 0 ? s_w[bk] : 0;
#pragma unroll
    for (int rr = 0; rr < B; ++rr)
#pragma unroll
      for (int cc = 0; cc < B; ++cc)
        v[rr * B + cc] = (bk >= 0 && rr < wi && cc < wk) ? D[(int64_t)(oi + rr) * n + ok + cc] : 0.f;
  };
  // entries lane and lane + 32 (< wi * wi <= 36) of block row bi's diagonal block
  auto fetch_diag = [&](int bi, float& d0, float& d1) {
    const int oi = s_off[bi], wi = s_w[bi];
    const int q1 = lane + 32;
    d0 = lane < wi * wi ? D[(int64_t)(oi + lane / wi) * n + oi + lane % wi] : 0.f;
    d1 = q1 < wi * wi ? D[(int64_t)(oi + q1 / wi) * n + oi + q1 % wi] : 0.f;
  };
  for (int dir = 0; dir < 2; ++dir) {   // 0: L (forward), 1: U (backward)
    const bool lower = dir == 0;
    int bk_n;
    bool dd_n;
    float v_n[B * B];
    float dg_n = 0.f, dg_n1 = 0.f;
    if (nb > 0) {
      const int b0 = lower ? 0 : nb - 1;
      fetch(b0, lane, lower, bk_n, dd_n, v_n);
      fetch_diag(b0, dg_n, dg_n1);
    }
    for (int s = 0; s < nb; ++s) {
      const int bi = lower ? s : nb - 1 - s;
      const int oi = s_off[bi], wi = s_w[bi];
      const int bk = bk_n;
      bool has_diag = dd_n;   // the pattern holds block row bi's diagonal block (node blocks)
      float v[B * B];
#pragma unroll
      for (int q = 0; q < B * B; ++q) v[q] = v_n[q];
      if (lane < wi * wi) dg[lane] = dg_n;
      if (lane + 32 < wi * wi) dg[lane + 32] = dg_n1;
      float acc[B];
#pragma unroll
      for (int rr = 0; rr < B; ++rr) acc[rr] = 0.f;
      if (bk >= 0) {
        const int ok = s_off[bk];
#pragma unroll
        for (int rr = 0; rr < B; ++rr)
#pragma unroll
          for (int cc = 0; cc < B; ++cc) acc[rr] += v[rr * B + cc] * (cc < s_w[bk] ? y[ok + cc] : 0.f);
      }
      // coupled blocks beyond the first 32 (3D), loaded now
      for (int t = 32 + lane; t < gp[bi + 1] - gp[bi]; t += 32) {
        int b2;
        bool d2;
        float w2[B * B];
        fetch(bi, t, lower, b2, d2, w2);
        has_diag |= d2;
        if (b2 >= 0) {
          const int o2 = s_off[b2], k2 = s_w[b2];
#pragma unroll
          for (int rr = 0; rr < B; ++rr)
#pragma unroll
            for (int cc = 0; cc < B; ++cc) acc[rr] += w2[rr * B + cc] * (cc < k2 ? y[o2 + cc] : 0.f);
        }
      }
      // the next block row's entries, loaded during the reduction and solve below
      if (s + 1 < nb) {
        const int bn = lower ? bi + 1 : bi - 1;
        fetch(bn, lane, lower, bk_n, dd_n, v_n);
        fetch_diag(bn, dg_n, dg_n1);
      }
      const bool self = __any_sync(0xffffffffu, has_diag);
#pragma unroll
      for (int rr = 0; rr < B; ++rr)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[rr] += __shfl_xor_sync(0xffffffffu, acc[rr], o);
      __syncwarp();
      if (lane == 0) {
        // a block in the pattern with itself (node blocks) is a full diagonal
        // block; otherwise only its diagonal is kept (element blocks)
        for (int q = 0; q < wi; ++q) {
          const int rr = lower ? q : wi - 1 - q;
          const int i = oi + rr;
          float vv = y[i] - acc[rr];
          if (self) {
            if (lower) {
              for (int c = 0; c < rr; ++c) vv -= dg[rr * wi + c] * y[oi + c];
            } else {
              for (int c = rr + 1; c < wi; ++c) vv -= dg[rr * wi + c] * y[oi + c];
            }
          }
          y[i] = lower ? vv : vv / dg[rr * wi + rr];
        }
      }
      __syncwarp();
    }
  }
  const int nown = p_nown[p];
  const int32_t* ow = own + own_off[p];
  for (int o = lane; o < nown; o += 32) {
    const int row = ow[o];
    if (FSI_IN(row, n, FSI_SITE(1)) && id[row] >= 0) x[id[row]] += omega * (Dc[row] * y[row]);
  }
}

void launch_patch_ilu0(int nsel, const int32_t* sel, const int32_t* p_n, const int64_t* dense_off,
                       const int64_t* gmap_off, const int32_t* gmap, const int64_t* boff_off, const int32_t* boff,
                       int B, float* dense, int32_t* status, cudaStream_t st) {
  if (nsel <= 0) return;
  k_patch_ilu0<<<nsel, 256, 0, st>>>(sel, p_n, dense_off, gmap_off, gmap, boff_off, boff, B, dense, status);
}

void launch_patch_apply_ilu(int nsel, int max_n, int max_nb, const int32_t* sel, const int32_t* p_n,
                            const int32_t* p_nown, const int64_t* idx_off, const int32_t* idx, const int64_t* own_off,
                            const int32_t* own, const int64_t* dense_off, const int64_t* gmap_off,
                            const int32_t* gmap, const int64_t* boff_off, const int32_t* boff, const int32_t* gptr,
                            int B, const float* dense, const float* r, float* x, double omega, const float* dr,
                            const float* dc, cudaStream_t st) {
  if (nsel <= 0) return;
  const size_t smem = (size_t)(max_n + 36) * sizeof(float) + (size_t)max_nb * (sizeof(int16_t) + sizeof(int8_t)) + 16;
  if (B == 4)
    k_patch_apply_ilu<4><<<nsel, 32, smem, st>>>(sel, p_n, p_nown, idx_off, idx, own_off, own, dense_off, gmap_off,
                                                 gmap, boff_off, boff, gptr, max_n, dense, r, x, (float)omega, dr, dc);
  else
    k_patch_apply_ilu<6><<<nsel, 32, smem, st>>>(sel, p_n, p_nown, idx_off, idx, own_off, own, dense_off, gmap_off,
                                                 gmap, boff_off, boff, gptr, max_n, dense, r, x, (float)omega, dr, dc);
}

#define FSI_INST(T)                                                                                              \
  template void launch_patch_gather_t<T>(int, const int32_t*, const int64_t*, const int64_t*, const int32_t*,  \
                                         const int64_t*, const int32_t*, const int64_t*, const int32_t*,        \
                                         const double*, int, T*, const int64_t*, T*, T*, cudaStream_t);         \
  template void launch_patch_gj_t<T>(int, int, const int32_t*, const int32_t*, const int64_t*, const int64_t*, \
                                     const int32_t*, const int64_t*, T*, T*, int32_t*, bool, cudaStream_t);     \
  template void launch_patch_apply_t<T>(int, int64_t, int, int, const int32_t*, const int32_t*, const int64_t*,\
                                        const int32_t*, const int64_t*, const int32_t*, const int64_t*,        \
                                        const T*, const T*, T*, double, const T*, const T*, int, int, int,     \
                                        cudaStream_t, const int32_t*);
FSI_INST(double)
FSI_INST(float)
#undef FSI_INST

// the bounds-check build's recorded site of this translation unit (0: none)
FSI_BOUNDS_READER(bounds_site_schwarz)

}  // namespace fsi
