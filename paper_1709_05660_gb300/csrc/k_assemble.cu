// Element-batched residual + exact Jacobian assembly and Galerkin coarsening.
//
// Assembly (Sec. 2.3, 2.5, 3): one thread per (element, unknown j) evaluates
// the element residual in forward-mode dual arithmetic seeded along e_j, so
// it produces column j of the exact element Jacobian (the derivative of the
// discrete residual, as the paper obtains with automatic differentiation)
// and the value of residual row j.  Element matrices are written to an
// element-matrix buffer; a coloured scatter adds them into the block-sparse
// Jacobian (elements of one colour share no node, so no atomics are needed
// and the summation order is fixed).
//
// Galerkin (Sec. 3.2): J_{l-1} = R J_l P is formed element by element.  A
// coarse element matrix is sum_children R_c A_c P_c, where P_c interpolates
// the coarse element's Q2 / P1disc unknowns to the child's and R_c is its
// transpose restricted to equations of the same kind (momentum, solid
// kinematic, ALE) with Dirichlet rows and columns dropped.
#include <cooperative_groups.h>

#include "kernels.h"

namespace fsi {

namespace {

struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double s) { return {a.v * s, a.d * s}; }
__device__ __forceinline__ Dual operator+(Dual a, double s) { return {a.v + s, a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double inv = 1.0 / b.v;
  const double q = a.v * inv;
  return {q, (a.d - b.d * q) * inv};
}
// a / b given inv = 1 / b.v (the same arithmetic as operator/, with the one
// reciprocal shared by several quotients of the same divisor)
__device__ __forceinline__ Dual div_inv(Dual a, Dual b, double inv) {
  const double q = a.v * inv;
  return {q, (a.d - b.d * q) * inv};
}

// 1D quadratic Lagrange basis (nodes -1, 0, 1) and derivative at the three
// Gauss points -sqrt(3/5), 0, sqrt(3/5).
__device__ __forceinline__ double gp(int q) { return q == 0 ? -0.7745966692414834 : (q == 1 ? 0.0 : 0.7745966692414834); }
__device__ __forceinline__ double gw(int q) { return q == 1 ? 8.0 / 9.0 : 5.0 / 9.0; }
__device__ __forceinline__ double L1(int m, double x) {
  return m == 0 ? 0.5 * x * (x - 1.0) : (m == 1 ? 1.0 - x * x : 0.5 * x * (x + 1.0));
}
__device__ __forceinline__ double dL1(int m, double x) { return m == 0 ? x - 0.5 : (m == 1 ? -2.0 * x : x + 0.5); }

constexpr int kDim = 2;
constexpr int kB = 4;           // unknowns per node block
constexpr int kNloc = 9;        // Q2 nodes per element
constexpr int kNN = kB * kNloc; // node unknowns per element
constexpr int kNdofe = kNN + kDim + 1;   // 39
constexpr int kEPB = 4;         // elements per thread block

}  // namespace

// ---------------------------------------------------------------------------
// element residual + Jacobian (2D)
//
// At a quadrature point the weak-form fluxes (stresses, convection, inertia,
// kinematic, ALE and mass terms) depend on the element unknowns only through
// 13 field quantities: d, grad d, u, grad u and p.  Column j of the element
// Jacobian is therefore sum_f (d flux / d field_f) (d field_f / d y_j), where
// d field_f / d y_j is a basis value or gradient of unknown j (nonzero for at
// most three fields).  The kernel differentiates the fluxes along the 13
// field directions with dual numbers (9 points x 13 directions = 117 dual
// evaluations per element, three per thread) and assembles the 39 columns
// from them; the result is the exact Jacobian of the discrete residual, as
// with one dual evaluation per unknown, at about a third of the FP64 work.
// ---------------------------------------------------------------------------
namespace {
constexpr int kQ = 9;            // Gauss points (3 x 3)
constexpr int kNF = 13;          // differentiated fields
constexpr int kNFV = 17;         // + BDF history values (u_old, d_old)
constexpr int kNFVcn = 26;       // Crank-Nicolson: + the t_n fields (u_n, d_n, grad d_n, grad u_n, p_n)
constexpr int kNO = 11;          // flux outputs per point
// fields: 0,1 d_i | 2..5 dd_i/dx_k (2 + 2 i + k) | 6,7 u_i | 8..11 du_i/dx_k (8 + 2 i + k) | 12 p
//         13,14 u-history | 15,16 d-history
// outputs, fluid: 0..3 T_ck (2 c + k) | 4,5 convection_c | 6..9 ALE A_ck (6 + 2 c + k) | 10 mass
//          solid: 0..3 T_ck | 4,5 inertia_c | 6,7 kinematic_c | 10 mass
// (every output carries its quadrature weight; T and A multiply a test gradient
// in reference coordinates scaled by 2 / h, the others a test value)
//         CN: 13,14 u_n | 15,16 d_n | 17..20 d d_n,i/dx_k (17 + 2 i + k) | 21..24 d u_n,i/dx_k | 25 p_n
constexpr size_t asm_elem_doubles(int nfv) { return (size_t)kQ * nfv + (size_t)kQ * kNF * kNO + (size_t)kQ * kNO; }
constexpr size_t kAsmElemDoubles = asm_elem_doubles(kNFV);

// First Piola stress of the incompressible solid (Sec. 2.2):
// P = -p J F^{-T} + 2 C1 J F - 2 C2 J F^{-T} F^{-1} F^{-T}, 2 C1 = mu_s - 2 C2
__device__ __forceinline__ void piola_2d(const Dual (&F)[2][2], const Dual (&Fi)[2][2], Dual J, Dual p,
                                         const PhysParams& pp, Dual (&P)[2][2]) {
  const Dual pJ = p * J;
  const Dual muJ = J * (pp.mu_s - 2.0 * pp.mr_c2);
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int k = 0; k < 2; ++k) P[c][k] = muJ * F[c][k] - pJ * Fi[k][c];
  if (pp.mr_c2 != 0.0) {
    Dual Q[2][2];   // F^{-1} F^{-T}
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) Q[a][b] = Fi[a][0] * Fi[b][0] + Fi[a][1] * Fi[b][1];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int k = 0; k < 2; ++k) P[c][k] = P[c][k] - (Fi[0][c] * Q[0][k] + Fi[1][c] * Q[1][k]) * J * (2.0 * pp.mr_c2);
  }
}
}  // namespace

// MODE: 0 steady, 1 BDF (yold = a1 y_n + a2 y_{n-1}), 2 Crank-Nicolson (yold = y_n)
template <bool SOLID, int MODE>
__global__ void __launch_bounds__(kEPB * kNdofe, 2)
k_assemble_2d(const int32_t* __restrict__ elems, int ne, const double* __restrict__ y,
              const int32_t* __restrict__ elem_nodes, const uint8_t* __restrict__ node_class,
              const double* __restrict__ elem_geo, int64_t n_nodes, PhysParams pp,
              double* __restrict__ Ke, double* __restrict__ Re, int32_t* __restrict__ status) {
  constexpr bool TRANS = MODE != 0;
  constexpr bool CN = MODE == 2;
  constexpr int NFV = CN ? kNFVcn : kNFV;
  __shared__ double s_y[kEPB][kNdofe];
  __shared__ double s_yo[kEPB][kNdofe];
  __shared__ double s_geo[kEPB][2 * kDim];
  __shared__ unsigned s_iface[kEPB];
  __shared__ double s_scl[kEPB][3];   // 2 / hx, 2 / hy, 1 / (hx hy): divided once per element
  __shared__ double s_wq[kEPB][kQ];    // quadrature weights times the Jacobian of the element map
  __shared__ double s_N[kQ][kNloc], s_Dx[kQ][kNloc], s_Dy[kQ][kNloc];   // reference basis at the points
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int le = threadIdx.x / kNdofe;
  const int j = threadIdx.x % kNdofe;
  const int el = blockIdx.x * kEPB + le;
  const bool active = le < kEPB && el < ne;
  const int e = active ? elems[el] : 0;
  for (int t = threadIdx.x; t < kQ * kNloc; t += blockDim.x) {
    const int q = t / kNloc, a = t % kNloc;
    const double xi = gp(q % 3), eta = gp(q / 3);
    const int ia = a % 3, ja = a / 3;
    s_N[q][a] = L1(ia, xi) * L1(ja, eta);
    s_Dx[q][a] = dL1(ia, xi) * L1(ja, eta);
    s_Dy[q][a] = L1(ia, xi) * dL1(ja, eta);
  }
  if (active) {
    if (j < kNN) {
      const int a = j / kB, s = j % kB;
      const int64_t gi = (int64_t)elem_nodes[(int64_t)e * kNloc + a] * kB + s;
      s_y[le][j] = y[gi];
      if (TRANS) s_yo[le][j] = pp.yold[gi];
    } else {
      s_y[le][j] = y[(n_nodes + e) * kB + (j - kNN)];
      if (CN) s_yo[le][j] = pp.yold[(n_nodes + e) * kB + (j - kNN)];
    }
    if (j < 2 * kDim) s_geo[le][j] = elem_geo[(int64_t)e * 2 * kDim + j];
    if (j == 0) {
      unsigned m = 0;
      for (int a = 0; a < kNloc; ++a)
        if (node_class[elem_nodes[(int64_t)e * kNloc + a]] == kIface) m |= 1u << a;
      s_iface[le] = m;
      const double ghx = elem_geo[(int64_t)e * 2 * kDim + 2], ghy = elem_geo[(int64_t)e * 2 * kDim + 3];
      s_scl[le][0] = 2.0 / ghx;
      s_scl[le][1] = 2.0 / ghy;
      s_scl[le][2] = 1.0 / (ghx * ghy);
    }
    if (j < kQ) {
      const double vol_e = elem_geo[(int64_t)e * 2 * kDim + 2] * elem_geo[(int64_t)e * 2 * kDim + 3];
      s_wq[le][j] = gw(j % 3) * gw(j / 3) * vol_e * 0.25;
    }
  }
  __syncthreads();
  const int le_c = le < kEPB ? le : 0;
  double* Fv = reinterpret_cast<double*>(smem_raw) + (size_t)le_c * asm_elem_doubles(NFV);   // [kQ][NFV]
  double* Dd = Fv + kQ * NFV;                                                               // [kQ][kNF][kNO]
  double* Vo = Dd + kQ * kNF * kNO;                                                     // [kQ][kNO]
  const double* ye = s_y[le_c];
  const double* yo = s_yo[le_c];
  const double hx = s_geo[le_c][2], hy = s_geo[le_c][3];
  const double sx = s_scl[le_c][0], sy = s_scl[le_c][1];
  const double vol = hx * hy;
  const double kale = s_scl[le_c][2];

  // 1. field values at the points
  if (active) {
    for (int it = j; it < kQ * NFV; it += kNdofe) {
      const int q = it / NFV, f = it % NFV;
      double v = 0.0;
      if (f == 12) {
        v = ye[kNN] + ye[kNN + 1] * gp(q % 3) + ye[kNN + 2] * gp(q / 3);
      } else if (CN && f == 25) {
        v = yo[kNN] + yo[kNN + 1] * gp(q % 3) + yo[kNN + 2] * gp(q / 3);
      } else if (f < 13 || TRANS) {
        // source component, basis kind (0 value, 1 d/dx, 2 d/dy), history flag
        int comp, kind;
        const double* src = ye;
        if (f < 2) { comp = f; kind = 0; }
        else if (f < 6) { comp = (f - 2) / 2; kind = 1 + (f - 2) % 2; }
        else if (f < 8) { comp = 2 + (f - 6); kind = 0; }
        else if (f < 12) { comp = 2 + (f - 8) / 2; kind = 1 + (f - 8) % 2; }
        else if (f < 15) { comp = 2 + (f - 13); kind = 0; src = yo; }
        else if (f < 17) { comp = f - 15; kind = 0; src = yo; }
        else if (f < 21) { comp = (f - 17) / 2; kind = 1 + (f - 17) % 2; src = yo; }
        else { comp = 2 + (f - 21) / 2; kind = 1 + (f - 21) % 2; src = yo; }
        const double* tb = kind == 0 ? s_N[q] : (kind == 1 ? s_Dx[q] : s_Dy[q]);
#pragma unroll
        for (int a = 0; a < kNloc; ++a) v += src[a * kB + comp] * tb[a];
        if (kind == 1) v *= sx;
        if (kind == 2) v *= sy;
      }
      Fv[q * NFV + f] = v;
    }
  }
  __syncthreads();

  // 2. flux values and their derivatives along each field direction
  bool tangled = false;
  if (active) {
#pragma unroll 1
    for (int it = j; it < kQ * kNF; it += kNdofe) {
      const int q = it / kNF, f = it % kNF;
      const double* fv = Fv + q * NFV;
      double* dout = Dd + (q * kNF + f) * kNO;
      if (!TRANS && f < 2) {   // d itself enters only the BDF terms
#pragma unroll
        for (int o = 0; o < kNO; ++o) dout[o] = 0.0;
        continue;
      }
      const double wq = s_wq[le_c][q];
      Dual gd[2][2], gu[2][2], u[2], ut[2], dt_[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          gd[i][k] = mk(fv[2 + 2 * i + k], f == 2 + 2 * i + k ? 1.0 : 0.0);
          gu[i][k] = mk(fv[8 + 2 * i + k], f == 8 + 2 * i + k ? 1.0 : 0.0);
        }
        u[i] = mk(fv[6 + i], f == 6 + i ? 1.0 : 0.0);
        if (TRANS) {
          const Dual di = mk(fv[i], f == i ? 1.0 : 0.0);
          ut[i] = (u[i] * pp.a0 + fv[13 + i]) * pp.idt;
          dt_[i] = (di * pp.a0 + fv[15 + i]) * pp.idt;
        }
      }
      const Dual p = mk(fv[12], f == 12 ? 1.0 : 0.0);
      Dual F[2][2];
      F[0][0] = gd[0][0] + 1.0; F[0][1] = gd[0][1];
      F[1][0] = gd[1][0];       F[1][1] = gd[1][1] + 1.0;
      const Dual J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
      if (!(J.v > 0.0)) tangled = true;
      Dual Fi[2][2];
      const double iJ = 1.0 / J.v;
      Fi[0][0] = div_inv(F[1][1], J, iJ); Fi[0][1] = div_inv(-F[0][1], J, iJ);
      Fi[1][0] = div_inv(-F[1][0], J, iJ); Fi[1][1] = div_inv(F[0][0], J, iJ);
      Dual out[kNO];
      if (CN) {
        // Crank-Nicolson (Sec. 2.5): stresses and convection averaged over
        // t_{n+1} and t_n, the conservative ALE inertia (rho J u)_{n+1} -
        // (rho J u)_n over dt with -(div w) u averaged, w = (d - d_n) / dt;
        // the t_n state enters as constants (zero derivative)
        const double un[2] = {fv[13], fv[14]};
        Dual Fn[2][2], Fin[2][2], gw[2][2], w[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          w[i] = (mk(fv[i], f == i ? 1.0 : 0.0) + (-fv[15 + i])) * pp.idt;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            Fn[i][k] = mk(fv[17 + 2 * i + k] + (i == k ? 1.0 : 0.0), 0.0);
            gw[i][k] = (gd[i][k] + (-fv[17 + 2 * i + k])) * pp.idt;
          }
        }
        const Dual Jn = Fn[0][0] * Fn[1][1] - Fn[0][1] * Fn[1][0];
        if (!(Jn.v > 0.0)) tangled = true;
        const double iJn = 1.0 / Jn.v;
        Fin[0][0] = div_inv(Fn[1][1], Jn, iJn); Fin[0][1] = div_inv(-Fn[0][1], Jn, iJn);
        Fin[1][0] = div_inv(-Fn[1][0], Jn, iJn); Fin[1][1] = div_inv(Fn[0][0], Jn, iJn);
        const Dual pn = mk(fv[25], 0.0);
        if (SOLID) {
          Dual P1[2][2], Pn[2][2];
          piola_2d(F, Fi, J, p, pp, P1);
          piola_2d(Fn, Fin, Jn, pn, pp, Pn);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int k = 0; k < 2; ++k) out[2 * c + k] = (P1[c][k] + Pn[c][k]) * (0.5 * wq);
            out[4 + c] = (u[c] * J - Jn * un[c]) * (pp.rho_s * pp.idt * wq);
            out[6 + c] = ((u[c] + un[c]) * 0.5 - w[c]) * wq;
          }
          out[8] = mk(0.0, 0.0);
          out[9] = mk(0.0, 0.0);
          out[10] = (J + (-1.0)) * wq;
        } else {
          Dual gx[2][2], gxn[2][2];
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              gx[i][k] = gu[i][0] * Fi[0][k] + gu[i][1] * Fi[1][k];
              gxn[i][k] = Fin[0][k] * fv[21 + 2 * i] + Fin[1][k] * fv[21 + 2 * i + 1];
            }
          Dual sig[2][2], sgn[2][2];
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              sig[i][k] = (gx[i][k] + gx[k][i]) * pp.mu_f;
              sgn[i][k] = (gxn[i][k] + gxn[k][i]) * pp.mu_f;
            }
          sig[0][0] = sig[0][0] - p;
          sig[1][1] = sig[1][1] - p;
          sgn[0][0] = sgn[0][0] - pn;
          sgn[1][1] = sgn[1][1] - pn;
          const Dual divw1 = gw[0][0] * Fi[0][0] + gw[0][1] * Fi[1][0] + gw[1][0] * Fi[0][1] + gw[1][1] * Fi[1][1];
          const Dual divwn =
              gw[0][0] * Fin[0][0] + gw[0][1] * Fin[1][0] + gw[1][0] * Fin[0][1] + gw[1][1] * Fin[1][1];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int k = 0; k < 2; ++k)
              out[2 * c + k] = ((sig[c][0] * Fi[k][0] + sig[c][1] * Fi[k][1]) * J +
                                (sgn[c][0] * Fin[k][0] + sgn[c][1] * Fin[k][1]) * Jn) * (0.5 * wq);
            const Dual conv1 = gx[c][0] * (u[0] - w[0]) + gx[c][1] * (u[1] - w[1]);
            const Dual convn = gxn[c][0] * (-w[0] + un[0]) + gxn[c][1] * (-w[1] + un[1]);
            const Dual val = (u[c] * J - Jn * un[c]) * pp.idt - divw1 * J * u[c] * 0.5 - divwn * Jn * (0.5 * un[c]) +
                             conv1 * J * 0.5 + convn * Jn * 0.5;
            out[4 + c] = val * (pp.rho_f * wq);
#pragma unroll
            for (int k = 0; k < 2; ++k)
              out[6 + 2 * c + k] = (pp.ale_op == 0 ? gd[c][k] + gd[k][c] : gd[c][k]) * (kale * wq);
          }
          out[10] = J * (gx[0][0] + gx[1][1]) * wq;
        }
      } else if (SOLID) {
        // P = J sigma F^{-T} = -p J F^{-T} + 2 C1 J F - 2 C2 J F^{-T} F^{-1} F^{-T}
        // (sigma = -p I + 2 C1 B - 2 C2 B^{-1}, 2 C1 = mu_s - 2 C2; C2 = 0: Neo-Hookean)
        Dual P[2][2];
        piola_2d(F, Fi, J, p, pp, P);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int k = 0; k < 2; ++k) out[2 * c + k] = P[c][k] * wq;
          out[4 + c] = TRANS ? ut[c] * J * (pp.rho_s * wq) : mk(0.0, 0.0);
          out[6 + c] = (TRANS ? u[c] - dt_[c] : u[c]) * wq;
        }
        out[8] = mk(0.0, 0.0);
        out[9] = mk(0.0, 0.0);
        out[10] = (J + (-1.0)) * wq;
      } else {
        Dual gx[2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int k = 0; k < 2; ++k) gx[i][k] = gu[i][0] * Fi[0][k] + gu[i][1] * Fi[1][k];
        Dual sig[2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int k = 0; k < 2; ++k) sig[i][k] = (gx[i][k] + gx[k][i]) * pp.mu_f;
        sig[0][0] = sig[0][0] - p;
        sig[1][1] = sig[1][1] - p;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int k = 0; k < 2; ++k) out[2 * c + k] = (sig[c][0] * Fi[k][0] + sig[c][1] * Fi[k][1]) * J * wq;
          const Dual cv = TRANS ? gx[c][0] * (u[0] - dt_[0]) + gx[c][1] * (u[1] - dt_[1]) + ut[c]
                                : gx[c][0] * u[0] + gx[c][1] * u[1];
          out[4 + c] = cv * J * (pp.rho_f * wq);
#pragma unroll
          for (int k = 0; k < 2; ++k)
            out[6 + 2 * c + k] = (pp.ale_op == 0 ? gd[c][k] + gd[k][c] : gd[c][k]) * (kale * wq);
        }
        out[10] = J * (gx[0][0] + gx[1][1]) * wq;
      }
#pragma unroll
      for (int o = 0; o < kNO; ++o) dout[o] = out[o].d;
      if (f == 12) {   // any direction carries the values
#pragma unroll
        for (int o = 0; o < kNO; ++o) Vo[q * kNO + o] = out[o].v;
      }
    }
  }
  if (tangled) atomicExch(&status[ST_TANGLED], 1);
  __syncthreads();
  if (!active) return;

  // 3. column j (and residual row j): chain rule through the fields, then the
  //    test functions.  Unknown j = (node aj, component sj) touches the fields
  //    value / d/dx / d/dy of its component; pressure unknown pk touches p with
  //    weight psi_pk = (1, xi, eta)[pk].
  const int aj = j < kNN ? j / kB : 0;
  const int sj = j < kNN ? j % kB : -1;
  const int pk = j >= kNN ? j - kNN : -1;
  const int f_val = sj == 0 ? 0 : (sj == 1 ? 1 : (sj == 2 ? 6 : 7));
  const int f_gx = sj < 2 ? 2 + 2 * sj : 8 + 2 * (sj - 2);
  const unsigned iface = s_iface[le];
  const bool ifc_j = (iface >> aj) & 1u;
  double kc[kNdofe];
#pragma unroll
  for (int i = 0; i < kNdofe; ++i) kc[i] = 0.0;
  double vj = 0.0;
#pragma unroll 1
  for (int q = 0; q < kQ; ++q) {
    const double xi = gp(q % 3), eta = gp(q / 3);
    const double* dq = Dd + q * kNF * kNO;
    const double* vq = Vo + q * kNO;
    double dj[kNO];
    double nj = 0.0, gxj = 0.0, gyj = 0.0, psj = 0.0;
    if (pk < 0) {
      nj = s_N[q][aj];
      gxj = s_Dx[q][aj] * sx;
      gyj = s_Dy[q][aj] * sy;
      const double* d0 = dq + f_val * kNO;
      const double* d1 = dq + f_gx * kNO;
      const double* d2 = dq + (f_gx + 1) * kNO;
#pragma unroll
      for (int o = 0; o < kNO; ++o) dj[o] = d0[o] * nj + d1[o] * gxj + d2[o] * gyj;
    } else {
      psj = pk == 0 ? 1.0 : (pk == 1 ? xi : eta);
      const double* d0 = dq + 12 * kNO;
#pragma unroll
      for (int o = 0; o < kNO; ++o) dj[o] = d0[o] * psj;
    }
    // gradient-type outputs pair with reference gradients: fold the 2 / h scale
    dj[0] *= sx; dj[1] *= sy; dj[2] *= sx; dj[3] *= sy;
    if (!SOLID) { dj[6] *= sx; dj[7] *= sy; dj[8] *= sx; dj[9] *= sy; }
#pragma unroll
    for (int a = 0; a < kNloc; ++a) {
      const double Na = s_N[q][a], Xa = s_Dx[q][a], Ya = s_Dy[q][a];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double md = dj[2 * c] * Xa + dj[2 * c + 1] * Ya + dj[4 + c] * Na;
        if (SOLID) {
          kc[a * kB + c] += md;
          kc[a * kB + 2 + c] += dj[6 + c] * Na;
        } else if ((iface >> a) & 1u) {
          // interface node: momentum in the d-row, no ALE row (psi = 0 on the interface)
          kc[a * kB + c] += md;
        } else {
          // fluid node: ALE in the d-row, momentum in the u-row
          kc[a * kB + c] += dj[6 + 2 * c] * Xa + dj[7 + 2 * c] * Ya;
          kc[a * kB + 2 + c] += md;
        }
      }
    }
    kc[kNN] += dj[10];
    kc[kNN + 1] += dj[10] * xi;
    kc[kNN + 2] += dj[10] * eta;
    // residual row j from the flux values
    if (pk < 0) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double mv = vq[2 * c] * gxj + vq[2 * c + 1] * gyj + vq[4 + c] * nj;
        if (SOLID) {
          if (sj == c) vj += mv;
          if (sj == 2 + c) vj += vq[6 + c] * nj;
        } else {
          if (sj == c) vj += ifc_j ? mv : vq[6 + 2 * c] * gxj + vq[7 + 2 * c] * gyj;
          if (sj == 2 + c && !ifc_j) vj += mv;
        }
      }
    } else {
      vj += vq[10] * psj;
    }
  }
  double* K = Ke + (int64_t)e * kNdofe * kNdofe;
#pragma unroll
  for (int i = 0; i < kNdofe; ++i) K[i * kNdofe + j] = kc[i];
  Re[(int64_t)e * kNdofe + j] = vj;
}

// Dirichlet rows -> identity rows; residual r_i = y_i - g_i
__global__ void k_dirichlet(const int32_t* __restrict__ dir_list, int64_t n_dir, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, double* __restrict__ val, int B,
                            const double* __restrict__ y, const double* __restrict__ g, double alpha,
                            double* __restrict__ res) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_dir) return;
  const int32_t i = dir_list[t];
  const int32_t br = i / B, ci = i % B;
  for (int32_t k = rowptr[br]; k < rowptr[br + 1]; ++k) {
    double* v = val + (int64_t)k * B * B + ci * B;
    for (int cj = 0; cj < B; ++cj) v[cj] = (col[k] == br && cj == ci) ? 1.0 : 0.0;
  }
  if (res != nullptr) res[i] = y[i] - alpha * g[i];
}

// ---------------------------------------------------------------------------
// element-wise Galerkin coarsening (2D)
// ---------------------------------------------------------------------------
namespace {
// weight of parent node m at the child's local node i, child side s: the
// 1D quadratic Lagrange basis m at the parent reference coordinate
// -1 + (2 s + i) / 2, i.e. at -1, -1/2, 0 (s = 0) or 0, 1/2, 1 (s = 1); the
// values are exact binary fractions, tabulated so that forming the weights
// costs one product each and no work on the FP64 pipe beyond it
__device__ const double kQw1[2][3][3] = {{{1.0, 0.0, 0.0}, {0.375, 0.75, -0.125}, {0.0, 1.0, 0.0}},
                                         {{0.0, 1.0, 0.0}, {-0.125, 0.75, 0.375}, {0.0, 0.0, 1.0}}};
// nonzero pattern of kQw1: bit (3 s + i) 3 + m
constexpr unsigned kQwNz = (1u << 0) | (7u << 3) | (1u << 7) | (1u << 10) | (7u << 12) | (1u << 17);
__device__ __forceinline__ bool qw_nz(int s, int i, int m) { return (kQwNz >> ((3 * s + i) * 3 + m)) & 1u; }
__device__ __forceinline__ int row_kind(int cls, int slot) {
  if (cls == kFluid) return slot < kDim ? 2 : 0;
  return slot < kDim ? 0 : 1;
}
}  // namespace

__global__ void __launch_bounds__(256)
k_galerkin_2d(int ncx, int ncy, const double* __restrict__ Kf, const int32_t* __restrict__ f_nodes,
              const uint8_t* __restrict__ f_class, const uint8_t* __restrict__ f_dir,
              const int32_t* __restrict__ c_nodes, const uint8_t* __restrict__ c_class,
              const uint8_t* __restrict__ c_dir, double* __restrict__ Kc) {
  __shared__ double sA[kNdofe * kNdofe];
  __shared__ double sT[kNdofe * kNdofe];
  __shared__ double sC[kNdofe * kNdofe];
  __shared__ double wP[kNN * kNloc];        // T[i][(b,s)] = sum_a A[i][(a,s)] wP[(b,s)][a]
  __shared__ double wR[kNN * kNloc * 2];    // C[(b,sc)][J] += sum_a sum_h wR[.][a][h] T[(a, sf_h)][J]
  __shared__ uint8_t c_cls[kNloc], c_msk[kNN], f_cls[kNloc], f_msk[kNN];
  // nonzero entries of each table row (zero weights cost no FP64 work; adding
  // an exact zero would not change the sums)
  __shared__ uint8_t nP[kNN], lP[kNN][kNloc], nR[kNN], lR[kNN][2 * kNloc];
  __shared__ uint8_t nzP[kNN * kNloc], nzR[kNN * kNloc * 2];   // the nonzero pattern of wP and wR
  __shared__ double sQ[2][3][3];
  if (threadIdx.x < 18) (&sQ[0][0][0])[threadIdx.x] = (&kQw1[0][0][0])[threadIdx.x];
  const int E = blockIdx.x;
  const int cx = E % ncx, cy = E / ncx;
  const int fcx = 2 * ncx;
  for (int t = threadIdx.x; t < kNdofe * kNdofe; t += blockDim.x) sC[t] = 0.0;
  if (threadIdx.x < kNloc) c_cls[threadIdx.x] = c_class[c_nodes[(int64_t)E * kNloc + threadIdx.x]];
  if (threadIdx.x < kNN) {
    const int a = threadIdx.x / kB, s = threadIdx.x % kB;
    c_msk[threadIdx.x] = c_dir[(int64_t)c_nodes[(int64_t)E * kNloc + a] * kB + s] ? 0 : 1;
  }
  for (int ch = 0; ch < 4; ++ch) {
    const int sx = ch & 1, sy = ch >> 1;
    const int64_t ef = (2 * cx + sx) + (int64_t)fcx * (2 * cy + sy);
    __syncthreads();
    for (int t = threadIdx.x; t < kNdofe * kNdofe; t += blockDim.x) sA[t] = Kf[ef * kNdofe * kNdofe + t];
    if (threadIdx.x < kNloc) f_cls[threadIdx.x] = f_class[f_nodes[ef * kNloc + threadIdx.x]];
    if (threadIdx.x < kNN) {
      const int a = threadIdx.x / kB, s = threadIdx.x % kB;
      f_msk[threadIdx.x] = f_dir[(int64_t)f_nodes[ef * kNloc + a] * kB + s] ? 0 : 1;
    }
    __syncthreads();
    // weight tables of this child: coarse basis b at the child's node a
    for (int t = threadIdx.x; t < kNN * kNloc; t += blockDim.x) {
      const int J = t / kNloc, a = t % kNloc;        // J = (b, s)
      const int b = J / kB, sl = J % kB;
      const int ax = a % 3, ay = a / 3, bx = b % 3, by = b / 3;
      const bool nq = qw_nz(sx, ax, bx) && qw_nz(sy, ay, by);
      const double q = nq ? sQ[sx][ax][bx] * sQ[sy][ay][by] : 0.0;
      const bool mp = nq && c_msk[J] && f_msk[a * kB + sl];
      wP[t] = mp ? q : 0.0;
      nzP[t] = mp;
      const int comp = sl % kDim;
      const int kc = row_kind(c_cls[b], sl);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int sf = h == 0 ? comp : kDim + comp;
        const bool mr = nq && c_msk[J] && f_msk[a * kB + sf] && row_kind(f_cls[a], sf) == kc;
        wR[t * 2 + h] = mr ? q : 0.0;
        nzR[t * 2 + h] = mr;
      }
    }
    __syncthreads();
    if (threadIdx.x < kNN) {
      const int J = threadIdx.x;
      int np = 0, nq = 0;
      for (int a = 0; a < kNloc; ++a) {
        if (nzP[J * kNloc + a]) lP[J][np++] = (uint8_t)a;
        for (int h = 0; h < 2; ++h)
          if (nzR[(J * kNloc + a) * 2 + h]) lR[J][nq++] = (uint8_t)(2 * a + h);
      }
      nP[J] = (uint8_t)np;
      nR[J] = (uint8_t)nq;
    }
    __syncthreads();
    // T = A_c P_c
    for (int t = threadIdx.x; t < kNdofe * kNdofe; t += blockDim.x) {
      const int i = t / kNdofe, J = t % kNdofe;
      const double* Ai = sA + i * kNdofe;
      double acc = 0.0;
      if (J < kNN) {
        const int sl = J % kB;
        const double* w = wP + J * kNloc;
        for (int q = 0; q < nP[J]; ++q) {
          const int a = lP[J][q];
          acc += Ai[a * kB + sl] * w[a];
        }
      } else {
        const int k = J - kNN;
        // child coefficients: c0 = p0 + sum_d sig_d/2 p_d ; c_d = p_d / 2
        if (k == 0) acc = Ai[kNN];
        else {
          const double sig = k == 1 ? (sx ? 0.5 : -0.5) : (sy ? 0.5 : -0.5);
          acc = Ai[kNN] * sig + Ai[kNN + k] * 0.5;
        }
      }
      sT[t] = acc;
    }
    __syncthreads();
    // C += R_c T
    for (int t = threadIdx.x; t < kNdofe * kNdofe; t += blockDim.x) {
      const int I = t / kNdofe, J = t % kNdofe;
      double acc = 0.0;
      if (I < kNN) {
        const int comp = (I % kB) % kDim;
        const double* w = wR + I * kNloc * 2;
        for (int q = 0; q < nR[I]; ++q) {
          const int ah = lR[I][q], a = ah >> 1, h = ah & 1;
          acc += w[ah] * sT[(a * kB + h * kDim + comp) * kNdofe + J];
        }
      } else {
        const int k = I - kNN;
        if (k == 0) acc = sT[kNN * kNdofe + J];
        else {
          const double sig = k == 1 ? (sx ? 0.5 : -0.5) : (sy ? 0.5 : -0.5);
          acc = sT[kNN * kNdofe + J] * sig + sT[(kNN + k) * kNdofe + J] * 0.5;
        }
      }
      sC[t] += acc;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kNdofe * kNdofe; t += blockDim.x) Kc[(int64_t)E * kNdofe * kNdofe + t] = sC[t];
}

// ---------------------------------------------------------------------------
// 3D: element residual + Jacobian (27-node hexahedra, 166 unknowns)
// ---------------------------------------------------------------------------
namespace {
constexpr int k3Dim = 3;
constexpr int k3B = 6;
constexpr int k3Nloc = 27;
constexpr int k3NN = k3B * k3Nloc;        // 162
constexpr int k3Ndofe = k3NN + k3Dim + 1; // 166
constexpr int k3Fields = 31;              // gd 9, gu 9, u 3, d 3, p 1, u_old 3, d_old 3
constexpr int k3FieldsCN = 50;            // + (Crank-Nicolson) gd_n 31..39, gu_n 40..48, p_n 49
__device__ __forceinline__ int row_kind3(int cls, int slot) {
  if (cls == kFluid) return slot < k3Dim ? 2 : 0;
  return slot < k3Dim ? 0 : 1;
}
}  // namespace

// As in 2D, the fluxes at a quadrature point depend on the element unknowns
// only through the fields (grad d 9, grad u 9, u 3, d 3, p 1: 25 directions
// against 166 unknowns).  k_flux_3d evaluates them along the 25 directions in
// dual arithmetic (27 x 25 = 675 evaluations per element) and stores the
// derivatives and values of the 22 flux outputs; k_assemble_3d then builds
// column j of the exact element Jacobian by the chain rule through the basis
// coefficients of unknown j (its value and three gradient components, or psi
// for a pressure unknown) and the test functions.  The 166 x 166 element
// matrix fills shared memory, so the flux derivatives (119 KB per element)
// pass through a global scratch, one chunk of elements at a time.
namespace {
constexpr int k3Q = 27;
constexpr int k3NF = 25;   // differentiated fields (fv indices 0..24)
constexpr int k3NO = 22;   // outputs: 0..8 T_ck (3 c + k) | 9..11 convection / inertia_c |
                           // solid 12..14 kinematic_c, fluid 12..20 ALE A_ck (12 + 3 c + k) | 21 mass
constexpr size_t k3FluxDoubles = (size_t)k3Q * k3NF * k3NO + (size_t)k3Q * k3NO;   // per element
constexpr int k3Chunk = 1024;                                                      // elements per pass
}  // namespace

size_t assemble_3d_smem() { return ((size_t)k3Ndofe * k3Ndofe + k3Nloc * 4) * sizeof(double); }

size_t assemble_3d_scratch_doubles(int max_ne) {
  return (size_t)std::min(max_ne, k3Chunk) * k3FluxDoubles;
}

// First Piola stress of the incompressible solid (Sec. 2.2), 3D:
// P = -p J F^{-T} + 2 C1 J F - 2 C2 J F^{-T} F^{-1} F^{-T}, 2 C1 = mu_s - 2 C2
__device__ __forceinline__ void piola_3d(const Dual (&F)[3][3], const Dual (&Fi)[3][3], Dual J, Dual p,
                                         const PhysParams& pp, Dual (&P)[3][3]) {
  const Dual pJ = p * J;
  const Dual muJ = J * (pp.mu_s - 2.0 * pp.mr_c2);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) P[c][k] = muJ * F[c][k] - pJ * Fi[k][c];
  if (pp.mr_c2 != 0.0) {
    Dual Q[3][3];   // F^{-1} F^{-T}
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Q[a][b] = Fi[a][0] * Fi[b][0] + Fi[a][1] * Fi[b][1] + Fi[a][2] * Fi[b][2];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        P[c][k] = P[c][k] - (Fi[0][c] * Q[0][k] + Fi[1][c] * Q[1][k] + Fi[2][c] * Q[2][k]) * J * (2.0 * pp.mr_c2);
  }
}

// F^{-1} and det F of a 3 x 3 Dual matrix (cofactors)
__device__ __forceinline__ Dual inv3(const Dual (&F)[3][3], Dual (&Fi)[3][3]) {
  Dual C[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      C[i][k] = F[i1][k1] * F[i2][k2] - F[i1][k2] * F[i2][k1];
    }
  const Dual J = F[0][0] * C[0][0] + F[0][1] * C[0][1] + F[0][2] * C[0][2];
  const double iJ = 1.0 / J.v;
  const Dual rJ = mk(iJ, -J.d * iJ * iJ);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) Fi[i][k] = C[k][i] * rJ;
  return J;
}

// fields at the 27 points, then flux values and derivatives along each field
// MODE: 0 steady, 1 BDF (yold = a1 y_n + a2 y_{n-1}), 2 Crank-Nicolson (yold = y_n)
template <bool SOLID, int MODE>
__global__ void __launch_bounds__(256)
k_flux_3d(const int32_t* __restrict__ elems, const double* __restrict__ y, const int32_t* __restrict__ elem_nodes,
          const double* __restrict__ elem_geo, int64_t n_nodes, PhysParams pp, double* __restrict__ Dg,
          int32_t* __restrict__ status) {
  constexpr bool TRANS = MODE != 0;
  constexpr bool CN = MODE == 2;
  constexpr int NFLD = CN ? k3FieldsCN : k3Fields;
  __shared__ double ye[k3Ndofe], yo[k3Ndofe];
  __shared__ double bt[k3Q][k3Nloc][4];   // physical basis: N, d/dx, d/dy, d/dz
  __shared__ double fvs[k3Q][NFLD];
  __shared__ double geo[2 * k3Dim];
  const int e = elems[blockIdx.x];
  for (int t = threadIdx.x; t < k3Ndofe; t += blockDim.x) {
    if (t < k3NN) {
      const int64_t gi = (int64_t)elem_nodes[(int64_t)e * k3Nloc + t / k3B] * k3B + t % k3B;
      ye[t] = y[gi];
      yo[t] = TRANS ? pp.yold[gi] : 0.0;
    } else {
      ye[t] = y[(n_nodes + e) * k3B + (t - k3NN)];
      yo[t] = CN ? pp.yold[(n_nodes + e) * k3B + (t - k3NN)] : 0.0;
    }
  }
  if (threadIdx.x < 2 * k3Dim) geo[threadIdx.x] = elem_geo[(int64_t)e * 2 * k3Dim + threadIdx.x];
  __syncthreads();
  const double hx = geo[3], hy = geo[4], hz = geo[5];
  const double vol = hx * hy * hz;
  const double kale = 1.0 / vol;
  for (int t = threadIdx.x; t < k3Q * k3Nloc; t += blockDim.x) {
    const int q = t / k3Nloc, a = t % k3Nloc;
    const double xi = gp(q % 3), eta = gp((q / 3) % 3), zeta = gp(q / 9);
    const int ia = a % 3, ja = (a / 3) % 3, ka = a / 9;
    const double lx = L1(ia, xi), ly = L1(ja, eta), lz = L1(ka, zeta);
    bt[q][a][0] = lx * ly * lz;
    bt[q][a][1] = dL1(ia, xi) * ly * lz * (2.0 / hx);
    bt[q][a][2] = lx * dL1(ja, eta) * lz * (2.0 / hy);
    bt[q][a][3] = lx * ly * dL1(ka, zeta) * (2.0 / hz);
  }
  __syncthreads();
  for (int it = threadIdx.x; it < k3Q * NFLD; it += blockDim.x) {
    const int q = it / NFLD, t = it % NFLD;
    double acc = 0.0;
    if (t < 18) {           // gd (t < 9) and gu: d_i / dx_k of d or u
      const int i = (t % 9) / 3, k = t % 3, off = t < 9 ? 0 : 3;
      for (int a = 0; a < k3Nloc; ++a) acc += ye[a * k3B + off + i] * bt[q][a][1 + k];
    } else if (t < 24) {    // u (18..20), d (21..23)
      const int i = (t - 18) % 3, off = t < 21 ? 3 : 0;
      for (int a = 0; a < k3Nloc; ++a) acc += ye[a * k3B + off + i] * bt[q][a][0];
    } else if (t == 24) {   // pressure
      acc = ye[k3NN] + ye[k3NN + 1] * gp(q % 3) + ye[k3NN + 2] * gp((q / 3) % 3) + ye[k3NN + 3] * gp(q / 9);
    } else if (TRANS && t < 31) {     // u_old (25..27), d_old (28..30)
      const int i = (t - 25) % 3, off = t < 28 ? 3 : 0;
      for (int a = 0; a < k3Nloc; ++a) acc += yo[a * k3B + off + i] * bt[q][a][0];
    } else if (CN && t < 49) {        // t_n gradients: d (31..39), u (40..48)
      const int tt = t - 31, i = (tt % 9) / 3, k = tt % 3, off = tt < 9 ? 0 : 3;
      for (int a = 0; a < k3Nloc; ++a) acc += yo[a * k3B + off + i] * bt[q][a][1 + k];
    } else if (CN) {                  // p_n
      acc = yo[k3NN] + yo[k3NN + 1] * gp(q % 3) + yo[k3NN + 2] * gp((q / 3) % 3) + yo[k3NN + 3] * gp(q / 9);
    }
    fvs[q][t] = acc;
  }
  __syncthreads();
  double* De = Dg + (size_t)blockIdx.x * k3FluxDoubles;   // [q][f][o], then values [q][o]
  double* Ve = De + (size_t)k3Q * k3NF * k3NO;
  bool tangled = false;
#pragma unroll 1
  for (int it = threadIdx.x; it < k3Q * k3NF; it += blockDim.x) {
    const int q = it / k3NF, f = it % k3NF;
    double* dout = De + (size_t)(q * k3NF + f) * k3NO;
    if (!TRANS && f >= 21 && f < 24) {   // d itself enters only the BDF terms
      for (int o = 0; o < k3NO; ++o) dout[o] = 0.0;
      continue;
    }
    const double* fv = fvs[q];
    const double wq = gw(q % 3) * gw((q / 3) % 3) * gw(q / 9) * vol * 0.125;
    Dual gd[3][3], u[3], ut[3], dt_[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) gd[i][k] = mk(fv[i * 3 + k], f == i * 3 + k ? 1.0 : 0.0);
      u[i] = mk(fv[18 + i], f == 18 + i ? 1.0 : 0.0);
      if (TRANS) {
        const Dual di = mk(fv[21 + i], f == 21 + i ? 1.0 : 0.0);
        ut[i] = (u[i] * pp.a0 + fv[25 + i]) * pp.idt;
        dt_[i] = (di * pp.a0 + fv[28 + i]) * pp.idt;
      }
    }
    const Dual p = mk(fv[24], f == 24 ? 1.0 : 0.0);
    Dual F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) F[i][k] = i == k ? gd[i][k] + 1.0 : gd[i][k];
    Dual C[3][3];   // cofactors
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        C[i][k] = F[i1][k1] * F[i2][k2] - F[i1][k2] * F[i2][k1];
      }
    const Dual J = F[0][0] * C[0][0] + F[0][1] * C[0][1] + F[0][2] * C[0][2];
    if (!(J.v > 0.0)) tangled = true;
    const double iJ = 1.0 / J.v;
    const Dual rJ = mk(iJ, -J.d * iJ * iJ);   // 1 / J
    Dual Fi[3][3];   // F^{-1} = C^T / J
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) Fi[i][k] = C[k][i] * rJ;
    Dual out[k3NO];
#pragma unroll
    for (int o = 0; o < k3NO; ++o) out[o] = mk(0.0, 0.0);
    if (CN) {
      // Crank-Nicolson (Sec. 2.5), as in the 2D kernel: stresses and convection
      // averaged over t_{n+1} and t_n, conservative ALE inertia, w = (d - d_n) / dt
      Dual Fn[3][3], Fin[3][3], gw[3][3], w[3];
      double un[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        un[i] = fv[25 + i];
        w[i] = (mk(fv[21 + i], f == 21 + i ? 1.0 : 0.0) + (-fv[28 + i])) * pp.idt;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Fn[i][k] = mk(fv[31 + 3 * i + k] + (i == k ? 1.0 : 0.0), 0.0);
          gw[i][k] = (gd[i][k] + (-fv[31 + 3 * i + k])) * pp.idt;
        }
      }
      const Dual Jn = inv3(Fn, Fin);
      if (!(Jn.v > 0.0)) tangled = true;
      const Dual pn = mk(fv[49], 0.0);
      if (SOLID) {
        Dual P1[3][3], Pn[3][3];
        piola_3d(F, Fi, J, p, pp, P1);
        piola_3d(Fn, Fin, Jn, pn, pp, Pn);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int k = 0; k < 3; ++k) out[3 * c + k] = (P1[c][k] + Pn[c][k]) * (0.5 * wq);
          out[9 + c] = (u[c] * J - Jn * un[c]) * (pp.rho_s * pp.idt * wq);
          out[12 + c] = ((u[c] + un[c]) * 0.5 - w[c]) * wq;
        }
        out[21] = (J + (-1.0)) * wq;
      } else {
        Dual gx[3][3], gxn[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const Dual gu0 = mk(fv[9 + i * 3 + 0], f == 9 + i * 3 + 0 ? 1.0 : 0.0);
            const Dual gu1 = mk(fv[9 + i * 3 + 1], f == 9 + i * 3 + 1 ? 1.0 : 0.0);
            const Dual gu2 = mk(fv[9 + i * 3 + 2], f == 9 + i * 3 + 2 ? 1.0 : 0.0);
            gx[i][k] = gu0 * Fi[0][k] + gu1 * Fi[1][k] + gu2 * Fi[2][k];
            gxn[i][k] = Fin[0][k] * fv[40 + 3 * i] + Fin[1][k] * fv[40 + 3 * i + 1] + Fin[2][k] * fv[40 + 3 * i + 2];
          }
        Dual divw1 = mk(0.0, 0.0), divwn = mk(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            divw1 = divw1 + gw[i][k] * Fi[k][i];
            divwn = divwn + gw[i][k] * Fin[k][i];
          }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Dual sig[3], sgn[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            sig[m] = (gx[c][m] + gx[m][c]) * pp.mu_f;
            sgn[m] = (gxn[c][m] + gxn[m][c]) * pp.mu_f;
            if (m == c) {
              sig[m] = sig[m] - p;
              sgn[m] = sgn[m] - pn;
            }
          }
#pragma unroll
          for (int k = 0; k < 3; ++k)
            out[3 * c + k] = ((sig[0] * Fi[k][0] + sig[1] * Fi[k][1] + sig[2] * Fi[k][2]) * J +
                              (sgn[0] * Fin[k][0] + sgn[1] * Fin[k][1] + sgn[2] * Fin[k][2]) * Jn) * (0.5 * wq);
          const Dual conv1 = gx[c][0] * (u[0] - w[0]) + gx[c][1] * (u[1] - w[1]) + gx[c][2] * (u[2] - w[2]);
          const Dual convn = gxn[c][0] * (-w[0] + un[0]) + gxn[c][1] * (-w[1] + un[1]) + gxn[c][2] * (-w[2] + un[2]);
          const Dual val = (u[c] * J - Jn * un[c]) * pp.idt - divw1 * J * u[c] * 0.5 - divwn * Jn * (0.5 * un[c]) +
                           conv1 * J * 0.5 + convn * Jn * 0.5;
          out[9 + c] = val * (pp.rho_f * wq);
#pragma unroll
          for (int k = 0; k < 3; ++k)
            out[12 + 3 * c + k] = (pp.ale_op == 0 ? gd[c][k] + gd[k][c] : gd[c][k]) * (kale * wq);
        }
        out[21] = J * (gx[0][0] + gx[1][1] + gx[2][2]) * wq;
      }
    } else if (SOLID) {
      // P = -p J F^{-T} + 2 C1 J F - 2 C2 J F^{-T} F^{-1} F^{-T}, 2 C1 = mu_s - 2 C2
      const Dual pJ = p * J;
      const Dual muJ = J * (pp.mu_s - 2.0 * pp.mr_c2);
      Dual G[3][3];
      if (pp.mr_c2 != 0.0) {
        Dual Q[3][3];   // F^{-1} F^{-T}
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) Q[a][b] = Fi[a][0] * Fi[b][0] + Fi[a][1] * Fi[b][1] + Fi[a][2] * Fi[b][2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k)
            G[c][k] = (Fi[0][c] * Q[0][k] + Fi[1][c] * Q[1][k] + Fi[2][c] * Q[2][k]) * J * (2.0 * pp.mr_c2);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k) G[c][k] = mk(0.0, 0.0);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * c + k] = (muJ * F[c][k] - pJ * Fi[k][c] - G[c][k]) * wq;
        if (TRANS) out[9 + c] = ut[c] * J * (pp.rho_s * wq);
        out[12 + c] = (TRANS ? u[c] - dt_[c] : u[c]) * wq;
      }
      out[21] = (J + (-1.0)) * wq;
    } else {
      Dual gx[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const Dual gu0 = mk(fv[9 + i * 3 + 0], f == 9 + i * 3 + 0 ? 1.0 : 0.0);
          const Dual gu1 = mk(fv[9 + i * 3 + 1], f == 9 + i * 3 + 1 ? 1.0 : 0.0);
          const Dual gu2 = mk(fv[9 + i * 3 + 2], f == 9 + i * 3 + 2 ? 1.0 : 0.0);
          gx[i][k] = gu0 * Fi[0][k] + gu1 * Fi[1][k] + gu2 * Fi[2][k];
        }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Dual sig[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          sig[m] = (gx[c][m] + gx[m][c]) * pp.mu_f;
          if (m == c) sig[m] = sig[m] - p;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * c + k] = (sig[0] * Fi[k][0] + sig[1] * Fi[k][1] + sig[2] * Fi[k][2]) * J * wq;
        const Dual cv = TRANS
                            ? gx[c][0] * (u[0] - dt_[0]) + gx[c][1] * (u[1] - dt_[1]) + gx[c][2] * (u[2] - dt_[2]) + ut[c]
                            : gx[c][0] * u[0] + gx[c][1] * u[1] + gx[c][2] * u[2];
        out[9 + c] = cv * J * (pp.rho_f * wq);
#pragma unroll
        for (int k = 0; k < 3; ++k)
          out[12 + 3 * c + k] = (pp.ale_op == 0 ? gd[c][k] + gd[k][c] : gd[c][k]) * (kale * wq);
      }
      out[21] = J * (gx[0][0] + gx[1][1] + gx[2][2]) * wq;
    }
#pragma unroll
    for (int o = 0; o < k3NO; ++o) dout[o] = out[o].d;
    if (f == 24) {   // any direction carries the values
#pragma unroll
      for (int o = 0; o < k3NO; ++o) Ve[q * k3NO + o] = out[o].v;
    }
  }
  if (tangled) atomicExch(&status[ST_TANGLED], 1);
}

// One thread block per element; thread j < 166 owns column j of the 166 x 166
// element Jacobian, accumulated in shared memory (no two threads write the
// same entry), and the value of residual row j.
template <bool SOLID>
__global__ void __launch_bounds__(192)
k_assemble_3d(const int32_t* __restrict__ elems, const int32_t* __restrict__ elem_nodes,
              const uint8_t* __restrict__ node_class, const double* __restrict__ elem_geo,
              const double* __restrict__ Dg, double* __restrict__ Ke, double* __restrict__ Re) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* K = reinterpret_cast<double*>(smem_raw);   // [i][j]
  double* bt = K + k3Ndofe * k3Ndofe;                 // per node: N, Gx, Gy, Gz
  __shared__ double geo[2 * k3Dim];
  __shared__ unsigned s_iface;
  const int e = elems[blockIdx.x];
  const int j = threadIdx.x;
  for (int t = threadIdx.x; t < k3Ndofe * k3Ndofe; t += blockDim.x) K[t] = 0.0;
  if (threadIdx.x < 2 * k3Dim) geo[threadIdx.x] = elem_geo[(int64_t)e * 2 * k3Dim + threadIdx.x];
  if (threadIdx.x == 0) {
    unsigned m = 0;
    for (int a = 0; a < k3Nloc; ++a)
      if (node_class[elem_nodes[(int64_t)e * k3Nloc + a]] == kIface) m |= 1u << a;
    s_iface = m;
  }
  __syncthreads();
  const double hx = geo[3], hy = geo[4], hz = geo[5];
  const unsigned iface = s_iface;
  const bool act = j < k3Ndofe;
  const int aj = (act && j < k3NN) ? j / k3B : -1;
  const int sj = (act && j < k3NN) ? j % k3B : -1;
  const int pk = (act && j >= k3NN) ? j - k3NN : -1;
  // the fields unknown j moves: value and gradient of its component, or p
  const int ci = sj >= 3 ? sj - 3 : sj;
  const int f_val = sj < 0 ? 24 : (sj < 3 ? 21 + ci : 18 + ci);
  const int f_grad = sj < 3 ? 3 * ci : 9 + 3 * ci;
  const double* De = Dg + (size_t)blockIdx.x * k3FluxDoubles;
  const double* Ve = De + (size_t)k3Q * k3NF * k3NO;
  double vj = 0.0;
  for (int q = 0; q < k3Q; ++q) {
    const double xi = gp(q % 3), eta = gp((q / 3) % 3), zeta = gp(q / 9);
    if (threadIdx.x < k3Nloc) {
      const int a = threadIdx.x, ia = a % 3, ja = (a / 3) % 3, ka = a / 9;
      const double lx = L1(ia, xi), ly = L1(ja, eta), lz = L1(ka, zeta);
      bt[a * 4 + 0] = lx * ly * lz;
      bt[a * 4 + 1] = dL1(ia, xi) * ly * lz * (2.0 / hx);
      bt[a * 4 + 2] = lx * dL1(ja, eta) * lz * (2.0 / hy);
      bt[a * 4 + 3] = lx * ly * dL1(ka, zeta) * (2.0 / hz);
    }
    __syncthreads();
    if (act) {
      const double* dq = De + (size_t)q * k3NF * k3NO;
      const double* vq = Ve + (size_t)q * k3NO;
      double dj[k3NO];
      double nj = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
      if (pk < 0) {
        nj = bt[aj * 4];
        g0 = bt[aj * 4 + 1];
        g1 = bt[aj * 4 + 2];
        g2 = bt[aj * 4 + 3];
        const double* d0 = dq + f_val * k3NO;
        const double* d1 = dq + f_grad * k3NO;
        const double* d2 = d1 + k3NO;
        const double* d3 = d2 + k3NO;
#pragma unroll
        for (int o = 0; o < k3NO; ++o) dj[o] = d0[o] * nj + d1[o] * g0 + d2[o] * g1 + d3[o] * g2;
      } else {
        const double ps = pk == 0 ? 1.0 : (pk == 1 ? xi : (pk == 2 ? eta : zeta));
        const double* d0 = dq + 24 * k3NO;
#pragma unroll
        for (int o = 0; o < k3NO; ++o) dj[o] = d0[o] * ps;
      }
      for (int a = 0; a < k3Nloc; ++a) {
        const double Na = bt[a * 4], G0 = bt[a * 4 + 1], G1 = bt[a * 4 + 2], G2 = bt[a * 4 + 3];
        const bool ifc = (iface >> a) & 1u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double md = dj[3 * c] * G0 + dj[3 * c + 1] * G1 + dj[3 * c + 2] * G2 + dj[9 + c] * Na;
          const int rd = a * k3B + c, ru = a * k3B + 3 + c;
          if (SOLID) {
            K[rd * k3Ndofe + j] += md;
            K[ru * k3Ndofe + j] += dj[12 + c] * Na;
          } else if (ifc) {
            // interface node: momentum in the d-row, no ALE row (psi = 0 on the interface)
            K[rd * k3Ndofe + j] += md;
          } else {
            // fluid node: ALE in the d-row, momentum in the u-row
            K[rd * k3Ndofe + j] += dj[12 + 3 * c] * G0 + dj[13 + 3 * c] * G1 + dj[14 + 3 * c] * G2;
            K[ru * k3Ndofe + j] += md;
          }
        }
      }
      K[k3NN * k3Ndofe + j] += dj[21];
      K[(k3NN + 1) * k3Ndofe + j] += dj[21] * xi;
      K[(k3NN + 2) * k3Ndofe + j] += dj[21] * eta;
      K[(k3NN + 3) * k3Ndofe + j] += dj[21] * zeta;
      // residual row j from the flux values
      if (pk < 0) {
        const bool ifc = (iface >> aj) & 1u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {   // unrolled select: no dynamic register-array index
          const double mv = vq[3 * c] * g0 + vq[3 * c + 1] * g1 + vq[3 * c + 2] * g2 + vq[9 + c] * nj;
          if (SOLID) {
            if (sj == c) vj += mv;
            if (sj == 3 + c) vj += vq[12 + c] * nj;
          } else {
            if (sj == c) vj += ifc ? mv : vq[12 + 3 * c] * g0 + vq[13 + 3 * c] * g1 + vq[14 + 3 * c] * g2;
            if (sj == 3 + c && !ifc) vj += mv;
          }
        }
      } else {
        vj += vq[21] * (pk == 0 ? 1.0 : (pk == 1 ? xi : (pk == 2 ? eta : zeta)));
      }
    }
    __syncthreads();
  }
  double* Kg = Ke + (int64_t)e * k3Ndofe * k3Ndofe;
  for (int t = threadIdx.x; t < k3Ndofe * k3Ndofe; t += blockDim.x) Kg[t] = K[t];
  if (act) Re[(int64_t)e * k3Ndofe + j] = vj;
}

// Element-wise Galerkin coarsening in 3D.  Per child: T = A_c P_c is formed
// in shared memory from the child's matrix (global, row-major), then the
// coarse element matrix (global, accumulated over the 8 children) gets
// R_c T.  The interpolation weights of a child are products of 1D
// quarter-point weights; each coarse node b keeps the compact list of the
// child nodes a with a nonzero weight (125 of the 27 x 27 pairs), built from
// an 18-entry 1D table, so no FP64 work is spent on zero weights.
size_t galerkin_3d_smem() { return (size_t)k3Ndofe * k3Ndofe * sizeof(double); }

__global__ void __launch_bounds__(512)
k_galerkin_3d(int ncx, int ncy, int ncz, const double* __restrict__ Kf, const int32_t* __restrict__ f_nodes,
              const uint8_t* __restrict__ f_class, const uint8_t* __restrict__ f_dir,
              const int32_t* __restrict__ c_nodes, const uint8_t* __restrict__ c_class,
              const uint8_t* __restrict__ c_dir, double* __restrict__ Kc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* T = reinterpret_cast<double*>(smem_raw);   // [i][J]
  __shared__ double w1[2][3][3];                     // [side][fine 1D][coarse 1D]
  __shared__ double l_w[125];
  __shared__ uint8_t l_a[125];
  __shared__ int l_ptr[k3Nloc + 1];
  __shared__ uint8_t c_cls[k3Nloc], c_msk[k3NN], f_cls[k3Nloc], f_msk[k3NN];
  const int E = blockIdx.x;
  const int cx = E % ncx, cy = (E / ncx) % ncy, cz = E / (ncx * ncy);
  const int fcx = 2 * ncx, fcy = 2 * ncy;
  (void)ncz;
  double* C = Kc + (int64_t)E * k3Ndofe * k3Ndofe;
  for (int t = threadIdx.x; t < k3Ndofe * k3Ndofe; t += blockDim.x) C[t] = 0.0;
  if (threadIdx.x < 18) (&w1[0][0][0])[threadIdx.x] = (&kQw1[0][0][0])[threadIdx.x];
  if (threadIdx.x < k3Nloc) c_cls[threadIdx.x] = c_class[c_nodes[(int64_t)E * k3Nloc + threadIdx.x]];
  if (threadIdx.x < k3NN) {
    const int a = threadIdx.x / k3B, s = threadIdx.x % k3B;
    c_msk[threadIdx.x] = c_dir[(int64_t)c_nodes[(int64_t)E * k3Nloc + a] * k3B + s] ? 0 : 1;
  }
  for (int ch = 0; ch < 8; ++ch) {
    const int sx = ch & 1, sy = (ch >> 1) & 1, sz = ch >> 2;
    const int64_t ef = (2 * cx + sx) + (int64_t)fcx * ((2 * cy + sy) + (int64_t)fcy * (2 * cz + sz));
    const double* A = Kf + ef * k3Ndofe * k3Ndofe;
    __syncthreads();
    if (threadIdx.x < k3Nloc) f_cls[threadIdx.x] = f_class[f_nodes[ef * k3Nloc + threadIdx.x]];
    if (threadIdx.x < k3NN) {
      const int a = threadIdx.x / k3B, s = threadIdx.x % k3B;
      f_msk[threadIdx.x] = f_dir[(int64_t)f_nodes[ef * k3Nloc + a] * k3B + s] ? 0 : 1;
    }
    // nonzero pattern of the child's weights: count per coarse node
    if (threadIdx.x < k3Nloc) {
      const int b = threadIdx.x, mx = b % 3, my = (b / 3) % 3, mz = b / 9;
      int n = 1;
      const int sd[3] = {sx, sy, sz}, mm[3] = {mx, my, mz};
      for (int d = 0; d < 3; ++d) {
        int c = 0;
        for (int i = 0; i < 3; ++i) c += w1[sd[d]][i][mm[d]] != 0.0;
        n *= c;
      }
      l_ptr[b + 1] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      l_ptr[0] = 0;
      for (int b = 0; b < k3Nloc; ++b) l_ptr[b + 1] += l_ptr[b];
    }
    __syncthreads();
    if (threadIdx.x < k3Nloc) {
      const int b = threadIdx.x, mx = b % 3, my = (b / 3) % 3, mz = b / 9;
      int q = l_ptr[b];
      for (int iz = 0; iz < 3; ++iz) {
        const double wz = w1[sz][iz][mz];
        if (wz == 0.0) continue;
        for (int iy = 0; iy < 3; ++iy) {
          const double wy = w1[sy][iy][my];
          if (wy == 0.0) continue;
          for (int ix = 0; ix < 3; ++ix) {
            const double wx = w1[sx][ix][mx];
            if (wx == 0.0) continue;
            l_a[q] = (uint8_t)(ix + 3 * iy + 9 * iz);
            l_w[q] = wx * wy * wz;
            ++q;
          }
        }
      }
    }
    __syncthreads();
    // T = A P  (J fastest: coalesced reads of A's row i)
    for (int t = threadIdx.x; t < k3Ndofe * k3Ndofe; t += blockDim.x) {
      const int i = t / k3Ndofe, J = t % k3Ndofe;
      const double* Ai = A + (int64_t)i * k3Ndofe;
      double acc = 0.0;
      if (J < k3NN) {
        const int b = J / k3B, sl = J % k3B;
        if (c_msk[J])
          for (int q = l_ptr[b]; q < l_ptr[b + 1]; ++q) {
            const int a = l_a[q];
            if (f_msk[a * k3B + sl]) acc += Ai[a * k3B + sl] * l_w[q];
          }
      } else {
        const int k = J - k3NN;
        if (k == 0) acc = Ai[k3NN];
        else {
          const int sd = k == 1 ? sx : (k == 2 ? sy : sz);
          acc = Ai[k3NN] * (sd ? 0.5 : -0.5) + Ai[k3NN + k] * 0.5;
        }
      }
      T[t] = acc;
    }
    __syncthreads();
    // C += R T  (row I uniform across a warp: uniform lists and masks)
    for (int t = threadIdx.x; t < k3Ndofe * k3Ndofe; t += blockDim.x) {
      const int I = t / k3Ndofe, J = t % k3Ndofe;
      double acc = 0.0;
      if (I < k3NN) {
        const int b = I / k3B, sc = I % k3B;
        if (c_msk[I]) {
          const int comp = sc % k3Dim;
          const int kc = row_kind3(c_cls[b], sc);
          for (int q = l_ptr[b]; q < l_ptr[b + 1]; ++q) {
            const int a = l_a[q];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int sf = h == 0 ? comp : k3Dim + comp;
              if (f_msk[a * k3B + sf] && row_kind3(f_cls[a], sf) == kc) acc += l_w[q] * T[(a * k3B + sf) * k3Ndofe + J];
            }
          }
        }
      } else {
        const int k = I - k3NN;
        if (k == 0) acc = T[k3NN * k3Ndofe + J];
        else {
          const int sd = k == 1 ? sx : (k == 2 ? sy : sz);
          acc = T[k3NN * k3Ndofe + J] * (sd ? 0.5 : -0.5) + T[(k3NN + k) * k3Ndofe + J] * 0.5;
        }
      }
      C[t] += acc;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
bool launch_assemble_2d(bool solid, const int32_t* elems, int ne, const double* y, const int32_t* elem_nodes,
                        const uint8_t* node_class, const double* elem_geo, int64_t n_nodes, PhysParams pp,
                        double* Ke, double* Re, int32_t* status, double* scratch, int scratch_ne, cudaStream_t st) {
  (void)scratch;
  (void)scratch_ne;
  if (ne <= 0) return true;
  const int grid = (ne + kEPB - 1) / kEPB;
  const size_t smem = (size_t)kEPB * asm_elem_doubles(pp.transient == 2 ? kNFVcn : kNFV) * sizeof(double);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, kEPB * kNdofe, smem, st>>>(elems, ne, y, elem_nodes, node_class, elem_geo, n_nodes, pp, Ke, Re,
                                           status);
  };
  if (solid) {
    if (pp.transient == 2) go(k_assemble_2d<true, 2>);
    else if (pp.transient) go(k_assemble_2d<true, 1>);
    else go(k_assemble_2d<true, 0>);
  } else {
    if (pp.transient == 2) go(k_assemble_2d<false, 2>);
    else if (pp.transient) go(k_assemble_2d<false, 1>);
    else go(k_assemble_2d<false, 0>);
  }
  return true;
}

// Deterministic gather of the element matrices into the block-sparse values
// and of the element residuals into the residual: one thread per matrix
// entry (or residual entry) sums its element contributions in list order
// (colour-group order, the order of a coloured scatter into zeroed arrays)
// and writes the entry once; padding entries of the pressure blocks get 0.
template <int NLOC, int B, int NDOFE>
__global__ void __launch_bounds__(256) k_gather_blocks(int64_t nnzb, const int32_t* __restrict__ ptr,
                                                       const int32_t* __restrict__ src,
                                                       const double* __restrict__ Ke, double* __restrict__ val) {
  constexpr int NN = NLOC * B, NP = NDOFE - NN, NL1 = NLOC + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb * B * B) return;
  const int64_t blk = t / (B * B);
  const int ij = (int)(t % (B * B)), ci = ij / B, cj = ij % B;
  double v = 0.0;
  const int32_t q1 = ptr[blk + 1];
  for (int32_t q = ptr[blk]; q < q1; ++q) {
    const int32_t sq = src[q];
    const int e = sq / (NL1 * NL1), ab = sq % (NL1 * NL1), a = ab / NL1, b = ab % NL1;
    const int i = a < NLOC ? a * B + ci : (ci < NP ? NN + ci : -1);
    const int j = b < NLOC ? b * B + cj : (cj < NP ? NN + cj : -1);
    if (i >= 0 && j >= 0) v += Ke[(int64_t)e * NDOFE * NDOFE + i * NDOFE + j];
  }
  val[t] = v;
}

template <int NLOC, int B, int NDOFE>
__global__ void __launch_bounds__(256) k_gather_res(int64_t nb, const int32_t* __restrict__ ptr,
                                                    const int32_t* __restrict__ src, const double* __restrict__ Re,
                                                    double* __restrict__ res) {
  constexpr int NN = NLOC * B, NP = NDOFE - NN, NL1 = NLOC + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * B) return;
  const int64_t r = t / B;
  const int ci = (int)(t % B);
  double v = 0.0;
  const int32_t q1 = ptr[r + 1];
  for (int32_t q = ptr[r]; q < q1; ++q) {
    const int32_t sq = src[q];
    const int e = sq / NL1, a = sq % NL1;
    const int i = a < NLOC ? a * B + ci : (ci < NP ? NN + ci : -1);
    if (i >= 0) v += Re[(int64_t)e * NDOFE + i];
  }
  res[t] = v;
}

void launch_gather_elements(int dim, int64_t nnzb, const int32_t* blk_ptr, const int32_t* blk_src, const double* Ke,
                            double* val, int64_t nb, const int32_t* res_ptr, const int32_t* res_src,
                            const double* Re, double* res, cudaStream_t st) {
  if (dim == 2) {
    k_gather_blocks<kNloc, kB, kNdofe><<<(unsigned)((nnzb * kB * kB + 255) / 256), 256, 0, st>>>(nnzb, blk_ptr,
                                                                                              blk_src, Ke, val);
    if (res)
      k_gather_res<kNloc, kB, kNdofe><<<(unsigned)((nb * kB + 255) / 256), 256, 0, st>>>(nb, res_ptr, res_src, Re,
                                                                                        res);
  } else {
    k_gather_blocks<k3Nloc, k3B, k3Ndofe><<<(unsigned)((nnzb * k3B * k3B + 255) / 256), 256, 0, st>>>(
        nnzb, blk_ptr, blk_src, Ke, val);
    if (res)
      k_gather_res<k3Nloc, k3B, k3Ndofe><<<(unsigned)((nb * k3B + 255) / 256), 256, 0, st>>>(nb, res_ptr, res_src,
                                                                                            Re, res);
  }
}

void launch_dirichlet(const int32_t* dir_list, int64_t n_dir, const int32_t* rowptr, const int32_t* col, double* val,
                      int B, const double* y, const double* g, double alpha, double* res, cudaStream_t st) {
  if (n_dir <= 0) return;
  k_dirichlet<<<(unsigned)((n_dir + 255) / 256), 256, 0, st>>>(dir_list, n_dir, rowptr, col, val, B, y, g, alpha,
                                                               res);
}

void launch_galerkin_2d(int ncx, int ncy, const double* Kf, const int32_t* f_nodes, const uint8_t* f_class,
                        const uint8_t* f_dir, const int32_t* c_nodes, const uint8_t* c_class, const uint8_t* c_dir,
                        double* Kc, cudaStream_t st) {
  k_galerkin_2d<<<ncx * ncy, 256, 0, st>>>(ncx, ncy, Kf, f_nodes, f_class, f_dir, c_nodes, c_class, c_dir, Kc);
}

}  // namespace fsi

namespace fsi {

bool launch_assemble_3d(bool solid, const int32_t* elems, int ne, const double* y, const int32_t* elem_nodes,
                        const uint8_t* node_class, const double* elem_geo, int64_t n_nodes, PhysParams pp,
                        double* Ke, double* Re, int32_t* status, double* scratch, int scratch_ne, cudaStream_t st) {
  if (ne <= 0) return true;
  if (std::min(ne, k3Chunk) > scratch_ne) return false;   // the flux scratch holds scratch_ne elements
  const size_t smem = assemble_3d_smem();
  auto go = [&](auto flux, auto cols) {
    cudaFuncSetAttribute(cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int e0 = 0; e0 < ne; e0 += k3Chunk) {
      const int nc = std::min(k3Chunk, ne - e0);
      flux<<<nc, 256, 0, st>>>(elems + e0, y, elem_nodes, elem_geo, n_nodes, pp, scratch, status);
      cols<<<nc, 192, smem, st>>>(elems + e0, elem_nodes, node_class, elem_geo, scratch, Ke, Re);
    }
  };
  if (solid) {
    if (pp.transient == 2) go(k_flux_3d<true, 2>, k_assemble_3d<true>);
    else if (pp.transient) go(k_flux_3d<true, 1>, k_assemble_3d<true>);
    else go(k_flux_3d<true, 0>, k_assemble_3d<true>);
  } else {
    if (pp.transient == 2) go(k_flux_3d<false, 2>, k_assemble_3d<false>);
    else if (pp.transient) go(k_flux_3d<false, 1>, k_assemble_3d<false>);
    else go(k_flux_3d<false, 0>, k_assemble_3d<false>);
  }
  return true;
}

// FP64 operations executed per element (2 per DFMA, 1 per DMUL / DADD) by the
// element-matrix kernels, counted with ncu on GB300 (sm_103a build of these
// kernels) for each dimension, material and time discretisation (0 steady,
// 1 BDF, 2 Crank-Nicolson; Mooney-Rivlin adds a few percent in the solid);
// used for the FP64-ALU fraction of the assembly in the per-class timings.
double assemble_flops_per_element(int dim, bool solid, int mode) {
  static const double f2[2][3] = {{113705.0, 121355.0, 155816.0}, {85909.0, 92740.0, 104785.0}};
  // 3D: flux derivatives + columns
  static const double f3[2][3] = {{437386.0 + 5908383.0, 539270.0 + 5908383.0, 1057103.0 + 5908383.0},
                                  {242394.0 + 4286875.0, 313563.0 + 4286875.0, 502750.0 + 4286875.0}};
  mode = mode < 0 ? 0 : (mode > 2 ? 2 : mode);
  return dim == 2 ? f2[solid][mode] : f3[solid][mode];
}
// the same count for the Galerkin kernels, per coarse element (2D: the
// 5-level channel's finest coarsening, 4,096 coarse elements, with the
// tabulated child weights)
double galerkin_flops_per_coarse_element(int dim) { return dim == 2 ? 69340.0 : 3030039.0; }

int assemble_launches(int dim, int ne) { return dim == 2 || ne <= 0 ? (ne > 0) : 2 * ((ne + k3Chunk - 1) / k3Chunk); }

void launch_galerkin_3d(int ncx, int ncy, int ncz, const double* Kf, const int32_t* f_nodes, const uint8_t* f_class,
                        const uint8_t* f_dir, const int32_t* c_nodes, const uint8_t* c_class, const uint8_t* c_dir,
                        double* Kc, cudaStream_t st) {
  const size_t smem = galerkin_3d_smem();
  cudaFuncSetAttribute(k_galerkin_3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_galerkin_3d<<<ncx * ncy * ncz, 512, smem, st>>>(ncx, ncy, ncz, Kf, f_nodes, f_class, f_dir, c_nodes, c_class,
                                                     c_dir, Kc);
}

}  // namespace fsi
