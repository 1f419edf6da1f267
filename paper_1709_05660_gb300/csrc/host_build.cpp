// Host-side hierarchy builder: tensor mesh levels by midpoint refinement
// (Sec. 3.2), node classes and Dirichlet data (Sec. 2.3, 3.1, 4), the
// block-sparse FE-graph pattern, element colouring for conflict-free scatter,
// the grid transfer matrices (Sec. 3.2) and the Schwarz blocks (Sec. 3.3).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <stdexcept>

#include "fsi_internal.h"

namespace fsi {

namespace {

std::vector<double> refine(const double* b, int n, int times) {
  std::vector<double> v(b, b + n);
  for (int t = 0; t < times; ++t) {
    std::vector<double> w(2 * v.size() - 1);
    for (size_t i = 0; i < v.size(); ++i) w[2 * i] = v[i];
    for (size_t i = 0; i + 1 < v.size(); ++i) w[2 * i + 1] = (v[i] + v[i + 1]) / 2.0;
    v.swap(w);
  }
  return v;
}

// Q2 node coordinate along one axis (vertices and cell midpoints).
double q2_coord(const std::vector<double>& v, int i) {
  if (i % 2 == 0) return v[i / 2];
  return (v[i / 2] + v[i / 2 + 1]) / 2.0;
}

double inflow_ux(const fsi_problem_desc& d, double y, double z) {
  const double Hy = d.breaks[1][d.n_breaks[1] - 1];
  if (d.dim == 2) return 1.5 * d.U * y * (Hy - y) / ((Hy / 2.0) * (Hy / 2.0));
  const double Hz = d.breaks[2][d.n_breaks[2] - 1];
  return 36.0 * d.U * y * (Hy - y) * z * (Hz - z) / (Hy * Hy * Hz * Hz);
}

// Equation kind held by a node row in the shuffled layout (Sec. 3.1):
// 0 momentum, 1 solid kinematic, 2 ALE.
int row_kind(int cls, int slot, int dim) {
  if (cls == kFluid) return slot < dim ? 2 : 0;
  return slot < dim ? 0 : 1;
}

void q2_weights_1d(double xi, double w[3]) {
  w[0] = 0.5 * xi * (xi - 1.0);
  w[1] = 1.0 - xi * xi;
  w[2] = 0.5 * xi * (xi + 1.0);
}

void build_mesh(const fsi_problem_desc& d, int l, HostLevel& L) {
  const int dim = d.dim;
  L.dim = dim;
  L.B = 2 * dim;
  L.nloc = dim == 2 ? 9 : 27;
  L.ndofe = L.B * L.nloc + dim + 1;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      L.verts[a] = refine(d.breaks[a], d.n_breaks[a], l);
      L.cells[a] = (int)L.verts[a].size() - 1;
      L.nodes_ax[a] = 2 * L.cells[a] + 1;
    } else {
      L.verts[a] = {0.0, 1.0};
      L.cells[a] = 1;
      L.nodes_ax[a] = 1;
    }
  }
  L.n_nodes = (int64_t)L.nodes_ax[0] * L.nodes_ax[1] * L.nodes_ax[2];
  L.n_elem = (int64_t)L.cells[0] * L.cells[1] * (dim == 3 ? L.cells[2] : 1);
  L.N = L.B * L.n_nodes + (dim + 1) * L.n_elem;
  L.nb = L.n_nodes + L.n_elem;
  L.Ni = L.nb * L.B;

  const int cx = L.cells[0], cy = L.cells[1], cz = dim == 3 ? L.cells[2] : 1;
  const int nx = L.nodes_ax[0], ny = L.nodes_ax[1];
  L.elem_nodes.assign(L.n_elem * L.nloc, 0);
  L.elem_solid.assign(L.n_elem, 0);
  for (int ez = 0; ez < cz; ++ez)
    for (int ey = 0; ey < cy; ++ey)
      for (int ex = 0; ex < cx; ++ex) {
        const int64_t e = ex + (int64_t)cx * (ey + (int64_t)cy * ez);
        for (int a = 0; a < L.nloc; ++a) {
          const int i = a % 3, j = (a / 3) % 3, k = a / 9;
          const int64_t node = (2 * ex + i) + (int64_t)nx * ((2 * ey + j) + (int64_t)ny * (dim == 3 ? 2 * ez + k : 0));
          L.elem_nodes[e * L.nloc + a] = (int32_t)node;
        }
        const int idx[3] = {ex, ey, ez};
        bool inside = true;
        for (int a = 0; a < dim; ++a) {
          const double c = 0.5 * (L.verts[a][idx[a]] + L.verts[a][idx[a] + 1]);
          inside = inside && (d.flap_lo[a] < c) && (c < d.flap_hi[a]);
        }
        L.elem_solid[e] = inside ? 1 : 0;
      }
  std::vector<uint8_t> ts(L.n_nodes, 0), tf(L.n_nodes, 0);
  for (int64_t e = 0; e < L.n_elem; ++e)
    for (int a = 0; a < L.nloc; ++a) (L.elem_solid[e] ? ts : tf)[L.elem_nodes[e * L.nloc + a]] = 1;
  L.node_class.assign(L.n_nodes, 0);
  for (int64_t n = 0; n < L.n_nodes; ++n)
    L.node_class[n] = (ts[n] && tf[n]) ? kIface : (ts[n] ? kSolid : kFluid);

  // Dirichlet data (internal layout)
  L.dir.assign(L.Ni, 0);
  L.dir_val.assign(L.Ni, 0.0);
  for (int64_t n = 0; n < L.n_nodes; ++n) {
    const int ix = (int)(n % nx), iy = (int)((n / nx) % ny), iz = dim == 3 ? (int)(n / ((int64_t)nx * ny)) : 0;
    const int ii[3] = {ix, iy, iz};
    bool bnd = false, wall_or_in = (ix == 0);
    for (int a = 0; a < dim; ++a) {
      const bool lo = ii[a] == 0, hi = ii[a] == L.nodes_ax[a] - 1;
      bnd = bnd || lo || hi;
      if (a > 0) wall_or_in = wall_or_in || lo || hi;
    }
    if (bnd)
      for (int c = 0; c < dim; ++c) L.dir[n * L.B + c] = 1;
    if (wall_or_in)
      for (int c = 0; c < dim; ++c) L.dir[n * L.B + dim + c] = 1;
    if (ix == 0) {
      const double y = q2_coord(L.verts[1], iy);
      const double z = dim == 3 ? q2_coord(L.verts[2], iz) : 0.0;
      L.dir_val[n * L.B + dim] = inflow_ux(d, y, z);
    }
  }
  L.canon_of_int.assign(L.Ni, -1);
  for (int64_t i = 0; i < L.n_nodes * L.B; ++i) L.canon_of_int[i] = (int32_t)i;
  for (int64_t e = 0; e < L.n_elem; ++e)
    for (int k = 0; k <= dim; ++k)
      L.canon_of_int[(L.n_nodes + e) * L.B + k] = (int32_t)(L.n_nodes * L.B + e * (dim + 1) + k);
}

void build_pattern(HostLevel& L) {
  const int nloc = L.nloc;
  std::vector<std::vector<int32_t>> nbr(L.n_nodes), elems_of(L.n_nodes);
  for (int64_t e = 0; e < L.n_elem; ++e) {
    const int32_t* en = &L.elem_nodes[e * nloc];
    for (int a = 0; a < nloc; ++a) {
      elems_of[en[a]].push_back((int32_t)e);
      for (int b = 0; b < nloc; ++b) nbr[en[a]].push_back(en[b]);
    }
  }
  L.rowptr.assign(L.nb + 1, 0);
  L.col.clear();
  for (int64_t n = 0; n < L.n_nodes; ++n) {
    auto& v = nbr[n];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    for (int32_t c : v) L.col.push_back(c);
    auto es = elems_of[n];
    std::sort(es.begin(), es.end());
    for (int32_t e : es) L.col.push_back((int32_t)(L.n_nodes + e));
    L.rowptr[n + 1] = (int32_t)L.col.size();
    std::vector<int32_t>().swap(v);
  }
  for (int64_t e = 0; e < L.n_elem; ++e) {
    std::vector<int32_t> v(&L.elem_nodes[e * nloc], &L.elem_nodes[e * nloc] + nloc);
    std::sort(v.begin(), v.end());
    for (int32_t c : v) L.col.push_back(c);
    L.rowptr[L.n_nodes + e + 1] = (int32_t)L.col.size();
  }
  L.nnzb = (int64_t)L.col.size();

  auto find = [&](int64_t row, int32_t c) -> int32_t {
    const int32_t* b = &L.col[L.rowptr[row]];
    const int32_t* en = &L.col[0] + L.rowptr[row + 1];
    const int32_t* it = std::lower_bound(b, en, c);
    return (it != en && *it == c) ? (int32_t)(it - &L.col[0]) : -1;
  };
  const int nl1 = nloc + 1;
  L.elem_map.assign(L.n_elem * nl1 * nl1, -1);
  for (int64_t e = 0; e < L.n_elem; ++e) {
    const int32_t* en = &L.elem_nodes[e * nloc];
    const int32_t pblk = (int32_t)(L.n_nodes + e);
    for (int a = 0; a <= nloc; ++a)
      for (int b = 0; b <= nloc; ++b) {
        int32_t v = -1;
        if (a < nloc && b < nloc) v = find(en[a], en[b]);
        else if (a < nloc) v = find(en[a], pblk);
        else if (b < nloc) v = find(pblk, en[b]);
        L.elem_map[(e * nl1 + a) * nl1 + b] = v;
      }
  }
  // colouring: parity of the element index along each axis; no two elements
  // of one colour share a node, so a colour's scatter is conflict free.
  const int ncol = 1 << L.dim;
  std::vector<std::vector<int32_t>> groups(ncol * 2);
  const int cx = L.cells[0], cy = L.cells[1];
  for (int64_t e = 0; e < L.n_elem; ++e) {
    const int ex = (int)(e % cx), ey = (int)((e / cx) % cy), ez = (int)(e / ((int64_t)cx * cy));
    const int c = (ex & 1) | ((ey & 1) << 1) | ((ez & 1) << 2);
    groups[c * 2 + L.elem_solid[e]].push_back((int32_t)e);
  }
  L.color_list.clear();
  L.color_ptr.assign(ncol * 2 + 1, 0);
  for (int g = 0; g < ncol * 2; ++g) {
    for (int32_t e : groups[g]) L.color_list.push_back(e);
    L.color_ptr[g + 1] = (int32_t)L.color_list.size();
  }
  // gather lists of the element contributions, in colour-group order
  if ((double)L.n_elem * nl1 * nl1 >= 2147483647.0) throw std::runtime_error("too many elements for the gather lists");
  L.blk_ptr.assign(L.nnzb + 1, 0);
  L.res_ptr.assign(L.nb + 1, 0);
  for (int64_t e = 0; e < L.n_elem; ++e) {
    for (int ab = 0; ab < nl1 * nl1; ++ab) {
      const int32_t v = L.elem_map[e * nl1 * nl1 + ab];
      if (v >= 0) ++L.blk_ptr[v + 1];
    }
    for (int a = 0; a < nloc; ++a) ++L.res_ptr[L.elem_nodes[e * nloc + a] + 1];
    ++L.res_ptr[L.n_nodes + e + 1];
  }
  for (int64_t i = 0; i < L.nnzb; ++i) L.blk_ptr[i + 1] += L.blk_ptr[i];
  for (int64_t i = 0; i < L.nb; ++i) L.res_ptr[i + 1] += L.res_ptr[i];
  L.blk_src.assign(L.blk_ptr[L.nnzb], 0);
  L.res_src.assign(L.res_ptr[L.nb], 0);
  {
    std::vector<int32_t> bp(L.blk_ptr.begin(), L.blk_ptr.end() - 1), rp(L.res_ptr.begin(), L.res_ptr.end() - 1);
    for (int32_t e : L.color_list) {
      for (int ab = 0; ab < nl1 * nl1; ++ab) {
        const int32_t v = L.elem_map[(int64_t)e * nl1 * nl1 + ab];
        if (v >= 0) L.blk_src[bp[v]++] = e * nl1 * nl1 + ab;
      }
      for (int a = 0; a < nloc; ++a) L.res_src[rp[L.elem_nodes[(int64_t)e * nloc + a]]++] = e * nl1 + a;
      L.res_src[rp[L.n_nodes + e]++] = e * nl1 + nloc;
    }
  }
  // element matrices need no colouring: fluid elements, then solid ones
  L.mat_list.clear();
  for (int pass = 0; pass < 2; ++pass)
    for (int64_t e = 0; e < L.n_elem; ++e)
      if ((L.elem_solid[e] != 0) == (pass == 1)) L.mat_list.push_back((int32_t)e);
  L.n_fluid_elem = 0;
  for (int64_t e = 0; e < L.n_elem; ++e) L.n_fluid_elem += L.elem_solid[e] == 0;
}

// Scalar node prolongation entries (fine node, coarse node, weight):
// fine Q2 nodes sit at the quarter points of the coarse cell.
struct Trip { int64_t f, c; double w; };

std::vector<Trip> node_prolongation(const HostLevel& C, const HostLevel& F) {
  std::vector<Trip> out;
  const int dim = F.dim;
  for (int64_t f = 0; f < F.n_nodes; ++f) {
    int fi[3] = {(int)(f % F.nodes_ax[0]), (int)((f / F.nodes_ax[0]) % F.nodes_ax[1]),
                 (int)(f / ((int64_t)F.nodes_ax[0] * F.nodes_ax[1]))};
    double w[3][3];
    int base[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
      if (a >= dim) { w[a][0] = 1.0; w[a][1] = 0.0; w[a][2] = 0.0; continue; }
      const int ec = std::min(fi[a] / 4, C.cells[a] - 1);
      const double xi = -1.0 + (double)(fi[a] - 4 * ec) / 2.0;
      q2_weights_1d(xi, w[a]);
      base[a] = 2 * ec;
    }
    const int nk = dim == 3 ? 3 : 1;
    for (int k = 0; k < nk; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          const double ww = w[0][i] * w[1][j] * w[2][k];
          if (ww == 0.0) continue;
          const int64_t c = (base[0] + i) + (int64_t)C.nodes_ax[0] *
                            ((base[1] + j) + (int64_t)C.nodes_ax[1] * (dim == 3 ? base[2] + k : 0));
          out.push_back({f, c, ww});
        }
  }
  return out;
}

void to_csr(int64_t nrows, std::vector<std::pair<int64_t, std::pair<int32_t, double>>>& e,
            std::vector<int32_t>& ptr, std::vector<int32_t>& col, std::vector<double>& val) {
  std::sort(e.begin(), e.end(), [](const auto& a, const auto& b) {
    return a.first != b.first ? a.first < b.first : a.second.first < b.second.first;
  });
  ptr.assign(nrows + 1, 0);
  col.resize(e.size());
  val.resize(e.size());
  for (size_t i = 0; i < e.size(); ++i) {
    ptr[e[i].first + 1]++;
    col[i] = e[i].second.first;
    val[i] = e[i].second.second;
  }
  for (int64_t r = 0; r < nrows; ++r) ptr[r + 1] += ptr[r];
}

void build_transfers(const HostLevel& C, HostLevel& F) {
  const int dim = F.dim, B = F.B;
  std::vector<Trip> S = node_prolongation(C, F);
  std::vector<std::pair<int64_t, std::pair<int32_t, double>>> pe, re, se;
  for (const Trip& t : S) {
    for (int s = 0; s < B; ++s) {
      const int64_t fr = t.f * B + s, cc = t.c * B + s;
      if (!F.dir[fr] && !C.dir[cc]) pe.push_back({fr, {(int32_t)cc, t.w}});
      se.push_back({fr, {(int32_t)cc, t.w}});   // unmasked: states (nested iteration)
    }
    // restriction: same component, same equation kind, no Dirichlet rows
    for (int sc = 0; sc < B; ++sc) {
      const int comp = sc % dim;
      const int64_t cr = t.c * B + sc;
      if (C.dir[cr]) continue;
      const int kc = row_kind(C.node_class[t.c], sc, dim);
      for (int q = 0; q < 2; ++q) {
        const int sf = q == 0 ? comp : dim + comp;
        const int64_t fr = t.f * B + sf;
        if (F.dir[fr]) continue;
        if (row_kind(F.node_class[t.f], sf, dim) != kc) continue;
        re.push_back({cr, {(int32_t)fr, t.w}});
      }
    }
  }
  // P1disc: xi_parent = (xi_child + (2 s - 1)) / 2 per axis
  for (int64_t ef = 0; ef < F.n_elem; ++ef) {
    int fi[3] = {(int)(ef % F.cells[0]), (int)((ef / F.cells[0]) % F.cells[1]),
                 (int)(ef / ((int64_t)F.cells[0] * F.cells[1]))};
    const int64_t ec = fi[0] / 2 + (int64_t)C.cells[0] * (fi[1] / 2 + (int64_t)C.cells[1] * (fi[2] / 2));
    const int64_t fb = (F.n_nodes + ef) * B, cb = (C.n_nodes + ec) * B;
    pe.push_back({fb, {(int32_t)cb, 1.0}});
    se.push_back({fb, {(int32_t)cb, 1.0}});
    re.push_back({cb, {(int32_t)fb, 1.0}});
    for (int a = 0; a < dim; ++a) {
      const double sig = 0.5 * (double)(2 * (fi[a] % 2) - 1);
      pe.push_back({fb, {(int32_t)(cb + 1 + a), sig}});
      se.push_back({fb, {(int32_t)(cb + 1 + a), sig}});
      re.push_back({cb + 1 + a, {(int32_t)fb, sig}});
      pe.push_back({fb + 1 + a, {(int32_t)(cb + 1 + a), 0.5}});
      se.push_back({fb + 1 + a, {(int32_t)(cb + 1 + a), 0.5}});
      re.push_back({cb + 1 + a, {(int32_t)(fb + 1 + a), 0.5}});
    }
  }
  to_csr(F.Ni, pe, F.P_ptr, F.P_col, F.P_val);
  to_csr(F.Ni, se, F.S_ptr, F.S_col, F.S_val);
  to_csr(C.Ni, re, F.R_ptr, F.R_col, F.R_val);
}

void build_patches(const fsi_solver_opts& o, HostLevel& L) {
  const int dim = L.dim, B = L.B, nloc = L.nloc;
  int tile[3] = {1, 1, 1}, ntile[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) {
    tile[a] = std::max(1, o.tile[a]);
    ntile[a] = (L.cells[a] + tile[a] - 1) / tile[a];
  }
  const int cx = L.cells[0], cy = L.cells[1];
  std::vector<int64_t> key(L.n_elem);
  for (int64_t e = 0; e < L.n_elem; ++e) {
    const int ex = (int)(e % cx), ey = (int)((e / cx) % cy), ez = (int)(e / ((int64_t)cx * cy));
    const int64_t t = ex / tile[0] + (int64_t)ntile[0] * (ey / tile[1] + (int64_t)ntile[1] * (ez / tile[2]));
    key[e] = t * 2 + (L.elem_solid[e] ? 0 : 1);
  }
  std::vector<int64_t> keys(key);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  std::vector<int32_t> patch_of(L.n_elem);
  std::vector<std::vector<int32_t>> pel(keys.size());
  for (int64_t e = 0; e < L.n_elem; ++e) {
    const int32_t p = (int32_t)(std::lower_bound(keys.begin(), keys.end(), key[e]) - keys.begin());
    patch_of[e] = p;
    pel[p].push_back((int32_t)e);
  }
  // owner element of each node: solid elements first, then lowest index
  std::vector<int32_t> owner(L.n_nodes, -1);
  for (int pass = 0; pass < 2; ++pass)
    for (int64_t e = 0; e < L.n_elem; ++e) {
      if ((pass == 0) != (L.elem_solid[e] != 0)) continue;
      for (int a = 0; a < nloc; ++a) {
        const int32_t n = L.elem_nodes[e * nloc + a];
        if (owner[n] < 0) owner[n] = (int32_t)e;
      }
    }
  const int np = (int)keys.size();
  L.n_patches = np;
  L.p_n.assign(np, 0); L.p_nown.assign(np, 0);
  L.p_idx_off.assign(np + 1, 0); L.p_own_off.assign(np + 1, 0); L.p_dense_off.assign(np + 1, 0);
  L.p_inv_off.assign(np + 1, 0); L.p_gmap_off.assign(np + 1, 0); L.p_pad_off.assign(np + 1, 0);
  L.p_elem_off.assign(np + 1, 0); L.p_boff_off.assign(np + 1, 0);
  L.p_idx.clear(); L.p_own.clear(); L.p_gmap.clear(); L.p_padpos.clear(); L.p_elems.clear(); L.p_boff.clear();
  L.p_gptr.clear();
  L.max_n = 0;
  L.max_nown = 0;
  for (int p = 0; p < np; ++p) {
    std::vector<int32_t> nodes;
    for (int32_t e : pel[p])
      for (int a = 0; a < nloc; ++a) nodes.push_back(L.elem_nodes[(int64_t)e * nloc + a]);
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    std::vector<int32_t> blocks(nodes);
    for (int32_t e : pel[p]) blocks.push_back((int32_t)(L.n_nodes + e));   // elements ascending
    const int nbk = (int)blocks.size();
    // dense layout: the B unknowns of each node block, then the dim + 1
    // pressures of each element block (its padding slots are left out), at
    // the offsets kept in p_boff; the size is padded to a multiple of 4 (the
    // FP32 factorisation kernels move rows as float4) by identity rows /
    // columns at the end whose index is an element padding slot (its vector
    // entries are always zero), never owned
    std::vector<int32_t> boff(nbk);
    int n_blk = 0;
    for (int lb = 0; lb < nbk; ++lb) {
      const int w = blocks[lb] < L.n_nodes ? B : dim + 1;
      boff[lb] = n_blk;
      L.p_boff.push_back(n_blk * 8 + w);
      n_blk += w;
    }
    const int n = (n_blk + 3) & ~3;
    L.p_n[p] = n;
    L.max_n = std::max(L.max_n, n);
    int nown = 0;
    for (int lb = 0; lb < nbk; ++lb) {
      const int32_t blk = blocks[lb];
      const bool is_node = blk < L.n_nodes;
      for (int c = 0; c < (is_node ? B : dim + 1); ++c) {
        L.p_idx.push_back(blk * B + c);
        const bool own = is_node ? (patch_of[owner[blk]] == p) : true;
        if (own) { L.p_own.push_back(boff[lb] + c); ++nown; }
      }
    }
    for (int q = n_blk; q < n; ++q) {
      L.p_idx.push_back((int32_t)((L.n_nodes + pel[p][0]) * B + B - 1));
      L.p_padpos.push_back(q);
    }
    L.p_nown[p] = nown;
    L.max_nown = std::max(L.max_nown, nown);
    const int64_t g_first = (int64_t)L.p_gmap.size() / 3;
    for (int lb = 0; lb < nbk; ++lb) {
      const int32_t br = blocks[lb];
      L.p_gptr.push_back((int32_t)((int64_t)L.p_gmap.size() / 3 - g_first));
      for (int32_t k = L.rowptr[br]; k < L.rowptr[br + 1]; ++k) {
        auto it = std::lower_bound(blocks.begin(), blocks.end(), L.col[k]);
        if (it != blocks.end() && *it == L.col[k]) {
          L.p_gmap.push_back(k);
          L.p_gmap.push_back(lb);
          L.p_gmap.push_back((int32_t)(it - blocks.begin()));
        }
      }
    }
    for (int32_t e : pel[p]) L.p_elems.push_back(e);
    L.p_idx_off[p + 1] = L.p_idx_off[p] + n;
    L.p_own_off[p + 1] = L.p_own_off[p] + nown;
    L.p_dense_off[p + 1] = L.p_dense_off[p] + (int64_t)n * n;
    L.p_inv_off[p + 1] = L.p_inv_off[p] + (int64_t)((nown + 3) & ~3) * n;   // owned rows padded to 4
    L.p_gmap_off[p + 1] = (int64_t)L.p_gmap.size() / 3;
    L.p_pad_off[p + 1] = (int64_t)L.p_padpos.size();
    L.p_elem_off[p + 1] = (int64_t)L.p_elems.size();
    L.p_boff_off[p + 1] = (int64_t)L.p_boff.size();
    L.p_gptr.push_back((int32_t)((int64_t)L.p_gmap.size() / 3 - g_first));   // row pointers end
  }
  L.dense_total = L.p_dense_off[np];
  L.inv_total = L.p_inv_off[np];
  L.idx_total = L.p_idx_off[np];
  L.own_total = L.p_own_off[np];
}

// Slab ordering of the coarse level for the banded LU: blocks sorted by
// their position along x (node x index; element 2 ex + 1, i.e. between its
// node planes), ties by index.  A node couples only to nodes and elements
// within two node planes, so the half-bandwidth is about two planes of
// unknowns (99 in 2D, 1193 in 3D for the 16x4(x4) coarse grids).
void build_coarse_ordering(HostLevel& L) {
  const int64_t nb = L.nb;
  std::vector<int64_t> key(nb);
  for (int64_t b = 0; b < L.n_nodes; ++b) key[b] = b % L.nodes_ax[0];
  for (int64_t e = 0; e < L.n_elem; ++e) key[L.n_nodes + e] = 2 * (e % L.cells[0]) + 1;
  std::vector<int32_t> order(nb);
  for (int64_t b = 0; b < nb; ++b) order[b] = (int32_t)b;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return key[a] < key[c]; });
  std::vector<int32_t> pos(nb);
  for (int64_t i = 0; i < nb; ++i) pos[order[i]] = (int32_t)i;
  L.coarse_perm.assign(L.Ni, 0);
  for (int64_t b = 0; b < nb; ++b)
    for (int c = 0; c < L.B; ++c) L.coarse_perm[b * L.B + c] = pos[b] * L.B + c;
  int64_t bw = 0;
  for (int64_t b = 0; b < nb; ++b)
    for (int32_t k = L.rowptr[b]; k < L.rowptr[b + 1]; ++k)
      bw = std::max<int64_t>(bw, std::llabs((int64_t)pos[b] - pos[L.col[k]]) * L.B + L.B - 1);
  L.coarse_bw = (int)bw;
  // slabs: nodes of x-planes 0..2 and element layer 0 form slab 0; x-planes
  // 2k+1, 2k+2 and element layer k form slab k.  An element of layer k
  // touches x-planes 2k, 2k+1, 2k+2 only, so slabs k-1 and k couple through
  // x-plane 2k alone, the last plane of slab k-1 in the banded ordering.
  const int K = L.cells[0];
  auto slab_of = [&](int64_t b) -> int {
    if (b < L.n_nodes) {
      const int ix = (int)(b % L.nodes_ax[0]);
      return ix <= 2 ? 0 : (ix - 1) / 2;
    }
    return (int)((b - L.n_nodes) % L.cells[0]);
  };
  std::vector<int64_t> cnt(K + 1, 0);
  for (int64_t b = 0; b < nb; ++b) cnt[slab_of(b) + 1] += L.B;
  L.slab_off.assign(K + 1, 0);
  for (int k = 0; k < K; ++k) L.slab_off[k + 1] = L.slab_off[k] + cnt[k + 1];
  L.slab_p = (int)((L.n_nodes / L.nodes_ax[0]) * L.B);
  bool ok = L.slab_off[K] == L.Ni;
  for (int64_t b = 0; b < nb && ok; ++b) {
    const int64_t q = (int64_t)pos[b] * L.B;
    const int sb = slab_of(b);
    ok = q >= L.slab_off[sb] && q < L.slab_off[sb + 1];
    for (int32_t k = L.rowptr[b]; k < L.rowptr[b + 1] && ok; ++k) {
      const int64_t qc = (int64_t)pos[L.col[k]] * L.B;
      const int sc = slab_of(L.col[k]);
      if (sc == sb) continue;
      if (std::abs(sc - sb) != 1) { ok = false; break; }
      // the slab-(min) side of the coupling lies in the last plane of that slab
      const int lo = std::min(sb, sc);
      const int64_t qlo = sb < sc ? q : qc;
      ok = qlo >= L.slab_off[lo + 1] - L.slab_p;
    }
  }
  if (!ok) L.slab_off.clear();   // no slab structure: the banded solve is used
}

}  // namespace

bool build_host_hierarchy(const fsi_problem_desc& d, const fsi_solver_opts& o,
                          std::vector<HostLevel>& lv, std::string& err) {
  if (d.dim != 2 && d.dim != 3) { err = "dim must be 2 or 3"; return false; }
  if (d.levels < 1 || d.levels > 10) { err = "levels must be in [1, 10]"; return false; }
  for (int a = 0; a < d.dim; ++a) {
    if (d.n_breaks[a] < 2 || d.n_breaks[a] > FSI_MAX_BREAKS) { err = "bad n_breaks"; return false; }
    for (int i = 1; i < d.n_breaks[a]; ++i)
      if (!(d.breaks[a][i] > d.breaks[a][i - 1])) { err = "breaks must ascend"; return false; }
  }
  lv.assign(d.levels, HostLevel());
  for (int l = 0; l < d.levels; ++l) {
    build_mesh(d, l, lv[l]);
    if (lv[l].Ni >= (int64_t)1 << 31) { err = "level too large for 32-bit indices"; return false; }
    build_pattern(lv[l]);
    if (l == 0) build_coarse_ordering(lv[l]);
    if (l > 0) {
      build_transfers(lv[l - 1], lv[l]);
      build_patches(o, lv[l]);
    }
  }
  return true;
}

}  // namespace fsi
