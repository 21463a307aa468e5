// Host construction of the structured mesh hierarchy: CSR patterns, element
// -> CSR gather lists and multigrid transfer operators (paper Sec. 3 spaces:
// P1 for phase fields / potentials / pressure, P2 for velocity).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "gather.h"
#include "internal.h"

namespace chnss {

std::atomic<long long> g_launch_count{0};

namespace {

// Nodes of element e on an n x n level: P1 vertex ids and P2 lattice ids
// (vertices, then midpoints of the edges opposite vertex 0, 1, 2).
void element_nodes(int n, int e, int v1[3], int v2[6]) {
  const int s = e >> 1, o = e & 1, i = s % n, j = s / n;
  int vi[3], vj[3];
  vi[0] = i; vj[0] = j;
  if (o == 0) { vi[1] = i + 1; vj[1] = j; vi[2] = i + 1; vj[2] = j + 1; }
  else        { vi[1] = i + 1; vj[1] = j + 1; vi[2] = i; vj[2] = j + 1; }
  const int m = 2 * n + 1;
  for (int k = 0; k < 3; ++k) {
    v1[k] = vj[k] * (n + 1) + vi[k];
    v2[k] = (2 * vj[k]) * m + 2 * vi[k];
  }
  auto mid = [&](int a, int b) { return (vj[a] + vj[b]) * m + (vi[a] + vi[b]); };
  v2[3] = mid(1, 2);
  v2[4] = mid(0, 2);
  v2[5] = mid(0, 1);
}

// Sorted-unique CSR pattern from per-element (row, col) node pairs.
}  // namespace

// SELL-C-sigma view of P (see internal.h); also returns the host map from
// SELL entries to CSR positions when hmap is given.
void build_sell(Arena &ar, Pattern &P, std::vector<int> *hmap) {
  const int C = Sell::C, S = Sell::SIGMA, n = P.nrows;
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  auto len = [&](int r) { return P.h_rowptr[r + 1] - P.h_rowptr[r]; };
  for (int w0 = 0; w0 < n; w0 += S) {
    const int w1 = std::min(n, w0 + S);
    std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int a, int b) { return len(a) > len(b); });
  }
  Sell &s = P.sell;
  s.nslices = (n + C - 1) / C;
  std::vector<int> sp(s.nslices + 1, 0), rowid((size_t)s.nslices * C, -1);
  for (int k = 0; k < s.nslices; ++k) {
    int w = 0;
    for (int r = 0; r < C; ++r) {
      const int i = k * C + r;
      if (i < n) {
        rowid[i] = perm[i];
        w = std::max(w, len(perm[i]));
      }
    }
    sp[k + 1] = sp[k] + w * C;
    s.wmax = std::max(s.wmax, w);
  }
  s.nent = sp[s.nslices];
  std::vector<int> col(s.nent), map(s.nent);
  for (int k = 0; k < s.nslices; ++k) {
    const int w = (sp[k + 1] - sp[k]) / C;
    for (int r = 0; r < C; ++r) {
      const int row = rowid[(size_t)k * C + r];
      const int l = row >= 0 ? len(row) : 0;
      int last = row >= 0 && l > 0 ? P.h_col[P.h_rowptr[row]] : 0;
      for (int j = 0; j < w; ++j) {
        const long e = sp[k] + (long)j * C + r;
        if (j < l) {
          const int q = P.h_rowptr[row] + j;
          col[e] = P.h_col[q];
          map[e] = q;
          last = col[e];
        } else {
          col[e] = last;   // padding: a column this row already touches, value 0
          map[e] = -1;
        }
      }
    }
  }
  s.slice_ptr = ar.upload(sp);
  s.rowid = ar.upload(rowid);
  s.col = ar.upload(col);
  s.map = ar.upload(map);
  if (P.nrows == P.ncols) {   // transposed values: entry (i, j) takes the CSR value at (j, i)
    bool symmetric = true;
    std::vector<int> mapT(s.nent, -1);
    for (int k = 0; k < s.nslices && symmetric; ++k) {
      const int w = (sp[k + 1] - sp[k]) / C;
      for (int r = 0; r < C && symmetric; ++r) {
        const int row = rowid[(size_t)k * C + r];
        for (int j = 0; j < w; ++j) {
          const long e = sp[k] + (long)j * C + r;
          if (map[e] < 0) continue;
          const int c = col[e];
          const int *b = P.h_col.data() + P.h_rowptr[c], *en = P.h_col.data() + P.h_rowptr[c + 1];
          const int *it = std::lower_bound(b, en, row);
          if (it == en || *it != row) { symmetric = false; break; }
          mapT[e] = (int)(it - P.h_col.data());
        }
      }
    }
    if (symmetric) s.mapT = ar.upload(mapT);
  }
  if (hmap) *hmap = std::move(map);
}

// Stencil layout of a P1 pattern on an nx-by-nx node lattice (nx = n + 1)
// whose triangles are split along the lower-left -> upper-right diagonal:
// row i couples at most to i + {-nx-1, -nx, -1, 0, 1, nx, nx+1}.  Returns
// false (building nothing) if some row has another column.
bool build_sell_stencil(Arena &ar, Pattern &P, int nx) {
  const int C = Sell::C, W = 7, n = P.nrows;
  const int off[W] = {-nx - 1, -nx, -1, 0, 1, nx, nx + 1};
  if (P.ncols != n || (long)nx * nx != n) return false;
  auto find = [&](int row, int c) -> int {
    if (c < 0 || c >= n) return -1;
    const int *b = P.h_col.data() + P.h_rowptr[row], *e = P.h_col.data() + P.h_rowptr[row + 1];
    const int *it = std::lower_bound(b, e, c);
    return (it != e && *it == c) ? (int)(it - P.h_col.data()) : -1;
  };
  for (int row = 0; row < n; ++row) {
    int hit = 0;
    for (int j = 0; j < W; ++j) hit += find(row, row + off[j]) >= 0 ? 1 : 0;
    if (hit != P.h_rowptr[row + 1] - P.h_rowptr[row]) return false;
  }
  Sell &s = P.sell;
  s.nslices = (n + C - 1) / C;
  s.wmax = W;
  s.nent = (long)s.nslices * W * C;
  std::vector<int> sp(s.nslices + 1), rowid((size_t)s.nslices * C, -1), col(s.nent), map(s.nent), mapT(s.nent, -1);
  for (int k = 0; k <= s.nslices; ++k) sp[k] = k * W * C;
  for (int k = 0; k < s.nslices; ++k)
    for (int r = 0; r < C; ++r) {
      const int row = k * C + r;
      if (row < n) rowid[(size_t)k * C + r] = row;
      for (int j = 0; j < W; ++j) {
        const long e = sp[k] + (long)j * C + r;
        const int q = row < n ? find(row, row + off[j]) : -1;
        col[e] = q >= 0 ? row + off[j] : (row < n ? row : 0);   // missing: own diagonal, value 0
        map[e] = q;
        if (q >= 0) mapT[e] = find(row + off[j], row);
      }
    }
  for (long e = 0; e < s.nent; ++e)
    if (map[e] >= 0 && mapT[e] < 0) throw Error{CHNSS_ERR_ARG, "stencil layout: unsymmetric P1 pattern"};
  s.slice_ptr = ar.upload(sp);
  s.rowid = ar.upload(rowid);
  s.col = ar.upload(col);
  s.map = ar.upload(map);
  s.mapT = ar.upload(mapT);
  s.stencil = 1;
  for (int j = 0; j < W; ++j) s.soff[j] = off[j];
  return true;
}

void upload_pattern(Arena &ar, Pattern &P, std::vector<int> *hmap) {
  P.rowptr = ar.upload(P.h_rowptr);
  P.col = ar.upload(P.h_col);
  build_sell(ar, P, hmap);
}

void upload_gather(Arena &ar, Gather &G, const std::vector<int> &ptr, const std::vector<int> &idx) {
  G.ptr = ar.upload(ptr);
  G.idx = ar.upload(idx);
}

void transpose(const Pattern &A, const std::vector<double> &av, Pattern &T, std::vector<double> &tv) {
  T.nrows = A.ncols;
  T.ncols = A.nrows;
  T.nnz = A.nnz;
  T.h_rowptr.assign(T.nrows + 1, 0);
  for (int k = 0; k < A.nnz; ++k) T.h_rowptr[A.h_col[k] + 1]++;
  for (int r = 0; r < T.nrows; ++r) T.h_rowptr[r + 1] += T.h_rowptr[r];
  T.h_col.assign(A.nnz, 0);
  tv.assign(A.nnz, 0.0);
  std::vector<int> fill(T.h_rowptr.begin(), T.h_rowptr.end() - 1);
  for (int r = 0; r < A.nrows; ++r)
    for (int k = A.h_rowptr[r]; k < A.h_rowptr[r + 1]; ++k) {
      int d = fill[A.h_col[k]]++;
      T.h_col[d] = r;
      tv[d] = av[k];
    }
}

void finish_transfer(Arena &ar, Transfer &t, const std::vector<double> &pv) {
  std::vector<double> rv;
  transpose(t.P, pv, t.R, rv);
  std::vector<int> pmap, rmap;
  upload_pattern(ar, t.P, &pmap);
  upload_pattern(ar, t.R, &rmap);
  t.Pv = ar.upload(pv);
  t.Rv = ar.upload(rv);
  auto sell_vals = [](const std::vector<int> &map, const std::vector<double> &v) {
    std::vector<double> out(map.size());
    for (size_t e = 0; e < map.size(); ++e) out[e] = map[e] >= 0 ? v[map[e]] : 0.0;
    return out;
  };
  const std::vector<double> ps = sell_vals(pmap, pv), rs = sell_vals(rmap, rv);
  t.Ps = ar.upload(ps);
  t.Rs = ar.upload(rs);
  t.Ps32 = ar.upload(std::vector<float>(ps.begin(), ps.end()));
  t.Rs32 = ar.upload(std::vector<float>(rs.begin(), rs.end()));
}

std::vector<int> diag_positions(const Pattern &P) {
  std::vector<int> d(P.nrows);
  for (int r = 0; r < P.nrows; ++r) d[r] = find_col(P, r, r);
  return d;
}

namespace {

// Linear interpolation of coarse P1 functions at the fine P1 nodes.
void build_p1_transfer(Arena &ar, int nc, Transfer &t) {
  const int nf = 2 * nc, mf = nf + 1, mc = nc + 1;
  Pattern &P = t.P;
  P.nrows = mf * mf;
  P.ncols = mc * mc;
  P.h_rowptr.assign(P.nrows + 1, 0);
  std::vector<double> pv;
  for (int J = 0; J <= nf; ++J)
    for (int I = 0; I <= nf; ++I) {
      const int r = J * mf + I, i = I / 2, j = J / 2;
      if (I % 2 == 0 && J % 2 == 0) {
        P.h_col.push_back(j * mc + i); pv.push_back(1.0);
      } else if (J % 2 == 0) {            // horizontal edge midpoint
        P.h_col.push_back(j * mc + i); pv.push_back(0.5);
        P.h_col.push_back(j * mc + i + 1); pv.push_back(0.5);
      } else if (I % 2 == 0) {            // vertical edge midpoint
        P.h_col.push_back(j * mc + i); pv.push_back(0.5);
        P.h_col.push_back((j + 1) * mc + i); pv.push_back(0.5);
      } else {                            // midpoint of the square's diagonal
        P.h_col.push_back(j * mc + i); pv.push_back(0.5);
        P.h_col.push_back((j + 1) * mc + i + 1); pv.push_back(0.5);
      }
      P.h_rowptr[r + 1] = (int)P.h_col.size();
    }
  P.nnz = (int)P.h_col.size();
  finish_transfer(ar, t, pv);
}

// Quadratic interpolation of coarse P2 functions at the fine P2 nodes, on
// the nodes without prescribed velocity of both levels (open top: the top
// edge except its corners is free).
void build_vel_transfer(Arena &ar, int nc, int top_bc, Transfer &t) {
  const int mf = 4 * nc + 1, mc = 2 * nc + 1;
  Pattern &P = t.P;
  P.nrows = mf * mf;
  P.ncols = mc * mc;
  P.h_rowptr.assign(P.nrows + 1, 0);
  std::vector<double> pv;
  auto cbnd = [&](int id) {
    int I = id % mc, J = id / mc;
    return I == 0 || J == 0 || I == mc - 1 || (top_bc == 0 && J == mc - 1);
  };
  for (int J = 0; J < mf; ++J)
    for (int I = 0; I < mf; ++I) {
      const int r = J * mf + I;
      const bool fb = I == 0 || J == 0 || I == mf - 1 || (top_bc == 0 && J == mf - 1);
      if (!fb) {
        const int i = std::min(I / 4, nc - 1), j = std::min(J / 4, nc - 1);
        const double xi = I / 4.0 - i, eta = J / 4.0 - j;   // exact quarters
        const bool lower = xi >= eta;
        double l[3];
        if (lower) { l[0] = 1 - xi; l[1] = xi - eta; l[2] = eta; }
        else       { l[0] = 1 - eta; l[1] = xi; l[2] = eta - xi; }
        int v1[3], v2[6];
        element_nodes(nc, 2 * (j * nc + i) + (lower ? 0 : 1), v1, v2);
        const double w[6] = {l[0] * (2 * l[0] - 1), l[1] * (2 * l[1] - 1), l[2] * (2 * l[2] - 1),
                             4 * l[1] * l[2], 4 * l[0] * l[2], 4 * l[0] * l[1]};
        std::vector<std::pair<int, double>> row;
        for (int k = 0; k < 6; ++k)
          if (w[k] != 0.0 && !cbnd(v2[k])) row.push_back({v2[k], w[k]});
        std::sort(row.begin(), row.end());
        for (auto &cw : row) { P.h_col.push_back(cw.first); pv.push_back(cw.second); }
      }
      P.h_rowptr[r + 1] = (int)P.h_col.size();
    }
  P.nnz = (int)P.h_col.size();
  finish_transfer(ar, t, pv);
}

}  // namespace

void build_mesh(Mesh &m, int n, double lx, double ly, int top_bc) {
  Arena &ar = m.arena;
  m.n = n;
  m.top_bc = top_bc;
  m.lx = lx;
  m.ly = ly;
  std::vector<int> sizes{n};
  while (sizes.back() % 2 == 0 && sizes.back() >= 4) sizes.push_back(sizes.back() / 2);
  m.lv.resize(sizes.size());
  std::vector<int> hptr, hidx;
  for (size_t l = 0; l < sizes.size(); ++l) {
    Level &L = m.lv[l];
    const int nl = sizes[l];
    L.n = nl;
    L.hx = lx / nl;
    L.hy = ly / nl;
    L.N1 = (nl + 1) * (nl + 1);
    L.N2 = (2 * nl + 1) * (2 * nl + 1);
    L.E = 2 * nl * nl;
    const int m2 = 2 * nl + 1;
    std::vector<int> bnd(L.N2);
    for (int id = 0; id < L.N2; ++id) {
      int I = id % m2, J = id / m2;
      bnd[id] = (I == 0 || J == 0 || I == m2 - 1 || (top_bc == 0 && J == m2 - 1)) ? 1 : 0;
    }
    auto p1pair = [&](int e, int *r, int *c) { int v2[6]; element_nodes(nl, e, r, v2); std::memcpy(c, r, 3 * sizeof(int)); };
    auto p2pair = [&](int e, int *r, int *c) { int v1[3]; element_nodes(nl, e, v1, r); std::memcpy(c, r, 6 * sizeof(int)); };
    pattern_from_elements(L.N1, L.N1, L.E, 3, 3, p1pair, L.p1);
    pattern_from_elements(L.N2, L.N2, L.E, 6, 6, p2pair, L.p2);
    L.p1.rowptr = ar.upload(L.p1.h_rowptr);
    L.p1.col = ar.upload(L.p1.h_col);
    if (!build_sell_stencil(ar, L.p1, nl + 1)) build_sell(ar, L.p1);
    upload_pattern(ar, L.p2);
    gather_from_elements(L.p1, L.E, 3, 3, p1pair, [](int e, int a, int b) { return e * 9 + a * 3 + b; },
                         [](int, int, int, int, int) { return true; }, L.g_p1, hptr, hidx);
    upload_gather(ar, L.g_p1, hptr, hidx);
    auto vkeep = [&](int, int, int, int r, int c) { return !bnd[r] && !bnd[c]; };
    gather_from_elements(L.p2, L.E, 6, 6, p2pair, [](int e, int a, int b) { return e * 36 + a * 6 + b; },
                         vkeep, L.g_p2v, hptr, hidx);
    upload_gather(ar, L.g_p2v, hptr, hidx);
    gather_from_elements(L.p2, L.E, 6, 6, p2pair, [](int e, int a, int b) { return e * 144 + (a * 6 + b) * 4; },
                         vkeep, L.g_ks, hptr, hidx);
    upload_gather(ar, L.g_ks, hptr, hidx);
    L.bnd2 = ar.upload(bnd);
    L.diag1 = ar.upload(diag_positions(L.p1));
    L.diag2 = ar.upload(diag_positions(L.p2));
    if (l == 0) {
      // B: P1 rows x P2 node cols; B^T: P2 node rows x P1 cols; element [E][3][6][2]
      auto bpair = [&](int e, int *r, int *c) { element_nodes(nl, e, r, c); };
      auto btpair = [&](int e, int *r, int *c) { element_nodes(nl, e, c, r); };
      pattern_from_elements(L.N1, L.N2, L.E, 3, 6, bpair, m.pb);
      pattern_from_elements(L.N2, L.N1, L.E, 6, 3, btpair, m.pbt);
      upload_pattern(ar, m.pb);
      upload_pattern(ar, m.pbt);
      gather_from_elements(m.pb, L.E, 3, 6, bpair, [](int e, int a, int b) { return e * 36 + (a * 6 + b) * 2; },
                           [&](int, int, int, int, int c) { return !bnd[c]; }, m.g_b, hptr, hidx);
      upload_gather(ar, m.g_b, hptr, hidx);
      gather_from_elements(m.pbt, L.E, 6, 3, btpair, [](int e, int b, int a) { return e * 36 + (a * 6 + b) * 2; },
                           [&](int, int, int, int r, int) { return !bnd[r]; }, m.g_bt, hptr, hidx);
      upload_gather(ar, m.g_bt, hptr, hidx);
      node_gather(L.N1, L.E, 3, [&](int e, int *nd) { int v2[6]; element_nodes(nl, e, nd, v2); },
                  [](int e, int a) { return e * 3 + a; }, [](int) { return true; }, hptr, hidx, m.g_l1);
      upload_gather(ar, m.g_l1, hptr, hidx);
      node_gather(L.N2, L.E, 6, [&](int e, int *nd) { int v1[3]; element_nodes(nl, e, v1, nd); },
                  [](int e, int a) { return e * 12 + a * 2; }, [&](int id) { return !bnd[id]; }, hptr, hidx, m.g_l2);
      upload_gather(ar, m.g_l2, hptr, hidx);
      m.ref_node = nl * (nl + 1) + nl / 2;
    }
  }
  for (size_t l = 0; l + 1 < sizes.size(); ++l) {
    build_p1_transfer(ar, sizes[l + 1], m.lv[l].t1);
    build_vel_transfer(ar, sizes[l + 1], top_bc, m.lv[l].tv);
  }
}

void destroy_mesh(Mesh &m) { m.arena.release(); }

// ---------------------------------------------------------------------------
// Reference tensors: exact integrals of products of barycentric monomials,
// int_T l0^a l1^b l2^c = 2 |T| a! b! c! / (a + b + c + 2)!.
namespace {
constexpr int PD = 9;  // degrees 0..8 per variable
struct Poly {
  double c[PD][PD][PD];
  Poly() { std::memset(c, 0, sizeof(c)); }
};
Poly lam(int k) {
  Poly p;
  int e[3] = {0, 0, 0};
  e[k] = 1;
  p.c[e[0]][e[1]][e[2]] = 1.0;
  return p;
}
Poly cst(double v) { Poly p; p.c[0][0][0] = v; return p; }
Poly add(const Poly &a, const Poly &b, double sb = 1.0) {
  Poly r;
  for (int i = 0; i < PD; ++i) for (int j = 0; j < PD; ++j) for (int k = 0; k < PD; ++k)
    r.c[i][j][k] = a.c[i][j][k] + sb * b.c[i][j][k];
  return r;
}
Poly mul(const Poly &a, const Poly &b) {
  Poly r;
  for (int i = 0; i < PD; ++i) for (int j = 0; j < PD; ++j) for (int k = 0; k < PD; ++k) {
    if (a.c[i][j][k] == 0.0) continue;
    for (int p = 0; p + i < PD; ++p) for (int q = 0; q + j < PD; ++q) for (int s = 0; s + k < PD; ++s)
      r.c[i + p][j + q][k + s] += a.c[i][j][k] * b.c[p][q][s];
  }
  return r;
}
Poly dlam(const Poly &a, int l) {
  Poly r;
  for (int i = 0; i < PD; ++i) for (int j = 0; j < PD; ++j) for (int k = 0; k < PD; ++k) {
    int e[3] = {i, j, k};
    if (e[l] == 0 || a.c[i][j][k] == 0.0) continue;
    double f = e[l];
    e[l] -= 1;
    r.c[e[0]][e[1]][e[2]] += f * a.c[i][j][k];
  }
  return r;
}
double fact(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }
double integ(const Poly &a) {   // divided by |T|
  double s = 0;
  for (int i = 0; i < PD; ++i) for (int j = 0; j < PD; ++j) for (int k = 0; k < PD; ++k)
    if (a.c[i][j][k] != 0.0) s += a.c[i][j][k] * 2.0 * fact(i) * fact(j) * fact(k) / fact(i + j + k + 2);
  return s;
}

RefTensors make_reference_tensors() {
  RefTensors t;
  Poly L[3] = {lam(0), lam(1), lam(2)};
  Poly P2[6];
  for (int k = 0; k < 3; ++k) P2[k] = add(mul(cst(2.0), mul(L[k], L[k])), L[k], -1.0);
  P2[3] = mul(cst(4.0), mul(L[1], L[2]));
  P2[4] = mul(cst(4.0), mul(L[0], L[2]));
  P2[5] = mul(cst(4.0), mul(L[0], L[1]));
  Poly D[6][3];
  for (int b = 0; b < 6; ++b) for (int l = 0; l < 3; ++l) D[b][l] = dlam(P2[b], l);
  for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) t.m1[a][b] = integ(mul(L[a], L[b]));
  for (int k = 0; k < 6; ++k) for (int a = 0; a < 3; ++a) t.c1[k][a] = integ(mul(P2[k], L[a]));
  for (int a = 0; a < 6; ++a) for (int b = 0; b < 6; ++b) t.m2[a][b] = integ(mul(P2[a], P2[b]));
  for (int k = 0; k < 6; ++k)
    for (int l = 0; l < 3; ++l)
      for (int b = 0; b < 6; ++b) {
        Poly kd = mul(P2[k], D[b][l]);
        for (int a = 0; a < 6; ++a) t.j[k][l][b][a] = integ(mul(kd, P2[a]));
      }
  for (int l = 0; l < 3; ++l) for (int b = 0; b < 6; ++b) for (int a = 0; a < 6; ++a)
    t.jg[l][b][a] = integ(mul(D[b][l], P2[a]));
  for (int l = 0; l < 3; ++l) for (int b = 0; b < 6; ++b) for (int mm = 0; mm < 3; ++mm) for (int a = 0; a < 6; ++a)
    t.s[l][b][mm][a] = integ(mul(D[b][l], D[a][mm]));
  for (int a = 0; a < 3; ++a) for (int b = 0; b < 6; ++b) for (int l = 0; l < 3; ++l)
    t.b[a][b][l] = integ(mul(L[a], D[b][l]));
  for (int a = 0; a < 6; ++a) for (int l = 0; l < 3; ++l) t.g[a][l] = integ(D[a][l]);
  // degree-7 rule: eta = u (5-point Gauss-Legendre), xi = v (1 - u) (4-point),
  // Jacobian (1 - u); closed-form Gauss-Legendre nodes on [-1, 1].
  const double s65 = std::sqrt(6.0 / 5.0), s30 = std::sqrt(30.0);
  const double x4[4] = {-std::sqrt(3.0 / 7 + 2.0 / 7 * s65), -std::sqrt(3.0 / 7 - 2.0 / 7 * s65),
                        std::sqrt(3.0 / 7 - 2.0 / 7 * s65), std::sqrt(3.0 / 7 + 2.0 / 7 * s65)};
  const double w4[4] = {(18 - s30) / 36, (18 + s30) / 36, (18 + s30) / 36, (18 - s30) / 36};
  const double s107 = std::sqrt(10.0 / 7.0), s70 = std::sqrt(70.0);
  const double x5[5] = {-std::sqrt(5 + 2 * s107) / 3, -std::sqrt(5 - 2 * s107) / 3, 0.0,
                        std::sqrt(5 - 2 * s107) / 3, std::sqrt(5 + 2 * s107) / 3};
  const double w5[5] = {(322 - 13 * s70) / 900, (322 + 13 * s70) / 900, 128.0 / 225,
                        (322 + 13 * s70) / 900, (322 - 13 * s70) / 900};
  int q = 0;
  for (int iu = 0; iu < 5; ++iu)
    for (int iv = 0; iv < 4; ++iv, ++q) {
      const double u = 0.5 * (x5[iu] + 1), v = 0.5 * (x4[iv] + 1);
      const double eta = u, xi = v * (1 - u);
      t.qlam[q][0] = 1 - xi - eta;
      t.qlam[q][1] = xi;
      t.qlam[q][2] = eta;
      t.qw[q] = 2.0 * (0.5 * w5[iu]) * (0.5 * w4[iv]) * (1 - u);
    }
  return t;
}
}  // namespace

const RefTensors &reference_tensors() {
  static const RefTensors t = make_reference_tensors();
  return t;
}

}  // namespace chnss
