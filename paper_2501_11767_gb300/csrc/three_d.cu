// Host setup of the tetrahedral (3D) discretisation: Kuhn meshes of a box,
// the exact reference integrals of the P1 / P2 element operators
// (three_d.h), host assembly of the element operators into CSR in element
// order, and the nested P1 / P2 transfers.  The 3D operators are exported
// through chnss3_host_operator for checks against a reference; the element
// operators are __host__ __device__ so that the device kernels of the 3D
// step use the same code.
#include <algorithm>
#include <array>
#include <exception>
#include <memory>
#include <thread>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "three_d.h"

namespace chnss {
namespace {

// Gauss-Legendre nodes and weights on [0, 1] (Newton on P_k).
void gauss_legendre01(int k, std::vector<double> &x, std::vector<double> &w) {
  x.assign(k, 0.0);
  w.assign(k, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < k; ++i) {
    double z = std::cos(pi * (i + 0.75) / (k + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= k; ++j) {
        const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (k == 1) p0 = 1.0;
      dp = k * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2 / ((1 - z^2) P'^2) on [-1, 1], halved
  }
}

// Collapsed Gauss rule on the reference tetrahedron exact to `degree`:
// barycentric points (Q x 4) and weights summing to 1.
void tetra_rule(int degree, std::vector<std::array<double, 4>> &lam, std::vector<double> &wt) {
  const int ks = (degree + 4) / 2, kt = (degree + 3) / 2, ku = (degree + 2) / 2;
  std::vector<double> xs, ws, xt, wtt, xu, wu;
  gauss_legendre01(ks, xs, ws);
  gauss_legendre01(kt, xt, wtt);
  gauss_legendre01(ku, xu, wu);
  lam.clear();
  wt.clear();
  for (int i = 0; i < ks; ++i)
    for (int j = 0; j < kt; ++j)
      for (int k = 0; k < ku; ++k) {
        const double s = xs[i], t = xt[j], u = xu[k];
        const double xi = s, eta = t * (1.0 - s), zeta = u * (1.0 - s) * (1.0 - t);
        lam.push_back({1.0 - xi - eta - zeta, xi, eta, zeta});
        wt.push_back(6.0 * ws[i] * wtt[j] * wu[k] * (1.0 - s) * (1.0 - s) * (1.0 - t));
      }
}

// P2 basis values N[10] and barycentric derivatives dN[10][4] at lambda.
void p2_basis(const std::array<double, 4> &l, double N[10], double dN[10][4]) {
  std::memset(dN, 0, sizeof(double) * 40);
  for (int a = 0; a < 4; ++a) {
    N[a] = l[a] * (2.0 * l[a] - 1.0);
    dN[a][a] = 4.0 * l[a] - 1.0;
  }
  for (int e = 0; e < 6; ++e) {
    const int a = kEdge3[e][0], b = kEdge3[e][1];
    N[4 + e] = 4.0 * l[a] * l[b];
    dN[4 + e][a] = 4.0 * l[b];
    dN[4 + e][b] = 4.0 * l[a];
  }
}

Tet3Ref build_reference() {
  Tet3Ref R;
  std::memset(&R, 0, sizeof(R));
  std::vector<std::array<double, 4>> lam;
  std::vector<double> w;
  tetra_rule(5, lam, w);   // every product below has degree <= 5
  for (size_t q = 0; q < w.size(); ++q) {
    double N[10], dN[10][4];
    p2_basis(lam[q], N, dN);
    for (int k = 0; k < 10; ++k)
      for (int a = 0; a < 4; ++a) R.r[k][a] += w[q] * N[k] * lam[q][a];
    for (int k = 0; k < 10; ++k)
      for (int l = 0; l < 4; ++l)
        for (int b = 0; b < 10; ++b)
          for (int a = 0; a < 10; ++a) R.t[k][l][b][a] += w[q] * N[k] * dN[b][l] * N[a];
    for (int l = 0; l < 4; ++l)
      for (int b = 0; b < 10; ++b)
        for (int a = 0; a < 10; ++a) R.s[l][b][a] += w[q] * dN[b][l] * N[a];
    for (int a = 0; a < 10; ++a)
      for (int l = 0; l < 4; ++l) R.d[a][l] += w[q] * dN[a][l];
    for (int a = 0; a < 10; ++a)
      for (int l = 0; l < 4; ++l)
        for (int b = 0; b < 10; ++b)
          for (int m = 0; m < 4; ++m) R.q[a][l][b][m] += w[q] * dN[a][l] * dN[b][m];
    for (int qq = 0; qq < 4; ++qq)
      for (int b = 0; b < 10; ++b)
        for (int l = 0; l < 4; ++l) R.w[qq][b][l] += w[q] * lam[q][qq] * dN[b][l];
    for (int a = 0; a < 10; ++a)
      for (int b = 0; b < 10; ++b) R.m2[a][b] += w[q] * N[a] * N[b];
  }
  tetra_rule(7, lam, w);
  if ((int)w.size() != kLoadPts3) throw Error{CHNSS_ERR_ARG, "degree-7 tetrahedral rule: unexpected size"};
  for (int q = 0; q < kLoadPts3; ++q) {
    for (int a = 0; a < 4; ++a) R.ql[q][a] = lam[q][a];
    R.qw[q] = w[q];
  }
  return R;
}

const Tet3Ref &reference3() {
  static const Tet3Ref R = build_reference();
  return R;
}

// One Kuhn mesh: element vertex lattice coordinates and node ids.
struct Mesh3Host {
  int n = 0;
  long N1 = 0, N2 = 0, E = 0;
  double h[3] = {0, 0, 0};
  std::vector<int> lat;    // E x 4 x 3 vertex lattice coordinates
  std::vector<int> tet;    // E x 4 P1 ids
  std::vector<int> tet2;   // E x 10 P2 ids
  int id1(int a, int b, int c) const { return (c * (n + 1) + b) * (n + 1) + a; }
  int id2(int A, int B, int C) const {
    const int m = 2 * n + 1;
    return (C * m + B) * m + A;
  }
  void coords(long e, double x[4][3]) const {
    for (int v = 0; v < 4; ++v)
      for (int d = 0; d < 3; ++d) x[v][d] = lat[(e * 4 + v) * 3 + d] * h[d];
  }
  bool top_free = false;   // open (do-nothing) top face
  // P2 nodes with prescribed (zero) velocity: every face, or all but the
  // open top face (its edges stay on the side walls)
  bool p2_boundary(int id) const {
    const int m = 2 * n + 1, A = id % m, B = (id / m) % m, C = id / (m * m);
    return A == 0 || B == 0 || C == 0 || A == m - 1 || B == m - 1 || (C == m - 1 && !top_free);
  }
  bool p1_top(int id) const { return id / ((n + 1) * (n + 1)) == n; }
};

Mesh3Host make_mesh3(int n, const double L[3], bool top_free = false) {
  Mesh3Host M;
  M.n = n;
  M.top_free = top_free;
  M.N1 = (long)(n + 1) * (n + 1) * (n + 1);
  M.N2 = (long)(2 * n + 1) * (2 * n + 1) * (2 * n + 1);
  M.E = 6L * n * n * n;
  for (int d = 0; d < 3; ++d) M.h[d] = L[d] / n;
  M.lat.resize(M.E * 12);
  M.tet.resize(M.E * 4);
  M.tet2.resize(M.E * 10);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        for (int p = 0; p < 6; ++p) {
          const long e = 6L * ((long)(k * n + j) * n + i) + p;
          int v[3] = {i, j, k};
          int *L3 = &M.lat[e * 12];
          for (int d = 0; d < 3; ++d) L3[d] = v[d];
          for (int s = 0; s < 3; ++s) {
            v[kPerm3[p][s]] += 1;
            for (int d = 0; d < 3; ++d) L3[(s + 1) * 3 + d] = v[d];
          }
          for (int a = 0; a < 4; ++a) {
            M.tet[e * 4 + a] = M.id1(L3[a * 3], L3[a * 3 + 1], L3[a * 3 + 2]);
            M.tet2[e * 10 + a] = M.id2(2 * L3[a * 3], 2 * L3[a * 3 + 1], 2 * L3[a * 3 + 2]);
          }
          for (int q = 0; q < 6; ++q) {
            const int a = kEdge3[q][0], b = kEdge3[q][1];
            M.tet2[e * 10 + 4 + q] = M.id2(L3[a * 3] + L3[b * 3], L3[a * 3 + 1] + L3[b * 3 + 1],
                                           L3[a * 3 + 2] + L3[b * 3 + 2]);
          }
        }
  return M;
}

// Host CSR built from element (row node list, col node list, dense block)
// contributions, summed in element order.
struct HostCSR {
  int nrows = 0, ncols = 0;
  std::vector<int> rowptr, col;
  std::vector<double> val;
};

template <class Fn>
HostCSR assemble_host(int nrows, int ncols, long E, int nr, int nc, Fn elem) {
  // elem(e, rows[nr], cols[nc], block[nr * nc]); a row or column index < 0
  // drops that contribution
  std::vector<std::vector<std::pair<int, double>>> rows(nrows);
  std::vector<int> rn(nr), cn(nc);
  std::vector<double> blk((size_t)nr * nc);
  for (long e = 0; e < E; ++e) {
    elem(e, rn.data(), cn.data(), blk.data());
    for (int a = 0; a < nr; ++a) {
      if (rn[a] < 0) continue;
      for (int b = 0; b < nc; ++b)
        if (cn[b] >= 0) rows[rn[a]].push_back({cn[b], blk[(size_t)a * nc + b]});
    }
  }
  HostCSR A;
  A.nrows = nrows;
  A.ncols = ncols;
  A.rowptr.assign(nrows + 1, 0);
  for (int r = 0; r < nrows; ++r) {
    auto &v = rows[r];
    std::stable_sort(v.begin(), v.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    for (size_t i = 0; i < v.size();) {   // element order inside each entry's sum
      size_t j = i;
      double s = 0.0;
      while (j < v.size() && v[j].first == v[i].first) s += v[j++].second;
      A.col.push_back(v[i].first);
      A.val.push_back(s);
      i = j;
    }
    A.rowptr[r + 1] = (int)A.col.size();
  }
  return A;
}

// Kuhn tetrahedron of a point given in coarse-cell units, and its
// barycentric coordinates.
long locate3(int nc, const double X[3], double lam[4]) {
  int cell[3];
  double loc[3];
  for (int d = 0; d < 3; ++d) {
    cell[d] = std::min((int)std::floor(X[d]), nc - 1);
    loc[d] = X[d] - cell[d];
  }
  int ord[3] = {0, 1, 2};
  std::stable_sort(ord, ord + 3, [&](int a, int b) { return loc[a] > loc[b]; });
  int p = 0;
  while (!(kPerm3[p][0] == ord[0] && kPerm3[p][1] == ord[1] && kPerm3[p][2] == ord[2])) ++p;
  lam[0] = 1.0 - loc[ord[0]];
  lam[1] = loc[ord[0]] - loc[ord[1]];
  lam[2] = loc[ord[1]] - loc[ord[2]];
  lam[3] = loc[ord[2]];
  return 6L * ((long)(cell[2] * nc + cell[1]) * nc + cell[0]) + p;
}

HostCSR p1_prolongation3(const Mesh3Host &c) {
  const int nf = 2 * c.n, m = nf + 1;
  HostCSR P;
  P.nrows = m * m * m;
  P.ncols = (int)c.N1;
  P.rowptr.assign(P.nrows + 1, 0);
  for (int r = 0; r < P.nrows; ++r) {
    const double X[3] = {(r % m) / 2.0, ((r / m) % m) / 2.0, (r / (m * m)) / 2.0};
    double lam[4];
    const long e = locate3(c.n, X, lam);
    std::vector<std::pair<int, double>> row;
    for (int a = 0; a < 4; ++a)
      if (lam[a] != 0.0) row.push_back({c.tet[e * 4 + a], lam[a]});
    std::sort(row.begin(), row.end());
    for (auto &x : row) {
      P.col.push_back(x.first);
      P.val.push_back(x.second);
    }
    P.rowptr[r + 1] = (int)P.col.size();
  }
  return P;
}

// Quadratic interpolation of coarse P2 functions at the fine P2 nodes,
// restricted to interior nodes of both meshes, per velocity component.
HostCSR velocity_prolongation3(const Mesh3Host &c, const Mesh3Host &f) {
  const int mf = 2 * f.n + 1;
  HostCSR P;
  P.nrows = 3 * (int)f.N2;
  P.ncols = 3 * (int)c.N2;
  P.rowptr.assign(P.nrows + 1, 0);
  for (int node = 0; node < (int)f.N2; ++node) {
    std::vector<std::pair<int, double>> row;
    if (!f.p2_boundary(node)) {
      const double X[3] = {(node % mf) / 4.0, ((node / mf) % mf) / 4.0, (node / (mf * mf)) / 4.0};
      double lam[4];
      const long e = locate3(c.n, X, lam);
      double N[10], dN[10][4];
      p2_basis({lam[0], lam[1], lam[2], lam[3]}, N, dN);
      for (int a = 0; a < 10; ++a) {
        const int cn = c.tet2[e * 10 + a];
        if (N[a] != 0.0 && !c.p2_boundary(cn)) row.push_back({cn, N[a]});
      }
      std::sort(row.begin(), row.end());
    }
    for (int comp = 0; comp < 3; ++comp) {
      const int r = 3 * node + comp;
      for (auto &x : row) {
        P.col.push_back(3 * x.first + comp);
        P.val.push_back(x.second);
      }
      P.rowptr[r + 1] = (int)P.col.size();
    }
  }
  return P;
}

enum Op3 {
  OP3_M1 = 0, OP3_K1, OP3_C1, OP3_CP, OP3_M2, OP3_J2, OP3_KSYM, OP3_B, OP3_P1PROL, OP3_VPROL,
  OP3_LOADS, OP3_KORTEWEG, OP3_TOP, OP3_KK0, OP3_KK1, OP3_KK2, OP3_VPROL_OPEN, OP3_COUNT
};

void element_fields(const Mesh3Host &M, long e, const double *v, double vk[10][3]) {
  for (int k = 0; k < 10; ++k)
    for (int d = 0; d < 3; ++d) vk[k][d] = v[3L * M.tet2[e * 10 + k] + d];
}

void element_shift(const Mesh3Host &M, long e, const double g[4][3], const chnss_params &p, const chnss_state &st,
                   double s[3]) {
  s[0] = s[1] = s[2] = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 4; ++a) {
      const double mv = st.mu[i][M.tet[e * 4 + a]];
      for (int d = 0; d < 3; ++d) s[d] += p.alpha[i] * mv * g[a][d];
    }
}

// Operators and vectors of the 3D discretisation on the host.
HostCSR host_operator3(int n, int which, const chnss_params &p, const chnss_state *st) {
  const double L[3] = {1.0, 1.0, 1.0};
  const Mesh3Host M = make_mesh3(n, L);
  const Tet3Ref &R = reference3();
  const int N1 = (int)M.N1, N2 = (int)M.N2;
  auto need = [&](bool ok) {
    if (!ok) throw Error{CHNSS_ERR_ARG, "this 3D operator needs the state fields"};
  };
  switch (which) {
    case OP3_KK0:
    case OP3_KK1:
    case OP3_KK2: {
      const int sp = which - OP3_KK0;
      need(st && st->phi[sp]);
      return assemble_host(N1, N1, M.E, 4, 4, [&](long e, int *r, int *c, double *b) {
        double x[4][3], g[4][3], f[4];
        M.coords(e, x);
        const double vol = tet_geometry(x, g);
        for (int a = 0; a < 4; ++a) {
          r[a] = c[a] = M.tet[e * 4 + a];
          f[a] = st->phi[sp][M.tet[e * 4 + a]];
        }
        tet_wstiff(vol, g, f, p.gamma[sp], p.mobility_m0, b);
      });
    }
    case OP3_M1:
    case OP3_K1:
    case OP3_C1:
    case OP3_CP: {
      if (which >= OP3_C1) need(st && st->v && (which == OP3_C1 || st->mu[0]));
      return assemble_host(N1, N1, M.E, 4, 4, [&](long e, int *r, int *c, double *b) {
        double x[4][3], g[4][3];
        M.coords(e, x);
        const double vol = tet_geometry(x, g);
        for (int a = 0; a < 4; ++a) r[a] = c[a] = M.tet[e * 4 + a];
        if (which == OP3_M1) {
          for (int a = 0; a < 4; ++a)
            for (int bb = 0; bb < 4; ++bb) b[a * 4 + bb] = vol * (a == bb ? 0.1 : 0.05);
        } else if (which == OP3_K1) {
          for (int a = 0; a < 4; ++a)
            for (int bb = 0; bb < 4; ++bb)
              b[a * 4 + bb] = vol * (g[a][0] * g[bb][0] + g[a][1] * g[bb][1] + g[a][2] * g[bb][2]);
        } else {
          double vk[10][3], s[3];
          element_fields(M, e, st->v, vk);
          if (which == OP3_CP) element_shift(M, e, g, p, *st, s);
          tet_p1_conv(R, vol, g, vk, which == OP3_CP ? s : nullptr, b);
        }
      });
    }
    case OP3_M2:
    case OP3_J2: {
      if (which == OP3_J2) need(st && st->v && st->mu[0]);
      return assemble_host(N2, N2, M.E, 10, 10, [&](long e, int *r, int *c, double *b) {
        double x[4][3], g[4][3];
        M.coords(e, x);
        const double vol = tet_geometry(x, g);
        for (int a = 0; a < 10; ++a) r[a] = c[a] = M.tet2[e * 10 + a];
        if (which == OP3_M2) {
          for (int a = 0; a < 10; ++a)
            for (int bb = 0; bb < 10; ++bb) b[a * 10 + bb] = vol * R.m2[a][bb];
        } else {
          double vk[10][3], s[3];
          element_fields(M, e, st->v, vk);
          element_shift(M, e, g, p, *st, s);
          tet_p2_conv(R, vol, g, vk, s, b);
        }
      });
    }
    case OP3_KSYM:
      return assemble_host(3 * N2, 3 * N2, M.E, 30, 30, [&](long e, int *r, int *c, double *b) {
        double x[4][3], g[4][3];
        M.coords(e, x);
        const double vol = tet_geometry(x, g);
        for (int a = 0; a < 10; ++a)
          for (int d = 0; d < 3; ++d) r[a * 3 + d] = c[a * 3 + d] = 3 * M.tet2[e * 10 + a] + d;
        tet_ksym(R, vol, g, p.eta, b);
      });
    case OP3_B:
      return assemble_host(N1, 3 * N2, M.E, 4, 30, [&](long e, int *r, int *c, double *b) {
        double x[4][3], g[4][3];
        M.coords(e, x);
        const double vol = tet_geometry(x, g);
        for (int a = 0; a < 4; ++a) r[a] = M.tet[e * 4 + a];
        for (int a = 0; a < 10; ++a)
          for (int d = 0; d < 3; ++d) c[a * 3 + d] = 3 * M.tet2[e * 10 + a] + d;
        tet_div(R, vol, g, b);
      });
    case OP3_P1PROL:
    case OP3_VPROL:
    case OP3_VPROL_OPEN: {
      if (n % 2) throw Error{CHNSS_ERR_ARG, "transfers need an even n (coarse mesh n / 2)"};
      const bool open = which == OP3_VPROL_OPEN;
      const Mesh3Host C = make_mesh3(n / 2, L, open);
      if (which == OP3_P1PROL) return p1_prolongation3(C);
      return velocity_prolongation3(C, open ? make_mesh3(n, L, true) : M);
    }
    case OP3_LOADS:
    case OP3_KORTEWEG:
    case OP3_TOP: {
      HostCSR V;
      const int len = which == OP3_LOADS ? 5 * N1 : which == OP3_KORTEWEG ? 3 * N2 : N1;
      V.nrows = len;
      V.ncols = 1;
      V.val.assign(len, 0.0);
      if (which == OP3_TOP) {   // int_{z = lz} psi_a: |triangle| / 3 per vertex
        const double area = M.h[0] * M.h[1] / 2.0;
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int t[2][3] = {{M.id1(i, j, n), M.id1(i + 1, j, n), M.id1(i + 1, j + 1, n)},
                                 {M.id1(i, j, n), M.id1(i + 1, j + 1, n), M.id1(i, j + 1, n)}};
            for (auto &tri : t)
              for (int a : tri) V.val[a] += area / 3.0;
          }
      } else if (which == OP3_LOADS) {
        need(st && st->phi[0] && st->Phi_v);
        for (long e = 0; e < M.E; ++e) {
          double x[4][3], g[4][3], f[4][4], out[20];
          M.coords(e, x);
          const double vol = tet_geometry(x, g);
          for (int a = 0; a < 4; ++a) {
            const int id = M.tet[e * 4 + a];
            for (int i = 0; i < 3; ++i) f[i][a] = st->phi[i][id];
            f[3][a] = st->Phi_v[id];
          }
          tet_loads(R, vol, f, out);
          for (int k = 0; k < 5; ++k)
            for (int a = 0; a < 4; ++a) V.val[(long)k * N1 + M.tet[e * 4 + a]] += out[k * 4 + a];
        }
      } else {
        need(st && st->phi[0] && st->Phi_v);
        for (long e = 0; e < M.E; ++e) {
          double x[4][3], g[4][3], out[30];
          M.coords(e, x);
          const double vol = tet_geometry(x, g);
          double gr[5][3] = {};
          for (int a = 0; a < 4; ++a) {
            const int id = M.tet[e * 4 + a];
            for (int d = 0; d < 3; ++d) {
              for (int i = 0; i < 3; ++i) gr[i][d] += st->phi[i][id] * g[a][d];
              gr[4][d] += st->Phi_v[id] * g[a][d];
            }
          }
          for (int d = 0; d < 3; ++d) gr[3][d] = -(gr[0][d] + gr[1][d] + gr[2][d]);
          double G[3][3];
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) {
              double s = 0.0;
              for (int i = 0; i < 4; ++i) s += p.beta[i] * gr[i][c] * gr[i][d];
              G[c][d] = s + p.beta_v * gr[4][c] * gr[4][d];
            }
          tet_korteweg(R, vol, g, G, out);
          for (int a = 0; a < 10; ++a)
            for (int c = 0; c < 3; ++c) V.val[3L * M.tet2[e * 10 + a] + c] += out[a * 3 + c];
        }
      }
      return V;
    }
    default:
      throw Error{CHNSS_ERR_ARG, "unknown 3D operator"};
  }
}

}  // namespace
}  // namespace chnss

extern "C" chnss_status chnss3_host_operator(int n, int which, const chnss_params *params, const chnss_state *state,
                                            int *nrows, int *ncols, long long *nnz, int *rowptr, int *col,
                                            double *val) {
  using namespace chnss;
  try {
    if (n < 1 || n > 64) throw Error{CHNSS_ERR_ARG, "3D host operators: 1 <= n <= 64"};
    if (!params || !nrows || !ncols || !nnz) throw Error{CHNSS_ERR_ARG, "null argument"};
    const HostCSR A = host_operator3(n, which, *params, state);
    *nrows = A.nrows;
    *ncols = A.ncols;
    const bool vec = A.ncols == 1 && A.rowptr.empty();
    *nnz = vec ? (long long)A.val.size() : (long long)A.col.size();
    if (val) {
      std::memcpy(val, A.val.data(), A.val.size() * sizeof(double));
      if (!vec) {
        if (!rowptr || !col) throw Error{CHNSS_ERR_ARG, "null rowptr or col"};
        std::memcpy(rowptr, A.rowptr.data(), A.rowptr.size() * sizeof(int));
        std::memcpy(col, A.col.data(), A.col.size() * sizeof(int));
      }
    }
    return CHNSS_OK;
  } catch (const Error &e) {
    set_global_error(e.msg);
    return e.status;
  } catch (const std::exception &e) {
    set_global_error(e.what());
    return CHNSS_ERR_ARG;
  }
}

// ---------------------------------------------------------------------------
// The 3D step on the device: the 2D step's systems and solvers (Sec. 4) on a
// Kuhn mesh.  Per-step assembly: one thread per tetrahedron evaluates an
// element operator of three_d.h into an element buffer, a gather kernel sums
// every CSR entry's contributions in element order (no atomics).  The
// velocity operator is a scalar CSR on the interleaved 3 N2 dofs; all
// hierarchies are scalar multigrid (FP64, or FP32 / BF16-stored values
// inside the FP64 Krylov solvers); the three solve groups run on library
// streams after the assembly.
#include "gather.h"
#include "solver.h"

namespace chnss {
namespace {

__constant__ Tet3Ref c3;

struct Geo3 {
  int n;
  double h[3];
};

struct Fields3 {
  const double *phi[3];
  const double *mu[4];
  const double *Phi;
  const double *v;
  double alpha[4], beta[4], beta_v;
};

constexpr int kTPB3 = 128;
inline int nb3(long n, int t = kTPB3) { return (int)((n + t - 1) / t); }

__device__ inline void tet_nodes(const Geo3 &g, long e, double x[4][3], int v1[4], int v2[10]) {
  // kPerm3 and kEdge3 of three_d.h, as device-side tables
  const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int kEdge3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  const int n = g.n, p = (int)(e % 6);
  const long c = e / 6;
  int lat[4][3];
  int v[3] = {(int)(c % n), (int)((c / n) % n), (int)(c / ((long)n * n))};
  for (int d = 0; d < 3; ++d) lat[0][d] = v[d];
  for (int s = 0; s < 3; ++s) {
    v[kPerm3[p][s]] += 1;
    for (int d = 0; d < 3; ++d) lat[s + 1][d] = v[d];
  }
  const int n1 = n + 1, m = 2 * n + 1;
  for (int a = 0; a < 4; ++a) {
    for (int d = 0; d < 3; ++d) x[a][d] = lat[a][d] * g.h[d];
    v1[a] = (lat[a][2] * n1 + lat[a][1]) * n1 + lat[a][0];
    v2[a] = (2 * lat[a][2] * m + 2 * lat[a][1]) * m + 2 * lat[a][0];
  }
  for (int q = 0; q < 6; ++q) {
    const int a = kEdge3[q][0], b = kEdge3[q][1];
    v2[4 + q] = ((lat[a][2] + lat[b][2]) * m + lat[a][1] + lat[b][1]) * m + lat[a][0] + lat[b][0];
  }
}

__device__ inline void elem_shift(const Fields3 &f, const int v1[4], const double gr[4][3], double s[3]) {
  s[0] = s[1] = s[2] = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 4; ++a) {
      const double mv = f.mu[i][v1[a]];
      for (int d = 0; d < 3; ++d) s[d] += f.alpha[i] * mv * gr[a][d];
    }
}

// mode 0: P1 convection (shift if `shift`), buf [E][16];  mode 1: P2
// convection with the shift, buf [E][100]
__global__ void k3_conv(Geo3 g, Fields3 f, int mode, int shift, double *buf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double x[4][3], gr[4][3], vk[10][3], s[3];
  int v1[4], v2[10];
  tet_nodes(g, e, x, v1, v2);
  const double vol = tet_geometry(x, gr);
  for (int k = 0; k < 10; ++k)
    for (int d = 0; d < 3; ++d) vk[k][d] = f.v[3L * v2[k] + d];
  if (shift) elem_shift(f, v1, gr, s);
  if (mode == 0) tet_p1_conv(c3, vol, gr, vk, shift ? s : nullptr, buf + e * 16);
  else tet_p2_conv(c3, vol, gr, vk, s, buf + e * 100);
}

// weighted stiffness of the concentration-dependent mobility
// gamma (phi (1 - phi) + m0), buf [E][16]
__global__ void k3_wstiff(Geo3 g, const double *phi, double gamma, double m0, double *buf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double x[4][3], gr[4][3], f[4];
  int v1[4], v2[10];
  tet_nodes(g, e, x, v1, v2);
  const double vol = tet_geometry(x, gr);
  for (int a = 0; a < 4; ++a) f[a] = phi[v1[a]];
  tet_wstiff(vol, gr, f, gamma, m0, buf + e * 16);
}

// potential loads [E][20] and Korteweg load [E][30]
__global__ void k3_loads(Geo3 g, Fields3 f, double *lbuf, double *kbuf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double x[4][3], gr[4][3], fl[4][4];
  int v1[4], v2[10];
  tet_nodes(g, e, x, v1, v2);
  const double vol = tet_geometry(x, gr);
  for (int a = 0; a < 4; ++a) {
    for (int i = 0; i < 3; ++i) fl[i][a] = f.phi[i][v1[a]];
    fl[3][a] = f.Phi[v1[a]];
  }
  tet_loads(c3, vol, fl, lbuf + e * 20);
  double grd[5][3] = {};
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) {
      for (int i = 0; i < 3; ++i) grd[i][d] += fl[i][a] * gr[a][d];
      grd[4][d] += fl[3][a] * gr[a][d];
    }
  for (int d = 0; d < 3; ++d) grd[3][d] = -(grd[0][d] + grd[1][d] + grd[2][d]);
  double G[3][3];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
      for (int i = 0; i < 4; ++i) s += f.beta[i] * grd[i][c] * grd[i][d];
      G[c][d] = s + f.beta_v * grd[4][c] * grd[4][d];
    }
  tet_korteweg(c3, vol, gr, G, kbuf + e * 30);
}

// ---- adjoint (transposed Jacobian) element kernels.  P1 results go to the
// [E][20] layout of the potential loads (field f, node a at 4 f + a; gathered
// by the load list), velocity results to the [E][30] Korteweg layout.

// d/dv of y^T C(v) x (P1 x, y): int zeta_k (d_d x) y = (d_d x) vol sum_a y_a
// r[k][a] -> buf [E][30]
__global__ void k3_adj_conv_p1(Geo3 g, const double *__restrict__ x, const double *__restrict__ y, double *buf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double xc[4][3], gr[4][3], gx[3] = {0.0, 0.0, 0.0}, ya[4];
  int v1[4], v2[10];
  tet_nodes(g, e, xc, v1, v2);
  const double vol = tet_geometry(xc, gr);
  for (int a = 0; a < 4; ++a) {
    const double xv = x[v1[a]];
    for (int d = 0; d < 3; ++d) gx[d] += xv * gr[a][d];
    ya[a] = y[v1[a]];
  }
  for (int k = 0; k < 10; ++k) {
    const double s = vol * (ya[0] * c3.r[k][0] + ya[1] * c3.r[k][1] + ya[2] * c3.r[k][2] + ya[3] * c3.r[k][3]);
    for (int d = 0; d < 3; ++d) buf[e * 30 + k * 3 + d] = s * gx[d];
  }
}

// d/dphi of y^T K_kappa(phi) x, kappa = gamma (phi (1 - phi) + m0): node c of
// an element gets int gamma (1 - 2 phi_h) psi_c grad x . grad y
// = vol gamma (grad x . grad y) (1/4 - (sum_a phi_a + phi_c) / 10) -> buf [E][20], slot 0
__global__ void k3_adj_wstiff(Geo3 g, const double *__restrict__ phi, double gamma, const double *__restrict__ x,
                              const double *__restrict__ y, double *buf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double xc[4][3], gr[4][3], gx[3] = {0.0, 0.0, 0.0}, gy[3] = {0.0, 0.0, 0.0}, ph[4], psum = 0.0;
  int v1[4], v2[10];
  tet_nodes(g, e, xc, v1, v2);
  const double vol = tet_geometry(xc, gr);
  for (int a = 0; a < 4; ++a) {
    const double xv = x[v1[a]], yv = y[v1[a]];
    for (int d = 0; d < 3; ++d) {
      gx[d] += xv * gr[a][d];
      gy[d] += yv * gr[a][d];
    }
    ph[a] = phi[v1[a]];
    psum += ph[a];
  }
  const double s = vol * gamma * (gx[0] * gy[0] + gx[1] * gy[1] + gx[2] * gy[2]);
  for (int c = 0; c < 4; ++c) buf[e * 20 + c] = s * (0.25 - (psum + ph[c]) / 10.0);
}

// d/dw of y^T (J(w) (x) I) x (velocities x, y): nodal part int N_k
// sum_c (d_d x_c) y_c -> bufv [E][30]; the part of the per-element shift
// (w = v - s) projected on the P1 gradients, (d/ds) . grad psi_a -> bufm [E][20], slot 0
__global__ void k3_adj_conv_p2(Geo3 g, const double *__restrict__ x, const double *__restrict__ y, double *bufv,
                               double *bufm) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double xc[4][3], gr[4][3], yk[10][3];
  int v1[4], v2[10];
  tet_nodes(g, e, xc, v1, v2);
  const double vol = tet_geometry(xc, gr);
  for (int a = 0; a < 10; ++a)
    for (int c = 0; c < 3; ++c) yk[a][c] = y[3L * v2[a] + c];
  // acc[k][l] = sum_(a,b) xy[b][a] t[k][l][b][a], accs[l] = sum xy[b][a] s[l][b][a],
  // xy[b][a] = sum_c x_(b,c) y_(a,c)
  double acc[10][4], accs[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 10; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[k][l] = 0.0;
  for (int b = 0; b < 10; ++b) {
    const double x0 = x[3L * v2[b]], x1 = x[3L * v2[b] + 1], x2 = x[3L * v2[b] + 2];
    for (int a = 0; a < 10; ++a) {
      const double xy = x0 * yk[a][0] + x1 * yk[a][1] + x2 * yk[a][2];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        accs[l] += xy * c3.s[l][b][a];
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k][l] += xy * c3.t[k][l][b][a];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 10; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d)
      bufv[e * 30 + k * 3 + d] =
          vol * (gr[0][d] * acc[k][0] + gr[1][d] * acc[k][1] + gr[2][d] * acc[k][2] + gr[3][d] * acc[k][3]);
  double sb[3];
  for (int d = 0; d < 3; ++d)
    sb[d] = -vol * (gr[0][d] * accs[0] + gr[1][d] * accs[1] + gr[2][d] * accs[2] + gr[3][d] * accs[3]);
  for (int a = 0; a < 4; ++a) bufm[e * 20 + a] = sb[0] * gr[a][0] + sb[1] * gr[a][1] + sb[2] * gr[a][2];
}

struct LoadWeights3 {
  const double *z[5];   // adjoint weights of the loads of df/dphi_p, _N, _s, _a, df/dPhi (null: zero)
};

// gradient of sum_i z_i^T F_i with respect to (phi_p, phi_N, phi_s, Phi):
// int (sum_i d g_i / d var) z_i psi_a with the Hessian at the degree-7 rule,
// d/dphi_j = H_ij - H_ia (phi_a = 1 - sum phi) -> buf [E][20] (field f, node a)
__global__ void k3_adj_loads(Geo3 g, Fields3 f, LoadWeights3 lw, double *buf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double xc[4][3], gr[4][3], fl[4][4], zz[5][4];
  int v1[4], v2[10];
  tet_nodes(g, e, xc, v1, v2);
  const double vol = tet_geometry(xc, gr);
  for (int a = 0; a < 4; ++a) {
    for (int i = 0; i < 3; ++i) fl[i][a] = f.phi[i][v1[a]];
    fl[3][a] = f.Phi[v1[a]];
    for (int i = 0; i < 5; ++i) zz[i][a] = lw.z[i] ? lw.z[i][v1[a]] : 0.0;
  }
  double acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 4; ++a) acc[i][a] = 0.0;
  for (int q = 0; q < kLoadPts3; ++q) {
    const double *lq = c3.ql[q];
    double v[4], z[5];
    for (int i = 0; i < 4; ++i) v[i] = lq[0] * fl[i][0] + lq[1] * fl[i][1] + lq[2] * fl[i][2] + lq[3] * fl[i][3];
    for (int i = 0; i < 5; ++i) z[i] = lq[0] * zz[i][0] + lq[1] * zz[i][1] + lq[2] * zz[i][2] + lq[3] * zz[i][3];
    double H[5][5];
    potential_hessian3(v[0], v[1], v[2], v[3], H);
    double gj[4];
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int i = 0; i < 5; ++i) s += z[i] * (H[i][j] - H[i][3]);
      gj[j] = s;
    }
    gj[3] = z[0] * H[0][4] + z[1] * H[1][4] + z[2] * H[2][4] + z[3] * H[3][4] + z[4] * H[4][4];
    for (int i = 0; i < 4; ++i) {
      const double wg = c3.qw[q] * gj[i];
      for (int a = 0; a < 4; ++a) acc[i][a] += wg * lq[a];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 4; ++a) buf[e * 20 + i * 4 + a] = vol * acc[i][a];
}

// gradient of y^T G (Korteweg load) with respect to (phi_p, phi_N, phi_s,
// Phi): grad psi_m . (Y + Y^T) u, u = beta_j grad phi_j - beta_a grad phi_a
// (beta_v grad Phi for Phi), Y[c][b] = int d_b y_c -> buf [E][20]
__global__ void k3_adj_korteweg(Geo3 g, Fields3 f, const double *__restrict__ y, double *buf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6L * g.n * g.n * g.n) return;
  double xc[4][3], gr[4][3];
  int v1[4], v2[10];
  tet_nodes(g, e, xc, v1, v2);
  const double vol = tet_geometry(xc, gr);
  double Y[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int a = 0; a < 10; ++a) {
    double da[3] = {0.0, 0.0, 0.0};   // int grad N_a / vol
    for (int l = 0; l < 4; ++l)
      for (int b = 0; b < 3; ++b) da[b] += c3.d[a][l] * gr[l][b];
    for (int c = 0; c < 3; ++c) {
      const double yc = y[3L * v2[a] + c];
      for (int b = 0; b < 3; ++b) Y[c][b] += vol * yc * da[b];
    }
  }
  double S[3][3];
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b) S[c][b] = Y[c][b] + Y[b][c];
  double grd[5][3] = {};
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) {
      for (int i = 0; i < 3; ++i) grd[i][d] += f.phi[i][v1[a]] * gr[a][d];
      grd[4][d] += f.Phi[v1[a]] * gr[a][d];
    }
  for (int d = 0; d < 3; ++d) grd[3][d] = -(grd[0][d] + grd[1][d] + grd[2][d]);
  for (int fi = 0; fi < 4; ++fi) {
    double u[3];
    for (int d = 0; d < 3; ++d)
      u[d] = fi < 3 ? f.beta[fi] * grd[fi][d] - f.beta[3] * grd[3][d] : f.beta_v * grd[4][d];
    double su[3];
    for (int c = 0; c < 3; ++c) su[c] = S[c][0] * u[0] + S[c][1] * u[1] + S[c][2] * u[2];
    for (int m = 0; m < 4; ++m) buf[e * 20 + fi * 4 + m] = gr[m][0] * su[0] + gr[m][1] * su[1] + gr[m][2] * su[2];
  }
}

__global__ void k3_add_at(double *x, int idx, double v) { x[idx] += v; }

// out = lp - m sum(lp) / vol (transpose of the zero-mean pressure shift)
__global__ void k3_mean_shift_T(int N1, const double *lp, const double *m, const double *sum, double vol,
                                double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N1) out[i] = lp[i] - m[i] * (*sum) / vol;
}

// coarse P1 node (a, b, c) <- fine (2a, 2b, 2c); coarse P2 node (A, B, C) <-
// fine P2 node (2A, 2B, 2C), three components
__global__ void k3_inject(int nf, int vel, const double *fine, double *coarse) {
  const int nc = nf / 2;
  const int mc = vel ? 2 * nc + 1 : nc + 1, mf = vel ? 2 * nf + 1 : nf + 1;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)mc * mc * mc) return;
  const int a = (int)(i % mc), b = (int)((i / mc) % mc), c = (int)(i / ((long)mc * mc));
  const long src = ((long)(2 * c) * mf + 2 * b) * mf + 2 * a;
  if (vel)
    for (int d = 0; d < 3; ++d) coarse[3 * i + d] = fine[3 * src + d];
  else
    coarse[i] = fine[src];
}

__global__ void k3_mask(long n, const int *bnd, double *x) {   // zero the boundary velocity dofs
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && bnd[i / 3]) x[i] = 0.0;
}

// out = -cc (load + sb j t), j = evap (phi_s[ref] - phi_inf)
__global__ void k3_flux_rhs(int N1, const double *load, const double *top, const double *phi_s, int ref, double evap,
                            double phi_inf, double sb, double cc, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N1) return;
  const double j = evap * (phi_s[ref] - phi_inf);
  out[i] = -cc * (load[i] + sb * j * top[i]);
}

// rhs += -tau gamma_v load_v + flux j t
__global__ void k3_ac_rhs(int N1, const double *load, const double *top, const double *phi_s, int ref, double evap,
                          double phi_inf, double tg, double flux, double *rhs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N1) return;
  const double j = evap * (phi_s[ref] - phi_inf);
  rhs[i] += -tg * load[i] + flux * j * top[i];
}

// vals[idx[k]] = value: the Dirichlet outflow rows and columns of A_p on the
// open top (zeros, then ones on the diagonal)
__global__ void k3_set_entries(int n, const int *idx, double value, double *vals) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) vals[idx[k]] = value;
}

__global__ void k3_air(int N1, const double *p0, const double *p1, const double *p2, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N1) out[i] = 1.0 - p0[i] - p1[i] - p2[i];
}

__global__ void k3_shift(int N1, double *p, const double *sum, double vol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N1) p[i] -= *sum / vol;
}

// one level of the 3D hierarchy on the device
struct Level3 {
  int n = 0;
  long N1 = 0, N2 = 0, E = 0;
  Geo3 geo{};
  Pattern p1, pv;
  // 3x3-block SELL view of the velocity operator: the P2 node pattern and the
  // CSR position in pv of each of its block values (-1: padding)
  Pattern pv3;
  int *map9 = nullptr;
  int *diag1 = nullptr, *diagv = nullptr;
  Transfer t1, tv;                 // from the next coarser level
  Gather g1, gj;                   // element buffers -> P1 CSR, P2 convection -> velocity CSR
  double *M1 = nullptr, *K1 = nullptr, *ACb = nullptr, *Aconst = nullptr;
  double *Kp = nullptr;            // K_p of the PCD: K1, or with Dirichlet rows on an open top
  double *L = nullptr, *AC = nullptr, *A = nullptr, *X[3] = {nullptr, nullptr, nullptr};
  double *vl = nullptr, *mul = nullptr;   // injected v (3 N2) and mu (4 N1), levels >= 1
  // concentration-dependent mobility: X2 = tau K_kappa + a M per species,
  // K_kappa itself (fine level), injected phi (3 N1, levels >= 1)
  double *X2[3] = {nullptr, nullptr, nullptr}, *Kk[3] = {nullptr, nullptr, nullptr}, *phil = nullptr;
};

// The block preconditioners' hierarchies and scratch in the arithmetic of
// precision 0 (T = double) or 1 / 2 (T = float; 2: the velocity hierarchy's
// values stored in BF16)
template <typename T>
struct Prec3 {
  MGHier<T> L, AC, X[3], X2[3], Kp, A;   // X2: concentration-dependent mobility only
  T *Ms = nullptr, *Aps = nullptr, *mdinv = nullptr, *mb = nullptr, *mx = nullptr, *mt = nullptr;
};

}  // namespace
}  // namespace chnss

struct chnss3_ctx {
  chnss::Arena ar;
  chnss_params p{};
  cudaStream_t s = nullptr;
  bool own_stream = false;
  std::vector<chnss::Level3> lv;
  chnss::Pattern pb, pbt;                       // B (N1 x 3 N2), B^T
  chnss::Gather gl, gk;                         // loads -> P1 nodes, Korteweg -> velocity dofs
  int *bnd = nullptr;                           // fine P2 boundary mask
  int ref = 0;
  int top_bc = 0;                               // 1: open (do-nothing) top face
  int *apz = nullptr, *apd = nullptr;           // open top: A_p entries set to 0, diagonal set to 1
  int napz = 0, napd = 0;
  double *Bs = nullptr, *Bts = nullptr, *Mv = nullptr, *Apb = nullptr, *Ap = nullptr, *top = nullptr;
  double *Ls = nullptr, *Ks = nullptr, *Ms = nullptr, *ACs = nullptr;
  double *As = nullptr;                         // velocity operator in 3x3-block SELL order (lv[0].pv3)
  double *Kks[3] = {nullptr, nullptr, nullptr};   // SELL copies of K_kappa (mobility_kind 1)
  double *ebuf = nullptr, *kbuf = nullptr, *loads = nullptr, *G = nullptr, *dinvM = nullptr, *massc = nullptr;
  double *rhs[6] = {}, *xsol[6] = {}, *mt = nullptr, *phia = nullptr;
  double *partial = nullptr, *sum = nullptr, *pinned = nullptr;
  std::unique_ptr<chnss::Prec3<double>> p64;
  std::unique_ptr<chnss::Prec3<float>> p32;
  chnss::KrylovWork kw, kwc, kwa;               // Oseen; CH and air potential; AC
  double *mt0 = nullptr;                        // air-potential scratch (CH group)
  // solve groups (CH + air potential, AC, Oseen) on their own streams, host threads
  bool concurrent = true;
  cudaStream_t sx[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_asm = nullptr, ev_done[3] = {nullptr, nullptr, nullptr};
  // captured preconditioners (0..2 CH species, 3 AC, 4 Oseen) replayed from
  // fixed staging vectors; each captured on a private stream of its own
  cudaStream_t cap[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // bodies of the inner multigrid loops (inner_rtol > 0), one stream per solve group
  cudaStream_t bodyq[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t gexec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *pin[5] = {}, *pout[5] = {};
  // adjoint step (allocated on first use): transposed fine operators, M 1, work
  double *LsT = nullptr, *ACsT = nullptr, *AsT = nullptr, *mvec = nullptr;
  double *arhs = nullptr, *ay = nullptr, *alam = nullptr, *az = nullptr, *atmp = nullptr, *atv = nullptr;
  double *alw[5] = {};
  double *adots = nullptr;                      // device scalars of the parameter gradients
  // per-group work and accumulators of the concurrent adjoint step (AC, CH)
  double *ay_ac = nullptr, *aPhi = nullptr, *v_ac = nullptr;
  double *arhs_ch = nullptr, *ay_ch = nullptr, *atmp_ch = nullptr, *aphi = nullptr, *v_ch = nullptr;
  std::string err;
  ~chnss3_ctx() {
    for (cudaGraphExec_t g : gexec)
      if (g) cudaGraphExecDestroy(g);
    for (cudaStream_t q : cap)
      if (q) cudaStreamDestroy(q);
    for (cudaStream_t q : bodyq)
      if (q) cudaStreamDestroy(q);
    for (cudaStream_t q : sx)
      if (q) cudaStreamDestroy(q);
    if (ev_asm) cudaEventDestroy(ev_asm);
    for (cudaEvent_t e : ev_done)
      if (e) cudaEventDestroy(e);
    if (pinned) cudaFreeHost(pinned);
    if (own_stream && s) cudaStreamDestroy(s);
  }
};

namespace chnss {
namespace {

constexpr double kMassLo3 = 0.5, kMassHi3 = 2.5;   // spectrum of D^-1 M for P1 tetrahedra (Wathen)

std::vector<double> on_pattern(const Pattern &P, const HostCSR &A) {
  std::vector<double> v(P.nnz, 0.0);
  for (int r = 0; r < A.nrows; ++r)
    for (int k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) v[find_col(P, r, A.col[k])] = A.val[k];
  return v;
}

void pattern_from_csr(const HostCSR &A, Pattern &P) {
  P.nrows = A.nrows;
  P.ncols = A.ncols;
  P.h_rowptr = A.rowptr;
  P.h_col = A.col;
  P.nnz = (int)A.col.size();
}

void make_transfer(Arena &ar, const HostCSR &A, Transfer &t) {
  pattern_from_csr(A, t.P);
  finish_transfer(ar, t, A.val);
}

void build_level3(chnss3_ctx *c, Level3 &L, int n, bool fine, const Mesh3Host *coarse) {
  Arena &ar = c->ar;
  const auto &p = c->p;
  const double box[3] = {1.0, 1.0, 1.0};
  const Mesh3Host M = make_mesh3(n, box, c->top_bc == 1);
  L.n = n;
  L.N1 = M.N1;
  L.N2 = M.N2;
  L.E = M.E;
  L.geo.n = n;
  for (int d = 0; d < 3; ++d) L.geo.h[d] = M.h[d];
  const int E = (int)M.E, N1 = (int)M.N1, N2 = (int)M.N2;
  auto p1n = [&](int e, int *r, int *cc) {
    for (int a = 0; a < 4; ++a) r[a] = cc[a] = M.tet[(long)e * 4 + a];
  };
  auto vdn = [&](int e, int *r, int *cc) {
    for (int a = 0; a < 10; ++a)
      for (int d = 0; d < 3; ++d) r[a * 3 + d] = cc[a * 3 + d] = 3 * M.tet2[(long)e * 10 + a] + d;
  };
  pattern_from_elements(N1, N1, E, 4, 4, p1n, L.p1);
  pattern_from_elements(3 * N2, 3 * N2, E, 30, 30, vdn, L.pv);
  upload_pattern(ar, L.p1);
  upload_pattern(ar, L.pv);
  {
    auto p2n = [&](int e, int *r, int *cc) {
      for (int a = 0; a < 10; ++a) r[a] = cc[a] = M.tet2[(long)e * 10 + a];
    };
    pattern_from_elements(N2, N2, E, 10, 10, p2n, L.pv3);
    std::vector<int> hmap;
    upload_pattern(ar, L.pv3, &hmap);
    // every node coupling carries all nine component couplings, so scalar row
    // 3 I + r lists the columns 3 J + d in node order: its entry for block
    // position k of node row I is rowptr[3 I + r] + 3 (k - rowptr3[I]) + d
    const std::vector<int> &r3 = L.pv3.h_rowptr, &rs = L.pv.h_rowptr, &cs = L.pv.h_col;
    std::vector<int> rowof(L.pv3.nnz);
    for (int I = 0; I < N2; ++I) {
      for (int k = r3[I]; k < r3[I + 1]; ++k) rowof[k] = I;
      for (int r = 0; r < 3; ++r)
        if (rs[3 * I + r + 1] - rs[3 * I + r] != 3 * (r3[I + 1] - r3[I]))
          throw Error{CHNSS_ERR_ARG, "velocity pattern without full 3x3 blocks"};
    }
    std::vector<int> m9(9 * (size_t)L.pv3.sell.nent, -1);
    for (long e = 0; e < L.pv3.sell.nent; ++e) {
      const int k = hmap[e];
      if (k < 0) continue;
      const int I = rowof[k], J = L.pv3.h_col[k], lane = (int)(e % 32);
      const size_t base = 9 * (size_t)(e - lane) + lane;
      for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) {
          const int q = rs[3 * I + r] + 3 * (k - r3[I]) + d;
          if (cs[q] != 3 * J + d) throw Error{CHNSS_ERR_ARG, "velocity pattern out of node order"};
          m9[base + 32 * (3 * r + d)] = q;
        }
    }
    L.map9 = ar.upload(m9);
  }
  L.diag1 = ar.upload(diag_positions(L.p1));
  L.diagv = ar.upload(diag_positions(L.pv));
  std::vector<int> hptr, hidx;
  gather_from_elements(L.p1, E, 4, 4, p1n, [](int e, int a, int b) { return e * 16 + a * 4 + b; },
                       [](int, int, int, int, int) { return true; }, L.g1, hptr, hidx);
  upload_gather(ar, L.g1, hptr, hidx);
  auto vkeep = [&](int, int i, int j, int r, int cc) {
    return i % 3 == j % 3 && !M.p2_boundary(r / 3) && !M.p2_boundary(cc / 3);
  };
  gather_from_elements(L.pv, E, 30, 30, vdn, [](int e, int i, int j) { return e * 100 + (i / 3) * 10 + j / 3; },
                       vkeep, L.gj, hptr, hidx);
  upload_gather(ar, L.gj, hptr, hidx);
  // constant operators
  chnss_params none = p;
  const HostCSR hM = host_operator3(n, OP3_M1, none, nullptr), hK = host_operator3(n, OP3_K1, none, nullptr);
  std::vector<double> m1 = on_pattern(L.p1, hM), k1 = on_pattern(L.p1, hK);
  L.M1 = ar.upload(m1);
  L.K1 = ar.upload(k1);
  L.Kp = L.K1;
  std::vector<int> zero_pos, diag_pos;   // open top: Dirichlet rows and columns on the top nodes
  if (M.top_free) {
    std::vector<double> kp = k1;
    for (int r = 0; r < N1; ++r)
      for (int k = L.p1.h_rowptr[r]; k < L.p1.h_rowptr[r + 1]; ++k) {
        const int cc = L.p1.h_col[k];
        if (!M.p1_top(r) && !M.p1_top(cc)) continue;
        kp[k] = r == cc ? 1.0 : 0.0;
        (r == cc ? diag_pos : zero_pos).push_back(k);
      }
    L.Kp = ar.upload(kp);
  }
  std::vector<double> acb(m1.size());
  for (size_t k = 0; k < m1.size(); ++k) acb[k] = m1[k] + p.tau * p.delta_v * k1[k];
  L.ACb = ar.upload(acb);
  for (int sp = 0; sp < 3; ++sp) {
    const double a = std::sqrt(p.tau * p.gamma[sp] / p.beta[sp]);
    std::vector<double> x(m1.size());
    for (size_t k = 0; k < m1.size(); ++k) x[k] = p.tau * p.gamma[sp] * k1[k] + a * m1[k];
    L.X[sp] = ar.upload(x);
    if (p.mobility_kind != 0) {
      L.X2[sp] = ar.alloc<double>(L.p1.nnz);
      if (fine) L.Kk[sp] = ar.alloc<double>(L.p1.nnz);
    }
  }
  if (p.mobility_kind != 0 && !fine) L.phil = ar.alloc<double>(3L * N1);
  // A const = M_v / tau + K_sym with identity rows / zero columns on the no-slip dofs
  const HostCSR hM2 = host_operator3(n, OP3_M2, none, nullptr), hKs = host_operator3(n, OP3_KSYM, none, nullptr);
  std::vector<double> av = on_pattern(L.pv, hKs), mv(L.pv.nnz, 0.0);
  for (int r = 0; r < hM2.nrows; ++r)
    for (int k = hM2.rowptr[r]; k < hM2.rowptr[r + 1]; ++k)
      for (int d = 0; d < 3; ++d) mv[find_col(L.pv, 3 * r + d, 3 * hM2.col[k] + d)] = hM2.val[k];
  for (int r = 0; r < 3 * N2; ++r)
    for (int k = L.pv.h_rowptr[r]; k < L.pv.h_rowptr[r + 1]; ++k) {
      const int cc = L.pv.h_col[k];
      av[k] += mv[k] / p.tau;
      if (M.p2_boundary(r / 3) || M.p2_boundary(cc / 3)) av[k] = r == cc ? 1.0 : 0.0;
    }
  L.Aconst = ar.upload(av);
  L.L = ar.alloc<double>(L.p1.nnz);
  L.AC = ar.alloc<double>(L.p1.nnz);
  L.A = ar.alloc<double>(L.pv.nnz);
  if (!fine) {
    L.vl = ar.alloc<double>(3L * N2);
    L.mul = ar.alloc<double>(4L * N1);
  }
  if (coarse) {
    make_transfer(ar, p1_prolongation3(*coarse), L.t1);
    make_transfer(ar, velocity_prolongation3(*coarse, M), L.tv);
  }
  if (!fine) return;
  // fine-level only: velocity mass, B and B^T (zero no-slip columns), A_p's constant part, loads
  c->Mv = ar.upload(mv);
  const HostCSR hB = host_operator3(n, OP3_B, none, nullptr);
  HostCSR hBz = hB;
  for (size_t k = 0; k < hBz.col.size(); ++k)
    if (M.p2_boundary(hBz.col[k] / 3)) hBz.val[k] = 0.0;
  pattern_from_csr(hBz, c->pb);
  std::vector<double> btv;
  transpose(c->pb, hBz.val, c->pbt, btv);
  std::vector<int> map_b, map_bt;
  upload_pattern(ar, c->pb, &map_b);
  upload_pattern(ar, c->pbt, &map_bt);
  auto sell_of = [](const std::vector<int> &map, const std::vector<double> &v) {
    std::vector<double> out(map.size());
    for (size_t e = 0; e < map.size(); ++e) out[e] = map[e] >= 0 ? v[map[e]] : 0.0;
    return out;
  };
  c->Bs = ar.upload(sell_of(map_b, hBz.val));
  c->Bts = ar.upload(sell_of(map_bt, btv));
  std::vector<double> apb(m1.size());
  for (size_t k = 0; k < m1.size(); ++k) apb[k] = m1[k] / p.tau + p.eta * k1[k];
  c->Apb = ar.upload(apb);
  const HostCSR hT = host_operator3(n, OP3_TOP, none, nullptr);
  c->top = ar.upload(hT.val);
  node_gather(N1, E, 4, [&](int e, int *nd) { for (int a = 0; a < 4; ++a) nd[a] = M.tet[(long)e * 4 + a]; },
              [](int e, int a) { return e * 20 + a; }, [](int) { return true; }, hptr, hidx, c->gl);
  upload_gather(ar, c->gl, hptr, hidx);
  node_gather(N2, E, 10, [&](int e, int *nd) { for (int a = 0; a < 10; ++a) nd[a] = M.tet2[(long)e * 10 + a]; },
              [](int e, int a) { return e * 30 + a * 3; }, [&](int nd) { return !M.p2_boundary(nd); }, hptr, hidx,
              c->gk);
  upload_gather(ar, c->gk, hptr, hidx);
  std::vector<int> bnd(N2);
  for (int i = 0; i < N2; ++i) bnd[i] = M.p2_boundary(i) ? 1 : 0;
  c->bnd = ar.upload(bnd);
  c->ref = M.id1(n / 2, n / 2, n);
  if (M.top_free) {
    c->apz = ar.upload(zero_pos);
    c->apd = ar.upload(diag_pos);
    c->napz = (int)zero_pos.size();
    c->napd = (int)diag_pos.size();
  }
  std::vector<double> dinv(N1);
  const std::vector<int> dpos = diag_positions(L.p1);
  for (int r = 0; r < N1; ++r) dinv[r] = 1.0 / m1[dpos[r]];
  c->dinvM = ar.upload(dinv);
}

template <typename T>
void init_prec3(chnss3_ctx *c, Prec3<T> &P, const std::vector<const Pattern *> &p1s,
                const std::vector<const int *> &d1s, const std::vector<const Transfer *> &t1s,
                const std::vector<const Pattern *> &pvs, const std::vector<const int *> &dvs,
                const std::vector<const Transfer *> &tvs, const std::vector<const double *> &Ls,
                const std::vector<const double *> &ACs, const std::vector<const double *> &K1s,
                const std::vector<const double *> &As, const std::vector<const double *> *Xs,
                const std::vector<const double *> *X2s) {
  Arena &ar = c->ar;
  const Level3 &F = c->lv[0];
  P.L.init(ar, 0, false, p1s, d1s, Ls, t1s, c->partial);
  P.AC.init(ar, 0, false, p1s, d1s, ACs, t1s, c->partial);
  for (int sp = 0; sp < 3; ++sp) {
    P.X[sp].init(ar, 0, false, p1s, d1s, Xs[sp], t1s, c->partial);
    if (X2s) P.X2[sp].init(ar, 0, false, p1s, d1s, X2s[sp], t1s, c->partial);   // set up every step
  }
  P.Kp.keep_dense = true;   // a pure Laplacian: its coarsest level is not mass-dominated
  P.Kp.init(ar, 0, c->top_bc != 1, p1s, d1s, K1s, t1s, c->partial);   // singular for enclosed flow
  P.A.degree = 4;      // as the 2D velocity operator: degree 4 on [hi / 16, hi]
  P.A.ratio = 16.0;
  for (const Level3 &L : c->lv) {   // sweeps through the 3x3-block view
    P.A.bpat.push_back(&L.pv3);
    P.A.bmap.push_back(L.map9);
  }
  P.A.init(ar, 2, false, pvs, dvs, As, tvs, c->partial);
  // inner multigrid solves to a tolerance (Sec. 5) in every block that the
  // paper gives to AMG; M_p^-1 stays the fixed Chebyshev iteration.  Each
  // solve group captures its loop bodies on a stream of its own.
  const double irt = c->p.inner_rtol;
  if (irt > 0.0) {
    const int imax = c->p.inner_maxit;
    P.L.enable_inner(ar, irt, imax, c->bodyq[0]);
    for (int sp = 0; sp < 3; ++sp) {
      P.X[sp].enable_inner(ar, irt, imax, c->bodyq[0]);
      if (X2s) P.X2[sp].enable_inner(ar, irt, imax, c->bodyq[0]);
    }
    P.AC.enable_inner(ar, irt, imax, c->bodyq[1]);
    P.A.enable_inner(ar, irt, imax, c->bodyq[2]);
    P.Kp.enable_inner(ar, irt, imax, c->bodyq[2]);
  }
  for (int sp = 0; sp < 3; ++sp) P.X[sp].setup(c->s);
  P.Kp.setup(c->s);
  const long N1 = F.N1, nent1 = F.p1.sell.nent;
  P.Ms = ar.alloc<T>(nent1);
  P.Aps = ar.alloc<T>(nent1);
  sell_gather<T>(F.p1.sell, 1, F.M1, P.Ms, c->s);
  P.mdinv = ar.alloc<T>(N1);
  vec_convert<double, T>(N1, c->dinvM, P.mdinv, c->s);
  P.mb = ar.alloc<T>(N1);
  P.mx = ar.alloc<T>(N1);
  P.mt = ar.alloc<T>(N1);
}

void create3(chnss3_ctx *c, int n) {
  Arena &ar = c->ar;
  const auto &p = c->p;
  std::vector<int> sizes{n};
  while (sizes.back() % 2 == 0 && sizes.back() >= 4) sizes.push_back(sizes.back() / 2);
  const int nl = (int)sizes.size();
  c->lv.resize(nl);
  const double box[3] = {1.0, 1.0, 1.0};
  for (int l = 0; l < nl; ++l) {
    const Mesh3Host coarse = l + 1 < nl ? make_mesh3(sizes[l + 1], box, c->top_bc == 1) : Mesh3Host{};
    build_level3(c, c->lv[l], sizes[l], l == 0, l + 1 < nl ? &coarse : nullptr);
  }
  const Level3 &F = c->lv[0];
  const long N1 = F.N1, nv = 3 * F.N2, E = F.E;
  CHNSS_CK(cudaMemcpyToSymbolAsync(c3, &reference3(), sizeof(Tet3Ref), 0, cudaMemcpyHostToDevice, c->s));
  c->ebuf = ar.alloc<double>(100 * E);
  c->kbuf = ar.alloc<double>(30 * E);
  c->loads = ar.alloc<double>(5 * N1);
  c->G = ar.alloc<double>(nv);
  c->Ap = ar.alloc<double>(F.p1.nnz);
  const long nent1 = F.p1.sell.nent;
  c->Ls = ar.alloc<double>(nent1);
  c->Ks = ar.alloc<double>(nent1);
  c->Ms = ar.alloc<double>(nent1);
  c->ACs = ar.alloc<double>(nent1);
  c->As = ar.alloc<double>(9 * F.pv3.sell.nent);
  sell_gather<double>(F.p1.sell, 1, F.K1, c->Ks, c->s);
  sell_gather<double>(F.p1.sell, 1, F.M1, c->Ms, c->s);
  for (int k = 0; k < 3; ++k) {
    c->rhs[k] = ar.alloc<double>(2 * N1);
    c->xsol[k] = ar.alloc<double>(2 * N1);
  }
  c->rhs[3] = ar.alloc<double>(N1);
  c->rhs[4] = ar.alloc<double>(N1);
  c->rhs[5] = ar.alloc<double>(nv + N1);
  c->xsol[5] = ar.alloc<double>(nv + N1);
  c->mt = ar.alloc<double>(N1);
  for (int g = 0; g < 5; ++g) {
    const long len = g < 3 ? 2 * N1 : g == 3 ? N1 : nv + N1;
    c->pin[g] = ar.alloc<double>(len);
    c->pout[g] = ar.alloc<double>(len);
  }
  for (cudaStream_t &q : c->cap) CHNSS_CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
  int prio_low = 0, prio_high = 0;   // the Oseen group is the longest: highest priority
  CHNSS_CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  for (int w = 0; w < 3; ++w)
    CHNSS_CK(cudaStreamCreateWithPriority(&c->sx[w], cudaStreamNonBlocking, w == 2 ? prio_high : prio_low));
  CHNSS_CK(cudaEventCreateWithFlags(&c->ev_asm, cudaEventDisableTiming));
  for (cudaEvent_t &e : c->ev_done) CHNSS_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  c->mt0 = ar.alloc<double>(N1);
  c->phia = ar.alloc<double>(N1);
  c->partial = ar.alloc<double>(64L * kReduceMaxBlocks);
  c->sum = ar.alloc<double>(4);
  CHNSS_CK(cudaHostAlloc(&c->pinned, 32 * sizeof(double), cudaHostAllocDefault));
  c->kw.init(ar, p.restart, nv + N1, c->pinned, p.ortho == 1);
  c->kwc.init(ar, p.restart, 2 * N1, c->pinned + 8, p.ortho == 1);
  c->kwa.init(ar, p.restart, N1, c->pinned + 16, p.ortho == 1);
  // Chebyshev coefficients of M_p^-1 (degree 5 on D^-1 M over [1/2, 5/2])
  {
    const double theta = 0.5 * (kMassHi3 + kMassLo3), delta = 0.5 * (kMassHi3 - kMassLo3), sigma = theta / delta;
    std::vector<double> mc(13);
    mc[0] = 1.0 / theta;
    double rho = 1.0 / sigma;
    for (int k = 1; k <= 4; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      mc[1 + 3 * (k - 1)] = 1.0 + rn * rho;
      mc[2 + 3 * (k - 1)] = -rn * rho;
      mc[3 + 3 * (k - 1)] = 2.0 * rn / delta;
      rho = rn;
    }
    c->massc = ar.upload(mc);
  }
  // hierarchies: P1 (L, AC, X per species, K_p singular) and the velocity operator (scalar)
  std::vector<const Pattern *> p1s, pvs;
  std::vector<const int *> d1s, dvs;
  std::vector<const Transfer *> t1s, tvs;
  std::vector<const double *> Ls, ACs, K1s, As, Xs[3], X2s[3];
  for (int l = 0; l < nl; ++l) {
    const Level3 &L = c->lv[l];
    p1s.push_back(&L.p1);
    pvs.push_back(&L.pv);
    d1s.push_back(L.diag1);
    dvs.push_back(L.diagv);
    t1s.push_back(&L.t1);
    tvs.push_back(&L.tv);
    Ls.push_back(L.L);
    ACs.push_back(L.AC);
    K1s.push_back(L.Kp);
    As.push_back(L.A);
    for (int sp = 0; sp < 3; ++sp) {
      Xs[sp].push_back(L.X[sp]);
      X2s[sp].push_back(L.X2[sp]);
    }
  }
  const std::vector<const double *> *x2 = p.mobility_kind != 0 ? X2s : nullptr;
  if (p.inner_rtol > 0.0)
    for (cudaStream_t &q : c->bodyq) CHNSS_CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
  if (p.mobility_kind != 0)
    for (int sp = 0; sp < 3; ++sp) c->Kks[sp] = ar.alloc<double>(nent1);
  if (p.precision == 0) {
    c->p64.reset(new Prec3<double>);
    init_prec3(c, *c->p64, p1s, d1s, t1s, pvs, dvs, tvs, Ls, ACs, K1s, As, Xs, x2);
  } else {
    c->p32.reset(new Prec3<float>);
    c->p32->A.bf16 = p.precision == 2;
    init_prec3(c, *c->p32, p1s, d1s, t1s, pvs, dvs, tvs, Ls, ACs, K1s, As, Xs, x2);
  }
  CHNSS_CK(cudaStreamSynchronize(c->s));
}

template <typename T>
void setup_prec3(chnss3_ctx *c, Prec3<T> &P, cudaStream_t s) {
  P.L.setup(s);
  P.AC.setup(s);
  P.A.setup(s);
  if (c->p.mobility_kind != 0)
    for (int sp = 0; sp < 3; ++sp) P.X2[sp].setup(s);
  sell_gather<T>(c->lv[0].p1.sell, 1, c->Ap, P.Aps, s);
}

void assemble3(chnss3_ctx *c, const chnss_state *st) {
  cudaStream_t s = c->s;
  const auto &p = c->p;
  const int nl = (int)c->lv.size();
  Fields3 f{};
  for (int i = 0; i < 4; ++i) {
    f.alpha[i] = p.alpha[i];
    f.beta[i] = p.beta[i];
  }
  f.beta_v = p.beta_v;
  for (int l = 0; l < nl; ++l) {
    Level3 &L = c->lv[l];
    if (l > 0) {
      const Level3 &Fn = c->lv[l - 1];
      const double *vf = l == 1 ? st->v : Fn.vl;
      k3_inject<<<nb3(3L * L.N2), kTPB3, 0, s>>>(Fn.n, 1, vf, L.vl);
      CHNSS_LAUNCH_CK();
      for (int i = 0; i < 4; ++i) {
        const double *mf = l == 1 ? st->mu[i] : Fn.mul + (long)i * Fn.N1;
        k3_inject<<<nb3(L.N1), kTPB3, 0, s>>>(Fn.n, 0, mf, L.mul + (long)i * L.N1);
        CHNSS_LAUNCH_CK();
      }
    }
    f.v = l == 0 ? st->v : L.vl;
    for (int i = 0; i < 4; ++i) f.mu[i] = l == 0 ? st->mu[i] : L.mul + (long)i * L.N1;
    k3_conv<<<nb3(L.E), kTPB3, 0, s>>>(L.geo, f, 0, 0, c->ebuf);
    CHNSS_LAUNCH_CK();
    launch_gather(L.g1, 1, c->ebuf, p.tau, L.M1, 1.0, L.L, s);
    launch_gather(L.g1, 1, c->ebuf, p.tau, L.ACb, 1.0, L.AC, s);
    k3_conv<<<nb3(L.E), kTPB3, 0, s>>>(L.geo, f, 1, 1, c->ebuf);
    CHNSS_LAUNCH_CK();
    launch_gather(L.gj, 1, c->ebuf, 1.0, L.Aconst, 1.0, L.A, s);
    if (p.mobility_kind != 0) {   // X2 = tau K_kappa(phi^k) + a M, phi injected on the coarse levels
      for (int sp = 0; sp < 3; ++sp) {
        if (l > 0) {
          const Level3 &Fn = c->lv[l - 1];
          const double *pf = l == 1 ? st->phi[sp] : Fn.phil + (long)sp * Fn.N1;
          k3_inject<<<nb3(L.N1), kTPB3, 0, s>>>(Fn.n, 0, pf, L.phil + (long)sp * L.N1);
          CHNSS_LAUNCH_CK();
        }
        const double *ph = l == 0 ? st->phi[sp] : L.phil + (long)sp * L.N1;
        const double a = std::sqrt(p.tau * p.gamma[sp] / p.beta[sp]);
        k3_wstiff<<<nb3(L.E), kTPB3, 0, s>>>(L.geo, ph, p.gamma[sp], p.mobility_m0, c->ebuf);
        CHNSS_LAUNCH_CK();
        launch_gather(L.g1, 1, c->ebuf, p.tau, L.M1, a, L.X2[sp], s);
        if (l == 0) launch_gather(L.g1, 1, c->ebuf, 1.0, nullptr, 0.0, L.Kk[sp], s);
      }
    }
  }
  const Level3 &F = c->lv[0];
  const int N1 = (int)F.N1;
  const long nv = 3 * F.N2;
  f.v = st->v;
  for (int i = 0; i < 4; ++i) f.mu[i] = st->mu[i];
  for (int i = 0; i < 3; ++i) f.phi[i] = st->phi[i];
  f.Phi = st->Phi_v;
  // A_p = M / tau + eta K + C(w)
  k3_conv<<<nb3(F.E), kTPB3, 0, s>>>(F.geo, f, 0, 1, c->ebuf);
  CHNSS_LAUNCH_CK();
  launch_gather(F.g1, 1, c->ebuf, 1.0, c->Apb, 1.0, c->Ap, s);
  if (c->napz > 0) {   // PCD outflow condition on the open top
    k3_set_entries<<<nb3(c->napz), kTPB3, 0, s>>>(c->napz, c->apz, 0.0, c->Ap);
    CHNSS_LAUNCH_CK();
    k3_set_entries<<<nb3(c->napd), kTPB3, 0, s>>>(c->napd, c->apd, 1.0, c->Ap);
    CHNSS_LAUNCH_CK();
  }
  // potential and Korteweg loads
  k3_loads<<<nb3(F.E), kTPB3, 0, s>>>(F.geo, f, c->ebuf, c->kbuf);
  CHNSS_LAUNCH_CK();
  for (int k = 0; k < 5; ++k) launch_gather(c->gl, 1, c->ebuf + 4 * k, 1.0, nullptr, 0.0, c->loads + (long)k * N1, s);
  launch_gather(c->gk, 3, c->kbuf, 1.0, nullptr, 0.0, c->G, s);
  // right-hand sides
  SpmvArgs none;
  for (int sp = 0; sp < 3; ++sp) {
    spmv_csr<double>(F.p1, F.M1, 1, st->phi[sp], c->rhs[sp], SPMV_PLAIN, none, s);
    const double cc = p.tau * p.gamma[sp] / p.beta[sp], sb = sp == 2 ? -p.beta[2] : 0.0;
    k3_flux_rhs<<<nb3(N1), kTPB3, 0, s>>>(N1, c->loads + (long)sp * N1, c->top, st->phi[2], c->ref, p.evap_rate,
                                         p.phi_s_inf, sb, cc, c->rhs[sp] + N1);
    CHNSS_LAUNCH_CK();
  }
  spmv_csr<double>(F.p1, F.M1, 1, st->Phi_v, c->rhs[3], SPMV_PLAIN, none, s);
  k3_ac_rhs<<<nb3(N1), kTPB3, 0, s>>>(N1, c->loads + 4L * N1, c->top, st->phi[2], c->ref, p.evap_rate, p.phi_s_inf,
                                     p.tau * p.gamma_v, p.ac_top_flux ? p.tau * p.delta_v : 0.0, c->rhs[3]);
  CHNSS_LAUNCH_CK();
  spmv_csr<double>(F.pv, c->Mv, 1, st->v, c->rhs[5], SPMV_PLAIN, none, s);
  vec_axpby(nv, 1.0, c->G, 1.0 / p.tau, c->rhs[5], s);
  k3_mask<<<nb3(nv), kTPB3, 0, s>>>(nv, c->bnd, c->rhs[5]);
  CHNSS_LAUNCH_CK();
  vec_fill(N1, 0.0, c->rhs[5] + nv, s);
  // SELL copies of the operators FGMRES applies, multigrid setup
  sell_gather<double>(F.p1.sell, 1, F.L, c->Ls, s);
  sell_gather<double>(F.p1.sell, 1, F.AC, c->ACs, s);
  sell_gather9<double>(F.pv3.sell.nent, F.map9, F.A, c->As, s);
  if (p.mobility_kind != 0)
    for (int sp = 0; sp < 3; ++sp) sell_gather<double>(F.p1.sell, 1, F.Kk[sp], c->Kks[sp], s);
  if (c->p32) setup_prec3(c, *c->p32, s);
  else setup_prec3(c, *c->p64, s);
}

// z = the hierarchy's result in FP64: the FP64 iterate of an inner solve
// (an FP32 rounding would cap the preconditioner's accuracy), else x[0]
template <typename T>
void mg_output(MGHier<T> &h, long n, double *z, cudaStream_t s) {
  if (h.inner_rtol > 0.0) vec_copy(n, h.iterate64(), z, s);
  else vec_convert<T, double>(n, h.output(), z, s);
}

template <typename T>
void mg_apply(MGHier<T> &h, long n, const double *r, double *z, cudaStream_t s) {
  vec_convert<double, T>(n, r, h.input(), s);
  h.apply(s);
  mg_output(h, n, z, s);
}

template <typename T>
void prec_ch3(chnss3_ctx *c, Prec3<T> &P, int sp, const double *r, double *z, cudaStream_t s) {
  const long N1 = c->lv[0].N1;
  mg_apply(P.L, N1, r, z, s);
  // S~^-1 = X2^-1 M X1^-1 (matching factors of eqn::schurCH; X2 = X1 with
  // constant mobility)
  MGHier<T> &X1 = P.X[sp], &X2 = c->p.mobility_kind != 0 ? P.X2[sp] : P.X[sp];
  vec_convert<double, T>(N1, r + N1, X1.input(), s);
  X1.apply(s);
  SpmvArgs none;
  spmv_sell<T>(c->lv[0].p1, P.Ms, 1, X1.output(), X2.input(), SPMV_PLAIN, none, s);
  X2.apply(s);
  mg_output(X2, N1, z + N1, s);
}

template <typename T>
void prec_ns3(chnss3_ctx *c, Prec3<T> &P, const double *r, double *z, cudaStream_t s) {
  const Level3 &F = c->lv[0];
  const long nv = 3 * F.N2, N1 = F.N1;
  mg_apply(P.A, nv, r, z, s);
  // pressure convection-diffusion: M_p^-1 A_p K_p^-1
  vec_convert<double, T>(N1, r + nv, P.Kp.input(), s);
  P.Kp.apply(s);
  SpmvArgs none;
  spmv_sell<T>(F.p1, P.Aps, 1, P.Kp.output(), P.mb, SPMV_PLAIN, none, s);
  vec_scale_dinv<T>((int)N1, c->massc, P.mdinv, P.mb, P.mx, s);
  SpmvArgs a;
  a.b = P.mb;
  a.dinv = P.mdinv;
  T *cur = P.mx, *other = P.mt;
  for (int k = 1; k <= 4; ++k) {
    a.coef = c->massc + 1 + 3 * (k - 1);
    a.w = k == 1 ? nullptr : other;
    spmv_sell<T>(F.p1, P.Ms, 1, cur, other, SPMV_CHEB, a, s);
    std::swap(cur, other);
  }
  vec_convert<T, double>(N1, cur, z + nv, s);
}

void prec_body3(chnss3_ctx *c, int g, const double *r, double *z, cudaStream_t s) {
  if (g < 3) {
    if (c->p32) prec_ch3(c, *c->p32, g, r, z, s);
    else prec_ch3(c, *c->p64, g, r, z, s);
  } else if (g == 3) {
    if (c->p32) mg_apply(c->p32->AC, c->lv[0].N1, r, z, s);
    else mg_apply(c->p64->AC, c->lv[0].N1, r, z, s);
  } else {
    if (c->p32) prec_ns3(c, *c->p32, r, z, s);
    else prec_ns3(c, *c->p64, r, z, s);
  }
}

// z = P_g r through the captured graph of preconditioner g (captured at the
// first application; the hierarchies' values change in place between steps)
void run_prec3(chnss3_ctx *c, int g, long n, const double *r, double *z, cudaStream_t s) {
  vec_copy(n, r, c->pin[g], s);
  if (!c->gexec[g]) {
    cudaGraph_t graph = nullptr;
    CHNSS_CK(cudaStreamBeginCapture(c->cap[g], cudaStreamCaptureModeThreadLocal));
    try {
      prec_body3(c, g, c->pin[g], c->pout[g], c->cap[g]);
    } catch (...) {
      cudaStreamEndCapture(c->cap[g], &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    CHNSS_CK(cudaStreamEndCapture(c->cap[g], &graph));
    const cudaError_t e = cudaGraphInstantiate(&c->gexec[g], graph, 0);
    cudaGraphDestroy(graph);
    CHNSS_CK(e);
  }
  CHNSS_CK(cudaGraphLaunch(c->gexec[g], s));
  vec_copy(n, c->pout[g], z, s);
}

struct CH3Op : LinearOperator {
  chnss3_ctx *c;
  int sp;
  CH3Op(chnss3_ctx *c_, int sp_) : c(c_), sp(sp_) {}
  long size() const override { return 2 * c->lv[0].N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const auto &p = c->p;
    const double tau = p.tau, g = p.gamma[sp], b = p.beta[sp];
    // [[M + tau C, tau K_kappa], [tau gamma K, -(tau gamma / beta) M]] (K_kappa = gamma K
    // with constant mobility)
    if (p.mobility_kind != 0)
      spmv_sell_ch(c->lv[0].p1, c->Ls, c->Ks, c->Kks[sp], c->Ms, tau, tau * g, -tau * g / b, x, y, s);
    else
      spmv_sell_ch(c->lv[0].p1, c->Ls, c->Ks, nullptr, c->Ms, tau * g, tau * g, -tau * g / b, x, y, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec3(c, sp, 2 * c->lv[0].N1, r, z, s); }
};

struct AC3Op : LinearOperator {
  chnss3_ctx *c;
  explicit AC3Op(chnss3_ctx *c_) : c(c_) {}
  long size() const override { return c->lv[0].N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    SpmvArgs none;
    spmv_sell<double>(c->lv[0].p1, c->ACs, 1, x, y, SPMV_PLAIN, none, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec3(c, 3, c->lv[0].N1, r, z, s); }
};

struct NS3Op : LinearOperator {
  chnss3_ctx *c;
  explicit NS3Op(chnss3_ctx *c_) : c(c_) {}
  long size() const override { return 3 * c->lv[0].N2 + c->lv[0].N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const long nv = 3 * c->lv[0].N2;
    SpmvArgs none;
    spmv_sell_bsr3<double>(c->lv[0].pv3, c->As, x, y, SPMV_PLAIN, none, s);
    spmv_sell<double>(c->pbt, c->Bts, 1, x + nv, y, SPMV_ADD, none, s);
    spmv_sell<double>(c->pb, c->Bs, 1, x, y + nv, SPMV_PLAIN, none, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override {
    run_prec3(c, 4, 3 * c->lv[0].N2 + c->lv[0].N1, r, z, s);
  }
};

// The Cahn-Hilliard species and then the air potential (which needs the
// new phase fields), on stream q.
chnss_status group_ch3(chnss3_ctx *c, const chnss_state *in, chnss_state *out, chnss_solve_info *inf,
                       cudaStream_t q) {
  const auto &p = c->p;
  const Level3 &F = c->lv[0];
  const int N1 = (int)F.N1;
  chnss_status worst = CHNSS_OK;
  auto keep = [&](chnss_status st) { if (worst == CHNSS_OK) worst = st; };
  for (int sp = 0; sp < 3; ++sp) {
    CH3Op op(c, sp);
    keep(fgmres(op, c->rhs[sp], c->xsol[sp], p.rtol, p.atol, p.maxit, c->kwc, &inf[sp], q));
    vec_copy(N1, c->xsol[sp], out->phi[sp], q);
    vec_copy(N1, c->xsol[sp] + N1, out->mu[sp], q);
  }
  // air potential: M mu_a = f_a + beta_a K phi_a^{k+1}
  k3_air<<<nb3(N1), kTPB3, 0, q>>>(N1, out->phi[0], out->phi[1], out->phi[2], c->phia);
  CHNSS_LAUNCH_CK();
  k3_flux_rhs<<<nb3(N1), kTPB3, 0, q>>>(N1, c->loads + 3L * N1, c->top, in->phi[2], c->ref, p.evap_rate,
                                       p.phi_s_inf, p.beta[3], -1.0, c->rhs[4]);
  CHNSS_LAUNCH_CK();
  SpmvArgs none;
  spmv_csr<double>(F.p1, F.K1, 1, c->phia, c->mt0, SPMV_PLAIN, none, q);
  vec_axpby(N1, p.beta[3], c->mt0, 1.0, c->rhs[4], q);
  keep(pcg(F.p1, F.M1, c->dinvM, c->rhs[4], out->mu[3], 1e-12, 1000, c->kwc, &inf[4], q));
  return worst;
}

chnss_status group_ns3(chnss3_ctx *c, chnss_state *out, chnss_solve_info *inf, cudaStream_t q) {
  const auto &p = c->p;
  const Level3 &F = c->lv[0];
  const int N1 = (int)F.N1;
  const long nv = 3 * F.N2;
  NS3Op op(c);
  const double rt = p.ns_rtol > 0.0 ? p.ns_rtol : p.rtol, at = p.ns_rtol > 0.0 ? p.ns_atol : p.atol;
  const chnss_status st = fgmres(op, c->rhs[5], c->xsol[5], rt, at, p.maxit, c->kw, &inf[5], q);
  vec_copy(nv, c->xsol[5], out->v, q);
  vec_copy(N1, c->xsol[5] + nv, out->p, q);
  if (c->top_bc == 1) return st;   // the do-nothing top fixes the pressure
  // zero-mean pressure: p -= (1^T M p) / (1^T M 1), 1^T M 1 = |box| = 1
  SpmvArgs none;
  spmv_csr<double>(F.p1, F.M1, 1, out->p, c->mt, SPMV_PLAIN, none, q);
  vsum<double>(N1, c->mt, c->sum, c->partial, q);
  k3_shift<<<nb3(N1), kTPB3, 0, q>>>(N1, out->p, c->sum, 1.0);
  CHNSS_LAUNCH_CK();
  return st;
}

// Assembly on the context stream, then the three independent solve groups
// (all coefficients at t_k): concurrently on their streams by three host
// threads, or one after the other; the results are the same either way.
chnss_status step3(chnss3_ctx *c, const chnss_state *in, chnss_state *out, chnss_solve_info *inf) {
  cudaStream_t s = c->s;
  assemble3(c, in);
  CHNSS_CK(cudaEventRecord(c->ev_asm, s));
  chnss_status st[3] = {CHNSS_OK, CHNSS_OK, CHNSS_OK};
  std::exception_ptr err[3];
  int dev = 0;
  CHNSS_CK(cudaGetDevice(&dev));
  auto run = [&](int w) {
    try {
      CHNSS_CK(cudaSetDevice(dev));
      cudaStream_t q = c->sx[w];
      CHNSS_CK(cudaStreamWaitEvent(q, c->ev_asm, 0));
      if (w == 0) {
        st[0] = group_ch3(c, in, out, inf, q);
      } else if (w == 1) {
        AC3Op op(c);
        st[1] = fgmres(op, c->rhs[3], out->Phi_v, c->p.rtol, c->p.atol, c->p.maxit, c->kwa, &inf[3], q);
      } else {
        st[2] = group_ns3(c, out, inf, q);
      }
      CHNSS_CK(cudaEventRecord(c->ev_done[w], q));
    } catch (...) {
      err[w] = std::current_exception();
    }
  };
  if (c->concurrent) {
    std::thread t_ac(run, 1), t_ns(run, 2);
    run(0);
    t_ac.join();
    t_ns.join();
  } else {
    for (int w = 0; w < 3; ++w) run(w);
  }
  for (std::exception_ptr &e : err)
    if (e) std::rethrow_exception(e);
  for (cudaEvent_t e : c->ev_done) CHNSS_CK(cudaStreamWaitEvent(s, e, 0));
  CHNSS_CK(cudaStreamSynchronize(s));
  for (chnss_status x : st)
    if (x != CHNSS_OK) return x;
  return CHNSS_OK;
}

// ---------------------------------------------------------------------------
// Adjoint of the 3D step: for each solve x = A(u)^-1 b(u), given the adjoint
// xbar of its solution, y = A^-T xbar (FGMRES on the transposed operator,
// preconditioned by the forward block preconditioner), then
// ubar += (db/du)^T y - (d(A(u) x)/du)^T y (the k3_adj_* element kernels).
constexpr double kAdjointRtol3 = 1e-12;

struct CH3OpT : LinearOperator {   // [[L^T, tau g K], [tau K_kappa, -(tau g / b) M]] (K, K_kappa symmetric)
  chnss3_ctx *c;
  int sp;
  CH3OpT(chnss3_ctx *c_, int sp_) : c(c_), sp(sp_) {}
  long size() const override { return 2 * c->lv[0].N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const auto &p = c->p;
    const double tau = p.tau, g = p.gamma[sp], b = p.beta[sp];
    if (p.mobility_kind != 0)
      spmv_sell_ch(c->lv[0].p1, c->LsT, c->Kks[sp], c->Ks, c->Ms, tau * g, tau, -tau * g / b, x, y, s);
    else
      spmv_sell_ch(c->lv[0].p1, c->LsT, c->Ks, nullptr, c->Ms, tau * g, tau * g, -tau * g / b, x, y, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec3(c, sp, 2 * c->lv[0].N1, r, z, s); }
};

struct AC3OpT : LinearOperator {
  chnss3_ctx *c;
  explicit AC3OpT(chnss3_ctx *c_) : c(c_) {}
  long size() const override { return c->lv[0].N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    SpmvArgs none;
    spmv_sell<double>(c->lv[0].p1, c->ACsT, 1, x, y, SPMV_PLAIN, none, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec3(c, 3, c->lv[0].N1, r, z, s); }
};

struct NS3OpT : LinearOperator {   // [[A^T, B^T], [B, 0]]
  chnss3_ctx *c;
  explicit NS3OpT(chnss3_ctx *c_) : c(c_) {}
  long size() const override { return 3 * c->lv[0].N2 + c->lv[0].N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const long nv = 3 * c->lv[0].N2;
    SpmvArgs none;
    spmv_sell<double>(c->lv[0].pv, c->AsT, 1, x, y, SPMV_PLAIN, none, s);
    spmv_sell<double>(c->pbt, c->Bts, 1, x + nv, y, SPMV_ADD, none, s);
    spmv_sell<double>(c->pb, c->Bs, 1, x, y + nv, SPMV_PLAIN, none, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override {
    run_prec3(c, 4, 3 * c->lv[0].N2 + c->lv[0].N1, r, z, s);
  }
};

void adjoint_alloc3(chnss3_ctx *c) {
  if (c->LsT) return;
  Arena &ar = c->ar;
  const Level3 &F = c->lv[0];
  const long N1 = F.N1, nv = 3 * F.N2;
  c->LsT = ar.alloc<double>(F.p1.sell.nent);
  c->ACsT = ar.alloc<double>(F.p1.sell.nent);
  c->AsT = ar.alloc<double>(F.pv.sell.nent);
  c->mvec = ar.alloc<double>(N1);
  c->arhs = ar.alloc<double>(nv + N1);
  c->ay = ar.alloc<double>(nv + N1);
  c->alam = ar.alloc<double>(3 * N1);
  c->az = ar.alloc<double>(N1);
  c->atmp = ar.alloc<double>(N1);
  c->atv = ar.alloc<double>(nv);
  for (double *&w : c->alw) w = ar.alloc<double>(N1);
  c->adots = ar.alloc<double>(32);
  c->ay_ac = ar.alloc<double>(N1);
  c->aPhi = ar.alloc<double>(N1);
  c->v_ac = ar.alloc<double>(nv);
  c->arhs_ch = ar.alloc<double>(2 * N1);
  c->ay_ch = ar.alloc<double>(2 * N1);
  c->atmp_ch = ar.alloc<double>(N1);
  c->aphi = ar.alloc<double>(3 * N1);
  c->v_ch = ar.alloc<double>(nv);
  vec_fill(N1, 1.0, c->atmp, c->s);
  SpmvArgs none;
  spmv_csr<double>(F.p1, F.M1, 1, c->atmp, c->mvec, SPMV_PLAIN, none, c->s);
}

// The adjoint of step3: three independent groups as in the forward step
// (Oseen; Allen-Cahn; air potential -> Cahn-Hilliard), each with its own
// Krylov work, scratch vectors, slice of the element buffers and
// accumulators.  The groups' contributions to the shared adjoints (v, phi,
// Phi_v) are added on the context stream after the join in a fixed order,
// then the potential-load adjoint and the parameter gradients, so the result
// does not depend on whether the groups overlap.
chnss_status adjoint_step3(chnss3_ctx *c, const chnss_state *stk, const chnss_state *st1, const chnss_state *lam,
                           chnss_state *out, double *grad, chnss_solve_info *inf) {
  const auto &p = c->p;
  const bool var = p.mobility_kind != 0;
  adjoint_alloc3(c);
  assemble3(c, stk);
  cudaStream_t s = c->s;
  const Level3 &F = c->lv[0];
  const int N1 = (int)F.N1;
  const long nv = 3 * F.N2, E = F.E;
  const double tau = p.tau;
  SpmvArgs none;
  sell_gather_transposed(F.p1.sell, 1, F.L, c->LsT, s);
  sell_gather_transposed(F.p1.sell, 1, F.AC, c->ACsT, s);
  sell_gather_transposed(F.pv.sell, 1, F.A, c->AsT, s);
  for (int k = 0; k < 3; ++k) vec_fill(N1, 0.0, out->phi[k], s);
  for (int k = 0; k < 4; ++k) vec_fill(N1, 0.0, out->mu[k], s);
  vec_fill(N1, 0.0, out->Phi_v, s);
  vec_fill(nv, 0.0, out->v, s);
  vec_fill(N1, 0.0, out->p, s);
  vec_fill(32, 0.0, c->adots, s);
  double *D = c->adots;
  Fields3 fk{};
  for (int i = 0; i < 3; ++i) fk.phi[i] = stk->phi[i];
  fk.Phi = stk->Phi_v;
  for (int i = 0; i < 4; ++i) fk.beta[i] = p.beta[i];
  fk.beta_v = p.beta_v;
  CHNSS_CK(cudaEventRecord(c->ev_asm, s));
  // ---- Oseen: [[A^T, B^T], [B, 0]] y = (masked lambda_v, lambda_p) ----------
  auto group_ns = [&](cudaStream_t q) -> chnss_status {
    double *bufP = c->ebuf, *bufV = c->ebuf + 20 * E;   // element scratch [0, 50 E)
    KrylovWork &kw = c->kw;
    vec_copy(nv, lam->v, c->arhs, q);
    k3_mask<<<nb3(nv), kTPB3, 0, q>>>(nv, c->bnd, c->arhs);
    CHNSS_LAUNCH_CK();
    if (c->top_bc == 0) {   // transpose of the zero-mean pressure shift (|box| = 1)
      vsum<double>(N1, lam->p, c->sum, kw.partial, q);
      k3_mean_shift_T<<<nb3(N1), kTPB3, 0, q>>>(N1, lam->p, c->mvec, c->sum, 1.0, c->arhs + nv);
      CHNSS_LAUNCH_CK();
    } else {                // open top: the outflow fixes the pressure level, no shift
      vec_copy(N1, lam->p, c->arhs + nv, q);
    }
    chnss_status st;
    {
      NS3OpT op(c);
      st = fgmres(op, c->arhs, c->ay, kAdjointRtol3, 0.0, p.maxit, kw, &inf[5], q);
    }
    const double *yv = c->ay;
    spmv_csr<double>(F.pv, c->Mv, 1, yv, c->atv, SPMV_PLAIN, none, q);
    vec_axpby(nv, 1.0 / tau, c->atv, 1.0, out->v, q);                          // (M_v / tau)^T y_v
    k3_adj_korteweg<<<nb3(E), kTPB3, 0, q>>>(F.geo, fk, yv, bufP);
    CHNSS_LAUNCH_CK();
    for (int f = 0; f < 4; ++f) {
      double *dst = f < 3 ? out->phi[f] : out->Phi_v;
      launch_gather(c->gl, 1, bufP + 4 * f, 1.0, dst, 1.0, dst, q);
    }
    vec_copy(nv, st1->v, c->atv, q);                                            // J(w) acts on v^(k+1)
    k3_mask<<<nb3(nv), kTPB3, 0, q>>>(nv, c->bnd, c->atv);
    CHNSS_LAUNCH_CK();
    k3_adj_conv_p2<<<nb3(E), kTPB3, 0, q>>>(F.geo, c->atv, yv, bufV, bufP);
    CHNSS_LAUNCH_CK();
    launch_gather(c->gk, 3, bufV, -1.0, out->v, 1.0, out->v, q);               // - (d J(w) x / dv)^T y
    launch_gather(c->gl, 1, bufP, 1.0, nullptr, 0.0, c->atmp, q);
    for (int i = 0; i < 4; ++i) vec_axpby(N1, -p.alpha[i], c->atmp, 1.0, out->mu[i], q);   // ds/dmu_i = alpha_i grad psi
    return st;
  };
  // ---- Allen-Cahn -------------------------------------------------------------
  auto group_ac = [&](cudaStream_t q) -> chnss_status {
    double *bufV = c->ebuf + 50 * E;                    // element scratch [50 E, 80 E)
    chnss_status st;
    {
      AC3OpT op(c);
      st = fgmres(op, lam->Phi_v, c->ay_ac, kAdjointRtol3, 0.0, p.maxit, c->kwa, &inf[3], q);
    }
    spmv_csr<double>(F.p1, F.M1, 1, c->ay_ac, c->aPhi, SPMV_PLAIN, none, q);
    vec_fill(N1, 0.0, c->alw[4], q);
    vec_axpby(N1, -tau * p.gamma_v, c->ay_ac, 0.0, c->alw[4], q);
    k3_adj_conv_p1<<<nb3(E), kTPB3, 0, q>>>(F.geo, st1->Phi_v, c->ay_ac, bufV);
    CHNSS_LAUNCH_CK();
    launch_gather(c->gk, 3, bufV, -tau, nullptr, 0.0, c->v_ac, q);
    dot<double>(N1, c->top, c->ay_ac, D + 1, c->kwa.partial, q);
    return st;
  };
  // ---- air potential (M z = lambda_mu_a), then Cahn-Hilliard, three species -----
  auto group_ch = [&](cudaStream_t q, chnss_status *st_mu) -> chnss_status {
    double *bufP = c->ebuf + 80 * E, *bufV = c->kbuf;   // element scratch [80 E, 100 E) and the Korteweg buffer
    double *tmp = c->atmp_ch;
    KrylovWork &kw = c->kwc;
    *st_mu = pcg(F.p1, F.M1, c->dinvM, lam->mu[3], c->az, kAdjointRtol3, 1000, kw, &inf[4], q);
    spmv_csr<double>(F.p1, F.K1, 1, c->az, tmp, SPMV_PLAIN, none, q);
    for (int i = 0; i < 3; ++i) {   // mu_a^(k+1) depends on phi^(k+1) through beta_a K (1 - sum phi)
      vec_copy(N1, lam->phi[i], c->alam + (long)i * N1, q);
      vec_axpby(N1, -p.beta[3], tmp, 1.0, c->alam + (long)i * N1, q);
    }
    vec_copy(N1, c->az, c->alw[3], q);
    dot<double>(N1, c->top, c->az, D + 0, kw.partial, q);
    chnss_status worst = CHNSS_OK;
    vec_fill(nv, 0.0, c->v_ch, q);
    for (int i = 0; i < 3; ++i) {
      vec_copy(N1, c->alam + (long)i * N1, c->arhs_ch, q);
      vec_copy(N1, lam->mu[i], c->arhs_ch + N1, q);
      {
        CH3OpT op(c, i);
        const chnss_status st = fgmres(op, c->arhs_ch, c->ay_ch, kAdjointRtol3, 0.0, p.maxit, kw, &inf[i], q);
        if (worst == CHNSS_OK) worst = st;
      }
      const double *y1 = c->ay_ch, *y2 = c->ay_ch + N1;
      double *aphi = c->aphi + (long)i * N1;
      const double cc = tau * p.gamma[i] / p.beta[i];
      spmv_csr<double>(F.p1, F.M1, 1, y1, aphi, SPMV_PLAIN, none, q);
      if (var) {   // - tau (d K_kappa(phi_i^k) / d phi_i)^T (y1, mu_i^(k+1))
        k3_adj_wstiff<<<nb3(E), kTPB3, 0, q>>>(F.geo, stk->phi[i], p.gamma[i], st1->mu[i], y1, bufP);
        CHNSS_LAUNCH_CK();
        launch_gather(c->gl, 1, bufP, -tau, aphi, 1.0, aphi, q);
      }
      vec_fill(N1, 0.0, c->alw[i], q);
      vec_axpby(N1, -cc, y2, 0.0, c->alw[i], q);
      k3_adj_conv_p1<<<nb3(E), kTPB3, 0, q>>>(F.geo, st1->phi[i], y1, bufV);
      CHNSS_LAUNCH_CK();
      launch_gather(c->gk, 3, bufV, -tau, c->v_ch, 1.0, c->v_ch, q);
      double *d = D + 4 + 5 * i;
      dot<double>(N1, c->loads + (long)i * N1, y2, d + 0, kw.partial, q);     // F_i . y2
      dot<double>(N1, c->top, y2, d + 1, kw.partial, q);                       // t . y2
      // y1 . K mu' (constant mobility) or y1 . K_kappa mu' (divided by gamma_i on the host)
      spmv_csr<double>(F.p1, var ? F.Kk[i] : F.K1, 1, st1->mu[i], tmp, SPMV_PLAIN, none, q);
      dot<double>(N1, y1, tmp, d + 2, kw.partial, q);
      spmv_csr<double>(F.p1, F.K1, 1, st1->phi[i], tmp, SPMV_PLAIN, none, q);
      dot<double>(N1, y2, tmp, d + 3, kw.partial, q);                          // y2 . K phi'
      spmv_csr<double>(F.p1, F.M1, 1, st1->mu[i], tmp, SPMV_PLAIN, none, q);
      dot<double>(N1, y2, tmp, d + 4, kw.partial, q);                          // y2 . M mu'
    }
    return worst;
  };
  chnss_status st[4] = {CHNSS_OK, CHNSS_OK, CHNSS_OK, CHNSS_OK};   // CH, AC, NS, air potential
  std::exception_ptr err[3];
  int dev = 0;
  CHNSS_CK(cudaGetDevice(&dev));
  auto run = [&](int w) {
    try {
      CHNSS_CK(cudaSetDevice(dev));
      cudaStream_t q = c->sx[w];
      CHNSS_CK(cudaStreamWaitEvent(q, c->ev_asm, 0));
      if (w == 0) st[0] = group_ch(q, &st[3]);
      else if (w == 1) st[1] = group_ac(q);
      else st[2] = group_ns(q);
      CHNSS_CK(cudaEventRecord(c->ev_done[w], q));
    } catch (...) {
      err[w] = std::current_exception();
    }
  };
  if (c->concurrent) {
    std::thread t_ac(run, 1), t_ns(run, 2);
    run(0);
    t_ac.join();
    t_ns.join();
  } else {
    for (int w = 0; w < 3; ++w) run(w);
  }
  for (std::exception_ptr &e : err)
    if (e) std::rethrow_exception(e);
  for (cudaEvent_t e : c->ev_done) CHNSS_CK(cudaStreamWaitEvent(s, e, 0));
  chnss_status worst = CHNSS_OK;
  for (chnss_status x : {st[2], st[3], st[1], st[0]})   // the order of the sequential adjoint: NS, mu_a, AC, CH
    if (worst == CHNSS_OK) worst = x;
  // ---- the groups' contributions to the shared adjoints --------------------------
  vec_axpby(nv, 1.0, c->v_ac, 1.0, out->v, s);
  vec_axpby(nv, 1.0, c->v_ch, 1.0, out->v, s);
  vec_axpby(N1, 1.0, c->aPhi, 1.0, out->Phi_v, s);
  for (int i = 0; i < 3; ++i) vec_axpby(N1, 1.0, c->aphi + (long)i * N1, 1.0, out->phi[i], s);
  // ---- potential loads ---------------------------------------------------------
  {
    double *bufP = c->ebuf;
    LoadWeights3 lw;
    for (int i = 0; i < 5; ++i) lw.z[i] = c->alw[i];
    k3_adj_loads<<<nb3(E), kTPB3, 0, s>>>(F.geo, fk, lw, bufP);
    CHNSS_LAUNCH_CK();
    for (int f = 0; f < 4; ++f) {
      double *dst = f < 3 ? out->phi[f] : out->Phi_v;
      launch_gather(c->gl, 1, bufP + 4 * f, 1.0, dst, 1.0, dst, s);
    }
  }
  // ---- parameter gradients and the evaporation flux ------------------------------
  double h[24], phis_ref = 0.0;
  CHNSS_CK(cudaMemcpyAsync(h, D, 24 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNSS_CK(cudaMemcpyAsync(&phis_ref, stk->phi[2] + c->ref, sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNSS_CK(cudaStreamSynchronize(s));
  const double j_out = p.evap_rate * (phis_ref - p.phi_s_inf);
  double jbar = p.beta[3] * h[0] + (p.ac_top_flux ? tau * p.delta_v * h[1] : 0.0);
  double gbar = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double *d = h + 4 + 5 * i;
    const double b_i = p.beta[i];
    const double cc = tau * p.gamma[i] / b_i;
    if (i == 2) jbar += cc * b_i * d[1];                                      // f_s = F_s - beta_s j t
    const double fy = d[0] - (i == 2 ? b_i * j_out * d[1] : 0.0);
    const double k2 = var ? d[2] / p.gamma[i] : d[2];   // tau K_kappa = gamma_i x (gamma-free matrix)
    gbar += -(tau / b_i) * fy - tau * k2 - (tau * d[3] - (tau / b_i) * d[4]);
  }
  k3_add_at<<<1, 1, 0, s>>>(out->phi[2], c->ref, jbar * p.evap_rate);
  CHNSS_LAUNCH_CK();
  k3_mask<<<nb3(nv), kTPB3, 0, s>>>(nv, c->bnd, out->v);
  CHNSS_LAUNCH_CK();
  CHNSS_CK(cudaStreamSynchronize(s));
  if (grad) {
    grad[0] += jbar * (phis_ref - p.phi_s_inf);
    grad[1] += gbar;
  }
  return worst;
}

}  // namespace
}  // namespace chnss

extern "C" chnss_status chnss3_ctx_create_ex(int n, int top_bc, const chnss_params *params, void *cuda_stream,
                                            chnss3_ctx_t *out) {
  using namespace chnss;
  chnss3_ctx *c = nullptr;
  try {
    if (!params || !out) throw Error{CHNSS_ERR_ARG, "null argument"};
    if (top_bc != 0 && top_bc != 1) throw Error{CHNSS_ERR_ARG, "top_bc must be 0 (no-slip) or 1 (open top)"};
    // the host setup counts element contributions in int: 6 n^3 x 900 for the
    // velocity pattern stays below 2^31 up to n = 72
    if (n < 2 || n % 2 || n > 64) throw Error{CHNSS_ERR_ARG, "3D meshes: n even, 2 <= n <= 64"};
    const chnss_params &p = *params;
    if (p.model != 0 || p.precision < 0 || p.precision > 2)
      throw Error{CHNSS_ERR_ARG, "the 3D step covers model 0, precision 0-2"};
    if (!(p.inner_rtol >= 0.0 && p.inner_rtol < 1.0)) throw Error{CHNSS_ERR_ARG, "inner_rtol must be in [0, 1)"};
    if (p.inner_rtol > 0.0 && (p.inner_maxit < 1 || p.inner_maxit > 1000))
      throw Error{CHNSS_ERR_ARG, "inner_maxit must be in [1, 1000]"};
    if (p.mobility_kind != 0 && p.mobility_kind != 1) throw Error{CHNSS_ERR_ARG, "mobility_kind must be 0 or 1"};
    if (p.ortho != 0 && p.ortho != 1) throw Error{CHNSS_ERR_ARG, "ortho must be 0 (FP64) or 1 (double-FP32)"};
    if (p.amg != 0) throw Error{CHNSS_ERR_ARG, "amg = 1 (smoothed aggregation of the AC block) is a 2D option"};
    if (!(p.tau > 0) || !(p.eta > 0) || p.restart < 1 || p.restart > 64 || p.maxit < 1)
      throw Error{CHNSS_ERR_ARG, "invalid parameters"};
    for (int i = 0; i < 3; ++i)
      if (!(p.beta[i] > 0) || !(p.gamma[i] > 0)) throw Error{CHNSS_ERR_ARG, "beta_i, gamma_i must be > 0"};
    c = new chnss3_ctx;
    c->p = p;
    c->top_bc = top_bc;
    if (cuda_stream) {
      c->s = static_cast<cudaStream_t>(cuda_stream);
    } else {
      CHNSS_CK(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    create3(c, n);
    *out = c;
    return CHNSS_OK;
  } catch (const Error &e) {
    delete c;
    set_global_error(e.msg);
    return e.status;
  } catch (const std::exception &e) {
    delete c;
    set_global_error(e.what());
    return CHNSS_ERR_ARG;
  }
}

extern "C" chnss_status chnss3_ctx_create(int n, const chnss_params *params, void *cuda_stream, chnss3_ctx_t *out) {
  return chnss3_ctx_create_ex(n, 0, params, cuda_stream, out);
}

extern "C" chnss_status chnss3_ctx_destroy(chnss3_ctx_t ctx) {
  delete ctx;
  return CHNSS_OK;
}

extern "C" chnss_status chnss3_sizes(chnss3_ctx_t ctx, int *N1, int *N2) {
  if (!ctx || !N1 || !N2) {
    chnss::set_global_error("null argument");
    return CHNSS_ERR_ARG;
  }
  *N1 = (int)ctx->lv[0].N1;
  *N2 = (int)ctx->lv[0].N2;
  return CHNSS_OK;
}

extern "C" chnss_status chnss3_step(chnss3_ctx_t ctx, const chnss_state *in, chnss_state *out,
                                   chnss_solve_info *info) {
  using namespace chnss;
  if (!ctx) {
    set_global_error("null context");
    return CHNSS_ERR_ARG;
  }
  try {
    const chnss_state *states[2] = {in, out};
    for (const chnss_state *st : states) {
      if (!st || !st->Phi_v || !st->v || !st->p) throw Error{CHNSS_ERR_ARG, "null state"};
      for (int k = 0; k < 3; ++k) if (!st->phi[k]) throw Error{CHNSS_ERR_ARG, "null phi pointer"};
      for (int k = 0; k < 4; ++k) if (!st->mu[k]) throw Error{CHNSS_ERR_ARG, "null mu pointer"};
    }
    chnss_solve_info loc[6];
    const chnss_status st = step3(ctx, in, out, info ? info : loc);
    if (st != CHNSS_OK) ctx->err = "a solve of the 3D step did not converge cleanly";
    return st;
  } catch (const Error &e) {
    ctx->err = e.msg;
    return e.status;
  }
}

extern "C" chnss_status chnss3_adjoint_step(chnss3_ctx_t ctx, const chnss_state *state_k,
                                            const chnss_state *state_k1, const chnss_state *adj_k1,
                                            chnss_state *adj_k, double *grad_params, chnss_solve_info *info) {
  using namespace chnss;
  if (!ctx) {
    set_global_error("null context");
    return CHNSS_ERR_ARG;
  }
  try {
    const chnss_state *states[4] = {state_k, state_k1, adj_k1, adj_k};
    for (const chnss_state *st : states) {
      if (!st || !st->Phi_v || !st->v || !st->p) throw Error{CHNSS_ERR_ARG, "null state"};
      for (int k = 0; k < 3; ++k) if (!st->phi[k]) throw Error{CHNSS_ERR_ARG, "null phi pointer"};
      for (int k = 0; k < 4; ++k) if (!st->mu[k]) throw Error{CHNSS_ERR_ARG, "null mu pointer"};
    }
    chnss_solve_info loc[6];
    const chnss_status st = adjoint_step3(ctx, state_k, state_k1, adj_k1, adj_k, grad_params, info ? info : loc);
    if (st != CHNSS_OK) ctx->err = "a transposed solve of the 3D adjoint step did not converge cleanly";
    return st;
  } catch (const Error &e) {
    ctx->err = e.msg;
    return e.status;
  }
}

extern "C" chnss_status chnss3_objective(chnss3_ctx_t ctx, const double *phi_p, double *J, double *grad_phi_p) {
  using namespace chnss;
  if (!ctx) {
    set_global_error("null context");
    return CHNSS_ERR_ARG;
  }
  try {
    if (!phi_p || !J) throw Error{CHNSS_ERR_ARG, "null phi_p or J"};
    adjoint_alloc3(ctx);
    const Level3 &F = ctx->lv[0];
    const long N1 = F.N1;
    SpmvArgs none;
    spmv_csr<double>(F.p1, F.K1, 1, phi_p, ctx->atmp, SPMV_PLAIN, none, ctx->s);
    dot<double>(N1, phi_p, ctx->atmp, ctx->adots + 30, ctx->partial, ctx->s);
    if (grad_phi_p) {
      vec_fill(N1, 0.0, grad_phi_p, ctx->s);
      vec_axpby(N1, 2.0, ctx->atmp, 0.0, grad_phi_p, ctx->s);
    }
    CHNSS_CK(cudaMemcpyAsync(J, ctx->adots + 30, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CHNSS_CK(cudaStreamSynchronize(ctx->s));
    return CHNSS_OK;
  } catch (const Error &e) {
    ctx->err = e.msg;
    return e.status;
  }
}

extern "C" chnss_status chnss3_set_step_concurrency(chnss3_ctx_t ctx, int on) {
  if (!ctx) {
    chnss::set_global_error("null context");
    return CHNSS_ERR_ARG;
  }
  ctx->concurrent = on != 0;
  return CHNSS_OK;
}

extern "C" const char *chnss3_last_error(chnss3_ctx_t ctx) { return ctx ? ctx->err.c_str() : ""; }
