// Host setup of the tetrahedral (3D) discretisation: Kuhn meshes of a box,
// the exact reference integrals of the P1 / P2 element operators
// (three_d.h), host assembly of the element operators into CSR in element
// order, and the nested P1 / P2 transfers.  The 3D operators are exported
// through chnss3_host_operator for checks against a reference; the element
// operators are __host__ __device__ so that the device kernels of the 3D
// step use the same code.
#include <algorithm>
#include <array>
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
  bool p2_boundary(int id) const {
    const int m = 2 * n + 1, A = id % m, B = (id / m) % m, C = id / (m * m);
    return A == 0 || B == 0 || C == 0 || A == m - 1 || B == m - 1 || C == m - 1;
  }
};

Mesh3Host make_mesh3(int n, const double L[3]) {
  Mesh3Host M;
  M.n = n;
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
  OP3_LOADS, OP3_KORTEWEG, OP3_TOP, OP3_COUNT
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
    case OP3_VPROL: {
      if (n % 2) throw Error{CHNSS_ERR_ARG, "transfers need an even n (coarse mesh n / 2)"};
      const Mesh3Host C = make_mesh3(n / 2, L);
      return which == OP3_P1PROL ? p1_prolongation3(C) : velocity_prolongation3(C, M);
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
