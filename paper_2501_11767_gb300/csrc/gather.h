// Host construction of CSR patterns and gather lists from element node
// lists (shared by the 2D and the 3D setup).
#pragma once

#include <algorithm>
#include <climits>
#include <vector>

#include "internal.h"

namespace chnss {

template <class PairFn>
inline void pattern_from_elements(int nrows, int ncols, int E, int nr, int nc, PairFn nodes, Pattern &P) {
  // the candidate counts below are int: refuse sizes whose total would overflow
  if ((long long)E * nr * nc > INT_MAX) throw Error{CHNSS_ERR_ARG, "mesh too large for int32 pattern counts"};
  std::vector<int> cnt(nrows + 1, 0);
  std::vector<int> rn(nr), cn(nc);
  for (int e = 0; e < E; ++e) {
    nodes(e, rn.data(), cn.data());
    for (int a = 0; a < nr; ++a) cnt[rn[a] + 1] += nc;
  }
  for (int r = 0; r < nrows; ++r) cnt[r + 1] += cnt[r];
  std::vector<int> cand(cnt[nrows]);
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int e = 0; e < E; ++e) {
    nodes(e, rn.data(), cn.data());
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b) cand[fill[rn[a]]++] = cn[b];
  }
  P.nrows = nrows;
  P.ncols = ncols;
  P.h_rowptr.assign(nrows + 1, 0);
  P.h_col.clear();
  P.h_col.reserve(cand.size() / 3);
  for (int r = 0; r < nrows; ++r) {
    int *b = cand.data() + cnt[r], *e = cand.data() + cnt[r + 1];
    std::sort(b, e);
    int *u = std::unique(b, e);
    P.h_col.insert(P.h_col.end(), b, u);
    P.h_rowptr[r + 1] = (int)P.h_col.size();
  }
  P.nnz = (int)P.h_col.size();
}

inline int find_col(const Pattern &P, int row, int col) {
  const int *b = P.h_col.data() + P.h_rowptr[row], *e = P.h_col.data() + P.h_rowptr[row + 1];
  const int *it = std::lower_bound(b, e, col);
  return (int)(it - P.h_col.data());
}

// Gather list: contribution j of element e, local (a, b) -> entry (row, col),
// element-buffer offset off(e, a, b); keep(e, a, b) masks entries out.
template <class PairFn, class OffFn, class KeepFn>
inline void gather_from_elements(const Pattern &P, int E, int nr, int nc, PairFn nodes, OffFn off, KeepFn keep,
                          Gather &G, std::vector<int> &hptr, std::vector<int> &hidx) {
  if ((long long)E * nr * nc > INT_MAX) throw Error{CHNSS_ERR_ARG, "mesh too large for int32 gather lists"};
  hptr.assign(P.nnz + 1, 0);
  std::vector<int> rn(nr), cn(nc);
  for (int e = 0; e < E; ++e) {
    nodes(e, rn.data(), cn.data());
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b)
        if (keep(e, a, b, rn[a], cn[b])) hptr[find_col(P, rn[a], cn[b]) + 1]++;
  }
  for (int k = 0; k < P.nnz; ++k) hptr[k + 1] += hptr[k];
  hidx.assign(hptr[P.nnz], 0);
  std::vector<int> fill(hptr.begin(), hptr.end() - 1);
  for (int e = 0; e < E; ++e) {   // element order: fixed summation order
    nodes(e, rn.data(), cn.data());
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b)
        if (keep(e, a, b, rn[a], cn[b])) hidx[fill[find_col(P, rn[a], cn[b])]++] = off(e, a, b);
  }
  G.nout = P.nnz;
  G.ncontrib = (int)hidx.size();
}

// node <- (element, local) gather for load vectors
template <class NodeFn, class OffFn, class KeepFn>
inline void node_gather(int nnodes, int E, int nl, NodeFn nodes, OffFn off, KeepFn keep, std::vector<int> &hptr,
                 std::vector<int> &hidx, Gather &G) {
  hptr.assign(nnodes + 1, 0);
  std::vector<int> nd(nl);
  for (int e = 0; e < E; ++e) {
    nodes(e, nd.data());
    for (int a = 0; a < nl; ++a)
      if (keep(nd[a])) hptr[nd[a] + 1]++;
  }
  for (int k = 0; k < nnodes; ++k) hptr[k + 1] += hptr[k];
  hidx.assign(hptr[nnodes], 0);
  std::vector<int> fill(hptr.begin(), hptr.end() - 1);
  for (int e = 0; e < E; ++e) {
    nodes(e, nd.data());
    for (int a = 0; a < nl; ++a)
      if (keep(nd[a])) hidx[fill[nd[a]]++] = off(e, a);
  }
  G.nout = nnodes;
  G.ncontrib = (int)hidx.size();
}

}  // namespace chnss
