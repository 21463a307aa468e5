// Multigrid V-cycle and Krylov drivers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>

#include "solver.h"

namespace chnss {


const char *Profiler::name(int k) {
  static const char *names[NKINDS] = {"mg_velocity_spmv_fine", "mg_p1_spmv_fine", "ns_operator_spmv",
                                      "krylov_orthogonalisation", "assembly", "mg_p1_coarse_levels",
                                      "mg_velocity_coarse_levels"};
  return k >= 0 && k < NKINDS ? names[k] : "?";
}

int Profiler::start(int k, cudaStream_t s) {
  if (sink) {
    if (sink_used >= sink->size()) return -1;
    Probe &p = (*sink)[sink_used];
    p.kind = k;
    p.bytes = 0.0;
    // during capture only an external record becomes an event node
    CHNSS_CK(cudaEventRecordWithFlags(p.e0, s, cudaEventRecordExternal));
    return (int)sink_used++;
  }
  if (!on) return -1;
  std::lock_guard<std::mutex> lock(mu);
  Rec &r = rec[k];
  if (r.used + 2 > r.ev.size()) {
    if (r.ev.size() >= 16384) return -1;   // pool full: later launches are counted, not timed
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      CHNSS_CK(cudaEventCreate(&e));
      r.ev.push_back(e);
    }
  }
  const int tok = (int)r.used;
  r.used += 2;
  CHNSS_CK(cudaEventRecord(r.ev[tok], s));
  return tok;
}

void Profiler::stop(int k, int token, cudaStream_t s, double bytes, double flops, int count) {
  if (sink) {
    if (token < 0) return;
    Probe &p = (*sink)[token];
    p.bytes = bytes;
    CHNSS_CK(cudaEventRecordWithFlags(p.e1, s, cudaEventRecordExternal));
    return;
  }
  if (!on) return;
  std::lock_guard<std::mutex> lock(mu);
  Rec &r = rec[k];
  if (token < 0) return;   // not timed (pool full, or profiling switched on mid-interval)
  CHNSS_CK(cudaEventRecord(r.ev[token + 1], s));
  r.launches += count;
  r.bytes += bytes;
  r.flops += flops;
}

void Profiler::harvest(const std::vector<Probe> &probes, size_t count) {
  if (!on) return;
  std::lock_guard<std::mutex> lock(mu);
  for (size_t i = 0; i < count && i < probes.size(); ++i) {
    const Probe &p = probes[i];
    float t = 0.f;
    CHNSS_CK(cudaEventElapsedTime(&t, p.e0, p.e1));
    Rec &r = rec[p.kind];
    r.ms_graph += t;
    r.launches += 1;
    r.bytes += p.bytes;
  }
}

void Profiler::reset() {
  for (Rec &r : rec) {
    r.launches = 0;
    r.bytes = 0.0;
    r.flops = 0.0;
    r.ms_graph = 0.0;
    r.used = 0;
  }
}

double Profiler::elapsed_ms(int k) {
  Rec &r = rec[k];
  double ms = r.ms_graph;
  for (size_t i = 0; i + 1 < r.used; i += 2) {
    float t = 0.f;
    CHNSS_CK(cudaEventElapsedTime(&t, r.ev[i], r.ev[i + 1]));
    ms += t;
  }
  return ms;
}

void Profiler::release() {
  for (Rec &r : rec) {
    for (cudaEvent_t e : r.ev) cudaEventDestroy(e);
    r.ev.clear();
    r.used = 0;
  }
}

namespace {
// algorithmic bytes of one SpMV launch: values + column indices + row
// pointers + one read of u, one write of out, plus the extra vector streams
// of the epilogue (b for RES, b + dinv (+ w) for CHEB, out read for ADD)
// Algorithmic bytes of one sweep: every stored nonzero once (value, plus a
// 4-byte column and the row pointers unless the stencil layout implies
// them), the input and output vectors once, and the epilogue's vectors.
double spmv_bytes(long nrows, long nnz, int vals_per_entry, long vec_len, size_t sv, size_t s, SpmvMode mode,
                  bool has_w, bool implicit_index) {
  double extra = 0.0;
  if (mode == SPMV_RES) extra = 1.0;
  if (mode == SPMV_ADD) extra = 1.0;
  if (mode == SPMV_CHEB) extra = has_w ? 3.0 : 2.0;
  const double index = implicit_index ? 0.0 : (double)nnz * 4.0 + 4.0 * (nrows + 1);
  return (double)nnz * vals_per_entry * (double)sv + index + (2.0 + extra) * vec_len * s;
}
}  // namespace

template <typename T>
void MGHier<T>::init(Arena &ar, int kind_, bool singular_, const std::vector<const Pattern *> &pats,
                     const std::vector<const int *> &diags, const std::vector<const double *> &vals,
                     const std::vector<const Transfer *> &trs, double *partial_buf) {
  diag = diags;
  kind = kind_;
  singular = singular_;
  nl = (int)pats.size();
  pat = pats;
  val64 = vals;
  tr = trs;
  if (bf16 && !std::is_same<T, float>::value) throw Error{CHNSS_ERR_ARG, "BF16 values need FP32 vectors"};
  if (kind == 2 && ((int)bpat.size() != nl || (int)bmap.size() != nl))
    throw Error{CHNSS_ERR_ARG, "3x3-block levels need a node pattern and value map per level"};
  n.resize(nl);
  val.resize(nl);
  val16.assign(nl, nullptr);
  dinv.resize(nl);
  x.resize(nl);
  t.resize(nl);
  r.resize(nl);
  b.resize(nl);
  hi.resize(nl);
  coef.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const long nu = (kind == 1 ? 2L : 1L) * pat[l]->nrows;
    n[l] = nu;
    const long nv = sell_values(l);   // SELL order
    if (bf16) {
      val[l] = nullptr;
      val16[l] = ar.alloc<__nv_bfloat16>(nv);
    } else {
      val[l] = ar.alloc<T>(nv);
    }
    dinv[l] = ar.alloc<T>(nu);
    x[l] = ar.alloc<T>(nu);
    t[l] = ar.alloc<T>(nu);
    r[l] = ar.alloc<T>(nu);
    b[l] = ar.alloc<T>(nu);
    hi[l] = ar.alloc<double>(1);
    coef[l] = ar.alloc<double>(4 + 3 * (kMaxSmoothDegree - 1));
  }
  nc = (int)n[nl - 1];
  coarse_iter = nl > 1 && !singular && !keep_dense && nc > kCoarseDenseMax;
  if (!coarse_iter) {
    dense = ar.alloc<double>((long)nc * nc);
    cinv = ar.alloc<double>((long)nc * nc);
  }
  status = ar.alloc<int>(1);
  partial = partial_buf;
  sum = ar.alloc<double>(1);
  if (kind == 0 && !bf16) {
    for (int l = 1; l < nl; ++l)
      if (n[l] <= kTailRows) {
        tail_l0 = l;
        break;
      }
    // the one-block tail sweeps rows of at most 16 entries (sell_w8m_slice;
    // 8 on the triangle meshes, 15 on the tetrahedral P1 levels)
    int wmax = 0;
    for (int l = std::max(tail_l0, 0); l < nl; ++l) {
      wmax = std::max(wmax, pat[l]->sell.wmax);
      if (l < nl - 1) wmax = std::max({wmax, tr[l]->R.sell.wmax, tr[l]->P.sell.wmax});
    }
    tail_width = wmax <= 8 ? 8 : 16;
    if (tail_l0 > 0 && nl - tail_l0 <= kMaxTailLevels && wmax <= 16) {
      std::vector<MultiPtr<T>> X(nl), Tt(nl), Rr(nl), B(nl);
      for (int l = 0; l < nl; ++l) {
        X[l].p[0] = x[l];
        Tt[l].p[0] = t[l];
        Rr[l].p[0] = r[l];
        B[l].p[0] = b[l];
      }
      tail = make_tail(ar, X, Tt, Rr, B);
    } else {
      tail_l0 = -1;
    }
  }
}

template <typename T>
static inline const T *transfer_vals(const Transfer &t, bool restrict_);

template <typename T>
TailDesc<T> *MGHier<T>::make_tail(Arena &ar, const std::vector<MultiPtr<T>> &X, const std::vector<MultiPtr<T>> &Tt,
                                  const std::vector<MultiPtr<T>> &Rr, const std::vector<MultiPtr<T>> &B) const {
  TailDesc<T> d;
  d.nlev = nl - tail_l0;
  d.degree = degree;
  d.nc = nc;
  d.cinv = cinv;
  d.coarse_degree = coarse_iter ? kCoarseDegree : 0;
  auto view = [](const Pattern &P) {
    if (P.sell.wmax > 16) throw Error{CHNSS_ERR_ARG, "coarse-level block: rows of at most 16 entries"};
    TailSell v;
    v.nslices = P.sell.nslices;
    v.sp = P.sell.slice_ptr;
    v.rowid = P.sell.rowid;
    v.col = P.sell.col;
    return v;
  };
  for (int l = tail_l0; l < nl; ++l) {
    TailLevel<T> &q = d.lv[l - tail_l0];
    q.n = (int)n[l];
    q.A = view(*pat[l]);
    q.val = val[l];
    q.dinv = dinv[l];
    q.coef = coef[l];
    q.x = X[l];
    q.t = Tt[l];
    q.r = Rr[l];
    q.b = B[l];
    if (l < nl - 1) {
      q.R = view(tr[l]->R);
      q.P = view(tr[l]->P);
      q.Rval = transfer_vals<T>(*tr[l], true);
      q.Pval = transfer_vals<T>(*tr[l], false);
    }
  }
  TailDesc<T> *dd = ar.alloc<TailDesc<T>>(1);
  CHNSS_CK(cudaMemcpy(dd, &d, sizeof(d), cudaMemcpyHostToDevice));
  return dd;
}

template <typename T>
long MGHier<T>::sell_values(int l) const {
  if (kind == 2) return 9L * bpat[l]->sell.nent;
  return (kind == 0 ? 1L : 4L) * pat[l]->sell.nent;
}

template <typename T>
template <typename VT>
void MGHier<T>::gather_values(int l, VT *out, cudaStream_t s) const {
  if (kind == 2) sell_gather9<VT>(bpat[l]->sell.nent, bmap[l], val64[l], out, s);
  else sell_gather<VT>(pat[l]->sell, kind == 0 ? 1 : 4, val64[l], out, s);
}

template <typename T>
void MGHier<T>::setup(cudaStream_t s) {
  for (int l = 0; l < nl; ++l) {
    if (bf16) gather_values<__nv_bfloat16>(l, val16[l], s);
    else gather_values<T>(l, val[l], s);
    if (l == 0 && val0_64) gather_values<double>(0, val0_64, s);
    if (l == nl - 1 && !coarse_iter) break;
    if (kind == 1)
      jacobi_bsr2<T>(*pat[l], val64[l], diag[l], dinv[l], hi[l], partial, s);
    else
      jacobi_csr<T>(*pat[l], val64[l], diag[l], dinv[l], hi[l], partial, s);
    if (!hi_ext.empty())
      CHNSS_CK(cudaMemcpyAsync(hi[l], hi_ext[l], sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (l == nl - 1)
      cheb_coefficients(hi[l], kCoarseRatio, kCoarseDegree, coef[l], s);
    else
      cheb_coefficients(hi[l], ratio, degree, coef[l], s);
  }
  if (coarse_iter) return;
  const int L = nl - 1;
  if (kind == 1)
    coarse_dense_bsr2(*pat[L], val64[L], dense, s);
  else
    coarse_dense_csr(*pat[L], val64[L], singular ? 1.0 : 0.0, dense, s);
  dense_invert(nc, dense, cinv, status, s);
}

template <typename T>
void MGHier<T>::op(int l, const T *u, T *out, SpmvMode mode, const SpmvArgs &a, cudaStream_t s) {
  const int k = kind == 0 ? Profiler::P1_SPMV_L0 : Profiler::VEL_SPMV_L0;
  const bool timed = prof && l == 0;
  const int tk = timed ? prof->start(k, s) : -1;
  spmv_level(l, u, out, mode, a, s);
  if (timed)
    prof->stop(k, tk, s,
               kind == 2 ? spmv_bytes(bpat[l]->nrows, bpat[l]->nnz, 9, n[l], bf16 ? 2 : sizeof(T), sizeof(T), mode,
                                      a.w != nullptr, false)
                         : spmv_bytes(pat[l]->nrows, pat[l]->nnz, kind == 0 ? 1 : 4, n[l], bf16 ? 2 : sizeof(T),
                                      sizeof(T), mode, a.w != nullptr, pat[l]->sell.stencil != 0));
}

template <typename T>
void MGHier<T>::spmv_level(int l, const T *u, T *out, SpmvMode mode, const SpmvArgs &a, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (bf16) {
      if (kind == 0) spmv_sell(*pat[l], val16[l], 1, u, out, mode, a, s);
      else if (kind == 1) spmv_sell_bsr2(*pat[l], val16[l], u, out, mode, a, s);
      else spmv_sell_bsr3(*bpat[l], val16[l], u, out, mode, a, s);
      return;
    }
  }
  if (kind == 0)
    spmv_sell<T>(*pat[l], val[l], 1, u, out, mode, a, s);
  else if (kind == 1)
    spmv_sell_bsr2<T>(*pat[l], val[l], u, out, mode, a, s);
  else
    spmv_sell_bsr3<T>(*bpat[l], val[l], u, out, mode, a, s);
}

template <typename T>
static inline const T *transfer_vals(const Transfer &t, bool restrict_) {
  if (std::is_same<T, double>::value) return reinterpret_cast<const T *>(restrict_ ? t.Rs : t.Ps);
  return reinterpret_cast<const T *>(restrict_ ? t.Rs32 : t.Ps32);
}

template <typename T>
void MGHier<T>::vcycle(int l, cudaStream_t s) {
  if (l == tail_l0) {
    mg_tail<T>(tail, 1, tail_width, s);
    return;
  }
  if (l == nl - 1 && !coarse_iter) {
    dense_apply<T>(nc, cinv, b[l], x[l], s);
    return;
  }
  if (l == nl - 1 && kind == 2 && bpat[l]->sell.nslices <= kChebBlockSlices) {
    // small 3x3-block coarsest level: its Chebyshev steps in one launch
    if constexpr (std::is_same<T, float>::value) {
      if (bf16) {
        cheb_block_bsr3<float, __nv_bfloat16>(*bpat[l], val16[l], dinv[l], b[l], x[l], t[l], coef[l], kCoarseDegree, s);
        return;
      }
    }
    cheb_block_bsr3<T, T>(*bpat[l], val[l], dinv[l], b[l], x[l], t[l], coef[l], kCoarseDegree, s);
    return;
  }
  const int nc_ = kind == 1 ? 2 : 1;   // transfers per node (BSR2) or per dof
  SpmvArgs a;
  a.b = b[l];
  a.dinv = dinv[l];
  // pre-smoothing from x = 0 (on the coarsest level of an iterative coarse
  // solve: kCoarseDegree steps): x_1 = D^-1 b / theta, then deg - 1 steps of
  // the three-term recurrence; x_{k+1} overwrites x_{k-1}, so x_1 starts in
  // the buffer that makes x_deg land in x[l]
  const int deg = l == nl - 1 ? kCoarseDegree : degree;
  T *cur = (deg - 1) % 2 == 0 ? x[l] : t[l];
  T *oth = cur == x[l] ? t[l] : x[l];
  vec_scale_dinv<T>((int)n[l], coef[l], dinv[l], b[l], cur, s);
  for (int k = 1; k < deg; ++k) {
    a.coef = coef[l] + 4 + 3 * (k - 1);
    a.w = k == 1 ? nullptr : oth;
    op(l, cur, oth, SPMV_CHEB, a, s);
    std::swap(cur, oth);
  }
  if (l == nl - 1) return;
  // residual, restriction, coarse correction, prolongation
  SpmvArgs ar;
  ar.b = b[l];
  op(l, x[l], r[l], SPMV_RES, ar, s);
  const Transfer &T_ = *tr[l];
  SpmvArgs none;
  spmv_sell<T>(T_.R, transfer_vals<T>(T_, true), nc_, r[l], b[l + 1], SPMV_PLAIN, none, s);
  const int kc = kind == 0 ? Profiler::P1_MG_COARSE : Profiler::VEL_MG_COARSE;
  const int tkc = prof && l == 0 ? prof->start(kc, s) : -1;
  vcycle(l + 1, s);
  if (prof && l == 0) prof->stop(kc, tkc, s, 0.0);   // time only: every level below the finest
  spmv_sell<T>(T_.P, transfer_vals<T>(T_, false), nc_, x[l + 1], x[l], SPMV_ADD, none, s);
  // post-smoothing from x_0 = x[l]
  a.coef = coef[l] + 1;
  a.w = nullptr;
  op(l, x[l], t[l], SPMV_CHEB, a, s);
  cur = t[l];
  oth = x[l];
  for (int k = 1; k < degree; ++k) {
    a.coef = coef[l] + 4 + 3 * (k - 1);
    a.w = oth;
    op(l, cur, oth, SPMV_CHEB, a, s);
    std::swap(cur, oth);
  }
  if (cur != x[l]) vec_convert<T, T>(n[l], cur, x[l], s);
}

template <typename T>
void MGHier<T>::cycle(cudaStream_t s) {
  double *pb = ipartial ? ipartial : partial;
  if (singular) {
    vsum<T>(n[0], b[0], sum, pb, s);
    vec_sub_mean<T>((int)n[0], b[0], sum, s);
  }
  vcycle(0, s);
  if (singular) {
    vsum<T>(n[0], x[0], sum, pb, s);
    vec_sub_mean<T>((int)n[0], x[0], sum, s);
  }
}

template <typename T>
void MGHier<T>::apply(cudaStream_t s) {
  if (inner_rtol > 0.0) solve(s);
  else cycle(s);
}

namespace {

constexpr int kAccTPB = 256;

template <typename T>
__global__ void k_acc(long n, const T *x, double *y) {
  const long i = (long)blockIdx.x * kAccTPB + threadIdx.x;
  if (i < n) y[i] += (double)x[i];
}

// continue while ||r||^2 > rtol^2 ||b||^2 (and finite) and fewer than maxit
// V-cycles have run; first = 1 after the first V-cycle (sets the count)
__global__ void k_inner_check(cudaGraphConditionalHandle h, double *ctl, int *it, double rtol2, int maxit,
                              int first) {
  const int k = first ? 1 : *it + 1;
  *it = k;
  ctl[2] = (double)k;
  const double nr2 = ctl[1];
  const bool more = isfinite(nr2) && nr2 > rtol2 * ctl[0] && k < maxit;
  if (!more) {
    ctl[3] += (double)k;
    ctl[4] += 1.0;
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_inner_tally(double *ctl, int k) {
  ctl[2] = (double)k;
  ctl[3] += (double)k;
  ctl[4] += 1.0;
}

}  // namespace

template <typename T>
void MGHier<T>::enable_inner(Arena &ar, double rtol, int maxit, cudaStream_t body_stream) {
  if (!(rtol > 0.0)) return;
  inner_rtol = rtol;
  inner_maxit = maxit;
  bodyq = body_stream;
  bsave = ar.alloc<double>(n[0]);
  acc = ar.alloc<double>(n[0]);
  if (!std::is_same<T, double>::value) {
    r64 = ar.alloc<double>(n[0]);
    val0_64 = ar.alloc<double>(sell_values(0));
  }
  ictl = ar.alloc<double>(8);
  iit = ar.alloc<int>(1);
  ipartial = ar.alloc<double>(64L * kReduceMaxBlocks);
  CHNSS_CK(cudaMemset(ictl, 0, 8 * sizeof(double)));
  CHNSS_CK(cudaMemset(iit, 0, sizeof(int)));
}

template <typename T>
void MGHier<T>::write_output(double *const *slot, long off, cudaStream_t s) {
  if (inner_rtol > 0.0) vec_convert_to_slot<double, double>(n[0], acc, slot, off, s);
  else vec_convert_to_slot<T, double>(n[0], x[0], slot, off, s);
}

template <typename T>
void MGHier<T>::inner_stats(bool reset, long long *solves, long long *cycles, double *last_rel, cudaStream_t s) {
  *solves = 0;
  *cycles = 0;
  *last_rel = 0.0;
  if (!ictl) return;
  double h[5];
  CHNSS_CK(cudaMemcpyAsync(h, ictl, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNSS_CK(cudaStreamSynchronize(s));
  *solves = (long long)h[4];
  *cycles = (long long)h[3];
  *last_rel = h[0] > 0.0 ? std::sqrt(h[1] / h[0]) : 0.0;
  if (reset) {
    CHNSS_CK(cudaMemsetAsync(ictl + 3, 0, 2 * sizeof(double), s));
    CHNSS_CK(cudaStreamSynchronize(s));
  }
}

template <typename T>
void MGHier<T>::inner_residual(cudaStream_t s) {
  SpmvArgs a;
  a.b = bsave;
  if constexpr (std::is_same<T, double>::value) {
    op(0, acc, b[0], SPMV_RES, a, s);
    dot<double>(n[0], b[0], b[0], ictl + 1, ipartial, s);
  } else {
    if (kind == 0) spmv_sell<double>(*pat[0], val0_64, 1, acc, r64, SPMV_RES, a, s);
    else if (kind == 1) spmv_sell_bsr2<double>(*pat[0], val0_64, acc, r64, SPMV_RES, a, s);
    else spmv_sell_bsr3<double>(*bpat[0], val0_64, acc, r64, SPMV_RES, a, s);
    dot<double>(n[0], r64, r64, ictl + 1, ipartial, s);
    vec_convert<double, T>(n[0], r64, b[0], s);
  }
}

template <typename T>
void MGHier<T>::solve(cudaStream_t s) {
  const long n0 = n[0];
  if (singular) {
    vsum<T>(n0, b[0], sum, ipartial, s);
    vec_sub_mean<T>((int)n0, b[0], sum, s);
  }
  vec_convert<T, double>(n0, b[0], bsave, s);
  dot<double>(n0, bsave, bsave, ictl, ipartial, s);
  cycle(s);
  vec_convert<T, double>(n0, x[0], acc, s);
  inner_residual(s);
  const double rtol2 = inner_rtol * inner_rtol;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CHNSS_CK(cudaStreamIsCapturing(s, &cs));
  if (cs == cudaStreamCaptureStatusActive) {
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t nd = 0;
    CHNSS_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    CHNSS_CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    k_inner_check<<<1, 1, 0, s>>>(h, ictl, iit, rtol2, inner_maxit, 1);
    CHNSS_LAUNCH_CK();
    CHNSS_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edata, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    CHNSS_CK(cudaGraphAddNode(&node, g, deps, edata, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CHNSS_CK(cudaStreamBeginCaptureToGraph(bodyq, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    Profiler *pf = prof;
    prof = nullptr;   // event-record nodes are not allowed in a conditional body
    try {
      cycle(bodyq);
      k_acc<T><<<(unsigned)((n0 + kAccTPB - 1) / kAccTPB), kAccTPB, 0, bodyq>>>(n0, x[0], acc);
      CHNSS_LAUNCH_CK();
      inner_residual(bodyq);
      k_inner_check<<<1, 1, 0, bodyq>>>(h, ictl, iit, rtol2, inner_maxit, 0);
      CHNSS_LAUNCH_CK();
    } catch (...) {
      prof = pf;
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(bodyq, &tmp);
      throw;
    }
    prof = pf;
    cudaGraph_t tmp = nullptr;
    CHNSS_CK(cudaStreamEndCapture(bodyq, &tmp));
    CHNSS_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  } else {
    double h2[2];
    int k = 1;
    for (;;) {
      CHNSS_CK(cudaMemcpyAsync(h2, ictl, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CHNSS_CK(cudaStreamSynchronize(s));
      if (!(std::isfinite(h2[1]) && h2[1] > rtol2 * h2[0] && k < inner_maxit)) break;
      cycle(s);
      k_acc<T><<<(unsigned)((n0 + kAccTPB - 1) / kAccTPB), kAccTPB, 0, s>>>(n0, x[0], acc);
      CHNSS_LAUNCH_CK();
      inner_residual(s);
      ++k;
    }
    k_inner_tally<<<1, 1, 0, s>>>(ictl, k);
    CHNSS_LAUNCH_CK();
  }
  vec_convert<double, T>(n0, acc, x[0], s);
}

template struct MGHier<double>;
template struct MGHier<float>;

// ---------------------------------------------------------------------------
template <typename T>
void MGBatch<T>::init(Arena &ar, MGHier<T> *hier, int nr_) {
  if (hier->kind != 0 || hier->singular || hier->bf16)
    throw Error{CHNSS_ERR_ARG, "batched V-cycle: scalar, non-singular, non-BF16 hierarchies only"};
  if (nr_ < 1 || nr_ > kMaxRhs) throw Error{CHNSS_ERR_ARG, "batched V-cycle: 1 to 3 vectors"};
  h = hier;
  nr = nr_;
  const int nl = h->nl;
  x.assign(nl, MultiPtr<T>());
  t.assign(nl, MultiPtr<T>());
  r.assign(nl, MultiPtr<T>());
  b.assign(nl, MultiPtr<T>());
  for (int l = 0; l < nl; ++l)
    for (int k = 0; k < nr; ++k) {
      x[l].p[k] = ar.alloc<T>(h->n[l]);
      t[l].p[k] = ar.alloc<T>(h->n[l]);
      r[l].p[k] = ar.alloc<T>(h->n[l]);
      b[l].p[k] = ar.alloc<T>(h->n[l]);
    }
  if (h->tail_l0 > 0) tail = h->make_tail(ar, x, t, r, b);
}

template <typename T>
void MGBatch<T>::op(int l, const MultiPtr<T> &u, const MultiPtr<T> &out, SpmvMode mode, const MultiArgs<T> &a,
                    cudaStream_t s) {
  Profiler *prof = h->prof;
  const bool timed = prof && l == 0;
  const int tk = timed ? prof->start(Profiler::P1_SPMV_L0, s) : -1;
  spmv_sell_multi<T>(*h->pat[l], h->val[l], nr, u, out, mode, a, s);
  if (timed) {
    // one matrix stream for nr vectors
    const long nnz = h->pat[l]->nnz, nrows = h->pat[l]->nrows;
    double extra = 0.0;
    if (mode == SPMV_RES || mode == SPMV_ADD) extra = 1.0;
    if (mode == SPMV_CHEB) extra = a.w.p[0] ? 3.0 : 2.0;
    const double bytes = (double)nnz * (sizeof(T) + 4.0) + 4.0 * (nrows + 1) +
                         (double)nr * (2.0 + extra) * h->n[l] * sizeof(T) + (mode == SPMV_CHEB ? h->n[l] * sizeof(T) : 0.0);
    prof->stop(Profiler::P1_SPMV_L0, tk, s, bytes);
  }
}

template <typename T>
void MGBatch<T>::vcycle(int l, cudaStream_t s) {
  const int nl = h->nl;
  if (l == h->tail_l0) {
    mg_tail<T>(tail, nr, h->tail_width, s);
    return;
  }
  if (l == nl - 1 && !h->coarse_iter) {
    dense_apply_multi<T>(h->nc, nr, h->cinv, b[l], x[l], s);
    return;
  }
  const int n = (int)h->n[l];
  const int degree = h->degree;
  MultiArgs<T> a;
  a.b = b[l];
  a.dinv = h->dinv[l];
  // same buffer rotation as MGHier<T>::vcycle
  const int deg = l == nl - 1 ? kCoarseDegree : degree;
  MultiPtr<T> cur = (deg - 1) % 2 == 0 ? x[l] : t[l];
  MultiPtr<T> oth = (deg - 1) % 2 == 0 ? t[l] : x[l];
  vec_scale_dinv_multi<T>(n, nr, h->coef[l], h->dinv[l], b[l], cur, s);
  for (int k = 1; k < deg; ++k) {
    a.coef = h->coef[l] + 4 + 3 * (k - 1);
    a.w = k == 1 ? MultiPtr<T>() : oth;
    op(l, cur, oth, SPMV_CHEB, a, s);
    std::swap(cur, oth);
  }
  if (l == nl - 1) return;
  MultiArgs<T> ar;
  ar.b = b[l];
  op(l, x[l], r[l], SPMV_RES, ar, s);
  const Transfer &T_ = *h->tr[l];
  const T *Rv = std::is_same<T, double>::value ? reinterpret_cast<const T *>(T_.Rs) : reinterpret_cast<const T *>(T_.Rs32);
  const T *Pv = std::is_same<T, double>::value ? reinterpret_cast<const T *>(T_.Ps) : reinterpret_cast<const T *>(T_.Ps32);
  MultiArgs<T> none;
  spmv_sell_multi<T>(T_.R, Rv, nr, r[l], b[l + 1], SPMV_PLAIN, none, s);
  const int tkc = h->prof && l == 0 ? h->prof->start(Profiler::P1_MG_COARSE, s) : -1;
  vcycle(l + 1, s);
  if (h->prof && l == 0) h->prof->stop(Profiler::P1_MG_COARSE, tkc, s, 0.0);
  spmv_sell_multi<T>(T_.P, Pv, nr, x[l + 1], x[l], SPMV_ADD, none, s);
  a.coef = h->coef[l] + 1;
  a.w = MultiPtr<T>();
  op(l, x[l], t[l], SPMV_CHEB, a, s);
  cur = t[l];
  oth = x[l];
  for (int k = 1; k < degree; ++k) {
    a.coef = h->coef[l] + 4 + 3 * (k - 1);
    a.w = oth;
    op(l, cur, oth, SPMV_CHEB, a, s);
    std::swap(cur, oth);
  }
  if (cur.p[0] != x[l].p[0]) vec_copy_multi<T>(n, nr, cur, x[l], s);
}

template <typename T>
void MGBatch<T>::apply(cudaStream_t s) {
  vcycle(0, s);
}

template struct MGBatch<double>;
template struct MGBatch<float>;

// ---------------------------------------------------------------------------
void KrylovWork::init(Arena &ar, int m_, long nmax_, double *pinned, bool pairs) {
  m = m_;
  nmax = nmax_;
  const long ldmax = (nmax + 31) / 32 * 32;   // basis stride: 256-byte aligned vectors
  V = ar.alloc<double>((long)(m + 1) * ldmax);
  if (pairs && cgs2_fast(m)) V2 = ar.alloc<float2>((long)(m + 1) * ldmax);
  Z = ar.alloc<double>((long)m * ldmax);
  w = ar.alloc<double>(nmax);
  H = ar.alloc<double>((long)(m + 1) * m);
  cs = ar.alloc<double>(m);
  sn = ar.alloc<double>(m);
  g = ar.alloc<double>(m + 1);
  y = ar.alloc<double>(m);
  h1 = ar.alloc<double>(m + 1);
  h2 = ar.alloc<double>(m + 1);
  sc = ar.alloc<double>(8);
  partial = ar.alloc<double>(64L * kReduceMaxBlocks);
  hstat = pinned;
  dv = ar.alloc<double>(8);
  di = ar.alloc<int>(8);
}

namespace {
double read_scalar(const double *dev, double *pinned, cudaStream_t s) {
  CHNSS_CK(cudaMemcpyAsync(pinned, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNSS_CK(cudaStreamSynchronize(s));
  return *pinned;
}
}  // namespace

chnss_status fgmres(LinearOperator &A, const double *b, double *x, double rtol, double atol, int maxit,
                    KrylovWork &ws, chnss_solve_info *info, cudaStream_t s, Profiler *prof) {
  const auto t0 = std::chrono::steady_clock::now();
  const long n = A.size();
  const long ld = (n + 31) / 32 * 32;   // basis stride (keeps every V_j, Z_j 256-byte aligned)
  const int m = ws.m;
  const int ldh = m + 1;
  double *sc = ws.sc;   // [0] ||b||^2, [1] ||r||^2
  vec_fill(n, 0.0, x, s);
  dot<double>(n, b, b, sc, ws.partial, s);
  const double bnorm = std::sqrt(read_scalar(sc, ws.hstat, s));
  const double target = std::max(rtol * bnorm, atol);
  double rnorm = bnorm;
  int iters = 0;
  chnss_status st = CHNSS_OK;
  bool converged = false;
  if (!std::isfinite(bnorm)) {
    st = CHNSS_ERR_NAN;
  } else if (rnorm <= target) {
    converged = true;
  } else {
    vec_copy(n, b, ws.w, s);
    set_scalar(sc + 2, sc, 1.0, true, s);   // sc[2] = ||r||
    while (true) {
      if (ws.V2)
        dfgs_first(n, ws.w, sc + 2, ws.V2, ws.V, s);
      else
        vec_scale_by_inv(n, ws.w, sc + 2, ws.V, s);
      vec_fill(m + 1, 0.0, ws.g, s);
      set_scalar(ws.g, sc + 2, 1.0, false, s);
      int k = 0;
      bool breakdown = false;
      for (int j = 0; j < m; ++j) {
        double *vj = ws.V + (long)j * ld;
        double *zj = ws.Z + (long)j * ld;
        A.precond(vj, zj, s);
        A.apply(zj, ws.w, s);
        const int kv = j + 1;
        const bool fast = cgs2_fast(kv);
        const int tko = prof ? prof->start(Profiler::ORTHO, s) : -1;
        if (ws.V2) {
          // the same passes in double-FP32 arithmetic (same bytes, no FP64 FMAs)
          dfgs_dots(n, ws.V2, ld, kv, ws.w, ws.h1, ws.partial, s);
          dfgs_update_dots(n, ws.V2, ld, kv, ws.h1, ws.w, ws.h2, ws.partial, s);
          if (prof) prof->stop(Profiler::ORTHO, tko, s, 8.0 * n * (2.0 * kv + 3.0), 0.0);
          arnoldi_finish_pyth(j, ldh, ws.H, ws.h1, ws.h2, ws.cs, ws.sn, ws.g, sc + 4, s);
        } else if (fast) {
          // CGS2 passes 1-2: h1 = V^T w; w -= V h1, h2 = V^T w and ||w||^2 in
          // one sweep (V read twice, w read twice and written once; 3k+1 FMAs
          // per element).  Pass 3 forms the next basis vector after the sync.
          cgs2_dots(n, ws.V, ld, kv, ws.w, ws.h1, ws.partial, s);
          cgs2_update_dots(n, ws.V, ld, kv, ws.h1, ws.w, ws.h2, ws.partial, s);
          if (prof) prof->stop(Profiler::ORTHO, tko, s, 8.0 * n * (2.0 * kv + 3.0), 2.0 * n * (3.0 * kv + 1.0));
          arnoldi_finish_pyth(j, ldh, ws.H, ws.h1, ws.h2, ws.cs, ws.sn, ws.g, sc + 4, s);
        } else {
          mdot(n, ws.V, ld, kv, ws.w, ws.h1, ws.partial, s);
          ortho_update_mdot(n, ws.V, ld, kv, ws.h1, ws.w, ws.h2, ws.partial, s);
          ortho_update_norm(n, ws.V, ld, kv, ws.h2, ws.w, sc + 3, ws.partial, s);
          // CGS2: three passes over V_0..V_j (w read 3x, written 2x) and
          // 4k+1 FP64 FMAs per vector element (dot, update + dot, update + norm)
          if (prof) prof->stop(Profiler::ORTHO, tko, s, 8.0 * n * (3.0 * kv + 5.0), 2.0 * n * (4.0 * kv + 1.0));
          arnoldi_finish(j, ldh, ws.H, ws.h1, ws.h2, sc + 3, ws.cs, ws.sn, ws.g, sc + 4, s);
        }
        CHNSS_CK(cudaMemcpyAsync(ws.hstat, sc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CHNSS_CK(cudaStreamSynchronize(s));
        A.after_sync();
        const double est = ws.hstat[0], hn = ws.hstat[1];
        ++iters;
        k = j + 1;
        if (!std::isfinite(est) || !std::isfinite(hn)) {
          st = CHNSS_ERR_NAN;
          break;
        }
        breakdown = hn == 0.0;
        if (!breakdown && ws.V2) {
          // pass 3 in pairs: V read once, w (pairs) read once, V_{j+1} written as pairs and FP64
          const int tk3 = prof ? prof->start(Profiler::ORTHO, s) : -1;
          dfgs_update_scale(n, ws.V2, ld, kv, ws.h2, ws.w, sc + 5, ws.V2 + (long)(j + 1) * ld,
                            ws.V + (long)(j + 1) * ld, s);
          if (prof) prof->stop(Profiler::ORTHO, tk3, s, 8.0 * n * (kv + 3.0), 0.0, 0);
        } else if (!breakdown && fast) {
          // pass 3: V_{j+1} = (w - V h2) / hn (V read once, w read once, V_{j+1} written; k FMAs)
          const int tk3 = prof ? prof->start(Profiler::ORTHO, s) : -1;
          cgs2_update_scale(n, ws.V, ld, kv, ws.h2, ws.w, sc + 5, ws.V + (long)(j + 1) * ld, s);
          if (prof) prof->stop(Profiler::ORTHO, tk3, s, 8.0 * n * (kv + 2.0), 2.0 * n * kv, 0);
        } else if (!breakdown) {
          vec_scale_by_inv(n, ws.w, sc + 5, ws.V + (long)(j + 1) * ld, s);
        }
        if (est <= target || iters >= maxit || breakdown) break;
      }
      if (st != CHNSS_OK) break;
      hessenberg_solve(k, ldh, ws.H, ws.g, ws.y, s);
      combine_columns(n, ws.Z, ld, k, ws.y, x, s);
      A.apply(x, ws.w, s);
      vec_axpby(n, 1.0, b, -1.0, ws.w, s);                 // w = b - A x
      dot<double>(n, ws.w, ws.w, sc + 1, ws.partial, s);
      set_scalar(sc + 2, sc + 1, 1.0, true, s);
      rnorm = std::sqrt(read_scalar(sc + 1, ws.hstat, s));
      if (!std::isfinite(rnorm)) { st = CHNSS_ERR_NAN; break; }
      if (rnorm <= target) { converged = true; break; }
      if (iters >= maxit) { st = CHNSS_ERR_NOCONV; break; }
      if (breakdown) { st = CHNSS_ERR_BREAKDOWN; break; }
    }
  }
  if (info) {
    info->iters = iters;
    info->converged = converged ? 1 : 0;
    info->rel_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return st;
}

chnss_status fgmres_batch(int K, LinearOperator *const *A, const double *const *b, double *const *x, double rtol,
                          double atol, int maxit, KrylovWork *const *ws, chnss_solve_info *info, BatchPrecond &P,
                          cudaStream_t s, Profiler *prof) {
  const auto t0 = std::chrono::steady_clock::now();
  struct Run {
    long n = 0, ld = 0;
    int m = 0, ldh = 0, j = 0, k = 0, iters = 0;
    double bnorm = 0, target = 0, rnorm = 0;
    chnss_status st = CHNSS_OK;
    bool converged = false, done = false, breakdown = false, cycle_start = false, end_cycle = false, fast = false;
  };
  std::vector<Run> R(K);
  // ||b|| of every system, one synchronisation
  for (int q = 0; q < K; ++q) {
    Run &r = R[q];
    KrylovWork &w = *ws[q];
    r.n = A[q]->size();
    r.ld = (r.n + 31) / 32 * 32;
    r.m = w.m;
    r.ldh = r.m + 1;
    vec_fill(r.n, 0.0, x[q], s);
    dot<double>(r.n, b[q], b[q], w.sc, w.partial, s);
    CHNSS_CK(cudaMemcpyAsync(w.hstat, w.sc, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  CHNSS_CK(cudaStreamSynchronize(s));
  for (int q = 0; q < K; ++q) {
    Run &r = R[q];
    KrylovWork &w = *ws[q];
    r.bnorm = std::sqrt(w.hstat[0]);
    r.target = std::max(rtol * r.bnorm, atol);
    r.rnorm = r.bnorm;
    if (!std::isfinite(r.bnorm)) {
      r.st = CHNSS_ERR_NAN;
      r.done = true;
    } else if (r.rnorm <= r.target) {
      r.converged = true;
      r.done = true;
    } else {
      vec_copy(r.n, b[q], w.w, s);
      set_scalar(w.sc + 2, w.sc, 1.0, true, s);   // ||r||
      r.cycle_start = true;
    }
  }
  std::vector<const double *> rin(K);
  std::vector<double *> zout(K);
  while (true) {
    bool any = false;
    for (int q = 0; q < K; ++q) {
      Run &r = R[q];
      KrylovWork &w = *ws[q];
      rin[q] = nullptr;
      zout[q] = nullptr;
      if (r.done) continue;
      if (r.cycle_start) {
        if (w.V2)
          dfgs_first(r.n, w.w, w.sc + 2, w.V2, w.V, s);
        else
          vec_scale_by_inv(r.n, w.w, w.sc + 2, w.V, s);
        vec_fill(r.m + 1, 0.0, w.g, s);
        set_scalar(w.g, w.sc + 2, 1.0, false, s);
        r.j = 0;
        r.breakdown = false;
        r.cycle_start = false;
      }
      rin[q] = w.V + (long)r.j * r.ld;
      zout[q] = w.Z + (long)r.j * r.ld;
      any = true;
    }
    if (!any) break;
    P.apply(K, rin.data(), zout.data(), s);
    {
      // the active systems' operator applies, fused when their operators allow it
      std::vector<LinearOperator *> ops;
      std::vector<const double *> xin;
      std::vector<double *> yout;
      for (int q = 0; q < K; ++q)
        if (rin[q]) {
          ops.push_back(A[q]);
          xin.push_back(zout[q]);
          yout.push_back(ws[q]->w);
        }
      const void *key = ops[0]->batch_key();
      bool same = key != nullptr && ops.size() > 1;
      for (LinearOperator *o : ops) same = same && o->batch_key() == key;
      if (same) ops[0]->apply_batch((int)ops.size(), ops.data(), xin.data(), yout.data(), s);
      else
        for (size_t i = 0; i < ops.size(); ++i) ops[i]->apply(xin[i], yout[i], s);
    }
    for (int q = 0; q < K; ++q) {
      Run &r = R[q];
      if (!rin[q]) continue;
      KrylovWork &w = *ws[q];
      const long n = r.n, ld = r.ld;
      double *sc = w.sc;
      const int kv = r.j + 1;
      r.fast = cgs2_fast(kv);
      const int tko = prof ? prof->start(Profiler::ORTHO, s) : -1;
      if (w.V2) {
        dfgs_dots(n, w.V2, ld, kv, w.w, w.h1, w.partial, s);
        dfgs_update_dots(n, w.V2, ld, kv, w.h1, w.w, w.h2, w.partial, s);
        if (prof) prof->stop(Profiler::ORTHO, tko, s, 8.0 * n * (2.0 * kv + 3.0), 0.0);
        arnoldi_finish_pyth(r.j, r.ldh, w.H, w.h1, w.h2, w.cs, w.sn, w.g, sc + 4, s);
      } else if (r.fast) {
        cgs2_dots(n, w.V, ld, kv, w.w, w.h1, w.partial, s);
        cgs2_update_dots(n, w.V, ld, kv, w.h1, w.w, w.h2, w.partial, s);
        if (prof) prof->stop(Profiler::ORTHO, tko, s, 8.0 * n * (2.0 * kv + 3.0), 2.0 * n * (3.0 * kv + 1.0));
        arnoldi_finish_pyth(r.j, r.ldh, w.H, w.h1, w.h2, w.cs, w.sn, w.g, sc + 4, s);
      } else {
        mdot(n, w.V, ld, kv, w.w, w.h1, w.partial, s);
        ortho_update_mdot(n, w.V, ld, kv, w.h1, w.w, w.h2, w.partial, s);
        ortho_update_norm(n, w.V, ld, kv, w.h2, w.w, sc + 3, w.partial, s);
        if (prof) prof->stop(Profiler::ORTHO, tko, s, 8.0 * n * (3.0 * kv + 5.0), 2.0 * n * (4.0 * kv + 1.0));
        arnoldi_finish(r.j, r.ldh, w.H, w.h1, w.h2, sc + 3, w.cs, w.sn, w.g, sc + 4, s);
      }
      CHNSS_CK(cudaMemcpyAsync(w.hstat, sc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CHNSS_CK(cudaStreamSynchronize(s));
    P.after_sync();
    for (int q = 0; q < K; ++q)
      if (rin[q]) A[q]->after_sync();
    bool any_end = false;
    for (int q = 0; q < K; ++q) {
      Run &r = R[q];
      if (!rin[q]) continue;
      KrylovWork &w = *ws[q];
      const double est = w.hstat[0], hn = w.hstat[1];
      ++r.iters;
      r.k = r.j + 1;
      if (!std::isfinite(est) || !std::isfinite(hn)) {
        r.st = CHNSS_ERR_NAN;
        r.done = true;
        continue;
      }
      r.breakdown = hn == 0.0;
      if (!r.breakdown && w.V2) {
        const int tk3 = prof ? prof->start(Profiler::ORTHO, s) : -1;
        dfgs_update_scale(r.n, w.V2, r.ld, r.k, w.h2, w.w, w.sc + 5, w.V2 + (long)(r.j + 1) * r.ld,
                          w.V + (long)(r.j + 1) * r.ld, s);
        if (prof) prof->stop(Profiler::ORTHO, tk3, s, 8.0 * r.n * (r.k + 3.0), 0.0, 0);
      } else if (!r.breakdown && r.fast) {
        const int tk3 = prof ? prof->start(Profiler::ORTHO, s) : -1;
        cgs2_update_scale(r.n, w.V, r.ld, r.k, w.h2, w.w, w.sc + 5, w.V + (long)(r.j + 1) * r.ld, s);
        if (prof) prof->stop(Profiler::ORTHO, tk3, s, 8.0 * r.n * (r.k + 2.0), 2.0 * r.n * r.k, 0);
      } else if (!r.breakdown) {
        vec_scale_by_inv(r.n, w.w, w.sc + 5, w.V + (long)(r.j + 1) * r.ld, s);
      }
      if (est <= r.target || r.iters >= maxit || r.breakdown) {
        r.end_cycle = true;
      } else if (++r.j == r.m) {
        r.end_cycle = true;
      }
      if (r.end_cycle) {
        // x += Z y; true residual
        hessenberg_solve(r.k, r.ldh, w.H, w.g, w.y, s);
        combine_columns(r.n, w.Z, r.ld, r.k, w.y, x[q], s);
        A[q]->apply(x[q], w.w, s);
        vec_axpby(r.n, 1.0, b[q], -1.0, w.w, s);
        dot<double>(r.n, w.w, w.w, w.sc + 1, w.partial, s);
        set_scalar(w.sc + 2, w.sc + 1, 1.0, true, s);
        CHNSS_CK(cudaMemcpyAsync(w.hstat, w.sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
        any_end = true;
      }
    }
    if (!any_end) continue;
    CHNSS_CK(cudaStreamSynchronize(s));
    for (int q = 0; q < K; ++q) {
      Run &r = R[q];
      if (!r.end_cycle) continue;
      r.end_cycle = false;
      r.rnorm = std::sqrt(ws[q]->hstat[0]);
      if (!std::isfinite(r.rnorm)) { r.st = CHNSS_ERR_NAN; r.done = true; }
      else if (r.rnorm <= r.target) { r.converged = true; r.done = true; }
      else if (r.iters >= maxit) { r.st = CHNSS_ERR_NOCONV; r.done = true; }
      else if (r.breakdown) { r.st = CHNSS_ERR_BREAKDOWN; r.done = true; }
      else r.cycle_start = true;
    }
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  chnss_status worst = CHNSS_OK;
  for (int q = 0; q < K; ++q) {
    const Run &r = R[q];
    if (info) {
      info[q].iters = r.iters;
      info[q].converged = r.converged ? 1 : 0;
      info[q].rel_residual = r.bnorm > 0 ? r.rnorm / r.bnorm : 0.0;
      info[q].seconds = secs;
    }
    if (worst == CHNSS_OK) worst = r.st;
  }
  return worst;
}

// ---------------------------------------------------------------------------
// Device-driven solves.
namespace {
constexpr int kMaxRecRestart = 31;

// x = 0 was done; sc[0] = ||b||^2.  Decide whether any cycle runs.
__global__ void k_fg_init(double *sc, double *dv, int *di, double rtol, double atol,
                          cudaGraphConditionalHandle hw) {
  const double bn = sqrt(sc[0]);
  const double target = fmax(rtol * bn, atol);
  dv[0] = bn;
  dv[1] = target;
  dv[2] = bn;
  for (int i = 0; i < 8; ++i) di[i] = 0;
  bool more = true;
  if (!isfinite(bn)) {
    di[2] = CHNSS_ERR_NAN;
    more = false;
  } else if (bn <= target) {
    di[3] = 1;
    more = false;
  }
  sc[2] = bn;                                         // ||r|| of the first cycle
  cudaGraphSetConditional(hw, more ? 1u : 0u);
}
__global__ void k_fg_cycle_begin(int *di) {
  di[1] = 0;
  di[4] = 0;
  di[6] = 1;                                          // Arnoldi step 0 runs
}
__global__ void k_fg_gate(cudaGraphConditionalHandle h, const int *di) { cudaGraphSetConditional(h, di[6] ? 1u : 0u); }
// after Arnoldi step j: sc[4] = |g_{j+1}| (the residual estimate), sc[5] = H(j+1, j)
__global__ void k_fg_step(int j, int m, const double *sc, const double *dv, int *di, int maxit) {
  const int it = di[0] + 1;
  di[0] = it;
  di[1] = j + 1;
  const double est = sc[4], hn = sc[5];
  bool stop;
  if (!isfinite(est) || !isfinite(hn)) {
    di[5] = 1;
    stop = true;
  } else {
    const bool breakdown = hn == 0.0;
    di[4] = breakdown ? 1 : 0;
    stop = est <= dv[1] || it >= maxit || breakdown;
  }
  di[6] = (!stop && j + 1 < m) ? 1 : 0;
}
// after the cycle's true residual: sc[1] = ||b - A x||^2
__global__ void k_fg_cycle_end(const double *sc, double *dv, int *di, int maxit, cudaGraphConditionalHandle hw) {
  bool more = false;
  if (di[5]) {
    di[2] = CHNSS_ERR_NAN;
  } else {
    const double rn = sqrt(sc[1]);
    dv[2] = rn;
    if (!isfinite(rn)) di[2] = CHNSS_ERR_NAN;
    else if (rn <= dv[1]) di[3] = 1;
    else if (di[0] >= maxit) di[2] = CHNSS_ERR_NOCONV;
    else if (di[4]) di[2] = CHNSS_ERR_BREAKDOWN;
    else more = true;
  }
  cudaGraphSetConditional(hw, more ? 1u : 0u);
}
// PCG: sc[0] = ||b||^2 (b copied to r)
__global__ void k_pcg_init(const double *sc, double *dv, int *di, double rtol, cudaGraphConditionalHandle hw) {
  const double bn = sqrt(sc[0]);
  dv[0] = bn;
  dv[1] = rtol * bn;
  dv[2] = bn;
  for (int i = 0; i < 8; ++i) di[i] = 0;
  bool more = true;
  if (!isfinite(bn)) {
    di[2] = CHNSS_ERR_NAN;
    more = false;
  } else if (bn <= dv[1]) {
    di[3] = 1;
    more = false;
  }
  cudaGraphSetConditional(hw, more ? 1u : 0u);
}
// after an iteration: sc[5] = ||r||^2
__global__ void k_pcg_decide(const double *sc, double *dv, int *di, int maxit, cudaGraphConditionalHandle hw) {
  const int it = di[0] + 1;
  di[0] = it;
  const double rn = sqrt(sc[5]);
  dv[2] = rn;
  bool more = false;
  if (!isfinite(rn)) di[2] = CHNSS_ERR_NAN;
  else if (rn <= dv[1]) di[3] = 1;
  else if (it >= maxit) di[2] = CHNSS_ERR_NOCONV;
  else more = true;
  cudaGraphSetConditional(hw, more ? 1u : 0u);
}
__global__ void k_copy_scalar(const double *src, double *dst) { *dst = *src; }
__global__ void k_krylov_record(const double *dv, const int *di, double *dst) {
  dst[0] = (double)di[0];
  dst[1] = (double)di[3];
  dst[2] = dv[0] > 0.0 ? dv[2] / dv[0] : 0.0;
  dst[3] = (double)di[2];
}

// Add a conditional node of the given type after the capture position of s
// (handle h, created on s's capture graph and set by an earlier node) and
// start capturing its body on q.  end_body() finishes the body and makes
// the node the capture position of s.
cudaGraphNode_t begin_body(cudaStream_t s, cudaStream_t q, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edata = nullptr;
  size_t nd = 0;
  CHNSS_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edata, &nd));
  if (cs != cudaStreamCaptureStatusActive) throw Error{CHNSS_ERR_STATE, "device-driven solve outside a stream capture"};
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CHNSS_CK(cudaGraphAddNode(&node, g, deps, edata, nd, &np));
  CHNSS_CK(cudaStreamBeginCaptureToGraph(q, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
  return node;
}
void end_body(cudaStream_t s, cudaStream_t q, cudaGraphNode_t node) {
  cudaGraph_t tmp = nullptr;
  CHNSS_CK(cudaStreamEndCapture(q, &tmp));
  CHNSS_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
}
cudaGraphConditionalHandle new_handle(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  CHNSS_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) throw Error{CHNSS_ERR_STATE, "device-driven solve outside a stream capture"};
  cudaGraphConditionalHandle h;
  CHNSS_CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  return h;
}
// a failed body capture must still end it, or the streams stay in capture mode
template <typename F>
void record_body(cudaStream_t s, cudaStream_t q, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                 F &&body) {
  const cudaGraphNode_t node = begin_body(s, q, h, type);
  try {
    body();
  } catch (...) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(q, &tmp);
    throw;
  }
  end_body(s, q, node);
}
}  // namespace

void fgmres_record(LinearOperator &A, const double *b, double *x, double rtol, double atol, int maxit,
                   KrylovWork &ws, cudaStream_t s, cudaStream_t bq1, cudaStream_t bq2) {
  const long n = A.size();
  const long ld = (n + 31) / 32 * 32;
  const int m = ws.m;
  const int ldh = m + 1;
  if (m > kMaxRecRestart) throw Error{CHNSS_ERR_ARG, "device-driven FGMRES needs restart <= 31"};
  double *sc = ws.sc;
  vec_fill(n, 0.0, x, s);
  dot<double>(n, b, b, sc, ws.partial, s);
  const cudaGraphConditionalHandle hw = new_handle(s);
  k_fg_init<<<1, 1, 0, s>>>(sc, ws.dv, ws.di, rtol, atol, hw);
  CHNSS_LAUNCH_CK();
  vec_copy(n, b, ws.w, s);
  record_body(s, bq1, hw, cudaGraphCondTypeWhile, [&] {
    if (ws.V2)
      dfgs_first(n, ws.w, sc + 2, ws.V2, ws.V, bq1);
    else
      vec_scale_by_inv(n, ws.w, sc + 2, ws.V, bq1);
    vec_fill(m + 1, 0.0, ws.g, bq1);
    set_scalar(ws.g, sc + 2, 1.0, false, bq1);
    k_fg_cycle_begin<<<1, 1, 0, bq1>>>(ws.di);
    CHNSS_LAUNCH_CK();
    for (int j = 0; j < m; ++j) {
      const cudaGraphConditionalHandle hj = new_handle(bq1);
      k_fg_gate<<<1, 1, 0, bq1>>>(hj, ws.di);
      CHNSS_LAUNCH_CK();
      record_body(bq1, bq2, hj, cudaGraphCondTypeIf, [&] {
        double *vj = ws.V + (long)j * ld;
        double *zj = ws.Z + (long)j * ld;
        A.precond(vj, zj, bq2);
        A.apply(zj, ws.w, bq2);
        const int kv = j + 1;
        if (ws.V2) {
          dfgs_dots(n, ws.V2, ld, kv, ws.w, ws.h1, ws.partial, bq2);
          dfgs_update_dots(n, ws.V2, ld, kv, ws.h1, ws.w, ws.h2, ws.partial, bq2);
          arnoldi_finish_pyth(j, ldh, ws.H, ws.h1, ws.h2, ws.cs, ws.sn, ws.g, sc + 4, bq2);
          dfgs_update_scale(n, ws.V2, ld, kv, ws.h2, ws.w, sc + 5, ws.V2 + (long)(j + 1) * ld,
                            ws.V + (long)(j + 1) * ld, bq2);
        } else {
          cgs2_dots(n, ws.V, ld, kv, ws.w, ws.h1, ws.partial, bq2);
          cgs2_update_dots(n, ws.V, ld, kv, ws.h1, ws.w, ws.h2, ws.partial, bq2);
          arnoldi_finish_pyth(j, ldh, ws.H, ws.h1, ws.h2, ws.cs, ws.sn, ws.g, sc + 4, bq2);
          cgs2_update_scale(n, ws.V, ld, kv, ws.h2, ws.w, sc + 5, ws.V + (long)(j + 1) * ld, bq2);
        }
        k_fg_step<<<1, 1, 0, bq2>>>(j, m, sc, ws.dv, ws.di, maxit);
        CHNSS_LAUNCH_CK();
      });
    }
    hessenberg_solve_dev(ws.di + 1, ldh, ws.H, ws.g, ws.y, bq1);
    combine_columns_dev(n, ws.Z, ld, ws.di + 1, ws.y, x, bq1);
    A.apply(x, ws.w, bq1);
    vec_axpby(n, 1.0, b, -1.0, ws.w, bq1);                 // w = b - A x
    dot<double>(n, ws.w, ws.w, sc + 1, ws.partial, bq1);
    set_scalar(sc + 2, sc + 1, 1.0, true, bq1);
    k_fg_cycle_end<<<1, 1, 0, bq1>>>(sc, ws.dv, ws.di, maxit, hw);
    CHNSS_LAUNCH_CK();
  });
}

void pcg_record(const Pattern &P, const double *val, const double *dinv, const double *b, double *x, double rtol,
                int maxit, KrylovWork &ws, cudaStream_t s, cudaStream_t bq1) {
  const long n = P.nrows;
  double *r = ws.w, *z = ws.V, *p = ws.V + n, *q = ws.V + 2 * n;
  double *sc = ws.sc;   // [0] bb [1] rz [2] rz_new [3] pq [4] alpha [5] rr
  vec_copy(n, b, r, s);
  dot<double>(n, r, r, sc, ws.partial, s);
  vec_fill(n, 0.0, x, s);
  const cudaGraphConditionalHandle hw = new_handle(s);
  k_pcg_init<<<1, 1, 0, s>>>(sc, ws.dv, ws.di, rtol, hw);
  CHNSS_LAUNCH_CK();
  vec_mul(n, dinv, r, z, s);
  vec_copy(n, z, p, s);
  dot<double>(n, r, z, sc + 1, ws.partial, s);
  record_body(s, bq1, hw, cudaGraphCondTypeWhile, [&] {
    SpmvArgs none;
    spmv_csr<double>(P, val, 1, p, q, SPMV_PLAIN, none, bq1);
    dot<double>(n, p, q, sc + 3, ws.partial, bq1);
    pcg_alpha(sc + 1, sc + 3, sc + 4, bq1);
    pcg_update_xr(n, sc + 4, p, q, x, r, bq1);
    dot<double>(n, r, r, sc + 5, ws.partial, bq1);
    k_pcg_decide<<<1, 1, 0, bq1>>>(sc, ws.dv, ws.di, maxit, hw);
    CHNSS_LAUNCH_CK();
    // the next direction (unused once the loop has stopped)
    vec_mul(n, dinv, r, z, bq1);
    dot<double>(n, r, z, sc + 2, ws.partial, bq1);
    pcg_update_p(n, sc + 2, sc + 1, z, p, bq1);
    k_copy_scalar<<<1, 1, 0, bq1>>>(sc + 2, sc + 1);
    CHNSS_LAUNCH_CK();
  });
}

void krylov_record(const KrylovWork &ws, double *dst, cudaStream_t s) {
  k_krylov_record<<<1, 1, 0, s>>>(ws.dv, ws.di, dst);
  CHNSS_LAUNCH_CK();
}

chnss_status pcg(const Pattern &P, const double *val, const double *dinv, const double *b, double *x, double rtol,
                 int maxit, KrylovWork &ws, chnss_solve_info *info, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const long n = P.nrows;
  double *r = ws.w, *z = ws.V, *p = ws.V + n, *q = ws.V + 2 * n;
  double *sc = ws.sc;   // [0] bb [1] rz [2] rz_new [3] pq [4] alpha [5] rr
  // b is read only here, into r, before x is cleared: x may alias b
  vec_copy(n, b, r, s);
  dot<double>(n, r, r, sc, ws.partial, s);
  vec_fill(n, 0.0, x, s);
  const double bnorm = std::sqrt(read_scalar(sc, ws.hstat, s));
  const double target = rtol * bnorm;
  double rn = bnorm;
  int it = 0;
  bool converged = false;
  chnss_status st = CHNSS_OK;
  if (!std::isfinite(bnorm)) {
    st = CHNSS_ERR_NAN;
  } else if (bnorm <= target) {
    converged = true;
  } else {
    vec_mul(n, dinv, r, z, s);
    vec_copy(n, z, p, s);
    dot<double>(n, r, z, sc + 1, ws.partial, s);
    double *rz = sc + 1, *rzn = sc + 2;
    SpmvArgs none;
    while (it < maxit) {
      spmv_csr<double>(P, val, 1, p, q, SPMV_PLAIN, none, s);
      dot<double>(n, p, q, sc + 3, ws.partial, s);
      pcg_alpha(rz, sc + 3, sc + 4, s);
      pcg_update_xr(n, sc + 4, p, q, x, r, s);
      ++it;
      dot<double>(n, r, r, sc + 5, ws.partial, s);
      rn = std::sqrt(read_scalar(sc + 5, ws.hstat, s));
      if (!std::isfinite(rn)) { st = CHNSS_ERR_NAN; break; }
      if (rn <= target) { converged = true; break; }
      vec_mul(n, dinv, r, z, s);
      dot<double>(n, r, z, rzn, ws.partial, s);
      pcg_update_p(n, rzn, rz, z, p, s);
      std::swap(rz, rzn);
    }
    if (!converged && st == CHNSS_OK) st = CHNSS_ERR_NOCONV;
  }
  if (info) {
    info->iters = it;
    info->converged = converged ? 1 : 0;
    info->rel_residual = bnorm > 0 ? rn / bnorm : 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return st;
}

}  // namespace chnss
