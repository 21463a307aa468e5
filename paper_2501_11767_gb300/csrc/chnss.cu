// Context, per-step assembly, block preconditioners, step orchestration and
// the C ABI of include/chnss.h.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <future>
#include <thread>

#include "amg.h"
#include "solver.h"

using namespace chnss;

struct chnss_mesh {
  Mesh m;
};

namespace {

thread_local std::string g_last_error;

}  // namespace

// the last error of calls without a context (chnss_last_error(NULL))
void chnss::set_global_error(const std::string &msg) { g_last_error = msg; }

namespace {

// ---------------------------------------------------------------------------
// small kernels of the step
constexpr int TPB = 256;
inline int nb(long n) { return (int)((n + TPB - 1) / TPB); }

__device__ __forceinline__ double top_load(int node, int n, double hx) {
  const int i = node % (n + 1), j = node / (n + 1);
  if (j != n) return 0.0;
  return (i == 0 || i == n) ? 0.5 * hx : hx;
}
__device__ __forceinline__ double evap_flux(const double *phi_s, int ref, double evap, double inf) {
  return evap * (phi_s[ref] - inf);
}

// out = -c (load + sgn * beta * j_out * t)   (second block of eqn:CH_linear)
__global__ void k_ch_rhs_mu(int N1, int n, double hx, const double *load, const double *phi_s, int ref, double evap,
                            double inf, double sgn_beta, double c, double *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= N1) return;
  const double j = evap_flux(phi_s, ref, evap, inf);
  out[i] = -c * (load[i] + sgn_beta * j * top_load(i, n, hx));
}
// out = out - tau gamma_v f_v + ctop j_out t   (AC right-hand side)
__global__ void k_ac_rhs(int N1, int n, double hx, const double *fv, double tg, double ctop, const double *phi_s,
                         int ref, double evap, double inf, double *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= N1) return;
  const double j = evap_flux(phi_s, ref, evap, inf);
  out[i] = out[i] - tg * fv[i] + ctop * j * top_load(i, n, hx);
}
// out = 1 - phi_p - phi_N - phi_s
__global__ void k_phi_a(int N1, const double *a, const double *b, const double *c, double *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < N1) out[i] = 1.0 - a[i] - b[i] - c[i];
}
// x -= sum / denom
__global__ void k_shift(int n, double *x, const double *sum, double denom) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < n) x[i] -= *sum / denom;
}
// constant velocity blocks: + (M2 / tau) I on every block, identity on
// Dirichlet diagonal blocks
__global__ void k_aconst_finish(int N2, const int *rowptr, const double *m2, const int *diag, const int *bnd,
                                double inv_tau, double *A) {
  const int r = blockIdx.x * TPB + threadIdx.x;
  if (r >= N2) return;
  for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    A[4L * k] += m2[k] * inv_tau;
    A[4L * k + 3] += m2[k] * inv_tau;
  }
  if (bnd[r]) {
    double *d = A + 4L * diag[r];
    d[0] = 1.0; d[1] = 0.0; d[2] = 0.0; d[3] = 1.0;
  }
}
// Homogeneous Dirichlet rows / columns on the top P1 nodes (j = n) of a P1
// CSR matrix: identity rows, zero coupling (outflow condition of the
// pressure convection-diffusion operators on an open top).
__global__ void k_p1_top_dirichlet(int n, const int *rowptr, const int *col, double *val) {
  const int N1 = (n + 1) * (n + 1);
  const int r = blockIdx.x * TPB + threadIdx.x;
  if (r >= N1) return;
  const bool rtop = r / (n + 1) == n;
  for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    const int c = col[k];
    if (rtop) val[k] = c == r ? 1.0 : 0.0;
    else if (c / (n + 1) == n) val[k] = 0.0;
  }
}

__global__ void k_inv_diag(int n, const double *val, const int *diag, double *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < n) out[i] = 1.0 / val[diag[i]];
}

Geo geo(const Level &L) { return Geo{L.n, L.hx, L.hy}; }

// ---------------------------------------------------------------------------
constexpr int kNumPrec = 6;          // 0..2 CH species, 3 AC, 4 NS, 5 the three CH species together
constexpr int kBatchSlot = 2 * kNumPrec;   // slots of preconditioner 5: in0, out0, in1, out1, in2, out2
constexpr int kMaxProbes = 32;
struct PrecGraph {
  cudaGraphExec_t plain = nullptr, prof = nullptr;
  std::vector<Profiler::Probe> probes;
  size_t nprobes = 0;
  long long nodes = 0;          // kernels launched by one replay
};

template <typename T>
struct PrecSet {
  MGHier<T> L, AC, A, Kp;
  MGHier<T> X1[3], X2[3];
  // the three CH species together (constant mobility): MG(L) on three
  // vectors, and one X1 V-cycle per group of species with equal X1
  MGBatch<T> LB, XB[3];
  int ngroups = 0, gsize[3] = {0, 0, 0}, gmem[3][3] = {};
  T *Mv = nullptr, *Apv = nullptr, *mdinv = nullptr;
  T *mx = nullptr, *mt = nullptr, *mb = nullptr;
};

}  // namespace

struct chnss_ctx {
  chnss_mesh *mesh = nullptr;
  chnss_params p{};
  cudaStream_t s = nullptr;
  Arena ar;
  std::string err;
  double *pinned = nullptr;
  int nlev = 0, N1 = 0, N2 = 0, E = 0;
  double *ebuf = nullptr, *lbuf = nullptr;
  std::vector<double *> M1, K1, ACb, M2v, Aconst, L, AC, A;
  std::vector<std::array<double *, 3>> X1, X2;
  std::vector<double *> vl, mul, phil;
  double *Apb = nullptr, *Ap = nullptr, *Bv = nullptr, *Btv = nullptr, *dinvM = nullptr;
  // SELL-ordered copies of the fine FP64 operators applied inside FGMRES
  double *Ls = nullptr, *ACs = nullptr, *As = nullptr, *Ks = nullptr, *Ms = nullptr, *Bs = nullptr, *Bts = nullptr;
  double *Kks[3] = {nullptr, nullptr, nullptr};
  double *Kk[3] = {nullptr, nullptr, nullptr};
  double *loads = nullptr, *G = nullptr, *fa = nullptr, *tmp = nullptr, *sum = nullptr, *partial = nullptr;
  double *partial_ch = nullptr;             // reductions of the CH / AC hierarchies' setup (own stream)
  double *rhs[6] = {};
  double *xsol[6] = {};
  double *massc = nullptr;
  double *diag = nullptr;                   // chnss_diagnostics: kDiagQuantities sums + ||B v||^2
  // device-driven step (chnss_set_step_mode 1): a whole step captured as one
  // CUDA graph per pair of state arrays (two pairs cached)
  struct StepGraph {
    std::array<const void *, 20> key{};
    cudaGraphExec_t exec = nullptr;
  };
  int step_mode = 0;
  bool recording = false;                   // preconditioners record their bodies inline
  StepGraph sgr[2];
  int sg_next = 0;
  unsigned long long sg_gen = 0;               // bumped whenever the recorded graphs are dropped
  cudaStream_t rq0 = nullptr;                  // private stream the step is recorded on
  cudaStream_t rq1 = nullptr, rq2 = nullptr;   // capture streams of the conditional bodies
  double *srec = nullptr, *srec_h = nullptr;   // per solve [iterations, converged, rel. residual, status]
  std::unique_ptr<PrecSet<double>> p64;
  std::unique_ptr<PrecSet<float>> p32;
  chnss::AmgHandle *amg_ac = nullptr;        // params.amg = 1: smoothed-aggregation levels of the AC block
  // captured preconditioner graphs (0..2 CH species, 3 AC, 4 NS)
  double **slots = nullptr;   // device [2 * kNumPrec] input / output pointers
  cudaStream_t cap = nullptr; // private stream used for capture only
  cudaStream_t bodyq = nullptr;  // captures the bodies of the inner multigrid loops
  // side branches of the preconditioner graphs (independent parts of one
  // preconditioner run as parallel graph branches): streams and the
  // fork / join events
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
  PrecGraph pg[kNumPrec];
  bool ch_batch = false;                    // step() solves the CH species together
  KrylovWork kwb[2];                        // Krylov work of the 2nd and 3rd CH species
  double *dummy_in = nullptr, *dummy_out = nullptr;   // idle batch members (2 N1 each)
  bool probe_pending[kNumPrec] = {};        // graph replays whose probes await harvesting
  KrylovWork kw;                            // NS (and single solves on the context stream)
  KrylovWork kwc0, kwa;                     // CH species 0 (step), AC (step)
  // step(): CH (+ air potential), AC and NS are independent given the step-k
  // data (Sec. 3), so they run on three streams driven by three host threads
  cudaStream_t sx[3] = {nullptr, nullptr, nullptr};
  bool concurrent = true;                   // chnss_set_step_concurrency
  cudaEvent_t ev_asm = nullptr, ev_done[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_chac = nullptr;            // CH / AC assembly done (concurrent step)
  double *tmp_ns = nullptr;
  std::vector<double *> Kpd;                // open top: K_p with Dirichlet top rows, per level
  Profiler prof;
  bool assembled = false;
  bool ch_done[3] = {false, false, false};
  double *hin = nullptr, *hout = nullptr;   // device staging of chnss_step_host
  // adjoint step (allocated on first use): transposed fine operators, work
  double *LsT = nullptr, *ACsT = nullptr, *AsT = nullptr;
  double *topv = nullptr, *mvec = nullptr;  // int_Gt psi, M 1
  double *arhs = nullptr, *ay = nullptr, *alam = nullptr, *az = nullptr, *atmp = nullptr, *atv = nullptr;
  double *alw[5] = {};
  // per-group work and accumulators of the concurrent adjoint step (AC, CH)
  double *ay_ac = nullptr, *aPhi = nullptr, *v_ac = nullptr;
  double *arhs_ch = nullptr, *ay_ch = nullptr, *atmp_ch = nullptr, *aphi = nullptr, *v_ch = nullptr;
  double *adots = nullptr;                  // device scalars of the parameter gradients
  const Level &lv(int l) const { return mesh->m.lv[l]; }
  ~chnss_ctx() {
    if (amg_ac) chnss::amg_release(amg_ac);
    for (PrecGraph &g : pg) {
      if (g.plain) cudaGraphExecDestroy(g.plain);
      if (g.prof) cudaGraphExecDestroy(g.prof);
      for (Profiler::Probe &pr : g.probes) {
        if (pr.e0) cudaEventDestroy(pr.e0);
        if (pr.e1) cudaEventDestroy(pr.e1);
      }
    }
    if (cap) cudaStreamDestroy(cap);
    if (bodyq) cudaStreamDestroy(bodyq);
    for (cudaStream_t q : side)
      if (q) cudaStreamDestroy(q);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (cudaEvent_t e : ev_join)
      if (e) cudaEventDestroy(e);
    for (cudaStream_t q : sx)
      if (q) cudaStreamDestroy(q);
    for (StepGraph &g : sgr)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    if (rq0) cudaStreamDestroy(rq0);
    if (rq1) cudaStreamDestroy(rq1);
    if (rq2) cudaStreamDestroy(rq2);
    if (srec_h) cudaFreeHost(srec_h);
    if (ev_asm) cudaEventDestroy(ev_asm);
    if (ev_chac) cudaEventDestroy(ev_chac);
    for (cudaEvent_t e : ev_done)
      if (e) cudaEventDestroy(e);
  }
};

namespace {

// ---------------------------------------------------------------------------
// preconditioner applications (Sec. 4).  The input r and output z are read
// and written through a device pointer slot (slot[0] = r, slot[1] = z), so
// the whole launch sequence is captured once into a CUDA graph and replayed
// for any pair of Krylov vectors.
// Fork side stream k off s (its work becomes a parallel branch when s is
// capturing) and join it back.
// Without concurrency (chnss_set_step_concurrency 0) the "side" is s itself.
cudaStream_t fork_side(chnss_ctx *c, cudaStream_t s, int k) {
  if (!c->concurrent) return s;
  CHNSS_CK(cudaEventRecord(c->ev_fork, s));
  CHNSS_CK(cudaStreamWaitEvent(c->side[k], c->ev_fork, 0));
  return c->side[k];
}
void join_side(chnss_ctx *c, cudaStream_t s, int k) {
  if (!c->concurrent) return;
  CHNSS_CK(cudaEventRecord(c->ev_join[k], c->side[k]));
  CHNSS_CK(cudaStreamWaitEvent(s, c->ev_join[k], 0));
}

template <typename T>
void ch_precond(chnss_ctx *c, PrecSet<T> &P, int sp, double **slot, cudaStream_t s) {
  const int N1 = c->N1;
  const double *const *in = const_cast<const double *const *>(slot);
  double *const *out = slot + 1;
  vec_convert_from_slot<double, T>(N1, in, 0, P.L.input(), s);
  P.L.apply(s);
  P.L.write_output(out, 0, s);
  // S~^-1 = X2^-1 M X1^-1 (matching factors of eqn::schurCH)
  MGHier<T> &X1 = P.X1[sp];
  MGHier<T> &X2 = c->p.mobility_kind == 0 ? P.X1[sp] : P.X2[sp];
  vec_convert_from_slot<double, T>(N1, in, N1, X1.input(), s);
  X1.apply(s);
  SpmvArgs none;
  spmv_sell<T>(c->lv(0).p1, P.Mv, 1, X1.output(), X2.input(), SPMV_PLAIN, none, s);
  X2.apply(s);
  X2.write_output(out, N1, s);
}

// The three species' preconditioners in one pass (slots kBatchSlot..+5):
// per species the same operations as ch_precond, with the matrix sweeps of
// MG(L) and of each X1 group shared by the group's vectors.
template <typename T>
void ch_precond_batched(chnss_ctx *c, PrecSet<T> &P, cudaStream_t s) {
  const int N1 = c->N1;
  double **slot = c->slots + kBatchSlot;
  const double *const *in = const_cast<const double *const *>(slot);
  const Pattern &p1 = c->lv(0).p1;
  // the Schur parts of the species groups are independent of MG(L) and of
  // each other: one side branch per group
  for (int g = 0; g < P.ngroups; ++g) {
    cudaStream_t q = fork_side(c, s, g);
    MGBatch<T> &X = P.XB[g];
    for (int j = 0; j < P.gsize[g]; ++j) vec_convert_from_slot<double, T>(N1, in + 2 * P.gmem[g][j], N1, X.input(j), q);
    X.apply(q);
    MultiArgs<T> none;
    if (c->p.mobility_kind == 0) {   // X2 = X1: a second batched V-cycle
      spmv_sell_multi<T>(p1, P.Mv, P.gsize[g], X.x[0], X.b[0], SPMV_PLAIN, none, q);
      X.apply(q);
      for (int j = 0; j < P.gsize[g]; ++j)
        vec_convert_to_slot<T, double>(N1, X.output(j), slot + 2 * P.gmem[g][j] + 1, N1, q);
    } else {                         // X2 per species (tau K_kappa + a M at t_k)
      MultiPtr<T> x2in;
      for (int j = 0; j < P.gsize[g]; ++j) x2in.p[j] = P.X2[P.gmem[g][j]].input();
      spmv_sell_multi<T>(p1, P.Mv, P.gsize[g], X.x[0], x2in, SPMV_PLAIN, none, q);
      for (int j = 0; j < P.gsize[g]; ++j) {
        MGHier<T> &X2 = P.X2[P.gmem[g][j]];
        X2.apply(q);
        vec_convert_to_slot<T, double>(N1, X2.output(), slot + 2 * P.gmem[g][j] + 1, N1, q);
      }
    }
  }
  for (int k = 0; k < 3; ++k) vec_convert_from_slot<double, T>(N1, in + 2 * k, 0, P.LB.input(k), s);
  P.LB.apply(s);
  for (int k = 0; k < 3; ++k) vec_convert_to_slot<T, double>(N1, P.LB.output(k), slot + 2 * k + 1, 0, s);
  for (int g = 0; g < P.ngroups; ++g) join_side(c, s, g);
}

template <typename T>
void ac_precond(chnss_ctx *c, PrecSet<T> &P, double **slot, cudaStream_t s) {
  vec_convert_from_slot<double, T>(c->N1, const_cast<const double *const *>(slot), 0, P.AC.input(), s);
  P.AC.apply(s);
  P.AC.write_output(slot + 1, 0, s);
}

template <typename T>
void ns_precond(chnss_ctx *c, PrecSet<T> &P, double **slot, cudaStream_t s) {
  const long nv = 2L * c->N2;
  const int N1 = c->N1;
  const double *const *in = const_cast<const double *const *>(slot);
  double *const *out = slot + 1;
  // the pressure block is independent of the velocity block: a side branch
  cudaStream_t q = fork_side(c, s, 0);
  // pressure convection-diffusion: M_p^-1 A_p K_p^-1
  vec_convert_from_slot<double, T>(N1, in, nv, P.Kp.input(), q);
  P.Kp.apply(q);
  SpmvArgs none;
  const Pattern &p1 = c->lv(0).p1;
  spmv_sell<T>(p1, P.Apv, 1, P.Kp.output(), P.mb, SPMV_PLAIN, none, q);
  // M_p^-1 by Chebyshev iteration of degree 5 on D^-1 M, spectrum [1/2, 2]
  vec_scale_dinv<T>(N1, c->massc, P.mdinv, P.mb, P.mx, q);
  SpmvArgs a;
  a.b = P.mb;
  a.dinv = P.mdinv;
  T *cur = P.mx, *other = P.mt;
  for (int k = 1; k <= 4; ++k) {
    a.coef = c->massc + 1 + 3 * (k - 1);
    a.w = k == 1 ? nullptr : other;
    spmv_sell<T>(p1, P.Mv, 1, cur, other, SPMV_CHEB, a, q);
    std::swap(cur, other);
  }
  vec_convert_to_slot<T, double>(N1, cur, out, nv, q);
  // velocity block on s
  vec_convert_from_slot<double, T>(nv, in, 0, P.A.input(), s);
  P.A.apply(s);
  P.A.write_output(out, 0, s);
  join_side(c, s, 0);
}

// preconditioner g: 0..2 CH species, 3 AC, 4 NS
template <typename T>
void prec_body_t(chnss_ctx *c, PrecSet<T> &P, int g, cudaStream_t s) {
  double **slot = c->slots + 2 * g;
  if (g < 3) ch_precond(c, P, g, slot, s);
  else if (g == 3) ac_precond(c, P, slot, s);
  else if (g == 4) ns_precond(c, P, slot, s);
  else ch_precond_batched(c, P, s);
}
void prec_body(chnss_ctx *c, int g, cudaStream_t s) {
  if (c->p32) prec_body_t(c, *c->p32, g, s);
  else prec_body_t(c, *c->p64, g, s);
}

void run_prec(chnss_ctx *c, int g, const double *r, double *z, cudaStream_t s) {
  set_ptr_slots(reinterpret_cast<void **>(c->slots + 2 * g), r, z, s);
  PrecGraph &pg = c->pg[g];
  if (!pg.plain || c->recording) {
    prec_body(c, g, s);
    return;
  }
  const bool prof = c->prof.on && pg.prof;
  CHNSS_CK(cudaGraphLaunch(prof ? pg.prof : pg.plain, s));
  g_launch_count.fetch_add(pg.nodes, std::memory_order_relaxed);
  if (prof) c->probe_pending[g] = true;
}

// batch members: inputs / outputs of the three species; idle members read
// zeros and write a scratch vector
struct CHBatchPrec : BatchPrecond {
  chnss_ctx *c;
  explicit CHBatchPrec(chnss_ctx *c_) : c(c_) {}
  void apply(int K, const double *const *r, double *const *z, cudaStream_t s) override;
  void after_sync() override;
};

// after the stream that replayed graph g has been synchronised
void harvest_probes(chnss_ctx *c, int g) {
  if (c->probe_pending[g]) {
    const PrecGraph &pg = c->pg[g];
    c->prof.harvest(pg.probes, pg.nprobes);
    c->probe_pending[g] = false;
  }
}

void CHBatchPrec::apply(int K, const double *const *r, double *const *z, cudaStream_t s) {
  const void *ptrs[6];
  for (int k = 0; k < 3; ++k) {
    ptrs[2 * k] = k < K && r[k] ? r[k] : c->dummy_in;
    ptrs[2 * k + 1] = k < K && z[k] ? z[k] : c->dummy_out;
  }
  set_ptr_slots_n(reinterpret_cast<void **>(c->slots + kBatchSlot), 6, ptrs, s);
  PrecGraph &pg = c->pg[5];
  if (!pg.plain) {
    prec_body(c, 5, s);
    return;
  }
  const bool prof = c->prof.on && pg.prof;
  CHNSS_CK(cudaGraphLaunch(prof ? pg.prof : pg.plain, s));
  g_launch_count.fetch_add(pg.nodes, std::memory_order_relaxed);
  if (prof) c->probe_pending[5] = true;
}
void CHBatchPrec::after_sync() { harvest_probes(c, 5); }

struct CHOp : LinearOperator {
  chnss_ctx *c;
  int sp;
  CHOp(chnss_ctx *c_, int sp_) : c(c_), sp(sp_) {}
  long size() const override { return 2L * c->N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const auto &p = c->p;
    const double tau = p.tau, g = p.gamma[sp], b = p.beta[sp];
    const bool var = p.mobility_kind != 0;
    spmv_sell_ch(c->lv(0).p1, c->Ls, c->Ks, var ? c->Kks[sp] : nullptr, c->Ms, var ? tau : tau * g, tau * g,
            -tau * g / b, x, y, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec(c, sp, r, z, s); }
  void after_sync() override { harvest_probes(c, sp); }
  // with constant mobility the species share L, K and M: one pass over them
  const void *batch_key() const override { return c->p.mobility_kind == 0 ? c : nullptr; }
  void apply_batch(int n, LinearOperator *const *ops, const double *const *x, double *const *y,
                   cudaStream_t s) override {
    const auto &p = c->p;
    ChCoef3 cf{};
    MultiPtr<const double> xs;
    MultiPtr<double> ys;
    for (int i = 0; i < n; ++i) {
      const int q = static_cast<const CHOp *>(ops[i])->sp;
      const double g = p.gamma[q], b = p.beta[q];
      cf.a12[i] = p.tau * g;
      cf.a21[i] = p.tau * g;
      cf.a22[i] = -p.tau * g / b;
      xs.p[i] = x[i];
      ys.p[i] = y[i];
    }
    spmv_sell_ch_multi(c->lv(0).p1, c->Ls, c->Ks, nullptr, c->Ms, n, cf, xs, ys, s);
  }
};

struct ACOp : LinearOperator {
  chnss_ctx *c;
  explicit ACOp(chnss_ctx *c_) : c(c_) {}
  long size() const override { return c->N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    SpmvArgs none;
    spmv_sell<double>(c->lv(0).p1, c->ACs, 1, x, y, SPMV_PLAIN, none, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec(c, 3, r, z, s); }
  void after_sync() override { harvest_probes(c, 3); }
};

struct NSOp : LinearOperator {
  chnss_ctx *c;
  explicit NSOp(chnss_ctx *c_) : c(c_) {}
  long size() const override { return 2L * c->N2 + c->N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const long nv = 2L * c->N2;
    SpmvArgs none;
    const Pattern &p2 = c->lv(0).p2;
    const int tk = c->prof.start(Profiler::NS_OUTER_SPMV, s);
    spmv_sell_bsr2<double>(p2, c->As, x, y, SPMV_PLAIN, none, s);
    c->prof.stop(Profiler::NS_OUTER_SPMV, tk, s, (double)p2.nnz * 36.0 + 4.0 * (p2.nrows + 1) + 2.0 * nv * 8.0);
    spmv_sell_bt_add(c->mesh->m.pbt, c->Bts, x + nv, y, s);
    spmv_sell_b(c->mesh->m.pb, c->Bs, x, y + nv, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec(c, 4, r, z, s); }
  void after_sync() override { harvest_probes(c, 4); }
};

// Capture every preconditioner into two graphs: plain, and with probe
// events around the fine-level sweeps (used while profiling is on).
void capture_graphs(chnss_ctx *c) {
  CHNSS_CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  for (int g = 0; g < kNumPrec; ++g) {
    if (g == 5 && !c->ch_batch) continue;
    PrecGraph &pg = c->pg[g];
    pg.probes.resize(kMaxProbes);
    for (Profiler::Probe &pr : pg.probes) {
      CHNSS_CK(cudaEventCreate(&pr.e0));
      CHNSS_CK(cudaEventCreate(&pr.e1));
    }
    for (int variant = 0; variant < 2; ++variant) {
      const long long before = g_launch_count.load();
      c->prof.sink = variant == 1 ? &pg.probes : nullptr;
      c->prof.sink_used = 0;
      CHNSS_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
      cudaGraph_t graph = nullptr;
      try {
        prec_body(c, g, c->cap);
      } catch (...) {
        c->prof.sink = nullptr;
        cudaStreamEndCapture(c->cap, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      if (variant == 1) pg.nprobes = c->prof.sink_used;
      c->prof.sink = nullptr;
      CHNSS_CK(cudaStreamEndCapture(c->cap, &graph));
      cudaGraphExec_t exec = nullptr;
      const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      CHNSS_CK(e);
      (variant == 0 ? pg.plain : pg.prof) = exec;
      pg.nodes = g_launch_count.load() - before;
      g_launch_count.store(before);
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T>
void init_precset(chnss_ctx *c, PrecSet<T> &P) {
  Arena &ar = c->ar;
  const int nl = c->nlev;
  std::vector<const Pattern *> p1s, p2s;
  std::vector<const int *> d1s, d2s;
  std::vector<const Transfer *> t1s, tvs;
  for (int l = 0; l < nl; ++l) {
    p1s.push_back(&c->lv(l).p1);
    p2s.push_back(&c->lv(l).p2);
    d1s.push_back(c->lv(l).diag1);
    d2s.push_back(c->lv(l).diag2);
    t1s.push_back(&c->lv(l).t1);
    tvs.push_back(&c->lv(l).tv);
  }
  auto vals = [&](const std::vector<double *> &v) { return std::vector<const double *>(v.begin(), v.end()); };
  // precision 2: BF16 values for the velocity hierarchy, where they cut the
  // dominant SpMV stream by 40 %.  (The P1 hierarchies save only 25 % per
  // entry and cost more CH iterations than they save: 39 -> 48 at 1024^2.)
  P.A.bf16 = c->p.precision == 2;
  // the CH / AC hierarchies reduce into partial_ch, the Oseen ones into
  // partial: the two groups assemble and solve on different streams
  P.L.init(ar, 0, false, p1s, d1s, vals(c->L), t1s, c->partial_ch);
  if (c->p.amg == 1) {
    // the paper's algebraic multigrid for the AC block (Sec. 5): smoothed
    // aggregation of the fine AC matrix, its levels set up again every step
    if (!c->amg_ac) c->amg_ac = amg_attach(c->lv(0).p1, c->AC[0], c->s);
    std::vector<const Pattern *> ap;
    std::vector<const int *> ad;
    std::vector<const double *> av, ah;
    std::vector<const Transfer *> at;
    amg_levels(c->amg_ac, ap, ad, av, at, ah);
    P.AC.hi_ext = ah;
    P.AC.init(ar, 0, false, ap, ad, av, at, c->partial_ch);
  } else {
    P.AC.init(ar, 0, false, p1s, d1s, vals(c->AC), t1s, c->partial_ch);
  }
  P.A.init(ar, 1, false, p2s, d2s, vals(c->A), tvs, c->partial);
  P.A.degree = 4;        // velocity smoothing: degree 4 on [hi / 16, hi]
  P.A.ratio = 16.0;
  P.Kp.keep_dense = true;       // a pure Laplacian: its coarsest level is not mass-dominated
  if (c->mesh->m.top_bc == 1)   // open top: Dirichlet outflow rows, non-singular
    P.Kp.init(ar, 0, false, p1s, d1s, vals(c->Kpd), t1s, c->partial);
  else
    P.Kp.init(ar, 0, true, p1s, d1s, vals(c->K1), t1s, c->partial);
  for (int sp = 0; sp < 3; ++sp) {
    std::vector<const double *> x1, x2;
    for (int l = 0; l < nl; ++l) {
      x1.push_back(c->X1[l][sp]);
      x2.push_back(c->X2[l][sp]);
    }
    P.X1[sp].init(ar, 0, false, p1s, d1s, x1, t1s, c->partial_ch);
    if (c->p.mobility_kind != 0) P.X2[sp].init(ar, 0, false, p1s, d1s, x2, t1s, c->partial_ch);
  }
  const int N1 = c->N1, nnz1 = c->lv(0).p1.nnz;
  const long nent1 = c->lv(0).p1.sell.nent;
  P.Mv = ar.alloc<T>(nent1);
  P.Apv = ar.alloc<T>(nent1);
  sell_gather<T>(c->lv(0).p1.sell, 1, c->M1[0], P.Mv, c->s);
  if (std::is_same<T, double>::value) {
    P.mdinv = reinterpret_cast<T *>(c->dinvM);
  } else {
    P.mdinv = ar.alloc<T>(N1);
    vec_convert<double, T>(N1, c->dinvM, P.mdinv, c->s);
  }
  P.mx = ar.alloc<T>(N1);
  P.mt = ar.alloc<T>(N1);
  P.mb = ar.alloc<T>(N1);
  for (MGHier<T> *h : {&P.L, &P.AC, &P.A, &P.Kp, &P.X1[0], &P.X1[1], &P.X1[2], &P.X2[0], &P.X2[1], &P.X2[2]})
    h->prof = &c->prof;
  // inner multigrid solves to a tolerance (Sec. 5) in every block that the
  // paper gives to AMG; M_p^-1 stays the fixed Chebyshev iteration
  if (c->p.inner_rtol > 0.0) {
    for (MGHier<T> *h : {&P.L, &P.AC, &P.A, &P.Kp, &P.X1[0], &P.X1[1], &P.X1[2]})
      h->enable_inner(ar, c->p.inner_rtol, c->p.inner_maxit, c->bodyq);
    if (c->p.mobility_kind != 0)
      for (int sp = 0; sp < 3; ++sp) P.X2[sp].enable_inner(ar, c->p.inner_rtol, c->p.inner_maxit, c->bodyq);
  }
  P.Kp.setup(c->s);
  for (int sp = 0; sp < 3; ++sp) P.X1[sp].setup(c->s);
  if (c->p.model == 0 && c->p.inner_rtol == 0.0) {
    // species with equal (gamma, beta) have bitwise equal X1 = tau gamma K + sqrt(tau gamma / beta) M
    // (the variable-mobility factors X2 stay per species)
    P.LB.init(ar, &P.L, 3);
    for (int sp = 0; sp < 3; ++sp) {
      int g = 0;
      while (g < P.ngroups && !(c->p.gamma[P.gmem[g][0]] == c->p.gamma[sp] && c->p.beta[P.gmem[g][0]] == c->p.beta[sp])) ++g;
      if (g == P.ngroups) ++P.ngroups;
      P.gmem[g][P.gsize[g]++] = sp;
    }
    for (int g = 0; g < P.ngroups; ++g) P.XB[g].init(ar, &P.X1[P.gmem[g][0]], P.gsize[g]);
    c->ch_batch = true;
  }
}

template <typename T>
void setup_step_precset_chac(chnss_ctx *c, PrecSet<T> &P, cudaStream_t s) {
  P.L.setup(s);
  if (c->amg_ac) amg_refresh(c->amg_ac, s);   // the AC block's SA levels from this step's matrix
  P.AC.setup(s);
  if (c->p.mobility_kind != 0)
    for (int sp = 0; sp < 3; ++sp) P.X2[sp].setup(s);
}

template <typename T>
void setup_step_precset_ns(chnss_ctx *c, PrecSet<T> &P, cudaStream_t s) {
  P.A.setup(s);
  sell_gather<T>(c->lv(0).p1.sell, 1, c->Ap, P.Apv, s);
}

void create_context(chnss_ctx *c) {
  Arena &ar = c->ar;
  const Mesh &m = c->mesh->m;
  const auto &p = c->p;
  cudaStream_t s = c->s;
  c->nlev = (int)m.lv.size();
  c->N1 = m.lv[0].N1;
  c->N2 = m.lv[0].N2;
  c->E = m.lv[0].E;
  CHNSS_CK(cudaHostAlloc(&c->pinned, 32 * sizeof(double), cudaHostAllocDefault));
  upload_reference_tensors(s);
  c->ebuf = ar.alloc<double>(144L * c->E);
  c->lbuf = ar.alloc<double>(15L * c->E);
  c->partial = ar.alloc<double>(64L * kReduceMaxBlocks);
  c->partial_ch = ar.alloc<double>(64L * kReduceMaxBlocks);
  c->sum = ar.alloc<double>(4);
  c->diag = ar.alloc<double>(kDiagQuantities + 1);
  c->srec = ar.alloc<double>(24);
  const int nl = c->nlev;
  c->M1.resize(nl); c->K1.resize(nl); c->ACb.resize(nl); c->M2v.resize(nl); c->Aconst.resize(nl);
  c->L.resize(nl); c->AC.resize(nl); c->A.resize(nl); c->X1.resize(nl); c->X2.resize(nl);
  c->vl.assign(nl, nullptr); c->mul.assign(nl, nullptr); c->phil.assign(nl, nullptr);
  for (int l = 0; l < nl; ++l) {
    const Level &L = m.lv[l];
    const Geo g = geo(L);
    const int nnz1 = L.p1.nnz, nnz2 = L.p2.nnz;
    c->M1[l] = ar.alloc<double>(nnz1);
    c->K1[l] = ar.alloc<double>(nnz1);
    c->ACb[l] = ar.alloc<double>(nnz1);
    c->L[l] = ar.alloc<double>(nnz1);
    c->AC[l] = ar.alloc<double>(nnz1);
    c->M2v[l] = ar.alloc<double>(nnz2);
    c->Aconst[l] = ar.alloc<double>(4L * nnz2);
    c->A[l] = ar.alloc<double>(4L * nnz2);
    launch_elem_p1_mass(g, c->ebuf, s);
    launch_gather(L.g_p1, 1, c->ebuf, 1.0, nullptr, 0.0, c->M1[l], s);
    launch_elem_p1_stiff(g, c->ebuf, s);
    launch_gather(L.g_p1, 1, c->ebuf, 1.0, nullptr, 0.0, c->K1[l], s);
    if (m.top_bc == 1) {
      if (l == 0) c->Kpd.assign(nl, nullptr);
      c->Kpd[l] = ar.alloc<double>(nnz1);
      vec_copy(nnz1, c->K1[l], c->Kpd[l], s);
      k_p1_top_dirichlet<<<nb(L.N1), TPB, 0, s>>>(L.n, L.p1.rowptr, L.p1.col, c->Kpd[l]);
      CHNSS_LAUNCH_CK();
    }
    // M + tau delta_v K
    vec_copy(nnz1, c->M1[l], c->ACb[l], s);
    vec_axpby(nnz1, p.tau * p.delta_v, c->K1[l], 1.0, c->ACb[l], s);
    for (int sp = 0; sp < 3; ++sp) {
      const double a = std::sqrt(p.tau * p.gamma[sp] / p.beta[sp]);
      double *x = ar.alloc<double>(nnz1);
      vec_copy(nnz1, c->M1[l], x, s);
      vec_axpby(nnz1, p.tau * p.gamma[sp], c->K1[l], a, x, s);   // tau gamma K + a M
      c->X1[l][sp] = x;
      c->X2[l][sp] = p.mobility_kind != 0 ? ar.alloc<double>(nnz1) : x;
    }
    launch_elem_p2_mass(g, c->ebuf, s);
    launch_gather(L.g_p2v, 1, c->ebuf, 1.0, nullptr, 0.0, c->M2v[l], s);
    launch_elem_ksym(g, p.eta, c->ebuf, s);
    launch_gather(L.g_ks, 4, c->ebuf, 1.0, nullptr, 0.0, c->Aconst[l], s);
    k_aconst_finish<<<nb(L.N2), TPB, 0, s>>>(L.N2, L.p2.rowptr, c->M2v[l], L.diag2, L.bnd2, 1.0 / p.tau,
                                            c->Aconst[l]);
    CHNSS_LAUNCH_CK();
    if (l > 0) {
      c->vl[l] = ar.alloc<double>(2L * L.N2);
      c->mul[l] = ar.alloc<double>(4L * L.N1);
      if (p.mobility_kind != 0) c->phil[l] = ar.alloc<double>(3L * L.N1);
    }
  }
  const Level &F = m.lv[0];
  const int nnz1 = F.p1.nnz;
  c->Apb = ar.alloc<double>(nnz1);
  c->Ap = ar.alloc<double>(nnz1);
  vec_copy(nnz1, c->M1[0], c->Apb, s);
  vec_axpby(nnz1, p.eta, c->K1[0], 1.0 / p.tau, c->Apb, s);    // M / tau + eta K
  launch_elem_bdiv(geo(F), c->ebuf, s);
  c->Bv = ar.alloc<double>(2L * m.pb.nnz);
  c->Btv = ar.alloc<double>(2L * m.pbt.nnz);
  launch_gather(m.g_b, 2, c->ebuf, 1.0, nullptr, 0.0, c->Bv, s);
  launch_gather(m.g_bt, 2, c->ebuf, 1.0, nullptr, 0.0, c->Btv, s);
  c->Bs = ar.alloc<double>(2L * m.pb.sell.nent);
  c->Bts = ar.alloc<double>(2L * m.pbt.sell.nent);
  sell_gather<double>(m.pb.sell, 2, c->Bv, c->Bs, s);
  sell_gather<double>(m.pbt.sell, 2, c->Btv, c->Bts, s);
  const long nent1 = F.p1.sell.nent;
  c->Ls = ar.alloc<double>(nent1);
  c->ACs = ar.alloc<double>(nent1);
  c->Ks = ar.alloc<double>(nent1);
  c->Ms = ar.alloc<double>(nent1);
  c->As = ar.alloc<double>(4L * F.p2.sell.nent);
  sell_gather<double>(F.p1.sell, 1, c->K1[0], c->Ks, s);
  sell_gather<double>(F.p1.sell, 1, c->M1[0], c->Ms, s);
  c->dinvM = ar.alloc<double>(c->N1);
  k_inv_diag<<<nb(c->N1), TPB, 0, s>>>(c->N1, c->M1[0], F.diag1, c->dinvM);
  CHNSS_LAUNCH_CK();
  if (p.mobility_kind != 0)
    for (int sp = 0; sp < 3; ++sp) {
      c->Kk[sp] = ar.alloc<double>(nnz1);
      c->Kks[sp] = ar.alloc<double>(nent1);
    }
  c->loads = ar.alloc<double>(5L * c->N1);
  c->G = ar.alloc<double>(2L * c->N2);
  c->fa = ar.alloc<double>(c->N1);
  c->tmp = ar.alloc<double>(c->N1);
  for (int k = 0; k < 3; ++k) {
    c->rhs[k] = ar.alloc<double>(2L * c->N1);
    c->xsol[k] = ar.alloc<double>(2L * c->N1);
  }
  c->rhs[3] = ar.alloc<double>(c->N1);
  c->xsol[3] = ar.alloc<double>(c->N1);
  c->rhs[4] = ar.alloc<double>(c->N1);
  c->xsol[4] = ar.alloc<double>(c->N1);
  c->rhs[5] = ar.alloc<double>(2L * c->N2 + c->N1);
  c->xsol[5] = ar.alloc<double>(2L * c->N2 + c->N1);
  // M_p^-1 Chebyshev coefficients (degree 5, [1/2, 2])
  {
    const double lo = 0.5, hi = 2.0, theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    std::vector<double> mc(13);
    mc[0] = 1.0 / theta;
    double rho = 1.0 / sigma;
    for (int k = 1; k <= 4; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      const double al = rn * rho, be = 2.0 * rn / delta;
      mc[1 + 3 * (k - 1)] = 1.0 + al;
      mc[2 + 3 * (k - 1)] = -al;
      mc[3 + 3 * (k - 1)] = be;
      rho = rn;
    }
    c->massc = ar.upload(mc);
  }
  const bool pairs = p.ortho == 1;
  c->kw.init(ar, p.restart, 2L * c->N2 + c->N1, c->pinned + 8, pairs);
  c->kwb[0].init(ar, p.restart, 2L * c->N1, c->pinned + 16, pairs);
  c->kwb[1].init(ar, p.restart, 2L * c->N1, c->pinned + 20, pairs);
  c->kwc0.init(ar, p.restart, 2L * c->N1, c->pinned + 24, pairs);
  c->kwa.init(ar, p.restart, c->N1, c->pinned + 28, pairs);
  c->tmp_ns = ar.alloc<double>(c->N1);
  // The Oseen group is the step's critical path (about three quarters of
  // the serial step's solve time); its stream gets the highest priority so
  // that the CH and AC groups fill the gaps it leaves (latency-bound coarse
  // levels, FP64-ALU-bound orthogonalisation, host round trips).
  int prio_low = 0, prio_high = 0;
  CHNSS_CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  for (int w = 0; w < 3; ++w)
    CHNSS_CK(cudaStreamCreateWithPriority(&c->sx[w], cudaStreamNonBlocking, w == 2 ? prio_high : prio_low));
  for (cudaStream_t &q : c->side) CHNSS_CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
  CHNSS_CK(cudaStreamCreateWithFlags(&c->bodyq, cudaStreamNonBlocking));
  CHNSS_CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  for (cudaEvent_t &e : c->ev_join) CHNSS_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CHNSS_CK(cudaEventCreateWithFlags(&c->ev_asm, cudaEventDisableTiming));
  CHNSS_CK(cudaEventCreateWithFlags(&c->ev_chac, cudaEventDisableTiming));
  for (cudaEvent_t &e : c->ev_done) CHNSS_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (p.model == 0) {   // idle members of the batched CH solves
    c->dummy_in = ar.alloc<double>(2L * c->N1);
    c->dummy_out = ar.alloc<double>(2L * c->N1);
    vec_fill(2L * c->N1, 0.0, c->dummy_in, s);
  }
  if (p.precision >= 1) {
    c->p32.reset(new PrecSet<float>());
    init_precset(c, *c->p32);
  } else {
    c->p64.reset(new PrecSet<double>());
    init_precset(c, *c->p64);
  }
  c->slots = ar.alloc<double *>(2 * kNumPrec + 6);
  CHNSS_CK(cudaStreamSynchronize(s));
  capture_graphs(c);
  CHNSS_CK(cudaStreamSynchronize(s));
}

// Coefficient fields on every level (injection), filled by assemble_prefix.
struct AsmLevels {
  std::vector<const double *> v;
  std::vector<std::array<const double *, 4>> mu;
  std::vector<std::array<const double *, 3>> ph;
};

void assemble_prefix(chnss_ctx *c, const chnss_state *st, AsmLevels &lv, cudaStream_t s) {
  const Mesh &m = c->mesh->m;
  const auto &p = c->p;
  const int nl = c->nlev;
  lv.v.assign(nl, nullptr);
  lv.mu.assign(nl, {});
  lv.ph.assign(nl, {});
  lv.v[0] = st->v;
  for (int f = 0; f < 4; ++f) lv.mu[0][f] = st->mu[f];
  for (int f = 0; f < 3; ++f) lv.ph[0][f] = st->phi[f];
  for (int l = 1; l < nl; ++l) {
    const Level &L = m.lv[l];
    const int nf = m.lv[l - 1].n;
    launch_inject_vel(nf, lv.v[l - 1], c->vl[l], s);
    lv.v[l] = c->vl[l];
    for (int f = 0; f < 4; ++f) {
      double *dst = c->mul[l] + (long)f * L.N1;
      launch_inject_p1(nf, lv.mu[l - 1][f], dst, s);
      lv.mu[l][f] = dst;
    }
    if (p.mobility_kind != 0)
      for (int f = 0; f < 3; ++f) {
        double *dst = c->phil[l] + (long)f * L.N1;
        launch_inject_p1(nf, lv.ph[l - 1][f], dst, s);
        lv.ph[l][f] = dst;
      }
  }
}

// Cahn-Hilliard / Allen-Cahn / air-potential part: C(v) on P1, the
// matching factors of the variable mobility, potential loads, right-hand
// sides, SELL copies and the P1 hierarchies' setup.  Element scratch:
// ebuf[0, 9E) and lbuf.
void assemble_chac(chnss_ctx *c, const chnss_state *st, const AsmLevels &lv, cudaStream_t s) {
  const Mesh &m = c->mesh->m;
  const auto &p = c->p;
  const int nl = c->nlev;
  for (int l = 0; l < nl; ++l) {
    const Level &L = m.lv[l];
    const Geo g = geo(L);
    // C(v) on P1: L = M + tau C, AC = M + tau delta_v K + tau C
    launch_elem_p1_conv(g, lv.v[l], nullptr, nullptr, c->ebuf, s);
    launch_gather(L.g_p1, 1, c->ebuf, p.tau, c->M1[l], 1.0, c->L[l], s);
    launch_gather(L.g_p1, 1, c->ebuf, p.tau, c->ACb[l], 1.0, c->AC[l], s);
    if (p.mobility_kind != 0)
      for (int sp = 0; sp < 3; ++sp) {
        const double a = std::sqrt(p.tau * p.gamma[sp] / p.beta[sp]);
        launch_elem_p1_wstiff(g, lv.ph[l][sp], p.gamma[sp], p.mobility_m0, c->ebuf, s);
        launch_gather(L.g_p1, 1, c->ebuf, p.tau, c->M1[l], a, c->X2[l][sp], s);   // tau K_kappa + a M
        if (l == 0) launch_gather(L.g_p1, 1, c->ebuf, 1.0, nullptr, 0.0, c->Kk[sp], s);
      }
  }
  const Level &F = m.lv[0];
  const Geo g0 = geo(F);
  // potential loads (eqn:appPotential)
  PotentialCoef pc;
  pc.model = p.model;
  pc.inv_ns = 1.0 / p.n_s;
  pc.inv_na = 1.0 / p.n_a;
  pc.chi_sa = p.chi_sa;
  pc.ln_sat_s = std::log(p.phi_sat_s);
  pc.ln_sat_a = std::log(p.phi_sat_a);
  launch_elem_loads(g0, st->phi[0], st->phi[1], st->phi[2], st->Phi_v, pc, c->lbuf, s);
  for (int f = 0; f < 5; ++f)
    launch_gather(m.g_l1, 1, c->lbuf + (long)f * c->E * 3, 1.0, nullptr, 0.0, c->loads + (long)f * c->N1, s);
  // right-hand sides
  const int N1 = c->N1, n = F.n, ref = m.ref_node;
  SpmvArgs none;
  for (int sp = 0; sp < 3; ++sp) {
    spmv_csr<double>(F.p1, c->M1[0], 1, st->phi[sp], c->rhs[sp], SPMV_PLAIN, none, s);
    const double cc = p.tau * p.gamma[sp] / p.beta[sp];
    const double sb = sp == 2 ? -p.beta[2] : 0.0;     // d phi_s / dn = j_out on Gamma_t
    k_ch_rhs_mu<<<nb(N1), TPB, 0, s>>>(N1, n, F.hx, c->loads + (long)sp * N1, st->phi[2], ref, p.evap_rate,
                                      p.phi_s_inf, sb, cc, c->rhs[sp] + N1);
    CHNSS_LAUNCH_CK();
  }
  spmv_csr<double>(F.p1, c->M1[0], 1, st->Phi_v, c->rhs[3], SPMV_PLAIN, none, s);
  k_ac_rhs<<<nb(N1), TPB, 0, s>>>(N1, n, F.hx, c->loads + 4L * N1, p.tau * p.gamma_v,
                                 p.ac_top_flux ? p.tau * p.delta_v : 0.0, st->phi[2], ref, p.evap_rate,
                                 p.phi_s_inf, c->rhs[3]);
  CHNSS_LAUNCH_CK();
  // f_a = load_a + beta_a j_out t  (d phi_a / dn = -j_out); stored as -(-1) f_a
  k_ch_rhs_mu<<<nb(N1), TPB, 0, s>>>(N1, n, F.hx, c->loads + 3L * N1, st->phi[2], ref, p.evap_rate, p.phi_s_inf,
                                    p.beta[3], -1.0, c->fa);
  CHNSS_LAUNCH_CK();
  // SELL copies of the fine operators applied by FGMRES
  sell_gather<double>(F.p1.sell, 1, c->L[0], c->Ls, s);
  sell_gather<double>(F.p1.sell, 1, c->AC[0], c->ACs, s);
  if (p.mobility_kind != 0)
    for (int sp = 0; sp < 3; ++sp) sell_gather<double>(F.p1.sell, 1, c->Kk[sp], c->Kks[sp], s);
  if (c->p32) setup_step_precset_chac(c, *c->p32, s);
  else setup_step_precset_chac(c, *c->p64, s);
}

// Oseen part: J(w) on the P2 velocity blocks of every level, A_p, the
// Korteweg load, the right-hand side, the SELL copy of A and the velocity
// hierarchy's setup.  Element scratch: ebuf[16E, 64E).
void assemble_ns(chnss_ctx *c, const chnss_state *st, const AsmLevels &lv, cudaStream_t s) {
  const Mesh &m = c->mesh->m;
  const auto &p = c->p;
  const int nl = c->nlev;
  double *eb = c->ebuf + 16L * c->E;
  for (int l = 0; l < nl; ++l) {
    const Level &L = m.lv[l];
    const Geo g = geo(L);
    // J(w) on P2 velocity blocks: A = M / tau + K_sym + J
    launch_elem_p2_conv(g, lv.v[l], lv.mu[l].data(), p.alpha, eb, s);
    launch_gather_diag2(L.g_p2v, eb, 1.0, c->Aconst[l], c->A[l], s);
  }
  const Level &F = m.lv[0];
  const Geo g0 = geo(F);
  // A_p = M / tau + eta K + J_p(w)
  launch_elem_p1_conv(g0, st->v, lv.mu[0].data(), p.alpha, eb, s);
  launch_gather(F.g_p1, 1, eb, 1.0, c->Apb, 1.0, c->Ap, s);
  if (m.top_bc == 1) {
    k_p1_top_dirichlet<<<nb(F.N1), TPB, 0, s>>>(F.n, F.p1.rowptr, F.p1.col, c->Ap);
    CHNSS_LAUNCH_CK();
  }
  // Korteweg term
  KortewegCoef kc;
  for (int f = 0; f < 4; ++f) kc.beta[f] = p.beta[f];
  kc.beta_v = p.beta_v;
  launch_elem_korteweg(g0, st->phi[0], st->phi[1], st->phi[2], st->Phi_v, kc, eb, s);
  launch_gather(m.g_l2, 2, eb, 1.0, nullptr, 0.0, c->G, s);
  // right-hand side
  const int N1 = c->N1;
  const long nv = 2L * c->N2;
  SpmvArgs none;
  spmv_csr<double>(F.p2, c->M2v[0], 2, st->v, c->rhs[5], SPMV_PLAIN, none, s);
  vec_axpby(nv, 1.0, c->G, 1.0 / p.tau, c->rhs[5], s);
  vec_fill(N1, 0.0, c->rhs[5] + nv, s);
  sell_gather<double>(F.p2.sell, 4, c->A[0], c->As, s);
  if (c->p32) setup_step_precset_ns(c, *c->p32, s);
  else setup_step_precset_ns(c, *c->p64, s);
}

// The whole per-step assembly on the context stream.
void assemble(chnss_ctx *c, const chnss_state *st) {
  cudaStream_t s = c->s;
  const int tka = c->prof.start(Profiler::ASSEMBLY, s);
  AsmLevels lv;
  assemble_prefix(c, st, lv, s);
  assemble_chac(c, st, lv, s);
  assemble_ns(c, st, lv, s);
  c->prof.stop(Profiler::ASSEMBLY, tka, s, 0.0);
  c->assembled = true;
  for (bool &d : c->ch_done) d = false;
}

int system_size(chnss_ctx *c, int sys) {
  switch (sys) {
    case CHNSS_SYS_CH_P: case CHNSS_SYS_CH_N: case CHNSS_SYS_CH_S: return 2 * c->N1;
    case CHNSS_SYS_AC: case CHNSS_SYS_MU_A: return c->N1;
    case CHNSS_SYS_NS: return 2 * c->N2 + c->N1;
    default: return -1;
  }
}

// One system on stream s with Krylov work kw and an N1 scratch vector tmp.
constexpr int kMaxCoarseCells = 25;  // largest coarsest level of a 2D mesh hierarchy (cells per side)

// device allocations of a debug entry point, freed when it returns
struct ScopedDeviceMem {
  std::vector<void *> p;
  template <typename T>
  T *get(long count) {
    void *q = nullptr;
    CHNSS_CK(cudaMalloc(&q, std::max(count, 1L) * sizeof(T)));
    p.push_back(q);
    return static_cast<T *>(q);
  }
  ~ScopedDeviceMem() {
    for (void *q : p) cudaFree(q);
  }
};

// [a, a + n) and [b, b + n) share at least one element
bool ranges_overlap(const double *a, const double *b, long n) {
  const auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  const uintptr_t len = (uintptr_t)n * sizeof(double);
  return x < y + len && y < x + len;
}

// right-hand side of the air-potential mass solve into rhs[4]:
// f_a + beta_a K phi_a^{k+1}, phi_a^{k+1} = 1 - sum of the new CH fractions
void mu_a_rhs(chnss_ctx *c, double *tmp, cudaStream_t s) {
  const int N1 = c->N1;
  const Level &F = c->lv(0);
  k_phi_a<<<nb(N1), TPB, 0, s>>>(N1, c->xsol[0], c->xsol[1], c->xsol[2], tmp);
  CHNSS_LAUNCH_CK();
  SpmvArgs none;
  spmv_csr<double>(F.p1, c->K1[0], 1, tmp, c->rhs[4], SPMV_PLAIN, none, s);
  vec_axpby(N1, 1.0, c->fa, c->p.beta[3], c->rhs[4], s);    // f_a + beta_a K phi_a^{k+1}
}

// enclosed flow: zero-mean pressure of the Oseen solution x = (v, p),
// p -= (1^T M p) / (1^T M 1); an open top fixes the pressure level itself
void ns_pressure_shift(chnss_ctx *c, double *x, double *tmp, cudaStream_t s) {
  const Mesh &m = c->mesh->m;
  if (m.top_bc != 0) return;
  const int N1 = c->N1;
  const long nv = 2L * c->N2;
  SpmvArgs none;
  spmv_csr<double>(c->lv(0).p1, c->M1[0], 1, x + nv, tmp, SPMV_PLAIN, none, s);
  vsum<double>(N1, tmp, c->sum, c->partial, s);   // c->sum, c->partial: NS only during a step
  k_shift<<<nb(N1), TPB, 0, s>>>(N1, x + nv, c->sum, m.lx * m.ly);
  CHNSS_LAUNCH_CK();
}

chnss_status solve_on(chnss_ctx *c, int sys, const double *rhs_or_null, double *x, chnss_solve_info *info,
                      cudaStream_t s, KrylovWork &kwk, double *tmp) {
  if (!c->assembled) throw Error{CHNSS_ERR_STATE, "chnss_solve before chnss_assemble"};
  const auto &p = c->p;
  const int N1 = c->N1;
  chnss_status st = CHNSS_OK;
  if (sys <= CHNSS_SYS_CH_S) {
    CHOp op(c, sys);
    st = fgmres(op, rhs_or_null ? rhs_or_null : c->rhs[sys], x, p.rtol, p.atol, p.maxit, kwk, info, s, &c->prof);
    if (x != c->xsol[sys]) vec_copy(2L * N1, x, c->xsol[sys], s);
    c->ch_done[sys] = true;
  } else if (sys == CHNSS_SYS_AC) {
    ACOp op(c);
    st = fgmres(op, rhs_or_null ? rhs_or_null : c->rhs[3], x, p.rtol, p.atol, p.maxit, kwk, info, s, &c->prof);
  } else if (sys == CHNSS_SYS_MU_A) {
    const double *b = rhs_or_null;
    if (!b) {
      if (!(c->ch_done[0] && c->ch_done[1] && c->ch_done[2]))
        throw Error{CHNSS_ERR_STATE, "MU_A needs the three CH solutions of this step"};
      mu_a_rhs(c, tmp, s);
      b = c->rhs[4];
    }
    st = pcg(c->lv(0).p1, c->M1[0], c->dinvM, b, x, 1e-12, 1000, kwk, info, s);
  } else if (sys == CHNSS_SYS_NS) {
    NSOp op(c);
    // the Oseen solve may have tolerances of its own (Sec. 5 stops it at a
    // looser relative residual than the phase-field solves)
    const double rt = p.ns_rtol > 0.0 ? p.ns_rtol : p.rtol, at = p.ns_rtol > 0.0 ? p.ns_atol : p.atol;
    st = fgmres(op, rhs_or_null ? rhs_or_null : c->rhs[5], x, rt, at, p.maxit, kwk, info, s, &c->prof);
    ns_pressure_shift(c, x, tmp, s);
  } else {
    throw Error{CHNSS_ERR_ARG, "unknown system"};
  }
  return st;
}

chnss_status solve(chnss_ctx *c, int sys, const double *rhs_or_null, double *x, chnss_solve_info *info) {
  return solve_on(c, sys, rhs_or_null, x, info, c->s, c->kw, c->tmp);
}

// The three CH systems (together when the mobility is constant), then the air
// potential, on stream s; outputs to out->phi, out->mu.
chnss_status step_ch(chnss_ctx *c, chnss_state *out, chnss_solve_info *inf, cudaStream_t s, chnss_status *st_mu) {
  const int N1 = c->N1;
  chnss_status worst = CHNSS_OK;
  auto keep = [&](chnss_status st) { if (worst == CHNSS_OK) worst = st; };
  if (c->p.model == 1) {
    // solvent-air sub-model (Sec. 5.1): no polymer / NFA; the new solvent
    // fraction is truncated to [0, 1] (eqn:truncateCH)
    for (int sp = 0; sp < 2; ++sp) {
      vec_fill(2L * N1, 0.0, c->xsol[sp], s);
      inf[sp].iters = 0;
      inf[sp].converged = 1;
      inf[sp].rel_residual = 0.0;
      inf[sp].seconds = 0.0;
    }
    keep(solve_on(c, 2, nullptr, c->xsol[2], &inf[2], s, c->kwc0, c->tmp));
    vec_clip01(N1, c->xsol[2], s);
    c->ch_done[0] = c->ch_done[1] = true;
  } else if (c->ch_batch) {
    // one batched preconditioner per Krylov tick
    CHOp o0(c, 0), o1(c, 1), o2(c, 2);
    LinearOperator *ops[3] = {&o0, &o1, &o2};
    const double *bs[3] = {c->rhs[0], c->rhs[1], c->rhs[2]};
    double *xs[3] = {c->xsol[0], c->xsol[1], c->xsol[2]};
    KrylovWork *wss[3] = {&c->kwc0, &c->kwb[0], &c->kwb[1]};
    CHBatchPrec bp(c);
    keep(fgmres_batch(3, ops, bs, xs, c->p.rtol, c->p.atol, c->p.maxit, wss, inf, bp, s, &c->prof));
    for (int sp = 0; sp < 3; ++sp) c->ch_done[sp] = true;
  } else {
    for (int sp = 0; sp < 3; ++sp) keep(solve_on(c, sp, nullptr, c->xsol[sp], &inf[sp], s, c->kwc0, c->tmp));
  }
  for (int sp = 0; sp < 3; ++sp) {
    vec_copy(N1, c->xsol[sp], out->phi[sp], s);
    vec_copy(N1, c->xsol[sp] + N1, out->mu[sp], s);
  }
  *st_mu = solve_on(c, CHNSS_SYS_MU_A, nullptr, out->mu[3], &inf[4], s, c->kwb[0], c->tmp);
  return worst;
}

chnss_status step(chnss_ctx *c, const chnss_state *in, chnss_state *out, chnss_solve_info *info) {
  chnss_solve_info loc[6];
  chnss_solve_info *inf = info ? info : loc;
  cudaStream_t s = c->s;
  const int N1 = c->N1;
  const long nv = 2L * c->N2;
  // Concurrent: after the injections on s, each group assembles its own
  // systems on its stream (the Oseen part is the longest and leads straight
  // into the Oseen solve); the AC solve waits for the CH / AC assembly.
  // Serial: the whole assembly on s first.
  AsmLevels lv;
  if (c->concurrent) {
    assemble_prefix(c, in, lv, s);
    c->assembled = true;
    for (bool &d : c->ch_done) d = false;
  } else {
    assemble(c, in);
  }
  CHNSS_CK(cudaEventRecord(c->ev_asm, s));
  chnss_status st[4] = {CHNSS_OK, CHNSS_OK, CHNSS_OK, CHNSS_OK};   // CH, AC, NS, air potential
  std::exception_ptr err[3];
  std::promise<void> chac_ready;
  std::shared_future<void> chac_done = chac_ready.get_future().share();
  int dev = 0;
  CHNSS_CK(cudaGetDevice(&dev));
  auto run = [&](int w) {
    bool handed_over = false;
    try {
      CHNSS_CK(cudaSetDevice(dev));
      cudaStream_t q = c->sx[w];
      CHNSS_CK(cudaStreamWaitEvent(q, c->ev_asm, 0));
      if (w == 0) {
        if (c->concurrent) {
          assemble_chac(c, in, lv, q);
          CHNSS_CK(cudaEventRecord(c->ev_chac, q));
          handed_over = true;
          chac_ready.set_value();
        }
        st[0] = step_ch(c, out, inf, q, &st[3]);
      } else if (w == 1) {
        if (c->concurrent) {
          chac_done.get();   // ev_chac is recorded before this returns
          CHNSS_CK(cudaStreamWaitEvent(q, c->ev_chac, 0));
        }
        st[1] = solve_on(c, CHNSS_SYS_AC, nullptr, out->Phi_v, &inf[3], q, c->kwa, nullptr);
      } else {
        if (c->concurrent) assemble_ns(c, in, lv, q);
        st[2] = solve_on(c, CHNSS_SYS_NS, nullptr, c->xsol[5], &inf[5], q, c->kw, c->tmp_ns);
        vec_copy(nv, c->xsol[5], out->v, q);
        vec_copy(N1, c->xsol[5] + nv, out->p, q);
      }
      CHNSS_CK(cudaEventRecord(c->ev_done[w], q));
    } catch (...) {
      err[w] = std::current_exception();
      if (w == 0 && c->concurrent && !handed_over) chac_ready.set_exception(std::current_exception());
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
  // the first failure in the order of the sequential step: CH, AC, air potential, NS
  for (chnss_status x : {st[0], st[1], st[3], st[2]})
    if (x != CHNSS_OK) return x;
  return CHNSS_OK;
}

// ---------------------------------------------------------------------------
// Device-driven step: the same work as step() recorded into one CUDA graph
// (assembly, the three solve groups as parallel branches, every Krylov loop
// a conditional node, the solve records copied to pinned memory at the end),
// replayed with one launch.  The CH species are solved one after the other
// (their preconditioners share the MG(M + tau C) hierarchy), each exactly as
// its own chnss_solve, so the result equals step()'s bitwise.
__global__ void k_rec_const(double *dst, double iters, double conv, double rel, double status) {
  dst[0] = iters;
  dst[1] = conv;
  dst[2] = rel;
  dst[3] = status;
}

std::array<const void *, 20> state_key(const chnss_state *in, const chnss_state *out) {
  std::array<const void *, 20> k{};
  int i = 0;
  for (const chnss_state *st : {in, out}) {
    for (int j = 0; j < 3; ++j) k[i++] = st->phi[j];
    for (int j = 0; j < 4; ++j) k[i++] = st->mu[j];
    k[i++] = st->Phi_v;
    k[i++] = st->v;
    k[i++] = st->p;
  }
  return k;
}

void record_step_body(chnss_ctx *c, const chnss_state *in, chnss_state *out) {
  const auto &p = c->p;
  cudaStream_t s = c->s;
  const int N1 = c->N1;
  const long nv = 2L * c->N2;
  AsmLevels lv;
  if (c->concurrent) {
    assemble_prefix(c, in, lv, s);
  } else {
    assemble(c, in);
  }
  CHNSS_CK(cudaEventRecord(c->ev_asm, s));
  for (cudaStream_t q : c->sx) CHNSS_CK(cudaStreamWaitEvent(q, c->ev_asm, 0));
  // CH species and the air potential
  {
    cudaStream_t q = c->sx[0];
    if (c->concurrent) {
      assemble_chac(c, in, lv, q);
      CHNSS_CK(cudaEventRecord(c->ev_chac, q));
    }
    for (int sp = 0; sp < 3; ++sp) {
      if (p.model == 1 && sp < 2) {
        vec_fill(2L * N1, 0.0, c->xsol[sp], q);
        k_rec_const<<<1, 1, 0, q>>>(c->srec + 4 * sp, 0.0, 1.0, 0.0, 0.0);
        CHNSS_LAUNCH_CK();
        continue;
      }
      CHOp op(c, sp);
      fgmres_record(op, c->rhs[sp], c->xsol[sp], p.rtol, p.atol, p.maxit, c->kwc0, q, c->rq1, c->rq2);
      krylov_record(c->kwc0, c->srec + 4 * sp, q);
    }
    if (p.model == 1) vec_clip01(N1, c->xsol[2], q);      // eqn:truncateCH
    for (int sp = 0; sp < 3; ++sp) {
      vec_copy(N1, c->xsol[sp], out->phi[sp], q);
      vec_copy(N1, c->xsol[sp] + N1, out->mu[sp], q);
    }
    mu_a_rhs(c, c->tmp, q);
    pcg_record(c->lv(0).p1, c->M1[0], c->dinvM, c->rhs[4], out->mu[3], 1e-12, 1000, c->kwb[0], q, c->rq1);
    krylov_record(c->kwb[0], c->srec + 16, q);
    CHNSS_CK(cudaEventRecord(c->ev_done[0], q));
  }
  // Allen-Cahn
  {
    cudaStream_t q = c->sx[1];
    if (c->concurrent) CHNSS_CK(cudaStreamWaitEvent(q, c->ev_chac, 0));
    ACOp op(c);
    fgmres_record(op, c->rhs[3], out->Phi_v, p.rtol, p.atol, p.maxit, c->kwa, q, c->rq1, c->rq2);
    krylov_record(c->kwa, c->srec + 12, q);
    CHNSS_CK(cudaEventRecord(c->ev_done[1], q));
  }
  // Navier-Stokes
  {
    cudaStream_t q = c->sx[2];
    if (c->concurrent) assemble_ns(c, in, lv, q);
    NSOp op(c);
    const double rt = p.ns_rtol > 0.0 ? p.ns_rtol : p.rtol, at = p.ns_rtol > 0.0 ? p.ns_atol : p.atol;
    fgmres_record(op, c->rhs[5], c->xsol[5], rt, at, p.maxit, c->kw, q, c->rq1, c->rq2);
    krylov_record(c->kw, c->srec + 20, q);
    ns_pressure_shift(c, c->xsol[5], c->tmp_ns, q);
    vec_copy(nv, c->xsol[5], out->v, q);
    vec_copy(N1, c->xsol[5] + nv, out->p, q);
    CHNSS_CK(cudaEventRecord(c->ev_done[2], q));
  }
  for (cudaEvent_t e : c->ev_done) CHNSS_CK(cudaStreamWaitEvent(s, e, 0));
  CHNSS_CK(cudaMemcpyAsync(c->srec_h, c->srec, 24 * sizeof(double), cudaMemcpyDeviceToHost, s));
}

// the private streams a step is recorded on, and the pinned solve records
void ensure_record_streams(chnss_ctx *c) {
  if (c->rq1) return;
  CHNSS_CK(cudaStreamCreateWithFlags(&c->rq0, cudaStreamNonBlocking));
  CHNSS_CK(cudaStreamCreateWithFlags(&c->rq1, cudaStreamNonBlocking));
  CHNSS_CK(cudaStreamCreateWithFlags(&c->rq2, cudaStreamNonBlocking));
  CHNSS_CK(cudaHostAlloc(&c->srec_h, 24 * sizeof(double), cudaHostAllocDefault));
}

cudaGraphExec_t step_graph_for(chnss_ctx *c, const chnss_state *in, chnss_state *out) {
  const auto key = state_key(in, out);
  for (auto &g : c->sgr)
    if (g.exec && g.key == key) return g.exec;
  ensure_record_streams(c);
  // record on the private stream (the context stream may be the legacy
  // default stream, which cannot be captured); everything that uses the
  // context stream follows it while recording
  CHNSS_CK(cudaStreamSynchronize(c->s));
  const bool prof_on = c->prof.on;
  cudaStream_t user = c->s;
  c->prof.on = false;          // no event nodes inside conditional bodies
  c->recording = true;
  c->s = c->rq0;
  cudaGraph_t graph = nullptr;
  auto restore = [&] {
    c->s = user;
    c->recording = false;
    c->prof.on = prof_on;
  };
  try {
    CHNSS_CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
  } catch (...) {
    restore();
    throw;
  }
  try {
    record_step_body(c, in, out);
  } catch (...) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(c->s, &tmp);
    if (tmp) cudaGraphDestroy(tmp);
    restore();
    throw;
  }
  const cudaError_t ec = cudaStreamEndCapture(c->s, &graph);
  restore();
  if (ec != cudaSuccess) throw Error{CHNSS_ERR_CUDA, std::string("recording the step graph: ") + cudaGetErrorString(ec)};
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) throw Error{CHNSS_ERR_CUDA, std::string("instantiating the step graph: ") + cudaGetErrorString(e)};
  auto &slot = c->sgr[c->sg_next];
  c->sg_next ^= 1;
  if (slot.exec) CHNSS_CK(cudaGraphExecDestroy(slot.exec));
  slot.exec = exec;
  slot.key = key;
  return exec;
}

void step_graph_launch(chnss_ctx *c, const chnss_state *in, chnss_state *out) {
  cudaGraphExec_t g = step_graph_for(c, in, out);
  CHNSS_CK(cudaGraphLaunch(g, c->s));
}

// after the context stream has been synchronised: the solve records
chnss_status step_graph_finish(chnss_ctx *c, chnss_solve_info *inf, double seconds) {
  c->assembled = true;
  for (bool &d : c->ch_done) d = true;
  chnss_status st[6];
  for (int i = 0; i < 6; ++i) {
    const double *r = c->srec_h + 4 * i;
    if (inf) {
      inf[i].iters = (int)r[0];
      inf[i].converged = r[1] != 0.0 ? 1 : 0;
      inf[i].rel_residual = r[2];
      inf[i].seconds = seconds;
    }
    st[i] = (chnss_status)(int)r[3];
  }
  // the first failure in the order of the sequential step: CH, AC, air potential, NS
  for (int i : {0, 1, 2, 3, 4, 5})
    if (st[i] != CHNSS_OK) return st[i];
  return CHNSS_OK;
}

chnss_status step_graph(chnss_ctx *c, const chnss_state *in, chnss_state *out, chnss_solve_info *info) {
  const auto t0 = std::chrono::steady_clock::now();
  step_graph_launch(c, in, out);
  CHNSS_CK(cudaStreamSynchronize(c->s));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return step_graph_finish(c, info, secs);
}

void check_state(const chnss_state *st) {
  if (!st) throw Error{CHNSS_ERR_ARG, "null state"};
  for (int k = 0; k < 3; ++k) if (!st->phi[k]) throw Error{CHNSS_ERR_ARG, "null phi pointer"};
  for (int k = 0; k < 4; ++k) if (!st->mu[k]) throw Error{CHNSS_ERR_ARG, "null mu pointer"};
  if (!st->Phi_v || !st->v || !st->p) throw Error{CHNSS_ERR_ARG, "null field pointer"};
}

void check_params(const chnss_params *p) {
  if (!p) throw Error{CHNSS_ERR_ARG, "null params"};
  if (!(p->tau > 0)) throw Error{CHNSS_ERR_ARG, "tau must be > 0"};
  for (int i = 0; i < 4; ++i) if (!(p->beta[i] > 0)) throw Error{CHNSS_ERR_ARG, "beta_i must be > 0"};
  for (int i = 0; i < 3; ++i) if (!(p->gamma[i] > 0)) throw Error{CHNSS_ERR_ARG, "gamma_i must be > 0"};
  if (!(p->eta > 0)) throw Error{CHNSS_ERR_ARG, "eta must be > 0"};
  if (p->restart < 1 || p->restart > 64) throw Error{CHNSS_ERR_ARG, "restart must be in [1, 64]"};
  if (p->maxit < 1) throw Error{CHNSS_ERR_ARG, "maxit must be >= 1"};
  if (p->precision < 0 || p->precision > 2) throw Error{CHNSS_ERR_ARG, "precision must be 0, 1 or 2"};
  if (p->model != 0 && p->model != 1) throw Error{CHNSS_ERR_ARG, "model must be 0 or 1"};
  if (p->model == 1 && !(p->n_s > 0 && p->n_a > 0 && p->phi_sat_s > 0 && p->phi_sat_a > 0))
    throw Error{CHNSS_ERR_ARG, "model 1 needs n_s, n_a, phi_sat_s, phi_sat_a > 0"};
  if (p->mobility_kind != 0 && p->mobility_kind != 1) throw Error{CHNSS_ERR_ARG, "mobility_kind must be 0 or 1"};
  if (!(p->inner_rtol >= 0.0 && p->inner_rtol < 1.0)) throw Error{CHNSS_ERR_ARG, "inner_rtol must be in [0, 1)"};
  if (!(p->ns_rtol >= 0.0 && p->ns_rtol < 1.0) || !(p->ns_atol >= 0.0))
    throw Error{CHNSS_ERR_ARG, "ns_rtol must be in [0, 1) and ns_atol >= 0"};
  if (p->ortho != 0 && p->ortho != 1) throw Error{CHNSS_ERR_ARG, "ortho must be 0 (FP64) or 1 (double-FP32)"};
  if (p->amg != 0 && p->amg != 1) throw Error{CHNSS_ERR_ARG, "amg must be 0 (geometric) or 1 (smoothed aggregation)"};
  if (p->inner_rtol > 0.0 && (p->inner_maxit < 1 || p->inner_maxit > 1000))
    throw Error{CHNSS_ERR_ARG, "inner_maxit must be in [1, 1000]"};
  if (!(p->rtol >= 0) || !(p->atol >= 0)) throw Error{CHNSS_ERR_ARG, "tolerances must be >= 0"};
}

chnss_status fail(chnss_ctx *c, chnss_status st, const std::string &msg) {
  if (c) c->err = msg;
  else g_last_error = msg;
  return st;
}

}  // namespace

#define ABI_TRY try {
#define ABI_CATCH(ctx)                                                      \
  }                                                                         \
  catch (const Error &e) { return fail(ctx, e.status, e.msg); }             \
  catch (const std::bad_alloc &) { return fail(ctx, CHNSS_ERR_OOM, "host allocation failed"); } \
  catch (const std::exception &e) { return fail(ctx, CHNSS_ERR_CUDA, e.what()); }

namespace chnss {
namespace debug_spmv_detail {

template <typename U>
U from_host(double v) {
  if constexpr (std::is_same<U, __nv_bfloat16>::value) return __float2bfloat16((float)v);
  else return (U)v;
}

// One SpMV of chnss_debug_spmv in vector type T with values stored as VT.
template <typename T, typename VT>
void debug_spmv_run(int layout, int mode, Pattern &P, const std::vector<int> &hmap, const std::vector<double> &cval,
                    long nx, long ny, const double *x, const double *b, const double *w, const double *dinv,
                    const double *coef, double *y) {
  ScopedDeviceMem mem;
  cudaStream_t s = nullptr;
  const int bs = layout == 0 ? 1 : layout + 1, nv = bs * bs;
  const Sell &S = P.sell;
  // values in the layout's SELL order, from the host CSR values (nv per entry)
  std::vector<double> sv;
  if (layout == 2) {
    sv.assign(9 * (size_t)S.nent, 0.0);
    for (long e = 0; e < S.nent; ++e) {
      if (hmap[e] < 0) continue;
      const long lane = e % 32, base = 9 * (e - lane) + lane;
      for (int m = 0; m < 9; ++m) sv[base + 32 * m] = cval[(size_t)hmap[e] * 9 + m];
    }
  } else {
    sv.assign((size_t)nv * S.nent, 0.0);
    for (long e = 0; e < S.nent; ++e)
      if (hmap[e] >= 0)
        for (int m = 0; m < nv; ++m) sv[(size_t)e * nv + m] = cval[(size_t)hmap[e] * nv + m];
  }
  auto up = [&](const double *h, long n, auto *tag) {
    using U = std::remove_pointer_t<decltype(tag)>;
    std::vector<U> t(n);
    for (long i = 0; i < n; ++i) t[i] = from_host<U>(h[i]);
    U *d = mem.get<U>(n);
    CHNSS_CK(cudaMemcpy(d, t.data(), n * sizeof(U), cudaMemcpyHostToDevice));
    return d;
  };
  VT *dval = up(sv.data(), (long)sv.size(), (VT *)nullptr);
  T *dx = up(x, nx, (T *)nullptr);
  T *dy = up(y, ny, (T *)nullptr);
  SpmvArgs a;
  if (mode == SPMV_RES || mode == SPMV_CHEB) a.b = up(b, ny, (T *)nullptr);
  if (mode == SPMV_CHEB) {
    a.dinv = up(dinv, ny, (T *)nullptr);
    if (w) a.w = up(w, ny, (T *)nullptr);
    double *dc = mem.get<double>(3);
    CHNSS_CK(cudaMemcpy(dc, coef, 3 * sizeof(double), cudaMemcpyHostToDevice));
    a.coef = dc;
  }
  if constexpr (std::is_same<VT, __nv_bfloat16>::value) {
    if (layout == 0) spmv_sell(P, dval, 1, dx, dy, (SpmvMode)mode, a, s);
    else if (layout == 1) spmv_sell_bsr2(P, dval, dx, dy, (SpmvMode)mode, a, s);
    else spmv_sell_bsr3(P, dval, dx, dy, (SpmvMode)mode, a, s);
  } else {
    if (layout == 0) spmv_sell<T>(P, dval, 1, dx, dy, (SpmvMode)mode, a, s);
    else if (layout == 1) spmv_sell_bsr2<T>(P, dval, dx, dy, (SpmvMode)mode, a, s);
    else spmv_sell_bsr3<T>(P, dval, dx, dy, (SpmvMode)mode, a, s);
  }
  std::vector<T> hy(ny);
  CHNSS_CK(cudaMemcpy(hy.data(), dy, ny * sizeof(T), cudaMemcpyDeviceToHost));
  for (long i = 0; i < ny; ++i) y[i] = (double)hy[i];
}

}  // namespace debug_spmv_detail
}  // namespace chnss

extern "C" {

chnss_status chnss_mesh_create(int nx, int ny, double lx, double ly, chnss_mesh_t *out) {
  return chnss_mesh_create_ex(nx, ny, lx, ly, 0, out);
}

chnss_status chnss_mesh_create_ex(int nx, int ny, double lx, double ly, int top_bc, chnss_mesh_t *out) {
  ABI_TRY
  if (!out) throw Error{CHNSS_ERR_ARG, "null output pointer"};
  if (top_bc != 0 && top_bc != 1) throw Error{CHNSS_ERR_ARG, "top_bc must be 0 or 1"};
  *out = nullptr;
  if (nx != ny) throw Error{CHNSS_ERR_ARG, "nx must equal ny"};
  // element-buffer offsets and gather counts are int: 144 E = 288 n^2 stays
  // below 2^31 up to n = 2730
  if (nx < 2 || nx % 2 != 0 || nx > 2048) throw Error{CHNSS_ERR_ARG, "n must be even and in [2, 2048]"};
  // the hierarchy halves n while it is even and >= 4; on the coarsest level
  // the pressure Laplacian keeps a dense inverse built once by one thread
  // block, with (n_c + 1)^2 rows (n_c = 25: 676 rows, about 0.1 s once; its
  // cost grows as n_c^6), so meshes must coarsen to at most 25 x 25 cells
  int nc = nx;
  while (nc % 2 == 0 && nc >= 4) nc /= 2;
  if (nc > kMaxCoarseCells)
    throw Error{CHNSS_ERR_ARG, "n = " + std::to_string(nx) + " coarsens to " + std::to_string(nc) + " x " +
                                   std::to_string(nc) + " cells; the dense coarse-level solve supports at most " +
                                   std::to_string(kMaxCoarseCells) + " x " + std::to_string(kMaxCoarseCells) +
                                   ": choose n = m 2^k with m <= " + std::to_string(kMaxCoarseCells)};
  if (!(lx > 0) || !(ly > 0)) throw Error{CHNSS_ERR_ARG, "domain lengths must be > 0"};
  std::unique_ptr<chnss_mesh> m(new chnss_mesh());
  build_mesh(m->m, nx, lx, ly, top_bc);
  *out = m.release();
  return CHNSS_OK;
  ABI_CATCH(nullptr)
}

chnss_status chnss_mesh_destroy(chnss_mesh_t mesh) {
  ABI_TRY
  if (mesh) {
    destroy_mesh(mesh->m);
    delete mesh;
  }
  return CHNSS_OK;
  ABI_CATCH(nullptr)
}

chnss_status chnss_mesh_sizes(chnss_mesh_t mesh, int *N1, int *N2, int *E, int *levels) {
  if (!mesh) return fail(nullptr, CHNSS_ERR_ARG, "null mesh");
  const Level &L = mesh->m.lv[0];
  if (N1) *N1 = L.N1;
  if (N2) *N2 = L.N2;
  if (E) *E = L.E;
  if (levels) *levels = (int)mesh->m.lv.size();
  return CHNSS_OK;
}

chnss_status chnss_ctx_create(chnss_mesh_t mesh, const chnss_params *params, void *cuda_stream, chnss_ctx_t *out) {
  ABI_TRY
  if (!out) throw Error{CHNSS_ERR_ARG, "null output pointer"};
  *out = nullptr;
  if (!mesh) throw Error{CHNSS_ERR_ARG, "null mesh"};
  check_params(params);
  std::unique_ptr<chnss_ctx> c(new chnss_ctx());
  c->mesh = mesh;
  c->p = *params;
  c->s = static_cast<cudaStream_t>(cuda_stream);
  create_context(c.get());
  *out = c.release();
  return CHNSS_OK;
  ABI_CATCH(nullptr)
}

namespace chnss {
void drop_batch_graphs(chnss_ctx *c);
}

chnss_status chnss_ctx_destroy(chnss_ctx_t ctx) {
  if (!ctx) return CHNSS_OK;
  cudaStreamSynchronize(ctx->s);
  chnss::drop_batch_graphs(ctx);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  delete ctx;
  return CHNSS_OK;
}

chnss_status chnss_assemble(chnss_ctx_t ctx, const chnss_state *state_k) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  check_state(state_k);
  assemble(ctx, state_k);
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

int chnss_system_size(chnss_ctx_t ctx, chnss_system sys) { return ctx ? system_size(ctx, sys) : -1; }

chnss_status chnss_solve(chnss_ctx_t ctx, chnss_system sys, const double *rhs_or_null, double *x_out,
                         chnss_solve_info *info) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  const int nsys = system_size(ctx, sys);
  if (nsys < 0) throw Error{CHNSS_ERR_ARG, "unknown system"};
  if (!x_out) throw Error{CHNSS_ERR_ARG, "null x_out"};
  // FGMRES reads b again at every restart; PCG reads it once, before x is
  // written, so only the mass solve may run in place
  if (rhs_or_null && ranges_overlap(rhs_or_null, x_out, nsys) && !(sys == CHNSS_SYS_MU_A && rhs_or_null == x_out))
    throw Error{CHNSS_ERR_ARG, "rhs and x_out overlap (only CHNSS_SYS_MU_A may solve in place, with rhs == x_out)"};
  const chnss_status st = solve(ctx, sys, rhs_or_null, x_out, info);
  if (st != CHNSS_OK) ctx->err = "solve did not converge cleanly (status " + std::to_string(st) + ")";
  return st;
  ABI_CATCH(ctx)
}

chnss_status chnss_step(chnss_ctx_t ctx, const chnss_state *in, chnss_state *out, chnss_solve_info *info) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  check_state(in);
  check_state(out);
  if (in->v == out->v || in->p == out->p || in->Phi_v == out->Phi_v)
    throw Error{CHNSS_ERR_ARG, "in and out states must not alias"};
  const chnss_status st = ctx->step_mode ? step_graph(ctx, in, out, info) : step(ctx, in, out, info);
  if (st != CHNSS_OK) ctx->err = "a solve of the step did not converge cleanly (status " + std::to_string(st) + ")";
  return st;
  ABI_CATCH(ctx)
}

chnss_status chnss_step_host(chnss_ctx_t ctx, const chnss_state *hin, chnss_state *hout, chnss_solve_info *info) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  check_state(hin);
  check_state(hout);
  const long N1 = ctx->N1, nv = 2L * ctx->N2;
  const long total = 9 * N1 + nv;   // phi 3, mu 4, Phi 1, p 1 (N1 each) + v
  if (!ctx->hin) {
    ctx->hin = ctx->ar.alloc<double>(total);
    ctx->hout = ctx->ar.alloc<double>(total);
  }
  auto bind = [&](double *base, chnss_state &d) {
    for (int k = 0; k < 3; ++k) d.phi[k] = base + k * N1;
    for (int k = 0; k < 4; ++k) d.mu[k] = base + (3 + k) * N1;
    d.Phi_v = base + 7 * N1;
    d.p = base + 8 * N1;
    d.v = base + 9 * N1;
  };
  chnss_state din{}, dout{};
  bind(ctx->hin, din);
  bind(ctx->hout, dout);
  cudaStream_t s = ctx->s;
  auto h2d = [&](double *d, const double *h, long n) {
    CHNSS_CK(cudaMemcpyAsync(d, h, n * sizeof(double), cudaMemcpyHostToDevice, s));
  };
  auto d2h = [&](double *h, const double *d, long n) {
    CHNSS_CK(cudaMemcpyAsync(h, d, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  };
  for (int k = 0; k < 3; ++k) h2d(din.phi[k], hin->phi[k], N1);
  for (int k = 0; k < 4; ++k) h2d(din.mu[k], hin->mu[k], N1);
  h2d(din.Phi_v, hin->Phi_v, N1);
  h2d(din.p, hin->p, N1);
  h2d(din.v, hin->v, nv);
  const chnss_status st = ctx->step_mode ? step_graph(ctx, &din, &dout, info) : step(ctx, &din, &dout, info);
  for (int k = 0; k < 3; ++k) d2h(hout->phi[k], dout.phi[k], N1);
  for (int k = 0; k < 4; ++k) d2h(hout->mu[k], dout.mu[k], N1);
  d2h(hout->Phi_v, dout.Phi_v, N1);
  d2h(hout->p, dout.p, N1);
  d2h(hout->v, dout.v, nv);
  CHNSS_CK(cudaStreamSynchronize(s));
  return st;
  ABI_CATCH(ctx)
}

chnss_status chnss_export_csr(chnss_ctx_t ctx, int which, int *nrows, int *nnz, int *rowptr, int *col, double *val) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  const Mesh &m = ctx->mesh->m;
  const Level &F = m.lv[0];
  const Pattern *P = nullptr;
  const double *dv = nullptr;
  int ncomp = 1;   // 2: B (two values per entry), 4: velocity blocks
  switch (which) {
    case 0: P = &F.p1; dv = ctx->L[0]; break;
    case 1: P = &F.p1; dv = ctx->AC[0]; break;
    case 2: P = &F.p2; dv = ctx->A[0]; ncomp = 4; break;
    case 3: P = &m.pb; dv = ctx->Bv; ncomp = 2; break;
    case 4: P = &F.p1; dv = ctx->Ap; break;
    case 5: P = &F.p1; dv = ctx->M1[0]; break;
    case 6: P = &F.p1; dv = ctx->K1[0]; break;
    default: throw Error{CHNSS_ERR_ARG, "unknown matrix id"};
  }
  if ((which == 0 || which == 1 || which == 2 || which == 4) && !ctx->assembled)
    throw Error{CHNSS_ERR_STATE, "export of a per-step matrix before chnss_assemble"};
  const int rows = ncomp == 4 ? 2 * P->nrows : P->nrows;
  const int total = P->nnz * ncomp;
  if (nrows) *nrows = rows;
  if (nnz) *nnz = total;
  if (!rowptr && !col && !val) return CHNSS_OK;
  if (!rowptr || !col || !val) throw Error{CHNSS_ERR_ARG, "export needs all three arrays"};
  std::vector<double> hv((size_t)total);
  CHNSS_CK(cudaStreamSynchronize(ctx->s));
  CHNSS_CK(cudaMemcpy(hv.data(), dv, total * sizeof(double), cudaMemcpyDeviceToHost));
  if (ncomp == 1) {
    std::copy(P->h_rowptr.begin(), P->h_rowptr.end(), rowptr);
    std::copy(P->h_col.begin(), P->h_col.end(), col);
    std::copy(hv.begin(), hv.end(), val);
  } else if (ncomp == 2) {   // B: columns 2*node + d
    int k = 0;
    rowptr[0] = 0;
    for (int r = 0; r < P->nrows; ++r) {
      for (int q = P->h_rowptr[r]; q < P->h_rowptr[r + 1]; ++q)
        for (int d = 0; d < 2; ++d) { col[k] = 2 * P->h_col[q] + d; val[k] = hv[2L * q + d]; ++k; }
      rowptr[r + 1] = k;
    }
  } else {                   // velocity blocks -> scalar rows 2*node + c
    int k = 0;
    rowptr[0] = 0;
    for (int r = 0; r < P->nrows; ++r)
      for (int cc = 0; cc < 2; ++cc) {
        for (int q = P->h_rowptr[r]; q < P->h_rowptr[r + 1]; ++q)
          for (int d = 0; d < 2; ++d) { col[k] = 2 * P->h_col[q] + d; val[k] = hv[4L * q + cc * 2 + d]; ++k; }
        rowptr[2 * r + cc + 1] = k;
      }
  }
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

chnss_status chnss_debug_cgs2(int arith, long n, int k, const double *V, long ld, const double *w, double *h,
                              double *vout) {
  ABI_TRY
  if (arith != 0 && arith != 1) throw Error{CHNSS_ERR_ARG, "arith must be 0 (FP64) or 1 (double-FP32)"};
  if (n < 1 || k < 1 || k > 31 || ld < n) throw Error{CHNSS_ERR_ARG, "need n >= 1, 1 <= k <= 31, ld >= n"};
  if (!V || !w || !h || !vout) throw Error{CHNSS_ERR_ARG, "null argument"};
  if (ld % 2 != 0) throw Error{CHNSS_ERR_ARG, "ld must be even (16-byte aligned basis vectors)"};
  ScopedDeviceMem mem;
  cudaStream_t s = nullptr;   // the legacy stream, synchronised before returning
  double *wc = mem.get<double>(n), *h1 = mem.get<double>(k + 1), *h2 = mem.get<double>(k + 1);
  double *partial = mem.get<double>(64L * kReduceMaxBlocks), *hn = mem.get<double>(1);
  CHNSS_CK(cudaMemcpyAsync(wc, w, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<double> hh(2 * k + 1);
  auto finish_norm = [&]() {
    CHNSS_CK(cudaMemcpyAsync(hh.data(), h1, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHNSS_CK(cudaMemcpyAsync(hh.data() + k, h2, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHNSS_CK(cudaStreamSynchronize(s));
    double sq = hh[2 * k];
    for (int j = 0; j < k; ++j) sq -= hh[k + j] * hh[k + j];
    const double nrm = std::sqrt(std::max(sq, 0.0));
    CHNSS_CK(cudaMemcpyAsync(hn, &nrm, sizeof(double), cudaMemcpyHostToDevice, s));
    CHNSS_CK(cudaStreamSynchronize(s));
  };
  if (arith == 0) {
    cgs2_dots(n, V, ld, k, wc, h1, partial, s);
    cgs2_update_dots(n, V, ld, k, h1, wc, h2, partial, s);
    finish_norm();
    cgs2_update_scale(n, V, ld, k, h2, wc, hn, vout, s);
  } else {
    float2 *V2 = mem.get<float2>((long)k * ld), *v2 = mem.get<float2>(n);
    double *one = mem.get<double>(1), *tmp = mem.get<double>(n);
    const double o = 1.0;
    CHNSS_CK(cudaMemcpyAsync(one, &o, sizeof(double), cudaMemcpyHostToDevice, s));
    for (int j = 0; j < k; ++j) dfgs_first(n, V + (long)j * ld, one, V2 + (long)j * ld, tmp, s);
    dfgs_dots(n, V2, ld, k, wc, h1, partial, s);
    dfgs_update_dots(n, V2, ld, k, h1, wc, h2, partial, s);
    finish_norm();
    dfgs_update_scale(n, V2, ld, k, h2, wc, hn, v2, vout, s);
  }
  CHNSS_CK(cudaStreamSynchronize(s));
  CHNSS_CK(cudaGetLastError());
  std::copy(hh.begin(), hh.end(), h);
  return CHNSS_OK;
  ABI_CATCH(nullptr)
}


chnss_status chnss_debug_spmv(int layout, int precision, int mode, int nrows, int ncols, const int *rowptr,
                              const int *col, const double *val, const double *x, const double *b, const double *w,
                              const double *dinv, const double *coef, double *y, int *warps_per_slice) {
  ABI_TRY
  if (layout < 0 || layout > 2) throw Error{CHNSS_ERR_ARG, "layout must be 0 (scalar), 1 (2x2) or 2 (3x3)"};
  if (precision < 0 || precision > 2) throw Error{CHNSS_ERR_ARG, "precision must be 0, 1 or 2"};
  if (mode < 0 || mode > 3) throw Error{CHNSS_ERR_ARG, "mode must be 0 (plain), 1 (residual), 2 (add), 3 (Chebyshev)"};
  if (nrows < 1 || ncols < 1 || !rowptr || !col || !val || !x || !y) throw Error{CHNSS_ERR_ARG, "bad size or null"};
  if ((mode == 1 || mode == 3) && !b) throw Error{CHNSS_ERR_ARG, "modes 1 and 3 need b"};
  if (mode == 3 && (!dinv || !coef)) throw Error{CHNSS_ERR_ARG, "mode 3 needs dinv and coef"};
  if (mode == 3 && nrows != ncols) throw Error{CHNSS_ERR_ARG, "mode 3 needs a square matrix"};
  if (layout > 0 && nrows != ncols) throw Error{CHNSS_ERR_ARG, "block layouts need a square node pattern"};
  Pattern P;
  P.nrows = nrows;
  P.ncols = ncols;
  P.h_rowptr.assign(rowptr, rowptr + nrows + 1);
  if (P.h_rowptr[0] != 0) throw Error{CHNSS_ERR_ARG, "rowptr[0] must be 0"};
  for (int r = 0; r < nrows; ++r)
    if (P.h_rowptr[r + 1] < P.h_rowptr[r]) throw Error{CHNSS_ERR_ARG, "rowptr must be non-decreasing"};
  P.nnz = P.h_rowptr[nrows];
  P.h_col.assign(col, col + P.nnz);
  for (int k = 0; k < P.nnz; ++k)
    if (P.h_col[k] < 0 || P.h_col[k] >= ncols) throw Error{CHNSS_ERR_ARG, "column out of range"};
  const int bs = layout == 0 ? 1 : layout + 1;
  Arena ar;
  std::vector<int> hmap;
  upload_pattern(ar, P, &hmap);
  std::vector<double> cval(val, val + (size_t)P.nnz * bs * bs);
  const long nx = (long)bs * ncols, ny = (long)bs * nrows;
  if (warps_per_slice)
    *warps_per_slice = layout == 0 ? (P.sell.wmax <= 8 ? 1 : sell_split(P.sell))
                                   : (layout == 1 ? sell_warps_bsr2(P.sell) : sell_warps_bsr3(P.sell));
  using debug_spmv_detail::debug_spmv_run;
  if (precision == 0) debug_spmv_run<double, double>(layout, mode, P, hmap, cval, nx, ny, x, b, w, dinv, coef, y);
  else if (precision == 1) debug_spmv_run<float, float>(layout, mode, P, hmap, cval, nx, ny, x, b, w, dinv, coef, y);
  else debug_spmv_run<float, __nv_bfloat16>(layout, mode, P, hmap, cval, nx, ny, x, b, w, dinv, coef, y);
  CHNSS_CK(cudaDeviceSynchronize());
  CHNSS_CK(cudaGetLastError());
  return CHNSS_OK;
  ABI_CATCH(nullptr)
}

chnss_status chnss_export_rhs(chnss_ctx_t ctx, chnss_system sys, double *host_out) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  const int n = system_size(ctx, sys);
  if (n < 0 || !host_out) throw Error{CHNSS_ERR_ARG, "bad system or null output"};
  if (!ctx->assembled) throw Error{CHNSS_ERR_STATE, "export_rhs before chnss_assemble"};
  const double *src = sys == CHNSS_SYS_MU_A ? ctx->rhs[4] : ctx->rhs[sys <= 2 ? sys : (sys == 3 ? 3 : 5)];
  CHNSS_CK(cudaStreamSynchronize(ctx->s));
  CHNSS_CK(cudaMemcpy(host_out, src, n * sizeof(double), cudaMemcpyDeviceToHost));
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

chnss_status chnss_profile_enable(chnss_ctx_t ctx, int on) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  CHNSS_CK(cudaStreamSynchronize(ctx->s));
  ctx->prof.reset();
  ctx->prof.on = on != 0;
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

chnss_status chnss_profile_read(chnss_ctx_t ctx, chnss_profile *out) {
  if (!ctx || !out) return fail(ctx, CHNSS_ERR_ARG, "null argument");
  ABI_TRY
  CHNSS_CK(cudaStreamSynchronize(ctx->s));
  std::memset(out, 0, sizeof(*out));
  out->launches = g_launch_count.load();
  out->nkinds = Profiler::NKINDS;
  for (int k = 0; k < Profiler::NKINDS; ++k) {
    std::strncpy(out->name[k], Profiler::name(k), sizeof(out->name[k]) - 1);
    out->kind_launches[k] = ctx->prof.rec[k].launches;
    out->kind_ms[k] = ctx->prof.elapsed_ms(k);
    out->kind_bytes[k] = ctx->prof.rec[k].bytes;
    out->kind_flops[k] = ctx->prof.rec[k].flops;
  }
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

chnss_status chnss_inner_stats_read(chnss_ctx_t ctx, int reset, chnss_inner_stats *out) {
  if (!ctx || !out) return fail(ctx, CHNSS_ERR_ARG, "null argument");
  ABI_TRY
  std::memset(out, 0, sizeof(*out));
  auto read = [&](auto &P) {
    using H = std::remove_reference_t<decltype(P.L)>;
    H *hs[CHNSS_INNER_BLOCKS] = {&P.L, &P.AC, &P.A, &P.Kp, &P.X1[0], &P.X1[1], &P.X1[2], &P.X2[0], &P.X2[1], &P.X2[2]};
    for (int i = 0; i < CHNSS_INNER_BLOCKS; ++i)
      hs[i]->inner_stats(reset != 0, &out->solves[i], &out->cycles[i], &out->last_rel_residual[i], ctx->s);
  };
  if (ctx->p32) read(*ctx->p32);
  else read(*ctx->p64);
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

const char *chnss_last_error(chnss_ctx_t ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Mass-matrix solve without allocation.  Its work vectors (r, z, p, q), the
// reduction partials and the device scalars live in a file-scope device array
// sized for meshes up to 256 x 256; every GPU that loads the library holds
// this array until the process exits.  Host code cannot use the array's name
// as a device address, so each device looks the address up once with
// cudaGetSymbolAddress (on the first call with that device current).
namespace {

constexpr int kNoAllocMaxN1 = 257 * 257;             // P1 nodes of a 256 x 256 mesh
constexpr long kNoAllocPartials = kReduceMaxBlocks;  // reduction blocks (reduce_blocks cap)
constexpr long kNoAllocScalars = 16;
constexpr long kNoAllocDoubles = 4L * kNoAllocMaxN1 + kNoAllocPartials + kNoAllocScalars;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

double *g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;

double *noalloc_scratch_address() {
  int dev = 0;
  CHNSS_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) throw Error{CHNSS_ERR_ARG, "device index out of range"};
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      throw Error{CHNSS_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e)};
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  return g_noalloc_addr[dev];
}

// Jacobi PCG on M x = b (the MU_A solve's pcg(): rtol 1e-12, x0 = 0) with a
// work view whose vectors, scalars and partials all point into the scratch
// array, and the context's own pinned host slot for the scalar reads.
chnss_status mass_solve_noalloc(chnss_ctx *c, const double *b, double *x, chnss_solve_info *info) {
  const Pattern &P = c->lv(0).p1;
  const long n = P.nrows;
  double *base = noalloc_scratch_address();
  KrylovWork view;                       // no storage of its own
  view.nmax = n;
  view.w = base;                         // r
  view.V = base + n;                     // z, p, q
  view.partial = base + 4L * kNoAllocMaxN1;
  view.sc = view.partial + kNoAllocPartials;
  view.hstat = c->pinned + 12;
  return pcg(P, c->M1[0], c->dinvM, b, x, 1e-12, 1000, view, info, c->s);
}

}  // namespace

extern "C" chnss_status chnss_mass_solve_noalloc(chnss_ctx_t ctx, const double *rhs, double *x_out,
                                                 chnss_solve_info *info) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  if (!rhs || !x_out) throw Error{CHNSS_ERR_ARG, "null rhs or x_out"};
  if (rhs != x_out && ranges_overlap(rhs, x_out, ctx->N1))
    throw Error{CHNSS_ERR_ARG, "rhs and x_out overlap without being the same array"};
  if (ctx->N1 > kNoAllocMaxN1)
    throw Error{CHNSS_ERR_ARG, "chnss_mass_solve_noalloc supports at most " + std::to_string(kNoAllocMaxN1) +
                                   " P1 nodes (a 256 x 256 mesh); this mesh has " + std::to_string(ctx->N1)};
  return mass_solve_noalloc(ctx, rhs, x_out, info);
  ABI_CATCH(ctx)
}

// ---------------------------------------------------------------------------
// Adjoint step: for each solve x = A(u)^-1 b(u) of the step, given the
// adjoint xbar of its solution, y = A^-T xbar (FGMRES on the transposed
// operator, preconditioned by the forward preconditioner), then
// ubar += (db/du)^T y - (d(A(u) x)/du)^T y (adjoint element kernels).
namespace {

constexpr double kAdjointRtol = 1e-12;

__global__ void k_top_load_vec(int N1, int n, double hx, double *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < N1) out[i] = top_load(i, n, hx);
}
__global__ void k_mask_velocity(int N2, const double *in, const int *bnd, double *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= N2) return;
  out[2 * i] = bnd[i] ? 0.0 : in[2 * i];
  out[2 * i + 1] = bnd[i] ? 0.0 : in[2 * i + 1];
}
// out = lp - m * sum(lp) / area (transpose of the zero-mean pressure shift)
__global__ void k_mean_shift_T(int N1, const double *lp, const double *m, const double *sum, double area, double *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < N1) out[i] = lp[i] - m[i] * (*sum) / area;
}
__global__ void k_add_at(double *x, int idx, double v) { x[idx] += v; }

struct CHOpT : LinearOperator {   // [[L^T, a21 K], [a12 K12, a22 M]]
  chnss_ctx *c;
  int sp;
  CHOpT(chnss_ctx *c_, int sp_) : c(c_), sp(sp_) {}
  long size() const override { return 2L * c->N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const auto &p = c->p;
    const double tau = p.tau, g = p.gamma[sp], b = p.beta[sp];
    // y1 = L^T x1 + tau g K x2 ; y2 = (var ? tau K_kappa : tau g K) x1 - (tau g / b) M x2
    // (K, K_kappa symmetric: the transposed blocks are the forward ones swapped)
    if (p.mobility_kind != 0)
      spmv_sell_ch(c->lv(0).p1, c->LsT, c->Kks[sp], c->Ks, c->Ms, tau * g, tau, -tau * g / b, x, y, s);
    else
      spmv_sell_ch(c->lv(0).p1, c->LsT, c->Ks, nullptr, c->Ms, tau * g, tau * g, -tau * g / b, x, y, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec(c, sp, r, z, s); }
  void after_sync() override { harvest_probes(c, sp); }
};

struct ACOpT : LinearOperator {
  chnss_ctx *c;
  explicit ACOpT(chnss_ctx *c_) : c(c_) {}
  long size() const override { return c->N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    SpmvArgs none;
    spmv_sell<double>(c->lv(0).p1, c->ACsT, 1, x, y, SPMV_PLAIN, none, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec(c, 3, r, z, s); }
  void after_sync() override { harvest_probes(c, 3); }
};

struct NSOpT : LinearOperator {   // [[A^T, B^T], [B, 0]]
  chnss_ctx *c;
  explicit NSOpT(chnss_ctx *c_) : c(c_) {}
  long size() const override { return 2L * c->N2 + c->N1; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    const long nv = 2L * c->N2;
    SpmvArgs none;
    spmv_sell_bsr2<double>(c->lv(0).p2, c->AsT, x, y, SPMV_PLAIN, none, s);
    spmv_sell_bt_add(c->mesh->m.pbt, c->Bts, x + nv, y, s);
    spmv_sell_b(c->mesh->m.pb, c->Bs, x, y + nv, s);
  }
  void precond(const double *r, double *z, cudaStream_t s) override { run_prec(c, 4, r, z, s); }
  void after_sync() override { harvest_probes(c, 4); }
};

void adjoint_alloc(chnss_ctx *c) {
  if (c->LsT) return;
  Arena &ar = c->ar;
  const Level &F = c->lv(0);
  const long N1 = c->N1, nmax = 2L * c->N2 + c->N1;
  c->LsT = ar.alloc<double>(F.p1.sell.nent);
  c->ACsT = ar.alloc<double>(F.p1.sell.nent);
  c->AsT = ar.alloc<double>(4L * F.p2.sell.nent);
  c->topv = ar.alloc<double>(N1);
  c->mvec = ar.alloc<double>(N1);
  c->arhs = ar.alloc<double>(nmax);
  c->ay = ar.alloc<double>(nmax);
  c->alam = ar.alloc<double>(3 * N1);
  c->az = ar.alloc<double>(N1);
  c->atmp = ar.alloc<double>(N1);
  c->atv = ar.alloc<double>(2L * c->N2);
  for (double *&w : c->alw) w = ar.alloc<double>(N1);
  c->ay_ac = ar.alloc<double>(N1);
  c->aPhi = ar.alloc<double>(N1);
  c->v_ac = ar.alloc<double>(2L * c->N2);
  c->arhs_ch = ar.alloc<double>(2L * N1);
  c->ay_ch = ar.alloc<double>(2L * N1);
  c->atmp_ch = ar.alloc<double>(N1);
  c->aphi = ar.alloc<double>(3L * N1);
  c->v_ch = ar.alloc<double>(2L * c->N2);
  c->adots = ar.alloc<double>(32);
  k_top_load_vec<<<nb(N1), TPB, 0, c->s>>>((int)N1, F.n, F.hx, c->topv);
  CHNSS_LAUNCH_CK();
  vec_fill(N1, 1.0, c->atmp, c->s);
  SpmvArgs none;
  spmv_csr<double>(F.p1, c->M1[0], 1, c->atmp, c->mvec, SPMV_PLAIN, none, c->s);
}

// out += alpha * (per-element P1 contributions gathered to nodes)
void gather_p1_add(chnss_ctx *c, const double *buf, double alpha, double *out, cudaStream_t s) {
  launch_gather(c->mesh->m.g_l1, 1, buf, alpha, out, 1.0, out, s);
}

chnss_status adjoint_step(chnss_ctx *c, const chnss_state *stk, const chnss_state *st1, const chnss_state *lam,
                          chnss_state *out, double *grad, chnss_solve_info *info) {
  const auto &p = c->p;
  const bool var = p.mobility_kind != 0;
  adjoint_alloc(c);
  assemble(c, stk);
  cudaStream_t s = c->s;
  const Mesh &m = c->mesh->m;
  const Level &F = m.lv[0];
  const Geo g0 = geo(F);
  const int N1 = c->N1, E = c->E;
  const long nv = 2L * c->N2;
  const double tau = p.tau;
  chnss_solve_info loc[6];
  chnss_solve_info *inf = info ? info : loc;
  SpmvArgs none;
  // transposed fine operators
  sell_gather_transposed(F.p1.sell, 1, c->L[0], c->LsT, s);
  sell_gather_transposed(F.p1.sell, 1, c->AC[0], c->ACsT, s);
  sell_gather_transposed(F.p2.sell, 4, c->A[0], c->AsT, s);
  for (int k = 0; k < 3; ++k) vec_fill(N1, 0.0, out->phi[k], s);
  for (int k = 0; k < 4; ++k) vec_fill(N1, 0.0, out->mu[k], s);
  vec_fill(N1, 0.0, out->Phi_v, s);
  vec_fill(nv, 0.0, out->v, s);
  vec_fill(N1, 0.0, out->p, s);
  vec_fill(32, 0.0, c->adots, s);
  double *D = c->adots;
  CHNSS_CK(cudaEventRecord(c->ev_asm, s));
  // Three independent groups, as in the forward step: Navier-Stokes, Allen-
  // Cahn, air potential -> Cahn-Hilliard.  Each has its own Krylov work,
  // scratch, slice of ebuf and accumulators; the groups' contributions to
  // the shared adjoints are summed on s after the join in a fixed order, so
  // the result does not depend on whether the groups overlap.
  auto group_ns = [&](cudaStream_t q) -> chnss_status {
    KrylovWork &kw = c->kw;
    k_mask_velocity<<<nb(c->N2), TPB, 0, q>>>(c->N2, lam->v, F.bnd2, c->arhs);
    CHNSS_LAUNCH_CK();
    if (m.top_bc == 0) {   // transpose of the zero-mean pressure shift
      vsum<double>(N1, lam->p, c->sum, kw.partial, q);
      k_mean_shift_T<<<nb(N1), TPB, 0, q>>>(N1, lam->p, c->mvec, c->sum, m.lx * m.ly, c->arhs + nv);
      CHNSS_LAUNCH_CK();
    } else {               // open top: the pressure level is fixed by the outflow, no shift
      vec_copy(N1, lam->p, c->arhs + nv, q);
    }
    NSOpT op(c);
    const chnss_status st = fgmres(op, c->arhs, c->ay, kAdjointRtol, 0.0, p.maxit, kw, &inf[5], q, &c->prof);
    const double *yv = c->ay;
    spmv_csr<double>(F.p2, c->M2v[0], 2, yv, c->atv, SPMV_PLAIN, none, q);
    vec_axpby(nv, 1.0 / tau, c->atv, 1.0, out->v, q);                       // (M_v / tau)^T y_v
    KortewegCoef kc;
    for (int f = 0; f < 4; ++f) kc.beta[f] = p.beta[f];
    kc.beta_v = p.beta_v;
    launch_adj_korteweg(g0, stk->phi[0], stk->phi[1], stk->phi[2], stk->Phi_v, yv, kc, c->lbuf, q);
    for (int f = 0; f < 3; ++f) gather_p1_add(c, c->lbuf + (long)f * E * 3, 1.0, out->phi[f], q);
    gather_p1_add(c, c->lbuf + 3L * E * 3, 1.0, out->Phi_v, q);
    launch_adj_conv_p2(g0, st1->v, yv, c->ebuf, c->ebuf + 12L * E, q);
    launch_gather(m.g_l2, 2, c->ebuf, -1.0, out->v, 1.0, out->v, q);       // - (dJ(w)x/dv)^T y
    launch_gather(m.g_l1, 1, c->ebuf + 12L * E, 1.0, nullptr, 0.0, c->atmp, q);
    for (int i = 0; i < 4; ++i) vec_axpby(N1, -p.alpha[i], c->atmp, 1.0, out->mu[i], q);
    return st;
  };
  auto group_ac = [&](cudaStream_t q) -> chnss_status {
    double *eb = c->ebuf + 16L * E;
    ACOpT op(c);
    const chnss_status st = fgmres(op, lam->Phi_v, c->ay_ac, kAdjointRtol, 0.0, p.maxit, c->kwa, &inf[3], q, &c->prof);
    spmv_csr<double>(F.p1, c->M1[0], 1, c->ay_ac, c->aPhi, SPMV_PLAIN, none, q);
    vec_fill(N1, 0.0, c->alw[4], q);
    vec_axpby(N1, -tau * p.gamma_v, c->ay_ac, 0.0, c->alw[4], q);
    launch_adj_conv_p1(g0, st1->Phi_v, c->ay_ac, eb, q);
    launch_gather(m.g_l2, 2, eb, -tau, nullptr, 0.0, c->v_ac, q);
    dot<double>(N1, c->topv, c->ay_ac, D + 1, c->kwa.partial, q);
    return st;
  };
  auto group_ch = [&](cudaStream_t q, chnss_status *st_mu) -> chnss_status {
    double *eb = c->ebuf + 32L * E;
    double *tmp = c->atmp_ch;
    // air potential
    *st_mu = pcg(F.p1, c->M1[0], c->dinvM, lam->mu[3], c->az, kAdjointRtol, 1000, c->kwb[0], &inf[4], q);
    spmv_csr<double>(F.p1, c->K1[0], 1, c->az, tmp, SPMV_PLAIN, none, q);
    for (int i = 0; i < 3; ++i) {
      vec_copy(N1, lam->phi[i], c->alam + (long)i * N1, q);
      vec_axpby(N1, -p.beta[3], tmp, 1.0, c->alam + (long)i * N1, q);
    }
    vec_copy(N1, c->az, c->alw[3], q);
    dot<double>(N1, c->topv, c->az, D + 0, c->kwb[0].partial, q);
    // Cahn-Hilliard
    chnss_status worst = CHNSS_OK;
    vec_fill(nv, 0.0, c->v_ch, q);
    KrylovWork &kw = c->kwc0;
    for (int i = 0; i < 3; ++i) {
      vec_copy(N1, c->alam + (long)i * N1, c->arhs_ch, q);
      vec_copy(N1, lam->mu[i], c->arhs_ch + N1, q);
      {
        CHOpT op(c, i);
        const chnss_status st = fgmres(op, c->arhs_ch, c->ay_ch, kAdjointRtol, 0.0, p.maxit, kw, &inf[i], q, &c->prof);
        if (worst == CHNSS_OK) worst = st;
      }
      const double *y1 = c->ay_ch, *y2 = c->ay_ch + N1;
      const double cc = tau * p.gamma[i] / p.beta[i];
      spmv_csr<double>(F.p1, c->M1[0], 1, y1, c->aphi + (long)i * N1, SPMV_PLAIN, none, q);
      if (var) {   // - tau (d K_kappa(phi_i^k) / d phi_i)^T (y1, mu_i')
        launch_adj_wstiff(g0, stk->phi[i], p.gamma[i], st1->mu[i], y1, eb, q);
        launch_gather(m.g_l1, 1, eb, -tau, c->aphi + (long)i * N1, 1.0, c->aphi + (long)i * N1, q);
      }
      vec_fill(N1, 0.0, c->alw[i], q);
      vec_axpby(N1, -cc, y2, 0.0, c->alw[i], q);
      launch_adj_conv_p1(g0, st1->phi[i], y1, eb, q);
      launch_gather(m.g_l2, 2, eb, -tau, c->v_ch, 1.0, c->v_ch, q);
      double *d = D + 4 + 5 * i;
      dot<double>(N1, c->loads + (long)i * N1, y2, d + 0, kw.partial, q);    // F_i . y2
      dot<double>(N1, c->topv, y2, d + 1, kw.partial, q);                     // t . y2
      // y1 . K mu' (constant mobility) or y1 . K_kappa mu' (divided by gamma_i on the host)
      spmv_csr<double>(F.p1, var ? c->Kk[i] : c->K1[0], 1, st1->mu[i], tmp, SPMV_PLAIN, none, q);
      dot<double>(N1, y1, tmp, d + 2, kw.partial, q);
      spmv_csr<double>(F.p1, c->K1[0], 1, st1->phi[i], tmp, SPMV_PLAIN, none, q);
      dot<double>(N1, y2, tmp, d + 3, kw.partial, q);                         // y2 . K phi'
      spmv_csr<double>(F.p1, c->M1[0], 1, st1->mu[i], tmp, SPMV_PLAIN, none, q);
      dot<double>(N1, y2, tmp, d + 4, kw.partial, q);                         // y2 . M mu'
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
  // ---- the groups' contributions to the shared adjoints ---------------------
  vec_axpby(nv, 1.0, c->v_ac, 1.0, out->v, s);
  vec_axpby(nv, 1.0, c->v_ch, 1.0, out->v, s);
  vec_axpby(N1, 1.0, c->aPhi, 1.0, out->Phi_v, s);
  for (int i = 0; i < 3; ++i) vec_axpby(N1, 1.0, c->aphi + (long)i * N1, 1.0, out->phi[i], s);
  // ---- potential loads ------------------------------------------------------
  const double *lw[5] = {c->alw[0], c->alw[1], c->alw[2], c->alw[3], c->alw[4]};
  launch_adj_loads(g0, stk->phi[0], stk->phi[1], stk->phi[2], stk->Phi_v, lw, c->lbuf, s);
  for (int f = 0; f < 3; ++f) gather_p1_add(c, c->lbuf + (long)f * E * 3, 1.0, out->phi[f], s);
  gather_p1_add(c, c->lbuf + 3L * E * 3, 1.0, out->Phi_v, s);
  // ---- parameter gradients --------------------------------------------------
  double h[24], phis_ref = 0.0;
  CHNSS_CK(cudaMemcpyAsync(h, D, 24 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNSS_CK(cudaMemcpyAsync(&phis_ref, stk->phi[2] + m.ref_node, sizeof(double), cudaMemcpyDeviceToHost, s));
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
  k_add_at<<<1, 1, 0, s>>>(out->phi[2], m.ref_node, jbar * p.evap_rate);
  CHNSS_LAUNCH_CK();
  if (grad) {
    grad[0] += jbar * (phis_ref - p.phi_s_inf);
    grad[1] += gbar;
  }
  return worst;
}

}  // namespace

extern "C" chnss_status chnss_adjoint_step(chnss_ctx_t ctx, const chnss_state *state_k, const chnss_state *state_k1,
                                           const chnss_state *adj_k1, chnss_state *adj_k, double *grad_params,
                                           chnss_solve_info *info) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  if (ctx->p.model != 0) return fail(ctx, CHNSS_ERR_ARG, "the adjoint step covers model 0 only");
  ABI_TRY
  check_state(state_k);
  check_state(state_k1);
  check_state(adj_k1);
  check_state(adj_k);
  const chnss_status st = adjoint_step(ctx, state_k, state_k1, adj_k1, adj_k, grad_params, info);
  if (st != CHNSS_OK) ctx->err = "an adjoint solve did not converge cleanly (status " + std::to_string(st) + ")";
  return st;
  ABI_CATCH(ctx)
}

extern "C" chnss_status chnss_objective(chnss_ctx_t ctx, const double *phi_p, double *J, double *grad_phi_p) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  if (!phi_p || !J) throw Error{CHNSS_ERR_ARG, "null phi_p or J"};
  adjoint_alloc(ctx);
  const Level &F = ctx->lv(0);
  SpmvArgs none;
  spmv_csr<double>(F.p1, ctx->K1[0], 1, phi_p, ctx->atmp, SPMV_PLAIN, none, ctx->s);
  dot<double>(ctx->N1, phi_p, ctx->atmp, ctx->adots + 30, ctx->partial, ctx->s);
  if (grad_phi_p) {
    vec_fill(ctx->N1, 0.0, grad_phi_p, ctx->s);
    vec_axpby(ctx->N1, 2.0, ctx->atmp, 0.0, grad_phi_p, ctx->s);
  }
  CHNSS_CK(cudaMemcpyAsync(J, ctx->adots + 30, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CHNSS_CK(cudaStreamSynchronize(ctx->s));
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

extern "C" chnss_status chnss_diagnostics(chnss_ctx_t ctx, const chnss_state *state, chnss_diag *out) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  if (!out) throw Error{CHNSS_ERR_ARG, "null output"};
  check_state(state);
  const chnss_params &p = ctx->p;
  const Mesh &m = ctx->mesh->m;
  cudaStream_t s = ctx->s;
  DiagArgs d;
  d.pp = state->phi[0];
  d.pn = state->phi[1];
  d.ps = state->phi[2];
  d.Ph = state->Phi_v;
  d.p = state->p;
  d.v = state->v;
  for (int i = 0; i < 4; ++i) d.beta[i] = p.beta[i];
  d.beta_v = p.beta_v;
  d.pc.model = p.model;
  d.pc.inv_ns = 1.0 / p.n_s;
  d.pc.inv_na = 1.0 / p.n_a;
  d.pc.chi_sa = p.chi_sa;
  d.pc.ln_sat_s = std::log(p.phi_sat_s);
  d.pc.ln_sat_a = std::log(p.phi_sat_a);
  const int nb = launch_diagnostics(geo(ctx->lv(0)), d, ctx->partial, s);
  sum_partials(nb, kDiagQuantities, ctx->partial, ctx->diag, s);
  // ||B v||: B v into the P1 scratch vector, then its FP64 dot product
  spmv_b(m.pb, ctx->Bv, state->v, ctx->tmp, s);
  dot<double>(ctx->N1, ctx->tmp, ctx->tmp, ctx->diag + kDiagQuantities, ctx->partial, s);
  double h[kDiagQuantities + 1];
  CHNSS_CK(cudaMemcpyAsync(h, ctx->diag, sizeof(h), cudaMemcpyDeviceToHost, s));
  CHNSS_CK(cudaStreamSynchronize(s));
  for (int i = 0; i < 4; ++i) out->mass[i] = h[i];
  out->p_mean = h[4];
  out->energy_local = h[5];
  out->energy_gradient = h[6];
  out->energy_kinetic = h[7];
  out->energy = h[5] + h[6] + h[7];
  out->div_norm = std::sqrt(h[kDiagQuantities]);
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

// ---------------------------------------------------------------------------
// Autotuner of the SpMV launch shape and the batched step.
namespace {

constexpr int kTuneCandidates[3] = {128, 256, 512};

void destroy_graphs(chnss_ctx *c) {
  ++c->sg_gen;                  // batch graphs recorded from this context are stale now
  for (auto &g : c->sgr) {      // recorded steps hold copies of the preconditioner bodies
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key = {};
  }
  for (PrecGraph &g : c->pg) {
    if (g.plain) cudaGraphExecDestroy(g.plain);
    if (g.prof) cudaGraphExecDestroy(g.prof);
    g.plain = g.prof = nullptr;
    for (Profiler::Probe &pr : g.probes) {
      if (pr.e0) cudaEventDestroy(pr.e0);
      if (pr.e1) cudaEventDestroy(pr.e1);
    }
    g.probes.clear();
    g.nprobes = 0;
  }
  if (c->cap) {
    cudaStreamDestroy(c->cap);
    c->cap = nullptr;
  }
}

template <typename T>
double time_spmv(chnss_ctx *c, MGHier<T> &h, int reps) {
  cudaStream_t s = c->s;
  SpmvArgs none;
  cudaEvent_t e0, e1;
  CHNSS_CK(cudaEventCreate(&e0));
  CHNSS_CK(cudaEventCreate(&e1));
  auto run = [&]() { h.spmv_level(0, h.b[0], h.t[0], SPMV_PLAIN, none, s); };
  run();
  run();
  CHNSS_CK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) run();
  CHNSS_CK(cudaEventRecord(e1, s));
  CHNSS_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CHNSS_CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

void set_block(chnss_ctx *c, bool velocity, int block) {
  Mesh &m = c->mesh->m;
  for (Level &L : m.lv) {
    if (velocity) {
      L.p2.sell.block = block;
      L.tv.P.sell.block = block;
      L.tv.R.sell.block = block;
    } else {
      L.p1.sell.block = block;
      L.t1.P.sell.block = block;
      L.t1.R.sell.block = block;
    }
  }
  if (velocity) {
    m.pbt.sell.block = block;
  } else {
    m.pb.sell.block = block;
  }
}

template <typename T>
void autotune_t(chnss_ctx *c, PrecSet<T> &P, chnss_tuning *out) {
  for (int group = 0; group < 2; ++group) {
    MGHier<T> &h = group == 0 ? P.L : P.A;
    double best = 1e300;
    int best_b = 256;
    for (int i = 0; i < 3; ++i) {
      set_block(c, group == 1, kTuneCandidates[i]);
      const double ms = time_spmv(c, h, 10);
      (group == 0 ? out->ms_p1 : out->ms_p2)[i] = ms;
      if (ms < best) { best = ms; best_b = kTuneCandidates[i]; }
    }
    set_block(c, group == 1, best_b);
    (group == 0 ? out->block_p1 : out->block_p2) = best_b;
  }
  for (int i = 0; i < 3; ++i) out->candidates[i] = kTuneCandidates[i];
}

}  // namespace

extern "C" chnss_status chnss_autotune(chnss_ctx_t ctx, chnss_tuning *out) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  if (!ctx->assembled) throw Error{CHNSS_ERR_STATE, "chnss_autotune needs an assembled context"};
  chnss_tuning t{};
  if (ctx->p32) autotune_t(ctx, *ctx->p32, &t);
  else autotune_t(ctx, *ctx->p64, &t);
  CHNSS_CK(cudaStreamSynchronize(ctx->s));
  destroy_graphs(ctx);          // launch shapes are baked into captured graphs
  capture_graphs(ctx);
  if (out) *out = t;
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

extern "C" chnss_status chnss_set_spmv_block(chnss_ctx_t ctx, int block_p1, int block_p2) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  for (int b : {block_p1, block_p2})
    if (b != kTuneCandidates[0] && b != kTuneCandidates[1] && b != kTuneCandidates[2])
      return fail(ctx, CHNSS_ERR_ARG, "threads per block must be 128, 256 or 512");
  ABI_TRY
  CHNSS_CK(cudaStreamSynchronize(ctx->s));
  set_block(ctx, false, block_p1);
  set_block(ctx, true, block_p2);
  destroy_graphs(ctx);
  capture_graphs(ctx);
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

extern "C" chnss_status chnss_set_step_mode(chnss_ctx_t ctx, int mode) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  if (mode != 0 && mode != 1) throw Error{CHNSS_ERR_ARG, "step mode must be 0 (host-driven) or 1 (one graph)"};
  if (mode == 1 && ctx->p.restart > 31) throw Error{CHNSS_ERR_ARG, "the one-graph step needs restart <= 31"};
  ctx->step_mode = mode;
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

extern "C" chnss_status chnss_set_step_concurrency(chnss_ctx_t ctx, int on) {
  if (!ctx) return fail(nullptr, CHNSS_ERR_ARG, "null context");
  ABI_TRY
  if (ctx->concurrent != (on != 0)) {
    CHNSS_CK(cudaStreamSynchronize(ctx->s));
    ctx->concurrent = on != 0;
    destroy_graphs(ctx);     // the graphs' branch structure follows the setting
    capture_graphs(ctx);
  }
  return CHNSS_OK;
  ABI_CATCH(ctx)
}

// ---------------------------------------------------------------------------
// One CUDA graph for a whole batch: every instance's step recorded as a
// parallel branch of one capture (a fork from the batch stream into each
// context's recording stream, a join back), launched once per call.  Kept
// for the two most recent (contexts, states) sets, since a trajectory
// alternates two state sets; dropped when a context is destroyed or its
// recorded graphs are (its generation changes).
namespace {
struct BatchGraph {
  std::vector<chnss_ctx *> ctx;
  std::vector<std::array<const void *, 20>> key;
  std::vector<unsigned long long> gen;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t s = nullptr;
  void release() {
    if (s) cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (s) cudaStreamDestroy(s);
    exec = nullptr;
    s = nullptr;
  }
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch;
std::atomic<int> g_batch_mode{0};    // chnss_set_batch_mode
std::atomic<long long> g_batch_one_graph{0}, g_batch_per_instance{0};

BatchGraph record_batch(int n, chnss_ctx *const *ctxs, const chnss_state *in, chnss_state *out) {
  BatchGraph b;
  for (int i = 0; i < n; ++i) {
    ensure_record_streams(ctxs[i]);
    CHNSS_CK(cudaStreamSynchronize(ctxs[i]->s));
    b.ctx.push_back(ctxs[i]);
    b.key.push_back(state_key(&in[i], &out[i]));
    b.gen.push_back(ctxs[i]->sg_gen);
  }
  CHNSS_CK(cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking));
  cudaEvent_t fork = nullptr, join = nullptr;
  CHNSS_CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  CHNSS_CK(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
  cudaGraph_t graph = nullptr;
  chnss_ctx *cur = nullptr;
  cudaStream_t user = nullptr;
  bool prof_on = false;
  auto restore = [&] {
    if (!cur) return;
    cur->s = user;
    cur->recording = false;
    cur->prof.on = prof_on;
    cur = nullptr;
  };
  try {
    CHNSS_CK(cudaStreamBeginCapture(b.s, cudaStreamCaptureModeThreadLocal));
    try {
      for (int i = 0; i < n; ++i) {
        cur = ctxs[i];
        user = cur->s;
        prof_on = cur->prof.on;
        cur->prof.on = false;          // no event nodes inside conditional bodies
        cur->recording = true;
        cur->s = cur->rq0;
        CHNSS_CK(cudaEventRecord(fork, b.s));
        CHNSS_CK(cudaStreamWaitEvent(cur->rq0, fork, 0));
        record_step_body(cur, &in[i], &out[i]);
        CHNSS_CK(cudaEventRecord(join, cur->rq0));
        CHNSS_CK(cudaStreamWaitEvent(b.s, join, 0));
        restore();
      }
    } catch (...) {
      restore();
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(b.s, &tmp);
      if (tmp) cudaGraphDestroy(tmp);
      throw;
    }
    const cudaError_t ec = cudaStreamEndCapture(b.s, &graph);
    if (ec != cudaSuccess)
      throw Error{CHNSS_ERR_CUDA, std::string("recording the batch graph: ") + cudaGetErrorString(ec)};
    const cudaError_t ei = cudaGraphInstantiate(&b.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess)
      throw Error{CHNSS_ERR_CUDA, std::string("instantiating the batch graph: ") + cudaGetErrorString(ei)};
  } catch (...) {
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    b.release();
    throw;
  }
  cudaEventDestroy(fork);
  cudaEventDestroy(join);
  return b;
}

// the cached graph of this batch (recorded on a miss)
BatchGraph &batch_graph_for(int n, chnss_ctx *const *ctxs, const chnss_state *in, chnss_state *out) {
  for (BatchGraph &b : g_batch) {
    if ((int)b.ctx.size() != n) continue;
    bool same = true;
    for (int i = 0; i < n && same; ++i)
      same = b.ctx[i] == ctxs[i] && b.gen[i] == ctxs[i]->sg_gen && b.key[i] == state_key(&in[i], &out[i]);
    if (same) return b;
  }
  BatchGraph b = record_batch(n, ctxs, in, out);
  if (g_batch.size() >= 2) {
    g_batch.front().release();
    g_batch.erase(g_batch.begin());
  }
  g_batch.push_back(std::move(b));
  return g_batch.back();
}
}  // namespace

namespace chnss {
void drop_batch_graphs(chnss_ctx *c) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t i = 0; i < g_batch.size();) {
    if (std::find(g_batch[i].ctx.begin(), g_batch[i].ctx.end(), c) != g_batch[i].ctx.end()) {
      g_batch[i].release();
      g_batch.erase(g_batch.begin() + i);
    } else {
      ++i;
    }
  }
}
}  // namespace chnss

extern "C" chnss_status chnss_set_batch_mode(int mode) {
  if (mode != 0 && mode != 1) return fail(nullptr, CHNSS_ERR_ARG, "batch mode must be 0 (a graph per instance) or 1 (one graph)");
  g_batch_mode = mode;
  return CHNSS_OK;
}

extern "C" chnss_status chnss_batch_stats(long long *one_graph, long long *per_instance) {
  if (one_graph) *one_graph = g_batch_one_graph.load();
  if (per_instance) *per_instance = g_batch_per_instance.load();
  return CHNSS_OK;
}

extern "C" chnss_status chnss_step_batched(int n_inst, chnss_ctx_t *ctxs, const chnss_state *in, chnss_state *out,
                                           chnss_solve_info *info, int max_threads) {
  ABI_TRY
  if (n_inst < 0 || (n_inst > 0 && (!ctxs || !in || !out))) throw Error{CHNSS_ERR_ARG, "bad batch arguments"};
  for (int i = 0; i < n_inst; ++i) {
    if (!ctxs[i]) throw Error{CHNSS_ERR_ARG, "null context in batch"};
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) throw Error{CHNSS_ERR_ARG, "a context appears twice in the batch"};
    check_state(&in[i]);
    check_state(&out[i]);
  }
  if (n_inst == 0) return CHNSS_OK;
  int dev = 0;
  CHNSS_CK(cudaGetDevice(&dev));
  std::vector<chnss_status> st(n_inst, CHNSS_OK);
  bool all_graphs = true;
  for (int i = 0; i < n_inst; ++i) all_graphs = all_graphs && ctxs[i]->step_mode == 1;
  if (all_graphs && n_inst > 1 && g_batch_mode == 1) {
    // the whole batch as one graph launch; if it cannot be recorded, one
    // graph launch per instance below
    std::unique_lock<std::mutex> lk(g_batch_mu);
    BatchGraph *bg = nullptr;
    std::string why;
    try {
      bg = &batch_graph_for(n_inst, ctxs, in, out);
    } catch (const Error &e) {
      why = e.msg;
    }
    if (bg) {
      const auto t0 = std::chrono::steady_clock::now();
      for (int i = 0; i < n_inst; ++i) CHNSS_CK(cudaStreamSynchronize(ctxs[i]->s));
      CHNSS_CK(cudaGraphLaunch(bg->exec, bg->s));
      g_launch_count.fetch_add(1, std::memory_order_relaxed);
      CHNSS_CK(cudaStreamSynchronize(bg->s));
      lk.unlock();
      ++g_batch_one_graph;
      const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      for (int i = 0; i < n_inst; ++i) st[i] = step_graph_finish(ctxs[i], info ? info + 6L * i : nullptr, secs);
      for (int i = 0; i < n_inst; ++i)
        if (st[i] != CHNSS_OK) {
          g_last_error = "instance " + std::to_string(i) + " failed with status " + std::to_string((int)st[i]);
          return st[i];
        }
      return CHNSS_OK;
    }
    g_last_error = "batch graph not recorded (" + why + "); one graph per instance";
  }
  if (all_graphs) {
    // one graph launch per instance from this thread, every instance on its
    // own stream; then one synchronisation per stream
    ++g_batch_per_instance;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<bool> launched(n_inst, false);
    for (int i = 0; i < n_inst; ++i) {
      try {
        step_graph_launch(ctxs[i], &in[i], &out[i]);
        launched[i] = true;
      } catch (const Error &e) {
        ctxs[i]->err = e.msg;
        st[i] = e.status;
      }
    }
    for (int i = 0; i < n_inst; ++i) {
      if (!launched[i]) continue;
      const cudaError_t e = cudaStreamSynchronize(ctxs[i]->s);
      if (e != cudaSuccess) {
        ctxs[i]->err = cudaGetErrorString(e);
        st[i] = CHNSS_ERR_CUDA;
        continue;
      }
      const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      st[i] = step_graph_finish(ctxs[i], info ? info + 6L * i : nullptr, secs);
    }
    for (int i = 0; i < n_inst; ++i)
      if (st[i] != CHNSS_OK) {
        g_last_error = "instance " + std::to_string(i) + " failed with status " + std::to_string((int)st[i]) +
                       (ctxs[i]->err.empty() ? std::string() : ": " + ctxs[i]->err);
        return st[i];
      }
    return CHNSS_OK;
  }
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (int i = next++; i < n_inst; i = next++) {
      chnss_ctx *c = ctxs[i];
      try {
        st[i] = c->step_mode ? step_graph(c, &in[i], &out[i], info ? info + 6L * i : nullptr)
                             : step(c, &in[i], &out[i], info ? info + 6L * i : nullptr);
      } catch (const Error &e) {
        c->err = e.msg;
        st[i] = e.status;
      } catch (const std::exception &e) {
        c->err = e.what();
        st[i] = CHNSS_ERR_CUDA;
      }
    }
  };
  const int nt = std::max(1, std::min(max_threads > 0 ? max_threads : n_inst, n_inst));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (std::thread &t : pool) t.join();
  for (int i = 0; i < n_inst; ++i)
    if (st[i] != CHNSS_OK) {
      g_last_error = "instance " + std::to_string(i) + " failed with status " + std::to_string((int)st[i]) +
                     (ctxs[i]->err.empty() ? std::string() : ": " + ctxs[i]->err);
      return st[i];
    }
  return CHNSS_OK;
  ABI_CATCH(nullptr)
}
