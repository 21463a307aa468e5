// Geometric multigrid V-cycle and Krylov drivers (host orchestration of the
// kernels in sparse.cu).
#pragma once

#include <mutex>

#include "kernels.h"

namespace chnss {

// CUDA-event timing of the hot kernel families, with their algorithmic
// bytes (values + indices + the vectors each launch must read or write).
struct Profiler {
  enum Kind { VEL_SPMV_L0 = 0, P1_SPMV_L0, NS_OUTER_SPMV, ORTHO, ASSEMBLY, P1_MG_COARSE, VEL_MG_COARSE, NKINDS };
  static const char *name(int k);
  bool on = false;
  struct Rec {
    long long launches = 0;
    double bytes = 0.0;
    double flops = 0.0;             // FP64 (or FP32) floating-point operations
    double ms_graph = 0.0;          // harvested from graph probes
    std::vector<cudaEvent_t> ev;   // start/stop pairs
    size_t used = 0;
  } rec[NKINDS];
  // A probe is a start/stop event pair recorded as nodes of a captured CUDA
  // graph; while `sink` is set, start/stop append probes instead of using the
  // eager pool.  After a replay has completed, harvest() adds the probes.
  struct Probe {
    int kind;
    double bytes;
    cudaEvent_t e0, e1;
  };
  std::vector<Probe> *sink = nullptr;   // preallocated events (created before capture)
  size_t sink_used = 0;
  std::mutex mu;                        // solves of one step run on several host threads
  // start returns a token for the matching stop (-1: not recorded)
  int start(int k, cudaStream_t s);
  // count: launches (or steps) the interval adds to the family
  void stop(int k, int token, cudaStream_t s, double bytes, double flops = 0.0, int count = 1);
  void harvest(const std::vector<Probe> &probes, size_t count);
  void reset();
  double elapsed_ms(int k);        // after a stream synchronisation
  void release();
  ~Profiler() { release(); }
};

// Scalar levels of at most this many rows (32 x 32 P1 meshes and coarser) are
// smoothed by one 512-thread block (mg_tail).
constexpr long kTailRows = 1100;

// One V-cycle of geometric multigrid (the inner solves that replace the
// paper's PyAMG blocks, Sec. 4): degree-2 Chebyshev-Jacobi pre/post
// smoothing on [hi/4, hi] (hi: Gershgorin bound of D^-1 A), restriction
// R = P^T, prolongation P, dense FP64 inverse on the coarsest level.
// kind 0: scalar P1 operators (CSR); kind 1: velocity operators (BSR2,
// interleaved vectors); kind 2: 3D velocity operators, scalar CSR over the
// interleaved dofs (Jacobi data, coarse level, transfers) applied through the
// 3x3-block SELL view bpat / bmap (set before init).  T is the smoothing
// precision.
template <typename T>
struct MGHier {
  int kind = 0;
  bool singular = false;   // pressure Laplacian: mean-zero projection, coarse K + 1 1^T
  int nl = 0;
  std::vector<const Pattern *> pat;
  std::vector<const int *> diag;
  std::vector<const double *> val64;
  std::vector<T *> val;
  std::vector<T *> dinv, x, t, r, b;
  std::vector<double *> hi, coef;
  std::vector<const Transfer *> tr;
  std::vector<const Pattern *> bpat;   // kind 2: node patterns (3x3-block SELL) per level
  std::vector<const int *> bmap;       // kind 2: their map9 (value -> CSR position)
  std::vector<long> n;
  int nc = 0;
  bool coarse_iter = false;   // coarsest level by Chebyshev steps (kCoarseDegree), no dense inverse
  bool keep_dense = false;    // set before init: dense coarsest level whatever its size (pressure Laplacian)
  double *dense = nullptr, *cinv = nullptr;
  int *status = nullptr;
  double *partial = nullptr, *sum = nullptr;
  Profiler *prof = nullptr;
  bool bf16 = false;       // level values stored in BF16 (T = float only; set before init)
  std::vector<__nv_bfloat16 *> val16;
  // set before setup: per-level smoothing bounds (device scalars) in place of
  // the Gershgorin bounds (the algebraic hierarchies of amg.cu)
  std::vector<const double *> hi_ext;
  int degree = 2;          // Chebyshev smoothing degree (pre and post)
  double ratio = 4.0;      // smoothing interval [hi / ratio, hi]
  // levels tail_l0.. (at most kTailRows rows each) run as one block launch
  int tail_l0 = -1;
  int tail_width = 8;            // widest tail row (operators and transfers): 8 or 16
  TailDesc<T> *tail = nullptr;   // device

  // levels: per level pattern + FP64 value pointer (values may change
  // between setups, the pointers may not); transfers tr[l] from level l+1.
  void init(Arena &ar, int kind, bool singular, const std::vector<const Pattern *> &pats,
            const std::vector<const int *> &diags, const std::vector<const double *> &vals,
            const std::vector<const Transfer *> &trs, double *partial_buf);
  // Recompute Jacobi data, Chebyshev coefficients, FP32 copies and the
  // coarse inverse from the current FP64 values.
  void setup(cudaStream_t s);
  T *input() { return b[0]; }
  T *output() { return x[0]; }
  // x[0] = V-cycle(b[0]); with inner_rtol > 0, x[0] = solve(b[0]) instead
  void apply(cudaStream_t s);
  // Multigrid as an inner solver with a tolerance (Sec. 5 applies its AMG
  // preconditioners to a relative tolerance): x <- x + V(b - A x) from x = 0
  // until ||b - A x|| <= inner_rtol ||b|| or inner_maxit V-cycles.  The
  // iterate, the right-hand side and the residual are FP64 whatever T is
  // (FP64 level-0 values): an FP32 residual of smooth iterates cancels down
  // to a floor of ~1e-4 relative on 1024^2 meshes, so the FP32 / BF16
  // hierarchies do mixed-precision iterative refinement (V-cycles in T,
  // residuals in FP64).  Under stream capture the loop is a conditional
  // WHILE node whose condition a one-thread kernel sets from the device
  // residual norm, so the captured preconditioner graph needs no host
  // synchronisation; otherwise the host reads the norms.  b[0] is
  // overwritten (it ends as the last residual).
  double inner_rtol = 0.0;
  int inner_maxit = 1;
  void enable_inner(Arena &ar, double rtol, int maxit, cudaStream_t body_stream);
  // the result as FP64 into *slot + off: the FP64 iterate of an inner
  // solve (an FP32 rounding of it would cap the preconditioner's accuracy),
  // else x[0] converted
  void write_output(double *const *slot, long off, cudaStream_t s);
  // the FP64 iterate of the last inner solve (null unless enable_inner)
  const double *iterate64() const { return acc; }
  // inner solves and V-cycles since the last reset, residual ratio of the
  // last solve (stream-ordered read on s, then a synchronisation)
  void inner_stats(bool reset, long long *solves, long long *cycles, double *last_rel, cudaStream_t s);
  // descriptor of levels tail_l0.. with the given vectors (device copy)
  TailDesc<T> *make_tail(Arena &ar, const std::vector<MultiPtr<T>> &X, const std::vector<MultiPtr<T>> &Tt,
                         const std::vector<MultiPtr<T>> &Rr, const std::vector<MultiPtr<T>> &B) const;
  // out = A_l u with the given epilogue (no profiling)
  void spmv_level(int l, const T *u, T *out, SpmvMode mode, const SpmvArgs &a, cudaStream_t s);

 private:
  double *bsave = nullptr, *acc = nullptr;   // inner solve: right-hand side, iterate (FP64)
  double *r64 = nullptr, *val0_64 = nullptr;  // T != double: FP64 residual, level-0 FP64 SELL values
  // [0] ||b||^2 [1] ||r||^2 [2] V-cycles of the last solve [3] V-cycles [4] solves since reset
  double *ictl = nullptr, *ipartial = nullptr;
  int *iit = nullptr;
  cudaStream_t bodyq = nullptr;               // captures the WHILE body
  void op(int l, const T *u, T *out, SpmvMode mode, const SpmvArgs &a, cudaStream_t s);
  long sell_values(int l) const;                  // values of level l in SELL order
  template <typename VT>
  void gather_values(int l, VT *out, cudaStream_t s) const;   // FP64 CSR values -> SELL order
  void vcycle(int l, cudaStream_t s);
  void cycle(cudaStream_t s);                 // one V-cycle with the singular projections
  void inner_residual(cudaStream_t s);        // b[0] = bsave - A acc (FP64); ictl[1] = ||b - A acc||^2
  void solve(cudaStream_t s);
};

// The same V-cycle as MGHier<T> (kind 0: scalar P1 operators, non-singular)
// on nr <= kMaxRhs vectors at once: the hierarchy's matrices, Jacobi data,
// coefficients, transfers and coarse inverse are shared; every sweep reads
// the matrix once for all vectors (spmv_sell_multi).  Vector k's result is
// bitwise the one MGHier<T>::apply gives for it alone.
template <typename T>
struct MGBatch {
  MGHier<T> *h = nullptr;
  int nr = 0;
  std::vector<MultiPtr<T>> x, t, r, b;     // per level
  TailDesc<T> *tail = nullptr;             // device, levels h->tail_l0..
  void init(Arena &ar, MGHier<T> *hier, int nr);
  T *input(int k) { return b[0].p[k]; }
  T *output(int k) { return x[0].p[k]; }
  void apply(cudaStream_t s);

 private:
  void op(int l, const MultiPtr<T> &u, const MultiPtr<T> &out, SpmvMode mode, const MultiArgs<T> &a,
          cudaStream_t s);
  void vcycle(int l, cudaStream_t s);
};

struct LinearOperator {
  virtual ~LinearOperator() = default;
  virtual long size() const = 0;
  virtual void apply(const double *x, double *y, cudaStream_t s) = 0;
  virtual void precond(const double *r, double *z, cudaStream_t s) = 0;
  // called by the Krylov driver after each host synchronisation of the stream
  virtual void after_sync() {}
  // Batched FGMRES: operators returning the same non-null key are applied
  // together by apply_batch of the first one (x[i] -> y[i] for ops[i]), with
  // results bitwise those of their own apply
  virtual const void *batch_key() const { return nullptr; }
  virtual void apply_batch(int n, LinearOperator *const *ops, const double *const *x, double *const *y,
                           cudaStream_t s) {
    for (int i = 0; i < n; ++i) ops[i]->apply(x[i], y[i], s);
  }
};

struct KrylovWork {
  int m = 0;
  long nmax = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *sc = nullptr, *partial = nullptr;
  double *hstat = nullptr;   // pinned host, 4 doubles
  // double-FP32 Gram-Schmidt (params.ortho = 1, restart <= 31): the basis
  // also as pairs of FP32 numbers, read by the Gram-Schmidt passes; V keeps
  // each vector's exact FP64 value for the preconditioner
  float2 *V2 = nullptr;
  // device-driven solves: [0] ||b|| [1] target [2] ||r||; [0] iterations
  // [1] k [2] status [3] converged [4] breakdown [5] non-finite [6] go on
  double *dv = nullptr;
  int *di = nullptr;
  void init(Arena &ar, int m, long nmax, double *pinned, bool pairs = false);
};

// Device-driven solves, recorded into the CUDA graph that s is capturing
// (no host synchronisation): the FGMRES restart cycles are a conditional
// WHILE node, the m Arnoldi steps of a cycle conditional IF nodes, every
// decision a one-thread kernel; the PCG iterations a WHILE node.  Bodies
// are captured on bq1 (WHILE) and bq2 (IF).  Same kernels, order and
// stopping rules as fgmres() / pcg(), so the results are bitwise theirs.
// The outcome stays on the device: krylov_record() writes [iterations,
// converged, relative residual, status] (doubles) to dst.
void fgmres_record(LinearOperator &A, const double *b, double *x, double rtol, double atol, int maxit,
                   KrylovWork &ws, cudaStream_t s, cudaStream_t bq1, cudaStream_t bq2);
void pcg_record(const Pattern &P, const double *val, const double *dinv, const double *b, double *x, double rtol,
                int maxit, KrylovWork &ws, cudaStream_t s, cudaStream_t bq1);
void krylov_record(const KrylovWork &ws, double *dst, cudaStream_t s);

// Right-preconditioned FGMRES(m), CGS2, Givens, x0 = 0; stop when the true
// residual satisfies ||b - A x|| <= max(rtol ||b||, atol) (Sec. 5).
chnss_status fgmres(LinearOperator &A, const double *b, double *x, double rtol, double atol, int maxit,
                    KrylovWork &ws, chnss_solve_info *info, cudaStream_t s, Profiler *prof = nullptr);

// Several independent FGMRES solves advanced together: every tick applies
// one batched preconditioner to the current basis vector of each active
// solve (one call, e.g. one graph launch), then runs each solve's operator,
// CGS2 and Givens step, and synchronises the stream once for all of them.
// Per solve, the arithmetic and its order are those of fgmres(), so the
// iterates are bitwise the same as solving one system after the other.
struct BatchPrecond {
  virtual ~BatchPrecond() = default;
  // z[k] = P_k r[k] for k < K; r[k] == nullptr: solve k is idle this tick
  virtual void apply(int K, const double *const *r, double *const *z, cudaStream_t s) = 0;
  virtual void after_sync() {}
};
chnss_status fgmres_batch(int K, LinearOperator *const *A, const double *const *b, double *const *x, double rtol,
                          double atol, int maxit, KrylovWork *const *ws, chnss_solve_info *info, BatchPrecond &P,
                          cudaStream_t s, Profiler *prof = nullptr);

// Jacobi PCG for an SPD CSR matrix (FP64), x0 = 0, recursive residual test.
// Work storage: r = ws.w, z / p / q = ws.V + {0, 1, 2} n, scalars ws.sc[0..6),
// reduction partials ws.partial, one pinned host double ws.hstat.  b is
// read once, before x is written, so x may alias b.
chnss_status pcg(const Pattern &P, const double *val, const double *dinv, const double *b, double *x, double rtol,
                 int maxit, KrylovWork &ws, chnss_solve_info *info, cudaStream_t s);

}  // namespace chnss
