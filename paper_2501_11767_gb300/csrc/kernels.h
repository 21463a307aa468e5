// Launch wrappers of the sparse, vector and reduction kernels (sparse.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace chnss {

// Fused SpMV epilogues (rows of A u):
//   PLAIN  out = A u
//   RES    out = b - A u
//   ADD    out += A u
//   CHEB   out = c0 u + c1 w + c2 dinv (b - A u), (c0, c1, c2) = coef[0..2] (device)
enum SpmvMode { SPMV_PLAIN = 0, SPMV_RES = 1, SPMV_ADD = 2, SPMV_CHEB = 3 };

// Up to kMaxRhs vectors that share one matrix (multi-right-hand-side kernels).
constexpr int kMaxRhs = 3;
template <typename T>
struct MultiPtr {
  T *p[kMaxRhs] = {nullptr, nullptr, nullptr};
};
template <typename T>
struct MultiArgs {              // per-vector b and w, shared Jacobi diagonal and coefficients
  MultiPtr<T> b, w;
  const T *dinv = nullptr;
  const double *coef = nullptr;
};

struct SpmvArgs {
  const void *b = nullptr;      // T*
  const void *w = nullptr;      // T*  (CHEB)
  const void *dinv = nullptr;   // T*  (CHEB)
  const double *coef = nullptr; // device [3] (CHEB)
};

// Scalar CSR; ncomp = 1 or 2 (the same scalar weights applied per component
// of an interleaved 2-vector: velocity mass and velocity transfers).
template <typename T>
void spmv_csr(const Pattern &P, const T *val, int ncomp, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
              cudaStream_t s);
// 2x2-block CSR (velocity operator), vectors interleaved.
template <typename T>
void spmv_bsr2(const Pattern &P, const T *val, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
               cudaStream_t s);

// SELL-C-sigma variants (see Sell in internal.h).  Values in SELL order:
// ncomp (1, 2 or 4) values per entry, out[e * ncomp + c].
template <typename Tout>
void sell_gather(const Sell &S, int ncomp, const double *csr_vals, Tout *out, cudaStream_t s);
// SELL values of the transposed matrix (square symmetric patterns; for
// ncomp = 4 each 2x2 block is transposed as well)
void sell_gather_transposed(const Sell &S, int ncomp, const double *csr_vals, double *out, cudaStream_t s);
template <typename T>
void spmv_sell(const Pattern &P, const T *sval, int ncomp, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
               cudaStream_t s);
template <typename T>
void spmv_sell_bsr2(const Pattern &P, const T *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                    cudaStream_t s);
// Warps per slice the SpMV dispatchers use for a pattern (1: one thread per
// row; a function of the pattern and the device only): scalar rows, 2x2
// blocks, 3x3 blocks
int sell_split(const Sell &S);
int sell_warps_bsr2(const Sell &S);
int sell_warps_bsr3(const Sell &S);
// 3x3-block SELL (3D velocity operators on the P2 node pattern, vectors
// interleaved): value m = 3 r + d of SELL entry e at 9 (e - e % 32) + 32 m +
// e % 32; map9 holds the CSR position of every such value (-1: padding)
template <typename Tout>
void sell_gather9(long nent, const int *map9, const double *csr_vals, Tout *out, cudaStream_t s);
template <typename T>
void spmv_sell_bsr3(const Pattern &P, const T *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                    cudaStream_t s);
void spmv_sell_bsr3(const Pattern &P, const __nv_bfloat16 *sval, const float *u, float *out, SpmvMode mode,
                    const SpmvArgs &a, cudaStream_t s);
// Coarsest level of a 3x3-block hierarchy: degree Chebyshev-Jacobi steps from
// zero (coef layout of cheb_coefficients) in one block; the iterate ends in x
// (t: scratch).  Levels of at most kChebBlockSlices SELL slices.
constexpr int kChebBlockSlices = 8;
template <typename T, typename VT>
void cheb_block_bsr3(const Pattern &P, const VT *sval, const T *dinv, const T *b, T *x, T *t, const double *coef,
                     int degree, cudaStream_t s);
// nr (1..3) vectors through one scalar matrix with rows of at most 8 entries;
// each output is bitwise the single-vector result (same per-row order).
template <typename T>
void spmv_sell_multi(const Pattern &P, const T *sval, int nr, const MultiPtr<T> &u, const MultiPtr<T> &out,
                     SpmvMode mode, const MultiArgs<T> &a, cudaStream_t s);
template <typename T>
void vec_scale_dinv_multi(int n, int nr, const double *scale, const T *dinv, const MultiPtr<T> &b,
                          const MultiPtr<T> &out, cudaStream_t s);
template <typename T>
void dense_apply_multi(int n, int nr, const double *inv, const MultiPtr<T> &b, const MultiPtr<T> &x,
                       cudaStream_t s);
template <typename T>
void vec_copy_multi(long n, int nr, const MultiPtr<T> &in, const MultiPtr<T> &out, cudaStream_t s);
// Coarse end of a scalar V-cycle run by one 512-thread block (see k_mg_tail):
// level 0 of the descriptor is the first level handled by the block, the last
// one is the coarsest (dense inverse).  Level sizes must allow every sweep's
// rows to be spread over the block; all pointers are device pointers.
constexpr int kMaxTailLevels = 8;
struct TailSell {                 // SELL view of one operator (rows of at most 16 entries)
  int nslices = 0;
  const int *sp = nullptr, *rowid = nullptr, *col = nullptr;
};
template <typename T>
struct TailLevel {
  int n = 0;                      // rows (vector length)
  TailSell A, R, P;               // operator; restriction to / prolongation from the next level
  const T *val = nullptr, *Rval = nullptr, *Pval = nullptr, *dinv = nullptr;
  const double *coef = nullptr;   // Chebyshev coefficients of the level
  MultiPtr<T> x, t, r, b;
};
template <typename T>
struct TailDesc {
  int nlev = 0, degree = 2, nc = 0;
  int coarse_degree = 0;          // > 0: Chebyshev steps on the coarsest level instead of cinv
  const double *cinv = nullptr;   // coarsest level, row-major nc x nc
  TailLevel<T> lv[kMaxTailLevels];
};
// width: 8 or 16, the widest row of any tail operator or transfer (rounded up)
template <typename T>
void mg_tail(const TailDesc<T> *d_desc, int nr, int width, cudaStream_t s);
// BF16-stored values, FP32 vectors and accumulation (preconditioner variant)
void spmv_sell(const Pattern &P, const __nv_bfloat16 *sval, int ncomp, const float *u, float *out, SpmvMode mode,
               const SpmvArgs &a, cudaStream_t s);
void spmv_sell_bsr2(const Pattern &P, const __nv_bfloat16 *sval, const float *u, float *out, SpmvMode mode,
                    const SpmvArgs &a, cudaStream_t s);
void spmv_sell_ch(const Pattern &P, const double *L, const double *K, const double *k12, const double *M, double a12,
                  double a21, double a22, const double *x, double *y, cudaStream_t s);
// nr (1..kMaxRhs) CH systems that share L, K, K12 (K when null) and M, with
// per-system coefficients: each output bitwise the spmv_sell_ch result
struct ChCoef3 {
  double a12[kMaxRhs], a21[kMaxRhs], a22[kMaxRhs];
};
void spmv_sell_ch_multi(const Pattern &P, const double *L, const double *K, const double *k12, const double *M, int nr,
                        const ChCoef3 &cf, const MultiPtr<const double> &x, const MultiPtr<double> &y,
                        cudaStream_t s);
void spmv_sell_b(const Pattern &P, const double *sval2, const double *v, double *y, cudaStream_t s);
void spmv_sell_bt_add(const Pattern &P, const double *sval2, const double *p, double *yv, cudaStream_t s);

// CH operator: y1 = L x1 + a12 K12 x2, y2 = a21 K x1 + a22 M x2 on the P1
// pattern (K12 = K when k12 == nullptr).
void spmv_ch(const Pattern &P, const double *L, const double *K, const double *k12, const double *M, double a12,
             double a21, double a22, const double *x, double *y, cudaStream_t s);
// y = B v (B: N1 x N2 nodes, 2 values per entry); y += B^T p into interleaved v.
void spmv_b(const Pattern &P, const double *val, const double *v, double *y, cudaStream_t s);
void spmv_bt_add(const Pattern &P, const double *val, const double *p, double *yv, cudaStream_t s);

// Jacobi data + Gershgorin bound of D^-1 A: dinv[i] = 1 / a_ii,
// hi = max_i sum_j |a_ij| / |a_ii| (device scalar).  Also the Chebyshev
// coefficient triples for a degree-2 smoother on [hi / ratio, hi].
template <typename T>
void jacobi_csr(const Pattern &P, const double *val, const int *diag, T *dinv, double *hi, double *partial,
                cudaStream_t s);
template <typename T>
void jacobi_bsr2(const Pattern &P, const double *val, const int *diag, T *dinv, double *hi, double *partial,
                 cudaStream_t s);
// Chebyshev smoother of degree d on [hi / ratio, hi]; coef layout (4 + 3(d-1)
// doubles): [beta0][first post step: 1, 0, beta0][(c0, c1, c2) for k = 1..d-1]
// with x_{k+1} = c0 x_k + c1 x_{k-1} + c2 D^-1 (b - A x_k).
constexpr int kMaxSmoothDegree = 16;
// Coarsest multigrid level: a dense FP64 inverse (rebuilt with the level's
// operator by one thread block) while it has at most kCoarseDenseMax rows or
// is the singular pressure Laplacian (constant, built once); otherwise
// kCoarseDegree Chebyshev-Jacobi steps from zero on [hi / kCoarseRatio, hi]
// (the non-singular blocks are mass-dominated on coarse meshes).
constexpr int kCoarseDenseMax = 256;
constexpr int kCoarseDegree = 16;
constexpr double kCoarseRatio = 64.0;
void cheb_coefficients(const double *hi, double ratio, int degree, double *coef, cudaStream_t s);

// vectors
template <typename T>
void vec_scale_dinv(int n, const double *scale, const T *dinv, const T *b, T *out, cudaStream_t s);
template <typename Ta, typename Tb>
void vec_convert(long n, const Ta *in, Tb *out, cudaStream_t s);
// conversions through a device pointer slot (*slot + off), so that a
// captured CUDA graph can read / write vectors chosen at replay time
template <typename Ta, typename Tb>
void vec_convert_from_slot(long n, const Ta *const *slot, long off, Tb *out, cudaStream_t s);
template <typename Ta, typename Tb>
void vec_convert_to_slot(long n, const Ta *in, Tb *const *slot, long off, cudaStream_t s);
void set_ptr_slots(void **slots, const void *a, const void *b, cudaStream_t s);
// slots[0..n) = ptrs[0..n) (host array of device pointers, n <= 8)
void set_ptr_slots_n(void **slots, int n, const void *const *ptrs, cudaStream_t s);   // slots[0] = a, slots[1] = b
void vec_axpby(long n, double a, const double *x, double b, double *y, cudaStream_t s);      // y = a x + b y
void vec_copy(long n, const double *x, double *y, cudaStream_t s);
void vec_clip01(long n, double *x, cudaStream_t s);   // x = min(max(x, 0), 1)
void vec_fill(long n, double v, double *y, cudaStream_t s);
void vec_scale_by_inv(long n, const double *src, const double *hn, double *dst, cudaStream_t s);  // dst = src / *hn
template <typename T>
void vec_sub_mean(int n, T *x, const double *sum, cudaStream_t s);   // x -= sum / n

// deterministic FP64 reductions: fixed grid of reduce_blocks(n) blocks
// (at most 8 per multiprocessor of the current device and never more than
// kReduceMaxBlocks), partial sums in fixed order, then one block sums the
// partials.  Partial buffers hold kReduceMaxBlocks doubles per reduced value.
constexpr int kReduceMaxBlocks = 2048;
int reduce_blocks(long n);
// multiprocessors of the current device (queried once per device)
int device_sm_count();
// out[v] = sum over b < nb of partial[v * nb + b], v < k (fixed order)
void sum_partials(int nb, int k, const double *partial, double *out, cudaStream_t s);
template <typename T>
void dot(long n, const T *x, const T *y, double *out, double *partial, cudaStream_t s);
template <typename T>
void vsum(long n, const T *x, double *out, double *partial, cudaStream_t s);
void mdot(long n, const double *V, long ldv, int k, const double *w, double *out, double *partial, cudaStream_t s);
void ortho_update_mdot(long n, const double *V, long ldv, int k, const double *h, double *w, double *out,
                       double *partial, cudaStream_t s);
void ortho_update_norm(long n, const double *V, long ldv, int k, const double *h, double *w, double *out,
                       double *partial, cudaStream_t s);
void combine_columns(long n, const double *Z, long ldz, int k, const double *y, double *x, cudaStream_t s);

// CGS2 in three passes with the vector count k as a compile-time constant
// (k <= 31; cgs2_fast(k) says whether it applies):
//   h1 = V^T w;   w -= V h1, h2w[0..k) = V^T w, h2w[k] = w^T w;
//   vout = (w - V h2) / *hn   (the next basis vector).
bool cgs2_fast(int k);
void cgs2_dots(long n, const double *V, long ld, int k, const double *w, double *h1, double *partial,
               cudaStream_t s);
void cgs2_update_dots(long n, const double *V, long ld, int k, const double *h1, double *w, double *h2w,
                      double *partial, cudaStream_t s);
void cgs2_update_scale(long n, const double *V, long ld, int k, const double *h2, const double *w, const double *hn,
                       double *vout, cudaStream_t s);

// The same three CGS2 passes in double-FP32 arithmetic (values as pairs of
// FP32 numbers, about 48 significant bits), reading the basis from V2, its
// pair copy; w enters pass 1 and 2 in FP64, pass 2 leaves it in place as
// pairs, pass 3 reads those pairs and writes the next basis vector both as
// pairs (vout2) and as their exact FP64 values (vout64).  k <= 31.
void dfgs_dots(long n, const float2 *V2, long ld, int k, const double *w, double *h1, double *partial,
               cudaStream_t s);
void dfgs_update_dots(long n, const float2 *V2, long ld, int k, const double *h1, double *w, double *h2w,
                      double *partial, cudaStream_t s);
void dfgs_update_scale(long n, const float2 *V2, long ld, int k, const double *h2, const double *w,
                       const double *hn, float2 *vout2, double *vout64, cudaStream_t s);
// first basis vector w / *hn as pairs and as their FP64 values
void dfgs_first(long n, const double *w, const double *hn, float2 *vout2, double *vout64, cudaStream_t s);

// Arnoldi bookkeeping on one thread: H(:, j) = h1 + h2, H(j+1, j) = sqrt(nrm2),
// previous Givens rotations, new rotation, g update.  Writes to status:
// [0] |g_{j+1}|, [1] H(j+1, j).
void arnoldi_finish(int j, int ldh, double *H, const double *h1, const double *h2, const double *nrm2,
                    double *cs, double *sn, double *g, double *status, cudaStream_t s);
// the same with hn^2 = h2w[j+1] - ||h2w[0..j]||^2 (Pythagoras after CGS2)
void arnoldi_finish_pyth(int j, int ldh, double *H, const double *h1, const double *h2w, double *cs, double *sn,
                         double *g, double *status, cudaStream_t s);
void hessenberg_solve(int k, int ldh, const double *H, const double *g, double *y, cudaStream_t s);
// the same two steps with the column count k read from device memory
void hessenberg_solve_dev(const int *k, int ldh, const double *H, const double *g, double *y, cudaStream_t s);
void combine_columns_dev(long n, const double *Z, long ldz, const int *k, const double *y, double *x,
                         cudaStream_t s);
void set_scalar(double *dst, const double *src, double scale, bool sqrt_first, cudaStream_t s);
// PCG scalars: alpha = rz / pq
void pcg_alpha(const double *rz, const double *pq, double *alpha, cudaStream_t s);
void pcg_update_xr(long n, const double *alpha, const double *p, const double *q, double *x, double *r,
                   cudaStream_t s);
void pcg_update_p(long n, const double *rz_new, const double *rz_old, const double *z, double *p, cudaStream_t s);
void vec_mul(long n, const double *a, const double *b, double *out, cudaStream_t s);

// dense coarse-grid inverse (one CTA, Gauss-Jordan with partial pivoting)
void coarse_dense_csr(const Pattern &P, const double *val, double add_all, double *dense, cudaStream_t s);
void coarse_dense_bsr2(const Pattern &P, const double *val, double *dense, cudaStream_t s);
void dense_invert(int n, double *a, double *inv, int *status, cudaStream_t s);
template <typename T>
void dense_apply(int n, const double *inv, const T *b, T *x, cudaStream_t s);

}  // namespace chnss
