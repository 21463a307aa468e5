// Smoothed-aggregation algebraic multigrid on the device (Sec. 5: the
// paper's block preconditioners come from PyAMG's algebraic multigrid,
// smoothed aggregation for the nonsymmetric Cahn-Hilliard blocks M + tau C
// and for every Navier-Stokes block in 3D).
//
// Setup, per level l (A_0 = the caller's matrix):
//   symbolic (depends on the pattern only; once per handle)
//     roots     maximal distance-2 independent set of the graph of A_l's
//               pattern (theta = 0 strength: every stored off-diagonal
//               entry), synchronous rounds of two max-propagations of the
//               keys (state << 62 | priority << 32 | i), priority = the 30
//               leading bits of SplitMix64 output number (l << 32) + i;
//     aggregates  roots numbered in node order (a block scan); pass 1: a
//               root's neighbours join the adjacent root of largest key;
//               pass 2: the others join the pass-1 neighbour of largest key;
//     patterns  P = pattern(A T) (T[i, agg(i)]), pattern(A P),
//               R = P^T (transpose with a position map, rows sorted),
//               A_{l+1} = pattern(R (A P)): thread-per-row sorted merges;
//   numeric (every chnss_amg_update)
//     hi_l      min(Gershgorin bound, 1.1 x 10 power steps on D^-1 A_l from a
//               +-1 start drawn with SplitMix64 outputs ((l + 64) << 32) + i)
//     P         T - (4 / (3 hi_l)) D^-1 (A T) on its pattern,
//     A P       one thread per row, terms in CSR order through term ->
//               position maps built with the patterns;
//     A_{l+1}   R (A P): one thread per entry, its terms in R's CSR order
//               (the order a row-by-row accumulation would add them).
// The V-cycle is MGHier<T> (kind 0) on these levels with hi_l as the
// smoothing bounds.  No atomics touch a floating-point value, so every
// result is bit-reproducible.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <vector>

#include "amg.h"
#include "solver.h"

namespace chnss {
namespace {

constexpr int TPB = 256;
constexpr int kAmgMaxRow = 512;      // widest row of a product pattern
constexpr int kAmgMaxLevels = 12;
constexpr int kAmgCoarseRows = 64;   // levels are added while a level is larger
constexpr int kAmgPowerSteps = 10;
constexpr double kAmgPowerSafety = 1.1;
constexpr int kAmgMaxRounds = 100000;
constexpr int kAmgRestart = 30;

inline int nblk(long n) { return (int)std::max<long>(1, (n + TPB - 1) / TPB); }

// Output number `key` (0-based) of SplitMix64 started from state 0
// (Steele, Lea and Flood, OOPSLA 2014): mix((key + 1) * golden gamma).
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t key) {
  uint64_t z = (key + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr uint64_t kUndecided = 1, kRoot = 2;

__global__ void k_mis_init(int n, int level, uint64_t *base, uint64_t *state) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  const uint64_t pr = splitmix64_out(((uint64_t)level << 32) + (uint64_t)i) >> 34;
  base[i] = (pr << 32) | (uint64_t)i;
  state[i] = kUndecided;
}

// m1[i] = max over the closed neighbourhood (row i's pattern) of the keys
__global__ void k_mis_max1(int n, const int *__restrict__ rp, const int *__restrict__ col,
                           const uint64_t *__restrict__ state, const uint64_t *__restrict__ base, uint64_t *m1) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  uint64_t m = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    m = max(m, (state[j] << 62) | base[j]);
  }
  m1[i] = m;
}

// m2 over the closed neighbourhood of m1; undecided nodes decide; undecided
// count of the round after the update in *und
__global__ void k_mis_max2(int n, const int *__restrict__ rp, const int *__restrict__ col,
                           const uint64_t *__restrict__ m1, const uint64_t *__restrict__ base, uint64_t *state,
                           int *und) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  if (state[i] != kUndecided) return;
  uint64_t m = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) m = max(m, m1[col[k]]);
  const uint64_t key = (kUndecided << 62) | base[i];
  if (m == key) state[i] = kRoot;
  else if ((m >> 62) == kRoot) state[i] = 0;
  else atomicAdd(und, 1);
}

__global__ void k_root_flag(int n, const uint64_t *state, int *flag) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < n) flag[i] = state[i] == kRoot ? 1 : 0;
}

// Exclusive prefix sum of in[0..n) by one block (in place allowed); the
// total in *total.  Chunks of 4 * 1024 entries, a carried offset.
__global__ void __launch_bounds__(1024) k_scan(int n, const int *in, int *out, int *total) {
  __shared__ int wsum[32];
  __shared__ int carry_s;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) carry_s = 0;
  __syncthreads();
  for (long base = 0; base < n; base += 4096) {
    int v[4], s = 0;
    for (int q = 0; q < 4; ++q) {
      const long i = base + 4L * t + q;
      v[q] = i < n ? in[i] : 0;
      s += v[q];
    }
    int incl = s;   // inclusive scan of the thread sums within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int carry = carry_s;
    int run = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - s;
    for (int q = 0; q < 4; ++q) {
      const long i = base + 4L * t + q;
      if (i < n) out[i] = run;
      run += v[q];
    }
    __syncthreads();
    if (t == 0) carry_s = carry + wsum[31];
    __syncthreads();
  }
  if (t == 0) *total = carry_s;
}

// pass 1: roots take their number; a root's neighbours join the adjacent
// root of largest key; others -1
__global__ void k_agg_pass1(int n, const int *__restrict__ rp, const int *__restrict__ col,
                            const uint64_t *__restrict__ state, const uint64_t *__restrict__ base,
                            const int *__restrict__ rootnum, int *agg1) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  if (state[i] == kRoot) {
    agg1[i] = rootnum[i];
    return;
  }
  int best = -1;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    if (j != i && state[j] == kRoot && (best < 0 || base[j] > base[best])) best = j;
  }
  agg1[i] = best >= 0 ? rootnum[best] : -1;
}

// pass 2: every node still alone joins the pass-1 neighbour of largest key
__global__ void k_agg_pass2(int n, const int *__restrict__ rp, const int *__restrict__ col,
                            const uint64_t *__restrict__ base, const int *__restrict__ agg1, int *agg, int *err) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  if (agg1[i] >= 0) {
    agg[i] = agg1[i];
    return;
  }
  int best = -1;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    if (j != i && agg1[j] >= 0 && (best < 0 || base[j] > base[best])) best = j;
  }
  if (best < 0) {
    atomicExch(err, 1);
    agg[i] = 0;
  } else {
    agg[i] = agg1[best];
  }
}

__global__ void k_agg_size(int n, const int *agg, int *size) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < n) atomicAdd(&size[agg[i]], 1);
}

__global__ void k_tval(int n, const int *agg, const int *size, double *tval, int *iota) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < n) {
    tval[i] = 1.0 / sqrt((double)size[agg[i]]);
    iota[i] = i;
  }
  if (i == n) iota[n] = n;
}

// Sorted distinct columns of row i of A B in buf (at most kAmgMaxRow);
// returns the count, or -1 when the row is wider.
__device__ int product_row(int i, const int *__restrict__ arp, const int *__restrict__ acol,
                           const int *__restrict__ brp, const int *__restrict__ bcol, int *buf) {
  int m = 0;
  for (int ka = arp[i]; ka < arp[i + 1]; ++ka) {
    const int k = acol[ka];
    for (int kb = brp[k]; kb < brp[k + 1]; ++kb) {
      const int c = bcol[kb];
      int lo = 0, hi = m;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (buf[mid] < c) lo = mid + 1;
        else hi = mid;
      }
      if (lo < m && buf[lo] == c) continue;
      if (m == kAmgMaxRow) return -1;
      for (int q = m; q > lo; --q) buf[q] = buf[q - 1];
      buf[lo] = c;
      ++m;
    }
  }
  return m;
}

__global__ void k_product_count(int n, const int *arp, const int *acol, const int *brp, const int *bcol, int *cnt,
                                int *err) {
  const int i = blockIdx.x * 128 + threadIdx.x;
  if (i >= n) return;
  int buf[kAmgMaxRow];
  const int m = product_row(i, arp, acol, brp, bcol, buf);
  if (m < 0) {
    atomicExch(err, 2);
    cnt[i] = 0;
  } else {
    cnt[i] = m;
  }
}

__global__ void k_product_fill(int n, const int *arp, const int *acol, const int *brp, const int *bcol,
                               const int *crp, int *ccol) {
  const int i = blockIdx.x * 128 + threadIdx.x;
  if (i >= n) return;
  int buf[kAmgMaxRow];
  const int m = product_row(i, arp, acol, brp, bcol, buf);
  const int c0 = crp[i];
  for (int q = 0; q < m && c0 + q < crp[i + 1]; ++q) ccol[c0 + q] = buf[q];
}

// products per row of A B (the length of its term list)
__global__ void k_product_terms(int n, const int *__restrict__ arp, const int *__restrict__ acol,
                                const int *__restrict__ brp, int *cnt) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  int t = 0;
  for (int ka = arp[i]; ka < arp[i + 1]; ++ka) t += brp[acol[ka] + 1] - brp[acol[ka]];
  cnt[i] = t;
}

// position in C of every term of row i of A B, in the order the numeric
// product sums them (A's CSR order, then B's)
__global__ void k_product_positions(int n, const int *__restrict__ arp, const int *__restrict__ acol,
                                    const int *__restrict__ brp, const int *__restrict__ bcol,
                                    const int *__restrict__ crp, const int *__restrict__ ccol,
                                    const int *__restrict__ tptr, int *tpos) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  const int c0 = crp[i], c1 = crp[i + 1];
  int t = tptr[i];
  for (int ka = arp[i]; ka < arp[i + 1]; ++ka) {
    const int k = acol[ka];
    for (int kb = brp[k]; kb < brp[k + 1]; ++kb) {
      const int c = bcol[kb];
      int lo = c0, hi = c1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ccol[mid] < c) lo = mid + 1;
        else hi = mid;
      }
      tpos[t++] = lo < c1 && ccol[lo] == c ? lo : -1;   // always found: C is the product's pattern
    }
  }
}

// C = A B on C's (sorted) pattern through the term positions: row i summed by
// one thread, term by term in the CSR order of A's row and then of B's rows
__global__ void k_product_values_mapped(int n, const int *__restrict__ arp, const int *__restrict__ acol,
                                        const double *__restrict__ aval, const int *__restrict__ brp,
                                        const double *__restrict__ bval, const int *__restrict__ crp,
                                        const int *__restrict__ tptr, const int *__restrict__ tpos,
                                        double *cval) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  for (int q = crp[i]; q < crp[i + 1]; ++q) cval[q] = 0.0;
  int t = tptr[i];
  for (int ka = arp[i]; ka < arp[i + 1]; ++ka) {
    const int k = acol[ka];
    const double a = aval[ka];
    for (int kb = brp[k]; kb < brp[k + 1]; ++kb) {
      const int q = tpos[t++];
      if (q >= 0) cval[q] += a * bval[kb];
    }
  }
}

// the row of every entry of a CSR pattern
__global__ void k_entry_rows(int n, const int *rp, int *row) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) row[e] = i;
}

// Galerkin product A_c = R (A P), one thread per ENTRY (c, j) of A_c: the sum
// over i in R's row c (CSR order) of R[c, i] (A P)[i, j], the (A P) entry
// found by a search in row i.  Per entry these are the terms, in the order,
// that a row-by-row accumulation adds them, with enough threads to hide the
// gather latency on the coarse rows (one thread per coarse row left most of
// the multiprocessors idle).
__global__ void k_galerkin_entries(long nnz, const int *__restrict__ crow, const int *__restrict__ ccol,
                                   const int *__restrict__ rrp, const int *__restrict__ rcol,
                                   const double *__restrict__ rval, const int *__restrict__ aprp,
                                   const int *__restrict__ apcol, const double *__restrict__ apval,
                                   double *cval) {
  const long e = (long)blockIdx.x * TPB + threadIdx.x;
  if (e >= nnz) return;
  const int c = crow[e], j = ccol[e];
  double sum = 0.0;
  for (int ka = rrp[c]; ka < rrp[c + 1]; ++ka) {
    const int i = rcol[ka];
    int lo = aprp[i], hi = aprp[i + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (apcol[mid] < j) lo = mid + 1;
      else hi = mid;
    }
    if (lo < aprp[i + 1] && apcol[lo] == j) sum += rval[ka] * apval[lo];
  }
  cval[e] = sum;
}

__global__ void k_col_count(int nnz, const int *col, int *cnt) {
  const int e = blockIdx.x * TPB + threadIdx.x;
  if (e < nnz) atomicAdd(&cnt[col[e]], 1);
}

__global__ void k_transpose_fill(int nrows, const int *rp, const int *col, int *fill, int *tcol, int *tmap) {
  const int r = blockIdx.x * TPB + threadIdx.x;
  if (r >= nrows) return;
  for (int e = rp[r]; e < rp[r + 1]; ++e) {
    const int d = atomicAdd(&fill[col[e]], 1);
    tcol[d] = r;
    tmap[d] = e;
  }
}

// rows of the transpose sorted by column (the fill order above is not fixed)
__global__ void k_transpose_sort(int nrows, const int *rp, int *tcol, int *tmap) {
  const int r = blockIdx.x * TPB + threadIdx.x;
  if (r >= nrows) return;
  for (int a = rp[r] + 1; a < rp[r + 1]; ++a) {
    const int c = tcol[a], m = tmap[a];
    int b = a - 1;
    while (b >= rp[r] && tcol[b] > c) {
      tcol[b + 1] = tcol[b];
      tmap[b + 1] = tmap[b];
      --b;
    }
    tcol[b + 1] = c;
    tmap[b + 1] = m;
  }
}

__global__ void k_diag_pos(int n, const int *rp, const int *col, int *diag, int *err) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  int d = -1;
  for (int k = rp[i]; k < rp[i + 1]; ++k)
    if (col[k] == i) d = k;
  if (d < 0) {
    atomicExch(err, 3);
    d = rp[i];
  }
  diag[i] = d;
}

// the +-1 start vector; *hn = its norm sqrt(n) (exact: the squares sum to n)
__global__ void k_power_init(int n, int level, double *x, double *hn) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  const uint64_t z = splitmix64_out(((uint64_t)(level + 64) << 32) + (uint64_t)i);
  x[i] = (z >> 63) ? 1.0 : -1.0;
  if (i == 0) *hn = sqrt((double)n);
}

// One power step: y = D^-1 (A x) / *hn, i.e. D^-1 A applied to the
// normalised x with the normalisation folded into the row (equal up to
// rounding; one FP64 division per thread instead of one per entry); the row
// sum in CSR order; per-block partial sums of y_i^2 in a fixed tree order
__global__ void k_power_step(int n, const int *__restrict__ rp, const int *__restrict__ col,
                             const double *__restrict__ val, const double *__restrict__ dinv,
                             const double *__restrict__ x, const double *__restrict__ hn, double *y,
                             double *partial) {
  __shared__ double sm[TPB];
  const double r = 1.0 / *hn;
  double acc = 0.0;
  for (int i = blockIdx.x * TPB + threadIdx.x; i < n; i += gridDim.x * TPB) {
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * x[col[k]];
    const double yi = dinv[i] * s * r;
    y[i] = yi;
    acc += yi * yi;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void k_rho(const double *gersh, const double *nrm, double *rho) {
  *rho = fmin(*gersh, kAmgPowerSafety * *nrm);
}

// P = T - (4 / (3 hi)) D^-1 (A T): at on P's pattern holds A T
__global__ void k_smooth_prolongator(int n, const int *__restrict__ prp, const int *__restrict__ pcol,
                                     const double *__restrict__ at, const int *__restrict__ agg,
                                     const double *__restrict__ tval, const double *__restrict__ dinv,
                                     const double *__restrict__ rho, double *pval) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  const double omega = 4.0 / (3.0 * *rho);
  const double s = omega * dinv[i];
  for (int e = prp[i]; e < prp[i + 1]; ++e) pval[e] = (pcol[e] == agg[i] ? tval[i] : 0.0) - s * at[e];
}

__global__ void k_gather_pos(int n, const int *map, const double *src, double *dst) {
  const int e = blockIdx.x * TPB + threadIdx.x;
  if (e < n) dst[e] = src[map[e]];
}

template <typename Tout>
__global__ void k_to(long n, const double *in, Tout *out) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) out[i] = (Tout)in[i];
}

template <typename Tin>
__global__ void k_from(long n, const Tin *in, double *out) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

}  // namespace

// One level of the hierarchy.
struct AmgLevel {
  Pattern A;                    // device + host copies, SELL view
  double *val = nullptr;        // FP64 CSR values (owned)
  int *diag = nullptr;
  double *dinv = nullptr;       // FP64 1 / a_ii
  double *gersh = nullptr;      // device scalar: Gershgorin bound
  double *rho = nullptr;        // device scalar: spectral bound hi_l
  // to level l + 1 (empty on the coarsest)
  int *agg = nullptr;
  double *tval = nullptr;
  int *iota = nullptr;          // T's row pointers (one entry per row)
  Transfer tr;                  // P (n_l x n_{l+1}) and R = P^T
  int *rmap = nullptr;          // position in P of every R entry
  Pattern AP;                   // pattern of A P (device only)
  double *apval = nullptr;
  double *atval = nullptr;      // A T on P's pattern
  // term positions of the products A T (in P) and A P (in AP): row pointers
  // and positions; the row of every entry of the next level's operator
  int *at_ptr = nullptr, *at_pos = nullptr, *ap_ptr = nullptr, *ap_pos = nullptr;
  int *next_rows = nullptr;
};

struct AmgHandle {
  int n = 0, nnz = 0, precision = 0;
  cudaStream_t s = nullptr;
  bool own_stream = true;       // false: the caller's stream (amg_attach)
  Arena ar;
  std::vector<std::unique_ptr<AmgLevel>> lv;
  double *partial = nullptr, *sc = nullptr, *px = nullptr, *py = nullptr;
  int *ictl = nullptr;          // [0] error flag [1] undecided count [2] scan total
  double *pinned = nullptr;     // host, 16 doubles
  int *pinned_i = nullptr;      // host, 4 ints
  double *a0sell = nullptr;     // level-0 values in SELL order (FP64 operator of the solve)
  std::unique_ptr<MGHier<double>> mg64;
  std::unique_ptr<MGHier<float>> mg32;
  KrylovWork ws;

  ~AmgHandle() {
    if (s) cudaStreamSynchronize(s);
    mg64.reset();
    mg32.reset();
    ar.release();
    if (pinned) cudaFreeHost(pinned);
    if (pinned_i) cudaFreeHost(pinned_i);
    if (s && own_stream) cudaStreamDestroy(s);
  }

  int read_int(const int *dev) {
    CHNSS_CK(cudaMemcpyAsync(pinned_i, dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CHNSS_CK(cudaStreamSynchronize(s));
    return pinned_i[0];
  }
  void clear_flag() { CHNSS_CK(cudaMemsetAsync(ictl, 0, 3 * sizeof(int), s)); }
  void check_flag(const char *what) {
    const int e = read_int(ictl);
    if (e == 1) throw Error{CHNSS_ERR_CUDA, std::string(what) + ": a node is not within distance 2 of a root"};
    if (e == 2)
      throw Error{CHNSS_ERR_ARG, std::string(what) + ": a product row has more than " + std::to_string(kAmgMaxRow) +
                                     " entries"};
    if (e == 3) throw Error{CHNSS_ERR_ARG, std::string(what) + ": a row without its diagonal entry"};
  }

  // exclusive scan of cnt[0..n) into rp[0..n), rp[n] = total (returns it)
  int scan(int n_, const int *cnt, int *rp) {
    k_scan<<<1, 1024, 0, s>>>(n_, cnt, rp, ictl + 2);
    CHNSS_LAUNCH_CK();
    CHNSS_CK(cudaMemcpyAsync(rp + n_, ictl + 2, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return read_int(ictl + 2);
  }

  // pattern of A B (device arrays + host copies), rows = A's rows
  void product_pattern(const Pattern &A, const int *brp, const int *bcol, int bcols, Pattern &C, const char *what) {
    C.nrows = A.nrows;
    C.ncols = bcols;
    int *cnt = ar.alloc<int>(A.nrows);
    clear_flag();
    k_product_count<<<nblk(A.nrows) * 2, 128, 0, s>>>(A.nrows, A.rowptr, A.col, brp, bcol, cnt, ictl);
    CHNSS_LAUNCH_CK();
    check_flag(what);
    C.rowptr = ar.alloc<int>(A.nrows + 1);
    C.nnz = scan(A.nrows, cnt, C.rowptr);
    C.col = ar.alloc<int>(C.nnz);
    k_product_fill<<<nblk(A.nrows) * 2, 128, 0, s>>>(A.nrows, A.rowptr, A.col, brp, bcol, C.rowptr, C.col);
    CHNSS_LAUNCH_CK();
  }

  // term positions of A B in C (C: the pattern of A B)
  void product_terms(const Pattern &A, const int *brp, const int *bcol, const Pattern &C, int **tptr, int **tpos) {
    int *cnt = ar.alloc<int>(A.nrows);
    k_product_terms<<<nblk(A.nrows), TPB, 0, s>>>(A.nrows, A.rowptr, A.col, brp, cnt);
    CHNSS_LAUNCH_CK();
    *tptr = ar.alloc<int>(A.nrows + 1);
    const int terms = scan(A.nrows, cnt, *tptr);
    *tpos = ar.alloc<int>(terms);
    k_product_positions<<<nblk(A.nrows), TPB, 0, s>>>(A.nrows, A.rowptr, A.col, brp, bcol, C.rowptr, C.col, *tptr,
                                                      *tpos);
    CHNSS_LAUNCH_CK();
  }

  void download(Pattern &P) {
    P.h_rowptr.resize(P.nrows + 1);
    P.h_col.resize(P.nnz);
    CHNSS_CK(cudaMemcpyAsync(P.h_rowptr.data(), P.rowptr, (P.nrows + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (P.nnz)
      CHNSS_CK(cudaMemcpyAsync(P.h_col.data(), P.col, P.nnz * sizeof(int), cudaMemcpyDeviceToHost, s));
    CHNSS_CK(cudaStreamSynchronize(s));
  }

  // symbolic setup of level l -> l + 1; false when aggregation does not
  // shrink the level (then l stays the coarsest)
  bool coarsen(int l) {
    AmgLevel &L = *lv[l];
    const int nl = L.A.nrows;
    uint64_t *base = ar.alloc<uint64_t>(nl), *state = ar.alloc<uint64_t>(nl), *m1 = ar.alloc<uint64_t>(nl);
    k_mis_init<<<nblk(nl), TPB, 0, s>>>(nl, l, base, state);
    CHNSS_LAUNCH_CK();
    int rounds = 0;
    while (true) {
      CHNSS_CK(cudaMemsetAsync(ictl + 1, 0, sizeof(int), s));
      k_mis_max1<<<nblk(nl), TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, state, base, m1);
      CHNSS_LAUNCH_CK();
      k_mis_max2<<<nblk(nl), TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, m1, base, state, ictl + 1);
      CHNSS_LAUNCH_CK();
      ++rounds;
      if (read_int(ictl + 1) == 0) break;
      if (rounds >= kAmgMaxRounds) throw Error{CHNSS_ERR_CUDA, "aggregation: independent-set rounds did not end"};
    }
    int *flag = ar.alloc<int>(nl), *rootnum = ar.alloc<int>(nl + 1), *agg1 = ar.alloc<int>(nl);
    k_root_flag<<<nblk(nl), TPB, 0, s>>>(nl, state, flag);
    CHNSS_LAUNCH_CK();
    const int nagg = scan(nl, flag, rootnum);
    if (nagg < 1) throw Error{CHNSS_ERR_CUDA, "aggregation: no root"};
    if (nagg >= nl) return false;
    L.agg = ar.alloc<int>(nl);
    clear_flag();
    k_agg_pass1<<<nblk(nl), TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, state, base, rootnum, agg1);
    CHNSS_LAUNCH_CK();
    k_agg_pass2<<<nblk(nl), TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, base, agg1, L.agg, ictl);
    CHNSS_LAUNCH_CK();
    check_flag("aggregation");
    int *size = ar.alloc<int>(nagg);
    CHNSS_CK(cudaMemsetAsync(size, 0, nagg * sizeof(int), s));
    k_agg_size<<<nblk(nl), TPB, 0, s>>>(nl, L.agg, size);
    CHNSS_LAUNCH_CK();
    L.tval = ar.alloc<double>(nl);
    L.iota = ar.alloc<int>(nl + 1);
    k_tval<<<nblk(nl + 1), TPB, 0, s>>>(nl, L.agg, size, L.tval, L.iota);
    CHNSS_LAUNCH_CK();
    // P = pattern(A T)
    Pattern &P = L.tr.P;
    product_pattern(L.A, L.iota, L.agg, nagg, P, "prolongator");
    // R = P^T with the position map
    Pattern &R = L.tr.R;
    R.nrows = nagg;
    R.ncols = nl;
    R.nnz = P.nnz;
    int *cnt = ar.alloc<int>(nagg);
    CHNSS_CK(cudaMemsetAsync(cnt, 0, nagg * sizeof(int), s));
    k_col_count<<<nblk(P.nnz), TPB, 0, s>>>(P.nnz, P.col, cnt);
    CHNSS_LAUNCH_CK();
    R.rowptr = ar.alloc<int>(nagg + 1);
    scan(nagg, cnt, R.rowptr);
    int *fill = ar.alloc<int>(nagg + 1);
    CHNSS_CK(cudaMemcpyAsync(fill, R.rowptr, (nagg + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
    R.col = ar.alloc<int>(R.nnz);
    L.rmap = ar.alloc<int>(R.nnz);
    k_transpose_fill<<<nblk(nl), TPB, 0, s>>>(nl, P.rowptr, P.col, fill, R.col, L.rmap);
    CHNSS_LAUNCH_CK();
    k_transpose_sort<<<nblk(nagg), TPB, 0, s>>>(nagg, R.rowptr, R.col, L.rmap);
    CHNSS_LAUNCH_CK();
    // pattern(A P) and A_{l+1} = pattern(R (A P))
    product_pattern(L.A, P.rowptr, P.col, nagg, L.AP, "A P");
    auto next = std::make_unique<AmgLevel>();
    product_pattern(R, L.AP.rowptr, L.AP.col, nagg, next->A, "coarse operator");
    // term positions of A T and A P (numeric setup without searches); the row
    // of every coarse-operator entry (the Galerkin product runs per entry)
    product_terms(L.A, L.iota, L.agg, P, &L.at_ptr, &L.at_pos);
    product_terms(L.A, P.rowptr, P.col, L.AP, &L.ap_ptr, &L.ap_pos);
    L.next_rows = ar.alloc<int>(next->A.nnz);
    k_entry_rows<<<nblk(nagg), TPB, 0, s>>>(nagg, next->A.rowptr, L.next_rows);
    CHNSS_LAUNCH_CK();
    // host copies and SELL views of the patterns the V-cycle sweeps
    download(P);
    download(R);
    download(next->A);
    build_sell(ar, P);
    build_sell(ar, R);
    build_sell(ar, next->A);
    L.tr.Pv = ar.alloc<double>(P.nnz);
    L.tr.Rv = ar.alloc<double>(R.nnz);
    L.tr.Ps = ar.alloc<double>(P.sell.nent);
    L.tr.Rs = ar.alloc<double>(R.sell.nent);
    L.tr.Ps32 = ar.alloc<float>(P.sell.nent);
    L.tr.Rs32 = ar.alloc<float>(R.sell.nent);
    L.atval = ar.alloc<double>(P.nnz);
    L.apval = ar.alloc<double>(L.AP.nnz);
    next->val = ar.alloc<double>(next->A.nnz);
    lv.push_back(std::move(next));
    level_scalars(*lv.back());
    return true;
  }

  void level_scalars(AmgLevel &L) {
    const int nl = L.A.nrows;
    L.diag = ar.alloc<int>(nl);
    clear_flag();
    k_diag_pos<<<nblk(nl), TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, L.diag, ictl);
    CHNSS_LAUNCH_CK();
    check_flag("level operator");
    L.dinv = ar.alloc<double>(nl);
    L.gersh = ar.alloc<double>(1);
    L.rho = ar.alloc<double>(1);
  }

  // spectral bound of D^-1 A_l (dinv and the Gershgorin bound first), on st
  void spectral_bound(int l, cudaStream_t st) {
    cudaStream_t s = st;
    AmgLevel &L = *lv[l];
    const int nl = L.A.nrows;
    jacobi_csr<double>(L.A, L.val, L.diag, L.dinv, L.gersh, partial, s);
    k_power_init<<<nblk(nl), TPB, 0, s>>>(nl, l, px, sc + 1);
    CHNSS_LAUNCH_CK();
    const int nb = std::min(nblk(nl), kReduceMaxBlocks);
    double *cur = px, *nxt = py;
    for (int k = 0; k < kAmgPowerSteps; ++k) {
      // nxt = D^-1 A (cur / ||cur||); then ||nxt|| in sc[1] for the next step
      k_power_step<<<nb, TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, L.val, L.dinv, cur, sc + 1, nxt, partial);
      CHNSS_LAUNCH_CK();
      sum_partials(nb, 1, partial, sc, s);
      set_scalar(sc + 1, sc, 1.0, true, s);
      std::swap(cur, nxt);
    }
    k_rho<<<1, 1, 0, s>>>(L.gersh, sc + 1, L.rho);
    CHNSS_LAUNCH_CK();
  }

  // numeric setup of every level from the current level-0 values, on st
  // (kernels and device copies only: no synchronisation)
  void levels_numeric(cudaStream_t st) {
    cudaStream_t s = st;
    const int nlev = (int)lv.size();
    for (int l = 0; l < nlev; ++l) {
      spectral_bound(l, s);
      if (l == nlev - 1) break;
      AmgLevel &L = *lv[l], &N = *lv[l + 1];
      const int nl = L.A.nrows;
      const Pattern &P = L.tr.P, &R = L.tr.R;
      k_product_values_mapped<<<nblk(nl), TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, L.val, L.iota, L.tval, P.rowptr,
                                                       L.at_ptr, L.at_pos, L.atval);
      CHNSS_LAUNCH_CK();
      k_smooth_prolongator<<<nblk(nl), TPB, 0, s>>>(nl, P.rowptr, P.col, L.atval, L.agg, L.tval, L.dinv, L.rho,
                                                    L.tr.Pv);
      CHNSS_LAUNCH_CK();
      k_gather_pos<<<nblk(R.nnz), TPB, 0, s>>>(R.nnz, L.rmap, L.tr.Pv, L.tr.Rv);
      CHNSS_LAUNCH_CK();
      k_product_values_mapped<<<nblk(nl), TPB, 0, s>>>(nl, L.A.rowptr, L.A.col, L.val, P.rowptr, L.tr.Pv,
                                                       L.AP.rowptr, L.ap_ptr, L.ap_pos, L.apval);
      CHNSS_LAUNCH_CK();
      k_galerkin_entries<<<nblk(N.A.nnz), TPB, 0, s>>>(N.A.nnz, L.next_rows, N.A.col, R.rowptr, R.col, L.tr.Rv,
                                                       L.AP.rowptr, L.AP.col, L.apval, N.val);
      CHNSS_LAUNCH_CK();
      sell_gather<double>(P.sell, 1, L.tr.Pv, L.tr.Ps, s);
      sell_gather<double>(R.sell, 1, L.tr.Rv, L.tr.Rs, s);
      sell_gather<float>(P.sell, 1, L.tr.Pv, L.tr.Ps32, s);
      sell_gather<float>(R.sell, 1, L.tr.Rv, L.tr.Rs32, s);
    }
  }

  // the handle's own numeric setup: the levels, the FP64 operator of the
  // solve and the V-cycle data, then a synchronisation
  void numeric() {
    levels_numeric(s);
    sell_gather<double>(lv[0]->A.sell, 1, lv[0]->val, a0sell, s);
    if (mg64) mg64->setup(s);
    else mg32->setup(s);
    CHNSS_CK(cudaStreamSynchronize(s));
  }

  template <typename T>
  void make_mg(std::unique_ptr<MGHier<T>> &mg) {
    mg = std::make_unique<MGHier<T>>();
    std::vector<const Pattern *> pats;
    std::vector<const int *> diags;
    std::vector<const double *> vals;
    std::vector<const Transfer *> trs;
    for (size_t l = 0; l < lv.size(); ++l) {
      pats.push_back(&lv[l]->A);
      diags.push_back(lv[l]->diag);
      vals.push_back(lv[l]->val);
      mg->hi_ext.push_back(lv[l]->rho);
      if (l + 1 < lv.size()) trs.push_back(&lv[l]->tr);
    }
    mg->init(ar, 0, false, pats, diags, vals, trs, partial);
  }

  void vcycle(const double *b, double *x) {
    const long n0 = n;
    if (mg64) {
      k_to<double><<<nblk(n0), TPB, 0, s>>>(n0, b, mg64->input());
      CHNSS_LAUNCH_CK();
      mg64->apply(s);
      k_from<double><<<nblk(n0), TPB, 0, s>>>(n0, mg64->output(), x);
      CHNSS_LAUNCH_CK();
    } else {
      k_to<float><<<nblk(n0), TPB, 0, s>>>(n0, b, mg32->input());
      CHNSS_LAUNCH_CK();
      mg32->apply(s);
      k_from<float><<<nblk(n0), TPB, 0, s>>>(n0, mg32->output(), x);
      CHNSS_LAUNCH_CK();
    }
  }
};

AmgHandle *amg_attach(const Pattern &P0, double *val0, cudaStream_t st) {
  if (P0.nrows != P0.ncols || P0.nrows < 1) throw Error{CHNSS_ERR_ARG, "smoothed aggregation needs a square operator"};
  auto h = std::make_unique<AmgHandle>();
  h->n = P0.nrows;
  h->nnz = P0.nnz;
  h->s = st;
  h->own_stream = false;
  CHNSS_CK(cudaHostAlloc((void **)&h->pinned, 16 * sizeof(double), cudaHostAllocDefault));
  CHNSS_CK(cudaHostAlloc((void **)&h->pinned_i, 4 * sizeof(int), cudaHostAllocDefault));
  h->partial = h->ar.alloc<double>(64L * kReduceMaxBlocks);
  h->sc = h->ar.alloc<double>(8);
  h->ictl = h->ar.alloc<int>(4);
  h->px = h->ar.alloc<double>(h->n);
  h->py = h->ar.alloc<double>(h->n);
  auto l0 = std::make_unique<AmgLevel>();
  l0->A = P0;                     // the caller's arrays (this arena never frees them)
  l0->val = val0;
  h->lv.push_back(std::move(l0));
  h->level_scalars(*h->lv[0]);
  while (h->lv.back()->A.nrows > kAmgCoarseRows && (int)h->lv.size() < kAmgMaxLevels)
    if (!h->coarsen((int)h->lv.size() - 1)) break;
  if (h->lv.size() == 1 && h->n > kAmgCoarseRows)
    throw Error{CHNSS_ERR_ARG, "aggregation does not coarsen this operator"};
  CHNSS_CK(cudaStreamSynchronize(st));
  return h.release();
}

void amg_refresh(AmgHandle *h, cudaStream_t st) { h->levels_numeric(st); }

void amg_levels(AmgHandle *h, std::vector<const Pattern *> &pats, std::vector<const int *> &diags,
                std::vector<const double *> &vals, std::vector<const Transfer *> &trs,
                std::vector<const double *> &his) {
  pats.clear();
  diags.clear();
  vals.clear();
  trs.clear();
  his.clear();
  for (size_t l = 0; l < h->lv.size(); ++l) {
    pats.push_back(&h->lv[l]->A);
    diags.push_back(h->lv[l]->diag);
    vals.push_back(h->lv[l]->val);
    his.push_back(h->lv[l]->rho);
    if (l + 1 < h->lv.size()) trs.push_back(&h->lv[l]->tr);
  }
}

void amg_release(AmgHandle *h) { delete h; }

namespace {
// A (FP64, level-0 SELL values) with one V-cycle as the right preconditioner
struct AmgOperator : LinearOperator {
  AmgHandle *h;
  explicit AmgOperator(AmgHandle *h_) : h(h_) {}
  long size() const override { return h->n; }
  void apply(const double *x, double *y, cudaStream_t s) override {
    SpmvArgs none;
    spmv_sell<double>(h->lv[0]->A, h->a0sell, 1, x, y, SPMV_PLAIN, none, s);
  }
  void precond(const double *r, double *z, cudaStream_t) override { h->vcycle(r, z); }
};

chnss_status amg_fail(chnss_status st, const std::string &msg) {
  set_global_error(msg);
  return st;
}
}  // namespace

}  // namespace chnss

using namespace chnss;

struct chnss_amg {
  AmgHandle h;
};

#define AMG_TRY try {
#define AMG_CATCH                                                                       \
  }                                                                                     \
  catch (const Error &e) { return amg_fail(e.status, e.msg); }                          \
  catch (const std::bad_alloc &) { return amg_fail(CHNSS_ERR_OOM, "host allocation failed"); } \
  catch (const std::exception &e) { return amg_fail(CHNSS_ERR_CUDA, e.what()); }

chnss_status chnss_amg_create(int n, int nnz, const int *rowptr, const int *col, const double *val, int precision,
                              chnss_amg_t *out) {
  if (!out) return amg_fail(CHNSS_ERR_ARG, "null output handle");
  *out = nullptr;
  if (n < 1 || nnz < n || !rowptr || !col || !val) return amg_fail(CHNSS_ERR_ARG, "bad size or null array");
  if (precision != 0 && precision != 1) return amg_fail(CHNSS_ERR_ARG, "precision must be 0 (FP64) or 1 (FP32)");
  std::unique_ptr<chnss_amg> H;
  AMG_TRY
  // validate the pattern on the host before any device work
  std::vector<int> hrp(n + 1), hcol(nnz);
  CHNSS_CK(cudaMemcpy(hrp.data(), rowptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (hrp[0] != 0 || hrp[n] != nnz) throw Error{CHNSS_ERR_ARG, "rowptr[0] must be 0 and rowptr[n] = nnz"};
  for (int i = 0; i < n; ++i)
    if (hrp[i + 1] < hrp[i]) throw Error{CHNSS_ERR_ARG, "rowptr must be non-decreasing"};
  CHNSS_CK(cudaMemcpy(hcol.data(), col, nnz * sizeof(int), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    bool has_diag = false;
    for (int k = hrp[i]; k < hrp[i + 1]; ++k) {
      const int c = hcol[k];
      if (c < 0 || c >= n) throw Error{CHNSS_ERR_ARG, "column out of range"};
      if (k > hrp[i] && hcol[k - 1] >= c) throw Error{CHNSS_ERR_ARG, "columns must be sorted and unique in each row"};
      has_diag |= c == i;
    }
    if (!has_diag) throw Error{CHNSS_ERR_ARG, "every row needs its diagonal entry"};
  }
  for (int i = 0; i < n; ++i)   // (rows sorted: binary search)
    for (int k = hrp[i]; k < hrp[i + 1]; ++k) {
      const int c = hcol[k];
      const int *b = hcol.data() + hrp[c], *e = hcol.data() + hrp[c + 1];
      if (!std::binary_search(b, e, i)) throw Error{CHNSS_ERR_ARG, "the pattern must be structurally symmetric"};
    }
  H = std::make_unique<chnss_amg>();
  AmgHandle &h = H->h;
  h.n = n;
  h.nnz = nnz;
  h.precision = precision;
  CHNSS_CK(cudaStreamCreateWithFlags(&h.s, cudaStreamNonBlocking));
  CHNSS_CK(cudaHostAlloc((void **)&h.pinned, 16 * sizeof(double), cudaHostAllocDefault));
  CHNSS_CK(cudaHostAlloc((void **)&h.pinned_i, 4 * sizeof(int), cudaHostAllocDefault));
  h.partial = h.ar.alloc<double>(64L * kReduceMaxBlocks);
  h.sc = h.ar.alloc<double>(8);
  h.ictl = h.ar.alloc<int>(4);
  h.px = h.ar.alloc<double>(n);
  h.py = h.ar.alloc<double>(n);
  auto l0 = std::make_unique<AmgLevel>();
  l0->A.nrows = l0->A.ncols = n;
  l0->A.nnz = nnz;
  l0->A.h_rowptr = std::move(hrp);
  l0->A.h_col = std::move(hcol);
  upload_pattern(h.ar, l0->A);
  l0->val = h.ar.alloc<double>(nnz);
  CHNSS_CK(cudaMemcpyAsync(l0->val, val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, h.s));
  h.lv.push_back(std::move(l0));
  h.level_scalars(*h.lv[0]);
  h.a0sell = h.ar.alloc<double>(h.lv[0]->A.sell.nent);
  // symbolic levels: needs the level-l values only for the next level's
  // pattern, which is value-independent (theta = 0)
  while (h.lv.back()->A.nrows > kAmgCoarseRows && (int)h.lv.size() < kAmgMaxLevels)
    if (!h.coarsen((int)h.lv.size() - 1)) break;
  if (h.lv.size() == 1 && n > kAmgCoarseRows)
    throw Error{CHNSS_ERR_ARG, "aggregation does not coarsen this matrix (no off-diagonal entries)"};
  if (precision == 0) h.make_mg(h.mg64);
  else h.make_mg(h.mg32);
  h.ws.init(h.ar, kAmgRestart, n, h.pinned);
  h.numeric();
  *out = H.release();
  return CHNSS_OK;
  AMG_CATCH
}

chnss_status chnss_amg_update(chnss_amg_t H, const double *val) {
  if (!H || !val) return amg_fail(CHNSS_ERR_ARG, "null argument");
  AMG_TRY
  AmgHandle &h = H->h;
  CHNSS_CK(cudaMemcpyAsync(h.lv[0]->val, val, h.nnz * sizeof(double), cudaMemcpyDeviceToDevice, h.s));
  h.numeric();
  return CHNSS_OK;
  AMG_CATCH
}

chnss_status chnss_amg_levels(chnss_amg_t H, int *nlevels, int *rows, int *nnz, int *pnnz) {
  if (!H || !nlevels) return amg_fail(CHNSS_ERR_ARG, "null argument");
  const AmgHandle &h = H->h;
  *nlevels = (int)h.lv.size();
  for (size_t l = 0; l < h.lv.size(); ++l) {
    if (rows) rows[l] = h.lv[l]->A.nrows;
    if (nnz) nnz[l] = h.lv[l]->A.nnz;
    if (pnnz) pnnz[l] = l + 1 < h.lv.size() ? h.lv[l]->tr.P.nnz : 0;
  }
  return CHNSS_OK;
}

chnss_status chnss_amg_export_level(chnss_amg_t H, int level, int *agg, double *hi, int *a_rowptr, int *a_col,
                                    double *a_val, int *p_rowptr, int *p_col, double *p_val) {
  if (!H) return amg_fail(CHNSS_ERR_ARG, "null handle");
  AMG_TRY
  AmgHandle &h = H->h;
  if (level < 0 || level >= (int)h.lv.size()) throw Error{CHNSS_ERR_ARG, "level out of range"};
  const AmgLevel &L = *h.lv[level];
  const bool last = level + 1 == (int)h.lv.size();
  if (last && (agg || p_rowptr || p_col || p_val)) throw Error{CHNSS_ERR_ARG, "the coarsest level has no prolongator"};
  CHNSS_CK(cudaStreamSynchronize(h.s));
  const int nl = L.A.nrows;
  if (agg) CHNSS_CK(cudaMemcpy(agg, L.agg, nl * sizeof(int), cudaMemcpyDeviceToHost));
  if (hi) CHNSS_CK(cudaMemcpy(hi, L.rho, sizeof(double), cudaMemcpyDeviceToHost));
  if (a_rowptr) CHNSS_CK(cudaMemcpy(a_rowptr, L.A.rowptr, (nl + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (a_col) CHNSS_CK(cudaMemcpy(a_col, L.A.col, L.A.nnz * sizeof(int), cudaMemcpyDeviceToHost));
  if (a_val) CHNSS_CK(cudaMemcpy(a_val, L.val, L.A.nnz * sizeof(double), cudaMemcpyDeviceToHost));
  if (p_rowptr) CHNSS_CK(cudaMemcpy(p_rowptr, L.tr.P.rowptr, (nl + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (p_col) CHNSS_CK(cudaMemcpy(p_col, L.tr.P.col, L.tr.P.nnz * sizeof(int), cudaMemcpyDeviceToHost));
  if (p_val) CHNSS_CK(cudaMemcpy(p_val, L.tr.Pv, L.tr.P.nnz * sizeof(double), cudaMemcpyDeviceToHost));
  return CHNSS_OK;
  AMG_CATCH
}

chnss_status chnss_amg_vcycle(chnss_amg_t H, const double *b, double *x) {
  if (!H || !b || !x) return amg_fail(CHNSS_ERR_ARG, "null argument");
  AMG_TRY
  AmgHandle &h = H->h;
  const char *pb = (const char *)b, *px_ = (const char *)x;
  if (pb < px_ + h.n * sizeof(double) && px_ < pb + h.n * sizeof(double))
    throw Error{CHNSS_ERR_ARG, "b and x overlap"};
  h.vcycle(b, x);
  CHNSS_CK(cudaStreamSynchronize(h.s));
  return CHNSS_OK;
  AMG_CATCH
}

chnss_status chnss_amg_solve(chnss_amg_t H, const double *b, double *x, double rtol, double atol, int maxit,
                             chnss_solve_info *info) {
  if (!H || !b || !x) return amg_fail(CHNSS_ERR_ARG, "null argument");
  if (maxit < 1 || !(rtol >= 0.0) || !(atol >= 0.0)) return amg_fail(CHNSS_ERR_ARG, "bad tolerance or maxit");
  AMG_TRY
  AmgHandle &h = H->h;
  const char *pb = (const char *)b, *px_ = (const char *)x;
  if (pb < px_ + h.n * sizeof(double) && px_ < pb + h.n * sizeof(double))
    throw Error{CHNSS_ERR_ARG, "b and x overlap"};
  AmgOperator op(&h);
  const chnss_status st = fgmres(op, b, x, rtol, atol, maxit, h.ws, info, h.s);
  CHNSS_CK(cudaStreamSynchronize(h.s));
  if (st != CHNSS_OK) set_global_error("amg solve: status " + std::to_string((int)st));
  return st;
  AMG_CATCH
}

void chnss_amg_destroy(chnss_amg_t H) { delete H; }
