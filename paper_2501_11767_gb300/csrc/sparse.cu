// Sparse matrix-vector products, vector updates and deterministic
// reductions.  SpMV uses LANES threads per row (sub-warp CSR-vector): the
// lanes of a group read consecutive entries of the row, so the value and
// column streams are read coalesced; partial sums are combined with warp
// shuffles.  Every reduction uses a grid size that depends only on the
// vector length and the device's multiprocessor count and sums in a fixed
// order, so results are bit-reproducible on a given device.
#include <atomic>
#include <cmath>

#include "kernels.h"

namespace chnss {
namespace {

constexpr int TPB = 256;
inline int nblocks(long n, int per_block) { return (int)((n + per_block - 1) / per_block); }

template <int LANES, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, LANES);
  return v;
}

// Chebyshev step of one row: c0 u + c2 dinv (b - A u) (+ c1 w)
template <typename T>
__device__ __forceinline__ T cheb_row(const double *coef, T ui, T di, T bi, T acc, bool has_w, T wi) {
  const T c0 = (T)coef[0], c1 = (T)coef[1], c2 = (T)coef[2];
  T v = c0 * ui + c2 * di * (bi - acc);
  if (has_w) v += c1 * wi;
  return v;
}

template <typename T>
__device__ __forceinline__ void epilogue(int mode, long i, T acc, const T *u, T *out, const SpmvArgs &a,
                                         const double *coef) {
  if (mode == SPMV_PLAIN) {
    out[i] = acc;
  } else if (mode == SPMV_RES) {
    out[i] = static_cast<const T *>(a.b)[i] - acc;
  } else if (mode == SPMV_ADD) {
    out[i] += acc;
  } else {
    const T *w = static_cast<const T *>(a.w);
    out[i] = cheb_row<T>(coef, u[i], static_cast<const T *>(a.dinv)[i], static_cast<const T *>(a.b)[i], acc,
                         w != nullptr, w ? w[i] : (T)0);
  }
}

template <int LANES, typename T>
__global__ void __launch_bounds__(TPB) k_spmv_csr(int nrows, int ncomp, const int *__restrict__ rowptr,
                                                  const int *__restrict__ col, const T *__restrict__ val,
                                                  const T *__restrict__ u, T *out, int mode, SpmvArgs a) {
  const int lane = threadIdx.x % LANES;
  const int row = (blockIdx.x * TPB + threadIdx.x) / LANES;
  const bool live = row < nrows;
  const int b0 = live ? rowptr[row] : 0, b1 = live ? rowptr[row + 1] : 0;
  if (ncomp == 1) {
    T acc = 0;
    for (int k = b0 + lane; k < b1; k += LANES) acc += val[k] * u[col[k]];
    acc = group_sum<LANES>(acc);
    if (live && lane == 0) epilogue<T>(mode, row, acc, u, out, a, a.coef);
  } else {
    T acc0 = 0, acc1 = 0;
    for (int k = b0 + lane; k < b1; k += LANES) {
      const T w = val[k];
      const long c = 2L * col[k];
      acc0 += w * u[c];
      acc1 += w * u[c + 1];
    }
    acc0 = group_sum<LANES>(acc0);
    acc1 = group_sum<LANES>(acc1);
    if (live && lane == 0) {
      epilogue<T>(mode, 2L * row, acc0, u, out, a, a.coef);
      epilogue<T>(mode, 2L * row + 1, acc1, u, out, a, a.coef);
    }
  }
}

template <typename T>
struct Vec2 { T x, y; };

template <int LANES, typename T>
__global__ void __launch_bounds__(TPB) k_spmv_bsr2(int nrows, const int *__restrict__ rowptr,
                                                   const int *__restrict__ col, const T *__restrict__ val,
                                                   const T *__restrict__ u, T *out, int mode, SpmvArgs a) {
  const int lane = threadIdx.x % LANES;
  const int row = (blockIdx.x * TPB + threadIdx.x) / LANES;
  const bool live = row < nrows;
  const int b0 = live ? rowptr[row] : 0, b1 = live ? rowptr[row + 1] : 0;
  T acc0 = 0, acc1 = 0;
  for (int k = b0 + lane; k < b1; k += LANES) {
    const T *blk = val + 4L * k;
    const long c = 2L * col[k];
    const T x0 = u[c], x1 = u[c + 1];
    acc0 += blk[0] * x0 + blk[1] * x1;
    acc1 += blk[2] * x0 + blk[3] * x1;
  }
  acc0 = group_sum<LANES>(acc0);
  acc1 = group_sum<LANES>(acc1);
  if (live && lane == 0) {
    epilogue<T>(mode, 2L * row, acc0, u, out, a, a.coef);
    epilogue<T>(mode, 2L * row + 1, acc1, u, out, a, a.coef);
  }
}

// CH operator on the P1 pattern
__global__ void __launch_bounds__(TPB) k_spmv_ch(int nrows, const int *__restrict__ rowptr,
                                                 const int *__restrict__ col, const double *__restrict__ L,
                                                 const double *__restrict__ K, const double *__restrict__ K12,
                                                 const double *__restrict__ M, double a12, double a21, double a22,
                                                 const double *__restrict__ x, double *__restrict__ y) {
  constexpr int LANES = 8;
  const int lane = threadIdx.x % LANES;
  const int row = (blockIdx.x * TPB + threadIdx.x) / LANES;
  const bool live = row < nrows;
  const int b0 = live ? rowptr[row] : 0, b1 = live ? rowptr[row + 1] : 0;
  const double *x1 = x, *x2 = x + nrows;
  double s11 = 0, s12 = 0, s21 = 0, s22 = 0;
  for (int k = b0 + lane; k < b1; k += LANES) {
    const int c = col[k];
    const double u1 = x1[c], u2 = x2[c], kv = K[k];
    s11 += L[k] * u1;
    s12 += (K12 ? K12[k] : kv) * u2;
    s21 += kv * u1;
    s22 += M[k] * u2;
  }
  s11 = group_sum<LANES>(s11);
  s12 = group_sum<LANES>(s12);
  s21 = group_sum<LANES>(s21);
  s22 = group_sum<LANES>(s22);
  if (live && lane == 0) {
    y[row] = s11 + a12 * s12;
    y[nrows + row] = a21 * s21 + a22 * s22;
  }
}

__global__ void __launch_bounds__(TPB) k_spmv_b(int nrows, const int *__restrict__ rowptr,
                                                const int *__restrict__ col, const double *__restrict__ val,
                                                const double *__restrict__ v, double *__restrict__ y) {
  constexpr int LANES = 8;
  const int lane = threadIdx.x % LANES;
  const int row = (blockIdx.x * TPB + threadIdx.x) / LANES;
  const bool live = row < nrows;
  const int b0 = live ? rowptr[row] : 0, b1 = live ? rowptr[row + 1] : 0;
  double acc = 0;
  for (int k = b0 + lane; k < b1; k += LANES) {
    const long c = 2L * col[k];
    acc += val[2L * k] * v[c] + val[2L * k + 1] * v[c + 1];
  }
  acc = group_sum<LANES>(acc);
  if (live && lane == 0) y[row] = acc;
}

__global__ void __launch_bounds__(TPB) k_spmv_bt_add(int nrows, const int *__restrict__ rowptr,
                                                     const int *__restrict__ col, const double *__restrict__ val,
                                                     const double *__restrict__ p, double *__restrict__ yv) {
  constexpr int LANES = 4;
  const int lane = threadIdx.x % LANES;
  const int row = (blockIdx.x * TPB + threadIdx.x) / LANES;
  const bool live = row < nrows;
  const int b0 = live ? rowptr[row] : 0, b1 = live ? rowptr[row + 1] : 0;
  double a0 = 0, a1 = 0;
  for (int k = b0 + lane; k < b1; k += LANES) {
    const double q = p[col[k]];
    a0 += val[2L * k] * q;
    a1 += val[2L * k + 1] * q;
  }
  a0 = group_sum<LANES>(a0);
  a1 = group_sum<LANES>(a1);
  if (live && lane == 0) {
    yv[2L * row] += a0;
    yv[2L * row + 1] += a1;
  }
}

// --------------------------------------------------------------------------
// SELL-C-sigma kernels: one warp per slice of 32 rows, one thread per row,
// entry j of the slice's rows is contiguous, so every value and column load
// is one coalesced warp access and a thread's loads are independent.
template <typename T> struct V2t;
template <> struct V2t<float> { using type = float2; };
template <> struct V2t<double> { using type = double2; };

__device__ __forceinline__ float ldv(const float *p) { return *p; }
__device__ __forceinline__ double ldv(const double *p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

__device__ __forceinline__ void load_blk(const __nv_bfloat16 *p, float b[4]) {   // 8-byte aligned
  const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
  const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
  const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
  b[0] = lo.x; b[1] = lo.y; b[2] = hi.x; b[3] = hi.y;
}
__device__ __forceinline__ void load_blk(const float *p, float b[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
}
__device__ __forceinline__ void load_blk(const double *p, double b[4]) {
  const double2 v0 = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  b[0] = v0.x; b[1] = v0.y; b[2] = v1.x; b[3] = v1.y;
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T> __device__ __forceinline__ T from_double(double x) { return (T)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x) {
  return __double2bfloat16(x);   // round to nearest even
}

template <typename T>
__global__ void k_sell_gather(long nent, int ncomp, const int *__restrict__ map, const double *__restrict__ csr,
                              T *__restrict__ out) {
  const long e = (long)blockIdx.x * TPB + threadIdx.x;
  if (e >= nent) return;
  const int q = map[e];
  for (int c = 0; c < ncomp; ++c) out[e * ncomp + c] = from_double<T>(q >= 0 ? csr[(long)q * ncomp + c] : 0.0);
}

__global__ void k_sell_gather_t(long nent, int ncomp, const int *__restrict__ mapT, const double *__restrict__ csr,
                                double *__restrict__ out) {
  const long e = (long)blockIdx.x * TPB + threadIdx.x;
  if (e >= nent) return;
  const int q = mapT[e];
  if (ncomp == 1) {
    out[e] = q >= 0 ? csr[q] : 0.0;
  } else {   // 2x2 block: (c, d) <- (d, c)
    out[4 * e + 0] = q >= 0 ? csr[4L * q + 0] : 0.0;
    out[4 * e + 1] = q >= 0 ? csr[4L * q + 2] : 0.0;
    out[4 * e + 2] = q >= 0 ? csr[4L * q + 1] : 0.0;
    out[4 * e + 3] = q >= 0 ? csr[4L * q + 3] : 0.0;
  }
}

template <typename T, typename VT, int NC, bool VEC>
__global__ void __launch_bounds__(kSellMaxBlock) k_sell(int nslices, const int *__restrict__ sp, const int *__restrict__ rowid,
                                              const int *__restrict__ col, const VT *__restrict__ val,
                                              const T *__restrict__ u, T *out, int mode, SpmvArgs a) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  const int *cp = col + b0 + lane;
  const VT *vp = val + b0 + lane;
  T acc0 = 0, acc1 = 0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const int c = cp[j * 32];
    const T v = ldv(vp + j * 32);
    if (NC == 1) {
      acc0 += v * u[c];
    } else if (VEC) {
      const typename V2t<T>::type x = reinterpret_cast<const typename V2t<T>::type *>(u)[c];
      acc0 += v * x.x;
      acc1 += v * x.y;
    } else {
      acc0 += v * u[2L * c];
      acc1 += v * u[2L * c + 1];
    }
  }
  if (row < 0) return;
  if (NC == 1) {
    epilogue<T>(mode, row, acc0, u, out, a, a.coef);
  } else {
    epilogue<T>(mode, 2L * row, acc0, u, out, a, a.coef);
    epilogue<T>(mode, 2L * row + 1, acc1, u, out, a, a.coef);
  }
}

// Wide rows and few slices (the coarse levels of the 3D velocity hierarchy,
// the 3D divergence B): K warps share a slice, warp k summing the entries
// j = k, k + K, ... of the slice's 32 rows, so the dependent chain of gathers
// per thread is w / K long instead of w.  The K partial sums are added in
// warp order through shared memory, so the result is deterministic and
// independent of the launch's block size.  SPB slices per block.
template <typename T, typename VT, int K>
__global__ void __launch_bounds__(K >= 8 ? 32 * K : 256) k_sell_split(int nslices, const int *__restrict__ sp,
                                                                       const int *__restrict__ rowid,
                                                                       const int *__restrict__ col,
                                                                       const VT *__restrict__ val,
                                                                       const T *__restrict__ u, T *out, int mode,
                                                                       SpmvArgs a) {
  constexpr int SPB = K >= 8 ? 1 : 8 / K;
  __shared__ T part[SPB][K][32];
  const int ls = threadIdx.x / (32 * K), k = (threadIdx.x >> 5) % K, lane = threadIdx.x & 31;
  const int slice = blockIdx.x * SPB + ls;
  T acc = 0;
  if (slice < nslices) {
    const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
    const int *cp = col + b0 + lane;
    const VT *vp = val + b0 + lane;
#pragma unroll 4
    for (int j = k; j < w; j += K) acc += ldv(vp + j * 32) * u[cp[j * 32]];
  }
  part[ls][k][lane] = acc;
  __syncthreads();
  if (k != 0 || slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  if (row < 0) return;
  T sum = part[ls][0][lane];
#pragma unroll
  for (int q = 1; q < K; ++q) sum += part[ls][q][lane];
  epilogue<T>(mode, row, sum, u, out, a, a.coef);
}

// 3x3-block SELL (the 3D velocity operators; vectors interleaved, node c at
// 3 c .. 3 c + 2).  Entry e of a slice column holds a 3x3 block, value
// m = 3 r + d (row component r, column component d) at
// 9 (e - e % 32) + 32 m + e % 32, so each of the nine value loads of a warp
// is one coalesced access.  One node row per thread (K = 1), or K warps per
// slice with the partial sums added in warp order through shared memory, as
// k_sell_split; three FMAs per block row and component, in d order.
// k_sell_bsr2 with K warps per slice (coarse velocity levels with fewer
// slices than one wave of warps): warp k sums the entries j = k, k + K, ...,
// the K partial sums are added in warp order through shared memory
template <typename T, typename VT, int K>
__global__ void __launch_bounds__(256) k_sell_bsr2_split(int nslices, const int *__restrict__ sp,
                                                         const int *__restrict__ rowid, const int *__restrict__ col,
                                                         const VT *__restrict__ val, const T *__restrict__ u, T *out,
                                                         int mode, SpmvArgs a) {
  constexpr int SPB = 8 / K;
  __shared__ T part[SPB][K][2][32];
  const int ls = threadIdx.x / (32 * K), k = (threadIdx.x >> 5) % K, lane = threadIdx.x & 31;
  const int slice = blockIdx.x * SPB + ls;
  T acc0 = 0, acc1 = 0;
  if (slice < nslices) {
    const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
#pragma unroll 2
    for (int j = k; j < w; j += K) {
      const long e = b0 + (long)j * 32 + lane;
      const int c = col[e];
      T b[4];
      load_blk(val + 4 * e, b);
      const T x0 = u[2L * c], x1 = u[2L * c + 1];
      acc0 = fma_t(b[1], x1, fma_t(b[0], x0, acc0));
      acc1 = fma_t(b[3], x1, fma_t(b[2], x0, acc1));
    }
  }
  part[ls][k][0][lane] = acc0;
  part[ls][k][1][lane] = acc1;
  __syncthreads();
  if (k != 0 || slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  if (row < 0) return;
  T s0 = part[ls][0][0][lane], s1 = part[ls][0][1][lane];
#pragma unroll
  for (int q = 1; q < K; ++q) {
    s0 += part[ls][q][0][lane];
    s1 += part[ls][q][1][lane];
  }
  epilogue<T>(mode, 2L * row, s0, u, out, a, a.coef);
  epilogue<T>(mode, 2L * row + 1, s1, u, out, a, a.coef);
}

template <typename T, typename VT, int K>
__global__ void __launch_bounds__(K >= 8 ? 32 * K : 256) k_sell_bsr3(int nslices, const int *__restrict__ sp,
                                                                      const int *__restrict__ rowid,
                                                                      const int *__restrict__ col,
                                                                      const VT *__restrict__ val,
                                                                      const T *__restrict__ u, T *out, int mode,
                                                                      SpmvArgs a) {
  constexpr int SPB = K >= 8 ? 1 : 8 / K;
  const int ls = threadIdx.x / (32 * K), k = (threadIdx.x >> 5) % K, lane = threadIdx.x & 31;
  const int slice = blockIdx.x * SPB + ls;
  // U entries per batch, their loads written ahead of their FMAs; the
  // entries are summed in slice-column order either way
  constexpr int U = sizeof(T) == 8 ? 2 : 4;
  T acc[3] = {0, 0, 0};
  auto fma_blk = [&](const T (&v)[9], const T (&x)[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      acc[r] = fma_t(v[3 * r], x[0], acc[r]);
      acc[r] = fma_t(v[3 * r + 1], x[1], acc[r]);
      acc[r] = fma_t(v[3 * r + 2], x[2], acc[r]);
    }
  };
  if (slice < nslices) {
    const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
    int j = k;
    for (; j + (U - 1) * K < w; j += U * K) {
      int c[U];
      T v[U][9], x[U][3];
#pragma unroll
      for (int q = 0; q < U; ++q) c[q] = col[b0 + (long)(j + q * K) * 32 + lane];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const VT *vb = val + 9 * (b0 + (long)(j + q * K) * 32) + lane;
#pragma unroll
        for (int m = 0; m < 9; ++m) v[q][m] = ldv(vb + 32 * m);
      }
#pragma unroll
      for (int q = 0; q < U; ++q)
#pragma unroll
        for (int d = 0; d < 3; ++d) x[q][d] = u[3L * c[q] + d];
#pragma unroll
      for (int q = 0; q < U; ++q) fma_blk(v[q], x[q]);
    }
    for (; j < w; j += K) {
      const int c = col[b0 + (long)j * 32 + lane];
      const VT *vb = val + 9 * (b0 + (long)j * 32) + lane;
      T v[9], x[3];
#pragma unroll
      for (int m = 0; m < 9; ++m) v[m] = ldv(vb + 32 * m);
#pragma unroll
      for (int d = 0; d < 3; ++d) x[d] = u[3L * c + d];
      fma_blk(v, x);
    }
  }
  if (K > 1) {
    __shared__ T part[SPB][K][3][32];
#pragma unroll
    for (int r = 0; r < 3; ++r) part[ls][k][r][lane] = acc[r];
    __syncthreads();
    if (k != 0 || slice >= nslices) return;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      T sum = part[ls][0][r][lane];
#pragma unroll
      for (int q = 1; q < K; ++q) sum += part[ls][q][r][lane];
      acc[r] = sum;
    }
  }
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  if (row < 0) return;
#pragma unroll
  for (int r = 0; r < 3; ++r) epilogue<T>(mode, 3L * row + r, acc[r], u, out, a, a.coef);
}

// The coarsest level of a 3x3-block hierarchy solved by degree Chebyshev-
// Jacobi steps from zero, all in one block of 32 warps (levels of at most
// eight slices, 256 node rows): K = 32 / slices warps share a slice as in
// k_sell_bsr3, a block barrier between steps.  The same expressions as the
// per-launch form (k_scale_dinv, then SPMV_CHEB sweeps), so the iterate
// lands in x after the last step.
template <typename T, typename VT>
__global__ void __launch_bounds__(1024) k_cheb_bsr3_block(int nslices, int K, const int *__restrict__ sp,
                                                          const int *__restrict__ rowid, const int *__restrict__ col,
                                                          const VT *__restrict__ val, const T *__restrict__ dinv,
                                                          const T *__restrict__ b, T *x, T *t,
                                                          const double *__restrict__ coef, int degree, int n) {
  __shared__ T part[32][3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slice = warp / K, k = warp % K;
  T *cur = (degree - 1) % 2 == 0 ? x : t;
  T *oth = cur == x ? t : x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) cur[i] = (T)(*coef) * dinv[i] * b[i];
  __syncthreads();
  for (int st = 1; st < degree; ++st) {
    T acc[3] = {0, 0, 0};
    if (slice < nslices) {
      const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
      for (int j = k; j < w; j += K) {
        const int c = col[b0 + j * 32 + lane];
        const VT *vb = val + 9 * (b0 + j * 32) + lane;
        const T x0 = cur[3 * c], x1 = cur[3 * c + 1], x2 = cur[3 * c + 2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          acc[r] = fma_t(ldv(vb + 32 * (3 * r)), x0, acc[r]);
          acc[r] = fma_t(ldv(vb + 32 * (3 * r + 1)), x1, acc[r]);
          acc[r] = fma_t(ldv(vb + 32 * (3 * r + 2)), x2, acc[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) part[warp][r][lane] = acc[r];
    __syncthreads();
    if (k == 0 && slice < nslices) {
      const int row = rowid[slice * 32 + lane];
      if (row >= 0) {
        const double *cf = coef + 4 + 3 * (st - 1);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          T sum = part[warp][r][lane];
          for (int q = 1; q < K; ++q) sum += part[warp + q][r][lane];
          const int i = 3 * row + r;
          oth[i] = cheb_row<T>(cf, cur[i], dinv[i], b[i], sum, st > 1, st > 1 ? oth[i] : (T)0);
        }
      }
    }
    __syncthreads();
    T *tmp = cur;
    cur = oth;
    oth = tmp;
  }
}

template <typename T>
__global__ void k_sell_gather9(long n9, const int *__restrict__ map9, const double *__restrict__ csr,
                               T *__restrict__ out) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i >= n9) return;
  const int q = map9[i];
  out[i] = from_double<T>(q >= 0 ? csr[q] : 0.0);
}

// Scalar rows of at most 8 entries (every P1 operator: 7-point stencil):
// the epilogue operands are loaded first and all column / value loads are
// issued before the gathers, so a thread waits for two memory round trips.
// Same per-row summation order as k_sell.
template <typename T, typename VT>
__global__ void __launch_bounds__(kSellMaxBlock) k_sell_w8(int nslices, const int *__restrict__ sp,
                                                  const int *__restrict__ rowid, const int *__restrict__ col,
                                                  const VT *__restrict__ val, const T *__restrict__ u, T *out,
                                                  int mode, SpmvArgs a) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  const T *wv = static_cast<const T *>(a.w);
  T bi = 0, di = 0, ui = 0, wi = 0, oi = 0;
  if (row >= 0) {
    if (mode == SPMV_RES || mode == SPMV_CHEB) bi = static_cast<const T *>(a.b)[row];
    if (mode == SPMV_CHEB) {
      di = static_cast<const T *>(a.dinv)[row];
      ui = u[row];
      if (wv) wi = wv[row];
    }
    if (mode == SPMV_ADD) oi = out[row];
  }
  int c[8];
  T v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j < w) {
      c[j] = col[b0 + j * 32 + lane];
      v[j] = ldv(val + b0 + j * 32 + lane);
    }
  }
  T acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (j < w) acc += v[j] * u[c[j]];
  if (row < 0) return;
  T r;
  if (mode == SPMV_PLAIN) r = acc;
  else if (mode == SPMV_RES) r = bi - acc;
  else if (mode == SPMV_ADD) r = oi + acc;
  else r = cheb_row<T>(a.coef, ui, di, bi, acc, wv != nullptr, wi);
  out[row] = r;
}

struct StencilOff {
  int o[7];
};

// P1 rows in the stencil layout (Sell::stencil): the same slots, values and
// per-row summation order as k_sell_w8 on that layout, with the columns
// computed from the row instead of loaded (no col / rowid traffic, one
// dependent memory round trip instead of two).  Missing neighbours hold a
// zero value; their column is clamped into range.
template <typename T, typename VT>
__global__ void __launch_bounds__(kSellMaxBlock) k_stencil7(int nrows, StencilOff so, const VT *__restrict__ val,
                                                   const T *__restrict__ u, T *out, int mode, SpmvArgs a) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  const long base = (long)(row >> 5) * (7 * 32) + (row & 31);
  const T *wv = static_cast<const T *>(a.w);
  T bi = 0, di = 0, ui = 0, wi = 0, oi = 0;
  if (mode == SPMV_RES || mode == SPMV_CHEB) bi = static_cast<const T *>(a.b)[row];
  if (mode == SPMV_CHEB) {
    di = static_cast<const T *>(a.dinv)[row];
    ui = u[row];
    if (wv) wi = wv[row];
  }
  if (mode == SPMV_ADD) oi = out[row];
  T v[7];
  int c[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    v[j] = ldv(val + base + j * 32);
    const int cj = row + so.o[j];
    c[j] = cj < 0 ? 0 : (cj >= nrows ? nrows - 1 : cj);
  }
  T acc = 0;
#pragma unroll
  for (int j = 0; j < 7; ++j) acc += v[j] * u[c[j]];
  T r;
  if (mode == SPMV_PLAIN) r = acc;
  else if (mode == SPMV_RES) r = bi - acc;
  else if (mode == SPMV_ADD) r = oi + acc;
  else r = cheb_row<T>(a.coef, ui, di, bi, acc, wv != nullptr, wi);
  out[row] = r;
}

template <typename T, typename VT, bool VEC>
__global__ void __launch_bounds__(kSellMaxBlock) k_sell_bsr2(int nslices, const int *__restrict__ sp,
                                                   const int *__restrict__ rowid, const int *__restrict__ col,
                                                   const VT *__restrict__ val, const T *__restrict__ u, T *out,
                                                   int mode, SpmvArgs a) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  const typename V2t<T>::type *u2 = reinterpret_cast<const typename V2t<T>::type *>(u);
  T acc0 = 0, acc1 = 0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const long e = b0 + (long)j * 32 + lane;
    const int c = col[e];
    T b[4];
    load_blk(val + 4 * e, b);
    T x0, x1;
    if (VEC) {
      const typename V2t<T>::type x = u2[c];
      x0 = x.x;
      x1 = x.y;
    } else {
      x0 = u[2L * c];
      x1 = u[2L * c + 1];
    }
    // two FMAs per component (not a multiply, an FMA and an add): the FP64
    // form of this kernel is bound by the FP64 pipe
    acc0 = fma_t(b[1], x1, fma_t(b[0], x0, acc0));
    acc1 = fma_t(b[3], x1, fma_t(b[2], x0, acc1));
  }
  if (row < 0) return;
  epilogue<T>(mode, 2L * row, acc0, u, out, a, a.coef);
  epilogue<T>(mode, 2L * row + 1, acc1, u, out, a, a.coef);
}

__global__ void __launch_bounds__(kSellMaxBlock) k_sell_ch(int nslices, int nrows, const int *__restrict__ sp,
                                                 const int *__restrict__ rowid, const int *__restrict__ col,
                                                 const double *__restrict__ L, const double *__restrict__ K,
                                                 const double *__restrict__ K12, const double *__restrict__ M,
                                                 double a12, double a21, double a22, const double *__restrict__ x,
                                                 double *__restrict__ y) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  const double *x1 = x, *x2 = x + nrows;
  double s11 = 0, s12 = 0, s21 = 0, s22 = 0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const int e = b0 + j * 32 + lane;
    const int c = col[e];
    const double u1 = x1[c], u2 = x2[c], kv = K[e];
    s11 += L[e] * u1;
    s12 += (K12 ? K12[e] : kv) * u2;
    s21 += kv * u1;
    s22 += M[e] * u2;
  }
  if (row < 0) return;
  y[row] = s11 + a12 * s12;
  y[nrows + row] = a21 * s21 + a22 * s22;
}

// k_sell_ch for NR systems that share L, K, K12 and M (the CH species with
// constant mobility): the matrix stream is read once; each system's sums are
// the single-system kernel's expressions in the same order, so every output
// is bitwise k_sell_ch's.
template <int NR>
__global__ void __launch_bounds__(kSellMaxBlock) k_sell_ch_multi(int nslices, int nrows, const int *__restrict__ sp,
                                                      const int *__restrict__ rowid, const int *__restrict__ col,
                                                      const double *__restrict__ L, const double *__restrict__ K,
                                                      const double *__restrict__ K12, const double *__restrict__ M,
                                                      ChCoef3 cf, MultiPtr<const double> x, MultiPtr<double> y) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  double s11[NR], s12[NR], s21[NR], s22[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) s11[q] = s12[q] = s21[q] = s22[q] = 0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const int e = b0 + j * 32 + lane;
    const int c = col[e];
    const double lv = L[e], kv = K[e], k12 = K12 ? K12[e] : kv, mv = M[e];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const double u1 = x.p[q][c], u2 = x.p[q][nrows + c];
      s11[q] += lv * u1;
      s12[q] += k12 * u2;
      s21[q] += kv * u1;
      s22[q] += mv * u2;
    }
  }
  if (row < 0) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    y.p[q][row] = s11[q] + cf.a12[q] * s12[q];
    y.p[q][nrows + row] = cf.a21[q] * s21[q] + cf.a22[q] * s22[q];
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kSellMaxBlock) k_sell_b(int nslices, const int *__restrict__ sp, const int *__restrict__ rowid,
                                                const int *__restrict__ col, const double *__restrict__ val2,
                                                const double *__restrict__ v, double *__restrict__ y) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  const double2 *v2 = reinterpret_cast<const double2 *>(v);
  const double2 *w2 = reinterpret_cast<const double2 *>(val2);
  double acc = 0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const int e = b0 + j * 32 + lane;
    const double2 b = __ldg(w2 + e);
    const int c = col[e];
    if (VEC) {
      const double2 x = v2[c];
      acc = fma(b.y, x.y, fma(b.x, x.x, acc));
    } else {
      acc = fma(b.y, v[2L * c + 1], fma(b.x, v[2L * c], acc));
    }
  }
  if (row >= 0) y[row] = acc;
}

__global__ void __launch_bounds__(kSellMaxBlock) k_sell_bt_add(int nslices, const int *__restrict__ sp,
                                                     const int *__restrict__ rowid, const int *__restrict__ col,
                                                     const double *__restrict__ val2, const double *__restrict__ p,
                                                     double *__restrict__ yv) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  const double2 *w2 = reinterpret_cast<const double2 *>(val2);
  double a0 = 0, a1 = 0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const int e = b0 + j * 32 + lane;
    const double2 b = __ldg(w2 + e);
    const double q = p[col[e]];
    a0 += b.x * q;
    a1 += b.y * q;
  }
  if (row >= 0) {
    yv[2L * row] += a0;
    yv[2L * row + 1] += a1;
  }
}

// --------------------------------------------------------------------------
// Jacobi / Gershgorin
template <typename T>
__global__ void k_jacobi_csr(int nrows, const int *__restrict__ rowptr, const double *__restrict__ val,
                             const int *__restrict__ diag, T *dinv, double *partial) {
  __shared__ double sm[TPB];
  double best = 0.0;
  for (int r = blockIdx.x * TPB + threadIdx.x; r < nrows; r += gridDim.x * TPB) {
    const double d = val[diag[r]];
    double s = 0.0;
    for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) s += fabs(val[k]);
    dinv[r] = (T)(1.0 / d);
    best = fmax(best, s / fabs(d));
  }
  sm[threadIdx.x] = best;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

template <typename T>
__global__ void k_jacobi_bsr2(int nrows, const int *__restrict__ rowptr, const double *__restrict__ val,
                              const int *__restrict__ diag, T *dinv, double *partial) {
  __shared__ double sm[TPB];
  double best = 0.0;
  for (int r = blockIdx.x * TPB + threadIdx.x; r < nrows; r += gridDim.x * TPB) {
    const double *dblk = val + 4L * diag[r];
    double s0 = 0.0, s1 = 0.0;
    for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      const double *b = val + 4L * k;
      s0 += fabs(b[0]) + fabs(b[1]);
      s1 += fabs(b[2]) + fabs(b[3]);
    }
    dinv[2L * r] = (T)(1.0 / dblk[0]);
    dinv[2L * r + 1] = (T)(1.0 / dblk[3]);
    best = fmax(best, fmax(s0 / fabs(dblk[0]), s1 / fabs(dblk[3])));
  }
  sm[threadIdx.x] = best;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void k_max_final(int nb, const double *partial, double *out) {
  __shared__ double sm[TPB];
  double best = 0.0;
  for (int i = threadIdx.x; i < nb; i += TPB) best = fmax(best, partial[i]);
  sm[threadIdx.x] = best;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// Chebyshev smoother of degree d on [hi/ratio, hi] (three-term recurrence,
// Saad Alg. 12.1 on D^-1 A): theta = (hi+lo)/2, delta = (hi-lo)/2,
// sigma = theta/delta, rho_0 = 1/sigma, rho_k = 1/(2 sigma - rho_{k-1});
// x_1 = x_0 + D^-1 r_0 / theta, x_{k+1} = x_k + rho_k rho_{k-1} (x_k - x_{k-1})
// + (2 rho_k / delta) D^-1 (b - A x_k).
__global__ void k_cheb_coef(const double *hi, double ratio, int degree, double *c) {
  const double h = *hi, lo = h / ratio;
  const double theta = 0.5 * (h + lo), delta = 0.5 * (h - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  c[0] = 1.0 / theta;                          // pre: x_1 = D^-1 b / theta
  c[1] = 1.0; c[2] = 0.0; c[3] = 1.0 / theta;  // post: x_1 = x_0 + D^-1 (b - A x_0) / theta
  for (int k = 1; k < degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    const double al = rn * rho;
    c[4 + 3 * (k - 1)] = 1.0 + al;
    c[5 + 3 * (k - 1)] = -al;
    c[6 + 3 * (k - 1)] = 2.0 * rn / delta;
    rho = rn;
  }
}

// --------------------------------------------------------------------------
template <typename T>
__global__ void k_scale_dinv(int n, const double *scale, const T *dinv, const T *b, T *out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < n) out[i] = (T)(*scale) * dinv[i] * b[i];
}
template <typename Ta, typename Tb>
__global__ void k_convert(long n, const Ta *in, Tb *out) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) out[i] = (Tb)in[i];
}
template <typename Ta, typename Tb>
__global__ void k_convert_from_slot(long n, const Ta *const *slot, long off, Tb *out) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) out[i] = (Tb)((*slot)[off + i]);
}
template <typename Ta, typename Tb>
__global__ void k_convert_to_slot(long n, const Ta *in, Tb *const *slot, long off) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) (*slot)[off + i] = (Tb)in[i];
}
__global__ void k_set_ptrs(void **slots, const void *a, const void *b) {
  slots[0] = const_cast<void *>(a);
  slots[1] = const_cast<void *>(b);
}
__global__ void k_axpby(long n, double a, const double *x, double b, double *y) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}
__global__ void k_copy(long n, const double *x, double *y) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) y[i] = x[i];
}
__global__ void k_fill(long n, double v, double *y) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) y[i] = v;
}
__global__ void k_scale_by_inv(long n, const double *src, const double *hn, double *dst) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) dst[i] = src[i] / *hn;
}
template <typename T>
__global__ void k_sub_mean(int n, T *x, const double *sum) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < n) x[i] = (T)((double)x[i] - *sum / n);
}
__global__ void k_mul(long n, const double *a, const double *b, double *out) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) out[i] = a[i] * b[i];
}

// --------------------------------------------------------------------------
// reductions
__device__ __forceinline__ double block_sum(double v, double *sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void k_dot(long n, const T *x, const T *y, double *partial) {
  __shared__ double sm[TPB];
  double s = 0.0;
  for (long i = (long)blockIdx.x * TPB + threadIdx.x; i < n; i += (long)gridDim.x * TPB)
    s += (double)x[i] * (double)(y ? y[i] : (T)1);
  s = block_sum(s, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// sum of nb partials for each of k vectors: partial[v * nb + b]
__global__ void k_sum_final(int nb, int k, const double *partial, double *out) {
  __shared__ double sm[TPB];
  for (int v = blockIdx.x; v < k; v += gridDim.x) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += TPB) s += partial[(long)v * nb + i];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) out[v] = s;
  }
}

constexpr int KC = 16;   // vectors per multi-dot chunk

// partial[v * nb + b] for v in [k0, k0 + kc)
__global__ void k_mdot(long n, const double *__restrict__ V, long ldv, int k0, int kc, const double *__restrict__ w,
                       double *partial) {
  __shared__ double sm[TPB];
  double acc[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) acc[j] = 0.0;
  for (long i = (long)blockIdx.x * TPB + threadIdx.x; i < n; i += (long)gridDim.x * TPB) {
    const double wi = w[i];
#pragma unroll
    for (int j = 0; j < KC; ++j)
      if (j < kc) acc[j] += V[(long)(k0 + j) * ldv + i] * wi;
  }
  for (int j = 0; j < kc; ++j) {
    const double s = block_sum(acc[j], sm);
    if (threadIdx.x == 0) partial[(long)(k0 + j) * gridDim.x + blockIdx.x] = s;
  }
}

// w -= V h (k vectors); then partial dots V^T w (mode 0) or w^T w (mode 1)
template <int MODE>
__global__ void k_ortho_update(long n, const double *__restrict__ V, long ldv, int k, const double *__restrict__ h,
                               double *__restrict__ w, double *partial, int k0, int kc) {
  __shared__ double sm[TPB];
  __shared__ double hs[64];
  if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) acc[j] = 0.0;
  for (long i = (long)blockIdx.x * TPB + threadIdx.x; i < n; i += (long)gridDim.x * TPB) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += hs[j] * V[(long)j * ldv + i];
    const double wi = w[i] - s;
    if (k0 == 0) w[i] = wi;          // the first chunk writes the update
    if (MODE == 0) {
#pragma unroll
      for (int j = 0; j < KC; ++j)
        if (j < kc) acc[j] += V[(long)(k0 + j) * ldv + i] * wi;
    } else {
      acc[0] += wi * wi;
    }
  }
  const int nv = MODE == 0 ? kc : 1;
  for (int j = 0; j < nv; ++j) {
    const double s = block_sum(acc[j], sm);
    if (threadIdx.x == 0) partial[(long)(k0 + j) * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_combine(long n, const double *__restrict__ Z, long ldz, int k0, const int *kd,
                          const double *__restrict__ y, double *__restrict__ x) {
  __shared__ double ys[64];
  const int k = kd ? *kd : k0;   // kd: the column count from device memory
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = 0; j < k; ++j) s += ys[j] * Z[(long)j * ldz + i];
  x[i] += s;
}

// pyth = 1: *nrm2 holds ||w||^2 after the first correction and the norm
// after the second one is ||w||^2 - ||h2||^2 (the basis is orthonormal)
__global__ void k_arnoldi_finish(int j, int ldh, double *H, const double *h1, const double *h2, const double *nrm2,
                                 double *cs, double *sn, double *g, double *status, int pyth) {
  double *col = H + (long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  double q = *nrm2;
  if (pyth) {
    for (int i = 0; i <= j; ++i) q -= h2[i] * h2[i];
    q = fmax(q, 0.0);
  }
  const double hn = sqrt(q);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = col[i], c = col[i + 1];
    col[i] = cs[i] * a + sn[i] * c;
    col[i + 1] = -sn[i] * a + cs[i] * c;
  }
  const double den = hypot(col[j], col[j + 1]);
  cs[j] = col[j] / den;
  sn[j] = col[j + 1] / den;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  status[0] = fabs(g[j + 1]);
  status[1] = hn;
}

__global__ void k_hessenberg_solve(int k0, const int *kd, int ldh, const double *H, const double *g, double *y) {
  const int k = kd ? *kd : k0;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(long)c * ldh + i] * y[c];
    y[i] = s / H[(long)i * ldh + i];
  }
}

__global__ void k_set_scalar(double *dst, const double *src, double scale, int sq) {
  const double v = sq ? sqrt(*src) : *src;
  *dst = scale * v;
}
__global__ void k_pcg_alpha(const double *rz, const double *pq, double *alpha) { *alpha = *rz / *pq; }
__global__ void k_pcg_xr(long n, const double *alpha, const double *p, const double *q, double *x, double *r) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) {
    const double a = *alpha;
    x[i] += a * p[i];
    r[i] -= a * q[i];
  }
}
__global__ void k_pcg_p(long n, const double *rzn, const double *rzo, const double *z, double *p) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) p[i] = z[i] + (*rzn / *rzo) * p[i];
}

// --------------------------------------------------------------------------
// coarse grid
__global__ void k_dense_csr(int nrows, const int *rowptr, const int *col, const double *val, double add_all,
                            double *dense) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  for (int c = 0; c < nrows; ++c) dense[(long)r * nrows + c] = add_all;
  for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) dense[(long)r * nrows + col[k]] += val[k];
}
__global__ void k_dense_bsr2(int nrows, const int *rowptr, const int *col, const double *val, double *dense) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int n = 2 * nrows;
  for (int c = 0; c < n; ++c) {
    dense[(long)(2 * r) * n + c] = 0.0;
    dense[(long)(2 * r + 1) * n + c] = 0.0;
  }
  for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    const int c = 2 * col[k];
    dense[(long)(2 * r) * n + c] = val[4L * k];
    dense[(long)(2 * r) * n + c + 1] = val[4L * k + 1];
    dense[(long)(2 * r + 1) * n + c] = val[4L * k + 2];
    dense[(long)(2 * r + 1) * n + c + 1] = val[4L * k + 3];
  }
}

// Gauss-Jordan inverse with partial pivoting of a (n x n, row-major,
// destroyed) into inv; one CTA.  status = 1 on an exactly zero pivot.
__global__ void k_dense_invert(int n, double *a, double *inv, int *status) {
  __shared__ int piv;
  __shared__ double sv[TPB];
  __shared__ int si[TPB];
  for (long t = threadIdx.x; t < (long)n * n; t += blockDim.x) inv[t] = (t / n == t % n) ? 1.0 : 0.0;
  if (threadIdx.x == 0) *status = 0;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    double best = -1.0;
    int bi = c;
    for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
      const double v = fabs(a[(long)r * n + c]);
      if (v > best || (v == best && r < bi)) { best = v; bi = r; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const double v2 = sv[threadIdx.x + o];
        const int i2 = si[threadIdx.x + o];
        if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
          sv[threadIdx.x] = v2;
          si[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      piv = si[0];
      if (sv[0] == 0.0) *status = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != c)
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double x = a[(long)c * n + t]; a[(long)c * n + t] = a[(long)p * n + t]; a[(long)p * n + t] = x;
        x = inv[(long)c * n + t]; inv[(long)c * n + t] = inv[(long)p * n + t]; inv[(long)p * n + t] = x;
      }
    __syncthreads();
    const double d = a[(long)c * n + c];
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      a[(long)c * n + t] /= d;
      inv[(long)c * n + t] /= d;
    }
    __syncthreads();
    for (long t = threadIdx.x; t < (long)n * n; t += blockDim.x) {
      const int r = (int)(t / n), q = (int)(t % n);
      if (r == c) continue;
      const double f = a[(long)r * n + c];
      if (q != c) a[t] -= f * a[(long)c * n + q];
      inv[t] -= f * inv[(long)c * n + q];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != c) a[(long)r * n + c] = 0.0;
    __syncthreads();
  }
}

template <typename T>
__global__ void k_dense_apply(int n, const double *inv, const T *b, T *x) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int c = 0; c < n; ++c) s += inv[(long)r * n + c] * (double)b[c];
  x[r] = (T)s;
}


// ---------------------------------------------------------------------------
// Multi-right-hand-side variants (up to kMaxRhs vectors sharing one matrix):
// the matrix stream is read once, each right-hand side is summed in the same
// order as by the single-vector kernels, so every output is bitwise the one
// the single-vector kernel would give.
// One slice (32 rows) of a multi-vector scalar SpMV with rows of at most W
// entries; shared by k_sell_w8m (W = 8) and the one-block coarse-level
// kernel (W = 8, or 16 for the 15-entry rows of the tetrahedral P1 levels).
template <typename T, int NR, int W = 8>
__device__ __forceinline__ void sell_w8m_slice(int slice, int lane, const int *sp, const int *rowid, const int *col,
                                               const T *val, const MultiPtr<T> &u, const MultiPtr<T> &out, int mode,
                                               const MultiArgs<T> &a) {
  const int row = rowid[slice * 32 + lane];
  const int b0 = sp[slice], w = (sp[slice + 1] - b0) >> 5;
  T bi[NR], ui[NR], wi[NR], oi[NR];
  T di = 0;
#pragma unroll
  for (int k = 0; k < NR; ++k) bi[k] = ui[k] = wi[k] = oi[k] = 0;
  if (row >= 0) {
    if (mode == SPMV_CHEB) di = a.dinv[row];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (mode == SPMV_RES || mode == SPMV_CHEB) bi[k] = a.b.p[k][row];
      if (mode == SPMV_CHEB) {
        ui[k] = u.p[k][row];
        if (a.w.p[k]) wi[k] = a.w.p[k][row];
      }
      if (mode == SPMV_ADD) oi[k] = out.p[k][row];
    }
  }
  T acc[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) acc[k] = 0;
  // entries in chunks of 8 (all loads of a chunk first), summed in order
#pragma unroll
  for (int j0 = 0; j0 < W; j0 += 8) {
    int c[8];
    T v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j0 + j < w) {
        c[j] = col[b0 + (j0 + j) * 32 + lane];
        v[j] = val[b0 + (j0 + j) * 32 + lane];
      }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j0 + j < w) acc[k] += v[j] * u.p[k][c[j]];
  }
  if (row < 0) return;
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    T r;
    if (mode == SPMV_PLAIN) r = acc[k];
    else if (mode == SPMV_RES) r = bi[k] - acc[k];
    else if (mode == SPMV_ADD) r = oi[k] + acc[k];
    else r = cheb_row<T>(a.coef, ui[k], di, bi[k], acc[k], a.w.p[k] != nullptr, wi[k]);
    out.p[k][row] = r;
  }
}

// Multi-vector form of k_stencil7: per vector the same expressions as
// sell_w8m_slice on the stencil layout.
template <typename T, int NR>
__global__ void __launch_bounds__(kSellMaxBlock) k_stencil7m(int nrows, StencilOff so, const T *__restrict__ val,
                                                    MultiPtr<T> u, MultiPtr<T> out, int mode, MultiArgs<T> a) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  const long base = (long)(row >> 5) * (7 * 32) + (row & 31);
  T bi[NR], ui[NR], wi[NR], oi[NR];
  T di = 0;
#pragma unroll
  for (int k = 0; k < NR; ++k) bi[k] = ui[k] = wi[k] = oi[k] = 0;
  if (mode == SPMV_CHEB) di = a.dinv[row];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (mode == SPMV_RES || mode == SPMV_CHEB) bi[k] = a.b.p[k][row];
    if (mode == SPMV_CHEB) {
      ui[k] = u.p[k][row];
      if (a.w.p[k]) wi[k] = a.w.p[k][row];
    }
    if (mode == SPMV_ADD) oi[k] = out.p[k][row];
  }
  T v[7];
  int c[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    v[j] = val[base + j * 32];
    const int cj = row + so.o[j];
    c[j] = cj < 0 ? 0 : (cj >= nrows ? nrows - 1 : cj);
  }
  T acc[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    acc[k] = 0;
#pragma unroll
    for (int j = 0; j < 7; ++j) acc[k] += v[j] * u.p[k][c[j]];
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    T r;
    if (mode == SPMV_PLAIN) r = acc[k];
    else if (mode == SPMV_RES) r = bi[k] - acc[k];
    else if (mode == SPMV_ADD) r = oi[k] + acc[k];
    else r = cheb_row<T>(a.coef, ui[k], di, bi[k], acc[k], a.w.p[k] != nullptr, wi[k]);
    out.p[k][row] = r;
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(kSellMaxBlock) k_sell_w8m(int nslices, const int *__restrict__ sp,
                                                   const int *__restrict__ rowid, const int *__restrict__ col,
                                                   const T *__restrict__ val, MultiPtr<T> u, MultiPtr<T> out,
                                                   int mode, MultiArgs<T> a) {
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (slice >= nslices) return;
  sell_w8m_slice<T, NR>(slice, lane, sp, rowid, col, val, u, out, mode, a);
}

// ---------------------------------------------------------------------------
// The coarse end of a scalar V-cycle in one block: levels l0..L of the
// hierarchy (a few thousand rows at most) are swept by the block's warps,
// with a block barrier between sweeps, instead of one launch per sweep.
// Every row is computed by the same code as in the per-sweep kernels
// (sell_w8m_slice, the same scale / copy / dense expressions), so the
// result is bitwise the multi-launch V-cycle's.
template <typename T, int NR, int W>
__device__ void tail_sweep(const TailSell &S, const T *val, const MultiPtr<T> &u, const MultiPtr<T> &out, int mode,
                           const MultiArgs<T> &a) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int slice = threadIdx.x >> 5; slice < S.nslices; slice += nw)
    sell_w8m_slice<T, NR, W>(slice, lane, S.sp, S.rowid, S.col, val, u, out, mode, a);
  __syncthreads();
}

template <typename T, int NR, int W>
__global__ void __launch_bounds__(512) k_mg_tail(const TailDesc<T> *__restrict__ dp) {
  const TailDesc<T> &d = *dp;
  const int L = d.nlev - 1;
  const int degree = d.degree;
  // down: pre-smoothing, residual, restriction
  for (int l = 0; l < L; ++l) {
    const TailLevel<T> &q = d.lv[l];
    MultiPtr<T> cur = (degree - 1) % 2 == 0 ? q.x : q.t;
    MultiPtr<T> oth = (degree - 1) % 2 == 0 ? q.t : q.x;
    for (int i = threadIdx.x; i < q.n; i += blockDim.x)
      for (int k = 0; k < NR; ++k) cur.p[k][i] = (T)(*q.coef) * q.dinv[i] * q.b.p[k][i];
    __syncthreads();
    MultiArgs<T> a;
    a.b = q.b;
    a.dinv = q.dinv;
    for (int s = 1; s < degree; ++s) {
      a.coef = q.coef + 4 + 3 * (s - 1);
      a.w = s == 1 ? MultiPtr<T>() : oth;
      tail_sweep<T, NR, W>(q.A, q.val, cur, oth, SPMV_CHEB, a);
      const MultiPtr<T> tmp = cur;
      cur = oth;
      oth = tmp;
    }
    MultiArgs<T> ar;
    ar.b = q.b;
    tail_sweep<T, NR, W>(q.A, q.val, q.x, q.r, SPMV_RES, ar);
    MultiArgs<T> none;
    tail_sweep<T, NR, W>(q.R, q.Rval, q.r, d.lv[l + 1].b, SPMV_PLAIN, none);
  }
  // coarsest: dense inverse, or Chebyshev steps from zero (same sweeps as
  // the pre-smoothing, coarse_degree of them)
  if (d.coarse_degree > 0) {
    const TailLevel<T> &q = d.lv[L];
    const int cd = d.coarse_degree;
    MultiPtr<T> cur = (cd - 1) % 2 == 0 ? q.x : q.t;
    MultiPtr<T> oth = (cd - 1) % 2 == 0 ? q.t : q.x;
    for (int i = threadIdx.x; i < q.n; i += blockDim.x)
      for (int k = 0; k < NR; ++k) cur.p[k][i] = (T)(*q.coef) * q.dinv[i] * q.b.p[k][i];
    __syncthreads();
    MultiArgs<T> a;
    a.b = q.b;
    a.dinv = q.dinv;
    for (int st = 1; st < cd; ++st) {
      a.coef = q.coef + 4 + 3 * (st - 1);
      a.w = st == 1 ? MultiPtr<T>() : oth;
      tail_sweep<T, NR, W>(q.A, q.val, cur, oth, SPMV_CHEB, a);
      const MultiPtr<T> tmp = cur;
      cur = oth;
      oth = tmp;
    }
  } else {
    const TailLevel<T> &q = d.lv[L];
    for (int r = threadIdx.x; r < d.nc; r += blockDim.x)
      for (int k = 0; k < NR; ++k) {
        double s = 0.0;
        for (int c = 0; c < d.nc; ++c) s += d.cinv[(long)r * d.nc + c] * (double)q.b.p[k][c];
        q.x.p[k][r] = (T)s;
      }
    __syncthreads();
  }
  // up: prolongation, post-smoothing
  for (int l = L - 1; l >= 0; --l) {
    const TailLevel<T> &q = d.lv[l];
    MultiArgs<T> none;
    tail_sweep<T, NR, W>(q.P, q.Pval, d.lv[l + 1].x, q.x, SPMV_ADD, none);
    MultiArgs<T> a;
    a.b = q.b;
    a.dinv = q.dinv;
    a.coef = q.coef + 1;
    tail_sweep<T, NR, W>(q.A, q.val, q.x, q.t, SPMV_CHEB, a);
    MultiPtr<T> cur = q.t, oth = q.x;
    for (int s = 1; s < degree; ++s) {
      a.coef = q.coef + 4 + 3 * (s - 1);
      a.w = oth;
      tail_sweep<T, NR, W>(q.A, q.val, cur, oth, SPMV_CHEB, a);
      const MultiPtr<T> tmp = cur;
      cur = oth;
      oth = tmp;
    }
    if (cur.p[0] != q.x.p[0]) {
      for (int i = threadIdx.x; i < q.n; i += blockDim.x)
        for (int k = 0; k < NR; ++k) q.x.p[k][i] = cur.p[k][i];
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void k_scale_dinv_m(int n, int nr, const double *scale, const T *dinv, MultiPtr<T> b, MultiPtr<T> out) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < nr; ++k) out.p[k][i] = (T)(*scale) * dinv[i] * b.p[k][i];
}

template <typename T>
__global__ void k_dense_apply_m(int n, int nr, const double *inv, MultiPtr<T> b, MultiPtr<T> x) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int k = 0; k < nr; ++k) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += inv[(long)r * n + c] * (double)b.p[k][c];
    x.p[k][r] = (T)s;
  }
}

template <typename T>
__global__ void k_copy_m(long n, int nr, MultiPtr<T> in, MultiPtr<T> out) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < nr; ++k) out.p[k][i] = in.p[k][i];
}

// ---------------------------------------------------------------------------
// CGS2 orthogonalisation kernels for k <= kCgsMaxK basis vectors.  The vector
// count is a template parameter, so every issued FP64 FMA is useful work (the
// FP64 pipe bounds these kernels on this part).  Each block reduces its NV
// partial sums with a transposing warp butterfly: NV is padded to P = 2^LP,
// LP halving steps leave lane l with the warp sum of vector l >> (5 - LP),
// the remaining steps fold the duplicate lanes; the warps' results are then
// summed in fixed order through shared memory.  Bit-reproducible.
constexpr int kCgsBlock = 256;
constexpr int kCgsBlocksPerSm = 2;   // grid cap of the update passes
constexpr int kCgsMaxK = 31;

constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }
constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

template <int P>
__device__ __forceinline__ double warp_transpose_sum(double (&v)[P]) {
  constexpr int LP = ilog2(P);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int st = 0; st < LP; ++st) {
    const int mask = 16 >> st;
    const int c = P >> (st + 1);
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int q = 0; q < c; ++q) {
      const double send = up ? v[q] : v[q + c];
      const double keep = up ? v[q + c] : v[q];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
  }
#pragma unroll
  for (int st = LP; st < 5; ++st) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16 >> st);
  return v[0];
}

// partial[j * gridDim.x + blockIdx.x] = block sum of a[j], j < NV
template <int NV>
__device__ __forceinline__ void cgs_block_reduce(double (&a)[pow2_at_least(NV)], double *__restrict__ partial) {
  constexpr int P = pow2_at_least(NV);
  constexpr int LP = ilog2(P);
  __shared__ double red[kCgsBlock / 32][P];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double v = warp_transpose_sum<P>(a);
  if ((lane & ((1 << (5 - LP)) - 1)) == 0) red[warp][lane >> (5 - LP)] = v;
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kCgsBlock / 32; ++w) t += red[w][threadIdx.x];
    partial[(long)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// h = V^T w over KC vectors (partials)
template <int KC>
__global__ void __launch_bounds__(kCgsBlock) k_cgs_dots(long n, const double *__restrict__ V, long ld,
                                                        const double *__restrict__ w, double *__restrict__ partial) {
  double acc[pow2_at_least(KC)];
#pragma unroll
  for (int j = 0; j < pow2_at_least(KC); ++j) acc[j] = 0.0;
  for (long i = (long)blockIdx.x * kCgsBlock + threadIdx.x; i < n; i += (long)gridDim.x * kCgsBlock) {
    const double wi = w[i];
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] += V[(long)j * ld + i] * wi;
  }
  cgs_block_reduce<KC>(acc, partial);
}

// w -= V h; then partials of V^T w (KC values) and w^T w (one more)
template <int KC>
__global__ void __launch_bounds__(kCgsBlock) k_cgs_update_dots(long n, const double *__restrict__ V, long ld,
                                                               const double *__restrict__ h, double *__restrict__ w,
                                                               double *__restrict__ partial) {
  __shared__ double hs[KC];
  if (threadIdx.x < KC) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[pow2_at_least(KC + 1)];
#pragma unroll
  for (int j = 0; j < pow2_at_least(KC + 1); ++j) acc[j] = 0.0;
  for (long i = (long)blockIdx.x * kCgsBlock + threadIdx.x; i < n; i += (long)gridDim.x * kCgsBlock) {
    double v[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) v[j] = V[(long)j * ld + i];
    double s0 = 0.0, s1 = 0.0;     // two chains: half the FP64 latency on the critical path
#pragma unroll
    for (int j = 0; j < KC; j += 2) s0 += hs[j] * v[j];
#pragma unroll
    for (int j = 1; j < KC; j += 2) s1 += hs[j] * v[j];
    const double wi = w[i] - (s0 + s1);
    w[i] = wi;
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] += v[j] * wi;
    acc[KC] += wi * wi;
  }
  cgs_block_reduce<KC + 1>(acc, partial);
}

// out = (w - V h) / hn  (the next basis vector; no reduction)
template <int KC>
__global__ void __launch_bounds__(kCgsBlock) k_cgs_update_scale(long n, const double *__restrict__ V, long ld,
                                                                const double *__restrict__ h,
                                                                const double *__restrict__ w,
                                                                const double *__restrict__ hn,
                                                                double *__restrict__ out) {
  __shared__ double hs[KC];
  __shared__ double inv;
  if (threadIdx.x < KC) hs[threadIdx.x] = h[threadIdx.x];
  if (threadIdx.x == 0) inv = 1.0 / *hn;
  __syncthreads();
  const long i = (long)blockIdx.x * kCgsBlock + threadIdx.x;
  if (i >= n) return;
  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int j = 0; j < KC; j += 2) s0 += hs[j] * V[(long)j * ld + i];
#pragma unroll
  for (int j = 1; j < KC; j += 2) s1 += hs[j] * V[(long)j * ld + i];
  out[i] = (w[i] - (s0 + s1)) * inv;
}

// ---------------------------------------------------------------------------
// CGS2 in double-FP32 arithmetic.  A value is carried as the unevaluated sum
// h + l of two FP32 numbers (h = the value rounded to FP32, l = the rest
// rounded to FP32: about 48 significant bits).  The exact product of two
// FP32 numbers is p + e with e = fma(a, b, -p) (Dekker's two-product,
// "A floating-point technique for extending the available precision",
// 1971); the exact sum is s + t with Knuth's two-sum (TAOCP vol. 2,
// 4.2.2).  One FP64 multiply-add of the Gram-Schmidt passes becomes about
// eleven FP32 operations, on a pipe 64 times wider than this part's FP64
// pipe, so the passes are bound by their memory traffic instead of by FP64
// arithmetic.  Every step of the error-free transformations uses the _rn
// intrinsics, which the compiler never contracts into FMAs.
__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(__dsub_rn(x, (double)h)));
}
__device__ __forceinline__ double df_join(float2 a) { return __dadd_rn((double)a.x, (double)a.y); }
// (s, t) with s + t = a + b exactly, |b| <= |a| not required
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, t);
}
// (s, t) with s + t = a + b exactly when |a| >= |b|
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// acc += a * b; acc is kept unnormalised (acc.x the running leading sum,
// acc.y the collected rounding errors and low-order products; a.y * b.y,
// of relative size 2^-48, is dropped)
__device__ __forceinline__ void df_mac(float2 &acc, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float2 st = two_sum(acc.x, p);
  acc.x = st.x;
  acc.y = __fadd_rn(acc.y, __fadd_rn(st.y, e));
}
// normalised a - b
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) {
  const float2 st = two_sum(a.x, -b.x);
  return fast_two_sum(st.x, __fadd_rn(st.y, __fsub_rn(a.y, b.y)));
}
// normalised a * b
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return fast_two_sum(p, e);
}

// pass 1: h = V^T w over KC vectors (partials); V in pairs, w in FP64
template <int KC>
__global__ void __launch_bounds__(kCgsBlock) k_dfgs_dots(long n, const float2 *__restrict__ V, long ld,
                                                         const double *__restrict__ w,
                                                         double *__restrict__ partial) {
  float2 acc[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) acc[j] = make_float2(0.f, 0.f);
  for (long i = (long)blockIdx.x * kCgsBlock + threadIdx.x; i < n; i += (long)gridDim.x * kCgsBlock) {
    const float2 wi = df_split(w[i]);
#pragma unroll
    for (int j = 0; j < KC; ++j) df_mac(acc[j], V[(long)j * ld + i], wi);
  }
  double a[pow2_at_least(KC)];
#pragma unroll
  for (int j = 0; j < pow2_at_least(KC); ++j) a[j] = j < KC ? df_join(acc[j]) : 0.0;
  cgs_block_reduce<KC>(a, partial);
}

// pass 2: w -= V h (w read in FP64, written back in place as pairs); then
// partials of V^T w (KC values) and w^T w (one more)
template <int KC>
__global__ void __launch_bounds__(kCgsBlock) k_dfgs_update_dots(long n, const float2 *__restrict__ V, long ld,
                                                                const double *__restrict__ h, double *w,
                                                                double *__restrict__ partial) {
  __shared__ float2 hs[KC];
  if (threadIdx.x < KC) hs[threadIdx.x] = df_split(h[threadIdx.x]);
  __syncthreads();
  float2 acc[KC + 1];
#pragma unroll
  for (int j = 0; j <= KC; ++j) acc[j] = make_float2(0.f, 0.f);
  float2 *w2 = reinterpret_cast<float2 *>(w);
  for (long i = (long)blockIdx.x * kCgsBlock + threadIdx.x; i < n; i += (long)gridDim.x * kCgsBlock) {
    float2 v[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) v[j] = V[(long)j * ld + i];
    float2 sv = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < KC; ++j) df_mac(sv, v[j], hs[j]);
    const float2 wi = df_sub(df_split(w[i]), sv);
    w2[i] = wi;
#pragma unroll
    for (int j = 0; j < KC; ++j) df_mac(acc[j], v[j], wi);
    df_mac(acc[KC], wi, wi);
  }
  double a[pow2_at_least(KC + 1)];
#pragma unroll
  for (int j = 0; j < pow2_at_least(KC + 1); ++j) a[j] = j <= KC ? df_join(acc[j]) : 0.0;
  cgs_block_reduce<KC + 1>(a, partial);
}

// pass 3: the next basis vector (w - V h) / hn, from w in pairs; written in
// pairs (for the Gram-Schmidt passes) and in FP64 (for the preconditioner),
// the FP64 copy being the exact value of the pair
template <int KC>
__global__ void __launch_bounds__(kCgsBlock) k_dfgs_update_scale(long n, const float2 *__restrict__ V, long ld,
                                                                 const double *__restrict__ h,
                                                                 const float2 *__restrict__ w,
                                                                 const double *__restrict__ hn,
                                                                 float2 *__restrict__ out2,
                                                                 double *__restrict__ out64) {
  __shared__ float2 hs[KC];
  __shared__ float2 inv;
  if (threadIdx.x < KC) hs[threadIdx.x] = df_split(h[threadIdx.x]);
  if (threadIdx.x == 0) inv = df_split(1.0 / *hn);
  __syncthreads();
  const long i = (long)blockIdx.x * kCgsBlock + threadIdx.x;
  if (i >= n) return;
  float2 sv = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < KC; ++j) df_mac(sv, V[(long)j * ld + i], hs[j]);
  const float2 r = df_mul(df_sub(w[i], sv), inv);
  out2[i] = r;
  out64[i] = df_join(r);
}

// the first basis vector: x = w / hn in FP64, kept as its pair and as the
// pair's exact FP64 value
__global__ void k_df_first(long n, const double *__restrict__ w, const double *__restrict__ hn,
                           float2 *__restrict__ out2, double *__restrict__ out64) {
  const long i = (long)blockIdx.x * kCgsBlock + threadIdx.x;
  if (i >= n) return;
  const float2 r = df_split(w[i] / *hn);
  out2[i] = r;
  out64[i] = df_join(r);
}

}  // namespace

// ============================================================================
template <typename T>
void spmv_csr(const Pattern &P, const T *val, int ncomp, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
              cudaStream_t s) {
  if (P.nrows == 0) return;
  const double avg = P.nnz / (double)P.nrows;
  if (avg <= 4.5) {
    k_spmv_csr<4, T><<<nblocks((long)P.nrows * 4, TPB), TPB, 0, s>>>(P.nrows, ncomp, P.rowptr, P.col, val, u, out,
                                                                    mode, a);
  } else {
    k_spmv_csr<8, T><<<nblocks((long)P.nrows * 8, TPB), TPB, 0, s>>>(P.nrows, ncomp, P.rowptr, P.col, val, u, out,
                                                                    mode, a);
  }
  CHNSS_LAUNCH_CK();
}
template <typename T>
void spmv_bsr2(const Pattern &P, const T *val, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
               cudaStream_t s) {
  if (P.nrows == 0) return;
  k_spmv_bsr2<8, T><<<nblocks((long)P.nrows * 8, TPB), TPB, 0, s>>>(P.nrows, P.rowptr, P.col, val, u, out, mode, a);
  CHNSS_LAUNCH_CK();
}
template void spmv_csr<double>(const Pattern &, const double *, int, const double *, double *, SpmvMode,
                               const SpmvArgs &, cudaStream_t);
template void spmv_csr<float>(const Pattern &, const float *, int, const float *, float *, SpmvMode,
                              const SpmvArgs &, cudaStream_t);
template void spmv_bsr2<double>(const Pattern &, const double *, const double *, double *, SpmvMode,
                                const SpmvArgs &, cudaStream_t);
template void spmv_bsr2<float>(const Pattern &, const float *, const float *, float *, SpmvMode,
                               const SpmvArgs &, cudaStream_t);

inline bool aligned(const void *p, size_t bytes) { return (reinterpret_cast<uintptr_t>(p) % bytes) == 0; }

template <typename Tout>
void sell_gather(const Sell &S, int ncomp, const double *csr_vals, Tout *out, cudaStream_t s) {
  if (S.nent == 0) return;
  k_sell_gather<Tout><<<nblocks(S.nent, TPB), TPB, 0, s>>>(S.nent, ncomp, S.map, csr_vals, out);
  CHNSS_LAUNCH_CK();
}
template void sell_gather<double>(const Sell &, int, const double *, double *, cudaStream_t);
template void sell_gather<float>(const Sell &, int, const double *, float *, cudaStream_t);
template void sell_gather<__nv_bfloat16>(const Sell &, int, const double *, __nv_bfloat16 *, cudaStream_t);

void sell_gather_transposed(const Sell &S, int ncomp, const double *csr_vals, double *out, cudaStream_t s) {
  if (!S.mapT) throw Error{CHNSS_ERR_ARG, "transposed values need a square symmetric pattern"};
  if (ncomp != 1 && ncomp != 4) throw Error{CHNSS_ERR_ARG, "transposed values: ncomp must be 1 or 4"};
  k_sell_gather_t<<<nblocks(S.nent, TPB), TPB, 0, s>>>(S.nent, ncomp, S.mapT, csr_vals, out);
  CHNSS_LAUNCH_CK();
}

// Warps per slice of a scalar SELL SpMV: 1 while the slices alone fill one
// wave of resident warps (48 per multiprocessor) or the rows are short;
// otherwise doubled (up to 32) until they do, keeping at least four entries of
// the widest slice per warp.  A function of the pattern and the device only.
int sell_split(const Sell &S) {
  if (S.wmax < 12) return 1;
  const long target = 48L * device_sm_count();
  int K = 1;
  while (K < 32 && (long)S.nslices * K < target && S.wmax / (2 * K) >= 4) K *= 2;
  return K;
}

template <typename T, typename VT, int K>
void launch_sell_split(const Sell &S, const VT *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                       cudaStream_t s) {
  constexpr int SPB = K >= 8 ? 1 : 8 / K;
  k_sell_split<T, VT, K><<<(S.nslices + SPB - 1) / SPB, 32 * K * SPB, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col,
                                                                           sval, u, out, mode, a);
}

template <typename T, typename VT>
void spmv_sell_impl(const Pattern &P, const VT *sval, int ncomp, const T *u, T *out, SpmvMode mode,
                    const SpmvArgs &a, cudaStream_t s) {
  const Sell &S = P.sell;
  if (S.nslices == 0) return;
  const int nb = nblocks((long)S.nslices * 32, S.block);
  const int K = ncomp == 1 && !S.stencil ? sell_split(S) : 1;
  if (ncomp == 1 && S.stencil) {
    StencilOff so;
    for (int j = 0; j < 7; ++j) so.o[j] = S.soff[j];
    k_stencil7<T, VT><<<nblocks(P.nrows, S.block), S.block, 0, s>>>(P.nrows, so, sval, u, out, mode, a);
  } else if (ncomp == 1 && S.wmax <= 8)
    k_sell_w8<T, VT><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
  else if (K == 2)
    launch_sell_split<T, VT, 2>(S, sval, u, out, mode, a, s);
  else if (K == 4)
    launch_sell_split<T, VT, 4>(S, sval, u, out, mode, a, s);
  else if (K == 8)
    launch_sell_split<T, VT, 8>(S, sval, u, out, mode, a, s);
  else if (K == 16)
    launch_sell_split<T, VT, 16>(S, sval, u, out, mode, a, s);
  else if (K == 32)
    launch_sell_split<T, VT, 32>(S, sval, u, out, mode, a, s);
  else if (ncomp == 1)
    k_sell<T, VT, 1, false><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
  else if (aligned(u, 2 * sizeof(T)))
    k_sell<T, VT, 2, true><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
  else
    k_sell<T, VT, 2, false><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
  CHNSS_LAUNCH_CK();
}

template <typename T, typename VT, int K>
void launch_sell_bsr3(const Sell &S, const VT *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                      cudaStream_t s) {
  constexpr int SPB = K >= 8 ? 1 : 8 / K;
  k_sell_bsr3<T, VT, K><<<(S.nslices + SPB - 1) / SPB, 32 * K * SPB, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col,
                                                                          sval, u, out, mode, a);
}

// Warps per slice of a 3x3-block SpMV: enough that the widest slice gives a
// warp about eight blocks (up to K = 8; on the 3D meshes the slices of
// vertex rows are twice as wide as the average, and whole slices per warp
// leave the multiprocessors waiting on them at the end of the launch:
// 32^3 cubes, K = 1 -> 8: 92 -> 84 ms per mixed step, 163 -> 141 ms FP64),
// then doubled up to 16 while the slices do not fill one wave of warps.
int sell_warps_bsr3(const Sell &S) {
  const long target = 48L * device_sm_count();
  int K = 1;
  while (K < 8 && S.wmax / (2 * K) >= 8) K *= 2;
  while (K < 16 && (long)S.nslices * K < target && S.wmax / (2 * K) >= 2) K *= 2;
  return K;
}

template <typename T, typename VT>
void spmv_sell_bsr3_impl(const Pattern &P, const VT *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                         cudaStream_t s) {
  const Sell &S = P.sell;
  if (S.nslices == 0) return;
  const int K = sell_warps_bsr3(S);
  switch (K) {
    case 1: launch_sell_bsr3<T, VT, 1>(S, sval, u, out, mode, a, s); break;
    case 2: launch_sell_bsr3<T, VT, 2>(S, sval, u, out, mode, a, s); break;
    case 4: launch_sell_bsr3<T, VT, 4>(S, sval, u, out, mode, a, s); break;
    case 8: launch_sell_bsr3<T, VT, 8>(S, sval, u, out, mode, a, s); break;
    default: launch_sell_bsr3<T, VT, 16>(S, sval, u, out, mode, a, s); break;
  }
  CHNSS_LAUNCH_CK();
}

template <typename T>
void spmv_sell_bsr3(const Pattern &P, const T *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                    cudaStream_t s) {
  spmv_sell_bsr3_impl<T, T>(P, sval, u, out, mode, a, s);
}
template void spmv_sell_bsr3<double>(const Pattern &, const double *, const double *, double *, SpmvMode,
                                     const SpmvArgs &, cudaStream_t);
template void spmv_sell_bsr3<float>(const Pattern &, const float *, const float *, float *, SpmvMode,
                                    const SpmvArgs &, cudaStream_t);
void spmv_sell_bsr3(const Pattern &P, const __nv_bfloat16 *sval, const float *u, float *out, SpmvMode mode,
                    const SpmvArgs &a, cudaStream_t s) {
  spmv_sell_bsr3_impl<float, __nv_bfloat16>(P, sval, u, out, mode, a, s);
}

template <typename T, typename VT>
void cheb_block_bsr3(const Pattern &P, const VT *sval, const T *dinv, const T *b, T *x, T *t, const double *coef,
                     int degree, cudaStream_t s) {
  const Sell &S = P.sell;
  if (S.nslices < 1 || S.nslices > kChebBlockSlices)
    throw Error{CHNSS_ERR_ARG, "one-block Chebyshev: 1 to 8 slices of node rows"};
  if (degree < 1 || degree > kMaxSmoothDegree + 1) throw Error{CHNSS_ERR_ARG, "one-block Chebyshev: bad degree"};
  int ns = 1;
  while (ns < S.nslices) ns *= 2;
  k_cheb_bsr3_block<T, VT><<<1, 1024, 0, s>>>(S.nslices, 32 / ns, S.slice_ptr, S.rowid, S.col, sval, dinv, b, x, t,
                                               coef, degree, 3 * P.nrows);
  CHNSS_LAUNCH_CK();
}
template void cheb_block_bsr3<double, double>(const Pattern &, const double *, const double *, const double *,
                                              double *, double *, const double *, int, cudaStream_t);
template void cheb_block_bsr3<float, float>(const Pattern &, const float *, const float *, const float *, float *,
                                            float *, const double *, int, cudaStream_t);
template void cheb_block_bsr3<float, __nv_bfloat16>(const Pattern &, const __nv_bfloat16 *, const float *,
                                                    const float *, float *, float *, const double *, int,
                                                    cudaStream_t);

template <typename Tout>
void sell_gather9(long nent, const int *map9, const double *csr_vals, Tout *out, cudaStream_t s) {
  if (nent == 0) return;
  k_sell_gather9<Tout><<<nblocks(9 * nent, TPB), TPB, 0, s>>>(9 * nent, map9, csr_vals, out);
  CHNSS_LAUNCH_CK();
}
template void sell_gather9<double>(long, const int *, const double *, double *, cudaStream_t);
template void sell_gather9<float>(long, const int *, const double *, float *, cudaStream_t);
template void sell_gather9<__nv_bfloat16>(long, const int *, const double *, __nv_bfloat16 *, cudaStream_t);

int sell_warps_bsr2(const Sell &S) {
  const long target = 48L * device_sm_count();
  int K = 1;
  while (K < 8 && (long)S.nslices * K < target && S.wmax / (2 * K) >= 2) K *= 2;
  return K;
}

template <typename T, typename VT>
void spmv_sell_bsr2_impl(const Pattern &P, const VT *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                         cudaStream_t s) {
  const Sell &S = P.sell;
  if (S.nslices == 0) return;
  const int nb = nblocks((long)S.nslices * 32, S.block);
  if (!aligned(sval, 4 * sizeof(VT)))
    throw Error{CHNSS_ERR_ARG, "2x2-block values must be aligned to one block"};
  // coarse levels with fewer slices than one wave of warps: K warps per slice
  const int K = sell_warps_bsr2(S);
  if (K > 1) {
    const int spb = 8 / K;
    const int g = (S.nslices + spb - 1) / spb;
    if (K == 2)
      k_sell_bsr2_split<T, VT, 2><<<g, 256, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
    else if (K == 4)
      k_sell_bsr2_split<T, VT, 4><<<g, 256, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
    else
      k_sell_bsr2_split<T, VT, 8><<<g, 256, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
  } else if (aligned(u, 2 * sizeof(T)))
    k_sell_bsr2<T, VT, true><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
  else
    k_sell_bsr2<T, VT, false><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a);
  CHNSS_LAUNCH_CK();
}

template <typename T>
void spmv_sell(const Pattern &P, const T *sval, int ncomp, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
               cudaStream_t s) {
  spmv_sell_impl<T, T>(P, sval, ncomp, u, out, mode, a, s);
}
template void spmv_sell<double>(const Pattern &, const double *, int, const double *, double *, SpmvMode,
                                const SpmvArgs &, cudaStream_t);
template void spmv_sell<float>(const Pattern &, const float *, int, const float *, float *, SpmvMode,
                               const SpmvArgs &, cudaStream_t);
void spmv_sell(const Pattern &P, const __nv_bfloat16 *sval, int ncomp, const float *u, float *out, SpmvMode mode,
               const SpmvArgs &a, cudaStream_t s) {
  spmv_sell_impl<float, __nv_bfloat16>(P, sval, ncomp, u, out, mode, a, s);
}

template <typename T>
void spmv_sell_bsr2(const Pattern &P, const T *sval, const T *u, T *out, SpmvMode mode, const SpmvArgs &a,
                    cudaStream_t s) {
  spmv_sell_bsr2_impl<T, T>(P, sval, u, out, mode, a, s);
}
template void spmv_sell_bsr2<double>(const Pattern &, const double *, const double *, double *, SpmvMode,
                                     const SpmvArgs &, cudaStream_t);
template void spmv_sell_bsr2<float>(const Pattern &, const float *, const float *, float *, SpmvMode,
                                    const SpmvArgs &, cudaStream_t);
void spmv_sell_bsr2(const Pattern &P, const __nv_bfloat16 *sval, const float *u, float *out, SpmvMode mode,
                    const SpmvArgs &a, cudaStream_t s) {
  spmv_sell_bsr2_impl<float, __nv_bfloat16>(P, sval, u, out, mode, a, s);
}

void spmv_sell_ch(const Pattern &P, const double *L, const double *K, const double *k12, const double *M, double a12,
                  double a21, double a22, const double *x, double *y, cudaStream_t s) {
  const Sell &S = P.sell;
  k_sell_ch<<<nblocks((long)S.nslices * 32, S.block), S.block, 0, s>>>(S.nslices, P.nrows, S.slice_ptr, S.rowid, S.col, L, K,
                                                               k12, M, a12, a21, a22, x, y);
  CHNSS_LAUNCH_CK();
}
void spmv_sell_ch_multi(const Pattern &P, const double *L, const double *K, const double *k12, const double *M, int nr,
                        const ChCoef3 &cf, const MultiPtr<const double> &x, const MultiPtr<double> &y,
                        cudaStream_t s) {
  const Sell &S = P.sell;
  const int nb = nblocks((long)S.nslices * 32, S.block);
  switch (nr) {
    case 1:
      k_sell_ch_multi<1><<<nb, S.block, 0, s>>>(S.nslices, P.nrows, S.slice_ptr, S.rowid, S.col, L, K, k12, M, cf, x, y);
      break;
    case 2:
      k_sell_ch_multi<2><<<nb, S.block, 0, s>>>(S.nslices, P.nrows, S.slice_ptr, S.rowid, S.col, L, K, k12, M, cf, x, y);
      break;
    case 3:
      k_sell_ch_multi<3><<<nb, S.block, 0, s>>>(S.nslices, P.nrows, S.slice_ptr, S.rowid, S.col, L, K, k12, M, cf, x, y);
      break;
    default: throw Error{CHNSS_ERR_ARG, "CH operator: 1 to 3 systems"};
  }
  CHNSS_LAUNCH_CK();
}
void spmv_sell_b(const Pattern &P, const double *sval2, const double *v, double *y, cudaStream_t s) {
  const Sell &S = P.sell;
  const int nb = nblocks((long)S.nslices * 32, S.block);
  if (aligned(v, 16))
    k_sell_b<true><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval2, v, y);
  else
    k_sell_b<false><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval2, v, y);
  CHNSS_LAUNCH_CK();
}
void spmv_sell_bt_add(const Pattern &P, const double *sval2, const double *p, double *yv, cudaStream_t s) {
  const Sell &S = P.sell;
  k_sell_bt_add<<<nblocks((long)S.nslices * 32, S.block), S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval2, p,
                                                                   yv);
  CHNSS_LAUNCH_CK();
}

void spmv_ch(const Pattern &P, const double *L, const double *K, const double *k12, const double *M, double a12,
             double a21, double a22, const double *x, double *y, cudaStream_t s) {
  k_spmv_ch<<<nblocks((long)P.nrows * 8, TPB), TPB, 0, s>>>(P.nrows, P.rowptr, P.col, L, K, k12, M, a12, a21, a22,
                                                           x, y);
  CHNSS_LAUNCH_CK();
}
void spmv_b(const Pattern &P, const double *val, const double *v, double *y, cudaStream_t s) {
  k_spmv_b<<<nblocks((long)P.nrows * 8, TPB), TPB, 0, s>>>(P.nrows, P.rowptr, P.col, val, v, y);
  CHNSS_LAUNCH_CK();
}
void spmv_bt_add(const Pattern &P, const double *val, const double *p, double *yv, cudaStream_t s) {
  k_spmv_bt_add<<<nblocks((long)P.nrows * 4, TPB), TPB, 0, s>>>(P.nrows, P.rowptr, P.col, val, p, yv);
  CHNSS_LAUNCH_CK();
}

int device_sm_count() {
  constexpr int kDevs = 64;
  static std::atomic<int> cache[kDevs];
  int dev = 0;
  CHNSS_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kDevs) throw Error{CHNSS_ERR_ARG, "device index out of range"};
  int sms = cache[dev].load(std::memory_order_relaxed);
  if (sms == 0) {
    CHNSS_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms < 1) sms = 1;
    cache[dev].store(sms, std::memory_order_relaxed);
  }
  return sms;
}

int reduce_blocks(long n) {
  long b = (n + 4L * TPB - 1) / (4L * TPB);
  const long cap = std::min(8L * device_sm_count(), (long)kReduceMaxBlocks);   // 8 resident per SM
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

template <typename T>
void jacobi_csr(const Pattern &P, const double *val, const int *diag, T *dinv, double *hi, double *partial,
                cudaStream_t s) {
  const int nb = reduce_blocks(P.nrows);
  k_jacobi_csr<T><<<nb, TPB, 0, s>>>(P.nrows, P.rowptr, val, diag, dinv, partial);
  CHNSS_LAUNCH_CK();
  k_max_final<<<1, TPB, 0, s>>>(nb, partial, hi);
  CHNSS_LAUNCH_CK();
}
template <typename T>
void jacobi_bsr2(const Pattern &P, const double *val, const int *diag, T *dinv, double *hi, double *partial,
                 cudaStream_t s) {
  const int nb = reduce_blocks(P.nrows);
  k_jacobi_bsr2<T><<<nb, TPB, 0, s>>>(P.nrows, P.rowptr, val, diag, dinv, partial);
  CHNSS_LAUNCH_CK();
  k_max_final<<<1, TPB, 0, s>>>(nb, partial, hi);
  CHNSS_LAUNCH_CK();
}
template void jacobi_csr<double>(const Pattern &, const double *, const int *, double *, double *, double *,
                                 cudaStream_t);
template void jacobi_csr<float>(const Pattern &, const double *, const int *, float *, double *, double *,
                                cudaStream_t);
template void jacobi_bsr2<double>(const Pattern &, const double *, const int *, double *, double *, double *,
                                  cudaStream_t);
template void jacobi_bsr2<float>(const Pattern &, const double *, const int *, float *, double *, double *,
                                 cudaStream_t);

void cheb_coefficients(const double *hi, double ratio, int degree, double *coef, cudaStream_t s) {
  if (degree < 1 || degree > kMaxSmoothDegree) throw Error{CHNSS_ERR_ARG, "smoother degree out of range"};
  k_cheb_coef<<<1, 1, 0, s>>>(hi, ratio, degree, coef);
  CHNSS_LAUNCH_CK();
}

template <typename T>
void vec_scale_dinv(int n, const double *scale, const T *dinv, const T *b, T *out, cudaStream_t s) {
  k_scale_dinv<T><<<nblocks(n, TPB), TPB, 0, s>>>(n, scale, dinv, b, out);
  CHNSS_LAUNCH_CK();
}
template void vec_scale_dinv<double>(int, const double *, const double *, const double *, double *, cudaStream_t);
template void vec_scale_dinv<float>(int, const double *, const float *, const float *, float *, cudaStream_t);

template <typename Ta, typename Tb>
void vec_convert(long n, const Ta *in, Tb *out, cudaStream_t s) {
  if (n == 0) return;
  k_convert<Ta, Tb><<<nblocks(n, TPB), TPB, 0, s>>>(n, in, out);
  CHNSS_LAUNCH_CK();
}
template void vec_convert<double, float>(long, const double *, float *, cudaStream_t);
template void vec_convert<float, double>(long, const float *, double *, cudaStream_t);
template void vec_convert<double, double>(long, const double *, double *, cudaStream_t);
template void vec_convert<float, float>(long, const float *, float *, cudaStream_t);

template <typename Ta, typename Tb>
void vec_convert_from_slot(long n, const Ta *const *slot, long off, Tb *out, cudaStream_t s) {
  if (n == 0) return;
  k_convert_from_slot<Ta, Tb><<<nblocks(n, TPB), TPB, 0, s>>>(n, slot, off, out);
  CHNSS_LAUNCH_CK();
}
template <typename Ta, typename Tb>
void vec_convert_to_slot(long n, const Ta *in, Tb *const *slot, long off, cudaStream_t s) {
  if (n == 0) return;
  k_convert_to_slot<Ta, Tb><<<nblocks(n, TPB), TPB, 0, s>>>(n, in, slot, off);
  CHNSS_LAUNCH_CK();
}
template void vec_convert_from_slot<double, float>(long, const double *const *, long, float *, cudaStream_t);
template void vec_convert_from_slot<double, double>(long, const double *const *, long, double *, cudaStream_t);
template void vec_convert_to_slot<float, double>(long, const float *, double *const *, long, cudaStream_t);
template void vec_convert_to_slot<double, double>(long, const double *, double *const *, long, cudaStream_t);
struct PtrPack {
  const void *p[8];
};
__global__ void k_set_ptrs_n(void **slots, int n, PtrPack pk) {
  for (int i = 0; i < n; ++i) slots[i] = const_cast<void *>(pk.p[i]);
}
void set_ptr_slots_n(void **slots, int n, const void *const *ptrs, cudaStream_t s) {
  if (n < 1 || n > 8) throw Error{CHNSS_ERR_ARG, "set_ptr_slots_n: 1 to 8 pointers"};
  PtrPack pk{};
  for (int i = 0; i < n; ++i) pk.p[i] = ptrs[i];
  k_set_ptrs_n<<<1, 1, 0, s>>>(slots, n, pk);
  CHNSS_LAUNCH_CK();
}

void set_ptr_slots(void **slots, const void *a, const void *b, cudaStream_t s) {
  k_set_ptrs<<<1, 1, 0, s>>>(slots, a, b);
  CHNSS_LAUNCH_CK();
}

__global__ void k_clip01(long n, double *x) {
  const long i = (long)blockIdx.x * TPB + threadIdx.x;
  if (i < n) x[i] = fmin(fmax(x[i], 0.0), 1.0);
}
void vec_clip01(long n, double *x, cudaStream_t s) {
  if (n == 0) return;
  k_clip01<<<nblocks(n, TPB), TPB, 0, s>>>(n, x);
  CHNSS_LAUNCH_CK();
}

void vec_axpby(long n, double a, const double *x, double b, double *y, cudaStream_t s) {
  k_axpby<<<nblocks(n, TPB), TPB, 0, s>>>(n, a, x, b, y);
  CHNSS_LAUNCH_CK();
}
void vec_copy(long n, const double *x, double *y, cudaStream_t s) {
  k_copy<<<nblocks(n, TPB), TPB, 0, s>>>(n, x, y);
  CHNSS_LAUNCH_CK();
}
void vec_fill(long n, double v, double *y, cudaStream_t s) {
  k_fill<<<nblocks(n, TPB), TPB, 0, s>>>(n, v, y);
  CHNSS_LAUNCH_CK();
}
void vec_scale_by_inv(long n, const double *src, const double *hn, double *dst, cudaStream_t s) {
  k_scale_by_inv<<<nblocks(n, TPB), TPB, 0, s>>>(n, src, hn, dst);
  CHNSS_LAUNCH_CK();
}
template <typename T>
void vec_sub_mean(int n, T *x, const double *sum, cudaStream_t s) {
  k_sub_mean<T><<<nblocks(n, TPB), TPB, 0, s>>>(n, x, sum);
  CHNSS_LAUNCH_CK();
}
template void vec_sub_mean<double>(int, double *, const double *, cudaStream_t);
template void vec_sub_mean<float>(int, float *, const double *, cudaStream_t);
void vec_mul(long n, const double *a, const double *b, double *out, cudaStream_t s) {
  k_mul<<<nblocks(n, TPB), TPB, 0, s>>>(n, a, b, out);
  CHNSS_LAUNCH_CK();
}

void sum_partials(int nb, int k, const double *partial, double *out, cudaStream_t s) {
  k_sum_final<<<std::min(k, 64), TPB, 0, s>>>(nb, k, partial, out);
  CHNSS_LAUNCH_CK();
}

template <typename T>
void dot(long n, const T *x, const T *y, double *out, double *partial, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  k_dot<T><<<nb, TPB, 0, s>>>(n, x, y, partial);
  CHNSS_LAUNCH_CK();
  k_sum_final<<<1, TPB, 0, s>>>(nb, 1, partial, out);
  CHNSS_LAUNCH_CK();
}
template void dot<double>(long, const double *, const double *, double *, double *, cudaStream_t);
template void dot<float>(long, const float *, const float *, double *, double *, cudaStream_t);
template <typename T>
void vsum(long n, const T *x, double *out, double *partial, cudaStream_t s) {
  dot<T>(n, x, nullptr, out, partial, s);
}
template void vsum<double>(long, const double *, double *, double *, cudaStream_t);
template void vsum<float>(long, const float *, double *, double *, cudaStream_t);

void mdot(long n, const double *V, long ldv, int k, const double *w, double *out, double *partial, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  for (int k0 = 0; k0 < k; k0 += KC) {
    k_mdot<<<nb, TPB, 0, s>>>(n, V, ldv, k0, std::min(KC, k - k0), w, partial);
    CHNSS_LAUNCH_CK();
  }
  k_sum_final<<<std::min(k, 64), TPB, 0, s>>>(nb, k, partial, out);
  CHNSS_LAUNCH_CK();
}
void ortho_update_mdot(long n, const double *V, long ldv, int k, const double *h, double *w, double *out,
                       double *partial, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  // chunk 0 updates w in place and dots against vectors [0, 16); later
  // chunks see the updated w only if they run after chunk 0 finished, which
  // stream order guarantees, but they must not subtract again: recompute the
  // dots of later chunks with plain k_mdot on the updated w.
  k_ortho_update<0><<<nb, TPB, 0, s>>>(n, V, ldv, k, h, w, partial, 0, std::min(KC, k));
  CHNSS_LAUNCH_CK();
  for (int k0 = KC; k0 < k; k0 += KC) {
    k_mdot<<<nb, TPB, 0, s>>>(n, V, ldv, k0, std::min(KC, k - k0), w, partial);
    CHNSS_LAUNCH_CK();
  }
  k_sum_final<<<std::min(k, 64), TPB, 0, s>>>(nb, k, partial, out);
  CHNSS_LAUNCH_CK();
}
void ortho_update_norm(long n, const double *V, long ldv, int k, const double *h, double *w, double *out,
                       double *partial, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  k_ortho_update<1><<<nb, TPB, 0, s>>>(n, V, ldv, k, h, w, partial, 0, 1);
  CHNSS_LAUNCH_CK();
  k_sum_final<<<1, TPB, 0, s>>>(nb, 1, partial, out);
  CHNSS_LAUNCH_CK();
}
void combine_columns(long n, const double *Z, long ldz, int k, const double *y, double *x, cudaStream_t s) {
  k_combine<<<nblocks(n, TPB), TPB, 0, s>>>(n, Z, ldz, k, nullptr, y, x);
  CHNSS_LAUNCH_CK();
}
void combine_columns_dev(long n, const double *Z, long ldz, const int *k, const double *y, double *x,
                         cudaStream_t s) {
  k_combine<<<nblocks(n, TPB), TPB, 0, s>>>(n, Z, ldz, 0, k, y, x);
  CHNSS_LAUNCH_CK();
}
void arnoldi_finish(int j, int ldh, double *H, const double *h1, const double *h2, const double *nrm2, double *cs,
                    double *sn, double *g, double *status, cudaStream_t s) {
  k_arnoldi_finish<<<1, 1, 0, s>>>(j, ldh, H, h1, h2, nrm2, cs, sn, g, status, 0);
  CHNSS_LAUNCH_CK();
}
void arnoldi_finish_pyth(int j, int ldh, double *H, const double *h1, const double *h2w, double *cs, double *sn,
                         double *g, double *status, cudaStream_t s) {
  k_arnoldi_finish<<<1, 1, 0, s>>>(j, ldh, H, h1, h2w, h2w + j + 1, cs, sn, g, status, 1);
  CHNSS_LAUNCH_CK();
}

// ---- CGS2 passes with the vector count as a template parameter ----
bool cgs2_fast(int k) { return k >= 1 && k <= kCgsMaxK; }

namespace {
int cgs_blocks(long n) {
  long b = (n + kCgsBlock - 1) / kCgsBlock;
  const long cap = std::min((long)kCgsBlocksPerSm * device_sm_count(), (long)kReduceMaxBlocks);
  return (int)std::max(1L, std::min(b, cap));
}
// pass 1 reads KC + 1 streams per element with little FP64 work per load, so
// it needs every resident block the registers allow (latency-bound at 2 per SM)
template <int KC>
int cgs_dots_blocks(long n) {
  static const int occ = [] {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_cgs_dots<KC>, kCgsBlock, 0);
    cudaGetLastError();
    return o;
  }();
  const int sms = device_sm_count();
  const int cap = std::max(kCgsBlocksPerSm * sms, std::min(sms * occ, std::min(8 * sms, kReduceMaxBlocks)));
  const long b = (n + kCgsBlock - 1) / kCgsBlock;
  return (int)std::max(1L, std::min(b, (long)cap));
}

template <int KC>
void cgs_pass(int pass, long n, const double *V, long ld, const double *h, const double *w_in, double *w,
              const double *hn, double *out, double *partial, cudaStream_t s) {
  if (pass == 1) {
    const int nb = cgs_dots_blocks<KC>(n);
    k_cgs_dots<KC><<<nb, kCgsBlock, 0, s>>>(n, V, ld, w_in, partial);
    CHNSS_LAUNCH_CK();
    k_sum_final<<<KC, TPB, 0, s>>>(nb, KC, partial, out);
  } else if (pass == 2) {
    const int nb = cgs_blocks(n);
    k_cgs_update_dots<KC><<<nb, kCgsBlock, 0, s>>>(n, V, ld, h, w, partial);
    CHNSS_LAUNCH_CK();
    k_sum_final<<<KC + 1, TPB, 0, s>>>(nb, KC + 1, partial, out);
  } else {
    k_cgs_update_scale<KC><<<nblocks(n, kCgsBlock), kCgsBlock, 0, s>>>(n, V, ld, h, w_in, hn, out);
  }
  CHNSS_LAUNCH_CK();
}
void cgs_dispatch(int k, int pass, long n, const double *V, long ld, const double *h, const double *w_in, double *w,
                  const double *hn, double *out, double *partial, cudaStream_t s) {
  switch (k) {
#define CHNSS_CGS_CASE(K) \
  case K: cgs_pass<K>(pass, n, V, ld, h, w_in, w, hn, out, partial, s); break;
    CHNSS_CGS_CASE(1) CHNSS_CGS_CASE(2) CHNSS_CGS_CASE(3) CHNSS_CGS_CASE(4) CHNSS_CGS_CASE(5)
    CHNSS_CGS_CASE(6) CHNSS_CGS_CASE(7) CHNSS_CGS_CASE(8) CHNSS_CGS_CASE(9) CHNSS_CGS_CASE(10)
    CHNSS_CGS_CASE(11) CHNSS_CGS_CASE(12) CHNSS_CGS_CASE(13) CHNSS_CGS_CASE(14) CHNSS_CGS_CASE(15)
    CHNSS_CGS_CASE(16) CHNSS_CGS_CASE(17) CHNSS_CGS_CASE(18) CHNSS_CGS_CASE(19) CHNSS_CGS_CASE(20)
    CHNSS_CGS_CASE(21) CHNSS_CGS_CASE(22) CHNSS_CGS_CASE(23) CHNSS_CGS_CASE(24) CHNSS_CGS_CASE(25)
    CHNSS_CGS_CASE(26) CHNSS_CGS_CASE(27) CHNSS_CGS_CASE(28) CHNSS_CGS_CASE(29) CHNSS_CGS_CASE(30)
    CHNSS_CGS_CASE(31)
#undef CHNSS_CGS_CASE
    default: throw Error{CHNSS_ERR_ARG, "CGS2 fast path: k must be in [1, 31]"};
  }
}
}  // namespace

void cgs2_dots(long n, const double *V, long ld, int k, const double *w, double *h1, double *partial,
               cudaStream_t s) {
  cgs_dispatch(k, 1, n, V, ld, nullptr, w, nullptr, nullptr, h1, partial, s);
}
void cgs2_update_dots(long n, const double *V, long ld, int k, const double *h1, double *w, double *h2w,
                      double *partial, cudaStream_t s) {
  cgs_dispatch(k, 2, n, V, ld, h1, nullptr, w, nullptr, h2w, partial, s);
}
void cgs2_update_scale(long n, const double *V, long ld, int k, const double *h2, const double *w, const double *hn,
                       double *vout, cudaStream_t s) {
  cgs_dispatch(k, 3, n, V, ld, h2, w, nullptr, hn, vout, nullptr, s);
}
namespace {
// passes 1 and 2 stream KC + 1 vectors with few operations per load: every
// block the registers allow stays resident (capped by the partial buffers)
template <int KC, int PASS>
int dfgs_blocks(long n) {
  static const int occ = [] {
    int o = 0;
    const void *f = PASS == 1 ? (const void *)k_dfgs_dots<KC> : (const void *)k_dfgs_update_dots<KC>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, f, kCgsBlock, 0);
    cudaGetLastError();
    return o;
  }();
  const int sms = device_sm_count();
  const int cap = std::max(kCgsBlocksPerSm * sms, std::min(sms * occ, std::min(8 * sms, kReduceMaxBlocks)));
  const long b = (n + kCgsBlock - 1) / kCgsBlock;
  return (int)std::max(1L, std::min(b, (long)cap));
}

template <int KC>
void dfgs_pass(int pass, long n, const float2 *V, long ld, const double *h, double *w, const double *hn,
               double *out, float2 *out2, double *partial, cudaStream_t s) {
  if (pass == 1) {
    const int nb = dfgs_blocks<KC, 1>(n);
    k_dfgs_dots<KC><<<nb, kCgsBlock, 0, s>>>(n, V, ld, w, partial);
    CHNSS_LAUNCH_CK();
    k_sum_final<<<KC, TPB, 0, s>>>(nb, KC, partial, out);
  } else if (pass == 2) {
    const int nb = dfgs_blocks<KC, 2>(n);
    k_dfgs_update_dots<KC><<<nb, kCgsBlock, 0, s>>>(n, V, ld, h, w, partial);
    CHNSS_LAUNCH_CK();
    k_sum_final<<<KC + 1, TPB, 0, s>>>(nb, KC + 1, partial, out);
  } else {
    k_dfgs_update_scale<KC><<<nblocks(n, kCgsBlock), kCgsBlock, 0, s>>>(
        n, V, ld, h, reinterpret_cast<const float2 *>(w), hn, out2, out);
  }
  CHNSS_LAUNCH_CK();
}
void dfgs_dispatch(int k, int pass, long n, const float2 *V, long ld, const double *h, double *w, const double *hn,
                   double *out, float2 *out2, double *partial, cudaStream_t s) {
  switch (k) {
#define CHNSS_DFGS_CASE(K) \
  case K: dfgs_pass<K>(pass, n, V, ld, h, w, hn, out, out2, partial, s); break;
    CHNSS_DFGS_CASE(1) CHNSS_DFGS_CASE(2) CHNSS_DFGS_CASE(3) CHNSS_DFGS_CASE(4) CHNSS_DFGS_CASE(5)
    CHNSS_DFGS_CASE(6) CHNSS_DFGS_CASE(7) CHNSS_DFGS_CASE(8) CHNSS_DFGS_CASE(9) CHNSS_DFGS_CASE(10)
    CHNSS_DFGS_CASE(11) CHNSS_DFGS_CASE(12) CHNSS_DFGS_CASE(13) CHNSS_DFGS_CASE(14) CHNSS_DFGS_CASE(15)
    CHNSS_DFGS_CASE(16) CHNSS_DFGS_CASE(17) CHNSS_DFGS_CASE(18) CHNSS_DFGS_CASE(19) CHNSS_DFGS_CASE(20)
    CHNSS_DFGS_CASE(21) CHNSS_DFGS_CASE(22) CHNSS_DFGS_CASE(23) CHNSS_DFGS_CASE(24) CHNSS_DFGS_CASE(25)
    CHNSS_DFGS_CASE(26) CHNSS_DFGS_CASE(27) CHNSS_DFGS_CASE(28) CHNSS_DFGS_CASE(29) CHNSS_DFGS_CASE(30)
    CHNSS_DFGS_CASE(31)
#undef CHNSS_DFGS_CASE
    default: throw Error{CHNSS_ERR_ARG, "double-FP32 Gram-Schmidt: k must be in [1, 31]"};
  }
}
}  // namespace

void dfgs_dots(long n, const float2 *V, long ld, int k, const double *w, double *h1, double *partial,
               cudaStream_t s) {
  dfgs_dispatch(k, 1, n, V, ld, nullptr, const_cast<double *>(w), nullptr, h1, nullptr, partial, s);
}
void dfgs_update_dots(long n, const float2 *V, long ld, int k, const double *h1, double *w, double *h2w,
                      double *partial, cudaStream_t s) {
  dfgs_dispatch(k, 2, n, V, ld, h1, w, nullptr, h2w, nullptr, partial, s);
}
void dfgs_update_scale(long n, const float2 *V, long ld, int k, const double *h2, const double *w,
                       const double *hn, float2 *vout2, double *vout64, cudaStream_t s) {
  dfgs_dispatch(k, 3, n, V, ld, h2, const_cast<double *>(w), hn, vout64, vout2, nullptr, s);
}
void dfgs_first(long n, const double *w, const double *hn, float2 *vout2, double *vout64, cudaStream_t s) {
  k_df_first<<<nblocks(n, kCgsBlock), kCgsBlock, 0, s>>>(n, w, hn, vout2, vout64);
  CHNSS_LAUNCH_CK();
}

void hessenberg_solve(int k, int ldh, const double *H, const double *g, double *y, cudaStream_t s) {
  k_hessenberg_solve<<<1, 1, 0, s>>>(k, nullptr, ldh, H, g, y);
  CHNSS_LAUNCH_CK();
}
void hessenberg_solve_dev(const int *k, int ldh, const double *H, const double *g, double *y, cudaStream_t s) {
  k_hessenberg_solve<<<1, 1, 0, s>>>(0, k, ldh, H, g, y);
  CHNSS_LAUNCH_CK();
}
void set_scalar(double *dst, const double *src, double scale, bool sq, cudaStream_t s) {
  k_set_scalar<<<1, 1, 0, s>>>(dst, src, scale, sq ? 1 : 0);
  CHNSS_LAUNCH_CK();
}
void pcg_alpha(const double *rz, const double *pq, double *alpha, cudaStream_t s) {
  k_pcg_alpha<<<1, 1, 0, s>>>(rz, pq, alpha);
  CHNSS_LAUNCH_CK();
}
void pcg_update_xr(long n, const double *alpha, const double *p, const double *q, double *x, double *r,
                   cudaStream_t s) {
  k_pcg_xr<<<nblocks(n, TPB), TPB, 0, s>>>(n, alpha, p, q, x, r);
  CHNSS_LAUNCH_CK();
}
void pcg_update_p(long n, const double *rzn, const double *rzo, const double *z, double *p, cudaStream_t s) {
  k_pcg_p<<<nblocks(n, TPB), TPB, 0, s>>>(n, rzn, rzo, z, p);
  CHNSS_LAUNCH_CK();
}

void coarse_dense_csr(const Pattern &P, const double *val, double add_all, double *dense, cudaStream_t s) {
  k_dense_csr<<<nblocks(P.nrows, 128), 128, 0, s>>>(P.nrows, P.rowptr, P.col, val, add_all, dense);
  CHNSS_LAUNCH_CK();
}
void coarse_dense_bsr2(const Pattern &P, const double *val, double *dense, cudaStream_t s) {
  k_dense_bsr2<<<nblocks(P.nrows, 128), 128, 0, s>>>(P.nrows, P.rowptr, P.col, val, dense);
  CHNSS_LAUNCH_CK();
}
void dense_invert(int n, double *a, double *inv, int *status, cudaStream_t s) {
  k_dense_invert<<<1, TPB, 0, s>>>(n, a, inv, status);
  CHNSS_LAUNCH_CK();
}
template <typename T>
void dense_apply(int n, const double *inv, const T *b, T *x, cudaStream_t s) {
  k_dense_apply<T><<<nblocks(n, 128), 128, 0, s>>>(n, inv, b, x);
  CHNSS_LAUNCH_CK();
}
template void dense_apply<double>(int, const double *, const double *, double *, cudaStream_t);
template void dense_apply<float>(int, const double *, const float *, float *, cudaStream_t);

template <typename T>
void spmv_sell_multi(const Pattern &P, const T *sval, int nr, const MultiPtr<T> &u, const MultiPtr<T> &out,
                     SpmvMode mode, const MultiArgs<T> &a, cudaStream_t s) {
  const Sell &S = P.sell;
  if (S.nslices == 0) return;
  if (S.wmax > 8) throw Error{CHNSS_ERR_ARG, "multi-vector SpMV needs rows of at most 8 entries"};
  const int nb = nblocks((long)S.nslices * 32, S.block);
  if (S.stencil) {
    StencilOff so;
    for (int j = 0; j < 7; ++j) so.o[j] = S.soff[j];
    const int nbs = nblocks(P.nrows, S.block);
    switch (nr) {
      case 1: k_stencil7m<T, 1><<<nbs, S.block, 0, s>>>(P.nrows, so, sval, u, out, mode, a); break;
      case 2: k_stencil7m<T, 2><<<nbs, S.block, 0, s>>>(P.nrows, so, sval, u, out, mode, a); break;
      case 3: k_stencil7m<T, 3><<<nbs, S.block, 0, s>>>(P.nrows, so, sval, u, out, mode, a); break;
      default: throw Error{CHNSS_ERR_ARG, "multi-vector SpMV: 1 to 3 vectors"};
    }
    CHNSS_LAUNCH_CK();
    return;
  }
  switch (nr) {
    case 1: k_sell_w8m<T, 1><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a); break;
    case 2: k_sell_w8m<T, 2><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a); break;
    case 3: k_sell_w8m<T, 3><<<nb, S.block, 0, s>>>(S.nslices, S.slice_ptr, S.rowid, S.col, sval, u, out, mode, a); break;
    default: throw Error{CHNSS_ERR_ARG, "multi-vector SpMV: 1 to 3 vectors"};
  }
  CHNSS_LAUNCH_CK();
}
template void spmv_sell_multi<double>(const Pattern &, const double *, int, const MultiPtr<double> &,
                                      const MultiPtr<double> &, SpmvMode, const MultiArgs<double> &, cudaStream_t);
template void spmv_sell_multi<float>(const Pattern &, const float *, int, const MultiPtr<float> &,
                                     const MultiPtr<float> &, SpmvMode, const MultiArgs<float> &, cudaStream_t);

template <typename T>
void vec_scale_dinv_multi(int n, int nr, const double *scale, const T *dinv, const MultiPtr<T> &b,
                          const MultiPtr<T> &out, cudaStream_t s) {
  k_scale_dinv_m<T><<<nblocks(n, TPB), TPB, 0, s>>>(n, nr, scale, dinv, b, out);
  CHNSS_LAUNCH_CK();
}
template void vec_scale_dinv_multi<double>(int, int, const double *, const double *, const MultiPtr<double> &,
                                           const MultiPtr<double> &, cudaStream_t);
template void vec_scale_dinv_multi<float>(int, int, const double *, const float *, const MultiPtr<float> &,
                                          const MultiPtr<float> &, cudaStream_t);

template <typename T>
void dense_apply_multi(int n, int nr, const double *inv, const MultiPtr<T> &b, const MultiPtr<T> &x,
                       cudaStream_t s) {
  k_dense_apply_m<T><<<nblocks(n, 128), 128, 0, s>>>(n, nr, inv, b, x);
  CHNSS_LAUNCH_CK();
}
template void dense_apply_multi<double>(int, int, const double *, const MultiPtr<double> &, const MultiPtr<double> &,
                                        cudaStream_t);
template void dense_apply_multi<float>(int, int, const double *, const MultiPtr<float> &, const MultiPtr<float> &,
                                       cudaStream_t);

template <typename T>
void mg_tail(const TailDesc<T> *d_desc, int nr, int width, cudaStream_t s) {
  if (width != 8 && width != 16) throw Error{CHNSS_ERR_ARG, "coarse-level block: rows of 8 or 16 entries"};
  const bool w16 = width == 16;
  switch (nr) {
    case 1:
      if (w16) k_mg_tail<T, 1, 16><<<1, 512, 0, s>>>(d_desc);
      else k_mg_tail<T, 1, 8><<<1, 512, 0, s>>>(d_desc);
      break;
    case 2:
      if (w16) k_mg_tail<T, 2, 16><<<1, 512, 0, s>>>(d_desc);
      else k_mg_tail<T, 2, 8><<<1, 512, 0, s>>>(d_desc);
      break;
    case 3:
      if (w16) k_mg_tail<T, 3, 16><<<1, 512, 0, s>>>(d_desc);
      else k_mg_tail<T, 3, 8><<<1, 512, 0, s>>>(d_desc);
      break;
    default: throw Error{CHNSS_ERR_ARG, "coarse-level block: 1 to 3 vectors"};
  }
  CHNSS_LAUNCH_CK();
}
template void mg_tail<double>(const TailDesc<double> *, int, int, cudaStream_t);
template void mg_tail<float>(const TailDesc<float> *, int, int, cudaStream_t);

template <typename T>
void vec_copy_multi(long n, int nr, const MultiPtr<T> &in, const MultiPtr<T> &out, cudaStream_t s) {
  if (n == 0) return;
  k_copy_m<T><<<nblocks(n, TPB), TPB, 0, s>>>(n, nr, in, out);
  CHNSS_LAUNCH_CK();
}
template void vec_copy_multi<double>(long, int, const MultiPtr<double> &, const MultiPtr<double> &, cudaStream_t);
template void vec_copy_multi<float>(long, int, const MultiPtr<float> &, const MultiPtr<float> &, cudaStream_t);

}  // namespace chnss
