// Finite-element assembly kernels (paper Sec. 3-4).
//
// One thread per triangle computes a dense element matrix (or load vector)
// from the nodal coefficients and the exact reference tensors (integrals of
// barycentric polynomials, held in constant memory) and writes it to an
// element buffer.  A gather kernel then sums, for every CSR entry, its
// element contributions in element order (precomputed lists): no atomics,
// bit-reproducible results.
#include <cmath>

#include "internal.h"

namespace chnss {

__constant__ RefTensors c_ref;

void upload_reference_tensors(cudaStream_t s) {
  const RefTensors &t = reference_tensors();
  CHNSS_CK(cudaMemcpyToSymbolAsync(c_ref, &t, sizeof(RefTensors), 0, cudaMemcpyHostToDevice, s));
}

namespace {

constexpr int TPB = 128;

inline int blocks_for(long n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

// Element e of a structured level: P1 vertex ids, P2 lattice ids (vertices,
// then midpoints of the edges opposite vertex 0, 1, 2), barycentric
// gradients and area.  Lower triangle (i,j),(i+1,j),(i+1,j+1); upper
// (i,j),(i+1,j+1),(i,j+1).
struct Elem {
  int v1[3];
  int v2[6];
  double gl[3][2];
  double area;
};

__device__ __forceinline__ void element(const Geo &g, int e, Elem &el) {
  const int n = g.n, s = e >> 1, o = e & 1, i = s % n, j = s / n;
  const double ix = 1.0 / g.hx, iy = 1.0 / g.hy;
  int vi[3], vj[3];
  vi[0] = i; vj[0] = j;
  if (o == 0) {
    vi[1] = i + 1; vj[1] = j; vi[2] = i + 1; vj[2] = j + 1;
    el.gl[0][0] = -ix; el.gl[0][1] = 0.0;
    el.gl[1][0] = ix;  el.gl[1][1] = -iy;
    el.gl[2][0] = 0.0; el.gl[2][1] = iy;
  } else {
    vi[1] = i + 1; vj[1] = j + 1; vi[2] = i; vj[2] = j + 1;
    el.gl[0][0] = 0.0; el.gl[0][1] = -iy;
    el.gl[1][0] = ix;  el.gl[1][1] = 0.0;
    el.gl[2][0] = -ix; el.gl[2][1] = iy;
  }
  const int m = 2 * n + 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    el.v1[k] = vj[k] * (n + 1) + vi[k];
    el.v2[k] = (2 * vj[k]) * m + 2 * vi[k];
  }
  el.v2[3] = (vj[1] + vj[2]) * m + (vi[1] + vi[2]);
  el.v2[4] = (vj[0] + vj[2]) * m + (vi[0] + vi[2]);
  el.v2[5] = (vj[0] + vj[1]) * m + (vi[0] + vi[1]);
  el.area = 0.5 * g.hx * g.hy;
}

// shift = sum_i alpha_i grad mu_i on the element (piecewise constant)
__device__ __forceinline__ void element_shift(const Elem &el, const double *const *mu, const double *alpha,
                                              double sh[2]) {
  sh[0] = sh[1] = 0.0;
  if (!mu) return;
  for (int f = 0; f < 4; ++f) {
    const double a = alpha[f];
    if (a == 0.0 || !mu[f]) continue;
    for (int k = 0; k < 3; ++k) {
      const double m = mu[f][el.v1[k]];
      sh[0] += a * m * el.gl[k][0];
      sh[1] += a * m * el.gl[k][1];
    }
  }
}

struct MuPtrs {
  const double *mu[4];
  double alpha[4];
  int has;
};

__global__ void k_p1_mass(Geo g, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  const double area = 0.5 * g.hx * g.hy;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) buf[(long)e * 9 + a * 3 + b] = area * c_ref.m1[a][b];
}

__global__ void k_p1_stiff(Geo g, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      buf[(long)e * 9 + a * 3 + b] = el.area * (el.gl[a][0] * el.gl[b][0] + el.gl[a][1] * el.gl[b][1]);
}

// C_ab = int ((v - shift) . grad lambda_b) lambda_a, v a P2 field
__global__ void k_p1_conv(Geo g, const double *__restrict__ v, MuPtrs mp, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  double sh[2];
  element_shift(el, mp.has ? mp.mu : nullptr, mp.alpha, sh);
  double vk[6][2];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    vk[k][0] = v[2 * el.v2[k]];
    vk[k][1] = v[2 * el.v2[k] + 1];
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    double vg[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) vg[k] = vk[k][0] * el.gl[b][0] + vk[k][1] * el.gl[b][1];
    const double sg = sh[0] * el.gl[b][0] + sh[1] * el.gl[b][1];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double s = -sg * (1.0 / 3.0);
#pragma unroll
      for (int k = 0; k < 6; ++k) s += vg[k] * c_ref.c1[k][a];
      buf[(long)e * 9 + a * 3 + b] = el.area * s;
    }
  }
}

// K_kappa with kappa = gamma (phi (1 - phi) + m0), phi P1
__global__ void k_p1_wstiff(Geo g, const double *__restrict__ phi, double gamma, double m0, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  double f[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = phi[el.v1[k]];
  double i1 = (f[0] + f[1] + f[2]) * (1.0 / 3.0), i2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) i2 += f[k] * f[l] * c_ref.m1[k][l];
  const double kint = el.area * gamma * (i1 - i2 + m0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      buf[(long)e * 9 + a * 3 + b] = kint * (el.gl[a][0] * el.gl[b][0] + el.gl[a][1] * el.gl[b][1]);
}

__global__ void k_p2_mass(Geo g, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  const double area = 0.5 * g.hx * g.hy;
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = 0; b < 6; ++b) buf[(long)e * 36 + a * 6 + b] = area * c_ref.m2[a][b];
}

// j_ab = int ((v - shift) . grad zeta_b) zeta_a (eqn:matrixns)
__global__ void k_p2_conv(Geo g, const double *__restrict__ v, MuPtrs mp, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  double sh[2];
  element_shift(el, mp.has ? mp.mu : nullptr, mp.alpha, sh);
  double c[6][3], sg[3];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double vx = v[2 * el.v2[k]], vy = v[2 * el.v2[k] + 1];
#pragma unroll
    for (int l = 0; l < 3; ++l) c[k][l] = vx * el.gl[l][0] + vy * el.gl[l][1];
  }
#pragma unroll
  for (int l = 0; l < 3; ++l) sg[l] = sh[0] * el.gl[l][0] + sh[1] * el.gl[l][1];
  for (int a = 0; a < 6; ++a) {
    for (int b = 0; b < 6; ++b) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        s -= sg[l] * c_ref.jg[l][b][a];
#pragma unroll
        for (int k = 0; k < 6; ++k) s += c[k][l] * c_ref.j[k][l][b][a];
      }
      buf[(long)e * 36 + a * 6 + b] = el.area * s;
    }
  }
}

// k_{(a,c),(b,d)} = eta int (delta_cd grad zeta_b . grad zeta_a + d_c zeta_b d_d zeta_a),
// element layout [e][a][b][c][d]
__global__ void k_ksym(Geo g, double eta, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double X[2][2] = {{0, 0}, {0, 0}};   // X[c][d] = int d_c zeta_b d_d zeta_a / |T|
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const double t = c_ref.s[l][b][m][a];
#pragma unroll
          for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int d = 0; d < 2; ++d) X[cc][d] += el.gl[l][cc] * el.gl[m][d] * t;
        }
      const double lap = X[0][0] + X[1][1];
      const double f = eta * el.area;
      double *o = buf + (long)e * 144 + (a * 6 + b) * 4;
      o[0] = f * (lap + X[0][0]);
      o[1] = f * X[0][1];
      o[2] = f * X[1][0];
      o[3] = f * (lap + X[1][1]);
    }
}

// b_{a,(b,d)} = - int lambda_a d_d zeta_b, layout [e][a][b][d]
__global__ void k_bdiv(Geo g, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 6; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < 3; ++l) s += el.gl[l][d] * c_ref.b[a][b][l];
        buf[(long)e * 36 + (a * 6 + b) * 2 + d] = -el.area * s;
      }
}

// Potential loads of eqn:appPotential: int df/dphi_i lambda_a (i = p, NFA,
// s, a with phi_a = 1 - sum) and int df/dPhi_v lambda_a, layout [f][e][a].
__global__ void k_loads(Geo g, const double *__restrict__ pp, const double *__restrict__ pn,
                        const double *__restrict__ ps, const double *__restrict__ Ph, double *buf) {
  const int E = 2 * g.n * g.n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  Elem el;
  element(g, e, el);
  double fp[3], fn[3], fs[3], fv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    fp[k] = pp[el.v1[k]]; fn[k] = pn[el.v1[k]]; fs[k] = ps[el.v1[k]]; fv[k] = Ph[el.v1[k]];
  }
  double acc[5][3];
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[f][a] = 0.0;
  for (int q = 0; q < 20; ++q) {
    const double l0 = c_ref.qlam[q][0], l1 = c_ref.qlam[q][1], l2 = c_ref.qlam[q][2], w = c_ref.qw[q];
    const double p = l0 * fp[0] + l1 * fp[1] + l2 * fp[2];
    const double nn = l0 * fn[0] + l1 * fn[1] + l2 * fn[2];
    const double s = l0 * fs[0] + l1 * fs[1] + l2 * fs[2];
    const double V = l0 * fv[0] + l1 * fv[1] + l2 * fv[2];
    const double a = 1.0 - p - nn - s;
    const double ip = V * V * (3.0 - 2.0 * V), dip = 6.0 * V * (1.0 - V);
    const double liq = 3.5 * p * p * nn * nn + 0.3 * s * s + 0.3 * a * a - 10.0 * s * a;
    const double gas = 3.5 * p * p + 3.5 * nn * nn + 2.0 * s * s + 0.1 * a * a;
    double d[5];
    d[0] = (1.0 - ip) * 7.0 * p * nn * nn + ip * 7.0 * p;
    d[1] = (1.0 - ip) * 7.0 * p * p * nn + ip * 7.0 * nn;
    d[2] = (1.0 - ip) * (0.6 * s - 10.0 * a) + ip * 4.0 * s;
    d[3] = (1.0 - ip) * (0.6 * a - 10.0 * s) + ip * 0.2 * a;
    d[4] = dip * (gas - liq);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const double wd = w * d[f];
      acc[f][0] += wd * l0;
      acc[f][1] += wd * l1;
      acc[f][2] += wd * l2;
    }
  }
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 3; ++a) buf[(long)f * E * 3 + (long)e * 3 + a] = el.area * acc[f][a];
}

// Korteweg load G_(a,c) = int sum_b G_cb d_b zeta_a with
// G = sum_i beta_i grad phi_i (x) grad phi_i + beta_v grad Phi (x) grad Phi.
__global__ void k_korteweg(Geo g, const double *__restrict__ pp, const double *__restrict__ pn,
                           const double *__restrict__ ps, const double *__restrict__ Ph, KortewegCoef kc,
                           double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  double gr[5][2];
  const double *fld[4] = {pp, pn, ps, Ph};
  for (int f = 0; f < 4; ++f) {
    const int dst = f < 3 ? f : 4;
    gr[dst][0] = gr[dst][1] = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double x = fld[f][el.v1[k]];
      gr[dst][0] += x * el.gl[k][0];
      gr[dst][1] += x * el.gl[k][1];
    }
  }
  gr[3][0] = -(gr[0][0] + gr[1][0] + gr[2][0]);
  gr[3][1] = -(gr[0][1] + gr[1][1] + gr[2][1]);
  double G[2][2] = {{0, 0}, {0, 0}};
  for (int f = 0; f < 5; ++f) {
    const double bta = f < 4 ? kc.beta[f] : kc.beta_v;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) G[c][b] += bta * gr[f][c] * gr[f][b];
  }
  for (int a = 0; a < 6; ++a) {
    double ga[2];   // int d_b zeta_a / |T|
#pragma unroll
    for (int b = 0; b < 2; ++b)
      ga[b] = el.gl[0][b] * c_ref.g[a][0] + el.gl[1][b] * c_ref.g[a][1] + el.gl[2][b] * c_ref.g[a][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) buf[(long)e * 12 + a * 2 + c] = el.area * (G[c][0] * ga[0] + G[c][1] * ga[1]);
  }
}

__global__ void k_gather(int nout, int ncomp, const int *__restrict__ ptr, const int *__restrict__ idx,
                         const double *__restrict__ buf, double alpha, const double *__restrict__ base,
                         double beta, double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nout) return;
  const int b0 = ptr[k], b1 = ptr[k + 1];
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (int j = b0; j < b1; ++j) s += buf[idx[j] + c];
    const double bv = base ? beta * base[(long)k * ncomp + c] : 0.0;
    out[(long)k * ncomp + c] = bv + alpha * s;
  }
}

__global__ void k_gather_diag2(int nout, const int *__restrict__ ptr, const int *__restrict__ idx,
                               const double *__restrict__ buf, double alpha, const double *__restrict__ base,
                               double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nout) return;
  double s = 0.0;
  for (int j = ptr[k]; j < ptr[k + 1]; ++j) s += buf[idx[j]];
  s *= alpha;
  const double *b = base + 4L * k;
  double *o = out + 4L * k;
  o[0] = b[0] + s;
  o[1] = b[1];
  o[2] = b[2];
  o[3] = b[3] + s;
}

__global__ void k_inject_p1(int nf, const double *__restrict__ fine, double *__restrict__ coarse) {
  const int nc = nf / 2, mc = nc + 1;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= mc * mc) return;
  const int i = id % mc, j = id / mc;
  coarse[id] = fine[(2 * j) * (nf + 1) + 2 * i];
}

__global__ void k_inject_vel(int nf, const double *__restrict__ fine, double *__restrict__ coarse) {
  const int mf = 2 * nf + 1, mc = nf + 1;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= mc * mc) return;
  const int I = id % mc, J = id / mc;
  const long f = (long)(2 * J) * mf + 2 * I;
  coarse[2 * id] = fine[2 * f];
  coarse[2 * id + 1] = fine[2 * f + 1];
}

MuPtrs mu_ptrs(const double *const *mu, const double *alpha) {
  MuPtrs m{};
  m.has = mu != nullptr;
  for (int f = 0; f < 4; ++f) {
    m.mu[f] = mu ? mu[f] : nullptr;
    m.alpha[f] = alpha ? alpha[f] : 0.0;
  }
  return m;
}

}  // namespace

void launch_elem_p1_mass(Geo g, double *buf, cudaStream_t s) {
  k_p1_mass<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_p1_stiff(Geo g, double *buf, cudaStream_t s) {
  k_p1_stiff<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_p1_conv(Geo g, const double *v, const double *const *mu, const double *alpha, double *buf,
                         cudaStream_t s) {
  k_p1_conv<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, v, mu_ptrs(mu, alpha), buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_p1_wstiff(Geo g, const double *phi, double gamma, double m0, double *buf, cudaStream_t s) {
  k_p1_wstiff<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, phi, gamma, m0, buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_p2_mass(Geo g, double *buf, cudaStream_t s) {
  k_p2_mass<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_p2_conv(Geo g, const double *v, const double *const *mu, const double *alpha, double *buf,
                         cudaStream_t s) {
  k_p2_conv<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, v, mu_ptrs(mu, alpha), buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_ksym(Geo g, double eta, double *buf, cudaStream_t s) {
  k_ksym<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, eta, buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_bdiv(Geo g, double *buf, cudaStream_t s) {
  k_bdiv<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_loads(Geo g, const double *pp, const double *pn, const double *ps, const double *Ph,
                       double *buf, cudaStream_t s) {
  k_loads<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, pp, pn, ps, Ph, buf);
  CHNSS_LAUNCH_CK();
}
void launch_elem_korteweg(Geo g, const double *pp, const double *pn, const double *ps, const double *Ph,
                          KortewegCoef c, double *buf, cudaStream_t s) {
  k_korteweg<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, pp, pn, ps, Ph, c, buf);
  CHNSS_LAUNCH_CK();
}
void launch_gather(const Gather &g, int ncomp, const double *buf, double alpha, const double *base, double beta,
                   double *out, cudaStream_t s) {
  if (g.nout == 0) return;
  k_gather<<<blocks_for(g.nout, 256), 256, 0, s>>>(g.nout, ncomp, g.ptr, g.idx, buf, alpha, base, beta, out);
  CHNSS_LAUNCH_CK();
}
void launch_gather_diag2(const Gather &g, const double *buf, double alpha, const double *base, double *out,
                         cudaStream_t s) {
  if (g.nout == 0) return;
  k_gather_diag2<<<blocks_for(g.nout, 256), 256, 0, s>>>(g.nout, g.ptr, g.idx, buf, alpha, base, out);
  CHNSS_LAUNCH_CK();
}
void launch_inject_p1(int nf, const double *fine, double *coarse, cudaStream_t s) {
  const int mc = nf / 2 + 1;
  k_inject_p1<<<blocks_for((long)mc * mc, 256), 256, 0, s>>>(nf, fine, coarse);
  CHNSS_LAUNCH_CK();
}
void launch_inject_vel(int nf, const double *fine, double *coarse, cudaStream_t s) {
  const int mc = nf + 1;
  k_inject_vel<<<blocks_for((long)mc * mc, 256), 256, 0, s>>>(nf, fine, coarse);
  CHNSS_LAUNCH_CK();
}

}  // namespace chnss
