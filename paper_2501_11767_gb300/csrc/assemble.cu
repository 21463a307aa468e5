// Finite-element assembly kernels (paper Sec. 3-4).
//
// One thread per triangle computes a dense element matrix (or load vector)
// from the nodal coefficients and the exact reference tensors (integrals of
// barycentric polynomials, held in constant memory) and writes it to an
// element buffer.  A gather kernel then sums, for every CSR entry, its
// element contributions in element order (precomputed lists): no atomics,
// bit-reproducible results.
#include <cmath>

#include "kernels.h"

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

// x ln x replaced by its Taylor polynomial of degree 4 at 1/2 (Sec. 5); with
// d = x - 1/2 the coefficients are the derivatives of x ln x at 1/2 over k!:
// -ln2/2, 1 - ln2, 2/2!, -4/3!, 16/4!.  Returns the derivative.
__device__ __forceinline__ double taylor_xlnx(double x, double *deriv) {
  const double ln2 = 0.69314718055994530942;
  const double c0 = -0.5 * ln2, c1 = 1.0 - ln2, c2 = 1.0, c3 = -2.0 / 3.0, c4 = 2.0 / 3.0;
  const double d = x - 0.5;
  *deriv = c1 + d * (2.0 * c2 + d * (3.0 * c3 + d * 4.0 * c4));
  return c0 + d * (c1 + d * (c2 + d * (c3 + d * c4)));
}

// Potential loads: int df/dphi_i lambda_a (i = p, NFA, s, a with phi_a = 1 -
// sum) and int df/dPhi_v lambda_a, layout [f][e][a].  Model 0: eqn:appPotential;
// model 1 (solvent-air, Sec. 5.1): f_liq = g(s)/N_s + g(a)/N_a + chi s a,
// f_gas = g(s) - s ln phi_sat(s) + g(a) - a ln phi_sat(a), g = Taylor(x ln x),
// the polymer / NFA loads are zero.
__global__ void k_loads(Geo g, const double *__restrict__ pp, const double *__restrict__ pn,
                        const double *__restrict__ ps, const double *__restrict__ Ph, PotentialCoef pc,
                        double *buf) {
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
    double d[5];
    if (pc.model == 0) {
      const double liq = 3.5 * p * p * nn * nn + 0.3 * s * s + 0.3 * a * a - 10.0 * s * a;
      const double gas = 3.5 * p * p + 3.5 * nn * nn + 2.0 * s * s + 0.1 * a * a;
      d[0] = (1.0 - ip) * 7.0 * p * nn * nn + ip * 7.0 * p;
      d[1] = (1.0 - ip) * 7.0 * p * p * nn + ip * 7.0 * nn;
      d[2] = (1.0 - ip) * (0.6 * s - 10.0 * a) + ip * 4.0 * s;
      d[3] = (1.0 - ip) * (0.6 * a - 10.0 * s) + ip * 0.2 * a;
      d[4] = dip * (gas - liq);
    } else {
      double gs1, ga1;
      const double gs = taylor_xlnx(s, &gs1), ga = taylor_xlnx(a, &ga1);
      const double liq = gs * pc.inv_ns + ga * pc.inv_na + pc.chi_sa * s * a;
      const double gas = gs - s * pc.ln_sat_s + ga - a * pc.ln_sat_a;
      d[0] = 0.0;
      d[1] = 0.0;
      d[2] = (1.0 - ip) * (gs1 * pc.inv_ns + pc.chi_sa * a) + ip * (gs1 - pc.ln_sat_s);
      d[3] = (1.0 - ip) * (ga1 * pc.inv_na + pc.chi_sa * s) + ip * (ga1 - pc.ln_sat_a);
      d[4] = dip * (gas - liq);
    }
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

// Free-energy density f at one point (model 0: eqn:appPotential; model 1:
// the solvent-air density of Sec. 5.1 with the Taylor-expanded x ln x).
__device__ __forceinline__ double potential_value(const PotentialCoef &pc, double p, double nn, double s, double a,
                                                  double V) {
  const double ip = V * V * (3.0 - 2.0 * V);
  if (pc.model == 0) {
    const double liq = 3.5 * p * p * nn * nn + 0.3 * s * s + 0.3 * a * a - 10.0 * s * a;
    const double gas = 3.5 * p * p + 3.5 * nn * nn + 2.0 * s * s + 0.1 * a * a;
    return (1.0 - ip) * liq + ip * gas;
  }
  double d;
  const double gs = taylor_xlnx(s, &d), ga = taylor_xlnx(a, &d);
  const double liq = gs * pc.inv_ns + ga * pc.inv_na + pc.chi_sa * s * a;
  const double gas = gs - s * pc.ln_sat_s + ga - a * pc.ln_sat_a;
  return (1.0 - ip) * liq + ip * gas;
}

// Diagnostics of a state, one pass over the elements (fixed grid, each
// thread its elements in grid-stride order, then the block in a fixed
// order: bit-reproducible).  Per element, exactly:
//   q 0..3  int phi_i = |T|/3 sum of the vertex values (i = p, NFA, s, and
//           phi_a = 1 - sum phi), the entries of 1^T M phi_i;
//   q 4     int p, likewise;
//   q 5     int f(phi, Phi_v), 20-point rule exact to degree 7;
//   q 6     |T| (sum_i beta_i |grad phi_i|^2 + beta_v |grad Phi_v|^2) / 2;
//   q 7     |T| / 2 sum_ab m2_ab (v_a . v_b), the P2 mass form of the velocity.
// partial[q * gridDim.x + blockIdx.x] = block sum of quantity q.
constexpr int kDiagBlock = 256;
__global__ void __launch_bounds__(kDiagBlock) k_diag(Geo g, DiagArgs d, double *__restrict__ partial) {
  const int E = 2 * g.n * g.n;
  double acc[kDiagQuantities];
#pragma unroll
  for (int q = 0; q < kDiagQuantities; ++q) acc[q] = 0.0;
  for (int e = blockIdx.x * kDiagBlock + threadIdx.x; e < E; e += gridDim.x * kDiagBlock) {
    Elem el;
    element(g, e, el);
    double f[5][3];
    const double *fld[5] = {d.pp, d.pn, d.ps, d.Ph, d.p};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < 5; ++c) f[c][k] = fld[c][el.v1[k]];
    const double a3 = el.area / 3.0;
    double sa = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double sc = f[c][0] + f[c][1] + f[c][2];
      acc[c] += a3 * sc;
      sa += sc;
    }
    acc[3] += a3 * (3.0 - sa);
    acc[4] += a3 * (f[4][0] + f[4][1] + f[4][2]);
    double loc = 0.0;
    for (int q = 0; q < 20; ++q) {
      const double l0 = c_ref.qlam[q][0], l1 = c_ref.qlam[q][1], l2 = c_ref.qlam[q][2];
      const double pp = l0 * f[0][0] + l1 * f[0][1] + l2 * f[0][2];
      const double pn = l0 * f[1][0] + l1 * f[1][1] + l2 * f[1][2];
      const double ps = l0 * f[2][0] + l1 * f[2][1] + l2 * f[2][2];
      const double V = l0 * f[3][0] + l1 * f[3][1] + l2 * f[3][2];
      loc += c_ref.qw[q] * potential_value(d.pc, pp, pn, ps, 1.0 - pp - pn - ps, V);
    }
    acc[5] += el.area * loc;
    double ge = 0.0;
    double ga[2] = {0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double gx = 0.0, gy = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gx += f[c][k] * el.gl[k][0];
        gy += f[c][k] * el.gl[k][1];
      }
      if (c < 3) {
        ge += d.beta[c] * (gx * gx + gy * gy);
        ga[0] -= gx;
        ga[1] -= gy;
      } else {
        ge += d.beta_v * (gx * gx + gy * gy);
      }
    }
    ge += d.beta[3] * (ga[0] * ga[0] + ga[1] * ga[1]);   // grad phi_a = -sum grad phi_i
    acc[6] += 0.5 * el.area * ge;
    double vx[6], vy[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      vx[k] = d.v[2L * el.v2[k]];
      vy[k] = d.v[2L * el.v2[k] + 1];
    }
    double ke = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = 0; b < 6; ++b) ke += c_ref.m2[a][b] * (vx[a] * vx[b] + vy[a] * vy[b]);
    acc[7] += 0.5 * el.area * ke;
  }
  // block sums in a fixed order: warp butterflies, then the warps' results
  __shared__ double red[kDiagBlock / 32][kDiagQuantities];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kDiagQuantities; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagQuantities) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kDiagBlock / 32; ++w) t += red[w][threadIdx.x];
    partial[(long)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
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

int launch_diagnostics(Geo g, const DiagArgs &d, double *partial, cudaStream_t s) {
  const long E = 2L * g.n * g.n;
  const int nb = reduce_blocks(E);
  k_diag<<<nb, kDiagBlock, 0, s>>>(g, d, partial);
  CHNSS_LAUNCH_CK();
  return nb;
}

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
                       PotentialCoef pc, double *buf, cudaStream_t s) {
  k_loads<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, pp, pn, ps, Ph, pc, buf);
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

// ===========================================================================
// Adjoint (transposed Jacobian) element kernels.  Each writes per-element
// contributions that the node gather lists sum in element order.
namespace chnss {
namespace {

// d/dv of y^T C(v) x (P1 x, y): int zeta_k (d_d x) y -> buf [E][6][2]
__global__ void k_adj_conv_p1(Geo g, const double *__restrict__ x, const double *__restrict__ y, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  double gx[2] = {0.0, 0.0}, ya[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double xv = x[el.v1[k]];
    gx[0] += xv * el.gl[k][0];
    gx[1] += xv * el.gl[k][1];
    ya[k] = y[el.v1[k]];
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double s = el.area * (ya[0] * c_ref.c1[k][0] + ya[1] * c_ref.c1[k][1] + ya[2] * c_ref.c1[k][2]);
    buf[(long)e * 12 + k * 2] = s * gx[0];
    buf[(long)e * 12 + k * 2 + 1] = s * gx[1];
  }
}

// d/dphi of y^T K_kappa(phi) x, kappa = gamma (phi (1 - phi) + m0):
// entry c of an element = int gamma (1 - 2 phi_h) psi_c grad x_h . grad y_h
// = |T| gamma (grad x . grad y) (1/3 - (sum_d phi_d + phi_c) / 6)  [E][3]
__global__ void k_adj_wstiff(Geo g, const double *__restrict__ phi, double gamma, const double *__restrict__ x,
                             const double *__restrict__ y, double *buf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  double gx[2] = {0.0, 0.0}, gy[2] = {0.0, 0.0}, ph[3], psum = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double xv = x[el.v1[k]], yv = y[el.v1[k]];
    gx[0] += xv * el.gl[k][0];
    gx[1] += xv * el.gl[k][1];
    gy[0] += yv * el.gl[k][0];
    gy[1] += yv * el.gl[k][1];
    ph[k] = phi[el.v1[k]];
    psum += ph[k];
  }
  const double s = el.area * gamma * (gx[0] * gy[0] + gx[1] * gy[1]);
#pragma unroll
  for (int c = 0; c < 3; ++c) buf[(long)e * 3 + c] = s * (1.0 / 3.0 - (psum + ph[c]) / 6.0);
}

// d/dw of y^T J(w) x (velocities): nodal part int zeta_k sum_c (d_d x_c) y_c
// -> bufv [E][6][2]; shift part (w = v - s, s per element) projected on the
// P1 gradients: (ds-gradient) . grad psi_m -> bufm [E][3]
__global__ void k_adj_conv_p2(Geo g, const double *__restrict__ x, const double *__restrict__ y, double *bufv,
                              double *bufm) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.n * g.n) return;
  Elem el;
  element(g, e, el);
  double xy[6][6];   // sum_c x_(b,c) y_(a,c)
#pragma unroll
  for (int b = 0; b < 6; ++b) {
    const double x0 = x[2 * el.v2[b]], x1 = x[2 * el.v2[b] + 1];
#pragma unroll
    for (int a = 0; a < 6; ++a) xy[b][a] = x0 * y[2 * el.v2[a]] + x1 * y[2 * el.v2[a] + 1];
  }
  double tg[3];
  for (int l = 0; l < 3; ++l) {
    double s = 0.0;
    for (int b = 0; b < 6; ++b)
#pragma unroll
      for (int a = 0; a < 6; ++a) s += xy[b][a] * c_ref.jg[l][b][a];
    tg[l] = s;
  }
  for (int k = 0; k < 6; ++k) {
    double t[3];
    for (int l = 0; l < 3; ++l) {
      double s = 0.0;
      for (int b = 0; b < 6; ++b)
#pragma unroll
        for (int a = 0; a < 6; ++a) s += xy[b][a] * c_ref.j[k][l][b][a];
      t[l] = s;
    }
#pragma unroll
    for (int d = 0; d < 2; ++d)
      bufv[(long)e * 12 + k * 2 + d] = el.area * (el.gl[0][d] * t[0] + el.gl[1][d] * t[1] + el.gl[2][d] * t[2]);
  }
  double sb[2];
#pragma unroll
  for (int d = 0; d < 2; ++d) sb[d] = -el.area * (el.gl[0][d] * tg[0] + el.gl[1][d] * tg[1] + el.gl[2][d] * tg[2]);
#pragma unroll
  for (int m = 0; m < 3; ++m) bufm[(long)e * 3 + m] = sb[0] * el.gl[m][0] + sb[1] * el.gl[m][1];
}

struct LoadWeights {
  const double *z[5];   // adjoint weights of the loads of df/dphi_p, _N, _s, _a, df/dPhi (may be null)
};

// gradient of sum_i z_i^T F_i with respect to (phi_p, phi_N, phi_s, Phi):
// int (sum_i d g_i / d var) z_i psi_m, Hessian of eqn:appPotential at the
// 20-point rule -> buf [4][E][3]
__global__ void k_adj_loads(Geo g, const double *__restrict__ pp, const double *__restrict__ pn,
                            const double *__restrict__ ps, const double *__restrict__ Ph, LoadWeights lw,
                            double *buf) {
  const int E = 2 * g.n * g.n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  Elem el;
  element(g, e, el);
  double fp[3], fn[3], fs[3], fv[3], zz[5][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    fp[k] = pp[el.v1[k]]; fn[k] = pn[el.v1[k]]; fs[k] = ps[el.v1[k]]; fv[k] = Ph[el.v1[k]];
  }
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 3; ++k) zz[i][k] = lw.z[i] ? lw.z[i][el.v1[k]] : 0.0;
  double acc[4][3];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[f][a] = 0.0;
  for (int q = 0; q < 20; ++q) {
    const double l0 = c_ref.qlam[q][0], l1 = c_ref.qlam[q][1], l2 = c_ref.qlam[q][2], w = c_ref.qw[q];
    const double p = l0 * fp[0] + l1 * fp[1] + l2 * fp[2];
    const double nn = l0 * fn[0] + l1 * fn[1] + l2 * fn[2];
    const double s = l0 * fs[0] + l1 * fs[1] + l2 * fs[2];
    const double V = l0 * fv[0] + l1 * fv[1] + l2 * fv[2];
    const double a = 1.0 - p - nn - s;
    double z[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) z[i] = l0 * zz[i][0] + l1 * zz[i][1] + l2 * zz[i][2];
    const double q_ = V * V * (3.0 - 2.0 * V), dq = 6.0 * V * (1.0 - V), ddq = 6.0 - 12.0 * V;
    const double liq = 3.5 * p * p * nn * nn + 0.3 * s * s + 0.3 * a * a - 10.0 * s * a;
    const double gas = 3.5 * p * p + 3.5 * nn * nn + 2.0 * s * s + 0.1 * a * a;
    // Hessian in (p, N, s, a, Phi)
    const double Hpp = (1 - q_) * 7.0 * nn * nn + 7.0 * q_, HpN = (1 - q_) * 14.0 * p * nn;
    const double HNN = (1 - q_) * 7.0 * p * p + 7.0 * q_;
    const double Hss = (1 - q_) * 0.6 + 4.0 * q_, Hsa = -(1 - q_) * 10.0, Haa = (1 - q_) * 0.6 + 0.2 * q_;
    const double HpV = dq * 7.0 * p * (1 - nn * nn), HNV = dq * 7.0 * nn * (1 - p * p);
    const double HsV = dq * (3.4 * s + 10.0 * a), HaV = dq * (10.0 * s - 0.4 * a), HVV = ddq * (gas - liq);
    // sum_i z_i dg_i/dphi_j with dg_i/dphi_j = H_ij - H_ia (phi_a = 1 - sum phi)
    const double gp = z[0] * Hpp + z[1] * HpN + z[4] * HpV;                 // H_ia = 0 for i = p, N
    const double gn = z[0] * HpN + z[1] * HNN + z[4] * HNV;
    const double gs = z[2] * (Hss - Hsa) + z[3] * (Hsa - Haa) + z[4] * (HsV - HaV);
    const double ga_s = -(z[2] * Hsa + z[3] * Haa + z[4] * HaV);            // the -H_ia part for j = p, N
    const double gV = z[0] * HpV + z[1] * HNV + z[2] * HsV + z[3] * HaV + z[4] * HVV;
    const double gj[4] = {gp + ga_s, gn + ga_s, gs, gV};
    const double lam[3] = {l0, l1, l2};
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) acc[f][aa] += w * gj[f] * lam[aa];
  }
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) buf[(long)f * E * 3 + (long)e * 3 + aa] = el.area * acc[f][aa];
}

// gradient of y^T G (Korteweg load) with respect to (phi_p, phi_N, phi_s,
// Phi): grad psi_m . (Y + Y^T)(beta_j g_j - beta_a g_a), Y = int grad y
// -> buf [4][E][3]
__global__ void k_adj_korteweg(Geo g, const double *__restrict__ pp, const double *__restrict__ pn,
                               const double *__restrict__ ps, const double *__restrict__ Ph,
                               const double *__restrict__ y, KortewegCoef kc, double *buf) {
  const int E = 2 * g.n * g.n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  Elem el;
  element(g, e, el);
  double Y[2][2] = {{0, 0}, {0, 0}};   // Y[c][b] = int d_b y_c
  for (int a = 0; a < 6; ++a) {
    double ga[2];
#pragma unroll
    for (int b = 0; b < 2; ++b)
      ga[b] = el.gl[0][b] * c_ref.g[a][0] + el.gl[1][b] * c_ref.g[a][1] + el.gl[2][b] * c_ref.g[a][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double yc = y[2 * el.v2[a] + c];
      Y[c][0] += el.area * yc * ga[0];
      Y[c][1] += el.area * yc * ga[1];
    }
  }
  const double S[2][2] = {{2 * Y[0][0], Y[0][1] + Y[1][0]}, {Y[0][1] + Y[1][0], 2 * Y[1][1]}};
  double gr[5][2];
  const double *fld[4] = {pp, pn, ps, Ph};
  for (int f = 0; f < 4; ++f) {
    const int dst = f < 3 ? f : 4;
    gr[dst][0] = gr[dst][1] = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double xv = fld[f][el.v1[k]];
      gr[dst][0] += xv * el.gl[k][0];
      gr[dst][1] += xv * el.gl[k][1];
    }
  }
  gr[3][0] = -(gr[0][0] + gr[1][0] + gr[2][0]);
  gr[3][1] = -(gr[0][1] + gr[1][1] + gr[2][1]);
  for (int f = 0; f < 4; ++f) {
    double u[2];
    if (f < 3) {
      u[0] = kc.beta[f] * gr[f][0] - kc.beta[3] * gr[3][0];
      u[1] = kc.beta[f] * gr[f][1] - kc.beta[3] * gr[3][1];
    } else {
      u[0] = kc.beta_v * gr[4][0];
      u[1] = kc.beta_v * gr[4][1];
    }
    const double su0 = S[0][0] * u[0] + S[0][1] * u[1], su1 = S[1][0] * u[0] + S[1][1] * u[1];
#pragma unroll
    for (int m = 0; m < 3; ++m) buf[(long)f * E * 3 + (long)e * 3 + m] = el.gl[m][0] * su0 + el.gl[m][1] * su1;
  }
}

}  // namespace

void launch_adj_conv_p1(Geo g, const double *x, const double *y, double *buf, cudaStream_t s) {
  k_adj_conv_p1<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, x, y, buf);
  CHNSS_LAUNCH_CK();
}
void launch_adj_wstiff(Geo g, const double *phi, double gamma, const double *x, const double *y, double *buf,
                       cudaStream_t s) {
  k_adj_wstiff<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, phi, gamma, x, y, buf);
  CHNSS_LAUNCH_CK();
}
void launch_adj_conv_p2(Geo g, const double *x, const double *y, double *bufv, double *bufm, cudaStream_t s) {
  k_adj_conv_p2<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, x, y, bufv, bufm);
  CHNSS_LAUNCH_CK();
}
void launch_adj_loads(Geo g, const double *pp, const double *pn, const double *ps, const double *Ph,
                      const double *const *z, double *buf, cudaStream_t s) {
  LoadWeights lw;
  for (int i = 0; i < 5; ++i) lw.z[i] = z[i];
  k_adj_loads<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, pp, pn, ps, Ph, lw, buf);
  CHNSS_LAUNCH_CK();
}
void launch_adj_korteweg(Geo g, const double *pp, const double *pn, const double *ps, const double *Ph,
                         const double *y, KortewegCoef c, double *buf, cudaStream_t s) {
  k_adj_korteweg<<<blocks_for(2L * g.n * g.n), TPB, 0, s>>>(g, pp, pn, ps, Ph, y, c, buf);
  CHNSS_LAUNCH_CK();
}

}  // namespace chnss
