// Tetrahedral (3D) element operators of the model (paper Sec. 3-5; the
// paper's 3D runs use uniform tetrahedral meshes of a cube).
//
// Mesh: the box in n^3 cubes, each split into the six Kuhn (Freudenthal)
// tetrahedra along its main diagonal: cube (i, j, k), axis order
// sigma = kPerm3[p], vertices v0 = (i, j, k), v1 = v0 + e_sigma0,
// v2 = v1 + e_sigma1, v3 = (i+1, j+1, k+1), element id 6 ((k n + j) n + i) + p.
// P1 node (a, b, c) has id (c (n+1) + b)(n+1) + a; P2 nodes are the doubled
// lattice, node (A, B, C) id (C m + B) m + A with m = 2n + 1; local P2
// numbering: the four vertices, then the midpoints of the edges kEdge3.
//
// Every element operator below is a __host__ __device__ function of one
// element's geometry and nodal values, with exact reference integrals of
// barycentric polynomials (Tet3Ref): the same code serves the host setup of
// the constant operators and the per-step device kernels.
#pragma once

namespace chnss {

constexpr int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
constexpr int kEdge3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
constexpr int kLoadPts3 = 100;   // collapsed Gauss rule exact to degree 7 (5 x 5 x 4 points)

// Reference integrals over a tetrahedron, divided by its volume (N: the ten
// P2 basis functions, lambda: barycentrics, dN/dl: derivative of N with
// respect to barycentric l, so grad N = sum_l dN/dl grad lambda_l).
struct Tet3Ref {
  double r[10][4];           // int N_k lambda_a                   (P1 convection by a P2 velocity)
  double t[10][4][10][10];   // int N_k dN_b/dl N_a  [k][l][b][a]  (P2 convection by a P2 velocity)
  double s[4][10][10];       // int dN_b/dl N_a      [l][b][a]     (P2 convection by a constant)
  double d[10][4];           // int dN_a/dl                        (Korteweg load)
  double q[10][4][10][4];    // int dN_a/dl dN_b/dm  [a][l][b][m]  (symmetric-gradient form)
  double w[4][10][4];        // int lambda_q dN_b/dl [q][b][l]     (divergence)
  double m2[10][10];         // int N_a N_b                        (P2 mass)
  double ql[kLoadPts3][4];   // barycentric points of the degree-7 rule
  double qw[kLoadPts3];      // its weights (sum 1)
};

// Volume and barycentric gradients g[a][d] of the tetrahedron with
// vertices x[a][d]; returns the volume.
__host__ __device__ inline double tet_geometry(const double x[4][3], double g[4][3]) {
  double J[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = x[c + 1][r] - x[0][r];   // columns x_c - x_0
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const double inv = 1.0 / det;
  // rows of J^-1 are the gradients of lambda_1..3
  g[1][0] = c00 * inv;
  g[1][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * inv;
  g[1][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * inv;
  g[2][0] = c01 * inv;
  g[2][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * inv;
  g[2][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * inv;
  g[3][0] = c02 * inv;
  g[3][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * inv;
  g[3][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * inv;
  for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  return (det < 0 ? -det : det) / 6.0;
}

// C_ab = int ((v - s) . grad psi_b) psi_a, v the P2 velocity vk[10][3] of
// the element, s a constant (null: none): out[a * 4 + b]
__host__ __device__ inline void tet_p1_conv(const Tet3Ref &R, double vol, const double g[4][3],
                                            const double vk[10][3], const double *s, double out[16]) {
  for (int b = 0; b < 4; ++b) {
    double vg[10];
    for (int k = 0; k < 10; ++k) vg[k] = vk[k][0] * g[b][0] + vk[k][1] * g[b][1] + vk[k][2] * g[b][2];
    const double sg = s ? s[0] * g[b][0] + s[1] * g[b][1] + s[2] * g[b][2] : 0.0;
    for (int a = 0; a < 4; ++a) {
      double acc = -0.25 * sg;
      for (int k = 0; k < 10; ++k) acc += vg[k] * R.r[k][a];
      out[a * 4 + b] = vol * acc;
    }
  }
}

// Weighted stiffness K_kappa,ab = int kappa grad psi_a . grad psi_b with the
// concentration-dependent mobility kappa = gamma (phi (1 - phi) + m0) of a P1
// field phi (nodal values f[4]).  The gradients are constant on the element,
// so only int kappa is needed, and it is exact: int phi = vol sum f / 4,
// int phi^2 = vol ((sum f)^2 + sum f^2) / 20.  out[a * 4 + b]
__host__ __device__ inline void tet_wstiff(double vol, const double g[4][3], const double f[4], double gamma,
                                           double m0, double out[16]) {
  const double s1 = f[0] + f[1] + f[2] + f[3];
  const double s2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];
  const double kint = vol * gamma * (0.25 * s1 - (s1 * s1 + s2) / 20.0 + m0);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) out[a * 4 + b] = kint * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
}

// J_ab = int ((v - s) . grad N_b) N_a on the P2 nodes: out[a * 10 + b]
__host__ __device__ inline void tet_p2_conv(const Tet3Ref &R, double vol, const double g[4][3],
                                            const double vk[10][3], const double *s, double out[100]) {
  double vg[10][4], sg[4];
  for (int l = 0; l < 4; ++l) {
    for (int k = 0; k < 10; ++k) vg[k][l] = vk[k][0] * g[l][0] + vk[k][1] * g[l][1] + vk[k][2] * g[l][2];
    sg[l] = s ? s[0] * g[l][0] + s[1] * g[l][1] + s[2] * g[l][2] : 0.0;
  }
  for (int a = 0; a < 10; ++a)
    for (int b = 0; b < 10; ++b) {
      double acc = 0.0;
      for (int l = 0; l < 4; ++l) {
        acc -= sg[l] * R.s[l][b][a];
        for (int k = 0; k < 10; ++k) acc += vg[k][l] * R.t[k][l][b][a];
      }
      out[a * 10 + b] = vol * acc;
    }
}

// eta int 2 sym(N_b e_d) : sym(N_a e_c) on the 30 velocity dofs (a, c):
// out[(a * 3 + c) * 30 + b * 3 + d]
__host__ __device__ inline void tet_ksym(const Tet3Ref &R, double vol, const double g[4][3], double eta,
                                         double *out) {
  double gg[4][4];
  for (int l = 0; l < 4; ++l)
    for (int m = 0; m < 4; ++m) gg[l][m] = g[l][0] * g[m][0] + g[l][1] * g[m][1] + g[l][2] * g[m][2];
  for (int a = 0; a < 10; ++a)
    for (int b = 0; b < 10; ++b) {
      double lap = 0.0, cross[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int l = 0; l < 4; ++l)
        for (int m = 0; m < 4; ++m) {
          const double qv = R.q[a][l][b][m];
          lap += gg[l][m] * qv;
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) cross[c][d] += g[m][c] * g[l][d] * qv;   // d_c N_b d_d N_a
        }
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d)
          out[(a * 3 + c) * 30 + b * 3 + d] = eta * vol * (cross[c][d] + (c == d ? lap : 0.0));
    }
}

// b_(q,(b,d)) = - int psi_q d_d N_b: out[q * 30 + b * 3 + d]
__host__ __device__ inline void tet_div(const Tet3Ref &R, double vol, const double g[4][3], double out[120]) {
  for (int q = 0; q < 4; ++q)
    for (int b = 0; b < 10; ++b)
      for (int d = 0; d < 3; ++d) {
        double acc = 0.0;
        for (int l = 0; l < 4; ++l) acc += g[l][d] * R.w[q][b][l];
        out[q * 30 + b * 3 + d] = -vol * acc;
      }
}

// Partial derivatives of the polynomial free energy eqn:appPotential with
// respect to phi_p, phi_N, phi_s, phi_a and Phi (un-reduced, evaluated at
// phi_a = 1 - sum phi): f = (1 - p(Phi)) f_liq + p(Phi) f_gas with
// p(Phi) = Phi^2 (3 - 2 Phi).
__host__ __device__ inline void potential_partials3(double p, double nn, double s, double V, double out[5]) {
  const double a = 1.0 - p - nn - s;
  const double ip = V * V * (3.0 - 2.0 * V), dip = 6.0 * V * (1.0 - V);
  const double liq = 3.5 * p * p * nn * nn + 0.3 * s * s + 0.3 * a * a - 10.0 * s * a;
  const double gas = 3.5 * p * p + 3.5 * nn * nn + 2.0 * s * s + 0.1 * a * a;
  out[0] = (1.0 - ip) * 7.0 * p * nn * nn + ip * 7.0 * p;
  out[1] = (1.0 - ip) * 7.0 * p * p * nn + ip * 7.0 * nn;
  out[2] = (1.0 - ip) * (0.6 * s - 10.0 * a) + ip * 4.0 * s;
  out[3] = (1.0 - ip) * (0.6 * a - 10.0 * s) + ip * 0.2 * a;
  out[4] = dip * (gas - liq);
}

// Second derivatives of the same free energy in (phi_p, phi_N, phi_s, phi_a,
// Phi), un-reduced, at phi_a = 1 - sum phi: H[i][j] (symmetric)
__host__ __device__ inline void potential_hessian3(double p, double nn, double s, double V, double H[5][5]) {
  const double a = 1.0 - p - nn - s;
  const double ip = V * V * (3.0 - 2.0 * V), dip = 6.0 * V * (1.0 - V), ddip = 6.0 - 12.0 * V;
  const double liq = 3.5 * p * p * nn * nn + 0.3 * s * s + 0.3 * a * a - 10.0 * s * a;
  const double gas = 3.5 * p * p + 3.5 * nn * nn + 2.0 * s * s + 0.1 * a * a;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) H[i][j] = 0.0;
  H[0][0] = (1.0 - ip) * 7.0 * nn * nn + 7.0 * ip;
  H[0][1] = H[1][0] = (1.0 - ip) * 14.0 * p * nn;
  H[1][1] = (1.0 - ip) * 7.0 * p * p + 7.0 * ip;
  H[2][2] = (1.0 - ip) * 0.6 + 4.0 * ip;
  H[2][3] = H[3][2] = -(1.0 - ip) * 10.0;
  H[3][3] = (1.0 - ip) * 0.6 + 0.2 * ip;
  // d/dPhi of the first partials: dip (gas_i - liq_i)
  H[0][4] = H[4][0] = dip * 7.0 * p * (1.0 - nn * nn);
  H[1][4] = H[4][1] = dip * 7.0 * nn * (1.0 - p * p);
  H[2][4] = H[4][2] = dip * (3.4 * s + 10.0 * a);
  H[3][4] = H[4][3] = dip * (10.0 * s - 0.4 * a);
  H[4][4] = ddip * (gas - liq);
}

// Potential loads int df/dfield psi_a of one element: fields[f][k] = nodal
// values of phi_p, phi_N, phi_s, Phi; out[f * 4 + a] for the five partials
__host__ __device__ inline void tet_loads(const Tet3Ref &R, double vol, const double fields[4][4], double out[20]) {
  for (int i = 0; i < 20; ++i) out[i] = 0.0;
  for (int q = 0; q < kLoadPts3; ++q) {
    double v[4];
    for (int f = 0; f < 4; ++f)
      v[f] = R.ql[q][0] * fields[f][0] + R.ql[q][1] * fields[f][1] + R.ql[q][2] * fields[f][2] +
             R.ql[q][3] * fields[f][3];
    double d[5];
    potential_partials3(v[0], v[1], v[2], v[3], d);
    for (int f = 0; f < 5; ++f) {
      const double wd = R.qw[q] * d[f];
      for (int a = 0; a < 4; ++a) out[f * 4 + a] += wd * R.ql[q][a];
    }
  }
  for (int i = 0; i < 20; ++i) out[i] *= vol;
}

// Korteweg load int sum_b G_cb d_b N_a for a constant tensor G: out[a * 3 + c]
__host__ __device__ inline void tet_korteweg(const Tet3Ref &R, double vol, const double g[4][3],
                                             const double G[3][3], double out[30]) {
  for (int a = 0; a < 10; ++a) {
    double da[3] = {0.0, 0.0, 0.0};   // int grad N_a / vol
    for (int l = 0; l < 4; ++l)
      for (int b = 0; b < 3; ++b) da[b] += R.d[a][l] * g[l][b];
    for (int c = 0; c < 3; ++c) out[a * 3 + c] = vol * (G[c][0] * da[0] + G[c][1] * da[1] + G[c][2] * da[2]);
  }
}

}  // namespace chnss
