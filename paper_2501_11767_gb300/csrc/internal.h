// Internal declarations of the chnss CUDA library (not part of the ABI).
//
// Layout in HBM (all int32 indices, FP64 values unless stated):
//   * CSR patterns per multigrid level: the P1 node pattern (7-point stencil
//     of the structured triangulation) and the P2 node pattern, which is also
//     the block pattern of the 2x2-block (BSR2) velocity operator.
//   * Gather lists: for every output entry (a CSR value, a BSR2 block or a
//     node of a load vector) the ordered list of offsets into an element
//     buffer whose contributions it sums.  Assembly = element kernel writing
//     dense element matrices + gather kernel; no atomics, so the sum order
//     is fixed and results are bit-reproducible.
//   * Vectors: P1 fields [N1]; velocity [2*N2] interleaved (x, y) per node;
//     system vectors are concatenations ([phi; mu], [v; p]).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/chnss.h"

namespace chnss {

struct Error {
  chnss_status status;
  std::string msg;
};

#define CHNSS_CK(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::chnss::Error{CHNSS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// kernels launched by the library in this process (gpu_launches of the bench)
extern std::atomic<long long> g_launch_count;

// the last error of calls without a context (chnss_last_error(NULL))
void set_global_error(const std::string &msg);

#define CHNSS_LAUNCH_CK()                                                \
  do {                                                                   \
    ::chnss::g_launch_count.fetch_add(1, std::memory_order_relaxed);     \
    CHNSS_CK(cudaGetLastError());                                        \
  } while (0)

// Owner of device allocations; frees everything it handed out.
struct Arena {
  std::vector<void *> ptrs;
  size_t bytes = 0;
  template <class T>
  T *alloc(size_t n) {
    if (n == 0) n = 1;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{CHNSS_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed: " +
                                     cudaGetErrorString(e)};
    }
    ptrs.push_back(p);
    bytes += n * sizeof(T);
    return static_cast<T *>(p);
  }
  template <class T>
  T *upload(const std::vector<T> &h) {
    T *d = alloc<T>(h.size());
    if (!h.empty()) CHNSS_CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
  }
  void release() {
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
  ~Arena() { release(); }
};

// SELL-C-sigma view of a CSR pattern (C = 32): rows are sorted by length
// (descending) inside windows of sigma rows and cut into slices of 32; a
// slice stores its entries column-major (entry j of the 32 rows is
// contiguous), padded to the slice's longest row.  One thread per row, every
// value / column load is one coalesced warp access.
constexpr int kSellMaxBlock = 512;   // largest threads-per-block of the SELL kernels
struct Sell {
  static constexpr int C = 32;
  static constexpr int SIGMA = 256;
  int block = 256;               // threads per block of its SpMV launches (autotuned)
  int nslices = 0;
  int wmax = 0;                  // widest slice (entries per row incl. padding)
  long nent = 0;                 // padded entries
  int *slice_ptr = nullptr;      // [nslices + 1] first entry of each slice
  int *rowid = nullptr;          // [nslices * 32] CSR row of each slot, -1 = padding
  int *col = nullptr;            // [nent] column (padding: a valid column, value 0)
  int *map = nullptr;            // [nent] CSR position, -1 = padding
  int *mapT = nullptr;           // [nent] CSR position of the transposed entry (square symmetric patterns)
  // Stencil layout (P1 patterns of the structured meshes): rows in natural
  // order, every slice 7 wide, slot j of row i holds column i + soff[j]
  // (ascending, so the CSR order) or a zero where that neighbour is not
  // coupled; kernels that know the layout compute the columns instead of
  // loading col / rowid.  The explicit arrays above stay valid for every
  // other SELL kernel.
  int stencil = 0;
  int soff[7] = {0, 0, 0, 0, 0, 0, 0};
};

struct Pattern {
  int nrows = 0, ncols = 0;
  int nnz = 0;
  int *rowptr = nullptr, *col = nullptr;  // device
  std::vector<int> h_rowptr, h_col;       // host copies
  Sell sell;
};

// Host setup helpers (setup.cu): SELL view of an uploaded pattern (hmap:
// host map SELL entry -> CSR position), pattern upload with its SELL view,
// gather-list upload, transpose of a host CSR, transfer operator finishing
// (R = P^T, SELL and FP32 copies), CSR positions of the diagonal.
struct Pattern;
struct Gather;
struct Transfer;
void build_sell(Arena &ar, Pattern &P, std::vector<int> *hmap = nullptr);
void upload_pattern(Arena &ar, Pattern &P, std::vector<int> *hmap = nullptr);
void upload_gather(Arena &ar, Gather &G, const std::vector<int> &ptr, const std::vector<int> &idx);
void transpose(const Pattern &A, const std::vector<double> &av, Pattern &T, std::vector<double> &tv);
void finish_transfer(Arena &ar, Transfer &t, const std::vector<double> &pv);
std::vector<int> diag_positions(const Pattern &P);

// out entry k sums buf[idx[j] + c] for j in [ptr[k], ptr[k+1]), c < ncomp.
struct Gather {
  int nout = 0;
  int ncontrib = 0;
  int *ptr = nullptr, *idx = nullptr;
};

struct Transfer {               // prolongation P (fine x coarse) and R = P^T
  Pattern P, R;
  double *Pv = nullptr, *Rv = nullptr;          // CSR order
  double *Ps = nullptr, *Rs = nullptr;          // SELL order
  float *Ps32 = nullptr, *Rs32 = nullptr;       // SELL order, FP32
};

struct Level {
  int n = 0;
  double hx = 0, hy = 0;
  int N1 = 0, N2 = 0, E = 0;
  Pattern p1, p2;
  Gather g_p1;    // P1 values <- element [E][3][3]
  Gather g_p2v;   // P2 velocity blocks <- element [E][6][6] (Dirichlet nodes masked)
  Gather g_ks;    // P2 velocity blocks <- element [E][6][2][6][2] (4 comps), masked
  int *bnd2 = nullptr;   // [N2] 1 on the boundary
  int *diag1 = nullptr;  // [N1] position of the diagonal in p1
  int *diag2 = nullptr;  // [N2] position of the diagonal block in p2
  Transfer t1;           // P1 transfer from level+1 (empty on the coarsest)
  Transfer tv;           // velocity (per node, masked) transfer from level+1
};

struct Mesh {
  double lx = 1, ly = 1;
  int n = 0;
  int top_bc = 0;              // 0: no-slip on the whole boundary; 1: open (do-nothing) top
  std::vector<Level> lv;
  Pattern pb, pbt;             // fine B (P1 rows x P2 node cols) and B^T
  Gather g_b, g_bt;            // <- element [E][3][6][2] (2 comps)
  Gather g_l1;                 // P1 nodes <- element [E][3]
  Gather g_l2;                 // P2 nodes <- element [E][6][2] (2 comps), masked
  int ref_node = 0;            // P1 node (n/2, n): reference point of phi_s^vap
  Arena arena;
};

// ---------------------------------------------------------------------------
// reference tensors (exact integrals over a triangle divided by its area)
struct RefTensors {
  double m1[3][3];            // lambda_a lambda_b
  double c1[6][3];            // phi2_k lambda_a
  double m2[6][6];            // phi2_a phi2_b
  double j[6][3][6][6];       // phi2_k d_l phi2_b phi2_a  (k, l, b, a)
  double jg[3][6][6];         // d_l phi2_b phi2_a         (l, b, a)
  double s[3][6][3][6];       // d_l phi2_b d_m phi2_a     (l, b, m, a)
  double b[3][6][3];          // lambda_a d_l phi2_b       (a, b, l)
  double g[6][3];             // d_l phi2_a                (a, l)
  double qlam[20][3];         // degree-7 rule: barycentric points
  double qw[20];              // weights, sum 1
};
const RefTensors &reference_tensors();

// ---------------------------------------------------------------------------
// host builders (setup.cu)
void build_mesh(Mesh &m, int n, double lx, double ly, int top_bc);
void destroy_mesh(Mesh &m);

// ---------------------------------------------------------------------------
// kernels launched from the host (assemble.cu, sparse.cu)
struct Geo {     // structured level geometry
  int n;
  double hx, hy;
};

void upload_reference_tensors(cudaStream_t s);
void launch_elem_p1_mass(Geo g, double *buf, cudaStream_t s);
void launch_elem_p1_stiff(Geo g, double *buf, cudaStream_t s);
// C or J_p: ((v - shift) . grad psi_b) psi_a, shift = sum alpha_i grad mu_i (mu may be null)
void launch_elem_p1_conv(Geo g, const double *v, const double *const *mu, const double *alpha,
                         double *buf, cudaStream_t s);
// weighted stiffness with kappa = gamma (phi (1 - phi) + m0)
void launch_elem_p1_wstiff(Geo g, const double *phi, double gamma, double m0, double *buf, cudaStream_t s);
void launch_elem_p2_mass(Geo g, double *buf, cudaStream_t s);
void launch_elem_p2_conv(Geo g, const double *v, const double *const *mu, const double *alpha,
                         double *buf, cudaStream_t s);
void launch_elem_ksym(Geo g, double eta, double *buf, cudaStream_t s);
void launch_elem_bdiv(Geo g, double *buf, cudaStream_t s);
// constants of the potential: model 0 eqn:appPotential; model 1 the
// solvent-air Flory-Huggins density with Taylor-expanded phi ln phi
struct PotentialCoef {
  int model = 0;
  double inv_ns = 1.0, inv_na = 1.0, chi_sa = 0.0;
  double ln_sat_s = 0.0, ln_sat_a = 0.0;
};
void launch_elem_loads(Geo g, const double *phi_p, const double *phi_n, const double *phi_s,
                       const double *Phi, PotentialCoef pc, double *buf, cudaStream_t s);
// Conservation and energy sums of a state (chnss_diagnostics): quantities
// int phi_p, int phi_NFA, int phi_s, int phi_a, int p, int f, gradient
// energy, kinetic energy; partial[q * nb + b] for the nb blocks returned.
constexpr int kDiagQuantities = 8;
struct DiagArgs {
  const double *pp, *pn, *ps, *Ph, *p, *v;
  double beta[4], beta_v;
  PotentialCoef pc;
};
int launch_diagnostics(Geo g, const DiagArgs &d, double *partial, cudaStream_t s);
struct KortewegCoef {
  double beta[4];
  double beta_v;
};
void launch_elem_korteweg(Geo g, const double *phi_p, const double *phi_n, const double *phi_s,
                          const double *Phi, KortewegCoef c, double *buf, cudaStream_t s);

// out[k*nc + c] = beta * base[k*nc + c] + alpha * sum buf[idx + c]   (base may be null)
void launch_gather(const Gather &g, int ncomp, const double *buf, double alpha, const double *base,
                   double beta, double *out, cudaStream_t s);
// velocity blocks: out[4k..4k+3] = base[4k..] + alpha * sum(buf) * I2
void launch_gather_diag2(const Gather &g, const double *buf, double alpha, const double *base, double *out,
                         cudaStream_t s);

// adjoint (transposed Jacobian) element kernels
void launch_adj_conv_p1(Geo g, const double *x, const double *y, double *buf, cudaStream_t s);   // [E][6][2]
// d/dphi of y^T K_kappa(phi) x for kappa = gamma (phi (1 - phi) + m0)  [E][3]
void launch_adj_wstiff(Geo g, const double *phi, double gamma, const double *x, const double *y, double *buf,
                       cudaStream_t s);
void launch_adj_conv_p2(Geo g, const double *x, const double *y, double *bufv, double *bufm,
                        cudaStream_t s);                                                        // [E][6][2], [E][3]
void launch_adj_loads(Geo g, const double *pp, const double *pn, const double *ps, const double *Ph,
                      const double *const *z, double *buf, cudaStream_t s);                   // [4][E][3]
void launch_adj_korteweg(Geo g, const double *pp, const double *pn, const double *ps, const double *Ph,
                         const double *y, KortewegCoef c, double *buf, cudaStream_t s);       // [4][E][3]

void launch_inject_p1(int nf, const double *fine, double *coarse, cudaStream_t s);
void launch_inject_vel(int nf, const double *fine, double *coarse, cudaStream_t s);

}  // namespace chnss
