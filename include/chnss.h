/*
 * chnss.h -- C ABI of the GB300 library for one semi-implicit step of the
 * Cahn-Hilliard / Allen-Cahn / Navier-Stokes thin-film model of
 * arXiv 2501.11767 (Ciloglu, Tretmans, Herzog, Pietschmann, Stoll).
 *
 * Discretisation (paper Sec. 3): uniform triangulation of [0,lx] x [0,ly]
 * with n x n squares, each split along its lower-left -> upper-right
 * diagonal; P1 elements for the volume fractions phi_i, the chemical
 * potentials mu_i, the vapour order parameter Phi_v and the pressure p;
 * Taylor-Hood P2 elements for the velocity v, which is zero on the whole
 * boundary (eqn:bc).  Semi-implicit Euler in time: every coefficient of the
 * linear systems is taken at t_k.
 *
 * Numbering shared by every array that crosses this ABI:
 *   P1 node (i, j), 0 <= i, j <= n, has index j*(n+1) + i   (N1 = (n+1)^2)
 *   P2 node (I, J) of the once-refined lattice, 0 <= I, J <= 2n, has index
 *   J*(2n+1) + I (N2 = (2n+1)^2); the vertex (i, j) is lattice point (2i, 2j).
 *   Velocity arrays hold 2*N2 doubles, interleaved (x, y) per P2 node.
 *
 * Memory and streams: every double* in chnss_state and every x/rhs pointer is
 * a DEVICE pointer owned by the caller (contiguous FP64), unless the function
 * says "host".  The library owns its workspace (matrices, multigrid
 * hierarchies, Krylov bases), allocated in chnss_ctx_create and released in
 * chnss_ctx_destroy.  All work is queued on the context's CUDA stream; the
 * Krylov drivers read one convergence scalar per iteration back to the host
 * and therefore synchronise that stream.  No call aborts and no C++
 * exception crosses the ABI: failures return a status and leave a message
 * for chnss_last_error.
 */
#ifndef CHNSS_H
#define CHNSS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CHNSS_OK = 0,
  CHNSS_ERR_ARG = 1,         /* invalid argument (size, null pointer, unsupported flag) */
  CHNSS_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  CHNSS_ERR_OOM = 3,         /* device allocation failed */
  CHNSS_ERR_NOCONV = 4,      /* a Krylov solve hit maxit; x holds the last iterate */
  CHNSS_ERR_BREAKDOWN = 5,   /* Arnoldi breakdown without convergence */
  CHNSS_ERR_NAN = 6,         /* NaN or Inf in a residual norm */
  CHNSS_ERR_TIMEOUT = 7,     /* reserved: a bounded device-side wait gave up */
  CHNSS_ERR_STATE = 8        /* call out of order (e.g. solve before assemble) */
} chnss_status;

typedef struct chnss_mesh *chnss_mesh_t;   /* opaque: level hierarchy, patterns, maps */
typedef struct chnss_ctx *chnss_ctx_t;     /* opaque: parameters, operators, workspace */

/* Linear systems of one step (Sec. 4). */
typedef enum {
  CHNSS_SYS_CH_P = 0,   /* eqn:CH_linear for the polymer: unknowns [phi (N1); mu (N1)] */
  CHNSS_SYS_CH_N = 1,   /* eqn:CH_linear for the NFA */
  CHNSS_SYS_CH_S = 2,   /* eqn:CH_linear for the solvent */
  CHNSS_SYS_AC = 3,     /* Allen-Cahn (M + tau delta_v K + tau C) Phi = rhs: unknowns Phi (N1) */
  CHNSS_SYS_MU_A = 4,   /* air potential M mu_a = f_a + beta_a K phi_a^{k+1} (Sec. 5): mu_a (N1) */
  CHNSS_SYS_NS = 5      /* eqn:linearnav: unknowns [v (2*N2); p (N1)] */
} chnss_system;

/* Model and solver parameters (nondimensional form eqn:model, Sec. 5). */
typedef struct {
  double tau;            /* time step */
  double beta[4];        /* gradient-energy coefficients beta_i, i = p, NFA, s, a */
  double gamma[3];       /* mobilities gamma_i (p, NFA, s); scale of the variable law */
  int mobility_kind;     /* 0: constant gamma_i; 1: gamma_i (phi_i (1 - phi_i) + m0) at t_k */
  double mobility_m0;    /* m0 of the variable mobility law */
  double eta;            /* viscosity */
  double alpha[4];       /* alpha_i of the convective velocity rho v - sum alpha_i grad mu_i */
  double beta_v, gamma_v, delta_v;  /* vapour gradient energy, rate and diffusion (eqn:model) */
  double evap_rate;      /* lumped Hertz-Knudsen factor: j_out = evap_rate (phi_s^vap - phi_s_inf) */
  double phi_s_inf;      /* solvent fraction of the ambient air */
  int ac_top_flux;       /* 1: also impose delta_v dPhi_v/dn = delta_v j_out on the top boundary */
  int precision;         /* 0: FP64 throughout; 1: FP32 preconditioners inside FP64 FGMRES;
                            2: as 1, with the velocity multigrid's matrix values stored in BF16
                            on every level (FP32 vectors, Jacobi diagonals and accumulation) */
  double rtol, atol;     /* stopping rule ||b - A x|| <= max(rtol ||b||, atol) (Sec. 5) */
  int restart, maxit;    /* FGMRES restart length (<= 64) and total iteration cap */
  int model;             /* 0: polymer, NFA, solvent, air with eqn:appPotential;
                            1: solvent-air sub-model (Sec. 5.1): no polymer / NFA (their
                            fields stay zero and are not solved for), the Flory-Huggins
                            density with every phi ln phi replaced by its degree-4 Taylor
                            polynomial at 1/2 (Sec. 5), RT/V0 = 1, and the new solvent
                            fraction truncated to [0, 1] (eqn:truncateCH) */
  double chi_sa;         /* model 1: Flory-Huggins interaction solvent-air */
  double n_s, n_a;       /* model 1: molar sizes N_s, N_a (> 0) */
  double phi_sat_s, phi_sat_a;  /* model 1: saturated vapour fractions (> 0) */
  double inner_rtol;     /* 0: every multigrid block of the preconditioners is one V-cycle;
                            > 0 (< 1): each is the V-cycle iteration x <- x + V(b - A x) from
                            x = 0 to ||b - A x|| <= inner_rtol ||b|| (Sec. 5 applies its AMG
                            preconditioners to a tolerance of 1e-4): MG(M + tau C), the
                            matching factors X, MG of the AC matrix, the velocity block and
                            K_p; the CH species are then solved one after the other */
  int inner_maxit;       /* cap on the V-cycles of one inner solve (1..1000, inner_rtol > 0) */
  double ns_rtol, ns_atol;  /* ns_rtol > 0: stopping rule of the Oseen solve alone (Sec. 5 uses
                               rtol 1e-4, atol 1e-8 for it and 1e-6, 1e-8 for CH and AC);
                               0: the Oseen solve uses rtol, atol */
  int ortho;             /* arithmetic of the FGMRES Gram-Schmidt passes (CGS2): 0: FP64;
                            1: double-FP32, every value a pair of FP32 numbers (about 48
                            significant bits; Dekker's exact product, Knuth's two-sum) on the
                            FP32 pipe, with the basis kept as pairs beside its FP64 copy (the
                            outer residuals, the Hessenberg data, the solution update and the
                            preconditioner input stay FP64); applies when restart <= 31 */
  int amg;               /* multigrid of the Allen-Cahn block M + tau delta_v K + tau C: 0 the
                            geometric hierarchy; 1 the device smoothed aggregation of the fine
                            AC matrix (chnss_amg_* below, Sec. 5's PyAMG for this block):
                            aggregates and patterns built once per context, the levels set up
                            again from the assembled matrix in every step.  2D only
                            (CHNSS_ERR_ARG in 3D) */
} chnss_params;

/* Fields of one time level (DEVICE pointers, caller-owned, FP64). */
typedef struct {
  double *phi[3];        /* phi_p, phi_NFA, phi_s           [N1] each */
  double *mu[4];         /* mu_p, mu_NFA, mu_s, mu_a        [N1] each */
  double *Phi_v;         /* vapour order parameter          [N1] */
  double *v;             /* velocity, interleaved (x, y)    [2*N2] */
  double *p;             /* pressure (zero mean)            [N1] */
} chnss_state;

typedef struct {
  int iters;             /* Krylov iterations (Arnoldi steps / CG steps) */
  int converged;         /* 1 if the stopping rule was met */
  double rel_residual;   /* final true ||b - A x|| / ||b|| (0 if b = 0) */
  double seconds;        /* host wall time of the solve */
} chnss_solve_info;

/* Mesh hierarchy for n x n squares on [0,lx] x [0,ly]: n even, 2 <= n <= 2048,
 * nx == ny required.  Multigrid levels n, n/2, ... while the size is even and
 * at least 4; the coarsest level (n = m 2^k with m odd or m = 2) must have
 * m <= 25 cells per side.  On it the pressure Laplacian of the PCD keeps a
 * dense FP64 inverse (built once by one thread block, (m + 1)^2 rows), as
 * does every block while the level has at most 256 unknowns; larger
 * non-singular coarsest levels (the velocity block for m >= 7, the P1 blocks
 * for m >= 17) take 16 Chebyshev-Jacobi steps from zero on [hi/64, hi]
 * instead.  n = 50, 100, 200 (m = 25) are accepted.  Builds the CSR patterns, the element -> CSR gather maps and
 * the transfer operators (host), and uploads them.  Returns CHNSS_ERR_ARG
 * for bad sizes, CHNSS_ERR_OOM / CHNSS_ERR_CUDA on device failures. */
chnss_status chnss_mesh_create(int nx, int ny, double lx, double ly, chnss_mesh_t *out);
/* The same with a choice of velocity condition on the top edge:
 * top_bc = 0: no-slip on the whole boundary (eqn:bc), pressure with zero
 * mean (as chnss_mesh_create); top_bc = 1: open top, i.e. no-slip on the
 * bottom and side walls and the do-nothing condition (2 eta eps(v) - p I) n = 0
 * on the top edge (its corners stay on the walls).  With an open top the
 * pressure is not shifted, and the pressure convection-diffusion
 * preconditioner puts homogeneous Dirichlet rows on the top pressure nodes
 * of A_p and K_p (outflow condition; K_p is then non-singular).  The
 * adjoint step returns CHNSS_ERR_ARG on such meshes.  CHNSS_ERR_ARG for
 * other top_bc values. */
chnss_status chnss_mesh_create_ex(int nx, int ny, double lx, double ly, int top_bc, chnss_mesh_t *out);
chnss_status chnss_mesh_destroy(chnss_mesh_t mesh);
/* Sizes: N1 P1 nodes, N2 P2 nodes, E triangles, number of multigrid levels. */
chnss_status chnss_mesh_sizes(chnss_mesh_t mesh, int *N1, int *N2, int *E, int *levels);

/* Context on `mesh` (which must outlive it) with a copy of *params; all work
 * goes to `cuda_stream` (a cudaStream_t, or NULL for the legacy stream).
 * Assembles the state-independent matrices (Sec. 4: M, K, K_sym, B, M_p,
 * K_p) on the device. */
chnss_status chnss_ctx_create(chnss_mesh_t mesh, const chnss_params *params, void *cuda_stream,
                              chnss_ctx_t *out);
chnss_status chnss_ctx_destroy(chnss_ctx_t ctx);

/* Per-step assembly from the fields at t_k (Sec. 3-4): C(v^k), J(w^k) with
 * w = v - sum alpha_i grad mu_i, A_p, the multigrid coarse operators by
 * rediscretisation with injected coefficients, the potential loads of
 * eqn:appPotential, the Korteweg term G^k and all right-hand sides. */
chnss_status chnss_assemble(chnss_ctx_t ctx, const chnss_state *state_k);

/* Unknown count of a system (2*N1, N1 or 2*N2 + N1). */
int chnss_system_size(chnss_ctx_t ctx, chnss_system sys);

/* Preconditioned FGMRES (CH, AC, NS) or Jacobi-PCG (MU_A) on an assembled
 * system.  rhs_or_null: device right-hand side of chnss_system_size doubles,
 * or NULL for the assembled one (for MU_A: built from the last three CH
 * solutions).  x_out: device array of the same size, overwritten (x0 = 0).
 * FGMRES reads the right-hand side again at every restart, so for CH, AC and
 * NS rhs and x_out must not overlap; MU_A may solve in place (rhs == x_out)
 * but not on partly overlapping arrays.  Overlap is refused with
 * CHNSS_ERR_ARG before any work.
 * Preconditioners (Sec. 4): CH diag(MG(M + tau C), X2^-1 M X1^-1) with the
 * matching factor X = tau gamma K + sqrt(tau gamma / beta) M (eqn::schurCH);
 * AC MG(M + tau delta_v K + tau C); NS diag(MG(A), M_p^-1 A_p K_p^-1)
 * (pressure convection-diffusion).  For NS the pressure is returned with
 * zero mean.  Returns CHNSS_ERR_NOCONV if maxit is reached. */
chnss_status chnss_solve(chnss_ctx_t ctx, chnss_system sys, const double *rhs_or_null, double *x_out,
                         chnss_solve_info *info);

/* One semi-implicit step t_k -> t_{k+1}: assemble, the three CH solves, AC,
 * the air potential, NS.  `in` and `out` must not alias.  info[6] (optional)
 * is filled in chnss_system order.  With every coefficient taken at t_k
 * (Sec. 3) the CH systems (+ air potential), AC and NS are independent once
 * assembled: by default they run concurrently on three library-owned
 * streams driven by three host threads (the call spawns two), ordered after
 * the assembly on the context stream, which waits for all three before the
 * call returns.  With constant mobility the three CH systems are solved
 * together (one batched preconditioner per Krylov iteration).  Results are
 * bitwise the same as solving every system alone with chnss_solve.  The
 * returned status is the first failure in the order CH (p, NFA, s), AC, air
 * potential, NS. */
chnss_status chnss_step(chnss_ctx_t ctx, const chnss_state *in, chnss_state *out, chnss_solve_info *info);
/* on = 0: chnss_step runs the three solve groups one after the other on the
 * context stream's host thread, and the preconditioner graphs launch one
 * kernel at a time (same results; used to time kernels alone); on != 0
 * (default): the solve groups run concurrently and the independent parts of
 * a preconditioner (Oseen pressure block, CH Schur groups) are parallel
 * graph branches.  Changing the setting re-captures the context's graphs. */
chnss_status chnss_set_step_concurrency(chnss_ctx_t ctx, int on);

/* Same step with HOST arrays (same layout as chnss_state): copies the input
 * to library-owned device fields, steps, copies the result back and
 * synchronises the stream. */
chnss_status chnss_step_host(chnss_ctx_t ctx, const chnss_state *host_in, chnss_state *host_out,
                             chnss_solve_info *info);

/* Adjoint of one step (discrete adjoint of chnss_step; model 0:
 * CHNSS_ERR_ARG for the solvent-air model; enclosed or open top, constant or
 * concentration-dependent mobility).
 * Every solve x = A(u)^-1 b(u) of the step contributes, with
 * y = A^-T xbar (FGMRES on the transposed operator to a relative residual of
 * 1e-12, preconditioned by the forward block preconditioner),
 * ubar += (db/du)^T y - (d(A(u) x)/du)^T y: the transposed convection
 * derivatives of C(v) (CH, AC) and J(w) (Oseen, w = v - sum alpha_i grad
 * mu_i), the Hessian of eqn:appPotential in the potential loads, the
 * Korteweg load, the evaporation flux j_out, and with mobility_kind 1 the
 * derivative of K_kappa(phi_i^k) in the first CH row.
 * state_k: fields at t_k; state_k1: the step's output at t_{k+1};
 * adj_k1: adjoint of the state at t_{k+1}; adj_k (out, overwritten):
 * adjoint of the state at t_k (all DEVICE arrays, chnss_state layout;
 * velocity adjoints are zero on the no-slip boundary, the pressure adjoint
 * is zero because p^k does not enter the step).  grad_params (HOST, 2
 * doubles, accumulated): d/d(evap_rate) and d/d(gamma) where gamma scales
 * all three mobilities.  info[6] (optional): the transposed solves.
 * Like chnss_step, the three independent groups (Oseen; Allen-Cahn; air
 * potential then Cahn-Hilliard) run concurrently on library streams unless
 * chnss_set_step_concurrency(ctx, 0); the result is bitwise the same either
 * way.  Synchronises the context stream before returning. */
chnss_status chnss_adjoint_step(chnss_ctx_t ctx, const chnss_state *state_k, const chnss_state *state_k1,
                                const chnss_state *adj_k1, chnss_state *adj_k, double *grad_params,
                                chnss_solve_info *info);
/* Final-morphology functional J = int |grad phi_p|^2 = phi_p^T K phi_p of a
 * device polymer field; *J on the host; grad_phi_p (device, optional) = 2 K phi_p. */
chnss_status chnss_objective(chnss_ctx_t ctx, const double *phi_p, double *J, double *grad_phi_p);

/* Conservation and energy diagnostics of a device state, in FP64 with
 * deterministic reductions (fixed grid and summation order: bit-reproducible
 * on a given device).  The scheme conserves int phi_i exactly for enclosed
 * flow (Sec. 3: the Cahn-Hilliard equations in divergence form with
 * homogeneous fluxes, the discrete velocity divergence-free against the P1
 * pressure space), keeps the pressure in L^2_0 (Sec. 3) and is driven by the
 * free energy of Sec. 2.2.  Fields of the result:
 *   mass[4]          int phi_i dx = 1^T M phi_i for i = p, NFA, s and the air
 *                    fraction phi_a = 1 - sum phi_i (exact for P1 fields);
 *   div_norm         ||B v||_2, the discrete divergence of the velocity;
 *   p_mean           int p dx = 1^T M p;
 *   energy_local     int f(phi, Phi_v) dx, f of eqn:appPotential (model 0) or
 *                    the solvent-air density (model 1), a rule exact to degree 7;
 *   energy_gradient  sum_i beta_i/2 int |grad phi_i|^2 + beta_v/2 int |grad Phi_v|^2
 *                    (i over the four species, phi_a = 1 - sum phi_i);
 *   energy_kinetic   1/2 int |v|^2 dx (rho = 1), the P2 mass form;
 *   energy           the sum of the three parts.
 * state: device arrays of ctx's mesh (chnss_state layout; mu is not read).
 * Runs on ctx's stream and synchronises it once; needs no assembly.  Uses
 * the context's scratch, so do not call it while a step of ctx is in flight
 * on another thread.  Errors: CHNSS_ERR_ARG for null arguments. */
typedef struct {
  double mass[4];
  double div_norm;
  double p_mean;
  double energy;
  double energy_local, energy_gradient, energy_kinetic;
} chnss_diag;
chnss_status chnss_diagnostics(chnss_ctx_t ctx, const chnss_state *state, chnss_diag *out);

/* Debug / test export of assembled fine-level objects to HOST memory.
 * which: 0 L = M + tau C, 1 AC matrix, 2 velocity block A (scalar CSR of the
 * interleaved dofs), 3 B (N1 x 2*N2), 4 A_p, 5 M, 6 K.  Call with null arrays
 * to get *nrows and *nnz, then again with rowptr[nrows+1], col[nnz],
 * val[nnz]. */
chnss_status chnss_export_csr(chnss_ctx_t ctx, int which, int *nrows, int *nnz, int *rowptr, int *col,
                              double *val);
/* Debug / test entry: one orthogonalisation step of FGMRES (Sec. 5 solves
 * with GMRES; the build's Krylov method orthogonalises by classical
 * Gram-Schmidt applied twice) of the device vector w against the k device
 * vectors V (column j at V + j ld, 1 <= k <= 31, ld >= n and even), with the
 * library's own kernels in FP64 (arith 0) or double-FP32 (arith 1, the
 * ortho = 1 path).  h (host, 2k + 1 doubles): the pass-1 dots V^T w, the
 * pass-2 dots V^T w' of w' = w - V h1, and ||w'||^2; vout (device, n): the
 * next basis vector (w' - V h2) / hn with hn^2 = ||w'||^2 - ||h2||^2.  V and
 * w are not modified.  Allocates its scratch with cudaMalloc on every call
 * and synchronises; CHNSS_ERR_ARG for bad sizes or null pointers. */
chnss_status chnss_debug_cgs2(int arith, long n, int k, const double *V, long ld, const double *w, double *h,
                              double *vout);
/* Test entry: one sparse matrix-vector product through the library's
 * SELL-C-sigma SpMV kernels, with the dispatch the solvers use (including the
 * number of warps that share a slice).  layout 0: scalar rows; 1: 2x2 blocks;
 * 2: 3x3 blocks (vectors interleaved per node, bs = 1, 2, 3).  precision 0:
 * FP64 values and vectors; 1: FP32; 2: BF16 values, FP32 vectors and sums.
 * mode 0: y = A x; 1: y = b - A x; 2: y += A x; 3 (square only):
 * y = c0 x + c1 w + c2 dinv (b - A x) with (c0, c1, c2) = coef (w may be
 * null: no c1 term).  HOST arrays: the (node) pattern in CSR with ascending
 * columns per row (rowptr[nrows + 1], col[nnz]), val (nnz blocks of bs^2
 * values, each block row-major), x (bs ncols), b, w, dinv (bs nrows),
 * coef[3]; y (bs nrows; read by mode 2, then written).  *warps_per_slice
 * (optional, out): the warps per SELL slice the dispatcher chose.  Allocates
 * its device copies and synchronises; CHNSS_ERR_ARG for bad sizes, modes,
 * columns or null pointers. */
chnss_status chnss_debug_spmv(int layout, int precision, int mode, int nrows, int ncols, const int *rowptr,
                              const int *col, const double *val, const double *x, const double *b, const double *w,
                              const double *dinv, const double *coef, double *y, int *warps_per_slice);
/* Assembled right-hand side of a system (host, chnss_system_size doubles). */
chnss_status chnss_export_rhs(chnss_ctx_t ctx, chnss_system sys, double *host_out);

/* Tracing: CUDA-event durations and algorithmic bytes of the hot kernel
 * families of one context, plus the number of kernels the library launched
 * in this process.  Families: multigrid fine-level velocity SpMV (smoother
 * and residual sweeps), multigrid fine-level P1 SpMV, Navier-Stokes operator
 * SpMV, Krylov orthogonalisation (one record per Arnoldi step), assembly
 * with preconditioner setup (bytes not counted), and the time of every
 * multigrid level below the finest, per V-cycle, for the P1 and the velocity
 * hierarchies (bytes not counted). */
typedef struct {
  long long launches;          /* kernels launched by the library in this process */
  int nkinds;
  char name[8][32];
  long long kind_launches[8];  /* timed launches (or Arnoldi steps) per family */
  double kind_ms[8];           /* summed CUDA-event durations */
  double kind_bytes[8];        /* summed algorithmic bytes */
  double kind_flops[8];        /* summed floating-point operations (orthogonalisation only) */
} chnss_profile;
/* on != 0: reset the counters and start recording (synchronises the stream). */
chnss_status chnss_profile_enable(chnss_ctx_t ctx, int on);
/* Read the counters (synchronises the stream). */
chnss_status chnss_profile_read(chnss_ctx_t ctx, chnss_profile *out);

/* Inner multigrid solves (inner_rtol > 0), per preconditioner block in the
 * order MG(M + tau C), MG(M + tau delta_v K + tau C), velocity MG(A),
 * MG(K_p), X1 of polymer / NFA / solvent, X2 of polymer / NFA / solvent
 * (CHNSS_INNER_BLOCKS): inner solves and V-cycles since the last reset, and
 * ||b - A x|| / ||b|| at the end of the last solve.  Blocks without inner
 * solves (inner_rtol = 0, X2 with constant mobility) report zeros.
 * reset != 0 clears the counts after reading.  Synchronises the stream. */
#define CHNSS_INNER_BLOCKS 10
typedef struct {
  long long solves[CHNSS_INNER_BLOCKS];
  long long cycles[CHNSS_INNER_BLOCKS];
  double last_rel_residual[CHNSS_INNER_BLOCKS];
} chnss_inner_stats;
chnss_status chnss_inner_stats_read(chnss_ctx_t ctx, int reset, chnss_inner_stats *out);

/* Tetrahedral (3D) discretisation, host side.  The box [0,1]^3 in n^3 cubes,
 * each split into the six Kuhn tetrahedra along its main diagonal (the 3D
 * form of the 2D diagonal split; the paper's 3D runs use uniform
 * tetrahedral meshes of a cube, Sec. 5).  P1 node (a, b, c) has id
 * (c (n+1) + b)(n+1) + a; velocity interleaved (x, y, z) per P2 node of the
 * doubled lattice, node (A, B, C) id (C m + B) m + A, m = 2n + 1.
 * chnss3_host_operator builds one operator on the HOST (no device use) with
 * the element operators the 3D device step uses, in CSR (duplicates summed in
 * element order) or, for the load vectors, as a dense vector:
 *   CHNSS3_OP_M1       P1 mass (N1 x N1)
 *   CHNSS3_OP_K1       P1 stiffness
 *   CHNSS3_OP_C1       P1 convection int (v . grad psi_b) psi_a by the P2 velocity state->v
 *   CHNSS3_OP_CP       the same with v - sum_i alpha_i grad mu_i (A_p of the PCD)
 *   CHNSS3_OP_M2       scalar P2 mass (N2 x N2)
 *   CHNSS3_OP_J2       scalar P2 convection by w = v - sum_i alpha_i grad mu_i
 *   CHNSS3_OP_KSYM     eta-weighted symmetric-gradient form on the velocity (3 N2 x 3 N2, no boundary rows)
 *   CHNSS3_OP_B        - int psi_q div zeta (N1 x 3 N2, no boundary columns)
 *   CHNSS3_OP_P1PROL   P1 prolongation from the n/2 mesh (n even)
 *   CHNSS3_OP_VPROL    velocity prolongation from the n/2 mesh, interior nodes of both meshes
 *   CHNSS3_OP_LOADS    the five potential loads of eqn:appPotential, concatenated (5 N1)
 *   CHNSS3_OP_KORTEWEG the Korteweg load (3 N2; beta_i, beta_v from params)
 *   CHNSS3_OP_TOP      int over the top face of each P1 hat (N1)
 *   CHNSS3_OP_KK0..2   weighted stiffness int kappa grad psi_a . grad psi_b of species 0..2 with the
 *                      concentration-dependent mobility kappa = gamma_i (phi_i (1 - phi_i) + mobility_m0)
 *                      (state->phi[i]; any mobility_kind)
 *   CHNSS3_OP_VPROL_OPEN  CHNSS3_OP_VPROL on meshes with an open top (the top face's interior nodes
 *                      are unknowns)
 * state (HOST arrays, 3D sizes) supplies v, mu, phi, Phi_v where needed
 * (may be NULL otherwise).  Call with val == NULL to get nrows, ncols and nnz
 * (the vector length for the loads); then with rowptr (nrows + 1), col and
 * val (nnz) allocated (vectors: val only).  1 <= n <= 64. */
enum {
  CHNSS3_OP_M1 = 0, CHNSS3_OP_K1, CHNSS3_OP_C1, CHNSS3_OP_CP, CHNSS3_OP_M2, CHNSS3_OP_J2, CHNSS3_OP_KSYM,
  CHNSS3_OP_B, CHNSS3_OP_P1PROL, CHNSS3_OP_VPROL, CHNSS3_OP_LOADS, CHNSS3_OP_KORTEWEG, CHNSS3_OP_TOP,
  CHNSS3_OP_KK0, CHNSS3_OP_KK1, CHNSS3_OP_KK2, CHNSS3_OP_VPROL_OPEN
};
chnss_status chnss3_host_operator(int n, int which, const chnss_params *params, const chnss_state *state,
                                  int *nrows, int *ncols, long long *nnz, int *rowptr, int *col, double *val);

/* One semi-implicit step on the 3D Kuhn mesh of n^3 cubes of the unit box
 * (n even, 2 <= n <= 64), on the device: the 2D step's systems and solvers
 * (CH for three species with diag(MG(M + tau C), X^-1 M X^-1), AC with MG,
 * the air potential by Jacobi-PCG, Oseen with diag(MG(A), M_p^-1 A_p K_p^-1),
 * FGMRES(restart) with CGS2, geometric multigrid on the nested Kuhn meshes)
 * with no-slip on every face (or the open top of chnss3_ctx_create_ex) and
 * evaporation through the top face z = 1 (reference point (1/2, 1/2, 1)).  Covers model 0, constant or
 * concentration-dependent mobility (mobility_kind 0 or 1: then the first
 * row's tau K_kappa and the Schur factor X2 = tau K_kappa + a M as in 2D),
 * precision 0, 1 or 2, and one V-cycle per multigrid block or (inner_rtol
 * > 0) V-cycles to inner_rtol as in 2D; other parameter sets get
 * CHNSS_ERR_ARG.  Assembly runs on the context's stream
 * (cuda_stream, or a library stream when NULL), the solve groups on library
 * streams after it (chnss3_set_step_concurrency).
 * States: chnss_state with DEVICE arrays of the 3D sizes (chnss3_sizes):
 * phi[3], mu[4], Phi_v, p of N1 = (n+1)^3, v of 3 N2 = 3 (2n+1)^3.
 * info[6] (optional): the six solves as in chnss_step.  chnss3_step
 * synchronises the stream before returning.  Ownership: the caller owns the
 * state arrays (in and out must not overlap); the context owns its device
 * workspace, streams and captured graphs, released by chnss3_ctx_destroy.
 * Errors: CHNSS_ERR_ARG (bad size or parameters: nothing is allocated; the
 * text is in chnss_last_error(NULL)), CHNSS_ERR_CUDA / CHNSS_ERR_OOM (the
 * device failed), and from chnss3_step the first non-OK status of the six
 * solves (CHNSS_ERR_NOCONV, CHNSS_ERR_BREAKDOWN, CHNSS_ERR_NAN), with the
 * outputs holding the last iterates and the text in chnss3_last_error. */
typedef struct chnss3_ctx *chnss3_ctx_t;
chnss_status chnss3_ctx_create(int n, const chnss_params *params, void *cuda_stream, chnss3_ctx_t *out);
/* As chnss3_ctx_create with the velocity condition on the top face z = 1:
 * top_bc 0: no-slip on every face (eqn:bc; the pressure normalised to zero
 * mean after the Oseen solve); 1: open top as chnss_mesh_create_ex's
 * top_bc = 1 in 2D: no-slip on the bottom and the side walls, the
 * do-nothing condition on the top face, Dirichlet outflow rows of A_p and
 * K_p on its nodes in the PCD, the pressure left as solved.  Other values:
 * CHNSS_ERR_ARG. */
chnss_status chnss3_ctx_create_ex(int n, int top_bc, const chnss_params *params, void *cuda_stream,
                                  chnss3_ctx_t *out);
chnss_status chnss3_ctx_destroy(chnss3_ctx_t ctx);
chnss_status chnss3_sizes(chnss3_ctx_t ctx, int *N1, int *N2);
chnss_status chnss3_step(chnss3_ctx_t ctx, const chnss_state *in, chnss_state *out, chnss_solve_info *info);
/* on != 0 (default): the three solve groups (CH species then the air
 * potential; AC; Oseen) of chnss3_step run concurrently on library streams;
 * 0: one after the other.  Results are bitwise the same. */
chnss_status chnss3_set_step_concurrency(chnss3_ctx_t ctx, int on);
const char *chnss3_last_error(chnss3_ctx_t ctx);
/* Adjoint of one 3D step: the discrete adjoint of chnss3_step, with the
 * same contributions as chnss_adjoint_step (transposed solves by FGMRES to a
 * relative residual of 1e-12 with the forward preconditioners; the
 * transposed convection derivatives of C(v) and J(w), w = v - sum alpha_i
 * grad mu_i, the potential Hessian at the degree-7 tetrahedral rule, the
 * Korteweg load, the evaporation flux and, with mobility_kind 1, the
 * derivative of K_kappa(phi_i^k)) on the tetrahedra; enclosed or open top.
 * state_k, state_k1 (the step's output), adj_k1, adj_k (out, overwritten):
 * DEVICE states of the 3D sizes; velocity adjoints are zero on the no-slip
 * dofs, the pressure adjoint is zero.  grad_params (HOST, 2 doubles,
 * accumulated): d/d(evap_rate), d/d(gamma) with gamma scaling the three
 * mobilities.  info[6] (optional): the transposed solves.  As in
 * chnss3_step the three groups (Oseen; Allen-Cahn; air potential then
 * Cahn-Hilliard) run concurrently on library streams unless
 * chnss3_set_step_concurrency(ctx, 0); their contributions are summed in a
 * fixed order, so the result is bitwise the same either way.  The context
 * stream is synchronised before the return.  Errors as chnss3_step (text in
 * chnss3_last_error). */
chnss_status chnss3_adjoint_step(chnss3_ctx_t ctx, const chnss_state *state_k, const chnss_state *state_k1,
                                 const chnss_state *adj_k1, chnss_state *adj_k, double *grad_params,
                                 chnss_solve_info *info);
/* J = int |grad phi_p|^2 = phi_p^T K phi_p of a device polymer field on the
 * 3D mesh; *J on the host; grad_phi_p (device, optional) = 2 K phi_p. */
chnss_status chnss3_objective(chnss3_ctx_t ctx, const double *phi_p, double *J, double *grad_phi_p);

/* Mass-matrix solve that allocates nothing.  The paper has no counterpart:
 * this is a service entry point of the library.  It solves M x = rhs for the
 * P1 mass matrix of ctx's mesh with the same Jacobi-preconditioned conjugate
 * gradients as the air-potential solve (relative tolerance 1e-12, x0 = 0),
 * but keeps its four work vectors and its reduction partials in a fixed
 * device array inside the library instead of context memory, and calls no
 * cudaMalloc / cudaFree.  It exists for callers that cannot allocate device
 * memory at the point of the call: programs whose device memory is entirely
 * reserved up front by their own pool (an allocation would fail or break
 * their accounting) and latency-critical loops that may not pay the implicit
 * synchronisation of cudaMalloc / cudaFree.
 * rhs, x_out: device arrays of N1 doubles, caller-owned.  rhs is read once,
 * before x_out is written, so an in-place solve (rhs == x_out) is allowed;
 * partly overlapping arrays return CHNSS_ERR_ARG.
 * Limit: N1 <= 66049 (meshes up to 256 x 256); larger meshes return
 * CHNSS_ERR_ARG with a message.  The array (about 2.13 MB) stays resident on
 * every GPU that loads the library until the process exits.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Every call shares the one array and overwrites it (the solver rewrites all
 * of it before reading), so calls whose work overlaps on the GPU (different
 * streams, threads or contexts at the same time) race and must not be
 * issued.  Synchronises ctx's stream once per iteration. */
chnss_status chnss_mass_solve_noalloc(chnss_ctx_t ctx, const double *rhs, double *x_out,
                                      chnss_solve_info *info);

/* Batched step for parameter sweeps (Sec. 5 runs the model over ranges of
 * evaporation rates and mesh sizes; every run is an independent time
 * integration).  Advances n_inst independent contexts by one chnss_step
 * each, concurrently: up to max_threads host threads (<= 0: one per
 * instance) each drive whole steps of one context at a time on that
 * context's own stream, so the instances' kernels overlap on the GPU.
 * ctxs[i] must be distinct (one context is not thread-safe), may differ in
 * mesh and parameters, and must all belong to the calling thread's current
 * device.  in[i] / out[i]: DEVICE states of ctxs[i] (chnss_step aliasing
 * rules); info (optional): 6 records per instance, instance i at
 * info + 6 i.  Each out[i] is bit-identical to chnss_step(ctxs[i], ...).
 * On failure every instance has still been attempted; the status and
 * message (chnss_last_error(NULL)) are those of the lowest failing index.
 * Returns after all instances' streams are synchronised. */
chnss_status chnss_step_batched(int n_inst, chnss_ctx_t *ctxs, const chnss_state *in, chnss_state *out,
                                chnss_solve_info *info, int max_threads);

/* How chnss_step (and chnss_step_host, chnss_step_batched) run a step.
 * mode 0 (default): host-driven, the Krylov loops decide on the host after
 * reading each iteration's residual estimate (one synchronisation per
 * iteration).  mode 1: the whole step as one CUDA graph launch with no host
 * synchronisation inside: every FGMRES restart cycle a conditional WHILE
 * node, every Arnoldi step a conditional IF node, every stopping decision a
 * one-thread kernel, the PCG iterations a WHILE node; the three solve groups
 * (Sec. 3: all coefficients at t_k) run as parallel graph branches, the
 * three CH species one after the other.  Same kernels, arithmetic and
 * stopping rules as mode 0, so the states and iteration counts are equal.
 * The graph is recorded on the first step with a given pair of state arrays
 * (two pairs are kept, so a ping-pong of two states records twice) and
 * replayed afterwards; it is recorded again after chnss_autotune,
 * chnss_set_spmv_block or chnss_set_step_concurrency.  Solve records
 * (iterations, convergence, residual, status) are returned as in mode 0
 * once the graph has finished.  Needs restart <= 31 (CHNSS_ERR_ARG).  With
 * every context of a chnss_step_batched call in mode 1, the batch is one
 * graph launch per instance, each on its instance's stream, from the calling
 * thread, then one synchronisation per stream (max_threads is ignored), or,
 * after chnss_set_batch_mode(1), one graph launch for the whole batch. */
chnss_status chnss_set_step_mode(chnss_ctx_t ctx, int mode);
/* Process-wide choice for chnss_step_batched calls whose contexts are all in
 * step mode 1.  mode 0 (default): one graph launch per instance, each on its
 * own stream.  mode 1: ONE graph launch per call for two or more instances:
 * every instance's step is recorded as a parallel branch of one graph (on
 * the first call with a given list of contexts and states; the two most
 * recent lists are kept, and a list is recorded again after one of its
 * contexts re-records its own graphs), launched on a library stream after
 * each context's stream has drained, then one synchronisation; if that graph
 * cannot be recorded, the call falls back to mode 0.  Destroying a context
 * drops the batch graphs that hold it.  Both modes give bitwise the same
 * states; mode 0 is faster on this part (64 sweep instances: 25.3 vs 15.0
 * instance steps/s).  CHNSS_ERR_ARG for another mode. */
chnss_status chnss_set_batch_mode(int mode);
/* Counters of chnss_step_batched calls in this process that ran as one
 * batch graph launch (*one_graph) and as one graph launch per instance
 * (*per_instance); either pointer may be NULL. */
chnss_status chnss_batch_stats(long long *one_graph, long long *per_instance);

/* Launch-shape autotuner.  Times the fine-level SpMV of the scalar (P1) and
 * of the velocity (2x2-block) multigrid operator of ctx for threads-per-block
 * 128, 256 and 512, keeps the fastest for each family (all levels and the
 * transfers of that family), and re-captures ctx's preconditioner graphs.
 * The choice is stored in the MESH, so it applies to every context sharing
 * it (contexts created earlier keep their captured shapes until they are
 * re-tuned).  Results do not depend on the launch shape: every row is summed
 * by one thread in the same order for any block size.  Needs an assembled
 * context (CHNSS_ERR_STATE otherwise).  out (host, optional): the timings
 * (ms per SpMV) and the choices. */
typedef struct {
  int candidates[3];   /* threads per block tried */
  double ms_p1[3];     /* fine scalar SpMV, ms */
  double ms_p2[3];     /* fine velocity SpMV, ms */
  int block_p1, block_p2;
} chnss_tuning;
chnss_status chnss_autotune(chnss_ctx_t ctx, chnss_tuning *out);
/* Set the SpMV threads-per-block of the scalar and velocity families by hand
 * (128, 256 or 512; CHNSS_ERR_ARG otherwise), with the same scope as
 * chnss_autotune (stored in the mesh; ctx's graphs are re-captured).  Do not
 * call it while another context on the same mesh is stepping. */
chnss_status chnss_set_spmv_block(chnss_ctx_t ctx, int block_p1, int block_p2);

/* Message of the last failure on ctx (or of the last failed create call
 * when ctx is NULL).  Valid until the next call on the same context. */
const char *chnss_last_error(chnss_ctx_t ctx);

/* ------------------------------------------------------------------------
 * Smoothed-aggregation algebraic multigrid for a general sparse operator.
 *
 * Sec. 5 builds the block preconditioners with PyAMG's algebraic multigrid:
 * smoothed aggregation (SA) for the nonsymmetric Cahn-Hilliard blocks
 * M + tau C (Sec. 4) and for every Navier-Stokes block of the 3D runs, on
 * meshes that need not be structured.  This handle runs the SA setup on the
 * device for a square CSR matrix A with the constant near-null space:
 *   strength graph: every stored off-diagonal entry (theta = 0);
 *   aggregates: a maximal distance-2 independent set of that graph (synchronous
 *     rounds on the keys (state, 30 leading bits of SplitMix64 output number
 *     (level << 32) + i, i)), every neighbour of a root joining its adjacent
 *     root of largest key, every remaining node its assigned neighbour of
 *     largest key;
 *   T[i, agg(i)] = 1 / sqrt(|agg(i)|);  P = T - (4 / (3 hi)) D^-1 (A T);
 *   A_c = P^T (A P);  hi = min(Gershgorin bound, 1.1 x a 10-step power
 *     estimate of rho(D^-1 A) from a +-1 start vector drawn with SplitMix64
 *     outputs ((level + 64) << 32) + i),
 * adding levels while a level has more than 64 rows (at most 12 levels).
 * Its V-cycle: Chebyshev-Jacobi pre- and post-smoothing of degree 2 on
 * [hi / 4, hi], restriction P^T, prolongation P, a dense FP64 inverse on a
 * coarsest level of at most 256 rows (otherwise 16 Chebyshev steps).  P and
 * A_c keep every structurally non-zero entry; every sum runs in a fixed
 * order, so the hierarchy and every result are bit-reproducible.
 *
 * A must be square with n >= 1 rows, its columns sorted and unique within
 * each row, a stored diagonal with non-zero values, and a structurally
 * symmetric pattern (entry (j, i) stored whenever (i, j) is: every finite-
 * element matrix); product rows of more than 512 entries are refused.
 * Errors are returned as statuses, with the message in chnss_last_error(NULL).
 * All pointers are DEVICE pointers unless the function says "host"; the
 * calls run on the handle's own stream and synchronise it before returning.
 */
typedef struct chnss_amg *chnss_amg_t;

/* Build the hierarchy of A (rowptr[n + 1], col[nnz], val[nnz]: device CSR,
 * read during the call only; the handle keeps its own copy of the values).
 * precision 0: the V-cycle in FP64; 1: level values, smoothing and
 * transfers in FP32 (the setup is FP64 either way).  CHNSS_ERR_ARG for a
 * matrix that breaks the rules above (nothing is kept), CHNSS_ERR_OOM /
 * CHNSS_ERR_CUDA on device failures. */
chnss_status chnss_amg_create(int n, int nnz, const int *rowptr, const int *col, const double *val, int precision,
                              chnss_amg_t *out);
/* New values of A on the same pattern (val: device, nnz doubles): the
 * aggregates and every pattern are kept (they depend on the pattern only),
 * the spectral bounds, prolongators, coarse operators and smoother data
 * are recomputed, as a per-step re-setup of the paper's time loop needs. */
chnss_status chnss_amg_update(chnss_amg_t h, const double *val);
/* Level count and, per level l < *nlevels (host arrays of at least 12
 * entries, each may be NULL): rows, nnz of A_l, nnz of P_l (0 on the
 * coarsest level). */
chnss_status chnss_amg_levels(chnss_amg_t h, int *nlevels, int *rows, int *nnz, int *pnnz);
/* Copy level l to HOST arrays (each may be NULL): agg[rows] (aggregate of
 * every node; level < nlevels - 1), hi (spectral bound), A_l as
 * a_rowptr[rows + 1], a_col[nnz], a_val[nnz], and P_l (rows x rows of level
 * l + 1) as p_rowptr[rows + 1], p_col[pnnz], p_val[pnnz]. */
chnss_status chnss_amg_export_level(chnss_amg_t h, int level, int *agg, double *hi, int *a_rowptr, int *a_col,
                                    double *a_val, int *p_rowptr, int *p_col, double *p_val);
/* x = one V-cycle applied to b (device, n doubles each; may not overlap). */
chnss_status chnss_amg_vcycle(chnss_amg_t h, const double *b, double *x);
/* Solve A x = b by right-preconditioned FGMRES(30) with one V-cycle as the
 * preconditioner, from x = 0, to ||b - A x|| <= max(rtol ||b||, atol) or
 * maxit iterations (Sec. 5 solver setup; the operator applied in FP64).
 * b and x: device, n doubles, may not overlap.  CHNSS_ERR_NOCONV at maxit
 * (x holds the last iterate); info (host, may be NULL) as chnss_solve. */
chnss_status chnss_amg_solve(chnss_amg_t h, const double *b, double *x, double rtol, double atol, int maxit,
                             chnss_solve_info *info);
/* Release everything the handle owns (NULL is ignored). */
void chnss_amg_destroy(chnss_amg_t h);

#ifdef __cplusplus
}
#endif
#endif /* CHNSS_H */
