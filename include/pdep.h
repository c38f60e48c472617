/*
 * pdep.h -- C ABI of the GB300 PDEP library (libpdep.so).
 *
 * The library computes the projective dielectric eigendecomposition (PDEP)
 * of Govoni & Galli, "Large scale GW calculations" (Sec. II C, "Projective
 * dielectric eigenpotential (PDEP) basis set"): the leading eigenpairs of the
 * symmetrised static irreducible polarizability
 *     chi0bar = v^{1/2} chi0 v^{1/2}          (Eq. symmoperator, omega = 0)
 * by a Davidson iteration (Sec. II C; Fig. pdepscheme) in which every
 * application of chi0bar is a batch of Sternheimer solves (Eq. stern)
 *     (H - eps_v) P_c dpsi_v = - P_c dV psi_v,   P_c = 1 - sum_v |v><v|,
 * one per occupied state v and perturbation, followed by the density
 * response of Eq. (deltani) and the projection of Eq. (chiisamatrixinpdep).
 *
 * Model and conventions
 *   - Hartree atomic units, Gamma point, spin-unpolarised, real orbitals,
 *     integer occupations (the n_occ lowest states), local potential only:
 *     H = -1/2 nabla^2 + V(r).  chi0bar eigenvalues are dimensionless, so
 *     the paper's Rydberg units give the same numbers.
 *   - Orthorhombic cell L1 x L2 x L3 (bohr) on an N1 x N2 x N3 grid; grid
 *     arrays are row-major with N3 fastest; point (i1,i2,i3) sits at
 *     (i1 L1/N1, i2 L2/N2, i3 L3/N3).
 *   - Basis (Eq. planewaveexpansionofwfc): plane waves with G =
 *     2 pi (n1/L1, n2/L2, n3/L3) and 0.5 |G|^2 <= ecut (compared in double
 *     precision).  ecut = 0 selects the alias-free grid rule
 *     ecut = 0.5 (min_i 2 pi r_i / L_i)^2 with r_i = (N_i - 1) / 4.
 *   - Real-coefficient layout of a sphere vector (length n_pw = 2 nh + 1):
 *     the half space {n3 > 0} u {n3 = 0, n2 > 0} u {n3 = n2 = 0, n1 > 0},
 *     restricted to the sphere and sorted by (n3, n2, n1) ascending, gives
 *     G_0 .. G_{nh-1}; a real function f(r) = Omega^{-1/2} sum_G c(G) e^{iG.r}
 *     is stored as x[2k] = sqrt2 Re c(G_k), x[2k+1] = sqrt2 Im c(G_k),
 *     x[2nh] = c(0).  Euclidean dot products are L2 inner products.
 *   - A PDEP vector (the PDEP basis excludes G = 0, the body of Table
 *     limitqchi0) has length n_pdep_dim = 2 nh: the first 2 nh entries.
 *   - chi0bar is restricted to that sphere minus G = 0; v^{1/2}(G) =
 *     sqrt(4 pi)/|G| (e^2 = 1).  The density response of a perturbation
 *     dV is dn(r) = 4 sum_v psi_v(r) dpsi_v(r) (2 for spin, 2 for the c.c.
 *     term of Eq. deltani).
 *
 * Memory, streams, errors
 *   - Array arguments may be host or device pointers; the library inspects
 *     each pointer and stages host data through its own device workspace.
 *     The caller owns every argument buffer; the library owns the context and
 *     its workspace and frees them in pdep_destroy.
 *   - 'stream' is a cudaStream_t (NULL = legacy default stream).
 *     chi0_apply and sternheimer_solve only enqueue work on it when every
 *     array argument is a device buffer: the Sternheimer CG loops and the
 *     mixed-precision refinement rounds are driven on the device, and
 *     nothing is read back; results are valid once the stream has been
 *     synchronised.  With a host buffer among the arguments the call copies
 *     through its workspace and synchronises before returning.  pdep_solve
 *     reads the Ritz values and residual norms back once per Davidson
 *     iteration (convergence test, correction choice) and synchronises at
 *     its end; the other calls synchronise before returning.
 *   - Every function returns a pdep_status.  pdep_last_error() gives a
 *     human-readable message for the most recent failure in this thread.
 *     Argument and launch errors are returned by the call.  Device-detected
 *     conditions (a non-finite CG scalar, a solve that ended above cg_tol,
 *     a spent clock budget) are OR-ed into a per-context device status word;
 *     a synchronising call (one with host outputs, pdep_solve,
 *     pdep_get_stats, pdep_sync_status) returns them as PDEP_ERR_NONFINITE,
 *     PDEP_ERR_TIMEOUT or PDEP_ERR_NOT_CONVERGED and clears the word, so the
 *     condition may stem from any call enqueued since the last such read.
 *     Outputs are written in every one of these cases.
 *   - One GPU (the device current when pdep_setup is called).  Calls on one
 *     context must not run concurrently.
 */
#ifndef PDEP_H
#define PDEP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdep_ctx pdep_ctx; /* opaque; owned by the library */

typedef enum {
  PDEP_OK = 0,
  PDEP_ERR_INVALID_ARG = 1,   /* bad size, unsupported grid, null pointer */
  PDEP_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  PDEP_ERR_OOM = 3,           /* device allocation failed or workspace limit hit */
  PDEP_ERR_NO_GAP = 4,        /* eps_{n_occ+1} - eps_{n_occ} < gap_min */
  PDEP_ERR_NOT_CONVERGED = 5, /* a solve reached its iteration cap */
  PDEP_ERR_NONFINITE = 6,     /* NaN/Inf met in the data or a CG scalar */
  PDEP_ERR_TIMEOUT = 7,       /* a CG loop spent its clock_budget_cycles */
  PDEP_ERR_UNSUPPORTED = 8,   /* option combination not implemented */
  PDEP_ERR_BOUNDS = 9         /* bounds-checked builds: a kernel met an index outside
                                 the sphere tables and skipped the access */
} pdep_status;

typedef enum {
  PDEP_FP64 = 0,       /* every step in FP64 */
  PDEP_MIXED_TF32 = 1, /* FP32 FFTs, H*psi and vector updates inside the
                          Sternheimer CG, its projection term on the tensor
                          cores (TF32 operands split in three for FP32
                          accuracy, FP32 accumulation); FP64 residual
                          refinement, density response, orthogonalisation and
                          Rayleigh-Ritz */
  PDEP_MIXED_BF16 = 2  /* as PDEP_MIXED_TF32, but inside the FP32 inner CG the
                          projection coefficients sum_k w_k x_k come from one BF16
                          product per term (tcgen05 kind::f16, FP32 accumulation),
                          which perturbs the CG operator at about 2^-9: each
                          inner solve then stops at max(inner_tol, 3e-3) and more
                          refinement rounds follow.  The refinement's products
                          are those of the TF32 mode, so solutions still reach
                          cg_tol in the FP64 residual.  On the 48^3 workload it
                          is 13% slower than PDEP_MIXED_TF32 (5 rounds instead of
                          2) and matches FP64 eigenvalues to 4e-10. */
} pdep_precision;
#define PDEP_MIXED PDEP_MIXED_TF32 /* the default mixed mode */

/* One system. v_r: [N1*N2*N3] local potential (Ha), host or device. */
typedef struct {
  int grid[3];
  double cell[3];
  double ecut;        /* Ha; 0 = alias-free grid rule */
  const double* v_r;
  int n_occ;          /* occupied states (>= 1) */
  int n_pdep;         /* PDEP eigenpairs wanted (>= 1) */
} pdep_system_desc;

typedef struct {
  int precision;             /* pdep_precision */
  double cg_tol;             /* Sternheimer: ||b - A x|| / ||b|| target (1e-10) */
  int cg_max_iter;           /* FP64 path: CG iteration cap of each refinement round */
  double inner_tol;          /* mixed: FP32 inner CG reduction per refinement round */
  int inner_max_iter;        /* mixed: FP32 CG iteration cap per round */
  int max_refine;            /* refinement rounds cap (both paths).  Every solve runs in
                                rounds: an inner CG on the residual scaled to unit norm
                                (FP64, or FP32 in the mixed modes), then x += delta and
                                the FP64 residual r -= A delta; the FP64 path's first
                                round normally meets cg_tol, a further round catching
                                solves whose recomputed residual drifted above it. */
  double dav_tol;            /* Davidson: max ||chi0bar x - theta x|| / |theta_1|; 0 = run dav_max_iter */
  int dav_max_iter;          /* Davidson iterations cap (each applies chi0bar once) */
  int dav_subspace_factor;   /* subspace holds at most factor * n_pdep vectors (>= 2) */
  unsigned long long seed;   /* Philox4x32-10 seed of the random start block */
  double gap_min;            /* minimum HOMO-LUMO gap (Ha) */
  double setup_tol;          /* setup eigensolver: ||H psi - eps psi|| target */
  int setup_max_iter;
  size_t workspace_limit_bytes; /* 0 = no limit */
  int n_deflate;             /* lowest empty states deflated from the Sternheimer CG
                                (0: occupied states only; default 16).  The setup
                                converges them with the occupied states; their
                                share of each solution is added exactly and the CG
                                works on the rest, whose smallest eigenvalue is
                                eps_{n_occ+n_deflate+1} - eps_v instead of the gap. */
  int proj_variant;          /* kernel of the FP32 (mixed-mode CG) projection term
                                sum_w sigma_w |w><w| x: -1 = autotuned (default; the
                                first large calls time all three), 0 = FP32 CUDA-core
                                GEMMs, 1 = 3xTF32 tensor-core GEMMs on mma.sync,
                                2 = the coefficient GEMM 3xTF32 on tcgen05 with
                                tensor-memory accumulators (its waits on the tensor
                                cores are bounded: one that runs out sets
                                PDEP_ERR_TIMEOUT), the update as in 1. */
  long long clock_budget_cycles; /* device time budget of every CG loop, in SM clock
                                cycles at the device's rated clock (0 = none).  A loop
                                whose budget runs out with unconverged RHS stops after
                                its current step and sets PDEP_ERR_TIMEOUT in the device
                                status word (outputs are still written). */
  int autotune;              /* 1 (default): the first large CG loops of a context time
                                the CG-step launch shapes and the projection kernels and
                                keep the fastest; 0: fixed defaults */
  int use_graph;             /* 1 (default): each Sternheimer CG loop runs as one CUDA
                                graph with a device-driven while node (no host round trip
                                per step) once the autotuner has fixed the launch shapes;
                                0: a host loop that reads the loop state after every step */
  int df_refine;             /* mixed modes, precision of the refinement's A delta (and of
                                the density response accumulated with it); vectors,
                                residuals and the density stay FP64 throughout.
                                2 (default): transforms in double-float arithmetic (pairs
                                of FP32 numbers, about 48 significant bits; the FP32 pipe
                                runs 64x the FP64 rate) in the first round, FP32 in later
                                rounds, whose correction is about inner_tol of the
                                solution, so that FP32 errs by ~1e-7 inner_tol ||b||;
                                1: double-float in every round; 0: FP64 transforms */
  int fused_hpsi;            /* 1 (default): the FP32 H x of the inner CG on the cubic grids
                                24^3 .. 48^3 in one launch that keeps each item's column
                                scratch in shared memory; 0: three launches through a
                                global-memory scratch (always used for other grids) */
} pdep_options;

typedef struct {
  int dav_iterations;           /* chi0bar applications performed */
  int converged;                /* 1 if dav_tol was met (or dav_tol = 0) */
  long long sternheimer_solves; /* (v, perturbation) systems solved to cg_tol */
  long long cg_iterations;      /* sum over solves (FP32 inner iterations in mixed mode) */
  int cg_iterations_max;        /* largest per-solve count */
  int refine_rounds_max;        /* mixed mode: largest refinement round count */
  double max_cg_residual;       /* largest final ||b - A x|| / ||b||, recomputed in FP64 */
  double max_dav_residual;      /* largest final ||chi0bar x - theta x|| / |theta_1| */
  double seconds;               /* wall time of the call */
  int cg_variant;               /* CG-step launch shape the autotuner chose (-1: untuned) */
  int proj_variant;             /* FP32 projection kernel in use (-1: untuned, 0, 1, 2;
                                   3: PDEP_MIXED_BF16, BF16 coefficients in the inner CG) */
  int chi0_chunks;              /* perturbation chunks of the last chi0bar application */
  long long kernel_launches;    /* library kernels the call ran, those inside CUDA graphs
                                   included (graph steps counted on the device) */
  long long graph_launches;     /* CG-loop graphs launched */
  int fused_planes;             /* x-planes per group of the fused FP32 transform the
                                   autotuner chose (-1: untuned or not used) */
  int gemm_shape;               /* tile shape of the FP64 / double-float projection GEMMs the
                                   autotuner chose: 0 64-row tiles, 1 80-row, 2 80-row with
                                   half the default split-K, 3 80-row with twice (-1 untuned) */
} pdep_stats;

/* Fill *opt with the defaults (FP64, cg_tol 1e-10, dav_tol 1e-8, ...). */
void pdep_default_options(pdep_options* opt);

/* Build one context for n_sys systems: sphere tables, potential upload and the
 * FP64 setup eigensolve of the n_occ lowest states (the unperturbed occupied
 * states of Sec. II C), with the gap check.  Returns PDEP_ERR_NO_GAP when
 * eps_{n_occ+1} - eps_{n_occ} < gap_min, PDEP_ERR_INVALID_ARG for an
 * unsupported grid (N1 in {24,32,40,48,64}; N2 = N3 in that set, or
 * N2 = 64 with N3 = 192). */
int pdep_setup(const pdep_system_desc* sys, int n_sys, const pdep_options* opt, void* stream,
               pdep_ctx** out);

/* Sizes of system 'sys': n_pw (sphere real DOF), n_r (grid points),
 * n_pdep_dim = n_pw - 1.  Any output pointer may be NULL. */
int pdep_get_sizes(const pdep_ctx* ctx, int sys, int* n_pw, int* n_r, int* n_pdep_dim);

/* Occupied states of the setup: psi [n_occ][n_pw] real layout (may be NULL),
 * eps [n_occ + 1] eigenvalues including the lowest empty state (may be NULL). */
int pdep_get_occupied(pdep_ctx* ctx, int sys, double* psi, double* eps, void* stream);

/* chi0bar applied to n_pert PDEP vectors (Eqs. stern, deltani,
 * chiisamatrixinpdep): phi [n_pert][n_pdep_dim] in, chi0_phi
 * [n_pert][n_pdep_dim] out; dn_r [n_pert][n_r] (may be NULL) receives the
 * density response dn(r) (electrons/bohr^3) to dV = v^{1/2} phi. */
int chi0_apply(pdep_ctx* ctx, int sys, const double* phi, int n_pert, double* chi0_phi,
               double* dn_r, void* stream);

/* chibar applied to n PDEP vectors with the Hartree-only self-consistent
 * response (Sec. II C, Eqs. LF and LFHartree; no exchange-correlation
 * kernel): the perturbation of Eq. stern becomes dV_tot = v^{1/2} phi +
 * v dn[dV_tot].  Writing dV_tot = v^{1/2} y gives (1 - chi0bar) y = phi,
 * which is solved by conjugate gradients (1 - chi0bar is SPD: chi0bar is
 * negative semi-definite), each iteration applying chi0bar to the n
 * directions as one batch of Sternheimer solves; then
 *     out = chibar phi = y - phi = (1 - chi0bar)^{-1} chi0bar phi
 * (Eq. linearalgebrachichi0).  phi, out [n][n_pdep_dim].  Stops when every
 * ||phi - (1 - chi0bar) y|| <= tol ||phi|| or after max_iter iterations
 * (*iterations, may be NULL, receives the count); PDEP_ERR_NOT_CONVERGED
 * then, with out written.  The accuracy is bounded by that of the chi0bar
 * applications (the Sternheimer tolerance cg_tol). */
int pdep_chibar_apply(pdep_ctx* ctx, int sys, const double* phi, int n, double* out, double tol,
                      int max_iter, int* iterations, void* stream);

/* Sternheimer solves (Eq. stern) for n_pert perturbing potentials dv_r
 * [n_pert][n_r] (Ha) against every occupied state: dpsi [n_pert][n_occ][n_pw]
 * receives P_c dpsi_v; iters and resid [n_pert*n_occ] (may be NULL) receive
 * the CG iteration count and the final relative residual recomputed in FP64. */
int sternheimer_solve(pdep_ctx* ctx, int sys, const double* dv_r, int n_pert, double* dpsi,
                      int* iters, double* resid, void* stream);

/* Davidson PDEP solve (Sec. II C): the n_pdep most negative eigenvalues of
 * chi0bar, ascending, into eigvals [n_pdep]; eigvecs [n_pdep][n_pdep_dim]
 * (may be NULL).  phi0 [n_pdep][n_pdep_dim] is the start block (NULL: seeded
 * Philox4x32-10 normal deviates).  sys = -1 solves every system in turn and
 * then eigvals/eigvecs are the concatenation over systems.  stats is a host
 * struct (may be NULL). */
int pdep_solve(pdep_ctx* ctx, int sys, const double* phi0, double* eigvals, double* eigvecs,
               pdep_stats* stats, void* stream);

/* Screening at omega = 0 from PDEP eigenpairs (Sec. II A): with
 * g_i = lambda_i / (1 - lambda_i), the eigenvalues of the symmetrised
 * reducible polarizability chibar = (1 - chi0bar)^{-1} chi0bar
 * (Eq. linearalgebrachichi0), which shares chi0bar's eigenvectors, applies
 *   PDEP_SCREEN_CHIBAR: out = Phi diag(g) Phi^T f
 *   PDEP_SCREEN_EPSINV: out = f + Phi diag(g) Phi^T f        (Eq. epsilonandchi)
 *   PDEP_SCREEN_WP:     out = D Phi diag(g) Phi^T D f,  D = v^{1/2} =
 *                       sqrt(4 pi)/|G|, the correlation part W^p of the
 *                       screened interaction (Eq. Wpnondiag with the Coulomb
 *                       factors 4 pi e^2 written out)
 * to n vectors f [n][n_pdep_dim] -> out [n][n_pdep_dim]: the rank-n_pdep
 * (PDEP-basis) form of Eq. eigendecompzerofreq at omega = 0.  eigvals
 * [n_pdep] and eigvecs [n_pdep][n_pdep_dim] are eigenpairs of chi0bar as
 * pdep_solve returns them (orthonormal vectors).  Returns
 * PDEP_ERR_INVALID_ARG for an unknown kind, n_pdep outside [1, n_pdep_dim],
 * or an eigenvalue that is non-finite or has 1 - lambda <= 1e-12 (chi0bar
 * is negative semi-definite, so its eigenvalues are <= 0).  The head and
 * wings (G = 0, Eq. integrationxiq) are not part of the PDEP sphere. */
#define PDEP_SCREEN_CHIBAR 0
#define PDEP_SCREEN_EPSINV 1
#define PDEP_SCREEN_WP 2
int pdep_screening_apply(pdep_ctx* ctx, int sys, int kind, const double* eigvals,
                         const double* eigvecs, int n_pdep, const double* f, int n, double* out,
                         void* stream);

/* Body of chi0bar at imaginary frequencies in the PDEP basis (Sec. II B,
 * Eq. finalB) and its RPA screening (Eq. Bfinal without head and wings):
 *     B_ij(i nu) = phi_i^T chi0bar(i nu) phi_j
 *               = 4 sum_v Re <xi_iv| P_c O(eps_v - i nu) P_c |xi_jv>,
 *     xi_jv = dV_j psi_v, dV_j = v^{1/2} phi_j, O(w) = -(H - w)^{-1},
 * each matrix element taken from the poles and weights of a Lanczos chain of
 * P_c H P_c started on P_c xi_jv (n_steps steps, 1..64; Sec. II D, Eq.
 * MCfinal), and
 *     Lambda(i nu) = (1 - B)^{-1} B.
 * phi [n_pdep][n_pdep_dim] (e.g. the eigenvectors from pdep_solve), nu
 * [n_freq] (Ha, real, usually >= 0); B and Lambda [n_freq][n_pdep][n_pdep]
 * (Lambda may be NULL).  B is symmetrised, (B + B^T)/2.  At nu = 0, B equals
 * phi^T chi0bar phi up to the chains' truncation error.  Returns
 * PDEP_ERR_INVALID_ARG for n_steps outside [1, 64] or n_pdep outside
 * [1, n_pdep_dim], PDEP_ERR_NONFINITE if B has an eigenvalue >= 1. */
int pdep_chi0_imag(pdep_ctx* ctx, int sys, const double* phi, int n_pdep, const double* nu,
                   int n_freq, int n_steps, double* B, double* Lambda, void* stream);

/* Batched Lanczos chains of the deflated Hamiltonian H~ = P_c H P_c
 * (Sec. II D, Eqs. MCdef and MCfinal), FP64.  For each of n start vectors
 * R [n][n_pw]: q_1 = P_c R / ||P_c R||, then n_steps (1..64; the paper uses
 * 40) steps of the three-term recursion
 *     alpha_k = <q_k|H~|q_k>,
 *     beta_{k+1} q_{k+1} = (H~ - alpha_k) q_k - beta_k q_{k-1},
 * without reorthogonalisation.  The tridiagonal T = tridiag(beta, alpha,
 * beta) is diagonalised, T = U diag(d) U^T, and for n_L vectors L
 * [n_L][n_pw] the omega-independent poles and weights of Eq. MCfinal are
 * returned:
 *     poles [n][n_steps]          d_k, ascending,
 *     weights [n][n_L][n_steps]   ||P_c R|| sum_m <L|q_m> U_{m k} U_{1 k},
 * so that for any complex omega off the spectrum
 *     M_c,LR(omega) = -<L|(H~ - omega)^{-1}|R> ~ sum_k weights[k] / (omega - poles[k]).
 * alpha and beta [n][n_steps] (may be NULL) receive the recursion: beta[0] =
 * ||P_c R||, beta[k] (k >= 1) the off-diagonal T[k-1][k].  A chain that
 * reaches an invariant subspace (beta_{k+1} <= 1e-12 ||H~ q_k||) stops; its
 * later alphas, betas and weights are 0; a start vector with ||P_c R|| <=
 * 1e-12 ||R|| gives an empty chain (all 0).  L and weights may be NULL when
 * n_L = 0.  Returns PDEP_ERR_INVALID_ARG for n_steps outside [1, 64]. */
int pdep_lanczos(pdep_ctx* ctx, int sys, const double* R, int n, int n_steps, const double* L,
                 int n_L, double* poles, double* weights, double* alpha, double* beta,
                 void* stream);

/* y = H x for n sphere vectors x [n][n_pw] -> y [n][n_pw], H = -nabla^2/2 + V
 * (the local-potential Hamiltonian of the setup), evaluated with the pruned
 * sphere <-> grid transforms; precision PDEP_FP64, PDEP_MIXED (FP32
 * transforms) or PDEP_APPLY_DF64 (double-float transforms on FP64 vectors,
 * those of the mixed modes' refinement).  This is the H*psi kernel the
 * Sternheimer CG applies. */
#define PDEP_APPLY_DF64 3
int pdep_apply_hamiltonian(pdep_ctx* ctx, int sys, const double* x, int n, double* y,
                           int precision, void* stream);

/* y = H x like pdep_apply_hamiltonian (FP64), for callers that cannot
 * allocate device memory when they need it: code issuing work while a CUDA
 * graph is being captured on its stream, code running in a host callback or
 * an allocator hook, and embedders whose memory pool owns the whole device.
 * The paper has no counterpart to this entry point.
 *   - It allocates nothing: no cudaMalloc/cudaFree, no allocating library
 *     call, no staging.  x [n][n_pw] and y [n][n_pw] must be device buffers
 *     (host pointers are rejected with PDEP_ERR_INVALID_ARG).
 *   - Its transform scratch is one file-scope device array of 16 MiB
 *     (16777216 bytes), held by every GPU that loads the library until the
 *     process exits.  Vectors are processed in chunks of
 *     2 * floor(16 MiB / (N1 * n_col * 16 bytes)) (n_col: x-columns of the
 *     sphere); a grid whose single chunk does not fit is rejected with
 *     PDEP_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the device address of that array
 *     (cudaGetSymbolAddress, once per device, with the device current); make
 *     that first call before any stream capture.  The context's device must
 *     be the current device (PDEP_ERR_INVALID_ARG otherwise).
 *   - All calls share the array and it keeps the last call's contents; the
 *     transforms overwrite every scratch element before reading it, so
 *     nothing needs clearing.  Calls that overlap on the GPU (other streams,
 *     other threads) race on the scratch: serialise them.
 *   - The call only enqueues work on 'stream'; y is complete once the stream
 *     has been synchronised. */
int pdep_apply_hamiltonian_noalloc(pdep_ctx* ctx, int sys, const double* x, int n, double* y,
                                   void* stream);

/* u [n][n_r]: u(r_k) = sum_G c(G) exp(i G.r_k) for n sphere vectors x
 * [n][n_pw] (so the normalised function is Omega^{-1/2} u). */
int pdep_to_grid(pdep_ctx* ctx, int sys, const double* x, int n, double* u, void* stream);

/* Kernel profile of this process's library calls (CUDA events around each
 * launch of the main kernel families, on the stream the kernel runs on).
 * enable = 1 clears the counters and starts recording; enable = 0 stops,
 * waits for the recorded events and fills *out (may be NULL).  flops and
 * bytes are the algorithmic counts of the launches (complex line FFT:
 * 5 L log2 L flops; bytes: every input read and output written once). */
#define PDEP_PROFILE_CLASSES 17
typedef struct {
  char name[24];
  long long launches;
  double ms;
  double flops;
  double bytes;
} pdep_kernel_class;
typedef struct {
  long long launches; /* every kernel the library launched while recording */
  pdep_kernel_class cls[PDEP_PROFILE_CLASSES];
} pdep_profile_t;
int pdep_profile(int enable, pdep_profile_t* out);

/* Device status word.  Kernels OR condition bits into a per-context word
 * (non-finite CG scalar, CG breakdown, a solve that ended above cg_tol, a
 * spent clock budget, and in bounds-checked builds an index outside the
 * sphere tables).  pdep_sync_status synchronises 'stream', returns the
 * condition of the word (PDEP_OK, PDEP_ERR_NONFINITE, PDEP_ERR_BOUNDS,
 * PDEP_ERR_TIMEOUT or PDEP_ERR_NOT_CONVERGED, in that priority) for every
 * call enqueued since the last synchronising read, and clears it.
 * PDEP_ERR_INVALID_ARG for a NULL context. */
int pdep_sync_status(pdep_ctx* ctx, void* stream);

/* Statistics of the last chi0_apply, sternheimer_solve, pdep_solve or
 * pdep_chibar_apply on this context (*stats, host): synchronises 'stream',
 * reads the device-side counters (CG iterations, residuals, refinement
 * rounds, kernel launches) and returns the device status word's condition
 * (then cleared) as pdep_sync_status does.  dav_* fields are those of the
 * last pdep_solve. */
int pdep_get_stats(pdep_ctx* ctx, pdep_stats* stats, void* stream);

/* 1 if this library was compiled with -DPDEP_BOUNDS_CHECK (every index read
 * from the host-built sphere tables is tested before use in the transform
 * kernels), else 0. */
int pdep_bounds_checked(void);

void pdep_destroy(pdep_ctx* ctx);
const char* pdep_status_string(int status);
const char* pdep_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PDEP_H */
