// Dense linear algebra and vector kernels used by the Sternheimer CG, the
// Davidson iteration and the setup eigensolver.  All matrices are
// column-major; a block of vectors stored one per row of a [n][ld] array is
// the column-major ld x n matrix whose columns are the vectors.
#pragma once

#include <vector>

#include "common.cuh"
#include "df64.cuh"

namespace pdep {

// C[m x n] = alpha * op(A)[m x k] * B[k x n] + beta * C, op(A) = A^T if transA.
// Split over k (atomic accumulation) when the tile count is small.  Optional
// column maps: column j of B is B[:, bmap[j]] and column j of C is C[:, cmap[j]].
// ndev (optional): device count of the mapped columns (<= n); the launch is
// sized for n and columns from *ndev on are left untouched.  R is the
// arithmetic type: float, double, or df (double-float arithmetic on the FP32
// pipe; the matrices are FP64).
// shape (optional): tile height (tm 4: 64 rows, 5: 80 rows; 0 = the one that
// pads m less) and split-K multiplier of the default split (split_x8 / 8,
// 0 = default); the autotuner picks it per GEMM shape.
struct GemmShape {
  int tm = 0;
  int split_x8 = 0;
};
template <typename R>
cudaError_t gemm(bool transA, int m, int n, int k, double alpha, const typename Io<R>::T* A,
                 long long lda, const typename Io<R>::T* B, long long ldb, double beta,
                 typename Io<R>::T* C, long long ldc, cudaStream_t st, const int* bmap = nullptr,
                 const int* cmap = nullptr, const int* ndev = nullptr, GemmShape shape = {});

// Symmetric eigendecomposition of the n x n matrix M (lda), FP64:
// one-sided (Hestenes) Jacobi on M - sigma I (sigma = twice the Gershgorin
// bound, so the shifted matrix is negative definite and well conditioned);
// the eigenvectors are the normalised columns of the converged (M - sigma I) V,
// the eigenvalues their Rayleigh quotients with the original M, sorted
// ascending.  W [n] eigenvalues, V [n x n] (ldv) vectors.
// Work needs 2 n*n + 4 n doubles of device scratch.
// Executable graphs of one Jacobi sweep (its nn - 1 dependent rounds), keyed
// by the matrix size and the device buffers the rounds were captured with.
// Owned by the caller (one per context, so calls on different contexts never
// share it); release() destroys the graphs.
struct EighGraphCache {
  struct Entry {
    int n;
    const void* a;
    const void* counter;
    cudaGraphExec_t exec;
  };
  std::vector<Entry> entries;
  void release() {
    for (Entry& e : entries) cudaGraphExecDestroy(e.exec);
    entries.clear();
  }
};

struct EighWork {
  double* a;      // n*n
  double* v;      // n*n
  double* tmp;    // n*n
  double* w;      // n (unsorted)
  int* flag;      // 1 int + 1 unsigned (rotation counter)
  EighGraphCache* graphs = nullptr;  // sweeps replayed from graphs (null: plain launches)
};
cudaError_t eigh(int n, const double* M, long long ldm, double* W, double* V, long long ldv,
                 EighWork wk, cudaStream_t st, int max_sweeps = 40);

// elementwise and per-column helpers
template <typename R>
cudaError_t symmetrize(R* M, int n, long long ld, cudaStream_t st);
template <typename Rd, typename Rs>
cudaError_t convert(Rd* dst, long long ldd, const Rs* src, long long lds, int rows, int cols,
                    cudaStream_t st);
template <typename R>
cudaError_t col_norms(const R* X, long long ld, int rows, int cols, double* out, cudaStream_t st);
template <typename R>
cudaError_t scale_cols(R* X, long long ld, int rows, int cols, const double* s, int invert,
                       cudaStream_t st);
cudaError_t ritz_residual(const double* AX, const double* X, long long ld, int rows, int cols,
                          const double* theta, double* Rout, cudaStream_t st);
cudaError_t philox_normal(double* X, long long ld, int rows, int cols, unsigned long long seed,
                          unsigned long long offset, cudaStream_t st);
// X[d][j] *= sqrt(4 pi)/|G| on the 2 n_half PDEP components of n columns
cudaError_t scale_sqrt_coulomb(double* X, long long ld, int n_half, int n, const double* g2,
                               cudaStream_t st);
// Lanczos chains (Sec. II D), Q_k blocks [n][ld], alpha/beta [n][K]:
// q_0 = r/||r|| and beta[j][0] = ||r||; one three-term step per call; the
// tridiagonal eigen-decompositions (K <= 64; d ascending, U[j][m][k]); the
// omega-independent weights of Eq. MCfinal from G = L^T Q (n_L x (K n)) for
// the chains j cs + c0, j < n.
cudaError_t lanczos_start(const double* R, long long ld, int n_pw, int n, int K,
                          const double* r0norm, double* Q0, double* beta, cudaStream_t st);
cudaError_t lanczos_step(const double* W, const double* Qk, const double* Qkm1, double* Qk1,
                         long long ld, int n_pw, int n, int K, int k, double* alpha, double* beta,
                         cudaStream_t st);
cudaError_t tridiag_eig(const double* alpha, const double* beta, int n, int K, double* d,
                        double* U, cudaStream_t st);
cudaError_t lanczos_weights(const double* G, int n_L, int n, int K, const double* U,
                            const double* beta, double* weights, int cs, int c0,
                            cudaStream_t st);
// Body of chi0bar at imaginary frequencies from Lanczos chains (Eq. finalB):
// per-chain resolvent vectors z [n_freq][n][K] for occupied energy eps_v,
// their accumulation B[f] += scale G z, and Lambda = V diag(w/(1-w)) V^T.
cudaError_t lanczos_z(const double* U, const double* d, const double* beta, int n, int K, int cs,
                      int c0, double eps_v, const double* nu, int n_freq, double* z,
                      cudaStream_t st);
cudaError_t body_accum(const double* G, int n_L, int n, int K, const double* z, int n_freq,
                       double scale, double* B, cudaStream_t st);
cudaError_t lambda_from_eig(const double* V, const double* w, int n, double* L, cudaStream_t st);
// Column-wise dots X_j . Y_j; q = p - q; and the updates of a block of
// independent CG problems with per-column alpha and beta (device arrays):
// x += alpha p, r -= alpha q, then p = r + beta p.
cudaError_t pair_dots(const double* X, const double* Y, long long ld, int rows, int n, double* out,
                      cudaStream_t st);
cudaError_t one_minus(double* q, const double* p, long long ld, int rows, int n, cudaStream_t st);
cudaError_t block_cg_xr(double* x, double* r, const double* p, const double* q, long long ld,
                        int rows, int n, const double* alpha, cudaStream_t st);
cudaError_t block_cg_p(double* p, const double* r, long long ld, int rows, int n,
                       const double* beta, cudaStream_t st);
// W = L^{-T} for the Cholesky factor of the m x m Gram matrix G (m <= 128);
// *fail = 1 (device) when a pivot is at or below rel_thr * max_i G_ii.
cudaError_t cholesky_winv(const double* G, int m, double rel_thr, double* W, int* fail,
                          cudaStream_t st);
cudaError_t scale_by_isqrt_clamped(double* Q, long long ldq, int n, const double* d, double dmin,
                                   int* keep, cudaStream_t st);
cudaError_t fill_zero(void* p, size_t bytes, cudaStream_t st);

// Tensor-core (3xTF32, mma.sync) FP32 projections, all matrices column-major:
// S (M x N, lds) = diag(sigma) P^T X(:, bmap)      (K = rows of P and X)
// Y(:, cmap) (M x N) += P (M x K) S (K x N, lds)
// Rows of P, X, Y and S must start on 16-byte boundaries (ldp, ldx, lds
// multiples of 4 floats; aligned bases).
// ndev (optional): device count of the mapped columns (<= N).
cudaError_t tc_proj_coeffs(int M, int N, int K, const float* P, long long ldp, const float* X,
                           long long ldx, const int* bmap, const float* sigma, float* S,
                           long long lds, cudaStream_t st, const int* ndev = nullptr);
cudaError_t tc_proj_update(int M, int N, int K, const float* P, long long ldp, const float* S,
                           long long lds, float* Y, long long ldy, const int* cmap,
                           cudaStream_t st, const int* ndev = nullptr);

// The coefficients on the Blackwell tensor cores (tcgen05.mma kind::tf32
// into tensor memory, 3xTF32, every 32-wide K stage flushed to FP32
// registers; warp-specialised, one CTA per SM over equal shares of the
// work).  The states come as hi / lo tiles written once by tc5_split_states
// (tc5_split_floats(n_ext, K) floats, 16-byte aligned); X rows as above;
// the result is S[j][w] = sigma_w <w|x_bmap(j)> at S + j lds + w (lds >=
// n_ext, a multiple of 4).  A wait on the tensor cores or a copy that runs
// out (about a second) sets DEV_TIMEOUT in *status and leaves S incomplete.
size_t tc5_split_floats(int n_ext, int K);
cudaError_t tc5_split_states(int n_ext, int K, const float* P, long long ldp, float* Pt,
                             cudaStream_t st);
// bf16: the states as BF16 tiles (tc5_split_states_bf16, tc5_split_bytes_bf16
// bytes) and one BF16 product per k-step (PDEP_MIXED_BF16)
size_t tc5_split_bytes_bf16(int n_ext, int K);
cudaError_t tc5_split_states_bf16(int n_ext, int K, const float* P, long long ldp, void* Pt,
                                  cudaStream_t st);
cudaError_t tc5_proj_coeffs(int n_ext, int N, int K, const void* Pt, const float* X,
                            long long ldx, const int* bmap, const float* sigma, float* S,
                            long long lds, cudaStream_t st, const int* ndev, unsigned* status,
                            bool bf16 = false);

// Per-RHS preconditioned CG kernels (one CTA per RHS vector).
// State of one RHS: x, r, p (length n_pw, stride ld), scalars in CgScal.
struct CgScal {
  double rz;      // r . K r
  double bnorm;   // ||b||
  double rnorm;   // ||r||
  int iters;
  int active;     // 1 while unconverged
};
template <typename R>
struct CgArgs {
  R* x;
  R* r;
  R* p;
  const R* ap;
  long long ld;
  int n_pw;
  int n_half;
  int n_rhs;
  const R* kprec;       // preconditioner K(G) per occupied state, [n_occ][ld]
  int n_occ;            // rhs index i uses occupied state i % n_occ
  CgScal* sc;
  double tol;
  unsigned* status;
  int* n_active;        // counter (atomic) of RHS still active after the step
  int variant;          // CgVariant (picked by the autotuner)
  const int* list_count = nullptr;  // device length of the active list (cg_step sized for
                                    // the largest; blocks past it exit)
  const double* mask = nullptr;     // cg_start: RHS i takes part only if mask[i] != 0
  const double* tolv = nullptr;     // per-RHS relative tolerance (replaces tol when set)
};

// Device state of one Sternheimer CG loop (context-owned device memory).
// The loop runs on the device: a control kernel after every step decides
// whether another step follows (CUDA-graph while node, or a flag the host
// reads in the eager form).
struct CgLoopState {
  int active;                     // RHS still active after the last step (cg_step adds)
  int listed;                     // length of the compacted active list
  int iter;                       // steps done in this loop
  int go;                         // 1 while another step is due
  unsigned long long t0;          // %globaltimer (ns) at the loop start
  unsigned long long steps[2];    // steps over all loops (FP32, FP64), for launch counts
};
// Device statistics of the Sternheimer solves since the last reset.
struct DevStats {
  unsigned long long cg_iters;      // CG iterations summed over RHS (all rounds)
  unsigned long long max_res_bits;  // largest final relative FP64 residual (bits of a double >= 0)
  int cg_max;                       // largest per-RHS iteration count of one CG loop
  int refine_max;                   // largest refinement-round count of one solve
  int rounds_cur;                   // rounds with unconverged RHS in the current solve
  int pad;
};
// Loop control: begin (iter = 0, go = active > 0 && max_iter > 0) and the
// step after each CG step (iter += 1; go = active > 0 && iter < max_iter &&
// elapsed <= budget_ns; a spent budget with RHS still active sets
// DEV_TIMEOUT).  With a graph handle (has_handle) the decision also drives
// the enclosing while node.  prec selects the launch-count slot (0 FP32, 1 FP64).
cudaError_t loop_begin(CgLoopState* ls, int max_iter, cudaGraphConditionalHandle h, int has_handle,
                       cudaStream_t st);
cudaError_t loop_next(CgLoopState* ls, int max_iter, unsigned long long budget_ns,
                      unsigned* status, int prec, cudaGraphConditionalHandle h, int has_handle,
                      cudaStream_t st);
// After a CG loop: its_total[i] += sc[i].iters (its_total may be null), and
// the sum / largest count into ds.
cudaError_t cg_collect(const CgScal* sc, int n, int* its_total, DevStats* ds, cudaStream_t st);
// End of a solve: ds->max_res = max(ds->max_res, max_i rel[i]); any rel[i] > tol
// sets DEV_NOT_CONVERGED; ds->refine_max = max(refine_max, rounds_cur).
cudaError_t solve_finish(const double* rel, int n, double tol, DevStats* ds, unsigned* status,
                         cudaStream_t st);
// launch shapes of one CG step: register-cached (the RHS read once) or
// streaming (three passes, more RHS resident per SM)
enum CgVariant : int {
  CG_REG256 = 0,
  CG_REG512 = 1,
  CG_STREAM128 = 2,
  CG_STREAM256 = 3,
  CG_STREAM512 = 4,
  CG_NUM_VARIANTS = 5
};
template <typename R>
cudaError_t cg_start(const CgArgs<R>& a, const R* b, long long ldb, cudaStream_t st);
// one PCG step for the n_list RHS of list (all n_rhs when list is null)
template <typename R>
cudaError_t cg_step(const CgArgs<R>& a, const int* list, int n_list, cudaStream_t st);
// K[v][j] = Teter-Payne-Allan K(|G_j|^2/2 / ekin[v]) (1 at G = 0), FP64 and FP32 copies
cudaError_t build_precond(const double* g2, int n_half, int n_pw, const double* ekin, int n_occ,
                          double* k64, float* k32, long long ld, cudaStream_t st);

// Ordered list of the RHS with sc[i].active (list[0..count)), one block.
cudaError_t active_list(const CgScal* sc, int n, int* list, int* count, cudaStream_t st);
// Ordered list of i with rel[i] > tol; a non-empty list adds 1 to *rounds
// (may be null).
cudaError_t unconverged_list(const double* rel, double tol, int n, int* list, int* count,
                             cudaStream_t st, int* rounds = nullptr);
// Ordered active list as active_list, also zeroing *reset (the step counter
// cg_step accumulates into).
cudaError_t active_list_reset(const CgScal* sc, int n, int* list, int* count, int* reset,
                              cudaStream_t st);

// Refinement rounds: for i with rel[i] > tol, rn[i] = ||r64_i|| and ri_i =
// r64_i / rn[i] in the inner precision Ri (float or double); otherwise rn[i]
// = 0 and ri_i is left as it is.  tolv (optional): tolv[i] = min(inner_cap,
// target / rel[i]), the relative tolerance that brings the FP64 residual to
// target x ||b_i||.
template <typename Ri>
cudaError_t refine_prepare(const double* r64, long long ld64, int n_pw, int n, const double* rel,
                           double tol, Ri* ri, long long ldi, double* rn, cudaStream_t st,
                           double* tolv = nullptr, double target = 0.0, double inner_cap = 0.0);
// x64_i += rn[i] * d32_i
cudaError_t refine_accumulate(double* x64, long long ld64, const float* d32, long long ld32,
                              int n_pw, int n, const double* rn, cudaStream_t st);

// Refinement update in FP64: delta_i = rn_i d_i (+ xd_i), x_i += delta_i,
// dl_i = delta_i (and dlf_i = fl32(delta_i) when dlf is given, stride ld);
// with d = null, delta_i = x_i + xd_i and x_i = delta_i.
template <typename Ri>
cudaError_t refine_delta(double* x, double* dl, long long ld, const Ri* d, long long ldd,
                         int n_pw, int n, const double* rn, const double* xd, cudaStream_t st,
                         float* dlf = nullptr);
// r_i -= ad_i (+ sv[i % n_occ] xd_i) in FP64, ad in FP64 or FP32;
// rel_i = ||r_i|| / ||b_i|| (listed vectors; ndev: device length of the
// list, <= n)
template <typename Ta>
cudaError_t residual_update(double* r, const Ta* ad, const double* b, long long ld, int n_pw,
                            int n, double* rel, const int* list, const double* xd,
                            const double* sv, int n_occ, cudaStream_t st,
                            const int* ndev = nullptr);
// rel[i] = v for i < n
cudaError_t fill_value(double* rel, int n, double v, cudaStream_t st);
// Kinetic energy sum_k |G_k|^2/2 (x_2k^2 + x_2k+1^2) of each column.
cudaError_t kinetic_energy(const double* X, long long ld, int n_half, int n, const double* g2,
                           double* out, cudaStream_t st);
// T_i <- K(|G|^2/2 / E_i) T_i with the Teter-Payne-Allan K.
cudaError_t precondition_tpa(double* T, long long ld, int n_pw, int n_half, int n,
                             const double* g2, const double* ekin, cudaStream_t st);
// Y[:, i] = X[:, idx[i]]
cudaError_t gather_cols(const double* X, long long ldx, double* Y, long long ldy, int rows,
                        const int* idx, int n, cudaStream_t st);
// X[comp[i], i] = 1 plus amp * Philox normal noise on every component
cudaError_t unit_start(double* X, long long ld, int rows, const int* comp, int n, double amp,
                       unsigned long long seed, cudaStream_t st);
// Chebyshev filter step: Ynew = a1 * (HY - c Y) + b1 * X  (n columns, rows entries)
cudaError_t cheb_step(double* Ynew, const double* HY, const double* Y, const double* X,
                      long long ld, int rows, int n, double a1, double c, double b1,
                      cudaStream_t st);
// S[n_occ + c, i] /= (eps[n_occ + c] - eps[i % n_occ]) for c < n_defl, i < n
// (S column-major with leading dimension lds)
cudaError_t deflation_coefficients(double* S, int lds, int n_occ, int n_defl, int n,
                                   const double* eps, cudaStream_t st);
// S[w, i] *= sigma[w] for w < rows, i < n (S column-major, leading dimension lds)
template <typename R>
cudaError_t scale_rows(R* S, int lds, int rows, int n, const R* sigma, cudaStream_t st);
// X[row, i] = 0 for every column i (e.g. the G = 0 slot of PDEP vectors)
cudaError_t zero_row(double* X, long long ld, int row, int n, cudaStream_t st);

}  // namespace pdep
