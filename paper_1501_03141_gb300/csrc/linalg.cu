// Dense linear algebra, vector and CG kernels (see linalg.cuh).
#include <type_traits>

#include "linalg.cuh"
#include "profile.cuh"

#include <vector>

namespace pdep {

static int num_sms() {
  // queried once (thread-safe static initialisation); 152 on GB300
  static const int n = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 152;
  }();
  return n;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of up to two doubles; warp 0 finishes, every thread gets the result
__device__ __forceinline__ double2 block_sum2(double a, double b) {
  __shared__ double sa[32], sb[32];
  __shared__ double2 res;
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double x = l < nw ? sa[l] : 0.0, y = l < nw ? sb[l] : 0.0;
    x = warp_sum(x);
    y = warp_sum(y);
    if (l == 0) res = make_double2(x, y);
  }
  __syncthreads();
  return res;
}

// Block sum of two values: warp sums in the callers' precision R, the
// per-warp partials summed in FP64 by warp 0 only.  Result in shared memory,
// valid for every thread after the call.
template <typename R>
__device__ __forceinline__ double2 block_sum2_r(R a, R b) {
  __shared__ double sa[32], sb[32];
  __shared__ double2 res;
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sa[w] = (double)a;
    sb[w] = (double)b;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double x = l < nw ? sa[l] : 0.0, y = l < nw ? sb[l] : 0.0;
    x = warp_sum(x);
    y = warp_sum(y);
    if (l == 0) res = make_double2(x, y);
  }
  __syncthreads();
  return res;
}

// ---------------------------------------------------------------------------
// GEMM (SIMT, register-tiled 64x64x16)
// ---------------------------------------------------------------------------
// C tile of (16 TM) x 64 per CTA of 256 threads (16 x 16, each thread TM x 4
// outputs), K tiles of 16 staged in shared memory.  TM = 5 gives 80-row tiles
// for the 80-state projection coefficients (n_occ + n_deflate on the 48^3
// workload), which 64-row tiles would cover with 37% padding.
// R: arithmetic type (float, double, or df: double-float on FP64 matrices);
// matrices are stored in Io<R>::T.
template <typename R, bool TA, int TM>
__global__ void __launch_bounds__(256) k_gemm(int m, int n, int k, R alpha,
                                              const typename Io<R>::T* __restrict__ A,
                                              long long lda, const typename Io<R>::T* __restrict__ B,
                                              long long ldb, R beta, typename Io<R>::T* __restrict__ C,
                                              long long ldc, int kchunk,
                                              int atomic, const int* __restrict__ bmap,
                                              const int* __restrict__ cmap,
                                              const int* __restrict__ ndev, int has_beta) {
  constexpr int BM = 16 * TM, BN = 64, BK = 16;
  __shared__ R As[BK][BM + 1];
  __shared__ R Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  if (ndev) n = min(n, *ndev);  // device count of the mapped columns
  if (col0 >= n) return;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(k, kbeg + kchunk);
  R acc[TM][4];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = R(0);

  for (int kb = kbeg; kb < kend; kb += BK) {
#pragma unroll
    for (int q = 0; q < TM; ++q) {
      const int e = tid + 256 * q;
      if (TA) {
        // A is k x m: consecutive threads read consecutive k of one row
        const int i = e >> 4, kk = e & 15;
        const int gi = row0 + i, gk = kb + kk;
        As[kk][i] = (gi < m && gk < kend) ? R(A[gk + (long long)gi * lda]) : R(0);
      } else {
        const int i = e % BM, kk = e / BM;
        const int gi = row0 + i, gk = kb + kk;
        As[kk][i] = (gi < m && gk < kend) ? R(A[gi + (long long)gk * lda]) : R(0);
      }
    }
    {
      const int j = tid >> 2, kk0 = (tid & 3) * 4;
      const int gj = col0 + j;
      const long long bc = gj < n ? (long long)(bmap ? bmap[gj] : gj) * ldb : 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gk = kb + kk0 + q;
        Bs[kk0 + q][j] = (gj < n && gk < kend) ? R(B[gk + bc]) : R(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R av[TM], bv[4];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mad(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int gi = row0 + tx + 16 * a;
    if (gi >= m) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = col0 + ty + 16 * b;
      if (gj >= n) continue;
      typename Io<R>::T* c = C + gi + (long long)(cmap ? cmap[gj] : gj) * ldc;
      if (atomic) {
        atomicAdd(c, io_of<R>(alpha * acc[a][b]));
      } else {
        R v = alpha * acc[a][b];
        if (has_beta) v += beta * R(*c);
        *c = io_of<R>(v);
      }
    }
  }
}

template <typename R>
__global__ void k_scale_mat(R* C, long long ldc, int m, int n, R beta, const int* cmap,
                            const int* ndev) {
  if (ndev) n = min(n, *ndev);
  const long long tot = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    R* c = C + i + (long long)(cmap ? cmap[j] : j) * ldc;
    *c = beta == R(0) ? R(0) : beta * *c;
  }
}

template <typename R>
cudaError_t gemm(bool transA, int m, int n, int k, double alpha, const typename Io<R>::T* A,
                 long long lda, const typename Io<R>::T* B, long long ldb, double beta,
                 typename Io<R>::T* C, long long ldc, cudaStream_t st, const int* bmap,
                 const int* cmap, const int* ndev, GemmShape shape) {
  using T = typename Io<R>::T;
  if (m <= 0 || n <= 0) return cudaSuccess;
  // 80-row tiles when they pad m less than 64-row tiles do (or as tuned)
  const bool t80 = shape.tm ? shape.tm == 5 : ((m + 79) / 80) * 80 < ((m + 63) / 64) * 64;
  const int bm = t80 ? 80 : 64;
  const int tm = (m + bm - 1) / bm, tn = (n + 63) / 64;
  int splits = 1;
  const long long tiles = (long long)tm * tn;
  if (tiles < 2LL * num_sms() && k > 256) {
    splits = (int)((2LL * num_sms() + tiles - 1) / tiles);
    splits = std::min(splits, (k + 255) / 256);
    splits = std::max(splits, 1);
  }
  if (shape.split_x8 > 0 && k > 256)
    splits = std::max(1, std::min((k + 127) / 128, (splits * shape.split_x8 + 7) / 8));
  int kchunk = (k + splits - 1) / splits;
  kchunk = ((kchunk + 15) / 16) * 16;
  if (kchunk == 0) kchunk = 16;
  splits = std::max(1, (k + kchunk - 1) / kchunk);
  if (k <= 0) splits = 1;
  int atomic = 0;
  if (splits > 1 || k <= 0) {
    const long long tot = (long long)m * n;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
    count_launch();
    k_scale_mat<T><<<blocks, 256, 0, st>>>(C, ldc, m, n, (T)beta, cmap, ndev);
    if (k <= 0) return cudaGetLastError();
    atomic = 1;
  }
  dim3 grid(tm, tn, splits);
  ProfScope ps(std::is_same<R, df>::value ? PC_GEMM_DF : sizeof(R) == 8 ? PC_GEMM_F64 : PC_GEMM_F32,
               st, 2.0 * m * n * (double)k,
               ((double)m * k + (double)k * n + (beta != 0.0 ? 2.0 : 1.0) * m * n) * sizeof(T),
               ndev, n);
  count_launch();
  const R al = R(alpha), be = R(beta);
  const int hb = beta != 0.0 ? 1 : 0;
  if (transA) {
    if (t80)
      k_gemm<R, true, 5><<<grid, 256, 0, st>>>(m, n, k, al, A, lda, B, ldb, be, C, ldc, kchunk,
                                               atomic, bmap, cmap, ndev, hb);
    else
      k_gemm<R, true, 4><<<grid, 256, 0, st>>>(m, n, k, al, A, lda, B, ldb, be, C, ldc, kchunk,
                                               atomic, bmap, cmap, ndev, hb);
  } else {
    if (t80)
      k_gemm<R, false, 5><<<grid, 256, 0, st>>>(m, n, k, al, A, lda, B, ldb, be, C, ldc, kchunk,
                                                atomic, bmap, cmap, ndev, hb);
    else
      k_gemm<R, false, 4><<<grid, 256, 0, st>>>(m, n, k, al, A, lda, B, ldb, be, C, ldc, kchunk,
                                                atomic, bmap, cmap, ndev, hb);
  }
  return cudaGetLastError();
}

template cudaError_t gemm<double>(bool, int, int, int, double, const double*, long long,
                                  const double*, long long, double, double*, long long,
                                  cudaStream_t, const int*, const int*, const int*, GemmShape);
template cudaError_t gemm<df>(bool, int, int, int, double, const double*, long long,
                              const double*, long long, double, double*, long long, cudaStream_t,
                              const int*, const int*, const int*, GemmShape);
template cudaError_t gemm<float>(bool, int, int, int, double, const float*, long long,
                                 const float*, long long, double, float*, long long, cudaStream_t,
                                 const int*, const int*, const int*, GemmShape);

// ---------------------------------------------------------------------------
// one-sided Jacobi eigensolver
// ---------------------------------------------------------------------------
__global__ void k_gershgorin(const double* __restrict__ M, long long ldm, int n, double* out) {
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += fabs(M[i + (long long)j * ldm]);
    mx = fmax(mx, s);
  }
  __shared__ double sm[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) m2 = fmax(m2, sm[w]);
    // twice the Gershgorin bound: M - sigma I is negative definite with every
    // |lambda_i - sigma| in [sigma/2, 3 sigma/2]
    *out = m2 > 0.0 ? 2.0 * m2 * (1.0 + 1e-3) : 1.0;
  }
}

__global__ void k_jacobi_init(const double* __restrict__ M, long long ldm, int n,
                              const double* __restrict__ sigma, double* A) {
  const long long tot = (long long)n * n;
  const double s = *sigma;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    double m = 0.5 * (M[i + (long long)j * ldm] + M[j + (long long)i * ldm]);
    A[e] = (i == j) ? m - s : m;
  }
}

// One round of the cyclic (round-robin) ordering, one CTA of two warps per
// column pair (p, q): the pair is rotated so that A_p . A_q = 0.  V is not
// carried: at convergence the columns of A = (M - sigma I) V are the
// eigenvectors scaled by lambda_i - sigma, and with sigma twice the
// Gershgorin bound every |lambda_i - sigma| lies in [sigma/2, 3 sigma/2]
// (condition number at most 3), so normalising them gives V to working
// accuracy.  E > 0: the
// two columns (n <= 64 E) are held in registers, one memory round trip per
// round; E = 0 streams them.
template <int E>
__global__ void __launch_bounds__(64) k_jacobi_pair(double* A, int n, int nn, int round,
                                                    unsigned* counter) {
  const int pair = blockIdx.x;
  int p, q;
  if (pair == 0) {
    p = nn - 1;
    q = round;
  } else {
    p = (round + pair) % (nn - 1);
    q = (round - pair + (nn - 1)) % (nn - 1);
  }
  if (p >= n || q >= n) return;
  double* ap = A + (long long)p * n;
  double* aq = A + (long long)q * n;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  __shared__ double red[2][3];
  double al = 0.0, be = 0.0, ga = 0.0;
  double x[E > 0 ? E : 1], y[E > 0 ? E : 1];
  if constexpr (E > 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int r = t + 64 * e;
      const bool in = r < n;
      x[e] = in ? ap[r] : 0.0;
      y[e] = in ? aq[r] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      al += x[e] * x[e];
      be += y[e] * y[e];
      ga += x[e] * y[e];
    }
  } else {
    for (int r = t; r < n; r += 64) {
      const double u = ap[r], w = aq[r];
      al += u * u;
      be += w * w;
      ga += u * w;
    }
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  if (lane == 0) {
    red[warp][0] = al;
    red[warp][1] = be;
    red[warp][2] = ga;
  }
  __syncthreads();
  al = red[0][0] + red[1][0];
  be = red[0][1] + red[1][1];
  ga = red[0][2] + red[1][2];
  // every thread holds the same sums, so this exit is uniform
  if (ga == 0.0 || ga * ga <= 1e-28 * (al * be)) return;
  const double zeta = (be - al) / (2.0 * ga);
  const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = rsqrt(1.0 + tt * tt);
  const double s = c * tt;
  if constexpr (E > 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int r = t + 64 * e;
      if (r < n) {
        ap[r] = c * x[e] - s * y[e];
        aq[r] = s * x[e] + c * y[e];
      }
    }
  } else {
    for (int r = t; r < n; r += 64) {
      const double u = ap[r], w = aq[r];
      ap[r] = c * u - s * w;
      aq[r] = s * u + c * w;
    }
  }
  if (t == 0) atomicAdd(counter, 1u);
}

using JacobiRound = void (*)(double*, int, int, int, unsigned*);
static JacobiRound jacobi_round_for(int n) {
  if (n <= 128) return k_jacobi_pair<2>;
  if (n <= 256) return k_jacobi_pair<4>;
  if (n <= 512) return k_jacobi_pair<8>;
  return k_jacobi_pair<0>;
}

// V_i = -A_i / ||A_i|| (one block per column)
__global__ void k_jacobi_vectors(const double* __restrict__ A, int n, double* V) {
  const int c = blockIdx.x;
  double ss = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double a = A[r + (long long)c * n];
    ss += a * a;
  }
  const double2 t = block_sum2(ss, 0.0);
  const double f = t.x > 0.0 ? -rsqrt(t.x) : 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    V[r + (long long)c * n] = f * A[r + (long long)c * n];
}

// w_i = v_i . (M v_i)
__global__ void k_col_dots(const double* __restrict__ V, const double* __restrict__ MV, int n,
                           double* w) {
  const int c = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    s += V[r + (long long)c * n] * MV[r + (long long)c * n];
  double2 t = block_sum2(s, 0.0);
  if (threadIdx.x == 0) w[c] = t.x;
}

// rank sort (ascending, stable) and column permutation
__global__ void k_sort_ranks(const double* __restrict__ w, int n, int* rank) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double wi = w[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const double wj = w[j];
      r += (wj < wi || (wj == wi && j < i)) ? 1 : 0;
    }
    rank[i] = r;
  }
}
__global__ void k_permute(const double* __restrict__ w, const double* __restrict__ V, int n,
                          const int* __restrict__ rank, double* W, double* Vout, long long ldv) {
  const int c = blockIdx.x;
  const int rc = rank[c];
  if (threadIdx.x == 0) W[rc] = w[c];
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    Vout[r + (long long)rc * ldv] = V[r + (long long)c * n];
}

cudaError_t eigh(int n, const double* M, long long ldm, double* W, double* V, long long ldv,
                 EighWork wk, cudaStream_t st, int max_sweeps) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps(PC_EIGH, st, 0.0, 0.0);
  double* sigma = wk.w;  // reuse w[0] for the shift; overwritten later
  unsigned* counter = reinterpret_cast<unsigned*>(wk.flag + 1);
  count_launch();
  k_gershgorin<<<1, 256, 0, st>>>(M, ldm, n, sigma);
  const long long tot = (long long)n * n;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  count_launch();
  k_jacobi_init<<<blocks, 256, 0, st>>>(M, ldm, n, sigma, wk.a);
  const int nn = n + (n & 1);
  const int jb = nn / 2;  // one CTA per column pair
  const int tpb = 64;
  const JacobiRound round_k = jacobi_round_for(n);
  // One sweep = nn - 1 dependent rounds; they are replayed from a CUDA graph
  // captured once per (size, buffers) to avoid nn - 1 stream launches.
  cudaGraphExec_t sweep = nullptr;
  if (nn - 1 > 8 && wk.graphs) {
    for (const EighGraphCache::Entry& k : wk.graphs->entries)
      if (k.n == n && k.a == wk.a && k.counter == counter) sweep = k.exec;
    if (!sweep) {
      cudaStream_t cap;
      cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int r = 0; r < nn - 1; ++r) round_k<<<jb, tpb, 0, cap>>>(wk.a, n, nn, r, counter);
        e = cudaStreamEndCapture(cap, &g);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&sweep, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cap);
      if (e != cudaSuccess) return e;
      wk.graphs->entries.push_back(EighGraphCache::Entry{n, wk.a, counter, sweep});
    }
  }
  unsigned hcount = 1;
  for (int sweep_i = 0; sweep_i < max_sweeps && hcount != 0; ++sweep_i) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (sweep) {
      for (int r = 0; r < nn - 1; ++r) count_launch();
      e = cudaGraphLaunch(sweep, st);
      if (e != cudaSuccess) return e;
    } else {
      for (int r = 0; r < nn - 1; ++r) {
        count_launch();
        round_k<<<jb, tpb, 0, st>>>(wk.a, n, nn, r, counter);
      }
    }
    if (nn - 1 == 0) break;
    e = cudaMemcpyAsync(&hcount, counter, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
  }
  { count_launch(); k_jacobi_vectors<<<n, 128, 0, st>>>(wk.a, n, wk.v); }
  // Rayleigh quotients with the original (symmetrised) matrix
  cudaError_t e = gemm<double>(false, n, n, n, 1.0, M, ldm, wk.v, n, 0.0, wk.tmp, n, st);
  if (e != cudaSuccess) return e;
  { count_launch(); k_col_dots<<<n, 128, 0, st>>>(wk.v, wk.tmp, n, wk.w); }
  int* rank = reinterpret_cast<int*>(wk.tmp);  // tmp no longer needed
  count_launch();
  k_sort_ranks<<<(n + 127) / 128, 128, 0, st>>>(wk.w, n, rank);
  count_launch();
  k_permute<<<n, 128, 0, st>>>(wk.w, wk.v, n, rank, W, V, ldv);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_symmetrize(R* M, int n, long long ld) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) {
      R a = M[i + (long long)j * ld], b = M[j + (long long)i * ld];
      R s = R(0.5) * (a + b);
      M[i + (long long)j * ld] = s;
      M[j + (long long)i * ld] = s;
    }
  }
}
template <typename R>
cudaError_t symmetrize(R* M, int n, long long ld, cudaStream_t st) {
  const long long tot = (long long)n * n;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((tot + 255) / 256, 4096));
  count_launch();
  k_symmetrize<R><<<blocks, 256, 0, st>>>(M, n, ld);
  return cudaGetLastError();
}
template cudaError_t symmetrize<double>(double*, int, long long, cudaStream_t);

template <typename Rd, typename Rs>
__global__ void k_convert(Rd* dst, long long ldd, const Rs* __restrict__ src, long long lds,
                          int rows, int cols) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % rows), c = (int)(e / rows);
    dst[r + (long long)c * ldd] = (Rd)src[r + (long long)c * lds];
  }
}
template <typename Rd, typename Rs>
cudaError_t convert(Rd* dst, long long ldd, const Rs* src, long long lds, int rows, int cols,
                    cudaStream_t st) {
  const long long tot = (long long)rows * cols;
  if (tot == 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 8192);
  count_launch();
  k_convert<Rd, Rs><<<blocks, 256, 0, st>>>(dst, ldd, src, lds, rows, cols);
  return cudaGetLastError();
}
template cudaError_t convert<double, double>(double*, long long, const double*, long long, int, int,
                                             cudaStream_t);
template cudaError_t convert<float, double>(float*, long long, const double*, long long, int, int,
                                            cudaStream_t);
template cudaError_t convert<df, double>(df*, long long, const double*, long long, int, int,
                                         cudaStream_t);
template cudaError_t convert<double, float>(double*, long long, const float*, long long, int, int,
                                            cudaStream_t);

template <typename R>
__global__ void k_col_norms(const R* __restrict__ X, long long ld, int rows, double* out) {
  const int c = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const double v = (double)X[r + (long long)c * ld];
    s += v * v;
  }
  double2 t = block_sum2(s, 0.0);
  if (threadIdx.x == 0) out[c] = sqrt(t.x);
}
template <typename R>
cudaError_t col_norms(const R* X, long long ld, int rows, int cols, double* out, cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  { count_launch(); k_col_norms<R><<<cols, 256, 0, st>>>(X, ld, rows, out); }
  return cudaGetLastError();
}
template cudaError_t col_norms<double>(const double*, long long, int, int, double*, cudaStream_t);
template cudaError_t col_norms<float>(const float*, long long, int, int, double*, cudaStream_t);

template <typename R>
__global__ void k_scale_cols(R* X, long long ld, int rows, const double* __restrict__ s, int inv) {
  const int c = blockIdx.x;
  double f = s[c];
  if (inv) f = f != 0.0 ? 1.0 / f : 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) X[r + (long long)c * ld] *= (R)f;
}
template <typename R>
cudaError_t scale_cols(R* X, long long ld, int rows, int cols, const double* s, int invert,
                       cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  { count_launch(); k_scale_cols<R><<<cols, 256, 0, st>>>(X, ld, rows, s, invert); }
  return cudaGetLastError();
}
template cudaError_t scale_cols<double>(double*, long long, int, int, const double*, int,
                                        cudaStream_t);
template cudaError_t scale_cols<float>(float*, long long, int, int, const double*, int,
                                       cudaStream_t);

__global__ void k_ritz_residual(const double* __restrict__ AX, const double* __restrict__ X,
                                long long ld, int rows, const double* __restrict__ th, double* Rr) {
  const int c = blockIdx.x;
  const double t = th[c];
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const long long e = r + (long long)c * ld;
    Rr[e] = AX[e] - t * X[e];
  }
}
cudaError_t ritz_residual(const double* AX, const double* X, long long ld, int rows, int cols,
                          const double* theta, double* Rout, cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  { count_launch(); k_ritz_residual<<<cols, 256, 0, st>>>(AX, X, ld, rows, theta, Rout); }
  return cudaGetLastError();
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller
__device__ __forceinline__ void philox_round(uint32_t (&c)[4], const uint32_t (&k)[2]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
  const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}
__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
  uint32_t k[2] = {k0, k1};
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
}
__global__ void k_philox_normal(double* X, long long ld, int rows, int cols,
                                unsigned long long seed, unsigned long long offset) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const unsigned long long ctr = offset + (unsigned long long)e;
    uint32_t c[4] = {(uint32_t)ctr, (uint32_t)(ctr >> 32), 0u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned long long a = ((unsigned long long)c[0] << 21) ^ (c[1] >> 11);  // 53 bits
    const unsigned long long b = ((unsigned long long)c[2] << 21) ^ (c[3] >> 11);
    const double u1 = ((double)(a & ((1ULL << 53) - 1)) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(b & ((1ULL << 53) - 1)) * (1.0 / 9007199254740992.0);
    const int r = (int)(e % rows), cc = (int)(e / rows);
    X[r + (long long)cc * ld] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}
cudaError_t philox_normal(double* X, long long ld, int rows, int cols, unsigned long long seed,
                          unsigned long long offset, cudaStream_t st) {
  const long long tot = (long long)rows * cols;
  if (tot == 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 8192);
  count_launch();
  k_philox_normal<<<blocks, 256, 0, st>>>(X, ld, rows, cols, seed, offset);
  return cudaGetLastError();
}

__global__ void k_isqrt_clamped(double* Q, long long ldq, int n, const double* __restrict__ d,
                                double dmin, int* keep) {
  const int c = blockIdx.x;
  const double dv = d[c];
  const bool k = dv > dmin;
  const double f = k ? 1.0 / sqrt(dv) : 0.0;
  if (threadIdx.x == 0 && keep) keep[c] = k ? 1 : 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) Q[r + (long long)c * ldq] *= f;
}
cudaError_t scale_by_isqrt_clamped(double* Q, long long ldq, int n, const double* d, double dmin,
                                   int* keep, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_isqrt_clamped<<<n, 128, 0, st>>>(Q, ldq, n, d, dmin, keep); }
  return cudaGetLastError();
}

// Cholesky factor G = L L^T of an m x m Gram matrix (column-major, m <= 128)
// in shared memory, then W = L^{-T} (upper triangular, column-major m x m):
// the columns of S W are orthonormal when G = S^T S.  A pivot at or below
// rel_thr * max_i G_ii leaves W unset and sets *fail = 1.
constexpr int kCholMax = 128;
__global__ void __launch_bounds__(512) k_chol_winv(const double* __restrict__ G, int m,
                                                   double rel_thr, double* W, int* fail) {
  extern __shared__ __align__(16) double sh[];
  const int ld = m + 1;  // odd row stride: column-wise walks hit distinct banks
  double* L = sh;        // row-major, lower triangle = L; upper = rows of L^{-1}^T
  double* dinv = sh + (size_t)m * ld;
  __shared__ int s_fail;
  __shared__ double s_gmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, j = e / m;
    L[i * ld + j] = G[e];
  }
  __syncthreads();
  if (tid == 0) {
    double g = 0.0;
    for (int i = 0; i < m; ++i) g = fmax(g, L[i * ld + i]);
    s_gmax = g;
    s_fail = !(g > 0.0) || !isfinite(g);
  }
  __syncthreads();
  const double thr = rel_thr * s_gmax;
  for (int k = 0; k < m && !s_fail; ++k) {
    if (tid == 0) {
      const double d = L[k * ld + k];
      if (d > thr && isfinite(d)) {
        L[k * ld + k] = sqrt(d);
      } else {
        s_fail = 1;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double piv = L[k * ld + k];
    for (int i = k + 1 + tid; i < m; i += nt) L[i * ld + k] /= piv;
    __syncthreads();
    const int w = m - k - 1;
    for (int e = tid; e < w * w; e += nt) {
      const int i = k + 1 + e / w, j = k + 1 + e % w;
      if (j <= i) L[i * ld + j] -= L[i * ld + k] * L[j * ld + k];
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) *fail = 1;
    return;
  }
  // X = L^{-1} by forward substitution, one column j per thread; X[i][j]
  // (i > j) is kept at L[j * ld + i], the unused upper triangle.
  if (tid < m) {
    const int j = tid;
    dinv[j] = 1.0 / L[j * ld + j];
    for (int i = j + 1; i < m; ++i) {
      double acc = L[i * ld + j] * dinv[j];
      for (int k = j + 1; k < i; ++k) acc += L[i * ld + k] * L[j * ld + k];
      L[j * ld + i] = -acc / L[i * ld + i];
    }
  }
  __syncthreads();
  // W = X^T: W[r][c] = X[c][r], nonzero for r <= c
  for (int e = tid; e < m * m; e += nt) {
    const int r = e % m, c = e / m;
    W[e] = r < c ? L[r * ld + c] : (r == c ? dinv[r] : 0.0);
  }
  if (tid == 0) *fail = 0;
}

cudaError_t cholesky_winv(const double* G, int m, double rel_thr, double* W, int* fail,
                          cudaStream_t st) {
  if (m <= 0 || m > kCholMax) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * ((size_t)m * (m + 1) + m);
  cudaError_t e = cudaFuncSetAttribute(k_chol_winv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * (kCholMax * (kCholMax + 1) + kCholMax)));
  if (e != cudaSuccess) return e;
  count_launch();
  k_chol_winv<<<1, 512, smem, st>>>(G, m, rel_thr, W, fail);
  return cudaGetLastError();
}

// X[d][j] *= sqrt(4 pi / |G_{d/2}|^2) for the 2 n_half PDEP components d
// (v^{1/2} of Eq. symmoperator on the real-coefficient layout)
__global__ void k_sqrt_coulomb(double* X, long long ld, int n_half, int n,
                               const double* __restrict__ g2) {
  const int j = blockIdx.y;
  const int dim = 2 * n_half;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < dim; d += gridDim.x * blockDim.x)
    X[d + (long long)j * ld] *= sqrt(4.0 * 3.14159265358979323846 / g2[d >> 1]);
}
cudaError_t scale_sqrt_coulomb(double* X, long long ld, int n_half, int n, const double* g2,
                               cudaStream_t st) {
  if (n <= 0 || n_half <= 0) return cudaSuccess;
  const int bx = std::min((2 * n_half + 255) / 256, 64);
  for (int j0 = 0; j0 < n; j0 += 65535) {
    const int nj = std::min(65535, n - j0);
    count_launch();
    k_sqrt_coulomb<<<dim3(bx, nj), 256, 0, st>>>(X + (long long)j0 * ld, ld, n_half, nj, g2);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lanczos chains of the deflated Hamiltonian (Sec. II D), one block per chain
// ---------------------------------------------------------------------------
// q_0 = r / ||r||, beta[j][0] = ||r|| (r already projected with P_c); a
// start vector whose projection is at or below 1e-12 of its norm before the
// projection (r0norm) gives an empty chain
__global__ void k_lanczos_start(const double* __restrict__ R, long long ld, int n_pw, int K,
                                const double* __restrict__ r0norm, double* Q0, double* beta) {
  const int j = blockIdx.x;
  const double* r = R + (long long)j * ld;
  double ss = 0.0;
  for (int i = threadIdx.x; i < n_pw; i += blockDim.x) ss += r[i] * r[i];
  double b = sqrt(block_sum2(ss, 0.0).x);
  if (!(b > 1e-12 * r0norm[j])) b = 0.0;
  const double f = b > 0.0 ? 1.0 / b : 0.0;
  double* q = Q0 + (long long)j * ld;
  for (int i = threadIdx.x; i < n_pw; i += blockDim.x) q[i] = f * r[i];
  if (threadIdx.x == 0) beta[(long long)j * K] = b;
}
cudaError_t lanczos_start(const double* R, long long ld, int n_pw, int n, int K,
                          const double* r0norm, double* Q0, double* beta, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_lanczos_start<<<n, 256, 0, st>>>(R, ld, n_pw, K, r0norm, Q0, beta); }
  return cudaGetLastError();
}

// Step k of every chain: W = H~ q_k on entry.  alpha_k = q_k . W,
// r = W - alpha_k q_k - beta_k q_{k-1}; unless k is the last step,
// beta_{k+1} = ||r|| and q_{k+1} = r / beta_{k+1}, or 0 and 0 when
// ||r|| <= 1e-12 ||W|| (an invariant subspace: the chain stops there).
__global__ void k_lanczos_step(const double* __restrict__ W, const double* __restrict__ Qk,
                               const double* __restrict__ Qkm1, double* Qk1, long long ld,
                               int n_pw, int K, int k, double* alpha, double* beta) {
  const int j = blockIdx.x;
  const long long o = (long long)j * ld;
  double aw = 0.0, ww = 0.0;
  for (int i = threadIdx.x; i < n_pw; i += blockDim.x) {
    const double w = W[o + i];
    aw += Qk[o + i] * w;
    ww += w * w;
  }
  const double2 t = block_sum2(aw, ww);
  // a chain that stopped (q_k = 0: beta_0 = 0, or beta_k = 0 for k >= 1) stays
  // stopped: W then holds only the rounding that the packed transforms leak
  // from the other vector of the pair, which must not restart it
  const double bk = beta[(long long)j * K + k];
  const bool dead = bk == 0.0;
  const double a = dead ? 0.0 : t.x, hn = sqrt(t.y);
  if (threadIdx.x == 0) alpha[(long long)j * K + k] = a;
  if (k + 1 >= K) return;
  double rr = 0.0;
  for (int i = threadIdx.x; i < n_pw; i += blockDim.x) {
    double r = W[o + i] - a * Qk[o + i];
    if (k > 0) r -= bk * Qkm1[o + i];
    Qk1[o + i] = r;
    rr += r * r;
  }
  const double b = sqrt(block_sum2(rr, 0.0).x);
  const bool stop = dead || !(b > 1e-12 * hn);
  const double f = stop ? 0.0 : 1.0 / b;
  for (int i = threadIdx.x; i < n_pw; i += blockDim.x) Qk1[o + i] *= f;
  if (threadIdx.x == 0) beta[(long long)j * K + k + 1] = stop ? 0.0 : b;
}
cudaError_t lanczos_step(const double* W, const double* Qk, const double* Qkm1, double* Qk1,
                         long long ld, int n_pw, int n, int K, int k, double* alpha, double* beta,
                         cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  {
    count_launch();
    k_lanczos_step<<<n, 256, 0, st>>>(W, Qk, Qkm1, Qk1, ld, n_pw, K, k, alpha, beta);
  }
  return cudaGetLastError();
}

// Eigen-decomposition of each chain's tridiagonal T (K <= 64) by parallel
// cyclic two-sided Jacobi in shared memory (Golub & Van Loan, Sec. 8.5):
// every round rotates K/2 disjoint (p, q) planes, J = [[c, s], [-s, c]] with
// t = s/c the smaller root of t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp)/(2 a_pq).
// Output: d [n][K] ascending and U [n][K][K] (U[j][m][k]: component m of
// eigenvector k).  Sweeps stop when the off-diagonal Frobenius norm is at or
// below 1e-15 of the whole or after 40 sweeps.
constexpr int kLzMax = 64;
__global__ void __launch_bounds__(256) k_tridiag_eig(const double* __restrict__ alpha,
                                                     const double* __restrict__ beta, int K,
                                                     double* d, double* U) {
  extern __shared__ __align__(16) double lz_sh[];
  const int ldk = K + 1;  // odd row stride
  double* Tm = lz_sh;
  double* Vm = lz_sh + K * ldk;
#define T(r, c) Tm[(r) * ldk + (c)]
#define V(r, c) Vm[(r) * ldk + (c)]
  __shared__ double cs[kLzMax / 2], sn[kLzMax / 2];
  __shared__ int pp[kLzMax / 2], qq[kLzMax / 2];
  __shared__ double dd[kLzMax];
  const int j = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const double* a = alpha + (long long)j * K;
  const double* b = beta + (long long)j * K;
  for (int e = tid; e < K * K; e += nt) {
    const int r = e / K, c = e % K;
    T(r, c) = r == c ? a[r] : (c == r + 1 ? b[c] : (r == c + 1 ? b[r] : 0.0));
    V(r, c) = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  const int nn = K + (K & 1);
  const int np = nn / 2;
  for (int sweep = 0; sweep < 40 && K > 1; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int e = tid; e < K * K; e += nt) {
      const int r = e / K, c = e % K;
      const double v = T(r, c) * T(r, c);
      all += v;
      if (r != c) off += v;
    }
    const double2 o = block_sum2(off, all);
    if (!(o.x > 1e-30 * o.y)) break;
    for (int round = 0; round < nn - 1; ++round) {
      if (tid < np) {
        int p, q;
        if (tid == 0) {
          p = nn - 1;
          q = round;
        } else {
          p = (round + tid) % (nn - 1);
          q = (round - tid + (nn - 1)) % (nn - 1);
        }
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        double c = 1.0, s = 0.0;
        if (q < K) {
          const double apq = T(p, q);
          if (apq != 0.0) {
            const double tau = (T(q, q) - T(p, p)) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = rsqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pp[tid] = p;
        qq[tid] = q;
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // rows: T <- J^T T
      for (int e = tid; e < np * K; e += nt) {
        const int w = e / K, col = e % K;
        const int p = pp[w], q = qq[w];
        if (q >= K) continue;
        const double c = cs[w], s = sn[w];
        const double tp = T(p, col), tq = T(q, col);
        T(p, col) = c * tp - s * tq;
        T(q, col) = s * tp + c * tq;
      }
      __syncthreads();
      // columns: T <- T J, V <- V J
      for (int e = tid; e < np * K; e += nt) {
        const int w = e / K, row = e % K;
        const int p = pp[w], q = qq[w];
        if (q >= K) continue;
        const double c = cs[w], s = sn[w];
        const double tp = T(row, p), tq = T(row, q);
        T(row, p) = c * tp - s * tq;
        T(row, q) = s * tp + c * tq;
        const double vp = V(row, p), vq = V(row, q);
        V(row, p) = c * vp - s * vq;
        V(row, q) = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  for (int k = tid; k < K; k += nt) dd[k] = T(k, k);
  __syncthreads();
  // ascending order (ties by index)
  for (int k = tid; k < K; k += nt) {
    int rank = 0;
    for (int m = 0; m < K; ++m) rank += (dd[m] < dd[k] || (dd[m] == dd[k] && m < k)) ? 1 : 0;
    d[(long long)j * K + rank] = dd[k];
    for (int m = 0; m < K; ++m) U[((long long)j * K + m) * K + rank] = V(m, k);
  }
}
#undef T
#undef V

cudaError_t tridiag_eig(const double* alpha, const double* beta, int n, int K, double* d,
                        double* U, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (K < 1 || K > kLzMax) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * 2 * K * (K + 1);
  cudaError_t e = cudaFuncSetAttribute(k_tridiag_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * 2 * kLzMax * (kLzMax + 1)));
  if (e != cudaSuccess) return e;
  { count_launch(); k_tridiag_eig<<<n, 256, smem, st>>>(alpha, beta, K, d, U); }
  return cudaGetLastError();
}

// weights[c][l][k] = beta[c][0] sum_m G[l][m n + j] U[c][m][k] U[c][0][k] for
// the chains c = j cs + c0, j < n; G[l][m n + j] = <L_l | q_m of chain c>
// (column-major n_L x (K n))
__global__ void k_lanczos_weights(const double* __restrict__ G, int n_L, int n, int K,
                                  const double* __restrict__ U, const double* __restrict__ beta,
                                  double* weights, int cs, int c0) {
  const int j = blockIdx.x;
  const long long ch = (long long)j * cs + c0;
  const double b0 = beta[ch * K];
  const double* u = U + ch * K * K;
  for (int e = threadIdx.x; e < n_L * K; e += blockDim.x) {
    const int l = e / K, k = e % K;
    double acc = 0.0;
    for (int m = 0; m < K; ++m) acc += G[l + ((long long)m * n + j) * n_L] * u[m * K + k];
    weights[(ch * n_L + l) * K + k] = b0 * acc * u[k];
  }
}
cudaError_t lanczos_weights(const double* G, int n_L, int n, int K, const double* U,
                            const double* beta, double* weights, int cs, int c0,
                            cudaStream_t st) {
  if (n <= 0 || n_L <= 0) return cudaSuccess;
  {
    count_launch();
    k_lanczos_weights<<<n, 128, 0, st>>>(G, n_L, n, K, U, beta, weights, cs, c0);
  }
  return cudaGetLastError();
}

// z[f][j][k] = beta[c][0] sum_k2 U[c][k][k2] U[c][0][k2] g(eps_v - d[c][k2], nu_f),
// g(D, nu) = D / (D^2 + nu^2), for the chains c = j cs + c0, j < n: the
// resolvent sum of Eq. finalB at the two frequencies eps_v -+ i nu, in the
// chain basis q_k
__global__ void k_lanczos_z(const double* __restrict__ U, const double* __restrict__ d,
                            const double* __restrict__ beta, int n, int K, int cs, int c0,
                            double eps_v, const double* __restrict__ nu, int n_freq, double* z) {
  const int j = blockIdx.x, f = blockIdx.y;
  const long long ch = (long long)j * cs + c0;
  const double b0 = beta[ch * K];
  const double* u = U + ch * K * K;
  const double* dd = d + ch * K;
  const double v2 = nu[f] * nu[f];
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double acc = 0.0;
    for (int k2 = 0; k2 < K; ++k2) {
      const double D = eps_v - dd[k2];
      const double den = D * D + v2;
      acc += u[k * K + k2] * u[k2] * (den > 0.0 ? D / den : 0.0);
    }
    z[((long long)f * n + j) * K + k] = b0 * acc;
  }
}
cudaError_t lanczos_z(const double* U, const double* d, const double* beta, int n, int K, int cs,
                      int c0, double eps_v, const double* nu, int n_freq, double* z,
                      cudaStream_t st) {
  if (n <= 0 || n_freq <= 0) return cudaSuccess;
  {
    count_launch();
    k_lanczos_z<<<dim3(n, n_freq), 64, 0, st>>>(U, d, beta, n, K, cs, c0, eps_v, nu, n_freq, z);
  }
  return cudaGetLastError();
}

// B[f] (n_L x n, column-major) += scale sum_k G[l][k n + j] z[f][j][k]
__global__ void k_body_accum(const double* __restrict__ G, int n_L, int n, int K,
                             const double* __restrict__ z, double scale, double* B) {
  const int j = blockIdx.x, f = blockIdx.y;
  const double* zz = z + ((long long)f * n + j) * K;
  double* b = B + (long long)f * n_L * n + (long long)j * n_L;
  for (int l = threadIdx.x; l < n_L; l += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += G[l + ((long long)k * n + j) * n_L] * zz[k];
    b[l] += scale * acc;
  }
}
cudaError_t body_accum(const double* G, int n_L, int n, int K, const double* z, int n_freq,
                       double scale, double* B, cudaStream_t st) {
  if (n <= 0 || n_freq <= 0) return cudaSuccess;
  { count_launch(); k_body_accum<<<dim3(n, n_freq), 128, 0, st>>>(G, n_L, n, K, z, scale, B); }
  return cudaGetLastError();
}

// Lambda = V diag(w / (1 - w)) V^T (n x n, column-major): the RPA body
// (1 - B)^{-1} B from the eigen-decomposition B = V diag(w) V^T
__global__ void k_lambda_from_eig(const double* __restrict__ V, const double* __restrict__ w,
                                  int n, double* L) {
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k)
      acc += V[i + (long long)k * n] * (w[k] / (1.0 - w[k])) * V[j + (long long)k * n];
    L[i + (long long)j * n] = acc;
  }
}
cudaError_t lambda_from_eig(const double* V, const double* w, int n, double* L, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_lambda_from_eig<<<n, 128, 0, st>>>(V, w, n, L); }
  return cudaGetLastError();
}

// out[j] = X_j . Y_j (one block per column)
__global__ void k_pair_dots(const double* __restrict__ X, const double* __restrict__ Y,
                            long long ld, int rows, double* out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x)
    s += X[(long long)j * ld + i] * Y[(long long)j * ld + i];
  const double2 t = block_sum2(s, 0.0);
  if (threadIdx.x == 0) out[j] = t.x;
}
cudaError_t pair_dots(const double* X, const double* Y, long long ld, int rows, int n, double* out,
                      cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_pair_dots<<<n, 256, 0, st>>>(X, Y, ld, rows, out); }
  return cudaGetLastError();
}

// One CG update per column j: x += a_j p, r -= a_j q (a = coef[j])
__global__ void k_cg_xr(double* x, double* r, const double* __restrict__ p,
                        const double* __restrict__ q, long long ld, int rows,
                        const double* __restrict__ coef) {
  const int j = blockIdx.y;
  const double a = coef[j];
  if (a == 0.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const long long o = (long long)j * ld + i;
    x[o] += a * p[o];
    r[o] -= a * q[o];
  }
}
// p = r + b_j p
__global__ void k_cg_p(double* p, const double* __restrict__ r, long long ld, int rows,
                       const double* __restrict__ coef) {
  const int j = blockIdx.y;
  const double b = coef[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const long long o = (long long)j * ld + i;
    p[o] = r[o] + b * p[o];
  }
}
// q = p - q (column blocks)
__global__ void k_one_minus(double* q, const double* __restrict__ p, long long ld, int rows) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const long long o = (long long)j * ld + i;
    q[o] = p[o] - q[o];
  }
}
cudaError_t one_minus(double* q, const double* p, long long ld, int rows, int n, cudaStream_t st) {
  const int bx = std::min((rows + 255) / 256, 64);
  for (int j0 = 0; j0 < n; j0 += 65535) {
    const int nj = std::min(65535, n - j0);
    const long long o = (long long)j0 * ld;
    count_launch();
    k_one_minus<<<dim3(bx, nj), 256, 0, st>>>(q + o, p + o, ld, rows);
  }
  return cudaGetLastError();
}
cudaError_t block_cg_xr(double* x, double* r, const double* p, const double* q, long long ld,
                        int rows, int n, const double* alpha, cudaStream_t st) {
  const int bx = std::min((rows + 255) / 256, 64);
  for (int j0 = 0; j0 < n; j0 += 65535) {
    const int nj = std::min(65535, n - j0);
    const long long o = (long long)j0 * ld;
    count_launch();
    k_cg_xr<<<dim3(bx, nj), 256, 0, st>>>(x + o, r + o, p + o, q + o, ld, rows, alpha + j0);
  }
  return cudaGetLastError();
}
cudaError_t block_cg_p(double* p, const double* r, long long ld, int rows, int n,
                       const double* beta, cudaStream_t st) {
  const int bx = std::min((rows + 255) / 256, 64);
  for (int j0 = 0; j0 < n; j0 += 65535) {
    const int nj = std::min(65535, n - j0);
    const long long o = (long long)j0 * ld;
    count_launch();
    k_cg_p<<<dim3(bx, nj), 256, 0, st>>>(p + o, r + o, ld, rows, beta + j0);
  }
  return cudaGetLastError();
}

cudaError_t fill_zero(void* p, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemsetAsync(p, 0, bytes, st);
}

// ---------------------------------------------------------------------------
// preconditioned CG on (H - eps_v + alpha P_v) x = b, one CTA per RHS
// ---------------------------------------------------------------------------
// Teter-Payne-Allan kinetic preconditioner (Phys. Rev. B 40, 12255 (1989)):
// K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),
// x = (|G|^2/2) / E_kin(v).
__device__ __forceinline__ double tpa(double x) {
  const double p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
  return p / (p + 16.0 * x * x * x * x);
}
__device__ __forceinline__ double precond(const double* __restrict__ g2, int n_half, int j,
                                          double inv_e) {
  if (j >= 2 * n_half) return 1.0;
  return tpa(0.5 * g2[j >> 1] * inv_e);
}

__global__ void k_build_precond(const double* __restrict__ g2, int n_half, int n_pw,
                                const double* __restrict__ ekin, double* k64, float* k32,
                                long long ld) {
  const int v = blockIdx.x;
  const double e = ekin[v] > 1e-3 ? ekin[v] : 1e-3;
  const double inv_e = 1.0 / e;
  for (int j = threadIdx.x; j < n_pw; j += blockDim.x) {
    const double k = precond(g2, n_half, j, inv_e);
    k64[(long long)v * ld + j] = k;
    k32[(long long)v * ld + j] = (float)k;
  }
}
cudaError_t build_precond(const double* g2, int n_half, int n_pw, const double* ekin, int n_occ,
                          double* k64, float* k32, long long ld, cudaStream_t st) {
  if (n_occ <= 0) return cudaSuccess;
  count_launch();
  k_build_precond<<<n_occ, 256, 0, st>>>(g2, n_half, n_pw, ekin, k64, k32, ld);
  return cudaGetLastError();
}

template <typename R>
__global__ void k_cg_start(CgArgs<R> a, const R* __restrict__ b, long long ldb) {
  const int i = blockIdx.x;
  if (a.mask && a.mask[i] == 0.0) {
    // not part of this solve (a converged RHS of a refinement round)
    if (threadIdx.x == 0) {
      CgScal s{};
      a.sc[i] = s;
    }
    return;
  }
  const long long o = (long long)i * a.ld;
  const R* K = a.kprec + (long long)(i % a.n_occ) * a.ld;
  R bb = R(0), rz = R(0);
  for (int j = threadIdx.x; j < a.n_pw; j += blockDim.x) {
    const R bv = b[(long long)i * ldb + j];
    const R kz = K[j];
    a.x[o + j] = R(0);
    a.r[o + j] = bv;
    a.p[o + j] = kz * bv;
    bb += bv * bv;
    rz += kz * bv * bv;
  }
  double2 t = block_sum2_r<R>(bb, rz);
  if (threadIdx.x == 0) {
    CgScal s;
    s.bnorm = sqrt(t.x);
    s.rnorm = s.bnorm;
    s.rz = t.y;
    s.iters = 0;
    s.active = t.x > 0.0 ? 1 : 0;
    a.sc[i] = s;
    if (s.active) atomicAdd(a.n_active, 1);
  }
}

// finish one RHS's step (thread 0): scalars, convergence, active count
template <typename R>
__device__ __forceinline__ void cg_finish(const CgArgs<R>& a, int i, const CgScal& s, double rn,
                                          double rkr, bool done) {
  CgScal n = s;
  n.iters = s.iters + 1;
  n.rnorm = rn;
  n.rz = rkr;
  n.active = done ? 0 : 1;
  if (!isfinite(rn)) {
    n.active = 0;
    atomicOr(a.status, (unsigned)DEV_NONFINITE);
  }
  a.sc[i] = n;
  if (n.active) atomicAdd(a.n_active, 1);
}

// Register-cached step: each thread keeps its E elements of p, Ap and r, so
// the RHS is read once (p, Ap, x, r) and written once (x, r, p).  Element
// arithmetic runs in R (FP32 costs 1/64 of FP64 on this part); only the
// per-thread partial sums are promoted to FP64 for the block reductions.
template <typename R, int E>
__global__ void __launch_bounds__(512) k_cg_step_reg(CgArgs<R> a, const int* __restrict__ list) {
  if (a.list_count && (int)blockIdx.x >= *a.list_count) return;
  const int i = list ? list[blockIdx.x] : blockIdx.x;
  __shared__ CgScal s;
  __shared__ R coef[2];  // alpha, then beta
  __shared__ int flag;   // 1: breakdown, 2: converged
  if (threadIdx.x == 0) s = a.sc[i];
  __syncthreads();
  if (!s.active) return;
  const long long o = (long long)i * a.ld;
  const R* K = a.kprec + (long long)(i % a.n_occ) * a.ld;
  R pv[E], av[E], rv[E];
  R pap = R(0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = threadIdx.x + e * blockDim.x;
    if (j < a.n_pw) {
      pv[e] = a.p[o + j];
      av[e] = a.ap[o + j];
      pap += pv[e] * av[e];
    } else {
      pv[e] = R(0);
      av[e] = R(0);
    }
  }
  const double2 t1 = block_sum2_r<R>(pap, R(0));
  if (threadIdx.x == 0) {
    const double al = s.rz / t1.x;
    flag = (!(t1.x > 0.0) || !isfinite(al)) ? 1 : 0;
    coef[0] = (R)al;
    if (flag) {
      atomicOr(a.status, isfinite(t1.x) ? (unsigned)DEV_BREAKDOWN : (unsigned)DEV_NONFINITE);
      a.sc[i].active = 0;
    }
  }
  __syncthreads();
  if (flag) return;
  const R alpha = coef[0];
  R rr = R(0), rkr = R(0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = threadIdx.x + e * blockDim.x;
    if (j < a.n_pw) {
      a.x[o + j] = a.x[o + j] + alpha * pv[e];
      const R r = a.r[o + j] - alpha * av[e];
      rv[e] = r;
      rr += r * r;
      rkr += K[j] * r * r;
    } else {
      rv[e] = R(0);
    }
  }
  const double2 t2 = block_sum2_r<R>(rr, rkr);
  if (threadIdx.x == 0) {
    const double rn = sqrt(t2.x);
    const bool done = rn <= (a.tolv ? a.tolv[i] : a.tol) * s.bnorm;
    flag = done ? 2 : 0;
    coef[1] = (R)(t2.y / s.rz);
    cg_finish(a, i, s, rn, t2.y, done);
  }
  __syncthreads();
  const bool done = flag == 2;
  const R beta = coef[1];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = threadIdx.x + e * blockDim.x;
    if (j < a.n_pw) {
      a.r[o + j] = rv[e];
      if (!done) a.p[o + j] = K[j] * rv[e] + beta * pv[e];
    }
  }
}

// Streaming step (three passes over the RHS, re-reads served by L1/L2):
// fewer registers, so more RHS in flight per SM than the cached variant.
template <typename R>
__global__ void __launch_bounds__(512) k_cg_step(CgArgs<R> a, const int* __restrict__ list) {
  if (a.list_count && (int)blockIdx.x >= *a.list_count) return;
  const int i = list ? list[blockIdx.x] : blockIdx.x;
  __shared__ CgScal s;
  __shared__ R coef[2];
  __shared__ int flag;
  if (threadIdx.x == 0) s = a.sc[i];
  __syncthreads();
  if (!s.active) return;
  const long long o = (long long)i * a.ld;
  const R* K = a.kprec + (long long)(i % a.n_occ) * a.ld;
  R pap = R(0);
  for (int j = threadIdx.x; j < a.n_pw; j += blockDim.x) pap += a.p[o + j] * a.ap[o + j];
  const double2 t1 = block_sum2_r<R>(pap, R(0));
  if (threadIdx.x == 0) {
    const double al = s.rz / t1.x;
    flag = (!(t1.x > 0.0) || !isfinite(al)) ? 1 : 0;
    coef[0] = (R)al;
    if (flag) {
      atomicOr(a.status, isfinite(t1.x) ? (unsigned)DEV_BREAKDOWN : (unsigned)DEV_NONFINITE);
      a.sc[i].active = 0;
    }
  }
  __syncthreads();
  if (flag) return;
  const R alpha = coef[0];
  R rr = R(0), rkr = R(0);
  for (int j = threadIdx.x; j < a.n_pw; j += blockDim.x) {
    a.x[o + j] = a.x[o + j] + alpha * a.p[o + j];
    const R r = a.r[o + j] - alpha * a.ap[o + j];
    a.r[o + j] = r;
    rr += r * r;
    rkr += K[j] * r * r;
  }
  const double2 t2 = block_sum2_r<R>(rr, rkr);
  if (threadIdx.x == 0) {
    const double rn = sqrt(t2.x);
    const bool done = rn <= (a.tolv ? a.tolv[i] : a.tol) * s.bnorm;
    flag = done ? 2 : 0;
    coef[1] = (R)(t2.y / s.rz);
    cg_finish(a, i, s, rn, t2.y, done);
  }
  __syncthreads();
  if (flag == 2) return;
  const R beta = coef[1];
  for (int j = threadIdx.x; j < a.n_pw; j += blockDim.x)
    a.p[o + j] = K[j] * a.r[o + j] + beta * a.p[o + j];
}

template <typename R>
cudaError_t cg_start(const CgArgs<R>& a, const R* b, long long ldb, cudaStream_t st) {
  if (a.n_rhs <= 0) return cudaSuccess;
  count_launch();
  k_cg_start<R><<<a.n_rhs, 256, 0, st>>>(a, b, ldb);
  return cudaGetLastError();
}
template <typename R>
cudaError_t cg_step(const CgArgs<R>& a, const int* list, int n_list, cudaStream_t st) {
  const int nb = list ? n_list : a.n_rhs;
  if (nb <= 0) return cudaSuccess;
  // x, r, p, Ap read once; x, r, p written once: 7 vector passes per active RHS
  ProfScope ps(sizeof(R) == 8 ? PC_CG_F64 : PC_CG_F32, st, 12.0 * nb * (double)a.n_pw,
               7.0 * nb * (double)a.n_pw * sizeof(R), list ? a.list_count : nullptr, nb);
  count_launch();
  int v = a.variant;
  if ((v == CG_REG256 && a.n_pw > 16 * 256) || (v == CG_REG512 && a.n_pw > 16 * 512))
    v = CG_STREAM256;
  switch (v) {
    case CG_REG256: k_cg_step_reg<R, 16><<<nb, 256, 0, st>>>(a, list); break;
    case CG_REG512: k_cg_step_reg<R, 16><<<nb, 512, 0, st>>>(a, list); break;
    case CG_STREAM128: k_cg_step<R><<<nb, 128, 0, st>>>(a, list); break;
    case CG_STREAM512: k_cg_step<R><<<nb, 512, 0, st>>>(a, list); break;
    default: k_cg_step<R><<<nb, 256, 0, st>>>(a, list); break;
  }
  return cudaGetLastError();
}
template cudaError_t cg_start<double>(const CgArgs<double>&, const double*, long long, cudaStream_t);
template cudaError_t cg_start<float>(const CgArgs<float>&, const float*, long long, cudaStream_t);
template cudaError_t cg_step<double>(const CgArgs<double>&, const int*, int, cudaStream_t);
template cudaError_t cg_step<float>(const CgArgs<float>&, const int*, int, cudaStream_t);

// ordered compaction with one block of 1024 threads (contiguous chunks + scan)
template <typename Pred>
__device__ void compact_block(int n, Pred pred, int* list, int* count) {
  __shared__ int offs[1024];
  const int T = blockDim.x;
  const int chunk = (n + T - 1) / T;
  const int lo = min(n, threadIdx.x * chunk), hi = min(n, lo + chunk);
  int c = 0;
  for (int i = lo; i < hi; ++i) c += pred(i) ? 1 : 0;
  offs[threadIdx.x] = c;
  __syncthreads();
  for (int d = 1; d < T; d <<= 1) {
    int v = threadIdx.x >= d ? offs[threadIdx.x - d] : 0;
    __syncthreads();
    offs[threadIdx.x] += v;
    __syncthreads();
  }
  int o = offs[threadIdx.x] - c;
  for (int i = lo; i < hi; ++i)
    if (pred(i)) list[o++] = i;
  if (threadIdx.x == T - 1) *count = offs[T - 1];
}
__global__ void k_active_list(const CgScal* __restrict__ sc, int n, int* list, int* count,
                              int* reset) {
  compact_block(n, [&](int i) { return sc[i].active != 0; }, list, count);
  if (reset && threadIdx.x == 0) *reset = 0;
}
__global__ void k_unconv_list(const double* __restrict__ rel, double tol, int n, int* list,
                              int* count, int* rounds) {
  compact_block(n, [&](int i) { return rel[i] > tol; }, list, count);
  if (rounds && threadIdx.x == blockDim.x - 1 && *count > 0) *rounds += 1;
}
cudaError_t active_list(const CgScal* sc, int n, int* list, int* count, cudaStream_t st) {
  count_launch();
  k_active_list<<<1, 1024, 0, st>>>(sc, n, list, count, nullptr);
  return cudaGetLastError();
}
cudaError_t active_list_reset(const CgScal* sc, int n, int* list, int* count, int* reset,
                              cudaStream_t st) {
  count_launch();
  k_active_list<<<1, 1024, 0, st>>>(sc, n, list, count, reset);
  return cudaGetLastError();
}
cudaError_t unconverged_list(const double* rel, double tol, int n, int* list, int* count,
                             cudaStream_t st, int* rounds) {
  count_launch();
  k_unconv_list<<<1, 1024, 0, st>>>(rel, tol, n, list, count, rounds);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// device-side loop control and statistics of the Sternheimer solves
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__global__ void k_loop_begin(CgLoopState* ls, int max_iter, cudaGraphConditionalHandle h,
                             int has_handle) {
  ls->iter = 0;
  ls->t0 = global_ns();
  const int go = (ls->active > 0 && max_iter > 0) ? 1 : 0;
  ls->go = go;
  if (has_handle) cudaGraphSetConditional(h, go);
}
__global__ void k_loop_next(CgLoopState* ls, int max_iter, unsigned long long budget_ns,
                            unsigned* status, int prec, cudaGraphConditionalHandle h,
                            int has_handle) {
  const int it = ls->iter + 1;
  ls->iter = it;
  ls->steps[prec] += 1;
  const bool active = ls->active > 0;
  bool go = active && it < max_iter;
  if (go && budget_ns > 0 && global_ns() - ls->t0 > budget_ns) {
    go = false;
    atomicOr(status, (unsigned)DEV_TIMEOUT);
  }
  ls->go = go ? 1 : 0;
  if (has_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
}
cudaError_t loop_begin(CgLoopState* ls, int max_iter, cudaGraphConditionalHandle h, int has_handle,
                       cudaStream_t st) {
  count_launch();
  k_loop_begin<<<1, 1, 0, st>>>(ls, max_iter, h, has_handle);
  return cudaGetLastError();
}
cudaError_t loop_next(CgLoopState* ls, int max_iter, unsigned long long budget_ns,
                      unsigned* status, int prec, cudaGraphConditionalHandle h, int has_handle,
                      cudaStream_t st) {
  count_launch();
  k_loop_next<<<1, 1, 0, st>>>(ls, max_iter, budget_ns, status, prec, h, has_handle);
  return cudaGetLastError();
}

__global__ void k_cg_collect(const CgScal* __restrict__ sc, int n, int* its_total, DevStats* ds) {
  unsigned long long sum = 0;
  int mx = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int it = sc[i].iters;
    if (its_total) its_total[i] += it;
    sum += (unsigned long long)it;
    mx = max(mx, it);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (sum) atomicAdd(&ds->cg_iters, sum);
    if (mx) atomicMax(&ds->cg_max, mx);
  }
}
cudaError_t cg_collect(const CgScal* sc, int n, int* its_total, DevStats* ds, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  const int blocks = std::min((n + 255) / 256, 4 * num_sms());
  k_cg_collect<<<blocks, 256, 0, st>>>(sc, n, its_total, ds);
  return cudaGetLastError();
}

__global__ void k_solve_finish(const double* __restrict__ rel, int n, double tol, DevStats* ds,
                               unsigned* status) {
  double mx = 0.0;
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double r = rel[i];
    if (!(r <= tol)) bad = 1;
    if (r > mx || r != r) mx = (r != r) ? INFINITY : r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax(&ds->max_res_bits, (unsigned long long)__double_as_longlong(mx));
    if (bad) atomicOr(status, (unsigned)DEV_NOT_CONVERGED);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ds->refine_max, ds->rounds_cur);
}
cudaError_t solve_finish(const double* rel, int n, double tol, DevStats* ds, unsigned* status,
                         cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  const int blocks = std::min((n + 255) / 256, 4 * num_sms());
  k_solve_finish<<<blocks, 256, 0, st>>>(rel, n, tol, ds, status);
  return cudaGetLastError();
}

__global__ void k_fill_value(double* x, int n, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}
cudaError_t fill_value(double* x, int n, double v, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_fill_value<<<std::min((n + 255) / 256, 1024), 256, 0, st>>>(x, n, v);
  return cudaGetLastError();
}

// Ri: the inner solve's precision (float: mixed modes, double: FP64 path).
// tolv (may be null): per-RHS relative tolerance of the inner solve,
// min(inner_cap, target / rel_i), so that the inner solve ends at an FP64
// residual of target x ||b_i||.
template <typename Ri>
__global__ void k_refine_prepare(const double* __restrict__ r64, long long ld64, int n_pw,
                                 const double* __restrict__ rel, double tol, Ri* ri,
                                 long long ldi, double* rn, double* tolv, double target,
                                 double inner_cap) {
  const int i = blockIdx.x;
  const bool act = rel[i] > tol;
  double ss = 0.0;
  if (act)
    for (int j = threadIdx.x; j < n_pw; j += blockDim.x) {
      const double v = r64[(long long)i * ld64 + j];
      ss += v * v;
    }
  const double2 t = block_sum2(ss, 0.0);
  const double nrm = sqrt(t.x);
  const double f = (act && nrm > 0.0) ? 1.0 / nrm : 0.0;
  // a converged RHS keeps rn = 0 and takes no part in the inner solve (its
  // scaled residual is not written)
  if (act)
    for (int j = threadIdx.x; j < n_pw; j += blockDim.x)
      ri[(long long)i * ldi + j] = (Ri)(f * r64[(long long)i * ld64 + j]);
  if (threadIdx.x == 0) {
    rn[i] = act ? nrm : 0.0;
    if (tolv) tolv[i] = act ? fmin(inner_cap, target / rel[i]) : inner_cap;
  }
}
template <typename Ri>
cudaError_t refine_prepare(const double* r64, long long ld64, int n_pw, int n, const double* rel,
                           double tol, Ri* ri, long long ldi, double* rn, cudaStream_t st,
                           double* tolv, double target, double inner_cap) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_refine_prepare<Ri><<<n, 256, 0, st>>>(r64, ld64, n_pw, rel, tol, ri, ldi, rn, tolv, target,
                                          inner_cap);
  return cudaGetLastError();
}
template cudaError_t refine_prepare<float>(const double*, long long, int, int, const double*, double,
                                           float*, long long, double*, cudaStream_t, double*,
                                           double, double);
template cudaError_t refine_prepare<double>(const double*, long long, int, int, const double*,
                                            double, double*, long long, double*, cudaStream_t,
                                            double*, double, double);
__global__ void k_refine_accumulate(double* x64, long long ld64, const float* __restrict__ d32,
                                    long long ld32, int n_pw, const double* __restrict__ rn) {
  const int i = blockIdx.x;
  const double f = rn[i];
  if (f == 0.0) return;
  for (int j = threadIdx.x; j < n_pw; j += blockDim.x)
    x64[(long long)i * ld64 + j] += f * (double)d32[(long long)i * ld32 + j];
}
cudaError_t refine_accumulate(double* x64, long long ld64, const float* d32, long long ld32,
                              int n_pw, int n, const double* rn, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_refine_accumulate<<<n, 256, 0, st>>>(x64, ld64, d32, ld32, n_pw, rn); }
  return cudaGetLastError();
}

// One refinement update in FP64.  With d32: delta_i = rn_i d32_i (+ xd_i);
// vectors with rn_i = 0 and no xd are skipped.  Without d32 (the FP64 path,
// x holding the whole CG solution): delta_i = x_i + xd_i.  Then x_i += delta_i
// (x_i = delta_i without d32) and dl_i = delta_i.
template <typename Ri>
__global__ void k_refine_delta(double* x, double* dl, long long ld, const Ri* __restrict__ d32,
                               long long ld32, int n_pw, const double* __restrict__ rn,
                               const double* __restrict__ xd, float* dlf) {
  const int i = blockIdx.x;
  const double f = rn ? rn[i] : 0.0;
  if (d32 && f == 0.0 && !xd) return;
  double* xi = x + (long long)i * ld;
  double* di = dl + (long long)i * ld;
  const double* xdi = xd ? xd + (long long)i * ld : nullptr;
  for (int j = threadIdx.x; j < n_pw; j += blockDim.x) {
    double d;
    if (d32) {
      d = (f != 0.0 ? f * (double)d32[(long long)i * ld32 + j] : 0.0) + (xdi ? xdi[j] : 0.0);
      xi[j] += d;
    } else {
      d = xi[j] + (xdi ? xdi[j] : 0.0);
      xi[j] = d;
    }
    di[j] = d;
    if (dlf) dlf[(long long)i * ld + j] = (float)d;
  }
}
template <typename Ri>
cudaError_t refine_delta(double* x, double* dl, long long ld, const Ri* d32, long long ld32,
                         int n_pw, int n, const double* rn, const double* xd, cudaStream_t st,
                         float* dlf) {
  if (n <= 0) return cudaSuccess;
  {
    count_launch();
    k_refine_delta<Ri><<<n, 256, 0, st>>>(x, dl, ld, d32, ld32, n_pw, rn, xd, dlf);
  }
  return cudaGetLastError();
}
template cudaError_t refine_delta<float>(double*, double*, long long, const float*, long long, int,
                                         int, const double*, const double*, cudaStream_t, float*);
template cudaError_t refine_delta<double>(double*, double*, long long, const double*, long long,
                                          int, int, const double*, const double*, cudaStream_t,
                                          float*);

// r_i -= ad_i (+ s_{i mod n_occ} xd_i), rel_i = ||r_i|| / ||b_i|| for the
// listed (or all) vectors.  s_v = eps_{n_ext} - eps_v is the shifted
// operator's eigenvalue on the deflated states, so s_v xd_i = A xd_i.
template <typename Ta>
__global__ void k_residual_update(double* r, const Ta* __restrict__ ad,
                                  const double* __restrict__ b, long long ld, int n_pw,
                                  double* rel, const int* __restrict__ list,
                                  const double* __restrict__ xd, const double* __restrict__ sv,
                                  int n_occ, const int* __restrict__ ndev) {
  if (ndev && (int)blockIdx.x >= *ndev) return;
  const int i = list ? list[blockIdx.x] : blockIdx.x;
  const long long o = (long long)i * ld;
  const double s = xd ? sv[i % n_occ] : 0.0;
  double rr = 0.0, bb = 0.0;
  for (int j = threadIdx.x; j < n_pw; j += blockDim.x) {
    double v = r[o + j] - (double)ad[o + j];
    if (xd) v += s * xd[o + j];
    r[o + j] = v;
    const double bv = b[o + j];
    rr += v * v;
    bb += bv * bv;
  }
  double2 t = block_sum2(rr, bb);
  if (threadIdx.x == 0) rel[i] = t.y > 0.0 ? sqrt(t.x / t.y) : 0.0;
}
template <typename Ta>
cudaError_t residual_update(double* r, const Ta* ad, const double* b, long long ld, int n_pw,
                            int n, double* rel, const int* list, const double* xd,
                            const double* sv, int n_occ, cudaStream_t st, const int* ndev) {
  if (n <= 0) return cudaSuccess;
  {
    count_launch();
    k_residual_update<Ta><<<n, 256, 0, st>>>(r, ad, b, ld, n_pw, rel, list, xd, sv, n_occ, ndev);
  }
  return cudaGetLastError();
}
template cudaError_t residual_update<double>(double*, const double*, const double*, long long, int,
                                             int, double*, const int*, const double*,
                                             const double*, int, cudaStream_t, const int*);
template cudaError_t residual_update<float>(double*, const float*, const double*, long long, int,
                                            int, double*, const int*, const double*,
                                            const double*, int, cudaStream_t, const int*);

__global__ void k_kinetic(const double* __restrict__ X, long long ld, int n_half,
                          const double* __restrict__ g2, double* out) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int k = threadIdx.x; k < n_half; k += blockDim.x) {
    const double a = X[(long long)i * ld + 2 * k], b = X[(long long)i * ld + 2 * k + 1];
    s += 0.5 * g2[k] * (a * a + b * b);
  }
  const double2 t = block_sum2(s, 0.0);
  if (threadIdx.x == 0) out[i] = t.x;
}
cudaError_t kinetic_energy(const double* X, long long ld, int n_half, int n, const double* g2,
                           double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_kinetic<<<n, 256, 0, st>>>(X, ld, n_half, g2, out); }
  return cudaGetLastError();
}
__global__ void k_precondition(double* T, long long ld, int n_pw, int n_half,
                               const double* __restrict__ g2, const double* __restrict__ ekin) {
  const int i = blockIdx.x;
  const double e = ekin[i] > 1e-3 ? ekin[i] : 1e-3;
  const double inv_e = 1.0 / e;
  for (int j = threadIdx.x; j < n_pw; j += blockDim.x)
    T[(long long)i * ld + j] *= precond(g2, n_half, j, inv_e);
}
cudaError_t precondition_tpa(double* T, long long ld, int n_pw, int n_half, int n,
                             const double* g2, const double* ekin, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_precondition<<<n, 256, 0, st>>>(T, ld, n_pw, n_half, g2, ekin); }
  return cudaGetLastError();
}
__global__ void k_gather_cols(const double* __restrict__ X, long long ldx, double* Y,
                              long long ldy, int rows, const int* __restrict__ idx) {
  const int i = blockIdx.x;
  const int src = idx[i];
  for (int r = threadIdx.x; r < rows; r += blockDim.x)
    Y[(long long)i * ldy + r] = X[(long long)src * ldx + r];
}
cudaError_t gather_cols(const double* X, long long ldx, double* Y, long long ldy, int rows,
                        const int* idx, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_gather_cols<<<n, 256, 0, st>>>(X, ldx, Y, ldy, rows, idx); }
  return cudaGetLastError();
}
__global__ void k_unit_start(double* X, long long ld, int rows, const int* __restrict__ comp,
                             double amp) {
  const int i = blockIdx.x;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) X[(long long)i * ld + r] *= amp;
  __syncthreads();
  if (threadIdx.x == 0) X[(long long)i * ld + comp[i]] += 1.0;
}
cudaError_t unit_start(double* X, long long ld, int rows, const int* comp, int n, double amp,
                       unsigned long long seed, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = philox_normal(X, ld, rows, n, seed, 0ULL, st);
  if (e != cudaSuccess) return e;
  { count_launch(); k_unit_start<<<n, 256, 0, st>>>(X, ld, rows, comp, amp); }
  return cudaGetLastError();
}
__global__ void k_cheb_step(double* Ynew, const double* __restrict__ HY,
                            const double* __restrict__ Y, const double* __restrict__ X,
                            long long ld, int rows, double a1, double c, double b1) {
  const long long o = (long long)blockIdx.y * ld;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const double xv = X ? X[o + r] : 0.0;
    Ynew[o + r] = a1 * (HY[o + r] - c * Y[o + r]) + b1 * xv;
  }
}
cudaError_t cheb_step(double* Ynew, const double* HY, const double* Y, const double* X,
                      long long ld, int rows, int n, double a1, double c, double b1,
                      cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid((rows + 255) / 256, n);
  count_launch();
  k_cheb_step<<<grid, 256, 0, st>>>(Ynew, HY, Y, X, ld, rows, a1, c, b1);
  return cudaGetLastError();
}

__global__ void k_deflation_coef(double* S, int lds, int n_occ, int n_defl, int n,
                                 const double* __restrict__ eps) {
  const long long tot = (long long)n_defl * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int cdx = (int)(e % n_defl), i = (int)(e / n_defl);
    S[(long long)i * lds + n_occ + cdx] /= (eps[n_occ + cdx] - eps[i % n_occ]);
  }
}
cudaError_t deflation_coefficients(double* S, int lds, int n_occ, int n_defl, int n,
                                   const double* eps, cudaStream_t st) {
  const long long tot = (long long)n_defl * n;
  if (tot <= 0) return cudaSuccess;
  count_launch();
  k_deflation_coef<<<(int)std::min<long long>((tot + 255) / 256, 4096), 256, 0, st>>>(
      S, lds, n_occ, n_defl, n, eps);
  return cudaGetLastError();
}
template <typename R>
__global__ void k_scale_rows(R* S, int lds, int rows, int n, const R* __restrict__ sigma) {
  const long long tot = (long long)rows * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(e % rows), i = (int)(e / rows);
    S[(long long)i * lds + w] *= sigma[w];
  }
}
template <typename R>
cudaError_t scale_rows(R* S, int lds, int rows, int n, const R* sigma, cudaStream_t st) {
  const long long tot = (long long)rows * n;
  if (tot <= 0) return cudaSuccess;
  count_launch();
  k_scale_rows<R><<<(int)std::min<long long>((tot + 255) / 256, 8192), 256, 0, st>>>(S, lds, rows,
                                                                                    n, sigma);
  return cudaGetLastError();
}
template cudaError_t scale_rows<double>(double*, int, int, int, const double*, cudaStream_t);
template cudaError_t scale_rows<float>(float*, int, int, int, const float*, cudaStream_t);


__global__ void k_zero_row(double* X, long long ld, int row, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    X[(long long)i * ld + row] = 0.0;
}
cudaError_t zero_row(double* X, long long ld, int row, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { count_launch(); k_zero_row<<<(n + 255) / 256, 256, 0, st>>>(X, ld, row, n); }
  return cudaGetLastError();
}

}  // namespace pdep
