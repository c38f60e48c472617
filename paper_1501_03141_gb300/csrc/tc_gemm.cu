// Tensor-core (TF32 mma.sync) kernels for the FP32 projection of the shifted
// Sternheimer operator: the term sum_w sigma_w |w><w| x of
// (H - eps_v + sum_w sigma_w |w><w|) x, applied to every active right-hand
// side of the inner CG (Eq. stern with the occupied and deflated states w).
//
//   coefficients:  S[w][j] = sigma_w * sum_k P[k][w] X[k][bmap(j)]   (K = n_pw)
//   update:        Y[r][cmap(j)] += sum_w P[r][w] S[w][j]            (K = n_ext)
//
// Both run as "3xTF32": every FP32 operand a is split into a_hi = tf32(a) and
// a_lo = tf32(a - a_hi), and a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32
// accumulation, which keeps the products at FP32 accuracy (a single TF32
// product would perturb the CG operator at the 1e-4 level).  Operand tiles
// are staged in shared memory with cp.async; fragment layouts follow the
// m16n8k8 .row.col TF32 shape of the PTX ISA.
#include <algorithm>
#include <cstdint>

#include "linalg.cuh"
#include "profile.cuh"

namespace pdep {
namespace {

__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += a b in 3xTF32 (small terms first)
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const uint32_t (&ah)[4],
                                           const uint32_t (&al)[4], const uint32_t (&bh)[2],
                                           const uint32_t (&bl)[2]) {
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

// 16-byte global -> shared copy of 'bytes' (0..16) valid bytes, zero-filled
__device__ __forceinline__ void cp16(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---------------------------------------------------------------------------
// coefficients: S (M x N, lds) += diag(sigma) P^T X(:, bmap) over the K range
// [blockIdx.z kchunk, +kchunk) (split K, FP32 atomics; S zeroed beforehand).
// CTA tile 32 x 64, 4 warps each 32 x 16, K tile 32.
// ---------------------------------------------------------------------------
constexpr int C_BM = 32, C_BN = 64, C_BK = 32, C_PAD = 36;

__global__ void __launch_bounds__(128)
    k_tc_coeffs(int M, int N, int K, const float* __restrict__ P, long long ldp,
                const float* __restrict__ X, long long ldx, const int* __restrict__ bmap,
                const float* __restrict__ sigma, float* __restrict__ S, long long lds,
                int kchunk, const int* __restrict__ ndev) {
  __shared__ __align__(16) float As[2][C_BM][C_PAD];
  __shared__ __align__(16) float Bs[2][C_BN][C_PAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int row0 = blockIdx.x * C_BM, col0 = blockIdx.y * C_BN;
  if (ndev) N = min(N, *ndev);  // device count of the mapped columns
  if (col0 >= N) return;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);

  auto load = [&](int stage, int k0) {
    // A: 32 rows x 8 chunks of 4 floats
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = tid + 128 * q;
      const int r = c >> 3, kc = (c & 7) * 4;
      const int gr = row0 + r, gk = k0 + kc;
      int bytes = 0;
      const float* src = P;
      if (gr < M && gk < kend) {
        bytes = 4 * min(4, kend - gk);
        src = P + (long long)gr * ldp + gk;
      }
      cp16(&As[stage][r][kc], src, bytes);
    }
    // B: 64 columns x 8 chunks
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = tid + 128 * q;
      const int j = c >> 3, kc = (c & 7) * 4;
      const int gj = col0 + j, gk = k0 + kc;
      int bytes = 0;
      const float* src = X;
      if (gj < N && gk < kend) {
        bytes = 4 * min(4, kend - gk);
        src = X + (long long)(bmap ? bmap[gj] : gj) * ldx + gk;
      }
      cp16(&Bs[stage][j][kc], src, bytes);
    }
  };

  float acc[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.f;

  const int nk = kend > kbeg ? (kend - kbeg + C_BK - 1) / C_BK : 0;
  if (nk > 0) load(0, kbeg);
  cp_commit();
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) load((kt + 1) & 1, kbeg + (kt + 1) * C_BK);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const int s = kt & 1;
    // this K tile's products accumulate in the tensor cores from zero and are
    // then added to acc with FP32 adds: the MMA accumulator adds with
    // truncation, so long in-MMA accumulation chains would bias S (whose
    // terms cancel: x is nearly orthogonal to the states w)
    float tacc[2][2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) tacc[a][b][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < C_BK; kk += 8) {
      uint32_t ah[2][4], al[2][4], bh[2][2], bl[2][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = mi * 16 + g;
        split_tf32(As[s][r][kk + t], ah[mi][0], al[mi][0]);
        split_tf32(As[s][r + 8][kk + t], ah[mi][1], al[mi][1]);
        split_tf32(As[s][r][kk + t + 4], ah[mi][2], al[mi][2]);
        split_tf32(As[s][r + 8][kk + t + 4], ah[mi][3], al[mi][3]);
      }
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) {
        const int j = warp * 16 + ni * 8 + g;
        split_tf32(Bs[s][j][kk + t], bh[ni][0], bl[ni][0]);
        split_tf32(Bs[s][j][kk + t + 4], bh[ni][1], bl[ni][1]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) mma_3xtf32(tacc[mi][ni], ah[mi], al[mi], bh[ni], bl[ni]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[a][b][e] += tacc[a][b][e];
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = row0 + mi * 16 + g + (e >= 2 ? 8 : 0);
        const int j = col0 + warp * 16 + ni * 8 + 2 * t + (e & 1);
        if (r < M && j < N && nk > 0) atomicAdd(S + r + (long long)j * lds, sigma[r] * acc[mi][ni][e]);
      }
}

// ---------------------------------------------------------------------------
// update: Y(:, cmap) (M x N) += P (M x K) S (K x N, lds)
// CTA tile 64 x 64, 4 warps of 32 x 32, K tile 16.
// ---------------------------------------------------------------------------
constexpr int U_BM = 64, U_BN = 64, U_BK = 16, U_APAD = 72, U_BPAD = 20;

__global__ void __launch_bounds__(128)
    k_tc_update(int M, int N, int K, const float* __restrict__ P, long long ldp,
                const float* __restrict__ S, long long lds, float* __restrict__ Y, long long ldy,
                const int* __restrict__ cmap, const int* __restrict__ ndev) {
  __shared__ __align__(16) float As[2][U_BK][U_APAD];  // A(r, w) at As[w][r]
  __shared__ __align__(16) float Bs[2][U_BN][U_BPAD];  // B(w, j) at Bs[j][w]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp >> 1, wn = warp & 1;
  const int row0 = blockIdx.x * U_BM, col0 = blockIdx.y * U_BN;
  if (ndev) N = min(N, *ndev);
  if (col0 >= N) return;

  auto load = [&](int stage, int k0) {
    // A: 16 state columns x 16 chunks of 4 rows
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = tid + 128 * q;
      const int w = c >> 4, rc = (c & 15) * 4;
      const int gw = k0 + w, gr = row0 + rc;
      int bytes = 0;
      const float* src = P;
      if (gw < K && gr < M) {
        bytes = 4 * min(4, M - gr);
        src = P + (long long)gw * ldp + gr;
      }
      cp16(&As[stage][w][rc], src, bytes);
    }
    // B: 64 columns x 4 chunks of 4 states
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = tid + 128 * q;
      const int j = c >> 2, wc = (c & 3) * 4;
      const int gj = col0 + j, gw = k0 + wc;
      int bytes = 0;
      const float* src = S;
      if (gj < N && gw < K) {
        bytes = 4 * min(4, K - gw);
        src = S + (long long)gj * lds + gw;
      }
      cp16(&Bs[stage][j][wc], src, bytes);
    }
  };

  // acc starts from Y: its loads overlap the K loop instead of stalling the
  // epilogue
  float acc[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = row0 + wm * 32 + mi * 16 + g + (e >= 2 ? 8 : 0);
        const int j = col0 + wn * 32 + ni * 8 + 2 * t + (e & 1);
        acc[mi][ni][e] = (r < M && j < N) ? Y[r + (long long)(cmap ? cmap[j] : j) * ldy] : 0.f;
      }

  const int nk = (K + U_BK - 1) / U_BK;
  load(0, 0);
  cp_commit();
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) load((kt + 1) & 1, (kt + 1) * U_BK);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const int s = kt & 1;
    float tacc[2][4][4];  // per K tile, as in k_tc_coeffs
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) tacc[a][b][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < U_BK; kk += 8) {
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16 + g;
        split_tf32(As[s][kk + t][r], ah[mi][0], al[mi][0]);
        split_tf32(As[s][kk + t][r + 8], ah[mi][1], al[mi][1]);
        split_tf32(As[s][kk + t + 4][r], ah[mi][2], al[mi][2]);
        split_tf32(As[s][kk + t + 4][r + 8], ah[mi][3], al[mi][3]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int j = wn * 32 + ni * 8 + g;
        split_tf32(Bs[s][j][kk + t], bh[ni][0], bl[ni][0]);
        split_tf32(Bs[s][j][kk + t + 4], bh[ni][1], bl[ni][1]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_3xtf32(tacc[mi][ni], ah[mi], al[mi], bh[ni], bl[ni]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[a][b][e] += tacc[a][b][e];
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = row0 + wm * 32 + mi * 16 + g + (e >= 2 ? 8 : 0);
        const int j = col0 + wn * 32 + ni * 8 + 2 * t + (e & 1);
        if (r < M && j < N) Y[r + (long long)(cmap ? cmap[j] : j) * ldy] = acc[mi][ni][e];
      }
}

}  // namespace

cudaError_t tc_proj_coeffs(int M, int N, int K, const float* P, long long ldp, const float* X,
                           long long ldx, const int* bmap, const float* sigma, float* S,
                           long long lds, cudaStream_t st, const int* ndev) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((M + C_BM - 1) / C_BM, (N + C_BN - 1) / C_BN);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  // split K so that about four CTAs per SM stream X
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (long long)grid.x * grid.y;
  int split = (int)std::max<long long>(1, (4LL * std::max(sms, 1) + tiles - 1) / tiles);
  split = std::min(split, std::max(1, K / (8 * C_BK)));
  int kchunk = (K + split - 1) / split;
  kchunk = ((kchunk + C_BK - 1) / C_BK) * C_BK;
  grid.z = (unsigned)((K + kchunk - 1) / kchunk);
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(float) * (size_t)lds * N, st);
  if (e != cudaSuccess) return e;
  ProfScope ps(PC_GEMM_TF32, st, 2.0 * M * N * (double)K,
               ((double)M * K + (double)K * N + (double)M * N) * sizeof(float), ndev, N);
  count_launch();
  k_tc_coeffs<<<grid, 128, 0, st>>>(M, N, K, P, ldp, X, ldx, bmap, sigma, S, lds, kchunk, ndev);
  return cudaGetLastError();
}

cudaError_t tc_proj_update(int M, int N, int K, const float* P, long long ldp, const float* S,
                           long long lds, float* Y, long long ldy, const int* cmap,
                           cudaStream_t st, const int* ndev) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  dim3 grid((M + U_BM - 1) / U_BM, (N + U_BN - 1) / U_BN);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  ProfScope ps(PC_GEMM_TF32, st, 2.0 * M * N * (double)K,
               ((double)M * K + (double)K * N + 2.0 * M * N) * sizeof(float), ndev, N);
  count_launch();
  k_tc_update<<<grid, 128, 0, st>>>(M, N, K, P, ldp, S, lds, Y, ldy, cmap, ndev);
  return cudaGetLastError();
}

}  // namespace pdep
