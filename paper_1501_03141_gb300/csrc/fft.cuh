// Register-resident line FFTs for the plane-wave sphere <-> grid transforms.
//
// A line of length N = TPL * M is held by TPL consecutive lanes of a warp
// (a "group", aligned to TPL).  Two data distributions are used:
//   A: lane t holds element n = t + TPL*i in register i      (i = 0..M-1)
//   B: lane t holds element k = i + M*rev(t) in register i   (rev = bit reversal
//      over log2(TPL) bits)
// fft_a2b computes an M-point DFT in registers, multiplies by the twiddles
// w_N^{S t k2} and finishes with a TPL-point DFT across the group using
// radix-2 decimation-in-frequency butterflies on warp shuffles.  fft_b2a is
// the transposed network (DIT shuffles, twiddles, local DFT); because the
// DFT matrix is symmetric it computes the same transform from B to A.  A
// sphere->grid pass therefore runs A->B and the grid->sphere pass B->A with
// no data exchange in between.
//
// Sign convention: S = +1 is sum_n x_n exp(+2 pi i n k / N) (sphere -> grid,
// unnormalised), S = -1 the forward transform (grid -> sphere).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "df64.cuh"

namespace pdep {

// ---------------------------------------------------------------------------
// twiddles of the in-register DFTs (compile-time indices -> constant bank)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int local_tw_offset(int M) {
  return M == 6 ? 0 : M == 8 ? 6 : M == 10 ? 14 : M == 12 ? 24 : M == 16 ? 36
       : M == 20 ? 52 : M == 24 ? 72 : M == 32 ? 96 : M == 48 ? 128 : M == 64 ? 176 : -1;
}
constexpr int LOCAL_TW_SIZE = 240;

// defined here: fft.cuh is included by a single translation unit (no -rdc)
__constant__ double2 c_local_tw_d[LOCAL_TW_SIZE];
__constant__ float2 c_local_tw_f[LOCAL_TW_SIZE];
__constant__ float4 c_local_tw_df[LOCAL_TW_SIZE];  // (re.hi, re.lo, im.hi, im.lo)

template <typename R>
struct LocalTw;
template <>
struct LocalTw<double> {
  static __device__ __forceinline__ cpx<double> get(int i) {
    double2 v = c_local_tw_d[i];
    return mk(v.x, v.y);
  }
};
template <>
struct LocalTw<float> {
  static __device__ __forceinline__ cpx<float> get(int i) {
    float2 v = c_local_tw_f[i];
    return mk(v.x, v.y);
  }
};
template <>
struct LocalTw<df> {
  static __device__ __forceinline__ cpx<df> get(int i) {
    float4 v = c_local_tw_df[i];
    return mk(df(v.x, v.y), df(v.z, v.w));
  }
};

// exp(S * 2 pi i j / M) for the local DFT of size M
template <typename R, int S, int M>
__device__ __forceinline__ cpx<R> local_w(int j) {
  cpx<R> w = LocalTw<R>::get(local_tw_offset(M) + j);
  return S > 0 ? w : conj(w);
}

__host__ __device__ constexpr int pick_radix(int M) {
  return (M % 4 == 0 && M != 4) ? 4 : (M % 2 == 0 && M != 2) ? 2 : (M % 3 == 0 && M != 3) ? 3 : 5;
}

// In-place DFT of compile-time size M over a register array:
//   a[k] <- sum_n a[n] exp(S 2 pi i n k / M)
template <typename R, int M, int S>
struct DFT {
  static constexpr int P = pick_radix(M);
  static constexpr int Q = M / P;
  static __device__ __forceinline__ void run(cpx<R>* a) {
    // n = p + P q,  k = k1 + Q k2
    cpx<R> y[P][Q];
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
      for (int q = 0; q < Q; ++q) y[p][q] = a[p + P * q];
      DFT<R, Q, S>::run(y[p]);
    }
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) {
      cpx<R> z[P];
#pragma unroll
      for (int p = 0; p < P; ++p)
        z[p] = (p * k1 == 0) ? y[p][k1] : y[p][k1] * local_w<R, S, M>((p * k1) % M);
      DFT<R, P, S>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) a[k1 + Q * k2] = z[k2];
    }
  }
};

template <typename R, int S>
struct DFT<R, 1, S> {
  static __device__ __forceinline__ void run(cpx<R>*) {}
};

template <typename R, int S>
struct DFT<R, 2, S> {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    cpx<R> t = a[0];
    a[0] = t + a[1];
    a[1] = t - a[1];
  }
};

template <typename R, int S>
struct DFT<R, 3, S> {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    const R h = R(0.8660254037844386467637231707529362);  // sqrt(3)/2
    cpx<R> t1 = a[1] + a[2];
    cpx<R> t2 = a[1] - a[2];
    cpx<R> m = a[0] - scale(t1, R(0.5));
    cpx<R> n = scale(mul_si<R, S>(t2), h);
    a[0] = a[0] + t1;
    a[1] = m + n;
    a[2] = m - n;
  }
};

template <typename R, int S>
struct DFT<R, 4, S> {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    cpx<R> t0 = a[0] + a[2];
    cpx<R> t1 = a[0] - a[2];
    cpx<R> t2 = a[1] + a[3];
    cpx<R> t3 = mul_si<R, S>(a[1] - a[3]);
    a[0] = t0 + t2;
    a[2] = t0 - t2;
    a[1] = t1 + t3;
    a[3] = t1 - t3;
  }
};

template <typename R, int S>
struct DFT<R, 5, S> {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    const R c1 = R(0.3090169943749474241022934171828191);   // cos(2 pi/5)
    const R c2 = R(-0.8090169943749474241022934171828191);  // cos(4 pi/5)
    const R s1 = R(0.9510565162951535721164393333793821);   // sin(2 pi/5)
    const R s2 = R(0.5877852522924731291687059546390728);   // sin(4 pi/5)
    cpx<R> t1 = a[1] + a[4];
    cpx<R> t2 = a[2] + a[3];
    cpx<R> t3 = a[1] - a[4];
    cpx<R> t4 = a[2] - a[3];
    cpx<R> b1 = a[0] + scale(t1, c1) + scale(t2, c2);
    cpx<R> b2 = a[0] + scale(t1, c2) + scale(t2, c1);
    cpx<R> d1 = mul_si<R, S>(scale(t3, s1) + scale(t4, s2));
    cpx<R> d2 = mul_si<R, S>(scale(t3, s2) - scale(t4, s1));
    a[0] = a[0] + t1 + t2;
    a[1] = b1 + d1;
    a[4] = b1 - d1;
    a[2] = b2 + d2;
    a[3] = b2 - d2;
  }
};

// ---------------------------------------------------------------------------
// line FFT across a lane group
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

__device__ __forceinline__ int bitrev(int t, int bits) {
  return bits == 0 ? 0 : (int)(__brev((unsigned)t) >> (32 - bits));
}

// exp(S 2 pi i j / N) from a global table of exp(+2 pi i j / N), j in [0, N)
template <typename R, int S>
__device__ __forceinline__ cpx<R> table_w(const cpx<R>* __restrict__ tw, int j) {
  cpx<R> w;
  if constexpr (std::is_same<R, df>::value) {
    // double-float: one 16-byte load of (re.hi, re.lo, im.hi, im.lo)
    const float4 v = __ldg(reinterpret_cast<const float4*>(tw + j));
    w = mk(R(v.x, v.y), R(v.z, v.w));
  } else {
    w.x = __ldg(&tw[j].x);
    w.y = __ldg(&tw[j].y);
  }
  return S > 0 ? w : conj(w);
}

// p + v (lower lane of a butterfly) or p - v (upper lane): one fused
// multiply-add per component in FP32 / FP64, a sign flip and one addition in
// double-float
template <typename R>
__device__ __forceinline__ cpx<R> pm(cpx<R> p, cpx<R> v, bool up) {
  const R sgn = up ? R(-1) : R(1);
  return mk(p.x + sgn * v.x, p.y + sgn * v.y);
}
template <>
__device__ __forceinline__ cpx<df> pm<df>(cpx<df> p, cpx<df> v, bool up) {
  const cpx<df> w = up ? mk(-v.x, -v.y) : v;
  return mk(p.x + w.x, p.y + w.y);
}

// Twiddle sources of the cross-lane line FFTs.  TableTw reads e^{2 pi i j/N}
// from the global table per use; RegTw holds, for one lane position t, the
// M twiddles w^{t k2} and the twiddles of the cross-lane stages with span
// L > 4 in registers, for kernels whose threads keep one lane position
// across many lines.
template <typename R>
struct TableTw {
  const cpx<R>* __restrict__ tw;
  template <int S>
  __device__ __forceinline__ cpx<R> k2w(int t, int k2) const {
    return table_w<R, S>(tw, t * k2);  // t k2 < TPL M = N
  }
  template <int S, int N>
  __device__ __forceinline__ cpx<R> stage(int j, int L) const {
    return table_w<R, S>(tw, j * (N / L));
  }
};
template <typename R, int N, int TPL>
struct RegTw {
  static constexpr int M = N / TPL;
  static constexpr int NS = 3;  // stages with L = 8, 16, 32 (TPL <= 32)
  cpx<R> w[M];
  cpx<R> sw[NS];
  __device__ __forceinline__ void init(const cpx<R>* __restrict__ tw, int t) {
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) w[k2] = table_w<R, +1>(tw, t * k2);
#pragma unroll
    for (int si = 0; si < NS; ++si) {
      const int half = 4 << si;  // L = 2 half
      sw[si] = half < TPL ? table_w<R, +1>(tw, (t & (half - 1)) * (N / (2 * half))) : w[0];
    }
  }
  template <int S>
  __device__ __forceinline__ cpx<R> k2w(int, int k2) const {
    return S > 0 ? w[k2] : conj(w[k2]);
  }
  // L: the stage's span (8, 16, ...), a constant once the stage loop unrolls
  template <int S, int N_>
  __device__ __forceinline__ cpx<R> stage(int, int L) const {
    const int si = L >= 32 ? 2 : L >= 16 ? 1 : 0;  // L = 8, 16, 32
    return S > 0 ? sw[si] : conj(sw[si]);
  }
};

// Distribution A -> B.  t = lane index inside the group (0..TPL-1).
template <typename R, int N, int TPL, int S, typename TW>
__device__ __forceinline__ void fft_a2b(cpx<R> (&v)[N / TPL], int t, const TW& src) {
  constexpr int M = N / TPL;
  DFT<R, M, S>::run(v);
  if constexpr (TPL > 1) {
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) v[k2] = v[k2] * src.template k2w<S>(t, k2);
#pragma unroll
    for (int half = TPL / 2; half >= 1; half >>= 1) {
      const int L = 2 * half;
      const int j = t & (half - 1);
      const bool up = (t & half) != 0;
      if (L <= 4) {
        // twiddles of 2- and 4-point butterflies are 1 and S*i: one fused
        // +-1 multiply-add per component, then a swap for j = 1 (upper lanes)
        const bool rot = up && j == 1;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const cpx<R> p = shfl_xor(v[i], half);
          const cpx<R> d = pm(p, v[i], up);
          v[i] = rot ? mul_si<R, S>(d) : d;
        }
      } else {
        const cpx<R> W = src.template stage<S, N>(j, L);
#pragma unroll
        for (int i = 0; i < M; ++i) {
          cpx<R> p = shfl_xor(v[i], half);
          const cpx<R> d = pm(p, v[i], up);
          v[i] = up ? d * W : d;
        }
      }
    }
  }
}
template <typename R, int N, int TPL, int S>
__device__ __forceinline__ void fft_a2b(cpx<R> (&v)[N / TPL], int t, const cpx<R>* __restrict__ tw) {
  fft_a2b<R, N, TPL, S>(v, t, TableTw<R>{tw});
}

// Distribution B -> A (the transposed network of fft_a2b).
template <typename R, int N, int TPL, int S, typename TW>
__device__ __forceinline__ void fft_b2a(cpx<R> (&v)[N / TPL], int t, const TW& src) {
  constexpr int M = N / TPL;
  if constexpr (TPL > 1) {
#pragma unroll
    for (int half = 1; half < TPL; half <<= 1) {
      const int L = 2 * half;
      const int j = t & (half - 1);
      const bool up = (t & half) != 0;
      if (L <= 4) {
        const bool rot = up && j == 1;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const cpx<R> own = rot ? mul_si<R, S>(v[i]) : v[i];
          const cpx<R> p = shfl_xor(own, half);
          v[i] = pm(p, own, up);
        }
      } else {
        const cpx<R> W = src.template stage<S, N>(j, L);
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const cpx<R> own = up ? v[i] * W : v[i];
          const cpx<R> p = shfl_xor(own, half);
          v[i] = pm(p, own, up);
        }
      }
    }
#pragma unroll
    for (int k2 = 1; k2 < M; ++k2) v[k2] = v[k2] * src.template k2w<S>(t, k2);
  }
  DFT<R, M, S>::run(v);
}
template <typename R, int N, int TPL, int S>
__device__ __forceinline__ void fft_b2a(cpx<R> (&v)[N / TPL], int t, const cpx<R>* __restrict__ tw) {
  fft_b2a<R, N, TPL, S>(v, t, TableTw<R>{tw});
}

// position held by (lane t, register i) in each distribution
template <int N, int TPL>
__device__ __forceinline__ int pos_a(int t, int i) { return t + TPL * i; }
template <int N, int TPL>
__device__ __forceinline__ int pos_b(int t, int i) {
  return i + (N / TPL) * bitrev(t, ilog2c(TPL));
}
// signed frequency of grid position p (|n| < N/2 for every sphere member)
__device__ __forceinline__ int freq_of(int p, int N) { return p < N / 2 ? p : p - N; }
// True when register i of distribution A holds, in every lane, a frequency
// with |n| >= N/4.  The setup's aliasing guard keeps every sphere member at
// |n| < N/4 on each axis, so such a register is zero on the way in and
// unused on the way out; the condition folds to a constant once the
// register loops unroll, and the compiler drops that register's work.
__host__ __device__ constexpr bool a_outside(int N, int TPL, int i) {
  for (int t = 0; t < TPL; ++t) {
    const int p = t + TPL * i;
    const int f = p < N / 2 ? p : p - N;
    if ((f < 0 ? -f : f) < N / 4) return false;
  }
  return true;
}

}  // namespace pdep
