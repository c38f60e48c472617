// Plane-wave sphere <-> grid transforms (see transforms.cuh for the scheme).
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "fft.cuh"
#include "transforms.cuh"
#include "profile.cuh"

namespace pdep {


cudaError_t upload_local_twiddles() {
  static const int sizes[] = {6, 8, 10, 12, 16, 20, 24, 32, 48, 64};
  double2 hd[LOCAL_TW_SIZE];
  float2 hf[LOCAL_TW_SIZE];
  float4 hdf[LOCAL_TW_SIZE];
  const double two_pi = 6.283185307179586476925286766559;
  for (int M : sizes) {
    int off = local_tw_offset(M);
    for (int j = 0; j < M; ++j) {
      double a = two_pi * (double)j / (double)M;
      hd[off + j] = make_double2(cos(a), sin(a));
      hf[off + j] = make_float2((float)cos(a), (float)sin(a));
      const df re(cos(a)), im(sin(a));
      hdf[off + j] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_local_tw_d, hd, sizeof(hd));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_local_tw_df, hdf, sizeof(hdf));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_local_tw_f, hf, sizeof(hf));
}

// Lanes per line for each supported length (N / TPL registers per lane).
// Four lanes per line up to N = 64 measured faster than two for FP32 too:
// the extra shuffle stage costs less than the occupancy two-lane lines lose.
template <typename R, int N>
struct Tpl;
template <typename R> struct Tpl<R, 24> { static constexpr int v = 2; };
template <typename R> struct Tpl<R, 32> { static constexpr int v = 4; };
template <typename R> struct Tpl<R, 40> { static constexpr int v = 4; };
// 48-point FP32 lines: 4 lanes measured fastest per PDEP solve once the
// line FFTs skip the registers outside every sphere — half of each lane's
// 12 here — 2.4% ahead of 8 lanes and 26% ahead of 2
template <typename R> struct Tpl<R, 48> { static constexpr int v = 4; };
template <typename R> struct Tpl<R, 64> { static constexpr int v = 4; };
template <typename R> struct Tpl<R, 192> { static constexpr int v = 8; };

bool grid_supported(int N1, int N2, int N3) {
  bool n1 = (N1 == 24 || N1 == 32 || N1 == 40 || N1 == 48 || N1 == 64);
  bool cube = (N2 == N3) && (N2 == 24 || N2 == 32 || N2 == 40 || N2 == 48 || N2 == 64);
  bool slab = (N2 == 64 && N3 == 192);
  return n1 && (cube || slab);
}

// profile class of a launch by arithmetic type
template <typename R>
static int prof_class(int f64, int f32, int fdf) {
  return std::is_same<R, df>::value ? fdf : std::is_same<R, float>::value ? f32 : f64;
}

static __device__ __forceinline__ int iabs(int a) { return a < 0 ? -a : a; }

template <typename R>
__device__ __forceinline__ cpx<R> zero() { return mk(R(0), R(0)); }

template <typename R>
__device__ __forceinline__ R coef_of(int kind, const double* __restrict__ g2, int k) {
  if (kind == COEF_SQRT_COULOMB) return R(sqrt(12.566370614359172953850573533118 / g2[k]));
  return R(1);
}

// ---------------------------------------------------------------------------
// column pass: sphere -> x-lines (inverse transform, S = +1)
// ---------------------------------------------------------------------------
template <typename R, int N1>
__device__ __forceinline__ void cols_fwd_line(const SphereDev<R>& s,
                                              const typename Io<R>::T* __restrict__ x,
                                              long long ldx, const ItemMap& map, int nl,
                                              int coef, cpx<R>* __restrict__ b1, long long g,
                                              long long total);
template <typename R, int N1, typename TW>
__device__ __forceinline__ void xline_inverse(const SphereDev<R>& s,
                                              const typename Io<R>::T* __restrict__ x,
                                              long long ldx, const ItemMap& map, int nl, int coef,
                                              int item, int uc, bool live, cpx<R>* base,
                                              const TW& tws);

// resident 128-thread blocks per SM the column kernels ask for: the
// double-float ones up to 48-point lines are latency-bound like their slab
// (the 64-point ones would spill hundreds of bytes at four blocks)
template <typename R, int N1>
struct ColsMinBlocks {
  static constexpr int v = (std::is_same<R, df>::value && N1 <= 48) ? 4 : 1;
};

template <typename R, int N1>
__global__ void __launch_bounds__(128, ColsMinBlocks<R, N1>::v) k_cols_fwd(SphereDev<R> s,
                                                  const typename Io<R>::T* __restrict__ x,
                                                  long long ldx, ItemMap map, int n_items,
                                                  int coef, cpx<R>* __restrict__ b1) {
  const int nl = listed_count(map);
  const long long total = (long long)items_of(map, n_items, nl) * s.n_ucol;
  const int per = blockDim.x / Tpl<R, N1>::v;
  // the launch covers the largest count; blocks past the device count exit
  // (a grid-stride loop here costs 40-70% more registers)
  const long long g0 = (long long)blockIdx.x * per;
  if (g0 < total)
    cols_fwd_line<R, N1>(s, x, ldx, map, nl, coef, b1, g0 + threadIdx.x / Tpl<R, N1>::v, total);
}

template <typename R, int N1>
__device__ __forceinline__ void cols_fwd_line(const SphereDev<R>& s,
                                              const typename Io<R>::T* __restrict__ x,
                                              long long ldx, const ItemMap& map, int nl,
                                              int coef, cpx<R>* __restrict__ b1, long long g,
                                              long long total) {
  const bool live = g < total;
  const int item = live ? (int)(g / s.n_ucol) : 0;
  const int uc = live ? (int)(g - (long long)item * s.n_ucol) : 0;
  xline_inverse<R, N1>(s, x, ldx, map, nl, coef, item, uc, live,
                       b1 + (long long)item * N1 * s.n_col, TableTw<R>{s.tw1});
}

// x-line uc of item (both members of its mirror pair) from the sphere into
// the item's column scratch 'base' ([N1][n_col], global or shared memory);
// every lane of the warp must call it (the FFT shuffles), live or not.
template <typename R, int N1, typename TW>
__device__ __forceinline__ void xline_inverse(const SphereDev<R>& s,
                                              const typename Io<R>::T* __restrict__ x,
                                              long long ldx, const ItemMap& map, int nl, int coef,
                                              int item, int uc, bool live, cpx<R>* base,
                                              const TW& tws) {
  constexpr int TPL = Tpl<R, N1>::v;
  constexpr int M = N1 / TPL;
  const int t = threadIdx.x & (TPL - 1);
  const UCol c = s.ucol[live ? uc : 0];
  const bool active = live && ucol_in_range(s, c);
  const bool self = (c.col == c.mcol);
  const int ia = map.vec(item, 0, nl), ib = map.vec(item, 1, nl);
  using T = typename Io<R>::T;
  const T* xa = (active && ia >= 0) ? x + (long long)ia * ldx : nullptr;
  const T* xb = (active && ib >= 0) ? x + (long long)ib * ldx : nullptr;
  const R rs2 = R(0.70710678118654752440084436210485);

  cpx<R> v0[M], v1[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    v0[i] = zero<R>();
    v1[i] = zero<R>();
    if (a_outside(N1, TPL, i)) continue;
    const int n1 = freq_of(pos_a<N1, TPL>(t, i), N1);
    if (!active) continue;
    if (!self) {
      if (iabs(n1) <= c.R1) {
        // line c at n1: member k;  mirror line at n1: conj of member k'
        const int k = c.h0 + n1 + c.R1;
        const int k2 = c.h0 - n1 + c.R1;
        const R w = coef_of<R>(coef, s.g2, k) * rs2;
        const R w2 = coef_of<R>(coef, s.g2, k2) * rs2;
        cpx<R> A = xa ? mk(ld_io<R>(xa + 2 * k) * w, ld_io<R>(xa + 2 * k + 1) * w) : zero<R>();
        cpx<R> B = xb ? mk(ld_io<R>(xb + 2 * k) * w, ld_io<R>(xb + 2 * k + 1) * w) : zero<R>();
        v0[i] = mk(A.x - B.y, A.y + B.x);
        cpx<R> A2 = xa ? mk(ld_io<R>(xa + 2 * k2) * w2, ld_io<R>(xa + 2 * k2 + 1) * w2) : zero<R>();
        cpx<R> B2 = xb ? mk(ld_io<R>(xb + 2 * k2) * w2, ld_io<R>(xb + 2 * k2 + 1) * w2) : zero<R>();
        v1[i] = mk(A2.x + B2.y, B2.x - A2.y);
      }
    } else {
      if (n1 == 0) {
        const R w = (coef == COEF_ONE) ? R(1) : R(0);
        const int k0 = 2 * s.n_half;
        v0[i] = mk(xa ? ld_io<R>(xa + k0) * w : R(0), xb ? ld_io<R>(xb + k0) * w : R(0));
      } else if (iabs(n1) <= c.R1) {
        const int k = c.h0 + iabs(n1) - 1;
        const R w = coef_of<R>(coef, s.g2, k) * rs2;
        cpx<R> A = xa ? mk(ld_io<R>(xa + 2 * k) * w, ld_io<R>(xa + 2 * k + 1) * w) : zero<R>();
        cpx<R> B = xb ? mk(ld_io<R>(xb + 2 * k) * w, ld_io<R>(xb + 2 * k + 1) * w) : zero<R>();
        v0[i] = n1 > 0 ? mk(A.x - B.y, A.y + B.x) : mk(A.x + B.y, B.x - A.y);
      }
    }
  }
  fft_a2b<R, N1, TPL, +1>(v0, t, tws);
  fft_a2b<R, N1, TPL, +1>(v1, t, tws);
  if (!active) return;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int i1 = pos_b<N1, TPL>(t, i);
    base[(long long)i1 * s.n_col + c.col] = v0[i];
    if (!self) base[(long long)i1 * s.n_col + c.mcol] = v1[i];
  }
}

// ---------------------------------------------------------------------------
// column pass back: x-lines -> sphere (forward transform, S = -1), Hermitian
// unpacking of the two real fields and the epilogue
// ---------------------------------------------------------------------------
// One output vector's epilogue state.  FP32 (the transform of the inner
// CG): its output and input rows and its shift, set up once per line.
// FP64 and double-float: recomputed per element, which keeps their column
// kernels' register counts (precomputing raised the double-float 64-point
// one from 192 to 253).
template <typename R, bool Pre = std::is_same<R, float>::value>
struct OutRow;
template <typename R>
struct OutRow<R, true> {
  typename Io<R>::T* y_;
  const typename Io<R>::T* x_;  // null: no diagonal term
  R sh_;
  __device__ __forceinline__ OutRow(const Epilogue<R>& ep, int vec) {
    y_ = ep.y + (long long)(vec >= 0 ? vec : 0) * ep.ldy;
    x_ = ep.x_in ? ep.x_in + (long long)(vec >= 0 ? vec : 0) * ep.ldx : nullptr;
    sh_ = (ep.x_in && ep.shift && vec >= 0) ? ld_io<R>(ep.shift + vec % ep.shift_period) : R(0);
  }
  __device__ __forceinline__ typename Io<R>::T* y(const Epilogue<R>&) const { return y_; }
  __device__ __forceinline__ const typename Io<R>::T* x(const Epilogue<R>&) const { return x_; }
  __device__ __forceinline__ R sh(const Epilogue<R>&) const { return sh_; }
};
template <typename R>
struct OutRow<R, false> {
  int vec;
  __device__ __forceinline__ OutRow(const Epilogue<R>&, int v) : vec(v) {}
  __device__ __forceinline__ typename Io<R>::T* y(const Epilogue<R>& ep) const {
    return ep.y + (long long)vec * ep.ldy;
  }
  __device__ __forceinline__ const typename Io<R>::T* x(const Epilogue<R>& ep) const {
    return ep.x_in ? ep.x_in + (long long)vec * ep.ldx : nullptr;
  }
  __device__ __forceinline__ R sh(const Epilogue<R>& ep) const {
    return ep.shift ? ld_io<R>(ep.shift + vec % ep.shift_period) : R(0);
  }
};
template <typename R>
__device__ __forceinline__ void write_out(const Epilogue<R>& ep, const OutRow<R>& o, int j, R val,
                                          R coefv, R diag) {
  typename Io<R>::T* y = o.y(ep);
  R r = ep.scale * coefv * val;
  if (const typename Io<R>::T* x = o.x(ep)) r += (diag + o.sh(ep)) * ld_io<R>(x + j);
  if (ep.beta != 0) r += R(ep.beta) * ld_io<R>(y + j);
  y[j] = io_of<R>(r);
}

template <typename R, int N1>
__device__ __forceinline__ void cols_bwd_line(const SphereDev<R>& s,
                                              const cpx<R>* __restrict__ b1, const ItemMap& map,
                                              int nl, const Epilogue<R>& ep, long long g,
                                              long long total);
template <typename R, int N1, typename TW>
__device__ __forceinline__ void xline_forward(const SphereDev<R>& s, const cpx<R>* base,
                                              const ItemMap& map, int nl, const Epilogue<R>& ep,
                                              int item, int uc, bool live, const TW& tws);

template <typename R, int N1>
__global__ void __launch_bounds__(128, ColsMinBlocks<R, N1>::v) k_cols_bwd(SphereDev<R> s, const cpx<R>* __restrict__ b1,
                                                  ItemMap map, int n_items, Epilogue<R> ep) {
  const int nl = listed_count(map);
  const long long total = (long long)items_of(map, n_items, nl) * s.n_ucol;
  const int per = blockDim.x / Tpl<R, N1>::v;
  const long long g0 = (long long)blockIdx.x * per;
  if (g0 < total)
    cols_bwd_line<R, N1>(s, b1, map, nl, ep, g0 + threadIdx.x / Tpl<R, N1>::v, total);
}

template <typename R, int N1>
__device__ __forceinline__ void cols_bwd_line(const SphereDev<R>& s,
                                              const cpx<R>* __restrict__ b1, const ItemMap& map,
                                              int nl, const Epilogue<R>& ep, long long g,
                                              long long total) {
  const bool live = g < total;
  const int item = live ? (int)(g / s.n_ucol) : 0;
  const int uc = live ? (int)(g - (long long)item * s.n_ucol) : 0;
  xline_forward<R, N1>(s, b1 + (long long)item * N1 * s.n_col, map, nl, ep, item, uc, live,
                       TableTw<R>{s.tw1});
}

// x-line uc of item from its column scratch 'base' back to the sphere, the
// two real fields unpacked, through the epilogue; every lane of the warp
// must call it.
template <typename R, int N1, typename TW>
__device__ __forceinline__ void xline_forward(const SphereDev<R>& s, const cpx<R>* base,
                                              const ItemMap& map, int nl, const Epilogue<R>& ep,
                                              int item, int uc, bool live, const TW& tws) {
  constexpr int TPL = Tpl<R, N1>::v;
  constexpr int M = N1 / TPL;
  const int lane = threadIdx.x & 31;
  const int t = threadIdx.x & (TPL - 1);
  const UCol c = s.ucol[live ? uc : 0];
  const bool active = live && ucol_in_range(s, c);
  const bool self = (c.col == c.mcol);

  cpx<R> v0[M], v1[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int i1 = pos_b<N1, TPL>(t, i);
    v0[i] = active ? base[(long long)i1 * s.n_col + c.col] : zero<R>();
    v1[i] = (active && !self) ? base[(long long)i1 * s.n_col + c.mcol] : zero<R>();
  }
  fft_b2a<R, N1, TPL, -1>(v0, t, tws);
  fft_b2a<R, N1, TPL, -1>(v1, t, tws);

  const int src = (lane & ~(TPL - 1)) | ((TPL - t) & (TPL - 1));
  const int ia = map.vec(item, 0, nl), ib = map.vec(item, 1, nl);
  const OutRow<R> oa(ep, ia), ob(ep, ib);
  const R rs2 = R(0.70710678118654752440084436210485);
#pragma unroll
  for (int i = 0; i < M; ++i) {
    if (a_outside(N1, TPL, i)) continue;  // the same i in every lane
    // value of the mirror line at position (N1 - p) mod N1
    cpx<R> send = self ? v0[M - 1 - i] : v1[M - 1 - i];
    cpx<R> dm = shfl_idx(send, src);
    if (t == 0) dm = self ? v0[(M - i) % M] : v1[(M - i) % M];
    if (!active) continue;
    const int n1 = freq_of(pos_a<N1, TPL>(t, i), N1);
    int k = -1;
    if (!self) {
      if (iabs(n1) <= c.R1) k = c.h0 + n1 + c.R1;
    } else if (n1 > 0 && n1 <= c.R1) {
      k = c.h0 + n1 - 1;
    }
    const cpx<R> d = v0[i];
    if (k >= 0) {
      const cpx<R> sa = d + conj(dm);   // 2 Va
      const cpx<R> sb = d - conj(dm);   // 2 i Vb
      const R cf = coef_of<R>(ep.coef, s.g2, k);
      const R dg = ep.kin * s.kin[k];
      if (ia >= 0) {
        write_out(ep, oa, 2 * k, rs2 * sa.x, cf, dg);
        write_out(ep, oa, 2 * k + 1, rs2 * sa.y, cf, dg);
      }
      if (ib >= 0) {
        write_out(ep, ob, 2 * k, rs2 * sb.y, cf, dg);
        write_out(ep, ob, 2 * k + 1, -rs2 * sb.x, cf, dg);
      }
    } else if (self && n1 == 0) {
      const R cf = (ep.coef == COEF_ONE) ? R(1) : R(0);
      const int j0 = 2 * s.n_half;
      if (ia >= 0) write_out(ep, oa, j0, d.x, cf, R(0));
      if (ib >= 0) write_out(ep, ob, j0, d.y, cf, R(0));
    }
  }
}

// ---------------------------------------------------------------------------
// slab pass: one x-plane i1 of one item (or of one group for DENSITY)
// ---------------------------------------------------------------------------
// largest block a slab of this shape launches with: every z-line (N2 lines)
// or every y-line (at most N3/2 + 1 planes) in one round
template <typename R, int N2, int N3>
struct SlabThreads {
  static constexpr int z = N2 * Tpl<R, N3>::v;
  static constexpr int y = (N3 / 2 + 1) * Tpl<R, N2>::v;
  static constexpr int v = (((z > y ? z : y) + 31) / 32) * 32;
};
// FP32 slabs keep three blocks of up to 256 threads per SM resident
// (register budget ~85-110); FP64 slabs are bound by the FP64 pipe at one
// block per SM.
// Double-float slabs run on the FP32 pipe and are latency-bound (ncu on 48^3
// at two blocks: 12 warps per SM, issue active 33%, short-scoreboard and
// wait stalls first): more resident blocks win although they spill — on
// 48^3, three blocks (64 bytes spilled) made the PDEP step 3.2% faster and
// four (184 bytes) 1.9% more; other shapes keep three.
template <typename R, int N2, int N3>
struct SlabMinBlocks {
  static constexpr int t = SlabThreads<R, N2, N3>::v;
  static constexpr int v = std::is_same<R, df>::value ? (t <= 192 ? (N2 == 48 ? 4 : 3) : 1)
                           : sizeof(R) != 4                ? 1
                           : t <= 128                      ? 384 / t
                           : t <= 256                      ? 3
                           : t <= 384                      ? 2
                                                           : 1;
};
// Row stride of the (n3, i2) shared-memory plane (FP32 rows padded by 8
// complex) and, in FP32, a column swizzle: element (row, col) sits at
// row * TS + (col ^ (row & 7)).  The swizzle stays inside each aligned block
// of 8 columns (N2 is a multiple of 8) and spreads the eight y-line slots a
// warp touches, whose four lanes' positions are 12 complex apart, over all
// banks (a third of the shared-memory wavefronts of the LSU-bound FP32 slab);
// the four n3 rows of a z-line access keep their distinct halves.  FP64 slabs
// are FP64-pipe bound and keep the plain layout: the swizzle's index
// arithmetic costs them a resident block per SM.
template <typename R, int N2>
struct T2Stride {
  static constexpr int v = sizeof(R) == 4 ? N2 + 8 : N2;
};
template <typename R>
__device__ __forceinline__ int t2_at(int row, int col, int ts) {
  if constexpr (sizeof(R) == 4) return row * ts + (col ^ (row & 7));
  return row * ts + col;
}

// tid / nthreads: the thread's index in, and the size of, the (warp-aligned)
// group of threads that transforms this plane
template <typename R, int N2, typename TW>
__device__ __forceinline__ void y_inverse(const SphereDev<R>& s, const cpx<R>* S1, cpx<R>* T2,
                                          int tid, int nthreads, const TW& tws) {
  constexpr int TL = Tpl<R, N2>::v;
  constexpr int TS = T2Stride<R, N2>::v;
  constexpr int M = N2 / TL;
  const int nslot = 2 * s.R3 + 1;
  const int per = nthreads / TL;
  const int t = tid & (TL - 1);
  // first slot of this warp in a round: warps whose slots all lie past the
  // last (n3) row skip the line FFTs instead of transforming zeros
  const int wslot0 = (tid & ~31) / TL;
  for (int base = 0; base < nslot; base += per) {
    if (base + wslot0 >= nslot) break;
    const int sl = base + tid / TL;
    const bool live = sl < nslot;
    const int2 info = live ? s.slot[sl] : make_int2(-1, 0);
    const bool act = live && slot_in_range(s, info);
    cpx<R> v[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int n2 = freq_of(pos_a<N2, TL>(t, i), N2);
      v[i] = (!a_outside(N2, TL, i) && act && iabs(n2) <= info.x) ? S1[info.y + n2 + info.x]
                                                                   : zero<R>();
    }
    fft_a2b<R, N2, TL, +1>(v, t, tws);
    if (act) {
#pragma unroll
      for (int i = 0; i < M; ++i) T2[t2_at<R>(sl, pos_b<N2, TL>(t, i), TS)] = v[i];
    }
  }
}

template <typename R, int N2, typename TW>
__device__ __forceinline__ void y_forward(const SphereDev<R>& s, const cpx<R>* T2, cpx<R>* S1,
                                          int tid, int nthreads, const TW& tws) {
  constexpr int TL = Tpl<R, N2>::v;
  constexpr int TS = T2Stride<R, N2>::v;
  constexpr int M = N2 / TL;
  const int nslot = 2 * s.R3 + 1;
  const int per = nthreads / TL;
  const int t = tid & (TL - 1);
  const int wslot0 = (tid & ~31) / TL;
  for (int base = 0; base < nslot; base += per) {
    if (base + wslot0 >= nslot) break;
    const int sl = base + tid / TL;
    const bool live = sl < nslot;
    const int2 info = live ? s.slot[sl] : make_int2(-1, 0);
    const bool act = live && slot_in_range(s, info);
    cpx<R> v[M];
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = act ? T2[t2_at<R>(sl, pos_b<N2, TL>(t, i), TS)] : zero<R>();
    fft_b2a<R, N2, TL, -1>(v, t, tws);
    if (act) {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        if (a_outside(N2, TL, i)) continue;
        const int n2 = freq_of(pos_a<N2, TL>(t, i), N2);
        if (iabs(n2) <= info.x) S1[info.y + n2 + info.x] = v[i];
      }
    }
  }
}

// one x-plane i1 of one item
template <typename R, int N2, int N3>
__device__ __forceinline__ void slab_unit(const SphereDev<R>& s, const SlabArgs<R>& a, int nl,
                                          int item, int i1, cpx<R>* S1, cpx<R>* T2) {
  constexpr int TL3 = Tpl<R, N3>::v;
  constexpr int M3 = N3 / TL3;
  constexpr int TS = T2Stride<R, N2>::v;
  const int R3 = s.R3;
  const int t3 = threadIdx.x & (TL3 - 1);
  const int zper = blockDim.x / TL3;
  const long long plane = (long long)i1 * N2 * N3;

  cpx<R>* row = a.b1 + ((long long)item * s.N1 + i1) * s.n_col;
  if (a.mode != SLAB_FROM_GRID) {
    for (int j = threadIdx.x; j < s.n_col; j += blockDim.x) S1[j] = row[j];
    __syncthreads();
    y_inverse<R, N2>(s, S1, T2, threadIdx.x, blockDim.x, TableTw<R>{s.tw2});
    __syncthreads();
  }

  for (int base = 0; base < N2; base += zper) {
    const int i2 = base + threadIdx.x / TL3;
    const bool act = i2 < N2;
    cpx<R> v[M3];
    if (a.mode == SLAB_FROM_GRID) {
      const int grp = item / a.map.items_per_group;
      const int w = item - grp * a.map.items_per_group;
      const int va = 2 * w, vb = 2 * w + 1;
      const long long off = plane + (long long)i2 * N3;
      using T = typename Io<R>::T;
      const T* f = (act && a.src.f) ? a.src.f + (long long)grp * a.src.f_stride + off : nullptr;
      const T* ga = act ? a.src.g + (long long)va * a.src.g_stride + off : nullptr;
      const T* gb = (act && vb < a.map.vecs_per_group) ? a.src.g + (long long)vb * a.src.g_stride + off
                                                        : nullptr;
#pragma unroll
      for (int i = 0; i < M3; ++i) {
        const int i3 = pos_b<N3, TL3>(t3, i);
        const R fv = f ? ld_io<R>(f + i3) : R(1);
        v[i] = act ? mk(fv * ld_io<R>(ga + i3), gb ? fv * ld_io<R>(gb + i3) : R(0)) : zero<R>();
      }
    } else {
#pragma unroll
      for (int i = 0; i < M3; ++i) {
        const int n3 = freq_of(pos_a<N3, TL3>(t3, i), N3);
        v[i] = (act && iabs(n3) <= R3) ? T2[t2_at<R>(n3 + R3, i2, TS)] : zero<R>();
      }
      fft_a2b<R, N3, TL3, +1>(v, t3, s.tw3);
      if (a.mode == SLAB_TO_GRID) {
        if (act) {
          const int ia = a.map.vec(item, 0, nl), ib = a.map.vec(item, 1, nl);
          const long long off = plane + (long long)i2 * N3;
          typename Io<R>::T* oa = ia >= 0 ? a.out + (long long)ia * a.out_stride + off : nullptr;
          typename Io<R>::T* ob = ib >= 0 ? a.out + (long long)ib * a.out_stride + off : nullptr;
#pragma unroll
          for (int i = 0; i < M3; ++i) {
            const int i3 = pos_b<N3, TL3>(t3, i);
            if (oa) oa[i3] = io_of<R>(v[i].x * R(a.out_scale));
            if (ob) ob[i3] = io_of<R>(v[i].y * R(a.out_scale));
          }
        }
        continue;
      }
      {
        if (a.dn && act) {
          // density response of the two vectors of the item on this z-line
          // (Eq. deltani), accumulated over the occupied states v
          const int ia = a.map.vec(item, 0, nl), ib = a.map.vec(item, 1, nl);
          const long long off = plane + (long long)i2 * N3;
          const int ja = ia / a.dn_nocc, vb_a = ia - ja * a.dn_nocc;
          const double* ua = a.u + (long long)vb_a * a.dn_stride + off;
          double* da = a.dn + (long long)ja * a.dn_stride + off;
          const int jb = ib >= 0 ? ib / a.dn_nocc : -1;
          const double* ub = ib >= 0 ? a.u + (long long)(ib - jb * a.dn_nocc) * a.dn_stride + off
                                     : nullptr;
          double* db = ib >= 0 ? a.dn + (long long)jb * a.dn_stride + off : nullptr;
          const double sc = a.dn_scale;
#pragma unroll
          for (int i = 0; i < M3; ++i) {
            const int i3 = pos_b<N3, TL3>(t3, i);
            const double ca = sc * as_double(v[i].x) * ua[i3];
            if (ub) {
              const double cb = sc * as_double(v[i].y) * ub[i3];
              if (jb == ja) {
                atomicAdd(da + i3, ca + cb);
              } else {
                atomicAdd(da + i3, ca);
                atomicAdd(db + i3, cb);
              }
            } else {
              atomicAdd(da + i3, ca);
            }
          }
        }
      }
      // SLAB_HPSI: multiply by the local potential on the grid
      const R* vr = a.v + plane + (long long)i2 * N3;
#pragma unroll
      for (int i = 0; i < M3; ++i) v[i] = scale(v[i], act ? vr[pos_b<N3, TL3>(t3, i)] : R(0));
    }
    fft_b2a<R, N3, TL3, -1>(v, t3, s.tw3);
    if (act) {
#pragma unroll
      for (int i = 0; i < M3; ++i) {
        const int n3 = freq_of(pos_a<N3, TL3>(t3, i), N3);
        if (iabs(n3) <= R3) T2[t2_at<R>(n3 + R3, i2, TS)] = v[i];
      }
    }
  }
  if (a.mode == SLAB_TO_GRID) return;
  __syncthreads();
  y_forward<R, N2>(s, T2, S1, threadIdx.x, blockDim.x, TableTw<R>{s.tw2});
  __syncthreads();
  for (int j = threadIdx.x; j < s.n_col; j += blockDim.x) row[j] = S1[j];
}

// FP64 and double-float: one block per (item, x-plane i1), grid (largest
// item count, N1); with a device count, blocks past it exit at once.
// FP32: a persistent grid of the resident blocks strides over the
// (item, plane) units, so a launch sized for a whole batch whose device
// count has shrunk costs no empty blocks (for the FP32 slab the loop costs
// no registers, unlike the FP64 one).
template <typename R, int N2, int N3>
__global__ void __launch_bounds__(SlabThreads<R, N2, N3>::v, (SlabMinBlocks<R, N2, N3>::v))
    k_slab(SphereDev<R> s, SlabArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* S1 = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* T2 = S1 + s.n_col;
  const int nl = listed_count(a.map);
  const int n_items = items_of(a.map, a.n_items, nl);
  if constexpr (std::is_same<R, float>::value) {
    const int units = n_items * s.N1;
#pragma unroll 1
    for (int w = blockIdx.x; w < units; w += gridDim.x) {
      const int item = w / s.N1;
      __syncthreads();  // the previous unit's shared-memory reads are done
      slab_unit<R, N2, N3>(s, a, nl, item, w - item * s.N1, S1, T2);
    }
  } else {
    const int item = blockIdx.x;
    if (item >= n_items) return;
    slab_unit<R, N2, N3>(s, a, nl, item, blockIdx.y, S1, T2);
  }
}

// ---------------------------------------------------------------------------
// fused FP32 H x: the whole transform of one item in one block
// ---------------------------------------------------------------------------
// For cubic grids whose column scratch of one item (N x n_col complex) fits
// in shared memory (24^3 .. 48^3), one block of 512 threads runs, per item:
// the x-line inverse FFTs of every column into shared memory, then the y and
// z passes of G x-planes at a time (each plane on its own warp-aligned group
// of 512/G threads, the potential multiplied between the z inverse and
// forward FFTs), then the x-line forward FFTs with the epilogue.  The column
// scratch never leaves the SM: per item the HBM traffic is the two input
// vectors (read for the transform and for the diagonal term) and the two
// outputs, against a write, a read-modify-write and a read of the whole
// scratch by the three-launch form.  Blocks are persistent over the items.
constexpr int FUSED_THREADS = 512;

// z-lines of one x-plane (T2: its (n3 slot, i2) plane), the potential
// multiplied on the grid between the inverse and forward FFTs
template <int N, typename TW>
__device__ __forceinline__ void z_hpsi(const SphereDev<float>& s, cpx<float>* T2,
                                       const float* __restrict__ vplane, int tid, int nthreads,
                                       const TW& tws) {
  constexpr int TL3 = Tpl<float, N>::v;
  constexpr int M3 = N / TL3;
  constexpr int TS = T2Stride<float, N>::v;
  const int R3 = s.R3;
  const int t3 = tid & (TL3 - 1);
  const int zper = nthreads / TL3;
  for (int base = 0; base < N; base += zper) {
    const int i2 = base + tid / TL3;
    const bool act = i2 < N;
    cpx<float> v[M3];
#pragma unroll
    for (int i = 0; i < M3; ++i) {
      const int n3 = freq_of(pos_a<N, TL3>(t3, i), N);
      v[i] = (!a_outside(N, TL3, i) && act && iabs(n3) <= R3) ? T2[t2_at<float>(n3 + R3, i2, TS)]
                                                              : zero<float>();
    }
    fft_a2b<float, N, TL3, +1>(v, t3, tws);
    // this lane's M3 (even) potential values are consecutive: 8-byte loads
    const float* vr = vplane + (act ? i2 : 0) * N + pos_b<N, TL3>(t3, 0);
    static_assert(M3 % 2 == 0, "paired potential loads");
#pragma unroll
    for (int i = 0; i < M3; i += 2) {
      const float2 f = act ? __ldg(reinterpret_cast<const float2*>(vr + i)) : make_float2(0.f, 0.f);
      v[i] = scale(v[i], f.x);
      v[i + 1] = scale(v[i + 1], f.y);
    }
    fft_b2a<float, N, TL3, -1>(v, t3, tws);
    if (act) {
#pragma unroll
      for (int i = 0; i < M3; ++i) {
        if (a_outside(N, TL3, i)) continue;
        const int n3 = freq_of(pos_a<N, TL3>(t3, i), N);
        if (iabs(n3) <= R3) T2[t2_at<float>(n3 + R3, i2, TS)] = v[i];
      }
    }
  }
}

// barrier of the warps of plane group g (nthreads of them, warp-aligned)
__device__ __forceinline__ void group_sync(int g, int nthreads) {
  if (nthreads == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(nthreads) : "memory");
  }
}

template <int N>
__global__ void __launch_bounds__(FUSED_THREADS, 1)
    k_hpsi_fused(SphereDev<float> s, const float* __restrict__ x, long long ldx, ItemMap map,
                 int n_items, const float* __restrict__ v, Epilogue<float> ep, int G,
                 DevTimer* timer, double item_flops, double item_bytes) {
  const unsigned long long t0 = dev_clock_ns();
  constexpr int TL = Tpl<float, N>::v;
  constexpr int TS = T2Stride<float, N>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<float>* B1 = reinterpret_cast<cpx<float>*>(smem_raw);
  const int nslot = 2 * s.R3 + 1;
  const int nl = listed_count(map);
  const int items = items_of(map, n_items, nl);
  const int VT = blockDim.x / G;  // threads per plane: a multiple of 32
  const int g = threadIdx.x / VT;
  const int vt = threadIdx.x - g * VT;
  cpx<float>* T2 = B1 + (size_t)N * s.n_col + (size_t)g * nslot * TS;
  const int lines = blockDim.x / TL;
  // a cubic grid: the x, y and z lines have one length and one twiddle
  // table, and every pass keeps this thread at lane position t of its lines
  RegTw<float, N, TL> rtw;
  rtw.init(s.tw1, threadIdx.x & (TL - 1));
#pragma unroll 1
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    __syncthreads();  // the previous item's reads of B1 are done
#pragma unroll 1
    for (int base = 0; base < s.n_ucol; base += lines) {
      const int uc = base + threadIdx.x / TL;
      xline_inverse<float, N>(s, x, ldx, map, nl, COEF_ONE, item, uc, uc < s.n_ucol, B1, rtw);
    }
    __syncthreads();
    // the plane groups touch disjoint data (their own plane row of B1 and
    // their own T2), so each synchronises only its own warps: one warp with
    // __syncwarp, several with a named barrier (ids 1..G)
#pragma unroll 1
    for (int p0 = 0; p0 < N; p0 += G) {
      const int i1 = p0 + g;
      if (i1 < N) {  // uniform over the plane group's warps
        cpx<float>* S1 = B1 + (size_t)i1 * s.n_col;
        y_inverse<float, N>(s, S1, T2, vt, VT, rtw);
        group_sync(g, VT);
        z_hpsi<N>(s, T2, v + (size_t)i1 * N * N, vt, VT, rtw);
        group_sync(g, VT);
        y_forward<float, N>(s, T2, S1, vt, VT, rtw);
        group_sync(g, VT);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int base = 0; base < s.n_ucol; base += lines) {
      const int uc = base + threadIdx.x / TL;
      xline_forward<float, N>(s, B1, map, nl, ep, item, uc, uc < s.n_ucol, rtw);
    }
  }
  if (threadIdx.x == 0) {
    const int mine = items > (int)blockIdx.x ? (items - 1 - (int)blockIdx.x) / gridDim.x + 1 : 0;
    dev_timer_block_end(timer, t0, mine * item_flops, mine * item_bytes);
  }
}

// resident blocks per SM of a kernel at a block size and shared memory
// (queried once per combination)
template <typename K>
static int occupancy(K kern, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_tuple((const void*)kern, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem) != cudaSuccess || o < 1) {
    cudaGetLastError();
    o = 1;
  }
  cache[key] = o;
  return o;
}

static int sm_count() {
  static const int n = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 152;
  }();
  return n;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t slab_smem_bytes(int n_col, int R3, int N2, size_t elem) {
  const int ts = elem == 4 ? N2 + 8 : N2;  // T2Stride
  return (size_t)(n_col + (2 * R3 + 1) * ts) * 2 * elem;
}

template <typename R, int N>
static int threads_for(int lines) {
  int n = lines * Tpl<R, N>::v;
  return ((n + 31) / 32) * 32;
}

template <typename R, int N1>
static cudaError_t cols_fwd_impl(const SphereDev<R>& s, const typename Io<R>::T* x, long long ldx,
                                 ItemMap map,
                                 int n_items, int coef, cpx<R>* b1, cudaStream_t st) {
  const int per = 128 / Tpl<R, N1>::v;
  const long long total = (long long)n_items * s.n_ucol;
  if (total == 0) return cudaSuccess;
  const long long blocks = (total + per - 1) / per;
  // one x-line per column (n_col lines per item): 5 L log2 L flops each
  const double lines = (double)n_items * s.n_col;
  ProfScope ps(prof_class<R>(PC_COLS_F64, PC_COLS_F32, PC_COLS_DF), st,
               lines * 5.0 * N1 * log2((double)N1),
               (double)n_items * 2.0 * s.n_pw * sizeof(typename Io<R>::T) +
                   lines * N1 * 2.0 * sizeof(R),
               map.list ? map.n_dev : nullptr, map.n_list);
  count_launch();
  k_cols_fwd<R, N1><<<(unsigned)blocks, 128, 0, st>>>(s, x, ldx, map, n_items, coef, b1);
  return cudaGetLastError();
}

template <typename R, int N1>
static cudaError_t cols_bwd_impl(const SphereDev<R>& s, const cpx<R>* b1, ItemMap map,
                                 int n_items, const Epilogue<R>& ep, cudaStream_t st) {
  const int per = 128 / Tpl<R, N1>::v;
  const long long total = (long long)n_items * s.n_ucol;
  if (total == 0) return cudaSuccess;
  const long long blocks = (total + per - 1) / per;
  const double lines = (double)n_items * s.n_col;
  const double vecs = (double)n_items * 2.0 * s.n_pw * sizeof(typename Io<R>::T);
  ProfScope ps(prof_class<R>(PC_COLS_F64, PC_COLS_F32, PC_COLS_DF), st,
               lines * 5.0 * N1 * log2((double)N1),
               lines * N1 * 2.0 * sizeof(R) + vecs * (1.0 + (ep.x_in ? 1.0 : 0.0) +
                                                      (ep.beta != 0 ? 1.0 : 0.0)),
               map.list ? map.n_dev : nullptr, map.n_list);
  count_launch();
  k_cols_bwd<R, N1><<<(unsigned)blocks, 128, 0, st>>>(s, b1, map, n_items, ep);
  return cudaGetLastError();
}

template <typename R, int N2, int N3>
static cudaError_t slab_impl(const SphereDev<R>& s, const SlabArgs<R>& a, cudaStream_t st) {
  int nt = threads_for<R, N3>(N2);
  int ny = threads_for<R, N2>(2 * s.R3 + 1);
  if (ny > nt) nt = ny;
  if (nt > SlabThreads<R, N2, N3>::v) return cudaErrorInvalidConfiguration;
  const size_t smem = slab_smem_bytes(s.n_col, s.R3, N2, sizeof(R));
  auto kern = k_slab<R, N2, N3>;
  static std::atomic<bool> attr_set{false};  // per instantiation; raised once
  if (!attr_set.load()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set.store(true);
  }
  const int gx = a.n_items;
  if (gx == 0) return cudaSuccess;
  dim3 grid(gx, s.N1);
  if (std::is_same<R, float>::value) {
    const long long units = (long long)gx * s.N1;
    grid = dim3((unsigned)std::min<long long>(units, (long long)occupancy(kern, nt, smem) * sm_count()));
  }
  // algorithmic work: y-lines over the |n3| <= R3 planes and z-lines over the
  // N2 rows of each x-plane, 5 L log2 L flops per complex line FFT
  const double ylines = (double)(2 * s.R3 + 1), zlines = (double)N2;
  const double fy = 5.0 * N2 * log2((double)N2), fz = 5.0 * N3 * log2((double)N3);
  const double planes = (double)a.n_items * s.N1;
  const double colb = (double)s.n_col * 2.0 * sizeof(R);     // one plane of B1
  const double gridb = (double)N2 * N3 * sizeof(R);          // one plane of a real grid
  double fl = 0, by = 0;
  switch (a.mode) {
    case SLAB_HPSI: fl = planes * (2 * ylines * fy + 2 * zlines * fz + 2.0 * N2 * N3);
                    by = planes * 2 * colb + s.N1 * gridb;
                    if (a.dn) {
                      // density response: 2 products per point and vector; dn
                      // read and written once per perturbation, u read once
                      fl += planes * 4.0 * N2 * N3;
                      by += (2.0 * a.n_items / a.dn_nocc) * s.N1 * 2.0 * gridb +
                            (double)a.dn_nocc * s.N1 * gridb;
                    }
                    break;
    case SLAB_TO_GRID: fl = planes * (ylines * fy + zlines * fz);
                       by = planes * (colb + 2 * gridb); break;
    case SLAB_FROM_GRID: fl = planes * (ylines * fy + zlines * fz + 3.0 * N2 * N3);
                         by = planes * (colb + 3 * gridb); break;
  }
  ProfScope ps(prof_class<R>(PC_SLAB_F64, PC_SLAB_F32, PC_SLAB_DF), st, fl, by,
               a.map.list ? a.map.n_dev : nullptr, a.map.n_list);
  count_launch();
  kern<<<grid, nt, smem, st>>>(s, a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cols_fwd(const SphereDev<R>& s, const typename Io<R>::T* x, long long ldx,
                            ItemMap map, int n_items, int coef, cpx<R>* b1, cudaStream_t st) {
  switch (s.N1) {
    case 24: return cols_fwd_impl<R, 24>(s, x, ldx, map, n_items, coef, b1, st);
    case 32: return cols_fwd_impl<R, 32>(s, x, ldx, map, n_items, coef, b1, st);
    case 40: return cols_fwd_impl<R, 40>(s, x, ldx, map, n_items, coef, b1, st);
    case 48: return cols_fwd_impl<R, 48>(s, x, ldx, map, n_items, coef, b1, st);
    case 64: return cols_fwd_impl<R, 64>(s, x, ldx, map, n_items, coef, b1, st);
  }
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_cols_bwd(const SphereDev<R>& s, const cpx<R>* b1, ItemMap map, int n_items,
                            const Epilogue<R>& ep, cudaStream_t st) {
  switch (s.N1) {
    case 24: return cols_bwd_impl<R, 24>(s, b1, map, n_items, ep, st);
    case 32: return cols_bwd_impl<R, 32>(s, b1, map, n_items, ep, st);
    case 40: return cols_bwd_impl<R, 40>(s, b1, map, n_items, ep, st);
    case 48: return cols_bwd_impl<R, 48>(s, b1, map, n_items, ep, st);
    case 64: return cols_bwd_impl<R, 64>(s, b1, map, n_items, ep, st);
  }
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_slab(const SphereDev<R>& s, const SlabArgs<R>& a, cudaStream_t st) {
  if (s.N2 == s.N3) {
    switch (s.N2) {
      case 24: return slab_impl<R, 24, 24>(s, a, st);
      case 32: return slab_impl<R, 32, 32>(s, a, st);
      case 40: return slab_impl<R, 40, 40>(s, a, st);
      case 48: return slab_impl<R, 48, 48>(s, a, st);
      case 64: return slab_impl<R, 64, 64>(s, a, st);
    }
  } else if (s.N2 == 64 && s.N3 == 192) {
    return slab_impl<R, 64, 192>(s, a, st);
  }
  return cudaErrorInvalidValue;
}

// planes per group of the fused kernel: the fewest planes whose thread
// group (a power of two, at least a warp) covers every y-line slot at once
static int fused_planes(int nslot, int tl) {
  int vt = 32;
  while (vt < nslot * tl && vt < FUSED_THREADS) vt *= 2;
  return FUSED_THREADS / vt;
}

// groups of more than one warp synchronise on named barriers 1..G, and the
// hardware has barriers 0..15 only
static bool fused_barriers_ok(int G) { return FUSED_THREADS / G == 32 || G <= 15; }

static int fused_tl(int N) {
  switch (N) {
    case 24: return Tpl<float, 24>::v;
    case 32: return Tpl<float, 32>::v;
    case 40: return Tpl<float, 40>::v;
    case 48: return Tpl<float, 48>::v;
  }
  return 0;
}

int hpsi_fused_planes(const SphereDev<float>& s, int planes) {
  const int tl = fused_tl(s.N1);
  if (!tl) return 0;
  const int nslot = 2 * s.R3 + 1;
  const int G0 = fused_planes(nslot, tl);
  // a requested group must be a power of two whose thread groups (512/G
  // threads) are at least a warp; fewer threads than a plane's y-lines take
  // two rounds per pass
  if (planes > 0 && FUSED_THREADS / planes >= 32 && (planes & (planes - 1)) == 0 &&
      fused_barriers_ok(planes))
    return planes;
  return fused_barriers_ok(G0) ? G0 : 0;
}

size_t hpsi_fused_smem(const SphereDev<float>& s, int planes) {
  if (s.N1 != s.N2 || s.N2 != s.N3 || !fused_tl(s.N1)) return 0;
  const int nslot = 2 * s.R3 + 1;
  const int G = hpsi_fused_planes(s, planes);
  if (G <= 0) return 0;
  const size_t bytes = ((size_t)s.N1 * s.n_col + (size_t)G * nslot * (s.N2 + 8)) * sizeof(cpx<float>);
  return bytes <= 225 * 1024 ? bytes : 0;
}

template <int N>
static cudaError_t hpsi_fused_impl(const SphereDev<float>& s, const float* x, long long ldx,
                                   ItemMap map, int n_items, const float* v,
                                   const Epilogue<float>& ep, size_t smem, int G,
                                   cudaStream_t st) {
  auto kern = k_hpsi_fused<N>;
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         225 * 1024);
    if (e != cudaSuccess) return e;
    attr_set.store(true);
  }
  const unsigned grid = (unsigned)std::min<long long>(
      n_items, (long long)occupancy(kern, FUSED_THREADS, smem) * sm_count());
  // algorithmic work: as the three launches it replaces (x-lines both ways,
  // y- and z-lines both ways, V products); bytes: the vectors only
  const double planes = (double)n_items * s.N1;
  const double fl = (double)n_items * 2.0 * s.n_col * 5.0 * N * log2((double)N) +
                    planes * (2.0 * (2 * s.R3 + 1) * 5.0 * N * log2((double)N) +
                              2.0 * N * 5.0 * N * log2((double)N) + 2.0 * N * N);
  const double by = (double)n_items * 2.0 * s.n_pw * sizeof(float) * 3.0;
  // timed on the device (this kernel also runs inside the CG graphs): the
  // work is counted per processed item
  count_launch();
  kern<<<grid, FUSED_THREADS, smem, st>>>(s, x, ldx, map, n_items, v, ep, G,
                                          dev_timer(PC_HPSI_FUSED), fl / n_items, by / n_items);
  return cudaGetLastError();
}

cudaError_t launch_hpsi_fused(const SphereDev<float>& s, const float* x, long long ldx, ItemMap map,
                              int n_items, const float* v, const Epilogue<float>& ep,
                              cudaStream_t st, int planes) {
  const size_t smem = hpsi_fused_smem(s, planes);
  if (smem == 0) return cudaErrorInvalidValue;
  if (n_items <= 0) return cudaSuccess;
  const int G = hpsi_fused_planes(s, planes);
  switch (s.N1) {
    case 24: return hpsi_fused_impl<24>(s, x, ldx, map, n_items, v, ep, smem, G, st);
    case 32: return hpsi_fused_impl<32>(s, x, ldx, map, n_items, v, ep, smem, G, st);
    case 40: return hpsi_fused_impl<40>(s, x, ldx, map, n_items, v, ep, smem, G, st);
    case 48: return hpsi_fused_impl<48>(s, x, ldx, map, n_items, v, ep, smem, G, st);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_cols_fwd<double>(const SphereDev<double>&, const double*, long long,
                                             ItemMap, int, int, cpx<double>*, cudaStream_t);
template cudaError_t launch_cols_fwd<float>(const SphereDev<float>&, const float*, long long,
                                            ItemMap, int, int, cpx<float>*, cudaStream_t);
template cudaError_t launch_cols_bwd<double>(const SphereDev<double>&, const cpx<double>*, ItemMap,
                                             int, const Epilogue<double>&, cudaStream_t);
template cudaError_t launch_cols_bwd<float>(const SphereDev<float>&, const cpx<float>*, ItemMap,
                                            int, const Epilogue<float>&, cudaStream_t);
template cudaError_t launch_slab<double>(const SphereDev<double>&, const SlabArgs<double>&,
                                         cudaStream_t);
template cudaError_t launch_slab<float>(const SphereDev<float>&, const SlabArgs<float>&,
                                        cudaStream_t);
template cudaError_t launch_cols_fwd<df>(const SphereDev<df>&, const double*, long long, ItemMap,
                                         int, int, cpx<df>*, cudaStream_t);
template cudaError_t launch_cols_bwd<df>(const SphereDev<df>&, const cpx<df>*, ItemMap, int,
                                         const Epilogue<df>&, cudaStream_t);
template cudaError_t launch_slab<df>(const SphereDev<df>&, const SlabArgs<df>&, cudaStream_t);

}  // namespace pdep
