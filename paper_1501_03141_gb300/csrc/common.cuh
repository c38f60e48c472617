// Common device/host definitions for the PDEP CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>

#include "../../include/pdep.h"

namespace pdep {

template <typename R>
struct cpx {
  R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) {
  cpx<R> c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename R>
__device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__device__ __forceinline__ cpx<R> scale(cpx<R> a, R s) { return mk(a.x * s, a.y * s); }
template <typename R>
__device__ __forceinline__ cpx<R> conj(cpx<R> a) { return mk(a.x, -a.y); }
// multiply by +i (S=+1) or -i (S=-1)
template <typename R, int S>
__device__ __forceinline__ cpx<R> mul_si(cpx<R> a) {
  return S > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}
template <typename R>
__device__ __forceinline__ cpx<R> shfl_xor(cpx<R> a, int m) {
  return mk(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
}
template <typename R>
__device__ __forceinline__ cpx<R> shfl_idx(cpx<R> a, int lane) {
  return mk(__shfl_sync(0xffffffffu, a.x, lane), __shfl_sync(0xffffffffu, a.y, lane));
}

// Device-side status word bits (OR-ed by kernels, read by the host after a sync).
enum : unsigned {
  DEV_NONFINITE = 1u,
  DEV_NOT_CONVERGED = 2u,
  DEV_BOUNDS = 4u,
  DEV_BREAKDOWN = 8u,
  DEV_TIMEOUT = 16u,
};

// Builds compiled with -DPDEP_BOUNDS_CHECK test every index that a kernel
// reads from the host-built sphere tables before using it: an index outside
// [0, n) sets DEV_BOUNDS in the status word and the access is skipped (the
// result is then wrong, and the call that reads the status returns
// PDEP_ERR_BOUNDS).  Normal builds compile the test to `true`.
__device__ __forceinline__ bool in_range(unsigned* status, long long i, long long n) {
#ifdef PDEP_BOUNDS_CHECK
  if (i >= 0 && i < n) return true;
  if (status) atomicOr(status, (unsigned)DEV_BOUNDS);
  return false;
#else
  return true;
#endif
}

}  // namespace pdep

#define PDEP_CUDA_CHECK(call)                                                  \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      pdep::set_last_error(__FILE__, __LINE__, cudaGetErrorString(e_));        \
      return PDEP_ERR_CUDA;                                                    \
    }                                                                          \
  } while (0)

namespace pdep {
void set_last_error(const char* file, int line, const char* msg);
}
