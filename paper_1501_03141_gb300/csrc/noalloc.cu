// H*x without any device allocation: pdep_apply_hamiltonian_noalloc.
//
// Some callers cannot allocate device memory at the moment they need H*x:
// code running while a CUDA graph is being captured on its stream, code
// inside a host callback or a custom allocator's hook, and embedders that
// hand every byte of device memory to their own pool at start-up.  For them
// this entry point runs the same pruned sphere <-> grid transforms as
// pdep_apply_hamiltonian, but its transform scratch lives in the fixed,
// file-scope device array below instead of the context's growable workspace,
// and it stages nothing: x and y must already be device buffers.
#include <atomic>
#include <cstring>

#include "common.cuh"
#include "transforms.cuh"

namespace pdep {

// 16 MiB of transform scratch, resident on every GPU that loads the library
// until the process exits.  One x-plane set of one packed vector pair needs
// N1 * n_col * 16 bytes (336 KiB on a 48^3 grid, 2.3 MiB on 64x64x192).
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
// concurrent first calls may both look the address up; they store the same
// value, and the atomics keep that free of data races
std::atomic<void*> g_scratch_addr[kMaxDevices] = {};

// Host code must not use g_noalloc_scratch directly: its host-side name is a
// stand-in, not a device address.  Look the address up once per device, with
// that device current: the context's device, which must be the current one
// (the scratch of another GPU would be given to this GPU's kernels).
int scratch_address(int ctx_device, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return PDEP_ERR_CUDA;
  }
  if (dev != ctx_device) {
    set_last_error(__FILE__, __LINE__,
                   "the current device is not the context's: make it current before the call");
    return PDEP_ERR_INVALID_ARG;
  }
  void* p = g_scratch_addr[dev].load();
  if (!p) {
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(__FILE__, __LINE__, cudaGetErrorString(e));
      return PDEP_ERR_CUDA;
    }
    g_scratch_addr[dev].store(p);
  }
  *out = p;
  return PDEP_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace

// Sphere description of one system and the context's device, filled from the
// context (no copies).
int noalloc_sphere(pdep_ctx* ctx, int sys, SphereDev<double>* sd, const double** v, int* n_pw,
                   int* device);

}  // namespace pdep

using namespace pdep;

extern "C" int pdep_apply_hamiltonian_noalloc(pdep_ctx* ctx, int sys, const double* x, int n,
                                              double* y, void* stream) {
  SphereDev<double> sd{};
  const double* v = nullptr;
  int n_pw = 0, device = 0;
  int r = noalloc_sphere(ctx, sys, &sd, &v, &n_pw, &device);
  if (r != PDEP_OK) return r;
  if (n < 0 || (n > 0 && (!x || !y))) {
    set_last_error(__FILE__, __LINE__, "bad arguments");
    return PDEP_ERR_INVALID_ARG;
  }
  if (n == 0) return PDEP_OK;
  if (!on_device(x) || !on_device(y)) {
    set_last_error(__FILE__, __LINE__, "x and y must be device buffers");
    return PDEP_ERR_INVALID_ARG;
  }
  const size_t per_item = (size_t)sd.N1 * sd.n_col * sizeof(cpx<double>);
  const long long max_items = (long long)(kNoallocScratchBytes / per_item);
  if (max_items < 1) {
    set_last_error(__FILE__, __LINE__,
                   "grid too large for the 16 MiB no-allocation scratch (needs N1*n_col*16 bytes)");
    return PDEP_ERR_UNSUPPORTED;
  }
  void* scratch = nullptr;
  r = scratch_address(device, &scratch);
  if (r != PDEP_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cpx<double>* b1 = reinterpret_cast<cpx<double>*>(scratch);
  // vectors in chunks of whole packed pairs; every chunk overwrites the scratch
  const long long chunk_vecs = 2 * max_items;
  for (long long v0 = 0; v0 < n; v0 += chunk_vecs) {
    const int m = (int)std::min<long long>(chunk_vecs, n - v0);
    const int n_items = (m + 1) / 2;
    ItemMap map{m, n_items};
    const double* xs = x + v0 * n_pw;
    double* ys = y + v0 * n_pw;
    cudaError_t e = launch_cols_fwd<double>(sd, xs, n_pw, map, n_items, COEF_ONE, b1, st);
    if (e == cudaSuccess) {
      SlabArgs<double> a{};
      a.mode = SLAB_HPSI;
      a.b1 = b1;
      a.n_items = n_items;
      a.v = v;
      a.map = map;
      e = launch_slab<double>(sd, a, st);
    }
    if (e == cudaSuccess) {
      Epilogue<double> ep{};
      ep.y = ys;
      ep.ldy = n_pw;
      ep.x_in = xs;
      ep.ldx = n_pw;
      ep.shift_period = 1;
      ep.scale = 1.0 / ((double)sd.N1 * sd.N2 * sd.N3);
      ep.kin = 1.0;
      ep.coef = COEF_ONE;
      e = launch_cols_bwd<double>(sd, b1, map, n_items, ep, st);
    }
    if (e != cudaSuccess) {
      set_last_error(__FILE__, __LINE__, cudaGetErrorString(e));
      return PDEP_ERR_CUDA;
    }
  }
  return PDEP_OK;
}
