// C ABI and host orchestration of the PDEP hot path (Sec. II C of Govoni &
// Galli): setup eigensolve, batched Sternheimer CG, density response,
// chi0bar application and the Davidson iteration.  Everything here only
// enqueues kernels on the caller's stream and reads small convergence flags
// back between steps.
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "linalg.cuh"
#include "profile.cuh"
#include "transforms.cuh"

namespace pdep {

static thread_local std::string g_last_error;

// NVTX range for the span of a scope (no cost unless a profiler is attached):
// pdep_solve, davidson_iteration, chi0bar_apply, refinement_round, setup, ...
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_last_error(const char* file, int line, const char* msg) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s:%d: %s", file, line, msg);
  g_last_error = buf;
}

static int fail(int status, const char* msg) {
  g_last_error = msg;
  return status;
}

#define CK(call)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      pdep::set_last_error(__FILE__, __LINE__, cudaGetErrorString(e_));          \
      return e_ == cudaErrorMemoryAllocation ? PDEP_ERR_OOM : PDEP_ERR_CUDA;     \
    }                                                                            \
  } while (0)

#define RET(call)                  \
  do {                             \
    int r_ = (call);               \
    if (r_ != PDEP_OK) return r_;  \
  } while (0)

// ---------------------------------------------------------------------------
// per-system data
// ---------------------------------------------------------------------------
struct SysData {
  int N[3] = {0, 0, 0};
  double L[3] = {0, 0, 0};
  double omega = 0, ecut = 0;
  int n_r = 0, n_half = 0, n_pw = 0, ld = 0, n_occ = 0, n_pdep = 0;
  int n_defl = 0;            // lowest empty states deflated from the CG operator
  int n_ext = 0;             // n_occ + n_defl: columns of d_psi
  double* d_eps_ext = nullptr;  // eps of the n_ext states
  double* d_sigma64 = nullptr;   // per-state shift eps_{n_ext} - eps_w, w < n_ext
  float* d_sigma32 = nullptr;
  int n_col = 0, n_ucol = 0, R3 = 0;
  std::vector<UCol> ucol;
  std::vector<int2> slot;
  std::vector<double> g2;
  UCol* d_ucol = nullptr;
  int2* d_slot = nullptr;
  double* d_g2 = nullptr;
  cpx<double>* d_tw64[3] = {nullptr, nullptr, nullptr};
  cpx<float>* d_tw32[3] = {nullptr, nullptr, nullptr};
  cpx<df>* d_twdf[3] = {nullptr, nullptr, nullptr};
  double* d_v = nullptr;
  float* d_vf = nullptr;
  df* d_vdf = nullptr;       // V(r) in double-float (refinement transforms)
  df* d_kindf = nullptr;
  double* d_psi = nullptr;   // [n_occ][ld]
  float* d_psif = nullptr;
  float* d_psit5 = nullptr;  // d_psif as TF32 hi / lo tiles of the tcgen05 coefficients
  unsigned short* d_psib16 = nullptr;  // d_psif as BF16 tiles (PDEP_MIXED_BF16)
  double* d_u = nullptr;     // [n_occ][n_r]  u_v(r) = Omega^{1/2} psi_v(r)
  double* d_negeps = nullptr;   // -eps_v
  float* d_negeps32 = nullptr;
  double* d_kin64 = nullptr;    // |G_k|^2 / 2
  float* d_kin32 = nullptr;
  double* d_ekin = nullptr;
  double* d_kprec64 = nullptr;  // CG preconditioner per occupied state [n_occ][ld]
  float* d_kprec32 = nullptr;
  std::vector<double> eps;   // n_occ + 1
  double vmax = 0;           // max_r V(r)
  SphereDev<double> sd{};
  SphereDev<float> sf{};
  SphereDev<df> sdf{};
};

}  // namespace pdep

using namespace pdep;

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// One autotuned choice: every candidate computes the same result, so each is
// timed on real calls (two calls each, alternating), its time per unit of
// work kept, and the fastest is used from then on.
struct Tune {
  int next = 0, calls = 0, best = -1;
  double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// One captured Sternheimer CG loop (prologue + while node over the steps),
// valid for the buffers and settings it was captured with.
struct CgGraph {
  int prec, sys, n, max_iter, cg_variant, proj_variant, tune_gen;
  double tol;
  const void *b, *x, *sc, *mask, *tolv;
  unsigned long long ws_gen, budget_ns;
  cudaGraphExec_t exec;
};

struct pdep_ctx {
  int device = 0;
  pdep_options opt{};
  std::vector<SysData> sys;
  std::map<std::string, DevBuf> bufs;
  size_t ws_bytes = 0;
  std::vector<void*> owned;
  unsigned* d_status = nullptr;
  int* d_counter = nullptr;
  // device-side loop state and statistics of the Sternheimer solves
  CgLoopState* d_loop = nullptr;
  DevStats* d_dstats = nullptr;
  int* d_refine = nullptr;        // [0]: unconverged count of the current refinement round
  cudaStream_t cap_stream = nullptr;  // private stream the CG graphs are captured on
  unsigned long long ws_gen = 0;  // bumped whenever a workspace buffer is reallocated
  unsigned long long budget_ns = 0;   // clock_budget_cycles in ns of %globaltimer
  std::vector<CgGraph> cg_graphs;     // executable CG-loop graphs, released in pdep_destroy
  int body_launches[2] = {0, 0};      // kernels per CG step in the graphs (FP32, FP64)
  long long graph_launches = 0;       // CG graphs launched
  long long eager_steps[2] = {0, 0};  // CG steps launched from the host loop (FP32, FP64)
  long long st_launch0 = 0;           // launch counter at the last statistics reset
  pdep_stats last_dav{};              // statistics of the last pdep_solve
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int* h_pin = nullptr;  // pinned host scratch (ints)
  // statistics of the current call
  long long st_solves = 0, st_cg_iters = 0;
  int st_cg_max = 0, st_refine_max = 0;
  int st_chunks = 0;  // perturbation chunks of the last chi0bar application
  double st_max_res = 0;
  // autotuned launch shape of the CG step, per precision (-1: not tuned yet)
  int cg_variant[2] = {-1, -1};
  // autotuned FP32 projection kernel (0 CUDA-core, 1 tensor-core; -1 untuned)
  int proj_variant = -1;
  bool cg_inner = false;  // inside an FP32 inner CG loop (BF16 coefficients in PDEP_MIXED_BF16)
  int proj_tune_next = 0;
  double proj_tune_ms[3] = {0, 0, 0};
  int proj_tune_calls = 0;
  double cg_tune_ms[2][CG_NUM_VARIANTS] = {};
  int cg_tune_next[2] = {0, 0};
  // executable graphs of the Jacobi sweeps, released in pdep_destroy
  EighGraphCache eig_graphs;
  // autotuner over the FFT batch (planes per group of the fused transform)
  // and the GEMM tile shapes, keyed by kernel and problem shape
  std::map<std::string, Tune> tunes;
  int tune_gen = 0;  // bumped whenever a choice is made (graphs keyed by it)
};

namespace {

template <typename T>
int persistent(pdep_ctx* c, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PDEP_ERR_OOM, "cudaMalloc failed for a persistent buffer");
  }
  c->owned.push_back(*p);
  return PDEP_OK;
}

// named, grow-only workspace buffer
template <typename T>
int ws(pdep_ctx* c, const char* name, size_t count, T** out) {
  if (count == 0) count = 1;
  size_t bytes = sizeof(T) * count;
  DevBuf& b = c->bufs[name];
  if (b.cap < bytes) {
    size_t newcap = bytes;
    if (c->opt.workspace_limit_bytes && c->ws_bytes - b.cap + newcap > c->opt.workspace_limit_bytes)
      return fail(PDEP_ERR_OOM, "workspace limit exceeded");
    if (b.p) {
      cudaFree(b.p);
      c->ws_bytes -= b.cap;
      b.p = nullptr;
      b.cap = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, newcap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PDEP_ERR_OOM, "cudaMalloc failed for the workspace");
    }
    b.cap = newcap;
    c->ws_bytes += newcap;
    ++c->ws_gen;  // graphs captured with the old buffer are stale now
  }
  *out = (T*)b.p;
  return PDEP_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaMemcpyKind kind_to_dev(const void* src) {
  return is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_dev(const void* dst) {
  return is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// host source -> host or device destination
int copy_from_host(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (is_device_ptr(dst)) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else {
    memcpy(dst, src, bytes);
  }
  return PDEP_OK;
}

int sync(cudaStream_t st) {
  CK(cudaStreamSynchronize(st));
  return PDEP_OK;
}

// Synchronises st, reads the device status word and clears it: the
// conditions of every call enqueued since the last read.
int check_status(pdep_ctx* c, cudaStream_t st) {
  unsigned h = 0;
  CK(cudaMemcpyAsync(c->h_pin, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), st));
  CK(cudaStreamSynchronize(st));
  memcpy(&h, c->h_pin, sizeof(unsigned));
  if (h & DEV_NONFINITE) return fail(PDEP_ERR_NONFINITE, "non-finite value met on the device");
  if (h & DEV_BREAKDOWN) return fail(PDEP_ERR_NONFINITE, "CG breakdown (p.Ap <= 0)");
  if (h & DEV_BOUNDS) return fail(PDEP_ERR_BOUNDS, "sphere-table index out of range");
  if (h & DEV_TIMEOUT) return fail(PDEP_ERR_TIMEOUT, "a CG loop spent its clock budget");
  if (h & DEV_NOT_CONVERGED)
    return fail(PDEP_ERR_NOT_CONVERGED, "a Sternheimer solve ended above cg_tol");
  return PDEP_OK;
}

// ---------------------------------------------------------------------------
// sphere tables (Eq. planewaveexpansionofwfc at Gamma, half-space layout)
// ---------------------------------------------------------------------------
int build_sphere(SysData& s, double ecut_in) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int a = 0; a < 3; ++a)
    if (s.N[a] <= 0 || !(s.L[a] > 0)) return fail(PDEP_ERR_INVALID_ARG, "bad grid or cell");
  double ecut = ecut_in;
  if (!(ecut > 0)) {
    double gmax = 1e300;
    for (int a = 0; a < 3; ++a) gmax = std::min(gmax, two_pi * ((s.N[a] - 1) / 4.0) / s.L[a]);
    ecut = 0.5 * gmax * gmax;
  }
  s.ecut = ecut;
  s.omega = s.L[0] * s.L[1] * s.L[2];
  s.n_r = s.N[0] * s.N[1] * s.N[2];
  int lim[3];
  for (int a = 0; a < 3; ++a) lim[a] = (s.N[a] - 1) / 2;
  auto inside = [&](int n1, int n2, int n3) {
    double gx = two_pi * n1 / s.L[0], gy = two_pi * n2 / s.L[1], gz = two_pi * n3 / s.L[2];
    return 0.5 * (gx * gx + gy * gy + gz * gz) <= ecut;
  };
  // x-extent of every (n2, n3) column
  auto r1 = [&](int n2, int n3) {
    if (!inside(0, n2, n3)) return -1;
    int r = 0;
    while (r + 1 <= lim[0] && inside(r + 1, n2, n3)) ++r;
    return r;
  };
  // aliasing guard: every product of two sphere functions must fit the grid
  for (int n3 = -lim[2]; n3 <= lim[2]; ++n3)
    for (int n2 = -lim[1]; n2 <= lim[1]; ++n2) {
      int r = r1(n2, n3);
      if (r < 0) continue;
      if (2 * std::abs(n2) >= s.N[1] / 2 || 2 * std::abs(n3) >= s.N[2] / 2 || 2 * r >= s.N[0] / 2)
        return fail(PDEP_ERR_INVALID_ARG, "ecut too large for the grid (products would alias)");
    }
  int R3 = -1;
  for (int n3 = 0; n3 <= lim[2]; ++n3)
    if (r1(0, n3) >= 0) R3 = n3;
  if (R3 < 0) return fail(PDEP_ERR_INVALID_ARG, "empty sphere");
  s.R3 = R3;
  // full column list in (n3, n2) order
  std::map<std::pair<int, int>, int> colidx;
  s.slot.assign(2 * R3 + 1, make_int2(0, 0));
  int ncol = 0;
  for (int n3 = -R3; n3 <= R3; ++n3) {
    int R2 = -1;
    for (int n2 = 0; n2 <= lim[1]; ++n2)
      if (r1(n2, n3) >= 0) R2 = n2;
    if (R2 < 0) return fail(PDEP_ERR_INVALID_ARG, "sphere not convex in n2");
    s.slot[n3 + R3] = make_int2(R2, ncol);
    for (int n2 = -R2; n2 <= R2; ++n2) {
      if (r1(n2, n3) < 0) return fail(PDEP_ERR_INVALID_ARG, "sphere not convex");
      colidx[{n2, n3}] = ncol++;
    }
  }
  s.n_col = ncol;
  // half space (n3 > 0 | n3 = 0, n2 > 0 | n3 = n2 = 0, n1 > 0) in (n3, n2, n1) order
  s.g2.clear();
  s.ucol.clear();
  int nh = 0;
  for (int n3 = 0; n3 <= R3; ++n3) {
    const int R2 = s.slot[n3 + R3].x;
    for (int n2 = (n3 == 0 ? 0 : -R2); n2 <= R2; ++n2) {
      const int R1 = r1(n2, n3);
      UCol u;
      u.n2 = n2;
      u.n3 = n3;
      u.R1 = R1;
      u.h0 = nh;
      u.col = colidx[{n2, n3}];
      u.mcol = colidx[{-n2, -n3}];
      const int lo = (n3 == 0 && n2 == 0) ? 1 : -R1;
      for (int n1 = lo; n1 <= R1; ++n1) {
        double gx = two_pi * n1 / s.L[0], gy = two_pi * n2 / s.L[1], gz = two_pi * n3 / s.L[2];
        s.g2.push_back(gx * gx + gy * gy + gz * gz);
        ++nh;
      }
      s.ucol.push_back(u);
    }
  }
  s.n_half = nh;
  s.n_pw = 2 * nh + 1;
  s.ld = ((s.n_pw + 31) / 32) * 32;
  s.n_ucol = (int)s.ucol.size();
  return PDEP_OK;
}

int upload_tables(pdep_ctx* c, SysData& s) {
  RET(persistent(c, &s.d_ucol, s.ucol.size()));
  RET(persistent(c, &s.d_slot, s.slot.size()));
  RET(persistent(c, &s.d_g2, s.g2.size()));
  CK(cudaMemcpy(s.d_ucol, s.ucol.data(), sizeof(UCol) * s.ucol.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s.d_slot, s.slot.data(), sizeof(int2) * s.slot.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s.d_g2, s.g2.data(), sizeof(double) * s.g2.size(), cudaMemcpyHostToDevice));
  {
    std::vector<double> k64(s.g2.size());
    std::vector<float> k32(s.g2.size());
    for (size_t k = 0; k < s.g2.size(); ++k) {
      k64[k] = 0.5 * s.g2[k];
      k32[k] = (float)k64[k];
    }
    std::vector<df> kdf(k64.begin(), k64.end());
    RET(persistent(c, &s.d_kin64, k64.size()));
    RET(persistent(c, &s.d_kin32, k32.size()));
    RET(persistent(c, &s.d_kindf, kdf.size()));
    CK(cudaMemcpy(s.d_kin64, k64.data(), sizeof(double) * k64.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s.d_kin32, k32.data(), sizeof(float) * k32.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s.d_kindf, kdf.data(), sizeof(df) * kdf.size(), cudaMemcpyHostToDevice));
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int a = 0; a < 3; ++a) {
    const int N = s.N[a];
    std::vector<cpx<double>> td(N);
    std::vector<cpx<float>> tf(N);
    std::vector<cpx<df>> tdf(N);
    for (int j = 0; j < N; ++j) {
      double ang = two_pi * j / N;
      td[j] = mk(cos(ang), sin(ang));
      tf[j] = mk((float)cos(ang), (float)sin(ang));
      tdf[j] = mk(df(cos(ang)), df(sin(ang)));
    }
    RET(persistent(c, &s.d_tw64[a], N));
    RET(persistent(c, &s.d_tw32[a], N));
    RET(persistent(c, &s.d_twdf[a], N));
    CK(cudaMemcpy(s.d_tw64[a], td.data(), sizeof(cpx<double>) * N, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s.d_tw32[a], tf.data(), sizeof(cpx<float>) * N, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s.d_twdf[a], tdf.data(), sizeof(cpx<df>) * N, cudaMemcpyHostToDevice));
  }
  auto fill = [&](auto& d, auto tw) {
    d.N1 = s.N[0];
    d.N2 = s.N[1];
    d.N3 = s.N[2];
    d.R3 = s.R3;
    d.n_half = s.n_half;
    d.n_pw = s.n_pw;
    d.n_col = s.n_col;
    d.n_ucol = s.n_ucol;
    d.ucol = s.d_ucol;
    d.slot = s.d_slot;
    d.g2 = s.d_g2;
    d.tw1 = tw[0];
    d.tw2 = tw[1];
    d.tw3 = tw[2];
#ifdef PDEP_BOUNDS_CHECK
    d.status = c->d_status;
#endif
  };
  fill(s.sd, s.d_tw64);
  fill(s.sf, s.d_tw32);
  fill(s.sdf, s.d_twdf);
  s.sd.kin = s.d_kin64;
  s.sf.kin = s.d_kin32;
  s.sdf.kin = s.d_kindf;
  return PDEP_OK;
}

// precision selectors
inline const SphereDev<double>& sph(const SysData& s, double*) { return s.sd; }
inline const SphereDev<float>& sph(const SysData& s, float*) { return s.sf; }
inline const SphereDev<df>& sph(const SysData& s, df*) { return s.sdf; }
inline const double* vgrid(const SysData& s, double*) { return s.d_v; }
inline const float* vgrid(const SysData& s, float*) { return s.d_vf; }
inline const df* vgrid(const SysData& s, df*) { return s.d_vdf; }
inline const double* psi_of(const SysData& s, double*) { return s.d_psi; }
inline const float* psi_of(const SysData& s, float*) { return s.d_psif; }
inline const double* kprec_of(const SysData& s, double*) { return s.d_kprec64; }
inline const double* negeps_of(const SysData& s, double*) { return s.d_negeps; }
inline const double* sigma_of(const SysData& s, double*) { return s.d_sigma64; }
inline const float* sigma_of(const SysData& s, float*) { return s.d_sigma32; }
inline const float* negeps_of(const SysData& s, float*) { return s.d_negeps32; }
inline const float* kprec_of(const SysData& s, float*) { return s.d_kprec32; }

size_t b1_count(const SysData& s, int n_items) {
  return (size_t)n_items * s.N[0] * s.n_col;
}

// Y = (H - eps_v) X for the vectors of 'map' (H = -nabla^2/2 + V); vector i
// uses occupied state i % n_occ; without with_shift Y = H X.  Then, if
// with_pv, the occupied and deflated states are shifted:
// Y += Psi_ext diag(sigma) (Psi_ext^T X) on the same columns.
// dn (FP64 only, may be null): the transform also accumulates the density
// response dn_j(r) += (4/Omega) u_v(r) x_i(r) of every vector i = j n_occ + v
// it transforms (Eq. deltani); dn must hold the (i / n_occ) perturbations.
bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Runs fn(candidate): the tuned choice once made, the default while
// autotuning is off or the call is too small (units < 256) or captured, else
// the next candidate, timed with events on st (this synchronises: only the
// first 2 x n_cand large calls of a shape do).
template <typename F>
int tuned_call(pdep_ctx* c, const std::string& key, int n_cand, int def, double units,
               cudaStream_t st, F fn) {
  auto it = c->tunes.find(key);
  if (it != c->tunes.end() && it->second.best >= 0) return fn(it->second.best);
  if (!c->opt.autotune || units < 256 || n_cand < 2 || capturing(st)) return fn(def);
  Tune& t = c->tunes[key];
  const int cand = t.next;
  CK(cudaEventRecord(c->ev[0], st));
  RET(fn(cand));
  CK(cudaEventRecord(c->ev[1], st));
  CK(cudaEventSynchronize(c->ev[1]));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  t.ms[cand] += ms / units;
  t.next = (t.next + 1) % n_cand;
  if (++t.calls == 2 * n_cand) {
    int best = 0;
    for (int k = 1; k < n_cand; ++k)
      if (t.ms[k] < t.ms[best]) best = k;
    t.best = best;
    ++c->tune_gen;
  }
  return PDEP_OK;
}
bool tune_done(const pdep_ctx* c, const std::string& key) {
  auto it = c->tunes.find(key);
  return it != c->tunes.end() && it->second.best >= 0;
}

// GEMM tile candidates of the projection GEMMs: tile height 64 or 80 rows,
// split-K at the default, half or twice the default
const GemmShape kGemmShapes[4] = {{4, 8}, {5, 8}, {5, 4}, {5, 16}};
std::string shape_key(const char* what, const SysData& s) {
  return std::string(what) + ":" + std::to_string(s.n_ext) + ":" + std::to_string(s.n_pw);
}

// d_count (with d_list): device length of the list; n_list is then the
// largest length, which sizes the launches (kernels read the count).
// C is the arithmetic type of the transforms (float, double, or df: double-
// float on FP32 vectors... on FP64 vectors); the vectors and the projection
// term use its storage type R (FP64 for df).
template <typename C, typename R = typename Io<C>::T>
int apply_h(pdep_ctx* c, SysData& s, const R* X, R* Y, int n, const int* d_list, int n_list,
            bool with_shift, bool with_pv, cudaStream_t st, double* dn = nullptr,
            const int* d_count = nullptr) {
  ItemMap map{n, (n + 1) / 2};
  int n_items = (n + 1) / 2;
  if (d_list) {
    map.list = d_list;
    map.n_list = n_list;
    map.n_dev = d_count;
    n_items = (n_list + 1) / 2;
  }
  bool fused = false;
  if constexpr (std::is_same<C, float>::value) {
    // FP32 on 24^3 .. 48^3: the whole transform in one launch, the column
    // scratch in shared memory
    if (n_items > 0 && !dn && c->opt.fused_hpsi && hpsi_fused_smem(s.sf) > 0) {
      Epilogue<float> ep{};
      ep.y = Y;
      ep.ldy = s.ld;
      ep.x_in = X;
      ep.ldx = s.ld;
      ep.shift = with_shift ? s.d_negeps32 : nullptr;
      ep.shift_period = with_shift ? s.n_occ : 1;
      ep.scale = 1.0f / s.n_r;
      ep.kin = 1.0f;
      ep.beta = 0.0f;
      ep.coef = COEF_ONE;
      // FFT batch: x-planes per group of the fused transform (half, the
      // default, or twice the default when shared memory allows)
      const int G0 = hpsi_fused_planes(s.sf);
      const int cands[3] = {G0, G0 / 2 > 0 ? G0 / 2 : G0,
                            hpsi_fused_smem(s.sf, 2 * G0) ? 2 * G0 : G0};
      RET(tuned_call(c, "fused_planes:" + std::to_string(s.N[0]), 3, 0, 2.0 * n_items, st,
                     [&](int k) -> int {
                       CK(launch_hpsi_fused(s.sf, X, s.ld, map, n_items, s.d_vf, ep, st, cands[k]));
                       return PDEP_OK;
                     }));
      fused = true;
    }
  }
  if (n_items > 0 && !fused) {
    cpx<C>* b1;   // double-float shares the FP64 scratch (16 bytes per complex)
    RET(ws(c, sizeof(C) == 8 ? "b1_64" : "b1_32", b1_count(s, n_items), &b1));
    const SphereDev<C>& sd = sph(s, (C*)nullptr);
    CK(launch_cols_fwd<C>(sd, X, s.ld, map, n_items, COEF_ONE, b1, st));
    SlabArgs<C> a{};
    a.mode = SLAB_HPSI;
    a.b1 = b1;
    a.n_items = n_items;
    a.v = vgrid(s, (C*)nullptr);
    a.map = map;
    if (dn) {
      a.dn = dn;
      a.u = s.d_u;
      a.dn_nocc = s.n_occ;
      a.dn_stride = s.n_r;
      a.dn_scale = 4.0 / s.omega;
    }
    CK(launch_slab<C>(sd, a, st));
    Epilogue<C> ep{};
    ep.y = Y;
    ep.ldy = s.ld;
    ep.x_in = X;
    ep.ldx = s.ld;
    ep.shift = with_shift ? negeps_of(s, (R*)nullptr) : nullptr;
    ep.shift_period = with_shift ? s.n_occ : 1;
    ep.scale = C(1.0 / s.n_r);
    ep.kin = C(1);
    ep.beta = R(0);
    ep.coef = COEF_ONE;
    CK(launch_cols_bwd<C>(sd, b1, map, n_items, ep, st));
  }
  if (with_pv) {
    // only the listed columns when a list is given
    const int m = d_list ? n_list : n;
    if constexpr (sizeof(R) == 4) {
      // FP32: CUDA-core GEMMs (variant 0), 3xTF32 on mma.sync (variant 1),
      // or the coefficients 3xTF32 on tcgen05 with tensor-memory
      // accumulators and the update on mma.sync (variant 2).  While untuned,
      // calls with many columns take the variants in turn and keep their
      // time per column; afterwards the fastest one is used.
      if (c->cg_inner && s.d_psib16) {
        // PDEP_MIXED_BF16, inside the inner CG: the coefficients as one BF16
        // product per k-step (tcgen05 kind::f16), the update in 3xTF32; the
        // refinement rounds' products never come here
        const long long lds = (s.n_ext + 3) & ~3;
        float* S;
        RET(ws(c, "pv_32", (size_t)lds * std::max(m, 1), &S));
        CK(tc5_proj_coeffs(s.n_ext, m, s.n_pw, s.d_psib16, X, s.ld, d_list, s.d_sigma32, S, lds,
                           st, d_count, c->d_status, true));
        CK(tc_proj_update(s.n_pw, m, s.n_ext, s.d_psif, s.ld, S, lds, Y, s.ld, d_list, st,
                          d_count));
        return PDEP_OK;
      }
      int pv = c->opt.proj_variant >= 0 ? c->opt.proj_variant : c->proj_variant;
      const bool tuning = c->opt.autotune && pv < 0 && m >= 256;
      if (pv < 0) pv = tuning ? c->proj_tune_next : 2;
      if (tuning) CK(cudaEventRecord(c->ev[0], st));
      if (pv == 1 || pv == 2) {
        const long long lds = (s.n_ext + 3) & ~3;
        float* S;
        RET(ws(c, "pv_32", (size_t)lds * std::max(m, 1), &S));
        if (pv == 1)
          CK(tc_proj_coeffs(s.n_ext, m, s.n_pw, s.d_psif, s.ld, X, s.ld, d_list, s.d_sigma32, S,
                            lds, st, d_count));
        else
          CK(tc5_proj_coeffs(s.n_ext, m, s.n_pw, s.d_psit5, X, s.ld, d_list, s.d_sigma32, S, lds,
                             st, d_count, c->d_status));
        CK(tc_proj_update(s.n_pw, m, s.n_ext, s.d_psif, s.ld, S, lds, Y, s.ld, d_list, st,
                          d_count));
      } else {
        float* S;
        RET(ws(c, "pv_32", (size_t)s.n_ext * std::max(m, 1), &S));
        CK(gemm<float>(true, s.n_ext, m, s.n_pw, 1.0, s.d_psif, s.ld, X, s.ld, 0.0, S, s.n_ext,
                       st, d_list, nullptr, d_count));
        CK(scale_rows<float>(S, s.n_ext, s.n_ext, m, s.d_sigma32, st));
        CK(gemm<float>(false, s.n_pw, m, s.n_ext, 1.0, s.d_psif, s.ld, S, s.n_ext, 1.0, Y, s.ld,
                       st, nullptr, d_list, d_count));
      }
      if (tuning) {
        CK(cudaEventRecord(c->ev[1], st));
        CK(cudaEventSynchronize(c->ev[1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->proj_tune_ms[pv] += ms / m;
        // two timed calls per variant, in turn
        if (++c->proj_tune_next == 3) c->proj_tune_next = 0;
        if (++c->proj_tune_calls == 6) {
          int best = 0;
          for (int v = 1; v < 3; ++v)
            if (c->proj_tune_ms[v] <= c->proj_tune_ms[best]) best = v;
          c->proj_variant = best;
        }
      }
      return PDEP_OK;
    }
    R* S;
    // shift of the occupied and the deflated empty states: state w moves to
    // eps_{n_ext} - eps_v, the bottom of the spectrum the CG still sees
    // (double-float transforms take double-float GEMMs too: FP64 matrices,
    // arithmetic on the FP32 pipe)
    using G = typename std::conditional<std::is_same<C, df>::value, df, R>::type;
    RET(ws(c, sizeof(R) == 8 ? "pv_64" : "pv_32", (size_t)s.n_ext * std::max(m, 1), &S));
    const R* P = psi_of(s, (R*)nullptr);
    // tile shapes of the pair, autotuned per problem shape
    RET(tuned_call(c, shape_key(std::is_same<G, df>::value ? "pv_df" : "pv_64", s), 4, 1, m, st,
                   [&](int k) -> int {
                     const GemmShape sh = kGemmShapes[k];
                     CK(gemm<G>(true, s.n_ext, m, s.n_pw, 1.0, P, s.ld, X, s.ld, 0.0, S,
                                s.n_ext, st, d_list, nullptr, d_count, sh));
                     CK(scale_rows<R>(S, s.n_ext, s.n_ext, m, sigma_of(s, (R*)nullptr), st));
                     CK(gemm<G>(false, s.n_pw, m, s.n_ext, 1.0, P, s.ld, S, s.n_ext, 1.0, Y, s.ld,
                                st, nullptr, d_list, d_count, sh));
                     return PDEP_OK;
                   }));
  }
  return PDEP_OK;
}

// RHS split for deflation: S = Psi_ext^T B; the deflated states' part of the
// solution is Xd = sum_c psi_c S_c,i / (eps_c - eps_v(i)) (exact, H psi_c =
// eps_c psi_c); then B <- B - Psi_ext S leaves the part the CG solves.
// (G: FP64, or double-float arithmetic on the FP64 matrices in the mixed modes)
template <typename G>
int split_rhs_t(pdep_ctx* c, SysData& s, double* B, int n, double* Xd, cudaStream_t st) {
  double* S;
  RET(ws(c, "pc_64", (size_t)s.n_ext * n, &S));
  RET(tuned_call(c, shape_key(std::is_same<G, df>::value ? "split_df" : "split_64", s), 4, 1, n, st,
                 [&](int k) -> int {
                   const GemmShape sh = kGemmShapes[k];
                   CK(gemm<G>(true, s.n_ext, n, s.n_pw, 1.0, s.d_psi, s.ld, B, s.ld, 0.0, S,
                              s.n_ext, st, nullptr, nullptr, nullptr, sh));
                   CK(gemm<G>(false, s.n_pw, n, s.n_ext, -1.0, s.d_psi, s.ld, S, s.n_ext, 1.0, B,
                              s.ld, st, nullptr, nullptr, nullptr, sh));
                   return PDEP_OK;
                 }));
  if (s.n_defl > 0) {
    CK(deflation_coefficients(S, s.n_ext, s.n_occ, s.n_defl, n, s.d_eps_ext, st));
    CK(gemm<G>(false, s.n_pw, n, s.n_defl, 1.0, s.d_psi + (size_t)s.n_occ * s.ld, s.ld,
               S + s.n_occ, s.n_ext, 0.0, Xd, s.ld, st));
  }
  return PDEP_OK;
}
int split_rhs(pdep_ctx* c, SysData& s, double* B, int n, double* Xd, cudaStream_t st) {
  if (c->opt.precision != PDEP_FP64 && c->opt.df_refine)
    return split_rhs_t<df>(c, s, B, n, Xd, st);
  return split_rhs_t<double>(c, s, B, n, Xd, st);
}

// ---------------------------------------------------------------------------
// small dense helpers on the device
// ---------------------------------------------------------------------------
int eigh_ws(pdep_ctx* c, int n, EighWork* wk) {
  RET(ws(c, "eig_a", (size_t)n * n, &wk->a));
  RET(ws(c, "eig_v", (size_t)n * n, &wk->v));
  RET(ws(c, "eig_t", (size_t)n * n + n, &wk->tmp));
  RET(ws(c, "eig_w", (size_t)n, &wk->w));
  RET(ws(c, "eig_f", (size_t)4, &wk->flag));
  wk->graphs = &c->eig_graphs;
  return PDEP_OK;
}

// Orthonormalise the m columns of T (rows = n_pw, ld) against the nb columns of
// B and among themselves (two passes of block Gram-Schmidt + symmetric
// normalisation through the Gram matrix's eigendecomposition).  Columns that
// are numerically dependent are dropped; the kept ones are written to OUT.
// Returns the kept count in *kept.
int orthonormalize(pdep_ctx* c, SysData& s, const double* B, int nb, double* T, int m, double* OUT,
                   int* kept, cudaStream_t st) {
  *kept = 0;
  if (m <= 0) return PDEP_OK;
  const int rows = s.n_pw;
  double *S, *G, *Q, *d;
  RET(ws(c, "on_s", (size_t)std::max(nb, 1) * m, &S));
  RET(ws(c, "on_g", (size_t)m * m, &G));
  RET(ws(c, "on_q", (size_t)m * m, &Q));
  RET(ws(c, "on_d", (size_t)m, &d));
  EighWork wk;
  RET(eigh_ws(c, m, &wk));
  int cur = m;
  double* src = T;
  for (int pass = 0; pass < 2; ++pass) {
    for (int rep = 0; rep < 2 && nb > 0; ++rep) {
      CK(gemm<double>(true, nb, cur, rows, 1.0, B, s.ld, src, s.ld, 0.0, S, nb, st));
      CK(gemm<double>(false, rows, cur, nb, -1.0, B, s.ld, S, nb, 1.0, src, s.ld, st));
    }
    CK(gemm<double>(true, cur, cur, rows, 1.0, src, s.ld, src, s.ld, 0.0, G, cur, st));
    if (cur <= 128) {
      // Cholesky QR: OUT = src L^{-T}; ill-conditioned blocks fall through to
      // the symmetric orthonormalisation below, which drops dependent columns
      int* fail;
      RET(ws(c, "on_f", 1, &fail));
      CK(cholesky_winv(G, cur, 1e-10, Q, fail, st));
      int hf = 1;
      CK(cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (hf == 0) {
        CK(gemm<double>(false, rows, cur, cur, 1.0, src, s.ld, Q, cur, 0.0, OUT, s.ld, st));
        if (pass == 0) {
          CK(cudaMemcpy2DAsync(T, s.ld * sizeof(double), OUT, s.ld * sizeof(double),
                               rows * sizeof(double), cur, cudaMemcpyDeviceToDevice, st));
          src = T;
        }
        continue;
      }
    }
    CK(eigh(cur, G, cur, d, Q, cur, wk, st));
    std::vector<double> hd(cur);
    CK(cudaMemcpyAsync(hd.data(), d, sizeof(double) * cur, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double dmax = hd[cur - 1];
    if (!(dmax > 0) || !std::isfinite(dmax)) return PDEP_OK;
    const double thr = 1e-12 * dmax;
    int first = 0;
    while (first < cur && !(hd[first] > thr)) ++first;
    const int keep = cur - first;
    CK(scale_by_isqrt_clamped(Q, cur, cur, d, thr, nullptr, st));
    // OUT[:, 0:keep] = src * Q[:, first:cur]
    CK(gemm<double>(false, rows, keep, cur, 1.0, src, s.ld, Q + (size_t)first * cur, cur, 0.0,
                    OUT, s.ld, st));
    cur = keep;
    if (pass == 0 && cur > 0) {
      // second pass works on OUT in place through T
      CK(cudaMemcpy2DAsync(T, s.ld * sizeof(double), OUT, s.ld * sizeof(double),
                           rows * sizeof(double), cur, cudaMemcpyDeviceToDevice, st));
      src = T;
    }
    if (cur == 0) break;
  }
  *kept = cur;
  return PDEP_OK;
}

// ---------------------------------------------------------------------------
// generic block Davidson for the lowest eigenpairs of a symmetric operator
// ---------------------------------------------------------------------------
struct DavidsonOut {
  int iterations = 0;
  int converged = 0;
  double max_res = 0;
};

using OpFn = std::function<int(const double* X, double* Y, int m)>;
using PrecFn = std::function<int(double* T, int m, const int* d_idx, const double* X)>;

// Block Davidson (Davidson 1975, as used for Eq. chiisamatrixinpdep): the
// nwant lowest Ritz pairs are carried; the first nconv must reach
// ||A x - theta x|| <= tol (times |theta_1| when rel_tol).
int davidson(pdep_ctx* c, SysData& s, int nwant, int nconv, int nb_max, const double* start,
             int nstart, double tol, bool rel_tol, int max_iter, int zero_slot, OpFn op,
             PrecFn prec, double* X /*[nwant][ld]*/, double* theta_host, DavidsonOut* out,
             cudaStream_t st) {
  const int rows = s.n_pw;
  const long long ld = s.ld;
  nb_max = std::max(nb_max, 2 * nwant);
  double *B, *AB, *M, *Y, *th, *AX, *R, *T, *nr;
  int* idx;
  RET(ws(c, "dv_B", (size_t)nb_max * ld, &B));
  RET(ws(c, "dv_AB", (size_t)nb_max * ld, &AB));
  RET(ws(c, "dv_M", (size_t)nb_max * nb_max, &M));
  RET(ws(c, "dv_Y", (size_t)nb_max * nb_max, &Y));
  RET(ws(c, "dv_th", (size_t)nb_max, &th));
  RET(ws(c, "dv_AX", (size_t)nwant * ld, &AX));
  RET(ws(c, "dv_R", (size_t)nwant * ld, &R));
  RET(ws(c, "dv_T", (size_t)nwant * ld, &T));
  RET(ws(c, "dv_nr", (size_t)nwant, &nr));
  RET(ws(c, "dv_idx", (size_t)nwant, &idx));
  EighWork wk;
  RET(eigh_ws(c, nb_max, &wk));

  CK(cudaMemsetAsync(B, 0, sizeof(double) * (size_t)nb_max * ld, st));
  CK(cudaMemsetAsync(AB, 0, sizeof(double) * (size_t)nb_max * ld, st));
  CK(cudaMemcpy2DAsync(T, ld * sizeof(double), start, ld * sizeof(double), rows * sizeof(double),
                       nstart, cudaMemcpyDeviceToDevice, st));
  if (zero_slot >= 0) CK(zero_row(T, ld, zero_slot, nstart, st));
  int nb = 0;
  RET(orthonormalize(c, s, B, 0, T, nstart, B, &nb, st));
  if (nb < nwant) return fail(PDEP_ERR_INVALID_ARG, "start block is rank deficient");
  int lo = 0, hi = nb;
  std::vector<double> hth(nb_max), hnr(nwant);
  out->iterations = 0;
  out->converged = 0;
  for (int it = 0; it < max_iter; ++it) {
    NvtxRange nv("davidson_iteration");
    RET(op(B + (size_t)lo * ld, AB + (size_t)lo * ld, hi - lo));
    out->iterations = it + 1;
    // Rayleigh-Ritz in span(B)
    CK(gemm<double>(true, nb, nb, rows, 1.0, B, ld, AB, ld, 0.0, M, nb, st));
    CK(symmetrize<double>(M, nb, nb, st));
    CK(eigh(nb, M, nb, th, Y, nb, wk, st));
    CK(gemm<double>(false, rows, nwant, nb, 1.0, B, ld, Y, nb, 0.0, X, ld, st));
    CK(gemm<double>(false, rows, nwant, nb, 1.0, AB, ld, Y, nb, 0.0, AX, ld, st));
    CK(ritz_residual(AX, X, ld, rows, nwant, th, R, st));
    CK(col_norms<double>(R, ld, rows, nwant, nr, st));
    CK(cudaMemcpyAsync(hth.data(), th, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hnr.data(), nr, sizeof(double) * nwant, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double scale = rel_tol ? std::max(std::fabs(hth[0]), 1e-300) : 1.0;
    std::vector<int> unconv;
    double mres = 0;
    bool done = true;
    for (int i = 0; i < nwant; ++i) {
      const double r = hnr[i] / scale;
      if (i < nconv) {
        mres = std::max(mres, r);
        if (!(r <= tol)) done = false;
      }
      if (!(r <= tol)) unconv.push_back(i);
    }
    out->max_res = mres;
    for (int i = 0; i < nwant; ++i) theta_host[i] = hth[i];
    if (done) {
      out->converged = 1;
      break;
    }
    if (it == max_iter - 1) break;
    // corrections: residuals of the unconverged Ritz pairs
    const int m = (int)unconv.size();
    CK(cudaMemcpyAsync(idx, unconv.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
    CK(gather_cols(R, ld, T, ld, rows, idx, m, st));
    if (prec) RET(prec(T, m, idx, X));
    if (zero_slot >= 0) CK(zero_row(T, ld, zero_slot, m, st));
    if (nb + m > nb_max) {
      // restart from the Ritz vectors
      CK(cudaMemcpy2DAsync(B, ld * sizeof(double), X, ld * sizeof(double), rows * sizeof(double),
                           nwant, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpy2DAsync(AB, ld * sizeof(double), AX, ld * sizeof(double),
                           rows * sizeof(double), nwant, cudaMemcpyDeviceToDevice, st));
      nb = nwant;
    }
    int kept = 0;
    RET(orthonormalize(c, s, B, nb, T, m, B + (size_t)nb * ld, &kept, st));
    if (kept == 0) break;
    lo = nb;
    hi = nb + kept;
    nb += kept;
  }
  return PDEP_OK;
}

// ---------------------------------------------------------------------------
// setup: lowest n_occ + 1 eigenpairs of H (FP64)
// ---------------------------------------------------------------------------
// Rayleigh-Ritz of the ns orthonormal columns of Y (HY = H Y): Ritz vectors
// into X, H X into HX, values into theta (host), residual norms into rn (host).
int ritz(pdep_ctx* c, SysData& s, const double* Y, const double* HY, int ns, double* X,
         double* HX, double* R, std::vector<double>& theta, std::vector<double>& rn,
         cudaStream_t st) {
  double *M, *V, *th, *nr;
  RET(ws(c, "rz_m", (size_t)ns * ns, &M));
  RET(ws(c, "rz_v", (size_t)ns * ns, &V));
  RET(ws(c, "rz_th", (size_t)ns, &th));
  RET(ws(c, "rz_nr", (size_t)ns, &nr));
  EighWork wk;
  RET(eigh_ws(c, ns, &wk));
  CK(gemm<double>(true, ns, ns, s.n_pw, 1.0, Y, s.ld, HY, s.ld, 0.0, M, ns, st));
  CK(symmetrize<double>(M, ns, ns, st));
  CK(eigh(ns, M, ns, th, V, ns, wk, st));
  CK(gemm<double>(false, s.n_pw, ns, ns, 1.0, Y, s.ld, V, ns, 0.0, X, s.ld, st));
  CK(gemm<double>(false, s.n_pw, ns, ns, 1.0, HY, s.ld, V, ns, 0.0, HX, s.ld, st));
  CK(ritz_residual(HX, X, s.ld, s.n_pw, ns, th, R, st));
  CK(col_norms<double>(R, s.ld, s.n_pw, ns, nr, st));
  theta.resize(ns);
  rn.resize(ns);
  CK(cudaMemcpyAsync(theta.data(), th, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rn.data(), nr, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PDEP_OK;
}

// Orthonormalise the ns columns of Y in place (into OUT); refill dropped
// directions with seeded random vectors orthogonal to the kept ones.
int orthonormalize_full(pdep_ctx* c, SysData& s, double* Y, int ns, double* OUT,
                        unsigned long long seed, cudaStream_t st) {
  int kept = 0;
  RET(orthonormalize(c, s, nullptr, 0, Y, ns, OUT, &kept, st));
  for (int tries = 0; kept < ns && tries < 4; ++tries) {
    const int miss = ns - kept;
    CK(philox_normal(Y, s.ld, s.n_pw, miss, seed + 7919ULL * (tries + 1), 0ULL, st));
    int k2 = 0;
    RET(orthonormalize(c, s, OUT, kept, Y, miss, OUT + (size_t)kept * s.ld, &k2, st));
    kept += k2;
  }
  if (kept < ns) return fail(PDEP_ERR_NOT_CONVERGED, "could not complete an orthonormal block");
  return PDEP_OK;
}

// Lowest n_occ + 1 eigenpairs of H by Chebyshev-filtered subspace iteration
// (Zhou, Saad, Tiago, Chelikowsky, J. Comput. Phys. 219, 172 (2006)): each
// pass applies a degree-m Chebyshev polynomial that damps [a, b] (a = the
// block's largest Ritz value, b >= the top of the spectrum) to the whole
// block, then orthonormalises and does Rayleigh-Ritz.
int chfsi(pdep_ctx* c, SysData& s, int ns, int nconv, double tol, int max_iter, double* X,
          std::vector<double>& theta, int* iters, cudaStream_t st) {
  double *Y, *Z, *HY, *HX, *R;
  RET(ws(c, "cf_y", (size_t)ns * s.ld, &Y));
  RET(ws(c, "cf_z", (size_t)ns * s.ld, &Z));
  RET(ws(c, "cf_hy", (size_t)ns * s.ld, &HY));
  RET(ws(c, "cf_hx", (size_t)ns * s.ld, &HX));
  RET(ws(c, "cf_r", (size_t)ns * s.ld, &R));
  // upper bound of the spectrum: max kinetic + max potential
  double tmax = 0.0;
  for (double g : s.g2) tmax = std::max(tmax, 0.5 * g);
  const double b = tmax + s.vmax + 1e-3 * (1.0 + std::fabs(tmax));
  std::vector<double> rn;
  // Rayleigh-Ritz of the start block (X is orthonormal on entry)
  RET(apply_h<double>(c, s, X, HY, ns, nullptr, 0, false, false, st));
  CK(cudaMemcpy2DAsync(Y, s.ld * sizeof(double), X, s.ld * sizeof(double),
                       s.n_pw * sizeof(double), ns, cudaMemcpyDeviceToDevice, st));
  RET(ritz(c, s, Y, HY, ns, X, HX, R, theta, rn, st));
  const int degree = 10;
  for (int it = 0; it < max_iter; ++it) {
    double mres = 0.0;
    for (int i = 0; i < nconv; ++i) mres = std::max(mres, rn[i]);
    *iters = it;
    if (mres <= tol) return PDEP_OK;
    const double a = theta[ns - 1], a0 = theta[0];
    const double e = 0.5 * (b - a), cc = 0.5 * (b + a);
    double sigma = e / (a0 - cc);
    const double tau = 2.0 / sigma;
    // Y = (H X - c X) sigma / e   (H X is HX from the last Rayleigh-Ritz)
    CK(cheb_step(Y, HX, X, nullptr, s.ld, s.n_pw, ns, sigma / e, cc, 0.0, st));
    double* prev = X;   // X is overwritten as the recurrence advances
    double* cur = Y;
    double* nxt = Z;
    for (int k = 2; k <= degree; ++k) {
      const double sig2 = 1.0 / (tau - sigma);
      RET(apply_h<double>(c, s, cur, HY, ns, nullptr, 0, false, false, st));
      CK(cheb_step(nxt, HY, cur, prev, s.ld, s.n_pw, ns, 2.0 * sig2 / e, cc, -sigma * sig2, st));
      double* t = prev;
      prev = cur;
      cur = nxt;
      nxt = t;
      sigma = sig2;
    }
    // cur holds the filtered block; orthonormalise it into a buffer that is
    // neither cur nor X (the Rayleigh-Ritz below writes X)
    double* out = (cur == Y) ? Z : Y;
    RET(orthonormalize_full(c, s, cur, ns, out, c->opt.seed + 31ULL * it, st));
    RET(apply_h<double>(c, s, out, HY, ns, nullptr, 0, false, false, st));
    RET(ritz(c, s, out, HY, ns, X, HX, R, theta, rn, st));
  }
  *iters = max_iter;
  double mres = 0.0;
  for (int i = 0; i < nconv; ++i) mres = std::max(mres, rn[i]);
  return mres <= tol ? PDEP_OK : fail(PDEP_ERR_NOT_CONVERGED, "setup eigensolver did not converge");
}

int setup_states(pdep_ctx* c, SysData& s, cudaStream_t st) {
  NvtxRange nv("setup_states");
  const int nocc = s.n_occ;
  s.n_defl = std::max(0, std::min(c->opt.n_deflate, s.n_pw - nocc - 2));
  s.n_ext = nocc + s.n_defl;
  if (nocc + 1 > s.n_pw) return fail(PDEP_ERR_INVALID_ARG, "n_occ too large for the basis");
  const int ns = std::min(s.n_pw, s.n_ext + std::max(16, s.n_ext / 4));
  // start vectors: plane waves of lowest kinetic energy plus small noise
  std::vector<std::pair<double, int>> comps;
  comps.push_back({0.0, 2 * s.n_half});
  for (int k = 0; k < s.n_half; ++k) {
    comps.push_back({s.g2[k] + 1e-12 * k, 2 * k});
    comps.push_back({s.g2[k] + 1e-12 * k + 5e-13, 2 * k + 1});
  }
  std::sort(comps.begin(), comps.end());
  std::vector<int> hc(ns);
  for (int i = 0; i < ns; ++i) hc[i] = comps[i].second;
  int* dcomp;
  double *X0, *X;
  RET(ws(c, "su_comp", ns, &dcomp));
  RET(ws(c, "su_x0", (size_t)ns * s.ld, &X0));
  RET(ws(c, "su_x", (size_t)ns * s.ld, &X));
  CK(cudaMemcpyAsync(dcomp, hc.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  CK(unit_start(X0, s.ld, s.n_pw, dcomp, ns, 1e-3, c->opt.seed ^ 0x5eed5eedULL, st));
  RET(orthonormalize_full(c, s, X0, ns, X, c->opt.seed ^ 0x0f0fULL, st));
  std::vector<double> th;
  const int nwant = s.n_ext + 1;
  int its = 0;
  RET(chfsi(c, s, ns, nwant, c->opt.setup_tol, c->opt.setup_max_iter, X, th, &its, st));
  s.eps.assign(th.begin(), th.begin() + nwant);
  const double gap = s.eps[nocc] - s.eps[nocc - 1];
  if (!(gap >= c->opt.gap_min)) return fail(PDEP_ERR_NO_GAP, "HOMO-LUMO gap below gap_min");
  // sigma_w lifts occupied and deflated state w to eps_{n_ext}: in
  // H - eps_v + sum_w sigma_w |w><w| it then sits at eps_{n_ext} - eps_v > 0,
  // the lowest eigenvalue of the part the CG solves for
  const int next = s.n_ext;
  {
    std::vector<double> sg(next);
    std::vector<float> sg32(next);
    for (int w = 0; w < next; ++w) {
      sg[w] = s.eps[next] - s.eps[w];
      sg32[w] = (float)sg[w];
    }
    RET(persistent(c, &s.d_sigma64, next));
    RET(persistent(c, &s.d_sigma32, next));
    CK(cudaMemcpyAsync(s.d_sigma64, sg.data(), sizeof(double) * next, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s.d_sigma32, sg32.data(), sizeof(float) * next, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  RET(persistent(c, &s.d_psi, (size_t)next * s.ld));
  RET(persistent(c, &s.d_psif, (size_t)next * s.ld));
  RET(persistent(c, &s.d_eps_ext, next));
  CK(cudaMemcpyAsync(s.d_eps_ext, s.eps.data(), sizeof(double) * next, cudaMemcpyHostToDevice, st));
  RET(persistent(c, &s.d_u, (size_t)nocc * s.n_r));
  RET(persistent(c, &s.d_negeps, nocc));
  RET(persistent(c, &s.d_ekin, nocc));
  CK(cudaMemsetAsync(s.d_psi, 0, sizeof(double) * (size_t)next * s.ld, st));
  CK(cudaMemcpy2DAsync(s.d_psi, s.ld * sizeof(double), X, s.ld * sizeof(double),
                       s.n_pw * sizeof(double), next, cudaMemcpyDeviceToDevice, st));
  CK((convert<float, double>(s.d_psif, s.ld, s.d_psi, s.ld, s.ld, next, st)));
  RET(persistent(c, &s.d_psit5, tc5_split_floats(next, s.n_pw)));
  CK(tc5_split_states(next, s.n_pw, s.d_psif, s.ld, s.d_psit5, st));
  if (c->opt.precision == PDEP_MIXED_BF16) {
    RET(persistent(c, &s.d_psib16, tc5_split_bytes_bf16(next, s.n_pw) / 2));
    CK(tc5_split_states_bf16(next, s.n_pw, s.d_psif, s.ld, s.d_psib16, st));
  }
  std::vector<double> ne(nocc);
  for (int v = 0; v < nocc; ++v) ne[v] = -s.eps[v];
  CK(cudaMemcpyAsync(s.d_negeps, ne.data(), sizeof(double) * nocc, cudaMemcpyHostToDevice, st));
  RET(persistent(c, &s.d_negeps32, nocc));
  CK((convert<float, double>(s.d_negeps32, nocc, s.d_negeps, nocc, nocc, 1, st)));
  CK(kinetic_energy(s.d_psi, s.ld, s.n_half, nocc, s.d_g2, s.d_ekin, st));
  RET(persistent(c, &s.d_kprec64, (size_t)nocc * s.ld));
  RET(persistent(c, &s.d_kprec32, (size_t)nocc * s.ld));
  CK(build_precond(s.d_g2, s.n_half, s.n_pw, s.d_ekin, nocc, s.d_kprec64, s.d_kprec32, s.ld, st));
  // occupied states on the grid: u_v(r) = sum_G c_v(G) e^{iG.r}
  {
    ItemMap map{nocc, (nocc + 1) / 2};
    const int n_items = (nocc + 1) / 2;
    cpx<double>* b1;
    RET(ws(c, "b1_64", b1_count(s, n_items), &b1));
    CK(launch_cols_fwd<double>(s.sd, s.d_psi, s.ld, map, n_items, COEF_ONE, b1, st));
    SlabArgs<double> a{};
    a.mode = SLAB_TO_GRID;
    a.b1 = b1;
    a.n_items = n_items;
    a.out = s.d_u;
    a.out_stride = s.n_r;
    a.out_scale = 1.0;
    a.map = map;
    CK(launch_slab<double>(s.sd, a, st));
  }
  RET(sync(st));
  return PDEP_OK;
}

// ---------------------------------------------------------------------------
// Sternheimer solves: (H - eps_v + sum_w sigma_w |w><w|) x = b, w over the
// occupied and deflated states, b orthogonal to them (equivalent to Eq. stern
// on that subspace: H commutes with the projector, so x has no component
// along any w; the deflated states' share is added exactly, see split_rhs)
// ---------------------------------------------------------------------------
// The CG step's launch shape and the FP32 projection kernel are fixed once
// the autotuner has timed them (or autotuning is off); only then is the loop
// captured in a graph.
bool tuned(const pdep_ctx* c, const SysData& s, int pi) {
  if (!c->opt.autotune) return true;
  const bool pv_ok = pi == 1 || c->opt.proj_variant >= 0 || c->proj_variant >= 0 ||
                     c->opt.precision == PDEP_MIXED_BF16;
  const bool fused_ok = pi == 1 || !c->opt.fused_hpsi || hpsi_fused_smem(s.sf) == 0 ||
                        tune_done(c, "fused_planes:" + std::to_string(s.N[0]));
  return c->cg_variant[pi] >= 0 && pv_ok && fused_ok;
}
int cg_variant_of(const pdep_ctx* c, int pi) {
  return c->cg_variant[pi] >= 0 ? c->cg_variant[pi] : (int)CG_STREAM256;
}

// Workspace the step of a CG loop over n RHS needs (allocated before a
// capture, so that nothing is allocated while capturing).
template <typename R>
int cg_workspace(pdep_ctx* c, SysData& s, int n, R** r, R** p, R** ap, int** list) {
  const char* tag = sizeof(R) == 8 ? "64" : "32";
  std::string nr = std::string("cg_r") + tag, np = std::string("cg_p") + tag,
              na = std::string("cg_ap") + tag;
  RET(ws(c, nr.c_str(), (size_t)n * s.ld, r));
  RET(ws(c, np.c_str(), (size_t)n * s.ld, p));
  RET(ws(c, na.c_str(), (size_t)n * s.ld, ap));
  RET(ws(c, "cg_list", (size_t)n, list));
  cpx<R>* b1;
  RET(ws(c, sizeof(R) == 8 ? "b1_64" : "b1_32", b1_count(s, (n + 1) / 2), &b1));
  const int pv = c->opt.proj_variant >= 0 ? c->opt.proj_variant : c->proj_variant;
  R* S;
  if (sizeof(R) == 4 && pv != 0) {
    RET(ws(c, "pv_32", (size_t)((s.n_ext + 3) & ~3) * std::max(n, 1), &S));
  } else {
    RET(ws(c, sizeof(R) == 8 ? "pv_64" : "pv_32", (size_t)s.n_ext * std::max(n, 1), &S));
  }
  return PDEP_OK;
}

// Captures one CG loop over n RHS into an executable graph:
//   prologue: active = 0, cg_start (r = b, p = K b, active count), loop_begin
//   while (go): active list, A p on the listed RHS, PCG step, loop_next
// Launches inside are sized for n; the kernels read the list length from
// the device loop state.  All workspace is allocated beforehand (cg_workspace).
template <typename R>
int capture_cg_graph(pdep_ctx* c, SysData& s, CgArgs<R> a, const R* b, int n, int max_iter,
                     int* list, cudaGraphExec_t* out) {
  const int pi = sizeof(R) == 8 ? 1 : 0;
  cudaStream_t cs = c->cap_stream;
  const unsigned long long gen = c->ws_gen;
  cudaGraph_t g = nullptr, pro = nullptr, body = nullptr;
  cudaGraphConditionalHandle h = 0;
  int status = PDEP_OK, launches = 0;
  auto abort_capture = [&]() {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(cs, &junk);
    if (junk && junk != body) cudaGraphDestroy(junk);
    cudaGetLastError();
  };
  auto chk = [&](cudaError_t e) {
    if (e != cudaSuccess && status == PDEP_OK) {
      set_last_error(__FILE__, __LINE__, cudaGetErrorString(e));
      status = PDEP_ERR_CUDA;
    }
    return e == cudaSuccess;
  };
  if (!chk(cudaGraphCreate(&g, 0))) return status;
  if (chk(cudaGraphConditionalHandleCreate(&h, g, 0, 0)) &&
      chk(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed))) {
    capture_begin();
    bool ok = chk(cudaMemsetAsync(&c->d_loop->active, 0, sizeof(int), cs)) &&
              chk(cg_start<R>(a, b, s.ld, cs)) && chk(loop_begin(c->d_loop, max_iter, h, 1, cs));
    capture_end();
    if (ok) {
      chk(cudaStreamEndCapture(cs, &pro));
    } else {
      abort_capture();
    }
  }
  cudaGraphNode_t pn = nullptr, wn = nullptr;
  cudaGraphNodeParams cp{};
  if (status == PDEP_OK && chk(cudaGraphAddChildGraphNode(&pn, g, nullptr, 0, pro))) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (chk(cudaGraphAddNode(&wn, g, &pn, nullptr, 1, &cp))) body = cp.conditional.phGraph_out[0];
  }
  if (status == PDEP_OK &&
      chk(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) {
    capture_begin();
    bool ok = chk(active_list_reset(a.sc, n, list, &c->d_loop->listed, &c->d_loop->active, cs));
    if (ok) {
      const int r = apply_h<R>(c, s, a.p, (R*)a.ap, n, list, n, true, true, cs, nullptr,
                               &c->d_loop->listed);
      if (r != PDEP_OK) {
        status = r;
        ok = false;
      }
    }
    a.list_count = &c->d_loop->listed;
    ok = ok && chk(cg_step<R>(a, list, n, cs)) &&
         chk(loop_next(c->d_loop, max_iter, c->budget_ns, c->d_status, pi, h, 1, cs));
    launches = capture_end();
    if (ok) {
      cudaGraph_t got = body;
      chk(cudaStreamEndCapture(cs, &got));
    } else {
      abort_capture();
    }
  }
  if (status == PDEP_OK && c->ws_gen != gen)
    status = fail(PDEP_ERR_CUDA, "workspace moved while capturing a CG graph");
  if (status == PDEP_OK) chk(cudaGraphInstantiate(out, g, 0));
  if (pro) cudaGraphDestroy(pro);
  cudaGraphDestroy(g);
  if (status == PDEP_OK) c->body_launches[pi] = launches;
  return status;
}

// Sternheimer PCG on (H - eps_v + sum_w sigma_w |w><w|) x = b for n RHS
// (b, x: [n][ld]), each to ||r|| <= tol ||b|| or max_iter steps.  mask
// (optional, device): RHS i takes part only if mask[i] != 0.  The loop runs on
// the device: a CUDA graph with a while node whose body is one CG step and a
// control kernel (no host round trip per step).  While the autotuner is
// still timing launch shapes (or use_graph is 0) the same steps are launched
// from a host loop that reads the control flag after each step.
template <typename R>
int cg_loop(pdep_ctx* c, SysData& s, const R* b, R* x, int n, double tol, int max_iter,
            CgScal* sc, const double* mask, cudaStream_t st, const double* tolv) {
  const int si = (int)(&s - c->sys.data());
  // H x inside this loop is the inner CG's (restored on every return)
  struct InnerFlag {
    bool& f;
    bool old;
    InnerFlag(bool& ff, bool v) : f(ff), old(ff) { f = v; }
    ~InnerFlag() { f = old; }
  } inner_flag(c->cg_inner, sizeof(R) == 4);
  R *r, *p, *ap;
  int* list;
  RET(cg_workspace<R>(c, s, n, &r, &p, &ap, &list));
  const int pi = sizeof(R) == 8 ? 1 : 0;
  CgArgs<R> a{};
  a.x = x;
  a.r = r;
  a.p = p;
  a.ap = ap;
  a.ld = s.ld;
  a.n_pw = s.n_pw;
  a.n_half = s.n_half;
  a.n_rhs = n;
  a.kprec = kprec_of(s, (R*)nullptr);
  a.n_occ = s.n_occ;
  a.sc = sc;
  a.tol = tol;
  a.status = c->d_status;
  a.n_active = &c->d_loop->active;
  a.mask = mask;
  a.tolv = tolv;
  // loops under 256 RHS are never timed by the autotuner: they run the
  // current (or default) shapes and are captured right away
  const bool graph = c->opt.use_graph && (tuned(c, s, pi) || n < 256);
  if (!graph) {
    // eager: host loop, one 8-byte read of the loop state per step
    CK(cudaMemsetAsync(&c->d_loop->active, 0, sizeof(int), st));
    CK(cg_start<R>(a, b, s.ld, st));
    CK(loop_begin(c->d_loop, max_iter, 0, 0, st));
    for (;;) {
      // active, listed, iter, go: one 16-byte read per step
      CK(cudaMemcpyAsync(c->h_pin, &c->d_loop->active, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                         st));
      CK(cudaStreamSynchronize(st));
      int h[4];
      memcpy(h, c->h_pin, sizeof(h));
      if (!h[3]) break;
      const int n_act = h[0];
      CK(active_list_reset(sc, n, list, &c->d_loop->listed, &c->d_loop->active, st));
      RET(apply_h<R>(c, s, p, ap, n, list, n_act, true, true, st));
      // Autotuner: while untuned, each large step tries the next launch shape
      // (all shapes compute the same update) and its time per RHS is kept;
      // afterwards the fastest shape is used.
      const bool tuning = c->opt.autotune && c->cg_variant[pi] < 0 && n_act >= 256;
      a.variant = tuning ? c->cg_tune_next[pi] : cg_variant_of(c, pi);
      a.list_count = nullptr;
      if (tuning) CK(cudaEventRecord(c->ev[0], st));
      CK(cg_step<R>(a, list, n_act, st));
      if (tuning) {
        CK(cudaEventRecord(c->ev[1], st));
        CK(cudaEventSynchronize(c->ev[1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->cg_tune_ms[pi][a.variant] = ms / n_act;
        if (++c->cg_tune_next[pi] == CG_NUM_VARIANTS) {
          int best = 0;
          for (int v = 1; v < CG_NUM_VARIANTS; ++v)
            if (c->cg_tune_ms[pi][v] < c->cg_tune_ms[pi][best]) best = v;
          c->cg_variant[pi] = best;
        }
      }
      CK(loop_next(c->d_loop, max_iter, c->budget_ns, c->d_status, pi, 0, 0, st));
      ++c->eager_steps[pi];
    }
    return PDEP_OK;
  }
  a.variant = cg_variant_of(c, pi);
  int pv = c->opt.proj_variant >= 0 ? c->opt.proj_variant : c->proj_variant;
  if (pv < 0) pv = 1;  // what apply_h uses while the projection kernel is untimed
  CgGraph* g = nullptr;
  for (CgGraph& e : c->cg_graphs)
    if (e.prec == pi && e.sys == si && e.n == n && e.max_iter == max_iter && e.tol == tol &&
        e.b == b && e.x == x && e.sc == sc && e.mask == mask && e.tolv == tolv &&
        e.ws_gen == c->ws_gen &&
        e.cg_variant == a.variant && e.proj_variant == pv && e.budget_ns == c->budget_ns &&
        e.tune_gen == c->tune_gen) {
      g = &e;
      break;
    }
  if (!g) {
    CgGraph e{};
    e.prec = pi;
    e.sys = si;
    e.n = n;
    e.max_iter = max_iter;
    e.tol = tol;
    e.b = b;
    e.x = x;
    e.sc = sc;
    e.mask = mask;
    e.tolv = tolv;
    e.ws_gen = c->ws_gen;
    e.cg_variant = a.variant;
    e.proj_variant = pv;
    e.budget_ns = c->budget_ns;
    e.tune_gen = c->tune_gen;
    RET(capture_cg_graph<R>(c, s, a, b, n, max_iter, list, &e.exec));
    if (c->cg_graphs.size() >= 16) {
      cudaGraphExecDestroy(c->cg_graphs.front().exec);
      c->cg_graphs.erase(c->cg_graphs.begin());
    }
    c->cg_graphs.push_back(e);
    g = &c->cg_graphs.back();
  }
  {
    ProfScope ps(sizeof(R) == 8 ? PC_CG_GRAPH_F64 : PC_CG_GRAPH_F32, st, 0.0, 0.0);
    CK(cudaGraphLaunch(g->exec, st));
  }
  ++c->graph_launches;
  return PDEP_OK;
}

// Refinement rounds (iterative refinement written in solution updates):
// round k solves A delta = r for every RHS still above cg_tol, with an inner
// CG in precision Ri on the residual scaled to unit norm, then x += delta
// and r -= A delta with A delta in FP64 arithmetic (or double-float, mixed
// modes) and the density response of delta accumulated by that same
// transform (dn is linear in x).  The FP64 path runs its inner solve to
// 0.9 cg_tol (round 0) or 0.5 cg_tol (later rounds) of ||b_i|| through
// per-RHS inner tolerances, so a second round only catches RHS whose
// recomputed residual drifted above the recursion's; the mixed modes run
// each FP32 inner solve to inner_tol.  d_refine[0] holds a round's
// unconverged count: the A delta and the residual update run on that many
// listed RHS (launches sized for n).  Rounds whose list is empty cost only
// their launches.
// Relative reduction each FP32 inner solve aims for.  With BF16
// coefficients the CG operator is perturbed at about 2^-9 of the projection
// term, so a round gains little more than ~3e-3 however long the inner CG
// runs (measured on 48^3: 5 rounds whatever the inner tolerance, fastest at
// 3e-3): the inner CG stops there.
inline double inner_tol_of(const pdep_ctx* c) {
  return c->opt.precision == PDEP_MIXED_BF16 ? std::max(c->opt.inner_tol, 3e-3)
                                             : c->opt.inner_tol;
}

template <typename Ri>
int refine_rounds(pdep_ctx* c, SysData& s, const double* b, const double* xd, double* x, int n,
                  double* dn, int* its_total, double* rel, double* r64, double* ad,
                  cudaStream_t st) {
  const bool fp64 = sizeof(Ri) == 8;
  const double tol = c->opt.cg_tol;
  const char* tag = fp64 ? "64" : "32";
  Ri *ri, *di;
  double *rn, *dl, *tolv = nullptr;
  CgScal* sc;
  int* list;
  RET(ws(c, (std::string("rf_r") + tag).c_str(), (size_t)n * s.ld, &ri));
  RET(ws(c, (std::string("rf_d") + tag).c_str(), (size_t)n * s.ld, &di));
  RET(ws(c, "mx_rn", (size_t)n, &rn));
  RET(ws(c, (std::string("cg_sc") + tag).c_str(), (size_t)n, &sc));
  RET(ws(c, "mx_list", (size_t)n, &list));
  RET(ws(c, "sv_dl", (size_t)n * s.ld, &dl));
  if (fp64) RET(ws(c, "rf_tolv", (size_t)n, &tolv));
  // mixed modes, df_refine 2: after the first round the correction delta is
  // about inner_tol of the solution, so its product A delta (and its share
  // of the density response) in FP32 errs by ~1e-7 inner_tol ||b||, far
  // below cg_tol: those rounds run the FP32 transforms on an FP32 copy
  float *dlf = nullptr, *adf = nullptr;
  const bool f32_later = !fp64 && c->opt.df_refine == 2;
  if (f32_later) {
    RET(ws(c, "rf_dlf", (size_t)n * s.ld, &dlf));
    RET(ws(c, "rf_adf", (size_t)n * s.ld, &adf));
  }
  CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n * s.ld, st));
  CK(fill_value(rel, n, 1.0, st));
  int* n_un = c->d_refine;
  for (int round = 0; round < c->opt.max_refine; ++round) {
    NvtxRange nv("refinement_round");
    CK(unconverged_list(rel, tol, n, list, n_un, st, &c->d_dstats->rounds_cur));
    CK(refine_prepare<Ri>(r64, s.ld, s.n_pw, n, rel, tol, ri, s.ld, rn, st, tolv,
                          (round == 0 ? 0.9 : 0.5) * tol, 0.5));
    if (fp64)
      RET(cg_loop<Ri>(c, s, ri, di, n, 0.0, c->opt.cg_max_iter, sc, rn, st, tolv));
    else
      RET(cg_loop<Ri>(c, s, ri, di, n, inner_tol_of(c), c->opt.inner_max_iter, sc, rn, st,
                      nullptr));
    CK(cg_collect(sc, n, its_total, c->d_dstats, st));
    // delta = rn d (+ xd in the first round, when every RHS is listed)
    const double* xr = round == 0 ? xd : nullptr;
    const bool f32_round = f32_later && round > 0;
    CK(refine_delta<Ri>(x, dl, s.ld, di, s.ld, s.n_pw, n, rn, xr, st, f32_round ? dlf : nullptr));
    if (f32_round) {
      RET(apply_h<float>(c, s, dlf, adf, n, list, n, true, true, st, dn, n_un));
      CK(residual_update(r64, adf, b, s.ld, s.n_pw, n, rel, list, xr, s.d_sigma64, s.n_occ, st,
                         n_un));
      continue;
    }
    if (!fp64 && c->opt.df_refine)
      RET(apply_h<df>(c, s, dl, ad, n, list, n, true, true, st, dn, n_un));
    else
      RET(apply_h<double>(c, s, dl, ad, n, list, n, true, true, st, dn, n_un));
    CK(residual_update(r64, ad, b, s.ld, s.n_pw, n, rel, list, xr, s.d_sigma64, s.n_occ, st,
                       n_un));
  }
  return PDEP_OK;
}

// Solve for n right-hand sides b (FP64, [n][ld]); x out (FP64).  Nothing is
// read back to the host: per-RHS iteration counts accumulate in its_total
// (device, may be null), the FP64 relative residuals are left in 'rel'
// (device, [n]), and the statistics and the not-converged condition go to the
// device statistics and status word.
int solve_rhs(pdep_ctx* c, SysData& s, const double* b, const double* xd, double* x, int n,
              double* dn, int* its_total, double** rel_out, cudaStream_t st) {
  double *rel, *r64, *ad;
  RET(ws(c, "sv_rel", (size_t)n, &rel));
  RET(ws(c, "sv_r64", (size_t)n * s.ld, &r64));
  RET(ws(c, "sv_ap64", (size_t)n * s.ld, &ad));
  if (rel_out) *rel_out = rel;
  if (its_total) CK(cudaMemsetAsync(its_total, 0, sizeof(int) * (size_t)n, st));
  CK(cudaMemsetAsync(&c->d_dstats->rounds_cur, 0, sizeof(int), st));
  // r64 = b: the FP64 residual, updated as r -= A delta for every update
  // delta of x (and checked against b's norm)
  CK(cudaMemcpyAsync(r64, b, sizeof(double) * (size_t)n * s.ld, cudaMemcpyDeviceToDevice, st));
  if (dn) CK(cudaMemsetAsync(dn, 0, sizeof(double) * (size_t)(n / s.n_occ) * s.n_r, st));
  if (c->opt.precision == PDEP_FP64)
    RET(refine_rounds<double>(c, s, b, xd, x, n, dn, its_total, rel, r64, ad, st));
  else
    RET(refine_rounds<float>(c, s, b, xd, x, n, dn, its_total, rel, r64, ad, st));
  // rel holds the FP64 residual of every RHS from its last update.  No final
  // P_c projection is needed: the shifted operator lifts occupied state w to
  // eps_{n_ext} - eps_v > 0, so the occupied component of x is at most
  // ||b - A x|| / (eps_{n_ext} - eps_v).
  CK(solve_finish(rel, n, c->opt.cg_tol, c->d_dstats, c->d_status, st));
  c->st_solves += n;
  return PDEP_OK;
}

// b_vj = -P_c [dV_j psi_v] for perturbation grids dv [m][n_r]  -> bvec [m*n_occ][ld].
// With deflation, bvec keeps only the part orthogonal to the deflated states
// and xdefl [m*n_occ][ld] receives their exact share of the solution.
// occupied_only: bvec = -P_c [dV_j psi_v] with P_c over the occupied states
// alone (no deflation split; xdefl unused).
// The products dV_j psi_v and their transforms to the sphere (C: FP64, or
// double-float in the mixed modes; vectors FP64 either way).
template <typename C>
int rhs_transform(pdep_ctx* c, SysData& s, const double* dv, int m, double* bvec,
                  cudaStream_t st) {
  const int nocc = s.n_occ;
  ItemMap map{nocc, (nocc + 1) / 2};
  const int n_items = m * ((nocc + 1) / 2);
  cpx<C>* b1;
  RET(ws(c, "b1_64", b1_count(s, n_items), &b1));
  SlabArgs<C> a{};
  a.mode = SLAB_FROM_GRID;
  a.b1 = b1;
  a.n_items = n_items;
  a.src.f = dv;
  a.src.f_stride = s.n_r;
  a.src.g = s.d_u;
  a.src.g_stride = s.n_r;
  a.map = map;
  const SphereDev<C>& sd = sph(s, (C*)nullptr);
  CK(launch_slab<C>(sd, a, st));
  Epilogue<C> ep{};
  ep.y = bvec;
  ep.ldy = s.ld;
  ep.shift_period = 1;
  ep.scale = C(-1.0 / s.n_r);
  ep.coef = COEF_ONE;
  CK(launch_cols_bwd<C>(sd, b1, map, n_items, ep, st));
  return PDEP_OK;
}

int build_rhs(pdep_ctx* c, SysData& s, const double* dv, int m, double* bvec, double* xdefl,
              cudaStream_t st, bool occupied_only = false) {
  const int nocc = s.n_occ;
  if (c->opt.precision != PDEP_FP64 && c->opt.df_refine)
    RET(rhs_transform<df>(c, s, dv, m, bvec, st));
  else
    RET(rhs_transform<double>(c, s, dv, m, bvec, st));
  if (occupied_only) {
    double* S;
    RET(ws(c, "po_S", (size_t)nocc * m * nocc, &S));
    CK(gemm<double>(true, nocc, m * nocc, s.n_pw, 1.0, s.d_psi, s.ld, bvec, s.ld, 0.0, S, nocc, st));
    CK(gemm<double>(false, s.n_pw, m * nocc, nocc, -1.0, s.d_psi, s.ld, S, nocc, 1.0, bvec, s.ld,
                    st));
    return PDEP_OK;
  }
  RET(split_rhs(c, s, bvec, m * nocc, xdefl, st));
  return PDEP_OK;
}

// dV_j(r) = Omega^{-1/2} sum_G sqrt(4pi)/|G| phi_j(G) e^{iG.r} for m PDEP
// vectors phi [m][ld] -> dv [m][n_r]
int perturbation_grids(pdep_ctx* c, SysData& s, const double* phi, int m, double* dv,
                       cudaStream_t st) {
  ItemMap map{m, (m + 1) / 2};
  const int n_items = (m + 1) / 2;
  cpx<double>* b1;
  RET(ws(c, "b1_64", b1_count(s, n_items), &b1));
  CK(launch_cols_fwd<double>(s.sd, phi, s.ld, map, n_items, COEF_SQRT_COULOMB, b1, st));
  SlabArgs<double> a{};
  a.mode = SLAB_TO_GRID;
  a.b1 = b1;
  a.n_items = n_items;
  a.out = dv;
  a.out_stride = s.n_r;
  a.out_scale = 1.0 / std::sqrt(s.omega);
  a.map = map;
  CK(launch_slab<double>(s.sd, a, st));
  return PDEP_OK;
}

// chi0bar phi for m PDEP vectors (internal layout [m][ld], G=0 slot zero)
int chi0_internal(pdep_ctx* c, SysData& s, const double* phi, int m, double* out, double* dn_out,
                  cudaStream_t st) {
  NvtxRange nv("chi0bar_apply");
  const int nocc = s.n_occ;
  // perturbation chunk: keep roughly 10 vectors of n_rhs*ld doubles bounded
  size_t per = (size_t)nocc * s.ld * sizeof(double) * 10 + b1_count(s, (nocc + 1) / 2) * 24 +
               (size_t)s.n_r * 16;
  size_t budget = (size_t)24 << 30;
  if (c->opt.workspace_limit_bytes) budget = c->opt.workspace_limit_bytes / 2;
  int mc_max = (int)std::max<size_t>(1, budget / per);
  // every chunk is solved and written; a solve left above cg_tol only marks
  // the device status word
  c->st_chunks = 0;
  for (int j0 = 0; j0 < m; j0 += mc_max) {
    ++c->st_chunks;
    const int mc = std::min(mc_max, m - j0);
    double *dv, *bvec, *xvec, *dn;
    RET(ws(c, "c0_dv", (size_t)mc * s.n_r, &dv));
    RET(ws(c, "c0_b", (size_t)mc * nocc * s.ld, &bvec));
    RET(ws(c, "c0_x", (size_t)mc * nocc * s.ld, &xvec));
    if (dn_out)
      dn = dn_out + (size_t)j0 * s.n_r;
    else
      RET(ws(c, "c0_dn", (size_t)mc * s.n_r, &dn));
    // dV_j(r) = Omega^{-1/2} sum_G sqrt(4pi)/|G| phi_j(G) e^{iG.r}
    RET(perturbation_grids(c, s, phi + (size_t)j0 * s.ld, mc, dv, st));
    double* xd = nullptr;
    if (s.n_defl > 0) RET(ws(c, "c0_xd", (size_t)mc * nocc * s.ld, &xd));
    RET(build_rhs(c, s, dv, mc, bvec, xd, st));
    // the density response dn (Eq. deltani) is accumulated inside the
    // solver's FP64 transforms of the solution updates
    RET(solve_rhs(c, s, bvec, xd, xvec, mc * nocc, dn, nullptr, nullptr, st));
    // (chi0bar phi_j)(G) = sqrt(4pi)/|G| * Omega^{1/2}/N_r * FFT[dn_j](G)
    {
      ItemMap map{mc, (mc + 1) / 2};
      const int n_items = (mc + 1) / 2;
      cpx<double>* b1;
      RET(ws(c, "b1_64", b1_count(s, n_items), &b1));
      SlabArgs<double> a{};
      a.mode = SLAB_FROM_GRID;
      a.b1 = b1;
      a.n_items = n_items;
      a.src.g = dn;
      a.src.g_stride = s.n_r;
      a.map = map;
      CK(launch_slab<double>(s.sd, a, st));
      Epilogue<double> ep{};
      ep.y = out + (size_t)j0 * s.ld;
      ep.ldy = s.ld;
      ep.shift_period = 1;
      ep.scale = std::sqrt(s.omega) / s.n_r;
      ep.coef = COEF_SQRT_COULOMB;
      CK(launch_cols_bwd<double>(s.sd, b1, map, n_items, ep, st));
    }
  }
  return PDEP_OK;
}

int check_sys(const pdep_ctx* c, int sys) {
  if (!c) return fail(PDEP_ERR_INVALID_ARG, "null context");
  if (sys < 0 || sys >= (int)c->sys.size()) return fail(PDEP_ERR_INVALID_ARG, "bad system index");
  return PDEP_OK;
}

int reset_stats(pdep_ctx* c, cudaStream_t st) {
  c->st_solves = 0;
  c->st_chunks = 0;
  c->graph_launches = 0;
  c->eager_steps[0] = c->eager_steps[1] = 0;
  c->st_launch0 = launch_count();
  CK(cudaMemsetAsync(c->d_dstats, 0, sizeof(DevStats), st));
  CK(cudaMemsetAsync(c->d_loop->steps, 0, sizeof(c->d_loop->steps), st));
  return PDEP_OK;
}

// Synchronises st and fills the solve statistics (device counters included).
int read_stats(pdep_ctx* c, pdep_stats* out, cudaStream_t st) {
  DevStats d;
  unsigned long long steps[2];
  CK(cudaMemcpyAsync(&d, c->d_dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(steps, c->d_loop->steps, sizeof(steps), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  out->sternheimer_solves = c->st_solves;
  out->cg_iterations = (long long)d.cg_iters;
  out->cg_iterations_max = d.cg_max;
  out->refine_rounds_max = d.refine_max;
  double mr;
  memcpy(&mr, &d.max_res_bits, sizeof(double));
  out->max_cg_residual = mr;
  out->cg_variant = c->cg_variant[c->opt.precision == PDEP_FP64 ? 1 : 0];
  out->proj_variant = c->opt.precision == PDEP_MIXED_BF16
                          ? 3
                          : (c->opt.proj_variant >= 0 ? c->opt.proj_variant : c->proj_variant);
  out->chi0_chunks = c->st_chunks;
  // launches outside graphs are counted on the host; a graph contributes its
  // prologue (2 kernels) per launch and its body per step, the steps counted
  // on the device (loop_next counts eager steps too: those are subtracted)
  long long in_graphs = 2 * c->graph_launches;
  for (int pi = 0; pi < 2; ++pi)
    in_graphs += ((long long)steps[pi] - c->eager_steps[pi]) * c->body_launches[pi];
  out->kernel_launches = (launch_count() - c->st_launch0) + in_graphs;
  out->graph_launches = c->graph_launches;
  out->fused_planes = -1;
  out->gemm_shape = -1;
  for (const auto& kv : c->tunes) {
    if (kv.second.best < 0) continue;
    if (kv.first.rfind("fused_planes:", 0) == 0 && !c->sys.empty()) {
      const int G0 = hpsi_fused_planes(c->sys[0].sf);
      const int k = kv.second.best;
      out->fused_planes = k == 0 ? G0 : k == 1 ? std::max(1, G0 / 2) : 2 * G0;
    }
    if (kv.first.rfind("pv_", 0) == 0) out->gemm_shape = kv.second.best;
  }
  return PDEP_OK;
}

int solve_one(pdep_ctx* c, int si, const double* phi0, double* eigvals, double* eigvecs,
              pdep_stats* stats, cudaStream_t st) {
  NvtxRange nv("pdep_solve");
  SysData& s = c->sys[si];
  const int np = s.n_pdep;
  const int dim = s.n_pw - 1;
  if (np > dim) return fail(PDEP_ERR_INVALID_ARG, "n_pdep exceeds the PDEP dimension");
  double *start, *X;
  RET(ws(c, "pd_start", (size_t)np * s.ld, &start));
  RET(ws(c, "pd_X", (size_t)np * s.ld, &X));
  CK(cudaMemsetAsync(start, 0, sizeof(double) * (size_t)np * s.ld, st));
  if (phi0) {
    CK(cudaMemcpy2DAsync(start, s.ld * sizeof(double), phi0, dim * sizeof(double),
                         dim * sizeof(double), np, kind_to_dev(phi0), st));
  } else {
    CK(philox_normal(start, s.ld, dim, np, c->opt.seed, 0ULL, st));
  }
  OpFn op = [&](const double* in, double* outv, int m) -> int {
    return chi0_internal(c, s, in, m, outv, nullptr, st);
  };
  std::vector<double> th(np);
  DavidsonOut dout;
  const bool fixed = !(c->opt.dav_tol > 0);
  RET(davidson(c, s, np, np, std::max(2, c->opt.dav_subspace_factor) * np, start, np,
               fixed ? 0.0 : c->opt.dav_tol, true, c->opt.dav_max_iter, s.n_pw - 1, op, nullptr,
               X, th.data(), &dout, st));
  RET(copy_from_host(eigvals, th.data(), sizeof(double) * np, st));
  if (eigvecs)
    CK(cudaMemcpy2DAsync(eigvecs, dim * sizeof(double), X, s.ld * sizeof(double),
                         dim * sizeof(double), np, kind_from_dev(eigvecs), st));
  RET(sync(st));
  if (stats) {
    stats->dav_iterations += dout.iterations;
    if (!fixed && !dout.converged) stats->converged = 0;
    stats->max_dav_residual = std::max(stats->max_dav_residual, dout.max_res);
  }
  if (!fixed && !dout.converged) return fail(PDEP_ERR_NOT_CONVERGED, "Davidson did not converge");
  return PDEP_OK;
}

}  // namespace

namespace pdep {
// Sphere description and potential of one system for pdep_apply_hamiltonian_noalloc.
int noalloc_sphere(pdep_ctx* c, int sys, SphereDev<double>* sd, const double** v, int* n_pw,
                   int* device) {
  RET(check_sys(c, sys));
  const SysData& s = c->sys[sys];
  *sd = s.sd;
  *v = s.d_v;
  *n_pw = s.n_pw;
  *device = c->device;
  return PDEP_OK;
}
}  // namespace pdep

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// Lanczos chains of H~ = P_c H P_c on the nc vectors of W ([nc][ld], already
// projected with P_c; W is overwritten), whose norms before the projection
// are r0 [nc]: Q [K][nc][ld] (step-major), alpha and beta [nc][K], and the
// tridiagonal eigen-decompositions d [nc][K], U [nc][K][K].
int lanczos_core(pdep_ctx* c, SysData& s, double* W, const double* r0, int nc, int K, double* Q,
                 double* da, double* db, double* dd, double* dU, cudaStream_t st) {
  double* S;
  RET(ws(c, "lz_S", (size_t)s.n_occ * nc, &S));
  CK(cudaMemsetAsync(da, 0, sizeof(double) * (size_t)nc * K, st));
  CK(cudaMemsetAsync(db, 0, sizeof(double) * (size_t)nc * K, st));
  CK(lanczos_start(W, s.ld, s.n_pw, nc, K, r0, Q, db, st));
  for (int k = 0; k < K; ++k) {
    double* Qk = Q + (size_t)k * nc * s.ld;
    // W = P_c H q_k (q_k lies in range(P_c), so this is H~ q_k)
    RET(apply_h<double>(c, s, Qk, W, nc, nullptr, 0, false, false, st));
    CK(gemm<double>(true, s.n_occ, nc, s.n_pw, 1.0, s.d_psi, s.ld, W, s.ld, 0.0, S, s.n_occ, st));
    CK(gemm<double>(false, s.n_pw, nc, s.n_occ, -1.0, s.d_psi, s.ld, S, s.n_occ, 1.0, W, s.ld,
                    st));
    const double* Qkm1 = k > 0 ? Q + (size_t)(k - 1) * nc * s.ld : nullptr;
    double* Qk1 = k + 1 < K ? Q + (size_t)(k + 1) * nc * s.ld : nullptr;
    CK(lanczos_step(W, Qk, Qkm1, Qk1, s.ld, s.n_pw, nc, K, k, da, db, st));
  }
  CK(tridiag_eig(da, db, nc, K, dd, dU, st));
  return PDEP_OK;
}

// P_c X for the n columns of X [n][ld] with the occupied states only
int project_occupied(pdep_ctx* c, SysData& s, double* X, int n, cudaStream_t st) {
  double* S;
  RET(ws(c, "po_S", (size_t)s.n_occ * n, &S));
  CK(gemm<double>(true, s.n_occ, n, s.n_pw, 1.0, s.d_psi, s.ld, X, s.ld, 0.0, S, s.n_occ, st));
  CK(gemm<double>(false, s.n_pw, n, s.n_occ, -1.0, s.d_psi, s.ld, S, s.n_occ, 1.0, X, s.ld, st));
  return PDEP_OK;
}

extern "C" {

void pdep_default_options(pdep_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = PDEP_FP64;
  o->cg_tol = 1e-10;
  o->cg_max_iter = 2000;
  o->inner_tol = 1e-5;
  o->inner_max_iter = 1000;
  o->max_refine = 6;
  o->dav_tol = 1e-8;
  o->dav_max_iter = 30;
  o->dav_subspace_factor = 4;
  o->seed = 1501031410ULL;
  o->gap_min = 1e-3;
  o->setup_tol = 1e-11;
  o->setup_max_iter = 400;
  o->workspace_limit_bytes = 0;
  o->n_deflate = 16;
  o->proj_variant = -1;
  o->clock_budget_cycles = 0;
  o->autotune = 1;
  o->use_graph = 1;
  o->df_refine = 2;
  o->fused_hpsi = 1;
}

const char* pdep_status_string(int s) {
  switch (s) {
    case PDEP_OK: return "ok";
    case PDEP_ERR_INVALID_ARG: return "invalid argument";
    case PDEP_ERR_CUDA: return "CUDA error";
    case PDEP_ERR_OOM: return "out of device memory";
    case PDEP_ERR_NO_GAP: return "no gap at the Fermi level";
    case PDEP_ERR_NOT_CONVERGED: return "not converged";
    case PDEP_ERR_NONFINITE: return "non-finite value";
    case PDEP_ERR_TIMEOUT: return "timeout";
    case PDEP_ERR_UNSUPPORTED: return "unsupported";
    case PDEP_ERR_BOUNDS: return "index out of range (bounds-checked build)";
  }
  return "unknown status";
}

const char* pdep_last_error(void) { return g_last_error.c_str(); }

int pdep_sync_status(pdep_ctx* c, void* stream) {
  if (!c) return fail(PDEP_ERR_INVALID_ARG, "null context");
  cudaStream_t st = (cudaStream_t)stream;
  const int r = check_status(c, st);
  CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), st));
  CK(cudaStreamSynchronize(st));
  return r;
}

int pdep_bounds_checked(void) {
#ifdef PDEP_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

void pdep_destroy(pdep_ctx* c) {
  if (!c) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  c->eig_graphs.release();
  for (CgGraph& g : c->cg_graphs) cudaGraphExecDestroy(g.exec);
  c->cg_graphs.clear();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->d_loop) cudaFree(c->d_loop);
  if (c->d_dstats) cudaFree(c->d_dstats);
  if (c->d_refine) cudaFree(c->d_refine);
  for (auto& kv : c->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  for (void* p : c->owned) cudaFree(p);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_counter) cudaFree(c->d_counter);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  cudaSetDevice(cur);
  delete c;
}

int pdep_setup(const pdep_system_desc* sys, int n_sys, const pdep_options* opt, void* stream,
               pdep_ctx** out) {
  if (!out) return fail(PDEP_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (!sys || n_sys <= 0) return fail(PDEP_ERR_INVALID_ARG, "no systems");
  cudaStream_t st = (cudaStream_t)stream;
  pdep_ctx* c = new pdep_ctx();
  if (opt)
    c->opt = *opt;
  else
    pdep_default_options(&c->opt);
  auto bail = [&](int r) {
    pdep_destroy(c);
    return r;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(fail(PDEP_ERR_CUDA, "no CUDA device"));
  if (upload_local_twiddles() != cudaSuccess) return bail(fail(PDEP_ERR_CUDA, "twiddle upload"));
  if (dev_timers_init() != 0) return bail(fail(PDEP_ERR_OOM, "device timers"));
  if (c->opt.precision != PDEP_FP64 && c->opt.precision != PDEP_MIXED_TF32 &&
      c->opt.precision != PDEP_MIXED_BF16)
    return bail(fail(PDEP_ERR_INVALID_ARG, "unknown precision mode"));
  if (c->opt.clock_budget_cycles < 0) return bail(fail(PDEP_ERR_INVALID_ARG, "negative clock budget"));
  if (c->opt.df_refine < 0 || c->opt.df_refine > 2)
    return bail(fail(PDEP_ERR_INVALID_ARG, "unknown df_refine mode"));
  if (c->opt.proj_variant < -1 || c->opt.proj_variant > 2)
    return bail(fail(PDEP_ERR_INVALID_ARG, "unknown projection kernel"));
  if (cudaMalloc(&c->d_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->d_counter, 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_loop, sizeof(CgLoopState)) != cudaSuccess ||
      cudaMalloc(&c->d_dstats, sizeof(DevStats)) != cudaSuccess ||
      cudaMalloc(&c->d_refine, 4 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_pin, 16 * sizeof(int)) != cudaSuccess)
    return bail(fail(PDEP_ERR_OOM, "context allocation"));
  cudaMemset(c->d_status, 0, sizeof(unsigned));
  cudaMemset(c->d_loop, 0, sizeof(CgLoopState));
  cudaMemset(c->d_dstats, 0, sizeof(DevStats));
  cudaMemset(c->d_refine, 0, 4 * sizeof(int));
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(PDEP_ERR_CUDA, "capture stream creation"));
  if (c->opt.clock_budget_cycles > 0) {
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device) != cudaSuccess || khz <= 0)
      khz = 2070000;
    // cycles at the rated SM clock -> ns of %globaltimer
    c->budget_ns = (unsigned long long)((double)c->opt.clock_budget_cycles * 1e6 / khz);
    if (c->budget_ns == 0) c->budget_ns = 1;
  }
  if (cudaEventCreate(&c->ev[0]) != cudaSuccess || cudaEventCreate(&c->ev[1]) != cudaSuccess)
    return bail(fail(PDEP_ERR_CUDA, "event creation"));
  c->sys.resize(n_sys);
  for (int i = 0; i < n_sys; ++i) {
    const pdep_system_desc& d = sys[i];
    SysData& s = c->sys[i];
    for (int a = 0; a < 3; ++a) {
      s.N[a] = d.grid[a];
      s.L[a] = d.cell[a];
    }
    s.n_occ = d.n_occ;
    s.n_pdep = d.n_pdep;
    if (!d.v_r || d.n_occ < 1 || d.n_pdep < 1)
      return bail(fail(PDEP_ERR_INVALID_ARG, "bad system descriptor"));
    if (!grid_supported(s.N[0], s.N[1], s.N[2]))
      return bail(fail(PDEP_ERR_INVALID_ARG, "unsupported grid shape"));
    int r = build_sphere(s, d.ecut);
    if (r != PDEP_OK) return bail(r);
    if (s.n_pdep > s.n_pw - 1) return bail(fail(PDEP_ERR_INVALID_ARG, "n_pdep too large"));
    const size_t smem = slab_smem_bytes(s.n_col, s.R3, s.N[1], sizeof(double));
    if (smem > 200 * 1024) return bail(fail(PDEP_ERR_UNSUPPORTED, "slab does not fit shared memory"));
    r = upload_tables(c, s);
    if (r != PDEP_OK) return bail(r);
    if ((r = persistent(c, &s.d_v, s.n_r)) != PDEP_OK) return bail(r);
    if ((r = persistent(c, &s.d_vf, s.n_r)) != PDEP_OK) return bail(r);
    if ((r = persistent(c, &s.d_vdf, s.n_r)) != PDEP_OK) return bail(r);
    if (cudaMemcpyAsync(s.d_v, d.v_r, sizeof(double) * s.n_r, kind_to_dev(d.v_r), st) != cudaSuccess)
      return bail(fail(PDEP_ERR_CUDA, "potential upload"));
    if (convert<float, double>(s.d_vf, s.n_r, s.d_v, s.n_r, s.n_r, 1, st) != cudaSuccess ||
        convert<df, double>(s.d_vdf, s.n_r, s.d_v, s.n_r, s.n_r, 1, st) != cudaSuccess)
      return bail(fail(PDEP_ERR_CUDA, "potential conversion"));
    // the potential must be finite
    std::vector<double> hv(s.n_r);
    if (cudaMemcpyAsync(hv.data(), s.d_v, sizeof(double) * s.n_r, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return bail(fail(PDEP_ERR_CUDA, "potential check"));
    s.vmax = -1e300;
    for (double v : hv) {
      if (!std::isfinite(v)) return bail(fail(PDEP_ERR_NONFINITE, "non-finite potential"));
      s.vmax = std::max(s.vmax, v);
    }
    r = setup_states(c, s, st);
    if (r != PDEP_OK) return bail(r);
    if ((r = check_status(c, st)) != PDEP_OK) return bail(r);
  }
  *out = c;
  return PDEP_OK;
}

int pdep_get_sizes(const pdep_ctx* c, int sys, int* n_pw, int* n_r, int* n_pdep_dim) {
  RET(check_sys(c, sys));
  const SysData& s = c->sys[sys];
  if (n_pw) *n_pw = s.n_pw;
  if (n_r) *n_r = s.n_r;
  if (n_pdep_dim) *n_pdep_dim = s.n_pw - 1;
  return PDEP_OK;
}

int pdep_get_occupied(pdep_ctx* c, int sys, double* psi, double* eps, void* stream) {
  RET(check_sys(c, sys));
  cudaStream_t st = (cudaStream_t)stream;
  SysData& s = c->sys[sys];
  if (psi)
    CK(cudaMemcpy2DAsync(psi, s.n_pw * sizeof(double), s.d_psi, s.ld * sizeof(double),
                         s.n_pw * sizeof(double), s.n_occ, kind_from_dev(psi), st));
  RET(sync(st));
  if (eps) RET(copy_from_host(eps, s.eps.data(), sizeof(double) * (s.n_occ + 1), st));
  return PDEP_OK;
}

int chi0_apply(pdep_ctx* c, int sys, const double* phi, int n_pert, double* chi0_phi, double* dn_r,
               void* stream) {
  RET(check_sys(c, sys));
  if (n_pert < 0 || (n_pert > 0 && (!phi || !chi0_phi)))
    return fail(PDEP_ERR_INVALID_ARG, "bad chi0_apply arguments");
  if (n_pert == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SysData& s = c->sys[sys];
  RET(reset_stats(c, st));
  const int dim = s.n_pw - 1;
  double *in, *outv, *dn = nullptr;
  RET(ws(c, "api_in", (size_t)n_pert * s.ld, &in));
  RET(ws(c, "api_out", (size_t)n_pert * s.ld, &outv));
  const bool host_io = !is_device_ptr(phi) || !is_device_ptr(chi0_phi) ||
                       (dn_r && !is_device_ptr(dn_r));
  CK(cudaMemsetAsync(in, 0, sizeof(double) * (size_t)n_pert * s.ld, st));
  CK(cudaMemcpy2DAsync(in, s.ld * sizeof(double), phi, dim * sizeof(double), dim * sizeof(double),
                       n_pert, kind_to_dev(phi), st));
  const bool dn_dev = dn_r && is_device_ptr(dn_r);
  if (dn_r) {
    if (dn_dev)
      dn = dn_r;
    else
      RET(ws(c, "api_dn", (size_t)n_pert * s.n_r, &dn));
  }
  RET(chi0_internal(c, s, in, n_pert, outv, dn, st));
  CK(cudaMemcpy2DAsync(chi0_phi, dim * sizeof(double), outv, s.ld * sizeof(double),
                       dim * sizeof(double), n_pert, kind_from_dev(chi0_phi), st));
  if (dn_r && !dn_dev)
    CK(cudaMemcpyAsync(dn_r, dn, sizeof(double) * (size_t)n_pert * s.n_r, cudaMemcpyDeviceToHost,
                       st));
  // device buffers only: enqueued, nothing waited for; conditions stay in the
  // status word until a synchronising call reads them
  if (!host_io) return PDEP_OK;
  return check_status(c, st);
}

// Screening operators at omega = 0 in the PDEP basis (Eqs. linearalgebrachichi0,
// epsilonandchi, Wpnondiag): Phi diag(lambda/(1-lambda)) Phi^T, plus the identity
// (epsbar^{-1}) or between v^{1/2} factors (W^p).
int pdep_screening_apply(pdep_ctx* c, int sys, int kind, const double* eigvals,
                         const double* eigvecs, int n_pdep, const double* f, int n, double* out,
                         void* stream) {
  RET(check_sys(c, sys));
  SysData& s = c->sys[sys];
  const int dim = s.n_pw - 1;
  if (kind < PDEP_SCREEN_CHIBAR || kind > PDEP_SCREEN_WP || n_pdep < 1 || n_pdep > dim ||
      n < 0 || !eigvals || !eigvecs || (n > 0 && (!f || !out)))
    return fail(PDEP_ERR_INVALID_ARG, "bad pdep_screening_apply arguments");
  if (n == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> lam(n_pdep), g(n_pdep);
  if (is_device_ptr(eigvals)) {
    CK(cudaMemcpyAsync(lam.data(), eigvals, sizeof(double) * n_pdep, cudaMemcpyDeviceToHost, st));
    RET(sync(st));
  } else {
    memcpy(lam.data(), eigvals, sizeof(double) * n_pdep);
  }
  for (int i = 0; i < n_pdep; ++i) {
    // chi0bar is negative semi-definite; 1 - lambda must stay away from 0
    if (!std::isfinite(lam[i]) || !(1.0 - lam[i] > 1e-12))
      return fail(PDEP_ERR_INVALID_ARG, "eigenvalue with lambda >= 1 or non-finite");
    g[i] = lam[i] / (1.0 - lam[i]);
  }
  double *phi, *fx, *S, *dg, *o;
  RET(ws(c, "sc_phi", (size_t)n_pdep * s.ld, &phi));
  RET(ws(c, "sc_f", (size_t)n * s.ld, &fx));
  RET(ws(c, "sc_o", (size_t)n * s.ld, &o));
  RET(ws(c, "sc_s", (size_t)n_pdep * n, &S));
  RET(ws(c, "sc_g", (size_t)n_pdep, &dg));
  CK(cudaMemcpyAsync(dg, g.data(), sizeof(double) * n_pdep, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpy2DAsync(phi, s.ld * sizeof(double), eigvecs, dim * sizeof(double),
                       dim * sizeof(double), n_pdep, kind_to_dev(eigvecs), st));
  CK(cudaMemcpy2DAsync(fx, s.ld * sizeof(double), f, dim * sizeof(double), dim * sizeof(double), n,
                       kind_to_dev(f), st));
  if (kind == PDEP_SCREEN_WP) CK(scale_sqrt_coulomb(fx, s.ld, s.n_half, n, s.sd.g2, st));
  // S = Phi^T f, scaled per row by lambda/(1-lambda); out = Phi S (+ f)
  CK(gemm<double>(true, n_pdep, n, dim, 1.0, phi, s.ld, fx, s.ld, 0.0, S, n_pdep, st));
  CK(scale_rows<double>(S, n_pdep, n_pdep, n, dg, st));
  double beta = 0.0;
  if (kind == PDEP_SCREEN_EPSINV) {
    CK(cudaMemcpyAsync(o, fx, sizeof(double) * (size_t)n * s.ld, cudaMemcpyDeviceToDevice, st));
    beta = 1.0;
  }
  CK(gemm<double>(false, dim, n, n_pdep, 1.0, phi, s.ld, S, n_pdep, beta, o, s.ld, st));
  if (kind == PDEP_SCREEN_WP) CK(scale_sqrt_coulomb(o, s.ld, s.n_half, n, s.sd.g2, st));
  CK(cudaMemcpy2DAsync(out, dim * sizeof(double), o, s.ld * sizeof(double), dim * sizeof(double),
                       n, kind_from_dev(out), st));
  RET(sync(st));
  return PDEP_OK;
}

// Body of chi0bar at imaginary frequencies in the PDEP basis (Eq. finalB,
// Sec. II B) from Lanczos chains (Sec. II D, Eq. MCfinal), and the RPA body
// Lambda = (1 - B)^{-1} B (Eq. Bfinal without head and wings).
int pdep_chi0_imag(pdep_ctx* c, int sys, const double* phi, int n_pdep, const double* nu,
                   int n_freq, int n_steps, double* B, double* Lambda, void* stream) {
  NvtxRange nv("chi0_imag");
  RET(check_sys(c, sys));
  SysData& s = c->sys[sys];
  const int dim = s.n_pw - 1;
  if (n_pdep < 1 || n_pdep > dim || n_freq < 0 || n_steps < 1 || n_steps > 64 ||
      (n_freq > 0 && (!phi || !nu || !B)))
    return fail(PDEP_ERR_INVALID_ARG, "bad pdep_chi0_imag arguments");
  if (n_freq == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int K = n_steps, nocc = s.n_occ, np = n_pdep;
  std::vector<double> hnu(n_freq);
  if (is_device_ptr(nu)) {
    CK(cudaMemcpyAsync(hnu.data(), nu, sizeof(double) * n_freq, cudaMemcpyDeviceToHost, st));
    RET(sync(st));
  } else {
    memcpy(hnu.data(), nu, sizeof(double) * n_freq);
  }
  for (double x : hnu)
    if (!std::isfinite(x)) return fail(PDEP_ERR_INVALID_ARG, "non-finite frequency");
  double *dphi, *dv, *R, *dnu, *Bd;
  RET(ws(c, "fq_phi", (size_t)np * s.ld, &dphi));
  RET(ws(c, "fq_dv", (size_t)np * s.n_r, &dv));
  RET(ws(c, "fq_R", (size_t)np * nocc * s.ld, &R));
  RET(ws(c, "fq_nu", (size_t)n_freq, &dnu));
  RET(ws(c, "fq_B", (size_t)n_freq * np * np, &Bd));
  CK(cudaMemcpyAsync(dnu, hnu.data(), sizeof(double) * n_freq, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(dphi, 0, sizeof(double) * (size_t)np * s.ld, st));
  CK(cudaMemcpy2DAsync(dphi, s.ld * sizeof(double), phi, dim * sizeof(double),
                       dim * sizeof(double), np, kind_to_dev(phi), st));
  CK(cudaMemsetAsync(Bd, 0, sizeof(double) * (size_t)n_freq * np * np, st));
  // R_{j v} = -P_c [dV_j psi_v] (row j n_occ + v): the chains' start vectors
  // and, for fixed v, the left vectors L_i of Eq. finalB
  RET(perturbation_grids(c, s, dphi, np, dv, st));
  RET(build_rhs(c, s, dv, np, R, nullptr, st, true));
  // chains of a group of occupied states at a time
  const size_t per_state = (size_t)np * ((size_t)K + 2) * s.ld * sizeof(double);
  size_t budget = (size_t)16 << 30;
  if (c->opt.workspace_limit_bytes) budget = c->opt.workspace_limit_bytes / 2;
  const int nv_max = (int)std::max<size_t>(1, std::min<size_t>(budget / per_state, nocc));
  std::vector<int> hidx, hmap((size_t)K * np);
  for (int v0 = 0; v0 < nocc; v0 += nv_max) {
    const int nvg = std::min(nv_max, nocc - v0);
    const int ng = np * nvg;
    double *Q, *W, *da, *db, *dd, *dU, *r0, *G, *z;
    int *idx, *bmap;
    RET(ws(c, "fq_Q", (size_t)K * ng * s.ld, &Q));
    RET(ws(c, "fq_W", (size_t)ng * s.ld, &W));
    RET(ws(c, "fq_a", (size_t)ng * K, &da));
    RET(ws(c, "fq_b", (size_t)ng * K, &db));
    RET(ws(c, "fq_d", (size_t)ng * K, &dd));
    RET(ws(c, "fq_U", (size_t)ng * K * K, &dU));
    RET(ws(c, "fq_r0", (size_t)ng, &r0));
    RET(ws(c, "fq_G", (size_t)np * K * np, &G));
    RET(ws(c, "fq_z", (size_t)n_freq * np * K, &z));
    RET(ws(c, "fq_idx", (size_t)ng, &idx));
    RET(ws(c, "fq_map", (size_t)K * np, &bmap));
    // chain (j, v) of the group sits at j nvg + (v - v0)
    hidx.resize(ng);
    for (int j = 0; j < np; ++j)
      for (int v = v0; v < v0 + nvg; ++v) hidx[(size_t)j * nvg + (v - v0)] = j * nocc + v;
    CK(cudaMemcpyAsync(idx, hidx.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)ng * s.ld, st));
    CK(gather_cols(R, s.ld, W, s.ld, s.n_pw, idx, ng, st));
    CK(col_norms<double>(W, s.ld, s.n_pw, ng, r0, st));
    RET(lanczos_core(c, s, W, r0, ng, K, Q, da, db, dd, dU, st));
    for (int v = v0; v < v0 + nvg; ++v) {
      // G[i][k np + j] = <R_{i v} | q_k of chain (j, v)>
      for (int k = 0; k < K; ++k)
        for (int j = 0; j < np; ++j) hmap[(size_t)k * np + j] = k * ng + j * nvg + (v - v0);
      CK(cudaMemcpyAsync(bmap, hmap.data(), sizeof(int) * K * np, cudaMemcpyHostToDevice, st));
      CK(gemm<double>(true, np, K * np, s.n_pw, 1.0, R + (size_t)v * s.ld, (long long)nocc * s.ld,
                      Q, s.ld, 0.0, G, np, st, bmap, nullptr));
      CK(lanczos_z(dU, dd, db, np, K, nvg, v - v0, s.eps[v], dnu, n_freq, z, st));
      // B_ij += 2 (spin) x 2 (the two frequencies eps_v -+ i nu, equal in
      // their real parts) x the chain sum
      CK(body_accum(G, np, np, K, z, n_freq, 4.0, Bd, st));
      RET(sync(st));  // hmap is reused for the next v
    }
  }
  for (int f = 0; f < n_freq; ++f) CK(symmetrize<double>(Bd + (size_t)f * np * np, np, np, st));
  CK(cudaMemcpyAsync(B, Bd, sizeof(double) * (size_t)n_freq * np * np, kind_from_dev(B), st));
  if (Lambda) {
    double *w, *V, *Ld;
    RET(ws(c, "fq_w", (size_t)np, &w));
    RET(ws(c, "fq_V", (size_t)np * np, &V));
    RET(ws(c, "fq_L", (size_t)n_freq * np * np, &Ld));
    EighWork wk;
    RET(eigh_ws(c, np, &wk));
    std::vector<double> hw(np);
    for (int f = 0; f < n_freq; ++f) {
      CK(eigh(np, Bd + (size_t)f * np * np, np, w, V, np, wk, st));
      CK(cudaMemcpyAsync(hw.data(), w, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
      RET(sync(st));
      for (double x : hw)
        if (!(1.0 - x > 1e-12)) return fail(PDEP_ERR_NONFINITE, "B(i nu) has an eigenvalue >= 1");
      CK(lambda_from_eig(V, w, np, Ld + (size_t)f * np * np, st));
    }
    CK(cudaMemcpyAsync(Lambda, Ld, sizeof(double) * (size_t)n_freq * np * np,
                       kind_from_dev(Lambda), st));
  }
  RET(sync(st));
  return PDEP_OK;
}

// Batched Lanczos chains of the deflated Hamiltonian P_c H P_c (Sec. II D):
// poles and omega-independent weights of M_c,LR(omega) (Eq. MCfinal).
int pdep_lanczos(pdep_ctx* c, int sys, const double* R, int n, int n_steps, const double* L,
                 int n_L, double* poles, double* weights, double* alpha, double* beta,
                 void* stream) {
  NvtxRange nv("lanczos");
  RET(check_sys(c, sys));
  if (n < 0 || n_steps < 1 || n_steps > 64 || n_L < 0 ||
      (n > 0 && (!R || !poles || (n_L > 0 && (!L || !weights)))))
    return fail(PDEP_ERR_INVALID_ARG, "bad pdep_lanczos arguments");
  if (n == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SysData& s = c->sys[sys];
  const int K = n_steps;
  double* dL = nullptr;
  if (n_L > 0) {
    RET(ws(c, "lz_L", (size_t)n_L * s.ld, &dL));
    CK(cudaMemsetAsync(dL, 0, sizeof(double) * (size_t)n_L * s.ld, st));
    CK(cudaMemcpy2DAsync(dL, s.ld * sizeof(double), L, s.n_pw * sizeof(double),
                         s.n_pw * sizeof(double), n_L, kind_to_dev(L), st));
  }
  // chains in chunks: Q holds K blocks of nc vectors (step-major)
  const size_t per_chain = (size_t)(K + 3) * s.ld * sizeof(double);
  size_t budget = (size_t)16 << 30;
  if (c->opt.workspace_limit_bytes) budget = c->opt.workspace_limit_bytes / 2;
  const int nc_max = (int)std::max<size_t>(1, std::min<size_t>(budget / per_chain, 65535));
  for (int j0 = 0; j0 < n; j0 += nc_max) {
    const int nc = std::min(nc_max, n - j0);
    double *Q, *W, *da, *db, *dd, *dU, *r0, *G = nullptr, *dw = nullptr;
    RET(ws(c, "lz_Q", (size_t)K * nc * s.ld, &Q));
    RET(ws(c, "lz_W", (size_t)nc * s.ld, &W));
    RET(ws(c, "lz_a", (size_t)nc * K, &da));
    RET(ws(c, "lz_b", (size_t)nc * K, &db));
    RET(ws(c, "lz_d", (size_t)nc * K, &dd));
    RET(ws(c, "lz_U", (size_t)nc * K * K, &dU));
    RET(ws(c, "lz_r0", (size_t)nc, &r0));
    CK(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)nc * s.ld, st));
    CK(cudaMemcpy2DAsync(W, s.ld * sizeof(double), R + (size_t)j0 * s.n_pw,
                         s.n_pw * sizeof(double), s.n_pw * sizeof(double), nc, kind_to_dev(R),
                         st));
    // P_c R (norms kept for the empty-chain test), then the chains
    CK(col_norms<double>(W, s.ld, s.n_pw, nc, r0, st));
    RET(project_occupied(c, s, W, nc, st));
    RET(lanczos_core(c, s, W, r0, nc, K, Q, da, db, dd, dU, st));
    if (n_L > 0) {
      RET(ws(c, "lz_G", (size_t)n_L * K * nc, &G));
      RET(ws(c, "lz_w", (size_t)nc * n_L * K, &dw));
      // G[l][k nc + j] = <L_l | q_k of chain j>
      CK(gemm<double>(true, n_L, K * nc, s.n_pw, 1.0, dL, s.ld, Q, s.ld, 0.0, G, n_L, st));
      CK(lanczos_weights(G, n_L, nc, K, dU, db, dw, 1, 0, st));
      CK(cudaMemcpyAsync(weights + (size_t)j0 * n_L * K, dw, sizeof(double) * (size_t)nc * n_L * K,
                         kind_from_dev(weights), st));
    }
    CK(cudaMemcpyAsync(poles + (size_t)j0 * K, dd, sizeof(double) * (size_t)nc * K,
                       kind_from_dev(poles), st));
    if (alpha)
      CK(cudaMemcpyAsync(alpha + (size_t)j0 * K, da, sizeof(double) * (size_t)nc * K,
                         kind_from_dev(alpha), st));
    if (beta)
      CK(cudaMemcpyAsync(beta + (size_t)j0 * K, db, sizeof(double) * (size_t)nc * K,
                         kind_from_dev(beta), st));
    RET(sync(st));
  }
  return PDEP_OK;
}

// chibar phi with the Hartree-only self-consistent perturbation (Sec. II C,
// Eqs. LF and LFHartree): dV_tot = v^{1/2} phi + v dn[dV_tot].  With
// dV_tot = v^{1/2} y this is (1 - chi0bar) y = phi, an SPD system solved by
// CG whose every operator application is a chi0bar application (a batch of
// Sternheimer solves); then chibar phi = v^{1/2} dn[dV_tot] = y - phi, the
// (1 - chi0bar)^{-1} chi0bar phi of Eq. linearalgebrachichi0.
int pdep_chibar_apply(pdep_ctx* c, int sys, const double* phi, int n, double* out, double tol,
                      int max_iter, int* iterations, void* stream) {
  NvtxRange nv("chibar_apply");
  RET(check_sys(c, sys));
  if (n < 0 || max_iter < 1 || !(tol > 0) || (n > 0 && (!phi || !out)))
    return fail(PDEP_ERR_INVALID_ARG, "bad pdep_chibar_apply arguments");
  if (iterations) *iterations = 0;
  if (n == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SysData& s = c->sys[sys];
  RET(reset_stats(c, st));
  const int dim = s.n_pw - 1;
  double *y, *r, *p, *q, *d_al, *d_be, *dots;
  RET(ws(c, "hx_y", (size_t)n * s.ld, &y));
  RET(ws(c, "hx_r", (size_t)n * s.ld, &r));
  RET(ws(c, "hx_p", (size_t)n * s.ld, &p));
  RET(ws(c, "hx_q", (size_t)n * s.ld, &q));
  RET(ws(c, "hx_al", (size_t)n, &d_al));
  RET(ws(c, "hx_be", (size_t)n, &d_be));
  RET(ws(c, "hx_dots", (size_t)n, &dots));
  // y = 0, r = p = phi
  CK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n * s.ld, st));
  CK(cudaMemsetAsync(r, 0, sizeof(double) * (size_t)n * s.ld, st));
  CK(cudaMemcpy2DAsync(r, s.ld * sizeof(double), phi, dim * sizeof(double), dim * sizeof(double),
                       n, kind_to_dev(phi), st));
  CK(cudaMemcpyAsync(p, r, sizeof(double) * (size_t)n * s.ld, cudaMemcpyDeviceToDevice, st));
  std::vector<double> rr(n), r0(n), al(n), be(n), pq(n);
  CK(pair_dots(r, r, s.ld, s.n_pw, n, dots, st));
  CK(cudaMemcpyAsync(rr.data(), dots, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  RET(sync(st));
  std::vector<char> active(n);
  int n_act = 0;
  for (int j = 0; j < n; ++j) {
    r0[j] = std::sqrt(rr[j]);
    active[j] = rr[j] > 0.0;
    n_act += active[j];
  }
  int it = 0;
  for (; it < max_iter && n_act > 0; ++it) {
    // q = (1 - chi0bar) p
    int rc = chi0_internal(c, s, p, n, q, nullptr, st);
    if (rc != PDEP_OK && rc != PDEP_ERR_NOT_CONVERGED) return rc;
    CK(one_minus(q, p, s.ld, s.n_pw, n, st));
    CK(pair_dots(p, q, s.ld, s.n_pw, n, dots, st));
    CK(cudaMemcpyAsync(pq.data(), dots, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    RET(sync(st));
    for (int j = 0; j < n; ++j) {
      if (active[j] && !(pq[j] > 0.0)) return fail(PDEP_ERR_NONFINITE, "1 - chi0bar not positive");
      al[j] = active[j] ? rr[j] / pq[j] : 0.0;
    }
    CK(cudaMemcpyAsync(d_al, al.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CK(block_cg_xr(y, r, p, q, s.ld, s.n_pw, n, d_al, st));
    CK(pair_dots(r, r, s.ld, s.n_pw, n, dots, st));
    std::vector<double> rn(n);
    CK(cudaMemcpyAsync(rn.data(), dots, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    RET(sync(st));
    n_act = 0;
    for (int j = 0; j < n; ++j) {
      if (!active[j]) {
        be[j] = 0.0;
        continue;
      }
      if (!std::isfinite(rn[j])) return fail(PDEP_ERR_NONFINITE, "non-finite residual");
      be[j] = rn[j] / rr[j];
      rr[j] = rn[j];
      if (std::sqrt(rn[j]) <= tol * r0[j]) {
        active[j] = 0;
        be[j] = 0.0;
      }
      n_act += active[j];
    }
    CK(cudaMemcpyAsync(d_be, be.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CK(block_cg_p(p, r, s.ld, s.n_pw, n, d_be, st));
  }
  if (iterations) *iterations = it;
  // chibar phi = y - phi: r = phi again, then out = y - r
  CK(cudaMemsetAsync(r, 0, sizeof(double) * (size_t)n * s.ld, st));
  CK(cudaMemcpy2DAsync(r, s.ld * sizeof(double), phi, dim * sizeof(double), dim * sizeof(double),
                       n, kind_to_dev(phi), st));
  CK(one_minus(r, y, s.ld, s.n_pw, n, st));
  CK(cudaMemcpy2DAsync(out, dim * sizeof(double), r, s.ld * sizeof(double), dim * sizeof(double),
                       n, kind_from_dev(out), st));
  const int dev = check_status(c, st);
  if (dev != PDEP_OK) return dev;
  if (n_act > 0) return fail(PDEP_ERR_NOT_CONVERGED, "self-consistent response: CG cap reached");
  return PDEP_OK;
}

int sternheimer_solve(pdep_ctx* c, int sys, const double* dv_r, int n_pert, double* dpsi,
                      int* iters, double* resid, void* stream) {
  RET(check_sys(c, sys));
  if (n_pert < 0 || (n_pert > 0 && (!dv_r || !dpsi)))
    return fail(PDEP_ERR_INVALID_ARG, "bad sternheimer_solve arguments");
  if (n_pert == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SysData& s = c->sys[sys];
  RET(reset_stats(c, st));
  const int n = n_pert * s.n_occ;
  const bool host_io = !is_device_ptr(dv_r) || !is_device_ptr(dpsi) ||
                       (iters && !is_device_ptr(iters)) || (resid && !is_device_ptr(resid));
  double *dv, *bvec, *xvec, *rel = nullptr;
  int* its;
  RET(ws(c, "st_dv", (size_t)n_pert * s.n_r, &dv));
  RET(ws(c, "st_b", (size_t)n * s.ld, &bvec));
  RET(ws(c, "st_x", (size_t)n * s.ld, &xvec));
  RET(ws(c, "st_its", (size_t)n, &its));
  CK(cudaMemcpyAsync(dv, dv_r, sizeof(double) * (size_t)n_pert * s.n_r, kind_to_dev(dv_r), st));
  double* xd = nullptr;
  if (s.n_defl > 0) RET(ws(c, "st_xd", (size_t)n * s.ld, &xd));
  RET(build_rhs(c, s, dv, n_pert, bvec, xd, st));
  RET(solve_rhs(c, s, bvec, xd, xvec, n, nullptr, its, &rel, st));
  CK(cudaMemcpy2DAsync(dpsi, s.n_pw * sizeof(double), xvec, s.ld * sizeof(double),
                       s.n_pw * sizeof(double), n, kind_from_dev(dpsi), st));
  if (iters) CK(cudaMemcpyAsync(iters, its, sizeof(int) * n, kind_from_dev(iters), st));
  if (resid) CK(cudaMemcpyAsync(resid, rel, sizeof(double) * n, kind_from_dev(resid), st));
  if (!host_io) return PDEP_OK;
  return check_status(c, st);
}

int pdep_apply_hamiltonian(pdep_ctx* c, int sys, const double* x, int n, double* y,
                           int precision, void* stream) {
  RET(check_sys(c, sys));
  if (n < 0 || (n > 0 && (!x || !y))) return fail(PDEP_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SysData& s = c->sys[sys];
  double *in, *outv;
  RET(ws(c, "api_in", (size_t)n * s.ld, &in));
  RET(ws(c, "api_out", (size_t)n * s.ld, &outv));
  CK(cudaMemsetAsync(in, 0, sizeof(double) * (size_t)n * s.ld, st));
  CK(cudaMemcpy2DAsync(in, s.ld * sizeof(double), x, s.n_pw * sizeof(double),
                       s.n_pw * sizeof(double), n, kind_to_dev(x), st));
  if (precision == PDEP_FP64) {
    RET(apply_h<double>(c, s, in, outv, n, nullptr, 0, false, false, st));
  } else if (precision == PDEP_APPLY_DF64) {
    RET(apply_h<df>(c, s, in, outv, n, nullptr, 0, false, false, st));
  } else {
    float *in32, *out32;
    RET(ws(c, "api_in32", (size_t)n * s.ld, &in32));
    RET(ws(c, "api_out32", (size_t)n * s.ld, &out32));
    CK((convert<float, double>(in32, s.ld, in, s.ld, s.ld, n, st)));
    RET(apply_h<float>(c, s, in32, out32, n, nullptr, 0, false, false, st));
    CK((convert<double, float>(outv, s.ld, out32, s.ld, s.n_pw, n, st)));
  }
  CK(cudaMemcpy2DAsync(y, s.n_pw * sizeof(double), outv, s.ld * sizeof(double),
                       s.n_pw * sizeof(double), n, kind_from_dev(y), st));
  return sync(st);
}

int pdep_to_grid(pdep_ctx* c, int sys, const double* x, int n, double* u, void* stream) {
  RET(check_sys(c, sys));
  if (n < 0 || (n > 0 && (!x || !u))) return fail(PDEP_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return PDEP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SysData& s = c->sys[sys];
  double *in, *grid;
  RET(ws(c, "api_in", (size_t)n * s.ld, &in));
  RET(ws(c, "api_grid", (size_t)n * s.n_r, &grid));
  CK(cudaMemsetAsync(in, 0, sizeof(double) * (size_t)n * s.ld, st));
  CK(cudaMemcpy2DAsync(in, s.ld * sizeof(double), x, s.n_pw * sizeof(double),
                       s.n_pw * sizeof(double), n, kind_to_dev(x), st));
  ItemMap map{n, (n + 1) / 2};
  const int n_items = (n + 1) / 2;
  cpx<double>* b1;
  RET(ws(c, "b1_64", b1_count(s, n_items), &b1));
  CK(launch_cols_fwd<double>(s.sd, in, s.ld, map, n_items, COEF_ONE, b1, st));
  SlabArgs<double> a{};
  a.mode = SLAB_TO_GRID;
  a.b1 = b1;
  a.n_items = n_items;
  a.out = grid;
  a.out_stride = s.n_r;
  a.out_scale = 1.0;
  a.map = map;
  CK(launch_slab<double>(s.sd, a, st));
  CK(cudaMemcpyAsync(u, grid, sizeof(double) * (size_t)n * s.n_r, kind_from_dev(u), st));
  return sync(st);
}

int pdep_solve(pdep_ctx* c, int sys, const double* phi0, double* eigvals, double* eigvecs,
               pdep_stats* stats, void* stream) {
  if (!c) return fail(PDEP_ERR_INVALID_ARG, "null context");
  if (!eigvals) return fail(PDEP_ERR_INVALID_ARG, "null eigvals");
  if (sys != -1) RET(check_sys(c, sys));
  cudaStream_t st = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  RET(reset_stats(c, st));
  pdep_stats local{};
  if (!stats) stats = &local;
  memset(stats, 0, sizeof(*stats));
  stats->converged = 1;
  int result = PDEP_OK;
  const int lo = sys == -1 ? 0 : sys, hi = sys == -1 ? (int)c->sys.size() : sys + 1;
  size_t off_val = 0, off_vec = 0;
  for (int i = lo; i < hi; ++i) {
    SysData& s = c->sys[i];
    const double* p0 = phi0 ? phi0 + off_vec : nullptr;
    int r = solve_one(c, i, p0, eigvals + off_val, eigvecs ? eigvecs + off_vec : nullptr, stats, st);
    if (r != PDEP_OK && r != PDEP_ERR_NOT_CONVERGED) return r;
    if (r != PDEP_OK) result = r;
    off_val += s.n_pdep;
    off_vec += (size_t)s.n_pdep * (s.n_pw - 1);
  }
  RET(read_stats(c, stats, st));
  stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->last_dav = *stats;
  const int dev = check_status(c, st);
  if (dev != PDEP_OK && dev != PDEP_ERR_NOT_CONVERGED) return dev;
  if (dev == PDEP_ERR_NOT_CONVERGED) result = dev;
  return result;
}

int pdep_get_stats(pdep_ctx* c, pdep_stats* stats, void* stream) {
  if (!c || !stats) return fail(PDEP_ERR_INVALID_ARG, "null context or stats");
  cudaStream_t st = (cudaStream_t)stream;
  memset(stats, 0, sizeof(*stats));
  stats->dav_iterations = c->last_dav.dav_iterations;
  stats->converged = c->last_dav.converged;
  stats->max_dav_residual = c->last_dav.max_dav_residual;
  RET(read_stats(c, stats, st));
  return check_status(c, st);
}

}  // extern "C"
