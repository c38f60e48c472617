// Kernel profiler of the library (see profile.cuh and pdep_profile in pdep.h).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

#include "profile.cuh"

namespace pdep {

namespace {
struct Rec {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes;
  bool closed;  // the end event has been recorded
  int* slot;    // device copy of the launch's unit count (or null)
  int units;
};
struct Acc {
  long long launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};
const char* kNames[PDEP_PROFILE_CLASSES] = {"cols_f64", "cols_f32",    "slab_f64",    "slab_f32",
                                            "gemm_f64", "gemm_f32",    "cg_f64",      "cg_f32",
                                            "eigh",     "other",       "gemm_tf32x3", "cg_graph_f32",
                                            "cg_graph_f64", "cols_df64", "slab_df64",
                                            "hpsi_fused_f32", "gemm_df64"};
thread_local bool t_capturing = false;
thread_local int t_capture_launches = 0;
std::atomic<long long> g_launches{0};
// Shared by every host thread that launches library kernels (the lanes of a
// chi0bar application): the record list and the event pool are guarded by mu;
// list nodes keep their addresses, so a scope can close its record later.
struct Profiler {
  std::atomic<bool> on{false};
  std::atomic<long long> launches{0};
  std::mutex mu;
  std::list<Rec> pending;
  std::vector<cudaEvent_t> pool;
  Acc acc[PDEP_PROFILE_CLASSES];
  std::vector<int*> slots;  // free device ints for unit counts (chunks of 4096)
  std::vector<int*> chunks;
  int* slot() {
    if (slots.empty()) {
      int* p = nullptr;
      if (cudaMalloc(&p, 4096 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      chunks.push_back(p);
      for (int i = 0; i < 4096; ++i) slots.push_back(p + i);
    }
    int* p = slots.back();
    slots.pop_back();
    return p;
  }
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // folds the closed records into acc (caller holds mu)
  void resolve() {
    for (auto it = pending.begin(); it != pending.end();) {
      if (!it->closed) {
        ++it;
        continue;
      }
      Rec& r = *it;
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        double f = 1.0;
        if (r.slot) {
          int n = 0;
          if (cudaMemcpy(&n, r.slot, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && r.units > 0)
            f = std::min(1.0, std::max(0.0, (double)n / r.units));
          else
            cudaGetLastError();
          slots.push_back(r.slot);
        }
        Acc& a = acc[r.cls];
        a.launches += 1;
        a.ms += ms;
        a.flops += f * r.flops;
        a.bytes += f * r.bytes;
      } else {
        cudaGetLastError();
        if (r.slot) slots.push_back(r.slot);
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
      it = pending.erase(it);
    }
  }
};
Profiler& prof() {
  static Profiler p;
  return p;
}
}  // namespace

void count_launch() {
  if (t_capturing) {
    ++t_capture_launches;
    return;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  Profiler& p = prof();
  if (p.on) p.launches.fetch_add(1, std::memory_order_relaxed);
}

void capture_begin() {
  t_capturing = true;
  t_capture_launches = 0;
}

int capture_end() {
  t_capturing = false;
  return t_capture_launches;
}

long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {
DevTimer* g_timers = nullptr;  // [PDEP_PROFILE_CLASSES], device memory
std::mutex g_timer_mu;
void reset_timers() {
  if (!g_timers) return;
  std::vector<DevTimer> h(PDEP_PROFILE_CLASSES);
  for (DevTimer& t : h) {
    memset(&t, 0, sizeof(t));
    t.t_min = ~0ull;
  }
  cudaMemcpy(g_timers, h.data(), sizeof(DevTimer) * h.size(), cudaMemcpyHostToDevice);
}
}  // namespace

int dev_timers_init() {
  std::lock_guard<std::mutex> g(g_timer_mu);
  if (g_timers) return 0;
  if (cudaMalloc(&g_timers, sizeof(DevTimer) * PDEP_PROFILE_CLASSES) != cudaSuccess) {
    cudaGetLastError();
    g_timers = nullptr;
    return 1;
  }
  reset_timers();
  return 0;
}

DevTimer* dev_timer(int cls) { return g_timers ? g_timers + cls : nullptr; }

// records nothing while the stream is being captured (events cannot time a
// kernel inside a graph, and resolving records waits on events, which a
// capture forbids)
ProfScope::ProfScope(int c, cudaStream_t s, double f, double b, const int* dcount, int units)
    : cls(c), st(s), flops(f), bytes(b), rec(nullptr) {
  Profiler& p = prof();
  if (!p.on || t_capturing) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> g(p.mu);
  if (p.pending.size() >= 8192) p.resolve();
  Rec r;
  r.cls = c;
  r.a = p.get();
  r.b = p.get();
  r.flops = f;
  r.bytes = b;
  r.closed = false;
  r.slot = nullptr;
  r.units = units;
  if (dcount && units > 0) {
    r.slot = p.slot();
    if (r.slot) cudaMemcpyAsync(r.slot, dcount, sizeof(int), cudaMemcpyDeviceToDevice, s);
  }
  cudaEventRecord(r.a, s);
  p.pending.push_back(r);
  rec = &p.pending.back();
}

ProfScope::~ProfScope() {
  if (!rec) return;
  Profiler& p = prof();
  Rec* r = static_cast<Rec*>(rec);
  cudaEventRecord(r->b, st);
  std::lock_guard<std::mutex> g(p.mu);
  r->closed = true;
}

}  // namespace pdep

extern "C" int pdep_profile(int enable, pdep_profile_t* out) {
  using namespace pdep;
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (enable) {
    p.resolve();
    for (auto& a : p.acc) a = Acc();
    p.launches = 0;
    {
      std::lock_guard<std::mutex> tg(g_timer_mu);
      cudaDeviceSynchronize();
      reset_timers();
    }
    p.on = true;
    return PDEP_OK;
  }
  p.resolve();
  p.on = false;
  {
    // kernels timed on the device (also those inside graphs)
    std::lock_guard<std::mutex> tg(g_timer_mu);
    if (g_timers) {
      std::vector<DevTimer> h(PDEP_PROFILE_CLASSES);
      cudaDeviceSynchronize();
      if (cudaMemcpy(h.data(), g_timers, sizeof(DevTimer) * h.size(), cudaMemcpyDeviceToHost) ==
          cudaSuccess) {
        for (int i = 0; i < PDEP_PROFILE_CLASSES; ++i) {
          p.acc[i].launches += (long long)h[i].launches;
          p.acc[i].ms += h[i].total_ns * 1e-6;
          p.acc[i].flops += h[i].flops;
          p.acc[i].bytes += h[i].bytes;
        }
      } else {
        cudaGetLastError();
      }
    }
  }
  if (out) {
    memset(out, 0, sizeof(*out));
    out->launches = p.launches.load();
    for (int i = 0; i < PDEP_PROFILE_CLASSES; ++i) {
      strncpy(out->cls[i].name, kNames[i], sizeof(out->cls[i].name) - 1);
      out->cls[i].launches = p.acc[i].launches;
      out->cls[i].ms = p.acc[i].ms;
      out->cls[i].flops = p.acc[i].flops;
      out->cls[i].bytes = p.acc[i].bytes;
    }
  }
  return PDEP_OK;
}
