// Per-kernel-class CUDA-event timing and launch counting.
#pragma once

#include "common.cuh"

namespace pdep {

enum ProfClass : int {
  PC_COLS_F64 = 0,
  PC_COLS_F32 = 1,
  PC_SLAB_F64 = 2,
  PC_SLAB_F32 = 3,
  PC_GEMM_F64 = 4,
  PC_GEMM_F32 = 5,
  PC_CG_F64 = 6,
  PC_CG_F32 = 7,
  PC_EIGH = 8,
  PC_OTHER = 9,
  PC_GEMM_TF32 = 10,  // tensor-core (3xTF32) FP32 projections
  PC_CG_GRAPH_F32 = 11,  // whole captured CG loops (FP32 steps; their kernels are not
  PC_CG_GRAPH_F64 = 12,  // timed one by one inside a graph)
  PC_COLS_DF = 13,       // double-float transforms (mixed-precision refinement)
  PC_SLAB_DF = 14,
  PC_HPSI_FUSED = 15,    // FP32 H x in one launch (column scratch in shared memory)
  PC_GEMM_DF = 16,       // double-float GEMMs (mixed-precision projections)
};

// counts one kernel launch (always cheap); while this thread captures a
// graph the launches are counted for the capture instead (capture_end
// returns that count) and ProfScope records nothing
void count_launch();
void capture_begin();
int capture_end();
// kernels launched by this process outside graph captures (always counted)
long long launch_count();

// Device-side timing of kernels that also run inside CUDA graphs, where
// events cannot time a single kernel: thread 0 of every block records
// %globaltimer at the block's start and end; the last block of a launch adds
// max(end) - min(start) and the launch's work to its class.  pdep_profile
// resets the timers when it starts and folds them into the profile when it
// stops.  The timers live in device memory allocated by dev_timers_init (on
// the current device, once per process, before any capture).
struct DevTimer {
  unsigned long long t_min, t_max;
  unsigned long long total_ns, launches;
  double flops, bytes;
  unsigned int done, pad;
};
int dev_timers_init();
DevTimer* dev_timer(int cls);

__device__ __forceinline__ unsigned long long dev_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// called by thread 0 of every block at its end (t0: its start)
__device__ __forceinline__ void dev_timer_block_end(DevTimer* t, unsigned long long t0,
                                                    double flops, double bytes) {
  if (!t) return;
  atomicMin(&t->t_min, t0);
  atomicMax(&t->t_max, dev_clock_ns());
  if (flops != 0.0) atomicAdd(&t->flops, flops);
  if (bytes != 0.0) atomicAdd(&t->bytes, bytes);
  __threadfence();
  if (atomicAdd(&t->done, 1u) == gridDim.x - 1) {
    __threadfence();
    const unsigned long long lo = atomicOr(&t->t_min, 0ull), hi = atomicOr(&t->t_max, 0ull);
    t->total_ns += hi > lo ? hi - lo : 0ull;
    t->launches += 1;
    t->t_min = ~0ull;
    t->t_max = 0ull;
    t->done = 0u;
  }
}

// RAII timer around one launch: events are recorded only while profiling.
// flops and bytes are those of a launch over 'units' work units; when the
// launch reads its unit count from the device (dcount), that count is
// copied aside with the launch and the counts are scaled by dcount/units
// when the record is resolved.
struct ProfScope {
  ProfScope(int cls, cudaStream_t st, double flops, double bytes, const int* dcount = nullptr,
            int units = 0);
  ~ProfScope();
  int cls;
  cudaStream_t st;
  double flops, bytes;
  void* rec;  // the open record, or null while not profiling
};

}  // namespace pdep
