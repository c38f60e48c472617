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
};

// counts one kernel launch (always cheap); while this thread captures a
// graph the launches are counted for the capture instead (capture_end
// returns that count) and ProfScope records nothing
void count_launch();
void capture_begin();
int capture_end();
// kernels launched by this process outside graph captures (always counted)
long long launch_count();

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
