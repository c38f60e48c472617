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
};

// counts one kernel launch (always cheap)
void count_launch();

// RAII timer around one launch: events are recorded only while profiling
struct ProfScope {
  ProfScope(int cls, cudaStream_t st, double flops, double bytes);
  ~ProfScope();
  int cls;
  cudaStream_t st;
  double flops, bytes;
  void* rec;  // the open record, or null while not profiling
};

}  // namespace pdep
