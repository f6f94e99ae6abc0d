// Lightweight launch accounting: a counter of every kernel this library launches and optional
// CUDA-event timing of the tensor-core GEMM kernel on the stream it runs on.
#pragma once
#include <cuda_runtime.h>

namespace negf {
void count_launch(int n = 1);
// Remember a CUDA error that made a public call fail (read back by negf_last_cuda_error).
cudaError_t note_error(cudaError_t e);
bool profiling_on();
// Record an event pair around one launch of kernel class `kind` on stream s.
void prof_begin(cudaStream_t s, int kind);
void prof_end(cudaStream_t s, int kind);
// Add the flops one launch dispatches: complex algorithmic 8 M N K and issued BF16 MMA flops.
void prof_flops(int kind, double alg, double hw);
enum { PROF_TC_GEMM = 0, PROF_SLICE = 1, PROF_INV = 2, PROF_GJ_PANEL = 3, PROF_KINDS = 4 };
}  // namespace negf
