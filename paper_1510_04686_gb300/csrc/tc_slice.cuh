// Operand slicing of the tensor-core complex GEMM (internal): every row of op(A) and column of
// op(B) is scaled by a power of two, rounded once to a fixed-point integer of beta * S bits and
// written as S balanced base-2^beta digits, each exact in BF16.
#pragma once
#include <cuda_bf16.h>

#include <atomic>

#include "common.cuh"

namespace negf {

constexpr int kMaxS = 12;  // most slices per value (beta * S <= 60 bits)

// Kernel attributes (the dynamic shared-memory limit) belong to a device context, so each
// kernel records, per device (ordinals below 32), whether it has set them there.
inline cudaError_t set_smem_once(std::atomic<unsigned>& done, const void* fn, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned bit = 1u << (dev & 31);
  if (done.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

// Slices of n_lines lines (rows of op(A) when kB is false; columns of op(B), written as the two
// rows [Re, -Im] and [Im, Re] of the real embedding, when kB is true) of P items (grid.y), K
// complex values each, padded with zeros to L BF16 columns: out[p][s][row][L], line exponents
// eo[p][line].  (beta, S) must be a pair that tc_plan produces; other pairs return
// cudaErrorInvalidValue.  Items with active[p] == 0 are skipped.
template <bool kB>
cudaError_t launch_slice(cudaStream_t s, int beta, int S, dim3 grid, int n_lines, int K, int L,
                         BMc<double> X, int op, bool line_is_col, __nv_bfloat16* out,
                         int32_t* eo, const int32_t* active);

}  // namespace negf
