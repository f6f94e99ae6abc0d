// Tensor-core complex GEMM with FP64-class accuracy from exact split-BF16 products.
//
//   C = alpha op(A) op(B) + beta C + gamma D (+ I)       (complex128 in and out)
//
// Each operand row (A) / column (B) is scaled by a power of two, rounded once to a fixed-point
// value of 40, 48 or 56 bits and cut into S slices of beta bits stored as BF16 (exact).  Slice
// products are exact in BF16 x BF16 -> FP32 and, with beta and a split of K into parts chosen
// from K, every group of slice pairs of one order s + t - 1 over one part sums to an integer
// below 2^24 and is exact in its FP32 TMEM accumulator (the tensor core's accumulation
// truncates, so inexact groups would lose bits linearly in K); the groups are added into a
// TMEM-resident FP32-pair sum and converted to FP64 once in the epilogue.  Products of order > S
// are dropped (below 2^-(beta S) of the scale).  The complex product uses the real embedding
// [Re A, Im A] x [[Re B, Im B], [-Im B, Re B]]  so that one MMA chain produces interleaved
// (re, im) outputs.
#pragma once
#include "common.cuh"

namespace negf {

struct TcWs {
  void* slicesA;        // bf16 [P][S][M][L]
  void* slicesB;        // bf16 [P][S][2N][L]
  int32_t* expA;        // [P][M]
  int32_t* expB;        // [P][N]
  int32_t* err;         // device error word (bounded waits that gave up)
};

// Fixed-point bits per operand value (the precision tier of the product): 40, 48 or 56.
bool tc_bits_ok(int bits);

// Bytes of TcWs scratch for P items of an M x N x K product at `bits` bits per value.
size_t tc_ws_bytes(int P, int M, int N, int K, int bits);
void tc_ws_carve(char* base, size_t& off, int P, int M, int N, int K, int bits, TcWs& w);

// Slices and exactness parameters of a contraction: digit width beta, slice count S (values of
// beta S - 1 >= bits - 1 bits), K split into `parts` and at most `gsize` slice products of one
// order summed per exact FP32 accumulator group.
struct TcPlan {
  int beta, S, parts, gsize;
};
// The plan for a contraction length K (complex) when at most max_parts K parts may be used.
// False when no exact plan exists.
bool tc_plan(int K, int bits, int max_parts, TcPlan* out);
// Whether the tensor-core GEMM covers K exactly under every configuration at `bits` bits per
// value (48 bits: K <= 28032).
bool tc_supports_k(int K, int bits);

// The device error word ws.err is set when a bounded wait inside the GEMM kernel gave up (the
// tile's outputs are then NaN).  tc_timeout_reset zeroes it; tc_timeout_flag ORs
// NEGF_PT_TIMEOUT into status[0..P) when it is set.  Both are asynchronous on s.
cudaError_t tc_timeout_reset(cudaStream_t s, const TcWs& ws);
cudaError_t tc_timeout_flag(cudaStream_t s, const TcWs& ws, int P, int32_t* status);

// Flops of the tensor-core GEMM launches made while profiling was on, counted on the device
// for the items that ran (the current device; both calls synchronise it): algorithmic complex
// 8 M N K, and the BF16 MMA flops issued over the padded tiles.
cudaError_t tc_prof_flops(double* alg, double* hw);
cudaError_t tc_prof_reset();

// n_distinct: number of different matrices an indexed operand (idx != NULL) selects from
// (0 = unknown: slice every item).  trunc_a: the product only needs to be accurate relative
// to the rows of op(A) (it is a correction much smaller than a term of that size, such as
// X R in the Newton-Schulz step X + X R with |R| < 1): each output tile drops the slice orders
// whose terms stay below 2^(-beta S) of the A row scale, given the largest column exponent of
// op(B) in the tile.  The issued-flop count of the launch is then an upper bound.
// bits: fixed-point bits per operand value (tc_bits_ok); the workspace must have been carved for
// the same bits.  rmax (nullable, float [P], zeroed by the caller): rmax[p] is raised to the
// largest |Re| or |Im| of item p's outputs (the Newton-Schulz residual norm when C = I - M X).
cudaError_t tc_gemm(cudaStream_t s, int P, int M, int N, int K, z64 alpha, BMc<double> A,
                    int opA, BMc<double> B, int opB, z64 beta, BM<double> C, z64 gamma,
                    BMc<double> D, bool add_identity, const int32_t* active, const TcWs& ws,
                    int bits, int n_distinct = 0, bool trunc_a = false, float* rmax = nullptr);

}  // namespace negf
