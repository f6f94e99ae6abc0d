// Block-operation engine of the sweeps: the batched complex GEMM and the batched block
// inverse for the precision chosen in negf_options.  FP64 form: CUDA-core GEMM and FP64
// Gauss-Jordan.  Mixed form: tensor-core GEMM of exact split-BF16 slices and an FP32
// Gauss-Jordan inverse polished by Newton-Schulz steps X <- X + X (I - M X).
#pragma once
#include <utility>

#include "common.cuh"

namespace negf {

struct EngineWs {
  // FP64 inverse scratch
  z64* invU;
  z64* invT;
  int32_t* piv;
  // mixed-precision scratch
  cx<float>* m32;    // FP32 copy of the matrices being inverted, P x b x b
  cx<float>* x32;    // FP32 inverse, P x b x b
  cx<float>* invU32;
  cx<float>* invT32;
  z64* r64;          // residual I - M X, P x b x b
  z64* t64;          // temporary, P x b x b
  void* tc;          // tensor-core GEMM operand slices
  size_t tc_bytes;
};

// Reserve the engine scratch for P concurrent b x b problems at `off` of `base` (base NULL:
// only advance `off`).
void carve_engine(char* base, size_t& off, int P, int b, int precision, EngineWs& w);

struct Engine {
  cudaStream_t s;
  const negf_options* opt;
  EngineWs w;
  int b;
  int n_sys = 0;  // distinct Hamiltonians an indexed operand selects from (0 = unknown)
  Engine(cudaStream_t s_, const negf_options* o, const EngineWs& w_, int b_, int n_sys_ = 0)
      : s(s_), opt(o), w(w_), b(b_), n_sys(n_sys_) {}
  // C = alpha op(A) op(B) + beta C + gamma D for P batch items of M x N x K.
  cudaError_t gemm(int P, int M, int N, int K, z64 alpha, BMc<double> A, int opA, BMc<double> B,
                   int opB, z64 beta, BM<double> C, z64 gamma, BMc<double> D,
                   const int32_t* active);
  // Mixed form: clear the tensor-core GEMM's timeout word / OR NEGF_PT_TIMEOUT into
  // status[0..P) if a GEMM since the reset gave up a bounded wait.  No-ops in the FP64 form.
  cudaError_t timeout_reset();
  cudaError_t timeout_flag(int P, int32_t* status);
  // X = Mm^-1 for P items of size b (Mm is destroyed); zero pivots flag status[item].
  cudaError_t inv(int P, BM<double> Mm, BM<double> X, int32_t* status, const int32_t* active);
};

// Whether this build implements the precision form (negf_precision) for blocks of size b: the
// block inverse launches up to b = 5147 (FP64) / 9266 (mixed, FP32 elimination), and the mixed
// form's tensor-core GEMM is exact up to a contraction length of 28032.
bool engine_supports(int precision, int b);

// Adjoint workspace helpers (adjoint.cu)
size_t adjoint_bytes(const negf_device* dev, int P, const negf_options* opt);
int adjoint_chunk(const negf_device* dev, int n_pts, const negf_options* opt);

}  // namespace negf
