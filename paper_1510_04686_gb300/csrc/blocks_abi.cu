// Block-level entry points: the batched complex GEMM and block inverse that the sweeps are
// built from, exposed for callers that assemble their own recursions.
#include <algorithm>

#include "engine.cuh"
#include "profile.cuh"
#include "tc_gemm.cuh"

using namespace negf;


extern "C" {

size_t negf_zgemm_workspace_size(int32_t precision, int32_t n_batch, int32_t M, int32_t N,
                                 int32_t K) {
  if (!prec_valid(precision) || n_batch < 1 || M < 1 || N < 1 || K < 1) return 0;
  if (precision == NEGF_PREC_FP64) return 256;
  if (!tc_supports_k(K, prec_bits(precision))) return 0;
  return tc_ws_bytes(n_batch, M, N, K, prec_bits(precision)) + 1024;
}

negf_status negf_zgemm_batched(int32_t precision, int32_t n_batch, int32_t M, int32_t N,
                               int32_t K, double alpha_re, double alpha_im, const double* A,
                               int64_t strideA, int32_t lda, int32_t opA, const double* B,
                               int64_t strideB, int32_t ldb, int32_t opB, double beta_re,
                               double beta_im, double* C, int64_t strideC, int32_t ldc,
                               void* ws, size_t ws_bytes, void* stream) {
  if (!prec_valid(precision) || n_batch < 0 || M < 0 || N < 0 || K < 0) return NEGF_ERR_ARG;
  if (n_batch == 0 || M == 0 || N == 0) return NEGF_OK;
  if (!A || !B || !C || opA < 0 || opA > 2 || opB < 0 || opB > 2) return NEGF_ERR_ARG;
  if (n_batch > 65535) return NEGF_ERR_UNSUPPORTED;
  if (prec_mixed(precision) && K > 0 && !tc_supports_k(K, prec_bits(precision)))
    return NEGF_ERR_UNSUPPORTED;
  const int rowsA = opA == OP_N ? M : K, colsA = opA == OP_N ? K : M;
  const int rowsB = opB == OP_N ? K : N, colsB = opB == OP_N ? N : K;
  (void)rowsA;
  (void)rowsB;
  if (lda < colsA || ldb < colsB || ldc < N) return NEGF_ERR_ARG;
  if (strideC == 0 && n_batch > 1) return NEGF_ERR_ARG;
  if (ws_bytes < negf_zgemm_workspace_size(precision, n_batch, M, N, K) || !ws)
    return NEGF_ERR_NOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BMc<double> a{reinterpret_cast<const z64*>(A), strideA, nullptr, lda};
  BMc<double> b{reinterpret_cast<const z64*>(B), strideB, nullptr, ldb};
  BM<double> c{reinterpret_cast<z64*>(C), strideC, nullptr, ldc};
  BMc<double> none{nullptr, 0, nullptr, 0};
  const z64 al = mkc(alpha_re, alpha_im), be = mkc(beta_re, beta_im), zero = mkc(0.0, 0.0);
  cudaError_t e;
  if (precision == NEGF_PREC_FP64) {
    if (K == 0) return NEGF_ERR_UNSUPPORTED;
    e = gemm_simt<double>(s, n_batch, M, N, K, al, a, opA, b, opB, be, c, zero, none, nullptr);
  } else {
    if (K == 0) return NEGF_ERR_UNSUPPORTED;
    size_t off = 0;
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 1023) & ~uintptr_t(1023));
    TcWs tw;
    const int bits = prec_bits(precision);
    tc_ws_carve(base, off, n_batch, M, N, K, bits, tw);
    e = tc_gemm(s, n_batch, M, N, K, al, a, opA, b, opB, be, c, zero, none, false, nullptr, tw,
                bits);
  }
  return note_error(e) == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}

size_t negf_zinv_workspace_size(int32_t precision, int32_t n_batch, int32_t n) {
  if (!prec_valid(precision) || n_batch < 1 || n < 1) return 0;
  if (!engine_supports(precision, n)) return 0;
  size_t off = 0;
  EngineWs w;
  carve_engine(nullptr, off, n_batch, n, precision, w);
  return off + 1024;
}

negf_status negf_zinv_batched(int32_t precision, int32_t n_batch, int32_t n, double* M,
                              double* X, int32_t refine_steps, int32_t* status, void* ws,
                              size_t ws_bytes, void* stream) {
  if (!prec_valid(precision) || n_batch < 0 || n < 0 || refine_steps < 0 || refine_steps > 8)
    return NEGF_ERR_ARG;
  if (n_batch == 0 || n == 0) return NEGF_OK;
  if (!M || !X || !status) return NEGF_ERR_ARG;
  if (n_batch > 65535 || !engine_supports(precision, n)) return NEGF_ERR_UNSUPPORTED;
  if (!ws || ws_bytes < negf_zinv_workspace_size(precision, n_batch, n)) return NEGF_ERR_NOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status, 0, (size_t)n_batch * sizeof(int32_t), s) != cudaSuccess)
    return NEGF_ERR_CUDA;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
  size_t off = 0;
  EngineWs w;
  carve_engine(base, off, n_batch, n, precision, w);
  negf_options o;
  negf_default_options(&o);
  Engine eng(s, precision, refine_steps, std::max(refine_steps, (int)o.refine_max), w, n);
  const long long nn = (long long)n * n;
  cudaError_t e = eng.timeout_reset();
  if (e == cudaSuccess)
    e = eng.inv(n_batch, BM<double>{reinterpret_cast<z64*>(M), nn, nullptr, n},
                BM<double>{reinterpret_cast<z64*>(X), nn, nullptr, n}, status, nullptr);
  if (e == cudaSuccess) e = eng.timeout_flag(n_batch, status);
  return note_error(e) == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}

}  // extern "C"
