// Engine dispatch: FP64 reference form and the mixed-precision tensor-core form.
#include "engine.cuh"

namespace negf {

namespace {
template <class T>
T* take(char* base, size_t& off, size_t n) {
  size_t a = (off + 255) & ~size_t(255);
  off = a + n * sizeof(T);
  return base ? reinterpret_cast<T*>(base + a) : nullptr;
}
}  // namespace

void carve_engine(char* base, size_t& off, int P, int b, int precision, EngineWs& w) {
  const size_t bb = (size_t)b * b;
  const int nb64 = gj_panel_width(b, (int)sizeof(z64));
  w.invU = take<z64>(base, off, (size_t)P * b * nb64);
  w.invT = take<z64>(base, off, (size_t)P * b * nb64);
  w.piv = take<int32_t>(base, off, (size_t)P * b);
  w.m32 = w.x32 = w.invU32 = w.invT32 = nullptr;
  w.r64 = w.t64 = nullptr;
  w.tc = nullptr;
  w.tc_bytes = 0;
  (void)precision;
  (void)bb;
}

bool engine_supports(int precision) { return precision == NEGF_PREC_FP64; }

cudaError_t Engine::gemm(int P, int M, int N, int K, z64 alpha, BMc<double> A, int opA,
                         BMc<double> B, int opB, z64 beta, BM<double> C, z64 gamma,
                         BMc<double> D, const int32_t* active) {
  return gemm_simt<double>(s, P, M, N, K, alpha, A, opA, B, opB, beta, C, gamma, D, active);
}

cudaError_t Engine::inv(int P, BM<double> Mm, BM<double> X, int32_t* status,
                        const int32_t* active) {
  return gj_inverse<double>(s, P, b, Mm, X, w.invU, w.invT, w.piv, status, active);
}

}  // namespace negf
