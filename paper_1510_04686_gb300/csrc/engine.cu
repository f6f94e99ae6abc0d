// Engine dispatch: FP64 reference form and the mixed-precision tensor-core form.
#include "engine.cuh"
#include "profile.cuh"
#include "tc_gemm.cuh"

namespace negf {

namespace {
template <class T>
T* take(char* base, size_t& off, size_t n) {
  size_t a = (off + 255) & ~size_t(255);
  off = a + n * sizeof(T);
  return base ? reinterpret_cast<T*>(base + a) : nullptr;
}

__global__ void k_to32(long long n, const z64* a, cx<float>* o, const int32_t* active,
                       long long per) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    if (active && !active[k / per]) continue;
    o[k] = mkc<float>((float)a[k].re, (float)a[k].im);
  }
}
__global__ void k_to64(long long n, const cx<float>* a, z64* o, const int32_t* active,
                       long long per) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    if (active && !active[k / per]) continue;
    o[k] = mkc<double>((double)a[k].re, (double)a[k].im);
  }
}
__global__ void k_copy64(long long n, const z64* a, z64* o, const int32_t* active,
                         long long per) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    if (active && !active[k / per]) continue;
    o[k] = a[k];
  }
}
inline unsigned nblk(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
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
  if (precision == NEGF_PREC_MIXED) {
    const int nb32 = gj_panel_width(b, (int)sizeof(cx<float>));
    w.m32 = take<cx<float>>(base, off, (size_t)P * bb);
    w.x32 = take<cx<float>>(base, off, (size_t)P * bb);
    w.invU32 = take<cx<float>>(base, off, (size_t)P * b * nb32);
    w.invT32 = take<cx<float>>(base, off, (size_t)P * b * nb32);
    w.r64 = take<z64>(base, off, (size_t)P * bb);
    w.t64 = take<z64>(base, off, (size_t)P * bb);
    size_t a = (off + 1023) & ~size_t(1023);
    size_t o2 = a;
    TcWs tw;
    tc_ws_carve(base, o2, P, b, b, b, tw);
    w.tc = base ? base + a : nullptr;
    w.tc_bytes = o2 - a;
    off = o2;
  }
}

bool engine_supports(int precision, int b) {
  if (precision == NEGF_PREC_FP64) return gj_supports(b, 16);
  return precision == NEGF_PREC_MIXED && tc_supports_k(b) && gj_supports(b, 8);
}

static TcWs tc_view(const EngineWs& w, int P, int b) {
  TcWs t;
  size_t off = 0;
  tc_ws_carve(static_cast<char*>(w.tc), off, P, b, b, b, t);
  return t;
}

cudaError_t Engine::gemm(int P, int M, int N, int K, z64 alpha, BMc<double> A, int opA,
                         BMc<double> B, int opB, z64 beta, BM<double> C, z64 gamma,
                         BMc<double> D, const int32_t* active) {
  if (opt->precision == NEGF_PREC_MIXED)
    return tc_gemm(s, P, M, N, K, alpha, A, opA, B, opB, beta, C, gamma, D, false, active,
                   tc_view(w, P, b), n_sys);
  return gemm_simt<double>(s, P, M, N, K, alpha, A, opA, B, opB, beta, C, gamma, D, active);
}

cudaError_t Engine::timeout_reset() {
  if (opt->precision != NEGF_PREC_MIXED) return cudaSuccess;
  return tc_timeout_reset(s, tc_view(w, 1, b));
}

cudaError_t Engine::timeout_flag(int P, int32_t* status) {
  if (opt->precision != NEGF_PREC_MIXED) return cudaSuccess;
  return tc_timeout_flag(s, tc_view(w, 1, b), P, status);
}

cudaError_t Engine::inv(int P, BM<double> Mm, BM<double> X, int32_t* status,
                        const int32_t* active) {
  if (opt->precision != NEGF_PREC_MIXED) {
    prof_begin(s, PROF_INV);
    cudaError_t e = gj_inverse<double>(s, P, b, Mm, X, w.invU, w.invT, w.piv, status, active);
    prof_end(s, PROF_INV);
    return e;
  }
  // FP32 Gauss-Jordan start X0, then X <- X + X (I - M X) with tensor-core products
  const long long bb = (long long)b * b, n = (long long)P * bb;
  if (Mm.idx || X.idx || Mm.stride != bb || X.stride != bb || Mm.ld != b || X.ld != b)
    return cudaErrorInvalidValue;
  k_to32<<<nblk(n), 256, 0, s>>>(n, Mm.p, w.m32, active, bb);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  BM<float> m32{w.m32, bb, nullptr, b}, x32{w.x32, bb, nullptr, b};
  prof_begin(s, PROF_INV);
  e = gj_inverse<float>(s, P, b, m32, x32, w.invU32, w.invT32, w.piv, status, active);
  prof_end(s, PROF_INV);
  if (e != cudaSuccess) return e;
  k_to64<<<nblk(n), 256, 0, s>>>(n, w.x32, X.p, active, bb);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const TcWs tw = tc_view(w, P, b);
  const BMc<double> none{nullptr, 0, nullptr, 0};
  z64* cur = X.p;
  z64* nxt = w.t64;
  for (int it = 0; it < opt->refine_steps; ++it) {
    BM<double> R{w.r64, bb, nullptr, b};
    BMc<double> Mc = cst(Mm);
    BMc<double> Xc{cur, bb, nullptr, b};
    e = tc_gemm(s, P, b, b, b, mkc(-1.0, 0.0), Mc, OP_N, Xc, OP_N, mkc(0.0, 0.0), R,
                mkc(0.0, 0.0), none, true, active, tw);
    if (e != cudaSuccess) return e;
    BM<double> Xn{nxt, bb, nullptr, b};
    // X + X R with |R| << 1: only accuracy relative to |X| matters for the correction
    e = tc_gemm(s, P, b, b, b, mkc(1.0, 0.0), Xc, OP_N, cst(R), OP_N, mkc(0.0, 0.0), Xn,
                mkc(1.0, 0.0), Xc, false, active, tw, 0, true);
    if (e != cudaSuccess) return e;
    std::swap(cur, nxt);
  }
  if (cur != X.p) {
    k_copy64<<<nblk(n), 256, 0, s>>>(n, cur, X.p, active, bb);
  count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace negf
