// Engine dispatch: FP64 reference form and the mixed-precision tensor-core form.
#include <atomic>

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
inline unsigned nblk(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}
}  // namespace

__device__ unsigned long long g_fp64_fallbacks;  // items recomputed by the FP64 fallback

// Newton-Schulz gating: act[p] = (active ? active[p] : 1) && (force || rmax[p] > tol); rmax[p]
// is reset to 0 for the next residual product.  With count set, the selected items are added
// to g_fp64_fallbacks.  act may alias active (each thread reads its own entry first).
__global__ void k_refine_gate(int P, const int32_t* active, int force, float* rmax, float tol,
                              int32_t* act, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const bool base = active ? active[p] != 0 : true;
  const bool on = base && (force || rmax[p] > tol);
  act[p] = on ? 1 : 0;
  rmax[p] = 0.0f;
  if (on && count) atomicAdd(&g_fp64_fallbacks, 1ull);
}

// Residual target of the mixed-form inverse: after a step with max |R| <= 2^-24 the next
// residual R^2 is at the rounding floor of the products.
constexpr float kRefineTol = 5.9604644775390625e-8f;
void carve_engine(char* base, size_t& off, int P, int b, int precision, EngineWs& w) {
  const size_t bb = (size_t)b * b;
  const int nb64 = gj_panel_width(b, (int)sizeof(z64));
  w.invU = take<z64>(base, off, (size_t)P * b * nb64);
  w.invT = take<z64>(base, off, (size_t)P * b * nb64);
  w.piv = take<int32_t>(base, off, (size_t)P * b);
  w.m32 = w.x32 = w.invU32 = w.invT32 = nullptr;
  w.r64 = nullptr;
  w.act = nullptr;
  w.rmax = nullptr;
  w.tc = nullptr;
  w.tc_bytes = 0;
  if (prec_mixed(precision)) {
    const int nb32 = gj_panel_width(b, (int)sizeof(cx<float>));
    w.m32 = take<cx<float>>(base, off, (size_t)P * bb);
    w.x32 = take<cx<float>>(base, off, (size_t)P * bb);
    w.invU32 = take<cx<float>>(base, off, (size_t)P * b * nb32);
    w.invT32 = take<cx<float>>(base, off, (size_t)P * b * nb32);
    w.r64 = take<z64>(base, off, (size_t)P * bb);
    w.act = take<int32_t>(base, off, (size_t)P);
    w.rmax = take<float>(base, off, (size_t)P);
    size_t a = (off + 1023) & ~size_t(1023);
    size_t o2 = a;
    TcWs tw;
    tc_ws_carve(base, o2, P, b, b, b, prec_bits(precision), tw);
    w.tc = base ? base + a : nullptr;
    w.tc_bytes = o2 - a;
    off = o2;
  }
}

bool engine_supports(int precision, int b) {
  if (precision == NEGF_PREC_FP64) return gj_supports(b, 16);
  return prec_mixed(precision) && tc_supports_k(b, prec_bits(precision)) && gj_supports(b, 8);
}

int lead_precision(const negf_options* o, int b) {
  if (o->lead_precision != NEGF_PREC_AUTO) return o->lead_precision;
  if (o->precision == NEGF_PREC_FP64) return NEGF_PREC_FP64;
  return engine_supports(NEGF_PREC_MIXED_56, b) ? NEGF_PREC_MIXED_56 : NEGF_PREC_MIXED;
}

int lead_step_precision(const negf_options* o, int b, int it) {
  const int p = lead_precision(o, b);
  if (o->lead_precision != NEGF_PREC_AUTO || p != NEGF_PREC_MIXED_56) return p;
  if (it == 0) return NEGF_PREC_MIXED;
  if (it <= 8) return NEGF_PREC_MIXED_56;
  return it <= 14 ? NEGF_PREC_MIXED : NEGF_PREC_MIXED_40;
}

long long engine_fp64_fallbacks() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_fp64_fallbacks, sizeof(v)) != cudaSuccess) return -1;
  return (long long)v;
}

static TcWs tc_view(const EngineWs& w, int P, int b, int bits) {
  TcWs t;
  size_t off = 0;
  tc_ws_carve(static_cast<char*>(w.tc), off, P, b, b, b, bits, t);
  return t;
}

cudaError_t Engine::gemm(int P, int M, int N, int K, z64 alpha, BMc<double> A, int opA,
                         BMc<double> B, int opB, z64 beta, BM<double> C, z64 gamma,
                         BMc<double> D, const int32_t* active) {
  if (prec_mixed(prec))
    return tc_gemm(s, P, M, N, K, alpha, A, opA, B, opB, beta, C, gamma, D, false, active,
                   tc_view(w, P, b, prec_bits(prec)), prec_bits(prec), n_sys);
  return gemm_simt<double>(s, P, M, N, K, alpha, A, opA, B, opB, beta, C, gamma, D, active);
}

cudaError_t Engine::timeout_reset() {
  if (!prec_mixed(prec)) return cudaSuccess;
  return tc_timeout_reset(s, tc_view(w, 1, b, prec_bits(prec)));
}

namespace {
std::atomic<int> g_fail_waits{0};
}

cudaError_t Engine::timeout_flag(int P, int32_t* status) {
  if (!prec_mixed(prec)) return cudaSuccess;
  const TcWs tw = tc_view(w, 1, b, prec_bits(prec));
  if (g_fail_waits.load()) {  // test hook: report as if a bounded wait had given up
    cudaError_t e = cudaMemsetAsync(tw.err, 1, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
  }
  return tc_timeout_flag(s, tw, P, status);
}

void engine_fail_waits(int on) { g_fail_waits.store(on ? 1 : 0); }

cudaError_t Engine::inv(int P, BM<double> Mm, BM<double> X, int32_t* status,
                        const int32_t* active) {
  if (!prec_mixed(prec)) {
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
  if (refine_max <= 0) return cudaSuccess;
  const int bits = prec_bits(prec);
  const TcWs tw = tc_view(w, P, b, bits);
  const BMc<double> none{nullptr, 0, nullptr, 0};
  const unsigned gb = (unsigned)((P + 255) / 256);
  BM<double> R{w.r64, bb, nullptr, b};
  const BMc<double> Mc = cst(Mm);
  const BMc<double> Xc{X.p, bb, nullptr, b};
  for (int it = 0; it < refine_max; ++it) {
    // items refined by this step: all of them for the first refine_min steps, afterwards those
    // whose previous residual stayed above the target
    k_refine_gate<<<gb, 256, 0, s>>>(P, active, (it == 0 || it < refine_min) ? 1 : 0, w.rmax,
                                     kRefineTol, w.act, 0);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = tc_gemm(s, P, b, b, b, mkc(-1.0, 0.0), Mc, OP_N, Xc, OP_N, mkc(0.0, 0.0), R,
                mkc(0.0, 0.0), none, true, w.act, tw, bits, 0, false, w.rmax);
    if (e != cudaSuccess) return e;
    // X <- X + X R in place (each output element reads only its own X entry; the product reads
    // the slices of X made before it).  With |R| << 1 only accuracy relative to |X| matters.
    e = tc_gemm(s, P, b, b, b, mkc(1.0, 0.0), Xc, OP_N, cst(R), OP_N, mkc(0.0, 0.0), X,
                mkc(1.0, 0.0), Xc, false, w.act, tw, bits, 0, true);
    if (e != cudaSuccess) return e;
  }
  // items whose last residual was still above the target: FP64 Gauss-Jordan (M is intact)
  k_refine_gate<<<gb, 256, 0, s>>>(P, w.act, 0, w.rmax, kRefineTol, w.act, 1);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  prof_begin(s, PROF_INV);
  e = gj_inverse<double>(s, P, b, Mm, X, w.invU, w.invT, w.piv, status, w.act);
  prof_end(s, PROF_INV);
  return e;
}

}  // namespace negf
