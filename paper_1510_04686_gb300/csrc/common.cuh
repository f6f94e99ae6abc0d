// Shared device/host helpers of the RGF library: complex arithmetic, batched operand
// descriptors and the internal launcher declarations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "negf.h"

namespace negf {

template <typename R>
struct cx {
  R re, im;
};
using z64 = cx<double>;

template <typename R>
__host__ __device__ __forceinline__ cx<R> mkc(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) {
  return mkc<R>(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) {
  return mkc<R>(a.re - b.re, a.im - b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mkc<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) {
  return mkc<R>(s * a.re, s * a.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> conjc(cx<R> a) {
  return mkc<R>(a.re, -a.im);
}
// acc += a * b with fused multiply-adds
template <typename R>
__device__ __forceinline__ void cfma(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// 1 / a in double precision (Smith's method avoids overflow of |a|^2)
__host__ __device__ __forceinline__ z64 crecip(z64 a) {
  double r, d;
  if (fabs(a.re) >= fabs(a.im)) {
    r = a.im / a.re;
    d = a.re + a.im * r;
    return mkc<double>(1.0 / d, -r / d);
  }
  r = a.re / a.im;
  d = a.re * r + a.im;
  return mkc<double>(r / d, -1.0 / d);
}

enum Op { OP_N = 0, OP_T = 1, OP_C = 2 };

// Batched matrix operand: batch item p lives at p_base + (idx ? idx[p] : p) * stride, and
// element (r, c) at + r * ld + c (row-major).  stride 0 with idx NULL means "shared".
template <typename R>
struct BM {
  cx<R>* p;
  long long stride;
  const int32_t* idx;
  int ld;
};
template <typename R>
struct BMc {
  const cx<R>* p;
  long long stride;
  const int32_t* idx;
  int ld;
};
template <typename R>
__host__ __device__ __forceinline__ BMc<R> cst(BM<R> a) {
  BMc<R> b;
  b.p = a.p;
  b.stride = a.stride;
  b.idx = a.idx;
  b.ld = a.ld;
  return b;
}
template <typename R>
__device__ __forceinline__ const cx<R>* bat(BMc<R> a, int p) {
  return a.p + (a.idx ? (long long)a.idx[p] : (long long)p) * a.stride;
}
template <typename R>
__device__ __forceinline__ cx<R>* bat(BM<R> a, int p) {
  return a.p + (a.idx ? (long long)a.idx[p] : (long long)p) * a.stride;
}

// ---- launchers (all asynchronous on `s`) ----------------------------------------------

// C[p] = alpha op(A[p]) op(B[p]) + beta C[p] + gamma D[p] on the CUDA cores (FP64 form).
// beta == 0 does not read C; D.p == NULL skips the D term.  Batch items with
// active[p] == 0 are skipped (active may be NULL).
template <typename R>
cudaError_t gemm_simt(cudaStream_t s, int P, int M, int N, int K, z64 alpha, BMc<R> A, int opA,
                      BMc<R> B, int opB, z64 beta, BM<R> C, z64 gamma, BMc<R> D,
                      const int32_t* active);

// X[p] = M[p]^-1 by Gauss-Jordan elimination with partial pivoting (largest |m|, lowest row
// on ties, pivots compared in FP64).  M is destroyed.  A zero pivot sets NEGF_PT_SINGULAR in
// status[p] and is replaced by a tiny number so the sweep continues.
// Scratch: U (P x n x nb), T (P x nb x n), piv (P x n) from gj_scratch_elems().
template <typename R>
cudaError_t gj_inverse(cudaStream_t s, int P, int n, BM<R> M, BM<R> X, cx<R>* U, cx<R>* T,
                       int32_t* piv, int32_t* status, const int32_t* active);
int gj_panel_width(int n, int elem_bytes);
bool gj_fits_small(int n, int elem_bytes);
// Whether the batched Gauss-Jordan inverse launches for n x n blocks of elem_bytes complex
// elements (shared-memory limits: n <= 9266 for FP32, n <= 5147 for FP64 elements).
bool gj_supports(int n, int elem_bytes);

}  // namespace negf
