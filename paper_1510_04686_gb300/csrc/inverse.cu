// Batched block inversion g = M^-1 of the sweeps of Eq. (1): Gauss-Jordan elimination with
// partial pivoting.  Pivot magnitudes are compared in FP64 (largest |m|^2, lowest row on ties)
// and the pivot reciprocal is taken in FP64 whatever the storage type R.
//
// n <= small limit: one CTA per matrix, the whole matrix in shared memory.
// larger n: blocked Gauss-Jordan.  A panel of nb columns is eliminated in shared memory, the
// recorded row swaps are applied to the rest of the matrix and the remaining columns get the
// rank-nb update  A[:, rest] += Panel * A[pivot rows, rest]  (pivot rows zeroed first), which is
// a batched GEMM.  The column permutation is undone at the end.
#include <algorithm>

#include "common.cuh"
#include "profile.cuh"

namespace negf {

namespace {

constexpr int kThreads = 256;
constexpr size_t kSmemBudget = 180 * 1024;

template <typename R>
__device__ __forceinline__ double mag2(cx<R> a) {
  return (double)a.re * (double)a.re + (double)a.im * (double)a.im;
}

// Block-wide argmax of |col[r]|^2 over r in [r0, n) (ties -> lowest r).  Returns the row.
template <typename R>
__device__ int block_argmax(const cx<R>* col, int stride, int r0, int n, double* sv, int* si) {
  double best = -1.0;
  int bi = n;
  for (int r = r0 + threadIdx.x; r < n; r += blockDim.x) {
    double v = mag2(col[(long long)r * stride]);
    if (v > best) {
      best = v;
      bi = r;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, best, off);
    int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sv[w] = best;
    si[w] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double b = sv[0];
    int i = si[0];
    for (int k = 1; k < nw; ++k)
      if (sv[k] > b || (sv[k] == b && si[k] < i)) {
        b = sv[k];
        i = si[k];
      }
    si[0] = (i >= n) ? r0 : i;
  }
  __syncthreads();
  int res = si[0];
  __syncthreads();
  return res;
}

template <typename R>
__device__ __forceinline__ cx<R> pivot_recip(cx<R> a, int32_t* st) {
  z64 ad = mkc<double>((double)a.re, (double)a.im);
  if (ad.re == 0.0 && ad.im == 0.0) {
    if (threadIdx.x == 0 && st) atomicOr(st, NEGF_PT_SINGULAR);
    ad.re = sizeof(R) == 8 ? 1e-300 : 1e-30;
  }
  z64 d = crecip(ad);
  return mkc<R>((R)d.re, (R)d.im);
}

// One Gauss-Jordan step on column jj of an (rows x w) shared-memory array P (row stride w)
// whose pivot row is `j`.  Uses f[rows] scratch.  Thread t works on column t % w of rows
// t / w, t / w + blockDim / w, ... (no index division in the loops).
template <typename R>
__device__ void gj_step(cx<R>* P, int rows, int w, int j, int jj, cx<R>* f, int32_t* st) {
  for (int r = threadIdx.x; r < rows; r += blockDim.x) f[r] = P[(long long)r * w + jj];
  __syncthreads();
  const cx<R> d = pivot_recip(f[j], st);
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    cx<R>& e = P[(long long)j * w + c];
    e = (c == jj) ? d : e * d;
  }
  __syncthreads();
  if (w <= (int)blockDim.x) {
    const int c = threadIdx.x % w;
    const int r0 = threadIdx.x / w, rstep = blockDim.x / w;
    if (r0 < rstep) {
      const cx<R> pj = P[(long long)j * w + c];
      for (int r = r0; r < rows; r += rstep) {
        if (r == j) continue;
        const cx<R> fr = f[r];
        cx<R>* e = P + (long long)r * w + c;
        if (c == jj) {
          *e = mkc<R>(R(0), R(0)) - fr * d;
        } else {
          cx<R> v = *e;
          v.re = v.re - (fr.re * pj.re - fr.im * pj.im);
          v.im = v.im - (fr.re * pj.im + fr.im * pj.re);
          *e = v;
        }
      }
    }
  } else {
    for (int r = 0; r < rows; ++r) {
      if (r == j) continue;
      const cx<R> fr = f[r];
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        cx<R>* e = P + (long long)r * w + c;
        if (c == jj) {
          *e = mkc<R>(R(0), R(0)) - fr * d;
        } else {
          const cx<R> pj = P[(long long)j * w + c];
          cx<R> v = *e;
          v.re = v.re - (fr.re * pj.re - fr.im * pj.im);
          v.im = v.im - (fr.re * pj.im + fr.im * pj.re);
          *e = v;
        }
      }
    }
  }
  __syncthreads();
}

template <typename R>
__device__ void swap_rows_smem(cx<R>* P, int w, int a, int b) {
  if (a == b) return;
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    cx<R> t = P[(long long)a * w + c];
    P[(long long)a * w + c] = P[(long long)b * w + c];
    P[(long long)b * w + c] = t;
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_gj_small(int n, BM<R> Mm, BM<R> X, int32_t* status,
                                                       const int32_t* active) {
  const int p = blockIdx.x;
  if (active && !active[p]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* A = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* f = A + (size_t)n * n;
  int* perm = reinterpret_cast<int*>(f + n);
  int* src = perm + n;
  __shared__ double sv[32];
  __shared__ int si[32];
  int32_t* st = status ? status + p : nullptr;
  const cx<R>* m = bat(Mm, p);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = m[(long long)(e / n) * Mm.ld + e % n];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    int pr = block_argmax(A + j, n, j, n, sv, si);
    if (threadIdx.x == 0) perm[j] = pr;
    swap_rows_smem(A, n, j, pr);
    gj_step(A, n, n, j, j, f, st);
  }
  if (threadIdx.x == 0) {
    for (int c = 0; c < n; ++c) src[c] = c;
    for (int j = n - 1; j >= 0; --j) {
      int t = src[j];
      src[j] = src[perm[j]];
      src[perm[j]] = t;
    }
  }
  __syncthreads();
  cx<R>* x = bat(X, p);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e % n;
    x[(long long)r * X.ld + c] = A[r * n + src[c]];
  }
}

// Panel step of the blocked form: columns [k0, k0 + w) of A (n x n, in global memory).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_gj_panel(int n, int k0, int w, int nb, BM<R> Am,
                                                       cx<R>* U, cx<R>* T, int32_t* piv,
                                                       int32_t* status, const int32_t* active) {
  const int p = blockIdx.x;
  if (active && !active[p]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* P = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* f = P + (size_t)n * w;
  __shared__ double sv[32];
  __shared__ int si[32];
  int32_t* st = status ? status + p : nullptr;
  cx<R>* a = bat(Am, p);
  const long long ld = Am.ld;
  int32_t* pv = piv + (long long)p * n;
  for (int r = threadIdx.x / w; r < n; r += blockDim.x / w) {
    const int c = threadIdx.x % w;
    if (threadIdx.x / w < (int)blockDim.x / w) P[(long long)r * w + c] = a[r * ld + k0 + c];
  }
  __syncthreads();
  for (int jj = 0; jj < w; ++jj) {
    const int j = k0 + jj;
    int pr = block_argmax(P + jj, w, j, n, sv, si);
    if (threadIdx.x == 0) pv[j] = pr;
    swap_rows_smem(P, w, j, pr);
    gj_step(P, n, w, j, jj, f, st);
  }
  // row swaps on the columns outside the panel, in elimination order
  for (int jj = 0; jj < w; ++jj) {
    const int j = k0 + jj;
    const int pr = pv[j];
    if (pr != j) {
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        if (c >= k0 && c < k0 + w) continue;
        cx<R> t = a[j * ld + c];
        a[j * ld + c] = a[pr * ld + c];
        a[pr * ld + c] = t;
      }
    }
    __syncthreads();
  }
  // T = pivot rows (panel columns zeroed); those rows of A are cleared outside the panel
  cx<R>* Tp = T + (long long)p * nb * n;
  for (int jj = 0; jj < w; ++jj) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      cx<R>* ae = a + (long long)(k0 + jj) * ld + c;
      if (c >= k0 && c < k0 + w) {
        Tp[(long long)jj * n + c] = mkc<R>(R(0), R(0));
      } else {
        Tp[(long long)jj * n + c] = *ae;
        *ae = mkc<R>(R(0), R(0));
      }
    }
  }
  cx<R>* Up = U + (long long)p * n * nb;
  for (int r = threadIdx.x / w; r < n; r += blockDim.x / w) {
    const int c = threadIdx.x % w;
    if (threadIdx.x / w < (int)blockDim.x / w) {
      const cx<R> v = P[(long long)r * w + c];
      a[r * ld + k0 + c] = v;
      Up[(long long)r * nb + c] = v;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_gj_unpermute(int n, BM<R> Am, BM<R> X,
                                                           const int32_t* piv,
                                                           const int32_t* active) {
  const int p = blockIdx.x;
  if (active && !active[p]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* src = reinterpret_cast<int*>(smem_raw);
  const int32_t* pv = piv + (long long)p * n;
  if (threadIdx.x == 0) {
    for (int c = 0; c < n; ++c) src[c] = c;
    for (int j = n - 1; j >= 0; --j) {
      int t = src[j];
      src[j] = src[pv[j]];
      src[pv[j]] = t;
    }
  }
  __syncthreads();
  const cx<R>* a = bat(Am, p);
  cx<R>* x = bat(X, p);
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    int r = (int)(e / n), c = (int)(e % n);
    x[(long long)r * X.ld + c] = a[(long long)r * Am.ld + src[c]];
  }
}

}  // namespace

bool gj_fits_small(int n, int elem_bytes) {
  size_t need = (size_t)n * n * elem_bytes + (size_t)n * elem_bytes + 2 * n * sizeof(int);
  return need <= kSmemBudget;
}

int gj_panel_width(int n, int elem_bytes) {
  size_t per_col = (size_t)n * elem_bytes;
  int w = (int)std::min<size_t>(32, (kSmemBudget - (size_t)n * elem_bytes) / per_col);
  int p2 = 1;
  while (p2 * 2 <= w) p2 *= 2;
  return std::max(1, p2);
}

template <typename R>
cudaError_t gj_inverse(cudaStream_t s, int P, int n, BM<R> M, BM<R> X, cx<R>* U, cx<R>* T,
                       int32_t* piv, int32_t* status, const int32_t* active) {
  if (P <= 0 || n <= 0) return cudaSuccess;
  const int eb = (int)sizeof(cx<R>);
  if (gj_fits_small(n, eb)) {
    size_t smem = (size_t)n * n * eb + (size_t)n * eb + 2 * n * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(k_gj_small<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBudget + 1024);
    if (e != cudaSuccess) return e;
    k_gj_small<R><<<P, kThreads, smem, s>>>(n, M, X, status, active);
    count_launch();
    return cudaGetLastError();
  }
  const int nb = gj_panel_width(n, eb);
  cudaError_t e = cudaFuncSetAttribute(k_gj_panel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemBudget + 1024);
  if (e != cudaSuccess) return e;
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int w = std::min(nb, n - k0);
    size_t smem = (size_t)n * w * eb + (size_t)n * eb;
    k_gj_panel<R><<<P, kThreads, smem, s>>>(n, k0, w, nb, M, U, T, piv, status, active);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    BMc<R> Ua{U, (long long)n * nb, nullptr, nb};
    BMc<R> Ta{T, (long long)nb * n, nullptr, n};
    BMc<R> none{nullptr, 0, nullptr, 0};
    e = gemm_simt<R>(s, P, n, n, w, mkc<double>(1.0, 0.0), Ua, OP_N, Ta, OP_N,
                     mkc<double>(1.0, 0.0), M, mkc<double>(0.0, 0.0), none, active);
    if (e != cudaSuccess) return e;
  }
  k_gj_unpermute<R><<<P, kThreads, n * sizeof(int), s>>>(n, M, X, piv, active);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t gj_inverse<double>(cudaStream_t, int, int, BM<double>, BM<double>,
                                        cx<double>*, cx<double>*, int32_t*, int32_t*,
                                        const int32_t*);
template cudaError_t gj_inverse<float>(cudaStream_t, int, int, BM<float>, BM<float>, cx<float>*,
                                       cx<float>*, int32_t*, int32_t*, const int32_t*);

}  // namespace negf
