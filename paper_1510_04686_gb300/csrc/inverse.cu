// Batched block inversion g = M^-1 of the sweeps of Eq. (1): Gauss-Jordan elimination with
// partial pivoting (largest |m|^2, lowest row on ties; magnitudes to FP64 accuracy, as FP32 pairs
// for FP32 storage) and the pivot reciprocal in the storage precision (the FP32 form is refined
// by Newton-Schulz steps afterwards).
//
// n <= small limit: one CTA per matrix, the whole matrix in shared memory.
// larger n: blocked Gauss-Jordan.  A panel of nb columns is eliminated in shared memory, the
// recorded row swaps are applied to the rest of the matrix and the remaining columns get the
// rank-nb update  A[:, rest] += Panel * A[pivot rows, rest]  (pivot rows zeroed first), which is
// a batched GEMM.  The column permutation is undone at the end.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "profile.cuh"

namespace negf {

namespace {

constexpr int kThreads = 256;
constexpr size_t kSmemBudget = 180 * 1024;

// Pivot magnitude |a|^2 = hi + lo.  FP64 storage: hi = |a|^2 in FP64, lo = 0.  FP32 storage: the
// exact squares as FP32 pairs (product and its fmaf residual) and the exact sum of the leading
// parts (TwoSum), so hi + lo carries about 48 bits: an FP64-class pivot decision without the
// FP64 pipe.  Intrinsics keep the compiler from fusing the steps.  (The entries of the blocks
// inverted here lie between about 1e-19 and 1e19 in magnitude, where no square over- or
// underflows in FP32.)
template <typename R>
struct Mag {
  R hi, lo;
};
template <typename R>
__device__ __forceinline__ Mag<R> mag2(cx<R> a) {
  if constexpr (sizeof(R) == 8) {
    return Mag<R>{a.re * a.re + a.im * a.im, 0.0};
  } else {
    const float p = __fmul_rn(a.re, a.re), q = __fmul_rn(a.im, a.im);
    const float ep = fmaf(a.re, a.re, -p), eq = fmaf(a.im, a.im, -q);
    const float s = __fadd_rn(p, q);
    const float bq = __fsub_rn(s, p);
    const float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bq)), __fsub_rn(q, bq));
    return Mag<R>{s, __fadd_rn(t, __fadd_rn(ep, eq))};
  }
}
// a (row ia) is a better pivot than b (row ib): larger magnitude, lower row on ties.  The sign of
// (a.hi - b.hi) + (a.lo - b.lo) is that of the exact difference except within FP64-level ties.
template <typename R>
__device__ __forceinline__ bool better(Mag<R> a, int ia, Mag<R> b, int ib) {
  const R d = (a.hi - b.hi) + (a.lo - b.lo);
  return d > R(0) || (d == R(0) && ia < ib);
}

// 1 / a, flagging an exactly zero pivot (replaced by a tiny number so the sweep goes on).  FP64
// for FP64 storage; for FP32, a is first scaled by the power of two 2^-e that brings its larger
// component into [0.5, 1), so |a'|^2 lies in [0.25, 2) and 1/a = conj(a') 2^-e / |a'|^2 loses
// nothing to overflow or underflow.
template <typename R>
__device__ __forceinline__ cx<R> pivot_recip(cx<R> a, int32_t* st) {
  if (a.re == R(0) && a.im == R(0)) {
    if (st) atomicOr(st, NEGF_PT_SINGULAR);
    a.re = sizeof(R) == 8 ? R(1e-300) : R(1e-30);
  }
  if constexpr (sizeof(R) == 8) {
    return crecip(a);
  } else {
    int e;
    frexpf(fmaxf(fabsf(a.re), fabsf(a.im)), &e);
    const float ar = ldexpf(a.re, -e), ai = ldexpf(a.im, -e);
    const float inv = ldexpf(1.0f / (ar * ar + ai * ai), -e);
    return mkc<float>(ar * inv, -ai * inv);
  }
}

// Per-CTA scratch of one Gauss-Jordan column step.
template <typename R>
struct GjScratch {
  Mag<R> sv[32];
  int si[32];
  cx<R> d;
};

// One Gauss-Jordan step on column jj of the shared-memory array P (rows x w, row stride w):
// pivot search over rows [j, rows) (largest |m|^2, lowest row on ties), swap of rows j and the
// pivot row, pivot reciprocal (pivot_recip), and elimination of column jj from all
// other rows.  f[rows] and prow[w] are shared scratch.  Three block barriers per column:
//   (1) after the per-warp argmax, (2) after the swap / column copy / reciprocal, (3) after the
//   update.  Every thread combines the per-warp winners itself, and the elimination scales the
//   pivot row on the fly from an unscaled copy, so no further barrier is needed.
// Returns the pivot row.
template <typename R>
__device__ int gj_column(cx<R>* P, int rows, int w, int j, int jj, cx<R>* f, cx<R>* prow,
                         GjScratch<R>& sc, int32_t* st) {
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, wid = tid >> 5;
  Mag<R> best{R(-1), R(0)};
  int bi = rows;
  for (int r = j + tid; r < rows; r += bd) {
    const Mag<R> v = mag2(P[(long long)r * w + jj]);
    if (better(v, r, best, bi)) {
      best = v;
      bi = r;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const Mag<R> ov{__shfl_down_sync(0xffffffffu, best.hi, off),
                    __shfl_down_sync(0xffffffffu, best.lo, off)};
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (better(ov, oi, best, bi)) {
      best = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    sc.sv[wid] = best;
    sc.si[wid] = bi;
  }
  __syncthreads();  // (1)
  Mag<R> b = sc.sv[0];
  int pi = sc.si[0];
  const int nw = bd >> 5;
  for (int k = 1; k < nw; ++k)
    if (better(sc.sv[k], sc.si[k], b, pi)) {
      b = sc.sv[k];
      pi = sc.si[k];
    }
  const int pr = (pi >= rows) ? j : pi;
  // swap rows j <-> pr, keep the unscaled pivot row, copy column jj (as it is after the swap)
  for (int c = tid; c < w; c += bd) {
    const cx<R> a = P[(long long)j * w + c], v = P[(long long)pr * w + c];
    P[(long long)j * w + c] = v;
    P[(long long)pr * w + c] = a;
    prow[c] = v;
    if (c == jj) {
      f[j] = v;
      f[pr] = a;
      sc.d = pivot_recip(v, st);
    }
  }
  for (int r = tid; r < rows; r += bd)
    if (r != j && r != pr) f[r] = P[(long long)r * w + jj];
  __syncthreads();  // (2)
  const cx<R> d = sc.d;
  if (w <= bd) {
    // Thread (r0, c) updates rows r0, r0 + rstep, ...  of column c, four rows per batch with the
    // loads ahead of the stores (P and f are disjoint).  The pivot column (c == jj) starts from 0
    // so that it becomes -f[r] d; row j is computed like the others and then overwritten with the
    // scaled pivot row by the thread that owns it.
    const int c = tid % w;
    const int r0 = tid / w, rstep = bd / w;
    if (r0 < rstep) {
      const bool pcol = (c == jj);
      const cx<R> pj = pcol ? d : prow[c] * d;
      const cx<R> zero = mkc<R>(R(0), R(0));
      int r = r0;
      for (; r + 3 * rstep < rows; r += 4 * rstep) {
        cx<R> v[4], fr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u] = P[(long long)(r + u * rstep) * w + c];
          fr[u] = f[r + u * rstep];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          cx<R> x = pcol ? zero : v[u];
          x.re = x.re - (fr[u].re * pj.re - fr[u].im * pj.im);
          x.im = x.im - (fr[u].re * pj.im + fr[u].im * pj.re);
          P[(long long)(r + u * rstep) * w + c] = x;
        }
      }
      for (; r < rows; r += rstep) {
        const cx<R> fr = f[r];
        cx<R> x = pcol ? zero : P[(long long)r * w + c];
        x.re = x.re - (fr.re * pj.re - fr.im * pj.im);
        x.im = x.im - (fr.re * pj.im + fr.im * pj.re);
        P[(long long)r * w + c] = x;
      }
      if (j % rstep == r0) P[(long long)j * w + c] = pj;
    }
  } else {
    for (int r = 0; r < rows; ++r) {
      const cx<R> fr = f[r];
      for (int c = tid; c < w; c += bd) {
        const cx<R> pj = (c == jj) ? d : prow[c] * d;
        cx<R>* e = P + (long long)r * w + c;
        if (r == j) {
          *e = pj;
        } else if (c == jj) {
          *e = mkc<R>(R(0), R(0)) - fr * d;
        } else {
          cx<R> v = *e;
          v.re = v.re - (fr.re * pj.re - fr.im * pj.im);
          v.im = v.im - (fr.re * pj.im + fr.im * pj.re);
          *e = v;
        }
      }
    }
  }
  __syncthreads();  // (3)
  return pr;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_gj_small(int n, BM<R> Mm, BM<R> X, int32_t* status,
                                                       const int32_t* active) {
  const int p = blockIdx.x;
  if (active && !active[p]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* A = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* f = A + (size_t)n * n;
  cx<R>* prow = f + n;
  int* perm = reinterpret_cast<int*>(prow + n);
  int* src = perm + n;
  __shared__ GjScratch<R> sc;
  int32_t* st = status ? status + p : nullptr;
  const cx<R>* m = bat(Mm, p);
  for (int r = 0; r < n; ++r)
    for (int c = threadIdx.x; c < n; c += blockDim.x) A[r * n + c] = m[(long long)r * Mm.ld + c];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int pr = gj_column(A, n, n, j, j, f, prow, sc, st);
    if (threadIdx.x == 0) perm[j] = pr;
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
  for (int r = 0; r < n; ++r)
    for (int c = threadIdx.x; c < n; c += blockDim.x)
      x[(long long)r * X.ld + c] = A[r * n + src[c]];
}

// Panel step of the blocked form: columns [k0, k0 + w) of A (n x n, in global memory).
// The panel is eliminated in shared memory; then, for the columns outside the panel, one pass
// per column (each column owned by one thread, so no barrier) moves the swapped rows to their
// final place, copies the pivot rows into T and zeroes them in A.  The row swaps of the panel
// only ever move a panel row's content to an outside row, so reading all sources before any
// panel row is cleared is enough to apply them at once.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_gj_panel(int n, int k0, int w, int nb, BM<R> Am,
                                                       cx<R>* U, cx<R>* T, int32_t* piv,
                                                       int32_t* status, const int32_t* active) {
  const int p = blockIdx.x;
  if (active && !active[p]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* P = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* f = P + (size_t)n * w;
  cx<R>* prow = f + n;
  int* cont = reinterpret_cast<int*>(prow + w);  // [n] source row of each row's final content
  int* spv = cont + n;                           // [w] pivot rows of this panel
  __shared__ GjScratch<R> sc;
  int32_t* st = status ? status + p : nullptr;
  cx<R>* a = bat(Am, p);
  const long long ld = Am.ld;
  int32_t* pv = piv + (long long)p * n;
  {
    // the panel columns, eight rows per batch with the loads ahead of the stores
    const int c = threadIdx.x % w, r0 = threadIdx.x / w, rs = blockDim.x / w;
    if (r0 < rs)
      for (int rb = r0; rb < n; rb += 8 * rs) {
        cx<R> v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (rb + u * rs < n) v[u] = a[(long long)(rb + u * rs) * ld + k0 + c];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (rb + u * rs < n) P[(long long)(rb + u * rs) * w + c] = v[u];
      }
  }
  for (int r = threadIdx.x; r < n; r += blockDim.x) cont[r] = r;
  __syncthreads();
  for (int jj = 0; jj < w; ++jj) {
    const int j = k0 + jj;
    const int pr = gj_column(P, n, w, j, jj, f, prow, sc, st);
    if (threadIdx.x == 0) {
      pv[j] = pr;
      spv[jj] = pr;
      const int t = cont[j];
      cont[j] = cont[pr];
      cont[pr] = t;
    }
  }
  __syncthreads();
  cx<R>* Tp = T + (long long)p * nb * n;
  const cx<R> zero = mkc<R>(R(0), R(0));
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    if (c >= k0 && c < k0 + w) {
      for (int jj = 0; jj < w; ++jj) Tp[(long long)jj * n + c] = zero;
      continue;
    }
    // (1) final pivot rows -> T, read before anything of this column is written
    for (int j0 = 0; j0 < w; j0 += 8) {
      cx<R> v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < w) v[u] = a[(long long)cont[k0 + j0 + u] * ld + c];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < w) Tp[(long long)(j0 + u) * n + c] = v[u];
    }
    // (2) rows below the panel that took part in a swap receive a panel row's content (all
    // sources are panel rows, read before any is cleared; loads batched ahead of the stores)
    for (int j0 = 0; j0 < w; j0 += 8) {
      cx<R> v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < w && spv[j0 + u] >= k0 + w)
          v[u] = a[(long long)cont[spv[j0 + u]] * ld + c];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < w && spv[j0 + u] >= k0 + w) a[(long long)spv[j0 + u] * ld + c] = v[u];
    }
    // (3) the pivot rows are cleared outside the panel
    for (int jj = 0; jj < w; ++jj) a[(long long)(k0 + jj) * ld + c] = zero;
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

// Trailing update of a Gauss-Jordan panel step: C += U T for every item, with U the eliminated
// panel (n x w, row stride nb), T the pivot rows (w x n) and w <= kMaxPanel (FP32 only: the
// FP64 blocks would not fit the static shared memory).  An 80 x 80 block of C per CTA (n = 400
// is 5 x 5 blocks with no padding; 64 x 64 blocks would pad it to 448^2, 25 % more work), each
// thread 5 x 5 complex accumulators: rows ty + 16 i, columns tx + 16 j.  The whole U and T blocks
// are staged in shared memory at once (one barrier), and C is read into the accumulators before
// the multiply-adds so that its latency overlaps the staging.
constexpr int kMaxPanel = 32;
constexpr int kUpdTile = 80;
template <typename R>
__global__ void __launch_bounds__(256) k_gj_update(int n, int w, int nb, const cx<R>* U,
                                                   const cx<R>* T, BM<R> C,
                                                   const int32_t* active) {
  const int p = blockIdx.z;
  if (active && !active[p]) return;
  __shared__ cx<R> Us[kUpdTile][kMaxPanel + 1];  // row-major like U; padded rows
  __shared__ cx<R> Ts[kMaxPanel][kUpdTile];
  const int m0 = blockIdx.y * kUpdTile, n0 = blockIdx.x * kUpdTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const cx<R>* u = U + (long long)p * n * nb;
  const cx<R>* t = T + (long long)p * nb * n;
  cx<R>* c = bat(C, p);
  const cx<R> zero = mkc<R>(R(0), R(0));
  cx<R> acc[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int r = m0 + ty + 16 * i, col = n0 + tx + 16 * j;
      acc[i][j] = (r < n && col < n) ? c[(long long)r * C.ld + col] : zero;
    }
  // staging: slot e of U is (row e / 32, column e % 32), of T (row e / 80, column e % 80); all
  // loads are issued before the first shared-memory store
  constexpr int kPer = kMaxPanel * kUpdTile / 256;  // 10
  cx<R> us[kPer], ts[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = threadIdx.x + 256 * q;
    const int r = e >> 5, k = e & 31;
    us[q] = (k < w && m0 + r < n) ? u[(long long)(m0 + r) * nb + k] : zero;
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = threadIdx.x + 256 * q;
    const int k = e / kUpdTile, col = e % kUpdTile;
    ts[q] = (k < w && n0 + col < n) ? t[(long long)k * n + n0 + col] : zero;
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = threadIdx.x + 256 * q;
    Us[e >> 5][e & 31] = us[q];
    Ts[e / kUpdTile][e % kUpdTile] = ts[q];
  }
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    cx<R> av[5], bv[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) av[i] = Us[ty + 16 * i][k];
#pragma unroll
    for (int j = 0; j < 5; ++j) bv[j] = Ts[k][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int j = 0; j < 5; ++j) cfma(acc[i][j], av[i], bv[j]);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int r = m0 + ty + 16 * i, col = n0 + tx + 16 * j;
      if (r < n && col < n) c[(long long)r * C.ld + col] = acc[i][j];
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

static size_t small_smem(int n, int elem_bytes) {
  return (size_t)n * n * elem_bytes + 2 * (size_t)n * elem_bytes + 2 * n * sizeof(int);
}
static size_t panel_smem(int n, int w, int elem_bytes) {
  return (size_t)n * w * elem_bytes + (size_t)n * elem_bytes + (size_t)w * elem_bytes +
         (size_t)(n + w) * sizeof(int);
}

bool gj_fits_small(int n, int elem_bytes) { return small_smem(n, elem_bytes) <= kSmemBudget; }

bool gj_supports(int n, int elem_bytes) {
  // the panel kernel holds n x nb panel values, the pivot column and the row map in shared
  // memory (nb = 1 at worst), and the final unpermutation n row indices
  if (n < 1) return false;
  if (gj_fits_small(n, elem_bytes)) return true;
  return panel_smem(n, gj_panel_width(n, elem_bytes), elem_bytes) <= kSmemBudget + 1024 &&
         (size_t)n * sizeof(int) <= 48 * 1024;
}


int gj_panel_width(int n, int elem_bytes) {
  size_t per_col = (size_t)n * elem_bytes + elem_bytes + sizeof(int);
  size_t fixed = (size_t)n * (elem_bytes + sizeof(int));
  int w = fixed >= kSmemBudget ? 1 : (int)std::min<size_t>(32, (kSmemBudget - fixed) / per_col);
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
    size_t smem = small_smem(n, eb);
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
    size_t smem = panel_smem(n, w, eb);
    prof_begin(s, PROF_GJ_PANEL);
    k_gj_panel<R><<<P, kThreads, smem, s>>>(n, k0, w, nb, M, U, T, piv, status, active);
    prof_end(s, PROF_GJ_PANEL);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if constexpr (std::is_same<R, float>::value) {
      // FP32: panels are at most kMaxPanel wide (gj_panel_width); FP64 is FMA-bound either way
      k_gj_update<R><<<dim3((n + kUpdTile - 1) / kUpdTile, (n + kUpdTile - 1) / kUpdTile, P),
                       256, 0, s>>>(n, w, nb, U, T, M, active);
      count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
      BMc<R> Ua{U, (long long)n * nb, nullptr, nb};
      BMc<R> Ta{T, (long long)nb * n, nullptr, n};
      BMc<R> none{nullptr, 0, nullptr, 0};
      e = gemm_simt<R>(s, P, n, n, w, mkc<double>(1.0, 0.0), Ua, OP_N, Ta, OP_N,
                       mkc<double>(1.0, 0.0), M, mkc<double>(0.0, 0.0), none, active);
      if (e != cudaSuccess) return e;
    }
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
