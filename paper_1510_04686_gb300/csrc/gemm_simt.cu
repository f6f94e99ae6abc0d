// Batched complex GEMM on the CUDA cores.  This is the arithmetic of the plain FP64 form of
// the recursive Green's function sweeps (Eqs. 1-2 evaluated block by block): every product
// of two b x b blocks of G, g, H or Sigma goes through here when precision == FP64.
#include "common.cuh"
#include "profile.cuh"

namespace negf {

namespace {

constexpr int BMT = 64;  // tile rows
constexpr int BNT = 64;  // tile cols
constexpr int BKT = 8;   // k chunk
constexpr int TY = 16, TX = 16;  // 256 threads, 4 x 4 outputs each

template <typename R>
__device__ __forceinline__ cx<R> load_op(const cx<R>* a, int ld, int op, int r, int c, int rows,
                                         int cols) {
  // element (r, c) of op(A) where op(A) has shape rows x cols
  if (r >= rows || c >= cols) return mkc<R>(R(0), R(0));
  if (op == OP_N) return a[(long long)r * ld + c];
  cx<R> v = a[(long long)c * ld + r];
  if (op == OP_C) v.im = -v.im;
  return v;
}

template <typename R>
__global__ void __launch_bounds__(256) k_gemm_simt(int M, int N, int K, z64 alpha, BMc<R> A,
                                                   int opA, BMc<R> B, int opB, z64 beta, BM<R> C,
                                                   z64 gamma, BMc<R> D,
                                                   const int32_t* active) {
  const int p = blockIdx.z;
  if (active && !active[p]) return;
  __shared__ cx<R> As[BKT][BMT];
  __shared__ cx<R> Bs[BKT][BNT];
  const cx<R>* a = bat(A, p);
  const cx<R>* b = bat(B, p);
  const int m0 = blockIdx.y * BMT, n0 = blockIdx.x * BNT;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  cx<R> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mkc<R>(R(0), R(0));

  for (int k0 = 0; k0 < K; k0 += BKT) {
    // 512 elements of each tile, 2 per thread
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int id = threadIdx.x + e * 256;
      // A tile: (m, k) -> As[k][m]; walk m fastest for op T/C coalescing, k fastest for N
      int mm, kk;
      if (opA == OP_N) {
        kk = id % BKT;
        mm = id / BKT;
      } else {
        mm = id % BMT;
        kk = id / BMT;
      }
      As[kk][mm] = load_op(a, A.ld, opA, m0 + mm, k0 + kk, M, K);
      int nn, kb;
      if (opB == OP_N) {
        nn = id % BNT;
        kb = id / BNT;
      } else {
        kb = id % BKT;
        nn = id / BKT;
      }
      Bs[kb][nn] = load_op(b, B.ld, opB, k0 + kb, n0 + nn, K, N);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKT; ++kk) {
      cx<R> av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + TY * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + TX * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], av[i], bv[j]);
    }
    __syncthreads();
  }
  cx<R>* c = bat(C, p);
  const cx<R>* d = D.p ? bat(D, p) : nullptr;
  const cx<R> al = mkc<R>(R(alpha.re), R(alpha.im));
  const cx<R> be = mkc<R>(R(beta.re), R(beta.im));
  const cx<R> ga = mkc<R>(R(gamma.re), R(gamma.im));
  const bool use_beta = (beta.re != 0.0 || beta.im != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = m0 + ty + TY * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int col = n0 + tx + TX * j;
      if (col >= N) continue;
      cx<R> v = al * acc[i][j];
      cx<R>* cp = c + (long long)r * C.ld + col;
      if (use_beta) v = v + be * (*cp);
      if (d) v = v + ga * d[(long long)r * D.ld + col];
      *cp = v;
    }
  }
}

}  // namespace

template <typename R>
cudaError_t gemm_simt(cudaStream_t s, int P, int M, int N, int K, z64 alpha, BMc<R> A, int opA,
                      BMc<R> B, int opB, z64 beta, BM<R> C, z64 gamma, BMc<R> D,
                      const int32_t* active) {
  if (P <= 0 || M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + BNT - 1) / BNT, (M + BMT - 1) / BMT, P);
  k_gemm_simt<R><<<grid, 256, 0, s>>>(M, N, K, alpha, A, opA, B, opB, beta, C, gamma, D, active);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t gemm_simt<double>(cudaStream_t, int, int, int, int, z64, BMc<double>, int,
                                       BMc<double>, int, z64, BM<double>, z64, BMc<double>,
                                       const int32_t*);
template cudaError_t gemm_simt<float>(cudaStream_t, int, int, int, int, z64, BMc<float>, int,
                                      BMc<float>, int, z64, BM<float>, z64, BMc<float>,
                                      const int32_t*);

}  // namespace negf
