// Tensor-core complex GEMM (tcgen05 + TMA + TMEM) with exact split-BF16 slices.
// See tc_gemm.cuh for the arithmetic; this file holds the slicing kernels, the MMA kernel and
// the host launcher.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "profile.cuh"
#include "tc_gemm.cuh"

namespace negf {
namespace {

constexpr int kBM = 128;      // tile rows = TMEM lanes
constexpr int kKC = 64;       // real K elements per stage (128 bytes of BF16 per row)
constexpr int kStages = 4;
constexpr int kMaxItems = 96;
constexpr int kThreads = 192;  // warps 0-3 epilogue, warp 4 TMA producer, warp 5 MMA issuer
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on every device wait

struct Item {
  int8_t acc, s, t0, nt;  // accumulator group, A slice, first B slice, number of B slices
};
struct Sched {
  int n_items;
  int n_acc;
  Item it[kMaxItems];
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the time limit passed or another role raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > kWaitNs) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// K-major operand tile, rows of 128 bytes, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
// kind::f16 instruction descriptor: BF16 x BF16 -> F32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ slicing kernels
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ z64 opelem(const z64* a, int ld, int op, int r, int c) {
  if (op == OP_N) return a[(long long)r * ld + c];
  z64 v = a[(long long)c * ld + r];
  if (op == OP_C) v.im = -v.im;
  return v;
}

// |x| as an ordered integer (the bit pattern without the sign)
__device__ __forceinline__ unsigned long long absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// exponent e with max|x| < 2^e (0 for an all-zero row)
__device__ __forceinline__ int scale_exp(double mx) {
  if (!(mx > 0.0)) return 0;
  int e;
  frexp(mx, &e);
  return e;
}

// S fixed-point slices of x * 2^-e (|.| < 1): slice s holds q_s 2^(-beta s) with integer q_s,
// |q_1| <= 2^beta, |q_s| <= 2^(beta-1) afterwards, so that every slice is exact in BF16.
// Integer arithmetic only: |x| 2^(62-e) as a 62-bit fixed-point number, then rounded base-2^beta
// digits taken from the top.
__device__ __forceinline__ void cut(double x, int e, int S, int beta, float* out) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  if (ex) mant |= 1ull << 52;
  const int sh = (ex ? ex : 1) - 1075 + 62 - e;  // |x| 2^(62-e) = mant 2^sh
  long long R;
  if (mant == 0 || sh <= -64) {
    R = 0;
  } else if (sh >= 0) {
    R = (long long)(mant << sh);
  } else {
    const int r = -sh;
    R = (long long)((mant + (1ull << (r - 1))) >> r);
  }
  const bool neg = (u >> 63) != 0;
  float scale = 1.0f;
  const float step = __int_as_float((127 - beta) << 23);  // 2^-beta
  for (int s = 0; s < S; ++s) {
    const int shs = 62 - beta * (s + 1);
    const long long q = (R + (1ll << (shs - 1))) >> shs;
    R -= q << shs;
    const float v = (float)q * scale;
    out[s] = neg ? -v : v;
    scale *= step;
  }
}

constexpr int kMaxS = 12;

// A' rows: [Re, Im] interleaved along K.  One warp per row of op(A).
__global__ void k_slice_a(int M, int K, int L, int S, int beta, BMc<double> A, int opA,
                          __nv_bfloat16* out, int32_t* eo, const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x * (blockDim.x >> 5) + w;
  if (m >= M) return;
  const z64* a = bat(A, p);
  unsigned long long mb = 0;
  for (int k = lane; k < K; k += 32) {
    z64 v = opelem(a, A.ld, opA, m, k);
    mb = max(mb, absbits(v.re));
    mb = max(mb, absbits(v.im));
  }
  mb = warp_max(mb);
  const int e = scale_exp(__longlong_as_double((long long)mb));
  if (lane == 0) eo[(long long)p * M + m] = e;
  float sr[kMaxS], si[kMaxS];
  for (int k2 = lane; k2 < L / 2; k2 += 32) {
    z64 v = (k2 < K) ? opelem(a, A.ld, opA, m, k2) : mkc(0.0, 0.0);
    cut(v.re, e, S, beta, sr);
    cut(v.im, e, S, beta, si);
    for (int s = 0; s < S; ++s) {
      __nv_bfloat162 pr;
      pr.x = __float2bfloat16_rn(sr[s]);
      pr.y = __float2bfloat16_rn(si[s]);
      reinterpret_cast<__nv_bfloat162*>(out + (((long long)p * S + s) * M + m) * L)[k2] = pr;
    }
  }
}

// B'^T rows 2n (= [Re, -Im]) and 2n + 1 (= [Im, Re]) from column n of op(B).
__global__ void k_slice_b(int K, int N, int L, int S, int beta, BMc<double> B, int opB,
                          __nv_bfloat16* out, int32_t* fo, const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = blockIdx.x * (blockDim.x >> 5) + w;
  if (n >= N) return;
  const z64* b = bat(B, p);
  unsigned long long mb = 0;
  for (int k = lane; k < K; k += 32) {
    z64 v = opelem(b, B.ld, opB, k, n);
    mb = max(mb, absbits(v.re));
    mb = max(mb, absbits(v.im));
  }
  mb = warp_max(mb);
  const int f = scale_exp(__longlong_as_double((long long)mb));
  if (lane == 0) fo[(long long)p * N + n] = f;
  const long long N2 = 2LL * N;
  float sr[kMaxS], si[kMaxS];
  for (int k2 = lane; k2 < L / 2; k2 += 32) {
    z64 v = (k2 < K) ? opelem(b, B.ld, opB, k2, n) : mkc(0.0, 0.0);
    cut(v.re, f, S, beta, sr);
    cut(v.im, f, S, beta, si);
    for (int s = 0; s < S; ++s) {
      __nv_bfloat16* base = out + ((long long)p * S + s) * N2 * L;
      __nv_bfloat162 r0, r1;
      r0.x = __float2bfloat16_rn(sr[s]);
      r0.y = __float2bfloat16_rn(-si[s]);
      r1.x = __float2bfloat16_rn(si[s]);
      r1.y = __float2bfloat16_rn(sr[s]);
      reinterpret_cast<__nv_bfloat162*>(base + (2LL * n) * L)[k2] = r0;
      reinterpret_cast<__nv_bfloat162*>(base + (2LL * n + 1) * L)[k2] = r1;
    }
  }
}

// ------------------------------------------------------------------ MMA kernel
template <int NT, int MAXT>
struct Cfg {
  static constexpr int kATile = kBM * kKC * 2;                // 16 KB
  static constexpr int kBTile = NT * kKC * 2;
  static constexpr int kStage = kATile + MAXT * kBTile;
  static constexpr int kSmem = kStages * kStage + 1024 + 256;  // + alignment + barriers
};

template <int NT, int MAXT>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const Sched sched, int M, int N2, int L, int S, int two_beta,
              const int32_t* __restrict__ eA, const int32_t* __restrict__ fB, double* T64,
              z64 alpha, z64 beta, z64 gamma, BM<double> C, BMc<double> D, int add_identity,
              const int32_t* active, int32_t* err) {
  using CF = Cfg<NT, MAXT>;
  const int p = blockIdx.z;
  if (active && !active[p]) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * CF::kStage);
  uint64_t* empty = full + kStages;
  uint64_t* accfull = empty + kStages;
  uint64_t* accempty = accfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * NT, m0 = blockIdx.y * kBM;
  const int nk = L / kKC;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], 4 * 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    // ---------------- TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int ii = 0; ii < sched.n_items && !*abort_flag; ++ii) {
        const Item it = sched.it[ii];
        for (int kc = 0; kc < nk; ++kc) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
          unsigned char* st = smem + stage * CF::kStage;
          mbar_expect_tx(&full[stage], CF::kATile + it.nt * CF::kBTile);
          tma_load_3d(st, &mapA, &full[stage], kc * kKC, m0, p * S + it.s - 1);
          for (int j = 0; j < it.nt; ++j)
            tma_load_3d(st + CF::kATile + j * CF::kBTile, &mapB, &full[stage], kc * kKC, n0,
                        p * S + it.t0 + j - 1);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // drain: wait (bounded) until the loads still in flight have landed
      for (int i = 0; i < kStages; ++i) {
        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, NT);
      int stage = 0;
      uint32_t phase = 0;
      int cur = -1;
      uint32_t acc_on = 0;
      for (int ii = 0; ii < sched.n_items && !*abort_flag; ++ii) {
        const Item it = sched.it[ii];
        const int buf = it.acc & 1;
        if (it.acc != cur) {
          cur = it.acc;
          acc_on = 0;
          if (cur >= 2) {
            if (!mbar_wait(&accempty[buf], ((cur >> 1) - 1) & 1, abort_flag)) break;
            tc_fence_after();
          }
        }
        const uint32_t dcol = tmem + (uint32_t)(buf * NT);
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + stage * CF::kStage);
#pragma unroll
          for (int k = 0; k < kKC / 16; ++k) {
            const uint64_t ad = sw128_desc(a0 + 32 * k);
            for (int j = 0; j < it.nt; ++j) {
              const uint64_t bd = sw128_desc(a0 + CF::kATile + j * CF::kBTile + 32 * k);
              mma_bf16(dcol, ad, bd, idesc, acc_on);
              acc_on = 1;
            }
          }
          mma_commit(&empty[stage]);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        const bool last_of_acc = (ii + 1 == sched.n_items) || (sched.it[ii + 1].acc != cur);
        if (last_of_acc) mma_commit(&accfull[buf]);
      }
    }
  } else {
    // ---------------- epilogue (warps 0-3 own TMEM lanes 32 w .. 32 w + 31)
    // Every group value is exact in FP32; the running sum over groups is kept as an unevaluated
    // pair hi + lo of FP32 numbers (TwoSum, renormalised), so FP64 arithmetic is needed only
    // once per output, when the pair is scaled back and combined with C and D.
    const int r = warp * 32 + lane;
    const int m = m0 + r;
    const bool row_ok = m < M;
    const int em = row_ok ? eA[(long long)p * M + m] : 0;
    const int N = N2 >> 1;
    float2* trow = reinterpret_cast<float2*>(T64) + ((long long)p * M + (row_ok ? m : 0)) * N2;
    z64* crow = row_ok ? bat(C, p) + (long long)m * C.ld : nullptr;
    const z64* drow = (row_ok && D.p) ? bat(D, p) + (long long)m * D.ld : nullptr;
    const bool use_beta = (beta.re != 0.0 || beta.im != 0.0);
    const bool unit_alpha = (alpha.re == 1.0 && alpha.im == 0.0);
    const bool unit_gamma = (gamma.re == 1.0 && gamma.im == 0.0);
    for (int acc = 0; acc < sched.n_acc; ++acc) {
      const int buf = acc & 1;
      if (!mbar_wait(&accfull[buf], (acc >> 1) & 1, abort_flag)) break;
      tc_fence_after();
      const bool last = (acc == sched.n_acc - 1);
      for (int c0 = 0; c0 < NT; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * NT + c0), v);
        if (!row_ok) continue;
        float lv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col >= N2) break;
          float hi = v[j], lo = 0.0f;
          if (acc > 0) {
            const float2 t = trow[col];
            const float s1 = t.x + v[j];
            const float bp = s1 - t.x;
            const float err = (t.x - (s1 - bp)) + (v[j] - bp);
            const float l1 = t.y + err;
            hi = s1 + l1;
            lo = l1 - (hi - s1);
          }
          if (!last) trow[col] = make_float2(hi, lo);
          v[j] = hi;
          lv[j] = lo;
        }
        if (last) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int col = n0 + c0 + j;
            if (col >= N2) break;
            const int n = col >> 1;
            const double sc = ldexp(1.0, em + fB[(long long)p * N + n] - two_beta);
            z64 t = mkc(((double)v[j] + (double)lv[j]) * sc, ((double)v[j + 1] + (double)lv[j + 1]) * sc);
            z64 o = unit_alpha ? t : alpha * t;
            if (use_beta) o = o + beta * crow[n];
            if (drow) o = o + (unit_gamma ? drow[n] : gamma * drow[n]);
            if (add_identity && n == m) o.re += 1.0;
            crow[n] = o;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&accempty[buf]);
    }
  }
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag && err) atomicExch(err, 1);
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, void* base, int L, int rows, long long zdim, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)rows, (cuuint64_t)zdim};
  cuuint64_t strides[2] = {(cuuint64_t)L * 2, (cuuint64_t)L * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)kKC, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Every order d = s + t - 1 <= S is its own exact accumulator group; within a group each
// (s, t) product is one item (A slice s, B slice t).
Sched build_sched(int S, int maxt) {
  Sched sc;
  std::memset(&sc, 0, sizeof(sc));
  (void)maxt;
  int n = 0;
  for (int d = 1; d <= S; ++d)
    for (int s = 1; s <= d && n < kMaxItems; ++s)
      sc.it[n++] = Item{(int8_t)(d - 1), (int8_t)s, (int8_t)(d + 1 - s), (int8_t)1};
  sc.n_items = n;
  sc.n_acc = S;
  return sc;
}

template <int NT, int MAXT>
cudaError_t launch_tc(cudaStream_t s, int P, int M, int N2, int K, int L, int S, int two_beta,
                      const CUtensorMap& mA, const CUtensorMap& mB, const TcWs& ws, z64 alpha,
                      z64 beta, z64 gamma, BM<double> C, BMc<double> D, bool add_identity,
                      const int32_t* active) {
  using CF = Cfg<NT, MAXT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<NT, MAXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, CF::kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  Sched sc = build_sched(S, MAXT);
  dim3 grid((N2 + NT - 1) / NT, (M + kBM - 1) / kBM, P);
  {
    const double alg = 8.0 * M * (N2 / 2) * (double)K * P;
    const double hw = 2.0 * grid.y * kBM * (double)grid.x * NT * L * sc.n_items * P;
    prof_flops(PROF_TC_GEMM, alg, hw);
  }
  prof_begin(s, PROF_TC_GEMM);
  k_tc_gemm<NT, MAXT><<<grid, kThreads, CF::kSmem, s>>>(
      mA, mB, sc, M, N2, L, S, two_beta, ws.expA, ws.expB, ws.T64, alpha, beta, gamma, C, D,
      add_identity ? 1 : 0, active, ws.err);
  prof_end(s, PROF_TC_GEMM);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

void tc_plan(int K, int* beta, int* S) {
  // Slice width beta and count S = ceil(48 / beta) such that every order group stays exact:
  // the integer sum of group d over the 2K real terms is below 2K 2^(2 beta) (1 + (d-2)/4),
  // which must not exceed 2^24 for d = S.
  const double K2 = 2.0 * std::max(K, 1);
  int b = 8;
  for (; b > 1; --b) {
    const int s = std::min(kMaxS, (48 + b - 1) / b);
    const double grow = 1.0 + std::max(0, s - 2) / 4.0;
    if (K2 * std::ldexp(1.0, 2 * b) * grow <= 16777216.0) break;
  }
  *beta = b;
  *S = std::min(kMaxS, (48 + b - 1) / b);
}

size_t tc_ws_bytes(int P, int M, int N, int K) {
  size_t off = 0;
  TcWs w;
  tc_ws_carve(nullptr, off, P, M, N, K, w);
  return off;
}

void tc_ws_carve(char* base, size_t& off, int P, int M, int N, int K, TcWs& w) {
  int beta, S;
  tc_plan(K, &beta, &S);
  const size_t L = (size_t)round_up(2 * K, kKC);
  auto take = [&](size_t bytes) -> void* {
    size_t a = (off + 1023) & ~size_t(1023);
    off = a + bytes;
    return base ? base + a : nullptr;
  };
  w.slicesA = take((size_t)P * S * M * L * 2);
  w.slicesB = take((size_t)P * S * 2 * N * L * 2);
  w.expA = static_cast<int32_t*>(take((size_t)P * M * 4));
  w.expB = static_cast<int32_t*>(take((size_t)P * N * 4));
  w.T64 = static_cast<double*>(take((size_t)P * M * 2 * N * 8));
  w.err = static_cast<int32_t*>(take(256));
}

cudaError_t tc_gemm(cudaStream_t s, int P, int M, int N, int K, z64 alpha, BMc<double> A,
                    int opA, BMc<double> B, int opB, z64 beta, BM<double> C, z64 gamma,
                    BMc<double> D, bool add_identity, const int32_t* active, const TcWs& ws) {
  if (P <= 0 || M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  int bta, S;
  tc_plan(K, &bta, &S);
  const int L = round_up(2 * K, kKC);
  const int N2 = 2 * N;
  __nv_bfloat16* sa = static_cast<__nv_bfloat16*>(ws.slicesA);
  __nv_bfloat16* sb = static_cast<__nv_bfloat16*>(ws.slicesB);
  prof_begin(s, PROF_SLICE);
  k_slice_a<<<dim3((M + 7) / 8, P), 256, 0, s>>>(M, K, L, S, bta, A, opA, sa, ws.expA, active);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_slice_b<<<dim3((N + 7) / 8, P), 256, 0, s>>>(K, N, L, S, bta, B, opB, sb, ws.expB, active);
  prof_end(s, PROF_SLICE);
  count_launch(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // tile width: least padding of the 2N real columns, wider on ties
  static const int widths[5] = {256, 224, 192, 160, 128};
  int best = 128;
  long long best_pad = -1;
  for (int wdt : widths) {
    long long pad = (long long)((N2 + wdt - 1) / wdt) * wdt;
    if (best_pad < 0 || pad < best_pad) {
      best_pad = pad;
      best = wdt;
    }
  }
  CUtensorMap mA, mB;
  if (!make_map(&mA, sa, L, M, (long long)P * S, kBM)) return cudaErrorInvalidValue;
  if (!make_map(&mB, sb, L, N2, (long long)P * S, best)) return cudaErrorInvalidValue;
  switch (best) {
    case 256: return launch_tc<256, 1>(s, P, M, N2, K, L, S, 2 * bta, mA, mB, ws, alpha, beta, gamma, C, D, add_identity, active);
    case 224: return launch_tc<224, 1>(s, P, M, N2, K, L, S, 2 * bta, mA, mB, ws, alpha, beta, gamma, C, D, add_identity, active);
    case 192: return launch_tc<192, 1>(s, P, M, N2, K, L, S, 2 * bta, mA, mB, ws, alpha, beta, gamma, C, D, add_identity, active);
    case 160: return launch_tc<160, 1>(s, P, M, N2, K, L, S, 2 * bta, mA, mB, ws, alpha, beta, gamma, C, D, add_identity, active);
    default: return launch_tc<128, 1>(s, P, M, N2, K, L, S, 2 * bta, mA, mB, ws, alpha, beta, gamma, C, D, add_identity, active);
  }
}

}  // namespace negf
