// Tensor-core complex GEMM (tcgen05 + TMA + TMEM) with exact split-BF16 slices.
// See tc_gemm.cuh for the arithmetic; this file holds the slicing kernels, the MMA kernel and
// the host launcher.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <type_traits>
#include <vector>

#include "profile.cuh"
#include "tc_gemm.cuh"
#include "tc_slice.cuh"

namespace negf {
namespace {

constexpr int kBM = 128;      // tile rows = TMEM lanes
constexpr int kKC = 64;       // real K elements per stage (128 bytes of BF16 per row)
constexpr int kMaxItems = 240;
constexpr int kThreads = 320;  // warps 0-7 epilogue, warp 8 TMA producer, warp 9 MMA issuer
constexpr int kEpiWarps = 8;
constexpr int kNT = 128;       // tile columns (real)
constexpr int kAccBufs = 2;    // TMEM: 2 accumulators + the hi and lo words of the running sums
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on every device wait

constexpr int kMaxParts = 8;
struct Item {
  uint8_t acc;          // exact accumulator group
  int8_t s, t, kp;      // A slice, B slice (1-based), K part
};
struct Sched {
  int n_items;
  int n_acc;
  int part_lo[kMaxParts];  // first K chunk of each part
  int part_hi[kMaxParts];  // one past the last K chunk
  Item it[kMaxItems];      // grouped: the items of one accumulator group are consecutive
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

// 32 consecutive TMEM columns of this warp's lane quarter, no wait (tcgen05.wait::ld follows)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32"
      " {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32"
      " [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
// 16 consecutive TMEM columns of this warp's lane quarter
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32"
      " [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}
// 8 consecutive TMEM columns of this warp's lane quarter
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                   taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
               "r"(r[7])
               : "memory");
}
template <int W>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* r) {
  if constexpr (W == 32)
    tmem_ld32(taddr, r);
  else if constexpr (W == 16)
    tmem_ld16(taddr, r);
  else
    tmem_ld8(taddr, r);
}
template <int W>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t* r) {
  if constexpr (W == 32)
    tmem_st32(taddr, r);
  else if constexpr (W == 16)
    tmem_st16(taddr, r);
  else
    tmem_st8(taddr, r);
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// (double)x * 2^k from the bit pattern of the FP32 number x with integer operations only
// (exact; x normal or zero, result in the normal double range).  FP64 arithmetic is scarce on
// this GPU, so the epilogue converts without cvt/mul.
__device__ __forceinline__ double f32_scaled(uint32_t xb, int k) {
  const uint32_t ex = (xb >> 23) & 0xFFu;
  if (ex == 0u) return 0.0;  // zero (FP32 subnormals do not occur: slices are integers x 2^-n)
  const unsigned long long sign = (unsigned long long)(xb >> 31) << 63;
  const unsigned long long e64 = (unsigned long long)(ex + (1023 - 127) + k) << 52;
  const unsigned long long man = (unsigned long long)(xb & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | e64 | man));
}


// Flops of the launches made while profiling is on: [0] algorithmic complex 8 M N K of the
// active items, [1] issued BF16 MMA flops (padded tiles, computed slice products).
__device__ double g_tc_prof[2];

// A scalar coefficient of the epilogue, by the work it needs: 0 zero, 1 one, 2 minus one (sign
// flips only), 3 real (two multiplies), 4 complex.  FP64 throughput is a small fraction of
// FP32's on this GPU, so the final pass spends FP64 operations only where the value needs them.
__device__ __forceinline__ int coef_class(z64 a) {
  if (a.im != 0.0) return 4;
  if (a.re == 0.0) return 0;
  if (a.re == 1.0) return 1;
  if (a.re == -1.0) return 2;
  return 3;
}
__device__ __forceinline__ z64 coef_mul(int cls, z64 a, z64 x) {
  switch (cls) {
    case 1: return x;
    case 2: return mkc(-x.re, -x.im);
    case 3: return mkc(a.re * x.re, a.re * x.im);
    default: return a * x;
  }
}
// |x| of a double as its bit pattern without the sign (orders like |x| for finite values)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// One accumulator group added into the running sums of this warp's TMEM lanes, columns
// [cbase, cbase + NCH FW): the exact FP32 group value v and the unevaluated pair hi + lo
// (TwoSum, renormalised); first = true initialises the pair (hi = v, lo = 0).  Chunk k + 1 is
// loaded from TMEM while chunk k is summed and stored, so the load latency overlaps the adds.
template <int FW, int NCH>
__device__ __forceinline__ void flush_group(bool first, uint32_t tacc, uint32_t thi,
                                            uint32_t tlo, int cbase) {
  uint32_t v[2][FW], h[2][FW], l[2][FW];
  tmem_ld<FW>(tacc + cbase, v[0]);
  if (!first) {
    tmem_ld<FW>(thi + cbase, h[0]);
    tmem_ld<FW>(tlo + cbase, l[0]);
  }
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    tmem_ld_wait();  // chunk k has landed (the only load in flight)
    if (k + 1 < NCH) {
      const uint32_t c = (uint32_t)(cbase + (k + 1) * FW);
      tmem_ld<FW>(tacc + c, v[nxt]);
      if (!first) {
        tmem_ld<FW>(thi + c, h[nxt]);
        tmem_ld<FW>(tlo + c, l[nxt]);
      }
    }
    if (first) {
#pragma unroll
      for (int j = 0; j < FW; ++j) {
        h[cur][j] = v[cur][j];
        l[cur][j] = 0u;
      }
    } else {
#pragma unroll
      for (int j = 0; j < FW; ++j) {
        const float hj = __uint_as_float(h[cur][j]), vj = __uint_as_float(v[cur][j]);
        const float s1 = hj + vj;
        const float bp = s1 - hj;
        const float e1 = (hj - (s1 - bp)) + (vj - bp);
        const float l1 = __uint_as_float(l[cur][j]) + e1;
        const float h2 = s1 + l1;
        h[cur][j] = __float_as_uint(h2);
        l[cur][j] = __float_as_uint(l1 - (h2 - s1));
      }
    }
    const uint32_t c = (uint32_t)(cbase + k * FW);
    tmem_st<FW>(thi + c, h[cur]);
    tmem_st<FW>(tlo + c, l[cur]);
  }
}

__device__ __forceinline__ float warp_max_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------ MMA kernel
// CG = 1: one CTA computes a 128-row tile with tcgen05.mma.cta_group::1 (M = 128).
// CG = 2: a cluster of two x-adjacent CTAs (consecutive row tiles) computes a 256-row tile with
// tcgen05.mma.cta_group::2 (M = 256) issued by the even CTA: each CTA loads its own 128 rows of
// A and one half of the B tile (NT / 2 rows of the embedded B), so a stage moves 24 KB per CTA
// instead of 32 KB, and each CTA's tensor memory receives the accumulator of its own rows.  Both
// CTAs' loads complete on the even CTA's barrier; the MMA commits arrive on both CTAs' barriers.
constexpr int kStgLd = 9;  // row stride (complex entries) of the final pass's output staging

template <int NT, int STAGES, int CG, int G, int KPS = 1>
struct Cfg {
  static_assert(STAGES % G == 0, "stages are released in whole groups");
  static constexpr int kStages = STAGES;
  static constexpr int kGroups = STAGES / G;                  // stage groups (one commit each)
  static constexpr int kBRows = NT / CG;                      // rows of the B tile this CTA loads
  static constexpr int kABox = kBM * kKC * 2;                 // one K chunk of A: 16 KB
  static constexpr int kBBox = kBRows * kKC * 2;              // one K chunk of B
  static constexpr int kATile = KPS * kABox;                  // a stage holds KPS K chunks
  static constexpr int kBTile = KPS * kBBox;
  static constexpr int kStage = kATile + kBTile;
  // 32 rows x 8 complex outputs, rows padded to 9 entries (144 bytes): a lane's 16-byte writes
  // of its own row then fall in distinct banks across each group of 8 lanes
  static constexpr int kStagingPerWarp = 32 * kStgLd * 16;
  static constexpr int kStaging = kEpiWarps * kStagingPerWarp;
  // the output staging of the tile's final pass reuses the pipeline stages (every MMA and load
  // of the tile has completed by then)
  static_assert(kStaging <= kStages * kStage, "staging fits the stage memory");
  static constexpr int kSmem = kStages * kStage + 1024 + 256;  // + align + barriers
  // barriers (per-chunk full, per-group empty, accumulator full / empty) and four words
  static_assert((kStages * KPS + kGroups + 2 * kAccBufs) * 8 + 16 <= 256, "barrier space");
};

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the variable at local shared address `a` in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}
// TMA load whose completion is counted on an mbarrier of this CTA or of its peer (cta_group::2)
__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t a, uint64_t b,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
// commit of the pair's MMAs, arriving on the barrier at this offset in both CTAs
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
               : "memory");
}

// KPS: K chunks (of 64 BF16 columns) per shared-memory stage; more chunks per stage put more
// MMAs behind each barrier wait and commit of the MMA thread.
template <int NT, int STAGES, int CG, int G, int KPS = 1, int MINB = 1>
__global__ void __launch_bounds__(kThreads, MINB)
    k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const Sched sched, int M, int N2, int S, int two_beta,
              const int32_t* __restrict__ eA, const int32_t* __restrict__ fB,
              const int32_t* __restrict__ zidxA, int zmodeA, const int32_t* __restrict__ zidxB,
              int zmodeB, z64 alpha,
              z64 beta, z64 gamma, BM<double> C, BMc<double> D, int add_identity,
              int trunc_beta, const int32_t* active, int32_t* err, float* rmax, int Kc,
              int count_flops) {
  // TMEM: kAccBufs accumulators + hi / lo sum words, a power of two of columns; two resident
  // CTAs per SM (MINB = 2) must fit the SM's 512 columns together
  constexpr uint32_t kTmemCols = NT * (kAccBufs + 2);
  static_assert(kTmemCols * MINB <= 512 && (kTmemCols & (kTmemCols - 1)) == 0, "TMEM budget");
  // columns per TMEM load of the final pass (and of the two-CTA form's flushes)
  constexpr int CW = 16;
  static_assert((NT / 2) % CW == 0, "epilogue chunks");
  static_assert(CG == 1 || CG == 2, "one CTA or a CTA pair per MMA");
  using CF = Cfg<NT, STAGES, CG, G, KPS>;
  constexpr int kStages = CF::kStages;
  const int p = blockIdx.z;
  // both CTAs of a pair have the same item, so they leave together (before any cluster barrier)
  if (active && !active[p]) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  z64* staging = reinterpret_cast<z64*>(smem);  // the final pass only (see Cfg)
  // one "full" barrier per K chunk of a stage: the MMAs of a chunk start as soon as its own
  // tiles have landed, so a stage's later chunks stream in behind its first MMAs
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * CF::kStage);
  uint64_t* empty = full + kStages * KPS;  // one per group of G stages
  uint64_t* accfull = empty + CF::kGroups;
  uint64_t* accempty = accfull + kAccBufs;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accempty + kAccBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* s_cut = reinterpret_cast<int*>(tmem_slot + 2);
  int* s_nexec = reinterpret_cast<int*>(tmem_slot + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * NT;  // pairs are adjacent along x
  const uint32_t rank = (CG == 2) ? cluster_rank() : 0u;
  const bool leader = (rank == 0);
  // slice set of this batch item: its own (mode 0), the indexed one (1) or the shared one (2)
  const int zA = zmodeA == 0 ? p : (zmodeA == 1 ? zidxA[p] : 0);
  const int zB = zmodeB == 0 ? p : (zmodeB == 1 ? zidxB[p] : 0);

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages * KPS; ++i) mbar_init(&full[i], 1);
    for (int i = 0; i < CF::kGroups; ++i) mbar_init(&empty[i], 1);
    for (int i = 0; i < kAccBufs; ++i) {
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], CG * kEpiWarps);  // one arrival per epilogue warp of the pair
    }
    *abort_flag = 0;
    // Highest slice order this tile computes.  With trunc_beta > 0 the product only has to be
    // accurate relative to |op(A)| rows (it is a small correction added to a term of that size):
    // orders whose terms fall below 2^(-beta S) of the A row scale are dropped, from the largest
    // column exponent f of op(B) over the tile (|B| < 2^f): keep d <= S + ceil(f / beta).
    int cut = S;
    if (trunc_beta > 0) {
      const int Nc = N2 >> 1;
      int fmax = -(1 << 30);
      for (int n = n0 / 2; n < min(Nc, n0 / 2 + NT / 2); ++n)
        fmax = max(fmax, fB[(long long)zB * Nc + n]);
      if (fmax < 0) cut = max(1, S - (-fmax) / trunc_beta);
    }
    *s_cut = cut;
    // accumulator groups this tile computes (a group holds products of one order)
    int nex = 0, prev = -1;
    for (int ii = 0; ii < sched.n_items; ++ii) {
      const Item it = sched.it[ii];
      if (it.s + it.t - 1 <= cut && (int)it.acc != prev) {
        ++nex;
        prev = it.acc;
      }
    }
    *s_nexec = nex;
    if (count_flops) {
      // this CTA's share of the launch (its own 128 rows; in a pair the even CTA's MMAs cover
      // both CTAs' rows): algorithmic complex flops of its outputs and issued BF16 MMA flops
      const int rows = max(0, min(kBM, M - m0));
      const int cols = max(0, min(NT / 2, (N2 >> 1) - n0 / 2));
      double chunks = 0.0;
      for (int ii = 0; ii < sched.n_items; ++ii) {
        const Item it = sched.it[ii];
        if (it.s + it.t - 1 <= cut) chunks += sched.part_hi[it.kp] - sched.part_lo[it.kp];
      }
      atomicAdd(&g_tc_prof[0], 8.0 * rows * cols * (double)Kc);
      atomicAdd(&g_tc_prof[1], 2.0 * kBM * NT * kKC * chunks);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) {
    if constexpr (CG == 2) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)), "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)), "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
  }
  __syncthreads();
  if constexpr (CG == 2) cluster_sync();  // the peer's barriers exist before any remote use
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int cut = *s_cut;
  const int n_exec = *s_nexec;

  if (warp == 8) {
    // ---------------- TMA producer: for every item, the K chunks of its part
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int ii = 0; ii < sched.n_items && !*abort_flag; ++ii) {
        const Item it = sched.it[ii];
        if (it.s + it.t - 1 > cut) continue;
        const int hi = sched.part_hi[it.kp];
        for (int kc = sched.part_lo[it.kp]; kc < hi; kc += KPS) {
          // a group of G stages is released by one MMA commit: wait at the group's first stage
          if (stage % G == 0 && !mbar_wait(&empty[stage / G], phase ^ 1, abort_flag)) break;
          unsigned char* st = smem + stage * CF::kStage;
          const int nch = min(KPS, hi - kc);  // K chunks in this stage
#pragma unroll
          for (int j = 0; j < KPS; ++j) {
            uint64_t* fj = &full[stage * KPS + j];
            if (j >= nch) {
              // no chunk j in this stage: complete the barrier's phase without data, so that
              // it stays in step with the stage's phase
              if (leader) mbar_arrive(fj);
              continue;
            }
            if constexpr (CG == 2) {
              // both CTAs' loads of this chunk complete on the even CTA's barrier
              if (leader) mbar_expect_tx(fj, CG * (CF::kABox + CF::kBBox));
              const uint32_t fb = map_rank(smem_u32(fj), 0);
              tma_load_3d_pair(st + j * CF::kABox, &mapA, fb, (kc + j) * kKC, m0,
                               zA * S + it.s - 1);
              tma_load_3d_pair(st + CF::kATile + j * CF::kBBox, &mapB, fb, (kc + j) * kKC,
                               n0 + (int)rank * CF::kBRows, zB * S + it.t - 1);
            } else {
              mbar_expect_tx(fj, CF::kABox + CF::kBBox);
              tma_load_3d(st + j * CF::kABox, &mapA, fj, (kc + j) * kKC, m0, zA * S + it.s - 1);
              tma_load_3d(st + CF::kATile + j * CF::kBBox, &mapB, fj, (kc + j) * kKC, n0,
                          zB * S + it.t - 1);
            }
          }
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // drain: wait (bounded) until every stage group holding loads was released by the MMAs
      if (stage % G != 0) {
        stage += G - stage % G;
        if (stage == kStages) {
          stage = 0;
          phase ^= 1;
        }
      }
      for (int i = 0; i < CF::kGroups; ++i) {
        if (!mbar_wait(&empty[stage / G], phase ^ 1, abort_flag)) break;
        stage += G;
        if (stage == kStages) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else if (warp == 9) {
    // ---------------- MMA issuer (the even CTA of a pair issues for both)
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_bf16(kBM * CG, NT);
      int stage = 0;
      uint32_t phase = 0;
      int cur = -1, gexec = -1, buf = 0;  // gexec: accumulator groups computed so far
      uint32_t acc_on = 0;
      for (int ii = 0; ii < sched.n_items && !*abort_flag; ++ii) {
        const Item it = sched.it[ii];
        if (it.s + it.t - 1 > cut) continue;
        if (it.acc != cur) {
          cur = it.acc;
          ++gexec;
          buf = gexec % kAccBufs;
          acc_on = 0;
          if (gexec >= kAccBufs) {  // the buffer's previous group must have been read out
            if (!mbar_wait(&accempty[buf], ((gexec / kAccBufs) - 1) & 1, abort_flag)) break;
            tc_fence_after();
          }
        }
        const uint32_t dcol = tmem + (uint32_t)(buf * NT);
        bool ok = true;
        const int hi = sched.part_hi[it.kp];
        for (int kc = sched.part_lo[it.kp]; kc < hi; kc += KPS) {
          const uint32_t a0 = smem_u32(smem + stage * CF::kStage);
          const int nch = min(KPS, hi - kc);
#pragma unroll
          for (int j = 0; j < KPS; ++j) {
            if (j >= nch) break;
            if (!mbar_wait(&full[stage * KPS + j], phase, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t aj = a0 + j * CF::kABox, bj = a0 + CF::kATile + j * CF::kBBox;
#pragma unroll
            for (int k = 0; k < kKC / 16; ++k) {
              if constexpr (CG == 2)
                mma_bf16_pair(dcol, sw128_desc(aj + 32 * k), sw128_desc(bj + 32 * k), idesc,
                              acc_on);
              else
                mma_bf16(dcol, sw128_desc(aj + 32 * k), sw128_desc(bj + 32 * k), idesc, acc_on);
              acc_on = 1;
            }
          }
          if (!ok) break;
          if (stage % G == G - 1) {  // last stage of its group: release the group
            if constexpr (CG == 2)
              mma_commit_pair(&empty[stage / G]);
            else
              mma_commit(&empty[stage / G]);
          }
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        int nx = ii + 1;  // next item that is computed
        while (nx < sched.n_items && sched.it[nx].s + sched.it[nx].t - 1 > cut) ++nx;
        const bool last_of_acc = (nx == sched.n_items) || (sched.it[nx].acc != cur);
        if (last_of_acc) {
          if constexpr (CG == 2)
            mma_commit_pair(&accfull[buf]);
          else
            mma_commit(&accfull[buf]);
        }
      }
      // the last, partly used stage group is released too (the producer's drain waits for it)
      if (!*abort_flag && stage % G != 0) {
        if constexpr (CG == 2)
          mma_commit_pair(&empty[stage / G]);
        else
          mma_commit(&empty[stage / G]);
      }
    }
  } else {
    // ---------------- epilogue: warp w owns TMEM lanes 32 (w % 4) .. + 31 (tile rows) and the
    // 64 columns starting at 64 (w / 4).  Each exact group value is added to a running sum kept
    // in TMEM as an unevaluated pair hi + lo of FP32 numbers (TwoSum, renormalised); FP64 is
    // used once per output at the end.
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;
    const int m = m0 + r;
    const bool row_ok = m < M;
    const int em = row_ok ? eA[(long long)zA * M + m] : 0;
    const int N = N2 >> 1;
    const int32_t* fBp = fB + (long long)zB * N;
    const int cls_alpha = coef_class(alpha), cls_beta = coef_class(beta);
    const int cls_gamma = D.p ? coef_class(gamma) : 0;
    const bool want_max = rmax != nullptr;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int cbase = half * (NT / 2);
    const uint32_t t_hi = tmem + lane_off + kAccBufs * NT, t_lo = t_hi + NT;
    unsigned long long omax = 0ull;  // largest |Re|, |Im| this thread stores (rmax), as bits
    for (int acc = 0; acc < n_exec; ++acc) {
      const int buf = acc % kAccBufs;
      if (!mbar_wait(&accfull[buf], (acc / kAccBufs) & 1, abort_flag)) break;
      tc_fence_after();
      const bool last = (acc == n_exec - 1);
      if (MINB == 1 && !last) {
        flush_group<8, NT / 16>(acc == 0, tmem + lane_off + (uint32_t)(buf * NT), t_hi, t_lo,
                                cbase);
      } else {
      for (int c0 = cbase; c0 < cbase + NT / 2; c0 += CW) {
        uint32_t v[CW], h[CW], l[CW];
        tmem_ld<CW>(tmem + lane_off + (uint32_t)(buf * NT + c0), v);
        if (acc > 0) {
          tmem_ld<CW>(t_hi + c0, h);
          tmem_ld<CW>(t_lo + c0, l);
        }
        tmem_ld_wait();
        if (acc == 0) {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            h[j] = v[j];
            l[j] = 0u;
          }
        } else {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            const float hj = __uint_as_float(h[j]), vj = __uint_as_float(v[j]);
            const float s1 = hj + vj;
            const float bp = s1 - hj;
            const float e1 = (hj - (s1 - bp)) + (vj - bp);
            const float l1 = __uint_as_float(l[j]) + e1;
            const float h2 = s1 + l1;
            h[j] = __float_as_uint(h2);
            l[j] = __float_as_uint(l1 - (h2 - s1));
          }
        }
        if (!last) {
          tmem_st<CW>(t_hi + c0, h);
          tmem_st<CW>(t_lo + c0, l);
        } else {
          // Final value of this row's 16 complex outputs, written through a per-warp staging
          // tile so that C, D and the stores are accessed as contiguous 128-byte row segments.
          z64* stg = staging + warp * (32 * kStgLd);
#pragma unroll
          for (int half8 = 0; half8 < CW / 16; ++half8) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              const int j = 16 * half8 + 2 * jj;
              const int n = (n0 + c0 + j) >> 1;
              const int sh = em + (n < N ? fBp[n] : 0) - two_beta;
              stg[lane * kStgLd + jj] = mkc(f32_scaled(h[j], sh) + f32_scaled(l[j], sh),
                                       f32_scaled(h[j + 1], sh) + f32_scaled(l[j + 1], sh));
            }
            __syncwarp();
            const int nb0 = (n0 + c0) / 2 + 8 * half8;  // first complex column of this piece
#pragma unroll
            for (int it = 0; it < 8; ++it) {
              const int rl = it * 4 + (lane >> 3), cj = lane & 7;
              const int mr = m0 + q * 32 + rl, n = nb0 + cj;
              if (mr < M && n < N) {
                z64 o = coef_mul(cls_alpha, alpha, stg[rl * kStgLd + cj]);
                z64* cp = bat(C, p) + (long long)mr * C.ld + n;
                if (cls_beta) o = o + coef_mul(cls_beta, beta, *cp);
                if (cls_gamma)
                  o = o + coef_mul(cls_gamma, gamma, bat(D, p)[(long long)mr * D.ld + n]);
                if (add_identity && n == mr) o.re += 1.0;
                *cp = o;
                if (want_max) {
                  const unsigned long long a = abs_bits(o.re), c = abs_bits(o.im);
                  omax = max(omax, max(a, c));
                }
              }
            }
            __syncwarp();
          }
        }
      }
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {  // the warp is done with this accumulator (and its sums are stored)
        if constexpr (CG == 2)
          mbar_arrive_cluster(map_rank(smem_u32(&accempty[buf]), 0));
        else
          mbar_arrive(&accempty[buf]);
      }
    }
    if (rmax) {  // per-item max |output| (non-negative floats order like their bit patterns)
      const float wm = warp_max_f((float)__longlong_as_double((long long)omax));
      if (lane == 0 && wm > 0.0f)
        atomicMax(reinterpret_cast<unsigned int*>(rmax + p), __float_as_uint(wm));
    }
    if (*abort_flag && row_ok) {
      // a bounded wait gave up: this tile's outputs are NaN, so that the caller's finite checks
      // see the failure instead of stale values
      const double qnan = __longlong_as_double(0x7FF8000000000000LL);
      z64* crow = bat(C, p) + (long long)m * C.ld;
      for (int n = (n0 + cbase) / 2; n < (n0 + cbase + NT / 2) / 2 && n < N; ++n)
        crow[n] = mkc(qnan, qnan);
    }
  }
  __syncthreads();
  // the pair leaves together: no MMA of the even CTA may still reach the odd CTA's memory
  if constexpr (CG == 2) cluster_sync();
  if (warp == 9) {
    tc_fence_after();
    if constexpr (CG == 2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols)
                   : "memory");
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

// Exact accumulator groups: for every K part and every order d = s + t - 1 <= S, the products
// (s, t) of that order over that part, gsize products per group.
Sched build_sched(const TcPlan& pl, int n_chunks) {
  Sched sc;
  std::memset(&sc, 0, sizeof(sc));
  const int n_parts = std::max(1, std::min(pl.parts, std::min(kMaxParts, n_chunks)));
  for (int q = 0; q < n_parts; ++q) {
    sc.part_lo[q] = (int)((long long)n_chunks * q / n_parts);
    sc.part_hi[q] = (int)((long long)n_chunks * (q + 1) / n_parts);
  }
  int n = 0, g = 0;
  for (int q = 0; q < n_parts; ++q)
    for (int d = 1; d <= pl.S; ++d, ++g)
      for (int s = 1; s <= d && n < kMaxItems; ++s) {
        if (s > 1 && (s - 1) % pl.gsize == 0) ++g;
        sc.it[n++] = Item{(uint8_t)g, (int8_t)s, (int8_t)(d + 1 - s), (int8_t)q};
      }
  sc.n_items = n;
  sc.n_acc = g;
  return sc;
}

template <int NT, int STAGES, int CG, int G, int KPS = 1, int MINB = 1>
cudaError_t launch_tc(cudaStream_t s, int P, int M, int N2, int K, int S, int two_beta,
                      const Sched& sc, const CUtensorMap& mA, const CUtensorMap& mB, const TcWs& ws,
                      const int32_t* zA, int zmA, const int32_t* zB, int zmB, z64 alpha,
                      z64 beta, z64 gamma, BM<double> C, BMc<double> D, bool add_identity,
                      int trunc_beta, const int32_t* active, float* rmax) {
  using CF = Cfg<NT, STAGES, CG, G, KPS>;
  static std::atomic<unsigned> attr{0};
  {
    cudaError_t e = set_smem_once(
        attr, reinterpret_cast<const void*>(&k_tc_gemm<NT, STAGES, CG, G, KPS, MINB>), CF::kSmem);
    if (e != cudaSuccess) return e;
  }
  const int mt = (M + kBM - 1) / kBM;
  // x: row tiles (a CTA pair is two x-adjacent CTAs, so the count is even for pairs), y: columns
  dim3 grid((mt + CG - 1) / CG * CG, (N2 + NT - 1) / NT, P);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  const int count_flops = profiling_on() ? 1 : 0;
  prof_begin(s, PROF_TC_GEMM);
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = dim3(kThreads, 1, 1);
  lc.dynamicSmemBytes = CF::kSmem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CG;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&lc, k_tc_gemm<NT, STAGES, CG, G, KPS, MINB>, mA, mB, sc,
                                     M, N2, S,
                                     two_beta, (const int32_t*)ws.expA, (const int32_t*)ws.expB,
                                     zA, zmA, zB, zmB, alpha, beta, gamma, C, D,
                                     add_identity ? 1 : 0, trunc_beta, active, ws.err, rmax,
                                     K, count_flops);
  prof_end(s, PROF_TC_GEMM);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

// Kernel configuration (autotuner knob): index = 2 * shape + part_choice, part_choice 0/1 = at
// most 4/8 K parts; shape = (pipeline stages, CTAs per MMA, stages released per MMA commit).
// Every tcgen05.commit stalls the tensor pipe for a few hundred cycles, so releasing shared-
// memory stages in groups (one commit per G stages) keeps the MMAs back to back.
struct TcShape {
  int stages, cg, grp, nt;  // nt: real output columns per tile
};
constexpr TcShape kShapes[] = {{6, 1, 1, 128}, {6, 1, 2, 128}, {6, 1, 3, 128}, {8, 2, 1, 128},
                               {8, 2, 2, 128}, {8, 2, 4, 128}, {3, 1, 1, 128}, {4, 2, 1, 128},
                               {2, 1, 1, 128}, {2, 2, 1, 128}, {3, 2, 1, 128}, {2, 2, 1, 64},
                               {2, 1, 1, 64}};
// shapes 6-10: several K chunks per stage: 2 (3 stages of 64 KB; a CTA pair: 4 stages of
// 48 KB), 3 (2 stages of 96 KB; a CTA pair: 3 stages of 72 KB), 4 (a CTA pair: 2 stages of
// 96 KB).  Shapes 11-12: 64-column tiles (256 TMEM columns) with 2 stages of 2 K chunks, two
// CTAs resident per SM so that one tile's waits and final pass overlap the other's MMAs.
constexpr int kNumCfg = 2 * (int)(sizeof(kShapes) / sizeof(kShapes[0]));
std::atomic<int> g_cfg{18};

bool tc_bits_ok(int bits) { return bits == 40 || bits == 48 || bits == 56; }

bool tc_plan(int K, int bits, int max_parts, TcPlan* out) {
  // Digits of beta bits, S = ceil(bits / beta) slices (beta S - 1 >= bits - 1 bits below the line
  // maximum, beta S <= 60, S <= kMaxS): every digit has |q| <= 2^(beta - 1), so a slice product
  // is an integer multiple of its order's unit of magnitude <= 2^(2 beta - 2), and a group of
  // gsize products of one order over a K part of Kp real terms is exact in FP32 when
  // gsize Kp 2^(2 beta - 2) <= 2^24.  Among the feasible (beta, parts, gsize) the plan with the
  // least estimated time wins: every group costs max(its MMA work, one accumulator flush), with
  // the work counted in products x K chunks and a flush worth about 8 of those (the epilogue
  // adds each group into the TMEM-resident sums while the MMAs fill the other accumulator).
  // False when no digit width from 8 down to 4 covers K within max_parts parts and the kernel's
  // item table (the placeholder plan must not be launched).
  constexpr double kFlush = 8.0;
  const int nch = std::max(1, (2 * K + kKC - 1) / kKC);
  double best = -1.0;
  if (tc_bits_ok(bits)) {
    for (int b = 8; b >= 4; --b) {
      const int s = (bits + b - 1) / b;
      if (s > kMaxS || b * s > 60) continue;
      const double per = std::ldexp(1.0, 2 * b - 2);                   // |q_s q_t| bound
      const int cpp = (int)std::floor(16777216.0 / per / kKC);         // chunks per part, gsize 1
      if (cpp < 1) continue;
      const int np = (nch + cpp - 1) / cpp;
      if (np > std::min(max_parts, kMaxParts) || (long long)np * s * (s + 1) / 2 > kMaxItems)
        continue;
      const int part_ch = (nch + np - 1) / np;                          // longest part
      const int gs = std::max(1, (int)std::floor(16777216.0 / (per * part_ch * kKC)));
      double cost = 0.0;
      for (int d = 1; d <= s; ++d)
        for (int left = d; left > 0; left -= gs)
          cost += std::max((double)std::min(left, gs) * part_ch, kFlush);
      cost *= np;
      if (best < 0.0 || cost < best) {
        best = cost;
        *out = TcPlan{b, s, np, gs};
      }
    }
  }
  if (best >= 0.0) return true;
  *out = TcPlan{4, kMaxS, 1, 1};
  return false;
}

bool tc_supports_k(int K, int bits) {
  TcPlan pl;
  return K >= 1 && tc_plan(K, bits, 4, &pl) && tc_plan(K, bits, 8, &pl);
}


namespace {
__global__ void k_flag_timeout(const int32_t* err, int P, int32_t* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P && *err) atomicOr(status + p, NEGF_PT_TIMEOUT);
}
}  // namespace

cudaError_t tc_prof_flops(double* alg, double* hw) {
  double v[2] = {0.0, 0.0};
  cudaError_t e = cudaMemcpyFromSymbol(v, g_tc_prof, sizeof(v));
  *alg = v[0];
  *hw = v[1];
  return e;
}

cudaError_t tc_prof_reset() {
  const double z[2] = {0.0, 0.0};
  return cudaMemcpyToSymbol(g_tc_prof, z, sizeof(z));
}

cudaError_t tc_timeout_reset(cudaStream_t s, const TcWs& ws) {
  return cudaMemsetAsync(ws.err, 0, sizeof(int32_t), s);
}

cudaError_t tc_timeout_flag(cudaStream_t s, const TcWs& ws, int P, int32_t* status) {
  if (P <= 0 || !status) return cudaSuccess;
  k_flag_timeout<<<(P + 255) / 256, 256, 0, s>>>(ws.err, P, status);
  count_launch();
  return cudaGetLastError();
}

size_t tc_ws_bytes(int P, int M, int N, int K, int bits) {
  size_t off = 0;
  TcWs w;
  tc_ws_carve(nullptr, off, P, M, N, K, bits, w);
  return off;
}

void tc_ws_carve(char* base, size_t& off, int P, int M, int N, int K, int bits, TcWs& w) {
  // sized for the largest slice count over the K-part policies, so that a configuration
  // change between sizing and use cannot overrun the workspace
  int S = 0;
  for (int mp : {4, 8}) {
    TcPlan pl;
    tc_plan(K, bits, mp, &pl);
    S = std::max(S, pl.S);
  }
  const size_t L = (size_t)round_up(2 * K, kKC);
  auto take = [&](size_t bytes) -> void* {
    size_t a = (off + 1023) & ~size_t(1023);
    off = a + bytes;
    return base ? base + a : nullptr;
  };
  w.err = static_cast<int32_t*>(take(256));  // first, so that its place does not depend on P
  w.slicesA = take((size_t)P * S * M * L * 2);
  w.slicesB = take((size_t)P * S * 2 * N * L * 2);
  w.expA = static_cast<int32_t*>(take((size_t)P * M * 4));
  w.expB = static_cast<int32_t*>(take((size_t)P * N * 4));
}

cudaError_t tc_gemm(cudaStream_t s, int P, int M, int N, int K, z64 alpha, BMc<double> A,
                    int opA, BMc<double> B, int opB, z64 beta, BM<double> C, z64 gamma,
                    BMc<double> D, bool add_identity, const int32_t* active, const TcWs& ws,
                    int bits, int n_distinct, bool trunc_a, float* rmax) {
  if (P <= 0 || M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  // Operands shared by all items (stride 0) or selected per item from n_distinct matrices are
  // sliced once per distinct matrix; the kernel maps each item to its slice set.
  auto plan_op = [&](BMc<double>& X, const int32_t*& z, int& mode, int& items) {
    z = nullptr;
    mode = 0;
    items = P;
    if (!X.idx && X.stride == 0) {
      mode = 2;
      items = 1;
    } else if (X.idx && n_distinct > 0 && n_distinct <= P) {
      mode = 1;
      z = X.idx;
      items = n_distinct;
      X.idx = nullptr;
    }
  };
  const int32_t *zA = nullptr, *zB = nullptr;
  int zmA = 0, zmB = 0, PA = P, PB = P;
  plan_op(A, zA, zmA, PA);
  plan_op(B, zB, zmB, PB);
  // with a shared operand the active mask cannot gate the slicing by item
  const int32_t* actA = zmA == 0 ? active : nullptr;
  const int32_t* actB = zmB == 0 ? active : nullptr;
  const int cfg = g_cfg.load();
  const int CG = kShapes[cfg / 2].cg;
  TcPlan pl;
  if (!tc_plan(K, bits, cfg % 2 == 0 ? 4 : 8, &pl))
    return cudaErrorInvalidValue;  // K beyond the exact range (callers check tc_supports_k)
  const int bta = pl.beta, S = pl.S;
  const int L = round_up(2 * K, kKC);
  const int N2 = 2 * N;
  __nv_bfloat16* sa = static_cast<__nv_bfloat16*>(ws.slicesA);
  __nv_bfloat16* sb = static_cast<__nv_bfloat16*>(ws.slicesB);
  prof_begin(s, PROF_SLICE);
  // a row of op(A) is a column of A in memory for op T/C; a column of op(B) is a column of B for
  // op N
  cudaError_t e = launch_slice<false>(s, bta, S, dim3((M + 31) / 32, PA), M, K, L, A, opA,
                                      opA != OP_N, sa, ws.expA, actA);
  if (e != cudaSuccess) return e;
  e = launch_slice<true>(s, bta, S, dim3((N + 31) / 32, PB), N, K, L, B, opB, opB == OP_N, sb,
                         ws.expB, actB);
  prof_end(s, PROF_SLICE);
  count_launch(2);
  if (e != cudaSuccess) return e;
  CUtensorMap mA, mB;
  if (!make_map(&mA, sa, L, M, (long long)PA * S, kBM)) return cudaErrorInvalidValue;
  const int NTc = kShapes[cfg / 2].nt;
  if (!make_map(&mB, sb, L, N2, (long long)PB * S, NTc / CG)) return cudaErrorInvalidValue;
  if ((long long)pl.parts * S * (S + 1) / 2 > kMaxItems) return cudaErrorInvalidValue;
  const Sched sc = build_sched(pl, L / kKC);
#define NEGF_TC_ARGS                                                                          \
  s, P, M, N2, K, S, 2 * bta, sc, mA, mB, ws, zA, zmA, zB, zmB, alpha, beta, gamma, C, D,       \
      add_identity, trunc_a ? bta : 0, active, rmax
  switch (cfg / 2) {
    case 0: return launch_tc<kNT, 6, 1, 1>(NEGF_TC_ARGS);
    case 1: return launch_tc<kNT, 6, 1, 2>(NEGF_TC_ARGS);
    case 2: return launch_tc<kNT, 6, 1, 3>(NEGF_TC_ARGS);
    case 3: return launch_tc<kNT, 8, 2, 1>(NEGF_TC_ARGS);
    case 4: return launch_tc<kNT, 8, 2, 2>(NEGF_TC_ARGS);
    case 5: return launch_tc<kNT, 8, 2, 4>(NEGF_TC_ARGS);
    case 6: return launch_tc<kNT, 3, 1, 1, 2>(NEGF_TC_ARGS);
    case 7: return launch_tc<kNT, 4, 2, 1, 2>(NEGF_TC_ARGS);
    case 8: return launch_tc<kNT, 2, 1, 1, 3>(NEGF_TC_ARGS);
    case 9: return launch_tc<kNT, 2, 2, 1, 4>(NEGF_TC_ARGS);
    case 10: return launch_tc<kNT, 3, 2, 1, 3>(NEGF_TC_ARGS);
    case 11: return launch_tc<64, 2, 2, 1, 2, 2>(NEGF_TC_ARGS);
    case 12: return launch_tc<64, 2, 1, 1, 2, 2>(NEGF_TC_ARGS);
    default: return launch_tc<kNT, 6, 1, 1>(NEGF_TC_ARGS);
  }
#undef NEGF_TC_ARGS
}

}  // namespace negf

using namespace negf;

extern "C" {

int32_t negf_tc_config_count(void) { return kNumCfg; }

negf_status negf_tc_config_set(int32_t idx) {
  if (idx < 0 || idx >= kNumCfg) return NEGF_ERR_ARG;
  g_cfg.store(idx);
  return NEGF_OK;
}

int32_t negf_tc_config_get(void) { return g_cfg.load(); }

}  // extern "C"
