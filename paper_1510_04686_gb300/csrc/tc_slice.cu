// Operand slicing kernels of the tensor-core complex GEMM (see tc_slice.cuh and tc_gemm.cuh).
#include <cuda_bf16.h>

#include <atomic>
#include <type_traits>

#include "tc_slice.cuh"

namespace negf {
namespace {

// ------------------------------------------------------------------ slicing kernels
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}


// |x| as an ordered integer (the bit pattern without the sign)
__device__ __forceinline__ unsigned long long absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// exponent e with max|x| < 2^e (0 for an all-zero row); the slicing uses e + 1
__device__ __forceinline__ int scale_exp(double mx) {
  if (!(mx > 0.0)) return 0;
  int e;
  frexp(mx, &e);
  return e;
}

// Fixed-point slicing of one value.  The line exponent e is one above the line maximum's
// (|x| < 2^(e - 1)), so x 2^(beta - e) is rounded once to the integer
// R = round(|x| 2^(beta S - e)) <= 2^(beta S - 1) and written in balanced base-2^beta digits
// q_0 .. q_{S-1} (value sum_s q_s 2^(-beta s)): q_0 in [0, 2^(beta-1)], q_s in [-2^(beta-1),
// 2^(beta-1)) for s >= 1, so |q_s q_t| <= 2^(2 beta - 2) for every slice product.  Adding
// H = 2^(beta-1) to every digit position below the top one turns the balanced digits into plain
// bit fields of R + H (minus 2^(beta-1)), so each digit is a constant shift and mask.  Every
// q_s 2^(-beta s) is exact in BF16.
template <int BETA, int S>
struct Digits {
  static constexpr int kBits = BETA * S;
  static_assert(kBits <= 60, "fixed-point value R + H must fit 64 bits");
  static constexpr unsigned long long kH = [] {
    unsigned long long h = 0;
    for (int s = 1; s < S; ++s) h |= (1ull << (BETA - 1)) << (BETA * (S - 1 - s));
    return h;
  }();
};

// R + H for |x| with line exponent e, and the sign of x.
template <int BETA, int S>
__device__ __forceinline__ unsigned long long fixed_point(double x, int e, bool& neg) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  neg = (u >> 63) != 0;
  const int ex = (int)((u >> 52) & 0x7FF);
  unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  if (ex) mant |= 1ull << 52;
  const int sh = (ex ? ex : 1) - 1075 + Digits<BETA, S>::kBits - e;  // |x| 2^(beta S - e) = mant 2^sh
  unsigned long long R;
  if (mant == 0 || sh <= -64) {
    R = 0;
  } else if (sh >= 0) {
    R = mant << sh;
  } else {
    const int r = -sh;
    R = (mant + (1ull << (r - 1))) >> r;
  }
  return R + Digits<BETA, S>::kH;
}

// Slice s of a value from its R + H: sign * q_s * 2^(-beta s) as FP32 (exact).
template <int BETA, int S, int SI>
__device__ __forceinline__ float digit(unsigned long long RH, bool neg) {
  constexpr int pos = BETA * (S - 1 - SI);
  int q = (SI == 0) ? (int)(RH >> pos) : (int)((RH >> pos) & ((1ull << BETA) - 1)) - (1 << (BETA - 1));
  // |q| <= 2^8: exact through the 1.5 * 2^23 bias
  float f = __int_as_float(0x4B400000 + q) - 12582912.0f;
  f *= __int_as_float((127 - BETA * SI) << 23);  // 2^(-beta s)
  return neg ? -f : f;
}

constexpr int kTK = 32;  // complex K values per tile

template <int S>
struct Unroll {
  template <class F>
  __device__ __forceinline__ static void run(F&& f) {
    Unroll<S - 1>::run(f);
    f(std::integral_constant<int, S - 1>{});
  }
};
template <>
struct Unroll<0> {
  template <class F>
  __device__ __forceinline__ static void run(F&&) {}
};

// Slicing of 32 "lines" per CTA (rows of op(A), or columns of op(B)).  Pass 1 finds each line's
// scale exponent with coalesced reads along the line's memory layout; pass 2 walks 32 x 32
// complex tiles through shared memory (so a line that is a column in memory costs the same as a
// row) and writes the S slices with 16-byte stores.  A lines become one output row
// [Re, Im, Re, Im, ...]; B lines (columns n of op(B)) become the two rows 2n = [Re, -Im, ...]
// and 2n + 1 = [Im, Re, ...] of the real embedding.  Padding columns up to L are written as 0.
template <bool kB, int BETA, int S>
__global__ void __launch_bounds__(256) k_slice(int n_lines, int K, int L, BMc<double> X, int op,
                                               bool line_is_col, __nv_bfloat16* out,
                                               int32_t* eo, const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  __shared__ z64 tile[32][kTK + 1];
  __shared__ unsigned long long smax[8][32];
  __shared__ int sexp[32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l0 = blockIdx.x * 32;
  const z64* x = bat(X, p);
  const long long ld = X.ld;
  const bool conj = (op == OP_C);

  // ---- pass 1: max |Re|, |Im| over each line (bit patterns compare as magnitudes)
  if (!line_is_col) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int li = w + 8 * j, line = l0 + li;
      unsigned long long m = 0;
      if (line < n_lines) {
        const z64* row = x + (long long)line * ld;
        for (int k = lane; k < K; k += 32) {
          const z64 v = row[k];
          m = max(m, max(absbits(v.re), absbits(v.im)));
        }
      }
      m = warp_max(m);
      if (lane == 0) smax[0][li] = m;
    }
  } else {
    const int line = l0 + lane;
    unsigned long long m = 0;
    if (line < n_lines)
      for (int k = w; k < K; k += 8) {
        const z64 v = x[(long long)k * ld + line];
        m = max(m, max(absbits(v.re), absbits(v.im)));
      }
    smax[w][lane] = m;
    __syncthreads();
    if (w == 0) {
      unsigned long long mm = smax[0][lane];
#pragma unroll
      for (int i = 1; i < 8; ++i) mm = max(mm, smax[i][lane]);
      smax[0][lane] = mm;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int li = threadIdx.x, line = l0 + li;
    const int e = scale_exp(__longlong_as_double((long long)smax[0][li])) + 1;
    sexp[li] = e;
    if (line < n_lines) eo[(long long)p * n_lines + line] = e;
  }
  __syncthreads();

  // ---- pass 2: tiles of 32 lines x 32 complex K values.  Thread (li, g) converts the four
  // values k = 4g .. 4g + 3 of line li; lanes 0-7 of a quarter-warp hold eight different lines
  // (conflict-free shared-memory reads), and the four quarter-warps cover 16 consecutive k.
  const int li = (w & 3) * 8 + (lane & 7);
  const int g = (w >> 2) * 4 + (lane >> 3);
  const int line = l0 + li;
  const int e = sexp[li];
  const long long rows_out = kB ? 2LL * n_lines : (long long)n_lines;
  for (int k0 = 0; k0 < L / 2; k0 += kTK) {
    if (k0 < K) {
      for (int t = threadIdx.x; t < 32 * kTK; t += 256) {
        const int a = t >> 5, c = t & 31;  // a: slow index, c: fast (contiguous) index
        int tl, tk;
        if (line_is_col) {
          tk = a;
          tl = c;  // memory x[k][line]
        } else {
          tl = a;
          tk = c;  // memory x[line][k]
        }
        const int ln = l0 + tl, kk = k0 + tk;
        z64 v = mkc(0.0, 0.0);
        if (ln < n_lines && kk < K)
          v = line_is_col ? x[(long long)kk * ld + ln] : x[(long long)ln * ld + kk];
        tile[tl][tk] = v;
      }
    }
    __syncthreads();
    if (line < n_lines) {
      unsigned long long rr[4], ri[4];
      bool nr[4], ni[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        z64 v = (k0 < K) ? tile[li][4 * g + j] : mkc(0.0, 0.0);
        if (conj) v.im = -v.im;
        rr[j] = fixed_point<BETA, S>(v.re, e, nr[j]);
        ri[j] = fixed_point<BETA, S>(v.im, e, ni[j]);
      }
      const long long col = 2LL * (k0 + 4 * g);  // first BF16 column of this thread's 4 values
      Unroll<S>::run([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        __nv_bfloat16* base = out + ((long long)p * S + s) * rows_out * L;
        uint32_t w0[4], w1[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float fr = digit<BETA, S, s>(rr[j], nr[j]);
          const float fi = digit<BETA, S, s>(ri[j], ni[j]);
          __nv_bfloat162 a, b2;
          if (!kB) {
            a = __floats2bfloat162_rn(fr, fi);
          } else {
            a = __floats2bfloat162_rn(fr, -fi);
            b2 = __floats2bfloat162_rn(fi, fr);
            w1[j] = *reinterpret_cast<uint32_t*>(&b2);
          }
          w0[j] = *reinterpret_cast<uint32_t*>(&a);
        }
        if (!kB) {
          *reinterpret_cast<uint4*>(base + (long long)line * L + col) =
              make_uint4(w0[0], w0[1], w0[2], w0[3]);
        } else {
          *reinterpret_cast<uint4*>(base + (2LL * line) * L + col) =
              make_uint4(w0[0], w0[1], w0[2], w0[3]);
          *reinterpret_cast<uint4*>(base + (2LL * line + 1) * L + col) =
              make_uint4(w1[0], w1[1], w1[2], w1[3]);
        }
      });
    }
    __syncthreads();
  }
}

// Slicing of kStripLines lines per CTA with the whole strip (lines x K complex values) held in
// shared memory: the operand is read from memory once (the exponent pass and the digit pass both
// read the strip), and each lane converts one complex value, so every slice store of a warp is
// one contiguous 128-byte row segment.  Used when the strip fits (K up to kStripMaxK).
constexpr int kStripLines = 4;    // 4 lines: 4 x 401 x 16 B = 25 KB at K = 400, 8 CTAs per SM
constexpr int kStripMaxK = 1717;  // 4 x (K + 1) x 16 B <= 110 KB
template <bool kB, int BETA, int S>
__global__ void __launch_bounds__(256) k_slice_strip(int n_lines, int K, int L, BMc<double> X,
                                                     int op, bool line_is_col,
                                                     __nv_bfloat16* out, int32_t* eo,
                                                     const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z64* strip = reinterpret_cast<z64*>(smem_raw);  // [kStripLines][K + 1] (padded rows)
  __shared__ int sexp[kStripLines];
  const int lds = K + 1;
  const int l0 = blockIdx.x * kStripLines;
  const z64* x = bat(X, p);
  const long long ld = X.ld;
  const bool conj = (op == OP_C);
  const z64 zero = mkc(0.0, 0.0);
  // load the strip along the operand's memory layout (coalesced either way): element e is
  // (line e / K, k = e % K) for row lines and (line e % L, k = e / L) for column lines (L =
  // kStripLines); eight loads per thread are in flight before their shared-memory stores
  const int tot = kStripLines * K;
  for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * 256) {
    z64 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256;
      v[u] = zero;
      if (e < tot) {
        const int li = line_is_col ? (e & (kStripLines - 1)) : e / K;
        const int k = line_is_col ? e / kStripLines : e - li * K;
        const int line = l0 + li;
        if (line < n_lines)
          v[u] = line_is_col ? x[(long long)k * ld + line] : x[(long long)line * ld + k];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256;
      if (e < tot) {
        const int li = line_is_col ? (e & (kStripLines - 1)) : e / K;
        const int k = line_is_col ? e / kStripLines : e - li * K;
        z64 w = v[u];
        if (conj) w.im = -w.im;
        strip[li * lds + k] = w;
      }
    }
  }
  __syncthreads();
  {  // scale exponent of each line: warp w reduces line w
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < kStripLines) {
      unsigned long long m = 0;
      for (int k = lane; k < K; k += 32) {
        const z64 v = strip[w * lds + k];
        m = max(m, max(absbits(v.re), absbits(v.im)));
      }
      m = warp_max(m);
      if (lane == 0) {
        const int e = scale_exp(__longlong_as_double((long long)m)) + 1;
        sexp[w] = e;
        if (l0 + w < n_lines) eo[(long long)p * n_lines + l0 + w] = e;
      }
    }
  }
  __syncthreads();
  const long long rows_out = kB ? 2LL * n_lines : (long long)n_lines;
  for (int li = 0; li < kStripLines; ++li) {
    const int line = l0 + li;
    if (line >= n_lines) break;
    const int e = sexp[li];
    for (int k = threadIdx.x; k < L / 2; k += blockDim.x) {
      const z64 v = k < K ? strip[li * lds + k] : zero;
      bool nr, ni;
      const unsigned long long rr = fixed_point<BETA, S>(v.re, e, nr);
      const unsigned long long ri = fixed_point<BETA, S>(v.im, e, ni);
      Unroll<S>::run([&](auto sc) {
        constexpr int sl = decltype(sc)::value;
        const float fr = digit<BETA, S, sl>(rr, nr);
        const float fi = digit<BETA, S, sl>(ri, ni);
        __nv_bfloat16* base = out + ((long long)p * S + sl) * rows_out * L;
        if (!kB) {
          reinterpret_cast<__nv_bfloat162*>(base + (long long)line * L)[k] =
              __floats2bfloat162_rn(fr, fi);
        } else {
          reinterpret_cast<__nv_bfloat162*>(base + (2LL * line) * L)[k] =
              __floats2bfloat162_rn(fr, -fi);
          reinterpret_cast<__nv_bfloat162*>(base + (2LL * line + 1) * L)[k] =
              __floats2bfloat162_rn(fi, fr);
        }
      });
    }
  }
}


}  // namespace

template <bool kB>
cudaError_t launch_slice(cudaStream_t s, int beta, int S, dim3 grid, int n_lines, int K, int L,
                         BMc<double> X, int op, bool line_is_col, __nv_bfloat16* out, int32_t* eo,
                         const int32_t* active) {
  const bool strip = K <= kStripMaxK;
  const size_t strip_smem = (size_t)kStripLines * (K + 1) * sizeof(z64);
  const dim3 sgrid((n_lines + kStripLines - 1) / kStripLines, grid.y);
#define NEGF_SLICE_CASE(B_, S_)                                                             \
  if (beta == B_ && S == S_) {                                                              \
    if (strip) {                                                                            \
      static std::atomic<unsigned> attr{0};                                                 \
      cudaError_t ea = set_smem_once(                                                       \
          attr, reinterpret_cast<const void*>(&k_slice_strip<kB, B_, S_>),                  \
          kStripLines * (kStripMaxK + 1) * 16);                                             \
      if (ea != cudaSuccess) return ea;                                                     \
      k_slice_strip<kB, B_, S_><<<sgrid, 256, strip_smem, s>>>(n_lines, K, L, X, op,        \
                                                                line_is_col, out, eo,       \
                                                                active);                    \
    } else {                                                                                \
      k_slice<kB, B_, S_><<<grid, 256, 0, s>>>(n_lines, K, L, X, op, line_is_col, out, eo,  \
                                               active);                                     \
    }                                                                                       \
    return cudaGetLastError();                                                              \
  }
  // 40-bit values
  NEGF_SLICE_CASE(8, 5)
  NEGF_SLICE_CASE(7, 6)
  NEGF_SLICE_CASE(6, 7)
  NEGF_SLICE_CASE(5, 8)
  NEGF_SLICE_CASE(4, 10)
  // 48-bit values
  NEGF_SLICE_CASE(8, 6)
  NEGF_SLICE_CASE(7, 7)
  NEGF_SLICE_CASE(6, 8)
  NEGF_SLICE_CASE(5, 10)
  NEGF_SLICE_CASE(4, 12)
  // 56-bit values
  NEGF_SLICE_CASE(8, 7)
  NEGF_SLICE_CASE(7, 8)
  NEGF_SLICE_CASE(6, 10)
  NEGF_SLICE_CASE(5, 12)
#undef NEGF_SLICE_CASE
  return cudaErrorInvalidValue;  // a (beta, S) pair tc_plan never produces
}

template cudaError_t launch_slice<false>(cudaStream_t, int, int, dim3, int, int, int, BMc<double>,
                                         int, bool, __nv_bfloat16*, int32_t*, const int32_t*);
template cudaError_t launch_slice<true>(cudaStream_t, int, int, dim3, int, int, int, BMc<double>,
                                        int, bool, __nv_bfloat16*, int32_t*, const int32_t*);

}  // namespace negf
