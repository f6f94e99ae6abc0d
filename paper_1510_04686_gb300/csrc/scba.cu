// Self-consistent Born step of the phonon self-energies, Eqs. (4)-(6), on orbital-diagonal
// arrays.  Bandwidth-bound gather over k' and the energy shift E +- hbar omega.
#include "common.cuh"
#include "profile.cuh"

namespace negf {
namespace {

__device__ __forceinline__ z64 ksum(const z64* d, const double* wk, int n_k, long long kstride,
                                    long long off) {
  z64 acc = mkc(0.0, 0.0);
  for (int k = 0; k < n_k; ++k) {  // fixed order: deterministic
    z64 v = d[(long long)k * kstride + off];
    acc.re = fma(wk[k], v.re, acc.re);
    acc.im = fma(wk[k], v.im, acc.im);
  }
  return acc;
}

__global__ void k_scba(int n_k, int n_E, int n_orb, const double* wk, double D_ac, double D_op,
                       int shift, double n0, double mix, const z64* dGR, const z64* dGL,
                       z64* sR, z64* sL, unsigned long long* delta_bits) {
  const long long tot = (long long)n_E * n_orb;
  const long long kstride = tot;
  double dmax = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n_orb), o = (int)(e % n_orb);
    const z64 R0 = ksum(dGR, wk, n_k, kstride, e);
    const z64 L0 = ksum(dGL, wk, n_k, kstride, e);
    const int up = j + shift, dn = j - shift;
    const z64 zero = mkc(0.0, 0.0);
    const z64 Rup = (up < n_E) ? ksum(dGR, wk, n_k, kstride, (long long)up * n_orb + o) : zero;
    const z64 Lup = (up < n_E) ? ksum(dGL, wk, n_k, kstride, (long long)up * n_orb + o) : zero;
    const z64 Rdn = (dn >= 0) ? ksum(dGR, wk, n_k, kstride, (long long)dn * n_orb + o) : zero;
    const z64 Ldn = (dn >= 0) ? ksum(dGL, wk, n_k, kstride, (long long)dn * n_orb + o) : zero;
    // Eq. (4) acoustic, Eq. (6) optical retarded, Eq. (5) optical lesser
    z64 nR, nL;
    nR.re = D_ac * R0.re + D_op * ((1.0 + n0) * Rdn.re + n0 * Rup.re + 0.5 * Ldn.re - 0.5 * Lup.re);
    nR.im = D_ac * R0.im + D_op * ((1.0 + n0) * Rdn.im + n0 * Rup.im + 0.5 * Ldn.im - 0.5 * Lup.im);
    nL.re = D_ac * L0.re + D_op * ((1.0 + n0) * Lup.re + n0 * Ldn.re);
    nL.im = D_ac * L0.im + D_op * ((1.0 + n0) * Lup.im + n0 * Ldn.im);
    const z64 oR = sR[e], oL = sL[e];
    z64 wR = mkc((1.0 - mix) * oR.re + mix * nR.re, (1.0 - mix) * oR.im + mix * nR.im);
    z64 wL = mkc((1.0 - mix) * oL.re + mix * nL.re, (1.0 - mix) * oL.im + mix * nL.im);
    dmax = fmax(dmax, fmax(hypot(wR.re - oR.re, wR.im - oR.im), hypot(wL.re - oL.re, wL.im - oL.im)));
    if (!(isfinite(wR.re) && isfinite(wR.im) && isfinite(wL.re) && isfinite(wL.im)))
      dmax = __longlong_as_double(0x7ff0000000000000LL);
    sR[e] = wR;
    sL[e] = wL;
  }
  for (int off = 16; off > 0; off >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
  if ((threadIdx.x & 31) == 0 && dmax > 0.0)
    atomicMax(delta_bits, (unsigned long long)__double_as_longlong(dmax));
}

// Linear interpolation weights of energy x on the sorted mesh E[0..n): x = (1 - t) E[m] + t E[m+1]
// with 0 <= t <= 1; false when x lies outside [E[0], E[n-1]] (it then contributes nothing).
__device__ __forceinline__ bool mesh_locate(const double* E, int n, double x, int& m, double& t) {
  if (!(x >= E[0] && x <= E[n - 1])) return false;
  if (n == 1) {
    m = 0;
    t = 0.0;
    return true;
  }
  int lo = 0, hi = n - 1;  // E[lo] <= x <= E[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (E[mid] <= x)
      lo = mid;
    else
      hi = mid;
  }
  m = lo;
  t = (x - E[lo]) / (E[hi] - E[lo]);
  return true;
}

// sum_k w_k d[k][.][o] at energy x, linearly interpolated between mesh points
__device__ __forceinline__ z64 ksum_at(const z64* d, const double* wk, int n_k, long long kstride,
                                       const double* E, int n_E, int n_orb, int o, double x) {
  int m;
  double t;
  if (!mesh_locate(E, n_E, x, m, t)) return mkc(0.0, 0.0);
  const z64 a = ksum(d, wk, n_k, kstride, (long long)m * n_orb + o);
  if (t == 0.0 || m + 1 >= n_E) return a;
  const z64 b = ksum(d, wk, n_k, kstride, (long long)(m + 1) * n_orb + o);
  return mkc((1.0 - t) * a.re + t * b.re, (1.0 - t) * a.im + t * b.im);
}

// Eqs. (4)-(6) on a non-uniform energy mesh: the optical terms take diag G at E_j +- hw by linear
// interpolation between the mesh points around it (zero off the mesh).
__global__ void k_scba_mesh(int n_k, int n_E, int n_orb, const double* E, const double* wk,
                            double D_ac, double D_op, double hw, double n0, double mix,
                            const z64* dGR, const z64* dGL, z64* sR, z64* sL,
                            unsigned long long* delta_bits) {
  const long long tot = (long long)n_E * n_orb;
  const long long kstride = tot;
  double dmax = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n_orb), o = (int)(e % n_orb);
    const double Ej = E[j];
    const z64 R0 = ksum(dGR, wk, n_k, kstride, e);
    const z64 L0 = ksum(dGL, wk, n_k, kstride, e);
    const z64 Rup = ksum_at(dGR, wk, n_k, kstride, E, n_E, n_orb, o, Ej + hw);
    const z64 Lup = ksum_at(dGL, wk, n_k, kstride, E, n_E, n_orb, o, Ej + hw);
    const z64 Rdn = ksum_at(dGR, wk, n_k, kstride, E, n_E, n_orb, o, Ej - hw);
    const z64 Ldn = ksum_at(dGL, wk, n_k, kstride, E, n_E, n_orb, o, Ej - hw);
    z64 nR, nL;
    nR.re = D_ac * R0.re + D_op * ((1.0 + n0) * Rdn.re + n0 * Rup.re + 0.5 * Ldn.re - 0.5 * Lup.re);
    nR.im = D_ac * R0.im + D_op * ((1.0 + n0) * Rdn.im + n0 * Rup.im + 0.5 * Ldn.im - 0.5 * Lup.im);
    nL.re = D_ac * L0.re + D_op * ((1.0 + n0) * Lup.re + n0 * Ldn.re);
    nL.im = D_ac * L0.im + D_op * ((1.0 + n0) * Lup.im + n0 * Ldn.im);
    const z64 oR = sR[e], oL = sL[e];
    z64 wR = mkc((1.0 - mix) * oR.re + mix * nR.re, (1.0 - mix) * oR.im + mix * nR.im);
    z64 wL = mkc((1.0 - mix) * oL.re + mix * nL.re, (1.0 - mix) * oL.im + mix * nL.im);
    dmax = fmax(dmax, fmax(hypot(wR.re - oR.re, wR.im - oR.im), hypot(wL.re - oL.re, wL.im - oL.im)));
    if (!(isfinite(wR.re) && isfinite(wR.im) && isfinite(wL.re) && isfinite(wL.im)))
      dmax = __longlong_as_double(0x7ff0000000000000LL);
    sR[e] = wR;
    sL[e] = wL;
  }
  for (int off = 16; off > 0; off >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
  if ((threadIdx.x & 31) == 0 && dmax > 0.0)
    atomicMax(delta_bits, (unsigned long long)__double_as_longlong(dmax));
}

}  // namespace
}  // namespace negf

using namespace negf;

extern "C" negf_status negf_scba_step_mesh(int32_t n_k, int32_t n_E, int32_t n_orb,
                                           const double* E, const double* w_k, double D_ac,
                                           double D_op, double hw, double n0, double mix,
                                           const double* diagGR, const double* diagGL,
                                           double* sigma_R, double* sigma_L, double* delta_out,
                                           void* stream) {
  if (n_k < 1 || n_E < 1 || n_orb < 1 || !E || !w_k || !diagGR || !diagGL || !sigma_R ||
      !sigma_L || !delta_out)
    return NEGF_ERR_ARG;
  if (!(mix > 0.0 && mix <= 1.0) || !(n0 >= 0.0) || !(hw >= 0.0)) return NEGF_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(delta_out, 0, sizeof(double), s) != cudaSuccess) return NEGF_ERR_CUDA;
  const long long tot = (long long)n_E * n_orb;
  long long blocks = (tot + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scba_mesh<<<(unsigned)blocks, 256, 0, s>>>(n_k, n_E, n_orb, E, w_k, D_ac, D_op, hw, n0, mix,
                                               reinterpret_cast<const z64*>(diagGR),
                                               reinterpret_cast<const z64*>(diagGL),
                                               reinterpret_cast<z64*>(sigma_R),
                                               reinterpret_cast<z64*>(sigma_L),
                                               reinterpret_cast<unsigned long long*>(delta_out));
  count_launch();
  return cudaGetLastError() == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}

extern "C" negf_status negf_scba_step(int32_t n_k, int32_t n_E, int32_t n_orb, const double* w_k,
                                      double D_ac, double D_op, int32_t shift, double n0,
                                      double mix, const double* diagGR, const double* diagGL,
                                      double* sigma_R, double* sigma_L, double* delta_out,
                                      void* stream) {
  if (n_k < 1 || n_E < 1 || n_orb < 1 || shift < 0 || !w_k || !diagGR || !diagGL || !sigma_R ||
      !sigma_L || !delta_out)
    return NEGF_ERR_ARG;
  if (!(mix > 0.0 && mix <= 1.0) || !(n0 >= 0.0)) return NEGF_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(delta_out, 0, sizeof(double), s) != cudaSuccess) return NEGF_ERR_CUDA;
  const long long tot = (long long)n_E * n_orb;
  long long blocks = (tot + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scba<<<(unsigned)blocks, 256, 0, s>>>(n_k, n_E, n_orb, w_k, D_ac, D_op, shift, n0, mix,
                                          reinterpret_cast<const z64*>(diagGR),
                                          reinterpret_cast<const z64*>(diagGL),
                                          reinterpret_cast<z64*>(sigma_R),
                                          reinterpret_cast<z64*>(sigma_L),
                                          reinterpret_cast<unsigned long long*>(delta_out));
  count_launch();
  return cudaGetLastError() == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}
