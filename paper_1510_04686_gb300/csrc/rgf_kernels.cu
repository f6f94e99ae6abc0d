// Elementwise and reduction kernels of the RGF sweeps: assembly of z - H - V - Sigma, source
// terms of Eq. (2), anti-Hermitian projection, observables of Eqs. (7)-(8) and transmission,
// and the per-step pieces of the Sancho-Rubio decimation.  All on complex128 storage.
#include "profile.cuh"
#include "rgf_kernels.cuh"

namespace negf {

namespace {
constexpr int kT = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];  // fixed order
  }
  return r;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, sh[k]);
  }
  return r;
}

// Scattering self-energies are block-diagonal with A x A blocks (A = 1: orbital-diagonal):
// entry (r, c) of a slab, for r and c in the same block, is sc[r A + c mod A].
__device__ __forceinline__ bool in_block(int r, int c, int A) { return r / A == c / A; }

__global__ void k_assemble(int b, const double* E, double eta, BMc<double> Hd, const double* V,
                           const z64* scat, long long scat_stride, int A, const int32_t* e_idx,
                           BMc<double> Y, int ny, BMc<double> SigA, BMc<double> SigB,
                           BM<double> M, const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  const z64* h = bat(Hd, p);
  const z64* y = Y.p ? bat(Y, p) : nullptr;
  const z64* sa = SigA.p ? bat(SigA, p) : nullptr;
  const z64* sb = SigB.p ? bat(SigB, p) : nullptr;
  const z64* sc = scat ? scat + (e_idx ? (long long)e_idx[p] : (long long)p) * scat_stride : nullptr;
  z64* m = bat(M, p);
  const double e = E[p];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 v = mkc<double>(0.0, 0.0) - h[(long long)r * Hd.ld + c];
    if (r == c) {
      v.re += e - (V ? V[r] : 0.0);
      v.im += eta;
    }
    if (sc && in_block(r, c, A)) v = v - sc[(long long)r * A + c % A];
    if (y && r < ny && c < ny) v = v - y[(long long)r * Y.ld + c];
    if (sa) v = v - sa[(long long)r * SigA.ld + c];
    if (sb) v = v - sb[(long long)r * SigB.ld + c];
    m[(long long)r * M.ld + c] = v;
  }
}

__global__ void k_source(int b, const z64* scat, long long scat_stride, int A,
                         const int32_t* e_idx, BMc<double> SigA, BMc<double> SigB, BM<double> S,
                         const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  const z64* sa = SigA.p ? bat(SigA, p) : nullptr;
  const z64* sb = SigB.p ? bat(SigB, p) : nullptr;
  const z64* sc = scat ? scat + (e_idx ? (long long)e_idx[p] : (long long)p) * scat_stride : nullptr;
  z64* s = bat(S, p);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 v = mkc<double>(0.0, 0.0);
    if (sa) v = v + sa[(long long)r * SigA.ld + c];
    if (sb) v = v + sb[(long long)r * SigB.ld + c];
    if (sc && in_block(r, c, A)) v = v + sc[(long long)r * A + c % A];
    s[(long long)r * S.ld + c] = v;
  }
}

__global__ void k_antiherm(int b, BMc<double> S, BM<double> O, const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  const z64* s = bat(S, p);
  z64* o = bat(O, p);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 a = s[(long long)r * S.ld + c], t = s[(long long)c * S.ld + r];
    o[(long long)r * O.ld + c] = mkc<double>(0.5 * (a.re - t.re), 0.5 * (a.im + t.im));
  }
}

// density from diag G^<; dGR / dGL: the A x A diagonal blocks of G^R, G^< (A = 1: diagonals),
// entry (r, c) at [p][i b A + r A + c mod A]
__global__ void k_slab_obs(int b, int i, int nb_tot, int A, BMc<double> G, BMc<double> GL,
                           double* density, z64* dGR, z64* dGL, const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  const z64* g = bat(G, p);
  const z64* gl = bat(GL, p);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < b; j += gridDim.x * blockDim.x)
    if (density)
      density[(long long)p * nb_tot + (long long)i * b + j] = gl[(long long)j * GL.ld + j].im / kTwoPi;
  if (!dGR && !dGL) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < b * A; j += gridDim.x * blockDim.x) {
    const int r = j / A, c = (r / A) * A + (j - r * A);
    const long long o = ((long long)p * nb_tot + (long long)i * b) * A + j;
    if (dGR) dGR[o] = g[(long long)r * G.ld + c];
    if (dGL) dGL[o] = gl[(long long)r * GL.ld + c];
  }
}

// j_i = 2 Re Tr[t G^<_{i+1,i}] with G^<_{i+1,i} = (U + Q) / 2  ->  Re Tr[t (U + Q)]
__global__ void k_bond_current(int b, BMc<double> Tm, BMc<double> U, BMc<double> Q, double* out,
                               long long out_stride, const int32_t* active) {
  const int p = blockIdx.x;
  if (active && !active[p]) return;
  __shared__ double sh[32];
  const z64* t = bat(Tm, p);
  const z64* u = bat(U, p);
  const z64* q = bat(Q, p);
  double acc = 0.0;
  for (long long k = threadIdx.x; k < (long long)b * b; k += blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 tv = t[(long long)r * Tm.ld + c];
    z64 x = u[(long long)c * U.ld + r] + q[(long long)c * Q.ld + r];
    acc += tv.re * x.re - tv.im * x.im;
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) out[(long long)p * out_stride] = s;
}

__global__ void k_gamma(int b, BMc<double> Sig, BM<double> Gam, const int32_t* active) {
  const int p = blockIdx.y;
  if (active && !active[p]) return;
  const z64* s = bat(Sig, p);
  z64* g = bat(Gam, p);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 a = s[(long long)r * Sig.ld + c], t = s[(long long)c * Sig.ld + r];
    // i (a - conj(t))
    g[(long long)r * Gam.ld + c] = mkc<double>(-(a.im + t.im), a.re - t.re);
  }
}

// T = Re{ Tr[Gamma A] - sum_jk Y_jk conj(Z_jk) },  A = i (G - G^H), Y = Gamma G, Z = G Gamma
__global__ void k_transmission(int b, BMc<double> Gam, BMc<double> G, BMc<double> Y,
                               BMc<double> Z, double* out, const int32_t* active) {
  const int p = blockIdx.x;
  if (active && !active[p]) return;
  __shared__ double sh[32];
  const z64* gm = bat(Gam, p);
  const z64* g = bat(G, p);
  const z64* y = bat(Y, p);
  const z64* z = bat(Z, p);
  double acc = 0.0;
  for (long long k = threadIdx.x; k < (long long)b * b; k += blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 gg = gm[(long long)r * Gam.ld + c];
    z64 a1 = g[(long long)c * G.ld + r], a2 = g[(long long)r * G.ld + c];
    // A_cr = i (G_cr - conj(G_rc))
    z64 A = mkc<double>(-(a1.im + a2.im), a1.re - a2.re);
    acc += gg.re * A.re - gg.im * A.im;
    z64 yv = y[(long long)r * Y.ld + c], zv = z[(long long)r * Z.ld + c];
    acc -= yv.re * zv.re + yv.im * zv.im;
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) out[p] = s;
}

__global__ void k_sr_init(int b, int N, BMc<double> Hd, BMc<double> Hu, BM<double> eps_s,
                          BM<double> eps, BM<double> al, BM<double> be, double* scale) {
  // batch item q = 2 p + side; Hd / Hu batch addressing already per point (index p)
  const int q = blockIdx.y, p = q >> 1, side = q & 1;
  __shared__ double sh[32];
  const z64* hd = Hd.p + (Hd.idx ? (long long)Hd.idx[p] : (long long)p) * Hd.stride +
                  (side ? (long long)(N - 1) * b * b : 0);
  const z64* tu = Hu.p + (Hu.idx ? (long long)Hu.idx[p] : (long long)p) * Hu.stride +
                  (side ? (long long)(N - 2) * b * b : 0);
  z64* es = bat(eps_s, q);
  z64* e = bat(eps, q);
  z64* a = bat(al, q);
  z64* bb = bat(be, q);
  double mx = 0.0;
  for (long long k = threadIdx.x; k < (long long)b * b; k += blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 hv = hd[k];
    es[k] = hv;
    e[k] = hv;
    // right lead: alpha = tau_R (surface -> deeper);  left lead: alpha = tau_L^H
    z64 tv = tu[k];
    z64 tT = tu[(long long)c * b + r];
    z64 av = side ? tv : conjc(tT);
    z64 bv = side ? conjc(tT) : tv;
    a[k] = av;
    bb[k] = bv;
    mx = fmax(mx, fmax(fmax(fabs(hv.re), fabs(hv.im)), fmax(fabs(av.re), fabs(av.im))));
  }
  double m = block_max(mx, sh);
  if (threadIdx.x == 0) scale[q] = m > 0.0 ? m : 1.0;
}

__global__ void k_zminus(int b, const double* E, double eta, BMc<double> X, BM<double> M,
                         const int32_t* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const z64* x = bat(X, q);
  z64* m = bat(M, q);
  const double e = E[q >> 1];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / b), c = (int)(k % b);
    z64 v = mkc<double>(0.0, 0.0) - x[k];
    if (r == c) {
      v.re += e;
      v.im += eta;
    }
    m[k] = v;
  }
}

__global__ void k_add2(int b, BMc<double> T1, BM<double> A1, BM<double> A2, int o0, int n0,
                       int o1, int n1, const int32_t* active) {
  // A1 += T1, A2 += T1 on the square block [o, o + n)^2 of item q (side q & 1 picks o, n)
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int o = (q & 1) ? o1 : o0, n = (q & 1) ? n1 : n0;
  const long long base = (long long)o * b + o;
  const z64* t = bat(T1, q) + base;
  z64* a = bat(A1, q) + base;
  z64* c = bat(A2, q) + base;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)n * n;
       k += (long long)gridDim.x * blockDim.x) {
    const long long e = (k / n) * b + (k % n);
    z64 v = t[e];
    a[e] = a[e] + v;
    c[e] = c[e] + v;
  }
}

__global__ void k_sr_check(int b, int it, double tol, BMc<double> al, BMc<double> be,
                           const double* scale, int32_t* active, int32_t* iters,
                           int32_t* n_active, int32_t* by_side) {
  const int q = blockIdx.x;
  if (!active[q]) return;
  __shared__ double sh[32];
  const z64* a = bat(al, q);
  const z64* c = bat(be, q);
  double mx = 0.0;
  for (long long k = threadIdx.x; k < (long long)b * b; k += blockDim.x) {
    z64 u = a[k], v = c[k];
    mx = fmax(mx, fmax(fmax(fabs(u.re), fabs(u.im)), fmax(fabs(v.re), fabs(v.im))));
  }
  double m = block_max(mx, sh);
  if (threadIdx.x == 0) {
    if (m < tol * scale[q]) {
      active[q] = 0;
      iters[q] = it;
      // per-side copy of the mask: by_side[side * P + p] for q = 2 p + side
      if (by_side) by_side[(q & 1) * (gridDim.x >> 1) + (q >> 1)] = 0;
    } else {
      atomicAdd(n_active, 1);
    }
  }
}

// Sigma^< = i f Gamma for side (q & 1) of point (q >> 1)
__global__ void k_lead_lesser(int b, const double* E, double mu_L, double mu_R, double kT,
                              BMc<double> Gam, BM<double> Les) {
  const int q = blockIdx.y, side = q & 1;
  const double mu = side ? mu_R : mu_L;
  const double x = (E[q >> 1] - mu) / kT;
  const double f = 0.5 * (1.0 - tanh(0.5 * x));
  const z64* g = bat(Gam, q);
  z64* l = bat(Les, q);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    z64 v = g[k];
    l[k] = mkc<double>(-f * v.im, f * v.re);
  }
}

__global__ void k_sr_status(int P, const int32_t* active, const int32_t* item_status,
                            int32_t* iters_in, int32_t* iters_out, int max_iter,
                            int32_t* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int st = 0;
  for (int side = 0; side < 2; ++side) {
    const int q = 2 * p + side;
    int it = iters_in[q];
    if (active[q]) {
      st |= NEGF_PT_NOT_CONVERGED;
      it = max_iter;
    }
    st |= item_status[q];
    if (iters_out) iters_out[q] = it;
  }
  status[p] |= st;
}

__global__ void k_check_finite(const double* x, long long per_pt, int P, int32_t* status) {
  const int p = blockIdx.y;
  if (p >= P) return;
  const double* a = x + (long long)p * per_pt;
  bool bad = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < per_pt;
       k += (long long)gridDim.x * blockDim.x)
    if (!isfinite(a[k])) bad = true;
  if (bad) atomicOr(status + p, NEGF_PT_NONFINITE);
}

__global__ void k_clamp_index(int P, const int32_t* in, int n, int32_t* out, int32_t* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int v = in[p];
  if (v < 0 || v >= n) {
    atomicOr(status + p, NEGF_PT_BAD_INDEX);
    v = v < 0 ? 0 : n - 1;
  }
  out[p] = v;
}

__global__ void k_fill_i32(int32_t* a, long long n, int32_t v) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    a[k] = v;
}

__global__ void k_integrate(int P, int len, const double* w, const int32_t* group, int g,
                            const double* in, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  double acc = 0.0;
  for (int p = 0; p < P; ++p)
    if (!group || group[p] == g) acc += w[p] * in[(long long)p * len + j];
  out[(long long)g * len + j] = acc;
}

inline dim3 grid2(long long work, int P) {
  long long bx = (work + kT - 1) / kT;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)P);
}

}  // namespace

cudaError_t launch_assemble(cudaStream_t s, int P, int b, const double* E, double eta,
                            BMc<double> Hd, const double* V, const z64* scat,
                            long long scat_stride, int A, const int32_t* e_idx, BMc<double> Y,
                            int ny, BMc<double> SigA, BMc<double> SigB, BM<double> M,
                            const int32_t* active) {
  k_assemble<<<grid2((long long)b * b, P), kT, 0, s>>>(b, E, eta, Hd, V, scat, scat_stride, A,
                                                       e_idx, Y, ny, SigA, SigB, M, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_source(cudaStream_t s, int P, int b, const z64* scat, long long scat_stride,
                          int A, const int32_t* e_idx, BMc<double> SigA, BMc<double> SigB,
                          BM<double> S, const int32_t* active) {
  k_source<<<grid2((long long)b * b, P), kT, 0, s>>>(b, scat, scat_stride, A, e_idx, SigA, SigB,
                                                     S, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_antiherm(cudaStream_t s, int P, int b, BMc<double> S, BM<double> O,
                            const int32_t* active) {
  k_antiherm<<<grid2((long long)b * b, P), kT, 0, s>>>(b, S, O, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_slab_obs(cudaStream_t s, int P, int b, int i, int nb_tot, int A,
                            BMc<double> G, BMc<double> GL, double* density, z64* dGR, z64* dGL,
                            const int32_t* active) {
  k_slab_obs<<<grid2(b, P), kT, 0, s>>>(b, i, nb_tot, A, G, GL, density, dGR, dGL, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_bond_current(cudaStream_t s, int P, int b, BMc<double> Tm, BMc<double> U,
                                BMc<double> Q, double* out, long long out_stride,
                                const int32_t* active) {
  k_bond_current<<<P, kT, 0, s>>>(b, Tm, U, Q, out, out_stride, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_gamma(cudaStream_t s, int P, int b, BMc<double> Sig, BM<double> Gam,
                         const int32_t* active) {
  k_gamma<<<grid2((long long)b * b, P), kT, 0, s>>>(b, Sig, Gam, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_transmission(cudaStream_t s, int P, int b, BMc<double> Gam, BMc<double> G,
                                BMc<double> Y, BMc<double> Z, double* out,
                                const int32_t* active) {
  k_transmission<<<P, kT, 0, s>>>(b, Gam, G, Y, Z, out, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_sr_init(cudaStream_t s, int P2, int b, int N, BMc<double> Hd, BMc<double> Hu,
                           BM<double> eps_s, BM<double> eps, BM<double> al, BM<double> be,
                           double* scale) {
  k_sr_init<<<dim3(1, P2), kT, 0, s>>>(b, N, Hd, Hu, eps_s, eps, al, be, scale);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_zminus(cudaStream_t s, int P2, int b, const double* E, double eta,
                          BMc<double> X, BM<double> M, const int32_t* active) {
  k_zminus<<<grid2((long long)b * b, P2), kT, 0, s>>>(b, E, eta, X, M, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_add2(cudaStream_t s, int P2, int b, BMc<double> T1, BM<double> A1,
                        BM<double> A2, int o0, int n0, int o1, int n1, const int32_t* active) {
  const int n = n0 > n1 ? n0 : n1;
  k_add2<<<grid2((long long)n * n, P2), kT, 0, s>>>(b, T1, A1, A2, o0, n0, o1, n1, active);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_sr_check(cudaStream_t s, int P2, int b, int it, double tol, BMc<double> al,
                            BMc<double> be, const double* scale, int32_t* active,
                            int32_t* iters, int32_t* n_active, int32_t* by_side) {
  k_sr_check<<<P2, kT, 0, s>>>(b, it, tol, al, be, scale, active, iters, n_active, by_side);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_lead_lesser(cudaStream_t s, int P2, int b, const double* E, double mu_L,
                               double mu_R, double kT_, BMc<double> Gam, BM<double> Les) {
  k_lead_lesser<<<grid2((long long)b * b, P2), kT, 0, s>>>(b, E, mu_L, mu_R, kT_, Gam, Les);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_sr_status(cudaStream_t s, int P, const int32_t* active,
                             const int32_t* item_status, int32_t* iters_in, int32_t* iters_out,
                             int max_iter, int32_t* status) {
  k_sr_status<<<(P + kT - 1) / kT, kT, 0, s>>>(P, active, item_status, iters_in, iters_out,
                                               max_iter, status);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_check_finite(cudaStream_t s, const double* x, long long per_pt, int P,
                                int32_t* status) {
  if (per_pt <= 0 || P <= 0) return cudaSuccess;
  k_check_finite<<<grid2(per_pt, P), kT, 0, s>>>(x, per_pt, P, status);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_clamp_index(cudaStream_t s, int P, const int32_t* in, int n, int32_t* out,
                               int32_t* status) {
  k_clamp_index<<<(P + kT - 1) / kT, kT, 0, s>>>(P, in, n, out, status);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_fill_i32(cudaStream_t s, int32_t* a, long long n, int32_t v) {
  if (n <= 0) return cudaSuccess;
  long long bx = (n + kT - 1) / kT;
  if (bx > 1024) bx = 1024;
  k_fill_i32<<<(unsigned)bx, kT, 0, s>>>(a, n, v);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_integrate(cudaStream_t s, int P, int len, int n_groups, const double* w,
                             const int32_t* group, const double* in, double* out) {
  for (int g = 0; g < n_groups; ++g) {
    k_integrate<<<(len + kT - 1) / kT, kT, 0, s>>>(P, len, w, group, g, in, out);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace negf
