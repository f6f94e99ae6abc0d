// Reverse-mode derivative of the RGF observables with respect to the on-site potential V (the
// e Phi of Eq. 1).  For L = sum_p [sum_j c_pj n_j(p) + sum_i d_pi j_i(p)] with n_j = Im G^<_jj/2pi
// and j_i = 2 Re Tr[t_i G^<_{i+1,i}], the sweep of negf_rgf_solve is run once more keeping its
// forward values, then every block operation is reversed:
//   Y = A B        ->  Abar += Ybar B^H,  Bbar += A^H Ybar
//   Y = M^-1       ->  Mbar  = -Y^H Ybar Y^H
//   G^< = AH(S)    ->  Sbar  = AH(G^<bar),   AH(X) = (X - X^H) / 2
//   M = ... - diag(V)  ->  Vbar_q = -Re Mbar_qq
// with xbar = dL/dRe x + i dL/dIm x.  The backward sweep is reversed first (slab 0 upwards),
// then the forward sweep (slab N-1 downwards).  Lead and scattering self-energies are held fixed.
//
// Sweep checkpointing (negf_options.adjoint_segment = s, 0 < s < N): the slabs are cut into
// segments of s.  Only the forward values (g, g^<) of the last slab of every segment and the
// backward values (G, G^<) of the first slab of every segment are kept; the blocks of one
// segment at a time are recomputed from them, once for the backward sweep, once for its reverse
// and once for the reverse of the forward sweep.  The cotangents of g, g^< and L stay
// full-length (they are written by the reverse of the backward sweep in increasing slab order
// and read by the reverse of the forward sweep in decreasing order), so the footprint drops
// from 8 N to 3 N + 5 s + 4 N / s blocks per point, for 3 more forward sweeps and 1 more
// backward sweep.  s = 0 (or s >= N) keeps every block and recomputes nothing.
#include <algorithm>
#include <vector>

#include "engine.cuh"
#include "profile.cuh"
#include "rgf_kernels.cuh"

namespace negf {
namespace {

constexpr int kT = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;

inline dim3 g2(long long work, int P) {
  long long bx = (work + kT - 1) / kT;
  bx = std::max(1LL, std::min(bx, 64LL));
  return dim3((unsigned)bx, (unsigned)P);
}

// X[p] = 0 except the diagonal i c_pj / (2 pi) (seed of the density cotangent)
__global__ void k_seed_density(int b, int i, int NB, const double* c, BM<double> X) {
  const int p = blockIdx.y;
  z64* x = bat(X, p);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / b), col = (int)(k % b);
    double v = 0.0;
    if (c && r == col) v = c[(long long)p * NB + (long long)i * b + r] / kTwoPi;
    x[(long long)r * X.ld + col] = mkc(0.0, v);
  }
}

// X[p] = d_p t^H (cotangent of Re Tr[t X] scaled by d_p); d NULL gives zero
__global__ void k_set_dtH(int b, BMc<double> Tm, const double* d, long long d_stride, BM<double> X) {
  const int p = blockIdx.y;
  const z64* t = bat(Tm, p);
  z64* x = bat(X, p);
  const double dp = d ? d[(long long)p * d_stride] : 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)b * b;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / b), col = (int)(k % b);
    z64 v = t[(long long)col * Tm.ld + r];
    x[(long long)r * X.ld + col] = mkc(dp * v.re, -dp * v.im);
  }
}

// Y += X
__global__ void k_axpy(long long n, const z64* x, z64* y) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    y[k] = y[k] + x[k];
}

// vb[p][i b + q] = -Re Mbar_qq
__global__ void k_vbar(int b, int i, int NB, BMc<double> Mb, double* vb) {
  const int p = blockIdx.y;
  const z64* m = bat(Mb, p);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < b; q += gridDim.x * blockDim.x)
    vb[(long long)p * NB + (long long)i * b + q] = -m[(long long)q * Mb.ld + q].re;
}

// out[j] (+)= sum over p in order of vb[p][j]
__global__ void k_sum_points(int P, int NB, const double* vb, double* out, int accumulate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= NB) return;
  double acc = accumulate ? out[j] : 0.0;
  for (int p = 0; p < P; ++p) acc += vb[(long long)p * NB + j];
  out[j] = acc;
}

template <class T>
T* take(char* base, size_t& off, size_t n) {
  size_t a = (off + 255) & ~size_t(255);
  off = a + n * sizeof(T);
  return base ? reinterpret_cast<T*>(base + a) : nullptr;
}

struct AdjWs {
  int32_t *sys, *erow;
  z64 *gbar, *glbar, *Lbar;                      // cotangents, all slabs
  z64 *sg, *sgl, *sL, *sG, *sGL;                 // blocks of the resident segment
  z64 *ckg, *ckgl;                               // forward checkpoints: slab c s - 1
  z64 *ckG, *ckGL;                               // backward checkpoints: slab (c + 1) s
  z64 *Gc, *Gn, *GLc, *GLn;                      // rolling cotangents of G, G^<
  z64 *t[14];                                    // temporaries
  double* vb;                                    // per-point V cotangent
  EngineWs eng;
};

// Slabs per segment: the option, or every slab when it is 0 or >= N.
int adj_segment(const negf_options* opt, int N) {
  const int sg = opt->adjoint_segment;
  return (sg <= 0 || sg >= N) ? N : sg;
}

void carve_adj(char* base, size_t& off, int P, int b, int N, int seg, int prec, bool ckpt,
               AdjWs& w) {
  const size_t PB = (size_t)P * b * b;
  const size_t N1 = (size_t)std::max(N - 1, 1);
  // with the solve's checkpoints no sweep block is recomputed or kept here
  const size_t nseg = ckpt ? 0 : (size_t)((N + seg - 1) / seg);
  if (ckpt) seg = 0;
  w.sys = take<int32_t>(base, off, P);
  w.erow = take<int32_t>(base, off, P);
  w.gbar = take<z64>(base, off, N * PB);
  w.glbar = take<z64>(base, off, N * PB);
  w.Lbar = take<z64>(base, off, N1 * PB);
  w.sg = take<z64>(base, off, seg * PB);
  w.sgl = take<z64>(base, off, seg * PB);
  w.sL = take<z64>(base, off, seg * PB);
  w.sG = take<z64>(base, off, seg * PB);
  w.sGL = take<z64>(base, off, seg * PB);
  w.ckg = take<z64>(base, off, nseg * PB);
  w.ckgl = take<z64>(base, off, nseg * PB);
  w.ckG = take<z64>(base, off, nseg * PB);
  w.ckGL = take<z64>(base, off, nseg * PB);
  w.Gc = take<z64>(base, off, PB);
  w.Gn = take<z64>(base, off, PB);
  w.GLc = take<z64>(base, off, PB);
  w.GLn = take<z64>(base, off, PB);
  for (int k = 0; k < 14; ++k) w.t[k] = take<z64>(base, off, PB);
  w.vb = take<double>(base, off, (size_t)P * N * b);
  carve_engine(base, off, P, b, prec, w.eng);
}

#define CK(x)                                    \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return note_error(e_), NEGF_ERR_CUDA; \
  } while (0)

struct AdjArgs {
  const negf_device* dev;
  const double* E;
  const int32_t* sys;
  const double* V;
  const z64* sigR;
  const z64* sigL;
  const z64* scatR;
  const z64* scatL;
  const int32_t* e_idx;
  int32_t n_rows;
  const negf_options* opt;
  const double* nbar;   // [P][N b] or NULL
  const double* jbar;   // [P][N-1] or NULL
  double* Vbar;         // [N b]
  bool accumulate;
  int32_t* status;
  int A;  // scattering self-energy block width (1: orbital-diagonal)
  const z64* ckpt;  // sweep checkpoints of negf_rgf_solve (nullable), [5][N][n_tot][b][b]
  int n_tot, p0;    // points of the checkpoints; first point of this chunk
};

negf_status adjoint_chunk_run(const AdjArgs& a, int P, char* wsbase, cudaStream_t s) {
  const negf_device* dev = a.dev;
  const int b = dev->block, N = dev->n_slabs;
  const size_t bb = (size_t)b * b, PB = (size_t)P * bb;
  const int NB = N * b;
  const z64 one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0), two = mkc(2.0, 0.0), mone = mkc(-1.0, 0.0);
  const BMc<double> none{nullptr, 0, nullptr, 0};
  size_t off = 0;
  AdjWs w;
  const bool have_ck = a.ckpt != nullptr;
  const int seg = have_ck ? N : adj_segment(a.opt, N);
  const int nseg = (N + seg - 1) / seg;
  carve_adj(wsbase, off, P, b, N, seg, a.opt->precision, have_ck, w);
  // block of kind k of slab i in the solve's checkpoints (read only)
  auto ck = [&](int k, int i) -> z64* {
    return const_cast<z64*>(a.ckpt) + ckpt_offset(k, i, N, a.n_tot, a.p0, bb);
  };
  Engine eng(s, a.opt->precision, a.opt->refine_steps, refine_limit(a.opt), w.eng, b,
             dev->n_sys);
  CK(eng.timeout_reset());
  CK(launch_clamp_index(s, P, a.sys, dev->n_sys, w.sys, a.status));
  const int32_t* sysc = w.sys;
  const int32_t* erow = nullptr;
  if (a.scatR && a.e_idx) {
    CK(launch_clamp_index(s, P, a.e_idx, a.n_rows, w.erow, a.status));
    erow = w.erow;
  }
  auto F = [&](z64* p) { return BM<double>{p, (long long)bb, nullptr, b}; };
  auto Fc = [&](const z64* p) { return BMc<double>{p, (long long)bb, nullptr, b}; };
  auto S = [&](z64* base, int i) { return base + (size_t)i * PB; };
  auto Hd = [&](int i) {
    return BMc<double>{reinterpret_cast<const z64*>(dev->H_diag) + (size_t)i * bb,
                       (long long)(N * bb), sysc, b};
  };
  auto Hu = [&](int i) {
    return BMc<double>{reinterpret_cast<const z64*>(dev->H_up) + (size_t)i * bb,
                       (long long)((N - 1) * bb), sysc, b};
  };
  const BMc<double> SigL_R{a.sigR, (long long)(2 * bb), nullptr, b};
  const BMc<double> SigR_R{a.sigR + bb, (long long)(2 * bb), nullptr, b};
  const BMc<double> SigL_L{a.sigL, (long long)(2 * bb), nullptr, b};
  const BMc<double> SigR_L{a.sigL + bb, (long long)(2 * bb), nullptr, b};
  z64** T = w.t;
  // Interface couplings: t_i is nonzero only on its last ir rows R and first ic columns C
  // (ir = ic = b: dense, and every view below is the whole block).  Then L = g t lives on the
  // columns C, K = g t^H and W = G t^H on the columns R, Y = t^H L on C x C, and so do the
  // cotangents that matter: every product with a hopping, and every product of an intermediate
  // with that structure, contracts over r or c and forms only the part of its output that
  // is read later (the other entries of those buffers are never read).
  const int ir = dev->iface_rows > 0 ? dev->iface_rows : b;
  const int ic = dev->iface_cols > 0 ? dev->iface_cols : b;
  const int R0 = b - ir;  // first row of R (C starts at column 0)
  auto cv = [](BMc<double> X, int c0) {
    X.p += c0;
    return X;
  };
  auto rv = [](BMc<double> X, int r0) {
    X.p += (long long)r0 * X.ld;
    return X;
  };
  auto bcv = [](BM<double> X, int c0) {
    X.p += c0;
    return X;
  };
  auto brv = [](BM<double> X, int r0) {
    X.p += (long long)r0 * X.ld;
    return X;
  };
  auto tv = [&](BMc<double> H) { return rv(H, R0); };  // the r x c support T of a hopping
  auto has_src = [&](int i) { return i == 0 || i == N - 1 || a.scatL != nullptr; };
  auto build_src = [&](int i, z64* out) -> cudaError_t {
    return launch_source(s, P, b, a.scatL ? a.scatL + (size_t)i * b * a.A : nullptr,
                         (long long)NB * a.A, a.A, erow,
                         i == 0 ? SigL_L : none, i == N - 1 ? SigR_L : none, F(out), nullptr);
  };
  const double eta = a.opt->eta_device;

  // ---- segment bookkeeping: which segment's forward / backward blocks are resident (with the
  // solve's checkpoints every block of the one segment is, and nothing is recomputed)
  int resF = have_ck ? 0 : -1, resB = have_ck ? 0 : -1;
  auto seg_lo = [&](int c) { return c * seg; };
  auto seg_hi = [&](int c) { return std::min(N, (c + 1) * seg); };
  // forward blocks of slab i: the resident segment, or the checkpoint just below it
  auto gF = [&](int i) -> z64* {
    if (have_ck) return ck(CK_G_FWD, i);
    if (i >= seg_lo(resF) && i < seg_hi(resF)) return S(w.sg, i - seg_lo(resF));
    return S(w.ckg, resF);  // i == seg_lo(resF) - 1
  };
  auto glF = [&](int i) -> z64* {
    if (have_ck) return ck(CK_GL_FWD, i);
    if (i >= seg_lo(resF) && i < seg_hi(resF)) return S(w.sgl, i - seg_lo(resF));
    return S(w.ckgl, resF);
  };
  auto Lb = [&](int i) -> z64* {
    if (have_ck) return ck(CK_L, i);
    return S(w.sL, i - seg_lo(resF));
  };
  // backward blocks of slab i: the resident segment, or the checkpoint just above it
  auto Gb = [&](int i) -> z64* {
    if (have_ck) return ck(CK_G, i);
    if (i >= seg_lo(resB) && i < seg_hi(resB)) return S(w.sG, i - seg_lo(resB));
    return S(w.ckG, resB);  // i == seg_hi(resB)
  };
  auto GLb = [&](int i) -> z64* {
    if (have_ck) return ck(CK_GL, i);
    if (i >= seg_lo(resB) && i < seg_hi(resB)) return S(w.sGL, i - seg_lo(resB));
    return S(w.ckGL, resB);
  };

  // ---- forward sweep over segment c from the checkpoint below it (values kept for the
  // segment; L_i = g_i t_i for every slab of the segment that has a right neighbour; the last
  // slab's g, g^< become the checkpoint of segment c + 1)
  auto forward_segment = [&](int c) -> negf_status {
    if (resF == c) return NEGF_OK;
    resF = c;
    const int lo = seg_lo(c), hi = seg_hi(c);
    for (int i = lo; i < hi; ++i) {
      BMc<double> Y = none;
      if (i > 0) {
        // L_{i-1} = g_{i-1} t_{i-1} (kept when slab i - 1 is in the segment);  Y = t^H L
        z64* Lprev = (i - 1 >= lo) ? Lb(i - 1) : T[6];
        // L[:, C] = g[:, R] T;  Y[C, C] = T^H L[R, C]
        CK(eng.gemm(P, b, ic, ir, one, cv(Fc(gF(i - 1)), R0), OP_N, tv(Hu(i - 1)), OP_N, zero,
                    F(Lprev), zero, none, nullptr));
        CK(eng.gemm(P, ic, ic, ir, one, tv(Hu(i - 1)), OP_C, rv(Fc(Lprev), R0), OP_N, zero,
                    F(T[0]), zero, none, nullptr));
        Y = Fc(T[0]);
      }
      CK(launch_assemble(s, P, b, a.E, eta, Hd(i), a.V ? a.V + (size_t)i * b : nullptr,
                         a.scatR ? a.scatR + (size_t)i * b * a.A : nullptr,
                         (long long)NB * a.A, a.A, erow, Y, ic,
                         i == 0 ? SigL_R : none, i == N - 1 ? SigR_R : none, F(T[1]), nullptr));
      CK(eng.inv(P, F(T[1]), F(gF(i)), a.status, nullptr));
      bool prev = false;
      if (i > 0) {
        // K[:, R] = g_i[:, C] T^H;  Vt = g^<_{i-1}[:, R] K[:, R]^H;  g^<_i = K[:, R] Vt[R, :]
        CK(eng.gemm(P, b, ir, ic, one, Fc(gF(i)), OP_N, tv(Hu(i - 1)), OP_C, zero,
                    bcv(F(T[2]), R0), zero, none, nullptr));
        CK(eng.gemm(P, b, b, ir, one, cv(Fc(glF(i - 1)), R0), OP_N, cv(Fc(T[2]), R0), OP_C, zero,
                    F(T[3]), zero, none, nullptr));
        CK(eng.gemm(P, b, b, ir, one, cv(Fc(T[2]), R0), OP_N, rv(Fc(T[3]), R0), OP_N, zero,
                    F(glF(i)), zero, none, nullptr));
        prev = true;
      }
      if (has_src(i)) {
        CK(build_src(i, T[4]));
        CK(eng.gemm(P, b, b, b, one, Fc(gF(i)), OP_N, Fc(T[4]), OP_N, zero, F(T[5]), zero, none,
                    nullptr));
        CK(eng.gemm(P, b, b, b, one, Fc(T[5]), OP_N, Fc(gF(i)), OP_C, prev ? one : zero,
                    F(glF(i)), zero, none, nullptr));
      } else if (!prev) {
        CK(cudaMemsetAsync(glF(i), 0, PB * sizeof(z64), s));
      }
    }
    if (hi - 1 <= N - 2)
      CK(eng.gemm(P, b, ic, ir, one, cv(Fc(gF(hi - 1)), R0), OP_N, tv(Hu(hi - 1)), OP_N, zero,
                  F(Lb(hi - 1)), zero, none, nullptr));
    if (c + 1 < nseg) {
      CK(cudaMemcpyAsync(S(w.ckg, c + 1), gF(hi - 1), PB * sizeof(z64),
                         cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(S(w.ckgl, c + 1), glF(hi - 1), PB * sizeof(z64),
                         cudaMemcpyDeviceToDevice, s));
    }
    return NEGF_OK;
  };

  negf_status r;
#define RUN(x)                          \
  do {                                  \
    if ((r = (x)) != NEGF_OK) return r; \
  } while (0)

  // W[:, R] = G_{i+1}[:, C] T^H;  LW[:, R] = L[:, C] W[C, R];  Q = G^<_{i+1}[:, C] L[:, C]^H;
  // U = 2 W[:, R] g^<_i[R, :] + Q  (backward step i, its blocks resident)
  auto backward_products = [&](int i, z64* Wm, z64* LW, z64* Q, z64* U) -> negf_status {
    z64* L = Lb(i);
    CK(eng.gemm(P, b, ir, ic, one, Fc(Gb(i + 1)), OP_N, tv(Hu(i)), OP_C, zero, bcv(F(Wm), R0),
                zero, none, nullptr));
    CK(eng.gemm(P, b, ir, ic, one, Fc(L), OP_N, cv(Fc(Wm), R0), OP_N, zero, bcv(F(LW), R0), zero,
                none, nullptr));
    CK(eng.gemm(P, b, b, ic, one, Fc(GLb(i + 1)), OP_N, Fc(L), OP_C, zero, F(Q), zero, none,
                nullptr));
    CK(eng.gemm(P, b, b, ir, two, cv(Fc(Wm), R0), OP_N, rv(Fc(glF(i)), R0), OP_N, zero, F(U), one,
                Fc(Q), nullptr));
    return NEGF_OK;
  };

  // ---- backward sweep over segment c (its forward blocks resident) from the checkpoint above
  // it; the segment's first slab becomes the checkpoint of segment c - 1
  auto backward_segment = [&](int c) -> negf_status {
    if (resB == c) return NEGF_OK;
    resB = c;
    const int lo = seg_lo(c), hi = seg_hi(c);
    int top = hi - 1;
    if (hi == N) {  // G_{N-1} = g_{N-1}, G^<_{N-1} = g^<_{N-1}
      CK(cudaMemcpyAsync(Gb(N - 1), gF(N - 1), PB * sizeof(z64), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(GLb(N - 1), glF(N - 1), PB * sizeof(z64), cudaMemcpyDeviceToDevice, s));
      top = N - 2;
    }
    for (int i = top; i >= lo; --i) {
      z64 *Wm = T[0], *LW = T[1], *Q = T[2], *U = T[3];
      RUN(backward_products(i, Wm, LW, Q, U));
      CK(eng.gemm(P, b, b, ir, one, cv(Fc(LW), R0), OP_N, rv(Fc(gF(i)), R0), OP_N, zero,
                  F(Gb(i)), one, Fc(gF(i)), nullptr));
      CK(eng.gemm(P, b, b, ic, one, Fc(Lb(i)), OP_N, Fc(U), OP_N, zero, F(T[4]), one,
                  Fc(glF(i)), nullptr));
      CK(launch_antiherm(s, P, b, Fc(T[4]), F(GLb(i)), nullptr));
    }
    if (c > 0) {
      CK(cudaMemcpyAsync(S(w.ckG, c - 1), Gb(lo), PB * sizeof(z64), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(S(w.ckGL, c - 1), GLb(lo), PB * sizeof(z64), cudaMemcpyDeviceToDevice,
                         s));
    }
    return NEGF_OK;
  };
  // ------------------------------------------------ forward sweep: checkpoints of every segment
  for (int c = 0; c < nseg; ++c) RUN(forward_segment(c));
  // ------------------------------------------------ backward sweep: checkpoints, top down
  for (int c = nseg - 1; c >= 0; --c) {
    RUN(forward_segment(c));
    RUN(backward_segment(c));
  }

  // ------------------------------------------------ reverse of the backward sweep
  CK(cudaMemsetAsync(w.gbar, 0, (size_t)N * PB * sizeof(z64), s));
  CK(cudaMemsetAsync(w.glbar, 0, (size_t)N * PB * sizeof(z64), s));
  CK(cudaMemsetAsync(w.Lbar, 0, (size_t)std::max(N - 1, 1) * PB * sizeof(z64), s));
  CK(cudaMemsetAsync(w.Gc, 0, PB * sizeof(z64), s));
  k_seed_density<<<g2((long long)bb, P), kT, 0, s>>>(b, 0, NB, a.nbar, F(w.GLc));
  count_launch();
  z64 *Gc = w.Gc, *Gn = w.Gn, *GLc = w.GLc, *GLn = w.GLn;
  for (int i = 0; i + 1 < N; ++i) {
    const int c = i / seg;
    RUN(forward_segment(c));
    if (resB != c) {
      resB = -1;  // recompute the segment's backward blocks from its checkpoint
      RUN(backward_segment(c));
    }
    z64 *Wm = T[0], *LW = T[1], *Q = T[2], *U = T[3], *Sb = T[4], *Ub = T[5], *Wb = T[6],
        *Qb = T[7], *LWb = T[8];
    z64* L = Lb(i);
    z64* Lbar = S(w.Lbar, i);
    // recompute W, LW, Q, U of backward step i
    RUN(backward_products(i, Wm, LW, Q, U));
    // current cotangent: Ubar = Qbar = d_i t_i^H (rows C; every later term of Ubar, Qbar too)
    k_set_dtH<<<g2((long long)bb, P), kT, 0, s>>>(b, Hu(i), a.jbar ? a.jbar + i : nullptr, N - 1, F(Ub));
    k_set_dtH<<<g2((long long)bb, P), kT, 0, s>>>(b, Hu(i), a.jbar ? a.jbar + i : nullptr, N - 1, F(Qb));
    count_launch(2);
    // G^<_i = AH(g^<_i + L U):  Lbar[:, C] += Sbar U[C, :]^H,  Ubar[C, :] += L[:, C]^H Sbar
    CK(launch_antiherm(s, P, b, Fc(GLc), F(Sb), nullptr));
    k_axpy<<<(unsigned)std::min<size_t>((PB + kT - 1) / kT, 4096), kT, 0, s>>>((long long)PB, Sb, S(w.glbar, i));
    count_launch();
    CK(eng.gemm(P, b, ic, b, one, Fc(Sb), OP_N, Fc(U), OP_C, one, F(Lbar), zero, none, nullptr));
    CK(eng.gemm(P, ic, b, b, one, Fc(L), OP_C, Fc(Sb), OP_N, one, F(Ub), zero, none, nullptr));
    // U = 2 W g^<_i + Q:  Wbar[C, R] = 2 Ubar[C, :] g^<_i[R, :]^H,
    // g^<bar_i[R, :] += 2 W[C, R]^H Ubar[C, :],  Qbar += Ubar
    CK(eng.gemm(P, ic, ir, b, two, Fc(Ub), OP_N, rv(Fc(glF(i)), R0), OP_C, zero, bcv(F(Wb), R0),
                zero, none, nullptr));
    CK(eng.gemm(P, ir, b, ic, two, cv(Fc(Wm), R0), OP_C, Fc(Ub), OP_N, one,
                brv(F(S(w.glbar, i)), R0), zero, none, nullptr));
    k_axpy<<<(unsigned)std::min<size_t>((PB + kT - 1) / kT, 4096), kT, 0, s>>>((long long)PB, Ub, Qb);
    count_launch();
    // Q = G^<_{i+1} L^H:  G^<bar_{i+1}[C, C] += Qbar[C, :] L[:, C],
    // Lbar[:, C] += Qbar[C, :]^H G^<_{i+1}[C, C]
    k_seed_density<<<g2((long long)bb, P), kT, 0, s>>>(b, i + 1, NB, a.nbar, F(GLn));
    count_launch();
    CK(eng.gemm(P, ic, ic, b, one, Fc(Qb), OP_N, Fc(L), OP_N, one, F(GLn), zero, none, nullptr));
    CK(eng.gemm(P, b, ic, ic, one, Fc(Qb), OP_C, Fc(GLb(i + 1)), OP_N, one, F(Lbar), zero, none,
                nullptr));
    // G_i = g_i + LW g_i:  LWbar[:, R] = Gbar g_i[R, :]^H,  gbar_i[R, :] += LW[:, R]^H Gbar
    k_axpy<<<(unsigned)std::min<size_t>((PB + kT - 1) / kT, 4096), kT, 0, s>>>((long long)PB, Gc, S(w.gbar, i));
    count_launch();
    CK(eng.gemm(P, b, ir, b, one, Fc(Gc), OP_N, rv(Fc(gF(i)), R0), OP_C, zero, bcv(F(LWb), R0),
                zero, none, nullptr));
    CK(eng.gemm(P, ir, b, b, one, cv(Fc(LW), R0), OP_C, Fc(Gc), OP_N, one,
                brv(F(S(w.gbar, i)), R0), zero, none, nullptr));
    // LW = L W:  Lbar[:, C] += LWbar[:, R] W[C, R]^H,  Wbar[C, R] += L[:, C]^H LWbar[:, R]
    CK(eng.gemm(P, b, ic, ir, one, cv(Fc(LWb), R0), OP_N, cv(Fc(Wm), R0), OP_C, one, F(Lbar),
                zero, none, nullptr));
    CK(eng.gemm(P, ic, ir, b, one, Fc(L), OP_C, cv(Fc(LWb), R0), OP_N, one, bcv(F(Wb), R0), zero,
                none, nullptr));
    // W = G_{i+1} t_i^H:  Gbar_{i+1} = Wbar t_i, nonzero on C x C only
    if (ir < b || ic < b) CK(cudaMemsetAsync(Gn, 0, PB * sizeof(z64), s));
    CK(eng.gemm(P, ic, ic, ir, one, cv(Fc(Wb), R0), OP_N, tv(Hu(i)), OP_N, zero, F(Gn), zero,
                none, nullptr));
    std::swap(Gc, Gn);
    std::swap(GLc, GLn);
  }
  // slab N-1: G = g, G^< = g^< directly
  k_axpy<<<(unsigned)std::min<size_t>((PB + kT - 1) / kT, 4096), kT, 0, s>>>((long long)PB, Gc, S(w.gbar, N - 1));
  k_axpy<<<(unsigned)std::min<size_t>((PB + kT - 1) / kT, 4096), kT, 0, s>>>((long long)PB, GLc, S(w.glbar, N - 1));
  count_launch(2);

  // ------------------------------------------------ reverse of the forward sweep
  for (int i = N - 1; i >= 0; --i) {
    RUN(forward_segment(i / seg));
    z64 *K = T[0], *Vt = T[1], *Kb = T[2], *Vtb = T[3], *Ssrc = T[4], *Wsrc = T[5], *Wbar = T[6],
        *T1 = T[7], *Mb = T[8];
    z64* gb = S(w.gbar, i);
    z64* glb = S(w.glbar, i);
    if (i > 0) {
      // K[:, R] = g_i[:, C] T^H;  Vt = g^<_{i-1}[:, R] K[:, R]^H
      CK(eng.gemm(P, b, ir, ic, one, Fc(gF(i)), OP_N, tv(Hu(i - 1)), OP_C, zero, bcv(F(K), R0),
                  zero, none, nullptr));
      CK(eng.gemm(P, b, b, ir, one, cv(Fc(glF(i - 1)), R0), OP_N, cv(Fc(K), R0), OP_C, zero,
                  F(Vt), zero, none, nullptr));
      // g^<_i = K[:, R] Vt[R, :] (+ source):  Kbar[:, R] = g^<bar Vt[R, :]^H,
      // Vtbar[R, :] = K[:, R]^H g^<bar
      CK(eng.gemm(P, b, ir, b, one, Fc(glb), OP_N, rv(Fc(Vt), R0), OP_C, zero, bcv(F(Kb), R0),
                  zero, none, nullptr));
      CK(eng.gemm(P, ir, b, b, one, cv(Fc(K), R0), OP_C, Fc(glb), OP_N, zero, brv(F(Vtb), R0),
                  zero, none, nullptr));
      // Vt = g^<_{i-1}[:, R] K[:, R]^H:  Kbar[:, R] += Vtbar[R, :]^H g^<_{i-1}[R, R],
      // g^<bar_{i-1}[R, R] += Vtbar[R, :] K[:, R]
      CK(eng.gemm(P, b, ir, ir, one, rv(Fc(Vtb), R0), OP_C, rv(cv(Fc(glF(i - 1)), R0), R0), OP_N,
                  one, bcv(F(Kb), R0), zero, none, nullptr));
      CK(eng.gemm(P, ir, ir, b, one, rv(Fc(Vtb), R0), OP_N, cv(Fc(K), R0), OP_N, one,
                  brv(bcv(F(S(w.glbar, i - 1)), R0), R0), zero, none, nullptr));
      // K = g_i t_{i-1}^H:  gbar_i[:, C] += Kbar[:, R] T
      CK(eng.gemm(P, b, ic, ir, one, cv(Fc(Kb), R0), OP_N, tv(Hu(i - 1)), OP_N, one, F(gb), zero,
                  none, nullptr));
    }
    if (has_src(i)) {
      CK(build_src(i, Ssrc));
      CK(eng.gemm(P, b, b, b, one, Fc(gF(i)), OP_N, Fc(Ssrc), OP_N, zero, F(Wsrc), zero, none, nullptr));
      // g^<_i += Wsrc g_i^H
      CK(eng.gemm(P, b, b, b, one, Fc(glb), OP_N, Fc(gF(i)), OP_N, zero, F(Wbar), zero, none, nullptr));
      CK(eng.gemm(P, b, b, b, one, Fc(glb), OP_C, Fc(Wsrc), OP_N, one, F(gb), zero, none, nullptr));
      // Wsrc = g_i S
      CK(eng.gemm(P, b, b, b, one, Fc(Wbar), OP_N, Fc(Ssrc), OP_C, one, F(gb), zero, none, nullptr));
    }
    // g_i = M_i^-1:  Mbar = -g^H gbar g^H
    CK(eng.gemm(P, b, b, b, one, Fc(gb), OP_N, Fc(gF(i)), OP_C, zero, F(T1), zero, none, nullptr));
    CK(eng.gemm(P, b, b, b, mone, Fc(gF(i)), OP_C, Fc(T1), OP_N, zero, F(Mb), zero, none, nullptr));
    k_vbar<<<g2(b, P), kT, 0, s>>>(b, i, NB, Fc(Mb), w.vb);
    count_launch();
    if (i > 0) {
      // M_i = ... - Y with Y[C, C] = T^H L_{i-1}[R, C]:  Lbar_{i-1}[R, C] -= T Mbar[C, C];
      // L_{i-1}[:, C] = g_{i-1}[:, R] T:  gbar_{i-1}[:, R] += Lbar[:, C] T^H
      CK(eng.gemm(P, ir, ic, ic, mone, tv(Hu(i - 1)), OP_N, Fc(Mb), OP_N, one,
                  brv(F(S(w.Lbar, i - 1)), R0), zero, none, nullptr));
      CK(eng.gemm(P, b, ir, ic, one, Fc(S(w.Lbar, i - 1)), OP_N, tv(Hu(i - 1)), OP_C, one,
                  bcv(F(S(w.gbar, i - 1)), R0), zero, none, nullptr));
    }
  }
#undef RUN
  k_sum_points<<<(NB + kT - 1) / kT, kT, 0, s>>>(P, NB, w.vb, a.Vbar, a.accumulate ? 1 : 0);
  count_launch();
  CK(cudaGetLastError());
  CK(eng.timeout_flag(P, a.status));
  return NEGF_OK;
}

constexpr size_t kAdjBudget = 32ull << 30;

}  // namespace

size_t adjoint_bytes(const negf_device* dev, int P, const negf_options* opt, bool ckpt) {
  size_t off = 0;
  AdjWs w;
  carve_adj(nullptr, off, P, dev->block, dev->n_slabs, adj_segment(opt, dev->n_slabs),
            opt->precision, ckpt, w);
  return off + 256;
}

int adjoint_chunk(const negf_device* dev, int n_pts, const negf_options* opt, bool ckpt) {
  if (opt->chunk > 0) return std::max(1, std::min(std::min(opt->chunk, n_pts), 16384));
  const size_t per = adjoint_bytes(dev, 2, opt, ckpt) - adjoint_bytes(dev, 1, opt, ckpt);
  size_t c = std::max<size_t>(1, kAdjBudget / std::max<size_t>(per, 1));
  return (int)std::max<size_t>(1, std::min<size_t>(c, (size_t)std::max(n_pts, 1)));
}

}  // namespace negf

using namespace negf;

extern "C" negf_status negf_rgf_adjoint(const negf_device* dev, int32_t n_pts, const double* E,
                                        const int32_t* sys_idx, const double* V,
                                        const double* sigma_R, const double* sigma_L,
                                        const double* scat_R, const double* scat_L,
                                        const int32_t* e_idx, int32_t n_rows,
                                        const negf_options* opt, const void* checkpoints,
                                        const double* density_bar, const double* current_bar,
                                        double* V_bar, int32_t* status, void* ws,
                                        size_t ws_bytes, void* stream) {
  if (!dev || !opt || dev->n_sys < 1 || dev->n_slabs < 1 || dev->block < 1 || !dev->H_diag ||
      (dev->n_slabs > 1 && !dev->H_up) || n_pts < 0)
    return NEGF_ERR_ARG;
  if (!engine_supports(opt->precision, dev->block)) return NEGF_ERR_UNSUPPORTED;
  if (!(opt->kT > 0.0) || opt->refine_steps < 0 || opt->refine_steps > 8 || opt->chunk < 0 ||
      opt->adjoint_segment < 0 || opt->refine_max < 0 || opt->refine_max > 16)
    return NEGF_ERR_ARG;
  if (!sigma_valid(opt, dev->block)) return NEGF_ERR_ARG;
  if (dev->iface_rows < 0 || dev->iface_rows > dev->block || dev->iface_cols < 0 ||
      dev->iface_cols > dev->block)
    return NEGF_ERR_ARG;
  if (!V_bar) return NEGF_ERR_ARG;
  const int b = dev->block, N = dev->n_slabs;
  const size_t NB = (size_t)N * b;
  const int A = sigma_width(opt);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n_pts == 0) {
    return cudaMemsetAsync(V_bar, 0, NB * sizeof(double), s) == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
  }
  if (!E || !sys_idx || !sigma_R || !sigma_L || !status) return NEGF_ERR_ARG;
  if ((scat_R == nullptr) != (scat_L == nullptr)) return NEGF_ERR_ARG;
  if (scat_R && (e_idx ? n_rows < 1 : n_rows < n_pts)) return NEGF_ERR_ARG;
  const bool ckpt = checkpoints != nullptr;
  const int C = adjoint_chunk(dev, n_pts, opt, ckpt);
  if (!ws || ws_bytes < adjoint_bytes(dev, C, opt, ckpt)) return NEGF_ERR_NOMEM;
  if (cudaMemsetAsync(status, 0, (size_t)n_pts * sizeof(int32_t), s) != cudaSuccess)
    return NEGF_ERR_CUDA;
  const size_t bb = (size_t)b * b;
  for (int p0 = 0; p0 < n_pts; p0 += C) {
    const int P = std::min(C, n_pts - p0);
    AdjArgs a;
    a.dev = dev;
    a.E = E + p0;
    a.sys = sys_idx + p0;
    a.V = V;
    a.sigR = reinterpret_cast<const z64*>(sigma_R) + (size_t)p0 * 2 * bb;
    a.sigL = reinterpret_cast<const z64*>(sigma_L) + (size_t)p0 * 2 * bb;
    a.e_idx = e_idx ? e_idx + p0 : nullptr;
    a.n_rows = n_rows;
    a.scatR = scat_R ? reinterpret_cast<const z64*>(scat_R) + (e_idx ? 0 : (size_t)p0 * NB * A)
                     : nullptr;
    a.scatL = scat_L ? reinterpret_cast<const z64*>(scat_L) + (e_idx ? 0 : (size_t)p0 * NB * A)
                     : nullptr;
    a.A = A;
    a.ckpt = static_cast<const z64*>(checkpoints);
    a.n_tot = n_pts;
    a.p0 = p0;
    a.opt = opt;
    a.nbar = density_bar ? density_bar + (size_t)p0 * NB : nullptr;
    a.jbar = (current_bar && N > 1) ? current_bar + (size_t)p0 * (N - 1) : nullptr;
    a.Vbar = V_bar;
    a.accumulate = p0 > 0;
    a.status = status + p0;
    negf_status r = adjoint_chunk_run(a, P, static_cast<char*>(ws), s);
    if (r != NEGF_OK) return r;
  }
  return NEGF_OK;
}
