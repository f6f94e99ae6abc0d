// C ABI of the RGF library (include/negf.h): argument validation, workspace layout and the
// host-side driver of the batched sweeps.  Every numerical step runs in this library's kernels.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "engine.cuh"
#include "profile.cuh"
#include "rgf_kernels.cuh"

using namespace negf;

namespace {

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return note_error(e_), NEGF_ERR_CUDA; \
  } while (0)

const BMc<double> kNone{nullptr, 0, nullptr, 0};

// Bump allocator over the caller's workspace; with base == nullptr it only measures.
struct Carver {
  char* base;
  size_t off;
  template <class T>
  T* take(size_t n) {
    size_t a = (off + 255) & ~size_t(255);
    off = a + n * sizeof(T);
    return base ? reinterpret_cast<T*>(base + a) : nullptr;
  }
};

constexpr size_t kDefaultBudget = 24ull << 30;

bool valid_dev(const negf_device* d) {
  if (!d || d->n_sys < 1 || d->n_slabs < 1 || d->block < 1 || !d->H_diag) return false;
  if (d->n_slabs > 1 && !d->H_up) return false;
  if (d->iface_rows < 0 || d->iface_rows > d->block || d->iface_cols < 0 ||
      d->iface_cols > d->block)
    return false;
  return true;
}

bool valid_opt(const negf_options* o) {
  if (!o) return false;
  if (!(o->eta_lead >= 0.0) || !(o->eta_device >= 0.0) || !(o->kT > 0.0)) return false;
  if (!(o->sr_tol > 0.0) || o->sr_max_iter < 1 || o->sr_max_iter > 100000) return false;
  if (!prec_valid(o->precision)) return false;
  if (o->lead_precision != NEGF_PREC_AUTO && !prec_valid(o->lead_precision)) return false;
  if (o->refine_steps < 0 || o->refine_steps > 8 || o->chunk < 0) return false;
  if (o->refine_max < 0 || o->refine_max > 16) return false;
  if (o->sr_host_check < 0 || o->adjoint_segment < 0) return false;
  if (o->sigma_structure != NEGF_SIGMA_ORBITAL_DIAG && o->sigma_structure != NEGF_SIGMA_ATOM_BLOCK)
    return false;
  return true;
}

// ---------------------------------------------------------------- workspace layouts
struct LeadWs {
  z64 *eps_s, *eps, *al, *be, *al2, *be2, *g, *ag, *bg, *T1, *M;
  double* scale;
  int32_t *active, *iters, *item_status, *n_active, *sys, *act_side;
  EngineWs eng;
};

void carve_lead(Carver& c, int P, int b, const negf_options* opt, LeadWs& w) {
  const size_t bb = (size_t)b * b, Q = 2 * (size_t)P;
  w.eps_s = c.take<z64>(Q * bb);
  w.eps = c.take<z64>(Q * bb);
  w.al = c.take<z64>(Q * bb);
  w.be = c.take<z64>(Q * bb);
  w.al2 = c.take<z64>(Q * bb);
  w.be2 = c.take<z64>(Q * bb);
  w.g = c.take<z64>(Q * bb);
  w.ag = c.take<z64>(Q * bb);
  w.bg = c.take<z64>(Q * bb);
  w.T1 = c.take<z64>(Q * bb);
  w.M = c.take<z64>(Q * bb);
  w.scale = c.take<double>(Q);
  w.active = c.take<int32_t>(Q);
  w.iters = c.take<int32_t>(Q);
  w.item_status = c.take<int32_t>(Q);
  w.n_active = c.take<int32_t>(1);
  w.sys = c.take<int32_t>((size_t)P);
  w.act_side = c.take<int32_t>(Q);
  carve_engine(c.base ? c.base : nullptr, c.off, (int)Q, b, lead_precision(opt, b), w.eng);
}

struct RgfWs {
  int32_t *sys, *erow;
  z64 *g, *gl, *Lb;
  z64 *Y, *K, *Vt, *S, *W, *LW, *Gn, *Qm, *U, *Mt;
  EngineWs eng;
};

void carve_rgf(Carver& c, int P, int b, int N, const negf_options* opt, RgfWs& w) {
  const size_t bb = (size_t)b * b, PB = (size_t)P * bb;
  w.sys = c.take<int32_t>((size_t)P);
  w.erow = c.take<int32_t>((size_t)P);
  w.g = c.take<z64>((size_t)N * PB);
  w.gl = c.take<z64>((size_t)N * PB);
  w.Lb = c.take<z64>((size_t)std::max(N - 1, 1) * PB);
  w.Y = c.take<z64>(PB);
  w.K = c.take<z64>(PB);
  w.Vt = c.take<z64>(PB);
  w.S = c.take<z64>(PB);
  w.W = c.take<z64>(PB);
  w.LW = c.take<z64>(PB);
  w.Gn = c.take<z64>(PB);
  w.Qm = c.take<z64>(PB);
  w.U = c.take<z64>(PB);
  w.Mt = c.take<z64>(PB);
  carve_engine(c.base, c.off, P, b, opt->precision, w.eng);
}

size_t lead_bytes(int P, int b, const negf_options* o) {
  Carver c{nullptr, 0};
  LeadWs w;
  carve_lead(c, P, b, o, w);
  return c.off + 256;
}
size_t rgf_bytes(int P, int b, int N, const negf_options* o) {
  Carver c{nullptr, 0};
  RgfWs w;
  carve_rgf(c, P, b, N, o, w);
  return c.off + 256;
}

// Points per chunk; capped so that 2 x chunk batch items fit a grid's z/y extent.
constexpr int kMaxChunk = 16384;
int pick_chunk(int n_pts, const negf_options* o, size_t per_pt) {
  if (o->chunk > 0) return std::max(1, std::min(std::min(o->chunk, n_pts), kMaxChunk));
  size_t c = std::max<size_t>(1, kDefaultBudget / std::max<size_t>(per_pt, 1));
  c = std::min<size_t>(c, (size_t)kMaxChunk);
  return (int)std::max<size_t>(1, std::min<size_t>(c, (size_t)n_pts));
}

int lead_chunk(const negf_device* d, int n_pts, const negf_options* o) {
  size_t per = lead_bytes(2, d->block, o) - lead_bytes(1, d->block, o);
  return pick_chunk(n_pts, o, per);
}
int rgf_chunk(const negf_device* d, int n_pts, const negf_options* o) {
  size_t per = rgf_bytes(2, d->block, d->n_slabs, o) - rgf_bytes(1, d->block, d->n_slabs, o);
  return pick_chunk(n_pts, o, per);
}

inline BM<double> flat(z64* base, size_t bb, int b) {
  return BM<double>{base, (long long)bb, nullptr, b};
}

// ---------------------------------------------------------------- lead self-energies
negf_status lead_chunk_run(const negf_device* dev, int P, const double* E, const int32_t* sys_in,
                           const negf_options* opt, z64* sigR, z64* sigL, int32_t* iters,
                           int32_t* status, char* wsbase, cudaStream_t s) {
  const int b = dev->block, N = dev->n_slabs;
  const size_t bb = (size_t)b * b;
  const int Q = 2 * P;
  const z64 one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  if (N < 2) {  // no hopping to continue the end slabs: flat leads
    CK(cudaMemsetAsync(sigR, 0, (size_t)Q * bb * sizeof(z64), s));
    CK(cudaMemsetAsync(sigL, 0, (size_t)Q * bb * sizeof(z64), s));
    if (iters) CK(cudaMemsetAsync(iters, 0, (size_t)Q * sizeof(int32_t), s));
    return NEGF_OK;
  }
  Carver c{wsbase, 0};
  LeadWs w;
  carve_lead(c, P, b, opt, w);
  Engine eng(s, lead_precision(opt, b), opt->refine_steps, refine_limit(opt), w.eng, b,
             dev->n_sys);
  CK(eng.timeout_reset());
  CK(launch_clamp_index(s, P, sys_in, dev->n_sys, w.sys, status));
  const int32_t* sys = w.sys;
  BMc<double> Hd{reinterpret_cast<const z64*>(dev->H_diag), (long long)(N * bb), sys, b};
  BMc<double> Hu{reinterpret_cast<const z64*>(dev->H_up), (long long)((N - 1) * bb), sys, b};
  CK(launch_sr_init(s, Q, b, N, Hd, Hu, flat(w.eps_s, bb, b), flat(w.eps, bb, b),
                    flat(w.al, bb, b), flat(w.be, bb, b), w.scale));
  CK(launch_fill_i32(s, w.active, Q, 1));
  CK(launch_fill_i32(s, w.iters, Q, 0));
  CK(launch_fill_i32(s, w.item_status, Q, 0));
  // Interface couplings: tau is nonzero only on its last ir rows R and first ic columns C.  Then
  // alpha_n keeps the support of alpha_0 (C x R for the left lead, tau_L^H; R x C for the right
  // lead, tau_R) and beta_n the transposed one through every doubling step, since
  // alpha' = alpha g alpha and beta' = beta g beta.  With Ra x Ca the support of alpha, the step
  //   ag[Ra, :] = alpha[Ra, Ca] g[Ca, :]      bg[Ca, :] = beta[Ca, Ra] g[Ra, :]
  //   eps_s[Ra, Ra], eps[Ra, Ra] += ag[Ra, Ca] beta[Ca, Ra]
  //   eps[Ca, Ca] += bg[Ca, Ra] alpha[Ra, Ca]
  //   alpha'[Ra, Ca] = ag[Ra, Ra] alpha[Ra, Ca]      beta'[Ca, Ra] = bg[Ca, Ca] beta[Ca, Ra]
  // contracts over r or c instead of b; the two leads are separate launches (their supports
  // differ), each with its own copy of the convergence mask.
  const int ir = dev->iface_rows > 0 ? dev->iface_rows : b;
  const int ic = dev->iface_cols > 0 ? dev->iface_cols : b;
  const bool iface = ir < b || ic < b;
  const int ra0[2] = {0, b - ir}, nra[2] = {ic, ir};  // alpha rows: C (left), R (right)
  const int ca0[2] = {b - ir, 0}, nca[2] = {ir, ic};  // alpha columns: R (left), C (right)
  // item (p, side) of a [P][2][b][b] array, from row r0 and column c0
  auto sub = [&](z64* base, int side, int r0, int c0) {
    return BM<double>{base + side * bb + (size_t)r0 * b + c0, (long long)(2 * bb), nullptr, b};
  };
  auto subc = [&](z64* base, int side, int r0, int c0) { return cst(sub(base, side, r0, c0)); };
  if (iface) {
    CK(launch_fill_i32(s, w.act_side, Q, 1));
    // alpha', beta' are written on their supports only: the rest of both buffers stays zero
    CK(cudaMemsetAsync(w.al2, 0, (size_t)Q * bb * sizeof(z64), s));
    CK(cudaMemsetAsync(w.be2, 0, (size_t)Q * bb * sizeof(z64), s));
  }
  z64 *al = w.al, *be = w.be, *al2 = w.al2, *be2 = w.be2;
  const double eta = opt->eta_lead;
  int32_t h_active = Q;
  for (int it = 1; it <= opt->sr_max_iter; ++it) {
    const int32_t* act = w.active;
    // the workspace is carved for lead_precision(opt, b), the widest tier of the schedule
    eng.prec = lead_step_precision(opt, b, it);
    CK(launch_zminus(s, Q, b, E, eta, cst(flat(w.eps, bb, b)), flat(w.M, bb, b), act));
    CK(eng.inv(Q, flat(w.M, bb, b), flat(w.g, bb, b), w.item_status, act));
    if (!iface) {
      CK(eng.gemm(Q, b, b, b, one, cst(flat(al, bb, b)), OP_N, cst(flat(w.g, bb, b)), OP_N,
                  zero, flat(w.ag, bb, b), zero, kNone, act));
      CK(eng.gemm(Q, b, b, b, one, cst(flat(be, bb, b)), OP_N, cst(flat(w.g, bb, b)), OP_N,
                  zero, flat(w.bg, bb, b), zero, kNone, act));
      CK(eng.gemm(Q, b, b, b, one, cst(flat(w.ag, bb, b)), OP_N, cst(flat(be, bb, b)), OP_N,
                  zero, flat(w.T1, bb, b), zero, kNone, act));
      CK(launch_add2(s, Q, b, cst(flat(w.T1, bb, b)), flat(w.eps_s, bb, b), flat(w.eps, bb, b),
                     0, b, 0, b, act));
      CK(eng.gemm(Q, b, b, b, one, cst(flat(w.bg, bb, b)), OP_N, cst(flat(al, bb, b)), OP_N, one,
                  flat(w.eps, bb, b), zero, kNone, act));
      CK(eng.gemm(Q, b, b, b, one, cst(flat(w.ag, bb, b)), OP_N, cst(flat(al, bb, b)), OP_N,
                  zero, flat(al2, bb, b), zero, kNone, act));
      CK(eng.gemm(Q, b, b, b, one, cst(flat(w.bg, bb, b)), OP_N, cst(flat(be, bb, b)), OP_N,
                  zero, flat(be2, bb, b), zero, kNone, act));
    } else {
      for (int sd = 0; sd < 2; ++sd) {
        const int32_t* as = w.act_side + (size_t)sd * P;
        const int r0 = ra0[sd], nr = nra[sd], c0 = ca0[sd], nc = nca[sd];
        CK(eng.gemm(P, nr, b, nc, one, subc(al, sd, r0, c0), OP_N, subc(w.g, sd, c0, 0), OP_N,
                    zero, sub(w.ag, sd, r0, 0), zero, kNone, as));
        CK(eng.gemm(P, nc, b, nr, one, subc(be, sd, c0, r0), OP_N, subc(w.g, sd, r0, 0), OP_N,
                    zero, sub(w.bg, sd, c0, 0), zero, kNone, as));
        CK(eng.gemm(P, nr, nr, nc, one, subc(w.ag, sd, r0, c0), OP_N, subc(be, sd, c0, r0), OP_N,
                    zero, sub(w.T1, sd, r0, r0), zero, kNone, as));
        CK(eng.gemm(P, nc, nc, nr, one, subc(w.bg, sd, c0, r0), OP_N, subc(al, sd, r0, c0), OP_N,
                    one, sub(w.eps, sd, c0, c0), zero, kNone, as));
        CK(eng.gemm(P, nr, nc, nr, one, subc(w.ag, sd, r0, r0), OP_N, subc(al, sd, r0, c0), OP_N,
                    zero, sub(al2, sd, r0, c0), zero, kNone, as));
        CK(eng.gemm(P, nc, nr, nc, one, subc(w.bg, sd, c0, c0), OP_N, subc(be, sd, c0, r0), OP_N,
                    zero, sub(be2, sd, c0, r0), zero, kNone, as));
      }
      CK(launch_add2(s, Q, b, cst(flat(w.T1, bb, b)), flat(w.eps_s, bb, b), flat(w.eps, bb, b),
                     ra0[0], nra[0], ra0[1], nra[1], act));
    }
    std::swap(al, al2);
    std::swap(be, be2);
    CK(cudaMemsetAsync(w.n_active, 0, sizeof(int32_t), s));
    CK(launch_sr_check(s, Q, b, it, opt->sr_tol, cst(flat(al, bb, b)), cst(flat(be, bb, b)),
                       w.scale, w.active, w.iters, w.n_active, iface ? w.act_side : nullptr));
    const int chk = opt->sr_host_check;
    if (chk > 0 && it >= 8 && (it % chk == 0 || it == opt->sr_max_iter)) {
      CK(cudaMemcpyAsync(&h_active, w.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h_active == 0) break;
    }
  }
  // surface Green's functions g_s = (z - eps_s)^-1 for every item
  eng.prec = lead_step_precision(opt, b, 0);
  CK(launch_zminus(s, Q, b, E, eta, cst(flat(w.eps_s, bb, b)), flat(w.M, bb, b), nullptr));
  CK(eng.inv(Q, flat(w.M, bb, b), flat(w.g, bb, b), w.item_status, nullptr));
  // left:  Sigma_L = tau_L^H g_L tau_L;  right: Sigma_R = tau_R g_R tau_R^H
  BMc<double> tauL{reinterpret_cast<const z64*>(dev->H_up), (long long)((N - 1) * bb), sys, b};
  BMc<double> tauR = tauL;
  tauR.p += (size_t)(N - 2) * bb;
  if (!iface) {
    BM<double> gL{w.g, (long long)(2 * bb), nullptr, b}, gR{w.g + bb, (long long)(2 * bb), nullptr, b};
    BM<double> tL{w.T1, (long long)(2 * bb), nullptr, b}, tR{w.T1 + bb, (long long)(2 * bb), nullptr, b};
    BM<double> sL{sigR, (long long)(2 * bb), nullptr, b}, sRr{sigR + bb, (long long)(2 * bb), nullptr, b};
    CK(eng.gemm(P, b, b, b, one, cst(gL), OP_N, tauL, OP_N, zero, tL, zero, kNone, nullptr));
    CK(eng.gemm(P, b, b, b, one, tauL, OP_C, cst(tL), OP_N, zero, sL, zero, kNone, nullptr));
    CK(eng.gemm(P, b, b, b, one, cst(gR), OP_N, tauR, OP_C, zero, tR, zero, kNone, nullptr));
    CK(eng.gemm(P, b, b, b, one, tauR, OP_N, cst(tR), OP_N, zero, sRr, zero, kNone, nullptr));
  } else {
    // with T = tau[R, C]:  Sigma_L[C, C] = T^H g_L[R, R] T,  Sigma_R[R, R] = T g_R[C, C] T^H
    tauL.p += (size_t)(b - ir) * b;
    tauR.p += (size_t)(b - ir) * b;
    const int R0 = b - ir;
    CK(cudaMemsetAsync(sigR, 0, (size_t)Q * bb * sizeof(z64), s));
    CK(eng.gemm(P, ir, ic, ir, one, subc(w.g, 0, R0, R0), OP_N, tauL, OP_N, zero,
                sub(w.T1, 0, R0, 0), zero, kNone, nullptr));
    CK(eng.gemm(P, ic, ic, ir, one, tauL, OP_C, subc(w.T1, 0, R0, 0), OP_N, zero,
                sub(sigR, 0, 0, 0), zero, kNone, nullptr));
    CK(eng.gemm(P, ic, ir, ic, one, subc(w.g, 1, 0, 0), OP_N, tauR, OP_C, zero,
                sub(w.T1, 1, 0, R0), zero, kNone, nullptr));
    CK(eng.gemm(P, ir, ir, ic, one, tauR, OP_N, subc(w.T1, 1, 0, R0), OP_N, zero,
                sub(sigR, 1, R0, R0), zero, kNone, nullptr));
  }
  CK(launch_gamma(s, Q, b, cst(flat(sigR, bb, b)), flat(w.M, bb, b), nullptr));
  CK(launch_lead_lesser(s, Q, b, E, opt->mu_L, opt->mu_R, opt->kT, cst(flat(w.M, bb, b)),
                        flat(sigL, bb, b)));
  CK(launch_sr_status(s, P, w.active, w.item_status, w.iters, iters, opt->sr_max_iter, status));
  CK(launch_check_finite(s, reinterpret_cast<const double*>(sigR), (long long)4 * bb, P, status));
  CK(eng.timeout_flag(P, status));
  return NEGF_OK;
}

// ---------------------------------------------------------------- RGF sweeps
struct RgfArgs {
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
  double* density;
  double* current;
  double* transmission;
  z64* dGR;
  z64* dGL;
  int A;  // scattering self-energy block width (1: orbital-diagonal)
  int32_t* status;
  z64* ckpt;  // sweep checkpoints for negf_rgf_adjoint (nullable), [5][N][n_tot][b][b]
  int n_tot, p0;
};

negf_status rgf_chunk_run(const RgfArgs& a, int P, char* wsbase, cudaStream_t s) {
  const negf_device* dev = a.dev;
  const int b = dev->block, N = dev->n_slabs;
  const size_t bb = (size_t)b * b;
  const int NB = N * b;
  const z64 one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0), two = mkc(2.0, 0.0);
  Carver c{wsbase, 0};
  RgfWs w;
  carve_rgf(c, P, b, N, a.opt, w);
  Engine eng(s, a.opt->precision, a.opt->refine_steps, refine_limit(a.opt), w.eng, b,
             dev->n_sys);
  CK(eng.timeout_reset());
  const double eta = a.opt->eta_device;
  CK(launch_clamp_index(s, P, a.sys, dev->n_sys, w.sys, a.status));
  const int32_t* sysc = w.sys;
  const int32_t* erow = nullptr;
  if (a.scatR && a.e_idx) {
    CK(launch_clamp_index(s, P, a.e_idx, a.n_rows, w.erow, a.status));
    erow = w.erow;
  }
  auto Hd = [&](int i) {
    return BMc<double>{reinterpret_cast<const z64*>(dev->H_diag) + (size_t)i * bb,
                       (long long)(N * bb), sysc, b};
  };
  auto Hu = [&](int i) {
    return BMc<double>{reinterpret_cast<const z64*>(dev->H_up) + (size_t)i * bb,
                       (long long)((N - 1) * bb), sysc, b};
  };
  BMc<double> SigL_R{a.sigR, (long long)(2 * bb), nullptr, b};
  BMc<double> SigR_R{a.sigR + bb, (long long)(2 * bb), nullptr, b};
  BMc<double> SigL_L{a.sigL, (long long)(2 * bb), nullptr, b};
  BMc<double> SigR_L{a.sigL + bb, (long long)(2 * bb), nullptr, b};
  std::vector<z64*> G(N), GL(N);
  for (int i = 0; i < N; ++i) {
    G[i] = w.g + (size_t)i * P * bb;
    GL[i] = w.gl + (size_t)i * P * bb;
  }
  auto F = [&](z64* p) { return flat(p, bb, b); };
  auto Fc = [&](z64* p) { return cst(flat(p, bb, b)); };
  auto Lb = [&](int i) { return w.Lb + (size_t)i * P * bb; };
  // Interface couplings: H_{i,i+1} is nonzero only in its last ir rows and first ic columns
  // (ir = ic = b: dense).  Views of the b x b blocks (same batch stride and leading dimension):
  // columns from c0, rows from r0, and the ir x ic support of a hopping block.
  const int ir = dev->iface_rows > 0 ? dev->iface_rows : b;
  const int ic = dev->iface_cols > 0 ? dev->iface_cols : b;
  auto cview = [](BMc<double> X, int c0) {
    X.p += c0;
    return X;
  };
  auto rview = [](BMc<double> X, int r0) {
    X.p += (long long)r0 * X.ld;
    return X;
  };
  auto bcview = [](BM<double> X, int c0) {
    X.p += c0;
    return X;
  };
  auto tview = [&](BMc<double> X) { return rview(X, b - ir); };

  // ---- forward sweep: left-connected g_i, g^<_i
  for (int i = 0; i < N; ++i) {
    const bool first = (i == 0), last = (i == N - 1);
    BMc<double> Y = kNone;
    if (!first) {
      // L_{i-1} = g_{i-1} t_{i-1} (kept for the backward sweep);  Y = t^H L.  Interface mode:
      // t = E_R T E_C^T, so only L[:, C] = g[:, R] T and Y[C, C] = T^H L[R, C] are formed.
      CK(eng.gemm(P, b, ic, ir, one, cview(Fc(G[i - 1]), b - ir), OP_N, tview(Hu(i - 1)), OP_N,
                  zero, F(Lb(i - 1)), zero, kNone, nullptr));
      CK(eng.gemm(P, ic, ic, ir, one, tview(Hu(i - 1)), OP_C, rview(Fc(Lb(i - 1)), b - ir), OP_N,
                  zero, F(w.Y), zero, kNone, nullptr));
      Y = Fc(w.Y);
    }
    CK(launch_assemble(s, P, b, a.E, eta, Hd(i), a.V ? a.V + (size_t)i * b : nullptr,
                       a.scatR ? a.scatR + (size_t)i * b * a.A : nullptr, (long long)NB * a.A,
                       a.A, erow, Y, ic,
                       first ? SigL_R : kNone, last ? SigR_R : kNone, F(w.Mt), nullptr));
    CK(eng.inv(P, F(w.Mt), F(G[i]), a.status, nullptr));
    bool have_prev = false;
    if (!first) {
      // g^<_i = K g^<_{i-1} K^H with K = g_i t_{i-1}^H; interface mode: only K[:, R] =
      // g_i[:, C] T^H, then Vt = g^<_{i-1}[:, R] K[:, R]^H and g^<_i = K[:, R] Vt[R, :]
      CK(eng.gemm(P, b, ir, ic, one, Fc(G[i]), OP_N, tview(Hu(i - 1)), OP_C, zero,
                  bcview(F(w.K), b - ir), zero, kNone, nullptr));
      CK(eng.gemm(P, b, b, ir, one, cview(Fc(GL[i - 1]), b - ir), OP_N, cview(Fc(w.K), b - ir),
                  OP_C, zero, F(w.Vt), zero, kNone, nullptr));
      CK(eng.gemm(P, b, b, ir, one, cview(Fc(w.K), b - ir), OP_N, rview(Fc(w.Vt), b - ir), OP_N,
                  zero, F(GL[i]), zero, kNone, nullptr));
      have_prev = true;
    }
    const bool has_src = first || last || a.scatL != nullptr;
    if (has_src) {
      // + g_i S_i g_i^H with S_i = diag(Sigma^<_scat) + lead Sigma^< on the end slabs
      CK(launch_source(s, P, b, a.scatL ? a.scatL + (size_t)i * b * a.A : nullptr,
                       (long long)NB * a.A, a.A, erow,
                       first ? SigL_L : kNone, last ? SigR_L : kNone, F(w.S), nullptr));
      CK(eng.gemm(P, b, b, b, one, Fc(G[i]), OP_N, Fc(w.S), OP_N, zero, F(w.W), zero, kNone,
                  nullptr));
      CK(eng.gemm(P, b, b, b, one, Fc(w.W), OP_N, Fc(G[i]), OP_C, have_prev ? one : zero,
                  F(GL[i]), zero, kNone, nullptr));
    } else if (!have_prev) {
      CK(cudaMemsetAsync(GL[i], 0, (size_t)P * bb * sizeof(z64), s));
    }
  }

  // ---- checkpoints of the forward sweep (g_i, g^<_i are overwritten by the backward sweep)
  const size_t blk = (size_t)P * bb * sizeof(z64);
  auto ckp = [&](int k, int i) { return a.ckpt + ckpt_offset(k, i, N, a.n_tot, a.p0, bb); };
  if (a.ckpt) {
    for (int i = 0; i < N; ++i) {
      CK(cudaMemcpyAsync(ckp(CK_G_FWD, i), G[i], blk, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(ckp(CK_GL_FWD, i), GL[i], blk, cudaMemcpyDeviceToDevice, s));
      if (i + 1 < N) CK(cudaMemcpyAsync(ckp(CK_L, i), Lb(i), blk, cudaMemcpyDeviceToDevice, s));
    }
  }

  // ---- transmission from G_NN = g_N and Gamma_R
  if (a.transmission) {
    CK(launch_gamma(s, P, b, SigR_R, F(w.S), nullptr));
    CK(eng.gemm(P, b, b, b, one, Fc(w.S), OP_N, Fc(G[N - 1]), OP_N, zero, F(w.W), zero, kNone,
                nullptr));
    CK(eng.gemm(P, b, b, b, one, Fc(G[N - 1]), OP_N, Fc(w.S), OP_N, zero, F(w.LW), zero, kNone,
                nullptr));
    CK(launch_transmission(s, P, b, Fc(w.S), Fc(G[N - 1]), Fc(w.W), Fc(w.LW), a.transmission,
                           nullptr));
  }
  CK(launch_slab_obs(s, P, b, N - 1, NB, a.A, Fc(G[N - 1]), Fc(GL[N - 1]), a.density, a.dGR,
                     a.dGL,
                     nullptr));

  // ---- backward sweep: G_ii, G^<_ii, G^<_{i+1,i}
  z64* spare = w.Gn;
  for (int i = N - 2; i >= 0; --i) {
    z64* L = Lb(i);
    // W = G_{i+1} t_i^H;  LW = L W;  G_i = g_i + LW g_i.  Interface mode (L has columns C,
    // t_i^H rows C and columns R): W[:, R] = G_{i+1}[:, C] T^H, LW[:, R] = L[:, C] W[C, R],
    // G_i = g_i + LW[:, R] g_i[R, :]
    CK(eng.gemm(P, b, ir, ic, one, Fc(G[i + 1]), OP_N, tview(Hu(i)), OP_C, zero,
                bcview(F(w.W), b - ir), zero, kNone, nullptr));
    CK(eng.gemm(P, b, ir, ic, one, Fc(L), OP_N, cview(Fc(w.W), b - ir), OP_N, zero,
                bcview(F(w.LW), b - ir), zero, kNone, nullptr));
    CK(eng.gemm(P, b, b, ir, one, cview(Fc(w.LW), b - ir), OP_N, rview(Fc(G[i]), b - ir), OP_N,
                zero, F(spare), one, Fc(G[i]), nullptr));
    // Q = G^<_{i+1} L^H;  U = 2 W g^<_i + Q;  G^<_{i+1,i} = (U + Q) / 2  (interface mode:
    // Q = G^<_{i+1}[:, C] L[:, C]^H, U = 2 W[:, R] g^<_i[R, :] + Q)
    CK(eng.gemm(P, b, b, ic, one, Fc(GL[i + 1]), OP_N, Fc(L), OP_C, zero, F(w.Qm), zero, kNone,
                nullptr));
    CK(eng.gemm(P, b, b, ir, two, cview(Fc(w.W), b - ir), OP_N, rview(Fc(GL[i]), b - ir), OP_N,
                zero, F(w.U), one, Fc(w.Qm), nullptr));
    if (a.current)
      CK(launch_bond_current(s, P, b, Hu(i), Fc(w.U), Fc(w.Qm), a.current + i, N - 1, nullptr));
    // G^<_ii = AH(g^<_i + L U)  (interface mode: L[:, C] U[C, :])
    CK(eng.gemm(P, b, b, ic, one, Fc(L), OP_N, Fc(w.U), OP_N, zero, F(w.Mt), one, Fc(GL[i]),
                nullptr));
    CK(launch_antiherm(s, P, b, Fc(w.Mt), F(GL[i]), nullptr));
    std::swap(G[i], spare);
    CK(launch_slab_obs(s, P, b, i, NB, a.A, Fc(G[i]), Fc(GL[i]), a.density, a.dGR, a.dGL,
                       nullptr));
  }
  if (a.ckpt) {
    for (int i = 0; i < N; ++i) {
      CK(cudaMemcpyAsync(ckp(CK_G, i), G[i], blk, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(ckp(CK_GL, i), GL[i], blk, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (a.density) CK(launch_check_finite(s, a.density, NB, P, a.status));
  if (a.current && N > 1) CK(launch_check_finite(s, a.current, N - 1, P, a.status));
  if (a.transmission) CK(launch_check_finite(s, a.transmission, 1, P, a.status));
  CK(eng.timeout_flag(P, a.status));
  return NEGF_OK;
}

}  // namespace

// ============================================================================ public ABI
extern "C" {

void negf_default_options(negf_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eta_lead = 1e-6;
  o->eta_device = 1e-6;
  o->mu_L = 0.1;
  o->mu_R = -0.1;
  o->kT = 0.025852;
  o->sr_tol = 1e-13;
  o->sr_max_iter = 100;
  o->precision = NEGF_PREC_FP64;
  o->refine_steps = 2;
  o->chunk = 0;
  o->sr_host_check = 4;
  o->adjoint_segment = 0;
  o->lead_precision = NEGF_PREC_AUTO;
  o->refine_max = 6;
  o->sigma_structure = NEGF_SIGMA_ORBITAL_DIAG;
  o->atom_orbitals = 10;
}

int32_t negf_abi_version(void) { return NEGF_ABI_VERSION; }

long long negf_fp64_fallback_count(void) { return engine_fp64_fallbacks(); }

void negf_debug_fail_waits(int32_t on) { engine_fail_waits(on); }

const char* negf_status_string(negf_status s) {
  switch (s) {
    case NEGF_OK: return "ok";
    case NEGF_ERR_ARG: return "invalid argument";
    case NEGF_ERR_CUDA: return "CUDA error";
    case NEGF_ERR_NOMEM: return "workspace too small";
    case NEGF_ERR_NOT_CONVERGED: return "lead decimation did not converge";
    case NEGF_ERR_SINGULAR: return "zero pivot in a block inverse";
    case NEGF_ERR_NONFINITE: return "non-finite output";
    case NEGF_ERR_TIMEOUT: return "bounded device wait timed out";
    case NEGF_ERR_UNSUPPORTED: return "unsupported option or size";
  }
  return "unknown status";
}

size_t negf_workspace_size(const negf_device* dev, int32_t n_pts, const negf_options* opt,
                           int32_t which) {
  if (!valid_dev(dev) || !valid_opt(opt) || n_pts < 1) return 0;
  if (which == NEGF_WS_LEAD ? !engine_supports(lead_precision(opt, dev->block), dev->block)
                            : !engine_supports(opt->precision, dev->block))
    return 0;
  const int b = dev->block, N = dev->n_slabs;
  switch (which) {
    case NEGF_WS_LEAD: return lead_bytes(lead_chunk(dev, n_pts, opt), b, opt);
    case NEGF_WS_RGF: return rgf_bytes(rgf_chunk(dev, n_pts, opt), b, N, opt);
    case NEGF_WS_ADJOINT:
      return adjoint_bytes(dev, adjoint_chunk(dev, n_pts, opt, false), opt, false);
    case NEGF_WS_ADJOINT_CKPT:
      return adjoint_bytes(dev, adjoint_chunk(dev, n_pts, opt, true), opt, true);
  }
  return 0;
}

size_t negf_checkpoint_bytes(const negf_device* dev, int32_t n_pts) {
  if (!valid_dev(dev) || n_pts < 1) return 0;
  const size_t bb = (size_t)dev->block * dev->block;
  return ckpt_offset(CK_KINDS, 0, dev->n_slabs, n_pts, 0, bb) * sizeof(z64);
}

negf_status negf_lead_selfenergy(const negf_device* dev, int32_t n_pts, const double* E,
                                 const int32_t* sys_idx, const negf_options* opt,
                                 double* sigma_R, double* sigma_L, int32_t* iters,
                                 int32_t* status, void* ws, size_t ws_bytes, void* stream) {
  if (!valid_dev(dev) || !valid_opt(opt) || n_pts < 0) return NEGF_ERR_ARG;
  if (!engine_supports(lead_precision(opt, dev->block), dev->block)) return NEGF_ERR_UNSUPPORTED;
  if (n_pts == 0) return NEGF_OK;
  if (!E || !sys_idx || !sigma_R || !sigma_L || !status) return NEGF_ERR_ARG;
  const int b = dev->block;
  const int C = lead_chunk(dev, n_pts, opt);
  if (dev->n_slabs > 1 && (!ws || ws_bytes < lead_bytes(C, b, opt))) return NEGF_ERR_NOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bb = (size_t)b * b;
  if (cudaMemsetAsync(status, 0, (size_t)n_pts * sizeof(int32_t), s) != cudaSuccess)
    return NEGF_ERR_CUDA;
  for (int p0 = 0; p0 < n_pts; p0 += C) {
    const int P = std::min(C, n_pts - p0);
    negf_status r = lead_chunk_run(dev, P, E + p0, sys_idx + p0, opt,
                                   reinterpret_cast<z64*>(sigma_R) + (size_t)p0 * 2 * bb,
                                   reinterpret_cast<z64*>(sigma_L) + (size_t)p0 * 2 * bb,
                                   iters ? iters + 2 * (size_t)p0 : nullptr, status + p0,
                                   static_cast<char*>(ws), s);
    if (r != NEGF_OK) return r;
  }
  return NEGF_OK;
}

negf_status negf_rgf_solve(const negf_device* dev, int32_t n_pts, const double* E,
                           const int32_t* sys_idx, const double* V, const double* sigma_R,
                           const double* sigma_L, const double* scat_R, const double* scat_L,
                           const int32_t* e_idx, int32_t n_rows, const negf_options* opt,
                           double* density, double* current, double* transmission,
                           double* diagGR, double* diagGL, void* checkpoints, int32_t* status,
                           void* ws, size_t ws_bytes, void* stream) {
  if (!valid_dev(dev) || !valid_opt(opt) || n_pts < 0) return NEGF_ERR_ARG;
  if (scat_R && (e_idx ? n_rows < 1 : n_rows < n_pts)) return NEGF_ERR_ARG;
  if (!sigma_valid(opt, dev->block)) return NEGF_ERR_ARG;
  if (!engine_supports(opt->precision, dev->block)) return NEGF_ERR_UNSUPPORTED;
  if (n_pts == 0) return NEGF_OK;
  if (!E || !sys_idx || !sigma_R || !sigma_L || !status) return NEGF_ERR_ARG;
  if ((scat_R == nullptr) != (scat_L == nullptr)) return NEGF_ERR_ARG;
  const int b = dev->block, N = dev->n_slabs;
  const int C = rgf_chunk(dev, n_pts, opt);
  if (!ws || ws_bytes < rgf_bytes(C, b, N, opt)) return NEGF_ERR_NOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bb = (size_t)b * b, NB = (size_t)N * b;
  const int A = sigma_width(opt);
  const size_t NBA = NB * A;  // entries of a scattering self-energy / diag-block row
  if (cudaMemsetAsync(status, 0, (size_t)n_pts * sizeof(int32_t), s) != cudaSuccess)
    return NEGF_ERR_CUDA;
  for (int p0 = 0; p0 < n_pts; p0 += C) {
    const int P = std::min(C, n_pts - p0);
    RgfArgs a;
    a.dev = dev;
    a.E = E + p0;
    a.sys = sys_idx + p0;
    a.V = V;
    a.sigR = reinterpret_cast<const z64*>(sigma_R) + (size_t)p0 * 2 * bb;
    a.sigL = reinterpret_cast<const z64*>(sigma_L) + (size_t)p0 * 2 * bb;
    a.e_idx = e_idx ? e_idx + p0 : nullptr;
    a.n_rows = n_rows;
    // without an index the scattering rows follow the points
    a.scatR = scat_R ? reinterpret_cast<const z64*>(scat_R) + (e_idx ? 0 : (size_t)p0 * NBA) : nullptr;
    a.scatL = scat_L ? reinterpret_cast<const z64*>(scat_L) + (e_idx ? 0 : (size_t)p0 * NBA) : nullptr;
    a.opt = opt;
    a.density = density ? density + (size_t)p0 * NB : nullptr;
    a.current = (current && N > 1) ? current + (size_t)p0 * (N - 1) : nullptr;
    a.transmission = transmission ? transmission + p0 : nullptr;
    a.dGR = diagGR ? reinterpret_cast<z64*>(diagGR) + (size_t)p0 * NBA : nullptr;
    a.dGL = diagGL ? reinterpret_cast<z64*>(diagGL) + (size_t)p0 * NBA : nullptr;
    a.A = A;
    a.ckpt = static_cast<z64*>(checkpoints);
    a.n_tot = n_pts;
    a.p0 = p0;
    a.status = status + p0;
    negf_status r = rgf_chunk_run(a, P, static_cast<char*>(ws), s);
    if (r != NEGF_OK) return r;
  }
  return NEGF_OK;
}

negf_status negf_integrate(int32_t n_pts, int32_t len, int32_t n_groups, const double* w,
                           const int32_t* group, const double* in, double* out, void* stream) {
  if (n_pts < 0 || len < 0 || n_groups < 1 || !w || !in || !out) return NEGF_ERR_ARG;
  if (len == 0) return NEGF_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_integrate(s, n_pts, len, n_groups, w, group, in, out) != cudaSuccess)
    return NEGF_ERR_CUDA;
  return NEGF_OK;
}

}  // extern "C"
