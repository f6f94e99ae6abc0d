// Block-operation engine of the sweeps: the batched complex GEMM and the batched block
// inverse for the precision chosen in negf_options.  FP64 form: CUDA-core GEMM and FP64
// Gauss-Jordan.  Mixed form: tensor-core GEMM of exact split-BF16 slices and an FP32
// Gauss-Jordan inverse polished by Newton-Schulz steps X <- X + X (I - M X).
#pragma once
#include <utility>

#include "common.cuh"

namespace negf {

struct EngineWs {
  // FP64 inverse scratch
  z64* invU;
  z64* invT;
  int32_t* piv;
  // mixed-precision scratch
  cx<float>* m32;    // FP32 copy of the matrices being inverted, P x b x b
  cx<float>* x32;    // FP32 inverse, P x b x b
  cx<float>* invU32;
  cx<float>* invT32;
  z64* r64;          // residual I - M X, P x b x b
  int32_t* act;      // items still refined by the current Newton-Schulz step, P
  float* rmax;       // max |I - M X| of each item after the last residual product, P
  void* tc;          // tensor-core GEMM operand slices
  size_t tc_bytes;
};

// Reserve the engine scratch for P concurrent b x b problems at `off` of `base` (base NULL:
// only advance `off`).  precision: a negf_precision value (it fixes the tensor-core slices).
void carve_engine(char* base, size_t& off, int P, int b, int precision, EngineWs& w);

// Precision tiers: FP64 on the CUDA cores, or tensor-core products of 40-, 48- or 56-bit
// fixed-point operand values.
inline bool prec_valid(int p) { return p >= NEGF_PREC_FP64 && p <= NEGF_PREC_MIXED_56; }
inline bool prec_mixed(int p) { return p >= NEGF_PREC_MIXED && p <= NEGF_PREC_MIXED_56; }
inline int prec_bits(int p) {
  return p == NEGF_PREC_MIXED ? 48 : p == NEGF_PREC_MIXED_40 ? 40 : p == NEGF_PREC_MIXED_56 ? 56 : 0;
}
// Precision of the lead decimation of b x b blocks under options o (NEGF_PREC_AUTO: FP64 when
// the sweeps are FP64, else the 56-bit tier where its products are exact (b <= 7008), else the
// 48-bit tier).
int lead_precision(const negf_options* o, int b);
// Precision of decimation step `it` (1-based; 0 = the surface Green's function and Sigma after
// the loop).  A fixed lead_precision applies to every step.  Under NEGF_PREC_AUTO in the mixed
// forms the tier falls with the step: 56 bits for steps 1-8, 48 bits for 9-14, 40 bits from 15,
// and 48 bits after the loop.  The near-singular (z - eps_n) blocks that amplify rounding by up
// to ~1e9 occur in the first steps, while the short lead segments still have isolated levels;
// a 1e-14 perturbation of g at step 5-10 moves Sigma by <= 3e-10 on the benchmark device, at
// step >= 15 by <= 3e-12.
int lead_step_precision(const negf_options* o, int b, int it);
// Newton-Schulz steps of the mixed-form inverse: always refine_steps, at most
// max(refine_steps, refine_max).
// Width A of the scattering self-energy blocks: 1 (orbital-diagonal) or the atom block size.
inline int sigma_width(const negf_options* o) {
  return o->sigma_structure == NEGF_SIGMA_ATOM_BLOCK ? o->atom_orbitals : 1;
}
// Valid sigma structure fields for blocks of b orbitals (b a whole number of atom blocks).
inline bool sigma_valid(const negf_options* o, int b) {
  if (o->sigma_structure == NEGF_SIGMA_ORBITAL_DIAG) return true;
  if (o->sigma_structure != NEGF_SIGMA_ATOM_BLOCK) return false;
  return o->atom_orbitals >= 1 && o->atom_orbitals <= 64 && b % o->atom_orbitals == 0;
}
inline int refine_limit(const negf_options* o) {
  return o->refine_max > o->refine_steps ? o->refine_max : o->refine_steps;
}

struct Engine {
  cudaStream_t s;
  int prec;        // negf_precision of every product and inverse of this engine
  int refine_min;  // mixed form: Newton-Schulz steps run for every block
  int refine_max;  // ... and at most this many for blocks whose residual stays above 2^-24
  EngineWs w;
  int b;
  int n_sys = 0;  // distinct Hamiltonians an indexed operand selects from (0 = unknown)
  Engine(cudaStream_t s_, int prec_, int rmin, int rmax_, const EngineWs& w_, int b_,
         int n_sys_ = 0)
      : s(s_), prec(prec_), refine_min(rmin), refine_max(rmax_ > rmin ? rmax_ : rmin), w(w_),
        b(b_), n_sys(n_sys_) {}
  // C = alpha op(A) op(B) + beta C + gamma D for P batch items of M x N x K.
  cudaError_t gemm(int P, int M, int N, int K, z64 alpha, BMc<double> A, int opA, BMc<double> B,
                   int opB, z64 beta, BM<double> C, z64 gamma, BMc<double> D,
                   const int32_t* active);
  // Mixed form: clear the tensor-core GEMM's timeout word / OR NEGF_PT_TIMEOUT into
  // status[0..P) if a GEMM since the reset gave up a bounded wait.  No-ops in the FP64 form.
  cudaError_t timeout_reset();
  cudaError_t timeout_flag(int P, int32_t* status);
  // X = Mm^-1 for P items of size b (Mm is destroyed); zero pivots flag status[item].
  // Mixed form: FP32 Gauss-Jordan start, refine_min Newton-Schulz steps for every item, further
  // steps (up to refine_max) only for items whose residual max |I - M X| is still above 2^-24,
  // and an FP64 Gauss-Jordan inverse for the items still above it after refine_max steps.
  cudaError_t inv(int P, BM<double> Mm, BM<double> X, int32_t* status, const int32_t* active);
};

// Number of block inverses (on the current device) that the mixed form recomputed in FP64
// because Newton-Schulz did not reach its residual target (synchronises the device).
long long engine_fp64_fallbacks();
// Test hook: with `on`, every mixed-form timeout check reports a given-up wait.
void engine_fail_waits(int on);

// Whether this build implements the precision form (negf_precision) for blocks of size b: the
// block inverse launches up to b = 5147 (FP64) / 9266 (mixed, FP32 elimination), and the mixed
// form's tensor-core GEMM is exact up to a contraction length that depends on the tier (48-bit
// values: 28032).
bool engine_supports(int precision, int b);

// Adjoint workspace helpers (adjoint.cu)
// ckpt: the sweep blocks come from negf_rgf_solve's checkpoints (no resident segment blocks)
size_t adjoint_bytes(const negf_device* dev, int P, const negf_options* opt, bool ckpt);
int adjoint_chunk(const negf_device* dev, int n_pts, const negf_options* opt, bool ckpt);
// Sweep checkpoints handed from negf_rgf_solve to negf_rgf_adjoint: complex128
// [5][N][n_pts][b][b], the kinds below, slab-major so that a chunk of consecutive points of one
// slab is contiguous (item stride b^2).
enum CkptKind { CK_G_FWD = 0, CK_GL_FWD = 1, CK_L = 2, CK_G = 3, CK_GL = 4, CK_KINDS = 5 };
inline size_t ckpt_offset(int kind, int slab, int N, int n_pts, int p, size_t bb) {
  return ((size_t)(kind * N + slab) * (size_t)n_pts + (size_t)p) * bb;
}

}  // namespace negf
