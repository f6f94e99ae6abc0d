/*
 * negf.h -- C ABI of the GB300 recursive Green's function (RGF) library.
 *
 * The library solves, for many independent (energy E, transverse momentum k, alloy sample)
 * points, the nonequilibrium Green's function equations of a block-tridiagonal device
 * Hamiltonian (NEMO5 paper, Eqs. 1-8):
 *
 *   G^R(k,E) = (E - H(k) - e Phi - Sigma^R(k,E))^-1                        (Eq. 1)
 *   G^<(k,E) = G^R Sigma^< G^R^H                                          (Eq. 2)
 *   Sigma    = Sigma_lead + Sigma_optical + Sigma_acoustic                   (Eq. 3)
 *   Sigma_acoustic, Sigma_optical from diag G at E and E +- hbar omega      (Eqs. 4-6)
 *   density and current integrands                                          (Eqs. 7-8)
 *
 * Only the diagonal and first off-diagonal blocks of G^R and G^< are formed (recursive
 * Green's function sweeps).  Lead self-energies come from Sancho-Rubio decimation of
 * semi-infinite periodic copies of the end slabs.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Complex numbers are interleaved {double re, double im} (the layout of torch.complex128
 *    and C99 double complex).  Every b x b block is row-major and contiguous.
 *  - Every array argument is a DEVICE pointer owned by the caller, unless its comment says
 *    "host".  The library never frees or keeps caller memory after a call returns.
 *  - Temporary device memory is the caller's workspace (`ws`, `ws_bytes`), sized by
 *    negf_workspace_size().  The library allocates no device memory of its own, apart from
 *    fixed device arrays reserved on every GPU that loads it: the 32 MiB scratch of
 *    negf_zinv_batched_noalloc and a few bytes of diagnostic counters (FP64 fallbacks,
 *    profiled flops).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *    Outputs are valid after the stream is synchronised.  Several points are solved
 *    concurrently; the workspace holds a chunk of them at a time.
 *  - Return value: NEGF_OK, or an error detected on the host before any launch
 *    (NEGF_ERR_ARG, NEGF_ERR_NOMEM, NEGF_ERR_UNSUPPORTED) or a CUDA launch error
 *    (NEGF_ERR_CUDA).  Numerical trouble of single points is reported per point in
 *    `status[n_pts]` (bit set of NEGF_PT_*), written on the device; the call itself still
 *    returns NEGF_OK.  No exception crosses the ABI and no kernel traps.
 *  - Units: energies and potentials in eV.  Slab i (0-based) owns orbitals i*b .. i*b+b-1.
 */
#ifndef NEGF_H_
#define NEGF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEGF_ABI_VERSION 4

typedef enum {
  NEGF_OK = 0,
  NEGF_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, bad option)    */
  NEGF_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed               */
  NEGF_ERR_NOMEM = 3,         /* workspace smaller than negf_workspace_size() asks for     */
  NEGF_ERR_NOT_CONVERGED = 4, /* (per-point status summary) decimation did not converge   */
  NEGF_ERR_SINGULAR = 5,      /* (per-point status summary) a zero pivot was met           */
  NEGF_ERR_NONFINITE = 6,     /* (per-point status summary) NaN or Inf in an output        */
  NEGF_ERR_TIMEOUT = 7,       /* a bounded device wait gave up                             */
  NEGF_ERR_UNSUPPORTED = 8    /* option or size not supported by this build                */
} negf_status;

/* Per-point status bits written to `status[p]`. */
#define NEGF_PT_OK 0
#define NEGF_PT_NOT_CONVERGED 1 /* Sancho-Rubio reached sr_max_iter without converging      */
#define NEGF_PT_SINGULAR 2      /* a pivot of a block inverse was exactly zero               */
#define NEGF_PT_NONFINITE 4     /* an output of this point is NaN or Inf                    */
#define NEGF_PT_BAD_INDEX 8     /* sys_idx / e_idx out of range: the point was clamped to a
                                   valid row and its results are meaningless               */
#define NEGF_PT_TIMEOUT 16      /* mixed form: a bounded wait inside a tensor-core GEMM of the
                                   call gave up after 2 s (that GEMM's outputs are NaN, so the
                                   point is also NEGF_PT_NONFINITE); set for every point of
                                   the chunk of points that was being solved                */

/* Precision forms.  The mixed forms run every block GEMM on the tensor cores: each row of
 * op(A) and column of op(B) is scaled by a power of two and rounded once to a fixed-point value
 * of 39, 47 or 55 bits below twice the line maximum (the tiers are named 40, 48 and 56 bits),
 * cut into exact BF16 slices whose products are summed exactly in FP32 groups; storage,
 * pivoting, norms and reductions stay FP64.  A product's error is about
 * 2^-bits x K x max|row of A| x max|column of B|.  Issued tensor work per complex product: 15
 * (40 bits), 21 (48 bits) or 28 (56 bits) slice products for blocks up to 512 x 512. */
typedef enum {
  NEGF_PREC_FP64 = 0,     /* every block operation in FP64 on the CUDA cores (reference form) */
  NEGF_PREC_MIXED = 1,    /* tensor cores, 48-bit operand values (the default mixed form)     */
  NEGF_PREC_MIXED_40 = 2, /* tensor cores, 40-bit operand values (cheaper, less accurate)     */
  NEGF_PREC_MIXED_56 = 3  /* tensor cores, 56-bit operand values (FP64-class products)        */
} negf_precision;

/* negf_options.lead_precision = NEGF_PREC_AUTO: FP64 when `precision` is FP64; else a schedule
 * over the doubling steps of the decimation, 56-bit products for steps 1-8, 48-bit for 9-14 and
 * 40-bit from step 15 (48-bit for the surface Green's function and Sigma after the loop), or
 * NEGF_PREC_MIXED throughout for blocks beyond the 56-bit exact range.  The decimation of a
 * lead whose finite segments have near-singular (z - eps) blocks amplifies the rounding of its
 * early steps by up to ~1e9 (measured on the benchmark device); 56-bit products keep its error
 * at the level of an FP64 decimation there, while rounding at later steps is amplified by at
 * most ~3e4 (steps 5-10) and ~300 (steps >= 15).  A fixed tier applies to every step. */
#define NEGF_PREC_AUTO (-1)

/* Structure of the scattering self-energies of Eqs. 4-6 (negf_options.sigma_structure).  The
 * Born update is linear in diag G entry by entry, so the same update applies to every entry
 * of a block.
 *   NEGF_SIGMA_ORBITAL_DIAG: Sigma_scat is diagonal (one value per orbital), built from the
 *     diagonals of G^R, G^< (default).
 *   NEGF_SIGMA_ATOM_BLOCK: Sigma_scat is block-diagonal with one A x A block per atom
 *     (A = negf_options.atom_orbitals consecutive orbitals of a slab), built from the same
 *     A x A diagonal blocks of G^R, G^<.  Rows then hold N b A entries: entry (r, c) of slab
 *     i, r and c in the same atom, at i b A + r A + (c mod A). */
typedef enum { NEGF_SIGMA_ORBITAL_DIAG = 0, NEGF_SIGMA_ATOM_BLOCK = 1 } negf_sigma_structure;

/* Block-tridiagonal device Hamiltonians H(k) of n_sys systems (transverse k x alloy sample).
 * H_diag[s][i]  = H_ii        (Hermitian b x b),  s < n_sys, i < n_slabs
 * H_up[s][i]    = H_{i,i+1}   (b x b),            i < n_slabs - 1;  H_{i+1,i} = H_up^H.
 * The left lead is the periodic continuation of slab 0 (cell H_00, hopping H_01), the
 * right lead that of slab N-1 (cell H_{N-1,N-1}, hopping H_{N-2,N-1}). */
typedef struct {
  int32_t n_sys;
  int32_t n_slabs;       /* N >= 1; N == 1 has no hopping and flat leads (Sigma_lead = 0) */
  int32_t block;         /* b >= 1 */
  int32_t iface_rows;    /* r in [0, b]: every H_{i,i+1} is nonzero only in its last r rows
                            (the atoms of slab i facing slab i+1); 0 = all b rows            */
  const double* H_diag;  /* device, complex128 [n_sys][N][b][b] */
  const double* H_up;    /* device, complex128 [n_sys][N-1][b][b]; may be NULL when N == 1 */
  int32_t iface_cols;    /* c in [0, b]: ... and only in its first c columns (the atoms of
                            slab i+1 facing slab i); 0 = all b columns                       */
  int32_t reserved;
} negf_device;
/* Interface couplings (iface_rows / iface_cols below b): real tight-binding hoppings connect
 * only the atoms at the facing surfaces of neighbouring slabs, so H_{i,i+1} = E_R T E_C^T with
 * T the r x c block of its last r rows and first c columns.  negf_rgf_solve then forms every
 * product with a hopping on that support only (the Sigma_eff term t^H g t costs 2 r c (b or c)
 * instead of 2 b^3, and each backward product contracts over r or c instead of b), and so does
 * negf_lead_selfenergy: the decimation's alpha_n, beta_n keep the support of the lead hopping
 * (C x R and R x C) through every doubling step, so its six products per step contract over r
 * or c and form only their r- or c-row blocks, and Sigma_L (Sigma_R) is nonzero only on its
 * first c (last r) rows and columns; negf_rgf_adjoint restricts its recomputed sweeps and
 * every reverse-mode product with a hopping, or with an intermediate of that structure (L, K,
 * W, LW and their cotangents), in the same way.  Entries of H_up outside the support must be
 * zero. */

typedef struct {
  double eta_lead;       /* imaginary part of z = E + i eta in the lead decimation (eV)   */
  double eta_device;     /* imaginary part of z in the device (eV), >= 0                   */
  double mu_L, mu_R;     /* Fermi levels of the left / right contact (eV)                  */
  double kT;             /* contact temperature (eV)                                        */
  double sr_tol;         /* decimation stop: max(|alpha|_max,|beta|_max) <
                            sr_tol * max(|h|_max, |tau|_max) (default 1e-13)                 */
  int32_t sr_max_iter;   /* decimation iteration cap (default 100)                          */
  int32_t precision;     /* negf_precision of the sweeps (negf_rgf_solve, negf_rgf_adjoint)  */
  int32_t refine_steps;  /* mixed precision: Newton-Schulz steps X <- X + X (I - M X) run after
                            every FP32 block inverse (default 2)                            */
  int32_t chunk;         /* points solved concurrently (0 = library default)                */
  int32_t sr_host_check; /* decimation: read the count of unconverged points back every this
                            many steps (after 8) and stop early; 0 = never read back: always run
                            sr_max_iter steps with converged points masked on the device, so the
                            call makes no host synchronisation (CUDA-graph capturable).  Default 4 */
  int32_t adjoint_segment; /* negf_rgf_adjoint: slabs per recomputed segment (sweep
                            checkpointing); 0 = keep every slab's blocks.  Default 0 */
  int32_t lead_precision; /* negf_precision of the lead decimation (negf_lead_selfenergy), or
                            NEGF_PREC_AUTO (default)                                        */
  int32_t refine_max;    /* mixed precision: further Newton-Schulz steps, up to refine_max in
                            all, run only for blocks whose residual max |I - M X| is still
                            above 2^-24; a block still above it after refine_max steps is
                            inverted again by FP64 Gauss-Jordan (default 6, range 0-16)      */
  int32_t sigma_structure; /* negf_sigma_structure of scat_R/L and diagGR/GL (default
                            NEGF_SIGMA_ORBITAL_DIAG)                                        */
  int32_t atom_orbitals; /* A: orbitals per atom block under NEGF_SIGMA_ATOM_BLOCK, 1..64,
                            dividing b (default 10)                                          */
} negf_options;

/* Fill `opt` with the defaults (eta 1e-6 in leads and device, mu_L = +0.1, mu_R = -0.1,
 * kT = 0.025852, sr_tol = 1e-13, sr_max_iter = 100, FP64, refine_steps = 2, chunk = 0,
 * sr_host_check = 4, adjoint_segment = 0, lead_precision = NEGF_PREC_AUTO, refine_max = 6,
 * sigma_structure = NEGF_SIGMA_ORBITAL_DIAG, atom_orbitals = 10). */
void negf_default_options(negf_options* opt);

int32_t negf_abi_version(void);
const char* negf_status_string(negf_status s);

/* Which call a workspace is sized for. */
#define NEGF_WS_LEAD 0
#define NEGF_WS_RGF 1
#define NEGF_WS_ADJOINT 2
#define NEGF_WS_ADJOINT_CKPT 3 /* negf_rgf_adjoint given negf_rgf_solve's checkpoints */

/* Bytes of device workspace a call of kind `which` needs for n_pts points (the library
 * works through the points `opt->chunk` at a time, so the size saturates). */
size_t negf_workspace_size(const negf_device* dev, int32_t n_pts, const negf_options* opt,
                           int32_t which);
/* Block inverses of the mixed forms (on the current device) that were recomputed by FP64
 * Gauss-Jordan because Newton-Schulz did not reach its residual target within refine_max
 * steps, since the library was loaded.  Diagnostic; synchronises the device; -1 on error. */
long long negf_fp64_fallback_count(void);

/* Lead self-energies (Eq. 3, Sigma_lead) by Sancho-Rubio decimation (Lopez Sancho, Lopez
 * Sancho & Rubio, J. Phys. F 15, 851 (1985)); the paper's own leads use the transfer matrix
 * or complex absorbing potential methods (text below Eq. 6), which reach the same unique
 * retarded surface Green's function.  Every product and inverse of the decimation runs in
 * lead_precision (see NEGF_PREC_AUTO); the workspace must be sized with the same options.
 *   E[n_pts]        device double: energy of each point
 *   sys_idx[n_pts]  device int32:  which Hamiltonian of `dev` the point uses (0..n_sys-1)
 *   sigma_R         device complex128 [n_pts][2][b][b] out: Sigma^R of side 0 = left lead
 *                   (acts on slab 0: H_01^H g_L H_01) and side 1 = right lead (acts on
 *                   slab N-1: H_{N-2,N-1} g_R H_{N-2,N-1}^H)
 *   sigma_L         device complex128 [n_pts][2][b][b] out: Sigma^< = i f(E) Gamma,
 *                   Gamma = i (Sigma^R - Sigma^R^H), f the contact's Fermi function
 *   iters           device int32 [n_pts][2] out (nullable): decimation steps per side
 *   status          device int32 [n_pts] out: NEGF_PT_* bits                            */
negf_status negf_lead_selfenergy(const negf_device* dev, int32_t n_pts, const double* E,
                                 const int32_t* sys_idx, const negf_options* opt,
                                 double* sigma_R, double* sigma_L, int32_t* iters,
                                 int32_t* status, void* ws, size_t ws_bytes, void* stream);

/* One RGF solve per point: forward sweep of left-connected g^R, g^< and backward sweep for
 * the diagonal blocks G^R_ii, G^<_ii and the off-diagonal G^<_{i+1,i} (Eqs. 1-2), then the
 * observables.
 *   V           device double [N][b] (nullable = 0): on-site potential (the e Phi of Eq. 1),
 *               added to the diagonal of H_ii for every point
 *   sigma_R/L   device complex128 [n_pts][2][b][b]: lead self-energies (negf_lead_selfenergy)
 *   scat_R/L    device complex128 [n_rows][N*b*A] (nullable = ballistic): phonon
 *               self-energies Sigma^R, Sigma^< of Eqs. 4-6, orbital-diagonal (A = 1) or
 *               atom blocks (A = atom_orbitals; layout at negf_sigma_structure); point p uses
 *               row e_idx[p] (e_idx nullable = row p, and then n_rows must be >= n_pts)
 *   density     device double [n_pts][N*b] out (nullable): n_j(E) = Im G^<_jj / (2 pi)
 *   current     device double [n_pts][N-1] out (nullable): bond current
 *               j_i(E) = 2 Re Tr[H_{i,i+1} G^<_{i+1,i}] (Eq. 8, per spin, units 1/h)
 *   transmission device double [n_pts] out (nullable):
 *               T(E) = Tr[Gamma_R A_NN] - Tr[Gamma_R G_NN Gamma_R G_NN^H]  (exact when
 *               ballistic; with scattering it is the flux into the right lead per unit
 *               occupation difference of all other sources)
 *   diagGR/GL   device complex128 [n_pts][N*b*A] out (nullable): diag G^R, diag G^< (A = 1)
 *               or their atom diagonal blocks (same layout as scat_R/L) for the
 *               self-consistent Born step (negf_scba_step, with n_orb = N b A)
 *   checkpoints device, negf_checkpoint_bytes(dev, n_pts) bytes, out (nullable): the sweep
 *               blocks negf_rgf_adjoint needs (forward g_i, g^<_i, L_i = g_i t_i; backward
 *               G_ii, G^<_ii), so that it runs only its reverse passes
 *   Returns NEGF_ERR_ARG when sigma_structure is invalid or A does not divide b.
 *   status      device int32 [n_pts] out                                                 */
negf_status negf_rgf_solve(const negf_device* dev, int32_t n_pts, const double* E,
                           const int32_t* sys_idx, const double* V, const double* sigma_R,
                           const double* sigma_L, const double* scat_R, const double* scat_L,
                           const int32_t* e_idx, int32_t n_rows, const negf_options* opt,
                           double* density,
                           double* current, double* transmission, double* diagGR,
                           double* diagGL, void* checkpoints, int32_t* status, void* ws,
                           size_t ws_bytes, void* stream);

/* Bytes of the sweep checkpoints of negf_rgf_solve for n_pts points: complex128
 * [5][N][n_pts][b][b] (forward g, forward g^<, L, backward G, backward G^<, each slab-major with
 * the points of a slab contiguous): 5 N b^2 complex numbers per point; 0 for an invalid
 * device or n_pts < 1. */
size_t negf_checkpoint_bytes(const negf_device* dev, int32_t n_pts);

/* One self-consistent Born update of the phonon self-energies (Eqs. 4-6), entry by entry
 * (orbital diagonals, or every entry of the atom blocks with n_orb = N b A):
 *   Sigma_ac^{R,<}(E_j) = D_ac sum_k w_k dG^{R,<}(k, E_j)                                (4)
 *   Sigma_op^<(E_j) = D_op sum_k w_k [(1+n0) dG^<(k,E_{j+s}) + n0 dG^<(k,E_{j-s})]       (5)
 *   Sigma_op^R(E_j) = D_op sum_k w_k [(1+n0) dG^R(k,E_{j-s}) + n0 dG^R(k,E_{j+s})
 *                                     + dG^<(k,E_{j-s})/2 - dG^<(k,E_{j+s})/2]           (6)
 * (the printed comma inside Eq. 6 is read as '+'; hbar omega = `shift` grid steps; energies
 * off the grid contribute zero; the prefactors of Eqs. 4-6 are D_ac, D_op in eV^2 and the k'
 * integral is the weighted sum).  Then Sigma <- (1-mix) Sigma_old + mix Sigma_new.
 *   w_k        device double [n_k]
 *   diagGR/GL  device complex128 [n_k][n_E][n_orb]   (negf_rgf_solve's diag outputs with
 *              points ordered k-major)
 *   sigma_R/L  device complex128 [n_E][n_orb] in: old Sigma, out: new Sigma
 *   delta_out  device double [1] out: max over entries of |Sigma_new - Sigma_old|        */
negf_status negf_scba_step(int32_t n_k, int32_t n_E, int32_t n_orb, const double* w_k,
                           double D_ac, double D_op, int32_t shift, double n0, double mix,
                           const double* diagGR, const double* diagGL, double* sigma_R,
                           double* sigma_L, double* delta_out, void* stream);

/* The Born update of negf_scba_step on a non-uniform energy mesh E[n_E] (device double,
 * strictly increasing; e.g. an adaptively refined mesh): the optical terms of Eqs. 5-6 take
 * sum_k w_k dG(k, E_j +- hw) by linear interpolation between the two mesh points around
 * E_j +- hw (hw in eV), and energies outside [E_0, E_{n_E - 1}] contribute zero.  On a uniform
 * mesh with hw a whole number of steps it equals negf_scba_step (to rounding).  Other arguments
 * and layouts as for negf_scba_step. */
negf_status negf_scba_step_mesh(int32_t n_k, int32_t n_E, int32_t n_orb, const double* E,
                                const double* w_k, double D_ac, double D_op, double hw,
                                double n0, double mix, const double* diagGR,
                                const double* diagGL, double* sigma_R, double* sigma_L,
                                double* delta_out, void* stream);

/* Reverse-mode derivative of the observables of negf_rgf_solve with respect to the on-site
 * potential V (the e Phi of Eq. 1), for a Newton-Poisson loop around Eq. 9.  With the
 * same inputs as negf_rgf_solve (self-energies held fixed) and the cotangents
 *   density_bar [n_pts][N*b] (nullable), current_bar [n_pts][N-1] (nullable),
 * it accumulates V_bar[N][b] += sum_p sum_j density_bar[p][j] dn_j(p)/dV
 *                                 + sum_i current_bar[p][i] dj_i(p)/dV.
 * V_bar is device double [N][b] and is overwritten (not accumulated into).
 * checkpoints (nullable): the blocks a negf_rgf_solve call wrote for the same device, points,
 * V, self-energies and options (its `checkpoints` output); the adjoint then recomputes no sweep
 * and keeps no sweep block of its own (workspace NEGF_WS_ADJOINT_CKPT: the cotangents, 3 N b^2
 * complex per point, and temporaries).  Without them every slab's forward and backward blocks
 * are recomputed and kept (8 N b^2 complex per point in flight, workspace NEGF_WS_ADJOINT)
 * unless opt->adjoint_segment = s with 0 < s < N: then only segment-boundary blocks are kept
 * and one segment at a time is recomputed (3 N + 5 s + 4 N / s blocks per point, about 3 more
 * forward sweeps and 1 more backward sweep); results agree to rounding.                    */
negf_status negf_rgf_adjoint(const negf_device* dev, int32_t n_pts, const double* E,
                             const int32_t* sys_idx, const double* V, const double* sigma_R,
                             const double* sigma_L, const double* scat_R,
                             const double* scat_L, const int32_t* e_idx, int32_t n_rows,
                             const negf_options* opt, const void* checkpoints,
                             const double* density_bar, const double* current_bar,
                             double* V_bar, int32_t* status, void* ws, size_t ws_bytes,
                             void* stream);

/* Energy / k quadrature of Eqs. 7-8 in FP64 in a fixed order (deterministic):
 *   out[g][j] = sum over p with group[p] == g (in increasing p) of w[p] * in[p][j]
 *   in [n_pts][len], w [n_pts], group [n_pts] (nullable = all in group 0), out [n_groups][len]
 * All device pointers. */
negf_status negf_integrate(int32_t n_pts, int32_t len, int32_t n_groups, const double* w,
                           const int32_t* group, const double* in, double* out, void* stream);

/* ---- electrostatics of the NEGF-Poisson loop (Eq. 9) ---------------------------------------
 * Eq. 9, div(eps grad Phi) = e (n - N_D), is written for the potential energy U = -e Phi that
 * enters Eq. 1 (negf_rgf_solve's V, one value per atom shared by its orbitals) and discretised
 * on the device's atom grid: slab i = 0..N-1 along transport, atom a = 0..A-1 across the slab
 * (periodic, the device being periodic in that direction), contacts held at U_L (slab -1) and
 * U_R (slab N).  With c_x, c_y the coupling constants eps / h^2 of the two directions and kappa
 * = e^2 per unit of them (eV per electron), Eq. 9 becomes F(U) = 0 with
 *   F[i][a] = c_x (2 U[i][a] - U[i-1][a] - U[i+1][a]) + c_y (2 U[i][a] - U[i][a-1] - U[i][a+1])
 *             - kappa (n[i][a] - n_D[i][a]),
 * n the electrons per atom (Eq. 7 summed over the atom's orbitals) and n_D the donor charge.
 * negf_poisson_apply writes F for U [N][A] (n nullable: the operator alone, K U - boundary
 * terms; n_D nullable = 0); all device double arrays, asynchronous on stream.  c_x, c_y >= 0.
 * (For A == 1 there is no transverse term; for A == 2 both transverse neighbours are the one
 * other atom.) */
negf_status negf_poisson_apply(int32_t n_slabs, int32_t n_atoms, double c_x, double c_y,
                               double U_L, double U_R, double kappa, const double* U,
                               const double* n, const double* n_D, double* out, void* stream);
/* Per-atom sums of per-orbital arrays and the reverse broadcast, for atoms of
 * `orbitals_per_atom` consecutive orbitals (the last atom of a slab may be short):
 *   atom[g][i][a] = sum_o orb[g][i][per a + o]   (groups stacked arrays [groups][N][block])
 *   orb[i][o]     = atom[i][o / per]                                                         */
negf_status negf_orbitals_to_atoms(int32_t groups, int32_t n_slabs, int32_t block,
                                   int32_t orbitals_per_atom, const double* orb, double* atom,
                                   void* stream);
negf_status negf_atoms_to_orbitals(int32_t n_slabs, int32_t block, int32_t orbitals_per_atom,
                                   const double* atom, double* orb, void* stream);

/* ---- block operations the sweeps are built from ------------------------------------------
 * Batched complex GEMM  C[p] = alpha op(A[p]) op(B[p]) + beta C[p]  (Eqs. 1-2 are evaluated
 * block by block as such products).  complex128 row-major; op 0 = none, 1 = transpose,
 * 2 = conjugate transpose; op(A) is M x K, op(B) is K x N; strides are in complex elements
 * between batch items (0 = the same matrix for every item; C needs a nonzero stride when
 * n_batch > 1).  `precision` is any negf_precision.  FP64 form: CUDA cores.  Mixed forms:
 * tensor cores with exact split-BF16 slices of 40-, 48- or 56-bit values (error about
 * 2^-bits x K relative to max|A| max|B| per row and column), exact for K <= 524288
 * (40 bits), 393216 (48 bits) or 98304 (56 bits): a longer contraction returns
 * NEGF_ERR_UNSUPPORTED (and a workspace size of 0) rather than losing accuracy.  The block
 * inverse (and so every sweep entry point) takes
 * blocks up to n = 5147 in FP64 and n = 9266 in the mixed form (its Gauss-Jordan panel lives
 * in shared memory); larger blocks are refused the same way.  n_batch <= 65535. */
size_t negf_zgemm_workspace_size(int32_t precision, int32_t n_batch, int32_t M, int32_t N,
                                 int32_t K);
negf_status negf_zgemm_batched(int32_t precision, int32_t n_batch, int32_t M, int32_t N,
                               int32_t K, double alpha_re, double alpha_im, const double* A,
                               int64_t strideA, int32_t lda, int32_t opA, const double* B,
                               int64_t strideB, int32_t ldb, int32_t opB, double beta_re,
                               double beta_im, double* C, int64_t strideC, int32_t ldc,
                               void* ws, size_t ws_bytes, void* stream);

/* Batched block inverse X[p] = M[p]^-1 (the (z - H - Sigma)^-1 of Eq. 1), n x n complex128,
 * contiguous items.  Gauss-Jordan with partial pivoting (largest |m|^2, lowest row on ties;
 * magnitudes in FP64, or as exact FP32 pairs to about 2^-47 in the mixed form's FP32
 * elimination), pivot reciprocal in the storage precision.
 * FP64 form: FP64 elimination, M is destroyed.  Mixed forms: FP32 elimination followed by
 * `refine_steps` Newton-Schulz steps X <- X + X (I - M X) with tensor-core products of the
 * tier's precision, then up to max(refine_steps, 6) steps for blocks whose residual
 * max |I - M X| is still above 2^-24, and FP64 Gauss-Jordan for blocks still above it (M is
 * destroyed only by that fallback).  status[p] gets NEGF_PT_SINGULAR on an exactly zero
 * pivot. */
size_t negf_zinv_workspace_size(int32_t precision, int32_t n_batch, int32_t n);
negf_status negf_zinv_batched(int32_t precision, int32_t n_batch, int32_t n, double* M,
                              double* X, int32_t refine_steps, int32_t* status, void* ws,
                              size_t ws_bytes, void* stream);

/* Allocation-free variant of negf_zinv_batched, FP64 form only (the paper has no counterpart;
 * this exists for callers that cannot allocate device memory at the point of the call, e.g. a
 * host application whose device memory is owned by an arena reserved at start-up, or code that
 * must not call cudaMalloc after initialisation because it can synchronise the device and fail
 * once memory is fragmented).  Same inputs and outputs as negf_zinv_batched with
 * precision = NEGF_PREC_FP64 and no workspace: the elimination scratch lives in a fixed 32 MiB
 * device array inside this library, reserved on every GPU that loads it until the process
 * exits.  The scratch needed, about n_batch * n * (2 * 16 * nb + 4) bytes with the panel width
 * nb <= 32 (none at all for n <= 106, which is done in shared memory), must fit those
 * 32 MiB, else the call returns NEGF_ERR_NOMEM before launching anything.  The first call on a
 * device looks up the array's device address for that device, with the device current, and
 * keeps it; calls after cudaDeviceReset() on that device are therefore not supported (the
 * reset may move the array).  Every call on a device shares the one array, which keeps the last call's
 * contents: calls that overlap on the GPU (different streams, or different host threads)
 * race on it and must be serialised by the caller.  It calls no cudaMalloc or cudaFree.
 * M is destroyed; status[p] gets NEGF_PT_SINGULAR on an exactly zero pivot. */
negf_status negf_zinv_batched_noalloc(int32_t n_batch, int32_t n, double* M, double* X,
                                      int32_t* status, void* stream);

/* ---- tensor-core GEMM configuration (autotuning) ----------------------------------------
 * The mixed-precision GEMM has negf_tc_config_count() kernel configurations, differing only in
 * speed: configuration c uses the kernel shape c / 2 of
 *   (6 stages, 1 CTA, 1), (6, 1, 2), (6, 1, 3), (8 stages, CTA pair, 1), (8, 2, 2), (8, 2, 4),
 *   (3, 1, 1, 2 K chunks per stage), (4, 2, 1, 2 K chunks per stage),
 *   (2, 1, 1, 3 K chunks per stage), (2, 2, 1, 4 K chunks per stage),
 *   (3, 2, 1, 3 K chunks per stage), (2, 2, 1, 2 K chunks, 64-column tiles, 2 CTAs per SM),
 *   (2, 1, 1, 2 K chunks, 64-column tiles, 2 CTAs per SM)
 * = (shared-memory pipeline stages, CTAs per MMA: one 128-row tile or a pair of CTAs with a
 * 256-row MMA, stages released per MMA commit; K chunks of 64 per stage; 128-column tiles unless
 * stated) and splits K into at most (4, 8)[c % 2] exactly accumulated parts (more parts allow
 * wider slices and fewer slice products for long contractions).
 * negf_tc_config_set selects one process-wide (default 18: the CTA pair with 2 stages of 4 K
 * chunks); results agree to the GEMM's rounding.  The package's autotuner times them per block
 * size and stores the choice. */
int32_t negf_tc_config_count(void);
negf_status negf_tc_config_set(int32_t idx);
int32_t negf_tc_config_get(void);

/* ---- accounting ----------------------------------------------------------------------------
 * Instrumentation for benchmarks, not part of the method.  negf_launch_count() is the number
 * of kernels this library has launched since it was loaded.  With profiling on, every launch of
 * the tensor-core GEMM kernel (kind 0), of its operand slicing (kind 1) and every Gauss-Jordan
 * elimination of a block inverse inside the sweeps (kind 2: the FP32 start of the mixed form or
 * the whole FP64 inverse, without the Newton-Schulz products, which count as kinds 0 and 1) and
 * every launch of its panel-elimination kernel (kind 3, a part of kind 2) is
 * bracketed by CUDA events on its own stream; negf_profile_read synchronises those events and
 * returns the cumulative launches and milliseconds of the kind since the last
 * negf_profile_reset. */
void negf_profile_enable(int32_t on);
void negf_profile_reset(void);
negf_status negf_profile_read(int32_t kind, long long* launches, double* total_ms);
/* Flops of kind 0 since the last reset, counted on the device for the batch items that ran
 * (items masked off, e.g. blocks whose Newton-Schulz refinement had converged, do not count):
 * complex algorithmic 8 M N K per item, and the BF16 tensor-core flops actually issued (the
 * computed slice products over the padded tiles).  Reading and resetting synchronise the
 * current device. */
negf_status negf_profile_flops(int32_t kind, double* algorithmic, double* hardware);
long long negf_launch_count(void);
/* Test hook for the timeout reporting path: while `on` is nonzero, every mixed-form call ends
 * as if a bounded wait inside one of its tensor-core GEMMs had given up (the device error word
 * is set on the call's stream before the per-point status is written), so NEGF_PT_TIMEOUT is
 * set for every point without any GPU wait having to expire.  The outputs are not touched.
 * Process-wide; off by default; for tests only. */
void negf_debug_fail_waits(int32_t on);
/* Name of the last CUDA runtime error that made a call of this library return NEGF_ERR_CUDA
 * (e.g. "cudaErrorInvalidValue"; "cudaSuccess" if none), for diagnostics.  Static string. */
const char* negf_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NEGF_H_ */
