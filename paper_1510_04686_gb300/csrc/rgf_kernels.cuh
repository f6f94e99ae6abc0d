// Launchers of the elementwise / reduction kernels of the sweeps (rgf_kernels.cu).
#pragma once
#include "common.cuh"

namespace negf {

// scat: the slab's scattering self-energy row (nullable), block-diagonal with A x A blocks
// (A = 1: orbital-diagonal), entry (r, c) at scat[r A + c mod A]; rows of scat_stride entries
// selected by e_idx (nullable: row p).
cudaError_t launch_assemble(cudaStream_t s, int P, int b, const double* E, double eta,
                            BMc<double> Hd, const double* V, const z64* scat,
                            long long scat_stride, int A, const int32_t* e_idx, BMc<double> Y,
                            int ny, BMc<double> SigA, BMc<double> SigB, BM<double> M,
                            const int32_t* active);
cudaError_t launch_source(cudaStream_t s, int P, int b, const z64* scat, long long scat_stride,
                          int A, const int32_t* e_idx, BMc<double> SigA, BMc<double> SigB,
                          BM<double> S, const int32_t* active);
cudaError_t launch_antiherm(cudaStream_t s, int P, int b, BMc<double> S, BM<double> O,
                            const int32_t* active);
// density[p][i b + j] (rows of nb_tot); dGR / dGL: A x A diagonal blocks, [p][(i b + r) A + c mod A]
cudaError_t launch_slab_obs(cudaStream_t s, int P, int b, int i, int nb_tot, int A,
                            BMc<double> G, BMc<double> GL, double* density, z64* dGR, z64* dGL,
                            const int32_t* active);
cudaError_t launch_bond_current(cudaStream_t s, int P, int b, BMc<double> Tm, BMc<double> U,
                                BMc<double> Q, double* out, long long out_stride,
                                const int32_t* active);
cudaError_t launch_gamma(cudaStream_t s, int P, int b, BMc<double> Sig, BM<double> Gam,
                         const int32_t* active);
cudaError_t launch_transmission(cudaStream_t s, int P, int b, BMc<double> Gam, BMc<double> G,
                                BMc<double> Y, BMc<double> Z, double* out,
                                const int32_t* active);
cudaError_t launch_sr_init(cudaStream_t s, int P2, int b, int N, BMc<double> Hd, BMc<double> Hu,
                           BM<double> eps_s, BM<double> eps, BM<double> al, BM<double> be,
                           double* scale);
cudaError_t launch_zminus(cudaStream_t s, int P2, int b, const double* E, double eta,
                          BMc<double> X, BM<double> M, const int32_t* active);
// A1 += T1 and A2 += T1 on the square block [o, o + n)^2 of each item: (o0, n0) for the even
// (left-lead) items q = 2 p, (o1, n1) for the odd (right-lead) ones.
cudaError_t launch_add2(cudaStream_t s, int P2, int b, BMc<double> T1, BM<double> A1,
                        BM<double> A2, int o0, int n0, int o1, int n1, const int32_t* active);
// by_side (nullable, [2][P2 / 2]): items that converge also clear by_side[side][p], q = 2 p + side.
cudaError_t launch_sr_check(cudaStream_t s, int P2, int b, int it, double tol, BMc<double> al,
                            BMc<double> be, const double* scale, int32_t* active,
                            int32_t* iters, int32_t* n_active, int32_t* by_side);
cudaError_t launch_lead_lesser(cudaStream_t s, int P2, int b, const double* E, double mu_L,
                               double mu_R, double kT_, BMc<double> Gam, BM<double> Les);
cudaError_t launch_sr_status(cudaStream_t s, int P, const int32_t* active,
                             const int32_t* item_status, int32_t* iters_in, int32_t* iters_out,
                             int max_iter, int32_t* status);
cudaError_t launch_check_finite(cudaStream_t s, const double* x, long long per_pt, int P,
                                int32_t* status);
// out[p] = in[p] clamped to [0, n); out-of-range entries set NEGF_PT_BAD_INDEX in status[p].
cudaError_t launch_clamp_index(cudaStream_t s, int P, const int32_t* in, int n, int32_t* out,
                               int32_t* status);
cudaError_t launch_fill_i32(cudaStream_t s, int32_t* a, long long n, int32_t v);
cudaError_t launch_integrate(cudaStream_t s, int P, int len, int n_groups, const double* w,
                             const int32_t* group, const double* in, double* out);

}  // namespace negf
