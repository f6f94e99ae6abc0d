// Electrostatics of the NEGF-Poisson loop (Eq. 9): the finite-difference Poisson operator on the
// atom grid of the device and the maps between per-orbital and per-atom quantities.
#include "common.cuh"
#include "profile.cuh"

namespace negf {
namespace {

// out[i][a] = c_x (2 U[i][a] - U[i-1][a] - U[i+1][a]) + c_y (2 U[i][a] - U[i][a-1] - U[i][a+1])
//             - kappa (n[i][a] - n_D[i][a])
// with U[-1][a] = U_L and U[N][a] = U_R (contacts) and a periodic across the slab.
__global__ void k_poisson(int N, int A, double cx, double cy, double UL, double UR, double kappa,
                          const double* U, const double* n, const double* nD, double* out) {
  const long long tot = (long long)N * A;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / A), a = (int)(e % A);
    const double u = U[e];
    const double left = i > 0 ? U[e - A] : UL;
    const double right = i < N - 1 ? U[e + A] : UR;
    double r = cx * (2.0 * u - left - right);
    if (A > 1) {
      const double up = U[(long long)i * A + (a + 1) % A];
      const double dn = U[(long long)i * A + (a + A - 1) % A];
      r += cy * (2.0 * u - up - dn);
    }
    if (n) r -= kappa * (n[e] - (nD ? nD[e] : 0.0));
    out[e] = r;
  }
}

// atom[g][i][a] = sum over the `per` orbitals of atom a of slab i of orb[g][i][b] (b orbitals per
// slab, atom a owning orbitals per*a .. per*a + per - 1), for `groups` stacked arrays
__global__ void k_to_atoms(int groups, int N, int b, int per, const double* orb, double* atom) {
  const int A = (b + per - 1) / per;
  const long long tot = (long long)groups * N * A;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long gi = e / A;  // (group, slab)
    const int a = (int)(e % A);
    const double* row = orb + gi * b;
    double s = 0.0;
    for (int o = per * a; o < per * a + per && o < b; ++o) s += row[o];
    atom[e] = s;
  }
}

// orb[i][b] = atom[i][a] for every orbital of atom a
__global__ void k_to_orbitals(int N, int b, int per, const double* atom, double* orb) {
  const int A = (b + per - 1) / per;
  const long long tot = (long long)N * b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / b), o = (int)(e % b);
    orb[e] = atom[(long long)i * A + o / per];
  }
}

inline unsigned blocks(long long n) {
  long long g = (n + 255) / 256;
  return (unsigned)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace
}  // namespace negf

using namespace negf;

extern "C" {

negf_status negf_poisson_apply(int32_t n_slabs, int32_t n_atoms, double c_x, double c_y,
                               double U_L, double U_R, double kappa, const double* U,
                               const double* n, const double* n_D, double* out, void* stream) {
  if (n_slabs < 1 || n_atoms < 1 || !U || !out || !(c_x >= 0.0) || !(c_y >= 0.0))
    return NEGF_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long tot = (long long)n_slabs * n_atoms;
  k_poisson<<<blocks(tot), 256, 0, s>>>(n_slabs, n_atoms, c_x, c_y, U_L, U_R, kappa, U, n, n_D,
                                        out);
  count_launch();
  return note_error(cudaGetLastError()) == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}

negf_status negf_orbitals_to_atoms(int32_t groups, int32_t n_slabs, int32_t block,
                                   int32_t orbitals_per_atom, const double* orb, double* atom,
                                   void* stream) {
  if (groups < 1 || n_slabs < 1 || block < 1 || orbitals_per_atom < 1 || !orb || !atom)
    return NEGF_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int A = (block + orbitals_per_atom - 1) / orbitals_per_atom;
  k_to_atoms<<<blocks((long long)groups * n_slabs * A), 256, 0, s>>>(groups, n_slabs, block,
                                                                      orbitals_per_atom, orb,
                                                                      atom);
  count_launch();
  return note_error(cudaGetLastError()) == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}

negf_status negf_atoms_to_orbitals(int32_t n_slabs, int32_t block, int32_t orbitals_per_atom,
                                   const double* atom, double* orb, void* stream) {
  if (n_slabs < 1 || block < 1 || orbitals_per_atom < 1 || !orb || !atom) return NEGF_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_to_orbitals<<<blocks((long long)n_slabs * block), 256, 0, s>>>(n_slabs, block,
                                                                   orbitals_per_atom, atom, orb);
  count_launch();
  return note_error(cudaGetLastError()) == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}

}  // extern "C"
