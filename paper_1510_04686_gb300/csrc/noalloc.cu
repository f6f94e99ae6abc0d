// Batched block inverse that allocates nothing: its scratch lives in a fixed file-scope device
// array instead of caller workspace, for callers that cannot allocate device memory.
#include <mutex>

#include "common.cuh"
#include "engine.cuh"

namespace negf {
namespace {

// Maximum scratch of the allocation-free inverse.  Every GPU that loads this library keeps
// this much device memory reserved until the process exits.
constexpr size_t kNoAllocBytes = 32ull << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device: in
// host code the array's name is only a host-side stand-in, not a device address).  The cached
// address belongs to the device context of the first call; after cudaDeviceReset the module is
// loaded again, possibly elsewhere, so calls after a reset are not supported.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace negf

using namespace negf;

extern "C" negf_status negf_zinv_batched_noalloc(int32_t n_batch, int32_t n, double* M, double* X,
                                                 int32_t* status, void* stream) {
  if (n_batch < 0 || n < 0) return NEGF_ERR_ARG;
  if (n_batch == 0 || n == 0) return NEGF_OK;
  if (!M || !X || !status) return NEGF_ERR_ARG;
  if (n_batch > 65535 || !gj_supports(n, 16)) return NEGF_ERR_UNSUPPORTED;
  // blocks small enough for the one-CTA shared-memory elimination use no scratch at all
  size_t need = 0;
  EngineWs w;
  if (!gj_fits_small(n, (int)sizeof(z64))) carve_engine(nullptr, need, n_batch, n, NEGF_PREC_FP64, w);
  if (need > kNoAllocBytes) return NEGF_ERR_NOMEM;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return NEGF_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status, 0, (size_t)n_batch * sizeof(int32_t), s) != cudaSuccess)
    return NEGF_ERR_CUDA;
  size_t off = 0;
  carve_engine(static_cast<char*>(base), off, n_batch, n, NEGF_PREC_FP64, w);
  const long long nn = (long long)n * n;
  cudaError_t e = gj_inverse<double>(s, n_batch, n, BM<double>{reinterpret_cast<z64*>(M), nn, nullptr, n},
                                     BM<double>{reinterpret_cast<z64*>(X), nn, nullptr, n}, w.invU,
                                     w.invT, w.piv, status, nullptr);
  return e == cudaSuccess ? NEGF_OK : NEGF_ERR_CUDA;
}
