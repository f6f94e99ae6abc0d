// Reverse-mode derivative of the RGF observables with respect to the on-site potential.
#include "engine.cuh"

namespace negf {
size_t adjoint_bytes(const negf_device* dev, int P, const negf_options* opt) {
  (void)dev; (void)P; (void)opt;
  return 0;
}
int adjoint_chunk(const negf_device* dev, int n_pts, const negf_options* opt) {
  (void)dev; (void)opt;
  return n_pts < 1 ? 1 : n_pts;
}
}  // namespace negf

extern "C" negf_status negf_rgf_adjoint(const negf_device*, int32_t, const double*,
                                        const int32_t*, const double*, const double*,
                                        const double*, const double*, const double*,
                                        const int32_t*, int32_t, const negf_options*,
                                        const double*,
                                        const double*, double*, int32_t*, void*, size_t, void*) {
  return NEGF_ERR_UNSUPPORTED;
}
