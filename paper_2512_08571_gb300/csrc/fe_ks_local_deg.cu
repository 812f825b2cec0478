// One FE degree and one quadrature order of the fused local kernel (compiled
// once per pair with -DFEKS_P=<p> -DFEKS_NQX=<n_q - n_p> so they build in
// parallel).
#include "fe_ks_local.cuh"

#ifndef FEKS_P
#error "FEKS_P must be defined"
#endif
#ifndef FEKS_NQX
#define FEKS_NQX 0
#endif

namespace feks {
template cudaError_t launch_local_deg<double, double, FEKS_P, FEKS_NQX>(const Ctx&, const LocalParams<double, double>&,
                                                                        cudaStream_t);
template cudaError_t launch_local_deg<float, float, FEKS_P, FEKS_NQX>(const Ctx&, const LocalParams<float, float>&,
                                                                      cudaStream_t);
template cudaError_t launch_local_deg<ff2, double, FEKS_P, FEKS_NQX>(const Ctx&, const LocalParams<ff2, double>&,
                                                                     cudaStream_t);
}  // namespace feks
