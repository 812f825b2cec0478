// One FE degree of the fused local kernel (compiled once per degree with
// -DFEKS_P=<p> so the degrees build in parallel).
#include "fe_ks_local.cuh"

#ifndef FEKS_P
#error "FEKS_P must be defined"
#endif

namespace feks {
template cudaError_t launch_local_deg<double, double, FEKS_P>(const Ctx&, const LocalParams<double, double>&,
                                                              cudaStream_t);
template cudaError_t launch_local_deg<float, float, FEKS_P>(const Ctx&, const LocalParams<float, float>&,
                                                            cudaStream_t);
template cudaError_t launch_local_deg<ff2, double, FEKS_P>(const Ctx&, const LocalParams<ff2, double>&,
                                                           cudaStream_t);
}  // namespace feks
