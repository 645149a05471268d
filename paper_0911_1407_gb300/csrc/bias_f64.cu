// bias_f64.cu -- FP64 instantiations of the linear-bias launchers (FP64
// state with FP64 or FP32 CG fields).
#include "bias.cuh"
#include "bias.h"

namespace plc {
template void bias_prior<double, double>(plc_ctx*, const double*, double, double*);
template void bias_prior<double, float>(plc_ctx*, const float*, double, double*);
template void bias_density<double, double>(plc_ctx*, const double*, const double*, double,
                                           double*, const double*, const double*, double*,
                                           const int32_t*, const double*, double, double*,
                                           double*);
template void bias_density<double, float>(plc_ctx*, const double*, const float*, double, double*,
                                          const double*, const double*, double*, const int32_t*,
                                          const double*, double, double*, float*);
template void bias_gradient<double, double>(plc_ctx*, const double*, const double*,
                                            const double*, const double*, double*, double*,
                                            double*, double*, double*, bool);
template void bias_gradient<double, float>(plc_ctx*, const double*, const double*, const double*,
                                           const float*, double*, float*, float*, float*, float*,
                                           bool);
template void bias_cg_hv<double>(plc_ctx*, const double*, const double*, double*, const double*,
                                 const double*, const double*, double*, double*, double*, bool);
template void bias_hv<double>(plc_ctx*, const double*, const double*, const double*,
                              const double*, double*, double*, double*);
template void bias_fallback<double>(plc_ctx*, const double*, double*);
}  // namespace plc
