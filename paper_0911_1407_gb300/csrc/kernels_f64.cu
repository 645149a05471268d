// kernels_f64.cu -- FP64 instantiations of the spectral pipeline and the
// element-wise kernels (the PLC_FP64 solve, and the FP64 gradients of the
// mixed solve).
#include "launch.cuh"

namespace plc {
template void prior_apply<double>(plc_ctx*, const double*, double*);
template void hessvec_s<double>(plc_ctx*, const double*, const double*, double, const double*, double*);
template void grad_public<double>(plc_ctx*, const double*, const double*, const int32_t*, double,
                                  double*);
template void grad_newton<double, double>(plc_ctx*, double*, const double*, double, const double*,
                                          const int32_t*, double, double*, double*, bool);
template void grad_newton<double, float>(plc_ctx*, double*, const float*, double, const double*,
                                         const int32_t*, double, float*, float*, bool);
template void cg_hv<double>(plc_ctx*, const double*, const double*, double*, double*, bool);
template void vjp_amplitude<double>(plc_ctx*, const double*, const double*);
template void cg_init<double>(plc_ctx*, const double*, const double*, double*, bool);
template void cg_update<double>(plc_ctx*, double*, double*, const double*, const double*,
                                const double*, bool, double, int);
template void diag<double>(plc_ctx*, const double*, const double*, double, double*);
}  // namespace plc
