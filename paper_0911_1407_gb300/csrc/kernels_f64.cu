// kernels_f64.cu -- FP64 instantiations of the spectral pipeline and the
// element-wise kernels (the PLC_FP64 solve, and the FP64 phase of the mixed
// solve).
#include "launch.cuh"

namespace plc {
bool grad_sums_ff(plc_ctx* c, const double* s, const double* w, const int32_t* N, double nbar,
                  bool jac) {
  return grad_sums_ff_impl(c, s, w, N, nbar, jac);
}
template void prior_apply<double>(plc_ctx*, const double*, double*);
template void hessvec_s<double>(plc_ctx*, const double*, const double*, double, const double*, double*);
template void grad_public<double>(plc_ctx*, const double*, const double*, const int32_t*, double,
                                  double*);
template void grad_newton<double, double, double>(plc_ctx*, const double*, const double*,
                                                  const int32_t*, double, double*, double*,
                                                  double*, double*, bool);
template void grad_newton<double, double, float>(plc_ctx*, const double*, const double*,
                                                 const int32_t*, double, double*, double*, float*,
                                                 float*, bool);
template void newton_update<double, double>(plc_ctx*, const double*, const double*, const double*,
                                            const double*, const double*, const double*,
                                            const int32_t*, const double*, double, double, bool,
                                            double*, double*, double*, double*, double*,
                                            const double*);
template void newton_update<double, float>(plc_ctx*, const double*, const double*, const double*,
                                           const float*, const float*, const float*,
                                           const int32_t*, const double*, double, double, bool,
                                           double*, double*, double*, float*, float*,
                                           const double*);
template void grad_newton_g<double, double, double>(plc_ctx*, const double*, const double*,
                                                    const int32_t*, double, double*, double*,
                                                    double*, double*, bool);
template void grad_newton_g<double, double, float>(plc_ctx*, const double*, const double*,
                                                   const int32_t*, double, double*, double*,
                                                   float*, float*, bool);
template void newton_update_g<double, double>(plc_ctx*, const double*, const double*,
                                              const double*, const double*, const double*,
                                              const double*, const int32_t*, const double*,
                                              double, double, bool, double*, double*, double*,
                                              double*, double*);
template void newton_update_g<double, float>(plc_ctx*, const double*, const double*,
                                             const double*, const float*, const float*,
                                             const float*, const int32_t*, const double*, double,
                                             double, bool, double*, double*, double*, float*,
                                             float*);
template void boundary_step<double, double>(plc_ctx*, const double*, const double*, const int32_t*);
template void boundary_step<double, float>(plc_ctx*, const double*, const float*, const int32_t*);
template void cg_hv<double>(plc_ctx*, const double*, const double*, double*, double*, bool);
template void vjp_amplitude<double>(plc_ctx*, const double*, const double*);
template void diag_start<double>(plc_ctx*, double*, const int32_t*, const double*, double);
template void diag_start_g<double>(plc_ctx*, double*, const int32_t*, const double*, double);
template void lsq_init<double>(plc_ctx*, const int32_t*, const double*, double, double*, double*,
                              bool);
template void cg_init<double>(plc_ctx*, const double*, const double*, double*, bool);
template void cg_update<double>(plc_ctx*, double*, double*, const double*, const double*,
                                const double*, bool, double, int);
template void diag<double>(plc_ctx*, const double*, const double*, double, double*);
}  // namespace plc
