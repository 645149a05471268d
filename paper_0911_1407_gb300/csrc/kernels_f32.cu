// kernels_f32.cu -- FP32 instantiations: the PLC_MIXED operators, the FP32
// phase of the mixed solve and its FP32 conjugate-gradient inner solve
// (FP64 reductions throughout).
#include "launch.cuh"

namespace plc {
template void prior_apply<float>(plc_ctx*, const float*, float*);
template void hessvec_s<float>(plc_ctx*, const float*, const float*, double, const float*, float*);
template void grad_public<float>(plc_ctx*, const float*, const float*, const int32_t*, double,
                                 float*);
template void grad_newton<float, float, float>(plc_ctx*, const float*, const double*,
                                               const int32_t*, double, float*, float*, float*,
                                               float*, bool);
template void newton_update<float, float>(plc_ctx*, const float*, const float*, const float*,
                                          const float*, const float*, const float*,
                                          const int32_t*, const double*, double, double, bool,
                                          float*, float*, float*, float*, float*, const double*);
template void grad_newton_g<float, float, float>(plc_ctx*, const float*, const double*,
                                                 const int32_t*, double, float*, float*, float*,
                                                 float*, bool);
template void newton_update_g<float, float>(plc_ctx*, const float*, const float*, const float*,
                                            const float*, const float*, const float*,
                                            const int32_t*, const double*, double, double, bool,
                                            float*, float*, float*, float*, float*);
template void boundary_step<float, float>(plc_ctx*, const float*, const float*, const int32_t*);
template void cg_hv<float>(plc_ctx*, const float*, const float*, float*, float*, bool);
template void vjp_amplitude<float>(plc_ctx*, const double*, const float*);
template void diag_start<float>(plc_ctx*, float*, const int32_t*, const double*, double);
template void diag_start_g<float>(plc_ctx*, float*, const int32_t*, const double*, double);
template void lsq_init<float>(plc_ctx*, const int32_t*, const double*, double, float*, float*,
                              bool);
template void cg_init<float>(plc_ctx*, const double*, const float*, float*, bool);
template void cg_update<float>(plc_ctx*, float*, float*, const float*, const float*, const float*,
                               bool, double, int);
template void diag<float>(plc_ctx*, const double*, const double*, double, float*);
template void convert<double, float>(plc_ctx*, const float*, double*);
template void convert<float, double>(plc_ctx*, const double*, float*);
}  // namespace plc
