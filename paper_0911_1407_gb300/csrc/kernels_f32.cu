// kernels_f32.cu -- FP32 instantiations (the PLC_MIXED operators and the
// FP32 conjugate-gradient inner solve with FP64 reductions) and the mixed
// FP64-state / FP32-direction Newton step.
#include "launch.cuh"

namespace plc {
template void prior_apply<float>(plc_ctx*, const float*, float*);
template void hessvec_s<float>(plc_ctx*, const float*, const float*, double, const float*, float*);
template void grad<float>(plc_ctx*, const float*, const float*, const int32_t*, double, float*,
                          float*, float*);
template void grad_step<double, float>(plc_ctx*, double*, const float*, double, const double*,
                                       const int32_t*, double, double*, double*, float*);
template void cg_hv<float>(plc_ctx*, const float*, const float*, float*, float*, bool);
template void vjp_amplitude<float>(plc_ctx*, const double*, const float*);
template void cg_init<float, double>(plc_ctx*, const double*, bool, const float*, float*, float*,
                                     double, int, bool);
template void cg_update<float>(plc_ctx*, float*, float*, const float*, const float*, const float*,
                               bool);
template void dirstats<float, double>(plc_ctx*, const float*, const double*, const float*,
                                      const double*, const int32_t*);
template void trial<float, double>(plc_ctx*, const float*, const double*, double);
template void diag<float>(plc_ctx*, const double*, const double*, double, float*);
template void convert<double, float>(plc_ctx*, const float*, double*);
template void convert<float, double>(plc_ctx*, const double*, float*);
}  // namespace plc
