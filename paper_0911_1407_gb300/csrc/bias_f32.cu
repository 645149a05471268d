// bias_f32.cu -- FP32 instantiations of the linear-bias launchers.
#include "bias.cuh"
#include "bias.h"

namespace plc {
template void bias_prior<float, float>(plc_ctx*, const float*, double, float*);
template void bias_density<float, float>(plc_ctx*, const float*, const float*, double, float*,
                                         const float*, const float*, float*, const int32_t*,
                                         const double*, double, float*, float*);
template void bias_gradient<float, float>(plc_ctx*, const float*, const float*, const float*,
                                          const float*, float*, float*, float*, float*, float*,
                                          bool);
template void bias_cg_hv<float>(plc_ctx*, const float*, const float*, float*, const float*,
                                const float*, const float*, float*, float*, float*, bool);
template void bias_hv<float>(plc_ctx*, const float*, const float*, const float*, const float*,
                             float*, float*, float*);
template void bias_fallback<float>(plc_ctx*, const float*, float*);
}  // namespace plc
