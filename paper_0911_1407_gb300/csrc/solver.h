// solver.h -- host drivers of the MAP solve and its adjoint.
#pragma once
#include "ctx.h"

namespace plc {
template <typename TC>
plc_status newton_map(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* s,
                      const plc_opts& o, plc_stats* st);
template <typename TC>
plc_status map_vjp(plc_ctx* c, const double* s_map, const double* w, double nbar, const double* u,
                   double* vjp_N, double* vjp_lnA, const plc_opts& o, plc_stats* st);
// MAP of the Gaussian-prior Poisson model (Eq. MAPG); delta in/out.
template <typename TC>
plc_status gauss_map(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* delta,
                     const plc_opts& o, plc_stats* st);
template <typename TC>
plc_status wiener_lsq(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* delta,
                      const plc_opts& o, plc_stats* st);
}  // namespace plc
