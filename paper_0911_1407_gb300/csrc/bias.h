// bias.h -- launchers (bias.cuh, instantiated in bias_f32.cu / bias_f64.cu)
// and host driver (bias.cu) of the linear-bias model of Sec. 2.4.1.
#pragma once
#include "ctx.h"

namespace plc {
// y = S^-1 (x - shift).
template <typename T, typename TX>
void bias_prior(plc_ctx* c, const TX* x, double shift, T* y);
// u = 1 + B(e^s - 1) at s (xi null) or at s2 = s + tau xi (y2 = y + tau yxi);
// q = nbar w - N / u, Q = N / u^2 and the likelihood sums.
template <typename T, typename TC>
void bias_density(plc_ctx* c, const T* s, const TC* xi, double tau, T* s2, const T* y,
                  const T* yxi, T* y2, const int32_t* N, const double* w, double nbar, T* q,
                  TC* Q);
// g = y + e^s . B q, CG start r = -g, E = e^s, d1 = e^s . B q, Jacobi Dj.
template <typename T, typename TC>
void bias_gradient(plc_ctx* c, const T* s, const T* y, const T* q, const TC* Q, T* g, TC* r,
                   TC* E, TC* d1, TC* Dj, bool jac);
// CG Hessian-vector product (direction from r; FinAlpha).
template <typename TC>
void bias_cg_hv(plc_ctx* c, const TC* r, const TC* Dj, TC* p, const TC* E, const TC* Q,
                const TC* d1, TC* t, TC* t2, TC* Hp, bool jac);
// H v at a point with E, Q, d1 (v^T H v into red[0]).
template <typename T>
void bias_hv(plc_ctx* c, const T* v, const T* E, const T* Q, const T* d1, T* t, T* t2, T* Hv);
// x = p and max |x| into the scalars' xmax.
template <typename TC> void bias_fallback(plc_ctx* c, const TC* p, TC* x);

// MAP of the linear-bias model (host-driven Newton-Krylov), s in/out (FP64).
template <typename TC>
plc_status bias_map(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* s,
                    const plc_opts& o, plc_stats* st);
}  // namespace plc
