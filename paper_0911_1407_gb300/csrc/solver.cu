// solver.cu -- host driver of the inexact Newton-Krylov MAP solve (Sec. 3.1)
// and of the implicit adjoint.  Scalars live on the device; the host reads
// them after each gradient and after each chunk of CG iterations.
//
// One Newton step:
//   1. CG on H xi = -g (r = -g and r^T M^-1 r come from the gradient pass),
//      to a relative residual eta = min(eta_max, sqrt(||g|| / ||g0||));
//   2. tau from Eq. (New5), tau = -xi^T g / xi^T H xi, with both sums taken
//      from the CG recurrences (xi^T b = sum alpha_k r_k^T z_k,
//      xi^T H xi = sum alpha_k^2 p_k^T H p_k), capped so max |tau xi| <=
//      step_cap;
//   3. Armijo backtracking in which every trial is a gradient evaluation at
//      s + tau xi (its epilogue also returns -ln P), so the accepted trial
//      leaves the next gradient, diagonal and CG start in place.
// PLC_MIXED evaluates the gradient in FP32 while ||g|| / ||g0|| >=
// mixed_switch and in FP64 after that; the stopping test is only passed on
// an FP64 gradient.  The CG always runs in the precision of its fields (FP32
// for PLC_MIXED).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>

#include "ctx.h"
#include "solver.h"

namespace plc {

namespace {

struct GradSums {
  double prior2;   // (s - mu)^T S^-1 (s - mu)
  double like;     // sum (D - N s)
  double gg;       // ||g||^2
  double Ns;       // sum N s
  double Nabs;     // sum N |s|
  double f() const { return 0.5 * prior2 + like; }
  // magnitude of the terms of -ln P, for the rounding level of f
  double scale() const { return (like + Ns) + Nabs + std::fabs(f()); }
};

GradSums grad_sums(const plc_ctx* c) {
  const double* r = c->sc_host->red;
  return GradSums{r[0], r[1], r[2], r[3], r[4]};
}

// Enqueue CG iterations in chunks until the device flags convergence,
// breakdown or the iteration cap.  Returns the iterations performed.
template <typename TC>
int run_cg(plc_ctx* c, TC* x, TC* r, TC* p, TC* Hp, const TC* D, bool jac, double rtol2,
           int max_cg, int chunk) {
  int launched = 0;
  read_scalars(c);
  while (!c->sc_host->done && launched < max_cg) {
    const int k = std::min(std::max(chunk, 1), max_cg - launched);
    for (int i = 0; i < k; ++i) {
      cg_hv<TC>(c, r, D, p, Hp, jac);
      cg_update<TC>(c, x, r, p, Hp, D, jac, rtol2, max_cg);
    }
    launched += k;
    read_scalars(c);
  }
  return c->sc_host->iter;
}

template <typename TC> TC* dfield(void* p) { return static_cast<TC*>(p); }

}  // namespace

template <typename TC>
plc_status newton_map(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* s,
                      const plc_opts& o, plc_stats* st) {
  constexpr bool kMixed = std::is_same<TC, float>::value;
  const auto t0 = std::chrono::steady_clock::now();
  TC* D = kMixed ? dfield<TC>(c->f_D32) : dfield<TC>(c->f_D);
  TC* r = dfield<TC>(c->f_r);
  TC* x = dfield<TC>(c->f_x);
  TC* p = dfield<TC>(c->f_p);
  TC* Hp = dfield<TC>(c->f_Hp);
  const bool jac = o.precond == 1;

  plc_stats S{};
  // Gradient at s (+ dtau xi); fp64 selects the transform precision.
  auto gradient = [&](bool fp64, const TC* xi, double dtau) {
    if constexpr (kMixed) {
      if (fp64) grad_newton<double, TC>(c, s, xi, dtau, w, N, nbar, D, r, jac);
      else grad_newton<float, TC>(c, s, xi, dtau, w, N, nbar, D, r, jac);
    } else {
      (void)fp64;
      grad_newton<double, TC>(c, s, xi, dtau, w, N, nbar, D, r, jac);
    }
    read_scalars(c);
    S.grad_evals += 1;
    if (fp64 || !kMixed) S.grad_evals_fp64 += 1;
    return grad_sums(c);
  };

  reset_ticket(c);
  bool fp64 = !kMixed || !(o.mixed_switch < 1.0);
  GradSums gs = gradient(fp64, nullptr, 0.0);
  const double g0 = o.g0_norm > 0.0 ? o.g0_norm : std::sqrt(gs.gg);
  S.g0_norm = g0;
  plc_status status = PLC_OK;
  int it = 0;
  for (;;) {
    const double gnorm = std::sqrt(gs.gg);
    if (!std::isfinite(gnorm) || !std::isfinite(gs.f())) { status = PLC_ERR_NONFINITE; break; }
    const double rel = g0 > 0.0 ? gnorm / g0 : 0.0;
    S.grad_rel = rel;
    S.neg_logpost = gs.f();
    if (rel < o.tol) {
      if (fp64) break;
      fp64 = true;                       // confirm on an FP64 gradient at the same point
      gs = gradient(true, nullptr, 0.0);
      continue;
    }
    if (it >= o.max_newton) { status = PLC_ERR_NOT_CONVERGED; break; }
    // 1. inexact Newton direction
    const double eta = std::min(o.eta_max, std::sqrt(rel));
    const int iters = run_cg<TC>(c, x, r, p, Hp, D, jac, eta * eta, o.max_cg, o.cg_chunk);
    S.cg_iters += iters;
    S.hv_count += iters;
    if (iters == 0) {
      status = c->sc_host->breakdown ? PLC_ERR_CG_BREAKDOWN : PLC_OK;
      break;
    }
    // 2. step length of Eq. (New5); b = -g, so xi^T g = -xi^T b
    const double xg = -c->sc_host->xb, xHx = c->sc_host->xHx, xmax = c->sc_host->xmax;
    double tau = -xg / xHx;
    if (tau * xmax > o.step_cap) tau = o.step_cap / xmax;
    // 3. Armijo backtracking on gradient evaluations at s + tau xi
    const bool next_fp64 = fp64 || rel < o.mixed_switch;
    const double eps = (fp64 && next_fp64) ? 1e-13 : 1e-6;   // rounding level of f
    const double f0 = gs.f(), scale = gs.scale();
    double applied = 0.0;
    for (int q = 0; q < 30; ++q) {
      gs = gradient(next_fp64, x, tau - applied);
      applied = tau;
      if (gs.f() <= f0 + 1e-4 * tau * xg || -tau * xg < eps * scale) break;
      tau *= 0.5;
    }
    fp64 = next_fp64;
    ++it;
  }
  S.newton_iters = it;
  S.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = S;
  return status;
}

template <typename TC>
plc_status map_vjp(plc_ctx* c, const double* s_map, const double* w, double nbar, const double* u,
                   double* vjp_N, double* vjp_lnA, const plc_opts& o, plc_stats* st) {
  constexpr bool kMixed = std::is_same<TC, float>::value;
  const auto t0 = std::chrono::steady_clock::now();
  TC* D = kMixed ? dfield<TC>(c->f_D32) : dfield<TC>(c->f_D);
  TC* r = dfield<TC>(c->f_r);
  TC* x = dfield<TC>(c->f_x);
  TC* p = dfield<TC>(c->f_p);
  TC* Hp = dfield<TC>(c->f_Hp);
  const bool jac = o.precond == 1;
  plc_stats S{};
  reset_ticket(c);
  diag<TC>(c, s_map, w, nbar, D);
  cg_init<TC>(c, u, D, r, jac);
  const double rtol2 = o.tol * o.tol;
  const int iters = run_cg<TC>(c, x, r, p, Hp, D, jac, rtol2, o.max_cg, o.cg_chunk);
  S.cg_iters = iters;
  S.hv_count = iters;
  const DevScalars& h = *c->sc_host;
  S.grad_rel = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
  plc_status status = PLC_OK;
  if (h.breakdown && iters == 0) status = PLC_ERR_CG_BREAKDOWN;
  else if (h.rr > rtol2 * h.bnorm2) status = PLC_ERR_NOT_CONVERGED;
  if (iters == 0)            // u = 0 gives lam = 0
    check(cudaMemsetAsync(x, 0, sizeof(TC) * c->n3(), c->stream), "clear");
  if (vjp_N) {
    if constexpr (kMixed) convert<double, float>(c, x, vjp_N);
    else check(cudaMemcpyAsync(vjp_N, x, sizeof(double) * c->n3(), cudaMemcpyDeviceToDevice, c->stream),
               "copy vjp_N");
  }
  if (vjp_lnA) {
    vjp_amplitude<TC>(c, s_map, x);
    read_scalars(c);
    *vjp_lnA = c->sc_host->red[0];
  } else {
    check(cudaStreamSynchronize(c->stream), "stream synchronize");
  }
  S.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = S;
  return status;
}

template plc_status newton_map<double>(plc_ctx*, const int32_t*, const double*, double, double*,
                                       const plc_opts&, plc_stats*);
template plc_status newton_map<float>(plc_ctx*, const int32_t*, const double*, double, double*,
                                      const plc_opts&, plc_stats*);
template plc_status map_vjp<double>(plc_ctx*, const double*, const double*, double, const double*,
                                    double*, double*, const plc_opts&, plc_stats*);
template plc_status map_vjp<float>(plc_ctx*, const double*, const double*, double, const double*,
                                   double*, double*, const plc_opts&, plc_stats*);

}  // namespace plc
