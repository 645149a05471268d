// solver.cu -- host driver of the inexact Newton-Krylov MAP solve (Sec. 3.1)
// and of the implicit adjoint.  Scalars live on the device; the host reads
// them once per gradient, once per chunk of CG iterations and once per
// line-search trial.
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
  double scale() const { return (like + Ns) + Nabs + std::fabs(f()); }
};

GradSums grad_sums(const plc_ctx* c) {
  const double* r = c->sc_host->red;
  return GradSums{r[0], r[1], r[2], r[3], r[4]};
}

// Enqueue CG iterations in chunks until the device flags convergence,
// breakdown or the iteration cap.  Returns the iterations performed.
template <typename TC>
int run_cg(plc_ctx* c, TC* x, TC* r, TC* p, TC* Hp, const TC* D, bool jac, int max_cg, int chunk) {
  int launched = 0;
  read_scalars(c);
  while (!c->sc_host->done && launched < max_cg) {
    const int k = std::min(std::max(chunk, 1), max_cg - launched);
    for (int i = 0; i < k; ++i) {
      cg_hv<TC>(c, r, D, p, Hp, jac);
      cg_update<TC>(c, x, r, p, Hp, D, jac);
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
  double* g = dfield<double>(c->f_g);
  double* D = dfield<double>(c->f_D);
  TC* Dc = kMixed ? dfield<TC>(c->f_D32) : dfield<TC>(c->f_D);
  float* D32 = kMixed ? dfield<float>(c->f_D32) : nullptr;
  TC* r = dfield<TC>(c->f_r);
  TC* x = dfield<TC>(c->f_x);
  TC* p = dfield<TC>(c->f_p);
  TC* Hp = dfield<TC>(c->f_Hp);
  const bool jac = o.precond == 1;

  plc_stats S{};
  reset_ticket(c);
  grad<double>(c, s, w, N, nbar, g, D, D32);
  read_scalars(c);
  S.grad_evals = 1;
  GradSums gs = grad_sums(c);
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
    if (rel < o.tol) break;
    if (it >= o.max_newton) { status = PLC_ERR_NOT_CONVERGED; break; }
    // inexact Newton direction: H xi = -g to relative residual eta
    const double eta = std::min(o.eta_max, std::sqrt(rel));
    cg_init<TC, double>(c, g, true, Dc, r, x, eta * eta, o.max_cg, jac);
    const int iters = run_cg<TC>(c, x, r, p, Hp, Dc, jac, o.max_cg, o.cg_chunk);
    S.cg_iters += iters;
    S.hv_count += iters;
    if (iters == 0) {
      status = c->sc_host->breakdown ? PLC_ERR_CG_BREAKDOWN : PLC_OK;
      break;
    }
    // step length of Eq. (New5) with xi^T H xi = -xi^T g - xi^T r
    dirstats<TC, double>(c, x, g, r, D, N);
    read_scalars(c);
    const double* ds = c->sc_host->red;
    const double xg = ds[0], xr = ds[1], Dxx = ds[2], xD = ds[3], xN = ds[4], xmax = ds[5];
    const double xHx = -xg - xr;
    double tau = -xg / xHx;
    if (tau * xmax > o.step_cap) tau = o.step_cap / xmax;
    // Armijo backtracking; the prior part of -ln P is quadratic in tau:
    //   1/2 (s + tau xi - mu)^T S^-1 (s + tau xi - mu) = P0 + tau a1 + tau^2 a2 / 2
    // with a1 = xi^T S^-1 (s - mu) = xi^T (g - D + N), a2 = xi^T S^-1 xi = xi^T (H xi - D xi).
    const double a1 = xg - xD + xN, a2 = -xg - xr - Dxx;
    const double P0 = 0.5 * gs.prior2;
    const double f0 = gs.f(), scale = gs.scale();
    for (int q = 0; q < 30; ++q) {
      trial<TC, double>(c, x, D, tau);
      read_scalars(c);
      const double ftry = P0 + tau * a1 + 0.5 * tau * tau * a2 + c->sc_host->red[0] - gs.Ns - tau * xN;
      if (ftry <= f0 + 1e-4 * tau * xg || -tau * xg < 1e-13 * scale) break;
      tau *= 0.5;
    }
    grad_step<double, TC>(c, s, x, tau, w, N, nbar, g, D, D32);
    read_scalars(c);
    S.grad_evals += 1;
    gs = grad_sums(c);
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
  TC* Dc = kMixed ? dfield<TC>(c->f_D32) : dfield<TC>(c->f_D);
  TC* r = dfield<TC>(c->f_r);
  TC* x = dfield<TC>(c->f_x);
  TC* p = dfield<TC>(c->f_p);
  TC* Hp = dfield<TC>(c->f_Hp);
  const bool jac = o.precond == 1;
  plc_stats S{};
  reset_ticket(c);
  diag<TC>(c, s_map, w, nbar, Dc);
  cg_init<TC, double>(c, u, false, Dc, r, x, o.tol * o.tol, o.max_cg, jac);
  const int iters = run_cg<TC>(c, x, r, p, Hp, Dc, jac, o.max_cg, o.cg_chunk);
  S.cg_iters = iters;
  S.hv_count = iters;
  const plc::DevScalars& h = *c->sc_host;
  S.grad_rel = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
  plc_status status = PLC_OK;
  if (h.breakdown && iters == 0) status = PLC_ERR_CG_BREAKDOWN;
  else if (!h.done || (h.rr > h.rtol2 * h.bnorm2)) status = PLC_ERR_NOT_CONVERGED;
  if (vjp_N) {
    if (kMixed) convert<double, float>(c, reinterpret_cast<const float*>(x), vjp_N);
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
