// solver.cu -- host driver of the inexact Newton-Krylov MAP solve (Sec. 3.1)
// and of the implicit adjoint.  Scalars live on the device; the host reads
// them after each gradient and after each chunk of CG iterations.
//
// One Newton step:
//   1. CG on H xi = -g (r = -g and r^T M^-1 r come from the gradient), to a
//      relative residual eta = min(eta_max, max(sqrt(rel), 0.3 tol / rel)),
//      rel = ||g|| / ||g0||;
//   2. tau from Eq. (New5), tau = -xi^T g / xi^T H xi, with both sums taken
//      from the CG recurrences (xi^T b = sum alpha_k r_k^T z_k,
//      xi^T H xi = sum alpha_k^2 p_k^T H p_k), capped so max |tau xi| <=
//      step_cap;
//   3. Armijo backtracking.  A trial point s + tau xi needs no FFT: S^-1 is
//      linear and the CG already holds S^-1 xi = (b - r) - D xi, so the
//      prior term is carried forward, y' = y + tau S^-1 xi, and the trial
//      gradient g' = y' + nbar w e^{s'} - N and -ln P come from one
//      element-wise pass (k_newton_update).
// y = S^-1 (s - mu) is evaluated through the FFT only at the start and, for
// PLC_MIXED, once more when the solve moves from FP32 to FP64 state.  The
// rounding of each carried increment is relative to the gradient at that
// step, so after that FP64 refresh the gradient stays accurate to FP64
// relative to ||g0|| (iterative refinement).  PLC_MIXED keeps s, y, g in FP32
// while ||g|| / ||g0|| >= max(mixed_switch, tol) and the FP32 steps still
// converge, in FP64 after that; the stopping test is only passed on an FP64
// gradient, so a solve that reaches tol in FP32 ends with one FP64 refresh.  The CG runs in the precision of its fields (FP32
// for PLC_MIXED).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <utility>

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
// breakdown or the iteration cap; chunks start at `first` iterations and
// double (up to `chunk`), so few iterations are enqueued past the end.
// Returns the iterations performed.
template <typename TC>
int run_cg(plc_ctx* c, TC* x, TC* r, TC* p, TC* Hp, const TC* D, bool jac, double rtol2,
           int max_cg, int chunk, int first) {
  int launched = 0;
  int k = std::max(1, std::min(first, chunk));
  read_scalars(c);
  while (!c->sc_host->done && launched < max_cg) {
    k = std::min(k, max_cg - launched);
    for (int i = 0; i < k; ++i) {
      cg_hv<TC>(c, r, D, p, Hp, jac);
      cg_update<TC>(c, x, r, p, Hp, D, jac, rtol2, max_cg);
    }
    launched += k;
    read_scalars(c);
    k = std::min(2 * k, std::max(chunk, 1));
  }
  return c->sc_host->iter;
}

template <typename T> T* as(void* p) { return static_cast<T*>(p); }

// One set of Newton state fields: s, y = S^-1 (s - mu), g (precision of the
// phase), the CG diagonal D and the CG start r = -g (CG precision).
struct State {
  void* s;
  void* y;
  void* g;
  void* D;
  void* r;
};

// The two models of the solve.  Lognormal prior (Sec. 2.3, Eq. MAPLNUB):
// unknown s = ln(1 + delta), steps capped by max |tau xi| <= step_cap.
// Gaussian prior (Sec. 2.2.2, Eq. MAPG): unknown delta, steps kept inside
// the domain 1 + delta > 0 (cells with N > 0) by the fraction to the
// boundary, tau <= 0.99 / max(-xi / (1 + delta)).
struct Lognormal {
  static constexpr bool kBoundary = false;
  // FP32 phase: g is not stored; the trial forms it from y, D and N
  static constexpr bool kNoG32 = true;
  // ||g||^2 at the prior mean mu, where S^-1 (s - mu) = 0: g = nbar w e^mu - N
  static void g0_at_mean(plc_ctx* c, const double* s, const int32_t* N, const double* w,
                         double nbar) {
    plc::g0_at_mean(c, s, N, w, c->mu, nbar * std::exp(c->mu));
  }
  template <typename TS>
  static void start(plc_ctx* c, TS* s, const int32_t* N, const double* w, double nbar) {
    diag_start<TS>(c, s, N, w, nbar);
  }
  template <typename T, typename TS, typename TC>
  static void gradient(plc_ctx* c, const TS* s, const double* w, const int32_t* N, double nbar,
                       T* y, T* g, TC* D, TC* r, bool jac) {
    grad_newton<T, TS, TC>(c, s, w, N, nbar, y, g, D, r, jac);
  }
  // the sums of the FP64 gradient alone (false: not offered for this length)
  static bool gradient_sums(plc_ctx* c, const double* s, const double* w, const int32_t* N,
                            double nbar, bool jac) {
    return grad_sums_ff(c, s, w, N, nbar, jac);
  }
  template <typename T, typename TC>
  static void trial(plc_ctx* c, const T* s, const T* y, const T* g, const TC* r, const TC* xi,
                    const TC* D, const int32_t* N, const double* w, double nbar, double tau,
                    bool jac, T* s2, T* y2, T* g2, TC* D2, TC* r2) {
    newton_update<T, TC>(c, s, y, g, r, xi, D, N, w, nbar, tau, jac, s2, y2, g2, D2, r2);
  }
};
struct GaussPrior {
  static constexpr bool kBoundary = true;
  static constexpr bool kNoG32 = false;
  // ||g||^2 at delta = 0, the prior mean: g = nbar w - N
  static void g0_at_mean(plc_ctx* c, const double* s, const int32_t* N, const double* w,
                         double nbar) {
    plc::g0_at_mean(c, s, N, w, 0.0, nbar);
  }
  template <typename TS>
  static void start(plc_ctx* c, TS* s, const int32_t* N, const double* w, double nbar) {
    diag_start_g<TS>(c, s, N, w, nbar);
  }
  template <typename T, typename TS, typename TC>
  static void gradient(plc_ctx* c, const TS* s, const double* w, const int32_t* N, double nbar,
                       T* y, T* g, TC* D, TC* r, bool jac) {
    grad_newton_g<T, TS, TC>(c, s, w, N, nbar, y, g, D, r, jac);
  }
  static bool gradient_sums(plc_ctx*, const double*, const double*, const int32_t*, double, bool) {
    return false;
  }
  template <typename T, typename TC>
  static void trial(plc_ctx* c, const T* s, const T* y, const T* g, const TC* r, const TC* xi,
                    const TC* D, const int32_t* N, const double* w, double nbar, double tau,
                    bool jac, T* s2, T* y2, T* g2, TC* D2, TC* r2) {
    newton_update_g<T, TC>(c, s, y, g, r, xi, D, N, w, nbar, tau, jac, s2, y2, g2, D2, r2);
  }
};

}  // namespace

template <typename Model, typename TC>
plc_status newton_map_model(plc_ctx* c, const int32_t* N, const double* w, double nbar,
                            double* s_out, const plc_opts& o, plc_stats* st) {
  constexpr bool kMixed = std::is_same<TC, float>::value;
  const auto t0 = std::chrono::steady_clock::now();
  void** F = c->wf;
  TC* x = as<TC>(F[10]);
  TC* p = as<TC>(F[11]);
  TC* Hp = as<TC>(F[12]);
  const bool jac = o.precond == 1;
  bool fp64 = !kMixed || !(o.mixed_switch < 1.0);
  State cur{fp64 ? (void*)s_out : F[0], F[2], F[4], F[6], F[8]};
  State alt{F[1], F[3], F[5], F[7], F[9]};

  plc_stats S{};
  double g0 = 0.0;   // ||g0|| of the stopping test (set below)
  auto g32 = [](const State& f) { return Model::kNoG32 ? nullptr : as<float>(f.g); };
  // y, g, D, r and the sums at cur.s through the FFT (phase precision)
  auto fft_gradient = [&]() {
    if (fp64) {
      Model::template gradient<double, double, TC>(c, as<double>(cur.s), w, N, nbar,
                                                   as<double>(cur.y), as<double>(cur.g),
                                                   as<TC>(cur.D), as<TC>(cur.r), jac);
      S.grad_ffts_fp64 += 1;
    } else if constexpr (kMixed) {
      Model::template gradient<float, float, float>(c, as<float>(cur.s), w, N, nbar,
                                                    as<float>(cur.y), g32(cur),
                                                    as<float>(cur.D), as<float>(cur.r), jac);
    }
    read_scalars(c);
    S.grad_evals += 1;
    S.grad_ffts += 1;
    return grad_sums(c);
  };
  auto trial = [&](double tau) {
    if (fp64) {
      Model::template trial<double, TC>(c, as<double>(cur.s), as<double>(cur.y),
                                        as<double>(cur.g), as<TC>(cur.r), x, as<TC>(cur.D), N, w,
                                        nbar, tau, jac, as<double>(alt.s), as<double>(alt.y),
                                        as<double>(alt.g), as<TC>(alt.D), as<TC>(alt.r));
    } else if constexpr (kMixed) {
      Model::template trial<float, float>(c, as<float>(cur.s), as<float>(cur.y), g32(cur),
                                          as<float>(cur.r), x, as<float>(cur.D), N, w, nbar,
                                          tau, jac, as<float>(alt.s), as<float>(alt.y),
                                          g32(alt), as<float>(alt.D), as<float>(alt.r));
    }
    read_scalars(c);
    S.grad_evals += 1;
    return grad_sums(c);
  };
  // move the FP32 state to FP64: s in the caller's buffer, fresh FP64
  // gradient.  When the FP32 gradient already passes the stopping test
  // (check), the FP64 gradient's sums are taken first without its fields:
  // if they pass too the solve ends there, else the full gradient follows.
  auto to_fp64 = [&](bool check) {
    if constexpr (kMixed) convert<double, float>(c, as<float>(cur.s), s_out);
    fp64 = true;
    cur.s = s_out;
    alt.s = F[1];
    if (check && Model::gradient_sums(c, s_out, w, N, nbar, jac)) {
      read_scalars(c);
      S.grad_evals += 1;
      S.grad_ffts += 1;
      S.grad_ffts_fp64 += 1;
      const GradSums gc = grad_sums(c);
      const double rel = std::sqrt(gc.gg) / g0;
      if (rel < o.tol && std::isfinite(gc.f())) return gc;
    }
    return fft_gradient();
  };

  reset_ticket(c);
  // ||g0|| at the caller's start.  With the diagonal start the gradient
  // there serves only this norm: none is taken when g0_norm is given, and
  // at the prior mean it needs no transform.
  GradSums gs{};
  g0 = o.g0_norm;
  bool first = true;
  if (o.start >= 1) {
    if (g0 > 0.0) {
      first = false;
    } else {
      // start 2: the caller's start is the prior mean by definition (s_out
      // is not read)
      Model::g0_at_mean(c, o.start == 2 ? nullptr : s_out, N, w, nbar);
      read_scalars(c);
      if (!c->sc_host->off_mean) {
        g0 = std::sqrt(c->sc_host->red[2]);
        first = false;
      }
    }
  }
  if (first) {
    if (!fp64) {
      if constexpr (kMixed) convert<float, double>(c, s_out, as<float>(cur.s));
    }
    gs = fft_gradient();
    if (!(g0 > 0.0)) g0 = std::sqrt(gs.gg);
  }
  S.g0_norm = g0;
  if (o.start >= 1) {
    // iterate from the per-cell diagonal-prior MAP (g0 stays at s_in)
    if (fp64) Model::template start<double>(c, as<double>(cur.s), N, w, nbar);
    else if constexpr (kMixed) Model::template start<float>(c, as<float>(cur.s), N, w, nbar);
    gs = fft_gradient();
  }
  plc_status status = PLC_OK;
  int it = 0, prev_cg = 1;
  double prev_rel = 1.0;
  for (;;) {
    const double gnorm = std::sqrt(gs.gg);
    // a non-finite g0 (NaN or Inf in the caller's start or in w) would make
    // every relative norm look converged
    if (!std::isfinite(gnorm) || !std::isfinite(gs.f()) || !std::isfinite(g0)) {
      status = PLC_ERR_NONFINITE;
      break;
    }
    const double rel = g0 > 0.0 ? gnorm / g0 : 0.0;
    S.grad_rel = rel;
    S.neg_logpost = gs.f();
    // FP32 -> FP64: below the switch point, at the tolerance, or when an
    // FP32 Newton step in the fast-convergence range (rel < 1e-3) fails to
    // halve the gradient (the FP32 rounding floor)
    if (!fp64 && (rel < o.mixed_switch || rel < o.tol ||
                  (it > 0 && rel < 1e-3 && rel > 0.5 * prev_rel))) {
      gs = to_fp64(rel < o.tol);
      continue;
    }
    prev_rel = rel;
    if (rel < o.tol) break;
    if (it >= o.max_newton) { status = PLC_ERR_NOT_CONVERGED; break; }
    // 1. inexact Newton direction
    // forcing term: superlinear sqrt(rel), but no tighter than the stop test
    // needs (0.3 tol / rel) and never above eta_max
    const double eta = std::min(o.eta_max, std::max(std::sqrt(rel), 0.3 * o.tol / rel));
    const int iters = run_cg<TC>(c, x, as<TC>(cur.r), p, Hp, as<TC>(cur.D), jac, eta * eta,
                                 o.max_cg, o.cg_chunk, prev_cg);
    prev_cg = iters;
    S.cg_iters += iters;
    S.hv_count += iters;
    if (iters == 0) {
      status = c->sc_host->breakdown ? PLC_ERR_CG_BREAKDOWN : PLC_OK;
      break;
    }
    // 2. step length of Eq. (New5); b = -g, so xi^T g = -xi^T b
    const double xg = -c->sc_host->xb, xHx = c->sc_host->xHx, xmax = c->sc_host->xmax;
    double tau = -xg / xHx;
    if constexpr (Model::kBoundary) {
      if (fp64) boundary_step<double, TC>(c, as<double>(cur.s), x, N);
      else if constexpr (kMixed) boundary_step<float, float>(c, as<float>(cur.s), x, N);
      read_scalars(c);
      const double bmax = c->sc_host->bmax;
      if (bmax > 0.0) tau = std::min(tau, 0.99 / bmax);
    } else {
      if (tau * xmax > o.step_cap) tau = o.step_cap / xmax;
    }
    // 3. Armijo backtracking on element-wise trial points
    const double eps = fp64 ? 1e-13 : 1e-6;     // rounding level of f
    const double f0 = gs.f(), scale = gs.scale();
    for (int q = 0; q < 30; ++q) {
      gs = trial(tau);
      if (gs.f() <= f0 + 1e-4 * tau * xg || -tau * xg < eps * scale) break;
      tau *= 0.5;
    }
    std::swap(cur, alt);
    ++it;
  }
  // leave the iterate in the caller's buffer
  if (!fp64) {
    if constexpr (kMixed) convert<double, float>(c, as<float>(cur.s), s_out);
  } else if (cur.s != s_out) {
    check(cudaMemcpyAsync(s_out, cur.s, sizeof(double) * c->n3(), cudaMemcpyDeviceToDevice,
                          c->stream), "copy s");
  }
  check(cudaStreamSynchronize(c->stream), "stream synchronize");
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
  void** F = c->wf;
  TC* D = as<TC>(F[6]);
  TC* r = as<TC>(F[8]);
  TC* x = as<TC>(F[10]);
  TC* p = as<TC>(F[11]);
  TC* Hp = as<TC>(F[12]);
  const bool jac = o.precond == 1;
  plc_stats S{};
  reset_ticket(c);
  diag<TC>(c, s_map, w, nbar, D);
  cg_init<TC>(c, u, D, r, jac);
  const double rtol2 = o.tol * o.tol;
  const int iters = run_cg<TC>(c, x, r, p, Hp, D, jac, rtol2, o.max_cg, o.cg_chunk, o.cg_chunk);
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

// LSQ-Wiener filter (Sec. 4.1.1, Eq. WF with unity bias; Table 1): one
// Jacobi-preconditioned CG solve of (S^-1 + diag(nbar w)) delta = N - nbar w
// from delta = 0 to relative residual tol, in the CG precision of the
// context (FP32 for PLC_MIXED, so a relative residual of about 1e-6 at best).
template <typename TC>
plc_status wiener_lsq(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* delta,
                      const plc_opts& o, plc_stats* st) {
  constexpr bool kMixed = std::is_same<TC, float>::value;
  const auto t0 = std::chrono::steady_clock::now();
  void** F = c->wf;
  TC* D = as<TC>(F[6]);
  TC* r = as<TC>(F[8]);
  TC* x = as<TC>(F[10]);
  TC* p = as<TC>(F[11]);
  TC* Hp = as<TC>(F[12]);
  const bool jac = o.precond == 1;
  reset_ticket(c);
  lsq_init<TC>(c, N, w, nbar, D, r, jac);
  const double rtol2 = o.tol * o.tol;
  const int iters = run_cg<TC>(c, x, r, p, Hp, D, jac, rtol2, o.max_cg, o.cg_chunk, o.cg_chunk);
  const DevScalars& h = *c->sc_host;
  plc_status status = PLC_OK;
  if (h.breakdown && iters == 0) status = PLC_ERR_CG_BREAKDOWN;
  else if (h.rr > rtol2 * h.bnorm2) status = PLC_ERR_NOT_CONVERGED;
  if (iters == 0)            // N = nbar w everywhere: delta = 0
    check(cudaMemsetAsync(x, 0, sizeof(TC) * c->n3(), c->stream), "clear");
  if constexpr (kMixed) convert<double, float>(c, x, delta);
  else check(cudaMemcpyAsync(delta, x, sizeof(double) * c->n3(), cudaMemcpyDeviceToDevice, c->stream),
             "copy delta");
  check(cudaStreamSynchronize(c->stream), "stream synchronize");
  if (st) {
    *st = plc_stats{};
    st->cg_iters = iters;
    st->hv_count = iters;
    st->grad_rel = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
    st->g0_norm = std::sqrt(h.bnorm2);
    st->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

template plc_status wiener_lsq<double>(plc_ctx*, const int32_t*, const double*, double, double*,
                                       const plc_opts&, plc_stats*);
template plc_status wiener_lsq<float>(plc_ctx*, const int32_t*, const double*, double, double*,
                                      const plc_opts&, plc_stats*);

template <typename TC>
plc_status newton_map(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* s,
                      const plc_opts& o, plc_stats* st) {
  return newton_map_model<Lognormal, TC>(c, N, w, nbar, s, o, st);
}

template <typename TC>
plc_status gauss_map(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* delta,
                     const plc_opts& o, plc_stats* st) {
  return newton_map_model<GaussPrior, TC>(c, N, w, nbar, delta, o, st);
}

template plc_status newton_map<double>(plc_ctx*, const int32_t*, const double*, double, double*,
                                       const plc_opts&, plc_stats*);
template plc_status newton_map<float>(plc_ctx*, const int32_t*, const double*, double, double*,
                                      const plc_opts&, plc_stats*);
template plc_status gauss_map<double>(plc_ctx*, const int32_t*, const double*, double, double*,
                                      const plc_opts&, plc_stats*);
template plc_status gauss_map<float>(plc_ctx*, const int32_t*, const double*, double, double*,
                                     const plc_opts&, plc_stats*);
template plc_status map_vjp<double>(plc_ctx*, const double*, const double*, double, const double*,
                                    double*, double*, const plc_opts&, plc_stats*);
template plc_status map_vjp<float>(plc_ctx*, const double*, const double*, double, const double*,
                                   double*, double*, const plc_opts&, plc_stats*);

}  // namespace plc
