// bias.cu -- host driver of the MAP solve with linear bias (Sec. 2.4.1):
// the lognormal prior of Sec. 2.3 with the Poisson likelihood of the galaxy
// field nbar w (1 + B delta_M), B the bias convolution.
//
// The inexact Newton-Krylov iteration of the unity-bias solve (Sec. 3.1):
// CG on H xi = -g with the exact Hessian (which need not be positive
// definite here: the CG stops at non-positive curvature and keeps its
// iterate, or takes the preconditioned gradient step when that happens on
// its first direction), tau from Eq. (New5) out of the CG sums (tau = 1 when
// xi^T H xi <= 0), max |tau xi| <= step_cap, Armijo backtracking with L = +inf
// (rejected) outside the domain u > 0.  The prior term y = S^-1 (s - mu) is
// carried forward with y + tau S^-1 xi (one pipeline per Newton step), so a
// trial costs one pipeline (u) and an accepted step one more (B q).
//
// Precision: PLC_FP64 runs everything in FP64.  PLC_MIXED keeps s, y, q in
// FP32 while ||g|| / ||g0|| >= max(mixed_switch, tol) and the FP32 steps
// still converge (as the unity-bias solve), then moves s to FP64, takes the
// gradient through FP64 pipelines and continues with FP64 state; the CG
// fields are FP32 throughout, and the stop test is passed on an FP64
// gradient.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "bias.h"

namespace plc {

namespace {

struct BSums {
  double prior2, like, gg, Nl, Nabs, rz;
  double f() const { return 0.5 * prior2 + like; }
  // magnitude of the terms of L, for the rounding level of f
  double scale() const { return (like + Nl) + Nabs + std::fabs(f()); }
};

BSums bsums(const plc_ctx* c) {
  const double* r = c->sc_host->red;
  return BSums{r[0], r[1], r[2], r[3], r[4], r[5]};
}

long long launches(const plc_ctx* c) {
  long long k = 0;
  for (int i = 0; i < S_NSITES; ++i) k += c->prof.launches[i];
  return k;
}

template <typename T> T* as(void* p) { return static_cast<T*>(p); }

// Fields of one precision phase: state in T, CG fields in TC.
template <typename T, typename TC> struct Fields {
  plc_ctx* c;
  const int32_t* N;
  const double* w;
  double nbar;
  bool jac;
  T* s[2];
  T* y[2];
  T* q;
  T* yxi;
  TC *E, *Q, *d1, *Dj, *t, *t2, *r, *x, *p, *Hp;
  int cur = 0;

  // gradient at s[cur] with y through the FFT
  BSums gradient() {
    bias_prior<T, T>(c, s[cur], c->mu, y[cur]);
    bias_density<T, TC>(c, s[cur], nullptr, 0.0, nullptr, y[cur], nullptr, nullptr, N, w, nbar,
                        q, Q);
    bias_gradient<T, TC>(c, s[cur], y[cur], q, Q, nullptr, r, E, d1, Dj, jac);
    read_scalars(c);
    return bsums(c);
  }
  // L at s[cur] + tau xi (into s[1 - cur], y[1 - cur], q, Q)
  BSums trial(double tau) {
    bias_density<T, TC>(c, s[cur], x, tau, s[1 - cur], y[cur], yxi, y[1 - cur], N, w, nbar, q,
                        Q);
    read_scalars(c);
    return bsums(c);
  }
  // gradient at the last trial point, which becomes the current one
  BSums accept() {
    cur = 1 - cur;
    bias_gradient<T, TC>(c, s[cur], y[cur], q, Q, nullptr, r, E, d1, Dj, jac);
    read_scalars(c);
    return bsums(c);
  }
  // CG in chunks (as the unity-bias driver); returns the iterations
  int cg(double rtol2, int max_cg, int chunk, int first) {
    int launched = 0;
    int k = std::max(1, std::min(first, chunk));
    read_scalars(c);
    while (!c->sc_host->done && launched < max_cg) {
      k = std::min(k, max_cg - launched);
      for (int i = 0; i < k; ++i) {
        bias_cg_hv<TC>(c, r, Dj, p, E, Q, d1, t, t2, Hp, jac);
        cg_update<TC>(c, x, r, p, Hp, Dj, jac, rtol2, max_cg);
      }
      launched += k;
      read_scalars(c);
      k = std::min(2 * k, std::max(chunk, 1));
    }
    return c->sc_host->iter;
  }
};

enum class End { kConverged, kSwitch, kCap, kNonFinite };

struct Progress {
  int it = 0, prev_cg = 1;
  double g0 = 0.0, prev_rel = 1.0;
  plc_stats S{};
};

// Newton steps in one precision until convergence, the FP32 -> FP64 switch
// (fp32_phase), the iteration cap or a non-finite value.
template <typename T, typename TC>
End newton_phase(Fields<T, TC>& F, BSums gs, const plc_opts& o, Progress& P, bool fp32_phase) {
  plc_ctx* c = F.c;
  for (;;) {
    const double gnorm = std::sqrt(gs.gg);
    if (!std::isfinite(gnorm) || !std::isfinite(gs.f()) || !std::isfinite(P.g0))
      return End::kNonFinite;
    const double rel = P.g0 > 0.0 ? gnorm / P.g0 : 0.0;
    P.S.grad_rel = rel;
    P.S.neg_logpost = gs.f();
    if (fp32_phase && (rel < o.mixed_switch || rel < o.tol ||
                       (P.it > 0 && rel < 1e-3 && rel > 0.5 * P.prev_rel)))
      return End::kSwitch;
    P.prev_rel = rel;
    if (rel < o.tol) return End::kConverged;
    if (P.it >= o.max_newton) return End::kCap;
    // 1. inexact Newton direction
    const double eta = std::min(o.eta_max, std::max(std::sqrt(rel), 0.3 * o.tol / rel));
    const int iters = F.cg(eta * eta, o.max_cg, o.cg_chunk, P.prev_cg);
    P.prev_cg = std::max(iters, 1);
    P.S.cg_iters += iters;
    P.S.hv_count += iters;
    // 2. step length of Eq. (New5) (b = -g: xi^T g = -xi^T b)
    double xg, xHx;
    if (iters == 0) {
      // non-positive curvature on the first direction p = M^-1 r: take it
      // (xi^T g = -r^T M^-1 r, xi^T H xi = p^T H p <= 0, so tau = 1)
      const double rz = c->sc_host->rz, pHp = c->sc_host->pHp;
      bias_fallback<TC>(c, F.p, F.x);
      read_scalars(c);
      xg = -rz;
      xHx = pHp;
    } else {
      xg = -c->sc_host->xb;
      xHx = c->sc_host->xHx;
    }
    const double xmax = c->sc_host->xmax;
    double tau = xHx > 0.0 ? -xg / xHx : 1.0;
    if (tau * xmax > o.step_cap) tau = o.step_cap / xmax;
    bias_prior<T, TC>(c, F.x, 0.0, F.yxi);
    // 3. Armijo backtracking; points outside the domain have L = +inf
    const double eps = sizeof(T) == 8 ? 1e-13 : 1e-6;
    const double f0 = gs.f(), scale = gs.scale();
    double ft = 0.0;
    for (int k = 0; k < 40; ++k) {
      ft = F.trial(tau).f();
      P.S.grad_evals += 1;
      if (std::isfinite(ft) && (ft <= f0 + 1e-4 * tau * xg || -tau * xg < eps * scale)) break;
      tau *= 0.5;
    }
    if (!std::isfinite(ft)) return End::kNonFinite;
    gs = F.accept();
    P.S.grad_ffts += 1;
    if (sizeof(T) == 8) P.S.grad_ffts_fp64 += 1;
    ++P.it;
  }
}

template <typename T, typename TC>
Fields<T, TC> make_fields(plc_ctx* c, const int32_t* N, const double* w, double nbar, bool jac,
                          T* s0, T* s1) {
  void** B = c->bwf;
  void** W = c->wf;
  Fields<T, TC> F{c, N, w, nbar, jac, {s0, s1}, {as<T>(B[2]), as<T>(B[3])}, as<T>(B[4]),
                  as<T>(B[5]), as<TC>(B[6]), as<TC>(B[7]), as<TC>(B[8]), as<TC>(B[9]),
                  as<TC>(B[10]), as<TC>(B[11]), as<TC>(W[8]), as<TC>(W[10]), as<TC>(W[11]),
                  as<TC>(W[12])};
  return F;
}

plc_status end_status(End e) {
  switch (e) {
    case End::kCap: return PLC_ERR_NOT_CONVERGED;
    case End::kNonFinite: return PLC_ERR_NONFINITE;
    default: return PLC_OK;
  }
}

}  // namespace

template <typename TC>
plc_status bias_map(plc_ctx* c, const int32_t* N, const double* w, double nbar, double* s_out,
                    const plc_opts& o, plc_stats* st) {
  constexpr bool kMixed = sizeof(TC) == 4;
  const auto t0 = std::chrono::steady_clock::now();
  const long long k0 = launches(c);
  const bool jac = o.precond == 1;
  Progress P;
  reset_ticket(c);
  End end;
  double* s64[2] = {s_out, as<double>(c->bwf[0])};
  if (kMixed && o.mixed_switch < 1.0) {
    auto F32 = make_fields<float, float>(c, N, w, nbar, jac, as<float>(c->bwf[0]),
                                         as<float>(c->bwf[1]));
    convert<float, double>(c, s_out, F32.s[0]);
    BSums gs = F32.gradient();
    P.S.grad_evals += 1;
    P.S.grad_ffts += 1;
    P.g0 = o.g0_norm > 0.0 ? o.g0_norm : std::sqrt(gs.gg);
    P.S.g0_norm = P.g0;
    end = newton_phase<float, float>(F32, gs, o, P, true);
    if (end == End::kSwitch) {
      // the FP32 iterate to FP64 (s_out; bwf[0] becomes the trial buffer
      // once the conversion has read it)
      convert<double, float>(c, F32.s[F32.cur], s_out);
      s64[1] = as<double>(c->bwf[F32.cur == 0 ? 1 : 0]);
      auto F64 = make_fields<double, TC>(c, N, w, nbar, jac, s64[0], s64[1]);
      gs = F64.gradient();
      P.S.grad_evals += 1;
      P.S.grad_ffts += 1;
      P.S.grad_ffts_fp64 += 1;
      end = newton_phase<double, TC>(F64, gs, o, P, false);
      if (F64.s[F64.cur] != s_out)
        check(cudaMemcpyAsync(s_out, F64.s[F64.cur], sizeof(double) * c->n3(),
                              cudaMemcpyDeviceToDevice, c->stream), "copy s");
    } else {
      convert<double, float>(c, F32.s[F32.cur], s_out);
    }
  } else {
    auto F64 = make_fields<double, TC>(c, N, w, nbar, jac, s64[0], s64[1]);
    BSums gs = F64.gradient();
    P.S.grad_evals += 1;
    P.S.grad_ffts += 1;
    P.S.grad_ffts_fp64 += 1;
    P.g0 = o.g0_norm > 0.0 ? o.g0_norm : std::sqrt(gs.gg);
    P.S.g0_norm = P.g0;
    end = newton_phase<double, TC>(F64, gs, o, P, false);
    if (F64.s[F64.cur] != s_out)
      check(cudaMemcpyAsync(s_out, F64.s[F64.cur], sizeof(double) * c->n3(),
                            cudaMemcpyDeviceToDevice, c->stream), "copy s");
  }
  check(cudaStreamSynchronize(c->stream), "stream synchronize");
  P.S.newton_iters = P.it;
  P.S.kernels = launches(c) - k0;
  P.S.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = P.S;
  return end_status(end);
}

template plc_status bias_map<double>(plc_ctx*, const int32_t*, const double*, double, double*,
                                     const plc_opts&, plc_stats*);
template plc_status bias_map<float>(plc_ctx*, const int32_t*, const double*, double, double*,
                                    const plc_opts&, plc_stats*);

}  // namespace plc
