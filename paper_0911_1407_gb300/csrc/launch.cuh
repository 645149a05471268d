// launch.cuh -- host launchers for the spectral pipeline and element-wise
// kernels.  Included by the per-type translation units, which instantiate
// the templates for their field types.
#pragma once

#include "ctx.h"
#include "ops.cuh"
#include <type_traits>

#include "passes.cuh"
#include "passes4.cuh"

namespace plc {

template <typename T> inline const cpx<T>* twiddles(const plc_ctx* c);
template <> inline const cpx<float>* twiddles<float>(const plc_ctx* c) { return c->tw32; }
template <> inline const cpx<double>* twiddles<double>(const plc_ctx* c) { return c->tw64; }
template <typename T> inline const T* multiplier(const plc_ctx* c);
template <> inline const float* multiplier<float>(const plc_ctx* c) { return c->M32; }
template <> inline const double* multiplier<double>(const plc_ctx* c) { return c->M64; }

// Raise a kernel's dynamic shared-memory limit to what the largest grid
// (n = 512) needs, once per kernel instantiation.
template <typename T, auto Kernel> inline void set_smem() {
  static const cudaError_t once = cudaFuncSetAttribute(
      Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassGeom<T>::smem_bytes_max(512));
  check(once, "cudaFuncSetAttribute");
}

inline RedArgs red_args(plc_ctx* c) { return RedArgs{c->partials, c->sc}; }

// Raise a kernel's dynamic shared-memory limit once (when above 48 KB).
template <auto Kernel> inline void set_smem4(size_t bytes) {
  if (bytes <= 48 * 1024) return;
  static const cudaError_t once =
      cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  check(once, "cudaFuncSetAttribute");
}

// The passes with register four-step line transforms (passes4.cuh) in
// transform arithmetic T: float (FP32 twiddles and multipliers) or ff
// (float-float, from the FP64 tables).
template <typename T, int N1, int N2, typename Pro, typename Epi, typename Fin>
void run_pipeline4(plc_ctx* c, Pro pro, Epi epi, Fin fin, int zero_dc, const int* done, int s0,
                   const void* m_override = nullptr) {
  using Gm = Geo4<T, N1, N2>;
  using C = cpx<T>;
  constexpr bool kFF = std::is_same<T, ff>::value;
  using TM = typename std::conditional<kFF, double, float>::type;
  constexpr int n = Gm::N, h = n / 2 + 1;
  C* A = static_cast<C*>(c->specA);
  C* B = static_cast<C*>(c->specB);
  const C* tw = kFF ? static_cast<const C*>(c->twff) : reinterpret_cast<const C*>(c->tw32);
  const TM* M = m_override ? static_cast<const TM*>(m_override)
                           : kFF ? reinterpret_cast<const TM*>(c->M64)
                                 : reinterpret_cast<const TM*>(c->M32);
  const dim3 gx(n / Gm::RY, n), gy(n / Gm::L, h);
  set_smem4<k4_xf<T, N1, N2, Pro>>(Gm::smem_x);
  set_smem4<k4_yf<T, N1, N2>>(Gm::smem_y);
  set_smem4<k4_z<T, N1, N2, TM>>(Gm::smem_z);
  set_smem4<k4_yi<T, N1, N2>>(Gm::smem_y);
  set_smem4<k4_xi<T, N1, N2, Epi, Fin>>(Gm::smem_x);
  {
    LaunchScope ls(c, Site(s0 + 0));
    k4_xf<T, N1, N2, Pro><<<gx, kThreads, Gm::smem_x, c->stream>>>(pro, A, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 1));
    k4_yf<T, N1, N2><<<gy, kThreads, Gm::smem_y, c->stream>>>(A, B, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 2));
    k4_z<T, N1, N2, TM><<<gy, kThreads, Gm::smem_z, c->stream>>>(B, M, zero_dc, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 3));
    k4_yi<T, N1, N2><<<gy, kThreads, Gm::smem_y, c->stream>>>(B, A, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 4));
    k4_xi<T, N1, N2, Epi, Fin><<<gx, kThreads, Gm::smem_x, c->stream>>>(A, epi, fin, red_args(c),
                                                                        tw, done);
  }
  check(cudaGetLastError(), "spectral pipeline launch");
}

// Dispatch on the context's four-step schedule (every entry of kFourStep,
// ctx.h); false when the plan has none (Stockham stages).
template <typename T, typename Pro, typename Epi, typename Fin>
bool run_four_step(plc_ctx* c, Pro pro, Epi epi, Fin fin, int zero_dc, const int* done, int s0,
                   const void* m_override = nullptr) {
  switch (c->plan.f1 * 64 + c->plan.f2) {
    case 16 * 64 + 16: run_pipeline4<T, 16, 16>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 16 * 64 + 12: run_pipeline4<T, 16, 12>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 12 * 64 + 16: run_pipeline4<T, 12, 16>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 16 * 64 + 8: run_pipeline4<T, 16, 8>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 8 * 64 + 16: run_pipeline4<T, 8, 16>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 12 * 64 + 8: run_pipeline4<T, 12, 8>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 8 * 64 + 12: run_pipeline4<T, 8, 12>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 8 * 64 + 8: run_pipeline4<T, 8, 8>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    case 8 * 64 + 4: run_pipeline4<T, 8, 4>(c, pro, epi, fin, zero_dc, done, s0, m_override); return true;
    default: return false;
  }
}

// The five passes XF -> YF -> Z -> YI -> XI on the context's stream.
template <typename T, typename Pro, typename Epi, typename Fin>
void run_pipeline(plc_ctx* c, Pro pro, Epi epi, Fin fin, int zero_dc, const int* done,
                  int sites = 0, const T* m_override = nullptr) {
  using G = PassGeom<T>;
  // site group: 0 the Hessian-vector product and public operators, 1 the
  // Newton gradient, 2 the linear-bias model
  constexpr bool k64 = sizeof(T) == 8;
  const int s0 = sites == 2   ? (k64 ? S_BXF64 : S_BXF32)
                 : sites == 1 ? (k64 ? S_GXF64 : S_GXF32)
                              : (k64 ? S_XF64 : S_XF32);
  if constexpr (sizeof(T) == 4) {
    if (run_four_step<float>(c, pro, epi, fin, zero_dc, done, s0, m_override)) return;
  }
  const int n = c->n, h = n / 2 + 1;
  const size_t sm = G::smem_bytes(c->plan);
  cpx<T>* A = static_cast<cpx<T>*>(c->specA);
  cpx<T>* B = static_cast<cpx<T>*>(c->specB);
  const cpx<T>* tw = twiddles<T>(c);
  const dim3 gx((n + G::RY - 1) / G::RY, n), gy((n + G::L - 1) / G::L, h);
  set_smem<T, k_xf<T, Pro>>();
  set_smem<T, k_yf<T>>();
  set_smem<T, k_z<T>>();
  set_smem<T, k_yi<T>>();
  set_smem<T, k_xi<T, Epi, Fin>>();
  {
    LaunchScope ls(c, Site(s0 + 0));
    k_xf<T, Pro><<<gx, kThreads, sm, c->stream>>>(pro, A, c->plan, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 1));
    k_yf<T><<<gy, kThreads, sm, c->stream>>>(A, B, c->plan, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 2));
    k_z<T><<<gy, kThreads, sm, c->stream>>>(B, m_override ? m_override : multiplier<T>(c), zero_dc,
                                            c->plan, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 3));
    k_yi<T><<<gy, kThreads, sm, c->stream>>>(B, A, c->plan, tw, done);
  }
  {
    LaunchScope ls(c, Site(s0 + 4));
    k_xi<T, Epi, Fin><<<gx, kThreads, sm, c->stream>>>(A, epi, fin, red_args(c), c->plan, tw, done);
  }
  check(cudaGetLastError(), "spectral pipeline launch");
}

template <typename T> void prior_apply(plc_ctx* c, const T* x, T* y) {
  run_pipeline<T>(c, ProLoad<T>{x}, EpiStore<T>{y}, FinNone{}, 0, nullptr);
}

template <typename T> void hessvec_s(plc_ctx* c, const T* s, const T* w, double nbar,
                                     const T* v, T* out) {
  run_pipeline<T>(c, ProLoad<T>{v}, EpiHessS<T>{s, w, (T)nbar, v, out}, FinNone{}, 0, nullptr);
}

template <typename T> void grad_public(plc_ctx* c, const T* s, const T* w, const int32_t* N,
                                       double nbar, T* g) {
  run_pipeline<T>(c, ProShift<T, T>{s, c->mu},
                  EpiGrad<T, T, T, T>{s, w, N, nbar, c->mu, nullptr, g, nullptr, nullptr,
                                      c->jac_c, 0},
                  FinStore<6>{}, 0, nullptr, true);
}

template <typename T, typename TS, typename TC>
void grad_newton(plc_ctx* c, const TS* s, const double* w, const int32_t* N, double nbar, T* y,
                 T* g, TC* D, TC* r, bool jac) {
  if constexpr (std::is_same<T, double>::value && std::is_same<TC, float>::value) {
    // the FP64 gradient of the mixed solve: float-float transforms and
    // epilogue where the length has a four-step schedule
    const EpiGradFF<true> epi{s, w, N, ff(nbar), ff(c->mu), y, g, D, r, (float)c->jac_c,
                              jac ? 1 : 0, static_cast<const ff*>(c->expff)};
    if (run_four_step<ff>(c, ProShiftFF{s, ff(c->mu)}, epi, FinGrad{}, 0, nullptr, S_GXFF)) return;
  }
  run_pipeline<T>(c, ProShift<T, TS>{s, c->mu},
                  EpiGrad<T, TS, double, TC>{s, w, N, nbar, c->mu, y, g, D, r, c->jac_c,
                                             jac ? 1 : 0},
                  FinGrad{}, 0, nullptr, true);
}

// The sums of the FP64 gradient of the mixed solve at an FP64 s (the
// float-float pipeline with nothing stored: -ln P, ||g||^2 and the scale of
// the rounding test into sc->red, FinGrad), for a stopping test that may end
// the solve before the gradient's fields are needed.  False (nothing run)
// when the length has no four-step schedule.
inline bool grad_sums_ff_impl(plc_ctx* c, const double* s, const double* w, const int32_t* N,
                              double nbar, bool jac) {
  const EpiGradFF<false> epi{s, w, N, ff(nbar), ff(c->mu), nullptr, nullptr, nullptr, nullptr,
                             (float)c->jac_c, jac ? 1 : 0, static_cast<const ff*>(c->expff)};
  return run_four_step<ff>(c, ProShiftFF{s, ff(c->mu)}, epi, FinGrad{}, 0, nullptr, S_GXFF);
}

template <typename T, typename TS, typename TC>
void grad_newton_g(plc_ctx* c, const TS* delta, const double* w, const int32_t* N, double nbar,
                   T* y, T* g, TC* D, TC* r, bool jac) {
  run_pipeline<T>(c, ProShift<T, TS>{delta, 0.0},
                  EpiGradG<T, TS, TC>{delta, w, N, nbar, y, g, D, r, c->jac_c, jac ? 1 : 0},
                  FinGrad{}, 0, nullptr, true);
}

template <typename T> void cg_hv(plc_ctx* c, const T* r, const T* D, T* p, T* Hp, bool jac) {
  const int* done = &c->sc->done;
  if (jac)
    run_pipeline<T>(c, ProCgDir<T, true>{r, D, (T)c->jac_c, p, c->sc},
                    EpiHessD<T>{D, p, Hp}, FinAlpha{}, 0, done);
  else
    run_pipeline<T>(c, ProCgDir<T, false>{r, D, (T)c->jac_c, p, c->sc},
                    EpiHessD<T>{D, p, Hp}, FinAlpha{}, 0, done);
}

template <typename TL> void vjp_amplitude(plc_ctx* c, const double* s, const TL* lam) {
  run_pipeline<double>(c, ProShift<double, double>{s, c->mu}, EpiDot<double, TL>{lam},
                       FinStore<1>{}, 1, nullptr);
}

inline int pw_blocks(plc_ctx* c) { return pointwise_blocks((long long)c->n3(), c->sms); }

template <typename T, typename TC>
void newton_update_g(plc_ctx* c, const T* s, const T* y, const T* g, const TC* r, const TC* xi,
                     const TC* D, const int32_t* N, const double* w, double nbar, double tau,
                     bool jac, T* s2, T* y2, T* g2, TC* D2, TC* r2) {
  LaunchScope ls(c, sizeof(T) == 4 ? S_NEWTON_UPDATE32 : S_NEWTON_UPDATE64);
  k_newton_update_g<T, TC><<<pw_blocks(c), kThreads, 0, c->stream>>>(
      s, y, g, r, xi, D, N, w, nbar, tau, c->jac_c, jac ? 1 : 0, s2, y2, g2, D2, r2, c->n3(),
      red_args(c));
  check(cudaGetLastError(), "k_newton_update_g");
}

template <typename T, typename TC>
void boundary_step(plc_ctx* c, const T* delta, const TC* xi, const int32_t* N) {
  LaunchScope ls(c, S_BOUNDARY);
  k_boundary<T, TC><<<pw_blocks(c), kThreads, 0, c->stream>>>(delta, xi, N, c->n3(), red_args(c));
  check(cudaGetLastError(), "k_boundary");
}


template <typename TC> void cg_init(plc_ctx* c, const double* b, const TC* D, TC* r, bool jac) {
  const int nb = pw_blocks(c);
  LaunchScope ls(c, S_CG_INIT);
  if (jac)
    k_cg_init<TC, double, true><<<nb, kThreads, 0, c->stream>>>(b, D, (TC)c->jac_c, r, c->n3(),
                                                                 red_args(c));
  else
    k_cg_init<TC, double, false><<<nb, kThreads, 0, c->stream>>>(b, D, (TC)c->jac_c, r, c->n3(),
                                                                  red_args(c));
  check(cudaGetLastError(), "k_cg_init");
}

template <typename TC> void lsq_init(plc_ctx* c, const int32_t* N, const double* w, double nbar,
                                     TC* D, TC* r, bool jac) {
  const int nb = pw_blocks(c);
  LaunchScope ls(c, S_CG_INIT);
  if (jac)
    k_lsq_init<TC, true><<<nb, kThreads, 0, c->stream>>>(N, w, nbar, (TC)c->jac_c, D, r,
                                                         c->n3(), red_args(c));
  else
    k_lsq_init<TC, false><<<nb, kThreads, 0, c->stream>>>(N, w, nbar, (TC)c->jac_c, D, r,
                                                          c->n3(), red_args(c));
  check(cudaGetLastError(), "k_lsq_init");
}

template <typename TC> void cg_update(plc_ctx* c, TC* x, TC* r, const TC* p, const TC* Hp,
                                      const TC* D, bool jac, double rtol2, int max_iter) {
  // one wave (4 blocks of 256 per SM at its 56 registers): 73.8 us against
  // 77.1 with two waves at 256^3
  const int nb = pointwise_blocks((long long)c->n3(), c->sms, 4);
  LaunchScope ls(c, sizeof(TC) == 4 ? S_CG_UPDATE32 : S_CG_UPDATE64);
  if (jac)
    k_cg_update<TC, true><<<nb, kThreads, 0, c->stream>>>(x, r, p, Hp, D, (TC)c->jac_c, c->n3(),
                                                           red_args(c), rtol2, max_iter);
  else
    k_cg_update<TC, false><<<nb, kThreads, 0, c->stream>>>(x, r, p, Hp, D, (TC)c->jac_c, c->n3(),
                                                            red_args(c), rtol2, max_iter);
  check(cudaGetLastError(), "k_cg_update");
}

template <typename T, typename TC>
void newton_update(plc_ctx* c, const T* s, const T* y, const T* g, const TC* r, const TC* xi,
                   const TC* D, const int32_t* N, const double* w, double nbar, double tau,
                   bool jac, T* s2, T* y2, T* g2, TC* D2, TC* r2, const double* tau_dev) {
  // g may be left out only where forming it again from y, D and N is exact
  if (!g && !std::is_same<T, TC>::value) check(cudaErrorInvalidValue, "newton_update without g");
  LaunchScope ls(c, sizeof(T) == 4 ? S_NEWTON_UPDATE32 : S_NEWTON_UPDATE64);
  k_newton_update<T, TC><<<pw_blocks(c), kThreads, 0, c->stream>>>(
      s, y, g, r, xi, D, N, w, nbar, c->mu, tau, tau_dev, c->jac_c, jac ? 1 : 0, s2, y2, g2, D2, r2,
      c->n3(), red_args(c));
  check(cudaGetLastError(), "k_newton_update");
}

template <typename TS> void diag_start(plc_ctx* c, TS* s, const int32_t* N, const double* w,
                                       double nbar) {
  LaunchScope ls(c, S_SETUP);
  k_diag_start<TS><<<pw_blocks(c), kThreads, 0, c->stream>>>(
      s, N, w, (float)nbar, (float)c->mu, (float)c->prior_var, c->n3());
  check(cudaGetLastError(), "k_diag_start");
}

template <typename TS> void diag_start_g(plc_ctx* c, TS* delta, const int32_t* N, const double* w,
                                         double nbar) {
  LaunchScope ls(c, S_SETUP);
  k_diag_start_g<TS><<<pw_blocks(c), kThreads, 0, c->stream>>>(delta, N, w, (float)nbar,
                                                              (float)c->prior_var, c->n3());
  check(cudaGetLastError(), "k_diag_start_g");
}

template <typename TC> void diag(plc_ctx* c, const double* s, const double* w, double nbar, TC* D) {
  LaunchScope ls(c, S_DIAG);
  k_diag<TC><<<pw_blocks(c), kThreads, 0, c->stream>>>(s, w, nbar, D, c->n3());
  check(cudaGetLastError(), "k_diag");
}

template <typename TD, typename TS> void convert(plc_ctx* c, const TS* src, TD* dst) {
  LaunchScope ls(c, S_CONVERT);
  k_convert<TD, TS><<<pw_blocks(c), kThreads, 0, c->stream>>>(src, dst, c->n3());
  check(cudaGetLastError(), "k_convert");
}

}  // namespace plc
