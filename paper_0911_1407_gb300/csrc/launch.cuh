// launch.cuh -- host launchers for the spectral pipeline and element-wise
// kernels.  Included by the per-type translation units, which instantiate
// the templates for their field types.
#pragma once

#include "ctx.h"
#include "ops.cuh"
#include "passes.cuh"

namespace plc {

template <typename T> inline const cpx<T>* twiddles(const plc_ctx* c);
template <> inline const cpx<float>* twiddles<float>(const plc_ctx* c) { return c->tw32; }
template <> inline const cpx<double>* twiddles<double>(const plc_ctx* c) { return c->tw64; }
template <typename T> inline const T* multiplier(const plc_ctx* c);
template <> inline const float* multiplier<float>(const plc_ctx* c) { return c->M32; }
template <> inline const double* multiplier<double>(const plc_ctx* c) { return c->M64; }

template <typename K> inline void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
          "cudaFuncSetAttribute");
}

inline RedArgs red_args(plc_ctx* c) { return RedArgs{c->partials, c->sc}; }

// The five passes XF -> YF -> Z -> YI -> XI on the context's stream.
template <typename T, typename Pro, typename Epi, typename Fin>
void run_pipeline(plc_ctx* c, Pro pro, Epi epi, Fin fin, int zero_dc, const int* done) {
  using G = PassGeom<T>;
  const int n = c->n, h = n / 2 + 1;
  const size_t sm = G::smem_bytes(n);
  cpx<T>* A = static_cast<cpx<T>*>(c->specA);
  cpx<T>* B = static_cast<cpx<T>*>(c->specB);
  const cpx<T>* tw = twiddles<T>(c);
  const dim3 gx((n + G::RY - 1) / G::RY, n), gy((n + G::L - 1) / G::L, h);
  const int s0 = sizeof(T) == 8 ? S_XF64 : S_XF32;
  set_smem(k_xf<T, Pro>, sm);
  set_smem(k_yf<T>, sm);
  set_smem(k_z<T>, sm);
  set_smem(k_yi<T>, sm);
  set_smem(k_xi<T, Epi, Fin>, sm);
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
    k_z<T><<<gy, kThreads, sm, c->stream>>>(B, multiplier<T>(c), zero_dc, c->plan, tw, done);
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

template <typename T> void grad(plc_ctx* c, const T* s, const T* w, const int32_t* N,
                                double nbar, T* g, T* D, float* D32) {
  run_pipeline<T>(c, ProShift<T>{s, (T)c->mu},
                  EpiGrad<T>{s, w, N, (T)nbar, (T)c->mu, g, D, D32}, FinStore<5>{}, 0, nullptr);
}

template <typename T, typename TX> void grad_step(plc_ctx* c, T* s, const TX* xi, double tau,
                                                  const T* w, const int32_t* N, double nbar,
                                                  T* g, T* D, float* D32) {
  run_pipeline<T>(c, ProStepShift<T, TX>{s, xi, tau, (T)c->mu},
                  EpiGrad<T>{s, w, N, (T)nbar, (T)c->mu, g, D, D32}, FinStore<5>{}, 0, nullptr);
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
  run_pipeline<double>(c, ProShift<double>{s, c->mu}, EpiDot<double, TL>{lam}, FinStore<1>{},
                       1, nullptr);
}

inline int pw_blocks(plc_ctx* c) { return pointwise_blocks((long long)c->n3(), c->sms); }

template <typename TC, typename TB> void cg_init(plc_ctx* c, const TB* b, bool negate,
                                                 const TC* D, TC* r, TC* x, double rtol2,
                                                 int max_iter, bool jac) {
  const int nb = pw_blocks(c);
  LaunchScope ls(c, S_CG_INIT);
  if (jac)
    k_cg_init<TC, TB, true><<<nb, kThreads, 0, c->stream>>>(b, negate, D, (TC)c->jac_c, r, x,
                                                             c->n3(), red_args(c), rtol2, max_iter);
  else
    k_cg_init<TC, TB, false><<<nb, kThreads, 0, c->stream>>>(b, negate, D, (TC)c->jac_c, r, x,
                                                              c->n3(), red_args(c), rtol2, max_iter);
  check(cudaGetLastError(), "k_cg_init");
}

template <typename TC> void cg_update(plc_ctx* c, TC* x, TC* r, const TC* p, const TC* Hp,
                                      const TC* D, bool jac) {
  const int nb = pw_blocks(c);
  LaunchScope ls(c, S_CG_UPDATE);
  if (jac)
    k_cg_update<TC, true><<<nb, kThreads, 0, c->stream>>>(x, r, p, Hp, D, (TC)c->jac_c, c->n3(),
                                                           red_args(c));
  else
    k_cg_update<TC, false><<<nb, kThreads, 0, c->stream>>>(x, r, p, Hp, D, (TC)c->jac_c, c->n3(),
                                                            red_args(c));
  check(cudaGetLastError(), "k_cg_update");
}

template <typename TC, typename TG> void dirstats(plc_ctx* c, const TC* xi, const TG* g,
                                                  const TC* r, const TG* D, const int32_t* N) {
  LaunchScope ls(c, S_DIRSTATS);
  k_dirstats<TC, TG><<<pw_blocks(c), kThreads, 0, c->stream>>>(xi, g, r, D, N, c->n3(),
                                                                red_args(c));
  check(cudaGetLastError(), "k_dirstats");
}

template <typename TC, typename TG> void trial(plc_ctx* c, const TC* xi, const TG* D, double tau) {
  LaunchScope ls(c, S_TRIAL);
  k_trial<TC, TG><<<pw_blocks(c), kThreads, 0, c->stream>>>(xi, D, tau, c->n3(), red_args(c));
  check(cudaGetLastError(), "k_trial");
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
