// capi.cu -- the extern "C" boundary of libplc (declared in include/plc.h).
//
// Validates every argument before anything is launched, owns the context's
// device scratch, and turns CUDA failures into status codes (no exception
// crosses the ABI).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "ctx.h"
#include "graph.h"
#include "bias.h"
#include "solver.h"

namespace {

thread_local std::string g_last_error;

plc_status fail(plc_ctx* c, plc_status st, const std::string& msg) {
  if (c) c->err = msg;
  g_last_error = msg;
  return st;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool valid_size(int n) {
  if (n < 4 || n > 512 || (n & 1)) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

// Radices for a length-n FFT: as many 8s as possible without leaving a lone
// 2 (then 4s), then the 3s.
plc::FftPlan make_plan(int n) {
  plc::FftPlan p{};
  p.n = n;
  int a = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  int b = 0;
  while (m % 3 == 0) { m /= 3; ++b; }
  std::vector<int> r;
  int q = a / 3, rem = a % 3;
  if (rem == 1 && q >= 1) { q -= 1; rem = 4; }
  for (int i = 0; i < q; ++i) r.push_back(8);
  if (rem == 1) r.push_back(2);
  if (rem == 2) r.push_back(4);
  if (rem == 4) { r.push_back(4); r.push_back(4); }
  for (int i = 0; i < b; ++i) r.push_back(3);
  p.nst = (int)r.size();
  int ns = 1;
  for (int i = 0; i < p.nst; ++i) {
    p.rad[i] = r[i];
    p.ns[i] = ns;
    p.tstep[i] = n / (ns * r[i]);
    p.ns_m[i] = ns > 1 ? plc::make_fastdiv(ns).m : 0u;
    ns *= r[i];
  }
  p.nd = plc::make_fastdiv(n);
  // FP32 transforms of these lengths use a register four-step schedule
  // n = f1 f2 (passes4.cuh); the first listed for n is the default
  p.f1 = p.f2 = 0;
  for (const plc::FourStepShape& q : plc::kFourStep)
    if (q.n == n) {
      p.f1 = q.f1;
      p.f2 = q.f2;
      break;
    }
  return p;
}

template <typename T> void dalloc(T** p, size_t bytes) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    throw std::bad_alloc();
  }
}

void release(plc_ctx* c) {
  plc::graph_release(c);
  plc::profile_release(c);
  void* ptrs[] = {c->specA, c->specB, c->tw64, c->tw32, c->twff, c->expff, c->M64, c->M32,
                  c->lk, c->lP, c->sc, c->partials, c->Mb64, c->Mb32, c->lkb, c->lbb, c->hist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : c->wf)
    if (p) cudaFree(p);
  for (void* p : c->bwf)
    if (p) cudaFree(p);
  if (c->sc_host) cudaFreeHost(c->sc_host);
}

void ensure_work_fields(plc_ctx* c) {
  const size_t b = sizeof(double) * c->n3();
  for (void*& p : c->wf)
    if (!p) dalloc(&p, b);
}

void ensure_bias_fields(plc_ctx* c) {
  ensure_work_fields(c);
  const size_t b = sizeof(double) * c->n3();
  for (void*& p : c->bwf)
    if (!p) dalloc(&p, b);
}

// Run `body`; map CUDA errors and allocation failures to status codes.
template <typename F> plc_status guarded(plc_ctx* c, F body) {
  try {
    return body();
  } catch (const plc::CudaError& e) {
    return fail(c, PLC_ERR_CUDA, std::string(e.where) + ": " + cudaGetErrorString(e.code));
  } catch (const std::bad_alloc&) {
    return fail(c, PLC_ERR_OOM, "device allocation failed");
  }
}

plc_status need_prior(plc_ctx* c) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  if (!c->have_prior) return fail(c, PLC_ERR_INVALID_ARG, "no prior: call plc_set_prior first");
  return PLC_OK;
}

plc_status need_field(plc_ctx* c, const void* p, const char* name, bool required) {
  if (!p) return required ? fail(c, PLC_ERR_INVALID_ARG, std::string(name) + " is NULL") : PLC_OK;
  if (!aligned16(p)) return fail(c, PLC_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
  return PLC_OK;
}

#define PLC_TRY(expr)                 \
  do {                                \
    plc_status _s = (expr);           \
    if (_s != PLC_OK) return _s;      \
  } while (0)

plc_opts resolve_opts(const plc_opts* o) {
  plc_opts d;
  plc_default_opts(&d);
  return o ? *o : d;
}

plc_status check_opts(plc_ctx* c, const plc_opts& o) {
  if (!(o.tol > 0.0) || !std::isfinite(o.tol)) return fail(c, PLC_ERR_INVALID_ARG, "opts.tol must be > 0");
  if (o.max_newton < 0 || o.max_cg < 1) return fail(c, PLC_ERR_INVALID_ARG, "bad iteration caps");
  if (o.precond != 0 && o.precond != 1) return fail(c, PLC_ERR_INVALID_ARG, "opts.precond must be 0 or 1");
  if (!(o.step_cap > 0.0) || !(o.eta_max > 0.0) || o.eta_max >= 1.0 || o.g0_norm < 0.0)
    return fail(c, PLC_ERR_INVALID_ARG, "bad step_cap / eta_max / g0_norm");
  if (o.cg_chunk < 1) return fail(c, PLC_ERR_INVALID_ARG, "opts.cg_chunk must be >= 1");
  if (!(o.mixed_switch >= 0.0)) return fail(c, PLC_ERR_INVALID_ARG, "opts.mixed_switch must be >= 0");
  if (o.device_driven != 0 && o.device_driven != 1)
    return fail(c, PLC_ERR_INVALID_ARG, "opts.device_driven must be 0 or 1");
  if (o.start < 0 || o.start > 2) return fail(c, PLC_ERR_INVALID_ARG, "opts.start must be 0, 1 or 2");
  return PLC_OK;
}

}  // namespace

namespace plc {
// Records a failure that has no context (read back by plc_last_error(NULL)).
void set_global_error(const std::string& msg) { g_last_error = msg; }
}  // namespace plc

extern "C" {

const char* plc_status_string(int s) {
  switch (s) {
    case PLC_OK: return "PLC_OK";
    case PLC_ERR_INVALID_ARG: return "PLC_ERR_INVALID_ARG";
    case PLC_ERR_CUDA: return "PLC_ERR_CUDA";
    case PLC_ERR_NOT_CONVERGED: return "PLC_ERR_NOT_CONVERGED";
    case PLC_ERR_NONFINITE: return "PLC_ERR_NONFINITE";
    case PLC_ERR_CG_BREAKDOWN: return "PLC_ERR_CG_BREAKDOWN";
    case PLC_ERR_OOM: return "PLC_ERR_OOM";
    default: return "PLC_ERR_UNKNOWN";
  }
}

const char* plc_last_error(const plc_ctx* c) { return c ? c->err.c_str() : g_last_error.c_str(); }

plc_status plc_default_opts(plc_opts* o) {
  if (!o) return fail(nullptr, PLC_ERR_INVALID_ARG, "opts is NULL");
  o->tol = 1e-6;
  o->max_newton = 200;
  o->max_cg = 1000;
  o->precond = 1;
  o->g0_norm = 0.0;
  o->step_cap = 2.0;
  o->eta_max = 0.5;
  o->cg_chunk = 8;
  o->mixed_switch = 1e-6;
  o->device_driven = 1;
  o->start = 1;
  return PLC_OK;
}

plc_status plc_create(plc_ctx** out, int n, double box, int precision, void* stream) {
  if (!out) return fail(nullptr, PLC_ERR_INVALID_ARG, "ctx out-pointer is NULL");
  *out = nullptr;
  if (!valid_size(n))
    return fail(nullptr, PLC_ERR_INVALID_ARG, "n must be even, 4..512, with prime factors 2 and 3 only");
  if (!(box > 0.0) || !std::isfinite(box)) return fail(nullptr, PLC_ERR_INVALID_ARG, "box must be > 0");
  if (precision != PLC_FP64 && precision != PLC_MIXED)
    return fail(nullptr, PLC_ERR_INVALID_ARG, "precision must be PLC_FP64 or PLC_MIXED");
  plc_ctx* c = new (std::nothrow) plc_ctx();
  if (!c) return fail(nullptr, PLC_ERR_OOM, "host allocation failed");
  c->n = n;
  c->box = box;
  c->precision = precision;
  c->stream = static_cast<cudaStream_t>(stream);
  c->plan = make_plan(n);
  plc_status st = guarded(c, [&]() -> plc_status {
    int dev = 0;
    plc::check(cudaGetDevice(&dev), "cudaGetDevice");
    plc::check(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const size_t h = n / 2 + 1;
    const size_t spec = sizeof(double2) * h * n * n;
    dalloc(&c->specA, spec);
    dalloc(&c->specB, spec);
    dalloc(&c->tw64, sizeof(double2) * n);
    dalloc(&c->tw32, sizeof(float2) * n);
    dalloc(&c->twff, sizeof(float4) * n);
    dalloc(&c->expff, sizeof(float2) * 64);
    dalloc(&c->sc, sizeof(plc::DevScalars));
    plc::check(cudaMallocHost(reinterpret_cast<void**>(&c->sc_host), sizeof(plc::DevScalars)),
               "cudaMallocHost");
    const size_t xi_blocks = (size_t)((n + 15) / 16) * n;
    c->partial_blocks = std::max(xi_blocks, (size_t)c->sms * 8);
    dalloc(&c->partials, sizeof(double) * plc::kMaxRed * c->partial_blocks);
    // twiddles W_n^m = exp(-2 pi i m / n), from the FP64 host sin/cos
    std::vector<double2> t64(n);
    std::vector<float2> t32(n);
    std::vector<float4> tff(n);   // float-float: (re hi, re lo, im hi, im lo)
    for (int m = 0; m < n; ++m) {
      const double ang = 2.0 * M_PI * (double)m / (double)n;
      t64[m] = make_double2(std::cos(ang), -std::sin(ang));
      t32[m] = make_float2((float)t64[m].x, (float)t64[m].y);
      tff[m] = make_float4(t32[m].x, (float)(t64[m].x - (double)t32[m].x), t32[m].y,
                           (float)(t64[m].y - (double)t32[m].y));
    }
    plc::check(cudaMemcpyAsync(c->tw64, t64.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, c->stream), "copy twiddles");
    plc::check(cudaMemcpyAsync(c->tw32, t32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, c->stream), "copy twiddles");
    plc::check(cudaMemcpyAsync(c->twff, tff.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, c->stream), "copy twiddles");
    // 2^(j/64), j < 64, in float-float (the table of the float-float exp)
    std::vector<float2> e2(64);
    for (int j = 0; j < 64; ++j) {
      const double v = std::exp2((double)j / 64.0);
      e2[j] = make_float2((float)v, (float)(v - (double)(float)v));
    }
    plc::check(cudaMemcpyAsync(c->expff, e2.data(), sizeof(float2) * 64, cudaMemcpyHostToDevice, c->stream), "copy exp table");
    plc::check(cudaMemsetAsync(c->sc, 0, sizeof(plc::DevScalars), c->stream), "clear scalars");
    plc::check(cudaStreamSynchronize(c->stream), "stream synchronize");
    return PLC_OK;
  });
  if (st != PLC_OK) {
    g_last_error = c->err;
    release(c);
    delete c;
    return st;
  }
  *out = c;
  return PLC_OK;
}

plc_status plc_destroy(plc_ctx* c) {
  if (!c) return PLC_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  release(c);
  delete c;
  return PLC_OK;
}

plc_status plc_set_prior(plc_ctx* c, const double* k, const double* P, int nk, double mu,
                         double inv_lambda_dc) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  if (!k || !P || nk < 2) return fail(c, PLC_ERR_INVALID_ARG, "need k, P arrays with nk >= 2");
  for (int i = 0; i < nk; ++i) {
    if (!(k[i] > 0.0) || !std::isfinite(k[i]) || !(P[i] > 0.0) || !std::isfinite(P[i]))
      return fail(c, PLC_ERR_INVALID_ARG, "k and P must be finite and > 0");
    if (i && !(k[i] > k[i - 1])) return fail(c, PLC_ERR_INVALID_ARG, "k must be strictly ascending");
  }
  const double kf = 2.0 * M_PI / c->box;
  const double kmax = std::sqrt(3.0) * M_PI * c->n / c->box;
  if (k[0] > kf * (1.0 + 1e-12) || k[nk - 1] < kmax * (1.0 - 1e-12))
    return fail(c, PLC_ERR_INVALID_ARG, "P(k) table must cover [2 pi / L, sqrt(3) pi n / L]");
  if (!std::isfinite(mu)) return fail(c, PLC_ERR_INVALID_ARG, "mu must be finite");
  if (!(inv_lambda_dc >= 0.0) || !std::isfinite(inv_lambda_dc))
    return fail(c, PLC_ERR_INVALID_ARG, "inv_lambda_dc must be finite and >= 0");
  return guarded(c, [&]() -> plc_status {
    const int half = c->n / 2;
    const int nm2 = 3 * half * half + 1;
    if (c->nm2 != nm2) {
      if (c->M64) cudaFree(c->M64);
      if (c->M32) cudaFree(c->M32);
      c->M64 = nullptr;
      c->M32 = nullptr;
      dalloc(&c->M64, sizeof(double) * nm2);
      dalloc(&c->M32, sizeof(float) * nm2);
      c->nm2 = nm2;
    }
    if (c->nk_cap < nk) {
      if (c->lk) cudaFree(c->lk);
      if (c->lP) cudaFree(c->lP);
      c->lk = nullptr;
      c->lP = nullptr;
      dalloc(&c->lk, sizeof(double) * nk);
      dalloc(&c->lP, sizeof(double) * nk);
      c->nk_cap = nk;
    }
    std::vector<double> lk(nk), lP(nk);
    for (int i = 0; i < nk; ++i) {
      lk[i] = std::log(k[i]);
      lP[i] = std::log(P[i]);
    }
    c->mu = mu;
    c->inv_dc = inv_lambda_dc;
    c->have_prior = false;
    plc::build_prior(c, lk.data(), lP.data(), nk);
    c->have_prior = true;
    c->err.clear();
    return PLC_OK;
  });
}

plc_status plc_prior_apply(plc_ctx* c, const void* x, void* y) {
  PLC_TRY(need_prior(c));
  PLC_TRY(need_field(c, x, "x", true));
  PLC_TRY(need_field(c, y, "y", true));
  return guarded(c, [&]() -> plc_status {
    if (c->precision == PLC_FP64)
      plc::prior_apply<double>(c, static_cast<const double*>(x), static_cast<double*>(y));
    else
      plc::prior_apply<float>(c, static_cast<const float*>(x), static_cast<float*>(y));
    return PLC_OK;
  });
}

plc_status plc_logpost_grad(plc_ctx* c, const void* s, const int32_t* N, const void* w,
                            double nbar, double* neg_logpost, void* grad) {
  PLC_TRY(need_prior(c));
  PLC_TRY(need_field(c, s, "s", true));
  PLC_TRY(need_field(c, N, "N", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, grad, "grad", false));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  return guarded(c, [&]() -> plc_status {
    plc::reset_ticket(c);
    if (c->precision == PLC_FP64)
      plc::grad_public<double>(c, static_cast<const double*>(s), static_cast<const double*>(w), N,
                               nbar, static_cast<double*>(grad));
    else
      plc::grad_public<float>(c, static_cast<const float*>(s), static_cast<const float*>(w), N,
                              nbar, static_cast<float*>(grad));
    if (neg_logpost) {
      plc::read_scalars(c);
      const double* r = c->sc_host->red;
      *neg_logpost = 0.5 * r[0] + r[1];
      if (!std::isfinite(*neg_logpost)) return fail(c, PLC_ERR_NONFINITE, "non-finite -ln P");
    }
    return PLC_OK;
  });
}

plc_status plc_hessvec(plc_ctx* c, const void* s, const void* w, double nbar, const void* v,
                       void* Hv) {
  PLC_TRY(need_prior(c));
  PLC_TRY(need_field(c, s, "s", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, v, "v", true));
  PLC_TRY(need_field(c, Hv, "Hv", true));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  return guarded(c, [&]() -> plc_status {
    if (c->precision == PLC_FP64)
      plc::hessvec_s<double>(c, static_cast<const double*>(s), static_cast<const double*>(w), nbar,
                             static_cast<const double*>(v), static_cast<double*>(Hv));
    else
      plc::hessvec_s<float>(c, static_cast<const float*>(s), static_cast<const float*>(w), nbar,
                            static_cast<const float*>(v), static_cast<float*>(Hv));
    return PLC_OK;
  });
}

plc_status plc_newton_krylov_map(plc_ctx* c, const int32_t* N, const void* w, double nbar,
                                 double* s_inout, const plc_opts* opts, plc_stats* stats) {
  PLC_TRY(need_prior(c));
  PLC_TRY(need_field(c, N, "N", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, s_inout, "s_inout", true));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  const plc_opts o = resolve_opts(opts);
  PLC_TRY(check_opts(c, o));
  return guarded(c, [&]() -> plc_status {
    ensure_work_fields(c);
    plc_status st;
    const double* wd = static_cast<const double*>(w);
    if (o.device_driven)
      st = c->precision == PLC_FP64
               ? plc::newton_map_graph<double>(c, N, wd, nbar, s_inout, o, stats)
               : plc::newton_map_graph<float>(c, N, wd, nbar, s_inout, o, stats);
    else
      st = c->precision == PLC_FP64 ? plc::newton_map<double>(c, N, wd, nbar, s_inout, o, stats)
                                    : plc::newton_map<float>(c, N, wd, nbar, s_inout, o, stats);
    if (st == PLC_ERR_NOT_CONVERGED) fail(c, st, "Newton iteration cap reached");
    else if (st == PLC_ERR_NONFINITE) fail(c, st, "non-finite gradient or objective");
    else if (st == PLC_ERR_CG_BREAKDOWN) fail(c, st, "CG breakdown on the first step");
    else c->err.clear();
    return st;
  });
}

plc_status plc_gauss_map(plc_ctx* c, const int32_t* N, const void* w, double nbar,
                         double* delta_inout, const plc_opts* opts, plc_stats* stats) {
  PLC_TRY(need_prior(c));
  PLC_TRY(need_field(c, N, "N", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, delta_inout, "delta_inout", true));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  const plc_opts o = resolve_opts(opts);
  PLC_TRY(check_opts(c, o));
  return guarded(c, [&]() -> plc_status {
    ensure_work_fields(c);
    const double* wd = static_cast<const double*>(w);
    const plc_status st = c->precision == PLC_FP64
                              ? plc::gauss_map<double>(c, N, wd, nbar, delta_inout, o, stats)
                              : plc::gauss_map<float>(c, N, wd, nbar, delta_inout, o, stats);
    if (st == PLC_ERR_NOT_CONVERGED) fail(c, st, "Newton iteration cap reached");
    else if (st == PLC_ERR_NONFINITE) fail(c, st, "non-finite gradient or objective");
    else if (st == PLC_ERR_CG_BREAKDOWN) fail(c, st, "CG breakdown on the first step");
    else c->err.clear();
    return st;
  });
}

plc_status plc_wiener_lsq(plc_ctx* c, const int32_t* N, const void* w, double nbar,
                          double* delta_out, const plc_opts* opts, plc_stats* stats) {
  PLC_TRY(need_prior(c));
  PLC_TRY(need_field(c, N, "N", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, delta_out, "delta_out", true));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  const plc_opts o = resolve_opts(opts);
  PLC_TRY(check_opts(c, o));
  return guarded(c, [&]() -> plc_status {
    ensure_work_fields(c);
    const double* wd = static_cast<const double*>(w);
    const plc_status st = c->precision == PLC_FP64
                              ? plc::wiener_lsq<double>(c, N, wd, nbar, delta_out, o, stats)
                              : plc::wiener_lsq<float>(c, N, wd, nbar, delta_out, o, stats);
    if (st == PLC_ERR_NOT_CONVERGED) fail(c, st, "CG did not reach the tolerance");
    else if (st == PLC_ERR_CG_BREAKDOWN) fail(c, st, "CG breakdown on the first step");
    else c->err.clear();
    return st;
  });
}

// ------------------------------ linear bias --------------------------------

plc_status plc_set_bias(plc_ctx* c, const double* k, const double* b, int nb, double b_dc) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  if (!k || !b || nb < 2) return fail(c, PLC_ERR_INVALID_ARG, "need k, b arrays with nb >= 2");
  for (int i = 0; i < nb; ++i) {
    if (!(k[i] > 0.0) || !std::isfinite(k[i]) || !(b[i] > 0.0) || !std::isfinite(b[i]))
      return fail(c, PLC_ERR_INVALID_ARG, "k and b must be finite and > 0");
    if (i && !(k[i] > k[i - 1])) return fail(c, PLC_ERR_INVALID_ARG, "k must be strictly ascending");
  }
  const double kf = 2.0 * M_PI / c->box;
  const double kmax = std::sqrt(3.0) * M_PI * c->n / c->box;
  if (k[0] > kf * (1.0 + 1e-12) || k[nb - 1] < kmax * (1.0 - 1e-12))
    return fail(c, PLC_ERR_INVALID_ARG, "b(k) table must cover [2 pi / L, sqrt(3) pi n / L]");
  if (!(b_dc > 0.0) || !std::isfinite(b_dc))
    return fail(c, PLC_ERR_INVALID_ARG, "b_dc must be finite and > 0");
  return guarded(c, [&]() -> plc_status {
    const int half = c->n / 2;
    const int nm2 = 3 * half * half + 1;
    if (!c->Mb64) {
      dalloc(&c->Mb64, sizeof(double) * nm2);
      dalloc(&c->Mb32, sizeof(float) * nm2);
    }
    if (c->nb_cap < nb) {
      if (c->lkb) cudaFree(c->lkb);
      if (c->lbb) cudaFree(c->lbb);
      c->lkb = nullptr;
      c->lbb = nullptr;
      dalloc(&c->lkb, sizeof(double) * nb);
      dalloc(&c->lbb, sizeof(double) * nb);
      c->nb_cap = nb;
    }
    std::vector<double> lk(nb), lb(nb);
    for (int i = 0; i < nb; ++i) {
      lk[i] = std::log(k[i]);
      lb[i] = std::log(b[i]);
    }
    c->have_bias = false;
    plc::build_bias(c, lk.data(), lb.data(), nb, b_dc);
    c->have_bias = true;
    c->err.clear();
    return PLC_OK;
  });
}

static plc_status need_bias(plc_ctx* c) {
  PLC_TRY(need_prior(c));
  if (!c->have_bias) return fail(c, PLC_ERR_INVALID_ARG, "no bias table: call plc_set_bias first");
  return PLC_OK;
}

// y, q, Q at s (work fields of the bias solve) and the gradient; E, d1 on
// request.  T: the context's field type.
extern "C++" template <typename T>
void bias_point(plc_ctx* c, const T* s, const int32_t* N, const double* w, double nbar,
                T* grad, bool hess) {
  T* y = static_cast<T*>(c->bwf[2]);
  T* q = static_cast<T*>(c->bwf[4]);
  T* E = static_cast<T*>(c->bwf[6]);
  T* Q = static_cast<T*>(c->bwf[7]);
  T* d1 = static_cast<T*>(c->bwf[8]);
  plc::reset_ticket(c);
  plc::bias_prior<T, T>(c, s, c->mu, y);
  plc::bias_density<T, T>(c, s, nullptr, 0.0, nullptr, y, nullptr, nullptr, N, w, nbar, q, Q);
  plc::bias_gradient<T, T>(c, s, y, q, Q, grad, nullptr, hess ? E : nullptr, hess ? d1 : nullptr,
                           nullptr, false);
}

plc_status plc_bias_logpost_grad(plc_ctx* c, const void* s, const int32_t* N, const void* w,
                                 double nbar, double* neg_logpost, void* grad) {
  PLC_TRY(need_bias(c));
  PLC_TRY(need_field(c, s, "s", true));
  PLC_TRY(need_field(c, N, "N", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, grad, "grad", false));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  return guarded(c, [&]() -> plc_status {
    ensure_bias_fields(c);
    const double* wd = static_cast<const double*>(w);
    if (c->precision == PLC_FP64)
      bias_point<double>(c, static_cast<const double*>(s), N, wd, nbar, static_cast<double*>(grad),
                         false);
    else
      bias_point<float>(c, static_cast<const float*>(s), N, wd, nbar, static_cast<float*>(grad),
                        false);
    if (neg_logpost) {
      plc::read_scalars(c);
      const double* r = c->sc_host->red;
      *neg_logpost = 0.5 * r[0] + r[1];
      if (!std::isfinite(*neg_logpost))
        return fail(c, PLC_ERR_NONFINITE, "non-finite -ln P (u <= 0 where N > 0?)");
    }
    return PLC_OK;
  });
}

plc_status plc_bias_hessvec(plc_ctx* c, const void* s, const int32_t* N, const void* w,
                            double nbar, const void* v, void* Hv) {
  PLC_TRY(need_bias(c));
  PLC_TRY(need_field(c, s, "s", true));
  PLC_TRY(need_field(c, N, "N", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, v, "v", true));
  PLC_TRY(need_field(c, Hv, "Hv", true));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  return guarded(c, [&]() -> plc_status {
    ensure_bias_fields(c);
    const double* wd = static_cast<const double*>(w);
    void** B = c->bwf;
    if (c->precision == PLC_FP64) {
      using T = double;
      bias_point<T>(c, static_cast<const T*>(s), N, wd, nbar, nullptr, true);
      plc::bias_hv<T>(c, static_cast<const T*>(v), static_cast<T*>(B[6]), static_cast<T*>(B[7]),
                      static_cast<T*>(B[8]), static_cast<T*>(B[10]), static_cast<T*>(B[11]),
                      static_cast<T*>(Hv));
    } else {
      using T = float;
      bias_point<T>(c, static_cast<const T*>(s), N, wd, nbar, nullptr, true);
      plc::bias_hv<T>(c, static_cast<const T*>(v), static_cast<T*>(B[6]), static_cast<T*>(B[7]),
                      static_cast<T*>(B[8]), static_cast<T*>(B[10]), static_cast<T*>(B[11]),
                      static_cast<T*>(Hv));
    }
    return PLC_OK;
  });
}

plc_status plc_bias_map(plc_ctx* c, const int32_t* N, const void* w, double nbar,
                        double* s_inout, const plc_opts* opts, plc_stats* stats) {
  PLC_TRY(need_bias(c));
  PLC_TRY(need_field(c, N, "N", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, s_inout, "s_inout", true));
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  const plc_opts o = resolve_opts(opts);
  PLC_TRY(check_opts(c, o));
  return guarded(c, [&]() -> plc_status {
    ensure_bias_fields(c);
    const double* wd = static_cast<const double*>(w);
    const plc_status st = c->precision == PLC_FP64
                              ? plc::bias_map<double>(c, N, wd, nbar, s_inout, o, stats)
                              : plc::bias_map<float>(c, N, wd, nbar, s_inout, o, stats);
    if (st == PLC_ERR_NOT_CONVERGED) fail(c, st, "Newton iteration cap reached");
    else if (st == PLC_ERR_NONFINITE)
      fail(c, st, "non-finite gradient or objective (start point outside u > 0?)");
    else c->err.clear();
    return st;
  });
}

plc_status plc_map_vjp(plc_ctx* c, const double* s_map, const void* w, double nbar,
                       const double* u, double* vjp_N, double* vjp_lnA, const plc_opts* opts,
                       plc_stats* stats) {
  PLC_TRY(need_prior(c));
  PLC_TRY(need_field(c, s_map, "s_map", true));
  PLC_TRY(need_field(c, w, "w", false));
  PLC_TRY(need_field(c, u, "u", true));
  PLC_TRY(need_field(c, vjp_N, "vjp_N", false));
  if (!vjp_N && !vjp_lnA) return fail(c, PLC_ERR_INVALID_ARG, "no output requested");
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
  const plc_opts o = resolve_opts(opts);
  PLC_TRY(check_opts(c, o));
  return guarded(c, [&]() -> plc_status {
    ensure_work_fields(c);
    plc_status st;
    if (c->precision == PLC_FP64)
      st = plc::map_vjp<double>(c, s_map, static_cast<const double*>(w), nbar, u, vjp_N, vjp_lnA, o, stats);
    else
      st = plc::map_vjp<float>(c, s_map, static_cast<const double*>(w), nbar, u, vjp_N, vjp_lnA, o, stats);
    if (st != PLC_OK) fail(c, st, "adjoint CG did not reach the tolerance");
    else c->err.clear();
    return st;
  });
}

plc_status plc_compare(plc_ctx* c, const double* a, const double* b, double* r, double* d_euc) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  PLC_TRY(need_field(c, a, "a", true));
  PLC_TRY(need_field(c, b, "b", true));
  if (!r && !d_euc) return fail(c, PLC_ERR_INVALID_ARG, "no output requested");
  return guarded(c, [&]() -> plc_status {
    double t[4];
    plc::compare_fields(c, a, b, t);
    if (r) *r = (t[1] > 0.0 && t[2] > 0.0) ? t[0] / (std::sqrt(t[1]) * std::sqrt(t[2])) : 0.0;
    if (d_euc) *d_euc = std::sqrt(t[3] / (double)c->n3());
    return PLC_OK;
  });
}

plc_status plc_smooth(plc_ctx* c, const double* x, double* y, double radius) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  PLC_TRY(need_field(c, x, "x", true));
  PLC_TRY(need_field(c, y, "y", true));
  if (!(radius >= 0.0) || !std::isfinite(radius))
    return fail(c, PLC_ERR_INVALID_ARG, "radius must be finite and >= 0");
  return guarded(c, [&]() -> plc_status {
    ensure_work_fields(c);
    plc::gaussian_smooth(c, x, y, radius, static_cast<double*>(c->wf[12]));
    return PLC_OK;
  });
}

plc_status plc_log_stats(plc_ctx* c, const double* delta, double lo, double width, int nbins,
                         long long* counts, long long* outside, double* moments) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  PLC_TRY(need_field(c, delta, "delta", true));
  if (!(width > 0.0) || !std::isfinite(width) || !std::isfinite(lo))
    return fail(c, PLC_ERR_INVALID_ARG, "bins need finite lo and width > 0");
  if (nbins < 1 || nbins > plc_ctx::kMaxBins)
    return fail(c, PLC_ERR_INVALID_ARG, "nbins must be 1..4096");
  if (!counts || !outside || !moments) return fail(c, PLC_ERR_INVALID_ARG, "NULL output");
  return guarded(c, [&]() -> plc_status {
    // the counts have their own buffer: a work field holds only n^3 entries,
    // fewer than nbins + 3 on small grids
    if (!c->hist) dalloc(&c->hist, sizeof(unsigned long long) * (plc_ctx::kMaxBins + 3));
    std::vector<long long> all(nbins + 3);
    plc::log_stats(c, delta, lo, width, nbins, all.data(), moments, c->hist);
    for (int j = 0; j < nbins; ++j) counts[j] = all[j];
    for (int j = 0; j < 3; ++j) outside[j] = all[nbins + j];
    return PLC_OK;
  });
}

plc_status plc_set_fft_schedule(plc_ctx* c, int f1, int f2) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  bool ok = f1 == 0 && f2 == 0;
  for (const plc::FourStepShape& q : plc::kFourStep)
    if (q.n == c->n && q.f1 == f1 && q.f2 == f2) ok = true;
  if (!ok) return fail(c, PLC_ERR_INVALID_ARG, "no such FFT schedule for this grid size");
  c->plan.f1 = f1;
  c->plan.f2 = f2;
  return PLC_OK;
}

plc_status plc_autotune(plc_ctx* c, int reps, int* f1_out, int* f2_out, double* us_out) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  if (reps < 1 || reps > 1000) return fail(c, PLC_ERR_INVALID_ARG, "reps must be 1..1000");
  PLC_TRY(need_prior(c));
  return guarded(c, [&]() -> plc_status {
    double best_us = 0.0;
    if (c->precision == PLC_MIXED) {
      ensure_work_fields(c);
      float* s = static_cast<float*>(c->wf[0]);
      float* v = static_cast<float*>(c->wf[1]);
      float* out = static_cast<float*>(c->wf[2]);
      const size_t bytes = sizeof(float) * c->n3();
      plc::check(cudaMemsetAsync(s, 0, bytes, c->stream), "clear");
      plc::check(cudaMemsetAsync(v, 0, bytes, c->stream), "clear");
      std::vector<std::pair<int, int>> cand{{0, 0}};
      for (const plc::FourStepShape& q : plc::kFourStep)
        if (q.n == c->n) cand.emplace_back(q.f1, q.f2);
      cudaEvent_t e0, e1;
      plc::check(cudaEventCreate(&e0), "event");
      plc::check(cudaEventCreate(&e1), "event");
      std::pair<int, int> best{c->plan.f1, c->plan.f2};
      best_us = -1.0;
      try {
        for (const auto& f : cand) {
          c->plan.f1 = f.first;
          c->plan.f2 = f.second;
          plc::hessvec_s<float>(c, s, nullptr, 1.0, v, out);   // warm-up
          plc::check(cudaEventRecord(e0, c->stream), "event");
          for (int i = 0; i < reps; ++i) plc::hessvec_s<float>(c, s, nullptr, 1.0, v, out);
          plc::check(cudaEventRecord(e1, c->stream), "event");
          plc::check(cudaEventSynchronize(e1), "event");
          float ms = 0.f;
          plc::check(cudaEventElapsedTime(&ms, e0, e1), "event");
          const double us = 1e3 * ms / reps;
          if (best_us < 0.0 || us < best_us) {
            best_us = us;
            best = f;
          }
        }
      } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      c->plan.f1 = best.first;
      c->plan.f2 = best.second;
    }
    if (f1_out) *f1_out = c->plan.f1;
    if (f2_out) *f2_out = c->plan.f2;
    if (us_out) *us_out = best_us;
    return PLC_OK;
  });
}

struct plc_batch {
  std::vector<plc_ctx*> ctxs;
  plc::BatchGraph graph;
};

plc_status plc_batch_create(plc_batch** out, plc_ctx* const* ctxs, int count) {
  if (!out) return fail(nullptr, PLC_ERR_INVALID_ARG, "batch out-pointer is NULL");
  *out = nullptr;
  if (!ctxs || count < 1) return fail(nullptr, PLC_ERR_INVALID_ARG, "need count >= 1 contexts");
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return fail(nullptr, PLC_ERR_INVALID_ARG, "NULL context in batch");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(nullptr, PLC_ERR_INVALID_ARG, "context repeated in batch");
  }
  plc_batch* b = new (std::nothrow) plc_batch();
  if (!b) return fail(nullptr, PLC_ERR_OOM, "host allocation failed");
  b->ctxs.assign(ctxs, ctxs + count);
  *out = b;
  return PLC_OK;
}

plc_status plc_batch_map(plc_batch* b, const int32_t* const* N, const double* const* w,
                         const double* nbar, double* const* s_inout, const plc_opts* opts,
                         plc_stats* stats, void* stream) {
  if (!b) return fail(nullptr, PLC_ERR_INVALID_ARG, "batch is NULL");
  if (!N || !nbar || !s_inout) return fail(nullptr, PLC_ERR_INVALID_ARG, "NULL array argument");
  const plc_opts o = resolve_opts(opts);
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    plc_ctx* c = b->ctxs[i];
    PLC_TRY(need_prior(c));
    PLC_TRY(need_field(c, N[i], "N", true));
    PLC_TRY(need_field(c, w ? w[i] : nullptr, "w", false));
    PLC_TRY(need_field(c, s_inout[i], "s_inout", true));
    if (!(nbar[i] > 0.0) || !std::isfinite(nbar[i])) return fail(c, PLC_ERR_INVALID_ARG, "nbar must be > 0");
    PLC_TRY(check_opts(c, o));
  }
  plc_ctx* c0 = b->ctxs[0];
  return guarded(c0, [&]() -> plc_status {
    for (plc_ctx* c : b->ctxs) ensure_work_fields(c);
    // the contexts' own streams must be idle before the batch graph runs
    for (plc_ctx* c : b->ctxs) plc::check(cudaStreamSynchronize(c->stream), "stream synchronize");
    const plc_status st = plc::batch_map(&b->graph, b->ctxs, N, w, nbar, s_inout, o, stats,
                                         static_cast<cudaStream_t>(stream));
    if (st != PLC_OK) fail(nullptr, st, "a solve of the batch did not converge");
    return st;
  });
}

plc_status plc_batch_destroy(plc_batch* b) {
  delete b;
  return PLC_OK;
}

plc_status plc_profile_enable(plc_ctx* c, int on) {
  if (!c) return fail(nullptr, PLC_ERR_INVALID_ARG, "null context");
  return guarded(c, [&]() -> plc_status {
    plc::profile_reset(c, on != 0);
    return PLC_OK;
  });
}

plc_status plc_profile_read(plc_ctx* c, plc_kernel_time* out, int cap, int* count) {
  if (!c || !count || (cap > 0 && !out)) return fail(c, PLC_ERR_INVALID_ARG, "bad profile_read arguments");
  return guarded(c, [&]() -> plc_status {
    plc::check(cudaStreamSynchronize(c->stream), "stream synchronize");
    plc::profile_collect(c);
    *count = plc::S_NSITES;
    for (int i = 0; i < plc::S_NSITES && i < cap; ++i) {
      std::memset(out[i].name, 0, sizeof(out[i].name));
      std::strncpy(out[i].name, plc::kSiteNames[i], sizeof(out[i].name) - 1);
      out[i].launches = c->prof.launches[i];
      out[i].timed = c->prof.timed[i];
      out[i].total_ms = c->prof.ms[i];
    }
    return PLC_OK;
  });
}

}  // extern "C"
