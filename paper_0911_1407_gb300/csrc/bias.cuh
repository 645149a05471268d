// bias.cuh -- pointwise parts and launchers of the lognormal-prior Poisson
// model with linear bias (Sec. 2.4.1).  The galaxy field is delta_g =
// B delta_M, B the convolution whose Fourier multiplier is the bias b(|k|)
// (Sec. 2.2.1, b = sqrt(P_g / P_M)); with s = ln(1 + delta_M) the expected
// counts are nbar w u, u = 1 + B(e^s - 1), and
//
//   L(s) = 1/2 (s - mu)^T S^-1 (s - mu) + sum_i [nbar w_i u_i - N_i ln u_i]
//   g    = S^-1 (s - mu) + e^s . B q,                  q = nbar w - N / u
//   H v  = S^-1 v + d1 . v + e^s . B(Q . B(e^s . v)),   d1 = e^s . B q,
//                                                       Q = N / u^2
//
// (B is symmetric: b depends on |k| only).  L is +inf where u <= 0 in a cell
// with N > 0.  B runs through the same five-pass spectral pipeline as S^-1,
// with the multiplier table b(|k|) / n^3 in place of 1 / (lambda n^3).
//
// One gradient takes three pipelines: y = S^-1 (s - mu); u from
// B(e^s - 1) (epilogue: q, Q and the likelihood sums); B q (epilogue: g, the
// CG diagonals and ||g||^2).  A line-search trial reuses y + tau S^-1 xi, so
// it needs one pipeline for u; a Hessian-vector product takes three.
#pragma once

#include "launch.cuh"
#include "bias.h"

namespace plc {

template <typename T> inline const T* bias_multiplier(const plc_ctx* c);
template <> inline const float* bias_multiplier<float>(const plc_ctx* c) { return c->Mb32; }
template <> inline const double* bias_multiplier<double>(const plc_ctx* c) { return c->Mb64; }

// ------------------------------- prologues --------------------------------
// e^s - 1 (the matter overdensity delta_M) at s.
template <typename T> struct ProExpm1 {
  const T* s;
  __device__ void prepare() {}
  __device__ void prefetch(size_t i, unsigned cnt) const { prefetch_l2(s + i, cnt * sizeof(T)); }
  __device__ T operator()(size_t i) const { return expm1(__ldg(s + i)); }
  __device__ V4<T> vec4(size_t i) const {
    V4<T> a = ld4(s + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) a.v[j] = expm1(a.v[j]);
    return a;
  }
};

// Trial point s' = s + tau xi (stored) and e^{s'} - 1.
template <typename T, typename TC> struct ProTrial {
  const T* s;
  const TC* xi;
  T tau;
  T* s2;
  __device__ void prepare() {}
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(s + i, cnt * sizeof(T));
    prefetch_l2(xi + i, cnt * sizeof(TC));
  }
  __device__ T operator()(size_t i) const {
    const T sn = __ldg(s + i) + tau * (T)__ldg(xi + i);
    s2[i] = sn;
    return expm1(sn);
  }
  __device__ V4<T> vec4(size_t i) const {
    const V4<T> sv = ld4(s + i);
    const V4<TC> xv = ld4(xi + i);
    V4<T> sn, o;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      sn.v[j] = sv.v[j] + tau * (T)xv.v[j];
      o.v[j] = expm1(sn.v[j]);
    }
    st4(s2 + i, sn);
    return o;
  }
};

// f . v (element-wise), e.g. e^s . v for the inner B of the Hessian.
template <typename T> struct ProMul {
  const T* f;
  const T* v;
  __device__ void prepare() {}
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(f + i, cnt * sizeof(T));
    prefetch_l2(v + i, cnt * sizeof(T));
  }
  __device__ T operator()(size_t i) const { return __ldg(f + i) * __ldg(v + i); }
  __device__ V4<T> vec4(size_t i) const {
    const V4<T> a = ld4(f + i), b = ld4(v + i);
    V4<T> o;
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[j] = a.v[j] * b.v[j];
    return o;
  }
};

// The CG direction p <- M^-1 r + beta p (stored, as ProCgDir), handed on as
// e^s . p.
template <typename T, bool JAC> struct ProCgDirE {
  ProCgDir<T, JAC> dir;
  const T* E;
  __device__ void prepare() { dir.prepare(); }
  __device__ void prefetch(size_t i, unsigned cnt) const {
    dir.prefetch(i, cnt);
    prefetch_l2(E + i, cnt * sizeof(T));
  }
  __device__ T operator()(size_t i) const { return dir(i) * __ldg(E + i); }
  __device__ V4<T> vec4(size_t i) const {
    V4<T> o = dir.vec4(i);
    const V4<T> e = ld4(E + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[j] *= e.v[j];
    return o;
  }
};

// ------------------------------- epilogues --------------------------------
// u = 1 + B(e^s - 1) at the point s (or the trial s' with y' = y + tau
// S^-1 xi); writes q = nbar w - N / u (T), Q = N / u^2 (TC), y' (when yxi is
// given) and accumulates
//   { sum (s - mu) y,  sum [nbar w u - N ln u],  sum N ln u,  sum |N ln u| }.
// A cell with N > 0 and u <= 0 adds +inf to the likelihood sum.
template <typename T, typename TC> struct EpiBiasU {
  static constexpr int NV = 4;
  static constexpr unsigned MAXMASK = 0;
  using Acc = typename AccOf<T>::type;
  const T* s;
  const T* y;
  const T* yxi;          // null: y is the point's own S^-1 (s - mu)
  T tau;
  T* y2;                 // y + tau yxi (when yxi is given)
  const double* w;       // may be null
  const int32_t* N;
  double nbar, mu;
  T* q;
  TC* Q;
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(s + i, cnt * sizeof(T));
    prefetch_l2(y + i, cnt * sizeof(T));
    if (yxi) prefetch_l2(yxi + i, cnt * sizeof(T));
    prefetch_l2(N + i, cnt * sizeof(int32_t));
    if (w) prefetch_l2(w + i, cnt * sizeof(double));
  }
  __device__ __forceinline__ void cell(T st, T yt, T wt, int32_t ni, T z, Acc* acc, T& qo,
                                       TC& Qo) const {
    const T u = (T)1 + z;
    const T nbw = (T)nbar * wt;
    acc[0].add((st - (T)mu) * yt);
    qo = nbw;
    Qo = (TC)0;
    if (ni > 0) {
      const T nf = (T)ni;
      if (u > (T)0) {
        const T inv = (T)1 / u;
        const T l = nf * log(u);
        acc[1].add(nbw * u - l);
        acc[2].add(l);
        acc[3].add(l < (T)0 ? -l : l);
        qo = nbw - nf * inv;
        Qo = (TC)(nf * inv * inv);
      } else {
        acc[1].add((T)INFINITY);
      }
    } else {
      acc[1].add(nbw * u);
    }
  }
  __device__ void operator()(size_t i, T z, Acc* acc) const {
    T yt = __ldg(y + i);
    if (yxi) {
      yt += tau * __ldg(yxi + i);
      y2[i] = yt;
    }
    T qo;
    TC Qo;
    cell(__ldg(s + i), yt, w ? (T)__ldg(w + i) : (T)1, __ldg(N + i), z, acc, qo, Qo);
    q[i] = qo;
    Q[i] = Qo;
  }
  __device__ void vec4(size_t i, const V4<T>& z, Acc* acc) const {
    const V4<T> sv = ld4(s + i);
    V4<T> yv = ld4(y + i);
    if (yxi) {
      const V4<T> xv = ld4(yxi + i);
#pragma unroll
      for (int j = 0; j < 4; ++j) yv.v[j] += tau * xv.v[j];
      st4(y2 + i, yv);
    }
    const V4<int32_t> nv = ld4(N + i);
    V4<double> wv{{1.0, 1.0, 1.0, 1.0}};
    if (w) wv = ld4(w + i);
    V4<T> qv;
    V4<TC> Qv;
#pragma unroll
    for (int j = 0; j < 4; ++j) cell(sv.v[j], yv.v[j], (T)wv.v[j], nv.v[j], z.v[j], acc, qv.v[j], Qv.v[j]);
    st4(q + i, qv);
    st4(Q + i, Qv);
  }
};

// The sums of EpiBiasU into red[0], red[1], red[3], red[4] (the slots of
// the unity-bias gradient: prior term, likelihood, sum N ln u, sum |N ln u|).
struct FinBiasU {
  __device__ void operator()(const double* t, DevScalars* sc) const {
    sc->red[0] = t[0];
    sc->red[1] = t[1];
    sc->red[3] = t[2];
    sc->red[4] = t[3];
  }
};

// Gradient g = y + e^s . B q from z = B q; writes g (T, may be null), the CG
// start r = -g, E = e^s, the Hessian diagonal d1 = e^s . B q and the Jacobi
// diagonal Dj = |d1| + e^{2s} Q (TC, each may be null); accumulates
// { ||g||^2, r^T M^-1 r } with M = diag(Dj + c) (Jacobi) or I.
template <typename T, typename TC> struct EpiBiasG {
  static constexpr int NV = 2;
  static constexpr unsigned MAXMASK = 0;
  using Acc = typename AccOf<T>::type;
  const T* s;
  const T* y;
  const TC* Q;
  T* g;
  TC* r;
  TC* E;
  TC* d1;
  TC* Dj;
  double c;
  int jac;
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(s + i, cnt * sizeof(T));
    prefetch_l2(y + i, cnt * sizeof(T));
    prefetch_l2(Q + i, cnt * sizeof(TC));
  }
  __device__ __forceinline__ void cell(T st, T yt, TC Qi, T z, Acc* acc, T& gi, TC& ei, TC& di,
                                       TC& dj) const {
    const T e = exp(st);
    const T dd = e * z;
    gi = yt + dd;
    ei = (TC)e;
    di = (TC)dd;
    dj = (di < (TC)0 ? -di : di) + ei * ei * Qi;
    acc[0].add(gi * gi);
    const TC gc = (TC)gi;
    acc[1].add((T)(jac ? gc * jacobi(gc, dj, (TC)c) : gc * gc));
  }
  __device__ void operator()(size_t i, T z, Acc* acc) const {
    T gi;
    TC ei, di, dj;
    cell(__ldg(s + i), __ldg(y + i), __ldg(Q + i), z, acc, gi, ei, di, dj);
    if (g) g[i] = gi;
    if (r) r[i] = (TC)(-gi);
    if (E) E[i] = ei;
    if (d1) d1[i] = di;
    if (Dj) Dj[i] = dj;
  }
  __device__ void vec4(size_t i, const V4<T>& z, Acc* acc) const {
    const V4<T> sv = ld4(s + i), yv = ld4(y + i);
    const V4<TC> Qv = ld4(Q + i);
    V4<T> gv;
    V4<TC> rv, ev, dv, jv;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cell(sv.v[j], yv.v[j], Qv.v[j], z.v[j], acc, gv.v[j], ev.v[j], dv.v[j], jv.v[j]);
      rv.v[j] = (TC)(-gv.v[j]);
    }
    if (g) st4(g + i, gv);
    if (r) st4(r + i, rv);
    if (E) st4(E + i, ev);
    if (d1) st4(d1 + i, dv);
    if (Dj) st4(Dj + i, jv);
  }
};

// The gradient's sums (red[2] = ||g||^2, red[5] = r^T M^-1 r) and the start
// of CG on H xi = -g from xi = 0, as FinGrad.
struct FinBiasG {
  __device__ void operator()(const double* t, DevScalars* sc) const {
    sc->red[2] = t[0];
    sc->red[5] = t[1];
    sc->rz = t[1];
    sc->rr = t[0];
    sc->bnorm2 = t[0];
    sc->iter = 0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->breakdown = 0;
    sc->xb = 0.0;
    sc->xHx = 0.0;
    sc->xmax = 0.0;
    sc->done = t[0] <= 0.0 ? 1 : 0;
  }
};

// out = f . z.
template <typename T> struct EpiMul {
  static constexpr int NV = 0;
  static constexpr unsigned MAXMASK = 0;
  using Acc = AccD;
  const T* f;
  T* out;
  __device__ void prefetch(size_t i, unsigned cnt) const { prefetch_l2(f + i, cnt * sizeof(T)); }
  __device__ void operator()(size_t i, T z, Acc*) const { out[i] = __ldg(f + i) * z; }
  __device__ void vec4(size_t i, const V4<T>& z, Acc*) const {
    const V4<T> a = ld4(f + i);
    V4<T> o;
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[j] = a.v[j] * z.v[j];
    st4(out + i, o);
  }
};

// H v = S^-1 v + d1 . v + t2 from z = S^-1 v and t2 = e^s . B(Q . B(e^s v));
// accumulates v^T H v.
template <typename T> struct EpiHessB {
  static constexpr int NV = 1;
  static constexpr unsigned MAXMASK = 0;
  using Acc = typename AccOf<T>::type;
  const T* d1;
  const T* v;
  const T* t2;
  T* out;
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(d1 + i, cnt * sizeof(T));
    prefetch_l2(v + i, cnt * sizeof(T));
    prefetch_l2(t2 + i, cnt * sizeof(T));
  }
  __device__ void operator()(size_t i, T z, Acc* acc) const {
    const T vi = __ldg(v + i);
    const T hv = z + __ldg(d1 + i) * vi + __ldg(t2 + i);
    out[i] = hv;
    acc[0].add(vi * hv);
  }
  __device__ void vec4(size_t i, const V4<T>& z, Acc* acc) const {
    const V4<T> dv = ld4(d1 + i), vv = ld4(v + i), tv = ld4(t2 + i);
    V4<T> o;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      o.v[j] = z.v[j] + dv.v[j] * vv.v[j] + tv.v[j];
      acc[0].add(vv.v[j] * o.v[j]);
    }
    st4(out + i, o);
  }
};

// x = p and max |x|: the preconditioned gradient step -M^-1 g taken when
// the CG meets non-positive curvature on its first direction.
template <typename TC>
__global__ void __launch_bounds__(kThreads)
k_copy_absmax(const TC* __restrict__ p, TC* __restrict__ x, size_t n3, RedArgs ra) {
  typename AccOf<TC>::type acc[1];
  acc[0].init(true);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const TC v = p[i];
    x[i] = v;
    acc[0].max(v < (TC)0 ? -v : v);
  }
  struct Fin {
    __device__ void operator()(const double* t, DevScalars* sc) const { sc->xmax = t[0]; }
  };
  block_reduce_finish_acc<1, 1u>(acc, ra, Fin{});
}

// -------------------------------- launchers --------------------------------
constexpr int kBiasSites = 2;   // run_pipeline's site group of the bias model

// y = S^-1 (x - shift), x held as TX.
template <typename T, typename TX>
void bias_prior(plc_ctx* c, const TX* x, double shift, T* y) {
  run_pipeline<T>(c, ProShift<T, TX>{x, shift}, EpiStore<T>{y}, FinNone{}, 0, nullptr,
                  kBiasSites);
}

// u at s (xi null) or at the trial s' = s + tau xi (stored in s2, with
// y2 = y + tau yxi); q, Q and the likelihood sums (FinBiasU).
template <typename T, typename TC>
void bias_density(plc_ctx* c, const T* s, const TC* xi, double tau, T* s2, const T* y,
                  const T* yxi, T* y2, const int32_t* N, const double* w, double nbar, T* q,
                  TC* Q) {
  if (xi)
    run_pipeline<T>(c, ProTrial<T, TC>{s, xi, (T)tau, s2},
                    EpiBiasU<T, TC>{s2, y, yxi, (T)tau, y2, w, N, nbar, c->mu, q, Q},
                    FinBiasU{}, 0, nullptr, kBiasSites, bias_multiplier<T>(c));
  else
    run_pipeline<T>(c, ProExpm1<T>{s},
                    EpiBiasU<T, TC>{s, y, nullptr, (T)0, nullptr, w, N, nbar, c->mu, q, Q},
                    FinBiasU{}, 0, nullptr, kBiasSites, bias_multiplier<T>(c));
}

// g from B q (FinBiasG starts the CG).
template <typename T, typename TC>
void bias_gradient(plc_ctx* c, const T* s, const T* y, const T* q, const TC* Q, T* g, TC* r,
                   TC* E, TC* d1, TC* Dj, bool jac) {
  run_pipeline<T>(c, ProLoad<T>{q},
                  EpiBiasG<T, TC>{s, y, Q, g, r, E, d1, Dj, c->jac_c, jac ? 1 : 0}, FinBiasG{}, 0,
                  nullptr, kBiasSites, bias_multiplier<T>(c));
}

// H p for the CG (p formed from r in the first pipeline), then FinAlpha.
template <typename TC>
void bias_cg_hv(plc_ctx* c, const TC* r, const TC* Dj, TC* p, const TC* E, const TC* Q,
                const TC* d1, TC* t, TC* t2, TC* Hp, bool jac) {
  const int* done = &c->sc->done;
  const TC* Mb = bias_multiplier<TC>(c);
  if (jac)
    run_pipeline<TC>(c, ProCgDirE<TC, true>{{r, Dj, (TC)c->jac_c, p, c->sc}, E}, EpiMul<TC>{Q, t},
                     FinNone{}, 0, done, kBiasSites, Mb);
  else
    run_pipeline<TC>(c, ProCgDirE<TC, false>{{r, Dj, (TC)c->jac_c, p, c->sc}, E},
                     EpiMul<TC>{Q, t}, FinNone{}, 0, done, kBiasSites, Mb);
  run_pipeline<TC>(c, ProLoad<TC>{t}, EpiMul<TC>{E, t2}, FinNone{}, 0, done, kBiasSites, Mb);
  run_pipeline<TC>(c, ProLoad<TC>{p}, EpiHessB<TC>{d1, p, t2, Hp}, FinAlpha{}, 0, done,
                   kBiasSites);
}

// H v at the point whose E, Q, d1 are given (the public operator).
template <typename T>
void bias_hv(plc_ctx* c, const T* v, const T* E, const T* Q, const T* d1, T* t, T* t2, T* Hv) {
  const T* Mb = bias_multiplier<T>(c);
  run_pipeline<T>(c, ProMul<T>{E, v}, EpiMul<T>{Q, t}, FinNone{}, 0, nullptr, kBiasSites, Mb);
  run_pipeline<T>(c, ProLoad<T>{t}, EpiMul<T>{E, t2}, FinNone{}, 0, nullptr, kBiasSites, Mb);
  run_pipeline<T>(c, ProLoad<T>{v}, EpiHessB<T>{d1, v, t2, Hv}, FinStore<1>{}, 0, nullptr,
                  kBiasSites);
}

template <typename TC> void bias_fallback(plc_ctx* c, const TC* p, TC* x) {
  LaunchScope ls(c, S_BIAS);
  k_copy_absmax<TC><<<pw_blocks(c), kThreads, 0, c->stream>>>(p, x, c->n3(), red_args(c));
  check(cudaGetLastError(), "k_copy_absmax");
}

}  // namespace plc
