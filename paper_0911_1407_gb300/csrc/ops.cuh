// ops.cuh -- pointwise parts of the Newton-Krylov MAP solve (Sec. 3.1, 3.1.2).
//
// Prologues (fused into the first FFT pass) produce the field to transform;
// epilogues (fused into the last pass) turn y = S^-1 x into the gradient or a
// Hessian-vector product and accumulate the dot products the solver needs;
// finalizers run once on the grid totals.  Element-wise kernels cover the CG
// recurrences and set-up work.  Reductions accumulate per thread in the
// field's own precision made compensated (Kahan pairs for FP32 fields,
// float-float for the float-float transforms, plain FP64 for FP64 fields),
// merge across lanes and warps in that arithmetic, and go to FP64 once per
// block; the block totals are summed in FP64 in block order.
#pragma once

#include "common.cuh"
#include "ff.cuh"

namespace plc {

// ------------------------- 4-wide element access ---------------------------
// Element-wise kernels move four consecutive elements per thread and step
// with 16-byte loads (n^3 is a multiple of 8; fields are 16-byte aligned).
template <typename T> struct V4 { T v[4]; };
__device__ __forceinline__ V4<float> ld4(const float* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return V4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return V4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ V4<int32_t> ld4(const int32_t* p) {
  const int4 a = __ldg(reinterpret_cast<const int4*>(p));
  return V4<int32_t>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& a) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a.v[0], a.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(a.v[2], a.v[3]);
}

// Jacobi preconditioner z = r / (D + c), the same expression wherever the CG
// needs it (a fast reciprocal for FP32; M stays a fixed positive diagonal).
__device__ __forceinline__ float jacobi(float r, float d, float c) { return __fdividef(r, d + c); }
__device__ __forceinline__ double jacobi(double r, double d, double c) { return r / (d + c); }

// ------------------------------- prologues --------------------------------
// Every prologue has prepare(), run once per block before the element loop.
// vec4(i) handles the four consecutive elements i .. i+3 (i a multiple of 4).
template <typename T> struct ProLoad {
  const T* x;
  __device__ void prepare() {}
  __device__ void prefetch(size_t i, unsigned cnt) const { prefetch_l2(x + i, cnt * sizeof(T)); }
  __device__ T operator()(size_t i) const { return __ldg(x + i); }
  __device__ V4<T> vec4(size_t i) const { return ld4(x + i); }
};

// s - mu: the prior term of the gradient (Sec. 2.3, Eq. priorlog).  s may be
// held in a wider type than the transform.
template <typename T, typename TS> struct ProShift {
  const TS* s;
  double mu;
  __device__ void prepare() {}
  __device__ void prefetch(size_t i, unsigned cnt) const { prefetch_l2(s + i, cnt * sizeof(TS)); }
  // difference taken in the transform precision (no FP64 work for float)
  __device__ T operator()(size_t i) const { return (T)__ldg(s + i) - (T)mu; }
  __device__ V4<T> vec4(size_t i) const {
    const V4<TS> a = ld4(s + i);
    V4<T> o;
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[j] = (T)a.v[j] - (T)mu;
    return o;
  }
};

// CG search direction p <- M^-1 r + beta p (beta from the device scalars;
// beta = 0 on the first step, where p is not read).
template <typename T, bool JAC> struct ProCgDir {
  // x-forward prologue steps in flight per thread: 60.8-61.5 us at 4 against
  // 63.0-63.3 at 8 and 61.3 at 2 for 256^3 (three loads per step)
  static constexpr int kBatch = 4;
  const T* r;
  const T* D;
  T c;                 // (S^-1)_ii, the prior's share of diag(H)
  T* p;
  const DevScalars* sc;
  T beta;              // loaded by prepare()
  __device__ void prepare() { beta = (T)__ldg(&sc->beta); }
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(r + i, cnt * sizeof(T));
    if (JAC) prefetch_l2(D + i, cnt * sizeof(T));
    if (beta != (T)0) prefetch_l2(p + i, cnt * sizeof(T));
  }
  __device__ T operator()(size_t i) const {
    const T ri = __ldg(r + i);
    const T zi = JAC ? jacobi(ri, __ldg(D + i), c) : ri;
    const T pn = beta == (T)0 ? zi : zi + beta * __ldg(p + i);
    p[i] = pn;
    return pn;
  }
  __device__ V4<T> vec4(size_t i) const {
    const V4<T> rv = ld4(r + i);
    V4<T> dv, pv, o;
    if (JAC) dv = ld4(D + i);
    if (beta != (T)0) pv = ld4(p + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T zi = JAC ? jacobi(rv.v[j], dv.v[j], c) : rv.v[j];
      o.v[j] = beta == (T)0 ? zi : zi + beta * pv.v[j];
    }
    st4(p + i, o);
    return o;
  }
};

// s - mu from an FP64 s, in float-float for float-float transforms: s split
// into float-float by its bit fields, mu given as a float-float (error a few
// 2^-48 of max(|s|, |mu|)).
struct ProShiftFF {
  const double* s;
  ff mu;
  __device__ void prepare() {}
  __device__ void prefetch(size_t i, unsigned cnt) const { prefetch_l2(s + i, cnt * sizeof(double)); }
  __device__ V4<ff> vec4(size_t i) const {
    const V4<double> a = ld4(s + i);
    return V4<ff>{{ff_split(a.v[0]) - mu, ff_split(a.v[1]) - mu, ff_split(a.v[2]) - mu,
                   ff_split(a.v[3]) - mu}};
  }
};

// ------------------------------- epilogues --------------------------------
// The gradient epilogue of EpiGrad for float-float transforms (the FP64
// gradient of the mixed solve), kept in float-float: y (from the transform),
// s (FP64 in memory, split by its bit fields), D = nbar w e^s (exp_ff),
// g = y + D - N and the six sums of EpiGrad are float-float; y and g are
// stored in FP64, D and r = -g in FP32.  With STORE false nothing is stored
// (the sums alone, for a stopping test that may end the solve).
template <bool STORE = true> struct EpiGradFF {
  static constexpr int NV = 6;
  static constexpr unsigned MAXMASK = 0;
  using Acc = AccFF;
  const double* s;
  const double* w;      // may be null
  const int32_t* N;
  ff nbar, mu;
  double* yout;
  double* g;
  float* D;
  float* r;
  float c;              // Jacobi constant (S^-1)_ii
  int jac;
  const ff* exptab;     // 2^(j/64), j < 64
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(s + i, cnt * sizeof(double));
    prefetch_l2(N + i, cnt * sizeof(int32_t));
    if (w) prefetch_l2(w + i, cnt * sizeof(double));
  }
  __device__ void vec4(size_t i, const V4<ff>& y, Acc* acc) const {
    const V4<double> sv = ld4(s + i);
    const V4<int32_t> nv = ld4(N + i);
    V4<double> wv{{1.0, 1.0, 1.0, 1.0}};
    if (w) wv = ld4(w + i);
    const ff nb = nbar, m = mu;
    V4<double> yo, go;
    V4<float> dv, rv;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const ff st = ff_split(sv.v[j]);
      ff d = nb * exp_ff(st, exptab);
      if (w) d = d * ff_split(wv.v[j]);
      const ff ni((float)nv.v[j], 0.f);    // counts below 2^24 are exact
      const ff gi = (y.v[j] + d) - ni;
      const ff ns = ni * st;
      acc[0].add((st - m) * y.v[j]);
      acc[1].add(d - ns);
      acc[2].add(gi * gi);
      acc[3].add(ns);
      acc[4].add(ni * ff_abs(st));
      const float gc = gi.hi + gi.lo, dc = d.hi + d.lo;
      acc[5].add(ff(jac ? gc * jacobi(gc, dc, c) : gc * gc, 0.f));
      if constexpr (STORE) {
        yo.v[j] = to_double(y.v[j]);
        go.v[j] = to_double(gi);
        dv.v[j] = dc;
        rv.v[j] = -gc;
      }
    }
    if constexpr (STORE) {
      if (yout) st4(yout + i, yo);
      if (g) st4(g + i, go);
      if (D) st4(D + i, dv);
      if (r) st4(r + i, rv);
    }
  }
};

// An FP64 epilogue behind float-float transforms: y = hi + lo in FP64.
template <typename Epi> struct EpiFF {
  static constexpr int NV = Epi::NV;
  static constexpr unsigned MAXMASK = Epi::MAXMASK;
  using Acc = typename Epi::Acc;
  Epi epi;
  __device__ void prefetch(size_t i, unsigned cnt) const { epi.prefetch(i, cnt); }
  __device__ void vec4(size_t i, const V4<ff>& y, Acc* acc) const {
    const V4<double> yd{{to_double(y.v[0]), to_double(y.v[1]), to_double(y.v[2]),
                         to_double(y.v[3])}};
    epi.vec4(i, yd, acc);
  }
};

template <typename T> struct EpiStore {
  static constexpr int NV = 0;
  static constexpr unsigned MAXMASK = 0;
  using Acc = AccD;
  T* out;
  __device__ void prefetch(size_t, unsigned) const {}
  __device__ void operator()(size_t i, T y, Acc*) const { out[i] = y; }
  __device__ void vec4(size_t i, const V4<T>& y, Acc*) const { st4(out + i, y); }
};

// H v = S^-1 v + nbar w e^s v (Sec. 3.1.2) with the diagonal computed here.
template <typename T> struct EpiHessS {
  static constexpr int NV = 0;
  static constexpr unsigned MAXMASK = 0;
  const T* s;
  const T* w;          // may be null (w = 1)
  T nbar;
  const T* v;
  T* out;
  using Acc = AccD;
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(s + i, cnt * sizeof(T));
    prefetch_l2(v + i, cnt * sizeof(T));
    if (w) prefetch_l2(w + i, cnt * sizeof(T));
  }
  __device__ void operator()(size_t i, T y, Acc*) const {
    const T d = nbar * (w ? __ldg(w + i) : (T)1) * exp(__ldg(s + i));
    out[i] = y + d * __ldg(v + i);
  }
  __device__ void vec4(size_t i, const V4<T>& y, Acc*) const {
    const V4<T> sv = ld4(s + i), vv = ld4(v + i);
    V4<T> wv{{(T)1, (T)1, (T)1, (T)1}}, o;
    if (w) wv = ld4(w + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[j] = y.v[j] + nbar * wv.v[j] * exp(sv.v[j]) * vv.v[j];
    st4(out + i, o);
  }
};

// CG product H p = S^-1 p + D p, accumulating p^T H p.
template <typename T> struct EpiHessD {
  static constexpr int NV = 1;
  static constexpr unsigned MAXMASK = 0;
  static constexpr int kUnroll = 4;     // measured: 58 us against 63 at unroll 2 (256^3)
  const T* D;
  const T* v;
  T* out;
  using Acc = typename AccOf<T>::type;
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(D + i, cnt * sizeof(T));
    prefetch_l2(v + i, cnt * sizeof(T));
  }
  __device__ void operator()(size_t i, T y, Acc* acc) const {
    const T vi = __ldg(v + i);
    const T hv = y + __ldg(D + i) * vi;
    out[i] = hv;
    acc[0].add(vi * hv);
  }
  __device__ void vec4(size_t i, const V4<T>& y, Acc* acc) const {
    const V4<T> vv = ld4(v + i), dv = ld4(D + i);
    V4<T> o;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      o.v[j] = y.v[j] + dv.v[j] * vv.v[j];
      acc[0].add(vv.v[j] * o.v[j]);
    }
    st4(out + i, o);
  }
};

// Gradient g = S^-1 (s - mu) + nbar w e^s - N (Sec. 3.1.2) and the pieces of
// -ln P.  T: transform type; TS: type of s; TW: type of w; TC: type of the CG
// fields.  Optionally writes y = S^-1 (s - mu), g, the diagonal
// D = nbar w e^s and the CG start r = -g.
// acc = { sum (s-mu) y, sum (D - N s), sum g^2, sum N s, sum N |s|,
//         sum r M^-1 r }  with M = diag(D + c) (Jacobi) or I.
template <typename T, typename TS, typename TW, typename TC> struct EpiGrad {
  static constexpr int NV = 6;
  static constexpr unsigned MAXMASK = 0;
  using Acc = typename AccOf<T>::type;
  const TS* s;
  const TW* w;          // may be null
  const int32_t* N;
  double nbar, mu;
  T* yout;              // may be null
  T* g;                 // may be null
  TC* D;                // may be null
  TC* r;                // may be null
  double c;             // Jacobi constant (S^-1)_ii
  int jac;
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(s + i, cnt * sizeof(TS));
    prefetch_l2(N + i, cnt * sizeof(int32_t));
    if (w) prefetch_l2(w + i, cnt * sizeof(TW));
  }
  // one cell: returns g and d, accumulates the sums
  __device__ __forceinline__ void cell(T st, T wt, T ni, T y, Acc* acc, T& gi, T& d) const {
    d = (T)nbar * wt * exp(st);
    gi = y + d - ni;
    acc[0].add((st - (T)mu) * y);
    acc[1].add(d - ni * st);
    acc[2].add(gi * gi);
    acc[3].add(ni * st);
    acc[4].add(ni * (st < (T)0 ? -st : st));
    // r^T M^-1 r in the precision of the CG fields
    const TC gc = (TC)gi;
    acc[5].add((T)(jac ? gc * jacobi(gc, (TC)d, (TC)c) : gc * gc));
  }
  __device__ void operator()(size_t i, T y, Acc* acc) const {
    T gi, d;
    cell((T)__ldg(s + i), w ? (T)__ldg(w + i) : (T)1, (T)__ldg(N + i), y, acc, gi, d);
    if (yout) yout[i] = y;
    if (g) g[i] = gi;
    if (D) D[i] = (TC)d;
    if (r) r[i] = (TC)(-gi);
  }
  __device__ void vec4(size_t i, const V4<T>& y, Acc* acc) const {
    const V4<TS> sv = ld4(s + i);
    const V4<int32_t> nv = ld4(N + i);
    V4<TW> wv{{(TW)1, (TW)1, (TW)1, (TW)1}};
    if (w) wv = ld4(w + i);
    V4<T> gv;
    V4<TC> dv, rv;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T gi, d;
      cell((T)sv.v[j], (T)wv.v[j], (T)nv.v[j], y.v[j], acc, gi, d);
      gv.v[j] = gi;
      dv.v[j] = (TC)d;
      rv.v[j] = (TC)(-gi);
    }
    if (yout) st4(yout + i, y);
    if (g) st4(g + i, gv);
    if (D) st4(D + i, dv);
    if (r) st4(r + i, rv);
  }
};

// ----------------------- Gaussian prior, Poisson likelihood -----------------
// One cell of the Gaussian-prior model (Sec. 2.2.2, Eq. MAPG; gradient and
// Hessian of Sec. 3.1.1 without the factor S): with u = 1 + delta,
//   g = y + nbar w - N / u,   D = N / u^2,
//   -ln P = 1/2 delta^T y + sum [nbar w u - N ln u],
// y = S^-1 delta.  The sums mirror the lognormal model's, with ln u in the
// place of s: {delta y, nbar w u - N ln u, g^2, N ln u, N |ln u|, r M^-1 r}.
// A cell with N > 0 and u <= 0 lies outside the domain: its likelihood term
// is +inf.
template <typename T, typename TC>
__device__ __forceinline__ void gauss_cell(T delta, T wt, T ni, T nb, T y, TC c, int jac,
                                           typename AccOf<T>::type* acc, T& gi, T& d) {
  const T u = (T)1 + delta;
  const bool occ = ni > (T)0;
  // 1/u only where the likelihood has its logarithm (an empty cell may sit
  // at u = 0 exactly)
  const T inv = occ ? (T)1 / u : (T)0;
  const T nio = ni * inv;
  gi = y + nb * wt - nio;
  d = nio * inv;
  const T lu = occ ? (u > (T)0 ? ni * log(u) : (T)INFINITY) : (T)0;
  acc[0].add(delta * y);
  acc[1].add(nb * wt * u - lu);
  acc[2].add(gi * gi);
  acc[3].add(lu);
  acc[4].add(lu < (T)0 ? -lu : lu);
  const TC gc = (TC)gi;
  acc[5].add((T)(jac ? gc * jacobi(gc, (TC)d, c) : gc * gc));
}

// Gradient epilogue of the Gaussian-prior model (the prologue passes delta:
// ProShift with mu = 0).  Writes y, g (T), D, r = -g (TC); sums as EpiGrad.
template <typename T, typename TS, typename TC> struct EpiGradG {
  static constexpr int NV = 6;
  static constexpr unsigned MAXMASK = 0;
  using Acc = typename AccOf<T>::type;
  const TS* s;           // delta
  const double* w;       // may be null
  const int32_t* N;
  double nbar;
  T* yout;
  T* g;
  TC* D;
  TC* r;
  double c;
  int jac;
  __device__ void prefetch(size_t i, unsigned cnt) const {
    prefetch_l2(s + i, cnt * sizeof(TS));
    prefetch_l2(N + i, cnt * sizeof(int32_t));
    if (w) prefetch_l2(w + i, cnt * sizeof(double));
  }
  __device__ void operator()(size_t i, T y, Acc* acc) const {
    T gi, d;
    gauss_cell<T, TC>((T)__ldg(s + i), w ? (T)__ldg(w + i) : (T)1, (T)__ldg(N + i), (T)nbar, y,
                      (TC)c, jac, acc, gi, d);
    if (yout) yout[i] = y;
    if (g) g[i] = gi;
    if (D) D[i] = (TC)d;
    if (r) r[i] = (TC)(-gi);
  }
  __device__ void vec4(size_t i, const V4<T>& y, Acc* acc) const {
    const V4<TS> sv = ld4(s + i);
    const V4<int32_t> nv = ld4(N + i);
    V4<double> wv{{1.0, 1.0, 1.0, 1.0}};
    if (w) wv = ld4(w + i);
    V4<T> gv;
    V4<TC> dv, rv;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T gi, d;
      gauss_cell<T, TC>((T)sv.v[j], (T)wv.v[j], (T)nv.v[j], (T)nbar, y.v[j], (TC)c, jac, acc, gi,
                        d);
      gv.v[j] = gi;
      dv.v[j] = (TC)d;
      rv.v[j] = (TC)(-gi);
    }
    if (yout) st4(yout + i, y);
    if (g) st4(g + i, gv);
    if (D) st4(D + i, dv);
    if (r) st4(r + i, rv);
  }
};

// sum lam_i y_i, y = S^-1 x.
template <typename T, typename TL> struct EpiDot {
  static constexpr int NV = 1;
  static constexpr unsigned MAXMASK = 0;
  const TL* lam;
  using Acc = AccD;
  __device__ void prefetch(size_t i, unsigned cnt) const { prefetch_l2(lam + i, cnt * sizeof(TL)); }
  __device__ void operator()(size_t i, T y, Acc* acc) const {
    acc[0].add((double)__ldg(lam + i) * (double)y);
  }
  __device__ void vec4(size_t i, const V4<T>& y, Acc* acc) const {
    const V4<TL> lv = ld4(lam + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[0].add((double)lv.v[j] * (double)y.v[j]);
  }
};

// ------------------------------- finalizers -------------------------------
struct FinNone {
  __device__ void operator()(const double*, DevScalars*) const {}
};

template <int NV> struct FinStore {
  __device__ void operator()(const double* t, DevScalars* sc) const {
#pragma unroll
    for (int j = 0; j < NV; ++j) sc->red[j] = t[j];
  }
};

// After a gradient: store the sums and start CG on H xi = -g from xi = 0
// (r = -g was written by the epilogue).  The CG tolerance and iteration cap
// are arguments of the CG update.
struct FinGrad {
  __device__ void operator()(const double* t, DevScalars* sc) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) sc->red[j] = t[j];
    sc->rz = t[5];
    sc->rr = t[2];
    sc->bnorm2 = t[2];
    sc->iter = 0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->breakdown = 0;
    sc->xb = 0.0;
    sc->xHx = 0.0;
    sc->xmax = 0.0;
    sc->done = t[2] <= 0.0 ? 1 : 0;
  }
};

// alpha = r^T z / p^T H p; a non-positive curvature stops the CG.  Also
// accumulates xi^T b = sum alpha_k r_k^T z_k and xi^T H xi =
// sum alpha_k^2 p_k^T H p_k (H-conjugate directions): the two sums of the
// step length of Eq. (New5).
struct FinAlpha {
  __device__ void operator()(const double* t, DevScalars* sc) const {
    sc->pHp = t[0];
    if (!(t[0] > 0.0)) {
      sc->breakdown = 1;
      sc->done = 1;
      sc->alpha = 0.0;
    } else {
      const double a = sc->rz / t[0];
      sc->alpha = a;
      sc->xb += a * sc->rz;
      sc->xHx += a * a * t[0];
    }
  }
};

// ------------------------------ CG kernels --------------------------------
// CG scalars at the start of a solve from x = 0 (t = {r^T M^-1 r, r^T r}).
struct FinCgStart {
  __device__ void operator()(const double* t, DevScalars* sc) const {
    sc->rz = t[0];
    sc->rr = t[1];
    sc->bnorm2 = t[1];
    sc->iter = 0;
    sc->beta = 0.0;
    sc->alpha = 0.0;
    sc->breakdown = 0;
    sc->xb = 0.0;
    sc->xHx = 0.0;
    sc->xmax = 0.0;
    sc->done = t[1] <= 0.0 ? 1 : 0;
  }
};

// LSQ-Wiener filter (Sec. 4.1.1, Eq. WF, unity bias): the diagonal
// D = nbar w of (S^-1 + diag(nbar w)) delta = N - nbar w and the CG start
// r = N - nbar w from delta = 0.
template <typename TC, bool JAC>
__global__ void __launch_bounds__(kThreads)
k_lsq_init(const int32_t* __restrict__ N, const double* __restrict__ w, double nbar, TC c,
           TC* __restrict__ D, TC* __restrict__ r, size_t n3, RedArgs ra) {
  typename AccOf<TC>::type acc[2];
  acc[0].init(false);
  acc[1].init(false);
  const TC nb = (TC)nbar;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const TC d = w ? (TC)(nbar * w[i]) : nb;
    const TC ri = (TC)N[i] - d;
    D[i] = d;
    r[i] = ri;
    const TC zi = JAC ? jacobi(ri, d, c) : ri;
    acc[0].add(ri * zi);
    acc[1].add(ri * ri);
  }
  block_reduce_finish_acc<2, 0u>(acc, ra, FinCgStart{});
}

// Start CG on H x = b from x = 0: r = b, rz = r^T M^-1 r, rr = r^T r.
template <typename TC, typename TB, bool JAC>
__global__ void __launch_bounds__(kThreads)
k_cg_init(const TB* __restrict__ b, const TC* __restrict__ D, TC c, TC* __restrict__ r,
          size_t n3, RedArgs ra) {
  typename AccOf<TC>::type a0, a1;
  a0.init(false);
  a1.init(false);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const TC ri = (TC)b[i];
    r[i] = ri;
    const TC zi = JAC ? jacobi(ri, D[i], c) : ri;
    a0.add(ri * zi);
    a1.add(ri * ri);
  }
  typename AccOf<TC>::type acc[2] = {a0, a1};
  block_reduce_finish_acc<2, 0u>(acc, ra, FinCgStart{});
}

// x += alpha p (x = alpha p on the first step, so x needs no clearing),
// r -= alpha H p, then r^T M^-1 r, ||r||^2 and max |x| for beta, the
// stopping test ||r||^2 <= rtol^2 ||b||^2 and the Newton step cap.
template <typename TC, bool JAC>
__global__ void __launch_bounds__(kThreads)
k_cg_update(TC* __restrict__ x, TC* __restrict__ r, const TC* __restrict__ p,
            const TC* __restrict__ Hp, const TC* __restrict__ D, TC c, size_t n3,
            RedArgs ra, double rtol2, int max_iter) {
  if (ra.sc->done) return;
  const TC alpha = (TC)ra.sc->alpha;
  const bool first = ra.sc->iter == 0;
  typename AccOf<TC>::type a0, a1, a2;
  a0.init(false);
  a1.init(false);
  a2.init(true);
  const size_t step = (size_t)gridDim.x * blockDim.x * 4;
#pragma unroll 2
  for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4; i < n3; i += step) {
    const V4<TC> pv = ld4(p + i), hv = ld4(Hp + i), dv = ld4(D + i);
    V4<TC> xv = first ? V4<TC>{} : ld4(x + i);
    V4<TC> rv = ld4(r + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const TC xn = first ? alpha * pv.v[j] : xv.v[j] + alpha * pv.v[j];
      xv.v[j] = xn;
      const TC ri = rv.v[j] - alpha * hv.v[j];
      rv.v[j] = ri;
      const TC zi = JAC ? jacobi(ri, dv.v[j], c) : ri;
      a0.add(ri * zi);
      a1.add(ri * ri);
      a2.max(xn < (TC)0 ? -xn : xn);
    }
    st4(x + i, xv);
    st4(r + i, rv);
  }
  typename AccOf<TC>::type acc[3] = {a0, a1, a2};
  struct Fin {
    double rtol2;
    int max_iter;
    __device__ void operator()(const double* t, DevScalars* sc) const {
      const double rt2 = rtol2 < 0.0 ? sc->rtol2 : rtol2;
      const int mi = rtol2 < 0.0 ? sc->max_iter : max_iter;
      sc->beta = t[0] / sc->rz;
      sc->rz = t[0];
      sc->rr = t[1];
      sc->xmax = t[2];
      sc->iter += 1;
      if (t[1] <= rt2 * sc->bnorm2 || sc->iter >= mi) sc->done = 1;
    }
  };
  block_reduce_finish_acc<3, 1u << 2>(acc, ra, Fin{rtol2, max_iter});
}

// A Newton trial point without an FFT.  S^-1 is linear, so with the CG's
// own quantities, S^-1 xi = H xi - D xi = (b - r) - D xi (b = -g the CG
// right-hand side, r its recursively updated residual), and at
// s' = s + tau xi:
//   y' = y + tau S^-1 xi,   D' = nbar w e^{s'},   g' = y' + D' - N.
// The increment carries the rounding of the CG fields relative to the
// current gradient only.  Writes the trial state to separate buffers (the
// line search may reject it) and the sums of EpiGrad, finalised by FinGrad.
// g null (only where T = TC): g = (y + D) - N is formed again from the
// fields read anyway, in the order and precision in which EpiGrad and this
// kernel form it, so it equals the stored value bit for bit; g2 null: not
// stored.  That saves 8 of the 48 B per cell of the FP32 phase.
template <typename T, typename TC>
__global__ void __launch_bounds__(kThreads)
k_newton_update(const T* __restrict__ s, const T* __restrict__ y, const T* __restrict__ g,
                const TC* __restrict__ r, const TC* __restrict__ xi, const TC* __restrict__ D,
                const int32_t* __restrict__ N, const double* __restrict__ w, double nbar,
                double mu, double tau_arg, const double* __restrict__ tau_dev, double c,
                int jac, T* __restrict__ s2,
                T* __restrict__ y2, T* __restrict__ g2, TC* __restrict__ D2,
                TC* __restrict__ r2, size_t n3, RedArgs ra) {
  using Acc = typename AccOf<T>::type;
  Acc acc[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) acc[j].init(false);
  const double tau = tau_dev ? *tau_dev : tau_arg;
  const T tt = (T)tau, nb = (T)nbar, m = (T)mu;
  const TC cc = (TC)c;
  const size_t step = (size_t)gridDim.x * blockDim.x * 4;
  for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4; i < n3; i += step) {
    const V4<TC> xv = ld4(xi + i), rv = ld4(r + i), dv = ld4(D + i);
    const V4<T> sv = ld4(s + i), yv = ld4(y + i);
    const V4<int32_t> nv = ld4(N + i);
    V4<T> gv;
    if (g) gv = ld4(g + i);
    V4<double> wv{{1.0, 1.0, 1.0, 1.0}};
    if (w) wv = ld4(w + i);
    V4<T> so, yo, go;
    V4<TC> dout, rout;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T g_j = g ? gv.v[j] : yv.v[j] + (T)dv.v[j] - (T)nv.v[j];
      const TC b_j = (TC)(-g_j);
      const TC sinv_xi = b_j - rv.v[j] - dv.v[j] * xv.v[j];
      const T yn = yv.v[j] + tt * (T)sinv_xi;
      const T sn = sv.v[j] + tt * (T)xv.v[j];
      const T d = nb * (T)wv.v[j] * exp(sn);
      const T ni = (T)nv.v[j];
      const T gn = yn + d - ni;
      so.v[j] = sn;
      yo.v[j] = yn;
      go.v[j] = gn;
      dout.v[j] = (TC)d;
      rout.v[j] = (TC)(-gn);
      acc[0].add((sn - m) * yn);
      acc[1].add(d - ni * sn);
      acc[2].add(gn * gn);
      const TC nc = (TC)nv.v[j], sc = (TC)sn;
      acc[3].add((T)(nc * sc));
      acc[4].add((T)(nc * (sc < (TC)0 ? -sc : sc)));
      const TC gc = (TC)gn;
      acc[5].add((T)(jac ? gc * jacobi(gc, (TC)d, cc) : gc * gc));
    }
    st4(s2 + i, so);
    st4(y2 + i, yo);
    if (g2) st4(g2 + i, go);
    st4(D2 + i, dout);
    st4(r2 + i, rout);
  }
  block_reduce_finish_acc<6, 0u>(acc, ra, FinGrad{});
}

// D = nbar w e^s (Sec. 3.1.2), from an FP64 s.
template <typename TC>
__global__ void __launch_bounds__(kThreads)
k_diag(const double* __restrict__ s, const double* __restrict__ w, double nbar,
       TC* __restrict__ D, size_t n3) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x)
    D[i] = (TC)(nbar * (w ? w[i] : 1.0) * exp(s[i]));
}

// Lambert W of x = e^L from L = ln x (x up to e^300 and beyond), in FP32:
// Newton's method on w + ln w = L, the defining equation w e^w = x in log
// form, from w = x / (1 + x) (L < 1) or w = L - ln L (L >= 1); four steps
// reach FP32 accuracy (fast division: the iteration corrects its rounding).
// L = -inf gives 0.
__device__ __forceinline__ float lambert_w_log(float L) {
  if (L == -INFINITY) return 0.f;
  float w;
  if (L < 1.f) {
    const float x = __expf(L);
    w = __fdividef(x, 1.f + x);
  } else {
    w = L - __logf(L);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) w = __fdividef(w * (1.f + L - __logf(w)), 1.f + w);
  return w;
}

// Per cell, the MAP of -ln P with S replaced by sigma2 I (Eq. MAPLNUB cell by
// cell): (s - mu) / sigma2 + nbar w e^s = N, s = mu + sigma2 N - W(x),
// x = sigma2 w nbar e^{mu + sigma2 N}.  A start point for the solve: the
// per-cell balance of prior and counts without the prior's correlations.
template <typename TS>
__global__ void __launch_bounds__(kThreads)
k_diag_start(TS* __restrict__ s, const int32_t* __restrict__ N, const double* __restrict__ w,
             float nbar, float mu, float sigma2, size_t n3) {
  const float lw0 = __logf(sigma2 * nbar);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const float a = mu + sigma2 * (float)N[i];
    const float wi = w ? (float)w[i] : 1.f;
    const float L = wi > 0.f ? lw0 + __logf(wi) + a : -INFINITY;
    s[i] = (TS)(a - lambert_w_log(L));
  }
}

// The same start for the Gaussian-prior model (Eq. MAPG cell by cell with
// S = sigma2 I): delta / sigma2 + nbar w - N / (1 + delta) = 0, i.e. with
// a = sigma2 nbar w, 1 + delta = (1 - a + sqrt((1 - a)^2 + 4 sigma2 N)) / 2
// for N > 0 (the root inside the domain; the rationalised form when
// 1 - a < 0) and delta = -a for N = 0 (no logarithm: a linear term).
template <typename TS>
__global__ void __launch_bounds__(kThreads)
k_diag_start_g(TS* __restrict__ delta, const int32_t* __restrict__ N,
               const double* __restrict__ w, float nbar, float sigma2, size_t n3) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const float a = sigma2 * nbar * (w ? (float)w[i] : 1.f);
    const int ni = N[i];
    float d;
    if (ni > 0) {
      const float q = 1.f - a, sn = 4.f * sigma2 * (float)ni;
      const float r = sqrtf(q * q + sn);
      const float u = q >= 0.f ? 0.5f * (q + r) : 0.5f * sn / (r - q);
      d = u - 1.f;
    } else {
      d = -a;
    }
    delta[i] = (TS)d;
  }
}

template <typename TD, typename TS>
__global__ void __launch_bounds__(kThreads)
k_convert(const TS* __restrict__ src, TD* __restrict__ dst, size_t n3) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (TD)src[i];
}

// Line-search trial of the Gaussian-prior model, without an FFT (as
// k_newton_update): delta' = delta + tau xi, y' = y + tau S^-1 xi with
// S^-1 xi = (b - r) - D xi from the CG, then g', D', r' and the sums.
template <typename T, typename TC>
__global__ void __launch_bounds__(kThreads)
k_newton_update_g(const T* __restrict__ s, const T* __restrict__ y, const T* __restrict__ g,
                  const TC* __restrict__ r, const TC* __restrict__ xi, const TC* __restrict__ D,
                  const int32_t* __restrict__ N, const double* __restrict__ w, double nbar,
                  double tau, double c, int jac, T* __restrict__ s2, T* __restrict__ y2,
                  T* __restrict__ g2, TC* __restrict__ D2, TC* __restrict__ r2, size_t n3,
                  RedArgs ra) {
  using Acc = typename AccOf<T>::type;
  Acc acc[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) acc[j].init(false);
  const T tt = (T)tau, nb = (T)nbar;
  const TC cc = (TC)c;
  const size_t step = (size_t)gridDim.x * blockDim.x * 4;
  for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4; i < n3; i += step) {
    const V4<TC> xv = ld4(xi + i), rv = ld4(r + i), dv = ld4(D + i);
    const V4<T> sv = ld4(s + i), yv = ld4(y + i), gv = ld4(g + i);
    const V4<int32_t> nv = ld4(N + i);
    V4<double> wv{{1.0, 1.0, 1.0, 1.0}};
    if (w) wv = ld4(w + i);
    V4<T> so, yo, go;
    V4<TC> dout, rout;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const TC sinv_xi = (TC)(-gv.v[j]) - rv.v[j] - dv.v[j] * xv.v[j];
      const T yn = yv.v[j] + tt * (T)sinv_xi;
      const T sn = sv.v[j] + tt * (T)xv.v[j];
      T gn, d;
      gauss_cell<T, TC>(sn, (T)wv.v[j], (T)nv.v[j], nb, yn, cc, jac, acc, gn, d);
      so.v[j] = sn;
      yo.v[j] = yn;
      go.v[j] = gn;
      dout.v[j] = (TC)d;
      rout.v[j] = (TC)(-gn);
    }
    st4(s2 + i, so);
    st4(y2 + i, yo);
    st4(g2 + i, go);
    st4(D2 + i, dout);
    st4(r2 + i, rout);
  }
  block_reduce_finish_acc<6, 0u>(acc, ra, FinGrad{});
}

// Fraction to the boundary of the Gaussian-prior model: the largest
// -xi / (1 + delta) over cells with N > 0 and xi < 0 (0 if none), so that
// any tau < 1 / that keeps 1 + delta + tau xi > 0 where the likelihood has
// its logarithm.  Stored in the device scalars' bmax.
template <typename T, typename TC>
__global__ void __launch_bounds__(kThreads)
k_boundary(const T* __restrict__ s, const TC* __restrict__ xi, const int32_t* __restrict__ N,
           size_t n3, RedArgs ra) {
  typename AccOf<T>::type acc[1];
  acc[0].init(true);
  const size_t step = (size_t)gridDim.x * blockDim.x * 4;
  for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4; i < n3; i += step) {
    const V4<T> sv = ld4(s + i);
    const V4<TC> xv = ld4(xi + i);
    const V4<int32_t> nv = ld4(N + i);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (nv.v[j] > 0 && xv.v[j] < (TC)0) acc[0].max((T)(-xv.v[j]) / ((T)1 + sv.v[j]));
  }
  struct Fin {
    __device__ void operator()(const double* t, DevScalars* sc) const {
      sc->bmax = t[0] > 0.0 ? t[0] : 0.0;
    }
  };
  block_reduce_finish_acc<1, 1u>(acc, ra, Fin{});
}

}  // namespace plc
