// ops.cuh -- pointwise parts of the Newton-Krylov MAP solve (Sec. 3.1, 3.1.2).
//
// Prologues (fused into the first FFT pass) produce the field to transform;
// epilogues (fused into the last pass) turn y = S^-1 x into the gradient or a
// Hessian-vector product and accumulate the dot products the solver needs;
// finalizers run once on the grid totals.  Element-wise kernels cover the CG
// recurrences, the line-search sums and set-up work.  All reductions are in
// FP64 whatever the field type.
#pragma once

#include "common.cuh"

namespace plc {

// ------------------------------- prologues --------------------------------
template <typename T> struct ProLoad {
  const T* x;
  __device__ T operator()(size_t i) const { return x[i]; }
};

// s - mu: the prior term of the gradient (Sec. 2.3, Eq. priorlog).
template <typename T> struct ProShift {
  const T* s;
  T mu;
  __device__ T operator()(size_t i) const { return s[i] - mu; }
};

// Newton update s <- s + tau xi (Sec. 3.1), then s - mu for the new gradient.
template <typename T, typename TX> struct ProStepShift {
  T* s;
  const TX* xi;
  double tau;
  T mu;
  __device__ T operator()(size_t i) const {
    const T sn = (T)((double)s[i] + tau * (double)xi[i]);
    s[i] = sn;
    return sn - mu;
  }
};

// CG search direction p <- M^-1 r + beta p (beta from the device scalars).
template <typename T, bool JAC> struct ProCgDir {
  const T* r;
  const T* D;
  T c;                 // (S^-1)_ii, the prior's share of diag(H)
  T* p;
  const DevScalars* sc;
  __device__ T operator()(size_t i) const {
    const T beta = (T)sc->beta;
    const T zi = JAC ? r[i] / (D[i] + c) : r[i];
    const T pn = beta == (T)0 ? zi : zi + beta * p[i];   // first step: p = z
    p[i] = pn;
    return pn;
  }
};

// ------------------------------- epilogues --------------------------------
template <typename T> struct EpiStore {
  static constexpr int NV = 0;
  static constexpr unsigned MAXMASK = 0;
  T* out;
  __device__ void operator()(size_t i, T y, double*) const { out[i] = y; }
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
  __device__ void operator()(size_t i, T y, double*) const {
    const T d = nbar * (w ? w[i] : (T)1) * exp(s[i]);
    out[i] = y + d * v[i];
  }
};

// CG product H p = S^-1 p + D p, accumulating p^T H p.
template <typename T> struct EpiHessD {
  static constexpr int NV = 1;
  static constexpr unsigned MAXMASK = 0;
  const T* D;
  const T* v;
  T* out;
  __device__ void operator()(size_t i, T y, double* acc) const {
    const T vi = v[i];
    const T hv = y + D[i] * vi;
    out[i] = hv;
    acc[0] += (double)vi * (double)hv;
  }
};

// Gradient g = S^-1 (s - mu) + nbar w e^s - N (Sec. 3.1.2) and the pieces of
// -ln P: acc = { sum (s-mu) y, sum (D - N s), sum g^2, sum N s, sum N |s| }.
template <typename T> struct EpiGrad {
  static constexpr int NV = 5;
  static constexpr unsigned MAXMASK = 0;
  const T* s;
  const T* w;
  const int32_t* N;
  T nbar, mu;
  T* g;                // may be null
  T* D;                // may be null
  float* D32;          // may be null: an FP32 copy of D for the mixed CG
  __device__ void operator()(size_t i, T y, double* acc) const {
    const T si = s[i];
    const T d = nbar * (w ? w[i] : (T)1) * exp(si);
    const T ni = (T)N[i];
    const T gi = y + d - ni;
    if (g) g[i] = gi;
    if (D) D[i] = d;
    if (D32) D32[i] = (float)d;
    acc[0] += (double)(si - mu) * (double)y;
    acc[1] += (double)d - (double)ni * (double)si;
    acc[2] += (double)gi * (double)gi;
    acc[3] += (double)ni * (double)si;
    acc[4] += (double)ni * fabs((double)si);
  }
};

// sum lam_i y_i, y = S^-1 x.
template <typename T, typename TL> struct EpiDot {
  static constexpr int NV = 1;
  static constexpr unsigned MAXMASK = 0;
  const TL* lam;
  __device__ void operator()(size_t i, T y, double* acc) const {
    acc[0] += (double)lam[i] * (double)y;
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

// alpha = r^T z / p^T H p; a non-positive curvature stops the CG.
struct FinAlpha {
  __device__ void operator()(const double* t, DevScalars* sc) const {
    sc->pHp = t[0];
    if (!(t[0] > 0.0)) {
      sc->breakdown = 1;
      sc->done = 1;
      sc->alpha = 0.0;
    } else {
      sc->alpha = sc->rz / t[0];
    }
  }
};

// ------------------------------ CG kernels --------------------------------
// Start CG on H x = b from x = 0: r = b (or -b), rz = r^T M^-1 r, rr = r^T r.
template <typename TC, typename TB, bool JAC>
__global__ void __launch_bounds__(kThreads)
k_cg_init(const TB* __restrict__ b, int negate, const TC* __restrict__ D, TC c,
          TC* __restrict__ r, TC* __restrict__ x, size_t n3, RedArgs ra,
          double rtol2, int max_iter) {
  double acc[2] = {0.0, 0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const TC ri = negate ? (TC)(-b[i]) : (TC)b[i];
    r[i] = ri;
    x[i] = (TC)0;
    const TC zi = JAC ? ri / (D[i] + c) : ri;
    acc[0] += (double)ri * (double)zi;
    acc[1] += (double)ri * (double)ri;
  }
  struct Fin {
    double rtol2; int max_iter;
    __device__ void operator()(const double* t, DevScalars* sc) const {
      sc->rz = t[0];
      sc->rr = t[1];
      sc->bnorm2 = t[1];
      sc->rtol2 = rtol2;
      sc->iter = 0;
      sc->max_iter = max_iter;
      sc->beta = 0.0;
      sc->alpha = 0.0;
      sc->breakdown = 0;
      sc->done = (t[1] <= 0.0 || max_iter <= 0) ? 1 : 0;
    }
  };
  block_reduce_finish<2, 0u>(acc, ra, Fin{rtol2, max_iter});
}

// x += alpha p, r -= alpha H p, then r^T M^-1 r and ||r||^2 for beta and the
// stopping test ||r||^2 <= rtol^2 ||b||^2.
template <typename TC, bool JAC>
__global__ void __launch_bounds__(kThreads)
k_cg_update(TC* __restrict__ x, TC* __restrict__ r, const TC* __restrict__ p,
            const TC* __restrict__ Hp, const TC* __restrict__ D, TC c, size_t n3,
            RedArgs ra) {
  if (ra.sc->done) return;
  const TC alpha = (TC)ra.sc->alpha;
  double acc[2] = {0.0, 0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const TC ri = r[i] - alpha * Hp[i];
    r[i] = ri;
    const TC zi = JAC ? ri / (D[i] + c) : ri;
    acc[0] += (double)ri * (double)zi;
    acc[1] += (double)ri * (double)ri;
  }
  struct Fin {
    __device__ void operator()(const double* t, DevScalars* sc) const {
      sc->beta = t[0] / sc->rz;
      sc->rz = t[0];
      sc->rr = t[1];
      sc->iter += 1;
      if (t[1] <= sc->rtol2 * sc->bnorm2 || sc->iter >= sc->max_iter) sc->done = 1;
    }
  };
  block_reduce_finish<2, 0u>(acc, ra, Fin{});
}

// Sums for the step length of Eq. (New5) and the line-search model:
// { xi.g, xi.r, sum D xi^2, xi.D, xi.N, max |xi| }.
template <typename TC, typename TG>
__global__ void __launch_bounds__(kThreads)
k_dirstats(const TC* __restrict__ xi, const TG* __restrict__ g, const TC* __restrict__ r,
           const TG* __restrict__ D, const int32_t* __restrict__ N, size_t n3, RedArgs ra) {
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, -INFINITY};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const double x = (double)xi[i], d = (double)D[i];
    acc[0] += x * (double)g[i];
    acc[1] += x * (double)r[i];
    acc[2] += d * x * x;
    acc[3] += x * d;
    acc[4] += x * (double)N[i];
    acc[5] = fmax(acc[5], fabs(x));
  }
  block_reduce_finish<6, 1u << 5>(acc, ra, FinStore<6>{});
}

// Likelihood part of the line search: sum_i D_i exp(tau xi_i).
template <typename TC, typename TG>
__global__ void __launch_bounds__(kThreads)
k_trial(const TC* __restrict__ xi, const TG* __restrict__ D, double tau, size_t n3, RedArgs ra) {
  double acc[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x)
    acc[0] += (double)D[i] * exp(tau * (double)xi[i]);
  block_reduce_finish<1, 0u>(acc, ra, FinStore<1>{});
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

template <typename TD, typename TS>
__global__ void __launch_bounds__(kThreads)
k_convert(const TS* __restrict__ src, TD* __restrict__ dst, size_t n3) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (TD)src[i];
}

}  // namespace plc
