// common.cuh -- shared device building blocks of libplc (sm_103a).
//
// * complex arithmetic on float2 / double2;
// * the radix-2/3/4/8 DFT butterflies and one Stockham autosort stage for a
//   batch of lines held in shared memory (the 3D FFT of the prior operator,
//   Sec. 2.2: S is a convolution, applied through FFTs as in Sec. 3);
// * a deterministic grid-wide reduction: warp shuffles, a per-block partial,
//   and a fixed-order final sum by the last block to finish.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace plc {

constexpr int kThreads = 256;          // threads per block (element-wise kernels and n <= 256)
constexpr int kMaxStages = 12;
constexpr int kMaxRed = 8;             // values per reduction

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cpx = typename CplxOf<T>::type;

// Lines per shared-memory tile: 128 bytes of complex values per tile row.
template <typename T> struct Tile { static constexpr int L = 128 / (2 * (int)sizeof(T)); };

// Division by a runtime divisor d >= 1 as one multiply-high:
// q = umulhi(x, m) with m = ceil(2^32 / d) equals floor(x / d) whenever
// x * d < 2^32 (here x < 2^16 and d <= 512).  d = 1 has no 32-bit m and is
// passed through.
struct FastDiv {
  unsigned d, m;
};
inline __host__ __device__ FastDiv make_fastdiv(unsigned d) {
  return FastDiv{d, d > 1 ? (unsigned)((0x100000000ull + d - 1) / d) : 0u};
}
__device__ __forceinline__ unsigned fdiv(unsigned x, FastDiv f) {
  return f.d > 1 ? __umulhi(x, f.m) : x;
}

struct FftPlan {
  int n;                     // transform length (the grid side)
  int nst;                   // number of radix stages
  int rad[kMaxStages];       // radix of each stage (2, 3, 4 or 8)
  int ns[kMaxStages];        // product of the radices before each stage
  int tstep[kMaxStages];     // twiddle index step n / (ns * rad)
  unsigned ns_m[kMaxStages]; // fast-division multiplier for ns (0 when ns = 1)
  FastDiv nd;                // division by n
  int f1, f2;                // FP32 register four-step factors n = f1 f2
                             // (0 = the Stockham stages)
};

// Device-resident scalars of the solver (one instance per context).
struct DevScalars {
  double red[kMaxRed];       // results of the last reduction
  double rz;                 // r^T M^-1 r
  double alpha, beta;
  double rr;                 // ||r||^2
  double bnorm2;             // ||b||^2 of the current CG solve
  double pHp;
  double xb;                 // xi^T b accumulated over the CG steps
  double xHx;                // xi^T H xi accumulated over the CG steps
  double xmax;               // max |xi| after the last CG step
  int iter;                  // CG iterations of the current solve
  int done, breakdown;
  unsigned ticket;           // last-block-done counter
  // CG stopping parameters set on the device (device-driven solve): used by
  // the CG update when it is launched with rtol2 < 0
  double rtol2;
  int max_iter;
  // step length of the next Newton trial (device-driven solve)
  double tau;
  // fraction-to-boundary quantity of the Gaussian-prior model (k_boundary)
  double bmax;
  // k_g0_at_mean: 1 when the start point differs from the prior mean somewhere
  int off_mean;
};

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return cmk<C>(a.x * s, a.y * s); }
// multiply by SIGN * i
template <int SIGN, typename C> __device__ __forceinline__ C cmul_si(C a) {
  return SIGN > 0 ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Small DFTs X_k = sum_j v_j exp(SIGN 2 pi i j k / R) on registers.
// ---------------------------------------------------------------------------
template <typename T, int SIGN> struct Dft {
  using C = cpx<T>;
  static __device__ __forceinline__ void r2(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  }
  static __device__ __forceinline__ void r3(C* v) {
    const T h = (T)0.86602540378443864676;   // sin(2 pi / 3)
    C s = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C m = cmk<C>(v[0].x - (T)0.5 * s.x, v[0].y - (T)0.5 * s.y);
    C t = cmul_si<SIGN>(cscale(d, h));
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, t);
    v[2] = csub(m, t);
  }
  static __device__ __forceinline__ void r4(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = cmul_si<SIGN>(csub(v[1], v[3]));
    v[0] = cadd(a, c); v[2] = csub(a, c);
    v[1] = cadd(b, d); v[3] = csub(b, d);
  }
  static __device__ __forceinline__ void r8(C* v) {
    const T q = (T)0.70710678118654752440;    // 1/sqrt(2)
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    r4(e); r4(o);
    // o_k *= exp(SIGN 2 pi i k / 8)
    C o1 = cmk<C>(q * (o[1].x - SIGN * o[1].y), q * (o[1].y + SIGN * o[1].x));
    C o2 = cmul_si<SIGN>(o[2]);
    C o3 = cmk<C>(q * (-o[3].x - SIGN * o[3].y), q * (-o[3].y + SIGN * o[3].x));
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
};

// One Stockham autosort stage of radix R on `nl` lines of length N held in
// shared memory; element i of line c lives at buf[i * P + c].  Ns is the
// product of the radices already applied.  Butterfly j of a line reads
// elements j + r N/R, twiddles them by W_{Ns R}^{r k} (k = j mod Ns), and
// writes elements (j - k) R + k + r Ns.  tw[m] = exp(-2 pi i m / N).
template <typename T, int R, int SIGN, int L>
__device__ __forceinline__ void stockham_stage(const cpx<T>* __restrict__ in,
                                               cpx<T>* __restrict__ out, int N,
                                               int Ns, unsigned ns_m, int tstep, int nl, int P,
                                               const cpx<T>* __restrict__ tw) {
  using C = cpx<T>;
  const int NR = N / R;
  const int total = L * NR;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int c = b % L;
    const int j = b / L;
    if (c >= nl) continue;
    const int k = ns_m ? j - (int)__umulhi((unsigned)j, ns_m) * Ns : 0;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[(j + r * NR) * P + c];
    if (k != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * tstep];
        if (SIGN > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    if (R == 2) Dft<T, SIGN>::r2(v);
    if (R == 3) Dft<T, SIGN>::r3(v);
    if (R == 4) Dft<T, SIGN>::r4(v);
    if (R == 8) Dft<T, SIGN>::r8(v);
    const int d = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[(d + r * Ns) * P + c] = v[r];
  }
}

// Full length-N transform of `nl` (<= L) lines, ping-ponging between two
// buffers.  On return `a` points at the result and `b` at the free buffer.
// Must be entered after a __syncthreads() that publishes the data; ends with
// one.
template <typename T, int SIGN, int L>
__device__ __forceinline__ void fft_lines(cpx<T>*& a, cpx<T>*& b, const FftPlan& plan,
                                          int nl, int P, const cpx<T>* tw) {
  const int N = plan.n;
  for (int s = 0; s < plan.nst; ++s) {
    const int R = plan.rad[s], Ns = plan.ns[s], ts = plan.tstep[s];
    const unsigned m = plan.ns_m[s];
    if (R == 8) stockham_stage<T, 8, SIGN, L>(a, b, N, Ns, m, ts, nl, P, tw);
    else if (R == 4) stockham_stage<T, 4, SIGN, L>(a, b, N, Ns, m, ts, nl, P, tw);
    else if (R == 2) stockham_stage<T, 2, SIGN, L>(a, b, N, Ns, m, ts, nl, P, tw);
    else stockham_stage<T, 3, SIGN, L>(a, b, N, Ns, m, ts, nl, P, tw);
    __syncthreads();
    cpx<T>* t = a; a = b; b = t;
  }
}

// ---------------------------------------------------------------------------
// Register-resident small DFTs (the building blocks of the four-step line
// transforms in passes4.cuh).
//
// exp(2 pi i m / R) for the radices used in registers (R in {2,3,4,6,8,12,16});
// after unrolling m and R are constants and the switch folds away.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double unit_cos(int R, int m) {
  const double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173;
  const double h = 0.70710678118654752440, t = 0.86602540378443864676;
  if (R == 16) {
    switch (m & 15) {
      case 0: return 1.0; case 1: return c1; case 2: return h; case 3: return s1;
      case 4: return 0.0; case 5: return -s1; case 6: return -h; case 7: return -c1;
      case 8: return -1.0; case 9: return -c1; case 10: return -h; case 11: return -s1;
      case 12: return 0.0; case 13: return s1; case 14: return h; default: return c1;
    }
  }
  if (R == 12) {
    switch (m % 12) {
      case 0: return 1.0; case 1: return t; case 2: return 0.5; case 3: return 0.0;
      case 4: return -0.5; case 5: return -t; case 6: return -1.0; case 7: return -t;
      case 8: return -0.5; case 9: return 0.0; case 10: return 0.5; default: return t;
    }
  }
  if (R == 8) return unit_cos(16, 2 * m);
  if (R == 6) return unit_cos(12, 2 * m);
  if (R == 4) return unit_cos(16, 4 * m);
  if (R == 3) return unit_cos(12, 4 * m);
  return (m & 1) ? -1.0 : 1.0;   // R == 2
}
__device__ __forceinline__ double unit_sin(int R, int m) {
  // sin(2 pi m / R) = cos(2 pi (m - R/4) / R) for R divisible by 4; the
  // radices 6 and 3 go through 12
  if (R == 6) return unit_sin(12, 2 * m);
  if (R == 3) return unit_sin(12, 4 * m);
  if (R == 2) return 0.0;
  return unit_cos(R, ((m - R / 4) % R + R) % R);
}

// a * exp(SIGN 2 pi i m / R)
template <typename T, int SIGN>
__device__ __forceinline__ cpx<T> rot(cpx<T> a, int R, int m) {
  using C = cpx<T>;
  m %= R;
  if (m == 0) return a;
  if (4 * m == R) return cmul_si<SIGN>(a);
  if (2 * m == R) return cmk<C>(-a.x, -a.y);
  if (4 * m == 3 * R) return cmul_si<-SIGN>(a);
  const T c = (T)unit_cos(R, m), sn = (T)SIGN * (T)unit_sin(R, m);
  return cmk<C>(a.x * c - a.y * sn, a.x * sn + a.y * c);
}

// In-register DFT of length R (natural order in and out).  R = 6, 12, 16 are
// done four-step as R1 x R2 (2x3, 3x4, 4x4).
template <typename T, int SIGN, int R>
__device__ __forceinline__ void dft_small(cpx<T>* v) {
  using C = cpx<T>;
  if constexpr (R == 2) Dft<T, SIGN>::r2(v);
  else if constexpr (R == 3) Dft<T, SIGN>::r3(v);
  else if constexpr (R == 4) Dft<T, SIGN>::r4(v);
  else if constexpr (R == 8) Dft<T, SIGN>::r8(v);
  else {
    constexpr int R1 = (R == 6) ? 2 : (R == 12 ? 3 : 4);
    constexpr int R2 = R / R1;
    C y[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      C a[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[R2 * n1 + n2];
      dft_small<T, SIGN, R1>(a);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) y[k1 * R2 + n2] = rot<T, SIGN>(a[k1], R, n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C b[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) b[n2] = y[k1 * R2 + n2];
      dft_small<T, SIGN, R2>(b);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
    }
  }
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async): every thread issues all of
// its copies before waiting, so a tile's loads are all in flight at once
// without passing through registers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async(float2* smem, const float2* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async(double2* smem, const double2* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Hint to bring [p, p + bytes) into L2 ahead of use: one TMA bulk prefetch,
// nothing to wait for.  p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// Per-thread accumulators.  Element-wise terms are formed and summed in the
// field precision: plain FP64 for double fields, Kahan-compensated FP32 for
// float fields (about one FP32 rounding of relative error, and no FP64
// arithmetic per element, which runs at a small fraction of the FP32 rate).
// Across threads and blocks the sums continue in FP64.
// ---------------------------------------------------------------------------
// Per-thread accumulators.  Besides add/max, each can merge another one of
// its kind (merge) and move across lanes (shfl_down), so that a block
// reduces them in their own arithmetic: GB300's FP64 rate is 1/64 of FP32,
// and FP64 adds in the warp reductions of FP32 kernels cost several
// microseconds per launch.
struct AccD {
  double v;
  __device__ __forceinline__ void init(bool is_max) { v = is_max ? -INFINITY : 0.0; }
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void max(double x) { v = fmax(v, x); }
  __device__ __forceinline__ double get() const { return v; }
  __device__ __forceinline__ void merge(const AccD& o, bool is_max) {
    v = is_max ? fmax(v, o.v) : v + o.v;
  }
  __device__ __forceinline__ AccD shfl_down(int o) const {
    return AccD{__shfl_down_sync(0xffffffffu, v, o)};
  }
};
// Kahan-compensated FP32 sum: value s - c.
struct AccK {
  float s, c;
  __device__ __forceinline__ void init(bool is_max) { s = is_max ? -INFINITY : 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ void max(float x) { s = fmaxf(s, x); }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
  // (s1 - c1) + (s2 - c2): the high parts by TwoSum (Knuth), the rounding
  // error folded into the compensation
  __device__ __forceinline__ void merge(const AccK& o, bool is_max) {
    if (is_max) {
      s = fmaxf(s, o.s);
      return;
    }
    const float t = s + o.s;
    const float bb = t - s;
    const float e = (s - (t - bb)) + (o.s - bb);
    c = (c + o.c) - e;
    s = t;
  }
  __device__ __forceinline__ AccK shfl_down(int o) const {
    return AccK{__shfl_down_sync(0xffffffffu, s, o), __shfl_down_sync(0xffffffffu, c, o)};
  }
};
template <typename T> struct AccOf;
template <> struct AccOf<double> { using type = AccD; };
template <> struct AccOf<float> { using type = AccK; };

// ---------------------------------------------------------------------------
// Deterministic grid reduction.  Every block calls block_reduce_finish with
// its per-thread accumulators; the last block to arrive sums the per-block
// partials in block order and calls fin(totals, scalars) on thread 0.
// ---------------------------------------------------------------------------
struct RedArgs {
  double* partials;          // [gridDim.x * gridDim.y * gridDim.z][kMaxRed]
  DevScalars* sc;
};

// MAXMASK bit j set: value j is reduced with max, otherwise with +.
template <unsigned MAXMASK>
__device__ __forceinline__ double red_op(int j, double a, double b) {
  return ((MAXMASK >> j) & 1u) ? fmax(a, b) : a + b;
}
template <unsigned MAXMASK>
__device__ __forceinline__ double red_identity(int j) {
  return ((MAXMASK >> j) & 1u) ? -INFINITY : 0.0;
}

template <int NV, unsigned MAXMASK>
__device__ __forceinline__ void warp_reduce(double* v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = red_op<MAXMASK>(j, v[j], __shfl_down_sync(0xffffffffu, v[j], o));
  }
}

// Reduce v[NV] over the block in a fixed order; thread 0 gets the result.
template <int NV, unsigned MAXMASK>
__device__ __forceinline__ void block_reduce(double* v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  warp_reduce<NV, MAXMASK>(v);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[warp * NV + j] = v[j];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = lane < nw ? sh[lane * NV + j] : red_identity<MAXMASK>(j);
    warp_reduce<NV, MAXMASK>(v);
  }
  __syncthreads();
}

// The grid reduction behind block_reduce_finish: v (thread 0's block
// totals) to the partials; the last block sums them in block order.
template <int NV, unsigned MAXMASK, typename Fin>
__device__ __forceinline__ void grid_finish(double* v, const RedArgs& ra, Fin fin, double* sh) {
  __shared__ int is_last;
  const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) ra.partials[(size_t)bid * kMaxRed + j] = v[j];
    __threadfence();
    unsigned t = atomicAdd(&ra.sc->ticket, 1u);
    is_last = (t == nblocks - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = red_identity<MAXMASK>(j);
  // U partials per thread loaded before they are summed (in the same
  // order, b = tid, tid + blockDim, ...), so that the last block waits for
  // about one L2 round trip per U instead of one per partial: this runs
  // while the rest of the GPU waits for the kernel to end
  constexpr int U = NV <= 1 ? 8 : (NV <= 3 ? 4 : 2);
  for (unsigned b0 = threadIdx.x; b0 < nblocks; b0 += U * blockDim.x) {
    double t[U][NV];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned b = b0 + u * blockDim.x;
#pragma unroll
      for (int j = 0; j < NV; ++j)
        t[u][j] = b < nblocks ? __ldcg(ra.partials + (size_t)b * kMaxRed + j) : red_identity<MAXMASK>(j);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < NV; ++j) acc[j] = red_op<MAXMASK>(j, acc[j], t[u][j]);
  }
  block_reduce<NV, MAXMASK>(acc, sh);
  if (threadIdx.x == 0) {
    fin(acc, ra.sc);
    ra.sc->ticket = 0u;
    __threadfence();
  }
}

// Deterministic grid reduction of per-thread FP64 values v[NV].
template <int NV, unsigned MAXMASK, typename Fin>
__device__ __forceinline__ void block_reduce_finish(double* v, const RedArgs& ra, Fin fin) {
  __shared__ double sh[32 * kMaxRed];
  block_reduce<NV, MAXMASK>(v, sh);
  grid_finish<NV, MAXMASK>(v, ra, fin, sh);
}

// The same from per-thread accumulators: lanes and warps are merged in the
// accumulators' own arithmetic in a fixed order, and each block's totals
// go to FP64 once.
template <int NV, unsigned MAXMASK, typename Acc, typename Fin>
__device__ __forceinline__ void block_reduce_finish_acc(Acc* a, const RedArgs& ra, Fin fin) {
  __shared__ Acc sa[32 * kMaxRed];
  __shared__ double sh[32 * kMaxRed];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < NV; ++j) a[j].merge(a[j].shfl_down(o), (MAXMASK >> j) & 1u);
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sa[warp * NV + j] = a[j];
  __syncthreads();
  double v[NV];
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      if (lane < nw) a[j] = sa[lane * NV + j];
      else a[j].init((MAXMASK >> j) & 1u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < NV; ++j) a[j].merge(a[j].shfl_down(o), (MAXMASK >> j) & 1u);
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = a[j].get();
  __syncthreads();
  grid_finish<NV, MAXMASK>(v, ra, fin, sh);
}

// Grid size for element-wise kernels: a fixed multiple of the SM count so
// that reductions are reproducible for a given problem size.  per_sm = 4 is
// one wave of a kernel that fits 4 blocks per SM.
inline int pointwise_blocks(long long nelem, int sms, int per_sm = 8) {
  long long want = (nelem + kThreads * 4 - 1) / (kThreads * 4);
  long long cap = (long long)sms * per_sm;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace plc
