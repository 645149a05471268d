// passes4.cuh -- the five FP32 passes of S^-1 (Sec. 2.2) with the line
// transforms done four-step straight out of and into registers.
//
// Same pipeline and global layouts as passes.cuh (XF -> A[z][kx][y] -> YF ->
// B[kx][ky][z] -> Z -> YI -> A -> XI), for n = N1 N2 with (N1, N2) in
// {(16,16), (16,12), (16,8), (12,8), (8,8), (8,4)}.  A line of length N is
// transformed in two register phases joined by one shared-memory exchange:
//
//   forward  Z[k1 + N1 k2] = sum_n2 W_N2^{n2 k2} W_N^{n2 k1}
//                                   sum_n1 W_N1^{n1 k1} x[N2 n1 + n2]
//     phase A, task (line c, n2): DFT_N1 of x[N2 n1 + n2] over n1, twiddle
//     phase B, task (line c, k1): DFT_N2 over n2 -> Z[k1 + N1 k2]
//   inverse  x[N2 n1 + n2] = sum_k1 W_N1^{-n1 k1} W_N^{-n2 k1}
//                                   sum_k2 W_N2^{-n2 k2} Z[k1 + N1 k2]
//     phase B' (c, k1): inverse DFT_N2 over k2, conjugate twiddle
//     phase A' (c, n2): inverse DFT_N1 over k1 -> x[N2 n1 + n2]
//
// Each phase reads or writes global memory directly from the registers of
// its task, choosing the lane order that makes the access coalesced: a
// phase that walks a line along its own (contiguous) axis puts n2 (or its
// position) on consecutive lanes; a phase that writes the line index as the
// contiguous axis (B[kx][ky][z] seen from the y pass) puts the line c on
// consecutive lanes.  The exchange buffer X[c][k1 N2 + n2] has an odd pitch
// N + 1 so that both lane orders are free of bank conflicts, and the
// twiddles sit in shared memory as tw2[k1 N2 + n2] = W_N^{k1 n2}.
//
// The x passes pack two real rows as one complex line.  Their phase B (XF)
// and B' (XI) run as pairs of tasks k1 and N1 - k1 on the two half-warps of
// one warp, which hold the partner frequencies N - k of each other's k, so
// the real-to-complex split and its inverse take a warp shuffle instead of
// another trip through shared memory.  The prologue and epilogue see rows in
// natural order through a staging buffer of real rows (pitch N + 8), so they
// keep their 16-byte vector accesses.
//
// T is the arithmetic of the transforms: float (the FP32 operators and the
// FP32 phase of the solve) or ff, float-float on the FP32 pipes (ff.cuh),
// for the FP64 gradient of the mixed solve.
#pragma once

#include "ff.cuh"
#include "ops.cuh"
#include "passes.cuh"

namespace plc {

template <typename T, int N1_, int N2_> struct Geo4 {
  using C = cpx<T>;
  static constexpr int N1 = N1_, N2 = N2_, N = N1 * N2;
  static constexpr int L = 16;            // lines per block
  static constexpr int S = N + 1;         // pitch of the exchange buffer (complex)
  static constexpr int RY = 2 * L;        // real rows per x-pass block
  static constexpr int SR = N + 8;        // pitch of the real-row staging (reals)
  static constexpr size_t tw_bytes = sizeof(C) * N;
  static constexpr size_t x_bytes = sizeof(C) * L * S;
  static constexpr size_t r_bytes = sizeof(T) * RY * SR;
  // Z multipliers Ms[c][|mz|], |mz| <= N/2: pitch N/2 + 1 (odd) for 8-byte
  // reals, N/2 + 2 (twice an odd number for N a multiple of 8) for floats, so
  // that the lines c of both half-warps of a phase-B warp (which differ by
  // one in |mz|) fall in distinct banks
  static constexpr int MP = sizeof(T) == 4 ? N / 2 + 2 : N / 2 + 1;
  static constexpr size_t m_bytes = sizeof(T) * L * MP;
  static constexpr size_t smem_y = tw_bytes + x_bytes;
  static constexpr size_t smem_z = tw_bytes + x_bytes + m_bytes;
  static constexpr size_t smem_x = tw_bytes + (x_bytes > r_bytes ? x_bytes : r_bytes);
  static_assert(L * N2 <= kThreads, "one phase-A task per thread at most");
  static_assert(N1 / 2 <= kThreads / 32, "one warp per pair of x-pass tasks");
};

// tw2[k1 N2 + n2] = W_N^{k1 n2} from the natural table tw[m] = W_N^m.
template <typename C, int N1, int N2>
__device__ __forceinline__ void load_tw2(C* tw2, const C* __restrict__ twg) {
  for (int i = threadIdx.x; i < N1 * N2; i += blockDim.x) tw2[i] = twg[(i / N2) * (i % N2)];
}

// Phase A: DFT_N1 over n1 (sign SIGN), then twiddle by W_N^{SIGN-conjugated n2 k1}.
template <typename T, int N1, int N2, int SIGN>
__device__ __forceinline__ void phase_a(cpx<T>* v, const cpx<T>* tw2, int n2) {
  dft_small<T, SIGN, N1>(v);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) {
    cpx<T> w = tw2[k1 * N2 + n2];
    if (SIGN > 0) w.y = -w.y;
    v[k1] = cmul(v[k1], w);
  }
}

// Phase B': inverse DFT_N2 over k2, then the conjugate twiddle W_N^{-n2 k1}.
template <typename T, int N1, int N2>
__device__ __forceinline__ void phase_b_inv(cpx<T>* v, const cpx<T>* tw2, int k1) {
  dft_small<T, +1, N2>(v);
#pragma unroll
  for (int n2 = 1; n2 < N2; ++n2) {
    cpx<T> w = tw2[k1 * N2 + n2];
    w.y = -w.y;
    v[n2] = cmul(v[n2], w);
  }
}

#define PLC_PASS4_SETUP(SMEM_TAIL)                                      \
  using Gm = Geo4<T, N1, N2>;                                           \
  using C = cpx<T>;                                                     \
  constexpr int N = Gm::N;                                              \
  if (done && *done) return;                                            \
  extern __shared__ __align__(16) unsigned char smem_raw[];             \
  C* tw2 = reinterpret_cast<C*>(smem_raw);                              \
  SMEM_TAIL

#define PLC_PASS4_PROLOGUE(SMEM_TAIL)                                   \
  PLC_PASS4_SETUP(SMEM_TAIL);                                           \
  load_tw2<C, N1, N2>(tw2, twg);                                        \
  __syncthreads()

// ---------------------------------------------------------------------------
// YF: c2c along y.  grid = (n / 16, n/2+1); block (zb, kx) owns the lines
// A[z0 + c][kx][:] and writes B[kx][:][z0 + c].  As in the z and y-inverse
// passes, a phase whose tasks match the threads one to one is compiled
// without its guard or task loop.
// ---------------------------------------------------------------------------
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(kThreads)
k4_yf(const cpx<T>* __restrict__ A, cpx<T>* __restrict__ B, const cpx<T>* __restrict__ twg,
      const int* __restrict__ done) {
  PLC_PASS4_SETUP(C* X = tw2 + N);
  const int h = N / 2 + 1, z0 = blockIdx.x * Gm::L, kx = blockIdx.y;
  const bool task_a = Gm::L * N2 == kThreads || threadIdx.x < Gm::L * N2;
  const int n2 = threadIdx.x % N2, c = threadIdx.x / N2;
  // the lines are loaded before the twiddle table, so that the two loads
  // overlap instead of waiting one after the other at its barrier
  C v[N1];
  if (task_a) {
    const C* src = A + ((size_t)(z0 + c) * h + kx) * N + n2;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) v[n1] = src[N2 * n1];
  }
  load_tw2<C, N1, N2>(tw2, twg);
  __syncthreads();
  if (task_a) {
    phase_a<T, N1, N2, -1>(v, tw2, n2);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) X[c * Gm::S + k1 * N2 + n2] = v[k1];
  }
  __syncthreads();
  auto task_b = [&](int t) {
    const int c = t % Gm::L, k1 = t / Gm::L;
    C v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = X[c * Gm::S + k1 * N2 + n2];
    dft_small<T, -1, N2>(v);
    C* dst = B + ((size_t)kx * N + k1) * N + z0 + c;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) dst[(size_t)N1 * k2 * N] = v[k2];
  };
  if constexpr (Gm::L * N1 == kThreads) {
    task_b(threadIdx.x);
  } else {
    for (int t = threadIdx.x; t < Gm::L * N1; t += kThreads) task_b(t);
  }
}

// A multiplier of the z pass in the transform arithmetic (float, or
// float-float split from the FP64 table without the FP64 pipe).
__device__ __forceinline__ float as_mult(float m, float) { return m; }
__device__ __forceinline__ ff as_mult(double m, ff) { return ff_split(m); }

// Resident blocks per SM asked of the compiler for the z pass.  FP32 at
// 16 x 16: three blocks (up to 85 registers, it takes 69) ran the pass at
// 256^3 in 32.8 us against 36.9 us at four blocks of 59 registers on
// L2-resident data, and in 36.8 against 38.9 us inside the solve, with
// identical results; the more registers let it keep more loads in flight.
// Elsewhere 0, which leaves the register budget to the compiler as a bound
// without a block count does (a count of 1 changes it).
template <typename T, int N1, int N2> struct ZMinBlocks { static constexpr int value = 0; };
template <> struct ZMinBlocks<float, 16, 16> { static constexpr int value = 3; };

// ---------------------------------------------------------------------------
// Z: forward c2c along z, times M[|m|^2] = 1/(lambda_k n^3), inverse c2c,
// in place.  grid = (n / 16, n/2+1); block (kyb, kx) owns B[kx][ky0 + c][:].
// The spectrum of each phase-B task stays in registers between the two
// transforms.  zero_dc drops the DC mode.  Where every thread holds exactly
// one task of each phase (L N1 = L N2 = kThreads) the guards and the task
// loop are compiled out.
// ---------------------------------------------------------------------------
template <typename T, int N1, int N2, typename TM>
__global__ void __launch_bounds__(kThreads, ZMinBlocks<T, N1, N2>::value)
k4_z(cpx<T>* __restrict__ B, const TM* __restrict__ M, int zero_dc,
     const cpx<T>* __restrict__ twg, const int* __restrict__ done) {
  PLC_PASS4_PROLOGUE(C* X = tw2 + N; T* Ms = reinterpret_cast<T*>(X + Gm::L * Gm::S));
  // planes in decreasing kx: the y-forward pass before it writes them in
  // increasing kx, so the most recently written (most likely still in L2)
  // are read first
  const int ky0 = blockIdx.x * Gm::L, kx = N / 2 - blockIdx.y;
  C* line0 = B + ((size_t)kx * N + ky0) * N;
  constexpr bool kOneA = Gm::L * N2 == kThreads, kOneB = Gm::L * N1 == kThreads;
  const bool task_a = kOneA || threadIdx.x < Gm::L * N2;
  const int n2a = threadIdx.x % N2, ca = threadIdx.x / N2;
  C v[N1 > N2 ? N1 : N2];
  if (task_a) {
    const C* src = line0 + (size_t)ca * N + n2a;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) v[n1] = src[N2 * n1];
  }
  // while the lines load: the block's multipliers Ms[c][|mz|] =
  // M[kx^2 + my^2 + mz^2], gathered from the L2-resident table
  constexpr int HM = N / 2 + 1, MI = (Gm::L * HM + kThreads - 1) / kThreads, MP = Gm::MP;
  T mv[MI];
#pragma unroll
  for (int j = 0; j < MI; ++j) {
    const int i = threadIdx.x + j * kThreads;
    const int c = i / HM, mz = i - c * HM;
    const int ky = ky0 + c, my = min(ky, N - ky);
    const int m2 = kx * kx + my * my + mz * mz;
    mv[j] = (i >= Gm::L * HM || (zero_dc && m2 == 0)) ? as_mult(TM(0), T())
                                                       : as_mult(__ldg(M + m2), T());
  }
#pragma unroll
  for (int j = 0; j < MI; ++j) {
    const int i = threadIdx.x + j * kThreads;
    if (i < Gm::L * HM) Ms[(i / HM) * MP + i % HM] = mv[j];
  }
  if (task_a) {
    phase_a<T, N1, N2, -1>(v, tw2, n2a);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) X[ca * Gm::S + k1 * N2 + n2a] = v[k1];
  }
  __syncthreads();
  auto task_b = [&](int t) {
    const int c = t % Gm::L, k1 = t / Gm::L;
    C u[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) u[n2] = X[c * Gm::S + k1 * N2 + n2];
    dft_small<T, -1, N2>(u);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int kz = k1 + N1 * k2, mz = min(kz, N - kz);
      u[k2] = cscale(u[k2], Ms[c * MP + mz]);
    }
    phase_b_inv<T, N1, N2>(u, tw2, k1);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) X[c * Gm::S + k1 * N2 + n2] = u[n2];
  };
  if constexpr (kOneB) {
    task_b(threadIdx.x);
  } else {
    for (int t = threadIdx.x; t < Gm::L * N1; t += kThreads) task_b(t);
  }
  __syncthreads();
  if (task_a) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = X[ca * Gm::S + k1 * N2 + n2a];
    dft_small<T, +1, N1>(v);
    C* dst = line0 + (size_t)ca * N + n2a;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) dst[N2 * n1] = v[n1];
  }
}

// ---------------------------------------------------------------------------
// YI: inverse c2c along y.  grid = (n / 16, n/2+1); block (zb, kx) reads
// B[kx][:][z0 + c] and writes A[z0 + c][kx][:].
// ---------------------------------------------------------------------------
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(kThreads)
k4_yi(const cpx<T>* __restrict__ B, cpx<T>* __restrict__ A, const cpx<T>* __restrict__ twg,
      const int* __restrict__ done) {
  PLC_PASS4_PROLOGUE(C* X = tw2 + N);
  const int h = N / 2 + 1, z0 = blockIdx.x * Gm::L, kx = blockIdx.y;
  auto task_b = [&](int t) {
    const int c = t % Gm::L, k1 = t / Gm::L;
    const C* src = B + ((size_t)kx * N + k1) * N + z0 + c;
    C u[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) u[k2] = src[(size_t)N1 * k2 * N];
    phase_b_inv<T, N1, N2>(u, tw2, k1);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) X[c * Gm::S + k1 * N2 + n2] = u[n2];
  };
  if constexpr (Gm::L * N1 == kThreads) {
    task_b(threadIdx.x);
  } else {
    for (int t = threadIdx.x; t < Gm::L * N1; t += kThreads) task_b(t);
  }
  __syncthreads();
  if (Gm::L * N2 == kThreads || threadIdx.x < Gm::L * N2) {
    const int n2 = threadIdx.x % N2, c = threadIdx.x / N2;
    C v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = X[c * Gm::S + k1 * N2 + n2];
    dft_small<T, +1, N1>(v);
    C* dst = A + ((size_t)(z0 + c) * h + kx) * N + n2;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) dst[N2 * n1] = v[n1];
  }
}

// Frequencies of the paired x-pass tasks: warp g < N1/2 takes k1 = g and
// N1 - g on its two half-warps (g = 0: k1 = 0 and N1/2, each its own partner).
template <int N1> __device__ __forceinline__ int pair_k1(int g, int member) {
  return g == 0 ? (member ? N1 / 2 : 0) : (member ? N1 - g : g);
}

__device__ __forceinline__ float shfl_xor16(float a) { return __shfl_xor_sync(0xffffffffu, a, 16); }
__device__ __forceinline__ ff shfl_xor16(ff a) { return ff(shfl_xor16(a.hi), shfl_xor16(a.lo)); }
template <typename C> __device__ __forceinline__ C shfl_xor16(C a) {
  return cmk<C>(shfl_xor16(a.x), shfl_xor16(a.y));
}

// Four consecutive reals of a staging row (16-byte aligned).
__device__ __forceinline__ void st_row4(float* p, const V4<float>& u) {
  *reinterpret_cast<float4*>(p) = make_float4(u.v[0], u.v[1], u.v[2], u.v[3]);
}
__device__ __forceinline__ void st_row4(ff* p, const V4<ff>& u) {
  reinterpret_cast<float4*>(p)[0] = make_float4(u.v[0].hi, u.v[0].lo, u.v[1].hi, u.v[1].lo);
  reinterpret_cast<float4*>(p)[1] = make_float4(u.v[2].hi, u.v[2].lo, u.v[3].hi, u.v[3].lo);
}
__device__ __forceinline__ V4<float> ld_row4(const float* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  return V4<float>{{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ V4<ff> ld_row4(const ff* p) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  return V4<ff>{{ff(a.x, a.y), ff(a.z, a.w), ff(b.x, b.y), ff(b.z, b.w)}};
}

// A pair of adjacent complex values (the spectra of the two packed rows).
__device__ __forceinline__ void ld_pair(const ffc* p, ffc& a, ffc& b) {
  a = p[0];
  b = p[1];
}
__device__ __forceinline__ void st_pair(ffc* p, ffc a, ffc b) {
  p[0] = a;
  p[1] = b;
}

// ---------------------------------------------------------------------------
// XF: r2c along x + prologue.  grid = (n / 32, n); block (yb, z) owns rows
// y0 .. y0+31 of plane z; rows 2c and 2c+1 form complex line c.  With
// Z = FFT(row_2c + i row_2c+1): X_a[k] = (Z[k] + conj Z[N-k]) / 2 and
// X_b[k] = (Z[k] - conj Z[N-k]) / 2i, stored as a pair at A[z][k][y0+2c].
// ---------------------------------------------------------------------------
// Resident blocks per SM the x-forward pass asks the compiler for: 1 (no
// register cap) except for the float-float prologue of the refresh gradient,
// which at 3 blocks (80 registers, shared memory allows 3) measured 152 us
// against 164 at 2 (89 registers) for 256^3.
template <typename Pro> struct XfMinBlocks {
  static constexpr int value = 1;
};
template <> struct XfMinBlocks<ProShiftFF> {
  static constexpr int value = 3;
};
// Prologue steps (four x each) a thread keeps in flight: eight, or
// Pro::kBatch where the prologue sets one.
template <typename Pro, typename = void> struct XfBatch {
  static constexpr int value = 8;
};
template <typename Pro> struct XfBatch<Pro, decltype((void)Pro::kBatch)> {
  static constexpr int value = Pro::kBatch;
};

template <typename T, int N1, int N2, typename Pro>
__global__ void __launch_bounds__(kThreads, XfMinBlocks<Pro>::value)
k4_xf(Pro pro, cpx<T>* __restrict__ A, const cpx<T>* __restrict__ twg,
      const int* __restrict__ done) {
  PLC_PASS4_SETUP(T* R = reinterpret_cast<T*>(tw2 + N); C* X = tw2 + N);
  // the twiddle table is first read after the barrier that ends the
  // prologue, which publishes it with the rows: it needs no barrier of its
  // own, and the row loads do not wait for it
  load_tw2<C, N1, N2>(tw2, twg);
  pro.prepare();
  const int h = N / 2 + 1, z = blockIdx.y, y0 = blockIdx.x * Gm::RY;
  // prologue: 32 rows in natural order, four x per thread and step, up to
  // XfBatch steps' loads in flight per thread; the block's rows are
  // contiguous and are first requested into L2 whole
  constexpr int Q = N / 4, TOT = Gm::RY * Q, B4 = XfBatch<Pro>::value;
  const size_t row0 = ((size_t)z * N + y0) * N;
  if (threadIdx.x == 0) pro.prefetch(row0, Gm::RY * N);
  for (int base = threadIdx.x; base < TOT; base += B4 * kThreads) {
    V4<T> u[B4];
#pragma unroll
    for (int q = 0; q < B4; ++q) {
      const int e = base + q * kThreads;
      if (e < TOT) u[q] = pro.vec4(row0 + (size_t)(e / Q) * N + 4 * (e % Q));
    }
#pragma unroll
    for (int q = 0; q < B4; ++q) {
      const int e = base + q * kThreads;
      if (e < TOT) st_row4(&R[(e / Q) * Gm::SR + 4 * (e % Q)], u[q]);
    }
  }
  __syncthreads();
  // phase A on (c, n2), n2 on consecutive lanes
  const bool task_a = threadIdx.x < Gm::L * N2;
  const int n2a = threadIdx.x % N2, ca = threadIdx.x / N2;
  C v[N1 > N2 ? N1 : N2];
  if (task_a) {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1)
      v[n1] = cmk<C>(R[(2 * ca) * Gm::SR + N2 * n1 + n2a],
                     R[(2 * ca + 1) * Gm::SR + N2 * n1 + n2a]);
    phase_a<T, N1, N2, -1>(v, tw2, n2a);
  }
  __syncthreads();   // X overlays R
  if (task_a) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) X[ca * Gm::S + k1 * N2 + n2a] = v[k1];
  }
  __syncthreads();
  // phase B in pairs k1, N1 - k1 (one warp per pair), split into X_a, X_b
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (g < N1 / 2) {
    const int c = lane & 15, member = lane >> 4;
    const int k1 = pair_k1<N1>(g, member);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = X[c * Gm::S + k1 * N2 + n2];
    dft_small<T, -1, N2>(v);
    C* dst = A + ((size_t)z * h + k1) * N + y0 + 2 * c;
    auto put = [&](int k2, C zk, C zm) {   // zm = Z[N - k]
      const C zc = cconj(zm);
      const C s = cadd(zk, zc), d = csub(zk, zc);
      st_pair(dst + (size_t)N1 * k2 * N, cmk<C>(halve(s.x), halve(s.y)),
              cmk<C>(halve(d.y), -halve(d.x)));
    };
    if (g != 0) {
      // Z[N - (k1 + N1 k2)] is the partner's element N2 - 1 - k2
      C pz[N2 / 2];
#pragma unroll
      for (int j = 0; j < N2 / 2; ++j) pz[j] = shfl_xor16(v[N2 - 1 - j]);
#pragma unroll
      for (int k2 = 0; k2 < N2 / 2; ++k2) put(k2, v[k2], pz[k2]);
    } else if (member == 0) {
      // k = N1 k2, N - k = N1 (N2 - k2): own elements, k2 = 0 .. N2/2
#pragma unroll
      for (int k2 = 0; k2 <= N2 / 2; ++k2) put(k2, v[k2], v[(N2 - k2) % N2]);
    } else {
      // k = N1/2 + N1 k2, N - k = N1/2 + N1 (N2 - 1 - k2)
#pragma unroll
      for (int k2 = 0; k2 < N2 / 2; ++k2) put(k2, v[k2], v[N2 - 1 - k2]);
    }
  }
}

// Unroll of the epilogue loop of the x-inverse pass: Epi::kUnroll where the
// epilogue sets one (a light epilogue gains from more loads in flight, a
// heavy one loses registers), else 2.
template <typename Epi, typename = void> struct EpiUnroll {
  static constexpr int value = 2;
};
template <typename Epi> struct EpiUnroll<Epi, decltype((void)Epi::kUnroll)> {
  static constexpr int value = Epi::kUnroll;
};

// ---------------------------------------------------------------------------
// XI: c2r along x + epilogue.  grid = (n / 32, n).  Line c is rebuilt from
// Z[k] = X_a[k] + i X_b[k] and Z[N-k] = conj X_a[k] + i conj X_b[k] (k <= n/2);
// the imaginary parts of the k = 0 and k = n/2 coefficients are dropped
// (projection onto real fields).  The epilogue sees y = (S^-1 x)_i per cell
// and accumulates Epi::NV sums; Fin runs once on the grid totals.
// ---------------------------------------------------------------------------
// Resident blocks per SM the x-inverse pass asks the compiler for: 1 (no
// register cap) except for the float-float gradient epilogue, which at 3
// blocks (80 registers, 32 bytes of spill; shared memory allows 3) measured
// 471 us against 598 at 2 blocks (128 registers) for 256^3.
template <typename Epi> struct XiMinBlocks {
  static constexpr int value = 1;
};
template <bool STORE> struct XiMinBlocks<EpiGradFF<STORE>> {
  static constexpr int value = 3;
};

template <typename T, int N1, int N2, typename Epi, typename Fin>
__global__ void __launch_bounds__(kThreads, XiMinBlocks<Epi>::value)
k4_xi(const cpx<T>* __restrict__ A, Epi epi, Fin fin, RedArgs ra,
      const cpx<T>* __restrict__ twg, const int* __restrict__ done) {
  PLC_PASS4_PROLOGUE(T* R = reinterpret_cast<T*>(tw2 + N); C* X = tw2 + N);
  const int h = N / 2 + 1, nh = N / 2, z = blockIdx.y, y0 = blockIdx.x * Gm::RY;
  const size_t row0 = ((size_t)z * N + y0) * N;
  // the epilogue's operands do not depend on the transform: request them
  // into L2 now, so that their latency hides behind the transform
  if (threadIdx.x == 0) epi.prefetch(row0, Gm::RY * N);
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C v[N1 > N2 ? N1 : N2];
  if (g < N1 / 2) {
    const int c = lane & 15, member = lane >> 4;
    const int k1 = pair_k1<N1>(g, member);
    const C* src = A + ((size_t)z * h + k1) * N + y0 + 2 * c;
    // own coefficients k = k1 + N1 k2 <= n/2: Z[k] and the partner form Zc
    constexpr int NL = N2 / 2 + 1;
    C za[NL], zb[NL];
    const int nload = (g == 0 && member == 0) ? N2 / 2 + 1 : N2 / 2;
#pragma unroll
    for (int k2 = 0; k2 < NL; ++k2)
      if (k2 < nload) ld_pair(src + (size_t)N1 * k2 * N, za[k2], zb[k2]);
    C zc[NL];
#pragma unroll
    for (int k2 = 0; k2 < NL; ++k2) {
      if (k2 >= nload) continue;
      C xa = za[k2], xb = zb[k2];
      const int k = k1 + N1 * k2;
      if (k == 0 || k == nh) { xa.y = T(0.0); xb.y = T(0.0); }
      v[k2] = cmk<C>(xa.x - xb.y, xa.y + xb.x);
      zc[k2] = cmk<C>(xa.x + xb.y, xb.x - xa.y);
    }
    if (g != 0) {
      // Z[k1 + N1 k2] for k2 >= N2/2 is the partner's Zc at N2 - 1 - k2
#pragma unroll
      for (int j = 0; j < N2 / 2; ++j) v[N2 - 1 - j] = shfl_xor16(zc[j]);
    } else if (member == 0) {
#pragma unroll
      for (int k2 = N2 / 2 + 1; k2 < N2; ++k2) v[k2] = zc[N2 - k2];
    } else {
#pragma unroll
      for (int k2 = N2 / 2; k2 < N2; ++k2) v[k2] = zc[N2 - 1 - k2];
    }
    phase_b_inv<T, N1, N2>(v, tw2, k1);
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) X[c * Gm::S + k1 * N2 + n2] = v[n2];
  }
  __syncthreads();
  const bool task_a = threadIdx.x < Gm::L * N2;
  const int n2a = threadIdx.x % N2, ca = threadIdx.x / N2;
  if (task_a) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = X[ca * Gm::S + k1 * N2 + n2a];
    dft_small<T, +1, N1>(v);
  }
  __syncthreads();   // R overlays X
  if (task_a) {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      R[(2 * ca) * Gm::SR + N2 * n1 + n2a] = v[n1].x;
      R[(2 * ca + 1) * Gm::SR + N2 * n1 + n2a] = v[n1].y;
    }
  }
  __syncthreads();
  typename Epi::Acc acc[Epi::NV > 0 ? Epi::NV : 1];
#pragma unroll
  for (int j = 0; j < Epi::NV; ++j) acc[j].init((Epi::MAXMASK >> j) & 1u);
  constexpr int Q = N / 4, TOT = Gm::RY * Q;
#pragma unroll (EpiUnroll<Epi>::value)
  for (int e = threadIdx.x; e < TOT; e += kThreads) {
    const int row = e / Q, x = 4 * (e % Q);
    epi.vec4(row0 + (size_t)row * N + x, ld_row4(&R[row * Gm::SR + x]), acc);
  }
  if constexpr (Epi::NV > 0) block_reduce_finish_acc<Epi::NV, Epi::MAXMASK>(acc, ra, fin);
}

#undef PLC_PASS4_PROLOGUE
#undef PLC_PASS4_SETUP

}  // namespace plc
