// passes.cuh -- the five passes of the spectral operator S^-1 (Sec. 2.2).
//
// S^-1 x = IDFT( DFT(x) / lambda_k ) on an n^3 periodic grid is evaluated in
// five HBM passes, each moving whole 128-byte rows and transposing in shared
// memory so that the next pass again reads contiguous lines:
//
//   XF  real x[z][y][x]     -> A[z][kx][y]   r2c along x (two real rows packed
//                                            as one complex line), + prologue
//   YF  A[z][kx][y]         -> B[kx][ky][z]  c2c along y
//   Z   B[kx][ky][z]        -> B             c2c along z, times 1/(lambda n^3),
//                                            inverse c2c along z
//   YI  B[kx][ky][z]        -> A[z][kx][y]   inverse c2c along y
//   XI  A[z][kx][y]         -> out[z][y][x]  c2r along x, + epilogue/reduction
//
// kx runs over the n/2+1 non-negative x-frequencies.  The prologue computes
// the transformed field on the fly (s - mu, a CG direction update, a Newton
// step) and the epilogue fuses the pointwise tail (gradient of Sec. 3.1.2,
// Hessian-vector product, dot products) into the last pass.
//
// These kernels serve FP64, and FP32 lengths (or schedules) without a
// register four-step form (passes4.cuh); their line transform is a
// mixed-radix Stockham FFT in shared memory.
//
// Every block has all global loads of a tile in flight at once: the pure data
// passes (YF, Z, YI) copy their tiles with cp.async straight into shared
// memory, and XF / XI batch their loads in registers.  In A the spectra of
// the two real rows packed into one complex line sit next to each other
// (y = y0 + 2j, y0 + 2j + 1), so XF and XI move them as one vector and need
// no staging tile.
#pragma once

#include "common.cuh"

namespace plc {

template <typename T> struct PassGeom {
  static constexpr int L = Tile<T>::L;    // complex lines per tile
  static constexpr int P = L + 1;         // padded pitch of a tile row
  static constexpr int RY = 2 * L;        // real rows per x-pass tile
  static __host__ __device__ int buf_elems(int n) { return n * P; }
  // twiddles and the two buffers the Stockham stages ping-pong between
  static __host__ __device__ size_t smem_bytes(const FftPlan& p) {
    return sizeof(cpx<T>) * ((size_t)p.n + 2 * (size_t)buf_elems(p.n));
  }
  static __host__ __device__ size_t smem_bytes_max(int n) {
    return sizeof(cpx<T>) * ((size_t)n + 2 * (size_t)buf_elems(n));
  }
};

// Forward line transform of the tile (natural order in and out); on return
// `a` points at the result.
template <typename T>
__device__ __forceinline__ void fft_tile_fwd(cpx<T>*& a, cpx<T>*& b, const FftPlan& plan, int nl,
                                             const cpx<T>* tw) {
  fft_lines<T, -1, PassGeom<T>::L>(a, b, plan, nl, PassGeom<T>::P, tw);
}

// Inverse line transform (unnormalised), natural order in and out.
template <typename T>
__device__ __forceinline__ void fft_tile_inv(cpx<T>*& a, cpx<T>*& b, const FftPlan& plan, int nl,
                                             const cpx<T>* tw) {
  fft_lines<T, +1, PassGeom<T>::L>(a, b, plan, nl, PassGeom<T>::P, tw);
}

// Forward transform, multiply by mul(line, kz), inverse transform: natural
// order in and out.
template <typename T, typename Mul>
__device__ __forceinline__ void filter_tile(cpx<T>*& a, cpx<T>*& b, const FftPlan& plan, int nl,
                                            const cpx<T>* tw, Mul mul) {
  using G = PassGeom<T>;
  fft_lines<T, -1, G::L>(a, b, plan, nl, G::P, tw);
  const int n = plan.n;
  const FastDiv ld = make_fastdiv(nl);
  for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
    const int kz = fdiv(e, ld), line = e - kz * nl;
    a[kz * G::P + line] = cscale(a[kz * G::P + line], mul(line, kz));
  }
  __syncthreads();
  fft_lines<T, +1, G::L>(a, b, plan, nl, G::P, tw);
}

template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* tw, const cpx<T>* __restrict__ twg, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
}

// Two adjacent complex values as one (float) or two (double) 16-byte moves.
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
  a = p[0];
  b = p[1];
}
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_pair(double2* p, double2 a, double2 b) {
  p[0] = a;
  p[1] = b;
}

#define PLC_PASS_PROLOGUE                                      \
  using G = PassGeom<T>;                                       \
  using C = cpx<T>;                                            \
  if (done && *done) return;                                   \
  extern __shared__ __align__(16) unsigned char smem_raw[];    \
  C* tw = reinterpret_cast<C*>(smem_raw);                      \
  C* a = tw + plan.n;                                          \
  C* b = a + G::buf_elems(plan.n);                             \
  load_twiddles<T>(tw, twg, plan.n)

// ---------------------------------------------------------------------------
// XF: r2c along x.  grid = (ceil(n / RY), n): block (yb, z) owns rows
// y0 .. y0+RY-1 of plane z.  Rows 2j and 2j+1 form complex line j; after the
// FFT, X_a[k] = (Z[k] + conj Z[n-k]) / 2 and X_b[k] = (Z[k] - conj Z[n-k]) / 2i.
// ---------------------------------------------------------------------------
template <typename T, typename Pro>
__global__ void __launch_bounds__(kThreads)
k_xf(Pro pro, cpx<T>* __restrict__ A, FftPlan plan, const cpx<T>* __restrict__ twg,
     const int* __restrict__ done) {
  PLC_PASS_PROLOGUE;
  pro.prepare();
  const int n = plan.n, h = n / 2 + 1;
  const int z = blockIdx.y, y0 = blockIdx.x * G::RY;
  const int rows = min(G::RY, n - y0);
  const int lines = rows >> 1;
  if (n & 3) {   // rows not a multiple of 4 long: one element per step
    for (int e = threadIdx.x; e < rows * n; e += kThreads) {
      const int row = fdiv(e, plan.nd), x = e - row * n;
      reinterpret_cast<T*>(&a[x * G::P + (row >> 1)])[row & 1] =
          pro(((size_t)z * n + (y0 + row)) * n + x);
    }
  }
  // four consecutive x per thread and step: 16-byte global accesses
  const int total4 = (n & 3) ? 0 : (rows * n) >> 2;
  constexpr int B = 4;
  for (int base = threadIdx.x; base < total4; base += B * kThreads) {
    V4<T> u[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int e = base + k * kThreads;
      if (e < total4) {
        const int row = fdiv(4 * e, plan.nd), x = 4 * e - row * n;
        u[k] = pro.vec4(((size_t)z * n + (y0 + row)) * n + x);
      }
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int e = base + k * kThreads;
      if (e < total4) {
        const int row = fdiv(4 * e, plan.nd), x = 4 * e - row * n;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          reinterpret_cast<T*>(&a[(x + j) * G::P + (row >> 1)])[row & 1] = u[k].v[j];
      }
    }
  }
  __syncthreads();
  fft_tile_fwd<T>(a, b, plan, lines, tw);
  const FastDiv ld = make_fastdiv(lines);
  for (int e = threadIdx.x; e < h * lines; e += kThreads) {
    const int k = fdiv(e, ld), j = e - k * lines;
    const C zk = a[k * G::P + j];
    const C zc = cconj(a[(k ? n - k : 0) * G::P + j]);
    const C s = cadd(zk, zc), d = csub(zk, zc);
    st_pair(&A[((size_t)z * h + k) * n + y0 + 2 * j], cmk<C>((T)0.5 * s.x, (T)0.5 * s.y),
            cmk<C>((T)0.5 * d.y, (T)-0.5 * d.x));
  }
}

// ---------------------------------------------------------------------------
// YF: c2c along y.  grid = (ceil(n / L), n/2+1): block (zb, kx) owns lines
// A[z][kx][:] for z in z0 .. z0+L-1 and writes B[kx][ky][z0 .. z0+L-1].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_yf(const cpx<T>* __restrict__ A, cpx<T>* __restrict__ B, FftPlan plan,
     const cpx<T>* __restrict__ twg, const int* __restrict__ done) {
  PLC_PASS_PROLOGUE;
  const int n = plan.n, h = n / 2 + 1;
  const int z0 = blockIdx.x * G::L, kx = blockIdx.y;
  const int lines = min(G::L, n - z0);
  const int total = lines * n;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int line = fdiv(e, plan.nd), y = e - line * n;
    cp_async(&a[y * G::P + line], &A[((size_t)(z0 + line) * h + kx) * n + y]);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_tile_fwd<T>(a, b, plan, lines, tw);
  const FastDiv ld = make_fastdiv(lines);
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int ky = fdiv(e, ld), line = e - ky * lines;
    B[((size_t)kx * n + ky) * n + z0 + line] = a[ky * G::P + line];
  }
}

// ---------------------------------------------------------------------------
// Z: forward c2c along z, multiply by M[|m|^2] = 1/(lambda_k n^3) (the 1/n^3
// of the inverse DFT is folded in), inverse c2c along z, in place.
// grid = (ceil(n / L), n/2+1): block (kyb, kx) owns lines B[kx][ky0..ky0+L-1][:].
// zero_dc drops the DC mode (used for the amplitude derivative).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_z(cpx<T>* __restrict__ B, const T* __restrict__ M, int zero_dc, FftPlan plan,
    const cpx<T>* __restrict__ twg, const int* __restrict__ done) {
  PLC_PASS_PROLOGUE;
  const int n = plan.n;
  const int ky0 = blockIdx.x * G::L, kx = blockIdx.y;
  const int lines = min(G::L, n - ky0);
  const size_t base = ((size_t)kx * n + ky0) * n;
  const int total = lines * n;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int line = fdiv(e, plan.nd), zz = e - line * n;
    cp_async(&a[zz * G::P + line], &B[base + e]);
  }
  cp_async_wait_all();
  __syncthreads();
  auto mul = [&](int line, int kz) -> T {
    const int ky = ky0 + line;
    const int my = min(ky, n - ky), mz = min(kz, n - kz);
    const int m2 = kx * kx + my * my + mz * mz;
    return (zero_dc && m2 == 0) ? (T)0 : __ldg(M + m2);
  };
  filter_tile<T>(a, b, plan, lines, tw, mul);
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int line = fdiv(e, plan.nd), zz = e - line * n;
    B[base + e] = a[zz * G::P + line];
  }
}

// ---------------------------------------------------------------------------
// YI: inverse c2c along y.  grid = (ceil(n / L), n/2+1).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_yi(const cpx<T>* __restrict__ B, cpx<T>* __restrict__ A, FftPlan plan,
     const cpx<T>* __restrict__ twg, const int* __restrict__ done) {
  PLC_PASS_PROLOGUE;
  const int n = plan.n, h = n / 2 + 1;
  const int z0 = blockIdx.x * G::L, kx = blockIdx.y;
  const int lines = min(G::L, n - z0);
  const int total = lines * n;
  const FastDiv ld = make_fastdiv(lines);
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int ky = fdiv(e, ld), line = e - ky * lines;
    cp_async(&a[ky * G::P + line],
             &B[((size_t)kx * n + ky) * n + z0 + line]);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_tile_inv<T>(a, b, plan, lines, tw);
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const int line = fdiv(e, plan.nd), y = e - line * n;
    A[((size_t)(z0 + line) * h + kx) * n + y] = a[y * G::P + line];
  }
}

// ---------------------------------------------------------------------------
// XI: c2r along x + epilogue.  grid = (ceil(n / RY), n).  Rows 2j and 2j+1
// are recovered together from Z[k] = X_a[k] + i X_b[k] (k <= n/2) and
// Z[n-k] = conj X_a[k] + i conj X_b[k]; the imaginary parts of the k = 0 and
// k = n/2 coefficients are dropped (projection onto real fields).
// The epilogue is called once per cell with the value y = (S^-1 x)_i and
// accumulates Epi::NV per-thread sums; Fin runs once on the grid totals.
// ---------------------------------------------------------------------------
template <typename T, typename Epi, typename Fin>
__global__ void __launch_bounds__(kThreads)
k_xi(const cpx<T>* __restrict__ A, Epi epi, Fin fin, RedArgs ra, FftPlan plan,
     const cpx<T>* __restrict__ twg, const int* __restrict__ done) {
  PLC_PASS_PROLOGUE;
  const int n = plan.n, h = n / 2 + 1, nh = n / 2;
  const int z = blockIdx.y, y0 = blockIdx.x * G::RY;
  const int rows = min(G::RY, n - y0);
  const int lines = rows >> 1;
  const int npairs = h * lines;
  const FastDiv ld = make_fastdiv(lines);
  constexpr int B4 = 4;
  for (int base = threadIdx.x; base < npairs; base += B4 * kThreads) {
    C xa[B4], xb[B4];
#pragma unroll
    for (int q = 0; q < B4; ++q) {
      const int e = base + q * kThreads;
      if (e < npairs) {
        const int k = fdiv(e, ld), j = e - k * lines;
        ld_pair(&A[((size_t)z * h + k) * n + y0 + 2 * j], xa[q], xb[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < B4; ++q) {
      const int e = base + q * kThreads;
      if (e < npairs) {
        const int k = fdiv(e, ld), j = e - k * lines;
        C va = xa[q], vb = xb[q];
        if (k == 0 || k == nh) { va.y = (T)0; vb.y = (T)0; }
        a[k * G::P + j] = cmk<C>(va.x - vb.y, va.y + vb.x);
        if (k > 0 && k < nh)
          a[(n - k) * G::P + j] = cmk<C>(va.x + vb.y, vb.x - va.y);
      }
    }
  }
  __syncthreads();
  fft_tile_inv<T>(a, b, plan, lines, tw);
  typename Epi::Acc acc[Epi::NV > 0 ? Epi::NV : 1];
#pragma unroll
  for (int j = 0; j < Epi::NV; ++j) acc[j].init((Epi::MAXMASK >> j) & 1u);
  if (n & 3) {   // rows not a multiple of 4 long: one element per step
    for (int e = threadIdx.x; e < rows * n; e += kThreads) {
      const int row = fdiv(e, plan.nd), x = e - row * n;
      const C zz = a[x * G::P + (row >> 1)];
      epi(((size_t)z * n + (y0 + row)) * n + x, (row & 1) ? zz.y : zz.x, acc);
    }
  }
  const int total4 = (n & 3) ? 0 : (rows * n) >> 2;
#pragma unroll 2
  for (int e = threadIdx.x; e < total4; e += kThreads) {
    const int row = fdiv(4 * e, plan.nd), x = 4 * e - row * n;
    V4<T> y;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const C zz = a[(x + j) * G::P + (row >> 1)];
      y.v[j] = (row & 1) ? zz.y : zz.x;
    }
    epi.vec4(((size_t)z * n + (y0 + row)) * n + x, y, acc);
  }
  if constexpr (Epi::NV > 0) block_reduce_finish_acc<Epi::NV, Epi::MAXMASK>(acc, ra, fin);
}

#undef PLC_PASS_PROLOGUE

}  // namespace plc
