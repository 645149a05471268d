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
#pragma once

#include "common.cuh"

namespace plc {

template <typename T> struct PassGeom {
  static constexpr int L = Tile<T>::L;    // complex lines per tile
  static constexpr int P = L + 1;         // padded pitch of a tile row
  static constexpr int RY = 2 * L;        // real rows per x-pass tile
  static constexpr int SP = RY + 1;       // pitch of the x-pass staging tile
  // complex elements per ping-pong buffer
  static __host__ __device__ int buf_elems(int n) {
    int a = n * P, b = (n / 2 + 1) * SP;
    return a > b ? a : b;
  }
  static __host__ __device__ size_t smem_bytes(int n) {
    return sizeof(cpx<T>) * ((size_t)n + 2 * (size_t)buf_elems(n));
  }
};

template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* tw, const cpx<T>* __restrict__ twg, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
}

// ---------------------------------------------------------------------------
// XF: r2c along x.  grid = (ceil(n / RY), n): block (yb, z) owns rows
// y0 .. y0+RY-1 of plane z.  Rows 2j and 2j+1 form complex line j; after the
// FFT, X_a[k] = (Z[k] + conj Z[n-k]) / 2 and X_b[k] = (Z[k] - conj Z[n-k]) / 2i.
// ---------------------------------------------------------------------------
template <typename T, typename Pro>
__global__ void __launch_bounds__(kThreads)
k_xf(Pro pro, cpx<T>* __restrict__ A, FftPlan plan, const cpx<T>* __restrict__ twg,
     const int* __restrict__ done) {
  using G = PassGeom<T>;
  using C = cpx<T>;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = plan.n, h = n / 2 + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* a = tw + n;
  C* b = a + G::buf_elems(n);
  const int z = blockIdx.y, y0 = blockIdx.x * G::RY;
  const int rows = min(G::RY, n - y0);
  const int lines = rows >> 1;
  load_twiddles<T>(tw, twg, n);
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int row = e / n, x = e - row * n;
    const size_t gi = ((size_t)z * n + (y0 + row)) * n + x;
    T u = pro(gi);
    reinterpret_cast<T*>(&a[x * G::P + (row >> 1)])[row & 1] = u;
  }
  __syncthreads();
  fft_lines<T, -1, G::L>(a, b, plan, lines, G::P, tw);
  C* st = b;
  for (int e = threadIdx.x; e < h * lines; e += blockDim.x) {
    const int k = e / lines, j = e - k * lines;
    const C zk = a[k * G::P + j];
    const C zc = cconj(a[((n - k) % n) * G::P + j]);
    const C s = cadd(zk, zc), d = csub(zk, zc);
    st[k * G::SP + 2 * j] = cmk<C>((T)0.5 * s.x, (T)0.5 * s.y);
    st[k * G::SP + 2 * j + 1] = cmk<C>((T)0.5 * d.y, (T)-0.5 * d.x);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < h * rows; e += blockDim.x) {
    const int k = e / rows, row = e - k * rows;
    A[((size_t)z * h + k) * n + y0 + row] = st[k * G::SP + row];
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
  using G = PassGeom<T>;
  using C = cpx<T>;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = plan.n, h = n / 2 + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* a = tw + n;
  C* b = a + G::buf_elems(n);
  const int z0 = blockIdx.x * G::L, kx = blockIdx.y;
  const int lines = min(G::L, n - z0);
  load_twiddles<T>(tw, twg, n);
  for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
    const int line = e / n, y = e - line * n;
    a[y * G::P + line] = A[((size_t)(z0 + line) * h + kx) * n + y];
  }
  __syncthreads();
  fft_lines<T, -1, G::L>(a, b, plan, lines, G::P, tw);
  for (int e = threadIdx.x; e < n * lines; e += blockDim.x) {
    const int ky = e / lines, line = e - ky * lines;
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
  using G = PassGeom<T>;
  using C = cpx<T>;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = plan.n;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* a = tw + n;
  C* b = a + G::buf_elems(n);
  const int ky0 = blockIdx.x * G::L, kx = blockIdx.y;
  const int lines = min(G::L, n - ky0);
  load_twiddles<T>(tw, twg, n);
  const size_t base = ((size_t)kx * n + ky0) * n;
  for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
    const int line = e / n, zz = e - line * n;
    a[zz * G::P + line] = B[base + (size_t)line * n + zz];
  }
  __syncthreads();
  fft_lines<T, -1, G::L>(a, b, plan, lines, G::P, tw);
  for (int e = threadIdx.x; e < n * lines; e += blockDim.x) {
    const int kz = e / lines, line = e - kz * lines;
    const int ky = ky0 + line;
    const int my = min(ky, n - ky), mz = min(kz, n - kz);
    const int m2 = kx * kx + my * my + mz * mz;
    T f = M[m2];
    if (zero_dc && m2 == 0) f = (T)0;
    a[kz * G::P + line] = cscale(a[kz * G::P + line], f);
  }
  __syncthreads();
  fft_lines<T, +1, G::L>(a, b, plan, lines, G::P, tw);
  for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
    const int line = e / n, zz = e - line * n;
    B[base + (size_t)line * n + zz] = a[zz * G::P + line];
  }
}

// ---------------------------------------------------------------------------
// YI: inverse c2c along y.  grid = (ceil(n / L), n/2+1).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_yi(const cpx<T>* __restrict__ B, cpx<T>* __restrict__ A, FftPlan plan,
     const cpx<T>* __restrict__ twg, const int* __restrict__ done) {
  using G = PassGeom<T>;
  using C = cpx<T>;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = plan.n, h = n / 2 + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* a = tw + n;
  C* b = a + G::buf_elems(n);
  const int z0 = blockIdx.x * G::L, kx = blockIdx.y;
  const int lines = min(G::L, n - z0);
  load_twiddles<T>(tw, twg, n);
  for (int e = threadIdx.x; e < n * lines; e += blockDim.x) {
    const int ky = e / lines, line = e - ky * lines;
    a[ky * G::P + line] = B[((size_t)kx * n + ky) * n + z0 + line];
  }
  __syncthreads();
  fft_lines<T, +1, G::L>(a, b, plan, lines, G::P, tw);
  for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
    const int line = e / n, y = e - line * n;
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
  using G = PassGeom<T>;
  using C = cpx<T>;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = plan.n, h = n / 2 + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* a = tw + n;
  C* b = a + G::buf_elems(n);
  const int z = blockIdx.y, y0 = blockIdx.x * G::RY;
  const int rows = min(G::RY, n - y0);
  const int lines = rows >> 1;
  load_twiddles<T>(tw, twg, n);
  C* st = b;
  for (int e = threadIdx.x; e < h * rows; e += blockDim.x) {
    const int k = e / rows, row = e - k * rows;
    st[k * G::SP + row] = A[((size_t)z * h + k) * n + y0 + row];
  }
  __syncthreads();
  const int nh = n / 2;
  for (int e = threadIdx.x; e < n * lines; e += blockDim.x) {
    const int k = e / lines, j = e - k * lines;
    C v;
    if (k <= nh) {
      C xa = st[k * G::SP + 2 * j], xb = st[k * G::SP + 2 * j + 1];
      if (k == 0 || k == nh) { xa.y = (T)0; xb.y = (T)0; }
      v = cmk<C>(xa.x - xb.y, xa.y + xb.x);
    } else {
      const int kk = n - k;
      const C xa = st[kk * G::SP + 2 * j], xb = st[kk * G::SP + 2 * j + 1];
      v = cmk<C>(xa.x + xb.y, xb.x - xa.y);
    }
    a[k * G::P + j] = v;
  }
  __syncthreads();
  fft_lines<T, +1, G::L>(a, b, plan, lines, G::P, tw);
  typename Epi::Acc acc[Epi::NV > 0 ? Epi::NV : 1];
#pragma unroll
  for (int j = 0; j < Epi::NV; ++j) acc[j].init((Epi::MAXMASK >> j) & 1u);
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int row = e / n, x = e - row * n;
    const C zz = a[x * G::P + (row >> 1)];
    const T y = (row & 1) ? zz.y : zz.x;
    const size_t gi = ((size_t)z * n + (y0 + row)) * n + x;
    epi(gi, y, acc);
  }
  if constexpr (Epi::NV > 0) {
    double tot[Epi::NV];
#pragma unroll
    for (int j = 0; j < Epi::NV; ++j) tot[j] = acc[j].get();
    block_reduce_finish<Epi::NV, Epi::MAXMASK>(tot, ra, fin);
  }
}

}  // namespace plc
