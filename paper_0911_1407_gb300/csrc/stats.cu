// stats.cu -- quality measures and matter statistics of a reconstruction
// (Sec. 4.1.2 and 4.3.3): correlation coefficient and Euclidean distance
// between two fields, Gaussian smoothing on the periodic grid, and the
// histogram and moments of ln(1 + delta).  FP64 fields; sums in FP64 (these
// are single passes over the data, not on the solver's path).
#include <vector>

#include "launch.cuh"

namespace plc {

namespace {

// {sum a b, sum a^2, sum b^2, sum (a - b)^2}
__global__ void __launch_bounds__(kThreads)
k_compare(const double* __restrict__ a, const double* __restrict__ b, size_t n3, RedArgs ra) {
  AccD acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j].init(false);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const double x = a[i], y = b[i], d = x - y;
    acc[0].add(x * y);
    acc[1].add(x * x);
    acc[2].add(y * y);
    acc[3].add(d * d);
  }
  block_reduce_finish_acc<4, 0u>(acc, ra, FinStore<4>{});
}

// A shift for the moments: the mean of x = ln(1 + delta) over a strided
// sample of at most 256 * 16 valid cells (one block), into red[7]; 0 when the
// sample has none.  Any shift gives the same moments in exact arithmetic; one
// near the mean keeps the one-pass power sums free of cancellation.
__global__ void __launch_bounds__(kThreads)
k_log_shift(const double* __restrict__ delta, size_t n3, DevScalars* sc) {
  __shared__ double ssum[kThreads];
  __shared__ double scnt[kThreads];
  const size_t stride = n3 / (kThreads * 16) + 1;
  double sum = 0.0, cnt = 0.0;
  for (int k = 0; k < 16; ++k) {
    const size_t i = ((size_t)k * kThreads + threadIdx.x) * stride;
    if (i < n3) {
      const double u = 1.0 + delta[i];
      if (u > 0.0) {
        sum += log(u);
        cnt += 1.0;
      }
    }
  }
  ssum[threadIdx.x] = sum;
  scnt[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ssum[threadIdx.x] += ssum[threadIdx.x + o];
      scnt[threadIdx.x] += scnt[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sc->red[7] = scnt[0] > 0.0 ? ssum[0] / scnt[0] : 0.0;
}

// In one pass: the power sums {sum d, d^2, d^3, d^4}, d = x - c about the
// shift c of k_log_shift, and the histogram of x on [lo + j width,
// lo + (j+1) width), j < nbins; counts[nbins + 0/1/2] are the cells below,
// above and with 1 + delta <= 0.  Per-block counts in shared memory, then
// integer atomics (exact, order-independent).  One FP64 log per cell.
__global__ void __launch_bounds__(kThreads)
k_log_hist(const double* __restrict__ delta, size_t n3, double lo, double width, int nbins,
           unsigned long long* __restrict__ counts, RedArgs ra) {
  extern __shared__ unsigned int hist[];
  for (int j = threadIdx.x; j < nbins + 3; j += blockDim.x) hist[j] = 0u;
  __syncthreads();
  const double shift = ra.sc->red[7];
  AccD acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j].init(false);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const double u = 1.0 + delta[i];
    int bin;
    if (u > 0.0) {
      const double x = log(u);
      const double d = x - shift, d2 = d * d;
      acc[0].add(d);
      acc[1].add(d2);
      acc[2].add(d2 * d);
      acc[3].add(d2 * d2);
      const double f = floor((x - lo) / width);
      bin = f < 0.0 ? nbins : (f >= (double)nbins ? nbins + 1 : (int)f);
    } else {
      bin = nbins + 2;
    }
    atomicAdd(&hist[bin], 1u);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nbins + 3; j += blockDim.x)
    if (hist[j]) atomicAdd(&counts[j], (unsigned long long)hist[j]);
  block_reduce_finish_acc<4, 0u>(acc, ra, FinStore<4>{});
}

// Multiplier of the Gaussian smoothing per |m|^2: exp(-|k|^2 r^2 / 2) / n^3
// (the 1/n^3 of the inverse DFT folded in, as in the prior's table).
__global__ void k_gauss_multiplier(double* __restrict__ M, int nm2, int n, double box,
                                   double radius) {
  const double kf = 2.0 * 3.14159265358979323846 / box, n3 = (double)n * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm2; i += gridDim.x * blockDim.x)
    M[i] = exp(-0.5 * kf * kf * (double)i * radius * radius) / n3;
}

// y (FP64) from float-float transforms
struct EpiStoreFF {
  static constexpr int NV = 0;
  static constexpr unsigned MAXMASK = 0;
  using Acc = AccD;
  double* out;
  __device__ void prefetch(size_t, unsigned) const {}
  __device__ void vec4(size_t i, const V4<ff>& y, Acc*) const {
    st4(out + i, V4<double>{{to_double(y.v[0]), to_double(y.v[1]), to_double(y.v[2]),
                            to_double(y.v[3])}});
  }
};

}  // namespace

void compare_fields(plc_ctx* c, const double* a, const double* b, double out[4]) {
  reset_ticket(c);
  {
    LaunchScope ls(c, S_SETUP);
    k_compare<<<pw_blocks(c), kThreads, 0, c->stream>>>(a, b, c->n3(), red_args(c));
    check(cudaGetLastError(), "k_compare");
  }
  read_scalars(c);
  for (int j = 0; j < 4; ++j) out[j] = c->sc_host->red[j];
}

void log_stats(plc_ctx* c, const double* delta, double lo, double width, int nbins,
               long long* counts, double* moments, unsigned long long* dcounts) {
  reset_ticket(c);
  {
    LaunchScope ls(c, S_SETUP);
    k_log_shift<<<1, kThreads, 0, c->stream>>>(delta, c->n3(), c->sc);
    check(cudaGetLastError(), "k_log_shift");
  }
  check(cudaMemsetAsync(dcounts, 0, sizeof(unsigned long long) * (nbins + 3), c->stream), "clear");
  {
    LaunchScope ls(c, S_SETUP);
    k_log_hist<<<pw_blocks(c), kThreads, sizeof(unsigned int) * (nbins + 3), c->stream>>>(
        delta, c->n3(), lo, width, nbins, dcounts, red_args(c));
    check(cudaGetLastError(), "k_log_hist");
  }
  std::vector<unsigned long long> h(nbins + 3);
  check(cudaMemcpyAsync(h.data(), dcounts, sizeof(unsigned long long) * (nbins + 3),
                        cudaMemcpyDeviceToHost, c->stream), "histogram copy");
  read_scalars(c);
  for (int j = 0; j < nbins + 3; ++j) counts[j] = (long long)h[j];
  // central moments from the power sums about the shift (exact algebra):
  // with a = S1 / cnt = mean - shift, m2 = S2/cnt - a^2,
  // m3 = S3/cnt - 3 a S2/cnt + 2 a^3, m4 = S4/cnt - 4 a S3/cnt + 6 a^2 S2/cnt - 3 a^4
  const double* r = c->sc_host->red;
  const double cnt = (double)((long long)c->n3() - counts[nbins + 2]);
  double mean = 0.0, m2 = 0.0, m3 = 0.0, m4 = 0.0;
  if (cnt > 0) {
    const double a = r[0] / cnt, p2 = r[1] / cnt, p3 = r[2] / cnt, p4 = r[3] / cnt;
    mean = r[7] + a;
    m2 = p2 - a * a;
    m3 = p3 - 3.0 * a * p2 + 2.0 * a * a * a;
    m4 = p4 - 4.0 * a * p3 + 6.0 * a * a * p2 - 3.0 * a * a * a * a;
  }
  moments[0] = mean;
  moments[1] = m2;
  moments[2] = m2 > 0 ? m3 / (m2 * std::sqrt(m2)) : 0.0;
  moments[3] = m2 > 0 ? m4 / (m2 * m2) - 3.0 : 0.0;
}

void gaussian_smooth(plc_ctx* c, const double* x, double* y, double radius, double* table) {
  const int nm2 = 3 * (c->n / 2) * (c->n / 2) + 1;
  {
    LaunchScope ls(c, S_SETUP);
    k_gauss_multiplier<<<(nm2 + kThreads - 1) / kThreads, kThreads, 0, c->stream>>>(
        table, nm2, c->n, c->box, radius);
    check(cudaGetLastError(), "k_gauss_multiplier");
  }
  // float-float transforms where the length has a four-step schedule (FP64
  // accuracy on the FP32 pipes), FP64 Stockham otherwise
  if (!run_four_step<ff>(c, ProShiftFF{x, ff(0.f, 0.f)}, EpiStoreFF{y}, FinNone{}, 0, nullptr, S_GXFF,
                         table))
    run_pipeline<double>(c, ProLoad<double>{x}, EpiStore<double>{y}, FinNone{}, 0, nullptr, false,
                         table);
  check(cudaStreamSynchronize(c->stream), "stream synchronize");
}

}  // namespace plc
