// prior.cu -- device set-up of the prior operator (Sec. 2.2): the inverse
// eigenvalue 1/(lambda n^3) for every |m|^2 of the grid and the Jacobi
// constant (S^-1)_ii; plus the small host helpers shared by the solver.
#include <cstring>

#include "launch.cuh"

namespace plc {

// ----------------------------- prior set-up -------------------------------
// ln f(|k|) at |k| = (2 pi / L) sqrt(m2), m2 > 0, for a table linear in
// (ln k, ln f) between the points lk = ln k, lf = ln f.
__device__ double interp_ln(int m2, double box, const double* __restrict__ lk,
                            const double* __restrict__ lf, int nk) {
  const double lnk = log(2.0 * 3.14159265358979323846 / box) + 0.5 * log((double)m2);
  int lo = 0, hi = nk - 1;                 // largest j with lk[j] <= lnk
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (lk[mid] <= lnk) lo = mid; else hi = mid;
  }
  const double t = (lnk - lk[lo]) / (lk[lo + 1] - lk[lo]);
  return lf[lo] + t * (lf[lo + 1] - lf[lo]);
}

// M[m2] = 1 / (lambda n^3) for |m|^2 = m2, lambda = P(|k|) n^3 / L^3 with
// |k| = (2 pi / L) sqrt(m2) and P linear in (ln k, ln P) between the table
// points lk = ln k, lP = ln P.  M[0] = inv_lambda_dc / n^3.
__global__ void k_build_multiplier(double* __restrict__ M64, float* __restrict__ M32, int nm2,
                                   int n, double box, const double* __restrict__ lk,
                                   const double* __restrict__ lP, int nk, double inv_dc) {
  const double n3 = (double)n * n * n;
  for (int m2 = blockIdx.x * blockDim.x + threadIdx.x; m2 < nm2; m2 += gridDim.x * blockDim.x) {
    double v;
    if (m2 == 0) {
      v = inv_dc / n3;
    } else {
      const double lam = exp(interp_ln(m2, box, lk, lP, nk)) * n3 / (box * box * box);
      v = 1.0 / (lam * n3);
    }
    M64[m2] = v;
    M32[m2] = (float)v;
  }
}

// The bias convolution B of Sec. 2.4.1: Mb[m2] = b(|k|) / n^3 (the inverse
// transform is unnormalised), b linear in (ln k, ln b); Mb[0] = b_dc / n^3.
__global__ void k_build_bias(double* __restrict__ M64, float* __restrict__ M32, int nm2, int n,
                             double box, const double* __restrict__ lk,
                             const double* __restrict__ lb, int nk, double b_dc) {
  const double n3 = (double)n * n * n;
  for (int m2 = blockIdx.x * blockDim.x + threadIdx.x; m2 < nm2; m2 += gridDim.x * blockDim.x) {
    const double v = (m2 == 0 ? b_dc : exp(interp_ln(m2, box, lk, lb, nk))) / n3;
    M64[m2] = v;
    M32[m2] = (float)v;
  }
}

// (S^-1)_ii = n^-3 sum_k 1/lambda_k = sum over all n^3 modes of M[|m|^2],
// and the prior variance per cell without the DC mode,
// S_ii = n^-3 sum_{k != 0} lambda_k = n^-6 sum_{k != 0} 1 / M[|m|^2].
__global__ void __launch_bounds__(kThreads)
k_jacobi_constant(const double* __restrict__ M64, int n, RedArgs ra) {
  double acc[2] = {0.0, 0.0};
  const size_t n3 = (size_t)n * n * n;
  const double inv_n6 = 1.0 / ((double)n3 * (double)n3);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % n), ky = (int)((i / n) % n), kz = (int)(i / ((size_t)n * n));
    const int mx = min(kx, n - kx), my = min(ky, n - ky), mz = min(kz, n - kz);
    const int m2 = mx * mx + my * my + mz * mz;
    const double v = M64[m2];
    acc[0] += v;
    if (m2 > 0 && v > 0.0) acc[1] += inv_n6 / v;
  }
  block_reduce_finish<2, 0u>(acc, ra, FinStore<2>{});
}

const char* const kSiteNames[S_NSITES] = {
    "xf_f64", "yf_f64", "z_f64", "yi_f64", "xi_f64",
    "xf_f32", "yf_f32", "z_f32", "yi_f32", "xi_f32",
    "grad_xf_f64", "grad_yf_f64", "grad_z_f64", "grad_yi_f64", "grad_xi_f64",
    "grad_xf_f32", "grad_yf_f32", "grad_z_f32", "grad_yi_f32", "grad_xi_f32",
    "grad_xf_ff", "grad_yf_ff", "grad_z_ff", "grad_yi_ff", "grad_xi_ff",
    "cg_init", "cg_update_f64", "cg_update_f32", "newton_update_f64", "newton_update_f32",
    "diag", "convert", "setup", "boundary",
    "bias_xf_f64", "bias_yf_f64", "bias_z_f64", "bias_yi_f64", "bias_xi_f64",
    "bias_xf_f32", "bias_yf_f32", "bias_z_f32", "bias_yi_f32", "bias_xi_f32",
    "bias_misc"};

constexpr int kProfSlots = 512;

LaunchScope::LaunchScope(plc_ctx* c, Site site) : c_(c), slot_(-1) {
  Profiler& p = c->prof;
  p.launches[site]++;
  if (!p.timing) return;
  if (p.ev.empty()) {
    p.ev.resize(2 * kProfSlots);
    for (auto& e : p.ev) check(cudaEventCreate(&e), "cudaEventCreate");
    p.site_of.assign(kProfSlots, 0);
  }
  if (p.used == kProfSlots) profile_collect(c);
  slot_ = p.used++;
  p.site_of[slot_] = site;
  check(cudaEventRecord(p.ev[2 * slot_], c->stream), "cudaEventRecord");
}

LaunchScope::~LaunchScope() {
  if (slot_ >= 0) cudaEventRecord(c_->prof.ev[2 * slot_ + 1], c_->stream);
}

void profile_collect(plc_ctx* c) {
  Profiler& p = c->prof;
  if (p.used == 0) return;
  check(cudaEventSynchronize(p.ev[2 * (p.used - 1) + 1]), "cudaEventSynchronize");
  for (int i = 0; i < p.used; ++i) {
    float ms = 0.f;
    check(cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]), "cudaEventElapsedTime");
    p.ms[p.site_of[i]] += ms;
    p.timed[p.site_of[i]] += 1;
  }
  p.used = 0;
}

void profile_reset(plc_ctx* c, bool timing) {
  Profiler& p = c->prof;
  if (p.used) profile_collect(c);
  for (int i = 0; i < S_NSITES; ++i) { p.launches[i] = 0; p.timed[i] = 0; p.ms[i] = 0.0; }
  p.timing = timing;
}

void profile_release(plc_ctx* c) {
  for (auto& e : c->prof.ev) cudaEventDestroy(e);
  c->prof.ev.clear();
}

void check(cudaError_t e, const char* where) {
  if (e != cudaSuccess) throw CudaError{e, where};
}

void reset_ticket(plc_ctx* c) {
  check(cudaMemsetAsync(&c->sc->ticket, 0, sizeof(unsigned), c->stream), "reset ticket");
}

void read_scalars(plc_ctx* c) {
  check(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream),
        "read scalars");
  check(cudaStreamSynchronize(c->stream), "stream synchronize");
}

void build_prior(plc_ctx* c, const double* lk_host, const double* lP_host, int nk) {
  check(cudaMemcpyAsync(c->lk, lk_host, sizeof(double) * nk, cudaMemcpyHostToDevice, c->stream),
        "copy ln k");
  check(cudaMemcpyAsync(c->lP, lP_host, sizeof(double) * nk, cudaMemcpyHostToDevice, c->stream),
        "copy ln P");
  const int nb = (c->nm2 + kThreads - 1) / kThreads;
  LaunchScope ls(c, S_SETUP);
  k_build_multiplier<<<nb, kThreads, 0, c->stream>>>(c->M64, c->M32, c->nm2, c->n, c->box, c->lk,
                                                      c->lP, nk, c->inv_dc);
  check(cudaGetLastError(), "k_build_multiplier");
  reset_ticket(c);
  LaunchScope ls2(c, S_SETUP);
  k_jacobi_constant<<<pw_blocks(c), kThreads, 0, c->stream>>>(c->M64, c->n, red_args(c));
  check(cudaGetLastError(), "k_jacobi_constant");
  read_scalars(c);
  c->jac_c = c->sc_host->red[0];
  c->prior_var = c->sc_host->red[1];
}

// ||g||^2 at the prior mean without a transform: at s = mean the prior term
// S^-1 (s - mean) vanishes and g = factor w - N (lognormal model: mean mu,
// factor nbar e^mu; Gaussian-prior model: mean 0, factor nbar).  Also sets
// off_mean when s differs from the mean anywhere (compared bit for bit, so
// -0.0 against +0.0 counts as different: the caller then takes the
// transform); s null: the start is the mean by definition, nothing is read
// and off_mean is 0.  ||g0|| only normalises the stop test: the Kahan FP32 sum
// (relative error ~1e-7) is ample.
__global__ void __launch_bounds__(kThreads)
k_g0_at_mean(const double* __restrict__ s, const int32_t* __restrict__ N,
             const double* __restrict__ w, long long mean_bits, float factor, size_t n3,
             RedArgs ra) {
  AccK acc[2];
  acc[0].init(false);
  acc[1].init(true);
  const size_t step = (size_t)gridDim.x * blockDim.x * 4;
  for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4; i < n3; i += step) {
    const V4<int32_t> nv = ld4(N + i);
    V4<float> wv{{1.f, 1.f, 1.f, 1.f}};
    if (w) {
      const V4<double> wd = ld4(w + i);
#pragma unroll
      for (int j = 0; j < 4; ++j) wv.v[j] = (float)wd.v[j];
    }
    if (s) {
      const longlong2 a = __ldg(reinterpret_cast<const longlong2*>(s + i));
      const longlong2 b = __ldg(reinterpret_cast<const longlong2*>(s + i) + 1);
      const bool off = a.x != mean_bits || a.y != mean_bits || b.x != mean_bits || b.y != mean_bits;
      acc[1].max(off ? 1.f : 0.f);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float d = factor * wv.v[j] - (float)nv.v[j];
      acc[0].add(d * d);
    }
  }
  struct Fin {
    __device__ void operator()(const double* t, DevScalars* sc) const {
      sc->red[2] = t[0];
      sc->off_mean = t[1] > 0.0 ? 1 : 0;
    }
  };
  block_reduce_finish_acc<2, 2u>(acc, ra, Fin{});
}

// ||g(mean)||^2 into red[2] and the off_mean flag (see k_g0_at_mean).
void g0_at_mean(plc_ctx* c, const double* s, const int32_t* N, const double* w,
                       double mean, double factor) {
  LaunchScope ls(c, S_SETUP);
  long long bits;
  static_assert(sizeof(bits) == sizeof(mean), "double is 64 bits");
  memcpy(&bits, &mean, sizeof(bits));
  k_g0_at_mean<<<pw_blocks(c), kThreads, 0, c->stream>>>(s, N, w, bits, (float)factor, c->n3(),
                                                         red_args(c));
  check(cudaGetLastError(), "k_g0_at_mean");
}

void build_bias(plc_ctx* c, const double* lk_host, const double* lb_host, int nb, double b_dc) {
  check(cudaMemcpyAsync(c->lkb, lk_host, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream),
        "copy ln k");
  check(cudaMemcpyAsync(c->lbb, lb_host, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream),
        "copy ln b");
  const int nm2 = 3 * (c->n / 2) * (c->n / 2) + 1;
  const int nblk = (nm2 + kThreads - 1) / kThreads;
  LaunchScope ls(c, S_SETUP);
  k_build_bias<<<nblk, kThreads, 0, c->stream>>>(c->Mb64, c->Mb32, nm2, c->n, c->box, c->lkb,
                                                 c->lbb, nb, b_dc);
  check(cudaGetLastError(), "k_build_bias");
  check(cudaStreamSynchronize(c->stream), "stream synchronize");
}

}  // namespace plc
