// ctx.h -- host-side state of a libplc context and the internal launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/plc.h"
#include "common.cuh"

namespace plc {

// Launch sites of the library's kernels, for the counters and the optional
// CUDA-event timing.
enum Site {
  // pipelines of the CG Hessian-vector product (and the public operators)
  S_XF64, S_YF64, S_Z64, S_YI64, S_XI64,
  S_XF32, S_YF32, S_Z32, S_YI32, S_XI32,
  // pipelines of the Newton gradient (and line-search trials)
  S_GXF64, S_GYF64, S_GZ64, S_GYI64, S_GXI64,
  S_GXF32, S_GYF32, S_GZ32, S_GYI32, S_GXI32,
  // the FP64 gradient of the mixed solve in float-float transforms
  S_GXFF, S_GYFF, S_GZFF, S_GYIFF, S_GXIFF,
  S_CG_INIT, S_CG_UPDATE64, S_CG_UPDATE32, S_NEWTON_UPDATE64, S_NEWTON_UPDATE32,
  S_DIAG, S_CONVERT, S_SETUP, S_BOUNDARY,
  // pipelines and element-wise kernels of the linear-bias model
  S_BXF64, S_BYF64, S_BZ64, S_BYI64, S_BXI64,
  S_BXF32, S_BYF32, S_BZ32, S_BYI32, S_BXI32,
  S_BIAS,
  S_NSITES
};
extern const char* const kSiteNames[S_NSITES];

// FP32 line-transform schedules with a register four-step form (passes4.cuh):
// n = f1 f2.  The first entry for an n is the default; plc_autotune times
// every entry for n and the Stockham form (f1 = f2 = 0).
struct FourStepShape {
  int n, f1, f2;
};
constexpr FourStepShape kFourStep[] = {
    {256, 16, 16}, {192, 16, 12}, {192, 12, 16}, {128, 16, 8}, {128, 8, 16},
    {96, 12, 8},   {96, 8, 12},   {64, 8, 8},    {32, 8, 4}};

struct Profiler {
  bool timing = false;
  long long launches[S_NSITES] = {};
  long long timed[S_NSITES] = {};
  double ms[S_NSITES] = {};
  std::vector<cudaEvent_t> ev;      // 2 per slot
  std::vector<int> site_of;         // site of each pending slot
  int used = 0;
};

}  // namespace plc

struct plc_ctx {
  int n = 0;
  double box = 0.0;
  int precision = PLC_FP64;
  cudaStream_t stream = nullptr;
  int sms = 0;
  plc::FftPlan plan{};

  // FFT scratch: two half-spectra sized for double2 (float2 reuses them).
  void* specA = nullptr;
  void* specB = nullptr;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  void* twff = nullptr;        // float-float twiddles (ffc, ff.cuh)
  void* expff = nullptr;       // 2^(j/64), j < 64, float-float (exp_ff)

  // Prior: inverse eigenvalue per |m|^2, its FP32 copy, ln-tables.
  double* M64 = nullptr;
  float* M32 = nullptr;
  int nm2 = 0;
  double* lk = nullptr;
  double* lP = nullptr;
  int nk_cap = 0;
  bool have_prior = false;
  double mu = 0.0;
  double inv_dc = 0.0;
  double jac_c = 0.0;          // (S^-1)_ii
  double prior_var = 0.0;      // S_ii without the DC mode (prior variance per cell)

  // Linear bias (Sec. 2.4.1): b(|k|) / n^3 per |m|^2, FP64 and FP32 copies,
  // and the ln-tables it was built from.
  double* Mb64 = nullptr;
  float* Mb32 = nullptr;
  double* lkb = nullptr;
  double* lbb = nullptr;
  int nb_cap = 0;
  bool have_bias = false;

  // Reductions and device scalars.
  plc::DevScalars* sc = nullptr;
  plc::DevScalars* sc_host = nullptr;   // pinned
  double* partials = nullptr;
  size_t partial_blocks = 0;

  // Histogram counts of plc_log_stats: kMaxBins + 3 entries (below, above,
  // invalid at the end), allocated on its first call.
  static constexpr int kMaxBins = 4096;
  unsigned long long* hist = nullptr;

  // Solver work fields, each n^3 doubles, allocated on first use.
  static constexpr int kNumWork = 13;
  void* wf[kNumWork] = {};
  // Extra work fields of the linear-bias solve, allocated on its first use.
  static constexpr int kNumBiasWork = 12;
  void* bwf[kNumBiasWork] = {};

  plc::Profiler prof;
  std::string err;

  // Device-driven solve: control block and the cached graph (graph.cu).
  void* graph = nullptr;

  size_t n3() const { return (size_t)n * n * n; }
};

namespace plc {

// Error plumbing: a CUDA failure is recorded on the context and turned into
// PLC_ERR_CUDA by the caller.
struct CudaError {
  cudaError_t code;
  const char* where;
};
void check(cudaError_t e, const char* where);   // throws CudaError

// Spectral pipelines (five passes).  T = field type of the FFT.
template <typename T> void prior_apply(plc_ctx* c, const T* x, T* y);
template <typename T> void hessvec_s(plc_ctx* c, const T* s, const T* w, double nbar,
                                     const T* v, T* out);
// Public gradient: g (may be null) and the sums of -ln P (FP64).
template <typename T> void grad_public(plc_ctx* c, const T* s, const T* w, const int32_t* N,
                                       double nbar, T* g);
// Newton gradient at s through the FFT, in transform type T (s held as TS);
// writes y = S^-1 (s - mu), g, D and r = -g (CG type TC) and starts the CG.
template <typename T, typename TS, typename TC>
void grad_newton(plc_ctx* c, const TS* s, const double* w, const int32_t* N, double nbar, T* y,
                 T* g, TC* D, TC* r, bool jac);
// Newton trial point s + tau xi without an FFT (see k_newton_update).
// The sums of the FP64 gradient of the mixed solve at s (float-float
// transforms, no field stored) into sc->red; false when the length has no
// four-step schedule (nothing launched).
bool grad_sums_ff(plc_ctx* c, const double* s, const double* w, const int32_t* N, double nbar,
                  bool jac);
template <typename T, typename TC>
void newton_update(plc_ctx* c, const T* s, const T* y, const T* g, const TC* r, const TC* xi,
                   const TC* D, const int32_t* N, const double* w, double nbar, double tau,
                   bool jac, T* s2, T* y2, T* g2, TC* D2, TC* r2,
                   const double* tau_dev = nullptr);   // non-null: tau read on the device
template <typename T> void cg_hv(plc_ctx* c, const T* r, const T* D, T* p, T* Hp, bool jac);
// The Gaussian-prior model (Eq. MAPG): gradient through the FFT at delta,
// line-search trial, and the fraction-to-boundary quantity (into sc->bmax).
template <typename T, typename TS, typename TC>
void grad_newton_g(plc_ctx* c, const TS* delta, const double* w, const int32_t* N, double nbar,
                   T* y, T* g, TC* D, TC* r, bool jac);
template <typename T, typename TC>
void newton_update_g(plc_ctx* c, const T* s, const T* y, const T* g, const TC* r, const TC* xi,
                     const TC* D, const int32_t* N, const double* w, double nbar, double tau,
                     bool jac, T* s2, T* y2, T* g2, TC* D2, TC* r2);
template <typename T, typename TC>
void boundary_step(plc_ctx* c, const T* delta, const TC* xi, const int32_t* N);
template <typename TL> void vjp_amplitude(plc_ctx* c, const double* s, const TL* lam);

// Element-wise kernels.
template <typename TC> void cg_init(plc_ctx* c, const double* b, const TC* D, TC* r, bool jac);
// LSQ-Wiener filter start: D = nbar w, r = N - nbar w, CG scalars.
template <typename TC> void lsq_init(plc_ctx* c, const int32_t* N, const double* w, double nbar,
                                     TC* D, TC* r, bool jac);
// rtol2 < 0: the stopping parameters are read from the device scalars.
template <typename TC> void cg_update(plc_ctx* c, TC* x, TC* r, const TC* p, const TC* Hp,
                                      const TC* D, bool jac, double rtol2, int max_iter);
template <typename TC> void diag(plc_ctx* c, const double* s, const double* w, double nbar, TC* D);
template <typename TD, typename TS> void convert(plc_ctx* c, const TS* src, TD* dst);
// Start point of the lognormal solve: the MAP of the same posterior with the
// prior replaced by its diagonal (variance prior_var per cell), cell by cell.
template <typename TS> void diag_start(plc_ctx* c, TS* s, const int32_t* N, const double* w,
                                       double nbar);
// ||g||^2 at the prior mean (s equal to `mean` bit for bit), where the prior
// term vanishes and g = factor w - N: into red[2], and off_mean = 1 when s
// differs from the mean anywhere.
void g0_at_mean(plc_ctx* c, const double* s, const int32_t* N, const double* w, double mean,
                double factor);
// The same for the Gaussian-prior model (delta, Eq. MAPG cell by cell).
template <typename TS> void diag_start_g(plc_ctx* c, TS* delta, const int32_t* N, const double* w,
                                         double nbar);

// Counts a launch and, when timing is on, brackets it with CUDA events.
class LaunchScope {
 public:
  LaunchScope(plc_ctx* c, Site site);
  ~LaunchScope();
 private:
  plc_ctx* c_;
  int slot_;
};
void profile_collect(plc_ctx* c);   // synchronises and accumulates pending timings
void profile_reset(plc_ctx* c, bool timing);
void profile_release(plc_ctx* c);

void build_prior(plc_ctx* c, const double* lk_host, const double* lP_host, int nk);
// Bias multipliers b(|k|) / n^3 from ln k, ln b tables (b_dc for the DC mode).
void build_bias(plc_ctx* c, const double* lk_host, const double* lb_host, int nb, double b_dc);

// Quality measures and matter statistics (stats.cu).  out = {sum ab, sum a^2,
// sum b^2, sum (a-b)^2}; counts[nbins + 3] (below, above, invalid at the end)
// through the device scratch dcounts[nbins + 3]; moments = {mean, variance,
// skewness, excess kurtosis}; table: scratch of 3 (n/2)^2 + 1 doubles for
// the smoothing multipliers.
void compare_fields(plc_ctx* c, const double* a, const double* b, double out[4]);
void log_stats(plc_ctx* c, const double* delta, double lo, double width, int nbins,
               long long* counts, double* moments, unsigned long long* dcounts);
void gaussian_smooth(plc_ctx* c, const double* x, double* y, double radius, double* table);
void reset_ticket(plc_ctx* c);
void read_scalars(plc_ctx* c);    // copies sc -> sc_host and synchronises

}  // namespace plc
