// noalloc.cu -- a Hessian-vector product that allocates no device memory.
//
// Some callers cannot call cudaMalloc: programs whose device memory is all
// reserved up front by an allocator they do not own (a framework's caching
// pool that already holds the GPU), real-time or certified code that forbids
// any allocation after start-up, and plug-ins that run under a host
// application which does not let them create allocations of their own.
// plc_hessvec_noalloc serves them: it computes the same H v as plc_hessvec
// (FP64, n <= 64) with no context, using as scratch one file-scope device
// array, g_noalloc_scratch, that every GPU which loads the library holds
// until the process exits.  The caller passes only inputs and outputs.
//
// The array's name is a host-side stand-in in host code, not a device
// address: the device address is looked up with cudaGetSymbolAddress once
// per device, on the first call made with that device current, and cached.
// A cudaDeviceReset (or anything else that destroys and re-creates the
// device's primary context) reloads the module at a new address, so after
// one the library must be unloaded and loaded again before this entry point
// is called on that device.
#include <mutex>
#include <string>

#include "launch.cuh"

namespace plc {
void set_global_error(const std::string& msg);   // capi.cu
}

namespace {

constexpr int kNoAllocMaxN = 64;          // largest grid side served
constexpr int kNoAllocMaxTable = 1024;    // largest P(k) table
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kSpecBytes =
    sizeof(double2) * (kNoAllocMaxN / 2 + 1) * kNoAllocMaxN * kNoAllocMaxN;
constexpr size_t kMBytes = sizeof(double) * (3 * (kNoAllocMaxN / 2) * (kNoAllocMaxN / 2) + 1);
constexpr size_t kTwBytes = sizeof(double2) * kNoAllocMaxN;
constexpr size_t kOffB = align256(kSpecBytes);
constexpr size_t kOffTw = kOffB + align256(kSpecBytes);
constexpr size_t kOffM = kOffTw + align256(kTwBytes);
constexpr size_t kScratchBytes = kOffM + align256(kMBytes);   // about 4.2 MiB

// The scratch: two half-spectra, the twiddles and the per-|m|^2 inverse
// eigenvalues of the largest grid served.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The passes run with dynamic shared memory below the 48 KB that needs no
// opt-in attribute (this file sets none): twiddles plus two padded tiles of
// the largest line length.
static_assert(sizeof(double2) * (kNoAllocMaxN + 2 * (size_t)kNoAllocMaxN * plc::PassGeom<double>::P) <=
                  48 * 1024,
              "FP64 Stockham tiles of the largest grid must fit the default shared-memory limit");

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Host-computed tables passed by value as a kernel parameter (no copies).
struct SetupArgs {
  int n, nk;
  double box, inv_dc;
  double2 tw[kNoAllocMaxN];
  double lk[kNoAllocMaxTable];
  double lP[kNoAllocMaxTable];
};

// Twiddles and M[m2] = 1 / (lambda n^3), lambda = P(|k|) n^3 / L^3 with P
// linear in (ln k, ln P) between table points; M[0] = inv_dc / n^3.
__global__ void k_noalloc_setup(double2* __restrict__ tw, double* __restrict__ M, SetupArgs a) {
  const int n = a.n;
  const int nm2 = 3 * (n / 2) * (n / 2) + 1;
  const double n3 = (double)n * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm2; i += gridDim.x * blockDim.x) {
    if (i < n) tw[i] = a.tw[i];
    double v;
    if (i == 0) {
      v = a.inv_dc / n3;
    } else {
      const double lnk = log(2.0 * 3.14159265358979323846 / a.box) + 0.5 * log((double)i);
      int lo = 0, hi = a.nk - 1;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.lk[mid] <= lnk) lo = mid; else hi = mid;
      }
      const double t = (lnk - a.lk[lo]) / (a.lk[lo + 1] - a.lk[lo]);
      const double lnP = a.lP[lo] + t * (a.lP[lo + 1] - a.lP[lo]);
      v = 1.0 / (exp(lnP) * n3 / (a.box * a.box * a.box) * n3);
    }
    M[i] = v;
  }
}

plc_status fail(const std::string& msg, plc_status st = PLC_ERR_INVALID_ARG) {
  plc::set_global_error(msg);
  return st;
}

bool valid_noalloc_size(int n) {
  if (n < 4 || n > kNoAllocMaxN || (n & 1)) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

plc::FftPlan noalloc_plan(int n) {
  plc::FftPlan p{};
  p.n = n;
  int a = 0, m = n, b = 0;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  int q = a / 3, rem = a % 3, k = 0;
  if (rem == 1 && q >= 1) { q -= 1; rem = 4; }
  for (int i = 0; i < q; ++i) p.rad[k++] = 8;
  if (rem == 1) p.rad[k++] = 2;
  if (rem == 2) p.rad[k++] = 4;
  if (rem == 4) { p.rad[k++] = 4; p.rad[k++] = 4; }
  for (int i = 0; i < b; ++i) p.rad[k++] = 3;
  p.nst = k;
  int ns = 1;
  for (int i = 0; i < k; ++i) {
    p.ns[i] = ns;
    p.tstep[i] = n / (ns * p.rad[i]);
    p.ns_m[i] = ns > 1 ? plc::make_fastdiv(ns).m : 0u;
    ns *= p.rad[i];
  }
  p.nd = plc::make_fastdiv(n);
  p.f1 = p.f2 = 0;                    // FP64: Stockham stages
  return p;
}

// Device address of the scratch on the current device (looked up once per
// device and cached).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

}  // namespace

extern "C" plc_status plc_hessvec_noalloc(int n, double box, const double* k, const double* P,
                                          int nk, double inv_lambda_dc, const double* s,
                                          const double* w, double nbar, const double* v,
                                          double* Hv, void* cuda_stream) {
  using namespace plc;
  if (!valid_noalloc_size(n))
    return fail("plc_hessvec_noalloc: n must be even, 4..64, with prime factors 2 and 3 only "
                "(its static scratch holds grids up to 64^3)");
  if (!(box > 0.0) || !std::isfinite(box)) return fail("plc_hessvec_noalloc: box must be > 0");
  if (!k || !P || nk < 2 || nk > kNoAllocMaxTable)
    return fail("plc_hessvec_noalloc: need host k, P arrays with 2 <= nk <= 1024");
  for (int i = 0; i < nk; ++i) {
    if (!(k[i] > 0.0) || !std::isfinite(k[i]) || !(P[i] > 0.0) || !std::isfinite(P[i]))
      return fail("plc_hessvec_noalloc: k and P must be finite and > 0");
    if (i && !(k[i] > k[i - 1])) return fail("plc_hessvec_noalloc: k must be strictly ascending");
  }
  const double kf = 2.0 * M_PI / box, kmax = std::sqrt(3.0) * M_PI * n / box;
  if (k[0] > kf * (1.0 + 1e-12) || k[nk - 1] < kmax * (1.0 - 1e-12))
    return fail("plc_hessvec_noalloc: P(k) table must cover [2 pi / L, sqrt(3) pi n / L]");
  if (!(inv_lambda_dc >= 0.0) || !std::isfinite(inv_lambda_dc))
    return fail("plc_hessvec_noalloc: inv_lambda_dc must be finite and >= 0");
  if (!(nbar > 0.0) || !std::isfinite(nbar)) return fail("plc_hessvec_noalloc: nbar must be > 0");
  const void* fields[] = {s, v, Hv};
  for (const void* f : fields)
    if (!f || (reinterpret_cast<uintptr_t>(f) & 15u))
      return fail("plc_hessvec_noalloc: s, v, Hv must be non-NULL and 16-byte aligned");
  if (w && (reinterpret_cast<uintptr_t>(w) & 15u))
    return fail("plc_hessvec_noalloc: w must be 16-byte aligned");

  // An error left pending by an earlier, unrelated call would be reported
  // (and cleared) by the launch check below as if it were this call's:
  // refuse to run while one is pending, and leave it for its owner.
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return fail(std::string("plc_hessvec_noalloc: a CUDA error is pending from an earlier call "
                            "(not cleared): ") + cudaGetErrorString(e), PLC_ERR_CUDA);
  unsigned char* base = nullptr;
  e = scratch_address(&base);
  if (e != cudaSuccess)
    return fail(std::string("plc_hessvec_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e),
                PLC_ERR_CUDA);
  double2* A = reinterpret_cast<double2*>(base);
  double2* B = reinterpret_cast<double2*>(base + kOffB);
  double2* tw = reinterpret_cast<double2*>(base + kOffTw);
  double* M = reinterpret_cast<double*>(base + kOffM);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  SetupArgs a;
  a.n = n;
  a.nk = nk;
  a.box = box;
  a.inv_dc = inv_lambda_dc;
  for (int m = 0; m < n; ++m) {
    const double ang = 2.0 * M_PI * (double)m / (double)n;
    a.tw[m] = make_double2(std::cos(ang), -std::sin(ang));
  }
  for (int i = 0; i < nk; ++i) {
    a.lk[i] = std::log(k[i]);
    a.lP[i] = std::log(P[i]);
  }
  const int nm2 = 3 * (n / 2) * (n / 2) + 1;
  k_noalloc_setup<<<(nm2 + kThreads - 1) / kThreads, kThreads, 0, st>>>(tw, M, a);

  using G = PassGeom<double>;
  using Pro = ProLoad<double>;
  using Epi = EpiHessS<double>;
  const FftPlan plan = noalloc_plan(n);
  const int h = n / 2 + 1;
  const size_t sm = G::smem_bytes(plan);
  const dim3 gx((n + G::RY - 1) / G::RY, n), gy((n + G::L - 1) / G::L, h);
  const Pro pro{v};
  const Epi epi{s, w, nbar, v, Hv};
  k_xf<double, Pro><<<gx, kThreads, sm, st>>>(pro, A, plan, tw, nullptr);
  k_yf<double><<<gy, kThreads, sm, st>>>(A, B, plan, tw, nullptr);
  k_z<double><<<gy, kThreads, sm, st>>>(B, M, 0, plan, tw, nullptr);
  k_yi<double><<<gy, kThreads, sm, st>>>(B, A, plan, tw, nullptr);
  k_xi<double, Epi, FinNone><<<gx, kThreads, sm, st>>>(
      A, epi, FinNone{}, RedArgs{nullptr, nullptr}, plan, tw, nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(std::string("plc_hessvec_noalloc: launch: ") + cudaGetErrorString(e), PLC_ERR_CUDA);
  return PLC_OK;
}
