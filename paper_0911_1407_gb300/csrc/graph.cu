// graph.cu -- the Newton-Krylov MAP solve of solver.cu, driven from the device.
//
// The host driver (solver.cu) reads the device scalars after every gradient,
// CG chunk and line-search trial to take its decisions.  Here the same
// decisions are taken by one-thread control kernels that read the device
// scalars and set the conditions of CUDA graph conditional nodes, so that a
// whole solve is one graph launch with no host round trip:
//
//   init:  [PLC_MIXED: s -> FP32]  FFT gradient  ctl_init
//   WHILE newton:
//     ctl_head                        FP32 -> FP64 switch?
//     IF switch:   s -> FP64, FP64 FFT gradient, ctl_switched
//     ctl_decide                      stop test, iteration cap, CG tolerance
//     SWITCH step (precision phase, current field set):
//       WHILE cg:  Hv pipeline, CG update, ctl_cg
//       ctl_step                      tau of Eq. (New5) and the step cap
//       WHILE ls:  Newton trial, ctl_ls (Armijo test or halving)
//   write-back of s to the caller's buffer
//
// The Newton state alternates between two field sets A and B; steps A -> B
// and B -> A are captured as separate bodies of the SWITCH node (times the
// two precision phases for PLC_MIXED), and the control block records which
// set is current.  Every loop is bounded by a counter in its control kernel
// (max_cg CG iterations, 30 trials, max_newton + 4 passes of the Newton
// loop), and every handle is reset to 0 at each launch, so a launch always
// ends.  The iteration, tolerances and tests are those of newton_map; the
// two drivers take the same steps.
//
// A batch of contexts (independent mocks of any sizes) is one graph with one
// such chain per context, launched once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "ctx.h"
#include "graph.h"

namespace plc {

namespace {

using Handle = cudaGraphConditionalHandle;

// Per-context control block (device memory).
struct DevCtl {
  // options (written by ctl_init at every launch)
  double tol, mixed_switch, eta_max, step_cap, g0_opt;
  int max_newton, max_cg, mixed;
  // state
  double g0, prev_rel, f0, xg, scale, eps;
  int it, q, par, fp64, stop, status, loops, cg_count;
  int check;   // the FP32 gradient passed the stopping test at the switch
  // statistics
  long long cg_iters, grad_evals, grad_ffts, grad_ffts_fp64, kernels;
  double grad_rel, neg_logpost;
};

struct CtlOpts {
  double tol, mixed_switch, eta_max, step_cap, g0_opt;
  int max_newton, max_cg, mixed, fp64;
};

struct StepHandles {
  Handle cg[4], ls[4];
};

__device__ __forceinline__ double f_of(const DevScalars* sc) { return 0.5 * sc->red[0] + sc->red[1]; }
__device__ __forceinline__ double scale_of(const DevScalars* sc) {
  return (sc->red[1] + sc->red[3]) + sc->red[4] + fabs(f_of(sc));
}

// first: 0 the gradient at the caller's start ran, 1 it ran when the start
// was off the prior mean (off_mean), 2 it did not run (g0 given), 3 it did
// not run (the start is the prior mean by definition); nk_first: its
// kernels when it ran conditionally.  g0 comes from red[2]: that gradient's, or the
// transform-free one at the prior mean.
__global__ void k_ctl_init(DevCtl* t, const DevScalars* sc, CtlOpts o, Handle h_newton, int nk,
                           int first, int nk_first) {
  const int ran = first == 0 ? 1 : (first == 1 ? sc->off_mean : 0);
  t->tol = o.tol;
  t->mixed_switch = o.mixed_switch;
  t->eta_max = o.eta_max;
  t->step_cap = o.step_cap;
  t->g0_opt = o.g0_opt;
  t->max_newton = o.max_newton;
  t->max_cg = o.max_cg;
  t->mixed = o.mixed;
  t->fp64 = o.fp64;
  t->g0 = o.g0_opt > 0.0 ? o.g0_opt : sqrt(sc->red[2]);
  t->prev_rel = 1.0;
  t->f0 = t->xg = t->scale = t->eps = 0.0;
  t->it = t->q = t->par = t->stop = t->loops = t->cg_count = 0;
  t->status = PLC_OK;
  t->cg_iters = 0;
  t->grad_evals = ran;
  t->grad_ffts = ran;
  t->grad_ffts_fp64 = ran && o.fp64 ? 1 : 0;
  t->kernels = nk + (first == 1 && ran ? nk_first : 0);
  t->grad_rel = 0.0;
  t->neg_logpost = 0.0;
  cudaGraphSetConditional(h_newton, 1);
}

// The first gradient runs only when the start is off the prior mean.
__global__ void k_ctl_first(const DevScalars* sc, Handle h_first) {
  cudaGraphSetConditional(h_first, sc->off_mean ? 1u : 0u);
}

// A second FFT gradient at the start point (the first one gave g0).
__global__ void k_ctl_restart(DevCtl* t, int nk, int fp64) {
  t->kernels += nk;
  t->grad_evals += 1;
  t->grad_ffts += 1;
  t->grad_ffts_fp64 += fp64;
}

// FP32 -> FP64 switch (PLC_MIXED): below the switch point, at the
// tolerance, or when an FP32 step below 1e-3 failed to halve ||g||.
__global__ void k_ctl_head(DevCtl* t, const DevScalars* sc, Handle h_switch, int nk) {
  t->kernels += nk;
  t->loops += 1;
  const double gnorm = sqrt(sc->red[2]), f = f_of(sc);
  int sw = 0;
  // a non-finite g0 (NaN or Inf in the caller's start or in w) would make
  // every relative norm look converged
  if (!isfinite(gnorm) || !isfinite(f) || !isfinite(t->g0)) {
    t->stop = 1;
    t->status = PLC_ERR_NONFINITE;
  } else if (t->mixed && !t->fp64) {
    const double rel = t->g0 > 0.0 ? gnorm / t->g0 : 0.0;
    sw = (rel < t->mixed_switch || rel < t->tol ||
          (t->it > 0 && rel < 1e-3 && rel > 0.5 * t->prev_rel)) ? 1 : 0;
    t->check = rel < t->tol ? 1 : 0;
  }
  cudaGraphSetConditional(h_switch, sw);
}

__global__ void k_ctl_switched(DevCtl* t, int nk, int count_grad) {
  t->kernels += nk;
  t->fp64 = 1;
  t->par = 0;
  t->grad_evals += count_grad;
  t->grad_ffts += count_grad;
  t->grad_ffts_fp64 += count_grad;
}

// After the FP64 gradient's sums alone (the switch's check): its fields are
// needed, and the full gradient runs, unless the FP32 gradient passed the
// stopping test and these sums pass it too (the decision kernel then ends
// the solve on the same sums).
__global__ void k_ctl_check(DevCtl* t, const DevScalars* sc, Handle h_full, int nk) {
  t->kernels += nk;
  t->grad_evals += 1;
  t->grad_ffts += 1;
  t->grad_ffts_fp64 += 1;
  const double gnorm = sqrt(sc->red[2]), f = f_of(sc);
  const bool pass = t->check && isfinite(gnorm) && isfinite(f) && t->g0 > 0.0 &&
                    gnorm / t->g0 < t->tol;
  cudaGraphSetConditional(h_full, pass ? 0u : 1u);
}

// Before the switch's check: run it only when the FP32 gradient passed the
// stopping test; the full FP64 gradient follows otherwise (k_ctl_check
// decides when the check runs).
__global__ void k_ctl_presw(const DevCtl* t, Handle h_chk, Handle h_full) {
  cudaGraphSetConditional(h_chk, t->check ? 1u : 0u);
  cudaGraphSetConditional(h_full, t->check ? 0u : 1u);
}

__global__ void k_ctl_full(DevCtl* t, int nk) {
  t->kernels += nk;
  t->grad_evals += 1;
  t->grad_ffts += 1;
  t->grad_ffts_fp64 += 1;
}

// Stop test and the CG of the next step; selects the SWITCH body.
__global__ void k_ctl_decide(DevCtl* t, DevScalars* sc, Handle h_newton, Handle h_step,
                             StepHandles hs, int nk) {
  t->kernels += nk;
  int step = -1;
  if (!t->stop) {
    const double gnorm = sqrt(sc->red[2]), f = f_of(sc);
    if (!isfinite(gnorm) || !isfinite(f) || !isfinite(t->g0)) {
      t->stop = 1;
      t->status = PLC_ERR_NONFINITE;
    } else {
      const double rel = t->g0 > 0.0 ? gnorm / t->g0 : 0.0;
      t->grad_rel = rel;
      t->neg_logpost = f;
      t->prev_rel = rel;
      if (rel < t->tol) {
        t->stop = 1;
      } else if (t->it >= t->max_newton || t->loops > t->max_newton + 4) {
        t->stop = 1;
        t->status = PLC_ERR_NOT_CONVERGED;
      } else {
        const double eta = fmin(t->eta_max, fmax(sqrt(rel), 0.3 * t->tol / rel));
        sc->rtol2 = eta * eta;
        sc->max_iter = t->max_cg;
        t->cg_count = 0;
        t->f0 = f;
        t->scale = scale_of(sc);
        step = (t->mixed && t->fp64 ? 2 : 0) + t->par;
      }
    }
  }
  cudaGraphSetConditional(h_newton, t->stop ? 0 : 1);
  cudaGraphSetConditional(h_step, step < 0 ? 255u : (unsigned)step);
  if (step >= 0) cudaGraphSetConditional(hs.cg[step], sc->done ? 0 : 1);
}

__global__ void k_ctl_cg(DevCtl* t, const DevScalars* sc, Handle h_cg, int nk) {
  t->kernels += nk;
  t->cg_count += 1;
  cudaGraphSetConditional(h_cg, (!sc->done && t->cg_count < t->max_cg) ? 1 : 0);
}

// Step length of Eq. (New5) from the CG sums, capped by max |tau xi|.
__global__ void k_ctl_step(DevCtl* t, DevScalars* sc, Handle h_ls, Handle h_newton, int nk) {
  t->kernels += nk;
  const int iters = sc->iter;
  t->cg_iters += iters;
  if (iters == 0) {
    t->stop = 1;
    t->status = sc->breakdown ? PLC_ERR_CG_BREAKDOWN : PLC_OK;
    cudaGraphSetConditional(h_newton, 0);
    cudaGraphSetConditional(h_ls, 0);
    return;
  }
  const double xg = -sc->xb, xHx = sc->xHx, xmax = sc->xmax;
  double tau = -xg / xHx;
  if (tau * xmax > t->step_cap) tau = t->step_cap / xmax;
  t->xg = xg;
  t->eps = t->fp64 ? 1e-13 : 1e-6;
  t->q = 0;
  sc->tau = tau;
  cudaGraphSetConditional(h_ls, 1);
}

// Armijo test of the trial just evaluated; accept (the trial's field set
// becomes current) or halve tau.  The 30th trial is accepted as it is.
__global__ void k_ctl_ls(DevCtl* t, DevScalars* sc, Handle h_ls, int nk) {
  t->kernels += nk;
  t->grad_evals += 1;
  const double f = f_of(sc), tau = sc->tau;
  const bool ok = f <= t->f0 + 1e-4 * tau * t->xg || -tau * t->xg < t->eps * t->scale || t->q >= 29;
  if (ok) {
    t->par ^= 1;
    t->it += 1;
    cudaGraphSetConditional(h_ls, 0);
  } else {
    sc->tau = 0.5 * tau;
    t->q += 1;
    cudaGraphSetConditional(h_ls, 1);
  }
}

// Leave the current iterate in the caller's FP64 buffer (field set A of the
// FP64 phase is that buffer itself).
__global__ void k_writeback(const DevCtl* t, double* __restrict__ s_out,
                            const float* __restrict__ s32a, const float* __restrict__ s32b,
                            const double* __restrict__ s64b, size_t n3) {
  const int fp64 = t->fp64, par = t->par;
  if (fp64 && par == 0) return;
  const float* s32 = par ? s32b : s32a;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x)
    s_out[i] = fp64 ? s64b[i] : (double)s32[i];
}

// s (FP64) <- the current FP32 iterate at the switch.
__global__ void k_to_fp64(const DevCtl* t, double* __restrict__ s_out, const float* __restrict__ s32a,
                          const float* __restrict__ s32b, size_t n3) {
  const float* s32 = t->par ? s32b : s32a;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3;
       i += (size_t)gridDim.x * blockDim.x)
    s_out[i] = (double)s32[i];
}

long long total_launches(const plc_ctx* c) {
  long long k = 0;
  for (int i = 0; i < S_NSITES; ++i) k += c->prof.launches[i];
  return k;
}

// Add a conditional node behind the current capture position of `st` and
// make it the new position; returns its body graph(s).
void add_conditional(cudaStream_t st, Handle h, cudaGraphConditionalNodeType type, unsigned size,
                     cudaGraph_t* bodies) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  check(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &nd), "capture info");
  if (cs != cudaStreamCaptureStatusActive) check(cudaErrorStreamCaptureInvalidated, "capture state");
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = size;
  cudaGraphNode_t node;
  check(cudaGraphAddNode(&node, g, deps, edges, nd, &p), "add conditional node");
  for (unsigned i = 0; i < size; ++i) bodies[i] = p.conditional.phGraph_out[i];
  check(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
        "capture dependencies");
}

// Capture what `f` enqueues on the context into `body` through stream `st`.
template <typename F> void capture_into(plc_ctx* c, cudaGraph_t body, cudaStream_t st, F&& f) {
  check(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
        "begin capture");
  cudaStream_t saved = c->stream;
  c->stream = st;
  try {
    f();
  } catch (...) {
    c->stream = saved;
    cudaGraph_t g;
    (void)cudaStreamEndCapture(st, &g);
    throw;
  }
  c->stream = saved;
  cudaGraph_t g;
  check(cudaStreamEndCapture(st, &g), "end capture");
}

template <typename T> T* as(void* p) { return static_cast<T*>(p); }

struct Fields {
  void* s;
  void* y;
  void* g;
  void* D;
  void* r;
};

// Capture one Newton step from field set `cur` to `alt` in precision T (CG
// fields TC) into the current capture of stream level `lv`.
template <typename T, typename TC>
void capture_step(plc_ctx* c, const std::vector<cudaStream_t>& st, int lv, DevCtl* t,
                  const Fields& cur, const Fields& alt, Handle h_cg, Handle h_ls, Handle h_newton,
                  const int32_t* N, const double* w, double nbar, bool jac) {
  void** F = c->wf;
  TC* x = as<TC>(F[10]);
  TC* p = as<TC>(F[11]);
  TC* Hp = as<TC>(F[12]);
  cudaGraph_t body;
  add_conditional(st[lv], h_cg, cudaGraphCondTypeWhile, 1, &body);
  capture_into(c, body, st[lv + 1], [&]() {
    const long long k0 = total_launches(c);
    cg_hv<TC>(c, as<TC>(cur.r), as<TC>(cur.D), p, Hp, jac);
    cg_update<TC>(c, x, as<TC>(cur.r), p, Hp, as<TC>(cur.D), jac, -1.0, 0);
    const int nk = (int)(total_launches(c) - k0) + 1;
    k_ctl_cg<<<1, 1, 0, c->stream>>>(t, c->sc, h_cg, nk);
    check(cudaGetLastError(), "k_ctl_cg");
  });
  k_ctl_step<<<1, 1, 0, st[lv]>>>(t, c->sc, h_ls, h_newton, 1);
  check(cudaGetLastError(), "k_ctl_step");
  add_conditional(st[lv], h_ls, cudaGraphCondTypeWhile, 1, &body);
  capture_into(c, body, st[lv + 1], [&]() {
    const long long k0 = total_launches(c);
    // the FP32 phase keeps no g: the trial forms it again from y, D and N
    constexpr bool kNoG = std::is_same<T, float>::value;
    newton_update<T, TC>(c, as<T>(cur.s), as<T>(cur.y), kNoG ? nullptr : as<T>(cur.g),
                         as<TC>(cur.r), x, as<TC>(cur.D), N, w, nbar, 0.0, jac, as<T>(alt.s),
                         as<T>(alt.y), kNoG ? nullptr : as<T>(alt.g), as<TC>(alt.D),
                         as<TC>(alt.r), &c->sc->tau);
    const int nk = (int)(total_launches(c) - k0) + 1;
    k_ctl_ls<<<1, 1, 0, c->stream>>>(t, c->sc, h_ls, nk);
    check(cudaGetLastError(), "k_ctl_ls");
  });
}

}  // namespace

// One instantiated single-solve graph and the key it was captured for.
struct SolveExec {
  cudaGraphExec_t exec = nullptr;
  const void* key_ptr[3] = {};
  double key_val[9] = {};
  int key_int[4] = {};
  unsigned long long used = 0;    // last use, for eviction
};

// Device state of the device-driven solve of one context: the control block
// and a few cached graphs (a caller that alternates between buffer sets,
// e.g. to overlap copies with solves, relaunches each set's graph).
struct GraphSolve {
  static constexpr int kCache = 4;
  DevCtl* ctl = nullptr;          // device
  DevCtl* ctl_host = nullptr;     // pinned copy
  SolveExec cache[kCache];
  unsigned long long clock = 0;
};

static GraphSolve* graph_state(plc_ctx* c) {
  if (!c->graph) {
    GraphSolve* g = new GraphSolve();
    c->graph = g;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&g->ctl), sizeof(DevCtl));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&g->ctl_host), sizeof(DevCtl));
    check(e, "control block allocation");
  }
  return static_cast<GraphSolve*>(c->graph);
}

void graph_release(plc_ctx* c) {
  GraphSolve* g = static_cast<GraphSolve*>(c->graph);
  if (!g) return;
  for (SolveExec& e : g->cache)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  if (g->ctl) cudaFree(g->ctl);
  if (g->ctl_host) cudaFreeHost(g->ctl_host);
  delete g;
  c->graph = nullptr;
}

// Append the whole device-driven solve of context c to `top` (a new root
// chain), capturing through the streams st[0..5].
template <typename TC>
void capture_solve(plc_ctx* c, cudaGraph_t top, const std::vector<cudaStream_t>& st,
                   const int32_t* N, const double* w, double nbar, double* s_out,
                   const plc_opts& o) {
  constexpr bool kMixed = std::is_same<TC, float>::value;
  GraphSolve* gs = graph_state(c);
  DevCtl* t = gs->ctl;
  void** F = c->wf;
  const bool jac = o.precond == 1;
  const bool start64 = !kMixed || !(o.mixed_switch < 1.0);
  const Fields f32a{F[0], F[2], F[4], F[6], F[8]}, f32b{F[1], F[3], F[5], F[7], F[9]};
  const Fields f64a{s_out, F[2], F[4], F[6], F[8]}, f64b{F[1], F[3], F[5], F[7], F[9]};

  Handle h_newton, h_switch, h_step, h_first, h_full, h_chk;
  StepHandles hs;
  auto mk = [&](Handle* h) {
    check(cudaGraphConditionalHandleCreate(h, top, 0, cudaGraphCondAssignDefault), "handle");
  };
  mk(&h_newton);
  mk(&h_switch);
  mk(&h_step);
  // the first gradient's IF node, when there is one (a handle must belong to
  // a conditional node for the graph to instantiate)
  const int first = o.start == 0 ? 0 : (o.g0_norm > 0.0 ? 2 : (o.start == 2 ? 3 : 1));
  if (first == 1) mk(&h_first);
  // the switch's sums-only check: mixed solves of lengths with float-float
  // transforms (a four-step schedule)
  bool has_check = false;
  if constexpr (kMixed) {
    for (const FourStepShape& q : kFourStep)
      if (q.n == c->n && q.f1 == c->plan.f1 && q.f2 == c->plan.f2) has_check = true;
  }
  if (has_check) {
    mk(&h_full);
    mk(&h_chk);
  }
  const int nvar = kMixed ? 4 : 2;
  for (int v = 0; v < nvar; ++v) {
    mk(&hs.cg[v]);
    mk(&hs.ls[v]);
  }
  CtlOpts co{o.tol, o.mixed_switch, o.eta_max, o.step_cap, o.g0_norm, o.max_newton, o.max_cg,
             kMixed ? 1 : 0, start64 ? 1 : 0};
  const bool timing = c->prof.timing;
  c->prof.timing = false;   // no event nodes in the graph

  capture_into(c, top, st[0], [&]() {
    const long long k0 = total_launches(c);
    reset_ticket(c);
    auto first_gradient = [&]() {
      if (start64) {
        grad_newton<double, double, TC>(c, s_out, w, N, nbar, as<double>(f64a.y),
                                        as<double>(f64a.g), as<TC>(f64a.D), as<TC>(f64a.r), jac);
      } else if constexpr (kMixed) {
        convert<float, double>(c, s_out, as<float>(f32a.s));
        grad_newton<float, float, float>(c, as<float>(f32a.s), w, N, nbar, as<float>(f32a.y),
                                         nullptr, as<float>(f32a.D),
                                         as<float>(f32a.r), jac);
      }
    };
    // ||g0|| at the caller's start; with the diagonal start the gradient
    // there serves only this norm: none when g0_norm is given, and at the
    // prior mean the transform-free one (the FFT gradient runs, in an IF
    // node, only when the start is off the mean)
    int nk_first = 0, nk_ctl = 1;
    if (first == 1) {
      nk_ctl = 2;
      g0_at_mean(c, s_out, N, w, c->mu, nbar * std::exp(c->mu));
      k_ctl_first<<<1, 1, 0, c->stream>>>(c->sc, h_first);
      check(cudaGetLastError(), "k_ctl_first");
      cudaGraph_t fbody;
      add_conditional(c->stream, h_first, cudaGraphCondTypeIf, 1, &fbody);
      capture_into(c, fbody, st[1], [&]() {
        const long long k1 = total_launches(c);
        first_gradient();
        nk_first = (int)(total_launches(c) - k1);
      });
    } else if (first == 3) {
      g0_at_mean(c, nullptr, N, w, c->mu, nbar * std::exp(c->mu));
    } else if (first == 0) {
      first_gradient();
    }
    const int nk = (int)(total_launches(c) - k0) - nk_first + nk_ctl;
    k_ctl_init<<<1, 1, 0, c->stream>>>(t, c->sc, co, h_newton, nk, first, nk_first);
    check(cudaGetLastError(), "k_ctl_init");
    if (o.start >= 1) {
      // iterate from the per-cell diagonal-prior MAP (g0 stays at s_in)
      const long long k1 = total_launches(c);
      if (start64) {
        diag_start<double>(c, s_out, N, w, nbar);
        grad_newton<double, double, TC>(c, s_out, w, N, nbar, as<double>(f64a.y),
                                        as<double>(f64a.g), as<TC>(f64a.D), as<TC>(f64a.r), jac);
      } else if constexpr (kMixed) {
        diag_start<float>(c, as<float>(f32a.s), N, w, nbar);
        grad_newton<float, float, float>(c, as<float>(f32a.s), w, N, nbar, as<float>(f32a.y),
                                         nullptr, as<float>(f32a.D), as<float>(f32a.r),
                                         jac);
      }
      const int nk1 = (int)(total_launches(c) - k1) + 1;
      k_ctl_restart<<<1, 1, 0, c->stream>>>(t, nk1, start64 ? 1 : 0);
      check(cudaGetLastError(), "k_ctl_restart");
    }

    cudaGraph_t nbody;
    add_conditional(c->stream, h_newton, cudaGraphCondTypeWhile, 1, &nbody);
    capture_into(c, nbody, st[1], [&]() {
      k_ctl_head<<<1, 1, 0, c->stream>>>(t, c->sc, h_switch, 1);
      check(cudaGetLastError(), "k_ctl_head");
      cudaGraph_t sbody;
      add_conditional(c->stream, h_switch, cudaGraphCondTypeIf, 1, &sbody);
      if constexpr (kMixed) {
        capture_into(c, sbody, st[2], [&]() {
          const long long k1 = total_launches(c);
          k_to_fp64<<<pointwise_blocks((long long)c->n3(), c->sms), kThreads, 0, c->stream>>>(
              t, s_out, as<float>(f32a.s), as<float>(f32b.s), c->n3());
          check(cudaGetLastError(), "k_to_fp64");
          auto full = [&]() {
            grad_newton<double, double, TC>(c, s_out, w, N, nbar, as<double>(f64a.y),
                                            as<double>(f64a.g), as<TC>(f64a.D),
                                            as<TC>(f64a.r), jac);
          };
          if (has_check) {
            // when the FP32 gradient passed the stopping test, the FP64
            // gradient's sums first (an IF node); the full gradient in a
            // second IF node, unless those sums pass it too
            k_ctl_presw<<<1, 1, 0, c->stream>>>(t, h_chk, h_full);
            check(cudaGetLastError(), "k_ctl_presw");
            cudaGraph_t cbody, fbody;
            add_conditional(c->stream, h_chk, cudaGraphCondTypeIf, 1, &cbody);
            capture_into(c, cbody, st[3], [&]() {
              const long long k2 = total_launches(c);
              grad_sums_ff(c, s_out, w, N, nbar, jac);
              const int nk_check = (int)(total_launches(c) - k2) + 1;
              k_ctl_check<<<1, 1, 0, c->stream>>>(t, c->sc, h_full, nk_check);
              check(cudaGetLastError(), "k_ctl_check");
            });
            add_conditional(c->stream, h_full, cudaGraphCondTypeIf, 1, &fbody);
            capture_into(c, fbody, st[3], [&]() {
              const long long k2 = total_launches(c);
              full();
              const int nk_full = (int)(total_launches(c) - k2) + 1;
              k_ctl_full<<<1, 1, 0, c->stream>>>(t, nk_full);
              check(cudaGetLastError(), "k_ctl_full");
            });
            // it, k_to_fp64 and k_ctl_presw
            k_ctl_switched<<<1, 1, 0, c->stream>>>(t, 3, 0);
          } else {
            full();
            const int nk1 = (int)(total_launches(c) - k1) + 2;
            k_ctl_switched<<<1, 1, 0, c->stream>>>(t, nk1, 1);
          }
          check(cudaGetLastError(), "k_ctl_switched");
        });
      } else {
        capture_into(c, sbody, st[2], [&]() {
          k_ctl_switched<<<1, 1, 0, c->stream>>>(t, 1, 1);   // never taken: FP64 throughout
          check(cudaGetLastError(), "k_ctl_switched");
        });
      }
      k_ctl_decide<<<1, 1, 0, c->stream>>>(t, c->sc, h_newton, h_step, hs, 1);
      check(cudaGetLastError(), "k_ctl_decide");
      cudaGraph_t bodies[4];
      add_conditional(c->stream, h_step, cudaGraphCondTypeSwitch, nvar, bodies);
      for (int v = 0; v < nvar; ++v) {
        capture_into(c, bodies[v], st[2], [&]() {
          const bool b2a = (v & 1) != 0;
          if (kMixed && v < 2) {
            if constexpr (kMixed)
              capture_step<float, float>(c, st, 2, t, b2a ? f32b : f32a, b2a ? f32a : f32b,
                                         hs.cg[v], hs.ls[v], h_newton, N, w, nbar, jac);
          } else {
            capture_step<double, TC>(c, st, 2, t, b2a ? f64b : f64a, b2a ? f64a : f64b, hs.cg[v],
                                     hs.ls[v], h_newton, N, w, nbar, jac);
          }
        });
      }
    });
    k_writeback<<<pointwise_blocks((long long)c->n3(), c->sms), kThreads, 0, c->stream>>>(
        t, s_out, as<float>(f32a.s), as<float>(f32b.s), as<double>(f64b.s), c->n3());
    check(cudaGetLastError(), "k_writeback");
  });
  c->prof.timing = timing;
}

namespace {

struct Streams {
  std::vector<cudaStream_t> s;
  Streams() : s(6, nullptr) {
    for (auto& x : s) check(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "capture stream");
  }
  ~Streams() {
    for (auto& x : s)
      if (x) cudaStreamDestroy(x);
  }
};

void fill_stats(const DevCtl& h, plc_stats* st, double ms) {
  if (!st) return;
  std::memset(st, 0, sizeof(*st));
  st->newton_iters = h.it;
  st->cg_iters = (int)h.cg_iters;
  st->hv_count = (int)h.cg_iters;
  st->grad_evals = (int)h.grad_evals;
  st->grad_ffts = (int)h.grad_ffts;
  st->grad_ffts_fp64 = (int)h.grad_ffts_fp64;
  st->grad_rel = h.grad_rel;
  st->g0_norm = h.g0;
  st->neg_logpost = h.neg_logpost;
  st->kernels = h.kernels + 1;   // and the write-back
  st->ms = ms;
}

bool same_key(const SolveExec& g, const void* const* p, const double* v, const int* k) {
  return g.exec && std::equal(p, p + 3, g.key_ptr) && std::equal(v, v + 9, g.key_val) &&
         std::equal(k, k + 4, g.key_int);
}

}  // namespace

template <typename TC>
plc_status newton_map_graph(plc_ctx* c, const int32_t* N, const double* w, double nbar,
                            double* s_out, const plc_opts& o, plc_stats* st) {
  const auto t0 = std::chrono::steady_clock::now();
  GraphSolve* gs = graph_state(c);
  const void* kp[3] = {N, w, s_out};
  const double kv[9] = {nbar, o.tol, o.g0_norm, o.step_cap, o.eta_max, o.mixed_switch, c->mu,
                        c->jac_c, c->prior_var};
  const int ki[4] = {o.max_newton, o.max_cg, o.precond * 3 + o.start,
                     c->plan.f1 * 64 + c->plan.f2};
  SolveExec* e = nullptr;
  for (SolveExec& x : gs->cache)
    if (same_key(x, kp, kv, ki)) e = &x;
  if (!e) {
    // capture into the least recently used slot
    e = &gs->cache[0];
    for (SolveExec& x : gs->cache)
      if (x.used < e->used) e = &x;
    if (e->exec) {
      cudaGraphExecDestroy(e->exec);
      e->exec = nullptr;
    }
    Streams ss;
    cudaGraph_t top;
    check(cudaGraphCreate(&top, 0), "graph create");
    try {
      capture_solve<TC>(c, top, ss.s, N, w, nbar, s_out, o);
      check(cudaGraphInstantiate(&e->exec, top, 0), "graph instantiate");
    } catch (...) {
      cudaGraphDestroy(top);
      throw;
    }
    cudaGraphDestroy(top);
    std::copy(kp, kp + 3, e->key_ptr);
    std::copy(kv, kv + 9, e->key_val);
    std::copy(ki, ki + 4, e->key_int);
  }
  e->used = ++gs->clock;
  check(cudaGraphLaunch(e->exec, c->stream), "graph launch");
  check(cudaMemcpyAsync(gs->ctl_host, gs->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream),
        "control block");
  check(cudaStreamSynchronize(c->stream), "stream synchronize");
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  fill_stats(*gs->ctl_host, st, ms);
  return static_cast<plc_status>(gs->ctl_host->status);
}

template plc_status newton_map_graph<double>(plc_ctx*, const int32_t*, const double*, double,
                                             double*, const plc_opts&, plc_stats*);
template plc_status newton_map_graph<float>(plc_ctx*, const int32_t*, const double*, double,
                                            double*, const plc_opts&, plc_stats*);

// A batch: one graph holding the solve chain of every context.
BatchGraph::~BatchGraph() {
  if (exec) cudaGraphExecDestroy(exec);
}

plc_status batch_map(BatchGraph* b, const std::vector<plc_ctx*>& cs, const int32_t* const* N,
                     const double* const* w, const double* nbar, double* const* s,
                     const plc_opts& o, plc_stats* stats, cudaStream_t stream) {
  const auto t0 = std::chrono::steady_clock::now();
  const size_t m = cs.size();
  std::vector<const void*> key;
  for (size_t i = 0; i < m; ++i) {
    key.push_back(N[i]);
    key.push_back(w ? w[i] : nullptr);
    key.push_back(s[i]);
  }
  std::vector<double> kv{o.tol, o.g0_norm, o.step_cap, o.eta_max, o.mixed_switch,
                         (double)o.max_newton, (double)o.max_cg, (double)o.precond,
                         (double)o.start};
  for (size_t i = 0; i < m; ++i) {
    kv.push_back(nbar[i]);
    kv.push_back(cs[i]->mu);
    kv.push_back(cs[i]->jac_c);
    kv.push_back(cs[i]->prior_var);
    kv.push_back((double)(cs[i]->plan.f1 * 64 + cs[i]->plan.f2));
  }
  if (!b->exec || key != b->key || kv != b->key_val) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    Streams ss;
    cudaGraph_t top;
    check(cudaGraphCreate(&top, 0), "graph create");
    try {
      for (size_t i = 0; i < m; ++i) {
        const double* wi = w ? w[i] : nullptr;
        if (cs[i]->precision == PLC_FP64)
          capture_solve<double>(cs[i], top, ss.s, N[i], wi, nbar[i], s[i], o);
        else
          capture_solve<float>(cs[i], top, ss.s, N[i], wi, nbar[i], s[i], o);
      }
      check(cudaGraphInstantiate(&b->exec, top, 0), "graph instantiate");
    } catch (...) {
      cudaGraphDestroy(top);
      throw;
    }
    cudaGraphDestroy(top);
    b->key = key;
    b->key_val = kv;
  }
  check(cudaGraphLaunch(b->exec, stream), "graph launch");
  for (size_t i = 0; i < m; ++i) {
    GraphSolve* gs = graph_state(cs[i]);
    check(cudaMemcpyAsync(gs->ctl_host, gs->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, stream),
          "control block");
  }
  check(cudaStreamSynchronize(stream), "stream synchronize");
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  plc_status worst = PLC_OK;
  for (size_t i = 0; i < m; ++i) {
    const DevCtl& h = *graph_state(cs[i])->ctl_host;
    if (stats) fill_stats(h, &stats[i], ms);
    if (h.status != PLC_OK && worst == PLC_OK) worst = static_cast<plc_status>(h.status);
  }
  return worst;
}

}  // namespace plc
