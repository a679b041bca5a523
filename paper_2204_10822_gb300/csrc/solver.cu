// Host orchestration of the svN implicit step and the C ABI of include/svn.h.
//
// Per Newton iteration (Sections 4.2, 5.1, 5.4):
//   residual R(v_l) and ||R||            -> stop test
//   linearisation at (v_l, pi_l)         -> level-0 stencil, Galerkin hierarchy
//   FGMRES(K dv = -R), V-cycle preconditioner
//   backtracking on Phi                  -> alpha
//   pi <- pi + alpha pi~,  v <- v + alpha dv
// All arithmetic runs in the CUDA kernels; the host only reads the handful of
// scalars that steer the iteration (norms, energies, the Hessenberg column).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "../../include/svn.h"
#include "kernels.h"

using namespace svn;

svn::NetImpl* svn_net_impl(svn_net* net);   // unet.cu

namespace {

struct Level {
  Layout g;
  double* st64 = nullptr;        // FP64 stencil (19 planes)
  __nv_bfloat16* st16 = nullptr; // mixed: BF16 copy used by the V-cycle
  float* st32 = nullptr;         // mixed with FP32 V-cycle storage
  void* dinv = nullptr;          // 3 planes (double or float)
  double* lmax = nullptr;        // device scalar: Gershgorin bound of D^-1 A
  void* cheb = nullptr;          // Chebyshev step coefficients (V-cycle scalar type)
  void* x[2] = {nullptr, nullptr};
  void* d = nullptr;
  void* d2 = nullptr;            // second direction buffer for the fused two-step sweep
  void* b = nullptr;
  void* r = nullptr;
};

}  // namespace

struct svn_handle {
  svn_grid grid{};
  svn_params prm{};
  cudaStream_t stream = nullptr;
  std::string err;
  int device = 0;
  bool mixed = false;

  Layout g0{};
  std::vector<Level> lv;
  int ncoarse = 0;              // dense size of the coarsest level
  double* dense = nullptr;      // coarsest matrix (factored in place)
  double* dense_inv = nullptr;  // its inverse
  int* info = nullptr;

  // forcing (caller layout) and precomputed fields
  double *in_h = nullptr, *in_A = nullptr, *in_wind = nullptr, *in_ocean = nullptr, *in_vold = nullptr;
  double *tr_h = nullptr, *tr_A = nullptr;   // transport ping-pong (N*N each)
  bool have_forcing = false;
  double *P = nullptr, *rhoH = nullptr, *fq = nullptr, *voq = nullptr;
  double cur_dt = -1.0;

  // Newton state
  double2 *v = nullptr, *dv = nullptr, *vt = nullptr, *R = nullptr, *rhs = nullptr;
  double2* Rt = nullptr;        // residual at the trial point v + dv
  double* pi = nullptr;
  double* pi_t = nullptr;       // dual state at the trial point
  double* pi_scratch = nullptr;
  bool state_set = false;
  double* eb = nullptr;         // element buffer, NELEM planes FP64

  // Krylov
  int restart = 30;
  double2* V = nullptr;
  double2* Z = nullptr;         // preconditioned basis (FP64)
  double2* w = nullptr;
  double* hbuf = nullptr;       // device: h1 [restart+1], h2 [restart+1], nrm2
  double* ybuf = nullptr;       // device: FGMRES coefficients
  double* partial = nullptr;    // reduction partials
  size_t partial_len = 0;
  double* scal = nullptr;       // device scalars
  double* hostbuf = nullptr;    // pinned host mirror
  size_t hostbuf_len = 0;

  // learned initial guess (not owned)
  svn::NetImpl* net = nullptr;

  // when set, the outer Krylov operator (the Q2 discretisation uses this
  // handle's V-cycle and FGMRES workspace around its own operator)
  std::function<void(const double2*, double2*)> outer;
  // when set, the FGMRES preconditioner (the Q2 discretisation smooths on its
  // own operator around this handle's V-cycle)
  std::function<int(const double2*, double2*)> pre_op;

  // the V-cycle as a CUDA graph: input in lv[0].b, output in lv[0].x[1]
  cudaGraph_t vc_graph = nullptr;
  cudaGraphExec_t vc_exec = nullptr;
  cudaStream_t cap_stream = nullptr;   // private stream used only to record the graph
  bool graph_dirty = false;            // re-record the graph before its next launch
  bool graph_events = false;           // the recorded graph times its level-0 sweeps
  bool recording = false;              // a V-cycle is being recorded
  cudaEvent_t gev[64] = {};            // event pairs around level-0 sweeps (graph nodes)
  int n_gev = 0;
  long long sweep_steps[2] = {0, 0};   // recorded finest-level single / fused sweeps

  // instrumentation
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  double prof_ms[SVN_K_COUNT] = {};
  long long prof_n[SVN_K_COUNT] = {};
};

namespace {

int fail(svn_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return code;
}

#define CK(call)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(h, SVN_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CKL()                                                                                      \
  do {                                                                                             \
    cudaError_t e_ = cudaGetLastError();                                                           \
    if (e_ != cudaSuccess) return fail(h, SVN_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != SVN_OK) return rc_; \
  } while (0)

template <typename T>
int dalloc(svn_handle* h, T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(h, SVN_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", sizeof(T) * n, cudaGetErrorString(e));
  }
  e = cudaMemset(*p, 0, sizeof(T) * (n ? n : 1));
  if (e != cudaSuccess) return fail(h, SVN_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
  return SVN_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Records CUDA events around the launches of one kernel class when enabled.
struct Prof {
  svn_handle* h;
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  static cudaEvent_t ev(svn_handle* h) {
    if (!h->pool.empty()) {
      cudaEvent_t e = h->pool.back();
      h->pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  Prof(svn_handle* hh, int c) : h(hh), cls(c) {
    if (h->prof_on) {
      a = ev(h);
      b = ev(h);
      cudaEventRecord(a, h->stream);
    }
  }
  ~Prof() {
    if (a) {
      cudaEventRecord(b, h->stream);
      h->recs.push_back({cls, a, b});
    }
  }
};

void prof_collect(svn_handle* h) {
  if (h->recs.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (auto& r : h->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    h->prof_ms[r.cls] += ms;
    h->prof_n[r.cls] += 1;
    h->pool.push_back(r.a);
    h->pool.push_back(r.b);
  }
  h->recs.clear();
}

Phys make_phys(const svn_handle* h, const Layout& g, double dt) {
  Phys ph;
  const double e = h->prm.e;
  ph.dt = dt;
  ph.dx = g.dx;
  ph.idx = 1.0 / g.dx;
  ph.w = 0.25 * g.dx * g.dx;
  ph.ta = 0.5 * (1.0 + 1.0 / e);
  ph.tb = 0.5 * (1.0 - 1.0 / e);
  ph.tc = 0.5 / e;
  ph.dmin2 = h->prm.delta_min * h->prm.delta_min;
  ph.cdrag = h->prm.Co * h->prm.rho_o;
  return ph;
}

PhysConst make_pc(const svn_params& p) {
  PhysConst c;
  c.rho_ice = p.rho_ice; c.rho_a = p.rho_a; c.rho_o = p.rho_o; c.Ca = p.Ca; c.Co = p.Co;
  c.f_c = p.f_c; c.Pstar = p.Pstar; c.C = p.C; c.e = p.e; c.delta_min = p.delta_min;
  return c;
}

int sync_read(svn_handle* h, const double* dsrc, size_t n, double* out) {
  CK(cudaMemcpyAsync(h->hostbuf, dsrc, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  memcpy(out, h->hostbuf, sizeof(double) * n);
  return SVN_OK;
}

// ---- step pieces ------------------------------------------------------------------
int precompute(svn_handle* h, double dt) {
  if (!h->have_forcing) return fail(h, SVN_ERR_STATE, "svn_set_forcing has not been called");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, SVN_ERR_ARG, "dt must be positive and finite");
  launch_precompute(h->stream, h->g0, dt, make_pc(h->prm), h->in_h, h->in_A, h->in_wind, h->in_ocean, h->in_vold,
                    h->P, h->rhoH, h->fq, h->voq);
  CKL();
  h->cur_dt = dt;
  return SVN_OK;
}

int residual(svn_handle* h, const double2* v, double2* R, double* norm) {
  const Phys ph = make_phys(h, h->g0, h->cur_dt);
  {
    Prof pr(h, SVN_K_RESIDUAL);
    launch_residual(h->stream, h->g0, ph, v, h->P, h->rhoH, h->fq, h->voq, h->eb, R, h->partial);
  }
  launch_sum_final(h->stream, h->partial, residual_partials(h->g0), h->scal);
  CKL();
  double s;
  TRY(sync_read(h, h->scal, 1, &s));
  *norm = std::sqrt(s);
  return SVN_OK;
}

int energy(svn_handle* h, const double2* v, const double2* dv, const double* alphas, int k, double* phi,
           double* scale) {
  if (k < 1 || k > MAX_ALPHA) return fail(h, SVN_ERR_ARG, "energy: 1 <= k <= %d", MAX_ALPHA);
  const Phys ph = make_phys(h, h->g0, h->cur_dt);
  AlphaSet al{};
  for (int a = 0; a < k; ++a) al.a[a] = alphas[a];
  {
    Prof pr(h, SVN_K_ENERGY);
    launch_energy(h->stream, h->g0, ph, k, al, v, dv, h->P, h->rhoH, h->fq, h->voq, h->partial, h->scal);
  }
  CKL();
  double out[MAX_ALPHA + 1];
  TRY(sync_read(h, h->scal, MAX_ALPHA + 1, out));
  for (int a = 0; a < k; ++a) phi[a] = out[a];
  if (scale) *scale = out[MAX_ALPHA];
  return SVN_OK;
}

// Two-step sweep kernel of launch_cheb_sweep2 for the cheb_fuse setting.
inline int sweep_mode(const svn_params& p) {
  switch (p.cheb_fuse) {
    case 1: return 1;   // row-streaming kernel on the FP32 levels with N >= 1024, tile kernel below
    case 3: return 2;   // row-streaming kernel on every FP32 level
    case 4: return 4;   // TMA-staged kernel on the FP32-stencil levels with N >= 1024
    case 5: return 3;   // TMA-staged kernel on every FP32-stencil level
    default: return 0;  // shared-memory tile kernel
  }
}

// Chebyshev degree used on multigrid level l
inline int level_degree(const svn_params& p, int l) {
  return (l > 0 && p.cheb_degree_coarse > 0) ? p.cheb_degree_coarse : p.cheb_degree;
}

// SVN_ERR_TIMEOUT if a TMA-staged sweep gave up waiting for its copies since the last check.
int check_sweep_timeouts(svn_handle* h) {
  unsigned* pinned = reinterpret_cast<unsigned*>(h->hostbuf + h->hostbuf_len - 1);
  const int n = sweep_tma_timeouts(h->stream, pinned, true);
  if (n < 0) return fail(h, SVN_ERR_CUDA, "reading the sweep timeout counter failed");
  if (n > 0)
    return fail(h, SVN_ERR_TIMEOUT, "%d multigrid sweep blocks gave up waiting for their TMA copies", n);
  return SVN_OK;
}

int linearize(svn_handle* h, const double2* v, const double* pi, bool hierarchy = true) {
  const Phys ph = make_phys(h, h->g0, h->cur_dt);
  cudaStream_t s = h->stream;
  {
    Prof pr(h, SVN_K_ELEMENT);
    launch_element_matrices<double>(s, h->g0, ph, v, pi, h->P, h->rhoH, h->voq, h->eb);
  }
  launch_stencil_from_elements<double, double>(s, h->g0, h->eb, h->lv[0].st64);
  CKL();
  if (!hierarchy) return SVN_OK;   // the V-cycle keeps its previous hierarchy
  const int L = (int)h->lv.size();
  for (int l = 1; l < L; ++l) {
    Prof pr(h, SVN_K_RAP);
    launch_rap<double, double>(s, h->lv[l - 1].g, h->lv[l].g, h->lv[l - 1].st64, h->lv[l].st64);
  }
  CKL();
  const int smode = sweep_mode(h->prm);   // two-step kernel choice
  for (int l = 0; l < L - 1; ++l) {
    Level& lv = h->lv[l];
    int nb;
    if (h->mixed) {
      if (h->prm.vcycle_fp32)
        launch_convert_stencil<double, float>(s, lv.g, lv.st64, lv.st32);
      else
        launch_convert_stencil<double, __nv_bfloat16>(s, lv.g, lv.st64, lv.st16);
      nb = launch_dinv_gershgorin<double, float>(s, lv.g, lv.st64, (float*)lv.dinv, h->partial,
                                                 h->prm.lmax_iters == 0);
    } else {
      nb = launch_dinv_gershgorin<double, double>(s, lv.g, lv.st64, (double*)lv.dinv, h->partial,
                                                  h->prm.lmax_iters == 0);
    }
    launch_max_final(s, h->partial, nb, lv.lmax);
    if (h->prm.lmax_iters > 0) {
      if (h->mixed && h->prm.vcycle_fp32)
        launch_power_lmax<float, float, float2>(s, lv.g, lv.st32, (const float*)lv.dinv, h->prm.lmax_iters,
                                                h->prm.lmax_safety, (float2*)lv.x[0], (float2*)lv.x[1], h->partial,
                                                lv.lmax, smode, (unsigned)h->prm.wait_polls);
      else if (h->mixed)
        launch_power_lmax<__nv_bfloat16, float, float2>(s, lv.g, lv.st16, (const float*)lv.dinv, h->prm.lmax_iters,
                                                        h->prm.lmax_safety, (float2*)lv.x[0], (float2*)lv.x[1],
                                                        h->partial, lv.lmax, smode, (unsigned)h->prm.wait_polls);
      else
        launch_power_lmax<double, double, double2>(s, lv.g, lv.st64, (const double*)lv.dinv, h->prm.lmax_iters,
                                                   h->prm.lmax_safety, (double2*)lv.x[0], (double2*)lv.x[1],
                                                   h->partial, lv.lmax, smode);
    }
    if (h->mixed)
      launch_cheb_coefs<float>(s, lv.lmax, h->prm.cheb_lo, level_degree(h->prm, l), (float*)lv.cheb);
    else
      launch_cheb_coefs<double>(s, lv.lmax, h->prm.cheb_lo, level_degree(h->prm, l), (double*)lv.cheb);
  }
  CKL();
  Level& lc = h->lv[L - 1];
  launch_coarse_dense<double>(s, lc.g, lc.st64, h->dense);
  launch_cholesky_inverse(s, h->ncoarse, h->dense, h->dense_inv, h->info);
  CKL();
  int info = 0;
  CK(cudaMemcpyAsync(h->hostbuf, h->info, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  memcpy(&info, h->hostbuf, sizeof(int));
  if (info != 0) return fail(h, SVN_ERR_ARG, "coarsest operator is not positive definite (pivot %d)", info);
  return check_sweep_timeouts(h);
}

// Times level-0 Chebyshev sweeps: CUDA events around the launch, either as
// ordinary records (eager V-cycle) or as event-record nodes of the graph.
struct SweepTimer {
  svn_handle* h;
  int idx = -1;
  Prof* pr = nullptr;
  SweepTimer(svn_handle* hh, int level, int steps) : h(hh) {
    if (level != 0) return;
    h->sweep_steps[steps == 2 ? 1 : 0] += 1;
    // with fusion on, only the fused two-step launches are timed (one kernel)
    if (h->prm.cheb_fuse && steps != 2) return;
    if (h->recording) {
      if (!h->graph_events || h->n_gev + 2 > 64) return;
      idx = h->n_gev;
      h->n_gev += 2;
      for (int e = idx; e < idx + 2; ++e)
        if (!h->gev[e]) cudaEventCreate(&h->gev[e]);
      cudaEventRecordWithFlags(h->gev[idx], h->stream, cudaEventRecordExternal);
    } else {
      pr = new Prof(h, SVN_K_CHEB);
    }
  }
  ~SweepTimer() {
    if (idx >= 0) cudaEventRecordWithFlags(h->gev[idx + 1], h->stream, cudaEventRecordExternal);
    delete pr;
  }
};

// Accumulate the sweep times of the last graph launch (call after a sync).
void collect_graph_events(svn_handle* h) {
  if (!h->prof_on || !h->graph_events) return;
  for (int e = 0; e + 1 < h->n_gev; e += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->gev[e], h->gev[e + 1]) == cudaSuccess) {
      h->prof_ms[SVN_K_CHEB] += ms;
      h->prof_n[SVN_K_CHEB] += 1;
    }
  }
  cudaGetLastError();
}

// One V-cycle on levels l..L-1: x_l = M_l^-1 b_l, both in level-l vectors (TV).
template <typename TS, typename TD, typename TV>
void vcycle(svn_handle* h, int l, const TV* b, TV* xout) {
  cudaStream_t s = h->stream;
  const int L = (int)h->lv.size();
  Level& lv = h->lv[l];
  if (l == L - 1) {
    launch_coarse_solve<TV>(s, lv.g, h->ncoarse, h->dense_inv, b, xout);
    return;
  }
  const TS* st = !h->mixed ? (const TS*)lv.st64 : h->prm.vcycle_fp32 ? (const TS*)lv.st32 : (const TS*)lv.st16;
  const TD* dinv = (const TD*)lv.dinv;
  TV* x0 = (TV*)lv.x[0];
  TV* x1 = (TV*)lv.x[1];
  TV* d = (TV*)lv.d;
  TV* r = (TV*)lv.r;
  using T = typename ScalarOf<TV>::type;
  const int deg = level_degree(h->prm, l);
  const T* coef = (const T*)lv.cheb;
  TV* dalt = (TV*)lv.d2;
  TV* cur = x0;
  const bool fuse = h->prm.cheb_fuse != 0;
  const int smode = sweep_mode(h->prm);   // two-step kernel choice
  // Chebyshev steps [k, kend) from cur; the result lands in `last_dst` when given
  auto smooth = [&](int k, int kend, TV* last_dst) {
    while (k < kend) {
      const bool pair = fuse && k + 1 < kend;
      const bool last = k + (pair ? 2 : 1) >= kend;
      TV* dst = (last && last_dst && last_dst != cur) ? last_dst : (cur == x0 ? x1 : x0);
      SweepTimer tm(h, l, pair ? 2 : 1);
      if (pair) {
        launch_cheb_sweep2<TS, TD, TV>(s, lv.g, st, dinv, coef, k, cur, dst, d, dalt, b, smode,
                                       (unsigned)h->prm.wait_polls);
        std::swap(d, dalt);
        k += 2;
      } else {
        launch_cheb_sweep<TS, TD, TV>(s, lv.g, st, dinv, coef, k, cur, dst, d, b);
        k += 1;
      }
      cur = dst;
    }
  };
  // pre-smoothing from x = 0: steps 0 and 1 in one streaming pass where that
  // kernel runs, else step 0 pointwise
  if (fuse && deg >= 2 && sizeof(T) == 4 && sweep2_streams(lv.g, smode)) {
    launch_cheb_sweep2<TS, TD, TV>(s, lv.g, st, dinv, coef, 0, nullptr, x0, nullptr, d, b, smode,
                                   (unsigned)h->prm.wait_polls);
    cur = x0;
    smooth(2, deg, nullptr);
  } else {
    launch_cheb_zero_start<TS, TD, TV>(s, lv.g, dinv, coef, b, x0, d);
    smooth(1, deg, nullptr);
  }
  // coarse-grid correction
  launch_residual_stencil<TS, TV>(s, lv.g, st, cur, b, r);
  Level& lc = h->lv[l + 1];
  launch_restrict<TV>(s, lv.g, lc.g, r, (TV*)lc.b);
  vcycle<TS, TD, TV>(h, l + 1, (const TV*)lc.b, (TV*)lc.x[0]);
  launch_prolong_add<TV>(s, lv.g, lc.g, (const TV*)lc.x[0], cur);
  // post-smoothing (same polynomial)
  smooth(0, deg, xout);
  if (cur != xout) cudaMemcpyAsync(xout, cur, sizeof(TV) * lv.g.plane, cudaMemcpyDeviceToDevice, s);
}

// Record the V-cycle launches from lv[0].b to lv[0].x[1] on the handle's stream.
void vcycle_record(svn_handle* h) {
  Level& l0 = h->lv[0];
  if (h->mixed && h->prm.vcycle_fp32)
    vcycle<float, float, float2>(h, 0, (const float2*)l0.b, (float2*)l0.x[1]);
  else if (h->mixed)
    vcycle<__nv_bfloat16, float, float2>(h, 0, (const float2*)l0.b, (float2*)l0.x[1]);
  else
    vcycle<double, double, double2>(h, 0, (const double2*)l0.b, (double2*)l0.x[1]);
}

// z = M^-1 r for level-0 FP64 vectors r, z (one V-cycle).
int precondition_mg(svn_handle* h, const double2* r, double2* z) {
  Level& l0 = h->lv[0];
  cudaStream_t s = h->stream;
  if (h->mixed)
    launch_cast_d2f(s, l0.g, r, (float2*)l0.b);
  else
    CK(cudaMemcpyAsync(l0.b, r, sizeof(double2) * l0.g.plane, cudaMemcpyDeviceToDevice, s));
  CKL();
  Prof pr(h, SVN_K_VCYCLE);
  if (h->prm.use_graphs) {
    if (h->graph_dirty && h->vc_exec) {
      cudaGraphExecDestroy(h->vc_exec);
      cudaGraphDestroy(h->vc_graph);
      h->vc_exec = nullptr;
      h->vc_graph = nullptr;
    }
    h->graph_dirty = false;
    if (!h->vc_exec) {
      // record on a private stream (the caller's stream may be the legacy
      // default stream, which cannot be captured); launch on the caller's
      if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      const bool prof = h->prof_on;
      h->prof_on = false;   // no ordinary event records inside the capture
      h->graph_events = prof;
      h->recording = true;
      h->n_gev = 0;
      h->stream = h->cap_stream;
      cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        vcycle_record(h);
        e = cudaStreamEndCapture(h->cap_stream, &h->vc_graph);
      }
      h->stream = s;
      h->recording = false;
      h->prof_on = prof;
      if (e != cudaSuccess) return fail(h, SVN_ERR_CUDA, "V-cycle capture: %s", cudaGetErrorString(e));
      CK(cudaGraphInstantiate(&h->vc_exec, h->vc_graph, 0));
    }
    CK(cudaGraphLaunch(h->vc_exec, s));
  } else {
    vcycle_record(h);
  }
  CKL();
  if (h->mixed)
    launch_cast_f2d(s, l0.g, (const float2*)l0.x[1], z);
  else
    CK(cudaMemcpyAsync(z, l0.x[1], sizeof(double2) * l0.g.plane, cudaMemcpyDeviceToDevice, s));
  CKL();
  return SVN_OK;
}

int precondition(svn_handle* h, const double2* r, double2* z) {
  if (h->pre_op) return h->pre_op(r, z);
  return precondition_mg(h, r, z);
}

// y = K0 z (FP64 outer operator).
void apply_outer(svn_handle* h, const double2* z, double2* y) {
  Prof pr(h, SVN_K_APPLY);
  if (h->outer)
    h->outer(z, y);
  else
    launch_apply<double, double2, double2, double>(h->stream, h->g0, h->lv[0].st64, z, y);
}

double2* zvec(svn_handle* h, int j) { return h->Z + (size_t)j * h->g0.plane; }

int norm2(svn_handle* h, const double2* x, double* out) {
  launch_norm2_partial(h->stream, h->g0, x, h->partial);
  launch_sum_final(h->stream, h->partial, reduce_blocks(h->g0.plane), h->scal);
  CKL();
  double s;
  TRY(sync_read(h, h->scal, 1, &s));
  *out = std::sqrt(s);
  return SVN_OK;
}

// Relative Krylov tolerance of Newton iteration `it` (residual norm r, previous
// norm r_prev, stopping threshold r_stop = tol ||R_0||).  Without
// eisenstat_walker: krylov_rtol.  With it: Eisenstat-Walker choice 2,
// eta_k = 0.9 (r_k / r_{k-1})^2, kept >= 0.9 eta_{k-1}^2 when that is above 0.1,
// clipped to [krylov_rtol, ew_eta_max]; then, with ew_tail > 0, raised to
// min(ew_eta_max, ew_tail r_stop / r_k) (Kelley 1995, Sect. 6.3): a step whose
// residual is already near the threshold is not solved far beyond it.
double forcing_term(const svn_params& p, int it, double r, double r_prev, double r_stop, double& eta_prev) {
  if (!p.eisenstat_walker) return p.krylov_rtol;
  double eta = p.ew_eta_max;
  if (it > 0) {
    const double ratio = r / r_prev;
    eta = 0.9 * ratio * ratio;
    const double prev = 0.9 * eta_prev * eta_prev;
    if (prev > 0.1) eta = std::max(eta, prev);
    eta = std::min(p.ew_eta_max, std::max(p.krylov_rtol, eta));
  }
  if (p.ew_tail > 0.0 && r > 0.0) eta = std::max(eta, std::min(p.ew_eta_max, p.ew_tail * r_stop / r));
  eta_prev = eta;
  return eta;
}

// FGMRES (right preconditioned, CGS2 Arnoldi) for K x = b, x = 0 on entry.
int fgmres(svn_handle* h, const double2* b, double2* x, double rtol, int maxit, int* iters) {
  cudaStream_t s = h->stream;
  const Layout& g = h->g0;
  const int m = h->restart;
  const long long vs = g.plane;
  const int nw = krylov_blocks(g);
  if ((size_t)nw * (m + 1) > h->partial_len || (size_t)energy_partials(g) * (2 * MAX_ALPHA + 1) +
                                                      (size_t)residual_partials(g) > h->partial_len)
    return fail(h, SVN_ERR_ARG, "internal: reduction buffer too small");
  CK(cudaMemsetAsync(x, 0, sizeof(double2) * g.plane, s));
  double bnorm;
  TRY(norm2(h, b, &bnorm));
  *iters = 0;
  if (bnorm == 0.0) return SVN_OK;
  if (!std::isfinite(bnorm)) return fail(h, SVN_ERR_NONFINITE, "FGMRES: non-finite right-hand side");
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), yv(m);
  double beta = bnorm;
  launch_scale_to(s, g, 1.0 / beta, b, h->V);   // V0 = b / beta
  int total = 0;
  bool done = false;
  while (!done) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double2* Vj = h->V + (size_t)j * vs;
      TRY(precondition(h, Vj, zvec(h, j)));
      apply_outer(h, zvec(h, j), h->w);
      // classical Gram-Schmidt; a second pass only when the first one cancelled
      // more than half of |w|^2 (Kahan's "twice is enough" criterion)
      double* h1 = h->hbuf;
      double* h2 = h->hbuf + (m + 1);
      double* nr = h->hbuf + 2 * (m + 1);
      std::vector<double> hh(2 * (m + 1) + 1, 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        double* hp = pass == 0 ? h1 : h2;
        {
          Prof pr(h, SVN_K_MULTIDOT);
          launch_multidot(s, g, h->V, vs, j + 1, h->w, h->partial, nw);
        }
        launch_multidot_final(s, h->partial, nw, j + 1, hp, 0);
        {
          Prof pr(h, SVN_K_UPDATE);
          launch_update_norm(s, g, h->V, vs, j + 1, hp, h->w, h->partial, nw);
        }
        launch_sum_final(s, h->partial, nw, nr);
        CKL();
        TRY(sync_read(h, h->hbuf, hh.size(), hh.data()));
        if (pass == 0) collect_graph_events(h);
        if (pass == 0) {
          for (int i = 0; i <= j; ++i) hh[m + 1 + i] = 0.0;
          double proj = 0.0;
          for (int i = 0; i <= j; ++i) proj += hh[i] * hh[i];
          const double after = hh[2 * (m + 1)];
          if (!h->prm.reorth_always && after >= 0.5 * (proj + after)) break;
        }
      }
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i] + hh[m + 1 + i];
      const double hn = std::sqrt(hh[2 * (m + 1)]);
      if (!std::isfinite(hn)) return fail(h, SVN_ERR_NONFINITE, "FGMRES: non-finite Arnoldi vector");
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) {
        launch_scale_to(s, g, 1.0 / hn, h->w, h->V + (size_t)(j + 1) * vs);   // V_{j+1} = w / hn
        CKL();
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = t;
      }
      const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      const double den = std::hypot(a, bb);
      if (den == 0.0) return fail(h, SVN_ERR_KRYLOV, "FGMRES breakdown (zero Hessenberg column)");
      cs[j] = a / den;
      sn[j] = bb / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++total;
      jdone = j + 1;
      if (std::fabs(gv[j + 1]) <= rtol * bnorm || total >= maxit || hn == 0.0) break;
    }
    // y = H^-1 g (upper triangular), x += Z y
    for (int i = jdone - 1; i >= 0; --i) {
      double sacc = gv[i];
      for (int k = i + 1; k < jdone; ++k) sacc -= H[(size_t)i * m + k] * yv[k];
      yv[i] = sacc / H[(size_t)i * m + i];
    }
    memcpy(h->hostbuf, yv.data(), sizeof(double) * jdone);
    CK(cudaMemcpyAsync(h->ybuf, h->hostbuf, sizeof(double) * jdone, cudaMemcpyHostToDevice, s));
    launch_lincomb<double2>(s, g, h->Z, vs, jdone, h->ybuf, x);
    CKL();
    CK(cudaStreamSynchronize(s));   // hostbuf reuse
    const double est = std::fabs(gv[jdone]);
    if (est <= rtol * bnorm) break;
    if (total >= maxit) break;   // inexact Newton direction; the line search safeguards it
    // restart: V0 = (b - K x) / |b - K x|
    apply_outer(h, x, h->w);
    launch_axpby_to(s, g, b, -1.0, h->w, h->w);
    CKL();
    TRY(norm2(h, h->w, &beta));
    if (beta <= rtol * bnorm) break;
    launch_scale_to(s, g, 1.0 / beta, h->w, h->V);
    CKL();
  }
  *iters = total;
  return check_sweep_timeouts(h);
}

int check_params(svn_handle* h, const svn_params* p) {
  if (!(p->e > 0) || !(p->delta_min > 0) || !(p->rho_ice > 0) || p->Pstar < 0 || p->Co < 0 || p->Ca < 0)
    return fail(h, SVN_ERR_ARG, "invalid physical constants");
  if (p->max_newton < 0 || p->max_newton > SVN_MAX_NEWTON) return fail(h, SVN_ERR_ARG, "max_newton out of range");
  if (p->max_halvings < 0 || p->max_halvings > 60) return fail(h, SVN_ERR_ARG, "max_halvings out of range");
  if (p->restart < 1 || p->restart > 200) return fail(h, SVN_ERR_ARG, "restart must be in [1, 200]");
  if (p->cheb_degree < 1 || p->cheb_degree > 16) return fail(h, SVN_ERR_ARG, "cheb_degree must be in [1, 16]");
  if (!(p->cheb_lo > 0.0 && p->cheb_lo < 1.0)) return fail(h, SVN_ERR_ARG, "cheb_lo must be in (0, 1)");
  if (p->precision != SVN_FP64 && p->precision != SVN_MIXED) return fail(h, SVN_ERR_ARG, "unknown precision");
  if (p->coarse_N < 2 || p->coarse_N > 16) return fail(h, SVN_ERR_ARG, "coarse_N must be in [2, 16]");
  if (p->lmax_iters < 0 || p->lmax_iters > 60) return fail(h, SVN_ERR_ARG, "lmax_iters must be in [0, 60]");
  if (p->method != 0 && p->method != 1) return fail(h, SVN_ERR_ARG, "method must be 0 (svN) or 1 (stdN)");
  if (p->learned_rule < 0 || p->learned_rule > 4) return fail(h, SVN_ERR_ARG, "learned_rule must be in [0, 4]");
  if (!(p->lmax_safety >= 1.0 && p->lmax_safety < 4.0)) return fail(h, SVN_ERR_ARG, "lmax_safety must be in [1, 4)");
  if (p->cheb_fuse < 0 || p->cheb_fuse > 5) return fail(h, SVN_ERR_ARG, "cheb_fuse must be in [0, 5]");
  if (p->wait_polls < 0) return fail(h, SVN_ERR_ARG, "wait_polls must be >= 0");
  if (p->q2_smooth_degree < 0 || p->q2_smooth_degree > 16)
    return fail(h, SVN_ERR_ARG, "q2_smooth_degree must be in [0, 16]");
  if (p->cheb_degree_coarse < 0 || p->cheb_degree_coarse > 16)
    return fail(h, SVN_ERR_ARG, "cheb_degree_coarse must be in [0, 16]");
  if (!(p->retry_alpha >= 0.0 && p->retry_alpha <= 1.0)) return fail(h, SVN_ERR_ARG, "retry_alpha must be in [0, 1]");
  if (!(p->ew_tail >= 0.0 && p->ew_tail <= 1.0)) return fail(h, SVN_ERR_ARG, "ew_tail must be in [0, 1]");
  return SVN_OK;
}

int create_impl(svn_handle* h, const svn_grid* g, const svn_params* p, void* stream) {
  if (!g || !p) return fail(h, SVN_ERR_ARG, "NULL grid or params");
  if (g->N < 8 || g->N > 16384 || (g->N & 1)) return fail(h, SVN_ERR_ARG, "N must be even and in [8, 16384]");
  if (!(g->L > 0) || !std::isfinite(g->L)) return fail(h, SVN_ERR_ARG, "L must be positive");
  TRY(check_params(h, p));
  h->grid = *g;
  h->prm = *p;
  h->stream = (cudaStream_t)stream;
  h->mixed = p->precision == SVN_MIXED;
  h->restart = p->restart;
  CK(cudaGetDevice(&h->device));
  h->g0 = make_layout(g->N, g->L);
  // multigrid levels: halve while even and above coarse_N
  int n = g->N;
  h->lv.clear();
  while (true) {
    Level L;
    L.g = make_layout(n, g->L);
    h->lv.push_back(L);
    if (n <= p->coarse_N || (n & 1) || n / 2 < 2) break;
    n /= 2;
  }
  const Layout& g0 = h->g0;
  const long long pl = g0.plane;
  TRY(dalloc(h, &h->in_h, (size_t)g->N * g->N));
  TRY(dalloc(h, &h->in_A, (size_t)g->N * g->N));
  const size_t nv = 2 * (size_t)(g->N + 1) * (g->N + 1);
  TRY(dalloc(h, &h->in_wind, nv));
  TRY(dalloc(h, &h->in_ocean, nv));
  TRY(dalloc(h, &h->in_vold, nv));
  TRY(dalloc(h, &h->tr_h, (size_t)g->N * g->N));
  TRY(dalloc(h, &h->tr_A, (size_t)g->N * g->N));
  TRY(dalloc(h, &h->P, pl));
  TRY(dalloc(h, &h->rhoH, pl));
  TRY(dalloc(h, &h->fq, 8 * pl));
  TRY(dalloc(h, &h->voq, 8 * pl));
  TRY(dalloc(h, &h->v, pl));
  TRY(dalloc(h, &h->dv, pl));
  TRY(dalloc(h, &h->vt, pl));
  TRY(dalloc(h, &h->R, pl));
  TRY(dalloc(h, &h->rhs, pl));
  TRY(dalloc(h, &h->w, pl));
  TRY(dalloc(h, &h->pi, 12 * pl));
  TRY(dalloc(h, &h->pi_t, 12 * pl));
  TRY(dalloc(h, &h->Rt, pl));
  TRY(dalloc(h, &h->eb, (size_t)NELEM * pl));
  const size_t vsz = h->mixed ? sizeof(float2) : sizeof(double2);
  for (size_t l = 0; l < h->lv.size(); ++l) {
    Level& L = h->lv[l];
    const long long lp = L.g.plane;
    TRY(dalloc(h, &L.st64, (size_t)NSTEN * lp));
    if (h->mixed && !p->vcycle_fp32) TRY(dalloc(h, &L.st16, (size_t)NSTEN * lp));
    if (h->mixed && p->vcycle_fp32) TRY(dalloc(h, &L.st32, (size_t)NSTEN * lp));
    TRY(dalloc(h, (char**)&L.dinv, 3 * lp * (h->mixed ? sizeof(float) : sizeof(double))));
    TRY(dalloc(h, &L.lmax, 1));
    TRY(dalloc(h, (double**)&L.cheb, 2 * 16));
    for (int k = 0; k < 2; ++k) TRY(dalloc(h, (char**)&L.x[k], lp * vsz));
    TRY(dalloc(h, (char**)&L.d, lp * vsz));
    TRY(dalloc(h, (char**)&L.d2, lp * vsz));
    TRY(dalloc(h, (char**)&L.b, lp * vsz));
    TRY(dalloc(h, (char**)&L.r, lp * vsz));
  }
  const int mc = h->lv.back().g.N - 1;
  h->ncoarse = 2 * mc * mc;
  TRY(dalloc(h, &h->dense, (size_t)h->ncoarse * h->ncoarse));
  TRY(dalloc(h, &h->dense_inv, (size_t)h->ncoarse * h->ncoarse));
  TRY(dalloc(h, &h->info, 4));
  TRY(dalloc(h, &h->V, (size_t)(h->restart + 1) * pl));
  TRY(dalloc(h, &h->Z, (size_t)h->restart * pl));
  TRY(dalloc(h, &h->hbuf, 2 * (size_t)(h->restart + 1) + 1));
  TRY(dalloc(h, &h->ybuf, (size_t)h->restart + 1));
  const int nw = krylov_blocks(g0);
  h->partial_len = (size_t)std::max<long long>(
      {(long long)nw * (h->restart + 1), (long long)residual_partials(g0),
       (long long)energy_partials(g0) * (2 * MAX_ALPHA + 1) + residual_partials(g0), (long long)reduce_blocks(pl),
       4096});
  TRY(dalloc(h, &h->partial, h->partial_len));
  TRY(dalloc(h, &h->scal, 64));
  h->hostbuf_len = 4 * (size_t)(h->restart + 2) + 64;
  CK(cudaMallocHost((void**)&h->hostbuf, sizeof(double) * h->hostbuf_len));
  return SVN_OK;
}

void destroy_impl(svn_handle* h) {
  dfree(h->in_h); dfree(h->in_A); dfree(h->in_wind); dfree(h->in_ocean); dfree(h->in_vold);
  dfree(h->tr_h); dfree(h->tr_A);
  dfree(h->P); dfree(h->rhoH); dfree(h->fq); dfree(h->voq);
  dfree(h->v); dfree(h->dv); dfree(h->vt); dfree(h->R); dfree(h->rhs); dfree(h->w);
  dfree(h->pi); dfree(h->pi_t); dfree(h->Rt); dfree(h->pi_scratch); dfree(h->eb);
  for (Level& L : h->lv) {
    dfree(L.st64); dfree(L.st16); dfree(L.st32); dfree(L.dinv); dfree(L.lmax); dfree(L.cheb);
    dfree(L.x[0]); dfree(L.x[1]); dfree(L.d); dfree(L.d2); dfree(L.b); dfree(L.r);
  }
  dfree(h->dense); dfree(h->dense_inv); dfree(h->info);
  if (h->vc_exec) cudaGraphExecDestroy(h->vc_exec);
  if (h->vc_graph) cudaGraphDestroy(h->vc_graph);
  h->vc_exec = nullptr;
  h->vc_graph = nullptr;
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->cap_stream = nullptr;
  for (cudaEvent_t& e : h->gev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  dfree(h->V); dfree(h->Z); dfree(h->hbuf); dfree(h->ybuf); dfree(h->partial); dfree(h->scal);
  if (h->hostbuf) cudaFreeHost(h->hostbuf);
  h->hostbuf = nullptr;
  for (auto& r : h->recs) {
    h->pool.push_back(r.a);
    h->pool.push_back(r.b);
  }
  h->recs.clear();
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  h->pool.clear();
}

// Validate the device copies of the inputs (counts of bad entries, one read-back).
int validate_forcing(svn_handle* h) {
  const long long nc = (long long)h->grid.N * h->grid.N;
  const long long nv = 2LL * (h->grid.N + 1) * (h->grid.N + 1);
  int* flags = (int*)h->info;   // 4 ints: info + 3 counters
  CK(cudaMemsetAsync(flags + 1, 0, 3 * sizeof(int), h->stream));
  launch_validate(h->stream, nc, nv, h->in_h, h->in_A, h->in_wind, h->in_ocean, h->in_vold, flags + 1);
  CKL();
  int cnt[3];
  CK(cudaMemcpyAsync(h->hostbuf, flags + 1, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  memcpy(cnt, h->hostbuf, sizeof(cnt));
  if (cnt[0]) return fail(h, SVN_ERR_NONFINITE, "%d non-finite input entries", cnt[0]);
  if (cnt[1]) return fail(h, SVN_ERR_ARG, "%d cells with thickness <= 0", cnt[1]);
  if (cnt[2]) return fail(h, SVN_ERR_ARG, "%d cells with concentration outside [0, 1]", cnt[2]);
  return SVN_OK;
}

int set_forcing_impl(svn_handle* h, const double* hc, const double* A, const double* wind, const double* ocean,
                     const double* vold, bool host) {
  if (!hc || !A || !wind || !ocean || !vold) return fail(h, SVN_ERR_ARG, "NULL forcing pointer");
  const size_t nc = (size_t)h->grid.N * h->grid.N;
  const size_t nv = 2 * (size_t)(h->grid.N + 1) * (h->grid.N + 1);
  const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(h->in_h, hc, sizeof(double) * nc, kind, h->stream));
  CK(cudaMemcpyAsync(h->in_A, A, sizeof(double) * nc, kind, h->stream));
  CK(cudaMemcpyAsync(h->in_wind, wind, sizeof(double) * nv, kind, h->stream));
  CK(cudaMemcpyAsync(h->in_ocean, ocean, sizeof(double) * nv, kind, h->stream));
  CK(cudaMemcpyAsync(h->in_vold, vold, sizeof(double) * nv, kind, h->stream));
  h->have_forcing = false;
  TRY(validate_forcing(h));
  h->have_forcing = true;
  h->state_set = false;
  return SVN_OK;
}

// Explicit upwind transport of the handle's H and A over dt with its v^n
// (Eqs. "model:A", "model:H"; Section 3), sub-cycled for the Courant number.
constexpr int kMaxSubsteps = 10000;
int transport_impl(svn_handle* h, double dt, int* nsub) {
  *nsub = 0;
  if (!h->have_forcing) return fail(h, SVN_ERR_STATE, "svn_set_forcing has not been called");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, SVN_ERR_ARG, "dt must be positive and finite");
  cudaStream_t s = h->stream;
  const int N = h->grid.N;
  const double dx = h->g0.dx;
  if ((size_t)transport_courant_blocks(N) > h->partial_len)
    return fail(h, SVN_ERR_ARG, "reduction buffer too small for the Courant maximum");
  launch_transport_courant(s, N, dt / dx, h->in_vold, h->partial);
  launch_max_final(s, h->partial, transport_courant_blocks(N), h->scal);
  CKL();
  double c = 0.0;
  TRY(sync_read(h, h->scal, 1, &c));
  if (!std::isfinite(c)) return fail(h, SVN_ERR_NONFINITE, "non-finite velocity in the transport step");
  const double nd = std::max(1.0, std::ceil(c));
  if (nd > kMaxSubsteps)
    return fail(h, SVN_ERR_ARG, "Courant number %g needs more than %d transport sub-steps", c, kMaxSubsteps);
  const int n = (int)nd;
  const double k = (dt / n) / dx;
  double *Hs = h->in_h, *As = h->in_A, *Hd = h->tr_h, *Ad = h->tr_A;
  for (int q = 0; q < n; ++q) {
    launch_transport_step(s, N, k, q == n - 1, h->in_vold, Hs, As, Hd, Ad);
    std::swap(Hs, Hd);
    std::swap(As, Ad);
  }
  if (Hs != h->in_h) {
    CK(cudaMemcpyAsync(h->in_h, Hs, sizeof(double) * N * (size_t)N, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->in_A, As, sizeof(double) * N * (size_t)N, cudaMemcpyDeviceToDevice, s));
  }
  CKL();
  h->have_forcing = false;
  TRY(validate_forcing(h));
  h->have_forcing = true;
  h->state_set = false;
  *nsub = n;
  return SVN_OK;
}

int step_impl(svn_handle* h, double dt, double tol, svn_stats* st) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = h->stream;
  const Layout& g = h->g0;
  st->status = SVN_OK;
  TRY(precompute(h, dt));
  if (!(tol > 0.0)) return fail(h, SVN_ERR_ARG, "tol must be positive");
  const Phys ph = make_phys(h, g, dt);
  // reference residual: the plain previous-step start v^n
  launch_unpack_nodes(s, g, h->in_vold, h->vt);
  CKL();
  TRY(residual(h, h->vt, h->R, &st->res0));
  if (!h->state_set) {
    CK(cudaMemcpyAsync(h->v, h->vt, sizeof(double2) * g.plane, cudaMemcpyDeviceToDevice, s));
    if (h->prm.learned && h->net && g.N % net_grid(h->net) == 0) {
      // learned start: kept only if its residual is below that of v^n
      st->learned_used = 1;
      net_predict_nodes(h->net, s, g, h->in_h, h->in_A, h->in_wind, h->in_ocean, h->in_vold, h->vt);
      CKL();
      bool take = false;
      if (h->prm.learned_rule == 4) {
        // the prediction as the velocity, the dual state of the plain start
        launch_pi_init(s, g, ph, h->v, h->pi);
        take = true;
      } else if (h->prm.learned_rule == 3) {
        // blend rule: v^n + alpha (v_pred - v^n) with the alpha in {1, 1/2, ..., 1/64}
        // of lowest Phi (one multi-alpha energy pass), kept if it is below Phi(v^n)
        launch_axpby_to(s, g, h->vt, -1.0, h->v, h->w);   // w = v_pred - v^n
        CKL();
        double al[MAX_ALPHA], phi[MAX_ALPHA];
        al[0] = 0.0;
        for (int a = 1; a < MAX_ALPHA; ++a) al[a] = std::ldexp(1.0, 1 - a);
        TRY(energy(h, h->v, h->w, al, MAX_ALPHA, phi, nullptr));
        int best = 0;
        for (int a = 1; a < MAX_ALPHA; ++a)
          if (std::isfinite(phi[a]) && phi[a] < phi[best]) best = a;
        if (best > 0) {
          launch_axpy(s, g, al[best], h->w, h->v);
          CKL();
          st->learned_alpha = al[best];
        } else {
          st->learned_fallback = 1;
        }
      } else if (h->prm.learned_rule == 2) {
        take = true;
      } else if (h->prm.learned_rule == 1) {
        // energy rule: keep the prediction if Phi(v_pred) < Phi(v^n)
        const double a0 = 0.0;
        double phi_p, phi_o;
        TRY(energy(h, h->vt, h->vt, &a0, 1, &phi_p, nullptr));
        TRY(energy(h, h->v, h->v, &a0, 1, &phi_o, nullptr));
        take = std::isfinite(phi_p) && phi_p < phi_o;
      } else {
        double rp;
        TRY(residual(h, h->vt, h->w, &rp));
        take = std::isfinite(rp) && rp < st->res0;
      }
      if (h->prm.learned_rule != 3) {
        if (take) {
          CK(cudaMemcpyAsync(h->v, h->vt, sizeof(double2) * g.plane, cudaMemcpyDeviceToDevice, s));
          st->learned_alpha = 1.0;
        } else {
          st->learned_fallback = 1;
        }
      }
    }
    if (!(st->learned_used && h->prm.learned_rule == 4)) launch_pi_init(s, g, ph, h->v, h->pi);
    CKL();
  }
  h->state_set = false;   // a later step restarts from its own v^n unless set_state is called again
  double phi0 = 0.0, scale0 = 0.0;
  {
    const double a0 = 0.0;
    TRY(energy(h, h->v, h->v, &a0, 1, &phi0, &scale0));
  }
  const svn_params& p = h->prm;
  double eta_prev = p.ew_eta_max;
  bool have_r = false;      // R and its norm at v were produced by the accepted trial
  double r_next = 0.0;
  for (int it = 0;; ++it) {
    double r;
    if (have_r) {
      r = r_next;
      have_r = false;
    } else {
      TRY(residual(h, h->v, h->R, &r));
    }
    st->res_hist[it] = r;
    st->newton_iters = it;
    st->res_final = r;
    st->rel_res_final = st->res0 > 0 ? r / st->res0 : 0.0;
    if (!std::isfinite(r)) return fail(h, SVN_ERR_NONFINITE, "non-finite residual norm at Newton iteration %d", it);
    if (r <= tol * st->res0 || r == 0.0) break;
    if (it >= p.max_newton)
      return fail(h, SVN_ERR_NO_CONVERGENCE, "no convergence in %d Newton iterations (rel-res %.3e)", it,
                  st->rel_res_final);
    if (p.method == 1) {
      // standard Newton (Section 4.1): its Jacobian is the svN operator at
      // pi = tau(v)/Delta(v) (where the modification is inactive)
      launch_pi_init(s, g, ph, h->v, h->pi);
      CKL();
    }
    const int every = std::max(1, p.mg_rebuild);
    TRY(linearize(h, h->v, h->pi, it % every == 0));
    launch_neg_copy(s, g, h->R, h->rhs);
    CKL();
    int kits = 0;
    double eta = forcing_term(p, it, r, it > 0 ? st->res_hist[it - 1] : 0.0, tol * st->res0, eta_prev);
    // Inexact Newton safeguard: a loose Krylov tolerance on this ill-conditioned
    // operator can give a direction along which Phi barely decreases; when the
    // line search fails or accepts a step shorter than retry_alpha, the
    // direction is recomputed with a 100x tighter tolerance (down to
    // krylov_rtol, at most 3 times).
    double alpha = 1.0, phi1 = 0.0, scale1 = 0.0;
    bool ok = false, committed = false;
    for (int attempt = 0;; ++attempt) {
      TRY(fgmres(h, h->rhs, h->dv, eta, p.max_krylov, &kits));
      st->krylov_per_newton[it] += kits;
      st->krylov_iters_total += kits;
      // backtracking on Phi (Section 5.1); the unit step is tried first in one
      // fused pass that also yields R and pi at the trial point
      alpha = 1.0;
      ok = false;
      int k0 = 0;
      if (p.fused_trial && p.method == 0) {
        {
          Prof pr(h, SVN_K_ENERGY);
          double* pr_res = h->partial + (size_t)energy_partials(g) * (2 * MAX_ALPHA + 1);
          launch_trial(s, g, ph, h->v, h->dv, h->P, h->rhoH, h->fq, h->voq, h->pi, h->pi_t, h->eb, h->Rt,
                       h->partial, h->scal, pr_res);
          launch_sum_final(s, pr_res, residual_partials(g), h->scal + MAX_ALPHA + 1);
        }
        CKL();
        double out[MAX_ALPHA + 2];
        TRY(sync_read(h, h->scal, MAX_ALPHA + 2, out));
        phi1 = out[0];
        scale1 = out[MAX_ALPHA];
        const double rt = std::sqrt(out[MAX_ALPHA + 1]);
        ok = phi1 < phi0 || (std::fabs(phi1 - phi0) <= p.ls_floor * scale0 && rt < r);
        if (ok) {
          st->alpha_hist[it] = 1.0;
          launch_axpy(s, g, 1.0, h->dv, h->v);
          CKL();
          std::swap(h->pi, h->pi_t);
          std::swap(h->R, h->Rt);
          r_next = rt;
          have_r = true;
          phi0 = phi1;
          scale0 = scale1;
          committed = true;
          break;
        }
        st->halvings_total += 1;
        alpha = 0.5;
        k0 = 1;
      }
      for (int k = k0; k <= p.max_halvings; ++k) {
        TRY(energy(h, h->v, h->dv, &alpha, 1, &phi1, &scale1));
        if (phi1 < phi0) {
          ok = true;
        } else if (std::fabs(phi1 - phi0) <= p.ls_floor * scale0) {
          launch_axpby_to(s, g, h->v, alpha, h->dv, h->vt);
          CKL();
          double rn;
          TRY(residual(h, h->vt, h->w, &rn));
          ok = rn < r;
        }
        if (ok) break;
        st->halvings_total += 1;
        alpha *= 0.5;
      }
      const bool short_step = !ok || alpha < p.retry_alpha;
      if (short_step && eta > p.krylov_rtol && attempt < 3) {
        eta = std::max(p.krylov_rtol, 0.01 * eta);
        eta_prev = eta;
        st->direction_retries += 1;
        continue;
      }
      break;
    }
    if (committed) continue;
    if (!ok) return fail(h, SVN_ERR_LINESEARCH, "line search failed after %d halvings", p.max_halvings);
    st->alpha_hist[it] = alpha;
    if (p.method == 0) {
      Prof pr(h, SVN_K_DUAL);
      launch_dual_update(s, g, ph, alpha, h->v, h->dv, h->pi);
    }
    launch_axpy(s, g, alpha, h->dv, h->v);
    CKL();
    phi0 = phi1;
    scale0 = scale1;
  }
  CK(cudaStreamSynchronize(s));
  st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SVN_OK;
}

// ---- Q2 velocity elements ----------------------------------------------------------
// The Q2 step owns its cell and quadrature data and borrows a Q1 handle on the
// 2N grid (the same (2N+1)^2 nodes): its FGMRES workspace, and its V-cycle of
// the Q1 operator linearised at the same node velocities as the
// preconditioner -- Q1 on the refined grid is spectrally equivalent to Q2 on
// the coarse one, and FGMRES only needs an approximate inverse.  The Q1
// operator takes the Q2 iterate's dual state at the nearest Q2 point (with its
// own tau/Delta instead, FGMRES stalled at its iteration cap from 256^2 cells
// on).  The outer operator is the FP64 Q2 Jacobian.
}  // namespace

struct svn_q2 {
  svn_grid grid{};
  svn_params prm{};
  svn_handle* pre = nullptr;         // Q1 handle on the 2N grid (owned)
  std::string err;
  Q2Geom q{};
  double *in_h = nullptr, *in_A = nullptr, *in_wind = nullptr, *in_ocean = nullptr, *in_vold = nullptr;
  double *h2 = nullptr, *A2 = nullptr;   // cell fields refined to the 2N grid
  double *P = nullptr, *rhoH = nullptr, *fq = nullptr, *voq = nullptr, *pi = nullptr, *ke = nullptr, *eb = nullptr;
  double *pi_scratch = nullptr;
  double2 *v = nullptr, *dv = nullptr, *vt = nullptr, *R = nullptr, *rhs = nullptr;
  double *partial = nullptr, *scal = nullptr;
  bool have_forcing = false;
  double cur_dt = -1.0;
  bool pre_pi_q2 = true;   // preconditioner linearised with the Q2 pi (else its own tau/Delta)
  // Q2 smoother around the Q1 V-cycle (p-multigrid)
  double *dinv2 = nullptr, *coef2 = nullptr, *lmax2 = nullptr;
  double2 *px = nullptr, *pd = nullptr, *py = nullptr, *prc = nullptr, *pzc = nullptr;
};

namespace {

Phys q2_phys(const svn_q2* Q, double dt) {
  Phys ph = make_phys(Q->pre, Q->pre->g0, dt);
  ph.dx = Q->grid.L / Q->grid.N;      // Q2 cell width (the Q1 grid has half of it)
  ph.idx = 1.0 / ph.dx;
  ph.w = ph.dx * ph.dx;
  return ph;
}

int q2_create_impl(svn_q2* Q, const svn_grid* g, const svn_params* p, void* stream) {
  svn_grid g2{2 * g->N, g->L};
  if (g->N < 4 || g->N > 8192 || (g->N & 1)) {
    Q->err = "Q2: N must be even and in [4, 8192]";
    return SVN_ERR_ARG;
  }
  svn_params pp = *p;
  pp.fused_trial = 0;
  pp.learned = 0;
  const int rc = svn_create(&g2, &pp, stream, &Q->pre);
  if (rc != SVN_OK) {
    Q->err = Q->pre ? Q->pre->err : std::string("Q2: preconditioner handle");
    return rc;
  }
  svn_handle* h = Q->pre;
  Q->grid = *g;
  Q->prm = *p;
  if (q2_init_tables() != 0) return fail(h, SVN_ERR_CUDA, "Q2 basis tables");
  Q->q.N = g->N;
  Q->q.cpl = ((long long)g->N * g->N + 63) / 64 * 64;
  Q->q.gq = h->g0;
  const long long cpl = Q->q.cpl, pl = h->g0.plane;
  const size_t nc = (size_t)g->N * g->N, nv = 2 * (size_t)(2 * g->N + 1) * (2 * g->N + 1);
  TRY(dalloc(h, &Q->in_h, nc));
  TRY(dalloc(h, &Q->in_A, nc));
  TRY(dalloc(h, &Q->in_wind, nv));
  TRY(dalloc(h, &Q->in_ocean, nv));
  TRY(dalloc(h, &Q->in_vold, nv));
  TRY(dalloc(h, &Q->h2, 4 * nc));
  TRY(dalloc(h, &Q->A2, 4 * nc));
  TRY(dalloc(h, &Q->P, cpl));
  TRY(dalloc(h, &Q->rhoH, cpl));
  TRY(dalloc(h, &Q->fq, 18 * cpl));
  TRY(dalloc(h, &Q->voq, 18 * cpl));
  TRY(dalloc(h, &Q->pi, 27 * cpl));
  TRY(dalloc(h, &Q->pi_scratch, 27 * cpl));
  TRY(dalloc(h, &Q->ke, 171 * cpl));
  TRY(dalloc(h, &Q->eb, 18 * cpl));
  TRY(dalloc(h, &Q->v, pl));
  TRY(dalloc(h, &Q->dv, pl));
  TRY(dalloc(h, &Q->vt, pl));
  TRY(dalloc(h, &Q->R, pl));
  TRY(dalloc(h, &Q->rhs, pl));
  const size_t np = std::max<size_t>({(size_t)q2_node_partials(Q->q),
                                      (size_t)q2_energy_partials(Q->q) * (2 * MAX_ALPHA + 1), 4096});
  TRY(dalloc(h, &Q->partial, np));
  TRY(dalloc(h, &Q->scal, 64));
  TRY(dalloc(h, &Q->dinv2, 3 * pl));
  TRY(dalloc(h, &Q->coef2, 2 * 16 + 2));
  TRY(dalloc(h, &Q->lmax2, 1));
  TRY(dalloc(h, &Q->px, pl));
  TRY(dalloc(h, &Q->pd, pl));
  TRY(dalloc(h, &Q->py, pl));
  TRY(dalloc(h, &Q->prc, pl));
  TRY(dalloc(h, &Q->pzc, pl));
  return SVN_OK;
}

void q2_destroy_impl(svn_q2* Q) {
  dfree(Q->in_h); dfree(Q->in_A); dfree(Q->in_wind); dfree(Q->in_ocean); dfree(Q->in_vold);
  dfree(Q->h2); dfree(Q->A2); dfree(Q->P); dfree(Q->rhoH); dfree(Q->fq); dfree(Q->voq); dfree(Q->pi);
  dfree(Q->pi_scratch); dfree(Q->ke); dfree(Q->eb);
  dfree(Q->v); dfree(Q->dv); dfree(Q->vt); dfree(Q->R); dfree(Q->rhs); dfree(Q->partial); dfree(Q->scal);
  dfree(Q->dinv2); dfree(Q->coef2); dfree(Q->lmax2);
  dfree(Q->px); dfree(Q->pd); dfree(Q->py); dfree(Q->prc); dfree(Q->pzc);
  if (Q->pre) svn_destroy(Q->pre);
  Q->pre = nullptr;
}

int q2_precompute(svn_q2* Q, double dt) {
  svn_handle* h = Q->pre;
  if (!Q->have_forcing) return fail(h, SVN_ERR_STATE, "svn_q2_set_forcing has not been called");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, SVN_ERR_ARG, "dt must be positive and finite");
  launch_q2_precompute(h->stream, Q->q, dt, make_pc(Q->prm), Q->in_h, Q->in_A, Q->in_wind, Q->in_ocean, Q->in_vold,
                       Q->P, Q->rhoH, Q->fq, Q->voq);
  CKL();
  TRY(precompute(h, dt));    // the preconditioner's fields on the 2N grid
  Q->cur_dt = dt;
  return SVN_OK;
}

int q2_residual(svn_q2* Q, const double2* v, double2* R, double* norm) {
  svn_handle* h = Q->pre;
  {
    Prof pr(h, SVN_K_RESIDUAL);
    launch_q2_residual(h->stream, Q->q, q2_phys(Q, Q->cur_dt), v, Q->P, Q->rhoH, Q->fq, Q->voq, Q->eb, R,
                       Q->partial);
  }
  launch_sum_final(h->stream, Q->partial, q2_node_partials(Q->q), Q->scal);
  CKL();
  double s2;
  TRY(sync_read(h, Q->scal, 1, &s2));
  *norm = std::sqrt(s2);
  return SVN_OK;
}

int q2_energy(svn_q2* Q, const double2* v, const double2* dv, const double* alphas, int k, double* phi,
              double* scale) {
  svn_handle* h = Q->pre;
  if (k < 1 || k > MAX_ALPHA) return fail(h, SVN_ERR_ARG, "energy: 1 <= k <= %d", MAX_ALPHA);
  AlphaSet al{};
  for (int a = 0; a < k; ++a) al.a[a] = alphas[a];
  {
    Prof pr(h, SVN_K_ENERGY);
    launch_q2_energy(h->stream, Q->q, q2_phys(Q, Q->cur_dt), k, al, v, dv, Q->P, Q->rhoH, Q->fq, Q->voq, Q->partial,
                     Q->scal);
  }
  CKL();
  double out[MAX_ALPHA + 1];
  TRY(sync_read(h, Q->scal, MAX_ALPHA + 1, out));
  for (int a = 0; a < k; ++a) phi[a] = out[a];
  if (scale) *scale = out[MAX_ALPHA];
  return SVN_OK;
}

// Q2 element matrices at (v, pi) and the preconditioner's Q1 hierarchy at v.
int q2_linearize(svn_q2* Q, const double2* v, const double* pi) {
  svn_handle* h = Q->pre;
  {
    Prof pr(h, SVN_K_ELEMENT);
    launch_q2_element_matrices(h->stream, Q->q, q2_phys(Q, Q->cur_dt), v, pi, Q->P, Q->rhoH, Q->voq, Q->ke);
  }
  CKL();
  if (Q->pre_pi_q2)
    launch_q2_pi_to_q1(h->stream, Q->q, pi, h->pi);   // the Q2 iterate's dual state
  else
    launch_pi_init(h->stream, h->g0, make_phys(h, h->g0, h->cur_dt), v, h->pi);
  CKL();
  TRY(linearize(h, v, h->pi));
  Q->pre->outer = [Q](const double2* x, double2* y) {
    launch_q2_apply(Q->pre->stream, Q->q, Q->ke, x, Q->eb, y);
  };
  const int deg = Q->prm.q2_smooth_degree;
  if (deg <= 0) {
    Q->pre->pre_op = nullptr;
    return SVN_OK;
  }
  // Chebyshev-block-Jacobi smoothing on the Q2 operator: D^-1 from the element
  // matrices, lambda_max(D^-1 A) by power steps from a checkerboard (a smooth
  // start vector underestimates it, and Chebyshev then amplifies the top modes)
  cudaStream_t s = h->stream;
  const Layout& g = Q->q.gq;
  launch_q2_dinv(s, Q->q, Q->ke, Q->dinv2);
  launch_q2_checker(s, Q->q, Q->px);
  CKL();
  double nx = 0.0, ny = 0.0;
  TRY(norm2(h, Q->px, &nx));
  for (int k = 0; k < std::max(10, Q->prm.lmax_iters) && nx > 0.0; ++k) {
    launch_scale_to(s, g, 1.0 / nx, Q->px, Q->px);
    launch_q2_apply(s, Q->q, Q->ke, Q->px, Q->eb, Q->py);
    launch_q2_dinv_apply(s, Q->q, Q->dinv2, Q->py, Q->px);
    CKL();
    TRY(norm2(h, Q->px, &ny));
    nx = ny;
  }
  const double lmax = (nx > 0.0 && std::isfinite(nx) ? nx : 1.0) * Q->prm.lmax_safety;
  double* hb = h->hostbuf;
  hb[0] = lmax;
  CK(cudaMemcpyAsync(Q->lmax2, hb, sizeof(double), cudaMemcpyHostToDevice, s));
  launch_cheb_coefs<double>(s, Q->lmax2, Q->prm.cheb_lo, deg, Q->coef2);
  CKL();
  CK(cudaStreamSynchronize(s));   // hostbuf reuse
  // M^-1 r: deg Chebyshev steps from 0, the Q1 V-cycle on the residual, deg steps again
  Q->pre->pre_op = [Q, deg](const double2* r, double2* z) -> int {
    svn_handle* hh = Q->pre;
    svn_handle* h = hh;   // for the error macros
    cudaStream_t st = hh->stream;
    const Layout& gg = Q->q.gq;
    const size_t bytes = sizeof(double2) * gg.plane;
    CK(cudaMemsetAsync(Q->px, 0, bytes, st));
    CK(cudaMemsetAsync(Q->pd, 0, bytes, st));
    CK(cudaMemsetAsync(Q->py, 0, bytes, st));
    for (int k = 0; k < deg; ++k) {
      if (k > 0) launch_q2_apply(st, Q->q, Q->ke, Q->px, Q->eb, Q->py);
      launch_q2_cheb_step(st, Q->q, Q->dinv2, Q->coef2, k, r, Q->py, Q->px, Q->pd);
    }
    launch_q2_apply(st, Q->q, Q->ke, Q->px, Q->eb, Q->py);
    launch_axpby_to(st, gg, r, -1.0, Q->py, Q->prc);
    CKL();
    TRY(precondition_mg(hh, Q->prc, Q->pzc));
    launch_axpy(st, gg, 1.0, Q->pzc, Q->px);
    CK(cudaMemsetAsync(Q->pd, 0, bytes, st));
    for (int k = 0; k < deg; ++k) {
      launch_q2_apply(st, Q->q, Q->ke, Q->px, Q->eb, Q->py);
      launch_q2_cheb_step(st, Q->q, Q->dinv2, Q->coef2, k, r, Q->py, Q->px, Q->pd);
    }
    CK(cudaMemcpyAsync(z, Q->px, bytes, cudaMemcpyDeviceToDevice, st));
    CKL();
    return SVN_OK;
  };
  return SVN_OK;
}

// One implicit step on Q2 elements: the damped svN iteration of step_impl with
// the Q2 residual, energy, operator and dual update (Sections 4.2 and 5.1).
int q2_step_impl(svn_q2* Q, double dt, double tol, svn_stats* st) {
  svn_handle* h = Q->pre;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = h->stream;
  const Layout& g = Q->q.gq;
  st->status = SVN_OK;
  TRY(q2_precompute(Q, dt));
  if (!(tol > 0.0)) return fail(h, SVN_ERR_ARG, "tol must be positive");
  const Phys ph = q2_phys(Q, dt);
  launch_unpack_nodes(s, g, Q->in_vold, Q->v);
  CKL();
  TRY(q2_residual(Q, Q->v, Q->R, &st->res0));
  launch_q2_pi_init(s, Q->q, ph, Q->v, Q->pi);
  CKL();
  const svn_params& p = Q->prm;
  double phi0 = 0.0, scale0 = 0.0;
  {
    const double a0 = 0.0;
    TRY(q2_energy(Q, Q->v, Q->v, &a0, 1, &phi0, &scale0));
  }
  double eta_prev = p.ew_eta_max;
  for (int it = 0;; ++it) {
    double r;
    TRY(q2_residual(Q, Q->v, Q->R, &r));
    st->res_hist[it] = r;
    st->newton_iters = it;
    st->res_final = r;
    st->rel_res_final = st->res0 > 0 ? r / st->res0 : 0.0;
    if (!std::isfinite(r)) return fail(h, SVN_ERR_NONFINITE, "non-finite residual norm at Newton iteration %d", it);
    if (r <= tol * st->res0 || r == 0.0) break;
    if (it >= p.max_newton)
      return fail(h, SVN_ERR_NO_CONVERGENCE, "no convergence in %d Newton iterations (rel-res %.3e)", it,
                  st->rel_res_final);
    if (p.method == 1) {
      launch_q2_pi_init(s, Q->q, ph, Q->v, Q->pi);
      CKL();
    }
    TRY(q2_linearize(Q, Q->v, Q->pi));
    launch_neg_copy(s, g, Q->R, Q->rhs);
    CKL();
    double eta = forcing_term(p, it, r, it > 0 ? st->res_hist[it - 1] : 0.0, tol * st->res0, eta_prev);
    // FGMRES on the Q2 operator, backtracking on Phi in batches of eight step
    // lengths per energy pass, and the retry_alpha safeguard of step_impl
    double alpha = 1.0, phi1 = 0.0, scale1 = 0.0;
    bool ok = false;
    for (int attempt = 0;; ++attempt) {
      int kits = 0;
      TRY(fgmres(h, Q->rhs, Q->dv, eta, p.max_krylov, &kits));
      st->krylov_per_newton[it] += kits;
      st->krylov_iters_total += kits;
      ok = false;
      double a = 1.0;
      for (int k0 = 0; k0 <= p.max_halvings && !ok; k0 += MAX_ALPHA) {
        const int nk = std::min(MAX_ALPHA, p.max_halvings + 1 - k0);
        double al[MAX_ALPHA], ph_[MAX_ALPHA];
        for (int k = 0; k < nk; ++k) al[k] = a * std::ldexp(1.0, -k);
        TRY(q2_energy(Q, Q->v, Q->dv, al, nk, ph_, &scale1));
        for (int k = 0; k < nk && !ok; ++k) {
          if (ph_[k] < phi0) {
            ok = true;
          } else if (std::fabs(ph_[k] - phi0) <= p.ls_floor * scale0) {
            launch_axpby_to(s, g, Q->v, al[k], Q->dv, Q->vt);
            CKL();
            double rn;
            TRY(q2_residual(Q, Q->vt, h->w, &rn));   // h->w: Krylov scratch, free after FGMRES
            ok = rn < r;
          }
          if (ok) {
            alpha = al[k];
            phi1 = ph_[k];
            st->halvings_total += k0 + k;
          }
        }
        a = std::ldexp(a, -nk);
      }
      if (!ok) st->halvings_total += p.max_halvings;
      const bool short_step = !ok || alpha < p.retry_alpha;
      if (short_step && eta > p.krylov_rtol && attempt < 3) {
        eta = std::max(p.krylov_rtol, 0.01 * eta);
        eta_prev = eta;
        st->direction_retries += 1;
        continue;
      }
      break;
    }
    if (!ok) return fail(h, SVN_ERR_LINESEARCH, "line search failed after %d halvings", p.max_halvings);
    st->alpha_hist[it] = alpha;
    if (p.method == 0) {
      Prof pr(h, SVN_K_DUAL);
      launch_q2_dual_update(s, Q->q, ph, alpha, Q->v, Q->dv, Q->pi);
    }
    launch_axpy(s, g, alpha, Q->dv, Q->v);
    CKL();
    phi0 = phi1;
    // the rounding scale of Phi at the new iterate (one more energy pass)
    {
      const double a0 = 0.0;
      double dummy;
      TRY(q2_energy(Q, Q->v, Q->v, &a0, 1, &dummy, &scale0));
    }
  }
  CK(cudaStreamSynchronize(s));
  st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SVN_OK;
}

int ensure_pi_scratch(svn_handle* h) {
  if (!h->pi_scratch) TRY(dalloc(h, &h->pi_scratch, 12 * (size_t)h->g0.plane));
  return SVN_OK;
}

}  // namespace

// ============================== C ABI ==============================================

extern "C" {

int svn_default_params(svn_params* p) {
  if (!p) return SVN_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->rho_ice = 900.0; p->rho_a = 1.3; p->rho_o = 1026.0; p->Ca = 1.2e-3; p->Co = 5.5e-3;
  p->f_c = 1.46e-4; p->Pstar = 27500.0; p->C = 20.0; p->e = 2.0; p->delta_min = 2e-9;
  p->max_newton = 200;
  p->max_halvings = 30;
  p->ls_floor = 1e-13;
  p->krylov_rtol = 1e-6;
  p->restart = 30;
  p->max_krylov = 600;
  p->precision = SVN_FP64;
  p->cheb_degree = 3;
  p->cheb_lo = 0.05;
  p->coarse_N = 4;
  p->eisenstat_walker = 0;
  p->learned = 0;
  p->use_graphs = 1;
  p->reorth_always = 0;
  p->ew_eta_max = 0.1;
  p->lmax_iters = 15;
  p->lmax_safety = 1.15;
  p->vcycle_fp32 = 1;
  p->cheb_degree_coarse = 0;
  p->fused_trial = 1;
  p->learned_rule = 0;
  p->cheb_fuse = 1;
  p->mg_rebuild = 1;
  p->method = 0;
  p->retry_alpha = 1.0 / 64.0;
  p->ew_tail = 0.5;
  p->q2_smooth_degree = 3;
  return SVN_OK;
}

int svn_create(const svn_grid* g, const svn_params* p, void* cuda_stream, svn_handle** out) {
  if (!out) return SVN_ERR_ARG;
  *out = nullptr;
  svn_handle* h = new (std::nothrow) svn_handle();
  if (!h) return SVN_ERR_OOM;
  int rc = create_impl(h, g, p, cuda_stream);
  if (rc != SVN_OK) {
    // keep the handle so the caller can read the message; it owns nothing usable
    destroy_impl(h);
  }
  *out = h;
  return rc;
}

int svn_destroy(svn_handle* h) {
  if (!h) return SVN_ERR_ARG;
  destroy_impl(h);
  delete h;
  return SVN_OK;
}

const char* svn_last_error(const svn_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

int svn_set_forcing(svn_handle* h, const double* hc, const double* A, const double* wind, const double* ocean,
                    const double* v_old) {
  if (!h) return SVN_ERR_ARG;
  return set_forcing_impl(h, hc, A, wind, ocean, v_old, false);
}

int svn_set_forcing_host(svn_handle* h, const double* hc, const double* A, const double* wind, const double* ocean,
                         const double* v_old) {
  if (!h) return SVN_ERR_ARG;
  return set_forcing_impl(h, hc, A, wind, ocean, v_old, true);
}

static int step_common(svn_handle* h, double dt, double tol, double* out_v, svn_stats* stats, bool host,
                       bool commit = false) {
  if (!h) return SVN_ERR_ARG;
  svn_stats local;
  svn_stats* st = stats ? stats : &local;
  memset(st, 0, sizeof(*st));
  int rc = step_impl(h, dt, tol, st);
  st->status = rc;
  const Layout& g = h->g0;
  const size_t nv = 2 * (size_t)(g.N + 1) * (g.N + 1);
  if (out_v && h->v) {
    if (host) {
      double* tmp = (double*)h->rhs;   // scratch of 2 * plane >= nv doubles
      launch_pack_nodes(h->stream, g, h->v, tmp);
      cudaMemcpyAsync(out_v, tmp, sizeof(double) * nv, cudaMemcpyDeviceToHost, h->stream);
      cudaStreamSynchronize(h->stream);
    } else {
      launch_pack_nodes(h->stream, g, h->v, out_v);
      cudaStreamSynchronize(h->stream);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && rc == SVN_OK) rc = fail(h, SVN_ERR_CUDA, "output copy: %s", cudaGetErrorString(e));
  }
  if (commit && rc == SVN_OK) {
    // the solution becomes v^n of the next time step
    launch_pack_nodes(h->stream, g, h->v, h->in_vold);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = fail(h, SVN_ERR_CUDA, "velocity commit: %s", cudaGetErrorString(e));
    st->status = rc;
  }
  return rc;
}

int svn_step(svn_handle* h, double dt, double tol, double* out_v, svn_stats* stats) {
  return step_common(h, dt, tol, out_v, stats, false);
}

int svn_step_host(svn_handle* h, double dt, double tol, double* out_v, svn_stats* stats) {
  return step_common(h, dt, tol, out_v, stats, true);
}

int svn_transport(svn_handle* h, double dt, int* substeps) {
  if (!h) return SVN_ERR_ARG;
  int n = 0;
  const int rc = transport_impl(h, dt, &n);
  if (substeps) *substeps = n;
  return rc;
}

int svn_get_ice(svn_handle* h, double* hcell, double* A) {
  if (!h || !hcell || !A) return SVN_ERR_ARG;
  const size_t nc = (size_t)h->grid.N * h->grid.N;
  CK(cudaMemcpyAsync(hcell, h->in_h, sizeof(double) * nc, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(A, h->in_A, sizeof(double) * nc, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_advance(svn_handle* h, double dt, double tol, const double* wind, const double* ocean, double* out_v,
                svn_stats* stats, int* substeps) {
  if (!h) return SVN_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  int n = 0;
  int rc = transport_impl(h, dt, &n);
  if (substeps) *substeps = n;
  if (rc == SVN_OK && (wind || ocean)) {
    const size_t nv = 2 * (size_t)(h->grid.N + 1) * (h->grid.N + 1);
    if (wind) CK(cudaMemcpyAsync(h->in_wind, wind, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream));
    if (ocean) CK(cudaMemcpyAsync(h->in_ocean, ocean, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->stream));
    h->have_forcing = false;
    rc = validate_forcing(h);
    if (rc == SVN_OK) h->have_forcing = true;
  }
  if (rc != SVN_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  return step_common(h, dt, tol, out_v, stats, false, true);
}

int svn_get_state(svn_handle* h, double* v, double* pi) {
  if (!h || !v || !pi) return SVN_ERR_ARG;
  launch_pack_nodes(h->stream, h->g0, h->v, v);
  launch_pack_pi(h->stream, h->g0, h->pi, pi);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_set_state(svn_handle* h, const double* v, const double* pi) {
  if (!h || !v || !pi) return SVN_ERR_ARG;
  launch_unpack_nodes(h->stream, h->g0, v, h->v);
  launch_unpack_pi(h->stream, h->g0, pi, h->pi);
  CKL();
  h->state_set = true;
  return SVN_OK;
}

int svn_residual(svn_handle* h, double dt, const double* v, double* R, double* norm) {
  if (!h || !v || !R) return SVN_ERR_ARG;
  TRY(precompute(h, dt));
  launch_unpack_nodes(h->stream, h->g0, v, h->vt);
  CKL();
  double nrm;
  TRY(residual(h, h->vt, h->w, &nrm));
  launch_pack_nodes(h->stream, h->g0, h->w, R);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  if (norm) *norm = nrm;
  return SVN_OK;
}

int svn_energy(svn_handle* h, double dt, const double* v, const double* dv, const double* alphas, int k, double* phi,
               double* scale) {
  if (!h || !v || !dv || !alphas || !phi) return SVN_ERR_ARG;
  TRY(precompute(h, dt));
  launch_unpack_nodes(h->stream, h->g0, v, h->vt);
  launch_unpack_nodes(h->stream, h->g0, dv, h->w);
  CKL();
  return energy(h, h->vt, h->w, alphas, k, phi, scale);
}

int svn_linearize(svn_handle* h, double dt, const double* v, const double* pi) {
  if (!h || !v || !pi) return SVN_ERR_ARG;
  TRY(precompute(h, dt));
  TRY(ensure_pi_scratch(h));
  launch_unpack_nodes(h->stream, h->g0, v, h->vt);
  launch_unpack_pi(h->stream, h->g0, pi, h->pi_scratch);
  CKL();
  return linearize(h, h->vt, h->pi_scratch);
}

int svn_apply(svn_handle* h, int level, const double* x, double* y) {
  if (!h || !x || !y) return SVN_ERR_ARG;
  if (level < 0 || level >= (int)h->lv.size()) return fail(h, SVN_ERR_ARG, "level out of range");
  const Layout& g = h->lv[level].g;
  launch_unpack_nodes(h->stream, g, x, h->vt);
  launch_apply<double, double2, double2, double>(h->stream, g, h->lv[level].st64, h->vt, h->w);
  launch_pack_nodes(h->stream, g, h->w, y);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_precondition(svn_handle* h, const double* r, double* z) {
  if (!h || !r || !z) return SVN_ERR_ARG;
  const Layout& g = h->g0;
  launch_unpack_nodes(h->stream, g, r, h->vt);
  CKL();
  TRY(precondition(h, h->vt, h->w));
  launch_pack_nodes(h->stream, g, h->w, z);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_krylov_solve(svn_handle* h, const double* b, double* x, double rtol, int* iters) {
  if (!h || !b || !x) return SVN_ERR_ARG;
  const Layout& g = h->g0;
  launch_unpack_nodes(h->stream, g, b, h->rhs);
  CKL();
  int its = 0;
  int rc = fgmres(h, h->rhs, h->dv, rtol, h->prm.max_krylov, &its);
  if (iters) *iters = its;
  launch_pack_nodes(h->stream, g, h->dv, x);
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

int svn_dual_update(svn_handle* h, double dt, const double* v, const double* dv, double alpha, double* pi) {
  if (!h || !v || !dv || !pi) return SVN_ERR_ARG;
  TRY(precompute(h, dt));
  TRY(ensure_pi_scratch(h));
  const Layout& g = h->g0;
  launch_unpack_nodes(h->stream, g, v, h->vt);
  launch_unpack_nodes(h->stream, g, dv, h->w);
  launch_unpack_pi(h->stream, g, pi, h->pi_scratch);
  launch_dual_update(h->stream, g, make_phys(h, g, dt), alpha, h->vt, h->w, h->pi_scratch);
  launch_pack_pi(h->stream, g, h->pi_scratch, pi);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_profile(svn_handle* h, int enable) {
  if (!h) return SVN_ERR_ARG;
  prof_collect(h);
  if ((enable != 0) != h->prof_on) h->graph_dirty = true;   // re-record with / without sweep events
  if (enable) {
    for (int c = 0; c < SVN_K_COUNT; ++c) {
      h->prof_ms[c] = 0.0;
      h->prof_n[c] = 0;
    }
  }
  h->prof_on = enable != 0;
  return SVN_OK;
}

int svn_profile_read(svn_handle* h, int kclass, double* ms_total, long long* launches) {
  if (!h || kclass < 0 || kclass >= SVN_K_COUNT) return SVN_ERR_ARG;
  prof_collect(h);
  if (ms_total) *ms_total = h->prof_ms[kclass];
  if (launches) *launches = h->prof_n[kclass];
  return SVN_OK;
}

unsigned long long svn_kernel_launches(void) { return launches_issued(); }

// ---- batched ensembles ------------------------------------------------------------
// n independent instances (any mix of grid sizes), one handle and one private
// non-blocking stream each; svn_batch_step drives them concurrently from a pool
// of host threads so that small grids share the GPU.

struct svn_batch {
  std::vector<svn_handle*> hs;
  std::vector<cudaStream_t> streams;
  int device = 0;
  int threads = 8;
  std::string err;
};

int svn_batch_create(int n, const svn_grid* grids, const svn_params* p, int host_threads, svn_batch** out) {
  if (!out) return SVN_ERR_ARG;
  *out = nullptr;
  if (n < 1 || n > 4096 || !grids || !p) return SVN_ERR_ARG;
  svn_batch* b = new (std::nothrow) svn_batch();
  if (!b) return SVN_ERR_OOM;
  *out = b;
  cudaGetDevice(&b->device);
  b->threads = std::max(1, std::min(host_threads > 0 ? host_threads : 8, n));
  for (int i = 0; i < n; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      b->err = "stream creation failed";
      return SVN_ERR_CUDA;
    }
    b->streams.push_back(st);
    svn_handle* h = nullptr;
    const int rc = svn_create(&grids[i], p, st, &h);
    b->hs.push_back(h);
    if (rc != SVN_OK) {
      b->err = "instance " + std::to_string(i) + ": " + (h ? h->err : std::string("create failed"));
      return rc;
    }
  }
  return SVN_OK;
}

int svn_batch_destroy(svn_batch* b) {
  if (!b) return SVN_ERR_ARG;
  for (svn_handle* h : b->hs)
    if (h) svn_destroy(h);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
  return SVN_OK;
}

const char* svn_batch_last_error(const svn_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

int svn_batch_size(const svn_batch* b) { return b ? (int)b->hs.size() : 0; }

svn_handle* svn_batch_instance(svn_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->hs.size()) return nullptr;
  return b->hs[i];
}

int svn_batch_step(svn_batch* b, double dt, double tol, double* const* out_v, svn_stats* stats) {
  if (!b || !out_v) return SVN_ERR_ARG;
  const int n = (int)b->hs.size();
  std::vector<int> rcs(n, SVN_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(b->device);
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1))
      rcs[i] = step_common(b->hs[i], dt, tol, out_v[i], stats ? &stats[i] : nullptr, false);
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < b->threads; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  // every failing instance is named in the message; the first one's code is returned
  int first = SVN_OK, nfail = 0;
  std::string msg;
  for (int i = 0; i < n; ++i)
    if (rcs[i] != SVN_OK) {
      if (first == SVN_OK) first = rcs[i];
      if (++nfail <= 8) msg += (msg.empty() ? "" : "; ") + std::string("instance ") + std::to_string(i) + ": " +
                               b->hs[i]->err;
    }
  if (nfail > 8) msg += "; ... (" + std::to_string(nfail) + " instances failed)";
  b->err = msg;
  return first;
}

// ---- autotuner --------------------------------------------------------------------
// Times FGMRES on the linearisation reached after `probe_newton` Newton
// iterations of the current forcing, for every (degree, lo) candidate, and
// keeps the fastest in the handle's parameters.
static int autotune_impl(svn_handle* h, double dt, int probe_newton, const int* degrees, int nd, const double* los,
                         int nl, const int* fuses, int nf, double* best_ms) {
  if (!h || !degrees || !los || !fuses || nd < 1 || nl < 1 || nf < 1) return SVN_ERR_ARG;
  for (int i = 0; i < nd; ++i)
    if (degrees[i] < 1 || degrees[i] > 16) return fail(h, SVN_ERR_ARG, "degree out of range");
  for (int i = 0; i < nl; ++i)
    if (!(los[i] > 0.0 && los[i] < 1.0)) return fail(h, SVN_ERR_ARG, "lo out of range");
  for (int i = 0; i < nf; ++i)
    if (fuses[i] < 0 || fuses[i] > 5) return fail(h, SVN_ERR_ARG, "sweep kernel setting out of range");
  svn_params saved = h->prm;
  svn_stats st;
  memset(&st, 0, sizeof(st));
  h->prm.max_newton = std::max(1, probe_newton);
  step_impl(h, dt, 1e-300, &st);   // ends with SVN_ERR_NO_CONVERGENCE by design
  h->prm = saved;
  TRY(precompute(h, dt));
  TRY(residual(h, h->v, h->R, &st.res_final));
  launch_neg_copy(h->stream, h->g0, h->R, h->rhs);
  CKL();
  double best = 1e300;
  int bd = saved.cheb_degree, bf = saved.cheb_fuse;
  double bl = saved.cheb_lo;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // every candidate runs inside this lambda, so that an error on any of them
  // still frees the events and restores the handle's own smoother settings
  auto sweep = [&]() -> int {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int f = 0; f < nf; ++f)
      for (int a = 0; a < nd; ++a)
        for (int c = 0; c < nl; ++c) {
          h->prm.cheb_degree = degrees[a];
          h->prm.cheb_lo = los[c];
          h->prm.cheb_fuse = fuses[f];
          h->graph_dirty = true;
          TRY(linearize(h, h->v, h->pi));
          int its = 0;
          TRY(fgmres(h, h->rhs, h->dv, saved.krylov_rtol, saved.max_krylov, &its));   // warm (records the graph)
          CK(cudaEventRecord(e0, h->stream));
          TRY(fgmres(h, h->rhs, h->dv, saved.krylov_rtol, saved.max_krylov, &its));
          CK(cudaEventRecord(e1, h->stream));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) {
            best = ms;
            bd = degrees[a];
            bl = los[c];
            bf = fuses[f];
          }
        }
    return SVN_OK;
  };
  const int rc = sweep();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != SVN_OK) {
    h->prm = saved;
    h->graph_dirty = true;
    return rc;
  }
  h->prm.cheb_degree = bd;
  h->prm.cheb_lo = bl;
  h->prm.cheb_fuse = bf;
  h->graph_dirty = true;
  if (best_ms) *best_ms = best;
  return SVN_OK;
}

int svn_autotune(svn_handle* h, double dt, int probe_newton, const int* degrees, int nd, const double* los, int nl,
                 double* best_ms) {
  if (!h) return SVN_ERR_ARG;
  const int fuse = h->prm.cheb_fuse;
  return autotune_impl(h, dt, probe_newton, degrees, nd, los, nl, &fuse, 1, best_ms);
}

int svn_set_smoother(svn_handle* h, int cheb_fuse, int cheb_degree, double cheb_lo) {
  if (!h) return SVN_ERR_ARG;
  svn_params p = h->prm;
  p.cheb_fuse = cheb_fuse;
  p.cheb_degree = cheb_degree;
  p.cheb_lo = cheb_lo;
  TRY(check_params(h, &p));
  h->prm = p;
  h->graph_dirty = true;   // the V-cycle graph is recorded again; the next linearisation recomputes its coefficients
  return SVN_OK;
}

int svn_autotune_kernels(svn_handle* h, double dt, int probe_newton, const int* degrees, int nd, const double* los,
                         int nl, const int* cheb_fuses, int nf, double* best_ms) {
  return autotune_impl(h, dt, probe_newton, degrees, nd, los, nl, cheb_fuses, nf, best_ms);
}

// ---- Q2 velocity elements ------------------------------------------------------------
int svn_q2_create(const svn_grid* g, const svn_params* p, void* cuda_stream, svn_q2** out) {
  if (!out) return SVN_ERR_ARG;
  *out = nullptr;
  if (!g || !p) return SVN_ERR_ARG;
  svn_q2* Q = new (std::nothrow) svn_q2();
  if (!Q) return SVN_ERR_OOM;
  const int rc = q2_create_impl(Q, g, p, cuda_stream);
  if (rc != SVN_OK) {
    if (Q->pre && !Q->pre->err.empty()) Q->err = Q->pre->err;
    q2_destroy_impl(Q);
  }
  *out = Q;
  return rc;
}

int svn_q2_destroy(svn_q2* Q) {
  if (!Q) return SVN_ERR_ARG;
  q2_destroy_impl(Q);
  delete Q;
  return SVN_OK;
}

const char* svn_q2_last_error(const svn_q2* Q) {
  if (!Q) return "NULL handle";
  return (Q->pre && !Q->pre->err.empty()) ? Q->pre->err.c_str() : Q->err.c_str();
}

int svn_q2_set_forcing(svn_q2* Q, const double* hc, const double* A, const double* wind, const double* ocean,
                       const double* v_old) {
  if (!Q || !Q->pre) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  if (!hc || !A || !wind || !ocean || !v_old) return fail(h, SVN_ERR_ARG, "NULL forcing pointer");
  const int N = Q->grid.N;
  const size_t nc = (size_t)N * N, nv = 2 * (size_t)(2 * N + 1) * (2 * N + 1);
  cudaStream_t s = h->stream;
  CK(cudaMemcpyAsync(Q->in_h, hc, sizeof(double) * nc, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(Q->in_A, A, sizeof(double) * nc, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(Q->in_wind, wind, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(Q->in_ocean, ocean, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(Q->in_vold, v_old, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
  launch_q2_refine_cells(s, N, Q->in_h, Q->h2);
  launch_q2_refine_cells(s, N, Q->in_A, Q->A2);
  CKL();
  Q->have_forcing = false;
  // the preconditioner's copy (and the checks of svn_set_forcing)
  TRY(set_forcing_impl(h, Q->h2, Q->A2, Q->in_wind, Q->in_ocean, Q->in_vold, false));
  Q->have_forcing = true;
  return SVN_OK;
}

int svn_q2_step(svn_q2* Q, double dt, double tol, double* out_v, svn_stats* stats) {
  if (!Q || !Q->pre) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  svn_stats local;
  svn_stats* st = stats ? stats : &local;
  memset(st, 0, sizeof(*st));
  int rc = q2_step_impl(Q, dt, tol, st);
  st->status = rc;
  if (out_v) {
    launch_pack_nodes(h->stream, Q->q.gq, Q->v, out_v);
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess && rc == SVN_OK) rc = fail(h, SVN_ERR_CUDA, "output copy: %s", cudaGetErrorString(e));
  }
  return rc;
}

int svn_q2_residual(svn_q2* Q, double dt, const double* v, double* R, double* norm) {
  if (!Q || !Q->pre || !v || !R) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  TRY(q2_precompute(Q, dt));
  launch_unpack_nodes(h->stream, Q->q.gq, v, Q->vt);
  CKL();
  double nrm;
  TRY(q2_residual(Q, Q->vt, h->w, &nrm));
  launch_pack_nodes(h->stream, Q->q.gq, h->w, R);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  if (norm) *norm = nrm;
  return SVN_OK;
}

int svn_q2_energy(svn_q2* Q, double dt, const double* v, const double* dv, const double* alphas, int k, double* phi,
                  double* scale) {
  if (!Q || !Q->pre || !v || !dv || !alphas || !phi) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  TRY(q2_precompute(Q, dt));
  launch_unpack_nodes(h->stream, Q->q.gq, v, Q->vt);
  launch_unpack_nodes(h->stream, Q->q.gq, dv, Q->rhs);
  CKL();
  return q2_energy(Q, Q->vt, Q->rhs, alphas, k, phi, scale);
}

int svn_q2_linearize(svn_q2* Q, double dt, const double* v, const double* pi) {
  if (!Q || !Q->pre || !v || !pi) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  TRY(q2_precompute(Q, dt));
  launch_unpack_nodes(h->stream, Q->q.gq, v, Q->vt);
  launch_q2_pi_layout(h->stream, Q->q, pi, Q->pi_scratch, true);
  CKL();
  TRY(q2_linearize(Q, Q->vt, Q->pi_scratch));
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_q2_apply(svn_q2* Q, const double* x, double* y) {
  if (!Q || !Q->pre || !x || !y) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  launch_unpack_nodes(h->stream, Q->q.gq, x, Q->vt);
  launch_q2_apply(h->stream, Q->q, Q->ke, Q->vt, Q->eb, h->w);
  launch_pack_nodes(h->stream, Q->q.gq, h->w, y);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_q2_dual_update(svn_q2* Q, double dt, const double* v, const double* dv, double alpha, double* pi) {
  if (!Q || !Q->pre || !v || !dv || !pi) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  TRY(q2_precompute(Q, dt));
  launch_unpack_nodes(h->stream, Q->q.gq, v, Q->vt);
  launch_unpack_nodes(h->stream, Q->q.gq, dv, Q->rhs);
  launch_q2_pi_layout(h->stream, Q->q, pi, Q->pi_scratch, true);
  launch_q2_dual_update(h->stream, Q->q, q2_phys(Q, dt), alpha, Q->vt, Q->rhs, Q->pi_scratch);
  launch_q2_pi_layout(h->stream, Q->q, Q->pi_scratch, pi, false);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_q2_get_state(svn_q2* Q, double* v, double* pi) {
  if (!Q || !Q->pre || !v || !pi) return SVN_ERR_ARG;
  svn_handle* h = Q->pre;
  launch_pack_nodes(h->stream, Q->q.gq, Q->v, v);
  launch_q2_pi_layout(h->stream, Q->q, Q->pi, pi, false);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return SVN_OK;
}

int svn_attach_net(svn_handle* h, svn_net* net) {
  if (!h) return SVN_ERR_ARG;
  h->net = svn_net_impl(net);
  return SVN_OK;
}

int svn_set_learned(svn_handle* h, int on) {
  if (!h) return SVN_ERR_ARG;
  h->prm.learned = on ? 1 : 0;
  return SVN_OK;
}

int svn_get_params(const svn_handle* h, svn_params* p) {
  if (!h || !p) return SVN_ERR_ARG;
  *p = h->prm;
  return SVN_OK;
}

}  // extern "C"
