// Allocation-free variant of the residual entry point (svn_residual_noalloc).
//
// Some callers cannot call cudaMalloc: a host model that gives the whole
// device to its own memory pool at start-up, or a runtime that must keep its
// device footprint fixed after initialisation and so forbids allocation
// (and the failures it can bring) in the middle of a run.  For them this file
// holds all intermediate data of the residual -- ice strength, the per-point
// source terms, padded copies of v and R, the element buffer and the
// reduction partials -- in one file-scope device array of fixed size, so the
// call needs nothing from the caller but its inputs and outputs.
//
// The array is shared by every call on a device and keeps the contents of the
// last call; every region a call reads is written earlier in the same call,
// so nothing needs clearing.  Calls that overlap on the GPU (on different
// streams, or from different host threads) race on the array.
#include <cmath>

#include "../../include/svn.h"
#include "kernels.h"

namespace {

using namespace svn;

// Largest grid: N = SVN_NOALLOC_MAX_N cells per side.  30 planes of the padded
// node layout plus room for the reduction partials.
constexpr int kMaxN = SVN_NOALLOC_MAX_N;
constexpr long long kPlaneMax = ((long long)(kMaxN + 1) * (((kMaxN + 1) + 7) / 8 * 8) + 63) / 64 * 64;
constexpr int kPlanes = 30;   // P 1, rhoH 1, fq 8, voq 8, v 2, R 2, element buffer 8
constexpr long long kTail = 2048;
constexpr long long kScratchDoubles = kPlanes * kPlaneMax + kTail;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

// Device address of g_scratch in the current device's context, looked up on
// every call (a cheap table lookup once the module is loaded), so that a call
// after a device reset or on a re-created primary context never launches with
// a stale address.
int scratch_address(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return SVN_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return SVN_OK;
}

}  // namespace

extern "C" int svn_residual_noalloc(const svn_grid* grid, const svn_params* prm, double dt, const double* hcell,
                                    const double* A, const double* wind, const double* ocean, const double* v_old,
                                    const double* v, double* R, double* norm, void* cuda_stream) {
  if (!grid || !prm || !hcell || !A || !wind || !ocean || !v_old || !v || !R) return SVN_ERR_ARG;
  const int N = grid->N;
  if (N < 8 || N > kMaxN || (N & 1)) return SVN_ERR_ARG;
  if (!(grid->L > 0.0) || !(dt > 0.0) || !std::isfinite(dt)) return SVN_ERR_ARG;
  if (!(prm->e > 0.0) || !(prm->delta_min > 0.0)) return SVN_ERR_ARG;
  double* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != SVN_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const Layout g = make_layout(N, grid->L);
  const long long pl = g.plane;
  double* P = base;
  double* rhoH = P + pl;
  double* fq = rhoH + pl;
  double* voq = fq + 8 * pl;
  double2* vp = reinterpret_cast<double2*>(voq + 8 * pl);
  double2* Rp = vp + pl;
  double* eb = reinterpret_cast<double*>(Rp + pl);
  double* partial = eb + 8 * pl;
  double* scal = partial + (kTail - 64);
  if (residual_partials(g) > kTail - 64) return SVN_ERR_ARG;

  PhysConst pc;
  pc.rho_ice = prm->rho_ice; pc.rho_a = prm->rho_a; pc.rho_o = prm->rho_o; pc.Ca = prm->Ca; pc.Co = prm->Co;
  pc.f_c = prm->f_c; pc.Pstar = prm->Pstar; pc.C = prm->C; pc.e = prm->e; pc.delta_min = prm->delta_min;
  Phys ph;
  ph.dt = dt;
  ph.dx = g.dx;
  ph.idx = 1.0 / g.dx;
  ph.w = 0.25 * g.dx * g.dx;
  ph.ta = 0.5 * (1.0 + 1.0 / prm->e);
  ph.tb = 0.5 * (1.0 - 1.0 / prm->e);
  ph.tc = 0.5 / prm->e;
  ph.dmin2 = prm->delta_min * prm->delta_min;
  ph.cdrag = prm->Co * prm->rho_o;

  launch_precompute(s, g, dt, pc, hcell, A, wind, ocean, v_old, P, rhoH, fq, voq);
  launch_unpack_nodes(s, g, v, vp);
  launch_residual(s, g, ph, vp, P, rhoH, fq, voq, eb, Rp, partial);
  launch_sum_final(s, partial, residual_partials(g), scal);
  launch_pack_nodes(s, g, Rp, R);
  if (cudaGetLastError() != cudaSuccess) return SVN_ERR_CUDA;
  if (norm) {
    double sq = 0.0;
    if (cudaMemcpyAsync(&sq, scal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SVN_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SVN_ERR_CUDA;
    *norm = std::sqrt(sq);
    if (!std::isfinite(*norm)) return SVN_ERR_NONFINITE;
  }
  return SVN_OK;
}
