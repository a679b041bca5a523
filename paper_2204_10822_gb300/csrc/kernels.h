// Host-side launchers of the svN CUDA kernels (all stream-ordered).
#pragma once

#include "svn_internal.cuh"

namespace svn {

constexpr int MAX_ALPHA = 8;

// Process-wide count of kernel launches issued by this library.
void note_launch();
unsigned long long launches_issued();
struct AlphaSet {
  double a[MAX_ALPHA];
};

struct PhysConst {
  double rho_ice, rho_a, rho_o, Ca, Co, f_c, Pstar, C, e, delta_min;
};

// ---- cell kernels (fem_kernels.cu) ----
void launch_precompute(cudaStream_t s, const Layout& g, double dt, const PhysConst& pc, const double* hcell,
                       const double* A, const double* wind, const double* ocean, const double* vold, double* P,
                       double* rhoH, double* fq, double* voq);
void launch_pi_init(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, double* pi);
int residual_partials(const Layout& g);
void launch_residual(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, const double* P,
                     const double* rhoH, const double* fq, const double* voq, double* eb, double2* R,
                     double* partial);
int energy_partials(const Layout& g);
void launch_energy(cudaStream_t s, const Layout& g, const Phys& ph, int k, const AlphaSet& al, const double2* v,
                   const double2* dv, const double* P, const double* rhoH, const double* fq, const double* voq,
                   double* partial, double* out);
template <typename TE>
void launch_element_matrices(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, const double* pi,
                             const double* P, const double* rhoH, const double* voq, TE* ke);
template <typename TE, typename TS>
void launch_stencil_from_elements(cudaStream_t s, const Layout& g, const TE* ke, TS* st);
void launch_dual_update(cudaStream_t s, const Layout& g, const Phys& ph, double alpha, const double2* v,
                        const double2* dv, double* pi);
// Fused unit-step trial at v + dv: energy -> out_e[0] (scale in out_e[MAX_ALPHA]),
// residual -> R (norm^2 partials in partial_r, residual_partials(g) of them),
// trial dual state -> pi_t.
void launch_trial(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, const double2* dv,
                  const double* P, const double* rhoH, const double* fq, const double* voq, const double* pi,
                  double* pi_t, double* eb, double2* R, double* partial_e, double* out_e, double* partial_r);

// Final compensated reduction of per-block energy partials (layout of launch_energy).
void launch_energy_final(cudaStream_t s, int k, const double* partial, int nblocks, double* out);

// ---- Q2 velocity elements (q2_kernels.cu) ----
// N x N cells (cell c = j N + i), nodes of the (2N+1)^2 grid in the node layout gq
// (= make_layout(2N, L)); quadrature planes of cpl entries (9 points per cell).
struct Q2Geom {
  int N;
  long long cpl;
  Layout gq;
};
int q2_init_tables();   // basis tables into constant memory of the current device
void launch_q2_precompute(cudaStream_t s, const Q2Geom& q, double dt, const PhysConst& pc, const double* hcell,
                          const double* A, const double* wind, const double* ocean, const double* vold, double* P,
                          double* rhoH, double* fq, double* voq);
void launch_q2_pi_init(cudaStream_t s, const Q2Geom& q, const Phys& ph, const double2* v, double* pi);
int q2_node_partials(const Q2Geom& q);
void launch_q2_residual(cudaStream_t s, const Q2Geom& q, const Phys& ph, const double2* v, const double* P,
                        const double* rhoH, const double* fq, const double* voq, double* eb, double2* R,
                        double* partial);
int q2_energy_partials(const Q2Geom& q);
void launch_q2_energy(cudaStream_t s, const Q2Geom& q, const Phys& ph, int k, const AlphaSet& al, const double2* v,
                      const double2* dv, const double* P, const double* rhoH, const double* fq, const double* voq,
                      double* partial, double* out);
void launch_q2_element_matrices(cudaStream_t s, const Q2Geom& q, const Phys& ph, const double2* v, const double* pi,
                                const double* P, const double* rhoH, const double* voq, double* ke);
void launch_q2_apply(cudaStream_t s, const Q2Geom& q, const double* ke, const double2* x, double* eb, double2* y);
void launch_q2_dual_update(cudaStream_t s, const Q2Geom& q, const Phys& ph, double alpha, const double2* v,
                           const double2* dv, double* pi);
void launch_q2_refine_cells(cudaStream_t s, int N, const double* src, double* dst);   // N^2 -> (2N)^2 cells
void launch_q2_pi_layout(cudaStream_t s, const Q2Geom& q, const double* src, double* dst, bool to_planes);
// Q2 block-Jacobi inverse (3 planes of gq.plane) from the element matrices
void launch_q2_dinv(cudaStream_t s, const Q2Geom& q, const double* ke, double* dinv);
// Chebyshev step k on the Q2 operator: d = c1 d + c2 D^-1 (b - Ax), x += d
void launch_q2_cheb_step(cudaStream_t s, const Q2Geom& q, const double* dinv, const double* coef, int k,
                         const double2* b, const double2* Ax, double2* x, double2* d);
void launch_q2_dinv_apply(cudaStream_t s, const Q2Geom& q, const double* dinv, const double2* x, double2* y);
void launch_q2_checker(cudaStream_t s, const Q2Geom& q, double2* x);   // power-iteration start vector
// pi of the Q1 operator on the 2N grid (12 planes of gq.plane) from the Q2 pi
void launch_q2_pi_to_q1(cudaStream_t s, const Q2Geom& q, const double* pi2, double* pi1);

// ---- transport of A and H (transport.cu) ----
int transport_courant_blocks(int N);
// per-block maxima of the outflow Courant number (dt_dx * outflow) into partial
void launch_transport_courant(cudaStream_t s, int N, double dt_dx, const double* v, double* partial);
// one explicit upwind sub-step, k = ds/dx; A capped at 1 when cap is set
void launch_transport_step(cudaStream_t s, int N, double k, bool cap, const double* v, const double* Hin,
                           const double* Ain, double* Hout, double* Aout);

// ---- stencil / multigrid kernels (mg_kernels.cu) ----
// y = A x on interior nodes (0 elsewhere); TA accumulates.
template <typename TS, typename TX, typename TY, typename TA>
void launch_apply(cudaStream_t s, const Layout& g, const TS* st, const TX* x, TY* y);
// r = b - A x
template <typename TS, typename TV>
void launch_residual_stencil(cudaStream_t s, const Layout& g, const TS* st, const TV* x, const TV* b, TV* r);
// Block-Jacobi inverse (3 planes: xx, xy, yy) and per-block Gershgorin maxima.
template <typename TS, typename TD>
int launch_dinv_gershgorin(cudaStream_t s, const Layout& g, const TS* st, TD* dinv, double* partial, bool bound);
void launch_max_final(cudaStream_t s, const double* partial, int n, double* out);
// lambda_max(D^-1 A) ~= safety |x_k| / |x_{k-1}| after k power steps from the
// checkerboard vector (x0, x1: level vectors used as scratch); stream as for
// launch_cheb_sweep2 (two steps per row-streaming pass where it applies).
template <typename TS, typename TD, typename TV>
void launch_power_lmax(cudaStream_t s, const Layout& g, const TS* st, const TD* dinv, int iters, double safety,
                       TV* x0, TV* x1, double* partial, double* lmax, int stream, unsigned polls = 0);
// Chebyshev smoothing (Saad Alg. 12.1 on D^-1 A over [lo lmax, lmax]); the
// step coefficients are computed on the device from lmax (launch_cheb_coefs).
template <typename T>
void launch_cheb_coefs(cudaStream_t s, const double* lmax, double lo, int deg, T* coef);
template <typename TS, typename TD, typename TV>
void launch_cheb_zero_start(cudaStream_t s, const Layout& g, const TD* dinv,
                            const typename ScalarOf<TV>::type* coef, const TV* b, TV* x, TV* d);
template <typename TS, typename TD, typename TV>
void launch_cheb_sweep(cudaStream_t s, const Layout& g, const TS* st, const TD* dinv,
                       const typename ScalarOf<TV>::type* coef, int step, const TV* xin, TV* xout, TV* d,
                       const TV* b);
// Steps (step, step + 1) fused; x0 != x2 and d0 != d2.  stream: 1 = the
// row-streaming kernel on FP32 levels with N >= 1024, the shared-memory tile
// kernel elsewhere; 2 = row-streaming on every FP32 level; 0 = tile kernel.
// 3 = the TMA-staged kernel (sweep_tma.cu) on every level with an FP32 stencil,
// 4 = the TMA-staged kernel on FP32-stencil levels with N >= 1024 (tile kernel
// below); polls bounds each of its mbarrier waits (0: default).
template <typename TS, typename TD, typename TV>
void launch_cheb_sweep2(cudaStream_t s, const Layout& g, const TS* st, const TD* dinv,
                        const typename ScalarOf<TV>::type* coef, int step, const TV* x0, TV* x2, const TV* d0,
                        TV* d2, const TV* b, int stream, unsigned polls = 0);
// TMA-staged two-step sweep on an FP32 level (power: x2 = (D^-1 A)^2 x0);
// false when it cannot run (no tensor-map entry point), nothing launched then.
bool launch_cheb_sweep2_tma(cudaStream_t s, const Layout& g, const float* st, const float* dinv, const float* coef,
                            int step, const float2* x0, float2* x2, const float2* d0, float2* d2, const float2* b,
                            bool power, unsigned polls);
// Number of TMA-sweep CTAs whose bounded wait gave up since the last reset
// (device-wide counter; -1 on a CUDA error).  pinned: one host-pinned unsigned.
int sweep_tma_timeouts(cudaStream_t s, unsigned* pinned, bool reset);
// Whether launch_cheb_sweep2 takes the row-streaming kernel on level g for
// FP32 vectors; only that kernel accepts x0 = d0 = NULL (start from zero).
bool sweep2_streams(const Layout& g, int stream);
template <typename TV>
void launch_restrict(cudaStream_t s, const Layout& gf, const Layout& gc, const TV* rf, TV* bc);
template <typename TV>
void launch_prolong_add(cudaStream_t s, const Layout& gf, const Layout& gc, const TV* xc, TV* xf);
template <typename TF, typename TC>
void launch_rap(cudaStream_t s, const Layout& gf, const Layout& gc, const TF* stf, TC* stc);
template <typename TS>
void launch_coarse_dense(cudaStream_t s, const Layout& g, const TS* st, double* dense);
void launch_cholesky_inverse(cudaStream_t s, int n, double* a, double* inv, int* info);
template <typename TV>
void launch_coarse_solve(cudaStream_t s, const Layout& g, int n, const double* inv, const TV* b, TV* x);
template <typename TA, typename TB>
void launch_convert_stencil(cudaStream_t s, const Layout& g, const TA* a, TB* b);

// ---- vector / Krylov kernels (krylov_kernels.cu) ----
int reduce_blocks(long long n);
void launch_sum_final(cudaStream_t s, const double* partial, int n, double* out);
// node vectors are double2 / float2 arrays of g.plane entries
void launch_unpack_nodes(cudaStream_t s, const Layout& g, const double* src, double2* dst);
void launch_pack_nodes(cudaStream_t s, const Layout& g, const double2* src, double* dst);
void launch_unpack_pi(cudaStream_t s, const Layout& g, const double* src, double* pi);
void launch_pack_pi(cudaStream_t s, const Layout& g, const double* pi, double* dst);
void launch_norm2_partial(cudaStream_t s, const Layout& g, const double2* x, double* partial);
void launch_scale_copy(cudaStream_t s, const Layout& g, const double2* x, const double* num, const double* den,
                       double2* y);   // y = x * (*num / *den)
void launch_axpy(cudaStream_t s, const Layout& g, double a, const double2* x, double2* y);   // y += a x
void launch_axpby_to(cudaStream_t s, const Layout& g, const double2* x, double a, const double2* d,
                     double2* y);   // y = x + a d
void launch_scale_to(cudaStream_t s, const Layout& g, double a, const double2* x, double2* y);   // y = a x
void launch_validate(cudaStream_t s, long long ncell, long long nvec, const double* h, const double* A,
                     const double* wind, const double* ocean, const double* vold, int* counts);
void launch_neg_copy(cudaStream_t s, const Layout& g, const double2* x, double2* y);
void launch_cast_d2f(cudaStream_t s, const Layout& g, const double2* x, float2* y);
void launch_cast_f2d(cudaStream_t s, const Layout& g, const float2* x, double2* y);
// Arnoldi: h[i] (i < m) partial dots of V_i with w; V_i at V + i * vstride.
void launch_multidot(cudaStream_t s, const Layout& g, const double2* V, long long vstride, int m, const double2* w,
                     double* partial, int nblk);
void launch_multidot_final(cudaStream_t s, const double* partial, int nblk, int m, double* h, int accumulate);
// w -= sum_i h[i] V_i; norm partials of w
void launch_update_norm(cudaStream_t s, const Layout& g, const double2* V, long long vstride, int m, const double* h,
                        double2* w, double* partial, int nblk);
// x += sum_j y[j] Z_j (Z in TZ precision)
template <typename TZ>
void launch_lincomb(cudaStream_t s, const Layout& g, const TZ* Z, long long zstride, int m, const double* y,
                    double2* x);
int krylov_blocks(const Layout& g);

// ---- learned initial guess (unet.cu) ----
struct NetImpl;
// Predict the node velocity of the handle's grid from the forcing (caller layouts).
void net_predict_nodes(NetImpl* n, cudaStream_t s, const Layout& g, const double* hcell, const double* A,
                       const double* wind, const double* ocean, const double* vold, double2* v);
int net_grid(const NetImpl* n);

}  // namespace svn
