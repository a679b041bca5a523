// Explicit transport of ice concentration A and thickness H (Section 2,
// Eqs. "model:A" and "model:H"; Section 3: an explicit step for A and H with
// the velocity of the previous time level, before the implicit momentum
// step; Section 5.1: A and H are cell-wise constants).
//
// First-order upwind finite volumes on the N x N cells.  The normal velocity
// on a face is the mean of the normal components at its two end nodes (the
// face average of the bilinear velocity); node velocities on the domain
// boundary count as zero (v = 0 there), so boundary faces carry no flux.
// The explicit Euler step is split into n_sub = max(1, ceil(max_K c_K))
// equal sub-steps, c_K = dt/dx * (sum of the outflow normal velocities of
// cell K), which keeps every sub-step positivity preserving; A is capped at
// 1 after the last sub-step.
//
// Inputs use the C-ABI layouts: cells [j][i] with stride N, node velocity
// interleaved [j][i][k] with stride N+1.  The update is evaluated with
// round-to-nearest intrinsics in a fixed order (no contraction into FMA), so
// the result does not depend on the compiler's choices.
#include <cmath>

#include "kernels.h"

namespace svn {

namespace {

__device__ __forceinline__ double vel(const double* __restrict__ v, int N, int i, int j, int k) {
  if (i <= 0 || j <= 0 || i >= N || j >= N) return 0.0;
  return v[2 * ((long long)j * (N + 1) + i) + k];
}

// x-velocity on the vertical face at x_i between node rows j and j+1
__device__ __forceinline__ double face_ux(const double* __restrict__ v, int N, int i, int j) {
  return __dmul_rn(0.5, __dadd_rn(vel(v, N, i, j, 0), vel(v, N, i, j + 1, 0)));
}
// y-velocity on the horizontal face at y_j between node columns i and i+1
__device__ __forceinline__ double face_uy(const double* __restrict__ v, int N, int i, int j) {
  return __dmul_rn(0.5, __dadd_rn(vel(v, N, i, j, 1), vel(v, N, i + 1, j, 1)));
}

constexpr int kBX = 32, kBY = 8;

__global__ void __launch_bounds__(kBX * kBY) k_transport_courant(int N, double dt_dx, const double* __restrict__ v,
                                                                 double* __restrict__ partial) {
  double m = 0.0;
  const long long nc = (long long)N * N;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  for (long long c = (long long)blockIdx.x * (kBX * kBY) + tid; c < nc; c += (long long)gridDim.x * (kBX * kBY)) {
    const int j = (int)(c / N), i = (int)(c - (long long)j * N);
    const double ue = face_ux(v, N, i + 1, j), uw = face_ux(v, N, i, j);
    const double un = face_uy(v, N, i, j + 1), us = face_uy(v, N, i, j);
    const double out = __dadd_rn(__dadd_rn(__dadd_rn(fmax(ue, 0.0), fmax(-uw, 0.0)), fmax(un, 0.0)), fmax(-us, 0.0));
    double ck = __dmul_rn(dt_dx, out);
    if (!isfinite(ck)) ck = INFINITY;
    m = ck > m ? ck : m;
  }
  m = block_max(m);
  if (tid == 0) partial[blockIdx.x] = m;
}

// upwind flux in +x through the face at x_i (1 <= i <= N-1) of field Q
__device__ __forceinline__ double flux_x(const double* __restrict__ Q, int N, int i, int j, double u) {
  return u > 0.0 ? __dmul_rn(u, Q[(long long)j * N + i - 1]) : __dmul_rn(u, Q[(long long)j * N + i]);
}
__device__ __forceinline__ double flux_y(const double* __restrict__ Q, int N, int i, int j, double u) {
  return u > 0.0 ? __dmul_rn(u, Q[(long long)(j - 1) * N + i]) : __dmul_rn(u, Q[(long long)j * N + i]);
}

__device__ __forceinline__ double fv_update(const double* __restrict__ Q, int N, int i, int j, double k, double ue,
                                            double uw, double un, double us) {
  const double fe = (i + 1 < N) ? flux_x(Q, N, i + 1, j, ue) : 0.0;
  const double fw = (i > 0) ? flux_x(Q, N, i, j, uw) : 0.0;
  const double fn = (j + 1 < N) ? flux_y(Q, N, i, j + 1, un) : 0.0;
  const double fs = (j > 0) ? flux_y(Q, N, i, j, us) : 0.0;
  const double div = __dadd_rn(__dsub_rn(fe, fw), __dsub_rn(fn, fs));
  return __dsub_rn(Q[(long long)j * N + i], __dmul_rn(k, div));
}

// One Euler sub-step of length ds (k = ds/dx) for A and H; cap A at 1 if asked.
__global__ void __launch_bounds__(kBX * kBY) k_transport_step(int N, double k, int cap, const double* __restrict__ v,
                                                              const double* __restrict__ Hin,
                                                              const double* __restrict__ Ain,
                                                              double* __restrict__ Hout, double* __restrict__ Aout) {
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  if (i >= N || j >= N) return;
  const double ue = face_ux(v, N, i + 1, j), uw = face_ux(v, N, i, j);
  const double un = face_uy(v, N, i, j + 1), us = face_uy(v, N, i, j);
  const long long c = (long long)j * N + i;
  Hout[c] = fv_update(Hin, N, i, j, k, ue, uw, un, us);
  const double a = fv_update(Ain, N, i, j, k, ue, uw, un, us);
  Aout[c] = cap ? fmin(a, 1.0) : a;
}

}  // namespace

int transport_courant_blocks(int N) {
  const long long nc = (long long)N * N;
  const long long b = (nc + kBX * kBY - 1) / (kBX * kBY);
  return (int)std::min<long long>(std::max<long long>(b, 1), 608);   // 4 blocks per SM on 152 SMs
}

void launch_transport_courant(cudaStream_t s, int N, double dt_dx, const double* v, double* partial) {
  note_launch();
  k_transport_courant<<<transport_courant_blocks(N), dim3(kBX, kBY), 0, s>>>(N, dt_dx, v, partial);
}

void launch_transport_step(cudaStream_t s, int N, double k, bool cap, const double* v, const double* Hin,
                           const double* Ain, double* Hout, double* Aout) {
  note_launch();
  dim3 grid((N + kBX - 1) / kBX, (N + kBY - 1) / kBY);
  k_transport_step<<<grid, dim3(kBX, kBY), 0, s>>>(N, k, cap ? 1 : 0, v, Hin, Ain, Hout, Aout);
}

}  // namespace svn
