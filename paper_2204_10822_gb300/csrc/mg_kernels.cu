// Stencil-form operator kernels: Jacobian apply, block-Jacobi Chebyshev
// smoothing, bilinear restriction / prolongation, Galerkin coarse operators
// and the dense coarsest-level solve (Section 5.4: FGMRES + multigrid with
// three smoothing steps and a direct solve on the coarsest level).
//
// Templates: TS = stencil storage (double, float, __nv_bfloat16), TD = block-
// Jacobi storage, TV = vector type (double2 / float2); arithmetic in the
// vector's scalar type.
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace svn {


template <typename TA, typename TS>
__device__ __forceinline__ TA ldc(const TS* p) {
  return (TA)to_d(*p);
}
template <>
__device__ __forceinline__ float ldc<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ float ldc<float, float>(const float* p) {
  return *p;
}
template <>
__device__ __forceinline__ double ldc<double, double>(const double* p) {
  return *p;
}

template <typename V, typename T> __device__ __forceinline__ V mk2(T a, T b);
template <> __device__ __forceinline__ double2 mk2<double2, double>(double a, double b) { return make_double2(a, b); }
template <> __device__ __forceinline__ float2 mk2<float2, float>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ float2 mk2<float2, double>(double a, double b) { return make_float2((float)a, (float)b); }
template <> __device__ __forceinline__ double2 mk2<double2, float>(float a, float b) { return make_double2(a, b); }

__device__ __forceinline__ bool is_interior(int i, int j, int N) { return i >= 1 && j >= 1 && i <= N - 1 && j <= N - 1; }

// y += a xa + b xb.  FP64 stencil rows are bound by the FP64 pipe, so they
// take two dependent FMAs (2 issues); FP32 rows are bound by memory latency,
// so they keep the pair product independent of y (MUL + FMA, then one ADD),
// which shortens the chain through the accumulator.
template <typename TA>
__device__ __forceinline__ void acc2(TA& y, TA a, TA xa, TA b, TA xb) {
  if constexpr (std::is_same<TA, double>::value) {
    y = fma(a, xa, y);
    y = fma(b, xb, y);
  } else {
    y += a * xa + b * xb;
  }
}

// y_p = sum_q K[p][q] x_q over the 9-point block stencil at node n.
template <typename TA, typename TS, typename TX>
__device__ __forceinline__ void stencil_row(const TS* __restrict__ st, long long pl, long long n, int ld,
                                            const TX* __restrict__ x, TA& yx, TA& yy) {
  const TA dxx = ldc<TA>(st + (S_D + 0) * pl + n);
  const TA dxy = ldc<TA>(st + (S_D + 1) * pl + n);
  const TA dyy = ldc<TA>(st + (S_D + 2) * pl + n);
  const TX xp = x[n];
  yx = dxx * (TA)xp.x + dxy * (TA)xp.y;
  yy = dxy * (TA)xp.x + dyy * (TA)xp.y;
  auto fwd = [&](int slot, long long q) {
    const TX xq = x[q];
    const TA b0 = ldc<TA>(st + (slot + 0) * pl + n), b1 = ldc<TA>(st + (slot + 1) * pl + n);
    const TA b2 = ldc<TA>(st + (slot + 2) * pl + n), b3 = ldc<TA>(st + (slot + 3) * pl + n);
    acc2<TA>(yx, b0, (TA)xq.x, b1, (TA)xq.y);
    acc2<TA>(yy, b2, (TA)xq.x, b3, (TA)xq.y);
  };
  auto bwd = [&](int slot, long long q) {   // block stored at q, used transposed
    const TX xq = x[q];
    const TA b0 = ldc<TA>(st + (slot + 0) * pl + q), b1 = ldc<TA>(st + (slot + 1) * pl + q);
    const TA b2 = ldc<TA>(st + (slot + 2) * pl + q), b3 = ldc<TA>(st + (slot + 3) * pl + q);
    acc2<TA>(yx, b0, (TA)xq.x, b2, (TA)xq.y);
    acc2<TA>(yy, b1, (TA)xq.x, b3, (TA)xq.y);
  };
  fwd(S_E, n + 1);
  fwd(S_N, n + ld);
  fwd(S_NE, n + ld + 1);
  fwd(S_NW, n + ld - 1);
  bwd(S_E, n - 1);
  bwd(S_N, n - ld);
  bwd(S_NE, n - ld - 1);
  bwd(S_NW, n - ld + 1);
}

// The same row product with x taken from an accessor xf(di, dj) (e.g. shared memory).
template <typename TA, typename TS, typename XF>
__device__ __forceinline__ void stencil_row_f(const TS* __restrict__ st, long long pl, long long n, int ld, XF xf,
                                              TA& yx, TA& yy) {
  const TA dxx = ldc<TA>(st + (S_D + 0) * pl + n);
  const TA dxy = ldc<TA>(st + (S_D + 1) * pl + n);
  const TA dyy = ldc<TA>(st + (S_D + 2) * pl + n);
  const auto xp = xf(0, 0);
  yx = dxx * (TA)xp.x + dxy * (TA)xp.y;
  yy = dxy * (TA)xp.x + dyy * (TA)xp.y;
  auto fwd = [&](int slot, int di, int dj) {
    const auto xq = xf(di, dj);
    const TA b0 = ldc<TA>(st + (slot + 0) * pl + n), b1 = ldc<TA>(st + (slot + 1) * pl + n);
    const TA b2 = ldc<TA>(st + (slot + 2) * pl + n), b3 = ldc<TA>(st + (slot + 3) * pl + n);
    acc2<TA>(yx, b0, (TA)xq.x, b1, (TA)xq.y);
    acc2<TA>(yy, b2, (TA)xq.x, b3, (TA)xq.y);
  };
  auto bwd = [&](int slot, int di, int dj) {
    const auto xq = xf(di, dj);
    const long long q = n + (long long)dj * ld + di;
    const TA b0 = ldc<TA>(st + (slot + 0) * pl + q), b1 = ldc<TA>(st + (slot + 1) * pl + q);
    const TA b2 = ldc<TA>(st + (slot + 2) * pl + q), b3 = ldc<TA>(st + (slot + 3) * pl + q);
    acc2<TA>(yx, b0, (TA)xq.x, b2, (TA)xq.y);
    acc2<TA>(yy, b1, (TA)xq.x, b3, (TA)xq.y);
  };
  fwd(S_E, 1, 0);
  fwd(S_N, 0, 1);
  fwd(S_NE, 1, 1);
  fwd(S_NW, -1, 1);
  bwd(S_E, -1, 0);
  bwd(S_N, 0, -1);
  bwd(S_NE, -1, -1);
  bwd(S_NW, 1, -1);
}

// Block K[p][p + (di, dj)], |di|, |dj| <= 1, as b[k][l] (row-major).
template <typename TA, typename TS>
__device__ __forceinline__ void get_block(const TS* __restrict__ st, long long pl, long long n, int ld, int di, int dj,
                                          TA b[4]) {
  if (di == 0 && dj == 0) {
    b[0] = ldc<TA>(st + (S_D + 0) * pl + n);
    b[1] = b[2] = ldc<TA>(st + (S_D + 1) * pl + n);
    b[3] = ldc<TA>(st + (S_D + 2) * pl + n);
    return;
  }
  int slot;
  bool tr;
  long long q;
  if (dj == 0) {
    slot = S_E; tr = di < 0; q = tr ? n - 1 : n;
  } else if (di == 0) {
    slot = S_N; tr = dj < 0; q = tr ? n - ld : n;
  } else if (di == dj) {
    slot = S_NE; tr = di < 0; q = tr ? n - ld - 1 : n;
  } else {
    slot = S_NW; tr = dj < 0; q = tr ? n - ld + 1 : n;
  }
  const TA c0 = ldc<TA>(st + (slot + 0) * pl + q), c1 = ldc<TA>(st + (slot + 1) * pl + q);
  const TA c2 = ldc<TA>(st + (slot + 2) * pl + q), c3 = ldc<TA>(st + (slot + 3) * pl + q);
  if (!tr) {
    b[0] = c0; b[1] = c1; b[2] = c2; b[3] = c3;
  } else {
    b[0] = c0; b[1] = c2; b[2] = c1; b[3] = c3;
  }
}

namespace {

template <typename TS, typename TX, typename TY, typename TA>
__global__ void k_apply(Layout g, const TS* __restrict__ st, const TX* __restrict__ x, TY* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  const long long n = (long long)j * g.ld + i;
  TA yx = 0, yy = 0;
  if (is_interior(i, j, g.N)) stencil_row<TA>(st, g.plane, n, g.ld, x, yx, yy);
  y[n] = mk2<TY>(yx, yy);
}

template <typename TS, typename TV>
__global__ void k_residual_stencil(Layout g, const TS* __restrict__ st, const TV* __restrict__ x,
                                   const TV* __restrict__ b, TV* __restrict__ r) {
  using T = typename ScalarOf<TV>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  const long long n = (long long)j * g.ld + i;
  T yx = 0, yy = 0;
  TV out = mk2<TV>(T(0), T(0));
  if (is_interior(i, j, g.N)) {
    stencil_row<T>(st, g.plane, n, g.ld, x, yx, yy);
    const TV bb = b[n];
    out = mk2<TV>(bb.x - yx, bb.y - yy);
  }
  r[n] = out;
}

template <typename TS, typename TD>
__global__ void k_dinv_gershgorin(Layout g, const TS* __restrict__ st, TD* __restrict__ dinv,
                                  double* __restrict__ partial, int bound) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double gmax = 0.0;
  if (i <= g.N && j <= g.N) {
    const long long n = (long long)j * g.ld + i;
    double i00 = 0, i01 = 0, i11 = 0;
    if (is_interior(i, j, g.N)) {
      double d[4];
      get_block<double>(st, g.plane, n, g.ld, 0, 0, d);
      const double det = d[0] * d[3] - d[1] * d[1];
      i00 = d[3] / det;
      i01 = -d[1] / det;
      i11 = d[0] / det;
      double r0 = 0, r1 = 0;
      for (int dj = -1; dj <= 1 && bound; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (!is_interior(i + di, j + dj, g.N)) continue;
          double b[4];
          get_block<double>(st, g.plane, n, g.ld, di, dj, b);
          // rows of D^-1 B
          r0 += fabs(i00 * b[0] + i01 * b[2]) + fabs(i00 * b[1] + i01 * b[3]);
          r1 += fabs(i01 * b[0] + i11 * b[2]) + fabs(i01 * b[1] + i11 * b[3]);
        }
      gmax = fmax(r0, r1);
    }
    dinv[0 * g.plane + n] = (TD)i00;
    dinv[1 * g.plane + n] = (TD)i01;
    dinv[2 * g.plane + n] = (TD)i11;
  }
  gmax = block_max(gmax);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = gmax;
}

// Start vector of the power method: ((-1)^(i+j), -(-1)^(i+j)) on interior nodes.
template <typename TV>
__global__ void k_checkerboard(Layout g, TV* __restrict__ x) {
  using T = typename ScalarOf<TV>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  const T sgn = ((i + j) & 1) ? T(-1) : T(1);
  x[(long long)j * g.ld + i] = is_interior(i, j, g.N) ? mk2<TV>(sgn, -sgn) : mk2<TV>(T(0), T(0));
}

// y = D^-1 (A x) on interior nodes (one power-method step).
template <typename TS, typename TD, typename TV>
__global__ void k_power_step(Layout g, const TS* __restrict__ st, const TD* __restrict__ dinv,
                             const TV* __restrict__ x, TV* __restrict__ y) {
  using T = typename ScalarOf<TV>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  const long long n = (long long)j * g.ld + i;
  TV out = mk2<TV>(T(0), T(0));
  if (is_interior(i, j, g.N)) {
    T ax, ay;
    stencil_row<T>(st, g.plane, n, g.ld, x, ax, ay);
    const T i00 = ldc<T>(dinv + n), i01 = ldc<T>(dinv + g.plane + n), i11 = ldc<T>(dinv + 2 * g.plane + n);
    out = mk2<TV>(i00 * ax + i01 * ay, i01 * ax + i11 * ay);
  }
  y[n] = out;
}

template <typename TV>
__global__ void k_norm2_vec(long long n, const TV* __restrict__ x, double* __restrict__ partial) {
  double s = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const TV v = x[t];
    s += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// lmax = safety * sqrt(sum(p_last) / sum(p_prev)) over nb block partials each.
__global__ void k_lmax_from_norms(const double* __restrict__ p_last, const double* __restrict__ p_prev, int nb,
                                  double safety, double* __restrict__ lmax) {
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    a += p_last[t];
    b += p_prev[t];
  }
  a = block_sum(a);
  b = block_sum(b);
  if (threadIdx.x == 0) *lmax = safety * sqrt(a / b);
}

__global__ void k_max_final(const double* __restrict__ partial, int n, double* __restrict__ out) {
  double m = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) m = fmax(m, partial[b]);
  m = block_max(m);
  if (threadIdx.x == 0) *out = m;
}

struct ChebCoef {
  double theta, delta, sigma;
};
__device__ __forceinline__ ChebCoef cheb_coef(double lmax, double lo) {
  ChebCoef c;
  const double a = lo * lmax, b = lmax;
  c.theta = 0.5 * (b + a);
  c.delta = 0.5 * (b - a);
  c.sigma = c.theta / c.delta;
  return c;
}

// Chebyshev step coefficients, once per level after lmax is known:
// coef[2k] = c1_k, coef[2k+1] = c2_k with d_k = c1_k d_{k-1} + c2_k D^-1 r_k
// (Saad Alg. 12.1: c1_0 = 0, c2_0 = 1/theta; rho_0 = 1/sigma,
//  rho_k = 1/(2 sigma - rho_{k-1}), c1_k = rho_k rho_{k-1}, c2_k = 2 rho_k / delta).
template <typename T>
__global__ void k_cheb_coefs(const double* __restrict__ lmax, double lo, int deg, T* __restrict__ coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const ChebCoef c = cheb_coef(*lmax, lo);
  double rho = 1.0 / c.sigma;
  coef[0] = (T)0;
  coef[1] = (T)(1.0 / c.theta);
  for (int k = 1; k < deg; ++k) {
    const double rn = 1.0 / (2.0 * c.sigma - rho);
    coef[2 * k] = (T)(rn * rho);
    coef[2 * k + 1] = (T)(2.0 * rn / c.delta);
    rho = rn;
  }
}

template <typename TD, typename TV>
__global__ void k_cheb_zero_start(Layout g, const TD* __restrict__ dinv,
                                  const typename ScalarOf<TV>::type* __restrict__ coef,
                                  const TV* __restrict__ b, TV* __restrict__ x, TV* __restrict__ d) {
  using T = typename ScalarOf<TV>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  const long long n = (long long)j * g.ld + i;
  const T it = coef[1];
  const TV bb = b[n];
  const T i00 = ldc<T>(dinv + n), i01 = ldc<T>(dinv + g.plane + n), i11 = ldc<T>(dinv + 2 * g.plane + n);
  const TV dd = mk2<TV>(it * (i00 * bb.x + i01 * bb.y), it * (i01 * bb.x + i11 * bb.y));
  d[n] = dd;
  x[n] = dd;
}

template <typename TS, typename TD, typename TV>
__global__ void k_cheb_sweep(Layout g, const TS* __restrict__ st, const TD* __restrict__ dinv,
                             const typename ScalarOf<TV>::type* __restrict__ coef, int step,
                             const TV* __restrict__ xin, TV* __restrict__ xout, TV* __restrict__ d,
                             const TV* __restrict__ b) {
  using T = typename ScalarOf<TV>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  const long long n = (long long)j * g.ld + i;
  if (!is_interior(i, j, g.N)) {
    xout[n] = mk2<TV>(T(0), T(0));
    return;
  }
  const T c1 = coef[2 * step], c2 = coef[2 * step + 1];
  T yx, yy;
  stencil_row<T>(st, g.plane, n, g.ld, xin, yx, yy);
  const TV bb = b[n];
  const T rx = bb.x - yx, ry = bb.y - yy;
  const T i00 = ldc<T>(dinv + n), i01 = ldc<T>(dinv + g.plane + n), i11 = ldc<T>(dinv + 2 * g.plane + n);
  const TV dold = d[n];
  const T dx = c1 * dold.x + c2 * (i00 * rx + i01 * ry);
  const T dy = c1 * dold.y + c2 * (i01 * rx + i11 * ry);
  d[n] = mk2<TV>(dx, dy);
  const TV xo = xin[n];
  xout[n] = mk2<TV>(xo.x + dx, xo.y + dy);
}

// Two consecutive Chebyshev steps (step, step + 1) in one pass.  A 32 x 8 tile
// keeps x0 on the tile plus a two-node ring, and the intermediate iterate x1
// and direction d1 on the tile plus a one-node ring, in shared memory; the
// stencil, D^-1, b and d0 are read once per pair of steps.  d0 -> d2 and
// x0 -> x2 must be distinct buffers (neighbouring tiles read d0 and x0).
template <typename TS, typename TD, typename TV>
__global__ void __launch_bounds__(256) k_cheb_sweep2(Layout g, const TS* __restrict__ st, const TD* __restrict__ dinv,
                                                     const typename ScalarOf<TV>::type* __restrict__ coef, int step,
                                                     const TV* __restrict__ x0, TV* __restrict__ x2,
                                                     const TV* __restrict__ d0, TV* __restrict__ d2,
                                                     const TV* __restrict__ b) {
  using T = typename ScalarOf<TV>::type;
  constexpr int TX = 32, TY = 8;
  __shared__ TV sx0[TY + 4][TX + 4];
  __shared__ TV sx1[TY + 2][TX + 2];
  __shared__ TV sd1[TY + 2][TX + 2];
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const TV zero = mk2<TV>(T(0), T(0));
  for (int e = tid; e < (TY + 4) * (TX + 4); e += TX * TY) {
    const int ly = e / (TX + 4), lx = e - ly * (TX + 4);
    const int i = i0 - 2 + lx, j = j0 - 2 + ly;
    sx0[ly][lx] = (i >= 0 && j >= 0 && i <= g.N && j <= g.N) ? x0[(long long)j * g.ld + i] : zero;
  }
  __syncthreads();
  const T c1a = coef[2 * step], c2a = coef[2 * step + 1];
  const T c1b = coef[2 * step + 2], c2b = coef[2 * step + 3];
  for (int e = tid; e < (TY + 2) * (TX + 2); e += TX * TY) {
    const int ly = e / (TX + 2), lx = e - ly * (TX + 2);
    const int i = i0 - 1 + lx, j = j0 - 1 + ly;
    TV x1 = zero, dd = zero;
    if (is_interior(i, j, g.N)) {
      const long long n = (long long)j * g.ld + i;
      T ax, ay;
      stencil_row_f<T>(st, g.plane, n, g.ld, [&](int di, int dj) { return sx0[ly + 1 + dj][lx + 1 + di]; }, ax, ay);
      const TV bb = b[n];
      const T rx = bb.x - ax, ry = bb.y - ay;
      const T i00 = ldc<T>(dinv + n), i01 = ldc<T>(dinv + g.plane + n), i11 = ldc<T>(dinv + 2 * g.plane + n);
      const TV dold = d0[n];
      const T dx = c1a * dold.x + c2a * (i00 * rx + i01 * ry);
      const T dy = c1a * dold.y + c2a * (i01 * rx + i11 * ry);
      const TV xo = sx0[ly + 1][lx + 1];
      dd = mk2<TV>(dx, dy);
      x1 = mk2<TV>(xo.x + dx, xo.y + dy);
    }
    sx1[ly][lx] = x1;
    sd1[ly][lx] = dd;
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = i0 + tx, j = j0 + ty;
  if (i > g.N || j > g.N) return;
  const long long n = (long long)j * g.ld + i;
  if (!is_interior(i, j, g.N)) {
    x2[n] = zero;
    return;
  }
  T ax, ay;
  stencil_row_f<T>(st, g.plane, n, g.ld, [&](int di, int dj) { return sx1[ty + 1 + dj][tx + 1 + di]; }, ax, ay);
  const TV bb = b[n];
  const T rx = bb.x - ax, ry = bb.y - ay;
  const T i00 = ldc<T>(dinv + n), i01 = ldc<T>(dinv + g.plane + n), i11 = ldc<T>(dinv + 2 * g.plane + n);
  const TV d1 = sd1[ty + 1][tx + 1];
  const T dx = c1b * d1.x + c2b * (i00 * rx + i01 * ry);
  const T dy = c1b * d1.y + c2b * (i01 * rx + i11 * ry);
  d2[n] = mk2<TV>(dx, dy);
  const TV x1 = sx1[ty + 1][tx + 1];
  x2[n] = mk2<TV>(x1.x + dx, x1.y + dy);
}

// ---- row-streaming two-step Chebyshev sweep ----------------------------------
// The same two Chebyshev steps as k_cheb_sweep2, organised for fewer loads: one
// warp walks up a strip of 32 node columns (kStreamCols output columns and two
// halo columns on each side) over a chunk of rows.  Per row a lane loads its
// node's 19 stencil values, block-Jacobi inverse, b and d0 once.  The
// transposed blocks that couple a node to its W, SW, S and SE neighbours are
// not loaded again: the W block comes from the neighbouring lane by a warp
// shuffle, and the S, SW and SE couplings are added to a partial sum for the
// row above while the row below is processed ("pushed").  Step 1 runs one row
// ahead of step 2; the next row's data is loaded while the current row is
// computed.  No shared memory and no barrier.
constexpr int kStreamCols = 28;

template <typename T>
__device__ __forceinline__ T shup(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shdn(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <>
__device__ __forceinline__ float2 shup<float2>(float2 v) { return make_float2(shup(v.x), shup(v.y)); }
template <>
__device__ __forceinline__ float2 shdn<float2>(float2 v) { return make_float2(shdn(v.x), shdn(v.y)); }

template <typename T, typename TV>
struct StreamRow {
  T S[NSTEN];
  T inv[3];
  TV b, d0;
};

template <typename TS, typename TD, typename TV, bool kPower>
__global__ void __launch_bounds__(128) k_cheb_sweep2s(Layout g, const TS* __restrict__ st,
                                                      const TD* __restrict__ dinv,
                                                      const typename ScalarOf<TV>::type* __restrict__ coef, int step,
                                                      const TV* __restrict__ x0, TV* __restrict__ x2,
                                                      const TV* __restrict__ d0, TV* __restrict__ d2,
                                                      const TV* __restrict__ b, int rows) {
  using T = typename ScalarOf<TV>::type;
  using Row = StreamRow<T, TV>;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nstrips = (g.n1 + kStreamCols - 1) / kStreamCols;
  const int strip = warp % nstrips, chunk = warp / nstrips;
  const int j_lo = chunk * rows;
  if (j_lo > g.N) return;   // the whole warp
  const int j_hi = min(j_lo + rows, g.N + 1);
  const int i = strip * kStreamCols + lane - 2;
  const bool col_ok = i >= 0 && i <= g.N;
  const bool out_lane = col_ok && lane >= 2 && lane < 30;
  const long long pl = g.plane;
  const T c1a = kPower ? T(0) : coef[2 * step], c2a = kPower ? T(0) : coef[2 * step + 1];
  const T c1b = kPower ? T(0) : coef[2 * step + 2], c2b = kPower ? T(0) : coef[2 * step + 3];
  const TV zero = mk2<TV>(T(0), T(0));

  auto load_row = [&](int q, Row& r) {
    const bool ok = col_ok && q >= 0 && q <= g.N;
    const long long n = ok ? (long long)q * g.ld + i : 0;
#pragma unroll
    for (int k = 0; k < NSTEN; ++k) r.S[k] = ok ? ldc<T>(st + k * pl + n) : T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.inv[k] = ok ? ldc<T>(dinv + k * pl + n) : T(0);
    r.b = (ok && !kPower) ? b[n] : zero;
    r.d0 = (ok && !kPower && d0) ? d0[n] : zero;
  };
  auto load_x0 = [&](int q) {
    return (x0 && col_ok && q >= 0 && q <= g.N) ? x0[(long long)q * g.ld + i] : zero;
  };

  // carried between rows
  TV x1p = zero, d1p = zero, x1pW = zero, x1pE = zero, x0W = zero, x0E = zero;
  T eWp[4] = {T(0), T(0), T(0), T(0)};
  T a1x = 0, a1y = 0;                          // row q: couplings to row q-1 (x0)
  T a2px = 0, a2py = 0, a2cx = 0, a2cy = 0;    // rows q-1, q: couplings to the row below (x1)

  // One row: P = row q-1, C = row q (loaded), N = row q+1 (loaded here);
  // xc, xn = x0 at rows q, q+1; xnn = x0 at row q+2 (loaded here).
  auto body = [&](int q, Row& P, Row& C, Row& N, TV& xc, TV& xn, TV& xnn) {
    load_row(q + 1, N);
    xnn = load_x0(q + 2);

    const TV x0nW = shup(xn), x0nE = shdn(xn);
    T eW[4], neW[4], nwE[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      eW[k] = shup(C.S[S_E + k]);
      neW[k] = shup(C.S[S_NE + k]);
      nwE[k] = shdn(C.S[S_NW + k]);
    }

    // step 1 at row q
    TV x1c = zero, d1c = zero;
    if (q >= j_lo - 1 && is_interior(i, q, g.N)) {
      const T* S = C.S;
      T yx = a1x, yy = a1y;
      yx = fma(S[S_D], (T)xc.x, yx);
      yx = fma(S[S_D + 1], (T)xc.y, yx);
      yy = fma(S[S_D + 1], (T)xc.x, yy);
      yy = fma(S[S_D + 2], (T)xc.y, yy);
      yx = fma(S[S_E], (T)x0E.x, yx);
      yx = fma(S[S_E + 1], (T)x0E.y, yx);
      yy = fma(S[S_E + 2], (T)x0E.x, yy);
      yy = fma(S[S_E + 3], (T)x0E.y, yy);
      yx = fma(S[S_N], (T)xn.x, yx);
      yx = fma(S[S_N + 1], (T)xn.y, yx);
      yy = fma(S[S_N + 2], (T)xn.x, yy);
      yy = fma(S[S_N + 3], (T)xn.y, yy);
      yx = fma(S[S_NE], (T)x0nE.x, yx);
      yx = fma(S[S_NE + 1], (T)x0nE.y, yx);
      yy = fma(S[S_NE + 2], (T)x0nE.x, yy);
      yy = fma(S[S_NE + 3], (T)x0nE.y, yy);
      yx = fma(S[S_NW], (T)x0nW.x, yx);
      yx = fma(S[S_NW + 1], (T)x0nW.y, yx);
      yy = fma(S[S_NW + 2], (T)x0nW.x, yy);
      yy = fma(S[S_NW + 3], (T)x0nW.y, yy);
      yx = fma(eW[0], (T)x0W.x, yx);
      yx = fma(eW[2], (T)x0W.y, yx);
      yy = fma(eW[1], (T)x0W.x, yy);
      yy = fma(eW[3], (T)x0W.y, yy);
      if constexpr (kPower) {
        x1c = mk2<TV>(C.inv[0] * yx + C.inv[1] * yy, C.inv[1] * yx + C.inv[2] * yy);
      } else {
        const T rx = (T)C.b.x - yx, ry = (T)C.b.y - yy;
        const T dx = c1a * (T)C.d0.x + c2a * (C.inv[0] * rx + C.inv[1] * ry);
        const T dy = c1a * (T)C.d0.y + c2a * (C.inv[1] * rx + C.inv[2] * ry);
        d1c = mk2<TV>(dx, dy);
        x1c = mk2<TV>((T)xc.x + dx, (T)xc.y + dy);
      }
    }
    // couplings of row q+1 to row q (x0): S, SW, SE blocks, transposed
    const T n1x = C.S[S_N] * (T)xc.x + C.S[S_N + 2] * (T)xc.y + neW[0] * (T)x0W.x + neW[2] * (T)x0W.y +
                  nwE[0] * (T)x0E.x + nwE[2] * (T)x0E.y;
    const T n1y = C.S[S_N + 1] * (T)xc.x + C.S[S_N + 3] * (T)xc.y + neW[1] * (T)x0W.x + neW[3] * (T)x0W.y +
                  nwE[1] * (T)x0E.x + nwE[3] * (T)x0E.y;

    // step 2 at row q - 1
    const TV x1W = shup(x1c), x1E = shdn(x1c);
    const int p = q - 1;
    if (p >= j_lo && p < j_hi && out_lane) {
      const long long np = (long long)p * g.ld + i;
      if (is_interior(i, p, g.N)) {
        const T* S = P.S;
        T yx = a2px, yy = a2py;
        yx = fma(S[S_D], (T)x1p.x, yx);
        yx = fma(S[S_D + 1], (T)x1p.y, yx);
        yy = fma(S[S_D + 1], (T)x1p.x, yy);
        yy = fma(S[S_D + 2], (T)x1p.y, yy);
        yx = fma(S[S_E], (T)x1pE.x, yx);
        yx = fma(S[S_E + 1], (T)x1pE.y, yx);
        yy = fma(S[S_E + 2], (T)x1pE.x, yy);
        yy = fma(S[S_E + 3], (T)x1pE.y, yy);
        yx = fma(S[S_N], (T)x1c.x, yx);
        yx = fma(S[S_N + 1], (T)x1c.y, yx);
        yy = fma(S[S_N + 2], (T)x1c.x, yy);
        yy = fma(S[S_N + 3], (T)x1c.y, yy);
        yx = fma(S[S_NE], (T)x1E.x, yx);
        yx = fma(S[S_NE + 1], (T)x1E.y, yx);
        yy = fma(S[S_NE + 2], (T)x1E.x, yy);
        yy = fma(S[S_NE + 3], (T)x1E.y, yy);
        yx = fma(S[S_NW], (T)x1W.x, yx);
        yx = fma(S[S_NW + 1], (T)x1W.y, yx);
        yy = fma(S[S_NW + 2], (T)x1W.x, yy);
        yy = fma(S[S_NW + 3], (T)x1W.y, yy);
        yx = fma(eWp[0], (T)x1pW.x, yx);
        yx = fma(eWp[2], (T)x1pW.y, yx);
        yy = fma(eWp[1], (T)x1pW.x, yy);
        yy = fma(eWp[3], (T)x1pW.y, yy);
        if constexpr (kPower) {
          x2[np] = mk2<TV>(P.inv[0] * yx + P.inv[1] * yy, P.inv[1] * yx + P.inv[2] * yy);
        } else {
          const T rx = (T)P.b.x - yx, ry = (T)P.b.y - yy;
          const T dx = c1b * (T)d1p.x + c2b * (P.inv[0] * rx + P.inv[1] * ry);
          const T dy = c1b * (T)d1p.y + c2b * (P.inv[1] * rx + P.inv[2] * ry);
          d2[np] = mk2<TV>(dx, dy);
          x2[np] = mk2<TV>((T)x1p.x + dx, (T)x1p.y + dy);
        }
      } else {
        x2[np] = zero;
      }
    }
    // couplings of row q+1 to row q (x1)
    const T n2x = C.S[S_N] * (T)x1c.x + C.S[S_N + 2] * (T)x1c.y + neW[0] * (T)x1W.x + neW[2] * (T)x1W.y +
                  nwE[0] * (T)x1E.x + nwE[2] * (T)x1E.y;
    const T n2y = C.S[S_N + 1] * (T)x1c.x + C.S[S_N + 3] * (T)x1c.y + neW[1] * (T)x1W.x + neW[3] * (T)x1W.y +
                  nwE[1] * (T)x1E.x + nwE[3] * (T)x1E.y;

    // carry to the next row (the row data rotates by the caller's argument order)
    a1x = n1x; a1y = n1y;
    a2px = a2cx; a2py = a2cy;
    a2cx = n2x; a2cy = n2y;
    d1p = d1c;
    x1p = x1c; x1pW = x1W; x1pE = x1E;
    x0W = x0nW; x0E = x0nE;
#pragma unroll
    for (int k = 0; k < 4; ++k) eWp[k] = eW[k];
  };

  Row ra, rb, rc;
  TV xa, xb, xc;
  int q = j_lo - 2;
  load_row(q, rb);
  xb = load_x0(q);
  xc = load_x0(q + 1);
  x0W = shup(xb);
  x0E = shdn(xb);
  // rows rotate through (ra, rb, rc) so that no row data is copied
  for (;;) {
    body(q, ra, rb, rc, xb, xc, xa);
    if (++q > j_hi) break;
    body(q, rb, rc, ra, xc, xa, xb);
    if (++q > j_hi) break;
    body(q, rc, ra, rb, xa, xb, xc);
    if (++q > j_hi) break;
  }
}

__device__ __forceinline__ double pw(int d) { return d == 0 ? 1.0 : 0.5; }

template <typename TV>
__global__ void k_restrict(Layout gf, Layout gc, const TV* __restrict__ rf, TV* __restrict__ bc) {
  using T = typename ScalarOf<TV>::type;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I > gc.N || J > gc.N) return;
  const long long nc = (long long)J * gc.ld + I;
  T sx = 0, sy = 0;
  if (is_interior(I, J, gc.N)) {
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const T w = (T)(pw(di) * pw(dj));
        const TV r = rf[(long long)(2 * J + dj) * gf.ld + (2 * I + di)];
        sx += w * r.x;
        sy += w * r.y;
      }
  }
  bc[nc] = mk2<TV>(sx, sy);
}

template <typename TV>
__global__ void k_prolong_add(Layout gf, Layout gc, const TV* __restrict__ xc, TV* __restrict__ xf) {
  using T = typename ScalarOf<TV>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (!is_interior(i, j, gf.N)) return;
  const long long n = (long long)j * gf.ld + i;
  const int I0 = i >> 1, J0 = j >> 1;
  const int I1 = (i & 1) ? I0 + 1 : I0, J1 = (j & 1) ? J0 + 1 : J0;
  const T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1);
  T sx = 0, sy = 0;
  // coarse boundary entries hold 0
  const TV a = xc[(long long)J0 * gc.ld + I0];
  sx += wi * wj * a.x; sy += wi * wj * a.y;
  if (i & 1) {
    const TV b = xc[(long long)J0 * gc.ld + I1];
    sx += wi * wj * b.x; sy += wi * wj * b.y;
  }
  if (j & 1) {
    const TV c = xc[(long long)J1 * gc.ld + I0];
    sx += wi * wj * c.x; sy += wi * wj * c.y;
  }
  if ((i & 1) && (j & 1)) {
    const TV d = xc[(long long)J1 * gc.ld + I1];
    sx += wi * wj * d.x; sy += wi * wj * d.y;
  }
  const TV xo = xf[n];
  xf[n] = mk2<TV>(xo.x + sx, xo.y + sy);
}

// Galerkin P^T A P, one coarse node per thread; arithmetic in double for a
// double fine stencil, float otherwise.
template <typename TA, typename TF, typename TC>
__global__ void k_rap(Layout gf, Layout gc, const TF* __restrict__ stf, TC* __restrict__ stc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (!is_interior(I, J, gc.N)) return;
  const long long nc = (long long)J * gc.ld + I;
  const int offs[5][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}, {-1, 1}};
  const int slots[5] = {S_D, S_E, S_N, S_NE, S_NW};
#pragma unroll 1
  for (int o = 0; o < 5; ++o) {
    const int DI = offs[o][0], DJ = offs[o][1];
    TA acc[4] = {0, 0, 0, 0};
    if (is_interior(I + DI, J + DJ, gc.N)) {
#pragma unroll 1
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll 1
        for (int di = -1; di <= 1; ++di) {
          const long long nf = (long long)(2 * J + dj) * gf.ld + (2 * I + di);
          const TA wf = (TA)(pw(di) * pw(dj));
          for (int ej = -1; ej <= 1; ++ej) {
            const int oj = 2 * DJ + ej - dj;
            if (oj < -1 || oj > 1) continue;
            for (int ei = -1; ei <= 1; ++ei) {
              const int oi = 2 * DI + ei - di;
              if (oi < -1 || oi > 1) continue;
              TA b[4];
              get_block<TA>(stf, gf.plane, nf, gf.ld, oi, oj, b);
              const TA w = wf * (TA)(pw(ei) * pw(ej));
              acc[0] += w * b[0]; acc[1] += w * b[1]; acc[2] += w * b[2]; acc[3] += w * b[3];
            }
          }
        }
    }
    if (o == 0) {
      stc[(S_D + 0) * gc.plane + nc] = (TC)acc[0];
      stc[(S_D + 1) * gc.plane + nc] = (TC)(0.5 * (acc[1] + acc[2]));
      stc[(S_D + 2) * gc.plane + nc] = (TC)acc[3];
    } else {
      for (int e = 0; e < 4; ++e) stc[(slots[o] + e) * gc.plane + nc] = (TC)acc[e];
    }
  }
}

template <typename TS>
__global__ void k_coarse_dense(Layout g, const TS* __restrict__ st, double* __restrict__ dense) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (!is_interior(i, j, g.N)) return;
  const int m = g.N - 1, n2 = 2 * m * m;
  const long long n = (long long)j * g.ld + i;
  const int row = 2 * ((j - 1) * m + (i - 1));
  for (int dj = -1; dj <= 1; ++dj)
    for (int di = -1; di <= 1; ++di) {
      if (!is_interior(i + di, j + dj, g.N)) continue;
      double b[4];
      get_block<double>(st, g.plane, n, g.ld, di, dj, b);
      const int col = 2 * ((j + dj - 1) * m + (i + di - 1));
      dense[(long long)row * n2 + col] = b[0];
      dense[(long long)row * n2 + col + 1] = b[1];
      dense[(long long)(row + 1) * n2 + col] = b[2];
      dense[(long long)(row + 1) * n2 + col + 1] = b[3];
    }
}

// In-place Cholesky (lower) of the n x n matrix a, then inv = a^-1 by
// forward/back substitution of the unit columns (one column per thread).
__global__ void k_cholesky_inverse(int n, double* __restrict__ a, double* __restrict__ inv, int* __restrict__ info) {
  const int tid = threadIdx.x;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double d = a[(long long)k * n + k];
      if (!(d > 0.0)) bad = k + 1;
      a[(long long)k * n + k] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double lkk = a[(long long)k * n + k];
    for (int r = k + 1 + tid; r < n; r += blockDim.x) a[(long long)r * n + k] /= lkk;
    __syncthreads();
    const int rem = n - k - 1;
    for (long long t = tid; t < (long long)rem * rem; t += blockDim.x) {
      const int r = k + 1 + (int)(t / rem), c = k + 1 + (int)(t % rem);
      if (c <= r) a[(long long)r * n + c] -= a[(long long)r * n + k] * a[(long long)c * n + k];
    }
    __syncthreads();
  }
  if (tid == 0) *info = bad;
  for (int col = tid; col < n; col += blockDim.x) {
    // L y = e_col
    for (int r = 0; r < n; ++r) {
      double s = (r == col) ? 1.0 : 0.0;
      for (int c = 0; c < r; ++c) s -= a[(long long)r * n + c] * inv[(long long)c * n + col];
      inv[(long long)r * n + col] = s / a[(long long)r * n + r];
    }
    // L^T x = y
    for (int r = n - 1; r >= 0; --r) {
      double s = inv[(long long)r * n + col];
      for (int c = r + 1; c < n; ++c) s -= a[(long long)c * n + r] * inv[(long long)c * n + col];
      inv[(long long)r * n + col] = s / a[(long long)r * n + r];
    }
  }
}

template <typename TV>
__global__ void k_coarse_solve(Layout g, int n2, const double* __restrict__ inv, const TV* __restrict__ b,
                               TV* __restrict__ x) {
  using T = typename ScalarOf<TV>::type;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n2) return;
  const int m = g.N - 1;
  double s = 0.0;
  for (int c = 0; c < n2; c += 2) {
    const int node = c >> 1;
    const int ii = node % m + 1, jj = node / m + 1;
    const TV bb = b[(long long)jj * g.ld + ii];
    s += inv[(long long)row * n2 + c] * (double)bb.x + inv[(long long)row * n2 + c + 1] * (double)bb.y;
  }
  const int node = row >> 1;
  const int ii = node % m + 1, jj = node / m + 1;
  T* xs = reinterpret_cast<T*>(x + (long long)jj * g.ld + ii);
  xs[row & 1] = (T)s;
}

template <typename TA, typename TB>
__global__ void k_convert(long long n, const TA* __restrict__ a, TB* __restrict__ b) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = from_d<TB>(to_d(a[t]));
}

}  // namespace

// ---- launchers -----------------------------------------------------------------------
static const dim3 kBlk(32, 8);
static inline dim3 ngrid(const Layout& g) { return dim3((g.n1 + kBlk.x - 1) / kBlk.x, (g.n1 + kBlk.y - 1) / kBlk.y); }

// Row-streaming sweep: levels with at least kStreamMinN cells per side, FP32
// vectors.  Rows per warp are chosen so that the launch is one wave of the
// resident warps (queried once), with at least 16 rows per warp.
constexpr int kStreamMinN = 1024;
template <typename TS, typename TD, typename TV, bool kPower>
static int stream_resident_warps() {
  static const int w = [] {
    int dev = 0, sms = 0, bps = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_cheb_sweep2s<TS, TD, TV, kPower>, 128, 0) !=
            cudaSuccess ||
        bps < 1)
      bps = 1;
    return sms * bps * 4;
  }();
  return w;
}
bool sweep2_streams(const Layout& g, int stream) {
  return stream == 2 || stream == 3 || ((stream == 1 || stream == 4) && g.N >= kStreamMinN);
}
static inline bool sweep2_tma(const Layout& g, int stream) {
  return stream == 3 || (stream == 4 && g.N >= kStreamMinN);
}

static inline int stream_rows(const Layout& g, int resident_warps) {
  const int nstrips = (g.n1 + kStreamCols - 1) / kStreamCols;
  const int target_chunks = std::max(1, resident_warps / nstrips);
  return std::max(16, (g.n1 + target_chunks - 1) / target_chunks);
}

template <typename TS, typename TX, typename TY, typename TA>
void launch_apply(cudaStream_t s, const Layout& g, const TS* st, const TX* x, TY* y) {
  note_launch();
  k_apply<TS, TX, TY, TA><<<ngrid(g), kBlk, 0, s>>>(g, st, x, y);
}
template void launch_apply<double, double2, double2, double>(cudaStream_t, const Layout&, const double*,
                                                             const double2*, double2*);
template void launch_apply<double, float2, double2, double>(cudaStream_t, const Layout&, const double*,
                                                            const float2*, double2*);
template void launch_apply<float, float2, float2, float>(cudaStream_t, const Layout&, const float*, const float2*,
                                                         float2*);
template void launch_apply<__nv_bfloat16, float2, float2, float>(cudaStream_t, const Layout&, const __nv_bfloat16*,
                                                                 const float2*, float2*);

template <typename TS, typename TV>
void launch_residual_stencil(cudaStream_t s, const Layout& g, const TS* st, const TV* x, const TV* b, TV* r) {
  note_launch();
  k_residual_stencil<TS, TV><<<ngrid(g), kBlk, 0, s>>>(g, st, x, b, r);
}

template <typename TS, typename TD>
int launch_dinv_gershgorin(cudaStream_t s, const Layout& g, const TS* st, TD* dinv, double* partial, bool bound) {
  dim3 gr = ngrid(g);
  note_launch();
  k_dinv_gershgorin<TS, TD><<<gr, kBlk, 0, s>>>(g, st, dinv, partial, bound ? 1 : 0);
  return gr.x * gr.y;
}

template <typename TS, typename TD, typename TV>
void launch_power_lmax(cudaStream_t s, const Layout& g, const TS* st, const TD* dinv, int iters, double safety,
                       TV* x0, TV* x1, double* partial, double* lmax, int stream, unsigned polls) {
  note_launch();
  k_checkerboard<TV><<<ngrid(g), kBlk, 0, s>>>(g, x0);
  TV* a = x0;
  TV* b = x1;
  int k = 0;
  if constexpr (sizeof(typename ScalarOf<TV>::type) == 4) {
    if (sweep2_streams(g, stream)) {
      // two power steps per row-streaming pass; the last one or two steps
      // stay single so that x_iters and x_{iters-1} are both at hand
      const int nstrips = (g.n1 + kStreamCols - 1) / kStreamCols;
      const int rows = stream_rows(g, stream_resident_warps<TS, TD, TV, true>());
      const int chunks = (g.n1 + rows - 1) / rows;
      const unsigned blocks = (unsigned)(((long long)nstrips * chunks * 32 + 127) / 128);
      for (; iters - k > 2; k += 2) {
        bool done = false;
        if constexpr (std::is_same<TS, float>::value)
          if (sweep2_tma(g, stream))
            done = launch_cheb_sweep2_tma(s, g, st, dinv, nullptr, 0, a, b, nullptr, nullptr, nullptr, true, polls);
        if (!done) {
          note_launch();
          k_cheb_sweep2s<TS, TD, TV, true><<<blocks, 128, 0, s>>>(g, st, dinv, nullptr, 0, a, b, nullptr, nullptr,
                                                                   nullptr, rows);
        }
        TV* t = a;
        a = b;
        b = t;
      }
    }
  }
  for (; k < iters; ++k) {
    note_launch();
    k_power_step<TS, TD, TV><<<ngrid(g), kBlk, 0, s>>>(g, st, dinv, a, b);
    TV* t = a;
    a = b;
    b = t;
  }
  // a = x_iters, b = x_{iters-1}
  long long nb = (g.plane + 255) / 256;
  if (nb > 1024) nb = 1024;
  note_launch();
  k_norm2_vec<TV><<<(unsigned)nb, 256, 0, s>>>(g.plane, a, partial);
  note_launch();
  k_norm2_vec<TV><<<(unsigned)nb, 256, 0, s>>>(g.plane, b, partial + nb);
  note_launch();
  k_lmax_from_norms<<<1, 1024, 0, s>>>(partial, partial + nb, (int)nb, safety, lmax);
}
template void launch_power_lmax<double, double, double2>(cudaStream_t, const Layout&, const double*, const double*,
                                                         int, double, double2*, double2*, double*, double*, int,
                                                         unsigned);
template void launch_power_lmax<float, float, float2>(cudaStream_t, const Layout&, const float*, const float*, int,
                                                       double, float2*, float2*, double*, double*, int, unsigned);
template void launch_power_lmax<__nv_bfloat16, float, float2>(cudaStream_t, const Layout&, const __nv_bfloat16*,
                                                              const float*, int, double, float2*, float2*, double*,
                                                              double*, int, unsigned);

void launch_max_final(cudaStream_t s, const double* partial, int n, double* out) {
  note_launch();
  k_max_final<<<1, 1024, 0, s>>>(partial, n, out);
}

template <typename T>
void launch_cheb_coefs(cudaStream_t s, const double* lmax, double lo, int deg, T* coef) {
  note_launch();
  k_cheb_coefs<T><<<1, 32, 0, s>>>(lmax, lo, deg, coef);
}
template void launch_cheb_coefs<double>(cudaStream_t, const double*, double, int, double*);
template void launch_cheb_coefs<float>(cudaStream_t, const double*, double, int, float*);

template <typename TS, typename TD, typename TV>
void launch_cheb_zero_start(cudaStream_t s, const Layout& g, const TD* dinv,
                            const typename ScalarOf<TV>::type* coef, const TV* b, TV* x, TV* d) {
  note_launch();
  k_cheb_zero_start<TD, TV><<<ngrid(g), kBlk, 0, s>>>(g, dinv, coef, b, x, d);
}

template <typename TS, typename TD, typename TV>
void launch_cheb_sweep(cudaStream_t s, const Layout& g, const TS* st, const TD* dinv,
                       const typename ScalarOf<TV>::type* coef, int step, const TV* xin, TV* xout, TV* d,
                       const TV* b) {
  note_launch();
  k_cheb_sweep<TS, TD, TV><<<ngrid(g), kBlk, 0, s>>>(g, st, dinv, coef, step, xin, xout, d, b);
}

template <typename TS, typename TD, typename TV>
void launch_cheb_sweep2(cudaStream_t s, const Layout& g, const TS* st, const TD* dinv,
                        const typename ScalarOf<TV>::type* coef, int step, const TV* x0, TV* x2, const TV* d0,
                        TV* d2, const TV* b, int stream, unsigned polls) {
  if constexpr (std::is_same<TS, float>::value) {
    if (sweep2_tma(g, stream) &&
        launch_cheb_sweep2_tma(s, g, st, dinv, coef, step, x0, x2, d0, d2, b, false, polls))
      return;
  }
  note_launch();
  if constexpr (sizeof(typename ScalarOf<TV>::type) == 4) {
    if (sweep2_streams(g, stream)) {
      const int nstrips = (g.n1 + kStreamCols - 1) / kStreamCols;
      const int rows = stream_rows(g, stream_resident_warps<TS, TD, TV, false>());
      const int chunks = (g.n1 + rows - 1) / rows;
      const long long warps = (long long)nstrips * chunks;
      const unsigned blocks = (unsigned)((warps * 32 + 127) / 128);
      k_cheb_sweep2s<TS, TD, TV, false><<<blocks, 128, 0, s>>>(g, st, dinv, coef, step, x0, x2, d0, d2, b, rows);
      return;
    }
  }
  k_cheb_sweep2<TS, TD, TV><<<ngrid(g), kBlk, 0, s>>>(g, st, dinv, coef, step, x0, x2, d0, d2, b);
}

template <typename TV>
void launch_restrict(cudaStream_t s, const Layout& gf, const Layout& gc, const TV* rf, TV* bc) {
  note_launch();
  k_restrict<TV><<<ngrid(gc), kBlk, 0, s>>>(gf, gc, rf, bc);
}

template <typename TV>
void launch_prolong_add(cudaStream_t s, const Layout& gf, const Layout& gc, const TV* xc, TV* xf) {
  note_launch();
  k_prolong_add<TV><<<ngrid(gf), kBlk, 0, s>>>(gf, gc, xc, xf);
}

template <typename TF, typename TC>
void launch_rap(cudaStream_t s, const Layout& gf, const Layout& gc, const TF* stf, TC* stc) {
  using TA = typename std::conditional<std::is_same<TF, double>::value, double, float>::type;
  note_launch();
  k_rap<TA, TF, TC><<<ngrid(gc), kBlk, 0, s>>>(gf, gc, stf, stc);
}

template <typename TS>
void launch_coarse_dense(cudaStream_t s, const Layout& g, const TS* st, double* dense) {
  const int m = g.N - 1, n2 = 2 * m * m;
  cudaMemsetAsync(dense, 0, sizeof(double) * (size_t)n2 * n2, s);
  note_launch();
  k_coarse_dense<TS><<<ngrid(g), kBlk, 0, s>>>(g, st, dense);
}

void launch_cholesky_inverse(cudaStream_t s, int n, double* a, double* inv, int* info) {
  note_launch();
  k_cholesky_inverse<<<1, 256, 0, s>>>(n, a, inv, info);
}

template <typename TV>
void launch_coarse_solve(cudaStream_t s, const Layout& g, int n2, const double* inv, const TV* b, TV* x) {
  cudaMemsetAsync(x, 0, sizeof(TV) * g.plane, s);
  note_launch();
  k_coarse_solve<TV><<<(n2 + 127) / 128, 128, 0, s>>>(g, n2, inv, b, x);
}

template <typename TA, typename TB>
void launch_convert_stencil(cudaStream_t s, const Layout& g, const TA* a, TB* b) {
  const long long n = (long long)NSTEN * g.plane;
  note_launch();
  k_convert<TA, TB><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b);
}

// explicit instantiations: FP64 path (double stencil, double vectors) and
// mixed path (bf16 / float stencils, float vectors)
#define SVN_INST_LEVEL(TS, TD, TV)                                                                                 \
  template void launch_residual_stencil<TS, TV>(cudaStream_t, const Layout&, const TS*, const TV*, const TV*,    \
                                                TV*);                                                            \
  template int launch_dinv_gershgorin<TS, TD>(cudaStream_t, const Layout&, const TS*, TD*, double*, bool);       \
  template void launch_cheb_zero_start<TS, TD, TV>(cudaStream_t, const Layout&, const TD*,                      \
                                                   const typename ScalarOf<TV>::type*, const TV*, TV*, TV*);     \
  template void launch_cheb_sweep<TS, TD, TV>(cudaStream_t, const Layout&, const TS*, const TD*,                 \
                                              const typename ScalarOf<TV>::type*, int, const TV*, TV*, TV*,      \
                                              const TV*);                                                        \
  template void launch_coarse_dense<TS>(cudaStream_t, const Layout&, const TS*, double*);                       \
  template void launch_cheb_sweep2<TS, TD, TV>(cudaStream_t, const Layout&, const TS*, const TD*,                \
                                               const typename ScalarOf<TV>::type*, int, const TV*, TV*,          \
                                               const TV*, TV*, const TV*, int, unsigned);

SVN_INST_LEVEL(double, double, double2)
SVN_INST_LEVEL(__nv_bfloat16, float, float2)
SVN_INST_LEVEL(float, float, float2)

template int launch_dinv_gershgorin<double, float>(cudaStream_t, const Layout&, const double*, float*, double*,
                                                   bool);
template void launch_restrict<double2>(cudaStream_t, const Layout&, const Layout&, const double2*, double2*);
template void launch_restrict<float2>(cudaStream_t, const Layout&, const Layout&, const float2*, float2*);
template void launch_prolong_add<double2>(cudaStream_t, const Layout&, const Layout&, const double2*, double2*);
template void launch_prolong_add<float2>(cudaStream_t, const Layout&, const Layout&, const float2*, float2*);
template void launch_coarse_solve<double2>(cudaStream_t, const Layout&, int, const double*, const double2*,
                                           double2*);
template void launch_coarse_solve<float2>(cudaStream_t, const Layout&, int, const double*, const float2*, float2*);
template void launch_rap<double, double>(cudaStream_t, const Layout&, const Layout&, const double*, double*);
template void launch_rap<float, float>(cudaStream_t, const Layout&, const Layout&, const float*, float*);
template void launch_rap<double, float>(cudaStream_t, const Layout&, const Layout&, const double*, float*);
template void launch_convert_stencil<double, __nv_bfloat16>(cudaStream_t, const Layout&, const double*,
                                                            __nv_bfloat16*);
template void launch_convert_stencil<double, float>(cudaStream_t, const Layout&, const double*, float*);
template void launch_convert_stencil<float, __nv_bfloat16>(cudaStream_t, const Layout&, const float*,
                                                           __nv_bfloat16*);

}  // namespace svn
