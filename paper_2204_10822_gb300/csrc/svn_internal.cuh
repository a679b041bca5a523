// Internal layout and device helpers of the svN solver (sm_103a).
//
// Layout in HBM (one multigrid level):
//   * node arrays: (N+1) rows of `ld` nodes, ld = round_up(N+1, 8), so rows
//     start on 64-byte boundaries for double2 and 16-byte boundaries for
//     bf16 planes; node (i, j) at j*ld + i.  Boundary and padding nodes of
//     every vector hold 0.
//   * vectors: interleaved (vx, vy) as double2 / float2 per node.
//   * cell arrays: cell (i, j) at j*ld + i (same stride; i < N).
//   * quadrature-point fields and stencils: structure of arrays, one plane of
//     `plane` entries per component (plane = round_up((N+1)*ld, 64)).
//   * stencil: 19 planes per node -- the symmetric 2x2 diagonal block
//     (xx, xy, yy) and the full 2x2 blocks coupling to the E, N, NE and NW
//     neighbours, [xx, xy, yx, yy] with y_k += K_kl x_l.  The blocks to the
//     W, S, SW, SE neighbours are the transposes of the neighbour's E, N, NE,
//     NW blocks (the operator is symmetric).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace svn {

constexpr int NSTEN = 19;
enum StencilSlot { S_D = 0, S_E = 3, S_N = 7, S_NE = 11, S_NW = 15 };
constexpr int NELEM = 36;   // unique entries of the symmetric 8x8 element matrix


// Gauss points on [0, 1]
constexpr double GQ0 = 0.21132486540518711775;   // 1/2 - 1/(2 sqrt 3)
constexpr double GQ1 = 0.78867513459481288225;   // 1/2 + 1/(2 sqrt 3)

struct Layout {
  int N;            // cells per side
  int n1;           // nodes per side (N + 1)
  int ld;           // row stride in nodes / cells
  long long plane;  // entries per SoA plane
  double dx;
};

inline Layout make_layout(int N, double L) {
  Layout g;
  g.N = N;
  g.n1 = N + 1;
  g.ld = (g.n1 + 7) / 8 * 8;
  long long nn = (long long)g.n1 * g.ld;
  g.plane = (nn + 63) / 64 * 64;
  g.dx = L / N;
  return g;
}

// Constants of one implicit step, as used by the cell kernels.
struct Phys {
  double dt;
  double dx;
  double idx;        // 1 / dx
  double w;          // quadrature weight dx^2 / 4
  double ta, tb, tc; // tau-hat coefficients: (1+1/e)/2, (1-1/e)/2, 1/(2e)
  double dmin2;      // Delta_min^2
  double cdrag;      // Co rho_o
};

// Element-matrix packing: upper triangle of the 8x8 matrix over local dofs
// d = 2*c + k (corner c = 2*b + a at node (i+a, j+b)), row-major.
__host__ __device__ constexpr int elem_index(int r, int c) {
  // requires r <= c
  return r * 8 - r * (r - 1) / 2 + (c - r);
}

// ---- reductions ------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum; result valid in thread 0.  blockDim.x*y multiple of 32, <= 1024.
template <typename T>
__device__ T block_sum(T v) {
  __shared__ T red[32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nw = (blockDim.x * blockDim.y) >> 5;
  v = warp_sum(v);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  T r = (tid < nw) ? red[tid] : T(0);
  if (tid < 32) r = warp_sum(r);
  __syncthreads();
  return r;
}

template <typename T>
__device__ T block_max(T v) {
  __shared__ T red[32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nw = (blockDim.x * blockDim.y) >> 5;
  v = warp_max(v);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  T r = (tid < nw) ? red[tid] : T(0);
  if (tid < 32) r = warp_max(r);
  __syncthreads();
  return r;
}

// Error-free transformation a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Compensated (double-double) accumulator.
struct DD {
  double hi, lo;
  __device__ __forceinline__ void add(double x) {
    double s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ void add(const DD& o) {
    double s, e;
    two_sum(hi, o.hi, s, e);
    hi = s;
    lo += e + o.lo;
  }
};

// ---- conversions -----------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_f(T x);
template <> __device__ __forceinline__ float to_f<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double x) { return __double2bfloat16(x); }

template <typename T> __device__ __forceinline__ double to_d(T x) { return (double)x; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <typename V> struct ScalarOf;
template <> struct ScalarOf<double2> { using type = double; };
template <> struct ScalarOf<float2> { using type = float; };

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

}  // namespace svn
