// Vector kernels: layout conversion, BLAS-1, and the fused FGMRES Arnoldi
// pieces (one-pass multi-dot, one-pass update + norm), FP64 throughout.
// Reductions are deterministic: per-warp partials, then a fixed-order final
// reduction.
#include <atomic>

#include "kernels.h"

namespace svn {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches_issued() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int EPT = 8;              // double2 elements per thread in Arnoldi kernels
constexpr int ARN_THREADS = 256;

__global__ void k_sum_final(const double* __restrict__ partial, int n, double* __restrict__ out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) s += partial[b];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_unpack_nodes(Layout g, const double* __restrict__ src, double2* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.ld || j > g.N) return;
  const long long n = (long long)j * g.ld + i;
  double2 v = make_double2(0.0, 0.0);
  if (i >= 1 && j >= 1 && i <= g.N - 1 && j <= g.N - 1) {
    const long long k = 2 * ((long long)j * g.n1 + i);
    v = make_double2(src[k], src[k + 1]);
  }
  dst[n] = v;
}

__global__ void k_pack_nodes(Layout g, const double2* __restrict__ src, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  const long long k = 2 * ((long long)j * g.n1 + i);
  double2 v = make_double2(0.0, 0.0);
  if (i >= 1 && j >= 1 && i <= g.N - 1 && j <= g.N - 1) v = src[(long long)j * g.ld + i];
  dst[k] = v.x;
  dst[k + 1] = v.y;
}

__global__ void k_unpack_pi(Layout g, const double* __restrict__ src, double* __restrict__ pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N || j >= g.N) return;
  const long long cell = (long long)j * g.ld + i;
  const long long base = ((long long)j * g.N + i) * 12;
  for (int t = 0; t < 12; ++t) pi[t * g.plane + cell] = src[base + t];
}

__global__ void k_pack_pi(Layout g, const double* __restrict__ pi, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N || j >= g.N) return;
  const long long cell = (long long)j * g.ld + i;
  const long long base = ((long long)j * g.N + i) * 12;
  for (int t = 0; t < 12; ++t) dst[base + t] = pi[t * g.plane + cell];
}

// Flat element-wise kernels over the padded plane (padding holds 0).
__global__ void k_norm2_partial(long long n, const double2* __restrict__ x, double* __restrict__ partial) {
  double s = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    s = fma(v.x, v.x, s);
    s = fma(v.y, v.y, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_scale_copy(long long n, const double2* __restrict__ x, const double* __restrict__ num,
                             const double* __restrict__ den, double2* __restrict__ y) {
  const double a = *num / *den;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    y[t] = make_double2(a * v.x, a * v.y);
  }
}

__global__ void k_axpy(long long n, double a, const double2* __restrict__ x, double2* __restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t], w = y[t];
    y[t] = make_double2(w.x + a * v.x, w.y + a * v.y);
  }
}

__global__ void k_axpby_to(long long n, const double2* __restrict__ x, double a, const double2* __restrict__ d,
                           double2* __restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t], w = d[t];
    y[t] = make_double2(v.x + a * w.x, v.y + a * w.y);
  }
}

__global__ void k_scale_to(long long n, double a, const double2* __restrict__ x, double2* __restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    y[t] = make_double2(a * v.x, a * v.y);
  }
}

// counts[0]: non-finite entries, [1]: h <= 0, [2]: A outside [0, 1]
__global__ void k_validate(long long nc, long long nv, const double* __restrict__ h, const double* __restrict__ A,
                           const double* __restrict__ wind, const double* __restrict__ ocean,
                           const double* __restrict__ vold, int* __restrict__ counts) {
  int bad = 0, hneg = 0, arng = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (long long)gridDim.x * blockDim.x) {
    if (t < nc) {
      const double hh = h[t], aa = A[t];
      bad += !isfinite(hh) + !isfinite(aa);
      hneg += isfinite(hh) && !(hh > 0.0);
      arng += isfinite(aa) && (aa < 0.0 || aa > 1.0);
    }
    bad += !isfinite(wind[t]) + !isfinite(ocean[t]) + !isfinite(vold[t]);
  }
  bad = warp_sum(bad);
  hneg = warp_sum(hneg);
  arng = warp_sum(arng);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicAdd(counts, bad);
    if (hneg) atomicAdd(counts + 1, hneg);
    if (arng) atomicAdd(counts + 2, arng);
  }
}

__global__ void k_neg_copy(long long n, const double2* __restrict__ x, double2* __restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    y[t] = make_double2(-v.x, -v.y);
  }
}

__global__ void k_cast_d2f(long long n, const double2* __restrict__ x, float2* __restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    y[t] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void k_cast_f2d(long long n, const float2* __restrict__ x, double2* __restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float2 v = x[t];
    y[t] = make_double2(v.x, v.y);
  }
}

// Sum of eight per-lane values over the warp by recursive halving: at each of
// the first three steps a lane keeps half of its values and adds the partner's
// copy of them (one shuffle per kept value), so the eight totals cost 9
// shuffle-adds per lane instead of 40.  On return every lane holds the total of
// value (lane >> 2).
__device__ __forceinline__ double warp_sum8(const double v[8], int lane) {
  const bool b0 = lane & 16, b1 = lane & 8, b2 = lane & 4;
  double u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double keep = b0 ? v[k + 4] : v[k];
    const double give = b0 ? v[k] : v[k + 4];
    u[k] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
  }
  double w[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double keep = b1 ? u[k + 2] : u[k];
    const double give = b1 ? u[k] : u[k + 2];
    w[k] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
  }
  double z = (b2 ? w[1] : w[0]) + __shfl_xor_sync(0xffffffffu, b2 ? w[0] : w[1], 4);
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return z;
}

// partial[i * nwarps + warp] = sum over the warp's elements of V_i . w; the
// basis vectors are taken eight at a time (FMA chains, one warp_sum8 each).
__global__ void __launch_bounds__(ARN_THREADS) k_multidot(long long n, const double2* __restrict__ V,
                                                          long long vstride, int m, const double2* __restrict__ w,
                                                          double* __restrict__ partial, int nwarps) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long base = warp * (32 * EPT) + lane;
  double2 wr[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const long long t = base + 32 * e;
    wr[e] = t < n ? w[t] : make_double2(0.0, 0.0);
  }
  for (int i0 = 0; i0 < m; i0 += 8) {
    double s[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      s[c] = 0.0;
      if (i0 + c < m) {
        const double2* Vi = V + (long long)(i0 + c) * vstride;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          const long long t = base + 32 * e;
          if (t < n) {
            const double2 a = Vi[t];
            s[c] = fma(a.x, wr[e].x, s[c]);
            s[c] = fma(a.y, wr[e].y, s[c]);
          }
        }
      }
    }
    const double tot = warp_sum8(s, lane);
    const int c = lane >> 2;
    if ((lane & 3) == 0 && i0 + c < m && warp < nwarps) partial[(long long)(i0 + c) * nwarps + warp] = tot;
  }
}

// h[i] (+)= sum_warp partial[i * nwarps + warp]; one block per i.
__global__ void k_multidot_final(const double* __restrict__ partial, int nwarps, double* __restrict__ h,
                                 int accumulate) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nwarps; b += blockDim.x) s += partial[(long long)i * nwarps + b];
  s = block_sum(s);
  if (threadIdx.x == 0) h[i] = accumulate ? h[i] + s : s;
}

// w -= sum_i h[i] V_i; partial[warp] = |w|^2 over the warp's elements.
__global__ void __launch_bounds__(ARN_THREADS) k_update_norm(long long n, const double2* __restrict__ V,
                                                             long long vstride, int m, const double* __restrict__ h,
                                                             double2* __restrict__ w, double* __restrict__ partial,
                                                             int nwarps) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long base = warp * (32 * EPT) + lane;
  double2 wr[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const long long t = base + 32 * e;
    wr[e] = t < n ? w[t] : make_double2(0.0, 0.0);
  }
  for (int i = 0; i < m; ++i) {
    const double2* Vi = V + (long long)i * vstride;
    const double hi = h[i];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const long long t = base + 32 * e;
      if (t < n) {
        const double2 a = Vi[t];
        wr[e].x = fma(-hi, a.x, wr[e].x);
        wr[e].y = fma(-hi, a.y, wr[e].y);
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const long long t = base + 32 * e;
    if (t < n) {
      w[t] = wr[e];
      s = fma(wr[e].x, wr[e].x, s);
      s = fma(wr[e].y, wr[e].y, s);
    }
  }
  s = warp_sum(s);
  if (lane == 0 && warp < nwarps) partial[warp] = s;
}

template <typename TZ>
__global__ void k_lincomb(long long n, const TZ* __restrict__ Z, long long zstride, int m, const double* __restrict__ y,
                          double2* __restrict__ x) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double2 acc = x[t];
    for (int j = 0; j < m; ++j) {
      const TZ z = Z[(long long)j * zstride + t];
      acc.x += y[j] * (double)z.x;
      acc.y += y[j] * (double)z.y;
    }
    x[t] = acc;
  }
}

const dim3 kBlk(32, 8);
inline dim3 ngrid(const Layout& g) { return dim3((g.n1 + kBlk.x - 1) / kBlk.x, (g.n1 + kBlk.y - 1) / kBlk.y); }
inline dim3 cgrid(const Layout& g) { return dim3((g.N + kBlk.x - 1) / kBlk.x, (g.N + kBlk.y - 1) / kBlk.y); }
inline unsigned flat_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

int reduce_blocks(long long n) { return (int)flat_blocks(n); }
int krylov_blocks(const Layout& g) { return (int)((g.plane + 32 * EPT - 1) / (32 * EPT)); }

void launch_sum_final(cudaStream_t s, const double* partial, int n, double* out) {
  note_launch();
  k_sum_final<<<1, 1024, 0, s>>>(partial, n, out);
}
void launch_unpack_nodes(cudaStream_t s, const Layout& g, const double* src, double2* dst) {
  dim3 gr((g.ld + kBlk.x - 1) / kBlk.x, (g.n1 + kBlk.y - 1) / kBlk.y);
  note_launch();
  k_unpack_nodes<<<gr, kBlk, 0, s>>>(g, src, dst);
}
void launch_pack_nodes(cudaStream_t s, const Layout& g, const double2* src, double* dst) {
  note_launch();
  k_pack_nodes<<<ngrid(g), kBlk, 0, s>>>(g, src, dst);
}
void launch_unpack_pi(cudaStream_t s, const Layout& g, const double* src, double* pi) {
  note_launch();
  k_unpack_pi<<<cgrid(g), kBlk, 0, s>>>(g, src, pi);
}
void launch_pack_pi(cudaStream_t s, const Layout& g, const double* pi, double* dst) {
  note_launch();
  k_pack_pi<<<cgrid(g), kBlk, 0, s>>>(g, pi, dst);
}
void launch_norm2_partial(cudaStream_t s, const Layout& g, const double2* x, double* partial) {
  note_launch();
  k_norm2_partial<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, x, partial);
}
void launch_scale_copy(cudaStream_t s, const Layout& g, const double2* x, const double* num, const double* den,
                       double2* y) {
  note_launch();
  k_scale_copy<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, x, num, den, y);
}
void launch_axpy(cudaStream_t s, const Layout& g, double a, const double2* x, double2* y) {
  note_launch();
  k_axpy<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, a, x, y);
}
void launch_axpby_to(cudaStream_t s, const Layout& g, const double2* x, double a, const double2* d, double2* y) {
  note_launch();
  k_axpby_to<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, x, a, d, y);
}
void launch_scale_to(cudaStream_t s, const Layout& g, double a, const double2* x, double2* y) {
  note_launch();
  k_scale_to<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, a, x, y);
}
void launch_validate(cudaStream_t s, long long ncell, long long nvec, const double* h, const double* A,
                     const double* wind, const double* ocean, const double* vold, int* counts) {
  note_launch();
  k_validate<<<flat_blocks(nvec), 256, 0, s>>>(ncell, nvec, h, A, wind, ocean, vold, counts);
}
void launch_neg_copy(cudaStream_t s, const Layout& g, const double2* x, double2* y) {
  note_launch();
  k_neg_copy<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, x, y);
}
void launch_cast_d2f(cudaStream_t s, const Layout& g, const double2* x, float2* y) {
  note_launch();
  k_cast_d2f<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, x, y);
}
void launch_cast_f2d(cudaStream_t s, const Layout& g, const float2* x, double2* y) {
  note_launch();
  k_cast_f2d<<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, x, y);
}
void launch_multidot(cudaStream_t s, const Layout& g, const double2* V, long long vstride, int m, const double2* w,
                     double* partial, int nwarps) {
  const long long threads = (long long)nwarps * 32;
  note_launch();
  k_multidot<<<(unsigned)((threads + ARN_THREADS - 1) / ARN_THREADS), ARN_THREADS, 0, s>>>(g.plane, V, vstride, m, w,
                                                                                          partial, nwarps);
}
void launch_multidot_final(cudaStream_t s, const double* partial, int nwarps, int m, double* h, int accumulate) {
  note_launch();
  k_multidot_final<<<m, 1024, 0, s>>>(partial, nwarps, h, accumulate);
}
void launch_update_norm(cudaStream_t s, const Layout& g, const double2* V, long long vstride, int m, const double* h,
                        double2* w, double* partial, int nwarps) {
  const long long threads = (long long)nwarps * 32;
  note_launch();
  k_update_norm<<<(unsigned)((threads + ARN_THREADS - 1) / ARN_THREADS), ARN_THREADS, 0, s>>>(g.plane, V, vstride, m,
                                                                                             h, w, partial, nwarps);
}
template <typename TZ>
void launch_lincomb(cudaStream_t s, const Layout& g, const TZ* Z, long long zstride, int m, const double* y,
                    double2* x) {
  note_launch();
  k_lincomb<TZ><<<flat_blocks(g.plane), 256, 0, s>>>(g.plane, Z, zstride, m, y, x);
}
template void launch_lincomb<double2>(cudaStream_t, const Layout&, const double2*, long long, int, const double*,
                                      double2*);
template void launch_lincomb<float2>(cudaStream_t, const Layout&, const float2*, long long, int, const double*,
                                     double2*);

}  // namespace svn
