// Learned Newton initial guess (no counterpart in the paper): a 4-level
// convolutional encoder-decoder (U-Net, 32/64/128/256 channels, 3x3
// convolutions, 2x2 average pooling, nearest upsampling with skip
// concatenation) on a G x G cell grid, trained on (forcing, h, A, v_old) ->
// converged velocity pairs produced by the solver itself.
//
// Numerics: BF16 activations and weights, FP32 accumulation.  The forward
// and backward-data convolutions are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16 BF16 -> FP32; GEMM M = pixels, N = output channels,
// K = 9 x input channels); weight and bias gradients accumulate in FP32 on the
// CUDA cores; Adam keeps FP32 master weights.  Layouts are NHWC (channels
// innermost); weights are [Cout][tap = 3 ky + kx][Cin].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/svn.h"
#include "kernels.h"

namespace svn {

namespace {

using bf16 = __nv_bfloat16;

// Scales of the network's inputs and output (fixed, documented in svn.h).
constexpr float kScaleH = 2.0f, kOffA = 0.9f, kScaleA = 0.1f, kScaleWind = 15.0f, kScaleOcean = 0.1f,
                kScaleV = 0.2f;
constexpr int kCin0 = 16;   // 8 input channels padded to the MMA K step

__device__ __forceinline__ uint32_t ld_b32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 3x3 convolution, stride 1, zero padding 1, as an implicit GEMM.
// Y[p][co] = act(bias[co] + sum_{tap,ci} X[p + off(tap)][ci] W[co][tap][ci]).
// Block: 4 warps x 16 pixels = 64 pixels; NT output channels (multiple of 8).
// Requires Cin % 16 == 0, Cout % NT == 0, (B H W) % 64 == 0.
template <int NT>
__global__ void __launch_bounds__(128) k_conv3x3(int B, int H, int W, int Cin, int Cout, const bf16* __restrict__ X,
                                                 const bf16* __restrict__ Wt, const float* __restrict__ bias,
                                                 bf16* __restrict__ Y, int relu) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const long long p0 = (long long)blockIdx.x * 64 + warp * 16;
  const int co0 = blockIdx.y * NT;
  const long long HW = (long long)H * W;
  long long pr[2];
  int yr[2], xr[2];
  long long br[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    pr[r] = p0 + g + 8 * r;
    br[r] = pr[r] / HW;
    const long long rem = pr[r] - br[r] * HW;
    yr[r] = (int)(rem / W);
    xr[r] = (int)(rem - (long long)yr[r] * W);
  }
  float acc[NT / 8][4];
#pragma unroll
  for (int n = 0; n < NT / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const bf16* src[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int yy = yr[r] + dy, xx = xr[r] + dx;
      src[r] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? X + ((br[r] * H + yy) * W + xx) * Cin : nullptr;
    }
    for (int ci0 = 0; ci0 < Cin; ci0 += 16) {
      uint32_t a[4];
      a[0] = src[0] ? ld_b32(src[0] + ci0 + 2 * t) : 0u;
      a[1] = src[1] ? ld_b32(src[1] + ci0 + 2 * t) : 0u;
      a[2] = src[0] ? ld_b32(src[0] + ci0 + 2 * t + 8) : 0u;
      a[3] = src[1] ? ld_b32(src[1] + ci0 + 2 * t + 8) : 0u;
#pragma unroll
      for (int n = 0; n < NT / 8; ++n) {
        const bf16* wp = Wt + ((long long)(co0 + n * 8 + g) * 9 + tap) * Cin + ci0 + 2 * t;
        uint32_t b[2] = {ld_b32(wp), ld_b32(wp + 8)};
        mma_bf16(acc[n], a, b);
      }
    }
  }
#pragma unroll
  for (int n = 0; n < NT / 8; ++n) {
    const int co = co0 + n * 8 + 2 * t;
    const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float v0 = acc[n][2 * r] + b0, v1 = acc[n][2 * r + 1] + b1;
      if (relu) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      __nv_bfloat162 o = __floats2bfloat162_rn(v0, v1);
      *reinterpret_cast<__nv_bfloat162*>(Y + pr[r] * Cout + co) = o;
    }
  }
}

// Weights for the backward-data convolution: Wb[ci][tap][co] = W[co][8 - tap][ci].
__global__ void k_flip_weights(int Cin, int Cout, const bf16* __restrict__ W, bf16* __restrict__ Wb) {
  const long long n = (long long)Cout * 9 * Cin;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(e % Cin);
    const int tap = (int)((e / Cin) % 9);
    const int co = (int)(e / ((long long)Cin * 9));
    Wb[((long long)ci * 9 + (8 - tap)) * Cout + co] = W[e];
  }
}

// dW[co][tap][ci] += sum_p dY[p][co] X[p + off(tap)][ci]; bias gradient from tap 4.
// Block: 32 x 8 threads, a 32 (ci) x 32 (co) tile of one tap over a pixel range.
__global__ void k_conv_wgrad(int B, int H, int W, int Cin, int Cout, const bf16* __restrict__ X,
                             const bf16* __restrict__ dY, float* __restrict__ dW, float* __restrict__ dB,
                             long long pix_per_block) {
  __shared__ float sx[32][33], sd[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int ci0 = blockIdx.x * 32, co0 = blockIdx.y * 32;
  const int tap = blockIdx.z % 9;
  const long long split = blockIdx.z / 9;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const long long P = (long long)B * H * W, HW = (long long)H * W;
  const long long pbeg = split * pix_per_block;
  const long long pend = pbeg + pix_per_block < P ? pbeg + pix_per_block : P;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  for (long long pc = pbeg; pc < pend; pc += 32) {
    // stage 32 pixels: sx[pixel][ci], sd[pixel][co]
    for (int r = ty; r < 32; r += 8) {
      const long long p = pc + r;
      float xv = 0.f, dv = 0.f;
      if (p < pend) {
        const long long b = p / HW, rem = p - b * HW;
        const int y = (int)(rem / W), x = (int)(rem - (long long)y * W);
        const int yy = y + dy, xx = x + dx;
        if (ci0 + tx < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
          xv = __bfloat162float(X[((b * H + yy) * W + xx) * Cin + ci0 + tx]);
        if (co0 + tx < Cout) dv = __bfloat162float(dY[p * Cout + co0 + tx]);
      }
      sx[r][tx] = xv;
      sd[r][tx] = dv;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float xv = sx[r][tx];
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += sd[r][ty * 4 + k] * xv;
    }
    if (tap == 4 && ty == 0 && blockIdx.x == 0)
      for (int r = 0; r < 32; ++r) bacc += sd[r][tx];
    __syncthreads();
  }
  if (ci0 + tx < Cin)
    for (int k = 0; k < 4; ++k) {
      const int co = co0 + ty * 4 + k;
      if (co < Cout) atomicAdd(&dW[((long long)co * 9 + tap) * Cin + ci0 + tx], acc[k]);
    }
  if (tap == 4 && ty == 0 && blockIdx.x == 0 && co0 + tx < Cout) atomicAdd(&dB[co0 + tx], bacc);
}

// dY <- dY * (Y > 0)
__global__ void k_relu_bwd(long long n, const bf16* __restrict__ Y, bf16* __restrict__ dY) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(Y[e]) > 0.f)) dY[e] = __float2bfloat16(0.f);
}

// 2x2 average pooling (forward) and its adjoint (backward, accumulating).
__global__ void k_pool(int B, int H, int W, int C, const bf16* __restrict__ X, bf16* __restrict__ Y) {
  const int H2 = H / 2, W2 = W / 2;
  const long long n = (long long)B * H2 * W2 * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const long long q = e / C;
    const int x = (int)(q % W2), y = (int)((q / W2) % H2);
    const long long b = q / ((long long)W2 * H2);
    const bf16* s = X + ((b * H + 2 * y) * W + 2 * x) * C + c;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[(long long)W * C]) +
                    __bfloat162float(s[(long long)W * C + C]);
    Y[e] = __float2bfloat16(0.25f * v);
  }
}

__global__ void k_pool_bwd_add(int B, int H, int W, int C, const bf16* __restrict__ dY, bf16* __restrict__ dX) {
  const long long n = (long long)B * H * W * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const long long q = e / C;
    const int x = (int)(q % W), y = (int)((q / W) % H);
    const long long b = q / ((long long)W * H);
    const float g = 0.25f * __bfloat162float(dY[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]);
    dX[e] = __float2bfloat16(__bfloat162float(dX[e]) + g);
  }
}

// Concatenation [nearest-upsampled U (Cu channels, H/2 x W/2) | S (Cs channels)].
__global__ void k_up_concat(int B, int H, int W, int Cu, int Cs, const bf16* __restrict__ U,
                            const bf16* __restrict__ S, bf16* __restrict__ Cat) {
  const int C = Cu + Cs;
  const long long n = (long long)B * H * W * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const long long q = e / C;
    const int x = (int)(q % W), y = (int)((q / W) % H);
    const long long b = q / ((long long)W * H);
    Cat[e] = c < Cu ? U[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * Cu + c] : S[q * Cs + (c - Cu)];
  }
}

// Adjoint of k_up_concat: dU (sum over 2x2) and dS (overwrite).
__global__ void k_up_concat_bwd(int B, int H, int W, int Cu, int Cs, const bf16* __restrict__ dCat,
                                bf16* __restrict__ dU, bf16* __restrict__ dS) {
  const int C = Cu + Cs;
  const long long nu = (long long)B * (H / 2) * (W / 2) * Cu;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nu; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % Cu);
    const long long q = e / Cu;
    const int x = (int)(q % (W / 2)), y = (int)((q / (W / 2)) % (H / 2));
    const long long b = q / ((long long)(W / 2) * (H / 2));
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
      for (int d = 0; d < 2; ++d) s += __bfloat162float(dCat[((b * H + 2 * y + a) * W + 2 * x + d) * C + c]);
    dU[e] = __float2bfloat16(s);
  }
  const long long ns = (long long)B * H * W * Cs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ns; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % Cs);
    const long long q = e / Cs;
    dS[e] = dCat[q * C + Cu + c];
  }
}

// Loss 0.5 * mean over pixels and the 2 used channels of (Y - T)^2 and its gradient.
__global__ void k_mse(long long P, int C, const bf16* __restrict__ Y, const float* __restrict__ T,
                      bf16* __restrict__ dY, float* __restrict__ loss) {
  float s = 0.f;
  const float inv = 1.f / (float)(2 * P);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < C; ++c) {
      float gr = 0.f;
      if (c < 2) {
        const float d = __bfloat162float(Y[p * C + c]) - T[p * 2 + c];
        s += 0.5f * d * d * inv;
        gr = d * inv;
      }
      dY[p * C + c] = __float2bfloat16(gr);
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(loss, s);
}

// Adam on FP32 master parameters; weights also refreshed in BF16.
__global__ void k_adam(long long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ pb, long long nb) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gg = gr[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float np = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = np;
    if (e < nb) pb[e] = __float2bfloat16(np);
  }
}

__global__ void k_f2bf(long long n, const float* __restrict__ a, bf16* __restrict__ b) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    b[e] = __float2bfloat16(a[e]);
}

// Network input at G x G cells from a problem on N x N cells (N = f G):
// block averages of h, A (cells) and of wind, ocean, v_old (nodes of the block).
__global__ void k_features(int N, int G, const double* __restrict__ h, const double* __restrict__ A,
                           const double* __restrict__ wind, const double* __restrict__ ocean,
                           const double* __restrict__ vold, bf16* __restrict__ X) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= G || J >= G) return;
  const int f = N / G, n1 = N + 1;
  double sh = 0, sa = 0;
  for (int j = J * f; j < (J + 1) * f; ++j)
    for (int i = I * f; i < (I + 1) * f; ++i) {
      sh += h[(long long)j * N + i];
      sa += A[(long long)j * N + i];
    }
  sh /= (double)f * f;
  sa /= (double)f * f;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int j = J * f; j <= (J + 1) * f; ++j)
    for (int i = I * f; i <= (I + 1) * f; ++i) {
      const long long k = 2 * ((long long)j * n1 + i);
      const bool bnd = i == 0 || j == 0 || i == N || j == N;
      s[0] += wind[k]; s[1] += wind[k + 1];
      s[2] += ocean[k]; s[3] += ocean[k + 1];
      if (!bnd) { s[4] += vold[k]; s[5] += vold[k + 1]; }
    }
  const double inv = 1.0 / ((double)(f + 1) * (f + 1));
  float c[kCin0] = {};
  c[0] = (float)(sh / kScaleH);
  c[1] = (float)((sa - kOffA) / kScaleA);
  c[2] = (float)(s[0] * inv / kScaleWind);
  c[3] = (float)(s[1] * inv / kScaleWind);
  c[4] = (float)(s[2] * inv / kScaleOcean);
  c[5] = (float)(s[3] * inv / kScaleOcean);
  c[6] = (float)(s[4] * inv / kScaleV);
  c[7] = (float)(s[5] * inv / kScaleV);
  bf16* o = X + ((long long)J * G + I) * kCin0;
  for (int k = 0; k < kCin0; ++k) o[k] = __float2bfloat16(c[k]);
}

// Training target at G x G cells (N = G): mean of v over the cell's 4 corners / v scale.
__global__ void k_target(int N, const double* __restrict__ v, float* __restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const int n1 = N + 1;
  double sx = 0, sy = 0;
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      const int ii = i + a, jj = j + b;
      if (ii == 0 || jj == 0 || ii == N || jj == N) continue;
      const long long k = 2 * ((long long)jj * n1 + ii);
      sx += v[k];
      sy += v[k + 1];
    }
  T[((long long)j * N + i) * 2] = (float)(0.25 * sx / kScaleV);
  T[((long long)j * N + i) * 2 + 1] = (float)(0.25 * sy / kScaleV);
}

// Prediction (G x G cell centres, channels 0, 1 of Y) -> node velocity of the
// N x N grid in the solver layout: bilinear in the cell-centre lattice
// (clamped at the outer half cell), zero on the boundary.
__global__ void k_prolong_pred(int G, int C, Layout g, const bf16* __restrict__ Y, double2* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.N || j > g.N) return;
  double2 out = make_double2(0.0, 0.0);
  if (i >= 1 && j >= 1 && i <= g.N - 1 && j <= g.N - 1) {
    const double fx = (double)i * G / g.N - 0.5, fy = (double)j * G / g.N - 0.5;
    const double cx = fmin(fmax(fx, 0.0), G - 1.0), cy = fmin(fmax(fy, 0.0), G - 1.0);
    int x0 = (int)floor(cx), y0 = (int)floor(cy);
    if (x0 > G - 2) x0 = G - 2;
    if (y0 > G - 2) y0 = G - 2;
    const double tx = cx - x0, ty = cy - y0;
    double acc[2] = {0, 0};
    for (int c = 0; c < 2; ++c) {
      const double y00 = __bfloat162float(Y[((long long)y0 * G + x0) * C + c]);
      const double y10 = __bfloat162float(Y[((long long)y0 * G + x0 + 1) * C + c]);
      const double y01 = __bfloat162float(Y[((long long)(y0 + 1) * G + x0) * C + c]);
      const double y11 = __bfloat162float(Y[((long long)(y0 + 1) * G + x0 + 1) * C + c]);
      acc[c] = kScaleV * ((1 - ty) * ((1 - tx) * y00 + tx * y10) + ty * ((1 - tx) * y01 + tx * y11));
    }
    out = make_double2(acc[0], acc[1]);
  }
  v[(long long)j * g.ld + i] = out;
}

inline unsigned nblk(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

// ============================ network host code =========================================

struct ConvLayer {
  int cin, cout, level;   // spatial size G >> level
  bool relu;
  long long woff, boff;   // offsets in the parameter vector (weights, then bias)
};

struct NetImpl {
  int G = 256, B = 8;
  std::vector<ConvLayer> layers;
  long long nparam = 0, nweight = 0;
  float *p = nullptr, *gr = nullptr, *m = nullptr, *v = nullptr;   // FP32 master, grads, Adam moments
  bf16* pb = nullptr;                                              // BF16 weights (first nweight of p)
  bf16* wflip = nullptr;                                           // scratch: flipped weights
  int adam_t = 0;
  // activations and their gradients (index = tensor id)
  std::vector<bf16*> act, grad;
  std::vector<long long> size;      // elements per tensor (batch included)
  float* target = nullptr;          // B x G x G x 2
  float* loss = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
};

namespace {

// Tensor ids of the U-Net.
enum T {
  T_X0, T_E1A, T_E1, T_P1, T_E2A, T_E2, T_P2, T_E3A, T_E3, T_P3, T_B1, T_B2, T_C3, T_D3A, T_D3, T_C2, T_D2A, T_D2,
  T_C1, T_D1A, T_D1, T_OUT, T_COUNT
};
struct TensorShape {
  int level, c;
};
const TensorShape kShapes[T_COUNT] = {
    {0, 16}, {0, 32}, {0, 32}, {1, 32}, {1, 64}, {1, 64}, {2, 64}, {2, 128}, {2, 128}, {3, 128}, {3, 256},
    {3, 256}, {2, 384}, {2, 128}, {2, 128}, {1, 192}, {1, 64}, {1, 64}, {0, 96}, {0, 32}, {0, 32}, {0, 16}};
// conv layers: (input tensor, output tensor, relu)
struct ConvDef {
  int in, out;
  bool relu;
};
const ConvDef kConvs[] = {{T_X0, T_E1A, true},  {T_E1A, T_E1, true},  {T_P1, T_E2A, true},  {T_E2A, T_E2, true},
                          {T_P2, T_E3A, true},  {T_E3A, T_E3, true},  {T_P3, T_B1, true},   {T_B1, T_B2, true},
                          {T_C3, T_D3A, true},  {T_D3A, T_D3, true},  {T_C2, T_D2A, true},  {T_D2A, T_D2, true},
                          {T_C1, T_D1A, true},  {T_D1A, T_D1, true},  {T_D1, T_OUT, false}};
constexpr int kNumConv = sizeof(kConvs) / sizeof(kConvs[0]);

void conv_launch(cudaStream_t s, int B, int H, int W, int Cin, int Cout, const bf16* X, const bf16* Wt,
                 const float* bias, bf16* Y, bool relu) {
  const long long P = (long long)B * H * W;
  note_launch();
  if (Cout % 64 == 0) {
    dim3 gr((unsigned)(P / 64), Cout / 64);
    k_conv3x3<64><<<gr, 128, 0, s>>>(B, H, W, Cin, Cout, X, Wt, bias, Y, relu ? 1 : 0);
  } else if (Cout % 32 == 0) {
    dim3 gr((unsigned)(P / 64), Cout / 32);
    k_conv3x3<32><<<gr, 128, 0, s>>>(B, H, W, Cin, Cout, X, Wt, bias, Y, relu ? 1 : 0);
  } else {
    dim3 gr((unsigned)(P / 64), Cout / 16);
    k_conv3x3<16><<<gr, 128, 0, s>>>(B, H, W, Cin, Cout, X, Wt, bias, Y, relu ? 1 : 0);
  }
}

int hw(const NetImpl* n, int level) { return n->G >> level; }

void forward(NetImpl* n, int B) {
  cudaStream_t s = n->stream;
  auto conv = [&](int k) {
    const ConvLayer& L = n->layers[k];
    const int H = hw(n, L.level);
    conv_launch(s, B, H, H, L.cin, L.cout, n->act[kConvs[k].in], n->pb + L.woff, n->p + L.boff,
                n->act[kConvs[k].out], L.relu);
  };
  auto pool = [&](int src, int dst) {
    const int H = hw(n, kShapes[src].level);
    note_launch();
    k_pool<<<nblk((long long)B * H * H * kShapes[src].c / 4), 256, 0, s>>>(B, H, H, kShapes[src].c, n->act[src],
                                                                          n->act[dst]);
  };
  auto upcat = [&](int u, int sk, int dst) {
    const int H = hw(n, kShapes[dst].level);
    note_launch();
    k_up_concat<<<nblk((long long)B * H * H * kShapes[dst].c), 256, 0, s>>>(B, H, H, kShapes[u].c, kShapes[sk].c,
                                                                           n->act[u], n->act[sk], n->act[dst]);
  };
  conv(0); conv(1); pool(T_E1, T_P1);
  conv(2); conv(3); pool(T_E2, T_P2);
  conv(4); conv(5); pool(T_E3, T_P3);
  conv(6); conv(7);
  upcat(T_B2, T_E3, T_C3); conv(8); conv(9);
  upcat(T_D3, T_E2, T_C2); conv(10); conv(11);
  upcat(T_D2, T_E1, T_C1); conv(12); conv(13);
  conv(14);
}

void backward(NetImpl* n, int B) {
  cudaStream_t s = n->stream;
  auto conv_bwd = [&](int k, bool need_dx) {
    const ConvLayer& L = n->layers[k];
    const int H = hw(n, L.level);
    const int out = kConvs[k].out, in = kConvs[k].in;
    const long long P = (long long)B * H * H;
    if (L.relu) {
      note_launch();
      k_relu_bwd<<<nblk(P * L.cout), 256, 0, s>>>(P * L.cout, n->act[out], n->grad[out]);
    }
    // weight and bias gradients
    const long long target_blocks = 152 * 4;
    const long long tiles = (long long)((L.cin + 31) / 32) * ((L.cout + 31) / 32) * 9;
    long long splits = target_blocks / tiles;
    if (splits < 1) splits = 1;
    long long ppb = (P + splits - 1) / splits;
    ppb = (ppb + 31) / 32 * 32;
    splits = (P + ppb - 1) / ppb;
    dim3 gr((L.cin + 31) / 32, (L.cout + 31) / 32, (unsigned)(9 * splits));
    note_launch();
    k_conv_wgrad<<<gr, dim3(32, 8), 0, s>>>(B, H, H, L.cin, L.cout, n->act[in], n->grad[out], n->gr + L.woff,
                                           n->gr + L.boff, ppb);
    if (need_dx) {
      note_launch();
      k_flip_weights<<<nblk((long long)L.cout * 9 * L.cin), 256, 0, s>>>(L.cin, L.cout, n->pb + L.woff, n->wflip);
      conv_launch(s, B, H, H, L.cout, L.cin, n->grad[out], n->wflip, nullptr, n->grad[in], false);
    }
  };
  auto pool_bwd = [&](int src, int dst) {   // src = pre-pool tensor, dst = pooled
    const int H = hw(n, kShapes[src].level);
    note_launch();
    k_pool_bwd_add<<<nblk((long long)B * H * H * kShapes[src].c), 256, 0, s>>>(B, H, H, kShapes[src].c,
                                                                              n->grad[dst], n->grad[src]);
  };
  auto upcat_bwd = [&](int u, int sk, int dst) {
    const int H = hw(n, kShapes[dst].level);
    note_launch();
    k_up_concat_bwd<<<nblk((long long)B * H * H * kShapes[dst].c), 256, 0, s>>>(
        B, H, H, kShapes[u].c, kShapes[sk].c, n->grad[dst], n->grad[u], n->grad[sk]);
  };
  conv_bwd(14, true);
  conv_bwd(13, true); conv_bwd(12, true); upcat_bwd(T_D2, T_E1, T_C1);
  conv_bwd(11, true); conv_bwd(10, true); upcat_bwd(T_D3, T_E2, T_C2);
  conv_bwd(9, true); conv_bwd(8, true); upcat_bwd(T_B2, T_E3, T_C3);
  conv_bwd(7, true); conv_bwd(6, true); pool_bwd(T_E3, T_P3);
  conv_bwd(5, true); conv_bwd(4, true); pool_bwd(T_E2, T_P2);
  conv_bwd(3, true); conv_bwd(2, true); pool_bwd(T_E1, T_P1);
  conv_bwd(1, true); conv_bwd(0, false);
}

int net_fail(NetImpl* n, int code, const char* msg) {
  n->err = msg;
  return code;
}

}  // namespace

void net_predict_nodes(NetImpl* n, cudaStream_t s, const Layout& g, const double* hcell, const double* A,
                       const double* wind, const double* ocean, const double* vold, double2* v) {
  cudaStream_t keep = n->stream;
  n->stream = s;
  dim3 blk(16, 16), gr((n->G + 15) / 16, (n->G + 15) / 16);
  note_launch();
  k_features<<<gr, blk, 0, s>>>(g.N, n->G, hcell, A, wind, ocean, vold, n->act[T_X0]);
  forward(n, 1);
  dim3 gn((g.n1 + 15) / 16, (g.n1 + 15) / 16);
  note_launch();
  k_prolong_pred<<<gn, blk, 0, s>>>(n->G, kShapes[T_OUT].c, g, n->act[T_OUT], v);
  n->stream = keep;
}

int net_grid(const NetImpl* n) { return n->G; }

}  // namespace svn

using svn::NetImpl;

struct svn_net {
  NetImpl impl;
};

svn::NetImpl* svn_net_impl(svn_net* net) { return net ? &net->impl : nullptr; }

extern "C" {

int svn_net_create(int G, int batch, void* cuda_stream, svn_net** out) {
  using namespace svn;
  if (!out) return SVN_ERR_ARG;
  *out = nullptr;
  if (G < 64 || G > 1024 || (G % 64) != 0 || batch < 1 || batch > 64) return SVN_ERR_ARG;
  svn_net* net = new (std::nothrow) svn_net();
  if (!net) return SVN_ERR_OOM;
  *out = net;
  NetImpl* n = &net->impl;
  n->G = G;
  n->B = batch;
  n->stream = (cudaStream_t)cuda_stream;
  long long off = 0;
  for (int k = 0; k < kNumConv; ++k) {
    ConvLayer L;
    L.cin = kShapes[kConvs[k].in].c;
    L.cout = kShapes[kConvs[k].out].c;
    L.level = kShapes[kConvs[k].out].level;
    L.relu = kConvs[k].relu;
    L.woff = off;
    off += (long long)L.cout * 9 * L.cin;
    n->layers.push_back(L);
  }
  n->nweight = off;
  for (auto& L : n->layers) {
    L.boff = off;
    off += L.cout;
  }
  n->nparam = off;
  auto alloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    return cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  bool ok = alloc((void**)&n->p, sizeof(float) * n->nparam) && alloc((void**)&n->gr, sizeof(float) * n->nparam) &&
            alloc((void**)&n->m, sizeof(float) * n->nparam) && alloc((void**)&n->v, sizeof(float) * n->nparam) &&
            alloc((void**)&n->pb, sizeof(bf16) * n->nweight);
  long long maxw = 0;
  for (auto& L : n->layers) maxw = std::max(maxw, (long long)L.cout * 9 * L.cin);
  ok = ok && alloc((void**)&n->wflip, sizeof(bf16) * maxw);
  n->act.assign(T_COUNT, nullptr);
  n->grad.assign(T_COUNT, nullptr);
  n->size.assign(T_COUNT, 0);
  for (int t = 0; t < T_COUNT && ok; ++t) {
    const long long hwv = (long long)(G >> kShapes[t].level) * (G >> kShapes[t].level);
    n->size[t] = (long long)batch * hwv * kShapes[t].c;
    ok = alloc((void**)&n->act[t], sizeof(bf16) * n->size[t]) && alloc((void**)&n->grad[t], sizeof(bf16) * n->size[t]);
  }
  ok = ok && alloc((void**)&n->target, sizeof(float) * (size_t)batch * G * G * 2) &&
       alloc((void**)&n->loss, sizeof(float) * 4);
  if (!ok) return net_fail(n, SVN_ERR_OOM, "device allocation failed");
  return SVN_OK;
}

int svn_net_destroy(svn_net* net) {
  if (!net) return SVN_ERR_ARG;
  NetImpl* n = &net->impl;
  for (void* q : {(void*)n->p, (void*)n->gr, (void*)n->m, (void*)n->v, (void*)n->pb, (void*)n->wflip,
                  (void*)n->target, (void*)n->loss})
    if (q) cudaFree(q);
  for (auto* q : n->act)
    if (q) cudaFree(q);
  for (auto* q : n->grad)
    if (q) cudaFree(q);
  delete net;
  return SVN_OK;
}

const char* svn_net_last_error(const svn_net* net) { return net ? net->impl.err.c_str() : "NULL net"; }

long long svn_net_num_params(const svn_net* net) { return net ? net->impl.nparam : 0; }

int svn_net_set_params(svn_net* net, const float* host_params, long long n) {
  using namespace svn;
  if (!net || !host_params || n != net->impl.nparam) return SVN_ERR_ARG;
  NetImpl* i = &net->impl;
  if (cudaMemcpyAsync(i->p, host_params, sizeof(float) * n, cudaMemcpyHostToDevice, i->stream) != cudaSuccess)
    return SVN_ERR_CUDA;
  note_launch();
  k_f2bf<<<nblk(i->nweight), 256, 0, i->stream>>>(i->nweight, i->p, i->pb);
  cudaMemsetAsync(i->m, 0, sizeof(float) * n, i->stream);
  cudaMemsetAsync(i->v, 0, sizeof(float) * n, i->stream);
  i->adam_t = 0;
  return cudaStreamSynchronize(i->stream) == cudaSuccess ? SVN_OK : SVN_ERR_CUDA;
}

int svn_net_get_params(svn_net* net, float* host_params, long long n) {
  if (!net || !host_params || n != net->impl.nparam) return SVN_ERR_ARG;
  NetImpl* i = &net->impl;
  if (cudaMemcpyAsync(host_params, i->p, sizeof(float) * n, cudaMemcpyDeviceToHost, i->stream) != cudaSuccess)
    return SVN_ERR_CUDA;
  return cudaStreamSynchronize(i->stream) == cudaSuccess ? SVN_OK : SVN_ERR_CUDA;
}

int svn_net_set_sample(svn_net* net, int slot, int N, const double* h, const double* A, const double* wind,
                       const double* ocean, const double* v_old, const double* v_target) {
  using namespace svn;
  if (!net || !h || !A || !wind || !ocean || !v_old) return SVN_ERR_ARG;
  NetImpl* n = &net->impl;
  if (slot < 0 || slot >= n->B || N < n->G || N % n->G != 0) return net_fail(n, SVN_ERR_ARG, "bad slot or N");
  if (v_target && N != n->G) return net_fail(n, SVN_ERR_ARG, "targets need N == G");
  dim3 blk(16, 16), gr((n->G + 15) / 16, (n->G + 15) / 16);
  note_launch();
  k_features<<<gr, blk, 0, n->stream>>>(N, n->G, h, A, wind, ocean, v_old,
                                        n->act[T_X0] + (long long)slot * n->G * n->G * kCin0);
  if (v_target) {
    note_launch();
    k_target<<<gr, blk, 0, n->stream>>>(N, v_target, n->target + (long long)slot * n->G * n->G * 2);
  }
  return cudaGetLastError() == cudaSuccess ? SVN_OK : SVN_ERR_CUDA;
}

int svn_net_forward(svn_net* net, int nb, float* out_host) {
  using namespace svn;
  if (!net || nb < 1 || nb > net->impl.B) return SVN_ERR_ARG;
  NetImpl* n = &net->impl;
  forward(n, nb);
  if (out_host) {
    const long long cnt = (long long)nb * n->G * n->G * kShapes[T_OUT].c;
    std::vector<bf16> tmp(cnt);
    if (cudaMemcpyAsync(tmp.data(), n->act[T_OUT], sizeof(bf16) * cnt, cudaMemcpyDeviceToHost, n->stream) !=
        cudaSuccess)
      return SVN_ERR_CUDA;
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) return SVN_ERR_CUDA;
    for (long long e = 0; e < cnt; ++e) {
      uint16_t bits;
      memcpy(&bits, &tmp[e], 2);
      uint32_t u = (uint32_t)bits << 16;
      memcpy(&out_host[e], &u, 4);
    }
  }
  return cudaGetLastError() == cudaSuccess ? SVN_OK : SVN_ERR_CUDA;
}

int svn_net_train_step(svn_net* net, int nb, float lr, int apply_update, float* loss_out) {
  using namespace svn;
  if (!net || nb < 1 || nb > net->impl.B) return SVN_ERR_ARG;
  NetImpl* n = &net->impl;
  cudaStream_t s = n->stream;
  forward(n, nb);
  cudaMemsetAsync(n->loss, 0, sizeof(float), s);
  cudaMemsetAsync(n->gr, 0, sizeof(float) * n->nparam, s);
  const long long P = (long long)nb * n->G * n->G;
  note_launch();
  k_mse<<<nblk(P), 256, 0, s>>>(P, kShapes[T_OUT].c, n->act[T_OUT], n->target, n->grad[T_OUT], n->loss);
  backward(n, nb);
  if (apply_update) {
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
    note_launch();
    k_adam<<<nblk(n->nparam), 256, 0, s>>>(n->nparam, lr, b1, b2, 1e-8f, c1, c2, n->p, n->gr, n->m, n->v, n->pb,
                                           n->nweight);
  }
  if (loss_out) {
    if (cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SVN_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return SVN_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? SVN_OK : SVN_ERR_CUDA;
}

int svn_net_get_grads(svn_net* net, float* host, long long n) {
  if (!net || !host || n != net->impl.nparam) return SVN_ERR_ARG;
  NetImpl* i = &net->impl;
  if (cudaMemcpyAsync(host, i->gr, sizeof(float) * n, cudaMemcpyDeviceToHost, i->stream) != cudaSuccess)
    return SVN_ERR_CUDA;
  return cudaStreamSynchronize(i->stream) == cudaSuccess ? SVN_OK : SVN_ERR_CUDA;
}

}  // extern "C"
