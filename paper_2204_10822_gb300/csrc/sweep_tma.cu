// TMA-staged two-step Chebyshev-Jacobi sweep for FP32 multigrid levels.
//
// The same two Chebyshev steps as the other two-step kernels (Saad, Alg. 12.1
// on D^-1 A: x1 = x0 + d1, x2 = x1 + d2 with d_{k+1} = c1 d_k + c2 D^-1 (b - A x_k)),
// organised around the Tensor Memory Accelerator.  One CTA of 128 threads owns
// a strip of 124 output columns and a chunk of rows; thread t sits on column
// c0 - 2 + t.  Each row of the level's data -- the 19 stencil planes, the
// three block-Jacobi planes, b, d0 and x0 -- reaches shared memory as one
// box of 132 columns per array (starting at c0 - 4, a 16-byte boundary), so a
// row costs five cp.async.bulk.tensor instructions issued by one thread, and a
// six-stage ring keeps rows q+2 .. q+4 in flight while row q is computed.
// Row q needs stencil rows q-1, q (own, E, N, NE, NW blocks and the
// transposed blocks of its W, S, SW, SE neighbours) and x0 rows q-1 .. q+1
// (step 1); step 2 runs one row behind on x1 rows q-2 .. q, which the CTA
// keeps in a three-row ring.  Out-of-range columns come back from the TMA
// unit as zeros; rows outside the grid are zero-filled by the CTA itself.
//
// Every wait on a stage's mbarrier is bounded: after `polls` failed
// (non-blocking) mbarrier.test_wait polls the
// CTA counts a timeout in a device counter (read by sweep_tma_timeouts), waits
// again (bounded) for the copies it has in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace svn {

namespace {

constexpr int kTT = 128;        // threads per CTA, one column each
constexpr int kTOut = 124;      // output columns per CTA
constexpr int kTBox = 132;      // staged columns per row (from c0 - 4)
constexpr int kTStages = 6;     // ring depth
constexpr int kBytesS = NSTEN * kTBox * 4;
constexpr int kBytesInv = 3 * kTBox * 4;
constexpr int kBytesV = kTBox * 8;
constexpr int align128(int x) { return (x + 127) / 128 * 128; }
constexpr int kOffS = 0;
constexpr int kOffInv = align128(kOffS + kBytesS);
constexpr int kOffB = align128(kOffInv + kBytesInv);
constexpr int kOffD = align128(kOffB + kBytesV);
constexpr int kOffX = align128(kOffD + kBytesV);
constexpr int kStageBytes = align128(kOffX + kBytesV);
constexpr int kOffRing = kTStages * kStageBytes;          // x1 ring, 3 rows x kTT float2
constexpr int kOffBars = kOffRing + 3 * kTT * 8;
constexpr int kSmemBytes = kOffBars + kTStages * 8;
constexpr unsigned kDefaultPolls = 1u << 22;

__device__ unsigned int g_tma_timeouts;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, unsigned polls) {
  for (unsigned k = 0; k < polls; ++k)
    if (mbar_try(a, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* m, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* m, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

struct StageView {
  const float* S;      // [NSTEN][kTBox]
  const float* inv;    // [3][kTBox]
  const float2* b;     // [kTBox]
  const float2* d0;
  const float2* x0;
};

__device__ __forceinline__ StageView stage_view(const unsigned char* st) {
  StageView v;
  v.S = reinterpret_cast<const float*>(st + kOffS);
  v.inv = reinterpret_cast<const float*>(st + kOffInv);
  v.b = reinterpret_cast<const float2*>(st + kOffB);
  v.d0 = reinterpret_cast<const float2*>(st + kOffD);
  v.x0 = reinterpret_cast<const float2*>(st + kOffX);
  return v;
}

// (A x) at one node of row q, staged column c: the own, E, N, NE, NW blocks
// from stencil row Sq and the transposed blocks that couple the node to its
// W (E block of column c - 1), S, SW and SE neighbours (N, NE, NW blocks of
// row Sm = q - 1).  X(dr, dc) returns x at row q + dr, column c + dc.
template <typename XF>
__device__ __forceinline__ void row_apply(const float* __restrict__ Sq, const float* __restrict__ Sm, int c, XF X,
                                          float& yx, float& yy) {
  auto at = [&](const float* S, int k, int col) { return S[k * kTBox + col]; };
  const float2 xc = X(0, 0);
  yx = at(Sq, S_D, c) * xc.x;
  yx = fmaf(at(Sq, S_D + 1, c), xc.y, yx);
  yy = at(Sq, S_D + 1, c) * xc.x;
  yy = fmaf(at(Sq, S_D + 2, c), xc.y, yy);
  auto fwd = [&](int slot, float2 xq) {
    const float b0 = at(Sq, slot, c), b1 = at(Sq, slot + 1, c), b2 = at(Sq, slot + 2, c), b3 = at(Sq, slot + 3, c);
    yx = fmaf(b0, xq.x, yx);
    yx = fmaf(b1, xq.y, yx);
    yy = fmaf(b2, xq.x, yy);
    yy = fmaf(b3, xq.y, yy);
  };
  auto bwd = [&](const float* S, int slot, int col, float2 xq) {
    const float b0 = at(S, slot, col), b1 = at(S, slot + 1, col), b2 = at(S, slot + 2, col),
                b3 = at(S, slot + 3, col);
    yx = fmaf(b0, xq.x, yx);
    yx = fmaf(b2, xq.y, yx);
    yy = fmaf(b1, xq.x, yy);
    yy = fmaf(b3, xq.y, yy);
  };
  fwd(S_E, X(0, 1));
  fwd(S_N, X(1, 0));
  fwd(S_NE, X(1, 1));
  fwd(S_NW, X(1, -1));
  bwd(Sq, S_E, c - 1, X(0, -1));
  bwd(Sm, S_N, c, X(-1, 0));
  bwd(Sm, S_NE, c - 1, X(-1, -1));
  bwd(Sm, S_NW, c + 1, X(-1, 1));
}

// kPower: x1 = D^-1 A x0, x2 = D^-1 A x1 (power iteration, no b or d).
// have_x0 == 0: start from x0 = d0 = 0 (the first pre-smoothing pass).
template <bool kPower>
__global__ void __launch_bounds__(kTT) k_cheb_sweep2t(
    Layout g, const __grid_constant__ CUtensorMap mS, const __grid_constant__ CUtensorMap mInv,
    const __grid_constant__ CUtensorMap mB, const __grid_constant__ CUtensorMap mD0,
    const __grid_constant__ CUtensorMap mX0, int have_x0, const float* __restrict__ coef, int step,
    float2* __restrict__ x2, float2* __restrict__ d2, int rows, int nstrips, unsigned polls) {
  extern __shared__ __align__(1024) unsigned char sm[];
  float2* ring = reinterpret_cast<float2*>(sm + kOffRing);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBars);
  const int t = threadIdx.x;
  const int strip = blockIdx.x % nstrips, chunk = blockIdx.x / nstrips;
  const int j_lo = chunk * rows;
  if (j_lo > g.N) return;   // uniform over the CTA
  const int j_hi = min(j_lo + rows, g.N + 1);
  const int c0 = strip * kTOut;
  const int i = c0 - 2 + t;          // this thread's column
  const int c = t + 2;               // its staged column
  const int xbox = c0 - 4;           // multiple of 4: 16-byte aligned box start
  const int r0 = j_lo - 3, r_last = j_hi + 1;
  const bool load_d = !kPower && have_x0;
  const bool load_x = kPower || have_x0;
  const uint32_t tx = kBytesS + kBytesInv + (kPower ? 0 : kBytesV) + (load_d ? kBytesV : 0) + (load_x ? kBytesV : 0);
  const float c1a = kPower ? 0.f : coef[2 * step], c2a = kPower ? 0.f : coef[2 * step + 1];
  const float c1b = kPower ? 0.f : coef[2 * step + 2], c2b = kPower ? 0.f : coef[2 * step + 3];
  const float2 zero = make_float2(0.f, 0.f);

  if (t == 0) {
    for (int s = 0; s < kTStages; ++s) mbar_init(saddr(&bars[s]));
    asm volatile("fence.mbarrier_init.release.cluster;\n fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  auto slot_of = [&](int r) { return (r - r0) % kTStages; };
  auto parity_of = [&](int r) { return (uint32_t)(((r - r0) / kTStages) & 1); };
  auto stage = [&](int r) { return sm + slot_of(r) * kStageBytes; };
  // Bring row r into its ring slot (all threads call it with the same r).
  auto prefetch = [&](int r) {
    if (r > r_last) return;
    unsigned char* st = stage(r);
    const uint32_t bar = saddr(&bars[slot_of(r)]);
    if (r >= 0 && r <= g.N) {
      if (t == 0) {
        mbar_expect_tx(bar, tx);
        tma_3d(saddr(st + kOffS), &mS, xbox, r, 0, bar);
        tma_3d(saddr(st + kOffInv), &mInv, xbox, r, 0, bar);
        if (!kPower) tma_2d(saddr(st + kOffB), &mB, xbox, r, bar);
        if (load_d) tma_2d(saddr(st + kOffD), &mD0, xbox, r, bar);
        if (load_x) tma_2d(saddr(st + kOffX), &mX0, xbox, r, bar);
      }
    } else {
      uint4* p = reinterpret_cast<uint4*>(st);
      for (int k = t; k < kStageBytes / 16; k += kTT) p[k] = make_uint4(0u, 0u, 0u, 0u);
      __syncthreads();
      if (t == 0) mbar_arrive(bar);
    }
  };
  bool failed = false;
  auto wait_row = [&](int r) {
    const bool ok = mbar_wait(saddr(&bars[slot_of(r)]), parity_of(r), polls);
    failed = __syncthreads_or(!ok) != 0;
  };

  for (int r = r0; r < r0 + kTStages; ++r) prefetch(r);
  int waited = r0 - 1;   // rows r0 .. waited have landed
  for (int r = r0; r <= r0 + 2 && !failed; ++r) {
    wait_row(r);
    waited = r;
  }

  float2 d1p = zero;   // d1 at this thread's node of the previous row
  for (int q = j_lo - 1; q <= j_hi && !failed; ++q) {
    wait_row(q + 1);
    if (failed) break;
    waited = q + 1;
    // step 1 at row q
    const StageView Vq = stage_view(stage(q)), Vm = stage_view(stage(q - 1)), Vp = stage_view(stage(q + 1));
    float2 x1 = zero, d1 = zero;
    if (t >= 1 && t <= kTT - 2 && i >= 1 && i <= g.N - 1 && q >= 1 && q <= g.N - 1) {
      float yx, yy;
      auto X0 = [&](int dr, int dc) {
        if (!load_x) return zero;
        const float2* xr = dr < 0 ? Vm.x0 : dr > 0 ? Vp.x0 : Vq.x0;
        return xr[c + dc];
      };
      row_apply(Vq.S, Vm.S, c, X0, yx, yy);
      const float i00 = Vq.inv[c], i01 = Vq.inv[kTBox + c], i11 = Vq.inv[2 * kTBox + c];
      if constexpr (kPower) {
        x1 = make_float2(i00 * yx + i01 * yy, i01 * yx + i11 * yy);
      } else {
        const float2 bb = Vq.b[c];
        const float rx = bb.x - yx, ry = bb.y - yy;
        const float2 dd = load_d ? Vq.d0[c] : zero;
        const float2 xx = load_x ? Vq.x0[c] : zero;
        d1 = make_float2(c1a * dd.x + c2a * (i00 * rx + i01 * ry), c1a * dd.y + c2a * (i01 * rx + i11 * ry));
        x1 = make_float2(xx.x + d1.x, xx.y + d1.y);
      }
    }
    ring[((q + 3) % 3) * kTT + t] = x1;
    __syncthreads();
    // step 2 at row p = q - 1
    const int p = q - 1;
    if (p >= j_lo && t >= 2 && t <= kTT - 3 && i <= g.N) {
      float2 out = zero;
      if (i >= 1 && i <= g.N - 1 && p >= 1 && p <= g.N - 1) {
        float yx, yy;
        auto X1 = [&](int dr, int dc) { return ring[((p + dr + 3) % 3) * kTT + t + dc]; };
        row_apply(Vm.S, stage_view(stage(p - 1)).S, c, X1, yx, yy);
        const float i00 = Vm.inv[c], i01 = Vm.inv[kTBox + c], i11 = Vm.inv[2 * kTBox + c];
        const float2 x1o = X1(0, 0);
        const long long np = (long long)p * g.ld + i;
        if constexpr (kPower) {
          out = make_float2(i00 * yx + i01 * yy, i01 * yx + i11 * yy);
        } else {
          const float2 bb = Vm.b[c];
          const float rx = bb.x - yx, ry = bb.y - yy;
          const float2 dd = make_float2(c1b * d1p.x + c2b * (i00 * rx + i01 * ry),
                                        c1b * d1p.y + c2b * (i01 * rx + i11 * ry));
          d2[np] = dd;
          out = make_float2(x1o.x + dd.x, x1o.y + dd.y);
        }
      }
      x2[(long long)p * g.ld + i] = out;
    }
    d1p = d1;
    __syncthreads();          // every read of row q - 2's slot is done
    prefetch(q + kTStages - 2);
  }
  if (failed) {
    // count the timeout, then wait (bounded) for the copies still in flight
    if (t == 0) {
      atomicAdd(&g_tma_timeouts, 1u);
      // rows issued so far: the first kTStages, then row q + 3 by every finished iteration q - 1
      const int issued = min(r_last, max(r0 + kTStages - 1, waited + 3));
      for (int r = waited + 1; r <= issued; ++r) mbar_wait(saddr(&bars[slot_of(r)]), parity_of(r), kDefaultPolls);
    }
    __syncthreads();
  }
}

// ---- host side ---------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    cudaGetLastError();
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

struct MapKey {
  const void* ptr;
  int n1, ld, planes, esize;
  long long plane;
  bool operator==(const MapKey& o) const {
    return ptr == o.ptr && n1 == o.n1 && ld == o.ld && planes == o.planes && esize == o.esize && plane == o.plane;
  }
};

// Tensor map of `planes` planes of one level's node layout (x = column, y = row,
// z = plane), box kTBox x 1 x planes; cached per buffer (the buffers live as
// long as their handle and keep their layout).
bool tensor_map(const void* ptr, const Layout& g, int planes, int esize, CUtensorMap* out) {
  static std::mutex mu;
  static std::vector<std::pair<MapKey, CUtensorMap>> cache;
  const MapKey key{ptr, g.n1, g.ld, planes, esize, g.plane};
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : cache)
    if (e.first == key) {
      *out = e.second;
      return true;
    }
  auto fn = encode_fn();
  if (!fn) return false;
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[3] = {(cuuint64_t)g.n1, (cuuint64_t)g.n1, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)g.ld * esize, (cuuint64_t)g.plane * esize};
  const cuuint32_t box[3] = {(cuuint32_t)kTBox, 1u, (cuuint32_t)planes};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_INT64;
  const cuuint32_t rank = planes > 1 ? 3u : 2u;
  const CUresult r = fn(&m, dt, rank, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  if (cache.size() > 4096) cache.clear();
  cache.push_back({key, m});
  *out = m;
  return true;
}

template <bool kPower>
int resident_ctas() {
  static int n = []() {
    int dev = 0, sms = 152, bps = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    if (cudaFuncSetAttribute(k_cheb_sweep2t<kPower>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_cheb_sweep2t<kPower>, kTT, kSmemBytes) !=
            cudaSuccess ||
        bps < 1)
      bps = 0;
    cudaGetLastError();
    return sms * bps;
  }();
  return n;
}

}  // namespace

bool launch_cheb_sweep2_tma(cudaStream_t s, const Layout& g, const float* st, const float* dinv, const float* coef,
                            int step, const float2* x0, float2* x2, const float2* d0, float2* d2, const float2* b,
                            bool power, unsigned polls) {
  const int res = power ? resident_ctas<true>() : resident_ctas<false>();
  if (res < 1) return false;
  CUtensorMap mS, mInv, mB, mD, mX;
  if (!tensor_map(st, g, NSTEN, 4, &mS) || !tensor_map(dinv, g, 3, 4, &mInv)) return false;
  mB = mD = mX = mS;   // unused maps (no copies are issued through them)
  if (!power && (!b || !tensor_map(b, g, 1, 8, &mB))) return false;
  const bool have_x0 = x0 != nullptr;
  if (have_x0 && !tensor_map(x0, g, 1, 8, &mX)) return false;
  if (!power && have_x0 && (!d0 || !tensor_map(d0, g, 1, 8, &mD))) return false;
  const int nstrips = (g.n1 + kTOut - 1) / kTOut;
  const int target_chunks = std::max(1, res / nstrips);
  const int rows = std::max(8, (g.n1 + target_chunks - 1) / target_chunks);
  const int chunks = (g.n1 + rows - 1) / rows;
  const unsigned blocks = (unsigned)(nstrips * chunks);
  const unsigned pl = polls ? polls : kDefaultPolls;
  note_launch();
  if (power)
    k_cheb_sweep2t<true><<<blocks, kTT, kSmemBytes, s>>>(g, mS, mInv, mB, mD, mX, 1, nullptr, 0, x2, nullptr, rows,
                                                         nstrips, pl);
  else
    k_cheb_sweep2t<false><<<blocks, kTT, kSmemBytes, s>>>(g, mS, mInv, mB, mD, mX, have_x0 ? 1 : 0, coef, step, x2,
                                                          d2, rows, nstrips, pl);
  return true;
}

int sweep_tma_timeouts(cudaStream_t s, unsigned* pinned, bool reset) {
  if (cudaMemcpyFromSymbolAsync(pinned, g_tma_timeouts, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  const int n = (int)*pinned;
  if (reset && n) {
    *pinned = 0;
    if (cudaMemcpyToSymbolAsync(g_tma_timeouts, pinned, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return -1;
  }
  return n;
}

}  // namespace svn
