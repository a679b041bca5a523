// Per-cell FP64 kernels of the svN step on Q2 (biquadratic) velocity elements.
//
// The paper's method does not depend on the discretisation (Section 5.1; the
// Problem II discussion of Section 5.3 shows quadratic velocity elements).
// Here each of the N x N cells carries the 9 Lagrange nodes of the
// tensor-product quadratic basis; the velocity lives on the (2N+1)^2 node grid
// of spacing dx/2, stored in the padded node layout of a 2N grid (node (I, J)
// at J ld + I).  H and A are constant per cell (cell c = j N + i); every
// integral uses 3 x 3 Gauss points per cell, so R is the exact gradient of the
// discrete energy as for Q1.  Quadrature fields are planes of `cpl` entries
// indexed by the cell.
//
// Basis tables (values and hat derivatives of the 9 local functions at the 9
// points, and the points' weights on the unit square) sit in constant memory,
// written once per device by q2_init_tables.
#include <cmath>

#include "kernels.h"

namespace svn {

namespace {

__constant__ double c_N9[9][9];    // [q][n] value of local function n at point q
__constant__ double c_DX9[9][9];   // d/dxi (hat units)
__constant__ double c_DY9[9][9];   // d/deta
__constant__ double c_W9[9];       // weight on the unit square (sum 1)

const dim3 kQBlk(32, 4);
inline dim3 q2_cell_grid(int N) { return dim3((N + kQBlk.x - 1) / kQBlk.x, (N + kQBlk.y - 1) / kQBlk.y); }
inline dim3 q2_node_grid(int n1) { return dim3((n1 + kQBlk.x - 1) / kQBlk.x, (n1 + kQBlk.y - 1) / kQBlk.y); }

__device__ __forceinline__ long long q2_node(const Layout& gq, int i, int j, int n) {
  return (long long)(2 * j + n / 3) * gq.ld + 2 * i + n % 3;
}

struct Q2Loc {
  double x[9], y[9];
};

__device__ __forceinline__ void q2_load(const double2* __restrict__ v, const Layout& gq, int i, int j, Q2Loc& L) {
#pragma unroll
  for (int n = 0; n < 9; ++n) {
    const double2 a = v[q2_node(gq, i, j, n)];
    L.x[n] = a.x;
    L.y[n] = a.y;
  }
}

struct Q2Qp {
  double vx, vy, gxx, gxy, gyx, gyy;   // value and hat gradient g[k][d]
};

__device__ __forceinline__ Q2Qp q2_eval(int q, const Q2Loc& L) {
  Q2Qp p{0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int n = 0; n < 9; ++n) {
    const double N = c_N9[q][n], dx = c_DX9[q][n], dy = c_DY9[q][n];
    p.vx = fma(N, L.x[n], p.vx);
    p.vy = fma(N, L.y[n], p.vy);
    p.gxx = fma(dx, L.x[n], p.gxx);
    p.gxy = fma(dy, L.x[n], p.gxy);
    p.gyx = fma(dx, L.y[n], p.gyx);
    p.gyy = fma(dy, L.y[n], p.gyy);
  }
  return p;
}

// true-unit tau components (xx, yy, xy) from the hat gradient
__device__ __forceinline__ void q2_tau(const Phys& ph, const Q2Qp& p, double& txx, double& tyy, double& txy) {
  txx = (ph.ta * p.gxx + ph.tb * p.gyy) * ph.idx;
  tyy = (ph.tb * p.gxx + ph.ta * p.gyy) * ph.idx;
  txy = ph.tc * (p.gxy + p.gyx) * ph.idx;
}

// ---- a1: precomputation ------------------------------------------------------------
__global__ void k_q2_precompute(int N, Layout gq, long long cpl, double dt, PhysConst pc,
                                const double* __restrict__ hcell, const double* __restrict__ A,
                                const double* __restrict__ wind, const double* __restrict__ ocean,
                                const double* __restrict__ vold, double* __restrict__ P, double* __restrict__ rhoH,
                                double* __restrict__ fq, double* __restrict__ voq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const long long c = (long long)j * N + i;
  const double h = hcell[c], a = A[c];
  const double Pc = pc.Pstar * h * exp(-pc.C * (1.0 - a));   // Eq. "ice-strength"
  const double rh = pc.rho_ice * h;
  P[c] = Pc;
  rhoH[c] = rh;
  const int n1 = 2 * N + 1;
  Q2Loc wd, oc, vn;
#pragma unroll
  for (int n = 0; n < 9; ++n) {
    const int I = 2 * i + n % 3, J = 2 * j + n / 3;
    const long long k = 2 * ((long long)J * n1 + I);
    const bool bnd = I == 0 || J == 0 || I == n1 - 1 || J == n1 - 1;
    wd.x[n] = wind[k];
    wd.y[n] = wind[k + 1];
    oc.x[n] = ocean[k];
    oc.y[n] = ocean[k + 1];
    vn.x[n] = bnd ? 0.0 : vold[k];
    vn.y[n] = bnd ? 0.0 : vold[k + 1];
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    double vax = 0, vay = 0, vox = 0, voy = 0, vnx = 0, vny = 0;
#pragma unroll
    for (int n = 0; n < 9; ++n) {
      const double s = c_N9[q][n];
      vax = fma(s, wd.x[n], vax);
      vay = fma(s, wd.y[n], vay);
      vox = fma(s, oc.x[n], vox);
      voy = fma(s, oc.y[n], voy);
      vnx = fma(s, vn.x[n], vnx);
      vny = fma(s, vn.y[n], vny);
    }
    // tau_atm = Ca rho_a |v_a| v_a (Eq. "force"); explicit Coriolis rho H f e_r x (v^n - v_o)
    const double sa = pc.Ca * pc.rho_a * sqrt(vax * vax + vay * vay);
    const double dwx = vnx - vox, dwy = vny - voy;
    const double corx = -rh * pc.f_c * dwy, cory = rh * pc.f_c * dwx;
    fq[(2 * q) * cpl + c] = -rh * vnx + dt * corx - dt * sa * vax;
    fq[(2 * q + 1) * cpl + c] = -rh * vny + dt * cory - dt * sa * vay;
    voq[(2 * q) * cpl + c] = vox;
    voq[(2 * q + 1) * cpl + c] = voy;
  }
}

// pi_0 = tau(v) / Delta(v) at the 9 points (Eq. "pi"), components (xx, yy, xy).
__global__ void k_q2_pi_init(int N, Layout gq, long long cpl, Phys ph, const double2* __restrict__ v,
                             double* __restrict__ pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const long long c = (long long)j * N + i;
  Q2Loc L;
  q2_load(v, gq, i, j, L);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const Q2Qp p = q2_eval(q, L);
    double txx, tyy, txy;
    q2_tau(ph, p, txx, tyy, txy);
    const double inv = rsqrt(ph.dmin2 + 2.0 * (txx * txx + tyy * tyy + 2.0 * txy * txy));
    pi[(3 * q) * cpl + c] = txx * inv;
    pi[(3 * q + 1) * cpl + c] = tyy * inv;
    pi[(3 * q + 2) * cpl + c] = txy * inv;
  }
}

// ---- a2: residual, per cell: the 18 local contributions to eb -------------------------
//   R_(n,k) = sum_q w_q [ N_n s_k + Fxx dN/dx + Fxy dN/dy  (k = x) | Fxy dN/dx + Fyy dN/dy  (k = y) ]
// with s = rho H v + fq - dt Co rho_o |w| w, S = dt P tau(v) / Delta,
// F = (ta Sxx + tb Syy - dt P/2, tb Sxx + ta Syy - dt P/2, 2 tc Sxy).
__global__ void k_q2_residual_cells(int N, Layout gq, long long cpl, Phys ph, const double2* __restrict__ v,
                                    const double* __restrict__ P, const double* __restrict__ rhoH,
                                    const double* __restrict__ fq, const double* __restrict__ voq,
                                    double* __restrict__ eb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const long long c = (long long)j * N + i;
  Q2Loc L;
  q2_load(v, gq, i, j, L);
  const double Pdt = ph.dt * P[c];
  const double rh = rhoH[c];
  const double w2 = ph.dx * ph.dx;    // cell area: weights are w2 c_W9[q]
  double rx[9], ry[9];
#pragma unroll
  for (int n = 0; n < 9; ++n) rx[n] = ry[n] = 0.0;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const Q2Qp p = q2_eval(q, L);
    double txx, tyy, txy;
    q2_tau(ph, p, txx, tyy, txy);
    const double inv = rsqrt(ph.dmin2 + 2.0 * (txx * txx + tyy * tyy + 2.0 * txy * txy));
    const double sf = Pdt * inv;
    const double Sxx = sf * txx, Syy = sf * tyy, Sxy = sf * txy;
    const double wq = w2 * c_W9[q];
    const double gw = wq * ph.idx;     // weight for hat derivatives
    const double Gxx = gw * (ph.ta * Sxx + ph.tb * Syy - 0.5 * Pdt);
    const double Gyy = gw * (ph.tb * Sxx + ph.ta * Syy - 0.5 * Pdt);
    const double Gxy = gw * (2.0 * ph.tc * Sxy);
    const double wx = voq[(2 * q) * cpl + c] - p.vx;
    const double wy = voq[(2 * q + 1) * cpl + c] - p.vy;
    const double dr = ph.dt * ph.cdrag * sqrt(wx * wx + wy * wy);
    const double sx = wq * (rh * p.vx + fq[(2 * q) * cpl + c] - dr * wx);
    const double sy = wq * (rh * p.vy + fq[(2 * q + 1) * cpl + c] - dr * wy);
#pragma unroll
    for (int n = 0; n < 9; ++n) {
      const double Nn = c_N9[q][n], dx = c_DX9[q][n], dy = c_DY9[q][n];
      rx[n] = fma(Nn, sx, rx[n]);
      rx[n] = fma(dx, Gxx, rx[n]);
      rx[n] = fma(dy, Gxy, rx[n]);
      ry[n] = fma(Nn, sy, ry[n]);
      ry[n] = fma(dx, Gxy, ry[n]);
      ry[n] = fma(dy, Gyy, ry[n]);
    }
  }
#pragma unroll
  for (int n = 0; n < 9; ++n) {
    eb[(2 * n) * cpl + c] = rx[n];
    eb[(2 * n + 1) * cpl + c] = ry[n];
  }
}

// Node gather of the 18 per-cell planes of eb: node (I, J) collects the cells
// whose local node (a, b) it is (a vertex up to 4 cells, an edge node 2, a
// centre 1); boundary nodes are 0.  With `partial`, per-block sums of |y|^2.
__global__ void k_q2_gather(int N, Layout gq, long long cpl, const double* __restrict__ eb, double2* __restrict__ y,
                            double* __restrict__ partial) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int n1 = 2 * N + 1;
  double s = 0.0;
  if (I < n1 && J < n1) {
    double2 r = make_double2(0.0, 0.0);
    if (I >= 1 && J >= 1 && I <= n1 - 2 && J <= n1 - 2) {
      int ci[2], ca[2], cj[2], cb[2], nx = 0, ny = 0;
      if (I & 1) {
        ci[nx] = I >> 1; ca[nx++] = 1;
      } else {
        if ((I >> 1) - 1 >= 0) { ci[nx] = (I >> 1) - 1; ca[nx++] = 2; }
        if ((I >> 1) < N) { ci[nx] = I >> 1; ca[nx++] = 0; }
      }
      if (J & 1) {
        cj[ny] = J >> 1; cb[ny++] = 1;
      } else {
        if ((J >> 1) - 1 >= 0) { cj[ny] = (J >> 1) - 1; cb[ny++] = 2; }
        if ((J >> 1) < N) { cj[ny] = J >> 1; cb[ny++] = 0; }
      }
      for (int u = 0; u < ny; ++u)
        for (int t = 0; t < nx; ++t) {
          const long long c = (long long)cj[u] * N + ci[t];
          const int n = 3 * cb[u] + ca[t];
          r.x += eb[(2 * n) * cpl + c];
          r.y += eb[(2 * n + 1) * cpl + c];
        }
      s = r.x * r.x + r.y * r.y;
    }
    y[(long long)J * gq.ld + I] = r;
  }
  if (partial) {
    s = block_sum(s);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// ---- a8: energy for k step lengths (compensated sums, as the Q1 kernel) -------------
__global__ void __launch_bounds__(128) k_q2_energy_cells(int N, Layout gq, long long cpl, Phys ph, int k,
                                                         AlphaSet al, const double2* __restrict__ v,
                                                         const double2* __restrict__ dv, const double* __restrict__ P,
                                                         const double* __restrict__ rhoH,
                                                         const double* __restrict__ fq,
                                                         const double* __restrict__ voq, double* __restrict__ partial,
                                                         int nblocks) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  DD acc[MAX_ALPHA];
  double asum = 0.0;
#pragma unroll
  for (int a = 0; a < MAX_ALPHA; ++a) acc[a] = DD{0.0, 0.0};
  if (i < N && j < N) {
    const long long c = (long long)j * N + i;
    Q2Loc L0, D0;
    q2_load(v, gq, i, j, L0);
    q2_load(dv, gq, i, j, D0);
    const double Ph = 0.5 * ph.dt * P[c];
    const double rh = rhoH[c];
    const double w2 = ph.dx * ph.dx;
    for (int a = 0; a < k; ++a) {
      const double al0 = al.a[a];
      Q2Loc L;
#pragma unroll
      for (int n = 0; n < 9; ++n) {
        L.x[n] = fma(al0, D0.x[n], L0.x[n]);
        L.y[n] = fma(al0, D0.y[n], L0.y[n]);
      }
      double csum = 0.0;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const Q2Qp p = q2_eval(q, L);
        double txx, tyy, txy;
        q2_tau(ph, p, txx, tyy, txy);
        const double Dl = sqrt(ph.dmin2 + 2.0 * (txx * txx + tyy * tyy + 2.0 * txy * txy));
        const double tr = (p.gxx + p.gyy) * ph.idx;
        const double wx = voq[(2 * q) * cpl + c] - p.vx;
        const double wy = voq[(2 * q + 1) * cpl + c] - p.vy;
        const double nw = sqrt(wx * wx + wy * wy);
        const double wq = w2 * c_W9[q];
        const double t1 = wq * 0.5 * rh * (p.vx * p.vx + p.vy * p.vy);
        const double t2 = wq * (fq[(2 * q) * cpl + c] * p.vx + fq[(2 * q + 1) * cpl + c] * p.vy);
        const double t3 = wq * Ph * (Dl - tr);
        const double t4 = wq * ph.dt * ph.cdrag * nw * nw * nw * (1.0 / 3.0);
        csum += (t1 + t2) + (t3 + t4);
        if (a == 0) asum += fabs(t1) + fabs(t2) + fabs(t3) + fabs(t4);
      }
      acc[a].add(csum);   // plain sum within the cell, compensated over cells
    }
  }
  __shared__ double sh_hi[128], sh_lo[128];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  for (int a = 0; a < k; ++a) {
    sh_hi[tid] = acc[a].hi;
    sh_lo[tid] = acc[a].lo;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) {
        DD x{sh_hi[tid], sh_lo[tid]};
        x.add(DD{sh_hi[tid + s], sh_lo[tid + s]});
        sh_hi[tid] = x.hi;
        sh_lo[tid] = x.lo;
      }
      __syncthreads();
    }
    if (tid == 0) {
      partial[(2 * a) * nblocks + bid] = sh_hi[0];
      partial[(2 * a + 1) * nblocks + bid] = sh_lo[0];
    }
    __syncthreads();
  }
  asum = block_sum(asum);
  if (tid == 0) partial[(2 * MAX_ALPHA) * nblocks + bid] = asum;
}

// ---- a3/a4: element matrices ---------------------------------------------------------
// K_e[(n,k)][(m,l)] = sum_q w_q [ (rho H delta_kl + O_kl) N_n N_m + t_nk^T C t_ml ]
// with the svN coefficient C = dt [ (P/Delta) I - P/(Delta^2 m) (t p^T + p t^T) ]
// (Eq. "linearSVNewton" with Eq. "modification", Voigt form, m = max(1, sqrt(2 pi:pi))),
// O = dt Co rho_o (|w| I + w w^T/|w|) (Eq. "standardNewton2"; rank-one term dropped for
// |w| < 1e-14), and t_n0 = (ta N_x, tb N_x, sqrt2 tc N_y), t_n1 = (tb N_y, ta N_y,
// sqrt2 tc N_x) the Voigt tau of the basis functions.  Upper triangle of the 18 x 18
// matrix over local dofs d = 2 n + k, row-major, in 171 planes.
__device__ __forceinline__ int elem18(int r, int s) { return r * 18 - r * (r - 1) / 2 + (s - r); }

__global__ void __launch_bounds__(128) k_q2_element_matrices(int N, Layout gq, long long cpl, Phys ph,
                                                             const double2* __restrict__ v,
                                                             const double* __restrict__ pi,
                                                             const double* __restrict__ P,
                                                             const double* __restrict__ rhoH,
                                                             const double* __restrict__ voq, double* __restrict__ ke) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const long long c = (long long)j * N + i;
  Q2Loc L;
  q2_load(v, gq, i, j, L);
  const double Pc = P[c], rh = rhoH[c];
  const double sq2 = 1.4142135623730950488;
  const double w2 = ph.dx * ph.dx;
  // per point: C (hat-unit scaled: C idx^2 w_q), the mass-like 2x2 tensor (rho H I + O) w_q
  double C00[9], C01[9], C02[9], C11[9], C12[9], C22[9], M00[9], M01[9], M11[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const Q2Qp p = q2_eval(q, L);
    double txx, tyy, txy;
    q2_tau(ph, p, txx, tyy, txy);
    const double t0 = txx, t1 = tyy, t2 = sq2 * txy;
    const double inv = rsqrt(ph.dmin2 + 2.0 * (t0 * t0 + t1 * t1 + t2 * t2));
    const double p0 = pi[(3 * q) * cpl + c], p1 = pi[(3 * q + 1) * cpl + c];
    const double p2 = sq2 * pi[(3 * q + 2) * cpl + c];
    const double pp = 2.0 * (p0 * p0 + p1 * p1 + p2 * p2);
    const double invm = pp > 1.0 ? rsqrt(pp) : 1.0;      // 1 / max(1, sqrt(2 pi:pi))
    const double wq = w2 * c_W9[q];
    const double sc = wq * ph.idx * ph.idx;              // hat derivatives carry 1/dx each
    const double a = sc * ph.dt * Pc * inv;
    const double b = sc * ph.dt * Pc * inv * inv * invm;
    C00[q] = a - 2.0 * b * t0 * p0;
    C11[q] = a - 2.0 * b * t1 * p1;
    C22[q] = a - 2.0 * b * t2 * p2;
    C01[q] = -b * (t0 * p1 + p0 * t1);
    C02[q] = -b * (t0 * p2 + p0 * t2);
    C12[q] = -b * (t1 * p2 + p1 * t2);
    const double wx = voq[(2 * q) * cpl + c] - p.vx;
    const double wy = voq[(2 * q + 1) * cpl + c] - p.vy;
    // |w| and od / |w| from one reciprocal square root (no sqrt and division)
    const double w2 = wx * wx + wy * wy;
    const double iw = w2 > 0.0 ? rsqrt(w2) : 0.0;
    const double nw = w2 * iw;
    const double od = ph.dt * ph.cdrag;
    double mxx = rh + od * nw, myy = rh + od * nw, mxy = 0.0;
    if (nw >= 1e-14) {
      const double r1 = od * iw;
      mxx += r1 * wx * wx;
      myy += r1 * wy * wy;
      mxy = r1 * wx * wy;
    }
    M00[q] = wq * mxx;
    M01[q] = wq * mxy;
    M11[q] = wq * myy;
  }
  const double ta = ph.ta, tb = ph.tb, s2 = sq2 * ph.tc;
  for (int r = 0; r < 18; ++r) {
    const int n = r >> 1, k = r & 1;
    for (int s = r; s < 18; ++s) {
      const int m = s >> 1, l = s & 1;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const double nx = c_DX9[q][n], ny = c_DY9[q][n], mx = c_DX9[q][m], my = c_DY9[q][m];
        // Voigt tau of the two basis functions (hat units)
        const double u0 = k ? tb * ny : ta * nx, u1 = k ? ta * ny : tb * nx, u2 = k ? s2 * nx : s2 * ny;
        const double z0 = l ? tb * my : ta * mx, z1 = l ? ta * my : tb * mx, z2 = l ? s2 * mx : s2 * my;
        const double Cz0 = C00[q] * z0 + C01[q] * z1 + C02[q] * z2;
        const double Cz1 = C01[q] * z0 + C11[q] * z1 + C12[q] * z2;
        const double Cz2 = C02[q] * z0 + C12[q] * z1 + C22[q] * z2;
        acc = fma(u0, Cz0, acc);
        acc = fma(u1, Cz1, acc);
        acc = fma(u2, Cz2, acc);
        const double Mkl = k == l ? (k ? M11[q] : M00[q]) : M01[q];
        acc = fma(Mkl * c_N9[q][n], c_N9[q][m], acc);
      }
      ke[(long long)elem18(r, s) * cpl + c] = acc;
    }
  }
}

// y_e = K_e x_e per cell into the 18 planes of eb (then gathered to nodes).
__global__ void __launch_bounds__(128) k_q2_apply_cells(int N, Layout gq, long long cpl,
                                                        const double* __restrict__ ke,
                                                        const double2* __restrict__ x, double* __restrict__ eb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const long long c = (long long)j * N + i;
  Q2Loc L;
  q2_load(x, gq, i, j, L);
  double xe[18], ye[18];
#pragma unroll
  for (int n = 0; n < 9; ++n) {
    xe[2 * n] = L.x[n];
    xe[2 * n + 1] = L.y[n];
  }
#pragma unroll
  for (int r = 0; r < 18; ++r) ye[r] = 0.0;
#pragma unroll
  for (int r = 0; r < 18; ++r) {
#pragma unroll
    for (int s = r; s < 18; ++s) {
      const double kv = ke[(long long)elem18(r, s) * cpl + c];
      ye[r] = fma(kv, xe[s], ye[r]);
      if (s != r) ye[s] = fma(kv, xe[r], ye[s]);
    }
  }
#pragma unroll
  for (int r = 0; r < 18; ++r) eb[(long long)r * cpl + c] = ye[r];
}

// ---- a9: dual update at the 9 points (Eq. "tautilde" with Eq. "modification") ----------
__global__ void k_q2_dual_update(int N, Layout gq, long long cpl, Phys ph, double alpha,
                                 const double2* __restrict__ v, const double2* __restrict__ dv,
                                 double* __restrict__ pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const long long c = (long long)j * N + i;
  Q2Loc L, D;
  q2_load(v, gq, i, j, L);
  q2_load(dv, gq, i, j, D);
  const double sq2 = 1.4142135623730950488;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const Q2Qp p = q2_eval(q, L), d = q2_eval(q, D);
    double txx, tyy, txy, sxx, syy, sxy;
    q2_tau(ph, p, txx, tyy, txy);
    q2_tau(ph, d, sxx, syy, sxy);
    const double t0 = txx, t1 = tyy, t2 = sq2 * txy;      // Voigt tau(v)
    const double u0 = sxx, u1 = syy, u2 = sq2 * sxy;      // Voigt tau(dv)
    const double inv = rsqrt(ph.dmin2 + 2.0 * (t0 * t0 + t1 * t1 + t2 * t2));
    const double p0 = pi[(3 * q) * cpl + c], p1 = pi[(3 * q + 1) * cpl + c];
    const double p2 = sq2 * pi[(3 * q + 2) * cpl + c];
    const double pp = 2.0 * (p0 * p0 + p1 * p1 + p2 * p2);
    const double invm = pp > 1.0 ? rsqrt(pp) : 1.0;
    const double tdt = t0 * u0 + t1 * u1 + t2 * u2, pdt = p0 * u0 + p1 * u1 + p2 * u2;
    const double f = inv * inv * invm;
    const double d0 = -p0 + (t0 + u0) * inv - (tdt * p0 + pdt * t0) * f;
    const double d1 = -p1 + (t1 + u1) * inv - (tdt * p1 + pdt * t1) * f;
    const double d2 = -p2 + (t2 + u2) * inv - (tdt * p2 + pdt * t2) * f;
    pi[(3 * q) * cpl + c] = p0 + alpha * d0;
    pi[(3 * q + 1) * cpl + c] = p1 + alpha * d1;
    pi[(3 * q + 2) * cpl + c] = (p2 + alpha * d2) / sq2;
  }
}

// Caller layout <-> padded node layout for the (2N+1)^2 Q2 nodes is the Q1
// layout of a 2N grid (launch_unpack_nodes / launch_pack_nodes with gq).

// Cell field of the N grid -> the 2N grid (each cell to its four sub-cells).
__global__ void k_q2_refine_cells(int N, const double* __restrict__ src, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= 2 * N || j >= 2 * N) return;
  dst[(long long)j * 2 * N + i] = src[(long long)(j >> 1) * N + (i >> 1)];
}

// Block-Jacobi inverse of the Q2 operator: the 2x2 diagonal block of every
// interior node summed over the cells that contain it (local dof pairs
// (2n, 2n+1) of K_e), inverted; 3 planes (xx, xy, yy) of gq.plane, 0 on the
// boundary.
__global__ void k_q2_dinv(int N, Layout gq, long long cpl, const double* __restrict__ ke, double* __restrict__ dinv) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int n1 = 2 * N + 1;
  if (I >= n1 || J >= n1) return;
  const long long nd = (long long)J * gq.ld + I;
  double i00 = 0.0, i01 = 0.0, i11 = 0.0;
  if (I >= 1 && J >= 1 && I <= n1 - 2 && J <= n1 - 2) {
    int ci[2], ca[2], cj[2], cb[2], nx = 0, ny = 0;
    if (I & 1) {
      ci[nx] = I >> 1; ca[nx++] = 1;
    } else {
      if ((I >> 1) - 1 >= 0) { ci[nx] = (I >> 1) - 1; ca[nx++] = 2; }
      if ((I >> 1) < N) { ci[nx] = I >> 1; ca[nx++] = 0; }
    }
    if (J & 1) {
      cj[ny] = J >> 1; cb[ny++] = 1;
    } else {
      if ((J >> 1) - 1 >= 0) { cj[ny] = (J >> 1) - 1; cb[ny++] = 2; }
      if ((J >> 1) < N) { cj[ny] = J >> 1; cb[ny++] = 0; }
    }
    double d00 = 0.0, d01 = 0.0, d11 = 0.0;
    for (int u = 0; u < ny; ++u)
      for (int t = 0; t < nx; ++t) {
        const long long c = (long long)cj[u] * N + ci[t];
        const int r = 2 * (3 * cb[u] + ca[t]);
        d00 += ke[(long long)elem18(r, r) * cpl + c];
        d01 += ke[(long long)elem18(r, r + 1) * cpl + c];
        d11 += ke[(long long)elem18(r + 1, r + 1) * cpl + c];
      }
    const double det = d00 * d11 - d01 * d01;
    i00 = d11 / det;
    i01 = -d01 / det;
    i11 = d00 / det;
  }
  dinv[nd] = i00;
  dinv[gq.plane + nd] = i01;
  dinv[2 * gq.plane + nd] = i11;
}

// One Chebyshev step on the Q2 operator (Saad, Alg. 12.1 on D^-1 A, step
// coefficients coef[2 k], coef[2 k + 1] from launch_cheb_coefs):
//   d <- c1 d + c2 D^-1 (b - Ax),  x <- x + d     (Ax = A x given).
__global__ void k_q2_cheb_step(long long n, const double* __restrict__ dinv, long long pl,
                               const double* __restrict__ coef, int k, const double2* __restrict__ b,
                               const double2* __restrict__ Ax, double2* __restrict__ x, double2* __restrict__ d) {
  const double c1 = coef[2 * k], c2 = coef[2 * k + 1];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double rx = b[t].x - Ax[t].x, ry = b[t].y - Ax[t].y;
    const double i00 = dinv[t], i01 = dinv[pl + t], i11 = dinv[2 * pl + t];
    double2 dd = d[t];
    dd.x = c1 * dd.x + c2 * (i00 * rx + i01 * ry);
    dd.y = c1 * dd.y + c2 * (i01 * rx + i11 * ry);
    d[t] = dd;
    double2 xx = x[t];
    xx.x += dd.x;
    xx.y += dd.y;
    x[t] = xx;
  }
}

// Start vector of the power iteration: a checkerboard in both components on
// the interior nodes (all the high-frequency modes the smoother must damp).
__global__ void k_q2_checker(int N, Layout gq, double2* __restrict__ x) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int n1 = 2 * N + 1;
  if (I >= n1 || J >= n1) return;
  const bool in = I >= 1 && J >= 1 && I <= n1 - 2 && J <= n1 - 2;
  const double a = ((I + J) & 1) ? 1.0 : -1.0, b = (I & 1) ? 1.0 : -1.0;
  x[(long long)J * gq.ld + I] = in ? make_double2(a, b) : make_double2(0.0, 0.0);
}

// y <- D^-1 x (the power iteration for lambda_max(D^-1 A)).
__global__ void k_q2_dinv_apply(long long n, const double* __restrict__ dinv, long long pl,
                                const double2* __restrict__ x, double2* __restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double i00 = dinv[t], i01 = dinv[pl + t], i11 = dinv[2 * pl + t];
    const double2 v = x[t];
    y[t] = make_double2(i00 * v.x + i01 * v.y, i01 * v.x + i11 * v.y);
  }
}

// Dual state of the Q1 operator on the 2N grid from the Q2 one: Q1 cell (I, J)
// is sub-cell (I & 1, J & 1) of Q2 cell (I/2, J/2), and its Gauss point
// (qa, qb) lies nearest to the Q2 point (a + qa, b + qb) (Q1 points at cell
// coordinates 0.106, 0.394, 0.606, 0.894; Q2 points at 0.113, 0.5, 0.887).
__global__ void k_q2_pi_to_q1(int N, long long cpl, Layout g1, const double* __restrict__ pi2,
                              double* __restrict__ pi1) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= 2 * N || J >= 2 * N) return;
  const long long c2 = (long long)(J >> 1) * N + (I >> 1);
  const long long c1 = (long long)J * g1.ld + I;
  const int a = I & 1, b = J & 1;
#pragma unroll
  for (int qb = 0; qb < 2; ++qb)
#pragma unroll
    for (int qa = 0; qa < 2; ++qa) {
      const int q1 = 2 * qb + qa, q2 = 3 * (b + qb) + (a + qa);
#pragma unroll
      for (int k = 0; k < 3; ++k) pi1[(3 * q1 + k) * g1.plane + c1] = pi2[(3 * q2 + k) * cpl + c2];
    }
}

// dual state, caller layout ((j N + i) 9 + q) 3 + c  <->  27 planes of cpl
__global__ void k_q2_pi_layout(int N, long long cpl, const double* __restrict__ src, double* __restrict__ dst,
                               int to_planes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  const long long c = (long long)j * N + i;
  for (int t = 0; t < 27; ++t) {
    if (to_planes)
      dst[t * cpl + c] = src[c * 27 + t];
    else
      dst[c * 27 + t] = src[t * cpl + c];
  }
}

}  // namespace

// ---- host side -----------------------------------------------------------------------
int q2_init_tables() {
  const double g = std::sqrt(3.0 / 5.0) / 2.0;
  const double xs[3] = {0.5 - g, 0.5, 0.5 + g}, ws[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  auto lag = [](double x, double val[3], double der[3]) {
    val[0] = 2 * (x - 0.5) * (x - 1);
    val[1] = -4 * x * (x - 1);
    val[2] = 2 * x * (x - 0.5);
    der[0] = 4 * x - 3;
    der[1] = -8 * x + 4;
    der[2] = 4 * x - 1;
  };
  double Nt[9][9], Dx[9][9], Dy[9][9], Wt[9];
  for (int qb = 0; qb < 3; ++qb)
    for (int qa = 0; qa < 3; ++qa) {
      const int q = 3 * qb + qa;
      double lx[3], dlx[3], ly[3], dly[3];
      lag(xs[qa], lx, dlx);
      lag(xs[qb], ly, dly);
      Wt[q] = ws[qa] * ws[qb];
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const int n = 3 * b + a;
          Nt[q][n] = lx[a] * ly[b];
          Dx[q][n] = dlx[a] * ly[b];
          Dy[q][n] = lx[a] * dly[b];
        }
    }
  if (cudaMemcpyToSymbol(c_N9, Nt, sizeof(Nt)) != cudaSuccess || cudaMemcpyToSymbol(c_DX9, Dx, sizeof(Dx)) != cudaSuccess ||
      cudaMemcpyToSymbol(c_DY9, Dy, sizeof(Dy)) != cudaSuccess || cudaMemcpyToSymbol(c_W9, Wt, sizeof(Wt)) != cudaSuccess)
    return -1;
  return 0;
}

void launch_q2_precompute(cudaStream_t s, const Q2Geom& q, double dt, const PhysConst& pc, const double* hcell,
                          const double* A, const double* wind, const double* ocean, const double* vold, double* P,
                          double* rhoH, double* fq, double* voq) {
  note_launch();
  k_q2_precompute<<<q2_cell_grid(q.N), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, dt, pc, hcell, A, wind, ocean, vold, P, rhoH,
                                                       fq, voq);
}
void launch_q2_pi_init(cudaStream_t s, const Q2Geom& q, const Phys& ph, const double2* v, double* pi) {
  note_launch();
  k_q2_pi_init<<<q2_cell_grid(q.N), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, ph, v, pi);
}
int q2_node_partials(const Q2Geom& q) {
  const dim3 g = q2_node_grid(2 * q.N + 1);
  return g.x * g.y;
}
void launch_q2_residual(cudaStream_t s, const Q2Geom& q, const Phys& ph, const double2* v, const double* P,
                        const double* rhoH, const double* fq, const double* voq, double* eb, double2* R,
                        double* partial) {
  note_launch();
  k_q2_residual_cells<<<q2_cell_grid(q.N), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, ph, v, P, rhoH, fq, voq, eb);
  note_launch();
  k_q2_gather<<<q2_node_grid(2 * q.N + 1), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, eb, R, partial);
}
int q2_energy_partials(const Q2Geom& q) {
  const dim3 g = q2_cell_grid(q.N);
  return g.x * g.y;
}
void launch_q2_energy(cudaStream_t s, const Q2Geom& q, const Phys& ph, int k, const AlphaSet& al, const double2* v,
                      const double2* dv, const double* P, const double* rhoH, const double* fq, const double* voq,
                      double* partial, double* out) {
  const dim3 g = q2_cell_grid(q.N);
  const int nb = g.x * g.y;
  note_launch();
  k_q2_energy_cells<<<g, kQBlk, 0, s>>>(q.N, q.gq, q.cpl, ph, k, al, v, dv, P, rhoH, fq, voq, partial, nb);
  launch_energy_final(s, k, partial, nb, out);
}
void launch_q2_element_matrices(cudaStream_t s, const Q2Geom& q, const Phys& ph, const double2* v, const double* pi,
                                const double* P, const double* rhoH, const double* voq, double* ke) {
  note_launch();
  k_q2_element_matrices<<<q2_cell_grid(q.N), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, ph, v, pi, P, rhoH, voq, ke);
}
void launch_q2_apply(cudaStream_t s, const Q2Geom& q, const double* ke, const double2* x, double* eb, double2* y) {
  note_launch();
  k_q2_apply_cells<<<q2_cell_grid(q.N), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, ke, x, eb);
  note_launch();
  k_q2_gather<<<q2_node_grid(2 * q.N + 1), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, eb, y, nullptr);
}
void launch_q2_refine_cells(cudaStream_t s, int N, const double* src, double* dst) {
  note_launch();
  k_q2_refine_cells<<<q2_cell_grid(2 * N), kQBlk, 0, s>>>(N, src, dst);
}
inline unsigned q2_flat_blocks(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}
void launch_q2_dinv(cudaStream_t s, const Q2Geom& q, const double* ke, double* dinv) {
  note_launch();
  k_q2_dinv<<<q2_node_grid(2 * q.N + 1), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, ke, dinv);
}
void launch_q2_cheb_step(cudaStream_t s, const Q2Geom& q, const double* dinv, const double* coef, int k,
                         const double2* b, const double2* Ax, double2* x, double2* d) {
  note_launch();
  k_q2_cheb_step<<<q2_flat_blocks(q.gq.plane), 256, 0, s>>>(q.gq.plane, dinv, q.gq.plane, coef, k, b, Ax, x, d);
}
void launch_q2_checker(cudaStream_t s, const Q2Geom& q, double2* x) {
  note_launch();
  k_q2_checker<<<q2_node_grid(2 * q.N + 1), kQBlk, 0, s>>>(q.N, q.gq, x);
}
void launch_q2_dinv_apply(cudaStream_t s, const Q2Geom& q, const double* dinv, const double2* x, double2* y) {
  note_launch();
  k_q2_dinv_apply<<<q2_flat_blocks(q.gq.plane), 256, 0, s>>>(q.gq.plane, dinv, q.gq.plane, x, y);
}
void launch_q2_pi_to_q1(cudaStream_t s, const Q2Geom& q, const double* pi2, double* pi1) {
  note_launch();
  k_q2_pi_to_q1<<<q2_cell_grid(2 * q.N), kQBlk, 0, s>>>(q.N, q.cpl, q.gq, pi2, pi1);
}
void launch_q2_pi_layout(cudaStream_t s, const Q2Geom& q, const double* src, double* dst, bool to_planes) {
  note_launch();
  k_q2_pi_layout<<<q2_cell_grid(q.N), kQBlk, 0, s>>>(q.N, q.cpl, src, dst, to_planes ? 1 : 0);
}
void launch_q2_dual_update(cudaStream_t s, const Q2Geom& q, const Phys& ph, double alpha, const double2* v,
                           const double2* dv, double* pi) {
  note_launch();
  k_q2_dual_update<<<q2_cell_grid(q.N), kQBlk, 0, s>>>(q.N, q.gq, q.cpl, ph, alpha, v, dv, pi);
}

}  // namespace svn
