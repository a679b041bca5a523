// Per-cell FP64 kernels of the svN step: precomputation, the nonlinear
// residual, the energy, the linearisation (quadrature coefficients, element
// matrices, level-0 stencil) and the dual update.
//
// Every cell kernel evaluates the Q1 velocity and its gradient at the four
// 2x2 Gauss points from the cell's four corner nodes.  Gradients are kept in
// "hat" units (derivatives with respect to the local coordinates xi, eta in
// [0, 1]); true gradients are hat / dx.
#include "kernels.h"

namespace svn {

namespace {

struct Corners {
  double2 v00, v10, v01, v11;
};

__device__ __forceinline__ Corners load_corners(const double2* __restrict__ v, long long n00, int ld) {
  Corners c;
  c.v00 = v[n00];
  c.v10 = v[n00 + 1];
  c.v01 = v[n00 + ld];
  c.v11 = v[n00 + ld + 1];
  return c;
}

struct Qp {
  double vx, vy;              // velocity
  double gxx, gxy, gyx, gyy;  // hat gradient g[k][d] = d v_k / d xi_d
};

__device__ __forceinline__ Qp eval_qp(const Corners& c, double xi, double eta) {
  Qp q;
  const double n00 = (1.0 - xi) * (1.0 - eta), n10 = xi * (1.0 - eta);
  const double n01 = (1.0 - xi) * eta, n11 = xi * eta;
  q.vx = n00 * c.v00.x + n10 * c.v10.x + n01 * c.v01.x + n11 * c.v11.x;
  q.vy = n00 * c.v00.y + n10 * c.v10.y + n01 * c.v01.y + n11 * c.v11.y;
  q.gxx = (1.0 - eta) * (c.v10.x - c.v00.x) + eta * (c.v11.x - c.v01.x);
  q.gyx = (1.0 - eta) * (c.v10.y - c.v00.y) + eta * (c.v11.y - c.v01.y);
  q.gxy = (1.0 - xi) * (c.v01.x - c.v00.x) + xi * (c.v11.x - c.v10.x);
  q.gyy = (1.0 - xi) * (c.v01.y - c.v00.y) + xi * (c.v11.y - c.v10.y);
  return q;
}

// Shape functions and hat derivatives of corner c at (xi, eta).
__device__ __forceinline__ void shape(int c, double xi, double eta, double& n, double& dxi, double& deta) {
  const double a = (c & 1) ? xi : 1.0 - xi;
  const double b = (c & 2) ? eta : 1.0 - eta;
  n = a * b;
  dxi = ((c & 1) ? 1.0 : -1.0) * b;
  deta = ((c & 2) ? 1.0 : -1.0) * a;
}

__device__ __forceinline__ double qxi(int q) { return (q & 1) ? GQ1 : GQ0; }
__device__ __forceinline__ double qeta(int q) { return (q & 2) ? GQ1 : GQ0; }

// hat tau (Voigt-free components) from the hat gradient:
// tau = e^-1 eps' + tr(eps) I / 2  ->  txx = ta gxx + tb gyy, tyy = tb gxx + ta gyy,
// txy = tc (gxy + gyx).
__device__ __forceinline__ void tau_hat(const Phys& ph, const Qp& q, double& txx, double& tyy, double& txy) {
  txx = ph.ta * q.gxx + ph.tb * q.gyy;
  tyy = ph.tb * q.gxx + ph.ta * q.gyy;
  txy = ph.tc * (q.gxy + q.gyx);
}

__device__ __forceinline__ bool interior(int i, int j, int N) { return i >= 1 && j >= 1 && i <= N - 1 && j <= N - 1; }

// ---- a1: precomputation ---------------------------------------------------------
__global__ void k_precompute(Layout g, double dt, PhysConst pc, const double* __restrict__ hcell,
                             const double* __restrict__ A, const double* __restrict__ wind,
                             const double* __restrict__ ocean, const double* __restrict__ vold,
                             double* __restrict__ P, double* __restrict__ rhoH, double* __restrict__ fq,
                             double* __restrict__ voq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N || j >= g.N) return;
  const int n1 = g.N + 1;
  const long long cell = (long long)j * g.ld + i;
  const double h = hcell[(long long)j * g.N + i];
  const double a = A[(long long)j * g.N + i];
  const double Pc = pc.Pstar * h * exp(-pc.C * (1.0 - a));   // Eq. "ice-strength"
  const double rh = pc.rho_ice * h;
  P[cell] = Pc;
  rhoH[cell] = rh;
  // corner values (unpadded caller layout); v^n is zero on the boundary
  double wx[4], wy[4], ox[4], oy[4], nx[4], ny[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int ii = i + (c & 1), jj = j + (c >> 1);
    const long long k = 2 * ((long long)jj * n1 + ii);
    wx[c] = wind[k];
    wy[c] = wind[k + 1];
    ox[c] = ocean[k];
    oy[c] = ocean[k + 1];
    const bool bnd = ii == 0 || jj == 0 || ii == g.N || jj == g.N;
    nx[c] = bnd ? 0.0 : vold[k];
    ny[c] = bnd ? 0.0 : vold[k + 1];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double xi = qxi(q), eta = qeta(q);
    double s[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double n, d1, d2;
      shape(c, xi, eta, n, d1, d2);
      s[c] = n;
    }
    double vax = 0, vay = 0, vox = 0, voy = 0, vnx = 0, vny = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      vax += s[c] * wx[c];
      vay += s[c] * wy[c];
      vox += s[c] * ox[c];
      voy += s[c] * oy[c];
      vnx += s[c] * nx[c];
      vny += s[c] * ny[c];
    }
    // tau_atm = Ca rho_a |v_a| v_a (Eq. "force"); explicit Coriolis
    // rho H f e_r x (v^n - v_o), e_r x w = (-w_y, w_x) (Eq. "F")
    const double sa = pc.Ca * pc.rho_a * sqrt(vax * vax + vay * vay);
    const double dwx = vnx - vox, dwy = vny - voy;
    const double corx = -rh * pc.f_c * dwy, cory = rh * pc.f_c * dwx;
    // constant part of the residual source: -rho H v^n + dt cor - dt tau_atm
    fq[(2 * q) * g.plane + cell] = -rh * vnx + dt * corx - dt * sa * vax;
    fq[(2 * q + 1) * g.plane + cell] = -rh * vny + dt * cory - dt * sa * vay;
    voq[(2 * q) * g.plane + cell] = vox;
    voq[(2 * q + 1) * g.plane + cell] = voy;
  }
}

// pi_0 = tau(v) / Delta(v) at every quadrature point (Eq. "pi").
__global__ void k_pi_init(Layout g, Phys ph, const double2* __restrict__ v, double* __restrict__ pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N || j >= g.N) return;
  const long long cell = (long long)j * g.ld + i;
  const Corners c = load_corners(v, cell, g.ld);
  const double idx = ph.idx;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const Qp p = eval_qp(c, qxi(q), qeta(q));
    double txx, tyy, txy;
    tau_hat(ph, p, txx, tyy, txy);
    txx *= idx; tyy *= idx; txy *= idx;
    const double inv = rsqrt(ph.dmin2 + 2.0 * (txx * txx + tyy * tyy + 2.0 * txy * txy));
    pi[(3 * q + 0) * g.plane + cell] = txx * inv;
    pi[(3 * q + 1) * g.plane + cell] = tyy * inv;
    pi[(3 * q + 2) * g.plane + cell] = txy * inv;
  }
}

// ---- a2: nonlinear residual ------------------------------------------------------
// Per cell: the 8 nodal contributions sum_q w [N_c s_q] + VP term, written to
// 8 planes (corner c, component k) of `eb`.
__global__ void k_residual_cells(Layout g, Phys ph, const double2* __restrict__ v, const double* __restrict__ P,
                                 const double* __restrict__ rhoH, const double* __restrict__ fq,
                                 const double* __restrict__ voq, double* __restrict__ eb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N || j >= g.N) return;
  const long long cell = (long long)j * g.ld + i;
  const Corners c = load_corners(v, cell, g.ld);
  const double Pdt = ph.dt * P[cell];
  const double rh = rhoH[cell];
  const double idx = ph.idx;
  const double vpw = 0.25 * ph.dx;   // w / dx
  double rx[4] = {0, 0, 0, 0}, ry[4] = {0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double xi = qxi(q), eta = qeta(q);
    const Qp p = eval_qp(c, xi, eta);
    double txx, tyy, txy;
    tau_hat(ph, p, txx, tyy, txy);
    const double tt = (txx * txx + tyy * tyy + 2.0 * txy * txy) * idx * idx;
    const double inv = rsqrt(ph.dmin2 + 2.0 * tt);            // 1 / Delta
    const double sfac = Pdt * inv * idx;                       // dt P / Delta / dx
    const double Sxx = sfac * txx, Syy = sfac * tyy, Sxy = sfac * txy;
    const double Fxx = ph.ta * Sxx + ph.tb * Syy - 0.5 * Pdt;
    const double Fyy = ph.tb * Sxx + ph.ta * Syy - 0.5 * Pdt;
    const double Fxy = 2.0 * ph.tc * Sxy;
    const double Gxx = vpw * Fxx, Gxy = vpw * Fxy, Gyy = vpw * Fyy;
    // source: rho H v + (-rho H v^n + dt cor - dt tau_atm) - dt Co rho_o |w| w
    const double wx = voq[(2 * q) * g.plane + cell] - p.vx;
    const double wy = voq[(2 * q + 1) * g.plane + cell] - p.vy;
    const double dr = ph.dt * ph.cdrag * sqrt(wx * wx + wy * wy);
    const double sx = ph.w * (rh * p.vx + fq[(2 * q) * g.plane + cell] - dr * wx);
    const double sy = ph.w * (rh * p.vy + fq[(2 * q + 1) * g.plane + cell] - dr * wy);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double n, dxi, deta;
      shape(k, xi, eta, n, dxi, deta);
      rx[k] = fma(n, sx, rx[k]);
      rx[k] = fma(dxi, Gxx, rx[k]);
      rx[k] = fma(deta, Gxy, rx[k]);
      ry[k] = fma(n, sy, ry[k]);
      ry[k] = fma(dxi, Gxy, ry[k]);
      ry[k] = fma(deta, Gyy, ry[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    eb[(2 * k) * g.plane + cell] = rx[k];
    eb[(2 * k + 1) * g.plane + cell] = ry[k];
  }
}

// Gather cell contributions into nodes; boundary rows are 0.  Per-block
// partial sums of |R|^2 go to `partial`.
__global__ void k_residual_nodes(Layout g, const double* __restrict__ eb, double2* __restrict__ R,
                                 double* __restrict__ partial) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double s = 0.0;
  if (i <= g.N && j <= g.N) {
    const long long n = (long long)j * g.ld + i;
    double2 r = make_double2(0.0, 0.0);
    if (interior(i, j, g.N)) {
      // cells (i-1, j-1): corner 3; (i, j-1): corner 2; (i-1, j): corner 1; (i, j): corner 0
      const long long c3 = n - g.ld - 1, c2 = n - g.ld, c1 = n - 1, c0 = n;
      r.x = eb[6 * g.plane + c3] + eb[4 * g.plane + c2] + eb[2 * g.plane + c1] + eb[0 * g.plane + c0];
      r.y = eb[7 * g.plane + c3] + eb[5 * g.plane + c2] + eb[3 * g.plane + c1] + eb[1 * g.plane + c0];
      s = r.x * r.x + r.y * r.y;
    }
    R[n] = r;
  }
  s = block_sum(s);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// ---- a8: energy for k step lengths --------------------------------------------------
// Phi_h(v + alpha dv) = sum over cells and quadrature points of
//   w [ rho H |u|^2 / 2 + fq . u + dt P/2 (Delta - tr eps) + dt Co rho_o |v_o - u|^3 / 3 ]
// with fq . u = -rho H v^n . u + dt cor . u - dt tau_atm . u.  Compensated sums.
__global__ void k_energy_cells(Layout g, Phys ph, int k, AlphaSet al, const double2* __restrict__ v,
                               const double2* __restrict__ dv, const double* __restrict__ P,
                               const double* __restrict__ rhoH, const double* __restrict__ fq,
                               const double* __restrict__ voq, double* __restrict__ partial, int nblocks) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  DD acc[MAX_ALPHA];
  double asum = 0.0;
#pragma unroll
  for (int a = 0; a < MAX_ALPHA; ++a) acc[a] = DD{0.0, 0.0};
  if (i < g.N && j < g.N) {
    const long long cell = (long long)j * g.ld + i;
    const Corners c0 = load_corners(v, cell, g.ld);
    const Corners d0 = load_corners(dv, cell, g.ld);
    const double Ph = 0.5 * ph.dt * P[cell];
    const double rh = rhoH[cell];
    const double idx = ph.idx;
    for (int a = 0; a < k; ++a) {
      const double al0 = al.a[a];
      Corners c;
      c.v00 = make_double2(c0.v00.x + al0 * d0.v00.x, c0.v00.y + al0 * d0.v00.y);
      c.v10 = make_double2(c0.v10.x + al0 * d0.v10.x, c0.v10.y + al0 * d0.v10.y);
      c.v01 = make_double2(c0.v01.x + al0 * d0.v01.x, c0.v01.y + al0 * d0.v01.y);
      c.v11 = make_double2(c0.v11.x + al0 * d0.v11.x, c0.v11.y + al0 * d0.v11.y);
      double csum = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const Qp p = eval_qp(c, qxi(q), qeta(q));
        double txx, tyy, txy;
        tau_hat(ph, p, txx, tyy, txy);
        const double tt = (txx * txx + tyy * tyy + 2.0 * txy * txy) * idx * idx;
        const double Dl = sqrt(ph.dmin2 + 2.0 * tt);
        const double tr = (p.gxx + p.gyy) * idx;
        const double wx = voq[(2 * q) * g.plane + cell] - p.vx;
        const double wy = voq[(2 * q + 1) * g.plane + cell] - p.vy;
        const double nw = sqrt(wx * wx + wy * wy);
        const double t1 = 0.5 * rh * (p.vx * p.vx + p.vy * p.vy);
        const double t2 = fq[(2 * q) * g.plane + cell] * p.vx + fq[(2 * q + 1) * g.plane + cell] * p.vy;
        const double t3 = Ph * (Dl - tr);
        const double t4 = ph.dt * ph.cdrag * nw * nw * nw * (1.0 / 3.0);
        csum += ph.w * ((t1 + t2) + (t3 + t4));
        if (a == 0) asum += ph.w * (fabs(t1) + fabs(t2) + fabs(t3) + fabs(t4));
      }
      acc[a].add(csum);   // plain sum within the cell, compensated over cells
    }
  }
  // block reduction of the (hi, lo) pairs, then write per-block partials:
  // layout partial[(2 a) * nblocks + bid] = hi, [(2 a + 1) * nblocks + bid] = lo,
  // partial[(2 MAX_ALPHA) * nblocks + bid] = sum |terms|
  __shared__ double sh_hi[256], sh_lo[256];
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

// Final compensated reduction of the energy partials: out[a] = Phi, out[MAX_ALPHA] = scale.
__global__ void k_energy_final(int k, const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  __shared__ double sh_hi[1024], sh_lo[1024];
  const int tid = threadIdx.x;
  for (int a = 0; a < k; ++a) {
    DD acc{0.0, 0.0};
    for (int b = tid; b < nblocks; b += blockDim.x) {
      acc.add(DD{partial[(2 * a) * nblocks + b], partial[(2 * a + 1) * nblocks + b]});
    }
    sh_hi[tid] = acc.hi;
    sh_lo[tid] = acc.lo;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (tid < s) {
        DD x{sh_hi[tid], sh_lo[tid]};
        x.add(DD{sh_hi[tid + s], sh_lo[tid + s]});
        sh_hi[tid] = x.hi;
        sh_lo[tid] = x.lo;
      }
      __syncthreads();
    }
    if (tid == 0) out[a] = sh_hi[0] + sh_lo[0];
    __syncthreads();
  }
  double s = 0.0;
  for (int b = tid; b < nblocks; b += blockDim.x) s += partial[(2 * MAX_ALPHA) * nblocks + b];
  s = block_sum(s);
  if (tid == 0) out[MAX_ALPHA] = s;
}

// ---- a3/a4: linearisation -------------------------------------------------------------
// Per cell: at every quadrature point the svN coefficient (Eq. "linearSVNewton"
// with Eq. "modification", Voigt form)
//   C = dt [ (P/Delta) I - P/(Delta^2 m) (t p^T + p t^T) ],  m = max(1, sqrt(2 pi:pi)),
// the mass tensor M = rho H I + dt Co rho_o (|w| I + w w^T / |w|) (Eq.
// "standardNewton2"; the rank-one term is dropped for |w| < 1e-14 m/s), and
// the element matrix K_e = sum_q w (N^T M N + B^T C B), upper triangle.
//
// Evaluation.  On the uniform grid the hat derivatives of the Q1 basis at a
// Gauss point are dN_c/dxi = sx_c G(b_c, qb), dN_c/deta = sy_c G(a_c, qa) with
// G(b, q) = g1 if b == q else g0 (sx, sy = -+1 for corner bits a, b = 0, 1),
// and N_c = G(a_c, qa) G(b_c, qb).  With u = (ta, tb, 0), u' = (tb, ta, 0),
// e2 = (0, 0, sqrt2 tc) and C' = C / 4 (hat-unit weight w / dx^2), the six
// scalars A1 = u C' u, A2 = u C' e2, A3 = e2 C' e2, A4 = u' C' u', A5 = u' C' e2,
// A6 = u C' u' give
//   Kxx[c][d] = sum_q A1 dxi_c dxi_d + A2 (dxi_c deta_d + deta_c dxi_d) + A3 deta_c deta_d
//   Kyy[c][d] = sum_q A4 deta_c deta_d + A5 (deta_c dxi_d + dxi_c deta_d) + A3 dxi_c dxi_d
//   Kxy[c][d] = sum_q A6 dxi_c deta_d + A2 dxi_c dxi_d + A5 deta_c deta_d + A3 deta_c dxi_d
// (plus the mass terms sum_q N_c N_d w M), so each entry is a signed sum of a
// few small "moment tables" of the six scalars over the four points.
__device__ __forceinline__ double gq(int b, int q) { return b == q ? GQ1 : GQ0; }

struct Moments {
  double xx[3];      // T_xixi[bc][bd]: [0][0], [0][1], [1][1]
  double ee[3];      // T_etaeta[ac][ad]
  double xe[2][2];   // T_xieta[bc][ad]
};

__device__ __forceinline__ void moments(const double F[4], Moments& m) {
  // q = qa + 2 qb
  const double fb0 = F[0] + F[1], fb1 = F[2] + F[3];   // sums over qa, per qb
  const double fa0 = F[0] + F[2], fa1 = F[1] + F[3];   // sums over qb, per qa
  const double g00 = GQ0 * GQ0, g11 = GQ1 * GQ1, g01 = GQ0 * GQ1;
  // T_xixi[bc][bd] = sum_qb G(bc,qb) G(bd,qb) fb(qb)
  m.xx[0] = g11 * fb0 + g00 * fb1;
  m.xx[1] = g01 * (fb0 + fb1);
  m.xx[2] = g00 * fb0 + g11 * fb1;
  m.ee[0] = g11 * fa0 + g00 * fa1;
  m.ee[1] = g01 * (fa0 + fa1);
  m.ee[2] = g00 * fa0 + g11 * fa1;
#pragma unroll
  for (int bc = 0; bc < 2; ++bc)
#pragma unroll
    for (int ad = 0; ad < 2; ++ad) {
      double t = 0.0;
#pragma unroll
      for (int qb = 0; qb < 2; ++qb)
#pragma unroll
        for (int qa = 0; qa < 2; ++qa) t += gq(bc, qb) * gq(ad, qa) * F[qa + 2 * qb];
      m.xe[bc][ad] = t;
    }
}

__device__ __forceinline__ double sym2(const double t[3], int i, int j) { return t[i + j]; }

template <typename TE>
__global__ void __launch_bounds__(128) k_element_matrices(Layout g, Phys ph, const double2* __restrict__ v,
                                                          const double* __restrict__ pi, const double* __restrict__ P,
                                                          const double* __restrict__ rhoH,
                                                          const double* __restrict__ voq, TE* __restrict__ ke) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N || j >= g.N) return;
  const long long cell = (long long)j * g.ld + i;
  const Corners c = load_corners(v, cell, g.ld);
  const double Pc = P[cell];
  const double rh = rhoH[cell];
  const double idx = ph.idx;
  const double sq2 = 1.4142135623730950488;
  const double ta = ph.ta, tb = ph.tb, s2 = sq2 * ph.tc;
  double A1[4], A2[4], A3[4], A4[4], A5[4], A6[4], Mxx[4], Myy[4], Mxy[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const Qp p = eval_qp(c, qxi(q), qeta(q));
    double txx, tyy, txy;
    tau_hat(ph, p, txx, tyy, txy);
    const double t0 = txx * idx, t1 = tyy * idx, t2 = sq2 * txy * idx;   // Voigt tau
    const double inv = rsqrt(ph.dmin2 + 2.0 * (t0 * t0 + t1 * t1 + t2 * t2));
    const double p0 = pi[(3 * q + 0) * g.plane + cell];
    const double p1 = pi[(3 * q + 1) * g.plane + cell];
    const double p2 = sq2 * pi[(3 * q + 2) * g.plane + cell];
    const double pp = 2.0 * (p0 * p0 + p1 * p1 + p2 * p2);
    const double invm = pp > 1.0 ? rsqrt(pp) : 1.0;   // 1 / max(1, sqrt(2 pi:pi)), the FP64 branch
    const double a = 0.25 * ph.dt * Pc * inv;               // C' = C / 4
    const double b = 0.25 * ph.dt * Pc * inv * inv * invm;
    const double C00 = a - 2.0 * b * t0 * p0, C11 = a - 2.0 * b * t1 * p1, C22 = a - 2.0 * b * t2 * p2;
    const double C01 = -b * (t0 * p1 + p0 * t1), C02 = -b * (t0 * p2 + p0 * t2), C12 = -b * (t1 * p2 + p1 * t2);
    A1[q] = ta * ta * C00 + 2.0 * ta * tb * C01 + tb * tb * C11;
    A4[q] = tb * tb * C00 + 2.0 * ta * tb * C01 + ta * ta * C11;
    A6[q] = ta * tb * (C00 + C11) + (ta * ta + tb * tb) * C01;
    A2[q] = s2 * (ta * C02 + tb * C12);
    A5[q] = s2 * (tb * C02 + ta * C12);
    A3[q] = s2 * s2 * C22;
    const double wx = voq[(2 * q) * g.plane + cell] - p.vx;
    const double wy = voq[(2 * q + 1) * g.plane + cell] - p.vy;
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
    Mxx[q] = ph.w * mxx;
    Myy[q] = ph.w * myy;
    Mxy[q] = ph.w * mxy;
  }
  Moments mA1, mA2, mA3, mA4, mA5, mA6;
  moments(A1, mA1);
  moments(A2, mA2);
  moments(A3, mA3);
  moments(A4, mA4);
  moments(A5, mA5);
  moments(A6, mA6);
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
#pragma unroll
    for (int dd = cc; dd < 4; ++dd) {
      const int ac = cc & 1, bc = cc >> 1, ad = dd & 1, bd = dd >> 1;
      const double sxc = ac ? 1.0 : -1.0, syc = bc ? 1.0 : -1.0, sxd = ad ? 1.0 : -1.0, syd = bd ? 1.0 : -1.0;
      // mass moments: sum_q N_c N_d M(q)
      double nxx = 0.0, nyy = 0.0, nxy = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int qa = q & 1, qb = q >> 1;
        const double nn = gq(ac, qa) * gq(bc, qb) * gq(ad, qa) * gq(bd, qb);
        nxx += nn * Mxx[q];
        nyy += nn * Myy[q];
        nxy += nn * Mxy[q];
      }
      const double kxx = sxc * sxd * sym2(mA1.xx, bc, bd) + sxc * syd * mA2.xe[bc][ad] +
                         syc * sxd * mA2.xe[bd][ac] + syc * syd * sym2(mA3.ee, ac, ad) + nxx;
      const double kyy = syc * syd * sym2(mA4.ee, ac, ad) + syc * sxd * mA5.xe[bd][ac] +
                         sxc * syd * mA5.xe[bc][ad] + sxc * sxd * sym2(mA3.xx, bc, bd) + nyy;
      const double kxy = sxc * syd * mA6.xe[bc][ad] + sxc * sxd * sym2(mA2.xx, bc, bd) +
                         syc * syd * sym2(mA5.ee, ac, ad) + syc * sxd * mA3.xe[bd][ac] + nxy;
      ke[(long long)elem_index(2 * cc, 2 * dd) * g.plane + cell] = (TE)kxx;
      ke[(long long)elem_index(2 * cc + 1, 2 * dd + 1) * g.plane + cell] = (TE)kyy;
      ke[(long long)elem_index(2 * cc, 2 * dd + 1) * g.plane + cell] = (TE)kxy;
      if (dd != cc) {
        // K[2cc+1][2dd] = Kyx[cc][dd] = Kxy[dd][cc]
        const double kyx = sxd * syc * mA6.xe[bd][ac] + sxd * sxc * sym2(mA2.xx, bd, bc) +
                           syd * syc * sym2(mA5.ee, ad, ac) + syd * sxc * mA3.xe[bc][ad] + nxy;
        ke[(long long)elem_index(2 * cc + 1, 2 * dd) * g.plane + cell] = (TE)kyx;
      }
    }
  }
}

// Element-matrix entry (r, s) of cell `cell`, either triangle.
template <typename TE>
__device__ __forceinline__ double kel(const TE* __restrict__ ke, long long plane, long long cell, int r, int s) {
  return (double)ke[(long long)(r <= s ? elem_index(r, s) : elem_index(s, r)) * plane + cell];
}

// Gather the level-0 stencil at interior nodes from the element matrices.
template <typename TE, typename TS>
__global__ void k_stencil_from_elements(Layout g, const TE* __restrict__ ke, TS* __restrict__ st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (!interior(i, j, g.N)) return;
  const long long n = (long long)j * g.ld + i;
  const long long pl = g.plane;
  // cells around node n, with the node's corner index in each
  const long long cl[4] = {n, n - 1, n - g.ld, n - g.ld - 1};
  const int cp[4] = {0, 1, 2, 3};
  double dxx = 0, dxy = 0, dyy = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int c = cp[t];
    dxx += kel(ke, pl, cl[t], 2 * c, 2 * c);
    dxy += kel(ke, pl, cl[t], 2 * c, 2 * c + 1);
    dyy += kel(ke, pl, cl[t], 2 * c + 1, 2 * c + 1);
  }
  st[(S_D + 0) * pl + n] = (TS)dxx;
  st[(S_D + 1) * pl + n] = (TS)dxy;
  st[(S_D + 2) * pl + n] = (TS)dyy;
  // off-diagonal blocks: (cell, corner of p, corner of q) pairs
  auto blk = [&](int slot, int npairs, const long long* cells, const int* cpp, const int* cqq) {
    double b[4] = {0, 0, 0, 0};
    for (int t = 0; t < npairs; ++t) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int l = 0; l < 2; ++l) b[2 * k + l] += kel(ke, pl, cells[t], 2 * cpp[t] + k, 2 * cqq[t] + l);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) st[(slot + e) * pl + n] = (TS)b[e];
  };
  {  // E: cells (i, j-1) [p=2, q=3] and (i, j) [p=0, q=1]
    const long long cs[2] = {n - g.ld, n};
    const int a[2] = {2, 0}, b[2] = {3, 1};
    blk(S_E, 2, cs, a, b);
  }
  {  // N: cells (i-1, j) [p=1, q=3] and (i, j) [p=0, q=2]
    const long long cs[2] = {n - 1, n};
    const int a[2] = {1, 0}, b[2] = {3, 2};
    blk(S_N, 2, cs, a, b);
  }
  {  // NE: cell (i, j) [p=0, q=3]
    const long long cs[1] = {n};
    const int a[1] = {0}, b[1] = {3};
    blk(S_NE, 1, cs, a, b);
  }
  {  // NW: cell (i-1, j) [p=1, q=2]
    const long long cs[1] = {n - 1};
    const int a[1] = {1}, b[1] = {2};
    blk(S_NW, 1, cs, a, b);
  }
}

// ---- a9: dual update ------------------------------------------------------------------
// pi <- pi + alpha pi~, pi~ = -pi + t/Delta + t~/Delta - [(t.t~) p + (p.t~) t] / (Delta^2 m)
// in Voigt form (Eq. "tautilde" with Eq. "modification"), t = tau(v), t~ = tau(dv).
__global__ void k_dual_update(Layout g, Phys ph, double alpha, const double2* __restrict__ v,
                              const double2* __restrict__ dv, double* __restrict__ pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.N || j >= g.N) return;
  const long long cell = (long long)j * g.ld + i;
  const Corners c = load_corners(v, cell, g.ld);
  const Corners d = load_corners(dv, cell, g.ld);
  const double idx = ph.idx;
  const double sq2 = 1.4142135623730950488;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double xi = qxi(q), eta = qeta(q);
    const Qp p = eval_qp(c, xi, eta);
    const Qp pd = eval_qp(d, xi, eta);
    double txx, tyy, txy, sxx, syy, sxy;
    tau_hat(ph, p, txx, tyy, txy);
    tau_hat(ph, pd, sxx, syy, sxy);
    const double t0 = txx * idx, t1 = tyy * idx, t2 = sq2 * txy * idx;
    const double s0 = sxx * idx, s1 = syy * idx, s2 = sq2 * sxy * idx;
    const double inv = rsqrt(ph.dmin2 + 2.0 * (t0 * t0 + t1 * t1 + t2 * t2));
    double* pq = pi + (long long)(3 * q) * g.plane + cell;
    const double p0 = pq[0], p1 = pq[g.plane], p2 = sq2 * pq[2 * g.plane];
    const double pp = 2.0 * (p0 * p0 + p1 * p1 + p2 * p2);
    const double invm = pp > 1.0 ? rsqrt(pp) : 1.0;   // 1 / max(1, sqrt(2 pi:pi))
    const double ts = t0 * s0 + t1 * s1 + t2 * s2;
    const double ps = p0 * s0 + p1 * s1 + p2 * s2;
    const double f = inv * inv * invm;
    const double n0 = -p0 + (t0 + s0) * inv - (ts * p0 + ps * t0) * f;
    const double n1 = -p1 + (t1 + s1) * inv - (ts * p1 + ps * t1) * f;
    const double n2 = -p2 + (t2 + s2) * inv - (ts * p2 + ps * t2) * f;
    pq[0] = p0 + alpha * n0;
    pq[g.plane] = p1 + alpha * n1;
    pq[2 * g.plane] = (p2 + alpha * n2) * (1.0 / sq2);
  }
}

// ---- fused trial point (a8 + a2 + a9 at alpha = 1) ---------------------------------------
// One pass over the cells evaluates, at u = v + dv:
//   * the energy contributions (compensated, as k_energy_cells) and sum |terms|,
//   * the residual cell contributions of R(u) into eb (as k_residual_cells),
//   * the trial dual state pi_t = pi + pi~(v, dv, pi) (as k_dual_update with alpha = 1),
// so that an accepted unit step needs no further pass.
__global__ void k_trial_cells(Layout g, Phys ph, const double2* __restrict__ v, const double2* __restrict__ dv,
                              const double* __restrict__ P, const double* __restrict__ rhoH,
                              const double* __restrict__ fq, const double* __restrict__ voq,
                              const double* __restrict__ pi, double* __restrict__ pi_t, double* __restrict__ eb,
                              double* __restrict__ partial, int nblocks) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  DD acc{0.0, 0.0};
  double asum = 0.0;
  if (i < g.N && j < g.N) {
    const long long cell = (long long)j * g.ld + i;
    const Corners c0 = load_corners(v, cell, g.ld);
    const Corners d0 = load_corners(dv, cell, g.ld);
    const double Pdt = ph.dt * P[cell];
    const double rh = rhoH[cell];
    const double idx = ph.idx;
    const double vpw = 0.25 * ph.dx;
    const double sq2 = 1.4142135623730950488;
    double rx[4] = {0, 0, 0, 0}, ry[4] = {0, 0, 0, 0};
    // the cell's 16 energy terms are summed in plain FP64 (their rounding is
    // ~1e-16 of the cell's terms); the sum over cells is compensated
    double csum = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double xi = qxi(q), eta = qeta(q);
      // v and dv at the point; u = v + dv and tau(u) by linearity
      const Qp pv = eval_qp(c0, xi, eta);
      const Qp pd = eval_qp(d0, xi, eta);
      double vxx, vyy, vxy, sxx, syy, sxy;
      tau_hat(ph, pv, vxx, vyy, vxy);
      tau_hat(ph, pd, sxx, syy, sxy);
      // dual step at the current point (uses tau(v), Delta(v), tau(dv))
      {
        const double t0 = vxx * idx, t1 = vyy * idx, t2 = sq2 * vxy * idx;
        const double s0 = sxx * idx, s1 = syy * idx, s2 = sq2 * sxy * idx;
        const double inv = rsqrt(ph.dmin2 + 2.0 * (t0 * t0 + t1 * t1 + t2 * t2));
        const double* pq = pi + (long long)(3 * q) * g.plane + cell;
        const double p0 = pq[0], p1 = pq[g.plane], p2 = sq2 * pq[2 * g.plane];
        const double pp = 2.0 * (p0 * p0 + p1 * p1 + p2 * p2);
        const double invm = pp > 1.0 ? rsqrt(pp) : 1.0;   // 1 / max(1, sqrt(2 pi:pi))
        const double ts = t0 * s0 + t1 * s1 + t2 * s2;
        const double ps = p0 * s0 + p1 * s1 + p2 * s2;
        const double f = inv * inv * invm;
        double* pt = pi_t + (long long)(3 * q) * g.plane + cell;
        pt[0] = (t0 + s0) * inv - (ts * p0 + ps * t0) * f;
        pt[g.plane] = (t1 + s1) * inv - (ts * p1 + ps * t1) * f;
        pt[2 * g.plane] = ((t2 + s2) * inv - (ts * p2 + ps * t2) * f) * (1.0 / sq2);
      }
      // energy and residual at u = v + dv
      Qp p;
      p.vx = pv.vx + pd.vx;
      p.vy = pv.vy + pd.vy;
      p.gxx = pv.gxx + pd.gxx;
      p.gxy = pv.gxy + pd.gxy;
      p.gyx = pv.gyx + pd.gyx;
      p.gyy = pv.gyy + pd.gyy;
      const double txx = vxx + sxx, tyy = vyy + syy, txy = vxy + sxy;
      const double tt = (txx * txx + tyy * tyy + 2.0 * txy * txy) * idx * idx;
      const double d2 = ph.dmin2 + 2.0 * tt;
      const double inv = rsqrt(d2);
      const double Dl = d2 * inv;
      const double tr = (p.gxx + p.gyy) * idx;
      const double wx = voq[(2 * q) * g.plane + cell] - p.vx;
      const double wy = voq[(2 * q + 1) * g.plane + cell] - p.vy;
      const double nw = sqrt(wx * wx + wy * wy);
      const double fx = fq[(2 * q) * g.plane + cell], fy = fq[(2 * q + 1) * g.plane + cell];
      const double e1 = ph.w * 0.5 * rh * (p.vx * p.vx + p.vy * p.vy);
      const double e2 = ph.w * (fx * p.vx + fy * p.vy);
      const double e3 = ph.w * 0.5 * Pdt * (Dl - tr);
      const double e4 = ph.w * ph.dt * ph.cdrag * nw * nw * nw * (1.0 / 3.0);
      csum += (e1 + e2) + (e3 + e4);
      asum += fabs(e1) + fabs(e2) + fabs(e3) + fabs(e4);
      const double sfac = Pdt * inv * idx;
      const double Sxx = sfac * txx, Syy = sfac * tyy, Sxy = sfac * txy;
      const double Fxx = ph.ta * Sxx + ph.tb * Syy - 0.5 * Pdt;
      const double Fyy = ph.tb * Sxx + ph.ta * Syy - 0.5 * Pdt;
      const double Fxy = 2.0 * ph.tc * Sxy;
      const double Gxx = vpw * Fxx, Gxy = vpw * Fxy, Gyy = vpw * Fyy;
      const double dr = ph.dt * ph.cdrag * nw;
      const double sx = ph.w * (rh * p.vx + fx - dr * wx);
      const double sy = ph.w * (rh * p.vy + fy - dr * wy);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double n, dxi, deta;
        shape(k, xi, eta, n, dxi, deta);
        rx[k] = fma(n, sx, rx[k]);
        rx[k] = fma(dxi, Gxx, rx[k]);
        rx[k] = fma(deta, Gxy, rx[k]);
        ry[k] = fma(n, sy, ry[k]);
        ry[k] = fma(dxi, Gxy, ry[k]);
        ry[k] = fma(deta, Gyy, ry[k]);
      }
    }
    acc.add(csum);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      eb[(2 * k) * g.plane + cell] = rx[k];
      eb[(2 * k + 1) * g.plane + cell] = ry[k];
    }
  }
  __shared__ double sh_hi[256], sh_lo[256];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  sh_hi[tid] = acc.hi;
  sh_lo[tid] = acc.lo;
  __syncthreads();
  for (int st = nt / 2; st > 0; st >>= 1) {
    if (tid < st) {
      DD x{sh_hi[tid], sh_lo[tid]};
      x.add(DD{sh_hi[tid + st], sh_lo[tid + st]});
      sh_hi[tid] = x.hi;
      sh_lo[tid] = x.lo;
    }
    __syncthreads();
  }
  if (tid == 0) {
    partial[bid] = sh_hi[0];
    partial[nblocks + bid] = sh_lo[0];
  }
  asum = block_sum(asum);
  if (tid == 0) partial[(2 * MAX_ALPHA) * nblocks + bid] = asum;
}

inline dim3 cell_grid(const Layout& g, dim3 blk) {
  return dim3((g.N + blk.x - 1) / blk.x, (g.N + blk.y - 1) / blk.y);
}
inline dim3 node_grid(const Layout& g, dim3 blk) {
  return dim3((g.n1 + blk.x - 1) / blk.x, (g.n1 + blk.y - 1) / blk.y);
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------
const dim3 kCellBlock(32, 4);
const dim3 kNodeBlock(32, 8);

void launch_precompute(cudaStream_t s, const Layout& g, double dt, const PhysConst& pc, const double* hcell,
                       const double* A, const double* wind, const double* ocean, const double* vold, double* P,
                       double* rhoH, double* fq, double* voq) {
  note_launch();
  k_precompute<<<cell_grid(g, kCellBlock), kCellBlock, 0, s>>>(g, dt, pc, hcell, A, wind, ocean, vold, P, rhoH,
                                                              fq, voq);
}

void launch_pi_init(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, double* pi) {
  note_launch();
  k_pi_init<<<cell_grid(g, kCellBlock), kCellBlock, 0, s>>>(g, ph, v, pi);
}

int residual_partials(const Layout& g) {
  dim3 gr = node_grid(g, kNodeBlock);
  return gr.x * gr.y;
}

void launch_residual(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, const double* P,
                     const double* rhoH, const double* fq, const double* voq, double* eb, double2* R,
                     double* partial) {
  note_launch();
  k_residual_cells<<<cell_grid(g, kCellBlock), kCellBlock, 0, s>>>(g, ph, v, P, rhoH, fq, voq, eb);
  note_launch();
  k_residual_nodes<<<node_grid(g, kNodeBlock), kNodeBlock, 0, s>>>(g, eb, R, partial);
}

int energy_partials(const Layout& g) {
  dim3 gr = cell_grid(g, kCellBlock);
  return gr.x * gr.y;
}

void launch_energy(cudaStream_t s, const Layout& g, const Phys& ph, int k, const AlphaSet& al, const double2* v,
                   const double2* dv, const double* P, const double* rhoH, const double* fq, const double* voq,
                   double* partial, double* out) {
  dim3 gr = cell_grid(g, kCellBlock);
  const int nb = gr.x * gr.y;
  note_launch();
  k_energy_cells<<<gr, kCellBlock, 0, s>>>(g, ph, k, al, v, dv, P, rhoH, fq, voq, partial, nb);
  note_launch();
  k_energy_final<<<1, 1024, 0, s>>>(k, partial, nb, out);
}

void launch_energy_final(cudaStream_t s, int k, const double* partial, int nblocks, double* out) {
  note_launch();
  k_energy_final<<<1, 1024, 0, s>>>(k, partial, nblocks, out);
}

template <typename TE>
void launch_element_matrices(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, const double* pi,
                             const double* P, const double* rhoH, const double* voq, TE* ke) {
  note_launch();
  k_element_matrices<TE><<<cell_grid(g, kCellBlock), kCellBlock, 0, s>>>(g, ph, v, pi, P, rhoH, voq, ke);
}
template void launch_element_matrices<double>(cudaStream_t, const Layout&, const Phys&, const double2*,
                                              const double*, const double*, const double*, const double*,
                                              double*);

template <typename TE, typename TS>
void launch_stencil_from_elements(cudaStream_t s, const Layout& g, const TE* ke, TS* st) {
  note_launch();
  k_stencil_from_elements<TE, TS><<<node_grid(g, kNodeBlock), kNodeBlock, 0, s>>>(g, ke, st);
}
template void launch_stencil_from_elements<double, double>(cudaStream_t, const Layout&, const double*, double*);

void launch_trial(cudaStream_t s, const Layout& g, const Phys& ph, const double2* v, const double2* dv,
                  const double* P, const double* rhoH, const double* fq, const double* voq, const double* pi,
                  double* pi_t, double* eb, double2* R, double* partial_e, double* out_e, double* partial_r) {
  dim3 gr = cell_grid(g, kCellBlock);
  const int nb = gr.x * gr.y;
  note_launch();
  k_trial_cells<<<gr, kCellBlock, 0, s>>>(g, ph, v, dv, P, rhoH, fq, voq, pi, pi_t, eb, partial_e, nb);
  note_launch();
  k_energy_final<<<1, 1024, 0, s>>>(1, partial_e, nb, out_e);
  note_launch();
  k_residual_nodes<<<node_grid(g, kNodeBlock), kNodeBlock, 0, s>>>(g, eb, R, partial_r);
}

void launch_dual_update(cudaStream_t s, const Layout& g, const Phys& ph, double alpha, const double2* v,
                        const double2* dv, double* pi) {
  note_launch();
  k_dual_update<<<cell_grid(g, kCellBlock), kCellBlock, 0, s>>>(g, ph, alpha, v, dv, pi);
}

}  // namespace svn
