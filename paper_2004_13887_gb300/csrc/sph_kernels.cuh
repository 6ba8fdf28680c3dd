// sph_kernels.cuh -- the device code of the scheme's stages (Section 2.2,
// eqs. chapter3mainsd, splitting2, spl1-spl3; operators of Appendix B): the
// averaging, coefficient and right-hand-side kernels and the one-thread-per-
// line block and scalar line solvers, shared by the single-problem library
// (sph.cu) and the batched launches over many problems (sph_batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_device.cuh"

namespace sph {}
using namespace sph;

#define FLAG_NONFINITE 1
#define FLAG_SINGULAR 2

// ------------------------------------------------------------------ kernels

// Ubar = (U^n + U^k)/2 for the five fields in one launch (blockIdx.y = field),
// two values per thread per pass (16-byte loads, 8-byte stores in FP32).
// Ubar = (a + b)/2 and D = b - a (a = U^n, b = U^{n+1,k}; D is the -(U^k - U^n)
// part of the right-hand side, so that stage reads neither FP64 state).  In
// FP32 mode both are formed as pairs on the FP32 pipe: o = Ubar rounded, and
// for the velocity components lo[f] (when not null) = the remainder, so that
// div(Ubar) can be formed to ~48 bits; D is rounded once from the exact pair.
// same = 1 (the first iteration of a step, U^k = U^n): b is not read and D is
// not written (the right-hand side does not read it then); Ubar = a is split
// into its pair directly, which gives the same bits as (a + a)/2 in pairs.
template <typename R>
struct AvgArgs { const double* a[5]; const double* b[5]; R* o[5]; R* lo[5]; R* d[5]; long n[5]; int same; };

template <typename R>
__device__ __forceinline__ void avg1(const double x, const double y, R* o, R* lo, R* d, long t) {
  if constexpr (sizeof(R) == sizeof(double)) {
    o[t] = (R)(0.5 * (x + y));
    d[t] = (R)(y - x);
  } else {
    float xh, xl, yh, yl, h, l;
    d2ff(x, xh, xl);
    d2ff(y, yh, yl);
    ff_add(xh, xl, yh, yl, h, l);
    o[t] = 0.5f * h;
    if (lo) lo[t] = 0.5f * l;
    ff_sub(yh, yl, xh, xl, h, l);
    d[t] = h + l;
  }
}

template <typename R>
__device__ __forceinline__ void split1(const double x, R* o, R* lo, long t) {
  if constexpr (sizeof(R) == sizeof(double)) {
    o[t] = (R)x;
  } else {
    float h, l;
    d2ff(x, h, l);
    o[t] = h;
    if (lo) lo[t] = l;
  }
}

template <typename R>
__global__ void k_avg(AvgArgs<R> A) {
  const int f = blockIdx.y;
  const double* __restrict__ a = A.a[f];
  const double* __restrict__ b = A.b[f];
  R* __restrict__ o = A.o[f];
  R* __restrict__ lo = A.lo[f];
  R* __restrict__ d = A.d[f];
  long n = A.n[f], n2 = n >> 1;
  long s = (long)gridDim.x * blockDim.x;
  if (A.same) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += s) {
      double2 x = reinterpret_cast<const double2*>(a)[t];
      split1(x.x, o, lo, 2 * t);
      split1(x.y, o, lo, 2 * t + 1);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) split1(a[n - 1], o, lo, n - 1);
    return;
  }
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += s) {
    double2 x = reinterpret_cast<const double2*>(a)[t], y = reinterpret_cast<const double2*>(b)[t];
    avg1(x.x, y.x, o, lo, d, 2 * t);
    avg1(x.y, y.y, o, lo, d, 2 * t + 1);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) avg1(a[n - 1], b[n - 1], o, lo, d, n - 1);
}

template <typename R>
__global__ void k_cvt(long n, const R* __restrict__ a, double* __restrict__ o) {
  long s = (long)gridDim.x * blockDim.x;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += s) o[t] = (double)a[t];
}

template <typename R>
__global__ void k_cvt_in(long n, const double* __restrict__ a, R* __restrict__ o) {
  long s = (long)gridDim.x * blockDim.x;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += s) o[t] = (R)a[t];
}

// The coefficients of centre (i, j, k) (flat index t) into c: the planes of a
// Coef (k_coef), or the adjoint's slots for the same values.
template <int CIJ, typename R, typename Out>
__device__ __forceinline__ void coef_at(const Geo<R>& g, const Par& P, const CF<R>& ub, const Out& c, int i, int j,
                                        int k, int t) {
  const auto UR = ub.f[1];
  const auto UT = ub.f[2];
  const auto UP = ub.f[3];
  // thermodynamics from background + perturbation.  The density perturbation
  // rho - rho_ref = (p' T_ref - (p_ref + pi_inf) T') / (Rg T_ref T) has no
  // cancellation between large terms, so the bulk type keeps its relative
  // precision for it.
  R pref = g.pcen[i], Tref = g.Tcen[i];
  R pp = ub.f[0][t], Tp = ub.f[4][t];
  Thermo<R> th = thermo(g, P, i, pp, Tp);
  R iRg = pick<R>(1.0 / P.Rg, P.iRg_f);
  R itb = sdiv(R(1), th.Tb);
  c.Pb[t] = th.Pb;
  c.Tb[t] = th.Tb;
  c.rho[t] = th.rho;
  c.drho[t] = sdiv((pp * Tref - pref * Tp) * itb * iRg, Tref);
  c.beta[t] = th.beta;
  R ur = hr<CIJ>(g, UR, i, j, k), ut = ht<CIJ>(g, UT, i, j, k), up = hp<CIJ>(g, UP, i, j, k);
  c.uc0[t] = ur; c.uc1[t] = ut; c.uc2[t] = up;
  R ir = g.irc[i], is = g.isc[j], cot = g.cotc[j], h = R(0.5);
  c.grr[t] = (vr<CIJ>(g, UR, i + 1, j, k) - vr<CIJ>(g, UR, i, j, k)) * g.idr;
  c.gtt[t] = (vt<CIJ>(g, UT, i, j + 1, k) - vt<CIJ>(g, UT, i, j, k)) * ir * g.idth + ur * ir;
  c.gpp[t] = (vp<CIJ>(g, UP, i, j, k + 1) - vp<CIJ>(g, UP, i, j, k)) * ir * is * g.idph + ur * ir + ut * cot * ir;
  R grt = (ht<CIJ>(g, UT, i + 1, j, k) - ht<CIJ>(g, UT, i - 1, j, k)) * h * g.idr;
  R gtr = (hr<CIJ>(g, UR, i, j + 1, k) - hr<CIJ>(g, UR, i, j - 1, k)) * h * ir * g.idth - ut * ir;
  R grp = (hp<CIJ>(g, UP, i + 1, j, k) - hp<CIJ>(g, UP, i - 1, j, k)) * h * g.idr;
  R gpr = (hr<CIJ>(g, UR, i, j, k + 1) - hr<CIJ>(g, UR, i, j, k - 1)) * h * ir * is * g.idph - up * ir;
  R gtp = (hp<CIJ>(g, UP, i, j + 1, k) - hp<CIJ>(g, UP, i, j - 1, k)) * h * ir * g.idth;
  R gpt = (ht<CIJ>(g, UT, i, j, k + 1) - ht<CIJ>(g, UT, i, j, k - 1)) * h * ir * is * g.idph - up * cot * ir;
  c.srt[t] = grt + gtr;
  c.srp[t] = grp + gpr;
  c.stp[t] = gtp + gpt;
  c.dvr[t] = (g.rf[i + 1] * g.rf[i + 1] * UR[IRf(g, i + 1, j, k)] - g.rf[i] * g.rf[i] * UR[IRf(g, i, j, k)]) * ir * ir
           * g.idr;
  c.dvt[t] = (g.sf[j + 1] * UT[ITf(g, i, j + 1, k)] - g.sf[j] * UT[ITf(g, i, j, k)]) * ir * is * g.idth;
  c.dvp[t] = (vp<CIJ>(g, UP, i, j, k + 1) - vp<CIJ>(g, UP, i, j, k)) * ir * is * g.idph;
}

// The stencil kernels run on tiles of TK x TJ x TI points (phi fastest; 128
// threads; the shape is set per context, sph_set_tile).  A block takes the
// fast path when its whole tile has its +-2 neighbourhood in r and theta
// inside the grid (a uniform choice).  On the 128 x 256 x 256 workload the
// tile shape made no measurable difference (128x1x1 to 16x4x2 all within 3 %),
// so the default is one phi row; the ensemble's autotuner picks it per grid
// shape.
template <typename G>
__device__ __forceinline__ bool tile_inner_at(const G& g, int i0, int j0, int ti, int tj) {
  return inner_ij(g, i0, j0) && inner_ij(g, i0 + ti - 1, j0 + tj - 1);
}
template <typename G>
__device__ __forceinline__ bool tile_inner(const G& g) {
  return tile_inner_at(g, blockIdx.z * blockDim.z, blockIdx.y * blockDim.y, (int)blockDim.z, (int)blockDim.y);
}
// The FP32 stencil kernels are bound by load latency: full occupancy (16
// blocks of 128 threads, 32 registers) pays for its few register spills
// (measured: the right-hand side 17 % faster than at 64 registers).  The FP64
// instantiations keep their registers: they are bound by the FP64 pipe, and
// capping them at 128, 96 or 80 registers (up to 6 blocks an SM) left the
// FP64 right-hand side at 20.8 ms per step.
#define STENCIL_MINB(R) (sizeof(R) == 4 ? 16 : 1)

// grid of tiles of tj x ti rows of phi points (128 / (tj ti) each) over an
// nk x nj x ni index box
static dim3 tile_grid_of(int tj, int ti, int nk, int nj, int ni) {
  int tk = 128 / (tj * ti);
  return dim3((nk + tk - 1) / tk, (nj + tj - 1) / tj, (ni + ti - 1) / ti);
}
#define tile_grid(nk, nj, ni) tile_grid_of(c->tile_j, c->tile_i, nk, nj, ni)
#define TILE_BLOCK dim3(128 / (c->tile_j * c->tile_i), c->tile_j, c->tile_i)

// one block per tile
template <typename R, bool W>
__global__ void __launch_bounds__(128, STENCIL_MINB(R)) k_coef(Geo<R> g, Par P, CF<R> ub, Coef<R> c) {
  int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
      i = blockIdx.z * blockDim.z + threadIdx.z;
  bool inner = tile_inner(g) && !g.hasw;  // with wall data every tile takes the checked path
  if (k >= g.np || j >= g.nt || i >= g.nr) return;
  int t = IC(g, i, j, k);
  if (inner) coef_at<0>(g, P, ub, c, i, j, k, t);
  else coef_at<W ? 2 : 1>(g, P, ub, c, i, j, k, t);
}

// div(Ubar) at centre (i,j,k), in FP64 from U^n and U^k (Ubar = (U^n+U^k)/2).
__device__ __forceinline__ double div_ubar(const Geo<double>& g, const CF<double>& un, const CF<double>& uk, int i,
                                           int j, int k) {
  const double *ur0 = un.f[1], *ur1 = uk.f[1], *ut0 = un.f[2], *ut1 = uk.f[2], *up0 = un.f[3], *up1 = uk.f[3];
  int a0 = IRf(g, i, j, k), a1 = IRf(g, i + 1, j, k);
  int b0 = ITf(g, i, j, k), b1 = ITf(g, i, j + 1, k);
  int kp = g.per ? wrapk(g, k + 1) : k + 1;
  int c0 = IPf(g, i, j, k), c1 = IPf(g, i, j, kp);
  double ir = g.irc[i], is = g.isc[j];
  double f0 = g.rf[i] * g.rf[i], f1 = g.rf[i + 1] * g.rf[i + 1];
  double dr_ = (f1 * (ur0[a1] + ur1[a1]) - f0 * (ur0[a0] + ur1[a0])) * ir * ir * g.idr;
  double dt_ = (g.sf[j + 1] * (ut0[b1] + ut1[b1]) - g.sf[j] * (ut0[b0] + ut1[b0])) * ir * is * g.idth;
  double dp_ = ((up0[c1] + up1[c1]) - (up0[c0] + up1[c0])) * ir * is * g.idph;
  return 0.5 * (dr_ + dt_ + dp_);
}

// div(Ubar) at centre (i,j,k) in FP32 mode, from the pair (hi = Ubar, lo) of the
// velocity components: each face flux and each difference is carried as a pair,
// so the cancellation of nearly equal fluxes (and of the three directions
// against each other) at low Mach number costs no accuracy.
__device__ __forceinline__ float div_ubar_ff(const Geo<float>& g, const CF<float>& ub, const CF<float>& ul, int i,
                                             int j, int k) {
  int a0 = IRf(g, i, j, k), a1 = IRf(g, i + 1, j, k);
  int b0 = ITf(g, i, j, k), b1 = ITf(g, i, j + 1, k);
  int kp = g.per ? wrapk(g, k + 1) : k + 1;
  int c0 = IPf(g, i, j, k), c1 = IPf(g, i, j, kp);
  float ir = g.irc[i], is = g.isc[j];
  float h0, l0, h1, l1, dh, dl, th, tl, sh, sl;
  // r: (rf1^2 u1 - rf0^2 u0) / rc^2 / dr
  ff_mul(g.rf2h[i + 1], g.rf2l[i + 1], ub.f[1][a1], ul.f[1][a1], h1, l1);
  ff_mul(g.rf2h[i], g.rf2l[i], ub.f[1][a0], ul.f[1][a0], h0, l0);
  ff_sub(h1, l1, h0, l0, dh, dl);
  float cr = ir * ir * g.idr;
  ff_mul(dh, dl, cr, 0.f, sh, sl);
  // theta: (sf1 u1 - sf0 u0) / (rc sc dtheta)
  ff_mul(g.sfh[j + 1], g.sfl[j + 1], ub.f[2][b1], ul.f[2][b1], h1, l1);
  ff_mul(g.sfh[j], g.sfl[j], ub.f[2][b0], ul.f[2][b0], h0, l0);
  ff_sub(h1, l1, h0, l0, dh, dl);
  ff_mul(dh, dl, ir * is * g.idth, 0.f, th, tl);
  ff_add(sh, sl, th, tl, sh, sl);
  // phi: (u1 - u0) / (rc sc dphi)
  ff_sub(ub.f[3][c1], ul.f[3][c1], ub.f[3][c0], ul.f[3][c0], dh, dl);
  ff_mul(dh, dl, ir * is * g.idph, 0.f, th, tl);
  ff_add(sh, sl, th, tl, sh, sl);
  return sh + sl;
}

// div(Ubar) at centre (i,j,k) from Ubar itself (the adjoint's evaluation: the
// FP64 kernels form it from U^n and U^k, the same value up to rounding)
template <typename R>
__device__ __forceinline__ R div_ubar_of(const Geo<R>& g, const CF<R>& ub, int i, int j, int k) {
  int a0 = IRf(g, i, j, k), a1 = IRf(g, i + 1, j, k);
  int b0 = ITf(g, i, j, k), b1 = ITf(g, i, j + 1, k);
  int kp = g.per ? wrapk(g, k + 1) : k + 1;
  int c0 = IPf(g, i, j, k), c1 = IPf(g, i, j, kp);
  auto ir = g.irc[i], is = g.isc[j];
  auto f0 = g.rf[i] * g.rf[i], f1 = g.rf[i + 1] * g.rf[i + 1];
  R dr_ = (f1 * ub.f[1][a1] - f0 * ub.f[1][a0]) * (ir * ir * g.idr);
  R dt_ = (g.sf[j + 1] * ub.f[2][b1] - g.sf[j] * ub.f[2][b0]) * (ir * is * g.idth);
  R dp_ = (ub.f[3][c1] - ub.f[3][c0]) * (ir * is * g.idph);
  return dr_ + dt_ + dp_;
}

// Line rows of the FP64 mode.  The right-hand side evaluates, at every unknown,
// the rows of D_r, D_theta and D_phi at Ubar -- the same rows each sweep's line
// matrix I + tau/2 D_d is assembled from.  In the FP64 mode the arithmetic, not
// memory, bounds the step, so the right-hand side stores the rows it has formed
// and the sweeps read them instead of forming them again (45 doubles a cell).
//   c[d]: 12 planes over the centres, the p- and T-rows of D_d: p-row wp0, wp2,
//         wT0, wT1, wT2, v0, v1 (wp1 is zero: advection has no diagonal); T-row
//         wT0, wT1, wT2, v0, v1; v_q = a gd_q + wv_q (the u_d couplings);
//   f[d]: 5 planes over the d-faces, the normal-velocity row of D_d (wp0, wp1,
//         wu0, wu1, wu2);
//   s[c]: 6 planes over the c-faces, the rows of velocity component c along its
//         two transverse directions in increasing order (3 weights each).
// NoRows (every other caller) stores nothing.
struct NoRows { static constexpr bool on = false; };
struct Rows64 {
  static constexpr bool on = true;
  double* c[3];
  double* f[3];
  double* s[3];
  long nc, nf[3];  // centres; faces of each kind
};
// slot of direction d among the transverse directions of component cc
__host__ __device__ constexpr int trans_slot(int cc, int d) { return d < cc ? d : d - 1; }

template <typename RowsT, typename R>
__device__ __forceinline__ void rows_put_c(const RowsT& o, int d, int isT, int t, const RowC<R>& w) {
  if constexpr (RowsT::on && std::is_same<R, double>::value) {
    double* p = o.c[d] + t;
    const long n = o.nc;
    if (!isT) {
      p[0] = w.wp[0]; p[n] = w.wp[2]; p[2 * n] = w.wT[0]; p[3 * n] = w.wT[1]; p[4 * n] = w.wT[2];
      p[5 * n] = w.a * w.gd[0] + w.wv[0]; p[6 * n] = w.a * w.gd[1] + w.wv[1];
    } else {
      p[7 * n] = w.wT[0]; p[8 * n] = w.wT[1]; p[9 * n] = w.wT[2];
      p[10 * n] = w.a * w.gd[0] + w.wv[0]; p[11 * n] = w.a * w.gd[1] + w.wv[1];
    }
  }
}
template <typename RowsT, typename R>
__device__ __forceinline__ void rows_put_f(const RowsT& o, int d, int t, const R* wp, const R* wu) {
  if constexpr (RowsT::on && std::is_same<R, double>::value) {
    double* p = o.f[d] + t;
    const long n = o.nf[d];
    p[0] = wp[0]; p[n] = wp[1]; p[2 * n] = wu[0]; p[3 * n] = wu[1]; p[4 * n] = wu[2];
  }
}
template <typename RowsT, typename R>
__device__ __forceinline__ void rows_put_s(const RowsT& o, int cc, int d, int t, const R* w) {
  if constexpr (RowsT::on && std::is_same<R, double>::value) {
    const long n = o.nf[cc];
    double* p = o.s[cc] + 3 * trans_slot(cc, d) * n + t;
    p[0] = w[0]; p[n] = w[1]; p[2 * n] = w[2];
  }
}

// R = -(U^k - U^n) - tau (N(Ubar) + G - S) for the p- and T-rows: one thread per
// centre; written to Rout.f[0][t], Rout.f[4][t] (a field pair, or the adjoint's
// slots).
template <int CIJ, typename R, typename Out, typename RowsT = NoRows>
__device__ __forceinline__ void rhs_c_at(const Geo<R>& g, const Geo<double>& gd, const Par& P, const Coef<R>& c,
                                         const CF<R>& ub, const CF<R>& ul, const CF<double>& un, const CF<double>& uk,
                                         const CF<R>& D, int hasD, const CF<double>& src, int has_src, R tau,
                                         const Out& Rout, int i, int j, int k, int t, const RowsT& rows = RowsT()) {
  const auto Pp = ub.f[0];
  const auto UR = ub.f[1];
  const auto UT = ub.f[2];
  const auto UP = ub.f[3];
  const auto TT = ub.f[4];
  R mu = pick<R>(P.mu, P.mu_f), gm = pick<R>(P.gamma, P.gamma_f);
  R ir = g.irc[i];
  R accp = R(0), accT = R(0);
  R ap = R(0), aT = R(0);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int di = d == 0, dj = d == 1, dk = d == 2;
    R pv[3], Tv[3], uv[2];
#pragma unroll
    for (int s = -1; s <= 1; s++) {
      pv[s + 1] = cpert<CIJ>(g, Pp, i + s * di, j + s * dj, k + s * dk);
      Tv[s + 1] = cpert<CIJ>(g, TT, i + s * di, j + s * dj, k + s * dk);
    }
    if (d == 0) { uv[0] = UR[IRf(g, i, j, k)]; uv[1] = UR[IRf(g, i + 1, j, k)]; }
    else if (d == 1) { uv[0] = UT[ITf(g, i, j, k)]; uv[1] = UT[ITf(g, i, j + 1, k)]; }
    else { uv[0] = vp<CIJ>(g, UP, i, j, k); uv[1] = vp<CIJ>(g, UP, i, j, k + 1); }
    RowC<R> w;
    row_c(g, P, c, d, 0, i, j, k, w);
    rows_put_c(rows, d, 0, t, w);
    accp += w.wp[0] * pv[0] + w.wp[2] * pv[2] + w.wT[0] * Tv[0] + w.wT[1] * Tv[1] + w.wT[2] * Tv[2]
          + w.wv[0] * uv[0] + w.wv[1] * uv[1];
    if (d == 0) accp += w.adv * g.dbgp[i] - w.dif * g.lapT[i];
    ap = w.a;
    row_c(g, P, c, d, 1, i, j, k, w);
    rows_put_c(rows, d, 1, t, w);
    accT += w.wT[0] * Tv[0] + w.wT[1] * Tv[1] + w.wT[2] * Tv[2] + w.wv[0] * uv[0] + w.wv[1] * uv[1];
    if (d == 0) accT += w.adv * g.dbgT[i] - w.dif * g.lapT[i];
    aT = w.a;
  }
  R divu;
  if constexpr (is_f32<R>) divu = div_ubar_ff(g, ub, ul, i, j, k);
  else if constexpr (std::is_same<R, double>::value) divu = div_ubar(gd, un, uk, i, j, k);
  else divu = div_ubar_of(g, ub, i, j, k);
  // Cross terms of the viscous dissipation: the centred derivative sums
  // d_r u_t + d_t u_r / r, d_r u_p + d_p u_r / (r sin), d_t u_p / r + d_p u_t / (r sin)
  // of the centre-averaged velocities.  k_coef forms the same sums minus the
  // metric terms u_t / r, u_p / r, u_p cot / r (S_rt, S_rp, S_tp, with the same
  // accessors in the same tiles), so they are S + those terms.
  R srt = c.srt[t], srp = c.srp[t], stp = c.stp[t];
  R ut = htc<CIJ>(g, c, UT, i, j, k), up = hpc<CIJ>(g, c, UP, i, j, k);
  R xrt = srt + ut * ir, xrp = srp + up * ir, xtp = stp + up * g.cotc[j] * ir;
  R cross = srt * xrt + srp * xrp + stp * xtp;
  accp += -mu * (gm - R(1)) * cross;
  accT += -mu * c.beta[t] * cross;
  R Np = ap * divu + accp, NT = aT * divu + accT;
  if (has_src) { Np -= to_bulk<R>(src.f[0][t]); NT -= to_bulk<R>(src.f[4][t]); }
  R d0 = hasD ? D.f[0][t] : R(0), d4 = hasD ? D.f[4][t] : R(0);
  Rout.f[0][t] = -d0 - tau * Np;
  Rout.f[4][t] = -d4 - tau * NT;
}

// one block per tile.  FP64: at least SPH_RHSC64_MINB blocks of 128 threads
// per SM (the compiler would otherwise take ~190 registers a thread for the
// centre rows it keeps live until their stores, leaving two blocks per SM).
#ifndef SPH_RHSC64_MINB
#define SPH_RHSC64_MINB 4
#endif
template <typename R, bool W>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? STENCIL_MINB(R) : SPH_RHSC64_MINB) k_rhs_c(Geo<R> g, Geo<double> gd, Par P, Coef<R> c, CF<R> ub, CF<R> ul,
                                               CF<double> un, CF<double> uk, CF<R> D, int hasD, CF<double> src,
                                               int has_src, R tau, MF<R> Rout, Rows64 rows) {
  int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
      i = blockIdx.z * blockDim.z + threadIdx.z;
  bool inner = tile_inner(g) && !g.hasw;  // with wall data every tile takes the checked path
  if (k >= g.np || j >= g.nt || i >= g.nr) return;
  int t = IC(g, i, j, k);
  if constexpr (std::is_same<R, double>::value) {  // the FP64 mode stores its line rows
    if (inner) rhs_c_at<0>(g, gd, P, c, ub, ul, un, uk, D, hasD, src, has_src, tau, Rout, i, j, k, t, rows);
    else rhs_c_at<W ? 2 : 1>(g, gd, P, c, ub, ul, un, uk, D, hasD, src, has_src, tau, Rout, i, j, k, t, rows);
  } else {
    if (inner) rhs_c_at<0>(g, gd, P, c, ub, ul, un, uk, D, hasD, src, has_src, tau, Rout, i, j, k, t);
    else rhs_c_at<W ? 2 : 1>(g, gd, P, c, ub, ul, un, uk, D, hasD, src, has_src, tau, Rout, i, j, k, t);
  }
}

// R for the momentum row of component D on its faces: one thread per face
// (zero on wall faces, which are not unknowns); written to Rout.f[1 + D][t].
template <int CIJ, int D, typename R, typename Out, typename RowsT = NoRows>
__device__ __forceinline__ void rhs_u_at(const Geo<R>& g, const Par& P, const Coef<R>& c, const CF<R>& ub,
                                         const CF<R>& Dv, int hasD, const CF<double>& src, int has_src, R tau,
                                         const Out& Rout, int i, int j, int k, int t, const RowsT& rows = RowsT()) {
  const auto Pp = ub.f[0];
  const auto UR = ub.f[1];
  const auto UT = ub.f[2];
  const auto UP = ub.f[3];
  R mu = pick<R>(P.mu, P.mu_f), om = pick<R>(P.omega, P.omega_f), h = R(0.5);
  R wp[2], wu[3], w[3];
  R acc;
  if (D == 0) {
    row_f(g, P, c, UR, 0, i, j, k, wp, wu);
    rows_put_f(rows, 0, t, wp, wu);
    acc = wp[1] * (cpert<CIJ>(g, Pp, i, j, k) - cpert<CIJ>(g, Pp, i - 1, j, k))
        + wu[0] * UR[IRf(g, i - 1, j, k)] + wu[1] * UR[t] + wu[2] * UR[IRf(g, i + 1, j, k)];
    row_s<CIJ>(g, P, c, ub, 0, 1, i, j, k, w);
    rows_put_s(rows, 0, 1, t, w);
    acc += w[0] * vr<CIJ>(g, UR, i, j - 1, k) + w[1] * UR[t] + w[2] * vr<CIJ>(g, UR, i, j + 1, k);
    row_s<CIJ>(g, P, c, ub, 0, 2, i, j, k, w);
    rows_put_s(rows, 0, 2, t, w);
    acc += w[0] * vr<CIJ>(g, UR, i, j, k - 1) + w[1] * UR[t] + w[2] * vr<CIJ>(g, UR, i, j, k + 1);
    // hydrostatic part: (1/rho_f) d p_ref/dr + g = (1 - b) e + g b, b = 1 - rho_ref,f / rho_f
    int c0 = IC(g, i - 1, j, k), c1 = IC(g, i, j, k);
    R rs = c.rho[c0] + c.rho[c1];
    R bf = sdiv(c.drho[c0] + c.drho[c1], rs);
    acc += (R(1) - bf) * g.ehyd[i] + pick<R>(P.g, P.g_f) * bf;
    // D_M
    R irf = g.irf[i], s = g.sc[j];
    R irh = sdiv(R(2), rs);
    R utf = h * (htc<CIJ>(g, c, UT, i - 1, j, k) + htc<CIJ>(g, c, UT, i, j, k));
    R upf = h * (hpc<CIJ>(g, c, UP, i - 1, j, k) + hpc<CIJ>(g, c, UP, i, j, k));
    // theta and phi parts of div(Ubar) at the centres i - 1, i
    R Q[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
      int cm = IC(g, i - 1 + q, j, k);
      Q[q] = c.dvt[cm] + c.dvp[cm];
    }
    acc += -utf * utf * irf - upf * upf * irf + R(2) * mu * irh * UR[t] * irf * irf - R(2) * om * s * upf
         - mu * irh * R(1.0 / 3.0) * g.idr * (Q[1] - Q[0]) + mu * irh * irf * (Q[0] + Q[1]);
  } else if (D == 1) {
    R ir = g.irc[i];
    row_f(g, P, c, UT, 1, i, j, k, wp, wu);
    rows_put_f(rows, 1, t, wp, wu);
    acc = wp[1] * (cpert<CIJ>(g, Pp, i, j, k) - cpert<CIJ>(g, Pp, i, j - 1, k))
        + wu[0] * UT[ITf(g, i, j - 1, k)] + wu[1] * UT[t] + wu[2] * UT[ITf(g, i, j + 1, k)];
    row_s<CIJ>(g, P, c, ub, 1, 0, i, j, k, w);
    rows_put_s(rows, 1, 0, t, w);
    acc += w[0] * vt<CIJ>(g, UT, i - 1, j, k) + w[1] * UT[t] + w[2] * vt<CIJ>(g, UT, i + 1, j, k);
    row_s<CIJ>(g, P, c, ub, 1, 2, i, j, k, w);
    rows_put_s(rows, 1, 2, t, w);
    acc += w[0] * vt<CIJ>(g, UT, i, j, k - 1) + w[1] * UT[t] + w[2] * vt<CIJ>(g, UT, i, j, k + 1);
    R isfj = g.isf[j], cfj = g.cf[j], cotf = g.cotf[j];
    R irh = sdiv(R(2), rho_at(g, c, i, j - 1, k) + rho_at(g, c, i, j, k));
    R ubt = UT[t];
    R upf = h * (hpc<CIJ>(g, c, UP, i, j - 1, k) + hpc<CIJ>(g, c, UP, i, j, k));
    R vrf = h * (hrc<CIJ>(g, c, UR, i, j - 1, k) + hrc<CIJ>(g, c, UR, i, j, k));
    // r and phi parts of div(Ubar) at the centres j - 1, j; dpf = the mean of
    // their d_p u_p (the phi part times r sin)
    R Dr[2], Dp[2], dpf = R(0);
#pragma unroll
    for (int q = 0; q < 2; q++) {
      int m = j - 1 + q, cm = IC(g, i, m, k);
      Dr[q] = c.dvr[cm];
      Dp[q] = c.dvp[cm];
      dpf += h * Dp[q] * g.rc[i] * g.sc[m];
    }
    acc += ubt * vrf * ir - upf * upf * cotf * ir + mu * irh * ubt * ir * ir * isfj * isfj - R(2) * om * cfj * upf
         - mu * irh * R(1.0 / 3.0) * ir * g.idth * ((Dr[1] - Dr[0]) + (Dp[1] - Dp[0]))
         - mu * irh * (R(2) * ir * ir * g.idth * (hrc<CIJ>(g, c, UR, i, j, k) - hrc<CIJ>(g, c, UR, i, j - 1, k))
                       - R(2) * cfj * ir * ir * isfj * isfj * dpf);
  } else {
    R ir = g.irc[i], is = g.isc[j], cot = g.cotc[j];
    row_f(g, P, c, UP, 2, i, j, k, wp, wu);
    rows_put_f(rows, 2, t, wp, wu);
    acc = wp[1] * (cpert<CIJ>(g, Pp, i, j, k) - cpert<CIJ>(g, Pp, i, j, k - 1))
        + wu[0] * vp<CIJ>(g, UP, i, j, k - 1) + wu[1] * UP[t] + wu[2] * vp<CIJ>(g, UP, i, j, k + 1);
    row_s<CIJ>(g, P, c, ub, 2, 0, i, j, k, w);
    rows_put_s(rows, 2, 0, t, w);
    acc += w[0] * vp<CIJ>(g, UP, i - 1, j, k) + w[1] * UP[t] + w[2] * vp<CIJ>(g, UP, i + 1, j, k);
    row_s<CIJ>(g, P, c, ub, 2, 1, i, j, k, w);
    rows_put_s(rows, 2, 1, t, w);
    acc += w[0] * vp<CIJ>(g, UP, i, j - 1, k) + w[1] * UP[t] + w[2] * vp<CIJ>(g, UP, i, j + 1, k);
    R s = g.sc[j], cj = g.cc[j];
    R irh = sdiv(R(2), rho_at(g, c, i, j, k - 1) + rho_at(g, c, i, j, k));
    R ubp = UP[t];
    R vrf = h * (hrc<CIJ>(g, c, UR, i, j, k - 1) + hrc<CIJ>(g, c, UR, i, j, k));
    R vtf = h * (htc<CIJ>(g, c, UT, i, j, k - 1) + htc<CIJ>(g, c, UT, i, j, k));
    // r and theta parts of div(Ubar) at the centres k - 1, k (interior faces: real
    // centres, wrapped on a periodic line)
    R Dr[2], Dt[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
      int m = k - 1 + q;
      if (g.per) m = wrapk(g, m);
      int cm = IC(g, i, j, m);
      Dr[q] = c.dvr[cm];
      Dt[q] = c.dvt[cm];
    }
    acc += ubp * vtf * cot * ir + ubp * vrf * ir + mu * irh * ubp * ir * ir * is * is + R(2) * om * (cj * vtf + s * vrf)
         - mu * irh * R(1.0 / 3.0) * ir * is * g.idph * ((Dr[1] - Dr[0]) + (Dt[1] - Dt[0]))
         - mu * irh * (R(2) * ir * ir * is * g.idph * (hrc<CIJ>(g, c, UR, i, j, k) - hrc<CIJ>(g, c, UR, i, j, k - 1))
                       + R(2) * cj * ir * ir * is * is * g.idph * (htc<CIJ>(g, c, UT, i, j, k) - htc<CIJ>(g, c, UT, i, j, k - 1)));
  }
  if (has_src) acc -= to_bulk<R>(src.f[1 + D][t]);
  R dd = hasD ? Dv.f[1 + D][t] : R(0);
  Rout.f[1 + D][t] = -dd - tau * acc;
}

// one block per tile of faces; zero on wall faces, which are not unknowns
template <typename R, int D, bool W>
__global__ void __launch_bounds__(128, STENCIL_MINB(R)) k_rhs_u(Geo<R> g, Par P, Coef<R> c, CF<R> ub, CF<R> Dv, int hasD,
                                               CF<double> src, int has_src, R tau, MF<R> Rout, Rows64 rows) {
  int nj = g.nt + (D == 1), nk = D == 2 ? g.npf : g.np;
  int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y,
      i = blockIdx.z * blockDim.z + threadIdx.z;
  bool inner = tile_inner(g) && !g.hasw;  // with wall data every tile takes the checked path
  if (k >= nk || j >= nj || i >= g.nr + (D == 0)) return;
  int t = (i * nj + j) * nk + k;
  bool wall = D == 0 ? (i == 0 || i == g.nr) : D == 1 ? (j == 0 || j == g.nt) : (!g.per && (k == 0 || k == g.np));
  if (wall) { Rout.f[1 + D][t] = R(0); return; }
  if constexpr (std::is_same<R, double>::value) {  // the FP64 mode stores its line rows
    if (inner) rhs_u_at<0, D>(g, P, c, ub, Dv, hasD, src, has_src, tau, Rout, i, j, k, t, rows);
    else rhs_u_at<W ? 2 : 1, D>(g, P, c, ub, Dv, hasD, src, has_src, tau, Rout, i, j, k, t, rows);
  } else {
    if (inner) rhs_u_at<0, D>(g, P, c, ub, Dv, hasD, src, has_src, tau, Rout, i, j, k, t);
    else rhs_u_at<W ? 2 : 1, D>(g, P, c, ub, Dv, hasD, src, has_src, tau, Rout, i, j, k, t);
  }
}

// ------------------------------------------------------------ line solvers

template <typename R>
__device__ __forceinline__ bool inv3(const R* S, R* I) {
  R c00 = S[4] * S[8] - S[5] * S[7];
  R c01 = S[5] * S[6] - S[3] * S[8];
  R c02 = S[3] * S[7] - S[4] * S[6];
  R det = S[0] * c00 + S[1] * c01 + S[2] * c02;
  if (det == R(0) || !isfinite(det)) return false;
  R id = sdiv(R(1), det);
  I[0] = c00 * id; I[3] = c01 * id; I[6] = c02 * id;
  I[1] = (S[2] * S[7] - S[1] * S[8]) * id;
  I[4] = (S[0] * S[8] - S[2] * S[6]) * id;
  I[7] = (S[1] * S[6] - S[0] * S[7]) * id;
  I[2] = (S[1] * S[5] - S[2] * S[4]) * id;
  I[5] = (S[2] * S[3] - S[0] * S[5]) * id;
  I[8] = (S[0] * S[4] - S[1] * S[3]) * id;
  return true;
}

// position of cell m on the line (a, b) along d
__device__ __forceinline__ void line_pos(int d, int a, int b, int m, int& i, int& j, int& k) {
  if (d == 0) { i = m; j = a; k = b; }
  else if (d == 1) { i = a; j = m; k = b; }
  else { i = a; j = b; k = m; }
}

template <typename G>
__device__ __forceinline__ int face_idx(const G& g, int d, int i, int j, int k) {
  return d == 0 ? IRf(g, i, j, k) : d == 1 ? ITf(g, i, j, k) : IPf(g, i, j, k);
}

// Assemble block m of (I + h D_d) on a line from the loaded centre values (cq)
// and, when the line has face m+1 (m < n-1 or cyclic), the face values fq at
// face coordinates (fi, fj); h = tau/2.
template <typename R>
__device__ __forceinline__ void assemble_pts(const Geo<R>& g, const Par& P, const CPt<R>& cq, const FPt<R>& fq, int d,
                                             int n, int cyc, int m, int i, int j, int fi, int fj, R h, R* A, R* B,
                                             R* C) {
  RowC<R> w;
#pragma unroll
  for (int q = 0; q < 9; q++) { A[q] = R(0); B[q] = R(0); C[q] = R(0); }
  row_cw(g, P, cq, d, 0, i, j, w);
  A[0] = h * w.wp[0]; A[1] = h * w.wT[0]; A[2] = h * (w.a * w.gd[0] + w.wv[0]);
  B[0] = h * w.wp[1]; B[1] = h * w.wT[1]; B[2] = h * (w.a * w.gd[1] + w.wv[1]);
  C[0] = h * w.wp[2]; C[1] = h * w.wT[2];
  row_cw(g, P, cq, d, 1, i, j, w);
  A[4] = h * w.wT[0]; A[5] = h * (w.a * w.gd[0] + w.wv[0]);
  B[4] = h * w.wT[1]; B[5] = h * (w.a * w.gd[1] + w.wv[1]);
  C[4] = h * w.wT[2];
  if (m < n - 1 || cyc) {
    R fp[2], fu[3];
    row_fw(g, P, fq, d, fi, fj, fp, fu);
    A[8] = h * fu[0];
    B[6] = h * fp[0]; B[8] = h * fu[1];
    C[6] = h * fp[1]; C[8] = h * fu[2];
  }
  B[0] += R(1); B[4] += R(1); B[8] += R(1);
  if (!cyc) {
    if (m == 0) {
      B[0] += A[0]; B[1] += A[1]; B[3] += A[3]; B[4] += A[4];
#pragma unroll
      for (int q = 0; q < 9; q++) A[q] = R(0);
    }
    if (m == n - 1) {
      B[0] += C[0]; B[1] += C[1]; B[3] += C[3]; B[4] += C[4];
#pragma unroll
      for (int q = 0; q < 9; q++) C[q] = R(0);
      B[2] = R(0); B[5] = R(0);
      A[8] = R(0); B[6] = R(0); B[7] = R(0); B[8] = R(1);
    }
  }
}

// face m+1 of cell m on a line along d (wrapping to 0 on a cyclic line)
__device__ __forceinline__ void next_face(int d, int n, int m, int i, int j, int k, int& fi, int& fj, int& fk) {
  fi = i; fj = j; fk = k;
  if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = (m + 1 == n) ? 0 : m + 1;
}

// Assemble block m of (I + h D_d) on a line; h = tau/2.
template <typename R>
__device__ void assemble_block(const Geo<R>& g, const Par& P, const Coef<R>& c, const CF<R>& ub, int d, int n, int cyc,
                               int m, int i, int j, int k, R h, R* A, R* B, R* C) {
  CPt<R> cq = load_c(c, d, IC(g, i, j, k));
  FPt<R> fq = {R(1), R(1), R(0)};
  int fi, fj, fk;
  next_face(d, n, m, i, j, k, fi, fj, fk);
  if (m < n - 1 || cyc) fq = load_f(g, c, ub.f[1 + d], d, fi, fj, fk);
  assemble_pts(g, P, cq, fq, d, n, cyc, m, i, j, fi, fj, h, A, B, C);
}

template <typename R>
struct SweepArgs {
  Geo<R> g; Par P; Coef<R> c; CF<R> ub;
  int d; R h;
  CF<R> rhs;              // right-hand side fields
  MF<R> x;                // output increments (mode 0)
  int update;             // mode 1: uk = base + x (FP64), accumulate norms
  CF<double> base; MF<double> uk;
  R* scr;                 // scratch
  int scr_off[3];         // offsets of the three kinds
  int nl[3];              // lines per kind
  int a0[3], nb[3], b0[3];
  double* acc;            // 5 sums of squares (mode 1)
  int* flag;
  Rows64 rows;            // FP64 mode: the line rows the right-hand side stored
};

// Per-thread sums of squares of the increments, per field (the iteration
// residual).  FP64 mode: plain FP64 sums.  FP32 mode: each sum is an
// unevaluated pair hi + lo (the square's rounding error by FMA, the addition's
// by two_sum), ~48 bits like an FP64 sum, on the FP32 pipe; the warp's pairs are
// combined the same way and reach the FP64 accumulator as hi + lo.
template <typename R>
struct SqSum {
  R h[5] = {0, 0, 0, 0, 0};
  __device__ __forceinline__ void add(int f, R r) { h[f] += r * r; }
  __device__ __forceinline__ double warp_total(int f) const {
    R v = h[f];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return f2d(v);
  }
};
template <>
struct SqSum<float> {
  float h[5] = {0, 0, 0, 0, 0}, l[5] = {0, 0, 0, 0, 0};
  __device__ __forceinline__ void add(int f, float r) {
    float p = r * r, e = fmaf(r, r, -p), s, t;
    two_sum(h[f], p, s, t);
    h[f] = s;
    l[f] += t + e;
  }
  __device__ __forceinline__ double warp_total(int f) const {
    float hv = h[f], lv = l[f];
    for (int o = 16; o > 0; o >>= 1) {
      float ho = __shfl_down_sync(0xffffffffu, hv, o), lo = __shfl_down_sync(0xffffffffu, lv, o), s, t;
      two_sum(hv, ho, s, t);
      hv = s;
      lv += lo + t;
    }
    return f2d(hv) + f2d(lv);
  }
};
// The same with plain FP32 partial sums per thread (a few squares each: the
// scalar line kernels, whose 48-register budget has no room for the pairs) and
// the pair combination from the warp reduction on.
struct SqSumLite {
  float h[5] = {0, 0, 0, 0, 0};
  __device__ __forceinline__ void add(int f, float r) { h[f] = fmaf(r, r, h[f]); }
  __device__ __forceinline__ double warp_total(int f) const {
    float hv = h[f], lv = 0.f;
    for (int o = 16; o > 0; o >>= 1) {
      float ho = __shfl_down_sync(0xffffffffu, hv, o), lo = __shfl_down_sync(0xffffffffu, lv, o), s, t;
      two_sum(hv, ho, s, t);
      hv = s;
      lv += lo + t;
    }
    return f2d(hv) + f2d(lv);
  }
};

// store a value of field f at flat index idx: x (mode 0) or uk = base + v (mode
// 1, the one FP64 add per value of the mixed path), with the square of v summed
template <typename R, typename V, typename Acc>
__device__ __forceinline__ void put(const SweepArgs<R>& A, int f, int idx, V v, Acc& ss, int* bad) {
  if (!A.update) {
    A.x.f[f][idx] = (R)v;
  } else {
    double nv = A.base.f[f][idx] + f2d(v);
    if (!isfinite(v)) *bad |= FLAG_NONFINITE;  // the state was finite; only a non-finite increment spoils it
    A.uk.f[f][idx] = nv;
    ss.add(f, (R)v);
  }
}
// the update-mode store with the FP64 state value already loaded
template <typename R, typename V, typename Acc>
__device__ __forceinline__ void put_upd(const SweepArgs<R>& A, int f, int idx, double base, V v, Acc& ss, int* bad) {
  if (!isfinite(v)) *bad |= FLAG_NONFINITE;
  A.uk.f[f][idx] = base + f2d(v);
  ss.add(f, (R)v);
}
// wall face of field f: x = 0, or uk = base (mode 1)
template <typename R>
__device__ __forceinline__ void put_wall(const SweepArgs<R>& A, int f, int idx) {
  if (!A.update) A.x.f[f][idx] = R(0);
  else A.uk.f[f][idx] = A.base.f[f][idx];
}

// Blocks of row m of the transposed line matrix: (M^T)_{m,m-1} = C_{m-1}^T,
// (M^T)_{m,m} = B_m^T, (M^T)_{m,m+1} = A_{m+1}^T, wrapping on a cyclic line and
// zero past the ends of a walled one (the adjoint's transposed line solves).
template <typename R>
__device__ __forceinline__ void transposed_blocks(const SweepArgs<R>& S, int d, int n, int cyc, int a, int b, int m,
                                                  R* A, R* B, R* C) {
  R X[9], Y[9], Z[9];
  int i, j, k;
  line_pos(d, a, b, m, i, j, k);
  assemble_block(S.g, S.P, S.c, S.ub, d, n, cyc, m, i, j, k, S.h, X, Y, Z);
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int q = 0; q < 3; q++) B[r * 3 + q] = Y[q * 3 + r];
  int mp = m - 1, mn = m + 1;
  if (cyc) { mp = mp < 0 ? n - 1 : mp; mn = mn == n ? 0 : mn; }
#pragma unroll
  for (int q = 0; q < 9; q++) { A[q] = R(0); C[q] = R(0); }
  if (mp >= 0) {
    line_pos(d, a, b, mp, i, j, k);
    assemble_block(S.g, S.P, S.c, S.ub, d, n, cyc, mp, i, j, k, S.h, X, Y, Z);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int q = 0; q < 3; q++) A[r * 3 + q] = Z[q * 3 + r];
  }
  if (mn < n) {
    line_pos(d, a, b, mn, i, j, k);
    assemble_block(S.g, S.P, S.c, S.ub, d, n, cyc, mn, i, j, k, S.h, X, Y, Z);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int q = 0; q < 3; q++) C[r * 3 + q] = X[q * 3 + r];
  }
}

// One block line along D: solve (I + h D_D) x = rhs (TR: its transpose) by
// block Thomas, Woodbury-corrected on a cyclic line.
template <typename R, int D, bool TR = false>
__device__ void block_line(const SweepArgs<R>& S, int line, int a, int b, SqSum<R>& ss, int* bad) {
  const Geo<R>& g = S.g;
  constexpr int d = D;
  int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
  int cyc = (d == 2 && g.per);
  int nl = S.nl[0];
  R* scr = S.scr + S.scr_off[0];
  const int W = cyc ? 21 : 12;  // C' (9) + d' (3 per right-hand side)
  const int NR = cyc ? 4 : 1;
  R Cp[9], dp[12];
  R GiA[9];                     // cyclic: Gam^{-1} A_0
  // The inputs of cell m + 1 (its centre coefficients, the face values of its
  // row, its right-hand side) are loaded before cell m is eliminated, so that
  // their memory latency overlaps the elimination (the forward pass).
  CPt<R> cqn;
  FPt<R> fqn;
  R r0n = R(0), r4n = R(0), run = R(0);
  auto fetch = [&](int m) {
    int i, j, k, fi, fj, fk;
    line_pos(d, a, b, m, i, j, k);
    const int ic = IC(g, i, j, k);
    cqn = load_c(S.c, d, ic);
    fqn = {R(1), R(1), R(0)};
    run = R(0);
    if (m < n - 1 || cyc) {
      next_face(d, n, m, i, j, k, fi, fj, fk);
      fqn = load_f(g, S.c, S.ub.f[1 + d], d, fi, fj, fk);
      run = S.rhs.f[1 + d][face_idx(g, d, fi, fj, fk)];
    }
    r0n = S.rhs.f[0][ic];
    r4n = S.rhs.f[4][ic];
  };
  if constexpr (!TR) fetch(0);
  for (int m = 0; m < n; m++) {
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    R A[9], B[9], C[9];
    R rr[12];
    if constexpr (TR) {
      transposed_blocks(S, d, n, cyc, a, b, m, A, B, C);
      int ic = IC(g, i, j, k);
      rr[0] = S.rhs.f[0][ic];
      rr[NR] = S.rhs.f[4][ic];
      R ru = R(0);
      if (m < n - 1 || cyc) {
        int fi = i, fj = j, fk = k;
        if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = (m + 1 == n) ? 0 : m + 1;
        ru = S.rhs.f[1 + d][face_idx(g, d, fi, fj, fk)];
      }
      rr[2 * NR] = ru;
    } else {
      const CPt<R> cq = cqn;
      const FPt<R> fq = fqn;
      rr[0] = r0n;
      rr[NR] = r4n;
      rr[2 * NR] = run;
      if (m + 1 < n) fetch(m + 1);
      int fi, fj, fk;
      next_face(d, n, m, i, j, k, fi, fj, fk);
      assemble_pts(g, S.P, cq, fq, d, n, cyc, m, i, j, fi, fj, S.h, A, B, C);
    }
    if (cyc) {
      // right-hand-side columns 1..3 of U = [Gam; 0; ..; C_{n-1}]
      for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) rr[r * NR + 1 + q] = R(0);
      if (m == 0) {
        R Gam[9], Gi[9];
        for (int q = 0; q < 9; q++) Gam[q] = -B[q];
        if (!inv3(Gam, Gi)) { *bad |= FLAG_SINGULAR; return; }
        for (int r = 0; r < 3; r++)
          for (int q = 0; q < 3; q++) GiA[r * 3 + q] = Gi[r * 3] * A[q] + Gi[r * 3 + 1] * A[3 + q] + Gi[r * 3 + 2] * A[6 + q];
        for (int q = 0; q < 9; q++) B[q] -= Gam[q];
        for (int r = 0; r < 3; r++)
          for (int q = 0; q < 3; q++) rr[r * NR + 1 + q] = Gam[r * 3 + q];
      }
      if (m == n - 1) {
        for (int r = 0; r < 3; r++)
          for (int q = 0; q < 3; q++) {
            B[r * 3 + q] -= C[r * 3] * GiA[q] + C[r * 3 + 1] * GiA[3 + q] + C[r * 3 + 2] * GiA[6 + q];
            rr[r * NR + 1 + q] = C[r * 3 + q];
          }
      }
    }
    // S = B - A C'_{m-1};  y = rr - A d'_{m-1}
    R Sm[9], y[12];
    if (m == 0) {
      for (int q = 0; q < 9; q++) Sm[q] = B[q];
      for (int q = 0; q < 3 * NR; q++) y[q] = rr[q];
    } else {
      for (int r = 0; r < 3; r++) {
        for (int q = 0; q < 3; q++)
          Sm[r * 3 + q] = B[r * 3 + q] - (A[r * 3] * Cp[q] + A[r * 3 + 1] * Cp[3 + q] + A[r * 3 + 2] * Cp[6 + q]);
        for (int q = 0; q < NR; q++)
          y[r * NR + q] = rr[r * NR + q] - (A[r * 3] * dp[q] + A[r * 3 + 1] * dp[NR + q] + A[r * 3 + 2] * dp[2 * NR + q]);
      }
    }
    R Si[9];
    if (!inv3(Sm, Si)) { *bad |= FLAG_SINGULAR; return; }
    for (int r = 0; r < 3; r++) {
      for (int q = 0; q < 3; q++)
        Cp[r * 3 + q] = Si[r * 3] * C[q] + Si[r * 3 + 1] * C[3 + q] + Si[r * 3 + 2] * C[6 + q];
      for (int q = 0; q < NR; q++)
        dp[r * NR + q] = Si[r * 3] * y[q] + Si[r * 3 + 1] * y[NR + q] + Si[r * 3 + 2] * y[2 * NR + q];
    }
    if (m < n - 1) {
      R* s = scr + m * W * nl + line;
      for (int q = 0; q < 9; q++) s[q * nl] = Cp[q];
      for (int q = 0; q < 3 * NR; q++) s[(9 + q) * nl] = dp[q];
    }
  }
  // back substitution, all NR columns; the factors of cell m - 1 are loaded
  // before cell m is substituted
  R xs[12];
  for (int q = 0; q < 3 * NR; q++) xs[q] = dp[q];
  R x0[12];
  R Cn[9], dn[12];
  if (n >= 2) {
    const R* s = scr + (n - 2) * W * nl + line;
    for (int q = 0; q < 9; q++) Cn[q] = s[q * nl];
    for (int q = 0; q < 3 * NR; q++) dn[q] = s[(9 + q) * nl];
  }
  for (int m = n - 1; m >= 0; m--) {
    if (m < n - 1) {
      R C_[9], d_[12];
      for (int q = 0; q < 9; q++) C_[q] = Cn[q];
      for (int q = 0; q < 3 * NR; q++) d_[q] = dn[q];
      if (m >= 1) {
        const R* s = scr + (m - 1) * W * nl + line;
        for (int q = 0; q < 9; q++) Cn[q] = s[q * nl];
        for (int q = 0; q < 3 * NR; q++) dn[q] = s[(9 + q) * nl];
      }
      R xn[12];
      for (int r = 0; r < 3; r++)
        for (int q = 0; q < NR; q++)
          xn[r * NR + q] = d_[r * NR + q] - (C_[r * 3] * xs[q] + C_[r * 3 + 1] * xs[NR + q] + C_[r * 3 + 2] * xs[2 * NR + q]);
      for (int q = 0; q < 3 * NR; q++) xs[q] = xn[q];
    }
    if (!cyc) {
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      int ic = IC(g, i, j, k);
      put(S, 0, ic, xs[0], ss, bad);
      put(S, 4, ic, xs[1], ss, bad);
      if (m < n - 1) {
        int fi = i, fj = j, fk = k;
        if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = m + 1;
        put(S, 1 + d, face_idx(g, d, fi, fj, fk), xs[2], ss, bad);
      } else {
        int fi = i, fj = j, fk = k;
        if (d == 0) fi = n; else if (d == 1) fj = n; else fk = n;
        put_wall(S, 1 + d, face_idx(g, d, fi, fj, fk));
        int gi = i, gj = j, gk = k;
        if (d == 0) gi = 0; else if (d == 1) gj = 0; else gk = 0;
        put_wall(S, 1 + d, face_idx(g, d, gi, gj, gk));
      }
    } else {
      // keep x (all columns) in the d'-slots for the Woodbury combination
      R* s = scr + m * W * nl + line;
      for (int q = 0; q < 3 * NR; q++) s[(9 + q) * nl] = xs[q];
      if (m == 0) for (int q = 0; q < 12; q++) x0[q] = xs[q];
    }
  }
  if (cyc) {
    // V^T y = y_0 + GiA y_{n-1};  V^T Z = Z_0 + GiA Z_{n-1};  f = (I + V^T Z)^{-1} V^T y  (FP64)
    const R* sl = scr + (n - 1) * W * nl + line;
    double xl[12], vy[3], vz[9], vi[9], fcor[3];
    for (int q = 0; q < 12; q++) xl[q] = (double)sl[(9 + q) * nl];
    for (int r = 0; r < 3; r++) {
      vy[r] = (double)x0[r * 4] + (double)GiA[r * 3] * xl[0] + (double)GiA[r * 3 + 1] * xl[4] + (double)GiA[r * 3 + 2] * xl[8];
      for (int q = 0; q < 3; q++)
        vz[r * 3 + q] = (double)x0[r * 4 + 1 + q] + (double)GiA[r * 3] * xl[1 + q] + (double)GiA[r * 3 + 1] * xl[5 + q]
                      + (double)GiA[r * 3 + 2] * xl[9 + q] + (r == q ? 1.0 : 0.0);
    }
    if (!inv3(vz, vi)) { *bad |= FLAG_SINGULAR; return; }
    for (int r = 0; r < 3; r++) fcor[r] = vi[r * 3] * vy[0] + vi[r * 3 + 1] * vy[1] + vi[r * 3 + 2] * vy[2];
    for (int m = 0; m < n; m++) {
      const R* s = scr + m * W * nl + line;
      double xv[3];
      for (int r = 0; r < 3; r++) {
        xv[r] = (double)s[(9 + r * 4) * nl];
        for (int q = 0; q < 3; q++) xv[r] -= (double)s[(9 + r * 4 + 1 + q) * nl] * fcor[q];
      }
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      int ic = IC(g, i, j, k);
      put(S, 0, ic, xv[0], ss, bad);
      put(S, 4, ic, xv[1], ss, bad);
      int fk = (m + 1 == n) ? 0 : m + 1;
      put(S, 3, IPf(g, i, j, fk), xv[2], ss, bad);
    }
  }
}

// transverse component of kind 1/2 along d
__host__ __device__ constexpr int trans_comp(int d, int kind) {
  return d == 0 ? (kind == 1 ? 1 : 2) : d == 1 ? (kind == 1 ? 0 : 2) : (kind == 1 ? 0 : 1);
}

// the wall faces of component cc next to the first / last transverse line
template <typename R>
__device__ __forceinline__ void scalar_walls(const SweepArgs<R>& S, int cc, int i, int j, int k) {
  const Geo<R>& g = S.g;
  int lo = (cc == 0) ? (i == 1) : (cc == 1) ? (j == 1) : (k == 1);
  int hi = (cc == 0) ? (i == g.nr - 1) : (cc == 1) ? (j == g.nt - 1) : (k == g.np - 1);
  if (cc == 2 && g.per) lo = hi = 0;
  if (lo) {
    int wi = i, wj = j, wk = k;
    if (cc == 0) wi = 0; else if (cc == 1) wj = 0; else wk = 0;
    put_wall(S, 1 + cc, face_idx(g, cc, wi, wj, wk));
  }
  if (hi) {
    int wi = i, wj = j, wk = k;
    if (cc == 0) wi = g.nr; else if (cc == 1) wj = g.nt; else wk = g.np;
    put_wall(S, 1 + cc, face_idx(g, cc, wi, wj, wk));
  }
}

// output of a transverse line value at cell m, plus the wall faces of that
// component next to the first / last line
template <typename R, typename V, typename Acc>
__device__ __forceinline__ void scalar_put(const SweepArgs<R>& S, int cc, int i, int j, int k, V v, Acc& ss, int* bad) {
  put(S, 1 + cc, face_idx(S.g, cc, i, j, k), v, ss, bad);
  scalar_walls(S, cc, i, j, k);
}

// coefficients (a_m, b_m, c_m) of row m of a transverse scalar line, the
// no-slip fold at the walls of a walled line included
template <typename R>
__device__ __forceinline__ void scalar_row(const SweepArgs<R>& S, int cc, int d, int n, int cyc, int a, int b, int m,
                                           R& am, R& bm, R& cm) {
  int i, j, k;
  line_pos(d, a, b, m, i, j, k);
  R w[3];
  row_s(S.g, S.P, S.c, S.ub, cc, d, i, j, k, w);
  am = S.h * w[0]; bm = R(1) + S.h * w[1]; cm = S.h * w[2];
  if (!cyc) {
    if (m == 0) { bm -= am; am = R(0); }
    if (m == n - 1) { bm -= cm; cm = R(0); }
  }
}

// One transverse scalar line (component trans_comp(D, KIND)) along D: Thomas,
// Sherman-Morrison-corrected on a cyclic line; TR: the transposed system.
template <typename R, int D, int KIND, bool TR = false>
__device__ void scalar_line(const SweepArgs<R>& S, int line, int a, int b, SqSum<R>& ss, int* bad) {
  const Geo<R>& g = S.g;
  constexpr int d = D, kind = KIND;
  int cc = trans_comp(d, kind);
  int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
  int cyc = (d == 2 && g.per);
  int nl = S.nl[kind];
  R* scr = S.scr + S.scr_off[kind];
  const R* rhs = S.rhs.f[1 + cc];
  R cp = R(0), dy = R(0), dz = R(0);
  R a0 = R(0), gam = R(1);
  // the row inputs and right-hand side of cell m + 1, loaded before cell m is
  // eliminated (the forward pass)
  SPt<R> qn;
  R rn = R(0);
  auto fetch = [&](int m) {
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    qn = load_s<2>(g, S.c, S.ub, cc, d, i, j, k);
    rn = rhs[face_idx(g, cc, i, j, k)];
  };
  if constexpr (!TR) fetch(0);
  for (int m = 0; m < n; m++) {
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    R am, bm, cm, r;
    if constexpr (TR) {
      // row m of the transpose: c_{m-1}, b_m, a_{m+1} (wrapping when cyclic)
      R x0, x1, x2;
      scalar_row(S, cc, d, n, cyc, a, b, m, x0, bm, x2);
      am = cm = R(0);
      int mp = m - 1, mn = m + 1;
      if (cyc) { mp = mp < 0 ? n - 1 : mp; mn = mn == n ? 0 : mn; }
      if (mp >= 0) scalar_row(S, cc, d, n, cyc, a, b, mp, x0, x1, am);
      if (mn < n) scalar_row(S, cc, d, n, cyc, a, b, mn, cm, x1, x2);
      r = rhs[face_idx(g, cc, i, j, k)];
    } else {
      const SPt<R> q = qn;
      r = rn;
      if (m + 1 < n) fetch(m + 1);
      R w[3];
      row_sw(g, S.P, q, cc, d, i, j, w);
      am = S.h * w[0]; bm = R(1) + S.h * w[1]; cm = S.h * w[2];
      if (!cyc) {
        if (m == 0) { bm -= am; am = R(0); }
        if (m == n - 1) { bm -= cm; cm = R(0); }
      }
    }
    R zr = R(0);
    if (cyc) {
      // Sherman-Morrison split: gam = -b_0, u = [gam, 0, .., c_{n-1}], v = [1, 0, .., a_0/gam]
      if (m == 0) { a0 = am; gam = -bm; bm -= gam; zr = gam; am = R(0); }
      if (m == n - 1) { bm -= a0 * cm / gam; zr = cm; cm = R(0); }
    }
    R den = bm - am * cp;
    if (den == R(0) || !isfinite(den)) { *bad |= FLAG_SINGULAR; return; }
    R iden = sdiv(R(1), den);
    cp = cm * iden;
    dy = (r - am * dy) * iden;
    R* s = scr + m * 3 * nl + line;
    s[0] = cp;
    s[nl] = dy;
    if (cyc) { dz = (zr - am * dz) * iden; s[2 * nl] = dz; }
  }
  if (!cyc) {
    R xy = dy;
    // the factors of cell m - 1 are loaded before cell m is substituted
    R cn = R(0), yn = R(0);
    if (n >= 2) { cn = scr[(n - 2) * 3 * nl + line]; yn = scr[(n - 2) * 3 * nl + nl + line]; }
    for (int m = n - 1; m >= 0; m--) {
      if (m < n - 1) {
        const R c_ = cn, y_ = yn;
        if (m >= 1) { cn = scr[(m - 1) * 3 * nl + line]; yn = scr[(m - 1) * 3 * nl + nl + line]; }
        xy = y_ - c_ * xy;
      }
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      scalar_put(S, cc, i, j, k, xy, ss, bad);
    }
    return;
  }
  // cyclic: back-substitute both columns, then combine in FP64
  R xy = dy, xz = dz, yl = dy, zl = dz;
  for (int m = n - 2; m >= 0; m--) {
    R* t = scr + m * 3 * nl + line;
    xy = t[nl] - t[0] * xy;
    xz = t[2 * nl] - t[0] * xz;
    t[nl] = xy;
    t[2 * nl] = xz;
  }
  {
    R* t = scr + (n - 1) * 3 * nl + line;
    t[nl] = yl;
    t[2 * nl] = zl;
  }
  double ag = (double)a0 / (double)gam;
  double vy = (double)xy + ag * (double)yl, vz = (double)xz + ag * (double)zl;
  double f = vy / (1.0 + vz);
  for (int m = 0; m < n; m++) {
    const R* t = scr + m * 3 * nl + line;
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    scalar_put(S, cc, i, j, k, (double)t[nl] - f * (double)t[2 * nl], ss, bad);
  }
}

template <typename R, int D, bool TR = false>
__global__ void __launch_bounds__(128) k_sweep(SweepArgs<R> S) {
  int kind = blockIdx.y;
  int line = blockIdx.x * blockDim.x + threadIdx.x;
  SqSum<R> ss;
  int bad = 0;
  if (line < S.nl[kind]) {
    int a = (int)(line / S.nb[kind]) + S.a0[kind];
    int b = (int)(line % S.nb[kind]) + S.b0[kind];
    if (kind == 0) block_line<R, D, TR>(S, line, a, b, ss, &bad);
    else if (kind == 1) scalar_line<R, D, 1, TR>(S, line, a, b, ss, &bad);
    else scalar_line<R, D, 2, TR>(S, line, a, b, ss, &bad);
  }
  if (bad) atomicOr(S.flag, bad);
  if (S.update) {
    for (int f = 0; f < 5; f++) {
      double v = ss.warp_total(f);
      if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(S.acc + f, v);
    }
  }
}

// ------------------------------------------------- two-sided line solvers
// Walled (non-cyclic) lines, forward sweeps: two threads per line, one
// eliminating downwards from the first cell, the other upwards from the last
// (block Thomas "burning at both ends"): the same block operations as the
// one-sided solver above in two dependent chains of half the length, so twice
// the threads for the same arithmetic.  Lanes 0-15 of a warp take the top side
// of 16 lines, lanes 16-31 the bottom side of the same lines (partner = lane ^ 16).
//   top (s = 0), cells 0 .. h-1 (h = ceil(n/2)):  S_m = B_m - A_m E_{m-1},
//     E_m = S_m^{-1} C_m, g_m = S_m^{-1} (r_m - A_m g_{m-1}),  x_m = g_m - E_m x_{m+1};
//   bottom (s = 1), cells n-1 .. h, the roles of A and C swapped:
//     S_m = B_m - C_m E_{m+1}, E_m = S_m^{-1} A_m, g_m = S_m^{-1} (r_m - C_m g_{m+1}),
//     x_m = g_m - E_m x_{m-1}.
// At the meeting cells h-1 and h each side solves for its own boundary value,
// (I - E_o E_p) x_o = g_o - E_o g_p, with the partner's (E_p, g_p) from a
// shuffle (the same instructions on both sides), then substitutes outwards.
// Every lane runs the same instructions: a lane past the last line works on
// the last line and stores nothing; a singular pivot sets the flag and carries
// NaN on, so that no lane leaves the shuffles early.
constexpr int SWEEP2_LINES = 16;  // lines per warp

template <typename R>
__device__ __forceinline__ void inv3_or_nan(const R* S, R* I, int* bad) {
  if (!inv3(S, I)) {
    *bad |= FLAG_SINGULAR;
#pragma unroll
    for (int q = 0; q < 9; q++) I[q] = R(NAN);
  }
}

// Block m of (I + h D_d) on a walled line from the stored rows: rc the 12 centre
// values of the p- and T-rows, rf the 5 values of the normal-velocity row on
// face m + 1 (m < n - 1); the same entries and wall folds as assemble_pts.
template <typename R>
__device__ __forceinline__ void assemble_rows(const R* rc, const R* rf, int n, int m, R h, R* A, R* B, R* C) {
#pragma unroll
  for (int q = 0; q < 9; q++) { A[q] = R(0); B[q] = R(0); C[q] = R(0); }
  A[0] = h * rc[0]; A[1] = h * rc[2]; A[2] = h * rc[5];
  B[1] = h * rc[3]; B[2] = h * rc[6];
  C[0] = h * rc[1]; C[1] = h * rc[4];
  A[4] = h * rc[7]; A[5] = h * rc[10];
  B[4] = h * rc[8]; B[5] = h * rc[11];
  C[4] = h * rc[9];
  if (m < n - 1) {
    A[8] = h * rf[2];
    B[6] = h * rf[0]; B[8] = h * rf[3];
    C[6] = h * rf[1]; C[8] = h * rf[4];
  }
  B[0] += R(1); B[4] += R(1); B[8] += R(1);
  if (m == 0) {
    B[0] += A[0]; B[1] += A[1]; B[3] += A[3]; B[4] += A[4];
#pragma unroll
    for (int q = 0; q < 9; q++) A[q] = R(0);
  }
  if (m == n - 1) {
    B[0] += C[0]; B[1] += C[1]; B[3] += C[3]; B[4] += C[4];
#pragma unroll
    for (int q = 0; q < 9; q++) C[q] = R(0);
    B[2] = R(0); B[5] = R(0);
    A[8] = R(0); B[6] = R(0); B[7] = R(0); B[8] = R(1);
  }
}

template <typename R, int D, bool ROWS>
__device__ void block_line2(const SweepArgs<R>& S, int line, bool valid, int a, int b, int side, SqSum<R>& ss,
                            int* bad) {
  const Geo<R>& g = S.g;
  constexpr int d = D;
  const int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
  const int nl = S.nl[0];
  R* scr = S.scr + S.scr_off[0];
  constexpr int W = 12;
  const int h = (n + 1) / 2;
  const int cnt = side ? n - h : h;  // cells of this side (the bottom side of a one-cell line has none)
  auto cell = [&](int s) { return side ? n - 1 - s : s; };
  CPt<R> cqn;
  FPt<R> fqn;
  R rcn[ROWS ? 12 : 1], rfn[ROWS ? 5 : 1];
  R r0n = R(0), r4n = R(0), run = R(0);
  auto fetch = [&](int m) {
    int i, j, k, fi, fj, fk;
    line_pos(d, a, b, m, i, j, k);
    const int ic = IC(g, i, j, k);
    if constexpr (ROWS) {
      const R* pc = S.rows.c[d] + ic;
#pragma unroll
      for (int q = 0; q < 12; q++) rcn[q] = pc[q * S.rows.nc];
    } else {
      cqn = load_c(S.c, d, ic);
      fqn = {R(1), R(1), R(0)};
    }
    run = R(0);
    if (m < n - 1) {
      next_face(d, n, m, i, j, k, fi, fj, fk);
      const int fx = face_idx(g, d, fi, fj, fk);
      if constexpr (ROWS) {
        const R* pf = S.rows.f[d] + fx;
#pragma unroll
        for (int q = 0; q < 5; q++) rfn[q] = pf[q * S.rows.nf[d]];
      } else {
        fqn = load_f(g, S.c, S.ub.f[1 + d], d, fi, fj, fk);
      }
      run = S.rhs.f[1 + d][fx];
    }
    r0n = S.rhs.f[0][ic];
    r4n = S.rhs.f[4][ic];
  };
  R E[9], gv[3];
#pragma unroll
  for (int q = 0; q < 9; q++) E[q] = R(0);
  gv[0] = gv[1] = gv[2] = R(0);
  if (cnt > 0) fetch(cell(0));
  for (int s = 0; s < cnt; s++) {
    const int m = cell(s);
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    R A[9], B[9], C[9];
    R rr[3] = {r0n, r4n, run};
    if constexpr (ROWS) {
      R rc[12], rf[5];
#pragma unroll
      for (int q = 0; q < 12; q++) rc[q] = rcn[q];
#pragma unroll
      for (int q = 0; q < 5; q++) rf[q] = rfn[q];
      if (s + 1 < cnt) fetch(cell(s + 1));
      assemble_rows(rc, rf, n, m, S.h, A, B, C);
    } else {
      const CPt<R> cq = cqn;
      const FPt<R> fq = fqn;
      if (s + 1 < cnt) fetch(cell(s + 1));
      int fi, fj, fk;
      next_face(d, n, m, i, j, k, fi, fj, fk);
      assemble_pts(g, S.P, cq, fq, d, n, 0, m, i, j, fi, fj, S.h, A, B, C);
    }
    // L couples to the cell already eliminated, U to the next one
    R L[9], U[9];
#pragma unroll
    for (int q = 0; q < 9; q++) { L[q] = side ? C[q] : A[q]; U[q] = side ? A[q] : C[q]; }
    R Sm[9], y[3];
#pragma unroll
    for (int r = 0; r < 3; r++) {
#pragma unroll
      for (int q = 0; q < 3; q++)
        Sm[r * 3 + q] = B[r * 3 + q] - (L[r * 3] * E[q] + L[r * 3 + 1] * E[3 + q] + L[r * 3 + 2] * E[6 + q]);
      y[r] = rr[r] - (L[r * 3] * gv[0] + L[r * 3 + 1] * gv[1] + L[r * 3 + 2] * gv[2]);
    }
    R Si[9];
    inv3_or_nan(Sm, Si, bad);
#pragma unroll
    for (int r = 0; r < 3; r++) {
#pragma unroll
      for (int q = 0; q < 3; q++) E[r * 3 + q] = Si[r * 3] * U[q] + Si[r * 3 + 1] * U[3 + q] + Si[r * 3 + 2] * U[6 + q];
      gv[r] = Si[r * 3] * y[0] + Si[r * 3 + 1] * y[1] + Si[r * 3 + 2] * y[2];
    }
    if (s + 1 < cnt && valid) {
      R* sp = scr + m * W * nl + line;
#pragma unroll
      for (int q = 0; q < 9; q++) sp[q * nl] = E[q];
#pragma unroll
      for (int q = 0; q < 3; q++) sp[(9 + q) * nl] = gv[q];
    }
  }
  // the meeting cells: the partner's last factors (zero for the empty bottom
  // side of a one-cell line, which leaves x = g on the top side)
  R Ep[9], gp[3];
#pragma unroll
  for (int q = 0; q < 9; q++) Ep[q] = __shfl_xor_sync(0xffffffffu, E[q], 16);
#pragma unroll
  for (int q = 0; q < 3; q++) gp[q] = __shfl_xor_sync(0xffffffffu, gv[q], 16);
  R Mm[9], rhs[3], Mi[9], xs[3];
#pragma unroll
  for (int r = 0; r < 3; r++) {
#pragma unroll
    for (int q = 0; q < 3; q++)
      Mm[r * 3 + q] = (r == q ? R(1) : R(0)) - (E[r * 3] * Ep[q] + E[r * 3 + 1] * Ep[3 + q] + E[r * 3 + 2] * Ep[6 + q]);
    rhs[r] = gv[r] - (E[r * 3] * gp[0] + E[r * 3 + 1] * gp[1] + E[r * 3 + 2] * gp[2]);
  }
  inv3_or_nan(Mm, Mi, bad);
#pragma unroll
  for (int r = 0; r < 3; r++) xs[r] = Mi[r * 3] * rhs[0] + Mi[r * 3 + 1] * rhs[1] + Mi[r * 3 + 2] * rhs[2];
  // substitution outwards from the meeting cell; the factors of the next cell
  // out are loaded before the current one is stored
  R En[9], gn[3];
  if (cnt >= 2) {
    const R* sp = scr + cell(cnt - 2) * W * nl + line;
#pragma unroll
    for (int q = 0; q < 9; q++) En[q] = sp[q * nl];
#pragma unroll
    for (int q = 0; q < 3; q++) gn[q] = sp[(9 + q) * nl];
  }
  for (int s = cnt - 1; s >= 0; s--) {
    const int m = cell(s);
    if (s < cnt - 1) {
      R E_[9], g_[3];
#pragma unroll
      for (int q = 0; q < 9; q++) E_[q] = En[q];
#pragma unroll
      for (int q = 0; q < 3; q++) g_[q] = gn[q];
      if (s >= 1) {
        const R* sp = scr + cell(s - 1) * W * nl + line;
#pragma unroll
        for (int q = 0; q < 9; q++) En[q] = sp[q * nl];
#pragma unroll
        for (int q = 0; q < 3; q++) gn[q] = sp[(9 + q) * nl];
      }
      R xn[3];
#pragma unroll
      for (int r = 0; r < 3; r++) xn[r] = g_[r] - (E_[r * 3] * xs[0] + E_[r * 3 + 1] * xs[1] + E_[r * 3 + 2] * xs[2]);
#pragma unroll
      for (int q = 0; q < 3; q++) xs[q] = xn[q];
    }
    if (valid) {
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      int ic = IC(g, i, j, k);
      put(S, 0, ic, xs[0], ss, bad);
      put(S, 4, ic, xs[1], ss, bad);
      int fi = i, fj = j, fk = k;
      if (m < n - 1) {
        if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = m + 1;
        put(S, 1 + d, face_idx(g, d, fi, fj, fk), xs[2], ss, bad);
      } else {
        if (d == 0) fi = n; else if (d == 1) fj = n; else fk = n;
        put_wall(S, 1 + d, face_idx(g, d, fi, fj, fk));
        int gi = i, gj = j, gk = k;
        if (d == 0) gi = 0; else if (d == 1) gj = 0; else gk = 0;
        put_wall(S, 1 + d, face_idx(g, d, gi, gj, gk));
      }
    }
  }
}

// The scalar (transverse-component) lines the same way: Thomas from both ends,
// (1 - e_o e_p) x_o = g_o - e_o g_p at the meeting cells.
template <typename R, int D, int KIND, bool ROWS>
__device__ void scalar_line2(const SweepArgs<R>& S, int line, bool valid, int a, int b, int side, SqSum<R>& ss,
                             int* bad) {
  const Geo<R>& g = S.g;
  constexpr int d = D, kind = KIND;
  const int cc = trans_comp(d, kind);
  const int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
  const int nl = S.nl[kind];
  R* scr = S.scr + S.scr_off[kind];
  const R* rhs = S.rhs.f[1 + cc];
  const int h = (n + 1) / 2;
  const int cnt = side ? n - h : h;
  auto cell = [&](int s) { return side ? n - 1 - s : s; };
  SPt<R> qn;
  R wn[3];
  R rn = R(0);
  auto fetch = [&](int m) {
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    const int fx = face_idx(g, cc, i, j, k);
    if constexpr (ROWS) {
      const long nfc = S.rows.nf[cc];
      const R* ps = S.rows.s[cc] + 3 * trans_slot(cc, d) * nfc + fx;
      wn[0] = ps[0]; wn[1] = ps[nfc]; wn[2] = ps[2 * nfc];
    } else {
      qn = load_s<2>(g, S.c, S.ub, cc, d, i, j, k);
    }
    rn = rhs[fx];
  };
  R e = R(0), gy = R(0);
  if (cnt > 0) fetch(cell(0));
  for (int s = 0; s < cnt; s++) {
    const int m = cell(s);
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    const R r = rn;
    R w[3];
    if constexpr (ROWS) {
      w[0] = wn[0]; w[1] = wn[1]; w[2] = wn[2];
      if (s + 1 < cnt) fetch(cell(s + 1));
    } else {
      const SPt<R> q = qn;
      if (s + 1 < cnt) fetch(cell(s + 1));
      row_sw(g, S.P, q, cc, d, i, j, w);
    }
    R am = S.h * w[0], bm = R(1) + S.h * w[1], cm = S.h * w[2];
    if (m == 0) { bm -= am; am = R(0); }
    if (m == n - 1) { bm -= cm; cm = R(0); }
    const R lo = side ? cm : am, up = side ? am : cm;
    R den = bm - lo * e;
    if (den == R(0) || !isfinite(den)) *bad |= FLAG_SINGULAR;
    R iden = sdiv(R(1), den);
    e = up * iden;
    gy = (r - lo * gy) * iden;
    if (s + 1 < cnt && valid) {
      R* sp = scr + m * 3 * nl + line;
      sp[0] = e;
      sp[nl] = gy;
    }
  }
  const R ep = __shfl_xor_sync(0xffffffffu, e, 16), gp = __shfl_xor_sync(0xffffffffu, gy, 16);
  R x = sdiv(gy - e * gp, R(1) - e * ep);
  R en = R(0), gn = R(0);
  if (cnt >= 2) {
    const int mm = cell(cnt - 2);
    en = scr[mm * 3 * nl + line];
    gn = scr[mm * 3 * nl + nl + line];
  }
  for (int s = cnt - 1; s >= 0; s--) {
    const int m = cell(s);
    if (s < cnt - 1) {
      const R e_ = en, g_ = gn;
      if (s >= 1) {
        const int mm = cell(s - 1);
        en = scr[mm * 3 * nl + line];
        gn = scr[mm * 3 * nl + nl + line];
      }
      x = g_ - e_ * x;
    }
    if (valid) {
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      scalar_put(S, cc, i, j, k, x, ss, bad);
    }
  }
}

// one warp per 16 lines of one kind (blockIdx.y): lanes l and l + 16 share a line
template <typename R, int D, bool ROWS>
__global__ void __launch_bounds__(128) k_sweep2(SweepArgs<R> S) {
  const int kind = blockIdx.y;
  const int nl = S.nl[kind];
  const int lane = threadIdx.x & 31;
  const int base = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / 2;  // first line of the warp
  if (base >= nl) return;  // the whole warp: no line of this kind left
  const int side = lane >> 4;
  const int l0 = base + (lane & (SWEEP2_LINES - 1));
  const bool valid = l0 < nl;
  const int line = valid ? l0 : nl - 1;
  SqSum<R> ss;
  int bad = 0;
  int a = (int)(line / S.nb[kind]) + S.a0[kind];
  int b = (int)(line % S.nb[kind]) + S.b0[kind];
  if (kind == 0) block_line2<R, D, ROWS>(S, line, valid, a, b, side, ss, &bad);
  else if (kind == 1) scalar_line2<R, D, 1, ROWS>(S, line, valid, a, b, side, ss, &bad);
  else scalar_line2<R, D, 2, ROWS>(S, line, valid, a, b, side, ss, &bad);
  if (bad) atomicOr(S.flag, bad);
  if (S.update) {
    for (int f = 0; f < 5; f++) {
      double v = ss.warp_total(f);
      if (lane == 0 && v != 0.0) atomicAdd(S.acc + f, v);
    }
  }
}
