// sph.cu -- GB300 (sm_103a) kernels and C ABI for the direction-splitting scheme of
// Frolov, Minev & Takhirov (arXiv 2004.13887): Picard-iterated Crank-Nicolson with
// Douglas factorisation and splitting-error reduction (Section 2.2, eqs.
// chapter3mainsd, splitting2, spl1-spl3), MAC grid in spherical coordinates,
// operators of Appendix B.
//
// One iteration k -> k+1 is five launches:
//   avg   : Ubar = (U^n + U^{n+1,k})/2                      (skipped at k = 0)
//   coef  : per-centre coefficients frozen at Ubar (p+pi_inf, T, rho, beta,
//           centre velocities, grad u with metric terms)
//   rhs   : R = -(U^k - U^n) - tau [N(Ubar) + G - S]  (the right-hand side of
//           eq. spl1 after the linearity of D(Ubar) is used: the D(U^k - U^n),
//           D U^n and D_M terms collapse to the full operator at Ubar)
//   sweep : r, theta, phi line solves (I + tau/2 D_d) x = rhs (eqs. spl1-spl3):
//           one thread per line, 3x3-block Thomas for (p, T, u_d) and scalar
//           Thomas for the two transverse velocities; cyclic lines (periodic phi)
//           by a rank-3 Woodbury / Sherman-Morrison correction.  The phi sweep
//           also applies U^{k+1} = U^k + x and accumulates the increment norm.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/sph.h"
#include "sph_device.cuh"

using namespace sph;

#define FLAG_NONFINITE 1
#define FLAG_SINGULAR 2

// ------------------------------------------------------------------ kernels

__global__ void k_avg(long n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ o) {
  long s = (long)gridDim.x * blockDim.x;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += s) o[t] = 0.5 * (a[t] + b[t]);
}

__global__ void k_coef(Geo g, Par P, CF ub, Coef c) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long N = (long)g.nr * g.nt * g.np;
  if (t >= N) return;
  int k = (int)(t % g.np), j = (int)((t / g.np) % g.nt), i = (int)(t / ((long)g.np * g.nt));
  const double *UR = ub.f[1], *UT = ub.f[2], *UP = ub.f[3];
  double pb = cval(g, ub.f[0], g.bgp, i, j, k) + P.pinf;
  double tb = cval(g, ub.f[4], g.bgT, i, j, k);
  double ipb = 1.0 / pb, itb = 1.0 / tb;
  c.Pb[t] = pb;
  c.Tb[t] = tb;
  c.rho[t] = pb * itb / P.Rg;
  c.beta[t] = (P.gamma - 1.0) * tb * ipb;
  double ur = hr(g, UR, i, j, k), ut = ht(g, UT, i, j, k), up = hp(g, UP, i, j, k);
  c.uc0[t] = ur; c.uc1[t] = ut; c.uc2[t] = up;
  double ir = g.irc[i], is = g.isc[j], cot = g.cotc[j];
  c.grr[t] = (vr(g, UR, i + 1, j, k) - vr(g, UR, i, j, k)) * g.idr;
  c.gtt[t] = (vt(g, UT, i, j + 1, k) - vt(g, UT, i, j, k)) * ir * g.idth + ur * ir;
  c.gpp[t] = (vp(g, UP, i, j, k + 1) - vp(g, UP, i, j, k)) * ir * is * g.idph + ur * ir + ut * cot * ir;
  double grt = (ht(g, UT, i + 1, j, k) - ht(g, UT, i - 1, j, k)) * 0.5 * g.idr;
  double gtr = (hr(g, UR, i, j + 1, k) - hr(g, UR, i, j - 1, k)) * 0.5 * ir * g.idth - ut * ir;
  double grp = (hp(g, UP, i + 1, j, k) - hp(g, UP, i - 1, j, k)) * 0.5 * g.idr;
  double gpr = (hr(g, UR, i, j, k + 1) - hr(g, UR, i, j, k - 1)) * 0.5 * ir * is * g.idph - up * ir;
  double gtp = (hp(g, UP, i, j + 1, k) - hp(g, UP, i, j - 1, k)) * 0.5 * ir * g.idth;
  double gpt = (ht(g, UT, i, j, k + 1) - ht(g, UT, i, j, k - 1)) * 0.5 * ir * is * g.idph - up * cot * ir;
  c.srt[t] = grt + gtr;
  c.srp[t] = grp + gpr;
  c.stp[t] = gtp + gpt;
}

// N(Ubar) rows and R = -(U^k - U^n) - tau (N + G - S); one thread per centre
// also owns the lower r-, theta- and phi-faces of its cell.
__global__ void k_rhs(Geo g, Par P, Coef c, CF ub, CF un, CF uk, CF src, int has_src, double tau, MF R) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long N = (long)g.nr * g.nt * g.np;
  if (t >= N) return;
  int k = (int)(t % g.np), j = (int)((t / g.np) % g.nt), i = (int)(t / ((long)g.np * g.nt));
  const double *Pp = ub.f[0], *UR = ub.f[1], *UT = ub.f[2], *UP = ub.f[3], *TT = ub.f[4];
  double mu = P.mu, gm = P.gamma, om = P.omega;
  double ir = g.irc[i], is = g.isc[j], cot = g.cotc[j];

  // ---- p- and T-rows at the centre
  {
    double accp = 0.0, accT = 0.0;
    for (int d = 0; d < 3; d++) {
      int di = d == 0, dj = d == 1, dk = d == 2;
      double pv[3], Tv[3], uv[2];
      for (int s = -1; s <= 1; s++) {
        pv[s + 1] = cval(g, Pp, g.bgp, i + s * di, j + s * dj, k + s * dk);
        Tv[s + 1] = cval(g, TT, g.bgT, i + s * di, j + s * dj, k + s * dk);
      }
      if (d == 0) { uv[0] = UR[IRf(g, i, j, k)]; uv[1] = UR[IRf(g, i + 1, j, k)]; }
      else if (d == 1) { uv[0] = UT[ITf(g, i, j, k)]; uv[1] = UT[ITf(g, i, j + 1, k)]; }
      else { uv[0] = vp(g, UP, i, j, k); uv[1] = vp(g, UP, i, j, k + 1); }
      double wp[3], wT[3], wu[2];
      row_c(g, P, c, d, 0, i, j, k, wp, wT, wu);
      accp += wp[0] * pv[0] + wp[1] * pv[1] + wp[2] * pv[2] + wT[0] * Tv[0] + wT[1] * Tv[1] + wT[2] * Tv[2]
            + wu[0] * uv[0] + wu[1] * uv[1];
      row_c(g, P, c, d, 1, i, j, k, wp, wT, wu);
      accT += wT[0] * Tv[0] + wT[1] * Tv[1] + wT[2] * Tv[2] + wu[0] * uv[0] + wu[1] * uv[1];
    }
    double xrt = (ht(g, UT, i + 1, j, k) - ht(g, UT, i - 1, j, k)) * 0.5 * g.idr
               + (hr(g, UR, i, j + 1, k) - hr(g, UR, i, j - 1, k)) * 0.5 * ir * g.idth;
    double xrp = (hp(g, UP, i + 1, j, k) - hp(g, UP, i - 1, j, k)) * 0.5 * g.idr
               + (hr(g, UR, i, j, k + 1) - hr(g, UR, i, j, k - 1)) * 0.5 * ir * is * g.idph;
    double xtp = (hp(g, UP, i, j + 1, k) - hp(g, UP, i, j - 1, k)) * 0.5 * ir * g.idth
               + (ht(g, UT, i, j, k + 1) - ht(g, UT, i, j, k - 1)) * 0.5 * ir * is * g.idph;
    double cross = c.srt[t] * xrt + c.srp[t] * xrp + c.stp[t] * xtp;
    accp += -mu * (gm - 1.0) * cross;
    accT += -mu * c.beta[t] * cross;
    double sp = has_src ? src.f[0][t] : 0.0, sT = has_src ? src.f[4][t] : 0.0;
    R.f[0][t] = -(uk.f[0][t] - un.f[0][t]) - tau * (accp - sp);
    R.f[4][t] = -(uk.f[4][t] - un.f[4][t]) - tau * (accT - sT);
  }

  // ---- r-momentum on r-face i (interior faces 1..nr-1)
  if (i >= 1) {
    long id = IRf(g, i, j, k);
    double wp[2], wu[3], w[3];
    row_f(g, P, c, UR, 0, i, j, k, wp, wu);
    double acc = wp[0] * cval(g, Pp, g.bgp, i - 1, j, k) + wp[1] * cval(g, Pp, g.bgp, i, j, k)
               + wu[0] * UR[IRf(g, i - 1, j, k)] + wu[1] * UR[id] + wu[2] * UR[IRf(g, i + 1, j, k)];
    row_s(g, P, c, ub, 0, 1, i, j, k, w);
    acc += w[0] * vr(g, UR, i, j - 1, k) + w[1] * UR[id] + w[2] * vr(g, UR, i, j + 1, k);
    row_s(g, P, c, ub, 0, 2, i, j, k, w);
    acc += w[0] * vr(g, UR, i, j, k - 1) + w[1] * UR[id] + w[2] * vr(g, UR, i, j, k + 1);
    // D_M
    double irf = g.irf[i], s = g.sc[j];
    double irh = 2.0 / (rho_at(g, c, i - 1, j, k) + rho_at(g, c, i, j, k));
    double utf = 0.5 * (ht(g, UT, i - 1, j, k) + ht(g, UT, i, j, k));
    double upf = 0.5 * (hp(g, UP, i - 1, j, k) + hp(g, UP, i, j, k));
    double Q[2];
    for (int q = 0; q < 2; q++) {
      int m = i - 1 + q;
      Q[q] = (g.sf[j + 1] * UT[ITf(g, m, j + 1, k)] - g.sf[j] * UT[ITf(g, m, j, k)]) * g.irc[m] * is * g.idth
           + (vp(g, UP, m, j, k + 1) - vp(g, UP, m, j, k)) * g.irc[m] * is * g.idph;
    }
    acc += -utf * utf * irf - upf * upf * irf + 2.0 * mu * irh * UR[id] * irf * irf - 2.0 * om * s * upf
         - mu * irh * (1.0 / 3.0) * g.idr * (Q[1] - Q[0]) + mu * irh * irf * (Q[0] + Q[1]);
    double sv = has_src ? src.f[1][id] : 0.0;
    R.f[1][id] = -(uk.f[1][id] - un.f[1][id]) - tau * (acc + P.g - sv);
  } else {
    R.f[1][IRf(g, 0, j, k)] = 0.0;
  }
  if (i == g.nr - 1) R.f[1][IRf(g, g.nr, j, k)] = 0.0;

  // ---- theta-momentum on theta-face j (interior faces 1..nt-1)
  if (j >= 1) {
    long id = ITf(g, i, j, k);
    double wp[2], wu[3], w[3];
    row_f(g, P, c, UT, 1, i, j, k, wp, wu);
    double acc = wp[0] * cval(g, Pp, g.bgp, i, j - 1, k) + wp[1] * cval(g, Pp, g.bgp, i, j, k)
               + wu[0] * UT[ITf(g, i, j - 1, k)] + wu[1] * UT[id] + wu[2] * UT[ITf(g, i, j + 1, k)];
    row_s(g, P, c, ub, 1, 0, i, j, k, w);
    acc += w[0] * vt(g, UT, i - 1, j, k) + w[1] * UT[id] + w[2] * vt(g, UT, i + 1, j, k);
    row_s(g, P, c, ub, 1, 2, i, j, k, w);
    acc += w[0] * vt(g, UT, i, j, k - 1) + w[1] * UT[id] + w[2] * vt(g, UT, i, j, k + 1);
    double isfj = g.isf[j], cfj = g.cf[j], cotf = g.cotf[j];
    double irh = 2.0 / (rho_at(g, c, i, j - 1, k) + rho_at(g, c, i, j, k));
    double ubt = UT[id];
    double upf = 0.5 * (hp(g, UP, i, j - 1, k) + hp(g, UP, i, j, k));
    double vrf = 0.5 * (hr(g, UR, i, j - 1, k) + hr(g, UR, i, j, k));
    double Dr[2], Dp[2], dpf = 0.0;
    for (int q = 0; q < 2; q++) {
      int m = j - 1 + q;
      Dr[q] = (g.rf[i + 1] * g.rf[i + 1] * UR[IRf(g, i + 1, m, k)] - g.rf[i] * g.rf[i] * UR[IRf(g, i, m, k)])
            * ir * ir * g.idr;
      double dv = vp(g, UP, i, m, k + 1) - vp(g, UP, i, m, k);
      Dp[q] = dv * ir * g.isc[m] * g.idph;
      dpf += 0.5 * dv * g.idph;
    }
    acc += ubt * vrf * ir - upf * upf * cotf * ir + mu * irh * ubt * ir * ir * isfj * isfj - 2.0 * om * cfj * upf
         - mu * irh * (1.0 / 3.0) * ir * g.idth * ((Dr[1] - Dr[0]) + (Dp[1] - Dp[0]))
         - mu * irh * (2.0 * ir * ir * g.idth * (hr(g, UR, i, j, k) - hr(g, UR, i, j - 1, k))
                       - 2.0 * cfj * ir * ir * isfj * isfj * dpf);
    double sv = has_src ? src.f[2][id] : 0.0;
    R.f[2][id] = -(uk.f[2][id] - un.f[2][id]) - tau * (acc - sv);
  } else {
    R.f[2][ITf(g, i, 0, k)] = 0.0;
  }
  if (j == g.nt - 1) R.f[2][ITf(g, i, g.nt, k)] = 0.0;

  // ---- phi-momentum on phi-face k (interior faces, or every face if periodic)
  if (k >= 1 || g.per) {
    long id = IPf(g, i, j, k);
    double wp[2], wu[3], w[3];
    row_f(g, P, c, UP, 2, i, j, k, wp, wu);
    double acc = wp[0] * cval(g, Pp, g.bgp, i, j, k - 1) + wp[1] * cval(g, Pp, g.bgp, i, j, k)
               + wu[0] * vp(g, UP, i, j, k - 1) + wu[1] * UP[id] + wu[2] * vp(g, UP, i, j, k + 1);
    row_s(g, P, c, ub, 2, 0, i, j, k, w);
    acc += w[0] * vp(g, UP, i - 1, j, k) + w[1] * UP[id] + w[2] * vp(g, UP, i + 1, j, k);
    row_s(g, P, c, ub, 2, 1, i, j, k, w);
    acc += w[0] * vp(g, UP, i, j - 1, k) + w[1] * UP[id] + w[2] * vp(g, UP, i, j + 1, k);
    double s = g.sc[j], cj = g.cc[j];
    double irh = 2.0 / (rho_at(g, c, i, j, k - 1) + rho_at(g, c, i, j, k));
    double ubp = UP[id];
    double vrf = 0.5 * (hr(g, UR, i, j, k - 1) + hr(g, UR, i, j, k));
    double vtf = 0.5 * (ht(g, UT, i, j, k - 1) + ht(g, UT, i, j, k));
    double Dr[2], Dt[2];
    for (int q = 0; q < 2; q++) {
      int m = k - 1 + q;
      Dr[q] = (g.rf[i + 1] * g.rf[i + 1] * vr(g, UR, i + 1, j, m) - g.rf[i] * g.rf[i] * vr(g, UR, i, j, m))
            * ir * ir * g.idr;
      Dt[q] = (g.sf[j + 1] * vt(g, UT, i, j + 1, m) - g.sf[j] * vt(g, UT, i, j, m)) * ir * is * g.idth;
    }
    acc += ubp * vtf * cot * ir + ubp * vrf * ir + mu * irh * ubp * ir * ir * is * is + 2.0 * om * (cj * vtf + s * vrf)
         - mu * irh * (1.0 / 3.0) * ir * is * g.idph * ((Dr[1] - Dr[0]) + (Dt[1] - Dt[0]))
         - mu * irh * (2.0 * ir * ir * is * g.idph * (hr(g, UR, i, j, k) - hr(g, UR, i, j, k - 1))
                       + 2.0 * cj * ir * ir * is * is * g.idph * (ht(g, UT, i, j, k) - ht(g, UT, i, j, k - 1)));
    double sv = has_src ? src.f[3][id] : 0.0;
    R.f[3][id] = -(uk.f[3][id] - un.f[3][id]) - tau * (acc - sv);
  } else {
    R.f[3][IPf(g, i, j, 0)] = 0.0;
  }
  if (!g.per && k == g.np - 1) R.f[3][IPf(g, i, j, g.np)] = 0.0;
}

// ------------------------------------------------------------ line solvers

__device__ __forceinline__ bool inv3(const double* S, double* I) {
  double c00 = S[4] * S[8] - S[5] * S[7];
  double c01 = S[5] * S[6] - S[3] * S[8];
  double c02 = S[3] * S[7] - S[4] * S[6];
  double det = S[0] * c00 + S[1] * c01 + S[2] * c02;
  if (det == 0.0 || !isfinite(det)) return false;
  double id = 1.0 / det;
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

__device__ __forceinline__ long face_idx(const Geo& g, int d, int i, int j, int k) {
  return d == 0 ? IRf(g, i, j, k) : d == 1 ? ITf(g, i, j, k) : IPf(g, i, j, k);
}

// Assemble block m of (I + h D_d) on the line (a, b); h = tau/2.
__device__ void assemble_block(const Geo& g, const Par& P, const Coef& c, const CF& ub, int d, int n, int cyc, int m,
                               int i, int j, int k, double h, double* A, double* B, double* C) {
  double wp[3], wT[3], wu[2];
#pragma unroll
  for (int q = 0; q < 9; q++) { A[q] = 0.0; B[q] = 0.0; C[q] = 0.0; }
  row_c(g, P, c, d, 0, i, j, k, wp, wT, wu);
  A[0] = h * wp[0]; A[1] = h * wT[0]; A[2] = h * wu[0];
  B[0] = h * wp[1]; B[1] = h * wT[1]; B[2] = h * wu[1];
  C[0] = h * wp[2]; C[1] = h * wT[2];
  row_c(g, P, c, d, 1, i, j, k, wp, wT, wu);
  A[4] = h * wT[0]; A[5] = h * wu[0];
  B[4] = h * wT[1]; B[5] = h * wu[1];
  C[4] = h * wT[2];
  if (m < n - 1 || cyc) {
    int fi = i, fj = j, fk = k;
    if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = (m + 1 == n) ? 0 : m + 1;
    double fp[2], fu[3];
    row_f(g, P, c, ub.f[1 + d], d, fi, fj, fk, fp, fu);
    A[8] = h * fu[0];
    B[6] = h * fp[0]; B[8] = h * fu[1];
    C[6] = h * fp[1]; C[8] = h * fu[2];
  }
  B[0] += 1.0; B[4] += 1.0; B[8] += 1.0;
  if (!cyc) {
    if (m == 0) {
      B[0] += A[0]; B[1] += A[1]; B[3] += A[3]; B[4] += A[4];
#pragma unroll
      for (int q = 0; q < 9; q++) A[q] = 0.0;
    }
    if (m == n - 1) {
      B[0] += C[0]; B[1] += C[1]; B[3] += C[3]; B[4] += C[4];
#pragma unroll
      for (int q = 0; q < 9; q++) C[q] = 0.0;
      B[2] = 0.0; B[5] = 0.0;
      A[8] = 0.0; B[6] = 0.0; B[7] = 0.0; B[8] = 1.0;
    }
  }
}

struct SweepArgs {
  Geo g; Par P; Coef c; CF ub;
  int d; double h;
  CF rhs;              // right-hand side fields
  MF x;                // output increments (mode 0)
  int update;          // mode 1: uk = base + x, accumulate norms
  CF base; MF uk;
  double* scr;         // scratch
  long scr_off[3];     // offsets of the three kinds
  long nl[3];          // lines per kind
  int a0[3], nb[3], b0[3];
  double* acc;         // 5 sums of squares (mode 1)
  int* flag;
};

// store a value of field f at flat index idx: x (mode 0) or uk = base + v (mode 1)
__device__ __forceinline__ void put(const SweepArgs& A, int f, long idx, double v, double* ss, int* bad) {
  if (!A.update) {
    A.x.f[f][idx] = v;
  } else {
    double nv = A.base.f[f][idx] + v;
    if (!isfinite(nv)) *bad |= FLAG_NONFINITE;
    A.uk.f[f][idx] = nv;
    ss[f] += v * v;
  }
}
// wall face of field f: x = 0, or uk = base (mode 1)
__device__ __forceinline__ void put_wall(const SweepArgs& A, int f, long idx) {
  if (!A.update) A.x.f[f][idx] = 0.0;
  else A.uk.f[f][idx] = A.base.f[f][idx];
}

__device__ void block_line(const SweepArgs& S, long line, int a, int b, double* ss, int* bad) {
  const Geo& g = S.g;
  int d = S.d;
  int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
  int cyc = (d == 2 && g.per);
  long nl = S.nl[0];
  double* scr = S.scr + S.scr_off[0];
  const int W = cyc ? 21 : 12;  // C' (9) + d' (3 per right-hand side)
  const int NR = cyc ? 4 : 1;
  double Cp[9], dp[12];
  double GiA[9];                // cyclic: Gam^{-1} A_0
  double Gam[9];
  for (int m = 0; m < n; m++) {
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    double A[9], B[9], C[9];
    assemble_block(g, S.P, S.c, S.ub, d, n, cyc, m, i, j, k, S.h, A, B, C);
    double rr[12];
    long ic = IC(g, i, j, k);
    rr[0] = S.rhs.f[0][ic];
    rr[NR] = S.rhs.f[4][ic];
    double ru = 0.0;
    if (m < n - 1 || cyc) {
      int fi = i, fj = j, fk = k;
      if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = (m + 1 == n) ? 0 : m + 1;
      ru = S.rhs.f[1 + d][face_idx(g, d, fi, fj, fk)];
    }
    rr[2 * NR] = ru;
    if (cyc) {
      // right-hand-side columns 1..3 of U = [Gam; 0; ..; C_{n-1}]
      for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) rr[r * NR + 1 + q] = 0.0;
      if (m == 0) {
        for (int q = 0; q < 9; q++) Gam[q] = -B[q];
        double Gi[9];
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
    double Sm[9], y[12];
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
    double Si[9];
    if (!inv3(Sm, Si)) { *bad |= FLAG_SINGULAR; return; }
    // the last block has no right neighbour on a non-cyclic line: C = 0
    for (int r = 0; r < 3; r++) {
      for (int q = 0; q < 3; q++)
        Cp[r * 3 + q] = Si[r * 3] * C[q] + Si[r * 3 + 1] * C[3 + q] + Si[r * 3 + 2] * C[6 + q];
      for (int q = 0; q < NR; q++)
        dp[r * NR + q] = Si[r * 3] * y[q] + Si[r * 3 + 1] * y[NR + q] + Si[r * 3 + 2] * y[2 * NR + q];
    }
    if (m < n - 1) {
      double* s = scr + (long)m * W * nl + line;
      for (int q = 0; q < 9; q++) s[(long)q * nl] = Cp[q];
      for (int q = 0; q < 3 * NR; q++) s[(long)(9 + q) * nl] = dp[q];
    }
  }
  // back substitution, all NR columns
  double xs[12];
  for (int q = 0; q < 3 * NR; q++) xs[q] = dp[q];
  double fcor[3] = {0.0, 0.0, 0.0};
  double x0[12];
  for (int m = n - 1; m >= 0; m--) {
    if (m < n - 1) {
      const double* s = scr + (long)m * W * nl + line;
      double C_[9], d_[12];
      for (int q = 0; q < 9; q++) C_[q] = s[(long)q * nl];
      for (int q = 0; q < 3 * NR; q++) d_[q] = s[(long)(9 + q) * nl];
      double xn[12];
      for (int r = 0; r < 3; r++)
        for (int q = 0; q < NR; q++)
          xn[r * NR + q] = d_[r * NR + q] - (C_[r * 3] * xs[q] + C_[r * 3 + 1] * xs[NR + q] + C_[r * 3 + 2] * xs[2 * NR + q]);
      for (int q = 0; q < 3 * NR; q++) xs[q] = xn[q];
    }
    if (!cyc) {
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      long ic = IC(g, i, j, k);
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
      // keep x (all columns) in scratch d'-slots for the Woodbury combination
      double* s = scr + (long)m * W * nl + line;
      for (int q = 0; q < 3 * NR; q++) s[(long)(9 + q) * nl] = xs[q];
      if (m == 0) for (int q = 0; q < 12; q++) x0[q] = xs[q];
    }
  }
  if (cyc) {
    // V^T y = y_0 + GiA y_{n-1};  V^T Z = Z_0 + GiA Z_{n-1};  f = (I + V^T Z)^{-1} V^T y
    const double* sl = scr + (long)(n - 1) * W * nl + line;
    double xl[12];
    for (int q = 0; q < 12; q++) xl[q] = sl[(long)(9 + q) * nl];
    double vy[3], vz[9];
    for (int r = 0; r < 3; r++) {
      vy[r] = x0[r * 4] + GiA[r * 3] * xl[0] + GiA[r * 3 + 1] * xl[4] + GiA[r * 3 + 2] * xl[8];
      for (int q = 0; q < 3; q++)
        vz[r * 3 + q] = x0[r * 4 + 1 + q] + GiA[r * 3] * xl[1 + q] + GiA[r * 3 + 1] * xl[5 + q] + GiA[r * 3 + 2] * xl[9 + q]
                      + (r == q ? 1.0 : 0.0);
    }
    double vi[9];
    if (!inv3(vz, vi)) { *bad |= FLAG_SINGULAR; return; }
    for (int r = 0; r < 3; r++) fcor[r] = vi[r * 3] * vy[0] + vi[r * 3 + 1] * vy[1] + vi[r * 3 + 2] * vy[2];
    for (int m = 0; m < n; m++) {
      const double* s = scr + (long)m * W * nl + line;
      double xv[3];
      for (int r = 0; r < 3; r++) {
        xv[r] = s[(long)(9 + r * 4) * nl];
        for (int q = 0; q < 3; q++) xv[r] -= s[(long)(9 + r * 4 + 1 + q) * nl] * fcor[q];
      }
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      long ic = IC(g, i, j, k);
      put(S, 0, ic, xv[0], ss, bad);
      put(S, 4, ic, xv[1], ss, bad);
      int fk = (m + 1 == n) ? 0 : m + 1;
      put(S, 3, IPf(g, i, j, fk), xv[2], ss, bad);
    }
  }
}

// transverse component of kind 1/2 along d
__device__ __forceinline__ int trans_comp(int d, int kind) {
  if (d == 0) return kind == 1 ? 1 : 2;
  if (d == 1) return kind == 1 ? 0 : 2;
  return kind == 1 ? 0 : 1;
}

// output of a transverse line value at cell m, plus the wall faces of that
// component next to the first / last line
__device__ __forceinline__ void scalar_put(const SweepArgs& S, int cc, int i, int j, int k, double v, double* ss,
                                           int* bad) {
  const Geo& g = S.g;
  put(S, 1 + cc, face_idx(g, cc, i, j, k), v, ss, bad);
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

__device__ void scalar_line(const SweepArgs& S, int kind, long line, int a, int b, double* ss, int* bad) {
  const Geo& g = S.g;
  int d = S.d;
  int cc = trans_comp(d, kind);
  int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
  int cyc = (d == 2 && g.per);
  long nl = S.nl[kind];
  double* scr = S.scr + S.scr_off[kind];
  const double* rhs = S.rhs.f[1 + cc];
  double cp = 0.0, dy = 0.0, dz = 0.0;
  double a0 = 0.0, gam = 1.0;
  for (int m = 0; m < n; m++) {
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    double w[3];
    row_s(g, S.P, S.c, S.ub, cc, d, i, j, k, w);
    double am = S.h * w[0], bm = 1.0 + S.h * w[1], cm = S.h * w[2];
    double zr = 0.0;
    if (!cyc) {
      if (m == 0) { bm -= am; am = 0.0; }
      if (m == n - 1) { bm -= cm; cm = 0.0; }
    } else {
      // Sherman-Morrison split: gam = -b_0, u = [gam, 0, .., c_{n-1}], v = [1, 0, .., a_0/gam]
      if (m == 0) { a0 = am; gam = -bm; bm -= gam; zr = gam; am = 0.0; }
      if (m == n - 1) { bm -= a0 * cm / gam; zr = cm; cm = 0.0; }
    }
    double r = rhs[face_idx(g, cc, i, j, k)];
    double den = bm - am * cp;
    if (den == 0.0 || !isfinite(den)) { *bad |= FLAG_SINGULAR; return; }
    double iden = 1.0 / den;
    cp = cm * iden;
    dy = (r - am * dy) * iden;
    double* s = scr + (long)m * 3 * nl + line;
    s[0] = cp;
    s[nl] = dy;
    if (cyc) { dz = (zr - am * dz) * iden; s[2 * nl] = dz; }
  }
  if (!cyc) {
    double xy = dy;
    for (int m = n - 1; m >= 0; m--) {
      if (m < n - 1) {
        const double* t = scr + (long)m * 3 * nl + line;
        xy = t[nl] - t[0] * xy;
      }
      int i, j, k;
      line_pos(d, a, b, m, i, j, k);
      scalar_put(S, cc, i, j, k, xy, ss, bad);
    }
    return;
  }
  // cyclic: back-substitute both columns, then combine
  double xy = dy, xz = dz, yl = dy, zl = dz;
  for (int m = n - 2; m >= 0; m--) {
    double* t = scr + (long)m * 3 * nl + line;
    xy = t[nl] - t[0] * xy;
    xz = t[2 * nl] - t[0] * xz;
    t[nl] = xy;
    t[2 * nl] = xz;
  }
  {
    double* t = scr + (long)(n - 1) * 3 * nl + line;
    t[nl] = yl;
    t[2 * nl] = zl;
  }
  double vy = xy + a0 / gam * yl, vz = xz + a0 / gam * zl;
  double f = vy / (1.0 + vz);
  for (int m = 0; m < n; m++) {
    const double* t = scr + (long)m * 3 * nl + line;
    int i, j, k;
    line_pos(d, a, b, m, i, j, k);
    scalar_put(S, cc, i, j, k, t[nl] - f * t[2 * nl], ss, bad);
  }
}

__global__ void k_sweep(SweepArgs S) {
  int kind = blockIdx.y;
  long line = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double ss[5] = {0, 0, 0, 0, 0};
  int bad = 0;
  if (line < S.nl[kind]) {
    int a = (int)(line / S.nb[kind]) + S.a0[kind];
    int b = (int)(line % S.nb[kind]) + S.b0[kind];
    if (kind == 0) block_line(S, line, a, b, ss, &bad);
    else scalar_line(S, kind, line, a, b, ss, &bad);
  }
  if (bad) atomicOr(S.flag, bad);
  if (S.update) {
    for (int f = 0; f < 5; f++) {
      double v = ss[f];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(S.acc + f, v);
    }
  }
}

// ============================================================== host side

struct sph_ctx {
  int dev;
  cudaStream_t st;
  Geo g;
  Par P;
  int prec;
  size_t nf[5];
  long N;
  double* metric;
  double* bg;
  double* U[2][5];
  int cur;
  int iterate_set;
  double* Ub[5];
  double* R[5];
  double* X1[5];
  double* src[5];
  double* coef;
  Coef c;
  double* scr;
  double* acc;   // 5 sums + spare
  int* flag;
  long long launches;
  long unknowns[5];
  // per-kernel timing
  int prof;
  cudaEvent_t* ev;
  int* evkind;
  int nev, evcap;
  long long kcount[SPH_NKERNELS];
  int cur_kind;
};

#define PROF_CAP 65536

static int cuda_ok(cudaError_t e) { return e == cudaSuccess; }

extern "C" size_t sph_field_size(const sph_grid* gr, int f) {
  if (!gr) return 0;
  size_t nr = gr->nr, nt = gr->nth, np = gr->nph, npf = gr->periodic_phi ? np : np + 1;
  switch (f) {
    case 0: case 4: return nr * nt * np;
    case 1: return (nr + 1) * nt * np;
    case 2: return nr * (nt + 1) * np;
    case 3: return nr * nt * npf;
    default: return 0;
  }
}

extern "C" const char* sph_strerror(int code) {
  switch (code) {
    case SPH_OK: return "ok";
    case SPH_ERR_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA runtime error";
    case SPH_ERR_NONFINITE: return "non-finite value in the new state (state left at U^n)";
    case SPH_ERR_SINGULAR: return "zero pivot in a line solve (state left at U^n)";
    case SPH_ERR_NOMEM: return "device allocation failed";
    default: return "unknown error";
  }
}

extern "C" long long sph_launch_count(const sph_ctx* ctx) { return ctx ? ctx->launches : 0; }

static void prof_free(sph_ctx* c) {
  for (int q = 0; q < c->evcap * 2; q++) cudaEventDestroy(c->ev[q]);
  free(c->ev); free(c->evkind);
  c->ev = NULL; c->evkind = NULL; c->evcap = 0; c->nev = 0;
}

static void free_all(sph_ctx* c) {
  prof_free(c);
  cudaFree(c->metric); cudaFree(c->bg); cudaFree(c->coef); cudaFree(c->scr); cudaFree(c->acc); cudaFree(c->flag);
  for (int f = 0; f < 5; f++) {
    cudaFree(c->U[0][f]); cudaFree(c->U[1][f]); cudaFree(c->Ub[f]); cudaFree(c->R[f]); cudaFree(c->X1[f]);
    cudaFree(c->src[f]);
  }
}

extern "C" void sph_destroy(sph_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->dev);
  cudaStreamSynchronize(ctx->st);
  free_all(ctx);
  cudaSetDevice(prev);
  free(ctx);
}

extern "C" int sph_create(const sph_grid* gr, const sph_params* pa, void* stream, sph_ctx** out) {
  if (!gr || !pa || !out) return SPH_ERR_ARG;
  *out = NULL;
  if (gr->nr < 2 || gr->nth < 2 || gr->nph < 2) return SPH_ERR_ARG;
  if (!(gr->r1 > 0) || !(gr->r2 > gr->r1) || !(gr->th2 > gr->th1) || !(gr->ph2 > gr->ph1)) return SPH_ERR_ARG;
  if (gr->th1 < 0 || gr->th2 > M_PI + 1e-12) return SPH_ERR_ARG;
  if (gr->periodic_phi && gr->nph < 3) return SPH_ERR_ARG;
  if (!(pa->gamma > 1) || !(pa->cv > 0) || !(pa->Pr > 0) || pa->mu < 0) return SPH_ERR_ARG;
  if (pa->precision != SPH_PREC_FP64) return SPH_ERR_ARG;   /* mixed precision: separate entry */
  sph_ctx* c = (sph_ctx*)calloc(1, sizeof(sph_ctx));
  if (!c) return SPH_ERR_NOMEM;
  cudaGetDevice(&c->dev);
  c->st = (cudaStream_t)stream;
  c->prec = pa->precision;
  Geo& g = c->g;
  g.nr = gr->nr; g.nt = gr->nth; g.np = gr->nph; g.per = gr->periodic_phi ? 1 : 0;
  g.npf = g.per ? g.np : g.np + 1;
  g.dr = (gr->r2 - gr->r1) / g.nr; g.dth = (gr->th2 - gr->th1) / g.nt; g.dph = (gr->ph2 - gr->ph1) / g.np;
  g.idr = 1.0 / g.dr; g.idth = 1.0 / g.dth; g.idph = 1.0 / g.dph;
  Par& P = c->P;
  P.gamma = pa->gamma; P.cv = pa->cv; P.Pr = pa->Pr; P.mu = pa->mu; P.pinf = pa->pi_inf; P.g = pa->g;
  P.omega = pa->omega;
  P.kappa = pa->mu * pa->gamma * pa->cv / pa->Pr;
  P.Rg = pa->cv * (pa->gamma - 1.0);
  c->N = (long)g.nr * g.nt * g.np;
  for (int f = 0; f < 5; f++) c->nf[f] = sph_field_size(gr, f);
  c->unknowns[0] = c->unknowns[4] = c->N;
  c->unknowns[1] = (long)(g.nr - 1) * g.nt * g.np;
  c->unknowns[2] = (long)g.nr * (g.nt - 1) * g.np;
  c->unknowns[3] = (long)g.nr * g.nt * (g.per ? g.np : g.np - 1);

  // metric tables on the host, then one copy
  int nr = g.nr, nt = g.nt;
  size_t nmet = 4 * (size_t)(nr + 1) + 8 * (size_t)(nt + 1);
  double* h = (double*)calloc(nmet, sizeof(double));
  double* rc = h; double* rf = rc + (nr + 1); double* irc = rf + (nr + 1); double* irf = irc + (nr + 1);
  double* sc = irf + (nr + 1); double* sf = sc + (nt + 1); double* isc = sf + (nt + 1); double* isf = isc + (nt + 1);
  double* cc = isf + (nt + 1); double* cf = cc + (nt + 1); double* cotc = cf + (nt + 1); double* cotf = cotc + (nt + 1);
  for (int i = 0; i < nr; i++) { rc[i] = gr->r1 + (i + 0.5) * g.dr; irc[i] = 1.0 / rc[i]; }
  for (int i = 0; i <= nr; i++) { rf[i] = gr->r1 + i * g.dr; irf[i] = 1.0 / rf[i]; }
  for (int j = 0; j < nt; j++) {
    double t = gr->th1 + (j + 0.5) * g.dth;
    sc[j] = sin(t); cc[j] = cos(t); isc[j] = 1.0 / sc[j]; cotc[j] = cc[j] / sc[j];
  }
  for (int j = 0; j <= nt; j++) {
    double t = gr->th1 + j * g.dth;
    sf[j] = sin(t); cf[j] = cos(t);
  }
  if (fabs(gr->th1) < 1e-14) sf[0] = 0.0;
  if (fabs(gr->th2 - M_PI) < 1e-14) sf[nt] = 0.0;
  for (int j = 0; j <= nt; j++) { isf[j] = sf[j] != 0.0 ? 1.0 / sf[j] : 0.0; cotf[j] = sf[j] != 0.0 ? cf[j] / sf[j] : 0.0; }
  for (int j = 0; j < nt; j++)
    if (!(sc[j] > 0)) { free(h); free(c); return SPH_ERR_ARG; }

  int err = SPH_OK;
#define ALLOC(p, n) do { if (err == SPH_OK && !cuda_ok(cudaMalloc((void**)&(p), (n) * sizeof(double)))) err = SPH_ERR_NOMEM; } while (0)
  ALLOC(c->metric, nmet);
  ALLOC(c->bg, 2 * (size_t)(nr + 2));
  for (int f = 0; f < 5; f++) {
    ALLOC(c->U[0][f], c->nf[f]); ALLOC(c->U[1][f], c->nf[f]); ALLOC(c->Ub[f], c->nf[f]);
    ALLOC(c->R[f], c->nf[f]); ALLOC(c->X1[f], c->nf[f]); ALLOC(c->src[f], c->nf[f]);
  }
  ALLOC(c->coef, 13 * (size_t)c->N);
  // scratch: block lines 12 (21 if cyclic) per point, scalar lines 3 per point each
  size_t wblk = g.per ? 21 : 12;
  size_t nscr = (wblk + 6) * (size_t)c->N + 64;
  ALLOC(c->scr, nscr);
  ALLOC(c->acc, 8);
  if (err == SPH_OK && !cuda_ok(cudaMalloc((void**)&c->flag, sizeof(int)))) err = SPH_ERR_NOMEM;
#undef ALLOC
  if (err != SPH_OK) { free(h); free_all(c); free(c); cudaGetLastError(); return err; }
  if (!cuda_ok(cudaMemcpy(c->metric, h, nmet * sizeof(double), cudaMemcpyHostToDevice)) ||
      !cuda_ok(cudaMemset(c->bg, 0, 2 * (size_t)(nr + 2) * sizeof(double))) ||
      !cuda_ok(cudaMemset(c->flag, 0, sizeof(int))))
    err = SPH_ERR_CUDA;
  for (int f = 0; f < 5 && err == SPH_OK; f++) {
    if (!cuda_ok(cudaMemset(c->U[0][f], 0, c->nf[f] * sizeof(double))) ||
        !cuda_ok(cudaMemset(c->U[1][f], 0, c->nf[f] * sizeof(double))))
      err = SPH_ERR_CUDA;
  }
  free(h);
  if (err != SPH_OK) { free_all(c); free(c); return err; }
  double* m = c->metric;
  g.rc = m; g.rf = m + (nr + 1); g.irc = m + 2 * (nr + 1); g.irf = m + 3 * (nr + 1);
  double* tb = m + 4 * (nr + 1);
  g.sc = tb; g.sf = tb + (nt + 1); g.isc = tb + 2 * (nt + 1); g.isf = tb + 3 * (nt + 1);
  g.cc = tb + 4 * (nt + 1); g.cf = tb + 5 * (nt + 1); g.cotc = tb + 6 * (nt + 1); g.cotf = tb + 7 * (nt + 1);
  g.bgp = c->bg; g.bgT = c->bg + (nr + 2);
  double* q = c->coef;
  long N = c->N;
  Coef& cf_ = c->c;
  cf_.Pb = q; cf_.Tb = q + N; cf_.rho = q + 2 * N; cf_.beta = q + 3 * N; cf_.uc0 = q + 4 * N; cf_.uc1 = q + 5 * N;
  cf_.uc2 = q + 6 * N; cf_.grr = q + 7 * N; cf_.gtt = q + 8 * N; cf_.gpp = q + 9 * N; cf_.srt = q + 10 * N;
  cf_.srp = q + 11 * N; cf_.stp = q + 12 * N;
  c->cur = 0;
  *out = c;
  return SPH_OK;
}

extern "C" int sph_set_background(sph_ctx* c, const double* p_ref, const double* T_ref) {
  if (!c) return SPH_ERR_ARG;
  size_t n = c->g.nr + 2;
  cudaError_t e = cudaSuccess;
  if (p_ref) e = cudaMemcpyAsync(c->bg, p_ref, n * sizeof(double), cudaMemcpyHostToDevice, c->st);
  else e = cudaMemsetAsync(c->bg, 0, n * sizeof(double), c->st);
  if (e == cudaSuccess) {
    if (T_ref) e = cudaMemcpyAsync(c->bg + n, T_ref, n * sizeof(double), cudaMemcpyHostToDevice, c->st);
    else e = cudaMemsetAsync(c->bg + n, 0, n * sizeof(double), c->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return e == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

static int copy_fields(sph_ctx* c, double* const* dst, const double* const* src, int kind) {
  for (int f = 0; f < 5; f++) {
    if (!dst[f] || !src[f]) return SPH_ERR_ARG;
    if (cudaMemcpyAsync(dst[f], src[f], c->nf[f] * sizeof(double), (cudaMemcpyKind)kind, c->st) != cudaSuccess)
      return SPH_ERR_CUDA;
  }
  return SPH_OK;
}

extern "C" int sph_set_state(sph_ctx* c, const double* const* fields, int on_device) {
  if (!c || !fields) return SPH_ERR_ARG;
  int e = copy_fields(c, c->U[c->cur], fields, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  c->iterate_set = 0;
  if (e == SPH_OK && !on_device && cudaStreamSynchronize(c->st) != cudaSuccess) e = SPH_ERR_CUDA;
  return e;
}

extern "C" int sph_get_state(sph_ctx* c, double* const* fields, int on_device) {
  if (!c || !fields) return SPH_ERR_ARG;
  int e = copy_fields(c, fields, (const double* const*)c->U[c->cur],
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  if (e == SPH_OK && !on_device && cudaStreamSynchronize(c->st) != cudaSuccess) e = SPH_ERR_CUDA;
  return e;
}

extern "C" int sph_set_iterate(sph_ctx* c, const double* const* fields, int on_device) {
  if (!c || !fields) return SPH_ERR_ARG;
  int e = copy_fields(c, c->U[1 - c->cur], fields, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (e == SPH_OK) c->iterate_set = 1;
  if (e == SPH_OK && !on_device && cudaStreamSynchronize(c->st) != cudaSuccess) e = SPH_ERR_CUDA;
  return e;
}

static CF cf_of(double* const* p) { CF r; for (int f = 0; f < 5; f++) r.f[f] = p[f]; return r; }
static MF mf_of(double* const* p) { MF r; for (int f = 0; f < 5; f++) r.f[f] = p[f]; return r; }

// bracket a launch: start event before, stop event after (when timing is on)
static void k_begin(sph_ctx* c, int kind) {
  c->cur_kind = kind;
  c->kcount[kind]++;
  if (c->prof && c->nev < c->evcap) cudaEventRecord(c->ev[2 * c->nev], c->st);
}

static int launch_ok(sph_ctx* c) {
  c->launches++;
  if (c->prof && c->nev < c->evcap) {
    cudaEventRecord(c->ev[2 * c->nev + 1], c->st);
    c->evkind[c->nev++] = c->cur_kind;
  }
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

extern "C" int sph_profile(sph_ctx* c, int enable) {
  if (!c) return SPH_ERR_ARG;
  if (enable && !c->ev) {
    c->ev = (cudaEvent_t*)calloc(2 * PROF_CAP, sizeof(cudaEvent_t));
    c->evkind = (int*)calloc(PROF_CAP, sizeof(int));
    if (!c->ev || !c->evkind) { free(c->ev); free(c->evkind); c->ev = NULL; c->evkind = NULL; return SPH_ERR_NOMEM; }
    for (int q = 0; q < 2 * PROF_CAP; q++)
      if (cudaEventCreate(&c->ev[q]) != cudaSuccess) { c->evcap = q / 2; prof_free(c); return SPH_ERR_CUDA; }
    c->evcap = PROF_CAP;
  }
  c->prof = enable ? 1 : 0;
  if (enable) {
    c->nev = 0;
    for (int q = 0; q < SPH_NKERNELS; q++) c->kcount[q] = 0;
  }
  return SPH_OK;
}

extern "C" int sph_profile_read(sph_ctx* c, double* ms, long long* count) {
  if (!c) return SPH_ERR_ARG;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_ERR_CUDA;
  double acc[SPH_NKERNELS] = {0};
  for (int q = 0; q < c->nev; q++) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->ev[2 * q], c->ev[2 * q + 1]) != cudaSuccess) return SPH_ERR_CUDA;
    acc[c->evkind[q]] += t;
  }
  for (int q = 0; q < SPH_NKERNELS; q++) {
    if (ms) ms[q] = acc[q];
    if (count) count[q] = c->kcount[q];
  }
  return SPH_OK;
}

// Ubar into c->Ub (or U^n itself when the iterate equals U^n); coefficients
static int prepare(sph_ctx* c, int have_iter, CF* ub_out) {
  double** un = c->U[c->cur];
  double** uk = c->U[1 - c->cur];
  CF ub;
  if (have_iter) {
    for (int f = 0; f < 5; f++) {
      long n = (long)c->nf[f];
      int blocks = (int)((n + 255) / 256);
      if (blocks > 152 * 16) blocks = 152 * 16;
      k_begin(c, SPH_K_AVG);
      k_avg<<<blocks, 256, 0, c->st>>>(n, un[f], uk[f], c->Ub[f]);
      if (launch_ok(c)) return SPH_ERR_CUDA;
    }
    ub = cf_of(c->Ub);
  } else {
    ub = cf_of(un);
  }
  k_begin(c, SPH_K_COEF);
  k_coef<<<(unsigned)((c->N + 127) / 128), 128, 0, c->st>>>(c->g, c->P, ub, c->c);
  if (launch_ok(c)) return SPH_ERR_CUDA;
  *ub_out = ub;
  return SPH_OK;
}

static int run_rhs(sph_ctx* c, CF ub, CF uk, double tau, CF src, int has_src, MF R) {
  CF un = cf_of(c->U[c->cur]);
  k_begin(c, SPH_K_RHS);
  k_rhs<<<(unsigned)((c->N + 127) / 128), 128, 0, c->st>>>(c->g, c->P, c->c, ub, un, uk, src, has_src, tau, R);
  return launch_ok(c);
}

// Lines of direction d: kind 0 = block lines (a, b) over cell centres, kinds 1/2 =
// the two transverse velocity components on their interior faces.  Half-open
// ranges [a_lo, a_hi) x [b_lo, b_hi); (a, b) = (j, k) for d = r, (i, k) for
// theta, (i, j) for phi.
static void line_layout(const sph_ctx* c, int d, SweepArgs& S) {
  const Geo& g = c->g;
  int nr = g.nr, nt = g.nt, np = g.np, k0 = g.per ? 0 : 1;
  int n = d == 0 ? nr : d == 1 ? nt : np;
  int lo_a[3], hi_a[3], lo_b[3], hi_b[3];
  if (d == 0) {
    lo_a[0] = 0; hi_a[0] = nt; lo_b[0] = 0;  hi_b[0] = np;
    lo_a[1] = 1; hi_a[1] = nt; lo_b[1] = 0;  hi_b[1] = np;   // u_theta, theta-faces 1..nt-1
    lo_a[2] = 0; hi_a[2] = nt; lo_b[2] = k0; hi_b[2] = np;   // u_phi, interior phi-faces
  } else if (d == 1) {
    lo_a[0] = 0; hi_a[0] = nr; lo_b[0] = 0;  hi_b[0] = np;
    lo_a[1] = 1; hi_a[1] = nr; lo_b[1] = 0;  hi_b[1] = np;   // u_r, r-faces 1..nr-1
    lo_a[2] = 0; hi_a[2] = nr; lo_b[2] = k0; hi_b[2] = np;   // u_phi
  } else {
    lo_a[0] = 0; hi_a[0] = nr; lo_b[0] = 0;  hi_b[0] = nt;
    lo_a[1] = 1; hi_a[1] = nr; lo_b[1] = 0;  hi_b[1] = nt;   // u_r
    lo_a[2] = 0; hi_a[2] = nr; lo_b[2] = 1;  hi_b[2] = nt;   // u_theta
  }
  long off = 0;
  for (int q = 0; q < 3; q++) {
    int na = hi_a[q] - lo_a[q], nb = hi_b[q] - lo_b[q];
    S.a0[q] = lo_a[q]; S.b0[q] = lo_b[q]; S.nb[q] = nb > 0 ? nb : 1;
    S.nl[q] = (na > 0 && nb > 0) ? (long)na * nb : 0;
    S.scr_off[q] = off;
    long w = q == 0 ? (g.per && d == 2 ? 21 : 12) : 3;
    off += w * (long)n * S.nl[q];
  }
}

static int run_sweep(sph_ctx* c, int d, double tau, CF ub, CF rhs, MF x, int update, CF base, MF uk) {
  SweepArgs S;
  memset(&S, 0, sizeof S);
  S.g = c->g; S.P = c->P; S.c = c->c; S.ub = ub; S.d = d; S.h = 0.5 * tau;
  S.rhs = rhs; S.x = x; S.update = update; S.base = base; S.uk = uk;
  S.scr = c->scr; S.acc = c->acc; S.flag = c->flag;
  line_layout(c, d, S);
  long mx = S.nl[0];
  if (S.nl[1] > mx) mx = S.nl[1];
  if (S.nl[2] > mx) mx = S.nl[2];
  dim3 grid((unsigned)((mx + 127) / 128), 3);
  k_begin(c, SPH_K_SWEEP_R + d);
  k_sweep<<<grid, 128, 0, c->st>>>(S);
  return launch_ok(c);
}

static int read_flag(sph_ctx* c, int* flag) {
  if (cudaMemcpyAsync(flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess) return SPH_ERR_CUDA;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_ERR_CUDA;
  return SPH_OK;
}

static int stage_source(sph_ctx* c, const double* const* source, int on_device, CF* out) {
  if (!source) { *out = cf_of(c->src); return 0; }
  if (on_device) {
    for (int f = 0; f < 5; f++) out->f[f] = source[f];
    return 1;
  }
  for (int f = 0; f < 5; f++)
    if (cudaMemcpyAsync(c->src[f], source[f], c->nf[f] * sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return -1;
  *out = cf_of(c->src);
  return 1;
}

extern "C" int sph_rhs(sph_ctx* c, double dt, const double* const* source, int on_device, double* const* R_out) {
  if (!c || !R_out || !(dt > 0)) return SPH_ERR_ARG;
  CF src;
  int has = stage_source(c, source, on_device, &src);
  if (has < 0) return SPH_ERR_CUDA;
  CF ub;
  int e = prepare(c, c->iterate_set, &ub);
  if (e) return e;
  CF uk = cf_of(c->iterate_set ? c->U[1 - c->cur] : c->U[c->cur]);
  return run_rhs(c, ub, uk, dt, src, has, mf_of(R_out));
}

extern "C" int sph_sweep(sph_ctx* c, int dir, double dt, const double* const* rhs, double* const* x) {
  if (!c || !rhs || !x || dir < 0 || dir > 2 || !(dt > 0)) return SPH_ERR_ARG;
  CF ub;
  int e = prepare(c, c->iterate_set, &ub);
  if (e) return e;
  if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->st) != cudaSuccess) return SPH_ERR_CUDA;
  e = run_sweep(c, dir, dt, ub, cf_of((double* const*)rhs), mf_of(x), 0, cf_of(c->U[c->cur]), mf_of(x));
  if (e) return e;
  int flag = 0;
  if ((e = read_flag(c, &flag))) return e;
  return (flag & FLAG_SINGULAR) ? SPH_ERR_SINGULAR : SPH_OK;
}

extern "C" int sph_step(sph_ctx* c, double dt, int n_iter, const double* const* source, int on_device,
                        double* residual_out) {
  if (!c || !(dt > 0) || n_iter < 1) return SPH_ERR_ARG;
  CF src;
  int has = stage_source(c, source, on_device, &src);
  if (has < 0) return SPH_ERR_CUDA;
  if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->st) != cudaSuccess) return SPH_ERR_CUDA;
  double** un = c->U[c->cur];
  double** uk = c->U[1 - c->cur];
  int e = SPH_OK;
  for (int it = 0; it < n_iter && !e; it++) {
    CF ub;
    e = prepare(c, it > 0, &ub);
    if (e) break;
    CF ukin = cf_of(it == 0 ? un : uk);
    e = run_rhs(c, ub, ukin, dt, src, has, mf_of(c->R));
    if (!e) e = run_sweep(c, 0, dt, ub, cf_of(c->R), mf_of(c->X1), 0, ukin, mf_of(uk));
    if (!e) e = run_sweep(c, 1, dt, ub, cf_of(c->X1), mf_of(c->R), 0, ukin, mf_of(uk));
    if (!e && it == n_iter - 1 && cudaMemsetAsync(c->acc, 0, 5 * sizeof(double), c->st) != cudaSuccess) e = SPH_ERR_CUDA;
    if (!e) e = run_sweep(c, 2, dt, ub, cf_of(c->R), mf_of(c->X1), 1, ukin, mf_of(uk));
  }
  if (e) return e;
  int flag = 0;
  if ((e = read_flag(c, &flag))) return e;
  if (flag & FLAG_SINGULAR) return SPH_ERR_SINGULAR;
  if (flag & FLAG_NONFINITE) return SPH_ERR_NONFINITE;
  if (residual_out) {
    double s[5];
    if (cudaMemcpy(s, c->acc, 5 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return SPH_ERR_CUDA;
    for (int f = 0; f < 5; f++) residual_out[f] = c->unknowns[f] > 0 ? sqrt(s[f] / (double)c->unknowns[f]) : 0.0;
  }
  c->cur = 1 - c->cur;
  c->iterate_set = 0;
  return SPH_OK;
}
