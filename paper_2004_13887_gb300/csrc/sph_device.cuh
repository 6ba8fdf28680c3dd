// sph_device.cuh -- device-side discretisation of the direction-splitting scheme
// of arXiv 2004.13887 (Section 2.2, Appendix B) on the MAC grid.
//
// Everything here is written for the GB300 library; the CPU reference in
// oracle/ is a separate implementation of the same equations.
//
// Rows of the split operators, with coefficients frozen at Ubar (eq.
// chapter3mainsd) and moved to staggered points by arithmetic means:
//   row_c : p-row (A1^d, A2^d, A3^d) or T-row (C2^d, C3^d) at a cell centre,
//           reading p and T at m-1, m, m+1 along d and u_d on faces m, m+1;
//   row_f : normal-velocity row (B1^d, B2^{d,d}) on a d-face;
//   row_s : transverse row B2^{d,c} of velocity component c along d;
//   M-rows: D_M (cross derivatives, curvature, Coriolis, the off-line parts of
//           grad(div v)/3 and of the vector Laplacian), applied explicitly.
// The viscous-heating linearisation follows A2/C2 of Appendix B except that the
// G_phiphi*cot(theta) term printed in A2^phi / C2^phi is dropped: it does not
// follow from grad(u):sigma(v) (only A2^theta has it).
#pragma once
#include <cuda_runtime.h>

namespace sph {

struct Geo {
  int nr, nt, np, npf, per;
  double dr, dth, dph, idr, idth, idph;
  // metric tables (device): centres rc[nr], faces rf[nr+1]; theta centres/faces
  const double *rc, *rf, *irc, *irf;
  const double *sc, *sf, *isc, *isf, *cc, *cf, *cotc, *cotf;
  const double *bgp, *bgT;  // nr+2, index i+1 for i in [-1, nr]
};

struct Par {
  double gamma, cv, Pr, mu, pinf, g, omega;
  double kappa, Rg;  // kappa = mu cp / Pr, Rg = cv (gamma-1)
};

struct Coef {  // per cell centre, frozen at Ubar
  double *Pb, *Tb, *rho, *beta, *uc0, *uc1, *uc2;
  double *grr, *gtt, *gpp, *srt, *srp, *stp;  // G_rr, G_tt, G_pp, G_rt+G_tr, G_rp+G_pr, G_tp+G_pt
};

struct CF { const double* f[5]; };
struct MF { double* f[5]; };

__device__ __forceinline__ long IC(const Geo& g, int i, int j, int k) { return ((long)i * g.nt + j) * g.np + k; }
__device__ __forceinline__ long IRf(const Geo& g, int i, int j, int k) { return ((long)i * g.nt + j) * g.np + k; }
__device__ __forceinline__ long ITf(const Geo& g, int i, int j, int k) { return ((long)i * (g.nt + 1) + j) * g.np + k; }
__device__ __forceinline__ long IPf(const Geo& g, int i, int j, int k) { return ((long)i * g.nt + j) * g.npf + k; }

__device__ __forceinline__ int wrapk(const Geo& g, int k) { return k < 0 ? k + g.np : (k >= g.np ? k - g.np : k); }
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---------------------------------------------------------------- accessors
// Centre scalar with background; zero Neumann ghost on the perturbation.
__device__ __forceinline__ double cval(const Geo& g, const double* f, const double* bg, int i, int j, int k) {
  double b = bg[i + 1];
  int ii = clampi(i, 0, g.nr - 1), jj = clampi(j, 0, g.nt - 1);
  int kk = g.per ? wrapk(g, k) : clampi(k, 0, g.np - 1);
  return b + f[IC(g, ii, jj, kk)];
}
// Velocities with no-slip ghosts (ghost = -interior) on tangential walls.
__device__ __forceinline__ double vr(const Geo& g, const double* u, int i, int j, int k) {
  if (j < 0) return -u[IRf(g, i, 0, k)];
  if (j >= g.nt) return -u[IRf(g, i, g.nt - 1, k)];
  if (k < 0 || k >= g.np) {
    if (g.per) k = wrapk(g, k);
    else return -u[IRf(g, i, j, k < 0 ? 0 : g.np - 1)];
  }
  return u[IRf(g, i, j, k)];
}
__device__ __forceinline__ double vt(const Geo& g, const double* u, int i, int j, int k) {
  if (i < 0) return -u[ITf(g, 0, j, k)];
  if (i >= g.nr) return -u[ITf(g, g.nr - 1, j, k)];
  if (k < 0 || k >= g.np) {
    if (g.per) k = wrapk(g, k);
    else return -u[ITf(g, i, j, k < 0 ? 0 : g.np - 1)];
  }
  return u[ITf(g, i, j, k)];
}
__device__ __forceinline__ double vp(const Geo& g, const double* u, int i, int j, int k) {
  if (g.per) k = wrapk(g, k);
  if (i < 0) return -u[IPf(g, 0, j, k)];
  if (i >= g.nr) return -u[IPf(g, g.nr - 1, j, k)];
  if (j < 0) return -u[IPf(g, i, 0, k)];
  if (j >= g.nt) return -u[IPf(g, i, g.nt - 1, k)];
  return u[IPf(g, i, j, k)];
}
__device__ __forceinline__ double hr(const Geo& g, const double* u, int i, int j, int k) {
  return 0.5 * (vr(g, u, i, j, k) + vr(g, u, i + 1, j, k));
}
__device__ __forceinline__ double ht(const Geo& g, const double* u, int i, int j, int k) {
  return 0.5 * (vt(g, u, i, j, k) + vt(g, u, i, j + 1, k));
}
__device__ __forceinline__ double hp(const Geo& g, const double* u, int i, int j, int k) {
  return 0.5 * (vp(g, u, i, j, k) + vp(g, u, i, j, k + 1));
}
__device__ __forceinline__ double rho_at(const Geo& g, const Coef& c, int i, int j, int k) {
  if (g.per) k = wrapk(g, k);
  return c.rho[IC(g, i, j, k)];
}

// ------------------------------------------------------------------- rows
// p-row (isT = 0) or T-row (isT = 1) of D_d at centre (i,j,k).
__device__ __forceinline__ void row_c(const Geo& g, const Par& P, const Coef& c, int d, int isT, int i, int j,
                                      int k, double wp[3], double wT[3], double wu[2]) {
  long id = IC(g, i, j, k);
  double gm = P.gamma, mu = P.mu;
  double be = c.beta[id];
  double alin = isT ? (gm - 1.0) * c.Tb[id] : gm * c.Pb[id];
  double visc = isT ? mu * be : mu * (gm - 1.0);
  double dif = isT ? be * P.kappa : (gm - 1.0) * P.kappa;
  double g_rr = c.grr[id], g_tt = c.gtt[id], g_pp = c.gpp[id];
  double tr = g_rr + g_tt + g_pp;
  double ir = g.irc[i];
  wp[0] = wp[1] = wp[2] = 0.0;
  wT[0] = wT[1] = wT[2] = 0.0;
  double* wa = isT ? wT : wp;
  if (d == 0) {
    double adv = 0.5 * c.uc0[id] * g.idr;
    wa[0] -= adv; wa[2] += adv;
    double f0 = g.rf[i] * g.rf[i], f1 = g.rf[i + 1] * g.rf[i + 1];
    double ir2 = ir * ir;
    double df = -dif * ir2 * g.idr * g.idr;
    wT[0] += df * f0; wT[1] -= df * (f0 + f1); wT[2] += df * f1;
    double a = alin + (2.0 / 3.0) * visc * tr;
    double m0 = 2.0 * visc * g_rr * g.idr, m1 = visc * (g_tt + g_pp) * ir;
    wu[0] = -a * f0 * ir2 * g.idr + m0 - m1;
    wu[1] = a * f1 * ir2 * g.idr - m0 - m1;
  } else if (d == 1) {
    double is = g.isc[j], cot = g.cotc[j];
    double adv = 0.5 * c.uc1[id] * ir * g.idth;
    wa[0] -= adv; wa[2] += adv;
    double f0 = g.sf[j], f1 = g.sf[j + 1];
    double df = -dif * ir * ir * is * g.idth * g.idth;
    wT[0] += df * f0; wT[1] -= df * (f0 + f1); wT[2] += df * f1;
    double a = alin + (2.0 / 3.0) * visc * tr;
    double lin = -visc * (2.0 * g_pp * cot - c.srt[id]) * 0.5 * ir;
    double m0 = 2.0 * visc * g_tt * ir * g.idth;
    wu[0] = -a * f0 * ir * is * g.idth + m0 + lin;
    wu[1] = a * f1 * ir * is * g.idth - m0 + lin;
  } else {
    double is = g.isc[j], cot = g.cotc[j];
    double adv = 0.5 * c.uc2[id] * ir * is * g.idph;
    wa[0] -= adv; wa[2] += adv;
    double df = -dif * ir * ir * is * is * g.idph * g.idph;
    wT[0] += df; wT[1] -= 2.0 * df; wT[2] += df;
    double a = alin + (2.0 / 3.0) * visc * (tr - 3.0 * g_pp);
    double lin = visc * (c.srp[id] + c.stp[id] * cot) * 0.5 * ir;
    wu[0] = -a * ir * is * g.idph + lin;
    wu[1] = a * ir * is * g.idph + lin;
  }
}

// Normal-velocity row of D_d on the d-face (i,j,k): p at centres m-1, m and
// u_d on faces m-1, m, m+1.  ub: the Ubar velocity component d.
__device__ __forceinline__ void row_f(const Geo& g, const Par& P, const Coef& c, const double* ubd, int d, int i,
                                      int j, int k, double wp[2], double wu[3]) {
  double mu = P.mu;
  if (d == 0) {
    double irh = 2.0 / (rho_at(g, c, i - 1, j, k) + rho_at(g, c, i, j, k));
    double irf = g.irf[i];
    wp[0] = -irh * g.idr; wp[1] = irh * g.idr;
    double adv = 0.5 * ubd[IRf(g, i, j, k)] * g.idr;
    double c0 = g.rc[i - 1] * g.rc[i - 1], c1 = g.rc[i] * g.rc[i];
    double ic0 = g.irc[i - 1] * g.irc[i - 1], ic1 = g.irc[i] * g.irc[i];
    double lap = -mu * irh * irf * irf * g.idr * g.idr;
    double gd = -mu * irh * (1.0 / 3.0) * g.idr * g.idr;
    double fm = g.rf[i - 1] * g.rf[i - 1], f0 = g.rf[i] * g.rf[i], fp = g.rf[i + 1] * g.rf[i + 1];
    wu[0] = -adv + lap * c0 + gd * fm * ic0;
    wu[1] = -lap * (c0 + c1) - gd * f0 * (ic1 + ic0);
    wu[2] = adv + lap * c1 + gd * fp * ic1;
  } else if (d == 1) {
    double irh = 2.0 / (rho_at(g, c, i, j - 1, k) + rho_at(g, c, i, j, k));
    double ir = g.irc[i], isf = g.isf[j];
    wp[0] = -irh * ir * g.idth; wp[1] = irh * ir * g.idth;
    double adv = 0.5 * ubd[ITf(g, i, j, k)] * ir * g.idth;
    double c0 = g.sc[j - 1], c1 = g.sc[j];
    double lap = -mu * irh * ir * ir * isf * g.idth * g.idth;
    double gd = -mu * irh * (1.0 / 3.0) * ir * ir * g.idth * g.idth;
    wu[0] = -adv + lap * c0 + gd * g.sf[j - 1] * g.isc[j - 1];
    wu[1] = -lap * (c0 + c1) - gd * g.sf[j] * (g.isc[j] + g.isc[j - 1]);
    wu[2] = adv + lap * c1 + gd * g.sf[j + 1] * g.isc[j];
  } else {
    double irh = 2.0 / (rho_at(g, c, i, j, k - 1) + rho_at(g, c, i, j, k));
    double ir = g.irc[i], is = g.isc[j];
    wp[0] = -irh * ir * is * g.idph; wp[1] = irh * ir * is * g.idph;
    double adv = 0.5 * ubd[IPf(g, i, j, k)] * ir * is * g.idph;
    double lap = -(4.0 / 3.0) * mu * irh * ir * ir * is * is * g.idph * g.idph;
    wu[0] = -adv + lap; wu[1] = -2.0 * lap; wu[2] = adv + lap;
  }
}

// Transverse row of D_d for velocity component cc at its location (i,j,k).
// ub: the Ubar velocity arrays (1 u_r, 2 u_theta, 3 u_phi of a CF).
__device__ __forceinline__ void row_s(const Geo& g, const Par& P, const Coef& c, const CF& ub, int cc, int d, int i,
                                      int j, int k, double w[3]) {
  double mu = P.mu;
  double rsum;
  if (cc == 0) rsum = rho_at(g, c, i - 1, j, k) + rho_at(g, c, i, j, k);
  else if (cc == 1) rsum = rho_at(g, c, i, j - 1, k) + rho_at(g, c, i, j, k);
  else rsum = rho_at(g, c, i, j, k - 1) + rho_at(g, c, i, j, k);
  double irh = 2.0 / rsum;
  double ir = cc == 0 ? g.irf[i] : g.irc[i];
  double is = cc == 1 ? g.isf[j] : g.isc[j];
  double ua;
  if (cc == 0) ua = d == 1 ? 0.5 * (ht(g, ub.f[2], i - 1, j, k) + ht(g, ub.f[2], i, j, k))
                           : 0.5 * (hp(g, ub.f[3], i - 1, j, k) + hp(g, ub.f[3], i, j, k));
  else if (cc == 1) ua = d == 0 ? 0.5 * (hr(g, ub.f[1], i, j - 1, k) + hr(g, ub.f[1], i, j, k))
                                : 0.5 * (hp(g, ub.f[3], i, j - 1, k) + hp(g, ub.f[3], i, j, k));
  else ua = d == 0 ? 0.5 * (hr(g, ub.f[1], i, j, k - 1) + hr(g, ub.f[1], i, j, k))
                   : 0.5 * (ht(g, ub.f[2], i, j, k - 1) + ht(g, ub.f[2], i, j, k));
  if (d == 0) {
    double adv = 0.5 * ua * g.idr, lap = -mu * irh * ir * ir * g.idr * g.idr;
    double f0 = g.rf[i] * g.rf[i], f1 = g.rf[i + 1] * g.rf[i + 1];
    w[0] = -adv + lap * f0; w[1] = -lap * (f0 + f1); w[2] = adv + lap * f1;
  } else if (d == 1) {
    double adv = 0.5 * ua * ir * g.idth, lap = -mu * irh * ir * ir * is * g.idth * g.idth;
    double f0 = g.sf[j], f1 = g.sf[j + 1];
    w[0] = -adv + lap * f0; w[1] = -lap * (f0 + f1); w[2] = adv + lap * f1;
  } else {
    double adv = 0.5 * ua * ir * is * g.idph, lap = -mu * irh * ir * ir * is * is * g.idph * g.idph;
    w[0] = -adv + lap; w[1] = -2.0 * lap; w[2] = adv + lap;
  }
}

}  // namespace sph
