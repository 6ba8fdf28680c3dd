/*
 * oracle.c -- plain FP64 CPU reference of the direction-splitting scheme of
 * Frolov, Minev & Takhirov, "An efficient algorithm for weakly compressible
 * flows in spherical geometries" (arXiv 2004.13887).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by __graft_entry__.smoke() and by
 * the cpu_baseline / reference legs of bench.py.  It shares no code with the
 * CUDA library.  Nothing here is blocked, fused or reordered: every operator
 * is applied to whole fields exactly as Appendix B splits it, the right-hand
 * side is formed in the order of eq. (spl1), and each line system is
 * assembled explicitly and solved by the block Thomas algorithm of Section 2.2.
 *
 * Discretisation (Section 2.2, MAC stencil): p and T at cell centres, each
 * velocity component on the faces normal to it; first derivatives by central
 * differences, second derivatives in flux (conservative) form; coefficients
 * taken at Ubar = (U^{n+1,k}+U^n)/2 (eq. chapter3mainsd) and moved to staggered
 * points by arithmetic means.  Dirichlet velocity on every wall (tangential
 * ghost = 2*wall - interior), zero Neumann for the p and T perturbations,
 * periodic phi optional.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ grid */

typedef struct {
  int nr, nt, np, per, npf;
  double dr, dth, dph;
  double *rc, *rf, *sc, *sf, *cc, *cf;
} Grid;

static int grid_init(Grid* G, const og_grid* g) {
  if (!g || g->nr < 2 || g->nt < 2 || g->np < 2) return -1;
  if (!(g->r2 > g->r1) || !(g->t2 > g->t1) || !(g->p2 > g->p1) || g->r1 <= 0) return -1;
  if (g->periodic && g->np < 3) return -1;
  G->nr = g->nr; G->nt = g->nt; G->np = g->np; G->per = g->periodic ? 1 : 0;
  G->npf = G->per ? g->np : g->np + 1;
  G->dr = (g->r2 - g->r1) / g->nr;
  G->dth = (g->t2 - g->t1) / g->nt;
  G->dph = (g->p2 - g->p1) / g->np;
  G->rc = malloc(sizeof(double) * g->nr);
  G->rf = malloc(sizeof(double) * (g->nr + 1));
  G->sc = malloc(sizeof(double) * g->nt);
  G->cc = malloc(sizeof(double) * g->nt);
  G->sf = malloc(sizeof(double) * (g->nt + 1));
  G->cf = malloc(sizeof(double) * (g->nt + 1));
  for (int i = 0; i < g->nr; i++) G->rc[i] = g->r1 + (i + 0.5) * G->dr;
  for (int i = 0; i <= g->nr; i++) G->rf[i] = g->r1 + i * G->dr;
  for (int j = 0; j < g->nt; j++) {
    double t = g->t1 + (j + 0.5) * G->dth;
    G->sc[j] = sin(t); G->cc[j] = cos(t);
  }
  for (int j = 0; j <= g->nt; j++) {
    double t = g->t1 + j * G->dth;
    G->sf[j] = sin(t); G->cf[j] = cos(t);
  }
  /* a pole face (theta = 0 or pi) has sin = 0 exactly */
  if (fabs(g->t1) < 1e-14) G->sf[0] = 0.0;
  if (fabs(g->t2 - M_PI) < 1e-14) G->sf[g->nt] = 0.0;
  for (int j = 0; j < g->nt; j++) if (!(G->sc[j] > 0)) return -1;
  return 0;
}

static void grid_free(Grid* G) {
  free(G->rc); free(G->rf); free(G->sc); free(G->cc); free(G->sf); free(G->cf);
}

static size_t IC(const Grid* G, int i, int j, int k) { return ((size_t)i * G->nt + j) * G->np + k; }
static size_t IR(const Grid* G, int i, int j, int k) { return ((size_t)i * G->nt + j) * G->np + k; }
static size_t IT(const Grid* G, int i, int j, int k) { return ((size_t)i * (G->nt + 1) + j) * G->np + k; }
static size_t IP(const Grid* G, int i, int j, int k) { return ((size_t)i * G->nt + j) * G->npf + k; }

static size_t field_size(const Grid* G, int f) {
  switch (f) {
    case 0: case 4: return (size_t)G->nr * G->nt * G->np;
    case 1: return (size_t)(G->nr + 1) * G->nt * G->np;
    case 2: return (size_t)G->nr * (G->nt + 1) * G->np;
    default: return (size_t)G->nr * G->nt * G->npf;
  }
}

/* size of wall array (component c, wall normal d) */
static size_t wall_size(const Grid* G, int c, int d) {
  int nr = G->nr, nt = G->nt, np = G->np, npf = G->npf;
  if (c == 0) return d == 1 ? (size_t)(nr + 1) * np : d == 2 ? (size_t)(nr + 1) * nt : (size_t)nt * np;
  if (c == 1) return d == 0 ? (size_t)(nt + 1) * np : d == 2 ? (size_t)nr * (nt + 1) : (size_t)nr * np;
  return d == 0 ? (size_t)nt * npf : d == 1 ? (size_t)nr * npf : (size_t)nr * nt;
}

static int wrapk(const Grid* G, int k) {
  if (k < 0) return k + G->np;
  if (k >= G->np) return k - G->np;
  return k;
}

/* --------------------------------------------------------------- operand */

typedef struct {
  const double* f[5];        /* p, ur, ut, up, T */
  const double *bgp, *bgT;   /* nr+2 or NULL */
  const double* w[18];
} Op;

static void op_set(Op* o, const double* const* f, const double* bgp, const double* bgT,
                   const double* const* w) {
  for (int q = 0; q < 5; q++) o->f[q] = f[q];
  o->bgp = bgp; o->bgT = bgT;
  for (int q = 0; q < 18; q++) o->w[q] = w ? w[q] : NULL;
}

static double wall(const Op* o, int c, int d, int s, size_t idx) {
  const double* a = o->w[(c * 3 + d) * 2 + s];
  return a ? a[idx] : 0.0;
}

/* scalar at a centre; ghosts: zero Neumann on the perturbation, the
   background keeps its own ghost values */
static double cval(const Grid* G, const double* f, const double* bg, int i, int j, int k) {
  double b = bg ? bg[i + 1] : 0.0;
  int ii = i < 0 ? 0 : (i >= G->nr ? G->nr - 1 : i);
  int jj = j < 0 ? 0 : (j >= G->nt ? G->nt - 1 : j);
  int kk = G->per ? wrapk(G, k) : (k < 0 ? 0 : (k >= G->np ? G->np - 1 : k));
  return b + f[IC(G, ii, jj, kk)];
}
static double P_(const Grid* G, const Op* o, int i, int j, int k) { return cval(G, o->f[0], o->bgp, i, j, k); }
static double T_(const Grid* G, const Op* o, int i, int j, int k) { return cval(G, o->f[4], o->bgT, i, j, k); }

/* u_r on r-face i (0..nr); j, k may be one cell outside */
static double vr(const Grid* G, const Op* o, int i, int j, int k) {
  const double* u = o->f[1];
  if (j < 0 || j >= G->nt) {
    int s = j >= G->nt, jn = s ? G->nt - 1 : 0;
    return 2.0 * wall(o, 0, 1, s, (size_t)i * G->np + k) - u[IR(G, i, jn, k)];
  }
  if (k < 0 || k >= G->np) {
    if (G->per) k = wrapk(G, k);
    else {
      int s = k >= G->np, kn = s ? G->np - 1 : 0;
      return 2.0 * wall(o, 0, 2, s, (size_t)i * G->nt + j) - u[IR(G, i, j, kn)];
    }
  }
  return u[IR(G, i, j, k)];
}

/* u_theta on theta-face j (0..nt); i, k may be one cell outside */
static double vt(const Grid* G, const Op* o, int i, int j, int k) {
  const double* u = o->f[2];
  if (i < 0 || i >= G->nr) {
    int s = i >= G->nr, in = s ? G->nr - 1 : 0;
    return 2.0 * wall(o, 1, 0, s, (size_t)j * G->np + k) - u[IT(G, in, j, k)];
  }
  if (k < 0 || k >= G->np) {
    if (G->per) k = wrapk(G, k);
    else {
      int s = k >= G->np, kn = s ? G->np - 1 : 0;
      return 2.0 * wall(o, 1, 2, s, (size_t)i * (G->nt + 1) + j) - u[IT(G, i, j, kn)];
    }
  }
  return u[IT(G, i, j, k)];
}

/* u_phi on phi-face k; i, j may be one cell outside */
static double vp(const Grid* G, const Op* o, int i, int j, int k) {
  const double* u = o->f[3];
  if (G->per) k = wrapk(G, k);
  if (i < 0 || i >= G->nr) {
    int s = i >= G->nr, in = s ? G->nr - 1 : 0;
    return 2.0 * wall(o, 2, 0, s, (size_t)j * G->npf + k) - u[IP(G, in, j, k)];
  }
  if (j < 0 || j >= G->nt) {
    int s = j >= G->nt, jn = s ? G->nt - 1 : 0;
    return 2.0 * wall(o, 2, 1, s, (size_t)i * G->npf + k) - u[IP(G, i, jn, k)];
  }
  return u[IP(G, i, j, k)];
}

/* velocity components averaged to the centre (i,j,k) */
static double hr(const Grid* G, const Op* o, int i, int j, int k) { return 0.5 * (vr(G, o, i, j, k) + vr(G, o, i + 1, j, k)); }
static double ht(const Grid* G, const Op* o, int i, int j, int k) { return 0.5 * (vt(G, o, i, j, k) + vt(G, o, i, j + 1, k)); }
static double hp(const Grid* G, const Op* o, int i, int j, int k) { return 0.5 * (vp(G, o, i, j, k) + vp(G, o, i, j, k + 1)); }

/* ----------------------------------------------------------- coefficients */

enum { Grr, Gtt, Gpp, Grt, Gtr, Grp, Gpr, Gtp, Gpt };

typedef struct {
  double *Pb, *Tb, *rho, *beta, *uc[3], *G[9];
  Op ub;
} Coef;

static void coef_free(Coef* c) {
  free(c->Pb); free(c->Tb); free(c->rho); free(c->beta);
  for (int q = 0; q < 3; q++) free(c->uc[q]);
  for (int q = 0; q < 9; q++) free(c->G[q]);
}

/* Everything the operators freeze at Ubar (eq. chapter3mainsd, App. B):
   p+pi_inf, T, rho by the stiffened-gas EOS (eq. nonconserveos),
   (gamma-1)T/(p+pi_inf), centre velocities and G = grad(u) with metric terms. */
static void coef_make(const Grid* G, const og_par* P, const Op* ub, Coef* c) {
  size_t n = field_size(G, 0);
  c->ub = *ub;
  c->Pb = malloc(n * sizeof(double)); c->Tb = malloc(n * sizeof(double));
  c->rho = malloc(n * sizeof(double)); c->beta = malloc(n * sizeof(double));
  for (int q = 0; q < 3; q++) c->uc[q] = malloc(n * sizeof(double));
  for (int q = 0; q < 9; q++) c->G[q] = malloc(n * sizeof(double));
  double gm = P->gamma, Rg = P->cv * (gm - 1.0);
#pragma omp parallel for collapse(2)
  for (int i = 0; i < G->nr; i++)
    for (int j = 0; j < G->nt; j++)
      for (int k = 0; k < G->np; k++) {
        size_t id = IC(G, i, j, k);
        double pb = P_(G, ub, i, j, k) + P->pinf, tb = T_(G, ub, i, j, k);
        c->Pb[id] = pb; c->Tb[id] = tb;
        c->rho[id] = pb / (Rg * tb);
        c->beta[id] = (gm - 1.0) * tb / pb;
        double ur = hr(G, ub, i, j, k), ut = ht(G, ub, i, j, k), up = hp(G, ub, i, j, k);
        c->uc[0][id] = ur; c->uc[1][id] = ut; c->uc[2][id] = up;
        double r = G->rc[i], s = G->sc[j], cot = G->cc[j] / G->sc[j];
        c->G[Grr][id] = (vr(G, ub, i + 1, j, k) - vr(G, ub, i, j, k)) / G->dr;
        c->G[Gtt][id] = (vt(G, ub, i, j + 1, k) - vt(G, ub, i, j, k)) / (r * G->dth) + ur / r;
        c->G[Gpp][id] = (vp(G, ub, i, j, k + 1) - vp(G, ub, i, j, k)) / (r * s * G->dph) + ur / r + ut * cot / r;
        c->G[Grt][id] = (ht(G, ub, i + 1, j, k) - ht(G, ub, i - 1, j, k)) / (2 * G->dr);
        c->G[Gtr][id] = (hr(G, ub, i, j + 1, k) - hr(G, ub, i, j - 1, k)) / (2 * r * G->dth) - ut / r;
        c->G[Grp][id] = (hp(G, ub, i + 1, j, k) - hp(G, ub, i - 1, j, k)) / (2 * G->dr);
        c->G[Gpr][id] = (hr(G, ub, i, j, k + 1) - hr(G, ub, i, j, k - 1)) / (2 * r * s * G->dph) - up / r;
        c->G[Gtp][id] = (hp(G, ub, i, j + 1, k) - hp(G, ub, i, j - 1, k)) / (2 * r * G->dth);
        c->G[Gpt][id] = (ht(G, ub, i, j, k + 1) - ht(G, ub, i, j, k - 1)) / (2 * r * s * G->dph) - up * cot / r;
      }
}

static double rho_at(const Grid* G, const Coef* c, int i, int j, int k) {
  if (G->per) k = wrapk(G, k);
  return c->rho[IC(G, i, j, k)];
}

/* ---------------------------------------------------- directional weights */

/* p-row (isT=0: A1^d, A2^d, A3^d) or T-row (isT=1: C2^d, C3^d) of D_d at the
   centre (i,j,k).  Reads p (wp) and T (wT) at centres m-1, m, m+1 along d and
   u_d (wu) on the faces m and m+1 that bound the cell. */
static void w_centre(const Grid* G, const og_par* P, const Coef* c, int d, int isT,
                     int i, int j, int k, double wp[3], double wT[3], double wu[2]) {
  size_t id = IC(G, i, j, k);
  double gm = P->gamma, mu = P->mu, kap = mu * gm * P->cv / P->Pr;
  double be = c->beta[id];
  double alin = isT ? (gm - 1.0) * c->Tb[id] : gm * c->Pb[id];
  double visc = isT ? mu * be : mu * (gm - 1.0);
  double dif = isT ? be * kap : (gm - 1.0) * kap;
  double g_rr = c->G[Grr][id], g_tt = c->G[Gtt][id], g_pp = c->G[Gpp][id];
  double g_rt = c->G[Grt][id], g_tr = c->G[Gtr][id], g_rp = c->G[Grp][id];
  double g_pr = c->G[Gpr][id], g_tp = c->G[Gtp][id], g_pt = c->G[Gpt][id];
  double tr = g_rr + g_tt + g_pp;
  double r = G->rc[i], s = G->sc[j], cot = G->cc[j] / G->sc[j];
  for (int q = 0; q < 3; q++) { wp[q] = 0; wT[q] = 0; }
  double* wa = isT ? wT : wp;
  if (d == 0) {
    double adv = c->uc[0][id] / (2 * G->dr);
    wa[0] -= adv; wa[2] += adv;
    double f0 = G->rf[i] * G->rf[i], f1 = G->rf[i + 1] * G->rf[i + 1];
    double df = -dif / (r * r * G->dr * G->dr);
    wT[0] += df * f0; wT[1] -= df * (f0 + f1); wT[2] += df * f1;
    double a = alin + 2.0 * visc / 3.0 * tr;
    wu[0] = -a * f0 / (r * r * G->dr) + 2 * visc * g_rr / G->dr - visc * (g_tt + g_pp) / r;
    wu[1] = a * f1 / (r * r * G->dr) - 2 * visc * g_rr / G->dr - visc * (g_tt + g_pp) / r;
  } else if (d == 1) {
    double adv = c->uc[1][id] / (2 * r * G->dth);
    wa[0] -= adv; wa[2] += adv;
    double f0 = G->sf[j], f1 = G->sf[j + 1];
    double df = -dif / (r * r * s * G->dth * G->dth);
    wT[0] += df * f0; wT[1] -= df * (f0 + f1); wT[2] += df * f1;
    double a = alin + 2.0 * visc / 3.0 * tr;
    double lin = -visc * (2 * g_pp * cot - g_rt - g_tr) / (2 * r);
    wu[0] = -a * f0 / (r * s * G->dth) + 2 * visc * g_tt / (r * G->dth) + lin;
    wu[1] = a * f1 / (r * s * G->dth) - 2 * visc * g_tt / (r * G->dth) + lin;
  } else {
    double adv = c->uc[2][id] / (2 * r * s * G->dph);
    wa[0] -= adv; wa[2] += adv;
    double df = -dif / (r * r * s * s * G->dph * G->dph);
    wT[0] += df; wT[1] -= 2 * df; wT[2] += df;
    double a = alin + 2.0 * visc / 3.0 * (tr - 3 * g_pp);
    double lin = visc * (g_rp + g_pr + (g_tp + g_pt) * cot) / (2 * r);
    wu[0] = -a / (r * s * G->dph) + lin;
    wu[1] = a / (r * s * G->dph) + lin;
  }
}

/* Normal-velocity row (B1^d, B2^{d,d}) of D_d on the d-face (i,j,k), index m
   along d: p at centres m-1, m (wp) and u_d on faces m-1, m, m+1 (wu). */
static void w_face(const Grid* G, const og_par* P, const Coef* c, int d,
                   int i, int j, int k, double wp[2], double wu[3]) {
  double mu = P->mu;
  const Op* ub = &c->ub;
  if (d == 0) {
    double ir = 2.0 / (rho_at(G, c, i - 1, j, k) + rho_at(G, c, i, j, k));
    double r = G->rf[i];
    wp[0] = -ir / G->dr; wp[1] = ir / G->dr;
    double adv = vr(G, ub, i, j, k) / (2 * G->dr);
    double c0 = G->rc[i - 1] * G->rc[i - 1], c1 = G->rc[i] * G->rc[i];
    double lap = -mu * ir / (r * r * G->dr * G->dr);
    double gd = -mu * ir / (3 * G->dr * G->dr);
    double fm = G->rf[i - 1] * G->rf[i - 1], f0 = G->rf[i] * G->rf[i], fp = G->rf[i + 1] * G->rf[i + 1];
    wu[0] = -adv + lap * c0 + gd * fm / c0;
    wu[1] = -lap * (c0 + c1) - gd * (f0 / c1 + f0 / c0);
    wu[2] = adv + lap * c1 + gd * fp / c1;
  } else if (d == 1) {
    double ir = 2.0 / (rho_at(G, c, i, j - 1, k) + rho_at(G, c, i, j, k));
    double r = G->rc[i], s = G->sf[j];
    wp[0] = -ir / (r * G->dth); wp[1] = ir / (r * G->dth);
    double adv = vt(G, ub, i, j, k) / (2 * r * G->dth);
    double c0 = G->sc[j - 1], c1 = G->sc[j];
    double lap = -mu * ir / (r * r * s * G->dth * G->dth);
    double gd = -mu * ir / (3 * r * r * G->dth * G->dth);
    wu[0] = -adv + lap * c0 + gd * G->sf[j - 1] / c0;
    wu[1] = -lap * (c0 + c1) - gd * (G->sf[j] / c1 + G->sf[j] / c0);
    wu[2] = adv + lap * c1 + gd * G->sf[j + 1] / c1;
  } else {
    double ir = 2.0 / (rho_at(G, c, i, j, k - 1) + rho_at(G, c, i, j, k));
    double r = G->rc[i], s = G->sc[j];
    wp[0] = -ir / (r * s * G->dph); wp[1] = ir / (r * s * G->dph);
    double adv = vp(G, ub, i, j, k) / (2 * r * s * G->dph);
    double lap = -4.0 / 3.0 * mu * ir / (r * r * s * s * G->dph * G->dph);
    wu[0] = -adv + lap; wu[1] = -2 * lap; wu[2] = adv + lap;
  }
}

/* Transverse scalar row B2^{d,cc} of D_d for velocity component cc at its own
   location (i,j,k): u_cc at m-1, m, m+1 along d. */
static void w_scal(const Grid* G, const og_par* P, const Coef* c, int cc, int d,
                   int i, int j, int k, double w[3]) {
  double mu = P->mu;
  const Op* ub = &c->ub;
  double rf_;
  if (cc == 0) rf_ = 0.5 * (rho_at(G, c, i - 1, j, k) + rho_at(G, c, i, j, k));
  else if (cc == 1) rf_ = 0.5 * (rho_at(G, c, i, j - 1, k) + rho_at(G, c, i, j, k));
  else rf_ = 0.5 * (rho_at(G, c, i, j, k - 1) + rho_at(G, c, i, j, k));
  double ir = 1.0 / rf_;
  double r = cc == 0 ? G->rf[i] : G->rc[i];
  double s = cc == 1 ? G->sf[j] : G->sc[j];
  double ua;
  if (cc == 0) ua = d == 1 ? 0.5 * (ht(G, ub, i - 1, j, k) + ht(G, ub, i, j, k))
                           : 0.5 * (hp(G, ub, i - 1, j, k) + hp(G, ub, i, j, k));
  else if (cc == 1) ua = d == 0 ? 0.5 * (hr(G, ub, i, j - 1, k) + hr(G, ub, i, j, k))
                                : 0.5 * (hp(G, ub, i, j - 1, k) + hp(G, ub, i, j, k));
  else ua = d == 0 ? 0.5 * (hr(G, ub, i, j, k - 1) + hr(G, ub, i, j, k))
                   : 0.5 * (ht(G, ub, i, j, k - 1) + ht(G, ub, i, j, k));
  if (d == 0) {
    double adv = ua / (2 * G->dr), lap = -mu * ir / (r * r * G->dr * G->dr);
    double f0 = G->rf[i] * G->rf[i], f1 = G->rf[i + 1] * G->rf[i + 1];
    w[0] = -adv + lap * f0; w[1] = -lap * (f0 + f1); w[2] = adv + lap * f1;
  } else if (d == 1) {
    double adv = ua / (2 * r * G->dth), lap = -mu * ir / (r * r * s * G->dth * G->dth);
    double f0 = G->sf[j], f1 = G->sf[j + 1];
    w[0] = -adv + lap * f0; w[1] = -lap * (f0 + f1); w[2] = adv + lap * f1;
  } else {
    double adv = ua / (2 * r * s * G->dph), lap = -mu * ir / (r * r * s * s * G->dph * G->dph);
    w[0] = -adv + lap; w[1] = -2 * lap; w[2] = adv + lap;
  }
}

/* ------------------------------------------------------- operator apply */

static void zero_fields(const Grid* G, double* const* out) {
  for (int f = 0; f < 5; f++) memset(out[f], 0, field_size(G, f) * sizeof(double));
}

/* value of velocity component cc at its location shifted by s along d */
static double vel_shift(const Grid* G, const Op* o, int cc, int d, int i, int j, int k, int s) {
  if (d == 0) i += s; else if (d == 1) j += s; else k += s;
  return cc == 0 ? vr(G, o, i, j, k) : cc == 1 ? vt(G, o, i, j, k) : vp(G, o, i, j, k);
}

static int kface_lo(const Grid* G) { return G->per ? 0 : 1; }

/* out += D_d(Ubar) V */
static void apply_dir(const Grid* G, const og_par* P, const Coef* c, int d, const Op* V,
                      double* const* out) {
  int di = d == 0, dj = d == 1, dk = d == 2;
  /* p- and T-rows at the centres */
#pragma omp parallel for collapse(2)
  for (int i = 0; i < G->nr; i++)
    for (int j = 0; j < G->nt; j++)
      for (int k = 0; k < G->np; k++) {
        double wp[3], wT[3], wu[2];
        double pv[3], Tv[3], uv[2];
        for (int s = -1; s <= 1; s++) {
          pv[s + 1] = P_(G, V, i + s * di, j + s * dj, k + s * dk);
          Tv[s + 1] = T_(G, V, i + s * di, j + s * dj, k + s * dk);
        }
        if (d == 0) { uv[0] = vr(G, V, i, j, k); uv[1] = vr(G, V, i + 1, j, k); }
        else if (d == 1) { uv[0] = vt(G, V, i, j, k); uv[1] = vt(G, V, i, j + 1, k); }
        else { uv[0] = vp(G, V, i, j, k); uv[1] = vp(G, V, i, j, k + 1); }
        size_t id = IC(G, i, j, k);
        for (int isT = 0; isT < 2; isT++) {
          w_centre(G, P, c, d, isT, i, j, k, wp, wT, wu);
          double acc = 0;
          for (int q = 0; q < 3; q++) acc += wp[q] * pv[q] + wT[q] * Tv[q];
          acc += wu[0] * uv[0] + wu[1] * uv[1];
          out[isT ? 4 : 0][id] += acc;
        }
      }
  /* velocity rows: the normal one (w_face) and the two transverse ones (w_scal) */
  for (int cc = 0; cc < 3; cc++) {
    int i0 = cc == 0 ? 1 : 0, i1 = cc == 0 ? G->nr - 1 : G->nr - 1;
    int j0 = cc == 1 ? 1 : 0, j1 = cc == 1 ? G->nt - 1 : G->nt - 1;
    int k0 = cc == 2 ? kface_lo(G) : 0, k1 = G->np - 1;
#pragma omp parallel for collapse(2)
    for (int i = i0; i <= i1; i++)
      for (int j = j0; j <= j1; j++)
        for (int k = k0; k <= k1; k++) {
          double acc = 0;
          size_t id = cc == 0 ? IR(G, i, j, k) : cc == 1 ? IT(G, i, j, k) : IP(G, i, j, k);
          if (cc == d) {
            double wp[2], wu[3];
            w_face(G, P, c, d, i, j, k, wp, wu);
            acc += wp[0] * P_(G, V, i - di, j - dj, k - dk) + wp[1] * P_(G, V, i, j, k);
            for (int s = -1; s <= 1; s++) acc += wu[s + 1] * vel_shift(G, V, cc, d, i, j, k, s);
          } else {
            double w[3];
            w_scal(G, P, c, cc, d, i, j, k, w);
            for (int s = -1; s <= 1; s++) acc += w[s + 1] * vel_shift(G, V, cc, d, i, j, k, s);
          }
          out[1 + cc][id] += acc;
        }
  }
}

/* out += D_M(Ubar) V: cross derivatives, curvature, Coriolis and the parts of
   grad(div v)/3 and of the vector Laplacian that are not along one line. */
static void apply_M(const Grid* G, const og_par* P, const Coef* c, const Op* V,
                    double* const* out) {
  double gm = P->gamma, mu = P->mu, om = P->omega;
  const Op* ub = &c->ub;
  double dr = G->dr, dth = G->dth, dph = G->dph;
#pragma omp parallel for collapse(2)
  for (int i = 0; i < G->nr; i++)
    for (int j = 0; j < G->nt; j++)
      for (int k = 0; k < G->np; k++) {
        size_t id = IC(G, i, j, k);
        double r = G->rc[i], s = G->sc[j];
        double xrt = (ht(G, V, i + 1, j, k) - ht(G, V, i - 1, j, k)) / (2 * dr)
                   + (hr(G, V, i, j + 1, k) - hr(G, V, i, j - 1, k)) / (2 * r * dth);
        double xrp = (hp(G, V, i + 1, j, k) - hp(G, V, i - 1, j, k)) / (2 * dr)
                   + (hr(G, V, i, j, k + 1) - hr(G, V, i, j, k - 1)) / (2 * r * s * dph);
        double xtp = (hp(G, V, i, j + 1, k) - hp(G, V, i, j - 1, k)) / (2 * r * dth)
                   + (ht(G, V, i, j, k + 1) - ht(G, V, i, j, k - 1)) / (2 * r * s * dph);
        double cross = (c->G[Grt][id] + c->G[Gtr][id]) * xrt + (c->G[Grp][id] + c->G[Gpr][id]) * xrp
                     + (c->G[Gtp][id] + c->G[Gpt][id]) * xtp;
        out[0][id] += -mu * (gm - 1.0) * cross;
        out[4][id] += -mu * c->beta[id] * cross;
      }
  /* r-momentum on interior r-faces */
#pragma omp parallel for collapse(2)
  for (int i = 1; i < G->nr; i++)
    for (int j = 0; j < G->nt; j++)
      for (int k = 0; k < G->np; k++) {
        double r = G->rf[i], s = G->sc[j];
        double ir = 2.0 / (rho_at(G, c, i - 1, j, k) + rho_at(G, c, i, j, k));
        double utf = 0.5 * (ht(G, ub, i - 1, j, k) + ht(G, ub, i, j, k));
        double upf = 0.5 * (hp(G, ub, i - 1, j, k) + hp(G, ub, i, j, k));
        double vtf = 0.5 * (ht(G, V, i - 1, j, k) + ht(G, V, i, j, k));
        double vpf = 0.5 * (hp(G, V, i - 1, j, k) + hp(G, V, i, j, k));
        double Q[2];
        for (int q = 0; q < 2; q++) {
          int m = i - 1 + q;
          Q[q] = (G->sf[j + 1] * vt(G, V, m, j + 1, k) - G->sf[j] * vt(G, V, m, j, k)) / (G->rc[m] * s * dth)
               + (vp(G, V, m, j, k + 1) - vp(G, V, m, j, k)) / (G->rc[m] * s * dph);
        }
        double acc = -utf * vtf / r - upf * vpf / r + 2 * mu * ir * vr(G, V, i, j, k) / (r * r)
                   - 2 * om * s * vpf
                   - mu * ir / (3 * dr) * (Q[1] - Q[0]) + 2 * mu * ir / r * 0.5 * (Q[0] + Q[1]);
        out[1][IR(G, i, j, k)] += acc;
      }
  /* theta-momentum on interior theta-faces */
#pragma omp parallel for collapse(2)
  for (int i = 0; i < G->nr; i++)
    for (int j = 1; j < G->nt; j++)
      for (int k = 0; k < G->np; k++) {
        double r = G->rc[i], sfj = G->sf[j], cfj = G->cf[j];
        double ir = 2.0 / (rho_at(G, c, i, j - 1, k) + rho_at(G, c, i, j, k));
        double ubt = vt(G, ub, i, j, k);
        double upf = 0.5 * (hp(G, ub, i, j - 1, k) + hp(G, ub, i, j, k));
        double vrf = 0.5 * (hr(G, V, i, j - 1, k) + hr(G, V, i, j, k));
        double vpf = 0.5 * (hp(G, V, i, j - 1, k) + hp(G, V, i, j, k));
        double Dr[2], Dp[2], dpf = 0;
        for (int q = 0; q < 2; q++) {
          int m = j - 1 + q;
          Dr[q] = (G->rf[i + 1] * G->rf[i + 1] * vr(G, V, i + 1, m, k) - G->rf[i] * G->rf[i] * vr(G, V, i, m, k))
                / (r * r * dr);
          double dvp = vp(G, V, i, m, k + 1) - vp(G, V, i, m, k);
          Dp[q] = dvp / (r * G->sc[m] * dph);
          dpf += 0.5 * dvp / dph;
        }
        double acc = ubt * vrf / r - upf * vpf * (cfj / sfj) / r + mu * ir * vt(G, V, i, j, k) / (r * r * sfj * sfj)
                   - 2 * om * cfj * vpf
                   - mu * ir / (3 * r * dth) * ((Dr[1] - Dr[0]) + (Dp[1] - Dp[0]))
                   - mu * ir * (2.0 / (r * r * dth) * (hr(G, V, i, j, k) - hr(G, V, i, j - 1, k))
                                - 2.0 * cfj / (r * r * sfj * sfj) * dpf);
        out[2][IT(G, i, j, k)] += acc;
      }
  /* phi-momentum on interior (or all, if periodic) phi-faces */
  int k0 = kface_lo(G);
#pragma omp parallel for collapse(2)
  for (int i = 0; i < G->nr; i++)
    for (int j = 0; j < G->nt; j++)
      for (int k = k0; k < G->np; k++) {
        double r = G->rc[i], s = G->sc[j], cj = G->cc[j];
        double ir = 2.0 / (rho_at(G, c, i, j, k - 1) + rho_at(G, c, i, j, k));
        double ubp = vp(G, ub, i, j, k);
        double vrf = 0.5 * (hr(G, V, i, j, k - 1) + hr(G, V, i, j, k));
        double vtf = 0.5 * (ht(G, V, i, j, k - 1) + ht(G, V, i, j, k));
        double Dr[2], Dt[2];
        for (int q = 0; q < 2; q++) {
          int m = k - 1 + q;
          Dr[q] = (G->rf[i + 1] * G->rf[i + 1] * vr(G, V, i + 1, j, m) - G->rf[i] * G->rf[i] * vr(G, V, i, j, m))
                / (r * r * dr);
          Dt[q] = (G->sf[j + 1] * vt(G, V, i, j + 1, m) - G->sf[j] * vt(G, V, i, j, m)) / (r * s * dth);
        }
        double acc = ubp * vtf * (cj / s) / r + ubp * vrf / r + mu * ir * vp(G, V, i, j, k) / (r * r * s * s)
                   + 2 * om * (cj * vtf + s * vrf)
                   - mu * ir / (3 * r * s * dph) * ((Dr[1] - Dr[0]) + (Dt[1] - Dt[0]))
                   - mu * ir * (2.0 / (r * r * s * dph) * (hr(G, V, i, j, k) - hr(G, V, i, j, k - 1))
                                + 2.0 * cj / (r * r * s * s * dph) * (ht(G, V, i, j, k) - ht(G, V, i, j, k - 1)));
        out[3][IP(G, i, j, k)] += acc;
      }
}

/* --------------------------------------------------------- line solvers */

/* Solve S X = Y for a 3x3 S and m right-hand-side columns (Y is 3 x m,
   row-major, overwritten by X), Gaussian elimination with partial pivoting. */
static int solve3(const double* S, double* Y, int m) {
  double a[9];
  memcpy(a, S, sizeof a);
  for (int col = 0; col < 3; col++) {
    int piv = col;
    for (int r = col + 1; r < 3; r++) if (fabs(a[r * 3 + col]) > fabs(a[piv * 3 + col])) piv = r;
    if (a[piv * 3 + col] == 0.0) return -1;
    if (piv != col) {
      for (int q = 0; q < 3; q++) { double t = a[col * 3 + q]; a[col * 3 + q] = a[piv * 3 + q]; a[piv * 3 + q] = t; }
      for (int q = 0; q < m; q++) { double t = Y[col * m + q]; Y[col * m + q] = Y[piv * m + q]; Y[piv * m + q] = t; }
    }
    for (int r = col + 1; r < 3; r++) {
      double f = a[r * 3 + col] / a[col * 3 + col];
      for (int q = col; q < 3; q++) a[r * 3 + q] -= f * a[col * 3 + q];
      for (int q = 0; q < m; q++) Y[r * m + q] -= f * Y[col * m + q];
    }
  }
  for (int r = 2; r >= 0; r--) {
    for (int q = 0; q < m; q++) {
      double v = Y[r * m + q];
      for (int t = r + 1; t < 3; t++) v -= a[r * 3 + t] * Y[t * m + q];
      Y[r * m + q] = v / a[r * 3 + r];
    }
  }
  return 0;
}

static void mm3(const double* A, const double* B, double* C) {   /* C = A B */
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) C[r * 3 + q] = A[r * 3] * B[q] + A[r * 3 + 1] * B[3 + q] + A[r * 3 + 2] * B[6 + q];
}
static void mv3(const double* A, const double* x, double* y) {   /* y = A x */
  for (int r = 0; r < 3; r++) y[r] = A[r * 3] * x[0] + A[r * 3 + 1] * x[1] + A[r * 3 + 2] * x[2];
}

int og_thomas(int n, const double* a, const double* b, const double* c, const double* d, double* x) {
  if (n < 1) return -1;
  double* cp = malloc(sizeof(double) * n);
  double* dp = malloc(sizeof(double) * n);
  double den = b[0];
  if (den == 0.0) { free(cp); free(dp); return -2; }
  cp[0] = c[0] / den; dp[0] = d[0] / den;
  for (int m = 1; m < n; m++) {
    den = b[m] - a[m] * cp[m - 1];
    if (den == 0.0) { free(cp); free(dp); return -2; }
    cp[m] = c[m] / den;
    dp[m] = (d[m] - a[m] * dp[m - 1]) / den;
  }
  x[n - 1] = dp[n - 1];
  for (int m = n - 2; m >= 0; m--) x[m] = dp[m] - cp[m] * x[m + 1];
  free(cp); free(dp);
  return 0;
}

/* Periodic scalar system, a[0] couples row 0 to x[n-1] and c[n-1] couples
   row n-1 to x[0]; Sherman-Morrison on the Thomas solver. */
int og_cyclic_thomas(int n, const double* a, const double* b, const double* c, const double* d, double* x) {
  if (n < 3) return -1;
  double gam = -b[0];
  if (gam == 0.0) return -2;
  double* bb = malloc(sizeof(double) * n);
  double* u = calloc(n, sizeof(double));
  double* z = malloc(sizeof(double) * n);
  memcpy(bb, b, sizeof(double) * n);
  bb[0] = b[0] - gam;
  bb[n - 1] = b[n - 1] - a[0] * c[n - 1] / gam;
  u[0] = gam; u[n - 1] = c[n - 1];
  int e = og_thomas(n, a, bb, c, d, x);
  if (!e) e = og_thomas(n, a, bb, c, u, z);
  if (!e) {
    double vy = x[0] + a[0] / gam * x[n - 1];
    double vz = z[0] + a[0] / gam * z[n - 1];
    double f = vy / (1.0 + vz);
    for (int m = 0; m < n; m++) x[m] -= f * z[m];
  }
  free(bb); free(u); free(z);
  return e;
}

/* Block Thomas (Section 2.2): forward elimination S_m = B_m - A_m C'_{m-1},
   C'_m = S_m^{-1} C_m, d'_m = S_m^{-1}(d_m - A_m d'_{m-1}); back substitution
   x_m = d'_m - C'_m x_{m+1}.  No pivoting between blocks.  d may hold nrhs
   columns per block (row-major 3 x nrhs). */
static int block_thomas_multi(int n, const double* A, const double* B, const double* C,
                              const double* d, double* x, int nrhs) {
  if (n < 1) return -1;
  int w = 3 + nrhs;
  double* Y = malloc(sizeof(double) * 3 * w * n);   /* [C'_m | d'_m] */
  double S[9], tmp[9];
  for (int m = 0; m < n; m++) {
    memcpy(S, B + 9 * m, sizeof S);
    double* y = Y + (size_t)3 * w * m;
    for (int r = 0; r < 3; r++) {
      for (int q = 0; q < 3; q++) y[r * w + q] = C[9 * m + r * 3 + q];
      for (int q = 0; q < nrhs; q++) y[r * w + 3 + q] = d[((size_t)m * 3 + r) * nrhs + q];
    }
    if (m > 0) {
      const double* yp = Y + (size_t)3 * w * (m - 1);
      double Cp[9];
      for (int r = 0; r < 3; r++) for (int q = 0; q < 3; q++) Cp[r * 3 + q] = yp[r * w + q];
      mm3(A + 9 * m, Cp, tmp);
      for (int q = 0; q < 9; q++) S[q] -= tmp[q];
      for (int q = 0; q < nrhs; q++)
        for (int r = 0; r < 3; r++) {
          double v = 0;
          for (int t = 0; t < 3; t++) v += A[9 * m + r * 3 + t] * yp[t * w + 3 + q];
          y[r * w + 3 + q] -= v;
        }
    }
    if (solve3(S, y, w)) { free(Y); return -2; }
  }
  for (int m = n - 1; m >= 0; m--) {
    const double* y = Y + (size_t)3 * w * m;
    for (int q = 0; q < nrhs; q++)
      for (int r = 0; r < 3; r++) {
        double v = y[r * w + 3 + q];
        if (m < n - 1)
          for (int t = 0; t < 3; t++) v -= y[r * w + t] * x[((size_t)(m + 1) * 3 + t) * nrhs + q];
        x[((size_t)m * 3 + r) * nrhs + q] = v;
      }
  }
  free(Y);
  return 0;
}

int og_block_thomas(int n, const double* A, const double* B, const double* C, const double* d, double* x) {
  return block_thomas_multi(n, A, B, C, d, x, 1);
}

/* Periodic block system (A_0 couples block 0 to block n-1, C_{n-1} couples
   block n-1 to block 0): Woodbury with the rank-3 split
   M = T + U V^T, U = [Gam; 0; ..; C_{n-1}], V^T = [I, 0, .., Gam^{-1} A_0],
   Gam = -B_0, T the block-tridiagonal part with corners adjusted. */
int og_block_cyclic(int n, const double* A, const double* B, const double* C, const double* d, double* x) {
  if (n < 3) return -1;
  double* BB = malloc(sizeof(double) * 9 * n);
  memcpy(BB, B, sizeof(double) * 9 * n);
  double Gam[9], GiA[9], tmp[9];
  for (int q = 0; q < 9; q++) Gam[q] = -B[q];
  /* Gam^{-1} A_0 */
  for (int q = 0; q < 9; q++) GiA[q] = A[q];
  if (solve3(Gam, GiA, 3)) { free(BB); return -2; }
  for (int q = 0; q < 9; q++) BB[q] = B[q] - Gam[q];
  mm3(C + 9 * (n - 1), GiA, tmp);
  for (int q = 0; q < 9; q++) BB[9 * (n - 1) + q] = B[9 * (n - 1) + q] - tmp[q];
  /* right-hand sides: column 0 = d, columns 1..3 = U */
  double* R = calloc((size_t)3 * 4 * n, sizeof(double));
  double* X = malloc(sizeof(double) * 3 * 4 * n);
  for (int m = 0; m < n; m++)
    for (int r = 0; r < 3; r++) R[((size_t)m * 3 + r) * 4] = d[m * 3 + r];
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) {
      R[((size_t)0 * 3 + r) * 4 + 1 + q] = Gam[r * 3 + q];
      R[((size_t)(n - 1) * 3 + r) * 4 + 1 + q] = C[9 * (n - 1) + r * 3 + q];
    }
  int e = block_thomas_multi(n, A, BB, C, R, X, 4);
  if (!e) {
    /* V^T y and V^T Z */
    double vy[3], vz[9], y0[3], yl[3], z0[9], zl[9];
    for (int r = 0; r < 3; r++) {
      y0[r] = X[(0 * 3 + r) * 4]; yl[r] = X[((size_t)(n - 1) * 3 + r) * 4];
      for (int q = 0; q < 3; q++) {
        z0[r * 3 + q] = X[(0 * 3 + r) * 4 + 1 + q];
        zl[r * 3 + q] = X[((size_t)(n - 1) * 3 + r) * 4 + 1 + q];
      }
    }
    mv3(GiA, yl, vy);
    for (int r = 0; r < 3; r++) vy[r] += y0[r];
    mm3(GiA, zl, vz);
    for (int q = 0; q < 9; q++) vz[q] += z0[q];
    for (int r = 0; r < 3; r++) vz[r * 3 + r] += 1.0;
    /* f = (I + V^T Z)^{-1} V^T y */
    double f[3] = {vy[0], vy[1], vy[2]};
    if (solve3(vz, f, 1)) e = -2;
    if (!e)
      for (int m = 0; m < n; m++)
        for (int r = 0; r < 3; r++) {
          double v = X[((size_t)m * 3 + r) * 4];
          for (int q = 0; q < 3; q++) v -= X[((size_t)m * 3 + r) * 4 + 1 + q] * f[q];
          x[m * 3 + r] = v;
        }
  }
  free(BB); free(R); free(X);
  return e;
}

/* --------------------------------------------------------- line assembly */

/* centre (i,j,k) of cell m on line (a,b) along d */
static void line_centre(int d, int a, int b, int m, int* i, int* j, int* k) {
  if (d == 0) { *i = m; *j = a; *k = b; }
  else if (d == 1) { *i = a; *j = m; *k = b; }
  else { *i = a; *j = b; *k = m; }
}

static int line_len(const Grid* G, int d) { return d == 0 ? G->nr : d == 1 ? G->nt : G->np; }

/* transverse component of kind 1/2 for direction d */
static int trans_comp(int d, int kind) {
  if (d == 0) return kind == 1 ? 1 : 2;
  if (d == 1) return kind == 1 ? 0 : 2;
  return kind == 1 ? 0 : 1;
}

/* assemble (I + tau/2 D_d) on one line; returns n */
static int assemble(const Grid* G, const og_par* P, const Coef* c, int d, int kind, int a, int b,
                    double tau, double* A, double* B, double* C) {
  int n = line_len(G, d);
  int cyc = (d == 2 && G->per);
  double h = 0.5 * tau;
  if (kind == 0) {
    for (int m = 0; m < n; m++) {
      double* Am = A + 9 * m; double* Bm = B + 9 * m; double* Cm = C + 9 * m;
      memset(Am, 0, 9 * sizeof(double)); memset(Bm, 0, 9 * sizeof(double)); memset(Cm, 0, 9 * sizeof(double));
      int i, j, k;
      line_centre(d, a, b, m, &i, &j, &k);
      double wp[3], wT[3], wu[2];
      for (int isT = 0; isT < 2; isT++) {
        w_centre(G, P, c, d, isT, i, j, k, wp, wT, wu);
        int row = isT ? 1 : 0;
        Am[row * 3 + 0] = h * wp[0]; Am[row * 3 + 1] = h * wT[0]; Am[row * 3 + 2] = h * wu[0];
        Bm[row * 3 + 0] = h * wp[1]; Bm[row * 3 + 1] = h * wT[1]; Bm[row * 3 + 2] = h * wu[1];
        Cm[row * 3 + 0] = h * wp[2]; Cm[row * 3 + 1] = h * wT[2];
      }
      /* normal-velocity row on face m+1 */
      if (m < n - 1 || cyc) {
        int fi = i, fj = j, fk = k;
        if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = (m + 1) % n;
        double fp[2], fu[3];
        w_face(G, P, c, d, fi, fj, fk, fp, fu);
        Am[2 * 3 + 2] = h * fu[0];
        Bm[2 * 3 + 0] = h * fp[0]; Bm[2 * 3 + 2] = h * fu[1];
        Cm[2 * 3 + 0] = h * fp[1]; Cm[2 * 3 + 2] = h * fu[2];
      }
      for (int q = 0; q < 3; q++) Bm[q * 3 + q] += 1.0;
      if (!cyc) {
        if (m == 0) {   /* Neumann ghost for p, T; wall face u_0 fixed */
          for (int row = 0; row < 2; row++) { Bm[row * 3] += Am[row * 3]; Bm[row * 3 + 1] += Am[row * 3 + 1]; }
          memset(Am, 0, 9 * sizeof(double));
        }
        if (m == n - 1) {   /* Neumann ghost for p, T; wall face u_n fixed */
          for (int row = 0; row < 2; row++) { Bm[row * 3] += Cm[row * 3]; Bm[row * 3 + 1] += Cm[row * 3 + 1]; }
          memset(Cm, 0, 9 * sizeof(double));
          Bm[0 * 3 + 2] = 0; Bm[1 * 3 + 2] = 0;
          Am[2 * 3 + 2] = 0; Bm[2 * 3 + 0] = 0; Bm[2 * 3 + 1] = 0; Bm[2 * 3 + 2] = 1.0;
        }
      }
    }
  } else {
    int cc = trans_comp(d, kind);
    for (int m = 0; m < n; m++) {
      int i, j, k;
      /* (a,b) index the unknown's own location: for cc's face direction they
         are face indices, which line_centre passes through unchanged */
      line_centre(d, a, b, m, &i, &j, &k);
      double w[3];
      w_scal(G, P, c, cc, d, i, j, k, w);
      A[m] = h * w[0]; B[m] = 1.0 + h * w[1]; C[m] = h * w[2];
    }
    if (!cyc) {   /* tangential Dirichlet ghost: delta_ghost = -delta_in */
      B[0] -= A[0]; A[0] = 0;
      B[n - 1] -= C[n - 1]; C[n - 1] = 0;
    }
  }
  return n;
}

/* number of lines of a given kind along d, and validity of (a,b) */
static void line_extent(const Grid* G, int d, int kind, int* a0, int* a1, int* b0, int* b1) {
  int nr = G->nr, nt = G->nt, np = G->np;
  int kf0 = G->per ? 0 : 1;   /* interior phi faces start */
  if (kind == 0) {
    if (d == 0) { *a0 = 0; *a1 = nt; *b0 = 0; *b1 = np; }
    else if (d == 1) { *a0 = 0; *a1 = nr; *b0 = 0; *b1 = np; }
    else { *a0 = 0; *a1 = nr; *b0 = 0; *b1 = nt; }
    return;
  }
  int cc = trans_comp(d, kind);
  if (d == 0) {   /* (j,k) */
    if (cc == 1) { *a0 = 1; *a1 = nt; *b0 = 0; *b1 = np; }
    else { *a0 = 0; *a1 = nt; *b0 = kf0; *b1 = np; }
  } else if (d == 1) {   /* (i,k) */
    if (cc == 0) { *a0 = 1; *a1 = nr; *b0 = 0; *b1 = np; }
    else { *a0 = 0; *a1 = nr; *b0 = kf0; *b1 = np; }
  } else {   /* (i,j) */
    if (cc == 0) { *a0 = 1; *a1 = nr; *b0 = 0; *b1 = nt; }
    else { *a0 = 0; *a1 = nr; *b0 = 1; *b1 = nt; }
  }
}

/* -------------------------------------------------------------- driver */

static size_t comp_index(const Grid* G, int cc, int i, int j, int k) {
  return cc == 0 ? IR(G, i, j, k) : cc == 1 ? IT(G, i, j, k) : IP(G, i, j, k);
}

/* solve (I + tau/2 D_d) x = rhs on every line of direction d */
static int sweep_c(const Grid* G, const og_par* P, const Coef* c, double tau, int d,
                   const double* const* rhs, double* const* x) {
  int cyc = (d == 2 && G->per);
  int n = line_len(G, d);
  int err = 0;
  for (int f = 0; f < 5; f++) memset(x[f], 0, field_size(G, f) * sizeof(double));
  for (int kind = 0; kind < 3; kind++) {
    int a0, a1, b0, b1;
    line_extent(G, d, kind, &a0, &a1, &b0, &b1);
#pragma omp parallel for collapse(2) reduction(| : err)
    for (int a = a0; a < a1; a++)
      for (int b = b0; b < b1; b++) {
        int w = kind == 0 ? 9 : 1, v = kind == 0 ? 3 : 1;
        double* A = malloc(sizeof(double) * w * n);
        double* B = malloc(sizeof(double) * w * n);
        double* C = malloc(sizeof(double) * w * n);
        double* dd = malloc(sizeof(double) * v * n);
        double* xx = malloc(sizeof(double) * v * n);
        assemble(G, P, c, d, kind, a, b, tau, A, B, C);
        if (kind == 0) {
          for (int m = 0; m < n; m++) {
            int i, j, k;
            line_centre(d, a, b, m, &i, &j, &k);
            dd[3 * m] = rhs[0][IC(G, i, j, k)];
            dd[3 * m + 1] = rhs[4][IC(G, i, j, k)];
            double uu = 0;
            if (m < n - 1 || cyc) {
              if (d == 0) uu = rhs[1][IR(G, m + 1, j, k)];
              else if (d == 1) uu = rhs[2][IT(G, i, m + 1, k)];
              else uu = rhs[3][IP(G, i, j, (m + 1) % n)];
            }
            dd[3 * m + 2] = uu;
          }
          int e = cyc ? og_block_cyclic(n, A, B, C, dd, xx) : og_block_thomas(n, A, B, C, dd, xx);
          if (e) err |= 1;
          for (int m = 0; m < n; m++) {
            int i, j, k;
            line_centre(d, a, b, m, &i, &j, &k);
            x[0][IC(G, i, j, k)] = xx[3 * m];
            x[4][IC(G, i, j, k)] = xx[3 * m + 1];
            if (m < n - 1 || cyc) {
              if (d == 0) x[1][IR(G, m + 1, j, k)] = xx[3 * m + 2];
              else if (d == 1) x[2][IT(G, i, m + 1, k)] = xx[3 * m + 2];
              else x[3][IP(G, i, j, (m + 1) % n)] = xx[3 * m + 2];
            }
          }
        } else {
          int cc = trans_comp(d, kind);
          for (int m = 0; m < n; m++) {
            int i, j, k;
            line_centre(d, a, b, m, &i, &j, &k);
            dd[m] = rhs[1 + cc][comp_index(G, cc, i, j, k)];
          }
          int e = cyc ? og_cyclic_thomas(n, A, B, C, dd, xx) : og_thomas(n, A, B, C, dd, xx);
          if (e) err |= 1;
          for (int m = 0; m < n; m++) {
            int i, j, k;
            line_centre(d, a, b, m, &i, &j, &k);
            x[1 + cc][comp_index(G, cc, i, j, k)] = xx[m];
          }
        }
        free(A); free(B); free(C); free(dd); free(xx);
      }
  }
  return err ? -2 : 0;
}

/* owned 5-field buffer */
typedef struct { double* f[5]; } Buf;
static void buf_alloc(const Grid* G, Buf* b) { for (int f = 0; f < 5; f++) b->f[f] = calloc(field_size(G, f), sizeof(double)); }
static void buf_free(Buf* b) { for (int f = 0; f < 5; f++) free(b->f[f]); }

/* wall sets combined: out = a*wa + b*wb (NULL entries count as zero) */
typedef struct { double* w[18]; } Walls;
static void walls_comb(const Grid* G, const double* const* wa, double a, const double* const* wb, double b, Walls* o) {
  for (int q = 0; q < 18; q++) {
    const double* x = wa ? wa[q] : NULL;
    const double* y = wb ? wb[q] : NULL;
    o->w[q] = NULL;
    if (!x && !y) continue;
    int c = q / 6, d = (q / 2) % 3;
    size_t n = wall_size(G, c, d);
    o->w[q] = malloc(n * sizeof(double));
    for (size_t t = 0; t < n; t++) o->w[q][t] = (x ? a * x[t] : 0.0) + (y ? b * y[t] : 0.0);
  }
}
static void walls_free(Walls* o) { for (int q = 0; q < 18; q++) free(o->w[q]); }

static void make_ubar(const Grid* G, const double* const* Un, const double* const* Uk, Buf* ub) {
  for (int f = 0; f < 5; f++) {
    size_t n = field_size(G, f);
    for (size_t t = 0; t < n; t++) ub->f[f][t] = 0.5 * (Un[f][t] + Uk[f][t]);
  }
}

/* mask of unknown locations: the normal velocity on wall faces is data */
static int is_unknown(const Grid* G, int f, size_t t) {
  if (f == 0 || f == 4) return 1;
  size_t np = G->np, nt = G->nt;
  if (f == 1) { size_t i = t / (nt * np); return i > 0 && i < (size_t)G->nr; }
  if (f == 2) { size_t j = (t / np) % (nt + 1); return j > 0 && j < nt; }
  if (G->per) return 1;
  { size_t k = t % (size_t)G->npf; return k > 0 && k < (size_t)G->np; }
}

/* RHS of eq. (spl1), in the paper's order:
   R = -(I + tau/2 D)(U^k - U^n) - tau D U^n - tau G - tau/2 D_M U^k - tau/2 D_M U^n + tau S */
static void rhs_c(const Grid* G, const og_par* P, const Coef* c, const double* bgp, const double* bgT,
                  const double* const* Un, const double* const* wn, const double* const* Uk,
                  const double* const* wk, double tau, const double* const* S, double* const* R) {
  Buf dU, t1, t2, t3, t4;
  buf_alloc(G, &dU); buf_alloc(G, &t1); buf_alloc(G, &t2); buf_alloc(G, &t3); buf_alloc(G, &t4);
  for (int f = 0; f < 5; f++) {
    size_t n = field_size(G, f);
    for (size_t t = 0; t < n; t++) dU.f[f][t] = Uk[f][t] - Un[f][t];
  }
  Walls wd;
  walls_comb(G, wk, 1.0, wn, -1.0, &wd);
  Op od, on, ok;
  op_set(&od, (const double* const*)dU.f, NULL, NULL, (const double* const*)wd.w);
  op_set(&on, Un, bgp, bgT, wn);
  op_set(&ok, Uk, bgp, bgT, wk);
  /* t1 = D (U^k - U^n), t2 = D U^n, t3 = D_M U^k, t4 = D_M U^n */
  for (int d = 0; d < 3; d++) {
    apply_dir(G, P, c, d, &od, t1.f);
    apply_dir(G, P, c, d, &on, t2.f);
  }
  apply_M(G, P, c, &ok, t3.f);
  apply_M(G, P, c, &on, t4.f);
  for (int f = 0; f < 5; f++) {
    size_t n = field_size(G, f);
    for (size_t t = 0; t < n; t++) {
      if (!is_unknown(G, f, t)) { R[f][t] = 0.0; continue; }
      double v = -(dU.f[f][t] + 0.5 * tau * t1.f[f][t]) - tau * t2.f[f][t]
               - 0.5 * tau * t3.f[f][t] - 0.5 * tau * t4.f[f][t];
      if (f == 1) v -= tau * P->g;   /* G = [0, g, 0, 0, 0], g along e_r */
      if (S && S[f]) v += tau * S[f][t];
      R[f][t] = v;
    }
  }
  walls_free(&wd);
  buf_free(&dU); buf_free(&t1); buf_free(&t2); buf_free(&t3); buf_free(&t4);
}

/* ------------------------------------------------------------ exported */

int og_apply(const og_grid* g, const og_par* par, const double* const* Ubar, const double* bgp,
             const double* bgT, const double* const* ubw, int which, const double* const* V,
             const double* vbgp, const double* vbgT, const double* const* vw, double* const* out) {
  Grid G;
  if (grid_init(&G, g) || which < 0 || which > 3) return -1;
  Op ub, v;
  op_set(&ub, Ubar, bgp, bgT, ubw);
  op_set(&v, V, vbgp, vbgT, vw);
  Coef c;
  coef_make(&G, par, &ub, &c);
  zero_fields(&G, out);
  if (which < 3) apply_dir(&G, par, &c, which, &v, out);
  else apply_M(&G, par, &c, &v, out);
  coef_free(&c);
  grid_free(&G);
  return 0;
}

int og_line_system(const og_grid* g, const og_par* par, const double* const* Ubar, const double* bgp,
                   const double* bgT, const double* const* ubw, int dir, int kind, int a, int b,
                   double tau, double* A, double* B, double* C) {
  Grid G;
  if (grid_init(&G, g) || dir < 0 || dir > 2 || kind < 0 || kind > 2) return -1;
  int a0, a1, b0, b1;
  line_extent(&G, dir, kind, &a0, &a1, &b0, &b1);
  if (a < a0 || a >= a1 || b < b0 || b >= b1) { grid_free(&G); return -1; }
  Op ub;
  op_set(&ub, Ubar, bgp, bgT, ubw);
  Coef c;
  coef_make(&G, par, &ub, &c);
  int n = assemble(&G, par, &c, dir, kind, a, b, tau, A, B, C);
  coef_free(&c);
  grid_free(&G);
  return n;
}

int og_rhs(const og_grid* g, const og_par* par, const double* bgp, const double* bgT,
           const double* const* Un, const double* const* wn, const double* const* Uk,
           const double* const* wk, double tau, const double* const* S, double* const* R) {
  Grid G;
  if (grid_init(&G, g) || !(tau > 0)) return -1;
  Buf ub; buf_alloc(&G, &ub);
  make_ubar(&G, Un, Uk, &ub);
  Walls wb; walls_comb(&G, wn, 0.5, wk, 0.5, &wb);
  Op o; op_set(&o, (const double* const*)ub.f, bgp, bgT, (const double* const*)wb.w);
  Coef c; coef_make(&G, par, &o, &c);
  rhs_c(&G, par, &c, bgp, bgT, Un, wn, Uk, wk, tau, S, R);
  coef_free(&c); walls_free(&wb); buf_free(&ub); grid_free(&G);
  return 0;
}

int og_sweep(const og_grid* g, const og_par* par, const double* bgp, const double* bgT,
             const double* const* Un, const double* const* wn, const double* const* Uk,
             const double* const* wk, double tau, int dir, const double* const* rhs, double* const* x) {
  Grid G;
  if (grid_init(&G, g) || !(tau > 0) || dir < 0 || dir > 2) return -1;
  Buf ub; buf_alloc(&G, &ub);
  make_ubar(&G, Un, Uk, &ub);
  Walls wb; walls_comb(&G, wn, 0.5, wk, 0.5, &wb);
  Op o; op_set(&o, (const double* const*)ub.f, bgp, bgT, (const double* const*)wb.w);
  Coef c; coef_make(&G, par, &o, &c);
  int e = sweep_c(&G, par, &c, tau, dir, rhs, x);
  coef_free(&c); walls_free(&wb); buf_free(&ub); grid_free(&G);
  return e;
}

int og_step(const og_grid* g, const og_par* par, const double* bgp, const double* bgT,
            double* const* U, const double* const* wn, const double* const* wnp1,
            double tau, int K, const double* const* S, double* resid) {
  Grid G;
  if (grid_init(&G, g) || !(tau > 0) || K < 1) return -1;
  const double* const* wk = wnp1 ? wnp1 : wn;
  Buf un, uk, ub, R, x1, x2, x3;
  buf_alloc(&G, &un); buf_alloc(&G, &uk); buf_alloc(&G, &ub);
  buf_alloc(&G, &R); buf_alloc(&G, &x1); buf_alloc(&G, &x2); buf_alloc(&G, &x3);
  for (int f = 0; f < 5; f++) {
    memcpy(un.f[f], U[f], field_size(&G, f) * sizeof(double));
    memcpy(uk.f[f], U[f], field_size(&G, f) * sizeof(double));
  }
  /* U^{n+1,0} = U^n, with the normal wall velocity of t^{n+1} */
  if (wk) {
    int nr = G.nr, nt = G.nt, np = G.np;
    for (int s = 0; s < 2; s++) {
      const double* a = wk[(0 * 3 + 0) * 2 + s];
      if (a) for (int j = 0; j < nt; j++) for (int k = 0; k < np; k++) uk.f[1][IR(&G, s ? nr : 0, j, k)] = a[j * np + k];
      const double* b = wk[(1 * 3 + 1) * 2 + s];
      if (b) for (int i = 0; i < nr; i++) for (int k = 0; k < np; k++) uk.f[2][IT(&G, i, s ? nt : 0, k)] = b[i * np + k];
      const double* c = wk[(2 * 3 + 2) * 2 + s];
      if (c && !G.per) for (int i = 0; i < nr; i++) for (int j = 0; j < nt; j++) uk.f[3][IP(&G, i, j, s ? np : 0)] = c[i * nt + j];
    }
  }
  Walls wb; walls_comb(&G, wn, 0.5, wk, 0.5, &wb);
  int e = 0;
  for (int it = 0; it < K && !e; it++) {
    make_ubar(&G, (const double* const*)un.f, (const double* const*)uk.f, &ub);
    Op o; op_set(&o, (const double* const*)ub.f, bgp, bgT, (const double* const*)wb.w);
    Coef c; coef_make(&G, par, &o, &c);
    rhs_c(&G, par, &c, bgp, bgT, (const double* const*)un.f, wn, (const double* const*)uk.f, wk, tau, S, R.f);
    e = sweep_c(&G, par, &c, tau, 0, (const double* const*)R.f, x1.f);
    if (!e) e = sweep_c(&G, par, &c, tau, 1, (const double* const*)x1.f, x2.f);
    if (!e) e = sweep_c(&G, par, &c, tau, 2, (const double* const*)x2.f, x3.f);
    coef_free(&c);
    for (int f = 0; f < 5 && !e; f++) {
      size_t n = field_size(&G, f);
      double ss = 0; size_t cnt = 0;
      for (size_t t = 0; t < n; t++) {
        if (!is_unknown(&G, f, t)) continue;
        uk.f[f][t] += x3.f[f][t];
        ss += x3.f[f][t] * x3.f[f][t]; cnt++;
      }
      if (resid) resid[f] = cnt ? sqrt(ss / cnt) : 0.0;
    }
  }
  if (!e)
    for (int f = 0; f < 5; f++) memcpy(U[f], uk.f[f], field_size(&G, f) * sizeof(double));
  walls_free(&wb);
  buf_free(&un); buf_free(&uk); buf_free(&ub); buf_free(&R); buf_free(&x1); buf_free(&x2); buf_free(&x3);
  grid_free(&G);
  return e;
}
