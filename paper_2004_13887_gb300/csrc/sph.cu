// sph.cu -- GB300 (sm_103a) kernels and C ABI for the direction-splitting scheme of
// Frolov, Minev & Takhirov (arXiv 2004.13887): Picard-iterated Crank-Nicolson with
// Douglas factorisation and splitting-error reduction (Section 2.2, eqs.
// chapter3mainsd, splitting2, spl1-spl3), MAC grid in spherical coordinates,
// operators of Appendix B.
//
// One iteration k -> k+1 is six stages:
//   avg   : Ubar = (U^n + U^{n+1,k})/2 in the bulk type, and D = U^k - U^n
//   coef  : per-centre coefficients frozen at Ubar (p+pi_inf, T, rho, rho-rho_ref,
//           beta, centre velocities, grad u with metric terms, the three parts
//           of div Ubar)
//   rhs   : R = -(U^k - U^n) - tau [N(Ubar) + G - S]  (the right-hand side of
//           eq. spl1 after the linearity of D(Ubar) is used: the D(U^k - U^n),
//           D U^n and D_M terms collapse to the full operator at Ubar); four
//           launches: centre rows (p, T) and the three momentum rows
//   sweep : r, theta, phi line solves (I + tau/2 D_d) x = rhs (eqs. spl1-spl3):
//           3x3-block systems for (p, T, u_d), scalar ones for the two
//           transverse velocities, cyclic along a periodic phi.  FP64 mode: one
//           thread per line (block Thomas, Woodbury / Sherman-Morrison on cyclic
//           lines).  Mixed mode: the partitioned solver of sph_lines.cuh (lanes
//           of a warp per line, chunk elimination + parallel cyclic reduction),
//           one launch for the block lines and one for both transverse kinds.
//           The phi sweep also applies U^{k+1} = U^k + x and accumulates the
//           increment norm.
//
// Precision: everything is templated on the bulk type R.  R = double is the
// plain FP64 scheme.  R = float ("mixed") keeps U^n, U^{n+1,k} and their update
// in FP64 and everything per iteration in FP32: Ubar and D are formed from the
// FP64 state as hi + lo pairs on the FP32 pipe, div(Ubar) -- which multiplies
// gamma (p + pi_inf) and nearly cancels at low Mach number -- is carried as a
// pair, the hydrostatic part of the r-momentum row goes through density
// perturbations, and the cyclic corrections of the Thomas path combine in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sph.h"
#include "sph_device.cuh"

using namespace sph;

#include "sph_kernels.cuh"

#include "sph_adjoint.cuh"
#include "sph_lines.cuh"

// ============================================================== host side

#include "sph_host.cuh"

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
    case SPH_ERR_TAPE: return "adjoint: a thread's tape was too short for its rows";
    default: return "unknown error";
  }
}

extern "C" int sph_set_line_solver(sph_ctx* ctx, int which) {
  if (!ctx || (which != SPH_LINES_THOMAS && which != SPH_LINES_PARTITIONED && which != SPH_LINES_PARTITIONED_WARP &&
               which != SPH_LINES_PARTITIONED_NARROW))
    return SPH_ERR_ARG;
  ctx->line_solver = which;
  return SPH_OK;
}

extern "C" int sph_set_tile(sph_ctx* ctx, int tj, int ti) {
  if (!ctx || tj < 1 || ti < 1 || tj * ti > 8 || (tj & (tj - 1)) || (ti & (ti - 1))) return SPH_ERR_ARG;
  ctx->tile_j = tj;
  ctx->tile_i = ti;
  return SPH_OK;
}

extern "C" long long sph_launch_count(const sph_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int sph_bounds_report(int* first) {
#ifdef SPH_CHECKED
  int h[5] = {0, 0, 0, 0, 0}, z[5] = {0, 0, 0, 0, 0}, hb[5] = {0, 0, 0, 0, 0};
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpyFromSymbol(h, g_bounds, sizeof h) != cudaSuccess ||
      cudaMemcpyToSymbol(g_bounds, z, sizeof z) != cudaSuccess || bounds_take_batch(hb) != SPH_OK)
    return SPH_ERR_CUDA;
  if (h[0] == 0)
    for (int q = 1; q < 5; q++) h[q] = hb[q];
  h[0] += hb[0];
  if (first)
    for (int q = 0; q < 4; q++) first[q] = h[1 + q];
  return h[0];
#else
  if (first)
    for (int q = 0; q < 4; q++) first[q] = 0;
  return -1;
#endif
}

static void prof_free(sph_ctx* c) {
  for (int q = 0; q < c->evcap * 2; q++) cudaEventDestroy(c->ev[q]);
  free(c->ev); free(c->evkind);
  c->ev = NULL; c->evkind = NULL; c->evcap = 0; c->nev = 0;
}

template <typename R>
static void bufs_free(Bufs<R>& b) {
  cudaFree(b.metric); cudaFree(b.bgder); cudaFree(b.mdf); cudaFree(b.coef); cudaFree(b.scr);
  for (int f = 0; f < 5; f++) {
    cudaFree(b.Ub[f]); cudaFree(b.UbLo[f]); cudaFree(b.Db[f]); cudaFree(b.Rb[f]); cudaFree(b.X1[f]);
  }
}

static void free_all(sph_ctx* c) {
  prof_free(c);
  for (int q = 0; q < 3; q++) {
    if (c->aux[q]) cudaStreamDestroy(c->aux[q]);
    if (c->ejoin[q]) cudaEventDestroy(c->ejoin[q]);
  }
  if (c->efork) cudaEventDestroy(c->efork);
  bufs_free(c->d64);
  bufs_free(c->d32);
  cudaFree(c->bg); cudaFree(c->acc); cudaFree(c->flag); cudaFree(c->rows64);
  cudaFree(c->wmean64); cudaFree(c->wmean32); cudaFree(c->wnext);
  cudaFree(c->wzero64); cudaFree(c->wzero32);
  cudaFree(c->adjS); cudaFree(c->adjW); cudaFree(c->adjC);
  cudaFree(c->tape_d); cudaFree(c->tape_ix); cudaFree(c->tape_li); cudaFree(c->tape_adj); cudaFree(c->adj_info);
  for (int f = 0; f < 5; f++) { cudaFree(c->U[0][f]); cudaFree(c->U[1][f]); cudaFree(c->src[f]); }
  free(c->hmet);
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

// metric tables: 4 (nr+1) radial + 8 (nt+1) polar values
static void fill_metric(const sph_grid* gr, double* h, int nr, int nt, double dr, double dth) {
  double* rc = h; double* rf = rc + (nr + 1); double* irc = rf + (nr + 1); double* irf = irc + (nr + 1);
  double* sc = irf + (nr + 1); double* sf = sc + (nt + 1); double* isc = sf + (nt + 1); double* isf = isc + (nt + 1);
  double* cc = isf + (nt + 1); double* cf = cc + (nt + 1); double* cotc = cf + (nt + 1); double* cotf = cotc + (nt + 1);
  for (int i = 0; i < nr; i++) { rc[i] = gr->r1 + (i + 0.5) * dr; irc[i] = 1.0 / rc[i]; }
  for (int i = 0; i <= nr; i++) { rf[i] = gr->r1 + i * dr; irf[i] = 1.0 / rf[i]; }
  for (int j = 0; j < nt; j++) {
    double t = gr->th1 + (j + 0.5) * dth;
    sc[j] = sin(t); cc[j] = cos(t); isc[j] = 1.0 / sc[j]; cotc[j] = cc[j] / sc[j];
  }
  for (int j = 0; j <= nt; j++) {
    double t = gr->th1 + j * dth;
    sf[j] = sin(t); cf[j] = cos(t);
  }
  if (fabs(gr->th1) < 1e-14) sf[0] = 0.0;
  if (fabs(gr->th2 - M_PI) < 1e-14) sf[nt] = 0.0;
  for (int j = 0; j <= nt; j++) { isf[j] = sf[j] != 0.0 ? 1.0 / sf[j] : 0.0; cotf[j] = sf[j] != 0.0 ? cf[j] / sf[j] : 0.0; }
}

template <typename R>
static void set_geo_ptrs(Bufs<R>& b, const Geo<double>& base, const double* bg, int nr, int nt) {
  Geo<R>& g = b.g;
  g.nr = base.nr; g.nt = base.nt; g.np = base.np; g.npf = base.npf; g.per = base.per;
  g.dr = (R)base.dr; g.dth = (R)base.dth; g.dph = (R)base.dph;
  g.idr = (R)base.idr; g.idth = (R)base.idth; g.idph = (R)base.idph;
  R* m = b.metric;
  g.rc = m; g.rf = m + (nr + 1); g.irc = m + 2 * (nr + 1); g.irf = m + 3 * (nr + 1);
  R* tb = m + 4 * (nr + 1);
  g.sc = tb; g.sf = tb + (nt + 1); g.isc = tb + 2 * (nt + 1); g.isf = tb + 3 * (nt + 1);
  g.cc = tb + 4 * (nt + 1); g.cf = tb + 5 * (nt + 1); g.cotc = tb + 6 * (nt + 1); g.cotf = tb + 7 * (nt + 1);
  g.bgp = bg; g.bgT = bg + (nr + 2);
  g.dbgp = b.bgder; g.dbgT = b.bgder + nr; g.lapT = b.bgder + 2 * nr; g.rhoref = b.bgder + 3 * nr;
  g.ehyd = b.bgder + 4 * nr;
  g.pcen = b.bgder + 5 * nr + 1; g.Tcen = b.bgder + 6 * nr + 1;
  g.rf2h = b.mdf; g.rf2l = b.mdf + (nr + 1); g.sfh = b.mdf + 2 * (nr + 1); g.sfl = b.mdf + 2 * (nr + 1) + (nt + 1);
}

template <typename R>
static int bufs_alloc(Bufs<R>& b, size_t nmet, int nr, const size_t* nf, long N, size_t nscr, int bulk) {
#define ALLOC(p, n) do { if (!cuda_ok(cudaMalloc((void**)&(p), (size_t)(n) * sizeof(R)))) return SPH_ERR_NOMEM; } while (0)
  ALLOC(b.metric, nmet);
  ALLOC(b.bgder, 7 * (size_t)nr + 1);
  ALLOC(b.mdf, nmet);
  if (!bulk) return SPH_OK;
  for (int f = 0; f < 5; f++) { ALLOC(b.Ub[f], nf[f]); ALLOC(b.Db[f], nf[f]); ALLOC(b.Rb[f], nf[f]); ALLOC(b.X1[f], nf[f]); }
  if (sizeof(R) == sizeof(float))
    for (int f = 1; f < 4; f++) ALLOC(b.UbLo[f], nf[f]);
  ALLOC(b.coef, (size_t)NCOEF * N);
  ALLOC(b.scr, nscr);
#undef ALLOC
  R* q = b.coef;
  Coef<R>& cf = b.c;
  cf.Pb = q; cf.Tb = q + N; cf.rho = q + 2 * N; cf.drho = q + 3 * N; cf.beta = q + 4 * N; cf.uc0 = q + 5 * N;
  cf.uc1 = q + 6 * N; cf.uc2 = q + 7 * N; cf.grr = q + 8 * N; cf.gtt = q + 9 * N; cf.gpp = q + 10 * N;
  cf.srt = q + 11 * N; cf.srp = q + 12 * N; cf.stp = q + 13 * N;
  cf.dvr = q + 14 * N; cf.dvt = q + 15 * N; cf.dvp = q + 16 * N;
  return SPH_OK;
}

template <typename R>
static int upload_tables(sph_ctx* c, Bufs<R>& b, const double* hmet, const double* hder, int nr) {
  size_t nd = 7 * (size_t)nr + 1;
  R* tm = (R*)malloc(c->nmet * sizeof(R));
  R* td = (R*)malloc(nd * sizeof(R));
  if (!tm || !td) { free(tm); free(td); return SPH_ERR_NOMEM; }
  for (size_t q = 0; q < c->nmet; q++) tm[q] = (R)hmet[q];
  for (size_t q = 0; q < nd; q++) td[q] = (R)hder[q];
  int e = SPH_OK;
  if (!cuda_ok(cudaMemcpy(b.metric, tm, c->nmet * sizeof(R), cudaMemcpyHostToDevice)) ||
      !cuda_ok(cudaMemcpy(b.bgder, td, nd * sizeof(R), cudaMemcpyHostToDevice)))
    e = SPH_ERR_CUDA;
  // rf^2 and sin(theta_f) as hi + lo pairs (tm has room: nmet > 2 (nr+1) + 2 (nt+1))
  int nt = c->d64.g.nt;
  const double* rf = hmet + (nr + 1);
  const double* sf = hmet + 4 * (nr + 1) + (nt + 1);
  R* rh = tm; R* rl = tm + (nr + 1); R* sh = tm + 2 * (nr + 1); R* sl = sh + (nt + 1);
  for (int i = 0; i <= nr; i++) { double v = rf[i] * rf[i]; rh[i] = (R)v; rl[i] = (R)(v - (double)rh[i]); }
  for (int j = 0; j <= nt; j++) { double v = sf[j]; sh[j] = (R)v; sl[j] = (R)(v - (double)sh[j]); }
  size_t nm = 2 * (size_t)(nr + 1) + 2 * (size_t)(nt + 1);
  if (e == SPH_OK && !cuda_ok(cudaMemcpy(b.mdf, tm, nm * sizeof(R), cudaMemcpyHostToDevice))) e = SPH_ERR_CUDA;
  free(tm); free(td);
  return e;
}

// Background-derived tables (FP64 on the host, then in each bulk type).
static int upload_background(sph_ctx* c, const double* pref, const double* Tref) {
  const Geo<double>& g = c->d64.g;
  int nr = g.nr;
  const double* rc = c->hmet;
  const double* rf = rc + (nr + 1);
  double* der = (double*)calloc(7 * (size_t)nr + 1, sizeof(double));
  if (!der) return SPH_ERR_NOMEM;
  double* dbgp = der; double* dbgT = der + nr; double* lapT = der + 2 * nr; double* rhoref = der + 3 * nr;
  double* ehyd = der + 4 * nr;
  double* pcen = der + 5 * nr + 1; double* Tcen = der + 6 * nr + 1;
  double Rg = c->P.Rg, pinf = c->P.pinf;
  for (int i = 0; i < nr; i++) {
    // index i+1 of the tables is centre i; 0 and nr+1 are the ghosts
    dbgp[i] = pref[i + 2] - pref[i];
    dbgT[i] = Tref[i + 2] - Tref[i];
    double f0 = rf[i] * rf[i], f1 = rf[i + 1] * rf[i + 1];
    lapT[i] = (f1 * (Tref[i + 2] - Tref[i + 1]) - f0 * (Tref[i + 1] - Tref[i])) / (rc[i] * rc[i] * g.dr * g.dr);
    rhoref[i] = Tref[i + 1] != 0.0 ? (pref[i + 1] + pinf) / (Rg * Tref[i + 1]) : 0.0;
    pcen[i] = pref[i + 1] + pinf;
    Tcen[i] = Tref[i + 1];
  }
  for (int i = 1; i < nr; i++) {
    double rf_ = 0.5 * (rhoref[i - 1] + rhoref[i]);
    ehyd[i] = rf_ != 0.0 ? (pref[i + 1] - pref[i]) / (g.dr * rf_) + c->P.g : c->P.g;
  }
  int e = upload_tables(c, c->d64, c->hmet, der, nr);
  if (e == SPH_OK && c->prec == SPH_PREC_MIXED) e = upload_tables(c, c->d32, c->hmet, der, nr);
  free(der);
  return e;
}

// elements of wall array (component c, wall normal to d)
static size_t wall_count(const Geo<double>& g, int c, int d) {
  size_t nr = g.nr, nt = g.nt, np = g.np, npf = g.npf;
  if (c == 0) return d == 1 ? (nr + 1) * np : d == 2 ? (nr + 1) * nt : nt * np;
  if (c == 1) return d == 0 ? (nt + 1) * np : d == 2 ? nr * (nt + 1) : nr * np;
  return d == 0 ? nt * npf : d == 1 ? nr * npf : nr * nt;
}

static int lines_prepare(const sph_ctx* c);
static size_t lines_scratch(int nr, int nt, int np, int per);

extern "C" int sph_create(const sph_grid* gr, const sph_params* pa, void* stream, sph_ctx** out) {
  if (!gr || !pa || !out) return SPH_ERR_ARG;
  *out = NULL;
  if (gr->nr < 2 || gr->nth < 2 || gr->nph < 2) return SPH_ERR_ARG;
  if (!(gr->r1 > 0) || !(gr->r2 > gr->r1) || !(gr->th2 > gr->th1) || !(gr->ph2 > gr->ph1)) return SPH_ERR_ARG;
  if (gr->th1 < 0 || gr->th2 > M_PI + 1e-12) return SPH_ERR_ARG;
  if (gr->periodic_phi && gr->nph < 3) return SPH_ERR_ARG;
  if (!(pa->gamma > 1) || !(pa->cv > 0) || !(pa->Pr > 0) || pa->mu < 0) return SPH_ERR_ARG;
  if (pa->precision != SPH_PREC_FP64 && pa->precision != SPH_PREC_MIXED) return SPH_ERR_ARG;
  sph_ctx* c = (sph_ctx*)calloc(1, sizeof(sph_ctx));
  if (!c) return SPH_ERR_NOMEM;
  cudaGetDevice(&c->dev);
  if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess || c->nsm < 1) c->nsm = 1;
  c->st = (cudaStream_t)stream;
  c->prec = pa->precision;
  c->line_solver = SPH_LINES_PARTITIONED;
  c->tile_j = c->tile_i = 1;
  Geo<double> g;
  memset(&g, 0, sizeof g);
  g.nr = gr->nr; g.nt = gr->nth; g.np = gr->nph; g.per = gr->periodic_phi ? 1 : 0;
  g.npf = g.per ? g.np : g.np + 1;
  g.dr = (gr->r2 - gr->r1) / g.nr; g.dth = (gr->th2 - gr->th1) / g.nt; g.dph = (gr->ph2 - gr->ph1) / g.np;
  g.idr = 1.0 / g.dr; g.idth = 1.0 / g.dth; g.idph = 1.0 / g.dph;
  Par& P = c->P;
  P.gamma = pa->gamma; P.cv = pa->cv; P.Pr = pa->Pr; P.mu = pa->mu; P.pinf = pa->pi_inf; P.g = pa->g;
  P.omega = pa->omega;
  P.kappa = pa->mu * pa->gamma * pa->cv / pa->Pr;
  P.Rg = pa->cv * (pa->gamma - 1.0);
  P.gamma_f = (float)P.gamma; P.mu_f = (float)P.mu; P.kappa_f = (float)P.kappa; P.g_f = (float)P.g;
  P.omega_f = (float)P.omega; P.iRg_f = (float)(1.0 / P.Rg);
  c->N = (long)g.nr * g.nt * g.np;
  for (int f = 0; f < 5; f++) c->nf[f] = sph_field_size(gr, f);
  c->unknowns[0] = c->unknowns[4] = c->N;
  c->unknowns[1] = (long)(g.nr - 1) * g.nt * g.np;
  c->unknowns[2] = (long)g.nr * (g.nt - 1) * g.np;
  c->unknowns[3] = (long)g.nr * g.nt * (g.per ? g.np : g.np - 1);

  int nr = g.nr, nt = g.nt;
  c->nmet = 4 * (size_t)(nr + 1) + 8 * (size_t)(nt + 1);
  c->hmet = (double*)calloc(c->nmet, sizeof(double));
  if (!c->hmet) { free(c); return SPH_ERR_NOMEM; }
  fill_metric(gr, c->hmet, nr, nt, g.dr, g.dth);
  const double* scs = c->hmet + 4 * (nr + 1);
  for (int j = 0; j < nt; j++)
    if (!(scs[j] > 0)) { free(c->hmet); free(c); return SPH_ERR_ARG; }

  size_t wblk = g.per ? 21 : 12;
  size_t nscr = (wblk + 6) * (size_t)c->N + 64;
  // the partitioned solver's factor slots (up to 18.4 floats per cell, more
  // where the lines of a launch's last group do not fill it)
  if (c->prec == SPH_PREC_MIXED) {
    size_t need = lines_scratch(g.nr, g.nt, g.np, g.per) + 64;
    if (nscr < need) nscr = need;
  }
  // kernels index with 32-bit ints: every array, and the scratch, must fit
  if (nscr >= (size_t)2147483647 || c->nf[1] >= (size_t)2147483647 || c->nf[3] >= (size_t)2147483647) {
    free(c->hmet); free(c); return SPH_ERR_ARG;
  }
  int mixed = c->prec == SPH_PREC_MIXED;
  c->nscr = nscr;
  int err = bufs_alloc(c->d64, c->nmet, nr, c->nf, c->N, nscr, !mixed);
  if (err == SPH_OK && mixed) err = bufs_alloc(c->d32, c->nmet, nr, c->nf, c->N, nscr, 1);
  for (int f = 0; f < 5 && err == SPH_OK; f++) {
    if (!cuda_ok(cudaMalloc((void**)&c->U[0][f], c->nf[f] * sizeof(double))) ||
        !cuda_ok(cudaMalloc((void**)&c->U[1][f], c->nf[f] * sizeof(double))) ||
        !cuda_ok(cudaMalloc((void**)&c->src[f], c->nf[f] * sizeof(double))))
      err = SPH_ERR_NOMEM;
  }
  if (err == SPH_OK && (!cuda_ok(cudaMalloc((void**)&c->bg, 2 * (size_t)(nr + 2) * sizeof(double))) ||
                        !cuda_ok(cudaMalloc((void**)&c->acc, 8 * sizeof(double))) ||
                        !cuda_ok(cudaMalloc((void**)&c->flag, sizeof(int)))))
    err = SPH_ERR_NOMEM;
  if (err == SPH_OK && !mixed) {
    // the line rows of the FP64 mode: 12 planes over the centres per direction,
    // 5 + 6 over the faces of each kind
    size_t nrows = 36 * (size_t)c->N + 11 * (c->nf[1] + c->nf[2] + c->nf[3]);
    if (!cuda_ok(cudaMalloc((void**)&c->rows64, nrows * sizeof(double)))) {
      err = SPH_ERR_NOMEM;
    } else {
      double* p = c->rows64;
      c->rows.nc = c->N;
      for (int d = 0; d < 3; d++) { c->rows.c[d] = p; p += 12 * (size_t)c->N; }
      for (int d = 0; d < 3; d++) {
        c->rows.nf[d] = (long)c->nf[1 + d];
        c->rows.f[d] = p; p += 5 * c->nf[1 + d];
        c->rows.s[d] = p; p += 6 * c->nf[1 + d];
      }
    }
  }
  if (err != SPH_OK) { cudaGetLastError(); free_all(c); free(c); return err; }
  if (!cuda_ok(cudaMemset(c->bg, 0, 2 * (size_t)(nr + 2) * sizeof(double))) || !cuda_ok(cudaMemset(c->flag, 0, sizeof(int))))
    err = SPH_ERR_CUDA;
  for (int f = 0; f < 5 && err == SPH_OK; f++)
    if (!cuda_ok(cudaMemset(c->U[0][f], 0, c->nf[f] * sizeof(double))) ||
        !cuda_ok(cudaMemset(c->U[1][f], 0, c->nf[f] * sizeof(double))))
      err = SPH_ERR_CUDA;
  if (err != SPH_OK) { free_all(c); free(c); return err; }
  set_geo_ptrs(c->d64, g, c->bg, nr, nt);
  if (mixed) set_geo_ptrs(c->d32, g, c->bg, nr, nt);
  {
    // homogeneous walls: every wall array is the zero buffer
    size_t wmax = 0;
    for (int cc = 0; cc < 3; cc++)
      for (int d = 0; d < 3; d++) {
        size_t w = wall_count(g, cc, d);
        if (w > wmax) wmax = w;
      }
    if (cudaMalloc((void**)&c->wzero64, wmax * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&c->wzero32, wmax * sizeof(float)) != cudaSuccess)
      err = SPH_ERR_NOMEM;
    else if (cudaMemset(c->wzero64, 0, wmax * sizeof(double)) != cudaSuccess ||
             cudaMemset(c->wzero32, 0, wmax * sizeof(float)) != cudaSuccess)
      err = SPH_ERR_CUDA;
    for (int q = 0; q < 18; q++) { c->d64.g.w[q] = c->wzero64; c->d32.g.w[q] = c->wzero32; }
    if (err) { cudaGetLastError(); free_all(c); free(c); return err; }
  }
  // zero background
  double* zb = (double*)calloc(nr + 2, sizeof(double));
  double* tb = (double*)calloc(nr + 2, sizeof(double));
  err = (zb && tb) ? upload_background(c, zb, tb) : SPH_ERR_NOMEM;
  free(zb); free(tb);
  if (err != SPH_OK) { free_all(c); free(c); return err; }
  if (mixed && (err = lines_prepare(c)) != SPH_OK) { free_all(c); free(c); return err; }
  if (cudaEventCreateWithFlags(&c->efork, cudaEventDisableTiming) != cudaSuccess) err = SPH_ERR_CUDA;
  for (int q = 0; q < 3 && !err; q++)
    if (cudaStreamCreateWithFlags(&c->aux[q], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ejoin[q], cudaEventDisableTiming) != cudaSuccess)
      err = SPH_ERR_CUDA;
  if (err) { free_all(c); free(c); return err; }
  c->cur = 0;
  *out = c;
  return SPH_OK;
}

extern "C" int sph_set_background(sph_ctx* c, const double* p_ref, const double* T_ref) {
  if (!c) return SPH_ERR_ARG;
  size_t n = c->d64.g.nr + 2;
  double* hp_ = (double*)calloc(n, sizeof(double));
  double* hT = (double*)calloc(n, sizeof(double));
  if (!hp_ || !hT) { free(hp_); free(hT); return SPH_ERR_NOMEM; }
  if (p_ref) memcpy(hp_, p_ref, n * sizeof(double));
  if (T_ref) memcpy(hT, T_ref, n * sizeof(double));
  int e = SPH_OK;
  if (cudaStreamSynchronize(c->st) != cudaSuccess ||
      cudaMemcpy(c->bg, hp_, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->bg + n, hT, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    e = SPH_ERR_CUDA;
  if (e == SPH_OK) e = upload_background(c, hp_, hT);
  free(hp_); free(hT);
  return e;
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

extern "C" int sph_set_bc(sph_ctx* c, const double* const* wn, const double* const* wnp1, int on_device) {
  if (!c) return SPH_ERR_ARG;
  const Geo<double>& g = c->d64.g;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_ERR_CUDA;  // steps in flight read the old data
  int any = 0;
  size_t tot = 0;
  for (int q = 0; q < 18; q++) {
    int cc = q / 6, d = (q / 2) % 3;
    int given = (wn && wn[q]) || (wnp1 && wnp1[q]);
    if (d == 2 && g.per) given = 0;  // no phi walls on a periodic line
    c->wset[q] = given;
    c->woff[q] = tot;
    if (given) { tot += wall_count(g, cc, d); any = 1; }
  }
  for (int q = 0; q < 18; q++) { c->d64.g.w[q] = c->wzero64; c->d32.g.w[q] = c->wzero32; }
  c->d64.g.hasw = c->d32.g.hasw = 0;
  c->hasbc = 0;
  cudaFree(c->wmean64); cudaFree(c->wmean32); cudaFree(c->wnext);
  c->wmean64 = NULL; c->wmean32 = NULL; c->wnext = NULL;
  c->wtot = tot;
  if (!any) return SPH_OK;
  double* hm = (double*)calloc(tot, sizeof(double));
  double* hn = (double*)calloc(tot, sizeof(double));
  float* hf = (float*)calloc(tot, sizeof(float));
  double* tmp = (double*)malloc(tot * sizeof(double));
  int e = (hm && hn && hf && tmp) ? SPH_OK : SPH_ERR_NOMEM;
  for (int q = 0; q < 18 && !e; q++) {
    if (!c->wset[q]) continue;
    size_t n = wall_count(g, q / 6, (q / 2) % 3), o = c->woff[q];
    for (int lev = 0; lev < 2 && !e; lev++) {
      const double* src = lev == 0 ? (wn ? wn[q] : NULL) : (wnp1 ? wnp1[q] : NULL);
      if (!src) continue;
      if (on_device) {
        if (cudaMemcpy(tmp, src, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) { e = SPH_ERR_CUDA; break; }
        src = tmp;
      }
      for (size_t t = 0; t < n; t++) {
        hm[o + t] += 0.5 * src[t];
        if (lev == 1) hn[o + t] = src[t];
      }
    }
    for (size_t t = 0; t < n; t++) hf[o + t] = (float)hm[o + t];
  }
  if (!e && (cudaMalloc((void**)&c->wmean64, tot * sizeof(double)) != cudaSuccess ||
             cudaMalloc((void**)&c->wnext, tot * sizeof(double)) != cudaSuccess ||
             (c->prec == SPH_PREC_MIXED && cudaMalloc((void**)&c->wmean32, tot * sizeof(float)) != cudaSuccess)))
    e = SPH_ERR_NOMEM;
  if (!e && (cudaMemcpy(c->wmean64, hm, tot * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(c->wnext, hn, tot * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
             (c->wmean32 && cudaMemcpy(c->wmean32, hf, tot * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)))
    e = SPH_ERR_CUDA;
  free(hm); free(hn); free(hf); free(tmp);
  if (e) { cudaGetLastError(); return e; }
  for (int q = 0; q < 18; q++) {
    if (!c->wset[q]) continue;
    c->d64.g.w[q] = c->wmean64 + c->woff[q];
    if (c->wmean32) c->d32.g.w[q] = c->wmean32 + c->woff[q];
  }
  c->d64.g.hasw = 1;
  c->d32.g.hasw = c->wmean32 ? 1 : 0;
  c->hasbc = 1;
  return SPH_OK;
}

// U^{n+1,0} = U^n with the t^{n+1} normal velocity on the wall faces (wall
// data set by sph_set_bc; the c == d arrays), in the iterate buffer
static int bc_first_iterate(sph_ctx* c) {
  const Geo<double>& g = c->d64.g;
  double** un = c->U[c->cur];
  double** uk = c->U[1 - c->cur];
  for (int f = 0; f < 5; f++)
    if (cudaMemcpyAsync(uk[f], un[f], c->nf[f] * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      return SPH_ERR_CUDA;
  size_t nr = g.nr, nt = g.nt, np = g.np, npf = g.npf, D = sizeof(double);
  for (int s = 0; s < 2; s++) {
    int q;
    if (c->wset[q = (0 * 3 + 0) * 2 + s] &&   // u_r on the r-faces 0 / nr: one contiguous plane
        cudaMemcpyAsync(uk[1] + (s ? nr : 0) * nt * np, c->wnext + c->woff[q], nt * np * D, cudaMemcpyDeviceToDevice,
                        c->st) != cudaSuccess)
      return SPH_ERR_CUDA;
    if (c->wset[q = (1 * 3 + 1) * 2 + s] &&   // u_theta on the theta-faces 0 / nt: np values per r index
        cudaMemcpy2DAsync(uk[2] + (s ? nt : 0) * np, (nt + 1) * np * D, c->wnext + c->woff[q], np * D, np * D, nr,
                          cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      return SPH_ERR_CUDA;
    if (!g.per && c->wset[q = (2 * 3 + 2) * 2 + s] &&   // u_phi on the phi-faces 0 / np: one value per line
        cudaMemcpy2DAsync(uk[3] + (s ? np : 0), npf * D, c->wnext + c->woff[q], D, D, nr * nt,
                          cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      return SPH_ERR_CUDA;
  }
  return SPH_OK;
}

template <typename R> static CF<R> cf_of(R* const* p) { CF<R> r; for (int f = 0; f < 5; f++) r.f[f] = p[f]; return r; }
template <typename R> static MF<R> mf_of(R* const* p) { MF<R> r; for (int f = 0; f < 5; f++) r.f[f] = p[f]; return r; }

// bracket a launch: start event before, stop event after (when timing is on).
// Each stage's launches are also an NVTX range on the host thread (named
// "sph <stage>"), so a profiler's timeline and its NVTX filters show the
// stages; without a tool attached the calls return at once.
static const char* const kStageName[SPH_NKERNELS] = {"sph avg", "sph coef", "sph rhs", "sph sweep r",
                                                     "sph sweep theta", "sph sweep phi", "sph other", "sph other"};

static void k_begin(sph_ctx* c, int kind) {
  c->cur_kind = kind;
  c->kcount[kind]++;
  if (c->nvtx_open) nvtxRangePop();
  nvtxRangePushA(kStageName[kind]);
  c->nvtx_open = 1;
  if (c->prof && c->nev < c->evcap) cudaEventRecord(c->ev[2 * c->nev], c->st);
}

static int launch_ok(sph_ctx* c) {
  if (c->nvtx_open) {
    nvtxRangePop();
    c->nvtx_open = 0;
  }
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

static int grid_stride_blocks(long n) {
  long b = (n + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

// Ubar into the bulk buffer (FP64 mode at k = 0: U^n itself); coefficients
template <typename R>
static int prepare(sph_ctx* c, Bufs<R>& b, int have_iter, CF<R>* ub_out, double* const* ukp = nullptr) {
  double** un = c->U[c->cur];
  double* const* uk = have_iter ? (ukp ? ukp : c->U[1 - c->cur]) : un;
  CF<R> ub;
  if (sizeof(R) == sizeof(double) && !have_iter) {
    for (int f = 0; f < 5; f++) ub.f[f] = (const R*)un[f];
  } else {
    AvgArgs<R> A;
    A.same = !have_iter;
    long mx = 0;
    for (int f = 0; f < 5; f++) {
      A.a[f] = un[f]; A.b[f] = uk[f]; A.o[f] = b.Ub[f]; A.lo[f] = b.UbLo[f]; A.d[f] = b.Db[f];
      A.n[f] = (long)c->nf[f];
      if (A.n[f] > mx) mx = A.n[f];
    }
    k_begin(c, SPH_K_AVG);
    k_avg<R><<<dim3(grid_stride_blocks((mx + 1) / 2) / 4 + 1, 5), 256, 0, c->st>>>(A);
    if (launch_ok(c)) return SPH_ERR_CUDA;
    ub = cf_of(b.Ub);
  }
  k_begin(c, SPH_K_COEF);
  const Geo<double>& gg = c->d64.g;
  if (b.g.hasw) k_coef<R, true><<<tile_grid(gg.np, gg.nt, gg.nr), TILE_BLOCK, 0, c->st>>>(b.g, c->P, ub, b.c);
  else k_coef<R, false><<<tile_grid(gg.np, gg.nt, gg.nr), TILE_BLOCK, 0, c->st>>>(b.g, c->P, ub, b.c);
  if (launch_ok(c)) return SPH_ERR_CUDA;
  *ub_out = ub;
  return SPH_OK;
}

// Independent launches of one stage run side by side: `fork` makes n side
// streams wait for the work enqueued so far on the context's stream, `join`
// makes the context's stream wait for them (both are stream-ordered, so a
// CUDA graph capture follows them).
static int fork_aux(sph_ctx* c, int n) {
  if (cudaEventRecord(c->efork, c->st) != cudaSuccess) return SPH_ERR_CUDA;
  for (int q = 0; q < n; q++)
    if (cudaStreamWaitEvent(c->aux[q], c->efork, 0) != cudaSuccess) return SPH_ERR_CUDA;
  return SPH_OK;
}
static int join_aux(sph_ctx* c, int n) {
  for (int q = 0; q < n; q++)
    if (cudaEventRecord(c->ejoin[q], c->aux[q]) != cudaSuccess || cudaStreamWaitEvent(c->st, c->ejoin[q], 0) != cudaSuccess)
      return SPH_ERR_CUDA;
  return SPH_OK;
}

// The right-hand side stage: centre rows on the context's stream, the
// momentum rows of the three components on side streams, concurrently (timed
// as one stage).
template <typename R>
static int run_rhs(sph_ctx* c, Bufs<R>& b, CF<R> ub, CF<double> uk, int hasD, double tau, CF<double> src, int has_src,
                   MF<R> Rout) {
  CF<double> un = cf_of(c->U[c->cur]);
  CF<R> Dv = cf_of(b.Db);  // U^k - U^n from the averaging stage (zero, and not read, when hasD = 0)
  CF<R> ul = sizeof(R) == sizeof(float) ? cf_of(b.UbLo) : ub;  // velocity remainders of Ubar (FP32 mode)
  R tr = (R)tau;
  // FP64 mode: the kernels also store the line rows the sweeps read
  Rows64 rows = c->rows;
  if (sizeof(R) != sizeof(double)) memset(&rows, 0, sizeof rows);
  k_begin(c, SPH_K_RHS);
  if (fork_aux(c, 3)) return SPH_ERR_CUDA;
  const Geo<double>& gg = c->d64.g;
  int nr = gg.nr, nt = gg.nt, np = gg.np, npf = gg.npf;
  if (b.g.hasw) {
    k_rhs_c<R, true><<<tile_grid(np, nt, nr), TILE_BLOCK, 0, c->st>>>(b.g, c->d64.g, c->P, b.c, ub, ul, un, uk, Dv,
                                                                      hasD, src, has_src, tr, Rout, rows);
    k_rhs_u<R, 0, true><<<tile_grid(np, nt, nr + 1), TILE_BLOCK, 0, c->aux[0]>>>(b.g, c->P, b.c, ub, Dv, hasD, src,
                                                                                 has_src, tr, Rout, rows);
    k_rhs_u<R, 1, true><<<tile_grid(np, nt + 1, nr), TILE_BLOCK, 0, c->aux[1]>>>(b.g, c->P, b.c, ub, Dv, hasD, src,
                                                                                 has_src, tr, Rout, rows);
    k_rhs_u<R, 2, true><<<tile_grid(npf, nt, nr), TILE_BLOCK, 0, c->aux[2]>>>(b.g, c->P, b.c, ub, Dv, hasD, src,
                                                                              has_src, tr, Rout, rows);
  } else {
    k_rhs_c<R, false><<<tile_grid(np, nt, nr), TILE_BLOCK, 0, c->st>>>(b.g, c->d64.g, c->P, b.c, ub, ul, un, uk, Dv,
                                                                       hasD, src, has_src, tr, Rout, rows);
    k_rhs_u<R, 0, false><<<tile_grid(np, nt, nr + 1), TILE_BLOCK, 0, c->aux[0]>>>(b.g, c->P, b.c, ub, Dv, hasD, src,
                                                                                  has_src, tr, Rout, rows);
    k_rhs_u<R, 1, false><<<tile_grid(np, nt + 1, nr), TILE_BLOCK, 0, c->aux[1]>>>(b.g, c->P, b.c, ub, Dv, hasD, src,
                                                                                  has_src, tr, Rout, rows);
    k_rhs_u<R, 2, false><<<tile_grid(npf, nt, nr), TILE_BLOCK, 0, c->aux[2]>>>(b.g, c->P, b.c, ub, Dv, hasD, src,
                                                                               has_src, tr, Rout, rows);
  }
  if (join_aux(c, 3)) return SPH_ERR_CUDA;
  c->launches += 3;  // launch_ok counts the fourth
  return launch_ok(c);
}


// Partitioned line solver (mixed path) for lines of n = L P cells, L lanes
// per line: one launch per line kind, one block per group of CB/n lines.
// The shared-memory size attributes of the kernels of a (D, P, L, CB), set
// once per process (at context creation, so that no attribute call falls
// inside a CUDA graph capture).
template <int D, int P, int L, int CB>
static int lines_attr() {
  static unsigned long long done = 0;  // one bit per device (attributes are per device)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (done & bit) return SPH_OK;
  const int smb = lines::NFB * lines::Shape<P, L, CB>::FS * (int)sizeof(float);
  const int sms = lines::NFS * lines::Shape<P, L, CB>::FS * (int)sizeof(float);
  if (cudaFuncSetAttribute(lines::k_lines_blk<D, P, L, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb) !=
          cudaSuccess ||
      cudaFuncSetAttribute(lines::k_lines_sca<D, P, L, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, sms) !=
          cudaSuccess)
    return SPH_ERR_CUDA;
  done |= bit;
  return SPH_OK;
}



// floats of factor slots the partitioned solver needs on a grid: the largest
// over the directions it takes and the lane counts (16, 32) it may use there
static size_t lines_scratch(int nr, int nt, int np, int per) {
  Geo<double> g;
  memset(&g, 0, sizeof g);
  g.nr = nr; g.nt = nt; g.np = np; g.per = per;
  size_t mx = 0;
  for (int d = 0; d < 3; d++) {
    int n = d == 0 ? nr : d == 1 ? nt : np;
    if (n != 16 && n != 32 && n != 48 && n != 64 && n != 128 && n != 192 && n != 256 &&
        !(d == 2 && (n == 512 || n == 1024)))
      continue;
    SweepArgs<float> S;
    memset(&S, 0, sizeof S);
    line_layout(g, d, S);
    for (int L = 4; L <= 128; L *= 2) {
      // the lane counts run_lines_d may take for n: 16 (or the narrow 4 for
      // 16 cells, 8 for 32 and 48) up to 48 cells; 8 (narrow), 16 and 32 for
      // 64; 16 and 32 for 128; 32 for 192 and 256; n / 8 beyond
      const int narrow = n == 16 ? 4 : n <= 64 ? 8 : 0;
      if (n <= 48 ? (L != 16 && L != narrow) : n == 64 ? (L < 8 || L > 32) : n <= 128 ? (L < 16 || L > 32)
                  : L != (n <= 256 ? 32 : n / 8))
        continue;
      int P = n / L, CB = lines_cb(d, n), NW = CB / n, NWW = CB / P / 32;
      size_t need = (size_t)lines_groups(S, 0, NW) * NWW * 32 * lines::slot_floats(P);
      if (need > mx) mx = need;
    }
  }
  return mx;
}


template <int D, int P, int L>
static int run_lines(sph_ctx* c, SweepArgs<float>& S) {
  constexpr int CB = lines_cb(D, L * P);
  using SH = lines::Shape<P, L, CB>;
  constexpr int NW = SH::NW, NT = SH::NT;
  const size_t smb = (size_t)lines::NFB * SH::FS * sizeof(float);
  const size_t sms = (size_t)lines::NFS * SH::FS * sizeof(float);
  int ng, e;
  k_begin(c, SPH_K_SWEEP_R + D);
  if ((e = lines_attr<D, P, L, CB>())) return e;
  if ((e = fork_aux(c, 1))) return e;
  if ((ng = lines_groups(S, 0, NW)) > 0) {
    // one factor slot per warp
    if ((size_t)ng * SH::NWW * 32 * lines::slot_floats(P) > c->nscr) return SPH_ERR_ARG;
    lines::k_lines_blk<D, P, L, CB><<<ng, NT, smb, c->st>>>(S);
    c->launches++;
  }
  const int ng1 = lines_groups(S, 1, NW), ng2 = lines_groups(S, 2, NW);
  if (ng1 + ng2 > 0) {
    lines::k_lines_sca<D, P, L, CB><<<ng1 + ng2, NT, sms, c->aux[0]>>>(S, ng1);
    c->launches++;
  }
  if ((e = join_aux(c, 1))) return e;
  c->launches--;  // launch_ok counts one more
  return launch_ok(c);
}

template <int D>
static int lines_attr_d(int n) {
  int e = SPH_OK;
  if (n == 16 && !(e = lines_attr<D, 1, 16, lines_cb(D, 16)>())) e = lines_attr<D, 4, 4, lines_cb(D, 16)>();
  if (n == 32 && !(e = lines_attr<D, 2, 16, lines_cb(D, 32)>())) e = lines_attr<D, 4, 8, lines_cb(D, 32)>();
  if (n == 48 && !(e = lines_attr<D, 3, 16, lines_cb(D, 48)>())) e = lines_attr<D, 6, 8, lines_cb(D, 48)>();
  if (n == 192) e = lines_attr<D, 6, 32, lines_cb(D, 192)>();
  if (n == 64 && !(e = lines_attr<D, 2, 32, lines_cb(D, 64)>()) && !(e = lines_attr<D, 4, 16, lines_cb(D, 64)>()))
    e = lines_attr<D, 8, 8, lines_cb(D, 64)>();
  if (n == 128 && !(e = lines_attr<D, 4, 32, lines_cb(D, 128)>())) e = lines_attr<D, 8, 16, lines_cb(D, 128)>();
  if (n == 256) e = lines_attr<D, 8, 32, lines_cb(D, 256)>();
  if constexpr (D == 2) {
    if (n == 512) e = lines_attr<D, 8, 64, lines_cb(D, 512)>();
    if (n == 1024) e = lines_attr<D, 8, 128, lines_cb(D, 1024)>();
  }
  return e;
}

static int lines_prepare(const sph_ctx* c) {
  const Geo<double>& g = c->d64.g;
  int e = lines_attr_d<0>(g.nr);
  if (!e) e = lines_attr_d<1>(g.nt);
  if (!e) e = lines_attr_d<2>(g.np);
  return e;
}

// the layout lines_pl picks for the context's line solver
template <int D>
static int run_lines_d(sph_ctx* c, SweepArgs<float>& S, int n) {
  int P = 0, L = 0;
  lines_pl(c->line_solver, D, n, &P, &L);
#define SPH_RUN_PL(p, l) \
  if (P == p && L == l) return run_lines<D, p, l>(c, S);
  SPH_LINES_EACH_PL(SPH_RUN_PL)
#undef SPH_RUN_PL
  if constexpr (D == 2) {
    if (P == 8 && L == 64) return run_lines<D, 8, 64>(c, S);
    if (P == 8 && L == 128) return run_lines<D, 8, 128>(c, S);
  }
  return SPH_ERR_ARG;
}

// Threads per block of the one-thread-per-line sweeps (k_sweep).  In FP64 mode
// a block line costs several times a scalar line and the FP64 pipe is the
// bound: warp-sized blocks spread the block lines evenly over the SMs
// (measured, 128 x 256 x 256 FP64 step: 64.9 ms at 128 threads a block, 62.6
// at 64, 60.1 at 32; theta and phi sweeps 13.7 and 15.9 -> 11.7 and 13.2 ms).
#ifndef SPH_SWEEP64_BLOCK
#define SPH_SWEEP64_BLOCK 32
#endif
template <typename R>
static constexpr int sweep_block() { return sizeof(R) == sizeof(double) ? SPH_SWEEP64_BLOCK : 128; }

template <typename R>
static int run_sweep(sph_ctx* c, Bufs<R>& b, int d, double tau, CF<R> ub, CF<R> rhs, MF<R> x, int update,
                     CF<double> base, MF<double> uk, int rows_ready = 0) {
  SweepArgs<R> S;
  memset(&S, 0, sizeof S);
  S.g = b.g; S.P = c->P; S.c = b.c; S.ub = ub; S.d = d; S.h = (R)(0.5 * tau);
  S.rhs = rhs; S.x = x; S.update = update; S.base = base; S.uk = uk;
  S.scr = b.scr; S.acc = c->acc; S.flag = c->flag;
  S.rows = c->rows;
  line_layout(c->d64.g, d, S);
  if (sizeof(R) == sizeof(float) && c->line_solver != SPH_LINES_THOMAS && lines_ok(c, d)) {
    SweepArgs<float>& Sf = *reinterpret_cast<SweepArgs<float>*>(&S);
    const Geo<double>& g = c->d64.g;
    int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
    if (d == 0) return run_lines_d<0>(c, Sf, n);
    if (d == 1) return run_lines_d<1>(c, Sf, n);
    return run_lines_d<2>(c, Sf, n);
  }
  int mx = S.nl[0];
  if (S.nl[1] > mx) mx = S.nl[1];
  if (S.nl[2] > mx) mx = S.nl[2];
  constexpr int TB = sweep_block<R>();
  if constexpr (sizeof(R) == sizeof(double)) {
    if (c->line_solver != SPH_LINES_THOMAS && !(d == 2 && c->d64.g.per)) {
      // walled lines in the FP64 mode: two threads per line, eliminating from both ends
      static_assert(TB % 32 == 0, "k_sweep2 takes whole warps");
      constexpr int LPB = TB / 2;
      dim3 grid2((unsigned)((mx + LPB - 1) / LPB), 3);
      k_begin(c, SPH_K_SWEEP_R + d);
      // rows_ready: the right-hand side of this iteration has just stored the
      // line rows (steps); a sweep on its own (sph_sweep) forms them
      if (rows_ready && c->rows64) {
        if (d == 0) k_sweep2<R, 0, true><<<grid2, TB, 0, c->st>>>(S);
        else if (d == 1) k_sweep2<R, 1, true><<<grid2, TB, 0, c->st>>>(S);
        else k_sweep2<R, 2, true><<<grid2, TB, 0, c->st>>>(S);
      } else {
        if (d == 0) k_sweep2<R, 0, false><<<grid2, TB, 0, c->st>>>(S);
        else if (d == 1) k_sweep2<R, 1, false><<<grid2, TB, 0, c->st>>>(S);
        else k_sweep2<R, 2, false><<<grid2, TB, 0, c->st>>>(S);
      }
      return launch_ok(c);
    }
  }
  dim3 grid((unsigned)((mx + TB - 1) / TB), 3);
  k_begin(c, SPH_K_SWEEP_R + d);
  if (d == 0) k_sweep<R, 0><<<grid, TB, 0, c->st>>>(S);
  else if (d == 1) k_sweep<R, 1><<<grid, TB, 0, c->st>>>(S);
  else k_sweep<R, 2><<<grid, TB, 0, c->st>>>(S);
  return launch_ok(c);
}

static int read_flag(sph_ctx* c, int* flag) {
  if (cudaMemcpyAsync(flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess) return SPH_ERR_CUDA;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_ERR_CUDA;
  return SPH_OK;
}

static int stage_source(sph_ctx* c, const double* const* source, int on_device, CF<double>* out) {
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

template <typename R>
static int convert_out(sph_ctx* c, R* const* in, double* const* out) {
  for (int f = 0; f < 5; f++) {
    long n = (long)c->nf[f];
    k_cvt<R><<<grid_stride_blocks(n), 256, 0, c->st>>>(n, in[f], out[f]);
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
  }
  return SPH_OK;
}

template <typename R>
static int convert_in(sph_ctx* c, const double* const* in, R* const* out) {
  for (int f = 0; f < 5; f++) {
    long n = (long)c->nf[f];
    k_cvt_in<R><<<grid_stride_blocks(n), 256, 0, c->st>>>(n, in[f], out[f]);
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
  }
  return SPH_OK;
}

template <typename R>
static int rhs_impl(sph_ctx* c, Bufs<R>& b, double dt, CF<double> src, int has, double* const* R_out) {
  CF<R> ub;
  int e = prepare(c, b, c->iterate_set, &ub);
  if (e) return e;
  CF<double> uk = cf_of(c->iterate_set ? c->U[1 - c->cur] : c->U[c->cur]);
  if (sizeof(R) == sizeof(double)) return run_rhs(c, b, ub, uk, c->iterate_set, dt, src, has, mf_of((R* const*)R_out));
  e = run_rhs(c, b, ub, uk, c->iterate_set, dt, src, has, mf_of(b.Rb));
  if (e) return e;
  return convert_out(c, b.Rb, R_out);
}

extern "C" int sph_rhs(sph_ctx* c, double dt, const double* const* source, int on_device, double* const* R_out) {
  if (!c || !R_out || !(dt > 0)) return SPH_ERR_ARG;
  CF<double> src;
  int has = stage_source(c, source, on_device, &src);
  if (has < 0) return SPH_ERR_CUDA;
  if (c->prec == SPH_PREC_MIXED) return rhs_impl(c, c->d32, dt, src, has, R_out);
  return rhs_impl(c, c->d64, dt, src, has, R_out);
}

template <typename R>
static int sweep_impl(sph_ctx* c, Bufs<R>& b, int dir, double dt, const double* const* rhs, double* const* x) {
  CF<R> ub;
  int e = prepare(c, b, c->iterate_set, &ub);
  if (e) return e;
  if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->st) != cudaSuccess) return SPH_ERR_CUDA;
  CF<double> base = cf_of(c->U[c->cur]);
  MF<double> ukm = mf_of(c->U[1 - c->cur]);
  if (sizeof(R) == sizeof(double)) {
    e = run_sweep(c, b, dir, dt, ub, cf_of((R* const*)rhs), mf_of((R* const*)x), 0, base, ukm);
  } else {
    e = convert_in(c, rhs, b.Rb);
    if (!e) e = run_sweep(c, b, dir, dt, ub, cf_of(b.Rb), mf_of(b.X1), 0, base, ukm);
    if (!e) e = convert_out(c, b.X1, x);
  }
  if (e) return e;
  int flag = 0;
  if ((e = read_flag(c, &flag))) return e;
  return (flag & FLAG_SINGULAR) ? SPH_ERR_SINGULAR : SPH_OK;
}

extern "C" int sph_sweep(sph_ctx* c, int dir, double dt, const double* const* rhs, double* const* x) {
  if (!c || !rhs || !x || dir < 0 || dir > 2 || !(dt > 0)) return SPH_ERR_ARG;
  if (c->prec == SPH_PREC_MIXED) return sweep_impl(c, c->d32, dir, dt, rhs, x);
  return sweep_impl(c, c->d64, dir, dt, rhs, x);
}

template <typename R>
static int step_impl(sph_ctx* c, Bufs<R>& b, double dt, int n_iter, CF<double> src, int has) {
  double** un = c->U[c->cur];
  double** uk = c->U[1 - c->cur];
  int e = SPH_OK;
  // with wall data, U^{n+1,0} differs from U^n on the normal wall faces: it is
  // formed in the iterate buffer and every iteration reads it from there
  const int first = c->hasbc ? 1 : 0;
  nvtxRangePushA("sph step");
  if (first) e = bc_first_iterate(c);
  for (int it = 0; it < n_iter && !e; it++) {
    CF<R> ub;
    const int iter = it > 0 || first;
    e = prepare(c, b, iter, &ub);
    if (e) break;
    CF<double> ukin = cf_of(iter ? uk : un);
    e = run_rhs(c, b, ub, ukin, iter, dt, src, has, mf_of(b.Rb));
    if (!e) e = run_sweep(c, b, 0, dt, ub, cf_of(b.Rb), mf_of(b.X1), 0, ukin, mf_of(uk), 1);
    if (!e) e = run_sweep(c, b, 1, dt, ub, cf_of(b.X1), mf_of(b.Rb), 0, ukin, mf_of(uk), 1);
    if (!e && it == n_iter - 1 && cudaMemsetAsync(c->acc, 0, 5 * sizeof(double), c->st) != cudaSuccess) e = SPH_ERR_CUDA;
    if (!e) e = run_sweep(c, b, 2, dt, ub, cf_of(b.Rb), mf_of(b.X1), 1, ukin, mf_of(uk), 1);
  }
  if (c->nvtx_open) {  // a stage that failed before its launch check
    nvtxRangePop();
    c->nvtx_open = 0;
  }
  nvtxRangePop();
  return e;
}

// Enqueue one step without waiting for it (no status read): the flags of
// enqueued steps accumulate until sph_status.  Only device sources (or none),
// so that nothing is copied from host memory.
extern "C" int sph_step_async(sph_ctx* c, double dt, int n_iter, const double* const* source, int on_device) {
  if (!c || !(dt > 0) || n_iter < 1 || (source && !on_device)) return SPH_ERR_ARG;
  CF<double> src;
  int has = stage_source(c, source, on_device, &src);
  if (has < 0) return SPH_ERR_CUDA;
  int e = c->prec == SPH_PREC_MIXED ? step_impl(c, c->d32, dt, n_iter, src, has)
                                    : step_impl(c, c->d64, dt, n_iter, src, has);
  if (e) return e;
  c->cur = 1 - c->cur;
  c->iterate_set = 0;
  return SPH_OK;
}

extern "C" int sph_status(sph_ctx* c, double* residual_out) {
  if (!c) return SPH_ERR_ARG;
  int flag = 0, e;
  if ((e = read_flag(c, &flag))) return e;
  if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->st) != cudaSuccess) return SPH_ERR_CUDA;
  if (residual_out) {
    double s[5];
    if (cudaMemcpyAsync(s, c->acc, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
      return SPH_ERR_CUDA;
    for (int f = 0; f < 5; f++) residual_out[f] = c->unknowns[f] > 0 ? sqrt(s[f] / (double)c->unknowns[f]) : 0.0;
  }
  if (flag & FLAG_SINGULAR) return SPH_ERR_SINGULAR;
  if (flag & FLAG_NONFINITE) return SPH_ERR_NONFINITE;
  return SPH_OK;
}

extern "C" int sph_step(sph_ctx* c, double dt, int n_iter, const double* const* source, int on_device,
                        double* residual_out) {
  if (!c || !(dt > 0) || n_iter < 1) return SPH_ERR_ARG;
  CF<double> src;
  int has = stage_source(c, source, on_device, &src);
  if (has < 0) return SPH_ERR_CUDA;
  if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->st) != cudaSuccess) return SPH_ERR_CUDA;
  int e = c->prec == SPH_PREC_MIXED ? step_impl(c, c->d32, dt, n_iter, src, has)
                                    : step_impl(c, c->d64, dt, n_iter, src, has);
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

// ------------------------------------------------------------ adjoint

#define ADJ_TAPE_CAP 512       // nodes per thread's tape (the longest location's rows record 370)
#define ADJ_TAPE_BLOCKS 608    // blocks of 128 threads of the gradient kernels (four per SM: their registers allow it)
#define ADJ_FLAG_TAPE 8

static int adj_alloc(sph_ctx* c, int K) {
  if (c->adjS && c->adjK >= K) return SPH_OK;
  cudaFree(c->adjS);
  c->adjS = NULL;
  c->adjK = 0;
  // every field of a set starts on a 256-byte boundary: the averaging kernel
  // reads the state in 16-byte pairs, and aligned rows keep the loads whole
  size_t fs = 0;
  for (int f = 0; f < 5; f++) { c->foff[f] = fs; fs += (c->nf[f] + 31) / 32 * 32; }
  c->fset = fs;
  if (cudaMalloc((void**)&c->adjS, (size_t)K * fs * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return SPH_ERR_NOMEM; }
  c->adjK = K;
  if (c->adjW) return SPH_OK;
  size_t slots = (size_t)ADJ_TAPE_BLOCKS * 128, cap = ADJ_TAPE_CAP;
  if (cudaMalloc((void**)&c->adjW, 10 * fs * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->adjC, (size_t)NCOEF * c->N * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->tape_d, 2 * cap * slots * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->tape_ix, 2 * cap * slots * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->tape_li, cap * slots * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->tape_adj, cap * slots * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->adj_info, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return SPH_ERR_NOMEM;
  }
  c->tape_cap = (int)cap;
  c->tape_blocks = ADJ_TAPE_BLOCKS;
  return cudaMemset(c->adj_info, 0, sizeof(int)) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

// the 5 fields of set q of a block of sets
static void adj_set(const sph_ctx* c, double* base, int q, double** out) {
  for (int f = 0; f < 5; f++) out[f] = base + (size_t)q * c->fset + c->foff[f];
}

// y += s x over whole 5-field sets
static int adj_axpy(sph_ctx* c, double s, double* x, double* y) {
  long n = (long)c->fset;
  adj::k_axpy<<<grid_stride_blocks(n), 256, 0, c->st>>>(n, s, x, y);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

// the transposed sweep along d: x = P A_d^{-T} P rhs (P: zero on the wall faces)
static int run_sweep_T(sph_ctx* c, int d, double tau, CF<double> ub, CF<double> rhs, MF<double> x) {
  Bufs<double>& b = c->d64;
  SweepArgs<double> S;
  memset(&S, 0, sizeof S);
  S.g = b.g; S.P = c->P; S.c = b.c; S.ub = ub; S.d = d; S.h = 0.5 * tau;
  S.rhs = rhs; S.x = x; S.update = 0;
  S.scr = b.scr; S.acc = c->acc; S.flag = c->flag;
  line_layout(c->d64.g, d, S);
  int mx = S.nl[0];
  if (S.nl[1] > mx) mx = S.nl[1];
  if (S.nl[2] > mx) mx = S.nl[2];
  constexpr int TB = sweep_block<double>();
  dim3 grid((unsigned)((mx + TB - 1) / TB), 3);
  if (d == 0) k_sweep<double, 0, true><<<grid, TB, 0, c->st>>>(S);
  else if (d == 1) k_sweep<double, 1, true><<<grid, TB, 0, c->st>>>(S);
  else k_sweep<double, 2, true><<<grid, TB, 0, c->st>>>(S);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

// the gradient over Ubar of <mu_r, R(Ubar)> - sum_d <mu_d, A_d(Ubar) x_d> into lu
// (5 fields, added to), by the tape kernels of sph_adjoint.cuh
static int adj_gradient(sph_ctx* c, double tau, CF<double> ub, double** mu, double** xs, double** lu) {
  Bufs<double>& b = c->d64;
  adj::AdjArgs A;
  memset(&A, 0, sizeof A);
  A.g = b.g; A.P = c->P; A.c = b.c; A.ub = ub; A.tau = tau;
  for (int d = 0; d < 3; d++) {
    double* m5[5];
    double* x5[5];
    adj_set(c, mu[d], 0, m5);
    adj_set(c, xs[d], 0, x5);
    A.mu[d] = cf_of(m5);
    A.x[d] = cf_of(x5);
  }
  for (int f = 0; f < 5; f++) A.lam[f] = lu[f];
  for (int q = 0; q < NCOEF; q++) A.lam[5 + q] = c->adjC + (size_t)q * c->N;
  A.td = c->tape_d; A.tix = c->tape_ix; A.tli = c->tape_li; A.tadj = c->tape_adj; A.cap = c->tape_cap;
  A.flag = c->flag; A.maxn = c->adj_info;
  if (cudaMemsetAsync(c->adjC, 0, (size_t)NCOEF * c->N * sizeof(double), c->st) != cudaSuccess) return SPH_ERR_CUDA;
  const int nb = c->tape_blocks;
  for (int kind = 0; kind < 4; kind++) adj::k_adj_rhs<<<nb, 128, 0, c->st>>>(A, kind);
  for (int d = 0; d < 3; d++) {
    SweepArgs<double> S;
    memset(&S, 0, sizeof S);
    line_layout(c->d64.g, d, S);
    if (d == 0) {
      adj::k_adj_blk<0><<<nb, 128, 0, c->st>>>(A, S.nl[0], S.nb[0], S.a0[0], S.b0[0]);
      adj::k_adj_sca<0, 1><<<nb, 128, 0, c->st>>>(A, S);
      adj::k_adj_sca<0, 2><<<nb, 128, 0, c->st>>>(A, S);
    } else if (d == 1) {
      adj::k_adj_blk<1><<<nb, 128, 0, c->st>>>(A, S.nl[0], S.nb[0], S.a0[0], S.b0[0]);
      adj::k_adj_sca<1, 1><<<nb, 128, 0, c->st>>>(A, S);
      adj::k_adj_sca<1, 2><<<nb, 128, 0, c->st>>>(A, S);
    } else {
      adj::k_adj_blk<2><<<nb, 128, 0, c->st>>>(A, S.nl[0], S.nb[0], S.a0[0], S.b0[0]);
      adj::k_adj_sca<2, 1><<<nb, 128, 0, c->st>>>(A, S);
      adj::k_adj_sca<2, 2><<<nb, 128, 0, c->st>>>(A, S);
    }
  }
  adj::k_adj_coef<<<nb, 128, 0, c->st>>>(A);
  c->launches += 14;
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

extern "C" int sph_step_adjoint(sph_ctx* c, double dt, int n_iter, const double* const* source,
                                const double* const* lam_out, double* const* lam_in) {
  if (!c || !(dt > 0) || n_iter < 1 || !lam_out || !lam_in) return SPH_ERR_ARG;
  if (c->prec != SPH_PREC_FP64) return SPH_ERR_ARG;
  for (int f = 0; f < 5; f++)
    if (!lam_out[f] || !lam_in[f]) return SPH_ERR_ARG;
  int e = adj_alloc(c, n_iter);
  if (e) return e;
  if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->st) != cudaSuccess) return SPH_ERR_CUDA;
  CF<double> src;
  int has = stage_source(c, source, 1, &src);
  Bufs<double>& b = c->d64;
  double** un = c->U[c->cur];
  const size_t FB = c->fset * sizeof(double);
  double *LN[5], *LB[5], *MU[3][5], *XS[3][5], *LU[5];
  adj_set(c, c->adjW, 0, LN);
  adj_set(c, c->adjW, 1, LB);
  for (int d = 0; d < 3; d++) { adj_set(c, c->adjW, 2 + d, MU[d]); adj_set(c, c->adjW, 5 + d, XS[d]); }
  adj_set(c, c->adjW, 8, LU);
  double* mu_base[3] = {MU[0][0], MU[1][0], MU[2][0]};
  double* x_base[3] = {XS[0][0], XS[1][0], XS[2][0]};
  // forward: the iterates U^{n+1,k}, k < K (U^{n+1,0} = U^n, with the t^{n+1}
  // normal wall velocity when wall data are set)
  double* S0[5];
  adj_set(c, c->adjS, 0, S0);
  for (int f = 0; f < 5 && !e; f++)
    if (cudaMemcpyAsync(S0[f], un[f], c->nf[f] * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      e = SPH_ERR_CUDA;
  if (!e && c->hasbc) {
    // the wall faces of the iterate buffer, written by bc_first_iterate, into S0
    e = bc_first_iterate(c);
    for (int f = 0; f < 5 && !e; f++)
      if (cudaMemcpyAsync(S0[f], c->U[1 - c->cur][f], c->nf[f] * sizeof(double), cudaMemcpyDeviceToDevice, c->st) !=
          cudaSuccess)
        e = SPH_ERR_CUDA;
  }
  const int first = c->hasbc ? 1 : 0;
  for (int k = 0; k + 1 < n_iter && !e; k++) {
    double *Sk[5], *Sn[5];
    adj_set(c, c->adjS, k, Sk);
    adj_set(c, c->adjS, k + 1, Sn);
    const int iter = k > 0 || first;
    CF<double> ub;
    e = prepare(c, b, iter, &ub, Sk);
    if (!e) e = run_rhs(c, b, ub, cf_of(iter ? Sk : un), iter, dt, src, has, mf_of(b.Rb));
    if (!e) e = run_sweep(c, b, 0, dt, ub, cf_of(b.Rb), mf_of(b.X1), 0, cf_of(Sk), mf_of(Sn), 1);
    if (!e) e = run_sweep(c, b, 1, dt, ub, cf_of(b.X1), mf_of(b.Rb), 0, cf_of(Sk), mf_of(Sn), 1);
    if (!e) e = run_sweep(c, b, 2, dt, ub, cf_of(b.Rb), mf_of(Sn), 1, cf_of(Sk), mf_of(Sn), 1);
  }
  // reverse
  if (!e && cudaMemsetAsync(LN[0], 0, FB, c->st) != cudaSuccess) e = SPH_ERR_CUDA;
  for (int f = 0; f < 5 && !e; f++)
    if (cudaMemcpyAsync(LB[f], lam_out[f], c->nf[f] * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      e = SPH_ERR_CUDA;
  for (int k = n_iter - 1; k >= 0 && !e; k--) {
    double* Sk[5];
    adj_set(c, c->adjS, k, Sk);
    const int iter = k > 0 || first;
    CF<double> ub;
    // the iteration's Ubar, coefficients and sweep solutions
    e = prepare(c, b, iter, &ub, Sk);
    if (!e) e = run_rhs(c, b, ub, cf_of(iter ? Sk : un), iter, dt, src, has, mf_of(b.Rb));
    if (!e) e = run_sweep(c, b, 0, dt, ub, cf_of(b.Rb), mf_of(XS[0]), 0, cf_of(Sk), mf_of(Sk), 1);
    if (!e) e = run_sweep(c, b, 1, dt, ub, cf_of(XS[0]), mf_of(XS[1]), 0, cf_of(Sk), mf_of(Sk), 1);
    if (!e) e = run_sweep(c, b, 2, dt, ub, cf_of(XS[1]), mf_of(XS[2]), 0, cf_of(Sk), mf_of(Sk), 1);
    // transposed solves, phi first
    if (!e) e = run_sweep_T(c, 2, dt, ub, cf_of(LB), mf_of(MU[2]));
    if (!e) e = run_sweep_T(c, 1, dt, ub, cf_of(MU[2]), mf_of(MU[1]));
    if (!e) e = run_sweep_T(c, 0, dt, ub, cf_of(MU[1]), mf_of(MU[0]));
    // R = -(b - a) - tau N: dJ/da += mu_r, dJ/db -= mu_r
    if (!e) e = adj_axpy(c, 1.0, MU[0][0], LN[0]);
    if (!e) e = adj_axpy(c, -1.0, MU[0][0], LB[0]);
    // the Ubar dependence, half to each of a and b
    if (!e && cudaMemsetAsync(LU[0], 0, FB, c->st) != cudaSuccess) e = SPH_ERR_CUDA;
    if (!e) e = adj_gradient(c, dt, ub, mu_base, x_base, LU);
    if (!e) e = adj_axpy(c, 0.5, LU[0], LN[0]);
    if (!e) e = adj_axpy(c, 0.5, LU[0], LB[0]);
  }
  if (!e && c->hasbc) {
    // U^{n+1,0}'s normal wall faces were data, not U^n
    const Geo<double>& g = c->d64.g;
    size_t nr = g.nr, nt = g.nt, np = g.np, npf = g.npf, D = sizeof(double);
    for (int s = 0; s < 2 && !e; s++) {
      if (c->wset[(0 * 3 + 0) * 2 + s] &&
          cudaMemsetAsync(LB[1] + (s ? nr : 0) * nt * np, 0, nt * np * D, c->st) != cudaSuccess) e = SPH_ERR_CUDA;
      if (!e && c->wset[(1 * 3 + 1) * 2 + s] &&
          cudaMemset2DAsync(LB[2] + (s ? nt : 0) * np, (nt + 1) * np * D, 0, np * D, nr, c->st) != cudaSuccess)
        e = SPH_ERR_CUDA;
      if (!e && !g.per && c->wset[(2 * 3 + 2) * 2 + s] &&
          cudaMemset2DAsync(LB[3] + (s ? np : 0), npf * D, 0, D, nr * nt, c->st) != cudaSuccess)
        e = SPH_ERR_CUDA;
    }
  }
  if (!e) e = adj_axpy(c, 1.0, LB[0], LN[0]);
  for (int f = 0; f < 5 && !e; f++)
    if (cudaMemcpyAsync(lam_in[f], LN[f], c->nf[f] * sizeof(double), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      e = SPH_ERR_CUDA;
  if (e) return e;
  int flag = 0;
  if ((e = read_flag(c, &flag))) return e;
  if (flag & ADJ_FLAG_TAPE) return SPH_ERR_TAPE;
  if (flag & FLAG_SINGULAR) return SPH_ERR_SINGULAR;
  return SPH_OK;
}

extern "C" int sph_adjoint_tape_use(sph_ctx* c, int* longest, int* capacity) {
  if (!c) return SPH_ERR_ARG;
  int n = 0;
  if (c->adj_info && (cudaStreamSynchronize(c->st) != cudaSuccess ||
                      cudaMemcpy(&n, c->adj_info, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess))
    return SPH_ERR_CUDA;
  if (longest) *longest = n;
  if (capacity) *capacity = c->adj_info ? c->tape_cap : ADJ_TAPE_CAP;
  return SPH_OK;
}

// ------------------------------------------------------------ batches


extern "C" void sph_batch_destroy(sph_batch* b) {
  if (!b) return;
  batch_fused_free(b);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->fork) cudaEventDestroy(b->fork);
  for (int q = 0; q < b->n && b->join; q++)
    if (b->join[q]) cudaEventDestroy(b->join[q]);
  free(b->join);
  free(b->c);
  free(b->cur);
  free(b->nlaunch);
  free(b);
}

extern "C" int sph_batch_create(sph_ctx* const* ctxs, int n, void* stream, sph_batch** out) {
  if (!ctxs || n < 1 || !stream || !out) return SPH_ERR_ARG;
  *out = NULL;
  for (int q = 0; q < n; q++) {
    if (!ctxs[q] || !ctxs[q]->st) return SPH_ERR_ARG;
    for (int r = 0; r < q; r++)
      if (ctxs[r] == ctxs[q]) return SPH_ERR_ARG;
  }
  sph_batch* b = (sph_batch*)calloc(1, sizeof(sph_batch));
  if (!b) return SPH_ERR_NOMEM;
  b->n = n;
  b->st = (cudaStream_t)stream;
  b->c = (sph_ctx**)calloc(n, sizeof(sph_ctx*));
  b->join = (cudaEvent_t*)calloc(n, sizeof(cudaEvent_t));
  b->cur = (int*)calloc(n, sizeof(int));
  b->nlaunch = (long long*)calloc(n, sizeof(long long));
  if (!b->c || !b->join || !b->cur || !b->nlaunch) { sph_batch_destroy(b); return SPH_ERR_NOMEM; }
  int err = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
  for (int q = 0; q < n && !err; q++) {
    b->c[q] = ctxs[q];
    if (cudaEventCreateWithFlags(&b->join[q], cudaEventDisableTiming) != cudaSuccess) err = SPH_ERR_CUDA;
  }
  if (err) { sph_batch_destroy(b); return err; }
  *out = b;
  return SPH_OK;
}

extern "C" int sph_batch_capture(sph_batch* b, double dt, int n_iter, int steps) {
  if (!b || !(dt > 0) || n_iter < 1 || steps < 2 || (steps & 1)) return SPH_ERR_ARG;
  for (int q = 0; q < b->n; q++)
    if (b->c[q]->prof) return SPH_ERR_ARG;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = NULL; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = NULL; }
  for (int q = 0; q < b->n; q++) { b->cur[q] = b->c[q]->cur; b->nlaunch[q] = b->c[q]->launches; }
  if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SPH_ERR_CUDA;
  int err = cudaEventRecord(b->fork, b->st) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
  for (int q = 0; q < b->n && !err; q++)
    if (cudaStreamWaitEvent(b->c[q]->st, b->fork, 0) != cudaSuccess) err = SPH_ERR_CUDA;
  // steps is even: every context's U^n ends in the buffer it started in, so
  // the graph can be replayed
  for (int s = 0; s < steps && !err; s++)
    for (int q = 0; q < b->n && !err; q++) err = sph_step_async(b->c[q], dt, n_iter, NULL, 0);
  for (int q = 0; q < b->n && !err; q++)
    if (cudaEventRecord(b->join[q], b->c[q]->st) != cudaSuccess || cudaStreamWaitEvent(b->st, b->join[q], 0) != cudaSuccess)
      err = SPH_ERR_CUDA;
  cudaGraph_t g = NULL;
  cudaError_t ce = cudaStreamEndCapture(b->st, &g);
  if (!err && ce != cudaSuccess) err = SPH_ERR_CUDA;
  if (!err && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) err = SPH_ERR_CUDA;
  for (int q = 0; q < b->n; q++) {
    // capturing launched nothing: count a replay's launches on each launch
    b->nlaunch[q] = b->c[q]->launches - b->nlaunch[q];
    b->c[q]->launches -= b->nlaunch[q];
  }
  if (err) {
    if (g) cudaGraphDestroy(g);
    b->exec = NULL;
    cudaGetLastError();
    return err;
  }
  b->graph = g;
  return SPH_OK;
}

extern "C" int sph_batch_launch(sph_batch* b, int times) {
  if (!b || !b->exec || times < 0) return SPH_ERR_ARG;
  // the graph holds the buffers of the capture: a context stepped an odd number
  // of times since then has its U^n in the other buffer
  for (int q = 0; q < b->n; q++)
    if (b->c[q]->cur != b->cur[q]) return SPH_ERR_ARG;
  for (int t = 0; t < times; t++)
    if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) return SPH_ERR_CUDA;
  for (int q = 0; q < b->n; q++) b->c[q]->launches += b->nlaunch[q] * times;
  return SPH_OK;
}

extern "C" int sph_batch_status(sph_batch* b, int* first_bad) {
  if (!b) return SPH_ERR_ARG;
  if (first_bad) *first_bad = -1;
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return SPH_ERR_CUDA;
  int worst = SPH_OK;
  for (int q = 0; q < b->n; q++) {
    int e = sph_status(b->c[q], NULL);
    if (e != SPH_OK && worst == SPH_OK) {
      worst = e;
      if (first_bad) *first_bad = q;
    }
  }
  return worst;
}
