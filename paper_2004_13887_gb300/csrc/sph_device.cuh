// sph_device.cuh -- device-side discretisation of the direction-splitting scheme
// of arXiv 2004.13887 (Section 2.2, Appendix B) on the MAC grid.
//
// Everything here is written for the GB300 library; the CPU reference in
// oracle/ is a separate implementation of the same equations.
//
// Rows of the split operators, with coefficients frozen at Ubar (eq.
// chapter3mainsd) and moved to staggered points by arithmetic means:
//   row_c : p-row (A1^d, A2^d, A3^d) or T-row (C2^d, C3^d) at a cell centre;
//   row_f : normal-velocity row (B1^d, B2^{d,d}) on a d-face;
//   row_s : transverse row B2^{d,c} of velocity component c along d;
//   D_M   : cross derivatives, curvature, Coriolis, the off-line parts of
//           grad(div v)/3 and of the vector Laplacian (explicit, in k_rhs).
// The viscous-heating linearisation follows A2/C2 of Appendix B except that the
// G_phiphi*cot(theta) term printed in A2^phi / C2^phi is dropped: it does not
// follow from grad(u):sigma(v) (only A2^theta has it).
//
// Templated on the bulk type R (double: every step in FP64; float: the mixed
// mode, where Ubar, coefficients, right-hand sides, increments and line solves
// are FP32 and the state, its update, the divergence in the pressure and
// temperature rows and the cyclic corrections stay FP64).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace sph {

// Value-type traits of the row templates.  R is the kernels' bulk type (float
// or double) or the adjoint's tape value: T is the type of the metric tables and
// of the grid spacings, CP what a row reads a field or a coefficient plane
// through, MP what the coefficient stage writes a plane through.  For float and
// double these are the plain types and pointers; the adjoint specialises them
// (tables stay double, reads record tape leaves).
template <typename R>
struct Val {
  using T = R;
  using CP = const R*;
  using MP = R*;
};
template <typename R> using TabT = typename Val<R>::T;
// whether R is the FP32 bulk type (the mixed mode's pair arithmetic) or an
// FP64 value (double, or the adjoint's tape value on doubles)
template <typename R> constexpr bool is_f32 = std::is_same<R, float>::value;

template <typename R>
struct Geo {
  using T = TabT<R>;
  int nr, nt, np, npf, per;
  T dr, dth, dph, idr, idth, idph;
  // metric tables: centres rc[nr], faces rf[nr+1]; theta centres/faces
  const T *rc, *rf, *irc, *irf;
  const T *sc, *sf, *isc, *isf, *cc, *cf, *cotc, *cotf;
  // radial background (index i+1 for i in [-1, nr]) and derived tables
  const double *bgp, *bgT;   // p_ref, T_ref (FP64, full values)
  const T* dbgp;             // [nr]   p_ref[i+1] - p_ref[i-1]
  const T* dbgT;             // [nr]   T_ref[i+1] - T_ref[i-1]
  const T* lapT;             // [nr]   (rf_{i+1}^2 (T_{i+1}-T_i) - rf_i^2 (T_i-T_{i-1})) / (rc^2 dr^2)
  const T* rhoref;           // [nr]   (p_ref + pi_inf) / (Rg T_ref)
  const T* ehyd;             // [nr+1] (p_ref[i]-p_ref[i-1]) / (dr rho_ref,f) + g on interior r-faces
  const T* pcen;             // [nr]   p_ref + pi_inf at the centres
  const T* Tcen;             // [nr]   T_ref at the centres
  // rf^2 and sin(theta_f) as hi + lo pairs (lo = 0 in FP64), for div(Ubar)
  const T *rf2h, *rf2l, *sfh, *sfl;
  // Dirichlet wall data of Ubar for the tangential ghosts (ghost = 2 w - the
  // interior value): w[(c*3 + d)*2 + s] is velocity component c on the wall
  // normal to direction d at side s, the mean of its t^n and t^{n+1} values.
  // Arrays without data point to a zero-filled buffer of the largest wall
  // size, so a ghost is always one load (no flag, no null test).  hasw: whether
  // any wall data are set (host bookkeeping).
  // Layouts: c = r: d = theta (nr+1)*np, d = phi (nr+1)*nt; c = theta:
  // d = r (nt+1)*np, d = phi nr*(nt+1); c = phi: d = r nt*npf, d = theta nr*npf.
  const T* w[18];
  int hasw;
};

// twice the wall value of component c on the wall normal to d at side s (c and
// d are constants at every call, so both candidate arrays are fixed parameter
// slots and the side only selects between them)
// (out of line: ghosts are a few threads' business, and inlined into every
// accessor the wall loads would take registers from the stencils' hot path)
template <typename T>
__device__ __noinline__ T wall2_load(const T* lo, const T* hi, int s, int idx) {
  return T(2) * (s ? hi : lo)[idx];
}
template <typename G>
__device__ __forceinline__ auto wall2(const G& g, int c, int d, int s, int idx) -> decltype(+*g.w[0]) {
  return wall2_load(g.w[(c * 3 + d) * 2], g.w[(c * 3 + d) * 2 + 1], s, idx);
}
// the wall term of a ghost on the checked paths: read only when the kernel was
// instantiated for wall data (CIJ == 2), compiled out otherwise (CIJ == 1)
#define WALL2(...) (CIJ == 2 ? wall2(g, __VA_ARGS__) : decltype(wall2(g, __VA_ARGS__))(0))

struct Par {
  double gamma, cv, Pr, mu, pinf, g, omega;
  double kappa, Rg;  // kappa = mu cp / Pr, Rg = cv (gamma-1)
  // the same in FP32, so that FP32 kernels convert nothing from FP64
  float gamma_f, mu_f, kappa_f, g_f, omega_f, iRg_f;
};

// a parameter in the kernel's bulk type: the FP64 value or its FP32 copy
template <typename R> __device__ __forceinline__ R pick(double d, float) { return (R)d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// ---------------------------------------------------------------------------
// FP64 values on the FP32 and integer pipes.  GB300 issues FP64 instructions
// (arithmetic and conversions alike) at 1/64 of the FP32 rate, so the
// mixed-precision kernels move values between double and float with integer
// operations on the IEEE bit patterns, and do the few operations that need more
// than FP32 precision in unevaluated sums of two floats (hi + lo, ~48 bits).

// float -> double, exact; zero and subnormal floats give a signed zero
__device__ __forceinline__ double f2d(float f) {
  unsigned u = __float_as_uint(f);
  unsigned sg = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  if (e == 0) return __hiloint2double((int)sg, 0);
  unsigned E = e == 0xffu ? 0x7ffu : e + 896u;  // rebias 127 -> 1023
  return __hiloint2double((int)(sg | (E << 20) | (m >> 3)), (int)(m << 29));
}
__device__ __forceinline__ double f2d(double d) { return d; }

// 2^k as a float for -126 <= k <= 127 (zero below)
__device__ __forceinline__ float pow2f(int k) { return k < -126 ? 0.f : __int_as_float((k + 127) << 23); }

// double -> hi + lo: hi = d rounded to nearest float (ties to even), lo = the
// remainder d - hi rounded to float.  NaN -> NaN, beyond the float range ->
// +-inf, below 2^-126 -> +-0; lo is dropped where it would be below 2^-126.
__device__ __forceinline__ void d2ff(double d, float& hi, float& lo) {
  unsigned H = (unsigned)__double2hiint(d), L = (unsigned)__double2loint(d);
  unsigned sg = H & 0x80000000u;
  int E = (int)((H >> 20) & 0x7ffu);
  lo = 0.f;
  if (E == 0x7ff) { hi = __uint_as_float(sg | 0x7f800000u | (((H & 0xfffffu) | L) ? 0x400000u : 0u)); return; }
  int e = E - 896;
  if (e >= 255) { hi = __uint_as_float(sg | 0x7f800000u); return; }
  if (e <= 0) { hi = __uint_as_float(sg); return; }
  unsigned m = ((H & 0xfffffu) << 3) | (L >> 29);
  unsigned r = L & 0x1fffffffu;
  unsigned up = (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u;
  hi = __uint_as_float((sg | ((unsigned)e << 23) | m) + up);  // a carry moves into the exponent
  int rem = (int)r - (up ? 0x20000000 : 0);                    // in units of 2^(E-1075)
  float lv = (float)rem * pow2f(E - 1075);
  lo = sg ? -lv : lv;
}
// the nearest float of a double
__device__ __forceinline__ float d2f(double d) { float h, l; d2ff(d, h, l); return h; }
// a double in the bulk type R (exact for R = double)
template <typename R> __device__ __forceinline__ R to_bulk(double d) { return (R)d; }
template <> __device__ __forceinline__ float to_bulk<float>(double d) { return d2f(d); }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// a pair (hi, lo) with |lo| <= ulp(hi)/2, from s + e
__device__ __forceinline__ void renorm(float s, float e, float& hi, float& lo) {
  hi = s + e;
  lo = e - (hi - s);
}
// (ah + al) - (bh + bl), as a pair
__device__ __forceinline__ void ff_sub(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, -bh, s, e);
  renorm(s, e + (al - bl), h, l);
}
// (ah + al) + (bh + bl), as a pair
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, bh, s, e);
  renorm(s, e + (al + bl), h, l);
}
// (ah + al) * (bh + bl), as a pair (error-free product of the high parts by FMA)
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  renorm(p, e, h, l);
}

template <typename R>
struct Coef {  // per cell centre, frozen at Ubar
  using MP = typename Val<R>::MP;
  MP Pb, Tb, rho, drho, beta, uc0, uc1, uc2;
  MP grr, gtt, gpp, srt, srp, stp;  // G_rr, G_tt, G_pp, G_rt+G_tr, G_rp+G_pr, G_tp+G_pt
  // the three parts of div(Ubar) at the centre, (1/r^2) d_r (r^2 u_r),
  // (1/(r sin)) d_t (sin u_t), (1/(r sin)) d_p u_p, for the grad-div viscous
  // terms of the momentum rows (each row reads them at its two centres)
  MP dvr, dvt, dvp;
};
constexpr int NCOEF = 17;

template <typename R> struct CF { typename Val<R>::CP f[5]; };
template <typename R> struct MF { R* f[5]; };

// 32-bit flat indices: the host refuses grids whose arrays (and line-solve
// scratch) would not fit in an int.
//
// Built with SPH_CHECKED (the bounds-checked debug library), every index is
// checked against its field's extents first: a violation is counted in
// g_bounds (with the first offending field and (i, j, k)) and the access is
// redirected to element 0, so that the run goes on and the host reports it.
#ifdef SPH_CHECKED
// (one counter per translation unit: the host merges them)
static __device__ int g_bounds[5];  // count, field, i, j, k of the first violation
__device__ __forceinline__ int checked(int f, int i, int j, int k, int ni, int nj, int nk, int idx) {
  if (i < 0 || i >= ni || j < 0 || j >= nj || k < 0 || k >= nk) {
    if (atomicAdd(&g_bounds[0], 1) == 0) { g_bounds[1] = f; g_bounds[2] = i; g_bounds[3] = j; g_bounds[4] = k; }
    return 0;
  }
  return idx;
}
#define SPH_IDX(f, ni, nj, nk, e) checked(f, i, j, k, ni, nj, nk, e)
#else
#define SPH_IDX(f, ni, nj, nk, e) (e)
#endif
template <typename G> __device__ __forceinline__ int IC(const G& g, int i, int j, int k) {
  return SPH_IDX(0, g.nr, g.nt, g.np, (i * g.nt + j) * g.np + k);
}
template <typename G> __device__ __forceinline__ int IRf(const G& g, int i, int j, int k) {
  return SPH_IDX(1, g.nr + 1, g.nt, g.np, (i * g.nt + j) * g.np + k);
}
template <typename G> __device__ __forceinline__ int ITf(const G& g, int i, int j, int k) {
  return SPH_IDX(2, g.nr, g.nt + 1, g.np, (i * (g.nt + 1) + j) * g.np + k);
}
template <typename G> __device__ __forceinline__ int IPf(const G& g, int i, int j, int k) {
  return SPH_IDX(3, g.nr, g.nt, g.npf, (i * g.nt + j) * g.npf + k);
}

// a / b; the mixed path uses the fast single-precision division (2 ulp)
template <typename R> __device__ __forceinline__ R sdiv(R a, R b) { return a / b; }
template <> __device__ __forceinline__ float sdiv<float>(float a, float b) { return __fdividef(a, b); }

template <typename G> __device__ __forceinline__ int wrapk(const G& g, int k) { return k < 0 ? k + g.np : (k >= g.np ? k - g.np : k); }
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---------------------------------------------------------------- accessors
// CIJ = 0 skips the checks on i and j: for points whose +-2 neighbourhood in
// r and theta is inside the grid (the kernels decide this per block, so warps
// do not diverge); k (phi) is always checked.
//
// Centre perturbation with zero Neumann ghosts (the background has its own).
template <typename P> using ValOf = typename std::decay<decltype(std::declval<P>()[0])>::type;

template <int CIJ = 2, typename G, typename P>
__device__ __forceinline__ ValOf<P> cpert(const G& g, const P& f, int i, int j, int k) {
  int ii = CIJ ? clampi(i, 0, g.nr - 1) : i, jj = CIJ ? clampi(j, 0, g.nt - 1) : j;
  int kk = g.per ? wrapk(g, k) : clampi(k, 0, g.np - 1);
  return f[IC(g, ii, jj, kk)];
}
// Velocities with Dirichlet ghosts on tangential walls: ghost = 2 w - interior
// (w = 0, no-slip, unless wall data were set).  CIJ = 0: interior points, no
// checks on i and j and the homogeneous rule for the phi walls; 1: checked,
// homogeneous walls; 2: checked, wall data read (the kernels send every tile
// to 2 when wall data are set and are instantiated without it otherwise, so
// the other paths carry no wall code).
template <int CIJ = 2, typename G, typename P>
__device__ __forceinline__ ValOf<P> vr(const G& g, const P& u, int i, int j, int k) {
  if (CIJ && j < 0) return WALL2(0, 1, 0, i * g.np + k) - u[IRf(g, i, 0, k)];
  if (CIJ && j >= g.nt) return WALL2(0, 1, 1, i * g.np + k) - u[IRf(g, i, g.nt - 1, k)];
  if (k < 0 || k >= g.np) {
    if (g.per) k = wrapk(g, k);
    else if constexpr (CIJ != 0) return WALL2(0, 2, k >= g.np, i * g.nt + j) - u[IRf(g, i, j, k < 0 ? 0 : g.np - 1)];
    else return -u[IRf(g, i, j, k < 0 ? 0 : g.np - 1)];
  }
  return u[IRf(g, i, j, k)];
}
template <int CIJ = 2, typename G, typename P>
__device__ __forceinline__ ValOf<P> vt(const G& g, const P& u, int i, int j, int k) {
  if (CIJ && i < 0) return WALL2(1, 0, 0, j * g.np + k) - u[ITf(g, 0, j, k)];
  if (CIJ && i >= g.nr) return WALL2(1, 0, 1, j * g.np + k) - u[ITf(g, g.nr - 1, j, k)];
  if (k < 0 || k >= g.np) {
    if (g.per) k = wrapk(g, k);
    else if constexpr (CIJ != 0) return WALL2(1, 2, k >= g.np, i * (g.nt + 1) + j) - u[ITf(g, i, j, k < 0 ? 0 : g.np - 1)];
    else return -u[ITf(g, i, j, k < 0 ? 0 : g.np - 1)];
  }
  return u[ITf(g, i, j, k)];
}
template <int CIJ = 2, typename G, typename P>
__device__ __forceinline__ ValOf<P> vp(const G& g, const P& u, int i, int j, int k) {
  if (g.per) k = wrapk(g, k);
  if (CIJ && i < 0) return WALL2(2, 0, 0, j * g.npf + k) - u[IPf(g, 0, j, k)];
  if (CIJ && i >= g.nr) return WALL2(2, 0, 1, j * g.npf + k) - u[IPf(g, g.nr - 1, j, k)];
  if (CIJ && j < 0) return WALL2(2, 1, 0, i * g.npf + k) - u[IPf(g, i, 0, k)];
  if (CIJ && j >= g.nt) return WALL2(2, 1, 1, i * g.npf + k) - u[IPf(g, i, g.nt - 1, k)];
  return u[IPf(g, i, j, k)];
}
template <int CIJ = 2, typename G, typename P>
__device__ __forceinline__ ValOf<P> hr(const G& g, const P& u, int i, int j, int k) {
  return ValOf<P>(0.5) * (vr<CIJ>(g, u, i, j, k) + vr<CIJ>(g, u, i + 1, j, k));
}
template <int CIJ = 2, typename G, typename P>
__device__ __forceinline__ ValOf<P> ht(const G& g, const P& u, int i, int j, int k) {
  return ValOf<P>(0.5) * (vt<CIJ>(g, u, i, j, k) + vt<CIJ>(g, u, i, j + 1, k));
}
template <int CIJ = 2, typename G, typename P>
__device__ __forceinline__ ValOf<P> hp(const G& g, const P& u, int i, int j, int k) {
  return ValOf<P>(0.5) * (vp<CIJ>(g, u, i, j, k) + vp<CIJ>(g, u, i, j, k + 1));
}
template <typename R>
__device__ __forceinline__ R rho_at(const Geo<R>& g, const Coef<R>& c, int i, int j, int k) {
  if (g.per) k = wrapk(g, k);
  return c.rho[IC(g, i, j, k)];
}

// A velocity component averaged to centre (i, j, k): in interior blocks
// (CIJ = 0) read from the coefficient plane k_coef wrote (uc0/uc1/uc2, the
// same FP32 operations, so the same value), with the no-slip ghost -- minus the
// mirrored centre -- beyond a phi wall (interior blocks run only without wall
// data) and the periodic wrap (only used for the components tangential to phi);
// elsewhere the face average with all checks.
template <int CC, typename R>
__device__ __forceinline__ R ucen(const Geo<R>& g, const typename Val<R>::CP& plane, int i, int j, int k) {
  if (k < 0 || k >= g.np) {
    if (g.per) k = wrapk(g, k);
    else return -plane[IC(g, i, j, k < 0 ? 0 : g.np - 1)];
  }
  return plane[IC(g, i, j, k)];
}
template <int CIJ, typename R, typename P>
__device__ __forceinline__ R hrc(const Geo<R>& g, const Coef<R>& c, const P& u, int i, int j, int k) {
  if constexpr (CIJ != 0) return hr<CIJ>(g, u, i, j, k);
  else return ucen<0>(g, c.uc0, i, j, k);
}
template <int CIJ, typename R, typename P>
__device__ __forceinline__ R htc(const Geo<R>& g, const Coef<R>& c, const P& u, int i, int j, int k) {
  if constexpr (CIJ != 0) return ht<CIJ>(g, u, i, j, k);
  else return ucen<1>(g, c.uc1, i, j, k);
}
template <int CIJ, typename R, typename P>
__device__ __forceinline__ R hpc(const Geo<R>& g, const Coef<R>& c, const P& u, int i, int j, int k) {
  if constexpr (CIJ != 0) return hp<CIJ>(g, u, i, j, k);
  else return ucen<2>(g, c.uc2, i, j, k);
}

// whether the +-2 neighbourhood of (i, j) in r and theta is inside the grid
template <typename G>
__device__ __forceinline__ bool inner_ij(const G& g, int i, int j) {
  return i >= 2 && i <= g.nr - 3 && j >= 2 && j <= g.nt - 3;
}

// --------------------------------------------------------- thermodynamics
// Coefficients of a centre from the midpoint perturbations p', T' and the
// background at radius index i; k_coef and the line kernels both call this, so
// their values are the same.
template <typename R>
struct Thermo { R Pb, Tb, rho, beta; };
template <typename R>
__device__ __forceinline__ Thermo<R> thermo(const Geo<R>& g, const Par& P, int i, R pp, R Tp) {
  R pref = g.pcen[i], Tref = g.Tcen[i];
  Thermo<R> t;
  t.Pb = pref + pp;
  t.Tb = Tref + Tp;
  R iRg = pick<R>(1.0 / P.Rg, P.iRg_f);
  R itb = sdiv(R(1), t.Tb);
  t.rho = t.Pb * itb * iRg;
  t.beta = sdiv((pick<R>(P.gamma, P.gamma_f) - R(1)) * t.Tb, t.Pb);
  return t;
}

// ------------------------------------------------------------------- rows
// Each row is split into a loader (the values it reads from memory) and a
// weight function (pure arithmetic on those values and the metric tables), so
// that the line solvers can fetch the next row while eliminating the current.
//
// p-row (isT = 0) or T-row (isT = 1) of D_d at centre (i,j,k).  The coupling to
// the normal velocity u_d on faces m, m+1 is split as
//   wu[q] = a * gd[q] + wv[q],
// a the divergence coefficient (gamma(p+pi_inf) or (gamma-1)T, plus
// (2 mu (gamma-1)/3) tr G or its T-row analogue), gd the geometric weights of
// the d-part of div u, wv the remaining viscous-heating and metric terms.
template <typename R>
struct RowC {
  R wp[3], wT[3];   // p (advection, p-row only) and T (conduction [+ advection]) at m-1, m, m+1
  R a, gd[2], wv[2];
  R adv;            // advection coefficient (wp or wT = [-adv, 0, adv] + ...)
  R dif;            // conduction coefficient: wT += -dif * geometric Laplacian
};

// centre coefficients the p- and T-rows of direction d read
template <typename R>
struct CPt { R Pb, Tb, beta, uc, grr, gtt, gpp, s1, s2; };

template <typename R>
__device__ __forceinline__ CPt<R> load_c(const Coef<R>& c, int d, int id) {
  CPt<R> q;
  q.Pb = c.Pb[id]; q.Tb = c.Tb[id]; q.beta = c.beta[id];
  q.uc = d == 0 ? c.uc0[id] : d == 1 ? c.uc1[id] : c.uc2[id];
  q.grr = c.grr[id]; q.gtt = c.gtt[id]; q.gpp = c.gpp[id];
  q.s1 = d == 1 ? c.srt[id] : d == 2 ? c.srp[id] : R(0);
  q.s2 = d == 2 ? c.stp[id] : R(0);
  return q;
}

template <typename R>
__device__ __forceinline__ void row_cw(const Geo<R>& g, const Par& P, const CPt<R>& q, int d, int isT, int i, int j,
                                       RowC<R>& w) {
  R gm = pick<R>(P.gamma, P.gamma_f), mu = pick<R>(P.mu, P.mu_f);
  R be = q.beta;
  R alin = isT ? (gm - R(1)) * q.Tb : gm * q.Pb;
  R visc = isT ? mu * be : mu * (gm - R(1));
  R kap = pick<R>(P.kappa, P.kappa_f);
  R dif = isT ? be * kap : (gm - R(1)) * kap;
  R g_rr = q.grr, g_tt = q.gtt, g_pp = q.gpp;
  R tr = g_rr + g_tt + g_pp;
  R ir = g.irc[i];
  w.wp[0] = w.wp[1] = w.wp[2] = R(0);
  w.wT[0] = w.wT[1] = w.wT[2] = R(0);
  R* wa = isT ? w.wT : w.wp;
  w.a = alin + R(2.0 / 3.0) * visc * tr;
  w.dif = dif;
  if (d == 0) {
    R adv = R(0.5) * q.uc * g.idr;
    w.adv = adv;
    wa[0] -= adv; wa[2] += adv;
    R f0 = g.rf[i] * g.rf[i], f1 = g.rf[i + 1] * g.rf[i + 1];
    R ir2 = ir * ir;
    R df = -dif * ir2 * g.idr * g.idr;
    w.wT[0] += df * f0; w.wT[1] -= df * (f0 + f1); w.wT[2] += df * f1;
    w.gd[0] = -f0 * ir2 * g.idr;
    w.gd[1] = f1 * ir2 * g.idr;
    R m0 = R(2) * visc * g_rr * g.idr, m1 = visc * (g_tt + g_pp) * ir;
    w.wv[0] = m0 - m1;
    w.wv[1] = -m0 - m1;
  } else if (d == 1) {
    R is = g.isc[j], cot = g.cotc[j];
    R adv = R(0.5) * q.uc * ir * g.idth;
    w.adv = adv;
    wa[0] -= adv; wa[2] += adv;
    R f0 = g.sf[j], f1 = g.sf[j + 1];
    R df = -dif * ir * ir * is * g.idth * g.idth;
    w.wT[0] += df * f0; w.wT[1] -= df * (f0 + f1); w.wT[2] += df * f1;
    w.gd[0] = -f0 * ir * is * g.idth;
    w.gd[1] = f1 * ir * is * g.idth;
    R lin = -visc * (R(2) * g_pp * cot - q.s1) * R(0.5) * ir;
    R m0 = R(2) * visc * g_tt * ir * g.idth;
    w.wv[0] = m0 + lin;
    w.wv[1] = -m0 + lin;
  } else {
    R is = g.isc[j], cot = g.cotc[j];
    R adv = R(0.5) * q.uc * ir * is * g.idph;
    w.adv = adv;
    wa[0] -= adv; wa[2] += adv;
    R df = -dif * ir * ir * is * is * g.idph * g.idph;
    w.wT[0] += df; w.wT[1] -= R(2) * df; w.wT[2] += df;
    w.gd[0] = -ir * is * g.idph;
    w.gd[1] = ir * is * g.idph;
    // the phi row's coefficient is a - 2 visc G_pp (Appendix B, A2^phi): the
    // -2 visc G_pp part goes with the remaining terms
    R lin = visc * (q.s1 + q.s2 * cot) * R(0.5) * ir;
    R m0 = R(2) * visc * g_pp * ir * is * g.idph;
    w.wv[0] = m0 + lin;
    w.wv[1] = -m0 + lin;
  }
}

template <typename R>
__device__ __forceinline__ void row_c(const Geo<R>& g, const Par& P, const Coef<R>& c, int d, int isT, int i, int j,
                                      int k, RowC<R>& w) {
  row_cw(g, P, load_c(c, d, IC(g, i, j, k)), d, isT, i, j, w);
}

// Normal-velocity row of D_d on the d-face (i,j,k): p at centres m-1, m and
// u_d on faces m-1, m, m+1.  It reads rho at the two centres and Ubar's u_d on
// the face.
template <typename R>
struct FPt { R rho0, rho1, ub; };

template <typename R>
__device__ __forceinline__ FPt<R> load_f(const Geo<R>& g, const Coef<R>& c, const typename Val<R>::CP& ubd, int d, int i,
                                         int j, int k) {
  FPt<R> q;
  if (d == 0) {
    q.rho0 = rho_at(g, c, i - 1, j, k); q.rho1 = rho_at(g, c, i, j, k); q.ub = ubd[IRf(g, i, j, k)];
  } else if (d == 1) {
    q.rho0 = rho_at(g, c, i, j - 1, k); q.rho1 = rho_at(g, c, i, j, k); q.ub = ubd[ITf(g, i, j, k)];
  } else {
    q.rho0 = rho_at(g, c, i, j, k - 1); q.rho1 = rho_at(g, c, i, j, k); q.ub = ubd[IPf(g, i, j, k)];
  }
  return q;
}

template <typename R>
__device__ __forceinline__ void row_fw(const Geo<R>& g, const Par& P, const FPt<R>& q, int d, int i, int j, R wp[2],
                                       R wu[3]) {
  R mu = pick<R>(P.mu, P.mu_f);
  R irh = sdiv(R(2), q.rho0 + q.rho1);
  if (d == 0) {
    R irf = g.irf[i];
    wp[0] = -irh * g.idr; wp[1] = irh * g.idr;
    R adv = R(0.5) * q.ub * g.idr;
    R c0 = g.rc[i - 1] * g.rc[i - 1], c1 = g.rc[i] * g.rc[i];
    R ic0 = g.irc[i - 1] * g.irc[i - 1], ic1 = g.irc[i] * g.irc[i];
    R lap = -mu * irh * irf * irf * g.idr * g.idr;
    R gdv = -mu * irh * R(1.0 / 3.0) * g.idr * g.idr;
    R fm = g.rf[i - 1] * g.rf[i - 1], f0 = g.rf[i] * g.rf[i], fp = g.rf[i + 1] * g.rf[i + 1];
    wu[0] = -adv + lap * c0 + gdv * fm * ic0;
    wu[1] = -lap * (c0 + c1) - gdv * f0 * (ic1 + ic0);
    wu[2] = adv + lap * c1 + gdv * fp * ic1;
  } else if (d == 1) {
    R ir = g.irc[i], isf = g.isf[j];
    wp[0] = -irh * ir * g.idth; wp[1] = irh * ir * g.idth;
    R adv = R(0.5) * q.ub * ir * g.idth;
    R c0 = g.sc[j - 1], c1 = g.sc[j];
    R lap = -mu * irh * ir * ir * isf * g.idth * g.idth;
    R gdv = -mu * irh * R(1.0 / 3.0) * ir * ir * g.idth * g.idth;
    wu[0] = -adv + lap * c0 + gdv * g.sf[j - 1] * g.isc[j - 1];
    wu[1] = -lap * (c0 + c1) - gdv * g.sf[j] * (g.isc[j] + g.isc[j - 1]);
    wu[2] = adv + lap * c1 + gdv * g.sf[j + 1] * g.isc[j];
  } else {
    R ir = g.irc[i], is = g.isc[j];
    wp[0] = -irh * ir * is * g.idph; wp[1] = irh * ir * is * g.idph;
    R adv = R(0.5) * q.ub * ir * is * g.idph;
    R lap = -R(4.0 / 3.0) * mu * irh * ir * ir * is * is * g.idph * g.idph;
    wu[0] = -adv + lap; wu[1] = -R(2) * lap; wu[2] = adv + lap;
  }
}

template <typename R>
__device__ __forceinline__ void row_f(const Geo<R>& g, const Par& P, const Coef<R>& c, const typename Val<R>::CP& ubd, int d, int i,
                                      int j, int k, R wp[2], R wu[3]) {
  row_fw(g, P, load_f(g, c, ubd, d, i, j, k), d, i, j, wp, wu);
}

// Transverse row of D_d for velocity component cc at its location (i,j,k): it
// reads rho at the two centres beside the face and the advecting Ubar component.
template <typename R>
struct SPt { R rho0, rho1, ua; };

template <int CIJ = 2, typename R>
__device__ __forceinline__ SPt<R> load_s(const Geo<R>& g, const Coef<R>& c, const CF<R>& ub, int cc, int d, int i,
                                         int j, int k) {
  SPt<R> q;
  if (cc == 0) { q.rho0 = rho_at(g, c, i - 1, j, k); q.rho1 = rho_at(g, c, i, j, k); }
  else if (cc == 1) { q.rho0 = rho_at(g, c, i, j - 1, k); q.rho1 = rho_at(g, c, i, j, k); }
  else { q.rho0 = rho_at(g, c, i, j, k - 1); q.rho1 = rho_at(g, c, i, j, k); }
  if (cc == 0) q.ua = d == 1 ? R(0.5) * (htc<CIJ>(g, c, ub.f[2], i - 1, j, k) + htc<CIJ>(g, c, ub.f[2], i, j, k))
                             : R(0.5) * (hpc<CIJ>(g, c, ub.f[3], i - 1, j, k) + hpc<CIJ>(g, c, ub.f[3], i, j, k));
  else if (cc == 1) q.ua = d == 0 ? R(0.5) * (hrc<CIJ>(g, c, ub.f[1], i, j - 1, k) + hrc<CIJ>(g, c, ub.f[1], i, j, k))
                                  : R(0.5) * (hpc<CIJ>(g, c, ub.f[3], i, j - 1, k) + hpc<CIJ>(g, c, ub.f[3], i, j, k));
  else q.ua = d == 0 ? R(0.5) * (hrc<CIJ>(g, c, ub.f[1], i, j, k - 1) + hrc<CIJ>(g, c, ub.f[1], i, j, k))
                     : R(0.5) * (htc<CIJ>(g, c, ub.f[2], i, j, k - 1) + htc<CIJ>(g, c, ub.f[2], i, j, k));
  return q;
}

template <typename R>
__device__ __forceinline__ void row_sw(const Geo<R>& g, const Par& P, const SPt<R>& q, int cc, int d, int i, int j,
                                       R w[3]) {
  R mu = pick<R>(P.mu, P.mu_f);
  R irh = sdiv(R(2), q.rho0 + q.rho1);
  R ir = cc == 0 ? g.irf[i] : g.irc[i];
  R is = cc == 1 ? g.isf[j] : g.isc[j];
  R ua = q.ua;
  if (d == 0) {
    R adv = R(0.5) * ua * g.idr, lap = -mu * irh * ir * ir * g.idr * g.idr;
    R f0 = g.rf[i] * g.rf[i], f1 = g.rf[i + 1] * g.rf[i + 1];
    w[0] = -adv + lap * f0; w[1] = -lap * (f0 + f1); w[2] = adv + lap * f1;
  } else if (d == 1) {
    R adv = R(0.5) * ua * ir * g.idth, lap = -mu * irh * ir * ir * is * g.idth * g.idth;
    R f0 = g.sf[j], f1 = g.sf[j + 1];
    w[0] = -adv + lap * f0; w[1] = -lap * (f0 + f1); w[2] = adv + lap * f1;
  } else {
    R adv = R(0.5) * ua * ir * is * g.idph, lap = -mu * irh * ir * ir * is * is * g.idph * g.idph;
    w[0] = -adv + lap; w[1] = -R(2) * lap; w[2] = adv + lap;
  }
}

template <int CIJ = 2, typename R>
__device__ __forceinline__ void row_s(const Geo<R>& g, const Par& P, const Coef<R>& c, const CF<R>& ub, int cc, int d,
                                      int i, int j, int k, R w[3]) {
  row_sw(g, P, load_s<CIJ>(g, c, ub, cc, d, i, j, k), cc, d, i, j, w);
}

}  // namespace sph
