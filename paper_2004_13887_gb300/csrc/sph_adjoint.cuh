// sph_adjoint.cuh -- reverse mode of one Picard iteration of the scheme of
// Section 2.2 (eqs. chapter3mainsd, splitting2, spl1-spl3), FP64.
//
// One iteration maps (a, b) = (U^n, U^{n+1,k}) to
//   out = b + x_phi,  x_phi = A_phi^{-1} x_theta,  x_theta = A_theta^{-1} x_r,
//   x_r = A_r^{-1} R,  R = -(b - a) - tau [N(Ubar) + G - S],  Ubar = (a + b)/2,
// with A_d = I + tau/2 D_d(Ubar) and every coefficient frozen at Ubar.  Given
// lambda = dJ/d out, the adjoint is
//   mu_phi = A_phi^{-T} lambda, mu_theta = A_theta^{-T} mu_phi, mu_r = A_r^{-T} mu_theta
//   dJ/db = lambda - mu_r + g/2,  dJ/da = mu_r + g/2,
//   g = grad over Ubar of  <mu_r, R(Ubar)> - sum_d <mu_d, A_d(Ubar) x_d>
// (the x_d and mu_d held fixed).  The transposed solves are the line solvers of
// sph.cu with TR = true.  g is taken here by reverse-mode differentiation of the
// same row functions the forward kernels run (rhs_c_at, rhs_u_at,
// assemble_block, scalar_row, coef_at), instantiated on the tape value `ad`: each
// thread evaluates the rows of one location, recording every operation on a
// tape, then sweeps the tape backwards and scatters the adjoints of its leaves
// -- values of Ubar and of the coefficient planes -- with FP64 atomics.  The
// planes are themselves functions of Ubar, so a last pass takes the planes'
// adjoints back to Ubar through coef_at.
#pragma once

namespace adj {

// The tape of one thread: node q holds up to two parents with their partial
// derivatives, or (a leaf) an array code and element index.  Arrays are
// interleaved by thread (element q of thread s at q * stride + s), so a warp
// recording the same node touches consecutive words.
struct Tape {
  double* d;      // partials, 2 per node
  int* ix;        // parents, 2 per node: node index, -1 none, <= -2 leaf of code -2 - ix
  int* li;        // leaf element index, 1 per node
  double* adj;    // adjoints, 1 per node
  int n, cap, stride, slot, ovf;
  __device__ __forceinline__ int node(int a, double da, int b, double db) {
    if (n >= cap) { ovf = 1; return -1; }
    int q = n++;
    size_t o = (size_t)(2 * q) * stride + slot;
    d[o] = da; d[o + stride] = db;
    ix[o] = a; ix[o + stride] = b;
    adj[(size_t)q * stride + slot] = 0.0;
    return q;
  }
  __device__ __forceinline__ int leaf(int code, int idx) {
    if (n >= cap) { ovf = 1; return -1; }
    int q = n++;
    ix[(size_t)(2 * q) * stride + slot] = -2 - code;
    li[(size_t)q * stride + slot] = idx;
    adj[(size_t)q * stride + slot] = 0.0;
    return q;
  }
  // adjoint 1 at node `out`, swept back to the leaves, whose adjoints are added
  // to lam[code][idx]
  __device__ void reverse(int out, double* const* lam) {
    if (out < 0) return;
    adj[(size_t)out * stride + slot] = 1.0;
    for (int q = out; q >= 0; q--) {
      double a = adj[(size_t)q * stride + slot];
      if (a == 0.0) continue;
      size_t o = (size_t)(2 * q) * stride + slot;
      int p0 = ix[o];
      if (p0 <= -2) {
        atomicAdd(lam[-2 - p0] + li[(size_t)q * stride + slot], a);
        continue;
      }
      if (p0 >= 0) adj[(size_t)p0 * stride + slot] += d[o] * a;
      int p1 = ix[o + stride];
      if (p1 >= 0) adj[(size_t)p1 * stride + slot] += d[o + stride] * a;
    }
  }
};

// A value on the tape (id >= 0) or a constant (id = -1).
struct ad {
  double v;
  int id;
  Tape* t;
  __device__ __forceinline__ ad() : v(0.0), id(-1), t(nullptr) {}
  __device__ __forceinline__ ad(double x) : v(x), id(-1), t(nullptr) {}
  __device__ __forceinline__ ad(double x, int i, Tape* tp) : v(x), id(i), t(tp) {}
};

__device__ __forceinline__ ad operator+(const ad& a, const ad& b) {
  if (b.id < 0) return ad(a.v + b.v, a.id, a.t);  // d(a + c)/da = 1: the same node
  if (a.id < 0) return ad(a.v + b.v, b.id, b.t);
  return ad(a.v + b.v, a.t->node(a.id, 1.0, b.id, 1.0), a.t);
}
__device__ __forceinline__ ad operator-(const ad& a, const ad& b) {
  if (b.id < 0) return ad(a.v - b.v, a.id, a.t);
  if (a.id < 0) return ad(a.v - b.v, b.t->node(b.id, -1.0, -1, 0.0), b.t);
  return ad(a.v - b.v, a.t->node(a.id, 1.0, b.id, -1.0), a.t);
}
__device__ __forceinline__ ad operator-(const ad& a) {
  if (a.id < 0) return ad(-a.v);
  return ad(-a.v, a.t->node(a.id, -1.0, -1, 0.0), a.t);
}
__device__ __forceinline__ ad operator*(const ad& a, const ad& b) {
  if (b.id < 0) {
    if (a.id < 0) return ad(a.v * b.v);
    return ad(a.v * b.v, a.t->node(a.id, b.v, -1, 0.0), a.t);
  }
  if (a.id < 0) return ad(a.v * b.v, b.t->node(b.id, a.v, -1, 0.0), b.t);
  return ad(a.v * b.v, a.t->node(a.id, b.v, b.id, a.v), a.t);
}
__device__ __forceinline__ ad operator/(const ad& a, const ad& b) {
  double q = a.v / b.v;
  if (b.id < 0) {
    if (a.id < 0) return ad(q);
    return ad(q, a.t->node(a.id, 1.0 / b.v, -1, 0.0), a.t);
  }
  double db = -q / b.v;
  if (a.id < 0) return ad(q, b.t->node(b.id, db, -1, 0.0), b.t);
  return ad(q, a.t->node(a.id, 1.0 / b.v, b.id, db), a.t);
}
__device__ __forceinline__ ad& operator+=(ad& a, const ad& b) { a = a + b; return a; }
__device__ __forceinline__ ad& operator-=(ad& a, const ad& b) { a = a - b; return a; }
__device__ __forceinline__ ad& operator*=(ad& a, const ad& b) { a = a * b; return a; }
__device__ __forceinline__ bool operator==(const ad& a, const ad& b) { return a.v == b.v; }
__device__ __forceinline__ bool isfinite(const ad& a) { return ::isfinite(a.v); }

// Reads of a field or coefficient plane that record tape leaves (code = the
// array's index in the adjoint accumulators: the 5 fields of Ubar, then the
// 17 coefficient planes in Coef's order).
struct LeafPtr {
  const double* p;
  int code;
  Tape* t;
  __device__ __forceinline__ ad operator[](int i) const { return ad(p[i], t->leaf(code, i), t); }
};

// the adjoint's stand-in for a Coef or MF the rows write into: slots that keep
// the written values
struct Slot {
  mutable ad v;
  __device__ __forceinline__ ad& operator[](int) const { return v; }
};
struct CoefOut { Slot Pb, Tb, rho, drho, beta, uc0, uc1, uc2, grr, gtt, gpp, srt, srp, stp, dvr, dvt, dvp; };
struct RowsOut { Slot f[5]; };

constexpr int NLAM = 5 + sph::NCOEF;  // accumulators: Ubar fields, then coefficient planes

}  // namespace adj

namespace sph {
template <>
struct Val<adj::ad> {
  using T = double;
  using CP = adj::LeafPtr;
  using MP = adj::LeafPtr;
};
}  // namespace sph

namespace adj {

// Everything a gradient kernel reads: the forward values at Ubar (FP64 planes and
// fields), the adjoint vectors, the accumulators and the tape.
struct AdjArgs {
  Geo<double> g;
  Par P;
  Coef<double> c;       // coefficient planes at Ubar
  CF<double> ub;        // Ubar
  double tau;
  CF<double> mu[3];     // mu_r (the right-hand side's weight), mu_theta, mu_phi
  CF<double> x[3];      // the forward sweeps' solutions x_r, x_theta, x_phi
  double* lam[NLAM];    // gradient accumulators (Ubar, then the planes)
  double* td; int* tix; int* tli; double* tadj;
  int cap;
  int* flag;            // bit 8: a tape overflowed
  int* maxn;            // the longest tape used
};

__device__ __forceinline__ Tape make_tape(const AdjArgs& A) {
  Tape T;
  T.d = A.td; T.ix = A.tix; T.li = A.tli; T.adj = A.tadj;
  T.n = 0; T.cap = A.cap; T.stride = gridDim.x * blockDim.x;
  T.slot = blockIdx.x * blockDim.x + threadIdx.x;
  T.ovf = 0;
  return T;
}

// the geometry with its tables as they are (doubles) for the tape instantiation
__device__ __forceinline__ Geo<ad> geo_ad(const Geo<double>& a) {
  static_assert(sizeof(Geo<ad>) == sizeof(Geo<double>), "Geo<ad> must have Geo<double>'s layout");
  Geo<ad> g;
  memcpy(&g, &a, sizeof g);
  return g;
}

__device__ __forceinline__ CF<ad> leaves_ub(const AdjArgs& A, Tape* t) {
  CF<ad> u;
  for (int f = 0; f < 5; f++) u.f[f] = LeafPtr{A.ub.f[f], f, t};
  return u;
}
__device__ __forceinline__ Coef<ad> leaves_coef(const AdjArgs& A, Tape* t) {
  const Coef<double>& c = A.c;
  Coef<ad> o;
  const double* src[NCOEF] = {c.Pb, c.Tb, c.rho, c.drho, c.beta, c.uc0, c.uc1, c.uc2,
                              c.grr, c.gtt, c.gpp, c.srt, c.srp, c.stp, c.dvr, c.dvt, c.dvp};
  LeafPtr* dst[NCOEF] = {&o.Pb, &o.Tb, &o.rho, &o.drho, &o.beta, &o.uc0, &o.uc1, &o.uc2,
                         &o.grr, &o.gtt, &o.gpp, &o.srt, &o.srp, &o.stp, &o.dvr, &o.dvt, &o.dvp};
  for (int q = 0; q < NCOEF; q++) *dst[q] = LeafPtr{src[q], 5 + q, t};
  return o;
}

__device__ __forceinline__ void finish(const AdjArgs& A, Tape& T, const ad& psi) {
  T.reverse(psi.t ? psi.id : -1, A.lam);
  if (T.ovf) atomicOr(A.flag, 8);
  atomicMax(A.maxn, T.n);
}

// (1) <mu_r, R(Ubar)>: one thread per location -- centres (kind = 0, the p- and
// T-rows) or the interior faces of u_r, u_theta, u_phi (kind 1, 2, 3).  D = U^k -
// U^n and the source do not depend on Ubar: hasD = has_src = 0.
__global__ void __launch_bounds__(128) k_adj_rhs(AdjArgs A, int kind) {
  Tape T = make_tape(A);
  const Geo<double>& g = A.g;
  const Geo<ad> ga = geo_ad(g);
  const int nt = g.nt + (kind == 2), np = kind == 3 ? g.npf : g.np, nr = g.nr + (kind == 1);
  const long total = (long)nr * nt * np;
  CF<ad> none;
  for (int f = 0; f < 5; f++) none.f[f] = LeafPtr{nullptr, 0, nullptr};
  CF<double> noned;
  for (int f = 0; f < 5; f++) noned.f[f] = nullptr;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    int t = (int)e;
    int k = t % np, j = (t / np) % nt, i = t / (np * nt);
    if (kind == 1 && (i == 0 || i == g.nr)) continue;
    if (kind == 2 && (j == 0 || j == g.nt)) continue;
    if (kind == 3 && !g.per && (k == 0 || k == g.np)) continue;
    double w0 = A.mu[0].f[kind == 0 ? 0 : kind][t];
    double w4 = kind == 0 ? A.mu[0].f[4][t] : 0.0;
    if (w0 == 0.0 && w4 == 0.0) continue;
    T.n = 0;
    CF<ad> ub = leaves_ub(A, &T);
    Coef<ad> c = leaves_coef(A, &T);
    RowsOut out;
    ad psi;
    if (kind == 0) {
      rhs_c_at<2>(ga, g, A.P, c, ub, none, noned, noned, none, 0, noned, 0, ad(A.tau), out, i, j, k, t);
      psi = out.f[0].v * w0 + out.f[4].v * w4;
    } else if (kind == 1) {
      rhs_u_at<2, 0>(ga, A.P, c, ub, none, 0, noned, 0, ad(A.tau), out, i, j, k, t);
      psi = out.f[1].v * w0;
    } else if (kind == 2) {
      rhs_u_at<2, 1>(ga, A.P, c, ub, none, 0, noned, 0, ad(A.tau), out, i, j, k, t);
      psi = out.f[2].v * w0;
    } else {
      rhs_u_at<2, 2>(ga, A.P, c, ub, none, 0, noned, 0, ad(A.tau), out, i, j, k, t);
      psi = out.f[3].v * w0;
    }
    finish(A, T, psi);
  }
}

// the unknowns (p, T, u_d on face m+1) of block m of the line (a, b) along d in
// the fields F (the wall face of a walled line's last block is 0)
__device__ __forceinline__ void block_vec(const Geo<double>& g, const CF<double>& F, int d, int n, int cyc, int a, int b,
                                          int m, double v[3]) {
  int i, j, k;
  line_pos(d, a, b, m, i, j, k);
  int ic = IC(g, i, j, k);
  v[0] = F.f[0][ic];
  v[1] = F.f[4][ic];
  v[2] = 0.0;
  if (m < n - 1 || cyc) {
    int fi = i, fj = j, fk = k;
    if (d == 0) fi = m + 1; else if (d == 1) fj = m + 1; else fk = (m + 1 == n) ? 0 : m + 1;
    v[2] = F.f[1 + d][face_idx(g, d, fi, fj, fk)];
  }
}

// (2) -<mu_d, A_d(Ubar) x_d> over the block rows of the lines along D: one thread
// per cell of a line; the block row m of A_d is assembled by the forward's
// assemble_block on tape values.
template <int D>
__global__ void __launch_bounds__(128) k_adj_blk(AdjArgs A, int nl, int nb, int a0, int b0) {
  Tape T = make_tape(A);
  const Geo<double>& g = A.g;
  const Geo<ad> ga = geo_ad(g);
  const int n = D == 0 ? g.nr : D == 1 ? g.nt : g.np;
  const int cyc = (D == 2 && g.per);
  const long total = (long)nl * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    int line = (int)(e / n), m = (int)(e % n);
    int a = line / nb + a0, b = line % nb + b0;
    double mu[3];
    block_vec(g, A.mu[D], D, n, cyc, a, b, m, mu);
    if (mu[0] == 0.0 && mu[1] == 0.0 && mu[2] == 0.0) continue;
    double xm[3], x0[3], xp[3];
    block_vec(g, A.x[D], D, n, cyc, a, b, m, x0);
    int mp = m - 1, mn = m + 1;
    if (cyc) { mp = mp < 0 ? n - 1 : mp; mn = mn == n ? 0 : mn; }
    xm[0] = xm[1] = xm[2] = xp[0] = xp[1] = xp[2] = 0.0;
    if (mp >= 0) block_vec(g, A.x[D], D, n, cyc, a, b, mp, xm);
    if (mn < n) block_vec(g, A.x[D], D, n, cyc, a, b, mn, xp);
    T.n = 0;
    CF<ad> ub = leaves_ub(A, &T);
    Coef<ad> c = leaves_coef(A, &T);
    int i, j, k;
    line_pos(D, a, b, m, i, j, k);
    ad Ab[9], Bb[9], Cb[9];
    assemble_block(ga, A.P, c, ub, D, n, cyc, m, i, j, k, ad(0.5 * A.tau), Ab, Bb, Cb);
    ad psi;
    for (int r = 0; r < 3; r++) {
      if (mu[r] == 0.0) continue;
      ad y = ad(0.0);
      for (int q = 0; q < 3; q++) y += Ab[r * 3 + q] * xm[q] + Bb[r * 3 + q] * x0[q] + Cb[r * 3 + q] * xp[q];
      psi -= y * mu[r];
    }
    finish(A, T, psi);
  }
}

// (2') the same over the transverse scalar lines of kind KIND along D
template <int D, int KIND>
__global__ void __launch_bounds__(128) k_adj_sca(AdjArgs A, SweepArgs<double> S) {
  Tape T = make_tape(A);
  const Geo<double>& g = A.g;
  const Geo<ad> ga = geo_ad(g);
  constexpr int cc = trans_comp(D, KIND);
  const int n = D == 0 ? g.nr : D == 1 ? g.nt : g.np;
  const int cyc = (D == 2 && g.per);
  const int nl = S.nl[KIND], nb = S.nb[KIND], a0 = S.a0[KIND], b0 = S.b0[KIND];
  const long total = (long)nl * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    int line = (int)(e / n), m = (int)(e % n);
    int a = line / nb + a0, b = line % nb + b0;
    int i, j, k;
    line_pos(D, a, b, m, i, j, k);
    double mu = A.mu[D].f[1 + cc][face_idx(g, cc, i, j, k)];
    if (mu == 0.0) continue;
    const double* X = A.x[D].f[1 + cc];
    double x0 = X[face_idx(g, cc, i, j, k)], xm = 0.0, xp = 0.0;
    int mp = m - 1, mn = m + 1;
    if (cyc) { mp = mp < 0 ? n - 1 : mp; mn = mn == n ? 0 : mn; }
    if (mp >= 0) { int ii, jj, kk; line_pos(D, a, b, mp, ii, jj, kk); xm = X[face_idx(g, cc, ii, jj, kk)]; }
    if (mn < n) { int ii, jj, kk; line_pos(D, a, b, mn, ii, jj, kk); xp = X[face_idx(g, cc, ii, jj, kk)]; }
    T.n = 0;
    SweepArgs<ad> Sa;
    Sa.g = ga; Sa.P = A.P; Sa.c = leaves_coef(A, &T); Sa.ub = leaves_ub(A, &T); Sa.h = ad(0.5 * A.tau);
    ad am, bm, cm;
    scalar_row(Sa, cc, D, n, cyc, a, b, m, am, bm, cm);
    ad psi = -((am * xm + bm * x0 + cm * xp) * mu);
    finish(A, T, psi);
  }
}

// (3) the coefficient planes' adjoints back to Ubar: one thread per centre,
// <lam_coef, coef(Ubar)> through the forward's coef_at on tape values
__global__ void __launch_bounds__(128) k_adj_coef(AdjArgs A) {
  Tape T = make_tape(A);
  const Geo<double>& g = A.g;
  const Geo<ad> ga = geo_ad(g);
  const long total = (long)g.nr * g.nt * g.np;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    int t = (int)e;
    double w[NCOEF];
    bool any = false;
    for (int q = 0; q < NCOEF; q++) { w[q] = A.lam[5 + q][t]; any |= w[q] != 0.0; }
    if (!any) continue;
    int k = t % g.np, j = (t / g.np) % g.nt, i = t / (g.np * g.nt);
    T.n = 0;
    CF<ad> ub = leaves_ub(A, &T);
    CoefOut o;
    coef_at<2>(ga, A.P, ub, o, i, j, k, t);
    const Slot* sl[NCOEF] = {&o.Pb, &o.Tb, &o.rho, &o.drho, &o.beta, &o.uc0, &o.uc1, &o.uc2,
                             &o.grr, &o.gtt, &o.gpp, &o.srt, &o.srp, &o.stp, &o.dvr, &o.dvt, &o.dvp};
    ad psi;
    for (int q = 0; q < NCOEF; q++)
      if (w[q] != 0.0) psi += sl[q]->v * w[q];
    finish(A, T, psi);
  }
}

// y += s * x over n elements
__global__ void k_axpy(long n, double s, const double* __restrict__ x, double* __restrict__ y) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) y[e] += s * x[e];
}

}  // namespace adj
