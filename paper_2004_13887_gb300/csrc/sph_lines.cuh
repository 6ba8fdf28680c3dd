// sph_lines.cuh -- partitioned line solver for the sweeps of the mixed path.
//
// The sweeps solve (I + tau/2 D_d(Ubar)) x = rhs on every line along d (eqs.
// spl1-spl3): 3x3-block tridiagonal systems for (p, T, u_d) and scalar
// tridiagonal systems for the two transverse velocity components; periodic phi
// makes the phi lines cyclic.  Here a line of n = 32 P cells (P = 2, 4, 8) is
// solved by one warp: lane l owns the cells [l P, l P + P).
//
//  1. Each lane eliminates its interior cells t = 1..P-2 downwards in terms of
//     its first and last unknowns X_F = x_0, X_L = x_{P-1}:
//         x_t = g_t - E_t x_{t+1} - H_t X_F,
//     storing (E, g, H) for the back substitution, and folds them into two rows
//     of a reduced system in the unknowns (X_F, X_L) of all lanes.
//  2. The 64 reduced rows (2 per lane, ordered F_0, L_0, F_1, L_1, ...) are
//     block tridiagonal, cyclic when the line is; they are solved by parallel
//     cyclic reduction with warp shuffles: one step at row stride 1 pairs each
//     lane's rows with its neighbours', leaving two decoupled 32-row systems
//     (the F rows and the L rows), then steps at lane strides 1, 2, 4, 8 and a
//     final 2x2 elimination with the lane 16 away.
//  3. Each lane back-substitutes its interior.
//
// This is block Gaussian elimination in a permuted order: the matrices I + h D_d
// of the scheme have a positive definite symmetric part at the time steps used,
// a property their Schur complements keep, so no pivoting between blocks is
// needed -- the same assumption as the sequential block Thomas algorithm.
//
// A thread block holds NW = 32/P lines.  Their inputs are staged in shared
// memory with coalesced loads (the lines of one block are adjacent in phi for
// the r- and theta-sweeps, so 4 or 8 lines share each 32-byte sector; a phi
// line is contiguous), and the increments leave the same way.  The (E, g, H)
// factors of a block line live in the block's slot of a scratch buffer; they
// are read back within microseconds, so they are served by L2, and once the
// back substitution is done the slot's cache lines are discarded from L2
// (discard.global.L2) so that the dead factors are never written to DRAM.
#pragma once

namespace lines {

constexpr int LS = 33;        // shared-memory stride of one lane's chunk: 32 values + 1 pad
constexpr int FS = 32 * LS;   // shared-memory stride of one staged field
constexpr int NFB = 15;       // staged fields of a block line
constexpr int NFS = 4;        // staged fields of a scalar line
constexpr int NFAC = 21;      // E (9), g (3), H (9) per interior cell
constexpr unsigned FULL = 0xffffffffu;

// per-lane floats of a block-line factor slot: the first row, then (E, g, H) per interior cell
__host__ __device__ constexpr int slot_floats(int P) { return 30 + (P > 2 ? P - 2 : 0) * NFAC; }

// position in shared memory of cell c (of chunk length P) on line w
template <int P>
__device__ __forceinline__ int sidx(int w, int c) {
  return (c / P) * LS + (c % P) * (32 / P) + w;
}

// element e of a block's staging pass -> (line w, cell c): lines adjacent in
// memory (r, theta sweeps) put w fastest; contiguous lines (phi) put c fastest
template <int D, int P>
__device__ __forceinline__ void elem(int e, int& w, int& c) {
  constexpr int NW = 32 / P;
  if (D == 2) { c = e % (32 * P); w = e / (32 * P); }
  else { w = e % NW; c = e / NW; }
}

__device__ __forceinline__ void mm3(const float* X, const float* Y, float* Z) {
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int q = 0; q < 3; q++) Z[r * 3 + q] = X[r * 3] * Y[q] + X[r * 3 + 1] * Y[3 + q] + X[r * 3 + 2] * Y[6 + q];
}
__device__ __forceinline__ void mv3(const float* X, const float* y, float* z) {
#pragma unroll
  for (int r = 0; r < 3; r++) z[r] = X[r * 3] * y[0] + X[r * 3 + 1] * y[1] + X[r * 3 + 2] * y[2];
}

// A reduced block row with its diagonal block scaled to the identity,
//   A x_{i-s} + x_i + C x_{i+s} = r,
// stored as 21 floats: A (0-8), C (9-17), r (18-20).  Normalised rows are
// also exactly what a row's neighbours need from it.
constexpr int NR3 = 21;

template <int NS>
__device__ __forceinline__ void shfl_get(const float* s, float* o, int src, bool zero) {
#pragma unroll
  for (int q = 0; q < NS; q++) {
    float v = __shfl_sync(FULL, s[q], src);
    o[q] = zero ? 0.f : v;
  }
}

// X <- B^-1 (A, C, r)
__device__ __forceinline__ void normalise3(const float* A, const float* B, const float* C, const float* r, float* X,
                                           int* bad) {
  float Bi[9];
  if (!inv3(B, Bi)) *bad |= FLAG_SINGULAR;
  mm3(Bi, A, X);
  mm3(Bi, C, X + 9);
  mv3(Bi, r, X + 18);
}

// The reduction keeps each lane's two normalised rows in shared memory, in the
// lane's own staging slots (already consumed by then), double-buffered:
// buffer q, row f (0 = F, 1 = L), element z sits at value number
// zz = 42 q + 21 f + z of the lane's chunk, i.e. field zz / P, cell zz % P.
template <int P>
__device__ __forceinline__ int pz(int w, int lane, int zz) {
  return (zz / P) * FS + (zz % P) * (32 / P) + lane * LS + w;
}
// fields a block kernel stages: the inputs, or the two reduction buffers if more
__host__ __device__ constexpr int blk_fields(int P) { return NFB > (84 + P - 1) / P ? NFB : (84 + P - 1) / P; }

// New row from the normalised row X (own, base bx) and its lower / upper
// neighbours (lanes ll, lu, same or other family, bases bl, bu):
//   B = I - A_X C_lo - C_X A_up,  A' = -A_X A_lo,  C' = -C_X C_up,
//   r' = r_X - A_X r_lo - C_X r_up,
// renormalised and written to base bo of the own lane.  A missing neighbour
// (end of a non-cyclic line) counts as a zero row.
template <int P>
__device__ __forceinline__ void pcr3_row(float* sm, int w, int lane, int bx, int ll, bool lo_ok, int bl, int lu,
                                         bool up_ok, int bu, int bo, int* bad) {
  float XA[9], XC[9], B[9], An[9], Cn[9], rn[3];
#pragma unroll
  for (int q = 0; q < 9; q++) { XA[q] = sm[pz<P>(w, lane, bx + q)]; XC[q] = sm[pz<P>(w, lane, bx + 9 + q)]; }
#pragma unroll
  for (int q = 0; q < 3; q++) rn[q] = sm[pz<P>(w, lane, bx + 18 + q)];
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int q = 0; q < 3; q++) {
      float loA = 0.f, loC = 0.f, upA = 0.f, upC = 0.f;
      float b = (r == q) ? 1.f : 0.f, an = 0.f, cn = 0.f;
#pragma unroll
      for (int z = 0; z < 3; z++) {
        loA = lo_ok ? sm[pz<P>(w, ll, bl + z * 3 + q)] : 0.f;
        loC = lo_ok ? sm[pz<P>(w, ll, bl + 9 + z * 3 + q)] : 0.f;
        upA = up_ok ? sm[pz<P>(w, lu, bu + z * 3 + q)] : 0.f;
        upC = up_ok ? sm[pz<P>(w, lu, bu + 9 + z * 3 + q)] : 0.f;
        b -= XA[r * 3 + z] * loC + XC[r * 3 + z] * upA;
        an -= XA[r * 3 + z] * loA;
        cn -= XC[r * 3 + z] * upC;
      }
      B[r * 3 + q] = b; An[r * 3 + q] = an; Cn[r * 3 + q] = cn;
    }
#pragma unroll
  for (int z = 0; z < 3; z++) {
    float lr = lo_ok ? sm[pz<P>(w, ll, bl + 18 + z)] : 0.f;
    float ur = up_ok ? sm[pz<P>(w, lu, bu + 18 + z)] : 0.f;
#pragma unroll
    for (int r = 0; r < 3; r++) rn[r] -= XA[r * 3 + z] * lr + XC[r * 3 + z] * ur;
  }
  float Bi[9], t[9];
  if (!inv3(B, Bi)) *bad |= FLAG_SINGULAR;
  mm3(Bi, An, t);
#pragma unroll
  for (int q = 0; q < 9; q++) sm[pz<P>(w, lane, bo + q)] = t[q];
  mm3(Bi, Cn, t);
#pragma unroll
  for (int q = 0; q < 9; q++) sm[pz<P>(w, lane, bo + 9 + q)] = t[q];
  mv3(Bi, rn, t);
#pragma unroll
  for (int q = 0; q < 3; q++) sm[pz<P>(w, lane, bo + 18 + q)] = t[q];
}

// Parallel cyclic reduction of the 64-row reduced block system, two
// normalised rows per lane (F = row 2l, L = row 2l+1) in buffer 0; returns
// X_F, X_L.
template <int P>
__device__ __forceinline__ void pcr3(float* sm, int w, int lane, int cyc, float* xF, float* xL, int* bad) {
  constexpr int F0 = 0, L0 = 21, F1 = 42, L1 = 63;
  __syncwarp();
  // row stride 1: F's neighbours are lane-1's L and its own L; L's are its own F and lane+1's F
  pcr3_row<P>(sm, w, lane, F0, (lane + 31) & 31, cyc || lane > 0, L0, lane, true, L0, F1, bad);
  pcr3_row<P>(sm, w, lane, L0, lane, true, F0, (lane + 1) & 31, cyc || lane < 31, F0, L1, bad);
  __syncwarp();
  // two decoupled 32-row systems (the F rows and the L rows), lane strides 1..8
  int cur = 1;
#pragma unroll
  for (int s = 1; s < 16; s <<= 1) {
    int src = cur ? 42 : 0, dst = cur ? 0 : 42;
    int ll = (lane - s) & 31, lu = (lane + s) & 31;
    bool lo_ok = cyc || lane >= s, up_ok = cyc || lane + s <= 31;
    pcr3_row<P>(sm, w, lane, src, ll, lo_ok, src, lu, up_ok, src, dst, bad);
    pcr3_row<P>(sm, w, lane, src + 21, ll, lo_ok, src + 21, lu, up_ok, src + 21, dst + 21, bad);
    __syncwarp();
    cur ^= 1;
  }
  // each row now couples only to the row of lane ^ 16 (both sides of a cyclic
  // line meet there; on a non-cyclic line one of A, C is zero):
  //   x + M x_p = r,  x_p + M_p x = r_p  =>  (I - M M_p) x = r - M r_p
  int base = cur ? 42 : 0, pl = lane ^ 16;
#pragma unroll
  for (int f = 0; f < 2; f++) {
    int bx = base + 21 * f;
    float M[9], Mp[9], Sm[9], Si[9], rr[3];
#pragma unroll
    for (int q = 0; q < 9; q++) {
      M[q] = sm[pz<P>(w, lane, bx + q)] + sm[pz<P>(w, lane, bx + 9 + q)];
      Mp[q] = sm[pz<P>(w, pl, bx + q)] + sm[pz<P>(w, pl, bx + 9 + q)];
    }
    mm3(M, Mp, Sm);
#pragma unroll
    for (int q = 0; q < 9; q++) Sm[q] = (q % 4 == 0 ? 1.f : 0.f) - Sm[q];
#pragma unroll
    for (int r = 0; r < 3; r++)
      rr[r] = sm[pz<P>(w, lane, bx + 18 + r)] - (M[r * 3] * sm[pz<P>(w, pl, bx + 18)] +
                                                 M[r * 3 + 1] * sm[pz<P>(w, pl, bx + 19)] +
                                                 M[r * 3 + 2] * sm[pz<P>(w, pl, bx + 20)]);
    if (!inv3(Sm, Si)) *bad |= FLAG_SINGULAR;
    mv3(Si, rr, f == 0 ? xF : xL);
  }
  __syncwarp();
}

// scalar rows: (a, b, c, r); shares a/b, c/b, r/b
struct Row1 { float a, b, c, r; };

__device__ __forceinline__ void share1(const Row1& w, float* s, int* bad) {
  if (w.b == 0.f || !isfinite(w.b)) *bad |= FLAG_SINGULAR;
  float ib = sdiv(1.f, w.b);
  s[0] = w.a * ib; s[1] = w.c * ib; s[2] = w.r * ib;
}
__device__ __forceinline__ void combine1(Row1& w, const float* sL, const float* sU) {
  float an = -w.a * sL[0], cn = -w.c * sU[1];
  w.b -= w.a * sL[1] + w.c * sU[0];
  w.r -= w.a * sL[2] + w.c * sU[2];
  w.a = an; w.c = cn;
}

__device__ __forceinline__ void pcr1_final(const Row1& w, int lane, float* x, int* bad) {
  float M = w.a + w.c;
  if (w.b == 0.f || !isfinite(w.b)) *bad |= FLAG_SINGULAR;
  float ib = sdiv(1.f, w.b);
  float sh[2] = {M * ib, w.r * ib}, ph[2];
  shfl_get<2>(sh, ph, lane ^ 16, false);
  float den = w.b - M * ph[0];
  if (den == 0.f || !isfinite(den)) *bad |= FLAG_SINGULAR;
  *x = sdiv(w.r - M * ph[1], den);
}

__device__ __forceinline__ void pcr1(Row1& F, Row1& L, int lane, int cyc, float* xF, float* xL, int* bad) {
  float sF[3], sL[3], o[3], lo[3];
  share1(F, sF, bad);
  share1(L, sL, bad);
  shfl_get<3>(sL, o, (lane + 31) & 31, !cyc && lane == 0);
  combine1(F, o, sL);
  shfl_get<3>(sF, o, (lane + 1) & 31, !cyc && lane == 31);
  combine1(L, sF, o);
#pragma unroll 1
  for (int s = 1; s < 16; s <<= 1) {
    share1(F, sF, bad);
    share1(L, sL, bad);
    shfl_get<3>(sF, lo, (lane - s) & 31, !cyc && lane < s);
    shfl_get<3>(sF, o, (lane + s) & 31, !cyc && lane + s > 31);
    combine1(F, lo, o);
    shfl_get<3>(sL, lo, (lane - s) & 31, !cyc && lane < s);
    shfl_get<3>(sL, o, (lane + s) & 31, !cyc && lane + s > 31);
    combine1(L, lo, o);
  }
  pcr1_final(F, lane, xF, bad);
  pcr1_final(L, lane, xL, bad);
}

// ------------------------------------------------------------------ staging

// stage the inputs of block-line cell c of line (a, b) at shared index si
template <int D>
__device__ __forceinline__ void stage_block(const SweepArgs<float>& S, float* sm, int si, int a, int b, int c, int n,
                                            int cyc) {
  const Geo<float>& g = S.g;
  int i, j, k;
  line_pos(D, a, b, c, i, j, k);
  int ic = IC(g, i, j, k);
  CPt<float> q = load_c(S.c, D, ic);
  sm[0 * FS + si] = q.Pb; sm[1 * FS + si] = q.Tb; sm[2 * FS + si] = q.beta; sm[3 * FS + si] = q.uc;
  sm[4 * FS + si] = q.grr; sm[5 * FS + si] = q.gtt; sm[6 * FS + si] = q.gpp;
  if (D > 0) { sm[7 * FS + si] = q.s1; sm[8 * FS + si] = q.s2; }
  FPt<float> f = {1.f, 1.f, 0.f};
  float ru = 0.f;
  if (c < n - 1 || cyc) {
    int fi, fj, fk;
    next_face(D, n, c, i, j, k, fi, fj, fk);
    f = load_f(g, S.c, S.ub.f[1 + D], D, fi, fj, fk);
    ru = S.rhs.f[1 + D][face_idx(g, D, fi, fj, fk)];
  }
  sm[9 * FS + si] = f.rho0; sm[10 * FS + si] = f.rho1; sm[11 * FS + si] = f.ub;
  sm[12 * FS + si] = S.rhs.f[0][ic]; sm[13 * FS + si] = S.rhs.f[4][ic]; sm[14 * FS + si] = ru;
}

// stage the inputs of scalar-line cell c (component cc) of line (a, b)
template <int D, int KIND>
__device__ __forceinline__ void stage_scalar(const SweepArgs<float>& S, float* sm, int si, int a, int b, int c) {
  const Geo<float>& g = S.g;
  constexpr int cc = trans_comp(D, KIND);
  int i, j, k;
  line_pos(D, a, b, c, i, j, k);
  SPt<float> q = load_s(g, S.c, S.ub, cc, D, i, j, k);
  sm[0 * FS + si] = q.rho0; sm[1 * FS + si] = q.rho1; sm[2 * FS + si] = q.ua;
  sm[3 * FS + si] = S.rhs.f[1 + cc][face_idx(g, cc, i, j, k)];
}

// line group -> first line (a, bb) and the number of valid lines
struct Group { int a, bb, nvalid; };
__device__ __forceinline__ Group group_of(const SweepArgs<float>& S, int kind, int grp, int NW) {
  int nb = S.nb[kind];
  int nbg = (nb + NW - 1) / NW;
  Group G;
  G.a = S.a0[kind] + grp / nbg;
  int b_off = (grp % nbg) * NW;
  G.bb = S.b0[kind] + b_off;
  G.nvalid = min(NW, nb - b_off);
  return G;
}

__device__ __forceinline__ void flush_norms(const SweepArgs<float>& S, double* ss, int bad) {
  if (bad) atomicOr(S.flag, bad);
  if (S.update) {
#pragma unroll
    for (int f = 0; f < 5; f++) {
      double v = ss[f];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
      if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(S.acc + f, v);
    }
  }
}

// ------------------------------------------------------------------ kernels

// Block lines (p, T, u_D) of direction D, n = 32 P cells per line.
template <int D, int P>
__global__ void __launch_bounds__(1024 / P, P == 8 ? 3 : P == 4 ? 2 : 1) k_lines_blk(SweepArgs<float> S) {
  constexpr int NW = 32 / P;
  constexpr int NT = 32 * NW;
  extern __shared__ float sm[];
  const Geo<float>& g = S.g;
  const int n = 32 * P, cyc = (D == 2 && g.per);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float h = S.h;
  double ss[5] = {0, 0, 0, 0, 0};
  int bad = 0;
  float* slot = S.scr + ((size_t)blockIdx.x * NW + w) * (32 * slot_floats(P));
  {
    Group G = group_of(S, 0, blockIdx.x, NW);
    // 1. stage
    for (int e = threadIdx.x; e < n * NW; e += NT) {
      int lw, c;
      elem<D, P>(e, lw, c);
      if (lw < G.nvalid) stage_block<D>(S, sm, sidx<P>(lw, c), G.a, G.bb + lw, c, n, cyc);
    }
    __syncthreads();
    if (w < G.nvalid) {
      // 2. chunk elimination.  The slot holds the raw first row (30 floats)
      // then (E, g, H) of each interior cell, lane-interleaved.
      float Lr[30];           // last row: A (0-8), B (9-17), C (18-26), r (27-29)
      float E[9], gg[3], H[9];
      int a = G.a, b = G.bb + w;
#pragma unroll 1
      for (int t = 0; t < P; t++) {
        int m = lane * P + t;
        int si = sidx<P>(w, m);
        CPt<float> cq;
        cq.Pb = sm[0 * FS + si]; cq.Tb = sm[1 * FS + si]; cq.beta = sm[2 * FS + si]; cq.uc = sm[3 * FS + si];
        cq.grr = sm[4 * FS + si]; cq.gtt = sm[5 * FS + si]; cq.gpp = sm[6 * FS + si];
        cq.s1 = D > 0 ? sm[7 * FS + si] : 0.f;
        cq.s2 = D > 0 ? sm[8 * FS + si] : 0.f;
        FPt<float> fq = {sm[9 * FS + si], sm[10 * FS + si], sm[11 * FS + si]};
        float rr[3] = {sm[12 * FS + si], sm[13 * FS + si], sm[14 * FS + si]};
        int i, j, k, fi, fj, fk;
        line_pos(D, a, b, m, i, j, k);
        next_face(D, n, m, i, j, k, fi, fj, fk);
        float A[9], B[9], C[9];
        assemble_pts(g, S.P, cq, fq, D, n, cyc, m, i, j, fi, fj, h, A, B, C);
        if (t == 0) {
          float* s = slot + lane;
#pragma unroll
          for (int q = 0; q < 9; q++) { s[q * 32] = A[q]; s[(9 + q) * 32] = B[q]; s[(18 + q) * 32] = C[q]; }
#pragma unroll
          for (int q = 0; q < 3; q++) s[(27 + q) * 32] = rr[q];
        } else if (t < P - 1) {
          float Sm[9], rv[3], Hs[9], Si[9];
          if (t == 1) {
#pragma unroll
            for (int q = 0; q < 9; q++) { Sm[q] = B[q]; Hs[q] = A[q]; }
#pragma unroll
            for (int q = 0; q < 3; q++) rv[q] = rr[q];
          } else {
            float T9[9], u[3];
            mm3(A, E, T9);
#pragma unroll
            for (int q = 0; q < 9; q++) Sm[q] = B[q] - T9[q];
            mv3(A, gg, u);
#pragma unroll
            for (int q = 0; q < 3; q++) rv[q] = rr[q] - u[q];
            mm3(A, H, T9);
#pragma unroll
            for (int q = 0; q < 9; q++) Hs[q] = -T9[q];
          }
          if (!inv3(Sm, Si)) bad |= FLAG_SINGULAR;
          mm3(Si, C, E);
          mv3(Si, rv, gg);
          mm3(Si, Hs, H);
          float* s = slot + (30 + (t - 1) * NFAC) * 32 + lane;
#pragma unroll
          for (int q = 0; q < 9; q++) s[q * 32] = E[q];
#pragma unroll
          for (int q = 0; q < 3; q++) s[(9 + q) * 32] = gg[q];
#pragma unroll
          for (int q = 0; q < 9; q++) s[(12 + q) * 32] = H[q];
        } else if (P == 2) {
#pragma unroll
          for (int q = 0; q < 9; q++) { Lr[q] = A[q]; Lr[9 + q] = B[q]; Lr[18 + q] = C[q]; }
#pragma unroll
          for (int q = 0; q < 3; q++) Lr[27 + q] = rr[q];
        } else {
          float T9[9], u[3];
          mm3(A, H, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) Lr[q] = -T9[q];
          mm3(A, E, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) { Lr[9 + q] = B[q] - T9[q]; Lr[18 + q] = C[q]; }
          mv3(A, gg, u);
#pragma unroll
          for (int q = 0; q < 3; q++) Lr[27 + q] = rr[q] - u[q];
        }
      }
      float Ln[NR3];
      normalise3(Lr, Lr + 9, Lr + 18, Lr + 27, Ln, &bad);
#pragma unroll
      for (int q = 0; q < NR3; q++) sm[pz<P>(w, lane, 21 + q)] = Ln[q];
      // fold the interior into the first row: x_1 = p + Q X_L + W X_F
      {
        float Fr[30];
        const float* s0 = slot + lane;
#pragma unroll
        for (int q = 0; q < 30; q++) Fr[q] = s0[q * 32];
        if (P > 2) {
          float p[3], Q[9], W[9];
#pragma unroll
          for (int q = 0; q < 3; q++) p[q] = gg[q];
#pragma unroll
          for (int q = 0; q < 9; q++) { Q[q] = -E[q]; W[q] = -H[q]; }
#pragma unroll 1
          for (int t = P - 3; t >= 1; t--) {
            const float* s = slot + (30 + (t - 1) * NFAC) * 32 + lane;
            float Et[9], gt[3], Ht[9], T9[9], u[3];
#pragma unroll
            for (int q = 0; q < 9; q++) Et[q] = s[q * 32];
#pragma unroll
            for (int q = 0; q < 3; q++) gt[q] = s[(9 + q) * 32];
#pragma unroll
            for (int q = 0; q < 9; q++) Ht[q] = s[(12 + q) * 32];
            mv3(Et, p, u);
#pragma unroll
            for (int q = 0; q < 3; q++) p[q] = gt[q] - u[q];
            mm3(Et, Q, T9);
#pragma unroll
            for (int q = 0; q < 9; q++) Q[q] = -T9[q];
            mm3(Et, W, T9);
#pragma unroll
            for (int q = 0; q < 9; q++) W[q] = -Ht[q] - T9[q];
          }
          float T9[9], u[3];
          mm3(Fr + 18, W, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) Fr[9 + q] += T9[q];
          mv3(Fr + 18, p, u);
#pragma unroll
          for (int q = 0; q < 3; q++) Fr[27 + q] -= u[q];
          mm3(Fr + 18, Q, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) Fr[18 + q] = T9[q];
        }
        float Fn[NR3];
        normalise3(Fr, Fr + 9, Fr + 18, Fr + 27, Fn, &bad);
#pragma unroll
        for (int q = 0; q < NR3; q++) sm[pz<P>(w, lane, q)] = Fn[q];
      }
      // 3. reduced system
      float xF[3], xL[3];
      pcr3<P>(sm, w, lane, cyc, xF, xL, &bad);
      // 4. back substitution; each warp writes its increments over its own
      // staged inputs (fields 0-2), which only it reads
      float xn[3] = {xL[0], xL[1], xL[2]};
      int sl = sidx<P>(w, lane * P + P - 1);
#pragma unroll
      for (int q = 0; q < 3; q++) sm[q * FS + sl] = xL[q];
#pragma unroll 1
      for (int t = P - 2; t >= 1; t--) {
        const float* s = slot + (30 + (t - 1) * NFAC) * 32 + lane;
        float Et[9], gt[3], Ht[9], u[3], v[3];
#pragma unroll
        for (int q = 0; q < 9; q++) Et[q] = s[q * 32];
#pragma unroll
        for (int q = 0; q < 3; q++) gt[q] = s[(9 + q) * 32];
#pragma unroll
        for (int q = 0; q < 9; q++) Ht[q] = s[(12 + q) * 32];
        mv3(Et, xn, u);
        mv3(Ht, xF, v);
        int st = sidx<P>(w, lane * P + t);
#pragma unroll
        for (int q = 0; q < 3; q++) {
          xn[q] = gt[q] - u[q] - v[q];
          sm[q * FS + st] = xn[q];
        }
      }
      int s0 = sidx<P>(w, lane * P);
#pragma unroll
      for (int q = 0; q < 3; q++) sm[q * FS + s0] = xF[q];
      // the slot is dead: drop its lines from L2 without writing them back
      __syncwarp();
      for (int q = lane; q < slot_floats(P); q += 32)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(slot + q * 32) : "memory");
    }
    __syncthreads();
    // 5. write back (coalesced like the staging)
    for (int e = threadIdx.x; e < n * NW; e += NT) {
      int lw, c;
      elem<D, P>(e, lw, c);
      if (lw >= G.nvalid) continue;
      int si = sidx<P>(lw, c);
      int i, j, k;
      line_pos(D, G.a, G.bb + lw, c, i, j, k);
      int ic = IC(g, i, j, k);
      put(S, 0, ic, (double)sm[si], ss, &bad);
      put(S, 4, ic, (double)sm[FS + si], ss, &bad);
      int fi, fj, fk;
      next_face(D, n, c, i, j, k, fi, fj, fk);
      if (c < n - 1 || cyc) {
        put(S, 1 + D, face_idx(g, D, fi, fj, fk), (double)sm[2 * FS + si], ss, &bad);
      } else {
        put_wall(S, 1 + D, face_idx(g, D, fi, fj, fk));
      }
      if (c == 0 && !cyc) {
        int wi = i, wj = j, wk = k;
        if (D == 0) wi = 0; else if (D == 1) wj = 0; else wk = 0;
        put_wall(S, 1 + D, face_idx(g, D, wi, wj, wk));
      }
    }
    __syncthreads();
  }
  flush_norms(S, ss, bad);
}

// Scalar lines of the transverse component trans_comp(D, KIND), n = 32 P.
template <int D, int P, int KIND>
__global__ void __launch_bounds__(1024 / P) k_lines_sca(SweepArgs<float> S) {
  constexpr int NW = 32 / P;
  constexpr int NT = 32 * NW;
  constexpr int cc = trans_comp(D, KIND);
  extern __shared__ float sm[];
  const Geo<float>& g = S.g;
  const int n = 32 * P, cyc = (D == 2 && g.per);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float h = S.h;
  double ss[5] = {0, 0, 0, 0, 0};
  int bad = 0;
  {
    Group G = group_of(S, KIND, blockIdx.x, NW);
    for (int e = threadIdx.x; e < n * NW; e += NT) {
      int lw, c;
      elem<D, P>(e, lw, c);
      if (lw < G.nvalid) stage_scalar<D, KIND>(S, sm, sidx<P>(lw, c), G.a, G.bb + lw, c);
    }
    __syncthreads();
    float xo[P];
    if (w < G.nvalid) {
      int a = G.a, b = G.bb + w;
      Row1 F, L;
      float e_[P > 2 ? P - 2 : 1], g_[P > 2 ? P - 2 : 1], h_[P > 2 ? P - 2 : 1];
      float ep = 0.f, gp = 0.f, hp_ = 0.f;
#pragma unroll
      for (int t = 0; t < P; t++) {
        int m = lane * P + t;
        int si = sidx<P>(w, m);
        SPt<float> q = {sm[si], sm[FS + si], sm[2 * FS + si]};
        float r = sm[3 * FS + si];
        int i, j, k;
        line_pos(D, a, b, m, i, j, k);
        float wt[3];
        row_sw(g, S.P, q, cc, D, i, j, wt);
        float am = h * wt[0], bm = 1.f + h * wt[1], cm = h * wt[2];
        if (!cyc) {
          if (m == 0) { bm -= am; am = 0.f; }
          if (m == n - 1) { bm -= cm; cm = 0.f; }
        }
        if (t == 0) {
          F.a = am; F.b = bm; F.c = cm; F.r = r;
        } else if (t < P - 1) {
          float sden = t == 1 ? bm : bm - am * ep;
          float rv = t == 1 ? r : r - am * gp;
          float hs = t == 1 ? am : -am * hp_;
          if (sden == 0.f || !isfinite(sden)) bad |= FLAG_SINGULAR;
          float is = sdiv(1.f, sden);
          ep = cm * is; gp = rv * is; hp_ = hs * is;
          e_[t - 1] = ep; g_[t - 1] = gp; h_[t - 1] = hp_;
        } else {
          if (P == 2) { L.a = am; L.b = bm; L.c = cm; L.r = r; }
          else { L.a = -am * hp_; L.b = bm - am * ep; L.c = cm; L.r = r - am * gp; }
        }
      }
      if (P > 2) {
        float p = gp, Q = -ep, W = -hp_;
#pragma unroll
        for (int t = P - 3; t >= 1; t--) {
          p = g_[t - 1] - e_[t - 1] * p;
          Q = -e_[t - 1] * Q;
          W = -h_[t - 1] - e_[t - 1] * W;
        }
        F.b += F.c * W;
        F.r -= F.c * p;
        F.c = F.c * Q;
      }
      float xF, xL;
      pcr1(F, L, lane, cyc, &xF, &xL, &bad);
      xo[0] = xF;
      xo[P - 1] = xL;
#pragma unroll
      for (int t = P - 2; t >= 1; t--) xo[t] = g_[t - 1] - e_[t - 1] * xo[t + 1] - h_[t - 1] * xF;
    }
    __syncthreads();
    if (w < G.nvalid) {
#pragma unroll
      for (int t = 0; t < P; t++) sm[sidx<P>(w, lane * P + t)] = xo[t];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * NW; e += NT) {
      int lw, c;
      elem<D, P>(e, lw, c);
      if (lw >= G.nvalid) continue;
      int i, j, k;
      line_pos(D, G.a, G.bb + lw, c, i, j, k);
      scalar_put(S, cc, i, j, k, (double)sm[sidx<P>(lw, c)], ss, &bad);
    }
    __syncthreads();
  }
  flush_norms(S, ss, bad);
}

}  // namespace lines
