// sph_lines.cuh -- partitioned line solver for the sweeps of the mixed path.
//
// The sweeps solve (I + tau/2 D_d(Ubar)) x = rhs on every line along d (eqs.
// spl1-spl3): 3x3-block tridiagonal systems for (p, T, u_d) and scalar
// tridiagonal systems for the two transverse velocity components; periodic phi
// makes the phi lines cyclic.  Here a line of n = L P cells is solved by a
// segment of L lanes (L = 32, or 16, 8, 4 with 2, 4, 8 lines per warp, or 64
// and 128 over several warps; P = 1 to 8): lane l owns the cells
// [l P, l P + P), and its last cell s_l = l P + P - 1 is a separator.
//
//  1. Each lane eliminates its interior cells t = 0..P-2 downwards, treating
//     the separator before its chunk (s_{l-1}, lane l-1's) as a parameter:
//         x_t = g_t - E_t x_{t+1} - H_t X_{l-1},
//     storing (E, g, H), and carries along the expression of its first
//     interior cell through the next unknown, x_0 = p + Q x_{t+1} + W X_{l-1}
//     (p += Q g_t, W -= Q H_t, Q = -Q E_t), which after the last interior cell
//     is x_0 = p + Q X_l + W X_{l-1}.
//  2. Separator row l, with x_{s-1} from its own chunk and x_{s+1} from lane
//     l+1's (p_0, Q_0, W_0), couples only X_{l-1}, X_l, X_{l+1}: an L-row block
//     tridiagonal system (cyclic when the line is), solved by parallel cyclic
//     reduction with warp shuffles, on rows scaled to an identity diagonal:
//     steps at lane strides 1, 2, .., L/4, then a 2x2 elimination with lane
//     l ^ L/2.  Fewer lanes per line mean longer chunks and one reduction step
//     less: less reduction work per cell.
//  3. Each lane back-substitutes its interior with X_l and X_{l-1}.
//
// This is block Gaussian elimination in a permuted order (the separators
// last): the matrices I + h D_d of the scheme have a positive definite
// symmetric part at the time steps used, a property their Schur complements
// keep, so no pivoting between blocks is needed -- the same assumption as the
// sequential block Thomas algorithm.
//
// A thread block holds NW = CB/n lines of CB cells.  Their inputs are staged
// in shared memory with coalesced loads (the lines of one block are adjacent in
// phi for the r- and theta-sweeps; CB = 2048 for lines of 256 cells there, so
// that 8 lines fill each 32-byte sector, else 1024; a phi line is contiguous),
// and the increments leave the same way.  The (E, g, H)
// factors of a warp's lines live in the warp's slot of a scratch buffer; they
// are read back within microseconds, so they are served by L2, and once the
// back substitution is done the slot's cache lines are discarded from L2
// (discard.global.L2) so that the dead factors are never written to DRAM.
#pragma once

namespace lines {

constexpr int NFB = 11;       // staged fields of a block line
constexpr int NFS = 5;        // staged fields of a scalar line
constexpr int NFAC = 21;      // E (9), g (3), H (9) per interior cell
constexpr int NR3 = 21;       // a normalised reduced row: A (0-8), C (9-17), r (18-20)
constexpr unsigned FULL = 0xffffffffu;

// per-lane floats of a block-line factor slot: (E, g, H) per interior cell
// (none for chunks of one cell, which have no interior)
__host__ __device__ constexpr int slot_floats(int P) { return (P > 1 ? P - 1 : 0) * NFAC; }

// Shape of a launch: lines of n = L P cells, L lanes per line (4, 8, 16 or 32,
// or 64 and 128 for lines spanning 2 and 4 warps), P cells per lane; a block
// holds NW lines and CB of their cells (NT = CB / P threads, NWW warps; thread
// w L + l takes lane l of block line w).  In shared memory each staged field
// is 32 rows of CB/32 values and one word of padding (LS), FS floats in all.
template <int P, int L, int CB>
struct Shape {
  static constexpr int n = L * P, NW = CB / n, NT = CB / P, NWW = NT / 32;
  static constexpr int LS = CB / 32 + 1, FS = 32 * LS;
};

// position in shared memory of cell c on block line w: the chunk of each
// thread is spread over its lane's padded row, so that the lanes of a warp
// reading one cell each of their chunks hit 32 distinct banks
template <int P, int L, int CB>
__device__ __forceinline__ int sidx(int w, int c) {
  using S = Shape<P, L, CB>;
  const int tid = w * L + c / P;
  return (tid % 32) * S::LS + (c % P) * S::NWW + tid / 32;
}

// element e of a block's staging pass -> (line w, cell c): lines adjacent in
// memory (r, theta sweeps) put w fastest; contiguous lines (phi) put c fastest
template <int D, int P, int L, int CB>
__device__ __forceinline__ void elem(int e, int& w, int& c) {
  using S = Shape<P, L, CB>;
  if (D == 2) { c = e % S::n; w = e / S::n; }
  else { w = e % S::NW; c = e / S::NW; }
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

// Products with the two sparse blocks of a line row.  The lower block A is
// upper triangular (A[3] = A[6] = A[7] = 0: the T row does not see p_{m-1} and
// the u row sees only u on face m); the upper block C has C[2] = C[3] = C[5] =
// C[7] = 0 (the p and T rows see u only on the cell's own faces, the T row no
// p_{m+1}, the u row no T_{m+1}).  Boundary folding only zeroes more entries.
__device__ __forceinline__ void mm3_A(const float* A, const float* Y, float* Z) {  // A Y
#pragma unroll
  for (int q = 0; q < 3; q++) {
    Z[q] = A[0] * Y[q] + A[1] * Y[3 + q] + A[2] * Y[6 + q];
    Z[3 + q] = A[4] * Y[3 + q] + A[5] * Y[6 + q];
    Z[6 + q] = A[8] * Y[6 + q];
  }
}
__device__ __forceinline__ void mv3_A(const float* A, const float* y, float* z) {
  z[0] = A[0] * y[0] + A[1] * y[1] + A[2] * y[2];
  z[1] = A[4] * y[1] + A[5] * y[2];
  z[2] = A[8] * y[2];
}
__device__ __forceinline__ void mm3_C(const float* C, const float* Y, float* Z) {  // C Y
#pragma unroll
  for (int q = 0; q < 3; q++) {
    Z[q] = C[0] * Y[q] + C[1] * Y[3 + q];
    Z[3 + q] = C[4] * Y[3 + q];
    Z[6 + q] = C[6] * Y[q] + C[8] * Y[6 + q];
  }
}
__device__ __forceinline__ void mv3_C(const float* C, const float* y, float* z) {
  z[0] = C[0] * y[0] + C[1] * y[1];
  z[1] = C[4] * y[1];
  z[2] = C[6] * y[0] + C[8] * y[2];
}
__device__ __forceinline__ void mm3_XC(const float* X, const float* C, float* Z) {  // X C
#pragma unroll
  for (int r = 0; r < 3; r++) {
    Z[r * 3] = X[r * 3] * C[0] + X[r * 3 + 2] * C[6];
    Z[r * 3 + 1] = X[r * 3] * C[1] + X[r * 3 + 1] * C[4];
    Z[r * 3 + 2] = X[r * 3 + 2] * C[8];
  }
}

// o = s of lane src of this lane's segment of L lanes (zero when `zero`)
template <int NS, int L = 32>
__device__ __forceinline__ void shfl_get(const float* s, float* o, int src, bool zero) {
#pragma unroll
  for (int q = 0; q < NS; q++) {
    float v = __shfl_sync(FULL, s[q], src, L);
    o[q] = zero ? 0.f : v;
  }
}

// The same for any L: a line of more than 32 lanes spans several warps, and its
// lanes exchange through the shared buffer xb (NS x blockDim.x floats; every
// thread of the block takes part, between two block barriers).
template <int NS, int L>
__device__ __forceinline__ void xget(const float* s, float* o, int src, bool zero, float* xb) {
  if constexpr (L <= 32) {
    shfl_get<NS, L>(s, o, src, zero);
  } else {
    const int nt = blockDim.x, tid = threadIdx.x, base = tid - tid % L;
#pragma unroll
    for (int q = 0; q < NS; q++) xb[q * nt + tid] = s[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NS; q++) {
      float v = xb[q * nt + base + src];
      o[q] = zero ? 0.f : v;
    }
    __syncthreads();
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

// Parallel cyclic reduction of the L-row reduced block system (L = 32 or 16),
// one row per lane of the line's segment, normalised (A x_{l-s} + x_l +
// C x_{l+s} = r).  A step with stride s eliminates x_{l-s} and x_{l+s} with
// the rows of lanes l -+ s:
//   B = I - A C_lo - C A_up,  A' = -A A_lo,  C' = -C C_up,
//   r' = r - A r_lo - C r_up,
// then renormalises; a missing neighbour (end of a non-cyclic line) is a zero
// row.  After strides 1, 2, .., L/4 every row couples only to the row of lane
// l ^ L/2 (both sides of a cyclic line meet there; on a non-cyclic line one of
// A, C is zero):  x + M x_p = r,  x_p + M_p x = r_p  =>  (I - M M_p) x = r - M r_p.
template <int L>
__device__ __forceinline__ void pcr3(float* X, int lane, int cyc, float* x, int* bad, float* xb) {
#pragma unroll 1
  for (int s = 1; s < L / 2; s <<= 1) {
    float o[NR3], A[9], B[9], C[9], r[3], t[9], u[3];
    xget<NR3, L>(X, o, (lane - s) & (L - 1), !cyc && lane < s, xb);
    mm3(X, o + 9, t);
#pragma unroll
    for (int q = 0; q < 9; q++) B[q] = (q % 4 == 0 ? 1.f : 0.f) - t[q];
    mm3(X, o, t);
#pragma unroll
    for (int q = 0; q < 9; q++) A[q] = -t[q];
    mv3(X, o + 18, u);
#pragma unroll
    for (int q = 0; q < 3; q++) r[q] = X[18 + q] - u[q];
    xget<NR3, L>(X, o, (lane + s) & (L - 1), !cyc && lane + s > L - 1, xb);
    mm3(X + 9, o, t);
#pragma unroll
    for (int q = 0; q < 9; q++) B[q] -= t[q];
    mm3(X + 9, o + 9, t);
#pragma unroll
    for (int q = 0; q < 9; q++) C[q] = -t[q];
    mv3(X + 9, o + 18, u);
#pragma unroll
    for (int q = 0; q < 3; q++) r[q] -= u[q];
    normalise3(A, B, C, r, X, bad);
  }
  float M[12], ph[12];
#pragma unroll
  for (int z = 0; z < 9; z++) M[z] = X[z] + X[9 + z];
#pragma unroll
  for (int z = 0; z < 3; z++) M[9 + z] = X[18 + z];
  xget<12, L>(M, ph, lane ^ (L / 2), false, xb);
  float Sm[9], Si[9], rr[3], u[3];
  mm3(M, ph, Sm);
#pragma unroll
  for (int z = 0; z < 9; z++) Sm[z] = (z % 4 == 0 ? 1.f : 0.f) - Sm[z];
  mv3(M, ph + 9, u);
#pragma unroll
  for (int z = 0; z < 3; z++) rr[z] = X[18 + z] - u[z];
  if (!inv3(Sm, Si)) *bad |= FLAG_SINGULAR;
  mv3(Si, rr, x);
}

// The same for the scalar reduced system (a x_{l-s} + x_l + c x_{l+s} = r).
template <int L>
__device__ __forceinline__ float pcr1(float a, float c, float r, int lane, int cyc, int* bad, float* xb) {
#pragma unroll 1
  for (int s = 1; s < L / 2; s <<= 1) {
    float v[3] = {a, c, r}, lv[3], uv[3];
    xget<3, L>(v, lv, (lane - s) & (L - 1), !cyc && lane < s, xb);
    xget<3, L>(v, uv, (lane + s) & (L - 1), !cyc && lane + s > L - 1, xb);
    float la = lv[0], lc = lv[1], lr = lv[2], ua = uv[0], uc = uv[1], ur = uv[2];
    float b = 1.f - a * lc - c * ua;
    if (b == 0.f || !isfinite(b)) *bad |= FLAG_SINGULAR;
    float ib = sdiv(1.f, b);
    float an = -a * la * ib, cn = -c * uc * ib;
    r = (r - a * lr - c * ur) * ib;
    a = an; c = cn;
  }
  float M = a + c;
  float mr[2] = {M, r}, pr[2];
  xget<2, L>(mr, pr, lane ^ (L / 2), false, xb);
  float Mp = pr[0], rp = pr[1];
  float den = 1.f - M * Mp;
  if (den == 0.f || !isfinite(den)) *bad |= FLAG_SINGULAR;
  return sdiv(r - M * rp, den);
}

// ------------------------------------------------------------------ staging

// 4-byte asynchronous copy global -> shared (no register holds the value, so a
// thread keeps all its staging copies in flight at once)
__device__ __forceinline__ void cpa4(float* dst, const float* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// stage the inputs of block-line cell c of line (a, b) at shared index si:
// Ubar's p' and T' (the thermodynamic coefficients follow from them), the
// velocity-gradient coefficients, Ubar's u_D on face c+1 (the centre velocity
// is the mean of the cell's two faces) and the three right-hand-side values
// (the last face of a walled line has no row: zero)
template <int D, int FS>
__device__ __forceinline__ void stage_block(const SweepArgs<float>& S, float* sm, int si, int a, int b, int c, int n,
                                            int cyc) {
  const Geo<float>& g = S.g;
  const Coef<float>& C = S.c;
  int i, j, k;
  line_pos(D, a, b, c, i, j, k);
  int ic = IC(g, i, j, k);
  cpa4(sm + 0 * FS + si, S.ub.f[0] + ic); cpa4(sm + 1 * FS + si, S.ub.f[4] + ic);
  cpa4(sm + 2 * FS + si, C.grr + ic); cpa4(sm + 3 * FS + si, C.gtt + ic); cpa4(sm + 4 * FS + si, C.gpp + ic);
  if (D == 1) { cpa4(sm + 5 * FS + si, C.srt + ic); sm[6 * FS + si] = 0.f; }
  if (D == 2) { cpa4(sm + 5 * FS + si, C.srp + ic); cpa4(sm + 6 * FS + si, C.stp + ic); }
  int fi, fj, fk;
  next_face(D, n, c, i, j, k, fi, fj, fk);
  int f = face_idx(g, D, fi, fj, fk);
  cpa4(sm + 7 * FS + si, S.ub.f[1 + D] + f);
  if (c < n - 1 || cyc) cpa4(sm + 10 * FS + si, S.rhs.f[1 + D] + f);
  else sm[10 * FS + si] = 0.f;
  cpa4(sm + 8 * FS + si, S.rhs.f[0] + ic);
  cpa4(sm + 9 * FS + si, S.rhs.f[4] + ic);
}

// stage the inputs of scalar-line cell c (component cc, on its face (i, j, k))
// of line (a, b): rho at the face's two centres (fields 0, 1), the advecting
// velocity u_D at those centres (fields 2, 3; the row takes their mean) and the
// right-hand side (field 4).  Away from the r and theta walls these are plain
// reads of the coefficient planes, copied asynchronously like the block
// lines' inputs; next to them the checked accessors give rho and the mean,
// which is stored twice (its mean is itself).
// the checked-accessor path of stage_scalar (cells next to the r and theta
// walls), out of line: inlined into the unrolled staging loop its wall-data
// branches would crowd the 48-register budget of the scalar kernels
template <int D, int KIND>
__device__ __noinline__ SPt<float> stage_scalar_edge(const SweepArgs<float>& S, int i, int j, int k) {
  return load_s<2>(S.g, S.c, S.ub, trans_comp(D, KIND), D, i, j, k);
}

template <int D, int KIND, int FS>
__device__ __forceinline__ void stage_scalar(const SweepArgs<float>& S, float* sm, int si, int a, int b, int c) {
  const Geo<float>& g = S.g;
  constexpr int cc = trans_comp(D, KIND);
  int i, j, k;
  line_pos(D, a, b, c, i, j, k);
  if (inner_ij(g, i, j)) {
    int i0 = i - (cc == 0), j0 = j - (cc == 1), k0 = k - (cc == 2);
    if (cc == 2 && g.per) k0 = wrapk(g, k0);  // k0 = -1 only on a periodic line
    const int c0 = IC(g, i0, j0, k0), c1 = IC(g, i, j, k);
    const float* ua = D == 0 ? S.c.uc0 : D == 1 ? S.c.uc1 : S.c.uc2;
    cpa4(sm + 0 * FS + si, S.c.rho + c0); cpa4(sm + 1 * FS + si, S.c.rho + c1);
    cpa4(sm + 2 * FS + si, ua + c0); cpa4(sm + 3 * FS + si, ua + c1);
  } else {
    SPt<float> q = stage_scalar_edge<D, KIND>(S, i, j, k);
    sm[0 * FS + si] = q.rho0; sm[1 * FS + si] = q.rho1; sm[2 * FS + si] = q.ua; sm[3 * FS + si] = q.ua;
  }
  cpa4(sm + 4 * FS + si, S.rhs.f[1 + cc] + face_idx(g, cc, i, j, k));
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

template <typename Acc>
__device__ __forceinline__ void flush_norms(const SweepArgs<float>& S, const Acc& ss, int bad) {
  if (bad) atomicOr(S.flag, bad);
  if (S.update) {
#pragma unroll
    for (int f = 0; f < 5; f++) {
      double v = ss.warp_total(f);
      if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(S.acc + f, v);
    }
  }
}

// ------------------------------------------------------------------ kernels
// ------------------------------------------------------------------ kernels

// Block lines (p, T, u_D) of direction D, n = L P cells per line, L lanes per
// line, CB cells per block: line group grp (k_lines_blk below, or a batched
// launch over many problems).
template <int D, int P, int L, int CB>
__device__ __forceinline__ void lines_blk(const SweepArgs<float>& S, int grp) {
  using SH = Shape<P, L, CB>;
  constexpr int NW = SH::NW, NT = SH::NT, FS = SH::FS;
  extern __shared__ float sm[];
  const Geo<float>& g = S.g;
  const int n = SH::n, cyc = (D == 2 && g.per);
  const int wid = threadIdx.x >> 5, wl = threadIdx.x & 31;  // warp, lane of the warp
  const int w = threadIdx.x / L, lane = threadIdx.x % L;    // block line, lane of the line
  const float h = S.h;
  SqSum<float> ss;
  int bad = 0;
  float* slot = S.scr + ((size_t)grp * SH::NWW + wid) * (32 * slot_floats(P));
  float* xb = sm + 3 * FS;  // lane exchanges of lines longer than a warp (after the elimination)
  Group G = group_of(S, 0, grp, NW);
  // 1. stage (n NW = P NT elements: P per thread, all copies in flight).  The
  // block lines past the group's last repeat it, so that every lane of a warp
  // solves a well-posed line; their results are not written back.
#pragma unroll
  for (int q = 0; q < P; q++) {
    int lw, c;
    elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
    stage_block<D, FS>(S, sm, sidx<P, L, CB>(lw, c), G.a, G.bb + min(lw, G.nvalid - 1), c, n, cyc);
  }
  cpa_wait_all();
  __syncthreads();
  {
    // 2. chunk elimination; the slot holds (E, g, H) of each interior cell, lane-interleaved
    float E[9], gg[3], H[9];
    float Xs[NR3];  // the separator row: lower (0-8), C (9-17), r (18-20); diagonal in Bs
    float Bs[9];
    // x_0 = p + Q x_{t+1} + W X_{l-1}, carried down the chunk with the elimination
    float p[3], Q[9], W[9];
    int a = G.a, b = G.bb + min(w, G.nvalid - 1);
    // the cell before the chunk's first: Ubar's u_D on the chunk's first face
    // (the wall value at the start of a walled line)
    float uf;
    {
      int m0 = lane * P;
      if (m0 > 0 || cyc) {
        uf = sm[7 * FS + sidx<P, L, CB>(w, m0 > 0 ? m0 - 1 : n - 1)];
      } else {
        int i, j, k;
        line_pos(D, a, b, 0, i, j, k);
        uf = S.ub.f[1 + D][face_idx(g, D, i, j, k)];
      }
    }
    Thermo<float> th;
    {
      int i, j, k, m0 = lane * P, s0 = sidx<P, L, CB>(w, m0);
      line_pos(D, a, b, m0, i, j, k);
      th = thermo(g, S.P, i, sm[s0], sm[FS + s0]);
    }
#pragma unroll 1
    for (int t = 0; t < P; t++) {
      int m = lane * P + t;
      int si = sidx<P, L, CB>(w, m);
      int i, j, k, fi, fj, fk;
      line_pos(D, a, b, m, i, j, k);
      next_face(D, n, m, i, j, k, fi, fj, fk);
      float ufn = sm[7 * FS + si];
      CPt<float> cq;
      cq.Pb = th.Pb; cq.Tb = th.Tb; cq.beta = th.beta;
      cq.uc = 0.5f * (uf + ufn);
      cq.grr = sm[2 * FS + si]; cq.gtt = sm[3 * FS + si]; cq.gpp = sm[4 * FS + si];
      cq.s1 = D > 0 ? sm[5 * FS + si] : 0.f;
      cq.s2 = D > 0 ? sm[6 * FS + si] : 0.f;
      FPt<float> fq = {th.rho, 1.f, ufn};
      if (m < n - 1 || cyc) {
        // the next cell along the line: its thermodynamics serve this face row and the next step
        int mn = m + 1 == n ? 0 : m + 1, sn = sidx<P, L, CB>(w, mn);
        int in_, jn, kn;
        line_pos(D, a, b, mn, in_, jn, kn);
        th = thermo(g, S.P, in_, sm[sn], sm[FS + sn]);
        fq.rho1 = th.rho;
      }
      uf = ufn;
      float rr[3] = {sm[8 * FS + si], sm[9 * FS + si], sm[10 * FS + si]};
      float A[9], B[9], C[9];
      assemble_pts(g, S.P, cq, fq, D, n, cyc, m, i, j, fi, fj, h, A, B, C);
      if (t < P - 1) {
        float Sm[9], rv[3], Hs[9], Si[9];
        if (t == 0) {
#pragma unroll
          for (int q = 0; q < 9; q++) { Sm[q] = B[q]; Hs[q] = A[q]; }
#pragma unroll
          for (int q = 0; q < 3; q++) rv[q] = rr[q];
        } else {
          float T9[9], u[3];
          mm3_A(A, E, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) Sm[q] = B[q] - T9[q];
          mv3_A(A, gg, u);
#pragma unroll
          for (int q = 0; q < 3; q++) rv[q] = rr[q] - u[q];
          mm3_A(A, H, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) Hs[q] = -T9[q];
        }
        if (!inv3(Sm, Si)) bad |= FLAG_SINGULAR;
        mm3_XC(Si, C, E);
        mv3(Si, rv, gg);
        mm3(Si, Hs, H);
        // with x_t = g_t - E_t x_{t+1} - H_t X_{l-1}:
        //   p <- p + Q g_t,  W <- W - Q H_t,  Q <- -Q E_t
        if (t == 0) {
#pragma unroll
          for (int q = 0; q < 3; q++) p[q] = gg[q];
#pragma unroll
          for (int q = 0; q < 9; q++) { Q[q] = -E[q]; W[q] = -H[q]; }
        } else {
          float T9[9], u[3];
          mv3(Q, gg, u);
#pragma unroll
          for (int q = 0; q < 3; q++) p[q] += u[q];
          mm3(Q, H, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) W[q] -= T9[q];
          mm3(Q, E, T9);
#pragma unroll
          for (int q = 0; q < 9; q++) Q[q] = -T9[q];
        }
        float* s = slot + t * NFAC * 32 + wl;
#pragma unroll
        for (int q = 0; q < 9; q++) s[q * 32] = E[q];
#pragma unroll
        for (int q = 0; q < 3; q++) s[(9 + q) * 32] = gg[q];
#pragma unroll
        for (int q = 0; q < 9; q++) s[(12 + q) * 32] = H[q];
      } else if (P == 1) {
#pragma unroll
        for (int q = 0; q < 9; q++) { Xs[q] = A[q]; Bs[q] = B[q]; Xs[9 + q] = C[q]; }
#pragma unroll
        for (int q = 0; q < 3; q++) Xs[18 + q] = rr[q];
      } else {
        // separator: x_{s-1} = g - E X_l - H X_{l-1}
        float T9[9], u[3];
        mm3_A(A, H, T9);
#pragma unroll
        for (int q = 0; q < 9; q++) Xs[q] = -T9[q];
        mm3_A(A, E, T9);
#pragma unroll
        for (int q = 0; q < 9; q++) { Bs[q] = B[q] - T9[q]; Xs[9 + q] = C[q]; }
        mv3_A(A, gg, u);
#pragma unroll
        for (int q = 0; q < 3; q++) Xs[18 + q] = rr[q] - u[q];
      }
    }
    if (P > 1) {
      // x_0 = p + Q X_l + W X_{l-1} (the elimination's last interior cell had x_{t+1} = X_l)
      // separator row: x_{s+1} = p' + Q' X_{l+1} + W' X_l from lane l+1 (lines
      // longer than a warp exchange through the staged fields 3-10, dead now
      // that every lane has eliminated its chunk)
      float pn[3], Qn[9], Wn[9], T9[9], u[3];
      bool none = !cyc && lane == L - 1;
      if (L > 32) __syncthreads();
      xget<3, L>(p, pn, (lane + 1) & (L - 1), none, xb);
      xget<9, L>(Q, Qn, (lane + 1) & (L - 1), none, xb);
      xget<9, L>(W, Wn, (lane + 1) & (L - 1), none, xb);
      mm3_C(Xs + 9, Wn, T9);
#pragma unroll
      for (int q = 0; q < 9; q++) Bs[q] += T9[q];
      mv3_C(Xs + 9, pn, u);
#pragma unroll
      for (int q = 0; q < 3; q++) Xs[18 + q] -= u[q];
      mm3_C(Xs + 9, Qn, T9);
#pragma unroll
      for (int q = 0; q < 9; q++) Xs[9 + q] = T9[q];
    }
    {
      float Xn[NR3];
      normalise3(Xs, Bs, Xs + 9, Xs + 18, Xn, &bad);
#pragma unroll
      for (int q = 0; q < NR3; q++) Xs[q] = Xn[q];
    }
    // 3. reduced system
    float xs[3], xp[3];
    pcr3<L>(Xs, lane, cyc, xs, &bad, xb);
    xget<3, L>(xs, xp, (lane + L - 1) & (L - 1), !cyc && lane == 0, xb);
    // 4. back substitution; each lane writes its increments over its own
    // staged inputs (fields 0-2), which only it reads
    int sl = sidx<P, L, CB>(w, lane * P + P - 1);
#pragma unroll
    for (int q = 0; q < 3; q++) sm[q * FS + sl] = xs[q];
    float xn[3] = {xs[0], xs[1], xs[2]};
#pragma unroll 1
    for (int t = P - 2; t >= 0; t--) {
      const float* s = slot + t * NFAC * 32 + wl;
      float Et[9], gt[3], Ht[9], u[3], v[3];
#pragma unroll
      for (int q = 0; q < 9; q++) Et[q] = s[q * 32];
#pragma unroll
      for (int q = 0; q < 3; q++) gt[q] = s[(9 + q) * 32];
#pragma unroll
      for (int q = 0; q < 9; q++) Ht[q] = s[(12 + q) * 32];
      mv3(Et, xn, u);
      mv3(Ht, xp, v);
      int st = sidx<P, L, CB>(w, lane * P + t);
#pragma unroll
      for (int q = 0; q < 3; q++) {
        xn[q] = gt[q] - u[q] - v[q];
        sm[q * FS + st] = xn[q];
      }
    }
    if (P > 1) {
      // the slot is dead: drop its lines from L2 without writing them back
      __syncwarp();
      for (int q = wl; q < slot_floats(P); q += 32)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(slot + q * 32) : "memory");
    }
  }
  __syncthreads();
  // 5. write back (coalesced like the staging).  In update mode every FP64
  // state value a thread needs is loaded before any store, so the loads are in
  // flight together (the compiler may not move a load above a possibly
  // aliasing store).
  if (!S.update) {
#pragma unroll
    for (int q = 0; q < P; q++) {
      int lw, c;
      elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
      if (lw >= G.nvalid) continue;
      int si = sidx<P, L, CB>(lw, c);
      int i, j, k;
      line_pos(D, G.a, G.bb + lw, c, i, j, k);
      int ic = IC(g, i, j, k);
      S.x.f[0][ic] = sm[si];
      S.x.f[4][ic] = sm[FS + si];
      int fi, fj, fk;
      next_face(D, n, c, i, j, k, fi, fj, fk);
      S.x.f[1 + D][face_idx(g, D, fi, fj, fk)] = (c < n - 1 || cyc) ? sm[2 * FS + si] : 0.f;
      if (c == 0 && !cyc) {
        int wi = i, wj = j, wk = k;
        if (D == 0) wi = 0; else if (D == 1) wj = 0; else wk = 0;
        S.x.f[1 + D][face_idx(g, D, wi, wj, wk)] = 0.f;
      }
    }
  } else {
    int ic[P], iu[P], iw[P];
    double bp[P], bT[P], bu[P], bw[P];
#pragma unroll
    for (int q = 0; q < P; q++) {
      int lw, c;
      elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
      ic[q] = iu[q] = iw[q] = -1;
      if (lw >= G.nvalid) continue;
      int i, j, k;
      line_pos(D, G.a, G.bb + lw, c, i, j, k);
      ic[q] = IC(g, i, j, k);
      int fi, fj, fk;
      next_face(D, n, c, i, j, k, fi, fj, fk);
      iu[q] = face_idx(g, D, fi, fj, fk);
      if (c == 0 && !cyc) {
        int wi = i, wj = j, wk = k;
        if (D == 0) wi = 0; else if (D == 1) wj = 0; else wk = 0;
        iw[q] = face_idx(g, D, wi, wj, wk);
      }
      bp[q] = S.base.f[0][ic[q]];
      bT[q] = S.base.f[4][ic[q]];
      bu[q] = S.base.f[1 + D][iu[q]];
      bw[q] = iw[q] >= 0 ? S.base.f[1 + D][iw[q]] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < P; q++) {
      if (ic[q] < 0) continue;
      int lw, c;
      elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
      int si = sidx<P, L, CB>(lw, c);
      put_upd(S, 0, ic[q], bp[q], sm[si], ss, &bad);
      put_upd(S, 4, ic[q], bT[q], sm[FS + si], ss, &bad);
      if (c < n - 1 || cyc) put_upd(S, 1 + D, iu[q], bu[q], sm[2 * FS + si], ss, &bad);
      else S.uk.f[1 + D][iu[q]] = bu[q];  // wall face: the state is kept
      if (iw[q] >= 0) S.uk.f[1 + D][iw[q]] = bw[q];
    }
  }
  flush_norms(S, ss, bad);
}

// one block per line group (at most 128 registers a thread)
template <int D, int P, int L, int CB>
__global__ void __launch_bounds__(CB / P, 512 * P / CB) k_lines_blk(SweepArgs<float> S) {
  lines_blk<D, P, L, CB>(S, blockIdx.x);
}

// Scalar lines of the transverse component trans_comp(D, KIND), n = L P, CB
// cells per block: line group grp of that kind.
template <int D, int P, int L, int CB, int KIND>
__device__ __forceinline__ void lines_sca(const SweepArgs<float>& S, int grp) {
  using SH = Shape<P, L, CB>;
  constexpr int NW = SH::NW, NT = SH::NT, FS = SH::FS;
  constexpr int NI = P > 1 ? P - 1 : 1;
  constexpr int cc = trans_comp(D, KIND);
  extern __shared__ float sm[];
  const Geo<float>& g = S.g;
  const int n = SH::n, cyc = (D == 2 && g.per);
  const int w = threadIdx.x / L, lane = threadIdx.x % L;
  float* xb = sm + FS;  // lane exchanges of lines longer than a warp (after the elimination)
  const float h = S.h;
  SqSumLite ss;
  int bad = 0;
  Group G = group_of(S, KIND, grp, NW);
#pragma unroll
  for (int q = 0; q < P; q++) {
    int lw, c;
    elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
    stage_scalar<D, KIND, FS>(S, sm, sidx<P, L, CB>(lw, c), G.a, G.bb + min(lw, G.nvalid - 1), c);  // see k_lines_blk
  }
  cpa_wait_all();
  __syncthreads();
  {
    int a = G.a, b = G.bb + min(w, G.nvalid - 1);
    float e_[NI], g_[NI], h_[NI];
    float ep = 0.f, gp = 0.f, hp_ = 0.f;
    float sa = 0.f, sb = 1.f, sc = 0.f, sr = 0.f;  // separator row
#pragma unroll
    for (int t = 0; t < P; t++) {
      int m = lane * P + t;
      int si = sidx<P, L, CB>(w, m);
      SPt<float> q = {sm[si], sm[FS + si], 0.5f * (sm[2 * FS + si] + sm[3 * FS + si])};
      float r = sm[4 * FS + si];
      int i, j, k;
      line_pos(D, a, b, m, i, j, k);
      float wt[3];
      row_sw(g, S.P, q, cc, D, i, j, wt);
      float am = h * wt[0], bm = 1.f + h * wt[1], cm = h * wt[2];
      if (!cyc) {
        if (m == 0) { bm -= am; am = 0.f; }
        if (m == n - 1) { bm -= cm; cm = 0.f; }
      }
      if (t < P - 1) {
        float sden = t == 0 ? bm : bm - am * ep;
        float rv = t == 0 ? r : r - am * gp;
        float hs = t == 0 ? am : -am * hp_;
        if (sden == 0.f || !isfinite(sden)) bad |= FLAG_SINGULAR;
        float is = sdiv(1.f, sden);
        ep = cm * is; gp = rv * is; hp_ = hs * is;
        e_[t] = ep; g_[t] = gp; h_[t] = hp_;
      } else if (P == 1) {
        sa = am; sb = bm; sc = cm; sr = r;
      } else {
        sa = -am * hp_; sb = bm - am * ep; sc = cm; sr = r - am * gp;
      }
    }
    if (P > 1) {
      float p = gp, Q = -ep, W = -hp_;
#pragma unroll
      for (int t = P - 3; t >= 0; t--) {
        p = g_[t] - e_[t] * p;
        Q = -e_[t] * Q;
        W = -h_[t] - e_[t] * W;
      }
      bool none = !cyc && lane == L - 1;
      float pqw[3] = {p, Q, W}, nx[3];
      if (L > 32) __syncthreads();
      xget<3, L>(pqw, nx, (lane + 1) & (L - 1), none, xb);
      float pn = nx[0], Qn = nx[1], Wn = nx[2];
      sb += sc * Wn;
      sr -= sc * pn;
      sc = sc * Qn;
    }
    if (sb == 0.f || !isfinite(sb)) bad |= FLAG_SINGULAR;
    float ib = sdiv(1.f, sb);
    float xs = pcr1<L>(sa * ib, sc * ib, sr * ib, lane, cyc, &bad, xb);
    float xp;
    xget<1, L>(&xs, &xp, (lane + L - 1) & (L - 1), !cyc && lane == 0, xb);
    float xo[P];
    xo[P - 1] = xs;
#pragma unroll
    for (int t = P - 2; t >= 0; t--) xo[t] = g_[t] - e_[t] * xo[t + 1] - h_[t] * xp;
#pragma unroll
    for (int t = 0; t < P; t++) sm[sidx<P, L, CB>(w, lane * P + t)] = xo[t];
  }
  __syncthreads();
  if (!S.update) {
#pragma unroll
    for (int q = 0; q < P; q++) {
      int lw, c;
      elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
      if (lw >= G.nvalid) continue;
      int i, j, k;
      line_pos(D, G.a, G.bb + lw, c, i, j, k);
      scalar_put(S, cc, i, j, k, sm[sidx<P, L, CB>(lw, c)], ss, &bad);
    }
  } else {
    // every FP64 state value first, then the stores (see the block-line kernel)
    int iv[P];
    double bv[P];
#pragma unroll
    for (int q = 0; q < P; q++) {
      int lw, c;
      elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
      iv[q] = -1;
      if (lw >= G.nvalid) continue;
      int i, j, k;
      line_pos(D, G.a, G.bb + lw, c, i, j, k);
      iv[q] = face_idx(g, cc, i, j, k);
      bv[q] = S.base.f[1 + cc][iv[q]];
    }
#pragma unroll
    for (int q = 0; q < P; q++) {
      if (iv[q] < 0) continue;
      int lw, c;
      elem<D, P, L, CB>(threadIdx.x + q * NT, lw, c);
      put_upd(S, 1 + cc, iv[q], bv[q], sm[sidx<P, L, CB>(lw, c)], ss, &bad);
      int i, j, k;
      line_pos(D, G.a, G.bb + lw, c, i, j, k);
      scalar_walls(S, cc, i, j, k);
    }
  }
  flush_norms(S, ss, bad);
}

// Both transverse components of the sweep in one launch: blocks [0, ng1) take
// the line groups of kind 1, the rest those of kind 2.  At most 48 registers a
// thread (measured: the sweeps 2-4 % faster than at the compiler's 56-64, with
// more resident warps for the serial chunk chains; 40 and 32 spill and lose).
template <int D, int P, int L, int CB>
__global__ void __launch_bounds__(CB / P, 65536 * P / (CB * 48)) k_lines_sca(SweepArgs<float> S, int ng1) {
  if ((int)blockIdx.x < ng1) lines_sca<D, P, L, CB, 1>(S, blockIdx.x);
  else lines_sca<D, P, L, CB, 2>(S, blockIdx.x - ng1);
}

}  // namespace lines
