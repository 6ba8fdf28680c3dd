// sph_batch.cu -- batched launches over a batch of independent problems of
// different sizes (sph_batch_capture_fused): every stage of the scheme's
// iteration (Section 2.2: the midpoint state and frozen coefficients of eq.
// chapter3mainsd, the right-hand side of eq. spl1, the line solves of eqs.
// spl1-spl3) runs as ONE launch over all problems, not one per problem.
//
// A launch reads an instance descriptor table (one entry per problem: its
// grid, coefficient planes, state and work buffers -- what the single-problem
// kernels take as parameters) and a block map (per block: which problem, and
// which tile or line group of it).  A block copies its problem's descriptor
// into shared memory and runs the same device code as the single-problem
// kernel on that tile or line group, so a batched step computes what
// per-problem steps compute (to FP32 rounding: the code is compiled into other
// kernels, where the compiler may contract other multiply-adds).  The sweeps
// launch once per line layout
// (lines of the same length and lane layout share a kernel instantiation),
// the layouts side by side on separate streams.  Everything is recorded into
// one CUDA graph of an even number of steps, like sph_batch_capture.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/sph.h"
#include "sph_kernels.cuh"
#include "sph_lines.cuh"
#include "sph_host.cuh"

namespace fused {

// the tile of a stencil launch: tk x tj x ti points (phi, theta, r) per block
// of 128 threads, gx x gy tiles in the phi x theta plane, n tiles in all
struct Tile { int tk, tj, ti, gx, gy, n; };

// Consecutive tiles of one problem a block of a stencil launch takes (one
// descriptor load for all of them), and the blocks per SM the coefficient and
// centre-row kernels are compiled for (48 and 64 registers a thread): the
// descriptor in shared memory costs registers that at the single-problem
// kernels' 32 spill heavily.  Measured on the 64-instance ensemble (ms per
// step): 1 tile at 32 registers 49.1, 4 tiles 49.4, 4 tiles at 48/64
// registers 45.8, 8 tiles at 48/64 45.5.
#ifndef FUSED_TILES
#define FUSED_TILES 8
#endif
constexpr int TILES = FUSED_TILES;
#ifndef FUSED_MINB_COEF
#define FUSED_MINB_COEF 10
#endif
#ifndef FUSED_MINB_RHSC
#define FUSED_MINB_RHSC 8
#endif
#ifndef FUSED_MINB_RHSU
#define FUSED_MINB_RHSU 16
#endif

struct CoefTab {
  Geo<float> g;
  Par P;
  CF<float> ub;
  Coef<float> c;
  Tile t;
};

struct RhsTab {
  Geo<float> g;
  Par P;
  Coef<float> c;
  CF<float> ub, ul, Dv;
  CF<double> un, uk, src;
  MF<float> Rout;
  float tau;
  int hasD;
  Tile t[4];  // centres (p, T rows), then the faces of u_r, u_theta, u_phi
};

struct LineTab {
  SweepArgs<float> S;
  int ng1;    // line groups of the first transverse kind (the scalar launch)
  int pad;
};

// Never read: rhs_c_at takes the FP64 grid for the FP64 kernels' div(Ubar),
// which the FP32 instantiation does not form.
__device__ Geo<double> g_unused_gd;

// dst = src for a descriptor (8-byte words, the whole block), then a barrier
template <typename T>
__device__ __forceinline__ void load_args(T& dst, const T& src) {
  static_assert(sizeof(T) % 8 == 0, "descriptors are whole 8-byte words");
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(&src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
  for (int w = threadIdx.x; w < (int)(sizeof(T) / 8); w += blockDim.x) d[w] = s[w];
  __syncthreads();
}

// point (i, j, k) of this thread in tile b of a launch with tile shape t
struct Pt { int i, j, k, i0, j0; };
__device__ __forceinline__ Pt point_of(const Tile& t, int b) {
  const int bx = b % t.gx, r = b / t.gx, by = r % t.gy, bz = r / t.gy;
  const int tid = threadIdx.x, tx = tid % t.tk, r2 = tid / t.tk, ty = r2 % t.tj, tz = r2 / t.tj;
  Pt p;
  p.i0 = bz * t.ti;
  p.j0 = by * t.tj;
  p.i = p.i0 + tz;
  p.j = p.j0 + ty;
  p.k = bx * t.tk + tx;
  return p;
}

// Ubar and D of one chunk of one field of one problem: map = (problem, field,
// first pair, pairs), the pairs of 16-byte loads as in k_avg; the chunk that
// ends the field also takes an odd last element.
__global__ void __launch_bounds__(256) k_avg_f(const AvgArgs<float>* tab, const int4* map) {
  const int4 m = map[blockIdx.x];
  const AvgArgs<float>& A = tab[m.x];
  const int f = m.y;
  const double* __restrict__ a = A.a[f];
  const double* __restrict__ b = A.b[f];
  float* __restrict__ o = A.o[f];
  float* __restrict__ lo = A.lo[f];
  float* __restrict__ d = A.d[f];
  const long n = A.n[f];
  const int same = A.same;
  for (int r = threadIdx.x; r < m.w; r += blockDim.x) {
    const long t = (long)m.z + r;
    double2 x = reinterpret_cast<const double2*>(a)[t];
    if (same) {
      split1(x.x, o, lo, 2 * t);
      split1(x.y, o, lo, 2 * t + 1);
    } else {
      double2 y = reinterpret_cast<const double2*>(b)[t];
      avg1(x.x, y.x, o, lo, d, 2 * t);
      avg1(x.y, y.y, o, lo, d, 2 * t + 1);
    }
  }
  if ((n & 1) && (long)m.z + m.w == (n >> 1) && threadIdx.x == 0) {
    if (same) split1(a[n - 1], o, lo, n - 1);
    else avg1(a[n - 1], b[n - 1], o, lo, d, n - 1);
  }
}

// the coefficient stage (k_coef) over the tiles of every problem
__global__ void __launch_bounds__(128, FUSED_MINB_COEF) k_coef_f(const CoefTab* tab, const int2* map) {
  __shared__ CoefTab A;
  const int2 m = map[blockIdx.x];
  load_args(A, tab[m.x]);
  const Geo<float>& g = A.g;
  const int b1 = min(m.y + TILES, A.t.n);
  for (int b = m.y; b < b1; b++) {
    const Pt p = point_of(A.t, b);
    const bool inner = tile_inner_at(g, p.i0, p.j0, A.t.ti, A.t.tj);
    if (p.k >= g.np || p.j >= g.nt || p.i >= g.nr) continue;
    const int t = IC(g, p.i, p.j, p.k);
    if (inner) coef_at<0>(g, A.P, A.ub, A.c, p.i, p.j, p.k, t);
    else coef_at<1>(g, A.P, A.ub, A.c, p.i, p.j, p.k, t);
  }
}

// the p- and T-rows of the right-hand side (k_rhs_c) over every problem
__global__ void __launch_bounds__(128, FUSED_MINB_RHSC) k_rhs_c_f(const RhsTab* tab, const int2* map) {
  __shared__ RhsTab A;
  const int2 m = map[blockIdx.x];
  load_args(A, tab[m.x]);
  const Geo<float>& g = A.g;
  const int b1 = min(m.y + TILES, A.t[0].n);
  for (int b = m.y; b < b1; b++) {
    const Pt p = point_of(A.t[0], b);
    const bool inner = tile_inner_at(g, p.i0, p.j0, A.t[0].ti, A.t[0].tj);
    if (p.k >= g.np || p.j >= g.nt || p.i >= g.nr) continue;
    const int t = IC(g, p.i, p.j, p.k);
    if (inner)
      rhs_c_at<0>(g, g_unused_gd, A.P, A.c, A.ub, A.ul, A.un, A.uk, A.Dv, A.hasD, A.src, 0, A.tau, A.Rout, p.i, p.j, p.k, t);
    else
      rhs_c_at<1>(g, g_unused_gd, A.P, A.c, A.ub, A.ul, A.un, A.uk, A.Dv, A.hasD, A.src, 0, A.tau, A.Rout, p.i, p.j, p.k, t);
  }
}

// the momentum rows of component D (k_rhs_u) over every problem; zero on wall faces
template <int D>
__global__ void __launch_bounds__(128, FUSED_MINB_RHSU) k_rhs_u_f(const RhsTab* tab, const int2* map) {
  __shared__ RhsTab A;
  const int2 m = map[blockIdx.x];
  load_args(A, tab[m.x]);
  const Geo<float>& g = A.g;
  const Tile& tl = A.t[1 + D];
  const int nj = g.nt + (D == 1), nk = D == 2 ? g.npf : g.np;
  const int b1 = min(m.y + TILES, tl.n);
  for (int b = m.y; b < b1; b++) {
    const Pt p = point_of(tl, b);
    const bool inner = tile_inner_at(g, p.i0, p.j0, tl.ti, tl.tj);
    if (p.k >= nk || p.j >= nj || p.i >= g.nr + (D == 0)) continue;
    const int t = (p.i * nj + p.j) * nk + p.k;
    const bool wall = D == 0 ? (p.i == 0 || p.i == g.nr) : D == 1 ? (p.j == 0 || p.j == g.nt)
                                                                  : (!g.per && (p.k == 0 || p.k == g.np));
    if (wall) A.Rout.f[1 + D][t] = 0.f;
    else if (inner) rhs_u_at<0, D>(g, A.P, A.c, A.ub, A.Dv, A.hasD, A.src, 0, A.tau, A.Rout, p.i, p.j, p.k, t);
    else rhs_u_at<1, D>(g, A.P, A.c, A.ub, A.Dv, A.hasD, A.src, 0, A.tau, A.Rout, p.i, p.j, p.k, t);
  }
}

// the iteration residual's sums of squares of every problem, zeroed
__global__ void k_zero_acc_f(double* const* acc, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 5 * n) acc[q / 5][q % 5] = 0.0;
}

// block lines of one layout over every problem that has it: map = (entry of
// the layout's table, line group)
template <int D, int P, int L, int CB>
__global__ void __launch_bounds__(CB / P, 512 * P / CB) k_lines_blk_f(const LineTab* tab, const int2* map) {
  __shared__ SweepArgs<float> S;
  const int2 m = map[blockIdx.x];
  load_args(S, tab[m.x].S);
  lines::lines_blk<D, P, L, CB>(S, m.y);
}

// both transverse kinds of one layout over every problem that has it: groups
// [0, ng1) of an entry are of the first kind, the rest of the second
template <int D, int P, int L, int CB>
__global__ void __launch_bounds__(CB / P, 65536 * P / (CB * 48)) k_lines_sca_f(const LineTab* tab, const int2* map) {
  __shared__ SweepArgs<float> S;
  const int2 m = map[blockIdx.x];
  load_args(S, tab[m.x].S);
  const int ng1 = tab[m.x].ng1;
  if (m.y < ng1) lines::lines_sca<D, P, L, CB, 1>(S, m.y);
  else lines::lines_sca<D, P, L, CB, 2>(S, m.y - ng1);
}

}  // namespace fused

// ============================================================== host side

namespace {

template <typename R> CF<R> cf5(R* const* p) { CF<R> r; for (int f = 0; f < 5; f++) r.f[f] = p[f]; return r; }
template <typename R> MF<R> mf5(R* const* p) { MF<R> r; for (int f = 0; f < 5; f++) r.f[f] = p[f]; return r; }

// host staging of the tables and maps: pieces at 256-byte offsets of one
// device buffer
struct Blob {
  std::vector<char> h;
  size_t put(const void* p, size_t n) {
    size_t off = (h.size() + 255) & ~(size_t)255;
    h.resize(off + (n ? n : 1));
    if (n) memcpy(h.data() + off, p, n);
    return off;
  }
  template <typename T> size_t put(const std::vector<T>& v) { return put(v.data(), v.size() * sizeof(T)); }
};

// the stencil tile of a context over an nk x nj x ni box
fused::Tile tile_of(const sph_ctx* c, int nk, int nj, int ni, int* blocks) {
  fused::Tile t;
  t.tj = c->tile_j;
  t.ti = c->tile_i;
  t.tk = 128 / (t.tj * t.ti);
  t.gx = (nk + t.tk - 1) / t.tk;
  t.gy = (nj + t.tj - 1) / t.tj;
  t.n = t.gx * t.gy * ((ni + t.ti - 1) / t.ti);
  *blocks = t.n;
  return t;
}

// the shared-memory attributes of a layout's batched kernels (per device, before any capture)
template <int D, int P, int L>
int attr_f() {
  constexpr int CB = lines_cb(D, L * P);
  static unsigned long long done = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (done & bit) return SPH_OK;
  const int smb = lines::NFB * lines::Shape<P, L, CB>::FS * (int)sizeof(float);
  const int sms = lines::NFS * lines::Shape<P, L, CB>::FS * (int)sizeof(float);
  if (cudaFuncSetAttribute(fused::k_lines_blk_f<D, P, L, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb) !=
          cudaSuccess ||
      cudaFuncSetAttribute(fused::k_lines_sca_f<D, P, L, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, sms) !=
          cudaSuccess)
    return SPH_ERR_CUDA;
  done |= bit;
  return SPH_OK;
}

template <int D, int P, int L>
void launch_f(const fused::LineTab* tab, const int2* mb, int nb, const int2* ms, int ns, cudaStream_t s1,
              cudaStream_t s2) {
  constexpr int CB = lines_cb(D, L * P);
  using SH = lines::Shape<P, L, CB>;
  const size_t smb = (size_t)lines::NFB * SH::FS * sizeof(float);
  const size_t sms = (size_t)lines::NFS * SH::FS * sizeof(float);
  if (nb > 0) fused::k_lines_blk_f<D, P, L, CB><<<nb, SH::NT, smb, s1>>>(tab, mb);
  if (ns > 0) fused::k_lines_sca_f<D, P, L, CB><<<ns, SH::NT, sms, s2>>>(tab, ms);
}

// one layout's attributes (attr) or launches, dispatched on (P, L)
template <int D>
int layout_f(int P, int L, bool attr, const fused::LineTab* tab, const int2* mb, int nb, const int2* ms, int ns,
             cudaStream_t s1, cudaStream_t s2) {
#define SPH_LAYOUT_F(p, l)                           \
  if (P == p && L == l) {                            \
    if (attr) return attr_f<D, p, l>();              \
    launch_f<D, p, l>(tab, mb, nb, ms, ns, s1, s2); \
    return SPH_OK;                                   \
  }
  SPH_LINES_EACH_PL(SPH_LAYOUT_F)
#undef SPH_LAYOUT_F
  if constexpr (D == 2) {
    if (P == 8 && L == 64) { if (attr) return attr_f<D, 8, 64>(); launch_f<D, 8, 64>(tab, mb, nb, ms, ns, s1, s2); return SPH_OK; }
    if (P == 8 && L == 128) { if (attr) return attr_f<D, 8, 128>(); launch_f<D, 8, 128>(tab, mb, nb, ms, ns, s1, s2); return SPH_OK; }
  }
  return SPH_ERR_ARG;
}

int layout_any(int D, int P, int L, bool attr, const fused::LineTab* tab, const int2* mb, int nb, const int2* ms,
               int ns, cudaStream_t s1, cudaStream_t s2) {
  if (D == 0) return layout_f<0>(P, L, attr, tab, mb, nb, ms, ns, s1, s2);
  if (D == 1) return layout_f<1>(P, L, attr, tab, mb, nb, ms, ns, s1, s2);
  return layout_f<2>(P, L, attr, tab, mb, nb, ms, ns, s1, s2);
}

// the problems of one batch whose lines along d share a layout (P, L)
struct Layout {
  int d, P, L;
  std::vector<int> q;                 // problems (batch indices)
  size_t tab[2][2];                   // LineTab arrays per (step parity, later iteration)
  size_t mb, ms;                      // block maps
  int nb, ns;                         // blocks of the block-line and scalar-line launches
};

}  // namespace

void batch_fused_free(sph_batch* b) {
  if (!b) return;
  if (b->ftab) {
    cudaStreamSynchronize(b->st);
    cudaFree(b->ftab);
    b->ftab = NULL;
  }
  for (int q = 0; q < b->fstreams; q++) {
    cudaStreamDestroy(b->fst[q]);
    cudaEventDestroy(b->fjoin[q]);
  }
  if (b->fstreams) cudaEventDestroy(b->ffork);
  b->fstreams = 0;
}

// n side streams wait for what the batch stream holds so far / the batch
// stream waits for them (stream-ordered, so the capture records the edges)
static int ffork(sph_batch* b, int n) {
  if (cudaEventRecord(b->ffork, b->st) != cudaSuccess) return SPH_ERR_CUDA;
  for (int q = 0; q < n; q++)
    if (cudaStreamWaitEvent(b->fst[q], b->ffork, 0) != cudaSuccess) return SPH_ERR_CUDA;
  return SPH_OK;
}
static int fjoin(sph_batch* b, int n) {
  for (int q = 0; q < n; q++)
    if (cudaEventRecord(b->fjoin[q], b->fst[q]) != cudaSuccess || cudaStreamWaitEvent(b->st, b->fjoin[q], 0) != cudaSuccess)
      return SPH_ERR_CUDA;
  return SPH_OK;
}

extern "C" int sph_batch_capture_fused(sph_batch* b, double dt, int n_iter, int steps) {
  if (!b || !(dt > 0) || n_iter < 1 || steps < 2 || (steps & 1)) return SPH_ERR_ARG;
  const int n = b->n;
  for (int q = 0; q < n; q++) {
    const sph_ctx* c = b->c[q];
    if (c->prof || c->prec != SPH_PREC_MIXED || c->hasbc || c->d32.g.hasw || c->line_solver == SPH_LINES_THOMAS)
      return SPH_ERR_ARG;
    for (int d = 0; d < 3; d++)
      if (!lines_ok(c, d)) return SPH_ERR_ARG;
  }
  // work the contexts have queued (state uploads) is finished before the
  // tables are built and the graph is first replayed on the batch stream
  for (int q = 0; q < n; q++)
    if (cudaStreamSynchronize(b->c[q]->st) != cudaSuccess) return SPH_ERR_CUDA;
  if (b->exec) {
    cudaStreamSynchronize(b->st);
    cudaGraphExecDestroy(b->exec);
    b->exec = NULL;
  }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = NULL; }
  if (b->ftab) { cudaFree(b->ftab); b->ftab = NULL; }
  if (!b->fstreams) {
    if (cudaEventCreateWithFlags(&b->ffork, cudaEventDisableTiming) != cudaSuccess) return SPH_ERR_CUDA;
    for (int q = 0; q < SPH_FUSED_STREAMS; q++) {
      if (cudaStreamCreateWithFlags(&b->fst[q], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->fjoin[q], cudaEventDisableTiming) != cudaSuccess) {
        b->fstreams = q + 1;  // batch_fused_free destroys what was made (a failed create leaves a null handle)
        batch_fused_free(b);
        return SPH_ERR_CUDA;
      }
      b->fstreams = q + 1;
    }
  }

  Blob blob;
  // ---- averaging: tables per (step parity, later iteration), one map
  std::vector<AvgArgs<float>> avg[2][2];
  std::vector<int4> mavg;
  // ---- stencil stages
  std::vector<fused::CoefTab> coef(n);
  std::vector<fused::RhsTab> rhs[2][2];
  std::vector<int2> mcoef, mrhs[4];
  std::vector<double*> accs(n);
  for (int p = 0; p < 2; p++)
    for (int it = 0; it < 2; it++) {
      avg[p][it].resize(n);
      rhs[p][it].resize(n);
    }
  for (int q = 0; q < n; q++) {
    sph_ctx* c = b->c[q];
    Bufs<float>& B = c->d32;
    const Geo<double>& g = c->d64.g;
    accs[q] = c->acc;
    for (int p = 0; p < 2; p++)
      for (int it = 0; it < 2; it++) {
        const int cur = c->cur ^ p;
        double* const* un = c->U[cur];
        double* const* uk = it ? c->U[1 - cur] : un;
        AvgArgs<float>& A = avg[p][it][q];
        memset(&A, 0, sizeof A);
        A.same = !it;
        for (int f = 0; f < 5; f++) {
          A.a[f] = un[f]; A.b[f] = uk[f]; A.o[f] = B.Ub[f]; A.lo[f] = B.UbLo[f]; A.d[f] = B.Db[f];
          A.n[f] = (long)c->nf[f];
        }
        fused::RhsTab& R = rhs[p][it][q];
        memset(&R, 0, sizeof R);
        R.g = B.g; R.P = c->P; R.c = B.c;
        R.ub = cf5(B.Ub); R.ul = cf5(B.UbLo); R.Dv = cf5(B.Db);
        R.un = cf5(un); R.uk = cf5(uk); R.src = cf5(c->src);
        R.Rout = mf5(B.Rb);
        R.tau = (float)dt;
        R.hasD = it;
      }
    int nb[5];
    fused::Tile tc = tile_of(c, g.np, g.nt, g.nr, &nb[0]);
    fused::Tile tu[3] = {tile_of(c, g.np, g.nt, g.nr + 1, &nb[1]), tile_of(c, g.np, g.nt + 1, g.nr, &nb[2]),
                         tile_of(c, g.npf, g.nt, g.nr, &nb[3])};
    fused::CoefTab& C = coef[q];
    memset(&C, 0, sizeof C);
    C.g = B.g; C.P = c->P; C.ub = cf5(B.Ub); C.c = B.c; C.t = tc;
    for (int p = 0; p < 2; p++)
      for (int it = 0; it < 2; it++) {
        fused::RhsTab& R = rhs[p][it][q];
        R.t[0] = tc;
        for (int d = 0; d < 3; d++) R.t[1 + d] = tu[d];
      }
    // a block per fused::TILES consecutive tiles of the problem
    for (int k = 0; k < nb[0]; k += fused::TILES) { mcoef.push_back(make_int2(q, k)); mrhs[0].push_back(make_int2(q, k)); }
    for (int d = 0; d < 3; d++)
      for (int k = 0; k < nb[1 + d]; k += fused::TILES) mrhs[1 + d].push_back(make_int2(q, k));
    for (int f = 0; f < 5; f++) {
      const long pairs = (long)c->nf[f] >> 1;
      for (long s = 0; s < pairs || (s == 0 && pairs == 0); s += 1024)
        mavg.push_back(make_int4(q, f, (int)s, (int)(pairs - s < 1024 ? pairs - s : 1024)));
    }
  }
  // ---- line layouts of each direction
  std::vector<Layout> lay;
  std::vector<fused::LineTab> ltab[64][2][2];   // per layout (at most 3 x 15 exist)
  std::vector<int2> lmb[64], lms[64];
  for (int d = 0; d < 3; d++)
    for (int q = 0; q < n; q++) {
      sph_ctx* c = b->c[q];
      const Geo<double>& g = c->d64.g;
      const int len = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
      int P = 0, L = 0;
      lines_pl(c->line_solver, d, len, &P, &L);
      int li = -1;
      for (int z = 0; z < (int)lay.size(); z++)
        if (lay[z].d == d && lay[z].P == P && lay[z].L == L) li = z;
      if (li < 0) {
        if (lay.size() >= 64) return SPH_ERR_ARG;
        Layout Ly;
        Ly.d = d; Ly.P = P; Ly.L = L; Ly.nb = Ly.ns = 0; Ly.mb = Ly.ms = 0;
        lay.push_back(Ly);
        li = (int)lay.size() - 1;
      }
      Layout& Ly = lay[li];
      const int e = (int)Ly.q.size();
      Ly.q.push_back(q);
      const int CB = lines_cb(d, len), NW = CB / len, NWW = CB / P / 32;
      Bufs<float>& B = c->d32;
      int ng[3] = {0, 0, 0};
      for (int p = 0; p < 2; p++)
        for (int it = 0; it < 2; it++) {
          const int cur = c->cur ^ p;
          double* const* un = c->U[cur];
          double* const* uk = it ? c->U[1 - cur] : un;
          fused::LineTab T;
          memset(&T, 0, sizeof T);
          SweepArgs<float>& S = T.S;
          S.g = B.g; S.P = c->P; S.c = B.c; S.ub = cf5(B.Ub); S.d = d; S.h = (float)(0.5 * dt);
          S.rhs = cf5(d == 1 ? B.X1 : B.Rb);
          S.x = mf5(d == 1 ? B.Rb : B.X1);
          S.update = d == 2;
          S.base = cf5(uk);
          S.uk = mf5(c->U[1 - cur]);
          S.scr = B.scr; S.acc = c->acc; S.flag = c->flag;
          line_layout(g, d, S);
          for (int k = 0; k < 3; k++) ng[k] = lines_groups(S, k, NW);
          T.ng1 = ng[1];
          ltab[li][p][it].push_back(T);
        }
      // one factor slot per warp of the block-line launch (as in the single-problem path)
      if ((size_t)ng[0] * NWW * 32 * lines::slot_floats(P) > c->nscr) return SPH_ERR_ARG;
      for (int k = 0; k < ng[0]; k++) lmb[li].push_back(make_int2(e, k));
      for (int k = 0; k < ng[1] + ng[2]; k++) lms[li].push_back(make_int2(e, k));
    }
  // ---- one device buffer
  size_t oavg[2][2], orhs[2][2];
  for (int p = 0; p < 2; p++)
    for (int it = 0; it < 2; it++) {
      oavg[p][it] = blob.put(avg[p][it]);
      orhs[p][it] = blob.put(rhs[p][it]);
    }
  const size_t ocoef = blob.put(coef), omavg = blob.put(mavg), omcoef = blob.put(mcoef), oacc = blob.put(accs);
  size_t omrhs[4];
  for (int k = 0; k < 4; k++) omrhs[k] = blob.put(mrhs[k]);
  for (size_t z = 0; z < lay.size(); z++) {
    for (int p = 0; p < 2; p++)
      for (int it = 0; it < 2; it++) lay[z].tab[p][it] = blob.put(ltab[z][p][it]);
    lay[z].mb = blob.put(lmb[z]);
    lay[z].ms = blob.put(lms[z]);
    lay[z].nb = (int)lmb[z].size();
    lay[z].ns = (int)lms[z].size();
  }
  if (cudaMalloc(&b->ftab, blob.h.size()) != cudaSuccess) { cudaGetLastError(); b->ftab = NULL; return SPH_ERR_NOMEM; }
  if (cudaMemcpy(b->ftab, blob.h.data(), blob.h.size(), cudaMemcpyHostToDevice) != cudaSuccess) return SPH_ERR_CUDA;
  char* base = (char*)b->ftab;
  for (size_t z = 0; z < lay.size(); z++)
    if (int e = layout_any(lay[z].d, lay[z].P, lay[z].L, true, NULL, NULL, 0, NULL, 0, NULL, NULL)) return e;
  // ---- the graph: `steps` steps of every problem
  for (int q = 0; q < n; q++) { b->cur[q] = b->c[q]->cur; b->nlaunch[q] = 0; }
  long long nk = 0;
  if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SPH_ERR_CUDA;
  int err = SPH_OK;
  const int nrc = (int)mrhs[0].size();
  for (int s = 0; s < steps && !err; s++) {
    const int p = s & 1;
    for (int it = 0; it < n_iter && !err; it++) {
      const int il = it > 0;
      fused::k_avg_f<<<(unsigned)mavg.size(), 256, 0, b->st>>>((const AvgArgs<float>*)(base + oavg[p][il]),
                                                               (const int4*)(base + omavg));
      fused::k_coef_f<<<(unsigned)mcoef.size(), 128, 0, b->st>>>((const fused::CoefTab*)(base + ocoef),
                                                                (const int2*)(base + omcoef));
      nk += 2;
      const fused::RhsTab* rt = (const fused::RhsTab*)(base + orhs[p][il]);
      if ((err = ffork(b, 3))) break;
      fused::k_rhs_c_f<<<nrc, 128, 0, b->st>>>(rt, (const int2*)(base + omrhs[0]));
      fused::k_rhs_u_f<0><<<(unsigned)mrhs[1].size(), 128, 0, b->fst[0]>>>(rt, (const int2*)(base + omrhs[1]));
      fused::k_rhs_u_f<1><<<(unsigned)mrhs[2].size(), 128, 0, b->fst[1]>>>(rt, (const int2*)(base + omrhs[2]));
      fused::k_rhs_u_f<2><<<(unsigned)mrhs[3].size(), 128, 0, b->fst[2]>>>(rt, (const int2*)(base + omrhs[3]));
      nk += 4;
      if ((err = fjoin(b, 3))) break;
      for (int d = 0; d < 3 && !err; d++) {
        if (d == 2 && it == n_iter - 1) {
          fused::k_zero_acc_f<<<(5 * n + 255) / 256, 256, 0, b->st>>>((double* const*)(base + oacc), n);
          nk++;
        }
        int used = 0;
        for (size_t z = 0; z < lay.size(); z++) used += lay[z].d == d ? 2 : 0;
        used = used < SPH_FUSED_STREAMS ? used : SPH_FUSED_STREAMS;
        if ((err = ffork(b, used))) break;
        int slot = 0;
        for (size_t z = 0; z < lay.size() && !err; z++) {
          const Layout& Ly = lay[z];
          if (Ly.d != d) continue;
          cudaStream_t s1 = b->fst[slot % SPH_FUSED_STREAMS], s2 = b->fst[(slot + 1) % SPH_FUSED_STREAMS];
          slot += 2;
          err = layout_any(d, Ly.P, Ly.L, false, (const fused::LineTab*)(base + Ly.tab[p][il]),
                           (const int2*)(base + Ly.mb), Ly.nb, (const int2*)(base + Ly.ms), Ly.ns, s1, s2);
          nk += (Ly.nb > 0) + (Ly.ns > 0);
        }
        if (!err) err = fjoin(b, used);
      }
      if (!err && cudaGetLastError() != cudaSuccess) err = SPH_ERR_CUDA;
    }
  }
  cudaGraph_t gr = NULL;
  cudaError_t ce = cudaStreamEndCapture(b->st, &gr);
  if (!err && ce != cudaSuccess) err = SPH_ERR_CUDA;
  if (!err && cudaGraphInstantiate(&b->exec, gr, 0) != cudaSuccess) err = SPH_ERR_CUDA;
  if (err) {
    if (gr) cudaGraphDestroy(gr);
    b->exec = NULL;
    cudaGetLastError();
    return err;
  }
  b->graph = gr;
  b->nlaunch[0] = nk;  // the batched kernels are shared: counted once, on the first problem
  return SPH_OK;
}

#ifdef SPH_CHECKED
int bounds_take_batch(int* h) {
  int z[5] = {0, 0, 0, 0, 0};
  if (cudaMemcpyFromSymbol(h, g_bounds, 5 * sizeof(int)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_bounds, z, sizeof z) != cudaSuccess)
    return SPH_ERR_CUDA;
  return SPH_OK;
}
#endif
