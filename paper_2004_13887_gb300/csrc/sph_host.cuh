// sph_host.cuh -- host-side state shared by the translation units of the
// library: the device buffers of a problem (Bufs), the context (sph_ctx), the
// batch of independent problems (sph_batch), and the layout of the line
// systems of a sweep (which lines exist, how the partitioned solver groups
// them into blocks).
#pragma once
#include <cuda_runtime.h>
#include <string.h>

#include "../../include/sph.h"
#include "sph_kernels.cuh"

// Device buffers of one precision.
template <typename R>
struct Bufs {
  R* metric;       // rc rf irc irf | sc sf isc isf cc cf cotc cotf (bulk type)
  R* bgder;        // dbgp dbgT lapT rhoref (nr each) ehyd (nr+1) pcen Tcen (nr each)
  R* mdf;          // rf^2 hi, lo (nr+1 each), sin(theta_f) hi, lo (nt+1 each)
  R* Ub[5];
  R* UbLo[5];      // FP32 mode: remainders of the velocity components of Ubar (1-3)
  R* Db[5];        // U^{n+1,k} - U^n
  R* Rb[5];
  R* X1[5];
  R* coef;
  R* scr;
  Geo<R> g;
  Coef<R> c;
};

struct sph_ctx {
  int dev;
  cudaStream_t st;
  int prec;
  Par P;
  size_t nf[5];
  long N;
  double* bg;            // p_ref, T_ref (nr+2 each)
  double* U[2][5];
  int cur;
  int iterate_set;
  double* src[5];
  double* acc;           // 5 sums + spare
  int* flag;
  double* hmet;          // host copy of the FP64 metric tables
  size_t nmet;
  Bufs<double> d64;      // FP64 metric/background tables always; bulk buffers in FP64 mode
  Bufs<float> d32;       // bulk buffers in mixed mode
  double* rows64;        // FP64 mode: the line rows the right-hand side stores for the sweeps
  Rows64 rows;           // pointers into rows64 (all null in mixed mode)
  long long launches;
  long unknowns[5];
  // per-kernel timing
  int prof;
  int nvtx_open;         // a stage's NVTX range is open (k_begin .. launch_ok)
  cudaEvent_t* ev;
  int* evkind;
  int nev, evcap;
  long long kcount[SPH_NKERNELS];
  int cur_kind;
  int nsm;               // multiprocessors of the device
  cudaStream_t aux[3];   // side streams for independent launches of one stage
  cudaEvent_t efork, ejoin[3];
  int line_solver;       // SPH_LINES_* for the mixed path
  int tile_j, tile_i;    // stencil tile: 128 / (tile_j tile_i) phi points x tile_j x tile_i
  size_t nscr;           // floats in each bulk scratch buffer
  // wall data (sph_set_bc): the mean of the t^n and t^{n+1} values of the 18
  // arrays (FP64, and FP32 in mixed mode) for the tangential ghosts, and the
  // t^{n+1} normal velocity (c == d entries) copied into U^{n+1,0}
  int hasbc;
  size_t woff[18], wtot;   // offsets of the arrays in the buffers (wtot = total)
  int wset[18];            // which arrays were given
  double* wmean64;
  float* wmean32;
  double* wnext;
  double* wzero64;        // zeros of the largest wall size: the arrays without data
  float* wzero32;
  // adjoint workspace (sph_step_adjoint), allocated on first use
  int adjK;               // iterates the workspace holds
  size_t fset;            // doubles of one 5-field set
  size_t foff[5];         // offsets of the fields in a set
  double* adjS;           // U^{n+1,k}, k < adjK
  double* adjW;           // 10 sets: lam_n, lam, mu_r, mu_theta, mu_phi, x_r, x_theta, x_phi, lam_Ubar, spare
  double* adjC;           // the coefficient planes' accumulators (17 planes)
  double* tape_d;
  int* tape_ix;
  int* tape_li;
  double* tape_adj;
  int* adj_info;          // longest tape used
  int tape_cap, tape_blocks;
};

#define SPH_FUSED_STREAMS 8

struct sph_batch {
  int n;
  sph_ctx** c;
  cudaStream_t st;
  cudaEvent_t fork;
  cudaEvent_t* join;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int* cur;                // each context's U^n buffer at capture
  long long* nlaunch;      // kernels one replay launches per context
  // batched launches (sph_batch_capture_fused): the descriptor tables and
  // block maps in one device buffer, side streams for independent launches
  void* ftab;
  cudaStream_t fst[SPH_FUSED_STREAMS];
  cudaEvent_t ffork, fjoin[SPH_FUSED_STREAMS];
  int fstreams;            // side streams created
};

// frees what sph_batch_capture_fused allocated (sph_batch.cu)
void batch_fused_free(sph_batch* b);
#ifdef SPH_CHECKED
// the bounds counter of the batched kernels' translation unit into h, then zeroed
int bounds_take_batch(int* h);
#endif


// Lines of direction d: kind 0 = block lines (a, b) over cell centres, kinds 1/2 =
// the two transverse velocity components on their interior faces.  Half-open
// ranges [a_lo, a_hi) x [b_lo, b_hi); (a, b) = (j, k) for d = r, (i, k) for
// theta, (i, j) for phi.
template <typename R>
static void line_layout(const Geo<double>& g, int d, SweepArgs<R>& S) {
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
    S.nl[q] = (na > 0 && nb > 0) ? na * nb : 0;
    S.scr_off[q] = (int)off;
    long w = q == 0 ? (g.per && d == 2 ? 21 : 12) : 3;
    off += w * (long)n * S.nl[q];
  }
}

// cells per block of the partitioned solver: 2048 for 256-cell lines along r
// and theta (8 adjacent lines per block fill each 32-byte sector) and for the
// phi lines of 512 and 1024 cells (4 and 2 lines a block); 512, 768 and 1536
// for lines of 16, 48 and 192 cells (32, 16 and 8 lines); else 1024
__host__ __device__ constexpr int lines_cb(int D, int n) {
  return n == 16 ? 512 : n == 48 ? 768 : n == 192 ? 1536 : n >= 512 || (D != 2 && n == 256) ? 2048 : 1024;
}

static int lines_groups(const SweepArgs<float>& S, int kind, int NW) {
  if (S.nl[kind] <= 0) return 0;
  int nb = S.nb[kind], na = S.nl[kind] / nb;
  return na * ((nb + NW - 1) / NW);
}

// whether the partitioned solver takes the lines along d: lines of 16, 32, 48,
// 64, 128, 192 and 256 cells, and phi lines of 512 and 1024 (one thread per
// line would read those uncoalesced).  Along r and theta, lines of 512 cells run faster on the
// block Thomas path, whose threads read adjacent lines together (measured:
// theta 4.3 vs 5.0 ms per step on 64 x 512 x 1024), and more accurately where
// I + tau/2 D_r is stiff.
static int lines_ok(const sph_ctx* c, int d) {
  const Geo<double>& g = c->d64.g;
  int n = d == 0 ? g.nr : d == 1 ? g.nt : g.np;
  return n == 16 || n == 32 || n == 48 || n == 64 || n == 128 || n == 192 || n == 256 ||
         (d == 2 && (n == 512 || n == 1024));
}

// Partitioned layout of lines of n cells along D for a line solver: P cells per
// lane, L lanes per line.  Lines of 16, 32, 48 cells: 16 lanes (chunks of 1, 2,
// 3), or in the narrow layout 4 lanes (chunks of 4) and 8 lanes (chunks of 4,
// 6); 64: 16 lanes, 32 (one warp per line) or 8 (narrow, chunks of 8); 128: 16
// lanes unless one warp per line is asked for; 192 and 256: one warp (chunks of
// 6, 8); phi lines of 512 and 1024: 2 and 4 warps (chunks of 8).
static inline void lines_pl(int solver, int D, int n, int* P, int* L) {
  const int warp = solver == SPH_LINES_PARTITIONED_WARP, narrow = solver == SPH_LINES_PARTITIONED_NARROW;
  int p = 8, l = 32;
  if (n == 16) { p = narrow ? 4 : 1; l = narrow ? 4 : 16; }
  else if (n == 32) { p = narrow ? 4 : 2; l = narrow ? 8 : 16; }
  else if (n == 48) { p = narrow ? 6 : 3; l = narrow ? 8 : 16; }
  else if (n == 64) { p = narrow ? 8 : warp ? 2 : 4; l = narrow ? 8 : warp ? 32 : 16; }
  else if (n == 128) { p = warp ? 4 : 8; l = warp ? 32 : 16; }
  else if (n == 192) { p = 6; l = 32; }
  else if (D == 2 && n == 512) { p = 8; l = 64; }
  else if (D == 2 && n == 1024) { p = 8; l = 128; }
  *P = p;
  *L = l;
}
// every (P, L) of lines_pl in every direction (X(P, L) once each); phi lines of
// 512 and 1024 add (8, 64) and (8, 128)
#define SPH_LINES_EACH_PL(X) \
  X(1, 16) X(4, 4) X(2, 16) X(4, 8) X(3, 16) X(6, 8) X(4, 16) X(2, 32) X(8, 8) X(8, 16) X(4, 32) X(6, 32) X(8, 32)
