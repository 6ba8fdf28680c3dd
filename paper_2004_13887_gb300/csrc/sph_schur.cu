// sph_schur.cu -- the partitioned (Schur-complement) block Thomas algorithm of
// Section 2.2, for 3x3-block tridiagonal lines whose blocks are split across P
// ranks: each rank eliminates its own segment, the segments' first and last
// blocks form a small reduced system that every rank solves after an
// all-gather of the interface rows, and each rank back-substitutes.
//
// Rank p owns blocks 0..m-1 of each line (m >= 2):
//   A_i x_{i-1} + B_i x_i + C_i x_{i+1} = d_i,
// where x_{-1} is the last block of rank p-1 and x_m the first block of rank
// p+1 (on a cyclic line rank 0's left neighbour is rank P-1 and rank P-1's
// right neighbour is rank 0; on a walled line the outer couplings are zero).
// With T the segment's own block-tridiagonal matrix (A_0 and C_{m-1} removed),
//   x = y - V x_{-1} - W x_m,  T y = d,  T V = A_0 e_0,  T W = C_{m-1} e_{m-1},
// so the first and last blocks f_p = x_0, l_p = x_{m-1} of every rank satisfy
//   f_p + V_0 l_{p-1} + W_0 f_{p+1} = y_0,
//   l_p + V_{m-1} l_{p-1} + W_{m-1} f_{p+1} = y_{m-1},
// a 6P x 6P system per line (block-tridiagonal in 6x6 blocks, cyclic on a
// cyclic line), solved here densely with partial pivoting.  No pivoting between
// the blocks of a segment, as in the sequential block Thomas algorithm.
//
// All pointers are device pointers; the library allocates nothing (the
// caller passes the scratch).  Blocks are 3x3 row-major.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/sph.h"

namespace {

__device__ bool inv3s(const double* S, double* I) {
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

constexpr int NC = 7;  // right-hand-side columns: d, the 3 of A_0 e_0, the 3 of C_{m-1} e_{m-1}

// One thread per line: block Thomas on the segment with NC right-hand sides.
// scr: 9 + 3 NC doubles per block (C' and the eliminated right-hand sides),
// interleaved by line.  Outputs per block: y (3), V (3x3), W (3x3).
__global__ void k_schur_local(int nlines, int m, const double* __restrict__ A, const double* __restrict__ B,
                              const double* __restrict__ C, const double* __restrict__ d, double* __restrict__ scr,
                              double* __restrict__ Y, double* __restrict__ V, double* __restrict__ W, int* flag) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  const int WS = 9 + 3 * NC;
  double Cp[9], dp[3 * NC];
  for (int i = 0; i < m; i++) {
    long b = (long)l * m + i;
    const double* Ai = A + 9 * b;
    const double* Bi = B + 9 * b;
    const double* Ci = C + 9 * b;
    // right-hand sides of row i, column-major in the 3 rows: rr[r * NC + q]
    double rr[3 * NC];
    for (int r = 0; r < 3; r++) {
      rr[r * NC] = d[3 * b + r];
      for (int q = 0; q < 3; q++) {
        rr[r * NC + 1 + q] = i == 0 ? Ai[r * 3 + q] : 0.0;
        rr[r * NC + 4 + q] = i == m - 1 ? Ci[r * 3 + q] : 0.0;
      }
    }
    double S[9], y[3 * NC];
    if (i == 0) {
      for (int q = 0; q < 9; q++) S[q] = Bi[q];
      for (int q = 0; q < 3 * NC; q++) y[q] = rr[q];
    } else {
      for (int r = 0; r < 3; r++) {
        for (int q = 0; q < 3; q++)
          S[r * 3 + q] = Bi[r * 3 + q] - (Ai[r * 3] * Cp[q] + Ai[r * 3 + 1] * Cp[3 + q] + Ai[r * 3 + 2] * Cp[6 + q]);
        for (int q = 0; q < NC; q++)
          y[r * NC + q] = rr[r * NC + q] - (Ai[r * 3] * dp[q] + Ai[r * 3 + 1] * dp[NC + q] + Ai[r * 3 + 2] * dp[2 * NC + q]);
      }
    }
    double Si[9];
    if (!inv3s(S, Si)) { atomicOr(flag, 1); return; }
    for (int r = 0; r < 3; r++) {
      for (int q = 0; q < 3; q++)
        Cp[r * 3 + q] = i == m - 1 ? 0.0 : Si[r * 3] * Ci[q] + Si[r * 3 + 1] * Ci[3 + q] + Si[r * 3 + 2] * Ci[6 + q];
      for (int q = 0; q < NC; q++)
        dp[r * NC + q] = Si[r * 3] * y[q] + Si[r * 3 + 1] * y[NC + q] + Si[r * 3 + 2] * y[2 * NC + q];
    }
    double* s = scr + (long)i * WS * nlines + l;
    for (int q = 0; q < 9; q++) s[(long)q * nlines] = Cp[q];
    for (int q = 0; q < 3 * NC; q++) s[(long)(9 + q) * nlines] = dp[q];
  }
  // back substitution, all columns
  double xs[3 * NC];
  for (int i = m - 1; i >= 0; i--) {
    const double* s = scr + (long)i * WS * nlines + l;
    double Cq[9], dq[3 * NC];
    for (int q = 0; q < 9; q++) Cq[q] = s[(long)q * nlines];
    for (int q = 0; q < 3 * NC; q++) dq[q] = s[(long)(9 + q) * nlines];
    if (i == m - 1) {
      for (int q = 0; q < 3 * NC; q++) xs[q] = dq[q];
    } else {
      double xn[3 * NC];
      for (int r = 0; r < 3; r++)
        for (int q = 0; q < NC; q++)
          xn[r * NC + q] = dq[r * NC + q] - (Cq[r * 3] * xs[q] + Cq[r * 3 + 1] * xs[NC + q] + Cq[r * 3 + 2] * xs[2 * NC + q]);
      for (int q = 0; q < 3 * NC; q++) xs[q] = xn[q];
    }
    long b = (long)l * m + i;
    for (int r = 0; r < 3; r++) {
      Y[3 * b + r] = xs[r * NC];
      for (int q = 0; q < 3; q++) {
        V[9 * b + r * 3 + q] = xs[r * NC + 1 + q];
        W[9 * b + r * 3 + q] = xs[r * NC + 4 + q];
      }
    }
  }
}

constexpr int MAXP = 8;
constexpr int IFACE = 42;  // per rank and line: V_0, V_{m-1}, W_0, W_{m-1} (9 each), y_0, y_{m-1} (3 each)

// One thread per line: assemble the 6P x 6P reduced system from every rank's
// interface rows (iface[(p * nlines + l) * 42 + ...]) and solve it by Gaussian
// elimination with partial pivoting; z[(l * 2P + 2p) * 3] = f_p, [.. + 2p + 1] = l_p.
__global__ void k_schur_reduced(int nlines, int P, int cyclic, const double* __restrict__ iface, double* __restrict__ z,
                                int* flag) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  const int n = 6 * P;
  double M[6 * MAXP][6 * MAXP + 1];
  for (int r = 0; r < n; r++)
    for (int q = 0; q <= n; q++) M[r][q] = (r == q) ? 1.0 : 0.0;
  for (int p = 0; p < P; p++) {
    const double* f = iface + ((long)p * nlines + l) * IFACE;
    const double *V0 = f, *Vm = f + 9, *W0 = f + 18, *Wm = f + 27, *y0 = f + 36, *ym = f + 39;
    int left = p - 1, right = p + 1;
    int has_left = left >= 0, has_right = right < P;
    if (cyclic) { left = (left + P) % P; right = right % P; has_left = has_right = 1; }
    for (int r = 0; r < 3; r++) {
      int rf = 6 * p + r, rl = 6 * p + 3 + r;  // the rows of f_p and l_p
      M[rf][n] = y0[r];
      M[rl][n] = ym[r];
      for (int q = 0; q < 3; q++) {
        if (has_left) {
          M[rf][6 * left + 3 + q] += V0[r * 3 + q];   // l_{p-1}
          M[rl][6 * left + 3 + q] += Vm[r * 3 + q];
        }
        if (has_right) {
          M[rf][6 * right + q] += W0[r * 3 + q];      // f_{p+1}
          M[rl][6 * right + q] += Wm[r * 3 + q];
        }
      }
    }
  }
  for (int c = 0; c < n; c++) {
    int piv = c;
    double best = fabs(M[c][c]);
    for (int r = c + 1; r < n; r++)
      if (fabs(M[r][c]) > best) { best = fabs(M[r][c]); piv = r; }
    if (best == 0.0 || !isfinite(best)) { atomicOr(flag, 1); return; }
    if (piv != c)
      for (int q = c; q <= n; q++) { double t = M[c][q]; M[c][q] = M[piv][q]; M[piv][q] = t; }
    double inv = 1.0 / M[c][c];
    for (int r = c + 1; r < n; r++) {
      double f = M[r][c] * inv;
      if (f == 0.0) continue;
      for (int q = c; q <= n; q++) M[r][q] -= f * M[c][q];
    }
  }
  for (int r = n - 1; r >= 0; r--) {
    double v = M[r][n];
    for (int q = r + 1; q < n; q++) v -= M[r][q] * M[q][n];
    M[r][n] = v / M[r][r];
  }
  // z: per rank f_p then l_p, 3 each
  for (int p = 0; p < P; p++)
    for (int r = 0; r < 3; r++) {
      z[((long)l * 2 * P + 2 * p) * 3 + r] = M[6 * p + r][n];
      z[((long)l * 2 * P + 2 * p + 1) * 3 + r] = M[6 * p + 3 + r][n];
    }
}

// x_i = y_i - V_i xl - W_i xr, one thread per block
__global__ void k_schur_back(long nb, int m, const double* __restrict__ Y, const double* __restrict__ V,
                             const double* __restrict__ W, const double* __restrict__ xl,
                             const double* __restrict__ xr, double* __restrict__ x) {
  long b = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  long l = b / m;
  const double *a = xl + 3 * l, *c = xr + 3 * l;
  for (int r = 0; r < 3; r++)
    x[3 * b + r] = Y[3 * b + r] - (V[9 * b + r * 3] * a[0] + V[9 * b + r * 3 + 1] * a[1] + V[9 * b + r * 3 + 2] * a[2])
                 - (W[9 * b + r * 3] * c[0] + W[9 * b + r * 3 + 1] * c[1] + W[9 * b + r * 3 + 2] * c[2]);
}

int status_of(int* flag, cudaStream_t st) {
  if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SPH_ERR_CUDA;
  return h ? SPH_ERR_SINGULAR : SPH_OK;
}

}  // namespace

extern "C" int sph_schur_local(int nlines, int m, const double* A, const double* B, const double* C, const double* d,
                               double* scratch, double* Y, double* V, double* W, int* flag, void* stream) {
  if (nlines < 1 || m < 2 || !A || !B || !C || !d || !scratch || !Y || !V || !W || !flag) return SPH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return SPH_ERR_CUDA;
  k_schur_local<<<(nlines + 127) / 128, 128, 0, st>>>(nlines, m, A, B, C, d, scratch, Y, V, W, flag);
  return status_of(flag, st);
}

extern "C" int sph_schur_reduced(int nlines, int P, int cyclic, const double* iface, double* z, int* flag,
                                 void* stream) {
  if (nlines < 1 || P < 1 || P > MAXP || !iface || !z || !flag) return SPH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return SPH_ERR_CUDA;
  k_schur_reduced<<<(nlines + 63) / 64, 64, 0, st>>>(nlines, P, cyclic ? 1 : 0, iface, z, flag);
  return status_of(flag, st);
}

extern "C" int sph_schur_back(int nlines, int m, const double* Y, const double* V, const double* W, const double* xl,
                              const double* xr, double* x, void* stream) {
  if (nlines < 1 || m < 2 || !Y || !V || !W || !xl || !xr || !x) return SPH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  long nb = (long)nlines * m;
  k_schur_back<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(nb, m, Y, V, W, xl, xr, x);
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
