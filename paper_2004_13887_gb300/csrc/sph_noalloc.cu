// sph_noalloc.cu -- a batched 3x3-block tridiagonal line solver that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool must
// not grow, inside a host that forbids runtime allocation after start-up, or in
// plug-ins that only receive device pointers from their host.  For them this
// file provides one entry point, sph_block_thomas_noalloc, which runs the same
// block Thomas elimination the line sweeps use (forward elimination with the
// block adjugate, no pivoting between blocks, back substitution) on line systems
// the caller has assembled.  Its elimination scratch (C'_m and d'_m, 12 doubles
// per block) lives in the file-scope array below instead of a cudaMalloc'd
// buffer.  The array is part of the library image: every GPU that loads the
// library holds it (SPH_NOALLOC_MAX_BLOCKS * 12 doubles, 12.6 MB) until the
// process exits.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/sph.h"

#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_scratch[(size_t)SPH_NOALLOC_MAX_BLOCKS * 12];

// Device address of the array on each device, looked up once per device: in
// host code the symbol's name is only a host-side stand-in, not an address.
static double* s_scratch[NOALLOC_MAX_DEVICES];

static __device__ __forceinline__ bool inv3_na(const double* S, double* I) {
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

// One thread per line.  Blocks of line l, cell m start at ((l*n + m)*9); the
// scratch is interleaved by line, [(m*12 + q)*nlines + l], so a warp's accesses
// are contiguous.
__global__ void k_block_thomas_noalloc(int nlines, int n, const double* __restrict__ A, const double* __restrict__ B,
                                       const double* __restrict__ C, const double* __restrict__ d,
                                       double* __restrict__ x, double* __restrict__ scr) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  double Cp[9], dp[3];
  for (int m = 0; m < n; m++) {
    long b = ((long)l * n + m);
    const double* Am = A + 9 * b;
    const double* Bm = B + 9 * b;
    const double* Cm = C + 9 * b;
    const double* dm = d + 3 * b;
    double S[9], y[3];
    if (m == 0) {
      for (int q = 0; q < 9; q++) S[q] = Bm[q];
      for (int q = 0; q < 3; q++) y[q] = dm[q];
    } else {
      for (int r = 0; r < 3; r++) {
        for (int q = 0; q < 3; q++)
          S[r * 3 + q] = Bm[r * 3 + q] - (Am[r * 3] * Cp[q] + Am[r * 3 + 1] * Cp[3 + q] + Am[r * 3 + 2] * Cp[6 + q]);
        y[r] = dm[r] - (Am[r * 3] * dp[0] + Am[r * 3 + 1] * dp[1] + Am[r * 3 + 2] * dp[2]);
      }
    }
    double Si[9];
    if (!inv3_na(S, Si)) {   // zero pivot: the whole line becomes NaN
      for (long q = 0; q < 3L * n; q++) x[3L * l * n + q] = NAN;
      return;
    }
    bool last = (m == n - 1);
    for (int r = 0; r < 3; r++) {
      for (int q = 0; q < 3; q++)
        Cp[r * 3 + q] = last ? 0.0 : Si[r * 3] * Cm[q] + Si[r * 3 + 1] * Cm[3 + q] + Si[r * 3 + 2] * Cm[6 + q];
      dp[r] = Si[r * 3] * y[0] + Si[r * 3 + 1] * y[1] + Si[r * 3 + 2] * y[2];
    }
    if (!last) {
      double* s = scr + (long)m * 12 * nlines + l;
      for (int q = 0; q < 9; q++) s[(long)q * nlines] = Cp[q];
      for (int q = 0; q < 3; q++) s[(long)(9 + q) * nlines] = dp[q];
    }
  }
  double xs[3] = {dp[0], dp[1], dp[2]};
  double* xo = x + 3 * ((long)l * n + (n - 1));
  xo[0] = xs[0]; xo[1] = xs[1]; xo[2] = xs[2];
  for (int m = n - 2; m >= 0; m--) {
    const double* s = scr + (long)m * 12 * nlines + l;
    double Cq[9], dq[3], xn[3];
    for (int q = 0; q < 9; q++) Cq[q] = s[(long)q * nlines];
    for (int q = 0; q < 3; q++) dq[q] = s[(long)(9 + q) * nlines];
    for (int r = 0; r < 3; r++) xn[r] = dq[r] - (Cq[r * 3] * xs[0] + Cq[r * 3 + 1] * xs[1] + Cq[r * 3 + 2] * xs[2]);
    xs[0] = xn[0]; xs[1] = xn[1]; xs[2] = xn[2];
    xo = x + 3 * ((long)l * n + m);
    xo[0] = xs[0]; xo[1] = xs[1]; xo[2] = xs[2];
  }
}

// Per-device set-up, with that device current: the device address of the array.
static int noalloc_setup(int dev) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SPH_ERR_ARG;
  if (s_scratch[dev]) return SPH_OK;
  void* p = NULL;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
  s_scratch[dev] = (double*)p;
  return SPH_OK;
}

extern "C" int sph_block_thomas_noalloc(int nlines, int n, const double* A, const double* B, const double* C,
                                        const double* d, double* x, void* stream) {
  if (nlines < 1 || n < 1 || !A || !B || !C || !d || !x) return SPH_ERR_ARG;
  if ((long long)nlines * (long long)n > (long long)SPH_NOALLOC_MAX_BLOCKS) return SPH_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
  int e = noalloc_setup(dev);
  if (e != SPH_OK) return e;
  cudaStream_t st = (cudaStream_t)stream;
  int threads = 128;
  int blocks = (nlines + threads - 1) / threads;
  k_block_thomas_noalloc<<<blocks, threads, 0, st>>>(nlines, n, A, B, C, d, x, s_scratch[dev]);
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
