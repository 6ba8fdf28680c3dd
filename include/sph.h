/*
 * sph.h -- C ABI of the GB300 (sm_103a) library for the direction-splitting
 * scheme of Frolov, Minev & Takhirov, "An efficient algorithm for weakly
 * compressible flows in spherical geometries" (arXiv 2004.13887).
 *
 * The library advances the non-conservative compressible Navier-Stokes system
 * of Section 2.1 (eqs. nonconservmass-nonconserveos) in a spherical sector by
 * the Picard-iterated, direction-split Crank-Nicolson scheme of Section 2.2
 * (eqs. chapter3mainsd, splitting2, spl1-spl3) on the MAC grid.
 *
 * Conventions (all calls):
 *  - Unknowns U = [p, u_r, u_theta, u_phi, T] (Section 2.1).  p and T are
 *    stored as perturbations p' = p - p_ref(r), T' = T - T_ref(r) about a radial
 *    background (the "a priori" pressure rescaling of Section 3.1).
 *  - Layout: FP64, C order, phi fastest.  Field f has sph_field_size(grid, f)
 *    elements:  p, T: nr*nt*np (centres); u_r: (nr+1)*nt*np (r-faces);
 *    u_theta: nr*(nt+1)*np (theta-faces); u_phi: nr*nt*npf (phi-faces) with
 *    npf = np+1, or np when phi is periodic.
 *  - Boundary conditions: Dirichlet velocity on every wall -- by default u = 0
 *    tangentially (no-slip; ghost = -interior) and the normal velocity on wall
 *    faces is whatever the state holds there, unchanged by sph_step; wall data
 *    that vary in time are set with sph_set_bc -- and zero normal derivative of
 *    p' and T' (Section 3.1: zero Neumann for pressure and temperature);
 *    optional periodic phi (cyclic line systems).
 *  - Pointers marked "device" are CUDA device pointers of the current device;
 *    "host" pointers are ordinary host memory.  The library never keeps a
 *    caller pointer after a call returns.
 *  - All work is queued on the stream given to sph_create; calls that return
 *    data to host memory synchronise that stream.
 *  - Return value: SPH_OK (0) or a negative SPH_ERR_* code; sph_strerror()
 *    describes it.  After SPH_ERR_CUDA the context should be destroyed.
 */
#ifndef SPH_H
#define SPH_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

#define SPH_OK 0
#define SPH_ERR_ARG (-1)        /* bad argument (sizes, pointers, dt <= 0, ...) */
#define SPH_ERR_CUDA (-2)       /* a CUDA runtime call failed */
#define SPH_ERR_NONFINITE (-3)  /* NaN/Inf in the new state; the state is left at U^n */
#define SPH_ERR_SINGULAR (-4)   /* a zero pivot in a line solve; state left at U^n */
#define SPH_ERR_NOMEM (-5)      /* device allocation failed */
#define SPH_ERR_TAPE (-6)       /* sph_step_adjoint: a per-thread tape was too short */

#define SPH_PREC_FP64 0          /* every step in FP64 */
#define SPH_PREC_MIXED 1         /* FP32 bulk stencils/line solves, FP64 iterate */

/* Domain [r1,r2] x [th1,th2] x [ph1,ph2] with nr x nth x nph uniform cells
 * (Section 2.1, Omega).  periodic_phi != 0 requires ph2 - ph1 = 2 pi in the
 * intended use (not checked).  th1 >= 0, th2 <= pi; a pole face is allowed. */
typedef struct {
  int nr, nth, nph;
  double r1, r2, th1, th2, ph1, ph2;
  int periodic_phi;
} sph_grid;

/* Material constants (Section 2.1): gamma = cp/cv, kappa = mu*cp/Pr, stiffened-gas
 * pi_inf, gravity g along e_r on the left-hand side (eq. nonconservmom),
 * rotation omega about the polar axis.  precision: SPH_PREC_*. */
typedef struct {
  double gamma, cv, Pr, mu, pi_inf, g, omega;
  int precision;
} sph_params;

typedef struct sph_ctx sph_ctx;

/* Number of elements of field f (0..4) for a grid. */
size_t sph_field_size(const sph_grid* grid, int f);

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL =
 * legacy default stream).  The context owns all device buffers (state U^n,
 * iterate U^{n+1,k}, coefficients, right-hand sides, line-solve scratch; in
 * SPH_PREC_FP64 also the line rows of D_r, D_theta, D_phi that each step's
 * right-hand side stores for its sweeps, about 45 doubles per cell).
 * Errors: SPH_ERR_ARG (nr, nth, nph < 2; r1 <= 0; empty ranges; periodic with
 * nph < 3; a grid too large for the kernels' 32-bit indexing: every field and
 * the line-solve scratch, 18 values per cell (27 with periodic phi), must stay
 * below 2^31 elements, i.e. at most about 1.19e8 cells on walled grids and
 * 7.9e7 with periodic phi), SPH_ERR_NOMEM, SPH_ERR_CUDA. */
int sph_create(const sph_grid* grid, const sph_params* params, void* stream, sph_ctx** out);

/* Radial background (Section 3.2 hydrostatic state, or a constant): host arrays
 * of nr+2 values each, index 0 the ghost below r1 and nr+1 the ghost above r2.
 * NULL sets that background to zero (the default). */
int sph_set_background(sph_ctx* ctx, const double* p_ref, const double* T_ref);

/* Dirichlet data for the velocity on the walls (Section 3.1: the
 * manufactured-solution test imposes the exact, time-dependent velocity on
 * every boundary; pressure and temperature keep zero normal derivatives).
 * w_n, w_np1: arrays of 18 pointers (host or device per on_device) with the
 * wall values at t^n and t^{n+1} of the coming steps; a NULL entry counts as
 * zero, and w_n = w_np1 = NULL returns to homogeneous walls.  Entry
 * (c*3 + d)*2 + s is velocity component c (0 r, 1 theta, 2 phi) on the wall
 * normal to direction d (0 r, 1 theta, 2 phi) at side s (0 low, 1 high), C
 * order with phi fastest over the wall's two other indices:
 *   c = r:     d = r  nth*nph,   d = theta (nr+1)*nph, d = phi (nr+1)*nth
 *   c = theta: d = r (nth+1)*nph, d = theta nr*nph,    d = phi nr*(nth+1)
 *   c = phi:   d = r nth*npf,    d = theta nr*npf,     d = phi nr*nth
 * (npf as for the u_phi field).  c != d: the tangential value w on the wall,
 * used by the ghost rule ghost = 2 w - interior, taken at the midpoint level
 * (w^n + w^{n+1})/2 with Ubar.  c == d: the normal velocity on the wall faces:
 * each sph_step starts its iteration from U^{n+1,0} = U^n with these faces set
 * to the t^{n+1} values (U^n keeps its own).  On a periodic phi line the d =
 * phi entries are ignored.  The data stay in effect for every later step until
 * the next call (a caller with moving walls calls it before each step).
 * Synchronises the context's stream.  Errors: SPH_ERR_NOMEM, SPH_ERR_CUDA. */
int sph_set_bc(sph_ctx* ctx, const double* const* w_n, const double* const* w_np1, int on_device);

/* Copy the 5 fields in (host or device per on_device) into U^n. */
int sph_set_state(sph_ctx* ctx, const double* const* fields, int on_device);

/* Copy U^n out into the 5 caller arrays (host or device per on_device). */
int sph_get_state(sph_ctx* ctx, double* const* fields, int on_device);

/* One time step t^n -> t^{n+1} (eq. splitting2 iterated n_iter = K times, each
 * iteration one right-hand side and the three sweeps spl1-spl3).
 * source: NULL or 5 arrays (host or device per source_on_device) holding the
 * forcing S at t^{n+1/2} of dU/dt + N(U) + G = S.  residual_out: NULL or 5 host
 * doubles, the RMS over unknowns of the last increment U^{k+1}-U^k per field
 * (synchronises).  On SPH_ERR_NONFINITE / SPH_ERR_SINGULAR U^n is unchanged. */
int sph_step(sph_ctx* ctx, double dt, int n_iter, const double* const* source, int source_on_device,
             double* residual_out);

/* sph_step without waiting: the step is only enqueued on the context's
 * stream (so it can be captured into a CUDA graph).  source: NULL or 5 device
 * arrays (host sources are SPH_ERR_ARG).  The non-finite / zero-pivot flags of
 * enqueued steps accumulate until sph_status, which synchronises the stream,
 * returns SPH_ERR_NONFINITE or SPH_ERR_SINGULAR if any step since the last
 * sph_status raised one (the state is then not usable; U^n is not restored),
 * clears the flags and optionally writes the residual of the last step.
 * sph_step itself clears pending flags. */
int sph_step_async(sph_ctx* ctx, double dt, int n_iter, const double* const* source, int source_on_device);
int sph_status(sph_ctx* ctx, double* residual_out);

/* Adjoint of one step (the reverse mode of the map U^n -> U^{n+1} that sph_step
 * computes: Section 2.2's K Picard iterations of eq. splitting2, each a
 * right-hand side (eq. spl1) and the sweeps spl1-spl3 with every coefficient
 * frozen at Ubar = (U^{n+1,k} + U^n)/2, eq. chapter3mainsd).  FP64 contexts only
 * (SPH_ERR_ARG otherwise).  The context's U^n is the step's input state; it is
 * not changed.  lam_out: 5 device arrays, dJ/dU^{n+1} of a functional J;
 * lam_in: 5 device arrays that receive dJ/dU^n (both in the field layout of
 * sph_set_state; may not alias).  source: NULL or the 5 device arrays the step
 * was given.  Wall data set by sph_set_bc are constants of the step.  The call
 * recomputes the step's iterates, then runs the iterations backwards: per
 * iteration the transposed line solves (phi, theta, r) and the gradient over
 * Ubar of the right-hand side and of the three line operators, by reverse-mode
 * differentiation of the library's own row functions.  Work buffers (about 16
 * fields plus 17 coefficient planes and 1.4 GB of per-thread tapes) are
 * allocated on the first call and kept with the context.  Synchronises.
 * Errors: SPH_ERR_ARG, SPH_ERR_NOMEM, SPH_ERR_CUDA, SPH_ERR_SINGULAR (a zero pivot
 * in a transposed solve), SPH_ERR_TAPE (a location's rows outgrew the tape). */
int sph_step_adjoint(sph_ctx* ctx, double dt, int n_iter, const double* const* source,
                     const double* const* lam_out, double* const* lam_in);
/* The longest per-thread tape the adjoint has used so far and the capacity
 * (synchronises). */
int sph_adjoint_tape_use(sph_ctx* ctx, int* longest, int* capacity);

/* Batches of independent contexts (an ensemble of problems, e.g. of different
 * grid sizes) stepped by one CUDA graph.  sph_batch_create: n distinct contexts
 * of one device with non-NULL streams (ideally one stream each), and the
 * non-NULL stream `stream` the graph runs on.  sph_batch_capture: records `steps` (even, >= 2)
 * sph_step_async calls of every context into a graph whose branches -- one per
 * context, on the context's stream -- run concurrently (per-kernel timing must
 * be off; contexts sharing a stream run one after the other in the graph).
 * sph_batch_launch: replays it `times` times on `stream` (each replay
 * advances every context by `steps` steps); SPH_ERR_ARG if a context was
 * stepped an odd number of times since the capture (its state moved to the
 * other buffer).  sph_batch_status: synchronises and returns the first
 * context's error (index in *first_bad, -1 if none), clearing all flags.
 * The contexts stay usable individually; destroy the batch before them. */
typedef struct sph_batch sph_batch;
int sph_batch_create(sph_ctx* const* ctxs, int n, void* stream, sph_batch** out);
int sph_batch_capture(sph_batch* batch, double dt, int n_iter, int steps);
/* sph_batch_capture_fused: the same graph of `steps` steps built from batched
 * launches instead of per-context ones -- each stage of an iteration (Ubar,
 * coefficients, the four right-hand-side kernels, and per sweep one block-line
 * and one scalar-line launch for each line layout present) is ONE kernel over
 * every context, reading a per-context descriptor table and a per-block map
 * (context, tile or line group) from device memory the batch allocates.  The
 * results are those of per-context steps to FP32 rounding (the same device
 * code, compiled into other kernels).  Every context must be
 * in SPH_PREC_MIXED mode with a partitioned line solver that takes all three
 * directions (line lengths 16, 32, 48, 64, 128, 192, 256; phi also 512,
 * 1024), without wall data (sph_set_bc) and with per-kernel timing off; else
 * SPH_ERR_ARG.  The launch counts of a replay are credited to the first
 * context.  Replay with sph_batch_launch as above. */
int sph_batch_capture_fused(sph_batch* batch, double dt, int n_iter, int steps);
int sph_batch_launch(sph_batch* batch, int times);
int sph_batch_status(sph_batch* batch, int* first_bad);
void sph_batch_destroy(sph_batch* batch);

/* Stage entry points (the same kernels sph_step runs), for testing each part.
 * sph_set_iterate: copy 5 fields into the iterate U^{n+1,k} (default: U^n).
 * sph_rhs: R = -(U^k - U^n) - dt [N(Ubar) + G - S], Ubar = (U^k + U^n)/2, the
 *   right-hand side of eq. (spl1) in its midpoint form; R_out: 5 device arrays.
 * sph_sweep: solve (I + dt/2 D_dir(Ubar)) x = rhs on every line of direction
 *   dir (0 r, 1 theta, 2 phi; eqs. spl1-spl3); rhs, x: 5 device arrays each
 *   (may not alias).  Values of rhs at wall faces are ignored; x is 0 there. */
int sph_set_iterate(sph_ctx* ctx, const double* const* fields, int on_device);
int sph_rhs(sph_ctx* ctx, double dt, const double* const* source, int source_on_device, double* const* R_out);
int sph_sweep(sph_ctx* ctx, int dir, double dt, const double* const* rhs, double* const* x);

/* Line solver of the sweeps in SPH_PREC_MIXED mode (eqs. spl1-spl3 leave the
 * method of solving each line open; Section 2.2 names the block Thomas
 * algorithm).  SPH_LINES_PARTITIONED (the default): for lines of 16, 32, 48,
 * 64, 128, 192 or 256 cells, and phi lines of 512 or 1024, a segment of lanes
 * per line -- each lane eliminates a chunk of the line, the chunk-boundary
 * unknowns are solved by parallel cyclic reduction across the segment, then
 * each lane back-substitutes; lines of up to 128 cells take 16 lanes (two
 * lines per warp, chunks of 1 to 8 cells), lines of 192 and 256 take 32
 * (chunks of 6 and 8), phi lines of 512 and 1024 take 64 and 128 lanes (2 and
 * 4 warps, chunks of 8); other lines use the block Thomas path.
 * SPH_LINES_PARTITIONED_WARP: the same with 32 lanes (one line per warp) for
 * the lines of 64 and 128 cells.  SPH_LINES_PARTITIONED_NARROW: fewer lanes and
 * longer chunks for the short lines -- 4 lanes with chunks of 4 for lines of
 * 16 cells, 8 lanes with chunks of 4, 6 and 8 for lines of 32, 48 and 64 --
 * so that less of the work is in the reduction; other lengths as
 * SPH_LINES_PARTITIONED.  SPH_LINES_THOMAS: block (and scalar) Thomas, one thread per
 * line, with the Woodbury / Sherman-Morrison correction on cyclic lines.  All
 * give the exact solution up to rounding (no pivoting between blocks in any).
 * The FP64 mode always uses block Thomas: with SPH_LINES_THOMAS one thread per
 * line; with any other value (the default) two threads per walled line, one
 * eliminating from each end, the two meeting at the middle cells (a 3x3 solve
 * there), which halves the dependent chain for the same arithmetic; cyclic
 * lines keep one thread and the Woodbury correction.  Returns SPH_ERR_ARG for
 * other values. */
#define SPH_LINES_THOMAS 0
#define SPH_LINES_PARTITIONED 1
#define SPH_LINES_PARTITIONED_WARP 2
#define SPH_LINES_PARTITIONED_NARROW 3
int sph_set_line_solver(sph_ctx* ctx, int which);

/* Tile shape of the stencil kernels (coefficients, right-hand side): blocks of
 * 128 threads over 128/(tj*ti) phi points x tj theta rows x ti r rows; tj, ti
 * powers of two with tj*ti <= 8 (SPH_ERR_ARG otherwise).  Default 1 x 1 (one
 * row of 128 phi points).  The results do not depend on it. */
int sph_set_tile(sph_ctx* ctx, int tj, int ti);

/* Number of this library's kernel launches since creation (for accounting). */
long long sph_launch_count(const sph_ctx* ctx);

/* The bounds-checked debug build (compiled with SPH_CHECKED; the stand-in for
 * a memory checker): every flat index the kernels form from (i, j, k) is
 * checked against its field's extents; a violation is counted, the access is
 * redirected to element 0 and the run goes on.  Returns the number of
 * violations since the last call on the current device and clears it (first:
 * NULL or 4 ints, the field -- 0 centres, 1 u_r, 2 u_theta, 3 u_phi -- and the
 * (i, j, k) of the first), synchronising the device; -1 from a regular build. */
int sph_bounds_report(int* first);

/* Per-kernel timing.  sph_profile(ctx, 1) clears the record and starts timing
 * every kernel stage (one launch, the four of the right-hand side, or the
 * two of a partitioned sweep) with a pair of CUDA events on the context's
 * stream, around the side streams' work; 0
 * stops.  sph_profile_read synchronises the stream and writes, for each kernel
 * kind SPH_K_* (SPH_NKERNELS entries), the summed duration in ms and the stage
 * count (either pointer may be NULL).  At most 65536 stages are recorded;
 * later ones are counted but not timed (the returned count includes them). */
#define SPH_K_AVG 0
#define SPH_K_COEF 1
#define SPH_K_RHS 2
#define SPH_K_SWEEP_R 3
#define SPH_K_SWEEP_TH 4
#define SPH_K_SWEEP_PH 5
#define SPH_NKERNELS 8
int sph_profile(sph_ctx* ctx, int enable);
int sph_profile_read(sph_ctx* ctx, double* ms, long long* count);

void sph_destroy(sph_ctx* ctx);
const char* sph_strerror(int code);

/* Batched 3x3-block tridiagonal solve that allocates no device memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc (a host that forbids allocation after start-up, a plug-in
 * that only receives device pointers, a capture-time memory budget).  It runs
 * the block Thomas elimination of the line sweeps (no pivoting between blocks)
 * on systems the caller assembled:
 *     A_m x_{m-1} + B_m x_m + C_m x_{m+1} = d_m,  m = 0..n-1  (A_0, C_{n-1} unused)
 * for nlines independent lines.  All pointers are device pointers of the current
 * device; blocks are 3x3 row-major, block (l, m) at offset (l*n + m)*9 of A, B,
 * C, and vectors at (l*n + m)*3 of d and x (x may not alias the inputs).
 * Scratch: a file-scope device array of SPH_NOALLOC_MAX_BLOCKS * 12 doubles
 * (12.6 MB) that every GPU loading the library holds until exit; nlines*n above
 * SPH_NOALLOC_MAX_BLOCKS returns SPH_ERR_ARG.  The first call on a device looks
 * up the array's device address, so make it before any stream capture.  The
 * work is queued on `stream` (NULL = legacy default) and the call returns
 * without synchronising; a zero pivot fills that line's x with NaN.  Every call
 * shares the one array, so calls that overlap on the GPU (other streams, other
 * host threads) race: serialise them. */
#define SPH_NOALLOC_MAX_BLOCKS 131072
int sph_block_thomas_noalloc(int nlines, int n, const double* A, const double* B, const double* C,
                             const double* d, double* x, void* stream);

/* The partitioned (Schur-complement) block Thomas algorithm for lines whose
 * blocks are split across P ranks (Section 2.2: the block Thomas algorithm
 * parallelised by a Schur complement over the subdomains of a line).  Rank p
 * holds m >= 2 consecutive blocks of each of nlines lines,
 *   A_i x_{i-1} + B_i x_i + C_i x_{i+1} = d_i,  i = 0..m-1,
 * where x_{-1} is rank p-1's last block and x_m rank p+1's first (cyclic: rank
 * 0 and rank P-1 are neighbours; walled: rank 0's A_0 and rank P-1's C_{m-1}
 * are zero).  Layouts: 3x3 row-major blocks, block (l, i) at (l*m + i)*9 of A,
 * B, C, V, W and at (l*m + i)*3 of d, Y, x.  Device pointers; nothing is
 * allocated (the caller passes scratch); work on `stream`; each call
 * synchronises to report a zero pivot as SPH_ERR_SINGULAR (except back).
 *  1. sph_schur_local: the segment's own solves T y = d, T V = A_0 e_0,
 *     T W = C_{m-1} e_{m-1} (T without the outer couplings), so that
 *     x = y - V x_{-1} - W x_m.  scratch: 30 * nlines * m doubles.
 *  2. Every rank gathers every rank's interface rows: per line 42 doubles,
 *     V_0, V_{m-1}, W_0, W_{m-1} (9 each) then y_0, y_{m-1} (3 each), laid out
 *     iface[(p * nlines + l) * 42 + ...].  sph_schur_reduced solves the 6P x 6P
 *     system of the ranks' first and last blocks (dense, partial pivoting;
 *     P <= 8) into z[((l * 2P) + 2p) * 3 + r] (first block of rank p) and
 *     [.. + 2p + 1 ..] (its last block).
 *  3. sph_schur_back: x = y - V xl - W xr with xl = rank p-1's last block and
 *     xr = rank p+1's first block from z (zero past a walled end), 3 values per
 *     line each.
 * flag: one device int of scratch. */
int sph_schur_local(int nlines, int m, const double* A, const double* B, const double* C, const double* d,
                    double* scratch, double* Y, double* V, double* W, int* flag, void* stream);
int sph_schur_reduced(int nlines, int P, int cyclic, const double* iface, double* z, int* flag, void* stream);
int sph_schur_back(int nlines, int m, const double* Y, const double* V, const double* W, const double* xl,
                   const double* xr, double* x, void* stream);

#ifdef __cplusplus
}
#endif
#endif
