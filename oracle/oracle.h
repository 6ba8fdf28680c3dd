/*
 * oracle.h -- plain FP64 CPU reference of the direction-split, Picard-iterated
 * Crank-Nicolson scheme of Frolov, Minev & Takhirov (arXiv 2004.13887) for the
 * weakly compressible Navier-Stokes equations in spherical coordinates.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA library in paper_2004_13887_gb300/.
 *
 * Layout (all arrays C order, phi fastest, FP64):
 *   p, T : nr * nt * np              cell centres  (p and T are perturbations
 *                                     about an optional radial background)
 *   ur   : (nr+1) * nt * np          r-faces   (faces 0 and nr are walls)
 *   ut   : nr * (nt+1) * np          theta-faces (faces 0 and nt are walls)
 *   up   : nr * nt * npf             phi-faces, npf = np+1 (walls at 0, np)
 *                                     or npf = np when phi is periodic
 * Background tables bgp, bgT hold nr+2 values: index 0 is the ghost below
 * r1, index nr+1 the ghost above r2 (NULL = zero background).
 *
 * Wall data (18 optional arrays, NULL = 0): w[(c*3+d)*2+s] is velocity
 * component c (0=r,1=theta,2=phi) on the wall normal to direction d at side s
 * (0 = low, 1 = high).  For d != c it is the tangential wall value used by the
 * ghost rule ghost = 2*w - interior; for d == c it is the normal velocity on
 * the boundary face, copied into the state at the start of a step.
 *   c=r : d=theta (nr+1)*np, d=phi (nr+1)*nt, d=r  nt*np
 *   c=th: d=r (nt+1)*np,     d=phi nr*(nt+1), d=th nr*np
 *   c=ph: d=r nt*npf,        d=th nr*npf,     d=ph nr*nt
 *
 * All functions return 0 on success, negative on bad arguments.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nr, nt, np, periodic;
  double r1, r2, t1, t2, p1, p2;
} og_grid;

typedef struct {
  double gamma, cv, Pr, mu, pinf, g, omega;
} og_par;

/* Line solvers (Section 2.2: block Thomas; cyclic variants for periodic phi).
 * Blocks are 3x3 row-major, 9 doubles per block; rhs/x 3 doubles per block. */
int og_thomas(int n, const double* a, const double* b, const double* c,
              const double* d, double* x);
int og_cyclic_thomas(int n, const double* a, const double* b, const double* c,
                     const double* d, double* x);
int og_block_thomas(int n, const double* A, const double* B, const double* C,
                    const double* d, double* x);
int og_block_cyclic(int n, const double* A, const double* B, const double* C,
                    const double* d, double* x);

/* Apply one split operator with coefficients frozen at Ubar (App. B):
 * which = 0 (D_r), 1 (D_theta), 2 (D_phi), 3 (D_M).  V is the operand with its
 * own background (vbgp, vbgT may be NULL) and wall data vw (array of 18).
 * out[5] receives the rows at the unknown locations (zero elsewhere). */
int og_apply(const og_grid* g, const og_par* par,
             const double* const* Ubar, const double* bgp, const double* bgT,
             const double* const* ubw, int which,
             const double* const* V, const double* vbgp, const double* vbgT,
             const double* const* vw, double* const* out);

/* Assemble the tau/2-scaled line system (I + tau/2 D_d) along one line.
 * dir: 0 r, 1 theta, 2 phi.  kind 0 = 3x3 block system in (p,T,u_d);
 * kind 1/2 = scalar system of the first/second transverse velocity.
 * (a,b) index the line: dir r -> (j,k), theta -> (i,k), phi -> (i,j), in the
 * index space of the unknown (faces for the transverse velocity component).
 * Writes n blocks (or n scalars) into A,B,C; returns n (line length) or <0. */
int og_line_system(const og_grid* g, const og_par* par,
                   const double* const* Ubar, const double* bgp, const double* bgT,
                   const double* const* ubw, int dir, int kind, int a, int b,
                   double tau, double* A, double* B, double* C);

/* Right-hand side of eq. (spl1) in the paper's form. */
int og_rhs(const og_grid* g, const og_par* par, const double* bgp, const double* bgT,
           const double* const* Un, const double* const* wn,
           const double* const* Uk, const double* const* wk,
           double tau, const double* const* S, double* const* R);

/* One directional sub-step (eqs. spl1-spl3): solve (I + tau/2 D_dir(Ubar)) x = rhs
 * line by line, Ubar = (Un+Uk)/2 with walls (wn+wk)/2. */
int og_sweep(const og_grid* g, const og_par* par, const double* bgp, const double* bgT,
             const double* const* Un, const double* const* wn,
             const double* const* Uk, const double* const* wk,
             double tau, int dir, const double* const* rhs, double* const* x);

/* One time step (eq. splitting2 iterated K times).  U (5 arrays) is updated in
 * place.  wn / wnp1: wall data at t^n and t^{n+1} (arrays of 18, entries may be
 * NULL; the whole array may be NULL).  S: source at t^{n+1/2} (NULL = none).
 * resid (5 doubles, may be NULL): RMS of the last increment per field. */
int og_step(const og_grid* g, const og_par* par, const double* bgp, const double* bgT,
            double* const* U, const double* const* wn, const double* const* wnp1,
            double tau, int K, const double* const* S, double* resid);

#ifdef __cplusplus
}
#endif
#endif
