/*
 * asterx.h -- C ABI of the GB300 (sm_103a) library for one method-of-lines RK stage of the Valencia GRMHD
 * equations on uniform Cartesian blocks over a frozen 3+1 metric (AsterX, arXiv:2406.11669).
 *
 * Method (paper sections): Valencia conservative form (Sec. 2.2, Eqs. fluxconseqs, grmhdeqs, grmhdsrc, cons);
 * vector potential on edges with B~ = curl A on faces and the generalised Lorenz gauge (Sec. 2.3, 3.4, Eqs.
 * BEulerian, Ainductioneqs, recastedAvec, recastedScalarPot); minmod / PPM / WENO-Z / MP5 reconstruction and HLLE
 * fluxes with magnetosonic speeds (Sec. 3.3, Eq. HLLEfluxes); upwind constrained transport (Sec. 3.4, Eqs.
 * uct1, uct2, eq3.20); Noble 2D recovery with a Palenzuela 1D fallback and atmosphere (Sec. 3.5, 3.6);
 * ideal-gas EOS (Sec. 3.7); 4th-order vertex-metric interpolation (Sec. 3.2); classical RK4 (Sec. 5).
 *
 * Data layout.  A block has n[d] interior cells and g = 3 ghost layers per side; N = n + 2g.  Every field is a
 * contiguous array of (N[0]+1)(N[1]+1)(N[2]+1) doubles, x fastest: index(i,j,k) = i + (N0+1)(j + (N1+1) k).
 * Index (i,j,k) names the object whose lower corner is vertex (i,j,k): cell centre (i+1/2, j+1/2, k+1/2),
 * x-face (i, j+1/2, k+1/2), x-edge (i+1/2, j, k), vertex (i, j, k).  Vertex i lies at x0 + (i - g) dx.
 *   state:  D~, S~x, S~y, S~z, tau~ (cells, densitised by sqrt(gamma)); A_x, A_y, A_z (edges); Psi (vertices)
 *   prims:  rho, p, v^x, v^y, v^z (cells; v^i Eulerian; eps = p / ((Gamma - 1) rho))
 *   metric: alpha, beta^x,y,z, gamma_xx,xy,xz,yy,yz,zz, K_xx,xy,xz,yy,yz,zz (vertices)
 *
 * Ownership.  The caller owns every pointer.  All array pointers are DEVICE pointers (8-byte aligned) unless a
 * comment says HOST.  The library never allocates: each call uses the caller's workspace `ws` of at least
 * asterx_workspace_size() bytes (256-byte aligned).  The workspace holds the frozen-metric geometry written by
 * asterx_prepare(), so one workspace serves one (block, metric) pair; pass it unchanged to the later calls.
 *
 * Execution.  Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy default stream) and
 * returns after enqueueing.  Device-side counters are written to device memory and read only after the caller
 * synchronises.  Calls on different streams with different workspaces are independent; calls that share a
 * workspace must be ordered by the caller.  The first launch of a kernel at a new item count outside stream
 * capture times the launch shapes the library can use (threads per block, grid, pencil length) and so waits for
 * the stream once; every shape computes the same results bit for bit.  Environment: ASTERX_AUTOTUNE=0 turns the
 * timing off (default shapes); with it off, ASTERX_PENCIL=16 selects the long pencils.
 *
 * Errors.  Argument errors are detected on the host before any launch (ASTERX_EINVAL); launch failures return
 * ASTERX_ECUDA.  Nothing aborts, throws across the ABI or traps on the device.  Recovery failures are soft: a
 * cell whose recovery fails gets the atmosphere and flag -1, and the per-call counters record it.
 */
#ifndef ASTERX_H
#define ASTERX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *asterx_stream; /* a cudaStream_t */

typedef enum {
  ASTERX_OK = 0,
  ASTERX_EINVAL = 1,   /* invalid argument (host check, nothing launched) */
  ASTERX_ECUDA = 2,    /* a CUDA launch or runtime call failed */
  ASTERX_ENOMEM = 3,   /* workspace smaller than asterx_workspace_size() */
  ASTERX_EC2P = 4,     /* reserved: soft recovery failures are reported through the counters */
  ASTERX_ETIMEOUT = 5  /* a bounded device-side wait gave up */
} asterx_status;

/* Reconstruction of the face states (Sec. 3.3 lists minmod, PPM, WENO-Z and MP5 among its methods). */
typedef enum {
  ASTERX_RECON_MINMOD = 0,
  ASTERX_RECON_PPM = 1,
  ASTERX_RECON_WENOZ = 2,
  ASTERX_RECON_MP5 = 3 /* Suresh & Huynh 1997, alpha = 4 */
} asterx_recon;
typedef enum { ASTERX_BC_PERIODIC = 0, ASTERX_BC_COPY = 1 } asterx_bc;
typedef enum { ASTERX_GAUGE_LORENZ = 0, ASTERX_GAUGE_ALGEBRAIC = 1 } asterx_gauge;
typedef enum { ASTERX_FLUX_HLLE = 0, ASTERX_FLUX_LXF = 1 } asterx_flux;
typedef enum { ASTERX_EFIELD_UCT = 0, ASTERX_EFIELD_FCT = 1 } asterx_efield;

/* Physics parameters (HOST struct, read during the call). */
typedef struct {
  double gamma;        /* ideal-gas adiabatic index, P = (Gamma-1) rho eps (Sec. 3.7) */
  double rho_atm;      /* atmosphere density: D~ < sqrt(gamma) rho_atm => atmosphere (Sec. 3.6) */
  double K_atm;        /* atmosphere polytrope P = K rho^Gamma_atm (Sec. 3.7) */
  double gamma_atm;
  double c2p_tol;      /* Noble Newton tolerance on |dz|/z and |dv^2| (e.g. 1e-13) */
  int c2p_maxiter;     /* Noble iteration cap (e.g. 100) */
  int brent_maxiter;   /* Palenzuela/Brent iteration cap (e.g. 300) */
  double W_max;        /* Lorentz-factor cap used on failure paths of the recovery (e.g. 50) */
  int recon;           /* asterx_recon */
  int gauge;           /* asterx_gauge; the generalised Lorenz gauge is the paper's default (Sec. 3.4) */
  double xi_lorenz;    /* Lorenz damping xi; 0 => 1.5 / dt (Sec. 3.4) */
  int use_fallback;    /* 1: Palenzuela fallback after a Noble failure */
  int flux;            /* asterx_flux: HLLE (Eq. HLLEfluxes, the default) or Lax-Friedrichs (Eq. LxFfluxes,
                          c_wave = max(c_max, c_min)) for the hydro fluxes */
  int efield;          /* asterx_efield: upwind constrained transport (Sec. 3.4 (i)-(iii), Eq. eq3.20, the
                          default) or flux constrained transport (Sec. 3.4: the average of the induction-equation
                          fluxes, from the same Riemann solver, on the four faces sharing an edge) */
} asterx_params;

/* Geometry of one block (HOST struct). */
typedef struct {
  int n[3];       /* interior cells per axis, >= 1 */
  int g;          /* ghost layers, must be 3 */
  double x0[3];   /* position of the first interior vertex */
  double dx[3];   /* grid spacing, > 0 */
  int bc[3];      /* asterx_bc per axis (both sides) */
} asterx_block;

/* Field pointer sets (HOST structs holding DEVICE pointers). */
typedef struct { double *D, *Sx, *Sy, *Sz, *tau, *Ax, *Ay, *Az, *Psi; } asterx_state;
typedef struct { const double *alp, *betax, *betay, *betaz, *gxx, *gxy, *gxz, *gyy, *gyz, *gzz,
                 *kxx, *kxy, *kxz, *kyy, *kyz, *kzz; } asterx_metric;
typedef struct { double *rho, *press, *velx, *vely, *velz; } asterx_prims;

/* Recovery counters (DEVICE memory, accumulated with atomics; the caller zeroes them when it wants). */
typedef struct {
  unsigned long long n_noble;     /* cells recovered by Noble 2D */
  unsigned long long n_fallback;  /* cells recovered by Palenzuela 1D after Noble failed */
  unsigned long long n_atm;       /* cells set to the atmosphere by the density test */
  unsigned long long n_failed;    /* cells where both solvers failed (atmosphere applied, flag -1) */
  unsigned long long iters;       /* total Noble iterations */
} asterx_c2p_stats;

/* ABI version of this header (checked by the binding). */
int asterx_abi_version(void);

/* Human-readable name of a status code (static string). */
const char *asterx_status_str(asterx_status s);

/* Bytes of workspace a block needs (0 if the block is invalid). */
size_t asterx_workspace_size(const asterx_block *blk);

/* Derive the frozen-metric geometry (Sec. 3.2: 4th-order Lagrange interpolation of the vertex metric to
 * centres and faces, 4th-order centre derivatives for the sources, inverse metric and sqrt(gamma)) into `ws`.
 * Must precede every other call that takes this workspace.  `metric` points to 16 device arrays. */
asterx_status asterx_prepare(const asterx_params *p, const asterx_block *blk, const asterx_metric *metric,
                             void *ws, size_t ws_bytes, asterx_stream stream);

/* Conserved variables from primitives (Eq. cons) at every cell of the padded block, with B~ = curl A of the
 * state's edge potential (Eq. BEulerian).  Reads P and U's A; writes U's D~, S~, tau~. */
asterx_status asterx_prim2con(const asterx_params *p, const asterx_block *blk, asterx_state *U,
                              const asterx_prims *P, void *ws, size_t ws_bytes, asterx_stream stream);

/* Primitive recovery on the interior cells (Sec. 3.5, 3.6): P holds the previous primitives (initial guess)
 * on entry and the recovered ones on exit; cells set to the atmosphere have U's D~, S~, tau~ reset in place.
 * `flags` (device, one signed char per array entry, may be NULL): 0 Noble, 1 Palenzuela, 2 atmosphere by the
 * density test, -1 both solvers failed.  `stats` (device, may be NULL) is accumulated.  U's ghosts must be
 * filled (A is differentiated across the block). */
asterx_status asterx_con2prim(const asterx_params *p, const asterx_block *blk, asterx_state *U,
                              asterx_prims *P, signed char *flags, asterx_c2p_stats *stats, void *ws,
                              size_t ws_bytes, asterx_stream stream);

/* Ghost fill of the 9 state fields (periodic wrap, or copy of the nearest owned value with linear
 * extrapolation of A along the normal), in place. */
asterx_status asterx_fill_ghosts(const asterx_params *p, const asterx_block *blk, asterx_state *U, void *ws,
                                 size_t ws_bytes, asterx_stream stream);

/* Right-hand side dU/dt of the 9 state fields (Sec. 3.12 workflow, Sec. 3.4): U and P must have their ghosts
 * filled (P after recovery).  Writes dUdt at the interior cells, at the edges/vertices of the owned range
 * (indices g..g+n along vertex-like axes, g..g+n-1 along cell-like axes), and nowhere else.  `dt` only sets
 * the Lorenz damping when xi_lorenz == 0. */
asterx_status asterx_rhs(const asterx_params *p, const asterx_block *blk, const asterx_state *U,
                         const asterx_prims *P, asterx_state *dUdt, double dt, void *ws, size_t ws_bytes,
                         asterx_stream stream);

/* One classical RK4 stage (stage = 0..3): ghost fill U_s, recovery on the interior (resetting U_s for
 * atmosphere cells), ghost fill of P, RHS k_s, then U_next = U_n + c dt k_s (c = 1/2, 1/2, 1) and U_acc += b dt
 * k_s (b = 1/6, 1/3, 1/3; stage 0 initialises U_acc); stage 3 writes U_next = U_n + U_acc + dt/6 k_3.  Us may
 * alias Un (stage 0).  Unext and Uacc are written on the owned ranges only. */
asterx_status asterx_rk_stage(const asterx_params *p, const asterx_block *blk, int stage, double dt,
                              const asterx_state *Un, asterx_state *Us, asterx_state *Unext, asterx_state *Uacc,
                              asterx_prims *P, signed char *flags, asterx_c2p_stats *stats, void *ws,
                              size_t ws_bytes, asterx_stream stream);

/* One full RK4 step in place: U <- U_{n+1}, using stage buffers inside the workspace.  P is updated to the
 * primitives recovered in the last stage.  `flags` and `stats` as in asterx_con2prim (accumulated over the
 * four stages). */
asterx_status asterx_rk4_step(const asterx_params *p, const asterx_block *blk, double dt, asterx_state *U,
                              asterx_prims *P, signed char *flags, asterx_c2p_stats *stats, void *ws,
                              size_t ws_bytes, asterx_stream stream);

/* HOST-buffer variant of asterx_rk4_step for callers without device memory management: copies U and P from
 * host (pinned for asynchrony) to the device buffers dU/dP, runs the step and copies U and P back.  The
 * device buffers have the same layout; `h_*` are HOST pointers.  The copy of P back to the host starts on an
 * internal second stream as soon as the last stage's primitives are final, while that stage's right-hand side
 * and the state update still run.  Synchronous at return (both streams). */
asterx_status asterx_rk4_step_host(const asterx_params *p, const asterx_block *blk, double dt,
                                   double *const *h_U9, double *const *h_P5, asterx_state *dU, asterx_prims *dP,
                                   asterx_c2p_stats *stats, void *ws, size_t ws_bytes, asterx_stream stream);

/* One RK2 step in place (Sec. 5 compares RK2 with RK4; read as the explicit midpoint method):
 * U_1 = U_n + dt/2 L(U_n), U_{n+1} = U_n + dt L(U_1), each stage with ghost fill and recovery as in
 * asterx_rk_stage.  Otherwise as asterx_rk4_step. */
asterx_status asterx_rk2_step(const asterx_params *p, const asterx_block *blk, double dt, asterx_state *U,
                              asterx_prims *P, signed char *flags, asterx_c2p_stats *stats, void *ws,
                              size_t ws_bytes, asterx_stream stream);

/* ---- two refinement levels (fixed box-in-box refinement, one time step for both levels) ----
 *
 * A fine block of half the coarse spacing (dx_fine = dx_coarse / 2 exactly, n_fine even along every axis) whose
 * interior covers the coarse interior cells L .. L + n_fine/2 - 1, with L = (x0_fine - x0_coarse) / dx_coarse
 * integer, L >= 0 and L + n_fine/2 <= n_coarse.  Prolongation (the paper's AMR test, Sec. 4): third-order
 * conservative along cell-centred directions with a minmod-limited linear fallback for both halves of a coarse
 * cell where either would leave its three coarse averages' range; cubic interpolation along vertex-centred
 * directions.  Restriction: the mean of the fine points covering a coarse point.
 *
 * asterx_prolong fills the fine block's ghost points (all != 0: every point, e.g. for initial data) of the 9
 * state fields and 5 primitives from the coarse arrays (their ghosts filled where the stencil reaches them). */
asterx_status asterx_prolong(const asterx_block *coarse, const asterx_block *fine, const asterx_state *Uc,
                             const asterx_prims *Pc, asterx_state *Uf, asterx_prims *Pf, int all,
                             asterx_stream stream);

/* One RK4 step of both levels with the fine time step dt: per stage, the coarse stage (asterx_rk_stage), the
 * prolongation of the coarse stage state and recovered primitives to the fine ghost points, and the fine stage
 * on them (no ghost fill of its own); after the step the coarse points under the fine interior are restricted.
 * ws_c / ws_f: the two blocks' prepared workspaces.  flags are not written; stats (may be NULL) accumulates both
 * levels. */
asterx_status asterx_rk4_step_refined(const asterx_params *p, const asterx_block *coarse, const asterx_block *fine,
                                      double dt, asterx_state *Uc, asterx_prims *Pc, asterx_state *Uf,
                                      asterx_prims *Pf, asterx_c2p_stats *stats, void *ws_c, size_t ws_c_bytes,
                                      void *ws_f, size_t ws_f_bytes, asterx_stream stream);

/* Subcycling in time (Sec. 3.10; the paper defers its method, so this follows the published stage-consistent
 * form of Mongwane 2015): one RK4 step of size dt on the coarse level and two of dt/2 on the fine one, with no
 * buffer zones.  The coarse step runs first and keeps its base U_n, stage states Y_1..Y_3 and result; before
 * each fine stage the coarse state U_n + sum_i beta_i h k_i is formed from them (the coarse step's dense
 * output and its time derivatives at the substep start, combined as the fine stage states of a linear problem:
 * fourth-order accurate ghost data), ghost-filled, recovered (seeded by the previous such recovery, starting
 * from the primitives the coarse step leaves) and prolonged to the fine ghost points as asterx_prolong does;
 * it is formed and recovered only on the coarse cells the prolongation reads (with the margin the field
 * needs), or along whole axes where those reach the boundary.
 * After both fine steps the coarse points under the fine interior are restricted.  ws_c / ws_f: the two
 * blocks' prepared workspaces; ws_t: scratch of asterx_subcycle_workspace_size(coarse) bytes (256-byte
 * aligned).  The Lorenz damping (xi_lorenz = 0) is 1.5 / dt on the coarse level and 3 / dt on the fine one.
 * flags are not written; stats (may be NULL) accumulates the stage recoveries of both levels. */
size_t asterx_subcycle_workspace_size(const asterx_block *coarse);
asterx_status asterx_rk4_step_subcycled(const asterx_params *p, const asterx_block *coarse,
                                        const asterx_block *fine, double dt, asterx_state *Uc, asterx_prims *Pc,
                                        asterx_state *Uf, asterx_prims *Pf, asterx_c2p_stats *stats, void *ws_c,
                                        size_t ws_c_bytes, void *ws_f, size_t ws_f_bytes, void *ws_t,
                                        size_t ws_t_bytes, asterx_stream stream);

/* ---- coupling to a spacetime solver ----
 *
 * Stress-energy tensor T_{mu nu} (Eq. tmunu with both indices lowered by the 4-metric; T lives at vertices,
 * Sec. 3.1), the matter input of a spacetime solver.  At every vertex g..g+n of each axis, the rest-mass
 * density, pressure, u^i = W v^i (W from the cell's metric) and centre field B^i of the eight cells around the
 * vertex are averaged to it and combined with the vertex metric of `metric` (alpha, beta^i, gamma_ij).  `ws`
 * must be prepared from the same metric.  U's A and P must have their ghosts filled, as asterx_rk_stage leaves
 * its stage state U_s and P.  Writes the 10 fields of T at those vertices and nowhere else. */
typedef struct { double *tt, *tx, *ty, *tz, *xx, *xy, *xz, *yy, *yz, *zz; } asterx_tmunu_fields;
asterx_status asterx_tmunu(const asterx_params *p, const asterx_block *blk, const asterx_metric *metric,
                           const asterx_state *U, const asterx_prims *P, asterx_tmunu_fields *T, void *ws,
                           size_t ws_bytes, asterx_stream stream);

/* One RK4 step over a time-dependent metric: stage s = 0..3 runs on metric[s], the spacetime of that stage
 * (t_n, t_n + dt/2, t_n + dt/2, t_n + dt for a prescribed metric; the spacetime solver's stage states when the
 * two are integrated together), with the geometry re-derived as asterx_prepare does before each stage.  Each
 * metric's K_ij must be the extrinsic curvature of its slicing (consistent with d gamma_ij / dt), which the
 * source terms use.  Otherwise as asterx_rk4_step; the workspace ends prepared from metric[3].  `metric` is a
 * HOST array of 4 pointers to metric sets (an entry may repeat). */
asterx_status asterx_rk4_step_metrics(const asterx_params *p, const asterx_block *blk, double dt,
                                      const asterx_metric *const *metric, asterx_state *U, asterx_prims *P,
                                      signed char *flags, asterx_c2p_stats *stats, void *ws, size_t ws_bytes,
                                      asterx_stream stream);

/* ---- adjoint (vector-Jacobian products) ----
 *
 * Reverse-mode derivatives of the stage operator and of one RK4 step, for gradients of a scalar loss with
 * respect to the state.  The adjoint recomputes the forward intermediates from the state it is given (a
 * checkpoint), so the caller keeps one state per RK4 step.  Recovery and wave speeds are differentiated by the
 * implicit-function theorem at the converged root; limiters, max/min and branch choices by the branch taken;
 * atmosphere cells pass no derivative through the recovery.  FP64 atomics accumulate shared adjoints, so the
 * last bits may differ from run to run.  Adjoint arrays use the state layout and cover the independent entries
 * only: g..g+n-1 along cell-like axes and along periodic axes (there the vertex index g+n is the periodic image
 * of g), g..g+n along vertex-like axes with copy BCs.  Adjoint inputs are read there only; outputs are zero
 * everywhere else.  `aws` is a second, caller-owned
 * workspace of asterx_adjoint_workspace_size() bytes (256-byte aligned); `ws` is the prepared forward one.
 * Every flux (HLLE, Lax-Friedrichs) and electric-field (UCT, FCT) switch is differentiated; c_wave's max takes
 * c_max's branch on ties. */
size_t asterx_adjoint_workspace_size(const asterx_block *blk);

/* lam = (dL/dU)^T mu for the right-hand side L of asterx_rhs at state U (U unchanged; P: guess in, the
 * primitives recovered from U out). */
asterx_status asterx_rhs_adjoint(const asterx_params *p, const asterx_block *blk, double dt,
                                 const asterx_state *U, asterx_prims *P, const asterx_state *mu,
                                 asterx_state *lam, void *ws, size_t ws_bytes, void *aws, size_t aws_bytes,
                                 asterx_stream stream);

/* Adjoint of one RK stage as asterx_rk_stage forms it (k = L(Us); Unext = Un + c dt k, Uacc' = Uacc + b dt k for
 * stages 0..2; Unext = Un + Uacc + dt/6 k for stage 3): given the adjoints lam_next of Unext and lam_acc of
 * Uacc' (ignored, may be NULL, for stage 3), writes lam_s = (dL/dUs)^T kbar with kbar = c dt lam_next + b dt
 * lam_acc (dt/6 lam_next for stage 3).  The linear parts (Un receives lam_next, Uacc receives lam_acc, or
 * lam_next at stage 3) are the caller's to add.  Us is the stage's input state (a checkpoint; unchanged), P a
 * primitive guess (overwritten by the recovery at Us). */
asterx_status asterx_rk_stage_adjoint(const asterx_params *p, const asterx_block *blk, int stage, double dt,
                                      const asterx_state *Us, asterx_prims *P, const asterx_state *lam_next,
                                      const asterx_state *lam_acc, asterx_state *lam_s, void *ws, size_t ws_bytes,
                                      void *aws, size_t aws_bytes, asterx_stream stream);

/* Adjoint of one classical RK4 step U_{n+1} = Phi(U_n): on entry lam holds dJ/dU_{n+1}, on exit dJ/dU_n.
 * Un is the checkpoint of the step's input state (unchanged); P is a primitive guess (overwritten). */
asterx_status asterx_rk4_step_adjoint(const asterx_params *p, const asterx_block *blk, double dt,
                                      const asterx_state *Un, asterx_prims *P, asterx_state *lam, void *ws,
                                      size_t ws_bytes, void *aws, size_t aws_bytes, asterx_stream stream);

/* Adjoint of the initial data U = (prim2con(P, B~ = curl A), A, Psi): lam holds dJ/dU on entry; on exit its
 * fields A and Psi hold dJ/dA and dJ/dPsi (independent entries) and its hydro fields are zero, and lamP holds
 * dJ/dP at the interior cells (zero elsewhere).  U supplies A (ghosts filled internally on a copy), P the
 * primitives; neither is modified. */
asterx_status asterx_prim2con_adjoint(const asterx_params *p, const asterx_block *blk, const asterx_state *U,
                                      const asterx_prims *P, asterx_state *lam, asterx_prims *lamP, void *ws,
                                      size_t ws_bytes, void *aws, size_t aws_bytes, asterx_stream stream);

/* nsteps RK4 steps in place (asterx_rk4_step), saving the state before step k into ckpt[k] (a host array of
 * nsteps device state structs, each of the block's padded size): the checkpoints of the adjoint below. */
asterx_status asterx_rk4_steps_checkpointed(const asterx_params *p, const asterx_block *blk, double dt, int nsteps,
                                            asterx_state *U, asterx_prims *P, const asterx_state *ckpt,
                                            asterx_c2p_stats *stats, void *ws, size_t ws_bytes,
                                            asterx_stream stream);

/* Adjoint of nsteps RK4 steps from their checkpoints: lam = dJ/dU_N on entry, dJ/dU_0 on exit (steps reversed
 * one by one with asterx_rk4_step_adjoint; P is a primitive guess, overwritten). */
asterx_status asterx_rk4_adjoint_steps(const asterx_params *p, const asterx_block *blk, double dt, int nsteps,
                                       const asterx_state *ckpt, asterx_prims *P, asterx_state *lam, void *ws,
                                       size_t ws_bytes, void *aws, size_t aws_bytes, asterx_stream stream);

/* ---- batched step over many blocks of uneven sizes ----
 *
 * Many AMR-like blocks advance together: every kernel of the stage is launched once for all blocks, over the
 * concatenation of the blocks' item spaces (cells, faces, edges), so small blocks do not each pay a launch per
 * kernel and the GPU sees one large balanced launch.  The blocks are independent (no exchange between them;
 * each keeps its own boundary conditions).  The per-block physics is exactly asterx_rk4_step's. */
typedef struct {
  asterx_block blk;      /* the block's geometry */
  asterx_metric metric;  /* its frozen vertex metric (device) */
  asterx_state U;        /* its state (device; advanced in place) */
  asterx_prims P;        /* its primitives (device; guess in, last recovery out) */
} asterx_batch_block;

/* Bytes of the pooled workspace of a batch (0 if a block is invalid): the per-block workspaces plus the
 * device block tables. */
size_t asterx_batch_workspace_size(const asterx_batch_block *blocks, int nblocks);

/* Derive every block's frozen-metric geometry into its slice of the pooled workspace and upload the block
 * tables (host `blocks` array read during the call; returns after the upload has completed on `stream`). */
asterx_status asterx_batch_prepare(const asterx_params *p, const asterx_batch_block *blocks, int nblocks,
                                   void *ws, size_t ws_bytes, asterx_stream stream);

/* Ghost fill of every block's state and its conserved variables from its primitives (Eq. cons). */
asterx_status asterx_batch_prim2con(const asterx_params *p, const asterx_batch_block *blocks, int nblocks,
                                    void *ws, size_t ws_bytes, asterx_stream stream);

/* `nsteps` classical RK4 steps of every block (the same `blocks` array as asterx_batch_prepare); `stats`
 * (device, may be NULL) accumulates the recovery counters of all blocks and stages.  The first call captures
 * one RK4 step (4 stages x 28 launches) as a CUDA graph on a private stream and caches it (host memory, guarded
 * by a mutex) for the workspace and launch parameters (dt, stats, params); this and later calls with the same
 * parameters replay it.  Inside the caller's own stream capture the launches are issued directly. */
asterx_status asterx_batched_step(const asterx_params *p, const asterx_batch_block *blocks, int nblocks,
                                  double dt, int nsteps, asterx_c2p_stats *stats, void *ws, size_t ws_bytes,
                                  asterx_stream stream);

/* Drops the step graphs cached for pooled workspace `ws` (call before freeing it; asterx_batch_prepare does it
 * for the workspace it prepares).  EINVAL for a null pointer. */
asterx_status asterx_batch_release(void *ws);

/* A batch whose blocks tile one rectangular domain on a common grid: nblk[0] x nblk[1] x nblk[2] blocks listed x
 * fastest (block bx + nblk[0] (by + nblk[1] bz)); along axis d block b covers the interior cells
 * cuts[d][b] .. cuts[d][b+1]-1 of the domain (cuts[d][0] = 0, every block at least 3 cells wide), all blocks
 * share dx and the domain's boundary conditions, and each block's x0 is the first block's plus cuts * dx.
 * asterx_batch_prepare_tiled replaces asterx_batch_prepare for such a batch: every later asterx_batch_prim2con
 * and asterx_batched_step on this workspace fills the ghost layers a block shares with its neighbours (and
 * across periodic boundaries) from the neighbours' owned values before the boundary-condition sweeps, so the
 * tiled domain evolves as one block covering it would (same-level ghost exchange; no refinement levels).
 * `cuts` are HOST arrays.  Returns ASTERX_EINVAL if the blocks do not tile the domain as described. */
typedef struct {
  int nblk[3];
  const int *cuts[3];
} asterx_tiling;
asterx_status asterx_batch_prepare_tiled(const asterx_params *p, const asterx_batch_block *blocks, int nblocks,
                                         const asterx_tiling *tiling, void *ws, size_t ws_bytes,
                                         asterx_stream stream);

/* ---- recovery for callers that cannot allocate device memory (the paper has no counterpart) ----
 *
 * Some callers cannot call cudaMalloc: a plugin inside a host application that owns all device memory and
 * hands out only the buffers it manages, or a time-critical loop that must not allocate because cudaMalloc
 * can synchronise the device and can fail in the middle of a run.  For them this entry point runs the
 * recovery of asterx_con2prim (the same face-field, centre-field and recovery kernels) without a caller
 * workspace.  Its centre metric record comes from a direct 4x4x4 contraction of the vertex metric instead of
 * asterx_prepare's separable passes; the two agree to rounding, so the recovered primitives agree with
 * asterx_con2prim's to rounding (not bit for bit) and the flags and counters match.  The scratch it needs
 * (the frozen-metric centre record, the face field B~ and the centre field B) lives in one fixed-size array
 * in the library's own device memory, which every GPU that loads the library holds until the process exits
 * ((53 + 6) * ASTERX_NOALLOC_MAX_ENTRIES doubles, about 31 MB).  The caller still passes the inputs and
 * outputs: the vertex metric, the state U (ghosts filled; D~, S~, tau~ reset in place for atmosphere
 * cells), the primitives P (guess in, result out), and optional flags and counters as in asterx_con2prim.
 * It allocates nothing and calls no allocating routine.
 *
 * Limits and rules:
 *  - the block must pass the checks of the workspace entry points (parameters, 3 ghosts, 1..2^20 cells per
 *    axis, finite origin and spacing), and the padded block (n[0]+7)(n[1]+7)(n[2]+7) may hold at most
 *    ASTERX_NOALLOC_MAX_ENTRIES entries per field (for example 33^3 interior cells); other blocks return
 *    ASTERX_EINVAL before anything is launched;
 *  - every call shares the one array, which keeps the last call's contents; calls that overlap on the GPU
 *    (different streams, or different host threads without ordering) race on it and must be serialised by
 *    the caller;
 *  - the first call on each device looks up the array's device address (cudaGetSymbolAddress) with that
 *    device current, and looks it up again when that device's context has changed (after a device reset by
 *    the host application); make the first call, and the first call after a reset, before any stream
 *    capture. */
#define ASTERX_NOALLOC_MAX_ENTRIES 65536L
asterx_status asterx_con2prim_noalloc(const asterx_params *p, const asterx_block *blk,
                                      const asterx_metric *metric, asterx_state *U, asterx_prims *P,
                                      signed char *flags, asterx_c2p_stats *stats, asterx_stream stream);

/* ---- measurement helpers (not part of the method) ---- */

/* Start recording a CUDA event pair around each launch of the face kernel (the dominant kernel: Sec. 3.3
 * face solve) on the stream it is launched on, for at most max_launches launches; resets earlier records.
 * Host-side event creation only (no device memory). */
asterx_status asterx_profile_enable(int max_launches);
/* Number of recorded face-kernel launches and their summed device time in ms (waits for the last event). */
asterx_status asterx_profile_read(int *launches, double *total_ms);
/* Stop recording and release the events. */
void asterx_profile_disable(void);

/* FP64 throughput probe: `blocks` x `threads` threads each run `iters` iterations of 8 independent dependent
 * chains of fused multiply-adds (16 flops per chain step); writes one double per thread to `out` (device,
 * blocks*threads doubles) so the work cannot be elided. */
asterx_status asterx_dfma_probe(double *out, int blocks, int threads, long iters, asterx_stream stream);

/* The reciprocal the magnetosonic-speed Newton iteration (Sec. 3.3) uses for its corrections: out[i] ~ 1/d[i]
 * for n device doubles (a hardware estimate refined by one Newton-Raphson step; relative error far below the
 * iteration's stopping threshold for 1e-290 < |d| < 1e290, the range it is used in).  Lets tests bound its
 * error; not part of the method's interface.  d and out: device, n doubles each, caller-owned. */
asterx_status asterx_newton_rcp(const double *d, double *out, long n, asterx_stream stream);

/* The reciprocal the face solve, the WENO-Z weights and the Noble iteration use where a correctly rounded
 * quotient is not needed: out[i] ~ 1/d[i] for n device doubles (the estimate refined by two Newton-Raphson steps
 * for binary exponents within +-960, the quotient 1/d elsewhere).  Lets tests bound its error; not part of the
 * method's interface.  d and out: device, n doubles each, caller-owned. */
asterx_status asterx_recip(const double *d, double *out, long n, asterx_stream stream);

/* The corrected quotient the recovery and the centre field use to divide by sqrt(gamma) like a division:
 * out[i] = a[i] / b[i] formed from the correctly rounded 1 / b[i] and one correction.  Lets tests check that it
 * equals the correctly rounded quotient; not part of the method's interface.  a, b, out: device, n doubles
 * each, caller-owned. */
asterx_status asterx_quotient(const double *a, const double *b, double *out, long n, asterx_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* ASTERX_H */
