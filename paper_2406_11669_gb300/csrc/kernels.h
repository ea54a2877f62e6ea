// Host-side launchers of the CUDA kernels (each .cu file owns its kernels).
#pragma once

#include <cuda_runtime.h>

#include "layout.h"

namespace asterx {

struct StageArgs {
  Blk b;
  Ws w;
  int recon;
  int gauge;
  int flux;    // 0 HLLE, 1 Lax-Friedrichs
  int efield;  // 0 upwind constrained transport, 1 flux constrained transport
  double gamma, rho_atm, K_atm, gamma_atm, c2p_tol, W_max, xi;
  double gfac;  // Gamma / (Gamma - 1)
  int c2p_maxiter, brent_maxiter, use_fallback;
};

cudaError_t launch_prepare(const Blk& b, const CF16& m, const Ws& w, cudaStream_t s);
// only the centre record (NCG fields at cg)
cudaError_t launch_prepare_centre(const Blk& b, const CF16& m, double* cg, cudaStream_t s);

// ghost fill of the 9 state fields (with linear extrapolation of A under copy BCs) or of the 5 primitives
cudaError_t launch_ghost_state(const Blk& b, const F9& U, cudaStream_t s);
cudaError_t launch_ghost_prims(const Blk& b, const F5& P, cudaStream_t s);

// B~ = curl A on faces, then the undensitised centre field of every cell
cudaError_t launch_bfield(const Blk& b, const Ws& w, const F9& U, cudaStream_t s);

// ghost layers of the state (record field Us) of every block of a table: exchange between the blocks of a
// tiling (device, may be null), then the boundary-condition sweeps
cudaError_t launch_batch_ghosts(const BlockRec* tab, const long* off, const long* host_total, int nb,
                                const Tiling* tiling, cudaStream_t s);

// u^i = W v^i at every cell into w.uvel (primitives with ghosts)
cudaError_t launch_uvel(const Blk& b, const Ws& w, const F5& P, cudaStream_t s);

// T_{mu nu} at the owned vertices (g..g+n per axis) into T (10 fields: tt, tx, ty, tz, xx, xy, xz, yy, yz, zz)
// from the primitives, w.uvel and w.bc (launch_bfield and launch_uvel first) and the vertex metric m
cudaError_t launch_tmunu(const Blk& b, const Ws& w, double gamma, const CF16& m, const F5& P, double* const T[10],
                         cudaStream_t s);

// conserved variables of every cell from primitives (needs launch_bfield first)
cudaError_t launch_prim2con(const StageArgs& a, const F9& U, const F5& P, cudaStream_t s);

// recovery on interior cells (needs launch_bfield first); flags/stats may be null
cudaError_t launch_c2p(const StageArgs& a, const F9& U, const F5& P, signed char* flags,
                       unsigned long long* stats, cudaStream_t s);
// the recovery on the interior cells lo..hi (inclusive) only, without flags or counters
cudaError_t launch_c2p_range(const StageArgs& a, const F9& U, const F5& P, const int lo[3], const int hi[3],
                             cudaStream_t s);

// right-hand side (stage < 0) or RK4 stage combine (stage 0..3): faces, edges, vertices and cells.
// Needs launch_bfield on U_s and primitives with ghosts.
cudaError_t launch_rhs(const StageArgs& a, const F9& Us, const F5& P, int stage, double dt, const F9& Un,
                       const F9& Unext, const F9& Uacc, const F9& dU, cudaStream_t s);

// one RK4 stage of every block of a device table (one launch per kernel); tab holds nb records of this stage,
// off the NKIND * (nb + 1) item offsets (device), host_total the NKIND totals (host); with a (device) tiling the
// ghost layers between blocks are filled from the neighbours before the boundary-condition sweeps
cudaError_t launch_batch_stage(const StageArgs& a, const BlockRec* tab, const long* off, const long* host_total,
                               int nb, int stage, double dt, unsigned long long* stats, cudaStream_t s,
                               const Tiling* tiling = nullptr);

// ---- adjoint ----
// accumulators cleared together at the start of each right-hand-side adjoint (contiguous, in this order)
constexpr int ADJ_ACC_FIELDS = 9 + 5 + 3 + 3 + 3 + 3 * NFD + 1 + 3 + 3;

// One stage's forward intermediates, kept from its forward pass for its reverse sweep: the primitives recovered
// at the stage state and their flags, the face and centre field, u = W v, the face data and reconstruction of
// every direction, and the face solves' roots.  KEEP_FIELDS fields (the flags take one).
constexpr int KEEP_FIELDS = 5 + 3 + 3 + 3 + 3 * NFD + 6 * NREC + 12 + 1;

struct AdjWs {
  F9 Y;            // the state the right-hand side is linearised at (a copy; ghost-filled, atmosphere-reset)
  F9 mu;           // adjoint of dU/dt (owned ranges read)
  // the stage's kept forward intermediates
  F5 P;             // primitives recovered from Y (the entry values are the guess)
  signed char* flags;
  double *kbf, *kbc, *kuvel, *kface;  // face B~ (3), centre B (3), u (3), face data (3 NFD)
  double* rec3[3];  // reconstructed values of each direction (2 NREC fields each)
  double* roots;    // 12 fields: the face solves' roots (lambda_+, lambda_- of left and right) per direction
  double* lY_base;  // start of the ADJ_ACC_FIELDS accumulators
  double* lY;       // 9: result, adjoint of Y
  double* lP;       // 5: primitives
  double* lu;       // 3: u = W v
  double* lBc;      // 3: centre field
  double* lBf;      // 3: face field B~
  double* lface;    // 3 * NFD: face data
  double* lGA;      // 1: G_A at vertices
  double* lFpsi;    // 3: F_Psi at vertices
  double* lAv;      // 3: vertex-averaged A
  double* lrec;     // 2 * NREC: reconstructed values of the current direction
};

struct AdjGhost {
  double* f[9];
  int cl[9];
  int lin[9];
};

// u = W v, then per direction D the reconstruction into rec[D] (2 NREC fields) and the face solve (face data of
// direction D in the workspace, its roots into `roots`, 12 fields); no right-hand side is formed
cudaError_t launch_face_data(const StageArgs& a, const F5& P, double* const rec[3], double* roots, cudaStream_t s);
// the forward pass of one stage at a.Y into the kept intermediates of a (ghost fill of a.Y, B~ and B, recovery
// into a.P with a.flags, primitive ghost fill, u and the face data of every direction); no right-hand side
cudaError_t launch_adjoint_forward(const StageArgs& sa, const AdjWs& a, cudaStream_t s);
// the right-hand side's remaining steps (vertex potentials, UCT edges, Psi, cells with the RK combine) from the
// kept intermediates of a: forms dU (stage < 0) or the stage's RK4 update, as launch_rhs does
cudaError_t launch_rhs_from_kept(const StageArgs& sa, const AdjWs& a, int stage, double dt, const F9& Un,
                                 const F9& Unext, const F9& Uacc, const F9& dU, cudaStream_t s);
// lambda = (dL/dY)^T mu from the kept intermediates (the reverse sweep alone)
cudaError_t launch_adjoint_reverse(const StageArgs& sa, const AdjWs& a, double dt, cudaStream_t s);
// forward pass, then reverse sweep
cudaError_t launch_rhs_adjoint(const StageArgs& sa, const AdjWs& a, double dt, cudaStream_t s);
// adjoint of the initial data U = (prim2con(P, B(A)), A, Psi) at the state a.Y (copy; ghost-filled here):
// lamP (interior cells) and a.lY (A, Psi entries; independent ranges) from lamU
cudaError_t launch_prim2con_adjoint(const StageArgs& sa, const AdjWs& a, const F9& lamU, const F5& lamP,
                                    cudaStream_t s);
void launch_ghost_adjoint(const Blk& b, const AdjGhost& g, int nf, cudaStream_t s);
// y = alpha x + beta y over every entry of 9 fields; zero the entries outside the owned ranges of 9 fields
cudaError_t launch_axpby9(const Blk& b, double alpha, const F9& x, double beta, const F9& y, cudaStream_t s);
cudaError_t launch_mask_owned9(const Blk& b, const F9& x, cudaStream_t s);

// two refinement levels: a fine block (spacing / 2) whose interior covers the coarse interior cells L .. L + n_f/2
// - 1; prolongation of the 9 state fields and 5 primitives to the fine ghost points (every point if all), and
// restriction of the 9 state fields to the coarse points under the fine interior
cudaError_t launch_prolong(const Blk& C, const Blk& F, const int L[3], const F9& Uc, const F5& Pc, const F9& Uf,
                           const F5& Pf, bool all, cudaStream_t s);
// subcycling: out = U_n + sum_i beta_i h k_i with the coarse slopes recovered from U_n, Y_1..Y_3 and U_1 (the
// points lo..hi, inclusive, of the padded block, 9 fields)
cudaError_t launch_subcycle_combine(const Blk& b, const int lo[3], const int hi[3], const F9& un, const F9& y1,
                                    const F9& y2, const F9& y3, const F9& u1, const F9& out, const double beta[4],
                                    cudaStream_t s);
cudaError_t launch_restrict(const Blk& C, const Blk& F, const int L[3], const F9& Uc, const F9& Uf, cudaStream_t s);

// face-kernel launch timing (measurement hook of the benchmark)
cudaError_t profile_enable(int cap);
void profile_disable();
cudaError_t profile_read(int* launches, double* total_ms);

// streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, read once per device);
// grid caps of grid-stride kernels are multiples of it
int device_sm_count();

// FP64 fused multiply-add throughput probe (measurement helper)
cudaError_t launch_dfma_probe(double* out, int blocks, int threads, long iters, cudaStream_t s);
// the quartic solver's Newton-correction reciprocal on n values (measurement helper)
cudaError_t launch_newton_rcp(const double* d, double* out, long n, cudaStream_t s);
// the two-step reciprocal of the face solve, the WENO-Z weights and the Noble iteration (measurement helper)
cudaError_t launch_recip(const double* d, double* out, long n, cudaStream_t s);
// the corrected quotient a / b from 1 / b (measurement helper)
cudaError_t launch_quotient(const double* a, const double* b, double* out, long n, cudaStream_t s);

}  // namespace asterx
