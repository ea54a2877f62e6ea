// Block constants and workspace layout shared by the host runtime and the kernels.
#pragma once

#include <cstddef>

namespace asterx {

// Centre geometry record (per cell): the vertex metric interpolated to the centre at 4th order, its inverse and
// sqrt(det), K_ij, and 4th-order centre derivatives d_i alpha, d_i beta^j, d_i gamma_jk (interior cells only).
enum {
  CG_ALP = 0,
  CG_BETA = 1,    // 3
  CG_G = 4,       // 6 (xx, xy, xz, yy, yz, zz)
  CG_GU = 10,     // 6
  CG_SQG = 16,
  CG_K = 17,      // 6
  CG_DALP = 23,   // 3: d_i alpha
  CG_DBETA = 26,  // 9: d_i beta^j at i*3 + j
  CG_DG = 35,     // 18: d_i gamma_jk at i*6 + sym(j,k)
  NCG = 53
};

// Face geometry record (per face, one set per direction): metric interpolated in the two transverse directions.
// Of the inverse metric the face solve needs gamma^dd alone (the normal component of faces normal to d).
enum { FG_ALP = 0, FG_BETA = 1, FG_G = 4, FG_GUDD = 10, FG_SQG = 11, FG_IALP = 12, FG_ISQG = 13, FG_WIDTH = 14,
       NFG = 15 };  // FG_WIDTH: light-cone half-width alpha sqrt(gamma^dd) along the face normal

// Vertex geometry record: lapse, shift, sqrt(det gamma), inverse metric.
enum { VG_ALP = 0, VG_BETA = 1, VG_SQG = 4, VG_GU = 5, NVG = 11 };

// Face data written by the face kernel (per face, one set per direction): HLLE (or Lax-Friedrichs) flux of the
// 5 hydro variables, the upwind transverse velocities of Eq. uct1 (components (d+1)%3 and (d+2)%3), c_max and
// c_min, and with flux constrained transport the induction fluxes along d of B~^((d+1)%3) and B~^((d+2)%3).
enum { FD_F = 0, FD_VB1 = 5, FD_VB2 = 6, FD_CMAX = 7, FD_CMIN = 8, FD_EB1 = 9, FD_EB2 = 10, NFD = 11 };

// Reconstructed variables per cell and direction: rho, p, u^x, u^y, u^z (u = W v), the two transverse B.
enum { NREC = 7 };

struct Blk {
  int n[3];
  int N[3];  // n + 2g
  int g;
  int bc[3];
  long sy, sz;  // strides of j and k
  long V;       // entries per field
  double dx[3];
  double idx[3];
  // blocks of a tiled domain: bit 2 a + s set = the lower (s = 0) or upper (s = 1) ghost layers along axis a are
  // filled from the neighbouring blocks (the boundary-condition sweeps skip them); the block's position in the
  // block grid and the domain index of its first interior cell per axis.  Zero for a lone block.
  int halo;
  int coord[3];
  int off[3];
};

// A domain tiled by a grid of blocks (same spacing; block (bx, by, bz) covers the interior cells
// cuts_d[b_d] .. cuts_d[b_d + 1] - 1 along each axis d; the batch lists the blocks x fastest).  Stored in the
// batch workspace; the cut offsets follow the struct (axis d's nblk[d] + 1 values from index cut_at[d]).
struct Tiling {
  int nblk[3];
  int ntot[3];   // interior cells of the domain per axis
  int bc[3];     // the domain's boundary condition per axis
  int cut_at[3];
  __host__ __device__ const int* cuts(int d) const { return reinterpret_cast<const int*>(this + 1) + cut_at[d]; }
};

struct Ws {
  double* cg;      // NCG fields
  double* fg;      // 3 * NFG fields
  double* vg;      // NVG fields
  double* bf;      // 3 fields: densitised face B~ (x-, y-, z-faces)
  double* bc;      // 3 fields: undensitised centre B
  double* uvel;    // 3 fields: u^i = W v^i at cells
  double* rec;     // 2 * NREC fields: lower-face values, then upper-face values (current direction)
  double* face;    // 3 * NFD fields
  double* ga;      // 1 field: G_A at vertices
  double* fpsi;    // 3 fields: F_Psi^j at vertices
  double* roots;   // null, or 12 fields: the face solves' (lambda_+, lambda_-) of the left and right states per
                   // direction, written by the face solve for the adjoint's reverse sweep
  double* erec;    // 24 fields: per face normal df and transverse direction dr (2 per df), the PPM lower and
                   // upper values along dr of the upwind velocity v~bar^dr and of B~^df (UCT's edge inputs)
  double* uacc;    // 9 fields: RK4 accumulator of asterx_rk4_step
  double* ustage;  // 2 * 9 fields: RK4 stage buffers of asterx_rk4_step
  unsigned long long* counters;  // 8 counters (internal statistics when the caller passes none)
};

constexpr int WS_FIELDS = NCG + 3 * NFG + NVG + 3 + 3 + 3 + 2 * NREC + 3 * NFD + 1 + 3 + 9 + 18 + 24;

struct F9 {
  double* f[9];
};
struct F5 {
  double* f[5];
};
struct CF16 {
  const double* f[16];
};

// Everything one block needs during one stage: geometry, workspace, and the field sets the stage reads and
// writes.  A single-block launch passes one record by value; a batched launch reads records from a device
// table (one table per RK stage, since the stage buffers differ).
struct BlockRec {
  Blk b;
  Ws w;
  F9 Un, Us, Unext, Uacc, dU;
  F5 P;
  signed char* flags;
};

// Item indices of one block's kernels are below its padded volume, which block validation keeps under 4e9 <
// 2^32, so they are split into coordinates with 32-bit unsigned division: the 64-bit form costs several times
// more instructions per item, a large share of the light kernels.  t = i + e0 (j + e1 k).
__host__ __device__ __forceinline__ void unflatten3(long t, unsigned e0, unsigned e1, int& i, int& j, int& k) {
  const unsigned u = (unsigned)t;
  const unsigned r = u / e0;
  i = (int)(u - r * e0);
  const unsigned q = r / e1;
  j = (int)(r - q * e1);
  k = (int)q;
}
// t = i + e0 j
__host__ __device__ __forceinline__ void unflatten2(long t, unsigned e0, int& i, int& j) {
  const unsigned u = (unsigned)t;
  const unsigned r = u / e0;
  i = (int)(u - r * e0);
  j = (int)r;
}

// Cells per work item of the chunked (sliding-stencil) kernels: PPM and WENO-Z reconstruction along an axis and
// the PPM of the edge inputs.  Each chunked item space exists for two pencil lengths; the launch autotuner picks
// one per kernel (the kernels take the length at run time, so both give the same results bit for bit).
constexpr int RCHUNK = 8;
constexpr int RCHUNK_LONG = 16;

// Item spaces of the kernels (per block).  The batched launches concatenate the blocks' item spaces in
// table order; off[kind][blk] is the first item of block blk.
enum Kind {
  KIND_GHOST_X = 0, KIND_GHOST_Y, KIND_GHOST_Z,
  KIND_VERTS_ALL,    // (N+1)^3: face B~
  KIND_CELLS_ALL,    // N^3: centre B, u, prim->cons
  KIND_INTERIOR,     // n^3: recovery, cell update
  KIND_RECON_X, KIND_RECON_Y, KIND_RECON_Z,
  KIND_FACES_X, KIND_FACES_Y, KIND_FACES_Z,  // faces g..g+n along the axis, without the corner columns
  KIND_VERTEX,       // (n+3)^3: G_A, F_Psi
  KIND_EDGES_X, KIND_EDGES_Y, KIND_EDGES_Z,
  KIND_PSI,          // (n+1)^3
  KIND_RCHUNK_X, KIND_RCHUNK_Y, KIND_RCHUNK_Z,  // PPM reconstruction by chunks of RCHUNK cells along the axis
  KIND_EREC,  // 6 kinds KIND_EREC + 2 df + k: face data of faces normal to df along dr = (df + 1 + k) % 3, by chunks
  KIND_RCHUNK16_X = KIND_EREC + 6, KIND_RCHUNK16_Y, KIND_RCHUNK16_Z,  // the same with pencils of RCHUNK_LONG cells
  KIND_EREC16,  // 6 kinds, as KIND_EREC with pencils of RCHUNK_LONG cells
  NKIND = KIND_EREC16 + 6
};

// pencil length of a chunked item space
__host__ __device__ inline int kind_chunk(int kind) {
  return (kind >= KIND_RCHUNK16_X && kind < KIND_EREC16 + 6) ? RCHUNK_LONG : RCHUNK;
}

__host__ __device__ inline long kind_count(int kind, const Blk& b) {
  const long N0 = b.N[0], N1 = b.N[1], N2 = b.N[2];
  const long n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
  const long slots = 2L * b.g + 1;
  switch (kind) {
    case KIND_GHOST_X: return slots * (N1 + 1) * (N2 + 1);
    case KIND_GHOST_Y: return slots * (N2 + 1) * (N0 + 1);
    case KIND_GHOST_Z: return slots * (N0 + 1) * (N1 + 1);
    case KIND_VERTS_ALL: return (N0 + 1) * (N1 + 1) * (N2 + 1);
    case KIND_CELLS_ALL: return N0 * N1 * N2;
    case KIND_INTERIOR: return n0 * n1 * n2;
    case KIND_RECON_X: return (n0 + 2) * N1 * N2;
    case KIND_RECON_Y: return N0 * (n1 + 2) * N2;
    case KIND_RECON_Z: return N0 * N1 * (n2 + 2);
    // faces along D whose transverse indices are not both in the ghost layers (the (2g)^2 corner columns feed
    // nothing): n_T1 n_T2 interior columns, then 2g (n_T1 + n_T2) columns read by the edge fields only
    case KIND_FACES_X: return (n0 + 1) * (n1 * n2 + 2L * b.g * (n1 + n2));
    case KIND_FACES_Y: return (n1 + 1) * (n2 * n0 + 2L * b.g * (n2 + n0));
    case KIND_FACES_Z: return (n2 + 1) * (n0 * n1 + 2L * b.g * (n0 + n1));
    case KIND_VERTEX: return (n0 + 3) * (n1 + 3) * (n2 + 3);
    case KIND_EDGES_X: return n0 * (n1 + 1) * (n2 + 1);
    case KIND_EDGES_Y: return (n0 + 1) * n1 * (n2 + 1);
    case KIND_EDGES_Z: return (n0 + 1) * (n1 + 1) * n2;
    case KIND_PSI: return (n0 + 1) * (n1 + 1) * (n2 + 1);
    case KIND_RCHUNK_X:
    case KIND_RCHUNK16_X: {
      const long ch = kind_chunk(kind);
      return ((n0 + 2 + ch - 1) / ch) * N1 * N2;
    }
    case KIND_RCHUNK_Y:
    case KIND_RCHUNK16_Y: {
      const long ch = kind_chunk(kind);
      return N0 * ((n1 + 2 + ch - 1) / ch) * N2;
    }
    case KIND_RCHUNK_Z:
    case KIND_RCHUNK16_Z: {
      const long ch = kind_chunk(kind);
      return N0 * N1 * ((n2 + 2 + ch - 1) / ch);
    }
    default: {
      int e = -1;
      if (kind >= KIND_EREC && kind < KIND_EREC + 6) e = kind - KIND_EREC;
      if (kind >= KIND_EREC16 && kind < KIND_EREC16 + 6) e = kind - KIND_EREC16;
      if (e >= 0) {
        const int df = e / 2, dr = (df + 1 + e % 2) % 3, de = 3 - df - dr;
        const long n[3] = {n0, n1, n2};
        const long ch = kind_chunk(kind);
        // faces g-1..g+n along dr (chunks), g..g+n along df, g..g+n-1 along de
        return ((n[dr] + 2 + ch - 1) / ch) * (n[df] + 1) * n[de];
      }
    }
  }
  return 0;
}

}  // namespace asterx
