// batch.cuh -- the solve of many systems at once (uaamg_solve_batch): descriptors and kernel
// arguments shared by the host driver (solve_batch.cu) and its kernels (kern_batch.cu).
//
// Every system keeps its own hierarchy (its handle from uaamg_setup) and its own workspace
// of R columns, interleaved [n][R] as for uaamg_solve_many.  A launch covers every
// participating system at one node of the K-cycle (Section 4.3): its blocks are tiles of
// the systems' rows, listed per launch as segments (one per system, in system order), and
// each block reads its system and tile from the launch's per-block table.  Inner
// products are reduced per system and per column in a fixed order (a tree inside a tile,
// then the system's tiles in order by the last of its tiles to finish), and a system's
// tiles depend only on its own level size and column count, so a system's result is the
// same bits whichever other systems share the launch.
#pragma once
#include "common.cuh"

namespace uaamg {

constexpr int kBMaxTiles = 256;  // tiles of one system at one level, at most
constexpr int kBMaxR = 32;       // columns of one system, at most
constexpr int kBPartStride = kBMaxR;  // partial sums of one (tile, inner product)

// Vector slots of a level, in the precision of the cycle (interleaved [n][R]); the last five
// exist on level 0 only and are FP64 (the outer flexible CG).
enum BSlot {
    BS_RHS = 0, BS_OUT, BS_W, BS_S, BS_C1, BS_V1, BS_RT, BS_C2, BS_V2,
    BS_B, BS_X, BS_R, BS_P, BS_Q,
    kBSlots
};

// One level of one system.
struct BLevel {
    int n;      // rows of the level
    int R;      // columns (right-hand sides) of the system
    int nc;     // rows of the next level (aggregates); 0 on the coarsest
    int inner;  // flexible-CG steps this level takes as a coarse level (1 or 2)
    double tau; // > 0: Notay's threshold on the second step
    const int* rowptr;
    const int* col;
    const void* val;     // cycle precision
    const double* val64; // FP64 values (the outer iteration reads level 0's)
    const void* minv;    // cycle precision
    const int* agg;      // fine -> coarse
    const int* aggptr;   // members of each aggregate, ascending
    const int* members;
    const double* inv;   // dense inverse when this is the system's coarsest level
    void* v[kBSlots];
    double* sc;  // K-cycle scalars of the level: 7 rows of R (as uaamg_solve_many)
    double* os;  // level 0: outer scalars, 8 rows of R (as uaamg_solve_many)
};

// Arguments of every batched kernel.
struct BArgs {
    const BLevel* lev;  // [nsys][kMaxLevels]
    // per block of the launch: its system, its tile within the system, the system's tile
    // count and the launch's first tile of that system (where its partial sums start)
    const int4* tinfo;
    int nseg;
    const int* active;  // [nsys] 0 once every column of the system has converged
    int level;
    // vector slots the kernel reads and writes (-1 = none); e is read on level + 1
    int s_r, s_x, s_y, s_y2, s_d1, s_d2, s_e;
    int res_os;   // inner products go to level 0's outer scalars (else the level's sc)
    int res_row;  // first row of the result
    int outer;    // the FP64 outer SpMV / residual: read val64
    double* partials;        // [tiles][ND][kBPartStride]
    unsigned int* counters;  // [nsys], zero between launches
};

// Rows of one tile: 256 / Rp rows per block step (Rp = R rounded up to a power of two),
// and as many steps as keep the system at most kBMaxTiles tiles.
__host__ __device__ inline int b_lg(int R) {
    int lg = 0;
    while ((1 << lg) < R) lg++;
    return lg;
}
__host__ __device__ inline int b_tile_rows(int n, int R) {
    const int rpb = kThreads >> b_lg(R);
    const int nt = (n + rpb - 1) / rpb;
    const int steps = (nt + kBMaxTiles - 1) / kBMaxTiles;
    return rpb * (steps > 1 ? steps : 1);
}
__host__ __device__ inline int b_tiles(int n, int R) {
    const int t = b_tile_rows(n, R);
    return n > 0 ? (n + t - 1) / t : 0;
}

// Launchers (kern_batch.cu).  `tiles` is the launch's block count (one block per tile);
// every launcher returns a status.
enum BKind {
    BK_ROW = 0,   // SpMV-based row kernel (mode, ndots as the single-system RB_* modes)
    BK_RESTRICT,  // r_c = P^T s
    BK_DENSE,     // exact coarsest solve
    BK_KC_RT,     // rho~ = rho - (alpha1/rho1) v1 (+ norms when tau > 0)
    BK_COMBINE,   // e = w1 c1 + w2 c2
    BK_CAST,      // FP64 outer residual -> cycle precision right-hand side
    BK_ZQ,        // (z, q)
    BK_P,         // p = z - beta p
    BK_XR,        // x += alpha p, r -= alpha q, (r, r)
    BK_NORM,      // (b, b)
    BK_INIT,      // x = p = q = 0
};
template <typename T>
int launch_batch(cudaStream_t st, int kind, int mode, int ndots, const BArgs& a, int tiles,
                 bool pdl);

}  // namespace uaamg
