// exx_dev.h -- device-visible structures of the EXX pair path (library-internal).
#pragma once
#include <cstdint>

namespace exx {

constexpr int kGuessBins = 64;   // radial bins of the multipole starting guess
constexpr int kNlm = 49;   // (lmax + 1)^2 for lmax = 6; tables are padded to this

// Multigrid preconditioner of the mixed-precision Step IV solve (V(1,1) cycle,
// weighted Jacobi, trilinear transfers; not in the paper, whose CG is plain).
// Level 0 is the set's dense CG box and its operator the kernel's stencil;
// coarse levels 1 .. nlev-2 are dense boxes with a margin of kMgPadDev points,
// each row applied over a pattern of K offsets with the level's interior
// weights (wrow = -1) or its own weights (a row of wexp); the coarsest level
// nlev-1 is solved with the inverse of its operator.
constexpr int kMgLevelsDev = 6;
constexpr int kMgKDev = 125;
constexpr int kMgPadDev = 2;
constexpr int kMgCoarsestDev = 256;
struct MgLevelDev {
    int n, K;                      // active points, pattern size
    int n_int, n_exp;              // interior rows (the first n_int points), rows with their own weights
    int Bp[3];                     // padded box
    long long box;                 // padded box elements
    long long off;                 // float offset of the level's R, Z, T boxes in the slot's region
    long long stride;              // floats between R, Z and T
    const int32_t *pts;            // [n] padded box offset of each active point
    const float *wexp;             // [K][n_exp] weights of the non-interior rows, pattern-major
    const float *dinv;             // [n] omega / diag(A_l)
    const float *dbox;             // [box] the same on the padded box, zero at inactive points
    int n_groups, n_pure;          // runs of 4 points along the last axis (Bp[2] % 4 == 0); the first
    const int32_t *groups;         // n_pure hold interior rows only: (offset / 4) << 4 | mask
    const float4 *wmix;            // [125][n_groups - n_pure] weights of the other runs by window position
};
struct MgDev {
    int nlev;                      // levels including the fine one; 0: no hierarchy
    float omega;                   // Jacobi weight (level 0 takes omega / diag of the stencil)
    long long floats;              // floats of the slot region the coarse boxes need
    MgLevelDev lv[kMgLevelsDev];   // lv[1 .. nlev-1]
    int kd[kMgLevelsDev][kMgKDev]; // pattern offsets, (dx+2) | (dy+2) << 3 | (dz+2) << 6
    float wint[kMgLevelsDev][kMgKDev];
    float wdense[kMgLevelsDev][125];   // interior weights on the 5 x 5 x 5 window ((dx+2) * 5 + dy+2) * 5 + dz+2
    int kmap[kMgLevelsDev][125];       // window position -> pattern entry, -1 outside the pattern
    int nrow[kMgLevelsDev];            // (dx, dy) rows of the window with pattern entries
    int rows[kMgLevelsDev][25];        // as (dx + 2) * 5 + dy + 2, ascending
    const float *cinv;             // [n][n] inverse of the coarsest operator, row-major
    const int32_t *pinfo;          // [fine groups] level-1 parents row << 2 | (u0 & 1) << 1 | (u1 & 1)
    const int32_t *pinfo1;         // [level-1 runs] the same onto level 2 (null below three levels)
};

// Geometry of one subdomain kind (self pairs or non-self pairs) of one cell.
struct SetDev {
    int n_pe, n_shell, n_halo;
    int B[3], c[3];
    long long box;                 // elements of the dense CG box
    int dstride[6];                // box stride of each stencil direction
    int gstride[3];                // box stride of each lattice axis
    const int32_t *pe_m;           // [n_pe] packed offsets (lexicographic)
    const int32_t *pe_off;         // [n_pe] dense-box offsets
    const int32_t *sh_m;           // [n_shell] packed offsets, halo points first
    const int32_t *halo_off;       // [n_halo] dense-box offsets
    const int32_t *groups;         // [n_groups] aligned 4-point groups: (offset/4) << 4 | PE mask
    int n_groups;
    const int32_t *bnd;            // [n_bnd] PE points with a halo point within the stencil's reach
    int n_bnd;
    int rstride[6];                // dstride without the last-axis component
    int d2[6];                     // last-axis component of each direction
    // radial bins of the PE points (multipole starting guess): points sorted by bin
    const int32_t *gs_perm;        // [n_pe] PE index of the sorted points
    const int32_t *gs_bstart;      // [kGuessBins + 1] first sorted point of each bin
    const uint8_t *gs_bin;         // [n_pe] bin of each PE point
    const float *gs_S32;           // [n_pe][kNlm] S32 rows in sorted order
    const int4 *gs_info;           // [n_pe] in sorted order: packed offset, box offset, bin, PE index
    // row partition over a cluster of CTAs (cluster path; cl_cta == NULL: not available)
    const int32_t *cl_cta;         // [nc][8]: G0, G1, K0, K1, rows, p_floats
    const int32_t *cl_rows;        // [B0 * B1][2]: owner rank (-2 halo-only row, -1 unused), offset of column 0
    const int32_t *cl_grc;         // [n_groups]: row id | column << 13
    const int32_t *cl_pe_gl;       // [n_pe]: group << 2 | lane
    int cl_pad, cl_row_stride;
    const double *S64;             // [n_pe][kNlm] regular solid harmonics r^l Y_lm(r-bar)
    const float *S32;
    const double *T64;             // [kNlm][n_shell] 4 pi / (2l+1) r^l Y_lm / r^(2l+1)
    const float *T32;
    const MgDev *mg;               // multigrid hierarchy (device memory), or NULL
};

// One unique pair (i <= j): lattice image k of j and grid-resolved centre g.
struct PairRec {
    int i, j;
    int k[3];
    int g[3];
    int cell;
    int pad;
};

// Everything a pair of one cell needs; one per cell, in device memory.
struct CellDev {
    double h[3][3], hinv[3][3], J[3][3];
    double vol, dv, dxi[3];
    int n[3];
    int ndir, fd_n, lmax, nlm;
    int dir[6][3];
    double cw64[6][8];             // coef_d * w2_s, s = 0..n
    float cw32[6][8];
    double w1dx[3][8];             // w1_s / dxi_alpha
    double tol;
    int max_iter, precision;
    double r_pair2;
    SetDev set[2];                 // [0] self pairs, [1] non-self pairs
    // orbitals (device copies)
    const double *phi;
    const int32_t *box_lo;
    int box[3];
    int n_orb;
    const double *centres;
    // D output
    double *dxx;
    const int32_t *dbox_lo;
    int dbox[3];
    // rows of the pair list of this cell: global row index base
    int row_base;
    int cell_index;
    int stress_mode;               // 2: simple-cubic shortcut, the sigma integrals are skipped
    int guess;                     // 1: CG starts from the free-space multipole potential
    int precond;                   // 1: multigrid-preconditioned mixed CG where the set has a hierarchy
    int inner_shift;               // reliable update after the FP32 residual fell by 2^-inner_shift (0: launch default)
    float mg_omega;                // Jacobi weight of the V-cycle (0: the tables' own)
    // warm start: initial guesses from the previous solve of the same plan
    const int32_t *warm_map;       // [n_orb][n_orb] index of pair (i, j) in warm_rows, -1 none; NULL: cold
    const PairRec *warm_rows;
    const float *warm_prev;        // [..][warm_stride] previous solutions on PE (PE order of the set)
    float *warm_next;              // [warm_cap][warm_stride] solutions of this solve, or NULL
    const int32_t *warm_inv[2];    // [box] dense-box offset -> PE index of each set, -1 outside PE
    long long warm_stride;
    int warm_cap;
};


// Per-pair outputs (indexed by the global pair index).
struct PairOut {
    double e;          // int_PE rho v
    double sig[9];     // [a][alpha] sum_b hinv_{alpha b} int r_b rho d_a v
    int iters;
    int refine;
    int status;
    int pad;
};

// Per-cell reduced results.
struct CellResult {
    double e_xx;
    double dedh[9];
    double stress[9];
    long long total_iter;
    long long total_refine;
    int n_pairs;
    int status;
    int failed_pair;
    int max_iter;
    int max_refine;
    int pad;           // n_warm: pairs that started from a previous solution
};

// Pair-list bookkeeping in device memory.
struct ListDev {
    int *row_count;      // [total rows]  pairs of row (cell, i)
    int *row_start;      // [total rows]
    int *cell_start;     // [n_cells]
    int *cell_count;     // [n_cells]
    int *total;          // [1]
    int *queue;          // [1] work-queue counter
    int *overflow;       // [1]
    PairRec *pairs;      // [capacity]
    PairOut *out;        // [capacity]
    int capacity;
    const int *perm;     // [*total] pair indices this launch solves (a rank's share), or NULL: 0 .. *total-1
};

}  // namespace exx
