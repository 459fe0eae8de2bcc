// plan.h -- host-side geometry of the EXX pair path (cell metric, Natan-Kronik
// stencil, proto-subdomain offset sets and the dense CG box layout).
//
// Everything here is computed once per cell (or per MD step for a fluctuating
// cell) on the host and uploaded as small constant tables; the per-pair work
// runs in the CUDA kernels.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/exx.h"

namespace exx {

constexpr int kMaxFd = 6;     // largest stencil half-width n
constexpr int kMaxL = 6;      // largest multipole order
constexpr int kNlmMax = (kMaxL + 1) * (kMaxL + 1);

// Cell tensor and the quantities of Sec. II B 1 and Eqs. jacb, lapG_.
struct Metric {
    double h[3][3];       // h[a][alpha] = (L_alpha)_a
    double hinv[3][3];    // adjugate / det, fixed operation order (pair-list bit-exactness)
    double J[3][3];       // J[a][alpha] = |L_alpha| hinv[alpha][a]
    double F[3][3];       // F = J^T J
    double vol, dv;
    double len[3], dxi[3];
    int n[3];
};
int make_metric(const double lattice[3][3], const int n[3], Metric &m);

// Green-Lagrange strain of a cell relative to a reference cell (both as
// lattice rows): F = h h0^-1, E = (F^T F - I) / 2.  eps_max = the largest
// |eigenvalue| of E, dvol = det F - 1.  Frozen proto-subdomains deform with the
// cell (Sec. III B 2); this is the criterion for re-assembling them.
int cell_strain(const double lattice0[3][3], const double lattice[3][3], double &eps_max, double &dvol);

// Pure-derivative directions of the NK Laplacian (Eq. lapG_mod_nk3d): the three
// lattice axes and n_aux auxiliary grid directions.
struct Stencil {
    int n_off = 0, n_aux = 0, ndir = 3;
    int dir[6][3] = {};
    double coef[6] = {};      // multiplies sum_q w_q f(g + q dir); includes 1/step^2
    double b[3] = {};
    double a[3][3] = {};
};
// aux == nullptr: choose the directions (2D bisector rule or Algorithm 1).
int make_stencil(const Metric &m, int fd_n, int nq, const int (*aux)[3], int n_aux_fixed, Stencil &st);

// Central-difference weights w2[0..n] (second derivative, Eq. d2_1) and
// w1[0..n] (first derivative, Eq. d1_1), from the moment conditions.
void fd_weights(int n, double *w2, double *w1);

// Integer offsets m of the proto-subdomains (Eqs. rbar, g0): PE points
// |h m/N| <= R_PE first, then the shell R_PE < |h m/N| <= R_ME, lexicographic.
struct OffsetSet {
    std::vector<int> m;   // [n_me][3]
    int n_pe = 0, n_me = 0;
};
int make_offsets(const Metric &mt, double r_pe, double r_me, OffsetSet &o);

// Dense CG box and the per-point index tables uploaded to the device.
//   box: PE bounding box plus the stencil reach on every side; element of
//   offset m sits at ((m0 + c0) B1 + (m1 + c1)) B2 + (m2 + c2).
//   shell points are reordered: halo (reached by a stencil from PE) first.
//   B2 is padded to a multiple of 4 so that rows start on 16-byte boundaries;
//   groups are the 4-aligned runs of 4 box elements along the last axis that
//   hold at least one PE point, packed as (offset / 4) << 4 | PE mask.
struct SetLayout {
    int n_pe = 0, n_shell = 0, n_halo = 0;
    int B[3] = {}, c[3] = {};
    long long box = 0;
    int dstride[6] = {};
    int gstride[3] = {};
    std::vector<int32_t> pe_m, pe_off;     // packed offsets and box offsets of PE points
    std::vector<int32_t> sh_m, halo_off;   // packed offsets of shell points; box offsets of halo points
    std::vector<int32_t> groups;           // aligned 4-point groups covering PE
    std::vector<int32_t> bnd;              // PE points with a halo point within the stencil's reach, ascending
    int rstride[6] = {};                   // box stride of a direction without its last-axis part
};
int make_layout(const OffsetSet &o, const Stencil &st, int fd_n, SetLayout &L);

// Multigrid hierarchy of one proto-subdomain, for preconditioning the Step IV
// CG (not in the paper, which uses plain CG: the preconditioner changes the
// iterates, not the discrete equations or the stopping rule).  Level 0: the PE
// points of the dense CG box with A = -L, the NK stencil with the halo moved to
// the right-hand side (Dirichlet zero).  Level l + 1: the active level-l points
// at even box coordinates u, as the points c = u/2 of a box half as fine (each
// coarse point has its own weight-1 child, so the columns of P are independent
// and every Galerkin operator stays positive definite); a level-l point at u
// interpolates from those of floor(u/2) and ceil(u/2) along each axis that are
// coarse points (trilinear prolongation, weight 1 on an even coordinate and 1/2
// on each side of an odd one), restriction is its transpose, and the Galerkin
// operator A_{l+1} = P^T A_l P.  Operators are CSR with columns sorted.
struct MgLevel {
    int B[3] = {};                 // box of the level (level 0: the dense CG box)
    int n = 0;                     // active points
    std::vector<int32_t> idx;      // box point -> active index, -1 when inactive
    std::vector<int32_t> pts;      // active index -> box point
    std::vector<int32_t> row, col; // CSR of A_l
    std::vector<double> val;
};
// Levels until one has at most min_points points (that one included).
int make_mg_levels(const SetLayout &L, const Stencil &st, int fd_n, int min_points, std::vector<MgLevel> &lv);

// The hierarchy in the form the pair solver applies it (V(1,1) cycle, weighted
// Jacobi smoothing, trilinear transfers).  Level 0 is the dense CG box itself,
// whose operator is the kernel's own stencil.  Coarse levels 1 .. nlev-2 are
// dense boxes with a margin of kMgPad points on every side (coordinate u of
// level l sits at u + kMgPad), each row of A_l applied over one pattern of K
// offsets: rows equal to the level's interior stencil (the row of the most
// central point) take the shared weights wint, the others (rows that the
// Dirichlet boundary of the subdomain truncates) their own K weights in wexp,
// zero where the row has no entry.  The active points are ordered interior
// rows first (n_int of them), then the others, each part by box offset, and
// wexp is stored pattern-major ([K][n - n_int]), so that the lanes of a warp
// take the same branch and read consecutive weights.  dinv = omega / diag(A_l),
// per point and as a padded box (dbox, zero at inactive points).  The coarsest
// level nlev-1 is solved exactly with the inverse of its operator (cinv,
// row-major over its active points).  Every operator is FP32.
constexpr int kMgPad = 2;          // margin of the coarse boxes (the coarse stencil reach)
constexpr int kMgMaxLevels = 6;    // fine level included
constexpr int kMgMaxK = 125;       // 5 x 5 x 5 pattern positions
constexpr int kMgMaxCoarsest = 256;
struct MgTables {
    int nlev = 0;                                   // 0: no hierarchy (too small, or a reach above kMgPad)
    int n[kMgMaxLevels] = {};                       // active points per level
    int Bp[kMgMaxLevels][3] = {};                   // padded boxes of the coarse levels
    long long box[kMgMaxLevels] = {};               // their sizes
    int K[kMgMaxLevels] = {};
    int kd[kMgMaxLevels][kMgMaxK] = {};             // pattern offsets (dx+2) | (dy+2) << 3 | (dz+2) << 6
    float wint[kMgMaxLevels][kMgMaxK] = {};
    int n_exp[kMgMaxLevels] = {};
    int n_int[kMgMaxLevels] = {};                   // interior rows (the first n_int active points)
    std::vector<int32_t> pts[kMgMaxLevels];         // padded box offset of each active point
    std::vector<float> wexp[kMgMaxLevels];          // [K][n_exp], n_exp = n - n_int
    std::vector<float> dinv[kMgMaxLevels];
    std::vector<float> dbox[kMgMaxLevels];          // dinv on the padded box
    // for the residual pass: the active points as aligned runs of 4 along the last
    // axis (the last axis of the padded box is a multiple of 4 long), each run as
    // (offset / 4) << 4 | mask with the row of wexp of each of its 4 points (-1:
    // interior or inactive); runs without explicit rows first
    std::vector<int32_t> groups[kMgMaxLevels], gexp[kMgMaxLevels];   // gexp: [n_groups][4]
    int n_pure[kMgMaxLevels] = {};                  // leading runs whose points are all interior
    // weights of the other runs by window position, four points at a time:
    // [125][n_groups - n_pure][4], the interior weight for interior points, the
    // point's own row for the others, zero for inactive points and outside the pattern
    std::vector<float> wmix[kMgMaxLevels];
    float wdense[kMgMaxLevels][125] = {};           // interior stencil on the 5 x 5 x 5 window (dx, dy, dz)
    int kmap[kMgMaxLevels][125] = {};               // window position -> pattern entry k, -1 outside the pattern
    int nrow[kMgMaxLevels] = {};                    // (dx, dy) rows of the window holding pattern entries
    int rows[kMgMaxLevels][25] = {};                // as (dx + 2) * 5 + dy + 2, ascending
    std::vector<float> cinv;                        // [n][n] of the coarsest level
    // per aligned fine group (SetLayout::groups): the level-1 box offset of the
    // last-axis parents of its first point in the row (u0/2, u1/2), shifted left
    // by 2, with u0 & 1 in bit 1 and u1 & 1 in bit 0 (odd rows also read the
    // next level-1 row along that axis)
    std::vector<int32_t> pinfo;
    // the same for the level-1 runs (groups[1], unpadded coordinates) onto level 2
    // (a run starts at an even last-axis coordinate too); empty below three levels
    std::vector<int32_t> pinfo1;
    long long slot_floats = 0;                      // three boxes per coarse level
};
// drop: pattern entries below drop x the interior diagonal are left out of the
// device operators of the coarse levels (each added, as |a|, to its row's diagonal)
int make_mg_tables(const SetLayout &L, const Stencil &st, int fd_n, int min_points, double omega, double drop,
                   MgTables &t);

// Candidate schedules of the autotuner (exx_plan_autotune), in the order that
// breaks ties: with a multigrid hierarchy, MG with omega 0.8, 0.7, 0.6, each
// with inner_shift 14 then 18; then plain CG with inner_shift 14, 18.
std::vector<exx_schedule> schedule_candidates(bool mg, double omega_default);
// Longest-processing-time partition of n jobs over n_ranks: jobs in order of
// decreasing cost (equal costs keep their order), each given to the rank with
// the least load so far (the lowest rank on ties).  owner[k] receives job k's rank.
void lpt_partition(const double *cost, int n, int n_ranks, int *owner);

// The autotuner's choice among n measured candidates: the index of the
// smallest finite time, the first on ties; -1 when none is finite.
int pick_schedule(const double *ms, int n);

// Row partition of one set over a cluster of nc CTAs (the cluster CG path).
// The box rows (plane z, row y) that hold PE or halo points are taken in
// (z, y) order and split into nc contiguous ranges with about equal numbers of
// PE groups.  CTA c keeps p for its rows that hold PE points in shared memory,
// each row as pad + B2 + pad2 floats (column x at pad + x), so that every
// stencil read of a PE group -- including the lanes outside PE -- stays inside
// one stored row; row 0 of every CTA's region is all zero and stands for the
// rows that hold only halo points.
struct ClusterPart {
    int nc = 0;
    int pad = 0, row_stride = 0;          // floats before column 0, floats per stored row
    std::vector<int32_t> cta;             // [nc][8]: G0, G1, K0, K1, rows, p_floats, 0, 0
    std::vector<int32_t> rows;            // [B0 * B1][2]: owner rank, float offset of column 0; owner -2:
                                          // a row of halo points only (all zero: read the reader's zero
                                          // row at offset pad); -1: never read
    std::vector<int32_t> grc;             // [n_groups]: row id (z * B1 + y) | column << 13
    std::vector<int32_t> pe_gl;           // [n_pe]: group index << 2 | lane of each PE point
    int max_p_floats = 0, max_groups = 0;
};
int make_cluster_part(const SetLayout &L, const Stencil &st, int fd_n, int nc, ClusterPart &cp);

// Packing of an offset triple with |m_alpha| <= 511 into one int32.
inline int32_t pack_m(int m0, int m1, int m2) {
    return (int32_t)(((uint32_t)(m0 + 512) << 20) | ((uint32_t)(m1 + 512) << 10) | (uint32_t)(m2 + 512));
}

}  // namespace exx
