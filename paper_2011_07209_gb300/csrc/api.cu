// api.cu -- the C ABI of include/exx.h: contexts, plans, workspace and the
// launch sequence of one EXX evaluation (pair list -> persistent pair solver
// -> ordered per-cell reductions), for one cell or a batch of cells.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/exx.h"
#include "exx_dev.h"
#include "kernels.h"
#include "plan.h"

using namespace exx;

namespace {
thread_local char g_err_detail[256] = "";
int cuda_fail(cudaError_t e, int line)
{
    std::snprintf(g_err_detail, sizeof(g_err_detail), "api.cu:%d: %s (%s)", line, cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return EXX_ERR_CUDA;
}
}  // namespace

int exx::note_cuda_error(const char *where, cudaError_t e)
{
    std::snprintf(g_err_detail, sizeof(g_err_detail), "%s: %s (%s)", where, cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return EXX_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, __LINE__); \
    } while (0)

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class T>
int dev_alloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return EXX_OK;
    if (cudaMalloc((void **)p, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return EXX_ERR_OOM;
    }
    return EXX_OK;
}

template <class T>
void dev_free(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

}  // namespace

struct exx_ctx {
    int device = 0;
    int n_sm = 0;
    // persistent solver slots (shared by every plan of the context)
    char *slots = nullptr;
    size_t slots_bytes = 0;
    SolveSlots sl_mixed{}, sl_fp64{};
    size_t box_max = 0, npe_max = 0, mg_max = 0;
    bool slots_dirty = false;
    // pair list
    ListDev list{};
    int rows_cap = 0;
    // cells and results
    CellDev *d_cells = nullptr;
    CellResult *d_res = nullptr;
    CellDev *h_cells = nullptr;       // pinned
    CellResult *h_res = nullptr;      // pinned
    int cells_cap = 0;
    int inner_shift = 14;             // reliable update when the FP32 residual fell by 2^-14 (EXX_INNER_SHIFT)
    int solver = EXX_SOLVER_CTA;   // exx_ctx_set_solver
    int cluster_cap = -1;     // dynamic shared memory a cluster CTA can take (bytes), -1 unknown
    int last_path = 0;        // 0: per-CTA solver, 1: cluster solver (of the last solve)
    int last_clusters = 0;
    bool timing = false;
    cudaEvent_t ev[5] = {};
    double ms[4] = {};
    // orbital rows and pairs of the live plans: the pair list is sized for all
    // of them at plan creation, so that a solve (or a batch of the plans) finds
    // its workspace in place
    long long plan_rows = 0, plan_pairs = 0;
    int sample_limit = 0;     // > 0: solve only the first pairs of the list (exx_plan_autotune)
    int *d_perm = nullptr;    // [list capacity] pair indices of this rank's share (sharded solves)
};

struct exx_plan {
    exx_ctx *ctx = nullptr;
    int device = 0;
    exx_cell cell0{};      // cell the offsets / aux directions were built for
    exx_cell cell{};       // cell of the last metric update
    exx_params params{};
    Metric metric{};
    Stencil stencil{};
    int aux[3][3] = {};
    int n_aux = 0;
    OffsetSet off[2];
    SetLayout lay[2];
    int32_t *d_pe_m[2] = {}, *d_pe_off[2] = {}, *d_sh_m[2] = {}, *d_halo_off[2] = {}, *d_groups[2] = {};
    int32_t *d_bnd[2] = {};
    int n_bnd[2] = {};
    double *d_S64[2] = {}, *d_T64[2] = {};
    float *d_S32[2] = {}, *d_T32[2] = {};
    bool tables_valid = false;
    // device copies for host-memory inputs
    int max_orb = 0;
    int box[3] = {};
    double *d_phi = nullptr, *d_centres = nullptr;
    int32_t *d_box_lo = nullptr;
    double *d_dxx = nullptr;
    size_t dxx_cap = 0;
    int32_t *d_dbox_lo = nullptr;
    double *d_pair_e = nullptr;   // per-pair staging for host-memory outputs
    PairRec *d_pairs = nullptr;   // pair list of the last solve
    int pairs_cap = 0;
    int last_count = 0;
    PairOut *d_out = nullptr;
    // warm start (params.warm_start): solutions of the last solve, one FP32 vector per pair
    int32_t *d_inv[2] = {};           // dense-box offset -> PE index of each set
    int32_t *d_gs_perm[2] = {}, *d_gs_bstart[2] = {};   // radial bins of the starting guess
    uint8_t *d_gs_bin[2] = {};
    float *d_gs_S32[2] = {};
    int4 *d_gs_info[2] = {};   // radius-sorted packed offset, box offset, bin, PE index
    // row partitions for the cluster path (mixed precision)
    ClusterPart cpart[2];
    bool cl_ok[2] = {false, false};
    int32_t *d_cl_cta[2] = {}, *d_cl_rows[2] = {}, *d_cl_grc[2] = {}, *d_cl_pegl[2] = {};
    // multigrid preconditioner of the mixed CG (params.precond), per set
    MgDev h_mg[2] = {};               // host copy (pointers are device pointers)
    MgDev *d_mg[2] = {};
    std::vector<void *> mg_bufs[2];
    bool mg_shared = false;           // self and non-self sets are the same offsets: set 1 uses set 0's tables
    int32_t *d_warm_map = nullptr;    // [max_orb][max_orb] pair index of (i, j) in d_pairs, -1 none
    float *d_warm_v[2] = {};          // solution stores; d_warm_v[warm_cur] holds the last solve's
    int warm_cap = 0;                 // pairs each store holds
    long long warm_stride = 0;        // floats per pair (largest N_PE of the two sets)
    int warm_cur = 0;
    int warm_n = 0;                   // valid pairs in d_warm_v[warm_cur]; 0: next solve starts cold
    int warm_norb = -1;
    bool counted = false;             // rows and pairs added to the context's totals
    exx_schedule sched{};             // solver schedule (exx_plan_set_schedule / exx_plan_autotune)
    int shard_rank = 0, shard_n = 1;  // exx_plan_set_shard
};

static bool same_cell(const exx_cell &a, const exx_cell &b)
{
    return std::memcmp(a.lattice, b.lattice, sizeof(a.lattice)) == 0 && a.n[0] == b.n[0] && a.n[1] == b.n[1] &&
           a.n[2] == b.n[2];
}

static int check_params(const exx_params *p)
{
    if (!p) return EXX_ERR_ARG;
    if (p->fd_order < 1 || p->fd_order > kMaxFd) return EXX_ERR_ARG;
    if (p->lmax < 0 || p->lmax > kMaxL) return EXX_ERR_ARG;
    if (!(p->r_pair >= 0.0) || !(p->cg_tol > 0.0) || p->cg_max_iter < 1 || p->nq < 1) return EXX_ERR_ARG;
    if (p->precision != EXX_FP64 && p->precision != EXX_MIXED) return EXX_ERR_ARG;
    if (p->stress_mode < EXX_STRESS_FULL || p->stress_mode > EXX_STRESS_CUBIC) return EXX_ERR_ARG;
    if (p->warm_start != 0 && p->warm_start != 1) return EXX_ERR_ARG;
    if (p->frozen < 0 || p->frozen > 2) return EXX_ERR_ARG;
    if (p->guess != 0 && p->guess != 1) return EXX_ERR_ARG;
    if (p->precond != EXX_PRECOND_NONE && p->precond != EXX_PRECOND_MG) return EXX_ERR_ARG;
    return EXX_OK;
}

// lattice = L I (simple cubic), the precondition of the EXX_STRESS_CUBIC shortcut
static bool simple_cubic(const exx_cell &c)
{
    const double L = c.lattice[0][0];
    if (!(L > 0.0)) return false;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double want = a == b ? L : 0.0;
            if (std::fabs(c.lattice[a][b] - want) > 1e-12 * L) return false;
        }
    return true;
}

constexpr double kMgOmega = 0.8;   // weighted-Jacobi smoothing of the multigrid V-cycle
#ifndef EXX_MG_DROP
#define EXX_MG_DROP 0.005
#endif
constexpr double kMgDrop = EXX_MG_DROP;   // coarse-operator entries below this x the diagonal are lumped into it
#ifndef EXX_MG_MIN_POINTS
#define EXX_MG_MIN_POINTS 200
#endif
constexpr int kMgMinPoints = EXX_MG_MIN_POINTS;   // coarsening stops at this many points (the coarsest is inverted)
constexpr int kMaxBatchCells = 64;  // cells of one exx_pairs_solve_batch call

static void free_mg(exx_plan *p, int s)
{
    for (void *b : p->mg_bufs[s]) cudaFree(b);
    p->mg_bufs[s].clear();
    if (p->mg_shared) {
        // set 1 points at set 0's tables: drop that reference either way
        p->d_mg[1] = nullptr;
        std::memset(&p->h_mg[1], 0, sizeof(MgDev));
        p->mg_shared = false;
    }
    dev_free(p->d_mg[s]);
    std::memset(&p->h_mg[s], 0, sizeof(MgDev));
}

template <class T>
static int mg_put(exx_plan *p, int s, const std::vector<T> &v, const T **out)
{
    *out = nullptr;
    if (v.empty()) return EXX_OK;
    T *d = nullptr;
    int e = dev_alloc(&d, v.size());
    if (e) return e;
    p->mg_bufs[s].push_back(d);
    CK(cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    *out = d;
    return EXX_OK;
}

// The multigrid hierarchy of set s for the plan's current layout and stencil
// (mixed precision with params.precond only; none when the set is too small
// or the stencil reaches too far for the coarse boxes).
static int upload_mg(exx_plan *p, int s, const SetLayout &L)
{
    free_mg(p, s);
    if (p->params.precision != EXX_MIXED || p->params.precond != EXX_PRECOND_MG || p->params.fd_order > 3)
        return EXX_OK;
    if (s == 1 && p->off[1].m == p->off[0].m) {
        // the same offset set (equal self and non-self radii): the same hierarchy
        if (p->d_mg[0]) {
            p->h_mg[1] = p->h_mg[0];
            p->d_mg[1] = p->d_mg[0];
            p->mg_shared = true;
        }
        return EXX_OK;
    }
    MgTables T;
    int e = make_mg_tables(L, p->stencil, p->params.fd_order, kMgMinPoints, kMgOmega, kMgDrop, T);
    if (e) return e;
    if (T.nlev < 2) return EXX_OK;
    MgDev &G = p->h_mg[s];
    std::memset(&G, 0, sizeof(G));
    G.nlev = T.nlev;
    G.omega = (float)kMgOmega;
    long long off = 0;
    for (int l = 1; l < T.nlev; ++l) {
        MgLevelDev &v = G.lv[l];
        v.n = T.n[l];
        v.K = T.K[l];
        v.n_int = T.n_int[l];
        v.n_exp = T.n_exp[l];
        for (int a = 0; a < 3; ++a) v.Bp[a] = T.Bp[l][a];
        v.box = T.box[l];
        v.stride = (T.box[l] + 63) & ~63LL;
        v.off = off;
        off += 3 * v.stride;
        if ((e = mg_put(p, s, T.pts[l], &v.pts)) || (e = mg_put(p, s, T.wexp[l], &v.wexp)) ||
            (e = mg_put(p, s, T.dinv[l], &v.dinv)) || (e = mg_put(p, s, T.dbox[l], &v.dbox)) ||
            (e = mg_put(p, s, T.groups[l], &v.groups)))
            return e;
        {
            const float *wm = nullptr;
            if ((e = mg_put(p, s, T.wmix[l], &wm))) return e;
            v.wmix = reinterpret_cast<const float4 *>(wm);
        }
        v.n_groups = (int)T.groups[l].size();
        v.n_pure = T.n_pure[l];
        for (int k = 0; k < 125; ++k) {
            G.wdense[l][k] = T.wdense[l][k];
            G.kmap[l][k] = T.kmap[l][k];
        }
        G.nrow[l] = T.nrow[l];
        for (int k = 0; k < 25; ++k) G.rows[l][k] = T.rows[l][k];
        for (int k = 0; k < T.K[l]; ++k) {
            G.kd[l][k] = T.kd[l][k];
            G.wint[l][k] = T.wint[l][k];
        }
    }
    G.floats = off;
    if ((e = mg_put(p, s, T.cinv, &G.cinv)) || (e = mg_put(p, s, T.pinfo, &G.pinfo)) ||
        (e = mg_put(p, s, T.pinfo1, &G.pinfo1)))
        return e;
    if ((e = dev_alloc(&p->d_mg[s], 1))) return e;
    CK(cudaMemcpy(p->d_mg[s], &G, sizeof(MgDev), cudaMemcpyHostToDevice));
    return EXX_OK;
}

static void free_geometry(exx_plan *p)
{
    for (int s = 0; s < 2; ++s) {
        dev_free(p->d_pe_m[s]);
        dev_free(p->d_pe_off[s]);
        dev_free(p->d_sh_m[s]);
        dev_free(p->d_halo_off[s]);
        dev_free(p->d_groups[s]);
        dev_free(p->d_bnd[s]);
        dev_free(p->d_inv[s]);
        dev_free(p->d_gs_perm[s]);
        dev_free(p->d_gs_bstart[s]);
        dev_free(p->d_gs_bin[s]);
        dev_free(p->d_gs_S32[s]);
        dev_free(p->d_gs_info[s]);
        dev_free(p->d_cl_cta[s]);
        dev_free(p->d_cl_rows[s]);
        dev_free(p->d_cl_grc[s]);
        dev_free(p->d_cl_pegl[s]);
        p->cl_ok[s] = false;
        free_mg(p, s);
        dev_free(p->d_S64[s]);
        dev_free(p->d_T64[s]);
        dev_free(p->d_S32[s]);
        dev_free(p->d_T32[s]);
    }
    p->tables_valid = false;
    p->warm_n = 0;   // the offsets change: stored solutions no longer apply
}

// Offsets, stencil and layout for cell0 (and the aux directions to freeze).
// Dense CG layouts of both offset sets for the plan's current stencil (box
// margins, strides, groups and halo order depend on the stencil directions),
// uploaded to the device.
static int upload_layouts(exx_plan *p)
{
    for (int s = 0; s < 2; ++s) {
        SetLayout L;
        int e = make_layout(p->off[s], p->stencil, p->params.fd_order, L);
        if (e) return e;
        dev_free(p->d_pe_m[s]);
        dev_free(p->d_pe_off[s]);
        dev_free(p->d_sh_m[s]);
        dev_free(p->d_halo_off[s]);
        dev_free(p->d_groups[s]);
        dev_free(p->d_bnd[s]);
        dev_free(p->d_inv[s]);
        if ((e = dev_alloc(&p->d_pe_m[s], L.n_pe)) || (e = dev_alloc(&p->d_pe_off[s], L.n_pe)) ||
            (e = dev_alloc(&p->d_sh_m[s], L.n_shell)) || (e = dev_alloc(&p->d_halo_off[s], L.n_halo)) ||
            (e = dev_alloc(&p->d_groups[s], L.groups.size())) || (e = dev_alloc(&p->d_bnd[s], L.bnd.size())))
            return e;
        p->n_bnd[s] = (int)L.bnd.size();
        if (!L.bnd.empty()) CK(cudaMemcpy(p->d_bnd[s], L.bnd.data(), 4 * L.bnd.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->d_pe_m[s], L.pe_m.data(), 4 * L.n_pe, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->d_pe_off[s], L.pe_off.data(), 4 * L.n_pe, cudaMemcpyHostToDevice));
        if (L.n_shell) CK(cudaMemcpy(p->d_sh_m[s], L.sh_m.data(), 4 * L.n_shell, cudaMemcpyHostToDevice));
        if (L.n_halo) CK(cudaMemcpy(p->d_halo_off[s], L.halo_off.data(), 4 * L.n_halo, cudaMemcpyHostToDevice));
        if (!L.groups.empty())
            CK(cudaMemcpy(p->d_groups[s], L.groups.data(), 4 * L.groups.size(), cudaMemcpyHostToDevice));
        if (p->params.warm_start) {
            std::vector<int32_t> inv((size_t)L.box, -1);
            for (int q = 0; q < L.n_pe; ++q) inv[(size_t)L.pe_off[q]] = q;
            if ((e = dev_alloc(&p->d_inv[s], inv.size()))) return e;
            CK(cudaMemcpy(p->d_inv[s], inv.data(), 4 * inv.size(), cudaMemcpyHostToDevice));
        }
        dev_free(p->d_cl_cta[s]);
        dev_free(p->d_cl_rows[s]);
        dev_free(p->d_cl_grc[s]);
        dev_free(p->d_cl_pegl[s]);
        p->cl_ok[s] = false;
        if (p->params.precision == EXX_MIXED && p->params.fd_order <= 4 &&
            make_cluster_part(L, p->stencil, p->params.fd_order, kClusterCTAs, p->cpart[s]) == EXX_OK) {
            const ClusterPart &cp = p->cpart[s];
            if ((e = dev_alloc(&p->d_cl_cta[s], cp.cta.size())) || (e = dev_alloc(&p->d_cl_rows[s], cp.rows.size())) ||
                (e = dev_alloc(&p->d_cl_grc[s], cp.grc.size())) || (e = dev_alloc(&p->d_cl_pegl[s], cp.pe_gl.size())))
                return e;
            CK(cudaMemcpy(p->d_cl_cta[s], cp.cta.data(), 4 * cp.cta.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(p->d_cl_rows[s], cp.rows.data(), 4 * cp.rows.size(), cudaMemcpyHostToDevice));
            if (!cp.grc.empty()) CK(cudaMemcpy(p->d_cl_grc[s], cp.grc.data(), 4 * cp.grc.size(), cudaMemcpyHostToDevice));
            if (!cp.pe_gl.empty())
                CK(cudaMemcpy(p->d_cl_pegl[s], cp.pe_gl.data(), 4 * cp.pe_gl.size(), cudaMemcpyHostToDevice));
            p->cl_ok[s] = true;
        }
        if ((e = upload_mg(p, s, L))) return e;
        p->lay[s] = std::move(L);
    }
    p->tables_valid = false;   // the shell order (halo first) may have changed
    return EXX_OK;
}

// Offsets, stencil and layout for cell0 (and the aux directions to freeze).
static int build_geometry(exx_plan *p)
{
    int e = make_metric(p->cell0.lattice, p->cell0.n, p->metric);
    if (e) return e;
    e = make_stencil(p->metric, p->params.fd_order, p->params.nq, nullptr, 0, p->stencil);
    if (e) return e;
    p->n_aux = p->stencil.n_aux;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) p->aux[a][k] = a < p->n_aux ? p->stencil.dir[3 + a][k] : 0;
    const double rpe[2] = {p->params.r_pe_self, p->params.r_pe_pair};
    const double rme[2] = {p->params.r_me_self, p->params.r_me_pair};
    free_geometry(p);
    for (int s = 0; s < 2; ++s) {
        e = make_offsets(p->metric, rpe[s], rme[s], p->off[s]);
        if (e) return e;
        const OffsetSet &o = p->off[s];
        if ((e = dev_alloc(&p->d_S64[s], (size_t)o.n_pe * kNlm)) ||
            (e = dev_alloc(&p->d_S32[s], (size_t)o.n_pe * kNlm)) ||
            (e = dev_alloc(&p->d_T64[s], (size_t)(o.n_me - o.n_pe) * kNlm)) ||
            (e = dev_alloc(&p->d_T32[s], (size_t)(o.n_me - o.n_pe) * kNlm)) ||
            (e = dev_alloc(&p->d_gs_perm[s], (size_t)o.n_pe)) || (e = dev_alloc(&p->d_gs_bstart[s], kGuessBins + 1)) ||
            (e = dev_alloc(&p->d_gs_bin[s], (size_t)o.n_pe)) ||
            (e = dev_alloc(&p->d_gs_S32[s], (size_t)o.n_pe * kNlm)) || (e = dev_alloc(&p->d_gs_info[s], (size_t)o.n_pe)))
            return e;
    }
    if ((e = upload_layouts(p))) return e;
    p->cell = p->cell0;
    p->tables_valid = false;
    return EXX_OK;
}

static bool same_directions(const Stencil &a, const Stencil &b)
{
    if (a.ndir != b.ndir) return false;
    for (int d = 0; d < a.ndir; ++d)
        for (int k = 0; k < 3; ++k)
            if (a.dir[d][k] != b.dir[d][k]) return false;
    return true;
}

// Metric and stencil for the current cell with the offsets held fixed
// (Sec. III B 2).  frozen = 1: the aux directions are chosen for the current
// cell, as Algorithm 1 runs at the beginning of every MD step (Sec. III C);
// frozen = 2: the plan cell's aux directions are kept as well.  When the
// directions change, the dense layouts are rebuilt from the same offsets (the
// halo check runs again there).
static int update_metric(exx_plan *p, const exx_cell &cell)
{
    Metric m;
    int e = make_metric(cell.lattice, cell.n, m);
    if (e) return e;
    Stencil st;
    static const int kNoAux[3][3] = {};
    if (p->params.frozen == 2)
        e = make_stencil(m, p->params.fd_order, p->params.nq, p->n_aux ? p->aux : kNoAux, p->n_aux, st);
    else
        e = make_stencil(m, p->params.fd_order, p->params.nq, nullptr, 0, st);
    if (e) return e;
    const bool relayout = !same_directions(st, p->stencil);
    if (!relayout) {
        // same directions: the layout stands; re-check the halo for safety
        for (int s = 0; s < 2; ++s) {
            SetLayout L;
            e = make_layout(p->off[s], st, p->params.fd_order, L);
            if (e) return e;
        }
    }
    p->metric = m;
    p->stencil = st;
    p->cell = cell;
    p->tables_valid = false;
    if (relayout && (e = upload_layouts(p))) return e;
    return EXX_OK;
}

// Radial bins of the PE points for the multipole starting guess, for the
// current cell: bin = floor(kGuessBins |r-bar| / R_PE), points sorted by bin.
static int upload_guess_bins(exx_plan *p)
{
    const double rpe[2] = {p->params.r_pe_self, p->params.r_pe_pair};
    for (int s = 0; s < 2; ++s) {
        const OffsetSet &o = p->off[s];
        const int n = o.n_pe;
        if (n == 0 || !p->d_gs_perm[s]) continue;
        std::vector<uint8_t> bin(n);
        std::vector<int32_t> count(kGuessBins + 1, 0), perm(n);
        for (int k = 0; k < n; ++k) {
            double r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double x = 0.0;
                for (int al = 0; al < 3; ++al) x += p->metric.h[a][al] * o.m[3 * k + al] / p->metric.n[al];
                r2 += x * x;
            }
            const int b = (int)std::min<double>(kGuessBins - 1, std::sqrt(r2) / rpe[s] * kGuessBins);
            bin[k] = (uint8_t)std::max(0, b);
            count[bin[k] + 1]++;
        }
        for (int b = 0; b < kGuessBins; ++b) count[b + 1] += count[b];
        std::vector<int32_t> fill(count.begin(), count.end() - 1);
        for (int k = 0; k < n; ++k) perm[fill[bin[k]]++] = k;
        CK(cudaMemcpy(p->d_gs_perm[s], perm.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->d_gs_bstart[s], count.data(), 4 * (size_t)(kGuessBins + 1), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->d_gs_bin[s], bin.data(), (size_t)n, cudaMemcpyHostToDevice));

    }
    return EXX_OK;
}

static void fill_celldev(const exx_plan *p, CellDev &C)
{
    std::memset(&C, 0, sizeof(C));
    const Metric &m = p->metric;
    std::memcpy(C.h, m.h, sizeof(C.h));
    std::memcpy(C.hinv, m.hinv, sizeof(C.hinv));
    std::memcpy(C.J, m.J, sizeof(C.J));
    C.vol = m.vol;
    C.dv = m.dv;
    for (int a = 0; a < 3; ++a) {
        C.dxi[a] = m.dxi[a];
        C.n[a] = m.n[a];
    }
    const Stencil &st = p->stencil;
    const int n = p->params.fd_order;
    C.ndir = st.ndir;
    C.fd_n = n;
    C.lmax = p->params.lmax;
    C.nlm = (C.lmax + 1) * (C.lmax + 1);
    double w2[kMaxFd + 1], w1[kMaxFd + 1];
    fd_weights(n, w2, w1);
    for (int d = 0; d < st.ndir; ++d) {
        for (int k = 0; k < 3; ++k) C.dir[d][k] = st.dir[d][k];
        for (int s = 0; s <= n; ++s) {
            C.cw64[d][s] = st.coef[d] * w2[s];
            C.cw32[d][s] = (float)C.cw64[d][s];
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s <= n; ++s) C.w1dx[a][s] = w1[s] / m.dxi[a];
    C.tol = p->params.cg_tol;
    C.max_iter = p->params.cg_max_iter;
    C.precision = p->params.precision;
    C.r_pair2 = p->params.r_pair * p->params.r_pair;
    C.stress_mode = p->params.stress_mode;
    C.guess = p->params.guess;
    C.precond = p->sched.precond;
    C.inner_shift = p->sched.inner_shift;
    C.mg_omega = p->sched.omega;
    for (int s = 0; s < 2; ++s) {
        const SetLayout &L = p->lay[s];
        SetDev &S = C.set[s];
        S.n_pe = L.n_pe;
        S.n_shell = L.n_shell;
        S.n_halo = L.n_halo;
        for (int a = 0; a < 3; ++a) {
            S.B[a] = L.B[a];
            S.c[a] = L.c[a];
            S.gstride[a] = L.gstride[a];
        }
        S.box = L.box;
        for (int d = 0; d < 6; ++d) S.dstride[d] = L.dstride[d];
        S.pe_m = p->d_pe_m[s];
        S.pe_off = p->d_pe_off[s];
        S.sh_m = p->d_sh_m[s];
        S.halo_off = p->d_halo_off[s];
        S.groups = p->d_groups[s];
        S.bnd = p->d_bnd[s];
        S.n_bnd = p->n_bnd[s];
        S.n_groups = (int)L.groups.size();
        for (int d = 0; d < 6; ++d) {
            S.rstride[d] = L.rstride[d];
            S.d2[d] = d < p->stencil.ndir ? p->stencil.dir[d][2] : 0;
        }
        S.gs_perm = p->d_gs_perm[s];
        S.gs_bstart = p->d_gs_bstart[s];
        S.gs_bin = p->d_gs_bin[s];
        S.gs_S32 = p->d_gs_S32[s];
        S.gs_info = p->d_gs_info[s];
        S.cl_cta = p->cl_ok[s] ? p->d_cl_cta[s] : nullptr;
        S.cl_rows = p->d_cl_rows[s];
        S.cl_grc = p->d_cl_grc[s];
        S.cl_pe_gl = p->d_cl_pegl[s];
        S.cl_pad = p->cpart[s].pad;
        S.cl_row_stride = p->cpart[s].row_stride;
        S.S64 = p->d_S64[s];
        S.S32 = p->d_S32[s];
        S.T64 = p->d_T64[s];
        S.T32 = p->d_T32[s];
        S.mg = p->d_mg[s];
    }
}

static int ensure_cells(exx_ctx *c, int n)
{
    if (n <= c->cells_cap) return EXX_OK;
    dev_free(c->d_cells);
    dev_free(c->d_res);
    if (c->h_cells) cudaFreeHost(c->h_cells);
    if (c->h_res) cudaFreeHost(c->h_res);
    c->h_cells = nullptr;
    c->h_res = nullptr;
    c->cells_cap = 0;
    int e;
    if ((e = dev_alloc(&c->d_cells, n)) || (e = dev_alloc(&c->d_res, n))) return e;
    if (cudaMallocHost((void **)&c->h_cells, sizeof(CellDev) * n) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_res, sizeof(CellResult) * n) != cudaSuccess) {
        cudaGetLastError();
        return EXX_ERR_OOM;
    }
    c->cells_cap = n;
    return EXX_OK;
}

static int ensure_list(exx_ctx *c, int rows, long long pairs)
{
    ListDev &L = c->list;
    if (rows <= c->rows_cap && pairs <= L.capacity && L.total) return EXX_OK;
    if (pairs > (1LL << 30)) return EXX_ERR_CAPACITY;
    dev_free(L.row_count);
    dev_free(L.row_start);
    dev_free(L.cell_start);
    dev_free(L.cell_count);
    dev_free(L.total);
    dev_free(c->d_perm);
    dev_free(L.pairs);
    dev_free(L.out);
    const int rcap = std::max(rows, 1);
    const int pcap = (int)std::max(pairs, 1LL);
    int e;
    if ((e = dev_alloc(&L.row_count, rcap)) || (e = dev_alloc(&L.row_start, rcap)) ||
        (e = dev_alloc(&L.cell_start, 64)) || (e = dev_alloc(&L.cell_count, 64)) || (e = dev_alloc(&L.total, 4)) ||
        (e = dev_alloc(&L.pairs, pcap)) || (e = dev_alloc(&L.out, pcap)) || (e = dev_alloc(&c->d_perm, pcap)))
        return e;
    L.queue = L.total + 1;
    L.overflow = L.total + 2;
    L.capacity = pcap;
    c->rows_cap = rcap;
    return EXX_OK;
}

static int ensure_slots(exx_ctx *c, size_t box_max, size_t npe_max, size_t mg_max, bool mixed)
{
    box_max = std::max(box_max, c->box_max);
    npe_max = std::max(npe_max, c->npe_max);
    mg_max = std::max(mg_max, c->mg_max);
    const int bpm = std::max(1, solve_blocks_per_sm(mixed));
    const int n_slots = bpm * c->n_sm;
    // one layout that serves both precisions: boxes and vectors sized for doubles
    // every array sits 128 bytes past a 256-byte boundary with 128 bytes of
    // padding after it, so aligned 16-byte group loads one group beyond either
    // end of a box stay inside the slot
    SolveSlots s{};
    size_t o = 0;
    const size_t boxb = align256(8 * box_max + 256), vecb = align256(8 * std::max(npe_max, box_max) + 256);
    s.off_vbox = o + 128;
    o += boxb;
    s.off_pbox = o + 128;
    o += boxb;
    s.off_rho = o + 128;
    o += align256(8 * npe_max + 256);
    s.off_r64 = o + 128;
    o += align256(8 * npe_max + 256);
    s.off_r = o + 128;
    o += vecb;
    s.off_q = o + 128;
    o += vecb;
    s.off_e = o + 128;
    o += vecb;
    s.off_gs = o + 128;
    o += align256(6 * kGuessBins * kNlm * 4 + 256);
    s.off_b2 = o + 128;
    o += align256(8 * npe_max + 256);
    s.off_zf = o + 128;
    o += align256(4 * box_max + 256);
    s.off_mg = o + 128;
    o += align256(4 * mg_max + 256);
    s.slot_bytes = o;
    s.n_slots = n_slots;
    const size_t need = s.slot_bytes * (size_t)n_slots;
    if (need > c->slots_bytes || box_max > c->box_max || npe_max > c->npe_max || mg_max > c->mg_max) {
        if (c->slots) cudaFree(c->slots);
        c->slots = nullptr;
        c->slots_bytes = 0;
        if (cudaMalloc((void **)&c->slots, need) != cudaSuccess) {
            cudaGetLastError();
            return EXX_ERR_OOM;
        }
        c->slots_bytes = need;
        c->box_max = box_max;
        c->npe_max = npe_max;
        c->mg_max = mg_max;
        c->slots_dirty = true;
    }
    if (c->slots_dirty) {
        CK(cudaMemset(c->slots, 0, c->slots_bytes));
        c->slots_dirty = false;
    }
    s.base = c->slots;
    // the slot count may differ per precision; the memory holds the larger
    const size_t fit = c->slots_bytes / s.slot_bytes;
    s.n_slots = (int)std::min<size_t>((size_t)n_slots, fit);
    (mixed ? c->sl_mixed : c->sl_fp64) = s;
    return EXX_OK;
}

extern "C" {

const char *exx_version(void) { return "exx-gb300 0.1 (sm_103a)"; }

const char *exx_last_error_detail(void) { return g_err_detail; }

const char *exx_error_string(int code)
{
    switch (code) {
    case EXX_OK: return "ok";
    case EXX_ERR_ARG: return "invalid argument";
    case EXX_ERR_CELL: return "cell tensor is singular or left-handed (det h <= 0)";
    case EXX_ERR_HALO: return "R_ME too small: a stencil neighbour of a Poisson point lies outside the ME sphere";
    case EXX_ERR_NK: return "no negative-definite Natan-Kronik stencil for this cell";
    case EXX_ERR_CG_NOT_CONVERGED: return "conjugate gradients reached cg_max_iter for a pair";
    case EXX_ERR_CAPACITY: return "more orbitals or pairs than the plan or context can hold";
    case EXX_ERR_BOX: return "a non-zero D_xx contribution falls outside its D box";
    case EXX_ERR_OOM: return "out of device or pinned host memory";
    case EXX_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown error";
    }
}

int exx_ctx_create(exx_ctx **ctx, int device)
{
    if (!ctx) return EXX_ERR_ARG;
    *ctx = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return EXX_ERR_CUDA;
    }
    CK(cudaSetDevice(device));
    exx_ctx *c = new (std::nothrow) exx_ctx();
    if (!c) return EXX_ERR_OOM;
    c->device = device;
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (const char *s = std::getenv("EXX_INNER_SHIFT")) c->inner_shift = std::max(4, std::min(22, std::atoi(s)));

    *ctx = c;
    return EXX_OK;
}

int exx_ctx_set_solver(exx_ctx *ctx, int solver)
{
    if (!ctx || (solver != EXX_SOLVER_CTA && solver != EXX_SOLVER_CLUSTER)) return EXX_ERR_ARG;
    ctx->solver = solver;
    return EXX_OK;
}

int exx_ctx_set_timing(exx_ctx *c, int enable)
{
    if (!c) return EXX_ERR_ARG;
    CK(cudaSetDevice(c->device));
    if (enable && !c->ev[0])
        for (int k = 0; k < 5; ++k) CK(cudaEventCreate(&c->ev[k]));
    c->timing = enable != 0;
    return EXX_OK;
}

int exx_ctx_get_timing(const exx_ctx *c, double ms[4])
{
    if (!c || !ms) return EXX_ERR_ARG;
    for (int k = 0; k < 4; ++k) ms[k] = c->ms[k];
    return EXX_OK;
}

void exx_ctx_destroy(exx_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    for (int k = 0; k < 5; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->slots) cudaFree(c->slots);
    ListDev &L = c->list;
    dev_free(L.row_count);
    dev_free(L.row_start);
    dev_free(L.cell_start);
    dev_free(L.cell_count);
    dev_free(L.total);
    dev_free(L.pairs);
    dev_free(L.out);
    dev_free(c->d_perm);
    dev_free(c->d_cells);
    dev_free(c->d_res);
    if (c->h_cells) cudaFreeHost(c->h_cells);
    if (c->h_res) cudaFreeHost(c->h_res);
    delete c;
}

int exx_plan_create(exx_ctx *ctx, const exx_cell *cell, const exx_params *params, int max_orb, const int box[3],
                    exx_plan **plan)
{
    if (!plan) return EXX_ERR_ARG;
    *plan = nullptr;
    if (!ctx || !cell || !box || max_orb < 0) return EXX_ERR_ARG;
    int e = check_params(params);
    if (e) return e;
    for (int a = 0; a < 3; ++a)
        if (cell->n[a] < 1 || box[a] < 1 || box[a] > cell->n[a]) return EXX_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    exx_plan *p = new (std::nothrow) exx_plan();
    if (!p) return EXX_ERR_OOM;
    p->ctx = ctx;
    p->device = ctx->device;
    p->cell0 = *cell;
    p->params = *params;
    p->max_orb = max_orb;
    for (int a = 0; a < 3; ++a) p->box[a] = box[a];
    p->sched.precond = params->precond;
    p->sched.omega = (float)kMgOmega;
    p->sched.inner_shift = ctx->inner_shift;
    e = build_geometry(p);
    if (!e && p->sched.precond == EXX_PRECOND_MG && !p->d_mg[0] && !p->d_mg[1])
        p->sched.precond = EXX_PRECOND_NONE;   // no hierarchy for this plan: plain CG
    if (!e) {
        const long long pairs = (long long)max_orb * (max_orb + 1) / 2;
        p->pairs_cap = (int)std::min<long long>(pairs, 1LL << 30);
        if ((e = dev_alloc(&p->d_pairs, std::max(p->pairs_cap, 1))) ||
            (e = dev_alloc(&p->d_out, std::max(p->pairs_cap, 1))))
            ;
    }
    if (!e) {
        // the context's workspace for this plan's solves: cell constants, pair
        // list (for every live plan together) and the persistent solver slots
        ctx->plan_rows += max_orb;
        ctx->plan_pairs += p->pairs_cap;
        p->counted = true;
        size_t box_max = 0, npe_max = 0, mg_max = 0;
        for (int s = 0; s < 2; ++s) {
            box_max = std::max(box_max, (size_t)p->lay[s].box);
            npe_max = std::max(npe_max, (size_t)p->lay[s].n_pe);
            mg_max = std::max(mg_max, (size_t)p->h_mg[s].floats);
        }
        if ((e = ensure_cells(ctx, kMaxBatchCells)) ||
            (e = ensure_list(ctx, (int)std::min<long long>(ctx->plan_rows, 1LL << 30), ctx->plan_pairs)) ||
            (e = ensure_slots(ctx, box_max, npe_max, mg_max, params->precision == EXX_MIXED)))
            ;
    }
    if (e) {
        exx_plan_destroy(p);
        return e;
    }
    *plan = p;
    return EXX_OK;
}

void exx_plan_destroy(exx_plan *p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->counted) {
        p->ctx->plan_rows -= p->max_orb;
        p->ctx->plan_pairs -= p->pairs_cap;
    }
    free_geometry(p);
    dev_free(p->d_phi);
    dev_free(p->d_centres);
    dev_free(p->d_box_lo);
    dev_free(p->d_dxx);
    dev_free(p->d_dbox_lo);
    dev_free(p->d_pairs);
    dev_free(p->d_out);
    dev_free(p->d_warm_map);
    dev_free(p->d_warm_v[0]);
    dev_free(p->d_warm_v[1]);
    delete p;
}

int exx_plan_query(const exx_plan *p, exx_plan_info *info)
{
    if (!p || !info) return EXX_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_pe_self = p->lay[0].n_pe;
    info->n_me_self = p->lay[0].n_pe + p->lay[0].n_shell;
    info->n_pe_pair = p->lay[1].n_pe;
    info->n_me_pair = p->lay[1].n_pe + p->lay[1].n_shell;
    info->mg_levels = p->h_mg[1].nlev;
    for (int l = 0; l < p->h_mg[1].nlev && l < 6; ++l) info->mg_points[l] = l == 0 ? p->lay[1].n_pe : p->h_mg[1].lv[l].n;
    info->n_halo_self = p->lay[0].n_halo;
    info->n_halo_pair = p->lay[1].n_halo;
    info->n_aux = p->stencil.n_aux;
    info->n_stcl = 2 * p->params.fd_order * p->stencil.ndir + 1;
    for (int d = 0; d < 6; ++d) {
        for (int k = 0; k < 3; ++k) info->dirs[d][k] = d < p->stencil.ndir ? p->stencil.dir[d][k] : 0;
        info->coef[d] = d < p->stencil.ndir ? p->stencil.coef[d] : 0.0;
    }
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) info->aux_frozen[a][k] = p->aux[a][k];
    for (int a = 0; a < 3; ++a) {
        info->box_self[a] = p->lay[0].B[a];
        info->box_pair[a] = p->lay[1].B[a];
    }
    const exx_ctx *c = p->ctx;
    const SolveSlots &s = p->params.precision == EXX_MIXED ? c->sl_mixed : c->sl_fp64;
    info->workspace_bytes = (long long)c->slots_bytes;
    info->pair_capacity = p->pairs_cap;
    info->ctas = c->last_path == 1 ? c->last_clusters * kClusterCTAs : s.n_slots;
    info->threads = kSolveThreads;
    info->cluster = c->last_path == 1 ? kClusterCTAs : 1;
    return EXX_OK;
}

int exx_geometry_query(const exx_cell *cell, const exx_params *params, exx_plan_info *info)
{
    if (!cell || !params || !info) return EXX_ERR_ARG;
    int e = check_params(params);
    if (e) return e;
    Metric m;
    if ((e = make_metric(cell->lattice, cell->n, m))) return e;
    Stencil st;
    if ((e = make_stencil(m, params->fd_order, params->nq, nullptr, 0, st))) return e;
    std::memset(info, 0, sizeof(*info));
    const double rpe[2] = {params->r_pe_self, params->r_pe_pair};
    const double rme[2] = {params->r_me_self, params->r_me_pair};
    for (int s = 0; s < 2; ++s) {
        OffsetSet o;
        if ((e = make_offsets(m, rpe[s], rme[s], o))) return e;
        SetLayout L;
        if ((e = make_layout(o, st, params->fd_order, L))) return e;
        (s ? info->n_pe_pair : info->n_pe_self) = L.n_pe;
        (s ? info->n_me_pair : info->n_me_self) = L.n_pe + L.n_shell;
        (s ? info->n_halo_pair : info->n_halo_self) = L.n_halo;
        for (int a = 0; a < 3; ++a) (s ? info->box_pair : info->box_self)[a] = L.B[a];
    }
    info->n_aux = st.n_aux;
    info->n_stcl = 2 * params->fd_order * st.ndir + 1;
    for (int d = 0; d < 6; ++d) {
        for (int k = 0; k < 3; ++k) info->dirs[d][k] = d < st.ndir ? st.dir[d][k] : 0;
        info->coef[d] = d < st.ndir ? st.coef[d] : 0.0;
    }
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) info->aux_frozen[a][k] = a < st.n_aux ? st.dir[3 + a][k] : 0;
    return EXX_OK;
}

int exx_dbox_halfwidth(const exx_cell *cell, const exx_params *params, int hw[3])
{
    if (!cell || !params || !hw) return EXX_ERR_ARG;
    Metric m;
    int e = make_metric(cell->lattice, cell->n, m);
    if (e) return e;
    const double rme = std::max(params->r_me_self, params->r_me_pair);
    for (int a = 0; a < 3; ++a) {
        const double rn = std::sqrt(m.hinv[a][0] * m.hinv[a][0] + m.hinv[a][1] * m.hinv[a][1] + m.hinv[a][2] * m.hinv[a][2]);
        hw[a] = (int)std::ceil((0.5 * params->r_pair + rme) * cell->n[a] * rn) + 1;
    }
    return EXX_OK;
}

int exx_dbox_layout(const exx_cell *cell, const exx_params *params, int n_orb, const double *centres, int dbox[3],
                    int *dbox_lo)
{
    if (!cell || !params || !dbox || n_orb < 0 || (n_orb > 0 && (!centres || !dbox_lo))) return EXX_ERR_ARG;
    int hw[3];
    int e = exx_dbox_halfwidth(cell, params, hw);
    if (e) return e;
    int need[3];
    for (int a = 0; a < 3; ++a) need[a] = std::min(2 * hw[a] + 1, cell->n[a]);
    if (dbox[0] <= 0) {
        for (int a = 0; a < 3; ++a) dbox[a] = need[a];
    } else {
        for (int a = 0; a < 3; ++a)
            if (dbox[a] < need[a] || dbox[a] > cell->n[a]) return EXX_ERR_ARG;
    }
    Metric m;
    if ((e = make_metric(cell->lattice, cell->n, m))) return e;
    for (int i = 0; i < n_orb; ++i) {
        const double *c = centres + 3 * (size_t)i;
        for (int a = 0; a < 3; ++a) {
            double f = m.hinv[a][0] * c[0] + m.hinv[a][1] * c[1] + m.hinv[a][2] * c[2];
            f -= std::floor(f);
            const long long g = (long long)std::floor(f * cell->n[a] + 0.5);
            dbox_lo[3 * (size_t)i + a] = (int)(g - dbox[a] / 2);
        }
    }
    return EXX_OK;
}

int exx_cell_strain(const double *lattice0, const double *lattice, double out[2])
{
    if (!lattice0 || !lattice || !out) return EXX_ERR_ARG;
    double l0[3][3], l1[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            l0[a][b] = lattice0[3 * a + b];
            l1[a][b] = lattice[3 * a + b];
        }
    return cell_strain(l0, l1, out[0], out[1]);
}

int exx_get_pair_list(exx_plan *p, int cap, int *n, int *rows)
{
    if (!p || !n) return EXX_ERR_ARG;
    *n = p->last_count;
    if (p->last_count > cap) return EXX_ERR_CAPACITY;
    if (p->last_count == 0) return EXX_OK;
    if (!rows) return EXX_ERR_ARG;
    std::vector<PairRec> h(p->last_count);
    CK(cudaSetDevice(p->device));
    CK(cudaMemcpy(h.data(), p->d_pairs, sizeof(PairRec) * p->last_count, cudaMemcpyDeviceToHost));
    for (int t = 0; t < p->last_count; ++t) {
        int *r = rows + 8 * (size_t)t;
        r[0] = h[t].i;
        r[1] = h[t].j;
        for (int a = 0; a < 3; ++a) {
            r[2 + a] = h[t].k[a];
            r[5 + a] = h[t].g[a];
        }
    }
    return EXX_OK;
}

int exx_pairs_solve_batch(exx_ctx *ctx, int n_cells, exx_plan *const *plans, const exx_cell *cells,
                          const exx_orbitals *orbs, exx_result *res, void *stream_)
{
    if (!ctx || n_cells < 1 || !plans || !cells || !orbs || !res) return EXX_ERR_ARG;
    if (n_cells > kMaxBatchCells) return EXX_ERR_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    CK(cudaSetDevice(ctx->device));
    cudaGetLastError();   // clear a stale non-sticky error of an earlier unrelated call
    const int prec = plans[0]->params.precision;
    for (int c = 0; c < n_cells; ++c) {
        exx_plan *p = plans[c];
        if (!p || p->ctx != ctx || p->params.precision != prec) return EXX_ERR_ARG;
        if (p->shard_n != plans[0]->shard_n || p->shard_rank != plans[0]->shard_rank) return EXX_ERR_ARG;
        const exx_orbitals &o = orbs[c];
        if (o.n_orb < 0 || o.n_orb > p->max_orb) return EXX_ERR_CAPACITY;
        if (o.n_orb > 0 && (!o.centres || !o.box_lo || !o.phi)) return EXX_ERR_ARG;
        for (int a = 0; a < 3; ++a)
            if (o.box[a] != p->box[a] || cells[c].n[a] != p->cell0.n[a]) return EXX_ERR_ARG;
        if (res[c].dxx && !res[c].dbox_lo) return EXX_ERR_ARG;
        if (p->params.stress_mode == EXX_STRESS_CUBIC && !simple_cubic(cells[c])) return EXX_ERR_ARG;
        if (res[c].dxx)
            for (int a = 0; a < 3; ++a)
                if (res[c].dbox[a] < 1 || res[c].dbox[a] > cells[c].n[a]) return EXX_ERR_ARG;
    }
    // geometry for the current cells
    for (int c = 0; c < n_cells; ++c) {
        exx_plan *p = plans[c];
        if (same_cell(cells[c], p->cell)) continue;
        int e;
        if (p->params.frozen) {
            e = update_metric(p, cells[c]);
        } else {
            p->cell0 = cells[c];
            e = build_geometry(p);
        }
        if (e) return e;
    }
    // cells queued by decreasing per-pair cost (largest Poisson subdomain first)
    std::vector<int> order(n_cells);
    for (int c = 0; c < n_cells; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return plans[a]->lay[1].n_pe > plans[b]->lay[1].n_pe;
    });
    int e = ensure_cells(ctx, n_cells);
    if (e) return e;
    int rows = 0;
    long long pairs = 0;
    size_t box_max = 0, npe_max = 0, mg_max = 0;
    for (int c = 0; c < n_cells; ++c) {
        rows += orbs[c].n_orb;
        pairs += (long long)orbs[c].n_orb * (orbs[c].n_orb + 1) / 2;
        for (int s = 0; s < 2; ++s) {
            box_max = std::max(box_max, (size_t)plans[c]->lay[s].box);
            npe_max = std::max(npe_max, (size_t)plans[c]->lay[s].n_pe);
            mg_max = std::max(mg_max, (size_t)plans[c]->h_mg[s].floats);
        }
    }
    if ((e = ensure_list(ctx, rows, pairs))) return e;
    if ((e = ensure_slots(ctx, box_max, npe_max, mg_max, prec == EXX_MIXED))) return e;

    // stage inputs and fill the per-cell constants (queue order)
    int row_base = 0;
    for (int qi = 0; qi < n_cells; ++qi) {
        const int c = order[qi];
        exx_plan *p = plans[c];
        const exx_orbitals &o = orbs[c];
        exx_result &r = res[c];
        CellDev &C = ctx->h_cells[qi];
        if (!p->tables_valid && (e = upload_guess_bins(p))) return e;   // radial bins for the current cell
        fill_celldev(p, C);
        C.n_orb = o.n_orb;
        for (int a = 0; a < 3; ++a) C.box[a] = o.box[a];
        C.row_base = row_base;
        C.cell_index = c;
        row_base += o.n_orb;
        if (p->params.warm_start) {
            if (p->warm_norb != o.n_orb) {
                p->warm_n = 0;
                p->warm_norb = o.n_orb;
            }
            if (!p->d_warm_map && p->max_orb > 0) {
                if ((e = dev_alloc(&p->d_warm_map, (size_t)p->max_orb * p->max_orb))) return e;
                CK(cudaMemsetAsync(p->d_warm_map, 0xff, 4 * (size_t)p->max_orb * p->max_orb, stream));
            }
            p->warm_stride = std::max(p->lay[0].n_pe, p->lay[1].n_pe);
            if (p->warm_n > 0) {
                C.warm_map = p->d_warm_map;
                C.warm_rows = p->d_pairs;
                C.warm_prev = p->d_warm_v[p->warm_cur];
            }
            C.warm_next = p->d_warm_v[1 - p->warm_cur];
            C.warm_cap = C.warm_next ? p->warm_cap : 0;
            for (int s2 = 0; s2 < 2; ++s2) C.warm_inv[s2] = p->d_inv[s2];
            C.warm_stride = p->warm_stride;
        }
        const size_t bsz = (size_t)o.box[0] * o.box[1] * o.box[2];
        if (o.mem == EXX_MEM_HOST && o.n_orb > 0) {
            if (!p->d_phi) {
                if ((e = dev_alloc(&p->d_phi, bsz * p->max_orb)) || (e = dev_alloc(&p->d_centres, 3 * (size_t)p->max_orb)) ||
                    (e = dev_alloc(&p->d_box_lo, 3 * (size_t)p->max_orb)))
                    return e;
            }
            CK(cudaMemcpyAsync(p->d_phi, o.phi, 8 * bsz * o.n_orb, cudaMemcpyHostToDevice, stream));
            CK(cudaMemcpyAsync(p->d_centres, o.centres, 24 * (size_t)o.n_orb, cudaMemcpyHostToDevice, stream));
            CK(cudaMemcpyAsync(p->d_box_lo, o.box_lo, 12 * (size_t)o.n_orb, cudaMemcpyHostToDevice, stream));
            C.phi = p->d_phi;
            C.centres = p->d_centres;
            C.box_lo = p->d_box_lo;
        } else {
            C.phi = o.phi;
            C.centres = o.centres;
            C.box_lo = o.box_lo;
        }
        C.dxx = nullptr;
        if (r.dxx) {
            const size_t dsz = (size_t)r.dbox[0] * r.dbox[1] * r.dbox[2] * o.n_orb;
            for (int a = 0; a < 3; ++a) C.dbox[a] = r.dbox[a];
            if (r.mem == EXX_MEM_HOST) {
                if (p->dxx_cap < dsz) {
                    dev_free(p->d_dxx);
                    dev_free(p->d_dbox_lo);
                    if ((e = dev_alloc(&p->d_dxx, dsz)) || (e = dev_alloc(&p->d_dbox_lo, 3 * (size_t)p->max_orb))) return e;
                    p->dxx_cap = dsz;
                }
                CK(cudaMemcpyAsync(p->d_dbox_lo, r.dbox_lo, 12 * (size_t)o.n_orb, cudaMemcpyHostToDevice, stream));
                C.dxx = p->d_dxx;
                C.dbox_lo = p->d_dbox_lo;
            } else {
                C.dxx = r.dxx;
                C.dbox_lo = r.dbox_lo;
            }
            if (dsz) CK(cudaMemsetAsync(C.dxx, 0, 8 * dsz, stream));
        }
    }
    CK(cudaMemcpyAsync(ctx->d_cells, ctx->h_cells, sizeof(CellDev) * n_cells, cudaMemcpyHostToDevice, stream));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[0], stream));
    for (int qi = 0; qi < n_cells; ++qi) {
        exx_plan *p = plans[order[qi]];
        if (p->tables_valid) continue;
        for (int s = 0; s < 2; ++s) {
            const SetLayout &L = p->lay[s];
            CK(launch_tables(ctx->d_cells + qi, s, L.n_pe + L.n_shell, p->d_S64[s], p->d_S32[s], p->d_T64[s],
                             p->d_T32[s], stream));
            CK(launch_gather_rows(p->d_S32[s], p->d_gs_perm[s], L.n_pe, p->d_gs_S32[s], stream));
            CK(launch_guess_info(p->d_gs_perm[s], p->d_gs_bin[s], p->d_pe_m[s], p->d_pe_off[s], L.n_pe,
                                 p->d_gs_info[s], stream));
        }
        p->tables_valid = true;
    }
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], stream));
    CK(launch_pair_list(ctx->d_cells, n_cells, rows, ctx->list, stream));
    if (ctx->sample_limit > 0) CK(launch_clamp_total(ctx->list, ctx->sample_limit, stream));
    ListDev Lsolve = ctx->list;   // the solver's view of the list (a rank's share when sharded)
    if (plans[0]->shard_n > 1) {
        // this rank's pairs by the LPT partition of the whole list (the same on every rank)
        int total = 0;
        CK(cudaMemcpyAsync(&total, ctx->list.total, 4, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        std::vector<PairRec> h_rows((size_t)std::max(total, 1));
        if (total > 0)
            CK(cudaMemcpy(h_rows.data(), ctx->list.pairs, sizeof(PairRec) * (size_t)total, cudaMemcpyDeviceToHost));
        std::vector<double> cost((size_t)total);
        for (int k = 0; k < total; ++k) {
            const PairRec &pr = h_rows[(size_t)k];
            cost[(size_t)k] = plans[order[pr.cell]]->lay[pr.i == pr.j ? 0 : 1].n_pe;
        }
        std::vector<int> owner((size_t)total), own;
        lpt_partition(cost.data(), total, plans[0]->shard_n, owner.data());
        for (int k = 0; k < total; ++k)
            if (owner[(size_t)k] == plans[0]->shard_rank) own.push_back(k);
        const int n_own = (int)own.size();
        if (n_own) CK(cudaMemcpy(ctx->d_perm, own.data(), 4 * (size_t)n_own, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->list.total, &n_own, 4, cudaMemcpyHostToDevice));
        if (total) CK(cudaMemsetAsync(ctx->list.out, 0, sizeof(PairOut) * (size_t)total, stream));
        Lsolve.perm = ctx->d_perm;
    }
    // warm start: the solution stores must hold this solve's pairs (count read back once)
    bool any_warm = false;
    for (int c = 0; c < n_cells; ++c) any_warm |= plans[c]->params.warm_start != 0;
    if (any_warm) {
        int cnt_now[64];
        CK(cudaMemcpyAsync(cnt_now, ctx->list.cell_count, 4 * n_cells, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        bool reupload = false;
        for (int qi = 0; qi < n_cells; ++qi) {
            exx_plan *p = plans[order[qi]];
            if (!p->params.warm_start || cnt_now[qi] <= p->warm_cap) continue;
            const int cap = (int)std::min<long long>((long long)cnt_now[qi] * 5 / 4 + 64, p->pairs_cap);
            float *nv[2] = {nullptr, nullptr};
            if ((e = dev_alloc(&nv[0], (size_t)cap * p->warm_stride)) ||
                (e = dev_alloc(&nv[1], (size_t)cap * p->warm_stride))) {
                dev_free(nv[0]);
                return e;
            }
            if (p->warm_n > 0)
                CK(cudaMemcpyAsync(nv[0], p->d_warm_v[p->warm_cur], 4 * (size_t)p->warm_n * p->warm_stride,
                                   cudaMemcpyDeviceToDevice, stream));
            CK(cudaStreamSynchronize(stream));
            dev_free(p->d_warm_v[0]);
            dev_free(p->d_warm_v[1]);
            p->d_warm_v[0] = nv[0];
            p->d_warm_v[1] = nv[1];
            p->warm_cur = 0;
            p->warm_cap = cap;
            CellDev &C = ctx->h_cells[qi];
            C.warm_prev = p->warm_n > 0 ? p->d_warm_v[0] : nullptr;
            C.warm_next = p->d_warm_v[1];
            C.warm_cap = cap;
            reupload = true;
        }
        if (reupload)
            CK(cudaMemcpyAsync(ctx->d_cells, ctx->h_cells, sizeof(CellDev) * n_cells, cudaMemcpyHostToDevice, stream));
    }
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[2], stream));
    const bool mixed = prec == EXX_MIXED;
    // the cluster path takes the launch when every set of every cell has a row
    // partition and its CG state fits in the cluster's shared memory
    bool use_cluster = mixed && ctx->solver == EXX_SOLVER_CLUSTER;
    int rowtab_words = 0, cl_p = 0, cl_g = 800;   // r, q, e regions double as the moments' scratch
    for (int c = 0; c < n_cells && use_cluster; ++c)
        for (int s = 0; s < 2; ++s) {
            const exx_plan *p = plans[c];
            if (!p->cl_ok[s]) {
                use_cluster = false;
                break;
            }
            rowtab_words = std::max(rowtab_words, p->lay[s].B[0] * p->lay[s].B[1]);
            cl_p = std::max(cl_p, p->cpart[s].max_p_floats);
            cl_g = std::max(cl_g, p->cpart[s].max_groups);
        }
    if (use_cluster) {
        if (ctx->cluster_cap < 0) ctx->cluster_cap = cluster_capacity_bytes();
        if (cluster_dyn_bytes(rowtab_words, cl_p, cl_g) > (size_t)ctx->cluster_cap) use_cluster = false;
    }
    ctx->last_path = use_cluster ? 1 : 0;
    if (use_cluster)
        CK(launch_solve_cluster(ctx->d_cells, Lsolve, ctx->sl_mixed, rowtab_words, cl_p, cl_g, ctx->inner_shift,
                                &ctx->last_clusters, stream));
    else
        CK(launch_solve(ctx->d_cells, Lsolve, mixed ? ctx->sl_mixed : ctx->sl_fp64, mixed, ctx->inner_shift, stream));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[3], stream));
    CK(launch_finalize(ctx->d_cells, n_cells, ctx->list, ctx->d_res, stream));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[4], stream));
    CK(cudaMemcpyAsync(ctx->h_res, ctx->d_res, sizeof(CellResult) * n_cells, cudaMemcpyDeviceToHost, stream));
    int h_start[64], h_count[64];
    CK(cudaMemcpyAsync(h_start, ctx->list.cell_start, 4 * n_cells, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(h_count, ctx->list.cell_count, 4 * n_cells, cudaMemcpyDeviceToHost, stream));
    if (cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        ctx->slots_dirty = true;
        return EXX_ERR_CUDA;
    }
    if (ctx->timing)
        for (int k = 0; k < 4; ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ctx->ev[k], ctx->ev[k + 1]);
            ctx->ms[k] = t;
        }
    int status = EXX_OK;
    for (int qi = 0; qi < n_cells; ++qi) {
        const int c = order[qi];
        exx_plan *p = plans[c];
        exx_result &r = res[c];
        const CellResult &cr = ctx->h_res[qi];
        const int cnt = cr.status == EXX_ERR_CAPACITY ? 0 : h_count[qi];
        r.e_xx = cr.e_xx;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                r.dedh[a][b] = cr.dedh[3 * a + b];
                r.stress[a][b] = cr.stress[3 * a + b];
            }
        r.n_pairs = cnt;
        r.n_aux = p->stencil.n_aux;
        r.n_stcl = 2 * p->params.fd_order * p->stencil.ndir + 1;
        r.max_cg_iter = cr.max_iter;
        r.total_cg_iter = cr.total_iter;
        r.max_refine = cr.max_refine;
        r.total_refine = cr.total_refine;
        r.failed_pair = cr.failed_pair;
        r.n_warm = cr.pad;
        r.p_int = (r.stress[0][0] + r.stress[1][1] + r.stress[2][2]) / 3.0;
        if (p->params.stress_mode == EXX_STRESS_CUBIC) {
            // Eqs. liq_press, dexxdL: p_int = E_xx / (3V), Tr sigma = -E_xx / L
            const double L = cells[c].lattice[0][0];
            r.p_int = r.e_xx / (3.0 * L * L * L);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) r.dedh[a][b] = a == b ? -r.e_xx / (3.0 * L) : 0.0;
        }
        if (p->params.stress_mode != EXX_STRESS_FULL)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) r.stress[a][b] = a == b ? r.p_int : 0.0;
        // keep this cell's pair list and per-pair outputs with the plan
        p->last_count = std::min(cnt, p->pairs_cap);
        if (p->last_count) {
            CK(cudaMemcpyAsync(p->d_pairs, ctx->list.pairs + h_start[qi], sizeof(PairRec) * p->last_count,
                               cudaMemcpyDeviceToDevice, stream));
            CK(cudaMemcpyAsync(p->d_out, ctx->list.out + h_start[qi], sizeof(PairOut) * p->last_count,
                               cudaMemcpyDeviceToDevice, stream));
        }
        if (p->params.warm_start && p->d_warm_map) {
            // the solutions just stored become the guesses of the next solve; index them by (i, j)
            p->warm_cur = 1 - p->warm_cur;
            p->warm_n = std::min(p->last_count, p->warm_cap);
            CK(cudaMemsetAsync(p->d_warm_map, 0xff, 4 * (size_t)p->max_orb * p->max_orb, stream));
            if (p->warm_n > 0) CK(launch_warm_map(p->d_pairs, p->warm_n, orbs[c].n_orb, p->d_warm_map, stream));
        }
        if (r.dxx && r.mem == EXX_MEM_HOST) {
            const size_t dsz = (size_t)r.dbox[0] * r.dbox[1] * r.dbox[2] * orbs[c].n_orb;
            if (dsz) CK(cudaMemcpyAsync(r.dxx, p->d_dxx, 8 * dsz, cudaMemcpyDeviceToHost, stream));
        }
        if (cr.status && status == EXX_OK) status = cr.status;
    }
    // optional per-pair outputs
    bool any_pair_out = false;
    for (int c = 0; c < n_cells; ++c)
        if (res[c].pair_e || res[c].pair_sig || res[c].pair_iter) any_pair_out = true;
    if (any_pair_out) {
        CK(cudaStreamSynchronize(stream));
        for (int c = 0; c < n_cells; ++c) {
            exx_plan *p = plans[c];
            exx_result &r = res[c];
            if (!(r.pair_e || r.pair_sig || r.pair_iter)) continue;
            if (p->last_count > r.pair_cap) {
                if (status == EXX_OK) status = EXX_ERR_CAPACITY;
                continue;
            }
            std::vector<PairOut> h(p->last_count);
            if (p->last_count)
                CK(cudaMemcpy(h.data(), p->d_out, sizeof(PairOut) * p->last_count, cudaMemcpyDeviceToHost));
            std::vector<double> e(p->last_count), sg(9 * (size_t)p->last_count);
            std::vector<int> it(p->last_count);
            for (int t = 0; t < p->last_count; ++t) {
                e[t] = h[t].e;
                for (int k = 0; k < 9; ++k) sg[9 * (size_t)t + k] = h[t].sig[k];
                it[t] = h[t].iters;
            }
            const cudaMemcpyKind kind = r.mem == EXX_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
            if (r.pair_e && p->last_count) CK(cudaMemcpy(r.pair_e, e.data(), 8 * (size_t)p->last_count, kind));
            if (r.pair_sig && p->last_count) CK(cudaMemcpy(r.pair_sig, sg.data(), 72 * (size_t)p->last_count, kind));
            if (r.pair_iter && p->last_count) CK(cudaMemcpy(r.pair_iter, it.data(), 4 * (size_t)p->last_count, kind));
        }
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return EXX_ERR_CUDA;
    }
    return status;
}

int exx_pairs_solve(exx_ctx *ctx, exx_plan *plan, const exx_cell *cell, const exx_orbitals *orb, exx_result *res,
                    void *stream)
{
    if (!plan) return EXX_ERR_ARG;
    exx_plan *plans[1] = {plan};
    return exx_pairs_solve_batch(ctx, 1, plans, cell, orb, res, stream);
}

int exx_plan_set_shard(exx_plan *plan, int rank, int n_ranks)
{
    if (!plan || n_ranks < 1 || rank < 0 || rank >= n_ranks) return EXX_ERR_ARG;
    plan->shard_rank = rank;
    plan->shard_n = n_ranks;
    return EXX_OK;
}

int exx_pair_partition(const exx_cell *cell, const exx_params *params, int n_pairs, const int *rows, int n_ranks,
                       int *owner)
{
    if (!cell || !params || n_pairs < 0 || n_ranks < 1 || (n_pairs > 0 && (!rows || !owner))) return EXX_ERR_ARG;
    int e = check_params(params);
    if (e) return e;
    Metric m;
    if ((e = make_metric(cell->lattice, cell->n, m))) return e;
    const double rpe[2] = {params->r_pe_self, params->r_pe_pair};
    const double rme[2] = {params->r_me_self, params->r_me_pair};
    double npe[2];
    for (int s = 0; s < 2; ++s) {
        OffsetSet o;
        if ((e = make_offsets(m, rpe[s], rme[s], o))) return e;
        npe[s] = o.n_pe;
    }
    std::vector<double> cost((size_t)n_pairs);
    for (int k = 0; k < n_pairs; ++k) cost[(size_t)k] = npe[rows[8 * (size_t)k] == rows[8 * (size_t)k + 1] ? 0 : 1];
    lpt_partition(cost.data(), n_pairs, n_ranks, owner);
    return EXX_OK;
}

int exx_plan_get_schedule(const exx_plan *plan, exx_schedule *sched)
{
    if (!plan || !sched) return EXX_ERR_ARG;
    *sched = plan->sched;
    return EXX_OK;
}

int exx_plan_set_schedule(exx_plan *plan, const exx_schedule *sched)
{
    if (!plan || !sched) return EXX_ERR_ARG;
    if (sched->precond != EXX_PRECOND_NONE && sched->precond != EXX_PRECOND_MG) return EXX_ERR_ARG;
    if (!(sched->omega > 0.f && sched->omega <= 1.f) || sched->inner_shift < 4 || sched->inner_shift > 22)
        return EXX_ERR_ARG;
    if (sched->precond == EXX_PRECOND_MG && !plan->d_mg[0] && !plan->d_mg[1]) return EXX_ERR_ARG;
    plan->sched = *sched;
    return EXX_OK;
}

int exx_plan_autotune(exx_ctx *ctx, exx_plan *plan, const exx_cell *cell, const exx_orbitals *orb, int sample_pairs,
                      exx_schedule *chosen, void *stream)
{
    if (!ctx || !plan || !cell || !orb || sample_pairs < 1 || plan->ctx != ctx) return EXX_ERR_ARG;
    std::vector<exx_schedule> cand =
        schedule_candidates(plan->params.precision == EXX_MIXED && (plan->d_mg[0] || plan->d_mg[1]), kMgOmega);
    if (plan->params.precision != EXX_MIXED) {
        plan->sched.precond = EXX_PRECOND_NONE;
        plan->sched.ms = 0.0;
        if (chosen) *chosen = plan->sched;
        return EXX_OK;
    }
    const exx_schedule keep = plan->sched;
    const bool timing = ctx->timing;
    ctx->timing = true;
    ctx->sample_limit = sample_pairs;
    std::vector<double> ms(cand.size(), 0.0);
    int e = EXX_OK;
    for (size_t k = 0; k < cand.size() && !e; ++k) {
        plan->sched = cand[k];
        double best = 1e300;
        for (int rep = 0; rep < 2 && !e; ++rep) {
            exx_result r{};
            e = exx_pairs_solve(ctx, plan, cell, orb, &r, stream);
            if (e == EXX_ERR_CG_NOT_CONVERGED) {   // a schedule that fails the sample is never chosen
                e = EXX_OK;
                best = 1e300;
                break;
            }
            best = std::min(best, ctx->ms[2]);
        }
        ms[k] = best;
    }
    ctx->sample_limit = 0;
    ctx->timing = timing;
    if (e) {
        plan->sched = keep;
        return e;
    }
    const int pick = pick_schedule(ms.data(), (int)ms.size());
    if (pick < 0) {
        plan->sched = keep;
        return EXX_ERR_CG_NOT_CONVERGED;
    }
    plan->sched = cand[pick];
    plan->sched.ms = ms[pick];
    if (chosen) *chosen = plan->sched;
    return EXX_OK;
}

}  // extern "C"
