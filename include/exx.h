/*
 * exx.h -- C ABI of the GB300 exact-exchange (EXX) pair path.
 *
 * The library evaluates, on one GPU, the linear-scaling exact-exchange
 * quantities of Ko, Santra & DiStasio (arXiv 2011.07209) for a set of
 * localized orbitals phi_i (maximally localized Wannier functions) in a
 * general, possibly fluctuating, simulation cell:
 *
 *   E_xx      = - sum_<ij> w_ij  int_PE rho_ij v_ij                 (Eq. exxGen_mlwf)
 *   D_xx^i    =   sum_j v_ij phi_j                                  (Eq. Dxx)
 *   sigma^{a alpha} = dE_xx/dh_{a alpha}
 *             = -2 sum_<ij> w_ij sum_b (h^-1)_{alpha b} int_PE r_b rho_ij d_a v_ij   (Eq. sxx_working)
 *   Pi_ab     = -(1/V) sum_alpha sigma^{a alpha} h_{b alpha}        (Eq. pixx_working)
 *
 * over the unique pairs <ij> (i <= j, w_ii = 1, w_ij = 2) whose centres are
 * within R_pair (Sec. III A, Step II).  For each pair the library forms
 * rho_ij = phi_i phi_j on the Poisson subdomain of radius R_PE around the
 * grid-resolved pair centre (Step III), takes its multipole moments up to
 * l_max (Eq. mepole), sets the far field on the shell R_PE < r <= R_ME
 * (Eq. me), and solves Poisson's equation (Eq. pe) by conjugate gradients with
 * the Natan-Kronik finite-difference Laplacian of Eq. lapG_mod_nk3d, whose
 * auxiliary directions come from the 2D bisector rule (Eqs. nk2d_aux,
 * kappa_def) or Algorithm 1 (Step IV).  Every step runs in CUDA kernels for
 * sm_103a; there is no CPU fallback.
 *
 * Units: Hartree atomic units (bohr, Ha).  E_xx is not scaled by the hybrid
 * mixing fraction a_x (Eq. hyb); D_xx carries no spin or occupation factor.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Cell: lattice[alpha][a] = (L_alpha)_a (rows are lattice vectors); the
 *    cell tensor of the paper is h = lattice^T (Sec. II B 1).  The cell must be
 *    right-handed (det h > 0).  Grid point g sits at r = h (g / n).
 *  - Orbital boxes: orbital i is stored on a box of box[0] x box[1] x box[2]
 *    grid points, C order, whose element (u0,u1,u2) is the grid point
 *    (box_lo[i] + u) mod n; the orbital is zero outside its box.  box[a] <= n[a].
 *  - D boxes: D_xx^i is written on a box of dbox[] points starting at
 *    dbox_lo[i], same layout.  A non-zero contribution that falls outside the
 *    D box is an error (EXX_ERR_BOX); exx_dbox_halfwidth() gives a size that
 *    always suffices.
 *  - Memory: pointers are device pointers unless the structure's mem field is
 *    EXX_MEM_HOST, in which case the library copies them through its own
 *    device workspace (host memory should be pinned for speed).  The caller
 *    owns every input and output buffer; the library owns its workspace.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  The
 *    solve entry points enqueue all work on it and return after it finishes,
 *    with the scalar results in host memory.
 *  - Errors: every entry point returns an exx_status; EXX_OK is 0.
 *    exx_error_string() gives a static message.  A failed call leaves the
 *    context usable.
 *  - Threads: a context may be used by one host thread at a time.
 */
#ifndef EXX_H
#define EXX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EXX_OK = 0,
    EXX_ERR_ARG = 1,                 /* bad argument or inconsistent sizes                  */
    EXX_ERR_CELL = 2,                /* det h <= 0: singular or left-handed cell            */
    EXX_ERR_HALO = 3,                /* R_ME too small: a stencil neighbour of a PE point   */
                                     /* lies outside PE u shell                              */
    EXX_ERR_NK = 4,                  /* no negative-definite Natan-Kronik stencil found     */
    EXX_ERR_CG_NOT_CONVERGED = 5,    /* a pair hit cg_max_iter; see exx_result.failed_pair  */
    EXX_ERR_CAPACITY = 6,            /* more orbitals/pairs than the plan was sized for     */
    EXX_ERR_BOX = 7,                 /* non-zero D contribution outside a D box             */
    EXX_ERR_OOM = 8,                 /* device or pinned allocation failed                  */
    EXX_ERR_CUDA = 9                 /* a CUDA runtime call failed                          */
} exx_status;

enum { EXX_FP64 = 0, EXX_MIXED = 1 };          /* exx_params.precision */
enum { EXX_SOLVER_CTA = 0, EXX_SOLVER_CLUSTER = 1 };   /* exx_ctx_set_solver */
enum { EXX_MEM_DEVICE = 0, EXX_MEM_HOST = 1 };  /* memory kind of caller buffers */
/* exx_params.stress_mode (Sec. II C, "Isotropic Constraints"):
 *   EXX_STRESS_FULL       sigma and the full Pi_xx^pot (Eqs. sxx_working, pixx_working);
 *   EXX_STRESS_ISOTROPIC  sigma as above, Pi_xx^pot replaced by p_int delta_ab with
 *                         p_int = Tr Pi / 3 (Eq. pxx_working);
 *   EXX_STRESS_CUBIC      simple cubic cells only (lattice = L I): the sigma integrals
 *                         are skipped and p_int = E_xx / (3V) (Eq. liq_press), Pi =
 *                         p_int delta_ab, sigma^{a alpha} = -E_xx / (3L) delta_{a alpha}
 *                         (so that Tr sigma = dE_xx/dL = -E_xx/L, Eq. dexxdL).  Any
 *                         other cell returns EXX_ERR_ARG. */
enum { EXX_STRESS_FULL = 0, EXX_STRESS_ISOTROPIC = 1, EXX_STRESS_CUBIC = 2 };
enum { EXX_PRECOND_NONE = 0, EXX_PRECOND_MG = 1 };   /* exx_params.precond */

typedef struct exx_ctx exx_ctx;
typedef struct exx_plan exx_plan;

typedef struct {
    double lattice[3][3];   /* rows = lattice vectors L_alpha, Cartesian bohr */
    int n[3];               /* grid points along L_alpha, each >= 1 */
} exx_cell;

typedef struct {
    double r_pair;          /* pair cutoff on |C_i - C_j| (minimum image), bohr (Sec. III A) */
    double r_pe_self;       /* Poisson-subdomain radius for i == j pairs */
    double r_pe_pair;       /* Poisson-subdomain radius for i != j pairs */
    double r_me_self;       /* outer radius of the multipole shell, i == j */
    double r_me_pair;       /* outer radius of the multipole shell, i != j */
    double cg_tol;          /* stop when |b - A v|_2 <= cg_tol |b|_2 (true residual) */
    int fd_order;           /* stencil half-width n of Eq. d2_1, 1..6 (paper default 3) */
    int lmax;               /* multipole order, 0..6 */
    int cg_max_iter;        /* cap on CG iterations per pair (summed over refinements) */
    int nq;                 /* NK candidate count N_q of Algorithm 1 (paper default 15) */
    int precision;          /* EXX_FP64: every step in FP64.  EXX_MIXED: FP32 stencil and */
                            /* axpy inside a true-residual refinement loop; dot products  */
                            /* exact-product double-float; moments and far field from     */
                            /* FP32 tables with FP64 sums; the true residuals, the        */
                            /* solution update and E, sigma in double-float (FP32 hi/lo   */
                            /* pairs, about 48 bits) on the CTA solver, FP64 on the       */
                            /* cluster solver and for fd_order > 4; D in FP64 from an     */
                            /* FP32 far field on the shell                                */
    int frozen;             /* 1: subdomain offsets and NK aux directions stay those of the */
                            /* plan's cell while h changes (fixed number of points,         */
                            /* Sec. III B 2); 0: rebuilt whenever the cell changes          */
    int stress_mode;        /* EXX_STRESS_FULL (0), EXX_STRESS_ISOTROPIC or EXX_STRESS_CUBIC */
    int warm_start;         /* 1: each pair's CG starts from that pair's solution of the     */
                            /* previous solve with this plan (same i, j and lattice image;   */
                            /* shifted by the change of the grid-resolved pair centre; zero  */
                            /* where the shifted point leaves PE) -- the guess from the      */
                            /* previous MD step of Sec. III B 2.  The plan keeps one FP32    */
                            /* solution per pair (2 x n_pairs x N_PE x 4 bytes of device     */
                            /* memory).  The stopping rule is unchanged (|b - A v| <= tol |b|). */
                            /* With guess = 1 the previous solution is kept only when its    */
                            /* residual is at most 5 % of |b|; otherwise the pair starts     */
                            /* from the multipole guess (large MD steps).                    */
                            /* 0: every CG starts from v = 0 (or the multipole guess).        */
    int guess;              /* 1 (default of the Python binding): a pair's CG without a warm */
                            /* start begins from the free-space potential of rho_ij on PE,   */
                            /* built from its multipole moments in radial bins (the far     */
                            /* field of Eq. me continued inside), which removes about a      */
                            /* quarter of the iterations; 0: from v = 0.  Only the starting  */
                            /* point changes: the stopping rule and the solution do not.     */
                            /* The cluster solver (exx_ctx_set_solver) ignores it.           */
    int precond;            /* EXX_PRECOND_MG (1, default of the Python binding): the mixed  */
                            /* path's CG is preconditioned by one multigrid V(1,1) cycle     */
                            /* per iteration (weighted Jacobi smoothing, trilinear transfers, */
                            /* Galerkin coarse operators built per plan on the host, the     */
                            /* inverse of the coarsest one), which cuts the iterations by    */
                            /* about a factor of ten.  The paper's CG is plain: only the     */
                            /* iterates change, not the discrete equations or the stopping   */
                            /* rule.  Used for fd_order <= 3 on the CTA solver; elsewhere,   */
                            /* and with EXX_PRECOND_NONE (0), the CG is plain.  The FP64     */
                            /* path is always plain CG.                                      */
} exx_params;

typedef struct {
    int n_orb;              /* number of orbitals */
    int box[3];             /* orbital box extent */
    const double *centres;  /* [n_orb][3] Cartesian centres C_i, bohr */
    const int *box_lo;      /* [n_orb][3] first grid index of each box */
    const double *phi;      /* [n_orb][box0][box1][box2] orbital values, FP64 (the only type) */
    int mem;                /* EXX_MEM_DEVICE or EXX_MEM_HOST for the three arrays */
} exx_orbitals;

typedef struct {
    /* ---- inputs describing the caller's output buffers ---- */
    double *dxx;            /* [n_orb][dbox0][dbox1][dbox2] D_xx (zeroed by the call), or NULL */
    const int *dbox_lo;     /* [n_orb][3] first grid index of each D box (required with dxx) */
    int dbox[3];            /* D box extent */
    int mem;                /* EXX_MEM_DEVICE or EXX_MEM_HOST for dxx, dbox_lo and pair arrays */
    int pair_cap;           /* capacity of the optional per-pair arrays below */
    double *pair_e;         /* [pair_cap] int_PE rho v per pair, or NULL */
    double *pair_sig;       /* [pair_cap][3][3] sum_b hinv_{alpha b} int r_b rho d_a v, [a][alpha], or NULL */
    int *pair_iter;         /* [pair_cap] CG iterations per pair, or NULL */
    /* ---- scalar outputs (host) ---- */
    double e_xx;            /* Ha */
    double dedh[3][3];      /* sigma^{a alpha} = dE_xx / dh_{a alpha}, Ha/bohr */
    double stress[3][3];    /* Pi_xx^pot, Ha/bohr^3 */
    int n_pairs;            /* unique pairs found */
    int n_aux;              /* NK auxiliary directions used (0, 1 or 3) */
    int n_stcl;             /* stencil points 2 n (3 + n_aux) + 1 */
    int max_cg_iter;        /* largest per-pair CG iteration count */
    long long total_cg_iter;/* CG iterations summed over pairs */
    int max_refine;         /* largest number of true-residual evaluations of a pair */
    int failed_pair;        /* index of the first failed pair, or -1 */
    long long total_refine; /* true-residual evaluations summed over pairs */
    double p_int;           /* EXX contribution to the internal pressure, Tr Pi_xx^pot / 3,  */
                            /* Ha/bohr^3 (Eq. pxx_working; Eq. liq_press in EXX_STRESS_CUBIC) */
    int n_warm;             /* pairs that started from a previous solution (warm_start)      */
} exx_result;

typedef struct {
    int n_pe_self, n_me_self, n_pe_pair, n_me_pair;   /* subdomain sizes N_PE, N_ME */
    int n_halo_self, n_halo_pair;                     /* shell points the stencil reaches */
    int n_aux, n_stcl;
    int dirs[6][3];         /* integer grid step of each pure-derivative direction */
    double coef[6];         /* coefficient of sum_q w_q f(g + q d) per direction, 1/bohr^2 */
    int aux_frozen[3][3];   /* aux directions held when params.frozen = 1 */
    int box_self[3], box_pair[3];    /* dense CG boxes (PE plus stencil margin) */
    long long workspace_bytes;
    int pair_capacity;      /* largest number of pairs a solve can hold */
    int ctas;               /* persistent CTAs of the pair kernel (of the context's last solve) */
    int threads;            /* threads per CTA */
    int cluster;            /* CTAs per pair: 1 (one CTA per pair) or the cluster size of the */
                            /* cluster path, which keeps a pair's FP32 CG state in the       */
                            /* distributed shared memory of a thread-block cluster           */
    int mg_levels;          /* multigrid levels of the non-self set (fine level included; 0: */
                            /* no hierarchy), and their active points                        */
    int mg_points[6];
} exx_plan_info;

/* Schedule of a plan's mixed-precision pair solver (Step IV): the knobs that
 * change how fast the CG converges, never what it converges to (the stopping
 * rule |b - A v| <= cg_tol |b| on the true residual is fixed).  Set from
 * exx_params at plan creation; chosen per plan by exx_plan_autotune. */
typedef struct {
    int precond;            /* EXX_PRECOND_NONE or EXX_PRECOND_MG */
    float omega;            /* weighted-Jacobi factor of the V-cycle, in (0, 1] (default 0.8) */
    int inner_shift;        /* reliable update (double-float true residual) once the FP32    */
                            /* residual fell by 2^-inner_shift, 4..22 (default 14)          */
    double ms;              /* exx_plan_autotune: measured solver time of the sample, ms    */
} exx_schedule;

/* Create a context on CUDA device `device` (made current for the call). */
int exx_ctx_create(exx_ctx **ctx, int device);
void exx_ctx_destroy(exx_ctx *ctx);

/* Build a plan for one cell (Sec. III B-C): cell metric (Eqs. jacb, lapG_), NK
 * stencil (Eqs. nk2d_aux .. lapG_mod_nk3d, Algorithm 1) and its definiteness
 * check, proto-subdomain offset sets PE and shell for self and non-self pairs
 * (Eqs. rbar, g0), the halo check, and device workspace for up to max_orb
 * orbitals of extent box[].  It also sizes the context's workspace for the
 * plan -- the pair list (for all live plans of the context together, so that
 * they can be solved as one batch), the per-cell constants and the persistent
 * solver slots -- and, for the mixed path with EXX_PRECOND_MG, builds the
 * multigrid hierarchy on the host.  A solve with device-memory buffers then
 * allocates nothing, with three exceptions: the first call with EXX_MEM_HOST
 * buffers allocates the plan's device staging copies; warm_start grows the
 * plan's solution stores when the pair count exceeds them; and a frozen-mode
 * cell whose auxiliary directions change rebuilds the layouts and hierarchy.
 * Returns EXX_ERR_CELL, EXX_ERR_NK, EXX_ERR_HALO, EXX_ERR_ARG or EXX_ERR_OOM
 * on failure (and *plan = NULL). */
int exx_plan_create(exx_ctx *ctx, const exx_cell *cell, const exx_params *params,
                    int max_orb, const int box[3], exx_plan **plan);
void exx_plan_destroy(exx_plan *plan);
int exx_plan_query(const exx_plan *plan, exx_plan_info *info);

/* Evaluate E_xx, D_xx and sigma_xx / Pi_xx for one cell (Steps II-V).
 * `cell` may differ from the plan's cell: with params.frozen = 1 the plan's
 * offsets and aux directions are kept and every metric quantity follows the
 * new cell (Sec. III B 2); otherwise the plan is rebuilt for it.  On
 * EXX_ERR_CG_NOT_CONVERGED the other outputs are still written. */
int exx_pairs_solve(exx_ctx *ctx, exx_plan *plan, const exx_cell *cell, const exx_orbitals *orb,
                    exx_result *res, void *stream);

/* Evaluate n_cells independent cells in one persistent launch: the pairs of
 * all cells share one work queue ordered by estimated cost.  plans[c],
 * cells[c], orbs[c], res[c] describe cell c; the plans must come from the
 * same context and use the same precision.  Returns the first non-OK status
 * over the cells. */
int exx_pairs_solve_batch(exx_ctx *ctx, int n_cells, exx_plan *const *plans, const exx_cell *cells,
                          const exx_orbitals *orbs, exx_result *res, void *stream);

/* Pair sharding over ranks (one process per GPU).  The paper distributes the
 * unique pairs over MPI processes and sums E_xx and sigma_xx over them, each
 * process returning its D_ji contributions to the owner of orbital j (Sec.
 * III A, Steps II and V).  After exx_plan_set_shard(plan, rank, n_ranks) the
 * plan's solves still build the whole pair list, but solve only the pairs
 * that exx_pair_partition assigns to `rank`; E_xx, dedh, stress, p_int and
 * D_xx (every orbital's box) are then this rank's partial sums, whose sums
 * over the ranks are the single-rank results (an all-reduce of 20 doubles and
 * of the D boxes).  Per-pair outputs of other ranks' pairs are zero.  Every
 * rank must use the same cell, orbitals and parameters.  n_ranks = 1 (the
 * default) solves every pair.  Errors: EXX_ERR_ARG unless 0 <= rank < n_ranks. */
int exx_plan_set_shard(exx_plan *plan, int rank, int n_ranks);

/* The partition behind exx_plan_set_shard, host only (needs no GPU): the
 * longest-processing-time rule over the pairs' estimated costs, the size N_PE
 * of the pair's Poisson subdomain (self pairs R_PE^self, others R_PE^pair, at
 * this cell): pairs by decreasing cost, stable, each to the least-loaded rank
 * (the lowest on ties).  rows: host [n_pairs][8] pair rows as exx_get_pair_list
 * returns them (only i and j are read); owner: host [n_pairs] output.
 * Errors: EXX_ERR_ARG, and the geometry errors of exx_geometry_query. */
int exx_pair_partition(const exx_cell *cell, const exx_params *params, int n_pairs, const int *rows, int n_ranks,
                       int *owner);

/* The plan's solver schedule (exx_schedule), and setting it by hand.
 * set: EXX_ERR_ARG for a value out of range, or EXX_PRECOND_MG on a plan
 * without a multigrid hierarchy (FP64 path, fd_order > 3, tiny subdomains). */
int exx_plan_get_schedule(const exx_plan *plan, exx_schedule *sched);
int exx_plan_set_schedule(exx_plan *plan, const exx_schedule *sched);

/* Autotuner of the solver schedule (the paper has no counterpart; its CG is
 * one fixed plain schedule).  Runs the plan's pair solver on the first
 * `sample_pairs` pairs of this cell (the whole path up to Step IV, no D_xx)
 * once for every candidate schedule -- the multigrid preconditioner with
 * omega in {0.8, 0.7, 0.6}, and plain CG, each with inner_shift in {14, 18} --
 * timing the solver launch with CUDA events on `stream`, twice per candidate
 * (the faster run counts), and keeps the fastest for the plan's later solves
 * (ties keep the earlier candidate, the order above).  `chosen` (may be NULL)
 * receives it with its time.  The FP64 path has one schedule (plain FP64 CG)
 * and returns it untimed.  A sample of several waves of the persistent grid
 * (a few times `ctas` of exx_plan_query) gives stable choices: with one wave
 * the slowest single pair decides each time.  cell and orb as for
 * exx_pairs_solve (device or host memory).  Errors: those of exx_pairs_solve,
 * EXX_ERR_ARG for sample_pairs < 1. */
int exx_plan_autotune(exx_ctx *ctx, exx_plan *plan, const exx_cell *cell, const exx_orbitals *orb, int sample_pairs,
                      exx_schedule *chosen, void *stream);

/* Copy the unique pair list of the plan's last solve to host memory: rows of
 * (i, j, k0, k1, k2, g0, g1, g2) with i <= j in lexicographic order, k the
 * lattice image of j nearest to i and g the grid-resolved pair centre
 * (Sec. III A Step II, Eq. l2g).  *n receives the pair count; fails with
 * EXX_ERR_CAPACITY if it exceeds cap. */
int exx_get_pair_list(exx_plan *plan, int cap, int *n, int *rows);

/* The unique pair list of one cell (the same rows, bit for bit, as
 * exx_get_pair_list after a solve) for callers that cannot allocate device
 * memory when they need it -- for instance code that runs while a CUDA graph
 * is captured under a fixed memory budget, or inside an engine whose device
 * memory is handed out once by its own pool.  The paper has no counterpart:
 * this is a deployment convenience.
 *   cell:     host struct; centres: device [n_orb][3]; r_pair: cutoff (bohr)
 *   rows:     device [cap][8] output rows (i, j, k0, k1, k2, g0, g1, g2);
 *             rows past cap are not written
 *   n_pairs:  device int, receives the total number of pairs (may exceed cap)
 * The call allocates nothing: its scratch (row counts and offsets) is a
 * static device array sized for n_orb <= 16384 (128 KB), held by every GPU
 * that loads the library until the process exits; larger n_orb returns
 * EXX_ERR_CAPACITY.  The first call on a device resolves that array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture.
 * The address is resolved again when the current context changes (for
 * instance after cudaDeviceReset).  Every call shares the array, so calls
 * that overlap on the GPU (on different streams, or from different threads)
 * race.  A CUDA error left pending by the caller's earlier work is returned
 * as EXX_ERR_CUDA and left pending (not cleared).  The work is enqueued on
 * `stream` and the call returns without waiting for it. */
int exx_pair_list_noalloc(const exx_cell *cell, const double *centres, int n_orb, double r_pair, int cap,
                          int *rows, int *n_pairs, void *stream);

/* The geometry that a plan for this cell and these parameters would have,
 * computed on the host with no device work or allocation (for example to size
 * buffers before exx_plan_create): the proto-subdomain point counts and dense
 * CG boxes of self and non-self pairs (Sec. III B), and the NK stencil of the
 * cell (Sec. III C, Algorithm 1).  Fills n_pe_*, n_me_*, n_halo_*, box_*,
 * n_aux, n_stcl, dirs, coef and aux_frozen (the auxiliary directions chosen
 * for this cell) as exx_plan_query does for a plan created at this cell; the
 * solver fields (workspace_bytes, pair_capacity, ctas, threads, cluster) are
 * zero.  Errors: EXX_ERR_ARG (null pointer or invalid parameters),
 * EXX_ERR_CELL, EXX_ERR_NK, EXX_ERR_HALO, as exx_plan_create. */
int exx_geometry_query(const exx_cell *cell, const exx_params *params, exx_plan_info *info);

/* Index half-widths of a D box that holds every contribution of the pairs of
 * an orbital: ceil((R_pair / 2 + R_ME) n |row alpha of h^-1|) + 1. */
int exx_dbox_halfwidth(const exx_cell *cell, const exx_params *params, int halfwidth[3]);

/* D-box layout of a cell (the boxes D_xx^i is written on, Step V): the extent
 * and, per orbital, the first grid index of a box centred on the grid point
 * nearest the orbital's centre, g_c = floor(N frac(h^-1 C) + 1/2), first index
 * g_c - dbox / 2 (it wraps mod n like every box).
 *   dbox:    in/out.  dbox[0] <= 0 on entry: receives the smallest extent that
 *            holds every contribution of the orbital's pairs,
 *            min(2 halfwidth + 1, n) with the half-widths of
 *            exx_dbox_halfwidth; otherwise the given extent is used (for
 *            instance one D buffer shared by the steps of a trajectory) and
 *            must lie between that minimum and n, else EXX_ERR_ARG.
 *   centres: host [n_orb][3] Cartesian centres (bohr), caller-owned.
 *   dbox_lo: host [n_orb][3] output, caller-owned.
 * Host arithmetic only: needs no GPU.  Errors: EXX_ERR_ARG, EXX_ERR_CELL. */
int exx_dbox_layout(const exx_cell *cell, const exx_params *params, int n_orb, const double *centres, int dbox[3],
                    int *dbox_lo);

/* Strain of a cell relative to a reference cell (both lattice[alpha][a], rows
 * are lattice vectors, 9 doubles each; caller-owned host memory), the
 * criterion for re-assembling frozen proto-subdomains: with subdomains of a
 * fixed number of points that deform with the cell (Sec. III B 2), strong
 * anisotropic strain calls for re-assembling quasi-spherical ones from scratch,
 * by a strain criterion or a step stride (done by creating a new plan whose
 * reference cell is the current one).  F = h h0^-1 with h = lattice^T,
 * E = (F^T F - I) / 2 (Green-Lagrange strain, invariant under rotations of
 * the cell).  out[0] = the largest |eigenvalue| of E, out[1] = det F - 1 (the
 * relative volume change).  Host arithmetic only: needs no GPU.  Errors:
 * EXX_ERR_ARG for a null pointer, EXX_ERR_CELL for a cell that is singular or
 * not right-handed. */
int exx_cell_strain(const double *lattice0, const double *lattice, double out[2]);

/* Choose the persistent pair solver of the mixed-precision path (Step IV).
 * EXX_SOLVER_CTA (default): one CTA of 1024 threads per pair, CG vectors in
 * HBM as dense boxes.  EXX_SOLVER_CLUSTER: one thread-block cluster of 16 CTAs
 * per pair with the pair's FP32 CG state (r, q, e and the rows of p) in the
 * cluster's distributed shared memory; it is used for a solve only when every
 * subdomain of every cell fits (about 200 KB per CTA: R_PE = 6 bohr at
 * 0.2 bohr spacing fits, R_PE = 7 does not) and otherwise the CTA solver runs.
 * Both give the same results to the CG tolerance.  The FP64 path always uses
 * the CTA solver.  Returns EXX_ERR_ARG for an unknown solver. */
int exx_ctx_set_solver(exx_ctx *ctx, int solver);

/* Stage timing of the context's last solve, measured with CUDA events
 * recorded on the solve's stream while enabled: ms[0] solid-harmonic tables
 * (only when the cell changed), ms[1] pair list, ms[2] persistent pair
 * solver, ms[3] per-cell reductions.  Disabled by default. */
int exx_ctx_set_timing(exx_ctx *ctx, int enable);
int exx_ctx_get_timing(const exx_ctx *ctx, double ms[4]);

const char *exx_error_string(int code);

/* The CUDA call and error behind the calling thread's last EXX_ERR_CUDA
 * ("" if none); valid until the next failing call on this thread. */
const char *exx_last_error_detail(void);

/* Library version string. */
const char *exx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EXX_H */
