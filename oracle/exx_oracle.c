/*
 * exx_oracle.c -- plain FP64 CPU oracle of the exact-exchange pair path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this library.  It shares no code
 * with the CUDA path: no headers, helpers, tables or generators.
 *
 * It follows the method of Ko, Santra & DiStasio, "Enabling large-scale
 * condensed-phase hybrid DFT based AIMD II: extensions to the NpH/NpT
 * ensembles" (arXiv 2011.07209), step by step, with no blocking, fusion or
 * reordering:
 *   - cell tensor, Jacobian J and metric F = J^T J           (Sec. III C, Eqs. jacb, lapG_)
 *   - Natan-Kronik Laplacian with auxiliary directions         (Eqs. nk3d_mu .. lapG_mod_nk3d,
 *     chosen by the 2D bisector rule or by Algorithm 1           Eqs. nk2d_aux, kappa_def, Alg. 1)
 *   - central-difference weights                               (Eqs. d2_1, d1_1)
 *   - proto-subdomains as integer offset sets                  (Eqs. rbar, g0, l2g)
 *   - unique pair list with |C_i - C_j| <= R_pair               (Sec. III A, Step II)
 *   - pair density, multipoles, far field                      (Eqs. rho_from_phi_mlwf, me, mepole)
 *   - conjugate-gradient Poisson solve                         (Eq. pe, Step IV)
 *   - E_xx, D_xx and sigma_xx / Pi_xx                          (Eqs. exxGen_mlwf, Dxx,
 *                                                                sxx_working, pixx_working)
 *
 * Every floating-point value is double precision.  Where the paper leaves a
 * point open, the reading taken is stated at the code that implements it.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared -o liboracle.so exx_oracle.c -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_CELL 2
#define ORC_ERR_HALO 3
#define ORC_ERR_NK 4
#define ORC_ERR_CG 5
#define ORC_ERR_CAP 6
#define ORC_ERR_BOX 7
#define ORC_ERR_MEM 8

#define MAXN 8          /* largest supported stencil half-width n */
#define MAXL 6          /* largest multipole order */
#define NLM ((MAXL + 1) * (MAXL + 1))

/* ------------------------------------------------------------------ */
/* Parameters (mirrored by a ctypes.Structure in oracle/__init__.py)    */
/* ------------------------------------------------------------------ */
typedef struct {
    double r_pair, r_pe_self, r_pe_pair, r_me_self, r_me_pair;
    double cg_tol;
    int fd_n, lmax, cg_max_iter, nq, n_threads;
    int frozen;             /* 1: offsets come from lattice0 (Sec. III B 2) and the aux directions are
                               chosen for the current cell, as Algorithm 1 runs at every MD step
                               (Sec. III C); 2: the aux directions of lattice0 are kept as well */
    double lattice0[9];     /* rows = lattice vectors of the reference cell */
} orc_params;

/* ------------------------------------------------------------------ */
/* Central-difference weights (Eqs. d2_1 and d1_1).                    */
/* The paper prints n = 3; general n uses the closed form of the        */
/* (2n+1)-point central formulas (Fornberg), w[q] for q = 0..n.         */
/* ------------------------------------------------------------------ */
static double fact(int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; }

int orc_fd2_weights(int n, double *w)
{
    if (n < 1 || n > MAXN) return ORC_ERR_ARG;
    double nf2 = fact(n) * fact(n);
    double w0 = 0.0;
    for (int q = 1; q <= n; ++q) {
        double sgn = (q % 2 == 1) ? 1.0 : -1.0;
        w[q] = 2.0 * sgn * nf2 / ((double)q * q * fact(n - q) * fact(n + q));
        w0 -= 2.0 / ((double)q * q);
    }
    w[0] = w0;
    return ORC_OK;
}

int orc_fd1_weights(int n, double *w)
{
    if (n < 1 || n > MAXN) return ORC_ERR_ARG;
    double nf2 = fact(n) * fact(n);
    w[0] = 0.0;
    for (int q = 1; q <= n; ++q) {
        double sgn = (q % 2 == 1) ? 1.0 : -1.0;
        w[q] = sgn * nf2 / ((double)q * fact(n - q) * fact(n + q));
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Cell metric (Sec. II B 1 and Eqs. s_to_xi, jacb, lapG_).            */
/* h[a][alpha] = (L_alpha)_a, i.e. the lattice rows transposed.         */
/* ------------------------------------------------------------------ */
typedef struct {
    double h[3][3], hinv[3][3];
    double vol, dv;
    int n[3];
    double len[3], dxi[3];
    double J[3][3], F[3][3];
} orc_cell;

/* h^{-1} by the adjugate: this exact operation order is shared (as a
 * written rule, not as code) with the CUDA path so that the pair list,
 * which turns these doubles into integers, agrees bit for bit. */
static int cell_init(orc_cell *c, const double *lattice, const int *n)
{
    for (int a = 0; a < 3; ++a)
        for (int al = 0; al < 3; ++al) c->h[a][al] = lattice[al * 3 + a];
    const double (*h)[3] = (const double (*)[3])c->h;
    double det = h[0][0] * (h[1][1] * h[2][2] - h[1][2] * h[2][1])
               - h[0][1] * (h[1][0] * h[2][2] - h[1][2] * h[2][0])
               + h[0][2] * (h[1][0] * h[2][1] - h[1][1] * h[2][0]);
    if (!(det > 0.0)) return ORC_ERR_CELL;
    c->hinv[0][0] = (h[1][1] * h[2][2] - h[1][2] * h[2][1]) / det;
    c->hinv[0][1] = (h[0][2] * h[2][1] - h[0][1] * h[2][2]) / det;
    c->hinv[0][2] = (h[0][1] * h[1][2] - h[0][2] * h[1][1]) / det;
    c->hinv[1][0] = (h[1][2] * h[2][0] - h[1][0] * h[2][2]) / det;
    c->hinv[1][1] = (h[0][0] * h[2][2] - h[0][2] * h[2][0]) / det;
    c->hinv[1][2] = (h[0][2] * h[1][0] - h[0][0] * h[1][2]) / det;
    c->hinv[2][0] = (h[1][0] * h[2][1] - h[1][1] * h[2][0]) / det;
    c->hinv[2][1] = (h[0][1] * h[2][0] - h[0][0] * h[2][1]) / det;
    c->hinv[2][2] = (h[0][0] * h[1][1] - h[0][1] * h[1][0]) / det;
    c->vol = det;
    for (int al = 0; al < 3; ++al) {
        if (n[al] < 1) return ORC_ERR_ARG;
        c->n[al] = n[al];
        c->len[al] = sqrt(h[0][al] * h[0][al] + h[1][al] * h[1][al] + h[2][al] * h[2][al]);
        c->dxi[al] = c->len[al] / n[al];
    }
    c->dv = det / ((double)n[0] * n[1] * n[2]);
    /* J_{a alpha} = |L_alpha| (h^{-1})_{alpha a}  (Eq. jacb) */
    for (int a = 0; a < 3; ++a)
        for (int al = 0; al < 3; ++al) c->J[a][al] = c->len[al] * c->hinv[al][a];
    /* F = J^T J  (Eq. lapG_) */
    for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += c->J[a][al] * c->J[a][be];
            c->F[al][be] = s;
        }
    return ORC_OK;
}

int orc_metric(const double *lattice, const int *n, double *h, double *hinv, double *vol,
               double *dxi, double *J, double *F)
{
    orc_cell c;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            h[a * 3 + b] = c.h[a][b];
            hinv[a * 3 + b] = c.hinv[a][b];
            J[a * 3 + b] = c.J[a][b];
            F[a * 3 + b] = c.F[a][b];
        }
    *vol = c.vol;
    for (int a = 0; a < 3; ++a) dxi[a] = c.dxi[a];
    return ORC_OK;
}

/* Cartesian vector of the integer grid offset m: h (m / N). */
static void offset_xyz(const orc_cell *c, const int *m, double *r)
{
    double s0 = (double)m[0] / (double)c->n[0];
    double s1 = (double)m[1] / (double)c->n[1];
    double s2 = (double)m[2] / (double)c->n[2];
    for (int a = 0; a < 3; ++a) r[a] = c->h[a][0] * s0 + c->h[a][1] * s1 + c->h[a][2] * s2;
}

static double offset_len(const orc_cell *c, const int *m)
{
    double r[3];
    offset_xyz(c, m, r);
    return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
}

/* ------------------------------------------------------------------ */
/* Natan-Kronik stencil (Sec. III C 1-2).                              */
/* L f(g) = sum_dir coef[dir] * sum_{q=-n..n} w_q f(g + q d[dir])        */
/* ------------------------------------------------------------------ */
typedef struct {
    int ndir, n_aux, n_off;
    int d[6][3];
    double coef[6];
    double a[3][3];      /* a_{p alpha} of the aux directions */
    double b[3];
} orc_stencil;

/* Candidate non-axial grid directions, sorted by grid spacing (the list v-hat
 * that Algorithm 1 takes as input).  Shells G_S = {max_alpha |m_alpha| = S} are
 * swept for S = 1, 2, ...; delta_> is the longest spacing in G_1; the sweep
 * stops after the first shell S >= 2 whose every point is longer than delta_>.
 * Only one of m and -m is kept (first non-zero component positive).  Ties in
 * length are ordered lexicographically by m. */
typedef struct { int m[3]; double len; } cand_t;

static int cand_cmp(const void *x, const void *y)
{
    const cand_t *p = (const cand_t *)x, *q = (const cand_t *)y;
    if (p->len < q->len) return -1;
    if (p->len > q->len) return 1;
    for (int k = 0; k < 3; ++k) {
        if (p->m[k] < q->m[k]) return -1;
        if (p->m[k] > q->m[k]) return 1;
    }
    return 0;
}

static int build_candidates(const orc_cell *c, int nq, cand_t *out, int *count)
{
    const int SMAX = 8;
    int cap = (2 * SMAX + 1) * (2 * SMAX + 1) * (2 * SMAX + 1);
    cand_t *all = (cand_t *)malloc(sizeof(cand_t) * cap);
    if (!all) return ORC_ERR_MEM;
    int na = 0;
    double dmax1 = 0.0;
    for (int S = 1; S <= SMAX; ++S) {
        double shell_min = INFINITY;
        for (int i = -S; i <= S; ++i)
            for (int j = -S; j <= S; ++j)
                for (int k = -S; k <= S; ++k) {
                    int ai = abs(i), aj = abs(j), ak = abs(k);
                    int mx = ai > aj ? ai : aj;
                    mx = mx > ak ? mx : ak;
                    if (mx != S) continue;
                    int m[3] = {i, j, k};
                    double l = offset_len(c, m);
                    if (S == 1 && l > dmax1) dmax1 = l;
                    if (l < shell_min) shell_min = l;
                    int nz = (i != 0) + (j != 0) + (k != 0);
                    if (nz < 2) continue;                     /* axial */
                    int first = (i != 0) ? i : ((j != 0) ? j : k);
                    if (first < 0) continue;                  /* keep one of +-m */
                    all[na].m[0] = i; all[na].m[1] = j; all[na].m[2] = k;
                    all[na].len = l;
                    ++na;
                }
        if (S >= 2 && shell_min > dmax1) break;
    }
    qsort(all, na, sizeof(cand_t), cand_cmp);
    int nout = na < nq ? na : nq;
    memcpy(out, all, sizeof(cand_t) * nout);
    *count = nout;
    free(all);
    return ORC_OK;
}

int orc_nk_candidates(const double *lattice, const int *n, int nq, int *m_out, double *len_out, int *count)
{
    orc_cell c;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    cand_t *buf = (cand_t *)malloc(sizeof(cand_t) * (nq > 0 ? nq : 1));
    e = build_candidates(&c, nq, buf, count);
    if (!e)
        for (int q = 0; q < *count; ++q) {
            for (int k = 0; k < 3; ++k) m_out[q * 3 + k] = buf[q].m[k];
            len_out[q] = buf[q].len;
        }
    free(buf);
    return e;
}

static void aux_coeffs(const orc_cell *c, const int *m, double *a, double *len)
{
    /* unit aux direction L'_p = sum_alpha a_{p alpha} L^_alpha, with the grid step
     * sum_alpha m_alpha (L_alpha / N_alpha) = sum_alpha m_alpha dxi_alpha L^_alpha */
    double l = offset_len(c, m);
    for (int al = 0; al < 3; ++al) a[al] = (double)m[al] * c->dxi[al] / l;
    *len = l;
}

static void m_column(const double *a, double *col)
{
    col[0] = a[0] * a[1];
    col[1] = a[0] * a[2];
    col[2] = a[1] * a[2];
}

static double det3(const double M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
         - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
         + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* Algorithm 1: walk the candidate list, accept the first candidate as L'_1,
 * the next one whose M column is not parallel to column 1 as L'_2 (strict
 * Cauchy-Schwarz inequality), and the next one that makes M non-singular as
 * L'_3. */
static int algorithm1(const orc_cell *c, const cand_t *cand, int ncand, int chosen[3][3])
{
    double M[3][3] = {{0}};
    int p = 0;
    for (int q = 0; q < ncand && p < 3; ++q) {
        double a[3], l, col[3];
        aux_coeffs(c, cand[q].m, a, &l);
        m_column(a, col);
        for (int r = 0; r < 3; ++r) M[r][p] = col[r];
        int accept = 0;
        if (p == 0) {
            accept = 1;
        } else if (p == 1) {
            double d01 = 0, n0 = 0, n1 = 0;
            for (int r = 0; r < 3; ++r) { d01 += M[r][0] * M[r][1]; n0 += M[r][0] * M[r][0]; n1 += M[r][1] * M[r][1]; }
            accept = fabs(d01) < (1.0 - 1e-8) * sqrt(n0 * n1);
        } else {
            double nrm = 1.0;
            for (int s = 0; s < 3; ++s) nrm *= sqrt(M[0][s] * M[0][s] + M[1][s] * M[1][s] + M[2][s] * M[2][s]);
            accept = fabs(det3(M)) > 1e-10 * nrm;
        }
        if (accept) {
            for (int k = 0; k < 3; ++k) chosen[p][k] = cand[q].m[k];
            ++p;
        }
    }
    return p == 3 ? ORC_OK : ORC_ERR_NK;
}

/* Solve the 3x3 system M b = f by Cramer's rule. */
static int solve3(const double M[3][3], const double *f, double *b)
{
    double d = det3(M);
    if (d == 0.0) return ORC_ERR_NK;
    for (int k = 0; k < 3; ++k) {
        double T[3][3];
        memcpy(T, M, sizeof(T));
        for (int r = 0; r < 3; ++r) T[r][k] = f[r];
        b[k] = det3(T) / d;
    }
    return ORC_OK;
}

/* Symbol of the 1D second-difference operator: w0 + 2 sum_q w_q cos(q t). */
static double symbol1(const double *w, int n, double t)
{
    double s = w[0];
    for (int q = 1; q <= n; ++q) s += 2.0 * w[q] * cos(q * t);
    return s;
}

/* Negative-definiteness check of the discrete operator: its symbol must be
 * strictly negative at every non-zero wave vector of a 32^3 grid. */
static int symbol_negative(const orc_stencil *st, int n)
{
    double w[MAXN + 1];
    orc_fd2_weights(n, w);
    const int G = 32;
    for (int i = 0; i < G; ++i)
        for (int j = 0; j < G; ++j)
            for (int k = 0; k < G; ++k) {
                if (i == 0 && j == 0 && k == 0) continue;
                double t[3] = {2.0 * M_PI * i / G, 2.0 * M_PI * j / G, 2.0 * M_PI * k / G};
                double s = 0.0;
                for (int d = 0; d < st->ndir; ++d) {
                    double ph = t[0] * st->d[d][0] + t[1] * st->d[d][1] + t[2] * st->d[d][2];
                    s += st->coef[d] * symbol1(w, n, ph);
                }
                if (!(s < 0.0)) return 0;
            }
    return 1;
}

/* Build the NK stencil for cell c.  aux_fixed (n_aux_fixed rows) replaces the
 * direction choice when the caller freezes it; otherwise:
 *   N_off = 0 -> no aux direction (orthorhombic);
 *   N_off = 1 -> the grid-resolved bisector m = e_alpha - sgn(L^_alpha . L^_beta) e_beta
 *                of Eqs. nk2d_aux / kappa_def;
 *   N_off >= 2 -> three directions from Algorithm 1.
 * Then b solves sum_p b_p a_{p alpha} a_{p beta} = F_{alpha beta} (Eq. nk3d_Mb_f) and
 * the pure coefficients are c_alpha = F_{alpha alpha} - sum_p b_p a_{p alpha}^2
 * (Eq. lapG_mod_nk3d). */
static int build_stencil(const orc_cell *c, int n, int nq, const int (*aux_fixed)[3], int n_aux_fixed,
                         orc_stencil *st)
{
    memset(st, 0, sizeof(*st));
    double fdiag = fmax(c->F[0][0], fmax(c->F[1][1], c->F[2][2]));
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    int off_idx = -1;
    for (int k = 0; k < 3; ++k)
        if (fabs(c->F[pa[k]][pb[k]]) > 1e-12 * fdiag) { st->n_off++; off_idx = k; }

    int aux[3][3];
    int n_aux = 0;
    if (aux_fixed) {
        n_aux = n_aux_fixed;
        for (int p = 0; p < n_aux; ++p)
            for (int k = 0; k < 3; ++k) aux[p][k] = aux_fixed[p][k];
    } else if (st->n_off == 1) {
        int al = pa[off_idx], be = pb[off_idx];
        double cosab = 0.0;
        for (int a = 0; a < 3; ++a) cosab += c->h[a][al] * c->h[a][be];
        int sg = cosab > 0.0 ? 1 : -1;
        aux[0][0] = aux[0][1] = aux[0][2] = 0;
        aux[0][al] = 1;
        aux[0][be] = -sg;
        n_aux = 1;
    } else if (st->n_off >= 2) {
        cand_t cand[64];
        int nc = 0;
        int e = build_candidates(c, nq > 64 ? 64 : nq, cand, &nc);
        if (e) return e;
        e = algorithm1(c, cand, nc, aux);
        if (e) return e;
        n_aux = 3;
    }

    double a[3][3] = {{0}}, len[3] = {0};
    for (int p = 0; p < n_aux; ++p) aux_coeffs(c, aux[p], a[p], &len[p]);
    double b[3] = {0, 0, 0};
    if (n_aux == 1) {
        /* one aux direction: only the single non-zero F_{alpha beta} is matched */
        int al = -1, be = -1;
        for (int k = 0; k < 3; ++k)
            if (aux[0][pa[k]] != 0 && aux[0][pb[k]] != 0) { al = pa[k]; be = pb[k]; }
        if (al < 0) return ORC_ERR_NK;
        double prod = a[0][al] * a[0][be];
        if (prod == 0.0) return ORC_ERR_NK;
        b[0] = c->F[al][be] / prod;
        /* every other off-diagonal element must vanish for this choice */
        for (int k = 0; k < 3; ++k) {
            if (pa[k] == al && pb[k] == be) continue;
            if (fabs(c->F[pa[k]][pb[k]] - b[0] * a[0][pa[k]] * a[0][pb[k]]) > 1e-12 * fdiag) return ORC_ERR_NK;
        }
    } else if (n_aux == 3) {
        double M[3][3], f[3];
        for (int p = 0; p < 3; ++p) {
            double col[3];
            m_column(a[p], col);
            for (int r = 0; r < 3; ++r) M[r][p] = col[r];
        }
        f[0] = c->F[0][1]; f[1] = c->F[0][2]; f[2] = c->F[1][2];
        int e = solve3(M, f, b);
        if (e) return e;
    } else if (n_aux != 0) {
        return ORC_ERR_NK;
    }
    if (n_aux == 0 && st->n_off != 0) return ORC_ERR_NK;

    st->n_aux = n_aux;
    st->ndir = 3 + n_aux;
    for (int al = 0; al < 3; ++al) {
        double cal = c->F[al][al];
        for (int p = 0; p < n_aux; ++p) cal -= b[p] * a[p][al] * a[p][al];
        st->d[al][0] = st->d[al][1] = st->d[al][2] = 0;
        st->d[al][al] = 1;
        st->coef[al] = cal / (c->dxi[al] * c->dxi[al]);
    }
    for (int p = 0; p < n_aux; ++p) {
        for (int k = 0; k < 3; ++k) {
            st->d[3 + p][k] = aux[p][k];
            st->a[p][k] = a[p][k];
        }
        st->b[p] = b[p];
        st->coef[3 + p] = b[p] / (len[p] * len[p]);
    }
    if (!symbol_negative(st, n)) return ORC_ERR_NK;
    return ORC_OK;
}

static int stencil_for(const orc_cell *cell, const orc_params *P, const orc_cell *cell0, orc_stencil *st)
{
    if (P->frozen != 2) return build_stencil(cell, P->fd_n, P->nq, NULL, 0, st);
    /* aux directions frozen too: directions from the reference cell, coefficients from the current one */
    orc_stencil st0;
    int e = build_stencil(cell0, P->fd_n, P->nq, NULL, 0, &st0);
    if (e) return e;
    int aux[3][3];
    for (int p = 0; p < st0.n_aux; ++p)
        for (int k = 0; k < 3; ++k) aux[p][k] = st0.d[3 + p][k];
    return build_stencil(cell, P->fd_n, P->nq, (const int (*)[3])aux, st0.n_aux, st);
}

int orc_stencil_info(const double *lattice, const int *n, int fd_n, int nq, const int *aux_in, int n_aux_in,
                     int *ndir, int *dirs, double *coef, int *n_aux, int *n_off, double *b)
{
    orc_cell c;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    orc_stencil st;
    e = build_stencil(&c, fd_n, nq, aux_in ? (const int (*)[3])aux_in : NULL, n_aux_in, &st);
    *n_off = st.n_off;
    if (e) return e;
    *ndir = st.ndir;
    *n_aux = st.n_aux;
    for (int d = 0; d < st.ndir; ++d) {
        coef[d] = st.coef[d];
        for (int k = 0; k < 3; ++k) dirs[d * 3 + k] = st.d[d][k];
    }
    for (int p = 0; p < 3; ++p) b[p] = st.b[p];
    return ORC_OK;
}

/* Apply L to a field sampled on a dense box (C order, dims bx).  Points whose
 * stencil leaves the box get NaN. */
int orc_apply_lap(const double *lattice, const int *n, int fd_n, int nq, const int *bx, const double *f, double *out)
{
    orc_cell c;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    orc_stencil st;
    e = build_stencil(&c, fd_n, nq, NULL, 0, &st);
    if (e) return e;
    double w[MAXN + 1];
    orc_fd2_weights(fd_n, w);
    for (int i = 0; i < bx[0]; ++i)
        for (int j = 0; j < bx[1]; ++j)
            for (int k = 0; k < bx[2]; ++k) {
                double s = 0.0;
                int ok = 1;
                for (int d = 0; d < st.ndir && ok; ++d)
                    for (int q = -fd_n; q <= fd_n; ++q) {
                        int ii = i + q * st.d[d][0], jj = j + q * st.d[d][1], kk = k + q * st.d[d][2];
                        if (ii < 0 || jj < 0 || kk < 0 || ii >= bx[0] || jj >= bx[1] || kk >= bx[2]) { ok = 0; break; }
                        s += st.coef[d] * w[abs(q)] * f[((size_t)ii * bx[1] + jj) * bx[2] + kk];
                    }
                out[((size_t)i * bx[1] + j) * bx[2] + k] = ok ? s : NAN;
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Real solid harmonics r^l Y_lm, orthonormal real Y_lm, l <= MAXL.      */
/* Index l*l + l + m, m = -l..l.  Y_lm = N_lm P_l^|m|(cos t) * {cos m p,  */
/* sin |m| p}, with the sqrt(2) for m != 0 and no Condon-Shortley phase. */
/* ------------------------------------------------------------------ */
static void solid_harmonics(int lmax, const double *r, double *out)
{
    double x = r[0], y = r[1], z = r[2];
    double rr = sqrt(x * x + y * y + z * z);
    int nlm = (lmax + 1) * (lmax + 1);
    if (rr == 0.0) {
        for (int k = 0; k < nlm; ++k) out[k] = 0.0;
        out[0] = sqrt(1.0 / (4.0 * M_PI));
        return;
    }
    double ct = z / rr;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double phi = atan2(y, x);
    double P[MAXL + 1][MAXL + 1];
    for (int m = 0; m <= lmax; ++m) {
        /* P_m^m = (2m-1)!! sin^m t */
        double pmm = 1.0;
        for (int k = 1; k <= m; ++k) pmm *= (2.0 * k - 1.0) * st;
        P[m][m] = pmm;
        if (m + 1 <= lmax) P[m + 1][m] = ct * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= lmax; ++l)
            P[l][m] = ((2.0 * l - 1.0) * ct * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
    }
    for (int l = 0; l <= lmax; ++l) {
        double rl = pow(rr, l);
        for (int m = 0; m <= l; ++m) {
            double nlm_ = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - m) / fact(l + m));
            if (m == 0) {
                out[l * l + l] = rl * nlm_ * P[l][0];
            } else {
                out[l * l + l + m] = rl * sqrt(2.0) * nlm_ * P[l][m] * cos(m * phi);
                out[l * l + l - m] = rl * sqrt(2.0) * nlm_ * P[l][m] * sin(m * phi);
            }
        }
    }
}

int orc_solid_harmonics(int lmax, int npts, const double *xyz, double *out)
{
    if (lmax < 0 || lmax > MAXL) return ORC_ERR_ARG;
    int nlm = (lmax + 1) * (lmax + 1);
    for (int p = 0; p < npts; ++p) solid_harmonics(lmax, xyz + 3 * p, out + (size_t)p * nlm);
    return ORC_OK;
}

/* Multipole moments Q_lm = sum_p q_p r_p^l Y_lm(r^_p) (Eq. mepole, with the
 * grid integral written as a sum of charges q_p = rho_p dV). */
static void multipoles(int lmax, int npts, const double *xyz, const double *q, double *Q)
{
    int nlm = (lmax + 1) * (lmax + 1);
    double S[NLM];
    for (int k = 0; k < nlm; ++k) Q[k] = 0.0;
    for (int p = 0; p < npts; ++p) {
        solid_harmonics(lmax, xyz + 3 * p, S);
        for (int k = 0; k < nlm; ++k) Q[k] += q[p] * S[k];
    }
}

/* Far field v(r) = 4 pi sum_lm Q_lm Y_lm(r^) / ((2l+1) r^{l+1})  (Eq. me). */
static double farfield(int lmax, const double *Q, const double *r)
{
    double S[NLM];
    solid_harmonics(lmax, r, S);
    double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double v = 0.0;
    for (int l = 0; l <= lmax; ++l) {
        double f = 4.0 * M_PI / ((2.0 * l + 1.0) * pow(rr, 2 * l + 1));
        for (int m = -l; m <= l; ++m) v += f * Q[l * l + l + m] * S[l * l + l + m];
    }
    return v;
}

int orc_multipoles(int lmax, int npts, const double *xyz, const double *q, double *Q)
{
    if (lmax < 0 || lmax > MAXL) return ORC_ERR_ARG;
    multipoles(lmax, npts, xyz, q, Q);
    return ORC_OK;
}

int orc_farfield(int lmax, const double *Q, int npts, const double *xyz, double *v)
{
    if (lmax < 0 || lmax > MAXL) return ORC_ERR_ARG;
    for (int p = 0; p < npts; ++p) v[p] = farfield(lmax, Q, xyz + 3 * p);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Proto-subdomains as integer offset sets (Eqs. rbar, g0).             */
/* PE = {m : |h(m/N)|^2 <= R_PE^2}, shell = {R_PE^2 < |h(m/N)|^2 <= R_ME^2}, */
/* each in lexicographic order of m, PE points first.                    */
/* ------------------------------------------------------------------ */
typedef struct {
    int n_pe, n_me;      /* n_me counts PE + shell */
    int *m;              /* [n_me][3] */
    int H[3], B[3];      /* bounding half-widths and box dims of the ME set */
    int *kind;           /* [B0*B1*B2]: 0 outside, 1 PE, 2 shell */
    int *box_index;      /* [n_me] index into the dense ME box */
} orc_offsets;

static void offsets_free(orc_offsets *o)
{
    free(o->m); free(o->kind); free(o->box_index);
    memset(o, 0, sizeof(*o));
}

static int build_offsets(const orc_cell *c, double r_pe, double r_me, orc_offsets *o)
{
    memset(o, 0, sizeof(*o));
    if (!(r_pe > 0.0) || !(r_me >= r_pe)) return ORC_ERR_ARG;
    int H[3];
    for (int al = 0; al < 3; ++al) {
        double rn = sqrt(c->hinv[al][0] * c->hinv[al][0] + c->hinv[al][1] * c->hinv[al][1] + c->hinv[al][2] * c->hinv[al][2]);
        H[al] = (int)ceil(r_me * c->n[al] * rn);
    }
    double pe2 = r_pe * r_pe, me2 = r_me * r_me;
    size_t cap = (size_t)(2 * H[0] + 1) * (2 * H[1] + 1) * (2 * H[2] + 1);
    int *pe = (int *)malloc(sizeof(int) * 3 * cap);
    int *sh = (int *)malloc(sizeof(int) * 3 * cap);
    if (!pe || !sh) { free(pe); free(sh); return ORC_ERR_MEM; }
    int npe = 0, nsh = 0;
    int Hm[3] = {0, 0, 0};
    for (int i = -H[0]; i <= H[0]; ++i)
        for (int j = -H[1]; j <= H[1]; ++j)
            for (int k = -H[2]; k <= H[2]; ++k) {
                int m[3] = {i, j, k};
                double r[3];
                offset_xyz(c, m, r);
                double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                if (d2 <= pe2) { memcpy(pe + 3 * npe, m, sizeof(m)); ++npe; }
                else if (d2 <= me2) { memcpy(sh + 3 * nsh, m, sizeof(m)); ++nsh; }
                else continue;
                if (abs(i) > Hm[0]) Hm[0] = abs(i);
                if (abs(j) > Hm[1]) Hm[1] = abs(j);
                if (abs(k) > Hm[2]) Hm[2] = abs(k);
            }
    o->n_pe = npe;
    o->n_me = npe + nsh;
    o->m = (int *)malloc(sizeof(int) * 3 * (size_t)o->n_me);
    memcpy(o->m, pe, sizeof(int) * 3 * (size_t)npe);
    memcpy(o->m + 3 * (size_t)npe, sh, sizeof(int) * 3 * (size_t)nsh);
    free(pe); free(sh);
    for (int al = 0; al < 3; ++al) { o->H[al] = Hm[al]; o->B[al] = 2 * Hm[al] + 1; }
    size_t nb = (size_t)o->B[0] * o->B[1] * o->B[2];
    o->kind = (int *)calloc(nb, sizeof(int));
    o->box_index = (int *)malloc(sizeof(int) * (size_t)o->n_me);
    for (int q = 0; q < o->n_me; ++q) {
        const int *m = o->m + 3 * (size_t)q;
        int idx = ((m[0] + o->H[0]) * o->B[1] + (m[1] + o->H[1])) * o->B[2] + (m[2] + o->H[2]);
        o->box_index[q] = idx;
        o->kind[idx] = (q < npe) ? 1 : 2;
    }
    return ORC_OK;
}

/* Every stencil neighbour (second- and first-derivative) of a PE point must
 * lie in PE or in the shell, so that the far field supplies it. */
static int check_halo(const orc_offsets *o, const orc_stencil *st, int n)
{
    for (int q = 0; q < o->n_pe; ++q) {
        const int *m = o->m + 3 * (size_t)q;
        for (int d = 0; d < st->ndir; ++d)
            for (int s = -n; s <= n; ++s) {
                int p0 = m[0] + s * st->d[d][0], p1 = m[1] + s * st->d[d][1], p2 = m[2] + s * st->d[d][2];
                if (abs(p0) > o->H[0] || abs(p1) > o->H[1] || abs(p2) > o->H[2]) return ORC_ERR_HALO;
                int idx = ((p0 + o->H[0]) * o->B[1] + (p1 + o->H[1])) * o->B[2] + (p2 + o->H[2]);
                if (o->kind[idx] == 0) return ORC_ERR_HALO;
            }
    }
    return ORC_OK;
}

int orc_offsets_count(const double *lattice, const int *n, double r_pe, double r_me, int *n_pe, int *n_me)
{
    orc_cell c;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    orc_offsets o;
    e = build_offsets(&c, r_pe, r_me, &o);
    if (e) return e;
    *n_pe = o.n_pe;
    *n_me = o.n_me;
    offsets_free(&o);
    return ORC_OK;
}

int orc_offsets_list(const double *lattice, const int *n, double r_pe, double r_me, int cap, int *m_out)
{
    orc_cell c;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    orc_offsets o;
    e = build_offsets(&c, r_pe, r_me, &o);
    if (e) return e;
    if (o.n_me > cap) { offsets_free(&o); return ORC_ERR_CAP; }
    memcpy(m_out, o.m, sizeof(int) * 3 * (size_t)o.n_me);
    offsets_free(&o);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Unique pair list (Step II).  For i <= j: s = h^{-1} C, ds = s_j - s_i,   */
/* ds -= round(ds); the image k in {-1,0,1}^3 minimizing |h(ds+k)|^2 (first  */
/* minimum in lexicographic k order); the pair is kept when that squared   */
/* distance is <= R_pair^2.  The grid-resolved midpoint is                 */
/* g_ij = NINT(N (s_i + (ds+k)/2)) mod N with NINT rounding half away      */
/* from zero.                                                              */
/* ------------------------------------------------------------------ */
static void frac_of(const orc_cell *c, const double *r, double *s)
{
    for (int al = 0; al < 3; ++al) s[al] = c->hinv[al][0] * r[0] + c->hinv[al][1] * r[1] + c->hinv[al][2] * r[2];
}

static long imod(long a, long n) { long r = a % n; return r < 0 ? r + n : r; }

int orc_pair_list(const double *lattice, const int *n, int n_orb, const double *centres, double r_pair,
                  int cap, int *n_pairs, int *rows /* [cap][8]: i, j, k0, k1, k2, g0, g1, g2 */)
{
    orc_cell c;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    double rp2 = r_pair * r_pair;
    int np = 0;
    for (int i = 0; i < n_orb; ++i) {
        double si[3];
        frac_of(&c, centres + 3 * i, si);
        for (int j = i; j < n_orb; ++j) {
            double sj[3], ds[3];
            frac_of(&c, centres + 3 * j, sj);
            for (int al = 0; al < 3; ++al) { ds[al] = sj[al] - si[al]; ds[al] = ds[al] - round(ds[al]); }
            double best = INFINITY;
            int kb[3] = {0, 0, 0};
            for (int k0 = -1; k0 <= 1; ++k0)
                for (int k1 = -1; k1 <= 1; ++k1)
                    for (int k2 = -1; k2 <= 1; ++k2) {
                        double t0 = ds[0] + k0, t1 = ds[1] + k1, t2 = ds[2] + k2;
                        double d[3];
                        for (int a = 0; a < 3; ++a) d[a] = c.h[a][0] * t0 + c.h[a][1] * t1 + c.h[a][2] * t2;
                        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (d2 < best) { best = d2; kb[0] = k0; kb[1] = k1; kb[2] = k2; }
                    }
            if (!(best <= rp2)) continue;
            if (np >= cap) return ORC_ERR_CAP;
            int *row = rows + 8 * (size_t)np;
            row[0] = i; row[1] = j;
            for (int al = 0; al < 3; ++al) {
                double sm = si[al] + (ds[al] + kb[al]) * 0.5;
                row[2 + al] = kb[al];
                row[5 + al] = (int)imod((long)round(c.n[al] * sm), c.n[al]);
            }
            ++np;
        }
    }
    *n_pairs = np;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Orbital boxes.                                                       */
/* ------------------------------------------------------------------ */
static double phi_at(const double *phi, const int *box, const int *lo, const int *n, const int *g)
{
    long u[3];
    for (int al = 0; al < 3; ++al) {
        u[al] = imod((long)g[al] - lo[al], n[al]);
        if (u[al] >= box[al]) return 0.0;
    }
    return phi[((size_t)u[0] * box[1] + u[1]) * box[2] + u[2]];
}

/* ------------------------------------------------------------------ */
/* One pair: density, multipoles, far field, CG Poisson solve, E, sigma, D. */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_cell *c;
    const orc_stencil *st;
    const orc_params *P;
    double w2[MAXN + 1], w1[MAXN + 1];
} orc_ctx;

typedef struct {
    double e_pair;          /* integral of rho v over PE */
    double sig[3][3];       /* sum_b hinv_{alpha b} int r_b rho d_a v, [a][alpha] */
    int n_cg;               /* CG iterations (stencil applications in the loop) */
    double resid;           /* final true relative residual */
    int status;
} pair_out;

/* A p = -L applied to p extended by zero outside PE, restricted to PE. */
static void apply_A(const orc_ctx *X, const orc_offsets *o, const double *p, double *box, double *Ap)
{
    int n = X->P->fd_n;
    const orc_stencil *st = X->st;
    int stride[6];
    for (int d = 0; d < st->ndir; ++d)
        stride[d] = (st->d[d][0] * o->B[1] + st->d[d][1]) * o->B[2] + st->d[d][2];
    for (int k = 0; k < o->n_pe; ++k) box[o->box_index[k]] = p[k];
    for (int k = 0; k < o->n_pe; ++k) {
        int idx = o->box_index[k];
        double s = 0.0;
        for (int d = 0; d < st->ndir; ++d) {
            double t = X->w2[0] * box[idx];
            for (int q = 1; q <= n; ++q) t += X->w2[q] * (box[idx + q * stride[d]] + box[idx - q * stride[d]]);
            s += st->coef[d] * t;
        }
        Ap[k] = -s;
    }
}

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* Conjugate gradients on A x = b with x0 = 0.  The loop stops when the
 * recursively updated residual satisfies |r| <= tol |b|; the true residual
 * b - A x is then recomputed and the loop resumes from it if it is not yet
 * below the tolerance. */
static int cg_solve(const orc_ctx *X, const orc_offsets *o, const double *b, double *x, double *box,
                    double *r, double *p, double *q, int *iters, double *resid)
{
    int np = o->n_pe;
    double tol = X->P->cg_tol;
    double bn = sqrt(dot(np, b, b));
    for (int k = 0; k < np; ++k) x[k] = 0.0;
    *iters = 0;
    *resid = 0.0;
    if (bn == 0.0) return ORC_OK;
    for (int k = 0; k < np; ++k) { r[k] = b[k]; p[k] = b[k]; }
    double rr = dot(np, r, r);
    int it = 0;
    for (;;) {
        if (sqrt(rr) <= tol * bn) {
            apply_A(X, o, x, box, q);
            for (int k = 0; k < np; ++k) r[k] = b[k] - q[k];
            rr = dot(np, r, r);
            if (sqrt(rr) <= tol * bn) break;
            for (int k = 0; k < np; ++k) p[k] = r[k];
        }
        if (it >= X->P->cg_max_iter) { *iters = it; *resid = sqrt(rr) / bn; return ORC_ERR_CG; }
        apply_A(X, o, p, box, q);
        double alpha = rr / dot(np, p, q);
        for (int k = 0; k < np; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
        double rr1 = dot(np, r, r);
        double beta = rr1 / rr;
        for (int k = 0; k < np; ++k) p[k] = r[k] + beta * p[k];
        rr = rr1;
        ++it;
    }
    *iters = it;
    *resid = sqrt(rr) / bn;
    return ORC_OK;
}

typedef struct {
    double *fi, *fj, *rho, *v, *b, *x, *r, *p, *q, *box, *xyz;
} pair_work;

static int work_alloc(pair_work *w, const orc_offsets *o)
{
    size_t nme = (size_t)o->n_me, npe = (size_t)o->n_pe;
    size_t nb = (size_t)o->B[0] * o->B[1] * o->B[2];
    w->fi = malloc(sizeof(double) * nme);
    w->fj = malloc(sizeof(double) * nme);
    w->rho = malloc(sizeof(double) * npe);
    w->v = malloc(sizeof(double) * nme);
    w->b = malloc(sizeof(double) * npe);
    w->x = malloc(sizeof(double) * npe);
    w->r = malloc(sizeof(double) * npe);
    w->p = malloc(sizeof(double) * npe);
    w->q = malloc(sizeof(double) * npe);
    w->box = calloc(nb, sizeof(double));
    w->xyz = malloc(sizeof(double) * 3 * nme);
    if (!w->fi || !w->fj || !w->rho || !w->v || !w->b || !w->x || !w->r || !w->p || !w->q || !w->box || !w->xyz)
        return ORC_ERR_MEM;
    return ORC_OK;
}

static void work_free(pair_work *w)
{
    free(w->fi); free(w->fj); free(w->rho); free(w->v); free(w->b); free(w->x);
    free(w->r); free(w->p); free(w->q); free(w->box); free(w->xyz);
}

/* Solve one pair; fills w->v on all ME points (PE then shell order) and the
 * per-pair integrals. */
static int solve_pair(const orc_ctx *X, const orc_offsets *o, const int *g_ij,
                      const double *phi_i, const int *lo_i, const double *phi_j, const int *lo_j,
                      const int *box, pair_work *w, pair_out *out)
{
    const orc_cell *c = X->c;
    const orc_stencil *st = X->st;
    int n = X->P->fd_n, lmax = X->P->lmax;
    int npe = o->n_pe, nme = o->n_me;
    size_t nb = (size_t)o->B[0] * o->B[1] * o->B[2];

    /* local Cartesian coordinates r-bar = h(m/N) of every subdomain point */
    for (int q = 0; q < nme; ++q) offset_xyz(c, o->m + 3 * (size_t)q, w->xyz + 3 * (size_t)q);

    /* Step III: orbitals on the translated subdomain, g = MOD(g_ij + m, N) (Eq. l2g) */
    for (int q = 0; q < nme; ++q) {
        int g[3];
        for (int al = 0; al < 3; ++al) g[al] = (int)imod((long)g_ij[al] + o->m[3 * (size_t)q + al], c->n[al]);
        w->fi[q] = phi_at(phi_i, box, lo_i, c->n, g);
        w->fj[q] = phi_at(phi_j, box, lo_j, c->n, g);
    }
    /* pair density on PE (Eq. rho_from_phi_mlwf) */
    for (int q = 0; q < npe; ++q) w->rho[q] = w->fi[q] * w->fj[q];

    /* multipoles about the grid-resolved centre (Eq. mepole) */
    double Q[NLM];
    double *chg = w->b;   /* scratch: rho dV */
    for (int q = 0; q < npe; ++q) chg[q] = w->rho[q] * c->dv;
    multipoles(lmax, npe, w->xyz, chg, Q);

    /* far field on the shell (Eq. me) */
    for (int q = npe; q < nme; ++q) w->v[q] = farfield(lmax, Q, w->xyz + 3 * (size_t)q);

    /* right-hand side 4 pi rho + (L applied to the shell values) on PE (Eq. pe) */
    memset(w->box, 0, sizeof(double) * nb);
    for (int q = npe; q < nme; ++q) w->box[o->box_index[q]] = w->v[q];
    int stride[6];
    for (int d = 0; d < st->ndir; ++d)
        stride[d] = (st->d[d][0] * o->B[1] + st->d[d][1]) * o->B[2] + st->d[d][2];
    for (int k = 0; k < npe; ++k) {
        int idx = o->box_index[k];
        double s = 0.0;
        for (int d = 0; d < st->ndir; ++d) {
            double t = 0.0;
            for (int q = 1; q <= n; ++q) t += X->w2[q] * (w->box[idx + q * stride[d]] + w->box[idx - q * stride[d]]);
            s += st->coef[d] * t;
        }
        w->b[k] = 4.0 * M_PI * w->rho[k] + s;
    }
    memset(w->box, 0, sizeof(double) * nb);

    /* Step IV: near field by CG */
    int e = cg_solve(X, o, w->b, w->x, w->box, w->r, w->p, w->q, &out->n_cg, &out->resid);
    out->status = e;
    for (int k = 0; k < npe; ++k) w->v[k] = w->x[k];

    /* Step V: energy integral over PE (Eq. exxGen_mlwf) */
    double es = 0.0;
    for (int k = 0; k < npe; ++k) es += w->rho[k] * w->v[k];
    out->e_pair = es * c->dv;

    /* stress integrand (Eq. sxx_working): grad v by central first differences
     * along the lattice directions (Eq. d1_1), grad_r = J grad_xi (Eq. jacb) */
    memset(w->box, 0, sizeof(double) * nb);
    for (int q = 0; q < nme; ++q) w->box[o->box_index[q]] = w->v[q];
    int ax[3];
    for (int al = 0; al < 3; ++al) ax[al] = (al == 0 ? o->B[1] * o->B[2] : (al == 1 ? o->B[2] : 1));
    double sig[3][3] = {{0}};
    for (int k = 0; k < npe; ++k) {
        int idx = o->box_index[k];
        double dxi[3];
        for (int al = 0; al < 3; ++al) {
            double t = 0.0;
            for (int q = 1; q <= n; ++q) t += X->w1[q] * (w->box[idx + q * ax[al]] - w->box[idx - q * ax[al]]);
            dxi[al] = t / c->dxi[al];
        }
        double dv_r[3];
        for (int a = 0; a < 3; ++a) dv_r[a] = c->J[a][0] * dxi[0] + c->J[a][1] * dxi[1] + c->J[a][2] * dxi[2];
        const double *rb = w->xyz + 3 * (size_t)k;
        for (int a = 0; a < 3; ++a)
            for (int al = 0; al < 3; ++al) {
                double hr = c->hinv[al][0] * rb[0] + c->hinv[al][1] * rb[1] + c->hinv[al][2] * rb[2];
                sig[a][al] += hr * w->rho[k] * dv_r[a];
            }
    }
    memset(w->box, 0, sizeof(double) * nb);
    for (int a = 0; a < 3; ++a)
        for (int al = 0; al < 3; ++al) out->sig[a][al] = sig[a][al] * c->dv;
    return e;
}

/* D^i += v phi_j and, for i != j, D^j += v phi_i on every ME point (Eq. Dxx,
 * Step V); repeated grid points under the MOD wrap add. */
static int scatter_d(const orc_cell *c, const orc_offsets *o, const int *g_ij, int i, int j,
                     const pair_work *w, double *dxx, const int *dbox, const int *dbox_lo)
{
    size_t dsz = (size_t)dbox[0] * dbox[1] * dbox[2];
    for (int q = 0; q < o->n_me; ++q) {
        int g[3];
        for (int al = 0; al < 3; ++al) g[al] = (int)imod((long)g_ij[al] + o->m[3 * (size_t)q + al], c->n[al]);
        int who[2] = {i, j};
        double val[2] = {w->v[q] * w->fj[q], w->v[q] * w->fi[q]};
        int nt = (i == j) ? 1 : 2;
        for (int t = 0; t < nt; ++t) {
            const int *lo = dbox_lo + 3 * who[t];
            long u[3];
            int inside = 1;
            for (int al = 0; al < 3; ++al) {
                u[al] = imod((long)g[al] - lo[al], c->n[al]);
                if (u[al] >= dbox[al]) inside = 0;
            }
            if (!inside) {
                if (val[t] != 0.0) return ORC_ERR_BOX;
                continue;
            }
            dxx[(size_t)who[t] * dsz + ((size_t)u[0] * dbox[1] + u[1]) * dbox[2] + u[2]] += val[t];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Whole EXX evaluation.                                                */
/* ------------------------------------------------------------------ */
int orc_exx(const double *lattice, const int *n, int n_orb, const double *centres,
            const int *box, const int *box_lo, const double *phi,
            const int *dbox, const int *dbox_lo, double *dxx,
            const orc_params *P,
            int n_sel, const int *sel,            /* NULL: all pairs */
            int pair_cap, int *n_pairs, int *pair_rows,       /* [cap][8] */
            double *pair_e, double *pair_sig, int *pair_ncg, double *pair_res,
            double *e_xx, double *dedh, double *stress, int *info /* [4]: n_aux, n_stcl, max_cg, failed */)
{
    orc_cell c, c0;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    if (P->fd_n < 1 || P->fd_n > MAXN || P->lmax < 0 || P->lmax > MAXL) return ORC_ERR_ARG;
    if (P->frozen) { e = cell_init(&c0, P->lattice0, n); if (e) return e; }
    const orc_cell *cref = P->frozen ? &c0 : &c;

    orc_stencil st;
    e = stencil_for(&c, P, &c0, &st);
    if (e) return e;

    orc_offsets off[2];
    e = build_offsets(cref, P->r_pe_self, P->r_me_self, &off[0]);
    if (e) return e;
    e = build_offsets(cref, P->r_pe_pair, P->r_me_pair, &off[1]);
    if (e) { offsets_free(&off[0]); return e; }
    e = check_halo(&off[0], &st, P->fd_n);
    if (!e) e = check_halo(&off[1], &st, P->fd_n);
    if (e) { offsets_free(&off[0]); offsets_free(&off[1]); return e; }

    int np = 0;
    e = orc_pair_list(lattice, n, n_orb, centres, P->r_pair, pair_cap, &np, pair_rows);
    if (e) { offsets_free(&off[0]); offsets_free(&off[1]); return e; }
    *n_pairs = np;

    orc_ctx X;
    X.c = &c; X.st = &st; X.P = P;
    orc_fd2_weights(P->fd_n, X.w2);
    orc_fd1_weights(P->fd_n, X.w1);

    int nsel = sel ? n_sel : np;
    size_t bsz = (size_t)box[0] * box[1] * box[2];
    size_t dsz = dbox ? (size_t)dbox[0] * dbox[1] * dbox[2] : 0;
    if (dxx) memset(dxx, 0, sizeof(double) * dsz * n_orb);
    int status = ORC_OK, failed = -1, maxcg = 0;
    if (P->n_threads > 0) omp_set_num_threads(P->n_threads);

    #pragma omp parallel
    {
        pair_work W[2];
        int ok[2];
        ok[0] = work_alloc(&W[0], &off[0]);
        ok[1] = work_alloc(&W[1], &off[1]);
        #pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < nsel; ++t) {
            int pi = sel ? sel[t] : t;
            if (pi < 0 || pi >= np) {
                #pragma omp critical
                status = ORC_ERR_ARG;
                continue;
            }
            const int *row = pair_rows + 8 * (size_t)pi;
            int i = row[0], j = row[1];
            int which = (i == j) ? 0 : 1;
            if (ok[which]) {
                #pragma omp critical
                status = ORC_ERR_MEM;
                continue;
            }
            pair_out po;
            memset(&po, 0, sizeof(po));
            int es = solve_pair(&X, &off[which], row + 5, phi + (size_t)i * bsz, box_lo + 3 * i,
                                phi + (size_t)j * bsz, box_lo + 3 * j, box, &W[which], &po);
            pair_e[pi] = po.e_pair;
            for (int a = 0; a < 3; ++a)
                for (int al = 0; al < 3; ++al) pair_sig[9 * (size_t)pi + 3 * a + al] = po.sig[a][al];
            pair_ncg[pi] = po.n_cg;
            pair_res[pi] = po.resid;
            int ed = ORC_OK;
            if (dxx) {
                #pragma omp critical(dscatter)
                ed = scatter_d(&c, &off[which], row + 5, i, j, &W[which], dxx, dbox, dbox_lo);
            }
            #pragma omp critical
            {
                if (po.n_cg > maxcg) maxcg = po.n_cg;
                if (es && status == ORC_OK) { status = es; failed = pi; }
                if (ed && status == ORC_OK) { status = ed; failed = pi; }
            }
        }
        work_free(&W[0]);
        work_free(&W[1]);
    }

    /* E_xx = -sum_<ij> w int rho v, w = 1 (i = j) or 2 (i != j) (Eq. exxGen_mlwf);
     * sigma^{a alpha} = -2 sum_<ij> w sum_b hinv_{alpha b} int r_b rho d_a v (Eq. sxx_working);
     * Pi_ab = -(1/V) sum_alpha sigma^{a alpha} h_{b alpha} (Eq. pixx_working).
     * Sums run over the selected pairs in list order. */
    double E = 0.0, S[3][3] = {{0}};
    for (int t = 0; t < nsel; ++t) {
        int pi = sel ? sel[t] : t;
        if (pi < 0 || pi >= np) continue;
        const int *row = pair_rows + 8 * (size_t)pi;
        double w = (row[0] == row[1]) ? 1.0 : 2.0;
        E -= w * pair_e[pi];
        for (int a = 0; a < 3; ++a)
            for (int al = 0; al < 3; ++al) S[a][al] -= 2.0 * w * pair_sig[9 * (size_t)pi + 3 * a + al];
    }
    *e_xx = E;
    for (int a = 0; a < 3; ++a)
        for (int al = 0; al < 3; ++al) dedh[3 * a + al] = S[a][al];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int al = 0; al < 3; ++al) s += S[a][al] * c.h[b][al];
            stress[3 * a + b] = -s / c.vol;
        }
    info[0] = st.n_aux;
    info[1] = 2 * P->fd_n * st.ndir + 1;
    info[2] = maxcg;
    info[3] = failed;
    offsets_free(&off[0]);
    offsets_free(&off[1]);
    return status;
}

/* The potential of one pair (i, j) with grid centre g_ij on its ME points,
 * PE points first: the near field of the CG solve and the far field on the
 * shell.  Used by the tests to compare with closed forms. */
int orc_pair_potential(const double *lattice, const int *n, const int *box,
                       const double *phi_i, const int *lo_i, const double *phi_j, const int *lo_j,
                       const int *g_ij, int self, const orc_params *P, int cap, double *v_out, int *n_pe, int *n_me,
                       int *n_cg, double *e_pair)
{
    orc_cell c, c0;
    int e = cell_init(&c, lattice, n);
    if (e) return e;
    if (P->frozen) { e = cell_init(&c0, P->lattice0, n); if (e) return e; }
    orc_stencil st;
    e = stencil_for(&c, P, &c0, &st);
    if (e) return e;
    orc_offsets o;
    e = build_offsets(P->frozen ? &c0 : &c, self ? P->r_pe_self : P->r_pe_pair, self ? P->r_me_self : P->r_me_pair, &o);
    if (e) return e;
    e = check_halo(&o, &st, P->fd_n);
    if (e) { offsets_free(&o); return e; }
    if (o.n_me > cap) { offsets_free(&o); return ORC_ERR_CAP; }
    orc_ctx X;
    X.c = &c; X.st = &st; X.P = P;
    orc_fd2_weights(P->fd_n, X.w2);
    orc_fd1_weights(P->fd_n, X.w1);
    pair_work W;
    if (work_alloc(&W, &o)) { work_free(&W); offsets_free(&o); return ORC_ERR_MEM; }
    pair_out po;
    e = solve_pair(&X, &o, g_ij, phi_i, lo_i, phi_j, lo_j, box, &W, &po);
    memcpy(v_out, W.v, sizeof(double) * (size_t)o.n_me);
    *n_pe = o.n_pe;
    *n_me = o.n_me;
    *n_cg = po.n_cg;
    *e_pair = po.e_pair;
    work_free(&W);
    offsets_free(&o);
    return e;
}
