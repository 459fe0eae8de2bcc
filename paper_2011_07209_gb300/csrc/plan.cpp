// plan.cpp -- host geometry of the EXX pair path.
//
// Cell metric (Sec. II B 1, Eqs. s_to_xi, jacb, lapG_), Natan-Kronik stencil
// with auxiliary grid directions (Eqs. nk2d_aux, kappa_def, nk3d_mu,
// nk3d_Mb_f, lapG_mod_nk3d, Algorithm 1), central-difference weights
// (Eqs. d2_1, d1_1) and proto-subdomain offset sets (Eqs. rbar, g0).
//
// Compiled with -ffp-contract=off: the PE / shell membership test and h^-1
// are integer-deciding arithmetic and follow a fixed operation order.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/exx.h"

namespace exx {

int make_metric(const double lattice[3][3], const int n[3], Metric &m)
{
    for (int a = 0; a < 3; ++a)
        for (int al = 0; al < 3; ++al) m.h[a][al] = lattice[al][a];
    const double(*h)[3] = m.h;
    // det and adjugate, left-to-right products and sums
    const double c00 = h[1][1] * h[2][2] - h[1][2] * h[2][1];
    const double c01 = h[1][0] * h[2][2] - h[1][2] * h[2][0];
    const double c02 = h[1][0] * h[2][1] - h[1][1] * h[2][0];
    const double det = h[0][0] * c00 - h[0][1] * c01 + h[0][2] * c02;
    if (!(det > 0.0) || !std::isfinite(det)) return EXX_ERR_CELL;
    m.hinv[0][0] = c00 / det;
    m.hinv[0][1] = (h[0][2] * h[2][1] - h[0][1] * h[2][2]) / det;
    m.hinv[0][2] = (h[0][1] * h[1][2] - h[0][2] * h[1][1]) / det;
    m.hinv[1][0] = (h[1][2] * h[2][0] - h[1][0] * h[2][2]) / det;
    m.hinv[1][1] = (h[0][0] * h[2][2] - h[0][2] * h[2][0]) / det;
    m.hinv[1][2] = (h[0][2] * h[1][0] - h[0][0] * h[1][2]) / det;
    m.hinv[2][0] = c02 / det;
    m.hinv[2][1] = (h[0][1] * h[2][0] - h[0][0] * h[2][1]) / det;
    m.hinv[2][2] = (h[0][0] * h[1][1] - h[0][1] * h[1][0]) / det;
    m.vol = det;
    for (int al = 0; al < 3; ++al) {
        if (n[al] < 1) return EXX_ERR_ARG;
        m.n[al] = n[al];
        m.len[al] = std::sqrt(h[0][al] * h[0][al] + h[1][al] * h[1][al] + h[2][al] * h[2][al]);
        m.dxi[al] = m.len[al] / n[al];
    }
    m.dv = det / ((double)n[0] * n[1] * n[2]);
    for (int a = 0; a < 3; ++a)
        for (int al = 0; al < 3; ++al) m.J[a][al] = m.len[al] * m.hinv[al][a];
    for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be)
            m.F[al][be] = m.J[0][al] * m.J[0][be] + m.J[1][al] * m.J[1][be] + m.J[2][al] * m.J[2][be];
    return EXX_OK;
}

// Eigenvalues of a symmetric 3x3 matrix by cyclic Jacobi rotations (each
// rotation zeroes one off-diagonal element; a few sweeps reach rounding level).
static void sym3_eigenvalues(double a[3][3], double ev[3])
{
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double diag = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {   // A <- A G (columns p, q)
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {   // A <- G^T A (rows p, q)
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
            }
    }
    for (int k = 0; k < 3; ++k) ev[k] = a[k][k];
}

int cell_strain(const double lattice0[3][3], const double lattice[3][3], double &eps_max, double &dvol)
{
    const int n1[3] = {1, 1, 1};
    Metric m0, m;
    int e = make_metric(lattice0, n1, m0);
    if (e) return e;
    if ((e = make_metric(lattice, n1, m))) return e;
    double F[3][3], E[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) F[a][b] = m.h[a][0] * m0.hinv[0][b] + m.h[a][1] * m0.hinv[1][b] + m.h[a][2] * m0.hinv[2][b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            E[a][b] = 0.5 * (F[0][a] * F[0][b] + F[1][a] * F[1][b] + F[2][a] * F[2][b] - (a == b ? 1.0 : 0.0));
    double ev[3];
    sym3_eigenvalues(E, ev);
    eps_max = std::max(std::fabs(ev[0]), std::max(std::fabs(ev[1]), std::fabs(ev[2])));
    dvol = m.vol / m0.vol - 1.0;
    return EXX_OK;
}

// r = h (m / N): the offset vector of a grid step, fixed operation order.
static inline void step_vec(const Metric &mt, const int *m, double *r)
{
    const double s0 = (double)m[0] / (double)mt.n[0];
    const double s1 = (double)m[1] / (double)mt.n[1];
    const double s2 = (double)m[2] / (double)mt.n[2];
    for (int a = 0; a < 3; ++a) r[a] = mt.h[a][0] * s0 + mt.h[a][1] * s1 + mt.h[a][2] * s2;
}

static inline double step_len(const Metric &mt, const int *m)
{
    double r[3];
    step_vec(mt, m, r);
    return std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
}

void fd_weights(int n, double *w2, double *w1)
{
    // Moment conditions of the central (2n+1)-point formulas solved by Gaussian
    // elimination in long double.
    long double A[kMaxFd + 1][kMaxFd + 2];
    // second derivative: unknowns w_0..w_n, moments k = 0, 2, ..., 2n
    for (int r = 0; r <= n; ++r) {
        const int k = 2 * r;
        for (int q = 0; q <= n; ++q) {
            if (q == 0) A[r][q] = (k == 0) ? 1.0L : 0.0L;
            else A[r][q] = 2.0L * std::pow((long double)q, (long double)k);
        }
        A[r][n + 1] = (k == 2) ? 2.0L : 0.0L;
    }
    auto solve = [](long double (*M)[kMaxFd + 2], int sz, long double *x) {
        for (int c = 0; c < sz; ++c) {
            int p = c;
            for (int r = c + 1; r < sz; ++r)
                if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
            for (int k = 0; k <= sz; ++k) std::swap(M[c][k], M[p][k]);
            for (int r = 0; r < sz; ++r) {
                if (r == c) continue;
                const long double f = M[r][c] / M[c][c];
                for (int k = c; k <= sz; ++k) M[r][k] -= f * M[c][k];
            }
        }
        for (int c = 0; c < sz; ++c) x[c] = M[c][sz] / M[c][c];
    };
    long double x[kMaxFd + 1];
    solve(A, n + 1, x);
    for (int q = 0; q <= n; ++q) w2[q] = (double)x[q];
    // first derivative: unknowns w_1..w_n, moments k = 1, 3, ..., 2n-1
    long double B[kMaxFd + 1][kMaxFd + 2];
    for (int r = 0; r < n; ++r) {
        const int k = 2 * r + 1;
        for (int q = 1; q <= n; ++q) B[r][q - 1] = 2.0L * std::pow((long double)q, (long double)k);
        B[r][n] = 0.0L;
    }
    // move rhs into column n (size n system)
    for (int r = 0; r < n; ++r) {
        const int k = 2 * r + 1;
        B[r][n] = (k == 1) ? 1.0L : 0.0L;
    }
    long double y[kMaxFd + 1];
    {
        long double Mx[kMaxFd + 1][kMaxFd + 2];
        for (int r = 0; r < n; ++r)
            for (int c = 0; c <= n; ++c) Mx[r][c] = B[r][c];
        solve(Mx, n, y);
    }
    w1[0] = 0.0;
    for (int q = 1; q <= n; ++q) w1[q] = (double)y[q - 1];
}

namespace {

struct Cand {
    int m[3];
    double len;
};

bool cand_less(const Cand &x, const Cand &y)
{
    if (x.len != y.len) return x.len < y.len;
    for (int k = 0; k < 3; ++k)
        if (x.m[k] != y.m[k]) return x.m[k] < y.m[k];
    return false;
}

// The sorted list of candidate non-axial grid directions (input of Algorithm
// 1): shells of max_alpha |m_alpha| = S swept outward; the sweep ends after the
// first shell S >= 2 lying wholly beyond the longest first-shell spacing.
std::vector<Cand> candidates(const Metric &mt, int nq)
{
    std::vector<Cand> out;
    double first_shell_max = 0.0;
    for (int S = 1; S <= 8; ++S) {
        double shell_min = HUGE_VAL;
        for (int i = -S; i <= S; ++i)
            for (int j = -S; j <= S; ++j)
                for (int k = -S; k <= S; ++k) {
                    if (std::max(std::abs(i), std::max(std::abs(j), std::abs(k))) != S) continue;
                    const int m[3] = {i, j, k};
                    const double l = step_len(mt, m);
                    if (S == 1) first_shell_max = std::max(first_shell_max, l);
                    shell_min = std::min(shell_min, l);
                    const int nz = (i != 0) + (j != 0) + (k != 0);
                    const int lead = i != 0 ? i : (j != 0 ? j : k);
                    if (nz >= 2 && lead > 0) out.push_back(Cand{{i, j, k}, l});
                }
        if (S >= 2 && shell_min > first_shell_max) break;
    }
    std::sort(out.begin(), out.end(), cand_less);
    if ((int)out.size() > nq) out.resize(nq);
    return out;
}

void unit_coeffs(const Metric &mt, const int *m, double *a, double *len)
{
    const double l = step_len(mt, m);
    for (int al = 0; al < 3; ++al) a[al] = (double)m[al] * mt.dxi[al] / l;
    *len = l;
}

double det3(const double M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

// Algorithm 1 of the paper on the candidate list.
int choose_aux(const Metric &mt, const std::vector<Cand> &cands, int aux[3][3])
{
    double col[3][3] = {};
    int p = 0;
    for (const Cand &c : cands) {
        double a[3], l;
        unit_coeffs(mt, c.m, a, &l);
        col[p][0] = a[0] * a[1];
        col[p][1] = a[0] * a[2];
        col[p][2] = a[1] * a[2];
        bool ok;
        if (p == 0) {
            ok = true;
        } else if (p == 1) {
            const double d = col[0][0] * col[1][0] + col[0][1] * col[1][1] + col[0][2] * col[1][2];
            const double n0 = col[0][0] * col[0][0] + col[0][1] * col[0][1] + col[0][2] * col[0][2];
            const double n1 = col[1][0] * col[1][0] + col[1][1] * col[1][1] + col[1][2] * col[1][2];
            ok = std::fabs(d) < (1.0 - 1e-8) * std::sqrt(n0 * n1);
        } else {
            double M[3][3];
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) M[r][s] = col[s][r];
            const double scale = std::sqrt(col[0][0] * col[0][0] + col[0][1] * col[0][1] + col[0][2] * col[0][2]) *
                                 std::sqrt(col[1][0] * col[1][0] + col[1][1] * col[1][1] + col[1][2] * col[1][2]) *
                                 std::sqrt(col[2][0] * col[2][0] + col[2][1] * col[2][1] + col[2][2] * col[2][2]);
            ok = std::fabs(det3(M)) > 1e-10 * scale;
        }
        if (ok) {
            for (int k = 0; k < 3; ++k) aux[p][k] = c.m[k];
            if (++p == 3) return EXX_OK;
        }
    }
    return EXX_ERR_NK;
}

// Symbol of the operator at wave vector t: sum_dir coef (w0 + 2 sum_q w_q cos(q t.d)).
bool negative_definite(const Stencil &st, int n)
{
    double w2[kMaxFd + 1], w1[kMaxFd + 1];
    fd_weights(n, w2, w1);
    const int G = 32;
    const double two_pi = 6.283185307179586;
    for (int i = 0; i < G; ++i)
        for (int j = 0; j < G; ++j)
            for (int k = 0; k < G; ++k) {
                if (!i && !j && !k) continue;
                const double t0 = two_pi * i / G, t1 = two_pi * j / G, t2 = two_pi * k / G;
                double s = 0.0;
                for (int d = 0; d < st.ndir; ++d) {
                    const double ph = t0 * st.dir[d][0] + t1 * st.dir[d][1] + t2 * st.dir[d][2];
                    double sym = w2[0];
                    for (int q = 1; q <= n; ++q) sym += 2.0 * w2[q] * std::cos(q * ph);
                    s += st.coef[d] * sym;
                }
                if (!(s < 0.0)) return false;
            }
    return true;
}

}  // namespace

int make_stencil(const Metric &mt, int fd_n, int nq, const int (*aux_in)[3], int n_aux_fixed, Stencil &st)
{
    st = Stencil();
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    const double fdiag = std::max(mt.F[0][0], std::max(mt.F[1][1], mt.F[2][2]));
    int last_off = -1;
    for (int k = 0; k < 3; ++k)
        if (std::fabs(mt.F[pa[k]][pb[k]]) > 1e-12 * fdiag) {
            ++st.n_off;
            last_off = k;
        }
    int aux[3][3] = {};
    int n_aux = 0;
    if (aux_in) {
        n_aux = n_aux_fixed;
        for (int p = 0; p < n_aux; ++p)
            for (int k = 0; k < 3; ++k) aux[p][k] = aux_in[p][k];
    } else if (st.n_off == 1) {
        // grid-resolved bisector L' ~ L^_alpha + kappa L^_beta (Eqs. nk2d_aux, kappa_def)
        const int al = pa[last_off], be = pb[last_off];
        const double dotab = mt.h[0][al] * mt.h[0][be] + mt.h[1][al] * mt.h[1][be] + mt.h[2][al] * mt.h[2][be];
        aux[0][al] = 1;
        aux[0][be] = dotab > 0.0 ? -1 : 1;
        n_aux = 1;
    } else if (st.n_off >= 2) {
        if (choose_aux(mt, candidates(mt, nq), aux) != EXX_OK) return EXX_ERR_NK;
        n_aux = 3;
    }
    double a[3][3] = {}, len[3] = {};
    for (int p = 0; p < n_aux; ++p) unit_coeffs(mt, aux[p], a[p], &len[p]);
    double b[3] = {};
    if (n_aux == 1) {
        int al = -1, be = -1;
        for (int k = 0; k < 3; ++k)
            if (aux[0][pa[k]] != 0 && aux[0][pb[k]] != 0) {
                al = pa[k];
                be = pb[k];
            }
        if (al < 0) return EXX_ERR_NK;
        b[0] = mt.F[al][be] / (a[0][al] * a[0][be]);
        for (int k = 0; k < 3; ++k) {
            if (pa[k] == al && pb[k] == be) continue;
            if (std::fabs(mt.F[pa[k]][pb[k]] - b[0] * a[0][pa[k]] * a[0][pb[k]]) > 1e-12 * fdiag) return EXX_ERR_NK;
        }
    } else if (n_aux == 3) {
        // M b = (F12, F13, F23), Eq. nk3d_Mb_f; Gaussian elimination with pivoting
        double M[3][4];
        for (int p = 0; p < 3; ++p) {
            M[0][p] = a[p][0] * a[p][1];
            M[1][p] = a[p][0] * a[p][2];
            M[2][p] = a[p][1] * a[p][2];
        }
        M[0][3] = mt.F[0][1];
        M[1][3] = mt.F[0][2];
        M[2][3] = mt.F[1][2];
        for (int c = 0; c < 3; ++c) {
            int piv = c;
            for (int r = c + 1; r < 3; ++r)
                if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
            if (M[piv][c] == 0.0) return EXX_ERR_NK;
            for (int k = 0; k < 4; ++k) std::swap(M[c][k], M[piv][k]);
            for (int r = c + 1; r < 3; ++r) {
                const double f = M[r][c] / M[c][c];
                for (int k = c; k < 4; ++k) M[r][k] -= f * M[c][k];
            }
        }
        for (int r = 2; r >= 0; --r) {
            double s = M[r][3];
            for (int k = r + 1; k < 3; ++k) s -= M[r][k] * b[k];
            b[r] = s / M[r][r];
        }
    } else if (n_aux != 0) {
        return EXX_ERR_NK;
    }
    if (n_aux == 0 && st.n_off != 0) return EXX_ERR_NK;
    st.n_aux = n_aux;
    st.ndir = 3 + n_aux;
    for (int al = 0; al < 3; ++al) {
        double c = mt.F[al][al];
        for (int p = 0; p < n_aux; ++p) c -= b[p] * a[p][al] * a[p][al];
        st.dir[al][0] = st.dir[al][1] = st.dir[al][2] = 0;
        st.dir[al][al] = 1;
        st.coef[al] = c / (mt.dxi[al] * mt.dxi[al]);
    }
    for (int p = 0; p < n_aux; ++p) {
        for (int k = 0; k < 3; ++k) {
            st.dir[3 + p][k] = aux[p][k];
            st.a[p][k] = a[p][k];
        }
        st.b[p] = b[p];
        st.coef[3 + p] = b[p] / (len[p] * len[p]);
    }
    if (!negative_definite(st, fd_n)) return EXX_ERR_NK;
    return EXX_OK;
}

int make_offsets(const Metric &mt, double r_pe, double r_me, OffsetSet &o)
{
    o = OffsetSet();
    if (!(r_pe > 0.0) || !(r_me >= r_pe)) return EXX_ERR_ARG;
    int H[3];
    for (int al = 0; al < 3; ++al) {
        const double rn = std::sqrt(mt.hinv[al][0] * mt.hinv[al][0] + mt.hinv[al][1] * mt.hinv[al][1] +
                                    mt.hinv[al][2] * mt.hinv[al][2]);
        H[al] = (int)std::ceil(r_me * mt.n[al] * rn);
        if (H[al] > 500) return EXX_ERR_ARG;
    }
    const double pe2 = r_pe * r_pe, me2 = r_me * r_me;
    std::vector<int> shell;
    for (int i = -H[0]; i <= H[0]; ++i)
        for (int j = -H[1]; j <= H[1]; ++j)
            for (int k = -H[2]; k <= H[2]; ++k) {
                const int m[3] = {i, j, k};
                double r[3];
                step_vec(mt, m, r);
                const double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                if (d2 <= pe2) {
                    o.m.insert(o.m.end(), m, m + 3);
                } else if (d2 <= me2) {
                    shell.insert(shell.end(), m, m + 3);
                }
            }
    o.n_pe = (int)(o.m.size() / 3);
    o.m.insert(o.m.end(), shell.begin(), shell.end());
    o.n_me = (int)(o.m.size() / 3);
    return EXX_OK;
}

int make_layout(const OffsetSet &o, const Stencil &st, int fd_n, SetLayout &L)
{
    L = SetLayout();
    int Hpe[3] = {0, 0, 0}, Hme[3] = {0, 0, 0};
    for (int q = 0; q < o.n_me; ++q)
        for (int al = 0; al < 3; ++al) {
            const int v = std::abs(o.m[3 * q + al]);
            Hme[al] = std::max(Hme[al], v);
            if (q < o.n_pe) Hpe[al] = std::max(Hpe[al], v);
        }
    int reach[3];
    for (int al = 0; al < 3; ++al) {
        int r = 1;
        for (int d = 0; d < st.ndir; ++d) r = std::max(r, std::abs(st.dir[d][al]));
        reach[al] = fd_n * r;
    }
    for (int al = 0; al < 3; ++al) {
        L.c[al] = Hpe[al] + reach[al];
        L.B[al] = 2 * L.c[al] + 1;
    }
    L.B[2] = (L.B[2] + 3) & ~3;
    L.box = (long long)L.B[0] * L.B[1] * L.B[2];
    if (L.box > (1LL << 30)) return EXX_ERR_ARG;
    for (int d = 0; d < st.ndir; ++d) {
        L.dstride[d] = (st.dir[d][0] * L.B[1] + st.dir[d][1]) * L.B[2] + st.dir[d][2];
        L.rstride[d] = (st.dir[d][0] * L.B[1] + st.dir[d][1]) * L.B[2];
    }
    L.gstride[0] = L.B[1] * L.B[2];
    L.gstride[1] = L.B[2];
    L.gstride[2] = 1;
    // membership map over the ME bounding box: 1 PE, 2 shell
    const int MB[3] = {2 * Hme[0] + 1, 2 * Hme[1] + 1, 2 * Hme[2] + 1};
    std::vector<int> memb((size_t)MB[0] * MB[1] * MB[2], 0), shell_idx((size_t)MB[0] * MB[1] * MB[2], -1);
    auto mindex = [&](int m0, int m1, int m2) -> long long {
        if (std::abs(m0) > Hme[0] || std::abs(m1) > Hme[1] || std::abs(m2) > Hme[2]) return -1;
        return ((long long)(m0 + Hme[0]) * MB[1] + (m1 + Hme[1])) * MB[2] + (m2 + Hme[2]);
    };
    for (int q = 0; q < o.n_me; ++q) {
        const long long id = mindex(o.m[3 * q], o.m[3 * q + 1], o.m[3 * q + 2]);
        memb[id] = q < o.n_pe ? 1 : 2;
        if (q >= o.n_pe) shell_idx[id] = q - o.n_pe;
    }
    const int n_shell = o.n_me - o.n_pe;
    std::vector<char> is_halo(n_shell, 0);
    for (int q = 0; q < o.n_pe; ++q) {
        const int *m = &o.m[3 * q];
        for (int d = 0; d < st.ndir; ++d)
            for (int s = -fd_n; s <= fd_n; ++s) {
                if (!s) continue;
                const long long id = mindex(m[0] + s * st.dir[d][0], m[1] + s * st.dir[d][1], m[2] + s * st.dir[d][2]);
                if (id < 0 || memb[id] == 0) return EXX_ERR_HALO;
                if (memb[id] == 2) {
                    is_halo[shell_idx[id]] = 1;
                    if (L.bnd.empty() || L.bnd.back() != q) L.bnd.push_back(q);
                }
            }
    }
    auto box_off = [&](const int *m) -> int32_t {
        return (int32_t)(((long long)(m[0] + L.c[0]) * L.B[1] + (m[1] + L.c[1])) * L.B[2] + (m[2] + L.c[2]));
    };
    L.n_pe = o.n_pe;
    L.n_shell = n_shell;
    L.pe_m.resize(o.n_pe);
    L.pe_off.resize(o.n_pe);
    for (int q = 0; q < o.n_pe; ++q) {
        const int *m = &o.m[3 * q];
        L.pe_m[q] = pack_m(m[0], m[1], m[2]);
        L.pe_off[q] = box_off(m);
    }
    L.sh_m.reserve(n_shell);
    for (int pass = 0; pass < 2; ++pass)
        for (int s = 0; s < n_shell; ++s) {
            if ((pass == 0) != (is_halo[s] != 0)) continue;
            const int *m = &o.m[3 * (o.n_pe + s)];
            L.sh_m.push_back(pack_m(m[0], m[1], m[2]));
            if (pass == 0) L.halo_off.push_back(box_off(m));
        }
    L.n_halo = (int)L.halo_off.size();
    // aligned 4-point groups: PE rows are runs of equal (m0, m1) in the lexicographic list
    for (int q = 0; q < o.n_pe;) {
        int e = q;
        while (e < o.n_pe && o.m[3 * e] == o.m[3 * q] && o.m[3 * e + 1] == o.m[3 * q + 1]) ++e;
        const int lo = o.m[3 * q + 2] + L.c[2], hi = o.m[3 * (e - 1) + 2] + L.c[2];   // box columns
        const long long row = ((long long)(o.m[3 * q] + L.c[0]) * L.B[1] + (o.m[3 * q + 1] + L.c[1])) * L.B[2];
        for (int g = lo & ~3; g <= hi; g += 4) {
            int mask = 0;
            for (int i = 0; i < 4; ++i)
                if (g + i >= lo && g + i <= hi) mask |= 1 << i;
            const long long off = row + g;
            L.groups.push_back((int32_t)(((off >> 2) << 4) | mask));
        }
        q = e;
    }
    return EXX_OK;
}

int make_cluster_part(const SetLayout &L, const Stencil &st, int fd_n, int nc, ClusterPart &cp)
{
    cp = ClusterPart();
    cp.nc = nc;
    const int ng = (int)L.groups.size();
    if (nc < 1 || ng == 0) return EXX_ERR_ARG;
    const int B0 = L.B[0], B1 = L.B[1], B2 = L.B[2];
    if ((long long)B0 * B1 >= (1 << 13) || B2 >= (1 << 18)) return EXX_ERR_ARG;
    int reach2 = 0;
    for (int d = 0; d < st.ndir; ++d) reach2 = std::max(reach2, fd_n * std::abs(st.dir[d][2]));
    // the 12-wide window reads columns x - 4 .. x + 7 of a group at x
    cp.pad = (std::max(4, reach2) + 3) & ~3;
    cp.row_stride = (cp.pad + B2 + std::max(8, reach2 + 4) + 3) & ~3;
    // rows that hold PE points (stored), rows that hold only halo points (read as
    // zeros: mapped to a zero row), and PE groups per row
    const long long nrow = (long long)B0 * B1;
    std::vector<char> used(nrow, 0);
    std::vector<int> gcount(nrow, 0);
    for (int32_t off : L.halo_off) used[off / B2] = 2;
    for (int32_t off : L.pe_off) used[off / B2] = 1;
    cp.grc.resize(ng);
    for (int g = 0; g < ng; ++g) {
        const long long off = (long long)(L.groups[g] >> 4) << 2;
        const long long rid = off / B2;
        gcount[rid]++;
        cp.grc[g] = (int32_t)(rid | ((off % B2) << 13));
    }
    // contiguous row ranges with about ng / nc groups each
    cp.cta.assign((size_t)nc * 8, 0);
    cp.rows.assign((size_t)nrow * 2, 0);
    for (long long r = 0; r < nrow; ++r) cp.rows[2 * r] = -1;
    std::vector<long long> first_row(nc + 1, nrow);
    {
        long long cum = 0;
        int c = 0;
        first_row[0] = 0;
        for (long long r = 0; r < nrow; ++r) {
            while (c + 1 < nc && cum >= (long long)ng * (c + 1) / nc) first_row[++c] = r;
            cum += gcount[r];
        }
        for (int k = c + 1; k <= nc; ++k) first_row[k] = nrow;
    }
    int g = 0, k = 0;
    for (int c = 0; c < nc; ++c) {
        int32_t *t = &cp.cta[8 * (size_t)c];
        t[0] = g;
        t[2] = k;
        long long nstored = 1;   // row 0 of every CTA's region is the zero row
        for (long long r = first_row[c]; r < first_row[c + 1]; ++r) {
            g += gcount[r];
            if (used[r] == 2) cp.rows[2 * r] = -2;
            if (used[r] != 1) continue;
            cp.rows[2 * r] = c;
            cp.rows[2 * r + 1] = (int32_t)(nstored * cp.row_stride + cp.pad);
            ++nstored;
        }
        while (k < L.n_pe && (long long)L.pe_off[k] / B2 < first_row[c + 1]) ++k;
        t[1] = g;
        t[3] = k;
        t[4] = (int32_t)nstored;
        if (nstored * cp.row_stride > (1LL << 30)) return EXX_ERR_ARG;
        t[5] = (int32_t)(nstored * cp.row_stride);
        cp.max_p_floats = std::max(cp.max_p_floats, t[5]);
        cp.max_groups = std::max(cp.max_groups, t[1] - t[0]);
    }
    if (g != ng || k != L.n_pe) return EXX_ERR_ARG;
    cp.pe_gl.resize(L.n_pe);
    for (int q = 0, gg = 0; q < L.n_pe; ++q) {
        const long long off = L.pe_off[q];
        while (gg + 1 < ng && ((long long)(L.groups[gg + 1] >> 4) << 2) <= off) ++gg;
        const long long go = (long long)(L.groups[gg] >> 4) << 2;
        if (!(go <= off && off < go + 4)) return EXX_ERR_ARG;
        cp.pe_gl[q] = (gg << 2) | (int)(off - go);
    }
    return EXX_OK;
}

// ---------------------------------------------------------------------------
// Multigrid hierarchy (see plan.h).
// ---------------------------------------------------------------------------

// Parents of a box coordinate u along one axis: (coarse coordinate, weight).
static inline int mg_parents(int u, int *c, double *w)
{
    if ((u & 1) == 0) {
        c[0] = u >> 1;
        w[0] = 1.0;
        return 1;
    }
    c[0] = u >> 1;
    c[1] = (u >> 1) + 1;
    w[0] = w[1] = 0.5;
    return 2;
}

// Level l + 1 from level l: active coarse points, then A_c = P^T A P
// accumulated per coarse row in a dense window of coarse offsets.
static int mg_coarsen(const MgLevel &f, MgLevel &c)
{
    for (int a = 0; a < 3; ++a) c.B[a] = f.B[a] / 2 + 1;
    const long long cbox = (long long)c.B[0] * c.B[1] * c.B[2];
    c.idx.assign((size_t)cbox, -1);
    auto coords = [](const int *B, long long o, int *u) {
        u[2] = (int)(o % B[2]);
        u[1] = (int)((o / B[2]) % B[1]);
        u[0] = (int)(o / ((long long)B[1] * B[2]));
    };
    // parents of every fine point (at most 8), and the active coarse set
    std::vector<int32_t> pc((size_t)f.n * 8, -1);
    std::vector<double> pw((size_t)f.n * 8, 0.0);
    std::vector<long long> pbox((size_t)f.n * 8, -1);
    for (int i = 0; i < f.n; ++i) {
        int u[3], cc[3][2];
        double ww[3][2];
        int np[3];
        coords(f.B, f.pts[i], u);
        for (int a = 0; a < 3; ++a) np[a] = mg_parents(u[a], cc[a], ww[a]);
        int k = 0;
        for (int x = 0; x < np[0]; ++x)
            for (int y = 0; y < np[1]; ++y)
                for (int z = 0; z < np[2]; ++z, ++k) {
                    const long long o = ((long long)cc[0][x] * c.B[1] + cc[1][y]) * c.B[2] + cc[2][z];
                    pbox[(size_t)i * 8 + k] = o;
                    pw[(size_t)i * 8 + k] = ww[0][x] * ww[1][y] * ww[2][z];
                }
        // the coarse points are the fine points at even coordinates: each has its
        // own weight-1 child, so the columns of P are independent and P^T A P
        // stays positive definite (parents of odd boundary points that are not
        // coarse points drop out of P)
        if (!(u[0] & 1) && !(u[1] & 1) && !(u[2] & 1))
            c.idx[(size_t)(((long long)(u[0] >> 1) * c.B[1] + (u[1] >> 1)) * c.B[2] + (u[2] >> 1))] = 0;
    }
    c.pts.clear();
    for (long long o = 0; o < cbox; ++o)
        if (c.idx[(size_t)o] == 0) {
            c.idx[(size_t)o] = (int32_t)c.pts.size();
            c.pts.push_back((int32_t)o);
        }
    c.n = (int)c.pts.size();
    for (size_t k = 0; k < pc.size(); ++k)
        if (pbox[k] >= 0) pc[k] = c.idx[(size_t)pbox[k]];
    // coarse reach: a fine operator of reach r couples parents at most (r + 2) / 2 apart
    int reach = 0;
    for (int i = 0; i < f.n; ++i) {
        int u[3];
        coords(f.B, f.pts[i], u);
        for (int k = f.row[i]; k < f.row[i + 1]; ++k) {
            int v[3];
            coords(f.B, f.pts[f.col[k]], v);
            for (int a = 0; a < 3; ++a) reach = std::max(reach, std::abs(v[a] - u[a]));
        }
    }
    const int R = (reach + 2) / 2, W = 2 * R + 1;
    std::vector<double> win((size_t)c.n * W * W * W, 0.0);
    for (int i = 0; i < f.n; ++i)
        for (int k = f.row[i]; k < f.row[i + 1]; ++k) {
            const int j = f.col[k];
            const double a = f.val[k];
            for (int p = 0; p < 8; ++p) {
                const int ci = pc[(size_t)i * 8 + p];
                if (ci < 0) continue;
                int uc[3];
                coords(c.B, c.pts[ci], uc);
                const double wi = pw[(size_t)i * 8 + p] * a;
                for (int q = 0; q < 8; ++q) {
                    const int cj = pc[(size_t)j * 8 + q];
                    if (cj < 0) continue;
                    int vc[3];
                    coords(c.B, c.pts[cj], vc);
                    const int dx = vc[0] - uc[0] + R, dy = vc[1] - uc[1] + R, dz = vc[2] - uc[2] + R;
                    if (dx < 0 || dx >= W || dy < 0 || dy >= W || dz < 0 || dz >= W) return EXX_ERR_ARG;
                    win[(((size_t)ci * W + dx) * W + dy) * W + dz] += wi * pw[(size_t)j * 8 + q];
                }
            }
        }
    c.row.assign((size_t)c.n + 1, 0);
    c.col.clear();
    c.val.clear();
    for (int ci = 0; ci < c.n; ++ci) {
        int uc[3];
        coords(c.B, c.pts[ci], uc);
        std::vector<std::pair<int, double>> r;
        for (int dx = 0; dx < W; ++dx)
            for (int dy = 0; dy < W; ++dy)
                for (int dz = 0; dz < W; ++dz) {
                    const double v = win[(((size_t)ci * W + dx) * W + dy) * W + dz];
                    if (v == 0.0) continue;
                    const int x = uc[0] + dx - R, y = uc[1] + dy - R, z = uc[2] + dz - R;
                    const int cj = c.idx[((size_t)x * c.B[1] + y) * c.B[2] + z];
                    r.push_back({cj, v});
                }
        std::sort(r.begin(), r.end());
        for (const auto &e : r) {
            c.col.push_back(e.first);
            c.val.push_back(e.second);
        }
        c.row[ci + 1] = (int32_t)c.col.size();
    }
    return EXX_OK;
}

int make_mg_levels(const SetLayout &L, const Stencil &st, int fd_n, int min_points, std::vector<MgLevel> &lv)
{
    lv.clear();
    if (fd_n < 1 || fd_n > kMaxFd || min_points < 1) return EXX_ERR_ARG;
    double w2[kMaxFd + 1], w1[kMaxFd + 1];
    fd_weights(fd_n, w2, w1);
    MgLevel f;
    for (int a = 0; a < 3; ++a) f.B[a] = L.B[a];
    f.n = L.n_pe;
    f.idx.assign((size_t)L.box, -1);
    f.pts = L.pe_off;
    for (int i = 0; i < f.n; ++i) f.idx[(size_t)L.pe_off[i]] = i;
    // A = -L: centre -sum_d coef_d w2[0], neighbours -coef_d w2[|q|] (PE only)
    double centre = 0.0;
    for (int d = 0; d < st.ndir; ++d) centre += st.coef[d] * w2[0];
    f.row.assign((size_t)f.n + 1, 0);
    for (int i = 0; i < f.n; ++i) {
        std::vector<std::pair<int, double>> r;
        r.push_back({i, -centre});
        for (int d = 0; d < st.ndir; ++d)
            for (int q = 1; q <= fd_n; ++q)
                for (int sg = -1; sg <= 1; sg += 2) {
                    const long long o = (long long)L.pe_off[i] + (long long)sg * q * L.dstride[d];
                    if (o < 0 || o >= L.box) continue;
                    const int j = f.idx[(size_t)o];
                    if (j >= 0) r.push_back({j, -st.coef[d] * w2[q]});
                }
        std::sort(r.begin(), r.end());
        for (const auto &e : r) {
            f.col.push_back(e.first);
            f.val.push_back(e.second);
        }
        f.row[i + 1] = (int32_t)f.col.size();
    }
    lv.push_back(std::move(f));
    while (lv.back().n > min_points) {
        MgLevel c;
        const int e = mg_coarsen(lv.back(), c);
        if (e) return e;
        if (c.n >= lv.back().n) break;   // no reduction (degenerate box): stop
        lv.push_back(std::move(c));
    }
    return EXX_OK;
}

// Device form of the hierarchy (see plan.h).
int make_mg_tables(const SetLayout &L, const Stencil &st, int fd_n, int min_points, double omega, double drop,
                   MgTables &t)
{
    t = MgTables();
    std::vector<MgLevel> lv;
    int e = make_mg_levels(L, st, fd_n, min_points, lv);
    if (e) return e;
    const int nl = (int)lv.size();
    if (nl < 2 || nl > kMgMaxLevels || lv.back().n > kMgMaxCoarsest) return EXX_OK;   // no hierarchy
    auto coords = [](const int *B, long long o, int *u) {
        u[2] = (int)(o % B[2]);
        u[1] = (int)((o / B[2]) % B[1]);
        u[0] = (int)(o / ((long long)B[1] * B[2]));
    };
    MgTables r;
    r.nlev = nl;
    r.n[0] = lv[0].n;
    for (int l = 1; l < nl; ++l) {
        const MgLevel &A = lv[l];
        r.n[l] = A.n;
        for (int a = 0; a < 3; ++a) r.Bp[l][a] = A.B[a] + 2 * kMgPad;
        r.Bp[l][2] = (r.Bp[l][2] + 3) & ~3;   // rows start on 16-byte boundaries
        r.box[l] = (long long)r.Bp[l][0] * r.Bp[l][1] * r.Bp[l][2];
        r.slot_floats += 3 * ((r.box[l] + 63) & ~63LL);
        std::vector<int> u((size_t)3 * A.n);
        r.pts[l].resize(A.n);
        for (int i = 0; i < A.n; ++i) {
            coords(A.B, A.pts[i], &u[3 * (size_t)i]);
            const int *v = &u[3 * (size_t)i];
            r.pts[l][i] = (int32_t)((((long long)v[0] + kMgPad) * r.Bp[l][1] + v[1] + kMgPad) * r.Bp[l][2] + v[2] +
                                    kMgPad);
        }
        if (l == nl - 1) {
            // coarsest: the inverse of A_l by Gauss-Jordan elimination (SPD, no pivoting needed)
            const int n = A.n;
            std::vector<double> a((size_t)n * n, 0.0), inv((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i) {
                inv[(size_t)i * n + i] = 1.0;
                for (int k = A.row[i]; k < A.row[i + 1]; ++k) a[(size_t)i * n + A.col[k]] = A.val[k];
            }
            for (int c = 0; c < n; ++c) {
                const double piv = a[(size_t)c * n + c];
                if (!(piv > 0.0)) return EXX_OK;
                for (int k = 0; k < n; ++k) {
                    a[(size_t)c * n + k] /= piv;
                    inv[(size_t)c * n + k] /= piv;
                }
                for (int i = 0; i < n; ++i) {
                    if (i == c) continue;
                    const double f = a[(size_t)i * n + c];
                    if (f == 0.0) continue;
                    for (int k = 0; k < n; ++k) {
                        a[(size_t)i * n + k] -= f * a[(size_t)c * n + k];
                        inv[(size_t)i * n + k] -= f * inv[(size_t)c * n + k];
                    }
                }
            }
            r.cinv.resize((size_t)n * n);
            for (size_t k = 0; k < r.cinv.size(); ++k) r.cinv[k] = (float)inv[k];
            continue;
        }
        // interior stencil: the row of the active point nearest the centre of the set
        double cm[3] = {0, 0, 0};
        for (int i = 0; i < A.n; ++i)
            for (int a = 0; a < 3; ++a) cm[a] += u[3 * (size_t)i + a];
        for (int a = 0; a < 3; ++a) cm[a] /= A.n;
        int i0 = 0;
        double best = 1e300;
        for (int i = 0; i < A.n; ++i) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) d2 += (u[3 * (size_t)i + a] - cm[a]) * (u[3 * (size_t)i + a] - cm[a]);
            if (d2 < best) {
                best = d2;
                i0 = i;
            }
        }
        int pidx[125];
        std::fill(pidx, pidx + 125, -1);
        int K = 0;
        std::vector<double> wint;
        auto key = [&](int i, int j, int *d) {
            for (int a = 0; a < 3; ++a) d[a] = u[3 * (size_t)j + a] - u[3 * (size_t)i + a];
            if (std::abs(d[0]) > kMgPad || std::abs(d[1]) > kMgPad || std::abs(d[2]) > kMgPad) return -1;
            return ((d[0] + 2) * 5 + d[1] + 2) * 5 + d[2] + 2;
        };
        for (int k = A.row[i0]; k < A.row[i0 + 1]; ++k) {
            int d[3];
            const int kk = key(i0, A.col[k], d);
            if (kk < 0 || K >= kMgMaxK) return EXX_OK;
            pidx[kk] = K;
            r.kd[l][K] = (d[0] + 2) | (d[1] + 2) << 3 | (d[2] + 2) << 6;
            r.wint[l][K] = (float)A.val[k];
            wint.push_back(A.val[k]);
            ++K;
        }
        // pattern entries kept on the device: |a| >= drop x the interior diagonal; a dropped
        // entry of any row is added, as |a|, to that row's diagonal (the change is
        // + |a| (e_i -+ e_j)(e_i -+ e_j)^T over each symmetric pair, so the operator stays
        // symmetric positive definite)
        int kc = -1;
        for (int k = 0; k < K; ++k)
            if (r.kd[l][k] == (2 | 2 << 3 | 2 << 6)) kc = k;
        if (kc < 0) return EXX_OK;
        std::vector<char> keep(K, 1);
        for (int k = 0; k < K; ++k) keep[k] = k == kc || std::fabs(wint[k]) >= drop * std::fabs(wint[kc]);
        r.K[l] = K;
        // rows of A_l over the pattern; interior rows first, then the others
        std::vector<double> w((size_t)A.n * K, 0.0), diag(A.n, 0.0);
        std::vector<char> interior(A.n, 0);
        for (int i = 0; i < A.n; ++i) {
            double *wi = &w[(size_t)i * K];
            bool same = (A.row[i + 1] - A.row[i]) == K;
            for (int k = A.row[i]; k < A.row[i + 1]; ++k) {
                int d[3];
                const int kk = key(i, A.col[k], d);
                if (kk < 0 || pidx[kk] < 0) return EXX_OK;   // an entry outside the interior pattern
                wi[pidx[kk]] = A.val[k];
                if (A.col[k] == i) diag[i] = A.val[k];
            }
            if (!(diag[i] > 0.0)) return EXX_OK;
            for (int k = 0; k < K && same; ++k) same = std::fabs(wi[k] - wint[k]) <= 1e-12 * std::fabs(wint[k]);
            interior[i] = same;
            for (int k = 0; k < K; ++k)
                if (!keep[k]) {
                    wi[kc] += std::fabs(wi[k]);
                    wi[k] = 0.0;
                }
            diag[i] = wi[kc];
        }
        // compact the pattern to the kept entries (row weights keep their order)
        {
            double dint = wint[kc];
            for (int k = 0; k < K; ++k)
                if (!keep[k]) dint += std::fabs(wint[k]);
            int Kn = 0;
            std::vector<int> nk(K, -1);
            for (int k = 0; k < K; ++k)
                if (keep[k]) {
                    nk[k] = Kn;
                    r.kd[l][Kn] = r.kd[l][k];
                    r.wint[l][Kn] = (float)(k == kc ? dint : wint[k]);
                    ++Kn;
                }
            for (int i = 0; i < A.n; ++i) {
                double *wi = &w[(size_t)i * K];
                for (int k = 0; k < K; ++k)
                    if (nk[k] >= 0) wi[nk[k]] = wi[k];   // nk[k] <= k: in place, ascending
            }
            for (int k = Kn; k < K; ++k) r.kd[l][k] = 0, r.wint[l][k] = 0.f;
            K = Kn;
            r.K[l] = K;
        }
        const int Kw = (int)keep.size();   // row stride of w
        std::vector<int> order;
        for (int pass = 1; pass >= 0; --pass)
            for (int i = 0; i < A.n; ++i)
                if (interior[i] == pass) order.push_back(i);   // i ascending: box-offset order within a part
        int n_int = 0;
        for (int i = 0; i < A.n; ++i) n_int += interior[i];
        const int n_exp = A.n - n_int;
        r.n_int[l] = n_int;
        r.n_exp[l] = n_exp;
        std::vector<int32_t> pts(A.n);
        r.dinv[l].resize(A.n);
        r.wexp[l].assign((size_t)K * n_exp, 0.f);
        r.dbox[l].assign((size_t)r.box[l], 0.f);
        for (int q = 0; q < A.n; ++q) {
            const int i = order[q];
            pts[q] = r.pts[l][i];
            r.dinv[l][q] = (float)(omega / diag[i]);
            r.dbox[l][(size_t)pts[q]] = r.dinv[l][q];
            if (q >= n_int)
                for (int k = 0; k < K; ++k) r.wexp[l][(size_t)k * n_exp + (q - n_int)] = (float)w[(size_t)i * Kw + k];
        }
        r.pts[l] = std::move(pts);
        // dense interior stencil, window -> pattern map, and runs of 4 points
        std::fill(r.kmap[l], r.kmap[l] + 125, -1);
        for (int k = 0; k < K; ++k) {
            const int kd = r.kd[l][k];
            const int pos = ((kd & 7) * 5 + ((kd >> 3) & 7)) * 5 + ((kd >> 6) & 7);   // (dx, dy, dz) + 2
            r.wdense[l][pos] = r.wint[l][k];
            r.kmap[l][pos] = k;
        }
        r.nrow[l] = 0;
        for (int dxy = 0; dxy < 25; ++dxy) {
            bool any = false;
            for (int dz = 0; dz < 5; ++dz) any |= r.kmap[l][dxy * 5 + dz] >= 0;
            if (any) r.rows[l][r.nrow[l]++] = dxy;
        }
        std::vector<int32_t> at((size_t)r.box[l], -1);
        for (int q = 0; q < A.n; ++q) at[(size_t)r.pts[l][q]] = q;
        const long long rows = (long long)r.Bp[l][0] * r.Bp[l][1];
        std::vector<int32_t> mixed_g, mixed_e;
        for (long long row = 0; row < rows; ++row)
            for (int g4 = 0; g4 < r.Bp[l][2] / 4; ++g4) {
                const long long off = row * r.Bp[l][2] + 4 * g4;
                int mask = 0, e4[4] = {-1, -1, -1, -1};
                bool pure = true;
                for (int i = 0; i < 4; ++i) {
                    const int q = at[(size_t)(off + i)];
                    if (q < 0) continue;
                    mask |= 1 << i;
                    if (q >= n_int) {
                        pure = false;
                        e4[i] = q - n_int;
                    }
                }
                if (!mask) continue;
                std::vector<int32_t> &G = pure ? r.groups[l] : mixed_g;
                std::vector<int32_t> &E = pure ? r.gexp[l] : mixed_e;
                G.push_back((int32_t)((off >> 2) << 4 | mask));
                for (int i = 0; i < 4; ++i) E.push_back(e4[i]);
            }
        r.n_pure[l] = (int)r.groups[l].size();
        r.groups[l].insert(r.groups[l].end(), mixed_g.begin(), mixed_g.end());
        r.gexp[l].insert(r.gexp[l].end(), mixed_e.begin(), mixed_e.end());
        const size_t nm = mixed_g.size();
        r.wmix[l].assign(125 * nm * 4, 0.f);
        for (size_t g = 0; g < nm; ++g)
            for (int pos = 0; pos < 125; ++pos) {
                const int k = r.kmap[l][pos];
                if (k < 0) continue;
                for (int i = 0; i < 4; ++i) {
                    if (!(mixed_g[g] & (1 << i))) continue;
                    const int e = mixed_e[4 * g + i];
                    r.wmix[l][((size_t)pos * nm + g) * 4 + i] =
                        e < 0 ? r.wdense[l][pos] : r.wexp[l][(size_t)k * n_exp + e];
                }
            }
    }
    // prolongation of level 1 onto the fine groups
    if (nl >= 2) {
        r.pinfo.resize(L.groups.size());
        for (size_t g = 0; g < L.groups.size(); ++g) {
            int u[3];
            coords(L.B, (long long)(L.groups[g] >> 4) << 2, u);
            const long long base = (((long long)(u[0] >> 1) + kMgPad) * r.Bp[1][1] + (u[1] >> 1) + kMgPad) * r.Bp[1][2] +
                                   (u[2] >> 1) + kMgPad;
            if (base >= (1LL << 29)) return EXX_ERR_ARG;
            r.pinfo[g] = (int32_t)(base << 2 | (u[0] & 1) << 1 | (u[1] & 1));
        }
    }
    if (nl >= 3) {
        r.pinfo1.resize(r.groups[1].size());
        for (size_t g = 0; g < r.groups[1].size(); ++g) {
            int u[3];
            coords(r.Bp[1], (long long)(r.groups[1][g] >> 4) << 2, u);
            for (int a = 0; a < 3; ++a) u[a] -= kMgPad;
            if (u[2] & 1) return EXX_ERR_ARG;   // runs start at an even coordinate (possibly -2, in the margin)
            const long long base =
                (((long long)(u[0] >> 1) + kMgPad) * r.Bp[2][1] + (u[1] >> 1) + kMgPad) * r.Bp[2][2] + (u[2] >> 1) + kMgPad;
            if (u[0] < 0 || u[1] < 0 || base >= (1LL << 29)) return EXX_ERR_ARG;
            r.pinfo1[g] = (int32_t)(base << 2 | (u[0] & 1) << 1 | (u[1] & 1));
        }
    }
    t = std::move(r);
    return EXX_OK;
}

int pick_schedule(const double *ms, int n)
{
    int best = -1;
    for (int k = 0; k < n; ++k)
        if (std::isfinite(ms[k]) && ms[k] < 1e299 && (best < 0 || ms[k] < ms[best])) best = k;
    return best;
}

std::vector<exx_schedule> schedule_candidates(bool mg, double omega_default)
{
    std::vector<exx_schedule> c;
    if (mg)
        for (float om : {0.8f, 0.7f, 0.6f})
            for (int sh : {14, 18}) c.push_back({EXX_PRECOND_MG, om, sh, 0.0});
    for (int sh : {14, 18}) c.push_back({EXX_PRECOND_NONE, (float)omega_default, sh, 0.0});
    return c;
}

void lpt_partition(const double *cost, int n, int n_ranks, int *owner)
{
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // min-heap of (load, rank): the least loaded rank, the lowest on ties
    std::vector<std::pair<double, int>> heap;
    for (int r = 0; r < n_ranks; ++r) heap.push_back({0.0, r});
    auto greater = [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
        return a.first > b.first || (a.first == b.first && a.second > b.second);
    };
    std::make_heap(heap.begin(), heap.end(), greater);
    for (int k : order) {
        std::pop_heap(heap.begin(), heap.end(), greater);
        owner[k] = heap.back().second;
        heap.back().first += cost[k];
        std::push_heap(heap.begin(), heap.end(), greater);
    }
}

}  // namespace exx
