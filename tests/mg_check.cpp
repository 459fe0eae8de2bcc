// Test harness (host only): the multigrid hierarchy of make_mg_levels on a
// benchmark cell, used as a V(1,1) preconditioner of CG on the PE Poisson
// problem with zero Dirichlet data, against plain CG.  Prints one JSON line.
//   usage: mg_check a b c n R_PE R_ME   (cell rows a, b, c: lattice scale and
//   the two shear terms of the cells used by the benchmarks)
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.h"

using namespace exx;
using Vec = std::vector<double>;

static void spmv(const MgLevel &A, const Vec &x, Vec &y)
{
    y.assign(A.n, 0.0);
    for (int i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int k = A.row[i]; k < A.row[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
        y[i] = s;
    }
}
static double dot(const Vec &a, const Vec &b)
{
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

// trilinear prolongation of level l + 1 onto level l, and its transpose
static void box_coords(const int *B, long long o, int *u)
{
    u[2] = (int)(o % B[2]);
    u[1] = (int)((o / B[2]) % B[1]);
    u[0] = (int)(o / ((long long)B[1] * B[2]));
}
static void transfer(const MgLevel &f, const MgLevel &c, const Vec &in, Vec &out, bool prolong)
{
    out.assign(prolong ? f.n : c.n, 0.0);
    for (int i = 0; i < f.n; ++i) {
        int u[3];
        box_coords(f.B, f.pts[i], u);
        int cc[3][2], np[3];
        double ww[3][2];
        for (int a = 0; a < 3; ++a) {
            cc[a][0] = u[a] >> 1;
            if (u[a] & 1) {
                cc[a][1] = (u[a] >> 1) + 1;
                ww[a][0] = ww[a][1] = 0.5;
                np[a] = 2;
            } else {
                ww[a][0] = 1.0;
                np[a] = 1;
            }
        }
        for (int x = 0; x < np[0]; ++x)
            for (int y = 0; y < np[1]; ++y)
                for (int z = 0; z < np[2]; ++z) {
                    const int j = c.idx[((size_t)cc[0][x] * c.B[1] + cc[1][y]) * c.B[2] + cc[2][z]];
                    if (j < 0) continue;   // a parent that is not a coarse point
                    const double w = ww[0][x] * ww[1][y] * ww[2][z];
                    if (prolong) out[i] += w * in[j];
                    else out[j] += w * in[i];
                }
    }
}

struct Mg {
    std::vector<MgLevel> lv;
    std::vector<double> chol;   // dense Cholesky factor of the coarsest operator
    int nc = 0;
    double omega = 0.7;

    void factor()
    {
        const MgLevel &A = lv.back();
        nc = A.n;
        chol.assign((size_t)nc * nc, 0.0);
        for (int i = 0; i < nc; ++i)
            for (int k = A.row[i]; k < A.row[i + 1]; ++k) chol[(size_t)i * nc + A.col[k]] = A.val[k];
        for (int j = 0; j < nc; ++j) {
            double d = chol[(size_t)j * nc + j];
            for (int k = 0; k < j; ++k) d -= chol[(size_t)j * nc + k] * chol[(size_t)j * nc + k];
            d = std::sqrt(d);
            chol[(size_t)j * nc + j] = d;
            for (int i = j + 1; i < nc; ++i) {
                double s = chol[(size_t)i * nc + j];
                for (int k = 0; k < j; ++k) s -= chol[(size_t)i * nc + k] * chol[(size_t)j * nc + k];
                chol[(size_t)i * nc + j] = s / d;
            }
        }
    }
    void coarse_solve(const Vec &b, Vec &x) const
    {
        x = b;
        for (int i = 0; i < nc; ++i) {
            for (int k = 0; k < i; ++k) x[i] -= chol[(size_t)i * nc + k] * x[k];
            x[i] /= chol[(size_t)i * nc + i];
        }
        for (int i = nc - 1; i >= 0; --i) {
            for (int k = i + 1; k < nc; ++k) x[i] -= chol[(size_t)k * nc + i] * x[k];
            x[i] /= chol[(size_t)i * nc + i];
        }
    }
    void apply_pre(const Vec &r, Vec &z) const { vcycle(0, r, z); }
    void vcycle(size_t l, const Vec &r, Vec &x) const
    {
        if (l + 1 == lv.size()) {
            coarse_solve(r, x);
            return;
        }
        const MgLevel &A = lv[l];
        Vec dinv(A.n), t;
        for (int i = 0; i < A.n; ++i)
            for (int k = A.row[i]; k < A.row[i + 1]; ++k)
                if (A.col[k] == i) dinv[i] = omega / A.val[k];
        x.assign(A.n, 0.0);
        for (int i = 0; i < A.n; ++i) x[i] = dinv[i] * r[i];   // one Jacobi sweep from zero
        spmv(A, x, t);
        for (int i = 0; i < A.n; ++i) t[i] = r[i] - t[i];
        Vec rc, xc, px;
        transfer(A, lv[l + 1], t, rc, false);
        vcycle(l + 1, rc, xc);
        transfer(A, lv[l + 1], xc, px, true);
        for (int i = 0; i < A.n; ++i) x[i] += px[i];
        spmv(A, x, t);
        for (int i = 0; i < A.n; ++i) x[i] += dinv[i] * (r[i] - t[i]);
    }
};

// The same V(1,1) cycle computed from the device tables (make_mg_tables), in
// FP32 on padded dense boxes, the way the pair solver applies it: level 0 is
// the CSR fine operator on the fine box, coarse rows take the interior stencil
// or their explicit weights, the coarsest level its inverse.
struct MgT {
    const MgTables *T;
    const MgLevel *fine;       // level 0 (box and active points)
    float c0;                  // omega / diag of the fine operator

    static void unpack(int kd, int *d)
    {
        d[0] = (kd & 7) - 2;
        d[1] = ((kd >> 3) & 7) - 2;
        d[2] = ((kd >> 6) & 7) - 2;
    }
    // y = A_l x on the active points of coarse level l (boxes)
    void apply(int l, const std::vector<float> &x, std::vector<float> &y) const
    {
        const MgTables &t = *T;
        y.assign(t.box[l], 0.f);
        for (int i = 0; i < t.n[l]; ++i) {
            const int o = t.pts[l][i];
            const int e = i - t.n_int[l];   // explicit rows follow the interior ones
            float s = 0.f;
            for (int k = 0; k < t.K[l]; ++k) {
                int d[3];
                unpack(t.kd[l][k], d);
                const float w = e < 0 ? t.wint[l][k] : t.wexp[l][(size_t)k * t.n_exp[l] + e];
                s += w * x[o + (d[0] * t.Bp[l][1] + d[1]) * t.Bp[l][2] + d[2]];
            }
            y[o] = s;
        }
    }
    // coordinates of level l's box element o (without the margin), and the inverse
    void coords(int l, long long o, int *u) const
    {
        const int *B = l == 0 ? fine->B : T->Bp[l];
        u[2] = (int)(o % B[2]);
        u[1] = (int)((o / B[2]) % B[1]);
        u[0] = (int)(o / ((long long)B[1] * B[2]));
        if (l > 0)
            for (int a = 0; a < 3; ++a) u[a] -= kMgPad;
    }
    long long offset(int l, const int *u) const
    {
        const int *B = l == 0 ? fine->B : T->Bp[l];
        const int p = l == 0 ? 0 : kMgPad;
        return (((long long)u[0] + p) * B[1] + u[1] + p) * B[2] + u[2] + p;
    }
    // coarse point c of level l+1 gathers level-l box values at 2c + delta
    void restrict_to(int l, const std::vector<float> &fb, std::vector<float> &cb) const
    {
        cb.assign(T->box[l + 1], 0.f);
        for (int i = 0; i < T->n[l + 1]; ++i) {
            int c[3];
            coords(l + 1, T->pts[l + 1][i], c);
            float s = 0.f;
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        const int u[3] = {2 * c[0] + dx, 2 * c[1] + dy, 2 * c[2] + dz};
                        const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
                        s += w * fb[offset(l, u)];
                    }
            cb[T->pts[l + 1][i]] = s;
        }
    }
    // value of the prolongation of level l+1's box at level-l point u
    float prolong_at(int l, const std::vector<float> &cb, const int *u) const
    {
        int cc[3][2], np[3];
        float ww[3][2];
        for (int a = 0; a < 3; ++a) {
            cc[a][0] = u[a] >> 1;
            if (u[a] & 1) {
                cc[a][1] = (u[a] >> 1) + 1;
                ww[a][0] = ww[a][1] = 0.5f;
                np[a] = 2;
            } else {
                ww[a][0] = 1.f;
                np[a] = 1;
            }
        }
        float s = 0.f;
        for (int x = 0; x < np[0]; ++x)
            for (int y = 0; y < np[1]; ++y)
                for (int z = 0; z < np[2]; ++z) {
                    const int c[3] = {cc[0][x], cc[1][y], cc[2][z]};
                    s += ww[0][x] * ww[1][y] * ww[2][z] * cb[offset(l + 1, c)];
                }
        return s;
    }
    // z_l = M_l r_l on coarse level l (boxes)
    void cycle(int l, const std::vector<float> &r, std::vector<float> &z) const
    {
        const MgTables &t = *T;
        z.assign(t.box[l], 0.f);
        if (l == t.nlev - 1) {
            const int n = t.n[l];
            for (int i = 0; i < n; ++i) {
                float s = 0.f;
                for (int j = 0; j < n; ++j) s += t.cinv[(size_t)i * n + j] * r[t.pts[l][j]];
                z[t.pts[l][i]] = s;
            }
            return;
        }
        // level 1 skips the pre-smoothing (as the solver does): R_1 is restricted as is
        if (l > 1)
            for (int i = 0; i < t.n[l]; ++i) z[t.pts[l][i]] = t.dinv[l][i] * r[t.pts[l][i]];
        std::vector<float> y, tb(t.box[l], 0.f), rc, zc;
        apply(l, z, y);
        for (int i = 0; i < t.n[l]; ++i) tb[t.pts[l][i]] = r[t.pts[l][i]] - y[t.pts[l][i]];
        restrict_to(l, tb, rc);
        cycle(l + 1, rc, zc);
        for (int i = 0; i < t.n[l]; ++i) {
            int u[3];
            coords(l, t.pts[l][i], u);
            z[t.pts[l][i]] += prolong_at(l, zc, u);
        }
        apply(l, z, y);
        for (int i = 0; i < t.n[l]; ++i) z[t.pts[l][i]] += t.dinv[l][i] * (r[t.pts[l][i]] - y[t.pts[l][i]]);
    }
    void apply_pre(const Vec &r, Vec &z) const { vcycle(r, z); }
    // z = M r on the fine level (compressed vectors in the fine point order)
    void vcycle(const Vec &r, Vec &z) const
    {
        const MgLevel &A = *fine;
        const size_t fbox = (size_t)A.B[0] * A.B[1] * A.B[2];
        Vec ar;
        spmv(A, r, ar);
        std::vector<float> tb(fbox, 0.f), rc, zc;
        for (int i = 0; i < A.n; ++i) tb[A.pts[i]] = (float)r[i] - c0 * (float)ar[i];
        restrict_to(0, tb, rc);
        cycle(1, rc, zc);
        Vec z0(A.n), az;
        for (int i = 0; i < A.n; ++i) {
            int u[3];
            coords(0, A.pts[i], u);
            z0[i] = c0 * (float)r[i] + prolong_at(0, zc, u);
        }
        spmv(A, z0, az);
        z.resize(A.n);
        for (int i = 0; i < A.n; ++i) z[i] = (float)(z0[i] + c0 * (float)(r[i] - az[i]));
    }
};

template <class Pre>
static int pcg(const MgLevel &A, const Vec &b, const Pre *M, double tol, Vec &x)
{
    const int n = A.n;
    x.assign(n, 0.0);
    Vec r = b, z, p, q;
    if (M) M->apply_pre(r, z);
    else z = r;
    p = z;
    double rz = dot(r, z);
    const double bn = std::sqrt(dot(b, b));
    for (int it = 1; it <= 5000; ++it) {
        spmv(A, p, q);
        const double a = rz / dot(p, q);
        for (int i = 0; i < n; ++i) {
            x[i] += a * p[i];
            r[i] -= a * q[i];
        }
        if (std::sqrt(dot(r, r)) <= tol * bn) return it;
        if (M) M->apply_pre(r, z);
        else z = r;
        const double rz2 = dot(r, z);
        for (int i = 0; i < n; ++i) p[i] = z[i] + (rz2 / rz) * p[i];
        rz = rz2;
    }
    return -1;
}

int main(int argc, char **argv)
{
    if (argc < 7) return 2;
    const double scale = std::atof(argv[1]), s1 = std::atof(argv[2]), s2 = std::atof(argv[3]);
    const int ng = std::atoi(argv[4]);
    const double rpe = std::atof(argv[5]), rme = std::atof(argv[6]);
    const double lat[3][3] = {{scale, 0, 0}, {s1 * scale, scale, 0}, {s2 * scale, -s2 * 1.6 * scale, scale}};
    const int n[3] = {ng, ng, ng};
    Metric m;
    Stencil st;
    OffsetSet o;
    SetLayout L;
    if (make_metric(lat, n, m) || make_stencil(m, 3, 15, nullptr, 0, st) || make_offsets(m, rpe, rme, o) ||
        make_layout(o, st, 3, L))
        return 3;
    Mg mg;
    if (make_mg_levels(L, st, 3, 600, mg.lv)) return 4;
    mg.factor();
    const MgLevel &A = mg.lv[0];
    // symmetry of every level's operator
    double asym = 0.0, amax = 0.0;
    for (const MgLevel &Al : mg.lv)
        for (int i = 0; i < Al.n; ++i)
            for (int k = Al.row[i]; k < Al.row[i + 1]; ++k) {
                const int j = Al.col[k];
                double aji = 0.0;
                for (int kk = Al.row[j]; kk < Al.row[j + 1]; ++kk)
                    if (Al.col[kk] == i) aji = Al.val[kk];
                asym = std::fmax(asym, std::fabs(Al.val[k] - aji));
                amax = std::fmax(amax, std::fabs(Al.val[k]));
            }
    // right-hand side: 4 pi times a distinct-pair density (two offset Gaussians)
    Vec b(A.n);
    for (int i = 0; i < A.n; ++i) {
        int u[3];
        box_coords(A.B, A.pts[i], u);
        double r[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            for (int al = 0; al < 3; ++al) r[a] += m.h[a][al] * (double)(u[al] - L.c[al]) / n[al];
        const double g1 = std::exp(-((r[0] - 1.2) * (r[0] - 1.2) + r[1] * r[1] + r[2] * r[2]));
        const double g2 = std::exp(-((r[0] + 1.2) * (r[0] + 1.2) + r[1] * r[1] + r[2] * r[2])) * (r[1] + 0.3);
        b[i] = 4.0 * M_PI * g1 * g2;
    }
    Vec x0, x1;
    const int k0 = pcg<Mg>(A, b, nullptr, 1e-9, x0);
    const int k1 = pcg(A, b, &mg, 1e-9, x1);
    // the device tables of the same hierarchy, applied in FP32 as the solver does
    MgTables T;
    if (make_mg_tables(L, st, 3, 200, 0.8, 0.005, T)) return 5;
    int k2 = -1, n_exp1 = 0;
    double rel2 = 1.0, runs_rel = 1.0, rruns_rel = 1.0, pinfo_rel = 1.0, pinfo1_rel = 1.0;
    bool aligned = true, pinfo_even = true, coarse_spd = true;
    double coarse_asym = 0.0;
    int coarse_checked = 0;
    if (T.nlev >= 2) {
        std::vector<MgLevel> lv2;
        make_mg_levels(L, st, 3, 200, lv2);
        MgT mt{&T, &lv2[0], 0.f};
        for (int k = lv2[0].row[0]; k < lv2[0].row[1]; ++k)
            if (lv2[0].col[k] == 0) mt.c0 = (float)(0.8 / lv2[0].val[k]);
        Vec x2;
        k2 = pcg(A, b, &mt, 1e-9, x2);
        double d2 = 0.0, n2 = 0.0;
        for (int i = 0; i < A.n; ++i) {
            d2 += (x2[i] - x0[i]) * (x2[i] - x0[i]);
            n2 += x0[i] * x0[i];
        }
        rel2 = std::sqrt(d2 / n2);
        n_exp1 = T.n_exp[1];
        // the device operators of the coarse levels small enough for a dense test
        // (interior rows from wint, explicit rows from wexp, entries below the drop
        // threshold lumped into the diagonal): symmetric and positive definite
        for (int l = 1; l < T.nlev - 1; ++l) {
            const int nl = T.n[l];
            if (nl > 2500) continue;
            std::vector<int> at((size_t)T.box[l], -1);
            for (int q = 0; q < nl; ++q) at[(size_t)T.pts[l][q]] = q;
            std::vector<double> M((size_t)nl * nl, 0.0);
            for (int q = 0; q < nl; ++q)
                for (int k = 0; k < T.K[l]; ++k) {
                    const int kd = T.kd[l][k];
                    const long long o = T.pts[l][q] + ((long long)((kd & 7) - 2) * T.Bp[l][1] + (((kd >> 3) & 7) - 2)) *
                                                          T.Bp[l][2] + (((kd >> 6) & 7) - 2);
                    const int j = (o >= 0 && o < T.box[l]) ? at[(size_t)o] : -1;
                    const double w = q < T.n_int[l] ? T.wint[l][k] : T.wexp[l][(size_t)k * T.n_exp[l] + (q - T.n_int[l])];
                    if (j >= 0) M[(size_t)q * nl + j] += w;
                }
            double am = 0.0, mm = 0.0;
            for (int q = 0; q < nl; ++q)
                for (int j = 0; j < nl; ++j) {
                    am = std::fmax(am, std::fabs(M[(size_t)q * nl + j] - M[(size_t)j * nl + q]));
                    mm = std::fmax(mm, std::fabs(M[(size_t)q * nl + j]));
                }
            coarse_asym = std::fmax(coarse_asym, am / mm);
            // Cholesky of the symmetric part
            for (int c = 0; c < nl && coarse_spd; ++c) {
                double d = M[(size_t)c * nl + c];
                for (int k = 0; k < c; ++k) d -= M[(size_t)c * nl + k] * M[(size_t)c * nl + k];
                if (!(d > 0.0)) {
                    coarse_spd = false;
                    break;
                }
                d = std::sqrt(d);
                M[(size_t)c * nl + c] = d;
                for (int r = c + 1; r < nl; ++r) {
                    double v = 0.5 * (M[(size_t)r * nl + c] + M[(size_t)c * nl + r]);
                    for (int k = 0; k < c; ++k) v -= M[(size_t)r * nl + k] * M[(size_t)c * nl + k];
                    M[(size_t)r * nl + c] = v / d;
                }
            }
            ++coarse_checked;
        }
        // level 1 in the solver's run form: runs of 4 points, interior runs from the
        // dense window, the others from wmix, against the row form of apply()
        {
            std::vector<float> x(T.box[1], 0.f), y, yr(T.box[1], 0.f);
            unsigned st_ = 12345u;
            for (int i = 0; i < T.n[1]; ++i) {
                st_ = st_ * 1664525u + 1013904223u;
                x[T.pts[1][i]] = (float)((st_ >> 8) * (1.0 / 16777216.0) - 0.5);
            }
            mt.apply(1, x, y);
            const int B1 = T.Bp[1][1], B2 = T.Bp[1][2];
            const int ngr = (int)T.groups[1].size(), npure = T.n_pure[1], nm = ngr - npure;
            for (int g = 0; g < ngr; ++g) {
                const int off = (T.groups[1][g] >> 4) << 2, mask = T.groups[1][g] & 15;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                for (int dxy = 0; dxy < 25; ++dxy)
                    for (int dz = 0; dz < 5; ++dz) {
                        const int pos = dxy * 5 + dz;
                        if (T.kmap[1][pos] < 0) continue;
                        const long long row = off + (long long)((dxy / 5 - 2) * B1 + (dxy % 5 - 2)) * B2;
                        for (int i = 0; i < 4; ++i) {
                            const float w = g < npure ? T.wdense[1][pos]
                                                      : T.wmix[1][((size_t)pos * nm + (g - npure)) * 4 + i];
                            acc[i] += w * x[row + i + dz - 2];
                        }
                    }
                for (int i = 0; i < 4; ++i)
                    if (mask & (1 << i)) yr[off + i] = acc[i];
            }
            double dd = 0.0, nn = 0.0;
            for (int i = 0; i < T.n[1]; ++i) {
                const long long o = T.pts[1][i];
                dd = std::fmax(dd, std::fabs((double)yr[o] - (double)y[o]));
                nn = std::fmax(nn, std::fabs((double)y[o]));
            }
            runs_rel = dd / nn;
            // fine -> level 1 restriction by runs: three aligned groups of four fine values per row
            const size_t fbox = (size_t)lv2[0].B[0] * lv2[0].B[1] * lv2[0].B[2];
            std::vector<float> fb(fbox, 0.f), cb, cr(T.box[1], 0.f);
            for (int i = 0; i < lv2[0].n; ++i) {
                st_ = st_ * 1664525u + 1013904223u;
                fb[lv2[0].pts[i]] = (float)((st_ >> 8) * (1.0 / 16777216.0) - 0.5);
            }
            mt.restrict_to(0, fb, cb);
            const int F1 = lv2[0].B[1], F2 = lv2[0].B[2];
            for (int g = 0; g < ngr; ++g) {
                const int off = (T.groups[1][g] >> 4) << 2, mask = T.groups[1][g] & 15;
                int c[3];
                mt.coords(1, off, c);
                if ((2 * c[2]) % 4 != 0) aligned = false;
                for (int i = 0; i < 4; ++i) {
                    if (!(mask & (1 << i))) continue;
                    float s = 0.f;
                    for (int dx = -1; dx <= 1; ++dx)
                        for (int dy = -1; dy <= 1; ++dy) {
                            const long long row = ((long long)(2 * c[0] + dx) * F1 + (2 * c[1] + dy)) * F2 + 2 * c[2];
                            const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
                            s += w * (fb[row + 2 * i] + 0.5f * (fb[row + 2 * i - 1] + fb[row + 2 * i + 1]));
                        }
                    cr[off + i] = s;
                }
            }
            dd = nn = 0.0;
            for (int i = 0; i < T.n[1]; ++i) {
                const long long o = T.pts[1][i];
                dd = std::fmax(dd, std::fabs((double)cr[o] - (double)cb[o]));
                nn = std::fmax(nn, std::fabs((double)cb[o]));
            }
            rruns_rel = dd / nn;
            // pass D's prolongation of level 1 onto the fine groups from pinfo,
            // against the generic trilinear prolongation
            std::vector<float> zc(T.box[1], 0.f);
            for (int i = 0; i < T.n[1]; ++i) {
                st_ = st_ * 1664525u + 1013904223u;
                zc[T.pts[1][i]] = (float)((st_ >> 8) * (1.0 / 16777216.0) - 0.5);
            }
            if (T.pinfo.size() != L.groups.size()) pinfo_rel = 1.0;
            else {
                dd = nn = 0.0;
                const long long sx = (long long)T.Bp[1][1] * T.Bp[1][2], sy = T.Bp[1][2];
                for (size_t g = 0; g < L.groups.size(); ++g) {
                    const long long off = (long long)(L.groups[g] >> 4) << 2;
                    const int mask = L.groups[g] & 15;
                    const int pi = T.pinfo[g];
                    const bool ox = pi & 2, oy = pi & 1;
                    const long long b = pi >> 2;
                    if ((b & 1) || (sy & 1) || (sx & 1)) pinfo_even = false;   // float2 reads of the parents
                    float c[3];
                    for (int k = 0; k < 3; ++k) {
                        c[k] = zc[b + k];
                        if (oy) c[k] += zc[b + sy + k];
                        if (ox) c[k] += zc[b + sx + k];
                        if (ox && oy) c[k] += zc[b + sx + sy + k];
                    }
                    const float wxy = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
                    const float zv[4] = {wxy * c[0], wxy * 0.5f * (c[0] + c[1]), wxy * c[1], wxy * 0.5f * (c[1] + c[2])};
                    for (int i = 0; i < 4; ++i) {
                        if (!(mask & (1 << i))) continue;
                        int u[3];
                        mt.coords(0, off + i, u);
                        const double ref = mt.prolong_at(0, zc, u);
                        dd = std::fmax(dd, std::fabs((double)zv[i] - ref));
                        nn = std::fmax(nn, std::fabs(ref));
                    }
                }
                pinfo_rel = dd / nn;
            }
            // the level-2 -> level-1 prolongation by level-1 runs (pinfo1)
            if (T.nlev >= 3) {
                std::vector<float> z2(T.box[2], 0.f);
                for (int i = 0; i < T.n[2]; ++i) {
                    st_ = st_ * 1664525u + 1013904223u;
                    z2[T.pts[2][i]] = (float)((st_ >> 8) * (1.0 / 16777216.0) - 0.5);
                }
                if (T.pinfo1.size() != T.groups[1].size()) pinfo1_rel = 1.0;
                else {
                    dd = nn = 0.0;
                    const long long sx = (long long)T.Bp[2][1] * T.Bp[2][2], sy = T.Bp[2][2];
                    for (size_t g = 0; g < T.groups[1].size(); ++g) {
                        const long long off = (long long)(T.groups[1][g] >> 4) << 2;
                        const int mask = T.groups[1][g] & 15;
                        const int pi = T.pinfo1[g];
                        const bool ox = pi & 2, oy = pi & 1;
                        const long long b = pi >> 2;
                        float c[3];
                        for (int k = 0; k < 3; ++k) {
                            c[k] = z2[b + k];
                            if (oy) c[k] += z2[b + sy + k];
                            if (ox) c[k] += z2[b + sx + k];
                            if (ox && oy) c[k] += z2[b + sx + sy + k];
                        }
                        const float wxy = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
                        const float zv[4] = {wxy * c[0], wxy * 0.5f * (c[0] + c[1]), wxy * c[1],
                                             wxy * 0.5f * (c[1] + c[2])};
                        for (int i = 0; i < 4; ++i) {
                            if (!(mask & (1 << i))) continue;
                            int u[3];
                            mt.coords(1, off + i, u);
                            const double ref = mt.prolong_at(1, z2, u);
                            dd = std::fmax(dd, std::fabs((double)zv[i] - ref));
                            nn = std::fmax(nn, std::fabs(ref));
                        }
                    }
                    pinfo1_rel = dd / nn;
                }
            }
        }
    }
    double d = 0.0, nx = 0.0;
    for (int i = 0; i < A.n; ++i) {
        d += (x1[i] - x0[i]) * (x1[i] - x0[i]);
        nx += x0[i] * x0[i];
    }
    int maxnnz = 0;
    for (int i = 0; i < mg.lv[1].n; ++i) maxnnz = std::max(maxnnz, mg.lv[1].row[i + 1] - mg.lv[1].row[i]);
    std::printf("{\"levels\": [");
    for (size_t l = 0; l < mg.lv.size(); ++l) std::printf("%s%d", l ? ", " : "", mg.lv[l].n);
    std::printf("], \"n_stcl\": %d, \"cg_iter\": %d, \"pcg_iter\": %d, \"rel_diff\": %.3e, \"asym\": %.3e, "
                "\"level1_max_nnz\": %d, \"tables_levels\": %d, \"tables_pcg_iter\": %d, "
                "\"tables_rel_diff\": %.3e, \"tables_level1_explicit\": %d, \"tables_level1_n\": %d, "
                "\"runs_rel_diff\": %.3e, \"restrict_runs_rel_diff\": %.3e, \"restrict_runs_aligned\": %d, "
                "\"prolong_groups_rel_diff\": %.3e, \"prolong_runs1_rel_diff\": %.3e, \"pinfo_even\": %d, "
                "\"coarse_checked\": %d, \"coarse_spd\": %d, \"coarse_asym\": %.3e}\n",
                2 * 3 * st.ndir + 1, k0, k1, std::sqrt(d / nx), asym / amax, maxnnz, T.nlev, k2, rel2, n_exp1, T.n[1],
                runs_rel, rruns_rel, aligned ? 1 : 0, pinfo_rel, pinfo1_rel, pinfo_even ? 1 : 0, coarse_checked,
                coarse_spd ? 1 : 0, coarse_asym);
    return 0;
}
