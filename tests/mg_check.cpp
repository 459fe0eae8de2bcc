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

static int pcg(const MgLevel &A, const Vec &b, const Mg *M, double tol, Vec &x)
{
    const int n = A.n;
    x.assign(n, 0.0);
    Vec r = b, z, p, q;
    if (M) M->vcycle(0, r, z);
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
        if (M) M->vcycle(0, r, z);
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
    const int k0 = pcg(A, b, nullptr, 1e-9, x0);
    const int k1 = pcg(A, b, &mg, 1e-9, x1);
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
                "\"level1_max_nnz\": %d}\n",
                2 * 3 * st.ndir + 1, k0, k1, std::sqrt(d / nx), asym / amax, maxnnz);
    return 0;
}
