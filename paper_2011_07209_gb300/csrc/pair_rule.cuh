// pair_rule.cuh -- the written rule of the unique pair list (library-internal),
// shared by the solve's pair-list kernel and the allocation-free entry point so
// that both lists agree bit for bit.
//
// For i <= j (Sec. III A, Step II; Eq. l2g): s = h^-1 C (row sums left to
// right, no FMA); ds = s_j - s_i - round(ds); the lattice image k in
// {-1,0,1}^3 with the smallest |h(ds+k)|^2 (first in lexicographic k on ties),
// kept when that is <= R_pair^2.  Grid-resolved centre
// g = NINT(N (s_i + (ds + k)/2)) mod N, NINT rounding half away from zero
// (round()).  Every product and sum is an explicit round-to-nearest intrinsic,
// so nothing is contracted and the operation order is the one the oracle uses.
#pragma once

namespace exx {

__device__ __forceinline__ double pair_dot3_rn(const double *r, double a, double b, double c)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(r[0], a), __dmul_rn(r[1], b)), __dmul_rn(r[2], c));
}

// Cell: any structure with double h[3][3], hinv[3][3], r_pair2, int n[3] and
// const double *centres ([n_orb][3] Cartesian, device memory).
template <class Cell>
__device__ __forceinline__ bool pair_rule(const Cell &C, int i, int j, int *kb, int *g)
{
    const double *ci = C.centres + 3 * i, *cj = C.centres + 3 * j;
    double si[3], ds[3];
    for (int al = 0; al < 3; ++al) {
        si[al] = pair_dot3_rn(C.hinv[al], ci[0], ci[1], ci[2]);
        const double sj = pair_dot3_rn(C.hinv[al], cj[0], cj[1], cj[2]);
        const double d = __dadd_rn(sj, -si[al]);
        ds[al] = __dadd_rn(d, -round(d));
    }
    double best = 1.0 / 0.0;
    kb[0] = kb[1] = kb[2] = 0;
    for (int k0 = -1; k0 <= 1; ++k0)
        for (int k1 = -1; k1 <= 1; ++k1)
            for (int k2 = -1; k2 <= 1; ++k2) {
                const double t0 = __dadd_rn(ds[0], (double)k0), t1 = __dadd_rn(ds[1], (double)k1),
                             t2 = __dadd_rn(ds[2], (double)k2);
                const double d0 = pair_dot3_rn(C.h[0], t0, t1, t2);
                const double d1 = pair_dot3_rn(C.h[1], t0, t1, t2);
                const double d2 = pair_dot3_rn(C.h[2], t0, t1, t2);
                const double dd = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
                if (dd < best) {
                    best = dd;
                    kb[0] = k0;
                    kb[1] = k1;
                    kb[2] = k2;
                }
            }
    if (!(best <= C.r_pair2)) return false;
    for (int al = 0; al < 3; ++al) {
        const double sm = __dadd_rn(si[al], __dmul_rn(__dadd_rn(ds[al], (double)kb[al]), 0.5));
        const long long gg = (long long)round(__dmul_rn((double)C.n[al], sm));
        long long r = gg % C.n[al];
        if (r < 0) r += C.n[al];
        g[al] = (int)r;
    }
    return true;
}

}  // namespace exx
