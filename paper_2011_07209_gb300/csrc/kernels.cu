// kernels.cu -- CUDA kernels of the EXX pair path for sm_103a.
//
//   k_tables       regular solid harmonics on PE points and far-field kernels
//                  on shell points of one subdomain kind (Eqs. me, mepole)
//   k_pair_rows    unique pair list, one CTA per orbital row (Step II)
//   k_pair_scan    row offsets and per-cell ranges of the pair list
//   k_pair_solve   persistent: one CTA owns one pair at a time and runs the
//                  whole per-pair path (Steps III-V): pair density, moments,
//                  far field, Poisson CG with the NK stencil, E / sigma
//                  integrals and the D scatter
//   k_finalize     ordered per-cell sums of E_xx, sigma and Pi
#include <cuda_runtime.h>
#include <cstdint>

#include <algorithm>
#include <type_traits>

#include "exx_dev.h"
#include "kernels.h"
#include "pair_rule.cuh"

namespace exx {

#ifndef EXX_UNROLL
#define EXX_UNROLL 4
#endif

constexpr double kFourPi = 12.566370614359172953850573533118;

__device__ __forceinline__ void unpack_m(int32_t p, int &m0, int &m1, int &m2)
{
    m0 = ((p >> 20) & 1023) - 512;
    m1 = ((p >> 10) & 1023) - 512;
    m2 = (p & 1023) - 512;
}

__device__ __forceinline__ int wrapi(int a, int n)
{
    // within one period of [0, n) (grid offsets inside the cell) without a division
    if (a >= n) a -= n;
    else if (a < 0) a += n;
    if ((unsigned)a < (unsigned)n) return a;
    const int r = a % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// Real solid harmonics r^l Y_lm from the Cartesian recurrences
//   (x + i y)^m = A_m + i B_m,
//   Q_m^m = (2m-1)!!,  Q_{m+1}^m = (2m+1) z Q_m^m,
//   (l - m) Q_l^m = (2l-1) z Q_{l-1}^m - (l+m-1) r^2 Q_{l-2}^m,
//   r^l Y_l0 = N_l0 Q_l^0,  r^l Y_{l,+-m} = sqrt2 N_lm Q_l^m {A_m, B_m},
// N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), index l^2 + l + m.
// ---------------------------------------------------------------------------
__device__ void solid_harmonics(int lmax, double x, double y, double z, double *S)
{
    double A[7], B[7];
    A[0] = 1.0;
    B[0] = 0.0;
    for (int m = 1; m <= lmax; ++m) {
        A[m] = x * A[m - 1] - y * B[m - 1];
        B[m] = x * B[m - 1] + y * A[m - 1];
    }
    const double r2 = x * x + y * y + z * z;
    double Q[7][7];
    double dfact = 1.0;
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) dfact *= (2.0 * m - 1.0);
        Q[m][m] = dfact;
        if (m + 1 <= lmax) Q[m + 1][m] = (2.0 * m + 1.0) * z * dfact;
        for (int l = m + 2; l <= lmax; ++l)
            Q[l][m] = ((2.0 * l - 1.0) * z * Q[l - 1][m] - (l + m - 1.0) * r2 * Q[l - 2][m]) / (double)(l - m);
    }
    for (int l = 0; l <= lmax; ++l) {
        for (int m = 0; m <= l; ++m) {
            double ratio = 1.0;   // (l-m)!/(l+m)!
            for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
            const double nlm = sqrt((2.0 * l + 1.0) / kFourPi * ratio);
            if (m == 0) {
                S[l * l + l] = nlm * Q[l][0];
            } else {
                const double c = 1.4142135623730951 * nlm * Q[l][m];
                S[l * l + l + m] = c * A[m];
                S[l * l + l - m] = c * B[m];
            }
        }
    }
    for (int k = (lmax + 1) * (lmax + 1); k < kNlm; ++k) S[k] = 0.0;
}

__global__ void k_tables(const CellDev *__restrict__ cell, int which, double *S64, float *S32, double *T64,
                         float *T32)
{
    const CellDev &C = *cell;
    const SetDev &st = C.set[which];
    const int total = st.n_pe + st.n_shell;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int m0, m1, m2;
        if (q < st.n_pe) unpack_m(st.pe_m[q], m0, m1, m2);
        else unpack_m(st.sh_m[q - st.n_pe], m0, m1, m2);
        const double s0 = (double)m0 / C.n[0], s1 = (double)m1 / C.n[1], s2 = (double)m2 / C.n[2];
        const double x = C.h[0][0] * s0 + C.h[0][1] * s1 + C.h[0][2] * s2;
        const double y = C.h[1][0] * s0 + C.h[1][1] * s1 + C.h[1][2] * s2;
        const double z = C.h[2][0] * s0 + C.h[2][1] * s1 + C.h[2][2] * s2;
        double S[kNlm];
        solid_harmonics(C.lmax, x, y, z, S);
        if (q < st.n_pe) {
            for (int k = 0; k < kNlm; ++k) {
                S64[(size_t)q * kNlm + k] = S[k];
                S32[(size_t)q * kNlm + k] = (float)S[k];
            }
        } else {
            const int s = q - st.n_pe;
            const double r = sqrt(x * x + y * y + z * z);
            double rpow = r;          // r^(2l+1)
            for (int l = 0; l < 7; ++l) {
                const double f = (l <= C.lmax) ? kFourPi / ((2.0 * l + 1.0) * rpow) : 0.0;
                for (int mm = -l; mm <= l; ++mm) {
                    const double t = f * S[l * l + l + mm];
                    T64[(size_t)(l * l + l + mm) * st.n_shell + s] = t;
                    T32[(size_t)(l * l + l + mm) * st.n_shell + s] = (float)t;
                }
                rpow *= r * r;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Pair list: the rule of pair_rule.cuh, one CTA per orbital row.
// ---------------------------------------------------------------------------
// One CTA of kRowThreads per orbital row (cell, i).  fill = 0: count; 1: write.
__global__ void __launch_bounds__(kRowThreads) k_pair_rows(const CellDev *__restrict__ cells, int n_cells,
                                                          ListDev L, int fill)
{
    const int row = blockIdx.x;
    int c = 0;
    while (c + 1 < n_cells && row >= cells[c + 1].row_base) ++c;
    const CellDev &C = cells[c];
    const int i = row - C.row_base;
    if (i >= C.n_orb) return;
    __shared__ int warp_tot[kRowThreads / 32];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = fill ? L.row_start[row] : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j0 = i; j0 < C.n_orb; j0 += kRowThreads) {
        const int j = j0 + threadIdx.x;
        int kb[3], g[3];
        const bool ok = (j < C.n_orb) && pair_rule(C, i, j, kb, g);
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
        for (int k = 0; k < kRowThreads / 32; ++k) {
            if (k < w) before += warp_tot[k];
            tot += warp_tot[k];
        }
        if (fill && ok) {
            const int pos = s_base + before + __popc(bal & ((1u << lane) - 1u));
            if (pos < L.capacity) {
                PairRec pr;
                pr.i = i;
                pr.j = j;
                pr.k[0] = kb[0];
                pr.k[1] = kb[1];
                pr.k[2] = kb[2];
                pr.g[0] = g[0];
                pr.g[1] = g[1];
                pr.g[2] = g[2];
                pr.cell = c;
                pr.pad = 0;
                L.pairs[pos] = pr;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (!fill && threadIdx.x == 0) L.row_count[row] = s_base;
}

// Exclusive scan of the row counts (single CTA), per-cell ranges, capacity check.
__global__ void __launch_bounds__(1024) k_pair_scan(const CellDev *__restrict__ cells, int n_cells, int n_rows,
                                                   ListDev L)
{
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_rows; base += 1024) {
        const int r = base + threadIdx.x;
        const int v = r < n_rows ? L.row_count[r] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (r < n_rows) L.row_start[r] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int total = carry;
        for (int c = 0; c < n_cells; ++c) {
            const int r0 = cells[c].row_base;
            const int r1 = r0 + cells[c].n_orb;
            L.cell_start[c] = r0 < n_rows ? L.row_start[r0] : total;
            L.cell_count[c] = (r1 < n_rows ? L.row_start[r1] : total) - L.cell_start[c];
        }
        *L.overflow = total > L.capacity ? 1 : 0;
        *L.total = total > L.capacity ? 0 : total;
        *L.queue = 0;
    }
}

// ---------------------------------------------------------------------------
// Block reductions (fixed tree: deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum K values over the CTA; every thread receives the totals.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = warp_sum(v[k]);
        if (lane == 0) red[w * K + k] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? red[lane * K + k] : 0.0;
            t = warp_sum(t);
            if (lane == 0) red[32 * K + k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[32 * K + k];
}

// Exact-product, double-float accumulation of FP32 dot products: the running
// sum is hi + lo; each product a*b is split exactly as p + pe by an FMA and
// added with TwoSum, so per-thread partial sums carry ~48 significant bits.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_fma(DF &acc, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fadd_rn(s, -acc.hi);
    const float err = __fadd_rn(__fadd_rn(acc.hi, -__fadd_rn(s, -bb)), __fadd_rn(p, -bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, pe));
}
__device__ __forceinline__ double df_val(const DF &a) { return (double)a.hi + (double)a.lo; }
// TwoSum of a float into the double-float accumulator.
__device__ __forceinline__ void df_add(DF &acc, float x)
{
    const float s = __fadd_rn(acc.hi, x);
    const float bb = __fadd_rn(s, -acc.hi);
    const float err = __fadd_rn(__fadd_rn(acc.hi, -__fadd_rn(s, -bb)), __fadd_rn(x, -bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, err);
}

// Sum of two double-float values (TwoSum on the high parts).
__device__ __forceinline__ DF df_sum(DF a, DF b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fadd_rn(s, -a.hi);
    const float err = __fadd_rn(__fadd_rn(a.hi, -__fadd_rn(s, -bb)), __fadd_rn(b.hi, -bb));
    return {s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}

// Sum K double-float values over the CTA in FP32 arithmetic; the totals end up
// in every lane of warp 0 (the scalar work that follows runs there, so the
// SM's FP64 pipe is not loaded by a thousand redundant copies of it).
template <int K>
__device__ __forceinline__ void block_sum_df(DF (&v)[K], float2 *red2)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const DF t = {__shfl_xor_sync(0xffffffffu, v[k].hi, o), __shfl_xor_sync(0xffffffffu, v[k].lo, o)};
            v[k] = df_sum(v[k], t);
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red2[w * K + k] = make_float2(v[k].hi, v[k].lo);
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 t = lane < nw ? red2[lane * K + k] : make_float2(0.f, 0.f);
            v[k] = {t.x, t.y};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const DF u = {__shfl_xor_sync(0xffffffffu, v[k].hi, o), __shfl_xor_sync(0xffffffffu, v[k].lo, o)};
                v[k] = df_sum(v[k], u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Orbital access.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double phi_at(const CellDev &C, int o, int g0, int g1, int g2)
{
    const int32_t *lo = C.box_lo + 3 * o;
    const int u0 = wrapi(g0 - lo[0], C.n[0]);
    const int u1 = wrapi(g1 - lo[1], C.n[1]);
    const int u2 = wrapi(g2 - lo[2], C.n[2]);
    if (u0 >= C.box[0] || u1 >= C.box[1] || u2 >= C.box[2]) return 0.0;
    return __ldg(C.phi + (((size_t)o * C.box[0] + u0) * C.box[1] + u1) * C.box[2] + u2);
}

// D^o(g) += val, with the D-box membership check.  Returns false when a
// non-zero value falls outside the box.
__device__ __forceinline__ bool d_add(const CellDev &C, int o, int g0, int g1, int g2, double val)
{
    const int32_t *lo = C.dbox_lo + 3 * o;
    const int u0 = wrapi(g0 - lo[0], C.n[0]);
    const int u1 = wrapi(g1 - lo[1], C.n[1]);
    const int u2 = wrapi(g2 - lo[2], C.n[2]);
    if (u0 >= C.dbox[0] || u1 >= C.dbox[1] || u2 >= C.dbox[2]) return val == 0.0;
    atomicAdd(C.dxx + (((size_t)o * C.dbox[0] + u0) * C.dbox[1] + u1) * C.dbox[2] + u2, val);
    return true;
}

// ---------------------------------------------------------------------------
// Stencil:  (L f)(off) = sum_d sum_{s=-n..n} cw[d][|s|] f(off + s stride_d).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T lap_at(const T *__restrict__ f, int off, const T (*cw)[8], const int *ds, int ndir,
                                    int n, T center)
{
    T acc = center * f[off];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (d < ndir) {
            const int st = ds[d];
#pragma unroll
            for (int s = 1; s <= 6; ++s)
                if (s <= n) acc += cw[d][s] * (f[off + s * st] + f[off - s * st]);
        }
    }
    return acc;
}

// r = 4 pi rho + L v on PE (v: x on PE, far field on the halo); returns sum r^2.
__device__ double residual_pass(const SetDev &S, const double *__restrict__ vbox, const double *__restrict__ rho,
                                double *__restrict__ r64, const double (*cw)[8], const int *ds, int ndir, int n,
                                double center, double *red)
{
    double acc[1] = {0.0};
    for (int k = threadIdx.x; k < S.n_pe; k += blockDim.x) {
        const int off = S.pe_off[k];
        const double r = kFourPi * rho[k] + lap_at<double>(vbox, off, cw, ds, ndir, n, center);
        r64[k] = r;
        acc[0] += r * r;
    }
    block_sum<1>(acc, red);
    return acc[0];
}

// ---------------------------------------------------------------------------
// Normalised double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2,
// 48 significant bits from FP32 operations (GB300 runs FP64 at 1/64 of the FP32
// rate).  Knuth's TwoSum, Dekker's FastTwoSum and the FMA TwoProd are exact;
// the sum and product below are the accurate double-word algorithms of
// Joldes, Muller and Popescu (2017), relative error a few 2^-48.  Round-to-
// nearest intrinsics throughout, so that no step is contracted into an FMA.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    return make_float2(s, __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb)));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b)   // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fadd_rn(b, -__fadd_rn(s, -a)));
}
__device__ __forceinline__ float2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return make_float2(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ float2 dw_add(float2 x, float2 y)
{
    const float2 s = two_sum(x.x, y.x), t = two_sum(x.y, y.y);
    const float2 v = fast_two_sum(s.x, __fadd_rn(s.y, t.x));
    return fast_two_sum(v.x, __fadd_rn(t.y, v.y));
}
__device__ __forceinline__ float2 dw_add_f(float2 x, float y)   // double-float + float
{
    const float2 s = two_sum(x.x, y);
    return fast_two_sum(s.x, __fadd_rn(x.y, s.y));
}
__device__ __forceinline__ float2 dw_mul(float2 x, float2 y)
{
    const float ph = __fmul_rn(x.x, y.x);
    float pl = __fmaf_rn(x.x, y.x, -ph);
    pl = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, pl));
    return fast_two_sum(ph, pl);
}
__device__ __forceinline__ float2 dw_split(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// Running sum of products of double-float pairs: s is the FP32 sum of the
// leading products w.hi x.hi, c (FP32) collects their exact rounding errors
// (TwoSum, and the FMA error of each product) and the cross terms w.hi x.lo +
// w.lo x.hi.  Error a few 2^-46 of the sum of the terms' magnitudes, in about a
// third of the operations of renormalised double-float arithmetic.
struct DfSum {
    float s, c;
    __device__ __forceinline__ void add_prod(float2 w, float2 x)
    {
        const float p = __fmul_rn(w.x, x.x);
        const float e = __fmaf_rn(w.x, x.x, -p);
        const float2 t = two_sum(s, p);
        s = t.x;
        c = __fadd_rn(c, __fadd_rn(__fadd_rn(t.y, e), __fmaf_rn(w.x, x.y, __fmul_rn(w.y, x.x))));
    }
    __device__ __forceinline__ void add(float2 x)
    {
        const float2 t = two_sum(s, x.x);
        s = t.x;
        c = __fadd_rn(c, __fadd_rn(t.y, x.y));
    }
};
// a + b of two double-float pairs as an unnormalised pair: the high parts'
// exact sum, the low parts added in FP32
__device__ __forceinline__ float2 pair_sum(float2 a, float2 b)
{
    const float2 t = two_sum(a.x, b.x);
    return make_float2(t.x, __fadd_rn(__fadd_rn(t.y, a.y), b.y));
}

// r = 4 pi rho + L v on PE in double-float arithmetic: v as (hi, lo) pairs in
// the dense box, 4 pi rho as pairs per PE point, stencil weights as pairs, the
// terms summed by DfSum.  The error is a few 2^-46 of the sum of the magnitudes
// of the stencil terms (FP64: 2^-53), far below the CG tolerance times |b|.  r
// is stored rounded to FP32, the precision of the inner solve it restarts;
// returns sum r^2 (per thread in double-float, over the CTA in FP64).
template <int FDN>
__device__ __noinline__ double residual_df(const SetDev &S, const float2 *__restrict__ vb, const float2 *__restrict__ b2,
                                           float *__restrict__ r32, const float2 (*cw)[8], float2 center,
                                           const int *ds, int ndir, double *red)
{
    DF a2 = {0.f, 0.f};
    for (int k = threadIdx.x; k < S.n_pe; k += blockDim.x) {
        const int off = S.pe_off[k];
        DfSum a = {0.f, 0.f};
        a.add_prod(center, vb[off]);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            if (d < ndir) {
                const int st = ds[d];
#pragma unroll
                for (int s_ = 1; s_ <= FDN; ++s_) a.add_prod(cw[d][s_], pair_sum(vb[off + s_ * st], vb[off - s_ * st]));
            }
        }
        a.add(b2[k]);
        const float r = __fadd_rn(a.s, a.c);
        r32[k] = r;
        df_fma(a2, r, r);
    }
    double acc[1] = {(double)a2.hi + (double)a2.lo};
    block_sum<1>(acc, red);
    return acc[0];
}
__device__ __forceinline__ double residual_df_n(int fdn, const SetDev &S, const float2 *vb, const float2 *b2,
                                                float *r32, const float2 (*cw)[8], float2 center, const int *ds,
                                                int ndir, double *red)
{
    switch (fdn) {
    case 1: return residual_df<1>(S, vb, b2, r32, cw, center, ds, ndir, red);
    case 2: return residual_df<2>(S, vb, b2, r32, cw, center, ds, ndir, red);
    case 3: return residual_df<3>(S, vb, b2, r32, cw, center, ds, ndir, red);
    default: return residual_df<4>(S, vb, b2, r32, cw, center, ds, ndir, red);
    }
}

// Step V integrals of one pair from the double-float solution (v as hi/lo
// pairs in the box, 4 pi rho as pairs): sum rho v and sum m_alpha rho d_b v,
// d_b v the central first difference along lattice axis b (weights w1).  Every
// product and sum in double-float; in thread 0, out[0] = sum rho v and
// out[1 + 3 b + alpha] = sum m_alpha rho d_b v (no dV).
__device__ __noinline__ void energy_stress_df(const SetDev &S, const float2 (*w1)[8], const float2 *__restrict__ vb,
                                              const float2 *__restrict__ b2, bool want_sigma, int fdn, float2 *red2,
                                              double *out)
{
    DF acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = {0.f, 0.f};
#pragma unroll 2
    for (int k = threadIdx.x; k < S.n_pe; k += blockDim.x) {
        const int off = S.pe_off[k];
        const float2 b = b2[k];
        const float2 e = dw_mul(b, vb[off]);
        acc[0] = df_sum(acc[0], {e.x, e.y});
        if (!want_sigma) continue;
        int m0, m1, m2;
        unpack_m(S.pe_m[k], m0, m1, m2);
        const float mf[3] = {(float)m0, (float)m1, (float)m2};
        // the derivative in FP32 from the differences of the double-float values (hi
        // and lo parts differenced separately): sigma needs about 1e-5 relative (its
        // tolerance 1e-8 Ha/bohr^3 against |Pi| ~ 1e-3), FP32 gives about 1e-7; only
        // the products with rho and the sums stay double-float
#pragma unroll
        for (int db = 0; db < 3; ++db) {
            const int st = S.gstride[db];
            float d_ = 0.f;
#pragma unroll
            for (int s_ = 1; s_ <= 4; ++s_) {
                if (s_ <= fdn) {
                    const float2 vp = vb[off + s_ * st], vm = vb[off - s_ * st];
                    d_ += w1[db][s_].x * ((vp.x - vm.x) + (vp.y - vm.y));
                }
            }
            const float2 rd = dw_mul(b, make_float2(d_, 0.f));   // 4 pi rho d_b v
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                const float2 p = two_prod(mf[al], rd.x);   // m_alpha is an integer below 2^10: exact
                acc[1 + 3 * db + al] = df_sum(acc[1 + 3 * db + al], {p.x, __fmaf_rn(mf[al], rd.y, p.y)});
            }
        }
    }
    block_sum_df<10>(acc, red2);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 10; ++k) out[k] = ((double)acc[k].hi + (double)acc[k].lo) / kFourPi;
}

// The double-float residual of residual_df and, from the same loads, the Step V
// sums of energy_stress_df (the stencil's first three directions are the lattice
// axes, so v at +-s along each axis is already at hand).  Taken for the residual
// that is expected to end the CG: when it does, the separate Step V pass is not
// needed.  Returns sum r^2 in every thread; es_out (thread 0) as energy_stress_df.
template <int FDN>
__device__ __noinline__ double residual_es_df(const SetDev &S, const float2 *__restrict__ vb,
                                              const float2 *__restrict__ b2, float *__restrict__ r32,
                                              const float2 (*cw)[8], float2 center, const int *ds, int ndir,
                                              double *red, const float2 (*w1)[8], bool want_sigma, double *es_out)
{
    DF a2 = {0.f, 0.f};
    DF acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = {0.f, 0.f};
    for (int k = threadIdx.x; k < S.n_pe; k += blockDim.x) {
        const int off = S.pe_off[k];
        const float2 v0 = vb[off];
        DfSum a = {0.f, 0.f};
        a.add_prod(center, v0);
        float dd[3] = {0.f, 0.f, 0.f};   // first differences along the lattice axes (energy_stress_df)
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            if (d < ndir) {
                const int st = ds[d];
#pragma unroll
                for (int s_ = 1; s_ <= FDN; ++s_) {
                    const float2 vp = vb[off + s_ * st], vm = vb[off - s_ * st];
                    a.add_prod(cw[d][s_], pair_sum(vp, vm));
                    if (d < 3) dd[d] += w1[d][s_].x * ((vp.x - vm.x) + (vp.y - vm.y));
                }
            }
        }
        const float2 b = b2[k];
        a.add(b);
        const float r = __fadd_rn(a.s, a.c);
        r32[k] = r;
        df_fma(a2, r, r);
        const float2 e = dw_mul(b, v0);
        acc[0] = df_sum(acc[0], {e.x, e.y});
        if (want_sigma) {
            int m0, m1, m2;
            unpack_m(S.pe_m[k], m0, m1, m2);
            const float mf[3] = {(float)m0, (float)m1, (float)m2};
#pragma unroll
            for (int db = 0; db < 3; ++db) {
                const float2 rd = dw_mul(b, make_float2(dd[db], 0.f));
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const float2 p = two_prod(mf[al], rd.x);
                    acc[1 + 3 * db + al] = df_sum(acc[1 + 3 * db + al], {p.x, __fmaf_rn(mf[al], rd.y, p.y)});
                }
            }
        }
    }
    double rr[1] = {(double)a2.hi + (double)a2.lo};
    block_sum<1>(rr, red);
    block_sum_df<10>(acc, reinterpret_cast<float2 *>(red));
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 10; ++k) es_out[k] = ((double)acc[k].hi + (double)acc[k].lo) / kFourPi;
    __syncthreads();
    return rr[0];
}
__device__ __forceinline__ double residual_es_df_n(int fdn, const SetDev &S, const float2 *vb, const float2 *b2,
                                                   float *r32, const float2 (*cw)[8], float2 center, const int *ds,
                                                   int ndir, double *red, const float2 (*w1)[8], bool want_sigma,
                                                   double *es_out)
{
    switch (fdn) {
    case 1: return residual_es_df<1>(S, vb, b2, r32, cw, center, ds, ndir, red, w1, want_sigma, es_out);
    case 2: return residual_es_df<2>(S, vb, b2, r32, cw, center, ds, ndir, red, w1, want_sigma, es_out);
    case 3: return residual_es_df<3>(S, vb, b2, r32, cw, center, ds, ndir, red, w1, want_sigma, es_out);
    default: return residual_es_df<4>(S, vb, b2, r32, cw, center, ds, ndir, red, w1, want_sigma, es_out);
    }
}

// x * sc in FP32 for any FP64 scale sc (sc = m 2^e, x m rounded once, then an
// exact power-of-two scaling), so that tiny residuals reach the O(1) frame.
struct F32Scale {
    float m;
    int e;
    __device__ float apply(float x) const { return ldexpf(__fmul_rn(x, m), e); }
};
__device__ __forceinline__ F32Scale f32_scale(double sc)
{
    int e;
    const double m = frexp(sc, &e);
    return {(float)m, e};
}

struct SlotWork {
    char *base;
    size_t slot_bytes;
    size_t off_vbox, off_pbox, off_rho, off_r64, off_r, off_q, off_e, off_gs, off_b2, off_zf, off_mg;
};

// Shared per-CTA state.
struct SmemCell {
    CellDev C;
    double cw64[6][8];
    float cw32[6][8];
    float2 cwdf[6][8];   // cw64 as double-float pairs
    float2 centerdf;
    float cn[kNlm];      // N_l0 at l^2 + l, sqrt2 N_lm at l^2 + l + m (m > 0)
    float hf[3][3];      // h[a][b] / N_b: Cartesian position of a grid offset, FP32
    float Qc[kNlm];      // 4 pi / (2l+1) Q_lm of the current pair, FP32
    float2 cq2[kNlm];    // at l^2 + l + m (m >= 0): cn Qc of (l, m) and of (l, -m), for solid_parts32
    float2 w1df[3][8];   // first-derivative weights w1dx as double-float pairs
    double Q[kNlm];
    float Qf[kNlm];
    double center64;
    float center32;
    int ds[6];
};

// The mixed-precision Poisson solve of one pair (see the comment inside).
struct CgMixed {
    const SetDev *S;
    double *vbox;
    const double *rho;
    double *r64;
    float *pf, *rf, *qf, *ef;
    const SmemCell *sm;
    double *red;
    int ndir, fdn, max_iter;
    double stop, bn, inner_red;
    double r0n;   // norm of the starting residual b - A v0 (the first frame)
    const float2 *b2;   // 4 pi rho as double-float pairs (one-sweep path)
};

__device__ __noinline__ void cg_mixed(const CgMixed &cg, int &iters, int &refine, int &status, double &rnorm)
{
    const SetDev &S = *cg.S;
    const SmemCell &sm = *cg.sm;
    double *__restrict__ vbox = cg.vbox;
    const double *__restrict__ rho = cg.rho;
    double *__restrict__ r64 = cg.r64;
    double *red = cg.red;
    const int ndir = cg.ndir, fdn = cg.fdn;
    const double stop = cg.stop, bn = cg.bn, inner_red = cg.inner_red;
    const int tid = threadIdx.x, nt = blockDim.x;
    struct {
        int max_iter;
    } C = {cg.max_iter};
            // Mixed: FP32 CG with reliable updates.  The FP32 vectors live in a frame
            // scaled by S (the true residual norm at the last update), so they stay O(1)
            // however small the pair density is.  The FP32 correction e accumulates
            // alpha p; when the recursive residual has dropped by inner_red since the
            // last update (or reaches the target), x += S e in FP64, the true residual
            // b - A x is recomputed in FP64 and replaces r, and the search direction is
            // carried over into the new frame.
            float *__restrict__ pf = cg.pf;
            float *__restrict__ rf = cg.rf;
            float *__restrict__ qf = cg.qf;
            float *__restrict__ ef = cg.ef;
            const int32_t *__restrict__ poff = S.pe_off;
            const int npe = S.n_pe;
            constexpr int U = EXX_UNROLL;
            if (bn > 0.0 && cg.r0n > stop) {
                double S_ = cg.r0n;
                double rr;
                {
                    double a0[1];
                    DF a = {0.f, 0.f};
                    const double sc = 1.0 / S_;
                    for (int k = tid; k < npe; k += nt) {
                        const float r = (float)(r64[k] * sc);
                        rf[k] = r;
                        ef[k] = 0.f;
                        pf[poff[k]] = r;
                        df_fma(a, r, r);
                    }
                    a0[0] = df_val(a);
                    block_sum<1>(a0, red);
                    rr = a0[0];
                }
                double rmax = sqrt(rr);
                for (;;) {
                    if (iters >= C.max_iter) {
                        status = 5;
                        break;
                    }
                    // pass A: q = A p, <p, q>
                    double pq[1];
                    {
                        DF a = {0.f, 0.f};
                        for (int kb = tid; kb < npe; kb += U * nt) {
                            int off[U];
                            float q[U], pc[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const int k = kb + u * nt;
                                off[u] = k < npe ? __ldg(poff + k) : -1;
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                if (off[u] >= 0) {
                                    pc[u] = pf[off[u]];
                                    q[u] = -lap_at<float>(pf, off[u], sm.cw32, sm.ds, ndir, fdn, sm.center32);
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                if (off[u] >= 0) {
                                    qf[kb + u * nt] = q[u];
                                    df_fma(a, pc[u], q[u]);
                                }
                            }
                        }
                        pq[0] = df_val(a);
                    }
                    block_sum<1>(pq, red);
                    const float alpha = (float)(rr / pq[0]);
                    // pass B: r -= alpha q, <r, r>
                    double rn[1];
                    {
                        DF a = {0.f, 0.f};
                        for (int kb = tid; kb < npe; kb += U * nt) {
                            float rv_[U], qv_[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const int k = kb + u * nt;
                                if (k < npe) {
                                    rv_[u] = rf[k];
                                    qv_[u] = qf[k];
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const int k = kb + u * nt;
                                if (k < npe) {
                                    const float r = rv_[u] - alpha * qv_[u];
                                    rf[k] = r;
                                    df_fma(a, r, r);
                                }
                            }
                        }
                        rn[0] = df_val(a);
                    }
                    block_sum<1>(rn, red);
                    ++iters;
                    const double rnrm = sqrt(rn[0]);
                    if (rnrm <= inner_red * rmax || rnrm * S_ <= 0.5 * stop || !(rnrm == rnrm)) {
                        // reliable update in FP64: x += S (e + alpha p)
                        for (int k = tid; k < npe; k += nt) {
                            const int off = poff[k];
                            vbox[off] += ((double)ef[k] + (double)alpha * (double)pf[off]) * S_;
                            ef[k] = 0.f;
                        }
                        __syncthreads();
                        rnorm = sqrt(residual_pass(S, vbox, rho, r64, sm.cw64, sm.ds, ndir, fdn, sm.center64, red));
                        ++refine;
                        if (rnorm <= stop) break;
                        // beta from the replaced residual, direction moved to the new frame
                        const double Snew = rnorm;
                        const float bscaled = (float)((rnorm / S_) * (rnorm / S_) / rr * (S_ / Snew));
                        const double sc = 1.0 / Snew;
                        double a0[1];
                        DF a = {0.f, 0.f};
                        for (int k = tid; k < npe; k += nt) {
                            const int off = poff[k];
                            const float r = (float)(r64[k] * sc);
                            rf[k] = r;
                            pf[off] = r + bscaled * pf[off];
                            df_fma(a, r, r);
                        }
                        a0[0] = df_val(a);
                        block_sum<1>(a0, red);
                        rr = a0[0];
                        rmax = sqrt(rr);
                        S_ = Snew;
                        continue;
                    }
                    // pass C: e += alpha p, p = r + beta p
                    const float beta = (float)(rn[0] / rr);
                    rr = rn[0];
                    for (int kb = tid; kb < npe; kb += U * nt) {
                        int off[U];
                        float pv_[U], rv_[U], ev_[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int k = kb + u * nt;
                            off[u] = k < npe ? __ldg(poff + k) : -1;
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int k = kb + u * nt;
                            if (off[u] >= 0) {
                                pv_[u] = pf[off[u]];
                                rv_[u] = rf[k];
                                ev_[u] = ef[k];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int k = kb + u * nt;
                            if (off[u] >= 0) {
                                ef[k] = ev_[u] + alpha * pv_[u];
                                pf[off[u]] = rv_[u] + beta * pv_[u];
                            }
                        }
                    }
                    __syncthreads();
                }
            }
}


__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
#ifndef EXX_STREAM_HINTS
#define EXX_STREAM_HINTS 0
#endif
__device__ __forceinline__ float4 ld4s(const float *p)
{
#if EXX_STREAM_HINTS
    return __ldcs(reinterpret_cast<const float4 *>(p));
#else
    return ld4(p);
#endif
}
__device__ __forceinline__ void st4s(float *p, float a, float b, float c, float d)
{
#if EXX_STREAM_HINTS
    __stcs(reinterpret_cast<float4 *>(p), make_float4(a, b, c, d));
#else
    st4(p, a, b, c, d);
#endif
}

// (L f) at the four points off .. off+3 of one aligned group (off a multiple of
// 4) into acc; returns f there.  The contiguous axis (d == 2) comes from the
// group and its two neighbours.  A direction with no step along the contiguous
// axis moves by rs[d], a multiple of 4, and reads whole groups.  A direction
// with a step d2[d] = +-1 along it lands s_ d2[d] points off the group
// boundary at the s_-th neighbour: the two aligned groups around that point
// hold all four values, picked by compile-time indices (the sign of d2[d] is
// the same for every thread).  Each group read holds at least one of the
// values needed, so no read leaves the box.  Longer steps along the contiguous
// axis read point by point.
template <int FDN>
__device__ __forceinline__ float4 lap4(const float *__restrict__ x_, int off, const float (*cw)[8], float center,
                                       const int *rs, const int *d2, int ndir, float (&acc)[4])
{
    const float4 c = ld4(x_ + off);
    const float4 cm = ld4(x_ + off - 4);
    const float4 cp = ld4(x_ + off + 4);
    const float x[12] = {cm.x, cm.y, cm.z, cm.w, c.x, c.y, c.z, c.w, cp.x, cp.y, cp.z, cp.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = center * x[4 + i];
#pragma unroll
    for (int s_ = 1; s_ <= FDN; ++s_)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += cw[2][s_] * (x[4 + i + s_] + x[4 + i - s_]);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (d == 2 || d >= ndir) continue;
        if (d2[d] == 0) {
#pragma unroll
            for (int s_ = 1; s_ <= FDN; ++s_) {
                const float4 a = ld4(x_ + off + s_ * rs[d]);
                const float4 b = ld4(x_ + off - s_ * rs[d]);
                acc[0] += cw[d][s_] * (a.x + b.x);
                acc[1] += cw[d][s_] * (a.y + b.y);
                acc[2] += cw[d][s_] * (a.z + b.z);
                acc[3] += cw[d][s_] * (a.w + b.w);
            }
        } else if (d2[d] == 1 || d2[d] == -1) {
            // f(off + i + s_ dsf) = f(bp + i + s_ d2) and f(off + i - s_ dsf) = f(bm + i - s_ d2)
            // with bp, bm = off +- s_ rs[d] on group boundaries
            const bool up = d2[d] > 0;
#pragma unroll
            for (int s_ = 1; s_ <= FDN; ++s_) {
                const int bp = off + s_ * rs[d], bm = off - s_ * rs[d];
                if (up) {
                    const float4 p0 = ld4(x_ + bp), p1 = ld4(x_ + bp + 4);   // bp .. bp+7
                    const float4 m0 = ld4(x_ + bm - 4), m1 = ld4(x_ + bm);   // bm-4 .. bm+3
                    const float P[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                    const float M[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[i] += cw[d][s_] * (P[i + s_] + M[4 + i - s_]);
                } else {
                    const float4 p0 = ld4(x_ + bp - 4), p1 = ld4(x_ + bp);   // bp-4 .. bp+3
                    const float4 m0 = ld4(x_ + bm), m1 = ld4(x_ + bm + 4);   // bm .. bm+7
                    const float P[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                    const float M[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[i] += cw[d][s_] * (P[4 + i - s_] + M[i + s_]);
                }
            }
        } else {
            // longer steps along the contiguous axis (auxiliary directions beyond the first shell)
            const int ds = rs[d] + d2[d];
#pragma unroll
            for (int s_ = 1; s_ <= FDN; ++s_)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] += cw[d][s_] * (x_[off + i + s_ * ds] + x_[off + i - s_ * ds]);
        }
    }
    return c;
}

// q = -(L p) on the PE lanes of one aligned group (zero on the others), stored,
// with the four products <p,q>, <q,q>, <r,q>, <r,p> of the group added to the
// double-float dot accumulators.
template <int FDN>
__device__ __forceinline__ void stencil_group(const float *__restrict__ pf, const float *__restrict__ rf,
                                              float *__restrict__ qf, int32_t gw, const float (*cw)[8], float center,
                                              const int *rs, const int *dsf, const int *d2, int ndir, DF &apq, DF &aqq,
                                              DF &arq, DF &arp)
{
    const int off = (gw >> 4) << 2;
    const int mask = gw & 15;
    float acc[4];
    const float4 c = lap4<FDN>(pf, off, cw, center, rs, d2, ndir, acc);
    const float q0 = (mask & 1) ? -acc[0] : 0.f, q1 = (mask & 2) ? -acc[1] : 0.f;
    const float q2 = (mask & 4) ? -acc[2] : 0.f, q3 = (mask & 8) ? -acc[3] : 0.f;
    st4s(qf + off, q0, q1, q2, q3);
    const float4 r = ld4s(rf + off);
    df_add(apq, c.x * q0 + c.y * q1 + c.z * q2 + c.w * q3);
    df_add(aqq, q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    df_add(arq, r.x * q0 + r.y * q1 + r.z * q2 + r.w * q3);
    df_add(arp, r.x * c.x + r.y * c.y + r.z * c.z + r.w * c.w);
}

// r -= alpha q, e += alpha p, p = r + beta p on one aligned group, with <r,r>
// of the updated residual added to a double-float accumulator.
__device__ __forceinline__ void update_group(float *__restrict__ rf, float *__restrict__ ef, float *__restrict__ pf,
                                             const float *__restrict__ qf, int off, float alpha, float beta, DF &arr)
{
    const float4 r = ld4(rf + off), q = ld4s(qf + off), p_ = ld4(pf + off), e = ld4s(ef + off);
    const float r0 = r.x - alpha * q.x, r1 = r.y - alpha * q.y, r2 = r.z - alpha * q.z, r3 = r.w - alpha * q.w;
    df_add(arr, r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    st4(rf + off, r0, r1, r2, r3);
    st4s(ef + off, e.x + alpha * p_.x, e.y + alpha * p_.y, e.z + alpha * p_.z, e.w + alpha * p_.w);
    st4(pf + off, r0 + beta * p_.x, r1 + beta * p_.y, r2 + beta * p_.z, r3 + beta * p_.w);
}

#ifndef EXX_SWEEP_GROUPS
#define EXX_SWEEP_GROUPS 8
#endif
constexpr int kSweepChunkGroups = EXX_SWEEP_GROUPS;   // groups per thread between two CTA barriers of the sweep
constexpr int kMaxSweepChunks = 512;   // chunks the one-sweep path can order

// Mixed-precision Poisson solve of one pair in ONE sweep over the vectors per
// iteration: FP32 CG in a frame scaled by the last true residual norm, with
// FP64 reliable updates, on the dense box of aligned 4-point groups.
//   * every FP32 vector (p, r, q, e) is a dense box, zero outside PE; the stencil
//     reads p with aligned float4 loads for the directions that do not step
//     along the last axis, a 12-wide register window for the last axis, and
//     scalar loads for auxiliary directions with a last-axis step;
//   * one reduction per iteration: the stencil sweep forms q = A p with <p,q>,
//     <q,q>, <r,q>, <r,p> (and <r,r> of the residual it has just updated); then
//     alpha = <r,p>/<p,q> (exact line search), the predicted
//     <r',r'> = <r,r> - 2 alpha <r,q> + alpha^2 <q,q> decides the FP64
//     replacement, and the Hestenes-Stiefel beta = -(<r,q> - alpha <q,q>)/<p,q>
//     keeps p' A-conjugate to p.  These forms stay exact when a replacement has
//     perturbed the Krylov relations; after one the new direction is
//     r' + gamma p with gamma chosen to keep it A-conjugate to the last one.
// The update r -= alpha q, e += alpha p, p = r + beta p of iteration k is not a pass of its
// own: it runs inside the stencil sweep of iteration k+1, ahead of it.  The
// groups are sorted by box offset, so the stencil of a chunk of groups reads p
// only up to a known group index (the chunk's last offset plus the stencil
// reach); the update front is kept past that index before the chunk's stencil
// runs, with one CTA barrier per chunk.  The stencil then reads p and r just
// written by the update (cache-resident), and every vector crosses HBM once
// per iteration: r, e, p, q read, r, e, p, q written.
// Inlined into the kernel: as a separate function its parameter block lives in
// local memory and is re-read inside the loop (measured 6 % slower).
// Scalars of a sweep-CG iteration, kept by thread 0 and broadcast through shared memory.
struct SweepScalars {
    double rr, rmax, S, pq;
    float alpha, beta;
    int act;   // 0 continue, 1 reliable update, 2 reliable update after a breakdown
};

// The reliable update of the sweep CG, out of line so that the registers of
// the sweep loop do not depend on it: v += (e + alpha p) S in double-float, the
// double-float true residual, and (unless it meets the tolerance) r restarted
// in the frame of its new norm with p = r + gamma p, gamma keeping p
// A-conjugate to the last direction (zero after a breakdown).  Returns true
// when the true residual meets the tolerance.
__device__ __noinline__ bool sweep_replace(const CgMixed &cg, SweepScalars &cs, float alpha, int act, double &rnorm)
{
    const SetDev &S = *cg.S;
    const SmemCell &sm = *cg.sm;
    float2 *vb = reinterpret_cast<float2 *>(cg.vbox);
    float *r32 = reinterpret_cast<float *>(cg.r64);
    float *__restrict__ pf = cg.pf;
    float *__restrict__ rf = cg.rf;
    const float *__restrict__ qf = cg.qf;
    float *__restrict__ ef = cg.ef;
    const int32_t *__restrict__ poff = S.pe_off;
    const int npe = S.n_pe, tid = threadIdx.x, nt = blockDim.x;
    const float2 S2 = dw_split(cs.S);
    for (int k = tid; k < npe; k += nt) {
        const int off = poff[k];
        const float2 t = dw_add_f(two_prod(alpha, pf[off]), ef[off]);
        vb[off] = dw_add(vb[off], dw_mul(t, S2));
        ef[off] = 0.f;
    }
    __syncthreads();
    rnorm = sqrt(residual_df_n(cg.fdn, S, vb, cg.b2, r32, sm.cwdf, sm.centerdf, sm.ds, cg.ndir, cg.red));
    if (rnorm <= cg.stop) return true;
    const F32Scale sc = f32_scale(1.0 / rnorm);
    DF ab[2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k = tid; k < npe; k += nt) {
        const int off = poff[k];
        const float r = sc.apply(r32[k]);
        rf[off] = r;
        df_fma(ab[0], r, r);
        df_fma(ab[1], r, qf[off]);
    }
    block_sum_df<2>(ab, reinterpret_cast<float2 *>(cg.red));
    if (tid == 0) {
        const double rr_ = (double)ab[0].hi + (double)ab[0].lo;
        const double rq_ = (double)ab[1].hi + (double)ab[1].lo;
        cs.beta = act == 2 ? 0.f : (float)(-rq_ / cs.pq);   // gamma of the carried direction
        cs.rr = rr_;
        cs.rmax = sqrt(rr_);
        cs.S = rnorm;
    }
    __syncthreads();
    const float gamma = cs.beta;
    for (int k = tid; k < npe; k += nt) {
        const int off = poff[k];
        pf[off] = rf[off] + gamma * pf[off];
    }
    __syncthreads();
    return false;
}

template <int FDN>
__device__ __forceinline__ void cg_mixed_sweep(const CgMixed &cg, int &iters, int &refine, int &status, double &rnorm)
{
    const SetDev &S = *cg.S;
    const SmemCell &sm = *cg.sm;
    const float *__restrict__ r32 = reinterpret_cast<const float *>(cg.r64);   // last true residual, FP32
    float *__restrict__ pf = cg.pf;
    float *__restrict__ rf = cg.rf;
    float *__restrict__ qf = cg.qf;
    float *__restrict__ ef = cg.ef;
    const int32_t *__restrict__ poff = S.pe_off;
    const int32_t *__restrict__ grp = S.groups;
    double *red = cg.red;
    const int npe = S.n_pe, ng = S.n_groups;
    const int ndir = cg.ndir;
    const double stop = cg.stop, inner_red = cg.inner_red;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (!(cg.bn > 0.0)) return;
    const int *rs = S.rstride, *dsf = S.dstride, *d2 = S.d2;
    const float(*cw)[8] = sm.cw32;
    const float center = sm.center32;

    // update front needed by each chunk: the number of groups whose offset is at
    // most the chunk's last offset plus the stencil reach
    __shared__ int s_need[kMaxSweepChunks];
    const int W = kSweepChunkGroups * nt;   // groups per chunk
    const int nchunk = (ng + W - 1) / W;
    {
        int reach = 7;
        for (int d = 0; d < ndir; ++d)
            reach = max(reach, 3 + FDN * max(abs(dsf[d]), abs(rs[d])));
        for (int c = tid; c < nchunk; c += nt) {
            const int last = min(ng, (c + 1) * W) - 1;
            const long long lim = (long long)((grp[last] >> 4) << 2) + reach;
            int lo = last + 1, hi = ng;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)((grp[mid] >> 4) << 2) <= lim) lo = mid + 1;
                else hi = mid;
            }
            s_need[c] = lo;
        }
    }

    if (!(cg.r0n > stop)) return;   // the starting guess already meets the tolerance
    double rr;
    {
        double a0[1];
        DF a = {0.f, 0.f};
        const F32Scale sc = f32_scale(1.0 / cg.r0n);
        for (int k = tid; k < npe; k += nt) {
            const int off = poff[k];
            const float r = sc.apply(r32[k]);
            rf[off] = r;
            ef[off] = 0.f;
            pf[off] = r;
            df_fma(a, r, r);
        }
        a0[0] = df_val(a);
        block_sum<1>(a0, red);
        rr = a0[0];
    }
    // scalars of the iteration, kept by thread 0 and broadcast through shared memory
    __shared__ SweepScalars cs;
    if (tid == 0) {
        cs.rr = rr;
        cs.rmax = sqrt(rr);
        cs.S = cg.r0n;
    }
    __syncthreads();
    float2 *red2 = reinterpret_cast<float2 *>(red);
    bool pending = false;          // an update (alpha_p, beta_p) waits for the next sweep
    float alpha_p = 0.f, beta_p = 0.f;
    for (;;) {
        if (iters >= cg.max_iter) {
            status = 5;
            break;
        }
        DF dv[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};   // <p,q> <q,q> <r,q> <r,p> <r,r>
        if (!pending) {
            for (int g = tid; g < ng; g += nt)
                stencil_group<FDN>(pf, rf, qf, __ldg(grp + g), cw, center, rs, dsf, d2, ndir, dv[0], dv[1], dv[2],
                                   dv[3]);
        } else {
            int front = 0;
            for (int c = 0; c < nchunk; ++c) {
                const int need = s_need[c];
                for (; front < need; front += nt) {
                    const int g = front + tid;
                    if (g < ng) update_group(rf, ef, pf, qf, (__ldg(grp + g) >> 4) << 2, alpha_p, beta_p, dv[4]);
                }
                __syncthreads();
                const int gend = min(ng, (c + 1) * W);
                for (int g = c * W + tid; g < gend; g += nt)
                    stencil_group<FDN>(pf, rf, qf, __ldg(grp + g), cw, center, rs, dsf, d2, ndir, dv[0], dv[1], dv[2],
                                       dv[3]);
            }
        }
        block_sum_df<5>(dv, red2);
        if (tid == 0) {
            double d[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) d[k] = (double)dv[k].hi + (double)dv[k].lo;
            const double rr_ = pending ? d[4] : cs.rr;
            const double alpha_d = d[3] / d[0];
            const double rn = rr_ - 2.0 * alpha_d * d[2] + alpha_d * alpha_d * d[1];
            const double rnrm = sqrt(fmax(rn, 0.0));
            const bool breakdown = !(d[0] > 0.0) || !(d[3] > 0.0) || !(alpha_d < 1e300);
            int act = 0;
            if (breakdown) act = 2;
            else if (!(rn > 0.0) || rnrm <= inner_red * cs.rmax || rnrm * cs.S <= 0.5 * stop) act = 1;
            cs.alpha = breakdown ? 0.f : (float)alpha_d;
            cs.beta = breakdown ? 0.f : (float)(-(d[2] - alpha_d * d[1]) / d[0]);
            cs.pq = d[0];
            cs.rr = rn;
            cs.act = act;
        }
        __syncthreads();
        const int act = cs.act;
        const float alpha = cs.alpha;
        pending = false;
        ++iters;
        if (act) {
            ++refine;
            if (sweep_replace(cg, cs, alpha, act, rnorm)) break;
            continue;
        }
        alpha_p = alpha;
        beta_p = cs.beta;
        pending = true;
    }
}


// ---------------------------------------------------------------------------
// Multigrid-preconditioned mixed CG (Step IV; the paper's CG is plain, this
// preconditioner changes the iterates only: the discrete equations of Eq. pe
// and the stopping rule |b - A v| <= tol |b| on the true residual stay the
// same).  FP32 preconditioned CG on A e = r in the frame of the last true
// residual, with the same reliable updates as the plain mixed CG: when the
// recursive residual has dropped by inner_red (or reaches the target), v += S e
// in double-float, the double-float true residual replaces r and the PCG
// restarts from it.  The preconditioner is one V(1,1) cycle: weighted Jacobi
// before and after the coarse correction, trilinear prolongation P and its
// transpose as restriction, Galerkin operators P^T A P on the coarse levels
// (built on the host per subdomain kind) and the inverse of the coarsest one.
// On the fine level the Jacobi weight omega / diag(A) is one constant c0 (the
// stencil's diagonal does not vary), so the pre-smoothed residual is
// r - c0 A r and needs no stored pre-smoothed vector.
// ---------------------------------------------------------------------------
struct MgSm {                      // the hierarchy of the pair's set, in shared memory
    int nlev;
    float c0;                      // omega / diag(A) of the fine level
    float dscale;                  // omega / (the tables' omega): scales the coarse dinv
    int n[kMgLevelsDev], K[kMgLevelsDev], Bp1[kMgLevelsDev], Bp2[kMgLevelsDev];
    int n_int[kMgLevelsDev], n_exp[kMgLevelsDev];
    float *R[kMgLevelsDev], *Z[kMgLevelsDev], *T[kMgLevelsDev];
    const int32_t *pts[kMgLevelsDev];
    const float *wexp[kMgLevelsDev], *dinv[kMgLevelsDev], *dbox[kMgLevelsDev];
    const float *cinv;
    const int32_t *pinfo, *pinfo1;
    int koff[kMgLevelsDev][kMgKDev];
    float wint[kMgLevelsDev][kMgKDev];
    int n_groups[kMgLevelsDev], n_pure[kMgLevelsDev];
    const int32_t *groups[kMgLevelsDev];
    const float4 *wmix[kMgLevelsDev];
    float wdense[125];             // the window weights and map of level 1 (the level of the run path)
    int kmap[125];
    int nrow1, rows1[25];          // level 1: (dx, dy) rows of the window with pattern entries
    float cr[kMgCoarsestDev];
};

// L x on the four lanes of one aligned group (the stencil of stencil_group).
template <int FDN>
__device__ __forceinline__ void lap_group(const float *__restrict__ x_, int off, const float (*cw)[8], float center,
                                          const int *rs, const int *dsf, const int *d2, int ndir, float (&acc)[4])
{
    (void)dsf;
    lap4<FDN>(x_, off, cw, center, rs, d2, ndir, acc);
}

__device__ __forceinline__ void mg_coords(int o, int B1, int B2, int &u0, int &u1, int &u2)
{
    u2 = o % B2;
    const int t = o / B2;
    u1 = t % B1;
    u0 = t / B1;
}

// R_{l+1} = P^T T_l on the active points of level l + 1: the values of level l
// at 2c + delta, weights 1 (delta = 0) and 1/2 per axis.  Level 0 reads the
// dense CG box (B1, B2, no margin), coarse levels their padded boxes.
__device__ __forceinline__ void mg_restrict(const MgSm &m, int l, const float *__restrict__ src, int B1, int B2,
                                            int pad)
{
    const int lc = l + 1;
    const int *pts = m.pts[lc];
    float *dst = m.R[lc];
    for (int i = threadIdx.x; i < m.n[lc]; i += blockDim.x) {
        const int o = pts[i];
        int c0, c1, c2;
        mg_coords(o, m.Bp1[lc], m.Bp2[lc], c0, c1, c2);
        c0 -= kMgPadDev;
        c1 -= kMgPadDev;
        c2 -= kMgPadDev;
        float s = 0.f;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const float *row = src + ((size_t)(2 * c0 + dx + pad) * B1 + (2 * c1 + dy + pad)) * B2 + 2 * c2 + pad;
                const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
                s += w * (row[0] + 0.5f * (row[-1] + row[1]));
            }
        dst[o] = s;
    }
}

// (P Z_{l+1}) at the level-l point with unpadded coordinates (u0, u1, u2).
__device__ __forceinline__ float mg_prolong_at(const MgSm &m, int l, int u0, int u1, int u2)
{
    const int lc = l + 1;
    const float *Zc = m.Z[lc];
    const int B1 = m.Bp1[lc], B2 = m.Bp2[lc];
    const int a0 = u0 >> 1, a1 = u1 >> 1, a2 = u2 >> 1;
    const int n0 = (u0 & 1) + 1, n1 = (u1 & 1) + 1;
    const float w0 = n0 == 2 ? 0.5f : 1.f, w1 = n1 == 2 ? 0.5f : 1.f;
    float s = 0.f;
    for (int x = 0; x < n0; ++x)
        for (int y = 0; y < n1; ++y) {
            const float *row = Zc + ((size_t)(a0 + x + kMgPadDev) * B1 + (a1 + y + kMgPadDev)) * B2 + a2 + kMgPadDev;
            s += (u2 & 1) ? 0.5f * (row[0] + row[1]) : row[0];
        }
    return w0 * w1 * s;
}

__shared__ MgSm g_mg_sm;          // one copy per kernel that uses the multigrid path

// Part of (A_l x) at active point i (box offset o) of coarse level l: the
// pattern entries k = sub, sub + tpr, ... (tpr threads share a row on the small
// levels).  U independent partial sums keep U weight and U value loads in
// flight (explicit rows read their weights from L2, pattern-major).
template <int U, class Wt>
__device__ __forceinline__ float mg_row_sum(int K, const int *koff, const float *__restrict__ x, int o, int sub, int tpr,
                                            Wt wt)
{
    float s[U];
#pragma unroll
    for (int j = 0; j < U; ++j) s[j] = 0.f;
    int k = sub;
    for (; k + (U - 1) * tpr < K; k += U * tpr) {
        float wv[U], xv[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            wv[j] = wt(k + j * tpr);
            xv[j] = x[o + koff[k + j * tpr]];
        }
#pragma unroll
        for (int j = 0; j < U; ++j) s[j] += wv[j] * xv[j];
    }
    for (; k < K; k += tpr) s[0] += wt(k) * x[o + koff[k]];
    float t = s[0];
#pragma unroll
    for (int j = 1; j < U; ++j) t += s[j];
    return t;
}
__device__ __forceinline__ float mg_row(int l, int i, int o, const float *__restrict__ x, int sub, int tpr)
{
    const MgSm &m = g_mg_sm;
    const int K = m.K[l];
    const int *koff = m.koff[l];
    const int e = i - m.n_int[l];
    if (e < 0) {
        const float *w = m.wint[l];
        return mg_row_sum<4>(K, koff, x, o, sub, tpr, [&](int k) { return w[k]; });
    }
    const int ne = m.n_exp[l];
    const float *__restrict__ w = m.wexp[l] + e;
    return mg_row_sum<6>(K, koff, x, o, sub, tpr, [&](int k) { return __ldg(w + (size_t)k * ne); });
}

// T = R - A_l X on coarse level 1, by runs of 4 points along the last axis:
// for each of the 25 (dx, dy) rows of the 5 x 5 x 5 window, three aligned float4
// loads give the 12 values that the run's four points need (the same loads
// serve all four), and the weights come from the interior stencil in shared
// memory or, for runs with rows of their own, one float4 per window position.
__device__ __noinline__ void mg_resid_runs(const float *__restrict__ R, const float *__restrict__ X,
                                              float *__restrict__ T, bool fold)
{
    const MgSm &m = g_mg_sm;
    const int l = 1;
    const int ng = m.n_groups[l], npure = m.n_pure[l];
    const int B1 = m.Bp1[l], B2 = m.Bp2[l], nrow = m.nrow1;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int32_t gw = __ldg(m.groups[l] + g);
        const int off = (gw >> 4) << 2, mask = gw & 15;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (g < npure) {
#pragma unroll 5
            for (int rw = 0; rw < nrow; ++rw) {
                const int dxy = m.rows1[rw];
                const float *row = X + off + ((dxy / 5 - 2) * B1 + (dxy % 5 - 2)) * B2;
                const float4 a = ld4(row - 4), b = ld4(row), c = ld4(row + 4);
                const float x[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
                for (int dz = 0; dz < 5; ++dz) {
                    const float w = m.wdense[dxy * 5 + dz];
                    if (w == 0.f) continue;
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[i] += w * x[2 + i + dz];
                }
            }
        } else {
            // one float4 of weights per window position for the run's four points
            const int nm = ng - npure;
            const float4 *__restrict__ wm = m.wmix[l] + (g - npure);
#pragma unroll 2
            for (int rw = 0; rw < nrow; ++rw) {
                const int dxy = m.rows1[rw];
                const float *row = X + off + ((dxy / 5 - 2) * B1 + (dxy % 5 - 2)) * B2;
                const float4 a = ld4(row - 4), b = ld4(row), c = ld4(row + 4);
                const float x[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
                for (int dz = 0; dz < 5; ++dz) {
                    if (m.kmap[dxy * 5 + dz] < 0) continue;
                    const float4 w = __ldg(wm + (size_t)(dxy * 5 + dz) * nm);
                    acc[0] += w.x * x[2 + dz];
                    acc[1] += w.y * x[3 + dz];
                    acc[2] += w.z * x[4 + dz];
                    acc[3] += w.w * x[5 + dz];
                }
            }
        }
        const float ds = m.dscale;
        const float *__restrict__ db = m.dbox[l];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (mask & (1 << i)) {
                const float t = R[off + i] - acc[i];
                T[off + i] = fold ? X[off + i] + ds * db[off + i] * t : t;
            }
    }
}

// Level 1 takes its post-smoothing inside the residual pass (T = X + D (R - A X),
// the smoothed correction, goes to the T box): the V-cycle's level-1 result is
// in T when the hierarchy has a level 2 and level 1 runs in the run form.
__device__ __forceinline__ bool mg_fold1(const MgSm &m) { return m.nlev > 2 && m.n_groups[1] > 0; }

// Z_1 = P Z_2 on the level-1 runs: a run's four points start at an even
// last-axis coordinate, so they take their last-axis parents from three level-2
// values of each (x, y) row, one row or two along each axis whose coordinate is
// odd (pinfo1), as pass D does for the fine groups.
__device__ __noinline__ void mg_prolong_runs1()
{
    const MgSm &m = g_mg_sm;
    const int ng = m.n_groups[1];
    const float *__restrict__ Z2 = m.Z[2];
    float *__restrict__ Z1 = m.Z[1];
    const int cB2 = m.Bp2[2], sx = m.Bp1[2] * m.Bp2[2];
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int32_t gw = __ldg(m.groups[1] + g);
        const int off = (gw >> 4) << 2, mask = gw & 15;
        const int32_t pinf = __ldg(m.pinfo1 + g);
        const bool ox = pinf & 2, oy = pinf & 1;
        const float *rb = Z2 + (pinf >> 2);
        float c_0 = rb[0], c_1 = rb[1], c_2 = rb[2];
        const float y0 = rb[cB2], y1 = rb[cB2 + 1], y2 = rb[cB2 + 2];
        const float x0 = rb[sx], x1 = rb[sx + 1], x2 = rb[sx + 2];
        const float xy0 = rb[sx + cB2], xy1 = rb[sx + cB2 + 1], xy2 = rb[sx + cB2 + 2];
        if (oy) {
            c_0 += y0;
            c_1 += y1;
            c_2 += y2;
        }
        if (ox) {
            c_0 += x0;
            c_1 += x1;
            c_2 += x2;
        }
        if (ox && oy) {
            c_0 += xy0;
            c_1 += xy1;
            c_2 += xy2;
        }
        const float wxy = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
        const float z[4] = {wxy * c_0, wxy * 0.5f * (c_0 + c_1), wxy * c_1, wxy * 0.5f * (c_1 + c_2)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (mask & (1 << i)) Z1[off + i] = z[i];
    }
}

// R_1 = P^T t from the fine CG box t (B1, B2, no margin) by runs of 4 level-1
// points along the last axis: their fine centres 2 c2 .. 2 c2 + 6 sit at a
// multiple of 4 (level-1 runs start at u2 = 0 mod 4 with a margin of 2), so
// three aligned float4 loads per fine (dx, dy) row give the nine values
// 2 c2 - 1 .. 2 c2 + 7 that the four points need.  Same weights and order of
// additions as mg_restrict.
__device__ __forceinline__ void mg_restrict_runs(const float *__restrict__ src, int B1, int B2)
{
    const MgSm &m = g_mg_sm;
    const int ng = m.n_groups[1];
    float *__restrict__ dst = m.R[1];
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const int32_t gw = __ldg(m.groups[1] + g);
        const int off = (gw >> 4) << 2, mask = gw & 15;
        int c0, c1, c2;
        mg_coords(off, m.Bp1[1], m.Bp2[1], c0, c1, c2);
        c0 -= kMgPadDev;
        c1 -= kMgPadDev;
        c2 -= kMgPadDev;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const float *row = src + ((size_t)(2 * c0 + dx) * B1 + (2 * c1 + dy)) * B2 + 2 * c2;
                const float4 a = ld4(row - 4), b = ld4(row), c = ld4(row + 4);
                const float x[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
                const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] += w * (x[4 + 2 * i] + 0.5f * (x[3 + 2 * i] + x[5 + 2 * i]));
            }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (mask & (1 << i)) dst[off + i] = acc[i];
    }
}

// T = R - A_l X on the active points of coarse level l.  Levels with fewer
// rows than half the CTA's threads give each row 2, 4 or 8 adjacent lanes,
// which split the pattern and add their parts by shuffles.
__device__ __forceinline__ void mg_resid(int l, const float *__restrict__ R, const float *__restrict__ X,
                                         float *__restrict__ T)
{
    const MgSm &m = g_mg_sm;
    const int n = m.n[l], nt = blockDim.x;
    int tpr = 1;
    while (tpr < 8 && n * tpr * 2 <= nt) tpr <<= 1;
    const int lane = threadIdx.x & 31, sub = lane & (tpr - 1);
    const unsigned gmask = ((1u << tpr) - 1u) << (lane & ~(tpr - 1));
    const int *pts = m.pts[l];
    for (int i = threadIdx.x / tpr; i < n; i += nt / tpr) {
        const int o = pts[i];
        float s = mg_row(l, i, o, X, sub, tpr);
        for (int d = tpr >> 1; d > 0; d >>= 1) s += __shfl_xor_sync(gmask, s, d);
        if (sub == 0) T[o] = R[o] - s;
    }
}

// Z_1 = M_1 R_1: the V(1,1) cycle on the coarse levels 1 .. nlev-1.
__device__ __noinline__ void mg_coarse_cycle()
{
    const MgSm &m = g_mg_sm;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int L = m.nlev - 1;   // coarsest
    // down: Jacobi smoothing from zero, Z = D R, its residual T = R - A Z, restriction.
    // Level 1 (the largest coarse level, 8x fewer points than the fine one but 81-99
    // pattern entries per row) skips the pre-smoothing: R_1 itself is restricted and
    // Z_1 starts from the coarse correction.  The cycle is then not exactly
    // symmetric; CG still takes it as a preconditioner (one iteration more at most on
    // the benchmark cells, against one residual pass of level 1 less per cycle).
    for (int l = 1; l < L; ++l) {
        const int *pts = m.pts[l];
        const float *R = m.R[l];
        float *Z = m.Z[l], *T = m.T[l];
        const float ds = m.dscale;
        if (l > 1) {
            for (int i = tid; i < m.n[l]; i += nt) {
                const int o = pts[i];
                Z[o] = ds * __ldg(m.dinv[l] + i) * R[o];
            }
            __syncthreads();
            mg_resid(l, R, Z, T);
            __syncthreads();
        }
        mg_restrict(m, l, l > 1 ? T : R, m.Bp1[l], m.Bp2[l], kMgPadDev);
        __syncthreads();
    }
    // coarsest: z = A_L^-1 r, one warp per row
    {
        const int n = m.n[L];
        float *cr = g_mg_sm.cr;
        for (int i = tid; i < n; i += nt) cr[i] = m.R[L][m.pts[L][i]];
        __syncthreads();
        const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
        for (int i = w; i < n; i += nw) {
            const float *row = m.cinv + (size_t)i * n;
            float s = 0.f;
            for (int j = lane; j < n; j += 32) s += __ldg(row + j) * cr[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) m.Z[L][m.pts[L][i]] = s;
        }
        __syncthreads();
    }
    // up: Z = D R + P Z_{l+1}, then post-smoothing Z += D (R - A Z)
    for (int l = L - 1; l >= 1; --l) {
        const int *pts = m.pts[l];
        const float *R = m.R[l];
        float *Z = m.Z[l], *T = m.T[l];
        const float ds = m.dscale;
        if (l == 1 && mg_fold1(m)) {
            // Z_1 = P Z_2 by runs, then T_1 = Z_1 + D_1 (R_1 - A_1 Z_1): the level's result
            mg_prolong_runs1();
            __syncthreads();
            mg_resid_runs(R, Z, T, true);
            __syncthreads();
            break;
        }
        for (int i = tid; i < m.n[l]; i += nt) {
            const int o = pts[i];
            int u0, u1, u2;
            mg_coords(o, m.Bp1[l], m.Bp2[l], u0, u1, u2);
            Z[o] = (l > 1 ? ds * __ldg(m.dinv[l] + i) * R[o] : 0.f) +
                   mg_prolong_at(m, l, u0 - kMgPadDev, u1 - kMgPadDev, u2 - kMgPadDev);
        }
        __syncthreads();
        if (l == 1 && m.n_groups[1] > 0) mg_resid_runs(R, Z, T, false);
        else mg_resid(l, R, Z, T);
        __syncthreads();
        for (int i = tid; i < m.n[l]; i += nt) {
            const int o = pts[i];
            Z[o] += ds * __ldg(m.dinv[l] + i) * T[o];
        }
        __syncthreads();
    }
}

// One pass over the aligned groups that runs a pointwise update ahead of a
// stencil: groups are sorted by box offset, so the stencil of chunk c (W groups)
// reads only groups below need[c] (the chunk's last offset plus the stencil
// reach); the update front is brought to need[c] before the chunk's stencil,
// with one CTA barrier per chunk.  The stencil then reads the updated vector
// while it is still cache-resident, and every group is updated exactly once.
template <class Upd, class Sten>
__device__ __forceinline__ void front_sweep(int ng, int nchunk, int W, const int *need, Upd upd, Sten sten)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    int front = 0;
    for (int c = 0; c < nchunk; ++c) {
        for (const int nd = need[c]; front < nd; front += nt) {
            const int g = front + tid;
            if (g < ng) upd(g);
        }
        __syncthreads();
        const int gend = min(ng, (c + 1) * W);
        for (int g = c * W + tid; g < gend; g += nt) sten(g);
    }
}

__shared__ int g_mg_need[kMaxSweepChunks];   // update front of each chunk (multigrid path)

struct MgScalars {
    double rz, rmax, S;
    float alpha, beta;
    int act;    // 0 continue, 1 reliable update, 2 reliable update after a breakdown
    int conv;   // the recursive residual predicts convergence (the reliable update may end the CG)
};
__shared__ MgScalars g_mg_cs;

// The fine-level passes of the multigrid PCG, each an out-of-line function so
// that its group loop has the registers to itself (the caller's state stays in
// the caller's frame across the call).  Each returns its thread's part of the
// pass's dot product as a double-float pair (hi, lo).

// t = r + c0 L r on one group (the stencil half of pass B and the frame's first
// pre-smoothing), into qf
template <int FDN>
__device__ __forceinline__ void mg_pre_smooth_group(const SetDev &S, const SmemCell &sm, const float *__restrict__ rf,
                                                    float *__restrict__ qf, float c0, int g)
{
    const int32_t gw = __ldg(S.groups + g);
    const int off = (gw >> 4) << 2, mask = gw & 15;
    float acc[4];
    lap4<FDN>(rf, off, sm.cw32, sm.center32, S.rstride, S.d2, sm.C.ndir, acc);
    const float4 r = ld4(rf + off);
    st4(qf + off, (mask & 1) ? r.x + c0 * acc[0] : 0.f, (mask & 2) ? r.y + c0 * acc[1] : 0.f,
        (mask & 4) ? r.z + c0 * acc[2] : 0.f, (mask & 8) ? r.w + c0 * acc[3] : 0.f);
}

template <int FDN>
__device__ __noinline__ void mg_pre_smooth_all(const SetDev &S, const SmemCell &sm, const float *rf, float *qf, float c0)
{
    for (int g = threadIdx.x; g < S.n_groups; g += blockDim.x) mg_pre_smooth_group<FDN>(S, sm, rf, qf, c0, g);
}

// pass A: p = z + beta p (p = z in a frame's first iteration; z is in qf) ahead
// of q = A p into qf, <p, q>
template <int FDN>
__device__ __noinline__ float2 mg_pass_a(const SetDev &S, const SmemCell &sm, float *__restrict__ pf,
                                         float *__restrict__ qf, float beta, bool copy, int nchunk, int W)
{
    const int32_t *__restrict__ grp = S.groups;
    DF a = {0.f, 0.f};
    front_sweep(
        S.n_groups, nchunk, W, g_mg_need,
        [&](int g) {
            const int off = (__ldg(grp + g) >> 4) << 2;
            const float4 z = ld4(qf + off);
            if (copy) {
                *reinterpret_cast<float4 *>(pf + off) = z;
            } else {
                const float4 p = ld4(pf + off);
                st4(pf + off, z.x + beta * p.x, z.y + beta * p.y, z.z + beta * p.z, z.w + beta * p.w);
            }
        },
        [&](int g) {
            const int32_t gw = __ldg(grp + g);
            const int off = (gw >> 4) << 2, mask = gw & 15;
            float acc[4];
            const float4 p = lap4<FDN>(pf, off, sm.cw32, sm.center32, S.rstride, S.d2, sm.C.ndir, acc);
            const float q0 = (mask & 1) ? -acc[0] : 0.f, q1 = (mask & 2) ? -acc[1] : 0.f;
            const float q2 = (mask & 4) ? -acc[2] : 0.f, q3 = (mask & 8) ? -acc[3] : 0.f;
            st4(qf + off, q0, q1, q2, q3);
            df_add(a, p.x * q0 + p.y * q1 + p.z * q2 + p.w * q3);
        });
    return make_float2(a.hi, a.lo);
}

// pass B: r -= alpha q, e += alpha p (<r, r>) ahead of t = r + c0 L r into qf
template <int FDN>
__device__ __noinline__ float2 mg_pass_b(const SetDev &S, const SmemCell &sm, float *__restrict__ rf,
                                         float *__restrict__ qf, const float *__restrict__ pf, float *__restrict__ ef,
                                         float alpha, float c0, int nchunk, int W)
{
    const int32_t *__restrict__ grp = S.groups;
    DF b = {0.f, 0.f};
    front_sweep(
        S.n_groups, nchunk, W, g_mg_need,
        [&](int g) {
            const int off = (__ldg(grp + g) >> 4) << 2;
            const float4 r = ld4(rf + off), q = ld4(qf + off), p = ld4(pf + off), e = ld4(ef + off);
            const float r0 = r.x - alpha * q.x, r1 = r.y - alpha * q.y, r2 = r.z - alpha * q.z, r3 = r.w - alpha * q.w;
            st4(rf + off, r0, r1, r2, r3);
            st4(ef + off, e.x + alpha * p.x, e.y + alpha * p.y, e.z + alpha * p.z, e.w + alpha * p.w);
            df_add(b, r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
        },
        [&](int g) { mg_pre_smooth_group<FDN>(S, sm, rf, qf, c0, g); });
    return make_float2(b.hi, b.lo);
}

// pass D: z0 = c0 r + P Z_1 into zf ahead of z = z0 + c0 (r + L z0) into qf, <r, z>.
// The group's four points u2 .. u2+3 (u2 a multiple of 4) take their last-axis
// parents from three level-1 values of each (x, y) row: one row, or two along
// each axis whose fine coordinate is odd (pinfo).
template <int FDN>
__device__ __noinline__ float2 mg_pass_d(const SetDev &S, const SmemCell &sm, const float *__restrict__ rf,
                                         float *__restrict__ zf, float *__restrict__ qf, float c0, int nchunk, int W)
{
    const MgSm &m = g_mg_sm;
    const int32_t *__restrict__ grp = S.groups;
    const int32_t *__restrict__ pinfo = m.pinfo;
    const float *__restrict__ Z1 = mg_fold1(m) ? m.T[1] : m.Z[1];   // the level-1 result of the cycle
    const int cB2 = m.Bp2[1], sx = m.Bp1[1] * m.Bp2[1];
    DF a = {0.f, 0.f};
    front_sweep(
        S.n_groups, nchunk, W, g_mg_need,
        [&](int g) {
            const int32_t gw = __ldg(grp + g);
            const int off = (gw >> 4) << 2, mask = gw & 15;
            const int32_t pinf = __ldg(pinfo + g);
            const bool ox = pinf & 2, oy = pinf & 1;
            // the parents' row offset is even (u2 / 2 + margin with u2 = 0 mod 4, rows
            // of a multiple of 4): the first two of each row's three values are one float2
            const float *rb = Z1 + (pinf >> 2);
            const float2 r00 = ld2(rb), r01 = ld2(rb + cB2), r10 = ld2(rb + sx), r11 = ld2(rb + sx + cB2);
            float c_0 = r00.x, c_1 = r00.y, c_2 = rb[2];
            const float y0 = r01.x, y1 = r01.y, y2 = rb[cB2 + 2];
            const float x0 = r10.x, x1 = r10.y, x2 = rb[sx + 2];
            const float xy0 = r11.x, xy1 = r11.y, xy2 = rb[sx + cB2 + 2];
            if (oy) {
                c_0 += y0;
                c_1 += y1;
                c_2 += y2;
            }
            if (ox) {
                c_0 += x0;
                c_1 += x1;
                c_2 += x2;
            }
            if (ox && oy) {
                c_0 += xy0;
                c_1 += xy1;
                c_2 += xy2;
            }
            const float wxy = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
            const float4 r = ld4(rf + off);
            st4(zf + off, (mask & 1) ? c0 * r.x + wxy * c_0 : 0.f,
                (mask & 2) ? c0 * r.y + wxy * 0.5f * (c_0 + c_1) : 0.f, (mask & 4) ? c0 * r.z + wxy * c_1 : 0.f,
                (mask & 8) ? c0 * r.w + wxy * 0.5f * (c_1 + c_2) : 0.f);
        },
        [&](int g) {
            const int32_t gw = __ldg(grp + g);
            const int off = (gw >> 4) << 2, mask = gw & 15;
            float acc[4];
            const float4 z0 = lap4<FDN>(zf, off, sm.cw32, sm.center32, S.rstride, S.d2, sm.C.ndir, acc);
            const float4 r = ld4(rf + off);
            const float z_0 = (mask & 1) ? z0.x + c0 * (r.x + acc[0]) : 0.f;
            const float z_1 = (mask & 2) ? z0.y + c0 * (r.y + acc[1]) : 0.f;
            const float z_2 = (mask & 4) ? z0.z + c0 * (r.z + acc[2]) : 0.f;
            const float z_3 = (mask & 8) ? z0.w + c0 * (r.w + acc[3]) : 0.f;
            st4(qf + off, z_0, z_1, z_2, z_3);
            df_add(a, r.x * z_0 + r.y * z_1 + r.z * z_2 + r.w * z_3);
        });
    return make_float2(a.hi, a.lo);
}

// The mixed-precision solve of one pair with the multigrid preconditioner (see
// the comment above MgSm).  zf: one more dense FP32 box; mgbase: the slot's
// region for the coarse boxes.  One PCG iteration is four passes over the fine
// groups, each a pointwise update run ahead of a stencil (front_sweep):
//   A  p = z + beta p           ahead of   q = A p, <p, q>
//   B  r -= alpha q, e += alpha p   ahead of   t = r + c0 L r (pre-smoothed residual)
//      restriction of t, the coarse levels
//   D  z0 = c0 r + P Z_1         ahead of   z = z0 + c0 (r + L z0), <r, z>
// (pass B's t is discarded when its <r, r> calls for a reliable update).
template <int FDN>
__device__ __noinline__ void cg_mixed_mg(const CgMixed &cg, float *zf, float *mgbase, int &iters, int &refine,
                                         int &status, double &rnorm, double *es, bool &es_done)
{
    es_done = false;
    const SetDev &S = *cg.S;
    const SmemCell &sm = *cg.sm;
    const int tid = threadIdx.x, nt = blockDim.x;
    float *__restrict__ pf = cg.pf;
    float *__restrict__ rf = cg.rf;
    float *__restrict__ qf = cg.qf;
    float *__restrict__ ef = cg.ef;
    float2 *vb = reinterpret_cast<float2 *>(cg.vbox);
    float *r32 = reinterpret_cast<float *>(cg.r64);
    const int32_t *__restrict__ poff = S.pe_off;
    const int32_t *__restrict__ grp = S.groups;
    const int npe = S.n_pe, ng = S.n_groups, ndir = cg.ndir;
    const int *rs = S.rstride, *dsf = S.dstride;
    const double stop = cg.stop, inner_red = cg.inner_red;
    float2 *red2 = reinterpret_cast<float2 *>(cg.red);
    const int B1 = S.B[1], B2 = S.B[2];

    MgSm &m = g_mg_sm;
    MgScalars &cs = g_mg_cs;
    {
        const MgDev &G = *S.mg;
        if (tid == 0) {
            m.nlev = G.nlev;
            const double om = sm.C.mg_omega > 0.f ? (double)sm.C.mg_omega : (double)G.omega;
            m.c0 = (float)(om / -(double)sm.center64);
            m.dscale = (float)(om / (double)G.omega);
            m.cinv = G.cinv;
            m.pinfo = G.pinfo;
            m.pinfo1 = G.pinfo1;
            for (int l = 1; l < G.nlev; ++l) {
                const MgLevelDev &v = G.lv[l];
                m.n[l] = v.n;
                m.K[l] = v.K;
                m.Bp1[l] = v.Bp[1];
                m.Bp2[l] = v.Bp[2];
                m.R[l] = mgbase + v.off;
                m.Z[l] = mgbase + v.off + v.stride;
                m.T[l] = mgbase + v.off + 2 * v.stride;
                m.pts[l] = v.pts;
                m.n_int[l] = v.n_int;
                m.n_exp[l] = v.n_exp;
                m.wexp[l] = v.wexp;
                m.dinv[l] = v.dinv;
                m.dbox[l] = v.dbox;
                m.n_groups[l] = v.n_groups;
                m.n_pure[l] = v.n_pure;
                m.groups[l] = v.groups;
                m.wmix[l] = v.wmix;
            }
        }
        if (G.nlev > 2)
            for (int k = tid; k < 125; k += nt) {
                m.wdense[k] = G.wdense[1][k];
                m.kmap[k] = G.kmap[1][k];
                if (k < 25) m.rows1[k] = G.rows[1][k];
                if (k == 0) m.nrow1 = G.nrow[1];
            }
        for (int l = 1; l < G.nlev; ++l)
            for (int k = tid; k < G.lv[l].K; k += nt) {
                const int kd = G.kd[l][k];
                const int dx = (kd & 7) - 2, dy = ((kd >> 3) & 7) - 2, dz = ((kd >> 6) & 7) - 2;
                m.koff[l][k] = (dx * G.lv[l].Bp[1] + dy) * G.lv[l].Bp[2] + dz;
                m.wint[l][k] = G.wint[l][k];
            }
        // the coarse boxes start all zero: points that are inactive for this set
        // are read by the restriction and must hold zeros
        for (long long k = tid; k < G.floats; k += nt) mgbase[k] = 0.f;
    }
    // update front of every chunk of the fused passes
    const int W = kSweepChunkGroups * nt;
    const int nchunk = (ng + W - 1) / W;
    {
        int reach = 7;
        for (int d = 0; d < ndir; ++d) reach = max(reach, 3 + FDN * max(abs(dsf[d]), abs(rs[d])));
        for (int c = tid; c < nchunk; c += nt) {
            const int last = min(ng, (c + 1) * W) - 1;
            const long long lim = (long long)((grp[last] >> 4) << 2) + reach;
            int lo = last + 1, hi = ng;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)((grp[mid] >> 4) << 2) <= lim) lo = mid + 1;
                else hi = mid;
            }
            g_mg_need[c] = lo;
        }
    }
    __syncthreads();
    if (!(cg.r0n > stop)) return;   // the starting guess already meets the tolerance
    const float c0 = m.c0;

    // restriction, coarse levels and pass D: z into qf, <r, z> returned (valid in warp 0)
    auto finish_precondition = [&]() -> double {
        __syncthreads();
        if (m.n_groups[1] > 0) mg_restrict_runs(qf, B1, B2);
        else mg_restrict(m, 0, qf, B1, B2, 0);
        __syncthreads();
        mg_coarse_cycle();
        const float2 d = mg_pass_d<FDN>(S, sm, rf, zf, qf, c0, nchunk, W);
        DF a[1] = {{d.x, d.y}};
        block_sum_df<1>(a, red2);
        return (double)a[0].hi + (double)a[0].lo;
    };

    // frame of the starting residual (r32 holds the last true residual in FP32)
    double Sc = cg.r0n;
    for (;;) {
        {
            const F32Scale sc = f32_scale(1.0 / Sc);
            DF a[1] = {{0.f, 0.f}};
            // (e is zero here: the boxes start zero for every pair and each reliable
            // update clears it)
            for (int k = tid; k < npe; k += nt) {
                const int off = poff[k];
                const float r = sc.apply(r32[k]);
                rf[off] = r;
                df_add(a[0], r * r);
            }
            block_sum_df<1>(a, red2);
            if (tid == 0) cs.rmax = sqrt((double)a[0].hi + (double)a[0].lo);
            __syncthreads();
        }
        // z = M r from the frame's residual (pass B without its update)
        mg_pre_smooth_all<FDN>(S, sm, rf, qf, c0);
        const double rz0 = finish_precondition();
        if (tid == 0) {
            cs.rz = rz0;
            cs.S = Sc;
            cs.beta = 0.f;
        }
        __syncthreads();
        bool first = true;   // p = z (no previous direction in this frame)
        bool restart = false;
        while (!restart) {
            if (iters >= cg.max_iter) {
                status = 5;
                return;
            }
            // pass A: p = z + beta p ahead of q = A p, <p, q>
            const float beta = cs.beta;
            const bool copy = first;
            first = false;
            const float2 pa = mg_pass_a<FDN>(S, sm, pf, qf, beta, copy, nchunk, W);
            DF a[1] = {{pa.x, pa.y}};
            block_sum_df<1>(a, red2);
            if (tid == 0) {
                const double pq = (double)a[0].hi + (double)a[0].lo;
                const double al = cs.rz / pq;
                cs.act = (!(pq > 0.0) || !(cs.rz > 0.0) || !(al < 1e300)) ? 2 : 0;
                cs.alpha = cs.act ? 0.f : (float)al;
            }
            __syncthreads();
            const float alpha = cs.alpha;
            int act = cs.act;
            if (!act) {
                // pass B: e += alpha p, r -= alpha q (<r, r>) ahead of t = r + c0 L r
                const float2 pb = mg_pass_b<FDN>(S, sm, rf, qf, pf, ef, alpha, c0, nchunk, W);
                DF b[1] = {{pb.x, pb.y}};
                block_sum_df<1>(b, red2);
                if (tid == 0) {
                    const double rr = (double)b[0].hi + (double)b[0].lo;
                    const double rn = sqrt(rr);
                    if (!(rn == rn) || rn <= inner_red * cs.rmax || rn * cs.S <= 0.5 * stop) cs.act = 1;
                    cs.conv = rn * cs.S <= 0.5 * stop;
                }
                __syncthreads();
                act = cs.act;
            }
            ++iters;
            if (act) {
                // reliable update: v += S e in double-float, the true residual replaces r
                ++refine;
                const float2 S2 = dw_split(cs.S);
                for (int k = tid; k < npe; k += nt) {
                    const int off = poff[k];
                    vb[off] = dw_add(vb[off], dw_mul(make_float2(ef[off], 0.f), S2));
                    ef[off] = 0.f;
                }
                __syncthreads();
                // when the recursive residual predicts the end of the CG, the same pass
                // takes the Step V sums
                const bool conv = act == 1 && cs.conv;
                rnorm = sqrt(conv ? residual_es_df_n(cg.fdn, S, vb, cg.b2, r32, sm.cwdf, sm.centerdf, sm.ds, ndir,
                                                     cg.red, sm.w1df, sm.C.stress_mode != 2, es)
                                  : residual_df_n(cg.fdn, S, vb, cg.b2, r32, sm.cwdf, sm.centerdf, sm.ds, ndir,
                                                  cg.red));
                if (rnorm <= stop) {
                    es_done = conv;
                    return;
                }
                if (!(rnorm == rnorm)) {
                    status = 5;
                    return;
                }
                Sc = rnorm;
                restart = true;
                continue;
            }
            // the rest of z = M r (t is in qf), beta = <r, z> / <r, z>_old
            const double rz = finish_precondition();
            if (tid == 0) {
                cs.beta = (float)(rz / cs.rz);
                cs.rz = rz;
            }
            __syncthreads();
        }
    }
}

// Starting guess of the CG: the free-space potential of rho on the PE points,
//   v(r) = sum_lm 4 pi / (2l+1) Y_lm(r^) [ r^-(l+1) q<_lm(r) + r^l q>_lm(r) ],
// q<_lm(r) = sum_{|r'| < r} rho r'^l Y_lm dV, q>_lm(r) = sum_{|r'| > r} rho r'^-(l+1) Y_lm dV,
// with |r'| < r decided by radial bin (half of the point's own bin on each side).
// Outside PE this is the far field of Eq. me, which is why it is close to the
// solution of Eq. pe; it only sets where CG starts, not what it converges to.
// gs: scratch of the CTA, [2][2 kGuessBins][kNlm] moments per half bin (later
// overwritten by the guess's per-bin coefficients, [kGuessBins][kNlm] float4),
// then [2][kGuessBins][kNlm] cumulative inner and outer moments per bin.
constexpr double kWarmAccept = 0.05;   // warm starts kept when |b - A v_prev| <= 5 % of |b|

// Sums over lm (l <= lmax) of S_lm(x, y, z) times coefficients, with r^l Y_lm
// from the Cartesian recurrences of solid_harmonics evaluated in FP32 (about
// 1e-6 of the largest term, against 6e-8 for the rounded FP64 tables),
// summed per degree: for NC coefficient channels,
// vl[c][l] = sum_m Q_l^m (A_m cf_c(l, m) + B_m cf_c(l, -m)) (Q_l^0 cf_c(l, 0) for
// m = 0), with the normalisation N_lm already folded into the coefficients.  cf
// fills k[2c] = cf_c(l, m) and k[2c + 1] = cf_c(l, -m).  The caller weights
// each degree (r^-(2l+1) for a far field), so no per-term factor of r is needed.
template <int NC, class Cf>
__device__ __forceinline__ void solid_parts32(float x, float y, float z, int lmax, const Cf &cf, float (&vl)[NC][7])
{
    const float r2 = x * x + y * y + z * z;
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int l = 0; l < 7; ++l) vl[c][l] = 0.f;
    float Am = 1.f, Bm = 0.f, dfact = 1.f;
#pragma unroll
    for (int m = 0; m <= 6; ++m) {
        if (m > 0) {
            const float An = x * Am - y * Bm;
            Bm = x * Bm + y * Am;
            Am = An;
            dfact *= (float)(2 * m - 1);
        }
        float q1 = 0.f, q2 = 0.f;
#pragma unroll
        for (int l = m; l <= 6; ++l) {
            float q;
            if (l == m) q = dfact;
            else if (l == m + 1) q = (float)(2 * m + 1) * z * dfact;
            else q = ((float)(2 * l - 1) * z * q1 - (float)(l + m - 1) * r2 * q2) * (1.f / (float)(l - m));
            q2 = q1;
            q1 = q;
            if (l <= lmax) {
                float k[2 * NC];
                cf(l, m, k);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (m == 0) vl[c][l] += q * k[2 * c];
                    else vl[c][l] += q * (Am * k[2 * c] + Bm * k[2 * c + 1]);
                }
            }
        }
    }
}

// r^-(2l+1), l = 0..6, from 1/r
struct RinvPows {
    float f[7];
    __device__ explicit RinvPows(float ri)
    {
        const float ri2 = ri * ri;
        f[0] = ri;
#pragma unroll
        for (int l = 1; l < 7; ++l) f[l] = f[l - 1] * ri2;
    }
};

__device__ __forceinline__ void xyz_of(const float (*h)[3], int32_t pm, float &x, float &y, float &z)
{
    int m0, m1, m2;
    unpack_m(pm, m0, m1, m2);
    x = h[0][0] * m0 + h[0][1] * m1 + h[0][2] * m2;
    y = h[1][0] * m0 + h[1][1] * m1 + h[1][2] * m2;
    z = h[2][0] * m0 + h[2][1] * m1 + h[2][2] * m2;
}

// Multipole moments of rho per radial bin over the radius-sorted copy of the
// solid-harmonic table (no atomics: the same sums on every run).  Each bin is
// split into two halves of its sorted range; the 2 kGuessBins pieces, in order
// of decreasing radius, are dealt to the warps in snake order so that warps
// get similar numbers of points (bin sizes grow as the square of the radius).
// gs receives per piece the inner moments rho r^l Y_lm dV and the outer
// moments rho r^-(l+1) Y_lm dV (FP32), and qpart[w] the FP64 sum of the inner
// moments of warp w's pieces; their sum over the warps is the moment Q_lm of
// Eq. mepole (up to dV), accumulated like the one-pass moments: FP32 over 32
// points, FP64 beyond.  Per 32 points the warp stages rho and rho r^-(2l+1)
// (l = 0..6) in shared memory, so each table row costs two loads and four FMAs.
constexpr int kGuessPieces = 2 * kGuessBins;
__device__ __noinline__ void bin_moments(const SetDev &S, const CellDev &C, const double *__restrict__ rho,
                                         float *__restrict__ gs, double (*qpart)[kNlm])
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int l0 = lane < 1 ? 0 : lane < 4 ? 1 : lane < 9 ? 2 : lane < 16 ? 3 : lane < 25 ? 4 : 5;   // l of lm = lane
    const int l1 = lane + 32 < 36 ? 5 : 6;                                                          // l of lm = lane + 32
    const bool has1 = lane + 32 < kNlm;
    const int lane1 = has1 ? lane + 32 : lane;
    float h[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) h[a][b] = (float)(C.h[a][b] / C.n[b]);
    float *PA = gs, *PB = gs + kGuessPieces * kNlm;   // per piece j: bin kGuessBins - 1 - j / 2, half j % 2
    const double dv = C.dv;
    __shared__ float s_mw[kSolveThreads / 32][32][8];
    float(*mw)[8] = s_mw[warp];
    double w0 = 0.0, w1 = 0.0;
    for (int base = 0; base < kGuessPieces; base += nwarps) {   // each round a permutation of base + [0, nwarps)
        const int j = base + (((base / nwarps) & 1) ? nwarps - 1 - warp : warp);
        if (j >= kGuessPieces) continue;
        const int b = kGuessBins - 1 - j / 2;
        const int b0_ = S.gs_bstart[b], b1_ = S.gs_bstart[b + 1], mid = b0_ + (b1_ - b0_) / 2;
        const int k0 = (j & 1) ? mid : b0_, k1 = (j & 1) ? b1_ : mid;
        double a0 = 0.0, a1 = 0.0;
        float b0 = 0.f, b1 = 0.f;
        for (int x = k0; x < k1; x += 32) {
            const bool live = x + lane < k1;
            const int4 inf = __ldg(S.gs_info + (live ? x + lane : x));
            const float rl = live ? (float)rho[inf.w] : 0.f;
            float px, py, pz;
            xyz_of(h, inf.x, px, py, pz);
            const float r2 = px * px + py * py + pz * pz;
            const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
            const int xq = min(32, k1 - x);
            // each lane's point: rho r^-(2l+1) for l = 0..6, and rho, for the warp to read
            __syncwarp();
            {
                const float ri2 = ri * ri;
                float pw = ri;
#pragma unroll
                for (int l = 0; l < 7; ++l) {
                    mw[lane][l] = rl * pw;
                    pw *= ri2;
                }
                mw[lane][7] = rl;
            }
            __syncwarp();
            float f0 = 0.f, f1 = 0.f;
#pragma unroll 16
            for (int q = 0; q < 32; ++q) {
                const float rp = mw[q][7];
                const float *row = S.gs_S32 + (size_t)(x + min(q, xq - 1)) * kNlm;   // rows in sorted order
                const float s0 = row[lane], s1 = row[lane1];
                f0 += rp * s0;
                f1 += rp * s1;
                b0 += s0 * mw[q][l0];
                b1 += s1 * mw[q][l1];
            }
            a0 += f0;
            a1 += f1;
        }
        PA[j * kNlm + lane] = (float)(a0 * dv);
        PB[j * kNlm + lane] = (float)(b0 * dv);
        if (has1) {
            PA[j * kNlm + lane + 32] = (float)(a1 * dv);
            PB[j * kNlm + lane + 32] = (float)(b1 * dv);
        }
        w0 += a0;
        w1 += a1;
    }
    qpart[warp][lane] = w0;
    if (has1) qpart[warp][lane + 32] = w1;
}

// The guess itself from the bin moments of bin_moments: cumulative inner and
// outer sums, then v at every PE point with r^l Y_lm from the Cartesian
// recurrences of solid_harmonics in FP32.  Points are visited in radius order,
// so the lanes of a warp share one or two bins and read the same moments.
__device__ __noinline__ void multipole_guess(const SetDev &S, const CellDev &C, const float *cn,
                                             const float (*hf)[3], double *vbox, float *__restrict__ gs, bool df)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const float *PA = gs, *PB = gs + kGuessPieces * kNlm;   // per piece (bin_moments)
    float *A = gs + 2 * kGuessPieces * kNlm, *B = A + kGuessBins * kNlm;
    // bin moments (both halves), then inner sums from below and outer sums from
    // above, half of the own bin each
    if (tid < 2 * kNlm) {
        const int lm = tid % kNlm;
        const float *P = tid < kNlm ? PA : PB;
        float *Q = tid < kNlm ? A : B;
        float acc = 0.f;
        for (int i = 0; i < kGuessBins; ++i) {
            const int b = tid < kNlm ? i : kGuessBins - 1 - i;
            const int jp = 2 * (kGuessBins - 1 - b);
            const float a = P[jp * kNlm + lm] + P[(jp + 1) * kNlm + lm];
            Q[b * kNlm + lm] = acc + 0.5f * a;
            acc += a;
        }
    }
    __syncthreads();
    // per bin and (l, m >= 0), over the per-piece moments (no longer needed):
    // 4 pi / (2l+1) N_lm times the inner and outer sums of (l, m) and (l, -m)
    float4 *G = reinterpret_cast<float4 *>(gs);
    for (int t = tid; t < kGuessBins * kNlm; t += nt) {
        const int b = t / kNlm, i = t - b * kNlm;
        int l = 0;
        while ((l + 1) * (l + 1) <= i) ++l;
        const int i0 = l * l + l, mm = i - i0;
        const float K = (12.566370614359172f / (float)(2 * l + 1)) * cn[i];
        const float *Ab = A + b * kNlm, *Bb = B + b * kNlm;
        G[t] = mm < 0 ? make_float4(0.f, 0.f, 0.f, 0.f)
                      : make_float4(K * Ab[i], mm > 0 ? K * Ab[i0 - mm] : 0.f, K * Bb[i], mm > 0 ? K * Bb[i0 - mm] : 0.f);
    }
    __syncthreads();
    const int lmax = C.lmax;
    for (int j = tid; j < S.n_pe; j += nt) {
        const int4 inf = __ldg(S.gs_info + j);
        const float4 *Gb = G + inf.z * kNlm;
        float x, y, z;
        xyz_of(hf, inf.x, x, y, z);
        const float r2 = x * x + y * y + z * z;
        const RinvPows rp(r2 > 0.f ? rsqrtf(r2) : 0.f);
        float vl[2][7];
        solid_parts32<2>(x, y, z, lmax,
                         [&](int l, int m, float *k) {
                             const float4 g = Gb[l * l + l + m];
                             k[0] = g.x;
                             k[1] = g.y;
                             k[2] = g.z;
                             k[3] = g.w;
                         },
                         vl);
        float v = 0.f;
#pragma unroll
        for (int l = 0; l < 7; ++l) v += rp.f[l] * vl[0][l] + vl[1][l];
        if (df) reinterpret_cast<float2 *>(vbox)[inf.y] = make_float2(v, 0.f);   // double-float pair
        else vbox[inf.y] = (double)v;
    }
}

// One orbital's box seen from one pair: the box coordinates of the pair's grid
// offset m are MOD(b + m, N) with b = MOD(g_ij - lo, N) taken once per pair
// (the same as MOD(MOD(g_ij + m, N) - lo, N) of Eq. l2g, without the second
// wrap per point).
struct PairBox {
    int b[3];
    __device__ PairBox(const CellDev &C, const int32_t *lo, int o, const int *g)
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) b[a] = wrapi(g[a] - lo[3 * o + a], C.n[a]);
    }
    // element index in a box of size dim, or -1 outside it
    __device__ __forceinline__ long long at(const CellDev &C, const int *dim, int m0, int m1, int m2) const
    {
        const int u0 = wrapi(b[0] + m0, C.n[0]), u1 = wrapi(b[1] + m1, C.n[1]), u2 = wrapi(b[2] + m2, C.n[2]);
        if (u0 >= dim[0] || u1 >= dim[1] || u2 >= dim[2]) return -1;
        return ((long long)u0 * dim[1] + u1) * dim[2] + u2;
    }
};

// |b|^2 for b = 4 pi rho + L v with v zero on PE and the far field on the halo
// (v as double-float pairs), the stencil in FP32 and the sum in double-float.
// Only the stopping threshold tol |b| uses it when the CG starts from the
// multipole guess, whose residual (double-float) is the CG's first residual.
// L v vanishes at PE points without a halo point in the stencil's reach, so
// the caller passes each thread's part of sum (4 pi rho)^2 over all PE points
// (init, taken in the density pass) and only the boundary points are visited
// here, replacing (4 pi rho)^2 by b^2.
__device__ __noinline__ double bnorm2_f32(const SetDev &S, const float2 *__restrict__ vb,
                                          const float2 *__restrict__ b2, const float (*cw)[8], float center,
                                          const int *ds, int ndir, int fdn, float2 *red2, float2 init)
{
    DF a[1] = {{init.x, init.y}};
    for (int j = threadIdx.x; j < S.n_bnd; j += blockDim.x) {
        const int k = __ldg(S.bnd + j);
        const int off = S.pe_off[k];
        float acc = center * vb[off].x;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            if (d < ndir) {
                const int st = ds[d];
#pragma unroll
                for (int s_ = 1; s_ <= 6; ++s_)
                    if (s_ <= fdn) acc += cw[d][s_] * (vb[off + s_ * st].x + vb[off - s_ * st].x);
            }
        }
        const float2 q = b2[k];
        const float b = (q.x + acc) + q.y, b0 = q.x + q.y;
        df_fma(a[0], b, b);
        df_fma(a[0], -b0, b0);
    }
    block_sum_df<1>(a, red2);
    // block_sum_df leaves the total in warp 0: broadcast it
    __shared__ double s_bn2;
    if (threadIdx.x == 0) s_bn2 = (double)a[0].hi + (double)a[0].lo;
    __syncthreads();
    return s_bn2;
}

// D^i += v phi_j and D^j += v phi_i on the PE points and the shell (Eq. Dxx,
// Step V), v on the shell from the multipole expansion (Eq. me): FP32 Cartesian
// recurrences on the mixed path, the FP64 table otherwise.  Returns false when
// a non-zero value falls outside a D box.
__device__ __noinline__ bool d_scatter(const SetDev &S, const SmemCell &sm, const PairRec &pr,
                                       const double *__restrict__ vbox, bool self, bool mixed)
{
    const CellDev &C = sm.C;
    const PairBox fi(C, C.box_lo, pr.i, pr.g), fj(C, C.box_lo, pr.j, pr.g);
    const PairBox di(C, C.dbox_lo, pr.i, pr.g), dj(C, C.dbox_lo, pr.j, pr.g);
    const size_t bvol = (size_t)C.box[0] * C.box[1] * C.box[2], dvol = (size_t)C.dbox[0] * C.dbox[1] * C.dbox[2];
    const double *__restrict__ phi_i = C.phi + (size_t)pr.i * bvol;
    const double *__restrict__ phi_j = C.phi + (size_t)pr.j * bvol;
    double *dx_i = C.dxx + (size_t)pr.i * dvol;
    double *dx_j = C.dxx + (size_t)pr.j * dvol;
    bool ok = true;
    // U points per thread and step: their values, then their orbital values, then
    // the atomics, so that the loads of all U points are in flight together
    auto scatter = [&](auto U, const int *m, const double *v, const bool *live) {
        constexpr int u_n = decltype(U)::value;
        double f[u_n], g[u_n];
#pragma unroll
        for (int u = 0; u < u_n; ++u) {
            const long long a = live[u] ? fj.at(C, C.box, m[3 * u], m[3 * u + 1], m[3 * u + 2]) : -1;
            f[u] = a >= 0 ? __ldg(phi_j + a) : 0.0;
            const long long b = (live[u] && !self) ? fi.at(C, C.box, m[3 * u], m[3 * u + 1], m[3 * u + 2]) : -1;
            g[u] = b >= 0 ? __ldg(phi_i + b) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < u_n; ++u) {
            if (!live[u]) continue;
            const double val = v[u] * f[u];
            const long long d = di.at(C, C.dbox, m[3 * u], m[3 * u + 1], m[3 * u + 2]);
            if (d >= 0) atomicAdd(dx_i + d, val);
            else ok &= val == 0.0;
            if (!self) {
                const double val2 = v[u] * g[u];
                const long long d2 = dj.at(C, C.dbox, m[3 * u], m[3 * u + 1], m[3 * u + 2]);
                if (d2 >= 0) atomicAdd(dx_j + d2, val2);
                else ok &= val2 == 0.0;
            }
        }
    };
    const int nt = blockDim.x, npe = S.n_pe, nsh = S.n_shell;
    constexpr int kUpe = 2, kUsh = 1;
    for (int k0 = threadIdx.x; k0 < npe; k0 += kUpe * nt) {
        int m[3 * kUpe];
        double v[kUpe];
        bool live[kUpe];
#pragma unroll
        for (int u = 0; u < kUpe; ++u) {
            const int k = k0 + u * nt;
            live[u] = k < npe;
            const int kk = live[u] ? k : k0;
            unpack_m(__ldg(S.pe_m + kk), m[3 * u], m[3 * u + 1], m[3 * u + 2]);
            v[u] = vbox[__ldg(S.pe_off + kk)];
        }
        scatter(std::integral_constant<int, kUpe>(), m, v, live);
    }
    for (int s0 = threadIdx.x; s0 < nsh; s0 += kUsh * nt) {
        int m[3 * kUsh];
        double v[kUsh];
        bool live[kUsh];
#pragma unroll
        for (int u = 0; u < kUsh; ++u) {
            const int s = s0 + u * nt;
            live[u] = s < nsh;
            const int ss = live[u] ? s : s0;
            const int32_t pm = __ldg(S.sh_m + ss);
            unpack_m(pm, m[3 * u], m[3 * u + 1], m[3 * u + 2]);
            if (mixed) {
                float x, y, z;
                xyz_of(sm.hf, pm, x, y, z);
                const RinvPows rp(rsqrtf(x * x + y * y + z * z));
                float vl[1][7];
                solid_parts32<1>(x, y, z, C.lmax,
                                 [&](int l, int mm, float *k) {
                                     const float2 c = sm.cq2[l * l + l + mm];
                                     k[0] = c.x;
                                     k[1] = c.y;
                                 },
                                 vl);
                float vf = 0.f;
#pragma unroll
                for (int l = 0; l < 7; ++l) vf += rp.f[l] * vl[0][l];
                v[u] = vf;
            } else {
                double w = 0.0;
                for (int lm = 0; lm < kNlm; ++lm) w += sm.Q[lm] * __ldg(S.T64 + (size_t)lm * nsh + ss);
                v[u] = w;
            }
        }
        scatter(std::integral_constant<int, kUsh>(), m, v, live);
    }
    return ok;
}

template <class T>
__global__ void __launch_bounds__(kSolveThreads, kSolveMinBlocks) k_pair_solve(const CellDev *__restrict__ cells, ListDev L,
                                                                 SlotWork W, int inner_shift)
{
    __shared__ SmemCell sm;
    __shared__ double red[33 * 10 + 64];
    __shared__ double qpart[kSolveThreads / 32][kNlm];
    __shared__ float2 s_bpart[kSolveThreads];   // per thread: sum (4 pi rho)^2 of its PE points
    __shared__ int s_pair, s_cell, s_flag;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    char *slot = W.base + (size_t)blockIdx.x * W.slot_bytes;
    double *vbox = (double *)(slot + W.off_vbox);
    T *pbox = (T *)(slot + W.off_pbox);
    double *rho = (double *)(slot + W.off_rho);
    double *r64 = (double *)(slot + W.off_r64);
    T *rv = (T *)(slot + W.off_r);
    T *qv = (T *)(slot + W.off_q);
    T *ev = (T *)(slot + W.off_e);
    const bool mixed = sizeof(T) == 4;
    const double inner_red = ldexp(1.0, -inner_shift);   // inner FP32 solve residual reduction

    if (tid == 0) s_cell = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_pair = atomicAdd(L.queue, 1);
        __syncthreads();
        const int tq = s_pair;
        if (tq >= *L.total) break;
        const int t = L.perm ? L.perm[tq] : tq;   // this rank's share of the list (exx_plan_set_shard)
        const PairRec pr = L.pairs[t];
        if (pr.cell != s_cell) {
            // load the cell constants into shared memory
            const int *src = (const int *)&cells[pr.cell];
            int *dst = (int *)&sm.C;
            for (int k = tid; k < (int)(sizeof(CellDev) / sizeof(int)); k += nt) dst[k] = src[k];
            __syncthreads();
            if (tid < 48) {
                const int d = tid / 8, s = tid % 8;
                sm.cw64[d][s] = sm.C.cw64[d][s];
                sm.cw32[d][s] = sm.C.cw32[d][s];
                sm.cwdf[d][s] = dw_split(sm.C.cw64[d][s]);
            } else if (tid >= 64 && tid < 64 + kNlm) {
                const int lm = tid - 64;
                int l = 0;
                while ((l + 1) * (l + 1) <= lm) ++l;
                const int m = lm - l * l - l;
                float c = 0.f;
                if (m >= 0) {
                    double ratio = 1.0;   // (l-m)!/(l+m)!
                    for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
                    const double nlm = sqrt((2.0 * l + 1.0) / kFourPi * ratio);
                    c = (float)(m == 0 ? nlm : 1.4142135623730951 * nlm);
                }
                sm.cn[lm] = c;
            } else if (tid >= 128 && tid < 137) {
                const int a = (tid - 128) / 3, b = (tid - 128) % 3;
                sm.hf[a][b] = (float)(sm.C.h[a][b] / sm.C.n[b]);
            } else if (tid >= 160 && tid < 184) {
                const int a = (tid - 160) / 8, b = (tid - 160) % 8;
                sm.w1df[a][b] = dw_split(sm.C.w1dx[a][b]);
            }
            if (tid == 0) {
                double c = 0.0;
                for (int d = 0; d < sm.C.ndir; ++d) c += sm.C.cw64[d][0];
                sm.center64 = c;
                sm.center32 = (float)c;
                sm.centerdf = dw_split(c);
                s_cell = pr.cell;
            }
            __syncthreads();
        }
        const CellDev &C = sm.C;
        const int self = (pr.i == pr.j);
        const SetDev &S = C.set[self ? 0 : 1];
        if (tid < 6) sm.ds[tid] = S.dstride[tid];
        if (tid == 0) s_flag = 0;
        const int ndir = C.ndir, fdn = C.fd_n;
        // mixed pairs on the one-sweep CG hold v as double-float pairs in vbox while
        // they solve (converted to FP64 afterwards) and take every residual in
        // double-float arithmetic; the others keep FP64 throughout
        const bool dfm = mixed && fdn <= 4 &&
                         (S.n_groups + kSweepChunkGroups * nt - 1) / (kSweepChunkGroups * nt) <= kMaxSweepChunks;
        float2 *vb = reinterpret_cast<float2 *>(vbox);
        float2 *b2 = reinterpret_cast<float2 *>(slot + W.off_b2);
        float *r32 = reinterpret_cast<float *>(r64);
        auto residual = [&]() -> double {
            return dfm ? residual_df_n(fdn, S, vb, b2, r32, sm.cwdf, sm.centerdf, sm.ds, ndir, red)
                       : residual_pass(S, vbox, rho, r64, sm.cw64, sm.ds, ndir, fdn, sm.center64, red);
        };

        // ---- Step III: pair density on PE, g = MOD(g_ij + m, N) (Eq. l2g) ----
        {
            const PairBox fi(C, C.box_lo, pr.i, pr.g), fj(C, C.box_lo, pr.j, pr.g);
            const size_t bvol = (size_t)C.box[0] * C.box[1] * C.box[2];
            const double *__restrict__ phi_i = C.phi + (size_t)pr.i * bvol;
            const double *__restrict__ phi_j = C.phi + (size_t)pr.j * bvol;
            DF bq = {0.f, 0.f};   // this thread's part of sum (4 pi rho)^2 (bnorm2_f32)
            for (int k = tid; k < S.n_pe; k += nt) {
                int m0, m1, m2;
                unpack_m(__ldg(S.pe_m + k), m0, m1, m2);
                const long long a = fi.at(C, C.box, m0, m1, m2), b = fj.at(C, C.box, m0, m1, m2);
                const double rk = (a >= 0 ? __ldg(phi_i + a) : 0.0) * (b >= 0 ? __ldg(phi_j + b) : 0.0);
                rho[k] = rk;
                if (dfm) {
                    const float2 bb = dw_split(kFourPi * rk);
                    b2[k] = bb;
                    const float bf = bb.x + bb.y;
                    df_fma(bq, bf, bf);
                }
            }
            s_bpart[tid] = make_float2(bq.hi, bq.lo);
        }
        __syncthreads();

        // ---- multipole moments Q_lm = dV sum_PE rho r^l Y_lm (Eq. mepole) ----
        float *gs = reinterpret_cast<float *>(slot + W.off_gs);
        if (mixed && S.gs_perm) {
            // by radial bin: the same pass gives the moments of the starting guess
            bin_moments(S, C, rho, gs, qpart);
        } else {
            double a0 = 0.0, a1 = 0.0;
            const int nchunk = (S.n_pe + 31) >> 5;
            // 32 points per step (rows past the end repeat the last one with weight 0),
            // unrolled so that the table rows of several points are in flight at once
            const int lane1 = lane + 32 < kNlm ? lane + 32 : lane;
            const float sel1 = lane + 32 < kNlm ? 1.f : 0.f;
            for (int ch = warp; ch < nchunk; ch += nwarps) {
                const int k0 = ch << 5;
                const double rl = (k0 + lane < S.n_pe) ? rho[k0 + lane] : 0.0;
                const int last = min(32, S.n_pe - k0) - 1;
                if (mixed) {
                    float f0 = 0.f, f1 = 0.f;
                    const float rlf = (float)rl;
#pragma unroll 8
                    for (int p = 0; p < 32; ++p) {
                        const float rp = __shfl_sync(0xffffffffu, rlf, p);
                        const float *row = S.S32 + (size_t)(k0 + min(p, last)) * kNlm;
                        f0 += rp * row[lane];
                        f1 += rp * row[lane1];
                    }
                    a0 += f0;
                    a1 += sel1 * f1;
                } else {
                    double f0 = 0.0, f1 = 0.0;
#pragma unroll 4
                    for (int p = 0; p < 32; ++p) {
                        const double rp = __shfl_sync(0xffffffffu, rl, p);
                        const double *row = S.S64 + (size_t)(k0 + min(p, last)) * kNlm;
                        f0 += rp * row[lane];
                        f1 += rp * row[lane1];
                    }
                    a0 += f0;
                    a1 += sel1 * f1;
                }
            }
            qpart[warp][lane] = a0;
            if (lane + 32 < kNlm) qpart[warp][lane + 32] = a1;
        }
        {
            __syncthreads();
            if (tid < kNlm) {
                double s = 0.0;
                for (int w = 0; w < nwarps; ++w) s += qpart[w][tid];
                const double q = (tid < (C.lmax + 1) * (C.lmax + 1)) ? s * C.dv : 0.0;
                sm.Q[tid] = q;
                sm.Qf[tid] = (float)q;
                int l = 0;
                while ((l + 1) * (l + 1) <= tid) ++l;
                sm.Qc[tid] = (float)(kFourPi / (2 * l + 1) * q);
            }
            __syncthreads();
            if (tid < kNlm) {
                int l = 0;
                while ((l + 1) * (l + 1) <= tid) ++l;
                const int i0 = l * l + l, mm = tid - i0;
                sm.cq2[tid] = mm < 0 ? make_float2(0.f, 0.f)
                                     : make_float2(sm.cn[tid] * sm.Qc[tid], mm > 0 ? sm.cn[tid] * sm.Qc[i0 - mm] : 0.f);
            }
            __syncthreads();
        }

        // ---- far field on the halo (Eq. me): Dirichlet data in vbox ----
        for (int h = tid; h < S.n_halo; h += nt) {
            double v = 0.0;
            if (mixed) {
                float vf = 0.f;
                for (int lm = 0; lm < kNlm; ++lm) vf += sm.Qf[lm] * S.T32[(size_t)lm * S.n_shell + h];
                v = vf;
            } else {
                for (int lm = 0; lm < kNlm; ++lm) v += sm.Q[lm] * S.T64[(size_t)lm * S.n_shell + h];
            }
            if (dfm) vb[S.halo_off[h]] = make_float2((float)v, 0.f);
            else vbox[S.halo_off[h]] = v;
        }
        __syncthreads();

        // ---- Step IV: Poisson solve (Eq. pe) ----
        // b = 4 pi rho + (Dirichlet terms): the residual of v = 0 on PE.  When the CG
        // will start from the multipole guess (no warm start), only |b| is needed here
        const bool b_only = dfm && C.guess && S.gs_perm && !C.warm_map;
        double rr2 = b_only ? bnorm2_f32(S, vb, b2, sm.cw32, sm.center32, sm.ds, ndir, fdn,
                                         reinterpret_cast<float2 *>(red), s_bpart[tid])
                            : residual();
        const double bn = sqrt(rr2);
        const double stop = C.tol * bn;
        int iters = 0, refine = 1, status = 0;
        double rnorm = bn;
        // warm start: this pair's solution of the previous solve, moved by the
        // change of the grid-resolved centre, as the starting guess
        int warm = -1;
        int dg[3] = {0, 0, 0};
        if (C.warm_map && bn > 0.0) {
            const int o = C.warm_map[(size_t)pr.i * C.n_orb + pr.j];
            if (o >= 0) {
                const PairRec q = C.warm_rows[o];
                if (q.i == pr.i && q.j == pr.j && q.k[0] == pr.k[0] && q.k[1] == pr.k[1] && q.k[2] == pr.k[2]) {
                    warm = o;
                    for (int a = 0; a < 3; ++a) {
                        int d = wrapi(pr.g[a] - q.g[a], C.n[a]);
                        if (2 * d >= C.n[a]) d -= C.n[a];
                        dg[a] = d;
                    }
                }
            }
        }
        if (warm >= 0) {
            const int32_t *inv = C.warm_inv[self ? 0 : 1];
            const float *src = C.warm_prev + (size_t)warm * C.warm_stride;
            for (int k = tid; k < S.n_pe; k += nt) {
                int m0, m1, m2;
                unpack_m(S.pe_m[k], m0, m1, m2);
                const int u0 = m0 + dg[0] + S.c[0], u1 = m1 + dg[1] + S.c[1], u2 = m2 + dg[2] + S.c[2];
                double v = 0.0;
                if (u0 >= 0 && u0 < S.B[0] && u1 >= 0 && u1 < S.B[1] && u2 >= 0 && u2 < S.B[2]) {
                    const int kk = inv[((size_t)u0 * S.B[1] + u1) * S.B[2] + u2];
                    if (kk >= 0) v = (double)src[kk];
                }
                if (dfm) vb[S.pe_off[k]] = make_float2((float)v, 0.f);
                else vbox[S.pe_off[k]] = v;
            }
            __syncthreads();
            rnorm = sqrt(residual());
            rr2 = rnorm * rnorm;
            ++refine;
            // a previous solution that the pair has moved away from starts worse than
            // the multipole potential (typically 3-18 % of |b|): keep it only when close
            if (C.guess && S.gs_perm && !(rnorm <= kWarmAccept * bn)) warm = -1;
        }
        if (warm < 0 && C.guess && bn > 0.0 && S.gs_perm) {
            if (!mixed) {
                bin_moments(S, C, rho, gs, qpart);
                __syncthreads();
            }
            multipole_guess(S, C, sm.cn, sm.hf, vbox, gs, dfm);
            __syncthreads();
            rnorm = sqrt(residual());
            rr2 = rnorm * rnorm;
            ++refine;
        }
        double es[10];   // Step V sums of the double-float path (valid in thread 0)
        if (!mixed) {
            // plain FP64 CG: x in vbox (PE), r in r64, p in pbox, q in qv
            double *pd = (double *)pbox;
            double *qd = (double *)qv;
            double rr = rr2;
            if (bn > 0.0) {
                for (int k = tid; k < S.n_pe; k += nt) pd[S.pe_off[k]] = r64[k];
                __syncthreads();
                for (;;) {
                    if (sqrt(rr) <= stop) {
                        rr = residual_pass(S, vbox, rho, r64, sm.cw64, sm.ds, ndir, fdn, sm.center64, red);
                        ++refine;
                        if (sqrt(rr) <= stop) break;
                        for (int k = tid; k < S.n_pe; k += nt) pd[S.pe_off[k]] = r64[k];
                        __syncthreads();
                    }
                    if (iters >= C.max_iter) {
                        status = 5;
                        break;
                    }
                    double pq[1] = {0.0};
                    for (int k = tid; k < S.n_pe; k += nt) {
                        const int off = S.pe_off[k];
                        const double q = -lap_at<double>(pd, off, sm.cw64, sm.ds, ndir, fdn, sm.center64);
                        qd[k] = q;
                        pq[0] += pd[off] * q;
                    }
                    block_sum<1>(pq, red);
                    const double alpha = rr / pq[0];
                    double rn[1] = {0.0};
                    for (int k = tid; k < S.n_pe; k += nt) {
                        const int off = S.pe_off[k];
                        vbox[off] += alpha * pd[off];
                        const double r = r64[k] - alpha * qd[k];
                        r64[k] = r;
                        rn[0] += r * r;
                    }
                    block_sum<1>(rn, red);
                    const double beta = rn[0] / rr;
                    rr = rn[0];
                    for (int k = tid; k < S.n_pe; k += nt) {
                        const int off = S.pe_off[k];
                        pd[off] = r64[k] + beta * pd[off];
                    }
                    ++iters;
                    __syncthreads();
                }
                rnorm = sqrt(rr);
            }
        } else {
            CgMixed cg;
            cg.S = &S;
            cg.vbox = vbox;
            cg.rho = rho;
            cg.r64 = r64;
            cg.pf = (float *)pbox;
            cg.rf = (float *)rv;
            cg.qf = (float *)qv;
            cg.ef = (float *)ev;
            cg.sm = &sm;
            cg.red = red;
            cg.ndir = ndir;
            cg.fdn = fdn;
            cg.max_iter = C.max_iter;
            cg.stop = stop;
            cg.bn = bn;
            cg.r0n = rnorm;
            cg.inner_red = C.inner_shift > 0 ? ldexp(1.0, -C.inner_shift) : inner_red;
            cg.b2 = b2;
            if (dfm) {
                bool es_done = false;   // the CG's last residual pass took the Step V sums
                if (C.precond && S.mg && fdn <= 3) {
                    float *zf = reinterpret_cast<float *>(slot + W.off_zf);
                    float *mgb = reinterpret_cast<float *>(slot + W.off_mg);
                    switch (fdn) {
                    case 1: cg_mixed_mg<1>(cg, zf, mgb, iters, refine, status, rnorm, es, es_done); break;
                    case 2: cg_mixed_mg<2>(cg, zf, mgb, iters, refine, status, rnorm, es, es_done); break;
                    default: cg_mixed_mg<3>(cg, zf, mgb, iters, refine, status, rnorm, es, es_done); break;
                    }
                } else {
                    switch (fdn) {
                    case 1: cg_mixed_sweep<1>(cg, iters, refine, status, rnorm); break;
                    case 2: cg_mixed_sweep<2>(cg, iters, refine, status, rnorm); break;
                    case 3: cg_mixed_sweep<3>(cg, iters, refine, status, rnorm); break;
                    default: cg_mixed_sweep<4>(cg, iters, refine, status, rnorm); break;
                    }
                }
                __syncthreads();
                // Step V integrals from the double-float solution (unless the CG's last
                // residual pass took them)
                if (!es_done)
                    energy_stress_df(S, sm.w1df, vb, b2, C.stress_mode != 2, fdn, reinterpret_cast<float2 *>(red), es);
                // v back to FP64 on PE for D and the warm-start store
                for (int k = tid; k < S.n_pe; k += nt) {
                    const int off = S.pe_off[k];
                    const float2 t = vb[off];
                    vbox[off] = (double)t.x + (double)t.y;
                }
                __syncthreads();
            } else {
                cg_mixed(cg, iters, refine, status, rnorm);
            }
        }

        // keep this pair's solution for the next warm-started solve
        if (C.warm_next) {
            const int tl = t - L.cell_start[pr.cell];
            if (tl >= 0 && tl < C.warm_cap) {
                float *dst = C.warm_next + (size_t)tl * C.warm_stride;
                for (int k = tid; k < S.n_pe; k += nt) dst[k] = (float)vbox[S.pe_off[k]];
            }
        }

        // ---- Step V: energy and stress integrals (Eqs. exxGen_mlwf, sxx_working, d1_1) ----
        double acc[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] = dfm ? es[k] : 0.0;
        const bool want_sigma = C.stress_mode != 2;
        for (int k = tid; k < (dfm ? 0 : S.n_pe); k += nt) {
            const int off = S.pe_off[k];
            const double rk = rho[k];
            const double v = vbox[off];
            acc[0] += rk * v;
            if (!want_sigma) continue;
            double dxi[3];
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                const int st = S.gstride[al];
                double t = 0.0;
#pragma unroll
                for (int s = 1; s <= 6; ++s)
                    if (s <= fdn) t += C.w1dx[al][s] * (vbox[off + s * st] - vbox[off - s * st]);
                dxi[al] = t;
            }
            // sum_PE m_alpha rho d_b v; the lattice Jacobian and 1/N_alpha are
            // constant over the cell and applied to the nine sums once per pair
            int m0, m1, m2;
            unpack_m(S.pe_m[k], m0, m1, m2);
            const double mb[3] = {(double)m0, (double)m1, (double)m2};
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double rd = rk * dxi[b];
#pragma unroll
                for (int al = 0; al < 3; ++al) acc[1 + 3 * b + al] += mb[al] * rd;
            }
        }
        if (!dfm) block_sum<10>(acc, red);

        // ---- D^i += v phi_j, D^j += v phi_i on PE and shell (Eq. Dxx, Step V) ----
        if (C.dxx) {
            if (!d_scatter(S, sm, pr, vbox, self, mixed)) s_flag = 1;
        }

        // ---- restore the all-zero boxes for the next pair ----
        __syncthreads();
        for (int k = tid; k < S.n_pe; k += nt) {
            const int off = S.pe_off[k];
            vbox[off] = 0.0;
            pbox[off] = (T)0;
            if (mixed) {
                // dense FP32 boxes (group path) and compressed vectors (generic path)
                ((float *)rv)[off] = 0.f;
                ((float *)qv)[off] = 0.f;
                ((float *)ev)[off] = 0.f;
                ((float *)rv)[k] = 0.f;
                ((float *)qv)[k] = 0.f;
                ((float *)ev)[k] = 0.f;
                reinterpret_cast<float *>(slot + W.off_zf)[off] = 0.f;
            } else {
                ((double *)qv)[k] = 0.0;   // q of the FP64 CG (compressed); the other paths read this region as a box
            }
        }
        for (int h = tid; h < S.n_halo; h += nt) vbox[S.halo_off[h]] = 0.0;
        if (tid == 0) {
            PairOut o;
            o.e = acc[0] * C.dv;
            // sigma[a][alpha] = dV / N_alpha sum_b J[a][b] sum_PE m_alpha rho d_b v
            for (int a = 0; a < 3; ++a)
                for (int al = 0; al < 3; ++al)
                    o.sig[3 * a + al] = (C.J[a][0] * acc[1 + al] + C.J[a][1] * acc[4 + al] + C.J[a][2] * acc[7 + al]) /
                                        C.n[al] * C.dv;
            o.iters = iters;
            o.refine = refine;
            o.status = status ? status : (s_flag ? 7 : 0);
            o.pad = warm >= 0 ? 1 : 0;   // started from a previous solution
            L.out[t] = o;
        }
        (void)rnorm;
    }
}

// ===========================================================================
// Cluster path: one pair per cluster of kClusterCTAs CTAs.  The pair's FP32 CG
// state lives in the cluster's distributed shared memory: CTA c holds r, q, e
// of its contiguous range of aligned groups and p of the box rows that hold
// them (row partition of the set, built on the host); the stencil reads p of
// rows owned by other CTAs through shared::cluster loads.  Everything a pair
// needs outside the CG (density, moments, far field, FP64 residuals, x, E,
// sigma, D) is split over the CTAs by index range; CTA partial sums meet in
// shared memory and every CTA adds them in rank order, so all CTAs take the
// same decisions.
// ===========================================================================
struct ClusterWork {
    char *base;                 // per-cluster slots (v box, rho, FP64 residual)
    size_t slot_bytes;
    size_t off_vbox, off_rho, off_r64;
    int rowtab_words;           // row-table entries (largest B0 * B1 of the launch)
    int p_floats;               // floats of the p region (largest over sets and CTAs, multiple of 4)
    int max_groups;             // groups of r, q, e per CTA
};

__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_nrank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// Cluster-wide barrier: release of this thread's prior writes, acquire of the others'.
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cl_map(unsigned a, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 cl_ld4(unsigned a)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float cl_ld(unsigned a)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double cl_ldd(unsigned a)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ int cl_ldi(unsigned a)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void cl_st4(unsigned a, float x, float y, float z, float w)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
__device__ __forceinline__ void cl_st(unsigned a, float x)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(x) : "memory");
}

// Shared state of the cluster solver's reductions.
struct ClusterRed {
    double *red;                // CTA reduction scratch (block_sum)
    double (*part)[64];         // [2][64] this CTA's partial sums, double-buffered by reduction count
    double *out;                // [64] cluster totals, broadcast to the CTA
    int par;
    unsigned nrank;
};

// Sum K doubles over the cluster; every thread of every CTA receives the totals,
// added in rank order (identical in all CTAs).
template <int K>
__device__ __forceinline__ void cl_sum(double (&v)[K], ClusterRed &R)
{
    block_sum<K>(v, R.red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) R.part[R.par][k] = v[k];
    cl_sync();
    if (threadIdx.x < K) {
        const unsigned a = smem_u32(&R.part[R.par][threadIdx.x]);
        double acc = 0.0;
        for (unsigned c = 0; c < R.nrank; ++c) acc += cl_ldd(cl_map(a, c));
        R.out[threadIdx.x] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = R.out[k];
    R.par ^= 1;
}

// Sum K double-float values over the cluster in FP32 arithmetic; the totals
// (as doubles) end up in R.out[0..K) after the call, in every CTA alike.
template <int K>
__device__ __forceinline__ void cl_sum_df(DF (&v)[K], ClusterRed &R)
{
    float2 *red2 = reinterpret_cast<float2 *>(R.red);
    block_sum_df<K>(v, red2);
    float2 *mine = reinterpret_cast<float2 *>(R.part[R.par]);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) mine[k] = make_float2(v[k].hi, v[k].lo);
    cl_sync();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned a = smem_u32(mine);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            DF t = {0.f, 0.f};
            if (lane < (int)R.nrank) {
                const unsigned ak = cl_map(a + 8u * k, lane);
                t.hi = cl_ld(ak);
                t.lo = cl_ld(ak + 4u);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const DF u = {__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)};
                t = df_sum(t, u);
            }
            if (lane == 0) R.out[k] = (double)t.hi + (double)t.lo;
        }
    }
    __syncthreads();
    R.par ^= 1;
}

// FP64 residual b - A v (Eq. pe) on PE points k0 .. k1; returns this thread's sum of squares.
__device__ __forceinline__ double residual_range(const SetDev &S, const double *__restrict__ vbox,
                                                 const double *__restrict__ rho, double *__restrict__ r64,
                                                 const double (*cw)[8], const int *ds, int ndir, int n, double center,
                                                 int k0, int k1)
{
    double acc = 0.0;
    for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
        const int off = S.pe_off[k];
        const double r = kFourPi * rho[k] + lap_at<double>(vbox, off, cw, ds, ndir, n, center);
        r64[k] = r;
        acc += r * r;
    }
    return acc;
}

// Stencil of one own group with p read from the cluster's row storage.
template <int FDN>
__device__ __forceinline__ float4 cl_stencil(const unsigned *__restrict__ rowtab, int rid, int col, int mask,
                                             const float (*cw)[8], float center, const int *drow, const int *dcol,
                                             int ndir, float4 &cout)
{
    const unsigned rb = rowtab[rid] + 4u * (unsigned)col;
    const float4 c = cl_ld4(rb);
    const float4 cm = cl_ld4(rb - 16u);
    const float4 cp = cl_ld4(rb + 16u);
    const float x[12] = {cm.x, cm.y, cm.z, cm.w, c.x, c.y, c.z, c.w, cp.x, cp.y, cp.z, cp.w};
    float acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = center * x[4 + i];
#pragma unroll
    for (int s_ = 1; s_ <= FDN; ++s_)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += cw[2][s_] * (x[4 + i + s_] + x[4 + i - s_]);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (d == 2 || d >= ndir) continue;
        const int dr = drow[d], dc = dcol[d];
        if (dc == 0) {
#pragma unroll
            for (int s_ = 1; s_ <= FDN; ++s_) {
                const float4 a = cl_ld4(rowtab[rid + s_ * dr] + 4u * (unsigned)col);
                const float4 b = cl_ld4(rowtab[rid - s_ * dr] + 4u * (unsigned)col);
                acc[0] += cw[d][s_] * (a.x + b.x);
                acc[1] += cw[d][s_] * (a.y + b.y);
                acc[2] += cw[d][s_] * (a.z + b.z);
                acc[3] += cw[d][s_] * (a.w + b.w);
            }
        } else {
#pragma unroll
            for (int s_ = 1; s_ <= FDN; ++s_) {
                const unsigned pa = rowtab[rid + s_ * dr] + (unsigned)(4 * (col + s_ * dc));
                const unsigned pb = rowtab[rid - s_ * dr] + (unsigned)(4 * (col - s_ * dc));
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] += cw[d][s_] * (cl_ld(pa + 4u * i) + cl_ld(pb + 4u * i));
            }
        }
    }
    cout = c;
    return make_float4((mask & 1) ? -acc[0] : 0.f, (mask & 2) ? -acc[1] : 0.f, (mask & 4) ? -acc[2] : 0.f,
                       (mask & 8) ? -acc[3] : 0.f);
}

struct ClusterCg {
    const SetDev *S;
    const SmemCell *sm;
    double *vbox;
    const double *rho;
    double *r64;
    const unsigned *rowtab;
    float4 *r4, *q4, *e4;
    int G0, G1, K0, K1;
    int ndir, fdn, max_iter;
    double stop, bn, r0n, inner_red;
    const int *drow, *dcol;
};

// Mixed-precision CG of one pair on the cluster: the arithmetic of
// cg_mixed_sweep (FP32 in a frame scaled by the last true residual norm,
// line-search alpha, Hestenes-Stiefel beta, FP64 replacements with a
// conjugate restart), with the update of iteration k done before the stencil
// of iteration k+1 and one cluster barrier between them.
template <int FDN>
__device__ __forceinline__ void cg_cluster(const ClusterCg &g, ClusterRed &R, int &iters, int &refine, int &status,
                                           double &rnorm)
{
    const SetDev &S = *g.S;
    const SmemCell &sm = *g.sm;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ngo = g.G1 - g.G0;
    const int32_t *__restrict__ grp = S.groups;
    const int32_t *__restrict__ grc = S.cl_grc;
    const int32_t *__restrict__ pegl = S.cl_pe_gl;
    const unsigned *__restrict__ rowtab = g.rowtab;
    float4 *__restrict__ r4 = g.r4;
    float4 *__restrict__ q4 = g.q4;
    float4 *__restrict__ e4 = g.e4;
    const float(*cw)[8] = sm.cw32;
    const float center = sm.center32;
    if (!(g.bn > 0.0) || !(g.r0n > g.stop)) return;
    __shared__ struct {
        double rr, rmax, S, pq;
        float alpha, beta;
        int act;
    } cs;
    // first frame: r = p = (b - A v0) / |b - A v0| on own PE points
    {
        DF a[1] = {{0.f, 0.f}};
        const double sc = 1.0 / g.r0n;
        for (int k = g.K0 + tid; k < g.K1; k += nt) {
            const int gl = pegl[k];
            const int gi = gl >> 2, lane = gl & 3;
            const int w = grc[gi];
            const float r = (float)(g.r64[k] * sc);
            reinterpret_cast<float *>(&r4[gi - g.G0])[lane] = r;
            cl_st(rowtab[w & 8191] + 4u * (unsigned)((w >> 13) + lane), r);
            df_fma(a[0], r, r);
        }
        cl_sum_df<1>(a, R);
        if (tid == 0) {
            cs.rr = R.out[0];
            cs.rmax = sqrt(R.out[0]);
            cs.S = g.r0n;
        }
        __syncthreads();
    }
    bool pending = false;
    float alpha_p = 0.f, beta_p = 0.f;
    for (;;) {
        if (iters >= g.max_iter) {
            status = 5;
            break;
        }
        DF dv[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};   // <p,q> <q,q> <r,q> <r,p> <r,r>
        if (pending) {
            for (int lg = tid; lg < ngo; lg += nt) {
                const int w = grc[g.G0 + lg];
                const unsigned pa = rowtab[w & 8191] + 4u * (unsigned)(w >> 13);
                const float4 r = r4[lg], q = q4[lg], e = e4[lg], p_ = cl_ld4(pa);
                const float r0 = r.x - alpha_p * q.x, r1 = r.y - alpha_p * q.y, r2 = r.z - alpha_p * q.z,
                            r3 = r.w - alpha_p * q.w;
                df_add(dv[4], r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
                r4[lg] = make_float4(r0, r1, r2, r3);
                e4[lg] = make_float4(e.x + alpha_p * p_.x, e.y + alpha_p * p_.y, e.z + alpha_p * p_.z,
                                     e.w + alpha_p * p_.w);
                cl_st4(pa, r0 + beta_p * p_.x, r1 + beta_p * p_.y, r2 + beta_p * p_.z, r3 + beta_p * p_.w);
            }
        }
        cl_sync();   // every CTA's p rows are current
        for (int lg = tid; lg < ngo; lg += nt) {
            const int gi = g.G0 + lg;
            const int w = grc[gi];
            float4 c;
            const float4 q = cl_stencil<FDN>(rowtab, w & 8191, w >> 13, __ldg(grp + gi) & 15, cw, center, g.drow,
                                             g.dcol, g.ndir, c);
            q4[lg] = q;
            const float4 r = r4[lg];
            df_add(dv[0], c.x * q.x + c.y * q.y + c.z * q.z + c.w * q.w);
            df_add(dv[1], q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
            df_add(dv[2], r.x * q.x + r.y * q.y + r.z * q.z + r.w * q.w);
            df_add(dv[3], r.x * c.x + r.y * c.y + r.z * c.z + r.w * c.w);
        }
        cl_sum_df<5>(dv, R);
        if (tid == 0) {
            const double *d = R.out;
            const double rr_ = pending ? d[4] : cs.rr;
            const double alpha_d = d[3] / d[0];
            const double rn = rr_ - 2.0 * alpha_d * d[2] + alpha_d * alpha_d * d[1];
            const double rnrm = sqrt(fmax(rn, 0.0));
            const bool breakdown = !(d[0] > 0.0) || !(d[3] > 0.0) || !(alpha_d < 1e300);
            int act = 0;
            if (breakdown) act = 2;
            else if (!(rn > 0.0) || rnrm <= g.inner_red * cs.rmax || rnrm * cs.S <= 0.5 * g.stop) act = 1;
            cs.alpha = breakdown ? 0.f : (float)alpha_d;
            cs.beta = breakdown ? 0.f : (float)(-(d[2] - alpha_d * d[1]) / d[0]);
            cs.pq = d[0];
            cs.rr = rn;
            cs.act = act;
        }
        __syncthreads();
        const int act = cs.act;
        const float alpha = cs.alpha;
        pending = false;
        ++iters;
        if (act) {
            // x += S (e + alpha p) in FP64 on own PE points
            const double S_ = cs.S;
            for (int k = g.K0 + tid; k < g.K1; k += nt) {
                const int gl = pegl[k];
                const int gi = gl >> 2, lane = gl & 3;
                const int w = grc[gi];
                float *ep = reinterpret_cast<float *>(&e4[gi - g.G0]) + lane;
                const float pv = cl_ld(rowtab[w & 8191] + 4u * (unsigned)((w >> 13) + lane));
                g.vbox[S.pe_off[k]] += ((double)*ep + (double)alpha * (double)pv) * S_;
                *ep = 0.f;
            }
            __threadfence();
            cl_sync();
            double rr2[1] = {residual_range(S, g.vbox, g.rho, g.r64, sm.cw64, sm.ds, g.ndir, g.fdn, sm.center64,
                                            g.K0, g.K1)};
            cl_sum<1>(rr2, R);
            rnorm = sqrt(rr2[0]);
            ++refine;
            if (rnorm <= g.stop) break;
            const double sc = 1.0 / rnorm;
            DF ab[2] = {{0.f, 0.f}, {0.f, 0.f}};
            for (int k = g.K0 + tid; k < g.K1; k += nt) {
                const int gl = pegl[k];
                const int lg = (gl >> 2) - g.G0, lane = gl & 3;
                const float r = (float)(g.r64[k] * sc);
                reinterpret_cast<float *>(&r4[lg])[lane] = r;
                df_fma(ab[0], r, r);
                df_fma(ab[1], r, reinterpret_cast<const float *>(&q4[lg])[lane]);
            }
            cl_sum_df<2>(ab, R);
            if (tid == 0) {
                cs.beta = act == 2 ? 0.f : (float)(-R.out[1] / cs.pq);   // gamma of the carried direction
                cs.rr = R.out[0];
                cs.rmax = sqrt(R.out[0]);
                cs.S = rnorm;
            }
            __syncthreads();
            const float gamma = cs.beta;
            for (int lg = tid; lg < ngo; lg += nt) {
                const int w = grc[g.G0 + lg];
                const unsigned pa = rowtab[w & 8191] + 4u * (unsigned)(w >> 13);
                const float4 r = r4[lg], p_ = cl_ld4(pa);
                cl_st4(pa, r.x + gamma * p_.x, r.y + gamma * p_.y, r.z + gamma * p_.z, r.w + gamma * p_.w);
            }
            continue;
        }
        alpha_p = alpha;
        beta_p = cs.beta;
        pending = true;
    }
}

__global__ void __launch_bounds__(kClusterThreads, 1) k_pair_solve_cluster(const CellDev *__restrict__ cells, ListDev L,
                                                                         ClusterWork W, int inner_shift)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ SmemCell sm;
    __shared__ double red[33 * 10 + 64];
    __shared__ double s_part[2][64];
    __shared__ double s_out[64];
    __shared__ int s_pair, s_t, s_cell, s_set, s_flag;
    __shared__ int s_drow[6], s_dcol[6];

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const unsigned rank = cl_rank(), nrank = cl_nrank();
    char *slot = W.base + (size_t)cl_id() * W.slot_bytes;
    double *vbox = (double *)(slot + W.off_vbox);
    double *rho = (double *)(slot + W.off_rho);
    double *r64 = (double *)(slot + W.off_r64);
    unsigned *rowtab = reinterpret_cast<unsigned *>(dyn);
    float *preg = reinterpret_cast<float *>(dyn + (((size_t)4 * W.rowtab_words + 15) & ~(size_t)15));
    float4 *r4 = reinterpret_cast<float4 *>(preg + W.p_floats);
    float4 *q4 = r4 + W.max_groups;
    float4 *e4 = q4 + W.max_groups;
    const unsigned p_s = smem_u32(preg);
    const double inner_red = ldexp(1.0, -inner_shift);
    ClusterRed R;
    R.red = red;
    R.part = s_part;
    R.out = s_out;
    R.par = 0;
    R.nrank = nrank;

    if (tid == 0) {
        s_cell = -1;
        s_set = -1;
    }
    for (;;) {
        if (rank == 0 && tid == 0) s_pair = atomicAdd(L.queue, 1);
        cl_sync();
        if (tid == 0) s_t = cl_ldi(cl_map(smem_u32(&s_pair), 0));
        __syncthreads();
        const int tq = s_t;
        if (tq >= *L.total) break;
        const int t = L.perm ? L.perm[tq] : tq;
        const PairRec pr = L.pairs[t];
        const int self = (pr.i == pr.j);
        if (pr.cell != s_cell) {
            const int *src = (const int *)&cells[pr.cell];
            int *dst = (int *)&sm.C;
            for (int k = tid; k < (int)(sizeof(CellDev) / sizeof(int)); k += nt) dst[k] = src[k];
            __syncthreads();
            if (tid < 48) {
                const int d = tid / 8, s = tid % 8;
                sm.cw64[d][s] = sm.C.cw64[d][s];
                sm.cw32[d][s] = sm.C.cw32[d][s];
            }
            if (tid == 0) {
                double c = 0.0;
                for (int d = 0; d < sm.C.ndir; ++d) c += sm.C.cw64[d][0];
                sm.center64 = c;
                sm.center32 = (float)c;
                s_cell = pr.cell;
                s_set = -1;
            }
            __syncthreads();
        }
        const CellDev &C = sm.C;
        const SetDev &S = C.set[self ? 0 : 1];
        const int ndir = C.ndir, fdn = C.fd_n;
        if (s_set != self) {
            // row table of this set: shared::cluster address of column 0 of every box row
            const int nrows = S.B[0] * S.B[1];
            for (int rid = tid; rid < nrows; rid += nt) {
                const int own = S.cl_rows[2 * rid];
                unsigned a = 0;
                if (own >= 0) a = cl_map(p_s + 4u * (unsigned)S.cl_rows[2 * rid + 1], (unsigned)own);
                else if (own == -2) a = cl_map(p_s + 4u * (unsigned)S.cl_pad, rank);
                rowtab[rid] = a;
            }
            if (tid < 6) {
                s_drow[tid] = tid < ndir ? C.dir[tid][0] * S.B[1] + C.dir[tid][1] : 0;
                s_dcol[tid] = tid < ndir ? C.dir[tid][2] : 0;
                sm.ds[tid] = S.dstride[tid];
            }
            __syncthreads();
            if (tid == 0) s_set = self;
        }
        if (tid == 0) s_flag = 0;
        const int32_t *cta = S.cl_cta + 8 * rank;
        const int G0 = cta[0], G1 = cta[1], K0 = cta[2], K1 = cta[3];
        __syncthreads();

        // ---- Step III: pair density on own PE points (Eq. l2g) ----
        for (int k = K0 + tid; k < K1; k += nt) {
            int m0, m1, m2;
            unpack_m(S.pe_m[k], m0, m1, m2);
            const int g0 = wrapi(pr.g[0] + m0, C.n[0]), g1 = wrapi(pr.g[1] + m1, C.n[1]),
                      g2 = wrapi(pr.g[2] + m2, C.n[2]);
            rho[k] = phi_at(C, pr.i, g0, g1, g2) * phi_at(C, pr.j, g0, g1, g2);
        }
        __syncthreads();

        // ---- moments Q_lm (Eq. mepole): own PE points, then the cluster sum ----
        {
            double *wpart = reinterpret_cast<double *>(q4);   // [nwarps][kNlm] scratch (CG state not live yet)
            double a0 = 0.0, a1 = 0.0;
            const int nchunk = (K1 - K0 + 31) >> 5;
            for (int ch = warp; ch < nchunk; ch += nwarps) {
                const int k0 = K0 + (ch << 5);
                const float rlf = (k0 + lane < K1) ? (float)rho[k0 + lane] : 0.f;
                const int cnt = min(32, K1 - k0);
                float f0 = 0.f, f1 = 0.f;
                for (int p = 0; p < cnt; ++p) {
                    const float rp = __shfl_sync(0xffffffffu, rlf, p);
                    const float *row = S.S32 + (size_t)(k0 + p) * kNlm;
                    f0 += rp * row[lane];
                    if (lane + 32 < kNlm) f1 += rp * row[lane + 32];
                }
                a0 += f0;
                a1 += f1;
            }
            wpart[warp * kNlm + lane] = a0;
            if (lane + 32 < kNlm) wpart[warp * kNlm + lane + 32] = a1;
            __syncthreads();
            if (tid < kNlm) {
                double s = 0.0;
                for (int w = 0; w < nwarps; ++w) s += wpart[w * kNlm + tid];
                s_part[R.par][tid] = s;
            }
            cl_sync();
            if (tid < kNlm) {
                const unsigned a = smem_u32(&s_part[R.par][tid]);
                double s = 0.0;
                for (unsigned c = 0; c < nrank; ++c) s += cl_ldd(cl_map(a, c));
                const double q = (tid < (C.lmax + 1) * (C.lmax + 1)) ? s * C.dv : 0.0;
                sm.Q[tid] = q;
                sm.Qf[tid] = (float)q;
            }
            R.par ^= 1;
            __syncthreads();
        }

        // ---- far field on this CTA's share of the halo (Eq. me) ----
        {
            const int h0 = (int)(((long long)S.n_halo * rank) / nrank);
            const int h1 = (int)(((long long)S.n_halo * (rank + 1)) / nrank);
            for (int h = h0 + tid; h < h1; h += nt) {
                float vf = 0.f;
                for (int lm = 0; lm < kNlm; ++lm) vf += sm.Qf[lm] * S.T32[(size_t)lm * S.n_shell + h];
                vbox[S.halo_off[h]] = vf;
            }
        }
        // CG state of this CTA: all zero (p rows including the zero row; r, q, e)
        for (int i = tid; i < (W.p_floats >> 2); i += nt)
            reinterpret_cast<float4 *>(preg)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = tid; i < G1 - G0; i += nt) {
            r4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            q4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            e4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __threadfence();
        cl_sync();

        // ---- Step IV: Poisson solve (Eq. pe) ----
        double bb[1] = {residual_range(S, vbox, rho, r64, sm.cw64, sm.ds, ndir, fdn, sm.center64, K0, K1)};
        cl_sum<1>(bb, R);
        const double bn = sqrt(bb[0]);
        const double stop = C.tol * bn;
        int iters = 0, refine = 1, status = 0;
        double rnorm = bn;
        int warm = -1;
        int dg[3] = {0, 0, 0};
        if (C.warm_map && bn > 0.0) {
            const int o = C.warm_map[(size_t)pr.i * C.n_orb + pr.j];
            if (o >= 0) {
                const PairRec q = C.warm_rows[o];
                if (q.i == pr.i && q.j == pr.j && q.k[0] == pr.k[0] && q.k[1] == pr.k[1] && q.k[2] == pr.k[2]) {
                    warm = o;
                    for (int a = 0; a < 3; ++a) {
                        int d = wrapi(pr.g[a] - q.g[a], C.n[a]);
                        if (2 * d >= C.n[a]) d -= C.n[a];
                        dg[a] = d;
                    }
                }
            }
        }
        if (warm >= 0) {
            const int32_t *inv = C.warm_inv[self ? 0 : 1];
            const float *src = C.warm_prev + (size_t)warm * C.warm_stride;
            for (int k = K0 + tid; k < K1; k += nt) {
                int m0, m1, m2;
                unpack_m(S.pe_m[k], m0, m1, m2);
                const int u0 = m0 + dg[0] + S.c[0], u1 = m1 + dg[1] + S.c[1], u2 = m2 + dg[2] + S.c[2];
                double v = 0.0;
                if (u0 >= 0 && u0 < S.B[0] && u1 >= 0 && u1 < S.B[1] && u2 >= 0 && u2 < S.B[2]) {
                    const int kk = inv[((size_t)u0 * S.B[1] + u1) * S.B[2] + u2];
                    if (kk >= 0) v = (double)src[kk];
                }
                vbox[S.pe_off[k]] = v;
            }
            __threadfence();
            cl_sync();
            double r0[1] = {residual_range(S, vbox, rho, r64, sm.cw64, sm.ds, ndir, fdn, sm.center64, K0, K1)};
            cl_sum<1>(r0, R);
            rnorm = sqrt(r0[0]);
            ++refine;
        }
        {
            ClusterCg g;
            g.S = &S;
            g.sm = &sm;
            g.vbox = vbox;
            g.rho = rho;
            g.r64 = r64;
            g.rowtab = rowtab;
            g.r4 = r4;
            g.q4 = q4;
            g.e4 = e4;
            g.G0 = G0;
            g.G1 = G1;
            g.K0 = K0;
            g.K1 = K1;
            g.ndir = ndir;
            g.fdn = fdn;
            g.max_iter = C.max_iter;
            g.stop = stop;
            g.bn = bn;
            g.r0n = rnorm;
            g.inner_red = inner_red;
            g.drow = s_drow;
            g.dcol = s_dcol;
            switch (fdn) {
            case 1: cg_cluster<1>(g, R, iters, refine, status, rnorm); break;
            case 2: cg_cluster<2>(g, R, iters, refine, status, rnorm); break;
            case 3: cg_cluster<3>(g, R, iters, refine, status, rnorm); break;
            default: cg_cluster<4>(g, R, iters, refine, status, rnorm); break;
            }
        }
        // the final x of every CTA is visible to all CTAs of the cluster
        __threadfence();
        cl_sync();

        if (C.warm_next) {
            const int tl = t - L.cell_start[pr.cell];
            if (tl >= 0 && tl < C.warm_cap) {
                float *dst = C.warm_next + (size_t)tl * C.warm_stride;
                for (int k = K0 + tid; k < K1; k += nt) dst[k] = (float)vbox[S.pe_off[k]];
            }
        }

        // ---- D^i += v phi_j, D^j += v phi_i on this CTA's share of PE and shell (Eq. Dxx) ----
        if (C.dxx) {
            bool ok = true;
            const int nme = S.n_pe + S.n_shell;
            const int q0 = (int)(((long long)nme * rank) / nrank), q1 = (int)(((long long)nme * (rank + 1)) / nrank);
            for (int k = q0 + tid; k < q1; k += nt) {
                int m0, m1, m2;
                double v;
                if (k < S.n_pe) {
                    unpack_m(S.pe_m[k], m0, m1, m2);
                    v = vbox[S.pe_off[k]];
                } else {
                    const int s = k - S.n_pe;
                    unpack_m(S.sh_m[s], m0, m1, m2);
                    float vf = 0.f;
                    for (int lm = 0; lm < kNlm; ++lm) vf += sm.Qf[lm] * S.T32[(size_t)lm * S.n_shell + s];
                    v = vf;
                }
                const int g0 = wrapi(pr.g[0] + m0, C.n[0]), g1 = wrapi(pr.g[1] + m1, C.n[1]),
                          g2 = wrapi(pr.g[2] + m2, C.n[2]);
                const double fj = phi_at(C, pr.j, g0, g1, g2);
                ok &= d_add(C, pr.i, g0, g1, g2, v * fj);
                if (!self) {
                    const double fi = phi_at(C, pr.i, g0, g1, g2);
                    ok &= d_add(C, pr.j, g0, g1, g2, v * fi);
                }
            }
            if (!ok) s_flag = 1;
        }

        // ---- Step V: energy and stress integrals on own PE points, cluster sums ----
        double acc[11];
#pragma unroll
        for (int k = 0; k < 11; ++k) acc[k] = 0.0;
        const bool want_sigma = C.stress_mode != 2;
        for (int k = K0 + tid; k < K1; k += nt) {
            const int off = S.pe_off[k];
            const double rk = rho[k];
            acc[0] += rk * vbox[off];
            if (!want_sigma) continue;
            double dxi[3];
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                const int st = S.gstride[al];
                double tt = 0.0;
#pragma unroll
                for (int s = 1; s <= 6; ++s)
                    if (s <= fdn) tt += C.w1dx[al][s] * (vbox[off + s * st] - vbox[off - s * st]);
                dxi[al] = tt;
            }
            int m0, m1, m2;
            unpack_m(S.pe_m[k], m0, m1, m2);
            const double mb[3] = {(double)m0, (double)m1, (double)m2};
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double rd = rk * dxi[b];
#pragma unroll
                for (int al = 0; al < 3; ++al) acc[1 + 3 * b + al] += mb[al] * rd;
            }
        }
        __syncthreads();
        if (tid == 0) acc[10] = s_flag ? 1.0 : 0.0;
        cl_sum<11>(acc, R);
        if (rank == 0 && tid == 0) {
            PairOut o;
            o.e = acc[0] * C.dv;
            // sigma[a][alpha] = dV / N_alpha sum_b J[a][b] sum_PE m_alpha rho d_b v
            for (int a = 0; a < 3; ++a)
                for (int al = 0; al < 3; ++al)
                    o.sig[3 * a + al] = (C.J[a][0] * acc[1 + al] + C.J[a][1] * acc[4 + al] + C.J[a][2] * acc[7 + al]) /
                                        C.n[al] * C.dv;
            o.iters = iters;
            o.refine = refine;
            o.status = status ? status : (acc[10] > 0.0 ? 7 : 0);
            o.pad = warm >= 0 ? 1 : 0;
            L.out[t] = o;
        }
        // every CTA has read v (epilogue, D); restore the all-zero v box
        cl_sync();
        for (int k = K0 + tid; k < K1; k += nt) vbox[S.pe_off[k]] = 0.0;
        {
            const int h0 = (int)(((long long)S.n_halo * rank) / nrank);
            const int h1 = (int)(((long long)S.n_halo * (rank + 1)) / nrank);
            for (int h = h0 + tid; h < h1; h += nt) vbox[S.halo_off[h]] = 0.0;
        }
        __threadfence();
    }
    cl_sync();   // no CTA leaves while another may still read its shared memory
}

// Ordered per-cell reductions (Eqs. exxGen_mlwf, sxx_working, pixx_working).
__global__ void __launch_bounds__(256) k_finalize(const CellDev *__restrict__ cells, ListDev L, CellResult *res)
{
    const int c = blockIdx.x;
    const CellDev &C = cells[c];
    __shared__ double red[33 * 10 + 64];
    __shared__ int s_fail, s_status, s_maxit, s_maxref, s_warm;
    __shared__ unsigned long long s_tot, s_tref;
    if (threadIdx.x == 0) {
        s_warm = 0;
        s_fail = 0x7fffffff;
        s_status = 0;
        s_maxit = 0;
        s_maxref = 0;
        s_tot = 0ull;
        s_tref = 0ull;
    }
    __syncthreads();
    const int start = *L.overflow ? 0 : L.cell_start[c];
    const int cnt = *L.overflow ? 0 : L.cell_count[c];
    double acc[10];
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    // contiguous chunks per thread: a fixed summation order
    const int per = (cnt + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * per, p1 = min(cnt, p0 + per);
    long long tot = 0, tref = 0;
    int maxit = 0, maxref = 0, fail = 0x7fffffff, status = 0, nwarm = 0;
    for (int p = p0; p < p1; ++p) {
        const PairRec pr = L.pairs[start + p];
        const PairOut o = L.out[start + p];
        const double w = (pr.i == pr.j) ? 1.0 : 2.0;
        acc[0] += w * o.e;
        for (int k = 0; k < 9; ++k) acc[1 + k] += w * o.sig[k];
        tot += o.iters;
        tref += o.refine;
        nwarm += o.pad;
        maxit = max(maxit, o.iters);
        maxref = max(maxref, o.refine);
        if (o.status && p < fail) {
            fail = p;
            status = o.status;
        }
    }
    block_sum<10>(acc, red);
    atomicMax(&s_maxit, maxit);
    atomicMax(&s_maxref, maxref);
    atomicAdd(&s_tot, (unsigned long long)tot);
    atomicAdd(&s_tref, (unsigned long long)tref);
    atomicMin(&s_fail, fail);
    atomicAdd(&s_warm, nwarm);
    __syncthreads();
    if (fail == s_fail && fail != 0x7fffffff) s_status = status;
    __syncthreads();
    if (threadIdx.x == 0) {
        CellResult r;
        r.e_xx = -acc[0];
        for (int k = 0; k < 9; ++k) r.dedh[k] = -2.0 * acc[1 + k];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int al = 0; al < 3; ++al) s += r.dedh[3 * a + al] * C.h[b][al];
                r.stress[3 * a + b] = -s / C.vol;
            }
        r.total_iter = (long long)s_tot;
        r.total_refine = (long long)s_tref;
        r.n_pairs = cnt;
        r.status = *L.overflow ? 6 : s_status;
        r.failed_pair = (s_fail == 0x7fffffff) ? -1 : s_fail;
        r.max_iter = s_maxit;
        r.max_refine = s_maxref;
        r.pad = s_warm;   // pairs that started from a previous solution
        res[c] = r;
    }
}

// ---------------------------------------------------------------------------
// Host-side launch wrappers.
// ---------------------------------------------------------------------------
cudaError_t launch_tables(const CellDev *cell, int which, int n_points, double *S64, float *S32, double *T64,
                          float *T32, cudaStream_t s)
{
    const int threads = 128;
    const int blocks = (n_points + threads - 1) / threads;
    if (blocks > 0) k_tables<<<blocks, threads, 0, s>>>(cell, which, S64, S32, T64, T32);
    return cudaGetLastError();
}

// dst[j] = src[perm[j]], rows of kNlm floats (the solid-harmonic table in radial-bin order)
__global__ void k_gather_rows(const float *__restrict__ src, const int32_t *__restrict__ perm, int n,
                              float *__restrict__ dst)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (long long)n * kNlm) {
        const int j = (int)(i / kNlm), lm = (int)(i % kNlm);
        dst[i] = src[(size_t)perm[j] * kNlm + lm];
    }
}

cudaError_t launch_gather_rows(const float *src, const int32_t *perm, int n, float *dst, cudaStream_t s)
{
    const long long total = (long long)n * kNlm;
    if (total > 0) k_gather_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(src, perm, n, dst);
    return cudaGetLastError();
}

__global__ void k_guess_info(const int32_t *__restrict__ perm, const uint8_t *__restrict__ bin,
                             const int32_t *__restrict__ pe_m, const int32_t *__restrict__ pe_off, int n,
                             int4 *__restrict__ info)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        const int k = perm[j];
        info[j] = make_int4(pe_m[k], pe_off[k], (int)bin[k], k);
    }
}

cudaError_t launch_guess_info(const int32_t *perm, const uint8_t *bin, const int32_t *pe_m, const int32_t *pe_off,
                              int n, int4 *info, cudaStream_t s)
{
    if (n > 0) k_guess_info<<<(n + 255) / 256, 256, 0, s>>>(perm, bin, pe_m, pe_off, n, info);
    return cudaGetLastError();
}

cudaError_t launch_pair_list(const CellDev *cells, int n_cells, int n_rows, const ListDev &L, cudaStream_t s)
{
    if (n_rows > 0) k_pair_rows<<<n_rows, kRowThreads, 0, s>>>(cells, n_cells, L, 0);
    k_pair_scan<<<1, 1024, 0, s>>>(cells, n_cells, n_rows, L);
    if (n_rows > 0) k_pair_rows<<<n_rows, kRowThreads, 0, s>>>(cells, n_cells, L, 1);
    return cudaGetLastError();
}

cudaError_t launch_solve(const CellDev *cells, const ListDev &L, const SolveSlots &slots, bool mixed,
                         int inner_shift, cudaStream_t s)
{
    SlotWork W;
    W.base = slots.base;
    W.slot_bytes = slots.slot_bytes;
    W.off_vbox = slots.off_vbox;
    W.off_pbox = slots.off_pbox;
    W.off_rho = slots.off_rho;
    W.off_r64 = slots.off_r64;
    W.off_r = slots.off_r;
    W.off_q = slots.off_q;
    W.off_e = slots.off_e;
    W.off_gs = slots.off_gs;
    W.off_b2 = slots.off_b2;
    W.off_zf = slots.off_zf;
    W.off_mg = slots.off_mg;
    if (mixed) k_pair_solve<float><<<slots.n_slots, kSolveThreads, 0, s>>>(cells, L, W, inner_shift);
    else k_pair_solve<double><<<slots.n_slots, kSolveThreads, 0, s>>>(cells, L, W, inner_shift);
    return cudaGetLastError();
}

// map[i n_orb + j] = t for the pairs t of a cell's list (the warm-start index)
__global__ void k_warm_map(const PairRec *__restrict__ rows, int n, int n_orb, int *__restrict__ map)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const PairRec r = rows[t];
        if (r.i >= 0 && r.j >= 0 && r.i < n_orb && r.j < n_orb) map[(size_t)r.i * n_orb + r.j] = t;
    }
}

cudaError_t launch_warm_map(const PairRec *rows, int n, int n_orb, int *map, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_warm_map<<<(n + 255) / 256, 256, 0, s>>>(rows, n, n_orb, map);
    return cudaGetLastError();
}

// Limit the solver's queue to the first `limit` pairs (schedule autotuning).
__global__ void k_clamp_total(ListDev L, int limit)
{
    if (threadIdx.x == 0 && *L.total > limit) *L.total = limit;
}
cudaError_t launch_clamp_total(const ListDev &L, int limit, cudaStream_t s)
{
    k_clamp_total<<<1, 32, 0, s>>>(L, limit);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const CellDev *cells, int n_cells, const ListDev &L, CellResult *res, cudaStream_t s)
{
    k_finalize<<<n_cells, 256, 0, s>>>(cells, L, res);
    return cudaGetLastError();
}

}  // namespace exx

namespace exx {
cudaError_t launch_solve_cluster(const CellDev *cells, const ListDev &L, const SolveSlots &slots, int rowtab_words,
                                 int p_floats, int max_groups, int inner_shift, int *n_clusters, cudaStream_t s)
{
    ClusterWork W;
    W.base = slots.base;
    W.slot_bytes = slots.slot_bytes;
    W.off_vbox = slots.off_vbox;
    W.off_rho = slots.off_rho;
    W.off_r64 = slots.off_r64;
    W.rowtab_words = rowtab_words;
    W.p_floats = (p_floats + 3) & ~3;
    W.max_groups = max_groups;
    const size_t dyn = cluster_dyn_bytes(rowtab_words, p_floats, max_groups);
    cudaError_t e = cudaFuncSetAttribute(k_pair_solve_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pair_solve_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCTAs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(kClusterCTAs, 1, 1);
    int nc = 0;
    e = cudaOccupancyMaxActiveClusters(&nc, k_pair_solve_cluster, &cfg);
    if (e != cudaSuccess) return e;
    nc = std::min(nc, slots.n_slots);
    if (nc < 1) return cudaErrorInvalidConfiguration;
    cfg.gridDim = dim3(kClusterCTAs * nc, 1, 1);
    *n_clusters = nc;
    return cudaLaunchKernelEx(&cfg, k_pair_solve_cluster, cells, L, W, inner_shift);
}

int cluster_capacity_bytes()
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_pair_solve_cluster) != cudaSuccess) return 0;
    return std::max(0, optin - (int)fa.sharedSizeBytes - 1024);
}

int solve_blocks_per_sm(bool mixed)
{
    int n = 0;
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair_solve<float>, kSolveThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pair_solve<double>, kSolveThreads, 0);
    return n;
}
}  // namespace exx
