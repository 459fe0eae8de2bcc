// noalloc.cu -- a pair-list entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc at the moment they need the pair list:
// code running while a CUDA graph is being captured with a fixed memory
// budget, engines whose device memory is handed out once by their own pool,
// or callers embedded in a process whose allocator must not be re-entered.
// exx_pair_list_noalloc builds the same unique pair list as the solve entry
// points (same arithmetic, bit for bit), but its scratch -- the per-row pair
// counts and row offsets -- lives in the file-scope device array below, which
// every GPU that loads the library holds until the process exits.  The caller
// passes the centres and receives the rows and the count in its own device
// buffers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/exx.h"
#include "plan.h"

namespace {

constexpr int kMaxOrbNoalloc = 16384;          // rows the static scratch can hold
constexpr int kThreads = 128;

// [0, kMax) pair count of each row, [kMax, 2 kMax) first pair of each row,
// [2 kMax] total number of pairs.
__device__ __align__(256) int g_pairlist_scratch[2 * kMaxOrbNoalloc + 64];

struct PairCell {
    double h[3][3], hinv[3][3];
    int n[3];
    double r_pair2;
    const double *centres;
    int n_orb;
};

__device__ __forceinline__ double dot3(const double *r, double a, double b, double c)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(r[0], a), __dmul_rn(r[1], b)), __dmul_rn(r[2], c));
}

// The written rule of the pair list: s = h^-1 C, ds = s_j - s_i - round(ds), the
// lattice image k in {-1,0,1}^3 (lexicographic, first minimum) with the smallest
// |h(ds+k)|^2, kept when <= R_pair^2; centre g = NINT(N (s_i + (ds+k)/2)) mod N.
__device__ bool pair_rule(const PairCell &C, int i, int j, int *kb, int *g)
{
    const double *ci = C.centres + 3 * i, *cj = C.centres + 3 * j;
    double si[3], ds[3];
    for (int a = 0; a < 3; ++a) {
        si[a] = dot3(C.hinv[a], ci[0], ci[1], ci[2]);
        const double d = __dadd_rn(dot3(C.hinv[a], cj[0], cj[1], cj[2]), -si[a]);
        ds[a] = __dadd_rn(d, -round(d));
    }
    double best = 1.0 / 0.0;
    kb[0] = kb[1] = kb[2] = 0;
    for (int k0 = -1; k0 <= 1; ++k0)
        for (int k1 = -1; k1 <= 1; ++k1)
            for (int k2 = -1; k2 <= 1; ++k2) {
                const double t0 = __dadd_rn(ds[0], (double)k0), t1 = __dadd_rn(ds[1], (double)k1),
                             t2 = __dadd_rn(ds[2], (double)k2);
                const double d0 = dot3(C.h[0], t0, t1, t2), d1 = dot3(C.h[1], t0, t1, t2),
                             d2 = dot3(C.h[2], t0, t1, t2);
                const double dd = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
                if (dd < best) {
                    best = dd;
                    kb[0] = k0;
                    kb[1] = k1;
                    kb[2] = k2;
                }
            }
    if (!(best <= C.r_pair2)) return false;
    for (int a = 0; a < 3; ++a) {
        const double sm = __dadd_rn(si[a], __dmul_rn(__dadd_rn(ds[a], (double)kb[a]), 0.5));
        long long r = (long long)round(__dmul_rn((double)C.n[a], sm)) % C.n[a];
        if (r < 0) r += C.n[a];
        g[a] = (int)r;
    }
    return true;
}

// One CTA per row i; fill = 0 counts, fill = 1 writes rows in (i, j) order.
__global__ void __launch_bounds__(kThreads) k_rows_noalloc(PairCell C, int *scratch, int fill, int cap, int *rows)
{
    const int i = blockIdx.x;
    __shared__ int warp_tot[kThreads / 32];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = fill ? scratch[kMaxOrbNoalloc + i] : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j0 = i; j0 < C.n_orb; j0 += kThreads) {
        const int j = j0 + threadIdx.x;
        int kb[3], g[3];
        const bool ok = (j < C.n_orb) && pair_rule(C, i, j, kb, g);
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
            if (k < w) before += warp_tot[k];
            tot += warp_tot[k];
        }
        if (fill && ok) {
            const int pos = s_base + before + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap) {
                int *r = rows + 8 * (size_t)pos;
                r[0] = i;
                r[1] = j;
                r[2] = kb[0];
                r[3] = kb[1];
                r[4] = kb[2];
                r[5] = g[0];
                r[6] = g[1];
                r[7] = g[2];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (!fill && threadIdx.x == 0) scratch[i] = s_base;
}

// Exclusive scan of the row counts (one CTA); writes the total to the scratch
// and to the caller's count.
__global__ void __launch_bounds__(1024) k_scan_noalloc(int *scratch, int n_rows, int *n_out)
{
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_rows; base += 1024) {
        const int r = base + threadIdx.x;
        const int v = r < n_rows ? scratch[r] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (r < n_rows) scratch[kMaxOrbNoalloc + r] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[2 * kMaxOrbNoalloc] = carry;
        *n_out = carry;
    }
}

// Device address of the static scratch, resolved once per device.
int *g_scratch_addr[64] = {};

}  // namespace

extern "C" int exx_pair_list_noalloc(const exx_cell *cell, const double *centres, int n_orb, double r_pair, int cap,
                                     int *rows, int *n_pairs, void *stream)
{
    if (!cell || !n_pairs || n_orb < 0 || cap < 0 || !(r_pair >= 0.0)) return EXX_ERR_ARG;
    if (n_orb > kMaxOrbNoalloc) return EXX_ERR_CAPACITY;
    if (n_orb > 0 && (!centres || (cap > 0 && !rows))) return EXX_ERR_ARG;
    exx::Metric m;
    const int e = exx::make_metric(cell->lattice, cell->n, m);
    if (e) return e;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return EXX_ERR_CUDA;
    }
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pairlist_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EXX_ERR_CUDA;
        }
        g_scratch_addr[dev] = (int *)p;
    }
    int *scratch = g_scratch_addr[dev];
    PairCell C;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            C.h[a][b] = m.h[a][b];
            C.hinv[a][b] = m.hinv[a][b];
        }
    for (int a = 0; a < 3; ++a) C.n[a] = m.n[a];
    C.r_pair2 = r_pair * r_pair;
    C.centres = centres;
    C.n_orb = n_orb;
    cudaStream_t s = (cudaStream_t)stream;
    cudaGetLastError();
    // the counts of every row are rewritten below; nothing else needs zeroing
    if (n_orb > 0) k_rows_noalloc<<<n_orb, kThreads, 0, s>>>(C, scratch, 0, cap, rows);
    k_scan_noalloc<<<1, 1024, 0, s>>>(scratch, n_orb, n_pairs);
    if (n_orb > 0) k_rows_noalloc<<<n_orb, kThreads, 0, s>>>(C, scratch, 1, cap, rows);
    if (cudaGetLastError() != cudaSuccess) return EXX_ERR_CUDA;
    return EXX_OK;
}
