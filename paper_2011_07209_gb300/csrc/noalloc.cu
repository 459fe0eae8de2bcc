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
#include <mutex>

#include "../../include/exx.h"
#include "kernels.h"
#include "pair_rule.cuh"
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
        const bool ok = (j < C.n_orb) && exx::pair_rule(C, i, j, kb, g);
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

// Device address of the static scratch, resolved once per device and context.
// The address belongs to the module loaded into one CUDA context: if the caller
// resets the device (cudaDeviceReset) and the primary context is created anew,
// the module is loaded again at another address, so the cached address is
// keyed on the context's unique id (cuCtxGetId, reached through the runtime's
// driver entry-point query so that the library does not link libcuda).
struct ScratchAddr {
    unsigned long long ctx_id;
    int *ptr;
};
ScratchAddr g_scratch_addr[64] = {};
std::mutex g_scratch_mu;

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Unique id of the calling thread's current context (0 on failure).
unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f2;
        cudaGetLastError();
        tried = true;
    }
    if (!get_current || !get_id) return 0;
    void *c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
    return id;
}

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
    // an error left pending by the caller's earlier work is reported, not cleared
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) return exx::note_cuda_error("noalloc.cu: pending error at entry", pending);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return exx::note_cuda_error("noalloc.cu: cudaGetDevice", ce);
    }
    if (dev < 0 || dev >= 64) return EXX_ERR_ARG;
    int *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        ScratchAddr &sa = g_scratch_addr[dev];
        const unsigned long long ctx_id = current_ctx_id();   // 0: no context current yet
        if (!sa.ptr || ctx_id == 0 || sa.ctx_id != ctx_id) {
            void *p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_pairlist_scratch);   // loads the module if needed
            if (ce != cudaSuccess || !p) {
                cudaGetLastError();
                sa.ptr = nullptr;
                return exx::note_cuda_error("noalloc.cu: cudaGetSymbolAddress", ce);
            }
            sa.ptr = (int *)p;
            sa.ctx_id = current_ctx_id();
        }
        scratch = sa.ptr;
    }
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
    // the counts of every row are rewritten below; nothing else needs zeroing
    if (n_orb > 0) k_rows_noalloc<<<n_orb, kThreads, 0, s>>>(C, scratch, 0, cap, rows);
    k_scan_noalloc<<<1, 1024, 0, s>>>(scratch, n_orb, n_pairs);
    if (n_orb > 0) k_rows_noalloc<<<n_orb, kThreads, 0, s>>>(C, scratch, 1, cap, rows);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return exx::note_cuda_error("noalloc.cu: launch", ce);
    return EXX_OK;
}
