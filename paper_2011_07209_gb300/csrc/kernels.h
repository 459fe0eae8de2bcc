// kernels.h -- launch wrappers of the EXX kernels (library-internal).
#pragma once
#include <cuda_runtime.h>

#include "exx_dev.h"

namespace exx {

constexpr int kRowThreads = 128;     // pair-list CTA size
// two 512-thread CTAs per SM, each on its own pair: one CTA's barriers and
// per-pair passes overlap the other's streaming passes (64 registers a thread
// either way)
#ifndef EXX_SOLVE_THREADS
#define EXX_SOLVE_THREADS 512
#endif
#ifndef EXX_SOLVE_MIN_BLOCKS
#define EXX_SOLVE_MIN_BLOCKS 2
#endif
constexpr int kSolveThreads = EXX_SOLVE_THREADS;       // persistent pair-solver CTA size
constexpr int kSolveMinBlocks = EXX_SOLVE_MIN_BLOCKS;  // resident CTAs per SM it is compiled for

// Per-CTA scratch of the persistent solver: one slot per CTA, all slots equal.
struct SolveSlots {
    char *base;
    size_t slot_bytes;
    size_t off_vbox, off_pbox, off_rho, off_r64, off_r, off_q, off_e;
    size_t off_gs;   // 6 kGuessBins kNlm floats: binned moments of the starting guess
    size_t off_b2;   // n_pe float pairs: 4 pi rho as hi + lo (double-float residuals)
    size_t off_zf;   // dense FP32 box: the smoothed part z0 of the preconditioned residual (multigrid)
    size_t off_mg;   // coarse-level boxes of the multigrid preconditioner
    int n_slots;
};

cudaError_t launch_tables(const CellDev *cell, int which, int n_points, double *S64, float *S32, double *T64,
                          float *T32, cudaStream_t s);
// dst[j][:] = src[perm[j]][:] for rows of kNlm floats
cudaError_t launch_gather_rows(const float *src, const int32_t *perm, int n, float *dst, cudaStream_t s);
// info[j] = (pe_m, pe_off, bin, k) of PE point k = perm[j] (the radius-sorted order of the guess)
cudaError_t launch_guess_info(const int32_t *perm, const uint8_t *bin, const int32_t *pe_m, const int32_t *pe_off,
                              int n, int4 *info, cudaStream_t s);
cudaError_t launch_pair_list(const CellDev *cells, int n_cells, int n_rows, const ListDev &L, cudaStream_t s);
cudaError_t launch_solve(const CellDev *cells, const ListDev &L, const SolveSlots &slots, bool mixed,
                         int inner_shift, cudaStream_t s);
cudaError_t launch_clamp_total(const ListDev &L, int limit, cudaStream_t s);
cudaError_t launch_finalize(const CellDev *cells, int n_cells, const ListDev &L, CellResult *res, cudaStream_t s);
int solve_blocks_per_sm(bool mixed);

// Cluster path of the mixed solver: one pair per cluster of kClusterCTAs CTAs
// with the CG state in distributed shared memory.
constexpr int kClusterCTAs = 16;
#ifndef EXX_CLUSTER_THREADS
#define EXX_CLUSTER_THREADS 512
#endif
constexpr int kClusterThreads = EXX_CLUSTER_THREADS;   // threads per cluster CTA
inline size_t cluster_dyn_bytes(int rowtab_words, int p_floats, int max_groups)
{
    return ((4 * (size_t)rowtab_words + 15) & ~(size_t)15) + 4 * (size_t)((p_floats + 3) & ~3) +
           48 * (size_t)max_groups;
}
// Largest dynamic shared memory a cluster CTA can take on the current device.
int cluster_capacity_bytes();
// Launches as many clusters as can be resident (at most slots.n_slots); *n_clusters receives the count.
cudaError_t launch_solve_cluster(const CellDev *cells, const ListDev &L, const SolveSlots &slots, int rowtab_words,
                                 int p_floats, int max_groups, int inner_shift, int *n_clusters, cudaStream_t s);
// Records the CUDA error behind an EXX_ERR_CUDA for exx_last_error_detail()
// (thread-local) and returns EXX_ERR_CUDA.
int note_cuda_error(const char *where, cudaError_t e);
cudaError_t launch_warm_map(const PairRec *rows, int n, int n_orb, int *map, cudaStream_t s);

}  // namespace exx
