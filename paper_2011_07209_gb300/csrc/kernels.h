// kernels.h -- launch wrappers of the EXX kernels (library-internal).
#pragma once
#include <cuda_runtime.h>

#include "exx_dev.h"

namespace exx {

constexpr int kRowThreads = 128;     // pair-list CTA size
#ifndef EXX_SOLVE_THREADS
#define EXX_SOLVE_THREADS 1024
#endif
#ifndef EXX_SOLVE_MIN_BLOCKS
#define EXX_SOLVE_MIN_BLOCKS 1
#endif
constexpr int kSolveThreads = EXX_SOLVE_THREADS;       // persistent pair-solver CTA size
constexpr int kSolveMinBlocks = EXX_SOLVE_MIN_BLOCKS;  // resident CTAs per SM it is compiled for

// Per-CTA scratch of the persistent solver: one slot per CTA, all slots equal.
struct SolveSlots {
    char *base;
    size_t slot_bytes;
    size_t off_vbox, off_pbox, off_rho, off_r64, off_r, off_q, off_e;
    int n_slots;
};

cudaError_t launch_tables(const CellDev *cell, int which, int n_points, double *S64, float *S32, double *T64,
                          float *T32, cudaStream_t s);
cudaError_t launch_pair_list(const CellDev *cells, int n_cells, int n_rows, const ListDev &L, cudaStream_t s);
cudaError_t launch_solve(const CellDev *cells, const ListDev &L, const SolveSlots &slots, bool mixed,
                         int inner_shift, cudaStream_t s);
cudaError_t launch_finalize(const CellDev *cells, int n_cells, const ListDev &L, CellResult *res, cudaStream_t s);
int solve_blocks_per_sm(bool mixed);
cudaError_t launch_warm_map(const PairRec *rows, int n, int n_orb, int *map, cudaStream_t s);

}  // namespace exx
