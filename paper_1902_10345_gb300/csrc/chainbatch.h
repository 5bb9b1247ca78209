// Host side of the skewed-chain kernel over many grids (chain_batch.cu), used
// by batch plans whose grids all run a fixed number of steps.  The scheme is
// the one of the single-grid chain kernel (skewed.cu): per grid, passes of k
// fused steps cut into chains of L rows per column strip, skewed down k rows
// per pass, chunk-level dependencies; work items (pass, grid, chain, strip)
// are dequeued pass-major, grids with more passes first within a pass.
#pragma once

#include <vector>

#include "launchset.h"
#include "runtime.h"

namespace sdfg {

// Boundary ring of one grid copied from `src` into up to two grids of the
// same layout (rows 0 and R-1, columns 0 and C-1).
struct RingCopy {
    const void *src;
    void *dst[2];  // nullptr: skipped
    int R, C, ld;
    int pad_;
};

// One copy of a whole grid (rows x cols, pitches in elements).
struct GridCopy {
    const void *src;
    void *dst;
    int rows, cols, ld_src, ld_dst;
};

// Shared memory of a chain-kernel CTA of `warps` warps: each warp's TMA ring
// of STAGES chunks of chain_chunk_rows rows.
inline size_t chain_smem_bytes(int dtype, int warps) {
    const int S = dtype_bytes(dtype);
    return static_cast<size_t>(warps) * STAGES * chain_chunk_rows(S) * 32 * lane_cols(S) * S;
}

// Copies n ring descriptors / grid descriptors that live in device memory.
int launch_ring_copy(const RingCopy *d_descs, int n, int max_ring, int dtype, cudaStream_t s);
int launch_grid_copy(const GridCopy *d_descs, int n, int max_rows, int dtype, cudaStream_t s);

struct ChainBatch {
    int dtype = SDFG_F32;
    int k = 8;
    int L = 512;
    int pub = 0;                // 0: the library default
    std::vector<int> last_dst;  // per grid: buffer written by its last pass (-1: no pass)
    int total_items = 0;
    int blocks = 1;             // CTAs
    void *slab = nullptr;
    size_t slab_bytes = 0, const_bytes = 0;
    void *params = nullptr;     // device-side launch parameters (inside the slab)
    const void *ring = nullptr; // ring descriptors (inside the slab)
    int n_ring = 0, max_ring = 0;
    unsigned long long timeout_ns = 0;

    // Plan the grids `runs` (steps > 0, tol == 0) and upload everything to one
    // slab on stream s; waits for the upload.
    int build(const std::vector<GridRun> &runs, cudaStream_t s);
    // Reset the counters, copy the boundary rings, launch.
    int enqueue(DeviceState *st, cudaStream_t s);
    void release(cudaStream_t s);
};

}  // namespace sdfg
