// Host-side builder of one persistent launch over many grids (used by batch
// plans, tolerance solves and the server's waves).
#pragma once

#include <vector>

#include "persistent.h"
#include "runtime.h"

namespace sdfg {

// One grid's share of a launch.
struct GridRun {
    void *buf[3] = {nullptr, nullptr, nullptr};  // 0: result side, 1: scratch, 2: input side
    int ld = 0;          // pitch of buf[] (elements)
    int R = 0, C = 0;
    int t0 = 0;          // steps completed before this launch
    int steps = 0;       // steps to run in this launch
    int T_cap = 0;       // total step cap of the solve
    int cur = 2;         // buffer holding the state at launch start
    double tol = 0.0;    // 0: fixed step count
    double r_ref2 = 0.0; // carried across launches
    int seg_rows = 0;    // 0: automatic
    const CUtensorMap *tmaps = nullptr;  // optional pre-encoded maps for buf[0..2]
};

struct LaunchSet {
    int dtype = SDFG_F32;
    int k = 8;
    int warps = 8;
    int check_stride = 64;

    std::vector<PGrid> grids;
    std::vector<PState> state0;
    std::vector<int> pass_info, chk_before, pass_tend, level_start, n_active, units_prefix, order;
    std::vector<int> last_dst;  // buffer written by each grid's last pass (-1: no pass)
    int total_items = 0, total_units = 0, P_max = 0, n_reduce = 0;
    int blocks = 1;  // persistent CTAs (computed by upload, outside any capture)

    // device storage (one slab)
    void *slab = nullptr;
    size_t slab_bytes = 0;
    PLaunch L{};

    // Fill the host arrays for `runs`.  Grids with steps == 0 take no items.
    int build(const std::vector<GridRun> &runs);
    // (Re)allocate the slab and copy the host arrays to it on stream s.
    int upload(cudaStream_t s);
    // Reset the per-launch counters (work head, done flags, reduce counters,
    // state) on stream s: everything a replay needs.
    int reset(cudaStream_t s);
    void release(cudaStream_t s);
};

// Pass schedule of one grid for steps (t0, t0+steps]: depth-k passes that end
// on every multiple of check_stride (tolerance mode) and on the last step.
void plan_grid_passes(int t0, int steps, int T_cap, bool tol_mode, int check_stride, int k, std::vector<int> &info,
                      std::vector<int> &tend);

int persistent_blocks_per_sm(int dtype, int warps);
int launch_persistent(const PLaunch &L, int dtype, int warps, int blocks, cudaStream_t s);
int launch_finalize(const void *fdescs, int n, const PGrid *grids, const PState *state, int dtype, int max_rows,
                    cudaStream_t s);
size_t final_desc_bytes();

// Layout of the finalise descriptor (mirrors persistent.cu).
struct FinalDescHost {
    const void *src;
    void *dst;
    int ld_src, ld_dst, rows, cols;
    int src_sel;
    int grid;
};

// Test hooks (sdfg_test_hook).
struct TestHooks {
    int inject_stuck_wait = 0;
    unsigned long long timeout_ns = 0;  // 0: default
    long long chain_min_points = -1;    // batches: fixed-step grids of >= this many points go on chains (-1: 2^20)
    int chain_rows = 0;                 // batches: chain length (0: 512)
};
TestHooks &test_hooks();

}  // namespace sdfg
