// Persistent batch execution: data structures shared by the host planner
// (batch.cpp, server.cpp) and the persistent kernel (persistent.cu).
//
// One launch advances many grids by a few passes each.  Work items are
// (pass p, grid g, unit u), ordered by pass, and within a pass by grid (grids
// with more passes first).  Warps dequeue items with one atomic add each
// (paper Sec. 3: a Consume scope whose workers pop a shared work stream with
// atomics).  A unit of pass p may start once the (up to nine) units around it
// finished pass p-1 -- they hold every row and column it reads, and they no
// longer read what it overwrites -- so passes of one grid overlap as a
// wavefront and different grids overlap freely.  Deadlock is impossible: an
// item only waits on items dequeued before it, which belong to running warps.
//
// Grids solved to a tolerance reduce, on "reduce passes", the squared updates
// of every unit in a fixed order (deterministic), and the last unit to finish
// such a pass decides whether the grid stops (paper Sec. 3 "State": a state
// transition whose condition depends on data).  A unit of pass p waits for all
// decisions of passes <= p-2, so the pass right after a check may run
// speculatively: it writes the buffer the check pass read, never the result.
#pragma once

#include <cuda.h>
#include <stdint.h>
#include <vector_types.h>

#include "geometry.h"

namespace sdfg {

// pass_info bits
constexpr int PASS_K_MASK = 0xff;
constexpr int PASS_REF = 1 << 8;     // accumulate ||A_1 - A_0||^2 (first step of a solve)
constexpr int PASS_CHECK = 1 << 9;   // a check step: stop if rel <= tol
constexpr int PASS_FINAL = 1 << 10;  // last step allowed (T cap): always stop, report rel
constexpr int PASS_REDUCE = PASS_REF | PASS_CHECK | PASS_FINAL;

// Buffers of a grid: 0 = caller's out (or its aligned stand-in), 1 = scratch,
// 2 = caller's in (or its aligned stand-in).
struct PGrid {  // (aligned as its CUtensorMap members: 128 bytes)
    CUtensorMap tm[3];
    void *buf[3];
    GridGeo geo;
    int n_units;     // strips * segments
    int unit_off;    // first index of this grid's units in done[] / partials
    int P;           // passes in this launch
    int pass_off;    // first index of this grid's passes in pass_info[] / chk_before[]
    int t0;          // steps completed before this launch
    int cur;         // buffer holding the state at launch start
    int first_dst;   // buffer written by pass 0 (then alternating 0/1)
    int chk_off;     // first index of this grid's reduce counters
    int tol_mode;    // 1 when solving to a tolerance (reduce passes present)
    int pad_;
    double tol;
};

// Per-grid state written by the kernel (host initialises it before a launch).
struct PState {
    int stop_pass;   // pass after which the grid stopped in this launch (-1: running)
    int steps_done;  // steps completed when it stopped
    int final_buf;   // buffer holding the result when it stopped
    int check_done;  // reduce-pass decisions applied in this launch
    double r_ref2;   // ||A_1 - A_0||^2 (kept across launches)
    double rel;      // relative residual at the last reduce pass
};

struct PLaunch {
    const PGrid *grids;
    PState *state;
    const int *pass_info;     // per (grid, pass): k | flags
    const int *chk_before;    // per (grid, pass): reduce passes before it in this launch
    const int *pass_tend;     // per (grid, pass): total steps completed at the end of the pass
    const int *level_start;   // [P_max + 1] first item of each pass level
    const int *n_active;      // [P_max] grids (sorted by P, descending) that have pass p
    const int *units_prefix;  // [n + 1] prefix sums of units over the sorted grids
    const int *order;         // [n] sorted position -> grid index
    int *done;                // per unit: passes completed
    double2 *partials;        // [2][total_units] squared-update sums (ref, check)
    int *chk_count;           // per (grid, reduce pass): units finished
    int *head;                // work-queue head
    int *err;                 // device error word
    int total_items;
    int total_units;
    int P_max;
    int inject_stuck_wait;    // test hook: the first item waits on a flag nothing sets
    unsigned long long timeout_ns;
};

}  // namespace sdfg
