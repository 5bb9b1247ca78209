// Device code of one chain of the skewed-chain kernels (skewed.cu: one grid;
// chain_batch.cu: many grids): the bounded dependency wait on the previous
// pass's progress, the UnitPipe hook that waits and publishes, and the
// streamed pass over one chain of one column strip.  The scheme is described
// at the top of skewed.cu.
#pragma once

#include <limits.h>

#include "temporal_unit.cuh"

namespace sdfg {

#ifndef SDFG_CHAIN_TURN
#define SDFG_CHAIN_TURN 6  // rows per turn of a chain's chunk loop (4 on the persistent units)
#endif

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Spin (lane-parallel) until every lane's predicate holds; false on timeout.
template <class Pred>
__device__ __forceinline__ bool chain_warp_wait(Pred pred, unsigned long long timeout_ns) {
    if (__all_sync(FULL_MASK, pred())) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        __nanosleep(64);
        if (__all_sync(FULL_MASK, pred())) return true;
        const bool late = globaltimer_ns() - t0 > timeout_ns;
        if (__any_sync(FULL_MASK, late)) return false;
    }
}

// Collective (whole warp): wait until pass p-1 has stored rows [from,
// need_hi] in the strips s-1, s, s+1.  Returns the largest row up to which
// that is now known (>= need_hi), or INT_MIN if a bounded wait ran out (the
// error word is set).  Out of line: a chain reaches it only when the
// producer's last known progress is not enough.
static __device__ __noinline__ int chain_wait_rows(const int *prog_prev, int beta_prev, int jmin_prev, int L, int R,
                                            int n_strips, int s, int from, int need_hi, int *err,
                                            unsigned long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const int ja = floor_div(from - beta_prev, L);
    const int jb = floor_div(need_hi - beta_prev, L);
    const int s2 = s + lane - 1;
    const bool mine = lane < 3 && s2 >= 0 && s2 < n_strips;
    int seen = INT_MAX;
    for (int jj = ja; jj <= jb; ++jj) {
        const int lo = max(0, jj * L + beta_prev);
        const int need = (jj < jb) ? min(R, (jj + 1) * L + beta_prev) - lo : need_hi - lo + 1;
        const int *f = prog_prev + (jj - jmin_prev) * n_strips + s2;  // dereferenced by `mine` lanes only
        int v = INT_MAX;
        const bool good = chain_warp_wait(
            [&] {
                if (!mine) return true;
                v = ld_acquire_gpu(f);
                return v >= need;
            },
            timeout_ns);
        if (!good) {
            if (lane == 0) set_device_error(err, DEV_ERR_TIMEOUT_DEP);
            return INT_MIN;
        }
        if (jj == jb) seen = static_cast<int>(__reduce_min_sync(FULL_MASK, static_cast<unsigned>(mine ? v : INT_MAX)));
    }
    // the acquiring lanes' view reaches lane 0 through the barrier; lane 0
    // then orders it before its TMA (async proxy) reads
    __syncwarp();
    if (lane == 0) fence_proxy_async_global();
    return max(0, jb * L + beta_prev) + seen - 1;
}

// UnitPipe hook of one chain: waits on pass p-1's progress before each chunk
// load (chunks of CR rows), publishes this chain's progress after its chunks.
template <int CR>
struct ChainHook {
    static constexpr bool EDGES = true;
    static constexpr int TURN = SDFG_CHAIN_TURN;
    static constexpr int ROWS = CR;
    const int *prog_prev;  // counters of pass p-1 (nullptr for pass 0: the input is ready)
    int *prog_own;         // this chain's counter
    int beta_prev, jmin_prev, L, R, n_strips, s, lane;
    int rb, extra, ok_hi;  // ok_hi: rows <= ok_hi of pass p-1 are known stored in strips s-1..s+1
    int y0, y1, K, n_chunks, pub;
    int *err;
    unsigned long long timeout_ns;

    // Collective: pass p-1's rows up to the end of chunk c (plus `extra`) are
    // stored in the three strips around s.
    __device__ __forceinline__ bool ready(int c) {
        if (!prog_prev) return true;
        const int r0 = rb + c * CR;
        const int need_hi = min(R - 1, r0 + CR - 1 + extra);
        if (need_hi <= ok_hi) return true;
        ok_hi = chain_wait_rows(prog_prev, beta_prev, jmin_prev, L, R, n_strips, s, ok_hi + 1, need_hi, err,
                                timeout_ns);
        return ok_hi != INT_MIN;
    }

    // Chunk c's rows are stored and the warp is synchronised: publish every
    // `pub` chunks and at the end.
    __device__ __forceinline__ void done(int c) {
        if (c != n_chunks - 1 && (c + 1) % pub != 0) return;
        const int r0 = rb + c * CR;
        const int v = max(0, min(r0 + CR - K, y1) - y0);
        if (lane == 0) st_release_gpu(prog_own, v);
    }
};

// One chain: output rows [lo, hi) of strip s, read through `tmap`, written to dst.
template <class ST, int V, int K, class Hook>
__device__ __forceinline__ bool run_chain(const void *tmap, ST *dst, const GridGeo &g, int s, int lo, int hi,
                                          ST *ring, uint64_t *bars, uint32_t &chunk_ctr, Hook &hk,
                                          unsigned long long timeout_ns) {
    constexpr int CR = Hook::ROWS;
    constexpr int W = 32 * V;
    const int lane = threadIdx.x & 31;
    const int X = s * g.wout - g.h;
    const int rb = max(0, lo - K);
    const int n_steps = hi + K - rb;
    const int n_chunks = (n_steps + CR - 1) / CR;
    const int gc0 = X + lane * V;
    const int hl = g.h / V;
    unsigned colmask = 0;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int gc = gc0 + e;
        if (gc <= 0 || gc >= g.C - 1) colmask |= 1u << e;
    }
    const bool own_lane = lane >= hl && lane < 32 - hl && gc0 < g.C;
    const bool full_vec = gc0 + V <= g.C;
    const bool colchk = (X <= 0) || (X + W > g.C - 1);
    hk.rb = rb;
    // The first wait starts `extra` rows above the first input row: when
    // pass p-1 fused more steps than pass p, its chain that ends at row rb
    // still reads up to extra - 1 rows into this chain's output rows, so it
    // must be complete before they are written.
    hk.ok_hi = max(0, rb - hk.extra) - 1;
    hk.y0 = lo;
    hk.y1 = hi;
    hk.K = K;
    hk.n_chunks = n_chunks;
    bool ok;
#define SDFG_CHAIN_PIPE(CHK, EX, SY0, SY1)                                                              \
    {                                                                                                   \
        UnitPipe<ST, V, K, CHK, false, EX, CR> p;                                                       \
        p.tmap = tmap; p.dst = dst; p.ld = g.ld; p.R = g.R; p.C = g.C;                                  \
        p.X = X; p.y0 = lo; p.y1 = hi; p.rb = rb; p.n_steps = n_steps; p.n_chunks = n_chunks;           \
        p.sy0 = (SY0); p.sy1 = (SY1);                                                                   \
        p.base = chunk_ctr; p.ring = ring; p.bars = bars; p.lane = lane;                                \
        p.colmask = colmask; p.resmask = 0; p.own_lane = own_lane; p.full_vec = full_vec;               \
        p.res_flags = 0; p.timeout_ns = timeout_ns;                                                     \
        ok = p.run(hk);                                                                                 \
    }
    // The reassociated pipe needs its two-row ring to handle the boundary
    // (rows 0 and R-1, and on a boundary strip columns 0 and C-1); it never
    // stores them, the caller's ring copy provides them.  FP64 keeps the
    // exact order everywhere and stores the ring itself.
    constexpr bool SCALED_OK = UnitPipe<ST, V, K, false, false, false, CR>::RING2;
    if (!SCALED_OK) {
        if (colchk)
            SDFG_CHAIN_PIPE(true, true, lo, hi)
        else
            SDFG_CHAIN_PIPE(false, true, lo, hi)
    } else if (colchk) {
        SDFG_CHAIN_PIPE(true, false, max(lo, 1), min(hi, g.R - 1))
    } else {
        SDFG_CHAIN_PIPE(false, false, max(lo, 1), min(hi, g.R - 1))
    }
#undef SDFG_CHAIN_PIPE
    chunk_ctr += static_cast<uint32_t>(n_chunks);
    return ok;
}

template <class ST, int V, class Hook>
__device__ __forceinline__ bool chain_depth(int k, const void *tmap, ST *dst, const GridGeo &g, int s, int lo, int hi,
                                            ST *ring, uint64_t *bars, uint32_t &ctr, Hook &hk,
                                            unsigned long long timeout_ns) {
    switch (k) {
        case 1: return run_chain<ST, V, 1, Hook>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
        case 2: return run_chain<ST, V, 2, Hook>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
        case 4: return run_chain<ST, V, 4, Hook>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
        default: return run_chain<ST, V, 8, Hook>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
    }
}

}  // namespace sdfg
