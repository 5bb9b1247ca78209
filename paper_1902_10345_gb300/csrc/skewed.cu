// The skewed-chain kernel (SDFG_KERNEL_SKEWED): one persistent launch runs
// every pass of one grid with no redundant rows between work units.
//
// Tiling in (row, time).  A pass of k fused steps is cut, per column strip,
// into CHAINS of L consecutive output rows; one warp streams a whole chain
// through the k-level register pipeline (temporal_unit.cuh), so the k-row
// ramp at a unit's ends -- the row halo that overlapped tiles recompute -- is
// paid once per L rows instead of once per segment.  Chain boundaries move
// down by k_p rows from pass p-1 to pass p (time skewing; the chains of pass p
// start at rows j*L + beta_p, beta_p = steps completed after pass p), so the
// rows a chain of pass p reads, [lo - k_p, hi + k_p), are the whole chain j of
// pass p-1 and the first 2 k_p rows of chain j+1: a chain depends only on the
// START of the previous pass's chains, and can follow them down the grid a
// few chunks behind, instead of waiting for a neighbour to finish (paper
// Sec. 6.1 names diamond and hybrid hexagonal tiling for the same purpose:
// temporal tiles without recomputed halos; App. B MapTiling and StateFusion).
// Along columns the strips still overlap by h >= k columns (the lane-local
// shuffle exchange), as in the other kernels.
//
// Dependencies are per chunk.  A warp publishes, every `pub` chunks and at
// the end, how many of its chain's rows are stored (a release store after a
// warp barrier; the release waits for the warp's stores in flight, about a
// microsecond under full HBM traffic, so publishing after every chunk costs
// ~13% and every 12 chunks ~2%, while a longer interval adds lag from pass to
// pass: 12 chunks and 512-row chains are the measured best on 8192^2); before loading input rows [r0, r0 + CHUNK_ROWS) it waits
// (bounded, acquire loads) until pass p-1 has stored those rows, plus
// e = max(0, k_{p-1} - k_p) more, in strips s-1, s, s+1 (the first wait
// starts e rows above the chain's first input row).  That also orders every
// write after the reads of the previous pass that it overwrites: a chain of
// pass p-1 that reads row r either lies within the rows waited for, and is
// then complete, or holds the last row waited for, and has then loaded
// every row up to it plus k_{p-1}, which includes r.  Work items (pass, chain, strip) are dequeued with one atomic add each,
// pass-major, and an item only waits on items dequeued before it, so there
// is no deadlock.
//
// Units away from the boundary columns use the reassociated pipe, also in the
// first and last chain of a strip: rows 0 and R-1 are handled by the pipe's
// edge body and never stored; the host copies them into both ping-pong grids
// before the launch.  Units on the boundary columns keep the exact order.
#include <limits.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "launchset.h"
#include "runtime.h"
#include "temporal_unit.cuh"

namespace sdfg {

struct ChainParams {
    CUtensorMap tm[3];        // 0: out (or its stand-in), 1: scratch, 2: in
    void *buf[3];
    GridGeo geo;              // strips (h, wout, n_strips); H and n_segs unused
    const int4 *blocks;       // per block of items: (pass, chain j, lo, hi); strips fastest within a block
    const int *pass_k;        // [P] fused depth of pass p
    const int *pass_beta;     // [P] steps completed after pass p: chain j of pass p starts at j*L + beta_p
    const int *pass_jmin;     // [P] index of the chain of pass p holding row 0
    const int *prog_off;      // [P] first progress counter of pass p
    int *prog;                // per (pass, chain, strip): rows stored from the chain's first row
    int *head;                // work-queue head
    int *err;                 // device error word
    int total_items;
    int L;                    // chain length (rows)
    int first_dst;            // buffer written by pass 0 (then alternating 0/1)
    int cur;                  // buffer read by pass 0
    int pub;                  // publish every `pub` chunks
    int pad_;
    unsigned long long timeout_ns;
};

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
__device__ __noinline__ int chain_wait_rows(const int *prog_prev, int beta_prev, int jmin_prev, int L, int R,
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
// load, publishes this chain's progress after its chunks.
struct ChainHook {
    static constexpr bool EDGES = true;
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
        const int r0 = rb + c * CHUNK_ROWS;
        const int need_hi = min(R - 1, r0 + CHUNK_ROWS - 1 + extra);
        if (need_hi <= ok_hi) return true;
        ok_hi = chain_wait_rows(prog_prev, beta_prev, jmin_prev, L, R, n_strips, s, ok_hi + 1, need_hi, err,
                                timeout_ns);
        return ok_hi != INT_MIN;
    }

    // Chunk c's rows are stored and the warp is synchronised: publish every
    // `pub` chunks and at the end.
    __device__ __forceinline__ void done(int c) {
        if (c != n_chunks - 1 && (c + 1) % pub != 0) return;
        const int r0 = rb + c * CHUNK_ROWS;
        const int v = max(0, min(r0 + CHUNK_ROWS - K, y1) - y0);
        if (lane == 0) st_release_gpu(prog_own, v);
    }
};

// One chain: output rows [lo, hi) of strip s, read through `tmap`, written to dst.
template <class ST, int V, int K>
__device__ __forceinline__ bool run_chain(const void *tmap, ST *dst, const GridGeo &g, int s, int lo, int hi,
                                          ST *ring, uint64_t *bars, uint32_t &chunk_ctr, ChainHook &hk,
                                          unsigned long long timeout_ns) {
    constexpr int W = 32 * V;
    const int lane = threadIdx.x & 31;
    const int X = s * g.wout - g.h;
    const int rb = max(0, lo - K);
    const int n_steps = hi + K - rb;
    const int n_chunks = (n_steps + CHUNK_ROWS - 1) / CHUNK_ROWS;
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
        UnitPipe<ST, V, K, CHK, false, EX> p;                                                           \
        p.tmap = tmap; p.dst = dst; p.ld = g.ld; p.R = g.R; p.C = g.C;                                  \
        p.X = X; p.y0 = lo; p.y1 = hi; p.rb = rb; p.n_steps = n_steps; p.n_chunks = n_chunks;           \
        p.sy0 = (SY0); p.sy1 = (SY1);                                                                   \
        p.base = chunk_ctr; p.ring = ring; p.bars = bars; p.lane = lane;                                \
        p.colmask = colmask; p.resmask = 0; p.own_lane = own_lane; p.full_vec = full_vec;               \
        p.res_flags = 0; p.timeout_ns = timeout_ns;                                                     \
        ok = p.run(hk);                                                                                 \
    }
    // the reassociated pipe needs its two-row ring to handle rows 0 and R-1
    constexpr bool SCALED_OK = UnitPipe<ST, V, K, false, false, false>::RING2;
    if (colchk || !SCALED_OK) {
        if (colchk)
            SDFG_CHAIN_PIPE(true, true, lo, hi)
        else
            SDFG_CHAIN_PIPE(false, true, lo, hi)
    } else {
        SDFG_CHAIN_PIPE(false, false, max(lo, 1), min(hi, g.R - 1))
    }
#undef SDFG_CHAIN_PIPE
    chunk_ctr += static_cast<uint32_t>(n_chunks);
    return ok;
}

template <class ST, int V>
__device__ __forceinline__ bool chain_depth(int k, const void *tmap, ST *dst, const GridGeo &g, int s, int lo, int hi,
                                            ST *ring, uint64_t *bars, uint32_t &ctr, ChainHook &hk,
                                            unsigned long long timeout_ns) {
    switch (k) {
        case 1: return run_chain<ST, V, 1>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
        case 2: return run_chain<ST, V, 2>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
        case 4: return run_chain<ST, V, 4>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
        default: return run_chain<ST, V, 8>(tmap, dst, g, s, lo, hi, ring, bars, ctr, hk, timeout_ns);
    }
}

#ifndef SDFG_CHAIN_PUB
#define SDFG_CHAIN_PUB 12  // chunks between two progress updates of a chain
#endif
#ifndef SDFG_CK_MINB
#define SDFG_CK_MINB 3  // 128-thread CTAs per SM the register allocation must allow
#endif

template <class ST, int V>
__global__ void __launch_bounds__(128, SDFG_CK_MINB) chain_kernel(const __grid_constant__ ChainParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[MAX_WARPS][STAGES];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[warp][s], 1);
        mbar_init_fence();
        if (warp == 0)
            for (int b = 0; b < 3; ++b)
                if (P.buf[b]) tmap_prefetch(&P.tm[b]);
    }
    __syncwarp();
    ST *ring = reinterpret_cast<ST *>(smem_raw) + static_cast<size_t>(warp) * STAGES * CHUNK_ROWS * 32 * V;
    uint32_t ctr = 0;
    const GridGeo geo = P.geo;
    const int ns = geo.n_strips;
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(P.head, 1);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item >= P.total_items) break;
        const int blk = item / ns;
        const int s = item - blk * ns;
        const int4 b = __ldg(P.blocks + blk);
        const int p = b.x, j = b.y, lo = b.z, hi = b.w;
        const int k = __ldg(P.pass_k + p);
        ChainHook hk;
        hk.prog_prev = p > 0 ? P.prog + __ldg(P.prog_off + p - 1) : nullptr;
        hk.beta_prev = p > 0 ? __ldg(P.pass_beta + p - 1) : 0;
        hk.jmin_prev = p > 0 ? __ldg(P.pass_jmin + p - 1) : 0;
        hk.extra = p > 0 ? max(0, __ldg(P.pass_k + p - 1) - k) : 0;
        hk.prog_own = P.prog + __ldg(P.prog_off + p) + (j - __ldg(P.pass_jmin + p)) * ns + s;
        hk.L = P.L;
        hk.R = geo.R;
        hk.n_strips = ns;
        hk.s = s;
        hk.lane = lane;
        hk.pub = P.pub;
        hk.err = P.err;
        hk.timeout_ns = P.timeout_ns;
        const int srcb = p == 0 ? P.cur : (P.first_dst ^ ((p - 1) & 1));
        const int dstb = P.first_dst ^ (p & 1);
        const bool ok = chain_depth<ST, V>(k, &P.tm[srcb], static_cast<ST *>(P.buf[dstb]), geo, s, lo, hi, ring,
                                           bars[warp], ctr, hk, P.timeout_ns);
        if (!ok) {
            if (lane == 0) set_device_error(P.err, DEV_ERR_TIMEOUT_TMA);
            break;
        }
    }
}

// ------------------------------------------------------------------ host ----
template <class ST>
static const void *ck_fn() {
    return reinterpret_cast<const void *>(
        &chain_kernel<ST, Store<ST>::bytes == 8 ? 2 : (Store<ST>::bytes == 4 ? SDFG_F32_V : 4)>);
}

static const void *chain_fn(int dtype) {
    switch (dtype) {
        case SDFG_F32: return ck_fn<float>();
        case SDFG_BF16: return ck_fn<__nv_bfloat16>();
        default: return ck_fn<double>();
    }
}

static int chain_blocks_per_sm(int dtype, int warps, size_t smem) {
    const void *fn = chain_fn(dtype);
    SDFG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int n = 0;
    SDFG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, warps * 32, smem));
    return n;
}

namespace {
// A planned launch for one grid: the constant arrays live in one device slab
// followed by the counters, which every call resets.
struct ChainPlan {
    // key
    const void *in = nullptr;
    void *out = nullptr;
    int R = 0, C = 0, ld = 0, dtype = 0, k = 0, L = 0, pub = 0, device = -1;
    long long T = 0;
    // state
    void *scratch = nullptr;
    void *slab = nullptr;
    size_t const_bytes = 0, slab_bytes = 0;
    int last = 0;      // buffer written by the last pass
    int blocks = 0;    // CTAs
    ChainParams prm{};
    unsigned long long stamp = 0;
};
constexpr size_t kChainCacheSize = 8;
std::mutex g_chain_mu;
std::vector<ChainPlan *> g_chain;
unsigned long long g_chain_clock = 0;

void chain_plan_free(ChainPlan *c, cudaStream_t s) {
    scratch_free(c->slab, s);
    scratch_free(c->scratch, s);
    delete c;
}

int chain_plan_build(ChainPlan *c, DeviceState *st, cudaStream_t s) {
    const int S = dtype_bytes(c->dtype);
    const int W = 32 * lane_cols(S);
    const std::vector<int> ks = plan_passes(c->T, c->k);
    const int P = static_cast<int>(ks.size());
    const int R = c->R, L = c->L;
    GridGeo g = plan_geometry(R, c->C, c->ld, c->dtype, c->k, L, 0);
    std::vector<int> beta(P), jmin(P), off(P);
    std::vector<int4> blocks;
    int acc = 0, n_prog = 0;
    auto fdiv = [](long long a, long long b) { return static_cast<int>(a >= 0 ? a / b : -((-a + b - 1) / b)); };
    for (int p = 0; p < P; ++p) {
        acc += ks[p];
        beta[p] = acc % L;  // only beta mod L matters for the boundaries; keeps the arithmetic small
        jmin[p] = fdiv(-static_cast<long long>(beta[p]), L);
        const int jmax = fdiv(static_cast<long long>(R) - 1 - beta[p], L);
        off[p] = n_prog;
        n_prog += (jmax - jmin[p] + 1) * g.n_strips;
        for (int j = jmin[p]; j <= jmax; ++j) {
            const int lo = std::max(0, j * L + beta[p]);
            const int hi = std::min(R, (j + 1) * L + beta[p]);
            blocks.push_back(make_int4(p, j, lo, hi));
        }
    }
    const long long total = static_cast<long long>(blocks.size()) * g.n_strips;
    if (total > INT_MAX / 2) return set_error(SDFG_ERR_INVAL, "chain kernel: too many work items");
    // slab: blocks | pass_k | beta | jmin | off || prog | head
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_blocks = 0;
    const size_t o_k = al(o_blocks + blocks.size() * sizeof(int4));
    const size_t o_beta = al(o_k + P * sizeof(int));
    const size_t o_jmin = al(o_beta + P * sizeof(int));
    const size_t o_off = al(o_jmin + P * sizeof(int));
    const size_t o_prog = al(o_off + P * sizeof(int));
    const size_t o_head = al(o_prog + static_cast<size_t>(n_prog) * sizeof(int));
    const size_t total_bytes = al(o_head + sizeof(int));
    int rc = scratch_alloc(&c->slab, total_bytes, s);
    if (rc != SDFG_OK) return rc;
    std::vector<unsigned char> img(o_prog, 0);
    memcpy(img.data() + o_blocks, blocks.data(), blocks.size() * sizeof(int4));
    memcpy(img.data() + o_k, ks.data(), P * sizeof(int));
    memcpy(img.data() + o_beta, beta.data(), P * sizeof(int));
    memcpy(img.data() + o_jmin, jmin.data(), P * sizeof(int));
    memcpy(img.data() + o_off, off.data(), P * sizeof(int));
    SDFG_CUDA(cudaMemcpyAsync(c->slab, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    SDFG_CUDA(cudaStreamSynchronize(s));  // the host image must outlive the copy
    c->const_bytes = o_prog;
    c->slab_bytes = total_bytes;
    unsigned char *base = static_cast<unsigned char *>(c->slab);
    ChainParams &q = c->prm;
    memset(&q, 0, sizeof(q));
    // buffers: 0 = out, 1 = scratch, 2 = in (absent when in == out)
    q.buf[0] = c->out;
    q.buf[1] = c->scratch;
    q.buf[2] = c->in == c->out ? nullptr : const_cast<void *>(c->in);
    for (int b = 0; b < 3; ++b)
        if (q.buf[b]) {
            rc = encode_tmap(&q.tm[b], q.buf[b], c->dtype, R, c->C, c->ld, W);
            if (rc != SDFG_OK) return rc;
        }
    q.geo = g;
    q.blocks = reinterpret_cast<const int4 *>(base + o_blocks);
    q.pass_k = reinterpret_cast<const int *>(base + o_k);
    q.pass_beta = reinterpret_cast<const int *>(base + o_beta);
    q.pass_jmin = reinterpret_cast<const int *>(base + o_jmin);
    q.prog_off = reinterpret_cast<const int *>(base + o_off);
    q.prog = reinterpret_cast<int *>(base + o_prog);
    q.head = reinterpret_cast<int *>(base + o_head);
    q.err = st->d_err;
    q.total_items = static_cast<int>(total);
    q.L = L;
    q.pub = std::max(1, c->pub);
    q.timeout_ns = DEFAULT_TIMEOUT_NS;
    if (c->in == c->out) {
        q.cur = 0;
        q.first_dst = 1;
    } else {
        q.cur = 2;
        q.first_dst = (P % 2 == 1) ? 0 : 1;
    }
    c->last = q.first_dst ^ ((P - 1) & 1);
    const size_t smem = temporal_smem_bytes(c->dtype, 4);
    int bps = 0;
    rc = chain_blocks_per_sm(c->dtype, 4, smem);
    if (rc < 0) return rc;
    bps = std::max(1, rc);
    const long long need = (total + 3) / 4;
    c->blocks = static_cast<int>(std::max<long long>(1, std::min<long long>(need, static_cast<long long>(bps) * st->sm_count)));
    return SDFG_OK;
}
}  // namespace

// The chain kernel's pass plan for T steps at depth k: plan_passes(T, k).
// L: chain length in rows (0 = 512); pub: chunks between progress updates
// (0 = SDFG_CHAIN_PUB).  FP32, BF16 and FP64 storage; in/out must be
// TMA-compatible.
int run_single_chain(const void *in, void *out, int R, int C, int ld, long long T, int dtype, int k, int L, int pub,
                     DeviceState *st, cudaStream_t s) {
    if (L <= 0) L = 512;
    if (pub <= 0) pub = SDFG_CHAIN_PUB;
    L = std::max(L, 4 * k);
    std::lock_guard<std::mutex> lk(g_chain_mu);
    ChainPlan *c = nullptr;
    for (ChainPlan *x : g_chain)
        if (x->in == in && x->out == out && x->R == R && x->C == C && x->ld == ld && x->dtype == dtype && x->k == k &&
            x->L == L && x->pub == pub && x->device == st->device && x->T == T)
            c = x;
    if (!c) {
        if (g_chain.size() >= kChainCacheSize) {
            cudaDeviceSynchronize();  // the evicted plan's last launch may run on another stream
            auto it = std::min_element(g_chain.begin(), g_chain.end(),
                                       [](ChainPlan *a, ChainPlan *b) { return a->stamp < b->stamp; });
            chain_plan_free(*it, s);
            g_chain.erase(it);
        }
        c = new ChainPlan();
        c->in = in;
        c->out = out;
        c->R = R;
        c->C = C;
        c->ld = ld;
        c->dtype = dtype;
        c->k = k;
        c->L = L;
        c->pub = pub;
        c->device = st->device;
        c->T = T;
        int rc = scratch_alloc(&c->scratch, static_cast<size_t>(R) * ld * dtype_bytes(dtype), s);
        if (rc == SDFG_OK) rc = chain_plan_build(c, st, s);
        if (rc != SDFG_OK) {
            chain_plan_free(c, s);
            return rc;
        }
        g_chain.push_back(c);
    }
    c->stamp = ++g_chain_clock;
    const size_t S = dtype_bytes(dtype);
    // the reassociated units never store rows 0 and R-1: both ping-pong grids
    // hold them before the launch (one 2-row copy per grid that is not `in`)
    for (int b = 0; b < 2; ++b) {
        void *d = c->prm.buf[b];
        if (d == in) continue;
        SDFG_CUDA(cudaMemcpy2DAsync(d, static_cast<size_t>(R - 1) * ld * S, in, static_cast<size_t>(R - 1) * ld * S,
                                    C * S, 2, cudaMemcpyDeviceToDevice, s));
    }
    unsigned char *base = static_cast<unsigned char *>(c->slab);
    SDFG_CUDA(cudaMemsetAsync(base + c->const_bytes, 0, c->slab_bytes - c->const_bytes, s));
    ChainParams prm = c->prm;
    prm.timeout_ns = test_hooks().timeout_ns ? test_hooks().timeout_ns : DEFAULT_TIMEOUT_NS;
    void *args[] = {&prm};
    const size_t smem = temporal_smem_bytes(dtype, 4);
    TimedLaunch t = stats_begin(FAM_SKEWED, s);
    cudaError_t e = cudaLaunchKernel(chain_fn(dtype), dim3(c->blocks), dim3(128), args, smem, s);
    stats_end(t, s);
    if (e != cudaSuccess) return cuda_error(e, "chain kernel launch");
    if (c->last != 0) return launch_copy2d(out, ld, c->scratch, ld, R, C, dtype, s);
    return SDFG_OK;
}

}  // namespace sdfg
