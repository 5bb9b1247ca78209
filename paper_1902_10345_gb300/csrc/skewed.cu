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
// the end, how many of its chain's rows are stored: a release store after a
// warp barrier.  The release waits for the warp's stores in flight, about a
// microsecond under full HBM traffic, so publishing after every chunk costs
// ~13% and every ~144 rows ~2%, while a longer interval adds lag from pass
// to pass (~144 rows and 640-row chains are the measured best on 8192^2).
// Before loading input rows [r0, r0 + CR) a warp waits (bounded,
// acquire loads) until pass p-1 has stored those rows, plus
// e = max(0, k_{p-1} - k_p) more, in strips s-1, s, s+1 (the first wait
// starts e rows above the chain's first input row).  That also orders every
// write after the reads of the previous pass that it overwrites: a chain of
// pass p-1 that reads row r either lies within the rows waited for, and is
// then complete, or holds the last row waited for, and has then loaded every
// row up to it plus k_{p-1}, which includes r.  Work items (pass, chain,
// strip) are dequeued with one atomic add each, pass-major, and an item only
// waits on items dequeued before it, so there is no deadlock.
//
// FP32 and BF16 storage use the reassociated pipe everywhere, also in the
// first and last chain of a strip and on the boundary strips: the boundary
// ring (rows 0 and R-1, columns 0 and C-1) is held scaled like every other
// value and never stored; a small kernel copies the ring into both ping-pong
// grids before the launch.  FP64 keeps the exact order and stores the ring.
#include <limits.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "chain.cuh"
#include "chainbatch.h"
#include "launchset.h"
#include "runtime.h"

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
    constexpr int CR = chain_chunk_rows(sizeof(ST));
    ST *ring = reinterpret_cast<ST *>(smem_raw) + static_cast<size_t>(warp) * STAGES * CR * 32 * V;
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
        ChainHook<CR> hk;
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
    const void *ring = nullptr;  // the ring-copy descriptor (inside the slab)
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
    const size_t o_ring = al(o_off + P * sizeof(int));
    const size_t o_prog = al(o_ring + sizeof(RingCopy));
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
    {
        // the input's boundary ring into both ping-pong grids (the
        // reassociated units never store it)
        RingCopy rcp{};
        rcp.src = c->in;
        int nd = 0;
        if (c->out != c->in) rcp.dst[nd++] = c->out;
        rcp.dst[nd++] = c->scratch;
        rcp.R = R;
        rcp.C = c->C;
        rcp.ld = c->ld;
        memcpy(img.data() + o_ring, &rcp, sizeof(rcp));
    }
    SDFG_CUDA(cudaMemcpyAsync(c->slab, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    SDFG_CUDA(cudaStreamSynchronize(s));  // the host image must outlive the copy
    c->const_bytes = o_prog;
    c->ring = static_cast<unsigned char *>(c->slab) + o_ring;
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
            rc = encode_tmap(&q.tm[b], q.buf[b], c->dtype, R, c->C, c->ld, W, chain_chunk_rows(S));
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
    const size_t smem = chain_smem_bytes(c->dtype, 4);
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
// L: chain length in rows (0: 640, 512 for BF16 storage, the measured best);
// pub: chunks between progress updates
// (0 = about every 144 rows).  FP32, BF16 and FP64 storage; in/out must be
// TMA-compatible.
int run_single_chain(const void *in, void *out, int R, int C, int ld, long long T, int dtype, int k, int L, int pub,
                     DeviceState *st, cudaStream_t s) {
    if (L <= 0) L = dtype == SDFG_BF16 ? 512 : 640;
    if (pub <= 0) pub = chain_pub_chunks(dtype_bytes(dtype));
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
    // the reassociated units never store the boundary ring: both ping-pong
    // grids receive it from the input before the launch
    int rc = launch_ring_copy(static_cast<const RingCopy *>(c->ring), 1, 2 * C + 2 * (R - 2), dtype, s);
    if (rc != SDFG_OK) return rc;
    unsigned char *base = static_cast<unsigned char *>(c->slab);
    SDFG_CUDA(cudaMemsetAsync(base + c->const_bytes, 0, c->slab_bytes - c->const_bytes, s));
    ChainParams prm = c->prm;
    prm.timeout_ns = test_hooks().timeout_ns ? test_hooks().timeout_ns : DEFAULT_TIMEOUT_NS;
    void *args[] = {&prm};
    const size_t smem = chain_smem_bytes(dtype, 4);
    TimedLaunch t = stats_begin(FAM_SKEWED, s);
    cudaError_t e = cudaLaunchKernel(chain_fn(dtype), dim3(c->blocks), dim3(128), args, smem, s);
    stats_end(t, s);
    if (e != cudaSuccess) return cuda_error(e, "chain kernel launch");
    if (c->last != 0) return launch_copy2d(out, ld, c->scratch, ld, R, C, dtype, s);
    return SDFG_OK;
}

}  // namespace sdfg
