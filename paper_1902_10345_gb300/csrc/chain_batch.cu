// The skewed-chain kernel over many grids (batches of uneven grids with a
// fixed number of steps each), and the small copy kernels of the chain
// kernels: the boundary ring into both ping-pong grids before a launch, and
// results that ended in scratch into the caller's grid after it.
//
// Every grid runs the scheme of the single-grid chain kernel (skewed.cu):
// passes of k fused steps cut into chains of L rows per column strip, chain
// boundaries skewed down k_p rows per pass, chunk-level dependencies on the
// previous pass of the same grid.  Work items (pass p, grid, chain, strip)
// are dequeued with one atomic add each, pass-major and, within a pass,
// grids with more passes first (their dependency chains are the longest);
// an item only waits on items of the same grid's previous pass, dequeued
// before it, so there is no deadlock.  Grids of different sizes and step
// counts fill each other's gaps (paper Sec. 3: a Consume scope over a shared
// work stream).
#include <limits.h>
#include <string.h>

#include <algorithm>
#include <numeric>

#include "chain.cuh"
#include "chainbatch.h"

namespace sdfg {

// ---------------------------------------------------------------- copies ----
template <class ST>
__global__ void ring_copy_kernel(const RingCopy *__restrict__ descs) {
    const RingCopy r = descs[blockIdx.y];
    const int n = 2 * r.C + 2 * max(r.R - 2, 0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int row, col;
        if (i < r.C) {
            row = 0;
            col = i;
        } else if (i < 2 * r.C) {
            row = r.R - 1;
            col = i - r.C;
        } else {
            const int t = i - 2 * r.C;
            row = 1 + (t >> 1);
            col = (t & 1) ? r.C - 1 : 0;
        }
        const size_t at = static_cast<size_t>(row) * r.ld + col;
        const ST v = static_cast<const ST *>(r.src)[at];
        if (r.dst[0]) static_cast<ST *>(r.dst[0])[at] = v;
        if (r.dst[1]) static_cast<ST *>(r.dst[1])[at] = v;
    }
}

template <class ST>
__global__ void grid_copy_kernel(const GridCopy *__restrict__ descs) {
    const GridCopy d = descs[blockIdx.y];
    const ST *src = static_cast<const ST *>(d.src);
    ST *dst = static_cast<ST *>(d.dst);
    for (int i = blockIdx.x; i < d.rows; i += gridDim.x)
        for (int j = threadIdx.x; j < d.cols; j += blockDim.x)
            dst[static_cast<size_t>(i) * d.ld_dst + j] = src[static_cast<size_t>(i) * d.ld_src + j];
}

int launch_ring_copy(const RingCopy *d_descs, int n, int max_ring, int dtype, cudaStream_t s) {
    if (n <= 0) return SDFG_OK;
    const dim3 grid(static_cast<unsigned>(std::min(std::max((max_ring + 255) / 256, 1), 64)), static_cast<unsigned>(n));
    TimedLaunch t = stats_begin(FAM_COPY, s);
    switch (dtype) {
        case SDFG_F32: ring_copy_kernel<float><<<grid, 256, 0, s>>>(d_descs); break;
        case SDFG_BF16: ring_copy_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(d_descs); break;
        default: ring_copy_kernel<double><<<grid, 256, 0, s>>>(d_descs); break;
    }
    stats_end(t, s);
    SDFG_CUDA(cudaGetLastError());
    return SDFG_OK;
}

int launch_grid_copy(const GridCopy *d_descs, int n, int max_rows, int dtype, cudaStream_t s) {
    if (n <= 0) return SDFG_OK;
    const dim3 grid(static_cast<unsigned>(std::min(std::max(max_rows, 1), 1024)), static_cast<unsigned>(n));
    TimedLaunch t = stats_begin(FAM_COPY, s);
    switch (dtype) {
        case SDFG_F32: grid_copy_kernel<float><<<grid, 256, 0, s>>>(d_descs); break;
        case SDFG_BF16: grid_copy_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(d_descs); break;
        default: grid_copy_kernel<double><<<grid, 256, 0, s>>>(d_descs); break;
    }
    stats_end(t, s);
    SDFG_CUDA(cudaGetLastError());
    return SDFG_OK;
}

// ---------------------------------------------------------------- kernel ----
// One grid of a chain batch (in device memory; tensor maps are acquired
// before use, as the host wrote them before the launch).
struct CGrid {
    CUtensorMap tm[3];  // 0: result side, 1: scratch, 2: input side
    void *buf[3];
    GridGeo geo;
    int pass_off;       // first index of this grid's passes in the pass arrays
    int first_dst;      // buffer written by pass 0 (then alternating 0/1)
    int cur;            // buffer read by pass 0
    int L;              // chain length
    int pub;            // chunks between progress updates
    int pad_[3];
};

struct CBatchParams {
    const CGrid *grids;
    const int4 *blk;        // per block of items: (grid, pass, chain j, first row)
    const int2 *blk2;       // per block: (end row, first item); the strips of the chain follow
    const int *pass_k;      // per (grid, pass), at grid.pass_off + p: fused depth
    const int *pass_beta;   // skew: chain j of the pass starts at j*L + beta
    const int *pass_jmin;   // index of the chain holding row 0
    const int *prog_off;    // first progress counter of the pass
    int *prog;              // per (grid, pass, chain, strip): rows stored
    int *head;              // work-queue head
    int *err;               // device error word
    int n_blocks;
    int total_items;
    unsigned long long timeout_ns;
};

#ifndef SDFG_CK_MINB
#define SDFG_CK_MINB 3  // 128-thread CTAs per SM the register allocation must allow
#endif

template <class ST, int V>
__global__ void __launch_bounds__(128, SDFG_CK_MINB) chain_batch_kernel(const CBatchParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[MAX_WARPS][STAGES];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[warp][s], 1);
        mbar_init_fence();
    }
    __syncwarp();
    constexpr int CR = chain_chunk_rows(sizeof(ST));
    ST *ring = reinterpret_cast<ST *>(smem_raw) + static_cast<size_t>(warp) * STAGES * CR * 32 * V;
    uint32_t ctr = 0;
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(P.head, 1);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item >= P.total_items) break;
        // the block holding the item: the last one whose first item is <= item
        int lo = 0, hi = P.n_blocks - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&P.blk2[mid].y) <= item)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int4 b = __ldg(P.blk + lo);
        const int2 b2 = __ldg(P.blk2 + lo);
        const int gi = b.x, p = b.y, j = b.z, clo = b.w, chi = b2.x;
        const int s = item - b2.y;
        const CGrid &G = P.grids[gi];
        const GridGeo geo = G.geo;
        const int ns = geo.n_strips;
        const int po = G.pass_off;
        const int k = __ldg(P.pass_k + po + p);
        ChainHook<CR> hk;
        hk.prog_prev = p > 0 ? P.prog + __ldg(P.prog_off + po + p - 1) : nullptr;
        hk.beta_prev = p > 0 ? __ldg(P.pass_beta + po + p - 1) : 0;
        hk.jmin_prev = p > 0 ? __ldg(P.pass_jmin + po + p - 1) : 0;
        hk.extra = p > 0 ? max(0, __ldg(P.pass_k + po + p - 1) - k) : 0;
        hk.prog_own = P.prog + __ldg(P.prog_off + po + p) + (j - __ldg(P.pass_jmin + po + p)) * ns + s;
        hk.L = G.L;
        hk.R = geo.R;
        hk.n_strips = ns;
        hk.s = s;
        hk.lane = lane;
        hk.pub = G.pub;
        hk.err = P.err;
        hk.timeout_ns = P.timeout_ns;
        const int srcb = p == 0 ? G.cur : (G.first_dst ^ ((p - 1) & 1));
        const int dstb = G.first_dst ^ (p & 1);
        const void *tm = &G.tm[srcb];
        if (lane == 0) tmap_acquire(tm);
        __syncwarp();
        const bool ok = chain_depth<ST, V>(k, tm, static_cast<ST *>(G.buf[dstb]), geo, s, clo, chi, ring, bars[warp],
                                           ctr, hk, P.timeout_ns);
        if (!ok) {
            if (lane == 0) set_device_error(P.err, DEV_ERR_TIMEOUT_TMA);
            break;
        }
    }
}

template <class ST>
static const void *cbk_fn() {
    return reinterpret_cast<const void *>(
        &chain_batch_kernel<ST, Store<ST>::bytes == 8 ? 2 : (Store<ST>::bytes == 4 ? SDFG_F32_V : 4)>);
}

static const void *chain_batch_fn(int dtype) {
    switch (dtype) {
        case SDFG_F32: return cbk_fn<float>();
        case SDFG_BF16: return cbk_fn<__nv_bfloat16>();
        default: return cbk_fn<double>();
    }
}

// ------------------------------------------------------------------ host ----
int ChainBatch::build(const std::vector<GridRun> &runs, cudaStream_t s) {
    const int n = static_cast<int>(runs.size());
    const int S = dtype_bytes(dtype);
    const int W = 32 * lane_cols(S);
    const int Lc = L > 0 ? std::max(L, 4 * k) : 512;
    const int pb = pub > 0 ? pub : chain_pub_chunks(dtype_bytes(dtype));
    auto fdiv = [](long long a, long long b) { return static_cast<int>(a >= 0 ? a / b : -((-a + b - 1) / b)); };
    std::vector<CGrid> grids(n);
    std::vector<int> pk, pbeta, pjmin, pjmax, poff, P(n);
    std::vector<RingCopy> rings;
    last_dst.assign(n, -1);
    long long n_prog = 0;
    max_ring = 0;
    for (int g = 0; g < n; ++g) {
        const GridRun &r = runs[g];
        CGrid &G = grids[g];
        memset(&G, 0, sizeof(G));
        const std::vector<int> ks = plan_passes(r.steps, k);
        P[g] = static_cast<int>(ks.size());
        G.geo = plan_geometry(r.R, r.C, r.ld, dtype, k, Lc, 0);
        G.pass_off = static_cast<int>(pk.size());
        G.L = Lc;
        G.pub = pb;
        G.cur = r.cur;
        G.first_dst = r.cur == 2 ? ((P[g] % 2 == 1) ? 0 : 1) : 1 - r.cur;
        last_dst[g] = P[g] > 0 ? (G.first_dst ^ ((P[g] - 1) & 1)) : r.cur;
        for (int b = 0; b < 3; ++b) {
            G.buf[b] = r.buf[b];
            if (!r.buf[b]) continue;
            if (r.tmaps) {
                G.tm[b] = r.tmaps[b];
            } else {
                int rc = encode_tmap(&G.tm[b], r.buf[b], dtype, r.R, r.C, r.ld, W, chain_chunk_rows(dtype_bytes(dtype)));
                if (rc != SDFG_OK) return rc;
            }
        }
        int acc = 0;
        for (int p = 0; p < P[g]; ++p) {
            acc += ks[p];
            const int beta = acc % Lc;
            const int jmin = fdiv(-static_cast<long long>(beta), Lc);
            const int jmax = fdiv(static_cast<long long>(r.R) - 1 - beta, Lc);
            pk.push_back(ks[p]);
            pbeta.push_back(beta);
            pjmin.push_back(jmin);
            pjmax.push_back(jmax);
            poff.push_back(static_cast<int>(n_prog));
            n_prog += static_cast<long long>(jmax - jmin + 1) * G.geo.n_strips;
        }
        if (n_prog > INT_MAX / 2) return set_error(SDFG_ERR_INVAL, "chain batch: too many progress counters");
        // the ring of the input into both ping-pong grids (the one that is the
        // input already holds it)
        RingCopy rc{};
        rc.src = r.buf[r.cur];
        int nd = 0;
        for (int b = 0; b < 2; ++b)
            if (r.buf[b] && r.buf[b] != r.buf[r.cur]) rc.dst[nd++] = r.buf[b];
        rc.R = r.R;
        rc.C = r.C;
        rc.ld = r.ld;
        if (P[g] > 0 && nd > 0) {
            rings.push_back(rc);
            max_ring = std::max(max_ring, 2 * r.C + 2 * std::max(r.R - 2, 0));
        }
    }
    // blocks in dequeue order: pass-major, grids with more passes first
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P[a] > P[b]; });
    const int P_max = n ? P[order[0]] : 0;
    std::vector<int4> blk;
    std::vector<int2> blk2;
    long long total = 0;
    for (int p = 0; p < P_max; ++p) {
        for (int g : order) {
            if (P[g] <= p) break;
            const int q = grids[g].pass_off + p;
            for (int j = pjmin[q]; j <= pjmax[q]; ++j) {
                const int lo = std::max(0, j * Lc + pbeta[q]);
                const int hi = std::min(runs[g].R, (j + 1) * Lc + pbeta[q]);
                blk.push_back(make_int4(g, p, j, lo));
                blk2.push_back(make_int2(hi, static_cast<int>(total)));
                total += grids[g].geo.n_strips;
            }
        }
    }
    if (total > INT_MAX / 2) return set_error(SDFG_ERR_INVAL, "chain batch: too many work items");
    total_items = static_cast<int>(total);
    n_ring = static_cast<int>(rings.size());
    if (blk.empty()) {  // keep device arrays non-empty
        blk.push_back(make_int4(0, 0, 0, 0));
        blk2.push_back(make_int2(0, 0));
    }
    if (pk.empty()) pk.push_back(0), pbeta.push_back(0), pjmin.push_back(0), poff.push_back(0);
    // one slab: constants, then the counters every launch resets
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_grids = 0;
    const size_t o_blk = al(o_grids + std::max<size_t>(1, grids.size()) * sizeof(CGrid));
    const size_t o_blk2 = al(o_blk + blk.size() * sizeof(int4));
    const size_t o_k = al(o_blk2 + blk2.size() * sizeof(int2));
    const size_t o_beta = al(o_k + pk.size() * sizeof(int));
    const size_t o_jmin = al(o_beta + pbeta.size() * sizeof(int));
    const size_t o_off = al(o_jmin + pjmin.size() * sizeof(int));
    const size_t o_ring = al(o_off + poff.size() * sizeof(int));
    const size_t o_prog = al(o_ring + std::max<size_t>(1, rings.size()) * sizeof(RingCopy));
    const size_t o_head = al(o_prog + static_cast<size_t>(std::max<long long>(1, n_prog)) * sizeof(int));
    const size_t bytes = al(o_head + sizeof(int));
    if (bytes > slab_bytes) {
        release(s);
        int rc = scratch_alloc(&slab, bytes, s);
        if (rc != SDFG_OK) return rc;
        slab_bytes = bytes;
    }
    std::vector<unsigned char> img(o_prog, 0);
    auto put = [&](size_t at, const void *src, size_t nb) {
        if (nb) memcpy(img.data() + at, src, nb);
    };
    put(o_grids, grids.data(), grids.size() * sizeof(CGrid));
    put(o_blk, blk.data(), blk.size() * sizeof(int4));
    put(o_blk2, blk2.data(), blk2.size() * sizeof(int2));
    put(o_k, pk.data(), pk.size() * sizeof(int));
    put(o_beta, pbeta.data(), pbeta.size() * sizeof(int));
    put(o_jmin, pjmin.data(), pjmin.size() * sizeof(int));
    put(o_off, poff.data(), poff.size() * sizeof(int));
    put(o_ring, rings.data(), rings.size() * sizeof(RingCopy));
    SDFG_CUDA(cudaMemcpyAsync(slab, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    SDFG_CUDA(cudaStreamSynchronize(s));  // the host image must outlive the copy
    const_bytes = o_prog;
    unsigned char *base = static_cast<unsigned char *>(slab);
    CBatchParams *q = static_cast<CBatchParams *>(params);
    if (!q) params = q = new CBatchParams();
    memset(q, 0, sizeof(*q));
    q->grids = reinterpret_cast<const CGrid *>(base + o_grids);
    q->blk = reinterpret_cast<const int4 *>(base + o_blk);
    q->blk2 = reinterpret_cast<const int2 *>(base + o_blk2);
    q->pass_k = reinterpret_cast<const int *>(base + o_k);
    q->pass_beta = reinterpret_cast<const int *>(base + o_beta);
    q->pass_jmin = reinterpret_cast<const int *>(base + o_jmin);
    q->prog_off = reinterpret_cast<const int *>(base + o_off);
    q->prog = reinterpret_cast<int *>(base + o_prog);
    q->head = reinterpret_cast<int *>(base + o_head);
    q->n_blocks = static_cast<int>(blk.size());
    q->total_items = total_items;
    ring = base + o_ring;
    // CTAs: every SM full, or fewer when there are fewer items than warps
    const void *fn = chain_batch_fn(dtype);
    const size_t smem = chain_smem_bytes(dtype, 4);
    SDFG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int bps = 0;
    SDFG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 128, smem));
    DeviceState *st = nullptr;
    int rc = current_device(&st);
    if (rc != SDFG_OK) return rc;
    const long long need = (total + 3) / 4;
    blocks = static_cast<int>(
        std::max<long long>(1, std::min<long long>(need, static_cast<long long>(std::max(bps, 1)) * st->sm_count)));
    return SDFG_OK;
}

int ChainBatch::enqueue(DeviceState *st, cudaStream_t s) {
    if (total_items == 0) return SDFG_OK;
    CBatchParams prm = *static_cast<CBatchParams *>(params);
    prm.err = st->d_err;
    prm.timeout_ns = test_hooks().timeout_ns ? test_hooks().timeout_ns : DEFAULT_TIMEOUT_NS;
    unsigned char *base = static_cast<unsigned char *>(slab);
    SDFG_CUDA(cudaMemsetAsync(base + const_bytes, 0, slab_bytes - const_bytes, s));
    int rc = launch_ring_copy(static_cast<const RingCopy *>(ring), n_ring, max_ring, dtype, s);
    if (rc != SDFG_OK) return rc;
    void *args[] = {&prm};
    TimedLaunch t = stats_begin(FAM_SKEWED, s);
    cudaError_t e = cudaLaunchKernel(chain_batch_fn(dtype), dim3(blocks), dim3(128), args,
                                     chain_smem_bytes(dtype, 4), s);
    stats_end(t, s);
    if (e != cudaSuccess) return cuda_error(e, "chain batch launch");
    return SDFG_OK;
}

void ChainBatch::release(cudaStream_t s) {
    if (slab) cudaFreeAsync(slab, s);
    slab = nullptr;
    slab_bytes = 0;
    delete static_cast<CBatchParams *>(params);
    params = nullptr;
}

}  // namespace sdfg
