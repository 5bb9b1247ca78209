// Batches of uneven grids in one persistent launch, replayable as a CUDA
// graph; single-grid tolerance solves reuse the same machinery.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>

#include "autotune.h"
#include "chainbatch.h"
#include "launchset.h"

namespace sdfg {

int validate_grid(const void *in, const void *out, int R, int C, int ld, long long T, int dtype, const char *who);

TestHooks &test_hooks() {
    static TestHooks h;
    return h;
}

// ------------------------------------------------------------ pass plans ----
void plan_grid_passes(int t0, int steps, int T_cap, bool tol_mode, int check_stride, int k, std::vector<int> &info,
                      std::vector<int> &tend) {
    int t = t0;
    const int t_end = t0 + steps;
    while (t < t_end) {
        // next stop: the end of this launch, or the next check step
        int stop = t_end;
        if (tol_mode) {
            const int next_chk = (t / check_stride + 1) * check_stride;
            stop = std::min(stop, next_chk);
        }
        int left = stop - t;
        while (left > 0) {
            int d = k;
            if (left < k) {
                d = 1;
                while (d * 2 <= left) d *= 2;
            }
            int flags = d;
            if (tol_mode) {
                if (t == 0) flags |= PASS_REF;
                if ((t + d) % check_stride == 0) flags |= PASS_CHECK;
                if (t + d == T_cap) flags |= PASS_FINAL;
            }
            info.push_back(flags);
            tend.push_back(t + d);
            t += d;
            left -= d;
        }
    }
}

// ------------------------------------------------------------ LaunchSet -----
int LaunchSet::build(const std::vector<GridRun> &runs) {
    const int n = static_cast<int>(runs.size());
    grids.assign(n, PGrid());
    state0.assign(n, PState());
    pass_info.clear();
    chk_before.clear();
    pass_tend.clear();
    last_dst.assign(n, -1);
    std::vector<int> P(n, 0), units(n, 0);
    total_units = 0;
    n_reduce = 0;
    const int W = 32 * lane_cols(dtype_bytes(dtype));
    for (int g = 0; g < n; ++g) {
        const GridRun &r = runs[g];
        PGrid &G = grids[g];
        memset(&G, 0, sizeof(G));
        const bool tol_mode = r.tol > 0.0;
        G.geo = plan_geometry(r.R, r.C, r.ld, dtype, k, r.seg_rows > 0 ? r.seg_rows : 96, 0);
        G.n_units = G.geo.n_strips * G.geo.n_segs;
        G.unit_off = total_units;
        G.pass_off = static_cast<int>(pass_info.size());
        G.t0 = r.t0;
        G.cur = r.cur;
        G.chk_off = n_reduce;
        G.tol_mode = tol_mode ? 1 : 0;
        G.tol = r.tol;
        for (int b = 0; b < 3; ++b) {
            G.buf[b] = r.buf[b];
            if (r.buf[b] && r.tmaps) {
                G.tm[b] = r.tmaps[b];
            } else if (r.buf[b]) {
                int rc = encode_tmap(&G.tm[b], r.buf[b], dtype, r.R, r.C, r.ld, W);
                if (rc != SDFG_OK) return rc;
            }
        }
        if (r.steps > 0 && r.R >= 3 && r.C >= 3)
            plan_grid_passes(r.t0, r.steps, r.T_cap, tol_mode, check_stride, k, pass_info, pass_tend);
        G.P = static_cast<int>(pass_info.size()) - G.pass_off;
        P[g] = G.P;
        units[g] = G.n_units;
        int nred = 0;
        for (int p = 0; p < G.P; ++p) {
            chk_before.push_back(nred);
            if (tol_mode && (pass_info[G.pass_off + p] & PASS_REDUCE)) ++nred;
        }
        n_reduce += nred;
        if (G.cur == 2)
            G.first_dst = (G.P % 2 == 1) ? 0 : 1;
        else
            G.first_dst = 1 - G.cur;
        last_dst[g] = G.P > 0 ? (G.first_dst ^ ((G.P - 1) & 1)) : G.cur;
        total_units += G.n_units;
        PState &S = state0[g];
        S.stop_pass = -1;
        S.steps_done = r.t0;
        S.final_buf = r.cur;
        S.check_done = 0;
        S.r_ref2 = r.r_ref2;
        S.rel = 0.0;
    }
    order.resize(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P[a] > P[b]; });
    P_max = n ? P[order[0]] : 0;
    units_prefix.assign(n + 1, 0);
    for (int j = 0; j < n; ++j) units_prefix[j + 1] = units_prefix[j] + units[order[j]];
    n_active.assign(std::max(P_max, 1), 0);
    level_start.assign(P_max + 1, 0);
    int na = n;
    for (int p = 0; p < P_max; ++p) {
        while (na > 0 && P[order[na - 1]] <= p) --na;
        n_active[p] = na;
        level_start[p + 1] = level_start[p] + units_prefix[na];
    }
    total_items = level_start[P_max];
    if (pass_info.empty()) {  // keep device arrays non-empty
        pass_info.push_back(0);
        chk_before.push_back(0);
        pass_tend.push_back(0);
    }
    return SDFG_OK;
}

namespace {
struct SlabLayout {
    size_t grids, state, state_init, pass_info, chk_before, pass_tend, level_start, n_active, units_prefix, order,
        done, partials, chk_count, head, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

SlabLayout layout_of(const LaunchSet &ls) {
    SlabLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes, size_t al) {
        o = align_up(o, al);
        size_t at = o;
        o += std::max<size_t>(bytes, al);
        return at;
    };
    const size_t n = ls.grids.size();
    L.grids = take(n * sizeof(PGrid), 128);
    L.state = take(n * sizeof(PState), 64);
    L.state_init = take(n * sizeof(PState), 64);
    L.pass_info = take(ls.pass_info.size() * 4, 16);
    L.chk_before = take(ls.chk_before.size() * 4, 16);
    L.pass_tend = take(ls.pass_tend.size() * 4, 16);
    L.level_start = take(ls.level_start.size() * 4, 16);
    L.n_active = take(ls.n_active.size() * 4, 16);
    L.units_prefix = take(ls.units_prefix.size() * 4, 16);
    L.order = take(ls.order.size() * 4, 16);
    L.done = take(static_cast<size_t>(ls.total_units) * 4, 16);
    L.partials = take(static_cast<size_t>(2) * ls.total_units * sizeof(double2), 16);
    L.chk_count = take(static_cast<size_t>(std::max(ls.n_reduce, 1)) * 4, 16);
    L.head = take(4, 16);
    L.total = align_up(o, 256);
    return L;
}
}  // namespace

int LaunchSet::upload(cudaStream_t s) {
    const SlabLayout lay = layout_of(*this);
    if (lay.total > slab_bytes) {
        if (slab) cudaFreeAsync(slab, s);
        slab = nullptr;
        slab_bytes = 0;
        int rc = scratch_alloc(&slab, lay.total, s);
        if (rc != SDFG_OK) return rc;
        slab_bytes = lay.total;
    }
    // host image of the constant part, then one copy
    std::vector<unsigned char> img(lay.done, 0);
    auto put = [&](size_t at, const void *src, size_t bytes) {
        if (bytes) memcpy(img.data() + at, src, bytes);
    };
    put(lay.grids, grids.data(), grids.size() * sizeof(PGrid));
    put(lay.state, state0.data(), state0.size() * sizeof(PState));
    put(lay.state_init, state0.data(), state0.size() * sizeof(PState));
    put(lay.pass_info, pass_info.data(), pass_info.size() * 4);
    put(lay.chk_before, chk_before.data(), chk_before.size() * 4);
    put(lay.pass_tend, pass_tend.data(), pass_tend.size() * 4);
    put(lay.level_start, level_start.data(), level_start.size() * 4);
    put(lay.n_active, n_active.data(), n_active.size() * 4);
    put(lay.units_prefix, units_prefix.data(), units_prefix.size() * 4);
    put(lay.order, order.data(), order.size() * 4);
    SDFG_CUDA(cudaMemcpyAsync(slab, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    // the host image must outlive the copy
    SDFG_CUDA(cudaStreamSynchronize(s));
    unsigned char *base = static_cast<unsigned char *>(slab);
    L.grids = reinterpret_cast<const PGrid *>(base + lay.grids);
    L.state = reinterpret_cast<PState *>(base + lay.state);
    L.pass_info = reinterpret_cast<const int *>(base + lay.pass_info);
    L.chk_before = reinterpret_cast<const int *>(base + lay.chk_before);
    L.pass_tend = reinterpret_cast<const int *>(base + lay.pass_tend);
    L.level_start = reinterpret_cast<const int *>(base + lay.level_start);
    L.n_active = reinterpret_cast<const int *>(base + lay.n_active);
    L.units_prefix = reinterpret_cast<const int *>(base + lay.units_prefix);
    L.order = reinterpret_cast<const int *>(base + lay.order);
    L.done = reinterpret_cast<int *>(base + lay.done);
    L.partials = reinterpret_cast<double2 *>(base + lay.partials);
    L.chk_count = reinterpret_cast<int *>(base + lay.chk_count);
    L.head = reinterpret_cast<int *>(base + lay.head);
    L.total_items = total_items;
    L.total_units = total_units;
    L.P_max = P_max;
    L.inject_stuck_wait = test_hooks().inject_stuck_wait;
    L.timeout_ns = test_hooks().timeout_ns ? test_hooks().timeout_ns : DEFAULT_TIMEOUT_NS;
    DeviceState *st = nullptr;
    int rc = current_device(&st);
    if (rc != SDFG_OK) return rc;
    const int bps = std::max(1, persistent_blocks_per_sm(dtype, warps));
    const long long need = (static_cast<long long>(total_items) + warps - 1) / warps;
    blocks = static_cast<int>(std::max<long long>(1, std::min<long long>(need, static_cast<long long>(bps) * st->sm_count)));
    return SDFG_OK;
}

int LaunchSet::reset(cudaStream_t s) {
    const SlabLayout lay = layout_of(*this);
    unsigned char *base = static_cast<unsigned char *>(slab);
    SDFG_CUDA(cudaMemsetAsync(base + lay.done, 0, lay.total - lay.done, s));
    SDFG_CUDA(cudaMemcpyAsync(base + lay.state, base + lay.state_init, grids.size() * sizeof(PState),
                              cudaMemcpyDeviceToDevice, s));
    return SDFG_OK;
}

void LaunchSet::release(cudaStream_t s) {
    if (slab) cudaFreeAsync(slab, s);
    slab = nullptr;
    slab_bytes = 0;
}

int enqueue_persistent(LaunchSet &ls, DeviceState *st, cudaStream_t s) {
    if (ls.total_items == 0) return SDFG_OK;
    int rc = ls.reset(s);
    if (rc != SDFG_OK) return rc;
    ls.L.err = st->d_err;
    return launch_persistent(ls.L, ls.dtype, ls.warps, ls.blocks, s);
}

}  // namespace sdfg

using namespace sdfg;

// ------------------------------------------------------------- the plan -----
struct sdfg_batch_plan {
    int n = 0;
    int dtype = SDFG_F32;
    int check_stride = 64;
    DeviceState *st = nullptr;
    std::vector<sdfg_desc> descs;
    std::vector<int> kind;  // 0 nothing, 1 copy only, 2 persistent
    std::vector<int> ld_int;
    std::vector<void *> owned;
    std::vector<int> staged_in;   // grid index of staged inputs
    std::vector<void *> staged_in_buf;
    LaunchSet ls;            // grids on the persistent kernel
    ChainBatch cb;           // large fixed-step grids on the skewed-chain kernel
    std::vector<char> on_chain;
    int n_pers = 0, n_chain = 0;
    void *d_final = nullptr;  // finalise descriptors of the persistent grids
    int n_final = 0;
    int max_rows = 0;
    void *d_gcopy = nullptr;  // result copies of the chain grids
    int n_gcopy = 0;
    int max_rows_gc = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done_ev = nullptr;
    std::vector<PState> state_host;
};

static int plan_enqueue(sdfg_batch_plan *p, cudaStream_t s) {
    const int S = dtype_bytes(p->dtype);
    for (int g = 0; g < p->n; ++g) {
        const sdfg_desc &d = p->descs[g];
        if (p->kind[g] == 1 && d.in != d.out) {
            SDFG_CUDA(cudaMemcpy2DAsync(d.out, static_cast<size_t>(d.ld) * S, d.in, static_cast<size_t>(d.ld) * S,
                                        static_cast<size_t>(d.cols) * S, d.rows, cudaMemcpyDeviceToDevice, s));
        }
    }
    for (size_t i = 0; i < p->staged_in.size(); ++i) {
        const sdfg_desc &d = p->descs[p->staged_in[i]];
        SDFG_CUDA(cudaMemcpy2DAsync(p->staged_in_buf[i], static_cast<size_t>(p->ld_int[p->staged_in[i]]) * S, d.in,
                                    static_cast<size_t>(d.ld) * S, static_cast<size_t>(d.cols) * S, d.rows,
                                    cudaMemcpyDeviceToDevice, s));
    }
    // the chain grids first (their launch is the longer-lived), then the
    // persistent grids, on the same stream
    int rc = SDFG_OK;
    if (p->n_chain) {
        rc = p->cb.enqueue(p->st, s);
        if (rc == SDFG_OK)
            rc = launch_grid_copy(static_cast<const GridCopy *>(p->d_gcopy), p->n_gcopy, p->max_rows_gc, p->dtype, s);
        if (rc != SDFG_OK) return rc;
    }
    if (p->n_pers) {
        rc = enqueue_persistent(p->ls, p->st, s);
        if (rc != SDFG_OK) return rc;
        if (p->n_final)
            rc = launch_finalize(p->d_final, p->n_final, p->ls.L.grids, p->ls.L.state, p->dtype, p->max_rows, s);
    }
    return rc;
}

static void plan_free(sdfg_batch_plan *p) {
    if (!p) return;
    cudaStream_t s = p->cap;
    if (p->done_ev) cudaEventSynchronize(p->done_ev);  // the last run may still use the buffers
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (void *b : p->owned) cudaFreeAsync(b, s);
    if (p->d_final) cudaFreeAsync(p->d_final, s);
    if (p->d_gcopy) cudaFreeAsync(p->d_gcopy, s);
    p->ls.release(s);
    p->cb.release(s);
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    delete p;
}

static int plan_build(sdfg_batch_plan **out, const sdfg_desc *desc, int n, int check_stride, const sdfg_config *cfg,
                      bool use_graph) {
    *out = nullptr;
    if (n < 0 || (n > 0 && !desc)) return set_error(SDFG_ERR_INVAL, "batch: bad descriptor array");
    int dtype = n ? desc[0].dtype : SDFG_F32;
    bool any_tol = false;
    for (int g = 0; g < n; ++g) {
        const sdfg_desc &d = desc[g];
        int rc = validate_grid(d.in, d.out, d.rows, d.cols, d.ld, d.T, d.dtype, "batch");
        if (rc != SDFG_OK) return rc;
        if (d.dtype != dtype) return set_error(SDFG_ERR_INVAL, "batch: all descriptors must share one dtype");
        if (!(d.tol >= 0.0) || !isfinite(d.tol)) return set_error(SDFG_ERR_INVAL, "batch: tol must be >= 0");
        if (d.t_start < 0 || d.t_start > d.T || !(d.r_first2 >= 0.0))
            return set_error(SDFG_ERR_INVAL, "batch: need 0 <= t_start <= T and r_first2 >= 0");
        any_tol |= d.tol > 0.0;
    }
    if (any_tol && check_stride < 1) return set_error(SDFG_ERR_INVAL, "batch: check_stride must be >= 1");
    sdfg_config c = {SDFG_KERNEL_PERSISTENT, 0, 0, 0};
    if (cfg) {
        c = *cfg;
    } else if (n > 0) {
        double area = 0.0;
        for (int g = 0; g < n; ++g) area += static_cast<double>(desc[g].rows) * desc[g].cols;
        area /= n;
        sdfg_config tuned;
        if (autotune_lookup(-n, -static_cast<int>(area > 2e9 ? 2e9 : area), dtype, &tuned)) c = tuned;
    }
    if (c.k != 0 && !depth_supported(c.k)) return set_error(SDFG_ERR_INVAL, "batch: k must be 1, 2, 4 or 8");
    if (c.warps < 0 || c.warps > MAX_WARPS || c.seg_rows < 0) return set_error(SDFG_ERR_INVAL, "batch: bad config");
    DeviceState *st = nullptr;
    int rc = current_device(&st);
    if (rc != SDFG_OK) return rc;

    sdfg_batch_plan *p = new sdfg_batch_plan();
    p->n = n;
    p->dtype = dtype;
    p->check_stride = std::max(check_stride, 1);
    p->st = st;
    p->descs.assign(desc, desc + n);
    p->kind.assign(n, 0);
    p->ld_int.assign(n, 0);
    p->ls.dtype = dtype;
    p->ls.k = c.k ? c.k : default_depth(dtype);
    p->ls.warps = c.warps ? c.warps : 4;
    p->ls.check_stride = p->check_stride;
    cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_error(e, "batch plan stream/event");
    }
    cudaStream_t s = p->cap;
    const int S = dtype_bytes(dtype);
    std::vector<GridRun> runs;
    std::vector<int> run_of(n, -1);
    std::vector<FinalDescHost> fin;
    for (int g = 0; g < n && rc == SDFG_OK; ++g) {
        const sdfg_desc &d = desc[g];
        if (d.rows == 0 || d.cols == 0) continue;
        if (d.rows < 3 || d.cols < 3 || d.T == d.t_start) {
            p->kind[g] = 1;
            continue;
        }
        p->kind[g] = 2;
        GridRun r;
        r.R = d.rows;
        r.C = d.cols;
        r.t0 = d.t_start;
        r.steps = d.T - d.t_start;
        r.T_cap = d.T;
        r.tol = d.tol;
        r.r_ref2 = d.r_first2;
        r.seg_rows = c.seg_rows;
        const bool aligned = tma_compatible(d.in, d.ld, dtype) && tma_compatible(d.out, d.ld, dtype);
        void *scr = nullptr;
        if (aligned) {
            r.ld = d.ld;
            rc = scratch_alloc(&scr, static_cast<size_t>(d.rows) * d.ld * S, s);
            if (rc != SDFG_OK) break;
            p->owned.push_back(scr);
            r.buf[0] = d.out;
            r.buf[1] = scr;
            r.buf[2] = const_cast<void *>(d.in);
            r.cur = (d.in == d.out) ? 0 : 2;
            if (d.in == d.out) r.buf[2] = nullptr;
        } else {
            r.ld = (d.cols + 31) / 32 * 32;
            const size_t bytes = static_cast<size_t>(d.rows) * r.ld * S;
            void *a = nullptr, *b = nullptr;
            rc = scratch_alloc(&a, bytes, s);
            if (rc == SDFG_OK) rc = scratch_alloc(&b, bytes, s);
            if (rc == SDFG_OK) rc = scratch_alloc(&scr, bytes, s);
            for (void *x : {a, b, scr})
                if (x) p->owned.push_back(x);
            if (rc != SDFG_OK) break;
            r.buf[0] = b;
            r.buf[1] = scr;
            r.buf[2] = a;
            r.cur = 2;
            p->staged_in.push_back(g);
            p->staged_in_buf.push_back(a);
        }
        p->ld_int[g] = r.ld;
        run_of[g] = static_cast<int>(runs.size());
        runs.push_back(r);
    }
    // SDFG_KERNEL_SKEWED: large fixed-step grids on the chain kernel, every
    // other grid on the persistent kernel (small grids keep more concurrent
    // work in its per-unit wavefront than in chains of a few chunks)
    const long long min_pts = test_hooks().chain_min_points >= 0 ? test_hooks().chain_min_points : (1LL << 20);
    std::vector<GridRun> runs_c, runs_p;
    std::vector<int> sub(n, -1);
    p->on_chain.assign(n, 0);
    for (int g = 0; g < n; ++g) {
        if (run_of[g] < 0) continue;
        const GridRun &r = runs[run_of[g]];
        const bool ch = c.kernel == SDFG_KERNEL_SKEWED && r.tol == 0.0 && static_cast<long long>(r.R) * r.C >= min_pts;
        p->on_chain[g] = ch ? 1 : 0;
        sub[g] = static_cast<int>(ch ? runs_c.size() : runs_p.size());
        (ch ? runs_c : runs_p).push_back(r);
    }
    p->n_chain = static_cast<int>(runs_c.size());
    p->n_pers = static_cast<int>(runs_p.size());
    if (rc == SDFG_OK && p->n_chain) {
        p->cb.dtype = dtype;
        // chains at the library's depth (8 for FP32/BF16): their long
        // streamed units make the deepest fusion pay; cfg->k applies to the
        // persistent part
        p->cb.k = default_depth(dtype);
        p->cb.L = test_hooks().chain_rows;
        rc = p->cb.build(runs_c, s);
        std::vector<GridCopy> gc;
        for (int g = 0; g < n && rc == SDFG_OK; ++g) {
            if (!p->on_chain[g]) continue;
            const GridRun &r = runs_c[sub[g]];
            const void *res = r.buf[p->cb.last_dst[sub[g]]];
            if (res == desc[g].out) continue;
            gc.push_back(GridCopy{res, desc[g].out, desc[g].rows, desc[g].cols, r.ld, desc[g].ld});
            p->max_rows_gc = std::max(p->max_rows_gc, desc[g].rows);
        }
        if (rc == SDFG_OK && !gc.empty()) {
            rc = scratch_alloc(&p->d_gcopy, gc.size() * sizeof(GridCopy), s);
            if (rc == SDFG_OK) {
                e = cudaMemcpyAsync(p->d_gcopy, gc.data(), gc.size() * sizeof(GridCopy), cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) rc = cuda_error(e, "batch plan upload");
            }
            p->n_gcopy = static_cast<int>(gc.size());
        }
    }
    if (rc == SDFG_OK) rc = p->ls.build(runs_p);
    if (rc == SDFG_OK) {
        for (int g = 0; g < n; ++g) {
            if (run_of[g] < 0 || p->on_chain[g]) continue;
            const int ri = sub[g];
            const bool staged = runs_p[ri].buf[0] != desc[g].out;
            const bool tol_mode = desc[g].tol > 0.0;
            if (!staged && !tol_mode && p->ls.last_dst[ri] == 0) continue;
            FinalDescHost f;
            f.src = nullptr;
            f.dst = desc[g].out;
            f.ld_src = runs_p[ri].ld;
            f.ld_dst = desc[g].ld;
            f.rows = desc[g].rows;
            f.cols = desc[g].cols;
            f.src_sel = tol_mode ? -1 : p->ls.last_dst[ri];
            f.grid = ri;
            fin.push_back(f);
            p->max_rows = std::max(p->max_rows, desc[g].rows);
        }
    }
    if (rc == SDFG_OK && p->n_pers) rc = p->ls.upload(s);
    if (rc == SDFG_OK && p->n_pers && !fin.empty()) {
        rc = scratch_alloc(&p->d_final, fin.size() * sizeof(FinalDescHost), s);
        if (rc == SDFG_OK) {
            e = cudaMemcpyAsync(p->d_final, fin.data(), fin.size() * sizeof(FinalDescHost), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_error(e, "batch plan upload");
        }
        p->n_final = static_cast<int>(fin.size());
    }
    if (rc == SDFG_OK && use_graph) {
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "cudaStreamBeginCapture");
        } else {
            stats_suspend(true);
            const int rc2 = plan_enqueue(p, s);
            stats_suspend(false);
            e = cudaStreamEndCapture(s, &p->graph);
            if (rc2 != SDFG_OK)
                rc = rc2;
            else if (e != cudaSuccess)
                rc = cuda_error(e, "cudaStreamEndCapture");
            else if ((e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess)
                rc = cuda_error(e, "cudaGraphInstantiate");
        }
    }
    if (rc != SDFG_OK) {
        plan_free(p);
        return rc;
    }
    p->state_host.resize(p->ls.grids.size());
    *out = p;
    return SDFG_OK;
}

static int plan_run(sdfg_batch_plan *p, cudaStream_t s) {
    // order the plan's work after everything already on `s`
    if (p->exec) {
        SDFG_CUDA(cudaGraphLaunch(p->exec, s));
    } else {
        int rc = plan_enqueue(p, s);
        if (rc != SDFG_OK) return rc;
    }
    SDFG_CUDA(cudaEventRecord(p->done_ev, s));
    return SDFG_OK;
}

static int plan_results(sdfg_batch_plan *p, sdfg_desc *desc, int n) {
    if (n != p->n) return set_error(SDFG_ERR_INVAL, "batch results: expected %d descriptors, got %d", p->n, n);
    SDFG_CUDA(cudaEventSynchronize(p->done_ev));
    int errw = 0;
    SDFG_CUDA(cudaMemcpy(&errw, p->st->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (errw) {
        cudaMemset(p->st->d_err, 0, sizeof(int));
        for (int g = 0; g < n; ++g) desc[g].status = SDFG_ERR_TIMEOUT;
        return set_error(SDFG_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", errw);
    }
    if (!p->state_host.empty())
        SDFG_CUDA(cudaMemcpy(p->state_host.data(), p->ls.L.state, p->state_host.size() * sizeof(PState),
                             cudaMemcpyDeviceToHost));
    int ri = 0;
    for (int g = 0; g < n; ++g) {
        const sdfg_desc &d = p->descs[g];
        desc[g].status = SDFG_OK;
        desc[g].rel_residual = 0.0;
        desc[g].r_first2 = d.r_first2;
        if (p->kind[g] == 0) {
            desc[g].steps_done = 0;
        } else if (p->kind[g] == 1) {
            desc[g].steps_done = (d.rows < 3 || d.cols < 3) ? d.T : d.t_start;
        } else if (p->on_chain[g]) {
            desc[g].steps_done = d.T;  // fixed-step grids only
        } else {
            const PState &S = p->state_host[ri++];
            if (d.tol > 0.0) {
                desc[g].steps_done = S.steps_done;
                desc[g].rel_residual = S.rel;
                desc[g].r_first2 = S.r_ref2;
            } else {
                desc[g].steps_done = d.T;
            }
        }
    }
    return SDFG_OK;
}

extern "C" int sdfg_batch_plan_create(sdfg_batch_plan **plan, const sdfg_desc *desc, int n, int check_stride,
                                      const sdfg_config *cfg, void *stream) {
    (void)stream;
    if (!plan) return set_error(SDFG_ERR_INVAL, "sdfg_batch_plan_create: null plan pointer");
    return plan_build(plan, desc, n, check_stride, cfg, true);
}

extern "C" int sdfg_batch_plan_run(sdfg_batch_plan *plan, void *stream) {
    if (!plan) return set_error(SDFG_ERR_INVAL, "sdfg_batch_plan_run: null plan");
    return plan_run(plan, static_cast<cudaStream_t>(stream));
}

extern "C" int sdfg_batch_plan_results(sdfg_batch_plan *plan, sdfg_desc *desc, int n) {
    if (!plan || (n > 0 && !desc)) return set_error(SDFG_ERR_INVAL, "sdfg_batch_plan_results: null argument");
    return plan_results(plan, desc, n);
}

extern "C" int sdfg_batch_plan_destroy(sdfg_batch_plan *plan) {
    plan_free(plan);
    return SDFG_OK;
}

extern "C" int sdfg_jacobi2d_batch(sdfg_desc *desc, int n, int check_stride, void *stream) {
    sdfg_batch_plan *p = nullptr;
    int rc = plan_build(&p, desc, n, check_stride, nullptr, false);
    if (rc != SDFG_OK) return rc;
    rc = plan_run(p, static_cast<cudaStream_t>(stream));
    if (rc == SDFG_OK) rc = plan_results(p, desc, n);
    plan_free(p);
    return rc;
}

extern "C" int sdfg_jacobi2d_solve(sdfg_desc *desc, int check_stride, const sdfg_config *cfg, void *stream) {
    if (!desc) return set_error(SDFG_ERR_INVAL, "sdfg_jacobi2d_solve: null descriptor");
    sdfg_config c = {SDFG_KERNEL_PERSISTENT, 0, 0, 0};
    if (cfg) c = *cfg;
    if (c.seg_rows == 0) {
        // one wave of units over the whole GPU for a single grid
        DeviceState *st = nullptr;
        int rc = current_device(&st);
        if (rc != SDFG_OK) return rc;
        const int k = c.k ? c.k : default_depth(desc->dtype);
        const GridGeo g = plan_geometry(desc->rows, desc->cols, desc->ld, desc->dtype, k, 0,
                                        static_cast<long long>(st->sm_count) * 8);
        c.seg_rows = g.H;
    }
    sdfg_batch_plan *p = nullptr;
    int rc = plan_build(&p, desc, 1, check_stride, &c, false);
    if (rc != SDFG_OK) return rc;
    rc = plan_run(p, static_cast<cudaStream_t>(stream));
    if (rc == SDFG_OK) rc = plan_results(p, desc, 1);
    plan_free(p);
    return rc;
}

// ---------------------------------------------------------- batch tuner -----
// Candidates: the persistent kernel at fused depth k in {4, 8} x segment
// height in {96, 128, 192, 256, 384}, and, when no grid solves to a
// tolerance, the hybrid (large grids on the chain kernel) at k in {4, 8} x
// segment height in {128, 256}.
// Each is built as a plan over the caller's batch, run once to warm up and
// once timed; the fastest is cached under the batch's class (dtype, grid
// count and mean area, both power-of-two buckets) and returned.
extern "C" int sdfg_autotune_batch(const sdfg_desc *desc, int n, int check_stride, sdfg_config *best, void *stream) {
    (void)stream;
    if (!best || n < 1 || !desc) return set_error(SDFG_ERR_INVAL, "sdfg_autotune_batch: bad argument");
    double area = 0.0;
    for (int g = 0; g < n; ++g) area += static_cast<double>(desc[g].rows) * desc[g].cols;
    area /= n;
    const int dtype = desc[0].dtype;
    const int ks[] = {4, 8};
    const int segs[] = {96, 128, 192, 256, 384};
    bool any_tol = false;
    for (int g = 0; g < n; ++g) any_tol |= desc[g].tol > 0.0;
    std::vector<sdfg_config> cands;
    for (int k : ks) {
        if (dtype == SDFG_F64 && k > 4) continue;
        for (int seg : segs) cands.push_back(sdfg_config{SDFG_KERNEL_PERSISTENT, k, seg, 4});
        // large fixed-step grids on the chain kernel, the rest on the
        // persistent kernel with this segment height
        if (!any_tol)
            for (int seg : {128, 256}) cands.push_back(sdfg_config{SDFG_KERNEL_SKEWED, k, seg, 4});
    }
    float best_ms = 1e30f;
    sdfg_config winner = {SDFG_KERNEL_PERSISTENT, default_depth(dtype), 96, 4};
    std::vector<sdfg_desc> tmp(desc, desc + n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = SDFG_OK;
    for (const sdfg_config &c : cands) {
        sdfg_batch_plan *p = nullptr;
        rc = plan_build(&p, desc, n, check_stride, &c, false);
        if (rc != SDFG_OK) break;
        cudaStream_t s = p->cap;
        rc = plan_run(p, s);
        if (rc == SDFG_OK) {
            cudaEventRecord(e0, s);
            rc = plan_run(p, s);
            cudaEventRecord(e1, s);
        }
        if (rc == SDFG_OK) rc = plan_results(p, tmp.data(), n);
        float ms = 0.f;
        if (rc == SDFG_OK) cudaEventElapsedTime(&ms, e0, e1);
        plan_free(p);
        if (rc != SDFG_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            winner = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SDFG_OK) return rc;
    autotune_store(-n, -static_cast<int>(area > 2e9 ? 2e9 : area), dtype, winner);
    *best = winner;
    return SDFG_OK;
}

extern "C" int sdfg_test_hook(int hook, long long value) {
    switch (hook) {
        case 1: test_hooks().inject_stuck_wait = value ? 1 : 0; return SDFG_OK;
        case 2: test_hooks().timeout_ns = value > 0 ? static_cast<unsigned long long>(value) : 0; return SDFG_OK;
        case 3: test_hooks().chain_min_points = value; return SDFG_OK;
        case 4: test_hooks().chain_rows = value > 0 ? static_cast<int>(value) : 0; return SDFG_OK;
        default: return set_error(SDFG_ERR_INVAL, "unknown test hook %d", hook);
    }
}
