// The persistent, dependency-driven Jacobi kernel (batches, tolerance solves,
// server waves) and the finalise copy.  Data structures and the scheduling
// rules are described in persistent.h.
#include "persistent.h"
#include "runtime.h"
#include "temporal_unit.cuh"

namespace sdfg {

// largest i in [0, n) with a[i] <= x (a non-decreasing, a[0] <= x)
__device__ __forceinline__ int find_le(const int *__restrict__ a, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(a + mid) <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Spin (lane-parallel) until every lane's predicate holds; false on timeout.
template <class Pred>
__device__ __forceinline__ bool warp_wait(Pred pred, unsigned long long timeout_ns) {
    if (__all_sync(FULL_MASK, pred())) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        __nanosleep(100);
        if (__all_sync(FULL_MASK, pred())) return true;
        const bool late = globaltimer_ns() - t0 > timeout_ns;
        if (__any_sync(FULL_MASK, late)) return false;
    }
}

template <class ST, int V>
__device__ __forceinline__ bool run_depth(int k, const void *tmap, ST *dst, const GridGeo &g, int s, int q, ST *ring,
                                          uint64_t *bars, uint32_t &ctr, int res, double2 *partial,
                                          unsigned long long timeout_ns) {
    switch (k) {
        case 1: return run_unit<ST, V, 1>(tmap, dst, g, s, q, ring, bars, ctr, res, partial, timeout_ns);
        case 2: return run_unit<ST, V, 2>(tmap, dst, g, s, q, ring, bars, ctr, res, partial, timeout_ns);
        case 4: return run_unit<ST, V, 4>(tmap, dst, g, s, q, ring, bars, ctr, res, partial, timeout_ns);
        default: return run_unit<ST, V, 8>(tmap, dst, g, s, q, ring, bars, ctr, res, partial, timeout_ns);
    }
}

#ifndef SDFG_PK_MINB
#define SDFG_PK_MINB 3  // 128-thread CTAs per SM the register allocation must allow
#endif

template <class ST, int V>
__global__ void __launch_bounds__(128, SDFG_PK_MINB) persistent_kernel(const PLaunch L) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[MAX_WARPS][STAGES];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[warp][s], 1);
        mbar_init_fence();
    }
    __syncwarp();
    ST *ring = reinterpret_cast<ST *>(smem_raw) + static_cast<size_t>(warp) * STAGES * CHUNK_ROWS * 32 * V;
    uint32_t ctr = 0;

    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(L.head, 1);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item >= L.total_items) break;

        // ---- decode (pass p, grid g, unit u) ----
        const int p = find_le(L.level_start, L.P_max, item);
        const int off = item - __ldg(L.level_start + p);
        const int j = find_le(L.units_prefix, __ldg(L.n_active + p), off);
        const int gi = __ldg(L.order + j);
        const int u = off - __ldg(L.units_prefix + j);
        const PGrid &G = L.grids[gi];
        PState *S = L.state + gi;
        const GridGeo geo = G.geo;
        const int s = u % geo.n_strips;
        const int q = u / geo.n_strips;
        const int unit_off = G.unit_off;
        const int pidx = G.pass_off + p;

        // ---- dependencies: the 3x3 neighbourhood finished pass p-1 ----
        if (L.inject_stuck_wait && item == 0) {
            // test hook: wait on a flag nothing ever sets; must time out
            if (!warp_wait([&] { return ld_acquire_gpu(L.done) >= 0x7fffffff; }, L.timeout_ns)) {
                if (lane == 0) set_device_error(L.err, DEV_ERR_TIMEOUT_DEP);
                break;
            }
        }
        if (p > 0) {
            int idx = -1;
            if (lane < 9) {
                const int s2 = s + lane % 3 - 1;
                const int q2 = q + lane / 3 - 1;
                if (s2 >= 0 && s2 < geo.n_strips && q2 >= 0 && q2 < geo.n_segs) idx = unit_off + q2 * geo.n_strips + s2;
            }
            if (!warp_wait([&] { return idx < 0 || ld_acquire_gpu(L.done + idx) >= p; }, L.timeout_ns)) {
                if (lane == 0) set_device_error(L.err, DEV_ERR_TIMEOUT_DEP);
                break;
            }
        }
        bool skip = false;
        if (G.tol_mode) {
            if (p >= 2) {
                const int need = __ldg(L.chk_before + pidx - 1);
                if (!warp_wait([&] { return ld_acquire_gpu(&S->check_done) >= need || ld_acquire_gpu(&S->stop_pass) >= 0; },
                               L.timeout_ns)) {
                    if (lane == 0) set_device_error(L.err, DEV_ERR_TIMEOUT_DEP);
                    break;
                }
            }
            const int stop = ld_acquire_gpu(&S->stop_pass);
            skip = stop >= 0 && stop < p;
        }

        const int info = __ldg(L.pass_info + pidx);
        const int dstb = G.first_dst ^ (p & 1);
        int res = 0;
        if (G.tol_mode) res = ((info & PASS_REF) ? 1 : 0) | ((info & (PASS_CHECK | PASS_FINAL)) ? 2 : 0);
        const int cnum = __ldg(L.chk_before + pidx);
        if (!skip) {
            const int srcb = (p == 0) ? G.cur : (G.first_dst ^ ((p - 1) & 1));
            const void *tm = &G.tm[srcb];
            if (lane == 0) {
                fence_proxy_async_global();  // order the acquired generic writes before TMA reads
                tmap_acquire(tm);
            }
            __syncwarp();
            double2 *partial = res ? L.partials + static_cast<size_t>(cnum & 1) * L.total_units + unit_off + u : nullptr;
            const bool ok = run_depth<ST, V>(info & PASS_K_MASK, tm, static_cast<ST *>(G.buf[dstb]), geo, s, q, ring,
                                             bars[warp], ctr, res, partial, L.timeout_ns);
            if (!ok) {
                if (lane == 0) set_device_error(L.err, DEV_ERR_TIMEOUT_TMA);
                break;
            }
        }
        // ---- publish: this unit finished pass p ----
        // The warp barrier orders every lane's stores before lane 0's release
        // store, which makes them visible at GPU scope before the flag; a
        // reader acquires the flag and then fences the async proxy before its
        // TMA loads.
        __syncwarp();
        if (lane == 0) st_release_gpu(L.done + unit_off + u, p + 1);
        if (skip || !res) continue;

        // ---- reduce pass: the last unit to finish decides ----
        int last = 0;
        if (lane == 0) {
            __threadfence();
            last = atomicAdd(L.chk_count + G.chk_off + cnum, 1) == G.n_units - 1;
        }
        last = __shfl_sync(FULL_MASK, last, 0);
        if (!last) continue;
        __threadfence();
        // decisions are applied in pass order
        if (!warp_wait([&] { return ld_acquire_gpu(&S->check_done) >= cnum; }, L.timeout_ns)) {
            if (lane == 0) set_device_error(L.err, DEV_ERR_TIMEOUT_DEP);
            break;
        }
        double sx = 0.0, sy = 0.0;
        const double2 *pp = L.partials + static_cast<size_t>(cnum & 1) * L.total_units + unit_off;
        for (int v = lane; v < G.n_units; v += 32) {
            const double2 pr = __ldcg(pp + v);
            sx += pr.x;
            sy += pr.y;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            sx += __shfl_xor_sync(FULL_MASK, sx, o);
            sy += __shfl_xor_sync(FULL_MASK, sy, o);
        }
        if (lane == 0) {
            if (ld_acquire_gpu(&S->stop_pass) < 0) {
                double r_ref2 = __ldcg(&S->r_ref2);
                if (info & PASS_REF) {
                    r_ref2 = sx;
                    S->r_ref2 = sx;
                }
                if (info & (PASS_CHECK | PASS_FINAL)) {
                    const double rel = r_ref2 > 0.0 ? sqrt(sy) / sqrt(r_ref2) : 0.0;
                    S->rel = rel;
                    const bool stop = (info & PASS_FINAL) || ((info & PASS_CHECK) && rel <= G.tol);
                    if (stop) {
                        S->steps_done = __ldg(L.pass_tend + pidx);
                        S->final_buf = dstb;
                        __threadfence();
                        st_release_gpu(&S->stop_pass, p);
                    }
                }
            }
            __threadfence();
            st_release_gpu(&S->check_done, cnum + 1);
        }
    }
}

// ------------------------------------------------------------- finalise ----
// Copy each grid's result buffer into the caller's `out` when they differ.
struct FinalDesc {
    const void *src;  // unused when the result already sits in dst
    void *dst;
    int ld_src, ld_dst, rows, cols;
    int src_sel;      // -1: use state[g].final_buf of `grids`; otherwise a buffer index
    int grid;         // index into grids/state
};

template <class ST>
__global__ void finalize_kernel(const FinalDesc *__restrict__ fd, const PGrid *__restrict__ grids,
                                const PState *__restrict__ state) {
    const FinalDesc d = fd[blockIdx.y];
    const int sel = d.src_sel >= 0 ? d.src_sel : state[d.grid].final_buf;
    const ST *src = static_cast<const ST *>(grids[d.grid].buf[sel]);
    ST *dst = static_cast<ST *>(d.dst);
    if (static_cast<const void *>(src) == static_cast<void *>(dst) && d.ld_src == d.ld_dst) return;
    for (int i = blockIdx.x; i < d.rows; i += gridDim.x)
        for (int j = threadIdx.x; j < d.cols; j += blockDim.x)
            dst[static_cast<size_t>(i) * d.ld_dst + j] = src[static_cast<size_t>(i) * d.ld_src + j];
}

// ------------------------------------------------------------- launchers ---
template <class ST>
static const void *pk_fn() {
    return reinterpret_cast<const void *>(
        &persistent_kernel<ST, Store<ST>::bytes == 8 ? 2 : (Store<ST>::bytes == 4 ? SDFG_F32_V : 4)>);
}

static const void *persistent_fn(int dtype) {
    switch (dtype) {
        case SDFG_F32: return pk_fn<float>();
        case SDFG_BF16: return pk_fn<__nv_bfloat16>();
        default: return pk_fn<double>();
    }
}

int persistent_blocks_per_sm(int dtype, int warps) {
    const void *fn = persistent_fn(dtype);
    const size_t smem = temporal_smem_bytes(dtype, warps);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, warps * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int launch_persistent(const PLaunch &L, int dtype, int warps, int blocks, cudaStream_t s) {
    const void *fn = persistent_fn(dtype);
    const size_t smem = temporal_smem_bytes(dtype, warps);  // attribute raised by persistent_blocks_per_sm
    PLaunch l = L;
    void *args[] = {&l};
    TimedLaunch t = stats_begin(FAM_PERSISTENT, s);
    cudaError_t e = cudaLaunchKernel(fn, dim3(blocks), dim3(warps * 32), args, smem, s);
    stats_end(t, s);
    if (e != cudaSuccess) return cuda_error(e, "persistent launch");
    return SDFG_OK;
}

int launch_finalize(const void *fdescs, int n, const PGrid *grids, const PState *state, int dtype, int max_rows,
                    cudaStream_t s) {
    if (n <= 0) return SDFG_OK;
    dim3 grid(static_cast<unsigned>(std::min(std::max(max_rows, 1), 1024)), static_cast<unsigned>(n));
    const FinalDesc *fd = static_cast<const FinalDesc *>(fdescs);
    TimedLaunch t = stats_begin(FAM_COPY, s);
    switch (dtype) {
        case SDFG_F32: finalize_kernel<float><<<grid, 256, 0, s>>>(fd, grids, state); break;
        case SDFG_BF16: finalize_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(fd, grids, state); break;
        default: finalize_kernel<double><<<grid, 256, 0, s>>>(fd, grids, state); break;
    }
    stats_end(t, s);
    SDFG_CUDA(cudaGetLastError());
    return SDFG_OK;
}

size_t final_desc_bytes() { return sizeof(FinalDesc); }

}  // namespace sdfg
