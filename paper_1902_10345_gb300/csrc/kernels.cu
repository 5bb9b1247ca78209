// Single-grid kernels: the naive one-step kernel, the temporal-blocked pass
// kernel (K fused steps per launch), and a pitched 2-D copy; plus their host
// launchers.
#include "runtime.h"
#include "temporal_unit.cuh"

namespace sdfg {

// ------------------------------------------------------------ naive step ----
// One timestep, one thread per point (paper Sec. 3: a map over the interior,
// scheduled as one GPU thread per map instance).  Boundary points are copied.
template <class ST>
__global__ void __launch_bounds__(256) naive_step_kernel(const ST *__restrict__ A, ST *__restrict__ B, int R, int C,
                                                         int ld) {
    using CT = typename Store<ST>::CT;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C) return;
    for (int i = blockIdx.y; i < R; i += gridDim.y) {
        const size_t at = static_cast<size_t>(i) * ld + j;
        ST v;
        if (i == 0 || i == R - 1 || j == 0 || j == C - 1) {
            v = A[at];
        } else {
            const CT c = to_ct<ST>(A[at]);
            const CT n = to_ct<ST>(A[at - ld]);
            const CT s = to_ct<ST>(A[at + ld]);
            const CT w = to_ct<ST>(A[at - 1]);
            const CT e = to_ct<ST>(A[at + 1]);
            v = from_ct<ST>(stencil_point(c, n, s, w, e));
        }
        B[at] = v;
    }
}

template <class ST>
static int launch_naive_t(const void *A, void *B, int R, int C, int ld, cudaStream_t s) {
    dim3 block(256);
    dim3 grid((C + 255) / 256, R < 65535 ? R : 65535);
    naive_step_kernel<ST><<<grid, block, 0, s>>>(static_cast<const ST *>(A), static_cast<ST *>(B), R, C, ld);
    SDFG_CUDA(cudaGetLastError());
    return SDFG_OK;
}

int launch_naive_step(const void *A, void *B, int R, int C, int ld, int dtype, cudaStream_t s) {
    TimedLaunch t = stats_begin(FAM_NAIVE, s);
    int rc;
    switch (dtype) {
        case SDFG_F32: rc = launch_naive_t<float>(A, B, R, C, ld, s); break;
        case SDFG_BF16: rc = launch_naive_t<__nv_bfloat16>(A, B, R, C, ld, s); break;
        default: rc = launch_naive_t<double>(A, B, R, C, ld, s); break;
    }
    stats_end(t, s);
    return rc;
}

// ------------------------------------------------------------- 2-D copy -----
int launch_copy2d(void *dst, int ldd, const void *src, int lds, int R, int C, int dtype, cudaStream_t s) {
    if (R <= 0 || C <= 0 || dst == src) return SDFG_OK;
    TimedLaunch t = stats_begin(FAM_COPY, s);
    const size_t S = dtype_bytes(dtype);
    cudaError_t e = cudaMemcpy2DAsync(dst, ldd * S, src, lds * S, C * S, R, cudaMemcpyDeviceToDevice, s);
    stats_end(t, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy2DAsync");
    return SDFG_OK;
}

// ------------------------------------------------------- temporal pass ------
// One launch = one pass of K fused timesteps over the whole grid; each warp
// owns one (strip, segment) unit, strips fastest so that neighbouring warps
// share halo columns through L2.
#ifndef SDFG_TP_MAXT
#define SDFG_TP_MAXT 128  // threads per CTA the temporal kernel is compiled for
#endif
#ifndef SDFG_TP_MINB
#define SDFG_TP_MINB 3    // CTAs per SM the register allocation must allow
#endif

template <class ST, int V, int K>
__global__ void __launch_bounds__(SDFG_TP_MAXT, SDFG_TP_MINB) temporal_pass_kernel(const __grid_constant__ CUtensorMap tm_src,
                                                            ST *__restrict__ dst, GridGeo g, int res_flags,
                                                            double2 *__restrict__ partials, int *err,
                                                            unsigned long long timeout_ns) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[MAX_WARPS][STAGES];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int unit = blockIdx.x * nw + warp;
    const int n_units = g.n_strips * g.n_segs;
    if (unit >= n_units) return;
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[warp][s], 1);
        mbar_init_fence();
        tmap_prefetch(&tm_src);
    }
    __syncwarp();
    ST *ring = reinterpret_cast<ST *>(smem_raw) + static_cast<size_t>(warp) * STAGES * CHUNK_ROWS * 32 * V;
    uint32_t ctr = 0;
    const int strip = unit % g.n_strips;
    const int seg = unit / g.n_strips;
    const bool ok = run_unit<ST, V, K>(&tm_src, dst, g, strip, seg, ring, bars[warp], ctr, res_flags,
                                       partials ? partials + unit : nullptr, timeout_ns);
    if (!ok && lane == 0) set_device_error(err, DEV_ERR_TIMEOUT_TMA);
}

size_t temporal_smem_bytes(int dtype, int warps) {
    const int S = dtype_bytes(dtype);
    return static_cast<size_t>(warps) * STAGES * CHUNK_ROWS * 32 * lane_cols(S) * S;
}

template <class ST, int K>
static const void *tp_fn() {
    return reinterpret_cast<const void *>(
        &temporal_pass_kernel<ST, Store<ST>::bytes == 8 ? 2 : (Store<ST>::bytes == 4 ? SDFG_F32_V : 4), K>);
}

static const void *temporal_fn(int dtype, int k) {
#define SDFG_TP_CASES(ST)                  \
    switch (k) {                           \
        case 1: return tp_fn<ST, 1>();     \
        case 2: return tp_fn<ST, 2>();     \
        case 4: return tp_fn<ST, 4>();     \
        case 8: return tp_fn<ST, 8>();     \
        default: return nullptr;           \
    }
    switch (dtype) {
        case SDFG_F32: SDFG_TP_CASES(float)
        case SDFG_BF16: SDFG_TP_CASES(__nv_bfloat16)
        case SDFG_F64: SDFG_TP_CASES(double)
    }
#undef SDFG_TP_CASES
    return nullptr;
}

static int prepare_fn(const void *fn, size_t smem) {
    // raise the dynamic shared memory limit once per kernel and size
    static std::mutex mu;
    static std::vector<std::pair<const void *, size_t>> done;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == fn && d.second >= smem) return SDFG_OK;
    SDFG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    done.emplace_back(fn, smem);
    return SDFG_OK;
}

int temporal_blocks_per_sm(int dtype, int k, int warps) {
    const void *fn = temporal_fn(dtype, k);
    if (!fn) return 0;
    const size_t smem = temporal_smem_bytes(dtype, warps);
    if (prepare_fn(fn, smem) != SDFG_OK) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, warps * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int launch_temporal_pass(const CUtensorMap *tm_src, void *dst, const GridGeo &g, int dtype, int k, int warps,
                         int res_flags, double2 *partials, int *err, unsigned long long timeout_ns,
                         cudaStream_t s) {
    const void *fn = temporal_fn(dtype, k);
    if (!fn) return set_error(SDFG_ERR_INVAL, "no temporal kernel for dtype %d, k=%d", dtype, k);
    if (warps < 1 || warps > MAX_WARPS || warps * 32 > SDFG_TP_MAXT)
        return set_error(SDFG_ERR_INVAL, "warps per CTA must be 1..%d", SDFG_TP_MAXT / 32);
    const size_t smem = temporal_smem_bytes(dtype, warps);
    int rc = prepare_fn(fn, smem);
    if (rc != SDFG_OK) return rc;
    const long long n_units = static_cast<long long>(g.n_strips) * g.n_segs;
    const unsigned blocks = static_cast<unsigned>((n_units + warps - 1) / warps);
    // argument block matching the kernel's parameter list
    CUtensorMap tm = *tm_src;
    GridGeo gg = g;
    void *dstp = dst;
    void *args[] = {&tm, &dstp, &gg, &res_flags, &partials, &err, &timeout_ns};
    TimedLaunch t = stats_begin(FAM_TEMPORAL, s);
    cudaError_t e = cudaLaunchKernel(fn, dim3(blocks), dim3(warps * 32), args, smem, s);
    stats_end(t, s);
    if (e != cudaSuccess) return cuda_error(e, "temporal pass launch");
    return SDFG_OK;
}

}  // namespace sdfg
