// The Jacobi method one dimension up: a 7-point stencil on a D x R x C box
// with a fixed one-cell shell, iterated T times between two copies of the box
// (paper Sec. 6.1's Jacobi benchmark, Fig. 1's ping-pong state loop).  Each
// interior point becomes
//   (1/7) * (c + (((n + s) + (w + e)) + (u + d)))
// (n, s: rows i-1, i+1; w, e: columns j-1, j+1; u, d: planes z-1, z+1), in
// this order, round to nearest, no contraction, in the compute type (FP32 for
// FP32 and BF16 storage, FP64 for FP64): an FP64 run equals the FP64
// definition bit for bit.
//
// One launch is one timestep.  A CTA owns a tile of TY rows x TX columns and
// streams through a range of planes (2.5-D blocking, paper App. B MapTiling
// applied to rows and columns, the plane loop kept sequential): plane after
// plane arrives by 3-D TMA -- the tile plus a one-row and a 16-byte column
// halo -- into a ring of NS shared-memory stages, fetched NS-1 planes ahead
// (DoubleBuffering).  A warp owns two rows of the tile; a lane owns V
// consecutive columns and keeps their values of the planes above and below
// in registers; north and south neighbours come from shared memory, west and
// east ones from the neighbouring lanes by shuffle.  Every point of the tile
// is stored: interior points computed, shell points copied, so every output
// box is complete.
#include <algorithm>

#include "device_common.cuh"
#include "runtime.h"

namespace sdfg {

constexpr int J3_TY = 16;               // output rows per tile
constexpr int J3_BY = J3_TY + 2;        // rows per TMA box (one-row halo each side)
constexpr int J3_NS = 4;                // ring stages (planes)
constexpr int J3_THREADS = 256;         // 8 warps, two tile rows each
constexpr int J3_MIN_ZSEG = 32;         // planes per CTA at least

struct J3Geo {
    int D, R, C, ld;
    long long plane;        // plane pitch (elements) = R * ld
    int tiles_x, tiles_y;   // tiles per plane
    int zseg, n_zseg;       // planes per CTA, CTAs along z
};

template <class ST>
__device__ __forceinline__ typename Store<ST>::CT one_seventh();
template <> __device__ __forceinline__ float one_seventh<float>() { return static_cast<float>(1.0 / 7.0); }
template <> __device__ __forceinline__ float one_seventh<__nv_bfloat16>() { return static_cast<float>(1.0 / 7.0); }
template <> __device__ __forceinline__ double one_seventh<double>() { return 1.0 / 7.0; }

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// The one-point update in the library's fixed order.
template <class CT>
__device__ __forceinline__ CT point7(CT c, CT n, CT s, CT w, CT e, CT u, CT d, CT k) {
    return mul_rn(k, add_rn(c, add_rn(add_rn(add_rn(n, s), add_rn(w, e)), add_rn(u, d))));
}

template <class ST, int V>
__global__ void __launch_bounds__(J3_THREADS) jacobi3d_kernel(const __grid_constant__ CUtensorMap tm,
                                                              ST *__restrict__ dst, const J3Geo g, int *err,
                                                              unsigned long long timeout_ns) {
    using CT = typename Store<ST>::CT;
    constexpr int W = 32 * V;                 // box columns
    constexpr int XH = Store<ST>::xalign;     // column halo: 16 bytes, so the box start stays TMA-aligned
    constexpr int TX = W - 2 * XH;            // output columns per tile
    constexpr uint32_t PLANE_BYTES = J3_BY * W * sizeof(ST);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[J3_NS];
    ST *ring = reinterpret_cast<ST *>(smem_raw);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    int b = blockIdx.x;
    const int tx = b % g.tiles_x;
    b /= g.tiles_x;
    const int ty = b % g.tiles_y;
    const int zs = b / g.tiles_y;
    const int x0 = tx * TX;                   // first output column
    const int y0 = ty * J3_TY;                // first output row
    const int z0 = zs * g.zseg;
    const int z1 = min(z0 + g.zseg, g.D);
    const int n_planes = z1 - z0 + 2;         // input planes z0-1 .. z1

    if (tid == 0) {
        for (int s = 0; s < J3_NS; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
        tmap_prefetch(&tm);
    }
    __syncthreads();
    // input plane m (global plane z0-1+m) -> stage m % NS; planes outside
    // the box, rows and columns outside it arrive zero-filled
    auto issue = [&](int m) {
        const int st = m % J3_NS;
        mbar_arrive_expect_tx(&bars[st], PLANE_BYTES);
        tma_load_3d(ring + st * (J3_BY * W), &tm, x0 - XH, y0 - 1, z0 - 1 + m, &bars[st]);
    };
    int issued = min(J3_NS, n_planes);
    if (tid == 0)
        for (int m = 0; m < issued; ++m) issue(m);
    // wait (every thread) for plane m; block-uniform outcome
    auto wait_plane = [&](int m) -> bool {
        const bool ok = mbar_wait_bounded(&bars[m % J3_NS], (m / J3_NS) & 1u, timeout_ns);
        return __syncthreads_and(ok) != 0;
    };
    // the wait for plane m_first ran out: give it and the copies after it a
    // bounded chance to land before the CTA leaves, then report
    auto fail = [&](int m_first) {
        for (int m = m_first; m < issued; ++m) mbar_wait_bounded(&bars[m % J3_NS], (m / J3_NS) & 1u, 1000000ull);
        if (tid == 0) set_device_error(err, DEV_ERR_TIMEOUT_TMA);
    };

    // this thread's points: rows r_i = 1 + warp + 8 i of the box, columns
    // lane*V .. lane*V+V-1 of the box
    const int gx = x0 - XH + lane * V;        // global column of element 0
    const bool own_cols = lane * V >= XH && lane * V < XH + TX && gx < g.C;
    const bool full_vec = gx + V <= g.C;
    CT u[2][V], c[2][V], d[2][V];

    if (!wait_plane(0)) return fail(0);
    if (!wait_plane(1)) return fail(1);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int r = 1 + warp + 8 * i;
        const ST *p0 = ring + (0 % J3_NS) * (J3_BY * W) + r * W + lane * V;
        const ST *p1 = ring + (1 % J3_NS) * (J3_BY * W) + r * W + lane * V;
        CT a[V], bb[V];
        VecIO<ST, V>::load(a, p0);
        VecIO<ST, V>::load(bb, p1);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            u[i][e] = a[e];
            c[i][e] = bb[e];
        }
    }
    // plane 0's stage is free once every thread has its values
    __syncthreads();
    if (tid == 0 && issued < n_planes) issue(issued);
    if (issued < n_planes) ++issued;

    const CT K7 = one_seventh<ST>();
    for (int j = 0; j + 2 < n_planes; ++j) {
        const int z = z0 + j;                 // output plane
        if (!wait_plane(j + 2)) return fail(j + 2);
        const ST *pc = ring + ((j + 1) % J3_NS) * (J3_BY * W);   // plane z
        const ST *pd = ring + ((j + 2) % J3_NS) * (J3_BY * W);   // plane z+1
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = 1 + warp + 8 * i;
            const int y = y0 + r - 1;         // output row
            CT n[V], s[V], dd[V];
            VecIO<ST, V>::load(n, pc + (r - 1) * W + lane * V);
            VecIO<ST, V>::load(s, pc + (r + 1) * W + lane * V);
            VecIO<ST, V>::load(dd, pd + r * W + lane * V);
#pragma unroll
            for (int e = 0; e < V; ++e) d[i][e] = dd[e];
            // west of element 0 and east of element V-1 from the neighbouring
            // lanes (lanes 0 and 31 get stale values: their columns are halo)
            const CT left = __shfl_up_sync(FULL_MASK, c[i][V - 1], 1);
            const CT right = __shfl_down_sync(FULL_MASK, c[i][0], 1);
            CT o[V];
            const bool shell_row = z == 0 || z == g.D - 1 || y == 0 || y == g.R - 1;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const CT w = e == 0 ? left : c[i][e - 1];
                const CT ea = e == V - 1 ? right : c[i][e + 1];
                const int x = gx + e;
                const CT v = point7(c[i][e], n[e], s[e], w, ea, u[i][e], d[i][e], K7);
                o[e] = (shell_row || x == 0 || x == g.C - 1) ? c[i][e] : v;
            }
            if (own_cols && y < g.R) {
                ST *q = dst + static_cast<long long>(z) * g.plane + static_cast<long long>(y) * g.ld + gx;
                if (full_vec) {
                    store_pred(q, o, 1);
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (gx + e < g.C) q[e] = from_ct<ST>(o[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < V; ++e) {
                u[i][e] = c[i][e];
                c[i][e] = d[i][e];
            }
        }
        // every thread is done with plane z's stage: refill it
        __syncthreads();
        if (issued < n_planes) {
            if (tid == 0) issue(issued);
            ++issued;
        }
    }
}

// ------------------------------------------------------------------ host -----
template <class ST, int V>
static const void *j3_fn() {
    return reinterpret_cast<const void *>(&jacobi3d_kernel<ST, V>);
}

static const void *j3_kernel(int dtype) {
    switch (dtype) {
        case SDFG_F32: return j3_fn<float, 4>();
        case SDFG_BF16: return j3_fn<__nv_bfloat16, 4>();
        default: return j3_fn<double, 2>();
    }
}

static int j3_box_cols(int dtype) { return dtype == SDFG_F64 ? 64 : 128; }
static int j3_tile_cols(int dtype) { return j3_box_cols(dtype) - 2 * (16 / dtype_bytes(dtype)); }
static size_t j3_smem(int dtype) { return static_cast<size_t>(J3_NS) * J3_BY * j3_box_cols(dtype) * dtype_bytes(dtype); }

static int launch_j3(const CUtensorMap &tm, void *dst, const J3Geo &g, int dtype, int *err, cudaStream_t s) {
    const void *fn = j3_kernel(dtype);
    const size_t smem = j3_smem(dtype);
    static bool attr_done[3] = {false, false, false};
    if (!attr_done[dtype]) {
        SDFG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        attr_done[dtype] = true;
    }
    CUtensorMap t = tm;
    J3Geo gg = g;
    void *dp = dst;
    unsigned long long to = DEFAULT_TIMEOUT_NS;
    void *args[] = {&t, &dp, &gg, &err, &to};
    const unsigned blocks = static_cast<unsigned>(static_cast<long long>(g.tiles_x) * g.tiles_y * g.n_zseg);
    TimedLaunch tl = stats_begin(FAM_STENCIL3D, s);
    cudaError_t e = cudaLaunchKernel(fn, dim3(blocks), dim3(J3_THREADS), args, smem, s);
    stats_end(tl, s);
    if (e != cudaSuccess) return cuda_error(e, "jacobi3d launch");
    return SDFG_OK;
}

static J3Geo plan_j3(int D, int R, int C, int ld, int dtype, int sm_count) {
    J3Geo g;
    g.D = D;
    g.R = R;
    g.C = C;
    g.ld = ld;
    g.plane = static_cast<long long>(R) * ld;
    const int TX = j3_tile_cols(dtype);
    g.tiles_x = (C + TX - 1) / TX;
    g.tiles_y = (R + J3_TY - 1) / J3_TY;
    // about 16 CTAs per SM in total, at least J3_MIN_ZSEG planes each
    const long long tiles = static_cast<long long>(g.tiles_x) * g.tiles_y;
    const long long target = 16LL * std::max(sm_count, 1);
    long long nz = std::max<long long>(1, (target + tiles - 1) / tiles);
    long long zseg = std::max<long long>(J3_MIN_ZSEG, (D + nz - 1) / nz);
    g.zseg = static_cast<int>(std::min<long long>(zseg, std::max(D, 1)));
    g.n_zseg = (D + g.zseg - 1) / g.zseg;
    return g;
}

static bool j3_tma_ok(const void *p, int ld, int dtype) {
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((static_cast<long long>(ld) * dtype_bytes(dtype)) % 16 == 0);
}

}  // namespace sdfg

using namespace sdfg;

extern "C" int sdfg_jacobi3d(const void *in, void *out, int depth, int rows, int cols, int ld, int T, int dtype,
                             void *stream) {
    if (depth < 0 || rows < 0 || cols < 0 || T < 0 || !dtype_valid(dtype))
        return set_error(SDFG_ERR_INVAL, "sdfg_jacobi3d: bad extents, T or dtype (%d x %d x %d, T=%d, dtype %d)", depth,
                         rows, cols, T, dtype);
    if (ld < cols) return set_error(SDFG_ERR_INVAL, "sdfg_jacobi3d: ld %d < cols %d", ld, cols);
    const long long n_rows = static_cast<long long>(depth) * rows;
    if (n_rows == 0 || cols == 0) return SDFG_OK;
    if (!in || !out) return set_error(SDFG_ERR_INVAL, "sdfg_jacobi3d: null box");
    if (n_rows > (1LL << 31) - 1) return set_error(SDFG_ERR_INVAL, "sdfg_jacobi3d: box too large");
    DeviceState *st = nullptr;
    int rc = current_device(&st);
    if (rc != SDFG_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nr = static_cast<int>(n_rows);
    if (T == 0 || depth < 3 || rows < 3 || cols < 3) {
        if (in == out) return SDFG_OK;
        return launch_copy2d(out, ld, in, ld, nr, cols, dtype, s);
    }
    const size_t S = dtype_bytes(dtype);
    // ping-pong between two aligned boxes; unaligned or pitched-oddly
    // callers are staged through an aligned copy
    const bool aligned = j3_tma_ok(in, ld, dtype) && j3_tma_ok(out, ld, dtype);
    const int ldw = aligned ? ld : (cols + 31) / 32 * 32;
    const size_t bytes = static_cast<size_t>(n_rows) * ldw * S;
    void *a = nullptr, *b = nullptr;
    const void *src0 = in;
    void *first = nullptr, *second = nullptr;
    if (aligned) {
        rc = scratch_alloc(&a, bytes, s);
        if (rc != SDFG_OK) return rc;
        if (in != out) {
            // the last of T passes must land in `out`
            first = (T % 2 == 1) ? out : a;
            second = first == out ? a : out;
        } else {
            first = a;
            second = out;
        }
    } else {
        rc = scratch_alloc(&a, bytes, s);
        if (rc == SDFG_OK) rc = scratch_alloc(&b, bytes, s);
        if (rc == SDFG_OK) rc = launch_copy2d(a, ldw, in, ld, nr, cols, dtype, s);
        if (rc != SDFG_OK) {
            scratch_free(a, s);
            scratch_free(b, s);
            return rc;
        }
        src0 = a;
        first = b;
        second = a;
    }
    const int box_cols = j3_box_cols(dtype);
    alignas(128) CUtensorMap tm_src0, tm_first, tm_second;
    rc = encode_tmap3d(&tm_src0, src0, dtype, depth, rows, cols, ldw, box_cols, J3_BY);
    if (rc == SDFG_OK) rc = encode_tmap3d(&tm_first, first, dtype, depth, rows, cols, ldw, box_cols, J3_BY);
    if (rc == SDFG_OK) rc = encode_tmap3d(&tm_second, second, dtype, depth, rows, cols, ldw, box_cols, J3_BY);
    const J3Geo g = plan_j3(depth, rows, cols, ldw, dtype, st->sm_count);
    const CUtensorMap *tsrc = &tm_src0;
    void *dst = first;
    void *fin = const_cast<void *>(src0);
    for (int t = 0; t < T && rc == SDFG_OK; ++t) {
        rc = launch_j3(*tsrc, dst, g, dtype, st->d_err, s);
        fin = dst;
        tsrc = dst == first ? &tm_first : &tm_second;
        dst = dst == first ? second : first;
    }
    if (rc == SDFG_OK && fin != out) rc = launch_copy2d(out, ld, fin, ldw, nr, cols, dtype, s);
    scratch_free(a, s);
    scratch_free(b, s);
    return rc;
}
