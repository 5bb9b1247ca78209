// Register-resident temporal pass of the 2-D Jacobi stencil (FP32 and BF16
// storage): one launch advances the grid by k <= 8 steps (StateFusion, paper
// App. B), each CTA holding its whole tile in registers for all k steps.
//
// The streamed temporal unit (temporal_unit.cuh) moves one warp down a
// (strip, segment) chunk by chunk, so a pass takes as long as one unit's
// chunks take to stream through the warp.  On a grid that fits in L2 -- the
// paper's 2048^2 workload -- that per-pass latency, not bandwidth, sets the
// speed.  Here a CTA of 16 warps loads its box with two TMA copies (half a
// box each, one mbarrier each: warps 0-7 start on the first half while the
// second lands), each warp takes a band of 17 consecutive box rows into
// registers, and all bands advance together, one barrier per step, so a pass
// costs one box load, k steps of arithmetic from registers and the stores,
// which the last step issues row by row as the rows become final.
// Consecutive passes overlap their launch with the previous pass's end.
//
// Geometry: the box is 272 rows x 128 columns; the tile it updates is the
// 256 x 112 interior of the box (8 halo rows and columns on each side).  A
// lane holds 4 columns.  Values that are wrong for want of a neighbour
// outside the box -- the rows above and below it read zeros, and the
// outermost lanes' shuffles wrap to their own values -- spread one row and
// one column per step, so after k <= 8 steps the halo has absorbed them.
// 2048^2 is exactly 8 x 19 = 152 tiles.
//
// Arithmetic: the exact order of the definition,
//   new = 0.2f * (c + ((n + s) + (w + e))),
// each operation rounded on its own (the FP64 oracle's order in FP32).  A
// row is updated in place: the (n + s) sum of the NEXT row is formed from
// this row's old values before they are overwritten, so no old copy of a
// row is kept.  Boundary-ring points keep their values; points outside the
// grid change but are never stored, and reach the interior only through the
// ring.  BF16 storage is converted to FP32 at the box load and rounded to
// BF16 (RNE) when the pass stores the tile.
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "launchset.h"
#include "runtime.h"

namespace sdfg {

constexpr int RS_THREADS = 512;                 // 16 warps
constexpr int RS_NW = RS_THREADS / 32;
constexpr int RS_RB = 17;                       // box rows per warp, in registers
constexpr int RS_BY = RS_NW * RS_RB;            // 272 box rows
constexpr int RS_HALO = 8;                      // halo rows and columns: up to 8 steps
constexpr int RS_TY = RS_BY - 2 * RS_HALO;      // 256 output rows per tile
constexpr int RS_W = 128;                       // box columns, 4 per lane
constexpr int RS_TX = RS_W - 2 * RS_HALO;       // 112 output columns per tile
constexpr int RS_BOX_ROWS = RS_BY / 2;          // rows per TMA copy (<= 256)

// Passes are launched as programmatic dependents of the previous pass: the
// next launch is scheduled as soon as every CTA of this one has started, and
// its prologue (barrier setup, descriptor prefetch) runs while this pass
// finishes; it reads the grid only after this pass has completed.
#ifndef SDFG_RESIDENT_PDL
#define SDFG_RESIDENT_PDL 1
#endif

struct ResGeo {
    int R, C, ld;
    int tiles_x, tiles_y;
};

template <int I, int N, class F> __device__ __forceinline__ void rs_static_for(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>());
        rs_static_for<I + 1, N>(f);
    }
}

// w + e for the lane's 4 columns; west of column 0 and east of column 3 come
// from the neighbouring lanes.
__device__ __forceinline__ void rs_west_east(float (&we)[4], const float (&c)[4]) {
    const float left = __shfl_up_sync(FULL_MASK, c[3], 1);
    const float right = __shfl_down_sync(FULL_MASK, c[0], 1);
    we[0] = __fadd_rn(left, c[1]);
    we[1] = __fadd_rn(c[0], c[2]);
    we[2] = __fadd_rn(c[1], c[3]);
    we[3] = __fadd_rn(c[2], right);
}

// Launch parameters of one pass: read through tm, write dst, fuse k steps.
struct ResParams {
    CUtensorMap tm;
    void *dst;
    ResGeo g;
    int k;
    int *err;
    unsigned long long timeout_ns;
};

template <class ST>
__global__ void __launch_bounds__(RS_THREADS, 1) resident_pass_kernel(const __grid_constant__ ResParams P) {
    constexpr int V = 4;
    constexpr uint32_t BOX_BYTES = RS_BY * RS_W * sizeof(ST);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];  // one per TMA copy (half box)
    // band-edge rows, double-buffered by step parity: top[p][w] is warp w's
    // first row, bot[p][w + 1] its last; bot[p][0] and top[p][NW] stand for
    // the rows beyond the box (zeros)
    __shared__ __align__(16) float top[2][RS_NW + 1][RS_W];
    __shared__ __align__(16) float bot[2][RS_NW + 1][RS_W];
    ST *box = reinterpret_cast<ST *>(smem_raw);

    const ResGeo g = P.g;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int tx = blockIdx.x % g.tiles_x;
    const int ty = blockIdx.x / g.tiles_x;
    const int x0 = tx * RS_TX;                // first output column
    const int y0 = ty * RS_TY;                // first output row
    // box row r <-> grid row y0 - HALO + r; box column q <-> grid column x0 - HALO + q
    const int gx = x0 - RS_HALO + lane * V;   // grid column of this lane's element 0
    const int yb = y0 - RS_HALO + warp * RS_RB;  // grid row of the band's first row

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
        tmap_prefetch(&P.tm);
    }
    if (warp == 0) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4 *>(bot[0][0])[lane] = z;
        reinterpret_cast<float4 *>(bot[1][0])[lane] = z;
        reinterpret_cast<float4 *>(top[0][RS_NW])[lane] = z;
        reinterpret_cast<float4 *>(top[1][RS_NW])[lane] = z;
    }
#if SDFG_RESIDENT_PDL
    // the next pass may launch now; this one reads the previous pass's output
    // only after that pass has completed and its writes are visible
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif

    // The points this warp must keep fixed.  Only the boundary ring matters:
    // points outside the grid (zero-filled rows and columns of the box) may
    // change freely, since they reach the interior only through the ring,
    // which never changes.  A band holds at most one ring row (row 0 or R-1)
    // and a lane at most one ring column (0 or C-1) unless the grid is only
    // a few rows or one box wide; then the band takes the general path, which
    // keeps every point outside the interior.
    const int bx0 = x0 - RS_HALO;  // grid column of box column 0
    int ncol = 0, fq = -1;         // fq: box column of the ring column in the box
    if (bx0 <= 0) {
        ++ncol;
        fq = -bx0;
    }
    if (g.C - 1 - bx0 < RS_W) {
        ++ncol;
        fq = g.C - 1 - bx0;
    }
    int nrow = 0, frow = -1;  // frow: band row of the ring row in the band
    if (yb <= 0 && 0 < yb + RS_RB) {
        ++nrow;
        frow = -yb;
    }
    if (g.R - 1 >= yb && g.R - 1 < yb + RS_RB) {
        ++nrow;
        frow = g.R - 1 - yb;
    }
    // variant: 0 plain; 1..4 ring column at element variant-1 of lane fq/V;
    // +5 with a ring row; 10 general.  u0, u1: the ring row's band row and
    // whether this lane holds the ring column; on the general path the
    // band's first grid row and this lane's interior-column mask.
    const int variant =
        (ncol > 1 || nrow > 1) ? 10 : (ncol == 1 ? fq % V + 1 : 0) + (nrow == 1 ? 5 : 0);
    int u0 = frow;
    unsigned u1 = ncol == 1 && lane == fq / V ? 1u : 0u;
    if (variant == 10) {
        u0 = yb;
        u1 = 0;
#pragma unroll
        for (int e = 0; e < V; ++e)
            if (gx + e >= 1 && gx + e <= g.C - 2) u1 |= 1u << e;
    }

    float X[RS_RB][V];
    // Stores: band rows [st_lo, st_hi) lie in the tile and the grid; lanes
    // whose columns lie in the tile (and the grid) store them, with one
    // vector store when all V columns are in the grid.
    ST *const row0 = static_cast<ST *>(P.dst) + static_cast<long long>(yb) * g.ld + gx;
    const int st_lo = max(0, RS_HALO - warp * RS_RB);
    const int st_hi = min(min(RS_RB, RS_HALO + RS_TY - warp * RS_RB), g.R - yb);
    const bool own_cols = lane * V >= RS_HALO && lane * V < RS_HALO + RS_TX && gx < g.C;
    const bool full_vec = gx + V <= g.C;
    auto put = [&](float *slot, const float (&x)[V]) {
        reinterpret_cast<float4 *>(slot)[lane] = make_float4(x[0], x[1], x[2], x[3]);
    };
    auto get = [&](float (&x)[V], const float *slot) {
        const float4 v = reinterpret_cast<const float4 *>(slot)[lane];
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    };
    // One step of the band from the edge rows of slot p; the new edge rows go
    // to slot p ^ 1.  CF: 0 no ring column, 1 + e ring column at element e
    // of the lanes with u1 set, -1 the general path; RF: a ring row at band
    // row u0.  LAST: the pass's last step, which stores the rows.
    auto step = [&](auto cf_t, auto rf_t, auto last_t, int p) {
        constexpr int CF = decltype(cf_t)::value;
        constexpr bool RF = decltype(rf_t)::value;
        constexpr bool LAST = decltype(last_t)::value;
        float N[V], S[V];
        get(N, bot[p][warp]);
        get(S, top[p][warp + 1]);
        float ns[V];  // n + s of the row being updated, from old values
#pragma unroll
        for (int e = 0; e < V; e += 2) {
            const float2 t = __fadd2_rn(make_float2(N[e], N[e + 1]), make_float2(X[1][e], X[1][e + 1]));
            ns[e] = t.x;
            ns[e + 1] = t.y;
        }
        rs_static_for<0, RS_RB>([&](auto i_t) {
            constexpr int i = decltype(i_t)::value;
            float we[V];
            rs_west_east(we, X[i]);
            // the next row's n + s (n = this row's old values) before this
            // row is overwritten
            float ns_next[V];
            if constexpr (i + 1 < RS_RB) {
                const float(&s2)[V] = (i + 2 < RS_RB) ? X[i + 2 < RS_RB ? i + 2 : 0] : S;
#pragma unroll
                for (int e = 0; e < V; e += 2) {
                    const float2 t = __fadd2_rn(make_float2(X[i][e], X[i][e + 1]), make_float2(s2[e], s2[e + 1]));
                    ns_next[e] = t.x;
                    ns_next[e + 1] = t.y;
                }
            }
            float o[V];
#pragma unroll
            for (int e = 0; e < V; e += 2) {
                const float2 t = __fadd2_rn(make_float2(ns[e], ns[e + 1]), make_float2(we[e], we[e + 1]));
                const float2 u = __fadd2_rn(make_float2(X[i][e], X[i][e + 1]), t);
                const float2 r = __fmul2_rn(make_float2(0.2f, 0.2f), u);
                o[e] = r.x;
                o[e + 1] = r.y;
            }
            if constexpr (CF < 0) {
                const bool row_in = u0 + i >= 1 && u0 + i <= g.R - 2;
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (!row_in || !((u1 >> e) & 1u)) o[e] = X[i][e];
            } else {
                if constexpr (CF > 0) {
                    if (u1) o[CF - 1] = X[i][CF - 1];
                }
                if constexpr (RF) {
                    if (i == u0) {
#pragma unroll
                        for (int e = 0; e < V; ++e) o[e] = X[i][e];
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < V; ++e) X[i][e] = o[e];
            if constexpr (LAST) {
                // the row is final: store it while the next rows compute
                if (own_cols && i >= st_lo && i < st_hi) {
                    ST *q = row0 + static_cast<long long>(i) * g.ld;
                    if (full_vec) {
                        VecIO<ST, V>::store(q, X[i]);
                    } else {
#pragma unroll
                        for (int e = 0; e < V; ++e)
                            if (gx + e < g.C) q[e] = static_cast<ST>(X[i][e]);
                    }
                }
            }
            if constexpr (i + 1 < RS_RB) {
#pragma unroll
                for (int e = 0; e < V; ++e) ns[e] = ns_next[e];
            }
        });
        if constexpr (!LAST) {
            put(top[p ^ 1][warp], X[0]);
            put(bot[p ^ 1][warp + 1], X[RS_RB - 1]);
        }
    };
    // all k steps of one variant (the loop is repeated per variant, so that
    // only that variant's values stay live across it)
    // the last step stores each row of the tile as soon as it is final
    auto steps = [&](auto cf_t, auto rf_t, int nk) {
        for (int t = 0; t < nk - 1; ++t) {
            step(cf_t, rf_t, std::false_type(), t & 1);
            __syncthreads();
        }
        step(cf_t, rf_t, std::true_type(), (nk - 1) & 1);
    };
    const int k = P.k;
    __syncthreads();
    if (tid == 0) {
        // two half boxes of 136 rows: warps 0-7 own the first, 8-15 the second
        mbar_arrive_expect_tx(&bar[0], BOX_BYTES / 2);
        tma_load_3d(box, &P.tm, x0 - RS_HALO, y0 - RS_HALO, 0, &bar[0]);
        mbar_arrive_expect_tx(&bar[1], BOX_BYTES / 2);
        tma_load_3d(box + RS_BOX_ROWS * RS_W, &P.tm, x0 - RS_HALO, y0 - RS_HALO + RS_BOX_ROWS, 0, &bar[1]);
    }
    static_assert(RS_BOX_ROWS == (RS_NW / 2) * RS_RB, "each half box holds the bands of half the warps");
    const bool ok = mbar_wait_bounded(&bar[warp < RS_NW / 2 ? 0 : 1], 0, P.timeout_ns);
    // (a warp whose wait ran out reads stale shared memory here; the check
    // below then ends the CTA before any value is used)
    rs_static_for<0, RS_RB>([&](auto i_t) {
        constexpr int i = decltype(i_t)::value;
        VecIO<ST, V>::load(X[i], box + (warp * RS_RB + i) * RS_W + lane * V);
    });
    put(top[0][warp], X[0]);
    put(bot[0][warp + 1], X[RS_RB - 1]);
    if (!__syncthreads_and(ok)) {
        // give the copies a bounded chance to land before leaving, then report
        mbar_wait_bounded(&bar[0], 0, 1000000ull);
        mbar_wait_bounded(&bar[1], 0, 1000000ull);
        if (tid == 0) set_device_error(P.err, DEV_ERR_TIMEOUT_TMA);
        return;
    }

    using F = std::false_type;
    using T = std::true_type;
    switch (variant) {
        case 0: steps(std::integral_constant<int, 0>(), F(), k); break;
        case 1: steps(std::integral_constant<int, 1>(), F(), k); break;
        case 2: steps(std::integral_constant<int, 2>(), F(), k); break;
        case 3: steps(std::integral_constant<int, 3>(), F(), k); break;
        case 4: steps(std::integral_constant<int, 4>(), F(), k); break;
        case 5: steps(std::integral_constant<int, 0>(), T(), k); break;
        case 6: steps(std::integral_constant<int, 1>(), T(), k); break;
        case 7: steps(std::integral_constant<int, 2>(), T(), k); break;
        case 8: steps(std::integral_constant<int, 3>(), T(), k); break;
        case 9: steps(std::integral_constant<int, 4>(), T(), k); break;
        default: steps(std::integral_constant<int, -1>(), F(), k); break;
    }

}

// ------------------------------------------------------------------ host -----
static const void *resident_fn(int dtype) {
    return dtype == SDFG_BF16 ? reinterpret_cast<const void *>(&resident_pass_kernel<__nv_bfloat16>)
                              : reinterpret_cast<const void *>(&resident_pass_kernel<float>);
}

bool resident_supported(int dtype) { return dtype == SDFG_F32 || dtype == SDFG_BF16; }

std::vector<int> plan_resident_passes(long long T, int k) {
    std::vector<int> p;
    if (T <= 0 || k < 1) return p;
    p.assign(static_cast<size_t>(T / k), k);
    if (T % k) p.push_back(static_cast<int>(T % k));
    return p;
}

// Runs the passes ks (each k <= 8) from src0, one launch per pass: the first
// pass writes `first`, then the passes alternate between `second` and
// `first`; *final receives the buffer the last pass wrote.
int run_resident_passes(const void *src0, void *first, void *second, const std::vector<int> &ks, int R, int C,
                        int ld, int dtype, DeviceState *st, cudaStream_t s, void **final) {
    *final = const_cast<void *>(src0);
    if (ks.empty()) return SDFG_OK;
    if (!resident_supported(dtype)) return set_error(SDFG_ERR_INVAL, "resident kernel: FP32 or BF16 storage only");
    for (int k : ks)
        if (k < 1 || k > RS_HALO) return set_error(SDFG_ERR_INVAL, "resident kernel: k=%d outside 1..%d", k, RS_HALO);
    const void *fn = resident_fn(dtype);
    const size_t smem = static_cast<size_t>(RS_BY) * RS_W * dtype_bytes(dtype);
    static bool attr_done[2] = {false, false};
    const int slot = dtype == SDFG_BF16 ? 1 : 0;
    if (!attr_done[slot]) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return cuda_error(e, "resident attribute");
        attr_done[slot] = true;
    }
    alignas(128) CUtensorMap tm_src0, tm_first, tm_second;
    int rc = encode_tmap3d(&tm_src0, src0, dtype, 1, R, C, ld, RS_W, RS_BOX_ROWS);
    if (rc == SDFG_OK) rc = encode_tmap3d(&tm_first, first, dtype, 1, R, C, ld, RS_W, RS_BOX_ROWS);
    if (rc == SDFG_OK) rc = encode_tmap3d(&tm_second, second, dtype, 1, R, C, ld, RS_W, RS_BOX_ROWS);
    if (rc != SDFG_OK) return rc;
    ResParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.g.R = R;
    prm.g.C = C;
    prm.g.ld = ld;
    prm.g.tiles_x = (C + RS_TX - 1) / RS_TX;
    prm.g.tiles_y = (R + RS_TY - 1) / RS_TY;
    prm.err = st->d_err;
    prm.timeout_ns = test_hooks().timeout_ns ? test_hooks().timeout_ns : DEFAULT_TIMEOUT_NS;
    const unsigned blocks = static_cast<unsigned>(static_cast<long long>(prm.g.tiles_x) * prm.g.tiles_y);
    const CUtensorMap *tsrc = &tm_src0;
    void *dst = first;
    for (size_t p = 0; p < ks.size(); ++p) {
        prm.tm = *tsrc;
        prm.dst = dst;
        prm.k = ks[p];
        void *args[] = {&prm};
        TimedLaunch tl = stats_begin(FAM_RESIDENT, s);
#if SDFG_RESIDENT_PDL
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(blocks);
        lc.blockDim = dim3(RS_THREADS);
        lc.dynamicSmemBytes = smem;
        lc.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelExC(&lc, fn, args);
#else
        const cudaError_t e = cudaLaunchKernel(fn, dim3(blocks), dim3(RS_THREADS), args, smem, s);
#endif
        stats_end(tl, s);
        if (e != cudaSuccess) return cuda_error(e, "resident launch");
        *final = dst;
        tsrc = (dst == first) ? &tm_first : &tm_second;
        dst = (dst == first) ? second : first;
    }
    return SDFG_OK;
}

}  // namespace sdfg
