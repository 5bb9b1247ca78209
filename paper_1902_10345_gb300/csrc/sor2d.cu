// Red-black successive over-relaxation of the 2-D 5-point Laplace problem:
// the in-place, ordered counterpart of the Jacobi stencil (paper Sec. 6.1's
// stencil on a 2-D domain with constant boundary).  One iteration updates
// every interior point with i + j even ("red"), then every one with i + j odd
// ("black"), each as
//   c <- (1 - omega) * c + (omega / 4) * ((n + s) + (w + e))
// in that order, round to nearest, no contraction, in FP32 (FP32 and BF16
// storage) or FP64 (bit-identical to a plain FP64 loop).  A point of one
// colour reads only points of the other colour, so each half-sweep is one
// map of independent instances (the paper's Map scope).
//
// One launch runs up to KI iterations (2 KI half-sweeps; StateFusion, paper
// App. B).  A CTA owns a tile of TY rows x TX columns and loads it by 2-D TMA
// with a halo of 2 KI rows and at least 2 KI columns on each side into shared
// memory.  Half-sweep h updates, in place, the points of its colour: they
// read only points of the other colour, none of which change during the
// half-sweep.  Values that are wrong for want of a neighbour outside the box
// spread one row and one column per half-sweep, so after 2 KI half-sweeps the
// halo has absorbed them.  A barrier separates the half-sweeps.  The tile is
// then written to the other buffer of a ping-pong pair, so that no CTA reads
// a value another CTA has already advanced.  The result equals the in-place
// sweeps.  Boundary-ring points are copied; every point of the grid is
// written by exactly one CTA.
//
// Two kernels.  FP64 storage (2 columns per lane) sweeps the box in shared
// memory, on box rows [1 + h, BY - 1 - h) in half-sweep h.  FP32 and BF16
// storage (4 columns per lane) load the box once into registers -- each warp
// holds a band of SOR_RB consecutive rows for the whole launch -- and pass
// only the bands' first and last rows through shared memory between
// half-sweeps.
#include <algorithm>
#include <type_traits>
#include <math.h>

#include "device_common.cuh"
#include "runtime.h"

namespace sdfg {

#ifndef SDFG_SOR_TY
#define SDFG_SOR_TY 60
#endif
constexpr int SOR_TY = SDFG_SOR_TY;     // output rows per tile
constexpr int SOR_THREADS = 256;        // 8 warps

// Iterations per launch: 4 for FP32 and BF16 storage (a 16-byte column halo
// of 8 elements or more), 2 for FP64 (a 32-byte halo of 4 doubles).
// Rows per warp held in registers by the FP32/BF16 kernel, and iterations
// per launch of that kernel.
#ifndef SDFG_SOR_RB
#define SDFG_SOR_RB 10
#endif
constexpr int SOR_RB = SDFG_SOR_RB;
#ifndef SDFG_SOR_KI
#define SDFG_SOR_KI 4
#endif

template <class ST> struct SorShape {
    static constexpr int KI = sizeof(ST) == 8 ? 2 : SDFG_SOR_KI;
    static constexpr int HR = 2 * KI;                         // halo rows (and least halo columns)
    static constexpr int V = sizeof(ST) == 8 ? 2 : 4;         // columns per lane
    static constexpr int XA = Store<ST>::xalign;              // TMA x alignment (elements)
    static constexpr int XH = (HR + XA - 1) / XA * XA;        // halo columns
    static constexpr int W = 32 * V;                          // box columns
    static constexpr int TX = W - 2 * XH;                     // output columns per tile
    // output rows: FP32/BF16 fill the 8 warps' register bands exactly
    static constexpr int TY = sizeof(ST) == 8 ? SOR_TY : (SOR_THREADS / 32) * SOR_RB - 2 * HR;
    static constexpr int BY = TY + 2 * HR;                    // box rows (<= 256: one TMA box)
};

struct SorGeo {
    int R, C, ld;
    int tiles_x;
};

__device__ __forceinline__ float sor_point(float c, float n, float s, float w, float e, float a, float b) {
    return __fadd_rn(__fmul_rn(a, c), __fmul_rn(b, __fadd_rn(__fadd_rn(n, s), __fadd_rn(w, e))));
}
__device__ __forceinline__ double sor_point(double c, double n, double s, double w, double e, double a, double b) {
    return __dadd_rn(__dmul_rn(a, c), __dmul_rn(b, __dadd_rn(__dadd_rn(n, s), __dadd_rn(w, e))));
}

template <class ST>
__global__ void __launch_bounds__(SOR_THREADS) sor2d_kernel(const __grid_constant__ CUtensorMap tm,
                                                            ST *__restrict__ dst, const SorGeo g,
                                                            typename Store<ST>::CT a, typename Store<ST>::CT b,
                                                            int n_half, int *err, unsigned long long timeout_ns) {
    using CT = typename Store<ST>::CT;
    using SH = SorShape<ST>;
    constexpr int V = SH::V;
    constexpr int W = SH::W;
    constexpr int XH = SH::XH;
    constexpr int TX = SH::TX;
    constexpr int HR = SH::HR;
    constexpr int SOR_BY = SH::BY;
    constexpr uint32_t BOX_BYTES = SOR_BY * W * sizeof(ST);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    ST *box = reinterpret_cast<ST *>(smem_raw);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int tx = blockIdx.x % g.tiles_x;
    const int ty = blockIdx.x / g.tiles_x;
    const int x0 = tx * TX;                   // first output column
    const int y0 = ty * SH::TY;               // first output row
    // box row r <-> grid row y0 - HR + r; box column k <-> grid column x0 - XH + k
    const int gx = x0 - XH + lane * V;        // grid column of this lane's element 0

    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        tmap_prefetch(&tm);
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, BOX_BYTES);
        tma_load_3d(box, &tm, x0 - XH, y0 - HR, 0, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, timeout_ns);
    if (!__syncthreads_and(ok)) {
        // give the copy a bounded chance to land before leaving, then report
        mbar_wait_bounded(&bar, 0, 1000000ull);
        if (tid == 0) set_device_error(err, DEV_ERR_TIMEOUT_TMA);
        return;
    }

    // interior columns among this lane's V (fixed for the CTA)
    unsigned colin = 0;
#pragma unroll
    for (int e = 0; e < V; ++e)
        if (gx + e >= 1 && gx + e <= g.C - 2) colin |= 1u << e;
    // One half-sweep over box rows [r_lo, r_hi) for the interior points of
    // colour `colour`, in place.  Warp w walks down its own band of
    // consecutive rows, keeping the north and centre rows in registers and
    // loading only the south row: a point of this colour is read by no one
    // in this half-sweep (its neighbours have the other colour), and the
    // other colour's values -- all that the next row reads from this one --
    // do not change.  A lane computes the points of this colour among its V
    // and writes its V values back as one vector (points of the other colour
    // get the value they already hold).
    // EDGE: the tile reaches the grid's first or last row or column, so rows
    // and columns outside the interior must keep their values; elsewhere
    // every point in the box is interior and needs no test.
    auto half_sweep = [&](auto edge_t, int colour, int r_lo, int r_hi) {
        constexpr bool EDGE = decltype(edge_t)::value;
        constexpr int NWARP = SOR_THREADS / 32;
        const int band = (r_hi - r_lo + NWARP - 1) / NWARP;
        const int b0 = r_lo + warp * band;
        const int b1 = min(b0 + band, r_hi);
        if (b0 >= b1) return;                 // warp-uniform
        CT n[V], c[V], s[V];
        VecIO<ST, V>::load(n, box + (b0 - 1) * W + lane * V);
        VecIO<ST, V>::load(c, box + b0 * W + lane * V);
        for (int r = b0; r < b1; ++r) {
            ST *row = box + r * W + lane * V;
            VecIO<ST, V>::load(s, row + W);
            const int y = y0 - HR + r;
            // element e has colour (y + gx + e) & 1: this row updates
            // elements e0, e0 + 2, ... (gx is even for every lane, so e0 is
            // the same across the warp); rows outside the interior keep
            // their values
            const bool row_in = !EDGE || (y >= 1 && y <= g.R - 2);
            const int e0 = (y + gx + colour) & 1;
            CT o[V];
#pragma unroll
            for (int e = 0; e < V; ++e) o[e] = c[e];
            // west of element 0 (for e0 = 0) or east of element V-1 (for
            // e0 = 1) from the neighbouring lane; lanes 0 and 31 get stale
            // values, which a half-sweep carries one column inward and the
            // column halo absorbs
            if (e0 == 0) {
                const CT left = __shfl_up_sync(FULL_MASK, c[V - 1], 1);
#pragma unroll
                for (int e = 0; e < V; e += 2) {
                    const CT w = e == 0 ? left : c[e - 1];
                    const CT v = sor_point(c[e], n[e], s[e], w, c[e + 1], a, b);
                    if (!EDGE || (row_in && ((colin >> e) & 1u))) o[e] = v;
                }
            } else {
                const CT right = __shfl_down_sync(FULL_MASK, c[0], 1);
#pragma unroll
                for (int e = 1; e < V; e += 2) {
                    const CT ea = e == V - 1 ? right : c[e + 1];
                    const CT v = sor_point(c[e], n[e], s[e], c[e - 1], ea, a, b);
                    if (!EDGE || (row_in && ((colin >> e) & 1u))) o[e] = v;
                }
            }
            VecIO<ST, V>::store(row, o);
            // the next row's north: this row's other-colour values are
            // unchanged, and its own colour is not read by the next row
#pragma unroll
            for (int e = 0; e < V; ++e) {
                n[e] = o[e];
                c[e] = s[e];
            }
        }
    };
    // half-sweep h: colour h & 1 (red first) on box rows [1 + h, BY - 1 - h)
    const bool edge = x0 - XH < 1 || x0 - XH + W > g.C - 1 || y0 - HR < 1 || y0 - HR + SOR_BY > g.R - 1;
    for (int h = 0; h < n_half; ++h) {
        if (edge)
            half_sweep(std::true_type(), h & 1, 1 + h, SOR_BY - 1 - h);
        else
            half_sweep(std::false_type(), h & 1, 1 + h, SOR_BY - 1 - h);
        __syncthreads();
    }

    // write the tile
    const bool own_cols = lane * V >= XH && lane * V < XH + TX && gx < g.C;
    if (own_cols) {
        const bool full_vec = gx + V <= g.C;
        for (int r = HR + warp; r < HR + SH::TY; r += SOR_THREADS / 32) {
            const int y = y0 - HR + r;
            if (y >= g.R) break;
            const ST *row = box + r * W + lane * V;
            ST *q = dst + static_cast<long long>(y) * g.ld + gx;
            if (full_vec) {
                CT v[V];
                VecIO<ST, V>::load(v, row);
                VecIO<ST, V>::store(q, v);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (gx + e < g.C) q[e] = row[e];
            }
        }
    }
}

// ------------------------------------------------- FP32 / BF16 storage ------
template <int I, int N, class F> __device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>());
        static_for<I + 1, N>(f);
    }
}

// Packed FP32x2 add, rounded to nearest.
__device__ __forceinline__ float2 add2_rn(float2 x, float2 y) {
    float2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\t"
        "mov.b64 a, {%2, %3};\n\t"
        "mov.b64 b, {%4, %5};\n\t"
        "add.rn.f32x2 d, a, b;\n\t"
        "mov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y));
    return r;
}
// One row of a half-sweep in registers.  Lane l holds the row's columns
// 4l .. 4l+3 in c; a row of colour parity P updates its elements P and P+2
// in place from the rows above (n) and below (s) -- of which only elements P
// and P+2 are read: they have the other colour -- and from c's other two
// elements.  The same operations, in the same order, as sor_point, each
// rounded on its own: the sums two points per packed FP32x2 add, the products
// scalar.  BF16 storage rounds the new values to BF16.
template <bool BF, int P, bool EDGE>
__device__ __forceinline__ void sor_row_reg(const float (&n)[4], float (&c)[4], const float (&s)[4], float a,
                                            float b, bool row_in, unsigned colin) {
    float2 we;
    if constexpr (P == 0) {
        const float left = __shfl_up_sync(FULL_MASK, c[3], 1);
        we = make_float2(__fadd_rn(left, c[1]), __fadd_rn(c[1], c[3]));
    } else {
        const float right = __shfl_down_sync(FULL_MASK, c[0], 1);
        we = make_float2(__fadd_rn(c[0], c[2]), __fadd_rn(c[2], right));
    }
    const float2 ns = add2_rn(make_float2(n[P], n[P + 2]), make_float2(s[P], s[P + 2]));
    const float2 q = add2_rn(ns, we);
    // the products are scalar: the code generator may fuse a packed product
    // that has a single use into the packed add consuming it (one rounding
    // instead of two), even when both carry an explicit rounding mode
    const float2 ac = make_float2(__fmul_rn(a, c[P]), __fmul_rn(a, c[P + 2]));
    const float2 bq = make_float2(__fmul_rn(b, q.x), __fmul_rn(b, q.y));
    float2 v = add2_rn(ac, bq);
    if constexpr (BF) v = __bfloat1622float2(__float22bfloat162_rn(v));
    if (!EDGE || (row_in && ((colin >> P) & 1u))) c[P] = v.x;
    if (!EDGE || (row_in && ((colin >> (P + 2)) & 1u))) c[P + 2] = v.y;
}

// Warp w holds box rows [w RB, w RB + RB) in registers.  Between half-sweeps
// it publishes its first row to top[w] and its last to bot[w + 1]; in the
// next half-sweep the row above its band is bot[w] and the row below is
// top[w + 1].  The slots are pair-major (elements 0 and 2 of the 32 lanes,
// then elements 1 and 3), and a half-sweep writes only the pair it updated,
// while the neighbouring warp reads only the other pair (adjacent rows have
// opposite parity), so one barrier per half-sweep suffices.  bot[0] and
// top[NW] stand for the rows beyond the box: zeros, whose effect the halo
// absorbs like any other missing neighbour.
template <class ST>
__global__ void __launch_bounds__(SOR_THREADS) sor2d_reg_kernel(const __grid_constant__ CUtensorMap tm,
                                                                ST *__restrict__ dst, const SorGeo g, float a,
                                                                float b, int n_half, int *err,
                                                                unsigned long long timeout_ns) {
    using SH = SorShape<ST>;
    constexpr int V = 4;
    static_assert(SH::V == V, "4 columns per lane");
    constexpr int W = SH::W;
    constexpr int XH = SH::XH;
    constexpr int TX = SH::TX;
    constexpr int HR = SH::HR;
    constexpr int TY = SH::TY;
    constexpr int BY = SH::BY;
    constexpr int NW = SOR_THREADS / 32;
    constexpr int RB = SOR_RB;
    static_assert(BY == NW * RB, "one band of RB rows per warp");
    constexpr bool BF = sizeof(ST) == 2;
    constexpr uint32_t BOX_BYTES = BY * W * sizeof(ST);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) float top[NW + 1][W];
    __shared__ __align__(16) float bot[NW + 1][W];
    ST *box = reinterpret_cast<ST *>(smem_raw);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int tx = blockIdx.x % g.tiles_x;
    const int ty = blockIdx.x / g.tiles_x;
    const int x0 = tx * TX;                   // first output column
    const int y0 = ty * TY;                   // first output row
    // box row r <-> grid row y0 - HR + r; box column k <-> grid column x0 - XH + k
    const int gx = x0 - XH + lane * V;        // grid column of this lane's element 0

    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        tmap_prefetch(&tm);
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, BOX_BYTES);
        tma_load_3d(box, &tm, x0 - XH, y0 - HR, 0, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, timeout_ns);
    if (!__syncthreads_and(ok)) {
        mbar_wait_bounded(&bar, 0, 1000000ull);
        if (tid == 0) set_device_error(err, DEV_ERR_TIMEOUT_TMA);
        return;
    }

    unsigned colin = 0;  // interior columns among this lane's 4
#pragma unroll
    for (int e = 0; e < V; ++e)
        if (gx + e >= 1 && gx + e <= g.C - 2) colin |= 1u << e;

    float X[RB][V];
    static_for<0, RB>([&](auto i_t) {
        constexpr int i = decltype(i_t)::value;
        VecIO<ST, V>::load(X[i], box + (warp * RB + i) * W + lane * V);
    });
    auto put = [&](float *slot, const float (&x)[V], int p) {
        reinterpret_cast<float2 *>(slot + (W / 2) * p)[lane] = make_float2(x[p], x[p + 2]);
    };
    put(top[warp], X[0], 0);
    put(top[warp], X[0], 1);
    put(bot[warp + 1], X[RB - 1], 0);
    put(bot[warp + 1], X[RB - 1], 1);
    if (warp == 0) {
        reinterpret_cast<float4 *>(bot[0])[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4 *>(top[NW])[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    const int yb = y0 - HR + warp * RB;       // grid row of the band's first row
    const bool edge = x0 - XH < 1 || x0 - XH + W > g.C - 1 || y0 - HR < 1 || y0 - HR + BY > g.R - 1;
    // One half-sweep of the band; P is the colour parity of its first row
    // (rows alternate; gx is even for every lane, so it is warp-uniform).
    auto sweep = [&](auto p_t, auto edge_t) {
        constexpr int P = decltype(p_t)::value;
        constexpr bool EDGE = decltype(edge_t)::value;
        constexpr int PL = P ^ ((RB - 1) & 1);  // parity of the band's last row
        float N[V] = {0.f, 0.f, 0.f, 0.f}, S[V] = {0.f, 0.f, 0.f, 0.f};
        {
            const float2 t = reinterpret_cast<const float2 *>(bot[warp] + (W / 2) * P)[lane];
            N[P] = t.x;
            N[P + 2] = t.y;
            const float2 u = reinterpret_cast<const float2 *>(top[warp + 1] + (W / 2) * PL)[lane];
            S[PL] = u.x;
            S[PL + 2] = u.y;
        }
        static_for<0, RB>([&](auto i_t) {
            constexpr int i = decltype(i_t)::value;
            const bool row_in = !EDGE || (yb + i >= 1 && yb + i <= g.R - 2);
            const float(&n)[V] = X[i == 0 ? 0 : i - 1];
            const float(&s)[V] = X[i == RB - 1 ? RB - 1 : i + 1];
            if constexpr (i == 0 && RB == 1)
                sor_row_reg<BF, P, EDGE>(N, X[i], S, a, b, row_in, colin);
            else if constexpr (i == 0)
                sor_row_reg<BF, P, EDGE>(N, X[i], s, a, b, row_in, colin);
            else if constexpr (i == RB - 1)
                sor_row_reg<BF, P ^ (i & 1), EDGE>(n, X[i], S, a, b, row_in, colin);
            else
                sor_row_reg<BF, P ^ (i & 1), EDGE>(n, X[i], s, a, b, row_in, colin);
        });
        put(top[warp], X[0], P);
        put(bot[warp + 1], X[RB - 1], PL);
    };
    for (int h = 0; h < n_half; ++h) {
        const bool p1 = ((yb + gx + (h & 1)) & 1) != 0;
        if (edge) {
            if (p1) sweep(std::integral_constant<int, 1>(), std::true_type());
            else sweep(std::integral_constant<int, 0>(), std::true_type());
        } else {
            if (p1) sweep(std::integral_constant<int, 1>(), std::false_type());
            else sweep(std::integral_constant<int, 0>(), std::false_type());
        }
        __syncthreads();
    }

    // write the tile's rows [HR, HR + TY) straight from registers
    const bool own_cols = lane * V >= XH && lane * V < XH + TX && gx < g.C;
    if (own_cols) {
        const bool full_vec = gx + V <= g.C;
        static_for<0, RB>([&](auto i_t) {
            constexpr int i = decltype(i_t)::value;
            const int r = warp * RB + i;
            const int y = y0 - HR + r;
            if (r >= HR && r < HR + TY && y < g.R) {
                ST *q = dst + static_cast<long long>(y) * g.ld + gx;
                if (full_vec) {
                    VecIO<ST, V>::store(q, X[i]);
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (gx + e < g.C) q[e] = static_cast<ST>(X[i][e]);
                }
            }
        });
    }
}

// ------------------------------------------------------------------ host -----
static const void *sor_kernel(int dtype) {
    switch (dtype) {
        case SDFG_F32: return reinterpret_cast<const void *>(&sor2d_reg_kernel<float>);
        case SDFG_BF16: return reinterpret_cast<const void *>(&sor2d_reg_kernel<__nv_bfloat16>);
        default: return reinterpret_cast<const void *>(&sor2d_kernel<double>);
    }
}

template <class ST> static void sor_shape_of(int &ki, int &w, int &tx, int &by, int &ty) {
    ki = SorShape<ST>::KI;
    w = SorShape<ST>::W;
    tx = SorShape<ST>::TX;
    by = SorShape<ST>::BY;
    ty = SorShape<ST>::TY;
}
static void sor_shape(int dtype, int &ki, int &w, int &tx, int &by, int &ty) {
    switch (dtype) {
        case SDFG_F32: sor_shape_of<float>(ki, w, tx, by, ty); break;
        case SDFG_BF16: sor_shape_of<__nv_bfloat16>(ki, w, tx, by, ty); break;
        default: sor_shape_of<double>(ki, w, tx, by, ty); break;
    }
}

static int launch_sor(const CUtensorMap &tm, void *dst, const SorGeo &g, int dtype, double omega, int n_iter,
                      int *err, cudaStream_t s) {
    const void *fn = sor_kernel(dtype);
    int ki, w, tx, by, ty;
    sor_shape(dtype, ki, w, tx, by, ty);
    const size_t smem = static_cast<size_t>(by) * w * dtype_bytes(dtype);
    int n_half = 2 * n_iter;
    CUtensorMap t = tm;
    SorGeo gg = g;
    void *dp = dst;
    unsigned long long to = DEFAULT_TIMEOUT_NS;
    // the two coefficients, evaluated once in double and then converted to
    // the compute type
    const double ad = 1.0 - omega, bd = 0.25 * omega;
    float af = static_cast<float>(ad), bf = static_cast<float>(bd);
    double a64 = ad, b64 = bd;
    void *args_f[] = {&t, &dp, &gg, &af, &bf, &n_half, &err, &to};
    void *args_d[] = {&t, &dp, &gg, &a64, &b64, &n_half, &err, &to};
    const unsigned blocks = static_cast<unsigned>(static_cast<long long>(g.tiles_x) * ((g.R + ty - 1) / ty));
    TimedLaunch tl = stats_begin(FAM_SOR, s);
    cudaError_t e = cudaLaunchKernel(fn, dim3(blocks), dim3(SOR_THREADS), dtype == SDFG_F64 ? args_d : args_f, smem, s);
    stats_end(tl, s);
    if (e != cudaSuccess) return cuda_error(e, "sor2d launch");
    return SDFG_OK;
}

static bool sor_tma_ok(const void *p, int ld, int dtype) {
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((static_cast<long long>(ld) * dtype_bytes(dtype)) % 16 == 0);
}

}  // namespace sdfg

using namespace sdfg;

extern "C" int sdfg_sor2d(const void *in, void *out, int rows, int cols, int ld, int T, double omega, int dtype,
                          void *stream) {
    if (rows < 0 || cols < 0 || T < 0 || !dtype_valid(dtype) || !isfinite(omega))
        return set_error(SDFG_ERR_INVAL, "sdfg_sor2d: bad extents, T, omega or dtype (%d x %d, T=%d, dtype %d)", rows,
                         cols, T, dtype);
    if (ld < cols) return set_error(SDFG_ERR_INVAL, "sdfg_sor2d: ld %d < cols %d", ld, cols);
    if (rows == 0 || cols == 0) return SDFG_OK;
    if (!in || !out) return set_error(SDFG_ERR_INVAL, "sdfg_sor2d: null grid");
    DeviceState *st = nullptr;
    int rc = current_device(&st);
    if (rc != SDFG_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (T == 0 || rows < 3 || cols < 3) {
        if (in == out) return SDFG_OK;
        return launch_copy2d(out, ld, in, ld, rows, cols, dtype, s);
    }
    const size_t S = dtype_bytes(dtype);
    int ki, box_cols, tile_cols, box_rows, tile_rows;
    sor_shape(dtype, ki, box_cols, tile_cols, box_rows, tile_rows);
    // launches of ki iterations, then one of the remainder
    const int n_pass = T / ki + (T % ki ? 1 : 0);
    const bool aligned = sor_tma_ok(in, ld, dtype) && sor_tma_ok(out, ld, dtype);
    const int ldw = aligned ? ld : (cols + 31) / 32 * 32;
    const size_t bytes = static_cast<size_t>(rows) * ldw * S;
    void *a = nullptr, *b = nullptr;
    const void *src0 = in;
    void *first = nullptr, *second = nullptr;
    if (aligned) {
        rc = scratch_alloc(&a, bytes, s);
        if (rc != SDFG_OK) return rc;
        if (in != out) {
            // the last pass must land in `out`
            first = (n_pass % 2 == 1) ? out : a;
            second = first == out ? a : out;
        } else {
            first = a;
            second = out;
        }
    } else {
        rc = scratch_alloc(&a, bytes, s);
        if (rc == SDFG_OK) rc = scratch_alloc(&b, bytes, s);
        if (rc == SDFG_OK) rc = launch_copy2d(a, ldw, in, ld, rows, cols, dtype, s);
        if (rc != SDFG_OK) {
            scratch_free(a, s);
            scratch_free(b, s);
            return rc;
        }
        src0 = a;
        first = b;
        second = a;
    }
    const void *fn = sor_kernel(dtype);
    const size_t smem = static_cast<size_t>(box_rows) * box_cols * S;
    static bool attr_done[3] = {false, false, false};
    if (!attr_done[dtype]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) rc = cuda_error(e, "sor2d attribute");
        else attr_done[dtype] = true;
    }
    alignas(128) CUtensorMap tm_src0, tm_first, tm_second;
    if (rc == SDFG_OK) rc = encode_tmap3d(&tm_src0, src0, dtype, 1, rows, cols, ldw, box_cols, box_rows);
    if (rc == SDFG_OK) rc = encode_tmap3d(&tm_first, first, dtype, 1, rows, cols, ldw, box_cols, box_rows);
    if (rc == SDFG_OK) rc = encode_tmap3d(&tm_second, second, dtype, 1, rows, cols, ldw, box_cols, box_rows);
    SorGeo g;
    g.R = rows;
    g.C = cols;
    g.ld = ldw;
    g.tiles_x = (cols + tile_cols - 1) / tile_cols;
    const CUtensorMap *tsrc = &tm_src0;
    void *dst = first;
    void *fin = const_cast<void *>(src0);
    for (int p = 0; p < n_pass && rc == SDFG_OK; ++p) {
        const int n_iter = (p < T / ki) ? ki : T % ki;
        rc = launch_sor(*tsrc, dst, g, dtype, omega, n_iter, st->d_err, s);
        fin = dst;
        tsrc = dst == first ? &tm_first : &tm_second;
        dst = dst == first ? second : first;
    }
    if (rc == SDFG_OK && fin != out) rc = launch_copy2d(out, ld, fin, ldw, rows, cols, dtype, s);
    scratch_free(a, s);
    scratch_free(b, s);
    return rc;
}
