// The temporal-blocked work unit: one warp advances one tile of the grid by
// K timesteps in a single pass over HBM.
//
// FP32 arithmetic reassociates the 5-point sum and applies 0.2^K once per pass
// (see level_sum); FP64 keeps the exact order 0.2 * (c + ((n + s) + (w + e))).
//
// Paper mapping (App. B transformations, applied by hand):
//   MapTiling      -- the interior map is cut into strips of `wout` columns and
//                     segments of `H` rows; one warp owns one (strip, segment);
//   LocalStorage   -- rows of the tile are staged in shared memory by TMA;
//   DoubleBuffering-- a ring of STAGES chunks: TMA fills chunk c+STAGES while
//                     the warp computes on chunk c;
//   Vectorization  -- each lane holds V consecutive columns (16-byte accesses
//                     for FP32/FP64, 8-byte for BF16);
//   StateFusion /
//   MapToForLoop   -- K timestep-states are fused (in FP32 registers; a BF16
//                     grid is rounded to BF16 when a pass stores it): the warp streams down its
//                     column strip and keeps, for every fused level l < K, the
//                     three most recent rows of level l in registers.  A new
//                     level-0 row from shared memory lets level 0 produce one
//                     row of level 1, which lets level 1 produce one row of
//                     level 2, and so on; level K rows are final and go
//                     straight to HBM.
// West/east neighbours come from the adjacent lanes by warp shuffle; the
// outermost lanes' values go stale by one column per level, so a strip
// overlaps its neighbours by h >= K columns on each side (overlapped temporal
// tiling); along rows a segment re-reads K rows above and below.
//
// The boundary ring is fixed (Dirichlet): a level never changes a point of
// row 0, row R-1, column 0 or column C-1; rows/columns outside the grid come
// from TMA's zero fill and only ever feed other outside points or the
// boundary, whose value is copied, so they never reach a stored result.
#pragma once

#include <type_traits>

#include "device_common.cuh"
#include "geometry.h"

namespace sdfg {

// ---------------------------------------------------------------- one level --
// o <- stencil(n, c, s) for the V columns of this lane; west of element 0 and
// east of element V-1 come from the neighbouring lanes.
template <int V, bool COLCHK>
__device__ __forceinline__ void level_row(float (&o)[V], const float (&n)[V], const float (&c)[V],
                                          const float (&s)[V], unsigned colmask) {
    const float left = __shfl_up_sync(FULL_MASK, c[V - 1], 1);
    const float right = __shfl_down_sync(FULL_MASK, c[0], 1);
    float we[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const float w = (e == 0) ? left : c[e - 1];
        const float ea = (e == V - 1) ? right : c[e + 1];
        we[e] = __fadd_rn(w, ea);
    }
#pragma unroll
    for (int p = 0; p < V / 2; ++p) {
        // packed FP32x2: (n+s), then (n+s)+(w+e), then c+(...), then *0.2
        const float2 ns = __fadd2_rn(make_float2(n[2 * p], n[2 * p + 1]), make_float2(s[2 * p], s[2 * p + 1]));
        const float2 t = __fadd2_rn(ns, make_float2(we[2 * p], we[2 * p + 1]));
        const float2 u = __fadd2_rn(make_float2(c[2 * p], c[2 * p + 1]), t);
        const float2 r = __fmul2_rn(make_float2(0.2f, 0.2f), u);
        o[2 * p] = r.x;
        o[2 * p + 1] = r.y;
    }
    if (COLCHK) {
#pragma unroll
        for (int e = 0; e < V; ++e)
            if ((colmask >> e) & 1u) o[e] = c[e];
    }
}

// Register pairing of a lane's V = 4 columns in the packed FP32x2 adds: the
// pairs (0, 1), (2, 3) as a 16-byte load lands them; the pairs (0, 2), (1, 3),
// which pack one more add; or the first in and the second out.
constexpr int PAIRS_NATURAL = 0, PAIRS_SPLIT = 1, PAIRS_ENTRY = 2;

// FP32 arithmetic (FP32 and BF16 storage): a fused level carries the UNSCALED
// 5-point sum, so interior values at level l are 5^l times the state and the
// factor 0.2^K is applied once, at the last level of the pass.  The row sum
// shares horizontal pairs: Q = u0 + u1 serves H0 = w + Q and H1 = Q + u2, so
// the 5-point sum costs 3.5 adds per point (n + s, H, H + (n + s)) and no
// multiply.  Boundary cells keep their unscaled value b at every level; a
// neighbour reads it as 5^l * b (`lscale`), and the last level copies b, so
// the Dirichlet ring is stored exactly.
template <int V, bool COLCHK, int PAIRS>
__device__ __forceinline__ void level_sum(float (&o)[V], const float (&n)[V], const float (&c)[V],
                                          const float (&s)[V], unsigned colmask, float lscale) {
    static_assert(V % 2 == 0, "pairs of columns");
    float cc[V];  // the centre row as its neighbours see it
#pragma unroll
    for (int e = 0; e < V; ++e) cc[e] = (COLCHK && ((colmask >> e) & 1u)) ? __fmul_rn(c[e], lscale) : c[e];
    const float left = __shfl_up_sync(FULL_MASK, cc[V - 1], 1);
    const float right = __shfl_down_sync(FULL_MASK, cc[0], 1);
    if constexpr (PAIRS == PAIRS_SPLIT && V == 4) {
        // The same sums, packed as the column pairs (0, 2) and (1, 3): then
        // Q = (u0 + u1, u2 + u3) is one FP32x2 add, and every other pair op
        // is elementwise, so the pairing changes no result.
        const float2 q = __fadd2_rn(make_float2(cc[0], cc[2]), make_float2(cc[1], cc[3]));
        const float2 h02 = make_float2(__fadd_rn(left, q.x), __fadd_rn(cc[1], q.y));
        const float2 h13 = make_float2(__fadd_rn(q.x, cc[2]), __fadd_rn(q.y, right));
        const float2 ns02 = __fadd2_rn(make_float2(n[0], n[2]), make_float2(s[0], s[2]));
        const float2 ns13 = __fadd2_rn(make_float2(n[1], n[3]), make_float2(s[1], s[3]));
        const float2 r02 = __fadd2_rn(h02, ns02);
        const float2 r13 = __fadd2_rn(h13, ns13);
        o[0] = r02.x;
        o[2] = r02.y;
        o[1] = r13.x;
        o[3] = r13.y;
    } else if constexpr (PAIRS == PAIRS_ENTRY && V == 4) {
        // Rows as a 16-byte load leaves them (pairs (0, 1), (2, 3)) in, the
        // split pairs out: the last adds are scalar, so no row is re-paired.
        const float q0 = __fadd_rn(cc[0], cc[1]);
        const float q1 = __fadd_rn(cc[2], cc[3]);
        const float2 ns01 = __fadd2_rn(make_float2(n[0], n[1]), make_float2(s[0], s[1]));
        const float2 ns23 = __fadd2_rn(make_float2(n[2], n[3]), make_float2(s[2], s[3]));
        o[0] = __fadd_rn(__fadd_rn(left, q0), ns01.x);
        o[1] = __fadd_rn(__fadd_rn(q0, cc[2]), ns01.y);
        o[2] = __fadd_rn(__fadd_rn(cc[1], q1), ns23.x);
        o[3] = __fadd_rn(__fadd_rn(q1, right), ns23.y);
    } else {
    float h[V];
#pragma unroll
    for (int p = 0; p < V / 2; ++p) {
        const float q = __fadd_rn(cc[2 * p], cc[2 * p + 1]);
        const float w = (p == 0) ? left : cc[2 * p - 1];
        const float ea = (2 * p + 2 == V) ? right : cc[2 * p + 2];
        h[2 * p] = __fadd_rn(w, q);
        h[2 * p + 1] = __fadd_rn(q, ea);
    }
#pragma unroll
    for (int p = 0; p < V / 2; ++p) {
        const float2 ns = __fadd2_rn(make_float2(n[2 * p], n[2 * p + 1]), make_float2(s[2 * p], s[2 * p + 1]));
        const float2 r = __fadd2_rn(make_float2(h[2 * p], h[2 * p + 1]), ns);
        o[2 * p] = r.x;
        o[2 * p + 1] = r.y;
    }
    }
    if (COLCHK) {
#pragma unroll
        for (int e = 0; e < V; ++e)
            if ((colmask >> e) & 1u) o[e] = c[e];
    }
}

// 0.2^k in double, for the hi/lo split of the last level's scale factor.
__host__ __device__ constexpr double pow_fifth(int k) { return k <= 0 ? 1.0 : 0.2 * pow_fifth(k - 1); }
// 5^k (exact in FP32 for k <= 10).
__host__ __device__ constexpr float pow_five(int k) { return k <= 0 ? 1.0f : 5.0f * pow_five(k - 1); }

// The reassociated level with a two-row register ring.  Level l keeps, for the
// row c it received last, that row itself (`a`) and its output's partial sum
// north + (w + c + e) (`p`); the output of row c is complete as soon as its
// south row x arrives:
//     o(c)   = p(c) + x            (one add on the level-to-level path)
//     p(x)   = a(c) + H3(x)        (H3: the horizontal three-point sum of x)
//     a      <- x
// H3 shares the pair sums q = u0 + u1 and u2 + u3 between neighbouring columns
// (h0 = w + q01, h1 = q01 + u2, h2 = u1 + q23, h3 = q23 + e).  The sum is
// carried unscaled (level l holds 5^l times the state), as in level_sum.
// PAIRS_SPLIT: x, a, p and o pack the column pairs (0, 2), (1, 3);
// PAIRS_ENTRY: x, a and p are pairs (0, 1), (2, 3) as a 16-byte load leaves a
// row, and o is formed by scalar adds (the next level packs it split).
template <int V, int PAIRS>
__device__ __forceinline__ void level_p(float (&o)[V], float (&a)[V], float (&p)[V], const float (&x)[V]) {
    static_assert(V == 4, "the two-row ring packs four columns per lane");
    const float left = __shfl_up_sync(FULL_MASK, x[V - 1], 1);
    const float right = __shfl_down_sync(FULL_MASK, x[0], 1);
    if constexpr (PAIRS == PAIRS_SPLIT) {
        const float2 o02 = __fadd2_rn(make_float2(p[0], p[2]), make_float2(x[0], x[2]));
        const float2 o13 = __fadd2_rn(make_float2(p[1], p[3]), make_float2(x[1], x[3]));
        o[0] = o02.x;
        o[2] = o02.y;
        o[1] = o13.x;
        o[3] = o13.y;
        const float2 q = __fadd2_rn(make_float2(x[0], x[2]), make_float2(x[1], x[3]));
        const float2 h02 = make_float2(__fadd_rn(left, q.x), __fadd_rn(x[1], q.y));
        const float2 h13 = make_float2(__fadd_rn(q.x, x[2]), __fadd_rn(q.y, right));
        const float2 p02 = __fadd2_rn(make_float2(a[0], a[2]), h02);
        const float2 p13 = __fadd2_rn(make_float2(a[1], a[3]), h13);
        p[0] = p02.x;
        p[2] = p02.y;
        p[1] = p13.x;
        p[3] = p13.y;
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) o[e] = __fadd_rn(p[e], x[e]);
        const float q01 = __fadd_rn(x[0], x[1]);
        const float q23 = __fadd_rn(x[2], x[3]);
        const float2 h01 = make_float2(__fadd_rn(left, q01), __fadd_rn(q01, x[2]));
        const float2 h23 = make_float2(__fadd_rn(x[1], q23), __fadd_rn(q23, right));
        const float2 p01 = __fadd2_rn(make_float2(a[0], a[1]), h01);
        const float2 p23 = __fadd2_rn(make_float2(a[2], a[3]), h23);
        p[0] = p01.x;
        p[1] = p01.y;
        p[2] = p23.x;
        p[3] = p23.y;
    }
#pragma unroll
    for (int e = 0; e < V; ++e) a[e] = x[e];
}

template <int V, bool COLCHK>
__device__ __forceinline__ void level_row(double (&o)[V], const double (&n)[V], const double (&c)[V],
                                          const double (&s)[V], unsigned colmask) {
    const double left = __shfl_up_sync(FULL_MASK, c[V - 1], 1);
    const double right = __shfl_down_sync(FULL_MASK, c[0], 1);
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const double w = (e == 0) ? left : c[e - 1];
        const double ea = (e == V - 1) ? right : c[e + 1];
        o[e] = stencil_point(c[e], n[e], s[e], w, ea);
    }
    if (COLCHK) {
#pragma unroll
        for (int e = 0; e < V; ++e)
            if ((colmask >> e) & 1u) o[e] = c[e];
    }
}

// A chunk wait ran out at chunk c0: give the copies already in flight a short
// bounded chance to land (so none writes shared memory after the warp has
// left), then report failure.
__device__ __noinline__ inline bool drain_after_timeout(uint64_t *bars, uint32_t base, int n_chunks, int c0) {
    for (int c = c0; c < n_chunks && c < c0 + STAGES; ++c) {
        const uint32_t g = base + static_cast<uint32_t>(c);
        mbar_wait_bounded(&bars[g % STAGES], (g / STAGES) & 1u, 1000000ull);
    }
    __syncwarp();
    return false;
}

// ---------------------------------------------------------- the unit pipe --
// Rows are consumed in chunks of CR rows (one TMA box: CHUNK_ROWS = 12 for
// the per-pass and persistent kernels, 18 or 24 for the chain kernels), each
// chunk a few turns of one unrolled body of rows: within a body all levels
// and rows can be interleaved by the compiler (level l of row i+1 only
// depends on level l-1 of rows i-1..i+1).  The exact-order pipe's chunks away
// from the grid's top and bottom rows and inside the unit's output rows take
// a FAST body, with no boundary or range test at all.
#ifndef SDFG_SCALED_ONE_BODY
#define SDFG_SCALED_ONE_BODY 1
#endif
#ifndef SDFG_SPLIT_PAIRS
#define SDFG_SPLIT_PAIRS 1
#endif
#ifndef SDFG_RING2
#define SDFG_RING2 1  // reassociated units keep two rows per level (level_p)
#endif
#ifndef SDFG_RING2_ALL_BODY
#define SDFG_RING2_ALL_BODY 1  // BF16 chains: a chunk body without the per-row store test where every row is stored
#endif
#ifndef SDFG_RES_FP64
#define SDFG_RES_FP64 0  // residual: square and sum every difference in FP64 (else FP32 groups)
#endif
#ifndef SDFG_RING2_TURN
#define SDFG_RING2_TURN 4  // rows per turn of the two-row-ring chunk loop (per-pass and persistent units)
#endif
static_assert(CHUNK_ROWS % SDFG_RING2_TURN == 0, "chunks are whole turns");

// Hook of UnitPipe::run for work units that depend on other units while they
// stream (the chain kernel, skewed.cu).  The whole warp calls ready(c) before
// chunk c is loaded (false: a bounded wait ran out) and done(c) once chunk c's
// rows are stored and the warp is synchronised.  EDGES: a unit of the
// reassociated pipe may hold row 0 or row R-1 (see step2).  The units of the
// per-pass and persistent kernels need none of it.  TURN: rows per turn of
// the two-row-ring chunk loop (one unrolled body); the best value differs
// between the kernels (measured).
struct NoHook {
    static constexpr bool EDGES = false;
    static constexpr int TURN = SDFG_RING2_TURN;
    __device__ __forceinline__ bool ready(int) { return true; }
    __device__ __forceinline__ void done(int) {}
};

// CR: rows per TMA chunk (CHUNK_ROWS; the chain kernels stream taller ones).
template <class ST, int V, int K, bool COLCHK, bool RES, bool EXACT, int CR = CHUNK_ROWS>
struct UnitPipe {
    static_assert(CR % 3 == 0, "chunks are whole turns of the 3-row rotation");
    using CT = typename Store<ST>::CT;
    // inner levels pack the column pairs (0, 2), (1, 3); BF16 rows (the
    // 2-byte type) enter registers through a conversion that can place them
    // so, FP32 rows as a 16-byte load pairs them and level 0 switches over
    static constexpr bool SPLIT = SDFG_SPLIT_PAIRS && V == 4;
    static constexpr int PAIRS0 = !SPLIT ? PAIRS_NATURAL : sizeof(ST) == 2 ? PAIRS_SPLIT : PAIRS_ENTRY;
    static constexpr int PAIRS1 = SPLIT ? PAIRS_SPLIT : PAIRS_NATURAL;
    static constexpr int W = 32 * V;
    static constexpr uint32_t CHUNK_BYTES = CR * W * sizeof(ST);
    // units away from the boundary ring reassociate (see level_sum); a unit
    // that holds a boundary row or column keeps the exact order throughout
    static constexpr bool SCALED = sizeof(CT) == 4 && !EXACT;
    // reassociated units with four columns per lane use the two-row ring
    static constexpr bool RING2 = SCALED && SDFG_RING2 && V == 4;

    CT b[K][3][V];  // level l, ring slot, column: rows r-l-2, r-l-1, r-l of level l
    CT ra[K][V];    // two-row ring (RING2): level l's last row ...
    CT rp[K][V];    // ... and its output's partial sum (see level_p)

    const void *tmap;
    ST *dst;
    int ld, R, C;
    int X, y0, y1, rb, n_steps, n_chunks;
    int sy0, sy1;  // rows the reassociated pipe stores: [y0, y1) without the boundary rows
    uint32_t base;
    ST *ring;
    uint64_t *bars;
    int lane;
    unsigned colmask, resmask;
    bool own_lane, full_vec;
    int res_flags;
    // group sums (at most CR rows of one lane's V columns): in the
    // storage type's arithmetic, or (SDFG_RES_FP64) every square in FP64
    using RT = typename std::conditional<SDFG_RES_FP64 != 0, double, CT>::type;
    RT g_ref, g_chk;
    double acc_ref, acc_chk;
    unsigned long long timeout_ns;

    __device__ __forceinline__ void issue(int c) {
        const uint32_t slot = (base + static_cast<uint32_t>(c)) % STAGES;
        mbar_arrive_expect_tx(&bars[slot], CHUNK_BYTES);
        tma_load_2d(ring + slot * (CR * W), tmap, X, rb + c * CR, &bars[slot]);
    }

    __device__ __forceinline__ void accumulate(RT &g, const CT (&o)[V], const CT (&c)[V]) {
        RT sum = RT(0);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            if ((resmask >> e) & 1u) {
                const RT d = static_cast<RT>(o[e] - c[e]);  // the difference in the storage arithmetic
                sum = fma(d, d, sum);
            }
        }
        g = g + sum;
    }

    // Store one output row at `p` (= row start + X + lane*V).  Away from
    // the boundary columns every owned lane holds V in-grid columns, so the
    // store is one predicated vector instruction.  The reassociated pipe on
    // a boundary strip (RING2 with COLCHK) never stores the boundary
    // columns: the caller provides them in the destination grid.
    __device__ __forceinline__ void store_row(ST *p, const CT (&o)[V]) {
        if (!COLCHK) {
            store_pred(p, o, own_lane ? 1 : 0);
        } else if (RING2) {
            if (own_lane) {
                if (colmask == 0u) {
                    VecIO<ST, V>::store(p, o);
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const int gc = X + lane * V + e;
                        if (gc >= 1 && gc <= C - 2) p[e] = from_ct<ST>(o[e]);
                    }
                }
            }
        } else if (own_lane) {
            if (full_vec) {
                VecIO<ST, V>::store(p, o);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (X + lane * V + e < C) p[e] = from_ct<ST>(o[e]);
            }
        }
    }

    // One input row r (level 0 from shared memory at `src`), all K levels.
    template <int PH, bool SLOW>
    __device__ __forceinline__ void step(int r, const ST *src, ST *out) {
        constexpr int SN = (PH + 1) % 3;  // slot of the north row
        constexpr int SC = (PH + 2) % 3;  // slot of the centre row
        constexpr int SS = PH;            // slot of the south (newest) row
        {
            CT tmp[V];
            VecIO<ST, V>::load(tmp, src);
#pragma unroll
            for (int e = 0; e < V; ++e) b[0][SS][e] = tmp[e];
        }
#pragma unroll
        for (int l = 0; l < K; ++l) {
            CT o[V];
            const int rc = r - l - 1;  // row index of this level's centre
            if constexpr (SCALED) {
                const float LS = 1.0f;  // (no boundary cell inside a scaled unit)
                // no boundary row or column reaches this unit: one fast sum
                if (l == 0)
                    level_sum<V, false, PAIRS0>(o, b[l][SN], b[l][SC], b[l][SS], colmask, LS);
                else
                    level_sum<V, false, PAIRS1>(o, b[l][SN], b[l][SC], b[l][SS], colmask, LS);
                if (l == K - 1) {
                    // the pass's scale factor 0.2^K, split hi + lo so the product is
                    // rounded once from a ~48-bit factor
                    constexpr double F = pow_fifth(K);
                    constexpr float FHI = static_cast<float>(F);
                    constexpr float FLO = static_cast<float>(F - static_cast<double>(FHI));
                    // the column pairs level_sum packs
                    constexpr bool SP = (K == 1 ? PAIRS0 : PAIRS1) != PAIRS_NATURAL;
                    constexpr int STEP = SP ? V / 2 : 1;
#pragma unroll
                    for (int p = 0; p < V / 2; ++p) {
                        const int e0 = SP ? p : 2 * p;
                        const float2 u = make_float2(o[e0], o[e0 + STEP]);
                        const float2 t = __fmul2_rn(u, make_float2(FLO, FLO));
                        const float2 f = __ffma2_rn(u, make_float2(FHI, FHI), t);
                        o[e0] = f.x;
                        o[e0 + STEP] = f.y;
                    }
                }
            } else {
                level_row<V, COLCHK>(o, b[l][SN], b[l][SC], b[l][SS], colmask);
            }
            if (!SCALED && SLOW && (rc <= 0 || rc >= R - 1)) {
                // the boundary ring (and rows outside the grid) keep their value
#pragma unroll
                for (int e = 0; e < V; ++e) o[e] = b[l][SC][e];
            }
            if (RES && l == 0 && (res_flags & 1)) {
                const int row = r - 1;
                if (row >= y0 && row < y1 && row >= 1 && row <= R - 2) {
                    CT a1[V];
#pragma unroll
                    for (int e = 0; e < V; ++e) a1[e] = (SCALED && K > 1) ? CT(0.2f) * o[e] : o[e];
                    accumulate(g_ref, a1, b[0][SC]);
                }
            }
            if (l == K - 1) {
                const int row = r - K;
                if (!SLOW || (row >= y0 && row < y1)) {
                    if (RES && (res_flags & 2) && row >= 1 && row <= R - 2) {
                        CT prev[V];
                        constexpr CT PS = SCALED ? CT(pow_fifth(K - 1)) : CT(1);
#pragma unroll
                        for (int e = 0; e < V; ++e) prev[e] = PS * b[l][SC][e];
                        accumulate(g_chk, o, prev);
                    }
                    store_row(out, o);
                }
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) b[l + 1][SS][e] = o[e];
            }
        }
    }

    // The pass's scale factor 0.2^K on the last level's output, split hi + lo
    // so the product is rounded once from a ~48-bit factor.
    template <int PAIRS_LAST>
    __device__ __forceinline__ static void scale_last(CT (&o)[V]) {
        constexpr double F = pow_fifth(K);
        constexpr float FHI = static_cast<float>(F);
        constexpr float FLO = static_cast<float>(F - static_cast<double>(FHI));
        constexpr bool SP = PAIRS_LAST != PAIRS_NATURAL;  // the column pairs the level packs
        constexpr int STEP = SP ? V / 2 : 1;
#pragma unroll
        for (int p = 0; p < V / 2; ++p) {
            const int e0 = SP ? p : 2 * p;
            const float2 u = make_float2(o[e0], o[e0 + STEP]);
            const float2 t = __fmul2_rn(u, make_float2(FLO, FLO));
            const float2 f = __ffma2_rn(u, make_float2(FHI, FHI), t);
            o[e0] = f.x;
            o[e0 + STEP] = f.y;
        }
    }

    // One input row r through all K levels of the two-row ring (RING2).
    // Level l's output at this row is centre row r-l-1, as in `step`.
    // EDGE: row 0 or row R-1 may be a centre row.  A boundary row keeps its
    // value, which a level holds scaled like every other row (5^l times the
    // state, each factor 5 rounded once), so its neighbours' sums stay
    // consistent; such rows are never stored by this pipe (sy0 >= 1,
    // sy1 <= R-1): the caller provides them in the destination grid.  With
    // COLCHK the same holds for columns 0 and C-1 of a boundary strip.
    // ALL: every row of the chunk is a stored row (no per-row range test).
    template <bool EDGE, bool ALL = false>
    __device__ __forceinline__ void step2(int r, const ST *src, ST *out) {
        CT x[V];
        VecIO<ST, V>::load(x, src);
#pragma unroll
        for (int l = 0; l < K; ++l) {
            CT o[V];
            CT cen[V];  // the centre row (for the residual sums and the boundary)
            if (RES || EDGE || COLCHK) {
#pragma unroll
                for (int e = 0; e < V; ++e) cen[e] = ra[l][e];
            }
            if (l == 0)
                level_p<V, PAIRS0>(o, ra[l], rp[l], x);
            else
                level_p<V, PAIRS_SPLIT>(o, ra[l], rp[l], x);
            if (EDGE) {
                const int rc = r - l - 1;
                if (rc == 0 || rc == R - 1) {
#pragma unroll
                    for (int e = 0; e < V; ++e) o[e] = __fmul_rn(5.0f, cen[e]);
                }
            }
            if (COLCHK) {
                // boundary columns (and columns outside the grid, which only
                // ever feed them) keep their value, scaled like the rows
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if ((colmask >> e) & 1u) o[e] = __fmul_rn(5.0f, cen[e]);
            }
            if (l == K - 1) scale_last<(K == 1 ? PAIRS0 : PAIRS_SPLIT)>(o);
            if (RES && l == 0 && (res_flags & 1)) {
                const int row = r - 1;
                if (row >= y0 && row < y1 && row >= 1 && row <= R - 2) {
                    CT a1[V];
#pragma unroll
                    for (int e = 0; e < V; ++e) a1[e] = K > 1 ? CT(0.2f) * o[e] : o[e];
                    accumulate(g_ref, a1, cen);
                }
            }
            if (l == K - 1) {
                const int row = r - K;
                if (ALL || (row >= sy0 && row < sy1)) {
                    if (RES && (res_flags & 2) && row >= 1 && row <= R - 2) {
                        CT prev[V];
                        constexpr CT PS = CT(pow_fifth(K - 1));
#pragma unroll
                        for (int e = 0; e < V; ++e) prev[e] = PS * cen[e];
                        accumulate(g_chk, o, prev);
                    }
                    store_row(out, o);
                }
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) x[e] = o[e];
            }
        }
    }

    template <bool EDGE, int TURN, bool ALL = false>
    __device__ __forceinline__ void chunk_body2(int r0, const ST *src, ST *out) {
        static_assert(CR % TURN == 0, "chunks are whole turns");
        const size_t ldr = static_cast<size_t>(ld);
#pragma unroll 1
        for (int h = 0; h < CR / TURN; ++h) {
#pragma unroll
            for (int i = 0; i < TURN; ++i) step2<EDGE, ALL>(r0 + i, src + i * W, out + i * ldr);
            r0 += TURN;
            src += TURN * W;
            out += TURN * ldr;
        }
    }

    // `out` points at output row r0-K (it is only dereferenced for rows the
    // unit owns).  The chunk is CR/3 turns of one 3-row body: a
    // small hot loop (instruction cache).
    template <bool SLOW>
    __device__ __forceinline__ void chunk_body(int r0, const ST *src, ST *out) {
        const size_t ldr = static_cast<size_t>(ld);
#pragma unroll 1
        for (int h = 0; h < CR / 3; ++h) {
            step<0, SLOW>(r0 + 0, src + 0 * W, out);
            step<1, SLOW>(r0 + 1, src + 1 * W, out + ldr);
            step<2, SLOW>(r0 + 2, src + 2 * W, out + 2 * ldr);
            r0 += 3;
            src += 3 * W;
            out += 3 * ldr;
        }
    }

    __device__ __forceinline__ bool run() {
        NoHook hk;
        return run(hk);
    }

    template <class Hook>
    __device__ __forceinline__ bool run(Hook &hk) {
        if constexpr (RING2) {
#pragma unroll
            for (int l = 0; l < K; ++l)
#pragma unroll
                for (int e = 0; e < V; ++e) ra[l][e] = rp[l][e] = CT(0);
        } else {
#pragma unroll
            for (int l = 0; l < K; ++l)
#pragma unroll
                for (int s = 0; s < 3; ++s)
#pragma unroll
                    for (int e = 0; e < V; ++e) b[l][s][e] = CT(0);
        }
        if (RES) {
            g_ref = g_chk = RT(0);
            acc_ref = acc_chk = 0.0;
        }
        int issued = 0;  // chunks whose load was issued
        {
            const int first = n_chunks < STAGES ? n_chunks : STAGES;
            for (int c = 0; c < first; ++c) {
                if (!hk.ready(c)) return drain_after_timeout(bars, base, issued, 0);
                if (lane == 0) issue(c);
                ++issued;
            }
        }
        for (int c = 0; c < n_chunks; ++c) {
            const uint32_t g = base + static_cast<uint32_t>(c);
            const uint32_t slot = g % STAGES;
            // every lane waits (acquiring the TMA-written rows); the outcome is
            // made warp-uniform so no lane is left behind in a shuffle
            const bool ok = mbar_wait_bounded(&bars[slot], (g / STAGES) & 1u, timeout_ns);
            if (!__all_sync(FULL_MASK, ok)) return drain_after_timeout(bars, base, issued, c);
            const int r0 = rb + c * CR;
            const ST *src = ring + slot * (CR * W) + lane * V;
            // Rows past the unit's last step are in the box (zero-filled past
            // the grid) and only produce rows that are never stored.
            const bool fast = (r0 >= K + 1) && (r0 + CR <= R) && (r0 - K >= y0) &&
                              (r0 + CR - K <= y1);
            // pointer arithmetic only: rows before 0 are never dereferenced
            ST *out = dst + (static_cast<ptrdiff_t>(r0) - K) * ld + (X + lane * V);
            // A reassociated unit's boundary-checked body differs from the fast
            // one only by a store predicate on the row: one body keeps the hot
            // code small (instruction cache).  Exact-order units keep both:
            // their checked body tests every level's row.
            constexpr bool ONE_BODY = SDFG_SCALED_ONE_BODY && sizeof(CT) == 4 && !EXACT;
            if constexpr (RING2) {
                // a centre row of some level may be row 0 or row R-1
                const bool edge = Hook::EDGES && (r0 <= K || (r0 + CR - 2 >= R - 1 && r0 - K <= R - 1));
                // every output row of the chunk stored (the common case): a
                // third body without the per-row test, for BF16 chains only
                // (measured: BF16 +3%; FP32 chains -22% and the persistent
                // kernel -6%, whose larger hot code it pushes out of the
                // instruction cache)
                constexpr bool ALL_BODY = SDFG_RING2_ALL_BODY && sizeof(ST) == 2 && Hook::EDGES;
                const bool all = ALL_BODY && (r0 - K >= sy0) && (r0 + CR - 1 - K < sy1);
                if (edge)
                    chunk_body2<true, Hook::TURN>(r0, src, out);
                else if (all)
                    chunk_body2<false, Hook::TURN, true>(r0, src, out);
                else
                    chunk_body2<false, Hook::TURN>(r0, src, out);
            } else if (fast && !ONE_BODY) {
                chunk_body<false>(r0, src, out);
            } else {
                chunk_body<true>(r0, src, out);
            }
            // every lane has consumed chunk c (and stored its rows): recycle its slot
            __syncwarp();
            hk.done(c);
            if (c + STAGES < n_chunks) {
                if (!hk.ready(c + STAGES)) return drain_after_timeout(bars, base, issued, c + 1);
                if (lane == 0) issue(c + STAGES);
                ++issued;
            }
            if (RES) {
                acc_ref += static_cast<double>(g_ref);
                acc_chk += static_cast<double>(g_chk);
                g_ref = RT(0);
                g_chk = RT(0);
            }
        }
        return true;
    }
};

// Process unit (strip, seg) of grid `g`: read through tensor map `tmap`
// (source buffer), write `dst`.  res_flags bit 0: accumulate the squared
// level-1 update (the first step of a solve), bit 1: the squared level-K
// update (a check step).  Returns false if a TMA wait ran out.
template <class ST, int V, int K>
__device__ __forceinline__ bool run_unit(const void *tmap, ST *dst, const GridGeo &g, int strip, int seg, ST *ring,
                                         uint64_t *bars, uint32_t &chunk_ctr, int res_flags, double2 *partial,
                                         unsigned long long timeout_ns) {
    constexpr int W = 32 * V;
    const int lane = threadIdx.x & 31;
    const int X = strip * g.wout - g.h;
    const int y0 = seg * g.H;
    const int y1 = min(y0 + g.H, g.R);
    const int rb = max(0, y0 - K);
    const int n_steps = y1 + K - rb;
    const int n_chunks = (n_steps + CHUNK_ROWS - 1) / CHUNK_ROWS;
    const int gc0 = X + lane * V;
    const int hl = g.h / V;

    unsigned colmask = 0, resmask = 0;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int gc = gc0 + e;
        if (gc <= 0 || gc >= g.C - 1) colmask |= 1u << e;
        if (gc >= 1 && gc <= g.C - 2) resmask |= 1u << e;
    }
    const bool own_lane = lane >= hl && lane < 32 - hl && gc0 < g.C;
    if (!own_lane) resmask = 0;
    const bool full_vec = gc0 + V <= g.C;
    const bool colchk = (X <= 0) || (X + W > g.C - 1);

    bool ok;
    double ar = 0.0, ac = 0.0;
#define SDFG_RUN_PIPE(CHK, RS, EX)                                                                          \
    {                                                                                                   \
        UnitPipe<ST, V, K, CHK, RS, EX> p;                                                                  \
        p.tmap = tmap; p.dst = dst; p.ld = g.ld; p.R = g.R; p.C = g.C;                                  \
        p.X = X; p.y0 = y0; p.y1 = y1; p.rb = rb; p.n_steps = n_steps; p.n_chunks = n_chunks;           \
        p.sy0 = y0; p.sy1 = y1;                                                                         \
        p.base = chunk_ctr; p.ring = ring; p.bars = bars; p.lane = lane;                                \
        p.colmask = colmask; p.resmask = resmask; p.own_lane = own_lane; p.full_vec = full_vec;         \
        p.res_flags = res_flags; p.timeout_ns = timeout_ns;                                             \
        ok = p.run();                                                                                   \
        if (RS) { ar = p.acc_ref; ac = p.acc_chk; }                                                     \
    }
    // rows rb .. y1+K-1 are read: a boundary row is among them in the first
    // and the last segments
    const bool rowedge = (rb <= 0) || (y1 + K - 1 >= g.R - 1);
    if (res_flags) {
        if (colchk) SDFG_RUN_PIPE(true, true, true)
        else if (rowedge) SDFG_RUN_PIPE(false, true, true)
        else SDFG_RUN_PIPE(false, true, false)
    } else {
        if (colchk) SDFG_RUN_PIPE(true, false, true)
        else if (rowedge) SDFG_RUN_PIPE(false, false, true)
        else SDFG_RUN_PIPE(false, false, false)
    }
#undef SDFG_RUN_PIPE
    chunk_ctr += static_cast<uint32_t>(n_chunks);

    if (res_flags && partial) {
        // fixed-order butterfly; lane 0's value is used
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            ar += __shfl_xor_sync(FULL_MASK, ar, off);
            ac += __shfl_xor_sync(FULL_MASK, ac, off);
        }
        if (lane == 0) *partial = make_double2(ar, ac);
    }
    return ok;
}

}  // namespace sdfg
