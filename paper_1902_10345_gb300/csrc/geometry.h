// Work decomposition shared by host planning code and the kernels.
#pragma once

namespace sdfg {

#ifndef SDFG_CHUNK_ROWS
#define SDFG_CHUNK_ROWS 12
#endif
#ifndef SDFG_STAGES
#define SDFG_STAGES 2
#endif
constexpr int CHUNK_ROWS = SDFG_CHUNK_ROWS;  // rows per TMA box (a multiple of the 3-row register rotation)
constexpr int STAGES = SDFG_STAGES;          // TMA ring depth per warp
static_assert(CHUNK_ROWS % 3 == 0, "chunks are whole turns of the 3-row rotation");

// The chain kernels (skewed.cu, chain_batch.cu) stream taller chunks: 18
// rows for 4- and 8-byte storage (three CTAs' TMA rings still fit in an SM's
// shared memory), 24 for 2-byte storage (measured best for each).  Their
// progress is published every ~144 rows.
#ifndef SDFG_CHAIN_CHUNK_ROWS_4
#define SDFG_CHAIN_CHUNK_ROWS_4 18
#endif
#ifndef SDFG_CHAIN_CHUNK_ROWS_2
#define SDFG_CHAIN_CHUNK_ROWS_2 24
#endif
#ifndef SDFG_CHAIN_PUB_ROWS
#define SDFG_CHAIN_PUB_ROWS 144
#endif
#ifdef __CUDACC__
#define SDFG_HD __host__ __device__
#else
#define SDFG_HD
#endif
SDFG_HD constexpr int chain_chunk_rows(int elem_bytes) {
    return elem_bytes == 2 ? SDFG_CHAIN_CHUNK_ROWS_2 : SDFG_CHAIN_CHUNK_ROWS_4;
}
// default chunks between two progress updates of a chain
SDFG_HD constexpr int chain_pub_chunks(int elem_bytes) {
    return SDFG_CHAIN_PUB_ROWS / chain_chunk_rows(elem_bytes) > 0 ? SDFG_CHAIN_PUB_ROWS / chain_chunk_rows(elem_bytes)
                                                                  : 1;
}
static_assert(chain_chunk_rows(2) % 6 == 0 && chain_chunk_rows(4) % 6 == 0, "chain chunks are whole 6-row turns");
constexpr int MAX_WARPS = 16;  // warps per CTA upper bound

// L2 promotion (bytes) of the 2-D tensor maps the streamed kernels load rows
// through: a strip's row (512 B) starts 32 B before a 256-B boundary, so
// 256-B promotion fetches three blocks for it; 64-B promotion measured 0.3%
// faster on 8192^2 (5710 against 5691 GUpdates/s), 128 B and none in between.
#ifndef SDFG_TMA2D_L2_PROMO
#define SDFG_TMA2D_L2_PROMO 64
#endif
constexpr int TMA2D_L2_PROMO = SDFG_TMA2D_L2_PROMO;

// Codes a kernel writes to the per-device error word (first writer wins).
constexpr int DEV_ERR_TIMEOUT_TMA = 1;  // an mbarrier wait for a TMA chunk ran out
constexpr int DEV_ERR_TIMEOUT_DEP = 2;  // a dependency wait (persistent kernel) ran out

// One grid cut into units of (strip, segment): strip s covers output columns
// [s*wout, (s+1)*wout), segment q covers output rows [q*H, (q+1)*H).  A warp
// loads columns [s*wout - h, s*wout - h + 32*V) (h halo columns per side).
struct GridGeo {
    int R, C, ld;   // rows, cols, pitch (elements)
    int h;          // halo columns per side
    int wout;       // output columns per strip (32*V - 2h)
    int n_strips;   // ceil(C / wout)
    int H;          // output rows per segment
    int n_segs;     // ceil(R / H)
};

#ifndef SDFG_F32_V
#define SDFG_F32_V 4  // FP32 columns per lane (the two-row reassociated pipe needs 4)
#endif

// Columns per lane for a storage size in bytes: FP32 SDFG_F32_V, BF16 4, FP64 2.
inline int lane_cols(int elem_bytes) { return elem_bytes == 8 ? 2 : (elem_bytes == 4 ? SDFG_F32_V : 4); }

// TMA x alignment in elements (16 bytes).
inline int tma_xalign(int elem_bytes) { return 16 / elem_bytes; }

}  // namespace sdfg
