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
constexpr int MAX_WARPS = 16;  // warps per CTA upper bound

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
#define SDFG_F32_V 4  // FP32 columns per lane (4 or 8)
#endif

// Columns per lane for a storage size in bytes: FP32 SDFG_F32_V, BF16 4, FP64 2.
inline int lane_cols(int elem_bytes) { return elem_bytes == 8 ? 2 : (elem_bytes == 4 ? SDFG_F32_V : 4); }

// TMA x alignment in elements (16 bytes).
inline int tma_xalign(int elem_bytes) { return 16 / elem_bytes; }

}  // namespace sdfg
