// Host-side runtime shared by every entry point: error reporting, per-device
// state, tensor-map encoding, stream-ordered scratch, launch timing, and the
// kernel launchers exported by kernels.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/sdfg_jacobi.h"
#include "geometry.h"

namespace sdfg {

// ---- errors ------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);    // records a thread-local message, returns code
int cuda_error(cudaError_t e, const char *what);  // SDFG_ERR_CUDA (or NOMEM) with the CUDA message
void clear_error();

#define SDFG_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::sdfg::cuda_error(e_, #call); \
    } while (0)

// ---- device state ------------------------------------------------------------
struct DeviceState {
    int device = -1;
    int sm_count = 0;
    int major = 0, minor = 0;
    bool arch_ok = false;
    int *d_err = nullptr;  // device error word (first failing code)
};
// State of the current device, created on first use.  Fails with
// SDFG_ERR_UNSUPPORTED when the device is not an sm_103 part.
int current_device(DeviceState **st);

// ---- dtype -------------------------------------------------------------------
inline bool dtype_valid(int dt) { return dt == SDFG_F32 || dt == SDFG_BF16 || dt == SDFG_F64; }
inline int dtype_bytes(int dt) { return dt == SDFG_F64 ? 8 : (dt == SDFG_BF16 ? 2 : 4); }

// ---- TMA ---------------------------------------------------------------------
// 2-D tensor map over a rows x cols grid with pitch ld; box = box_cols x
// box_rows (CHUNK_ROWS by default); out-of-range elements read as zero.
int encode_tmap(CUtensorMap *tm, const void *base, int dtype, int rows, int cols, int ld, int box_cols,
                int box_rows = CHUNK_ROWS);
// Rank-3 map over a depth x rows x cols box (row pitch ld elements, plane
// pitch rows*ld): boxes of box_cols x box_rows x 1; l2_promo: L2 promotion
// in bytes (0, 64, 128 or 256).
int encode_tmap3d(CUtensorMap *tm, const void *base, int dtype, int depth, int rows, int cols, int ld, int box_cols,
                  int box_rows, int l2_promo = 256);
// True when a buffer can be read by TMA as laid out.
inline bool tma_compatible(const void *p, int ld, int dtype) {
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((static_cast<long long>(ld) * dtype_bytes(dtype)) % 16 == 0);
}

// ---- stream-ordered scratch --------------------------------------------------
int scratch_alloc(void **p, size_t bytes, cudaStream_t s);
void scratch_free(void *p, cudaStream_t s);

// ---- planning ----------------------------------------------------------------
// Geometry of a grid for fused depth k (halo >= k).  seg_rows 0 = automatic,
// aiming at `target_units` units; segments are at least k rows high.
GridGeo plan_geometry(int rows, int cols, int ld, int dtype, int k, int seg_rows, long long target_units);
// Pass depths for T steps at main depth k: k, k, ..., then the remainder in
// powers of two (largest first).
std::vector<int> plan_passes(long long T, int k);
bool depth_supported(int k);
int default_depth(int dtype);

// ---- launch timing (sdfg_stats_*) ---------------------------------------------
struct TimedLaunch {
    cudaEvent_t a = nullptr, b = nullptr;
    int family = -1;
    bool active() const { return family >= 0; }
};
enum Family {
    FAM_NAIVE = 0,
    FAM_TEMPORAL,
    FAM_PERSISTENT,
    FAM_REDUCE,
    FAM_COPY,
    FAM_STENCIL3D,
    FAM_SOR,
    FAM_RESIDENT,
    FAM_SKEWED,
    FAM_H2D,  // host -> device copies of sdfg_jacobi2d_host
    FAM_D2H,  // device -> host copies of sdfg_jacobi2d_host
    FAM_COUNT
};
TimedLaunch stats_begin(int family, cudaStream_t s);
// No launch is timed on this thread while suspended (stream capture).
void stats_suspend(bool on);
void stats_end(TimedLaunch &t, cudaStream_t s);

// ---- kernel launchers (kernels.cu) -------------------------------------------
constexpr unsigned long long DEFAULT_TIMEOUT_NS = 2000000000ull;  // 2 s per wait

int launch_naive_step(const void *A, void *B, int rows, int cols, int ld, int dtype, cudaStream_t s);
int launch_temporal_pass(const CUtensorMap *tm_src, void *dst, const GridGeo &g, int dtype, int k, int warps,
                         int res_flags, double2 *partials, int *err, unsigned long long timeout_ns,
                         cudaStream_t s);
// CTAs of `warps` warps resident per SM for the temporal kernel.
int temporal_blocks_per_sm(int dtype, int k, int warps);
size_t temporal_smem_bytes(int dtype, int warps);
int launch_copy2d(void *dst, int ld_dst, const void *src, int ld_src, int rows, int cols, int dtype, cudaStream_t s);

// ---- register-resident passes (resident.cu) ----------------------------------
bool resident_supported(int dtype);
// T steps as passes of k (1..8) and one pass for the remainder.
std::vector<int> plan_resident_passes(long long T, int k);
// The passes `ks` (each 1..8 steps) from src0, alternating between `first`
// and `second`; *final receives the buffer holding the result.
int run_resident_passes(const void *src0, void *first, void *second, const std::vector<int> &ks, int R, int C,
                        int ld, int dtype, DeviceState *st, cudaStream_t s, void **final);

// ---- skewed chains (skewed.cu) ------------------------------------------------
// T steps of one grid in one launch of the chain kernel: passes of depth k,
// chains of L rows (0: 512), progress published every `pub` chunks (0: 12).
// in/out must be TMA-compatible; in == out allowed.
int run_single_chain(const void *in, void *out, int R, int C, int ld, long long T, int dtype, int k, int L, int pub,
                     DeviceState *st, cudaStream_t s);

}  // namespace sdfg
