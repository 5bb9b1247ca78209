// Host runtime: errors, device state, tensor maps, scratch, planning, timing.
#include "runtime.h"

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>

namespace sdfg {

// ---------------------------------------------------------------- errors ------
static thread_local std::string g_last_error;

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    const int code = (e == cudaErrorMemoryAllocation) ? SDFG_ERR_NOMEM : SDFG_ERR_CUDA;
    return set_error(code, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_last_error.clear(); }

// ---------------------------------------------------------- device state ------
static std::mutex g_dev_mu;
static DeviceState g_dev[64];

int current_device(DeviceState **st) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(SDFG_ERR_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceState &d = g_dev[dev];
    if (d.device < 0) {
        SDFG_CUDA(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
        SDFG_CUDA(cudaDeviceGetAttribute(&d.major, cudaDevAttrComputeCapabilityMajor, dev));
        SDFG_CUDA(cudaDeviceGetAttribute(&d.minor, cudaDevAttrComputeCapabilityMinor, dev));
        d.arch_ok = (d.major == 10 && d.minor == 3);
        if (d.arch_ok) {
            SDFG_CUDA(cudaMalloc(&d.d_err, sizeof(int)));
            SDFG_CUDA(cudaMemset(d.d_err, 0, sizeof(int)));
            // keep freed scratch in the device's default pool between calls
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
        }
        d.device = dev;
    }
    if (!d.arch_ok)
        return set_error(SDFG_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a only", dev,
                         d.major, d.minor);
    *st = &d;
    return SDFG_OK;
}

// ------------------------------------------------------------------- TMA ------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

static CUtensorMapL2promotion l2_promotion(int bytes) {
    return bytes == 64    ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
           : bytes == 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
           : bytes == 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                          : CU_TENSOR_MAP_L2_PROMOTION_NONE;
}

int encode_tmap(CUtensorMap *tm, const void *base, int dtype, int rows, int cols, int ld, int box_cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(SDFG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const CUtensorMapDataType t = dtype == SDFG_F64    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                  : dtype == SDFG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * dtype_bytes(dtype)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, t, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, l2_promotion(TMA2D_L2_PROMO),
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(SDFG_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for %dx%d ld=%d", static_cast<int>(r),
                         rows, cols, ld);
    return SDFG_OK;
}


int encode_tmap3d(CUtensorMap *tm, const void *base, int dtype, int depth, int rows, int cols, int ld, int box_cols,
                  int box_rows, int l2_promo) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(SDFG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const CUtensorMapDataType t = dtype == SDFG_F64    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                  : dtype == SDFG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t S = static_cast<cuuint64_t>(dtype_bytes(dtype));
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows),
                                static_cast<cuuint64_t>(depth)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * S, static_cast<cuuint64_t>(ld) * rows * S};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(tm, t, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, l2_promotion(l2_promo),
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(SDFG_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (%d) for %dx%dx%d ld=%d",
                         static_cast<int>(r), depth, rows, cols, ld);
    return SDFG_OK;
}

// --------------------------------------------------------------- scratch ------
int scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) return SDFG_OK;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(SDFG_ERR_NOMEM, "scratch allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return SDFG_OK;
}

void scratch_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// -------------------------------------------------------------- planning ------
bool depth_supported(int k) { return k == 1 || k == 2 || k == 4 || k == 8; }

int default_depth(int dtype) { return dtype == SDFG_F64 ? 4 : 8; }

static int gcd_i(int a, int b) { return b ? gcd_i(b, a % b) : a; }

GridGeo plan_geometry(int rows, int cols, int ld, int dtype, int k, int seg_rows, long long target_units) {
    GridGeo g;
    const int S = dtype_bytes(dtype);
    const int V = lane_cols(S);
    const int W = 32 * V;
    const int xa = tma_xalign(S);
    const int align = V / gcd_i(V, xa) * xa;
    g.R = rows;
    g.C = cols;
    g.ld = ld;
    g.h = ((std::max(k, 1) + align - 1) / align) * align;
    g.wout = W - 2 * g.h;
    g.n_strips = std::max(1, (cols + g.wout - 1) / g.wout);
    int H = seg_rows;
    if (H <= 0) {
        long long segs = target_units > 0 ? (target_units + g.n_strips / 2) / g.n_strips : 1;
        segs = std::max<long long>(1, segs);
        H = static_cast<int>((rows + segs - 1) / segs);
        H = std::max(H, 2 * std::max(k, 1));
        H = std::max(H, 16);
    }
    // a unit's input rows (k above and below its own) must lie within the
    // segments next to its own: the persistent kernel waits on those alone
    H = std::max(H, std::max(k, 1));
    g.H = std::max(1, std::min(H, std::max(rows, 1)));
    g.n_segs = std::max(1, (rows + g.H - 1) / g.H);
    return g;
}

std::vector<int> plan_passes(long long T, int k) {
    std::vector<int> p;
    if (T <= 0) return p;
    const long long full = T / k;
    p.assign(static_cast<size_t>(full), k);
    long long rem = T - full * k;  // < k <= 8
    for (int d = 8; d >= 1; d >>= 1)
        while (rem >= d) {
            p.push_back(d);
            rem -= d;
        }
    return p;
}

// ------------------------------------------------------------------ stats -----
namespace {
struct Rec {
    int family;
    cudaEvent_t a, b;
};
std::mutex g_stats_mu;
bool g_stats_on = false;
std::vector<Rec> g_recs;
const char *kFamilies[FAM_COUNT] = {"naive", "temporal", "persistent", "reduce", "copy",   "stencil3d",
                                    "sor",   "resident", "skewed",     "h2d",    "d2h"};
}  // namespace

static thread_local bool g_stats_suspended = false;

void stats_suspend(bool on) { g_stats_suspended = on; }

TimedLaunch stats_begin(int family, cudaStream_t s) {
    TimedLaunch t;
    if (g_stats_suspended) return t;
    {
        std::lock_guard<std::mutex> lk(g_stats_mu);
        if (!g_stats_on) return t;
    }
    if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) {
        cudaGetLastError();
        return TimedLaunch();
    }
    cudaEventRecord(t.a, s);
    t.family = family;
    return t;
}

void stats_end(TimedLaunch &t, cudaStream_t s) {
    if (!t.active()) return;
    cudaEventRecord(t.b, s);
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_recs.push_back(Rec{t.family, t.a, t.b});
    t.family = -1;
}

}  // namespace sdfg

using namespace sdfg;

extern "C" int sdfg_stats_enable(int on) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_stats_on = on != 0;
    return SDFG_OK;
}

extern "C" int sdfg_stats_reset(void) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    for (Rec &r : g_recs) {
        cudaEventSynchronize(r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
    return SDFG_OK;
}

extern "C" int sdfg_stats_get(const char *name, long long *launches, double *total_ms) {
    if (!name || !launches || !total_ms) return set_error(SDFG_ERR_INVAL, "sdfg_stats_get: null argument");
    int fam = -1;
    for (int i = 0; i < FAM_COUNT; ++i)
        if (strcmp(name, kFamilies[i]) == 0) fam = i;
    if (fam < 0) return set_error(SDFG_ERR_INVAL, "sdfg_stats_get: unknown kernel family '%s'", name);
    std::lock_guard<std::mutex> lk(g_stats_mu);
    long long n = 0;
    double ms = 0.0;
    for (Rec &r : g_recs) {
        if (r.family != fam) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_error(e, "cudaEventSynchronize");
        float x = 0.f;
        e = cudaEventElapsedTime(&x, r.a, r.b);
        if (e != cudaSuccess) return cuda_error(e, "cudaEventElapsedTime");
        ms += x;
        ++n;
    }
    *launches = n;
    *total_ms = ms;
    return SDFG_OK;
}

namespace sdfg {
int noalloc_error_word(int dev, int clear, int *value);  // noalloc.cu
}

// Reads the current device's error words: the one of every allocating entry
// point (only if this device was already set up: a call here creates no
// device state) and the one of sdfg_jacobi2d_noalloc.
extern "C" int sdfg_device_error(int clear) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(SDFG_ERR_UNSUPPORTED, "device index %d out of range", dev);
    int *word = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        if (g_dev[dev].device >= 0 && g_dev[dev].arch_ok) word = g_dev[dev].d_err;
    }
    int v = 0;
    if (word) {
        SDFG_CUDA(cudaMemcpy(&v, word, sizeof(int), cudaMemcpyDeviceToHost));
        if (clear && v) SDFG_CUDA(cudaMemset(word, 0, sizeof(int)));
    }
    int w = 0;
    const int rc = noalloc_error_word(dev, clear, &w);
    if (rc != SDFG_OK) return rc;
    if (!v) v = w;
    if (v == DEV_ERR_TIMEOUT_TMA || v == DEV_ERR_TIMEOUT_DEP) return SDFG_ERR_TIMEOUT;
    return v == 0 ? SDFG_OK : SDFG_ERR_CUDA;
}

extern "C" const char *sdfg_last_error(void) { return g_last_error.c_str(); }

extern "C" int sdfg_version(void) { return 100; }

extern "C" int sdfg_plan_geometry(int rows, int cols, int dtype, int k, int seg_rows, int *info) {
    if (!info || rows < 0 || cols < 0 || !dtype_valid(dtype) || !depth_supported(k) || seg_rows < 0)
        return set_error(SDFG_ERR_INVAL, "sdfg_plan_geometry: bad argument");
    const GridGeo g = plan_geometry(rows, cols, cols, dtype, k, seg_rows, 0);
    info[0] = g.h;
    info[1] = 32 * lane_cols(dtype_bytes(dtype));
    info[2] = g.wout;
    info[3] = g.n_strips;
    info[4] = g.H;
    info[5] = g.n_segs;
    info[6] = CHUNK_ROWS;
    info[7] = STAGES;
    return SDFG_OK;
}
