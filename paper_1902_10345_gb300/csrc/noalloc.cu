// sdfg_jacobi2d_noalloc: the single-grid FP32 solve with its ping-pong
// scratch grid in a fixed, file-scope device array instead of memory the
// library allocates.  For callers that must not allocate device memory.
//
// The array's name is a host-side stand-in, not a device address: host code
// gets the address with cudaGetSymbolAddress, once per device with that
// device current, and passes it to the kernels.
#include <mutex>

#include "runtime.h"

namespace sdfg {

constexpr size_t NOALLOC_MAX_ELEMS = size_t(8) << 20;  // 8 Mi floats = 32 MiB

// The scratch grid, resident on every GPU that loads the library until exit.
// No element needs a starting value: every pass writes each element of the
// grid before any later pass reads it.
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_MAX_ELEMS];
// Error word for the kernels launched from this entry point.
static __device__ __align__(16) int g_noalloc_err[4];

int run_single_with_scratch(const void *in, void *out, void *scratch, int R, int C, int ld, long long T, int dtype,
                            const sdfg_config *cfg, DeviceState *st, cudaStream_t s);

namespace {
struct NoallocDevice {
    bool ready = false;
    DeviceState st;         // built without allocating
    void *scratch = nullptr;
};
std::mutex g_mu;
NoallocDevice g_dev[64];

// Once per device, with that device current: resolve the device addresses of
// the static arrays.  Allocates nothing.
int noalloc_setup(NoallocDevice **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(SDFG_ERR_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    NoallocDevice &d = g_dev[dev];
    if (!d.ready) {
        int major = 0, minor = 0, sms = 0;
        SDFG_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
        SDFG_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
        SDFG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (!(major == 10 && minor == 3))
            return set_error(SDFG_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a only", dev,
                             major, minor);
        void *scratch = nullptr;
        void *err = nullptr;
        e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
        e = cudaGetSymbolAddress(&err, g_noalloc_err);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(error word)");
        d.st.device = dev;
        d.st.sm_count = sms;
        d.st.major = major;
        d.st.minor = minor;
        d.st.arch_ok = true;
        d.st.d_err = static_cast<int *>(err);
        d.scratch = scratch;
        d.ready = true;
    }
    *out = &d;
    return SDFG_OK;
}
}  // namespace

// The error word of the kernels launched by sdfg_jacobi2d_noalloc on device
// `dev` (read with cudaMemcpyFromSymbol, reset with cudaMemcpyToSymbol when
// `clear`): *value = 0 when nothing was recorded, or when the entry point was
// never set up on that device (then the symbol is not touched, so reading the
// word never loads this file's module and its static scratch).  Allocates
// nothing.  Synchronous: waits for the work already on the device.
int noalloc_error_word(int dev, int clear, int *value) {
    *value = 0;
    if (dev < 0 || dev >= 64) return SDFG_OK;
    bool ready;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        ready = g_dev[dev].ready;
    }
    if (!ready) return SDFG_OK;
    int w = 0;
    SDFG_CUDA(cudaMemcpyFromSymbol(&w, g_noalloc_err, sizeof(int)));
    if (clear && w) {
        const int zero = 0;
        SDFG_CUDA(cudaMemcpyToSymbol(g_noalloc_err, &zero, sizeof(int)));
    }
    *value = w;
    return SDFG_OK;
}

}  // namespace sdfg

using namespace sdfg;

extern "C" int sdfg_jacobi2d_noalloc(const float *in, float *out, int rows, int cols, int T, void *stream) {
    if (rows < 0 || cols < 0 || T < 0)
        return set_error(SDFG_ERR_INVAL, "sdfg_jacobi2d_noalloc: rows=%d cols=%d T=%d must be >= 0", rows, cols, T);
    if (rows == 0 || cols == 0) {
        // an empty grid does only the per-device set-up (a warm-up call)
        NoallocDevice *d = nullptr;
        return noalloc_setup(&d);
    }
    if (!in || !out) return set_error(SDFG_ERR_INVAL, "sdfg_jacobi2d_noalloc: null grid pointer");
    if (static_cast<size_t>(rows) * static_cast<size_t>(cols) > NOALLOC_MAX_ELEMS)
        return set_error(SDFG_ERR_INVAL,
                         "sdfg_jacobi2d_noalloc: %d x %d grid exceeds the static scratch of %zu elements", rows, cols,
                         NOALLOC_MAX_ELEMS);
    if (!tma_compatible(in, cols, SDFG_F32) || !tma_compatible(out, cols, SDFG_F32))
        return set_error(SDFG_ERR_INVAL,
                         "sdfg_jacobi2d_noalloc: needs 16-byte aligned grids and cols a multiple of 4");
    const char *a = reinterpret_cast<const char *>(in);
    const char *b = reinterpret_cast<const char *>(out);
    const size_t span = static_cast<size_t>(rows) * cols * sizeof(float);
    if (a != b && a < b + span && b < a + span)
        return set_error(SDFG_ERR_INVAL, "sdfg_jacobi2d_noalloc: in and out overlap without being the same grid");
    NoallocDevice *d = nullptr;
    int rc = noalloc_setup(&d);
    if (rc != SDFG_OK) return rc;
    return run_single_with_scratch(in, out, d->scratch, rows, cols, cols, T, SDFG_F32, nullptr, &d->st,
                                   static_cast<cudaStream_t>(stream));
}
