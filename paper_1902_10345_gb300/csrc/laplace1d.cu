// The 1-D Laplace program of the paper's Fig. 1 on the GPU:
//   for t in range(T): for i in map[1:N-1]:
//       A[(t+1)%2, i] = A[t%2, i-1:i+2] * [1, -2, 1]      (A: float64[2, N])
// Each row's two end cells are never written, so a step reading row r sees
// row r's own ends.  The array is updated in place exactly as the program
// leaves it (both rows).  FP64, in the program's order: (a - 2b) + c.
#include <algorithm>

#include "runtime.h"

namespace sdfg {

__device__ __forceinline__ double fig1_point(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(a * 1.0, b * -2.0), c * 1.0);
}

// Whole problem in one CTA's shared memory (2N doubles): T steps with a
// barrier between steps, then both rows back to HBM.
__global__ void __launch_bounds__(1024) laplace1d_smem_kernel(double *__restrict__ A, int N, int T) {
    extern __shared__ double rows[];  // [2][N]
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) rows[i] = A[i];
    __syncthreads();
    for (int t = 0; t < T; ++t) {
        const double *src = rows + (t & 1) * N;
        double *dst = rows + ((t + 1) & 1) * N;
        for (int i = 1 + threadIdx.x; i < N - 1; i += blockDim.x) dst[i] = fig1_point(src[i - 1], src[i], src[i + 1]);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) A[i] = rows[i];
}

// One step over HBM (large N).
__global__ void __launch_bounds__(256) laplace1d_step_kernel(double *__restrict__ A, int N, int t) {
    const double *src = A + static_cast<size_t>(t & 1) * N;
    double *dst = A + static_cast<size_t>((t + 1) & 1) * N;
    for (int i = 1 + blockIdx.x * blockDim.x + threadIdx.x; i < N - 1; i += gridDim.x * blockDim.x)
        dst[i] = fig1_point(src[i - 1], src[i], src[i + 1]);
}

}  // namespace sdfg

using namespace sdfg;

extern "C" int sdfg_laplace1d(double *A, int N, int T, void *stream) {
    if (N < 0 || T < 0) return set_error(SDFG_ERR_INVAL, "sdfg_laplace1d: N=%d T=%d must be >= 0", N, T);
    if (N == 0 || T == 0 || N < 3) return SDFG_OK;
    if (!A) return set_error(SDFG_ERR_INVAL, "sdfg_laplace1d: null array");
    DeviceState *st = nullptr;
    int rc = current_device(&st);
    if (rc != SDFG_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = static_cast<size_t>(2) * N * sizeof(double);
    int max_smem = 0;
    SDFG_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, st->device));
    TimedLaunch tl = stats_begin(FAM_NAIVE, s);
    if (smem <= static_cast<size_t>(max_smem)) {
        SDFG_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(&laplace1d_smem_kernel),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        laplace1d_smem_kernel<<<1, 1024, smem, s>>>(A, N, T);
        SDFG_CUDA(cudaGetLastError());
    } else {
        const int blocks = std::min((N + 255) / 256, st->sm_count * 8);
        for (int t = 0; t < T; ++t) {
            laplace1d_step_kernel<<<blocks, 256, 0, s>>>(A, N, t);
            SDFG_CUDA(cudaGetLastError());
        }
    }
    stats_end(tl, s);
    return SDFG_OK;
}
