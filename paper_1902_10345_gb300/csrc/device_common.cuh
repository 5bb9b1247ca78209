// Device-side building blocks shared by every kernel of the library:
// inline-PTX wrappers for mbarriers and TMA (cp.async.bulk.tensor), bounded
// waits, element load/convert/store helpers for the three storage types.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "geometry.h"

namespace sdfg {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false if `timeout_ns` elapsed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
}

// 2-D tiled TMA load of a box {x: inner, y: rows} into shared memory,
// completing `bytes` of transaction count on `bar`.
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 3-D box {x, y, z} of a rank-3 tensor map into shared memory.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const void *tmap, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmap_prefetch(const void *tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// Acquire a tensor map that lives in global memory (written before the launch).
__device__ __forceinline__ void tmap_acquire(const void *tmap) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tmap))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void set_device_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ----------------------------------------------------------------------------
// Storage-type traits: compute type, bytes, TMA x alignment (elements).
// ----------------------------------------------------------------------------
template <class ST> struct Store;

template <> struct Store<float> {
    using CT = float;
    static constexpr int bytes = 4;
    static constexpr int xalign = 4;   // 16 B / 4 B
};
template <> struct Store<__nv_bfloat16> {
    using CT = float;
    static constexpr int bytes = 2;
    static constexpr int xalign = 8;   // 16 B / 2 B
};
template <> struct Store<double> {
    using CT = double;
    static constexpr int bytes = 8;
    static constexpr int xalign = 2;   // 16 B / 8 B
};

// V consecutive elements <-> registers.
template <class ST, int V> struct VecIO;

template <> struct VecIO<float, 4> {
    __device__ __forceinline__ static void load(float (&d)[4], const float *p) {
        float4 v = *reinterpret_cast<const float4 *>(p);
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
    __device__ __forceinline__ static void store(float *p, const float (&s)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(s[0], s[1], s[2], s[3]);
    }
};

template <> struct VecIO<float, 8> {
    __device__ __forceinline__ static void load(float (&d)[8], const float *p) {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
        d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
    }
    __device__ __forceinline__ static void store(float *p, const float (&s)[8]) {
        reinterpret_cast<float4 *>(p)[0] = make_float4(s[0], s[1], s[2], s[3]);
        reinterpret_cast<float4 *>(p)[1] = make_float4(s[4], s[5], s[6], s[7]);
    }
};

template <> struct VecIO<__nv_bfloat16, 4> {
    __device__ __forceinline__ static void load(float (&d)[4], const __nv_bfloat16 *p) {
        uint2 u = *reinterpret_cast<const uint2 *>(p);
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&u.x);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        d[0] = fa.x; d[1] = fa.y; d[2] = fb.x; d[3] = fb.y;
    }
    __device__ __forceinline__ static void store(__nv_bfloat16 *p, const float (&s)[4]) {
        // values are already BF16-representable: the conversion is exact
        __nv_bfloat162 a = __floats2bfloat162_rn(s[0], s[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(s[2], s[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};

template <> struct VecIO<double, 2> {
    __device__ __forceinline__ static void load(double (&d)[2], const double *p) {
        double2 v = *reinterpret_cast<const double2 *>(p);
        d[0] = v.x; d[1] = v.y;
    }
    __device__ __forceinline__ static void store(double *p, const double (&s)[2]) {
        *reinterpret_cast<double2 *>(p) = make_double2(s[0], s[1]);
    }
};

// Predicated vector stores (one instruction, no branch): write V elements at
// p when `pred` is non-zero.
__device__ __forceinline__ void store_pred(float *p, const float (&s)[4], int pred) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t"
        "@q st.global.v4.f32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
        "f"(s[0]), "f"(s[1]), "f"(s[2]), "f"(s[3]), "r"(pred)
        : "memory");
}
__device__ __forceinline__ void store_pred(float *p, const float (&s)[8], int pred) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %9, 0;\n\t"
        "@q st.global.v4.f32 [%0], {%1, %2, %3, %4};\n\t"
        "@q st.global.v4.f32 [%0+16], {%5, %6, %7, %8};\n\t}" ::"l"(p),
        "f"(s[0]), "f"(s[1]), "f"(s[2]), "f"(s[3]), "f"(s[4]), "f"(s[5]), "f"(s[6]), "f"(s[7]), "r"(pred)
        : "memory");
}
__device__ __forceinline__ void store_pred(__nv_bfloat16 *p, const float (&s)[4], int pred) {
    __nv_bfloat162 a = __floats2bfloat162_rn(s[0], s[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(s[2], s[3]);
    const uint32_t ua = *reinterpret_cast<uint32_t *>(&a);
    const uint32_t ub = *reinterpret_cast<uint32_t *>(&b);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t"
        "@q st.global.v2.b32 [%0], {%1, %2};\n\t}" ::"l"(p),
        "r"(ua), "r"(ub), "r"(pred)
        : "memory");
}
__device__ __forceinline__ void store_pred(double *p, const double (&s)[2], int pred) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t"
        "@q st.global.v2.f64 [%0], {%1, %2};\n\t}" ::"l"(p),
        "d"(s[0]), "d"(s[1]), "r"(pred)
        : "memory");
}

template <class ST> __device__ __forceinline__ typename Store<ST>::CT to_ct(ST v);
template <> __device__ __forceinline__ float to_ct<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_ct<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double to_ct<double>(double v) { return v; }

template <class ST> __device__ __forceinline__ ST from_ct(typename Store<ST>::CT v);
template <> __device__ __forceinline__ float from_ct<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_ct<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ double from_ct<double>(double v) { return v; }

// The stencil expression for one point, in the library's fixed order:
// 0.2 * (c + ((n + s) + (w + e))), round-to-nearest, no contraction.
__device__ __forceinline__ float stencil_point(float c, float n, float s, float w, float e) {
    return __fmul_rn(0.2f, __fadd_rn(c, __fadd_rn(__fadd_rn(n, s), __fadd_rn(w, e))));
}
__device__ __forceinline__ double stencil_point(double c, double n, double s, double w, double e) {
    return __dmul_rn(0.2, __dadd_rn(c, __dadd_rn(__dadd_rn(n, s), __dadd_rn(w, e))));
}

// Round an FP32 value to the nearest BF16 (ties to even) and widen it back.
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

}  // namespace sdfg
