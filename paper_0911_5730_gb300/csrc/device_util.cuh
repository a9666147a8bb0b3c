// device_util.cuh - device helpers shared by the apply kernels: typed loads
// of the operator storage, mbarrier-completed bulk copies with bounded waits,
// and programmatic dependent launch.
#pragma once

#include <cstdlib>
#include <string>

#include "internal.h"

namespace bddc {

template <class T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

template <class T, class ACC> __device__ __forceinline__ ACC ld(const T *p) {
    return static_cast<ACC>(to_f<T>(*p));
}
template <> __device__ __forceinline__ double ld<double, double>(const double *p) { return *p; }

template <class T> struct Ops;
template <> struct Ops<double> {
    __host__ __device__ static const OpSet<double> &get(const DevLevel &L) { return L.f64; }
};
template <> struct Ops<float> {
    __host__ __device__ static const OpSet<float> &get(const DevLevel &L) { return L.f32; }
};
template <> struct Ops<__nv_bfloat16> {
    __host__ __device__ static const OpSet<__nv_bfloat16> &get(const DevLevel &L) { return L.b16; }
};


constexpr long kWaitPolls = 1L << 20;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The one arrival of the barrier's phase, announcing `bytes` of copies.
__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One bulk copy global -> shared completing `bytes` on the barrier (no arrival).
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
    mbar_expect(bar, bytes);
    bulk_copy(dst, src, bytes, bar);
}
__device__ __forceinline__ bool mbar_try(unsigned long long *bar, unsigned phase) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase) {
    for (long i = 0; i < kWaitPolls; ++i)
        if (mbar_try(bar, phase)) return true;
    return false;
}
// Wait for the phase of parity `phase` of the warp's barrier; false (after
// flagging) if the wait gave up.
__device__ __forceinline__ bool warp_wait_copy(unsigned long long *bar, int *err, int lane,
                                               unsigned phase = 0) {
    const bool ok = mbar_wait(bar, phase);
    if (__all_sync(0xffffffffu, ok)) return true;
    if (lane == 0 && err) atomicExch(err, 1);
    mbar_wait(bar, phase);   // bounded: let the copy in flight land before the warp exits
    return false;
}

__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

// Conversions between binary32 and binary64 (IEEE 754-2008, Sec. 5.4.2; the
// narrowing one rounds to nearest, ties to even) done with integer
// operations.  On this GPU the hardware conversion issues on the FP64 pipe,
// which retires two lanes per clock per SM; these use the integer pipes.
// Inputs outside the normal binary32 range (zero, subnormal, overflow,
// infinity, NaN) take the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    // exponent rebias 127 -> 1023; the 23 fraction bits become the top of 52
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ float f64_to_f32(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e < 897u || e > 1150u) return (float)d;    // result not a normal binary32
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;         // the 29 fraction bits dropped
    if (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) f += 1u;   // carries into the exponent
    return __uint_as_float(f);
}
template <class ACC> __device__ __forceinline__ ACC from_f64(double v);
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_f64<float>(double v) { return f64_to_f32(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }

// Programmatic dependent launch.  The kernels of the apply and of the PCG
// iteration are launched so that each may start while its predecessor in the
// stream drains.  pdl_wait() returns once the predecessor grid has completed
// and its writes are visible (at once for an ordinary launch), so a kernel
// reads nothing another kernel of the iteration writes before it, and every
// thread calls it before it exits; only setup-time data (factors, records) is
// read earlier.  pdl_trigger() lets the successor be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}


// Launch with programmatic stream serialisation (see pdl_wait); setting the
// environment variable BDDC_PDL=0 launches in plain stream order instead.
inline bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("BDDC_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Launch with (pdl) or without programmatic stream serialisation.
template <class... KArgs, class... Args>
inline void launch_k(bool pdl, void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (pdl && pdl_enabled()) ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, args...);
    if (e != cudaSuccess) {
        const char *name = nullptr;
        if (cudaFuncGetName(&name, reinterpret_cast<const void *>(k)) != cudaSuccess || !name) name = "?";
        throw Error(BDDC_E_CUDA, std::string("launch of ") + name + " (grid " + std::to_string(grid) +
                                     ", block " + std::to_string(block) + ", shared " + std::to_string(smem) +
                                     "): " + cudaGetErrorString(e));
    }
}

template <class... KArgs, class... Args>
inline void launch_pdl(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                       Args... args) {
    launch_k(true, k, grid, block, smem, s, args...);
}


}  // namespace bddc
