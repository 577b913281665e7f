// Internal helpers shared by the library's translation units: error reporting, the
// allocation hook, the sticky device status word, and small inline-PTX wrappers
// (packed FP32 pairs, bulk global->shared copies completed on an mbarrier).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <utility>

#include "../../include/spiir.h"

namespace spiir {

int fail(int code, const char *fmt, ...);  // records the message, returns code
void clear_error();

// Device allocation through the test hook (spiir_debug_fail_allocs).
int dev_alloc(void **p, size_t bytes, const char *what);
void dev_free(void *p);
int host_alloc_pinned(void **p, size_t bytes, const char *what);
void host_free_pinned(void *p);

// Sticky status word of the current device (a file-scope device variable; nothing is
// allocated).  NULL if its address cannot be found.
int *device_status_word();

// Raise a kernel's dynamic shared-memory limit to `bytes`, once per (device, kernel, bytes);
// safe to call from several host threads.
int set_max_dyn_smem(const void *func, int bytes);
// Resident blocks per SM of a kernel at a launch shape, cached per (device, kernel, shape).
int resident_blocks_per_sm(const void *func, int threads, size_t smem, int *out);

// Maximum iterations of any bounded device-side wait before it gives up.
constexpr uint32_t kWaitLimit = 1u << 26;
constexpr int kStatusTimeout = 1;

#define SPIIR_CUDA_TRY(call)                                                                \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::spiir::fail(SPIIR_ECUDA, "%s failed: %s (%s:%d)", #call,               \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);               \
    } while (0)

#define SPIIR_TRY(expr)                  \
    do {                                 \
        int rc_ = (expr);                \
        if (rc_ != SPIIR_OK) return rc_; \
    } while (0)

// ---------------------------------------------------------------------------------------
// Device helpers

typedef unsigned long long u64;

__device__ __forceinline__ u64 pack2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpack2(u64 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
// Packed pair arithmetic: two independent IEEE FP32 operations, round to nearest.
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 neg2(u64 a) { return a ^ 0x8000000080000000ull; }

// Programmatic dependent launch.  A kernel launched with launch_dependent() may be scheduled
// before the previous kernel on its stream has completed; it calls grid_dependency_wait()
// before it reads anything that kernel wrote (without the launch attribute the wait returns at
// once).  grid_dependents_trigger() lets the stream's next dependent launch be scheduled once
// every block of this grid has called it or exited.
__device__ __forceinline__ void grid_dependents_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                           cudaStream_t stream, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One elected thread: announce the byte count and start a bulk copy global -> shared.
// dst and src 16-byte aligned, bytes a multiple of 16 and below 2^20.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for the given phase parity of an mbarrier.  Returns false when the
// iteration limit ran out (the caller records a timeout and leaves).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    uint32_t ok = 0;
    for (uint32_t it = 0; it < limit; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 "
            "%0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void report_timeout(int *status) {
    if (status) atomicOr(status, kStatusTimeout);
}

// Debug build only: record the first out-of-range index (code in the status word's upper bits).
constexpr int kStatusBounds = 4;
__device__ __forceinline__ void report_bounds(int *status, int code) {
    if (status) atomicOr(status, kStatusBounds | (code << 8));
}

}  // namespace spiir
