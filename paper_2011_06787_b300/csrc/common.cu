// Error reporting, allocation hook and device status word of the C ABI.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>

#include "common.cuh"

namespace spiir {

static thread_local std::string g_last_error;
static std::atomic<int> g_fail_allocs{0};
static std::atomic<int> g_fail_at{0};

int fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

static bool take_injected_failure() {
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    }
    int k = g_fail_at.load();
    while (k > 0) {
        if (g_fail_at.compare_exchange_weak(k, k - 1)) return k == 1;
    }
    return false;
}

int dev_alloc(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (bytes == 0) return SPIIR_OK;
    if (take_injected_failure())
        return fail(SPIIR_ENOMEM, "device allocation of %zu bytes for %s failed (injected)", bytes,
                    what);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SPIIR_ENOMEM : SPIIR_ECUDA,
                    "cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    return SPIIR_OK;
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

int host_alloc_pinned(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (bytes == 0) return SPIIR_OK;
    if (take_injected_failure())
        return fail(SPIIR_ENOMEM, "pinned host allocation of %zu bytes for %s failed (injected)",
                    bytes, what);
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(SPIIR_ENOMEM, "cudaMallocHost of %zu bytes for %s failed: %s", bytes, what,
                    cudaGetErrorString(e));
    }
    return SPIIR_OK;
}

void host_free_pinned(void *p) {
    if (p) cudaFreeHost(p);
}

// The sticky status word is a file-scope device variable: reading or clearing it allocates
// nothing.  Its device address is looked up on every call, so that it stays right after the
// context of the current device has been re-created.
static __device__ int g_status_word;

int *device_status_word() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<int *>(p);
}

static std::mutex g_attr_mu;
static std::set<std::tuple<int, const void *, int>> g_attr_done;

int set_max_dyn_smem(const void *func, int bytes) {
    int dev = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const auto key = std::make_tuple(dev, func, bytes);
    if (g_attr_done.count(key)) return SPIIR_OK;
    SPIIR_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    g_attr_done.insert(key);
    return SPIIR_OK;
}

static std::map<std::tuple<int, const void *, int, size_t>, int> g_occupancy;

int resident_blocks_per_sm(const void *func, int threads, size_t smem, int *out) {
    int dev = 0;
    SPIIR_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const auto key = std::make_tuple(dev, func, threads, smem);
    auto it = g_occupancy.find(key);
    if (it == g_occupancy.end()) {
        int nb = 0;
        SPIIR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, smem));
        it = g_occupancy.emplace(key, nb).first;
    }
    *out = it->second;
    return SPIIR_OK;
}

}  // namespace spiir

using namespace spiir;

extern "C" int spiir_version(void) { return 100; }

extern "C" int spiir_last_error(char *buf, size_t len) {
    const std::string &m = g_last_error;
    if (buf && len) {
        size_t n = m.size() < len - 1 ? m.size() : len - 1;
        memcpy(buf, m.data(), n);
        buf[n] = 0;
    }
    return (int)m.size();
}

extern "C" void spiir_debug_fail_allocs(int n) { g_fail_allocs.store(n > 0 ? n : 0); }

extern "C" void spiir_debug_fail_alloc_at(int k) { g_fail_at.store(k > 0 ? k : 0); }

namespace spiir {

// One block waits on an mbarrier that nothing arrives on: the bounded wait gives up after
// `limit` tries and records the timeout, as every production wait does.
__global__ void k_debug_wait(uint32_t limit, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, limit);
    if (!ok && threadIdx.x == 0) report_timeout(status);
}

}  // namespace spiir

extern "C" int spiir_debug_wait_timeout(uint32_t iterations, void *stream) {
    clear_error();
    if (iterations < 1 || iterations > kWaitLimit)
        return fail(SPIIR_EINVAL, "iterations = %u outside [1, %u]", iterations, kWaitLimit);
    int *w = device_status_word();
    if (!w) return fail(SPIIR_ECUDA, "device status word unavailable");
    k_debug_wait<<<1, 32, 0, (cudaStream_t)stream>>>(iterations, w);
    SPIIR_CUDA_TRY(cudaGetLastError());
    return SPIIR_OK;
}

extern "C" int spiir_device_status(int clear) {
    int *w = device_status_word();
    if (!w) return fail(SPIIR_ECUDA, "device status word unavailable");
    SPIIR_CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    SPIIR_CUDA_TRY(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear) SPIIR_CUDA_TRY(cudaMemset(w, 0, sizeof(int)));
    if (v & kStatusTimeout) return fail(SPIIR_ETIMEOUT, "a bounded device-side wait gave up");
    if (v & kStatusBounds) return fail(SPIIR_ECUDA, "bounds check failed (codes 0x%x, checked build)", v >> 8);
    return SPIIR_OK;
}
