// Error state, device memory and small C-ABI helpers of libsptt.
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace sptt {

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_fail_alloc_countdown{0};
std::atomic<int64_t> g_launches{0};
std::mutex g_pool_mu;
bool g_pool_ready[64] = {false};
int g_sm_count[64] = {0};
}  // namespace

sptt_status set_error(sptt_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

sptt_status cuda_error(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return SPTT_ERR_OOM;
    return SPTT_ERR_CUDA;
}

void clear_error() { g_last_error.clear(); }

void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 0;
    return d;
}

int device_sm_count() {
    const int d = current_device();
    if (!g_sm_count[d]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) n = kNumSMs;
        g_sm_count[d] = n;
    }
    return g_sm_count[d];
}

sptt_status dev_alloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    const int64_t c = g_fail_alloc_countdown.load();
    if (c > 0 && g_fail_alloc_countdown.fetch_sub(1) == 1)
        return set_error(SPTT_ERR_OOM, "injected allocation failure");
    const int d = current_device();
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_ready[d]) {
            // keep freed blocks in this process's pool instead of returning
            // them to the driver at every synchronisation
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            g_pool_ready[d] = true;
        }
    }
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_error(e, "cudaMallocAsync");
    }
    return SPTT_OK;
}

void dev_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

}  // namespace sptt

using namespace sptt;

extern "C" const char *sptt_status_str(sptt_status s) {
    switch (s) {
        case SPTT_OK: return "SPTT_OK";
        case SPTT_ERR_BAD_ARG: return "SPTT_ERR_BAD_ARG";
        case SPTT_ERR_OOM: return "SPTT_ERR_OOM";
        case SPTT_ERR_CUDA: return "SPTT_ERR_CUDA";
        case SPTT_ERR_TIMEOUT: return "SPTT_ERR_TIMEOUT";
        case SPTT_ERR_NOT_PD: return "SPTT_ERR_NOT_PD";
        case SPTT_ERR_UNSUPPORTED: return "SPTT_ERR_UNSUPPORTED";
        case SPTT_ERR_INTERNAL: return "SPTT_ERR_INTERNAL";
        default: return "SPTT_ERR_UNKNOWN";
    }
}

extern "C" const char *sptt_last_error(void) { return g_last_error.c_str(); }

extern "C" int32_t sptt_version(void) { return 100; }

extern "C" int64_t sptt_debug_launch_count(void) { return g_launches.load(); }

extern "C" void sptt_debug_fail_alloc_after(int64_t countdown) {
    g_fail_alloc_countdown.store(countdown > 0 ? countdown : 0);
}
