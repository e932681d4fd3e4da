// sptt_gram_noalloc: the Gram kernel (G = A^T A) for callers that must not
// allocate device memory.
//
// Who needs this: code whose device memory belongs entirely to another
// allocator (a framework's caching allocator that has already reserved the
// device, or a fixed arena in an embedded deployment), and code on a latency
// path where a cudaMalloc/cudaMallocAsync call -- which can synchronise the
// device or grow a pool -- is not acceptable. sptt_gram needs a workspace of
// per-block partial sums that it allocates on every call; this entry point
// keeps that workspace in one static device array instead.
//
// The array is file-scope `static __device__` storage of kScratchDoubles
// doubles (2 MiB). Every GPU that loads this library holds it until the
// process exits. Host code may not use the array's name as a device address
// (on the host it is only a stand-in), so the device address is looked up
// once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "internal.cuh"

namespace sptt {
namespace {

constexpr int64_t kScratchDoubles = int64_t(1) << 18;  // 2 MiB per device

static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on
// the first call made with that device current).
sptt_status scratch_for_current_device(double **out) {
    int dev = 0;
    SPTT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(SPTT_ERR_UNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        SPTT_CUDA(cudaGetSymbolAddress(&p, g_gram_scratch));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return SPTT_OK;
}

}  // namespace
}  // namespace sptt

using namespace sptt;

extern "C" sptt_status sptt_gram_noalloc(const float *A, int64_t rows, int32_t rank, int32_t ld, double *G,
                                         sptt_stream stream) {
    clear_error();
    if (!G || (!A && rows > 0)) return set_error(SPTT_ERR_BAD_ARG, "A (when rows > 0) and G must be non-NULL");
    if (rows < 0) return set_error(SPTT_ERR_BAD_ARG, "rows < 0");
    if (rank < 1 || rank > SPTT_MAX_RANK_ALS)
        return set_error(SPTT_ERR_UNSUPPORTED, "sptt_gram_noalloc: rank must be in [1, 64] (the static "
                                               "workspace holds at most 2^18 partial sums)");
    if (ld < rank) return set_error(SPTT_ERR_BAD_ARG, "ld < rank");
    double *scratch = nullptr;
    SPTT_TRY(scratch_for_current_device(&scratch));
    // One block per slot of (rank*rank + rank) partial sums that fits the
    // array, at most two per SM. Each block writes all of its rank*rank
    // entries before the reduction reads them, so nothing needs zeroing.
    const int64_t pstride = (int64_t)rank * rank + rank;
    int64_t nblocks = kScratchDoubles / pstride;
    const int64_t cap = (int64_t)device_sm_count() * 2;
    if (nblocks > cap) nblocks = cap;
    return gram_launch(A, rows, rank, ld, G, scratch, (int32_t)nblocks, reinterpret_cast<cudaStream_t>(stream));
}
