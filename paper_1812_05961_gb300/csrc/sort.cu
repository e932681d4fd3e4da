// Exclusive scan and stable LSD radix sort for the non-zero sort (Section V-C,
// "Sort"). The paper's C code sorts with a counting sort plus a quicksort
// specialised to 3 modes; on the GPU the same lexicographic order comes from
// a stable least-significant-digit radix sort on packed coordinate keys.
//
// Every kernel is a plain pass over tiles: per-tile digit histograms, one
// exclusive scan of the digit-major histogram table, then a stable scatter.
// No kernel waits on another CTA, so nothing here can spin.
#include "internal.cuh"

namespace sptt {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kWarpSpan = 32 * kSortItems;            // 512 keys per warp
// Digits of 8 or 9 bits (RB): a key of nbits bits takes ceil(nbits / RB)
// passes, and 9-bit digits save a pass where that count drops (45-bit keys:
// 5 passes instead of 6). Each thread owns RB - 7 digits of a tile's table.
constexpr int kMaxRadix = 1 << 9;

__device__ __forceinline__ int pad_idx(int i) { return i + (i >> 5); }

// Block-wide exclusive scan of one int per thread; returns the prefix and the
// block total (visible to every thread).
template <int THREADS>
__device__ __forceinline__ int block_exclusive_scan(int v, int &total) {
    constexpr int NW = THREADS / 32;
    static_assert(NW <= 32, "at most 1024 threads");
    __shared__ int warp_sums[NW + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int s = (lane < NW) ? warp_sums[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < NW) warp_sums[lane] = si - s;
        if (lane == NW - 1) warp_sums[NW] = si;
    }
    __syncthreads();
    const int r = warp_sums[warp] + incl - v;
    total = warp_sums[NW];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Scan (of an int32 array, or of the predicate d[i] <= level over a byte array)
// ---------------------------------------------------------------------------
struct InI32 {
    const int32_t *p;
    __device__ __forceinline__ int operator()(int64_t i) const { return p[i]; }
};

struct InLevelLE {
    const uint8_t *d;
    int level;
    __device__ __forceinline__ int operator()(int64_t i) const { return d[i] <= level; }
};

template <typename In>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const In in, int64_t n,
                                                                   int32_t *__restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) s += in(i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ int ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        tile_sums[blockIdx.x] = t;
    }
}

// One CTA scans the tile sums in place (exclusive) and writes the total.
__global__ void __launch_bounds__(1024) scan_spine_kernel(int32_t *__restrict__ sums, int64_t m,
                                                          int32_t *__restrict__ total) {
    const int T = 1024;
    const int64_t per = (m + T - 1) / T;
    const int64_t b = threadIdx.x * per;
    const int64_t e = (b + per < m) ? b + per : m;
    int local = 0;
    for (int64_t i = b; i < e; ++i) local += sums[i];
    int tot;
    int off = block_exclusive_scan<1024>(local, tot);
    for (int64_t i = b; i < e; ++i) {
        int v = sums[i];
        sums[i] = off;
        off += v;
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

template <typename In>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const In in,  // may alias out
                                                                 int32_t *out, int64_t n,
                                                                 const int32_t *__restrict__ tile_off) {
    __shared__ int s[kScanTile + kScanTile / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int li = j * kScanThreads + threadIdx.x;
        int64_t i = base + li;
        s[pad_idx(li)] = (i < n) ? in(i) : 0;
    }
    __syncthreads();
    int v[kScanItems];
    int local = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = s[pad_idx(threadIdx.x * kScanItems + j)];
        local += v[j];
    }
    int tot;
    int off = block_exclusive_scan<kScanThreads>(local, tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        s[pad_idx(threadIdx.x * kScanItems + j)] = off;
        off += v[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int li = j * kScanThreads + threadIdx.x;
        int64_t i = base + li;
        if (i < n) out[i] = s[pad_idx(li)];
    }
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
template <int RB>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t *__restrict__ keys,
                                                                  int64_t n, int shift, int64_t ntiles,
                                                                  int32_t *__restrict__ counts) {
    constexpr int R = 1 << RB;
    __shared__ int hist[kSortWarps][R];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    // all of the thread's keys are requested before the first is counted
    uint64_t k[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j * kSortThreads + threadIdx.x;
        k[j] = i < n ? keys[i] : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[warp][(int)((k[j] >> shift) & (R - 1))], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += kSortThreads) {
        int s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s += hist[w][d];
        counts[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

template <int RB>
struct ScatterSmem {
    int whist[kSortWarps][1 << RB];
    int tile_start[1 << RB];
    uint64_t keys[kSortTile];
    uint32_t vals[kSortTile];
};

template <int RB>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint64_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n, int shift,
    int64_t ntiles, const int32_t *__restrict__ offsets) {
    constexpr int R = 1 << RB;
    constexpr int DPT = R / kSortThreads;  // digits per thread in the tile's offset scan
    static_assert(DPT * kSortThreads == R, "whole digits per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<RB> &sm = *reinterpret_cast<ScatterSmem<RB> *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&sm.whist[0][0])[i] = 0;
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int64_t tile_n64 = n - base;
    const int tile_n = tile_n64 < kSortTile ? (int)tile_n64 : kSortTile;

    uint64_t k[kSortItems];
    uint32_t v[kSortItems];
    int dg[kSortItems];
    int loc[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int li = warp * kWarpSpan + j * 32 + lane;
        const bool valid = li < tile_n;
        k[j] = valid ? keys_in[base + li] : 0ull;
        v[j] = valid ? vals_in[base + li] : 0u;
        dg[j] = (int)((k[j] >> shift) & (R - 1));
    }
    // Stable rank of every key within its warp's span, in (j, lane) order.
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int li = warp * kWarpSpan + j * 32 + lane;
        const bool valid = li < tile_n;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        int r = 0, cnt = 0, old = 0;
        if (valid) {
            const unsigned peers = __match_any_sync(vmask, dg[j]);
            r = __popc(peers & lt_mask);
            cnt = __popc(peers);
            old = sm.whist[warp][dg[j]];
        }
        __syncwarp();
        if (valid && r == 0) sm.whist[warp][dg[j]] = old + cnt;
        __syncwarp();
        loc[j] = old + r;
    }
    __syncthreads();
    // Per digit: exclusive offsets of the warps, then of the digits in the
    // tile (thread t owns digits t * DPT .. t * DPT + DPT - 1).
    {
        int run[DPT];
        int sum = 0;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = threadIdx.x * DPT + q;
            int r = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const int c = sm.whist[w][d];
                sm.whist[w][d] = r;
                r += c;
            }
            run[q] = r;
            sum += r;
        }
        int tot;
        int start = block_exclusive_scan<kSortThreads>(sum, tot);
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            sm.tile_start[threadIdx.x * DPT + q] = start;
            start += run[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int li = warp * kWarpSpan + j * 32 + lane;
        if (li < tile_n) {
            const int p = sm.tile_start[dg[j]] + sm.whist[warp][dg[j]] + loc[j];
            sm.keys[p] = k[j];
            sm.vals[p] = v[j];
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < tile_n; p += kSortThreads) {
        const uint64_t key = sm.keys[p];
        const int d = (int)((key >> shift) & (R - 1));
        const int64_t g = (int64_t)offsets[(int64_t)d * ntiles + blockIdx.x] + (p - sm.tile_start[d]);
        keys_out[g] = key;
        vals_out[g] = sm.vals[p];
    }
}

}  // namespace

template <typename In>
sptt_status scan_exclusive(const In in, int32_t *out, int64_t n, bool with_total, cudaStream_t st) {
    if (n <= 0) {
        if (with_total) return fill_zero_launch(out, sizeof(int32_t), st);
        return SPTT_OK;
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    DevBuf sums;
    SPTT_TRY(sums.alloc<int32_t>(ntiles, st));
    scan_reduce_kernel<In><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums.as<int32_t>());
    SPTT_CHECK_LAUNCH("scan_reduce_kernel");
    scan_spine_kernel<<<1, 1024, 0, st>>>(sums.as<int32_t>(), ntiles, with_total ? out + n : nullptr);
    SPTT_CHECK_LAUNCH("scan_spine_kernel");
    scan_down_kernel<In><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n, sums.as<int32_t>());
    SPTT_CHECK_LAUNCH("scan_down_kernel");
    return SPTT_OK;
}

sptt_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, bool with_total,
                               cudaStream_t st) {
    return scan_exclusive(InI32{in}, out, n, with_total, st);
}

sptt_status scan_exclusive_level(const uint8_t *d, int level, int32_t *out, int64_t n, bool with_total,
                                 cudaStream_t st) {
    return scan_exclusive(InLevelLE{d, level}, out, n, with_total, st);
}

namespace {

template <int RB>
sptt_status radix_sort_passes(uint64_t *&keys, uint32_t *&vals, uint64_t *&keys_alt, uint32_t *&vals_alt,
                              int64_t n, int nbits, int64_t ntiles, int32_t *counts, cudaStream_t st) {
    SPTT_CUDA(cudaFuncSetAttribute(radix_scatter_kernel<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(ScatterSmem<RB>)));
    for (int shift = 0; shift < nbits; shift += RB) {
        radix_hist_kernel<RB><<<(unsigned)ntiles, kSortThreads, 0, st>>>(keys, n, shift, ntiles, counts);
        SPTT_CHECK_LAUNCH("radix_hist_kernel");
        SPTT_TRY(scan_exclusive_i32(counts, counts, (int64_t)(1 << RB) * ntiles, false, st));
        radix_scatter_kernel<RB><<<(unsigned)ntiles, kSortThreads, sizeof(ScatterSmem<RB>), st>>>(
            keys, vals, keys_alt, vals_alt, n, shift, ntiles, counts);
        SPTT_CHECK_LAUNCH("radix_scatter_kernel");
        uint64_t *tk = keys;
        keys = keys_alt;
        keys_alt = tk;
        uint32_t *tv = vals;
        vals = vals_alt;
        vals_alt = tv;
    }
    return SPTT_OK;
}

}  // namespace

sptt_status radix_sort_pairs(uint64_t *&keys, uint32_t *&vals, uint64_t *&keys_alt,
                             uint32_t *&vals_alt, int64_t n, int nbits, cudaStream_t st) {
    if (n <= 1 || nbits <= 0) return SPTT_OK;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    DevBuf counts;
    SPTT_TRY(counts.alloc<int32_t>((size_t)kMaxRadix * ntiles + 1, st));
    // 9-bit digits where they need fewer passes than 8-bit ones
    if ((nbits + 8) / 9 < (nbits + 7) / 8)
        return radix_sort_passes<9>(keys, vals, keys_alt, vals_alt, n, nbits, ntiles, counts.as<int32_t>(), st);
    return radix_sort_passes<8>(keys, vals, keys_alt, vals_alt, n, nbits, ntiles, counts.as<int32_t>(), st);
}

}  // namespace sptt
