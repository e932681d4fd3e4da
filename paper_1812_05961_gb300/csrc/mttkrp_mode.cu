// MTTKRP for any mode from one CSF (Section III; the MTTKRP step of Algorithm 1),
// the single-CSF form of SPLATT that the paper's lock pool and privatised
// outputs serve (Section IV-A, Section V-D-2).
//
// For the CSF with level order (o_0, ..., o_{N-1}) and the target mode
// n = o_L, L >= 1: a level-L fiber f with index i = fids[L][f] contributes
//   M[i, :] += (prod_{l < L} A^(o_l)[path row at level l, :]) *
//              (sum over the leaves below f of v * prod_{l > L} A^(o_l)[...])
// (for L = N-1 the fiber is a leaf and the second factor is its value). The
// walk keeps the Hadamard products of the ancestor rows and, below level L,
// the same bottom-up sums as the root walk, and emits one row segment per
// level-L fiber (per leaf when L = N-1) that closes in its chunk.
//
// Output conflicts: many fibers share an index, in any chunk. GPU form of
// the paper's choice between locking and privatising:
//   * hot rows (the indices with the most contributions, as many as fit in
//     64 KB of shared memory per CTA) are privatised per CTA: summed with
//     shared-memory atomics and added to the output every few rounds of
//     chunks, which also bounds the number of FP32 additions per partial;
//   * every other row is updated with red.global.add.v4.f32.
// sched->variant for a non-root mode: 0 / 2 = privatise the hot rows,
// 1 = global reductions only.
#include "walk.cuh"

namespace sptt {
namespace {

constexpr int kModeThreads = 256;
constexpr int kHotBytes = 64 * 1024;  // shared memory per CTA for the hot rows
constexpr int kMinHot = 64;           // contributions below which a row is never privatised
constexpr int kFlushRounds = 4;       // chunk rounds between flushes of the hot rows

struct LevelArgs {
    walk::Args w;            // CSF arrays and factors by level (w.out, w.heavy, w.hidx unused)
    float *out;              // dims[o_L] x ld, zeroed
    const int32_t *hslot;    // per index of the target mode: hot slot or -1 (NULL: no hot rows)
    const int32_t *hrow;     // hot slot -> row
    int32_t nhot;
};

template <int VEC>
__device__ __forceinline__ void emit(const LevelArgs &a, float *hot, int32_t row, int32_t slot, int col,
                                     const float (&x)[VEC]) {
    const int ld = a.w.ld;
    if (slot >= 0) {
        float *p = hot + slot * ld + col;
#pragma unroll
        for (int i = 0; i < VEC; ++i) atomicAdd(p + i, x[i]);
    } else {
        float *dst = a.out + (int64_t)row * ld + col;
#pragma unroll
        for (int i = 0; i < VEC; i += 4)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + i), "f"(x[i]), "f"(x[i + 1]),
                         "f"(x[i + 2]), "f"(x[i + 3])
                         : "memory");
    }
}

__device__ __forceinline__ int32_t slot_of(const LevelArgs &a, int32_t row) {
    return a.hslot ? __ldg(a.hslot + row) : -1;
}

// One chunk of leaves for target level L.
template <int NM, int L, typename T>
__device__ __forceinline__ void level_chunk(const LevelArgs &a, int64_t c, int col, float *hot) {
    using Rw = walk::Raw<T>;
    using Row = typename Rw::Row;
    constexpr int VEC = Rw::VEC;
    constexpr int NL = NM - 1;                     // fiber levels 0..NM-2
    constexpr int LF = NM - 2;                     // the leaves' parent level
    constexpr bool LEAF = (L == NM - 1);           // target is the leaf level
    constexpr int NA = LEAF ? 1 : (LF - L + 1);    // sums for levels L..LF (index l - L)
    const walk::Args &w = a.w;
    const int ld = w.ld;
    const int64_t k0 = c * (int64_t)w.chunk;
    const int64_t k1 = (k0 + w.chunk < w.nnz) ? k0 + w.chunk : w.nnz;
    int32_t f[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) f[l] = __ldg(w.part + c * NL + l);
    // up[l] = Hadamard product of the rows of the open fibers at levels 0..l
    float up[L][VEC];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        float r[VEC];
        Rw::widen(Rw::load(w.fac[l], __ldg(w.fids[l] + f[l]), ld, col), r);
#pragma unroll
        for (int i = 0; i < VEC; ++i) up[l][i] = l ? up[l - 1][i] * r[i] : r[i];
    }
    float acc[NA][VEC];
#pragma unroll
    for (int q = 0; q < NA; ++q)
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[q][i] = 0.f;
    Row rowc[NA];  // rows of the open fibers at levels L+1..LF (index l - L)
#pragma unroll
    for (int l = L + 1; l <= LF; ++l) rowc[l - L] = Rw::load(w.fac[l], __ldg(w.fids[l] + f[l]), ld, col);
    int32_t orow = 0, oslot = -1;  // output row (and hot slot) of the open level-L fiber
    if constexpr (!LEAF) {
        orow = __ldg(w.fids[L] + f[L]);
        oslot = slot_of(a, orow);
    }

    for (int64_t kb = k0; kb < k1; kb += 4) {
        const float4 va = __ldg(reinterpret_cast<const float4 *>(w.vals + kb));
        const int4 ia = __ldg(reinterpret_cast<const int4 *>(w.fids[NM - 1] + kb));
        const uint32_t lw = __ldg(reinterpret_cast<const uint32_t *>(w.lvl + kb));
        const float v[4] = {va.x, va.y, va.z, va.w};
        const int32_t li[4] = {ia.x, ia.y, ia.z, ia.w};
        const int nvalid = (k1 - kb < 4) ? (int)(k1 - kb) : 4;
        Row x[4];
        int32_t ls[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= nvalid) break;
            if constexpr (LEAF) ls[j] = slot_of(a, li[j]);
            else x[j] = Rw::load(w.fac[NM - 1], li[j], ld, col);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= nvalid) break;
            const int d = (int)((lw >> (8 * j)) & 0xffu);
            if (kb + j != k0 && d <= LF) {
                // close the fibers at levels >= max(d, L+1), bottom-up
#pragma unroll
                for (int l = LF; l >= L + 1; --l)
                    if (d <= l) walk::fold<T>(acc[l - 1 - L], acc[l - L], rowc[l - L]);
                if constexpr (!LEAF) {
                    if (d <= L) {
                        float y[VEC];
#pragma unroll
                        for (int i = 0; i < VEC; ++i) {
                            y[i] = up[L - 1][i] * acc[0][i];
                            acc[0][i] = 0.f;
                        }
                        emit<VEC>(a, hot, orow, oslot, col, y);
                    }
                }
                // open the next fibers at levels >= d
#pragma unroll
                for (int l = 0; l <= LF; ++l)
                    if (l >= d) ++f[l];
#pragma unroll
                for (int l = 0; l < L; ++l)
                    if (l >= d) {
                        float r[VEC];
                        Rw::widen(Rw::load(w.fac[l], __ldg(w.fids[l] + f[l]), ld, col), r);
#pragma unroll
                        for (int i = 0; i < VEC; ++i) up[l][i] = l ? up[l - 1][i] * r[i] : r[i];
                    }
#pragma unroll
                for (int l = L + 1; l <= LF; ++l)
                    if (l >= d) rowc[l - L] = Rw::load(w.fac[l], __ldg(w.fids[l] + f[l]), ld, col);
                if constexpr (!LEAF) {
                    if (d <= L) {
                        orow = __ldg(w.fids[L] + f[L]);
                        oslot = slot_of(a, orow);
                    }
                }
            }
            if constexpr (LEAF) {
                float y[VEC];
#pragma unroll
                for (int i = 0; i < VEC; ++i) y[i] = v[j] * up[L - 1][i];
                emit<VEC>(a, hot, li[j], ls[j], col, y);
            } else {
                float xr[VEC];
                Rw::widen(x[j], xr);
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc[LF - L][i] = fmaf(v[j], xr[i], acc[LF - L][i]);
            }
        }
    }
    // chunk end: fold the open fibers below L and emit the open level-L fiber's part
#pragma unroll
    for (int l = LF; l >= L + 1; --l) walk::fold<T>(acc[l - 1 - L], acc[l - L], rowc[l - L]);
    if constexpr (!LEAF) {
        float y[VEC];
#pragma unroll
        for (int i = 0; i < VEC; ++i) y[i] = up[L - 1][i] * acc[0][i];
        emit<VEC>(a, hot, orow, oslot, col, y);
    }
}

// Each CTA takes a contiguous range of chunks, its lane groups interleaved,
// in rounds of one chunk per group; every kFlushRounds rounds (and at the
// end) the CTA adds its hot-row partials to the output and clears them.
// Idle lanes stay for the CTA barriers.
template <int NM, int L, typename T>
__global__ void __launch_bounds__(kModeThreads, 2) mttkrp_level_kernel(const LevelArgs a) {
    extern __shared__ __align__(16) float hot[];
    constexpr int VEC = walk::Raw<T>::VEC;
    const int ld = a.w.ld;
    const walk::Lanes Ln = walk::lanes_for(ld, VEC);
    const int nh = a.nhot;
    for (int e = threadIdx.x; e < nh * ld; e += blockDim.x) hot[e] = 0.f;
    __syncthreads();
    const int64_t nchunks = a.w.nchunks;
    const int64_t per = (nchunks + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per;
    const int64_t b1 = (b0 + per < nchunks) ? b0 + per : nchunks;
    const int64_t step = (int64_t)(blockDim.x >> 5) * Ln.gpw;
    const int64_t g = (int64_t)(threadIdx.x >> 5) * Ln.gpw + Ln.gi;
    const int64_t rounds = (b1 > b0) ? (b1 - b0 + step - 1) / step : 0;
    for (int64_t round = 0; round < rounds; ++round) {
        const int64_t c = b0 + round * step + g;
        if (!Ln.idle && c < b1) level_chunk<NM, L, T>(a, c, Ln.col, hot);
        if (nh > 0 && ((round + 1) % kFlushRounds == 0 || round + 1 == rounds)) {
            __syncthreads();
            for (int e = threadIdx.x; e < nh * ld; e += blockDim.x) {
                const float v = hot[e];
                if (v != 0.f) {
                    const int s = e / ld;
                    atomicAdd(a.out + (int64_t)__ldg(a.hrow + s) * ld + (e - s * ld), v);
                    hot[e] = 0.f;
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Hot rows of a level: contributions per index (level-L fibers, or leaves),
// a log2 histogram of the counts, and the slots of the indices above the
// threshold the host picks from the histogram.
// ---------------------------------------------------------------------------
__global__ void count_index_kernel(const int32_t *__restrict__ ids, int64_t n, int32_t *__restrict__ cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + __ldg(ids + e), 1);
}

__global__ void count_hist_kernel(const int32_t *__restrict__ cnt, int64_t n, unsigned long long *__restrict__ hist) {
    __shared__ unsigned long long h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = cnt[e];
        if (k > 0) atomicAdd(h + (31 - __clz(k)), 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

__global__ void hot_assign_kernel(const int32_t *__restrict__ cnt, int64_t n, int32_t threshold,
                                  int32_t *__restrict__ counter, int32_t cap, int32_t *__restrict__ hslot,
                                  int32_t *__restrict__ hrow) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = -1;
        if (cnt[e] >= threshold) {
            s = atomicAdd(counter, 1);
            if (s < cap) hrow[s] = (int32_t)e;
            else s = -1;
        }
        hslot[e] = s;
    }
}

int grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// Builds (once per level and row width) the hot-row table of level L.
sptt_status ensure_hot(sptt_csf *c, int L, int32_t ld, cudaStream_t st) {
    const int cap = kHotBytes / (ld * (int)sizeof(float));
    if (c->hslot[L] && c->hot_cap[L] == cap) return SPTT_OK;
    const int64_t rows = c->dims[c->order[L]];
    const int64_t n = c->nfibs[L];
    if (!c->hslot[L]) {
        SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->hslot[L]),
                       (size_t)(rows + 64) * sizeof(int32_t), st));
        SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->hrow[L]),
                       (size_t)(kHotBytes / (4 * (int)sizeof(float)) + 64) * sizeof(int32_t), st));
    }
    DevBuf cnt, hist, counter;
    SPTT_TRY(cnt.alloc<int32_t>((size_t)rows, st));
    SPTT_TRY(hist.alloc<unsigned long long>(32, st));
    SPTT_TRY(counter.alloc<int32_t>(1, st));
    SPTT_TRY(fill_zero_launch(cnt.as<int32_t>(), rows * sizeof(int32_t), st));
    SPTT_TRY(fill_zero_launch(hist.as<unsigned long long>(), 32 * sizeof(unsigned long long), st));
    SPTT_TRY(fill_zero_launch(counter.as<int32_t>(), sizeof(int32_t), st));
    if (n > 0) {
        count_index_kernel<<<grid_of(n), 256, 0, st>>>(c->fids[L], n, cnt.as<int32_t>());
        SPTT_CHECK_LAUNCH("count_index_kernel");
    }
    if (rows > 0) {
        count_hist_kernel<<<grid_of(rows), 256, 0, st>>>(cnt.as<int32_t>(), rows, hist.as<unsigned long long>());
        SPTT_CHECK_LAUNCH("count_hist_kernel");
    }
    unsigned long long h[32];
    SPTT_CUDA(cudaMemcpyAsync(h, hist.as<unsigned long long>(), sizeof(h), cudaMemcpyDeviceToHost, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    // smallest power-of-two threshold (>= kMinHot) whose rows fit the cap
    int b = 31;
    unsigned long long above = h[31];
    while (b > 0 && (1 << (b - 1)) >= kMinHot && above + h[b - 1] <= (unsigned long long)cap) {
        --b;
        above += h[b];
    }
    const int64_t thr = (int64_t)1 << b;
    const int32_t threshold = (above == 0 || thr < kMinHot || thr > INT32_MAX) ? INT32_MAX : (int32_t)thr;
    if (rows > 0) {
        hot_assign_kernel<<<grid_of(rows), 256, 0, st>>>(cnt.as<int32_t>(), rows, threshold, counter.as<int32_t>(),
                                                         cap, c->hslot[L], c->hrow[L]);
        SPTT_CHECK_LAUNCH("hot_assign_kernel");
    }
    int32_t nh = 0;
    SPTT_CUDA(cudaMemcpyAsync(&nh, counter.as<int32_t>(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    c->nhot[L] = nh < cap ? nh : cap;
    c->hot_cap[L] = cap;
    return SPTT_OK;
}

template <int NM, int L, typename T>
sptt_status launch_level(const LevelArgs &a, cudaStream_t st) {
    auto kern = mttkrp_level_kernel<NM, L, T>;
    const size_t smem = (size_t)a.nhot * a.w.ld * sizeof(float);
    SPTT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kHotBytes));
    int per_sm = 0;
    SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kModeThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const int gpb = (kModeThreads / 32) * (32 / (a.w.ld / walk::Raw<T>::VEC));
    const int64_t need = (a.w.nchunks + gpb - 1) / gpb;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t grid = need < cap ? need : cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kModeThreads, smem, st>>>(a);
    SPTT_CHECK_LAUNCH("mttkrp_level_kernel");
    return SPTT_OK;
}

template <typename T>
sptt_status launch_level_t(int nm, int L, const LevelArgs &a, cudaStream_t st) {
#define SPTT_LEVEL_CASE(NM_, L_) \
    if (nm == NM_ && L == L_) return launch_level<NM_, L_, T>(a, st);
    SPTT_LEVEL_CASE(2, 1)
    SPTT_LEVEL_CASE(3, 1)
    SPTT_LEVEL_CASE(3, 2)
    SPTT_LEVEL_CASE(4, 1)
    SPTT_LEVEL_CASE(4, 2)
    SPTT_LEVEL_CASE(4, 3)
    SPTT_LEVEL_CASE(5, 1)
    SPTT_LEVEL_CASE(5, 2)
    SPTT_LEVEL_CASE(5, 3)
    SPTT_LEVEL_CASE(5, 4)
#undef SPTT_LEVEL_CASE
    return set_error(SPTT_ERR_UNSUPPORTED, "nmodes");
}

}  // namespace

int csf_level_of(const sptt_csf *c, int32_t mode) {
    for (int l = 0; l < c->nmodes; ++l)
        if (c->order[l] == mode) return l;
    return -1;
}

sptt_status mttkrp_mode_prepare(sptt_csf *c, int32_t L, int32_t ld, const sptt_sched *sched, cudaStream_t st) {
    const int32_t chunk = (sched && sched->chunk) ? sched->chunk : default_chunk(c->nfibs[c->nmodes - 1]);
    SPTT_TRY(csf_ensure_partition(c, chunk, st));
    const bool priv = !(sched && sched->variant == 1);
    if (priv) SPTT_TRY(ensure_hot(c, L, ld, st));
    return SPTT_OK;
}

sptt_status mttkrp_mode_launch(sptt_csf *c, int32_t L, const void *const *factors, int32_t dtype, int32_t ld,
                               float *out, const sptt_sched *sched, cudaStream_t st) {
    const int N = c->nmodes;
    SPTT_TRY(fill_zero_launch(out, (size_t)c->dims[c->order[L]] * ld * sizeof(float), st));
    const int64_t nnz = c->nfibs[N - 1];
    if (nnz == 0) return SPTT_OK;
    const int32_t chunk = (sched && sched->chunk) ? sched->chunk : default_chunk(nnz);
    SPTT_TRY(csf_ensure_partition(c, chunk, st));
    const bool priv = !(sched && sched->variant == 1);
    LevelArgs a{};
    for (int l = 0; l < N; ++l) {
        a.w.fptr[l] = c->fptr[l];
        a.w.fids[l] = c->fids[l];
        a.w.fac[l] = (l == L) ? nullptr : factors[c->order[l]];
    }
    a.w.vals = c->vals;
    a.w.lvl = c->lvl;
    a.w.part = c->part;
    a.w.nchunks = c->part_nchunks;
    a.w.nnz = nnz;
    a.w.chunk = chunk;
    a.w.ld = ld;
    a.out = out;
    const int cap = kHotBytes / (ld * (int)sizeof(float));
    if (priv && c->hslot[L] && c->hot_cap[L] == cap && c->nhot[L] > 0) {
        a.hslot = c->hslot[L];
        a.hrow = c->hrow[L];
        a.nhot = c->nhot[L];
    }
    if (dtype == SPTT_BF16) return launch_level_t<__nv_bfloat16>(N, L, a, st);
    return launch_level_t<float>(N, L, a, st);
}

}  // namespace sptt

using namespace sptt;

extern "C" sptt_status sptt_mttkrp_mode(const sptt_csf *csf, int32_t mode, const void *const *factors,
                                        int32_t factor_dtype, int32_t ld, float *out, const sptt_sched *sched,
                                        sptt_stream stream) {
    clear_error();
    if (!csf) return set_error(SPTT_ERR_BAD_ARG, "csf must be non-NULL");
    if (mode < 0 || mode >= csf->nmodes) return set_error(SPTT_ERR_BAD_ARG, "mode out of range");
    if (mode == csf->root) return sptt_mttkrp(csf, factors, factor_dtype, ld, out, sched, stream);
    if (!factors || !out) return set_error(SPTT_ERR_BAD_ARG, "factors and out must be non-NULL");
    if (factor_dtype != SPTT_F32 && factor_dtype != SPTT_BF16)
        return set_error(SPTT_ERR_BAD_ARG, "factor_dtype must be SPTT_F32 or SPTT_BF16");
    const int vec = factor_dtype == SPTT_BF16 ? 8 : 4;
    if (ld < vec || ld > 32 * vec || ld % vec)
        return set_error(SPTT_ERR_BAD_ARG, "ld must be a multiple of " + std::to_string(vec) + " in [" +
                                               std::to_string(vec) + ", " + std::to_string(32 * vec) + "]");
    if (reinterpret_cast<uintptr_t>(out) % 16) return set_error(SPTT_ERR_BAD_ARG, "out must be 16-byte aligned");
    const int L = csf_level_of(csf, mode);
    for (int l = 0; l < csf->nmodes; ++l) {
        if (l == L) continue;
        const void *p = factors[csf->order[l]];
        if (!p) return set_error(SPTT_ERR_BAD_ARG, "a factor other than the target's is NULL");
        if (reinterpret_cast<uintptr_t>(p) % 16) return set_error(SPTT_ERR_BAD_ARG, "factors must be 16-byte aligned");
        if (p == out) return set_error(SPTT_ERR_BAD_ARG, "out aliases a factor");
    }
    if (sched) {
        if (sched->chunk && (sched->chunk < 16 || sched->chunk > 4096 || (sched->chunk & (sched->chunk - 1))))
            return set_error(SPTT_ERR_BAD_ARG, "sched->chunk must be a power of two in [16, 4096]");
        if (sched->variant < 0 || sched->variant > 2)
            return set_error(SPTT_ERR_BAD_ARG, "sched->variant for a non-root mode must be in [0, 2]");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    sptt_csf *c = const_cast<sptt_csf *>(csf);
    SPTT_TRY(mttkrp_mode_prepare(c, L, ld, sched, st));
    return mttkrp_mode_launch(c, L, factors, factor_dtype, ld, out, sched, st);
}
