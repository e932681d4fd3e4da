// COO -> CSF on the device (Section III; the non-zero sort of Section V-C).
//
// 1. validate every index against its mode length;
// 2. stable LSD radix sort of the non-zero positions by packed coordinate
//    keys in level order (levels grouped into 64-bit words from the leaf up;
//    each word sorted stably after the less significant ones);
// 3. gather coordinates and values in sorted order;
// 4. coalesce duplicate coordinates (FP64 sum in input order, one rounding);
// 5. per level l < N-1: "prefix changed" flags -> exclusive scan -> fiber ids,
//    then fids/fptr written at each fiber's first non-zero.
// All integer work is exact, so the result is bit-identical to a plain
// sequential construction.
#include <string.h>

#include <vector>

#include "internal.cuh"

namespace sptt {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int threads = kThreads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g < 1 ? 1 : g);
}

// The streaming passes over the non-zeros take kItems elements per thread,
// blockDim apart (each of a warp's loads stays coalesced), and issue all of
// their loads before the first use, so a thread keeps several requests in
// flight instead of one dependent chain.
constexpr int kItems = 4;
inline unsigned grid_items(int64_t n) {
    const int64_t per = (int64_t)kThreads * kItems;
    int64_t g = (n + per - 1) / per;
    return (unsigned)(g < 1 ? 1 : g);
}
__device__ __forceinline__ int64_t item_index(int j) {
    return (int64_t)blockIdx.x * (kThreads * kItems) + (int64_t)j * kThreads + threadIdx.x;
}

inline int bits_for(int64_t dim) {  // bits to hold 0..dim-1
    int b = 0;
    while (b < 63 && (int64_t(1) << b) < dim) ++b;
    return b;
}

struct IdxPtrs {
    const int32_t *p[kMaxModes];
};

// key[k] = sum over the group's levels of idx << shift, taken at src(k).
// Every index of the group's levels (length-1 modes included, which add no
// key bits) is checked against its mode length on the way: each level
// belongs to one group, so every index of the tensor is checked once.
struct KeyGroup {
    int nchk;                        // the group's levels, length-1 modes included
    const int32_t *chk[kMaxModes];
    int64_t dim[kMaxModes];
    int shift[kMaxModes];            // bit position in the key, or -1 (a length-1 mode adds no bits)
};

// vals[k] = src, or (when the whole key is this one group) the bits of the
// value at src, which the sort then carries: the sorted values need no
// gather through a permutation.
__global__ void __launch_bounds__(kThreads) build_keys_kernel(KeyGroup g, const uint32_t *__restrict__ perm, int64_t n,
                                                              uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                              int32_t *__restrict__ err,
                                                              const float *__restrict__ carry_vals) {
    uint32_t src[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        src[j] = k < n ? (perm ? perm[k] : (uint32_t)k) : 0u;
    }
    int32_t x[kItems][kMaxModes];
    uint32_t cv[kItems];
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m)
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            x[j][m] = (m < g.nchk && item_index(j) < n) ? g.chk[m][src[j]] : 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) cv[j] = (carry_vals && item_index(j) < n) ? __float_as_uint(carry_vals[src[j]]) : 0u;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        if (k >= n) continue;
        uint64_t key = 0;
#pragma unroll
        for (int m = 0; m < kMaxModes; ++m) {
            if (m >= g.nchk) break;
            bad |= x[j][m] < 0 || (int64_t)x[j][m] >= g.dim[m];
            if (g.shift[m] >= 0) key |= (uint64_t)(uint32_t)x[j][m] << g.shift[m];
        }
        keys[k] = key;
        vals[k] = carry_vals ? cv[j] : src[j];
    }
    if (bad) atomicOr(err, 1);
}

struct OutPtrs {
    int32_t *p[kMaxModes];
};

// Where each level's sorted index comes from: levels of the last-sorted key
// group are bit fields of the sorted key (shift[l] >= 0, width bits[l]);
// the others are gathered through the permutation.
struct Decode {
    int shift[kMaxModes];
    int bits[kMaxModes];
};

// perm = NULL: every level is in the key and sorted_bits holds the values.
__global__ void __launch_bounds__(kThreads) gather_sorted_kernel(IdxPtrs lev_inds, int nlev, const float *__restrict__ vals,
                                                                 const uint32_t *__restrict__ perm,
                                                                 const uint32_t *__restrict__ sorted_bits,
                                                                 const uint64_t *__restrict__ keys, Decode dec, int64_t n,
                                                                 OutPtrs out, float *__restrict__ out_vals) {
    uint32_t src[kItems], vb[kItems];
    uint64_t key[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        const bool in = k < n;
        src[j] = (perm && in) ? perm[k] : 0u;
        key[j] = in ? keys[k] : 0ull;
        vb[j] = (!perm && in) ? sorted_bits[k] : 0u;
    }
    int32_t g[kItems][kMaxModes];
#pragma unroll
    for (int l = 0; l < kMaxModes; ++l)
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            g[j][l] = (l < nlev && dec.shift[l] < 0 && item_index(j) < n) ? lev_inds.p[l][src[j]] : 0;
    if (perm) {
#pragma unroll
        for (int j = 0; j < kItems; ++j) vb[j] = item_index(j) < n ? __float_as_uint(vals[src[j]]) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        if (k >= n) continue;
#pragma unroll
        for (int l = 0; l < kMaxModes; ++l) {
            if (l >= nlev) break;
            out.p[l][k] = dec.shift[l] >= 0
                              ? (dec.bits[l] ? (int32_t)((key[j] >> dec.shift[l]) & ((uint64_t(1) << dec.bits[l]) - 1)) : 0)
                              : g[j][l];
        }
        out_vals[k] = __uint_as_float(vb[j]);
    }
}

// flag[k] = 1 if the coordinate prefix of levels 0..upto differs from k-1.
__global__ void prefix_flags_kernel(IdxPtrs s, int upto, int64_t n, int32_t *__restrict__ flags) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int f = (k == 0);
        if (!f)
            for (int l = 0; l <= upto; ++l)
                if (s.p[l][k] != s.p[l][k - 1]) { f = 1; break; }
        flags[k] = f;
    }
}

// d[k] = the first level whose index differs from position k - 1 (0 at
// k = 0; nlev when all are equal, i.e. a duplicate coordinate). Fiber
// starts, duplicate runs and the CSF's per-leaf level flags all follow.
__global__ void __launch_bounds__(kThreads) level_diff_kernel(IdxPtrs s, int nlev, int64_t n, uint8_t *__restrict__ d,
                                                              unsigned long long *__restrict__ ndup) {
    int32_t cur[kItems][kMaxModes], prv[kItems][kMaxModes];
#pragma unroll
    for (int l = 0; l < kMaxModes; ++l)
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t k = item_index(j);
            const bool in = l < nlev && k < n;
            cur[j][l] = in ? s.p[l][k] : 0;
            prv[j][l] = (in && k > 0) ? s.p[l][k - 1] : 0;
        }
    unsigned long long dup = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        if (k >= n) continue;
        int x = 0;
        if (k > 0) {
            x = nlev;
#pragma unroll
            for (int l = kMaxModes - 1; l >= 0; --l)
                if (l < nlev && cur[j][l] != prv[j][l]) x = l;  // the lowest differing level
        }
        dup += (x == nlev);
        d[k] = (uint8_t)x;
    }
    for (int o = 16; o > 0; o >>= 1) dup += __shfl_xor_sync(0xffffffffu, dup, o);
    if ((threadIdx.x & 31) == 0 && dup) atomicAdd(ndup, dup);
}

// For each distinct coordinate u starting at k: starts[u] = k.
__global__ void run_starts_kernel(const int32_t *__restrict__ uid, int64_t n,
                                  int32_t *__restrict__ starts) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (uid[k + 1] != uid[k]) starts[uid[k]] = (int32_t)k;
    }
}

// Coalesce: coordinates of each run's first entry; value = FP64 sum of the
// run in order (input order, since the sort is stable), rounded once.
__global__ void coalesce_kernel(IdxPtrs s, int nlev, const float *__restrict__ sv,
                                const int32_t *__restrict__ starts, int64_t u_count, int64_t n,
                                OutPtrs out, float *__restrict__ out_vals) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < u_count;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = starts[u];
        const int64_t e = (u + 1 < u_count) ? starts[u + 1] : n;
        double sum = 0.0;
        for (int64_t k = b; k < e; ++k) sum += (double)sv[k];
        out_vals[u] = (float)sum;
        for (int l = 0; l < nlev; ++l) out.p[l][u] = s.p[l][b];
    }
}

// Write fids/fptr of every level l < N-1 at each fiber's first non-zero.
struct LevelScan {
    const int32_t *fidx[kMaxModes];  // exclusive scans (length n+1) for l = 0..N-2
    int32_t *fids[kMaxModes];
    int32_t *fptr[kMaxModes];
};

// Position k starts a level-l fiber when d[k] <= l (then it starts one at
// every deeper level too); its fiber index is the exclusive scan fidx[l][k].
__global__ void __launch_bounds__(kThreads) fill_levels_kernel(IdxPtrs s, LevelScan ls, const uint8_t *__restrict__ d,
                                                               int nlev, int64_t n) {
    int dk[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        dk[j] = k < n ? d[k] : nlev;
    }
#pragma unroll
    for (int l = 0; l < kMaxModes - 1; ++l) {
        if (l >= nlev - 1) break;
        int32_t f[kItems], id[kItems], nx[kItems];
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t k = item_index(j);
            const bool starts = dk[j] <= l;  // k opens a level-l fiber (dk = nlev past the end)
            f[j] = starts ? ls.fidx[l][k] : 0;
            id[j] = starts ? s.p[l][k] : 0;
            nx[j] = (starts && l < nlev - 2) ? ls.fidx[l + 1][k] : (int32_t)k;
        }
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (dk[j] > l) continue;
            ls.fids[l][f[j]] = id[j];
            ls.fptr[l][f[j]] = nx[j];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int l = 0; l < kMaxModes - 1; ++l) {
            if (l >= nlev - 1) break;
            const int32_t nl = ls.fidx[l][n];
            ls.fptr[l][nl] = (l == nlev - 2) ? (int32_t)n : ls.fidx[l + 1][n];
        }
    }
}

// lvl[k] = first level whose coordinate changes at k (0 for k = 0).

// part[c*(N-1) + l] = level-l fiber holding leaf c*chunk (binary search up the tree).
struct FptrPtrs {
    const int32_t *p[kMaxModes];
    int64_t n[kMaxModes];
};

__global__ void partition_kernel(FptrPtrs fp, int nlev, int64_t nnz, int32_t chunk, int64_t nchunks,
                                 int32_t *__restrict__ part) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t child = c * (int64_t)chunk;
        for (int l = nlev - 2; l >= 0; --l) {
            // largest f in [0, n_l) with fptr[l][f] <= child
            int64_t lo = 0, hi = fp.n[l];  // invariant: fptr[lo] <= child < fptr[hi]
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (fp.p[l][mid] <= child) lo = mid;
                else hi = mid;
            }
            part[c * (nlev - 1) + l] = (int32_t)lo;
            child = lo;
        }
    }
}

// flag[f] = 1 if slice f's leaves span more than heavy_chunks chunks.
__global__ void heavy_flags_kernel(FptrPtrs fp, int nlev, int64_t nslices, int32_t chunk, int heavy_chunks,
                                   int32_t *__restrict__ flags) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nslices;
         f += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = f, e = f + 1;
        for (int l = 0; l < nlev - 1; ++l) {  // descend to the slice's leaf range [b, e)
            b = fp.p[l][b];
            e = fp.p[l][e];
        }
        const int64_t span = (e - 1) / chunk - b / chunk + 1;
        flags[f] = span > heavy_chunks ? 1 : 0;
    }
}

// hidx[f] = scan[f] where flagged, else -1.
__global__ void heavy_index_kernel(const int32_t *__restrict__ flags, const int32_t *__restrict__ scan,
                                   int64_t nslices, int32_t *__restrict__ hidx) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nslices;
         f += (int64_t)gridDim.x * blockDim.x)
        hidx[f] = flags[f] ? scan[f] : -1;
}

}  // namespace

// ---------------------------------------------------------------------------
// COO helpers
// ---------------------------------------------------------------------------
sptt_status coo_validate_shape(const sptt_coo *coo) {
    if (!coo) return set_error(SPTT_ERR_BAD_ARG, "coo is NULL");
    if (coo->nmodes < 2 || coo->nmodes > kMaxModes)
        return set_error(SPTT_ERR_BAD_ARG, "nmodes must be in [2, " + std::to_string(kMaxModes) + "]");
    if (coo->nnz < 0 || coo->nnz >= (int64_t(1) << 31))
        return set_error(SPTT_ERR_BAD_ARG, "nnz must be in [0, 2^31)");
    if (!coo->dims || !coo->inds) return set_error(SPTT_ERR_BAD_ARG, "dims/inds is NULL");
    for (int m = 0; m < coo->nmodes; ++m) {
        if (coo->dims[m] < 1 || coo->dims[m] > INT32_MAX)
            return set_error(SPTT_ERR_BAD_ARG, "dims[" + std::to_string(m) + "] must be in [1, 2^31-1]");
        if (coo->nnz > 0 && !coo->inds[m])
            return set_error(SPTT_ERR_BAD_ARG, "inds[" + std::to_string(m) + "] is NULL");
    }
    if (coo->nnz > 0 && !coo->vals) return set_error(SPTT_ERR_BAD_ARG, "vals is NULL");
    return SPTT_OK;
}

DevCoo::~DevCoo() {
    for (int m = 0; m < kMaxModes; ++m)
        if (inds_store[m]) dev_free(inds_store[m], st);
    if (vals_store) dev_free(vals_store, st);
}

sptt_status coo_to_device(const sptt_coo *coo, cudaStream_t st, DevCoo *out) {
    SPTT_TRY(coo_validate_shape(coo));
    out->st = st;
    out->coo = *coo;
    for (int m = 0; m < coo->nmodes; ++m) out->dims[m] = coo->dims[m];
    out->coo.dims = out->dims;
    if (coo->on_device) {
        for (int m = 0; m < coo->nmodes; ++m) out->inds_ptrs[m] = coo->inds[m];
        out->coo.inds = out->inds_ptrs;
        return SPTT_OK;
    }
    const int64_t n = coo->nnz;
    for (int m = 0; m < coo->nmodes; ++m) {
        SPTT_TRY(dev_alloc_n(&out->inds_store[m], (size_t)n, st));
        if (n) SPTT_CUDA(cudaMemcpyAsync(out->inds_store[m], coo->inds[m], n * sizeof(int32_t),
                                         cudaMemcpyDefault, st));
        out->inds_ptrs[m] = out->inds_store[m];
    }
    SPTT_TRY(dev_alloc_n(&out->vals_store, (size_t)n, st));
    if (n) SPTT_CUDA(cudaMemcpyAsync(out->vals_store, coo->vals, n * sizeof(float), cudaMemcpyDefault, st));
    out->coo.inds = out->inds_ptrs;
    out->coo.vals = out->vals_store;
    out->coo.on_device = 1;
    return SPTT_OK;
}

void csf_destroy(sptt_csf *c) {
    if (!c) return;
    cudaDeviceSynchronize();  // no pending work may still read the arrays
    for (int l = 0; l < kMaxModes; ++l) {
        if (c->fptr[l]) dev_free(c->fptr[l], nullptr);
        if (c->fids[l]) dev_free(c->fids[l], nullptr);
        if (c->hslot[l]) dev_free(c->hslot[l], nullptr);
        if (c->hrow[l]) dev_free(c->hrow[l], nullptr);
    }
    if (c->vals) dev_free(c->vals, nullptr);
    if (c->lvl) dev_free(c->lvl, nullptr);
    if (c->part) dev_free(c->part, nullptr);
    if (c->hidx) dev_free(c->hidx, nullptr);
    if (c->leafrec) dev_free(c->leafrec, nullptr);
    if (c->err) dev_free(c->err, nullptr);
    delete c;
}

sptt_status csf_ensure_partition(sptt_csf *c, int32_t chunk, cudaStream_t st) {
    if (c->part && c->part_chunk == chunk) return SPTT_OK;
    const int N = c->nmodes;
    const int64_t nnz = c->nfibs[N - 1];
    const int64_t nchunks = (nnz + chunk - 1) / chunk;
    if (c->part) {
        SPTT_CUDA(cudaStreamSynchronize(st));
        dev_free(c->part, st);
        c->part = nullptr;
    }
    if (!c->hidx) SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->hidx),
                       (size_t)(c->nfibs[0] + 64) * sizeof(int32_t), st));
    SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->part),
                       (size_t)(nchunks * (N - 1) + 1) * sizeof(int32_t), st));
    c->part_chunk = chunk;
    c->part_nchunks = nchunks;
    c->nheavy = 0;
    if (nchunks == 0) return SPTT_OK;
    FptrPtrs fp{};
    for (int l = 0; l < N - 1; ++l) {
        fp.p[l] = c->fptr[l];
        fp.n[l] = c->nfibs[l];
    }
    partition_kernel<<<grid_for(nchunks), kThreads, 0, st>>>(fp, N, nnz, chunk, nchunks, c->part);
    SPTT_CHECK_LAUNCH("partition_kernel");
    const int64_t ns = c->nfibs[0];
    DevBuf flags, scan;
    SPTT_TRY(flags.alloc<int32_t>(ns, st));
    SPTT_TRY(scan.alloc<int32_t>(ns + 1, st));
    heavy_flags_kernel<<<grid_for(ns), kThreads, 0, st>>>(fp, N, ns, chunk, kHeavyChunks, flags.as<int32_t>());
    SPTT_CHECK_LAUNCH("heavy_flags_kernel");
    SPTT_TRY(scan_exclusive_i32(flags.as<int32_t>(), scan.as<int32_t>(), ns, true, st));
    heavy_index_kernel<<<grid_for(ns), kThreads, 0, st>>>(flags.as<int32_t>(), scan.as<int32_t>(), ns, c->hidx);
    SPTT_CHECK_LAUNCH("heavy_index_kernel");
    int32_t nh = 0;
    SPTT_CUDA(cudaMemcpyAsync(&nh, scan.as<int32_t>() + ns, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    c->nheavy = nh;
    return SPTT_OK;
}

namespace {

__global__ void __launch_bounds__(kThreads) leafrec_kernel(const int32_t *__restrict__ idx, const float *__restrict__ vals,
                                                           const uint8_t *__restrict__ lvl, int64_t nnz,
                                                           uint4 *__restrict__ rec) {
    uint32_t x[kItems], v[kItems], d[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        const bool in = k < nnz;
        x[j] = in ? (uint32_t)idx[k] : 0u;
        v[j] = in ? __float_as_uint(vals[k]) : 0u;
        d[j] = in ? (uint32_t)lvl[k] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t k = item_index(j);
        if (k < nnz) rec[k] = make_uint4(x[j], v[j], 0u, d[j]);
    }
}

// The slack records after the last leaf: value 0, leaf row 0, and the level
// flag N-1 (a leaf that opens no fiber), so a walk's last batch may run past
// the end and add nothing.
__global__ void leafrec_slack_kernel(uint4 *__restrict__ rec, int n, uint32_t flag) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) rec[k] = make_uint4(0u, 0u, 0u, flag);
}

// The leaf that starts level-LF fiber f carries that fiber's index.
__global__ void leafrec_fiber_kernel(const int32_t *__restrict__ fptr, const int32_t *__restrict__ fids, int64_t nf,
                                     uint4 *__restrict__ rec) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x)
        rec[fptr[f]].z = (uint32_t)fids[f];
}

}  // namespace

sptt_status csf_ensure_leafrec(sptt_csf *c, cudaStream_t st) {
    if (c->leafrec) return SPTT_OK;
    const int N = c->nmodes;
    const int64_t nnz = c->nfibs[N - 1];
    SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->leafrec),
                       (size_t)(nnz + kLeafSlack) * sizeof(uint4), st));
    leafrec_slack_kernel<<<(kLeafSlack + kThreads - 1) / kThreads, kThreads, 0, st>>>(c->leafrec + nnz, kLeafSlack,
                                                                                    (uint32_t)(N - 1));
    SPTT_CHECK_LAUNCH("leafrec_slack_kernel");
    if (nnz > 0) {
        leafrec_kernel<<<grid_items(nnz), kThreads, 0, st>>>(c->fids[N - 1], c->vals, c->lvl, nnz, c->leafrec);
        SPTT_CHECK_LAUNCH("leafrec_kernel");
        if (N >= 3) {
            // level N-2 fibers: fptr[N-2][f] is the first leaf of fiber f
            const int LF = N - 2;
            leafrec_fiber_kernel<<<grid_for(c->nfibs[LF]), kThreads, 0, st>>>(c->fptr[LF], c->fids[LF], c->nfibs[LF],
                                                                              c->leafrec);
            SPTT_CHECK_LAUNCH("leafrec_fiber_kernel");
        }
    }
    return SPTT_OK;
}

void level_order(const int64_t *dims, int nmodes, int root, int kind, int32_t *order) {
    order[0] = root;
    int k = 1;
    for (int m = 0; m < nmodes; ++m)
        if (m != root) order[k++] = m;
    for (int a = 2; a < nmodes; ++a)  // stable insertion sort of levels 1..
        for (int b = a; b > 1; --b) {
            const int64_t x = dims[order[b]], y = dims[order[b - 1]];
            if (!(kind == 1 ? x > y : x < y)) break;
            const int32_t t = order[b];
            order[b] = order[b - 1];
            order[b - 1] = t;
        }
    if (kind == 2 && nmodes > 2) {
        // ascending below the root; the shortest (now at level 1) moves to the leaves
        const int32_t s = order[1];
        for (int l = 1; l < nmodes - 1; ++l) order[l] = order[l + 1];
        order[nmodes - 1] = s;
    }
}

sptt_status csf_build_device(const sptt_coo *coo, int32_t root, const int32_t *order_in,
                             cudaStream_t st, sptt_csf **out) {
    const int N = coo->nmodes;
    const int64_t n = coo->nnz;
    int32_t order[kMaxModes];
    if (order_in) {
        bool seen[kMaxModes] = {false};
        for (int l = 0; l < N; ++l) {
            if (order_in[l] < 0 || order_in[l] >= N || seen[order_in[l]])
                return set_error(SPTT_ERR_BAD_ARG, "level_order must be a permutation of the modes");
            seen[order_in[l]] = true;
            order[l] = order_in[l];
        }
        if (order[0] != root) return set_error(SPTT_ERR_BAD_ARG, "level_order[0] must be root_mode");
    } else {
        level_order(coo->dims, N, root, 0, order);
    }

    sptt_csf *c = new sptt_csf();
    c->nmodes = N;
    c->root = root;
    for (int m = 0; m < N; ++m) c->dims[m] = coo->dims[m];
    for (int l = 0; l < N; ++l) c->order[l] = order[l];
    struct Guard {
        sptt_csf *c;
        ~Guard() { if (c) csf_destroy(c); }
    } guard{c};

    // 1. the indices are checked while the sort keys are built (step 2); the
    // error word and the duplicate count are read back together (step 4)
    DevBuf word;  // [0] index error flag (int32), [1] duplicate count (u64)
    SPTT_TRY(word.alloc<unsigned long long>(2, st));
    SPTT_TRY(fill_zero_launch(word.p, 2 * sizeof(unsigned long long), st));
    int32_t *d_err = reinterpret_cast<int32_t *>(word.as<unsigned long long>());
    unsigned long long *d_ndup = word.as<unsigned long long>() + 1;

    // 2. sort positions by level-ordered keys, least significant word first
    const int32_t *lev_src[kMaxModes];
    for (int l = 0; l < N; ++l) lev_src[l] = coo->inds[order[l]];
    DevBuf kA, kB, vA, vB;
    uint32_t *perm = nullptr;
    uint32_t *sorted_bits = nullptr;  // the values, when the sort carried them
    uint64_t *sorted_keys = nullptr;
    Decode dec{};
    for (int j = 0; j < kMaxModes; ++j) dec.shift[j] = -1;
    if (n > 0) {
        SPTT_TRY(kA.alloc<uint64_t>(n, st));
        SPTT_TRY(kB.alloc<uint64_t>(n, st));
        SPTT_TRY(vA.alloc<uint32_t>(n, st));
        SPTT_TRY(vB.alloc<uint32_t>(n, st));
        uint64_t *keys = kA.as<uint64_t>(), *keys_alt = kB.as<uint64_t>();
        uint32_t *vals = vA.as<uint32_t>(), *vals_alt = vB.as<uint32_t>();
        int l = N - 1;
        bool first = true;
        while (l >= 0) {
            KeyGroup g{};
            int bits = 0;
            // take levels l, l-1, ... while they fit in 64 bits (at least one)
            int lo_level = l;
            while (lo_level >= 0 && (bits + bits_for(c->dims[order[lo_level]]) <= 64 || lo_level == l)) {
                bits += bits_for(c->dims[order[lo_level]]);
                --lo_level;
            }
            int shift = 0;
            const bool last = lo_level < 0;  // this group holds level 0: it is sorted last
            for (int j = l; j > lo_level; --j) {  // leaf-most level in the low bits
                const int b = bits_for(c->dims[order[j]]);
                if (last) {
                    dec.shift[j] = shift;
                    dec.bits[j] = b;
                }
                g.chk[g.nchk] = lev_src[j];
                g.dim[g.nchk] = c->dims[order[j]];
                g.shift[g.nchk] = b ? shift : -1;  // a length-1 mode contributes no key bits
                ++g.nchk;
                shift += b;
            }
            const bool carry = first && last;  // one group: the sort carries the values
            build_keys_kernel<<<grid_items(n), kThreads, 0, st>>>(g, first ? nullptr : vals, n, keys_alt,
                                                                vals_alt, d_err, carry ? coo->vals : nullptr);
            SPTT_CHECK_LAUNCH("build_keys_kernel");
            {
                uint64_t *t = keys; keys = keys_alt; keys_alt = t;
                uint32_t *tv = vals; vals = vals_alt; vals_alt = tv;
            }
            SPTT_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, bits, st));
            if (carry) sorted_bits = vals;
            first = false;
            l = lo_level;
        }
        perm = sorted_bits ? nullptr : vals;
        sorted_keys = keys;
    }

    // 3. gather sorted coordinates (level order) and values
    std::vector<DevBuf> s_store(N);
    DevBuf sv_store;
    IdxPtrs s{};
    OutPtrs so{};
    if (n > 0) {
        for (int l = 0; l < N; ++l) {
            SPTT_TRY(s_store[l].alloc<int32_t>(n, st));
            so.p[l] = s_store[l].as<int32_t>();
            s.p[l] = so.p[l];
        }
        SPTT_TRY(sv_store.alloc<float>(n, st));
        IdxPtrs lp{};
        for (int l = 0; l < N; ++l) lp.p[l] = lev_src[l];
        gather_sorted_kernel<<<grid_items(n), kThreads, 0, st>>>(lp, N, coo->vals, perm, sorted_bits, sorted_keys,
                                                               dec, n, so, sv_store.as<float>());
        SPTT_CHECK_LAUNCH("gather_sorted_kernel");
    }
    kA.reset();
    kB.reset();
    vA.reset();
    vB.reset();

    // 4. coalesce duplicates. dlev[k] = first level whose index differs from
    // position k - 1 (N: a duplicate); it gives the fiber starts of every
    // level and the CSF's per-leaf level flags.
    int64_t u = n;
    DevBuf flags, scan, dlev;
    float *sv = sv_store.as<float>();
    std::vector<DevBuf> c_store(N);
    DevBuf cv_store;
    if (n > 0) {
        SPTT_TRY(dlev.alloc<uint8_t>(n, st));
        level_diff_kernel<<<grid_items(n), kThreads, 0, st>>>(s, N, n, dlev.as<uint8_t>(), d_ndup);
        SPTT_CHECK_LAUNCH("level_diff_kernel");
        unsigned long long hw[2] = {0, 0};
        SPTT_CUDA(cudaMemcpyAsync(hw, word.p, sizeof(hw), cudaMemcpyDeviceToHost, st));
        SPTT_CUDA(cudaStreamSynchronize(st));
        if ((int32_t)(hw[0] & 0xffffffffu))
            return set_error(SPTT_ERR_BAD_ARG, "an index is outside [0, dim) of its mode");
        SPTT_TRY(flags.alloc<int32_t>(n, st));
        SPTT_TRY(scan.alloc<int32_t>(n + 1, st));
        if (hw[1] > 0) {  // duplicates: sum each run, then the level bytes of the coalesced tensor
            prefix_flags_kernel<<<grid_for(n), kThreads, 0, st>>>(s, N - 1, n, flags.as<int32_t>());
            SPTT_CHECK_LAUNCH("prefix_flags_kernel");
            SPTT_TRY(scan_exclusive_i32(flags.as<int32_t>(), scan.as<int32_t>(), n, true, st));
            u = n - (int64_t)hw[1];
            DevBuf starts;
            SPTT_TRY(starts.alloc<int32_t>(u + 1, st));
            run_starts_kernel<<<grid_for(n), kThreads, 0, st>>>(scan.as<int32_t>(), n, starts.as<int32_t>());
            SPTT_CHECK_LAUNCH("run_starts_kernel");
            OutPtrs co{};
            for (int l = 0; l < N; ++l) {
                SPTT_TRY(c_store[l].alloc<int32_t>(u, st));
                co.p[l] = c_store[l].as<int32_t>();
            }
            SPTT_TRY(cv_store.alloc<float>(u, st));
            coalesce_kernel<<<grid_for(u), kThreads, 0, st>>>(s, N, sv, starts.as<int32_t>(), u, n, co,
                                                             cv_store.as<float>());
            SPTT_CHECK_LAUNCH("coalesce_kernel");
            for (int l = 0; l < N; ++l) s.p[l] = co.p[l];
            sv = cv_store.as<float>();
            level_diff_kernel<<<grid_items(u), kThreads, 0, st>>>(s, N, u, dlev.as<uint8_t>(), d_ndup);
            SPTT_CHECK_LAUNCH("level_diff_kernel");
        }
    }

    // 5. fiber levels
    c->nfibs[N - 1] = u;
    std::vector<DevBuf> fidx(N);
    if (u > 0) {
        for (int l = 0; l < N - 1; ++l) {
            SPTT_TRY(fidx[l].alloc<int32_t>(u + 1, st));
            SPTT_TRY(scan_exclusive_level(dlev.as<uint8_t>(), l, fidx[l].as<int32_t>(), u, true, st));
        }
        std::vector<int32_t> tot(N, 0);
        for (int l = 0; l < N - 1; ++l)
            SPTT_CUDA(cudaMemcpyAsync(&tot[l], fidx[l].as<int32_t>() + u, sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, st));
        SPTT_CUDA(cudaStreamSynchronize(st));
        for (int l = 0; l < N - 1; ++l) c->nfibs[l] = tot[l];
    }
    for (int l = 0; l < N - 1; ++l) {
        SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->fptr[l]),
                       (size_t)(c->nfibs[l] + 1 + 64) * sizeof(int32_t), st));
        SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->fids[l]),
                       (size_t)(c->nfibs[l] + 64) * sizeof(int32_t), st));
    }
    SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->fids[N - 1]),
                       (size_t)(u + kLeafSlack) * sizeof(int32_t), st));
    SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->vals),
                       (size_t)(u + kLeafSlack) * sizeof(float), st));
    SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->lvl),
                       (size_t)(u + kLeafSlack), st));
    SPTT_TRY(dev_alloc(reinterpret_cast<void **>(&c->err),
                       sizeof(int32_t), st));
    SPTT_TRY(fill_zero_launch(c->err, sizeof(int32_t), st));
    if (u > 0) {
        LevelScan ls{};
        for (int l = 0; l < N - 1; ++l) {
            ls.fidx[l] = fidx[l].as<int32_t>();
            ls.fids[l] = c->fids[l];
            ls.fptr[l] = c->fptr[l];
        }
        fill_levels_kernel<<<grid_items(u), kThreads, 0, st>>>(s, ls, dlev.as<uint8_t>(), N, u);
        SPTT_CHECK_LAUNCH("fill_levels_kernel");
        SPTT_CUDA(cudaMemcpyAsync(c->lvl, dlev.p, (size_t)u, cudaMemcpyDeviceToDevice, st));
        SPTT_CUDA(cudaMemcpyAsync(c->fids[N - 1], s.p[N - 1], u * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        SPTT_CUDA(cudaMemcpyAsync(c->vals, sv, u * sizeof(float), cudaMemcpyDeviceToDevice, st));
    } else {
        for (int l = 0; l < N - 1; ++l) SPTT_TRY(fill_zero_launch(c->fptr[l], sizeof(int32_t), st));
    }
    SPTT_CUDA(cudaStreamSynchronize(st));
    guard.c = nullptr;
    *out = c;
    return SPTT_OK;
}

}  // namespace sptt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace sptt;

extern "C" sptt_status sptt_csf_build(const sptt_coo *coo, int32_t root_mode, const int32_t *level_order,
                                      sptt_stream stream, sptt_csf **out) {
    clear_error();
    if (!out) return set_error(SPTT_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    SPTT_TRY(coo_validate_shape(coo));
    if (root_mode < 0 || root_mode >= coo->nmodes) return set_error(SPTT_ERR_BAD_ARG, "root_mode out of range");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevCoo dc;
    SPTT_TRY(coo_to_device(coo, st, &dc));
    return csf_build_device(&dc.coo, root_mode, level_order, st, out);
}

extern "C" void sptt_csf_free(sptt_csf *csf) { csf_destroy(csf); }

extern "C" sptt_status sptt_csf_shape(const sptt_csf *csf, int32_t *nmodes, int32_t *order, int64_t *nfibs) {
    clear_error();
    if (!csf) return set_error(SPTT_ERR_BAD_ARG, "csf is NULL");
    if (nmodes) *nmodes = csf->nmodes;
    for (int l = 0; l < csf->nmodes; ++l) {
        if (order) order[l] = csf->order[l];
        if (nfibs) nfibs[l] = csf->nfibs[l];
    }
    return SPTT_OK;
}

extern "C" sptt_status sptt_csf_check(const sptt_csf *csf, sptt_stream stream) {
    clear_error();
    if (!csf) return set_error(SPTT_ERR_BAD_ARG, "csf is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t e = 0;
    SPTT_CUDA(cudaMemcpyAsync(&e, csf->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    if (e) {
        SPTT_TRY(fill_zero_launch(csf->err, sizeof(int32_t), st));
        return set_error(SPTT_ERR_TIMEOUT, "a bounded wait of an MTTKRP on this CSF ran out");
    }
    return SPTT_OK;
}

extern "C" sptt_status sptt_csf_copy_level(const sptt_csf *csf, int32_t level, int32_t *fptr, int32_t *fids,
                                           float *vals, sptt_stream stream) {
    clear_error();
    if (!csf) return set_error(SPTT_ERR_BAD_ARG, "csf is NULL");
    const int N = csf->nmodes;
    if (level < 0 || level >= N) return set_error(SPTT_ERR_BAD_ARG, "level out of range");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t nl = csf->nfibs[level];
    if (fptr) {
        if (level == N - 1) return set_error(SPTT_ERR_BAD_ARG, "the leaf level has no fptr");
        SPTT_CUDA(cudaMemcpyAsync(fptr, csf->fptr[level], (nl + 1) * sizeof(int32_t), cudaMemcpyDefault, st));
    }
    if (fids && nl) SPTT_CUDA(cudaMemcpyAsync(fids, csf->fids[level], nl * sizeof(int32_t), cudaMemcpyDefault, st));
    if (vals) {
        if (level != N - 1) return set_error(SPTT_ERR_BAD_ARG, "vals live on the leaf level");
        if (nl) SPTT_CUDA(cudaMemcpyAsync(vals, csf->vals, nl * sizeof(float), cudaMemcpyDefault, st));
    }
    SPTT_CUDA(cudaStreamSynchronize(st));
    return SPTT_OK;
}
