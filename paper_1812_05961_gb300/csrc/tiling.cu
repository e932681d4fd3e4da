// Mode tiling of the root-mode MTTKRP (the SPLATT option the paper's port
// leaves out, Section V and the conclusion).
//
// The non-zeros of a tensor are split by the index they carry in the mode at
// the CSF's leaves: tile t holds the non-zeros whose leaf index lies in
// [t * rows, (t + 1) * rows), rebased to start at 0. Each tile is a CSF of
// its own with the same root and level order, whose leaf factor is the row
// block A^(leaf)[t * rows, ...) - small enough for the table kernels to keep
// in shared memory. The MTTKRP is linear in the non-zeros, so the root-mode
// MTTKRP of the tensor is the sum over tiles of the tiles' MTTKRPs:
//   M[i, :] = sum_t sum_{non-zeros of tile t in slice i} v * prod_m A^(m)[i_m, :].
// Each tile's compact result (one row per slice of that tile) is added into
// a full result (one row per root index) tile after tile, in tile order, so
// the sum does not depend on timing.
#include <vector>

#include "walk.cuh"

namespace sptt {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// counts[t] += number of non-zeros whose leaf index falls in tile t
// (per-CTA shared histogram, then one atomic per tile per CTA).
// An index outside [0, dleaf) is not counted (the caller compares the total
// with nnz and rejects the tensor).
__global__ void tile_hist_kernel(const int32_t *__restrict__ leaf, int64_t n, int64_t dleaf, int32_t rows,
                                 int32_t ntiles, unsigned long long *__restrict__ counts) {
    extern __shared__ unsigned long long sh[];
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) sh[t] = 0ull;
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = __ldg(leaf + k);
        if (x >= 0 && x < dleaf) atomicAdd(&sh[x / rows], 1ull);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        if (sh[t]) atomicAdd(counts + t, sh[t]);
}

// key = tile of non-zero k, value = k (a stable sort by key groups the tiles)
__global__ void tile_keys_kernel(const int32_t *__restrict__ leaf, int64_t n, int32_t rows,
                                 uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        keys[k] = (uint64_t)(__ldg(leaf + k) / rows);
        vals[k] = (uint32_t)k;
    }
}

struct IdxSet {
    const int32_t *src[kMaxModes];
    int32_t *dst[kMaxModes];
};

// Non-zeros in tile order: indices and values gathered through perm, the
// leaf index rebased to its tile.
__global__ void tile_gather_kernel(const uint32_t *__restrict__ perm, int64_t n, IdxSet ix, int nmodes, int leaf_mode,
                                   int32_t rows, const float *__restrict__ vals, float *__restrict__ vals_out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = __ldg(perm + k);
        for (int m = 0; m < nmodes; ++m) {
            const int32_t x = __ldg(ix.src[m] + s);
            ix.dst[m][k] = m == leaf_mode ? x % rows : x;
        }
        vals_out[k] = __ldg(vals + s);
    }
}

// out[fids0[f] * ld + c] += row f of a tile's compact MTTKRP (its FP64 row
// where the slice has one); one tile's slices have distinct root indices.
__global__ void tile_accumulate_kernel(const float *__restrict__ compact, const double *__restrict__ heavy,
                                       const int32_t *__restrict__ hidx, const int32_t *__restrict__ fids0,
                                       int64_t nrows, int ld, float *__restrict__ out) {
    const int64_t n = nrows * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e / ld;
        const int c = (int)(e - f * ld);
        out[(int64_t)__ldg(fids0 + f) * ld + c] += walk::read_row(compact, heavy, hidx, f, ld, c);
    }
}

}  // namespace

sptt_status tiles_build(const sptt_coo *coo_dev, int32_t root, const int32_t *order, int32_t rows,
                        cudaStream_t st, std::vector<sptt_csf *> *csfs, std::vector<int64_t> *base) {
    const int N = coo_dev->nmodes;
    const int leaf = order[N - 1];
    const int64_t n = coo_dev->nnz;
    const int64_t dleaf = coo_dev->dims[leaf];
    const int32_t ntiles = (int32_t)((dleaf + rows - 1) / rows);
    if (ntiles < 1 || ntiles > kMaxTiles) return set_error(SPTT_ERR_BAD_ARG, "tile count outside [1, kMaxTiles]");
    std::vector<unsigned long long> counts(ntiles, 0ull);
    DevBuf dcount;
    SPTT_TRY(dcount.alloc<unsigned long long>(ntiles, st));
    SPTT_TRY(fill_zero_launch(dcount.p, ntiles * sizeof(unsigned long long), st));
    DevBuf keys, vals, keys_alt, vals_alt, gvals;
    DevBuf gidx[kMaxModes];
    if (n > 0) {
        tile_hist_kernel<<<grid_for(n), kThreads, ntiles * sizeof(unsigned long long), st>>>(
            coo_dev->inds[leaf], n, dleaf, rows, ntiles, dcount.as<unsigned long long>());
        SPTT_CHECK_LAUNCH("tile_hist_kernel");
    }
    SPTT_CUDA(cudaMemcpyAsync(counts.data(), dcount.p, ntiles * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    int64_t total = 0;
    for (auto x : counts) total += (int64_t)x;
    if (total != n) return set_error(SPTT_ERR_BAD_ARG, "a leaf index is out of range");
    if (n > 0) {
        SPTT_TRY(keys.alloc<uint64_t>(n, st));
        SPTT_TRY(vals.alloc<uint32_t>(n, st));
        SPTT_TRY(keys_alt.alloc<uint64_t>(n, st));
        SPTT_TRY(vals_alt.alloc<uint32_t>(n, st));
        tile_keys_kernel<<<grid_for(n), kThreads, 0, st>>>(coo_dev->inds[leaf], n, rows, keys.as<uint64_t>(),
                                                           vals.as<uint32_t>());
        SPTT_CHECK_LAUNCH("tile_keys_kernel");
        uint64_t *k = keys.as<uint64_t>(), *ka = keys_alt.as<uint64_t>();
        uint32_t *v = vals.as<uint32_t>(), *va = vals_alt.as<uint32_t>();
        int nbits = 1;
        while ((int64_t(1) << nbits) < ntiles) ++nbits;
        SPTT_TRY(radix_sort_pairs(k, v, ka, va, n, nbits, st));
        IdxSet ix{};
        for (int m = 0; m < N; ++m) {
            SPTT_TRY(gidx[m].alloc<int32_t>(n, st));
            ix.src[m] = coo_dev->inds[m];
            ix.dst[m] = gidx[m].as<int32_t>();
        }
        SPTT_TRY(gvals.alloc<float>(n, st));
        tile_gather_kernel<<<grid_for(n), kThreads, 0, st>>>(v, n, ix, N, leaf, rows, coo_dev->vals, gvals.as<float>());
        SPTT_CHECK_LAUNCH("tile_gather_kernel");
    }
    int64_t off = 0;
    for (int32_t t = 0; t < ntiles; ++t) {
        const int64_t cnt = (int64_t)counts[t];
        if (cnt == 0) {
            off += cnt;
            continue;
        }
        int64_t dims[kMaxModes];
        const int32_t *ptrs[kMaxModes];
        for (int m = 0; m < N; ++m) {
            dims[m] = coo_dev->dims[m];
            ptrs[m] = gidx[m].as<int32_t>() + off;
        }
        const int64_t b0 = (int64_t)t * rows;
        dims[leaf] = (dleaf - b0 < rows) ? dleaf - b0 : rows;
        sptt_coo sub{};
        sub.nmodes = N;
        sub.nnz = cnt;
        sub.dims = dims;
        sub.inds = ptrs;
        sub.vals = gvals.as<float>() + off;
        sub.on_device = 1;
        sptt_csf *c = nullptr;
        SPTT_TRY(csf_build_device(&sub, root, order, st, &c));
        csfs->push_back(c);
        base->push_back(b0);
        off += cnt;
    }
    SPTT_CUDA(cudaStreamSynchronize(st));  // the gathered arrays are freed on return
    return SPTT_OK;
}

sptt_status tile_accumulate_launch(const sptt_csf *tile, const float *compact, const double *heavy, int32_t ld,
                                   float *out, cudaStream_t st) {
    const int64_t ns = tile->nfibs[0];
    if (ns == 0) return SPTT_OK;
    tile_accumulate_kernel<<<grid_for(ns * ld), kThreads, 0, st>>>(compact, heavy, tile->hidx, tile->fids[0], ns, ld,
                                                                    out);
    SPTT_CHECK_LAUNCH("tile_accumulate_kernel");
    return SPTT_OK;
}

}  // namespace sptt
