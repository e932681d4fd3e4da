// Internal declarations shared by the CUDA translation units of libsptt.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sptt.h"

namespace sptt {

constexpr int kMaxModes = SPTT_MAX_MODES;
// A slice whose leaves span more than kHeavyChunks chunks gets an FP64
// output row: with 1, every slice cut by a chunk boundary. Its per-chunk
// FP32 partials are then summed in FP64, exactly whenever they lie within
// 2^29 of each other in magnitude, so the result does not depend on the order
// in which the chunks finish.
constexpr int kHeavyChunks = 1;
constexpr int kMaxVariant = 15;  // largest sptt_sched::variant
constexpr int kLeafSlack = 512;  // elements past the end of every leaf array (whole-chunk copies)
constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (queried at run time where it matters)

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
sptt_status set_error(sptt_status s, const std::string &msg);
sptt_status cuda_error(cudaError_t e, const char *what);
void clear_error();
void count_launch(int64_t n = 1);

#define SPTT_CUDA(call)                                        \
    do {                                                       \
        cudaError_t e__ = (call);                              \
        if (e__ != cudaSuccess) return ::sptt::cuda_error(e__, #call); \
    } while (0)

// Every kernel launch site is followed by this check, which also counts the
// launch (sptt_debug_launch_count).
#define SPTT_CHECK_LAUNCH(what)                                \
    do {                                                       \
        ::sptt::count_launch();                                \
        cudaError_t e__ = cudaGetLastError();                  \
        if (e__ != cudaSuccess) return ::sptt::cuda_error(e__, what); \
    } while (0)

#define SPTT_TRY(expr)                                         \
    do {                                                       \
        sptt_status s__ = (expr);                              \
        if (s__ != SPTT_OK) return s__;                        \
    } while (0)

// ---------------------------------------------------------------------------
// Device memory (stream-ordered)
// ---------------------------------------------------------------------------
sptt_status dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

template <typename T>
sptt_status dev_alloc_n(T **p, size_t n, cudaStream_t st) {
    // 64 elements of slack so vector loads past the logical end stay inside the allocation
    return dev_alloc(reinterpret_cast<void **>(p), (n + 64) * sizeof(T), st);
}

// RAII holder for temporaries of one call.
struct DevBuf {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    void reset() {
        if (p) dev_free(p, st);
        p = nullptr;
    }
    template <typename T>
    sptt_status alloc(size_t n, cudaStream_t s) {
        st = s;
        return dev_alloc_n(reinterpret_cast<T **>(&p), n, s);
    }
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

int device_sm_count();

// ---------------------------------------------------------------------------
// Scan and radix sort (sort.cu)
// ---------------------------------------------------------------------------
// Exclusive prefix sum of n int32 values; out[n] (if with_total) = total.
// Workspace is allocated internally on the stream.
sptt_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, bool with_total,
                               cudaStream_t st);
// The same scan of the predicate d[i] <= level over a byte array.
sptt_status scan_exclusive_level(const uint8_t *d, int level, int32_t *out, int64_t n, bool with_total,
                                 cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs by the low `nbits` bits of key,
// ping-ponging between (keys, vals) and (keys_alt, vals_alt); on return
// keys/vals point at the sorted data (the pointers may have been swapped).
sptt_status radix_sort_pairs(uint64_t *&keys, uint32_t *&vals, uint64_t *&keys_alt,
                             uint32_t *&vals_alt, int64_t n, int nbits, cudaStream_t st);

// ---------------------------------------------------------------------------
// CSF (csf.cu)
// ---------------------------------------------------------------------------
}  // namespace sptt

struct sptt_csf {
    int32_t nmodes = 0;
    int32_t root = 0;
    int32_t order[SPTT_MAX_MODES] = {0};
    int64_t dims[SPTT_MAX_MODES] = {0};     // by mode
    int64_t nfibs[SPTT_MAX_MODES] = {0};    // by level; nfibs[N-1] = nnz
    int32_t *fptr[SPTT_MAX_MODES] = {nullptr};  // levels 0..N-2
    int32_t *fids[SPTT_MAX_MODES] = {nullptr};  // levels 0..N-1
    float *vals = nullptr;
    // lvl[k] = the first tree level whose fiber changes at leaf k (0 for
    // k = 0; N-1 when only the leaf index changes). Lets the MTTKRP walk
    // find fiber boundaries from the leaf stream alone.
    uint8_t *lvl = nullptr;
    // Work partition for the MTTKRP kernels: for leaf chunk c (leaves
    // [c*part_chunk, ...)), part[c*(N-1) + l] = the level-l fiber holding
    // the chunk's first leaf. Rebuilt when another chunk size is requested.
    int32_t *part = nullptr;
    int32_t part_chunk = 0;
    int64_t part_nchunks = 0;
    // Heavy slices: those whose leaves span more than kHeavyChunks chunks of
    // the partition (every split slice). hidx[f] = index of slice f among the
    // heavy ones, or -1; their MTTKRP partials are summed in FP64 (walk.cuh).
    int32_t *hidx = nullptr;
    int64_t nheavy = 0;
    // Device error word of the kernels that read this CSF (bit 2: a bounded
    // wait for a staged copy ran out); read by sptt_csf_check.
    int32_t *err = nullptr;
    // Hot rows of the MTTKRP for the mode at level l >= 1 (mttkrp_mode.cu):
    // hslot[l][i] = shared-memory slot of row i or -1, hrow[l][s] = row of
    // slot s; built for a row width whose slot capacity is hot_cap[l].
    // Packed leaf records of the flag walk (walk.cuh PackedRecs): per leaf
    // {leaf index, value bits, index of the level-(N-2) fiber it opens or 0,
    // level flag}, with kLeafSlack records {0, 0, 0, N-1} (value zero, opens
    // nothing) after the last; built on first use.
    uint4 *leafrec = nullptr;
    int32_t *hslot[SPTT_MAX_MODES] = {nullptr};
    int32_t *hrow[SPTT_MAX_MODES] = {nullptr};
    int32_t nhot[SPTT_MAX_MODES] = {0};
    int32_t hot_cap[SPTT_MAX_MODES] = {0};
};

namespace sptt {

sptt_status csf_build_device(const sptt_coo *coo_dev, int32_t root, const int32_t *order,
                             cudaStream_t st, sptt_csf **out);
// Level order of a CSF rooted at `root`: the root, then the other modes by
// ascending (kind 0) or descending (kind 1) length, ties to the lower mode
// id; kind 2: the shortest non-root mode at the leaves and the others above
// it by ascending length (ties as before).
void level_order(const int64_t *dims, int nmodes, int root, int kind, int32_t *order);
sptt_status csf_ensure_partition(sptt_csf *csf, int32_t chunk, cudaStream_t st);
sptt_status csf_ensure_leafrec(sptt_csf *csf, cudaStream_t st);
void csf_destroy(sptt_csf *c);

// Copy a host COO to the device (arrays owned by the returned holder).
struct DevCoo {
    sptt_coo coo{};
    int32_t *inds_store[kMaxModes] = {nullptr};
    const int32_t *inds_ptrs[kMaxModes] = {nullptr};
    float *vals_store = nullptr;
    int64_t dims[kMaxModes] = {0};
    cudaStream_t st = nullptr;
    ~DevCoo();
};
sptt_status coo_validate_shape(const sptt_coo *coo);
sptt_status coo_to_device(const sptt_coo *coo, cudaStream_t st, DevCoo *out);

// ---------------------------------------------------------------------------
// MTTKRP (mttkrp.cu)
// ---------------------------------------------------------------------------
// out: compact FP32 (nfibs[0] x ld), heavy: FP64 (nheavy x ld); both are
// zeroed here, then filled. Call mttkrp_prepare first (it sets nheavy).
sptt_status mttkrp_launch(sptt_csf *csf, const void *const *factors, int32_t dtype, int32_t ld,
                          float *out, double *heavy, const sptt_sched *sched, cudaStream_t st);
// Builds the work partition the launch will use (allocates on first use, so
// call it before any stream capture).
sptt_status mttkrp_prepare(sptt_csf *csf, const sptt_sched *sched, cudaStream_t st);
// Leaves per chunk when the schedule does not say (depends on nnz and the SM count).
int32_t default_chunk(int64_t nnz);
// Largest leaf-factor copy the table kernels (variants 14, 15) keep in shared
// memory; the rest of an SM's 228 KB stays L1 for the records and the rows
// of the fibers above the leaves.
constexpr size_t kTableMaxBytes = 160 * 1024;
// Whether a leaf factor of leaf_rows rows of ld elements of esz bytes fits.
bool leaf_table_fits(int64_t leaf_rows, int32_t ld, int esz);
// Smallest tensor for which the defaults take the table kernel: on smaller
// tensors, and on any tensor of 4 or more modes (whose leaf-parent fibers are
// tuples of 3 or more indices, nearly one per leaf), putting the shortest mode
// at the leaves multiplies the fibers more than the shared-memory table saves.
constexpr int64_t kTableMinNnz = int64_t(1) << 25;
// Smallest tensor for which the FP32 defaults take the 32-byte-segment walk
// (variant 12) where the row width allows it (ld >= 16, ld % 8 == 0): on
// smaller tensors the 16-byte walk in batches of 4 keeps more leaves in
// flight per SM than the grid has chunks to spare.
constexpr int64_t kWideMinNnz = int64_t(1) << 23;
// The default MTTKRP variant for a gather type, row width, leaf-mode length,
// size and mode count: the table kernel (14 FP32, 15 BF16) for a 3-mode
// tensor of at least kTableMinNnz non-zeros whose leaf factor fits, else 12
// for FP32 gathers on a tensor of at least kWideMinNnz non-zeros with a row
// width that allows it, else 13.
int default_variant(int32_t dtype, int32_t ld, int64_t leaf_rows, int64_t nnz, int nmodes);
// The default CSF level-order kind of the CSF rooted at `root` (see
// level_order): on a 3-mode tensor of at least kTableMinNnz non-zeros, 2
// when the shortest other mode's factor (in the gather type) fits the
// shared-memory table, else 0.
int default_order_kind(const int64_t *dims, int nmodes, int root, int32_t ld, int32_t dtype, int64_t nnz);

// MTTKRP for the mode at level L >= 1 of the CSF (mttkrp_mode.cu): out is
// full (dims[order[L]] x ld FP32), zeroed here, then filled. Call
// mttkrp_mode_prepare first (partition and hot-row table; synchronises).
sptt_status mttkrp_mode_prepare(sptt_csf *csf, int32_t L, int32_t ld, const sptt_sched *sched, cudaStream_t st);
sptt_status mttkrp_mode_launch(sptt_csf *csf, int32_t L, const void *const *factors, int32_t dtype, int32_t ld,
                               float *out, const sptt_sched *sched, cudaStream_t st);
int csf_level_of(const sptt_csf *csf, int32_t mode);

// ---------------------------------------------------------------------------
// Mode tiling (tiling.cu)
// ---------------------------------------------------------------------------
constexpr int kMaxTiles = 1024;
// The CSFs (rooted at `root`, level order `order`) of the tiles of a device
// COO whose leaf-mode index lies in [t * rows, (t + 1) * rows), leaf index
// rebased; base[i] = the first leaf index of csfs[i]'s tile (empty tiles are
// skipped). BAD_ARG for an index out of range. Synchronises.
sptt_status tiles_build(const sptt_coo *coo_dev, int32_t root, const int32_t *order, int32_t rows,
                        cudaStream_t st, std::vector<sptt_csf *> *csfs, std::vector<int64_t> *base);
// out[fids0[f]] += row f of the tile's compact MTTKRP (FP64 rows where it has them).
sptt_status tile_accumulate_launch(const sptt_csf *tile, const float *compact, const double *heavy, int32_t ld,
                                   float *out, cudaStream_t st);

// ---------------------------------------------------------------------------
// Dense kernels (dense.cu)
// ---------------------------------------------------------------------------
struct DenseWork {
    int32_t rank = 0, ld = 0;
    int32_t nblocks = 0;          // blocks of the row kernels (partials per block)
    int32_t solve_resident = 0;   // row-solve CTAs resident on the GPU at once (its rank's tile)
    double *partials = nullptr;   // [nblocks][rank*rank + rank]
    double *gram_un = nullptr;    // rank*rank (+ rank dots)
    float *W = nullptr;           // rank*rank (FP32 copy of V^dagger)
    double *lambda = nullptr;     // rank
    float *inv_lambda = nullptr;  // rank (FP32, for the normalise pass)
    double *inner = nullptr;      // 1: sum_r sum_i M[i,r] A_un[i,r] of the last mode update
    int32_t *branch = nullptr;    // counters: [0] pinv updates, [1] total updates
    int32_t *error = nullptr;     // device error word (timeouts)
};
sptt_status dense_work_alloc(DenseWork *w, int32_t rank, int32_t ld, int64_t max_rows,
                             cudaStream_t st);
void dense_work_free(DenseWork *w, cudaStream_t st);

sptt_status gram_launch(const float *A, int64_t rows, int32_t rank, int32_t ld, double *G,
                        double *partials, int32_t nblocks, cudaStream_t st);
// V = Hadamard_{m != n} grams[m]; W = V^dagger (FP64 Cholesky or pinv), stored FP32.
sptt_status normal_prep_launch(double *const *grams, int32_t nmodes, int32_t n, int32_t rank,
                               DenseWork *w, cudaStream_t st);
// A_un[fids0[f]] = M[f] W over the rows f < rows of the compact M, with
// Gram(A_un) and the column dots M.A_un into per-block partials, reduced.
sptt_status postsolve_launch(const float *M, const double *heavy, const int32_t *hidx, const int32_t *fids0,
                             float *A, int64_t rows, DenseWork *w, cudaStream_t st);
// lambda = sqrt(diag G_un); G_n = D^-1 G_un D^-1; inner = sum dots; and
// A[fids0[f]] *= 1/lambda (columns) for f < rows, optional BF16 shadow.
sptt_status finalize_normalize_launch(double *G_n, float *A, __nv_bfloat16 *A_bf16, const int32_t *fids0,
                                     int64_t rows, DenseWork *w, cudaStream_t st);
// fit = 1 - sqrt(max(0, normx2 + lambda^T (*G) lambda - 2 inner)) / sqrt(normx2),
// written to ring[*counter % ring_len], then ++*counter (device side).
sptt_status fit_launch(double *const *grams, int32_t nmodes, const double *normx2, DenseWork *w,
                       double *ring, int32_t ring_len, int64_t *counter, cudaStream_t st);
sptt_status sumsq_launch(const float *vals, int64_t n, double *out, cudaStream_t st);
sptt_status init_factor_launch(uint64_t seed, int32_t mode, int64_t rows, int32_t rank,
                               int32_t ld, float *A, cudaStream_t st);
sptt_status fill_zero_launch(void *p, size_t bytes, cudaStream_t st);
sptt_status to_bf16_launch(const float *A, __nv_bfloat16 *B, int64_t n, cudaStream_t st);

}  // namespace sptt
