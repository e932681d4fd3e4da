// Root-mode MTTKRP over CSF (Section III; the MTTKRP step of Algorithm 1).
//
// For the CSF rooted at mode n with level order (n, o_1, ..., o_{N-1}):
//   M[i, :] = sum_{level-1 fibers f of slice i} A^(o_1)[j_f, :] *
//             ( ... sum_{leaves k of the level-(N-2) fiber} v_k A^(o_{N-1})[k_idx, :])
// i.e. the Khatri-Rao product is never formed; each fiber's partial sum is
// multiplied by its factor row once (the CSF factorisation of the sum).
//
// GPU mapping (replaces the paper's thread-per-slice loops with locks or
// privatised outputs, Section IV-A / V-D-2):
//   * a "lane group" of G = ld / VEC lanes owns one output row; lane g holds
//     columns [g*VEC, g*VEC+VEC) and gathers them with one 16- or 32-byte load
//     per factor row (VEC = 4 or 8 FP32 values, 8 or 16 BF16 values);
//   * the leaves are cut into equal chunks (the CSF's precomputed partition
//     gives, per chunk, the fiber at every level holding its first leaf); a
//     lane group walks its chunk in order, keeping one register accumulator
//     per tree level, so the load is balanced whatever the slice sizes
//     (power-law slices are split across many chunks);
//   * output conflicts: a slice that lies entirely inside one chunk is owned
//     by that lane group and stored; a slice cut by a chunk boundary is
//     combined with red.global.add.v4.f32 into a zeroed output, a heavy one
//     in FP64 (the GPU form of the paper's lock pool: no lock, no spin).
// The per-chunk tree walks live in walk.cuh; the kernels here spread the
// chunks over the lane groups of the grid and hold the sptt_mttkrp entry point.
#include "walk.cuh"

namespace sptt {
namespace {

using walk::Lanes;
using walk::lanes_for;

// The 32-byte-segment walks on packed leaf records.
bool wide_variant(int v) { return v == 7 || v == 10 || v == 12; }
// The select walk with the leaf factor copied into shared memory.
bool table_variant(int v) { return v == 14 || v == 15; }

// Each CTA takes a contiguous range of chunks; its lane groups interleave
// within the range, so a group's consecutive chunks are close together and a
// heavy slice's partial can be carried from one to the next.
struct ChunkRange {
    int64_t begin, end, step;
};

__device__ __forceinline__ ChunkRange cta_chunks(int64_t nchunks, const Lanes &L) {
    const int64_t per = (nchunks + gridDim.x - 1) / gridDim.x;
    const int64_t b = (int64_t)blockIdx.x * per;
    ChunkRange r;
    r.step = (int64_t)(blockDim.x >> 5) * L.gpw;
    r.begin = b + (int64_t)(threadIdx.x >> 5) * L.gpw + L.gi;
    r.end = (b + per < nchunks) ? b + per : nchunks;
    return r;
}

// PACKED: the walk reads the packed leaf records (with the cache hints of
// walk.cuh load_rec_pair) instead of the separate leaf arrays.
template <int NM, typename T, int B, int MINB, int W = 16, bool PIPE = true, bool PACKED = false, bool DIRECT = false>
__global__ void __launch_bounds__(256, MINB) mttkrp_flag_kernel(const walk::Args a) {
    const Lanes L = lanes_for(a.ld, walk::Raw<T, W>::VEC);
    if (L.idle) return;  // no warp collectives in the walk
    const ChunkRange r = cta_chunks(a.nchunks, L);
    walk::Carry<walk::Raw<T, W>::VEC> cy;
    if constexpr (PACKED) {
        const walk::PackedRecs rec{a.leafrec};
        for (int64_t c = r.begin; c < r.end; c += r.step)
            walk::flag_chunk<NM, T, B, walk::PackedRecs, W, PIPE, DIRECT>(a, c, L.col, cy, rec);
    } else {
        const walk::GlobalRecs rec{a.vals, a.fids[NM - 1], a.lvl};
        for (int64_t c = r.begin; c < r.end; c += r.step)
            walk::flag_chunk<NM, T, B, walk::GlobalRecs, W, PIPE>(a, c, L.col, cy, rec);
    }
    walk::flush_carry(a, L.col, cy);
}

// The select walk (walk.cuh select_chunk) on packed leaf records.
// The select walk (walk.cuh select_chunk) on packed leaf records.
template <int NM, typename T, int B, int MINB, int W>
__global__ void __launch_bounds__(256, MINB) mttkrp_select_kernel(const walk::Args a) {
    const Lanes L = lanes_for(a.ld, walk::Raw<T, W>::VEC);
    if (L.idle) return;  // no warp collectives in the walk
    const ChunkRange r = cta_chunks(a.nchunks, L);
    walk::Carry<walk::Raw<T, W>::VEC> cy;
    const walk::PackedRecs rec{a.leafrec};
    for (int64_t c = r.begin; c < r.end; c += r.step) walk::select_chunk<NM, T, B, W>(a, c, L.col, cy, rec);
    walk::flush_carry(a, L.col, cy);
}

// The table kernels: each CTA first copies the whole leaf factor (leaf_rows
// rows of ld values, row-major) into shared memory, then runs the select walk
// with its leaf rows read from that copy; only the records and the rows of
// the fibers above the leaves still come through the L1 load path. One CTA
// of NT threads per SM.
template <int NM, typename T, int B, int NT, int W>
__global__ void __launch_bounds__(NT, 1) mttkrp_table_kernel(const walk::Args a, int32_t leaf_rows) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t rowbytes = (uint32_t)a.ld * (uint32_t)sizeof(T);
    const uint4 *src = static_cast<const uint4 *>(a.fac[NM - 1]);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    const int64_t n16 = (int64_t)leaf_rows * rowbytes / 16;
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    const Lanes L = lanes_for(a.ld, walk::Raw<T, W>::VEC);
    if (L.idle) return;  // no barrier after this point
    const ChunkRange r = cta_chunks(a.nchunks, L);
    walk::Carry<walk::Raw<T, W>::VEC> cy;
    const walk::PackedRecs rec{a.leafrec};
    const uint32_t tab = (uint32_t)__cvta_generic_to_shared(smem);
    for (int64_t c = r.begin; c < r.end; c += r.step)
        walk::select_chunk<NM, T, B, W, true>(a, c, L.col, cy, rec, tab, rowbytes);
    walk::flush_carry(a, L.col, cy);
}

template <int NM, typename T>
__global__ void __launch_bounds__(256) mttkrp_root_kernel(const walk::Args a) {
    const Lanes L = lanes_for(a.ld, walk::Raw<T>::VEC);
    if (L.idle) return;
    const ChunkRange r = cta_chunks(a.nchunks, L);
    walk::Carry<walk::Raw<T>::VEC> cy;
    for (int64_t c = r.begin; c < r.end; c += r.step) walk::plain_chunk<NM, T>(a, c, L.col, cy);
    walk::flush_carry(a, L.col, cy);
}

// ---------------------------------------------------------------------------
// Variant 6: the flag walk with its leaf records staged in shared memory.
// Each lane group owns two stage buffers of one chunk's records (values,
// leaf indices, level flags: 9 bytes per leaf) and an mbarrier per stage.
// The group's first lane issues three bulk copies (cp.async.bulk) for the
// chunk after next while the group walks the current one, so the record
// stream arrives in shared memory without occupying the L1 load pipe, and
// the walk reads it with conflict-free shared loads. Every wait is bounded:
// past kWaitNs the CSF's error word is set and the group stops.
// ---------------------------------------------------------------------------
constexpr int kStageChunk = 64;
constexpr uint32_t kStageBytes = 9 * kStageChunk;          // 576
constexpr uint32_t kStageStride = kStageBytes + 16;        // 592
constexpr uint32_t kGroupStride = 1200;                    // 2 stages + pad; 300 words = 12 mod 32 banks
constexpr uint64_t kWaitNs = 1000000000ull;                // 1 s

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (it == 0) t0 = gtimer();
        else if ((it & 31) == 0 && gtimer() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void stage_issue(const walk::Args &a, const int32_t *leaf_idx, int64_t c, uint32_t bar,
                                            uint32_t dst) {
    const int64_t k0 = c * kStageChunk;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kStageBytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(a.vals + k0), "r"(kStageChunk * 4), "r"(bar) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst + kStageChunk * 4), "l"(leaf_idx + k0), "r"(kStageChunk * 4), "r"(bar) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst + kStageChunk * 8), "l"(a.lvl + k0), "r"(kStageChunk), "r"(bar) : "memory");
}

template <int NM, typename T, int W>
__global__ void __launch_bounds__(256, 2) mttkrp_staged_kernel(const walk::Args a, int32_t *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int VEC = walk::Raw<T, W>::VEC;
    const Lanes L = lanes_for(a.ld, VEC);
    if (L.idle) return;  // no CTA-wide barrier below: every group runs on its own
    const int G = a.ld / VEC;
    const int gcta = (threadIdx.x >> 5) * L.gpw + L.gi;
    const int groups = (blockDim.x >> 5) * L.gpw;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t bar = sbase + gcta * 16;  // stage s barrier at bar + 8 s
    const uint32_t buf = sbase + ((groups * 16 + 127) & ~127) + gcta * kGroupStride;
    const int lane = threadIdx.x & 31;
    const bool leader = lane == L.gi * G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (L.gi * G));
    const int32_t *leaf_idx = a.fids[NM - 1];
    const ChunkRange r = cta_chunks(a.nchunks, L);
    if (leader) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (r.begin < r.end) stage_issue(a, leaf_idx, r.begin, bar, buf);
        if (r.begin + r.step < r.end) stage_issue(a, leaf_idx, r.begin + r.step, bar + 8, buf + kStageStride);
    }
    __syncwarp(gmask);
    walk::Carry<VEC> cy;
    int64_t n = 0;
    for (int64_t c = r.begin; c < r.end; c += r.step, ++n) {
        const uint32_t s = (uint32_t)(n & 1);
        if (!mbar_wait(bar + 8 * s, (uint32_t)((n >> 1) & 1))) {
            atomicOr(err, 2);
            // the other stage may still have a copy in flight: wait for it (bounded) before leaving
            if (c + r.step < r.end) mbar_wait(bar + 8 * (s ^ 1u), (uint32_t)(((n + 1) >> 1) & 1));
            return;
        }
        const walk::SharedRecs rec{buf + s * kStageStride, buf + s * kStageStride + kStageChunk * 4,
                                   buf + s * kStageStride + kStageChunk * 8, c * (int64_t)kStageChunk};
        walk::flag_chunk<NM, T, (W == 32 ? 2 : 4), walk::SharedRecs, W>(a, c, L.col, cy, rec);
        __syncwarp(gmask);  // the whole group is done with stage s
        const int64_t cn = c + 2 * r.step;
        if (leader && cn < r.end) stage_issue(a, leaf_idx, cn, bar + 8 * s, buf + s * kStageStride);
    }
    walk::flush_carry(a, L.col, cy);
}

// out[fids0[f] * ld + :] = row f of the compact result; other rows stay as
// they are (zeroed by the caller).
__global__ void scatter_rows_kernel(const float *__restrict__ compact, const double *__restrict__ heavy,
                                    const int32_t *__restrict__ hidx, const int32_t *__restrict__ fids0,
                                    int64_t nrows, int ld, float *__restrict__ out) {
    const int64_t n = nrows * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e / ld;
        const int c = (int)(e - f * ld);
        out[(int64_t)__ldg(fids0 + f) * ld + c] = walk::read_row(compact, heavy, hidx, f, ld, c);
    }
}

template <int NM, typename T, int W>
sptt_status launch_staged(const walk::Args &a, int32_t *err, cudaStream_t st) {
    auto kern = mttkrp_staged_kernel<NM, T, W>;
    const int vec = walk::Raw<T, W>::VEC;
    const int gpw = 32 / (a.ld / vec);
    const int block = gpw >= 16 ? 128 : 256;  // keep the stage buffers of a CTA near 80 KB
    const int groups = (block / 32) * gpw;
    const size_t smem = (size_t)((groups * 16 + 127) & ~127) + (size_t)groups * kGroupStride;
    SPTT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t need = (a.nchunks + groups - 1) / groups;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t grid = need < cap ? need : cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, smem, st>>>(a, err);
    SPTT_CHECK_LAUNCH("mttkrp_staged_kernel");
    return SPTT_OK;
}

template <int NM, typename T, int B, int NT, int W>
sptt_status launch_table(const walk::Args &a, int64_t leaf_rows, cudaStream_t st) {
    auto kern = mttkrp_table_kernel<NM, T, B, NT, W>;
    const size_t smem = (size_t)leaf_rows * a.ld * sizeof(T);
    SPTT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    if (per_sm < 1) per_sm = 1;
    const int vec = walk::Raw<T, W>::VEC;
    const int64_t groups_per_block = (int64_t)(NT / 32) * (32 / (a.ld / vec));
    const int64_t need = (a.nchunks + groups_per_block - 1) / groups_per_block;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t grid = need < cap ? need : cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, NT, smem, st>>>(a, (int32_t)leaf_rows);
    SPTT_CHECK_LAUNCH("mttkrp_table_kernel");
    return SPTT_OK;
}

template <int NM, typename T>
sptt_status launch_table_nm(const walk::Args &a, int64_t leaf_rows, int variant, cudaStream_t st) {
    if (variant == 15) return launch_table<NM, T, 4, 512, 16>(a, leaf_rows, st);
    return launch_table<NM, T, 2, 1024, 16>(a, leaf_rows, st);
}

template <int NM, typename T>
sptt_status launch_nm(const walk::Args &a, int block, int variant, cudaStream_t st) {
    void (*kern)(const walk::Args) = nullptr;
    switch (variant) {
        case 1: kern = mttkrp_root_kernel<NM, T>; break;
        case 2: kern = mttkrp_flag_kernel<NM, T, 8, 1>; break;
        case 3: kern = mttkrp_flag_kernel<NM, T, 4, 3, 16, false>; break;
        case 4: kern = mttkrp_flag_kernel<NM, T, 4, 2>; break;
        case 5: kern = mttkrp_flag_kernel<NM, T, 2, 3>; break;
        case 7: kern = mttkrp_flag_kernel<NM, T, 2, 2, 32, true, true>; break;
        case 9: kern = mttkrp_flag_kernel<NM, T, 4, 2, 16, true, true>; break;
        case 10: kern = mttkrp_flag_kernel<NM, T, 2, 2, 32, true, true, true>; break;
        case 11: kern = mttkrp_flag_kernel<NM, T, 4, 2, 16, true, true, true>; break;
        case 12: kern = mttkrp_select_kernel<NM, T, 2, 2, 32>; break;
        case 13: kern = mttkrp_select_kernel<NM, T, 4, 2, 16>; break;
        default: kern = mttkrp_flag_kernel<NM, T, 4, 3, 16, false>; break;
    }
    int per_sm = 0;
    SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0));
    if (per_sm < 1) per_sm = 1;
    const int vec = wide_variant(variant) ? walk::Raw<T, 32>::VEC : walk::Raw<T>::VEC;
    const int64_t groups_per_block = (int64_t)(block / 32) * (32 / (a.ld / vec));
    const int64_t need = (a.nchunks + groups_per_block - 1) / groups_per_block;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t grid = need < cap ? need : cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, 0, st>>>(a);
    SPTT_CHECK_LAUNCH("mttkrp kernel");
    return SPTT_OK;
}

template <typename T>
sptt_status launch_t(sptt_csf *csf, int nm, const walk::Args &a, int block, int variant, int32_t *err,
                     int64_t leaf_rows, cudaStream_t st) {
    if (table_variant(variant)) {
        switch (nm) {
            case 2: return launch_table_nm<2, T>(a, leaf_rows, variant, st);
            case 3: return launch_table_nm<3, T>(a, leaf_rows, variant, st);
            case 4: return launch_table_nm<4, T>(a, leaf_rows, variant, st);
            case 5: return launch_table_nm<5, T>(a, leaf_rows, variant, st);
            default: return set_error(SPTT_ERR_UNSUPPORTED, "nmodes");
        }
    }
    if (variant == 6 || variant == 8) {
        const bool wide = variant == 8;
        switch (nm) {
            case 2: return wide ? launch_staged<2, T, 32>(a, err, st) : launch_staged<2, T, 16>(a, err, st);
            case 3: return wide ? launch_staged<3, T, 32>(a, err, st) : launch_staged<3, T, 16>(a, err, st);
            case 4: return wide ? launch_staged<4, T, 32>(a, err, st) : launch_staged<4, T, 16>(a, err, st);
            case 5: return wide ? launch_staged<5, T, 32>(a, err, st) : launch_staged<5, T, 16>(a, err, st);
            default: return set_error(SPTT_ERR_UNSUPPORTED, "nmodes");
        }
    }
    switch (nm) {
        case 2: return launch_nm<2, T>(a, block, variant, st);
        case 3: return launch_nm<3, T>(a, block, variant, st);
        case 4: return launch_nm<4, T>(a, block, variant, st);
        case 5: return launch_nm<5, T>(a, block, variant, st);
        default: return set_error(SPTT_ERR_UNSUPPORTED, "nmodes");
    }
}

}  // namespace

// Default leaves per chunk: 128, halved (down to 32) while the tensor would
// give fewer than 128 chunks per SM, so that small tensors still fill the GPU.
// (Measured on 80 generated tensors of 1e5-2e7 non-zeros, 3-5 modes, every
// root, both gather types: shorter chunks cost more in per-chunk work than
// they gain in balance.)
int32_t default_chunk(int64_t nnz) {
    const int64_t target = (int64_t)device_sm_count() * 128;
    int32_t c = 128;
    while (c > 32 && nnz / c < target) c >>= 1;
    return c;
}

static bool staged_variant(int v) { return v == 6 || v == 8; }

// The default variant: the select walk with 16-byte segments in batches of 4
// (the best single candidate over generated tensors of 1e5-2e7 non-zeros,
// 3-5 modes, ranks 8-64, both gather types: 11 % above the best per tensor on
// average), and for large 3-mode tensors with FP32 gathers whose leaf factor
// fits in shared memory the table kernel (on the 1e8-non-zero 3-mode
// power-law tensor 12 % faster than the best global-memory walk).
int default_variant(int32_t dtype, int32_t ld, int64_t leaf_rows, int64_t nnz, int nmodes) {
    const bool bf16 = dtype == SPTT_BF16;
    if (nmodes == 3 && nnz >= kTableMinNnz && leaf_table_fits(leaf_rows, ld, bf16 ? 2 : 4)) return bf16 ? 15 : 14;
    if (!bf16 && nnz >= kWideMinNnz && ld >= 16 && ld % 8 == 0) return 12;
    return 13;
}

bool leaf_table_fits(int64_t leaf_rows, int32_t ld, int esz) {
    return (size_t)leaf_rows * ld * esz <= kTableMaxBytes;
}

int default_order_kind(const int64_t *dims, int nmodes, int root, int32_t ld, int32_t dtype, int64_t nnz) {
    if (nmodes != 3 || nnz < kTableMinNnz) return 0;
    int64_t shortest = -1;
    for (int k = 0; k < nmodes; ++k)
        if (k != root && (shortest < 0 || dims[k] < shortest)) shortest = dims[k];
    return leaf_table_fits(shortest, ld, dtype == SPTT_BF16 ? 2 : 4) ? 2 : 0;
}

// Variants that read the packed leaf records (sptt_csf::leafrec).
static bool packed_variant(int v) { return v == 7 || v >= 9; }

sptt_status mttkrp_prepare(sptt_csf *csf, const sptt_sched *sched, cudaStream_t st) {
    const int32_t chunk = (sched && staged_variant(sched->variant)) ? kStageChunk
                          : ((sched && sched->chunk) ? sched->chunk : default_chunk(csf->nfibs[csf->nmodes - 1]));
    if (csf->nfibs[csf->nmodes - 1] == 0) return SPTT_OK;
    const int v = sched ? sched->variant : 0;
    if (v == 0 || packed_variant(v)) SPTT_TRY(csf_ensure_leafrec(csf, st));
    return csf_ensure_partition(csf, chunk, st);
}

sptt_status mttkrp_launch(sptt_csf *csf, const void *const *factors, int32_t dtype, int32_t ld,
                          float *out, double *heavy, const sptt_sched *sched, cudaStream_t st) {
    const int N = csf->nmodes;
    SPTT_TRY(fill_zero_launch(out, (size_t)csf->nfibs[0] * ld * sizeof(float), st));
    const int64_t nnz = csf->nfibs[N - 1];
    if (nnz == 0) return SPTT_OK;
    int variant = sched ? sched->variant : 0;
    if (variant == 0) variant = default_variant(dtype, ld, csf->dims[csf->order[N - 1]], nnz, N);
    // the table kernels need the whole leaf factor in shared memory
    if (table_variant(variant) && !leaf_table_fits(csf->dims[csf->order[N - 1]], ld, dtype == SPTT_BF16 ? 2 : 4))
        variant = 13;
    if (wide_variant(variant) || variant == 8) {
        // 32-byte row segments need ld * sizeof(T) and every gathered factor
        // 32-byte aligned; otherwise the 16-byte form of the same walk runs
        const int esz = dtype == SPTT_BF16 ? 2 : 4;
        bool wide_ok = (ld * esz) % 32 == 0;
        for (int l = 1; l < N; ++l)
            wide_ok = wide_ok && reinterpret_cast<uintptr_t>(factors[csf->order[l]]) % 32 == 0;
        if (!wide_ok) variant = variant == 8 ? 6 : (variant == 12 ? 13 : 3);
    }
    const int32_t chunk = staged_variant(variant) ? kStageChunk
                                                  : ((sched && sched->chunk) ? sched->chunk : default_chunk(csf->nfibs[csf->nmodes - 1]));
    const int block = (sched && sched->block) ? sched->block : 256;
    SPTT_TRY(csf_ensure_partition(csf, chunk, st));
    if (packed_variant(variant)) SPTT_TRY(csf_ensure_leafrec(csf, st));
    if (csf->nheavy > 0) SPTT_TRY(fill_zero_launch(heavy, (size_t)csf->nheavy * ld * sizeof(double), st));
    walk::Args a{};
    for (int l = 0; l < N; ++l) {
        a.fptr[l] = csf->fptr[l];
        a.fids[l] = csf->fids[l];
        a.fac[l] = l ? factors[csf->order[l]] : nullptr;
    }
    a.vals = csf->vals;
    a.lvl = csf->lvl;
    a.part = csf->part;
    a.nchunks = csf->part_nchunks;
    a.nnz = nnz;
    a.chunk = chunk;
    a.ld = ld;
    a.out = out;
    a.heavy = heavy;
    a.hidx = csf->hidx;
    a.leafrec = csf->leafrec;
    const int64_t leaf_rows = csf->dims[csf->order[N - 1]];
    if (dtype == SPTT_BF16) return launch_t<__nv_bfloat16>(csf, N, a, block, variant, csf->err, leaf_rows, st);
    return launch_t<float>(csf, N, a, block, variant, csf->err, leaf_rows, st);
}

}  // namespace sptt

using namespace sptt;

extern "C" sptt_status sptt_mttkrp(const sptt_csf *csf, const void *const *factors, int32_t factor_dtype,
                                   int32_t ld, float *out, const sptt_sched *sched, sptt_stream stream) {
    clear_error();
    if (!csf || !factors || !out) return set_error(SPTT_ERR_BAD_ARG, "csf, factors and out must be non-NULL");
    if (factor_dtype != SPTT_F32 && factor_dtype != SPTT_BF16)
        return set_error(SPTT_ERR_BAD_ARG, "factor_dtype must be SPTT_F32 or SPTT_BF16");
    const int vec = factor_dtype == SPTT_BF16 ? 8 : 4;
    const int max_ld = 32 * vec;
    if (ld < vec || ld > max_ld || ld % vec)
        return set_error(SPTT_ERR_BAD_ARG, "ld must be a multiple of " + std::to_string(vec) + " in [" +
                                               std::to_string(vec) + ", " + std::to_string(max_ld) + "]");
    if (reinterpret_cast<uintptr_t>(out) % 16) return set_error(SPTT_ERR_BAD_ARG, "out must be 16-byte aligned");
    for (int l = 1; l < csf->nmodes; ++l) {
        const void *p = factors[csf->order[l]];
        if (!p) return set_error(SPTT_ERR_BAD_ARG, "a non-root factor is NULL");
        if (reinterpret_cast<uintptr_t>(p) % 16) return set_error(SPTT_ERR_BAD_ARG, "factors must be 16-byte aligned");
        if (p == out) return set_error(SPTT_ERR_BAD_ARG, "out aliases a factor");
    }
    if (sched) {
        if (sched->chunk && (sched->chunk < 16 || sched->chunk > 4096 || (sched->chunk & (sched->chunk - 1))))
            return set_error(SPTT_ERR_BAD_ARG, "sched->chunk must be a power of two in [16, 4096]");
        if (sched->block && (sched->block < 32 || sched->block > 256 || sched->block % 32))
            return set_error(SPTT_ERR_BAD_ARG, "sched->block must be a multiple of 32 in [32, 256]");
        if (sched->variant < 0 || sched->variant > kMaxVariant)
            return set_error(SPTT_ERR_BAD_ARG, "sched->variant must be in [0, " + std::to_string(kMaxVariant) + "]");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    sptt_csf *c = const_cast<sptt_csf *>(csf);
    const int64_t rows = c->dims[c->root];
    const int64_t ns = c->nfibs[0];
    SPTT_TRY(mttkrp_prepare(c, sched, st));
    DevBuf acc, heavy;  // compact result (one row per slice) and the heavy slices' FP64 rows
    SPTT_TRY(acc.alloc<float>((size_t)ns * ld, st));
    SPTT_TRY(heavy.alloc<double>((size_t)c->nheavy * ld, st));
    SPTT_TRY(mttkrp_launch(c, factors, factor_dtype, ld, acc.as<float>(), heavy.as<double>(), sched, st));
    SPTT_TRY(fill_zero_launch(out, (size_t)rows * ld * sizeof(float), st));
    if (ns > 0) {
        int64_t grid = (ns * ld + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        if (grid > cap) grid = cap;
        scatter_rows_kernel<<<(unsigned)grid, 256, 0, st>>>(acc.as<float>(), heavy.as<double>(), c->hidx, c->fids[0],
                                                            ns, ld, out);
        SPTT_CHECK_LAUNCH("scatter_rows_kernel");
    }
    return SPTT_OK;
}
