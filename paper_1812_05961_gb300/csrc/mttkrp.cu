// Root-mode MTTKRP over CSF (Section III; Algorithm 1 lines 5, 8, 11).
//
// For the CSF rooted at mode n with level order (n, o_1, ..., o_{N-1}):
//   M[i, :] = sum_{level-1 fibers f of slice i} A^(o_1)[j_f, :] *
//             ( ... sum_{leaves k of the level-(N-2) fiber} v_k A^(o_{N-1})[k_idx, :])
// i.e. the Khatri-Rao product is never formed; each fiber's partial sum is
// multiplied by its factor row once (the CSF factorisation of the sum).
//
// GPU mapping (replaces the paper's thread-per-slice loops with locks or
// privatised outputs, Section IV-A / V-D-2):
//   * a "lane group" of G = ld / VEC lanes owns one output row segment; lane g
//     holds columns [g*VEC, g*VEC+VEC) (VEC = 4 for FP32 factors, 8 for BF16)
//     and gathers them with one 128-bit load per factor row;
//   * the leaves are cut into equal chunks (the CSF's precomputed partition
//     gives, per chunk, the fiber at every level holding its first leaf); a
//     lane group walks its chunk in order, keeping one register accumulator
//     per tree level, so the load is balanced whatever the slice sizes
//     (power-law slices are split across many chunks);
//   * output conflicts: a slice that lies entirely inside one chunk is owned
//     by that lane group and written with a plain 128-bit store; a slice cut
//     by a chunk boundary is combined with red.global.add.v4.f32 into a
//     zeroed output (the GPU form of the paper's lock pool: no lock, no spin).
#include "internal.cuh"

namespace sptt {
namespace {

struct MttkrpArgs {
    const int32_t *fptr[kMaxModes];
    const int32_t *fids[kMaxModes];
    const void *fac[kMaxModes];  // by level; fac[0] unused
    const float *vals;
    const uint8_t *lvl;
    const int32_t *part;
    int64_t nchunks;
    int64_t nnz;
    int32_t chunk;
    int32_t ld;
    int32_t G;    // lanes per row
    int32_t gpw;  // lane groups per warp
    double *out;
};

template <typename T>
struct Gather;

template <>
struct Gather<float> {
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void load(const void *base, int64_t row, int ld, int col, float (&x)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(base) + row * ld + col));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
};

template <>
struct Gather<__nv_bfloat16> {
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void load(const void *base, int64_t row, int ld, int col, float (&x)[8]) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(base) + row * ld + col));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {  // bf16 -> f32 is exact: the bits move to the top half
            x[2 * i] = __uint_as_float(w[i] << 16);
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};

// Output rows are FP64. A slice owned by one lane group (it starts and ends
// inside the group's chunk) is stored; a slice cut by chunk boundaries gets
// one FP32 partial per chunk, and those are summed with FP64 atomics, so a
// power-law slice split over 10^5 chunks keeps FP32-of-one-chunk accuracy.
template <int VEC>
__device__ __forceinline__ void store_row(double *dst, const float (&a)[VEC]) {
#pragma unroll
    for (int i = 0; i < VEC; i += 2)
        *reinterpret_cast<double2 *>(dst + i) = make_double2((double)a[i], (double)a[i + 1]);
}

template <int VEC>
__device__ __forceinline__ void red_add_row(double *dst, const float (&a)[VEC]) {
#pragma unroll
    for (int i = 0; i < VEC; ++i)
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(dst + i), "d"((double)a[i]) : "memory");
}

__global__ void f64_to_f32_kernel(const double2 *__restrict__ in, float2 *__restrict__ out, int64_t n2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 d = in[i];
        out[i] = make_float2((float)d.x, (float)d.y);
    }
}

// A factor row segment as loaded (16 bytes: 4 FP32 or 8 BF16), widened to
// FP32 only where it is used.
template <typename T>
struct Raw;

template <>
struct Raw<float> {
    static constexpr int VEC = 4;
    __device__ __forceinline__ static uint4 load(const void *base, int64_t row, int ld, int col) {
        return __ldg(reinterpret_cast<const uint4 *>(static_cast<const float *>(base) + row * ld + col));
    }
    __device__ __forceinline__ static void widen(const uint4 &u, float (&x)[4]) {
        x[0] = __uint_as_float(u.x); x[1] = __uint_as_float(u.y);
        x[2] = __uint_as_float(u.z); x[3] = __uint_as_float(u.w);
    }
};

template <>
struct Raw<__nv_bfloat16> {
    static constexpr int VEC = 8;
    __device__ __forceinline__ static uint4 load(const void *base, int64_t row, int ld, int col) {
        return __ldg(reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(base) + row * ld + col));
    }
    __device__ __forceinline__ static void widen(const uint4 &u, float (&x)[8]) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = __uint_as_float(w[i] << 16);
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};

// Variant 0: batched walk driven by the per-leaf level flags.
// Each lane group takes a chunk of leaves in batches of B = 8: the batch's
// values, leaf indices and level flags arrive in three vector loads; then
// every factor row the batch needs (the 8 leaf rows, and the rows of the
// level-(N-2) fibers that start inside the batch, whose ids are consecutive)
// is requested before any of them is used, so a group keeps up to 16 row
// gathers in flight instead of walking one dependent load at a time. Rows of
// fibers at levels above N-2 are requested when the fiber opens and used when
// it closes.
template <int NM, typename T, int B, int MINB>
__global__ void __launch_bounds__(256, MINB) mttkrp_flag_kernel(const MttkrpArgs a) {
    using Rw = Raw<T>;
    constexpr int VEC = Rw::VEC;
    constexpr int NL = NM - 1;  // accumulator levels 0..NM-2
    constexpr int LF = NM - 2;  // level of the leaves' parent fibers
    static_assert(B == 4 || B == 8, "batch of 4 or 8 leaves");
    const int lane = threadIdx.x & 31;
    const int gi = lane / a.G;
    const int gl = lane - gi * a.G;
    if (gi >= a.gpw) return;  // no warp collectives below
    const int col = gl * VEC;
    const int ld = a.ld;
    const int64_t gwarp = (int64_t)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t)(gridDim.x * blockDim.x) >> 5;

    for (int64_t c = gwarp * a.gpw + gi; c < a.nchunks; c += nwarps * a.gpw) {
        const int64_t k0 = c * (int64_t)a.chunk;
        const int64_t k1 = (k0 + a.chunk < a.nnz) ? k0 + a.chunk : a.nnz;
        int32_t f[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) f[l] = __ldg(a.part + c * NL + l);
        float acc[NL][VEC];
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[l][i] = 0.f;
        uint4 rowc[NL];  // rows of the open fibers, levels 1..NL-1
#pragma unroll
        for (int l = 1; l < NL; ++l) rowc[l] = Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col);
        int32_t fid0 = __ldg(a.fids[0] + f[0]);
        bool first_slice = true;

        for (int64_t kb = k0; kb < k1; kb += B) {
            float v[B];
            int32_t li[B];
            uint32_t lw[2] = {0u, 0u};
            {
                const float4 va = __ldg(reinterpret_cast<const float4 *>(a.vals + kb));
                const int4 ia = __ldg(reinterpret_cast<const int4 *>(a.fids[NM - 1] + kb));
                v[0] = va.x; v[1] = va.y; v[2] = va.z; v[3] = va.w;
                li[0] = ia.x; li[1] = ia.y; li[2] = ia.z; li[3] = ia.w;
                if (B == 8) {
                    const float4 vb = __ldg(reinterpret_cast<const float4 *>(a.vals + kb + 4));
                    const int4 ib = __ldg(reinterpret_cast<const int4 *>(a.fids[NM - 1] + kb + 4));
                    v[4 % B] = vb.x; v[5 % B] = vb.y; v[6 % B] = vb.z; v[7 % B] = vb.w;
                    li[4 % B] = ib.x; li[5 % B] = ib.y; li[6 % B] = ib.z; li[7 % B] = ib.w;
                    const uint2 l2 = __ldg(reinterpret_cast<const uint2 *>(a.lvl + kb));
                    lw[0] = l2.x;
                    lw[1] = l2.y;
                } else {
                    lw[0] = __ldg(reinterpret_cast<const uint32_t *>(a.lvl + kb));
                }
            }
            const int nvalid = (k1 - kb < B) ? (int)(k1 - kb) : B;
            uint4 x[B];
#pragma unroll
            for (int j = 0; j < B; ++j)
                if (j < nvalid) x[j] = Rw::load(a.fac[NM - 1], li[j], ld, col);
            // leaves that open a new level-LF fiber (never the chunk's first leaf)
            uint32_t sm = 0;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const uint32_t d = (lw[j >> 2] >> (8 * (j & 3))) & 0xffu;
                if (j < nvalid && d <= (uint32_t)LF && (kb + j) != k0) sm |= 1u << j;
            }
            uint4 nr[B];
            if (LF >= 1) {
#pragma unroll
                for (int j = 0; j < B; ++j)
                    if ((sm >> j) & 1u) {
                        const int pos = __popc(sm & ((1u << j) - 1u)) + 1;
                        nr[j] = Rw::load(a.fac[LF], __ldg(a.fids[LF] + f[LF] + pos), ld, col);
                    }
            }
#pragma unroll
            for (int j = 0; j < B; ++j) {
                if (j >= nvalid) break;
                if ((sm >> j) & 1u) {
                    const int d = (int)((lw[j >> 2] >> (8 * (j & 3))) & 0xffu);
                    if (LF >= 1) {
                        float r[VEC];
                        Rw::widen(rowc[LF], r);
#pragma unroll
                        for (int i = 0; i < VEC; ++i) {
                            acc[LF - 1][i] = fmaf(r[i], acc[LF][i], acc[LF - 1][i]);
                            acc[LF][i] = 0.f;
                        }
                        ++f[LF];
                        rowc[LF] = nr[j];
                    }
#pragma unroll
                    for (int l = LF - 1; l >= 1; --l) {
                        if (d <= l) {
                            float r[VEC];
                            Rw::widen(rowc[l], r);
#pragma unroll
                            for (int i = 0; i < VEC; ++i) {
                                acc[l - 1][i] = fmaf(r[i], acc[l][i], acc[l - 1][i]);
                                acc[l][i] = 0.f;
                            }
                            ++f[l];
                            rowc[l] = Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col);
                        }
                    }
                    if (d == 0) {  // the slice is complete
                        double *dst = a.out + (int64_t)fid0 * ld + col;
                        if (first_slice) red_add_row<VEC>(dst, acc[0]);
                        else store_row<VEC>(dst, acc[0]);
                        first_slice = false;
#pragma unroll
                        for (int i = 0; i < VEC; ++i) acc[0][i] = 0.f;
                        ++f[0];
                        fid0 = __ldg(a.fids[0] + f[0]);
                    }
                }
                float xr[VEC];
                Rw::widen(x[j], xr);
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc[LF][i] = fmaf(v[j], xr[i], acc[LF][i]);
            }
        }
        // chunk end: fold the open fibers and add the partial slice
#pragma unroll
        for (int l = LF; l >= 1; --l) {
            float r[VEC];
            Rw::widen(rowc[l], r);
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[l - 1][i] = fmaf(r[i], acc[l][i], acc[l - 1][i]);
        }
        red_add_row<VEC>(a.out + (int64_t)fid0 * ld + col, acc[0]);
    }
}

// Variant 1: the plain walk (one leaf at a time, fiber ends from fptr).
template <int NM, typename T>
__global__ void __launch_bounds__(256) mttkrp_root_kernel(const MttkrpArgs a) {
    using G_ = Gather<T>;
    constexpr int VEC = G_::VEC;
    constexpr int NL = NM - 1;  // accumulator levels 0..NM-2
    const int lane = threadIdx.x & 31;
    const int gi = lane / a.G;
    const int gl = lane - gi * a.G;
    if (gi >= a.gpw) return;  // lanes beyond the last whole group idle (no warp collectives below)
    const int col = gl * VEC;
    const int ld = a.ld;
    const int64_t gwarp = (int64_t)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t)(gridDim.x * blockDim.x) >> 5;

    for (int64_t c = gwarp * a.gpw + gi; c < a.nchunks; c += nwarps * a.gpw) {
        const int64_t k0 = c * (int64_t)a.chunk;
        const int64_t k1 = (k0 + a.chunk < a.nnz) ? k0 + a.chunk : a.nnz;
        int32_t f[NL], end[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            f[l] = __ldg(a.part + c * NL + l);
            end[l] = __ldg(a.fptr[l] + f[l] + 1);
        }
        float acc[NL][VEC];
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[l][i] = 0.f;
        bool first_slice = true;

        for (int64_t k = k0; k < k1; ++k) {
            if (k != k0 && k == end[NL - 1]) {
                // leaf k opens a new level-(N-2) fiber: close the finished
                // fibers bottom-up, folding each into its parent with the
                // fiber's factor row.
                bool to_root = true;
#pragma unroll
                for (int l = NL - 1; l >= 1; --l) {
                    float x[VEC];
                    G_::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col, x);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        acc[l - 1][i] = fmaf(x[i], acc[l][i], acc[l - 1][i]);
                        acc[l][i] = 0.f;
                    }
                    ++f[l];
                    end[l] = __ldg(a.fptr[l] + f[l] + 1);
                    if (f[l] != end[l - 1]) {
                        to_root = false;
                        break;
                    }
                }
                if (to_root) {  // the slice is complete
                    double *dst = a.out + (int64_t)__ldg(a.fids[0] + f[0]) * ld + col;
                    if (first_slice) red_add_row<VEC>(dst, acc[0]);
                    else store_row<VEC>(dst, acc[0]);
                    first_slice = false;
#pragma unroll
                    for (int i = 0; i < VEC; ++i) acc[0][i] = 0.f;
                    ++f[0];
                    end[0] = __ldg(a.fptr[0] + f[0] + 1);
                }
            }
            const float v = __ldg(a.vals + k);
            float x[VEC];
            G_::load(a.fac[NM - 1], __ldg(a.fids[NM - 1] + k), ld, col, x);
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[NL - 1][i] = fmaf(v, x[i], acc[NL - 1][i]);
        }
        // chunk end: fold the open fibers (all hold leaf k1-1) and add the
        // partial slice into the output.
#pragma unroll
        for (int l = NL - 1; l >= 1; --l) {
            float x[VEC];
            G_::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col, x);
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[l - 1][i] = fmaf(x[i], acc[l][i], acc[l - 1][i]);
        }
        red_add_row<VEC>(a.out + (int64_t)__ldg(a.fids[0] + f[0]) * ld + col, acc[0]);
    }
}

template <int NM, typename T>
sptt_status launch_nm(const MttkrpArgs &a, int block, int variant, cudaStream_t st) {
    void (*kern)(const MttkrpArgs) = nullptr;
    switch (variant) {
        case 1: kern = mttkrp_root_kernel<NM, T>; break;
        case 2: kern = mttkrp_flag_kernel<NM, T, 8, 2>; break;
        case 3: kern = mttkrp_flag_kernel<NM, T, 4, 3>; break;
        case 4: kern = mttkrp_flag_kernel<NM, T, 4, 4>; break;
        case 5: kern = mttkrp_flag_kernel<NM, T, 8, 1>; break;
        default: kern = mttkrp_flag_kernel<NM, T, 4, 3>; break;
    }
    int per_sm = 0;
    SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t groups_per_block = (int64_t)(block / 32) * a.gpw;
    int64_t need = (a.nchunks + groups_per_block - 1) / groups_per_block;
    int64_t cap = (int64_t)device_sm_count() * per_sm;
    int64_t grid = need < cap ? need : cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, 0, st>>>(a);
    SPTT_CHECK_LAUNCH("mttkrp_root_kernel");
    return SPTT_OK;
}

template <typename T>
sptt_status launch_t(int nm, const MttkrpArgs &a, int block, int variant, cudaStream_t st) {
    switch (nm) {
        case 2: return launch_nm<2, T>(a, block, variant, st);
        case 3: return launch_nm<3, T>(a, block, variant, st);
        case 4: return launch_nm<4, T>(a, block, variant, st);
        case 5: return launch_nm<5, T>(a, block, variant, st);
        default: return set_error(SPTT_ERR_UNSUPPORTED, "nmodes");
    }
}

}  // namespace

constexpr int32_t kDefaultChunk = 128;

sptt_status mttkrp_prepare(sptt_csf *csf, const sptt_sched *sched, cudaStream_t st) {
    const int32_t chunk = (sched && sched->chunk) ? sched->chunk : kDefaultChunk;
    if (csf->nfibs[csf->nmodes - 1] == 0) return SPTT_OK;
    return csf_ensure_partition(csf, chunk, st);
}

sptt_status mttkrp_launch(sptt_csf *csf, const void *const *factors, int32_t dtype, int32_t ld,
                          double *out, const sptt_sched *sched, cudaStream_t st) {
    const int N = csf->nmodes;
    const int vec = (dtype == SPTT_BF16) ? 8 : 4;
    const int64_t rows = csf->dims[csf->root];
    SPTT_TRY(fill_zero_launch(out, (size_t)rows * ld * sizeof(double), st));
    const int64_t nnz = csf->nfibs[N - 1];
    if (nnz == 0) return SPTT_OK;
    int32_t chunk = (sched && sched->chunk) ? sched->chunk : kDefaultChunk;
    int block = (sched && sched->block) ? sched->block : 256;
    int variant = sched ? sched->variant : 0;
    if (variant == 0) variant = (dtype == SPTT_BF16) ? 2 : 3;  // fastest measured per gather type
    SPTT_TRY(csf_ensure_partition(csf, chunk, st));
    MttkrpArgs a{};
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
    a.G = ld / vec;
    a.gpw = 32 / a.G;
    a.out = out;
    if (dtype == SPTT_BF16) return launch_t<__nv_bfloat16>(N, a, block, variant, st);
    return launch_t<float>(N, a, block, variant, st);
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
        if (sched->variant < 0 || sched->variant > 5)
            return set_error(SPTT_ERR_BAD_ARG, "sched->variant must be in [0, 5]");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t rows = csf->dims[csf->root];
    DevBuf acc;  // FP64 accumulation buffer, converted into out
    SPTT_TRY(acc.alloc<double>((size_t)rows * ld, st));
    SPTT_TRY(mttkrp_launch(const_cast<sptt_csf *>(csf), factors, factor_dtype, ld, acc.as<double>(), sched, st));
    const int64_t n2 = rows * ld / 2;
    if (n2 > 0) {
        int64_t grid = (n2 + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        if (grid > cap) grid = cap;
        f64_to_f32_kernel<<<(unsigned)grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(acc.as<double>()),
                                                          reinterpret_cast<float2 *>(out), n2);
        SPTT_CHECK_LAUNCH("f64_to_f32_kernel");
    }
    return SPTT_OK;
}
