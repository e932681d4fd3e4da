// Device-side walk of one work chunk of a CSF tree for the root-mode MTTKRP
// (Section III; the MTTKRP step of Algorithm 1). Shared by the standalone MTTKRP
// kernels and the batched CP-ALS kernel.
//
// For the CSF rooted at mode n with level order (n, o_1, ..., o_{N-1}):
//   M[i, :] = sum_{level-1 fibers f of slice i} A^(o_1)[j_f, :] *
//             ( ... sum_{leaves k of the level-(N-2) fiber} v_k A^(o_{N-1})[k_idx, :])
// The Khatri-Rao product is never formed: each fiber's partial sum is
// multiplied by its factor row once.
//
// Mapping (in place of the paper's thread-per-slice loops with a lock pool
// or privatised outputs, Section IV-A and V-D-2):
//   * a lane group of G = ld / VEC lanes owns one output row; lane g holds
//     columns [g*VEC, g*VEC + VEC) and gathers them with one 16- or 32-byte
//     load per factor row (VEC = 4 or 8 FP32 values, 8 or 16 BF16 values);
//   * the leaves are cut into equal chunks; the CSF's partition gives, per
//     chunk, the fiber at every level holding the chunk's first leaf, and a
//     lane group walks its chunk in order with one register accumulator per
//     tree level, so the work is balanced whatever the slice sizes;
//   * the output is compact: row f of M is slice f of the tree (the slice's
//     mode index is fids[0][f]). A slice that starts and ends inside one
//     chunk is owned by its lane group and stored (FP32). A slice cut by chunk
//     boundaries (up to 10^5 chunks for the power-law head) gets one FP32
//     partial per chunk, added with red.global.add.f64 into its own zeroed
//     FP64 row heavy[hidx[f]] (no lock, no spin): the sum keeps the accuracy
//     of one chunk's FP32 partial and, being exact for partials of similar
//     magnitude, does not depend on the order of the atomics. Readers take
//     that row in place of row f. (The red.global.add.v4.f32 path of
//     add_partial serves a slice inside one chunk that is not the chunk's
//     first: its single partial lands on a zero.)
#pragma once

#include "internal.cuh"

namespace sptt {
namespace walk {

// Lane-group layout of a warp: G = ld / VEC lanes per output row.
struct Lanes {
    int col;     // first column of this lane
    int gi;      // lane group index within the warp
    int gpw;     // lane groups per warp
    bool idle;   // lanes past the last whole group
};

__device__ __forceinline__ Lanes lanes_for(int ld, int vec) {
    Lanes L;
    const int G = ld / vec;
    const int lane = threadIdx.x & 31;
    L.gpw = 32 / G;
    L.gi = lane / G;
    L.col = (lane - L.gi * G) * vec;
    L.idle = L.gi >= L.gpw;
    return L;
}

struct Args {
    const int32_t *fptr[kMaxModes];  // levels 0..N-2 (used by the plain walk only)
    const int32_t *fids[kMaxModes];  // levels 0..N-1
    const void *fac[kMaxModes];      // by level; fac[0] unused
    const float *vals;
    const uint8_t *lvl;              // per-leaf first changed level
    const int32_t *part;             // [nchunks][N-1]
    int64_t nchunks;
    int64_t nnz;
    int32_t chunk;
    int32_t ld;
    float *out;                      // compact: nfibs[0] x ld, zeroed
    double *heavy;                   // nheavy x ld, zeroed
    const int32_t *hidx;             // per slice: heavy row index or -1
    const uint4 *leafrec;            // packed leaf records (flag kernels of mttkrp.cu)
};

// A factor row segment as loaded: W = 16 or 32 bytes per lane (4 or 8 FP32
// values, 8 or 16 BF16 values), widened to FP32 only where it is used. The
// 32-byte form is one 256-bit load, so a lane group of ld / VEC lanes still
// requests a whole row with one instruction while half as many lanes (and
// their per-leaf bookkeeping) are spent on it; it needs 32-byte aligned
// rows (ld * sizeof(T) and the base pointer multiples of 32).
template <int W>
struct Seg {
    uint32_t w[W / 4];
};

// SPLIT: a 32-byte segment is loaded as two 16-byte loads (for the batched
// kernel's non-inlined walk, where ptxas 13.0 fails on the 32-byte form).
template <typename T, int W = 16, bool SPLIT = false>
struct Raw {
    static_assert(W == 16 || W == 32, "16- or 32-byte row segments");
    static constexpr int VEC = W / (int)sizeof(T);
    using Row = Seg<W>;
    __device__ __forceinline__ static Row load(const void *base, int64_t row, int ld, int col) {
        const T *p = static_cast<const T *>(base) + row * ld + col;
        Row r;
        if constexpr (W == 16) {
            const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
            r.w[0] = u.x; r.w[1] = u.y; r.w[2] = u.z; r.w[3] = u.w;
        } else if constexpr (SPLIT) {
            const uint4 u0 = __ldg(reinterpret_cast<const uint4 *>(p));
            const uint4 u1 = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
            r.w[0] = u0.x; r.w[1] = u0.y; r.w[2] = u0.z; r.w[3] = u0.w;
            r.w[4] = u1.x; r.w[5] = u1.y; r.w[6] = u1.z; r.w[7] = u1.w;
        } else {
            asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]),
                  "=r"(r.w[4]), "=r"(r.w[5]), "=r"(r.w[6]), "=r"(r.w[7])
                : "l"(p));
        }
        return r;
    }
    // The same load issued only where p != 0; elsewhere the row is left
    // undefined (callers select it only where p != 0), so a warp requests
    // the sectors of its predicated-on lanes alone.
    __device__ __forceinline__ static Row load_if(uint32_t p, const void *base, int64_t row, int ld, int col) {
        const T *q = static_cast<const T *>(base) + row * ld + col;
        Row r;
        if constexpr (W == 16) {
            asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %5, 0;\n\t"
                "@p ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
                : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]) : "l"(q), "r"(p));
        } else if constexpr (SPLIT) {
            asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %9, 0;\n\t"
                "@p ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%8];\n\t"
                "@p ld.global.nc.v4.u32 {%4, %5, %6, %7}, [%8+16];\n\t}"
                : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]),
                  "=r"(r.w[4]), "=r"(r.w[5]), "=r"(r.w[6]), "=r"(r.w[7])
                : "l"(q), "r"(p));
        } else {
            asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %9, 0;\n\t"
                "@p ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t}"
                : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]),
                  "=r"(r.w[4]), "=r"(r.w[5]), "=r"(r.w[6]), "=r"(r.w[7])
                : "l"(q), "r"(p));
        }
        return r;
    }
    __device__ __forceinline__ static void widen(const Row &u, float (&x)[VEC]) {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) x[i] = __uint_as_float(u.w[i]);
        } else {
#pragma unroll
            for (int i = 0; i < W / 4; ++i) {  // bf16 -> f32 is exact: the bits move to the top half
                x[2 * i] = __uint_as_float(u.w[i] << 16);
                x[2 * i + 1] = __uint_as_float(u.w[i] & 0xffff0000u);
            }
        }
    }
};

// A leaf-factor row segment read from a copy of the whole leaf factor in
// shared memory (the table kernels of mttkrp.cu): row r starts at byte
// r * rowbytes of the table; a 32-byte segment is two 16-byte shared loads.
template <typename T, int W>
__device__ __forceinline__ Seg<W> load_table_row(uint32_t tab, int32_t row, uint32_t rowbytes, int col) {
    Seg<W> r;
    const uint32_t a = tab + (uint32_t)row * rowbytes + (uint32_t)col * (uint32_t)sizeof(T);
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]) : "r"(a));
    if constexpr (W == 32)
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.w[4]), "=r"(r.w[5]), "=r"(r.w[6]), "=r"(r.w[7]) : "r"(a + 16u));
    return r;
}

// Slice f is complete and owned by this lane group.
template <int VEC>
__device__ __forceinline__ void store_owned(const Args &a, int64_t f, int col, const float (&x)[VEC]) {
    float *dst = a.out + f * a.ld + col;
#pragma unroll
    for (int i = 0; i < VEC; i += 4)
        *reinterpret_cast<float4 *>(dst + i) = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
}

// A partial of slice f, which other chunks also touch.
template <int VEC>
__device__ __forceinline__ void add_partial(const Args &a, int64_t f, int col, const float (&x)[VEC]) {
    const int32_t h = __ldg(a.hidx + f);
    if (h >= 0) {
        double *dst = a.heavy + (int64_t)h * a.ld + col;
#pragma unroll
        for (int i = 0; i < VEC; ++i)
            asm volatile("red.global.add.f64 [%0], %1;" ::"l"(dst + i), "d"((double)x[i]) : "memory");
    } else {
        float *dst = a.out + f * a.ld + col;
#pragma unroll
        for (int i = 0; i < VEC; i += 4)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + i), "f"(x[i]),
                         "f"(x[i + 1]), "f"(x[i + 2]), "f"(x[i + 3])
                         : "memory");
    }
}

// Row f of the finished MTTKRP, column c.
__device__ __forceinline__ float read_row(const float *out, const double *heavy, const int32_t *hidx, int64_t f,
                                          int ld, int c) {
    const int32_t h = __ldg(hidx + f);
    return h >= 0 ? (float)heavy[(int64_t)h * ld + c] : out[f * ld + c];
}

// The partial of a heavy slice that a lane group holds back between its
// chunks (f < 0: none). Consecutive chunks of a group that lie in the same
// heavy slice are summed here and flushed once, which turns one FP64 atomic
// per chunk into one per run of chunks.
template <int VEC>
struct Carry {
    int64_t f = -1;
    float acc[VEC];
};

template <int VEC>
__device__ __forceinline__ void flush_carry(const Args &a, int col, Carry<VEC> &cy) {
    if (cy.f >= 0) add_partial<VEC>(a, cy.f, col, cy.acc);
    cy.f = -1;
}

// Start a chunk whose first slice is f0: a held-back partial of the same
// slice seeds the slice accumulator; any other is flushed.
template <int VEC>
__device__ __forceinline__ void take_carry(const Args &a, int col, Carry<VEC> &cy, int64_t f0, float (&acc0)[VEC]) {
    if (cy.f == f0) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc0[i] = cy.acc[i];
        cy.f = -1;
    } else {
        flush_carry<VEC>(a, col, cy);
    }
}

// End of a chunk: the open slice f's partial is held back if f is heavy.
template <int VEC>
__device__ __forceinline__ void end_chunk(const Args &a, int col, Carry<VEC> &cy, int64_t f, const float (&acc0)[VEC]) {
    if (__ldg(a.hidx + f) >= 0) {
        cy.f = f;
#pragma unroll
        for (int i = 0; i < VEC; ++i) cy.acc[i] = acc0[i];
    } else {
        add_partial<VEC>(a, f, col, acc0);
    }
}

// acc += x * y element-wise over VEC values; with 32-byte segments as packed
// FP32x2 FMAs (each element rounded exactly as fmaf rounds it).
template <int VEC, bool PACKED>
__device__ __forceinline__ void fma_vec(float (&acc)[VEC], const float (&x)[VEC], const float (&y)[VEC]) {
    if constexpr (PACKED) {
#pragma unroll
        for (int i = 0; i < VEC; i += 2) {
            const float2 r = __ffma2_rn(make_float2(x[i], x[i + 1]), make_float2(y[i], y[i + 1]),
                                        make_float2(acc[i], acc[i + 1]));
            acc[i] = r.x;
            acc[i + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[i] = fmaf(x[i], y[i], acc[i]);
    }
}

// t = x * y element-wise (packed FP32x2 multiplies with 32-byte segments).
template <int VEC, bool PACKED>
__device__ __forceinline__ void mul_vec(float (&t)[VEC], const float (&x)[VEC], const float (&y)[VEC]) {
    if constexpr (PACKED) {
#pragma unroll
        for (int i = 0; i < VEC; i += 2) {
            const float2 r = __fmul2_rn(make_float2(x[i], x[i + 1]), make_float2(y[i], y[i + 1]));
            t[i] = r.x;
            t[i + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) t[i] = __fmul_rn(x[i], y[i]);
    }
}

// acc += s * x element-wise (s broadcast).
template <int VEC, bool PACKED>
__device__ __forceinline__ void fma_scalar(float (&acc)[VEC], float s, const float (&x)[VEC]) {
    if constexpr (PACKED) {
#pragma unroll
        for (int i = 0; i < VEC; i += 2) {
            const float2 r = __ffma2_rn(make_float2(s, s), make_float2(x[i], x[i + 1]),
                                        make_float2(acc[i], acc[i + 1]));
            acc[i] = r.x;
            acc[i + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[i] = fmaf(s, x[i], acc[i]);
    }
}

// parent += row * child (element-wise); child = 0.
template <typename T, int W = 16>
__device__ __forceinline__ void fold(float (&parent)[Raw<T, W>::VEC], float (&child)[Raw<T, W>::VEC],
                                     const typename Raw<T, W>::Row &row) {
    constexpr int VEC = Raw<T, W>::VEC;
    float r[VEC];
    Raw<T, W>::widen(row, r);
    fma_vec<VEC, W == 32>(parent, r, child);
#pragma unroll
    for (int i = 0; i < VEC; ++i) child[i] = 0.f;
}

// Where a chunk's leaf records (values, leaf indices, level flags) are read
// from: global memory, or a copy staged in shared memory.
struct GlobalRecs {
    static constexpr bool kPacked = false;
    static constexpr bool kSplit = false;
    const float *vals;
    const int32_t *idx;
    const uint8_t *lvl;
    __device__ __forceinline__ float4 v4(int64_t k) const { return __ldg(reinterpret_cast<const float4 *>(vals + k)); }
    __device__ __forceinline__ int4 i4(int64_t k) const { return __ldg(reinterpret_cast<const int4 *>(idx + k)); }
    __device__ __forceinline__ uint32_t l4(int64_t k) const { return __ldg(reinterpret_cast<const uint32_t *>(lvl + k)); }
    __device__ __forceinline__ uint2 l8(int64_t k) const { return __ldg(reinterpret_cast<const uint2 *>(lvl + k)); }
    __device__ __forceinline__ float2 v2(int64_t k) const { return __ldg(reinterpret_cast<const float2 *>(vals + k)); }
    __device__ __forceinline__ int2 i2(int64_t k) const { return __ldg(reinterpret_cast<const int2 *>(idx + k)); }
    __device__ __forceinline__ uint32_t l2(int64_t k) const {
        return __ldg(reinterpret_cast<const unsigned short *>(lvl + k));
    }
};

struct SharedRecs {  // shared-memory addresses of the chunk's copy; k0 = the chunk's first leaf
    static constexpr bool kPacked = false;
    static constexpr bool kSplit = false;
    uint32_t sv, si, sl;
    int64_t k0;
    __device__ __forceinline__ float4 v4(int64_t k) const {
        float4 r;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(sv + (uint32_t)(k - k0) * 4u));
        return r;
    }
    __device__ __forceinline__ int4 i4(int64_t k) const {
        int4 r;
        asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(si + (uint32_t)(k - k0) * 4u));
        return r;
    }
    __device__ __forceinline__ uint32_t l4(int64_t k) const {
        uint32_t r;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(sl + (uint32_t)(k - k0)));
        return r;
    }
    __device__ __forceinline__ uint2 l8(int64_t k) const {
        uint2 r;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(sl + (uint32_t)(k - k0)));
        return r;
    }
    __device__ __forceinline__ float2 v2(int64_t k) const {
        float2 r;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(sv + (uint32_t)(k - k0) * 4u));
        return r;
    }
    __device__ __forceinline__ int2 i2(int64_t k) const {
        int2 r;
        asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(si + (uint32_t)(k - k0) * 4u));
        return r;
    }
    __device__ __forceinline__ uint32_t l2(int64_t k) const {
        uint32_t r;
        asm volatile("ld.shared.u16 %0, [%1];" : "=r"(r) : "r"(sl + (uint32_t)(k - k0)));
        return r;
    }
};

// The records of the B leaves from kb on: values, leaf indices and the
// packed level flags (byte j of lw[j / 4] = leaf kb + j).
template <int B, typename Recs>
__device__ __forceinline__ void fetch_batch(const Recs &rec, int64_t kb, float (&v)[B], int32_t (&li)[B],
                                            uint32_t (&lw)[2]) {
    if constexpr (B == 2) {
        const float2 va = rec.v2(kb);
        const int2 ia = rec.i2(kb);
        v[0] = va.x; v[1 % B] = va.y;
        li[0] = ia.x; li[1 % B] = ia.y;
        lw[0] = rec.l2(kb);
    } else {
        const float4 va = rec.v4(kb);
        const int4 ia = rec.i4(kb);
        v[0] = va.x; v[1 % B] = va.y; v[2 % B] = va.z; v[3 % B] = va.w;
        li[0] = ia.x; li[1 % B] = ia.y; li[2 % B] = ia.z; li[3 % B] = ia.w;
        if constexpr (B == 8) {
            const float4 vb = rec.v4(kb + 4);
            const int4 ib = rec.i4(kb + 4);
            v[4 % B] = vb.x; v[5 % B] = vb.y; v[6 % B] = vb.z; v[7 % B] = vb.w;
            li[4 % B] = ib.x; li[5 % B] = ib.y; li[6 % B] = ib.z; li[7 % B] = ib.w;
            const uint2 l2 = rec.l8(kb);
            lw[0] = l2.x;
            lw[1] = l2.y;
        } else {
            lw[0] = rec.l4(kb);
        }
    }
}

// One 16-byte record per leaf (sptt_csf::leafrec): x = leaf index, y = the
// value's bits, z = the index of the level-(N-2) fiber the leaf opens (0 if
// it opens none), w = the leaf's level flag. A batch of leaves arrives in
// 32-byte loads, and the factor row of a fiber that opens needs no other
// load first.
// Two records are loaded with L1::no_allocate (a record is read once, so an
// L1 line given to it only evicts factor rows) and an L2 prefetch size of
// 256 bytes (the chunk's next records arrive in L2 with the first). Measured
// on the 1e8-non-zero 3-mode power-law tensor, R = 16: 5-6 % off the MTTKRP,
// each hint giving about half; L1::evict_last on the factor rows adds nothing.
// On the separate leaf arrays the same hints cost 13-20 %: their 4- to
// 16-byte loads reuse the 32-byte sector that an earlier batch brought to L1.
// SPLIT issues the pair as two 16-byte loads (ptxas 13.0 stops with a
// segmentation fault on the 32-byte form inside the batched kernel's
// non-inlined walk).
template <bool SPLIT = false>
__device__ __forceinline__ void load_rec_pair(const uint4 *p, uint32_t (&r)[8]) {
    if constexpr (SPLIT) {
        asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(p));
        asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
            : "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) : "l"(p + 1));
    } else {
        asm("ld.global.nc.L1::no_allocate.L2::256B.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
            : "l"(p));
    }
}

template <bool SPLIT = false>
struct PackedRecsT {
    static constexpr bool kPacked = true;
    static constexpr bool kSplit = SPLIT;
    const uint4 *rec;
};
using PackedRecs = PackedRecsT<false>;

// Records of the B leaves from kb on, and nf: for packed records the index
// of the fiber each leaf opens; otherwise the indices of the B level-LF
// fibers after fiber fb (the fibers a batch can open, in order).
template <int B, int LF, typename Recs>
__device__ __forceinline__ void fetch_all(const Recs &rec, const int32_t *fids_lf, int64_t fb, int64_t kb,
                                          float (&v)[B], int32_t (&li)[B], uint32_t (&lw)[2], int32_t (&nf)[B]) {
    if constexpr (Recs::kPacked) {
        lw[0] = 0u;
        lw[1] = 0u;
#pragma unroll
        for (int h = 0; h < B; h += 2) {
            uint32_t r[8];
            load_rec_pair<Recs::kSplit>(rec.rec + kb + h, r);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = h + q;
                li[j] = (int32_t)r[4 * q];
                v[j] = __uint_as_float(r[4 * q + 1]);
                nf[j] = (int32_t)r[4 * q + 2];
                lw[j >> 2] |= (r[4 * q + 3] & 0xffu) << (8 * (j & 3));
            }
        }
    } else {
        fetch_batch<B>(rec, kb, v, li, lw);
        if constexpr (LF >= 1) {
            const int32_t *fp = fids_lf + fb + 1;
#pragma unroll
            for (int q = 0; q < B; ++q) nf[q] = __ldg(fp + q);
        }
    }
}

// The batched walk driven by the per-leaf level flags. A lane group takes
// its chunk in batches of B leaves: the batch's values, leaf indices and
// level flags arrive in vector loads; then every factor row the batch needs
// (the B leaf rows, and the rows of the level-(N-2) fibers that open inside
// the batch, whose ids are consecutive) is requested before any is used.
// Rows of fibers at higher levels are requested when the fiber opens and
// used when it closes.
//
// DIRECT (N >= 3): a leaf adds v * (row of its level-(N-2) fiber) * (leaf row)
// straight into the fiber's parent accumulator, instead of summing the
// fiber's leaves first and multiplying by the fiber's row when it closes.
// One more multiply per leaf, but an opening fiber only switches the row:
// no fold and no clearing, which in a warp of 16 lane groups runs at almost
// every leaf (some group nearly always opens a fiber).
template <int NM, typename T, int B, typename Recs = GlobalRecs, int W = 16, bool PIPE = true, bool DIRECT = false>
__device__ __forceinline__ void flag_chunk(const Args &a, int64_t c, int col, Carry<Raw<T, W>::VEC> &cy,
                                           const Recs &rec) {
    using Rw = Raw<T, W, Recs::kSplit>;
    using Row = typename Rw::Row;
    constexpr int VEC = Rw::VEC;
    constexpr int NL = NM - 1;  // accumulator levels 0..NM-2
    constexpr int LF = NM - 2;  // level of the leaves' parent fibers
    static_assert(B == 2 || B == 4 || B == 8, "batch of 2, 4 or 8 leaves");
    const int ld = a.ld;
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
    Row rowc[NL];  // rows of the open fibers, levels 1..NL-1
#pragma unroll
    for (int l = 1; l < NL; ++l) rowc[l] = Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col);
    constexpr bool kDirect = DIRECT && LF >= 1;
    float rf[VEC];  // DIRECT: the open leaf-parent fiber's row, widened
    if constexpr (kDirect) Rw::widen(rowc[LF], rf);
    bool first_slice = true;
    take_carry<VEC>(a, col, cy, f[0], acc[0]);

    // Each batch requests, with its records, the ids of the next B level-LF
    // fibers: the fibers a batch opens have consecutive ids, so their rows
    // need not wait for the flags and then for the ids. With PIPE the walk
    // is also software-pipelined: while a batch's factor rows are in flight,
    // the next batch's records and next fiber ids (after the ones this batch
    // opens, which its flags count) are requested, so a batch's row requests
    // wait for no load of their own batch; it costs about 3B + 2 registers.
    // The level arrays carry 64 elements of slack past their end and the
    // leaf arrays more; a prefetched id is used only for a fiber that really
    // opens.
    float v[B];
    int32_t li[B];
    uint32_t lw[2] = {0u, 0u};
    int32_t nf[B];
    const int32_t *fids_lf = a.fids[LF > 0 ? LF : 0];
    if constexpr (PIPE) fetch_all<B, LF>(rec, fids_lf, f[LF], k0, v, li, lw, nf);
    for (int64_t kb = k0; kb < k1; kb += B) {
        if constexpr (!PIPE) fetch_all<B, LF>(rec, fids_lf, f[LF], kb, v, li, lw, nf);
        const int nvalid = (k1 - kb < B) ? (int)(k1 - kb) : B;
        Row x[B];
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (j < nvalid) x[j] = Rw::load(a.fac[NM - 1], li[j], ld, col);
        // leaves that open a new level-LF fiber (never the chunk's first
        // leaf): a per-byte compare of the packed flags, whose 0/1 bytes a
        // multiply gathers into bits 24..27 (bit 24 + j = byte j)
        uint32_t sm = 0;
#pragma unroll
        for (int w = 0; w < (B + 3) / 4; ++w) {
            const uint32_t le = __vcmpleu4(lw[w], (uint32_t)LF * 0x01010101u) & 0x01010101u;
            sm |= (((le * 0x01020408u) >> 24) & 0xfu) << (4 * w);
        }
        sm &= (nvalid >= 32) ? 0xffffffffu : ((1u << nvalid) - 1u);
        if (kb == k0) sm &= ~1u;
        Row nr[B];
        if constexpr (LF >= 1) {
#pragma unroll
            for (int j = 0; j < B; ++j)
                if ((sm >> j) & 1u) {
                    int32_t id;
                    if constexpr (Recs::kPacked) {
                        id = nf[j];
                    } else {
                        const int pos = __popc(sm & ((1u << j) - 1u));  // openings before leaf j
                        id = nf[0];
#pragma unroll
                        for (int q = 1; q <= j; ++q) id = (pos == q) ? nf[q] : id;
                    }
                    nr[j] = Rw::load(a.fac[LF], id, ld, col);
                }
        }
        const bool more = PIPE && kb + B < k1;
        float vn[B];
        int32_t lin[B];
        uint32_t lwn[2] = {0u, 0u};
        int32_t nfn[B];
        if (more) fetch_all<B, LF>(rec, fids_lf, f[LF] + __popc(sm), kb + B, vn, lin, lwn, nfn);
#pragma unroll
        for (int j = 0; j < B; ++j) {
            if (j >= nvalid) break;
            if ((sm >> j) & 1u) {
                const int d = (int)((lw[j >> 2] >> (8 * (j & 3))) & 0xffu);
                if constexpr (kDirect) {
                    ++f[LF];
                    Rw::widen(nr[j], rf);
                } else if constexpr (LF >= 1) {
                    fold<T, W>(acc[LF - 1], acc[LF], rowc[LF]);
                    ++f[LF];
                    rowc[LF] = nr[j];
                }
#pragma unroll
                for (int l = LF - 1; l >= 1; --l) {
                    if (d <= l) {
                        fold<T, W>(acc[l - 1], acc[l], rowc[l]);
                        ++f[l];
                        rowc[l] = Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col);
                    }
                }
                if (d == 0) {  // the slice is complete
                    if (first_slice) add_partial<VEC>(a, f[0], col, acc[0]);
                    else store_owned<VEC>(a, f[0], col, acc[0]);
                    first_slice = false;
#pragma unroll
                    for (int i = 0; i < VEC; ++i) acc[0][i] = 0.f;
                    ++f[0];
                }
            }
            float xr[VEC];
            Rw::widen(x[j], xr);
            if constexpr (kDirect) {
                float t[VEC];
                mul_vec<VEC, W == 32>(t, rf, xr);
                fma_scalar<VEC, W == 32>(acc[LF - 1], v[j], t);
            } else {
                fma_scalar<VEC, W == 32>(acc[LF], v[j], xr);
            }
        }
        if (more) {
#pragma unroll
            for (int q = 0; q < B; ++q) {
                v[q] = vn[q];
                li[q] = lin[q];
                if constexpr (LF >= 1) nf[q] = nfn[q];
            }
            lw[0] = lwn[0];
            lw[1] = lwn[1];
        }
    }
    // chunk end: fold the open fibers; the open slice's partial is added
    // (or held back when the slice is heavy)
#pragma unroll
    for (int l = kDirect ? LF - 1 : LF; l >= 1; --l) fold<T, W>(acc[l - 1], acc[l], rowc[l]);
    end_chunk<VEC>(a, col, cy, f[0], acc[0]);
}

// The select walk: the DIRECT form of flag_chunk on packed records with the
// per-leaf work kept free of branches, so that the lane groups of a warp,
// which open fibers at different leaves, no longer serialise each other.
//
// Per leaf j of a batch: the row of the fiber the leaf opens (if it opens
// one) was requested with the batch's leaf rows; the open leaf-parent
// fiber's row rf is replaced by it with a select, and v * (rf * x) is added
// to the accumulator of the level above (one multiply and one FMA per
// element, the same arithmetic as DIRECT). Only a change at a level above
// the leaf parents -- a new slice, or for N >= 4 a new upper fiber --
// branches, and at most a few groups take that branch per batch.
//
// Loads are issued unconditionally: a leaf that opens no fiber has fiber
// index 0 in its record (row 0, which every such lane shares), and the
// leaves of a ragged last batch read the zero records past the end of the
// array (their values are masked to 0 and their flags ignored).
//
// TAB: the leaf rows come from the shared-memory copy of the whole leaf
// factor at shared address tab (row r at byte r * tab_rowbytes), not from
// global memory.
//
// SPLIT: 32-byte loads issued as 16-byte halves (the batched kernel's
// non-inlined walk; see Raw).
// Records of the B leaves from k on for the select walk: leaf index, value,
// the row index of the leaf-parent fiber a leaf opens (0 where it opens
// none), and the level flags packed one per byte (bytes past B undefined).
template <int B, bool SPLIT>
__device__ __forceinline__ void fetch_sel(const uint4 *p, float (&v)[B], int32_t (&li)[B], int32_t (&nf)[B],
                                          uint32_t (&lw)[(B + 3) / 4]) {
    uint32_t fl[B];
#pragma unroll
    for (int h = 0; h < B; h += 2) {
        uint32_t r[8];
        load_rec_pair<SPLIT>(p + h, r);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            li[h + q] = (int32_t)r[4 * q];
            v[h + q] = __uint_as_float(r[4 * q + 1]);
            nf[h + q] = (int32_t)r[4 * q + 2];
            fl[h + q] = r[4 * q + 3];
        }
    }
#pragma unroll
    for (int w = 0; w < (B + 3) / 4; ++w) {
        const uint32_t lo = __byte_perm(fl[4 * w], fl[4 * w + 1], 0x3340u);
        lw[w] = (B - 4 * w >= 4) ? __byte_perm(lo, __byte_perm(fl[4 * w + 2], fl[4 * w + 3], 0x3340u), 0x5410u)
                                 : lo;
    }
}

// The select walk: each leaf is added straight into the accumulator of the
// level above its leaf-parent fiber, v * (row of the open leaf-parent fiber)
// (.) (leaf row); a leaf that opens a new leaf-parent fiber swaps that row
// (a select, so the per-leaf work has no branch). A batch in which a fiber
// above the leaf parents closes (a slice change for N = 3) in some lane
// group of the warp takes the general path, which tests every leaf and
// folds the closing levels at the right one.
//
// The level flags d (the first tree level that changes at a leaf, 0..NM-1;
// the zero-value slack records past the last leaf carry NM-1, "opens
// nothing") are tested a byte at a time: with d <= 4, d + (0x80 - k) sets
// bit 7 of its byte exactly when d >= k, with no carry between bytes.
// Chunks are whole batches (a power-of-two chunk of at least 16 leaves), so
// only the tensor's last batch reaches the slack, whose records add zero.
// The rows of newly opened fibers are loaded only by the lanes that need
// them (a predicated load), so a warp requests no sectors for the others.
template <int B>
__device__ __forceinline__ void opening_bits(const uint32_t (&lw)[(B + 3) / 4], uint32_t (&opn)[(B + 3) / 4],
                                             uint32_t k_open) {
#pragma unroll
    for (int w = 0; w < (B + 3) / 4; ++w)
        opn[w] = ~(lw[w] + k_open) & ((B - 4 * w >= 4) ? 0x80808080u : 0x00008080u);
}

template <int NM, typename T, int B, int W = 32, bool TAB = false, bool SPLIT = false>
__device__ __forceinline__ void select_chunk(const Args &a, int64_t c, int col, Carry<Raw<T, W>::VEC> &cy,
                                             const PackedRecsT<SPLIT> &rec, uint32_t tab = 0,
                                             uint32_t tab_rowbytes = 0) {
    using Rw = Raw<T, W, SPLIT>;
    using Row = typename Rw::Row;
    constexpr int VEC = Rw::VEC;
    constexpr int NL = NM - 1;             // accumulator levels 0..NM-2
    constexpr int LF = NM - 2;             // level of the leaves' parent fibers
    constexpr int AL = LF >= 1 ? LF - 1 : 0;  // the level leaves add into
    constexpr int NACC = AL + 1;
    constexpr int UP = LF >= 1 ? LF : 1;   // d < UP: a fiber above the leaf parents (or the slice) closes
    constexpr int NW = (B + 3) / 4;
    constexpr uint32_t kOpen = (0x80u - (uint32_t)(NM - 1)) * 0x01010101u;
    constexpr uint32_t kUp = (0x80u - (uint32_t)UP) * 0x01010101u;
    static_assert(B == 2 || B == 4 || B == 8, "batch of 2, 4 or 8 leaves");
    static_assert(NM <= 5, "level flags up to 4");
    const int ld = a.ld;
    const int64_t k0 = c * (int64_t)a.chunk;
    const int n = (int)(((k0 + a.chunk < a.nnz) ? k0 + a.chunk : a.nnz) - k0);
    const uint4 *rp = rec.rec + k0;
    int32_t f[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) f[l] = __ldg(a.part + c * NL + l);
    float acc[NACC][VEC];
#pragma unroll
    for (int l = 0; l < NACC; ++l)
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[l][i] = 0.f;
    Row rowc[NL];  // rows of the open fibers at levels 1..LF-1
#pragma unroll
    for (int l = 1; l < LF; ++l) rowc[l] = Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col);
    float rf[VEC];
    if constexpr (LF >= 1) Rw::widen(Rw::load(a.fac[LF], __ldg(a.fids[LF] + f[LF]), ld, col), rf);
    bool first_slice = true;
    take_carry<VEC>(a, col, cy, f[0], acc[0]);

    float v[B];
    int32_t li[B];
    int32_t nf[B];
    uint32_t lw[NW];
    fetch_sel<B, SPLIT>(rp, v, li, nf, lw);
    uint32_t first = ~0x80u;  // the chunk's first leaf continues the fibers the partition gives
    for (int o = 0; o < n; o += B) {
        // bit 7 of byte j: leaf j opens a leaf-parent fiber (opn); rare: some
        // leaf of the batch also closes a fiber above the leaf parents
        uint32_t opn[NW];
        opening_bits<B>(lw, opn, kOpen);
        opn[0] &= first;
        first = ~0u;
        bool rare = false;
#pragma unroll
        for (int w = 0; w < NW; ++w) rare |= (~(lw[w] + kUp) & opn[w]) != 0u;
        Row x[B], nr[B];
        if constexpr (LF >= 1) {
#pragma unroll
            for (int j = 0; j < B; ++j)
                nr[j] = Rw::load_if((opn[j >> 2] >> (8 * (j & 3) + 7)) & 1u, a.fac[LF], nf[j], ld, col);
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            if constexpr (TAB) x[j] = load_table_row<T, W>(tab, li[j], tab_rowbytes, col);
            else x[j] = Rw::load(a.fac[NM - 1], li[j], ld, col);
        }
        // the next batch's records (past the chunk end they belong to the
        // next chunk or to the slack; never used there)
        float vn[B];
        int32_t lin[B];
        int32_t nfn[B];
        uint32_t lwn[NW];
        fetch_sel<B, SPLIT>(rp + o + B, vn, lin, nfn, lwn);
        // one path for the whole warp: the general path when any of its lane
        // groups needs it, so the two never run one after the other
        if (!__any_sync(__activemask(), rare)) {
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const bool op = (opn[j >> 2] >> (8 * (j & 3) + 7)) & 1u;
                float xr[VEC];
                Rw::widen(x[j], xr);
                if constexpr (LF >= 1) {
                    float nw[VEC];
                    Rw::widen(nr[j], nw);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) rf[i] = op ? nw[i] : rf[i];
                    float t[VEC];
                    mul_vec<VEC, W == 32>(t, rf, xr);
                    fma_scalar<VEC, W == 32>(acc[AL], v[j], t);
                } else {
                    fma_scalar<VEC, W == 32>(acc[0], v[j], xr);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const bool op = (opn[j >> 2] >> (8 * (j & 3) + 7)) & 1u;
                const int d = (int)((lw[j >> 2] >> (8 * (j & 3))) & 0xffu);
                if (op && d < UP) {
                    // a fiber above the leaf parents closes: fold the levels
                    // that close into their parents, and store a finished slice
#pragma unroll
                    for (int l = LF - 1; l >= 1; --l) {
                        if (d <= l) {
                            fold<T, W>(acc[l - 1], acc[l], rowc[l]);
                            ++f[l];
                            rowc[l] = Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col);
                        }
                    }
                    if (d == 0) {
                        if (first_slice) add_partial<VEC>(a, f[0], col, acc[0]);
                        else store_owned<VEC>(a, f[0], col, acc[0]);
                        first_slice = false;
#pragma unroll
                        for (int i = 0; i < VEC; ++i) acc[0][i] = 0.f;
                        ++f[0];
                    }
                }
                float xr[VEC];
                Rw::widen(x[j], xr);
                if constexpr (LF >= 1) {
                    float nw[VEC];
                    Rw::widen(nr[j], nw);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) rf[i] = op ? nw[i] : rf[i];
                    float t[VEC];
                    mul_vec<VEC, W == 32>(t, rf, xr);
                    fma_scalar<VEC, W == 32>(acc[AL], v[j], t);
                } else {
                    fma_scalar<VEC, W == 32>(acc[0], v[j], xr);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < B; ++q) {
            v[q] = vn[q];
            li[q] = lin[q];
            nf[q] = nfn[q];
        }
#pragma unroll
        for (int w = 0; w < NW; ++w) lw[w] = lwn[w];
    }
    // chunk end: fold the open upper fibers; the open slice's partial is
    // added (or held back when the slice is heavy)
#pragma unroll
    for (int l = LF - 1; l >= 1; --l) fold<T, W>(acc[l - 1], acc[l], rowc[l]);
    end_chunk<VEC>(a, col, cy, f[0], acc[0]);
}

// The plain walk: one leaf at a time, fiber ends read from fptr.
template <int NM, typename T>
__device__ __forceinline__ void plain_chunk(const Args &a, int64_t c, int col, Carry<Raw<T>::VEC> &cy) {
    using Rw = Raw<T>;
    constexpr int VEC = Rw::VEC;
    constexpr int NL = NM - 1;
    const int ld = a.ld;
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
    take_carry<VEC>(a, col, cy, f[0], acc[0]);
    for (int64_t k = k0; k < k1; ++k) {
        if (k != k0 && k == end[NL - 1]) {
            // leaf k opens a new level-(N-2) fiber: close the finished fibers
            // bottom-up, folding each into its parent with the fiber's row
            bool to_root = true;
#pragma unroll
            for (int l = NL - 1; l >= 1; --l) {
                fold<T>(acc[l - 1], acc[l], Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col));
                ++f[l];
                end[l] = __ldg(a.fptr[l] + f[l] + 1);
                if (f[l] != end[l - 1]) {
                    to_root = false;
                    break;
                }
            }
            if (to_root) {  // the slice is complete
                if (first_slice) add_partial<VEC>(a, f[0], col, acc[0]);
                else store_owned<VEC>(a, f[0], col, acc[0]);
                first_slice = false;
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc[0][i] = 0.f;
                ++f[0];
                end[0] = __ldg(a.fptr[0] + f[0] + 1);
            }
        }
        const float v = __ldg(a.vals + k);
        float x[VEC];
        Rw::widen(Rw::load(a.fac[NM - 1], __ldg(a.fids[NM - 1] + k), ld, col), x);
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[NL - 1][i] = fmaf(v, x[i], acc[NL - 1][i]);
    }
#pragma unroll
    for (int l = NL - 1; l >= 1; --l)
        fold<T>(acc[l - 1], acc[l], Rw::load(a.fac[l], __ldg(a.fids[l] + f[l]), ld, col));
    end_chunk<VEC>(a, col, cy, f[0], acc[0]);
}

}  // namespace walk
}  // namespace sptt
