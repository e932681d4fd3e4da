// Dense R x R work of CP-ALS (Algorithm 1): Grams and their Hadamard product,
// the normal-equation solve A = M V^dagger (V^dagger through Cholesky,
// Section V-A), column normalisation into lambda and the fit.
//
// Precision: the R x R matrices (Grams, V, its factor and inverse) are FP64.
// The row-wise work over I_n x R data runs on FP32 CUDA cores: products in
// FP32, summed in FP32 over a tile of rows, tile sums accumulated in FP64
// (GB300's FP64 pipe is too slow for I_n * R^2 FP64 FMAs).
#include "dense_dev.cuh"
#include "walk.cuh"

namespace sptt {
namespace {

using dense::GramPtrs;
using dense::block_sum_d;

constexpr int kThreads = 256;
constexpr int kGramRows = 64;   // rows per tile of the Gram kernel

// ---------------------------------------------------------------------------
// Gram: partials[block][a*rank+b] = sum over the block's rows of A[i,a] A[i,b]
// ---------------------------------------------------------------------------
template <int RP>
__global__ void __launch_bounds__(kThreads) gram_kernel(const float *__restrict__ A, int64_t rows, int rank,
                                                        int ld, double *__restrict__ partials, int pstride) {
    constexpr int E = RP / 16;
    __shared__ float T[kGramRows][RP + 1];
    const int t = threadIdx.x, ta = t / 16, tb = t % 16;
    double acc[E][E];
#pragma unroll
    for (int x = 0; x < E; ++x)
#pragma unroll
        for (int y = 0; y < E; ++y) acc[x][y] = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * kGramRows; i0 < rows; i0 += (int64_t)gridDim.x * kGramRows) {
        for (int e = t; e < kGramRows * RP; e += kThreads) {
            const int r = e / RP, c = e % RP;
            const int64_t i = i0 + r;
            T[r][c] = (i < rows && c < rank) ? A[i * ld + c] : 0.f;
        }
        __syncthreads();
        float s[E][E];
#pragma unroll
        for (int x = 0; x < E; ++x)
#pragma unroll
            for (int y = 0; y < E; ++y) s[x][y] = 0.f;
#pragma unroll 4
        for (int r = 0; r < kGramRows; ++r) {
            float xa[E], xb[E];
#pragma unroll
            for (int x = 0; x < E; ++x) {
                xa[x] = T[r][ta * E + x];
                xb[x] = T[r][tb * E + x];
            }
#pragma unroll
            for (int x = 0; x < E; ++x)
#pragma unroll
                for (int y = 0; y < E; ++y) s[x][y] = fmaf(xa[x], xb[y], s[x][y]);
        }
#pragma unroll
        for (int x = 0; x < E; ++x)
#pragma unroll
            for (int y = 0; y < E; ++y) acc[x][y] += (double)s[x][y];
        __syncthreads();
    }
    double *P = partials + (int64_t)blockIdx.x * pstride;
#pragma unroll
    for (int x = 0; x < E; ++x)
#pragma unroll
        for (int y = 0; y < E; ++y) {
            const int a = ta * E + x, b = tb * E + y;
            if (a < rank && b < rank) P[a * rank + b] = acc[x][y];
        }
}

// out[e] = sum_b partials[b][e]: 32 lanes per element each sum every 32nd
// block, then the 32 lane sums are added in lane order (deterministic).
constexpr int kRedLanes = 32;
__global__ void reduce_partials_kernel(const double *__restrict__ partials, int nblocks, int pstride, int nelem,
                                       double *__restrict__ out) {
    __shared__ double s[kRedLanes][33];
    const int e = blockIdx.x * 32 + threadIdx.x;
    double v = 0.0;
    if (e < nelem) {
#pragma unroll 4
        for (int b = threadIdx.y; b < nblocks; b += kRedLanes) v += partials[(int64_t)b * pstride + e];
    }
    s[threadIdx.y][threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.y == 0 && e < nelem) {
        double t = 0.0;
#pragma unroll
        for (int y = 0; y < kRedLanes; ++y) t += s[y][threadIdx.x];
        out[e] = t;
    }
}

// ---------------------------------------------------------------------------
// Fused post-solve: A_un = M W, plus Gram(A_un) and column dots M.A_un.
// M is compact (row f = slice f, whose mode index is fids0[f]); the result
// rows are scattered to A[fids0[f]]. Rows of A with no slice are zero (the
// caller zeroes A first), and contribute nothing to the Gram or the dots.
// ---------------------------------------------------------------------------
template <int RP>
__global__ void __launch_bounds__(kThreads) postsolve_kernel(const float *__restrict__ M,
                                                             const double *__restrict__ heavy,
                                                             const int32_t *__restrict__ hidx,
                                                             const int32_t *__restrict__ fids0,
                                                             float *__restrict__ A,
                                                             int64_t rows, int rank, int ld,
                                                             const float *__restrict__ Wg,
                                                             double *__restrict__ partials, int pstride) {
    using ST = dense::SolveTile<RP>;
    extern __shared__ __align__(16) unsigned char solve_smem[];
    ST &sm = *reinterpret_cast<ST *>(solve_smem);
    dense::solve_load_w(sm, Wg, rank);
    dense::SolveRun acc;
    dense::solve_begin(sm, acc);
    for (int64_t i0 = (int64_t)blockIdx.x * ST::TR; i0 < rows; i0 += (int64_t)gridDim.x * ST::TR)
        dense::solve_tile<RP, false>(sm, acc, const_cast<float *>(M), const_cast<double *>(heavy), hidx, fids0, A,
                                     i0, rows, rank, ld);
    double *P = partials + (int64_t)blockIdx.x * pstride;
    dense::solve_reduce(sm, acc, rank, [&](int e, double v) { P[e] = v; });
}

// ---------------------------------------------------------------------------
// V = Hadamard_{m != n} G_m; W = V^dagger in FP64 (one CTA).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) normal_prep_kernel(GramPtrs g, int nmodes, int n, int rank,
                                                               float *__restrict__ W, int32_t *__restrict__ branch) {
    extern __shared__ double sm[];
    dense::normal_prep_body(g, nmodes, n, rank, W, branch, sm);
}

// lambda_r = sqrt(Gun_rr); G_n = D^-1 Gun D^-1; inner = sum of column dots
// (CTA 0), and every CTA scales its share of the rows of A by 1 / lambda
// (with its BF16 copy): the column normalisation of Algorithm 1 in one
// launch. Each CTA forms 1 / lambda from Gun itself, with the same FP64
// expression as CTA 0, so every row sees the values stored in inv_lambda.
__global__ void finalize_normalize_kernel(const double *__restrict__ gun, int rank, double *__restrict__ Gn,
                                          double *__restrict__ lambda, float *__restrict__ inv_lambda,
                                          double *__restrict__ inner, float *__restrict__ A,
                                          __nv_bfloat16 *__restrict__ Ab, const int32_t *__restrict__ fids0,
                                          int64_t rows, int ld) {
    __shared__ float inv[SPTT_MAX_RANK_ALS];
    if (blockIdx.x == 0) dense::finalize_body(gun, rank, Gn, lambda, inv_lambda, inner);
    for (int t = threadIdx.x; t < rank; t += blockDim.x) {
        const double d = gun[t * rank + t];
        const double l = d > 0.0 ? sqrt(d) : 0.0;
        inv[t] = (float)(l > 0.0 ? 1.0 / l : 0.0);
    }
    __syncthreads();
    const int qpr = ld / 4;  // float4 groups per row
    const int64_t total4 = rows * qpr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total4;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / qpr;
        const int c0 = (int)(t - f * qpr) * 4;
        const int64_t q = ((fids0 ? (int64_t)__ldg(fids0 + f) : f) * ld + c0) / 4;
        float4 v = reinterpret_cast<float4 *>(A)[q];
        float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = (c0 + j < rank) ? x[j] * inv[c0 + j] : 0.f;
        reinterpret_cast<float4 *>(A)[q] = make_float4(x[0], x[1], x[2], x[3]);
        if (Ab) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(x[0], x[1]);
            __nv_bfloat162 hi = __floats2bfloat162_rn(x[2], x[3]);
            reinterpret_cast<__nv_bfloat162 *>(Ab)[2 * q] = lo;
            reinterpret_cast<__nv_bfloat162 *>(Ab)[2 * q + 1] = hi;
        }
    }
}

// fit = 1 - sqrt(max(0, |X|^2 + lambda^T (*_m G_m) lambda - 2 inner)) / |X|,
// stored at ring[*counter % ring_len]; the counter is then advanced, so the
// same launch can be replayed from a captured graph.
__global__ void fit_kernel(GramPtrs g, int nmodes, int rank, const double *__restrict__ normx2,
                           const double *__restrict__ lambda, const double *__restrict__ inner,
                           double *__restrict__ ring, int ring_len, int64_t *__restrict__ counter) {
    __shared__ double red[32];
    double s = 0.0;
    for (int e = threadIdx.x; e < rank * rank; e += blockDim.x) {
        double h = lambda[e / rank] * lambda[e % rank];
        for (int m = 0; m < nmodes; ++m) h *= g.p[m][e];
        s += h;
    }
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) {
        const double nx = *normx2;
        double r2 = nx + s - 2.0 * (*inner);
        if (r2 < 0.0) r2 = 0.0;
        const int64_t it = *counter;
        ring[it % ring_len] = (nx == 0.0) ? (r2 == 0.0 ? 1.0 : 0.0) : 1.0 - sqrt(r2) / sqrt(nx);
        *counter = it + 1;
    }
}

__global__ void sumsq_partial_kernel(const float *__restrict__ v, int64_t n, double *__restrict__ part) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = v[i];
        s += x * x;
    }
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_kernel(const double *__restrict__ part, int n, double *__restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) *out = s;
}

// Philox4x64-10 (Salmon et al., SC'11): 10 rounds; multipliers
// 0xD2E7470EE14C6C93 / 0xCA5A826395121157, key bumps 0x9E3779B97F4A7C15 /
// 0xBB67AE8584CAA73B.
__device__ __forceinline__ void philox4x64_10(uint64_t (&c)[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B97F4A7C15ull;
            k1 += 0xBB67AE8584CAA73Bull;
        }
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * c[0], hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c[0]);
        const uint64_t lo1 = 0xCA5A826395121157ull * c[2], hi1 = __umul64hi(0xCA5A826395121157ull, c[2]);
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// A[row*ld + col] = U(0,1) for e = row*rank + col, from word e%4 of
// philox((e/4, 0, 0, 0), (seed, mode)); ((w >> 41) + 0.5) / 2^23.
__global__ void init_factor_kernel(uint64_t seed, int mode, int64_t rows, int rank, int ld, float *__restrict__ A) {
    const int64_t total = rows * rank;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q * 4 < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        uint64_t c[4] = {(uint64_t)q, 0, 0, 0};
        philox4x64_10(c, seed, (uint64_t)mode);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t e = q * 4 + j;
            if (e < total) {
                const float m = (float)(uint32_t)(c[j] >> 41);
                A[(e / rank) * ld + (e % rank)] = (m + 0.5f) * (1.0f / 8388608.0f);
            }
        }
    }
}

__global__ void fill_zero_words_kernel(uint32_t *__restrict__ p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

__global__ void fill_zero_vec_kernel(uint4 *__restrict__ p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void fill_zero_bytes_kernel(unsigned char *__restrict__ p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0;
}

__global__ void to_bf16_kernel(const float *__restrict__ A, __nv_bfloat16 *__restrict__ B, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        B[i] = __float2bfloat16_rn(A[i]);
}

inline unsigned grid_cap(int64_t work, int threads = kThreads) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

int rank_pad(int rank) { return rank <= 16 ? 16 : (rank <= 32 ? 32 : 64); }

size_t prep_smem_bytes(int rank) {
    const int half = (rank + 2) / 2;
    return (3 * (size_t)rank * rank + 16 + 2 * half) * sizeof(double) + 2 * half * sizeof(int) + 64;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
sptt_status fill_zero_launch(void *p, size_t bytes, cudaStream_t st) {
    if (!bytes) return SPTT_OK;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (a % 16 == 0 && bytes % 16 == 0) {
        fill_zero_vec_kernel<<<grid_cap(bytes / 16), kThreads, 0, st>>>(static_cast<uint4 *>(p), bytes / 16);
    } else if (a % 4 == 0 && bytes % 4 == 0) {
        fill_zero_words_kernel<<<grid_cap(bytes / 4), kThreads, 0, st>>>(static_cast<uint32_t *>(p), bytes / 4);
    } else {
        fill_zero_bytes_kernel<<<grid_cap(bytes), kThreads, 0, st>>>(static_cast<unsigned char *>(p), bytes);
    }
    SPTT_CHECK_LAUNCH("fill_zero");
    return SPTT_OK;
}

sptt_status to_bf16_launch(const float *A, __nv_bfloat16 *B, int64_t n, cudaStream_t st) {
    if (n <= 0) return SPTT_OK;
    to_bf16_kernel<<<grid_cap(n), kThreads, 0, st>>>(A, B, n);
    SPTT_CHECK_LAUNCH("to_bf16_kernel");
    return SPTT_OK;
}

sptt_status dense_work_alloc(DenseWork *w, int32_t rank, int32_t ld, int64_t /*max_rows*/, cudaStream_t st) {
    w->rank = rank;
    w->ld = ld;
    w->nblocks = device_sm_count() * 4;
    const int64_t pstride = (int64_t)rank * rank + rank;
    SPTT_TRY(dev_alloc_n(&w->partials, (size_t)w->nblocks * pstride, st));
    SPTT_TRY(dev_alloc_n(&w->gram_un, (size_t)pstride, st));
    SPTT_TRY(dev_alloc_n(&w->W, (size_t)rank * rank, st));
    SPTT_TRY(dev_alloc_n(&w->lambda, (size_t)rank, st));
    SPTT_TRY(dev_alloc_n(&w->inv_lambda, (size_t)rank, st));
    SPTT_TRY(dev_alloc_n(&w->inner, 1, st));
    SPTT_TRY(dev_alloc_n(&w->branch, 2, st));
    SPTT_TRY(dev_alloc_n(&w->error, 1, st));
    SPTT_TRY(fill_zero_launch(w->branch, 2 * sizeof(int32_t), st));
    SPTT_TRY(fill_zero_launch(w->error, sizeof(int32_t), st));
    SPTT_TRY(fill_zero_launch(w->lambda, rank * sizeof(double), st));
    SPTT_TRY(fill_zero_launch(w->inner, sizeof(double), st));
    SPTT_CUDA(cudaFuncSetAttribute(normal_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)prep_smem_bytes(SPTT_MAX_RANK_ALS)));
    SPTT_CUDA(cudaFuncSetAttribute(postsolve_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(dense::SolveTile<16>)));
    SPTT_CUDA(cudaFuncSetAttribute(postsolve_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(dense::SolveTile<32>)));
    SPTT_CUDA(cudaFuncSetAttribute(postsolve_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(dense::SolveTile<64>)));
    int per_sm = 0;
    switch (rank_pad(rank)) {
        case 16:
            SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, postsolve_kernel<16>, kThreads,
                                                                    sizeof(dense::SolveTile<16>)));
            break;
        case 32:
            SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, postsolve_kernel<32>, kThreads,
                                                                    sizeof(dense::SolveTile<32>)));
            break;
        default:
            SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, postsolve_kernel<64>, kThreads,
                                                                    sizeof(dense::SolveTile<64>)));
            break;
    }
    w->solve_resident = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    return SPTT_OK;
}

void dense_work_free(DenseWork *w, cudaStream_t st) {
    void *ps[] = {w->partials, w->gram_un, w->W, w->lambda, w->inv_lambda, w->inner, w->branch, w->error};
    for (void *p : ps)
        if (p) dev_free(p, st);
    *w = DenseWork();
}

template <int RP>
static void gram_dispatch(const float *A, int64_t rows, int rank, int ld, double *partials, int nblocks,
                          int pstride, cudaStream_t st) {
    gram_kernel<RP><<<nblocks, kThreads, 0, st>>>(A, rows, rank, ld, partials, pstride);
}

sptt_status gram_launch(const float *A, int64_t rows, int32_t rank, int32_t ld, double *G, double *partials,
                        int32_t nblocks, cudaStream_t st) {
    const int pstride = rank * rank + rank;
    switch (rank_pad(rank)) {
        case 16: gram_dispatch<16>(A, rows, rank, ld, partials, nblocks, pstride, st); break;
        case 32: gram_dispatch<32>(A, rows, rank, ld, partials, nblocks, pstride, st); break;
        default: gram_dispatch<64>(A, rows, rank, ld, partials, nblocks, pstride, st); break;
    }
    SPTT_CHECK_LAUNCH("gram_kernel");
    const int ne = rank * rank;
    reduce_partials_kernel<<<(ne + 31) / 32, dim3(32, kRedLanes), 0, st>>>(partials, nblocks, pstride, ne, G);
    SPTT_CHECK_LAUNCH("reduce_partials_kernel");
    return SPTT_OK;
}

sptt_status normal_prep_launch(double *const *grams, int32_t nmodes, int32_t n, int32_t rank, DenseWork *w,
                               cudaStream_t st) {
    GramPtrs g{};
    for (int m = 0; m < nmodes; ++m) g.p[m] = grams[m];
    normal_prep_kernel<<<1, kThreads, prep_smem_bytes(rank), st>>>(g, nmodes, n, rank, w->W, w->branch);
    SPTT_CHECK_LAUNCH("normal_prep_kernel");
    return SPTT_OK;
}

// One CTA per tile of rows up to the CTAs the GPU holds at once: a mode with
// few rows leaves no CTA idle that the partial reduction would then read, and
// a large one runs in one wave, each CTA looping over its tiles.
template <int RP>
static int postsolve_dispatch(const float *M, const double *heavy, const int32_t *hidx, const int32_t *fids0,
                              float *A, int64_t rows, DenseWork *w, int pstride, cudaStream_t st) {
    const int64_t tiles = (rows + dense::SolveTile<RP>::TR - 1) / dense::SolveTile<RP>::TR;
    const int cap = w->solve_resident > 0 && w->solve_resident < w->nblocks ? w->solve_resident : w->nblocks;
    const int nb = (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
    postsolve_kernel<RP><<<nb, kThreads, sizeof(dense::SolveTile<RP>), st>>>(
        M, heavy, hidx, fids0, A, rows, w->rank, w->ld, w->W, w->partials, pstride);
    return nb;
}

sptt_status postsolve_launch(const float *M, const double *heavy, const int32_t *hidx, const int32_t *fids0,
                             float *A, int64_t rows, DenseWork *w, cudaStream_t st) {
    const int rank = w->rank;
    const int pstride = rank * rank + rank;
    int nb = 0;
    switch (rank_pad(rank)) {
        case 16: nb = postsolve_dispatch<16>(M, heavy, hidx, fids0, A, rows, w, pstride, st); break;
        case 32: nb = postsolve_dispatch<32>(M, heavy, hidx, fids0, A, rows, w, pstride, st); break;
        default: nb = postsolve_dispatch<64>(M, heavy, hidx, fids0, A, rows, w, pstride, st); break;
    }
    SPTT_CHECK_LAUNCH("postsolve_kernel");
    reduce_partials_kernel<<<(pstride + 31) / 32, dim3(32, kRedLanes), 0, st>>>(w->partials, nb, pstride,
                                                                               pstride, w->gram_un);
    SPTT_CHECK_LAUNCH("reduce_partials_kernel");
    return SPTT_OK;
}

sptt_status finalize_normalize_launch(double *G_n, float *A, __nv_bfloat16 *A_bf16, const int32_t *fids0,
                                     int64_t rows, DenseWork *w, cudaStream_t st) {
    const int64_t q = rows * w->ld / 4;
    finalize_normalize_kernel<<<q > 0 ? grid_cap(q) : 1, kThreads, 0, st>>>(
        w->gram_un, w->rank, G_n, w->lambda, w->inv_lambda, w->inner, A, A_bf16, fids0, rows, w->ld);
    SPTT_CHECK_LAUNCH("finalize_normalize_kernel");
    return SPTT_OK;
}

sptt_status fit_launch(double *const *grams, int32_t nmodes, const double *normx2, DenseWork *w, double *ring,
                       int32_t ring_len, int64_t *counter, cudaStream_t st) {
    GramPtrs g{};
    for (int m = 0; m < nmodes; ++m) g.p[m] = grams[m];
    fit_kernel<<<1, kThreads, 0, st>>>(g, nmodes, w->rank, normx2, w->lambda, w->inner, ring, ring_len, counter);
    SPTT_CHECK_LAUNCH("fit_kernel");
    return SPTT_OK;
}

sptt_status sumsq_launch(const float *vals, int64_t n, double *out, cudaStream_t st) {
    const int nb = 1024;
    DevBuf part;
    SPTT_TRY(part.alloc<double>(nb, st));
    sumsq_partial_kernel<<<nb, kThreads, 0, st>>>(vals, n, part.as<double>());
    SPTT_CHECK_LAUNCH("sumsq_partial_kernel");
    sum_kernel<<<1, kThreads, 0, st>>>(part.as<double>(), nb, out);
    SPTT_CHECK_LAUNCH("sum_kernel");
    return SPTT_OK;
}

sptt_status init_factor_launch(uint64_t seed, int32_t mode, int64_t rows, int32_t rank, int32_t ld, float *A,
                               cudaStream_t st) {
    SPTT_TRY(fill_zero_launch(A, (size_t)rows * ld * sizeof(float), st));
    const int64_t q = (rows * rank + 3) / 4;
    if (q == 0) return SPTT_OK;
    init_factor_kernel<<<grid_cap(q), kThreads, 0, st>>>(seed, mode, rows, rank, ld, A);
    SPTT_CHECK_LAUNCH("init_factor_kernel");
    return SPTT_OK;
}

}  // namespace sptt

using namespace sptt;

extern "C" sptt_status sptt_gram(const float *A, int64_t rows, int32_t rank, int32_t ld, double *G,
                                 sptt_stream stream) {
    clear_error();
    if (!G || (!A && rows > 0)) return set_error(SPTT_ERR_BAD_ARG, "A (when rows > 0) and G must be non-NULL");
    if (rows < 0) return set_error(SPTT_ERR_BAD_ARG, "rows < 0");
    if (rank < 1 || rank > SPTT_MAX_RANK_ALS) return set_error(SPTT_ERR_UNSUPPORTED, "rank must be in [1, 64]");
    if (ld < rank) return set_error(SPTT_ERR_BAD_ARG, "ld < rank");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nblocks = device_sm_count() * 2;
    DevBuf part;
    SPTT_TRY(part.alloc<double>((size_t)nblocks * (rank * rank + rank), st));
    return gram_launch(A, rows, rank, ld, G, part.as<double>(), nblocks, st);
}
