// Schedule selection for the MTTKRP: the candidate schedules, the exhaustive
// autotuner that times them, the tensor statistics the learned scheduler
// reads, and the scheduler itself (a small MLP with its own FP32 training and
// inference kernels). None of this is in the paper, whose C code decides only
// between locks and privatisation by a fixed rule; here the choice covers the
// CSF level order, the walk variant and the chunk size, and is learned from
// timings the autotuner measures.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace sptt {
namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Candidate schedules: CSF level order (0: ascending lengths below the root;
// 2: the shortest mode at the leaves) x walk variant (12 / 13: select walk
// with 32-byte segments in batches of 2 / 16-byte segments in batches of 4;
// 14 / 15: select walk with the leaf factor in shared memory, 1024 threads
// in batches of 2 / 512 threads in batches of 4, 13 where the factor does
// not fit) x chunk (the default for the tensor's size, and twice it). The
// library's default schedule is always one of them.
// ---------------------------------------------------------------------------
constexpr int kNumCands = 16;
const int kCandOrders[2] = {0, 2};
const int kCandVariants[4] = {12, 13, 14, 15};

sptt_sched candidate(int i, int64_t nnz) {
    sptt_sched s{};
    s.order = kCandOrders[i / 8];
    s.variant = kCandVariants[(i / 2) % 4];
    const int32_t c0 = default_chunk(nnz);
    s.chunk = (i % 2) ? (c0 * 2 <= 4096 ? c0 * 2 : 4096) : c0;
    s.block = 256;
    return s;
}

// ---------------------------------------------------------------------------
// Features: log2 histogram of slice sizes (leaves per slice)
// ---------------------------------------------------------------------------
struct FptrSet {
    const int32_t *p[kMaxModes];
};

__global__ void slice_hist_kernel(FptrSet fp, int nlev, int64_t nslices, unsigned long long *__restrict__ cnt,
                                  unsigned long long *__restrict__ sum, unsigned long long *__restrict__ mx) {
    __shared__ unsigned long long s_cnt[32], s_sum[32];
    __shared__ unsigned long long s_max;
    if (threadIdx.x < 32) {
        s_cnt[threadIdx.x] = 0;
        s_sum[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nslices;
         f += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = f, e = f + 1;
        for (int l = 0; l < nlev - 1; ++l) {
            b = fp.p[l][b];
            e = fp.p[l][e];
        }
        const unsigned long long size = (unsigned long long)(e - b);
        const int bin = 63 - __clzll((long long)size);  // floor(log2(size)), size >= 1
        atomicAdd(&s_cnt[bin < 31 ? bin : 31], 1ull);
        atomicAdd(&s_sum[bin < 31 ? bin : 31], size);
        atomicMax(&s_max, size);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        atomicAdd(cnt + threadIdx.x, s_cnt[threadIdx.x]);
        atomicAdd(sum + threadIdx.x, s_sum[threadIdx.x]);
    }
    if (threadIdx.x == 0) atomicMax(mx, s_max);
}

inline float lg(double x) { return (float)log2(x > 1.0 ? x : 1.0); }

// ---------------------------------------------------------------------------
// MLP kernels (FP32): in -> h (ReLU) -> h (ReLU) -> out, parameters packed as
// W1[h][in], b1[h], W2[h][h], b2[h], W3[out][h], b3[out]. Inputs are
// standardised with the model's feature mean and scale.
// ---------------------------------------------------------------------------
constexpr int kNin = 16, kNh = 64, kNout = kNumCands;
constexpr int kNparams = kNh * kNin + kNh + kNh * kNh + kNh + kNout * kNh + kNout;
constexpr int kTile = 32;  // samples per CTA

struct MlpSmem {
    float P[kNparams];
    float x[kTile][kNin];
    float p1[kTile][kNh], p2[kTile][kNh];  // pre-activations
    float y[kTile][kNout];
    float d2[kTile][kNh], d1[kTile][kNh];
};

__device__ void mlp_tile_forward(MlpSmem &s, const float *__restrict__ X, const float *__restrict__ mu,
                                 const float *__restrict__ sd, int64_t s0, int ns) {
    const int t = threadIdx.x;  // 64 threads: one hidden unit each
    const float *W1 = s.P, *b1 = W1 + kNh * kNin, *W2 = b1 + kNh, *b2 = W2 + kNh * kNh, *W3 = b2 + kNh,
                *b3 = W3 + kNout * kNh;
    for (int e = t; e < kTile * kNin; e += blockDim.x) {
        const int r = e / kNin, c = e % kNin;
        s.x[r][c] = (r < ns) ? (X[(s0 + r) * kNin + c] - mu[c]) / sd[c] : 0.f;
    }
    __syncthreads();
    for (int r = 0; r < ns; ++r) {
        float a = b1[t];
        for (int i = 0; i < kNin; ++i) a = fmaf(W1[t * kNin + i], s.x[r][i], a);
        s.p1[r][t] = a;
    }
    __syncthreads();
    for (int r = 0; r < ns; ++r) {
        float a = b2[t];
        for (int i = 0; i < kNh; ++i) a = fmaf(W2[t * kNh + i], fmaxf(s.p1[r][i], 0.f), a);
        s.p2[r][t] = a;
    }
    __syncthreads();
    if (t < kNout)
        for (int r = 0; r < ns; ++r) {
            float a = b3[t];
            for (int i = 0; i < kNh; ++i) a = fmaf(W3[t * kNh + i], fmaxf(s.p2[r][i], 0.f), a);
            s.y[r][t] = a;
        }
    __syncthreads();
}

__global__ void __launch_bounds__(kNh) mlp_forward_kernel(const float *__restrict__ P, const float *__restrict__ mu,
                                                          const float *__restrict__ sd, const float *__restrict__ X,
                                                          int64_t n, float *__restrict__ Y) {
    extern __shared__ __align__(16) unsigned char raw[];
    MlpSmem &s = *reinterpret_cast<MlpSmem *>(raw);
    for (int e = threadIdx.x; e < kNparams; e += blockDim.x) s.P[e] = P[e];
    __syncthreads();
    for (int64_t s0 = (int64_t)blockIdx.x * kTile; s0 < n; s0 += (int64_t)gridDim.x * kTile) {
        const int ns = (int)((n - s0) < kTile ? (n - s0) : kTile);
        mlp_tile_forward(s, X, mu, sd, s0, ns);
        for (int e = threadIdx.x; e < ns * kNout; e += blockDim.x) Y[(s0 + e / kNout) * kNout + e % kNout] = s.y[e / kNout][e % kNout];
        __syncthreads();
    }
}

// Loss 1/(n*out) sum (y - t)^2 and its gradient, accumulated into G and
// *loss with atomics (one CTA per tile of samples).
__global__ void __launch_bounds__(kNh) mlp_grad_kernel(const float *__restrict__ P, const float *__restrict__ mu,
                                                       const float *__restrict__ sd, const float *__restrict__ X,
                                                       const float *__restrict__ T, int64_t n,
                                                       float *__restrict__ G, float *__restrict__ loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    MlpSmem &s = *reinterpret_cast<MlpSmem *>(raw);
    const int t = threadIdx.x;
    for (int e = t; e < kNparams; e += blockDim.x) s.P[e] = P[e];
    __syncthreads();
    const float *W2 = s.P + kNh * kNin + kNh, *W3 = W2 + kNh * kNh + kNh;
    float *gW1 = G, *gb1 = gW1 + kNh * kNin, *gW2 = gb1 + kNh, *gb2 = gW2 + kNh * kNh, *gW3 = gb2 + kNh,
          *gb3 = gW3 + kNout * kNh;
    const float scale = 1.0f / ((float)n * kNout);
    for (int64_t s0 = (int64_t)blockIdx.x * kTile; s0 < n; s0 += (int64_t)gridDim.x * kTile) {
        const int ns = (int)((n - s0) < kTile ? (n - s0) : kTile);
        mlp_tile_forward(s, X, mu, sd, s0, ns);
        // dy (kept in y), loss
        float lpart = 0.f;
        for (int e = t; e < ns * kNout; e += blockDim.x) {
            const int r = e / kNout, o = e % kNout;
            const float err = s.y[r][o] - T[(s0 + r) * kNout + o];
            lpart += err * err * scale;
            s.y[r][o] = 2.f * err * scale;
        }
        atomicAdd(loss, lpart);
        __syncthreads();
        // layer 3 grads (thread t = hidden unit j) and d2
        {
            const int j = t;
            float gw[kNout];
#pragma unroll
            for (int o = 0; o < kNout; ++o) gw[o] = 0.f;
            for (int r = 0; r < ns; ++r) {
                const float h2 = fmaxf(s.p2[r][j], 0.f);
                float back = 0.f;
#pragma unroll
                for (int o = 0; o < kNout; ++o) {
                    gw[o] = fmaf(s.y[r][o], h2, gw[o]);
                    back = fmaf(s.y[r][o], W3[o * kNh + j], back);
                }
                s.d2[r][j] = s.p2[r][j] > 0.f ? back : 0.f;
            }
#pragma unroll
            for (int o = 0; o < kNout; ++o) atomicAdd(gW3 + o * kNh + j, gw[o]);
            if (j < kNout) {
                float gb = 0.f;
                for (int r = 0; r < ns; ++r) gb += s.y[r][j];
                atomicAdd(gb3 + j, gb);
            }
        }
        __syncthreads();
        // layer 2 grads (row j = t) and d1
        {
            const int j = t;
            float gb = 0.f;
            for (int r = 0; r < ns; ++r) gb += s.d2[r][j];
            atomicAdd(gb2 + j, gb);
            for (int i = 0; i < kNh; ++i) {
                float g = 0.f;
                for (int r = 0; r < ns; ++r) g = fmaf(s.d2[r][j], fmaxf(s.p1[r][i], 0.f), g);
                atomicAdd(gW2 + j * kNh + i, g);
            }
            const int i = t;  // d1 for hidden unit i
            for (int r = 0; r < ns; ++r) {
                float back = 0.f;
                for (int jj = 0; jj < kNh; ++jj) back = fmaf(s.d2[r][jj], W2[jj * kNh + i], back);
                s.d1[r][i] = s.p1[r][i] > 0.f ? back : 0.f;
            }
        }
        __syncthreads();
        // layer 1 grads (row i = t)
        {
            const int i = t;
            float gb = 0.f;
            for (int r = 0; r < ns; ++r) gb += s.d1[r][i];
            atomicAdd(gb1 + i, gb);
            for (int k = 0; k < kNin; ++k) {
                float g = 0.f;
                for (int r = 0; r < ns; ++r) g = fmaf(s.d1[r][i], s.x[r][k], g);
                atomicAdd(gW1 + i * kNin + k, g);
            }
        }
        __syncthreads();
    }
}

// Adam (Kingma & Ba 2015) step on every parameter; t is the 1-based step.
__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ m,
                            float *__restrict__ v, int np, float lr, float b1, float b2, float eps, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    P[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Feature mean and scale over the training set (one CTA per feature).
__global__ void feature_stats_kernel(const float *__restrict__ X, int64_t n, float *__restrict__ mu,
                                     float *__restrict__ sd) {
    __shared__ double s1[kThreads], s2[kThreads];
    const int c = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double x = X[r * kNin + c];
        a += x;
        b += x * x;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = s1[0] / (double)n;
        const double var = s2[0] / (double)n - m * m;
        mu[c] = (float)m;
        sd[c] = (float)(var > 1e-12 ? sqrt(var) : 1.0);
    }
}

// He-uniform initial weights from the Philox stream, biases 0.
__global__ void mlp_init_kernel(float *__restrict__ P, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNparams) return;
    int fan_in = 0;
    int off = i;
    if (off < kNh * kNin) fan_in = kNin;
    else if ((off -= kNh * kNin) < kNh) fan_in = 0;
    else if ((off -= kNh) < kNh * kNh) fan_in = kNh;
    else if ((off -= kNh * kNh) < kNh) fan_in = 0;
    else if ((off -= kNh) < kNout * kNh) fan_in = kNh;
    else fan_in = 0;
    if (fan_in == 0) {
        P[i] = 0.f;
        return;
    }
    // splitmix64 of (seed, i) -> uniform in (-1, 1)
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = ((float)(z >> 40) + 0.5f) * (1.0f / 16777216.0f) * 2.f - 1.f;
    P[i] = u * sqrtf(6.f / (float)fan_in);
}

size_t mlp_smem() { return sizeof(MlpSmem); }

}  // namespace
}  // namespace sptt

using namespace sptt;

struct sptt_mlp {
    float *P = nullptr, *G = nullptr, *m = nullptr, *v = nullptr, *mu = nullptr, *sd = nullptr;
    float *loss = nullptr;
    int step = 0;
};

namespace {

sptt_status mlp_grad_launch(sptt_mlp *mlp, const float *X, const float *T, int64_t n, cudaStream_t st) {
    SPTT_TRY(fill_zero_launch(mlp->G, kNparams * sizeof(float), st));
    SPTT_TRY(fill_zero_launch(mlp->loss, sizeof(float), st));
    int64_t grid = (n + kTile - 1) / kTile;
    const int64_t cap = (int64_t)device_sm_count() * 2;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    mlp_grad_kernel<<<(unsigned)grid, kNh, mlp_smem(), st>>>(mlp->P, mlp->mu, mlp->sd, X, T, n, mlp->G, mlp->loss);
    SPTT_CHECK_LAUNCH("mlp_grad_kernel");
    return SPTT_OK;
}

}  // namespace

extern "C" int32_t sptt_sched_candidates(int64_t nnz, sptt_sched *out, int32_t cap) {
    for (int i = 0; i < kNumCands && i < cap; ++i)
        if (out) out[i] = candidate(i, nnz);
    return kNumCands;
}

extern "C" sptt_status sptt_level_order(const int64_t *dims, int32_t nmodes, int32_t root, int32_t kind,
                                        int32_t *order_out) {
    clear_error();
    if (!dims || !order_out) return set_error(SPTT_ERR_BAD_ARG, "dims and order_out must be non-NULL");
    if (nmodes < 2 || nmodes > kMaxModes || root < 0 || root >= nmodes || kind < 0 || kind > 2)
        return set_error(SPTT_ERR_BAD_ARG, "nmodes, root or kind out of range");
    level_order(dims, nmodes, root, kind, order_out);
    return SPTT_OK;
}

extern "C" sptt_status sptt_sched_default(const int64_t *dims, int32_t nmodes, int32_t root, int32_t rank,
                                          int32_t factor_dtype, int64_t nnz, sptt_sched *out) {
    clear_error();
    if (!dims || !out) return set_error(SPTT_ERR_BAD_ARG, "dims and out must be non-NULL");
    if (nmodes < 2 || nmodes > kMaxModes || root < 0 || root >= nmodes)
        return set_error(SPTT_ERR_BAD_ARG, "nmodes or root out of range");
    if (rank < 1) return set_error(SPTT_ERR_BAD_ARG, "rank must be >= 1");
    if (factor_dtype != SPTT_F32 && factor_dtype != SPTT_BF16)
        return set_error(SPTT_ERR_BAD_ARG, "factor_dtype must be SPTT_F32 or SPTT_BF16");
    const int32_t ld = (rank + 7) / 8 * 8;
    sptt_sched s{};
    s.order = default_order_kind(dims, nmodes, root, ld, factor_dtype, nnz);
    int32_t order[kMaxModes];
    level_order(dims, nmodes, root, s.order, order);
    s.variant = default_variant(factor_dtype, ld, dims[order[nmodes - 1]], nnz, nmodes);
    s.chunk = default_chunk(nnz);
    s.block = 256;
    *out = s;
    return SPTT_OK;
}

extern "C" sptt_status sptt_csf_features(const sptt_csf *csf, int32_t rank, int32_t factor_dtype, float *feat,
                                         sptt_stream stream) {
    clear_error();
    if (!csf || !feat) return set_error(SPTT_ERR_BAD_ARG, "csf and feat must be non-NULL");
    if (rank < 1) return set_error(SPTT_ERR_BAD_ARG, "rank must be >= 1");
    if (factor_dtype != SPTT_F32 && factor_dtype != SPTT_BF16)
        return set_error(SPTT_ERR_BAD_ARG, "factor_dtype must be SPTT_F32 or SPTT_BF16");
    const double rowbytes = (double)((rank + 7) / 8 * 8) * (factor_dtype == SPTT_BF16 ? 2.0 : 4.0);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int N = csf->nmodes;
    const int64_t ns = csf->nfibs[0], nnz = csf->nfibs[N - 1];
    DevBuf buf;
    SPTT_TRY(buf.alloc<unsigned long long>(65, st));
    SPTT_TRY(fill_zero_launch(buf.p, 65 * sizeof(unsigned long long), st));
    unsigned long long *cnt = buf.as<unsigned long long>(), *sum = cnt + 32, *mx = cnt + 64;
    if (ns > 0) {
        FptrSet fp{};
        for (int l = 0; l < N - 1; ++l) fp.p[l] = csf->fptr[l];
        int64_t grid = (ns + kThreads - 1) / kThreads;
        if (grid > device_sm_count() * 4) grid = device_sm_count() * 4;
        slice_hist_kernel<<<(unsigned)grid, kThreads, 0, st>>>(fp, N, ns, cnt, sum, mx);
        SPTT_CHECK_LAUNCH("slice_hist_kernel");
    }
    unsigned long long h[65];
    SPTT_CUDA(cudaMemcpyAsync(h, buf.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    const double dn = (double)(nnz > 0 ? nnz : 1), dns = (double)(ns > 0 ? ns : 1);
    const int64_t leafpar = N >= 2 ? csf->nfibs[N - 2] : 1;
    double heavy = 0.0, single = 0.0, ent = 0.0;
    for (int b = 0; b < 32; ++b) {
        if (b >= 10) heavy += (double)h[32 + b];
        if (b == 0) single += (double)h[b];
        const double p = (double)h[b] / dns;
        if (p > 0) ent -= p * log2(p);
    }
    const int64_t d_root = csf->dims[csf->order[0]];
    const int64_t d_l1 = N > 2 ? csf->dims[csf->order[1]] : 1;
    const int64_t d_leaf = csf->dims[csf->order[N - 1]];
    float f[16];
    f[0] = lg(dn);
    f[1] = (float)N;
    f[2] = lg(rowbytes);
    f[3] = lg((double)d_root);
    f[4] = lg((double)d_l1);
    f[5] = lg((double)d_leaf);
    f[6] = lg(dns);
    f[7] = lg((double)leafpar);
    f[8] = lg(dn / (double)(leafpar > 0 ? leafpar : 1));
    f[9] = lg(dn / dns);
    f[10] = lg((double)h[64]);
    f[11] = (float)(heavy / dn);
    f[12] = (float)(single / dns);
    f[13] = lg((double)d_leaf * rowbytes);
    f[14] = lg((double)d_l1 * rowbytes);
    f[15] = (float)(ent / 5.0);
    memcpy(feat, f, sizeof(f));
    return SPTT_OK;
}

extern "C" sptt_status sptt_autotune(const sptt_coo *coo, int32_t root, int32_t rank, int32_t dtype, int32_t reps,
                                     float *ms, sptt_stream stream) {
    clear_error();
    if (!ms) return set_error(SPTT_ERR_BAD_ARG, "ms is NULL");
    SPTT_TRY(coo_validate_shape(coo));
    if (root < 0 || root >= coo->nmodes) return set_error(SPTT_ERR_BAD_ARG, "root out of range");
    if (dtype != SPTT_F32 && dtype != SPTT_BF16) return set_error(SPTT_ERR_BAD_ARG, "dtype");
    const int vec = dtype == SPTT_BF16 ? 8 : 4;
    if (rank < 1 || rank > 32 * vec) return set_error(SPTT_ERR_UNSUPPORTED, "rank");
    if (reps < 1) reps = 3;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int N = coo->nmodes;
    const int ld = (rank + 7) / 8 * 8;
    DevCoo dc;
    SPTT_TRY(coo_to_device(coo, st, &dc));
    // random factors (values do not change the timing)
    std::vector<DevBuf> fac(N), facb(N);
    const void *fptrs[kMaxModes] = {nullptr};
    for (int m = 0; m < N; ++m) {
        if (m == root) continue;
        SPTT_TRY(fac[m].alloc<float>((size_t)coo->dims[m] * ld, st));
        SPTT_TRY(init_factor_launch(1234 + m, m, coo->dims[m], ld, ld, fac[m].as<float>(), st));
        if (dtype == SPTT_BF16) {
            SPTT_TRY(facb[m].alloc<__nv_bfloat16>((size_t)coo->dims[m] * ld, st));
            SPTT_TRY(to_bf16_launch(fac[m].as<float>(), facb[m].as<__nv_bfloat16>(), coo->dims[m] * ld, st));
            fptrs[m] = facb[m].p;
        } else {
            fptrs[m] = fac[m].p;
        }
    }
    cudaEvent_t e0, e1;
    SPTT_CUDA(cudaEventCreate(&e0));
    SPTT_CUDA(cudaEventCreate(&e1));
    sptt_status status = SPTT_OK;
    for (int oi = 0; oi < 2 && status == SPTT_OK; ++oi) {
        const int ord = kCandOrders[oi];
        int32_t order[kMaxModes];
        level_order(coo->dims, N, root, ord, order);
        sptt_csf *csf = nullptr;
        status = csf_build_device(&dc.coo, root, order, st, &csf);
        if (status != SPTT_OK) break;
        DevBuf out, heavy;
        for (int i = 0; i < kNumCands && status == SPTT_OK; ++i) {
            const sptt_sched s = candidate(i, coo->nnz);
            if (s.order != ord) continue;
            status = mttkrp_prepare(csf, &s, st);
            if (status != SPTT_OK) break;
            out.reset();
            heavy.reset();
            if ((status = out.alloc<float>((size_t)csf->nfibs[0] * ld, st)) != SPTT_OK) break;
            if ((status = heavy.alloc<double>((size_t)csf->nheavy * ld, st)) != SPTT_OK) break;
            status = mttkrp_launch(csf, fptrs, dtype, ld, out.as<float>(), heavy.as<double>(), &s, st);  // warm-up
            std::vector<float> t(reps);
            for (int r = 0; r < reps && status == SPTT_OK; ++r) {
                cudaEventRecord(e0, st);
                status = mttkrp_launch(csf, fptrs, dtype, ld, out.as<float>(), heavy.as<double>(), &s, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) status = cuda_error(cudaGetLastError(), "autotune");
                else cudaEventElapsedTime(&t[r], e0, e1);
            }
            if (status == SPTT_OK) {
                std::sort(t.begin(), t.end());
                ms[i] = t[reps / 2];
            }
        }
        csf_destroy(csf);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}

extern "C" void sptt_mlp_free(sptt_mlp *m);

extern "C" sptt_status sptt_mlp_create(uint64_t seed, sptt_mlp **out) {
    clear_error();
    if (!out) return set_error(SPTT_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    sptt_mlp *m = new sptt_mlp();
    struct Guard {
        sptt_mlp *m;
        ~Guard() { if (m) sptt_mlp_free(m); }
    } guard{m};
    cudaStream_t st = nullptr;
    float **bufs[] = {&m->P, &m->G, &m->m, &m->v};
    for (float **b : bufs) SPTT_CUDA(cudaMalloc(b, kNparams * sizeof(float)));
    SPTT_CUDA(cudaMalloc(&m->mu, kNin * sizeof(float)));
    SPTT_CUDA(cudaMalloc(&m->sd, kNin * sizeof(float)));
    SPTT_CUDA(cudaMalloc(&m->loss, sizeof(float)));
    std::vector<float> ones(kNin, 1.f);
    SPTT_TRY(fill_zero_launch(m->mu, kNin * sizeof(float), st));
    SPTT_CUDA(cudaMemcpy(m->sd, ones.data(), kNin * sizeof(float), cudaMemcpyHostToDevice));
    SPTT_TRY(fill_zero_launch(m->m, kNparams * sizeof(float), st));
    SPTT_TRY(fill_zero_launch(m->v, kNparams * sizeof(float), st));
    mlp_init_kernel<<<(kNparams + 255) / 256, 256, 0, st>>>(m->P, seed);
    SPTT_CHECK_LAUNCH("mlp_init_kernel");
    SPTT_CUDA(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem()));
    SPTT_CUDA(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem()));
    SPTT_CUDA(cudaDeviceSynchronize());
    guard.m = nullptr;
    *out = m;
    return SPTT_OK;
}

extern "C" void sptt_mlp_free(sptt_mlp *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    float *b[] = {m->P, m->G, m->m, m->v, m->mu, m->sd, m->loss};
    for (float *p : b)
        if (p) cudaFree(p);
    delete m;
}

extern "C" int32_t sptt_mlp_nparams(void) { return kNparams; }

extern "C" sptt_status sptt_mlp_get(const sptt_mlp *m, float *params, float *mu, float *sd) {
    clear_error();
    if (!m) return set_error(SPTT_ERR_BAD_ARG, "mlp is NULL");
    if (params) SPTT_CUDA(cudaMemcpy(params, m->P, kNparams * sizeof(float), cudaMemcpyDefault));
    if (mu) SPTT_CUDA(cudaMemcpy(mu, m->mu, kNin * sizeof(float), cudaMemcpyDefault));
    if (sd) SPTT_CUDA(cudaMemcpy(sd, m->sd, kNin * sizeof(float), cudaMemcpyDefault));
    return SPTT_OK;
}

extern "C" sptt_status sptt_mlp_set(sptt_mlp *m, const float *params, const float *mu, const float *sd) {
    clear_error();
    if (!m) return set_error(SPTT_ERR_BAD_ARG, "mlp is NULL");
    if (params) SPTT_CUDA(cudaMemcpy(m->P, params, kNparams * sizeof(float), cudaMemcpyDefault));
    if (mu) SPTT_CUDA(cudaMemcpy(m->mu, mu, kNin * sizeof(float), cudaMemcpyDefault));
    if (sd) SPTT_CUDA(cudaMemcpy(m->sd, sd, kNin * sizeof(float), cudaMemcpyDefault));
    return SPTT_OK;
}

extern "C" sptt_status sptt_mlp_forward(const sptt_mlp *m, const float *X, int64_t n, float *Y, sptt_stream stream) {
    clear_error();
    if (!m || !X || !Y) return set_error(SPTT_ERR_BAD_ARG, "mlp, X and Y must be non-NULL");
    if (n <= 0) return SPTT_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int64_t grid = (n + kTile - 1) / kTile;
    if (grid > device_sm_count() * 2) grid = device_sm_count() * 2;
    mlp_forward_kernel<<<(unsigned)grid, kNh, mlp_smem(), st>>>(m->P, m->mu, m->sd, X, n, Y);
    SPTT_CHECK_LAUNCH("mlp_forward_kernel");
    return SPTT_OK;
}

extern "C" sptt_status sptt_mlp_loss_grad(sptt_mlp *m, const float *X, const float *T, int64_t n, float *loss,
                                          float *grad, sptt_stream stream) {
    clear_error();
    if (!m || !X || !T) return set_error(SPTT_ERR_BAD_ARG, "mlp, X and T must be non-NULL");
    if (n <= 0) return set_error(SPTT_ERR_BAD_ARG, "n must be > 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SPTT_TRY(mlp_grad_launch(m, X, T, n, st));
    if (loss) SPTT_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDefault, st));
    if (grad) SPTT_CUDA(cudaMemcpyAsync(grad, m->G, kNparams * sizeof(float), cudaMemcpyDefault, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    return SPTT_OK;
}

extern "C" sptt_status sptt_mlp_train(sptt_mlp *m, const float *X, const float *T, int64_t n, int32_t steps,
                                      float lr, float *loss_history, sptt_stream stream) {
    clear_error();
    if (!m || !X || !T) return set_error(SPTT_ERR_BAD_ARG, "mlp, X and T must be non-NULL");
    if (n <= 0 || steps < 0) return set_error(SPTT_ERR_BAD_ARG, "n must be > 0, steps >= 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (m->step == 0) {  // standardise the features on the first training call
        feature_stats_kernel<<<kNin, kThreads, 0, st>>>(X, n, m->mu, m->sd);
        SPTT_CHECK_LAUNCH("feature_stats_kernel");
    }
    for (int s = 0; s < steps; ++s) {
        SPTT_TRY(mlp_grad_launch(m, X, T, n, st));
        ++m->step;
        adam_kernel<<<(kNparams + 255) / 256, 256, 0, st>>>(m->P, m->G, m->m, m->v, kNparams, lr, 0.9f, 0.999f,
                                                            1e-8f, m->step);
        SPTT_CHECK_LAUNCH("adam_kernel");
        if (loss_history) SPTT_CUDA(cudaMemcpyAsync(loss_history + s, m->loss, sizeof(float), cudaMemcpyDefault, st));
    }
    SPTT_CUDA(cudaStreamSynchronize(st));
    return SPTT_OK;
}

extern "C" sptt_status sptt_mlp_predict(const sptt_mlp *m, const float *feat, int64_t n, int32_t *choice, float *pred,
                                        sptt_stream stream) {
    clear_error();
    if (!m || !feat || n <= 0) return set_error(SPTT_ERR_BAD_ARG, "mlp and feat must be non-NULL, n > 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf dx, dy;
    SPTT_TRY(dx.alloc<float>((size_t)n * kNin, st));
    SPTT_TRY(dy.alloc<float>((size_t)n * kNout, st));
    SPTT_CUDA(cudaMemcpyAsync(dx.p, feat, (size_t)n * kNin * sizeof(float), cudaMemcpyDefault, st));
    SPTT_TRY(sptt_mlp_forward(m, dx.as<float>(), n, dy.as<float>(), stream));
    std::vector<float> y((size_t)n * kNout);
    SPTT_CUDA(cudaMemcpyAsync(y.data(), dy.p, y.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    SPTT_CUDA(cudaStreamSynchronize(st));
    for (int64_t r = 0; r < n; ++r) {
        int best = 0;
        for (int k = 1; k < kNout; ++k)
            if (y[r * kNout + k] < y[r * kNout + best]) best = k;
        if (choice) choice[r] = best;
    }
    if (pred) memcpy(pred, y.data(), y.size() * sizeof(float));
    return SPTT_OK;
}
