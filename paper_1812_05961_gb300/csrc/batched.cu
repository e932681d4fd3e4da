// Batched CP-ALS: many independent small tensors decomposed by one
// persistent kernel (Algorithm 1 for each tensor), so a batch of hundreds of
// uneven tensors costs one launch instead of tens of thousands.
//
// The kernel is launched cooperatively (every CTA resident) and walks the
// same schedule for all tensors. For each iteration and each mode position
// n, five phases separated by grid barriers:
//   M  MTTKRP of mode n for every tensor that has it: the lane groups share
//      one global list of work chunks (all tensors' chunks back to back), so
//      large and small tensors are balanced together (walk.cuh);
//   P  per tensor (one CTA each): V = Hadamard of the other Grams, W = V^+
//      (FP64 Cholesky / pseudo-inverse, dense_dev.cuh);
//   S  row solve A_un = M W over one global list of 4096/R-row tiles, with the
//      Gram of A_un and the fit's dots accumulated in FP64 (each CTA takes a
//      contiguous run of tiles and flushes once per tensor it touches);
//      M is cleared as it is read, ready for the next mode;
//   F  per tensor: lambda, G_n, and (after the tensor's last mode) the fit;
//   N  A_n *= 1/lambda over the tile list.
//
// The grid barrier waits are bounded: a CTA that waits longer than the
// configured limit (globaltimer) sets the error word and the kernel returns;
// every other CTA sees the word at its next wait and returns as well, so a
// missing arrival ends in SPTT_ERR_TIMEOUT, never in a hung GPU.
#include <vector>

#include "dense_dev.cuh"
#include "walk.cuh"

namespace sptt {
namespace {

constexpr int kBThreads = 256;
constexpr int kFitRing = 4096;

struct BTensor {
    int32_t nmodes;
    int32_t pad_;
    int64_t dims[kMaxModes];
    walk::Args w[kMaxModes];  // per root mode (out = M)
    const int32_t *fids0[kMaxModes];
    int64_t nslices[kMaxModes];
    float *A[kMaxModes];
    double *G[kMaxModes];
    float *M;           // compact MTTKRP output, max slices x ld, kept zero between uses
    double *Mh;         // FP64 rows of heavy slices, max heavy x ld, kept zero between uses
    const int32_t *hidx[kMaxModes];
    double *gun;        // rank*rank + rank FP64 accumulators, kept zero between uses
    float *W;           // rank*rank
    double *lambda;     // rank
    float *inv_lambda;  // rank
    double *inner;      // 1
    double *normx2;     // 1
    double *fits;       // kFitRing
    int32_t *branch;    // [0] pseudo-inverse updates, [1] all updates
};

struct BatchArgs {
    const BTensor *T;
    int32_t count, rank, ld, iters, max_modes;
    const int64_t *chunk_prefix[kMaxModes];  // [count + 1] per mode position
    const int32_t *chunk_owner[kMaxModes];   // [total_chunks] tensor of each global chunk
    const int64_t *tile_prefix[kMaxModes];   // [count + 1]
    int64_t total_chunks[kMaxModes];
    int64_t total_tiles[kMaxModes];
    unsigned *bar;       // [0] arrivals, [1] generation
    int32_t *err;        // error word (1 = a barrier wait timed out)
    int64_t *it_base;    // iterations run before this launch (indexes the fit ring)
    uint64_t timeout_ns;
    int32_t skip_block;  // test hook: this CTA leaves before the first barrier (-1: none)
    unsigned long long *phase_ns;  // [10] wall time CTA 0 spends in each phase (M, P, S, F, N; the barrier
                                   // that ends it included) and, in [5 + phase], its wait in that barrier
    int32_t zero_first;  // clear A_n before its first update (rows without a slice end at 0)
    int32_t walk;        // MTTKRP walk (batch_walk): 0 leaf arrays, 1 packed records, 2 packed, 32-byte rows
};

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier with a bounded wait. Returns false (on every thread of the
// CTA) when the error word is set, by this CTA or another.
__device__ bool grid_barrier(const BatchArgs &a, int ph) {
    __shared__ int s_ok;
    __syncthreads();
    const uint64_t tb = (blockIdx.x == 0 && threadIdx.x == 0) ? globaltimer() : 0;
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = a.bar + 1;
        volatile int32_t *verr = a.err;
        int ok = 1;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            a.bar[0] = 0u;  // reset before release: nobody re-arrives until gen moves
            __threadfence();
            atomicAdd(a.bar + 1, 1u);
        } else {
            const uint64_t t0 = globaltimer();
            while (*vgen == g) {
                if (*verr) { ok = 0; break; }
                if (globaltimer() - t0 > a.timeout_ns) {
                    atomicOr(a.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = ok && (*verr == 0);
        if (blockIdx.x == 0) a.phase_ns[5 + ph] += globaltimer() - tb;
    }
    __syncthreads();
    return s_ok != 0;
}

// index t with prefix[t] <= x < prefix[t + 1]
__device__ __forceinline__ int find_owner(const int64_t *prefix, int count, int64_t x) {
    int lo = 0, hi = count;  // prefix[lo] <= x < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Rows per tile of the S and N phases: 4096 / RP (256 at RP = 16, 128 at
// RP = 32), so one tile is 16 KB of M whatever the rank.
__host__ __device__ constexpr int tile_rows(int rp) { return 4096 / rp; }

// The contiguous run [g0, g1) of a global work list that this CTA takes.
struct Span {
    int64_t g0, g1;
};

__device__ __forceinline__ Span cta_span(int64_t total) {
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    Span s;
    s.g0 = (int64_t)blockIdx.x * per;
    s.g1 = (s.g0 + per < total) ? s.g0 + per : total;
    return s;
}

// Owner of item g, advanced from a previous owner at or before g.
__device__ __forceinline__ int advance_owner(const int64_t *prefix, int tt, int64_t g) {
    while (g >= __ldg(prefix + tt + 1)) ++tt;
    return tt;
}

// M: MTTKRP of mode n over the global chunk list. The lane groups of the
// whole grid interleave over it, so every tensor's chunks (whose costs differ
// from tensor to tensor) are spread over all CTAs; a group's chunks are far
// apart, so its heavy-slice partial is flushed after each chunk.
template <int NM>
__device__ __noinline__ void walk_chunk(const walk::Args &w, int64_t c, int col) {
    const walk::GlobalRecs rec{w.vals, w.fids[NM - 1], w.lvl};
    walk::Carry<4> cy;
    walk::flag_chunk<NM, float, 4, walk::GlobalRecs, 16, false>(w, c, col, cy, rec);
    walk::flush_carry(w, col, cy);
}

// The select walk on the packed leaf records (walk.cuh select_chunk: no
// per-leaf branch, two leaves per pair of 16-byte record loads past L1),
// 16-byte row segments in batches of 2: it fits the 2-CTA-per-SM build
// without spilling (the flag walk it replaced spilled 160-176 bytes per call).
template <int NM>
__device__ __noinline__ void walk_chunk_packed(const walk::Args &w, int64_t c, int col) {
    using Recs = walk::PackedRecsT<true>;
    const Recs rec{w.leafrec};
    walk::Carry<4> cy;
    walk::select_chunk<NM, float, 2, 16, false, true>(w, c, col, cy, rec);
    walk::flush_carry(w, col, cy);
}

// The select walk with 32-byte row segments (2 lanes per R = 16 row), its
// row and record loads split in 16-byte halves (walk.cuh SPLIT: ptxas 13.0
// fails on the 32-byte form inside this non-inlined function). It needs
// more registers than a CTA of the 2-per-SM build has, so it runs in the
// 1-CTA-per-SM build (batch_walk).
template <int NM>
__device__ __noinline__ void walk_chunk_wide(const walk::Args &w, int64_t c, int col) {
    using Recs = walk::PackedRecsT<true>;
    const Recs rec{w.leafrec};
    walk::Carry<8> cy;
    walk::select_chunk<NM, float, 2, 32, false, true>(w, c, col, cy, rec);
    walk::flush_carry(w, col, cy);
}

__device__ __noinline__ void mttkrp_phase_wide(const BatchArgs &a, int n) {
    const walk::Lanes L = walk::lanes_for(a.ld, 8);
    if (L.idle) return;
    const int64_t gwarp = (int64_t)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t)(gridDim.x * blockDim.x) >> 5;
    const int64_t *prefix = a.chunk_prefix[n];
    for (int64_t gc = gwarp * L.gpw + L.gi; gc < a.total_chunks[n]; gc += nwarps * L.gpw) {
        const int tt = __ldg(a.chunk_owner[n] + gc);
        const BTensor &T = a.T[tt];
        const int64_t c = gc - __ldg(prefix + tt);
        switch (T.nmodes) {
            case 2: walk_chunk_wide<2>(T.w[n], c, L.col); break;
            case 3: walk_chunk_wide<3>(T.w[n], c, L.col); break;
            default: walk_chunk_wide<4>(T.w[n], c, L.col); break;
        }
    }
}

__device__ __noinline__ void mttkrp_phase(const BatchArgs &a, int n, int gi, int gpw, int col) {
    const int64_t gwarp = (int64_t)(blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t)(gridDim.x * blockDim.x) >> 5;
    const int64_t *prefix = a.chunk_prefix[n];
    for (int64_t gc = gwarp * gpw + gi; gc < a.total_chunks[n]; gc += nwarps * gpw) {
        const int tt = __ldg(a.chunk_owner[n] + gc);
        const BTensor &T = a.T[tt];
        const int64_t c = gc - __ldg(prefix + tt);
        if (a.walk == 1) {
            switch (T.nmodes) {
                case 2: walk_chunk_packed<2>(T.w[n], c, col); break;
                case 3: walk_chunk_packed<3>(T.w[n], c, col); break;
                default: walk_chunk_packed<4>(T.w[n], c, col); break;
            }
        } else {
            switch (T.nmodes) {
                case 2: walk_chunk<2>(T.w[n], c, col); break;
                case 3: walk_chunk<3>(T.w[n], c, col); break;
                default: walk_chunk<4>(T.w[n], c, col); break;
            }
        }
    }
}

// S: A_un = M W over the tile list (dense_dev.cuh's tile body, which clears
// M as it reads it); each CTA takes a contiguous run of tiles and adds its
// Gram and dot totals to a tensor's accumulators when it moves on.
template <int RP>
__device__ __noinline__ void solve_phase(const BatchArgs &a, int n, dense::SolveTile<RP> &sm) {
    static_assert(dense::SolveTile<RP>::TR == tile_rows(RP), "tile lists and tile body agree");
    const Span sp = cta_span(a.total_tiles[n]);
    if (sp.g0 >= sp.g1) return;
    const int64_t *prefix = a.tile_prefix[n];
    const int rank = a.rank;
    int tt = find_owner(prefix, a.count, sp.g0);
    int cur = -1;
    dense::SolveRun acc;
    dense::solve_begin(sm, acc);
    for (int64_t gt = sp.g0; gt < sp.g1; ++gt) {
        tt = advance_owner(prefix, tt, gt);
        const BTensor &T = a.T[tt];
        if (tt != cur) {
            if (cur >= 0) {
                double *gun = a.T[cur].gun;
                dense::solve_reduce(sm, acc, rank, [&](int e, double v) { atomicAdd(gun + e, v); });
            }
            cur = tt;
            dense::solve_load_w(sm, T.W, rank);  // the last tile (or reduction) ended with a barrier
        }
        const int64_t i0 = (gt - __ldg(prefix + tt)) * tile_rows(RP);
        dense::solve_tile<RP, true>(sm, acc, T.M, T.Mh, T.hidx[n], T.fids0[n], T.A[n], i0, T.nslices[n], rank,
                                    a.ld);
    }
    double *gun = a.T[cur].gun;
    dense::solve_reduce(sm, acc, rank, [&](int e, double v) { atomicAdd(gun + e, v); });
}

// N: A_n *= 1 / lambda over the tile list (the slices' rows only; rows of
// empty slices are zero already).
template <int RP>
__device__ __noinline__ void normalize_phase(const BatchArgs &a, int n) {
    constexpr int TR = tile_rows(RP);
    const int ld = a.ld, rank = a.rank, qpr = ld / 4;
    const Span sp = cta_span(a.total_tiles[n]);
    if (sp.g0 >= sp.g1) return;
    const int64_t *prefix = a.tile_prefix[n];
    int tt = find_owner(prefix, a.count, sp.g0);
    for (int64_t gt = sp.g0; gt < sp.g1; ++gt) {
        tt = advance_owner(prefix, tt, gt);
        const BTensor &T = a.T[tt];
        const int64_t i0 = (gt - __ldg(prefix + tt)) * TR;
        const int64_t rows = T.nslices[n];
        const int32_t *fids0 = T.fids0[n];
        float *A = T.A[n];
        // the thread's row indices, then its rows, then the stores: the loads
        // of one tile are in flight together (TR * qpr <= 4 * kBThreads)
        constexpr int IT = 4;
        float4 *p[IT];
        float4 v[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int e = threadIdx.x + it * kBThreads;
            const int64_t i = i0 + e / qpr;
            p[it] = (e < TR * qpr && i < rows)
                        ? reinterpret_cast<float4 *>(A + (int64_t)__ldg(fids0 + i) * ld + (e % qpr) * 4)
                        : nullptr;
        }
#pragma unroll
        for (int it = 0; it < IT; ++it)
            if (p[it]) v[it] = *p[it];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            if (!p[it]) continue;
            const int c0 = ((threadIdx.x + it * kBThreads) % qpr) * 4;
            float4 x = v[it];
            x.x = (c0 + 0 < rank) ? x.x * T.inv_lambda[c0 + 0] : 0.f;
            x.y = (c0 + 1 < rank) ? x.y * T.inv_lambda[c0 + 1] : 0.f;
            x.z = (c0 + 2 < rank) ? x.z * T.inv_lambda[c0 + 2] : 0.f;
            x.w = (c0 + 3 < rank) ? x.w * T.inv_lambda[c0 + 3] : 0.f;
            *p[it] = x;
        }
    }
}

template <int RP, int MINB = 2>
__global__ void __launch_bounds__(kBThreads, MINB) batched_cpals_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *prep_sm = reinterpret_cast<double *>(smem);
    dense::SolveTile<RP> &solve_sm = *reinterpret_cast<dense::SolveTile<RP> *>(smem);
    if ((int)blockIdx.x == a.skip_block) return;  // test hook: a CTA that never arrives
    const int64_t it0 = *a.it_base;
    const int lane = threadIdx.x & 31;
    const int G = a.ld / 4;
    const int gpw = 32 / G;
    const int gi = lane / G;
    const int col = (lane - gi * G) * 4;
    const int rank = a.rank;

    uint64_t tp = globaltimer();
    auto phase_done = [&](int ph) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const uint64_t now = globaltimer();
            a.phase_ns[ph] += now - tp;
            tp = now;
        }
    };
    for (int it = 0; it < a.iters; ++it) {
        for (int n = 0; n < a.max_modes; ++n) {
            // M: MTTKRP of mode n over the global chunk list
            if (a.walk == 2) mttkrp_phase_wide(a, n);
            else if (gi < gpw) mttkrp_phase(a, n, gi, gpw, col);
            if (!grid_barrier(a, 0)) return;
            phase_done(0);
            // P: normal equations per tensor
            for (int tt = blockIdx.x; tt < a.count; tt += gridDim.x) {
                const BTensor &T = a.T[tt];
                if (T.nmodes <= n) continue;
                if (it == 0 && a.zero_first) {
                    float4 *p = reinterpret_cast<float4 *>(T.A[n]);
                    const int64_t nq = T.dims[n] * a.ld / 4;
                    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) p[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                dense::GramPtrs g{};
                for (int m = 0; m < T.nmodes; ++m) g.p[m] = T.G[m];
                dense::normal_prep_body(g, T.nmodes, n, rank, T.W, T.branch, prep_sm);
                __syncthreads();
            }
            if (!grid_barrier(a, 1)) return;
            phase_done(1);
            // S: row solve + Gram + dots
            solve_phase<RP>(a, n, solve_sm);
            if (!grid_barrier(a, 2)) return;
            phase_done(2);
            // F: lambda, G_n, fit
            for (int tt = blockIdx.x; tt < a.count; tt += gridDim.x) {
                const BTensor &T = a.T[tt];
                if (T.nmodes <= n) continue;
                dense::finalize_body(T.gun, rank, T.G[n], T.lambda, T.inv_lambda, T.inner);
                __syncthreads();
                for (int e = threadIdx.x; e < rank * rank + rank; e += blockDim.x) T.gun[e] = 0.0;
                if (n == T.nmodes - 1) {
                    __shared__ double red[32];
                    double s = 0.0;
                    for (int e = threadIdx.x; e < rank * rank; e += blockDim.x) {
                        double h = T.lambda[e / rank] * T.lambda[e % rank];
                        for (int m = 0; m < T.nmodes; ++m) h *= T.G[m][e];
                        s += h;
                    }
                    s = dense::block_sum_d(s, red);
                    if (threadIdx.x == 0) {
                        const double nx = *T.normx2;
                        double r2 = nx + s - 2.0 * (*T.inner);
                        if (r2 < 0.0) r2 = 0.0;
                        T.fits[(it0 + it) % kFitRing] =
                            (nx == 0.0) ? (r2 == 0.0 ? 1.0 : 0.0) : 1.0 - sqrt(r2) / sqrt(nx);
                    }
                }
                __syncthreads();
            }
            if (!grid_barrier(a, 3)) return;
            phase_done(3);
            // N: normalise the updated factor
            normalize_phase<RP>(a, n);
            if (!grid_barrier(a, 4)) return;
            phase_done(4);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.it_base = it0 + a.iters;
}

size_t batched_smem_bytes(int rank, int rp) {
    const int half = (rank + 2) / 2;
    const size_t prep = (3 * (size_t)rank * rank + 16 + 2 * half) * sizeof(double) + 2 * half * sizeof(int) + 64;
    const size_t solve = rp == 16 ? sizeof(dense::SolveTile<16>) : sizeof(dense::SolveTile<32>);
    return prep > solve ? prep : solve;
}

}  // namespace
}  // namespace sptt

using namespace sptt;

struct sptt_batch {
    int32_t count = 0, rank = 0, ld = 0, max_modes = 0;
    sptt_opts opts{};
    sptt_sched sched{};
    bool has_sched = false;
    int walk = 1;  // MTTKRP walk (batch_walk)
    int minb = 2;  // CTAs per SM the kernel is built for (1 for the 32-byte walk)
    cudaStream_t st = nullptr;
    std::vector<sptt_csf *> csfs;       // count * max_modes (null where absent)
    std::vector<BTensor> host;          // descriptors as copied to the device
    std::vector<int64_t> m_elems;       // per tensor: elements of its compact M
    std::vector<int64_t> mh_elems;      // per tensor: elements of its heavy rows
    std::vector<void *> allocs;         // every device buffer owned by the batch
    BTensor *d_tensors = nullptr;
    int64_t *d_prefix = nullptr;        // 2 * max_modes * (count + 1)
    int32_t *d_owner[kMaxModes] = {nullptr};  // per mode position: tensor of each global chunk
    int64_t total_chunks[kMaxModes] = {0};
    int64_t total_tiles[kMaxModes] = {0};
    unsigned *d_bar = nullptr;
    int32_t *d_err = nullptr;
    unsigned long long *d_phase = nullptr;
    int64_t *d_it_base = nullptr;
    double *partials = nullptr;         // Gram workspace for init
    int32_t gram_blocks = 0;
    int64_t iters_run = 0;
    int grid = 0;
    uint64_t timeout_ns = 2000000000ull;
    int32_t skip_block = -1;
    cudaGraphExec_t graph = nullptr;
    int32_t graph_iters = -1;
    bool zero_first = true;
    int32_t chunk = 128;                // leaves per MTTKRP chunk of every CSF
    float tuned_ms = 0.f;               // plan 1: time of the chosen candidate's timed run
    int32_t tuned_candidates = 0;       // plan 1: candidates timed
};

namespace {

void batch_destroy(sptt_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->st);
    for (auto *c : b->csfs)
        if (c) csf_destroy(c);
    for (void *p : b->allocs) dev_free(p, b->st);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaStreamSynchronize(b->st);
    delete b;
}

// The batched MTTKRP walk reads the packed leaf records (16 bytes per
// non-zero more on the device) unless the schedule names variant 3 (the
// 16-byte walk on the separate leaf arrays). With ld a multiple of 8 (R = 8,
// 16, 32) it is the 32-byte-segment walk in the 1-CTA-per-SM build of the
// kernel, unless the schedule names variant 4 (the 16-byte walk on packed
// records, 2 CTAs per SM). Measured on the 512-tensor batch at R = 16: 0.43 s
// per run against 0.49 s for the 16-byte walk (its MTTKRP phase is 23 %
// faster, the other phases slower with half the CTAs).
bool batch_packed(const sptt_sched *sched) { return !(sched && sched->variant == 3); }
int batch_walk(const sptt_sched *sched, int32_t ld) {
    if (!batch_packed(sched)) return 0;
    if (ld % 8 == 0 && !(sched && sched->variant == 4)) return 2;
    return 1;
}

// The schedule variant that names a walk (inverse of batch_walk).
int32_t walk_variant(int walk) { return walk == 0 ? 3 : (walk == 1 ? 4 : 7); }

using BatchKernel = void (*)(const BatchArgs);
BatchKernel batch_kernel(int rp, int minb) {
    if (minb == 1) return rp == 16 ? batched_cpals_kernel<16, 1> : batched_cpals_kernel<32, 1>;
    return rp == 16 ? batched_cpals_kernel<16, 2> : batched_cpals_kernel<32, 2>;
}

template <typename T>
sptt_status batch_alloc(sptt_batch *b, T **p, size_t n, bool zero) {
    SPTT_TRY(dev_alloc_n(p, n, b->st));
    b->allocs.push_back(*p);
    if (zero) SPTT_TRY(fill_zero_launch(*p, n * sizeof(T), b->st));
    return SPTT_OK;
}

sptt_status launch_batch(sptt_batch *b, int32_t iters) {
    BatchArgs a{};
    a.T = b->d_tensors;
    a.count = b->count;
    a.rank = b->rank;
    a.ld = b->ld;
    a.iters = iters;
    a.max_modes = b->max_modes;
    for (int n = 0; n < b->max_modes; ++n) {
        a.chunk_prefix[n] = b->d_prefix + (2 * n) * (b->count + 1);
        a.chunk_owner[n] = b->d_owner[n];
        a.tile_prefix[n] = b->d_prefix + (2 * n + 1) * (b->count + 1);
        a.total_chunks[n] = b->total_chunks[n];
        a.total_tiles[n] = b->total_tiles[n];
    }
    a.bar = b->d_bar;
    a.err = b->d_err;
    a.it_base = b->d_it_base;
    a.timeout_ns = b->timeout_ns;
    a.skip_block = b->skip_block;
    a.phase_ns = b->d_phase;
    a.zero_first = b->zero_first ? 1 : 0;
    a.walk = b->walk;
    SPTT_TRY(fill_zero_launch(b->d_bar, 2 * sizeof(unsigned), b->st));
    SPTT_TRY(fill_zero_launch(b->d_err, sizeof(int32_t), b->st));
    const int rp = b->rank <= 16 ? 16 : 32;
    const size_t smem = batched_smem_bytes(b->rank, rp);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SPTT_CUDA(cudaLaunchKernelEx(&cfg, batch_kernel(rp, b->minb), a));
    count_launch();
    return SPTT_OK;
}

// Everything that depends on the chunk size and the walk: every CSF's work
// partition, the tensors' walk arguments, the global chunk and tile lists,
// the kernel build (CTAs per SM) and the cooperative grid. Called once, or
// once per candidate by the plan-1 timing.
sptt_status batch_layout(sptt_batch *b, int32_t chunk, int walk) {
    const int count = b->count, rank = b->rank;
    SPTT_CUDA(cudaStreamSynchronize(b->st));  // no run may still read the old layout
    b->chunk = chunk;
    std::vector<int64_t> prefix((size_t)2 * b->max_modes * (count + 1), 0);
    for (int t = 0; t < count; ++t) {
        BTensor &T = b->host[t];
        int64_t heavy = 0;
        for (int m = 0; m < T.nmodes; ++m) {
            sptt_csf *cs = b->csfs[(size_t)t * b->max_modes + m];
            SPTT_TRY(csf_ensure_partition(cs, chunk, b->st));
            if (cs->nheavy > heavy) heavy = cs->nheavy;
            walk::Args &w = T.w[m];
            w = walk::Args{};
            for (int l = 0; l < T.nmodes; ++l) {
                w.fptr[l] = cs->fptr[l];
                w.fids[l] = cs->fids[l];
                w.fac[l] = l ? T.A[cs->order[l]] : nullptr;
            }
            w.vals = cs->vals;
            w.lvl = cs->lvl;
            w.leafrec = cs->leafrec;
            w.part = cs->part;
            w.nchunks = cs->part_nchunks;
            w.nnz = cs->nfibs[T.nmodes - 1];
            w.chunk = cs->part_chunk;
            w.ld = b->ld;
            w.out = T.M;
            w.heavy = T.Mh;
            w.hidx = cs->hidx;
            T.hidx[m] = cs->hidx;
            T.fids0[m] = cs->fids[0];
            T.nslices[m] = cs->nfibs[0];
        }
        if (heavy * b->ld > b->mh_elems[t]) return set_error(SPTT_ERR_INTERNAL, "heavy rows outgrow their buffer");
    }
    // global work lists: per mode position, chunk and tile prefix sums over the tensors
    for (int n = 0; n < b->max_modes; ++n) {
        int64_t *cp = prefix.data() + (2 * n) * (count + 1);
        int64_t *tp = prefix.data() + (2 * n + 1) * (count + 1);
        for (int t = 0; t < count; ++t) {
            const BTensor &T = b->host[t];
            const bool has = T.nmodes > n;
            cp[t + 1] = cp[t] + (has ? T.w[n].nchunks : 0);
            const int tr = tile_rows(rank <= 16 ? 16 : 32);
            tp[t + 1] = tp[t] + (has ? (T.nslices[n] + tr - 1) / tr : 0);
        }
        b->total_chunks[n] = cp[count];
        b->total_tiles[n] = tp[count];
    }
    SPTT_CUDA(cudaMemcpyAsync(b->d_tensors, b->host.data(), sizeof(BTensor) * count, cudaMemcpyHostToDevice, b->st));
    SPTT_TRY(batch_alloc(b, &b->d_prefix, prefix.size(), false));
    SPTT_CUDA(cudaMemcpyAsync(b->d_prefix, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                              b->st));
    {
        // chunk -> tensor tables (one load per chunk in the MTTKRP phase)
        std::vector<int32_t> owner;
        for (int n = 0; n < b->max_modes; ++n) {
            const int64_t *cp = prefix.data() + (2 * n) * (count + 1);
            owner.assign((size_t)cp[count], 0);
            for (int t = 0; t < count; ++t)
                for (int64_t g = cp[t]; g < cp[t + 1]; ++g) owner[(size_t)g] = t;
            SPTT_TRY(batch_alloc(b, &b->d_owner[n], owner.size() + 1, false));
            if (!owner.empty())
                SPTT_CUDA(cudaMemcpyAsync(b->d_owner[n], owner.data(), owner.size() * sizeof(int32_t),
                                          cudaMemcpyHostToDevice, b->st));
            SPTT_CUDA(cudaStreamSynchronize(b->st));  // the host vectors are reused
        }
    }
    // a grid that is fully resident (cooperative launch)
    const int rp = rank <= 16 ? 16 : 32;
    const size_t smem = batched_smem_bytes(rank, rp);
    b->walk = walk;
    if (b->walk == 2) {  // 32-byte row loads need 32-byte aligned factors
        for (int t = 0; t < count; ++t)
            for (int m = 0; m < b->host[t].nmodes; ++m)
                if (reinterpret_cast<uintptr_t>(b->host[t].A[m]) % 32) b->walk = 1;
    }
    b->minb = b->walk == 2 ? 1 : 2;
    auto kern = batch_kernel(rp, b->minb);
    SPTT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SPTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem));
    if (per_sm < 1) return set_error(SPTT_ERR_INTERNAL, "batched kernel does not fit on an SM");
    b->grid = device_sm_count() * per_sm;
    if (b->graph) {  // a captured run belongs to the old layout
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_iters = -1;
    }
    SPTT_CUDA(cudaStreamSynchronize(b->st));
    return SPTT_OK;
}

}  // namespace

extern "C" sptt_status sptt_batch_init(sptt_batch *b);
extern "C" sptt_status sptt_batch_run(sptt_batch *b, int32_t iters);

extern "C" sptt_status sptt_batch_create(const sptt_coo *coos, int32_t count, int32_t rank, const sptt_opts *opts,
                                         sptt_stream stream, sptt_batch **out) {
    clear_error();
    if (!out || !coos) return set_error(SPTT_ERR_BAD_ARG, "coos and out must be non-NULL");
    *out = nullptr;
    if (count < 1) return set_error(SPTT_ERR_BAD_ARG, "count must be >= 1");
    if (rank < 1 || rank > 32) return set_error(SPTT_ERR_UNSUPPORTED, "batched rank must be in [1, 32]");
    sptt_batch *b = new sptt_batch();
    struct Guard {
        sptt_batch *b;
        ~Guard() { if (b) batch_destroy(b); }
    } guard{b};
    if (opts) b->opts = *opts;
    if (b->opts.sched) {
        b->sched = *b->opts.sched;
        b->has_sched = true;
    }
    b->opts.sched = nullptr;
    b->st = reinterpret_cast<cudaStream_t>(stream);
    b->count = count;
    b->rank = rank;
    b->ld = (rank + 3) / 4 * 4;
    for (int t = 0; t < count; ++t) {
        SPTT_TRY(coo_validate_shape(&coos[t]));
        if (coos[t].nnz == 0) return set_error(SPTT_ERR_BAD_ARG, "every tensor needs a non-zero");
        if (coos[t].nmodes > 4) return set_error(SPTT_ERR_UNSUPPORTED, "batched tensors have 2 to 4 modes");
        if (coos[t].nmodes > b->max_modes) b->max_modes = coos[t].nmodes;
    }
    const sptt_sched *sched = b->has_sched ? &b->sched : nullptr;
    if (b->opts.plan < 0 || b->opts.plan > 1) return set_error(SPTT_ERR_BAD_ARG, "batched opts.plan must be 0 or 1");
    const bool tune = b->opts.plan == 1;
    b->chunk = (sched && sched->chunk) ? sched->chunk : 128;
    if (b->chunk < 16 || b->chunk > 4096 || (b->chunk & (b->chunk - 1)))
        return set_error(SPTT_ERR_BAD_ARG, "sched->chunk must be a power of two in [16, 4096]");
    // the chunk sizes the layout may take (plan 1 times each of them)
    std::vector<int32_t> chunks = tune ? std::vector<int32_t>{64, 128, 256} : std::vector<int32_t>{b->chunk};
    b->csfs.assign((size_t)count * b->max_modes, nullptr);
    b->host.resize(count);
    int64_t max_rows = 0;
    for (int t = 0; t < count; ++t) {
        const sptt_coo &c = coos[t];
        BTensor &T = b->host[t];
        T = BTensor{};
        T.nmodes = c.nmodes;
        int64_t max_slices = 0, max_heavy = 0;
        {
            DevCoo dc;
            SPTT_TRY(coo_to_device(&c, b->st, &dc));
            for (int m = 0; m < c.nmodes; ++m) {
                sptt_csf *cs = nullptr;
                SPTT_TRY(csf_build_device(&dc.coo, m, nullptr, b->st, &cs));
                b->csfs[(size_t)t * b->max_modes + m] = cs;
                // the FP64 rows of split slices are sized for the largest count any layout gives
                for (int32_t ch : chunks) {
                    SPTT_TRY(csf_ensure_partition(cs, ch, b->st));
                    if (cs->nheavy > max_heavy) max_heavy = cs->nheavy;
                }
                if (tune || batch_packed(sched)) SPTT_TRY(csf_ensure_leafrec(cs, b->st));
                if (cs->nfibs[0] > max_slices) max_slices = cs->nfibs[0];
            }
        }
        for (int m = 0; m < c.nmodes; ++m) {
            T.dims[m] = c.dims[m];
            if (c.dims[m] > max_rows) max_rows = c.dims[m];
            SPTT_TRY(batch_alloc(b, &T.A[m], (size_t)c.dims[m] * b->ld, true));
            SPTT_TRY(batch_alloc(b, &T.G[m], (size_t)rank * rank, true));
        }
        SPTT_TRY(batch_alloc(b, &T.M, (size_t)max_slices * b->ld, true));
        SPTT_TRY(batch_alloc(b, &T.Mh, (size_t)max_heavy * b->ld, true));
        b->mh_elems.push_back(max_heavy * b->ld);
        b->m_elems.push_back(max_slices * b->ld);
        SPTT_TRY(batch_alloc(b, &T.gun, (size_t)rank * rank + rank, true));
        SPTT_TRY(batch_alloc(b, &T.W, (size_t)rank * rank, true));
        SPTT_TRY(batch_alloc(b, &T.lambda, (size_t)rank, true));
        SPTT_TRY(batch_alloc(b, &T.inv_lambda, (size_t)rank, true));
        SPTT_TRY(batch_alloc(b, &T.inner, 1, true));
        SPTT_TRY(batch_alloc(b, &T.normx2, 1, true));
        SPTT_TRY(batch_alloc(b, &T.fits, kFitRing, true));
        SPTT_TRY(batch_alloc(b, &T.branch, 2, true));
        const sptt_csf *c0 = b->csfs[(size_t)t * b->max_modes];
        SPTT_TRY(sumsq_launch(c0->vals, c0->nfibs[c.nmodes - 1], T.normx2, b->st));
    }
    SPTT_TRY(batch_alloc(b, &b->d_tensors, (size_t)count, false));
    SPTT_TRY(batch_alloc(b, &b->d_bar, 2, true));
    SPTT_TRY(batch_alloc(b, &b->d_err, 1, true));
    SPTT_TRY(batch_alloc(b, &b->d_it_base, 1, true));
    SPTT_TRY(batch_alloc(b, &b->d_phase, 10, true));
    b->gram_blocks = device_sm_count() * 2;
    SPTT_TRY(batch_alloc(b, &b->partials, (size_t)b->gram_blocks * (rank * rank + rank), false));
    if (!tune) {
        SPTT_TRY(batch_layout(b, b->chunk, batch_walk(sched, b->ld)));
    } else {
        // plan 1: time every (walk, chunk) candidate on the batch itself, one
        // warm-up run and one timed run of 2 iterations each from fresh
        // factors, and keep the fastest (the factors are re-initialised by
        // sptt_batch_init before the caller's runs)
        std::vector<int> walks = {1};
        if (b->ld % 8 == 0) walks.push_back(2);
        cudaEvent_t e0, e1;
        SPTT_CUDA(cudaEventCreate(&e0));
        SPTT_CUDA(cudaEventCreate(&e1));
        struct Ev {
            cudaEvent_t a, b;
            ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
        } evg{e0, e1};
        const bool graph = b->opts.use_graph;
        b->opts.use_graph = 0;
        float best = -1.f;
        int best_walk = 1;
        int32_t best_chunk = 128;
        for (int wk : walks)
            for (int32_t ch : chunks) {
                SPTT_TRY(batch_layout(b, ch, wk));
                if (b->walk != wk) continue;  // the 32-byte walk was refused (alignment)
                SPTT_TRY(sptt_batch_init(b));
                SPTT_TRY(sptt_batch_run(b, 2));
                SPTT_TRY(sptt_batch_init(b));
                SPTT_CUDA(cudaEventRecord(e0, b->st));
                SPTT_TRY(sptt_batch_run(b, 2));
                SPTT_CUDA(cudaEventRecord(e1, b->st));
                SPTT_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                SPTT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                ++b->tuned_candidates;
                if (best < 0.f || ms < best) {
                    best = ms;
                    best_walk = wk;
                    best_chunk = ch;
                }
            }
        b->opts.use_graph = graph;
        b->tuned_ms = best;
        SPTT_TRY(batch_layout(b, best_chunk, best_walk));
    }
    SPTT_CUDA(cudaStreamSynchronize(b->st));
    guard.b = nullptr;
    *out = b;
    return SPTT_OK;
}

extern "C" void sptt_batch_free(sptt_batch *b) { batch_destroy(b); }

extern "C" sptt_status sptt_batch_init(sptt_batch *b) {
    clear_error();
    if (!b) return set_error(SPTT_ERR_BAD_ARG, "batch is NULL");
    for (int t = 0; t < b->count; ++t) {
        const BTensor &T = b->host[t];
        for (int m = 0; m < T.nmodes; ++m) {
            SPTT_TRY(init_factor_launch(b->opts.seed + (uint64_t)t, m, T.dims[m], b->rank, b->ld, T.A[m], b->st));
            SPTT_TRY(gram_launch(T.A[m], T.dims[m], b->rank, b->ld, T.G[m], b->partials, b->gram_blocks, b->st));
        }
        SPTT_TRY(fill_zero_launch(T.branch, 2 * sizeof(int32_t), b->st));
        SPTT_TRY(fill_zero_launch(T.fits, kFitRing * sizeof(double), b->st));
        // a run that stopped early may have left partial sums behind
        SPTT_TRY(fill_zero_launch(T.M, (size_t)b->m_elems[t] * sizeof(float), b->st));
        SPTT_TRY(fill_zero_launch(T.Mh, (size_t)b->mh_elems[t] * sizeof(double), b->st));
        SPTT_TRY(fill_zero_launch(T.gun, ((size_t)b->rank * b->rank + b->rank) * sizeof(double), b->st));
    }
    SPTT_TRY(fill_zero_launch(b->d_it_base, sizeof(int64_t), b->st));
    b->iters_run = 0;
    b->zero_first = true;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_iters = -1;
    }
    return SPTT_OK;
}

extern "C" sptt_status sptt_batch_run(sptt_batch *b, int32_t iters) {
    clear_error();
    if (!b) return set_error(SPTT_ERR_BAD_ARG, "batch is NULL");
    if (iters < 1) return set_error(SPTT_ERR_BAD_ARG, "iters must be >= 1");
    const bool graph = b->opts.use_graph && b->st != nullptr && b->skip_block < 0;
    if (graph) {
        // the graph replays runs after the first (factors already zeroed on empty rows)
        if (b->zero_first) {
            SPTT_TRY(launch_batch(b, iters));
            b->zero_first = false;
        } else {
            if (!b->graph || b->graph_iters != iters) {
                if (b->graph) cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
                cudaGraph_t g = nullptr;
                SPTT_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
                const int64_t l0 = sptt_debug_launch_count();
                sptt_status s = launch_batch(b, iters);
                const int64_t l1 = sptt_debug_launch_count();
                cudaError_t e = cudaStreamEndCapture(b->st, &g);
                if (s != SPTT_OK) {
                    if (g) cudaGraphDestroy(g);
                    return s;
                }
                if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&b->graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
                b->graph_iters = iters;
                count_launch(-(l1 - l0));
            }
            SPTT_CUDA(cudaGraphLaunch(b->graph, b->st));
            count_launch(3);  // two clears and the persistent kernel
        }
    } else {
        SPTT_TRY(launch_batch(b, iters));
        b->zero_first = false;
    }
    b->iters_run += iters;
    int32_t err = 0;
    SPTT_CUDA(cudaMemcpyAsync(&err, b->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, b->st));
    SPTT_CUDA(cudaStreamSynchronize(b->st));
    if (err) return set_error(SPTT_ERR_TIMEOUT, "a grid barrier wait of the batched kernel ran out");
    return SPTT_OK;
}

extern "C" sptt_status sptt_batch_fit_history(sptt_batch *b, int32_t t, double *fits, int32_t cap, int32_t *count) {
    clear_error();
    if (!b || !fits) return set_error(SPTT_ERR_BAD_ARG, "batch and fits must be non-NULL");
    if (t < 0 || t >= b->count) return set_error(SPTT_ERR_BAD_ARG, "tensor index out of range");
    const int64_t avail = b->iters_run < kFitRing ? b->iters_run : kFitRing;
    const int64_t n = avail < cap ? avail : cap;
    std::vector<double> ring(kFitRing);
    SPTT_CUDA(cudaMemcpyAsync(ring.data(), b->host[t].fits, kFitRing * sizeof(double), cudaMemcpyDeviceToHost, b->st));
    SPTT_CUDA(cudaStreamSynchronize(b->st));
    for (int64_t j = 0; j < n; ++j) fits[j] = ring[(b->iters_run - n + j) % kFitRing];
    if (count) *count = (int32_t)n;
    return SPTT_OK;
}

extern "C" sptt_status sptt_batch_factor(sptt_batch *b, int32_t t, int32_t mode, float *dst) {
    clear_error();
    if (!b || !dst) return set_error(SPTT_ERR_BAD_ARG, "batch and dst must be non-NULL");
    if (t < 0 || t >= b->count) return set_error(SPTT_ERR_BAD_ARG, "tensor index out of range");
    const BTensor &T = b->host[t];
    if (mode < 0 || mode >= T.nmodes) return set_error(SPTT_ERR_BAD_ARG, "mode out of range");
    SPTT_CUDA(cudaMemcpy2DAsync(dst, b->rank * sizeof(float), T.A[mode], b->ld * sizeof(float),
                                b->rank * sizeof(float), T.dims[mode], cudaMemcpyDefault, b->st));
    SPTT_CUDA(cudaStreamSynchronize(b->st));
    return SPTT_OK;
}

extern "C" sptt_status sptt_batch_lambda(sptt_batch *b, int32_t t, double *lambda) {
    clear_error();
    if (!b || !lambda) return set_error(SPTT_ERR_BAD_ARG, "batch and lambda must be non-NULL");
    if (t < 0 || t >= b->count) return set_error(SPTT_ERR_BAD_ARG, "tensor index out of range");
    SPTT_CUDA(cudaMemcpyAsync(lambda, b->host[t].lambda, b->rank * sizeof(double), cudaMemcpyDefault, b->st));
    SPTT_CUDA(cudaStreamSynchronize(b->st));
    return SPTT_OK;
}

extern "C" sptt_status sptt_batch_info(sptt_batch *b, int32_t *grid, int64_t *chunks, int64_t *tiles) {
    clear_error();
    if (!b) return set_error(SPTT_ERR_BAD_ARG, "batch is NULL");
    if (grid) *grid = b->grid;
    for (int n = 0; n < SPTT_MAX_MODES; ++n) {
        if (chunks) chunks[n] = n < b->max_modes ? b->total_chunks[n] : 0;
        if (tiles) tiles[n] = n < b->max_modes ? b->total_tiles[n] : 0;
    }
    return SPTT_OK;
}

extern "C" sptt_status sptt_batch_schedule(sptt_batch *b, sptt_sched *out, float *tuned_ms, int32_t *candidates) {
    clear_error();
    if (!b || !out) return set_error(SPTT_ERR_BAD_ARG, "batch and out must be non-NULL");
    sptt_sched s{};
    s.chunk = b->chunk;
    s.block = kBThreads;
    s.variant = walk_variant(b->walk);
    *out = s;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    if (candidates) *candidates = b->tuned_candidates;
    return SPTT_OK;
}

extern "C" sptt_status sptt_batch_phase_ms(sptt_batch *b, double *ms) {
    clear_error();
    if (!b || !ms) return set_error(SPTT_ERR_BAD_ARG, "batch and ms must be non-NULL");
    unsigned long long ns[10];
    SPTT_CUDA(cudaMemcpyAsync(ns, b->d_phase, sizeof(ns), cudaMemcpyDeviceToHost, b->st));
    SPTT_CUDA(cudaStreamSynchronize(b->st));
    for (int i = 0; i < 10; ++i) ms[i] = ns[i] * 1e-6;
    return SPTT_OK;
}

extern "C" sptt_status sptt_debug_batch_stall(sptt_batch *b, int32_t skip_block, int64_t timeout_ns) {
    clear_error();
    if (!b) return set_error(SPTT_ERR_BAD_ARG, "batch is NULL");
    if (skip_block >= b->grid) return set_error(SPTT_ERR_BAD_ARG, "skip_block >= grid size");
    b->skip_block = skip_block < 0 ? -1 : skip_block;
    b->timeout_ns = timeout_ns > 0 ? (uint64_t)timeout_ns : 2000000000ull;
    return SPTT_OK;
}
