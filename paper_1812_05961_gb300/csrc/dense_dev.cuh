// Device-side bodies of the dense R x R steps of CP-ALS (Algorithm 1),
// shared by the per-step kernels in dense.cu and the batched persistent
// kernel in batched.cu.
#pragma once

#include "internal.cuh"

namespace sptt {
namespace dense {
namespace {

struct GramPtrs {
    const double *p[kMaxModes];
};

__device__ __forceinline__ double block_sum_d(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------------------
// Row solve after each MTTKRP (Algorithm 1: solve and normalise): for one
// tile of TR = 4096 / RP rows of the compact MTTKRP result M (heavy slices
// from their FP64 rows), A_un = M W is written to A at the slices' mode
// indices, and each thread adds its share of the Gram A_un^T A_un and of the
// column dots <M, A_un> (for the fit) to FP32 sums; every 64 rows (16 for
// the dots) those are added to the thread's FP64 totals (kept in shared
// memory), and a block reduction finally hands the totals to the caller. Shared by the per-step kernel (per-block
// partials) and the batched kernel (atomics per tensor). 256 threads.
// ---------------------------------------------------------------------------
template <int RP>
struct SolveTile {
    static constexpr int TR = 4096 / RP;             // rows per tile
    static constexpr int S = RP + 4;                 // row stride: 16-byte rows, conflict-free float4 access
    static constexpr int TPR = RP / 16;              // product: threads per row, 16 columns each
    static constexpr int NB = (RP / 4) * (RP / 4);   // Gram: 4 x 4 blocks of entries
    static constexpr int RG = 256 / NB;              // Gram: row groups
    static constexpr int GROWS = TR / RG;            // Gram: rows per thread per tile
    static constexpr int DG = 256 / RP;              // dots: row groups
    static constexpr int CONV = GROWS >= 64 ? 1 : 64 / GROWS;  // tiles per FP32 run
    float W[RP][RP];
    float Mt[TR][S];
    float At[TR][S];
    double G[256][17];  // per thread: FP64 totals of its 4 x 4 Gram block (padded: conflict-free)
    double D[256];      // per thread: FP64 total of its dot
};

// Per-thread FP32 run sums (registers).
struct SolveRun {
    float gs[16];
    float ds;
    int run;
};

template <int RP>
__device__ __forceinline__ void solve_begin(SolveTile<RP> &sm, SolveRun &acc) {
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        acc.gs[q] = 0.f;
        sm.G[t][q] = 0.0;
    }
    acc.ds = 0.f;
    sm.D[t] = 0.0;
    acc.run = 0;
}

template <int RP>
__device__ __forceinline__ void solve_end_run(SolveTile<RP> &sm, SolveRun &acc) {
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        sm.G[t][q] += (double)acc.gs[q];
        acc.gs[q] = 0.f;
    }
    sm.D[t] += (double)acc.ds;
    acc.ds = 0.f;
    acc.run = 0;
}

// W (rank x rank, FP32, row-major) into the tile's zero-padded RP x RP copy.
// The caller orders it against the tile's readers (the tile starts and ends
// with a barrier).
template <int RP>
__device__ __forceinline__ void solve_load_w(SolveTile<RP> &sm, const float *__restrict__ Wg, int rank) {
    for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
        const int r = e / RP, c = e % RP;
        sm.W[r][c] = (r < rank && c < rank) ? Wg[r * rank + c] : 0.f;
    }
}

// One tile starting at compact row i0. CLEAR leaves the rows of M (and the
// heavy rows) it read at zero, ready for the next MTTKRP. fids0 = NULL: row i
// of M is row i of A (a full MTTKRP result); hidx = NULL: no heavy rows.
template <int RP, bool CLEAR>
__device__ __forceinline__ void solve_tile(SolveTile<RP> &sm, SolveRun &acc, float *M, double *heavy,
                                           const int32_t *__restrict__ hidx, const int32_t *__restrict__ fids0,
                                           float *A, int64_t i0, int64_t rows, int rank, int ld) {
    using ST = SolveTile<RP>;
    constexpr int Q = RP / 4;
    constexpr int IT = ST::TR * Q / 256;  // float4 pieces per thread (4)
    static_assert(ST::TR * Q == IT * 256, "a tile is whole float4 pieces per thread");
    const int t = threadIdx.x;
    // all of the thread's heavy-row indices, then all of its M pieces, then
    // the clearing stores: the loads of one tile are in flight together
    int32_t h[IT];
    bool live[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int e = t + it * 256;
        const int r = e / Q, c = (e % Q) * 4;
        const int64_t i = i0 + r;
        live[it] = i < rows && c < ld;
        h[it] = (live[it] && hidx) ? __ldg(hidx + i) : -1;
    }
    float4 v[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int e = t + it * 256;
        const int r = e / Q, c = (e % Q) * 4;
        const int64_t i = i0 + r;
        v[it] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live[it]) {
            if (h[it] >= 0) {
                const double2 *ph = reinterpret_cast<const double2 *>(heavy + (int64_t)h[it] * ld + c);
                const double2 d0 = ph[0], d1 = ph[1];
                v[it] = make_float4((float)d0.x, (float)d0.y, (float)d1.x, (float)d1.y);
            } else {
                v[it] = *reinterpret_cast<const float4 *>(M + i * ld + c);
            }
        }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int e = t + it * 256;
        const int r = e / Q, c = (e % Q) * 4;
        const int64_t i = i0 + r;
        if (CLEAR && live[it]) {
            *reinterpret_cast<float4 *>(M + i * ld + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            if (h[it] >= 0) {
                double2 *ph = reinterpret_cast<double2 *>(heavy + (int64_t)h[it] * ld + c);
                ph[0] = make_double2(0.0, 0.0);
                ph[1] = make_double2(0.0, 0.0);
            }
        }
        float4 x = v[it];
        if (c + 0 >= rank) x.x = 0.f;
        if (c + 1 >= rank) x.y = 0.f;
        if (c + 2 >= rank) x.z = 0.f;
        if (c + 3 >= rank) x.w = 0.f;
        *reinterpret_cast<float4 *>(&sm.Mt[r][c]) = x;
    }
    __syncthreads();
    {
        const int r = t / ST::TPR, cb = (t % ST::TPR) * 16;
        const int64_t irow = i0 + r;
        const int64_t arow = irow < rows ? (fids0 ? (int64_t)__ldg(fids0 + irow) : irow) : 0;  // requested before the product
        float o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = 0.f;
#pragma unroll 2
        for (int k = 0; k < RP; k += 4) {
            const float4 m4 = *reinterpret_cast<const float4 *>(&sm.Mt[r][k]);
            const float mk[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 w4 = *reinterpret_cast<const float4 *>(&sm.W[k + kk][cb + 4 * q]);
                    o[4 * q + 0] = fmaf(mk[kk], w4.x, o[4 * q + 0]);
                    o[4 * q + 1] = fmaf(mk[kk], w4.y, o[4 * q + 1]);
                    o[4 * q + 2] = fmaf(mk[kk], w4.z, o[4 * q + 2]);
                    o[4 * q + 3] = fmaf(mk[kk], w4.w, o[4 * q + 3]);
                }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4 *>(&sm.At[r][cb + 4 * q]) =
                make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        if (irow < rows) {
            float *dst = A + arow * ld + cb;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (cb + 4 * q < ld)
                    *reinterpret_cast<float4 *>(dst + 4 * q) =
                        make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        }
    }
    __syncthreads();
    {
        const int blk = t % ST::NB, g = t / ST::NB;
        const int bx = blk / (RP / 4), by = blk % (RP / 4);
        const int live = (rows - i0 < ST::TR) ? (int)(rows - i0) : ST::TR;  // rows past the end are zero
        for (int r = g; r < live; r += ST::RG) {
            const float4 a4 = *reinterpret_cast<const float4 *>(&sm.At[r][bx * 4]);
            const float4 b4 = *reinterpret_cast<const float4 *>(&sm.At[r][by * 4]);
            const float xa[4] = {a4.x, a4.y, a4.z, a4.w}, xb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc.gs[x * 4 + y] = fmaf(xa[x], xb[y], acc.gs[x * 4 + y]);
        }
        const int c = t % RP;
        for (int r = t / RP; r < live; r += ST::DG) acc.ds = fmaf(sm.Mt[r][c], sm.At[r][c], acc.ds);
    }
    __syncthreads();
    if (++acc.run == ST::CONV) solve_end_run(sm, acc);
}

// Block-wide totals of the Gram (entry r * rank + c) and of the dots (entry
// rank * rank + c), handed to emit(entry, value) in a fixed order; then the
// totals restart from zero. Every thread of the block calls it.
template <int RP, typename Emit>
__device__ __forceinline__ void solve_reduce(SolveTile<RP> &sm, SolveRun &acc, int rank, Emit emit) {
    using ST = SolveTile<RP>;
    solve_end_run(sm, acc);
    const int t = threadIdx.x;
    __syncthreads();
    for (int e = t; e < ST::NB * 16; e += 256) {
        const int b = e / 16, q = e % 16;
        double v = 0.0;
        for (int gg = 0; gg < ST::RG; ++gg) v += sm.G[gg * ST::NB + b][q];
        const int r = (b / (RP / 4)) * 4 + q / 4, c = (b % (RP / 4)) * 4 + q % 4;
        if (r < rank && c < rank) emit(r * rank + c, v);
    }
    if (t < RP) {
        double v = 0.0;
        for (int gg = 0; gg < ST::DG; ++gg) v += sm.D[gg * RP + t];
        if (t < rank) emit(rank * rank + t, v);
    }
    __syncthreads();
    solve_begin(sm, acc);
}

// V = Hadamard_{m != n} G_m; W = V^dagger (FP64: Cholesky with the
// positive-definite test, else the pseudo-inverse by parallel cyclic
// Jacobi). One CTA; sm holds 3 R^2 + 16 + (R + 2) doubles and R + 2 ints.
__device__ __noinline__ void normal_prep_body(const GramPtrs &g, int nmodes, int n, int rank, float *__restrict__ W,
                                              int32_t *__restrict__ branch, double *sm) {
    const int R = rank, RR = R * R;
    double *V = sm;            // Hadamard product (kept for the pinv branch)
    double *S = sm + RR;       // Cholesky factor, or Jacobi working matrix
    double *X = sm + 2 * RR;   // L^-1, or the Jacobi eigenvectors
    double *misc = sm + 3 * RR;  // [0] threshold, [1] pd flag, [2..9] reduction scratch, [16..] rotations
    const int t = threadIdx.x;
    for (int e = t; e < RR; e += blockDim.x) {
        double h = 1.0;
        for (int m = 0; m < nmodes; ++m)
            if (m != n) h *= g.p[m][e];
        V[e] = h;
        S[e] = h;
    }
    __syncthreads();
    if (t == 0) {
        double dmax = 0.0;
        for (int i = 0; i < R; ++i) dmax = fmax(dmax, V[i * R + i]);
        misc[0] = 1e-14 * dmax;
        misc[1] = 1.0;
    }
    __syncthreads();
    // Right-looking Cholesky of S (lower triangle), with the positive-definite test.
    for (int j = 0; j < R; ++j) {
        if (t == 0) {
            const double d = S[j * R + j];
            if (!(d > misc[0])) misc[1] = 0.0;
            else S[j * R + j] = sqrt(d);
        }
        __syncthreads();
        if (misc[1] == 0.0) break;
        const double ljj = S[j * R + j];
        for (int i = j + 1 + t; i < R; i += blockDim.x) S[i * R + j] /= ljj;
        __syncthreads();
        const int m = R - j - 1;
        for (int e = t; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e / m, k = j + 1 + e % m;
            if (k <= i) S[i * R + k] -= S[i * R + j] * S[k * R + j];
        }
        __syncthreads();
    }
    const bool pd = misc[1] != 0.0;
    if (pd) {
        // X = L^-1 (lower triangular), one column per thread
        for (int c = t; c < R; c += blockDim.x) {
            for (int i = 0; i < c; ++i) X[i * R + c] = 0.0;
            for (int i = c; i < R; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                for (int k = c; k < i; ++k) s -= S[i * R + k] * X[k * R + c];
                X[i * R + c] = s / S[i * R + i];
            }
        }
        __syncthreads();
        // V^-1 = L^-T L^-1
        for (int e = t; e < RR; e += blockDim.x) {
            const int a = e / R, b = e % R;
            const int k0 = a > b ? a : b;
            double s = 0.0;
            for (int k = k0; k < R; ++k) s += X[k * R + a] * X[k * R + b];
            W[e] = (float)s;
        }
    } else {
        // Moore-Penrose pseudo-inverse by parallel cyclic Jacobi (round-robin
        // pairing: Re/2 disjoint rotations per step, Re-1 steps per sweep).
        for (int e = t; e < RR; e += blockDim.x) {
            S[e] = V[e];
            X[e] = (e / R == e % R) ? 1.0 : 0.0;
        }
        const int Re = (R + 1) & ~1;
        const int half = Re / 2;
        double *rc = misc + 16;           // cos per pair
        double *rs = rc + half;           // sin per pair
        int *rp = reinterpret_cast<int *>(rs + half);  // p per pair
        int *rq = rp + half;                            // q per pair
        __syncthreads();
        for (int sweep = 0; sweep < 60; ++sweep) {
            double off = 0.0, tot = 0.0;
            for (int e = t; e < RR; e += blockDim.x) {
                const double v = S[e] * S[e];
                tot += v;
                if (e / R != e % R) off += v;
            }
            off = block_sum_d(off, misc + 2);
            tot = block_sum_d(tot, misc + 2);
            if (off == 0.0 || off <= 1e-30 * tot) break;
            for (int step = 0; step < Re - 1; ++step) {
                for (int i = t; i < half; i += blockDim.x) {
                    const int pa = i, pb = Re - 1 - i;
                    const int p0 = pa == 0 ? 0 : ((pa - 1 + step) % (Re - 1)) + 1;
                    const int q0 = pb == 0 ? 0 : ((pb - 1 + step) % (Re - 1)) + 1;
                    const int p = p0 < q0 ? p0 : q0, q = p0 < q0 ? q0 : p0;
                    double c = 1.0, s = 0.0;
                    if (q < R) {
                        const double apq = S[p * R + q];
                        if (apq != 0.0) {
                            const double theta = (S[q * R + q] - S[p * R + p]) / (2.0 * apq);
                            const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                            c = 1.0 / sqrt(tt * tt + 1.0);
                            s = tt * c;
                        }
                    }
                    rc[i] = c;
                    rs[i] = s;
                    rp[i] = p;
                    rq[i] = q < R ? q : -1;
                }
                __syncthreads();
                for (int e = t; e < R * half; e += blockDim.x) {  // S <- S J
                    const int i = e / R, k = e % R;
                    if (rq[i] < 0 || rs[i] == 0.0) continue;
                    const int p = rp[i], q = rq[i];
                    const double c = rc[i], s = rs[i];
                    const double skp = S[k * R + p], skq = S[k * R + q];
                    S[k * R + p] = c * skp - s * skq;
                    S[k * R + q] = s * skp + c * skq;
                }
                __syncthreads();
                for (int e = t; e < R * half; e += blockDim.x) {  // S <- J^T S, Q <- Q J
                    const int i = e / R, k = e % R;
                    if (rq[i] < 0 || rs[i] == 0.0) continue;
                    const int p = rp[i], q = rq[i];
                    const double c = rc[i], s = rs[i];
                    const double spk = S[p * R + k], sqk = S[q * R + k];
                    S[p * R + k] = c * spk - s * sqk;
                    S[q * R + k] = s * spk + c * sqk;
                    const double qkp = X[k * R + p], qkq = X[k * R + q];
                    X[k * R + p] = c * qkp - s * qkq;
                    X[k * R + q] = s * qkp + c * qkq;
                }
                __syncthreads();
            }
        }
        if (t == 0) {
            double wmax = 0.0;
            for (int i = 0; i < R; ++i) wmax = fmax(wmax, fabs(S[i * R + i]));
            misc[0] = (double)R * 2.220446049250313e-16 * wmax;
        }
        __syncthreads();
        const double cut = misc[0];
        for (int e = t; e < RR; e += blockDim.x) {
            const int a = e / R, b = e % R;
            double s = 0.0;
            for (int k = 0; k < R; ++k) {
                const double w = S[k * R + k];
                if (fabs(w) > cut) s += X[a * R + k] * X[b * R + k] / w;
            }
            W[e] = (float)s;
        }
    }
    if (t == 0) {
        if (!pd) branch[0] += 1;
        branch[1] += 1;
    }
}

// lambda_r = sqrt(Gun_rr); G_n = D^-1 Gun D^-1; inner = sum of column dots.
__device__ __noinline__ void finalize_body(const double *__restrict__ gun, int rank, double *__restrict__ Gn,
                                           double *__restrict__ lambda, float *__restrict__ inv_lambda,
                                           double *__restrict__ inner) {
    __shared__ double inv[SPTT_MAX_RANK_ALS];
    __shared__ double red[32];
    const int t = threadIdx.x;
    if (t < rank) {
        const double d = gun[t * rank + t];
        const double l = d > 0.0 ? sqrt(d) : 0.0;
        lambda[t] = l;
        inv[t] = l > 0.0 ? 1.0 / l : 0.0;
        inv_lambda[t] = (float)inv[t];
    }
    __syncthreads();
    for (int e = t; e < rank * rank; e += blockDim.x) {
        const int a = e / rank, b = e % rank;
        Gn[e] = gun[e] * inv[a] * inv[b];
    }
    double d = (t < rank) ? gun[rank * rank + t] : 0.0;
    d = block_sum_d(d, red);
    if (t == 0) *inner = d;
}

}  // namespace
}  // namespace dense
}  // namespace sptt
