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
