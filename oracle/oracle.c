/*
 * FP64 CPU oracle for sparse CP-ALS over COO (test infrastructure only).
 *
 * This file is the reference the CUDA path is checked against. Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never links or calls it, and the two share no code.
 *
 * Everything follows "Parallel Sparse Tensor Decomposition in Chapel"
 * (Rolinger, Simon, Krieger; arXiv:1812.05961), Section III and Algorithm 1,
 * generalised from 3 modes to N modes as the paper states CP-ALS allows.
 * Arithmetic is IEEE FP64 throughout (the paper does not fix a precision).
 * Loops are written in the most literal order; nothing is blocked or fused.
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *  - initial factors: U(0,1) from a Philox4x64-10 stream (key = (seed, mode),
 *    counter = (e/4, 0, 0, 0), word e%4, e = row*rank + col);
 *  - duplicate coordinates are summed (coalesced) in input order;
 *  - the column normalisation uses the 2-norm every iteration; a zero column keeps
 *    lambda = 0 and is left at zero;
 *  - V^dagger is applied through a Cholesky factorisation (Section V-A: potrf /
 *    potrs); when V is not positive definite (a pivot <= 1e-14 * max diag) the
 *    Moore-Penrose pseudo-inverse from a symmetric eigendecomposition is used,
 *    eigenvalues below n * eps * max|eig| treated as zero;
 *  - the fit is computed once per iteration after the last mode, as
 *    1 - sqrt(max(0, |X|^2 + |Xhat|^2 - 2<X,Xhat>)) / |X|, and iteration stops
 *    when |fit - fit_prev| < tol (Algorithm 1 stops once the fit no longer improves).
 *
 * Parity pins: every function here is pinned in tests/test_oracle_*.py against
 * brute force (dense unfolding times explicit Khatri-Rao), closed forms,
 * invariants and independent library routines. None is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 counter-based generator, from its published definition     */
/* (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,  */
/* 3", SC'11): 10 rounds of two 64x64->128 multiplies with the constants    */
/* M0 = 0xD2E7470EE14C6C93, M1 = 0xCA5A826395121157 and Weyl key increments */
/* W0 = 0x9E3779B97F4A7C15, W1 = 0xBB67AE8584CAA73B.                        */
/* ------------------------------------------------------------------------ */

static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mul128(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mul128(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A 64-bit word to a uniform in (0,1): the top 23 bits m give (2m+1)/2^24,
 * which is exact in both FP32 and FP64. */
static double unit_from_word(uint64_t x) {
    uint64_t m = x >> 41;
    return ((double)m + 0.5) * (1.0 / 8388608.0);
}

/* Initial factor for one mode: A[row*rank + col] ~ U(0,1) (Algorithm 1,
 * "initialize A^(n)"). */
void oracle_init_factor(uint64_t seed, int32_t mode, int64_t rows, int32_t rank, double *A) {
    uint64_t key[2] = {seed, (uint64_t)mode};
    for (int64_t e = 0; e < rows * (int64_t)rank; ++e) {
        uint64_t ctr[4] = {(uint64_t)(e / 4), 0, 0, 0};
        uint64_t w[4];
        oracle_philox4x64(ctr, key, w);
        A[e] = unit_from_word(w[e % 4]);
    }
}

/* ------------------------------------------------------------------------ */
/* Pre-processing: sort non-zeros and coalesce duplicates (Section V-C,     */
/* "Sort"), then build the compressed sparse fiber levels (Section III).    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t nmodes;
    const int32_t *const *inds;
    const int32_t *order;
} cmp_ctx;

/* Lexicographic compare of non-zeros a and b in level order. */
static int coord_cmp(const cmp_ctx *c, int64_t a, int64_t b) {
    for (int l = 0; l < c->nmodes; ++l) {
        int32_t m = c->order[l];
        int32_t x = c->inds[m][a], y = c->inds[m][b];
        if (x < y) return -1;
        if (x > y) return 1;
    }
    return 0;
}

/* Stable top-down merge sort of a permutation. */
static void merge_sort(const cmp_ctx *c, int64_t *perm, int64_t *tmp, int64_t n) {
    if (n < 2) return;
    int64_t h = n / 2;
    merge_sort(c, perm, tmp, h);
    merge_sort(c, perm + h, tmp, n - h);
    int64_t i = 0, j = h, k = 0;
    while (i < h && j < n) {
        if (coord_cmp(c, perm[j], perm[i]) < 0) tmp[k++] = perm[j++];
        else tmp[k++] = perm[i++];
    }
    while (i < h) tmp[k++] = perm[i++];
    while (j < n) tmp[k++] = perm[j++];
    memcpy(perm, tmp, (size_t)n * sizeof(int64_t));
}

/*
 * Sort the non-zeros lexicographically by (inds[order[0]], ..., inds[order[N-1]])
 * and sum duplicate coordinates. The sum of a duplicate group is taken in
 * FP64 in input order and rounded once to FP32.
 * out_inds[m] (capacity nnz) receive mode m's indices in sorted order.
 * Returns the number of distinct coordinates, or -1 on an index out of range.
 */
int64_t oracle_coalesce(int32_t nmodes, int64_t nnz, const int64_t *dims,
                        const int32_t *const *inds, const float *vals,
                        const int32_t *order, int32_t *const *out_inds, float *out_vals) {
    for (int m = 0; m < nmodes; ++m)
        for (int64_t k = 0; k < nnz; ++k)
            if (inds[m][k] < 0 || (int64_t)inds[m][k] >= dims[m]) return -1;
    if (nnz == 0) return 0;
    int64_t *perm = (int64_t *)malloc((size_t)nnz * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)nnz * sizeof(int64_t));
    for (int64_t k = 0; k < nnz; ++k) perm[k] = k;
    cmp_ctx c = {nmodes, inds, order};
    merge_sort(&c, perm, tmp, nnz);
    int64_t u = 0;
    int64_t k = 0;
    while (k < nnz) {
        int64_t first = perm[k];
        double sum = 0.0;
        int64_t j = k;
        while (j < nnz && coord_cmp(&c, perm[j], first) == 0) {
            sum += (double)vals[perm[j]];
            ++j;
        }
        for (int m = 0; m < nmodes; ++m) out_inds[m][u] = inds[m][first];
        out_vals[u] = (float)sum;
        ++u;
        k = j;
    }
    free(perm);
    free(tmp);
    return u;
}

/*
 * CSF levels from coalesced, sorted non-zeros (Section III). Level l holds the
 * distinct prefixes (i_{order[0]}, ..., i_{order[l]}); a new level-l fiber
 * starts wherever that prefix changes. For l < N-1:
 *   fids[l][f]  = i_{order[l]} of fiber f,
 *   fptr[l][f]  = index of fiber f's first child at level l+1,
 *   fptr[l][nfibs[l]] = nfibs[l+1].
 * The leaf level is fids[N-1][k] = i_{order[N-1]} of non-zero k.
 * Capacities: fids[l] >= nnz, fptr[l] >= nnz + 1.
 */
void oracle_csf(int32_t nmodes, int64_t nnz, const int32_t *const *sorted_inds,
                const int32_t *order, int64_t *nfibs, int32_t *const *fptr,
                int32_t *const *fids) {
    /* fiber id at every level for every non-zero, built top-down */
    int64_t *count = (int64_t *)calloc((size_t)nmodes, sizeof(int64_t));
    for (int64_t k = 0; k < nnz; ++k) {
        /* the first level at which this non-zero's prefix differs */
        int first_new = nmodes - 1;
        if (k == 0) {
            first_new = 0;
        } else {
            for (int l = 0; l < nmodes; ++l) {
                int32_t m = order[l];
                if (sorted_inds[m][k] != sorted_inds[m][k - 1]) {
                    first_new = l;
                    break;
                }
            }
        }
        for (int l = first_new; l < nmodes; ++l) {
            int32_t m = order[l];
            int64_t f = count[l];
            fids[l][f] = sorted_inds[m][k];
            if (l < nmodes - 1) fptr[l][f] = (int32_t)count[l + 1];
            count[l] = f + 1;
        }
    }
    for (int l = 0; l < nmodes; ++l) nfibs[l] = count[l];
    for (int l = 0; l < nmodes - 1; ++l) fptr[l][count[l]] = (int32_t)count[l + 1];
    free(count);
}

/* ------------------------------------------------------------------------ */
/* MTTKRP (Section III): M = X_(n) (Khatri-Rao of A^(m), m != n), by its    */
/* element definition M[i_n, r] += v * prod_{m != n} A^(m)[i_m, r].         */
/* ------------------------------------------------------------------------ */

/*
 * out (dims[mode] x rank, row-major) is overwritten. out_abs, if not NULL,
 * receives the same sum taken over |v| and |A| (the scale used for
 * element-wise tolerances). row_mask, if not NULL, restricts the work to the
 * rows i with row_mask[i] != 0; other rows are left at zero.
 */
/* Threads of the MTTKRP (1 = the literal single-loop order). */
static int32_t g_threads = 1;

/*
 * Set the number of host threads oracle_mttkrp uses (n < 1 means 1) and
 * return the number in effect: 1 when the oracle was compiled without OpenMP.
 */
int32_t oracle_set_threads(int32_t n) {
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* M[i_n, :] += v * prod_{m != n} A^(m)[i_m, :] over non-zeros [k0, k1). */
static void mttkrp_range(int32_t nmodes, int64_t k0, int64_t k1, const int32_t *const *inds,
                         const float *vals, const double *const *factors, int32_t rank, int32_t mode,
                         double *out, double *out_abs, const uint8_t *row_mask) {
    for (int64_t k = k0; k < k1; ++k) {
        int64_t i = inds[mode][k];
        if (row_mask && !row_mask[i]) continue;
        double v = (double)vals[k];
        for (int r = 0; r < rank; ++r) {
            double p = v;
            double pa = fabs(v);
            for (int m = 0; m < nmodes; ++m) {
                if (m == mode) continue;
                double a = factors[m][(int64_t)inds[m][k] * rank + r];
                p *= a;
                pa *= fabs(a);
            }
            out[i * rank + r] += p;
            if (out_abs) out_abs[i * rank + r] += pa;
        }
    }
}

void oracle_mttkrp(int32_t nmodes, int64_t nnz, const int64_t *dims,
                   const int32_t *const *inds, const float *vals,
                   const double *const *factors, int32_t rank, int32_t mode,
                   double *out, double *out_abs, const uint8_t *row_mask) {
    int64_t rows = dims[mode];
    size_t cells = (size_t)(rows * rank);
    memset(out, 0, cells * sizeof(double));
    if (out_abs) memset(out_abs, 0, cells * sizeof(double));
#ifdef _OPENMP
    /*
     * With T > 1 threads: thread t sums non-zeros [nnz*t/T, nnz*(t+1)/T) into
     * its own zeroed copy of M, and the copies are added in thread order.
     * Only the FP64 summation order differs from the single loop.
     */
    int32_t T = g_threads;
    if (T > 1 && nnz >= 4096) {
        size_t per = cells * (out_abs ? 2 : 1);
        double *priv = (double *)calloc((size_t)T * per, sizeof(double));
        if (priv) {
#pragma omp parallel num_threads(T)
            {
                int t = omp_get_thread_num();
                double *mine = priv + (size_t)t * per;
                mttkrp_range(nmodes, nnz * t / T, nnz * (t + 1) / T, inds, vals, factors, rank, mode, mine,
                             out_abs ? mine + cells : NULL, row_mask);
            }
#pragma omp parallel for num_threads(T) schedule(static)
            for (int64_t e = 0; e < (int64_t)cells; ++e) {
                double s = 0.0, sa = 0.0;
                for (int t = 0; t < T; ++t) {
                    s += priv[(size_t)t * per + e];
                    if (out_abs) sa += priv[(size_t)t * per + cells + e];
                }
                out[e] = s;
                if (out_abs) out_abs[e] = sa;
            }
            free(priv);
            return;
        }
    }
#endif
    mttkrp_range(nmodes, 0, nnz, inds, vals, factors, rank, mode, out, out_abs, row_mask);
}

/* ------------------------------------------------------------------------ */
/* Dense R x R algebra of Algorithm 1.                                      */
/* ------------------------------------------------------------------------ */

/* G = A^T A (Algorithm 1, "A^(m)T A^(m)"), A rows x rank row-major. */
void oracle_gram(int64_t rows, int32_t rank, const double *A, double *G) {
    /* entries are independent; each keeps the row order of its sum */
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1) schedule(static)
    for (int a = 0; a < rank; ++a)
        for (int b = 0; b < rank; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < rows; ++i) s += A[i * rank + a] * A[i * rank + b];
            G[a * rank + b] = s;
        }
}

/*
 * Cholesky V = L L^T (lower L, row-major n x n). Returns 0 when every pivot
 * is above 1e-14 * max diag(V) (the positive-definite test), else -1.
 */
int oracle_cholesky(int32_t n, const double *V, double *L) {
    double dmax = 0.0;
    for (int i = 0; i < n; ++i)
        if (V[i * n + i] > dmax) dmax = V[i * n + i];
    double thresh = 1e-14 * dmax;
    memset(L, 0, (size_t)n * n * sizeof(double));
    for (int j = 0; j < n; ++j) {
        double d = V[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > thresh)) return -1;
        double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = V[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
    return 0;
}

/*
 * Symmetric eigendecomposition by cyclic Jacobi rotations (Golub & Van Loan,
 * Matrix Computations, Sec. 8.5): V = Q diag(w) Q^T. Q row-major, columns are
 * eigenvectors.
 */
void oracle_sym_eig(int32_t n, const double *V, double *w, double *Q) {
    double *S = (double *)malloc((size_t)n * n * sizeof(double));
    memcpy(S, V, (size_t)n * n * sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Q[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += S[i * n + j] * S[i * n + j];
                if (i != j) off += S[i * n + j] * S[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = S[p * n + q];
                if (apq == 0.0) continue;
                double app = S[p * n + p], aqq = S[q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* S <- S J (columns p, q) */
                    double skp = S[k * n + p], skq = S[k * n + q];
                    S[k * n + p] = c * skp - s * skq;
                    S[k * n + q] = s * skp + c * skq;
                }
                for (int k = 0; k < n; ++k) { /* S <- J^T S (rows p, q) */
                    double spk = S[p * n + k], sqk = S[q * n + k];
                    S[p * n + k] = c * spk - s * sqk;
                    S[q * n + k] = s * spk + c * sqk;
                }
                for (int k = 0; k < n; ++k) { /* Q <- Q J */
                    double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - s * qkq;
                    Q[k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = S[i * n + i];
    free(S);
}

/* Moore-Penrose pseudo-inverse of symmetric V through its eigenvalues:
 * eigenvalues with |w| <= n * eps * max|w| are treated as zero. */
void oracle_pinv_sym(int32_t n, const double *V, double *P) {
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *Q = (double *)malloc((size_t)n * n * sizeof(double));
    oracle_sym_eig(n, V, w, Q);
    double wmax = 0.0;
    for (int i = 0; i < n; ++i)
        if (fabs(w[i]) > wmax) wmax = fabs(w[i]);
    double cut = (double)n * 2.220446049250313e-16 * wmax;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k)
                if (fabs(w[k]) > cut) s += Q[i * n + k] * Q[j * n + k] / w[k];
            P[i * n + j] = s;
        }
    free(w);
    free(Q);
}

/*
 * Row-wise normal-equation solve A = M V^dagger (Algorithm 1, the solve of each mode update),
 * in place on M (rows x n). Through Cholesky (forward then back substitution
 * per row) when V is positive definite, else through the pseudo-inverse.
 * Returns 0 on the Cholesky branch, 1 on the pseudo-inverse branch.
 */
int oracle_solve_normals(int64_t rows, int32_t n, const double *V, double *M) {
    double *L = (double *)malloc((size_t)n * n * sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    int branch;
    /* rows are independent: with several threads each takes a block of
       rows and its own y, and every row's arithmetic is unchanged */
    if (oracle_cholesky(n, V, L) == 0) {
        branch = 0;
#pragma omp parallel num_threads(g_threads) if (g_threads > 1)
        {
            double *yt = g_threads > 1 ? (double *)malloc((size_t)n * sizeof(double)) : y;
#pragma omp for schedule(static)
            for (int64_t i = 0; i < rows; ++i) {
                double *m = M + i * n;
                /* V x = m, i.e. L y = m then L^T x = y (V symmetric, so x^T = m^T V^-1) */
                for (int a = 0; a < n; ++a) {
                    double s = m[a];
                    for (int b = 0; b < a; ++b) s -= L[a * n + b] * yt[b];
                    yt[a] = s / L[a * n + a];
                }
                for (int a = n - 1; a >= 0; --a) {
                    double s = yt[a];
                    for (int b = a + 1; b < n; ++b) s -= L[b * n + a] * m[b];
                    m[a] = s / L[a * n + a];
                }
            }
            if (yt != y) free(yt);
        }
    } else {
        branch = 1;
        double *P = (double *)malloc((size_t)n * n * sizeof(double));
        oracle_pinv_sym(n, V, P);
#pragma omp parallel num_threads(g_threads) if (g_threads > 1)
        {
            double *yt = g_threads > 1 ? (double *)malloc((size_t)n * sizeof(double)) : y;
#pragma omp for schedule(static)
            for (int64_t i = 0; i < rows; ++i) {
                double *m = M + i * n;
                for (int a = 0; a < n; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < n; ++b) s += m[b] * P[b * n + a];
                    yt[a] = s;
                }
                memcpy(m, yt, (size_t)n * sizeof(double));
            }
            if (yt != y) free(yt);
        }
        free(P);
    }
    free(L);
    free(y);
    return branch;
}

/* Normalise the columns of A (rows x rank) by their 2-norms, stored in lambda
 * (Algorithm 1 scales each column to unit norm and keeps the norms as lambda). */
void oracle_normalize(int64_t rows, int32_t rank, double *A, double *lambda) {
    /* columns are independent; each keeps the row order of its sum */
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1) schedule(static)
    for (int r = 0; r < rank; ++r) {
        double s = 0.0;
        for (int64_t i = 0; i < rows; ++i) s += A[i * rank + r] * A[i * rank + r];
        double nrm = sqrt(s);
        lambda[r] = nrm;
        if (nrm > 0.0)
            for (int64_t i = 0; i < rows; ++i) A[i * rank + r] /= nrm;
    }
}

/*
 * Fit of the model (Algorithm 1 checks it once per iteration):
 *   |X - Xhat|^2 = |X|^2 + lambda^T (*_m G_m) lambda - 2 sum_r lambda_r sum_i M[i,r] A[i,r]
 * where G_m are the Grams of the (normalised) factors, M is the MTTKRP of the
 * last-updated mode n and A its normalised factor. Returns 1 - |X - Xhat| / |X|
 * (1 when |X| = 0 and the residual is 0).
 */
double oracle_fit(int32_t nmodes, int32_t rank, double normx_sq, const double *const *grams,
                  const double *lambda, int64_t rows_n, const double *M, const double *A) {
    double model = 0.0;
    for (int a = 0; a < rank; ++a)
        for (int b = 0; b < rank; ++b) {
            double h = 1.0;
            for (int m = 0; m < nmodes; ++m) h *= grams[m][a * rank + b];
            model += lambda[a] * lambda[b] * h;
        }
    double inner = 0.0;
    for (int r = 0; r < rank; ++r) {
        double s = 0.0;
        for (int64_t i = 0; i < rows_n; ++i) s += M[i * rank + r] * A[i * rank + r];
        inner += lambda[r] * s;
    }
    double resid_sq = normx_sq + model - 2.0 * inner;
    if (resid_sq < 0.0) resid_sq = 0.0;
    if (normx_sq == 0.0) return resid_sq == 0.0 ? 1.0 : 0.0;
    return 1.0 - sqrt(resid_sq) / sqrt(normx_sq);
}

/*
 * One factor update of Algorithm 1 for mode n (the first three steps of the loop body for n = 1):
 *   V = Hadamard of G_m over m != n;  A^(n) = MTTKRP_n V^dagger;  normalise;
 *   G_n = A^(n)T A^(n).
 * factors[n] (dims[n] x rank) and grams[n] are overwritten; lambda receives
 * the column norms. If M_out is not NULL it receives the MTTKRP (for the fit).
 * Returns the solve branch (0 Cholesky, 1 pseudo-inverse).
 */
int oracle_als_mode_update(int32_t nmodes, int64_t nnz, const int64_t *dims,
                           const int32_t *const *inds, const float *vals, int32_t rank,
                           int32_t n, double *const *factors, double *const *grams,
                           double *lambda, double *M_out) {
    int64_t rows = dims[n];
    double *M = (double *)malloc((size_t)(rows * rank) * sizeof(double));
    double *V = (double *)malloc((size_t)rank * rank * sizeof(double));
    oracle_mttkrp(nmodes, nnz, dims, inds, vals, (const double *const *)factors, rank, n, M,
                  NULL, NULL);
    if (M_out) memcpy(M_out, M, (size_t)(rows * rank) * sizeof(double));
    for (int a = 0; a < rank * rank; ++a) {
        double h = 1.0;
        for (int m = 0; m < nmodes; ++m)
            if (m != n) h *= grams[m][a];
        V[a] = h;
    }
    int branch = oracle_solve_normals(rows, rank, V, M);
    oracle_normalize(rows, rank, M, lambda);
    memcpy(factors[n], M, (size_t)(rows * rank) * sizeof(double));
    oracle_gram(rows, rank, factors[n], grams[n]);
    free(M);
    free(V);
    return branch;
}

/*
 * CP-ALS (Algorithm 1) for N modes over a coalesced COO tensor.
 * factors[m] (dims[m] x rank) hold the initial factors on entry (the caller
 * fills them, e.g. with oracle_init_factor) and the result on exit.
 * fit_history (capacity max_iters) receives the fit after each iteration.
 * Returns the number of iterations run.
 */
int32_t oracle_cpd_als(int32_t nmodes, int64_t nnz, const int64_t *dims,
                       const int32_t *const *inds, const float *vals, int32_t rank,
                       int32_t max_iters, double tol, double *const *factors, double *lambda,
                       double *fit_history) {
    double **grams = (double **)malloc((size_t)nmodes * sizeof(double *));
    for (int m = 0; m < nmodes; ++m) {
        grams[m] = (double *)malloc((size_t)rank * rank * sizeof(double));
        oracle_gram(dims[m], rank, factors[m], grams[m]);
    }
    double normx_sq = 0.0;
    for (int64_t k = 0; k < nnz; ++k) normx_sq += (double)vals[k] * (double)vals[k];
    int last = nmodes - 1;
    double *M_last = (double *)malloc((size_t)(dims[last] * rank) * sizeof(double));
    double fit_prev = 0.0;
    int32_t it;
    for (it = 0; it < max_iters; ++it) {
        for (int n = 0; n < nmodes; ++n)
            oracle_als_mode_update(nmodes, nnz, dims, inds, vals, rank, n, factors, grams,
                                   lambda, n == last ? M_last : NULL);
        double fit = oracle_fit(nmodes, rank, normx_sq, (const double *const *)grams, lambda,
                                dims[last], M_last, factors[last]);
        fit_history[it] = fit;
        if (it > 0 && fabs(fit - fit_prev) < tol) {
            ++it;
            break;
        }
        fit_prev = fit;
    }
    for (int m = 0; m < nmodes; ++m) free(grams[m]);
    free(grams);
    free(M_last);
    return it;
}

/* ------------------------------------------------------------------------ */
/* The scheduler's MLP, FP64 reference (the learned scheduler is not in the */
/* paper; this is the reference its GPU training kernels are checked with). */
/* in -> h (ReLU) -> h (ReLU) -> out, parameters packed as                   */
/* W1[h][in], b1[h], W2[h][h], b2[h], W3[out][h], b3[out] (row-major).       */
/* ------------------------------------------------------------------------ */

static void mlp_layer(const double *W, const double *b, const double *x, int nin, int nout, int relu,
                      double *pre, double *y) {
    for (int o = 0; o < nout; ++o) {
        double s = b[o];
        for (int i = 0; i < nin; ++i) s += W[o * nin + i] * x[i];
        if (pre) pre[o] = s;
        y[o] = (relu && s < 0.0) ? 0.0 : s;
    }
}

/* y[n][nout] = MLP(x[n][nin]) */
void oracle_mlp_forward(int32_t nin, int32_t nh, int32_t nout, const double *P, int64_t n, const double *x,
                        double *y) {
    const double *W1 = P, *b1 = W1 + nh * nin, *W2 = b1 + nh, *b2 = W2 + nh * nh, *W3 = b2 + nh,
                 *b3 = W3 + nout * nh;
    double *h1 = (double *)malloc((size_t)nh * sizeof(double));
    double *h2 = (double *)malloc((size_t)nh * sizeof(double));
    for (int64_t s = 0; s < n; ++s) {
        mlp_layer(W1, b1, x + s * nin, nin, nh, 1, NULL, h1);
        mlp_layer(W2, b2, h1, nh, nh, 1, NULL, h2);
        mlp_layer(W3, b3, h2, nh, nout, 0, NULL, y + s * nout);
    }
    free(h1);
    free(h2);
}

/*
 * Loss L = 1/(n*nout) * sum (y - t)^2 over the batch and its gradient with
 * respect to every parameter (back-propagation), into G (same layout as P).
 * Returns L.
 */
double oracle_mlp_loss_grad(int32_t nin, int32_t nh, int32_t nout, const double *P, int64_t n, const double *x,
                            const double *t, double *G) {
    const int np = nh * nin + nh + nh * nh + nh + nout * nh + nout;
    const double *W1 = P, *b1 = W1 + nh * nin, *W2 = b1 + nh, *b2 = W2 + nh * nh, *W3 = b2 + nh,
                 *b3 = W3 + nout * nh;
    double *gW1 = G, *gb1 = gW1 + nh * nin, *gW2 = gb1 + nh, *gb2 = gW2 + nh * nh, *gW3 = gb2 + nh,
           *gb3 = gW3 + nout * nh;
    memset(G, 0, (size_t)np * sizeof(double));
    double *p1 = (double *)malloc((size_t)nh * sizeof(double)), *h1 = (double *)malloc((size_t)nh * sizeof(double));
    double *p2 = (double *)malloc((size_t)nh * sizeof(double)), *h2 = (double *)malloc((size_t)nh * sizeof(double));
    double *y = (double *)malloc((size_t)nout * sizeof(double)), *dy = (double *)malloc((size_t)nout * sizeof(double));
    double *d2 = (double *)malloc((size_t)nh * sizeof(double)), *d1 = (double *)malloc((size_t)nh * sizeof(double));
    const double scale = 1.0 / ((double)n * nout);
    double loss = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        const double *xs = x + s * nin, *ts = t + s * nout;
        mlp_layer(W1, b1, xs, nin, nh, 1, p1, h1);
        mlp_layer(W2, b2, h1, nh, nh, 1, p2, h2);
        mlp_layer(W3, b3, h2, nh, nout, 0, NULL, y);
        for (int o = 0; o < nout; ++o) {
            const double e = y[o] - ts[o];
            loss += e * e * scale;
            dy[o] = 2.0 * e * scale;
        }
        for (int o = 0; o < nout; ++o) {
            gb3[o] += dy[o];
            for (int j = 0; j < nh; ++j) gW3[o * nh + j] += dy[o] * h2[j];
        }
        for (int j = 0; j < nh; ++j) {
            double s2 = 0.0;
            for (int o = 0; o < nout; ++o) s2 += dy[o] * W3[o * nh + j];
            d2[j] = p2[j] > 0.0 ? s2 : 0.0;
        }
        for (int j = 0; j < nh; ++j) {
            gb2[j] += d2[j];
            for (int i = 0; i < nh; ++i) gW2[j * nh + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < nh; ++i) {
            double s1 = 0.0;
            for (int j = 0; j < nh; ++j) s1 += d2[j] * W2[j * nh + i];
            d1[i] = p1[i] > 0.0 ? s1 : 0.0;
        }
        for (int i = 0; i < nh; ++i) {
            gb1[i] += d1[i];
            for (int k = 0; k < nin; ++k) gW1[i * nin + k] += d1[i] * xs[k];
        }
    }
    free(p1); free(h1); free(p2); free(h2); free(y); free(dy); free(d2); free(d1);
    return loss;
}
