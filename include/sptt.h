/*
 * sptt — sparse CP-ALS on one GB300 GPU (sm_103a). C ABI.
 *
 * The method is CP-ALS over a tensor stored in compressed sparse fiber (CSF)
 * form, as studied in "Parallel Sparse Tensor Decomposition in Chapel"
 * (Rolinger, Simon, Krieger; arXiv:1812.05961): Section III (CP-ALS, MTTKRP,
 * CSF), Algorithm 1 (the ALS loop), Section V-A (V^dagger through
 * potrf/potrs), Section V-C (the non-zero sort).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an sptt_status: SPTT_OK (0) or a negative error.
 *    No exception, abort or exit crosses this boundary. A human-readable
 *    detail of the last error on the calling thread is sptt_last_error().
 *  - Input arrays are borrowed for the duration of the call only.
 *  - Handles (sptt_csf, sptt_cpd) are owned by the library and released by
 *    their *_free function; caller-owned output buffers stay caller-owned.
 *  - "device" pointers are CUDA device (or managed) memory of the current
 *    device; "host or device" pointers may be either (unified addressing
 *    decides the copy direction).
 *  - Work is enqueued on the given stream (NULL = the legacy default
 *    stream). Functions that must read a result back (sizes, error flags,
 *    fits) synchronise that stream and say so.
 *  - Indices are 0-based int32; dims are int64 but each must be <= 2^31 - 1;
 *    nnz must be < 2^31. 2 <= nmodes <= SPTT_MAX_MODES.
 *  - There is no CPU fallback: without a usable CUDA device every compute
 *    entry point returns SPTT_ERR_CUDA.
 */
#ifndef SPTT_H
#define SPTT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sptt_stream; /* a cudaStream_t */
typedef int32_t sptt_status;

#define SPTT_OK 0
#define SPTT_ERR_BAD_ARG (-1)     /* invalid argument: sizes, null pointers, index >= dim */
#define SPTT_ERR_OOM (-2)         /* a device allocation failed */
#define SPTT_ERR_CUDA (-3)        /* a CUDA runtime call or kernel failed */
#define SPTT_ERR_TIMEOUT (-4)     /* a bounded device-side wait ran out */
#define SPTT_ERR_NOT_PD (-5)      /* reported by sptt_cpd_solve_branch only (not an error) */
#define SPTT_ERR_UNSUPPORTED (-6) /* valid but outside the library's limits (e.g. rank > 64) */
#define SPTT_ERR_INTERNAL (-7)

#define SPTT_MAX_MODES 5
#define SPTT_MAX_RANK_ALS 64      /* rank limit of the CP-ALS entry points */

/* Factor element types for MTTKRP gathers. */
#define SPTT_F32 0
#define SPTT_BF16 1

/* Readable name of a status code (static string). */
const char *sptt_status_str(sptt_status s);
/* Detail of the last error raised on this thread ("" if none). */
const char *sptt_last_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int32_t sptt_version(void);

/*
 * A coordinate-format (COO) tensor, borrowed by every call that takes it.
 *   nmodes      number of modes N (2..SPTT_MAX_MODES)
 *   nnz         number of stored entries (may include duplicate coordinates,
 *               which are summed, Section V-C "Sort")
 *   dims        host array [nmodes], mode lengths I_m
 *   inds        host array of nmodes pointers; inds[m] points to nnz int32
 *               indices of mode m (device memory if on_device, else host)
 *   vals        nnz float values (device if on_device, else host)
 *   on_device   1: inds[m] and vals are device pointers; 0: host pointers
 *               (copied to the device inside the call)
 */
typedef struct {
    int32_t nmodes;
    int64_t nnz;
    const int64_t *dims;
    const int32_t *const *inds;
    const float *vals;
    int32_t on_device;
} sptt_coo;

/* ------------------------------------------------------------------------ */
/* CSF (Section III): one tree per root mode.                               */
/* ------------------------------------------------------------------------ */

typedef struct sptt_csf sptt_csf;

/*
 * Build the CSF of a COO tensor rooted at root_mode (Section III), after
 * sorting its non-zeros lexicographically in level order and summing
 * duplicates (Section V-C). level_order (host, nmodes entries, NULL = default)
 * is the mode stored at each tree level and must start with root_mode; the
 * default is root_mode followed by the other modes in ascending length, ties
 * to the lower mode id. The result lives in device memory and is identical,
 * integer for integer, to the plain construction:
 *   level l < N-1: fids[l][f] = index of fiber f, fptr[l][f] = its first child
 *   at level l+1, fptr[l][nfibs[l]] = nfibs[l+1];
 *   leaf level N-1: fids[N-1][k] and vals[k] per coalesced non-zero, where a
 *   duplicate group's value is its FP64 sum in input order rounded to FP32.
 * Errors: BAD_ARG (bad sizes/pointers, an index outside [0, dim), bad
 * order), OOM, CUDA. Synchronises the stream (it reads back sizes).
 */
sptt_status sptt_csf_build(const sptt_coo *coo, int32_t root_mode, const int32_t *level_order,
                           sptt_stream stream, sptt_csf **out);

/* Release a CSF (NULL is ignored). The caller ensures no work using it is
 * still pending. */
void sptt_csf_free(sptt_csf *csf);

/*
 * Shape of a CSF: nmodes, the level order (order[l] = mode at level l) and
 * nfibs[l] (fibers at level l; nfibs[N-1] = coalesced nnz). Output arrays are
 * host, nmodes entries each; any may be NULL.
 */
sptt_status sptt_csf_shape(const sptt_csf *csf, int32_t *nmodes, int32_t *order, int64_t *nfibs);

/* Synchronise the stream and report whether a kernel that read this CSF
 * gave up a bounded wait (SPTT_ERR_TIMEOUT; the word is then cleared). */
sptt_status sptt_csf_check(const sptt_csf *csf, sptt_stream stream);

/*
 * Copy level l of a CSF into caller buffers (host or device; any may be
 * NULL): fptr (nfibs[l]+1 int32, only for l < N-1), fids (nfibs[l] int32),
 * vals (nfibs[N-1] float, only for l = N-1). Synchronises the stream.
 */
sptt_status sptt_csf_copy_level(const sptt_csf *csf, int32_t level, int32_t *fptr, int32_t *fids,
                                float *vals, sptt_stream stream);

/* ------------------------------------------------------------------------ */
/* MTTKRP (Section III; the MTTKRP step of Algorithm 1).                    */
/* ------------------------------------------------------------------------ */

/*
 * Optional schedule for the MTTKRP kernels (the autotuner's knobs).
 *   chunk       non-zeros per work unit of a lane group; power of two in
 *               [16, 4096]; 0 = default (128, halved down to 32 while the
 *               tensor gives fewer than 128 chunks per SM)
 *   block       threads per CTA (multiple of 32, <= 256); 0 = default
 *   variant     kernel variant: 0 = default (the fastest measured for the
 *               gather type and ld); 1 = plain walk (fiber ends from fptr,
 *               one leaf at a time); 2..5 = walk driven by the per-leaf
 *               level flags, (leaves per batch, CTAs per SM, pipelined) =
 *               (8, 1, yes), (4, 3, no), (4, 2, yes), (2, 3, yes); 6 = the
 *               pipelined walk with its leaf records staged in shared memory
 *               by bulk copies (chunk fixed at 64); 7 = flag walk and 8 =
 *               staged walk with 32-byte row segments (one 256-bit gather per
 *               lane, half the lanes per row) and batches of 2 leaves; 7 and
 *               8 need ld * element size and every non-root factor 32-byte
 *               aligned, and otherwise run as variant 3 / 6; 9 = variant 4
 *               reading packed leaf records; 10 / 11 = variant 7 / 9 with
 *               each leaf added straight into its fiber's parent (one more
 *               multiply per leaf, no per-fiber fold; 10 falls back to 3
 *               like 7); 12 / 13 = the select walk on packed records (the
 *               form of 10 whose per-leaf work has no branch: an opening
 *               fiber's row replaces the open one by a select), 32-byte
 *               segments in batches of 2 / 16-byte segments in batches of
 *               4, two CTAs per SM (12 falls back to 13 like 7); 14 / 15 =
 *               the select walk with the whole leaf factor copied into
 *               shared memory once per CTA, 16-byte segments, one CTA of
 *               1024 threads in batches of 2 / 512 threads in batches of 4,
 *               used when that copy is at most 160 KB (else run as 13).
 *               Default: on a 3-mode tensor of at least 2^25 non-zeros
 *               whose leaf factor fits the table, 14 (F32 gathers) / 15
 *               (BF16); else with F32 gathers on a tensor of at least 2^23
 *               non-zeros and ld >= 16, ld % 8 == 0, 12; else 13. Variants 7 and 9..15
 *               (and so the default) read packed
 *               16-byte leaf records that the first call builds (16 bytes
 *               per non-zero on the device, kept with the CSF)
 */
typedef struct {
    int32_t chunk;
    int32_t block;
    int32_t variant;
    int32_t order;  /* CSF level order below the root for CP-ALS plans: 0 = ascending
                       length, 1 = descending, 2 = the shortest mode at the leaves and
                       the others ascending above it; ignored by sptt_mttkrp. CP-ALS
                       without a schedule builds order 2 on a 3-mode tensor of at
                       least 2^25 non-zeros when the shortest mode's factor (in the
                       gather type) fits the shared-memory table of the default
                       kernel (160 KB), else order 0 */
} sptt_sched;

/*
 * M = X_(n) (Khatri-Rao product of A^(m), m != n), n = the CSF's root mode,
 * computed by traversing the CSF tree (Section III):
 *   M[i, c] = sum over non-zeros (i, i_1, ..., v) of v * prod_{m != n} A^(m)[i_m, c].
 *   factors   host array of nmodes device pointers; factors[m] is A^(m),
 *             row-major dims[m] x ld, of factor_dtype (SPTT_F32 or SPTT_BF16);
 *             factors[n] is not read and may be NULL. Rows must be 16-byte
 *             aligned (base 16-byte aligned and ld a multiple of 4 for F32 /
 *             8 for BF16).
 *   ld        row stride in elements and the number of columns computed;
 *             4 <= ld <= 128 (F32) or 8 <= ld <= 256 (BF16). Callers with a
 *             rank below ld pad the extra columns (zero columns give zero
 *             output columns).
 *   out       device float, dims[n] x ld row-major, overwritten (rows absent
 *             from the tensor become 0). Must not alias a factor.
 *   sched     NULL = default schedule.
 * Accumulation is FP32 within a work chunk; a slice split over several
 * chunks sums its chunk partials in FP64 (an FP64 workspace of dims[n] x ld
 * is allocated on the stream and converted into out). Asynchronous on the
 * stream. Errors: BAD_ARG, OOM.
 */
sptt_status sptt_mttkrp(const sptt_csf *csf, const void *const *factors, int32_t factor_dtype,
                        int32_t ld, float *out, const sptt_sched *sched, sptt_stream stream);

/*
 * MTTKRP for any mode n of the tensor from one CSF (Section III; the MTTKRP
 * step of Algorithm 1), the single-CSF form whose output conflicts the paper
 * resolves with a lock pool or privatised copies (Section IV-A, V-D-2).
 * mode = the CSF's root runs sptt_mttkrp. For a mode at tree level L >= 1,
 * each level-L fiber (each leaf when L = N-1) adds the Hadamard product of
 * its ancestors' factor rows times the sum below it to M[fids[L][f], :]:
 * the same M as the element definition of sptt_mttkrp.
 *   factors   as for sptt_mttkrp; factors[n] is not read and may be NULL.
 *   ld, out   as for sptt_mttkrp (out: dims[n] x ld, overwritten).
 *   sched     chunk as for sptt_mttkrp; variant: 0 = default (privatised hot
 *             rows), 1 = every row through global reductions, 2 = privatised
 *             hot rows: the rows with the most contributions (up to 64 KB
 *             of them) are summed per CTA in shared memory and added to out
 *             every few rounds of chunks. order is ignored.
 * Accumulation is FP32 (global and shared-memory atomics, so the summation
 * order varies from run to run). A privatised row is summed in FP32 runs of
 * a few rounds of chunks per CTA; with variant 1 a row's n contributions
 * form one FP32 sum (error about sqrt(n) 2^-24 of the row's scale, so rows
 * with ~10^5 contributions or more miss the 1e-5 bound that the privatised
 * default keeps). The first call for a mode and row width
 * builds the work partition and the hot-row table (allocates and
 * synchronises); later calls are asynchronous. Errors: BAD_ARG, OOM.
 */
sptt_status sptt_mttkrp_mode(const sptt_csf *csf, int32_t mode, const void *const *factors,
                             int32_t factor_dtype, int32_t ld, float *out, const sptt_sched *sched,
                             sptt_stream stream);

/* ------------------------------------------------------------------------ */
/* Dense R x R pieces (the Gram products of Algorithm 1).                   */
/* ------------------------------------------------------------------------ */

/*
 * G = A^T A over the first `rank` columns of A (device, rows x ld row-major
 * FP32, ld >= rank, ld multiple of 4), into G (device, rank x rank FP64,
 * row-major). Products are formed in FP32 and summed in FP32 over 64-row
 * tiles, the tile sums in FP64. A may be NULL when rows = 0 (G = 0).
 * Asynchronous. rank in [1, SPTT_MAX_RANK_ALS] (else SPTT_ERR_UNSUPPORTED).
 */
sptt_status sptt_gram(const float *A, int64_t rows, int32_t rank, int32_t ld, double *G,
                      sptt_stream stream);

/*
 * sptt_gram with no device allocation, for callers that cannot call
 * cudaMalloc: code whose device memory is owned entirely by another
 * allocator (a framework's caching allocator or a fixed arena), or a latency
 * path where an allocation that may synchronise or grow a pool is not
 * acceptable. (The paper has no counterpart; this is an interface variant.)
 * Same arguments and result as sptt_gram. Its workspace is one static device
 * array of 2^18 doubles (2 MiB) that every GPU loading the library holds until
 * the process exits; no cudaMalloc, cudaFree or allocating library routine is
 * called. The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and caches it, so make the first call for each
 * device, with that device current, before any stream capture. All calls
 * share the one array: calls that can overlap on the GPU (different streams
 * without ordering between them) race on it and must be serialised by the
 * caller. rank must be in [1, SPTT_MAX_RANK_ALS] (else SPTT_ERR_UNSUPPORTED,
 * as for sptt_gram). Asynchronous.
 */
sptt_status sptt_gram_noalloc(const float *A, int64_t rows, int32_t rank, int32_t ld, double *G,
                              sptt_stream stream);

/* ------------------------------------------------------------------------ */
/* CP-ALS (Algorithm 1, N modes).                                           */
/* ------------------------------------------------------------------------ */

/*
 * Options of a CP-ALS run (zero-initialise for the defaults).
 *   seed          seed of the U(0,1) Philox4x64-10 initial factors
 *   precision     SPTT_F32: FP32 factor gathers; SPTT_BF16: BF16 gathers
 *                 with FP32 accumulation, followed by refine_iters FP32
 *                 iterations (the FP32 refinement sweep)
 *   refine_iters  FP32 iterations after a BF16 run (default 1 when
 *                 precision = SPTT_BF16; ignored for F32)
 *   use_graph     1: run each iteration as one captured CUDA graph
 *   profile       1: record per-routine CUDA-event timers (sptt_cpd_timers)
 *   sched         schedule of every mode's MTTKRP (NULL = default)
 *   mode_sched    array of nmodes schedules, one per root mode (overrides sched)
 *   plan          0: use sched / mode_sched; 1: choose each mode's schedule with
 *                 the autotuner (sptt_autotune); 2: choose it with the learned
 *                 scheduler `mlp` (sptt_mlp_predict on sptt_csf_features)
 *   mlp           the trained scheduler for plan = 2
 *   csf_mode      0: one CSF per mode, each rooted at its mode (root-mode
 *                 MTTKRPs only; N times the CSF memory); 1: one CSF for all
 *                 modes, the shortest mode at the root and the others below
 *                 by ascending length; 2: one CSF, the longest mode at the
 *                 root. With one CSF the non-root modes use sptt_mttkrp_mode's
 *                 kernels, sched (not mode_sched) applies to every mode, and
 *                 plan must be 0; with the default schedule each non-root
 *                 mode takes the output-conflict strategy (privatised hot
 *                 rows or global reductions) that ran faster in a timing
 *                 at create time (which therefore synchronises).
 *   leaf_tile_rows  mode tiling (SPLATT's tiling option, which the paper's
 *                 port omits, Section V): 0 = off; > 0: every mode whose CSF
 *                 has a leaf mode longer than this splits its non-zeros into
 *                 tiles of that many leaf indices, each its own CSF, and runs
 *                 its MTTKRP tile by tile with that tile's leaf rows in shared
 *                 memory (rows x round_up(rank, 8) x 4 bytes must be at most
 *                 160 KB, else BAD_ARG), adding the tiles' results in tile
 *                 order; -1: tiles as large as that table holds. Needs
 *                 csf_mode 0 and plan 0; tensors of 3 or more modes; at most
 *                 1024 tiles per mode (a mode with more stays untiled)
 */
typedef struct sptt_mlp sptt_mlp;
typedef struct {
    uint64_t seed;
    int32_t precision;
    int32_t refine_iters;
    int32_t use_graph;
    int32_t profile;
    const sptt_sched *sched;
    const sptt_sched *mode_sched;
    int32_t plan;
    const sptt_mlp *mlp;
    int32_t csf_mode;
    int32_t leaf_tile_rows;
} sptt_opts;

typedef struct sptt_cpd sptt_cpd;

/*
 * Prepare a CP-ALS run: copy the COO to the device if needed, build one CSF
 * per mode (rooted at that mode), allocate factors and workspace, and
 * compute |X|^2. Factors are not initialised (see sptt_cpd_init). rank in
 * [1, SPTT_MAX_RANK_ALS]. All later work of the handle runs on `stream`.
 * Synchronises the stream. Errors: BAD_ARG, UNSUPPORTED, OOM, CUDA.
 */
sptt_status sptt_cpd_create(const sptt_coo *coo, int32_t rank, const sptt_opts *opts,
                            sptt_stream stream, sptt_cpd **out);

/* Release a CP-ALS handle (NULL is ignored). Synchronises its stream. */
void sptt_cpd_free(sptt_cpd *cpd);

/*
 * Initialise the factors (Algorithm 1, initialisation). init = NULL: U(0,1) from the
 * Philox4x64-10 stream of opts.seed (key (seed, mode), counter (e/4,0,0,0),
 * word e mod 4, e = row*rank + col; value ((w >> 41) + 0.5) / 2^23). Else
 * init is a host array of nmodes pointers (host or device) to dims[m] x rank
 * row-major float factors. Resets the fit history. Asynchronous.
 */
sptt_status sptt_cpd_init(sptt_cpd *cpd, const float *const *init);

/*
 * Run up to `iters` ALS iterations (the loop of Algorithm 1): per mode n in
 * order, V = Hadamard of the other modes' Grams, A^(n) = MTTKRP_n V^dagger
 * (Cholesky in FP64; pseudo-inverse when V is not positive definite),
 * normalise the columns into lambda, refresh G_n; then the fit. With
 * tol > 0 the stream is synchronised after each iteration and the run stops
 * once |fit - fit_prev| < tol (not before the second iteration overall);
 * with tol = 0 all iterations are enqueued without synchronising.
 * iters_done (may be NULL) receives the iterations run by this call.
 * The precision of these iterations is opts.precision.
 */
sptt_status sptt_cpd_iterate(sptt_cpd *cpd, int32_t iters, double tol, int32_t *iters_done);

/*
 * Run `iters` iterations with FP32 gathers regardless of opts.precision
 * (the refinement sweep of a mixed-precision run). Same semantics as
 * sptt_cpd_iterate with tol = 0.
 */
sptt_status sptt_cpd_refine(sptt_cpd *cpd, int32_t iters);

/* Fit after the last iteration and the number of iterations run since
 * sptt_cpd_init. Synchronises. */
sptt_status sptt_cpd_fit(sptt_cpd *cpd, double *fit, int32_t *iters);

/* The fits of the last min(cap, iterations since init, 4096) iterations,
 * oldest first, into fits (host); *count (may be NULL) receives how many.
 * Synchronises. */
sptt_status sptt_cpd_fit_history(sptt_cpd *cpd, double *fits, int32_t cap, int32_t *count);

/* lambda (rank doubles, host or device): the column norms of the last mode
 * updated. Synchronises. */
sptt_status sptt_cpd_lambda(sptt_cpd *cpd, double *lambda);

/* Copy factor `mode` (normalised, dims[mode] x rank row-major float) into dst
 * (host or device). Synchronises. */
sptt_status sptt_cpd_factor(sptt_cpd *cpd, int32_t mode, float *dst);

/* Copy the FP64 Gram of factor `mode` (rank x rank) into dst (host or
 * device). Synchronises. */
sptt_status sptt_cpd_gram(sptt_cpd *cpd, int32_t mode, double *dst);

/*
 * Checkpoint / resume of a CP-ALS run (no counterpart in the paper; a
 * long run can be stopped and continued). The state is what the next
 * iteration reads: the normalised factors, their FP64 Grams, lambda, the
 * iteration count and the last (up to 4096) fits. sptt_cpd_save writes it
 * into buf (host, caller-owned): with buf = NULL or cap too small it only
 * sets *needed (bytes) and returns SPTT_ERR_BAD_ARG for a non-NULL buf that
 * is too small, SPTT_OK for buf = NULL. The format: a header (magic
 * "SPTTCKP1", version, shape, rank, iteration count, number of fits, FNV-1a
 * 64 checksum of the payload) followed by the factors (dims[m] x rank
 * float, row-major), the Grams (rank x rank double), lambda (rank double)
 * and the fits (double), host byte order. sptt_cpd_load restores a buffer
 * into a handle created for a tensor of the same shape and the same rank
 * (precision, schedules and CSF layout may differ): it checks the magic,
 * version, shape, rank, length and checksum (SPTT_ERR_BAD_ARG if any
 * differs); the BF16 copies are regenerated. Both synchronise. The CSFs,
 * which depend only on the tensor, are not part of the state.
 */
sptt_status sptt_cpd_save(sptt_cpd *cpd, void *buf, size_t cap, size_t *needed);
sptt_status sptt_cpd_load(sptt_cpd *cpd, const void *buf, size_t len);

/*
 * Solve branches taken since sptt_cpd_init: *n_pinv = mode updates that used
 * the pseudo-inverse (V not positive definite), *n_total = all mode updates.
 * Synchronises.
 */
sptt_status sptt_cpd_solve_branch(sptt_cpd *cpd, int64_t *n_pinv, int64_t *n_total);

/*
 * Per-routine device time in milliseconds since sptt_cpd_init, in the
 * routine categories of the paper's Table III (requires opts.profile = 1):
 *   ms[0] MTTKRP, ms[1] Inverse (Hadamard + Cholesky/pinv), ms[2] row solve
 *   + Gram ("Mat A^T A"), ms[3] Mat norm, ms[4] CPD fit.
 * counts (may be NULL) receives the number of timed launches of each.
 * Synchronises.
 */
#define SPTT_NUM_TIMERS 5
sptt_status sptt_cpd_timers(sptt_cpd *cpd, double *ms, int64_t *counts);

/*
 * One-shot CP-ALS: create, init (Philox from opts->seed), iterate up to
 * max_iters with tol (plus the refinement sweep for BF16), copy the results
 * out and free. factors_out: host array of nmodes pointers (host or device)
 * to dims[m] x rank floats; lambda_out: rank doubles (host or device); fit_out
 * and iters_out: host scalars. Any output may be NULL. Synchronous.
 */
sptt_status sptt_cpd_als(const sptt_coo *coo, int32_t rank, int32_t max_iters, double tol,
                         const sptt_opts *opts, sptt_stream stream, float *const *factors_out,
                         double *lambda_out, double *fit_out, int32_t *iters_out);

/* ------------------------------------------------------------------------ */
/* Schedule selection: candidates, autotuner, learned scheduler.            */
/* (Not in the paper, whose code picks locks vs privatisation by a rule.)   */
/* ------------------------------------------------------------------------ */

/* The candidate MTTKRP schedules for a tensor of nnz non-zeros: order {0, 2}
 * x variant {12, 13, 14, 15} x chunk {the default for nnz, twice it (at most
 * 4096)}, candidate i = (order i / 8, variant (i / 2) % 4, chunk i % 2).
 * Copies up to cap of them into out (may be NULL) and returns how many
 * there are (16). The default schedule (sptt_sched_default) is one of them. */
int32_t sptt_sched_candidates(int64_t nnz, sptt_sched *out, int32_t cap);

/* The schedule the library uses for the root-`root` MTTKRP of a tensor of
 * nnz non-zeros with these mode lengths (host array), rank and gather type
 * when none is given: the level order CP-ALS builds (2 on a 3-mode tensor of
 * at least 2^25 non-zeros when the shortest other mode's factor, in the
 * gather type, fits the 160 KB shared-memory table, else 0), the default variant for that
 * order's leaf mode and size, and the default chunk.
 * This is the fixed rule the learned scheduler is measured against. */
sptt_status sptt_sched_default(const int64_t *dims, int32_t nmodes, int32_t root, int32_t rank,
                               int32_t factor_dtype, int64_t nnz, sptt_sched *out);

/* The CSF level order of kind `kind` (sptt_sched::order: 0, 1 or 2) for the
 * tree rooted at `root`, into order_out (host, nmodes entries; ties to the
 * lower mode id). BAD_ARG on a bad root, kind or nmodes. */
sptt_status sptt_level_order(const int64_t *dims, int32_t nmodes, int32_t root, int32_t kind, int32_t *order_out);

/* Exhaustive autotuner: times the MTTKRP rooted at `root` under every
 * candidate schedule (random factors of `rank` columns, dtype SPTT_F32 or
 * SPTT_BF16), median of `reps` runs after one warm-up, into ms[candidate]
 * (host, one float per candidate). Builds the CSF in both orders.
 * Synchronises. */
sptt_status sptt_autotune(const sptt_coo *coo, int32_t root, int32_t rank, int32_t dtype, int32_t reps,
                          float *ms, sptt_stream stream);

/* The 16 statistics the learned scheduler reads for one CSF, rank and
 * factor gather type (SPTT_F32 or SPTT_BF16; host output): log2 nnz, modes,
 * log2 bytes of one factor row (rank rounded up to 8, times the element
 * size), log2 of the root / level-1 / leaf mode lengths, log2 slices, log2
 * leaf-parent fibers, log2 leaves per leaf-parent fiber and per slice, log2
 * largest slice, share of non-zeros in slices of >= 1024 leaves, share of
 * one-leaf slices, log2 of the leaf and level-1 factor table bytes,
 * slice-size histogram entropy / 5 (a device histogram kernel).
 * Synchronises. */
sptt_status sptt_csf_features(const sptt_csf *csf, int32_t rank, int32_t factor_dtype, float *feat,
                              sptt_stream stream);

/* The learned scheduler: an MLP 16 -> 64 (ReLU) -> 64 (ReLU) -> 16 in FP32
 * that predicts, per candidate, log2(time / best time) from the 16
 * statistics (standardised with the training set's mean and scale). */
sptt_status sptt_mlp_create(uint64_t seed, sptt_mlp **out);
void sptt_mlp_free(sptt_mlp *mlp);
/* Number of parameters (packed W1[64][16], b1, W2[64][64], b2, W3[16][64], b3). */
int32_t sptt_mlp_nparams(void);
/* Copy the parameters and the feature mean / scale (16 each) out of / into
 * the model (host or device buffers; any may be NULL). Synchronous. */
sptt_status sptt_mlp_get(const sptt_mlp *mlp, float *params, float *mu, float *sd);
sptt_status sptt_mlp_set(sptt_mlp *mlp, const float *params, const float *mu, const float *sd);
/* Y[n][16] = MLP(X[n][16]) (device buffers). Asynchronous. */
sptt_status sptt_mlp_forward(const sptt_mlp *mlp, const float *X, int64_t n, float *Y, sptt_stream stream);
/* Loss 1/(16 n) sum (Y - T)^2 over the batch and its gradient (nparams
 * floats, host or device). X, T device. Synchronises. */
sptt_status sptt_mlp_loss_grad(sptt_mlp *mlp, const float *X, const float *T, int64_t n, float *loss,
                               float *grad, sptt_stream stream);
/* `steps` full-batch Adam steps (lr; beta 0.9 / 0.999) on (X, T) (device);
 * the first call also sets the feature mean / scale from X. loss_history
 * (host or device, steps floats, may be NULL) receives each step's loss.
 * Synchronises. */
sptt_status sptt_mlp_train(sptt_mlp *mlp, const float *X, const float *T, int64_t n, int32_t steps, float lr,
                           float *loss_history, sptt_stream stream);
/* Candidate choice (argmin of the predicted times) for n feature rows
 * (host); pred (host, n x 16, may be NULL) receives the predictions.
 * Synchronises. */
sptt_status sptt_mlp_predict(const sptt_mlp *mlp, const float *feat, int64_t n, int32_t *choice, float *pred,
                             sptt_stream stream);

/* ------------------------------------------------------------------------ */
/* Batched CP-ALS: many small tensors in one persistent launch.             */
/* ------------------------------------------------------------------------ */

typedef struct sptt_batch sptt_batch;

/*
 * Prepare CP-ALS (Algorithm 1) for `count` independent tensors (each 2..4
 * modes, any sizes) with one rank in [1, 32] (else SPTT_ERR_UNSUPPORTED):
 * builds every tensor's CSF per mode, allocates factors and workspace, and
 * lays out global work lists (MTTKRP chunks and row tiles of all tensors back
 * to back). opts: seed (tensor t is initialised from seed + t), use_graph
 * (replay runs from a captured CUDA graph), sched (chunk size, a power of
 * two in [16, 4096], else SPTT_ERR_BAD_ARG; the MTTKRP
 * walk reads packed 16-byte leaf records, 16 bytes per non-zero more on the
 * device, and with the factor row width a multiple of 8 floats (rank 8, 16,
 * 32) gathers 32-byte row segments in a build of the kernel with one CTA per
 * SM; variant 4 keeps 16-byte segments at two CTAs per SM, variant 7 names
 * the 32-byte walk, variant 3 also reads the separate leaf arrays instead of
 * the packed records; both packed walks are the branch-free select walk),
 * plan (0: sched or the defaults, chunk 128; 1: the batched autotuner, which
 * times every walk (16-byte, and 32-byte when the row width allows) x chunk
 * (64, 128, 256) candidate on the batch itself, one warm-up and one timed
 * run of 2 iterations each, and keeps the fastest; the factors are left for
 * sptt_batch_init to set). Synchronises.
 */
sptt_status sptt_batch_create(const sptt_coo *coos, int32_t count, int32_t rank, const sptt_opts *opts,
                              sptt_stream stream, sptt_batch **out);
void sptt_batch_free(sptt_batch *batch);

/* The schedule the batch runs with (chunk, block, variant 3 / 4 / 7 as for
 * sptt_batch_create's opts.sched) into out; with plan 1, the timed run of
 * the chosen candidate (ms, may be NULL) and how many candidates were timed
 * (may be NULL; 0 without plan 1). */
sptt_status sptt_batch_schedule(sptt_batch *batch, sptt_sched *out, float *tuned_ms, int32_t *candidates);

/* U(0,1) Philox initial factors for every tensor (as sptt_cpd_init with
 * seed opts.seed + t) and their Grams; resets the fit history. */
sptt_status sptt_batch_init(sptt_batch *batch);

/*
 * Run `iters` ALS iterations of every tensor in ONE cooperative persistent
 * kernel launch (phases separated by grid barriers whose waits are bounded in
 * time). Synchronises and returns SPTT_ERR_TIMEOUT if a barrier wait ran out
 * (the kernel then stops early; the results are invalid).
 */
sptt_status sptt_batch_run(sptt_batch *batch, int32_t iters);

/* The last min(cap, iterations run, 4096) fits of tensor t, oldest first. */
sptt_status sptt_batch_fit_history(sptt_batch *batch, int32_t t, double *fits, int32_t cap, int32_t *count);

/* Factor `mode` of tensor t (dims x rank floats, host or device) and its
 * lambda (rank doubles). Synchronise. */
sptt_status sptt_batch_factor(sptt_batch *batch, int32_t t, int32_t mode, float *dst);
sptt_status sptt_batch_lambda(sptt_batch *batch, int32_t t, double *lambda);

/* Launch shape: grid (CTAs), and per mode position the number of MTTKRP
 * chunks and row tiles in the global lists (arrays of SPTT_MAX_MODES; any
 * output may be NULL). */
sptt_status sptt_batch_info(sptt_batch *batch, int32_t *grid, int64_t *chunks, int64_t *tiles);

/* Wall time (ms, summed over all runs since create) that CTA 0 of the
 * batched kernel spent in each phase: ms[0..4] = MTTKRP, normal equations,
 * row solve, finalise/fit, normalise (each including the wait at the grid
 * barrier that ends it), ms[5 + p] = the part of phase p spent waiting in
 * that barrier (10 doubles, host). Synchronises. */
sptt_status sptt_batch_phase_ms(sptt_batch *batch, double *ms);

/*
 * Test hook for the bounded barrier: on the next runs, CTA `skip_block` leaves
 * the kernel before its first barrier (so the others' waits run out), and
 * every wait gives up after timeout_ns (<= 0: the default of 2 s).
 * skip_block < 0 restores normal runs.
 */
sptt_status sptt_debug_batch_stall(sptt_batch *batch, int32_t skip_block, int64_t timeout_ns);

/*
 * Fault injection for tests (host side only): the countdown-th device
 * allocation made by the library from now on fails with SPTT_ERR_OOM, as if
 * the device were out of memory; 0 disables. Process-wide.
 */
void sptt_debug_fail_alloc_after(int64_t countdown);

/* Number of CUDA kernels this library has launched in this process so far
 * (every launch site counts once per launch). */
int64_t sptt_debug_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SPTT_H */
