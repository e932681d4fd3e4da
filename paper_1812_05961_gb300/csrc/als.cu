// CP-ALS driver (Algorithm 1, N modes) on one GPU.
//
// Per iteration, for each mode n in order (Gauss-Seidel: every update sees the
// latest factors):
//   MTTKRP over the CSF rooted at n
//   V = Hadamard of the other modes' Grams, W = V^dagger
//   A_un = M W, fused with Gram(A_un) and the fit's dots
//   lambda = column norms, G_n = D^-1 Gram(A_un) D^-1, normalise A
// then the fit at the end of the iteration. All of it is enqueued on the handle's stream; the
// host reads back only when asked (tol > 0, or an accessor).
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.cuh"

using namespace sptt;

extern "C" int64_t sptt_debug_launch_count(void);

namespace {
constexpr int kFitHistory = 4096;

struct TimerRec {
    int cat;
    cudaEvent_t a, b;
};
}  // namespace

struct sptt_cpd {
    int32_t N = 0;
    int64_t dims[SPTT_MAX_MODES] = {0};
    int32_t rank = 0;
    int32_t ld = 0;
    sptt_opts opts{};
    sptt_sched msched[SPTT_MAX_MODES] = {};  // schedule of each mode's MTTKRP
    bool has_msched[SPTT_MAX_MODES] = {false};
    cudaStream_t st = nullptr;
    // the normal equations of mode n depend only on the other modes' Grams,
    // so they run on a second stream while mode n's MTTKRP runs
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork[SPTT_MAX_MODES] = {nullptr};
    cudaEvent_t ev_join[SPTT_MAX_MODES] = {nullptr};
    sptt_csf *csf[SPTT_MAX_MODES] = {nullptr};
    // opts.leaf_tile_rows: the modes whose MTTKRP runs over leaf-index tiles
    // (tiling.cu), each tile a CSF of its own; tbase = each tile's first leaf
    // index; their MTTKRP result is full (Mfull, dims x ld)
    std::vector<sptt_csf *> tcsf[SPTT_MAX_MODES];
    std::vector<int64_t> tbase[SPTT_MAX_MODES];
    int32_t tleaf[SPTT_MAX_MODES] = {0};  // the leaf mode of a tiled mode's CSFs
    float *Mfull = nullptr;
    // csf_mode 1/2: one CSF for every mode; one_level[n] = the tree level of mode n
    sptt_csf *one = nullptr;
    int32_t one_level[SPTT_MAX_MODES] = {0};
    sptt_sched one_sched[SPTT_MAX_MODES] = {};  // schedule of each non-root mode's MTTKRP
    float *A[SPTT_MAX_MODES] = {nullptr};
    __nv_bfloat16 *Ab[SPTT_MAX_MODES] = {nullptr};
    double *G[SPTT_MAX_MODES] = {nullptr};
    float *M = nullptr;      // MTTKRP output: compact (one row per slice) for a root mode, full otherwise
    double *Mh = nullptr;    // FP64 rows of the heavy slices
    double *normx2 = nullptr;
    double *fits = nullptr;  // device ring of fit values, kFitHistory entries
    int64_t *iter_dev = nullptr;  // device iteration counter (indexes the ring)
    DenseWork w;
    // one captured iteration per gather precision (index 1 = BF16)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};
    int64_t iters = 0;       // iterations run since init
    // profiling
    std::vector<TimerRec> pending;
    std::vector<cudaEvent_t> free_events;
    double ms[SPTT_NUM_TIMERS] = {0};
    int64_t counts[SPTT_NUM_TIMERS] = {0};
};

namespace {

cudaEvent_t take_event(sptt_cpd *c) {
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records a timer interval around the enqueued work of one routine.
struct Timed {
    sptt_cpd *c;
    int cat;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Timed(sptt_cpd *c_, int cat_, cudaStream_t s_) : c(c_), cat(cat_), s(s_) {
        if (c->opts.profile) {
            a = take_event(c);
            cudaEventRecord(a, s);
        }
    }
    Timed(sptt_cpd *c_, int cat_) : Timed(c_, cat_, c_->st) {}
    ~Timed() {
        if (a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, s);
            c->pending.push_back({cat, a, b});
        }
    }
};

sptt_status resolve_timers(sptt_cpd *c) {
    if (c->pending.empty()) return SPTT_OK;
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    for (auto &r : c->pending) {
        float ms = 0.f;
        SPTT_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        c->ms[r.cat] += ms;
        c->counts[r.cat] += 1;
        c->free_events.push_back(r.a);
        c->free_events.push_back(r.b);
    }
    c->pending.clear();
    return SPTT_OK;
}

// Level order of mode m's CSF when no schedule fixes it: with FP32 gathers
// on a large tensor, the shortest other mode at the leaves (kind 2) if its
// factor fits the shared-memory table of the default MTTKRP kernel, so that
// every leaf row is read from there; otherwise ascending lengths below the
// root (kind 0).
int default_order_kind(const sptt_cpd *c, int m, int64_t nnz) {
    return sptt::default_order_kind(c->dims, c->N, m, c->ld, c->opts.precision, nnz);
}

sptt_status run_iteration(sptt_cpd *c, bool bf16) {
    const int N = c->N;
    const void *fac[SPTT_MAX_MODES];
    for (int m = 0; m < N; ++m) fac[m] = bf16 ? (const void *)c->Ab[m] : (const void *)c->A[m];
    for (int n = 0; n < N; ++n) {
        const sptt_sched *sched = c->has_msched[n] ? &c->msched[n] : nullptr;
        sptt_csf *cs = c->one ? c->one : c->csf[n];
        const int L = c->one ? c->one_level[n] : 0;  // L > 0: a non-root mode of the one CSF
        const int32_t dt = bf16 ? SPTT_BF16 : SPTT_F32;
        const bool fork = c->side != nullptr;
        if (fork) {
            SPTT_CUDA(cudaEventRecord(c->ev_fork[n], c->st));
            SPTT_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork[n], 0));
            {
                Timed t(c, 1, c->side);
                SPTT_TRY(normal_prep_launch(c->G, N, n, c->rank, &c->w, c->side));
            }
            SPTT_CUDA(cudaEventRecord(c->ev_join[n], c->side));
        }
        const bool tiled = !c->tcsf[n].empty();
        {
            Timed t(c, 0);
            if (tiled) {
                // the tiles' MTTKRPs, each added into the full result in tile order
                SPTT_TRY(fill_zero_launch(c->Mfull, (size_t)c->dims[n] * c->ld * sizeof(float), c->st));
                // the leaf rows of a tile fit the shared-memory table (the 512-thread form for BF16 rows)
                sptt_sched ts = sched ? *sched : sptt_sched{};
                if (!sched) ts.variant = bf16 ? 15 : 14;
                const int esz = bf16 ? 2 : 4;
                for (size_t k = 0; k < c->tcsf[n].size(); ++k) {
                    const void *tf[SPTT_MAX_MODES];
                    for (int m = 0; m < N; ++m) tf[m] = fac[m];
                    const int lm = c->tleaf[n];
                    tf[lm] = static_cast<const char *>(fac[lm]) + (size_t)c->tbase[n][k] * c->ld * esz;
                    SPTT_TRY(mttkrp_launch(c->tcsf[n][k], tf, dt, c->ld, c->M, c->Mh, &ts, c->st));
                    SPTT_TRY(tile_accumulate_launch(c->tcsf[n][k], c->M, c->Mh, c->ld, c->Mfull, c->st));
                }
            } else if (L == 0) {
                SPTT_TRY(mttkrp_launch(cs, fac, dt, c->ld, c->M, c->Mh, sched, c->st));
            } else {
                SPTT_TRY(mttkrp_mode_launch(cs, L, fac, dt, c->ld, c->M, &c->one_sched[n], c->st));
            }
        }
        if (fork) {
            SPTT_CUDA(cudaStreamWaitEvent(c->st, c->ev_join[n], 0));
        } else {
            Timed t(c, 1);
            SPTT_TRY(normal_prep_launch(c->G, N, n, c->rank, &c->w, c->st));
        }
        // the compact result of a root mode maps slice f to row fids[0][f];
        // a non-root mode's result and a tiled mode's are full (row i is row i)
        const int32_t *rowmap = (L == 0 && !tiled) ? cs->fids[0] : nullptr;
        const int64_t nrows = (L == 0 && !tiled) ? cs->nfibs[0] : c->dims[n];
        const float *Mres = tiled ? c->Mfull : c->M;
        {
            Timed t(c, 2);
            // rows of mode n without a slice come out zero: clear A (and its
            // BF16 copy) before the solve writes the rows that have one,
            // unless every index of mode n has a slice
            if (nrows < c->dims[n]) {
                SPTT_TRY(fill_zero_launch(c->A[n], (size_t)c->dims[n] * c->ld * sizeof(float), c->st));
                if (c->Ab[n])
                    SPTT_TRY(fill_zero_launch(c->Ab[n], (size_t)c->dims[n] * c->ld * sizeof(__nv_bfloat16), c->st));
            }
            const bool compact = L == 0 && !tiled;
            SPTT_TRY(postsolve_launch(Mres, compact ? c->Mh : nullptr, compact ? cs->hidx : nullptr, rowmap, c->A[n],
                                      nrows, &c->w, c->st));
        }
        {
            Timed t(c, 3);
            SPTT_TRY(finalize_normalize_launch(c->G[n], c->A[n], c->Ab[n], rowmap, nrows, &c->w, c->st));
        }
    }
    {
        Timed t(c, 4);
        SPTT_TRY(fit_launch(c->G, N, c->normx2, &c->w, c->fits, kFitHistory, c->iter_dev, c->st));
    }
    return SPTT_OK;
}

// Work partitions (and, with one CSF, the hot-row tables of the non-root
// levels) of every mode's MTTKRP; their first build allocates and
// synchronises, so this runs before any capture.
sptt_status prepare_all(sptt_cpd *c) {
    if (c->one) {
        const sptt_sched *s = c->has_msched[0] ? &c->msched[0] : nullptr;
        SPTT_TRY(mttkrp_prepare(c->one, s, c->st));
        for (int n = 0; n < c->N; ++n)
            if (c->one_level[n] > 0)
                SPTT_TRY(mttkrp_mode_prepare(c->one, c->one_level[n], c->ld, &c->one_sched[n], c->st));
        return SPTT_OK;
    }
    for (int n = 0; n < c->N; ++n) {
        const sptt_sched *s = c->has_msched[n] ? &c->msched[n] : nullptr;
        if (c->tcsf[n].empty()) {
            SPTT_TRY(mttkrp_prepare(c->csf[n], s, c->st));
            continue;
        }
        sptt_sched ts = s ? *s : sptt_sched{};
        if (!s) ts.variant = 14;
        for (auto *t : c->tcsf[n]) SPTT_TRY(mttkrp_prepare(t, &ts, c->st));
    }
    return SPTT_OK;
}

// With one CSF and the default schedule, each non-root mode's MTTKRP takes
// whichever output-conflict strategy (privatised hot rows, or global
// reductions only) ran faster in a short timing on the handle's own factors
// and buffers (the results are discarded; the factors are re-initialised
// by sptt_cpd_init).
sptt_status choose_conflict_strategy(sptt_cpd *c) {
    const void *fac[SPTT_MAX_MODES];
    for (int m = 0; m < c->N; ++m) fac[m] = c->A[m];
    cudaEvent_t e[3];
    for (auto &x : e) SPTT_CUDA(cudaEventCreate(&x));
    struct Ev {
        cudaEvent_t *e;
        ~Ev() { for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]); }
    } guard{e};
    for (int n = 0; n < c->N; ++n) {
        const int L = c->one_level[n];
        if (L == 0) continue;
        float best = 0.f;
        int best_v = 2;
        for (int v = 2; v >= 1; --v) {
            sptt_sched s = c->one_sched[n];
            s.variant = v;
            SPTT_TRY(mttkrp_mode_prepare(c->one, L, c->ld, &s, c->st));
            SPTT_TRY(mttkrp_mode_launch(c->one, L, fac, SPTT_F32, c->ld, c->M, &s, c->st));  // warm-up
            SPTT_CUDA(cudaEventRecord(e[0], c->st));
            SPTT_TRY(mttkrp_mode_launch(c->one, L, fac, SPTT_F32, c->ld, c->M, &s, c->st));
            SPTT_CUDA(cudaEventRecord(e[1], c->st));
            SPTT_CUDA(cudaEventSynchronize(e[1]));
            float ms = 0.f;
            SPTT_CUDA(cudaEventElapsedTime(&ms, e[0], e[1]));
            if (v == 2 || ms < best) {
                best = ms;
                best_v = v;
            }
        }
        c->one_sched[n].variant = best_v;
    }
    return SPTT_OK;
}

// Captures one iteration into a graph (built once per precision) and
// replays it. Partitions are prepared before capture (their first build
// allocates and synchronises).
sptt_status run_iteration_graph(sptt_cpd *c, bool bf16) {
    const int p = bf16 ? 1 : 0;
    if (!c->graph[p]) {
        SPTT_TRY(prepare_all(c));
        SPTT_CUDA(cudaStreamSynchronize(c->st));
        cudaGraph_t g = nullptr;
        SPTT_CUDA(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = sptt_debug_launch_count();
        sptt_status s = run_iteration(c, bf16);
        const int64_t l1 = sptt_debug_launch_count();
        cudaError_t e = cudaStreamEndCapture(c->st, &g);
        if (s != SPTT_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->graph[p], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        c->graph_kernels[p] = l1 - l0;
        count_launch(-(l1 - l0));  // capture launched nothing; replays are counted below
    }
    SPTT_CUDA(cudaGraphLaunch(c->graph[p], c->st));
    count_launch(c->graph_kernels[p]);
    return SPTT_OK;
}

sptt_status step(sptt_cpd *c, bool bf16) {
    if (c->opts.use_graph && !c->opts.profile && c->st != nullptr) SPTT_TRY(run_iteration_graph(c, bf16));
    else SPTT_TRY(run_iteration(c, bf16));
    c->iters += 1;
    return SPTT_OK;
}

sptt_status read_fit(sptt_cpd *c, int64_t it, double *out) {
    SPTT_CUDA(cudaMemcpyAsync(out, c->fits + (it % kFitHistory), sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (c->one) SPTT_TRY(sptt_csf_check(c->one, c->st));  // synchronises
    for (int m = 0; m < c->N; ++m) {
        if (c->csf[m]) SPTT_TRY(sptt_csf_check(c->csf[m], c->st));
        for (auto *t : c->tcsf[m]) SPTT_TRY(sptt_csf_check(t, c->st));
    }
    return SPTT_OK;
}

void destroy(sptt_cpd *c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->one) csf_destroy(c->one);
    for (int m = 0; m < SPTT_MAX_MODES; ++m) {
        if (c->csf[m]) csf_destroy(c->csf[m]);
        for (auto *t : c->tcsf[m]) csf_destroy(t);
        if (c->A[m]) dev_free(c->A[m], c->st);
        if (c->Ab[m]) dev_free(c->Ab[m], c->st);
        if (c->G[m]) dev_free(c->G[m], c->st);
    }
    if (c->M) dev_free(c->M, c->st);
    if (c->Mfull) dev_free(c->Mfull, c->st);
    if (c->Mh) dev_free(c->Mh, c->st);
    if (c->normx2) dev_free(c->normx2, c->st);
    if (c->fits) dev_free(c->fits, c->st);
    if (c->iter_dev) dev_free(c->iter_dev, c->st);
    for (int p = 0; p < 2; ++p)
        if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
    dense_work_free(&c->w, c->st);
    for (auto &r : c->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->free_events) cudaEventDestroy(e);
    for (int m = 0; m < SPTT_MAX_MODES; ++m) {
        if (c->ev_fork[m]) cudaEventDestroy(c->ev_fork[m]);
        if (c->ev_join[m]) cudaEventDestroy(c->ev_join[m]);
    }
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    cudaStreamSynchronize(c->st);
    delete c;
}

}  // namespace

extern "C" sptt_status sptt_cpd_create(const sptt_coo *coo, int32_t rank, const sptt_opts *opts, sptt_stream stream,
                                       sptt_cpd **out) {
    clear_error();
    if (!out) return set_error(SPTT_ERR_BAD_ARG, "out is NULL");
    *out = nullptr;
    SPTT_TRY(coo_validate_shape(coo));
    if (coo->nnz == 0) return set_error(SPTT_ERR_BAD_ARG, "CP-ALS needs at least one non-zero");
    if (rank < 1) return set_error(SPTT_ERR_BAD_ARG, "rank must be >= 1");
    if (rank > SPTT_MAX_RANK_ALS) return set_error(SPTT_ERR_UNSUPPORTED, "rank must be <= 64");
    sptt_opts o{};
    if (opts) o = *opts;
    if (o.precision != SPTT_F32 && o.precision != SPTT_BF16)
        return set_error(SPTT_ERR_BAD_ARG, "opts.precision must be SPTT_F32 or SPTT_BF16");
    for (int m = 0; m < (o.mode_sched ? coo->nmodes : 1); ++m) {
        const sptt_sched *s = o.mode_sched ? &o.mode_sched[m] : o.sched;
        if (!s) break;
        if (s->chunk && (s->chunk < 16 || s->chunk > 4096 || (s->chunk & (s->chunk - 1))))
            return set_error(SPTT_ERR_BAD_ARG, "sched->chunk must be a power of two in [16, 4096]");
        if (s->block && (s->block < 32 || s->block > 256 || s->block % 32))
            return set_error(SPTT_ERR_BAD_ARG, "sched->block must be a multiple of 32 in [32, 256]");
        if (s->variant < 0 || s->variant > kMaxVariant || s->order < 0 || s->order > 2)
            return set_error(SPTT_ERR_BAD_ARG, "sched->variant must be in [0, " + std::to_string(kMaxVariant) +
                                                   "] and order in [0, 2]");
    }
    if (o.plan < 0 || o.plan > 2) return set_error(SPTT_ERR_BAD_ARG, "opts.plan must be 0, 1 or 2");
    if (o.csf_mode < 0 || o.csf_mode > 2) return set_error(SPTT_ERR_BAD_ARG, "opts.csf_mode must be 0, 1 or 2");
    if (o.csf_mode != 0 && (o.plan != 0 || o.mode_sched))
        return set_error(SPTT_ERR_BAD_ARG, "one CSF for all modes takes one schedule (opts.sched) and plan 0");
    if (o.plan == 2 && !o.mlp) return set_error(SPTT_ERR_BAD_ARG, "opts.plan = 2 needs opts.mlp");
    if (o.leaf_tile_rows < -1) return set_error(SPTT_ERR_BAD_ARG, "opts.leaf_tile_rows must be -1, 0 or > 0");
    if (o.leaf_tile_rows != 0 && (o.csf_mode != 0 || o.plan != 0))
        return set_error(SPTT_ERR_BAD_ARG, "leaf tiling takes one CSF per mode and plan 0");
    if (o.leaf_tile_rows > 0 && !leaf_table_fits(o.leaf_tile_rows, (rank + 7) / 8 * 8, 4))
        return set_error(SPTT_ERR_BAD_ARG, "opts.leaf_tile_rows rows of the factor must fit the 160 KB shared-memory table");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    sptt_cpd *c = new sptt_cpd();
    struct Guard {
        sptt_cpd *c;
        ~Guard() { if (c) destroy(c); }
    } guard{c};
    c->N = coo->nmodes;
    c->rank = rank;
    c->ld = (rank + 7) / 8 * 8;
    c->opts = o;
    c->opts.sched = nullptr;
    c->opts.mode_sched = nullptr;
    c->opts.mlp = nullptr;
    c->st = st;
    SPTT_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    for (int m = 0; m < c->N; ++m) {
        SPTT_CUDA(cudaEventCreateWithFlags(&c->ev_fork[m], cudaEventDisableTiming));
        SPTT_CUDA(cudaEventCreateWithFlags(&c->ev_join[m], cudaEventDisableTiming));
    }
    for (int m = 0; m < c->N; ++m) {
        c->dims[m] = coo->dims[m];
        const sptt_sched *s = o.mode_sched ? &o.mode_sched[m] : o.sched;
        if (s) {
            c->msched[m] = *s;
            c->has_msched[m] = true;
        }
    }
    if (o.csf_mode != 0) {
        // one CSF: the shortest (csf_mode 1) or longest (2) mode at the root,
        // ties to the lower mode id, the others below by ascending length
        int root = 0;
        for (int m = 1; m < c->N; ++m)
            if (o.csf_mode == 1 ? c->dims[m] < c->dims[root] : c->dims[m] > c->dims[root]) root = m;
        int32_t order[SPTT_MAX_MODES];
        level_order(c->dims, c->N, root, 0, order);
        DevCoo dc;
        SPTT_TRY(coo_to_device(coo, st, &dc));
        SPTT_TRY(csf_build_device(&dc.coo, root, order, st, &c->one));
        for (int l = 0; l < c->N; ++l) c->one_level[order[l]] = l;
        for (int m = 0; m < c->N; ++m) {
            c->one_sched[m] = c->has_msched[m] ? c->msched[m] : sptt_sched{};
            if (c->one_sched[m].variant != 1) c->one_sched[m].variant = 2;  // privatise unless told otherwise
        }
    } else {
        DevCoo dc;
        SPTT_TRY(coo_to_device(coo, st, &dc));
        for (int m = 0; m < c->N; ++m) {
            if (o.plan == 1) {  // exhaustive autotuner
                float ms[32];
                const int32_t nc = sptt_sched_candidates(coo->nnz, nullptr, 0);
                SPTT_TRY(sptt_autotune(&dc.coo, m, rank, o.precision, 3, ms, stream));
                int best = 0;
                for (int i = 1; i < nc; ++i)
                    if (ms[i] < ms[best]) best = i;
                sptt_sched cands[32];
                sptt_sched_candidates(coo->nnz, cands, 32);
                c->msched[m] = cands[best];
                c->has_msched[m] = true;
            }
            // with leaf tiling and no schedule, 3-mode tensors put the shortest other
            // mode at the leaves (fewest tiles)
            const int kind = c->has_msched[m] ? c->msched[m].order
                             : (o.leaf_tile_rows != 0 && c->N == 3) ? 2
                                                                     : default_order_kind(c, m, coo->nnz);
            int32_t order[SPTT_MAX_MODES];
            level_order(c->dims, c->N, m, kind, order);
            if (o.leaf_tile_rows != 0) {
                // leaf tiling: tiles of leaf_tile_rows rows (-1: as many as the table holds)
                // wherever the leaf factor is larger than one tile and the tiles are few enough
                const int32_t rows = o.leaf_tile_rows > 0 ? o.leaf_tile_rows
                                                          : (int32_t)(kTableMaxBytes / ((size_t)c->ld * 4));
                const int64_t dl = c->dims[order[c->N - 1]];
                const int64_t nt = (dl + rows - 1) / rows;
                if (c->N >= 3 && nt > 1 && nt <= kMaxTiles) {
                    c->tleaf[m] = order[c->N - 1];
                    SPTT_TRY(tiles_build(&dc.coo, m, order, rows, st, &c->tcsf[m], &c->tbase[m]));
                    continue;
                }
            }
            SPTT_TRY(csf_build_device(&dc.coo, m, order, st, &c->csf[m]));
            if (o.plan == 2) {  // learned scheduler on the default CSF's statistics
                float feat[16];
                int32_t choice = 0;
                SPTT_TRY(sptt_csf_features(c->csf[m], rank, o.precision, feat, stream));
                SPTT_TRY(sptt_mlp_predict(o.mlp, feat, 1, &choice, nullptr, stream));
                sptt_sched cands[32];
                sptt_sched_candidates(coo->nnz, cands, 32);
                c->msched[m] = cands[choice];
                c->has_msched[m] = true;
                if (c->msched[m].order != kind) {
                    csf_destroy(c->csf[m]);
                    c->csf[m] = nullptr;
                    level_order(c->dims, c->N, m, c->msched[m].order, order);
                    SPTT_TRY(csf_build_device(&dc.coo, m, order, st, &c->csf[m]));
                }
            }
        }
    }
    int64_t max_rows = 0, max_slices = 0, max_heavy = 0;
    SPTT_TRY(prepare_all(c));
    int64_t max_full = 0;  // rows of the full result of the tiled modes
    for (int m = 0; m < c->N; ++m) {
        const int64_t rows = c->dims[m];
        if (rows > max_rows) max_rows = rows;
        if (!c->tcsf[m].empty()) {
            // a tile's compact result goes through M and Mh, the sum of the tiles through Mfull
            if (rows > max_full) max_full = rows;
            for (auto *t : c->tcsf[m]) {
                if (t->nfibs[0] > max_slices) max_slices = t->nfibs[0];
                if (t->nheavy > max_heavy) max_heavy = t->nheavy;
            }
        } else {
            // rows of the MTTKRP result of mode m: compact for a root mode, full otherwise
            const sptt_csf *cs = c->one ? c->one : c->csf[m];
            const int64_t mrows = (c->one && c->one_level[m] > 0) ? rows : cs->nfibs[0];
            if (mrows > max_slices) max_slices = mrows;
            if (cs->nheavy > max_heavy) max_heavy = cs->nheavy;
        }
        SPTT_TRY(dev_alloc_n(&c->A[m], (size_t)rows * c->ld, st));
        SPTT_TRY(fill_zero_launch(c->A[m], (size_t)rows * c->ld * sizeof(float), st));
        if (o.precision == SPTT_BF16) {
            SPTT_TRY(dev_alloc_n(&c->Ab[m], (size_t)rows * c->ld, st));
            SPTT_TRY(fill_zero_launch(c->Ab[m], (size_t)rows * c->ld * sizeof(__nv_bfloat16), st));
        }
        SPTT_TRY(dev_alloc_n(&c->G[m], (size_t)rank * rank, st));
    }
    SPTT_TRY(dev_alloc_n(&c->M, (size_t)max_slices * c->ld, st));
    if (max_full > 0) SPTT_TRY(dev_alloc_n(&c->Mfull, (size_t)max_full * c->ld, st));
    SPTT_TRY(dev_alloc_n(&c->Mh, (size_t)max_heavy * c->ld, st));
    SPTT_TRY(dev_alloc_n(&c->normx2, 1, st));
    SPTT_TRY(dev_alloc_n(&c->fits, kFitHistory, st));
    SPTT_TRY(fill_zero_launch(c->fits, kFitHistory * sizeof(double), st));
    SPTT_TRY(dev_alloc_n(&c->iter_dev, 1, st));
    SPTT_TRY(fill_zero_launch(c->iter_dev, sizeof(int64_t), st));
    SPTT_TRY(dense_work_alloc(&c->w, rank, c->ld, max_rows, st));
    // |X|^2 over the coalesced non-zeros: any untiled CSF holds all of them, a
    // tiled mode's tiles together do
    const sptt_csf *c0 = c->one;
    for (int m = 0; m < c->N && !c0; ++m) c0 = c->csf[m];
    if (c0) {
        SPTT_TRY(sumsq_launch(c0->vals, c0->nfibs[c0->nmodes - 1], c->normx2, st));
    } else {
        double total = 0.0;
        for (auto *t : c->tcsf[0]) {
            double part = 0.0;
            SPTT_TRY(sumsq_launch(t->vals, t->nfibs[t->nmodes - 1], c->normx2, st));
            SPTT_CUDA(cudaMemcpyAsync(&part, c->normx2, sizeof(double), cudaMemcpyDeviceToHost, st));
            SPTT_CUDA(cudaStreamSynchronize(st));
            total += part;
        }
        SPTT_CUDA(cudaMemcpyAsync(c->normx2, &total, sizeof(double), cudaMemcpyHostToDevice, st));
        SPTT_CUDA(cudaStreamSynchronize(st));
    }
    if (c->one && !(c->has_msched[0] && c->msched[0].variant != 0)) {
        for (int m = 0; m < c->N; ++m)
            SPTT_TRY(init_factor_launch(c->opts.seed, m, c->dims[m], c->rank, c->ld, c->A[m], st));
        SPTT_TRY(choose_conflict_strategy(c));
    }
    SPTT_CUDA(cudaStreamSynchronize(st));
    guard.c = nullptr;
    *out = c;
    return SPTT_OK;
}

extern "C" void sptt_cpd_free(sptt_cpd *cpd) { destroy(cpd); }

extern "C" sptt_status sptt_cpd_init(sptt_cpd *c, const float *const *init) {
    clear_error();
    if (!c) return set_error(SPTT_ERR_BAD_ARG, "cpd is NULL");
    cudaStream_t st = c->st;
    for (int m = 0; m < c->N; ++m) {
        if (init) {
            if (!init[m]) return set_error(SPTT_ERR_BAD_ARG, "init[m] is NULL");
            SPTT_TRY(fill_zero_launch(c->A[m], (size_t)c->dims[m] * c->ld * sizeof(float), st));
            SPTT_CUDA(cudaMemcpy2DAsync(c->A[m], c->ld * sizeof(float), init[m], c->rank * sizeof(float),
                                        c->rank * sizeof(float), c->dims[m], cudaMemcpyDefault, st));
        } else {
            SPTT_TRY(init_factor_launch(c->opts.seed, m, c->dims[m], c->rank, c->ld, c->A[m], st));
        }
        if (c->Ab[m]) SPTT_TRY(to_bf16_launch(c->A[m], c->Ab[m], c->dims[m] * c->ld, st));
        SPTT_TRY(gram_launch(c->A[m], c->dims[m], c->rank, c->ld, c->G[m], c->w.partials, c->w.nblocks, st));
    }
    SPTT_TRY(fill_zero_launch(c->w.branch, 2 * sizeof(int32_t), st));
    SPTT_TRY(fill_zero_launch(c->fits, kFitHistory * sizeof(double), st));
    SPTT_TRY(fill_zero_launch(c->iter_dev, sizeof(int64_t), st));
    c->iters = 0;
    SPTT_TRY(resolve_timers(c));
    for (int i = 0; i < SPTT_NUM_TIMERS; ++i) {
        c->ms[i] = 0;
        c->counts[i] = 0;
    }
    return SPTT_OK;
}

static sptt_status iterate(sptt_cpd *c, int32_t iters, double tol, bool bf16, int32_t *done) {
    if (done) *done = 0;
    double prev = 0.0;
    if (tol > 0.0 && c->iters > 0) SPTT_TRY(read_fit(c, c->iters - 1, &prev));
    for (int32_t i = 0; i < iters; ++i) {
        SPTT_TRY(step(c, bf16));
        if (done) *done = i + 1;
        if (tol > 0.0) {
            double f = 0.0;
            SPTT_TRY(read_fit(c, c->iters - 1, &f));
            if (c->iters >= 2 && fabs(f - prev) < tol) break;
            prev = f;
        }
    }
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_iterate(sptt_cpd *c, int32_t iters, double tol, int32_t *iters_done) {
    clear_error();
    if (!c) return set_error(SPTT_ERR_BAD_ARG, "cpd is NULL");
    if (iters < 0 || !(tol >= 0.0)) return set_error(SPTT_ERR_BAD_ARG, "iters must be >= 0 and tol >= 0");
    return iterate(c, iters, tol, c->opts.precision == SPTT_BF16, iters_done);
}

extern "C" sptt_status sptt_cpd_refine(sptt_cpd *c, int32_t iters) {
    clear_error();
    if (!c) return set_error(SPTT_ERR_BAD_ARG, "cpd is NULL");
    if (iters < 0) return set_error(SPTT_ERR_BAD_ARG, "iters must be >= 0");
    return iterate(c, iters, 0.0, false, nullptr);
}

extern "C" sptt_status sptt_cpd_fit(sptt_cpd *c, double *fit, int32_t *iters) {
    clear_error();
    if (!c) return set_error(SPTT_ERR_BAD_ARG, "cpd is NULL");
    if (iters) *iters = (int32_t)c->iters;
    if (fit) {
        if (c->iters == 0) *fit = 0.0;
        else SPTT_TRY(read_fit(c, c->iters - 1, fit));
    }
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_fit_history(sptt_cpd *c, double *fits, int32_t cap, int32_t *count) {
    clear_error();
    if (!c || !fits) return set_error(SPTT_ERR_BAD_ARG, "cpd and fits must be non-NULL");
    const int64_t avail = c->iters < kFitHistory ? c->iters : kFitHistory;
    const int64_t n = avail < cap ? avail : cap;
    std::vector<double> ring(kFitHistory);
    SPTT_CUDA(cudaMemcpyAsync(ring.data(), c->fits, kFitHistory * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    // the last n fits, oldest first
    for (int64_t j = 0; j < n; ++j) fits[j] = ring[(c->iters - n + j) % kFitHistory];
    if (count) *count = (int32_t)n;
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_lambda(sptt_cpd *c, double *lambda) {
    clear_error();
    if (!c || !lambda) return set_error(SPTT_ERR_BAD_ARG, "cpd and lambda must be non-NULL");
    SPTT_CUDA(cudaMemcpyAsync(lambda, c->w.lambda, c->rank * sizeof(double), cudaMemcpyDefault, c->st));
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_factor(sptt_cpd *c, int32_t mode, float *dst) {
    clear_error();
    if (!c || !dst) return set_error(SPTT_ERR_BAD_ARG, "cpd and dst must be non-NULL");
    if (mode < 0 || mode >= c->N) return set_error(SPTT_ERR_BAD_ARG, "mode out of range");
    SPTT_CUDA(cudaMemcpy2DAsync(dst, c->rank * sizeof(float), c->A[mode], c->ld * sizeof(float),
                                c->rank * sizeof(float), c->dims[mode], cudaMemcpyDefault, c->st));
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_gram(sptt_cpd *c, int32_t mode, double *dst) {
    clear_error();
    if (!c || !dst) return set_error(SPTT_ERR_BAD_ARG, "cpd and dst must be non-NULL");
    if (mode < 0 || mode >= c->N) return set_error(SPTT_ERR_BAD_ARG, "mode out of range");
    SPTT_CUDA(cudaMemcpyAsync(dst, c->G[mode], (size_t)c->rank * c->rank * sizeof(double), cudaMemcpyDefault, c->st));
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_solve_branch(sptt_cpd *c, int64_t *n_pinv, int64_t *n_total) {
    clear_error();
    if (!c) return set_error(SPTT_ERR_BAD_ARG, "cpd is NULL");
    int32_t b[2] = {0, 0};
    SPTT_CUDA(cudaMemcpyAsync(b, c->w.branch, sizeof(b), cudaMemcpyDeviceToHost, c->st));
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    if (n_pinv) *n_pinv = b[0];
    if (n_total) *n_total = b[1];
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_timers(sptt_cpd *c, double *ms, int64_t *counts) {
    clear_error();
    if (!c) return set_error(SPTT_ERR_BAD_ARG, "cpd is NULL");
    SPTT_TRY(resolve_timers(c));
    for (int i = 0; i < SPTT_NUM_TIMERS; ++i) {
        if (ms) ms[i] = c->ms[i];
        if (counts) counts[i] = c->counts[i];
    }
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_als(const sptt_coo *coo, int32_t rank, int32_t max_iters, double tol,
                                    const sptt_opts *opts, sptt_stream stream, float *const *factors_out,
                                    double *lambda_out, double *fit_out, int32_t *iters_out) {
    clear_error();
    if (max_iters < 0 || !(tol >= 0.0)) return set_error(SPTT_ERR_BAD_ARG, "max_iters must be >= 0 and tol >= 0");
    sptt_cpd *c = nullptr;
    SPTT_TRY(sptt_cpd_create(coo, rank, opts, stream, &c));
    struct Guard {
        sptt_cpd *c;
        ~Guard() { destroy(c); }
    } guard{c};
    SPTT_TRY(sptt_cpd_init(c, nullptr));
    int32_t done = 0;
    SPTT_TRY(sptt_cpd_iterate(c, max_iters, tol, &done));
    if (c->opts.precision == SPTT_BF16) {
        const int32_t refine = c->opts.refine_iters > 0 ? c->opts.refine_iters : 1;
        SPTT_TRY(sptt_cpd_refine(c, refine));
    }
    if (factors_out)
        for (int m = 0; m < c->N; ++m)
            if (factors_out[m]) SPTT_TRY(sptt_cpd_factor(c, m, factors_out[m]));
    if (lambda_out) SPTT_TRY(sptt_cpd_lambda(c, lambda_out));
    int32_t it = 0;
    SPTT_TRY(sptt_cpd_fit(c, fit_out, &it));
    if (iters_out) *iters_out = it;
    return SPTT_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume
// ---------------------------------------------------------------------------
namespace {

struct CkpHeader {
    char magic[8];
    uint32_t version;
    int32_t nmodes;
    int32_t rank;
    int32_t pad_;
    int64_t dims[SPTT_MAX_MODES];
    int64_t iters;
    int64_t nfits;
    uint64_t checksum;  // FNV-1a 64 of the payload
};

constexpr char kCkpMagic[8] = {'S', 'P', 'T', 'T', 'C', 'K', 'P', '1'};
constexpr uint32_t kCkpVersion = 1;

uint64_t fnv1a(const unsigned char *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

size_t ckp_payload(const sptt_cpd *c, int64_t nfits) {
    size_t b = 0;
    for (int m = 0; m < c->N; ++m) b += (size_t)c->dims[m] * c->rank * sizeof(float);
    b += (size_t)c->N * c->rank * c->rank * sizeof(double);
    b += (size_t)c->rank * sizeof(double);
    b += (size_t)nfits * sizeof(double);
    return b;
}

}  // namespace

extern "C" sptt_status sptt_cpd_save(sptt_cpd *c, void *buf, size_t cap, size_t *needed) {
    clear_error();
    if (!c) return set_error(SPTT_ERR_BAD_ARG, "cpd is NULL");
    const int64_t nfits = c->iters < kFitHistory ? c->iters : kFitHistory;
    const size_t total = sizeof(CkpHeader) + ckp_payload(c, nfits);
    if (needed) *needed = total;
    if (!buf) return SPTT_OK;
    if (cap < total) return set_error(SPTT_ERR_BAD_ARG, "checkpoint buffer too small");
    unsigned char *out = static_cast<unsigned char *>(buf);
    unsigned char *p = out + sizeof(CkpHeader);
    for (int m = 0; m < c->N; ++m) {
        SPTT_CUDA(cudaMemcpy2DAsync(p, c->rank * sizeof(float), c->A[m], c->ld * sizeof(float),
                                    c->rank * sizeof(float), c->dims[m], cudaMemcpyDeviceToHost, c->st));
        p += (size_t)c->dims[m] * c->rank * sizeof(float);
    }
    for (int m = 0; m < c->N; ++m) {
        SPTT_CUDA(cudaMemcpyAsync(p, c->G[m], (size_t)c->rank * c->rank * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->st));
        p += (size_t)c->rank * c->rank * sizeof(double);
    }
    SPTT_CUDA(cudaMemcpyAsync(p, c->w.lambda, c->rank * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    p += (size_t)c->rank * sizeof(double);
    std::vector<double> ring(kFitHistory);
    SPTT_CUDA(cudaMemcpyAsync(ring.data(), c->fits, kFitHistory * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    for (int64_t j = 0; j < nfits; ++j) {
        const double f = ring[(c->iters - nfits + j) % kFitHistory];
        memcpy(p, &f, sizeof(double));
        p += sizeof(double);
    }
    CkpHeader h{};
    memcpy(h.magic, kCkpMagic, 8);
    h.version = kCkpVersion;
    h.nmodes = c->N;
    h.rank = c->rank;
    for (int m = 0; m < c->N; ++m) h.dims[m] = c->dims[m];
    h.iters = c->iters;
    h.nfits = nfits;
    h.checksum = fnv1a(out + sizeof(CkpHeader), total - sizeof(CkpHeader));
    memcpy(out, &h, sizeof(h));
    return SPTT_OK;
}

extern "C" sptt_status sptt_cpd_load(sptt_cpd *c, const void *buf, size_t len) {
    clear_error();
    if (!c || !buf) return set_error(SPTT_ERR_BAD_ARG, "cpd and buf must be non-NULL");
    if (len < sizeof(CkpHeader)) return set_error(SPTT_ERR_BAD_ARG, "checkpoint shorter than its header");
    CkpHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, kCkpMagic, 8) != 0) return set_error(SPTT_ERR_BAD_ARG, "not a checkpoint (magic)");
    if (h.version != kCkpVersion) return set_error(SPTT_ERR_BAD_ARG, "unsupported checkpoint version");
    if (h.nmodes != c->N || h.rank != c->rank) return set_error(SPTT_ERR_BAD_ARG, "checkpoint of another shape or rank");
    for (int m = 0; m < c->N; ++m)
        if (h.dims[m] != c->dims[m]) return set_error(SPTT_ERR_BAD_ARG, "checkpoint of another shape");
    if (h.iters < 0 || h.nfits < 0 || h.nfits > kFitHistory || h.nfits > h.iters)
        return set_error(SPTT_ERR_BAD_ARG, "corrupt checkpoint header");
    const size_t total = sizeof(CkpHeader) + ckp_payload(c, h.nfits);
    if (len != total) return set_error(SPTT_ERR_BAD_ARG, "checkpoint length does not match its header");
    const unsigned char *in = static_cast<const unsigned char *>(buf);
    if (fnv1a(in + sizeof(CkpHeader), total - sizeof(CkpHeader)) != h.checksum)
        return set_error(SPTT_ERR_BAD_ARG, "checkpoint checksum mismatch");
    // drop any captured iteration: the state it was captured against is replaced
    for (int p = 0; p < 2; ++p)
        if (c->graph[p]) {
            cudaGraphExecDestroy(c->graph[p]);
            c->graph[p] = nullptr;
        }
    const unsigned char *p = in + sizeof(CkpHeader);
    for (int m = 0; m < c->N; ++m) {
        SPTT_TRY(fill_zero_launch(c->A[m], (size_t)c->dims[m] * c->ld * sizeof(float), c->st));
        SPTT_CUDA(cudaMemcpy2DAsync(c->A[m], c->ld * sizeof(float), p, c->rank * sizeof(float),
                                    c->rank * sizeof(float), c->dims[m], cudaMemcpyHostToDevice, c->st));
        if (c->Ab[m]) SPTT_TRY(to_bf16_launch(c->A[m], c->Ab[m], c->dims[m] * c->ld, c->st));
        p += (size_t)c->dims[m] * c->rank * sizeof(float);
    }
    for (int m = 0; m < c->N; ++m) {
        SPTT_CUDA(cudaMemcpyAsync(c->G[m], p, (size_t)c->rank * c->rank * sizeof(double), cudaMemcpyHostToDevice,
                                  c->st));
        p += (size_t)c->rank * c->rank * sizeof(double);
    }
    SPTT_CUDA(cudaMemcpyAsync(c->w.lambda, p, c->rank * sizeof(double), cudaMemcpyHostToDevice, c->st));
    p += (size_t)c->rank * sizeof(double);
    std::vector<double> ring(kFitHistory, 0.0);
    for (int64_t j = 0; j < h.nfits; ++j) memcpy(&ring[(h.iters - h.nfits + j) % kFitHistory], p + j * 8, 8);
    SPTT_CUDA(cudaMemcpyAsync(c->fits, ring.data(), kFitHistory * sizeof(double), cudaMemcpyHostToDevice, c->st));
    const int64_t it = h.iters;
    SPTT_CUDA(cudaMemcpyAsync(c->iter_dev, &it, sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
    SPTT_CUDA(cudaStreamSynchronize(c->st));
    c->iters = h.iters;
    return SPTT_OK;
}
