/*
 * palmad.h -- C ABI of the GB300-native PALMAD discord engine (libpalmad.so).
 *
 * PALMAD (Zymbler & Kraeva, "High-performance Time Series Anomaly Discovery
 * on Graphics Processor") finds, for every subsequence length m in
 * [minL, maxL], the range discords of a time series: the length-m windows
 * whose z-normalised Euclidean distance to their nearest non-self match
 * (|i - j| >= m) is at least r (Sec. 2.1).  Each length runs the two DRAG
 * phases (candidate selection, then refinement to the exact nearest-neighbour
 * distance; Algorithm 2, parallelised as Algorithms 3-4) under the MERLIN
 * threshold schedule (Algorithm 1), with the window statistics carried from
 * m to m+1 by Eq. 7-8.
 *
 * Conventions used by every entry point:
 *   - Indices are 0-based (paper index i+1 <-> index i here).
 *   - Distances are plain z-normalised Euclidean distances ED_norm (not
 *     squared); r is in the same unit.  A window is a range discord when its
 *     nearest-neighbour distance d satisfies d >= r (Sec. 2.1); pruning uses
 *     the strict d < r of Algorithm 2.
 *   - A window with sigma <= 2^-22 |mu| is flat: two flat windows are at
 *     distance 0, a flat and a non-flat window at sqrt(2m).  A window with
 *     no non-self match (possible only when n - m + 1 < 2m) is never a
 *     discord.
 *   - Per length, the top-K are the range discords at that length's final r
 *     sorted by (distance desc, index asc) and taken greedily; with
 *     exclusive_topk set, each pick lies at least m away from earlier picks.
 *     MERLIN's schedule reads the distance of the K-th pick.  A length whose
 *     schedule reached r = 0 without K picks reports fewer (index -1,
 *     distance 0).
 *   - The schedule (Algorithm 1): r = 2 sqrt(minL), halved until K picks;
 *     for the next four lengths r = 0.99 d_{m-1}, times 0.99 on failure;
 *     afterwards r = mean - 2 sd of the previous five d (sample deviation),
 *     minus sd on failure (0.01 mean when sd = 0).  After 60 halvings, 3000
 *     shrink steps or r <= 0 the call uses r = 0.
 *   - Results are exact: discord indices equal those of an FP64 evaluation
 *     and distances are recomputed in FP64.
 *
 * Ownership: every pointer argument belongs to the caller and is only read
 * or written during the call.  The context owns all device memory it
 * allocates (grown on demand, freed by palmad_destroy) and one CUDA stream
 * (or borrows the caller's).  A context must not be used by two threads at
 * once.
 *
 * Errors: every entry point returns a palmad_status.  On a negative status
 * no output array has been written, and palmad_last_error() describes the
 * failure.
 */
#ifndef PALMAD_H
#define PALMAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct palmad_ctx palmad_ctx;

typedef enum {
    PALMAD_OK = 0,
    PALMAD_ERR_ARG = -1,         /* an argument violates the rules above */
    PALMAD_ERR_NONFINITE = -2,   /* T holds a NaN or an infinity */
    PALMAD_ERR_OOM = -3,         /* device or pinned host allocation failed */
    PALMAD_ERR_CUDA = -4,        /* a CUDA runtime call or kernel failed */
    PALMAD_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    PALMAD_ERR_UNSUPPORTED = -6, /* option or size not supported by the library */
    PALMAD_ERR_INTERNAL = -7,    /* an internal consistency check failed */
    PALMAD_ERR_TOO_LARGE = -8    /* size beyond the fixed scratch of palmad_topk_profile_noalloc */
} palmad_status;

/* Arithmetic of the pair evaluations (the candidate-select and refine dot
 * products).  Every form re-checks undecided pairs and recomputes the final
 * nearest-neighbour distances in FP64, so all forms return identical
 * results. */
typedef enum {
    PALMAD_PREC_FP32 = 0,   /* CUDA-core FP32 (plain form) */
    PALMAD_PREC_MIXED = 1   /* tensor-core refine where supported, else FP32 */
} palmad_precision;

typedef struct {
    int32_t struct_size;     /* sizeof(palmad_options); set by palmad_default_options */
    int32_t precision;       /* palmad_precision */
    int32_t exclusive_topk;  /* 1 (default): top-K picks mutually >= m apart; 0: plain top-K */
    int32_t batch_lengths;   /* 0/1: one DRAG call per schedule step (plain form);
                                W > 1: lengths run W at a time with a speculative r
                                and an exact host replay of the schedule (batched form) */
    double band_rel;         /* pairs with |d - r| < band_rel * r are re-checked in FP64
                                (floor; the build's FP32 error bound is applied on top);
                                default 1e-3, must lie in [1e-6, 0.1] */
    int32_t select_cap;      /* max columns a select strip scans past its first
                                (0 = default); pairs left unscanned go to refine */
    int32_t reserved_a;      /* reserved, must be 0 */
    int32_t profile;         /* 1: time every kernel launch with CUDA events
                                (palmad_get_stats) */
    int32_t pool_slots;      /* cap on the survivors refined at once (0 = as many as
                                about 4 GiB of per-survivor buffers holds, at most
                                131072); more survivors are refined in several rounds */
    int32_t direct_below;    /* 0: the plan's own split between the refine forms; k > 0:
                                every strip with fewer than k survivors uses the direct
                                form (k = 129 sends every survivor there) */
    int32_t tc_seed_min;     /* mixed precision: k > 0 gives refine strips with at least k
                                survivors top-row seeds from the tensor cores; 0 (default)
                                keeps every seed on the CUDA cores, which measured faster */
    int32_t seed_rows_max;   /* cap on tensor-core seed rows per refine round (0 = as many
                                as 1 GiB holds); strips past the cap seed on the CUDA cores */
    int32_t refine_seg;      /* columns per refine sweep work item: 0 = automatic (2048 for
                                passes holding >= 2e6 columns, else 1024), or 1024 / 2048 */
    int32_t knn_k;           /* k-th neighbour variant (the top-k discord definition of
                                Sec. 2.1 read literally): 0 or 1 = the nearest non-self
                                match (DRAG); k in 2..16 = every distance, range test, top-K,
                                heatmap and schedule value uses the k-th smallest distance
                                to the non-self matches, every match counted; a window with
                                fewer than k non-self matches is never a discord.  With
                                k > 1 no pair prunes (every window is refined over all its
                                columns), so a call costs a full pass over the pairs. */
    int32_t no_hints;        /* 0 (default): survivors of candidate select are first tried
                                against the columns near a pair that pruned the same window
                                at an earlier length (witness hints; results unchanged);
                                1: no hints */
    int32_t spec_scale;      /* batched form: the speculative r of a window of lengths lies
                                below the schedule's predicted first try by a margin
                                (2 sd of the last five nnDist, 6% of their mean or 1.5x the
                                recent shortfall, whichever is largest), and a length whose
                                schedule needs a lower r is rerun below that r by a similar
                                margin; this scales both margins in percent (0 = 100).
                                Smaller margins mean fewer survivors per pass and more
                                reruns; results are the same for any value */
    int32_t autotune;        /* 1: palmad_find_discords / _device use the options the
                                autotuner keeps for this workload bucket (precision,
                                k, exclusive, and log2 of n, minL, the number of lengths
                                and topK), tuning on the call's own series first when the
                                bucket has none (palmad_stats.tune_ms); 0 (default): the
                                options as given.  Results are the same either way */
    int32_t refine_rows;     /* rows per strip of the recurrence-form refine: 0 or 128
                                (default), or 256 (half the top-row dot products per row,
                                strips live until their last survivor is decided) */
    int32_t direct_below_long; /* as direct_below, for passes whose windows are longer than
                                256 (0 = direct_below): the direct form costs 2m flops per
                                survivor-column, so the best split depends on m */
    int32_t tc_group;        /* mixed precision: survivors per tensor-core MMA, 0 (64, or 32
                                for windows above 512), 32, 64, 128 (windows up to 256) or
                                256 (windows up to 128) */
    int32_t tc_chunks;       /* mixed precision: the direct refine of a round runs over the
                                columns in this many chunks (0 = 1), re-packing the
                                survivors still alive into full groups between chunks */
    int32_t tc_form;         /* mixed precision, tensor-core direct refine: 0 (default)
                                survivor-major where the windows allow it (up to 256 points:
                                128 survivors per MMA, 256 columns per tile, warp-specialised),
                                column-major otherwise; 1 column-major always; 2 survivor-
                                major where the windows allow it.  Results are the same */
} palmad_options;

/* Per-call counters of the most recent find/drag call. */
typedef struct {
    int32_t struct_size;        /* sizeof(palmad_stats) */
    int32_t lengths;            /* lengths processed */
    int64_t drag_calls;         /* DRAG evaluations the schedule asked for */
    int64_t device_passes;      /* select+refine passes actually launched */
    int64_t reruns;             /* batched form: lengths rerun with a lower r */
    int64_t select_pairs;       /* pairs evaluated by candidate select */
    int64_t refine_pairs;       /* pairs evaluated by refine (FP32 or tensor) */
    int64_t fp64_pairs;         /* pairs re-evaluated in FP64 */
    int64_t survivors;          /* candidates handed from select to refine (sum) */
    int64_t discords;           /* range discords at the final r (sum over lengths) */
    double max_fp32_rho_err;    /* max |rho_fast - rho_fp64| seen on re-checked pairs */
    double select_flops;        /* algorithmic FP32 work of select: 8 per valid pair (the
                                   diagonal update of the dot product, its correlation and
                                   distance, Eq. 6) + 2m per top-row seed */
    double refine_flops;        /* direct-form refine: 2m per evaluated pair */
    double sweep_flops;         /* recurrence-form refine: 8 per evaluated pair + 2m per
                                   direct dot product (top-row and first-column seeds) */
    /* per-kernel launch counts (always) and summed event times in ms
       (profile == 1 only); index = PALMAD_K_* */
    int64_t launches[12];
    double kernel_ms[12];
    int64_t seed_pairs;         /* tensor-core top-row seeds computed (strip x column) */
    double seed_flops;          /* their algorithmic work: 2m per seed */
    int64_t hint_pairs;         /* pairs evaluated by the witness-hint check */
    int64_t hint_kills;         /* survivors of select it removed before refine */
    int64_t refine_strips;      /* strips the recurrence-form refine swept (sum over rounds) */
    int64_t sweep_survivors;    /* survivors in those strips */
    double tune_ms;             /* autotuning done by this call (wall ms), 0 if none */
    int64_t direct_pairs;       /* of refine_pairs, those the direct form evaluated
                                   (FP32 or tensor cores) */
} palmad_stats;

/* What palmad_autotune timed and chose. */
typedef struct {
    int32_t struct_size;        /* sizeof(palmad_tune_report) */
    int32_t candidates;         /* configurations timed */
    int32_t block_lo, block_hi; /* first and last length of the timed blocks */
    double tune_ms;             /* wall time of the whole tuning */
    double best_ms;             /* summed block time of the chosen configuration */
    double default_ms;          /* summed block time of the options passed in */
} palmad_tune_report;

/* Kernel ids for palmad_stats.launches / kernel_ms. */
enum {
    PALMAD_K_STATS = 0,         /* window statistics init / Eq. 7-8 advance */
    PALMAD_K_SELECT = 1,        /* candidate select (Algorithm 3) */
    PALMAD_K_COMPACT = 2,       /* bitmap -> survivor list (Algorithm 4) */
    PALMAD_K_PLAN = 3,          /* survivor split (sweep / direct) + centred windows */
    PALMAD_K_REFINE_SWEEP = 4,  /* refine, recurrence form over dense strips (Algorithm 4) */
    PALMAD_K_REFINE_DIRECT = 5, /* refine, direct form over scattered survivors */
    PALMAD_K_RECHECK = 6,       /* FP64 re-check of the near-minimum pairs */
    PALMAD_K_GATHER = 7,        /* range discords of the call */
    PALMAD_K_TOPK = 8,          /* per-length top-K */
    PALMAD_K_HEAT = 9,          /* heatmap row write (Eq. 10) */
    PALMAD_K_HINT = 10,         /* witness-hint check of select survivors */
    PALMAD_K_SEED_TC = 11,      /* tensor-core top-row seeds of the refine sweep */
    PALMAD_K_COUNT = 12
};

/* Fills *opt with the defaults (FP32, exclusive top-K, plain form,
 * band_rel 1e-3).  Returns PALMAD_ERR_ARG when opt is NULL. */
palmad_status palmad_default_options(palmad_options *opt);

/* Creates a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to borrow (the context then never destroys it) or NULL to
 * create a private non-blocking stream.  *out is NULL on failure. */
palmad_status palmad_create(palmad_ctx **out, int device, void *cuda_stream);

/* Frees every resource of the context (NULL is a no-op). */
void palmad_destroy(palmad_ctx *ctx);

/* Message of the last failure on this context ("" if none); valid until the
 * next call on the context. */
const char *palmad_last_error(const palmad_ctx *ctx);

/*
 * MERLIN over one series (Algorithm 1; DRAG per schedule step, Algorithms
 * 2-4).  Host pointers.
 *   T           [n] float32 series, finite.
 *   n           series length; must satisfy n >= 2 * maxL.
 *   minL, maxL  3 <= minL <= maxL (Eq. 2: 3 <= m).
 *   topK        1 <= topK <= 1024.
 *   opt         NULL for the defaults.
 *   out_idx     [L * topK] int64, L = maxL - minL + 1, row-major by length;
 *               discord start indices, -1 where fewer than topK were found.
 *   out_nndist  [L * topK] double, their nearest-neighbour distances
 *               (ED_norm, FP64), 0.0 where the index is -1.
 *   out_count   [L] or NULL: number of range discords at each final r.
 *   out_r       [L] or NULL: the final r of each length.
 *   out_heatmap [L * (n - minL + 1)] float32 or NULL: row l = length
 *               minL + l holds nnDist^2 / (2m) at every range discord of
 *               that length and 0 elsewhere (Eq. 10).  It is computed in a
 *               device buffer of the same size that the context keeps for
 *               later calls (freed by palmad_destroy); pinned host memory
 *               makes the copy out fastest.
 */
palmad_status palmad_find_discords(palmad_ctx *ctx, const float *T, int64_t n, int32_t minL, int32_t maxL,
                                   int32_t topK, const palmad_options *opt, int64_t *out_idx,
                                   double *out_nndist, int64_t *out_count, double *out_r, float *out_heatmap);

/*
 * Resume a MERLIN run at length m0 (checkpoint / resume per length; the
 * schedule of Algorithm 1 depends on earlier lengths only through their
 * nnDist, Sec. 3.1).  The run started at length minL_sched; hist holds the
 * schedule inputs of lengths m0 - h .. m0 - 1, h = min(5, m0 - minL_sched):
 * per length, the nnDist of its K-th pick, or of its last pick when fewer,
 * or 0 when none (row l of out_nndist gives it).  The outputs cover lengths
 * m0..maxL exactly as rows m0 - minL_sched .. of the uninterrupted run; the
 * heatmap is [(maxL - m0 + 1) * (n - m0 + 1)], the uninterrupted rows cut
 * to that width.  Host pointers; other rules as palmad_find_discords, plus
 * 3 <= minL_sched <= m0 and hist values finite and >= 0.
 */
palmad_status palmad_find_discords_resume(palmad_ctx *ctx, const float *T, int64_t n, int32_t minL_sched, int32_t m0,
                                          int32_t maxL, int32_t topK, const palmad_options *opt, const double *hist,
                                          int64_t *out_idx, double *out_nndist, int64_t *out_count, double *out_r,
                                          float *out_heatmap);

/*
 * The values the schedule of Sec. 2.2 carries from each length to the next
 * (reading R6): per length, the nnDist of its topK-th pick, of its last pick
 * when fewer, 0 when none.  idx / nndist: [L * topK] results of a find call
 * (host); out: [L] (host).  A checkpoint at length m0 of a run that started
 * at minL is out[max(0, l0 - 5) .. l0 - 1], l0 = m0 - minL (the hist of
 * palmad_find_discords_resume).  No context, no GPU.  Errors: PALMAD_ERR_ARG.
 */
palmad_status palmad_schedule_inputs(const int64_t *idx, const double *nndist, int32_t L, int32_t topK,
                                     double *out);

/* As palmad_find_discords, but T and every output are DEVICE pointers on
 * the context's device; the call is stream-ordered on the context's stream
 * and returns after the results are written. */
palmad_status palmad_find_discords_device(palmad_ctx *ctx, const float *T_dev, int64_t n, int32_t minL,
                                          int32_t maxL, int32_t topK, const palmad_options *opt,
                                          int64_t *out_idx_dev, double *out_nndist_dev,
                                          int64_t *out_count_dev, double *out_r_dev, float *out_heatmap_dev);

/*
 * MERLIN over `count` independent series (the batched form's multi-series
 * entry).  Host pointers; series s has T[s][0..n[s]), lengths
 * minL[s]..maxL[s] and writes out_idx[s] / out_nndist[s]
 * ([L_s * topK] each) and, when the arrays are non-NULL, out_count[s] and
 * out_r[s] ([L_s] each).  Same rules per series as palmad_find_discords.
 */
palmad_status palmad_find_discords_batch(palmad_ctx *ctx, int32_t count, const float *const *T, const int64_t *n,
                                         const int32_t *minL, const int32_t *maxL, int32_t topK,
                                         const palmad_options *opt, int64_t *const *out_idx,
                                         double *const *out_nndist, int64_t *const *out_count,
                                         double *const *out_r);

/*
 * Autotuner (no counterpart in the paper, which fixes its launch shapes):
 * chooses the pass configuration for one series and length range --
 * lengths per pass (batch_lengths) and the batched form's speculation margin
 * (spec_scale), the select cap, the refine segment and the refine-form split
 * (direct_below, direct_below_long), the refine strip height (refine_rows) and the
 * column chunks of the tensor-core direct refine (tc_chunks) -- by timing
 * candidates one setting at a time on blocks of up to 12 lengths at the
 * start, a third, two thirds and the end of [minL, maxL] of the caller's
 * series; every block after the first resumes from the schedule inputs of
 * its preceding lengths, so it meets the thresholds the whole run meets.
 * Every candidate returns the same results; only the time differs.
 *   T_dev       [n] float32 device series (the context's device).
 *   base        options to start from (NULL: defaults); precision, k,
 *               exclusive_topk and band_rel are kept as given.
 *   out_opt     receives the chosen options (base with the tuned fields).
 *   report      NULL or a palmad_tune_report with struct_size set.
 * The choice is also kept in the context for the workload bucket of
 * (n, minL, maxL, topK, base) (see palmad_options.autotune).  Synchronous;
 * takes tens of block runs (seconds on 10^6-point series).
 */
palmad_status palmad_autotune(palmad_ctx *ctx, const float *T_dev, int64_t n, int32_t minL, int32_t maxL,
                              int32_t topK, const palmad_options *base, palmad_options *out_opt,
                              palmad_tune_report *report);

/*
 * One DRAG call (Algorithm 2; Algorithms 3-4): every range discord of
 * length m at threshold r, in ascending index order.  Host pointers.
 *   T [n] float32, finite; 3 <= m; n >= 2m.
 *   out_idx / out_nndist: [cap] arrays receiving the first min(cap, count)
 *   discords (index, FP64 distance); *out_count receives the full count.
 */
palmad_status palmad_drag(palmad_ctx *ctx, const float *T, int64_t n, int32_t m, double r, const palmad_options *opt,
                          int64_t *out_idx, double *out_nndist, int64_t cap, int64_t *out_count);

/*
 * One DRAG call split over ranks (the cluster DRAG of the paper's related
 * work, Sec. 1): each rank runs one phase on a shard of the pair space and
 * the ranks exchange one array per phase.
 *
 * palmad_drag_select_shard: candidate select (Algorithm 2's first phase;
 * Algorithm 3) for the rows [row_lo, row_hi) -- every pair (i, j), i in the
 * rows, j >= i + m, that a select strip scans.  out_bits [(N + 31) / 32]
 * uint32 (host; bit i of word w is window 32 w + i, N = n - m + 1): set for
 * the windows no pair of this shard pruned.  The candidates of the whole
 * call are the bitwise AND of every rank's bitmap (row ranges that cover
 * [0, N) between them; rounded out to whole 128-row strips).
 *
 * palmad_drag_refine_shard: refinement (the second phase; Algorithm 4) of
 * the candidates cand_bits (host, the ANDed bitmap) against the columns
 * [col_lo, col_hi) only.  out_nn [N] double (host): -1 for a candidate some
 * pair of these columns prunes (distance < r), else its FP64
 * nearest-neighbour distance over the non-self columns of the range (+inf
 * when there is none), +inf for a window that is no candidate.  With
 * column ranges that cover [0, N), the elementwise minimum over the ranks
 * is -1 for every pruned candidate and the exact nearest-neighbour
 * distance of every other one: the range discords at r are the windows
 * whose minimum is >= r (every finite one when r <= 0), as palmad_drag
 * returns them.
 *
 * Host pointers; T, m, r as palmad_drag; FP32 forms only (precision MIXED
 * runs the FP32 direct form here), nearest-neighbour distance only
 * (knn_k > 1: PALMAD_ERR_UNSUPPORTED).  Errors: PALMAD_ERR_ARG for a bad
 * range or pointer.
 */
palmad_status palmad_drag_select_shard(palmad_ctx *ctx, const float *T, int64_t n, int32_t m, double r,
                                       int64_t row_lo, int64_t row_hi, const palmad_options *opt,
                                       uint32_t *out_bits);
palmad_status palmad_drag_refine_shard(palmad_ctx *ctx, const float *T, int64_t n, int32_t m, double r,
                                       const uint32_t *cand_bits, int64_t col_lo, int64_t col_hi,
                                       const palmad_options *opt, double *out_nn);

/*
 * Greedy top-K range discords of a nearest-neighbour profile the caller
 * already holds, WITHOUT ANY ALLOCATION.  The paper has no counterpart: it is
 * for callers that cannot call cudaMalloc, such as code running while
 * another component owns all device memory through its own allocator, or a
 * latency-critical path that cannot afford cudaMalloc's implicit device
 * synchronisation.  It needs no context.
 *   nn_dev         [N] FP64 nearest-neighbour distances (device); +inf or NaN
 *                  marks a window without a nearest neighbour.
 *   N              1 <= N <= PALMAD_NOALLOC_MAX_WINDOWS; larger N returns
 *                  PALMAD_ERR_TOO_LARGE.
 *   m, r, K        window length (for the exclusion zone), threshold and
 *                  1 <= K <= 1024.  Range discords: finite entries >= r (every
 *                  finite entry when r <= 0), picked as in
 *                  palmad_find_discords (distance desc, index asc; with
 *                  exclusive != 0 each pick >= m from earlier picks).
 *   out_idx_dev    [K] int64 picks, -1 past the last one (device).
 *   out_nn_dev     [K] double, their distances, 0.0 past the last one (device).
 *   out_count_dev  [1] int64 number of range discords (device) or NULL.
 *   cuda_stream    stream to run on (NULL: the default stream).
 * The call runs on the calling thread's current CUDA device, which must be
 * the device holding nn_dev, the outputs and cuda_stream.
 * The call is asynchronous: results are ready once the stream reaches them.
 * Its one intermediate buffer is a fixed device array of the library
 * (PALMAD_NOALLOC_MAX_WINDOWS x 12 bytes per GPU, resident until the process
 * exits).  The first call on each device looks up that array's address with
 * cudaGetSymbolAddress, so make it before any stream capture.  All calls on
 * a device share the array: calls whose kernels overlap on the GPU race.
 */
#define PALMAD_NOALLOC_MAX_WINDOWS (1 << 18)
palmad_status palmad_topk_profile_noalloc(const double *nn_dev, int64_t N, int32_t m, double r, int32_t K,
                                          int32_t exclusive, int64_t *out_idx_dev, double *out_nn_dev,
                                          int64_t *out_count_dev, void *cuda_stream);

/*
 * The most interesting discords across lengths (Eq. 11, Sec. 5), from a
 * discord heatmap the caller holds on the device (the out_heatmap_dev of
 * palmad_find_discords_device, Eq. 10).  No allocation, no context.
 *   heat_dev       [L * W] float32, row l = length minL + l (device).
 *   score_dev      [W] float32 out: interest of each index, the largest
 *                  heatmap value over the lengths (device, caller-owned).
 *   best_m_dev     [W] int32 out: the smallest length reaching it (device).
 *   out_idx_dev    [K] int64 picks, -1 past the last one (device).
 *   out_m_dev      [K] int32 their lengths, 0 past the last one (device).
 *   out_score_dev  [K] float32 their interest, 0 past the last one (device).
 * Picks are greedy by (interest desc, index asc) among indices of positive
 * interest; with exclusive != 0 a pick's window [i, i + m) overlaps no
 * earlier pick's window.  1 <= K <= 1024.  Asynchronous on cuda_stream
 * (NULL: the default stream).  Errors: PALMAD_ERR_ARG, PALMAD_ERR_CUDA.
 */
palmad_status palmad_discord_interest(const float *heat_dev, int32_t L, int64_t W, int32_t minL, int32_t K,
                                      int32_t exclusive, float *score_dev, int32_t *best_m_dev,
                                      int64_t *out_idx_dev, int32_t *out_m_dev, float *out_score_dev,
                                      void *cuda_stream);

/* Counters of the most recent find/drag call on this context. */
palmad_status palmad_get_stats(const palmad_ctx *ctx, palmad_stats *out);

/*
 * Measured arithmetic throughput of GPU `device` in TFLOP/s (2 flops per
 * fused multiply-add lane): the best of five timed launches of independent
 * FMA chains filling every SM.  It denominates the roofline of the pair
 * kernels, which are bound by FP32 arithmetic.  Synchronises the device;
 * allocates and frees a small buffer; not for a hot path.
 *   kind  PALMAD_PEAK_FP32 (scalar fma.rn.f32), PALMAD_PEAK_FP32X2 (packed
 *         fma.rn.f32x2) or PALMAD_PEAK_FP64.
 * Errors: PALMAD_ERR_ARG for a NULL pointer or unknown kind, PALMAD_ERR_CUDA.
 */
typedef enum { PALMAD_PEAK_FP32 = 0, PALMAD_PEAK_FP32X2 = 1, PALMAD_PEAK_FP64 = 2 } palmad_peak_kind;
palmad_status palmad_measure_peak(int device, int32_t kind, double *tflops);

/* Library version string. */
const char *palmad_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PALMAD_H */
