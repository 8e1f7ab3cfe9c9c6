/*
 * asaga.h -- C ABI of a GB300 (sm_103a) solver for lock-free asynchronous
 * Sparse SAGA (ASAGA; Leblond, Pedregosa, Lacoste-Julien, arXiv:1606.04809).
 *
 * Problem (Eq. finiteSum with the model of Sec. 4.1):
 *     min_x f(x) = 1/n sum_i phi_i(a_i . x) + lambda/2 |x|^2,
 *     logistic phi_i(z) = log(1 + exp(-b_i z)), b_i in {-1,+1},
 *     squared  phi_i(z) = (z - y_i)^2 / 2.
 * Update (Eq. SparseSAGA with the projected l2 term of Sec. 4.2, run as in
 * Algorithm 2): for a uniformly sampled row i with support S_i,
 *     delta = phi'_i(a_i . x^) - alpha_i,
 *     x_v   -= gamma (delta a_iv + D_v abar_v + lambda D_v x^_v),  v in S_i,
 *     abar_v += delta a_iv / n,                                   v in S_i,
 *     alpha_i = phi'_i(a_i . x^),
 * where x^ is the (inconsistent) value read for the dot product and
 * D_v = n / |{i : v in S_i}| (Sec. 2), 0 for columns that no row touches.
 * Many GPU warps run this update concurrently without locks; the adds to x
 * and abar are atomic (Sec. 3.3, Property "atomicity").
 *
 * Conventions for every entry point:
 *   - the library owns all device state; it copies the problem at create
 *     time and never keeps a caller pointer after a call returns;
 *   - every call returns an asaga_status and never aborts the process;
 *     asaga_last_error() gives a one-line reason for the last failure;
 *   - host pointers are plain CPU memory (pinned or not); "device" pointers
 *     are CUDA global-memory addresses on the current device;
 *   - a context is used by one host thread at a time.
 */
#ifndef ASAGA_H
#define ASAGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque solver context (one problem, its device copy and the solver state). */
typedef struct asaga_ctx asaga_ctx;

typedef enum {
    ASAGA_OK = 0,
    ASAGA_EINVAL = 1,         /* invalid argument or problem; nothing changed  */
    ASAGA_ENOMEM = 2,         /* a device allocation failed                    */
    ASAGA_ECUDA = 3,          /* a CUDA call failed (no GPU, launch error, ...) */
    ASAGA_ETIMEOUT = 4,       /* the run stopped at options.timeout_s          */
    ASAGA_EDIVERGED = 5,      /* objective or iterate became non-finite        */
    ASAGA_ENOTCONVERGED = 6,  /* max_epochs reached before the target          */
    ASAGA_ECANCELLED = 7      /* asaga_cancel / asaga_batch_cancel stopped it  */
} asaga_status;

typedef enum { ASAGA_LOSS_LOGISTIC = 0, ASAGA_LOSS_SQUARED = 1 } asaga_loss;

typedef enum { ASAGA_F64 = 0, ASAGA_F32 = 1, ASAGA_BF16 = 2, ASAGA_F16 = 3 } asaga_dtype;

/* Row sampling of the asynchronous updates (asaga_options.sampling). */
typedef enum { ASAGA_SAMPLE_UNIFORM = 0, ASAGA_SAMPLE_PERMUTATION = 1 } asaga_sampling;

/*
 * The data matrix A (n rows a_i, d columns) in CSR form, and the labels.
 *   row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz;
 *   col_idx  int32[nnz], each in [0, d), distinct within a row (any order);
 *   values   nnz numbers of type values_dtype (F64, F32, BF16 or F16), finite;
 *   labels   float64[n]: +1/-1 for logistic, finite targets for squared.
 * The support S_i of row i is its stored pattern (an explicitly stored 0
 * counts as support).  dense = 1 means values holds n*d numbers row-major
 * and row_ptr/col_idx are NULL.  on_device = 1 means all four arrays are
 * device pointers; they are read only during asaga_create.
 */
typedef struct {
    int64_t n, d, nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const void *values;
    asaga_dtype values_dtype;
    const double *labels;
    int dense;
    int on_device;
} asaga_problem;

/*
 * Solver options; asaga_default_options() fills every field.
 *   loss                 the phi_i above.
 *   lambda               l2 weight, >= 0 (the paper uses 1/n, Sec. 4.2).
 *   gamma                step size; <= 0 picks 1/(3L), where L = max_i (c |a_i|^2
 *                        + lambda max_{v in S_i} D_v), c = 1/4 (logistic) or 1
 *                        (squared), is the smoothness constant of the component
 *                        the sparse update samples (its l2 part is projected
 *                        and reweighted by D_i, Sec. 4.2).
 *   storage_dtype        device type of A's values: F32, BF16 or F16 (the
 *                        iterate, memory and dot products are always F32).
 *   max_warps            concurrent solver warps; 0 = automatic
 *                        (a bound derived from n keeps the overlap well below
 *                        n/10, the condition of Theorem 2).
 *   deterministic        1 = one warp processes the updates strictly in
 *                        order (bitwise reproducible; parity mode).
 *   seed                 seed of the row sampler (counter-based SplitMix64).
 *   epochs_per_segment   epochs between float64 objective evaluations.
 *   abar_recompute_every segments between float64 recomputations of abar
 *                        from the memory (0 = never), counted over the
 *                        context's life across asaga_run calls (restarted
 *                        by asaga_set_state and asaga_autotune).
 *   timeout_s            wall-clock limit of one asaga_run (0 = none).
 *   cuda_stream          cudaStream_t to run on; NULL = a stream the library
 *                        creates.  All work of a context is ordered on it.
 *   column_stride        spacing of the per-column state {x_v, abar_v} in
 *                        8-byte units (1 = packed; 16 = one 128-byte line per
 *                        column, which spreads atomics on very small d);
 *                        0 = automatic (16 when d <= 1024, else 1).
 *   plain_writes         1 = replace the atomic adds by non-thread-safe
 *                        load-add-store updates, which lose concurrent adds:
 *                        the comparison of App. G.2 ("Necessity of
 *                        compare-and-swap"), for diagnostics only; 0 = atomic.
 *   sampling             ASAGA_SAMPLE_UNIFORM (default): rows drawn uniformly
 *                        with replacement, as Algorithm 2 does;
 *                        ASAGA_SAMPLE_PERMUTATION: every epoch visits each row
 *                        once, in a seeded pseudo-random order (a variant
 *                        the paper does not analyse; see asaga_sample_rows).
 *   compact              1 = store A compactly where that changes no number
 *                        the solver computes with: uint16 column indices when
 *                        d <= 65536, and one float32 value per row when every
 *                        stored value of each row is equal (binary rows
 *                        scaled to unit norm); 0 (default) = int32 indices and
 *                        one value per entry.  A batch compacts only what all
 *                        its instances allow (options[0].compact).
 */
typedef struct {
    asaga_loss loss;
    double lambda;
    double gamma;
    asaga_dtype storage_dtype;
    int max_warps;
    int deterministic;
    uint64_t seed;
    int epochs_per_segment;
    int abar_recompute_every;
    double timeout_s;
    void *cuda_stream;
    int column_stride;
    int plain_writes;
    int sampling;
    int compact;
} asaga_options;

/* Outcome of asaga_run.  seconds = wall time of the call; solver_seconds and
 * eval_seconds split the device time (CUDA events) between the update kernel
 * and the float64 evaluations.  abar_drift = max_v |abar_v - (1/n) sum_i
 * alpha_i a_iv| seen at the last recomputation (0 if none ran). */
typedef struct {
    double epochs;
    double seconds;
    double solver_seconds;
    double eval_seconds;
    double f_last;
    double rel_subopt;
    int64_t updates;
    double abar_drift;
    int64_t segments;
    int64_t kernel_launches;
} asaga_result;

/* Static facts about a context. */
typedef struct {
    int64_t n, d, nnz;
    double L;            /* max_i (c |a_i|^2 + lambda max_{v in S_i} D_v), stored values */
    double gamma;        /* step size in use                                    */
    double delta;        /* max_v |{i : v in S_i}| / n (Sec. 3.4, "Sparsity")   */
    int warps;           /* concurrent solver warps of asaga_run                */
    int column_stride;   /* per-column state spacing in 8-byte units            */
    int64_t device_bytes;/* device memory held by the context                   */
    int64_t max_row_len; /* longest row                                          */
    int n_hot;           /* frequent columns accumulated in shared memory by the
                            float64 scatters                                    */
    int warps_per_block; /* update kernel blocks: 8 warps, or fewer when the
                            autotuner found the warps faster spread over the SMs */
    int col_index_bytes; /* 4, 2 (compact uint16 indices) or 0 (dense)          */
    int row_values;      /* 1 when A is held as one value per row (compact)     */
    int64_t row_threshold; /* rows longer than this take the multi-warp row path
                              (0: every row; -1: none; see asaga_set_row_path)  */
    int row_group;       /* warps per core of the multi-warp row path (1: none)  */
    int draw_ahead;      /* 1: each core draws its next row while an update's
                            gathers are in flight (asaga_set_draw_ahead)        */
} asaga_info;

/* Outcome of asaga_autotune. */
typedef struct {
    int warps;           /* chosen number of concurrent solver warps            */
    double gamma;        /* chosen step size                                    */
    double score;        /* higher is better; -1 when no trial settled          */
    int trials;          /* (warps, gamma) pairs tried                          */
    double seconds;      /* device time spent in the trials                      */
    int64_t row_threshold; /* chosen row path (asaga_set_row_path): threshold... */
    int row_group;       /* ...and warps per multi-warp core                     */
    int draw_ahead;      /* chosen draw placement (asaga_set_draw_ahead)         */
} asaga_tune_result;

/* Fills *opt with defaults: logistic, lambda 0, gamma 1/(3L), F32 storage,
 * automatic warps, asynchronous, seed 0, 1 epoch per segment, no abar
 * recomputation, no timeout, own stream, automatic column stride. */
void asaga_default_options(asaga_options *opt);

/* Validates the problem, copies it to the device in options->storage_dtype,
 * computes D, L and gamma, and zeroes x, alpha and abar (Sec. 2: x0 = 0,
 * alpha0 = 0).  On success *out owns the context (free with asaga_destroy).
 * EINVAL: NULL pointer, n or d < 1, nnz < 0, malformed CSR (row_ptr not
 * monotone, column out of range or repeated in a row), non-finite value or
 * label, logistic label not +-1, lambda < 0 or non-finite, unsupported dtype.
 * ECUDA / ENOMEM: no usable GPU or not enough device memory. */
asaga_status asaga_create(asaga_ctx **out, const asaga_problem *problem,
                          const asaga_options *options);

/* Runs asynchronous Sparse SAGA (Algorithm 2) in segments of
 * options.epochs_per_segment epochs (an epoch is n updates), evaluating f in
 * float64 after each segment.  Stops when target_rel_subopt > 0 and
 * (f - f_star) / |f_star| <= target_rel_subopt (returns OK), or after
 * max_epochs (returns OK if target_rel_subopt <= 0, else ENOTCONVERGED).
 * Continues from the current state; the sampler stream continues too.
 * EDIVERGED if f turns non-finite; ETIMEOUT at options.timeout_s;
 * ECANCELLED after asaga_cancel; ECUDA if the kernel found a malformed row
 * range on the device.  After ETIMEOUT or ECANCELLED, res->updates and the
 * sampler position count the stopped segment as if it had completed.
 * res may be NULL. */
asaga_status asaga_run(asaga_ctx *ctx, double max_epochs, double target_rel_subopt,
                       double f_star, asaga_result *res);

/* Asks the asaga_run in progress on ctx (called from another host thread)
 * to stop: the update kernel polls a flag in mapped host memory every 256
 * updates of each warp, and asaga_run returns ASAGA_ECANCELLED after the
 * segment, with the state as the finished updates left it and the context
 * usable.  Thread-safe; a request made while no run is in progress is
 * dropped when the next asaga_run starts.  The paper has no counterpart.
 * EINVAL: ctx NULL. */
asaga_status asaga_cancel(asaga_ctx *ctx);

/* Picks the number of concurrent warps and the step size for asaga_run.
 * The overlap tau of asynchronous updates grows with the number of warps,
 * and the largest stable step shrinks with tau (Theorem 2: a <= a*(tau)).
 * Measured on a GB300: warps x step has a stability frontier, above which
 * the iterate stalls on a plateau (logistic loss) or diverges (squared loss);
 * below it the epochs needed depend on the step only, while the epoch time
 * falls with the number of warps.  Steps are gamma0 * 2^(-k/2), gamma0 =
 * options.gamma or 1/(3L), k = -3..16 (the largest, 0.94/L, below 1/L).
 * Each trial starts from x = 0,
 * alpha = 0 and records the float64 |grad f|^2 after every epoch:
 *  1. frontier: at min(1024, n/64, resident) warps (Theorem 2 asks for
 *     tau < n/10, and tau measures 1.5 to 4 times the warps; no candidate
 *     exceeds n/64 warps), bisection over k for the
 *     largest step whose 16-epoch trial converges (|grad f|^2 shrinks by
 *     1e6, or its log falls with a least-squares t-statistic >= 3.5);
 *     if none does, again with 8x fewer warps (twice at most);
 *  2. race: warp counts W = probe * 2^j at one notch inside the frontier
 *     (W x step constant), scored by the predicted update time for
 *     |grad f|^2 to shrink by 1e10 (the least-squares trend of the trial's
 *     last two thirds, if its t-statistic is >= 3); trials run trial_epochs
 *     epochs (<= 0: 24), more (up to 8x, within 250 ms of update time)
 *     while the prediction lies beyond twice their length, and stop when
 *     slower than 1.5x the best so far;
 *     A candidate with fewer warps (a larger step) wins within a 1.2x
 *     tolerance, one with more warps must be 1.2x faster.  If no candidate
 *     settles, the race is run again one notch further inside (twice at
 *     most);
 *  3. smaller steps at the winning warp count while they score better (if
 *     none does and the warps are at most n/256, one notch larger, kept if
 *     it scores better), then a
 *     confirmation trial of twice the length that must still show a
 *     downward trend (else one notch smaller a step, three times at most);
 *     where the warps exceed n/256 and the winner's predicted epochs are
 *     within 16/3 race lengths, it runs to 1.5x those epochs and must
 *     bring |grad f|^2 down by 1e10 instead;
 *  4. the update kernel's block shape at the winner: eight warps per block
 *     or the warps spread evenly over the SMs, whichever epoch is faster;
 *  5. the row path at the winner (the same warps and step, regrouped into
 *     cores; see asaga_set_row_path): multi-warp cores of G = 2, 4, 8 warps
 *     for every row (when the mean row has at least 32 G entries) or for the
 *     rows longer than T = 128, 256, 512 entries (when they hold at least 2%
 *     of the nonzeros), each timed over two epochs after one untimed; the
 *     two fastest that beat single warps by 3% run a race trial in turn,
 *     and the first whose predicted time beats the winner's by 3% is kept;
 *  6. the draw placement at the winner (asaga_set_draw_ahead), where the
 *     warps are at most n/256: two trials
 *     of twice the race length with the next row drawn inside the updates'
 *     windows; kept if both bring |grad f|^2 down by 1e10 and the slower
 *     one's update time to that level beats the winner's prediction by 3%
 *     (the longer window adds
 *     overlap, which can put the same warps and step past the frontier, and
 *     such a run can fall steadily for dozens of epochs before it stalls).
 * If no trial converges, the defaults stay.  score = 1 / (predicted
 * seconds of the winner), -1 when none settled.  Leaves the state at x = 0,
 * alpha = 0, abar = 0 (sampler position 0) with the chosen pair in use.
 * EINVAL in deterministic mode. */
asaga_status asaga_autotune(asaga_ctx *ctx, double trial_epochs, asaga_tune_result *res);

/* The rows that updates t_begin .. t_begin+count-1 of a context with this
 * seed, n and sampling visit, computed by the solver's own device sampler
 * (the same function the update kernel calls) and written to rows[count]
 * (host memory).  A context numbers its updates from 0 (after asaga_create
 * and asaga_autotune; asaga_set_state sets the count).
 *  - ASAGA_SAMPLE_UNIFORM (Algorithm 2 samples i uniformly, with
 *    replacement): u_t = the (t+1)-th output of SplitMix64 (Steele, Lea and
 *    Flood, OOPSLA 2014) seeded with `seed`, row = floor(u_t n / 2^64).
 *  - ASAGA_SAMPLE_PERMUTATION: epoch e = floor(t / n) visits position
 *    p = t - e n at row pi_e(p), where pi_e is a bijection of [0, n): a
 *    4-round balanced Feistel network on 2h bits (h >= 1 the smallest with
 *    4^h >= n; left half = high h bits), round r = 0..3 mapping
 *    (L, R) -> (R, L xor (M((k_e xor R) + (r+1) G) mod 2^h)), iterated until
 *    the value falls below n (cycle walking).  G = 0x9E3779B97F4A7C15, M is
 *    SplitMix64's output mix, k_e = the (e+1)-th output of SplitMix64 seeded
 *    with seed xor 0xD1B54A32D192ED03.
 * EINVAL: n < 1 (or n > 2^62 with permutation sampling), count < 0, rows
 * NULL with count > 0, unknown sampling.  ECUDA / ENOMEM: no usable GPU.
 * The paper has no counterpart of this call; it exposes the sampler for
 * checking and for replaying a run's row sequence. */
asaga_status asaga_sample_rows(uint64_t seed, int64_t n, int sampling, uint64_t t_begin, int64_t count,
                               int64_t *rows);

/* Overlap of the asynchronous updates (the tau of Assumption 1). */
typedef struct {
    int64_t updates;        /* updates traced                                        */
    int warps;              /* concurrent warps of the run                           */
    double tau_mean;        /* mean over updates of the number of others overlapping */
    double tau_max;         /* largest such number                                   */
    double tau_paper;       /* max over windows of 100 updates of the mean (App. E.2) */
    double window_ns_mean;  /* mean time from an update's reads to its writes        */
    double seconds;         /* device time of the traced launch                      */
} asaga_overlap;

/* Runs `epochs` epochs like asaga_run (same schedule; the state advances) while
 * lane 0 of every warp records %globaltimer just before an update's reads and
 * just after its writes are issued; two updates overlap when those intervals
 * intersect.  tau_paper follows App. E.2: the average overlap over windows of
 * 100 consecutive updates, maximised over windows (a lower bound on the true
 * maximum).  Needs 16 bytes of scratch per update (allocated and freed on the
 * context's stream) and no objective evaluation.  EINVAL: epochs <= 0, fewer
 * than 2 updates, out NULL. */
asaga_status asaga_measure_overlap(asaga_ctx *ctx, double epochs, asaga_overlap *out);

/* As asaga_measure_overlap, and also copies the raw trace to times (host
 * memory, at least 2 x updates values): times[2t] and times[2t + 1] are the
 * %globaltimer values (ns) just before update t's reads and just after its
 * writes were issued, t = 0 .. updates - 1 in the launch's update order.
 * The estimates follow from it: overlap(t) = #{r != t : times[2r] <=
 * times[2t+1] and times[2r+1] >= times[2t]}; tau_mean its mean, tau_max
 * its maximum; tau_paper the largest mean over consecutive windows of 100
 * updates in start order (ties in update order), a trailing partial window
 * left out; window_ns_mean the mean of times[2t+1] - times[2t].  EINVAL as
 * asaga_measure_overlap, or capacity < 2 x updates with times not NULL. */
asaga_status asaga_measure_overlap_trace(asaga_ctx *ctx, double epochs, asaga_overlap *out, uint64_t *times,
                                         int64_t capacity);

/* Service time of one column's state line under the update's access
 * pattern: the 8-byte read of {x^_v, abar_v} and then the 2-wide float
 * reduction into x_v and abar_v that depends on it (Algorithm 2's read of x^
 * and write of x and abar, for one column v).  `warps` warps each repeat the
 * pair `pairs` times on one line; *ns_per_pair = elapsed device time /
 * (warps x pairs).  With enough warps the line saturates and this is the
 * time its L2 slice takes per pair, so a problem whose most frequent column
 * is in c rows needs at least c x ns_per_pair per epoch (the update kernel's
 * roofline when that column is in most rows).  Allocates and frees 256 bytes
 * of device memory and a stream on the current device, and waits for the
 * probe.  EINVAL: warps outside [1, 65536], pairs < 1, ns_per_pair NULL
 * (asaga_last_error(NULL) says which); ECUDA: a CUDA error. */
asaga_status asaga_probe_line_rate(int warps, int64_t pairs, double *ns_per_pair);

/* Deterministic replay: runs one update per entry of idx (row indices in
 * [0,n)), strictly in order, on a single warp.  idx is a host pointer if
 * idx_on_device = 0, else a device pointer.  This is the serial Sparse SAGA
 * iteration in float32 and matches a float64 serial run on the same index
 * sequence to rounding.  EINVAL on an index out of range (checked on the
 * host for host input; on the device otherwise, with no update applied
 * past the bad entry). */
asaga_status asaga_run_indices(asaga_ctx *ctx, const int64_t *idx, int64_t count,
                               int idx_on_device);

/* f(x) at the current iterate, computed on the GPU in float64 (float32 x and
 * stored values widened exactly). */
asaga_status asaga_objective(asaga_ctx *ctx, double *f);

/* grad f(x) = 1/n A^T phi'(A x) + lambda x in float64 on the GPU.  If grad is
 * not NULL it receives d float64 values (host memory); norm2 (may be NULL)
 * receives |grad f(x)|^2. */
asaga_status asaga_full_grad(asaga_ctx *ctx, double *grad, double *norm2);

/* Recomputes abar = (1/n) sum_i alpha_i a_i from the memory with float64
 * accumulation (cancelling the float32 drift of the running sums) and stores
 * it.  drift (may be NULL) receives max_v |abar_v(before) - abar_v(exact)|. */
asaga_status asaga_recompute_abar(asaga_ctx *ctx, double *drift);

/* Copies the state to host memory: x and abar (d floats each), alpha (n
 * floats).  Any pointer may be NULL. */
asaga_status asaga_get_state(asaga_ctx *ctx, float *x, float *abar, float *alpha);

/* Overwrites the state from host memory (checkpoint restore); any pointer may
 * be NULL to keep that part.  The sampler position is set to updates_done. */
asaga_status asaga_set_state(asaga_ctx *ctx, const float *x, const float *abar,
                             const float *alpha, int64_t updates_done);

asaga_status asaga_get_info(asaga_ctx *ctx, asaga_info *info);

/* Sets the schedule asaga_run uses, e.g. one asaga_autotune found for the
 * same problem earlier (asaga_get_info reports warps, gamma and
 * warps_per_block): warps >= 1 (at most the resident maximum), gamma > 0,
 * warps_per_block 0 (eight warps per block) or the value asaga_get_info
 * reported (spread over the SMs when below 8).  EINVAL on other values or
 * in deterministic mode (one warp). */
asaga_status asaga_set_schedule(asaga_ctx *ctx, int warps, double gamma, int warps_per_block);

/* The multi-warp row path (Algorithm 2's update of one row spread over the
 * warps of a block).  Every concurrent update runs on a "core": a single
 * warp, except that rows with more than `threshold` entries are updated by
 * cores of `group` warps of one block: lane l of warp w owns the row's
 * entries 32 (q group + w) + l,
 * q = 0, 1, ...; the warps add their partial dot products a_i . x^ in shared
 * memory behind a named barrier and scatter their own entries with the same
 * delta.  A core of g warps stages 256 g entries of a row in shared memory
 * and holds them in registers; every entry's state is still read once per
 * update, the entries past that in a per-core scratch array the library
 * allocates.
 *   threshold  -1: no row takes the multi-warp path (the default); 0: every
 *              row; T > 0: rows longer than T entries, the others on
 *              single-warp cores.
 * The path regroups the warps of the schedule (asaga_set_schedule; with
 * T > 0 the long rows' cores get the share of the warps that those rows
 * hold of the nonzeros) and keeps their number: measured on a GB300, the
 * stability frontier lies at a product of total warps and step, not of
 * concurrent updates, so a step that converges on W single warps also does
 * on W warps grouped by 4.
 *              Each path's cores take the launch's updates t = core,
 *              core + cores, ... whose rows belong to that path, so every
 *              sampled update is applied exactly once (Algorithm 2's row
 *              sequence is unchanged; only its assignment to cores is).
 *   group      warps per multi-warp core: 1, 2, 4 or 8 (1 = none).
 * In deterministic mode (one core, strictly in order) only threshold -1 or
 * 0 applies: threshold 0 replays the updates on one core of `group` warps.
 * EINVAL on other values.  asaga_autotune chooses this too (its step 5). */
asaga_status asaga_set_row_path(asaga_ctx *ctx, int64_t threshold, int group);

/* Where each core draws the row it stages next (Algorithm 2 samples i
 * before the update's reads; the draw of a later row can go anywhere).
 * 0 (default): at the top of an update, before its reads, so the interval
 * between the reads of x^ and the writes (the window whose overlap with
 * other updates is the tau of Assumption 1) holds no sampling work.  1: the
 * first warp of the core draws it while the update's gathers are in flight,
 * hiding the sampler's latency at the cost of a longer window: faster epochs
 * at the same warps and step, and more overlap, which can move the same
 * warps and step past the stability frontier.  The rows drawn and their
 * order are the same in both placements (a replay in order gives the same
 * iterate).  asaga_autotune chooses it (its step 6) and resets it to 0
 * first.  EINVAL: on not 0 or 1. */
asaga_status asaga_set_draw_ahead(asaga_ctx *ctx, int on);

/* Reason for the last failure of a call on ctx (or, when ctx is NULL, of
 * the calling thread's last asaga_create, asaga_sample_rows,
 * asaga_probe_line_rate or asaga_recompute_abar_noalloc); never NULL. */
const char *asaga_last_error(const asaga_ctx *ctx);

const char *asaga_status_string(asaga_status s);

/* ------------------------------------------------------------------------
 * Batches: many independent problems (regularisation paths, cross-validation
 * folds) solved together.  Each instance keeps its own data and state, as a
 * context would; one persistent update launch per segment covers every
 * unfinished instance (a block of 4 warps serves one instance, and each
 * instance owns a fixed set of blocks), the float64 objectives of all
 * instances come from one batched launch, and the segment's work (parameter
 * upload, update launch, objective launches, download of the objectives) is
 * captured once into a CUDA graph and replayed every segment.
 */
typedef struct asaga_batch asaga_batch;

/* Creates `count` instances from problems[i] and options[i] (loss, lambda,
 * gamma, seed per instance).  All instances share options[0].storage_dtype,
 * the sparse or dense layout, options[0].epochs_per_segment and
 * options[0].abar_recompute_every, and run on options[0].cuda_stream.  The
 * initial schedule gives instance i warps in proportion to n_i (1 + k_i/128),
 * k_i its mean row length (an update's cost is mostly a fixed latency; a
 * multiple of 4, at least 4, at most max(4, n_i/64), which keeps tau below
 * n_i/10 as Theorem 2 asks) within the warps that
 * can be resident at once.  EINVAL as asaga_create, or for mixed dtypes or
 * layouts, deterministic options, or count < 1. */
asaga_status asaga_batch_create(asaga_batch **out, int count, const asaga_problem *problems,
                                const asaga_options *options);

/* Runs segments over all unfinished instances until each has
 * (f_i - f_star[i])/|f_star[i]| <= target (then it stops receiving updates)
 * or max_epochs epochs have run.  results[i] (may be NULL) holds instance
 * i's epochs, updates, f_last and rel_subopt; its solver_seconds is the
 * device time of the shared segments up to the one after which it stopped,
 * i.e. its time to target inside the batch: every segment's update
 * launch, batched float64 objective and (every
 * options[0].abar_recompute_every-th segment, counted over the batch's life)
 * batched float64 abar recomputation, all captured in the segment's CUDA
 * graph; abar_drift is the drift that instance's last recomputation found.
 * f_star may be NULL when target <= 0.  OK when every instance reached the
 * target (or target <= 0), ENOTCONVERGED otherwise, EDIVERGED if an
 * objective turned non-finite, ECANCELLED after asaga_batch_cancel, ECUDA if
 * the update kernel reported a malformed row range or a staging failure. */
asaga_status asaga_batch_run(asaga_batch *b, double max_epochs, double target, const double *f_star,
                             asaga_result *results);

/* Asks the asaga_batch_run in progress (from another host thread) to stop
 * after the current segment; it returns ASAGA_ECANCELLED with every
 * instance's state as its updates left it.  Thread-safe; dropped when the
 * next asaga_batch_run starts.  EINVAL: b NULL. */
asaga_status asaga_batch_cancel(asaga_batch *b);

/* Per-instance step sizes, and warps, from shared trials.  Every trial runs
 * all instances at once for trial_epochs epochs (<= 0: 16) from x = 0 with
 * gamma_i = s * gamma0_i, s = 2^(-k/2) on the ladder k = -3..12 (stopping
 * once smaller steps help no instance), recording each float64
 * |grad f_i|^2 after every epoch.  Each instance takes the largest step
 * that converges (the test of asaga_autotune) and then, from one notch
 * inside it on, the step with the fewest predicted epochs (the trend test
 * of asaga_autotune); an instance whose prediction lies beyond twice the
 * trial runs on alone (up to 8x longer) to refine it.  Two passes: under
 * the default schedule, then with
 * warps in proportion to each instance's predicted work (epochs x epoch
 * cost, within the same caps); the second is kept, except that an
 * instance predicted under the first but not under the second keeps its
 * first step at no more warps than the first schedule gave it.  Last, the
 * row paths (asaga_batch_set_row_paths) at the tuned warps and steps: every
 * row of instance i on cores of G_i = min(4, 2^floor(log2(k_i / E))) warps
 * (k_i its mean row length), for E = 512 and 256 entries per warp, against
 * single warps, each schedule's batch epoch timed (the faster of two after
 * one untimed) and the fastest kept if 3% faster.  Leaves every instance at
 * x = 0.  results[i] may be NULL; its score is 1 / predicted epochs. */
asaga_status asaga_batch_autotune(asaga_batch *b, double trial_epochs, asaga_tune_result *results);

/* Overrides the schedule: warps[i] (rounded up to a multiple of 4) and/or
 * gamma[i]; either array may be NULL.  EINVAL if the warps cannot all be
 * resident at once. */
asaga_status asaga_batch_set_schedule(asaga_batch *b, const int *warps, const double *gamma);

/* Per-instance row paths (see asaga_set_row_path): threshold[i] >= -1 and
 * group[i] in {1, 2, 4} (a block of the batch kernel has 4 warps).  An
 * instance's blocks then hold 4 single-warp cores or 4/group multi-warp
 * cores; with both paths in use (threshold[i] > 0) its blocks are split in
 * proportion to the share of its nonzeros in the long rows.  EINVAL on
 * NULL arrays or other values. */
asaga_status asaga_batch_set_row_paths(asaga_batch *b, const int64_t *threshold, const int *group);

/* Every instance back to x = 0, alpha = 0, abar = 0 and sampler position 0,
 * keeping the schedule (warps, steps, row paths); the abar recomputation
 * cadence restarts.  EINVAL: b NULL. */
asaga_status asaga_batch_reset(asaga_batch *b);

/* As asaga_get_state / asaga_get_info for instance i. */
asaga_status asaga_batch_get_state(asaga_batch *b, int i, float *x, float *abar, float *alpha);
asaga_status asaga_batch_get_info(asaga_batch *b, int i, asaga_info *info);

/* f_i of every instance (float64, one batched launch); f holds count values. */
asaga_status asaga_batch_objective(asaga_batch *b, double *f);

const char *asaga_batch_last_error(const asaga_batch *b);
void asaga_batch_destroy(asaga_batch *b);

/* Columns the scratch of asaga_recompute_abar_noalloc holds (4 MiB of float64). */
#define ASAGA_NOALLOC_MAX_D 524288

/*
 * asaga_recompute_abar_noalloc -- abar = (1/n) sum_i alpha_i a_i in float64,
 * like asaga_recompute_abar, for data the caller keeps in device memory, and
 * without allocating any device memory.  The paper has no counterpart: this
 * is a service for callers that cannot allocate -- a process that must keep
 * a fixed device-memory footprint reserved up front (where an allocation at
 * run time can fail or stall), code embedded in a framework that owns all
 * device memory through its own allocator, or a path where the device-wide
 * synchronisation of cudaFree is not acceptable.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   n, d      rows and columns; n >= 1, 1 <= d <= ASAGA_NOALLOC_MAX_D.
 *   row_ptr   device int64[n+1], col_idx device int32[nnz], values device
 *             float32[nnz]: the CSR matrix with the invariants of
 *             asaga_problem (not validated here; the caller guarantees them).
 *   alpha     device float32[n], the scalar memories alpha_i.
 *   abar      device float32[d]; on entry the running averages (used only for
 *             the drift), on return the recomputed values rounded to float32.
 *   drift     device float64[1] or NULL; receives max_v |abar_v(entry) - exact_v|.
 *   stream    cudaStream_t to run on (NULL: the default stream).  The call
 *             only enqueues work; results are ready when the stream is.
 * Scratch: a fixed float64[ASAGA_NOALLOC_MAX_D] array (plus 1024 float64
 * partials) in the library's device code.  A GPU holds it from the time that
 * code is loaded on it until the process exits.  Every call shares it and
 * leaves the last call's sums in it (each call zeroes it first), so calls
 * that overlap on the GPU -- on different streams or from different host
 * threads -- race and corrupt each other's results; order them.  The first
 * call on a device looks the scratch address up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The
 * address belongs to the device's CUDA context: after a cudaDeviceReset the
 * next call on that device finds a new context and looks the address up
 * again, so that call too should come before any stream capture.
 * EINVAL: n < 1, d outside [1, ASAGA_NOALLOC_MAX_D], a NULL array; ECUDA: a
 * CUDA call failed.  asaga_last_error(NULL) gives the reason.
 */
asaga_status asaga_recompute_abar_noalloc(int64_t n, int64_t d, const int64_t *row_ptr,
                                          const int32_t *col_idx, const float *values,
                                          const float *alpha, float *abar, double *drift,
                                          void *stream);

/* Frees the context and its device memory; NULL is a no-op. */
void asaga_destroy(asaga_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ASAGA_H */
