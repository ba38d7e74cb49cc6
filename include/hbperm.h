/*
 * hbperm.h -- C ABI of the GB300 (sm_103a) Householder-aligned permutation
 * test (Ehara, "Accurate and Efficient Statistical Testing for Word Semantic
 * Breadth", ACL 2026).
 *
 * Problem statement (Sec. 3.1, "Problem setting"): two clouds of unit-norm
 * token embeddings X (n x d) and Y (m x d); H0 = equal dispersion with the
 * mean directions allowed to differ.  The test reflects one cloud onto the
 * other's mean direction (Sec. 3.1, "Householder mean-direction alignment"),
 * pools Z = X' u Y, draws B relabellings (fixed-space permutation), and
 * returns p = (1 + #{b : T_b exceeds T_obs})/(B + 1) (Eq. pvalue).
 *
 * Conventions for every entry point:
 *  - Data pointers (X, Y, Z, label bits, T_out) are DEVICE pointers owned by
 *    the caller, except where an argument says "host".  The library never
 *    frees caller memory.  hb_perm_test_batched also accepts host memory for
 *    XY (pinned memory copies fastest): it then copies XY itself, in pieces
 *    of whole pairs whose alignment starts as each piece arrives, and reads
 *    the host buffer only until the call returns.
 *  - Matrices are row-major, one embedding per row, rows contiguous.
 *    dtype HB_F32 = IEEE binary32, HB_BF16 = bfloat16 (16-bit patterns).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Calls that fill an hb_result synchronise that stream before
 *    returning; hb_align and hb_perm_labels return after enqueueing.
 *  - Errors are status codes; nothing aborts or throws across the ABI.  The
 *    calling thread's last message is available from hb_last_error().
 *  - Limits: 1 <= d <= 8192; n, m >= 2 for tests (>= 1 for hb_align);
 *    n + m <= 2^20; every input value finite with |v| < 16 (unit-normalised
 *    rows satisfy this); HB_PATH_MIXED additionally needs n + m <= 65536.
 *
 * Arithmetic contract (identical results to the FP64/exact CPU oracle):
 *  - Column and group sums are exact (values widened to a 2^-87 fixed-point
 *    grid; |v| < 2^-64 counts as 0) and rounded once to FP64.
 *  - Mean directions, the axis and every reflected row use IEEE FP64 with
 *    sequential fused multiply-add chains; reflected rows are rounded once to
 *    the input storage type.
 *  - Group sums of the B relabellings run on tensor cores (HB_PATH_MIXED) or
 *    FP32 SIMT (HB_PATH_FP32_PLAIN); every relabelling whose approximate
 *    statistic falls inside a rigorous error band around the observed one is
 *    re-decided exactly, so counts and p-values are bit-identical to the
 *    oracle's.
 */
#ifndef HBPERM_H
#define HBPERM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HB_OK = 0,
    HB_ERR_INVALID_ARG = 1,  /* bad size, enum, pointer or non-finite/|v|>=16 input      */
    HB_ERR_DEGENERATE = 2,   /* n<2 or m<2, zero mean vector, observed r = 0 or r >= 1    */
    HB_ERR_CUDA = 3,         /* a CUDA runtime call failed (message in hb_last_error)      */
    HB_ERR_OOM = 4,          /* workspace allocation failed                                */
    HB_ERR_TIMEOUT = 5,      /* a bounded device wait expired; results are not valid       */
    HB_ERR_UNSUPPORTED = 6   /* valid request outside this build's limits                  */
} hb_status;

typedef enum { HB_F32 = 0, HB_BF16 = 1 } hb_dtype;

/* Dispersion statistic (Sec. 3.1, Eqs. r, v, tobs).  With r_g = ||sum of
 * group g|| / n_g the mean resultant length:
 *   HB_STAT_LOGVOL_VMF  T = log v(G1) - log v(G2), v = 1/g_d(r),
 *                       g_d(r) = r (d - r^2)/(1 - r^2)   (the paper's log-volume
 *                       difference; g_d is the approximation of Banerjee et
 *                       al., JMLR 2005, since the paper does not print it)
 *   HB_STAT_ONE_MINUS_R2  T = (1 - r_1^2) - (1 - r_2^2)
 *   HB_STAT_MEAN_COSDIST  T = s_1 - s_2, s_g = (n_g^2 - ||sum||^2)/(n_g (n_g - 1))
 *                       (mean pairwise cosine distance of unit rows)        */
typedef enum { HB_STAT_LOGVOL_VMF = 0, HB_STAT_ONE_MINUS_R2 = 1, HB_STAT_MEAN_COSDIST = 2 } hb_stat;

/* Exceedance rule: two-sided |T_b| >= |T_obs| (default), T_b >= T_obs
 * (Eq. pvalue as printed), or T_b <= T_obs.  Ties count. */
typedef enum { HB_ALT_TWO_SIDED = 0, HB_ALT_GREATER = 1, HB_ALT_LESS = 2 } hb_alt;

/* HB_PATH_MIXED: group sums on tcgen05 tensor cores (BF16 operands, FP32
 * accumulators in TMEM) over exact slices of Z, 256-column accumulator tiles.
 * BF16 input: each column of a pair is split into two BF16 slices on
 * power-of-two grids chosen from the column's L1 norm, so that every FP32
 * accumulator is exact; pairs with n + m up to a limit (HB_OPT_SINGLE_SLICE_MAX_N)
 * first run the first slice alone (256 z-columns per tile: half the tensor
 * work) and re-run both slices only for the relabellings that fall inside
 * that pass's error band.  FP32 input: three fixed-point slices of 64
 * z-columns per tile.  HB_PATH_MIXED runs single CTAs (one SM per MMA, each
 * loading its own Z-slice tiles); HB_PATH_MIXED_NARROW the same with
 * half-width tiles; HB_PATH_MIXED_2SM tcgen05 cta_group::2 on pairs of SMs
 * (256 relabellings per MMA, each SM loading half of every Z-slice tile, so
 * half the B bytes per SM: the fastest route on GB300).  No route copies data
 * by TMA multicast.  HB_PATH_FP32_PLAIN: the paper's Algorithm 2 taken
 * literally (+-1 signs, FP32 SIMT GEMM).  HB_PATH_AUTO: each pair takes the
 * route the context's route table holds for its size (hb_autotune; untuned:
 * HB_PATH_MIXED_2SM up to n + m = 65536, the SIMT path above).  All paths
 * give identical results. */
typedef enum {
    HB_PATH_MIXED = 0,
    HB_PATH_FP32_PLAIN = 1,
    HB_PATH_AUTO = 2,
    HB_PATH_MIXED_NARROW = 3,
    HB_PATH_MIXED_2SM = 4
} hb_path;

typedef struct {
    uint64_t seed;        /* Philox key (key0 = low 32 bits, key1 = high 32 bits)           */
    uint32_t stream;      /* Philox counter word 2; 0 = labels depend on (seed, b, n, N)     */
    int64_t B;            /* number of relabellings (ignored when exhaustive)                */
    int32_t stat;         /* hb_stat                                                         */
    int32_t alt;          /* hb_alt                                                          */
    int32_t align;        /* 1 = Householder alignment (the paper), 0 = naive test            */
    int32_t reflect_side; /* 0 = reflect X onto Y's direction (the paper), 1 = reflect Y     */
    int32_t exhaustive;   /* 1 = all C(N, n) splits in colex order, N <= 24; p = count/C     */
    int32_t path;         /* hb_path                                                         */
} hb_opts;

typedef struct {
    double p;                   /* (1 + count)/(B + 1), or count/C when exhaustive          */
    int64_t count;              /* #{b : T_b exceeds T_obs}                                  */
    int64_t B_eff;              /* B, or C(N, n) when exhaustive                             */
    double T_obs;               /* observed statistic (FP64)                                 */
    double r_x;                 /* observed MRL of group 1 (rows 0..n-1 of Z)                */
    double r_y;                 /* observed MRL of group 2                                   */
    int32_t reflection_skipped; /* 1 when no reflection was applied (align = 0 or the mean    */
                                /*   directions differ by <= 2^-27 in 2-norm)                */
    int32_t status;             /* hb_status of this pair                                    */
    int64_t n_rechecked;        /* relabellings re-decided exactly (inside the error band)   */
    double band_max;            /* largest error band used for a decision                    */
} hb_result;

typedef struct hb_ctx hb_ctx;
typedef struct hb_plan hb_plan;

/* Create a context bound to CUDA device `device`.  It owns the device
 * workspace (grown on demand), pinned staging buffers and captured graphs.
 * One context must not be used by two threads at once. */
hb_status hb_ctx_create(hb_ctx **ctx, int device);
void hb_ctx_destroy(hb_ctx *ctx);

/* Steps 1-3 of Algorithm 1 (Sec. 3.1 alignment equations; Eq.
 * householder_fast).  Writes the pooled, aligned Z = [X' ; Y] (or [X ; Y']
 * with reflect_side = 1) as (n + m) x d rows of `dtype` into Z_out (device).
 * u_out (device, nullable) receives the FP64 axis u (zeros when skipped);
 * skipped (host, nullable) receives 1 when no reflection was applied, and
 * forces a stream synchronisation.  align = 0 copies X and Y unchanged. */
hb_status hb_align(hb_ctx *ctx, const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int32_t dtype,
                   int32_t align, int32_t reflect_side, void *Z_out, double *u_out, int32_t *skipped, void *stream);

/* The whole test of one pair (Algorithm 1; Algorithm 2 for the
 * relabellings).  out (host) receives the result.  T_out (device, nullable,
 * B_eff floats) receives each relabelling's statistic T_b (FP32; exact FP64
 * value rounded to FP32 for the relabellings re-decided exactly). */
hb_status hb_perm_test(hb_ctx *ctx, const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int32_t dtype,
                       const hb_opts *opts, hb_result *out, float *T_out, void *stream);

/* P independent pairs in one grouped launch sequence (the paper's
 * "Reusability" note, Sec. 3.2: pairs with equal (n, m) share label draws
 * when opts->stream is equal).  XY (device or host) packs, for each pair p in
 * order, n[p] rows of X then m[p] rows of Y, each row d values of `dtype`.
 * n, m (host, P entries) are the group sizes; out (host, P entries) receives
 * one result per pair.  Returns the first non-OK pair status, else HB_OK;
 * pairs are independent, so one pair's failure leaves the others valid. */
hb_status hb_perm_test_batched(hb_ctx *ctx, int64_t P, const void *XY, const int64_t *n, const int64_t *m,
                               int64_t d, int32_t dtype, const hb_opts *opts, hb_result *out, void *stream);

/* A batch shape planned once and replayed as one CUDA graph.  The label
 * draws, the work list and every launch of a test depend only on the group
 * sizes and opts, never on the data (Sec. 3.2, "Reusability"), so
 * hb_plan_create builds the work list for sizes n, m (host, P entries) and
 * opts, allocates the plan's own device workspace and pinned host staging,
 * and captures every device stage of the call -- label draws, alignment,
 * statistics, the group-sum GEMM with its fused decision, the exact recheck,
 * finalize and the copy of the results -- in one CUDA graph.  The plan keeps
 * ctx (which must outlive it) and no caller memory.  HB_ERR_OOM when the
 * workspace cannot be allocated; other errors as hb_perm_test_batched. */
hb_status hb_plan_create(hb_ctx *ctx, int64_t P, const int64_t *n, const int64_t *m, int64_t d, int32_t dtype,
                         const hb_opts *opts, hb_plan **plan);

/* Runs the planned test on XY (device or host, packed as for
 * hb_perm_test_batched with the plan's sizes; for host XY the bytes are
 * copied into a plan-owned device buffer first) with one graph launch on
 * `stream`.  The pair pointers are re-uploaded only when XY differs from the
 * previous call's.  out (host, P entries): results identical to
 * hb_perm_test_batched's.  Synchronises `stream`; calls on one plan must not
 * overlap.  If the exact-recheck list outgrows the capacity planned for it,
 * the call reruns through hb_perm_test_batched (same results, no graph). */
hb_status hb_plan_execute(hb_plan *plan, const void *XY, hb_result *out, void *stream);

/* Frees the plan's graph, streams, workspace and staging (NULL is a no-op). */
void hb_plan_destroy(hb_plan *plan);

/* The launch layout hb_perm_test_batched would use for sizes n, m (host, P
 * entries), d, dtype and opts (opts->path must not be HB_PATH_AUTO, whose
 * routes live in a context).  Host computation only: no context, no GPU and
 * no CUDA call, so it serves diagnostics and host-side tests.  counts (host)
 * receives the four sizes below; each array (host, nullable, int32) receives
 * its rows when not NULL, so a first call with NULL arrays sizes them:
 *   chunks       [n_chunks][4]   pair, side (0 = X, 1 = Y), first row, rows:
 *                the row chunks of the alignment and Z-statistics kernels
 *   pieces       [n_pieces][4]   first pair, end pair, first chunk, end chunk:
 *                the pieces a host input is copied and aligned in
 *   label_chunks [n_label_chunks + 1][2]  position in `order`, first item:
 *                the cuts of the label draws and GEMM launches
 *   items        [n_items][3]    pair, group of 128-relabelling tiles (2 on
 *                HB_PATH_MIXED_2SM, else 1), mode
 *                (0 = every slice, 1 = the single-slice pass): the GEMM work
 *                list, costliest pairs first
 *   order        [P]             the pairs in the work list's order
 * The last three are empty unless the path is a tensor-core path.
 * Errors as hb_perm_test_batched's argument checks. */
typedef struct {
    int32_t n_chunks;
    int32_t n_pieces;
    int32_t n_label_chunks;
    int32_t n_items;
} hb_layout_counts;
hb_status hb_plan_layout(int64_t P, const int64_t *n, const int64_t *m, int64_t d, int32_t dtype,
                         const hb_opts *opts, hb_layout_counts *counts, int32_t *chunks, int32_t *pieces,
                         int32_t *label_chunks, int32_t *items, int32_t *order);

/* Route tuning (the paper's Sec. 3.2 leaves the block size and the GEMM
 * route to the implementation; none of them changes a result).  Pair sizes
 * N = n + m fall into HB_ROUTE_BUCKETS buckets: bucket 0 holds N <= 64,
 * bucket k holds 2^(k+5) < N <= 2^(k+6).  hb_autotune times, for every
 * bucket up to min(max_N, 65536), a synthetic batch of about 2^18 rows of
 * d unit-norm values of `dtype` (pairs of size 2^(k+6), split evenly) with
 * min(opts->B, 1023) relabellings on HB_PATH_MIXED, HB_PATH_MIXED_NARROW,
 * HB_PATH_FP32_PLAIN and HB_PATH_MIXED_2SM, and stores the fastest in the
 * context's route table,
 * which HB_PATH_AUTO then follows; buckets above 65536 always take the SIMT
 * path.  ms_out (host, nullable) receives [HB_ROUTE_BUCKETS][4] wall-clock
 * milliseconds in that path order, -1 where not timed.  The other fields of
 * opts (stat, alt, align, seed) are those of the timed runs.  Synchronous;
 * allocates and frees its own device buffer. */
#define HB_ROUTE_BUCKETS 15
hb_status hb_autotune(hb_ctx *ctx, int64_t d, int32_t dtype, const hb_opts *opts, int64_t max_N, float *ms_out);

/* The path (hb_path, never HB_PATH_AUTO) HB_PATH_AUTO gives a pair of size N. */
hb_status hb_route(hb_ctx *ctx, int64_t N, int32_t *path_out);

/* HB-LABEL-v1 label rows for relabellings b0 .. b0+count-1 of a pool of N
 * with group-1 size n (Sec. 3.2: the sign matrix S with exactly n entries
 * +1 per row; here bit 1 = group 1).  bits_out (device) is row-major
 * [count][ceil(N/32)] uint32, position i in bit i%32 of word i/32,
 * positions >= N zero.  Philox4x32-10 key (seed_lo, seed_hi), counter
 * (i/4, b_lo, stream_id, b_hi); sequential selection sampling (Knuth,
 * Algorithm S) with a 32-bit multiply-high. */
hb_status hb_perm_labels(uint64_t seed, uint32_t stream_id, int64_t n, int64_t N, int64_t b0, int64_t count,
                         uint32_t *bits_out, void *stream);

/* hb_align without any device allocation, for callers that cannot call
 * cudaMalloc: applications whose device memory is fully reserved by their own
 * pool allocator, or latency-critical code that cannot take cudaMalloc's
 * implicit device synchronisation.  (The paper has no counterpart; this is a
 * deployment variant of hb_align.)  Same arguments, layouts and results as
 * hb_align, bit for bit, on the current device; no hb_ctx is needed.
 * All scratch comes from one fixed 2 MiB array in device global memory that
 * every GPU loading this library holds until the process exits.  Limits:
 * d <= 1024 and n + m <= 8192, else HB_ERR_UNSUPPORTED with a message in
 * hb_last_error().  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current), so make it before
 * any stream capture.  Every call reuses the same array, which keeps the last
 * call's contents (the call clears what must start at zero); calls that
 * overlap on the GPU -- from several streams or host threads -- race on it. */
hb_status hb_align_noalloc(const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int32_t dtype,
                           int32_t align, int32_t reflect_side, void *Z_out, double *u_out, int32_t *skipped,
                           void *stream);

/* ---------------------------------------------------------------------------
 * Learned triage.  A component of this library's batched workflow; the paper
 * has no learned part.  A network predicts, from cheap per-pair features,
 * quantiles of the null distribution of |T| that the full test (Eq. pvalue)
 * would draw; pairs whose predicted p is clearly outside a band around alpha
 * skip the full test.
 * ------------------------------------------------------------------------- */
#define HB_TRIAGE_NFEAT 19
#define HB_TRIAGE_NQ 9

/* Features of P pairs (packed as for hb_perm_test_batched; XY device):
 * log n, log m, log(d * lambda_k) for the 16 Ritz values lambda_k of the
 * pooled scatter Z^T Z / N of the aligned pair (Sec. 3.1) after 2 block
 * subspace iterations V <- orth(Z^T Z V / N) from a fixed Philox start block
 * (any orthonormal basis of the iterate's span gives the same Ritz values),
 * and 10 * T_obs.  Runs the alignment and T_obs only (no relabellings).
 * feat_out: device [P][19]; tobs_out: device [P] FP64, nullable; out: host [P]
 * (status, T_obs, r_x, r_y).  Needs d <= 1024. */
hb_status hb_triage_features(hb_ctx *ctx, int64_t P, const void *XY, const int64_t *n, const int64_t *m, int64_t d,
                             int32_t dtype, const hb_opts *opts, float *feat_out, double *tobs_out, hb_result *out,
                             void *stream);

/* Training targets from the method's own relabellings: runs the full test of
 * P pairs exactly as hb_perm_test_batched and writes, per pair, the empirical
 * quantiles of |T_b| (b = 0..B-1; the ceil(level * B)-th smallest) at levels
 * 0.5, 0.8, 0.9, 0.95, 0.975, 0.99, 0.995, 0.998, 0.999, times 100, into
 * quant_out (device [P][9]).  out: host [P].  Needs B <= 32768. */
hb_status hb_null_quantiles(hb_ctx *ctx, int64_t P, const void *XY, const int64_t *n, const int64_t *m, int64_t d,
                            int32_t dtype, const hb_opts *opts, float *quant_out, hb_result *out, void *stream);

/* The triage network 19 -> 256 (ReLU) -> 256 (ReLU) -> 9.  Parameters form one
 * flat FP32 vector [W1 19x256 | b1 256 | W2 256x256 | b2 256 | W3 256x9 | b3 9]
 * (weights input-major, row-major); the forward uses the weights rounded to
 * BF16 (params_bf16, same layout) with FP32 accumulation.  All pointers are
 * device memory owned by the caller, each hb_mlp_param_count() long. */
typedef struct {
    float *params;
    uint16_t *params_bf16;
    float *grad;
    float *adam_m;
    float *adam_v;
} hb_mlp;

int64_t hb_mlp_param_count(void);
/* params_bf16 <- BF16(params) */
hb_status hb_mlp_sync(const hb_mlp *net, void *stream);
/* out (device [P][9]) <- network(feat (device [P][19])) */
hb_status hb_mlp_forward(hb_ctx *ctx, const hb_mlp *net, int64_t P, const float *feat, float *out, void *stream);
/* net->grad <- gradient of the mean pinball loss of network(feat) against
 * target (device [P][9]; levels as hb_null_quantiles); loss (device, 1 float). */
hb_status hb_mlp_grad(hb_ctx *ctx, const hb_mlp *net, int64_t P, const float *feat, const float *target, float *loss,
                      void *stream);
/* One Adam step (Kingma and Ba, 2015; beta 0.9/0.999, eps 1e-8) at step t >= 1
 * on params with net->grad, updating the moments and params_bf16. */
hb_status hb_mlp_adam(const hb_mlp *net, float lr, int64_t t, void *stream);
/* Predicted p of P pairs from predicted quantiles (x100, device [P][9], made
 * non-decreasing) and T_obs (device [P]): 1 - F(|T_obs|), F linear between
 * (q_k, level_k), from (0, 0) below q_1, the last slope continued above q_9
 * and floored at p = 1e-4.  p_out: device [P]. */
hb_status hb_triage_predict_p(int64_t P, const float *quant, const double *tobs, float *p_out, void *stream);

/* Tracing: per-stage device timing of the calls made on this context, from
 * CUDA events recorded on the caller's stream between the stages (off by
 * default; enabling it adds no synchronisation). */
hb_status hb_ctx_set_timing(hb_ctx *ctx, int32_t enable);

/* Stage durations of the last hb_perm_test / hb_perm_test_batched call on
 * this context, in milliseconds (ms_out, host, 7 floats): [0] alignment
 * (column sums, axis, reflection), [1] Z statistics, fixed-point slices and
 * T_obs, [2] label draws not hidden behind steps 1-4, [3] group-sum GEMM
 * with the fused statistic epilogue, including waits for label chunks still
 * being drawn, [4] exact recheck, [5] p-values and the result copy, [6] the
 * sum of the GEMM launches' own durations.
 * n_launches (host, nullable) receives the kernel launches of that call.
 * HB_ERR_INVALID_ARG if timing was not enabled for that call. */
hb_status hb_ctx_stage_times(hb_ctx *ctx, float *ms_out, int32_t *n_launches);

/* Context options (hb_ctx_set_option).  None changes a result.
 *   HB_OPT_WAIT_LIMIT_NS        wall-clock limit of every device barrier wait of
 *                               the tensor-core kernels (default 4e9; 1e3..6e10);
 *                               a wait that runs out ends the call with
 *                               HB_ERR_TIMEOUT and leaves the context usable
 *   HB_OPT_SINGLE_SLICE_MAX_N   BF16 input: pairs with n + m <= value start with
 *                               the single-slice pass (default 65536: every pair
 *                               of the tensor-core path; 0 = never).  Its cost is
 *                               one slice plus two slices for the relabellings
 *                               inside its band, which is wide only for very
 *                               large pairs whose T_obs lies in the null's bulk
 *   HB_OPT_TEST_WITHHOLD_ARRIVAL  test hook: 1 = the next tensor-core call on
 *                               this context withholds one barrier arrival of
 *                               its first GEMM launch, so that a bounded wait
 *                               runs out and the call returns HB_ERR_TIMEOUT
 *                               (the hook then clears itself; plans ignore it)
 *   HB_OPT_A_OPERAND_TMEM       1 = CTA pairs on BF16 input keep the label
 *                               operand of the group-sum GEMM in tensor memory
 *                               (written by the producer warps with tcgen05.st;
 *                               192-column accumulator tiles) instead of shared
 *                               memory (256-column tiles; default 0, faster on
 *                               the batched workload)
 * Options apply to later calls and plans created later. */
#define HB_OPT_WAIT_LIMIT_NS 1
#define HB_OPT_SINGLE_SLICE_MAX_N 2
#define HB_OPT_TEST_WITHHOLD_ARRIVAL 4
#define HB_OPT_A_OPERAND_TMEM 8
hb_status hb_ctx_set_option(hb_ctx *ctx, int32_t option, int64_t value);

/* Message of the last failing call on this thread ("" if none). */
const char *hb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HBPERM_H */
