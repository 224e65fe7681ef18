/*
 * sng.h -- C ABI of the GB300 (sm_103a) SNG-DBSCAN library (libsng.so).
 *
 * SNG-DBSCAN is Algorithm 1 of Jiang, Jang & Lacki, "Faster DBSCAN via
 * subsampled similarity queries" (NeurIPS 2020), Section 3.  Its inputs are
 * the points X, a sampling rate s, a radius eps and MinPts; its output is a
 * partition of the points into clusters plus noise.  Steps:
 *   2  every point draws ceil(s n) partners and keeps an edge to each partner
 *      within distance eps                              (sng_build_graph)
 *   3  points of degree >= MinPts are core points; the connected components
 *      of the core subgraph are the cluster cores
 *   4  a non-core point with an edge to a core joins that core's cluster
 *   5  every other point is noise                       (sng_cluster)
 *
 * Conventions shared by every call
 *  - Pointers named "device" must be CUDA device (or managed) memory on the
 *    current device; "host" pointers are ordinary host memory.  Nothing in
 *    this header depends on a framework: plain pointers and sizes only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls return once it is enqueued unless
 *    stated otherwise.
 *  - The caller owns inputs and outputs.  Library-owned memory appears only in
 *    sng_graph (freed by sng_graph_free) and in plan objects.
 *  - Every call returns an sng_status.  Invalid arguments are rejected with
 *    SNG_EINVAL before any work is enqueued; sng_last_error() returns a
 *    one-line reason.  No call aborts or throws across the ABI.
 *  - Partner draws (step 2) are fixed by a counter-based hash so that any
 *    implementation sees the same pairs: mix = SplitMix64 output function,
 *    k_i = mix(seed ^ mix(i)), h = mix(k_i ^ j), r = h mod (n-1),
 *    partner(i,j) = r + (r >= i), for j = 0..m-1, m = ceil(s n).
 *  - The eps-test keeps (i,p) iff d2(x_i,x_p) <= eps^2 where d2 is the FP64
 *    sum of squared coordinate differences, left to right.  The kernels test
 *    in FP32 and recompute in FP64, in exactly that order, every pair whose
 *    FP32 value lies within a guard band of eps^2, so FP32 inputs give the
 *    FP64 decision on every pair.
 *  - Labels: -1 = noise; otherwise the smallest core-point index of the
 *    cluster (a border point adjacent to several clusters takes the smallest
 *    such label: the paper's "choose one arbitrarily" fixed to the minimum).
 */
#ifndef SNG_H
#define SNG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sng_status;
#define SNG_OK 0
#define SNG_EINVAL (-1)     /* bad argument; nothing was enqueued             */
#define SNG_ENOMEM (-2)     /* a device allocation failed; nothing leaked     */
#define SNG_ECUDA (-3)      /* a CUDA runtime call failed                     */
#define SNG_ETIMEOUT (-4)   /* a bounded device loop gave up (status word)    */
#define SNG_EINTERNAL (-5)  /* a device-side consistency check failed         */

/* element type of X */
#define SNG_F32 0
#define SNG_BF16 1          /* bfloat16 bit patterns, uint16 per element       */

/* degree used by the MinPts test (Algorithm 1, step 3) */
#define SNG_DEG_UNDIRECTED_MULTI 0 /* each kept draw (i,p) adds 1 to i and to p */
#define SNG_DEG_OUT 1              /* kept draws of i only (the count thresholded in
                                      the proof of Lemma 2)                      */
#define SNG_DEG_SIMPLE 2           /* distinct neighbours of i in the simple
                                      undirected graph G (repeated draws and both
                                      directions of a pair count once); costs a
                                      pair set of 2E..4E 8-byte slots.  Not in the
                                      batched or no-allocation forms, nor with the
                                      surrogate's reweighted degrees             */

/* how partners are drawn (Algorithm 1, step 2) */
#define SNG_SAMPLE_HASH 0   /* m hashed draws with replacement, never i itself */
#define SNG_SAMPLE_ALL 1    /* every other point once (m = n-1): s = 1, textbook
                               DBSCAN's full eps-neighbourhood graph           */

/* neighbourhood test of Algorithm 1, step 2 (the method needs only
 * similarity queries, Section 1).  FP32 inputs: every decision equals the
 * FP64 result computed in the stated order (unfused, left to right). */
#define SNG_METRIC_L2 0     /* edge iff sum_k (a_k - b_k)^2 <= eps^2          */
#define SNG_METRIC_DOT 1    /* edge iff <a, b> >= eps                          */
#define SNG_METRIC_COSINE 2 /* edge iff <a, b> / (sqrt(<a,a>) sqrt(<b,b>)) >= eps;
                               a zero vector is similar to nothing            */
#define SNG_METRIC_L1 3     /* edge iff sum_k |a_k - b_k| <= eps (Manhattan)   */
#define SNG_METRIC_LINF 4   /* edge iff max_k |a_k - b_k| <= eps (Chebyshev);
                               L1 / LINF: FP32 points, four lanes per pair of
                               the direct gather (no tiles, no tensor-core
                               screens); with SNG_FLAG_SCREEN16 or
                               SNG_FLAG_SCREEN8 the pairs are tested on a BF16
                               copy (map_screen = 1) and certified from each
                               row's copy error bound (sqrt(d) times its
                               Euclidean norm for L1, that norm for LINF);
                               open pairs are decided from the FP32 points.
                               A NaN difference is within eps of nothing      */

/* flags */
#define SNG_FLAG_TIMING 1u  /* fill sng_stats.ms with per-phase CUDA-event times */
#define SNG_FLAG_PREFETCH 2u /* gather: bulk-prefetch partner rows into L2 one stage
                                ahead (16-byte rows; measured slower at d = 64)  */
#define SNG_FLAG_WARP_ROWS 8u /* one warp per source row even where the default
                                is one lane per source row: the Euclidean form
                                with one lane per pair (rows of at most 4
                                vectors and at least 32 x 64 rows per SM, or
                                32 x 16 with SNG_SAMPLE_ALL; in
                                the batched form, rows of one float4), where
                                each lane hashes, tests and
                                records its own row's draws with 2 or 4
                                batches in flight (map_unroll 1 or 8 selects
                                one warp per row as well)                    */
#define SNG_FLAG_TILED 16u  /* step 2 tile by tile: every draw is first bucketed by
                                (source slice, partner slice) -- map_tile slices
                                per axis, 0 = enough for two slices to fit in L2 --
                                then each tile is tested while its two slices
                                stay in L2.  Euclidean form, 16-byte vectors;
                                same results; ~8 bytes of scratch per draw.
                                Falls back to the direct gather (stats
                                map_tiles = 0) where it does not apply: other
                                metrics, one lane per row, map_passes > 1,
                                SNG_FLAG_NO_SYNC, no device memory for the
                                buckets, or a bucket past its capacity (mean +
                                8 standard deviations)                         */
#define SNG_FLAG_SCREEN16 32u /* FP32 points: the gather tests pairs on a BF16 copy
                                of the points made inside the call (2 bytes per
                                value of scratch, plus 16 per point), and
                                decides a pair from it only where a bound on
                                the copy's rounding cannot change the decision;
                                every other pair is summed again from the FP32
                                points and decided as without the flag.
                                Results are identical; stats report map_screen
                                and screen_pairs.  On CUDA cores (Euclidean
                                form) the bound is 2^-8 of the two rows'
                                norms and the direct and tiled gathers apply
                                (the tiled one not with SNG_FLAG_NO_SYNC);
                                ignored for BF16 points, one lane per row and
                                map_passes > 1.  The Manhattan and Chebyshev
                                distances have a screen of their own (see
                                SNG_METRIC_LINF)                               */
#define SNG_FLAG_SCREEN_MMA 64u /* with SNG_FLAG_SCREEN16 and d <= 128: the direct
                                gather takes each pair's dot product on the
                                BF16 copy from tensor-core MMAs (16 partners at
                                a time, FP32 accumulation) -- the squared
                                distance as |a|^2 + |b|^2 - 2 a.b, or the inner
                                product or cosine for those metrics -- and
                                certifies it from the rows' own rounding-error
                                bounds (|a - a'| + |b - b'|) and the bound of
                                the MMA.  Pairs it leaves open are queued and
                                decided after the gather from the FP32 points.
                                Same results.  map_unroll selects the register
                                budget (2, 3 or 4 blocks per SM)               */
#define SNG_FLAG_SCREEN8 256u /* FP32 points, d <= 128: the tensor-core screen of
                                SNG_FLAG_SCREEN_MMA on an FP8 (E4M3) copy of
                                x * 2^k (one power of two for the point set;
                                1 byte per value of scratch), with FP8 MMAs;
                                Euclidean, inner product and cosine (the
                                Manhattan and Chebyshev distances take the BF16
                                copy, as with SNG_FLAG_SCREEN16).  The copy's rounding is coarser,
                                so more pairs are left open and decided from
                                the FP32 points; results are identical.  Stats
                                report map_screen = 4.  Same exclusions as
                                SNG_FLAG_SCREEN16; takes precedence over it  */
#define SNG_FLAG_TCGEN05 128u /* with SNG_FLAG_SCREEN16 | SNG_FLAG_SCREEN_MMA,
                                Euclidean form, d <= 64: the partner rows of
                                the BF16 copy are fetched by the tensor memory
                                accelerator (tile::gather4, four rows per copy)
                                into shared memory and the dot products come
                                from tcgen05 MMAs (128 partners x 4 source rows
                                per MMA, FP32 accumulators in tensor memory).
                                Same thresholds, same results; stats
                                map_screen = 3; map_unroll selects the ring's
                                stages (2..5).  SNG_ECUDA where the driver
                                offers no tensor-map encoder                  */
#define SNG_FLAG_NO_SYNC 4u  /* sng_cluster only: no host synchronisation inside the
                                call, so it can be captured in a CUDA graph.  The
                                edge arrays are sized for all n*m draws (8 bytes
                                each; SNG_ENOMEM when that does not fit) instead
                                of the counted E; stats must be NULL;
                                counters go to counters_out (if set); not with
                                SNG_FLAG_TIMING or SNG_DEG_SIMPLE.  Device-side
                                status bits are reported only in counters_out.  */

typedef struct {
    int64_t n;            /* number of points, 2 <= n <= 2^31 - 1            */
    int32_t d;            /* dimensions, >= 1                                */
    int32_t ld;           /* row stride of X in elements, >= d               */
    int32_t dtype;        /* SNG_F32 or SNG_BF16                             */
    int32_t degree_mode;  /* SNG_DEG_*                                       */
    int32_t sample_mode;  /* SNG_SAMPLE_*                                    */
    int32_t min_pts;      /* MinPts, >= 1                                    */
    float eps;            /* SNG_METRIC_L2 / _L1 / _LINF: radius,
                             1e-15 <= eps <= 1e18;
                             SNG_METRIC_DOT / _COSINE: similarity threshold,
                             any finite value                               */
    float band_rel;       /* half-width of the reported band |d2-eps^2| <=
                             band_rel*eps^2 (similarity: |sim-eps| <=
                             band_rel*|eps|; L1 / LINF: |dist-eps| <=
                             band_rel*eps); 0 selects 1e-5 (F32) / 1e-3 (BF16) */
    double s;             /* sampling rate in (0, 1]; m = ceil(s*n)          */
    int64_t m_override;   /* > 0: use this m instead of ceil(s*n); every m
                             must be in [1, 2^31 - 1025]                     */
    uint64_t seed;        /* partner-hash seed                               */
    const float *x_f32_master; /* device, n x ld FP32; BF16 form: the FP32 values
                             the FP64 recheck reads (required for SNG_BF16)    */
    uint32_t flags;       /* SNG_FLAG_*                                      */
    int32_t map_group;    /* gather mapping override: lanes per pair (1..32,
                             power of two), 0 = library default             */
    int32_t map_unroll;   /* partner batches in flight per warp, 0 = default */
    int32_t map_block;    /* threads per block of the gather, 0 = default    */
    int32_t map_tile;     /* batched form: source rows per work item, 0 = default;
                             tiled gather (SNG_FLAG_TILED): slices per axis,
                             clamped to [2, 32], 0 = two slices in ~88 MiB  */
    int32_t map_passes;   /* gather: 0/1 = one pass over all partners; k > 1 = k
                             launches, each testing only the draws whose partner
                             lies in one of k equal slices of X (L2-resident) */
    int32_t metric;       /* SNG_METRIC_*; similarity metrics in sng_cluster and
                             sng_build_graph only, one pass (map_passes <= 1) */
    /* Source rows [row_begin, row_end) draw partners; 0, 0 = all rows.  Other
     * rows draw nothing (their CSR rows are empty) but still receive
     * in-degree from the rows that do: a shard of step 2 for multi-GPU runs
     * (sng_build_graph only; the other calls reject a partial range).      */
    int64_t row_begin;
    int64_t row_end;
    /* SNG_FLAG_NO_SYNC: device uint64[9] receiving, at the end of the call,
     * [0] reserved (0), [1] band pairs, [2] FP64 rechecks, [3] band points,
     * [4] cores, [5] clusters, [6] noise points, [7] kept draws (edges),
     * [8] device status bits (nonzero: a bounded loop gave up or an index
     * check failed).  NULL: not written.  Ignored without the flag. */
    unsigned long long *counters_out;
} sng_params;

typedef struct {
    int64_t queries;      /* sampled distance queries = n * m (hash mode)    */
    int64_t kept_edges;   /* kept draws, E                                   */
    int64_t band_pairs;   /* draws with |d2_fp64 - eps^2| <= band_rel*eps^2  */
    int64_t band_points;  /* points touching at least one band pair          */
    int64_t cores;        /* points with degree >= MinPts                    */
    int64_t clusters;     /* connected components of the core subgraph       */
    int64_t noise;        /* points labelled -1                              */
    int64_t recheck_pairs;/* draws recomputed in FP64 (guard band)           */
    int64_t surrogate_core;  /* surrogate form: points gated as confident core */
    int64_t surrogate_noise; /* surrogate form: points gated as confident noise */
    float ms[8];          /* SNG_FLAG_TIMING: [0] gather [1] scan [2] fill
                             [3] core+union [4] labels [5] finalize [6] total
                             (gather to finalize) [7] surrogate gate        */
    int32_t map_vec, map_group, map_nch, map_unroll; /* gather mapping used     */
    int32_t map_tiles;    /* slices per axis of the tiled gather (SNG_FLAG_TILED)
                             when it ran; 0 = the direct gather             */
    int32_t map_tex;      /* tiled gather: 16-byte chunks of each partner row
                             read through the texture unit (0 or 1)        */
    int32_t map_screen;   /* 1: pairs were tested on the BF16 copy
                             (SNG_FLAG_SCREEN16); map_vec .. map_unroll then
                             describe the mapping over that copy; 2: with
                             tensor-core dot products (SNG_FLAG_SCREEN_MMA;
                             map_group 16 partners per MMA, map_nch k-tiles);
                             3: rows gathered by TMA, tcgen05 dot products
                             (SNG_FLAG_TCGEN05; map_group 128 partners per
                             MMA); 4: FP8 copy, tensor-core dot products
                             (SNG_FLAG_SCREEN8; map_nch k-tiles of 32)     */
    int64_t screen_pairs; /* SNG_FLAG_SCREEN16 / SCREEN8: pairs the screen
                             left open, decided again from the FP32 points */
} sng_stats;

typedef struct {
    int64_t n;            /* points                                          */
    int64_t m;            /* draws per point                                 */
    int64_t num_edges;    /* E                                               */
    int64_t *row_ptr;     /* device, n+1: row i = col[row_ptr[i]..row_ptr[i+1]) */
    int32_t *col;         /* device, E: kept partners of each row in draw order */
    int32_t *deg;         /* device, n: degree per params.degree_mode        */
    uint8_t *core;        /* device, n: deg >= min_pts                       */
} sng_graph;

/*
 * Algorithm 1, step 2 (and the degree / core mask of step 3): the sampled
 * eps-neighbourhood graph of X as CSR by source point.  x: device, n rows of
 * ld elements of params->dtype.  On SNG_OK `out` holds library-owned device
 * arrays; release them with sng_graph_free.  Synchronises `stream` once (to
 * size col) and again at the end when stats != NULL.
 */
sng_status sng_build_graph(const void *x, const sng_params *params, sng_graph *out,
                           sng_stats *stats, void *stream);

/* Frees the arrays of a graph from sng_build_graph (device-synchronising). */
void sng_graph_free(sng_graph *g);

/*
 * Algorithm 1, steps 3-5 on a given sampled graph: src/col (device int32[E])
 * list its kept draws (src[e] drew col[e]), deg (device int32[n]) the degree
 * of every point in params->degree_mode (e.g. summed over the ranks that
 * built parts of the graph).  With SNG_DEG_SIMPLE the degrees are computed
 * from src/col here and deg is not read (may be NULL).  Core = deg >=
 * params->min_pts; labels
 * (device int32[n]) and core (device uint8[n] or NULL) as in sng_cluster.
 * Only n, min_pts and degree_mode of params are read.  Synchronises `stream`
 * when stats != NULL.
 */
sng_status sng_cluster_edges(int64_t n, const int32_t *src, const int32_t *col, int64_t num_edges,
                             const int32_t *deg, const sng_params *params, int32_t *labels,
                             uint8_t *core, sng_stats *stats, void *stream);

/*
 * The whole of Algorithm 1: graph (step 2), degrees and core mask, core
 * components (step 3), border labels (step 4), noise (step 5).
 * x: device, n x ld.  labels: device int32[n] (output).  core: device
 * uint8[n] (output) or NULL.  Synchronises `stream` once mid-way (to size the
 * edge list) and at the end when stats != NULL.
 */
sng_status sng_cluster(const void *x, const sng_params *params, int32_t *labels,
                       uint8_t *core, sng_stats *stats, void *stream);

/*
 * sng_cluster on HOST buffers: x_host (n x ld elements of params->dtype;
 * with SNG_BF16, params->x_f32_master is a HOST n x ld FP32 array as well)
 * is copied to the device (in up to four concurrent pieces, so several copy
 * engines can serve it; pinned memory runs at full speed, pageable memory
 * works), Algorithm 1 runs as in sng_cluster, and labels_host (int32[n]) and
 * core_host (uint8[n] or NULL) receive the result.  Device memory for the
 * copies is allocated and freed inside the call.  Synchronises `stream`
 * before returning (the host outputs are then valid).
 */
sng_status sng_cluster_host(const void *x_host, const sng_params *params, int32_t *labels_host,
                            uint8_t *core_host, sng_stats *stats, void *stream);

/*
 * Many independent point clouds in one persistent launch.  x_concat: device,
 * clouds stored back to back (rows of ld elements, F32 only).  offsets: HOST
 * int64[n_clouds+1], cloud b = rows offsets[b]..offsets[b+1]-1, each cloud
 * 2..2^31-1 points.  base: shared parameters; cloud b uses seed base->seed + b
 * and m = m_per_cloud[b] (HOST, nullable) else base->m_override else
 * ceil(base->s * n_b).  labels: device int32[total], cloud-local indices.
 * Equivalent to calling sng_cluster on every cloud.  Synchronises `stream`
 * when stats != NULL.
 */
sng_status sng_cluster_batched(const void *x_concat, const int64_t *offsets, int32_t n_clouds,
                               const sng_params *base, const int64_t *m_per_cloud,
                               int32_t *labels, sng_stats *stats, void *stream);

/* Reusable form of sng_cluster_batched: the plan holds the validated cloud
 * table and device scratch, and sng_batch_run replays the launch as a CUDA
 * graph (captured on the first run for a given x/labels/stream). */
typedef struct sng_batch_plan sng_batch_plan;
sng_status sng_batch_plan_create(const int64_t *offsets, int32_t n_clouds, const sng_params *base,
                                 const int64_t *m_per_cloud, sng_batch_plan **plan);
sng_status sng_batch_run(sng_batch_plan *plan, const void *x_concat, int32_t *labels,
                         sng_stats *stats, void *stream);
void sng_batch_plan_destroy(sng_batch_plan *plan);

/*
 * Partner draws of Algorithm 1, step 2, materialised for checking: out[r*m+j]
 * = partner(i0 + r, j) for r < rows, j < m.  out: device int32[rows*m].
 */
sng_status sng_sample_partners(int64_t n, uint64_t seed, int64_t i0, int64_t rows, int64_t m,
                               int32_t sample_mode, int32_t *out, void *stream);

/* Adjusted Rand index (Hubert & Arabie 1985; the first score of the paper's
 * Section 5) of two labelings a, b (device int32[n], values in [-1, n)),
 * noise as one label.  Synchronises `stream`; result in *ari (host).
 * Labels outside [-1, n) -> SNG_EINVAL. */
sng_status sng_ari(const int32_t *a, const int32_t *b, int64_t n, double *ari, void *stream);

/* normaliser of the adjusted mutual information */
#define SNG_AMI_MIN 0
#define SNG_AMI_GEOMETRIC 1
#define SNG_AMI_ARITHMETIC 2  /* mean of the two entropies (the usual default) */
#define SNG_AMI_MAX 3

typedef struct {
    double ami;           /* (mi - emi) / (avg(h_a, h_b) - emi)               */
    double mi;            /* mutual information (natural log)                 */
    double emi;           /* its expectation under random relabelling         */
    double h_a, h_b;      /* entropies of the two labelings                   */
    int64_t clusters_a;   /* distinct labels (noise counts as one)            */
    int64_t clusters_b;
} sng_mi_terms;

/* Adjusted mutual information (Vinh, Epps & Bailey 2010; the second score
 * of the paper's Section 5) of two labelings a, b (device int32[n], values in
 * [-1, n)), noise as one label, with normaliser `average` (SNG_AMI_*).  The
 * expectation sums every term of the hypergeometric model (terms below the
 * FP64 underflow threshold are zero).  Two trivial labelings of the same
 * kind (both one cluster, or both all singletons) score 1; a normaliser that
 * does not exceed the expectation scores 0.  Synchronises `stream` three
 * times; result and terms in *out (host).  Labels outside [-1, n) or an
 * unknown normaliser -> SNG_EINVAL. */
sng_status sng_ami(const int32_t *a, const int32_t *b, int64_t n, int32_t average,
                   sng_mi_terms *out, void *stream);

/*
 * Core-point surrogate (no counterpart in the paper): a d -> 128 -> 128 -> 1
 * perceptron, exact-erf GELU, FP16-rounded weights with FP32 accumulation,
 * predicting whether Algorithm 1 makes a point a core point (step 3).  Points
 * it is confident about skip most of their sampled queries (step 2).
 *
 * Parameter vector: device FP32, sng_mlp_param_count(d, 128) entries, laid out
 *   [W1 (128 x d) | b1 (128) | W2 (128 x 128) | b2 (128) | w3 (128) | b3 (1) |
 *    mean (d) | std (d)]
 * W rows are output units.  The first count - 2d entries are trained; mean and
 * std standardise the inputs, u = (x - mean) / std.  Points are n x d FP32
 * rows (row stride d) unless stated otherwise.
 */
typedef struct {
    int32_t d;            /* input features, 1..64 (= the points' d)          */
    int32_t hidden;       /* hidden width; must be 128                         */
    int32_t batch;        /* training batch size (sng_mlp_train)              */
    float lr, beta1, beta2, adam_eps; /* Adam (Kingma & Ba 2015)               */
    uint64_t seed;        /* batch rows drawn with replacement by the hash    */
    int32_t sequential;   /* 1: batch b of step t takes rows (t*batch + b) mod n
                             in order instead of hashed draws                 */
    int32_t fp32_activations; /* inference: 0 = tensor cores through warp-level
                             mma.sync (FP16 activations at the MMA inputs, FP32
                             accumulation); 1 = CUDA cores with FP32
                             activations; 2 = tensor cores through tcgen05.mma
                             (same FP16 operands, FP32 accumulators in tensor
                             memory, 128 points per CTA)                      */
} sng_mlp_config;

/* Entries of the parameter vector, or -1 for an unsupported shape. */
int64_t sng_mlp_param_count(int32_t d, int32_t hidden);

/* Column mean / std of x (device n x d) into the mean/std slots of params. */
sng_status sng_mlp_standardize(const float *x, int64_t n, int32_t d, float *params,
                               void *stream);

/* Mean binary cross-entropy of the logits against y (device uint8 0/1, n <=
 * 2^24) and its gradient w.r.t. the trained entries (grad: device FP32,
 * count - 2d).  *loss is written on the host; synchronises `stream`. */
sng_status sng_mlp_loss_grad(const float *x, const uint8_t *y, int64_t n,
                             const sng_mlp_config *cfg, const float *params, float *grad,
                             double *loss, void *stream);

/* `steps` Adam steps (step numbers step0+1 .. step0+steps), each on a batch
 * of cfg->batch rows drawn by the hash from (seed, step) (or taken in order,
 * cfg->sequential).  params / adam_m /
 * adam_v: device FP32 (moments count - 2d entries, zero before the first
 * step).  loss_trace: device FP32[steps] batch losses, or NULL. */
sng_status sng_mlp_train(const float *x, const uint8_t *y, int64_t n, const sng_mlp_config *cfg,
                         float *params, float *adam_m, float *adam_v, int64_t step0,
                         int64_t steps, float *loss_trace, void *stream);

/* p(core) = sigmoid(logit) for every row of x (device n x d) into prob. */
sng_status sng_mlp_predict(const float *x, int64_t n, const sng_mlp_config *cfg,
                           const float *params, float *prob, void *stream);

/*
 * How the surrogate gates points (sng_cluster_surrogate).  p = network
 * probability that the point is core.  p < p_noise: not core, draws the first
 * ceil(noise_draw_frac * m) partners (0: none; it can still become a border
 * point through other points' draws).  p > p_core: core, draws the first
 * ceil(core_draw_frac * m) partners of the same hash stream.  Otherwise all m
 * draws and the core test by degree.  reweight = 1 counts every kept draw of
 * a point that drew m_i < m partners as m / m_i draws (in units of 1/16, at
 * both ends), an unbiased estimate of the degree the plain method would see.
 */
typedef struct {
    float p_noise;
    float p_core;
    float core_draw_frac;   /* (0, 1] */
    float noise_draw_frac;  /* [0, 1] */
    int32_t reweight;       /* 0 or 1 */
    int32_t by_degree;      /* 0: gated points are declared core / not core;
                               1: the gate sets only their draw budgets and
                               every point keeps the degree test (with
                               reweight, an unbiased estimate of its degree) */
} sng_gate;

/*
 * Algorithm 1 gated by the surrogate (see sng_gate).  Same arguments and
 * outputs as sng_cluster (x: FP32, row stride params->ld); stats->queries
 * counts the queries actually issued, stats->surrogate_core / _noise the
 * points gated each way.
 */
sng_status sng_cluster_surrogate(const void *x, const sng_params *params,
                                 const sng_mlp_config *cfg, const float *mlp_params,
                                 const sng_gate *gate, int32_t *labels, uint8_t *core,
                                 sng_stats *stats, void *stream);

/*
 * Clustering that allocates no memory.  The paper has no counterpart: this
 * is an interface for callers that cannot allocate device memory when they
 * cluster -- a plugin whose host application reserved all device memory up
 * front, or a real-time loop that cannot afford cudaMalloc's implicit device
 * synchronisation or its failure under memory pressure.  It gives the same
 * labels and counts as sng_cluster on the same arguments, computed by the
 * batched form's persistent kernel with all scratch in one fixed 16 MiB
 * device array compiled into the library.
 * x: device FP32, n x ld; d <= 64 with ld a multiple of 4 and 16-byte aligned
 * rows, or d <= 4 with any ld.  labels: device int32[n] (caller-owned).
 * Requires n * (4 * ceil(m/32) + 10) bytes plus a few KiB of scratch to fit
 * in 16 MiB, otherwise SNG_EINVAL before any work.  Calls no cudaMalloc,
 * cudaFree or allocating library routine.  The array belongs to this entry
 * point's device code, which CUDA loads on a device the first time it is
 * used there: the first call on each device therefore makes the driver
 * reserve the 16 MiB (kept until the process exits) and looks up the
 * array's device address; make that first call before reserving the rest of
 * device memory and before any stream capture.  Every call shares the array
 * and clears what must start at zero; calls that overlap on the GPU race and
 * must be serialised by the caller.  Synchronises `stream` (to read the
 * status word and fill stats, which may be NULL).
 */
sng_status sng_cluster_noalloc(const float *x, const sng_params *params, int32_t *labels,
                               sng_stats *stats, void *stream);

/*
 * The gather mapping sng_cluster / sng_build_graph would use for these
 * arguments (x is only inspected for its alignment; no CUDA call is made):
 * mapping[0..6] = vector width, lanes per pair, chunks per lane, batches in
 * flight, block size, L2 slices, and 1 if that mapping is compiled (0: the
 * call would fail with SNG_EINVAL).
 */
sng_status sng_gather_mapping(const void *x, const sng_params *params, int32_t *mapping);

/*
 * Measurement aid (no counterpart in the paper): the rate at which the SMs of
 * the current device read from L2.  A device buffer of `bytes` (1 MiB .. 1
 * GiB; pick one well below the L2 size) is allocated, filled, read twice to
 * warm L2, then read `passes` times with 16-byte loads that bypass L1, by
 * every SM; *gbs receives the bytes read per second / 1e9 between two CUDA
 * events.  The roofline of the L2-resident gather forms.  Allocates and
 * frees its buffer; synchronises `stream`.
 */
sng_status sng_measure_l2_read(int64_t bytes, int32_t passes, double *gbs, void *stream);

/*
 * Measurement aid (no counterpart in the paper): the rate at which the SMs
 * of the current device fetch rows at random from a device buffer of n_rows
 * rows of row_bytes (64, 128 or 256) bytes -- the tensor-core gather's
 * access pattern (four lanes per row, eight rows per load instruction,
 * loads that bypass L1) without its hashing, MMAs or decisions, with
 * blocks_per_sm blocks of 8 warps per SM (0: as many as fit).  About
 * `fetches` rows are read after a warm-up; *rows_per_s receives rows per
 * second between two CUDA events.  The ceiling of a gather bound by random
 * row fetches.  Allocates and frees its buffer; synchronises `stream`.
 */
sng_status sng_measure_random_rows(int64_t n_rows, int32_t row_bytes, int64_t fetches,
                                   int32_t blocks_per_sm, double *rows_per_s, void *stream);

/* Number of kernels this library has launched in this process. */
int64_t sng_launch_count(void);

/* One-line reason for the last non-OK status on this thread. */
const char *sng_last_error(void);
const char *sng_strerror(sng_status status);

#ifdef __cplusplus
}
#endif

#endif /* SNG_H */
