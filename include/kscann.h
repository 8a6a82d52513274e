/*
 * kscann.h -- C ABI of the GB300-native KScaNN query path.
 *
 * Method: "KScaNN: Scalable ANN Search on Kunpeng" (arXiv 2511.03298).
 *   build  : Alg. 1 (IVF k-means, PQ with K = 16 on residuals, SIMD blocks,
 *            intra-cluster graphs) with the mean-centroid residual of Sec. 4.6.1.
 *   search : Alg. 2 / Alg. 3 -- rank IVF centroids, per-query residual LUTs
 *            quantised to 8 bits (Sec. 2.5, Sec. 4.5), LUT16 ADC scan of the
 *            probed lists (Eq. 1), candidate pool of size `rerank` (the paper's
 *            `reorder`, Table 1), exact re-rank, top-k.
 *
 * Conventions (every entry point):
 *  - Array arguments named *_dev are DEVICE pointers, caller-allocated, read or
 *    written in order on `stream` (a cudaStream_t passed as void*; NULL = the
 *    legacy default stream).  Arguments named *_host are host pointers.
 *  - Every call is asynchronous on `stream` unless stated; results are valid
 *    once the caller synchronises that stream.
 *  - Return value: a ksc_status.  On failure nothing has been enqueued unless
 *    stated, and ksc_last_error() returns a message (thread-local).
 *  - Row-major layouts: X [n x d] fp32, Q [nq x d] fp32, ids [nq x k] int64,
 *    dists [nq x k] fp32.  Ids are row numbers of X (n < 2^31).
 *  - Distances returned: L2 -> squared Euclidean distance, ascending;
 *    IP -> inner product (similarity), descending.  Ties -> lower id.
 *    Fewer than k results: id -1 and dist +inf (L2) / -inf (IP).
 *  - A handle owns one search workspace: searches through one handle must
 *    not overlap on the GPU.  Searches on different streams may run at the
 *    same time through different handles on the same data (ksc_index_view).
 */
#ifndef KSCANN_H
#define KSCANN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ksc_index ksc_index; /* opaque; owns its device memory */

typedef enum {
    KSC_OK = 0,
    KSC_EINVAL = -1,        /* bad argument (null pointer, size out of range) */
    KSC_ENOMEM = -2,        /* device or host allocation failed */
    KSC_ECUDA = -3,         /* a CUDA runtime call failed */
    KSC_EUNSUPPORTED = -4,  /* valid but unsupported (e.g. nbits != 4) */
    KSC_ETIMEOUT = -5,      /* a bounded device wait gave up */
    KSC_ESTATE = -6         /* object in the wrong state (e.g. no MLP trained) */
} ksc_status;

typedef enum { KSC_L2 = 0, KSC_IP = 1 } ksc_metric;

/* Limits of this implementation (EINVAL beyond them). */
#define KSC_MAX_DIM 1024       /* d */
#define KSC_MAX_M 256          /* PQ subspaces: 256 * 255 < 2^16, u16 lane sums never saturate */
#define KSC_MAX_RERANK 4096    /* candidate pool size R */
#define KSC_MAX_K 1024         /* results per query, k <= R */
#define KSC_MAX_NLIST 65536

/* ------------------------------------------------------------------ */
/* Index construction (Alg. 1)                                         */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t kmeans_iters;      /* Lloyd iterations for IVF and PQ k-means; 0 -> 20 */
    int32_t spherical;         /* 1: rank lists by -<q, c/|c|> (angular data, Sec. 4.6.1);
                                  forced to 1 for KSC_IP */
    const int64_t* perm_host;  /* optional: a permutation of 0..n-1 (host); the IVF
                                  k-means sample is its first min(n, 256 nlist) rows and
                                  also its initial centroids, the PQ sample its first
                                  min(n, 65536).  NULL: the library draws one (seed). */
    uint64_t seed;             /* used when perm_host is NULL */
    int32_t build_graph;       /* 1: build the per-list 32-NN graphs of Sec. 4.4 */
    float filter_threshold;    /* component filtration (Sec. 4.3), 0 = off: dimensions in which
                                  more than this fraction of the values are 0 or within one
                                  standard deviation of the mean are dropped (see
                                  ksc_index_dims) */
} ksc_build_opts;

/* Build an IVF-PQ index from X_dev [n x d] fp32 (device).  nlist = L IVF lists,
 * M PQ subspaces (d % M == 0), nbits must be 4 (K = 16; KSC_EUNSUPPORTED
 * otherwise).  The index copies X (for the exact re-rank).  Blocking: returns
 * after the build has finished on `stream`.  *out is set on success. */
int ksc_build_index(const float* X_dev, int64_t n, int32_t d, int32_t nlist, int32_t M,
                    int32_t nbits, ksc_metric metric, const ksc_build_opts* opts,
                    void* stream, ksc_index** out);

void ksc_index_free(ksc_index* ix);

/* Interchange form of an index, all HOST arrays (used to move an index
 * between this library and other programs).  Codes are unpacked: one byte
 * (0..15) per (vector, subspace).  graph/entry are optional (NULL). */
typedef struct {
    int64_t n;
    int32_t d, nlist, M, metric, spherical;
    float* X;         /* [n x d] */
    float* c_rank;    /* [nlist x d] centroids used to rank lists */
    float* c_mean;    /* [nlist x d] mean centroids used for residuals (Sec. 4.6.1) */
    float* codebook;  /* [M x 16 x d/M] */
    uint8_t* codes;   /* [n x M] */
    int32_t* assign;  /* [n] list of each vector */
    int32_t* graph;   /* [n x 32] neighbours inside the list, -1 padded (optional) */
    int32_t* entry;   /* [nlist] graph entry node per list, -1 if empty (optional) */
} ksc_index_arrays;

/* Create an index from host arrays (copied; the caller keeps ownership).
 * Before any device work the arrays are checked on the host: every code
 * below 16, every assignment in [0, nlist), and, with a graph, every
 * neighbour -1 or a row of the same list and every entry -1 or a row of its
 * list; KSC_EINVAL otherwise.  Blocking. */
int ksc_index_import(const ksc_index_arrays* a, void* stream, ksc_index** out);

/* Query the sizes of an index: fills n, d, nlist, M, metric, spherical of *a
 * and leaves the pointers untouched. */
int ksc_index_info(const ksc_index* ix, ksc_index_arrays* a);

/* Copy an index out into caller-allocated host arrays sized from
 * ksc_index_info (pointers left NULL are skipped).  Blocking. */
int ksc_index_export(const ksc_index* ix, ksc_index_arrays* a);

/* Persistence (not in the paper: an index built once is reused).  Write the
 * index to the file at `path`: the interchange arrays (as ksc_index_export)
 * and, where the index holds them, the intra-list graph, the learned
 * predictor (weights and parameters), the pruning statistics, model and
 * threshold, and the component-filtration state (kept dimensions and full
 * vectors).  Little-endian binary with a 64-byte header; a view writes the
 * index it came from.  Blocking.  KSC_EINVAL if the file cannot be written
 * (then nothing is left at `path`). */
int ksc_index_save(const ksc_index* ix, const char* path);

/* Read a file written by ksc_index_save into a new index (free it with
 * ksc_index_free).  The whole file is checked on the host -- header, exact
 * size, and every code, list, neighbour and dimension index in it -- before
 * any device work: KSC_EINVAL for a missing, truncated, corrupt or foreign
 * file.  Blocking. */
int ksc_index_load(const char* path, void* stream, ksc_index** out);

/* ------------------------------------------------------------------ */
/* Search (Alg. 2, Alg. 3)                                             */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t lanes_per_query;   /* scan kernel: 0 auto; 4: each lane sums all subspaces of one block
                                   (M <= 128); 8/16/32: lanes split the subspaces of a query */
    int32_t hybrid;            /* 1: hybrid intra-cluster search of Sec. 4.4 (needs graphs) */
    int32_t n_near;            /* hybrid: probes of rank < n_near are scanned fully (2) */
    int32_t efs;               /* hybrid: graph-search result capacity (64) */
    int32_t tau;               /* hybrid: full scan when >= tau results beat theta (8) */
    int32_t cand_cap;          /* candidate store per query; 0 -> max(32R, 8192) */
    int32_t rank_fp32;         /* 1: list scores on FP32 CUDA cores instead of 16-bit tensor cores */
    int32_t precision;         /* re-rank: 0 FP32 over R; 1 BF16 rows / 2 FP8-e4m3 rows with a
                                  per-row scale over R (the widened shortlist), then FP32
                                  over the best rerank_final of them */
    int32_t rerank_final;      /* precision 1/2: FP32 re-rank size; 0 -> max(k, R/2) */
    int32_t tile_blocks;       /* scan: 32-vector blocks per work item; 0 auto */
    int32_t scan_tc;           /* 1: the scan on the tensor cores (one-hot codes x FP16 tables,
                                  FP32 sums of integers: the same keys as the byte-permute scan;
                                  M <= 128, not with hybrid); 0: byte permutes on the CUDA cores */
    int32_t rank_fp8;          /* 1: list scores from FP8-e4m3 operands (queries and centroids
                                  scaled per row by a power of two) on the tensor cores, FP32
                                  accumulate; the lists their error bound cannot exclude are
                                  re-scored exactly, so the ranking is the same (rank_fp32 wins
                                  when both are set) */
    int32_t rerank_band;       /* exact FP32 re-rank (precision 0, k <= 32, d <= 128): 1 first reads
                                  low-precision copies of the candidate rows and bounds each FP32
                                  distance (the row's own rounding error plus FP32 evaluation
                                  error); only candidates whose lower bound is at most the k-th
                                  smallest upper bound are read in FP32, so the results are those
                                  of the plain pass; -1 every candidate in FP32; 0 auto: the band
                                  for L2 indexes.  The copies are made on first use: U8 rows
                                  (n d bytes, exact) when every re-rank coordinate is an integer
                                  in [0, 255], else BF16 rows (n d 2 bytes), and two bounds per
                                  row (n 8 bytes).  That first use synchronises the stream once
                                  (the check's result is read on the host), so run one banded
                                  search before capturing the stream in a graph */
} ksc_search_opts;

/* k nearest neighbours of Q_dev [nq x d] with a fixed nprobe (1..nlist) and
 * candidate pool rerank (R, clamped up to k).  ids_dev [nq x k] int64,
 * dists_dev [nq x k] fp32.  opts may be NULL. */
int ksc_search(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int32_t nprobe,
               int32_t rerank, int64_t* ids_dev, float* dists_dev,
               const ksc_search_opts* opts, void* stream);

/* As ksc_search with per-query nprobe_dev [nq] and rerank_dev [nq] (int32,
 * device); nprobe_max / rerank_max bound them (values are clamped into
 * [1, nprobe_max] and [k, rerank_max]). */
int ksc_search_varprobe(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k,
                        const int32_t* nprobe_dev, int32_t nprobe_max,
                        const int32_t* rerank_dev, int32_t rerank_max,
                        int64_t* ids_dev, float* dists_dev,
                        const ksc_search_opts* opts, void* stream);

/* ------------------------------------------------------------------ */
/* List-sharded search (the multi-process protocol of Sec. 5.1 with the  */
/* lists themselves partitioned, for an index larger than one device)   */
/* ------------------------------------------------------------------ */
/* Create shard `shard` of a list-partitioned index from the whole index's
 * host arrays (copied; graph / entry ignored): the lists p with
 * list_owner[p] == shard keep their members, in ascending row id, every
 * other list is empty; centroids and codebooks are replicated.  The shard
 * keeps the global row id of each of its vectors.  Checked on the host before
 * device work: arrays as ksc_index_import, owners >= 0, at least one vector
 * in the shard (KSC_EINVAL).  Blocking.  Free with ksc_index_free. */
int ksc_index_import_shard(const ksc_index_arrays* full, const int32_t* list_owner, int32_t shard,
                           void* stream, ksc_index** out);

/* Shard step 1 (Alg. 2 / Alg. 3 up to the candidate pool): rank all lists,
 * build the tables of every probed list (so the per-query scale is the whole
 * index's), scan the shard's own lists and keep its R = max(rerank, k)
 * smallest keys per query: keys_dev [nq x R] uint64, ((D + 2^31) << 32) |
 * global id, ascending, padded with all-ones.  Fixed nprobe; opts as
 * ksc_search except hybrid and the low-precision re-rank (KSC_EINVAL). */
int ksc_shard_candidates(ksc_index* shard, const float* Q_dev, int64_t nq, int32_t nprobe, int32_t rerank,
                         int32_t k, uint64_t* keys_dev, const ksc_search_opts* opts, void* stream);

/* Shard step 2 (Alg. 2 re-rank), after an exchange of every shard's keys:
 * all_keys_dev [parts x nq x R] (shard-major, as an all-gather lays them
 * out), own_keys_dev [nq x R] this shard's from step 1.  theta = the R-th
 * smallest of all keys of the query (the whole index's R-th key); the
 * shard's own keys at or below it are re-ranked exactly -> ids_dev
 * [nq x k] int64 (global ids) and dists_dev [nq x k] as ksc_search (short
 * lists padded with -1 / +-inf).  parts x R <= 8192. */
int ksc_shard_rerank(ksc_index* shard, const float* Q_dev, int64_t nq, int32_t k, int32_t rerank,
                     const uint64_t* own_keys_dev, const uint64_t* all_keys_dev, int32_t parts,
                     int64_t* ids_dev, float* dists_dev, void* stream);

/* Final merge of the shards' results: ids_dev / dists_dev [parts x nq x k]
 * -> the k best per query by distance (ip = 0: ascending L2 distance;
 * ip = 1: descending similarity), then id; pads (id -1) last.  The merged
 * result of steps 1-2 on every shard equals ksc_search on the whole index.
 * parts x k <= 8192. */
int ksc_merge_topk(const int64_t* ids_dev, const float* dists_dev, int64_t nq, int32_t parts, int32_t k,
                   int32_t ip, int64_t* ids_out_dev, float* dists_out_dev, void* stream);

/* Test entry: search with caller-given probe lists probes_dev [nq x P]
 * (list ids, in rank order).  Optional outputs (NULL to skip):
 * cand_dev [nq x R] uint64 candidate keys ((D + 2^31) << 32 | id), sorted
 * ascending, padded with all-ones; ncand_dev [nq] int32 number of candidates. */
int ksc_search_with_probes(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev,
                           int32_t P, int32_t k, int32_t rerank, int64_t* ids_dev, float* dists_dev,
                           uint64_t* cand_dev, int32_t* ncand_dev,
                           const ksc_search_opts* opts, void* stream);

/* ------------------------------------------------------------------ */
/* Batched execution: captured plans and the autotuner                 */
/* ------------------------------------------------------------------ */
/* A plan fixes an index, batch size nq, k, nprobe, rerank and options,
 * warms the index workspace and captures the whole search (every kernel and
 * memset) into one CUDA graph that reads its queries from, and writes its
 * results to, plan-owned device buffers.  adaptive = 1 captures
 * ksc_search_adaptive (nprobe/rerank then ignored).  `stream` must not be the
 * legacy default stream (capture is not allowed there).  Blocking. */
typedef struct ksc_plan ksc_plan;
int ksc_plan_create(ksc_index* ix, int64_t nq, int32_t k, int32_t nprobe, int32_t rerank, int32_t adaptive,
                    const ksc_search_opts* opts, void* stream, ksc_plan** out);

/* Replay a plan on `stream`: Q_dev [nq x d] is copied into the plan's input
 * buffer (skipped when it is that buffer), the graph is launched and the
 * results are copied to ids_dev / dists_dev (skipped when NULL or the plan's
 * own buffers).  If the index workspace was reallocated since the capture
 * (another search with larger shapes), the plan re-captures first. */
int ksc_plan_execute(ksc_plan* plan, const float* Q_dev, int64_t* ids_dev, float* dists_dev, void* stream);

/* The plan's own device buffers (input queries, output ids / distances). */
int ksc_plan_buffers(ksc_plan* plan, float** Q_dev, int64_t** ids_dev, float** dists_dev);

void ksc_plan_free(ksc_plan* plan);

/* Autotuner: times the scan's lanes-per-query (8/16/32) and tile length
 * (auto, 8, 16, 32, 64 blocks) on the batch Q_dev [nq x d] with the given k,
 * nprobe, rerank and options, and writes the fastest into
 * opts_inout->lanes_per_query / tile_blocks; *best_ms_host (may be NULL)
 * receives its time per search.  Blocking. */
int ksc_autotune(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int32_t nprobe, int32_t rerank,
                 ksc_search_opts* opts_inout, void* stream, float* best_ms_host);

/* Step a1 alone (TopNClusters of Alg. 2): the P best lists per query,
 * probes_dev [nq x P] int32, scores_dev [nq x P] fp32 (L2 distance to the
 * ranking centroid, or -<q, c> for spherical indexes); scores may be NULL. */
int ksc_rank_lists(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t P, int32_t* probes_dev,
                   float* scores_dev, void* stream);

/* Raw list scores of step a1: scores_dev [nq x L] fp32 = ||c||^2 - 2<q, c>
 * (L2; ||q||^2 omitted) or -<q, c> (spherical), c the ranking centroids.
 * tensor_cores = 1: 16-bit operands on the tensor cores (tcgen05, d <= 256);
 * tensor_cores = 2: FP8-e4m3 operands with per-row power-of-two scales on
 * the tensor cores (kind::f8f6f4, d <= 256); tensor_cores = 0 (or d > 256):
 * FP32 CUDA cores.  err_dev [nq] (may be
 * NULL) receives a bound on |score - exact score| for every list of the
 * query; ranking re-scores exactly every list within twice that bound. */
int ksc_list_scores(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t tensor_cores, float* scores_dev,
                    float* err_dev, void* stream);

/* Step a2 alone: quantised LUTs lut_dev [nq x P x M x 16] uint8, biases
 * bias_dev [nq x P] int32 and scales scale_dev [nq] fp32 for the given probes. */
int ksc_compute_luts(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev,
                     int32_t P, uint8_t* lut_dev, int32_t* bias_dev, float* scale_dev, void* stream);

/* Allocation-free variant of ksc_compute_luts (the paper has no counterpart:
 * this entry point exists for callers that cannot let the library call
 * cudaMalloc -- a program whose device memory is reserved by its own
 * allocator, or a latency-critical path that cannot take the device
 * synchronisation an allocation may cause).  Same arguments, layouts and
 * results as ksc_compute_luts; it calls no cudaMalloc / cudaFree.  Its only
 * scratch (4 bytes per query) lives in a fixed device array of
 * KSC_NOALLOC_MAX_NQ entries that every GPU loading the library holds until
 * the process exits; nq > KSC_NOALLOC_MAX_NQ is rejected with KSC_EINVAL.
 * The first call on a device, with that device current, looks up the
 * array's device address; make that first call before any stream capture.
 * Every call shares the array: calls whose work overlaps on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller. */
#define KSC_NOALLOC_MAX_NQ 65536
int ksc_compute_luts_noalloc(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev,
                             int32_t P, uint8_t* lut_dev, int32_t* bias_dev, float* scale_dev, void* stream);

/* ------------------------------------------------------------------ */
/* Learned per-query nprobe / reorder (Sec. 4.2.1-4.2.2, Eq. 2)        */
/* ------------------------------------------------------------------ */
/* A small MLP stands in for the paper's gradient-boosted classifier.
 * Features: the 32 smallest list distances of the query (ranking step) as
 * d_i / mean(d) and d_1 / d_i (64 values).  Network 64 -> 64 -> 64 -> 2,
 * ReLU, two sigmoid heads p_n (nprobe) and p_r (rerank), FP32 weights packed
 * as W1[64x64], b1, W2[64x64], b2, W3[2x64], b3 (KSC_MLP_NPARAMS floats);
 * inference rounds weights and activations to BF16.  Eq. 2 maps p to
 *   P = min(Pmax, Pmin + ceil((Pmax - Pmin) * max(0, p - p0) * (p + p1)))
 * and likewise R with (rmin, rmax, r0, r1). */
#define KSC_MLP_NPARAMS 8450
#define KSC_MLP_FEATURES 64

typedef struct {
    int32_t pmin, pmax;   /* nprobe range */
    int32_t rmin, rmax;   /* rerank range */
    float p0, p1;         /* Eq. 2 parameters of the nprobe head */
    float r0, r1;         /* Eq. 2 parameters of the rerank head */
    int32_t regression;   /* 1: regression heads (ksc_train_opts.regression): p is the
                             normalised log of the setting, u = clamp(p (1 + p1) + p0, 0, 1),
                             P = clamp(ceil(pmin (pmax / pmin)^u - 1e-3), pmin, pmax), and
                             likewise R with (rmin, rmax, r0, r1); 0: Eq. 2 */
} ksc_adaptive_params;

typedef struct {
    int32_t k;              /* neighbours used by the labels (10) */
    int32_t target_hits;    /* a setting suffices when >= target_hits of them are found (9) */
    int32_t rerank_label;   /* rerank while labelling nprobe (200) */
    int32_t epochs;         /* training epochs (8) */
    int32_t batch;          /* minibatch size (256) */
    float lr;               /* Adam learning rate (1e-3) */
    uint64_t seed;          /* weight initialisation and sample order */
    const int32_t* grid_host;   /* ascending nprobe grid; NULL -> 4,6,8,12,16,24,32,48,64,96,128 */
    int32_t ngrid;
    const int32_t* rgrid_host;  /* ascending rerank grid; NULL -> 20,50,100,200,400 */
    int32_t nrgrid;
    int32_t regression;     /* 1: regression heads trained on soft targets, the normalised
                               logs (log label - log grid min) / (log grid max - log grid min);
                               sets ksc_adaptive_params.regression (0: "hard" labels, Eq. 2) */
} ksc_train_opts;

/* Train the predictor of this index on the queries Qtrain_dev [nt x d] whose
 * true k-th neighbour distances are kth_dev [nt] (device; L2 distance, or
 * similarity for IP).  Labels come from the plain search: for each query the
 * smallest grid nprobe whose top-k holds at least target_hits ids with
 * distance within the true k-th ("hard" = above the median of these labels),
 * and likewise the smallest grid rerank at that nprobe.  Hand-written FP32
 * forward / backward / Adam kernels.  Blocking.  Sets default Eq. 2
 * parameters (grid ends, p0 = r0 = 0.3, p1 = r1 = 0.5); *loss_host (may be
 * NULL) receives the last epoch's mean loss.  opts may be NULL. */
int ksc_train_predictor(ksc_index* ix, const float* Qtrain_dev, int64_t nt, const float* kth_dev,
                        const ksc_train_opts* opts, void* stream, float* loss_host);

/* Set the Eq. 2 parameters used by ksc_search_adaptive. */
int ksc_predictor_params(ksc_index* ix, const ksc_adaptive_params* prm);

/* Copy the predictor weights out (w_host != NULL) and/or in (w_in_host !=
 * NULL), KSC_MLP_NPARAMS floats each.  Blocking.  KSC_ESTATE if neither is
 * given a trained model to read. */
int ksc_predictor_weights(ksc_index* ix, float* w_host, const float* w_in_host);

/* Search with per-query nprobe and rerank predicted by the trained MLP
 * (KSC_ESTATE if none).  nprobe_dev / rerank_dev [nq] (may be NULL) receive
 * the predicted values. */
int ksc_search_adaptive(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int64_t* ids_dev,
                        float* dists_dev, int32_t* nprobe_dev, int32_t* rerank_dev,
                        const ksc_search_opts* opts, void* stream);

/* Predictor features of Q_dev: feats_dev [nq x 64]. */
int ksc_query_features(ksc_index* ix, const float* Q_dev, int64_t nq, float* feats_dev, void* stream);

/* Training kernels alone (for checks): loss and gradient of the mean
 * binary cross-entropy of the two heads over x_dev [B x 64] with targets
 * y_dev [B x 2] at weights w_dev; grad_dev [KSC_MLP_NPARAMS], loss_dev [1]. */
int ksc_mlp_grad(const float* w_dev, const float* x_dev, const float* y_dev, int64_t B, float* grad_dev,
                 float* loss_dev, void* stream);

/* BF16 inference alone: prob_dev [B x 2]. */
int ksc_mlp_forward(const float* w_dev, const float* x_dev, int64_t B, float* prob_dev, void* stream);

/* ------------------------------------------------------------------ */
/* Predictive cluster pruning (Sec. 4.2.3, Table 4; Alg. 2 f_prune)    */
/* ------------------------------------------------------------------ */
/* A classifier per (query, probed list) predicts whether the list holds one
 * of the query's true nearest neighbours; Alg. 2 searches a list only when
 * f_prune > theta.  Here the nearest probe (rank 0) is always searched and
 * the others are dropped before the work lists are built, so the scan runs
 * unchanged on the shorter per-query probe lists (no divergence in it).
 *
 * Per-list statistics (build time, KSC_PRUNE_STATS floats per list) of the
 * members' offsets r = x - c from the list's mean centroid: 0 size n,
 * 1 radius rho = max |r|, 2 mean mu and 3 population std sigma of |r|,
 * 4..7 the distance histogram (fractions in [0, rho/4], (rho/4, rho/2],
 * (rho/2, 3 rho/4], (3 rho/4, rho]), 8 the outlier fraction (|r| > mu + 2
 * sigma), 9, 10 the variances along the two principal axes, 11 zero; and
 * 3 vectors of d floats per list: the principal axes v1, v2 of the
 * offsets' second moment (30 power iterations each, v1 from (1,..,1),
 * v2 from (+1,-1,+1,..) with v1 projected out) and the mean outlier offset.
 *
 * Features of (q, rank r) (KSC_PRUNE_FEATURES floats), with p the list,
 * D = |q - c_p|, u = (q - c_p) / D, D0 = |q - c_{rank 0}|, g = max(D0, 1e-9):
 * D / rho, D / g, (D - rho) / g, log(1 + n), rho / g, mu / g, sigma / g,
 * the 4 histogram fractions, the outlier fraction, lambda1 <v1, u>^2 / g^2,
 * lambda2 <v2, u>^2 / g^2, <outlier offset, u> / g, D0 / rho_{rank 0}.
 *
 * Model (KSC_PRUNE_MODEL floats): MLP weights W1[32x16], b1, W2[32x32], b2,
 * W3[2x32], b3 (KSC_PRUNE_NPARAMS; ReLU, sigmoid; head 0 is the keep
 * probability), then the per-feature means and standard deviations that
 * standardise the features before the MLP.  FP32 inference. */
#define KSC_PRUNE_STATS 12
#define KSC_PRUNE_FEATURES 16
#define KSC_PRUNE_NPARAMS 1666
#define KSC_PRUNE_MODEL (KSC_PRUNE_NPARAMS + 2 * KSC_PRUNE_FEATURES)

/* Compute the per-list statistics of this index (iters power iterations per
 * axis, <= 0: 30).  Done by ksc_train_pruner when missing.  d <= 1024. */
int ksc_pruner_stats(ksc_index* ix, int32_t iters, void* stream);

/* Copy out the statistics stats_host [L x KSC_PRUNE_STATS], the vectors
 * vecs_host [L x 3 x d] and the model model_host [KSC_PRUNE_MODEL] (host
 * buffers, each may be NULL).  Blocking.  KSC_ESTATE when a requested part
 * has not been computed or trained. */
int ksc_pruner_export(ksc_index* ix, float* stats_host, float* vecs_host, float* model_host);

/* Set the model from model_host [KSC_PRUNE_MODEL] (host).  Blocking. */
int ksc_pruner_import_model(ksc_index* ix, const float* model_host);

/* Features, keep probabilities and pruned probe lists for given probes.
 * probes_dev [nq x Pmax] list ids by rank (device); the query's probes are
 * the first nprobe_dev[q] (device, may be NULL: P for every query).  Outputs
 * (device, each may be NULL): feats_dev [nq x Pmax x KSC_PRUNE_FEATURES]
 * (rows at rank >= the query's nprobe are zero), prob_dev [nq x Pmax] (keep
 * probability; needs a model; rows at rank >= the query's nprobe are left
 * unwritten), probes_out_dev [nq x Pmax] the kept probes in
 * rank order then -1, nprobe_out_dev [nq] their number (rank 0 and every
 * rank with probability > theta; needs a model).  Needs the statistics
 * (KSC_ESTATE otherwise). */
int ksc_prune_probes(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev, int32_t Pmax,
                     const int32_t* nprobe_dev, int32_t P, float theta, float* feats_dev, float* prob_dev,
                     int32_t* probes_out_dev, int32_t* nprobe_out_dev, void* stream);

/* Training labels: label_dev [nq x Pmax] = 1 where the list probes_dev[q][r]
 * (r < P) holds one of the returned ids_dev [nq x k] whose distance
 * dists_dev [nq x k] is within the true k-th kth_dev [nq] (L2: at most it,
 * IP: at least it, both up to 1e-5 relative + 1e-6), else 0 (device). */
int ksc_prune_labels(ksc_index* ix, const int64_t* ids_dev, const float* dists_dev, int64_t nq, int32_t k,
                     const float* kth_dev, const int32_t* probes_dev, int32_t Pmax, int32_t P, float* label_dev,
                     void* stream);

/* Train the pruning model on the queries Qtrain_dev [nt x d] with true k-th
 * distances kth_dev [nt]: each query's P nearest lists are searched with
 * rerank R, labelled as in ksc_prune_labels and featurised; the features are
 * standardised over all rows; the MLP is trained with binary cross-entropy
 * (both heads on the label) by the FP32 kernels and Adam.  opts: epochs (4),
 * batch (1024 rows), lr (1e-3), seed; other fields unused; may be NULL.
 * Blocking.  *loss_host (may be NULL) receives the mean loss of the last
 * epoch. */
int ksc_train_pruner(ksc_index* ix, const float* Qtrain_dev, int64_t nt, const float* kth_dev, int32_t k,
                     int32_t P, int32_t R, const ksc_train_opts* opts, void* stream, float* loss_host);

/* ksc_search with pruning: the nprobe nearest lists of each query, then
 * those the model keeps at theta (as ksc_prune_probes), then the search of
 * the kept lists.  nprobe_out_dev [nq] (device, may be NULL) receives the
 * number of lists searched per query.  KSC_ESTATE without a model. */
int ksc_search_pruned(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int32_t nprobe, int32_t rerank,
                      float theta, int64_t* ids_dev, float* dists_dev, int32_t* nprobe_out_dev,
                      const ksc_search_opts* opts, void* stream);

/* Pruning inside ksc_search_adaptive (Alg. 2 order: predicted nprobe, then
 * f_prune > theta over those lists; nprobe_dev there receives the number of
 * lists searched).  theta < 0, the default, turns it off; KSC_ESTATE for
 * theta >= 0 without statistics and model.  Captured adaptive plans
 * re-capture before their next execution. */
int ksc_pruner_theta(ksc_index* ix, float theta);

/* Loss and gradient of the pruning MLP (16 -> 32 -> 32 -> 2, mean binary
 * cross-entropy of both heads) over x_dev [B x 16], y_dev [B x 2] at w_dev
 * [KSC_PRUNE_NPARAMS]; grad_dev [KSC_PRUNE_NPARAMS], loss_dev [1] (device). */
int ksc_prune_mlp_grad(const float* w_dev, const float* x_dev, const float* y_dev, int64_t B, float* grad_dev,
                       float* loss_dev, void* stream);

/* ------------------------------------------------------------------ */
/* Component filtration (Sec. 4.3; Alg. 1 / Alg. 2 FilterComponents)  */
/* ------------------------------------------------------------------ */
/* With ksc_build_opts.filter_threshold > 0 the build keeps the dimensions
 * whose fraction (ksc_component_stats) is at most the threshold, in
 * ascending order, and builds the index on those: the sub-vector width stays
 * d / M, so the filtered index has ceil(kept / (d / M)) subspaces, the last
 * completed with zero dimensions.  Queries are still passed with all d
 * dimensions; every search drops the same ones before ranking, tables and
 * scan, and re-ranks with the full query against the full vectors (Alg. 2).
 * ksc_index_info and ksc_index_export then describe the filtered (working)
 * index, whose X holds the kept dimensions.  Not with ksc_index_import or
 * ksc_compute_luts_noalloc (KSC_EUNSUPPORTED). */

/* The working dimension list of the index: d_full_host receives the query
 * width d; dims_host (may be NULL) receives, for each working dimension, the
 * query dimension it takes (-1: a zero padding dimension).  Without
 * filtration the list is 0..d-1.  Blocking. */
int ksc_index_dims(ksc_index* ix, int32_t* dims_host, int32_t* d_full_host);

/* Per-dimension statistics of X_dev [n x d] (device): mean mu_dev, population
 * standard deviation sd_dev and the fraction of values that are 0 or within
 * one standard deviation of the mean frac_dev ([d] doubles each, device),
 * FP64 with a fixed summation order. */
int ksc_component_stats(const float* X_dev, int64_t n, int32_t d, double* mu_dev, double* sd_dev, double* frac_dev,
                        void* stream);

/* Device status word of the last search on this index: 0 = clean, else a
 * bitwise OR of KSC_STATUS_* (blocking read). */
#define KSC_STATUS_CAND_OVERFLOW 1  /* a query's candidate store overflowed and was redone exactly */
int ksc_last_status(ksc_index* ix, int32_t* status_host);

/* Stage timing of searches on this index (CUDA events recorded on the
 * search stream; off by default).  Stages, in order: 0 rank lists (a1),
 * 1 work lists, 2 LUT build + quantise (a2), 3 LUT16 scan of each query's
 * nearest list + candidate threshold, 4 LUT16 scan of the other probed lists
 * (a3), 5 candidate select (a5), 6 rerank (a6).  ksc_profile_read
 * synchronises with the last profiled search and writes its per-stage
 * milliseconds into ms_host[0..n) (n <= 8) and the number of kernels it
 * launched into *launches_host (may be NULL). */
#define KSC_NUM_STAGES 7
int ksc_profile_enable(ksc_index* ix, int32_t on);
int ksc_profile_read(ksc_index* ix, float* ms_host, int32_t n, int32_t* launches_host);

/* Diagnostic: runs the scan's lookup/accumulate instruction sequences with
 * no global memory traffic on every SM and returns the rates reached, in
 * 10^9 lookups per second, into glookups_host[2]: [0] the sequence of items
 * whose query slots share a block (selectors computed once per warp, read
 * from shared memory; two lookups per byte dot product), [1] the per-slot
 * sequence (selectors in registers; sparse items).  The integer-ALU
 * ceilings of the a3 scan.  Blocking. */
int ksc_lut16_peak(double* glookups_host, void* stream);

/* Diagnostic: distances of the pairs (query q, ids_dev[q][i]) [nq x c] in
 * precision 0 (FP32 rows), 1 (BF16 rows) or 2 (FP8-e4m3 rows with a per-row
 * scale), FP32 query and accumulation; out_dev [nq x c] (L2 squared distance
 * or IP similarity; NaN for id < 0). */
int ksc_pair_distances(ksc_index* ix, const float* Q_dev, int64_t nq, const int64_t* ids_dev, int32_t c,
                       int32_t precision, float* out_dev, void* stream);

/* Counters of the last search on this index (blocking read), stats_host[4]:
 * [0] queries whose candidate store overflowed (redone exactly),
 * [1] candidates kept by the scan's threshold filter (all queries),
 * [2] most candidates kept for one query, [3] reserved (0). */
int ksc_search_stats(ksc_index* ix, int64_t* stats_host);

/* A second handle on the index data of ix (device arrays, models and
 * statistics shared, not copied) with its own search workspace, status word,
 * counters and stage events, so that searches on different streams can run
 * at the same time, one handle each (e.g. single-query searches on several
 * streams).  Free every view (ksc_index_free) before the handle it came from.
 * A view does not train or set models or statistics (KSC_ESTATE); do not
 * retrain the index while views of it exist. */
int ksc_index_view(ksc_index* ix, ksc_index** out);

/* Message of the last failure on this thread ("" if none). */
const char* ksc_last_error(void);

/* Library version string. */
const char* ksc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KSCANN_H */
