/*
 * finger.h — C ABI of the GB300 (sm_103a) FINGER search library, libfinger.so.
 *
 * FINGER (Chen, Chang, Yu, Dhillon, Hsieh, arXiv 2206.11408) speeds up greedy
 * search on a proximity graph by estimating most neighbour distances from a
 * rank-r model of the residual angle and computing the exact distance only
 * when the estimate does not exceed the current upper bound.
 *
 * Conventions for every entry point
 *   - Distances are squared L2 (the paper's L2 distance, Sec. 3.2, squared; the
 *     order is the same).  Keys are (distance, id), compared lexicographically.
 *   - "device" pointers are CUDA global-memory addresses on the index's device;
 *     "host" pointers are ordinary (preferably pinned) CPU memory.  The caller
 *     owns every buffer it passes; the library owns the index and its scratch.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream are asynchronous on it; argument errors are
 *     returned synchronously, before anything is enqueued.  Errors raised
 *     inside a kernel (an iteration or capacity limit) are latched in a device
 *     status word and returned by finger_get_stats() and finger_sync().
 *   - No entry point falls back to the CPU: the compute runs in this library's
 *     CUDA kernels or the call fails.
 *   - The library is not thread-safe for concurrent calls on one index.
 */
#ifndef FINGER_H
#define FINGER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct finger_index finger_index; /* opaque, library-owned */

typedef enum {
    FINGER_OK = 0,
    FINGER_ERR_INVALID_ARG = 1, /* bad pointer, size, K > ef, ef above capacity, ... */
    FINGER_ERR_IO = 2,          /* file could not be opened, read or written */
    FINGER_ERR_FORMAT = 3,      /* index file with wrong magic, version or sizes */
    FINGER_ERR_OOM = 4,         /* device or host allocation failed */
    FINGER_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    FINGER_ERR_NOT_BUILT = 6,   /* graph or FINGER tables missing for the request */
    FINGER_ERR_LIMIT = 7,       /* a kernel hit an iteration/capacity bound (latched) */
    FINGER_ERR_UNSUPPORTED = 8  /* a size this build does not handle (e.g. m > 1024) */
} finger_status;

/* search modes (finger_set_mode) */
enum {
    FINGER_MODE_PLAIN = 0,      /* Algorithm 1: exact distance for every new neighbour */
    FINGER_MODE_FINGER = 1,     /* Algorithm 4 with Algorithm 3 as the gate */
    FINGER_MODE_FINGER_LP = 2,  /* Algorithm 4 on BF16 rows and FP8-e4m3 residual codes,
                                   FP32 accumulation, final top-K re-ranked in FP32 */
    FINGER_MODE_FINGER_MLP = 3, /* Algorithm 4 with a learned angle predictor in place of
                                   distribution matching; matching is the fallback */
    FINGER_MODE_FINGER_F16 = 4, /* Algorithm 4 with the per-edge unit residual projections
                                   (Supplementary G) stored as FP16 codes; FP32 vectors and
                                   FP32 arithmetic.  Needs tables built with
                                   FINGER_BUILD_HALF_CODES.  The whole code block of the
                                   expanded node (deg0 rows, contiguous) is read together
                                   with its adjacency row, so an expansion needs one
                                   dependent round trip to memory fewer than in mode FINGER */
    FINGER_MODE_FINGER_F8 = 5   /* as FINGER_F16 with the codes stored as FP8-e4m3 of
                                   256 u (the LP mode's code table: half the bytes and
                                   half the registers per code block); the product is
                                   an FP8 tensor-core MMA with 256 u_q split into an
                                   e4m3 part and the e4m3 rounding of the rest, FP32
                                   accumulation; FP32 vectors.  Needs tables built
                                   with FINGER_BUILD_FP8_CODES or build_lp */
};

/* --------------------------------------------------------------- index */

/* Create an index on CUDA device `device` from n row-major FP32 vectors of
 * dimension m (host pointer, n*m floats, copied).  1 <= m <= 1024, n < 2^31.
 * The index has no graph yet. */
finger_status finger_index_create(int device, int64_t n, int m, const float* vectors_host,
                                  finger_index** out);

/* Attach an HNSW-style graph given in host arrays (copied):
 *   adj0     n x deg0 int32  layer-0 neighbour lists, valid ids first, -1 pad,
 *                            no duplicates and no self-loops within a row
 *   level    n int32         top level of each node (0 for layer-0 only)
 *   up_off   n int64         row of (v, level 1) in up_adj, -1 if level[v] == 0;
 *                            rows of levels 1..level[v] are consecutive
 *   up_adj   up_rows x M int32  upper-level neighbour lists, -1 pad
 *   entry, maxlevel          entry point (level[entry] == maxlevel)
 * deg0 <= 64, M <= 32.  Invalidates FINGER tables built for a previous graph. */
finger_status finger_index_set_graph(finger_index* ix, int deg0, const int32_t* adj0,
                                     const int32_t* level, const int64_t* up_off,
                                     int64_t up_rows, int M, const int32_t* up_adj,
                                     int32_t entry, int32_t maxlevel);

typedef struct {
    int M;                /* degree cap on levels >= 1; layer 0 allows 2M (<= 32) */
    int candidates;       /* exact nearest neighbours offered to the pruning step
                             (efConstruction; <= 256; 0 = 2 * 2M) */
    uint64_t level_seed;  /* seed of the level draw floor(-ln U / ln M) */
    int symmetric;        /* 0 (default): HNSW insertion order, node i draws its
                             candidates from the nodes j < i of its level only;
                             1: from all nodes of its level */
    int flat;             /* 1: every node on level 0 (no hierarchy, entry point
                             node 0): a single-layer navigable small-world graph */
    int fp32_candidates;  /* 1: layer-0 candidates by FP32 FFMA distances; 0
                             (default): on the tensor cores (BF16 high/low split
                             products, ~1e-5 relative distance error) */
} finger_graph_params;

/* Build an HNSW graph on the device.  Levels are drawn as in HNSW from a
 * counter-based generator; nodes are inserted in id order.  For every level
 * and node i: the exact `candidates` nearest among the level's nodes inserted
 * before i (brute force on the GPU: HNSW's efConstruction beam search made
 * exact), HNSW's heuristic selection of M forward links (keep a candidate
 * only if it is closer to the node than to every neighbour kept so far),
 * reverse links from later nodes, and a second heuristic pass over forward
 * and reverse links to the level's cap (2M on layer 0, M above).  The upper
 * levels use up to 256 candidates.  Synchronous. */
finger_status finger_build_graph(finger_index* ix, const finger_graph_params* p, void* stream);

/* Copy the graph back to host arrays of the sizes given by finger_get_info().
 * Any pointer may be NULL to skip that array. */
finger_status finger_get_graph(const finger_index* ix, int32_t* adj0, int32_t* level,
                               int64_t* up_off, int32_t* up_adj, int32_t* entry,
                               int32_t* maxlevel);

typedef struct {
    int64_t n;
    int m;
    int deg0;
    int M;
    int maxlevel;
    int entry;
    int64_t up_rows;
    int r;               /* FINGER rank, 0 before finger_build_tables */
    int has_lp;          /* BF16 rows and FP8 codes present (mode LP) */
    int has_mlp;         /* learned predictor present */
    int64_t device_bytes;/* device memory held by the index */
    int has_half_codes;  /* FP16 codes present (mode FINGER_F16) */
    int has_fp8_codes;   /* FP8 codes present (mode FINGER_F8) */
} finger_info;

finger_status finger_get_info(const finger_index* ix, finger_info* out);

/* Save / load the whole search index in a versioned little-endian binary
 * file: the vectors, the graph, and what FINGER precomputes once and stores
 * with the index before any query (Sec. 3.3: the basis P and the matching
 * statistics; Supplementary G: c^T c and P c per node, and per layer-0 edge
 * the unit projected residual, ||d_res|| and b, whose memory Supplementary F
 * accounts as (r + 2) floats per edge), plus the LP tables and the learned
 * predictor when present.  load places it on `device`.  The caller owns
 * `path`; *out receives a new index the caller frees with finger_index_free.
 * Errors: FINGER_ERR_IO (open/read/write), FINGER_ERR_FORMAT (magic, version
 * or sizes), FINGER_ERR_OOM, FINGER_ERR_CUDA. */
finger_status finger_index_save(const finger_index* ix, const char* path);
finger_status finger_index_load(const char* path, int device, finger_index** out);
void finger_index_free(finger_index* ix);

/* ------------------------------------------------------- FINGER tables */

typedef struct {
    int r;                    /* rank, 1 <= r <= 64 (Sec. 3.3, Supplementary E) */
    uint64_t seed;            /* seed of the neighbour-pair draw of Algorithm 2 */
    int samples_per_node;     /* pairs drawn per node (Algorithm 2 draws one); 0 = 1 */
    const float* basis_host;  /* optional r x m row-major P; NULL = SVD on the device */
    const double* stats_host; /* optional {mu, sigma, mu_hat, sigma_hat, eps};
                                 NULL = computed from the sampled pairs */
    int build_lp;             /* also build BF16 rows and FP8-e4m3 codes (mode LP) */
    int flags;                /* ablations of Sec. 4.3, 0 = the full method:
                                 FINGER_BUILD_NO_MATCHING: t = t_hat + eps
                                 (stored as mu = mu_hat = 0, sigma = sigma_hat
                                 = 1; eps = mean |Y - X|);
                                 FINGER_BUILD_NO_EPS: eps = 0;
                                 and FINGER_BUILD_HALF_CODES /
                                 FINGER_BUILD_FP8_CODES (below) */
} finger_build_params;

#define FINGER_BUILD_NO_MATCHING 1
#define FINGER_BUILD_NO_EPS 2
/* also store every edge's unit residual projection P d_res / ||P d_res|| as
 * FP16 codes (round to nearest even from FP32) for FINGER_MODE_FINGER_F16:
 * per node 32 (deg0 <= 32) or 64 slots x 32 or 64 codes (r <= 32 or 64),
 * zero padded, in the tensor cores' operand order, plus a copy of the
 * layer-0 adjacency whose ids carry one flag bit (the neighbour has more than
 * half of deg0's slots' worth of neighbours).  Needs n < 2^30, else
 * FINGER_ERR_UNSUPPORTED.  Not an ablation: the matching statistics are those
 * of the FP32 tables. */
#define FINGER_BUILD_HALF_CODES 4
/* also store the same unit projections as FP8-e4m3 codes of 256 u (round to
 * nearest even, saturating) for FINGER_MODE_FINGER_F8, in the same operand
 * order with two k steps per 16 bytes, plus the tagged adjacency; build_lp
 * builds them as well.  Needs n < 2^30, else FINGER_ERR_UNSUPPORTED. */
#define FINGER_BUILD_FP8_CODES 8

/* Algorithm 2 and Supplementary G on the device.  For every node c with at
 * least two layer-0 neighbours a pair (d, d') is drawn with the counter rule
 *   h1 = splitmix64(seed ^ (c * spn + k)), h2 = splitmix64(h1),
 *   i = h1 mod deg(c), j = h2 mod (deg(c) - 1), j += (j >= i)
 * (i, j index the valid neighbours in row order); D_res collects
 * d_res = d - (c^T d / c^T c) c; P = top-r eigenvectors of D_res D_res^T
 * (= U_{1:r}^T of the SVD, Proposition 1) by FP64 Jacobi; then per node
 * ||c||^2 and P c, per layer-0 edge (c, d) the row (P d_res / ||P d_res||,
 * ||d_res||, c^T d / c^T c) — (r + 2) floats per edge slot, Supplementary F —
 * and the matching statistics mu, sigma, mu_hat, sigma_hat (standard
 * deviations) and eps of Algorithm 2 over the drawn pairs, with
 * X = cos(d_res, d'_res), Y = cos(P d_res, P d'_res).  Synchronous. */
finger_status finger_build_tables(finger_index* ix, const finger_build_params* p, void* stream);

/* Rank rule of Supplementary E, then finger_build_tables at the chosen rank.
 * The candidate ranks are r_step, 2 r_step, ... capped at r_max (<= 64 and
 * <= m); the chosen rank is the first whose correlation of X and Y over the
 * drawn pairs (Pearson, population moments) is >= threshold, else the last
 * candidate.  All candidates use prefixes of the same SVD basis (p->basis_host
 * must be NULL; p->r is ignored; the other fields apply to the final build).
 * *r_out gets the rank; corr_trace (may be NULL) gets one correlation per
 * candidate tried, ceil(r_max / r_step) entries at most.  Synchronous. */
finger_status finger_select_rank(finger_index* ix, const finger_build_params* p,
                                 double threshold, int r_step, int r_max, int* r_out,
                                 double* corr_trace, void* stream);

/* Copy FINGER tables to host buffers (any may be NULL):
 *   P r x m, stats[5] as above, node_proj n x r (P c), edge_u (n*deg0) x r,
 *   edge_s (n*deg0) x 2 {||d_res||, b} (zeros for -1 slots). */
finger_status finger_get_tables(const finger_index* ix, float* P, double* stats, float* node_proj,
                                float* edge_u, float* edge_s);

/* Bytes of the per-edge FINGER tables for n nodes, layer-0 degree deg0 and
 * rank r: (r + 2) * n * deg0 * 4 for FP32 (Supplementary F); for the LP
 * tables FP8 codes of 32 (deg0 <= 32) or 64 slots x 32 (r <= 32) or 64 codes
 * per node, plus 8 bytes of scalars per edge slot. */
int64_t finger_table_bytes(int64_t n, int deg0, int r, int lp);

/* -------------------------------------------------------------- search */

/* Set the search mode (FINGER_MODE_*) and the warm-up: the first `warmup`
 * layer-0 expansions of every query use exact distances only (Algorithm 4
 * starts skipping after five updates of cur; default 5).  warmup < 0 leaves it unchanged. */
finger_status finger_set_mode(finger_index* ix, int mode, int warmup);

/* Greedy search for nq queries (device, nq x m row-major FP32): descent with
 * ef = 1 through levels maxlevel..1, then Algorithm 1 (PLAIN) or Algorithm 4
 * (FINGER modes) on layer 0 with a result list of ef entries.  Writes the K
 * best (ascending (distance, id)) to out_ids (device, nq x K int64) and
 * out_dists (device, nq x K float); rows with fewer than K results are padded
 * with id -1 and distance +inf.  1 <= K <= ef <= 1024.  Asynchronous. */
finger_status finger_search(finger_index* ix, const float* queries, int64_t nq, int K, int ef,
                            int64_t* out_ids, float* out_dists, void* stream);

/* finger_search on HOST buffers: copies the queries in, searches, copies the
 * results out and synchronises `stream` before returning. */
finger_status finger_search_host(finger_index* ix, const float* queries_host, int64_t nq, int K,
                                 int ef, int64_t* out_ids_host, float* out_dists_host,
                                 void* stream);

/* finger_search without any device-memory allocation during the call.  The
 * paper has no counterpart; this exists for callers that must not allocate on
 * the query path (processes that reserve their device-memory budget at
 * start-up, loops where cudaMalloc/cudaFree latency or synchronisation is not
 * acceptable).  Same arguments, modes and results as finger_search; the
 * visited-set scratch comes from one fixed 64 MiB device array that the
 * library reserves on every device that loads it, shared by all calls: calls
 * whose kernels overlap on the GPU race on it and must be serialised.  The
 * first call on a device looks up the array's device address and caches it;
 * make that first call before any stream capture.  A launch uses as many
 * resident warps as the array holds (ceil(n/32) bitmap words + the same spill
 * list as finger_search, min(max(n, 64), 65536) ids, per warp: about 176
 * warps at n = 1M, so large batches run on fewer warps than finger_search);
 * if not even one fits (n above roughly 5e8) the call returns
 * FINGER_ERR_UNSUPPORTED.  Asynchronous on `stream`. */
finger_status finger_search_noalloc(finger_index* ix, const float* queries, int64_t nq, int K,
                                    int ef, int64_t* out_ids, float* out_dists, void* stream);

/* Uneven batch: per-query K[i] and ef[i] (device int32 arrays, K[i] <= ef[i]),
 * results of query i at out_ids[out_off[i] .. out_off[i] + K[i]) (device
 * int64 offsets).  One persistent launch sized for max ef; replayed from a
 * captured CUDA graph when the (nq, max ef) shape was seen before.
 * max_ef must bound every ef[i] (the host does not read the device arrays). */
finger_status finger_search_batch(finger_index* ix, const float* queries, int64_t nq,
                                  const int32_t* K, const int32_t* ef, int max_ef,
                                  const int64_t* out_off, int64_t* out_ids, float* out_dists,
                                  void* stream);

/* Autotuner: times the candidate launch shapes (warps per block x visited-hash
 * size x the kernel's register variant: the one with the most resident warps
 * that shared memory admits and each one with fewer that the mode has x the
 * exact-row shape: the default lanes per row, or rows on all 32 lanes, with
 * fewer rows in flight per warp) on a sample batch (device queries, nq x m,
 * uniform K and ef; scratch outputs of nq x K) in the current mode, and keeps
 * the fastest for that mode and the
 * power-of-two ef bucket of `ef` (16, 32, ..., 1024).  finger_search,
 * finger_search_host and finger_search_batch then launch with it at any ef of
 * that bucket where it fits (a batch plans for the bucket's largest ef), else
 * with the default shape.  The best time in milliseconds is written to
 * *best_ms when it is not NULL. */
finger_status finger_autotune(finger_index* ix, const float* queries, int64_t nq, int K, int ef,
                              int64_t* scratch_ids, float* scratch_dists, float* best_ms,
                              void* stream);

/* The autotuner's pick for the current mode and the ef bucket of `ef` (any
 * pointer may be NULL): warps per block, visited-hash slots, resident warps
 * per SM, exact rows in flight per warp (the staging depth of the row
 * gathers) and the best sample-batch time in milliseconds.
 * FINGER_ERR_NOT_BUILT when that bucket was not tuned in this mode (it then
 * uses the default plan). */
finger_status finger_get_tuned(const finger_index* ix, int ef, int* warps_per_block,
                               int* hash_slots, int* resident_warps, int* rows_per_warp,
                               float* best_ms);

/* Cap on the layer-0 expansions (and upper-layer steps) of one query; a query
 * that reaches it stops, keeps its results so far and latches
 * FINGER_ERR_LIMIT.  0 restores the default (n + 16). */
finger_status finger_set_limit(finger_index* ix, int max_expansions);

/* Slot width of the per-query visited set (an exact hash in shared memory
 * that spills to a per-query bitmap in global memory).  0 (default): 16-bit
 * slots whenever the ids fit (n <= 4096 x the table's slot count) and the
 * buffers that reuse the table fit its half size, which halves the table and
 * lets more queries reside per SM; 32: always 32-bit slots.  Results are
 * identical either way.
 * Any other value returns FINGER_ERR_INVALID_ARG. */
finger_status finger_set_visited_slots(finger_index* ix, int bits);

/* Per-query traversal counters of the last search (device int32, nq x 8:
 * expansions, examined, estimates, skipped, exact, admitted, upper, gathered)
 * are written when `counters` is set here (NULL disables). */
finger_status finger_set_counters(finger_index* ix, int32_t* counters_device);

/* ------------------------------------ learned angle predictor (extension)
 * The paper matches the low-rank cosine's distribution to the true one
 * (Sec. 3.3).  This extension replaces that step by a small MLP trained on
 * (q, c, d) triples harvested from FINGER's own traversals: inputs are the
 * r + 4 features [u_q * u_d (r values), t_hat, ||q_res||/||q||,
 * ||d_res||/||d||, a/(|a|+|b|+1e-6)] (u = unit P-projected residuals,
 * a = c^T q / c^T c, b = c^T d / c^T c), target cos(q_res, d_res); network
 * r+4 -> 64 -> 64 -> 1 with ReLU, BF16 weights, FP32 accumulation, the inputs
 * of both hidden layers rounded to BF16.  Flat FP32 weight order: W1 (64 x
 * (r+4), row = hidden unit), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3.
 * In FINGER_MODE_FINGER_MLP the estimate uses t = prediction + eps', eps' the
 * mean absolute error on held-out triples; a non-finite prediction falls back
 * to the distribution-matched t. */

/* number of floats of the flat predictor for rank r (64 (r+4) + 64 + 4096 + 64 + 64 + 1) */
int64_t finger_mlp_size(int r);

/* Run FINGER searches (mode FINGER semantics, warm-up as set) over nq device
 * queries with the given ef and record, for every estimate made while the
 * result list is full, the features (cap x (r+4) FP32, device), the target
 * cos(q_res, d_res) computed from the exact distance (cap FP32, device) and the
 * triple (query index, centre id, neighbour id) (cap x 3 int32, device).
 * *count (host) receives the number of records written (<= cap). Synchronous. */
finger_status finger_harvest(finger_index* ix, const float* queries, int64_t nq, int ef,
                             int64_t cap, float* feat, float* target, int32_t* triples,
                             int64_t* count, void* stream);

typedef struct {
    const float* feat;     /* device, (n_train + n_val) x (r + 4) */
    const float* target;   /* device, n_train + n_val */
    int64_t n_train;       /* first n_train rows train, the next n_val give eps' */
    int64_t n_val;
    int epochs;
    int batch;             /* rows per Adam step */
    float lr;
    uint64_t seed;         /* weight initialisation and shuffling */
} finger_train_params;

/* Train the predictor on the device (hand-written forward, backward and Adam
 * kernels; MSE loss) and install it in the index.  losses (host, may be NULL)
 * receives the mean training loss of each epoch.  Synchronous. */
finger_status finger_train_predictor(finger_index* ix, const finger_train_params* p,
                                     float* losses, void* stream);

/* Install / read a predictor as flat FP32 weights (host) with its eps'. */
finger_status finger_set_predictor(finger_index* ix, const float* weights, int64_t count,
                                   float eps);
finger_status finger_get_predictor(const finger_index* ix, float* weights, float* eps);

/* Where the predictor runs in FINGER_MODE_FINGER_MLP.  delta < 0 (default):
 * on every estimate.  delta >= 0: only for a neighbour whose distribution-
 * matched estimate (Algorithm 3) lies within delta * ub of the upper bound ub
 * at the start of its centre's expansion (and only while the result list is
 * full then); elsewhere the matched estimate stands.  The network's cost is
 * then paid where its better cosine can change the gate.  NaN returns
 * FINGER_ERR_INVALID_ARG. */
finger_status finger_set_predictor_gate(finger_index* ix, float delta);

/* Mean squared error and its gradient (host, finger_mlp_size floats) of the
 * predictor with the given flat weights (host, nf = r + 4 inputs) on n device
 * rows, computed by the training kernels (gradient checks). Synchronous. */
finger_status finger_mlp_loss_grad(finger_index* ix, int nf, const float* weights,
                                   const float* feat, const float* target, int64_t n, float* grad,
                                   double* loss, void* stream);

/* Predictions of the installed predictor for n device feature rows. */
finger_status finger_mlp_predict(finger_index* ix, const float* feat, int64_t n, float* out,
                                 void* stream);

/* ------------------------------------------------------- ground truth */

/* Exact K nearest neighbours of nq queries (device, nq x m) over all n base
 * rows by brute force on the GPU; ascending (distance, id), distances summed
 * as (q - x)^2 in FP32.  K <= 256.  For K <= 40 the distance matrix runs on
 * the tensor cores (q.x from BF16 high/low split products accumulated in FP32
 * in tensor memory, candidate lists of 32 or 64 per row, then an exact FP32
 * re-rank); larger K use FP32 FFMA tiles.  Asynchronous (stream-ordered
 * temporaries; the first tensor-core call caches a BF16 split of the base rows,
 * 4 bytes per element). */
finger_status finger_knn(finger_index* ix, const float* queries, int64_t nq, int K,
                         int64_t* out_ids, float* out_dists, void* stream);

/* ------------------------------------------- partitioned-database search
 * A database split into S disjoint parts, each with its own index (graph and
 * FINGER tables), is searched part by part (on one or several GPUs); the
 * answer for a query is the K smallest (distance, id) keys of the union of
 * the parts' K nearest (the kNN problem of Sec. 1 over the union).  This
 * merge is the exchange step of that search.
 *
 * ids, dists: device, S x nq x K (part-major), each part's rows as returned by
 *   finger_search on that part: ascending, ids local to the part, -1 / +inf
 *   padded.
 * id_offsets: host, S values >= 0 added to a part's ids (its first global id).
 * out_ids, out_dists: device, nq x K, ascending by (distance, global id),
 *   -1 / +inf padded when the parts hold fewer than K results in total.
 * 1 <= S <= 64, 1 <= K <= 1024, otherwise FINGER_ERR_INVALID_ARG (also for a
 * NULL pointer with nq > 0 or a negative offset).  Runs on the calling
 * thread's current device, asynchronously on `stream`; the caller owns every
 * buffer. */
finger_status finger_merge_topk(const int64_t* ids, const float* dists, int shards, int64_t nq,
                                int K, const int64_t* id_offsets, int64_t* out_ids,
                                float* out_dists, void* stream);

/* --------------------------------------------------- status and stats */

typedef struct {
    int64_t searches;       /* queries searched since the last reset */
    int64_t counters[8];    /* summed traversal counters (order as above) */
    int32_t device_error;   /* latched FINGER_ERR_* from kernels, 0 if none */
    double mu, sigma, mu_hat, sigma_hat, eps; /* matching statistics */
    double build_ms;        /* wall time of the last table build */
    double corr;            /* correlation of X and Y over the drawn pairs
                               (Supplementary E), NaN before a build */
    int64_t code_bytes;     /* bytes of code blocks read by the FINGER_F16, FINGER_F8
                               and LP searches (a block's second half only for
                               centres whose degree needs it) */
} finger_stats;

/* Synchronise the index's device and return the latched kernel status. */
finger_status finger_sync(finger_index* ix);

/* Synchronise and copy the summed traversal counters and the latched status
 * into *out (caller-owned).  The counters are the quantities the paper
 * measures the method by: "exact" plus "upper" are the full m-dimensional
 * distance calls and "estimates" the r-dimensional ones, which combine into
 * Sec. 4.3's effective number of distance calls (full + estimates * r / m);
 * "skipped" counts the estimates that exceeded the upper bound, the calls
 * Sec. 3.1 observes to be the large majority after the first steps. */
finger_status finger_get_stats(finger_index* ix, finger_stats* out);
finger_status finger_reset_stats(finger_index* ix);
const char* finger_status_str(finger_status s);

#ifdef __cplusplus
}
#endif
#endif /* FINGER_H */
