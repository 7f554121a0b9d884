/* aqr.h — C ABI of the GB300 (sm_103a) AQR-HNSW query library, libaqr.so.
 *
 * The library runs the query path of AQR-HNSW (density-aware 8-bit
 * quantisation plus multi-stage re-ranking on an HNSW graph) on one GPU:
 *   1. quantise the query                 (Section 3.2; Alg. 2; Section 3.3)
 *   2. greedy descent through layers L..1 (Section 2; HNSW search, ef = 1)
 *   3. beam search on layer 0 over uint8 codes, ef-bounded
 *                                          (Section 3.2 Stage 1; Alg. 2)
 *   4. asymmetric distances to decoded candidates, sort, early termination
 *                                          (Section 3.2 Stage 2; Alg. 2)
 *   5. exact FP32 distances on the shortlist, merge, top-k
 *                                          (Section 3.2 Stage 3; Alg. 2)
 * plus the build-phase pieces the query path needs (Section 3.1, Alg. 1):
 * base encode, quantiser training, graph construction on codes, and an
 * exact brute-force kNN.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an aqr_status; none aborts, traps or exits.
 *    On failure aqr_last_error(ctx) holds a one-line message (per context,
 *    valid until the next call on that context from the same thread).
 *  - "_dev" pointers are device pointers on the context's device; "_host"
 *    pointers are host memory.  The caller owns every buffer it passes; the
 *    library owns the index and its own working memory.
 *  - stream arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream).  Functions that take a stream only enqueue work;
 *    the caller synchronises.  Functions without a stream are synchronous.
 *  - Distances are squared L2: the asymmetric and exact distances of Alg. 2
 *    carry no square root.
 *  - Row-major layouts; leading dimensions are in elements.
 *  - A context is not thread-safe except for the serving calls
 *    (aqr_submit / aqr_poll / aqr_cancel), which may be called from any thread
 *    but not concurrently with aqr_serve_stop or aqr_destroy.  While serving,
 *    the index cannot be replaced (AQR_ERR_BUSY); search parameters and
 *    kernel configurations may change and apply to later micro-batches.
 */
#ifndef AQR_H_
#define AQR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum aqr_status {
    AQR_OK = 0,
    AQR_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
    AQR_ERR_NO_MEMORY = 2,   /* device or host allocation failed / admission refused */
    AQR_ERR_NO_INDEX = 3,    /* the call needs an index and none is loaded */
    AQR_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error) */
    AQR_ERR_TIMEOUT = 5,     /* a bounded wait ran out */
    AQR_ERR_BAD_FILE = 6,    /* index file missing, truncated, wrong magic or checksum */
    AQR_ERR_BUSY = 7,        /* serving queue full / serving not started */
    AQR_ERR_NOT_READY = 8,   /* a submitted request has not completed yet */
    AQR_ERR_INTERNAL = 9     /* a device-side consistency check failed */
} aqr_status;

typedef struct aqr_ctx aqr_ctx;

/* Search parameters (Section 3.2; defaults = Table 3, row "0.97+"):
 *   m_ef        ef multiplier: N_c = ceil(ef_eff / m_ef) when n_coarse = 0   (default 3)
 *   rerank_pct  N_rerank = ceil(N_c * rerank_pct / 100) when n_rerank = 0  (default 40,
 *               Table 3's 28 of 70)
 *   n_coarse    explicit N_c (0 = derive); clamped to [k, ef_eff]
 *   n_rerank    explicit N_rerank (0 = derive); clamped to [k, N_c]
 *   tau_gap     early-termination gap threshold   (default 0.010)
 *   tau_ratio   early-termination ratio threshold (default 1.008)
 *   eps         denominator guard of gap and ratio (default 1e-6)
 * ef_eff = max(ef, k) bounds the layer-0 result set. */
typedef struct aqr_search_params {
    int32_t m_ef;
    int32_t rerank_pct;
    int32_t n_coarse;
    int32_t n_rerank;
    float tau_gap;
    float tau_ratio;
    float eps;
} aqr_search_params;

/* Kernel configuration of the batched query kernel for one ef class
 * (max(ef, k) <= 64, 128, 256, 512, 1024).  Every field: 0 = automatic.
 * No field changes results, only speed and shared memory.
 *   hash_slots     ids the per-query visited hash holds in shared memory
 *                  (64..16384; with 16-bit tags rounded down to a power of
 *                  two, with 32-bit ids up to a multiple of 64; raised to
 *                  cover the FP32 query and to at least 32 sets)
 *   tile_rows      neighbour tile: candidate rows gathered into shared
 *                  memory per round of Stage 1 (1..32)
 *   team_lanes     lanes per candidate distance in Stage 1: 1 = one lane per
 *                  candidate (code rows <= 256 bytes), 2 = the team width of
 *                  the row size
 *   hash_tag_bits  visited-hash entries: 16 = 16-bit quotient tags, four
 *                  per 8-byte set (2 bytes per id; sets are added when the
 *                  index has too many ids for 15-bit tags), 32 = whole ids,
 *                  two per set (4 bytes per id); 0 = 16-bit tags when the
 *                  requested size gives them at most 15 bits, else 32
 *   warps_per_block block shape of the one-lane-per-candidate kernel: 4 =
 *                  blocks of 4 warps (up to 8 per SM, 64 registers); 11 =
 *                  blocks of 11 warps limited to 56 registers, three per SM
 *                  (33 resident queries per SM, for batches that then need
 *                  one round of queries per warp fewer); the neighbour tile
 *                  defaults to the largest that lets three blocks fit.
 *                  Other kernels always run blocks of 4 warps.
 *   warps_per_query warps that search one query together (1, 2 or 4): the
 *                  query's result set and visited hash are shared by the
 *                  group, each warp filters, gathers and evaluates its part
 *                  of every expanded neighbour list, one warp merges; the
 *                  same expansions and results as one warp, lower latency
 *                  per query.  0 = automatic: groups (4 warps for code rows
 *                  over 256 bytes, else 2) when the launch has at most one
 *                  query per SM, one warp otherwise.  Such a small launch
 *                  also takes a visited hash of 32 ids per result-set entry
 *                  (4,096 to 16,384) when hash_slots is automatic. */
typedef struct aqr_kernel_config {
    int32_t hash_slots;
    int32_t tile_rows;
    int32_t team_lanes;
    int32_t hash_tag_bits;
    int32_t warps_per_block;
    int32_t warps_per_query;
} aqr_kernel_config;

/* Shape of the loaded index. */
typedef struct aqr_index_info {
    int64_t n;          /* base vectors */
    int32_t d;          /* dimensions */
    int32_t d_pad;      /* bytes per code row on the device (d rounded up to 16) */
    int32_t M_i;        /* adaptive connectivity (Alg. 1) */
    int32_t R0;         /* layer-0 list capacity = 2 M_i */
    int32_t R1;         /* upper-layer list capacity = M_i */
    int32_t ef_c;       /* construction beam width (Alg. 1) */
    int32_t max_level;  /* top layer of the graph */
    uint32_t entry;     /* entry point (first node reaching max_level) */
    int64_t n_upper;    /* number of upper-layer rows */
    double s_dist;      /* distance scale (Eq. 1) */
    int64_t device_bytes; /* device memory held by the index */
} aqr_index_info;

/* Counters of the last search call on the context (sums over its queries).
 * Bytes are the algorithmic bytes each stage must read: adjacency entries of
 * expanded nodes (4 B per listed neighbour), d code bytes per distance
 * evaluation, d code bytes per Stage-2 candidate, 4d bytes per exact
 * distance, the FP32 query (4d) and the k results (12 B each). */
typedef struct aqr_stats {
    int64_t queries;
    int64_t expansions;      /* layer-0 and upper-layer node expansions */
    int64_t dist_evals;      /* quantised distance evaluations (all layers) */
    int64_t adj_entries;     /* neighbour ids read */
    int64_t stage2_evals;    /* asymmetric distances (|C| per query) */
    int64_t exact_evals;     /* exact FP32 distances (n_exact per query) */
    int64_t early_exits;     /* queries that took the early-termination branch */
    int64_t algo_bytes;      /* algorithmic bytes, formula above (evaluations as counted) */
    int32_t device_errors;   /* non-zero if a device-side bound was hit */
    int64_t l0_evals;        /* layer-0 distance evaluations, hash re-evaluations included */
    int32_t knn_tensor;      /* 1 if the context's last aqr_bruteforce_knn (or the density
                                kNN of aqr_train_quantizer) computed its distances on the
                                tensor cores, 0 on the CUDA cores; read once that call's
                                stream is synchronized */
} aqr_stats;

/* Optional per-query traces of one search (device pointers, each may be
 * NULL).  cap_c must be >= ef_eff of the call when c_* or a_* is set. */
typedef struct aqr_trace {
    uint32_t* l0_entry;  /* [n]            layer-0 entry point after the greedy descent */
    uint32_t* c_ids;     /* [n * cap_c]    Stage-1 candidates C, ascending (dist, id) */
    int32_t* c_dist;     /* [n * cap_c]    their integer code distances (sum of squares) */
    int32_t* c_count;    /* [n]            |C| */
    uint32_t* a_ids;     /* [n * cap_c]    Stage-2 list A, ascending (d^a, id) */
    float* a_dist;       /* [n * cap_c]    asymmetric distances */
    uint8_t* et;         /* [n]            1 if early termination was taken */
    int32_t* n_exact;    /* [n]            number of exact re-ranks */
    uint32_t* exp_seq;   /* [n * cap_exp]  layer-0 expansion order */
    int32_t* exp_count;  /* [n]            layer-0 expansions */
    int32_t cap_c;
    int32_t cap_exp;
} aqr_trace;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  Allocates a few KB of device
 * counters.  *out is NULL on failure. */
aqr_status aqr_create(aqr_ctx** out, int32_t device);
/* Release the context, its index and all its device memory (NULL is a no-op). */
aqr_status aqr_destroy(aqr_ctx* ctx);
/* Static text for a status code. */
const char* aqr_status_string(aqr_status s);
/* Last error message of the context ("" if none). */
const char* aqr_last_error(aqr_ctx* ctx);
/* Default search parameters (Table 3, row "0.97+"). */
aqr_status aqr_default_search_params(aqr_search_params* out);
/* Recommended parameters for a target recall (Table 3, Section 4.4).  The
 * table's bands 0.85-0.90, 0.90-0.95, 0.95-0.97 and 0.97+ are taken as
 * target < 0.90, < 0.95, < 0.97 and >= 0.97 (0 < target_recall <= 1, else
 * AQR_ERR_INVALID_ARG).  *out: n_coarse = the row's coarse candidates,
 * n_rerank = its rerank K, tau_gap, tau_ratio, m_ef = its EF multiplier,
 * other fields at their defaults.  *ef_out (may be NULL): the layer-0 search
 * depth ef = N_c * m_ef of Section 3.2, Stage 1.  Host-only; no context. */
aqr_status aqr_search_params_for_recall(double target_recall, aqr_search_params* out,
                                        int32_t* ef_out);
/* Set the context's search parameters (validated: m_ef >= 1, 0 <= rerank_pct
 * <= 100, n_coarse/n_rerank >= 0, eps > 0). */
aqr_status aqr_set_search_params(aqr_ctx* ctx, const aqr_search_params* p);

/* ---- quantiser ---------------------------------------------------------- */

/* Encode n vectors (Alg. 1, Alg. 2, Section 3.3):
 * code = round-half-even(clip((x - min_j) * scale_j, 0, 255)), computed in
 * IEEE FP32 as a subtract then a multiply (no fused multiply-add); NaN
 * encodes to 0.  x_dev [n, ldx] float32; min_dev, scale_dev [d] float32;
 * codes_dev [n, ldc] uint8, bytes d..ldc-1 of each row are written as 0.
 * Requires ldx >= d, ldc >= d.  Async on stream.  n = 0 is a no-op. */
aqr_status aqr_quantize(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d, int64_t ldx,
                        const float* min_dev, const float* scale_dev, uint8_t* codes_dev,
                        int64_t ldc, void* stream);

/* Train the quantiser and graph parameters (Section 3.1; Alg. 1):
 * density rho_i = 1/(mean squared L2 to the 10 nearest other points + 1e-6)
 * (computed on the GPU for every point when n <= 10,000, else for the given
 * sample of n_s ids, the others taking the sample mean); delta; P_l =
 * delta * p_max, P_h = 1 - delta * p_max; per-dimension type-7 percentiles
 * min_j, max_j; scale_j = 255 / (max_j - min_j + 1e-6); w, s_dist (Eq. 1),
 * eta; M_i = floor(M0 (1 + delta (1 + eta))); ef_c = floor(ef0 / (1 + delta eta)).
 * x_dev [n, d] float32 (dense rows).  sample_host [n_s] int64 ids (may be
 * NULL when n <= 10,000).  Outputs (host): min, max, scale [d]; scalars[11] =
 * {delta, rho_bar, w, s_dist, eta, M_i, ef_c, P_l, P_h, rho_min, rho_max}.
 * The percentile step copies x to the host once.  Synchronous. */
aqr_status aqr_train_quantizer(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d,
                               const int64_t* sample_host, int64_t n_s, double p_max, int32_t M0,
                               int32_t ef0, float* min_host, float* max_host, float* scale_host,
                               double* scalars_host);

/* ---- index -------------------------------------------------------------- */

/* Load an index file (format "AQRIDX01": 80-byte header, min[d], scale[d],
 * codes[n*d], x[n*d], adj0[n*R0], upper_base[n] int64, upper[rows*R1],
 * FNV-1a-64 checksum) into device memory owned by the context, replacing any
 * index it holds.  AQR_ERR_BAD_FILE on a missing/short file, bad magic,
 * version, sizes or checksum, ids out of range, a row that names a node
 * twice, or an upper-layer structure the search cannot walk (upper rows not
 * in id order, a listed node below the row's layer, an entry point off the
 * top level).  Synchronous. */
aqr_status aqr_load_graph(aqr_ctx* ctx, const char* path);

/* Build an index on the GPU (Alg. 1): encode x with
 * (min, scale), draw levels l = floor(-ln(U_i) / ln(M_i)), and insert the
 * nodes in id order in batches (node 0 alone, then b = min(max(1, s /
 * batch_div), batch_max) nodes starting at node s).  Every node of a batch
 * searches the graph as it stood before the batch with ef_c, selects at most
 * M_i neighbours per layer with the HNSW heuristic, and the batch's reverse
 * links are then applied per target in ascending source id (append, or
 * re-select the full list with the same heuristic when it is full; layer-0
 * capacity 2 M_i, upper capacity M_i).
 * x_dev [n, d] float32 (copied into the index), min/scale/U on the host.
 * Synchronous; replaces any index the context holds. */
aqr_status aqr_build_graph(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d,
                           const float* min_host, const float* scale_host, const double* U_host,
                           int32_t M_i, int32_t ef_c, int32_t batch_div, int32_t batch_max,
                           double s_dist);

/* Describe the loaded index. */
aqr_status aqr_index_info_get(aqr_ctx* ctx, aqr_index_info* out);

/* Copy the loaded graph to host arrays: adj0_host [n * R0] (0xFFFFFFFF in
 * unused slots), upper_base_host [n] (-1 for level-0 nodes), upper_host
 * [n_upper * R1], codes_host [n * d] (may be NULL), entry_level_host[2] =
 * {entry, max_level}.  Synchronous. */
aqr_status aqr_export_graph(aqr_ctx* ctx, uint32_t* adj0_host, int64_t* upper_base_host,
                            uint32_t* upper_host, uint8_t* codes_host, int32_t* entry_level_host);

/* ---- search ------------------------------------------------------------- */

/* Batched query (Alg. 2) for n queries with one k and one ef:
 * queries_dev [n, d] float32 (dense rows); ids_dev [n, k] int64 and
 * dists_dev [n, k] float32 receive the top-k ascending by (distance, id);
 * entries past the candidates found are id -1, distance +inf.  Returned
 * distances are exact FP32 squared L2 for re-ranked ids and asymmetric
 * distances for the rest (Alg. 2).  1 <= k <= ef_eff <= 1024.
 * Async on stream; n = 0 is a no-op.  Up to 16 searches of one context may
 * be in flight at once on different streams (each launch has its own work
 * counter); aqr_get_stats describes the last call only when calls do not
 * overlap. */
aqr_status aqr_search(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k, int32_t ef,
                      int64_t* ids_dev, float* dists_dev, void* stream);

/* aqr_search plus optional outputs: exact_dev [n, k] uint8 (1 where the
 * distance is exact; may be NULL) and per-query traces (may be NULL). */
aqr_status aqr_search_trace(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k,
                            int32_t ef, int64_t* ids_dev, float* dists_dev, uint8_t* exact_dev,
                            const aqr_trace* trace, void* stream);

/* Mixed batch: per-query k_host[i] and ef_host[i] (host arrays).  Queries
 * are grouped by ef class (<=64, <=128, <=256, <=512, <=1024), each class
 * runs as one persistent launch, and the classes run concurrently; the whole
 * call is captured once into a CUDA graph per (n, class mix) and replayed.
 * ids_dev / dists_dev are [n, k_stride] with k_stride >= max k; columns past
 * a query's k are written as -1 / +inf.  Async on stream. */
aqr_status aqr_search_mixed(aqr_ctx* ctx, const float* queries_dev, int64_t n,
                            const int32_t* k_host, const int32_t* ef_host, int32_t k_stride,
                            int64_t* ids_dev, float* dists_dev, void* stream);

/* End-to-end call on host buffers: copies queries_host [n, d] to the device,
 * runs aqr_search, copies ids_host [n, k] / dists_host [n, k] back.  Uses
 * context-owned device buffers (grown on demand).  Synchronous. */
aqr_status aqr_search_host(aqr_ctx* ctx, const float* queries_host, int64_t n, int32_t k,
                           int32_t ef, int64_t* ids_host, float* dists_host);

/* The plain comparison path on the same graph: FP32 distances on the FP32
 * vectors throughout (no codes, no re-rank), layer-0 beam ef_eff = max(ef, k),
 * top-k of the result set.  Same layouts as aqr_search.  Async on stream. */
aqr_status aqr_search_plain_f32(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k,
                                int32_t ef, int64_t* ids_dev, float* dists_dev, void* stream);

/* Set the kernel configuration used for queries of the ef class of
 * max(ef, k) (ranges in aqr_kernel_config; 0 fields = automatic). */
aqr_status aqr_set_kernel_config(aqr_ctx* ctx, int32_t ef, int32_t k, const aqr_kernel_config* cfg);

/* Autotuner: times the candidate kernel configurations (hash size, tile
 * width, lanes per candidate, block shape, warps per query) on the given
 * resident batch (queries_dev
 * [n, d]), keeps the fastest for the ef class of max(ef, k) and returns it
 * in *chosen.  Results do not depend on the configuration, only speed does.
 * Synchronous; allocates its own temporary output buffers. */
aqr_status aqr_autotune(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k, int32_t ef,
                        aqr_kernel_config* chosen);

/* Result of aqr_autotune_recall: the chosen shortlist policy (params: the
 * context's thresholds with m_ef and rerank_pct of the winner, N_c and
 * N_rerank derived), search depth ef, kernel configuration, the sample's
 * recall@k there, the time of one search of the sample (ms, CUDA events on
 * the context's stream, no cache flush), and reached = 1 if that recall is
 * at least the target (0: no setting reached it; the best recall found). */
typedef struct aqr_tune_result {
    aqr_search_params params;
    int32_t ef;
    aqr_kernel_config kernel;
    double recall;
    double ms;
    int32_t reached;
} aqr_tune_result;

/* Autotuner of the shortlist and the search depth for a target recall (no
 * counterpart in the paper, whose Section 4.4 / Table 3 sets them by hand).
 * For each shortlist policy -- m_ef in {3, 2, 1}, each with N_rerank = 40%
 * of N_c (Table 3's rerank / coarse ratio) or all of N_c (Section 3.2) --
 * the smallest ef of ef_list_host whose recall@k on the sample reaches
 * target_recall; for each such candidate the fastest kernel configuration
 * (as aqr_autotune); the fastest candidate wins.
 *   queries_dev [n, d] float32 (device): the sample queries;
 *   gt_ids_host [n, gt_stride] int64 (host): their true neighbours, the
 *     first k of each row the k nearest (ties in any order);
 *   ef_list_host [n_ef] strictly ascending, each a valid ef with k;
 *   out: the winner; sweep_recall_host (optional, [6, n_ef]): the recall of
 *     every policy (in the order above) and ef measured, -1 where not.
 * 1 <= k <= gt_stride, 0 < target_recall <= 1, else AQR_ERR_INVALID_ARG.
 * Leaves the context's search parameters and the kernel configuration of
 * the winner's ef class set to the winner.  Synchronous; allocates
 * temporaries. */
aqr_status aqr_autotune_recall(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k,
                               const int64_t* gt_ids_host, int32_t gt_stride,
                               double target_recall, const int32_t* ef_list_host, int32_t n_ef,
                               aqr_tune_result* out, double* sweep_recall_host);

/* Counters of the last search on the context.  Synchronises the context's
 * last search stream, which must still exist (not destroyed since). */
aqr_status aqr_get_stats(aqr_ctx* ctx, aqr_stats* out);

/* Exact k nearest neighbours by FP32 squared L2 (ties by id) of q_dev [nq, d]
 * among base_dev [n, d].  self_ids_dev (optional, [nq] int64) names the base
 * row to skip for each query.  ids_dev [nq, k] int64, dists_dev [nq, k]
 * float32 (padded with -1 / +inf when n is smaller than k).  1 <= k <= 128.
 * Allocates its per-split partial lists (stream-ordered).  Async on stream.
 * When every value of both sets is an integer of magnitude <= 256, the sum
 * of the largest query and base squared norms is below 2^24, d <= 256 and
 * the kernel's per-query lists fit shared memory (k <= 32 for d <= 128, k <= 8
 * for d = 256), the distances come from tensor-core MMAs (BF16 operands, FP32
 * accumulation), which are then exact and equal to the CUDA-core kernel's
 * bit for bit (the test runs on the device; no host sync). */
aqr_status aqr_bruteforce_knn(aqr_ctx* ctx, const float* base_dev, int64_t n, int32_t d,
                              const float* q_dev, int64_t nq, int32_t k,
                              const int64_t* self_ids_dev, int64_t* ids_dev, float* dists_dev,
                              void* stream);

/* aqr_bruteforce_knn without any allocation.  No counterpart in the paper:
 * this is a service of the library for callers that cannot allocate device
 * memory during the call -- callers whose device memory belongs to another
 * allocator (a framework's caching pool, an arena sized once at start-up) or
 * that run under a fixed device-memory budget, where a transient allocation
 * inside a library call can fail or fragment the pool.  The caller passes
 * inputs and outputs exactly as for aqr_bruteforce_knn (same layouts, the
 * current CUDA device, no context, 1 <= k <= 128).  The working memory is a
 * file-scope device array of 16 MiB that every GPU which loads the library
 * holds until the process exits; nq * k must be <= 2,097,152
 * (AQR_ERR_INVALID_ARG otherwise, nothing launched).  When the usual number
 * of base-set splits would not fit the array, fewer splits are used (same
 * results, less parallelism).  The first call on a device looks up the
 * array's device address for that device (set-up, once per device); make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents (nothing in it needs to start at zero):
 * calls that overlap on the GPU -- on different streams, or from different
 * threads -- race on it and must be serialised by the caller.  Async on
 * stream. */
aqr_status aqr_bruteforce_knn_static(const float* base_dev, int64_t n, int32_t d,
                                     const float* q_dev, int64_t nq, int32_t k,
                                     const int64_t* self_ids_dev, int64_t* ids_dev,
                                     float* dists_dev, void* stream);

/* ---- database sharding ------------------------------------------------ */

/* Merge per-shard result lists (no counterpart in the paper: the base set is
 * split into S shards, each searched on its own graph by aqr_search, and the
 * lists are merged with Alg. 2's final ranking: ascending distance, ties by
 * id, over the union of the shards' results).
 *   dists_dev [S, n, k] float32, ids_dev [S, n, k] int64 (device; shard s's
 *     n x k result block at offset s * n * k, each row sorted by (distance,
 *     id) with padding id -1 at its end, as aqr_search writes it);
 *   id_offsets_host [S] (may be NULL = all 0): added to shard s's ids, so
 *     that the output holds global ids;
 *   ids_out_dev [n, k] int64, dists_out_dev [n, k] float32: the k smallest
 *     (distance, global id) pairs of the S lists, padded with id -1 and +inf
 *     when the lists hold fewer than k.
 * 1 <= S <= 32, 1 <= k <= 1024, offsets >= 0, else AQR_ERR_INVALID_ARG.
 * Allocates nothing; asynchronous on stream. */
aqr_status aqr_merge_topk(aqr_ctx* ctx, const float* dists_dev, const int64_t* ids_dev,
                          int32_t S, int64_t n, int32_t k, const int64_t* id_offsets_host,
                          int64_t* ids_out_dev, float* dists_out_dev, void* stream);

/* ---- serving (continuous batching) ------------------------------------- */

/* Serving configuration:
 *   max_batch     queries per micro-batch launch (>= 1)
 *   n_streams     concurrent micro-batches in flight on separate streams (1..16)
 *   hbm_budget    device bytes the request slots may hold (0 = 1/4 of free memory)
 *   max_pending   admitted-but-not-launched request cap (queue bound)
 *   batch_wait_us how long the scheduler waits to fill a micro-batch */
typedef struct aqr_serve_config {
    int32_t max_batch;
    int32_t n_streams;
    int64_t hbm_budget;
    int32_t max_pending;
    int32_t batch_wait_us;
} aqr_serve_config;

/* Per-request timing reported by aqr_poll (microseconds since submit). */
typedef struct aqr_request_stats {
    double queue_us;    /* submit -> launch */
    double latency_us;  /* submit -> results on the host */
    int32_t batch_size; /* queries in the micro-batch that carried it */
} aqr_request_stats;

/* Start the serving scheduler thread on the loaded index.  While micro-batches
 * are on the GPU the thread polls their completion every few microseconds
 * (its timer slack is lowered to 1 us for that), so a finished request is
 * handed back and a waiting one launched within microseconds; idle, it
 * blocks until a submit. */
aqr_status aqr_serve_start(aqr_ctx* ctx, const aqr_serve_config* cfg);
/* Submit one query (query_host [d] float32, copied) with its own k and ef;
 * *ticket identifies it.  AQR_ERR_BUSY if the pending queue is full,
 * AQR_ERR_NO_MEMORY if its slot can never fit the budget, AQR_ERR_CUDA once
 * the scheduler has stopped on an error (every later submit is refused;
 * aqr_serve_stop then aqr_serve_start begin a new service). */
aqr_status aqr_submit(aqr_ctx* ctx, const float* query_host, int32_t k, int32_t ef,
                      uint64_t* ticket);
/* Poll a ticket: AQR_OK with ids_host [k] / dists_host [k] filled (and
 * st_host if non-NULL), or AQR_ERR_NOT_READY.  A ticket is released after
 * the first AQR_OK.  timeout_us > 0 waits up to that long. */
aqr_status aqr_poll(aqr_ctx* ctx, uint64_t ticket, int64_t* ids_host, float* dists_host,
                    aqr_request_stats* st_host, int64_t timeout_us);
/* Cancel a request that has not been launched yet (AQR_ERR_NOT_READY if it
 * is already on the device). */
aqr_status aqr_cancel(aqr_ctx* ctx, uint64_t ticket);
/* Stop the scheduler after in-flight work completes (bounded wait). */
aqr_status aqr_serve_stop(aqr_ctx* ctx);
/* Test hook for the scheduler's failure path (no counterpart in the paper):
 * the scheduler thread throws a host exception (std::bad_alloc) at its next
 * pass, exactly as when host memory runs out.  The service then refuses
 * submits with AQR_ERR_CUDA, waits for the micro-batches already on the GPU,
 * releases their slots and completes every unfinished request with
 * AQR_ERR_CUDA.  No GPU fault is involved.  AQR_ERR_BUSY if not serving. */
aqr_status aqr_serve_inject_host_fault(aqr_ctx* ctx);
/* Open-loop load generator (no counterpart in the paper; it measures the
 * serving loop).  On the calling thread, request i (queries_host [n, d]
 * float32 row i, k[i] <= k_stride, ef[i]) is submitted once arrival_us[i]
 * (non-decreasing, microseconds from the call) has passed, and finished
 * requests are collected between submissions.  Outputs per request:
 * ids_host / dists_host [n, k_stride] (rows padded with -1 / +inf after
 * k[i]) and stats_host [n] (latency from submit to results on the host).
 * Needs aqr_serve_start; returns when every request has finished, or
 * AQR_ERR_TIMEOUT timeout_us after the last arrival. */
aqr_status aqr_serve_replay(aqr_ctx* ctx, const float* queries_host, int64_t n, const int32_t* k,
                            const int32_t* ef, const double* arrival_us, int32_t k_stride,
                            int64_t* ids_host, float* dists_host, aqr_request_stats* stats_host,
                            int64_t timeout_us);

#ifdef __cplusplus
}
#endif

#endif /* AQR_H_ */
