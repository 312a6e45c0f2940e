/*
 * crisp.h -- C ABI of the GB300 (sm_103a) CRISP engine.
 *
 * CRISP (Correlation-Resilient Indexing via Subspace Partitioning, arXiv
 * 2603.05180) is an approximate-nearest-neighbour index for very high
 * dimensional vectors under squared L2.  This library builds the index on the
 * GPU (§4.1 correlation test and rotation, §4.2 IMI k-means cells and CSR lists)
 * and answers batches of k-NN queries with the dual-mode engine of Algorithm 1
 * (§4.3): per-subspace partial distances, multi-sequence cell traversal,
 * collision counting, threshold cut, and exact re-rank (Guaranteed Mode) or
 * Hamming-ordered ADSampling with patience (Optimized Mode).
 *
 * Conventions for every entry point below:
 *  - Pointers are DEVICE pointers unless the argument says "host".  The caller
 *    owns every buffer it passes; the library owns what it allocates inside a
 *    crisp_index and frees it in crisp_free.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    asynchronous on that stream unless stated; argument errors are reported
 *    before anything is enqueued, and then nothing is written.  Errors raised by
 *    the device surface as CRISP_ECUDA from this or a later call.
 *  - Row-major layouts.  Ids are 0-based row numbers of the indexed matrix X.
 *    Distances are squared L2 (monotone in L2, §3 "Exact and Approximate
 *    Similarity Search").
 *  - On error, crisp_last_error() returns a message for the calling thread.
 *
 * Fixed readings of the paper (the library and its tests agree on them):
 *  - tau = ceil(alpha*M - 1e-9) collisions (Theorem 1, tau = alpha M);
 *    budget = max(1, ceil(rho*N - 1e-9)) ids per subspace (Algorithm 1).
 *  - Subspace m covers dims [floor(mD/M), floor((m+1)D/M)); its left half is
 *    the first floor(d_m/2) of them (§3, IMI halves).
 *  - cell = cL*K + cR with cL, cR the nearest left/right centroid (§3 u(x)).
 *  - Stored rows are padded with zeros to Dp = 32*ceil(D/32) dims.
 *  - FP32 orders.  SEQ: acc = fmaf(a_i - b_i, a_i - b_i, acc) over i in order
 *    (half distances, k-means).  GEMV: y_j = fmaf chain over d of x_d R[d][j]
 *    (rotation).  CR32: per 32-dim block eight fmaf chains over 4 dims each,
 *    block sum ((a0+a4)+(a2+a6))+((a1+a5)+(a3+a7)), blocks summed in order
 *    (re-rank and ADSampling distances; every ADSampling partial d_t is a
 *    prefix of the same sum).
 */
#ifndef CRISP_H
#define CRISP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crisp_index crisp_index; /* opaque; owns its device memory */

typedef enum {
    CRISP_OK = 0,
    CRISP_EINVAL = -1,        /* invalid argument; nothing was enqueued */
    CRISP_ENOMEM = -2,        /* device or host allocation failed */
    CRISP_ECUDA = -3,         /* a CUDA runtime error (message in crisp_last_error) */
    CRISP_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
    CRISP_EUNSUPPORTED = -5   /* a size the kernels do not handle (e.g. K > 64) */
} crisp_status;

/* Index-build parameters (§4.1, §4.2).  The random draws of the build may be
 * given explicitly (host arrays, copied before return); NULL means "draw from
 * `seed`" with the library's own generator. */
typedef struct {
    int32_t M;                 /* subspaces, 1 <= M <= D/2 */
    int32_t K;                 /* centroids per half, 2 <= K <= 64 (paper: 50) */
    double tau_cev;            /* CEV threshold (paper: 0.85); rotate iff CEV > tau_cev */
    int32_t rotate;            /* -1 decide by the CEV test, 0 never, 1 always */
    int32_t kmeans_iters;      /* Lloyd iterations (20) */
    int64_t kmeans_train;      /* training rows when kmeans_sample is NULL (1e5) */
    uint64_t seed;
    const int64_t *cev_sample;    /* host [cev_sample_n] row numbers, or NULL */
    int64_t cev_sample_n;         /* NULL sample: min(floor(0.1N), 1e5), at least 2 */
    const double *gaussian;       /* host [D][D] G_ij ~ N(0,1) (§3 rotation), or NULL */
    const int64_t *kmeans_sample; /* host [kmeans_sample_n] row numbers, or NULL */
    int64_t kmeans_sample_n;
    const int32_t *kmeans_init;   /* host [M][2][K] positions in the k-means sample, or NULL */
    uint32_t copies;              /* low-precision row copies to keep: bit 0 BF16, bit 1 FP8 E4M3 */
    int32_t adaptive;             /* §7 Adaptive Subspace Decomposition: 0 equal split of §3; 1
                                     contiguous subspaces of near-equal variance shares
                                     (crisp_adaptive_bounds of the stored rows' per-dimension
                                     variances over the covariance sample; needs D <= 256 M) */
    int32_t block_dims;           /* §7 Partial Variance Redistribution: 0 the global test and
                                     rotation of §4.1; b > 0 (a multiple of 4) cuts the dims into
                                     contiguous blocks [jb, min((j+1)b, D)), tests each block's own
                                     CEV (of its block of the sample covariance) against tau_cev
                                     (rotate = 1: every block, 0: none) and rotates each chosen
                                     block B by the orthogonal factor of the QR of G's diagonal
                                     block G_BB (sign-fixed as in §3); R is block-diagonal, the
                                     identity elsewhere, and the rows cost O(N sum w^2) */
} crisp_build_params;

/* Search parameters (Algorithm 1, §4.3, Table 1). */
typedef struct {
    int32_t k;                 /* neighbours returned (k_size), 1 <= k <= 256 */
    int32_t mode;              /* 0 Guaranteed (phi = 0), 1 Optimized (phi = 1), 2 Learned (F1) */
    double rho;                /* coverage: ids retrieved per subspace / N, in (0, 1] */
    double alpha;              /* minimum collision fraction, in [0, 1]; tau = ceil(alpha M) */
    int32_t patience_factor;   /* Optimized: stop after P = patience_factor*k unchanged; <= 0 off */
    float eps0;                /* Optimized: ADSampling margin of Eq. 2 (2.1); may be +inf */
    int64_t max_candidates;    /* 0 = no cap; else keep the cap best (V desc, id asc), cap >= k */
    int32_t precision;         /* Guaranteed mode coarse scoring: 0 none (FP32 re-rank of every
                                  candidate), 1 BF16 rows, 2 FP8 E4M3 rows with per-row scales */
    int32_t shortlist;         /* precision > 0: candidates kept by the coarse score for the FP32
                                  re-rank (>= k) */
    float depth_margin;        /* mode 2: added to the predicted log2 depths (score prefix, */
    float short_margin;        /*         coarse shortlist) before quantisation */
    int32_t verify_order;      /* Optimized mode: 0 candidates by (Hamming distance, id) (§4.3.2 Stage 2),
                                  1 by id alone (the paper's ablation without Hamming re-ranking) */
    int32_t reserved;          /* 0 */
} crisp_search_params;

/* Per-query counters written by crisp_search (device array, may be NULL). */
typedef struct {
    int64_t n_candidates;      /* |C| after the cut */
    int64_t n_verified;        /* candidates visited by the verification stage */
    int64_t n_full;            /* full-dimension distances computed */
    int64_t n_retrieved;       /* ids retrieved over all subspaces */
    int32_t fallback;          /* 1 if |C| < k triggered the fallback of Stage 1 */
    int32_t capped;            /* 1 if max_candidates cut C */
    int32_t tau;
    int32_t _pad;
} crisp_query_stats;

typedef struct {
    int64_t N;
    int32_t D, Dp, M, K, H;    /* H = widest subspace half */
    int32_t rotated;
    double cev;                /* CEV of the sample covariance (§4.1) */
    int32_t max_cell;          /* largest cell population over all subspaces */
    int32_t id_tile_log2;      /* ids per counting tile = 2^id_tile_log2 */
    int64_t device_bytes;      /* device memory held by the index */
    /* device arrays owned by the index (read-only for callers) */
    const float *R32;          /* [D][D] or NULL */
    const float *cent;         /* [M][2][K][H] */
    const int32_t *offsets;    /* [M][K*K+1] */
    const int32_t *ids;        /* [M][N] */
    const float *Xr;           /* [N][Dp] */
    const uint32_t *codes;     /* [N][Dp/32] */
    const uint16_t *Xb;        /* [N][Dp] BF16 bits, or NULL */
    const uint8_t *X8;         /* [N][Dp] FP8 E4M3 codes, or NULL */
    const float *S8;           /* [N] FP8 row scales, or NULL */
    const int32_t *sub;        /* [M+1] subspace boundaries: subspace m is [sub[m], sub[m+1]) */
    int32_t block_dims;        /* build's block width (0: global rotation test) */
    int32_t rotated_blocks;    /* blocks the block-wise test rotated */
} crisp_index_info;

/* ================================================================ index */

/* Build the index of §4.1-§4.2 from X (device [N][D] float32, caller-owned,
 * copied): spectral check, rotation when CEV > tau_cev (the library keeps the
 * rotated copy and R), k-means per subspace half, cells, CSR, sign codes;
 * with params->block_dims or params->adaptive, the §7 extensions described
 * beside those fields.  Synchronises `stream` before returning.  *out receives
 * a new index.  EINVAL: N < 2, D < 2, M outside [1, D/2], K outside [2, 64],
 * K > N, block_dims not a multiple of 4.  EUNSUPPORTED: a subspace half wider
 * than 128 dims (equal split), or D > 256 M with adaptive = 1. */
crisp_status crisp_build(const float *X, int64_t N, int32_t D, const crisp_build_params *params,
                         void *stream, crisp_index **out);

/* Release an index (NULL is a no-op).  Synchronises the device first. */
void crisp_free(crisp_index *index);

/* Serialise an index into a host buffer.  With host_buf == NULL only the size
 * is written to *bytes.  Format: a 256-byte header (magic "CRISPIX1", then
 * int64 version, N, D, Dp, M, K, H, rotated, float64 CEV at byte 72), then
 * the arrays R32 (only if rotated), cent, offsets, ids, Xr, codes of
 * crisp_index_info, each starting at a multiple of 256 bytes.  Version 1
 * has the equal split of §3; version 2 (other boundaries) adds a last
 * section, the int32 boundaries sub[M+1].  Synchronous. */
crisp_status crisp_index_export(const crisp_index *index, void *host_buf, size_t *bytes);

/* Create an index from a blob in the export format (host memory), e.g. one
 * written by another implementation of the method.  Synchronous. */
crisp_status crisp_index_import(const void *host_buf, size_t bytes, void *stream, crisp_index **out);

crisp_status crisp_index_get_info(const crisp_index *index, crisp_index_info *out);

/* The index's subspace boundaries into host memory (bounds: host [M+1] int32). */
crisp_status crisp_index_get_bounds(const crisp_index *index, int32_t *bounds);

/* Add low-precision copies of the stored rows to an index (bit 0: BF16, bit 1:
 * FP8 E4M3), as crisp_quantize_bf16 / crisp_quantize_e4m3 define them.  Copies
 * already present are kept.  Synchronous. */
crisp_status crisp_index_add_copies(crisp_index *index, uint32_t copies, void *stream);

const char *crisp_last_error(void);

/* Number of kernels this library has launched in the process so far (search
 * path and step entry points; the index build is not counted).  For launch
 * accounting by benchmarks; thread-safe, never resets. */
uint64_t crisp_kernel_launches(void);

/* ================================================================ search */

/* Answer nq queries (Algorithm 1; the problem of §3 "Exact and Approximate
 * Similarity Search": the k nearest rows of X to each query under L2).
 * Q: device [nq][D] float32 in the original space (rotated inside when the
 * index is rotated).  params: host array of p_count parameter sets, p_count = 1
 * (one set for every query) or nq (set i for query i: each query may have its
 * own k, mode, rho, alpha, precision, ...; queries are run class by class and
 * their results put back in place).  ids: device [nq][kmax] int64, sqdist:
 * device [nq][kmax] float32; row i holds query i's k_i neighbours ascending by
 * (distance, id), padded with -1 / +inf past k_i or when fewer than k_i points
 * qualify; kmax >= every k_i (kmax <= 0: the largest k_i).  stats: device [nq]
 * or NULL.  A query's result does not depend on the other queries of the batch.
 * Scratch comes from a stream-ordered memory pool the library keeps per device
 * (it holds its memory between calls; crisp_search_scratch_bytes tells how much).
 * With p_count = nq the call waits for its small host-to-device copy of the
 * per-query parameters before it returns.
 * EINVAL (nothing written): p_count not 1 or nq, kmax < some k_i, or a
 * parameter set with k outside [1, 256] or > N, rho outside (0, 1], alpha
 * outside [0, 1], mode outside {0, 1, 2}, 0 < max_candidates < k, nq < 0,
 * precision outside {0, 1, 2} or used outside Guaranteed mode, shortlist < k,
 * or a precision whose row copy the index lacks; mode 2 without a model or a
 * BF16 copy.
 *
 * Mode 2 (Learned, the engine's F1 extension; the paper's patience and
 * ordering are what it replaces, §4.3.2 Stage 3): after the Guaranteed cut, a
 * small MLP (crisp_index_set_model) reads per-query features (crisp_learned_data)
 * and predicts two log2 depths; the first depth_V candidates by (V desc, id asc)
 * are scored on the BF16 rows, the depth_S best form the shortlist, and the FP32
 * re-rank of the shortlist gives the top-k.  Depth = ceil(2^(j/4)), j =
 * ceil(4 (prediction + margin)), clamped to [k, |C|] and [k, depth_V]. */
crisp_status crisp_search(const crisp_index *index, const float *Q, int32_t nq, const crisp_search_params *params,
                          int32_t p_count, int64_t *ids, float *sqdist, int32_t kmax, crisp_query_stats *stats,
                          void *stream);

/* As crisp_search, with HOST buffers (Q [nq][D], ids [nq][kmax], sqdist
 * [nq][kmax], stats [nq] or NULL): copies in, searches, copies out, and
 * synchronises. */
crisp_status crisp_search_host(const crisp_index *index, const float *Q, int32_t nq,
                               const crisp_search_params *params, int32_t p_count, int64_t *ids, float *sqdist,
                               int32_t kmax, crisp_query_stats *stats, void *stream);

/* Device bytes of scratch crisp_search needs for nq queries with these
 * parameter sets (p_count = 1 or nq; for admission). */
crisp_status crisp_search_scratch_bytes(const crisp_index *index, int32_t nq, const crisp_search_params *params,
                                        int32_t p_count, size_t *bytes);

/* The library's readings of the paper's parameters (Theorem 1: tau = alpha M;
 * Algorithm 1: the per-subspace retrieval budget): tau = ceil(alpha M - 1e-9),
 * budget = max(1, ceil(rho N - 1e-9)). */
int32_t crisp_search_tau(double alpha, int32_t M);
int64_t crisp_search_budget(double rho, int64_t N);

/* =========================================== serving (continuous batching)
 * A request server over one index: requests (one query each, any search
 * parameters) arrive from any thread; a dispatcher thread batches the waiting
 * requests oldest first (up to max_batch, whatever their k and mode: one
 * crisp_search with per-query parameters), admits a batch when one of
 * `streams` stream slots is free and its search scratch
 * (crisp_search_scratch_bytes) fits within scratch_budget next to the batches
 * already on the GPU, and runs copy-in, crisp_search and copy-out on that
 * slot's stream.  Batches on different slots overlap on the GPU.  A request's
 * result does not depend on the batch it ran in (each query is searched
 * independently).  The server owns pinned host and device staging buffers. */
typedef struct crisp_server crisp_server;

typedef struct {
    int32_t streams;           /* concurrent batches (stream slots), 1..64 */
    int32_t max_batch;         /* requests per batch */
    int64_t scratch_budget;    /* device bytes of search scratch in flight (0: half the device memory
                                  free at creation, between 8 and 64 GiB) */
} crisp_server_params;

typedef struct {
    uint64_t submitted, completed, failed, batches;
    double mean_batch;         /* requests per admitted batch */
    double p50_us, p99_us, max_us, mean_us;   /* arrival -> completion latency */
    int64_t scratch_peak;      /* largest scratch in flight (bytes) */
} crisp_server_stats;

/* Start a server (its dispatcher thread) on the index's device.  The index
 * must outlive the server. */
crisp_status crisp_server_create(const crisp_index *index, const crisp_server_params *params, crisp_server **out);

/* Queue one query (host [D] float32, copied) with its search parameters
 * (validated now: EINVAL as crisp_search).  *ticket identifies the request. */
crisp_status crisp_server_submit(crisp_server *server, const float *q, const crisp_search_params *params,
                                 uint64_t *ticket);

/* Wait for a request (timeout_ms < 0: no limit) and take its result: ids /
 * sqdist host [k], stats and latency (microseconds) may be NULL.  The ticket
 * is consumed.  ETIMEOUT if it did not finish in time (the ticket stays valid). */
crisp_status crisp_server_wait(crisp_server *server, uint64_t ticket, int32_t timeout_ms, int64_t *ids,
                               float *sqdist, crisp_query_stats *stats, double *latency_us);

/* Open-loop trace replay (a load generator for measuring the server; the
 * paper has no counterpart).  Request i (of n) asks query Q[qidx[i]] (host
 * [nq][D] float32) with params[pidx[i]] (host [n_params]) and enters the server at arrival_us[i]
 * microseconds after the call starts (nondecreasing), whatever the server's
 * state; its latency counts from that scheduled time.  The calling thread
 * submits on schedule, then waits for every request: results go to ids /
 * sqdist (host [n][kmax], -1 / +inf padded past each request's k), latencies
 * to latency_us (host [n], NaN for a failed request), the whole replay's wall
 * time to *wall_us (may be NULL).  EINVAL (nothing submitted) for an index
 * outside its array, k > kmax or unsorted arrivals; otherwise the first failed
 * request's status after all have finished. */
crisp_status crisp_server_replay(crisp_server *server, const float *Q, int32_t nq, int64_t n, const int32_t *qidx,
                                 const crisp_search_params *params, int32_t n_params, const int32_t *pidx,
                                 const double *arrival_us, int32_t kmax, int64_t *ids, float *sqdist,
                                 double *latency_us, double *wall_us);

crisp_status crisp_server_get_stats(crisp_server *server, crisp_server_stats *out);
crisp_status crisp_server_reset_stats(crisp_server *server);

/* Finish every queued request, stop the dispatcher and free the server. */
void crisp_server_destroy(crisp_server *server);

/* ================================= F1: learned re-rank depth (small MLP)
 * MLP F -> H -> H -> O, GELU on both hidden layers, parameters packed in one
 * device float array: W1 [F][H], b1 [H], W2 [H][H], b2 [H], W3 [H][O], b3 [O]
 * (crisp_mlp_param_count floats).  GELU(z) = z/2 (1 + erf(z/sqrt 2)) with erf by
 * Abramowitz & Stegun 7.1.28.  For the search the index's model has F = 2M + 68
 * features and O = 2 outputs (log2 depths). */
int64_t crisp_mlp_param_count(int32_t F, int32_t H, int32_t O);

/* Seeded Xavier-uniform weights, zero biases.  EINVAL: H > 256 or O > 8. */
crisp_status crisp_mlp_init(float *params, int32_t F, int32_t H, int32_t O, uint64_t seed, void *stream);

/* Inference in the fixed FP32 order the search uses: every unit an fmaf chain
 * over its inputs in order from its bias.  X device [B][F], Y device [B][O]. */
crisp_status crisp_mlp_infer(const float *params, int32_t F, int32_t H, int32_t O, const float *X, int64_t B, float *Y,
                             void *stream);

/* Mean squared error of a batch (X [B][F], targets T [B][O]) and its gradient,
 * packed like params (device [param_count]); *loss is a device float. */
crisp_status crisp_mlp_loss_grad(const float *params, int32_t F, int32_t H, int32_t O, const float *X, const float *T,
                                 int64_t B, float *grads, float *loss, void *stream);

/* One Adam step (step number t >= 1) on n parameters; m, v: device state. */
crisp_status crisp_mlp_adam(float *params, const float *grads, float *m, float *v, int64_t n, float lr, float beta1,
                            float beta2, float eps, int32_t t, void *stream);

/* Train params (already initialised) on n rows of X / T for `epochs` epochs of
 * shuffled mini-batches with Adam (lr, betas 0.9 / 0.999, eps 1e-8).  The mean
 * loss of each epoch goes to epoch_loss (host [epochs], may be NULL).
 * Synchronous. */
crisp_status crisp_mlp_train(float *params, int32_t F, int32_t H, int32_t O, const float *X, const float *T,
                             int64_t n, int32_t epochs, int32_t batch, float lr, uint64_t seed, float *epoch_loss,
                             void *stream);

/* Attach a learned-depth model (device params, copied) with H hidden units,
 * F = 2M + 68 inputs and 2 outputs to the index. */
crisp_status crisp_index_set_model(crisp_index *index, const float *params, int32_t H, void *stream);

/* Training data generated by the plain method: for nq queries (device [nq][D],
 * original space) with the Guaranteed parameters p (k, rho, alpha,
 * max_candidates), the feature rows (device [nq][2M+68]) and the labels
 * (device [nq][2] int64): the smallest prefix of C by (V desc, id asc) that
 * holds the exact top-k over C, and the smallest BF16 coarse-score prefix of
 * that prefix that holds them.  targets (device [nq][2] float, may be NULL)
 * receives log2 of the labels.  Needs the BF16 copy. */
crisp_status crisp_learned_data(const crisp_index *index, const float *Q, int32_t nq, const crisp_search_params *p,
                                float *features, int64_t *labels, float *targets, void *stream);

/* ====================================== steps of the path (one per stage) */

/* B1 (§4.1): sample covariance, FP64, mean-centred, divided by S-1, of the
 * rows X[rows[s]] (X device [N][ldx] float32, rows device [S] int64 < N).
 * cov: device [D][D] float64.  EINVAL: S < 2, D < 1. */
crisp_status crisp_covariance(const float *X, int64_t N, int32_t D, int32_t ldx, const int64_t *rows, int64_t S,
                              double *cov, void *stream);

/* B1 (§4.1 "Eigenvalue Decomposition"): all eigenvalues of the symmetric
 * matrix A (device [D][D] float64, overwritten), descending, into eig (device
 * [D] float64): Householder tridiagonalisation, then Sturm-sequence bisection. */
crisp_status crisp_eigvalsh(double *A, int32_t D, double *eig, void *stream);

/* B1: CEV = (sum of the top floor(0.2 D) eigenvalues) / (sum of all) of the
 * sample covariance of X[rows] (§4.1).  *cev is a host double; synchronous. */
crisp_status crisp_cev(const float *X, int64_t N, int32_t D, int32_t ldx, const int64_t *rows, int64_t S,
                       double *cev, void *stream);

/* §7 Adaptive Subspace Decomposition: per-dimension sample variance, FP64,
 * mean-centred, divided by S-1, of the rows X[rows[s]] (X device [N][ldx]
 * float32, rows device [S] int64 < N) into var (device [D] float64). */
crisp_status crisp_column_variance(const float *X, int64_t N, int32_t D, int32_t ldx, const int64_t *rows,
                                   int64_t S, double *var, void *stream);

/* §7 Adaptive Subspace Decomposition (host arithmetic): boundaries (host
 * [M+1] int32) of M contiguous subspaces with near-equal shares of the total
 * variance (var: host [D] float64).  With V_j = var[0] + ... + var[j-1]
 * (FP64, in order), boundary m is the last j with V_j <= m V_D / M, held to
 * [b_{m-1} + 2, b_{m-1} + 256] and to what leaves every later subspace 2..256
 * dims; zero total variance gives the equal split.  EINVAL unless
 * 2M <= D <= 256 M. */
crisp_status crisp_adaptive_bounds(const double *var, int32_t D, int32_t M, int32_t *bounds);

/* B2 (§3 Randomized Orthogonal Rotation): R = Q diag(sign(diag R')) where
 * G = Q R' is the Householder QR of G (device [D][D] float64, row-major,
 * not modified).  R: device [D][D] float64. */
crisp_status crisp_rotation_from_gaussian(const double *G, int32_t D, double *R, void *stream);

/* B2 / Q1: Y = X R in the GEMV order (FP32), X device [N][ldx], R device
 * [D][D] float32, Y device [N][ldy] with ldy >= D; columns D..ldy-1 of Y are
 * zeroed.  Y must not overlap X. */
crisp_status crisp_rotate_rows(const float *X, int64_t N, int32_t D, int32_t ldx, const float *R, float *Y,
                               int32_t ldy, void *stream);

/* B2 on the tensor cores (tcgen05, TF32 pipe): Y = X R with each product
 * split as a_hi b_hi + a_hi b_lo + a_lo b_hi (hi = the value with its low 13
 * mantissa bits cleared, lo = the rest), FP32 accumulation in tensor memory.
 * The result agrees with the FP32 product to about 1e-6 of |x| |R e_j| per
 * output, but not bitwise with crisp_rotate_rows (another summation order).
 * The build uses it for the rows of the index (§4.1: X' = X R); queries keep
 * crisp_rotate_rows.  X device [N][ldx], 16-byte aligned with ldx a multiple
 * of 4 (rows are fetched by TMA); R device [D][D] float32; Y device [N][ldy],
 * ldy >= D, columns D..ldy-1 zeroed; Y must not overlap X.  Synchronous on
 * the stream (it reads back the kernel's error word): ECUDA if a pipeline
 * wait of the kernel timed out. */
crisp_status crisp_rotate_rows_tc(const float *X, int64_t N, int32_t D, int32_t ldx, const float *R, float *Y,
                                  int32_t ldy, void *stream);

/* B3 (§4.2, IMI codebooks): Lloyd's k-means over dims [off, off+h) of the S
 * training rows T (device [S][ldt] float32): centroids start at the rows
 * init (device [K] int32 < S) and are updated `iters` times (assignment by
 * the SEQ distance, ties to the lowest index; means in FP64 rounded to FP32;
 * an empty cluster keeps its centroid).  C: device [K][H] float32, columns
 * h..H-1 zeroed. */
crisp_status crisp_kmeans(const float *T, int64_t S, int32_t ldt, int32_t off, int32_t h, int32_t K, int32_t H,
                          const int32_t *init, int32_t iters, float *C, void *stream);

/* B3 (§3 u(x)): cells[m][n] = argmin_left*K + argmin_right of row n of Xr
 * (device [N][Dp]) in subspace m, SEQ distances, ties to the lowest index.
 * sub: host [M+1] subspace boundaries (NULL: the equal split floor(mD/M));
 * cent: device [M][2][K][H]; cells: device [M][N] uint16.  EINVAL: a
 * subspace outside 2..256 dims or a half wider than H. */
crisp_status crisp_assign_cells(const float *Xr, int64_t N, int32_t D, int32_t Dp, int32_t M, int32_t K,
                                int32_t H, const int32_t *sub, const float *cent, uint16_t *cells, void *stream);

/* B3 on the tensor cores (tcgen05), same result as crisp_assign_cells bit
 * for bit: the tensor cores score every centroid (|c|^2 - 2 x.c), and the
 * centroids whose score is within its proven error bound of the best are
 * re-measured with the SEQ distance on the FP32 rows (ties to the lowest
 * index).  Xb NULL: one TF32 pass over Xr; else Xb (device [N][Dp] BF16 bits,
 * the round-to-nearest-even copy of Xr, as crisp_quantize_bf16 writes it) is
 * scored in one BF16 pass against the centroids rounded to BF16 (half the
 * bytes, a bound about twice as wide, so more centroids are re-measured).
 * The build uses the TF32 form for every row.  Xr and Xb must be 16-byte
 * aligned with Dp a multiple of 32 (rows are fetched by TMA); K <= 64.
 * Synchronous on the stream: ECUDA if a pipeline wait of the kernel timed out. */
crisp_status crisp_assign_cells_tc(const float *Xr, const uint16_t *Xb, int64_t N, int32_t D, int32_t Dp, int32_t M,
                                   int32_t K, int32_t H, const int32_t *sub, const float *cent, uint16_t *cells,
                                   void *stream);

/* B4 (§4.2 CSR): for one subspace, Offsets (device [K2+1] int32) and ids
 * (device [N] int32): ids grouped by ascending cell, ascending inside a cell.
 * cells: device [N] uint16 < K2.  EINVAL: K2 > 4096 or N >= 2^31. */
crisp_status crisp_csr_build(const uint16_t *cells, int64_t N, int32_t K2, int32_t *offsets, int32_t *ids,
                             void *stream);

/* B5 (§3 Binary Quantization): codes[n][w] bit b = (Xr[n][32w+b] > 0).
 * Xr device [N][Dp] (Dp multiple of 32), codes device [N][Dp/32] uint32. */
crisp_status crisp_sign_codes(const float *Xr, int64_t N, int32_t Dp, uint32_t *codes, void *stream);

/* F2 (coarse scoring): BF16 copy of Xr (device [N][Dp] float32) with round to
 * nearest even; Xb: device [N][Dp] uint16 (the BF16 bit patterns). */
crisp_status crisp_quantize_bf16(const float *Xr, int64_t N, int32_t Dp, uint16_t *Xb, void *stream);

/* F2: FP8 E4M3 copy with one scale per row: s = fl(max_d |x_d| / 448) (1 for a
 * zero row), code = e4m3(fl(x_d / s)), round to nearest even, saturating to
 * +-448 (OCP E4M3, no infinities).  X8: device [N][Dp] uint8; scale: device [N]. */
crisp_status crisp_quantize_e4m3(const float *Xr, int64_t N, int32_t Dp, uint8_t *X8, float *scale, void *stream);

/* F2: coarse scoring of the candidates.  For each query row of Qr (device
 * [nq][Dp]) the CR32 distance to every candidate's dequantised row (BF16 widened
 * exactly, or the E4M3 value times the row scale, precision 1 or 2), then the S
 * smallest by (distance, id), written in ascending id to out (device
 * [nq][out_stride] int32) with their number in nout (device [nq] int64).
 * cand/ncand as written by crisp_count_cut.  Large batches of BF16 scoring
 * take the tensor-core path described at crisp_rerank: one BF16 pass (the
 * query rounded to BF16) bounds every coarse score, and only the candidates
 * whose lower bound reaches the S-th smallest upper bound are scored exactly;
 * large E4M3 batches are scored in groups of queries that read each shared row
 * once.  Every path gives the same shortlist.  EINVAL: the index lacks the
 * copy, S < 1, out_stride < S. */
crisp_status crisp_shortlist(const crisp_index *index, const float *Qr, int32_t nq, const int32_t *cand,
                             int64_t cand_stride, const int64_t *ncand, int32_t precision, int32_t S, int32_t *out,
                             int64_t out_stride, int64_t *nout, void *stream);

/* Q2 (Algorithm 1 "Dist1, Dist2"): for every query row of Qr (device [nq][Dp],
 * already rotated) and subspace m, the K partial squared distances to each
 * half's centroids (SEQ order), sorted ascending with ties by centroid index.
 * sorted, perm: device [nq][M][2][K] (float32, int32 centroid index). */
crisp_status crisp_half_dists(const crisp_index *index, const float *Qr, int32_t nq, float *sorted, int32_t *perm,
                              void *stream);

/* Q2+Q3 (Algorithm 1 lines 3-17, §4.3.1 multi-sequence): per query and
 * subspace, the cells visited in ascending (cost, i, j), cost = fl(Dist1s[i] +
 * Dist2s[j]), until the ids retrieved reach `budget` (a visited cell is
 * consumed whole).  act: device [nq][M][K*K] int32 entries (w << 16) | cell in
 * visit order, w = 2 if phi == 1 and rank <= k else 1; nact: device [nq][M]
 * int32; retrieved: device [nq][M] int64 (may be NULL). */
crisp_status crisp_activate(const crisp_index *index, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                            int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved, void *stream);

/* crisp_activate that also writes the cost of the first and of the last
 * visited cell of each (query, subspace): device [nq][M] float each (may be NULL). */
crisp_status crisp_activate_costs(const crisp_index *index, const float *Qr, int32_t nq, int32_t phi, int32_t k,
                                  int64_t budget, int32_t *act, int32_t *nact, int64_t *retrieved, float *cost_first,
                                  float *cost_last, void *stream);

/* Q4+Q5 (Eq. 1 collision counting, Algorithm 1 line 20, §4.3.2 Stage 1):
 * V[x] = sum over subspaces of the weight of the activated cell holding x;
 * C = {x : V[x] >= tau} in ascending id; if tau >= 1 and |C| < k, C is the
 * min(k, #{V >= 1}) points of highest (V, -id) (fallback); if cap > 0 and
 * |C| > cap, C keeps its cap points of highest (V, -id).  act/nact as written
 * by crisp_activate.  cand: device [nq][cand_stride] int32, ncand: device
 * [nq] int64, score: device [nq][cand_stride] uint8 (V of each candidate) or
 * NULL, how: device [nq] int32 (0 plain, 1 fallback, 2 capped) or NULL.
 * cand_stride must bound |C|: EINVAL if cap > cand_stride; when cap == 0 a
 * query whose |C| exceeds cand_stride reports CRISP_EINVAL at the next sync
 * through how = -1 and ncand = the true |C| (nothing past the stride is written).
 * EUNSUPPORTED: weighted scores above 255 (M > 127). */
crisp_status crisp_count_cut(const crisp_index *index, const int32_t *act, const int32_t *nact, int32_t nq,
                             int32_t tau, int32_t k, int64_t cap, int32_t *cand, int64_t cand_stride,
                             int64_t *ncand, uint8_t *score, int32_t *how, void *stream);

/* Q6 (§4.3.2 Stage 3, phi = 0): exact CR32 distance from each query row of Qr
 * (device [nq][Dp]) to each of its candidates, then the k smallest by
 * (distance, id).  cand/ncand as written by crisp_count_cut (ascending ids).
 * ids: device [nq][k] int64, sqdist: device [nq][k] float32, padded -1/+inf.
 * Batches of 256 to 16,384 queries with cand_stride >= 2,048 are ordered by
 * a k-d partition of the query rows along the batch's top principal
 * directions (queries close in space share most candidates) and scored in
 * groups of 64 queries that
 * fetch each shared candidate row once: one TF32 pass on the tensor cores
 * gives every (query, candidate) pair an upper and a lower bound of its CR32
 * distance, and only the candidates whose lower bound reaches the k-th
 * smallest upper bound are measured exactly.  Other batches stream (query,
 * candidate) pairs.  Both give the same bits: every returned distance is the
 * CR32 value of its own (query, row) pair. */
crisp_status crisp_rerank(const crisp_index *index, const float *Qr, int32_t nq, const int32_t *cand,
                          int64_t cand_stride, const int64_t *ncand, int32_t k, int64_t *ids, float *sqdist,
                          void *stream);

/* crisp_rerank for callers that cannot allocate device memory while they
 * search -- for instance when another allocator owns all of the GPU's memory,
 * or when the query path must not call cudaMalloc/cudaFree (both can block and
 * synchronise the device).  Same arguments, same results as crisp_rerank, but
 * nothing is allocated: the per-candidate distance scratch is a fixed array of
 * CRISP_RERANK_NOALLOC_MAX floats (16 MiB) that every GPU loading this library
 * holds until the process exits.  The paper has no counterpart to this entry
 * point; it exists for such callers only.
 *  - EINVAL if nq * cand_stride > CRISP_RERANK_NOALLOC_MAX (nothing is run).
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any stream
 *    capture.
 *  - All calls share the one array and it keeps the previous call's contents;
 *    every value is written before it is read, so nothing needs clearing.
 *    Calls that overlap on the GPU (e.g. on two streams) race on the array:
 *    order them on one stream or synchronise between them. */
#define CRISP_RERANK_NOALLOC_MAX (4 * 1024 * 1024)
crisp_status crisp_rerank_noalloc(const crisp_index *index, const float *Qr, int32_t nq, const int32_t *cand,
                                  int64_t cand_stride, const int64_t *ncand, int32_t k, int64_t *ids, float *sqdist,
                                  void *stream);

/* Profiling aid (the paper has no counterpart): while enabled, the tensor-core
 * re-rank of large batches (crisp_rerank, crisp_search) records CUDA events on
 * its stream around its scoring kernel and copies the kernel's work counts.
 * crisp_rerank_profile_read waits for what was recorded and returns, for the
 * scoring launches since the previous read: their number, their summed
 * duration, the (query group, row) entries multiplied on the tensor cores (each
 * one row against a group's 64 queries over Dp dims, one TF32 pass over the
 * FP32 rows or one BF16 pass over the index's BF16 copy) and the (row, query)
 * pairs whose distance bounds were written.  Call both from one thread;
 * reading also clears.  Synchronous. */
typedef struct {
    int64_t launches;
    double ms;                 /* summed kernel duration, CUDA events on the launching stream */
    int64_t rows;              /* (query group, row) entries scored */
    int64_t pairs;             /* (row, query) pairs bounded */
    int32_t Dp;                /* padded dimension of the last launch */
    int32_t group;             /* queries per group (the MMA's N) */
    int32_t elem_bytes;        /* bytes per row element of the last launch: 4 (TF32 pass), 2 (BF16 pass) */
    int32_t _pad;
} crisp_rerank_profile;

crisp_status crisp_rerank_profile_enable(int32_t on);
crisp_status crisp_rerank_profile_read(crisp_rerank_profile *out);

/* The query order of a large batch's row-sharing groups (an engineering step
 * of the grouped re-rank and coarse scorers; the paper's engine scores one
 * query at a time, §4.3.2): qord (device [nq] int32) receives a permutation of
 * 0..nq-1 such that each run of G consecutive entries (the last one shorter)
 * is one group.  Queries are ordered by a k-d partition of their coordinates
 * along the batch's top four principal directions (from subspace iteration
 * on up to 1,024 evenly spaced rows): every node larger than max(G, 64)
 * splits at a group-aligned median of its coordinate with the widest range,
 * ties by position, and for G < 64 each leaf of 64 splits on down to G the
 * same way.  Qr: device [nq][Dp] float32 (the rotated queries).  The order
 * decides only which queries share a group, never a search result.
 * Deterministic.  EINVAL: nq > 16,384, G < 1, Dp < 1, or more than 256 leaves
 * of max(G, 64). */
crisp_status crisp_query_order(const float *Qr, int32_t nq, int32_t Dp, int32_t G, int32_t *qord, void *stream);

/* Q7 (§4.3.2 Stages 2-3, phi = 1; Eq. 2): candidates ordered by (Hamming
 * distance of sign codes, id); each is pruned by ADSampling checks at t = 32,
 * 64, ... < D when the running top-k is full (d_t > fl(r_k^2 * f_t), f_t =
 * fl32((t/D)(1 + eps0/sqrt t)^2) evaluated in FP64), else measured exactly and
 * offered to the top-k; the walk stops once P = patience consecutive
 * candidates left the top-k unchanged (patience <= 0: never).  Results equal
 * the sequential walk exactly.  n_verified, n_full: device [nq] int64 or NULL;
 * n_blocks: device [nq] int64 or NULL, the 32-dim row blocks the kernel read
 * (its row traffic is 128 bytes per block).
 * EUNSUPPORTED: a query with more than 32768 candidates (cap them). */
crisp_status crisp_verify_opt(const crisp_index *index, const float *Qr, int32_t nq, const int32_t *cand,
                              int64_t cand_stride, const int64_t *ncand, int32_t k, float eps0, int64_t patience,
                              int32_t order, int64_t *ids, float *sqdist, int64_t *n_verified, int64_t *n_full,
                              int64_t *n_blocks, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CRISP_H */
