/*
 * farm.h -- C ABI of the GB300 (sm_103a) relational-retrieval library.
 *
 * The library implements the query-time scoring stage of FARM ("Find Anything
 * using Relational Spatial Memory"): given an object-level memory M and a
 * parsed query q, it returns y_hat = g(q, M) (Sec. 2.1, "Relational object
 * retrieval"), realised as
 *
 *   score(e; q, M) = max over bindings eta with eta(x*) = e of Verify(eta),
 *   y_hat          = TopK_e score(e)                          (Sec. 2.3; App. B)
 *
 * with the unary score s_sem given by reciprocal-rank fusion of descriptor
 * similarity (App. D.2 step 3), the closed-form relation evaluators of App. D.2
 * step 4 (Above, Below, LeftOf, RightOf, Near, NextTo, On, InFrontOf, Behind,
 * Closest, Farthest, Inside), the Hellinger form of Near (Sec. 2.3) and the
 * ternary Between of App. B,
 * anchors bound greedily to
 * their best witness among the top-K_a landmark candidates (App. B,
 * "Query-time complexity"; App. D.2 step 4) and the composite
 * s = s_sem * [(1 - w) + w * gbar] of App. D.2 step 5.
 *
 * Conventions for every call:
 *  - Every call returns a farm_status and never aborts the process.  On an
 *    error, farm_last_error(ctx) holds a one-line message.
 *  - Inputs are owned by the caller and never retained after the call
 *    returns (device inputs: after the work the call enqueues has run).
 *    The context owns all device memory it allocates.
 *  - Work is enqueued on the context's CUDA stream in call order.  Calls that
 *    write host memory synchronise that stream before returning.
 *  - A context is used by one host thread at a time.
 *  - Invalid arguments (null pointers, non-positive sizes, unknown scene,
 *    more than FARM_MAX_CONSTRAINTS constraints, k out of range, non-finite
 *    host data) are reported as FARM_EINVAL before anything is enqueued.
 *    Embeddings in device memory are checked on the GPU: a zero or non-finite
 *    row is reported by the next synchronising call (farm_topk with host
 *    outputs, or farm_sync) as FARM_EINVAL.
 */
#ifndef FARM_H
#define FARM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct farm_ctx farm_ctx;

typedef enum {
    FARM_OK = 0,
    FARM_EINVAL = 1,    /* bad argument or input data */
    FARM_ENOMEM = 2,    /* a device or host allocation failed */
    FARM_ECUDA = 3,     /* a CUDA call failed (message has the CUDA error) */
    FARM_ESTATE = 4,    /* call out of order (e.g. stale batch handle) */
    FARM_ETIMEOUT = 5   /* a bounded device-side wait gave up */
} farm_status;

/* Predicate codes (App. B predicate vocabulary; evaluators of App. D.2 step 4). */
typedef enum {
    FARM_ABOVE = 0,     /* sig((z_e - z_a) / tau_v) */
    FARM_BELOW = 1,     /* sig((z_a - z_e) / tau_v) */
    FARM_LEFT_OF = 2,   /* mean over the candidate's stored views of sig((u_a - u_e) / tau_h) */
    FARM_RIGHT_OF = 3,  /* mean over the candidate's stored views of sig((u_e - u_a) / tau_h) */
    FARM_NEAR = 4,      /* exp(-|p_e - p_a|^2 / (2 sigma_near^2)) */
    FARM_NEXT_TO = 5,   /* exp(-|p_e - p_a|^2 / (2 sigma_next^2)) */
    FARM_ON = 6,        /* sig((rho_a - d_xy) / on_gate) * exp(-g^2 / (2 on_band^2)): rho_a half the
                           landmark's larger horizontal size, d_xy the horizontal centre distance,
                           g = e's bottom - a's top */
    FARM_IN_FRONT_OF = 7, /* mean over the candidate's stored views of sig((Z_a - Z_e) / tau_d) */
    FARM_BEHIND = 8,    /* mean over the candidate's stored views of sig((Z_e - Z_a) / tau_d) */
    FARM_CLOSEST = 9,   /* 1 / rank_d: e's rank by distance to a among the query's k_closest
                           best target candidates other than a (0 for e outside them) */
    FARM_FARTHEST = 10, /* 1 / (|C| - rank_d + 1) over the same set C */
    FARM_NEAR_H = 11,   /* 1 - H(N_e, N_a): the Hellinger form of Near (Sec. 2.3), with each object the
                           Gaussian of its box centre and covariance diag(s^2) / 12 */
    FARM_INSIDE = 12,   /* containment (App. D.2 step 4): the fraction of e's box volume inside a's box */
    FARM_BETWEEN = 13,  /* Between(e, a_p, a_q) (App. B), first landmark a_p: the constraint right after it
                           must be FARM_BETWEEN_AND with the second landmark a_q.  The pair is bound jointly
                           (the best (a_p, a_q) over L_p x L_q, a_p != a_q, neither = e; lower a_p, then
                           lower a_q on ties) and is one factor of the geometric mean; both constraints
                           report its score.  sig(t / 0.1) sig((1 - t) / 0.1) exp(-d^2 / (2 sigma_near^2)):
                           t = e's centre projected on the segment a_p -> a_q (0 at a_p, 1 at a_q), d its
                           distance from the line; 0 when the two centres coincide */
    FARM_BETWEEN_AND = 14 /* the second landmark of a Between */
} farm_pred;

/* Arithmetic of the descriptor-similarity stage (App. D.2 step 3). */
typedef enum {
    FARM_PREC_FP32 = 0,       /* FP32-accurate: tcgen05 tensor cores, 3-term FP16 split (22-bit operands) */
    FARM_PREC_BF16 = 1,       /* BF16 operands, FP32 accumulate, FP32 rescore of the borderline */
    FARM_PREC_FP8 = 2,        /* FP8-E4M3 operands with per-row scales, FP32 accumulate, FP32 rescore */
    FARM_PREC_FP32_SIMT = 3,  /* FP32 FMA on the CUDA cores (independent check path) */
    FARM_PREC_LEARNED = 4     /* learned 128-d prefilter (farm_mlp_*), top 512 re-scored in FP32 */
} farm_precision;

#define FARM_MAX_CONSTRAINTS 4
#define FARM_MAX_VIEWS 16

/* flags */
#define FARM_PTR_DEVICE 1u    /* the call's array arguments are device pointers */
#define FARM_GRAPH 2u         /* farm_query_batch: run the batch's device work as a CUDA graph (see there) */
#define FARM_UNFUSED 4u       /* farm_query_batch: write the whole similarity block and select from it (see there) */
#define FARM_ASYNC 8u         /* farm_topk with host outputs: do not synchronise (see there) */
#define FARM_FUSED 16u        /* farm_query_batch: the fused rank selection for every scene (see there) */

/*
 * The method's constants.  mu = 5 (reciprocal-rank offset), w = 0.5 (blend
 * weight), class_mis = 0.3 (soft class factor), sigma_near = 0.5 m are given in
 * App. D.2 steps 3-5.  tau_v (m), tau_h (image-plane units), z_min (m) and
 * k_anchor (landmark candidates per constraint, K_a of App. B) are not given
 * by the paper; farm_default_params sets 0.25, 0.10, 0.05 and 16.
 * k_max is the largest k a later farm_topk may ask for: farm_query_batch keeps
 * only candidates that can still reach the top k_max (see farm_query_batch).
 * rescore (1 .. 512) is the number of candidates per target row the BF16 path
 * re-scores in FP32 (at least the rank bound R of farm_query_batch; the FP8
 * path keeps twice as many, at most 512); landmark rows re-score a quarter of
 * that, at least k_anchor.  Of those, only the borderline ones are re-scored:
 * candidates whose reduced-precision cosine lies within rescore_band (>= 0) of
 * the R-th (or K_a-th) reduced-precision value, 16 times that band for FP8
 * (four fewer significant bits); farm_default_params sets 2e-3, about thirty
 * standard deviations of the BF16 stage's cosine error on unit descriptors
 * of length 1152.
 * sigma_next = 1.0 m (NextTo) is given in App. D.2 step 4; on_gate, on_band
 * (m), tau_d (m) and k_closest (the candidate set of Closest / Farthest: the
 * query's k_closest objects of smallest target rank; 1 .. the rank bound R)
 * are not; farm_default_params sets 0.10, 0.10, 0.25 and 16.
 */
typedef struct {
    float mu;
    float w;
    float class_mis;
    float sigma_near;
    float tau_v;
    float tau_h;
    float z_min;
    int32_t k_anchor;
    int32_t k_max;
    int32_t rescore;
    float rescore_band;
    float sigma_next;
    float on_gate;
    float on_band;
    float tau_d;
    int32_t k_closest;
} farm_params;

/* Fills *p with the defaults above (k_max = 10, rescore = 256, rescore_band = 2e-3). */
void farm_default_params(farm_params *p);

/*
 * Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * the context enqueues on (NULL: the context creates and owns a stream).
 * `params` may be NULL (defaults).  Requirements: 0 < w < 1, 0 < class_mis <= 1,
 * mu >= 0, sigma_near, tau_v, tau_h > 0, z_min >= 0, 1 <= k_anchor <= 256,
 * 1 <= k_max and the resulting target-candidate bound <= 512 (see
 * farm_query_batch).
 */
farm_status farm_create(farm_ctx **out, int device, void *cuda_stream, const farm_params *params);

/* Frees every device buffer of the context (synchronises its stream). */
farm_status farm_destroy(farm_ctx *ctx);

/*
 * Uploads (or replaces) scene `scene_id` (0 <= scene_id < 4096): the memory
 * M_t of Sec. 2.2, one entity per object.
 *   n       number of objects (>= 1)
 *   dim     descriptor length (1 .. 8192)
 *   desc    [n, dim] row-major FP32 descriptors; normalised to unit length on
 *           the GPU (a zero or non-finite row is FARM_EINVAL for host data)
 *   cls     [n] int32 object classes (compared with a query's target class)
 *   box     [6, n] FP32 SoA rows cx, cy, cz, sx, sy, sz (metres, z up); the
 *           centre stands in for the entity's Gaussian mean
 *   n_views number of stored views per object (0 .. FARM_MAX_VIEWS)
 *   views   [6, n_views, n] FP32 SoA rows ox, oy, oz, fx, fy, fz: camera
 *           position and viewing direction of each stored view (App. D.1
 *           step 6 keeps such views); NULL when n_views == 0
 *   flags   FARM_PTR_DEVICE when the arrays are device pointers
 * The data is copied; the call returns once the copies are enqueued.
 */
farm_status farm_memory_upload(farm_ctx *ctx, int32_t scene_id, int64_t n, int32_t dim,
                               const float *desc, const int32_t *cls, const float *box,
                               int32_t n_views, const float *views, uint32_t flags);

/*
 * Enqueues the scoring of n_q queries (n_q >= 0).  Each query is the typed
 * QueryGraph of App. D.2 step 1 reduced to a star: a target embedding, a
 * target class, and up to 4 constraints rho_i(x*, a_i), each a predicate and a
 * landmark embedding.
 *   scene_of_q [n_q]       host int32 scene of each query (uploaded scene ids)
 *   tgt_emb    [n_q, dim]  FP32 target embeddings (any norm; normalised on the GPU)
 *   tgt_cls    [n_q]       host int32 target class, -1 = none (class factor off)
 *   c_off      [n_q + 1]   host int32 CSR offsets: query q owns constraints
 *                          c_off[q] .. c_off[q+1]-1 (at most 4); c_off[0] = 0
 *   c_pred     [n_c]       host int32 farm_pred codes, n_c = c_off[n_q]
 *   c_emb      [n_c, dim]  FP32 landmark embeddings
 *   precision  a farm_precision value.  With FARM_PREC_BF16 (unless
 *              FARM_FUSED) or FARM_PREC_FP8 the scenes of fewer than 16,384
 *              objects run the FP32-accurate similarity in the same batch,
 *              their lists final without a rescore: re-reading the FP32
 *              descriptors of the candidates costs more there than the
 *              FP32-accurate GEMM over the whole scene.  A batch of such
 *              scenes only runs as a FARM_PREC_FP32 batch.
 *   flags      FARM_PTR_DEVICE: tgt_emb and c_emb are device pointers (the
 *              other arrays are always host memory).
 *              FARM_GRAPH: the batch's kernels (row normalisation,
 *              similarity, rank selection, rescore, relations and composite)
 *              run as a CUDA graph; the copies of the batch's metadata and
 *              piece tables are issued on the stream before each replay.  Graphs are cached by the
 *              batch's shape: precision, n_q, n_c, and the scenes in order of
 *              first use with each one's query and constraint counts, and, for
 *              device embeddings, their addresses.  A batch of a cached shape
 *              replays the graph; the host still plans each call (query order,
 *              metadata).  Host embeddings are copied into library buffers
 *              before the graph runs; device embeddings are read in place, so
 *              a caller that reuses its buffers replays without copies.
 *              Re-uploading a scene, changing the prefilter weights or growing
 *              a work buffer starts new captures.  At most 8 graphs are kept
 *              (least recently used go).
 *              FARM_UNFUSED / FARM_FUSED: whether the rows of a scene
 *              select their ranks from the whole similarity block written
 *              to memory (as FP8 and the learned path always do) or by the
 *              fused selection, which writes only a sample of each row
 *              (every s-th tile of 256 objects), takes the row's threshold
 *              from the sample's ranks and has the similarity kernel keep
 *              only the entries reaching it (rows whose kept entries
 *              overflow their buffer are recomputed exactly).  FARM_FUSED
 *              fuses every scene of a FARM_PREC_FP32 or FARM_PREC_BF16
 *              batch, FARM_UNFUSED none; by default FARM_PREC_FP32 fuses
 *              the scenes whose sample holds at least 16 times the target
 *              list (about 12,000 objects and more) and FARM_PREC_BF16
 *              none, the faster choices measured.  All give the same ranks.
 *   batch_handle  receives the handle that farm_topk takes
 * Only target candidates whose rank r can still place them in the top k_max
 * are scored: a candidate scores at most 1/(mu + r) while k_max objects score
 * at least (1 - w) * class_mis / (mu + k_max), so candidates of rank above
 * R = floor((mu + k_max) / ((1 - w) * class_mis) - mu) + 1 (95 with the default
 * single-precision constants: 0.3f is slightly above 0.3)
 * cannot enter the result.  The result is the same as scoring every object.
 * A new farm_query_batch call invalidates the previous handle.
 */
farm_status farm_query_batch(farm_ctx *ctx, int64_t n_q, const int32_t *scene_of_q,
                             const float *tgt_emb, const int32_t *tgt_cls, const int32_t *c_off,
                             const int32_t *c_pred, const float *c_emb, int32_t precision,
                             uint32_t flags, uint64_t *batch_handle);

/*
 * Several retrieval channels (App. D.2 step 3).  The paper ranks the whole
 * candidate pool once per query channel -- four channels over three
 * embedding spaces of every object (caption text, two image embeddings) --
 * and takes the reciprocal-rank fusion
 *   F(j) = sum_c w_c / (mu + rank_c(j))
 * as the target similarity, s_sem = cf * F; landmark variables are retrieved
 * the same way (L_i = the K_a objects of largest fused landmark score) and
 * the Closest / Farthest candidate set is the k_closest objects of largest F.
 * Everything after that (relations, binding, composite, TopK) is as for
 * farm_query_batch.
 *
 * farm_memory_add_space: stores descriptor space `space` (1 ..
 * FARM_MAX_SPACES - 1) of an uploaded scene: desc [n, dim] FP32 rows of the
 * scene's n objects in the same order (host, or device with
 * FARM_PTR_DEVICE), unit-normalised on upload; space 0 is the descriptor
 * array of farm_memory_upload.  Replaces an earlier upload of that space;
 * re-uploading the scene drops its extra spaces.  Rows with zero or
 * non-finite norm: FARM_EINVAL (host input) or reported by the next
 * synchronising call (device input).
 */
#define FARM_MAX_SPACES 4
#define FARM_MAX_CHANNELS 4
farm_status farm_memory_add_space(farm_ctx *ctx, int32_t scene_id, int32_t space, int32_t dim, const float *desc,
                                  uint32_t flags);

typedef struct {
    int32_t space;   /* descriptor space the channel is scored in */
    float weight;    /* its reciprocal-rank-fusion weight w_c (> 0) */
} farm_channel;

/*
 * A batch of n_q queries against one scene over n_ch channels (1 ..
 * FARM_MAX_CHANNELS), FP32-accurate similarity (as FARM_PREC_FP32):
 *   ch        [n_ch]  the channels
 *   tgt_emb   the target's channel embeddings, channel after channel: block
 *             c is [n_q, dim of ch[c].space] FP32
 *   tgt_cls, c_off, c_pred  as farm_query_batch (host)
 *   c_emb     the landmarks' channel embeddings, channel after channel:
 *             block c is [n_c, dim of ch[c].space] FP32
 *   flags     FARM_PTR_DEVICE: tgt_emb and c_emb are device pointers
 *             (FARM_GRAPH is not supported here: FARM_EINVAL)
 * Each channel keeps its R_t best objects per target row and R_l per landmark
 * row, with R_t and R_l chosen so that no object outside every channel's list
 * can reach the result: an unlisted object fuses to at most
 * W / (mu + R + 1) (W the sum of the weights), below the k_max-th composite
 * and the k_closest-th / K_a-th fused score.  Listed objects that could reach
 * the result get their exact rank in the channels that did not list them
 * (by counting over that channel's similarity row), so the result equals
 * scoring every object.  Weights so uneven that R_t would exceed 512 (or R_l
 * 256) are rejected (FARM_EINVAL).  A query whose objects that can still
 * reach its TopK exceed 512 is reported by the next synchronising call
 * (FARM_EINVAL).  The similarity block of every channel is kept until the
 * fusion: n_ch x (n_q + n_c) x n x 4 bytes of device memory (at most 32 GiB
 * per call, else FARM_EINVAL; split the batch).  farm_topk reads the result
 * as for farm_query_batch; a new batch of either kind invalidates the handle.
 */
farm_status farm_query_batch_rrf(farm_ctx *ctx, int32_t scene_id, int64_t n_q, int32_t n_ch,
                                 const farm_channel *ch, const float *tgt_emb, const int32_t *tgt_cls,
                                 const int32_t *c_off, const int32_t *c_pred, const float *c_emb, uint32_t flags,
                                 uint64_t *batch_handle);

/*
 * Mapping-side association (App. D.1 steps 3-5): a batch of n_det detections
 * against the memory's n_ent entities, each a 3D Gaussian -- mean [3, n] SoA
 * and covariance packed [6, n] SoA (xx, xy, xz, yy, yz, zz) -- with an
 * appearance feature ([n, F] row-major FP32); entities also carry a weight
 * ent_w (the detections fused so far, finite and >= 0) and an active flag.
 *  - neighbour search: for each detection, the active entities whose feature
 *    cosine is >= tau_f (computed as the FP32-accurate similarity), then the
 *    Hellinger distance of the two Gaussians, keeping those with H <= h_max
 *    sorted by (H, index): match_cnt [n_det] (all within the budget),
 *    match_idx / match_h [n_det, max_m] (the first max_m; -1 after);
 *  - correspondence: the connected components of the graph joining every
 *    detection to its (at most max_m) matches (union-find); in a component
 *    with entities the entity of largest weight (lower index on ties) wins
 *    and the others merge into it; a detection without a match starts a new
 *    entity;
 *  - fusion: the winner absorbs its component by the sufficient-statistics
 *    merge (w = sum w_i, M1 = sum w_i mu_i, M2 = sum w_i (S_i + mu_i mu_i'),
 *    mu = M1 / w, S = M2 / w - mu mu'; detections weigh 1), and its feature
 *    becomes the w-weighted average.
 * Outputs over T = n_ent + n_det slots (the entities, then one per
 * detection): parent [T] (the slot each merges into; itself for a winner, an
 * untouched entity or a new entity), out_w [T] (0 for slots merged away),
 * out_mu [3, T], out_cov [6, T], out_feat [T, F] (zero for merged slots).
 * 1 <= max_m <= 64, F <= 8192, tau_f in [-1, 1], h_max in [0, 1].  All
 * arrays host memory, or all device memory with FARM_PTR_DEVICE.  With host
 * arrays the call synchronises and reports device-side errors; with device
 * arrays its work is enqueued on the context's stream (errors come with the
 * next synchronising call).  A detection with more than 1,024 entities
 * within the budget is reported as FARM_EINVAL.
 */
farm_status farm_associate(farm_ctx *ctx, int64_t n_ent, const float *ent_mu, const float *ent_cov,
                           const float *ent_feat, const int32_t *ent_active, const float *ent_w, int64_t n_det,
                           const float *det_mu, const float *det_cov, const float *det_feat, int32_t F, float tau_f,
                           float h_max, int32_t max_m, int32_t *match_cnt, int32_t *match_idx, float *match_h,
                           int32_t *parent, float *out_w, float *out_mu, float *out_cov, float *out_feat,
                           uint32_t flags);

/*
 * Writes the TopK of every query of a batch, the ScoredCandidate records of
 * App. D.2 step 7: for query q and rank j < k,
 *   out_idx   [n_q, k]     int32 object index, best first (lower index on ties)
 *   out_score [n_q, k]     FP32 composite score s
 *   out_pred  [n_q, k, 4]  FP32 per-constraint score t_i (-1 beyond the
 *                          query's constraints; NULL to skip)
 *   out_anchor[n_q, k, 4]  int32 bound landmark object (-1 without a witness
 *                          or beyond the constraints; NULL to skip)
 * 1 <= k <= k_max and k <= n of every scene in the batch.
 * flags: FARM_PTR_DEVICE when the outputs are device pointers (no
 * synchronisation); otherwise the call synchronises and reports device-side
 * input errors, unless FARM_ASYNC is given: then the copies into the host
 * outputs are only enqueued (from pinned memory they overlap the host's next
 * calls; from pageable memory CUDA copies synchronously anyway), the outputs
 * are valid after the next farm_sync, which also reports device-side errors,
 * and a following batch may already be enqueued meanwhile -- its host input
 * copies then overlap this batch's kernels.
 */
farm_status farm_topk(farm_ctx *ctx, uint64_t batch_handle, int32_t k, int32_t *out_idx,
                      float *out_score, float *out_pred, int32_t *out_anchor, uint32_t flags);

/* Synchronises the context's stream and reports device-side errors. */
farm_status farm_sync(farm_ctx *ctx);

/*
 * Rows that the rank selection of the tensor-core paths handed to an exact
 * fallback since the context was created (or last reset).  The thresholded
 * select takes its threshold from per-tile maxima of the stored similarity
 * values; a row whose entries at or above it overflow the candidate buffer
 * (many exact ties, or top-ranked objects crowded into a few 256-object
 * tiles) is selected by a slower exact radix select.  The fused selection
 * takes its threshold from the row's sample; a row whose kept entries
 * overflow its buffer (a sample unlike the rest of the row, e.g. objects
 * ordered by class) is recomputed over all objects on the CUDA cores and
 * selected exactly.  Results are exact either way.  Synchronises the
 * context's stream; reset != 0 zeroes the count afterwards.
 */
farm_status farm_select_fallbacks(farm_ctx *ctx, int64_t *rows_out, int32_t reset);

/*
 * The tensor-core similarity kernel comes in three tile configurations
 * ("variants": 0 = 128 query rows x 256 objects per CTA; 1 = 128 x 128 per
 * CTA; 2 = 256 x 256 tiles computed by a pair of CTAs with two-SM MMAs).
 * All compute each cosine with the same sequence of products, so they give
 * bitwise identical results.  The first farm_query_batch of each class of
 * batch (similarity mode, and the powers of two of its total rows and of its
 * mean objects per row) times every variant on its first similarity block and
 * keeps the fastest for the context.
 *
 * farm_sim_tuning: the decisions so far, up to cap records of four int32:
 * mode (0 = FP32-accurate, 1 = BF16 and the learned prefilter, 2 = FP8; plus
 * 10 for batches with the fused selection, whose two launches are timed
 * together; plus 20 for BF16 / FP8 batches whose small scenes run the
 * FP32-accurate similarity, the two launches timed together),
 * log2 of the rows, log2 of the mean objects per row, chosen variant.
 * *count receives the number of decisions.
 */
farm_status farm_sim_tuning(farm_ctx *ctx, int32_t *entries, int32_t cap, int32_t *count);

/*
 * Pins every later batch of the context to one tile variant (0 .. 2), or,
 * with -1, returns to the autotuner: for reproducible configurations, and for
 * runs under a profiler, whose serialisation distorts the autotuner's timings.
 */
farm_status farm_sim_variant_pin(farm_ctx *ctx, int32_t variant);

/*
 * Cosines as farm_similarity (FARM_PREC_FP32, FARM_PREC_BF16 or FARM_PREC_FP8),
 * computed by the given tile variant (0 .. 2), for checking the variants
 * against one another.
 */
farm_status farm_similarity_variant(farm_ctx *ctx, int32_t scene_id, int64_t n_rows, const float *emb,
                                    int32_t precision, int32_t variant, float *out, uint32_t flags);

/*
 * Frees an uploaded scene's device memory (after the context's queued work);
 * the scene id may then be uploaded again.  FARM_EINVAL for an id that holds
 * no scene.  Synchronises.
 */
farm_status farm_memory_release(farm_ctx *ctx, int32_t scene_id);

/*
 * Object count n and descriptor length dim of an uploaded scene, for sizing
 * the output of farm_similarity (n_rows x n floats).  Either pointer may be
 * NULL.  FARM_EINVAL for a scene id that holds no scene.
 */
farm_status farm_scene_info(farm_ctx *ctx, int32_t scene_id, int64_t *n, int32_t *dim);

/*
 * Cosine similarity of n_rows embeddings against every object of a scene,
 * computed by the kernels of `precision` (App. D.2 step 3; FARM_PREC_BF16 and
 * FARM_PREC_FP8 return the reduced-precision stage's approximate cosines):
 *   emb [n_rows, dim] FP32, out [n_rows, n] FP32 (host or device per flags).
 */
farm_status farm_similarity(farm_ctx *ctx, int32_t scene_id, int64_t n_rows, const float *emb,
                            int32_t precision, float *out, uint32_t flags);

/*
 * The ranked candidate lists of the last batch (host outputs, synchronises):
 *   tgt_idx [n_q, r_tgt]   target candidates in rank order (rank 1 first)
 *   lm_idx  [n_c, k_lm]    each constraint's landmark candidates in rank order
 * *r_tgt_out and *k_lm_out receive the list lengths (taken per batch as
 * min(R, n) and min(k_anchor, n) over its scenes; shorter lists are padded
 * with -1).  Any pointer may be NULL.
 */
farm_status farm_candidates(farm_ctx *ctx, uint64_t batch_handle, int32_t *tgt_idx,
                            int32_t *lm_idx, int32_t *r_tgt_out, int32_t *k_lm_out);

/*
 * Ranked object lists for embedding rows, without allocating device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate GPU memory while serving queries: a process on a robot
 * whose GPU memory budget is fixed at start-up (mapping and model workers own
 * the rest of it), or a real-time loop that must not call cudaMalloc/cudaFree
 * because they may synchronise the device and take unbounded time.
 * farm_query_batch grows its workspace on demand; this call does not.
 *
 * For each of n_rows embeddings (device pointer emb, [n_rows, dim] FP32, dim
 * of the scene) it writes the r objects of scene `scene_id` with the largest
 * cosine, in rank order (larger cosine first, lower index on ties), to
 * out_idx ([n_rows, r] int32, device) and their cosines to out_cos
 * ([n_rows, r] FP32, device, may be NULL), using the similarity arithmetic of
 * `precision` (FARM_PREC_FP32 or FARM_PREC_FP32_SIMT).  1 <= r <= min(512, n).
 *
 * Memory: every intermediate array (normalised rows and the
 * n_rows x round_up(n, 32) similarity block) lives in one statically
 * allocated device array of FARM_NOALLOC_SCRATCH_BYTES per GPU.  farm_create
 * looks up its device address (cudaGetSymbolAddress, with the context's
 * device current), which loads it: the array's memory is taken when the
 * first context on a device is created and held until the process exits.
 * The call itself allocates, frees and loads nothing.  Sizes that do not fit
 * return FARM_EINVAL (split the rows into smaller calls).  All calls share
 * the array and it keeps the last call's contents (nothing in it needs to
 * start at zero): calls whose work overlaps on the GPU -- on different
 * streams or contexts of the same device -- race on it and must be
 * serialised by the caller.
 * Work is enqueued on the context's stream; nothing is synchronised.  A zero
 * or non-finite row is reported by the next farm_sync as FARM_EINVAL.
 */
#define FARM_NOALLOC_SCRATCH_BYTES (32u << 20)
farm_status farm_rank_rows_noalloc(farm_ctx *ctx, int32_t scene_id, int64_t n_rows, const float *emb,
                                   int32_t r, int32_t precision, int32_t *out_idx, float *out_cos);

/*
 * Learned prefilter.  A small network f(x) = normalize(W2 gelu(W1 x + b1) + b2)
 * (x: a unit row of length dim; W1: hidden x dim; W2: out_dim x hidden; GELU
 * in its erf form) compresses descriptors and query rows to out_dim values.
 * With FARM_PREC_LEARNED, farm_query_batch ranks objects by f(q).f(d) (BF16
 * tensor-core products), keeps the best 512 per target row (128 per landmark
 * row) and re-scores them with exact FP32 cosines before ranking; the
 * full-descriptor paths are its fallback and the judge of its recall.
 * Requirements: 1 <= dim <= 8192, hidden in [64, 4096] and out_dim in
 * [64, 1024], both multiples of 64; dim equal to the scenes' dim.  The paper
 * ranks with full embeddings (App. D.2 step 3); this compression is an
 * addition of this library.
 *
 * farm_mlp_set: install weights (host FP32; W1 [hidden, dim], b1 [hidden],
 *   W2 [out_dim, hidden], b2 [out_dim], row-major).  Scenes' cached
 *   embeddings are recomputed on their next learned query.
 * farm_mlp_get: copy the current weights out (any pointer may be NULL).
 * farm_mlp_loss_grad: for n_pairs (query row xq[i], descriptor xd[i], target
 *   y[i], weight w[i] (NULL: 1)) rows used as given, writes the loss
 *   L = sum_i w_i (f(xq_i).f(xd_i) - y_i)^2 / sum_i w_i and its gradient with
 *   respect to [W1 | b1 | W2 | b2] (grad, hidden*dim + hidden + out_dim*hidden
 *   + out_dim floats; NULL to skip), in the arithmetic of `precision`:
 *   FARM_PREC_FP32_SIMT (FP32 on the CUDA cores, the reference) or
 *   FARM_PREC_BF16 (the training step's: inputs, weights and activations
 *   rounded to BF16 for the tensor-core contractions, FP32 accumulation and
 *   elementwise steps).  Host pointers; synchronises.
 * farm_mlp_train: minimises that loss with Adam (lr, betas 0.9/0.999) over
 *   `epochs` passes of mini-batches of `batch` pairs, shuffled each epoch by
 *   SplitMix64 from `seed`, every contraction on the BF16 tensor cores (FP32
 *   master weights).  Pair i joins row pair_row[i] of `rows` ([n_rows, dim],
 *   host, normalised on the GPU) with object pair_obj[i] of scene
 *   scene_ids[pair_scene[i]] (pair_scene may be NULL when n_scenes == 1).
 *   loss_out[epoch] (nullable) receives the mean batch loss.  Starts from the
 *   installed weights.  Synchronises.
 * farm_mlp_embed: f of n_rows host rows x (normalised first) into host
 *   out [n_rows, out_dim], with FP32 CUDA-core kernels (FARM_PREC_FP32_SIMT)
 *   or the BF16 tensor-core inference path (FARM_PREC_BF16).
 */
farm_status farm_mlp_set(farm_ctx *ctx, int32_t dim, int32_t hidden, int32_t out_dim, const float *W1,
                         const float *b1, const float *W2, const float *b2);
farm_status farm_mlp_get(farm_ctx *ctx, float *W1, float *b1, float *W2, float *b2);
farm_status farm_mlp_loss_grad(farm_ctx *ctx, int64_t n_pairs, const float *xq, const float *xd, const float *y,
                               const float *w, int32_t precision, float *loss, float *grad);
farm_status farm_mlp_train(farm_ctx *ctx, int32_t n_scenes, const int32_t *scene_ids, int64_t n_rows,
                           const float *rows, int64_t n_pairs, const int32_t *pair_row, const int32_t *pair_scene,
                           const int32_t *pair_obj, const float *y, const float *w, int32_t epochs, int32_t batch,
                           float lr, uint64_t seed, float *loss_out);
farm_status farm_mlp_embed(farm_ctx *ctx, int64_t n_rows, const float *x, int32_t precision, float *out);

/*
 * Stage timing.  With profiling on, every farm_query_batch records CUDA events
 * around its stages on the context stream.  farm_stage_times synchronises and
 * writes the accumulated milliseconds of FARM_N_STAGES stages (prepare,
 * similarity, select, compose) to ms_out, the number of kernels the context
 * launched to *launches_out, and with reset != 0 clears both.
 */
#define FARM_N_STAGES 4
farm_status farm_set_profiling(farm_ctx *ctx, int32_t on);
farm_status farm_stage_times(farm_ctx *ctx, float *ms_out, int64_t *launches_out, int32_t reset);

/* One-line description of the last error on this context ("" if none). */
const char *farm_last_error(farm_ctx *ctx);

/* Library version string. */
const char *farm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FARM_H */
