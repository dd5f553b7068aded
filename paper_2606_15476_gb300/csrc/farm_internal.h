// farm_internal.h -- device data layout and kernel entry points shared by the
// translation units of libfarm (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/farm.h"

namespace farm {

// Descriptor rows are zero-padded to a multiple of this many elements so
// that every row starts on a 256-byte boundary for the tensor-memory-access
// (TMA) loads of the tensor-core kernels; zero padding leaves dot products
// unchanged.
constexpr int kDimAlign = 64;

// Largest target-candidate list (ranks kept per target row) and landmark
// list (K_a) the select and compose kernels handle.
constexpr int kMaxTargetCands = 512;
constexpr int kMaxAnchorCands = 256;

// Per stored view, the compose kernel reads 8 floats: camera origin (3),
// unit viewing direction f (3) and unit right vector r = f x z_up (2; its z
// component is 0).  A view whose direction is zero or vertical has f = 0,
// which no depth test passes (z_min >= 0).
constexpr int kViewStride = 12;

// Bits of the device error word.
constexpr int kErrBadRow = 1;        // zero or non-finite embedding row
constexpr int kErrBadDesc = 2;       // zero or non-finite descriptor row
constexpr int kErrTimeout = 4;       // a bounded wait gave up
constexpr int kErrPieceTable = 8;    // a similarity piece carried a misaligned tensor-map pointer
constexpr int kErrFusedOverflow = 16; // a query of a fused batch kept more candidates than its list holds
constexpr int kErrAssocOverflow = 32; // a detection had more matches within the budget than the search holds

// A further descriptor space of a scene (farm_memory_add_space): the FP16
// split of its unit rows, as desc_hi / desc_lo below.
struct SpaceDesc {
    int32_t dim = 0, dim_pad = 0;
    uint16_t *hi = nullptr;      // [n, dim_pad]
    uint16_t *lo = nullptr;      // [n, dim_pad]
};

struct Scene {
    bool present = false;
    int64_t n = 0;
    int32_t dim = 0;
    int32_t dim_pad = 0;
    int32_t n_views = 0;
    float *desc32 = nullptr;    // [n, dim_pad] unit rows, FP32
    uint16_t *desc_hi = nullptr;    // [n, dim_pad] FP16 high part of desc32
    uint16_t *desc_lo = nullptr;    // [n, dim_pad] FP16 of 2^11 (desc32 - desc_hi)
    uint16_t *desc_bf16 = nullptr;  // [n, dim_pad] BF16 of desc32
    uint8_t *desc_fp8 = nullptr;    // [n, dim_pad] E4M3 of desc32 / desc_scale
    float *desc_scale = nullptr;    // [n] per-row FP8 scale
    uint16_t *comp = nullptr;       // [n, P] BF16 learned embeddings f(d) (cache)
    uint64_t comp_version = 0;      // Mlp::version the cache was computed with
    int32_t *cls = nullptr;     // [n]
    float *pos = nullptr;       // [3, n] centres (SoA)
    float *size = nullptr;      // [3, n]
    float *views = nullptr;     // [n, n_views, kViewStride]
    SpaceDesc spaces[FARM_MAX_SPACES];   // [1 ..]: further descriptor spaces (space 0 is desc_hi / desc_lo)
};

enum Buf {
    B_RAW = 0,      // raw embedding rows as given [n_q + n_c, dim]
    B_Q32,          // normalised rows [rows, dim_pad]
    B_QHI,          // FP16 high part
    B_QLO,          // FP16 scaled residual
    B_QBF,          // BF16 rows
    B_SIM,          // similarity block [rows_chunk, n]
    B_ROWMAP,       // int32 [n_q + n_c] planned row of each source row
    B_PERM,         // int32 [n_q] planned position of each caller query
    B_TSEL_IDX,     // int32 [n_q, r_tgt] target candidates
    B_TSEL_COS,     // float [n_q, r_tgt]
    B_LSEL_IDX,     // int32 [n_c, k_lm] landmark candidates
    B_QMETA,        // int32 [n_q, 8] per-query metadata
    B_OUT_IDX,      // int32 [n_q, r_tgt] composed candidates, best first
    B_OUT_SCORE,    // float [n_q, r_tgt]
    B_OUT_T,        // float [n_q, r_tgt, 4]
    B_OUT_ANCHOR,   // int32 [n_q, r_tgt, 4]
    B_TOPK,         // int32/float [n_q, k, 10] TopK staging for host outputs
    B_BSEL_T,       // int32 [n_q, C_t] BF16-stage target candidates (before FP32 rescore)
    B_BSEL_L,       // int32 [n_c, C_l] BF16-stage landmark candidates
    B_BSEL_TV,      // float [n_q, C_t] their reduced-precision values
    B_BSEL_LV,      // float [n_c, C_l]
    B_QF8,          // uint8 [rows, dim_pad] E4M3 rows
    B_QSCALE,       // float [rows] their scales
    B_QCOMP,        // bf16 [rows, P] learned embeddings of the rows
    B_MLP_H,        // float [chunk, H] pre-activations (inference)
    B_MLP_A,        // float [chunk, H] activations
    B_MLP_AB,       // bf16 [chunk, H]
    B_MLP_Z,        // float [chunk, P]
    B_MLP_E,        // float [chunk, P]
    B_PIECES,       // Piece tables of the batch's grouped launches
    B_CHUNK_IDX,    // int32 chunk lists of long rows (select, then merge)
    B_CHUNK_VAL,    // float their values
    B_TOPS,         // float per-row group maxima of the tensor-core similarity (thresholded select)
    B_VARIANT,      // one piece and its tensor maps (farm_similarity_variant)
    B_MC_SIM,       // float [n_ch, rows, ld] every channel's similarity block (fused batches)
    B_MC_TOPS,      // float [n_ch, rows, group_stride] their group maxima
    B_MC_TLIST,     // int32 [n_ch, n_q, R_t] per-channel target lists
    B_MC_LLIST,     // int32 [n_ch, n_c, R_l] per-channel landmark lists
    B_MC_FUSED,     // float [n_q, RF] fused scores of the kept target candidates
    B_SELLIST,      // int32 [1 + rows] rows the warp-level select hands to the block-level one
    B_ASSOC,        // farm_associate: its inputs' copies, operand rows, similarity block and scratch
    B_LSEL_COS,     // float [n_c, k_lm] landmark list values (fused selection)
    B_FUSE_TAU,     // uint32 [rows] per operand row: the fused selection's threshold key
    B_FUSE_CNT,     // int32 [rows] its appended candidate count
    B_FUSE_CAND,    // uint64 [rows, cap] its candidate words
    B_FUSE_OVF,     // int32 [2 + 2 rows] overflow count, long-row count, overflowed launch rows, long launch rows
    B_FUSE_SLAB,    // float [blocks, n] the exact fallback's similarity rows
    B_RAW_PIPE,     // farm_query_batch's host rows: two slots, each [n_q + n_c, dim] (copy stream)
    B_COUNT
};

struct Workspace {
    // grow-only device buffers, one per Buf (bytes recorded alongside)
    void *ptr[B_COUNT] = {};
    size_t bytes[B_COUNT] = {};
};

// Per-query metadata row (int32 x 8) consumed by the compose kernel.
enum QMeta {
    QM_SCENE = 0, QM_CLS, QM_M, QM_C0, QM_PRED01, QM_PRED23, QM_R, QM_KLM
};

// The learned prefilter f(x) = normalize(W2 gelu(W1 x + b1) + b2).
struct Mlp {
    bool set = false;
    int32_t D = 0, H = 0, P = 0, D_pad = 0;
    float *params = nullptr;      // FP32 [W1 (H x D) | b1 (H) | W2 (P x H) | b2 (P)]
    uint16_t *w1b = nullptr;      // BF16 [H, D_pad], zero padded
    uint16_t *w2b = nullptr;      // BF16 [P, H]
    uint16_t *w2t = nullptr;      // BF16 [H, P] (W2 transposed, for the backward pass)
    uint64_t version = 0;         // bumped whenever the weights change
    int64_t count() const { return (int64_t)H * D + H + (int64_t)P * H + P; }
    float *W1() const { return params; }
    float *b1() const { return params + (int64_t)H * D; }
    float *W2() const { return b1() + H; }
    float *b2() const { return W2() + (int64_t)P * H; }
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    farm_params params{};
    std::string err;
    std::vector<Scene> scenes;
    Workspace ws;
    int32_t *d_err = nullptr;     // device error word
    uint64_t ws_gen = 0;          // bumped whenever a workspace buffer moves
    uint64_t scene_gen = 0;       // bumped on every scene upload
    std::map<int64_t, int> tuned; // similarity class -> fastest tile variant (autotuner)
    int pinned_variant = -1;      // >= 0: every grouped similarity launch uses this variant
    int32_t *d_fallback = nullptr;  // rows the thresholded select handed to its exact fallback
    int32_t *h_err = nullptr;     // pinned host mirror
    // batch state
    uint64_t batch_gen = 0;
    bool batch_valid = false;
    int64_t batch_nq = 0;
    int64_t batch_nc = 0;
    int32_t batch_rtgt = 0;       // candidate list length (stride)
    int32_t batch_klm = 0;        // landmark list length (stride)
    int32_t batch_min_n = 0;      // smallest scene size in the batch
    // profiling
    bool profiling = false;
    double stage_ms[FARM_N_STAGES] = {};
    int64_t launches = 0;
    int num_sms = 0;
    Mlp mlp;
};

// ---- learned prefilter (k_mlp.cu) ----
cudaError_t mlp_gemm(bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda, const float *B,
                     int ldb, float beta, float *C, int ldc, cudaStream_t s);
cudaError_t mlp_bias_gelu(float *h, const float *b, float *a, int64_t rows, int cols, cudaStream_t s,
                          uint16_t *ab = nullptr);
// BF16 rows gathered from several tables: dst[r] = base[sel[r]] + idx[r] * lds
// (sel null: base[0]); cols, lds, ldd multiples of 8, dst 16-byte aligned.
cudaError_t mlp_gather_rows_bf16(const uint16_t *const *base, const int32_t *sel, const int32_t *idx, int64_t lds,
                                 int64_t rows, int cols, uint16_t *dst, int64_t ldd, cudaStream_t s);
// dst[c * ldd + col0 + r] = bf16(src[r * lds + c]) (src FP32 src32, or BF16 src16).
cudaError_t mlp_transpose_bf16(const float *src32, const uint16_t *src16, int64_t lds, int64_t rows, int cols,
                               uint16_t *dst, int64_t ldd, int64_t col0, cudaStream_t s);
// BF16 copy of a row-major FP32 [rows, cols] matrix with rows zero-padded to ldd.
cudaError_t mlp_to_bf16_padded(const float *src, int64_t rows, int cols, uint16_t *dst, int ldd, cudaStream_t s);
cudaError_t mlp_bias_normalize(float *z, const float *b, float *e, float *norm, int64_t rows, int cols,
                               cudaStream_t s);
cudaError_t mlp_pair_loss(const float *eq, const float *ed, const float *y, const float *w, float wsum, int64_t pairs,
                          int cols, float *deq, float *ded, float *loss, cudaStream_t s);
cudaError_t mlp_normalize_backward(const float *e, const float *norm, float *de, int64_t rows, int cols,
                                   cudaStream_t s);
cudaError_t mlp_gelu_backward(const float *h, float *da, int64_t count, cudaStream_t s);
cudaError_t mlp_colsum(const float *x, int64_t rows, int cols, float *out, bool accumulate, cudaStream_t s);
cudaError_t mlp_gather_rows(const float *src, int lds, const int32_t *idx, int64_t rows, int cols, float *dst,
                            cudaStream_t s);
cudaError_t mlp_adam(float *p, const float *g, float *m, float *v, int64_t count, float lr, int t, cudaStream_t s);
cudaError_t mlp_to_bf16(const float *x, int64_t count, uint16_t *y, cudaStream_t s);

// Grow-only workspace buffer of the context (synchronises before a regrow).
cudaError_t ws_alloc(farm_ctx *ctx, Buf b, size_t bytes, void **out);

// Learned embeddings f(x) of BF16 unit rows xb [rows, D_pad] into BF16
// out [rows, P], on the tensor cores, in chunks (the prefilter's host code).
// Grow the prefilter's work buffers for embedding `rows` rows, so that
// learned_embed_rows then allocates nothing (required before graph capture).
cudaError_t learned_reserve(farm_ctx *ctx, int64_t rows);
cudaError_t learned_embed_rows(farm_ctx *ctx, const uint16_t *xb, int64_t rows, uint16_t *out);
// Recompute a scene's cached learned embeddings if the weights changed.
cudaError_t learned_refresh_scene(farm_ctx *ctx, int32_t scene_id);


// The internal state behind a public farm_ctx handle.
Ctx *ctx_of(farm_ctx *ctx);

// Device address of farm_rank_rows_noalloc's static scratch array for the
// current device `device`, resolved once (loads its module); farm_create calls it.
cudaError_t noalloc_setup(int device);
// Force-load the kernels farm_rank_rows_noalloc launches, so that its calls
// load no code (modules and functions load lazily on first use).
cudaError_t preload_prep();
cudaError_t preload_sim_simt();
cudaError_t preload_select_rows();
cudaError_t preload_sim_tc_f16x3();

// ---- kernel launchers (each returns cudaGetLastError() after launching) ----

// Unit-normalise `rows` rows of length dim into dst rows of length dim_pad
// (zero tail); optionally also write the FP16 split and BF16 copies.  Rows
// with zero or non-finite norm set err_bit in *err and are written as zeros.
// dst_rows: optional int32 [rows] scatter map (src row r goes to dst row dst_rows[r]).
// split >= 0: dst rows below split get only dst32 / dst_bf16, the others only
// the FP16 split (a reduced-precision batch whose last rows run FP32-accurate).
cudaError_t launch_normalize_rows(const float *src, const int32_t *dst_rows, int64_t rows,
                                  int32_t dim, int32_t dim_pad, float *dst32, uint16_t *dst_hi,
                                  uint16_t *dst_lo, uint16_t *dst_bf16, int32_t *err, int err_bit,
                                  cudaStream_t s, int64_t split = -1);

// E4M3 copy of unit rows with a per-row scale (max|x| / 448).
cudaError_t launch_quantize_fp8_rows(const float *src, int64_t rows, int32_t dim_pad, uint8_t *dst, float *scale,
                                     cudaStream_t s);

// Pre-compute the per-view record of kViewStride floats from SoA views and
// the objects' centres pos [3, n]: {ox, oy, oz, fx, fy, fz, rx, ry} (origin,
// unit forward, unit right in the ground plane), then the centre's depth Z_e
// and image coordinate u_e in that view, and two zeros.
cudaError_t launch_prepare_views(const float *views_soa, const float *pos, int64_t n, int32_t n_views,
                                 float *out, cudaStream_t s);

// S[r, j] = <Q[r], D[j]> for r < rows, j < n (FP32 FMA, CUDA cores).
cudaError_t launch_sim_simt(const float *q, const float *d, float *S, int64_t rows, int64_t n,
                            int32_t dim_pad, int64_t ld_s, cudaStream_t s);

// Tiles of the tensor-core similarity kernels: kSimTileM query rows per CTA;
// a tile configuration ("variant") fixes the tile width and whether two CTAs
// compute one tile together:
//   0: 128 x 256 tiles, one CTA each;  1: 128 x 128, one CTA each;
//   2: 256 x 256 tiles, a CTA pair with two-SM MMAs.
// Every variant computes each output with the same K order, so they give
// bitwise identical results; the planner's autotuner picks the fastest.
constexpr int kSimTileM = 128;
constexpr int kSimVariants = 3;
constexpr int kSimPairVariant = 2;      // the single-problem launches use the CTA pairs
inline int sim_variant_bn(int v) { return v == 1 ? 128 : 256; }
inline int sim_variant_cluster(int v) { return v == 2 ? 2 : 1; }
enum SimMode { kSimF16x3 = 0, kSimBf16 = 1, kSimFp8 = 2 };

// Group maxima: with a non-null `tops` the similarity epilogue also writes,
// per row, the maximum of every group of 2^gshift consecutive objects
// (gshift 5: groups of 32; 3: groups of 8, for small scenes; -inf for
// positions past the row end), group_stride(n, gshift) floats per row,
// 16-byte aligned.  The epilogue writes the groups of whole column tiles, so
// a row holds every group of ceil(n / 256) tiles of 256 objects (the widest
// tile variant).  They are entries of the row, so their R-th largest value
// bounds the row's R-th largest from below (the thresholded select uses it).
__host__ __device__ constexpr int64_t group_count(int64_t n, int gshift)
{
    return (n + (int64_t(1) << gshift) - 1) >> gshift;
}
__host__ __device__ constexpr int64_t group_stride(int64_t n, int gshift)
{
    return (n + 255) / 256 * (256 >> gshift);
}
constexpr int kGroupShiftSmall = 3;     // scenes of fewer than kSmallScene objects
constexpr int kGroupShift = 5;
constexpr int64_t kSmallScene = 8192;
inline int group_shift_for(int64_t n) { return n < kSmallScene ? kGroupShiftSmall : kGroupShift; }
// Rows of at most this many objects may be selected by sorting every entry.
constexpr int kSelectSortAll = 2048;

// Column tiles of a similarity launch.  kColAll: every tile of the row.
// With a sampling stride s (in tiles of 256 objects):
//   kColSample: the sample tiles 0, s, 2s, ...; the block stores its values
//     compacted (the j-th sample tile at columns [256 j, 256 j + 256)), so a
//     row holds sample_width(n, s) valid entries;
//   kColRest:   every other tile; values are not stored but compared with the
//     row's threshold, and those reaching it are appended to the row's
//     candidate buffer (the fused rank selection).
enum ColMode { kColAll = 0, kColSample = 1, kColRest = 2 };
__host__ __device__ inline int64_t col_tiles(int64_t n, int bn, int mode, int s)
{
    const int64_t nt = (n + bn - 1) / bn;
    if (mode == kColAll) return nt;
    const int64_t ns = (nt + s - 1) / s;
    return mode == kColSample ? ns : nt - ns;
}
// The object tile of the launch's j-th column tile of a block.
__host__ __device__ inline int64_t col_tile_of(int64_t j, int mode, int s)
{
    return mode == kColAll ? j : (mode == kColSample ? j * s : j + j / (s - 1) + 1);
}
// Valid entries of a sample row: full sample tiles, then the last one, which may be the row's ragged tail.
__host__ __device__ inline int64_t sample_width(int64_t n, int s)
{
    const int64_t ns = col_tiles(n, 256, kColSample, s);
    const int64_t last = (ns - 1) * s * 256;
    return (ns - 1) * 256 + (n - last < 256 ? n - last : 256);
}

// One block of query rows against one scene in a grouped similarity launch.
struct GemmPiece {
    int64_t q_row0;          // first row of the block in the operand arrays
    int64_t s_off;           // S offset of the block's first row (floats; a multiple of 4); -1: values not stored
    int64_t tops_off;        // group-maxima offset of the first row (floats, a multiple of 8); -1: none
    const float *scale_d;    // FP8 per-object scales of the scene
    const void *bmap;        // the scene's two B tensor maps (device memory, 64-byte aligned)
    int32_t rows, n, ld;     // rows of the block, objects, leading dimension of S
    int32_t tile_begin;      // first cluster tile of the block in the launch
    int32_t gshift;          // group maxima over 2^gshift objects (of the stored columns)
    int32_t col_mode;        // ColMode
    int32_t col_stride;      // sampling stride s (kColSample / kColRest)
    int32_t n_store;         // valid stored columns: n, or sample_width(n, s) for kColSample
};
constexpr size_t kTensorMapBytes = 128;

// Cluster tiles of one block of `rows` rows against `n` objects in a variant
// (column mode and sampling stride as GemmPiece).
inline int64_t sim_cluster_tiles(int64_t rows, int64_t n, int variant, int mode = kColAll, int s = 0)
{
    const int64_t bn = sim_variant_bn(variant), cm = sim_variant_cluster(variant);
    const int64_t mt = (rows + kSimTileM - 1) / kSimTileM;
    return (mt + cm - 1) / cm * col_tiles(n, (int)bn, mode, s);
}

// The fused rank selection's outputs of a kColRest launch, indexed by operand
// row: each row's threshold (order-preserving key of its sample's R-th
// value), candidate count and buffer of `cap` candidate words
// (key << 32 | (2^32 - 1 - object index)).
struct FuseEmit {
    uint32_t *tau_key;
    int32_t *cnt;
    uint64_t *cand;
    int32_t cap;
};

// The two B tensor maps (hi / lo, or the one operand twice) of a scene's
// descriptor operand in `mode` for `variant`, written to host memory `out`
// (2 * kTensorMapBytes, 64-byte aligned).  False when the encoder fails.
bool sim_tc_encode_b(int mode, int variant, void *out, const void *d0, const void *d1, int64_t n, int32_t dim_pad);

// Grouped launch of `variant`: every piece of the device table `pieces`
// (n_pieces, ordered by tile_begin, numbered with the variant's tiles;
// total_tiles cluster tiles) against its scene, the query operands q0 / q1
// ([rows_total, dim_pad] in the mode's element type) and FP8 row scales
// scale_q.  S and tops are the bases the pieces' offsets refer to (tops
// nullable).
// With `emit` (its pieces in kColRest mode, or kColAll for two-pass rows;
// variants 0 and 2 only) the values reaching each row's threshold are
// appended to the rows' candidate buffers instead of stored.  A piece with
// s_off -1 stores no values, only its group maxima.
cudaError_t launch_sim_tc_grouped(int mode, int variant, const void *q0, const void *q1, int64_t rows_total,
                                  int32_t dim_pad, const GemmPiece *pieces, int32_t n_pieces, int64_t total_tiles,
                                  float *S, float *tops, const float *scale_q, int num_sms, int32_t *err,
                                  cudaStream_t s, const FuseEmit *emit = nullptr);

// One problem (rows x n, S leading dimension ld_s, group maxima at tops with
// group_stride(n) floats per row, nullable) on the tensor cores, variant 2 (CTA pairs).
// Three FP16 terms, hi*hi + 2^-11 (hi*lo + lo*hi), from the split the
// normalisation writes.
cudaError_t launch_sim_tc_f16x3(const uint16_t *q_hi, const uint16_t *q_lo, const uint16_t *d_hi,
                                const uint16_t *d_lo, float *S, int64_t rows, int64_t n, int32_t dim_pad,
                                int64_t ld_s, float *tops, int num_sms, int32_t *err, cudaStream_t s);
// BF16 operands, FP32 accumulation (first stage of the reduced-precision path).
cudaError_t launch_sim_tc_bf16(const uint16_t *q, const uint16_t *d, float *S, int64_t rows, int64_t n,
                               int32_t dim_pad, int64_t ld_s, float *tops, int num_sms, int32_t *err,
                               cudaStream_t s);
// FP8 E4M3 operands with per-row scales applied in the epilogue.
cudaError_t launch_sim_tc_fp8(const uint8_t *q, const float *scale_q, const uint8_t *d, const float *scale_d,
                              float *S, int64_t rows, int64_t n, int32_t dim_pad, int64_t ld_s, float *tops,
                              int num_sms, int32_t *err, cudaStream_t s);
bool sim_tc_available();

// Per row r of S (rows x n, leading dim ld_s): the R_r largest entries in
// (value desc, index asc) order, R_r = r < n_tgt_rows ? r_tgt : r_lm.
// Target rows write tsel_idx/tsel_cos[r * r_tgt + k]; landmark rows write
// lsel_idx[(r - n_tgt_rows) * k_lm + k].  Rows are numbered from row0 in the
// output arrays (tsel row = tsel_row0 + r, lsel row = lsel_row0 + r - n_tgt_rows).
cudaError_t launch_select_rows(const float *S, int64_t ld_s, int64_t n, int64_t rows,
                               int64_t n_tgt_rows, int32_t r_tgt, int32_t k_lm,
                               int32_t *tsel_idx, float *tsel_cos, int64_t tsel_row0,
                               int32_t stride_t, int32_t *lsel_idx, int64_t lsel_row0,
                               int32_t stride_l, cudaStream_t s);

// As launch_select_rows, also writing the landmark rows' values to lsel_cos
// (same layout as lsel_idx; nullable).
cudaError_t launch_select_rows_ex(const float *S, int64_t ld_s, int64_t n, int64_t rows, int64_t n_tgt_rows,
                                  int32_t r_tgt, int32_t k_lm, int32_t *tsel_idx, float *tsel_cos, int64_t tsel_row0,
                                  int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int64_t lsel_row0,
                                  int32_t stride_l, cudaStream_t s);

// One scene's block of rows within a grouped select / merge / rescore
// launch.  The block's rows are rows [row_begin, row_begin + rows) of the
// launch, stored at S + s_off with leading dimension ld; the first ntr are
// target rows.  Rows [0, th0) are selected by the shared-memory select
// (launch_select_grouped, blocks from block_begin), rows [th0, rows) by the
// thresholded select (launch_select_thresh, blocks from tblock_begin, group
// maxima at tops + tops_off, group_stride(n, gshift) floats per row).
// A row of the shared-memory select longer than its limit is selected in
// `chunks` column chunks of chunk_len entries, whose lists (tmp_stride
// entries each, rows at tmp + tmp_off + i * chunks * tmp_stride) are merged
// afterwards.  Pieces of a launch are ordered by every *_begin field.
struct Piece {
    const float *d32;       // the scene's unit FP32 descriptors (rescore)
    int64_t s_off;          // offset of the block's first row in S (floats)
    int64_t row_begin;      // first launch row of the block
    int64_t block_begin;    // first shared-memory-select block (th0 x chunks blocks)
    int64_t tblock_begin;   // first thresholded-select block (rows - th0 blocks)
    int64_t q_row0;         // row of the block's first row in the normalised operand rows
    int64_t t_row0;         // list row of the first target row
    int64_t l_row0;         // list row of the first landmark row
    int64_t tmp_off;        // chunk-list offset of the first row (entries)
    int64_t tops_off;       // group-maxima offset of the first row (floats)
    int32_t rows, ntr, n, ld;
    int32_t keep_t, keep_l; // list lengths the select keeps (R / K_a, or the rescore's C)
    int32_t R, klm;         // list lengths after a rescore
    int32_t chunks, chunk_len;
    int32_t th0;
    int32_t gshift;         // group maxima over 2^gshift objects (thresholded select)
    int32_t fkeep_t, fkeep_l; // fused selection: list lengths over the whole row (keep_t / keep_l: over its sample)
    int32_t n_obj;          // objects of the scene (n: the selected row length, its sample's when fused)
    int32_t fs;             // fused selection: the sampling stride (every fs-th tile of 256); 0: not fused;
                            // -1: two-pass (the group maxima of every tile, then every tile emits)
    int32_t exact;          // reduced-precision batch: 1 when the piece's scene runs the FP32-accurate
                            // similarity, its lists final (the rescore copies them)
};

// Grouped select over `pieces` (device; n_pieces entries) in one launch of
// total_blocks = sum of rows x chunks blocks.  Unchunked rows write their
// lists to (t|l)sel_(idx|cos) rows t_row0 + i / l_row0 + i - ntr (strides
// stride_t / stride_l; the cos pointers may be null); chunked rows write
// their chunk lists to tmp_(idx|val).  smem_n: the longest row or chunk of
// the launch, <= kSelectRowMax.  S + s_off and ld keep rows 16-byte aligned.
cudaError_t launch_select_grouped(const float *S, const Piece *pieces, int32_t n_pieces, int64_t total_blocks,
                                  int32_t smem_n, int32_t *tsel_idx, float *tsel_cos, int32_t stride_t,
                                  int32_t *lsel_idx, float *lsel_cos, int32_t stride_l, int32_t *tmp_idx,
                                  float *tmp_val, int32_t tmp_stride, cudaStream_t s);
// Merge the chunk lists of chunked rows into their final lists (one block per
// launch row; rows of unchunked pieces return at once).  smem_n: the longest
// merged list, chunks x tmp_stride, <= kSelectRowMax.
cudaError_t launch_merge_chunks(const Piece *pieces, int32_t n_pieces, int64_t total_rows, int32_t smem_n,
                                const int32_t *tmp_idx, const float *tmp_val, int32_t tmp_stride,
                                int32_t *tsel_idx, float *tsel_cos, int32_t stride_t, int32_t *lsel_idx,
                                float *lsel_cos, int32_t stride_l, cudaStream_t s);
// Thresholded select of rows [th0, rows) of every piece (one block per row,
// total_blocks of them), from the group maxima `tops` the tensor-core
// similarity kernel wrote; each row needs group_count(n, gshift) >= its list
// length, or n <= kSelectSortAll (then every entry is a candidate).
// max_union: the largest group count of the launch (at most 8,192 are used).  Rows
// whose candidates overflow fall back to an exact global-memory select and
// are counted in *n_fallback (device).  Outputs as launch_select_grouped.
// With row_list (device, total_blocks + 1 int32 of scratch) a warp-level
// select takes every row of a list of at most 256 entries and at most 1,024
// group maxima first (one warp per row, no block barriers) and hands the
// rest to the block-level select; both give the same lists.
cudaError_t launch_select_thresh(const float *S, const float *tops, const Piece *pieces, int32_t n_pieces,
                                 int64_t total_blocks, int32_t max_union, int32_t *tsel_idx, float *tsel_cos,
                                 int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l,
                                 int32_t *n_fallback, int32_t *row_list, cudaStream_t s);
// The fused rank selection (k_fuse_select.cu) over the launch rows of the
// fused pieces (fs > 0; the other pieces' rows are skipped), whose sample
// rows (sampling stride fs) the similarity kernel
// stored at S with their group maxima at tops (each piece's n, ld, s_off,
// tops_off and gshift describe the sample rows): sample_tau sets each row's
// threshold in `emit` (the R-th largest group maximum of its sample, R =
// fkeep) and appends the sample's entries reaching it; after the similarity
// kernel appended the other tiles' entries, fuse_final writes each row's
// final list of fkeep_t / fkeep_l entries from its buffer and records rows
// whose candidates overflowed (count in *n_overflow, launch rows in
// overflow_rows); rows of more than 1,024 candidates are listed in big_rows
// (count in *n_big) and merged by a second launch of one-warp blocks.  Both
// counts start at zero.
cudaError_t launch_fuse_sample_tau(const float *S, const float *tops, const Piece *pieces, int32_t n_pieces,
                                   int64_t total_rows, const FuseEmit &emit, cudaStream_t st);
// Two-pass rows (Piece::fs < 0): each row's threshold from the group maxima
// of its whole row (the similarity launch stored no values), at most gmax of
// them per row (<= kMaximaTauKeys), and a zero count.
constexpr int kMaximaTauKeys = 12288;
cudaError_t launch_fuse_maxima_tau(const float *tops, const Piece *pieces, int32_t n_pieces, int64_t total_rows,
                                   const FuseEmit &emit, int32_t gmax, cudaStream_t st);
cudaError_t launch_fuse_final(const Piece *pieces, int32_t n_pieces, int64_t total_rows, int32_t *tsel_idx,
                              float *tsel_cos, int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l,
                              const FuseEmit &emit, int32_t *n_overflow, int32_t *overflow_rows, int32_t *n_big,
                              int32_t *big_rows, int32_t max_keep, cudaStream_t st);

// The exact fallback of the fused selection for the rows fuse_final recorded
// (*n_overflow of them, launch rows in overflow_rows): a grid-stride loop of
// blocks, each computing a row's FP32 cosines against all n_obj objects on
// the CUDA cores (unit row from q32, or from the FP16 split q_hi + 2^-11 q_lo
// when q32 is null) into its slab of `slab` (slab_ld floats per block, >= the
// longest n_obj) and selecting the row's fkeep best exactly into its list.
// The number of such rows is added to *n_fallback (nullable).
cudaError_t launch_fuse_fallback(const Piece *pieces, int32_t n_pieces, const int32_t *n_overflow,
                                 const int32_t *overflow_rows, const float *q32, const uint16_t *q_hi,
                                 const uint16_t *q_lo, int32_t dim_pad, int32_t *tsel_idx, float *tsel_cos,
                                 int32_t stride_t, int32_t *lsel_idx, float *lsel_cos, int32_t stride_l, float *slab,
                                 int64_t slab_ld, int32_t blocks, int32_t *n_fallback, cudaStream_t st);
constexpr int kFuseFallbackBlocks = 64;

// The words a row can merge when no list is longer than max_keep; a row
// with more candidates is recomputed by the fallback.  Use it as FuseEmit::cap.
int fuse_merge_capacity(int32_t max_keep);

// The final lists of launch rows [row0, row0 + rows), rows of pieces whose
// scene ran the FP32-accurate similarity in a reduced-precision batch
// (Piece::exact): the first R (klm) entries of bsel_t / bsel_tv (bsel_l)
// copied to tsel_idx / tsel_cos (lsel_idx), -1 / 0 past them.
cudaError_t launch_copy_lists(const Piece *pieces, int32_t n_pieces, int64_t row0, int64_t rows, const int32_t *bsel_t,
                              const float *bsel_tv, int32_t cstride_t, const int32_t *bsel_l, int32_t cstride_l,
                              int32_t *tsel_idx, float *tsel_cos, int32_t stride_t, int32_t *lsel_idx,
                              int32_t stride_l, cudaStream_t s);
// Grouped FP32 rescore (one block per launch row): the keep_t / keep_l
// candidates of bsel_* (strides cstride_t / cstride_l; descending by their
// reduced-precision values bsel_tv / bsel_lv, nullable) are re-scored with
// exact FP32 dot products of the unit rows Q32 and the descriptors d32, and
// the R / klm best in rank order go to tsel_idx / tsel_cos and lsel_idx (-1 /
// 0 past the list).  With values, a candidate more than `band` below the
// list's R-th value is skipped.  A bulk copy that does not arrive within the
// bounded wait sets kErrTimeout in *err and leaves that row's list empty.
cudaError_t launch_rescore_grouped(const Piece *pieces, int32_t n_pieces, int64_t total_rows, const float *Q32,
                                   int32_t dim_pad, const int32_t *bsel_t, const float *bsel_tv, int32_t cstride_t,
                                   const int32_t *bsel_l, const float *bsel_lv, int32_t cstride_l, float band,
                                   int32_t *tsel_idx, float *tsel_cos, int32_t stride_t, int32_t *lsel_idx,
                                   int32_t stride_l, int32_t *err, cudaStream_t s);
constexpr int kSelectRowMax = 24576;    // longest row the shared-memory select stages

#ifdef __CUDACC__
// The last piece whose begin(piece) <= b, for a table ordered by that field
// (binary search by thread 0, broadcast through shared memory; every thread
// of the block must call it).
template <class F>
__device__ __forceinline__ int find_piece(const Piece *pieces, int n_pieces, int64_t b, F begin)
{
    __shared__ int s_piece;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_pieces - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (begin(pieces[mid]) <= b) lo = mid;
            else hi = mid - 1;
        }
        s_piece = lo;
    }
    __syncthreads();
    return s_piece;
}
#endif

// Device-side view of one scene, indexed by scene id in a device table.
struct SceneDev {
    const float *pos;       // [3, n]
    const float *views;     // [n, n_views, kViewStride]
    const int32_t *cls;     // [n]
    const float *size;      // [3, n]
    int64_t n;
    int32_t n_views;
    int32_t pad;
};

struct ComposeArgs {
    int64_t n_q;
    const int32_t *qmeta;       // [n_q, 8] (planned query order)
    const int32_t *tsel_idx;    // [n_q, stride_t]
    const int32_t *lsel_idx;    // [n_c, stride_l]
    int32_t stride_t, stride_l;
    const SceneDev *scenes;     // device table indexed by scene id
    farm_params p;
    int32_t *out_idx;           // [n_q, stride_t]
    float *out_score;
    float *out_t;               // [n_q, stride_t, 4]
    int32_t *out_anchor;
    // fused batches: the target similarity F of each listed candidate
    // ([n_q, stride_t]; s_sem = cf * F); null: s_sem = cf / (mu + rank)
    const float *tsel_F = nullptr;
};
cudaError_t launch_compose(const ComposeArgs &a, cudaStream_t s);

// Reciprocal-rank fusion of a batch's channels (k_fuse.cu).  Rows of every
// channel's similarity block: the n_q target rows, then the n_c landmark rows.
struct FuseArgs {
    int64_t n_q, n_c;
    int32_t n_ch;
    float w[FARM_MAX_CHANNELS];  // channel weights
    int32_t Rt, Rl;             // per-channel list lengths (target, landmark rows)
    const int32_t *tlist;       // [n_ch, n_q, Rt]
    const int32_t *llist;       // [n_ch, n_c, Rl]
    const float *S;             // [n_ch, rows, ld]
    int64_t rows, ld;
    const float *tops;          // [n_ch, rows, gstride] group maxima of S (over 2^gshift objects)
    int64_t gstride;
    int32_t gshift;
    int32_t n;                  // objects of the scene
    const int32_t *cls;         // [n]
    int32_t *qmeta;             // [n_q, 8]: reads QM_CLS, writes QM_R (the kept count)
    farm_params p;
    int32_t RF;                 // kept target candidates per query (list stride)
    int32_t *out_tidx;          // [n_q, RF] in (F desc, index asc) order
    float *out_tF;              // [n_q, RF]
    int32_t Ka;                 // landmark list length
    int32_t *out_lidx;          // [n_c, Ka]
    int32_t *err;               // device error word (kErrFusedOverflow)
};
// part 0: target rows, part 1: landmark rows.
cudaError_t launch_fuse(const FuseArgs &a, int part, cudaStream_t s);

// Mapping-side association (k_assoc.cu): device arrays only.
struct AssocArgs {
    int32_t N, B, F;                    // entities, detections, feature length
    const float *S;                     // [B, ld] detection-by-entity feature cosines
    int64_t ld;
    const float *ent_mu, *ent_cov, *ent_feat, *ent_w;   // [3, N], [6, N], [N, F], [N]
    const int32_t *ent_active;          // [N]
    const float *det_mu, *det_cov, *det_feat;           // [3, B], [6, B], [B, F]
    float tau_f, h_max;
    int32_t max_m;
    int32_t *match_cnt, *match_idx;     // [B], [B, max_m]
    float *match_h;                     // [B, max_m]
    int32_t *label;                     // [N + B] scratch
    unsigned long long *win;            // [N + B] scratch
    float *acc;                         // [(N + B) * (10 + F)] scratch
    int32_t *parent;                    // [N + B]
    float *out_w, *out_mu, *out_cov, *out_feat;         // [T], [3, T], [6, T], [T, F]
    int32_t *err;
};
cudaError_t launch_assoc(const AssocArgs &a, cudaStream_t s);

// out[q * k + j] = src[perm[q] * ld + j] (and the 4-wide breakdown): the TopK
// prefix of each query's sorted candidates, back in the caller's query order.
cudaError_t launch_gather_topk(int64_t n_q, int32_t k, int32_t ld, const int32_t *perm,
                               const int32_t *idx,
                               const float *score, const float *t, const int32_t *anchor,
                               int32_t *o_idx, float *o_score, float *o_t, int32_t *o_anchor,
                               cudaStream_t s);

}  // namespace farm
