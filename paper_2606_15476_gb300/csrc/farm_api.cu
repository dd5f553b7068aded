// farm_api.cu -- the C ABI of include/farm.h: argument checks, device memory,
// query planning and the stream-ordered launch sequence
//
//   normalise rows -> similarity (App. D.2 step 3) -> per-row rank select
//   (steps 3-4) -> relations, best witnesses, composite and sort (steps 4-5)
//   -> TopK prefix copy (step 7).
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "farm_internal.h"

using farm::Buf;
using farm::Ctx;
using farm::Scene;
using farm::SceneDev;

struct farm_ctx {
    Ctx c;
    SceneDev *d_scenes = nullptr;
    // host copies of the last batch's plan (for farm_candidates)
    std::vector<int32_t> h_perm;      // caller query -> planned query
    std::vector<int32_t> h_cplan;     // caller constraint -> planned constraint
    // pinned staging for per-batch metadata
    int32_t *h_stage = nullptr;
    size_t h_stage_n = 0;
    uint8_t *h_blob = nullptr;        // pinned staging of the batch's piece tables and tensor maps
    size_t h_blob_n = 0;
    cudaEvent_t stage_done = nullptr;
    // host embedding rows of farm_query_batch travel on their own stream into
    // one of two slots, so that a batch's copy overlaps the previous batch's
    // kernels: the copy waits until the batch before last is done with the
    // slot, the ctx stream waits for the copy
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_slot_free[2] = {nullptr, nullptr};
    int raw_slot = 0;
    // CUDA graphs of batch shapes (FARM_GRAPH), least recently used evicted
    struct GraphEntry { std::vector<int64_t> key; cudaGraphExec_t exec = nullptr; int64_t launches = 0; uint64_t used = 0; };
    std::vector<GraphEntry> graphs;
    uint64_t graph_clock = 0;
    bool capturing = false;
    // The last FARM_GRAPH batch's query graphs and plan.  A batch whose query
    // graphs equal them (scenes, classes, constraint offsets and predicates,
    // precision, flags; device embeddings at the same addresses) is replayed
    // from its cached graph without planning: the staging buffers the graph
    // reads still hold the plan, since only farm_query_batch and
    // farm_query_batch_rrf write them and both clear `valid` first.
    struct Replay {
        bool valid = false;
        int32_t precision = 0, dim = 0, pinned = -1;
        uint32_t flags = 0;
        int64_t n_q = 0, n_c = 0;
        const float *src_t = nullptr, *src_c = nullptr;
        uint64_t ws_gen = 0, scene_gen = 0, mlp_version = 0;
        std::vector<int32_t> scene_of_q, tgt_cls, c_off, c_pred;
        std::vector<int64_t> key[2];      // graph key per host-row slot (slot 0 for device rows)
        int32_t rtgt = 0, klm = 0, min_n = 0;
    } replay;
    // profiling marks
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
};

namespace farm {
Ctx *ctx_of(farm_ctx *ctx) { return &ctx->c; }
cudaError_t ws_alloc(farm_ctx *ctx, Buf b, size_t bytes, void **out);
}  // namespace farm

namespace {

constexpr int kMaxScenes = 4096;
constexpr size_t kSimCapBytes = size_t(4) << 30;   // similarity block per launch group

farm_status fail(farm_ctx *ctx, farm_status st, const std::string &msg)
{
    if (ctx) ctx->c.err = msg;
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FARM_ENOMEM : FARM_ECUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

#define LAUNCH(call)              \
    do {                          \
        ctx->c.launches += 1;     \
        CK(call);                 \
    } while (0)

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// A query's predicate codes: each known, and every FARM_BETWEEN directly
// followed by its FARM_BETWEEN_AND (and only there).
bool preds_ok(const int32_t *pr, int32_t m, std::string &why)
{
    for (int32_t i = 0; i < m; ++i) {
        if (pr[i] < 0 || pr[i] > FARM_BETWEEN_AND) {
            why = "unknown predicate code " + std::to_string(pr[i]);
            return false;
        }
        if (pr[i] == FARM_BETWEEN && !(i + 1 < m && pr[i + 1] == FARM_BETWEEN_AND)) {
            why = "FARM_BETWEEN must be followed by FARM_BETWEEN_AND";
            return false;
        }
        if (pr[i] == FARM_BETWEEN_AND && !(i > 0 && pr[i - 1] == FARM_BETWEEN)) {
            why = "FARM_BETWEEN_AND must follow FARM_BETWEEN";
            return false;
        }
    }
    return true;
}

int64_t target_bound(const farm_params &p)
{
    // A candidate of rank r scores at most 1/(mu + r); k_max objects score at
    // least (1 - w) * class_mis / (mu + k_max).  Keep every rank that can tie.
    double r = ((double)p.mu + (double)p.k_max) / ((1.0 - (double)p.w) * (double)p.class_mis) -
               (double)p.mu;
    return (int64_t)std::floor(r) + 1;
}

bool params_ok(const farm_params &p, std::string &why)
{
    if (!(p.w > 0.f && p.w < 1.f)) { why = "w must lie in (0, 1)"; return false; }
    if (!(p.class_mis > 0.f && p.class_mis <= 1.f)) { why = "class_mis must lie in (0, 1]"; return false; }
    if (!(p.mu >= 0.f) || !std::isfinite(p.mu)) { why = "mu must be >= 0"; return false; }
    if (!(p.sigma_near > 0.f && p.tau_v > 0.f && p.tau_h > 0.f)) { why = "sigma_near, tau_v, tau_h must be > 0"; return false; }
    if (!(p.z_min >= 0.f) || !std::isfinite(p.z_min)) { why = "z_min must be >= 0"; return false; }
    if (p.k_anchor < 1 || p.k_anchor > farm::kMaxAnchorCands) { why = "k_anchor must lie in [1, 256]"; return false; }
    if (p.k_max < 1) { why = "k_max must be >= 1"; return false; }
    if (target_bound(p) > farm::kMaxTargetCands) {
        why = "(mu + k_max) / ((1 - w) * class_mis) - mu exceeds 512 target candidates";
        return false;
    }
    if (p.rescore < 1 || p.rescore > farm::kMaxTargetCands) { why = "rescore must lie in [1, 512]"; return false; }
    if (!(p.rescore_band >= 0.f) || !std::isfinite(p.rescore_band)) { why = "rescore_band must be >= 0"; return false; }
    if (!(p.sigma_next > 0.f && p.on_gate > 0.f && p.on_band > 0.f && p.tau_d > 0.f) ||
        !std::isfinite(p.sigma_next) || !std::isfinite(p.on_gate) || !std::isfinite(p.on_band) || !std::isfinite(p.tau_d)) {
        why = "sigma_next, on_gate, on_band, tau_d must be > 0";
        return false;
    }
    if (p.k_closest < 1 || p.k_closest > target_bound(p)) {
        why = "k_closest must lie in [1, R]: the candidate set of Closest / Farthest lies within the kept ranks";
        return false;
    }
    return true;
}

cudaError_t ws_get(farm_ctx *ctx, Buf b, size_t bytes, void **out)
{
    auto &ws = ctx->c.ws;
    if (bytes == 0) bytes = 16;
    if (ws.bytes[b] < bytes) {
        if (ws.ptr[b]) {
            cudaError_t e = cudaStreamSynchronize(ctx->c.stream);
            if (e != cudaSuccess) return e;
            cudaFree(ws.ptr[b]);
            ws.ptr[b] = nullptr;
            ws.bytes[b] = 0;
        }
        size_t grow = bytes + bytes / 8;
        cudaError_t e = cudaMalloc(&ws.ptr[b], grow);
        if (e != cudaSuccess) return e;
        ws.bytes[b] = grow;
        ctx->c.ws_gen += 1;     // captured graphs that use the old buffer no longer match
    }
    *out = ws.ptr[b];
    return cudaSuccess;
}

}  // namespace

cudaError_t farm::ws_alloc(farm_ctx *ctx, Buf b, size_t bytes, void **out) { return ws_get(ctx, b, bytes, out); }

namespace {

template <class T>
cudaError_t ws_get(farm_ctx *ctx, Buf b, size_t count, T **out)
{
    void *p = nullptr;
    cudaError_t e = ws_get(ctx, b, count * sizeof(T), &p);
    *out = static_cast<T *>(p);
    return e;
}

void free_scene(Scene &s)
{
    cudaFree(s.desc32); cudaFree(s.desc_hi); cudaFree(s.desc_lo); cudaFree(s.desc_bf16);
    cudaFree(s.desc_fp8); cudaFree(s.desc_scale); cudaFree(s.comp);
    cudaFree(s.cls); cudaFree(s.pos); cudaFree(s.size); cudaFree(s.views);
    for (auto &sp : s.spaces) { cudaFree(sp.hi); cudaFree(sp.lo); }
    s = Scene{};
}

int mark_begin(farm_ctx *ctx, int stage)
{
    if (!ctx->c.profiling || ctx->capturing) return -1;
    cudaEvent_t a, b;
    if (ctx->pool.size() >= 2) {
        a = ctx->pool.back(); ctx->pool.pop_back();
        b = ctx->pool.back(); ctx->pool.pop_back();
    } else {
        if (cudaEventCreate(&a) != cudaSuccess) return -1;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
    }
    cudaEventRecord(a, ctx->c.stream);
    ctx->marks.push_back({stage, a, b});
    return (int)ctx->marks.size() - 1;
}

void mark_end(farm_ctx *ctx, int m)
{
    if (m >= 0) cudaEventRecord(ctx->marks[m].b, ctx->c.stream);
}

bool all_finite(const float *x, int64_t count)
{
    for (int64_t i = 0; i < count; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

farm_status check_device_errors(farm_ctx *ctx)
{
    Ctx &c = ctx->c;
    CK(cudaMemcpyAsync(c.h_err, c.d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    const int32_t e = *c.h_err;
    if (e == 0) return FARM_OK;
    CK(cudaMemsetAsync(c.d_err, 0, sizeof(int32_t), c.stream));
    CK(cudaStreamSynchronize(c.stream));
    c.batch_valid = false;
    if (e & farm::kErrTimeout) return fail(ctx, FARM_ETIMEOUT, "a bounded device-side wait gave up");
    if (e & farm::kErrPieceTable) return fail(ctx, FARM_ECUDA, "a similarity piece table entry was malformed");
    if (e & farm::kErrFusedOverflow)
        return fail(ctx, FARM_EINVAL, "a fused query kept more than 512 candidates that can reach its TopK");
    if (e & farm::kErrAssocOverflow)
        return fail(ctx, FARM_EINVAL, "a detection has more than 1,024 entities within the Hellinger budget");
    if (e & farm::kErrBadDesc)
        return fail(ctx, FARM_EINVAL, "a descriptor row has zero or non-finite norm");
    return fail(ctx, FARM_EINVAL, "an embedding row has zero or non-finite norm");
}

// Normalised operand rows for `prec` into the workspace; returns pointers.
struct RowOps {
    float *q32 = nullptr;
    uint16_t *qhi = nullptr, *qlo = nullptr;
    uint16_t *qbf = nullptr;
    uint8_t *qf8 = nullptr;
    float *qscale = nullptr;
    uint16_t *qcomp = nullptr;   // learned embeddings of the rows
};

bool reduced_precision(int32_t prec)
{
    return prec == FARM_PREC_BF16 || prec == FARM_PREC_FP8 || prec == FARM_PREC_LEARNED;
}

cudaError_t alloc_rows(farm_ctx *ctx, int32_t prec, int64_t rows, int32_t dim_pad, RowOps &r)
{
    const size_t cnt = (size_t)std::max<int64_t>(rows, 1) * dim_pad;
    cudaError_t e = cudaSuccess;
    if (prec == FARM_PREC_FP32_SIMT || reduced_precision(prec)) {
        if ((e = ws_get(ctx, farm::B_Q32, cnt, &r.q32)) != cudaSuccess) return e;
    }
    if (prec == FARM_PREC_BF16 || prec == FARM_PREC_LEARNED) {
        if ((e = ws_get(ctx, farm::B_QBF, cnt, &r.qbf)) != cudaSuccess) return e;
    }
    if (prec == FARM_PREC_LEARNED) {
        const size_t ccnt = (size_t)std::max<int64_t>(rows, 1) * ctx->c.mlp.P;
        if ((e = ws_get(ctx, farm::B_QCOMP, ccnt, &r.qcomp)) != cudaSuccess) return e;
    }
    if (prec == FARM_PREC_FP8) {
        if ((e = ws_get(ctx, farm::B_QF8, cnt, &r.qf8)) != cudaSuccess) return e;
        if ((e = ws_get(ctx, farm::B_QSCALE, (size_t)std::max<int64_t>(rows, 1), &r.qscale)) != cudaSuccess)
            return e;
    }
    if (prec == FARM_PREC_FP32) {
        if ((e = ws_get(ctx, farm::B_QHI, cnt, &r.qhi)) != cudaSuccess) return e;
        if ((e = ws_get(ctx, farm::B_QLO, cnt, &r.qlo)) != cudaSuccess) return e;
    }
    return e;
}

// S rows [r0, r0 + rows) of the planned row space against scene s.
farm_status run_similarity(farm_ctx *ctx, int32_t prec, const RowOps &ops, int64_t r0,
                           int64_t rows, const Scene &s, float *S, int64_t ld_s, float *tops = nullptr)
{
    Ctx &c = ctx->c;
    const int64_t off = r0 * s.dim_pad;
    switch (prec) {
    case FARM_PREC_FP32_SIMT:
        LAUNCH(farm::launch_sim_simt(ops.q32 + off, s.desc32, S, rows, s.n, s.dim_pad, ld_s, c.stream));
        return FARM_OK;
    case FARM_PREC_FP32:
        if (!farm::sim_tc_available())
            return fail(ctx, FARM_EINVAL, "the tensor-core FP32 similarity path is not built");
        LAUNCH(farm::launch_sim_tc_f16x3(ops.qhi + off, ops.qlo + off, s.desc_hi, s.desc_lo, S,
                                         rows, s.n, s.dim_pad, ld_s, tops, c.num_sms, c.d_err, c.stream));
        return FARM_OK;
    case FARM_PREC_BF16:
        if (!farm::sim_tc_available())
            return fail(ctx, FARM_EINVAL, "the tensor-core similarity path is not built");
        LAUNCH(farm::launch_sim_tc_bf16(ops.qbf + off, s.desc_bf16, S, rows, s.n, s.dim_pad, ld_s, tops, c.num_sms,
                                        c.d_err, c.stream));
        return FARM_OK;
    case FARM_PREC_LEARNED:
        if (!farm::sim_tc_available())
            return fail(ctx, FARM_EINVAL, "the tensor-core similarity path is not built");
        LAUNCH(farm::launch_sim_tc_bf16(ops.qcomp + r0 * c.mlp.P, s.comp, S, rows, s.n, c.mlp.P, ld_s, tops, c.num_sms,
                                        c.d_err, c.stream));
        return FARM_OK;
    case FARM_PREC_FP8:
        if (!farm::sim_tc_available())
            return fail(ctx, FARM_EINVAL, "the tensor-core similarity path is not built");
        LAUNCH(farm::launch_sim_tc_fp8(ops.qf8 + off, ops.qscale + r0, s.desc_fp8, s.desc_scale, S, rows, s.n,
                                       s.dim_pad, ld_s, tops, c.num_sms, c.d_err, c.stream));
        return FARM_OK;
    default:
        return fail(ctx, FARM_EINVAL, "precision not supported by this build");
    }
}

// Candidates kept per row by the reduced-precision stage before the FP32
// rescore: `rescore` for BF16 target rows, twice that for FP8 (whose E4M3
// operands carry 4 significant bits against BF16's 8), at most 512; landmark
// rows keep a quarter of it, at least K_a.
int32_t reduced_keep_target(const farm_params &p, int32_t prec, int32_t R, int64_t n)
{
    if (prec == FARM_PREC_LEARNED) return (int32_t)std::min<int64_t>(farm::kMaxTargetCands, n);
    const int32_t c = std::min<int32_t>(prec == FARM_PREC_FP8 ? 2 * p.rescore : p.rescore, farm::kMaxTargetCands);
    return (int32_t)std::min<int64_t>(std::max<int32_t>(c, R), n);
}
int32_t reduced_keep_landmark(const farm_params &p, int32_t prec, int32_t klm, int64_t n)
{
    const int32_t c = prec == FARM_PREC_LEARNED ? farm::kMaxTargetCands / 4
                                                : (prec == FARM_PREC_FP8 ? 2 * p.rescore : p.rescore) / 4;
    return (int32_t)std::min<int64_t>(std::max<int32_t>(std::min<int32_t>(c, farm::kMaxAnchorCands), klm), n);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

namespace {

// Host embedding rows of a batch: slot `slot` (one half) of the two-slot
// device buffer (sized by the batch that planned it).
float *raw_slot_ptr(farm_ctx *ctx, int slot)
{
    const farm::Ctx &c = ctx->c;
    const size_t half = c.ws.bytes[farm::B_RAW_PIPE] / 2 / 256 * 256;
    return reinterpret_cast<float *>(static_cast<uint8_t *>(c.ws.ptr[farm::B_RAW_PIPE]) + slot * half);
}

// The host rows into d_raw on the copy stream once the slot is free again;
// the ctx stream waits for the copy.
cudaError_t copy_host_rows(farm_ctx *ctx, int slot, float *d_raw, const float *tgt_emb, const float *c_emb,
                           int64_t n_q, int64_t n_c, int32_t dim)
{
    cudaError_t e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_slot_free[slot], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_raw, tgt_emb, (size_t)n_q * dim * 4, cudaMemcpyHostToDevice, ctx->copy_stream);
    if (e == cudaSuccess && n_c > 0)
        e = cudaMemcpyAsync(d_raw + (size_t)n_q * dim, c_emb, (size_t)n_c * dim * 4, cudaMemcpyHostToDevice,
                            ctx->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_copied[slot], ctx->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->c.stream, ctx->ev_copied[slot], 0);
    return e;
}

template <class T>
bool same_array(const std::vector<T> &v, const T *p, int64_t n)
{
    return (int64_t)v.size() == n && (n == 0 || std::memcmp(v.data(), p, (size_t)n * sizeof(T)) == 0);
}

// Whether the recorded batch has the same query graphs and launch inputs as
// the call's (everything the recorded plan and its graphs depend on).
bool replay_same(const farm_ctx *ctx, int64_t n_q, const int32_t *scene_of_q, const float *tgt_emb,
                 const int32_t *tgt_cls, const int32_t *c_off, const int32_t *c_pred, const float *c_emb,
                 int32_t precision, uint32_t flags)
{
    const farm_ctx::Replay &r = ctx->replay;
    const farm::Ctx &c = ctx->c;
    if (r.precision != precision || r.flags != flags || r.n_q != n_q || r.pinned != c.pinned_variant ||
        r.ws_gen != c.ws_gen || r.scene_gen != c.scene_gen || r.mlp_version != c.mlp.version)
        return false;
    if ((flags & FARM_PTR_DEVICE) && (r.src_t != tgt_emb || r.src_c != c_emb)) return false;
    if (!same_array(r.c_off, c_off, n_q + 1)) return false;
    const int64_t n_c = c_off[n_q];
    if (n_c != r.n_c || (n_c > 0 && !c_pred)) return false;
    return same_array(r.scene_of_q, scene_of_q, n_q) && same_array(r.tgt_cls, tgt_cls, n_q) &&
           (n_c == 0 || same_array(r.c_pred, c_pred, n_c));
}

// A batch equal to the recorded one, replayed from its graph: the host rows'
// copy (host embeddings) and the graph launch.  `done` is false when the call
// needs planning (no record, a different batch, or its graph evicted).
farm_status replay_batch(farm_ctx *ctx, int64_t n_q, const int32_t *scene_of_q, const float *tgt_emb,
                         const int32_t *tgt_cls, const int32_t *c_off, const int32_t *c_pred, const float *c_emb,
                         int32_t precision, uint32_t flags, uint64_t *batch_handle, bool &done)
{
    done = false;
    farm_ctx::Replay &r = ctx->replay;
    Ctx &c = ctx->c;
    if (!r.valid || !replay_same(ctx, n_q, scene_of_q, tgt_emb, tgt_cls, c_off, c_pred, c_emb, precision, flags))
        return FARM_OK;
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    const int slot = dev ? 0 : ctx->raw_slot;
    if (r.key[slot].empty()) return FARM_OK;
    farm_ctx::GraphEntry *hit = nullptr;
    for (auto &ge : ctx->graphs)
        if (ge.key == r.key[slot]) hit = &ge;
    if (!hit) return FARM_OK;
    done = true;
    c.batch_valid = false;
    *batch_handle = 0;
    CK(cudaSetDevice(c.device));
    if (!dev) {
        CK(copy_host_rows(ctx, slot, raw_slot_ptr(ctx, slot), tgt_emb, c_emb, n_q, r.n_c, r.dim));
        ctx->raw_slot ^= 1;
    }
    hit->used = ++ctx->graph_clock;
    CK(cudaGraphLaunch(hit->exec, c.stream));
    c.launches += hit->launches;
    if (!dev) CK(cudaEventRecord(ctx->ev_slot_free[slot], c.stream));
    c.batch_gen += 1;
    c.batch_valid = true;
    c.batch_nq = n_q;
    c.batch_nc = r.n_c;
    c.batch_rtgt = r.rtgt;
    c.batch_klm = r.klm;
    c.batch_min_n = r.min_n;
    *batch_handle = c.batch_gen;
    return FARM_OK;
}

}  // namespace

extern "C" {

const char *farm_version(void) { return "farm-gb300 0.1 (sm_103a)"; }

void farm_default_params(farm_params *p)
{
    if (!p) return;
    p->mu = 5.0f;
    p->w = 0.5f;
    p->class_mis = 0.3f;
    p->sigma_near = 0.5f;
    p->tau_v = 0.25f;
    p->tau_h = 0.10f;
    p->z_min = 0.05f;
    p->k_anchor = 16;
    p->k_max = 10;
    p->rescore = 256;
    p->rescore_band = 2e-3f;
    p->sigma_next = 1.0f;
    p->on_gate = 0.10f;
    p->on_band = 0.10f;
    p->tau_d = 0.25f;
    p->k_closest = 16;
}

const char *farm_last_error(farm_ctx *ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

farm_status farm_destroy(farm_ctx *ctx)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    cudaSetDevice(c.device);
    if (c.stream) cudaStreamSynchronize(c.stream);
    for (auto &s : c.scenes)
        if (s.present) free_scene(s);
    for (int b = 0; b < farm::B_COUNT; ++b) cudaFree(c.ws.ptr[b]);
    cudaFree(c.d_err);
    cudaFree(c.d_fallback);
    cudaFree(ctx->d_scenes);
    cudaFree(c.mlp.params);
    cudaFree(c.mlp.w1b);
    cudaFree(c.mlp.w2b);
    cudaFree(c.mlp.w2t);
    if (c.h_err) cudaFreeHost(c.h_err);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->h_blob) cudaFreeHost(ctx->h_blob);
    if (ctx->stage_done) cudaEventDestroy(ctx->stage_done);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (int k = 0; k < 2; ++k) {
        if (ctx->ev_copied[k]) cudaEventDestroy(ctx->ev_copied[k]);
        if (ctx->ev_slot_free[k]) cudaEventDestroy(ctx->ev_slot_free[k]);
    }
    for (auto &m : ctx->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
    delete ctx;
    return FARM_OK;
}

farm_status farm_create(farm_ctx **out, int device, void *cuda_stream, const farm_params *params)
{
    if (!out) return FARM_EINVAL;
    *out = nullptr;
    farm_params p;
    farm_default_params(&p);
    if (params) p = *params;
    std::string why;
    if (!params_ok(p, why)) return FARM_EINVAL;
    farm_ctx *ctx = new farm_ctx();
    Ctx &c = ctx->c;
    c.device = device;
    c.params = p;
    c.scenes.resize(kMaxScenes);
    auto bail = [&](farm_status st) {
        farm_destroy(ctx);
        return st;
    };
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return bail(FARM_ECUDA);
    if (cudaSetDevice(device) != cudaSuccess) return bail(FARM_ECUDA);
    if (cuda_stream) {
        c.stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) return bail(FARM_ECUDA);
        c.own_stream = true;
    }
    if (cudaMalloc(&c.d_err, sizeof(int32_t)) != cudaSuccess) return bail(FARM_ENOMEM);
    if (cudaMemset(c.d_err, 0, sizeof(int32_t)) != cudaSuccess) return bail(FARM_ECUDA);
    if (cudaMalloc(&c.d_fallback, sizeof(int32_t)) != cudaSuccess) return bail(FARM_ENOMEM);
    if (cudaMemset(c.d_fallback, 0, sizeof(int32_t)) != cudaSuccess) return bail(FARM_ECUDA);
    if (cudaHostAlloc(&c.h_err, sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) return bail(FARM_ENOMEM);
    if (cudaMalloc(&ctx->d_scenes, kMaxScenes * sizeof(SceneDev)) != cudaSuccess) return bail(FARM_ENOMEM);
    if (cudaMemset(ctx->d_scenes, 0, kMaxScenes * sizeof(SceneDev)) != cudaSuccess) return bail(FARM_ECUDA);
    if (cudaEventCreateWithFlags(&ctx->stage_done, cudaEventDisableTiming) != cudaSuccess) return bail(FARM_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(FARM_ECUDA);
    for (int k = 0; k < 2; ++k)
        if (cudaEventCreateWithFlags(&ctx->ev_copied[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_slot_free[k], cudaEventDisableTiming) != cudaSuccess)
            return bail(FARM_ECUDA);
    if (cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(FARM_ECUDA);
    // the static scratch array of farm_rank_rows_noalloc: resolved here, so
    // that calls of that entry point take no memory and load no module
    if (farm::noalloc_setup(device) != cudaSuccess) return bail(FARM_ECUDA);
    *out = ctx;
    return FARM_OK;
}

farm_status farm_memory_upload(farm_ctx *ctx, int32_t scene_id, int64_t n, int32_t dim,
                               const float *desc, const int32_t *cls, const float *box,
                               int32_t n_views, const float *views, uint32_t flags)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (scene_id < 0 || scene_id >= kMaxScenes) return fail(ctx, FARM_EINVAL, "scene_id out of range");
    if (n < 1 || n > 0x7fffffff) return fail(ctx, FARM_EINVAL, "n must lie in [1, 2^31)");
    if (dim < 1 || dim > 8192) return fail(ctx, FARM_EINVAL, "dim must lie in [1, 8192]");
    if (!desc || !cls || !box) return fail(ctx, FARM_EINVAL, "desc, cls and box must be non-null");
    if (n_views < 0 || n_views > FARM_MAX_VIEWS) return fail(ctx, FARM_EINVAL, "n_views must lie in [0, 16]");
    if (n_views > 0 && !views) return fail(ctx, FARM_EINVAL, "views must be non-null when n_views > 0");
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    if (!dev) {
        if (!all_finite(box, 6 * n)) return fail(ctx, FARM_EINVAL, "box holds a non-finite value");
        if (n_views > 0 && !all_finite(views, 6 * (int64_t)n_views * n))
            return fail(ctx, FARM_EINVAL, "views hold a non-finite value");
        for (int64_t j = 0; j < n; ++j) {
            double ss = 0.0;
            const float *d = desc + j * dim;
            for (int32_t k = 0; k < dim; ++k) ss += (double)d[k] * (double)d[k];
            if (!(ss > 0.0) || !std::isfinite(ss))
                return fail(ctx, FARM_EINVAL, "descriptor row " + std::to_string(j) + " has zero or non-finite norm");
        }
    }
    CK(cudaSetDevice(c.device));
    Scene &s = c.scenes[scene_id];
    if (s.present) {
        CK(cudaStreamSynchronize(c.stream));
        free_scene(s);
    }
    Scene ns;
    ns.n = n;
    ns.dim = dim;
    ns.dim_pad = (int32_t)round_up(dim, farm::kDimAlign);
    ns.n_views = n_views;
    const size_t nd = (size_t)n * ns.dim_pad;
    auto bailmem = [&](cudaError_t e) {
        free_scene(ns);
        return fail(ctx, e == cudaErrorMemoryAllocation ? FARM_ENOMEM : FARM_ECUDA,
                    std::string("scene upload: ") + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&ns.desc32, nd * 4)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.desc_hi, nd * 2)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.desc_lo, nd * 2)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.desc_bf16, nd * 2)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.desc_fp8, nd)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.desc_scale, (size_t)n * 4)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.cls, (size_t)n * 4)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.pos, (size_t)n * 12)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.size, (size_t)n * 12)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMalloc(&ns.views, (size_t)n * std::max(n_views, 1) * farm::kViewStride * 4)) != cudaSuccess)
        return bailmem(e);
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const float *d_desc = desc;
    float *tmp_desc = nullptr, *tmp_views = nullptr;
    if (!dev) {
        if ((e = cudaMallocAsync(&tmp_desc, (size_t)n * dim * 4, c.stream)) != cudaSuccess) return bailmem(e);
        if ((e = cudaMemcpyAsync(tmp_desc, desc, (size_t)n * dim * 4, kind, c.stream)) != cudaSuccess)
            return bailmem(e);
        d_desc = tmp_desc;
    }
    ctx->c.launches += 1;
    if ((e = farm::launch_normalize_rows(d_desc, nullptr, n, dim, ns.dim_pad, ns.desc32, ns.desc_hi,
                                         ns.desc_lo, ns.desc_bf16, c.d_err, farm::kErrBadDesc,
                                         c.stream)) != cudaSuccess)
        return bailmem(e);
    ctx->c.launches += 1;
    if ((e = farm::launch_quantize_fp8_rows(ns.desc32, n, ns.dim_pad, ns.desc_fp8, ns.desc_scale, c.stream)) !=
        cudaSuccess)
        return bailmem(e);
    if ((e = cudaMemcpyAsync(ns.cls, cls, (size_t)n * 4, kind, c.stream)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMemcpyAsync(ns.pos, box, (size_t)n * 12, kind, c.stream)) != cudaSuccess) return bailmem(e);
    if ((e = cudaMemcpyAsync(ns.size, box + 3 * n, (size_t)n * 12, kind, c.stream)) != cudaSuccess)
        return bailmem(e);
    if (n_views > 0) {
        const float *d_views = views;
        if (!dev) {
            const size_t vb = (size_t)6 * n_views * n * 4;
            if ((e = cudaMallocAsync(&tmp_views, vb, c.stream)) != cudaSuccess) return bailmem(e);
            if ((e = cudaMemcpyAsync(tmp_views, views, vb, kind, c.stream)) != cudaSuccess) return bailmem(e);
            d_views = tmp_views;
        }
        ctx->c.launches += 1;
        if ((e = farm::launch_prepare_views(d_views, ns.pos, n, n_views, ns.views, c.stream)) != cudaSuccess)
            return bailmem(e);
    }
    if (tmp_desc) cudaFreeAsync(tmp_desc, c.stream);
    if (tmp_views) cudaFreeAsync(tmp_views, c.stream);
    SceneDev sd{ns.pos, ns.views, ns.cls, ns.size, n, n_views, 0};
    if ((e = cudaMemcpyAsync(ctx->d_scenes + scene_id, &sd, sizeof(sd), cudaMemcpyHostToDevice, c.stream)) !=
        cudaSuccess)
        return bailmem(e);
    // the host-side SceneDev is a stack value: make sure it has been consumed
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return bailmem(e);
    ns.present = true;
    s = ns;
    c.batch_valid = false;
    c.scene_gen += 1;
    return FARM_OK;
}

farm_status farm_query_batch(farm_ctx *ctx, int64_t n_q, const int32_t *scene_of_q,
                             const float *tgt_emb, const int32_t *tgt_cls, const int32_t *c_off,
                             const int32_t *c_pred, const float *c_emb, int32_t precision,
                             uint32_t flags, uint64_t *batch_handle)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (!batch_handle) return fail(ctx, FARM_EINVAL, "batch_handle must be non-null");
    if (n_q < 0 || n_q > 0x7fffffff) return fail(ctx, FARM_EINVAL, "n_q out of range");
    if (precision != FARM_PREC_FP32 && precision != FARM_PREC_BF16 && precision != FARM_PREC_FP32_SIMT &&
        precision != FARM_PREC_FP8 && precision != FARM_PREC_LEARNED)
        return fail(ctx, FARM_EINVAL, "unknown precision");
    if (precision == FARM_PREC_LEARNED && !c.mlp.set)
        return fail(ctx, FARM_ESTATE, "FARM_PREC_LEARNED needs prefilter weights (farm_mlp_set or farm_mlp_train)");
    if (n_q > 0 && (!scene_of_q || !tgt_emb || !tgt_cls || !c_off))
        return fail(ctx, FARM_EINVAL, "scene_of_q, tgt_emb, tgt_cls and c_off must be non-null");
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    bool graph = (flags & FARM_GRAPH) != 0;
    if (graph && n_q > 0) {
        bool done = false;
        const farm_status st = replay_batch(ctx, n_q, scene_of_q, tgt_emb, tgt_cls, c_off, c_pred, c_emb, precision,
                                            flags, batch_handle, done);
        if (done) return st;
    }
    ctx->replay.valid = false;       // planning rewrites the staging buffers
    int64_t n_c = 0;
    int32_t dim = -1;
    int64_t min_n = INT64_MAX, max_n = 0;
    if (n_q > 0) {
        if (c_off[0] != 0) return fail(ctx, FARM_EINVAL, "c_off[0] must be 0");
        for (int64_t q = 0; q < n_q; ++q) {
            const int32_t m = c_off[q + 1] - c_off[q];
            if (m < 0 || m > FARM_MAX_CONSTRAINTS)
                return fail(ctx, FARM_EINVAL, "query " + std::to_string(q) + " has " + std::to_string(m) +
                                                  " constraints (0..4 allowed)");
            const int32_t sid = scene_of_q[q];
            if (sid < 0 || sid >= kMaxScenes || !c.scenes[sid].present)
                return fail(ctx, FARM_EINVAL, "query " + std::to_string(q) + " names an unknown scene");
            const Scene &s = c.scenes[sid];
            if (dim < 0) dim = s.dim;
            if (s.dim != dim) return fail(ctx, FARM_EINVAL, "all scenes of a batch must share dim");
            if (precision == FARM_PREC_LEARNED && s.dim != c.mlp.D)
                return fail(ctx, FARM_EINVAL, "the prefilter network's input length differs from the scene's dim");
            min_n = std::min(min_n, s.n);
            max_n = std::max(max_n, s.n);
        }
        n_c = c_off[n_q];
        if (n_c > 0 && (!c_pred || !c_emb)) return fail(ctx, FARM_EINVAL, "c_pred and c_emb must be non-null");
        std::string why;
        for (int64_t q = 0; q < n_q; ++q)
            if (!preds_ok(c_pred + c_off[q], c_off[q + 1] - c_off[q], why))
                return fail(ctx, FARM_EINVAL, "query " + std::to_string(q) + ": " + why);
    }
    c.batch_valid = false;
    *batch_handle = 0;
    CK(cudaSetDevice(c.device));
    const farm_params &p = c.params;
    const int64_t Rb = target_bound(p);
    if (n_q == 0) {
        c.batch_gen += 1;
        c.batch_valid = true;
        c.batch_nq = 0;
        c.batch_nc = 0;
        c.batch_min_n = 0;
        ctx->h_perm.clear();
        ctx->h_cplan.clear();
        *batch_handle = c.batch_gen;
        return FARM_OK;
    }
    const int32_t stride_t = (int32_t)std::min<int64_t>(Rb, max_n);
    const int32_t stride_l = (int32_t)std::min<int64_t>(p.k_anchor, max_n);
    const int32_t dim_pad = (int32_t)round_up(dim, farm::kDimAlign);

    // BF16 and FP8 batches: a scene of fewer objects than the bound runs the
    // FP32-accurate similarity (three-term FP16 split) in the same batch and
    // its lists are final, with no rescore -- re-reading the FP32 descriptors
    // of C candidates per row costs more than the FP32-accurate GEMM over a
    // small scene (rows of an n-object scene: the GEMM saves about
    // 2.8e-12 n s per row at BF16 rates, the rescore and the longer select
    // cost about 4.7e-8 s per row, so BF16 gains from about 16,000 objects).
    // FP8 takes the same bound, although its rescore of twice the candidates
    // in a wider band only pays from about 32,000 objects: a 20,000-object
    // scene then still runs the precision the caller asked for.
    const int64_t exact_below =
        (precision == FARM_PREC_BF16 && !(flags & FARM_FUSED)) || precision == FARM_PREC_FP8 ? 16384 : 0;
    // ---- plan: group queries by scene (stable; the scenes that run
    //      FP32-accurate in a reduced-precision batch last, so that their rows
    //      end the row space), rows = [targets, constraints] per group
    struct Group { int32_t sid; int64_t nq = 0, nc = 0, row0 = 0, q0 = 0, cp0 = 0; };
    auto scene_key = [&](int32_t sid) { return ((int64_t)(c.scenes[sid].n < exact_below) << 32) | sid; };
    std::vector<int32_t> order((size_t)n_q);
    for (int64_t q = 0; q < n_q; ++q) order[q] = (int32_t)q;
    bool sorted = true;
    for (int64_t q = 1; q < n_q; ++q) sorted &= scene_key(scene_of_q[q]) >= scene_key(scene_of_q[q - 1]);
    if (!sorted)
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return scene_key(scene_of_q[a]) < scene_key(scene_of_q[b]); });
    std::vector<Group> groups;
    for (int64_t i = 0; i < n_q; ++i) {
        const int32_t q = order[i];
        if (groups.empty() || groups.back().sid != scene_of_q[q]) {
            Group g;
            g.sid = scene_of_q[q];
            g.q0 = i;
            groups.push_back(g);
        }
        groups.back().nq += 1;
        groups.back().nc += c_off[q + 1] - c_off[q];
    }
    // Reduced-precision batches: within a scene the queries are ordered by
    // target class (stable, a counting sort).  The FP32 rescore gathers each
    // target row's candidates -- mostly the objects of its class -- and the
    // CTAs of consecutive rows then find those descriptor rows in L2.  Rows
    // are independent, so the order changes no result.
    if (reduced_precision(precision)) {
        std::vector<int32_t> tmp, cnt;
        for (const auto &g : groups) {
            if (g.nq < 2) continue;
            int32_t cmax = -1;
            bool small = true;
            for (int64_t k = 0; k < g.nq; ++k) {
                const int32_t cl = tgt_cls[order[g.q0 + k]];
                small &= cl < (1 << 20);
                cmax = std::max(cmax, cl);
            }
            if (!small) continue;
            cnt.assign((size_t)cmax + 3, 0);
            for (int64_t k = 0; k < g.nq; ++k) cnt[(size_t)std::max(tgt_cls[order[g.q0 + k]], -1) + 2] += 1;
            for (size_t j = 1; j < cnt.size(); ++j) cnt[j] += cnt[j - 1];
            tmp.resize((size_t)g.nq);
            for (int64_t k = 0; k < g.nq; ++k) {
                const int32_t q = order[g.q0 + k];
                tmp[(size_t)cnt[(size_t)std::max(tgt_cls[q], -1) + 1]++] = q;
            }
            std::copy(tmp.begin(), tmp.end(), order.begin() + g.q0);
        }
    }
    int64_t row = 0, cp = 0;
    for (auto &g : groups) {
        g.row0 = row;
        g.cp0 = cp;
        row += g.nq + g.nc;
        cp += g.nc;
    }
    const int64_t rows_total = row;
    auto exact_scene = [&](const Scene &s) { return s.n < exact_below; };
    bool any_exact = false, all_exact = exact_below > 0;
    for (const auto &g : groups) {
        any_exact |= exact_scene(c.scenes[g.sid]);
        all_exact &= exact_scene(c.scenes[g.sid]);
    }
    // a batch of small scenes only is an FP32 batch (fused where that pays)
    if (all_exact) {
        precision = FARM_PREC_FP32;
        any_exact = false;
    }
    // the first planned row of the FP32-accurate scenes (rows_total: none)
    int64_t exact_row0 = rows_total;
    for (const auto &g : groups)
        if (any_exact && exact_scene(c.scenes[g.sid])) {
            exact_row0 = g.row0;
            break;
        }
    // staging layout (int32): rowmap[n_q + n_c] | perm[n_q] | qmeta[n_q * 8]
    const size_t need = (size_t)(n_q + n_c) + (size_t)n_q + (size_t)n_q * 8;
    CK(cudaEventSynchronize(ctx->stage_done));
    if (ctx->h_stage_n < need) {
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        ctx->h_stage_n = 0;
        CK(cudaHostAlloc(&ctx->h_stage, need * sizeof(int32_t) * 5 / 4, cudaHostAllocDefault));
        ctx->h_stage_n = need * 5 / 4;
    }
    int32_t *h_rowmap = ctx->h_stage;
    int32_t *h_perm = h_rowmap + (n_q + n_c);
    int32_t *h_meta = h_perm + n_q;
    ctx->h_perm.assign((size_t)n_q, 0);
    ctx->h_cplan.assign((size_t)n_c, 0);
    for (const auto &g : groups) {
        const Scene &s = c.scenes[g.sid];
        const int32_t Rs = (int32_t)std::min<int64_t>(Rb, s.n);
        const int32_t klm = (int32_t)std::min<int64_t>(p.k_anchor, s.n);
        int64_t cpos = 0;
        for (int64_t k = 0; k < g.nq; ++k) {
            const int64_t pq = g.q0 + k;       // planned query index
            const int32_t q = order[pq];
            h_rowmap[q] = (int32_t)(g.row0 + k);
            h_perm[q] = (int32_t)pq;
            ctx->h_perm[q] = (int32_t)pq;
            const int32_t m = c_off[q + 1] - c_off[q];
            int32_t pr[4] = {0, 0, 0, 0};
            for (int32_t i = 0; i < m; ++i) {
                const int64_t cc = c_off[q] + i;                  // caller constraint
                const int64_t pc = g.cp0 + cpos + i;              // planned constraint
                h_rowmap[n_q + cc] = (int32_t)(g.row0 + g.nq + cpos + i);
                ctx->h_cplan[cc] = (int32_t)pc;
                pr[i] = c_pred[cc];
            }
            int32_t *mt = h_meta + pq * 8;
            mt[farm::QM_SCENE] = g.sid;
            mt[farm::QM_CLS] = tgt_cls[q];
            mt[farm::QM_M] = m;
            mt[farm::QM_C0] = (int32_t)(g.cp0 + cpos);
            mt[farm::QM_PRED01] = pr[0] | (pr[1] << 16);
            mt[farm::QM_PRED23] = pr[2] | (pr[3] << 16);
            mt[farm::QM_R] = Rs;
            mt[farm::QM_KLM] = klm;
            cpos += m;
        }
    }

    // ---- device buffers
    int32_t *d_rowmap, *d_perm, *d_meta, *tsel_idx, *lsel_idx, *o_idx, *o_anc;
    float *tsel_cos, *o_score, *o_t, *d_raw = nullptr;
    CK(ws_get(ctx, farm::B_ROWMAP, (size_t)(n_q + n_c), &d_rowmap));
    CK(ws_get(ctx, farm::B_PERM, (size_t)n_q, &d_perm));
    CK(ws_get(ctx, farm::B_QMETA, (size_t)n_q * 8, &d_meta));
    CK(ws_get(ctx, farm::B_TSEL_IDX, (size_t)n_q * stride_t, &tsel_idx));
    CK(ws_get(ctx, farm::B_TSEL_COS, (size_t)n_q * stride_t, &tsel_cos));
    CK(ws_get(ctx, farm::B_LSEL_IDX, (size_t)std::max<int64_t>(n_c, 1) * stride_l, &lsel_idx));
    CK(ws_get(ctx, farm::B_OUT_IDX, (size_t)n_q * stride_t, &o_idx));
    CK(ws_get(ctx, farm::B_OUT_SCORE, (size_t)n_q * stride_t, &o_score));
    CK(ws_get(ctx, farm::B_OUT_T, (size_t)n_q * stride_t * 4, &o_t));
    CK(ws_get(ctx, farm::B_OUT_ANCHOR, (size_t)n_q * stride_t * 4, &o_anc));
    RowOps ops;
    CK(alloc_rows(ctx, precision, rows_total, dim_pad, ops));
    if (any_exact) {
        const size_t cnt = (size_t)rows_total * dim_pad;
        CK(ws_get(ctx, farm::B_QHI, cnt, &ops.qhi));
        CK(ws_get(ctx, farm::B_QLO, cnt, &ops.qlo));
    }
    int32_t *bsel_t = nullptr, *bsel_l = nullptr;
    float *bsel_tv = nullptr, *bsel_lv = nullptr;
    const int32_t cstride_t = reduced_keep_target(p, precision, stride_t, max_n);
    const int32_t cstride_l = reduced_keep_landmark(p, precision, stride_l, max_n);
    if (reduced_precision(precision)) {
        CK(ws_get(ctx, farm::B_BSEL_T, (size_t)n_q * cstride_t, &bsel_t));
        CK(ws_get(ctx, farm::B_BSEL_L, (size_t)std::max<int64_t>(n_c, 1) * cstride_l, &bsel_l));
        if (precision != FARM_PREC_LEARNED) {
            CK(ws_get(ctx, farm::B_BSEL_TV, (size_t)n_q * cstride_t, &bsel_tv));
            CK(ws_get(ctx, farm::B_BSEL_LV, (size_t)std::max<int64_t>(n_c, 1) * cstride_l, &bsel_lv));
        }
    }
    // host rows: the next of two slots (each half of the buffer)
    const int raw_slot = ctx->raw_slot;
    if (!dev) {
        uint8_t *pipe = nullptr;
        CK(ws_get(ctx, farm::B_RAW_PIPE, 2 * (size_t)round_up((int64_t)(n_q + n_c) * dim * 4, 256), &pipe));
        d_raw = raw_slot_ptr(ctx, raw_slot);
        ctx->raw_slot ^= 1;
    }
    if (graph && precision == FARM_PREC_LEARNED) CK(farm::learned_reserve(ctx, rows_total));

    // ---- similarity batches: row ranges ("pieces") of the scene groups are
    //      laid end to end in S while they fit kSimCapBytes; each batch takes
    //      one similarity launch per piece, then the rank selection: on the
    //      tensor-core paths the thresholded select (from the 32-object group
    //      maxima the similarity epilogue writes) for every row with at least
    //      as many groups as its list length, the shared-memory select (+ chunk
    //      merge) for the others; then one FP32 rescore launch on the
    //      reduced-precision paths
    struct Batch { size_t p0 = 0, np = 0; int64_t s_floats = 0, rows = 0, blocks = 0, tblocks = 0, tmp = 0,
                   tops = 0, fused_rows = 0, twopass_rows = 0, exact_rows = 0; int32_t smem_sel = 1, smem_merge = 0,
                   max_union = 1, gmax_twopass = 1; bool chunked = false; };
    std::vector<farm::Piece> pieces;
    std::vector<int32_t> piece_sid;
    std::vector<Batch> batches;
    const bool reduced = reduced_precision(precision);
    const bool tile_tops = precision != FARM_PREC_FP32_SIMT;
    int sim_mode = -1;
    if (precision == FARM_PREC_FP32) sim_mode = farm::kSimF16x3;
    else if (precision == FARM_PREC_BF16 || precision == FARM_PREC_LEARNED) sim_mode = farm::kSimBf16;
    else if (precision == FARM_PREC_FP8) sim_mode = farm::kSimFp8;
    // the fused selection (tensor-core paths, tiles of 256 objects): each row's
    // sample -- every fs-th tile -- is stored; the row's threshold is the R-th
    // largest of its group maxima, and the other tiles keep only the entries
    // reaching it.  fs sizes the sample so that the kept entries stay well
    // inside the merge capacity (fuse_merge_capacity: 2,048 words): somewhat
    // over R fs of them for a list of R
    // (FP32 and BF16 only: E4M3's few significant bits tie many FP8 entries at
    // any threshold, and the learned path's lists of 512 would need a sample
    // of half the row and still crowd the buffer -- it takes the two-pass
    // form below on long rows)
    // Which scenes' rows are fused: FARM_FUSED fuses every scene, FARM_UNFUSED
    // none; by default the FP32 path fuses a scene whose sample holds at
    // least 16 times its target list (a shorter sample sets a threshold that
    // lets a large part of the other tiles through, whose appends then cost
    // more than storing the row), and BF16 none (measured on a 20,000-object
    // scene: with its lists of 256 the threshold and the merge cost more
    // than the stores of S).  A batch may hold fused and unfused scenes.
    const bool fusable = (precision == FARM_PREC_FP32 || precision == FARM_PREC_BF16) && c.pinned_variant != 1 &&
                         !(flags & FARM_UNFUSED);
    // The learned path's lists (512 target, 128 landmark candidates) over
    // long rows take the two-pass form instead: the similarity kernel first
    // stores only the group maxima of every tile (its 128-d products are
    // cheap to compute twice; the values of S are the cost), the threshold is
    // each row's R-th largest group maximum, and the second launch keeps the
    // entries reaching it.  With G groups of 32 in a row, about R of them
    // reach the threshold and the kept entries number about
    // -n ln(1 - R/G) / 32: a scene takes it when G >= 4 R (some 600 entries per
    // 512-list, inside the merge capacity), i.e. from 65,536 objects.
    auto twopass_scene = [&](const Scene &s) {
        if (precision != FARM_PREC_LEARNED || (flags & FARM_UNFUSED) || c.pinned_variant == 1) return false;
        const int64_t Rs = std::min<int64_t>(Rb, s.n);
        const int64_t kt = reduced_keep_target(p, precision, (int32_t)Rs, s.n);
        const int64_t G = farm::group_count(s.n, farm::group_shift_for(s.n));
        return G >= 4 * kt && G <= farm::kMaximaTauKeys;
    };
    const int32_t keep_max = reduced ? std::max(cstride_t, cstride_l) : std::max(stride_t, stride_l);
    const int32_t fs = keep_max <= 128 ? 8 : (keep_max <= 256 ? 4 : 2);
    auto fuse_scene = [&](const Scene &s) {
        if (twopass_scene(s)) return true;
        if (!fusable) return false;
        if (flags & FARM_FUSED) return true;
        if (precision != FARM_PREC_FP32) return false;
        const int64_t Rs = std::min<int64_t>(Rb, s.n);
        return farm::sample_width(s.n, fs) >= 16 * Rs;
    };
    bool fused = false;            // some scene of the batch is fused
    for (const auto &g : groups) fused |= fuse_scene(c.scenes[g.sid]);
    // the length of a scene's selected rows: its sample's when it is fused
    auto sel_len = [&](const Scene &s) {
        return fuse_scene(s) && !twopass_scene(s) ? farm::sample_width(s.n, fs) : s.n;
    };
    int32_t tmp_stride = 4;
    for (const auto &g : groups) {
        const Scene &s = c.scenes[g.sid];
        const int32_t Rs = (int32_t)std::min<int64_t>(Rb, s.n);
        const int32_t klm = (int32_t)std::min<int64_t>(p.k_anchor, s.n);
        const int32_t kt = reduced ? reduced_keep_target(p, precision, Rs, s.n) : Rs;
        const int32_t kl = reduced ? reduced_keep_landmark(p, precision, klm, s.n) : klm;
        if (sel_len(s) > farm::kSelectRowMax)
            tmp_stride = std::max<int32_t>(tmp_stride, (int32_t)round_up(std::max(kt, kl), 4));
    }
    int32_t max_fkeep = 1;
    for (const auto &g : groups) {
        const Scene &s = c.scenes[g.sid];
        const bool fz = fuse_scene(s);
        const bool two = twopass_scene(s);
        const int64_t nsel = sel_len(s);
        // fused: the stored sample tiles, compacted; two-pass: no stored values
        const int64_t ld = two ? 0 : (fz ? farm::col_tiles(s.n, 256, farm::kColSample, fs) * 256 : round_up(s.n, 32));
        const int64_t rows_g = g.nq + g.nc;
        const int32_t Rs = (int32_t)std::min<int64_t>(Rb, s.n);
        const int32_t klm = (int32_t)std::min<int64_t>(p.k_anchor, s.n);
        const int64_t chunk =
            ld == 0 ? rows_g : std::max<int64_t>(1, std::min<int64_t>(rows_g, (int64_t)(kSimCapBytes / (ld * 4))));
        const int gshift = farm::group_shift_for(nsel);
        const int32_t uni = (int32_t)std::min<int64_t>(farm::group_count(nsel, gshift), 8192);
        // long rows of the shared-memory select: column chunks, merged after
        int32_t chunks = 1, chunk_len = (int32_t)nsel;
        bool global_select = false;
        if (nsel > farm::kSelectRowMax) {
            const int64_t c0 = (nsel + farm::kSelectRowMax - 1) / farm::kSelectRowMax;
            chunk_len = (int32_t)round_up((nsel + c0 - 1) / c0, 32);
            chunks = (int32_t)((nsel + chunk_len - 1) / chunk_len);
            global_select = (int64_t)chunks * tmp_stride > farm::kSelectRowMax;
        }
        for (int64_t r0 = 0; r0 < rows_g; r0 += chunk) {
            const int64_t r1 = std::min(rows_g, r0 + chunk);
            const int64_t nr = r1 - r0;
            if (batches.empty() || (batches.back().np > 0 && (batches.back().s_floats + nr * ld) * 4 > (int64_t)kSimCapBytes)) {
                Batch bt;
                bt.p0 = pieces.size();
                batches.push_back(bt);
            }
            Batch &bt = batches.back();
            farm::Piece pc{};
            pc.d32 = s.desc32;
            pc.s_off = bt.s_floats;
            pc.row_begin = bt.rows;
            pc.block_begin = bt.blocks;
            pc.tblock_begin = bt.tblocks;
            pc.q_row0 = g.row0 + r0;
            pc.ntr = (int32_t)std::max<int64_t>(0, std::min<int64_t>(g.nq - r0, nr));
            pc.t_row0 = g.q0 + r0;
            pc.l_row0 = g.cp0 + r0 + pc.ntr - g.nq;
            pc.rows = (int32_t)nr;
            pc.n = (int32_t)nsel;
            pc.n_obj = (int32_t)s.n;
            pc.ld = (int32_t)ld;
            pc.R = Rs;
            pc.klm = klm;
            pc.exact = reduced && exact_scene(s) ? 1 : 0;
            pc.fkeep_t = reduced && !pc.exact ? reduced_keep_target(p, precision, Rs, s.n) : Rs;
            pc.fkeep_l = reduced && !pc.exact ? reduced_keep_landmark(p, precision, klm, s.n) : klm;
            // the select keeps the whole-row lengths, or, fused, as many of them as the sample holds
            pc.keep_t = (int32_t)std::min<int64_t>(pc.fkeep_t, nsel);
            pc.keep_l = (int32_t)std::min<int64_t>(pc.fkeep_l, nsel);
            pc.fs = two ? -1 : (fz ? fs : 0);
            max_fkeep = std::max(max_fkeep, std::max(pc.fkeep_t, pc.fkeep_l));
            pc.tmp_off = -1;
            pc.tops_off = -1;
            // rows [0, th0): shared-memory select; rows [th0, rows): thresholded select
            pc.th0 = pc.rows;
            pc.gshift = gshift;
            if (fz) {
                // (the fused selection's kernels take every row of the piece)
                pc.tops_off = bt.tops;
                bt.tops += nr * farm::group_stride(nsel, gshift);
                bt.fused_rows += nr;
                if (two) {
                    bt.twopass_rows += nr;
                    bt.gmax_twopass = std::max<int32_t>(bt.gmax_twopass, (int32_t)farm::group_count(nsel, gshift));
                }
            } else if (tile_tops) {
                // a row goes to the thresholded select when its group maxima
                // number at least its list length, or it is short enough to sort whole
                const bool small = nsel <= farm::kSelectSortAll;
                pc.th0 = (small || uni >= pc.keep_t) ? 0 : (uni >= pc.keep_l ? pc.ntr : pc.rows);
                pc.tops_off = bt.tops;
                bt.tops += nr * farm::group_stride(nsel, gshift);
                if (pc.th0 < pc.rows) {
                    bt.tblocks += pc.rows - pc.th0;
                    bt.max_union = std::max(bt.max_union, uni);
                }
            }
            pc.chunks = fz ? 1 : (global_select ? 0 : chunks);
            pc.chunk_len = global_select ? (int32_t)s.n : chunk_len;
            if (fz) pc.th0 = pc.rows;     // no select of the unfused path
            if (pc.th0 > 0 && !global_select && !fz) {
                bt.blocks += (int64_t)pc.th0 * pc.chunks;
                bt.smem_sel = std::max(bt.smem_sel, pc.chunk_len);
                if (pc.chunks > 1) {
                    pc.tmp_off = bt.tmp;
                    bt.tmp += (int64_t)pc.th0 * pc.chunks * tmp_stride;
                    bt.chunked = true;
                    bt.smem_merge = std::max(bt.smem_merge, pc.chunks * tmp_stride);
                }
            }
            bt.s_floats += nr * ld;
            bt.rows += nr;
            if (pc.exact) bt.exact_rows += nr;
            bt.np += 1;
            pieces.push_back(pc);
            piece_sid.push_back(g.sid);
        }
    }
    int64_t s_need = 1, tmp_need = 4, tops_need = 4;
    for (const auto &bt : batches) {
        s_need = std::max(s_need, bt.s_floats);
        tmp_need = std::max(tmp_need, bt.tmp);
        tops_need = std::max(tops_need, bt.tops);
    }
    float *d_sim, *tmp_val = nullptr, *d_tops = nullptr;
    int32_t *tmp_idx = nullptr;
    CK(ws_get(ctx, farm::B_SIM, (size_t)s_need, &d_sim));
    if (tile_tops) CK(ws_get(ctx, farm::B_TOPS, (size_t)tops_need, &d_tops));
    bool any_chunked = false;
    int64_t tblocks_max = 1;
    for (const auto &bt : batches) {
        any_chunked |= bt.chunked;
        tblocks_max = std::max(tblocks_max, bt.tblocks);
    }
    int32_t *d_rowlist;
    CK(ws_get(ctx, farm::B_SELLIST, (size_t)tblocks_max + 1, &d_rowlist));
    if (any_chunked) {
        CK(ws_get(ctx, farm::B_CHUNK_IDX, (size_t)tmp_need, &tmp_idx));
        CK(ws_get(ctx, farm::B_CHUNK_VAL, (size_t)tmp_need, &tmp_val));
    }
    // the fused selection's buffers (per operand row) and the landmark list values it ranks by
    farm::FuseEmit emit{};
    int32_t *d_ovf = nullptr;
    float *d_slab = nullptr, *lsel_cos = nullptr;
    if (fused) {
        emit.cap = farm::fuse_merge_capacity(max_fkeep);
        CK(ws_get(ctx, farm::B_FUSE_TAU, (size_t)rows_total, &emit.tau_key));
        CK(ws_get(ctx, farm::B_FUSE_CNT, (size_t)rows_total, &emit.cnt));
        CK(ws_get(ctx, farm::B_FUSE_CAND, (size_t)rows_total * emit.cap, &emit.cand));
        CK(ws_get(ctx, farm::B_FUSE_OVF, 2 * (size_t)rows_total + 2, &d_ovf));
        CK(ws_get(ctx, farm::B_FUSE_SLAB, (size_t)farm::kFuseFallbackBlocks * round_up(max_n, 4), &d_slab));
        if (!reduced) CK(ws_get(ctx, farm::B_LSEL_COS, (size_t)std::max<int64_t>(n_c, 1) * stride_l, &lsel_cos));
        if (precision == FARM_PREC_LEARNED) {
            // the sample lists' values give the thresholds
            CK(ws_get(ctx, farm::B_BSEL_TV, (size_t)n_q * cstride_t, &bsel_tv));
            CK(ws_get(ctx, farm::B_BSEL_LV, (size_t)std::max<int64_t>(n_c, 1) * cstride_l, &bsel_lv));
        }
    }
    // tensor-core similarity: one grouped launch per batch over its pieces
    // (fused: two, the sample tiles and the others); each scene's two B
    // tensor maps are encoded once per call
    if (sim_mode >= 0 && !farm::sim_tc_available())
        return fail(ctx, FARM_EINVAL, "the tensor-core similarity path is not built");
    std::vector<int32_t> map_of_scene;
    std::vector<int32_t> map_scenes;
    if (precision == FARM_PREC_LEARNED)     // (re)computes the scenes' learned embeddings the maps point at
        for (const auto &g : groups) CK(farm::learned_refresh_scene(ctx, g.sid));
    if (sim_mode >= 0) {
        map_of_scene.assign(kMaxScenes, -1);
        for (const auto &g : groups)
            if (map_of_scene[g.sid] < 0) {
                map_of_scene[g.sid] = (int32_t)map_scenes.size();
                map_scenes.push_back(g.sid);
            }
    }
    // tile variant of the grouped similarity: the autotuner's choice for this
    // class of batch (mode, total rows, mean objects per row, each to a power
    // of two), or, the first time, every variant timed on the first
    // similarity batch (a graph is captured only once the class is tuned)
    std::vector<int> vlist = {0};
    int64_t tune_key = -1;
    if (sim_mode >= 0) {
        double wn = 0.0;
        for (const auto &g : groups) wn += (double)(g.nq + g.nc) * (double)c.scenes[g.sid].n;
        auto log2i = [](int64_t x) { int b = 0; while (b < 62 && (int64_t(1) << (b + 1)) <= x) ++b; return b; };
        tune_key = (any_exact ? 200000 : 0) + (fused ? 100000 : 0) + (int64_t)sim_mode * 10000 +
                   log2i(rows_total) * 100 +
                   log2i((int64_t)(wn / (double)rows_total));
        auto it = c.tuned.find(tune_key);
        if (c.pinned_variant >= 0) {
            vlist = {c.pinned_variant};
        } else if (it != c.tuned.end()) {
            vlist = {it->second};
        } else {
            vlist = fused ? std::vector<int>{0, 2} : std::vector<int>{0, 1, 2};     // fused: tiles of 256 objects
            graph = false;
        }
    }
    const int nv = (int)vlist.size();
    // device blob: select pieces | GEMM pieces, one table per variant | tensor maps (128-byte aligned sections)
    const size_t off_gp = round_up((int64_t)(pieces.size() * sizeof(farm::Piece)), 128);
    const size_t gp_table = round_up((int64_t)(pieces.size() * sizeof(farm::GemmPiece)), 128);
    // fused: the sample tiles' table, then the others'; a reduced-precision
    // batch with FP32-accurate scenes: its own pieces' table, then theirs
    const int n_tables = fused || any_exact ? 2 : 1;
    const size_t off_maps = off_gp + nv * n_tables * gp_table;
    const size_t blob_bytes = off_maps + map_scenes.size() * nv * 2 * farm::kTensorMapBytes;
    uint8_t *d_blob;
    CK(ws_get(ctx, farm::B_PIECES, blob_bytes, &d_blob));
    if (ctx->h_blob_n < blob_bytes) {
        if (ctx->h_blob) cudaFreeHost(ctx->h_blob);
        ctx->h_blob = nullptr;
        ctx->h_blob_n = 0;
        CK(cudaHostAlloc(&ctx->h_blob, blob_bytes * 5 / 4 + 256, cudaHostAllocDefault));
        ctx->h_blob_n = blob_bytes * 5 / 4 + 256;
    }
    farm::Piece *d_pieces = reinterpret_cast<farm::Piece *>(d_blob);
    std::memcpy(ctx->h_blob, pieces.data(), pieces.size() * sizeof(farm::Piece));
    // tiles of batch b, variant vi, table t at batch_tiles[(b * nv + vi) * n_tables + t]
    std::vector<int64_t> batch_tiles(batches.size() * nv * n_tables, 0);
    auto gp_base = [&](int vi, int t) { return off_gp + (size_t)(vi * n_tables + t) * gp_table; };
    if (sim_mode >= 0) {
        for (int vi = 0; vi < nv; ++vi) {
            for (int t = 0; t < n_tables; ++t) {
                farm::GemmPiece *hg = reinterpret_cast<farm::GemmPiece *>(ctx->h_blob + gp_base(vi, t));
                for (size_t b = 0; b < batches.size(); ++b) {
                    int64_t tiles = 0;
                    for (size_t k = batches[b].p0; k < batches[b].p0 + batches[b].np; ++k) {
                        const farm::Piece &pc = pieces[k];
                        const Scene &sc = c.scenes[piece_sid[k]];
                        // fused pieces: their sample tiles (table 0), the others (table 1);
                        // two-pass pieces: every tile's group maxima (table 0), every tile
                        // emitting (table 1); the others' pieces: every tile (table 0), none
                        // (table 1); in a batch with FP32-accurate scenes (never fused)
                        // theirs are table 1's
                        const int mode = any_exact ? ((t == 1) == (pc.exact != 0) ? farm::kColAll : -1)
                                         : pc.fs == 0 ? (t == 0 ? farm::kColAll : -1)
                                         : pc.fs < 0  ? farm::kColAll
                                                      : (t == 0 ? farm::kColSample : farm::kColRest);
                        farm::GemmPiece gp{};
                        gp.q_row0 = pc.q_row0;
                        gp.s_off = pc.fs < 0 ? -1 : (mode == farm::kColRest ? 0 : pc.s_off);
                        gp.tops_off = (tile_tops && mode != farm::kColRest && !(pc.fs < 0 && t == 1)) ? pc.tops_off : -1;
                        gp.scale_d = sim_mode == farm::kSimFp8 && !pc.exact ? sc.desc_scale : nullptr;
                        gp.bmap = d_blob + off_maps +
                                  ((size_t)map_of_scene[piece_sid[k]] * nv + vi) * 2 * farm::kTensorMapBytes;
                        gp.rows = pc.rows;
                        gp.n = pc.n_obj;
                        gp.ld = pc.ld;
                        gp.tile_begin = (int32_t)tiles;
                        gp.gshift = pc.gshift;
                        gp.col_mode = mode < 0 ? farm::kColRest : mode;
                        gp.col_stride = fs;
                        gp.n_store = mode == farm::kColAll || mode == farm::kColSample ? pc.n : 0;
                        if (mode >= 0) tiles += farm::sim_cluster_tiles(pc.rows, pc.n_obj, vlist[vi], mode, fs);
                        hg[k] = gp;
                    }
                    if (tiles > 0x7fffffffLL) return fail(ctx, FARM_EINVAL, "similarity batch exceeds 2^31 tiles");
                    batch_tiles[((size_t)b * nv + vi) * n_tables + t] = tiles;
                }
            }
        }
        for (size_t m = 0; m < map_scenes.size(); ++m) {
            const Scene &sc = c.scenes[map_scenes[m]];
            for (int vi = 0; vi < nv; ++vi) {
                void *out = ctx->h_blob + off_maps + (m * nv + vi) * 2 * farm::kTensorMapBytes;
                bool ok;
                if (precision == FARM_PREC_FP32 || (reduced && exact_scene(sc)))
                    ok = farm::sim_tc_encode_b(farm::kSimF16x3, vlist[vi], out, sc.desc_hi, sc.desc_lo, sc.n,
                                               sc.dim_pad);
                else if (precision == FARM_PREC_BF16)
                    ok = farm::sim_tc_encode_b(sim_mode, vlist[vi], out, sc.desc_bf16, nullptr, sc.n, sc.dim_pad);
                else if (precision == FARM_PREC_LEARNED)
                    ok = farm::sim_tc_encode_b(sim_mode, vlist[vi], out, sc.comp, nullptr, sc.n, c.mlp.P);
                else
                    ok = farm::sim_tc_encode_b(sim_mode, vlist[vi], out, sc.desc_fp8, nullptr, sc.n, sc.dim_pad);
                if (!ok)
                    return fail(ctx, FARM_ECUDA, "tensor map encoding failed for scene " + std::to_string(map_scenes[m]));
            }
        }
    }

    // The batch's device work, in stream order: run directly, or captured
    // into a CUDA graph (FARM_GRAPH), in which case everything it reads was
    // staged into library buffers first.
    const float *src_t = dev ? tgt_emb : d_raw;
    const float *src_c = dev ? c_emb : d_raw + (size_t)n_q * dim;
    // Staging copies, always issued directly on the stream (never inside a
    // graph): the host refills the pinned buffers for its next batch once the
    // stage_done event after them has completed.  (Stage marks are taken for
    // batches run directly only.)
    const int m0 = graph ? -1 : mark_begin(ctx, 0);
    CK(cudaMemcpyAsync(d_rowmap, h_rowmap, (size_t)(n_q + n_c) * 4, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(d_perm, h_perm, (size_t)n_q * 4, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(d_meta, h_meta, (size_t)n_q * 8 * 4, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(d_blob, ctx->h_blob, blob_bytes, cudaMemcpyHostToDevice, c.stream));
    CK(cudaEventRecord(ctx->stage_done, c.stream));
    if (!dev) CK(copy_host_rows(ctx, raw_slot, d_raw, tgt_emb, c_emb, n_q, n_c, dim));
    auto enqueue = [&]() -> farm_status {
        // ---- stage 0: normalisation (the staging copies above are not part of it)
        // (with FP32-accurate scenes in a reduced-precision batch, their rows
        // -- the last ones -- get the FP16 split only, the others no split)
        const int64_t split = any_exact ? exact_row0 : -1;
        LAUNCH(farm::launch_normalize_rows(src_t, d_rowmap, n_q, dim, dim_pad, ops.q32, ops.qhi, ops.qlo, ops.qbf,
                                           c.d_err, farm::kErrBadRow, c.stream, split));
        if (n_c > 0)
            LAUNCH(farm::launch_normalize_rows(src_c, d_rowmap + n_q, n_c, dim, dim_pad, ops.q32, ops.qhi, ops.qlo,
                                               ops.qbf, c.d_err, farm::kErrBadRow, c.stream, split));
        if (precision == FARM_PREC_FP8)
            LAUNCH(farm::launch_quantize_fp8_rows(ops.q32, exact_row0, dim_pad, ops.qf8, ops.qscale, c.stream));
        if (precision == FARM_PREC_LEARNED) CK(farm::learned_embed_rows(ctx, ops.qbf, rows_total, ops.qcomp));
        mark_end(ctx, m0);

        // ---- stages 1-2: similarity per piece, then the batch's rank selection
        int32_t *sel_ti = reduced ? bsel_t : tsel_idx, *sel_li = reduced ? bsel_l : lsel_idx;
        float *sel_tc = reduced ? bsel_tv : tsel_cos, *sel_lc = reduced ? bsel_lv : lsel_cos;
        const int32_t sel_st = reduced ? cstride_t : stride_t, sel_sl = reduced ? cstride_l : stride_l;
        int vsel = nv == 1 ? 0 : -1;     // index into vlist of the variant in use
        for (size_t b = 0; b < batches.size(); ++b) {
            const Batch &bt = batches[b];
            const int m1 = mark_begin(ctx, 1);
            const void *q0 = nullptr, *q1 = nullptr;
            int32_t kdim = dim_pad;
            if (precision == FARM_PREC_FP32) { q0 = ops.qhi; q1 = ops.qlo; }
            else if (precision == FARM_PREC_BF16) q0 = ops.qbf;
            else if (precision == FARM_PREC_LEARNED) { q0 = ops.qcomp; kdim = c.mlp.P; }
            else q0 = ops.qf8;
            // table t of variant vi (fused: 0 the sample tiles, 1 the others, appending to
            // the rows' buffers; with FP32-accurate scenes: 1 theirs, in that mode)
            auto launch_variant = [&](int vi, int t) {
                const bool ex = any_exact && t == 1;
                return farm::launch_sim_tc_grouped(
                    ex ? farm::kSimF16x3 : sim_mode, vlist[vi], ex ? ops.qhi : q0, ex ? ops.qlo : q1, rows_total,
                    kdim, reinterpret_cast<farm::GemmPiece *>(d_blob + gp_base(vi, t)) + bt.p0, (int32_t)bt.np,
                    batch_tiles[((size_t)b * nv + vi) * n_tables + t], d_sim, tile_tops ? d_tops : nullptr,
                    precision == FARM_PREC_FP8 && !ex ? ops.qscale : nullptr, c.num_sms, c.d_err, c.stream,
                    fused && t == 1 ? &emit : nullptr);
            };
            // the tables launched before the selection (fused: the sample tiles only)
            const int n_now = fused ? 1 : n_tables;
            if (sim_mode >= 0) {
                if (vsel < 0) {
                    // autotune: every variant twice, the second run timed (fused:
                    // both launches, the second with no threshold reached, so
                    // that it appends nothing); the sample tiles' values are
                    // the same whichever variant stores them last
                    cudaEvent_t e0, e1;
                    CK(cudaEventCreate(&e0));
                    CK(cudaEventCreate(&e1));
                    if (fused) {
                        CK(cudaMemsetAsync(emit.tau_key, 0xff, (size_t)rows_total * 4, c.stream));
                        CK(cudaMemsetAsync(emit.cnt, 0, (size_t)rows_total * 4, c.stream));
                    }
                    float best_ms = 0.f;
                    for (int vi = 0; vi < nv; ++vi) {
                        for (int rep = 0; rep < 2; ++rep) {
                            if (rep == 1) CK(cudaEventRecord(e0, c.stream));
                            for (int t = 0; t < n_tables; ++t) LAUNCH(launch_variant(vi, t));
                        }
                        CK(cudaEventRecord(e1, c.stream));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        if (vsel < 0 || ms < best_ms) {
                            best_ms = ms;
                            vsel = vi;
                        }
                    }
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    c.tuned[tune_key] = vlist[vsel];
                    // the batch's results come from the chosen variant, as every later batch's will
                    if (fused || vsel != nv - 1)
                        for (int t = 0; t < n_now; ++t) LAUNCH(launch_variant(vsel, t));
                } else {
                    for (int t = 0; t < n_now; ++t) LAUNCH(launch_variant(vsel, t));
                }
            } else {
                for (size_t k = bt.p0; k < bt.p0 + bt.np; ++k) {
                    const farm::Piece &pc = pieces[k];
                    farm_status st = run_similarity(ctx, precision, ops, pc.q_row0, pc.rows, c.scenes[piece_sid[k]],
                                                    d_sim + pc.s_off, pc.ld, nullptr);
                    if (st != FARM_OK) return st;
                }
            }
            mark_end(ctx, m1);
            const int m2 = mark_begin(ctx, 2);
            const farm::Piece *dp = d_pieces + bt.p0;
            if (bt.fused_rows > bt.twopass_rows) {
                // each row's threshold from its sample's group maxima; the sample's entries reaching it
                LAUNCH(farm::launch_fuse_sample_tau(d_sim, d_tops, dp, (int32_t)bt.np, bt.rows, emit, c.stream));
            }
            if (bt.twopass_rows > 0) {
                // two-pass rows: each row's threshold from the group maxima of its whole row
                LAUNCH(farm::launch_fuse_maxima_tau(d_tops, dp, (int32_t)bt.np, bt.rows, emit, bt.gmax_twopass,
                                                    c.stream));
            }
            if (bt.blocks > 0)
                LAUNCH(farm::launch_select_grouped(d_sim, dp, (int32_t)bt.np, bt.blocks, bt.smem_sel, sel_ti, sel_tc,
                                                   sel_st, sel_li, sel_lc, sel_sl, tmp_idx, tmp_val, tmp_stride,
                                                   c.stream));
            if (bt.chunked)
                LAUNCH(farm::launch_merge_chunks(dp, (int32_t)bt.np, bt.rows, bt.smem_merge, tmp_idx, tmp_val, tmp_stride,
                                                 sel_ti, sel_tc, sel_st, sel_li, sel_lc, sel_sl, c.stream));
            if (bt.tblocks > 0)
                LAUNCH(farm::launch_select_thresh(d_sim, d_tops, dp, (int32_t)bt.np, bt.tblocks, bt.max_union, sel_ti,
                                                  sel_tc, sel_st, sel_li, sel_lc, sel_sl, c.d_fallback, d_rowlist,
                                                  c.stream));
            for (size_t k = bt.p0; k < bt.p0 + bt.np; ++k) {
                const farm::Piece &pc = pieces[k];
                if (pc.fs != 0 || pc.chunks != 0 || pc.th0 == 0) continue;
                LAUNCH(farm::launch_select_rows_ex(d_sim + pc.s_off, pc.ld, pc.n, pc.th0, pc.ntr, pc.keep_t, pc.keep_l,
                                                   sel_ti, sel_tc, pc.t_row0, sel_st, sel_li, sel_lc, pc.l_row0, sel_sl,
                                                   c.stream));
            }
            if (bt.fused_rows > 0) {
                // the other tiles append what reaches the thresholds; the merge, and
                // the exact recomputation of rows whose candidates overflowed
                mark_end(ctx, m2);
                const int m1b = mark_begin(ctx, 1);
                CK(cudaMemsetAsync(d_ovf, 0, 2 * sizeof(int32_t), c.stream));
                LAUNCH(launch_variant(vsel, 1));
                mark_end(ctx, m1b);
                const int m2b = mark_begin(ctx, 2);
                LAUNCH(farm::launch_fuse_final(dp, (int32_t)bt.np, bt.rows, sel_ti, sel_tc, sel_st, sel_li, sel_lc,
                                               sel_sl, emit, d_ovf, d_ovf + 2, d_ovf + 1, d_ovf + 2 + rows_total,
                                               max_fkeep, c.stream));
                LAUNCH(farm::launch_fuse_fallback(dp, (int32_t)bt.np, d_ovf, d_ovf + 2,
                                                  precision == FARM_PREC_FP32 ? nullptr : ops.q32, ops.qhi, ops.qlo,
                                                  dim_pad, sel_ti, sel_tc, sel_st, sel_li, sel_lc, sel_sl, d_slab,
                                                  round_up(max_n, 4), farm::kFuseFallbackBlocks, c.d_fallback,
                                                  c.stream));
                mark_end(ctx, m2b);
            }
            const int m2c = bt.fused_rows > 0 ? mark_begin(ctx, 2) : -1;
            if (reduced) {
                const float band = precision == FARM_PREC_FP8 ? 16.f * p.rescore_band : p.rescore_band;
                // (the learned path's list values are compressed-space scores: no band)
                // (the rows of FP32-accurate scenes, the batch's last ones, are final: copied)
                LAUNCH(farm::launch_copy_lists(dp, (int32_t)bt.np, bt.rows - bt.exact_rows, bt.exact_rows, bsel_t,
                                               bsel_tv, cstride_t, bsel_l, cstride_l, tsel_idx, tsel_cos, stride_t,
                                               lsel_idx, stride_l, c.stream));
                LAUNCH(farm::launch_rescore_grouped(dp, (int32_t)bt.np, bt.rows - bt.exact_rows, ops.q32, dim_pad, bsel_t,
                                                    precision == FARM_PREC_LEARNED ? nullptr : bsel_tv, cstride_t,
                                                    bsel_l, precision == FARM_PREC_LEARNED ? nullptr : bsel_lv,
                                                    cstride_l, band, tsel_idx, tsel_cos, stride_t, lsel_idx, stride_l,
                                                    c.d_err, c.stream));
            }
            mark_end(ctx, bt.fused_rows > 0 ? m2c : m2);
        }

        // ---- stage 3: relations, composite, sort
        const int m3 = mark_begin(ctx, 3);
        farm::ComposeArgs ca;
        ca.n_q = n_q;
        ca.qmeta = d_meta;
        ca.tsel_idx = tsel_idx;
        ca.lsel_idx = lsel_idx;
        ca.stride_t = stride_t;
        ca.stride_l = stride_l;
        ca.scenes = ctx->d_scenes;
        ca.p = p;
        ca.out_idx = o_idx;
        ca.out_score = o_score;
        ca.out_t = o_t;
        ca.out_anchor = o_anc;
        LAUNCH(farm::launch_compose(ca, c.stream));
        mark_end(ctx, m3);
        return FARM_OK;
    };

    std::vector<int64_t> graph_key;
    if (!graph) {
        const farm_status st = enqueue();
        if (st != FARM_OK) return st;
    } else {
        // the batch's shape: everything that fixes the launch sequence and its
        // arguments (device inputs are read where the caller keeps them)
        std::vector<int64_t> key = {precision, (int64_t)(flags & (FARM_FUSED | FARM_UNFUSED)), n_q, n_c, dim, (int64_t)c.ws_gen, (int64_t)c.scene_gen,
                                    (int64_t)c.mlp.version, (int64_t)(intptr_t)src_t, (int64_t)(intptr_t)src_c,
                                    (int64_t)c.pinned_variant, (int64_t)groups.size()};
        for (const auto &g : groups) {
            key.push_back(g.sid);
            key.push_back(g.nq);
            key.push_back(g.nc);
        }
        graph_key = key;
        farm_ctx::GraphEntry *hit = nullptr;
        for (auto &ge : ctx->graphs)
            if (ge.key == key) hit = &ge;
        if (!hit) {
            const int64_t launches0 = c.launches;
            CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeRelaxed));
            ctx->capturing = true;
            const farm_status st = enqueue();
            ctx->capturing = false;
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(c.stream, &g);
            if (st != FARM_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (ec != cudaSuccess) return fail(ctx, FARM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
            cudaGraphExec_t exec = nullptr;
            const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) return fail(ctx, FARM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
            if (ctx->graphs.size() >= 8) {
                auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                            [](const farm_ctx::GraphEntry &x, const farm_ctx::GraphEntry &y) {
                                                return x.used < y.used;
                                            });
                cudaGraphExecDestroy(lru->exec);
                ctx->graphs.erase(lru);
            }
            farm_ctx::GraphEntry ge;
            ge.key = std::move(key);
            ge.exec = exec;
            ge.launches = c.launches - launches0;
            ctx->graphs.push_back(std::move(ge));
            hit = &ctx->graphs.back();
            c.launches = launches0;
        }
        hit->used = ++ctx->graph_clock;
        CK(cudaGraphLaunch(hit->exec, c.stream));
        c.launches += hit->launches;
    }
    if (!dev) CK(cudaEventRecord(ctx->ev_slot_free[raw_slot], c.stream));   // the batch is done with its slot

    c.batch_gen += 1;
    c.batch_valid = true;
    c.batch_nq = n_q;
    c.batch_nc = n_c;
    c.batch_rtgt = stride_t;
    c.batch_klm = stride_l;
    c.batch_min_n = (int32_t)std::min<int64_t>(min_n, 0x7fffffff);
    *batch_handle = c.batch_gen;
    if (graph && !graph_key.empty()) {
        // record the batch for replay (its other slot's graph stays usable
        // when the query graphs are the same as the record's)
        farm_ctx::Replay &r = ctx->replay;
        if (!replay_same(ctx, n_q, scene_of_q, tgt_emb, tgt_cls, c_off, c_pred, c_emb, precision, flags)) {
            r.precision = precision;
            r.flags = flags;
            r.n_q = n_q;
            r.n_c = n_c;
            r.pinned = c.pinned_variant;
            r.ws_gen = c.ws_gen;
            r.scene_gen = c.scene_gen;
            r.mlp_version = c.mlp.version;
            r.src_t = dev ? tgt_emb : nullptr;
            r.src_c = dev ? c_emb : nullptr;
            r.scene_of_q.assign(scene_of_q, scene_of_q + n_q);
            r.tgt_cls.assign(tgt_cls, tgt_cls + n_q);
            r.c_off.assign(c_off, c_off + n_q + 1);
            r.c_pred.assign(c_pred, c_pred + n_c);
            r.key[0].clear();
            r.key[1].clear();
        }
        r.dim = dim;
        r.key[dev ? 0 : raw_slot] = graph_key;
        r.rtgt = stride_t;
        r.klm = stride_l;
        r.min_n = c.batch_min_n;
        r.valid = true;
    }
    return FARM_OK;
}

farm_status farm_memory_add_space(farm_ctx *ctx, int32_t scene_id, int32_t space, int32_t dim, const float *desc,
                                  uint32_t flags)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (scene_id < 0 || scene_id >= kMaxScenes || !c.scenes[scene_id].present)
        return fail(ctx, FARM_EINVAL, "unknown scene");
    if (space < 1 || space >= FARM_MAX_SPACES) return fail(ctx, FARM_EINVAL, "space must lie in [1, FARM_MAX_SPACES)");
    if (dim < 1 || dim > 8192) return fail(ctx, FARM_EINVAL, "dim must lie in [1, 8192]");
    if (!desc) return fail(ctx, FARM_EINVAL, "desc must be non-null");
    Scene &s = c.scenes[scene_id];
    const int64_t n = s.n;
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    if (!dev) {
        for (int64_t j = 0; j < n; ++j) {
            double ss = 0.0;
            const float *d = desc + j * dim;
            for (int32_t k = 0; k < dim; ++k) ss += (double)d[k] * (double)d[k];
            if (!(ss > 0.0) || !std::isfinite(ss))
                return fail(ctx, FARM_EINVAL, "descriptor row " + std::to_string(j) + " has zero or non-finite norm");
        }
    }
    CK(cudaSetDevice(c.device));
    CK(cudaStreamSynchronize(c.stream));
    farm::SpaceDesc &sp = s.spaces[space];
    cudaFree(sp.hi);
    cudaFree(sp.lo);
    sp = farm::SpaceDesc{};
    farm::SpaceDesc ns;
    ns.dim = dim;
    ns.dim_pad = (int32_t)round_up(dim, farm::kDimAlign);
    const size_t nd = (size_t)n * ns.dim_pad;
    auto bail = [&](cudaError_t e) {
        cudaFree(ns.hi);
        cudaFree(ns.lo);
        return fail(ctx, e == cudaErrorMemoryAllocation ? FARM_ENOMEM : FARM_ECUDA,
                    std::string("space upload: ") + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&ns.hi, nd * 2)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&ns.lo, nd * 2)) != cudaSuccess) return bail(e);
    const float *d_desc = desc;
    float *tmp = nullptr;
    if (!dev) {
        if ((e = cudaMallocAsync(&tmp, (size_t)n * dim * 4, c.stream)) != cudaSuccess) return bail(e);
        if ((e = cudaMemcpyAsync(tmp, desc, (size_t)n * dim * 4, cudaMemcpyHostToDevice, c.stream)) != cudaSuccess)
            return bail(e);
        d_desc = tmp;
    }
    c.launches += 1;
    if ((e = farm::launch_normalize_rows(d_desc, nullptr, n, dim, ns.dim_pad, nullptr, ns.hi, ns.lo, nullptr, c.d_err,
                                         farm::kErrBadDesc, c.stream)) != cudaSuccess)
        return bail(e);
    if (tmp) cudaFreeAsync(tmp, c.stream);
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return bail(e);
    sp = ns;
    c.batch_valid = false;
    c.scene_gen += 1;
    return FARM_OK;
}

farm_status farm_query_batch_rrf(farm_ctx *ctx, int32_t scene_id, int64_t n_q, int32_t n_ch,
                                 const farm_channel *ch, const float *tgt_emb, const int32_t *tgt_cls,
                                 const int32_t *c_off, const int32_t *c_pred, const float *c_emb, uint32_t flags,
                                 uint64_t *batch_handle)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (!batch_handle) return fail(ctx, FARM_EINVAL, "batch_handle must be non-null");
    if (flags & FARM_GRAPH) return fail(ctx, FARM_EINVAL, "FARM_GRAPH is not supported for fused batches");
    ctx->replay.valid = false;       // this batch rewrites the staging buffers
    if (scene_id < 0 || scene_id >= kMaxScenes || !c.scenes[scene_id].present)
        return fail(ctx, FARM_EINVAL, "unknown scene");
    if (n_q < 1 || n_q > 0x7fffffff) return fail(ctx, FARM_EINVAL, "n_q must lie in [1, 2^31)");
    if (n_ch < 1 || n_ch > FARM_MAX_CHANNELS || !ch) return fail(ctx, FARM_EINVAL, "n_ch must lie in [1, 4]");
    if (!tgt_emb || !tgt_cls || !c_off) return fail(ctx, FARM_EINVAL, "tgt_emb, tgt_cls and c_off must be non-null");
    if (!farm::sim_tc_available()) return fail(ctx, FARM_EINVAL, "the tensor-core similarity path is not built");
    const Scene &s = c.scenes[scene_id];
    const farm_params &p = c.params;
    const int64_t n = s.n;
    int32_t dims[FARM_MAX_CHANNELS], dpad[FARM_MAX_CHANNELS];
    const uint16_t *dhi[FARM_MAX_CHANNELS], *dlo[FARM_MAX_CHANNELS];
    double W = 0.0, wmax = 0.0;
    for (int32_t k = 0; k < n_ch; ++k) {
        const int32_t sp = ch[k].space;
        if (sp < 0 || sp >= FARM_MAX_SPACES) return fail(ctx, FARM_EINVAL, "channel space out of range");
        if (!(ch[k].weight > 0.f) || !std::isfinite(ch[k].weight))
            return fail(ctx, FARM_EINVAL, "channel weights must be positive and finite");
        if (sp == 0) {
            dims[k] = s.dim; dpad[k] = s.dim_pad; dhi[k] = s.desc_hi; dlo[k] = s.desc_lo;
        } else {
            if (!s.spaces[sp].hi) return fail(ctx, FARM_EINVAL, "channel names a space the scene does not hold");
            dims[k] = s.spaces[sp].dim; dpad[k] = s.spaces[sp].dim_pad; dhi[k] = s.spaces[sp].hi; dlo[k] = s.spaces[sp].lo;
        }
        W += ch[k].weight;
        wmax = std::max(wmax, (double)ch[k].weight);
    }
    if (c_off[0] != 0) return fail(ctx, FARM_EINVAL, "c_off[0] must be 0");
    for (int64_t q = 0; q < n_q; ++q) {
        const int32_t m = c_off[q + 1] - c_off[q];
        if (m < 0 || m > FARM_MAX_CONSTRAINTS)
            return fail(ctx, FARM_EINVAL, "query " + std::to_string(q) + " has more than 4 constraints");
    }
    const int64_t n_c = c_off[n_q];
    if (n_c > 0 && (!c_pred || !c_emb)) return fail(ctx, FARM_EINVAL, "c_pred and c_emb must be non-null");
    {
        std::string why;
        for (int64_t q = 0; q < n_q; ++q)
            if (!preds_ok(c_pred + c_off[q], c_off[q + 1] - c_off[q], why))
                return fail(ctx, FARM_EINVAL, "query " + std::to_string(q) + ": " + why);
    }
    if (p.k_max > n) return fail(ctx, FARM_EINVAL, "k_max exceeds the scene's object count");
    // list depths: an object no channel lists fuses to at most W / (mu + R + 1);
    // keep that below the k_max-th composite's floor (1 - w) class_mis wmax / (mu + k_max),
    // the k_closest-th fused score's floor wmax / (mu + k_closest) and, for
    // landmark rows, the K_a-th fused score's floor wmax / (mu + K_a)
    const double mu = p.mu;
    const double bt = std::min((1.0 - p.w) * p.class_mis * wmax / (mu + p.k_max), wmax / (mu + p.k_closest));
    const double bl = wmax / (mu + p.k_anchor);
    const int64_t Rt_need = (int64_t)std::floor(W / bt - mu - 1.0) + 2;
    const int64_t Rl_need = (int64_t)std::floor(W / bl - mu - 1.0) + 2;
    if (Rt_need > farm::kMaxTargetCands || Rl_need > farm::kMaxAnchorCands)
        return fail(ctx, FARM_EINVAL, "channel weights too uneven: the per-channel lists would exceed 512 / 256");
    const int32_t Rt = (int32_t)std::min<int64_t>(std::max<int64_t>(Rt_need, p.k_max), n);
    const int32_t Rl = (int32_t)std::min<int64_t>(std::max<int64_t>(Rl_need, p.k_anchor), n);
    const int32_t Ka = (int32_t)std::min<int64_t>(p.k_anchor, n);
    const int32_t RF = (int32_t)std::min<int64_t>(farm::kMaxTargetCands, n);
    const int64_t rows = n_q + n_c;
    const int64_t ld = round_up(n, 32);
    const int gshift = farm::group_shift_for(n);
    const int64_t gstride = farm::group_stride(n, gshift);
    const double s_bytes = (double)n_ch * rows * ld * 4.0;
    if (s_bytes > 32.0 * (1ull << 30)) return fail(ctx, FARM_EINVAL, "fused batch too large (similarity blocks > 32 GiB)");
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;    // (zero or non-finite rows are caught on the GPU)
    c.batch_valid = false;
    *batch_handle = 0;
    CK(cudaSetDevice(c.device));

    // ---- buffers
    int32_t dmax = 0;
    int64_t emb_t = 0, emb_c = 0;
    for (int32_t k = 0; k < n_ch; ++k) {
        dmax = std::max(dmax, dpad[k]);
        emb_t += n_q * dims[k];
        emb_c += n_c * dims[k];
    }
    uint16_t *qhi, *qlo;
    float *d_sim, *d_tops, *d_fused, *d_raw = nullptr;
    int32_t *d_tl, *d_ll, *d_meta, *d_perm, *tsel_idx, *lsel_idx, *o_idx, *o_anc;
    float *o_score, *o_t;
    CK(ws_get(ctx, farm::B_QHI, (size_t)rows * dmax, &qhi));
    CK(ws_get(ctx, farm::B_QLO, (size_t)rows * dmax, &qlo));
    CK(ws_get(ctx, farm::B_MC_SIM, (size_t)(n_ch * rows * ld), &d_sim));
    CK(ws_get(ctx, farm::B_MC_TOPS, (size_t)(n_ch * rows * gstride), &d_tops));
    CK(ws_get(ctx, farm::B_MC_TLIST, (size_t)(n_ch * n_q * Rt), &d_tl));
    CK(ws_get(ctx, farm::B_MC_LLIST, (size_t)std::max<int64_t>(n_ch * n_c * Rl, 1), &d_ll));
    CK(ws_get(ctx, farm::B_MC_FUSED, (size_t)(n_q * RF), &d_fused));
    CK(ws_get(ctx, farm::B_QMETA, (size_t)n_q * 8, &d_meta));
    CK(ws_get(ctx, farm::B_PERM, (size_t)n_q, &d_perm));
    CK(ws_get(ctx, farm::B_TSEL_IDX, (size_t)n_q * RF, &tsel_idx));
    CK(ws_get(ctx, farm::B_LSEL_IDX, (size_t)std::max<int64_t>(n_c, 1) * Ka, &lsel_idx));
    CK(ws_get(ctx, farm::B_OUT_IDX, (size_t)n_q * RF, &o_idx));
    CK(ws_get(ctx, farm::B_OUT_SCORE, (size_t)n_q * RF, &o_score));
    CK(ws_get(ctx, farm::B_OUT_T, (size_t)n_q * RF * 4, &o_t));
    CK(ws_get(ctx, farm::B_OUT_ANCHOR, (size_t)n_q * RF * 4, &o_anc));
    if (!dev) CK(ws_get(ctx, farm::B_RAW, (size_t)(emb_t + emb_c), &d_raw));
    uint8_t *d_pieces;
    CK(ws_get(ctx, farm::B_PIECES, (size_t)n_ch * sizeof(farm::Piece), &d_pieces));
    int32_t *d_rowlist;
    CK(ws_get(ctx, farm::B_SELLIST, (size_t)rows + 1, &d_rowlist));

    // ---- metadata (caller order is the planned order), select pieces
    std::vector<int32_t> meta((size_t)n_q * 8), perm((size_t)n_q);
    ctx->h_perm.assign((size_t)n_q, 0);
    ctx->h_cplan.assign((size_t)n_c, 0);
    for (int64_t q = 0; q < n_q; ++q) {
        const int32_t m = c_off[q + 1] - c_off[q];
        int32_t pr[4] = {0, 0, 0, 0};
        for (int32_t i = 0; i < m; ++i) pr[i] = c_pred[c_off[q] + i];
        int32_t *mt = meta.data() + q * 8;
        mt[farm::QM_SCENE] = scene_id;
        mt[farm::QM_CLS] = tgt_cls[q];
        mt[farm::QM_M] = m;
        mt[farm::QM_C0] = c_off[q];
        mt[farm::QM_PRED01] = pr[0] | (pr[1] << 16);
        mt[farm::QM_PRED23] = pr[2] | (pr[3] << 16);
        mt[farm::QM_R] = RF;            // (the fusion writes the kept count)
        mt[farm::QM_KLM] = Ka;
        perm[q] = (int32_t)q;
        ctx->h_perm[q] = (int32_t)q;
    }
    for (int64_t i = 0; i < n_c; ++i) ctx->h_cplan[i] = (int32_t)i;
    // rows [0, th0) of a channel take the shared-memory select, [th0, rows) the thresholded one
    const int32_t uni = (int32_t)std::min<int64_t>(farm::group_count(n, gshift), 8192);
    const bool small = n <= farm::kSelectSortAll;
    const bool t_thresh = small || uni >= Rt || n > farm::kSelectRowMax;
    const bool l_thresh = small || uni >= Rl || n > farm::kSelectRowMax;
    const int64_t th0 = t_thresh ? (l_thresh ? 0 : -1) : (l_thresh ? n_q : rows);
    if (th0 < 0) return fail(ctx, FARM_EINVAL, "unsupported scene size for a fused batch");
    std::vector<farm::Piece> pcs((size_t)n_ch);
    for (int32_t k = 0; k < n_ch; ++k) {
        farm::Piece pc{};
        pc.d32 = nullptr;
        pc.s_off = (int64_t)k * rows * ld;
        pc.tops_off = (int64_t)k * rows * gstride;
        pc.row_begin = 0;
        pc.block_begin = 0;
        pc.tblock_begin = 0;
        pc.q_row0 = 0;
        pc.t_row0 = 0;
        pc.l_row0 = 0;
        pc.tmp_off = -1;
        pc.rows = (int32_t)rows;
        pc.ntr = (int32_t)n_q;
        pc.n = (int32_t)n;
        pc.ld = (int32_t)ld;
        pc.keep_t = Rt;
        pc.keep_l = Rl;
        pc.fkeep_t = Rt;
        pc.fkeep_l = Rl;
        pc.n_obj = (int32_t)n;
        pc.R = Rt;
        pc.klm = Rl;
        pc.chunks = 1;
        pc.chunk_len = (int32_t)n;
        pc.th0 = (int32_t)th0;
        pc.gshift = gshift;
        pcs[k] = pc;
    }
    // (pageable sources: each copy has been staged when the call returns)
    CK(cudaMemcpyAsync(d_meta, meta.data(), meta.size() * 4, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(d_perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(d_pieces, pcs.data(), pcs.size() * sizeof(farm::Piece), cudaMemcpyHostToDevice, c.stream));
    if (!dev) {
        CK(cudaMemcpyAsync(d_raw, tgt_emb, (size_t)emb_t * 4, cudaMemcpyHostToDevice, c.stream));
        if (n_c > 0) CK(cudaMemcpyAsync(d_raw + emb_t, c_emb, (size_t)emb_c * 4, cudaMemcpyHostToDevice, c.stream));
    }
    const float *src_t = dev ? tgt_emb : d_raw;
    const float *src_c = dev ? c_emb : d_raw + emb_t;

    // ---- per channel: normalise its rows, FP32-accurate similarity, rank select
    int64_t off_t = 0, off_c = 0;
    for (int32_t k = 0; k < n_ch; ++k) {
        const int m0 = mark_begin(ctx, 0);
        LAUNCH(farm::launch_normalize_rows(src_t + off_t, nullptr, n_q, dims[k], dpad[k], nullptr, qhi, qlo, nullptr,
                                           c.d_err, farm::kErrBadRow, c.stream));
        if (n_c > 0)
            LAUNCH(farm::launch_normalize_rows(src_c + off_c, nullptr, n_c, dims[k], dpad[k], nullptr,
                                               qhi + (size_t)n_q * dpad[k], qlo + (size_t)n_q * dpad[k], nullptr,
                                               c.d_err, farm::kErrBadRow, c.stream));
        mark_end(ctx, m0);
        off_t += n_q * dims[k];
        off_c += n_c * dims[k];
        const int m1 = mark_begin(ctx, 1);
        LAUNCH(farm::launch_sim_tc_f16x3(qhi, qlo, dhi[k], dlo[k], d_sim + pcs[k].s_off, rows, n, dpad[k], ld,
                                         d_tops + pcs[k].tops_off, c.num_sms, c.d_err, c.stream));
        mark_end(ctx, m1);
        const int m2 = mark_begin(ctx, 2);
        int32_t *tl = d_tl + (size_t)k * n_q * Rt, *ll = d_ll + (size_t)k * n_c * Rl;
        if (th0 > 0)
            LAUNCH(farm::launch_select_rows_ex(d_sim + pcs[k].s_off, ld, n, th0, n_q, Rt, Rl, tl, nullptr, 0, Rt, ll,
                                               nullptr, 0, Rl, c.stream));
        if (th0 < rows)
            LAUNCH(farm::launch_select_thresh(d_sim, d_tops, reinterpret_cast<farm::Piece *>(d_pieces) + k, 1,
                                              rows - th0, uni, tl, nullptr, Rt, ll, nullptr, Rl, c.d_fallback,
                                              d_rowlist, c.stream));
        mark_end(ctx, m2);
    }

    // ---- fusion, then relations / composite / sort
    const int m2 = mark_begin(ctx, 2);
    farm::FuseArgs fa{};
    fa.n_q = n_q;
    fa.n_c = n_c;
    fa.n_ch = n_ch;
    for (int32_t k = 0; k < n_ch; ++k) fa.w[k] = ch[k].weight;
    fa.Rt = Rt;
    fa.Rl = Rl;
    fa.tlist = d_tl;
    fa.llist = d_ll;
    fa.S = d_sim;
    fa.rows = rows;
    fa.ld = ld;
    fa.tops = d_tops;
    fa.gstride = gstride;
    fa.gshift = gshift;
    fa.n = (int32_t)n;
    fa.cls = s.cls;
    fa.qmeta = d_meta;
    fa.p = p;
    fa.RF = RF;
    fa.out_tidx = tsel_idx;
    fa.out_tF = d_fused;
    fa.Ka = Ka;
    fa.out_lidx = lsel_idx;
    fa.err = c.d_err;
    LAUNCH(farm::launch_fuse(fa, 0, c.stream));
    if (n_c > 0) LAUNCH(farm::launch_fuse(fa, 1, c.stream));
    mark_end(ctx, m2);
    const int m3 = mark_begin(ctx, 3);
    farm::ComposeArgs ca;
    ca.n_q = n_q;
    ca.qmeta = d_meta;
    ca.tsel_idx = tsel_idx;
    ca.lsel_idx = lsel_idx;
    ca.stride_t = RF;
    ca.stride_l = Ka;
    ca.scenes = ctx->d_scenes;
    ca.p = p;
    ca.out_idx = o_idx;
    ca.out_score = o_score;
    ca.out_t = o_t;
    ca.out_anchor = o_anc;
    ca.tsel_F = d_fused;
    LAUNCH(farm::launch_compose(ca, c.stream));
    mark_end(ctx, m3);

    c.batch_gen += 1;
    c.batch_valid = true;
    c.batch_nq = n_q;
    c.batch_nc = n_c;
    c.batch_rtgt = RF;
    c.batch_klm = Ka;
    c.batch_min_n = (int32_t)std::min<int64_t>(n, 0x7fffffff);
    *batch_handle = c.batch_gen;
    return FARM_OK;
}

farm_status farm_topk(farm_ctx *ctx, uint64_t batch_handle, int32_t k, int32_t *out_idx, float *out_score,
                      float *out_pred, int32_t *out_anchor, uint32_t flags)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (!c.batch_valid || batch_handle != c.batch_gen || batch_handle == 0)
        return fail(ctx, FARM_ESTATE, "stale or unknown batch handle");
    if (k < 1 || k > c.params.k_max) return fail(ctx, FARM_EINVAL, "k must lie in [1, k_max]");
    if (c.batch_nq == 0) return FARM_OK;
    if (k > c.batch_min_n) return fail(ctx, FARM_EINVAL, "k exceeds the object count of a scene in the batch");
    if (!out_idx || !out_score) return fail(ctx, FARM_EINVAL, "out_idx and out_score must be non-null");
    CK(cudaSetDevice(c.device));
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    const int64_t n_q = c.batch_nq;
    int32_t *d_perm = static_cast<int32_t *>(c.ws.ptr[farm::B_PERM]);
    const int32_t *i_idx = static_cast<int32_t *>(c.ws.ptr[farm::B_OUT_IDX]);
    const float *i_score = static_cast<float *>(c.ws.ptr[farm::B_OUT_SCORE]);
    const float *i_t = static_cast<float *>(c.ws.ptr[farm::B_OUT_T]);
    const int32_t *i_anc = static_cast<int32_t *>(c.ws.ptr[farm::B_OUT_ANCHOR]);
    if (dev) {
        LAUNCH(farm::launch_gather_topk(n_q, k, c.batch_rtgt, d_perm, i_idx, i_score, i_t, i_anc, out_idx,
                                        out_score, out_pred, out_anchor, c.stream));
        return FARM_OK;
    }
    // device staging: idx | score | t[4] | anchor[4] per entry
    int32_t *s_idx;
    CK(ws_get(ctx, farm::B_TOPK, (size_t)n_q * k * 10, &s_idx));
    float *s_score = reinterpret_cast<float *>(s_idx + n_q * k);
    float *s_t = out_pred ? reinterpret_cast<float *>(s_idx + n_q * k * 2) : nullptr;
    int32_t *s_anc = out_anchor ? s_idx + n_q * k * 6 : nullptr;
    LAUNCH(farm::launch_gather_topk(n_q, k, c.batch_rtgt, d_perm, i_idx, i_score, i_t, i_anc, s_idx, s_score,
                                    s_t, s_anc, c.stream));
    CK(cudaMemcpyAsync(out_idx, s_idx, (size_t)n_q * k * 4, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(out_score, s_score, (size_t)n_q * k * 4, cudaMemcpyDeviceToHost, c.stream));
    if (out_pred) CK(cudaMemcpyAsync(out_pred, s_t, (size_t)n_q * k * 16, cudaMemcpyDeviceToHost, c.stream));
    if (out_anchor) CK(cudaMemcpyAsync(out_anchor, s_anc, (size_t)n_q * k * 16, cudaMemcpyDeviceToHost, c.stream));
    if (flags & FARM_ASYNC) return FARM_OK;      // valid after the next farm_sync
    return check_device_errors(ctx);
}

farm_status farm_sync(farm_ctx *ctx)
{
    if (!ctx) return FARM_EINVAL;
    CK(cudaSetDevice(ctx->c.device));
    return check_device_errors(ctx);
}

farm_status farm_memory_release(farm_ctx *ctx, int32_t scene_id)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (scene_id < 0 || scene_id >= kMaxScenes || !c.scenes[scene_id].present)
        return fail(ctx, FARM_EINVAL, "unknown scene");
    CK(cudaSetDevice(c.device));
    // queued work may still read the scene
    CK(cudaStreamSynchronize(c.stream));
    free_scene(c.scenes[scene_id]);
    CK(cudaMemsetAsync(ctx->d_scenes + scene_id, 0, sizeof(SceneDev), c.stream));
    CK(cudaStreamSynchronize(c.stream));
    c.batch_valid = false;
    c.scene_gen += 1;
    return FARM_OK;
}

farm_status farm_scene_info(farm_ctx *ctx, int32_t scene_id, int64_t *n, int32_t *dim)
{
    if (!ctx) return FARM_EINVAL;
    const Ctx &c = ctx->c;
    if (scene_id < 0 || scene_id >= kMaxScenes || !c.scenes[scene_id].present)
        return fail(ctx, FARM_EINVAL, "unknown scene");
    if (n) *n = c.scenes[scene_id].n;
    if (dim) *dim = c.scenes[scene_id].dim;
    return FARM_OK;
}

farm_status farm_similarity(farm_ctx *ctx, int32_t scene_id, int64_t n_rows, const float *emb, int32_t precision,
                            float *out, uint32_t flags)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (scene_id < 0 || scene_id >= kMaxScenes || !c.scenes[scene_id].present)
        return fail(ctx, FARM_EINVAL, "unknown scene");
    if (n_rows < 0) return fail(ctx, FARM_EINVAL, "n_rows must be >= 0");
    if (n_rows == 0) return FARM_OK;
    if (!emb || !out) return fail(ctx, FARM_EINVAL, "emb and out must be non-null");
    if (precision != FARM_PREC_FP32 && precision != FARM_PREC_FP32_SIMT && precision != FARM_PREC_BF16 &&
        precision != FARM_PREC_FP8)
        return fail(ctx, FARM_EINVAL, "unknown precision");
    CK(cudaSetDevice(c.device));
    const Scene &s = c.scenes[scene_id];
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    const float *src = emb;
    if (!dev) {
        float *raw;
        CK(ws_get(ctx, farm::B_RAW, (size_t)n_rows * s.dim, &raw));
        CK(cudaMemcpyAsync(raw, emb, (size_t)n_rows * s.dim * 4, cudaMemcpyHostToDevice, c.stream));
        src = raw;
    }
    RowOps ops;
    CK(alloc_rows(ctx, precision, n_rows, s.dim_pad, ops));
    LAUNCH(farm::launch_normalize_rows(src, nullptr, n_rows, s.dim, s.dim_pad, ops.q32, ops.qhi, ops.qlo, ops.qbf,
                                       c.d_err, farm::kErrBadRow, c.stream));
    if (precision == FARM_PREC_FP8)
        LAUNCH(farm::launch_quantize_fp8_rows(ops.q32, n_rows, s.dim_pad, ops.qf8, ops.qscale, c.stream));
    float *S = out;
    if (!dev) CK(ws_get(ctx, farm::B_SIM, (size_t)n_rows * s.n, &S));
    farm_status st = run_similarity(ctx, precision, ops, 0, n_rows, s, S, s.n);
    if (st != FARM_OK) return st;
    if (!dev) {
        CK(cudaMemcpyAsync(out, S, (size_t)n_rows * s.n * 4, cudaMemcpyDeviceToHost, c.stream));
        return check_device_errors(ctx);
    }
    return FARM_OK;
}

farm_status farm_sim_tuning(farm_ctx *ctx, int32_t *entries, int32_t cap, int32_t *count)
{
    if (!ctx) return FARM_EINVAL;
    if (cap < 0 || (cap > 0 && !entries)) return fail(ctx, FARM_EINVAL, "entries must hold cap records");
    int32_t i = 0;
    for (const auto &kv : ctx->c.tuned) {
        if (i < cap) {
            entries[4 * i + 0] = (int32_t)(kv.first / 10000 % 10) + (kv.first / 100000 % 2 ? 10 : 0) +
                                 (kv.first / 200000 % 2 ? 20 : 0);
            entries[4 * i + 1] = (int32_t)(kv.first / 100 % 100);
            entries[4 * i + 2] = (int32_t)(kv.first % 100);
            entries[4 * i + 3] = kv.second;
        }
        ++i;
    }
    if (count) *count = i;
    return FARM_OK;
}

farm_status farm_sim_variant_pin(farm_ctx *ctx, int32_t variant)
{
    if (!ctx) return FARM_EINVAL;
    if (variant < -1 || variant >= farm::kSimVariants) return fail(ctx, FARM_EINVAL, "variant must lie in [-1, 3)");
    ctx->c.pinned_variant = variant;
    return FARM_OK;
}

farm_status farm_similarity_variant(farm_ctx *ctx, int32_t scene_id, int64_t n_rows, const float *emb,
                                    int32_t precision, int32_t variant, float *out, uint32_t flags)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (scene_id < 0 || scene_id >= kMaxScenes || !c.scenes[scene_id].present)
        return fail(ctx, FARM_EINVAL, "unknown scene");
    if (n_rows < 0) return fail(ctx, FARM_EINVAL, "n_rows must be >= 0");
    if (variant < 0 || variant >= farm::kSimVariants) return fail(ctx, FARM_EINVAL, "variant must lie in [0, 3)");
    int mode;
    if (precision == FARM_PREC_FP32) mode = farm::kSimF16x3;
    else if (precision == FARM_PREC_BF16) mode = farm::kSimBf16;
    else if (precision == FARM_PREC_FP8) mode = farm::kSimFp8;
    else return fail(ctx, FARM_EINVAL, "precision must be FARM_PREC_FP32, FARM_PREC_BF16 or FARM_PREC_FP8");
    if (n_rows == 0) return FARM_OK;
    if (!emb || !out) return fail(ctx, FARM_EINVAL, "emb and out must be non-null");
    if (!farm::sim_tc_available()) return fail(ctx, FARM_EINVAL, "the tensor-core similarity path is not built");
    CK(cudaSetDevice(c.device));
    const Scene &s = c.scenes[scene_id];
    const bool dev = (flags & FARM_PTR_DEVICE) != 0;
    const float *src = emb;
    if (!dev) {
        float *raw;
        CK(ws_get(ctx, farm::B_RAW, (size_t)n_rows * s.dim, &raw));
        CK(cudaMemcpyAsync(raw, emb, (size_t)n_rows * s.dim * 4, cudaMemcpyHostToDevice, c.stream));
        src = raw;
    }
    RowOps ops;
    CK(alloc_rows(ctx, precision, n_rows, s.dim_pad, ops));
    LAUNCH(farm::launch_normalize_rows(src, nullptr, n_rows, s.dim, s.dim_pad, ops.q32, ops.qhi, ops.qlo, ops.qbf,
                                       c.d_err, farm::kErrBadRow, c.stream));
    if (precision == FARM_PREC_FP8)
        LAUNCH(farm::launch_quantize_fp8_rows(ops.q32, n_rows, s.dim_pad, ops.qf8, ops.qscale, c.stream));
    const int64_t ld = round_up(s.n, 32);
    float *S;
    CK(ws_get(ctx, farm::B_SIM, (size_t)n_rows * ld, &S));
    // one piece and its scene's tensor maps, copied from pageable host memory
    // (the copy completes before the call returns, so the host buffer is free)
    std::vector<uint8_t> blob(128 + 2 * farm::kTensorMapBytes + 64);
    uint8_t *hb = blob.data() + ((64 - (reinterpret_cast<uintptr_t>(blob.data()) & 63)) & 63);
    uint8_t *d_blob;
    CK(ws_get(ctx, farm::B_VARIANT, 128 + 2 * farm::kTensorMapBytes, &d_blob));
    bool ok;
    if (mode == farm::kSimF16x3) ok = farm::sim_tc_encode_b(mode, variant, hb + 128, s.desc_hi, s.desc_lo, s.n, s.dim_pad);
    else if (mode == farm::kSimBf16) ok = farm::sim_tc_encode_b(mode, variant, hb + 128, s.desc_bf16, nullptr, s.n, s.dim_pad);
    else ok = farm::sim_tc_encode_b(mode, variant, hb + 128, s.desc_fp8, nullptr, s.n, s.dim_pad);
    if (!ok) return fail(ctx, FARM_ECUDA, "tensor map encoding failed");
    farm::GemmPiece gp{};
    gp.q_row0 = 0;
    gp.s_off = 0;
    gp.tops_off = -1;
    gp.scale_d = mode == farm::kSimFp8 ? s.desc_scale : nullptr;
    gp.bmap = d_blob + 128;
    gp.rows = (int32_t)n_rows;
    gp.n = (int32_t)s.n;
    gp.ld = (int32_t)ld;
    gp.tile_begin = 0;
    gp.gshift = farm::group_shift_for(s.n);
    gp.col_mode = farm::kColAll;
    gp.col_stride = 0;
    gp.n_store = (int32_t)s.n;
    std::memcpy(hb, &gp, sizeof(gp));
    CK(cudaMemcpyAsync(d_blob, hb, 128 + 2 * farm::kTensorMapBytes, cudaMemcpyHostToDevice, c.stream));
    const void *q0 = mode == farm::kSimF16x3 ? (const void *)ops.qhi : (mode == farm::kSimBf16 ? (const void *)ops.qbf : (const void *)ops.qf8);
    LAUNCH(farm::launch_sim_tc_grouped(mode, variant, q0, ops.qlo, n_rows, s.dim_pad,
                                       reinterpret_cast<const farm::GemmPiece *>(d_blob), 1,
                                       farm::sim_cluster_tiles(n_rows, s.n, variant), S, nullptr,
                                       mode == farm::kSimFp8 ? ops.qscale : nullptr, c.num_sms, c.d_err, c.stream));
    if (dev) {
        CK(cudaMemcpy2DAsync(out, (size_t)s.n * 4, S, (size_t)ld * 4, (size_t)s.n * 4, (size_t)n_rows,
                             cudaMemcpyDeviceToDevice, c.stream));
        return FARM_OK;
    }
    CK(cudaMemcpy2DAsync(out, (size_t)s.n * 4, S, (size_t)ld * 4, (size_t)s.n * 4, (size_t)n_rows,
                         cudaMemcpyDeviceToHost, c.stream));
    return check_device_errors(ctx);
}

farm_status farm_candidates(farm_ctx *ctx, uint64_t batch_handle, int32_t *tgt_idx, int32_t *lm_idx,
                            int32_t *r_tgt_out, int32_t *k_lm_out)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    if (!c.batch_valid || batch_handle != c.batch_gen || batch_handle == 0)
        return fail(ctx, FARM_ESTATE, "stale or unknown batch handle");
    if (r_tgt_out) *r_tgt_out = c.batch_rtgt;
    if (k_lm_out) *k_lm_out = c.batch_klm;
    if (c.batch_nq == 0) return FARM_OK;
    CK(cudaSetDevice(c.device));
    const int64_t n_q = c.batch_nq, n_c = c.batch_nc;
    std::vector<int32_t> t((size_t)n_q * c.batch_rtgt), l((size_t)std::max<int64_t>(n_c, 1) * c.batch_klm);
    CK(cudaMemcpyAsync(t.data(), c.ws.ptr[farm::B_TSEL_IDX], t.size() * 4, cudaMemcpyDeviceToHost, c.stream));
    if (n_c > 0)
        CK(cudaMemcpyAsync(l.data(), c.ws.ptr[farm::B_LSEL_IDX], (size_t)n_c * c.batch_klm * 4,
                           cudaMemcpyDeviceToHost, c.stream));
    farm_status st = check_device_errors(ctx);
    if (st != FARM_OK) return st;
    if (tgt_idx)
        for (int64_t q = 0; q < n_q; ++q)
            std::memcpy(tgt_idx + q * c.batch_rtgt, t.data() + (size_t)ctx->h_perm[q] * c.batch_rtgt,
                        (size_t)c.batch_rtgt * 4);
    if (lm_idx)
        for (int64_t i = 0; i < n_c; ++i)
            std::memcpy(lm_idx + i * c.batch_klm, l.data() + (size_t)ctx->h_cplan[i] * c.batch_klm,
                        (size_t)c.batch_klm * 4);
    return FARM_OK;
}

farm_status farm_select_fallbacks(farm_ctx *ctx, int64_t *rows_out, int32_t reset)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    CK(cudaSetDevice(c.device));
    int32_t v = 0;
    CK(cudaMemcpyAsync(&v, c.d_fallback, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (rows_out) *rows_out = v;
    if (reset) {
        CK(cudaMemsetAsync(c.d_fallback, 0, sizeof(int32_t), c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    return FARM_OK;
}

farm_status farm_set_profiling(farm_ctx *ctx, int32_t on)
{
    if (!ctx) return FARM_EINVAL;
    ctx->c.profiling = on != 0;
    return FARM_OK;
}

farm_status farm_stage_times(farm_ctx *ctx, float *ms_out, int64_t *launches_out, int32_t reset)
{
    if (!ctx) return FARM_EINVAL;
    Ctx &c = ctx->c;
    CK(cudaSetDevice(c.device));
    CK(cudaStreamSynchronize(c.stream));
    for (auto &m : ctx->marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess && m.stage >= 0 && m.stage < FARM_N_STAGES)
            c.stage_ms[m.stage] += ms;
        ctx->pool.push_back(m.a);
        ctx->pool.push_back(m.b);
    }
    ctx->marks.clear();
    if (ms_out)
        for (int i = 0; i < FARM_N_STAGES; ++i) ms_out[i] = (float)c.stage_ms[i];
    if (launches_out) *launches_out = c.launches;
    if (reset) {
        for (int i = 0; i < FARM_N_STAGES; ++i) c.stage_ms[i] = 0.0;
        c.launches = 0;
    }
    return FARM_OK;
}

}  // extern "C"
